"""Write tests/golden/synth_digests.json: SHA-256 digests of the seeded synthetic inputs
(points, weights, poses, pairs) of every workload family at test sizes.

The digests pin the generators: the oracle runs, the GPU tests and the benchmark all draw
their inputs from `synth`, and a change of those inputs (a different numpy random stream,
an edited scene) shows up as a digest mismatch instead of as shifted timings or tolerances.
Run from the repository root: python tests/golden/make_synth_digests.py
"""
import hashlib
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

CASES = {
    "box_room": lambda: synth.box_room(),
    "corridor_small": lambda: synth.corridor(n_cur=3000, kf_range=(2000, 3000), n_kf=3, weights=True),
    "urban_small": lambda: synth.urban(n_submaps=400, neighbours=3, point_scale=0.02, keep=4),
    "terrain_small": lambda: synth.terrain(n_src=20_000, n_map=100_000),
}


def digest(w) -> str:
    h = hashlib.sha256()
    for p in w.points:
        h.update(np.ascontiguousarray(p, dtype=np.float32).tobytes())
    for wt in (w.weights or []):
        h.update(np.ascontiguousarray(wt, dtype=np.float32).tobytes())
    h.update(np.ascontiguousarray(w.poses, dtype=np.float64).tobytes())
    h.update(np.ascontiguousarray(w.pairs, dtype=np.int32).tobytes())
    h.update(np.ascontiguousarray(w.resolutions, dtype=np.float64).tobytes())
    return h.hexdigest()


def main():
    out = {name: digest(make()) for name, make in CASES.items()}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "synth_digests.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)
        f.write("\n")
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()
