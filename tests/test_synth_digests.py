"""The seeded synthetic inputs are the same on every machine and in every run: their SHA-256
digests equal the ones stored in tests/golden/synth_digests.json (written by
tests/golden/make_synth_digests.py, which calls only `synth`)."""
import importlib.util
import json
import os

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def _maker():
    spec = importlib.util.spec_from_file_location("make_synth_digests",
                                                  os.path.join(HERE, "golden", "make_synth_digests.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


M = _maker()
STORED = json.load(open(os.path.join(HERE, "golden", "synth_digests.json")))


@pytest.mark.parametrize("name", sorted(M.CASES))
def test_synthetic_inputs_match_their_stored_digests(name):
    w = M.CASES[name]()
    assert M.digest(w) == STORED[name]
    assert M.digest(M.CASES[name]()) == STORED[name]  # and again in the same process
