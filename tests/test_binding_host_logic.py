"""Host-side logic of the Python binding that needs no GPU: a plan refuses to launch once one
of its target maps has been freed (its device tables no longer exist), and checks its maps
again only after some map has been freed."""
import types

import pytest

from paper_2407_10344_b300 import api


def _plan_with(maps):
    plan = object.__new__(api.Plan)  # the host fields only; no library plan behind it
    plan.vmaps = maps
    plan._freed_seen = api._FREED_MAPS
    return plan


def test_plan_refuses_a_freed_target_map():
    alive = types.SimpleNamespace(h=object())
    freed = types.SimpleNamespace(h=object())
    plan = _plan_with([None, alive, freed])
    plan._maps_alive()  # nothing freed since creation
    freed.h = None      # as VoxelMap.free leaves it
    plan._maps_alive()  # the counter did not move: no re-check yet
    api._FREED_MAPS += 1
    with pytest.raises(api.GlimError, match="freed"):
        plan._maps_alive()
    other = _plan_with([None, alive])
    api._FREED_MAPS += 1
    other._maps_alive()  # its own maps are alive
    assert other._freed_seen == api._FREED_MAPS
