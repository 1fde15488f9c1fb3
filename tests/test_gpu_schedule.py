"""The chain kernel's scheduling changes speed only, never results.

A warp's lanes traverse, shade and finish their mutations in batches whose
sizes are tuning knobs (`batch_shade`, `batch_setup`, the adaptive-batch
flag), and lanes whose ray waits at a leaf test it in leaf turns together
with other lanes.  None of this may change a chain's trajectory: every lane
evaluates its own path with the same arithmetic in the same order and draws
the same Philox numbers.  Traces, lambdas, final states, region counts and
parameters and the statistics are compared bit for bit across extreme
settings, for both BVH layouts and for the 4-D partition; the raw image only
to the order of its binary64 atomic splats.
"""
import numpy as np
import pytest

from paper_2402_08273_gb300 import scenes as S

pytestmark = pytest.mark.gpu

STAT_KEYS = ("mutations", "accepted", "large", "small", "early_reject", "invalid_paths", "rays",
             "stack_overflow", "epochs")
SCHEDULES = (
    {"batch_shade": 1, "batch_setup": 1},
    {"batch_shade": 32, "batch_setup": 32},
    {"batch_shade": 5, "batch_setup": 3, "adaptive_batch": True},
)


def _kw(**extra):
    # 1500 chains: the last 64-thread block of the epoch kernel is ragged
    kw = dict(scene=S.two_rooms(20_000, seed=4), n_epochs=2, n_chains=1500, width=96, height=64, region_px=8,
              max_depth=10, epoch_len=16, n_bootstrap=1 << 14, p_large=0.3, seed=11)
    kw.update(extra)
    return kw


def _assert_identical(ref, other):
    for name in ("f", "a", "qhash", "flags"):
        assert np.array_equal(ref["trace"][name], other["trace"][name]), f"trace field {name} differs"
    assert np.array_equal(ref["lambdas"], other["lambdas"])
    for name in ("q", "f", "k"):
        assert np.array_equal(ref["final"][name], other["final"][name]), f"final {name} differs"
    assert np.array_equal(ref["hist"], other["hist"])
    for name, v in ref["region"].items():
        assert np.array_equal(v, other["region"][name]), f"region {name} differs"
    for name in STAT_KEYS:
        assert ref["stats"][name] == other["stats"][name], name
    np.testing.assert_allclose(other["image_raw"], ref["image_raw"], rtol=1e-12, atol=1e-300)


@pytest.mark.parametrize("bvh_width", [2, 4])
def test_batch_sizes_change_nothing(bvh_width):
    from gpu_run import traced_run
    ref = traced_run(bvh_width=bvh_width, **_kw())
    assert ref["stats"]["rays"] > 0 and ref["stats"]["stack_overflow"] == 0
    for tuning in SCHEDULES:
        _assert_identical(ref, traced_run(bvh_width=bvh_width, tuning=tuning, **_kw()))


def test_batch_sizes_change_nothing_4d_partition():
    from gpu_run import traced_run
    ref = traced_run(bvh_width=4, **_kw(dir_cells=2))
    assert ref["R"].n_regions() == 4 * (96 // 8) * (64 // 8)
    for tuning in SCHEDULES:
        _assert_identical(ref, traced_run(bvh_width=4, tuning=tuning, **_kw(dir_cells=2)))
