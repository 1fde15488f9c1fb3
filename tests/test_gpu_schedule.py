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


def _mala_run(tuning, brute_force_max):
    from paper_2402_08273_gb300 import rmlt
    R = rmlt.Renderer()
    R.load_scene(S.cornell_box(), brute_force_max=brute_force_max)
    if tuning:
        R.set_tuning(**tuning)
    R.init_chains(n_chains=1000, width=64, height=64, region_px=8, max_depth=5, epoch_len=16, n_bootstrap=1 << 14,
                  p_large=0.3, p_mala=0.3, mala_tau=1e-3, mala_drift_max=0.1, seed=3)
    R.step(48)
    R.synchronize()
    out = {"final": R.read_chain_state(), "hist": R.read_region_hist(), "region": R.read_region_params(),
           "stats": R.read_stats(), "image_raw": R.read_image(normalized=False)}
    R.close()
    return out


@pytest.mark.parametrize("brute_force_max", [0, 1])   # 0: brute force (36 triangles), 1: BVH4
def test_batch_sizes_change_nothing_langevin(brute_force_max):
    """Langevin moves run in their own batches; the batch sizes around them
    must not change the chains either (the trace instrument is not available
    with the Langevin strategy, so states, counts and statistics are compared)."""
    ref = _mala_run(None, brute_force_max)
    assert ref["stats"]["mala"] > 0
    for tuning in SCHEDULES:
        other = _mala_run(tuning, brute_force_max)
        for name in ("q", "f", "k"):
            assert np.array_equal(ref["final"][name], other["final"][name]), f"final {name} differs"
        assert np.array_equal(ref["hist"], other["hist"])
        for name, v in ref["region"].items():
            assert np.array_equal(v, other["region"][name]), f"region {name} differs"
        for name in STAT_KEYS + ("mala", "mala_accepted"):
            assert ref["stats"][name] == other["stats"][name], name
        np.testing.assert_allclose(other["image_raw"], ref["image_raw"], rtol=1e-12, atol=1e-300)
