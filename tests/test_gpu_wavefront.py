"""The wavefront form of the epoch (RMLT_TUNE_WAVEFRONT) against the chain kernel.

Both forms evaluate every path with the same functions in the same order and
draw the same Philox numbers, so their trajectories are identical: trace
records (f, a, proposal hash, flags) bit for bit, lambda after every update,
final chain states, region counts and parameters, and the statistics.  Only
the image differs by the order of the binary64 atomic splats (1e-12
relative).  The Cornell-box case is also replayed against the oracle
independently, and the launch-shape knobs must not change any result.
"""
import numpy as np
import pytest

from paper_2402_08273_gb300 import scenes as S

pytestmark = pytest.mark.gpu

# the most mutations each window may let through, measured on a GB300
PINS = {"f_bounded": 12}

WF = {"wavefront": True}
STAT_KEYS = ("mutations", "accepted", "large", "small", "early_reject", "invalid_paths", "rays",
             "stack_overflow", "epochs")


def _both(n_epochs, stride=1, wf_shape=None, tuning=None, **kw):
    from gpu_run import traced_run
    ref = traced_run(n_epochs=n_epochs, stride=stride, tuning=tuning, **kw)
    wf = traced_run(n_epochs=n_epochs, stride=stride, tuning={**(tuning or {}), **WF}, wavefront=wf_shape, **kw)
    return ref, wf


def _assert_identical(ref, wf):
    tr, tw = ref["trace"], wf["trace"]
    assert tr.shape == tw.shape
    for name in ("f", "a", "qhash", "flags"):
        assert np.array_equal(tr[name], tw[name]), f"trace field {name} differs"
    assert np.array_equal(ref["lambdas"], wf["lambdas"])
    for name in ("q", "f", "k"):
        assert np.array_equal(ref["final"][name], wf["final"][name]), f"final {name} differs"
    assert np.array_equal(ref["hist"], wf["hist"])
    for name, v in ref["region"].items():
        assert np.array_equal(v, wf["region"][name]), f"region {name} differs"
    for name in STAT_KEYS:
        assert ref["stats"][name] == wf["stats"][name], name
    np.testing.assert_allclose(wf["image_raw"], ref["image_raw"], rtol=1e-12, atol=1e-300)
    st = wf["stats"]
    assert st["wave_limit_hits"] == 0
    return st


def test_wavefront_identical_cornell_brute_force():
    ref, wf = _both(40, scene=S.cornell_box(), n_chains=200, width=64, height=64, region_px=8, max_depth=5,
                    epoch_len=16, n_bootstrap=1 << 16, seed=1, p_large=0.3)
    st = _assert_identical(ref, wf)
    assert st["waves"] > 0
    assert ref["stats"]["waves"] == 0


@pytest.mark.parametrize("node_format", ["float", "quantised"])
def test_wavefront_identical_bvh_scene(node_format):
    """Two-rooms geometry (BVH4, both node layouts), 4096 chains, depth 10,
    three epochs."""
    ref, wf = _both(3, stride=3, scene=S.two_rooms(20_000, seed=1), node_format=node_format, n_chains=4096,
                    width=128, height=96, region_px=16, max_depth=10, epoch_len=16, n_bootstrap=1 << 16,
                    p_large=0.3, seed=5)
    st = _assert_identical(ref, wf)
    assert st["node_bytes"] == (128 if node_format == "float" else 64)
    assert st["rays"] > 0 and st["stack_overflow"] == 0
    # a wave per camera ray, bounce and last shadow ray at most
    assert st["waves"] <= 3 * (16 * 11 + 2)


@pytest.mark.parametrize("target_mode", [0, 1])
def test_wavefront_identical_toy(target_mode):
    ref, wf = _both(12, toy=S.TOY_DEFAULT, n_chains=300, width=64, height=64, region_px=8, max_depth=0,
                    epoch_len=16, n_bootstrap=1 << 14, p_large=0.2, target_mode=target_mode)
    _assert_identical(ref, wf)
    assert wf["stats"]["rays"] == 0


def test_wavefront_identical_weighted_large_ahead():
    """Region-weighted target with large steps traced ahead of the epoch."""
    ref, wf = _both(8, tuning={"large_ahead": True}, scene=S.two_rooms(20_000, seed=2), n_chains=2048,
                    width=128, height=128, region_px=16, max_depth=6, epoch_len=16, n_bootstrap=1 << 15,
                    p_large=0.3, target_mode=1)
    _assert_identical(ref, wf)


def test_wavefront_identical_quadtree():
    """Quadtree partition with refinement passes between epochs."""
    ref, wf = _both(12, scene=S.two_rooms(20_000, seed=2), n_chains=2048, width=128, height=128, region_px=16,
                    max_depth=6, epoch_len=16, n_bootstrap=1 << 15, p_large=0.3, partition=1,
                    qt_max_leaves=256, qt_max_depth=6, qt_split=200, qt_refine=2048 * 32)
    _assert_identical(ref, wf)
    for a, b in zip(ref["quadtree"], wf["quadtree"]):
        assert np.array_equal(a, b)
    assert ref["R"].n_regions() > 1


@pytest.mark.parametrize("shape", [{"trace_ctas_per_sm": 1, "setup_ctas_per_sm": 1, "refill_lanes": 1},
                                   {"trace_ctas_per_sm": 3, "setup_ctas_per_sm": 0, "refill_lanes": 32},
                                   {"host_loop": True}, {"short_stack": True},
                                   {"short_stack": True, "host_loop": True}, {"leaf_batch": 1},
                                   {"leaf_batch": 32, "short_stack": True}])
def test_wavefront_launch_shape_changes_nothing(shape):
    from gpu_run import traced_run
    kw = dict(scene=S.two_rooms(5_000, seed=3), n_epochs=2, n_chains=1000, width=64, height=64, region_px=8,
              max_depth=8, epoch_len=8, n_bootstrap=1 << 14, p_large=0.3, seed=9)
    a = traced_run(tuning=WF, **kw)
    b = traced_run(tuning=WF, wavefront=shape, **kw)
    _assert_identical(a, b)


def test_wavefront_cornell_oracle_replay(oracle_mod):
    """Independent of the chain kernel: 64 Cornell chains x 2000 mutations of
    the wavefront form replayed by the oracle."""
    from gpu_run import traced_run, replay_full, check_counters
    gpu = traced_run(scene=S.cornell_box(), n_epochs=125, tuning=WF, n_chains=64, width=64, height=64,
                     region_px=8, max_depth=5, epoch_len=16, n_bootstrap=1 << 16, seed=1, p_large=0.3)
    ch, rp, adopted = replay_full(oracle_mod, gpu, oracle_mod.Scene(S.cornell_box(), use_bvh=False))
    check_counters(ch, gpu, rp, PINS, adopted, PINS.get("adopted", 0))
    assert rp.s["mutations"] == 64 * 2000


def test_wavefront_bench_size_stays_identical():
    """The bench workload's launch configuration (2^16 chains, 512^2, depth 10,
    200k-triangle BVH4) for one epoch: sampled chains traced in both forms."""
    ref, wf = _both(1, stride=97, scene=S.two_rooms(200_000, seed=0), n_chains=1 << 16, width=512,
                    height=512, region_px=16, max_depth=10, epoch_len=16, n_bootstrap=1 << 20, p_large=0.3)
    _assert_identical(ref, wf)


def test_short_stack_identical_on_deep_stacks():
    """The trace kernel's split stack (16 entries in shared memory, the rest
    in device memory) on the glossy corridor's 2M-triangle BVH4, whose rays
    use more than 16 entries: identical to the chain kernel."""
    ref, wf = _both(1, stride=61, wf_shape={"short_stack": True}, scene=S.glossy_corridor(2_000_000, seed=0),
                    n_chains=1 << 15, width=480, height=270, region_px=32, max_depth=12, epoch_len=16,
                    n_bootstrap=1 << 17, p_large=0.3)
    st = _assert_identical(ref, wf)
    assert st["stack_overflow"] == 0 and st["rays"] > 0
    assert st["node_bytes"] == 64   # 2M triangles: quantised nodes by default
