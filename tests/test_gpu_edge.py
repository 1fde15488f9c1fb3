"""GPU edge cases and variants, each replayed against the oracle or checked
against a property that holds at any size."""
import numpy as np
import pytest

from paper_2402_08273_gb300 import scenes as S

pytestmark = pytest.mark.gpu

TOY = S.TOY_DEFAULT


# the most mutations each window may let through, per test, measured on a GB300
PINS = {"depth12": {"f_bounded": 1}, "global": {"f_bounded": 3}, "fixed": {"f_bounded": 1},
        "weighted": {"f_bounded": 8}}


def _full(oracle_mod, scene=None, toy=None, use_bvh=False, n_epochs=8, bvh_width=0, pin=None, **params):
    from gpu_run import traced_run, replay_full, check_counters
    gpu = traced_run(scene=scene, toy=toy, n_epochs=n_epochs, bvh_width=bvh_width, **params)
    osc = oracle_mod.Scene(toy=toy) if toy is not None else oracle_mod.Scene(scene, use_bvh=use_bvh)
    ch, rp, adopted = replay_full(oracle_mod, gpu, osc)
    pins = PINS.get(pin, {})
    check_counters(ch, gpu, rp, pins, adopted, pins.get("adopted", 0))
    return gpu, ch, rp


def test_single_chain(oracle_mod):
    _full(oracle_mod, scene=S.cornell_box(), n_epochs=30, n_chains=1, epoch_len=8, n_bootstrap=4096, pin="single")


def test_max_depth_all_dimensions(oracle_mod):
    """depth 12: D = 62 primary-sample dimensions, the largest supported"""
    gpu, ch, rp = _full(oracle_mod, scene=S.cornell_box(), n_epochs=6, n_chains=40, max_depth=12,
                        n_bootstrap=1 << 12, pin="depth12")
    assert gpu["init"]["q"].shape[0] == 62


def test_ragged_regions_and_image(oracle_mod):
    """W, H not multiples of the region size; partial last row and column"""
    gpu, ch, rp = _full(oracle_mod, scene=S.cornell_box(), n_epochs=10, n_chains=96, width=100,
                        height=60, region_px=16, n_bootstrap=1 << 12, pin="ragged")
    assert ch.m == 7 * 4


def test_global_variant_one_region(oracle_mod):
    _full(oracle_mod, scene=S.cornell_box(), n_epochs=10, n_chains=64, region_px=64, n_bootstrap=1 << 12,
          pin="global")


def test_fixed_variant_no_adaptation(oracle_mod):
    gpu, ch, rp = _full(oracle_mod, scene=S.cornell_box(), n_epochs=10, n_chains=64, gamma_max=0.0,
                        gamma_scale=0.0, n_bootstrap=1 << 12, pin="fixed")
    assert np.all(gpu["region"]["lambda"] == 0.0)
    assert gpu["stats"]["early_reject"] == 0


def test_weighted_target_cornell(oracle_mod):
    gpu, ch, rp = _full(oracle_mod, scene=S.cornell_box(), n_epochs=20, n_chains=128, target_mode=1,
                        n_bootstrap=1 << 13, pin="weighted")
    assert np.array_equal(ch.weight, gpu["region"]["w"])


@pytest.mark.parametrize("bvh_width,node_format", [(4, "float"), (4, "quantised"), (2, "auto")])
def test_bvh_scene_full_trajectory(oracle_mod, bvh_width, node_format):
    """A 20k-triangle two-rooms scene through the BVH path (BVH4 with binary32
    and with quantised bounds, BVH2), every mutation replayed (the oracle uses
    its own median-split BVH)."""
    gpu, ch, rp = _full(oracle_mod, scene=S.two_rooms(20_000, seed=4), use_bvh=True, n_epochs=6,
                        bvh_width=bvh_width, node_format=node_format, n_chains=64, width=128, height=128,
                        region_px=16, max_depth=8, n_bootstrap=1 << 12, pin=f"bvh{bvh_width}")
    assert gpu["stats"]["stack_overflow"] == 0


def test_step_zero_and_call_order():
    from paper_2402_08273_gb300 import rmlt
    R = rmlt.Renderer()
    with pytest.raises(rmlt.RmltError) as e:
        R.step(1)
    assert e.value.status == -5
    R.load_scene(S.cornell_box())
    with pytest.raises(rmlt.RmltError) as e:
        R.read_region_hist()
    assert e.value.status == -5
    R.init_chains(n_chains=32, n_bootstrap=1 << 10)
    q0 = R.read_chain_state()["q"].copy()
    R.step(0)
    assert R.read_stats()["mutations"] == 0
    assert np.array_equal(R.read_chain_state()["q"], q0)
    R.step(1)   # rounded up to one epoch
    assert R.read_stats()["mutations"] == 16


@pytest.mark.parametrize("bad", [dict(n_chains=0), dict(width=0), dict(max_depth=13), dict(s1=0.1, s2=0.05),
                                 dict(p_large=1.5), dict(lambda_max=10.0), dict(n_bootstrap=8, n_chains=16),
                                 dict(alpha_star=1.0), dict(target_mode=3)])
def test_invalid_parameters_rejected(bad):
    from paper_2402_08273_gb300 import rmlt
    R = rmlt.Renderer()
    R.load_scene(S.cornell_box())
    with pytest.raises(rmlt.RmltError) as e:
        R.init_chains(**bad)
    assert e.value.status == -1


def test_invalid_scene_rejected():
    from paper_2402_08273_gb300 import rmlt
    R = rmlt.Renderer()
    sc = S.cornell_box()
    bad = dict(sc)
    bad["tris"] = sc["tris"].copy()
    bad["tris"][3, 1] = 10_000
    with pytest.raises(rmlt.RmltError) as e:
        R.load_scene(bad)
    assert e.value.status == -2
    bad = dict(sc)
    bad["verts"] = sc["verts"].copy()
    bad["verts"][0, 0] = np.nan
    with pytest.raises(rmlt.RmltError) as e:
        R.load_scene(bad)
    assert e.value.status == -2


def _run(scene, steps, **params):
    from paper_2402_08273_gb300 import rmlt
    R = rmlt.Renderer()
    R.load_scene(scene)
    R.init_chains(**params)
    for n in steps:
        R.step(n)
    return R


def test_determinism_and_checkpoint_resume(tmp_path):
    """Philox streams make runs reproducible; a checkpoint resumed and run on
    equals the uninterrupted run (integers exact, image to rounding)."""
    sc = S.two_rooms(20_000, seed=5)
    params = dict(n_chains=512, width=96, height=96, region_px=16, max_depth=6, n_bootstrap=1 << 12)
    A = _run(sc, [80, 80], **params)
    B = _run(sc, [80], **params)
    ck = tmp_path / "c.ckpt"
    B.save(ck)
    B.close()
    C = _run(sc, [], **params)
    C.restore(ck)
    C.step(80)
    for X in (C,):
        assert np.array_equal(A.read_chain_state()["q"], X.read_chain_state()["q"])
        assert np.array_equal(A.read_region_hist(), X.read_region_hist())
        ra, rx = A.read_region_params(), X.read_region_params()
        for k in ("lambda", "n", "i", "A"):
            assert np.array_equal(ra[k], rx[k]), k
        np.testing.assert_allclose(A.read_image(), X.read_image(), rtol=1e-12, atol=1e-300)
        assert A.read_stats()["accepted"] == X.read_stats()["accepted"]


def test_corridor_full_size_sampled(oracle_mod):
    """1920x1080, 32-px regions (60 x 34, partial last row), depth 12, 2^20
    chains, 2M-triangle glossy corridor: 64 sampled chains replayed over one
    epoch from their GPU states."""
    from oracle.replay import Replay
    from gpu_run import traced_run, oracle_params
    scene = S.glossy_corridor(2_000_000, seed=0)
    stride = 1 << 14
    gpu = traced_run(scene=scene, n_epochs=1, stride=stride, n_chains=1 << 20, width=1920, height=1080,
                     region_px=32, max_depth=12, epoch_len=16, n_bootstrap=1 << 21, p_large=0.3)
    p = gpu["params"]
    ch = oracle_mod.Chains(oracle_mod.Scene(scene, use_bvh=True), **oracle_params(p))
    ch.init_tables()
    traced = np.arange(0, p["n_chains"], stride)
    for c in traced:
        ch.set_state(int(c), gpu["init"]["q"][:, c])
    rp = Replay(ch, gpu["trace"], gpu["lambdas"], stride=stride, init_f=gpu["init"]["f"])
    rp.run_sampled(1, traced)
    print("corridor sampled replay:", rp.summary())
    assert rp.ok(), rp.summary()
    for key, n in rp.counts().items():
        assert n <= PINS.get("corridor_sampled", {}).get(key, 0), (key, n)
    # the corridor is lit: light reaches the chains through the slit
    assert np.count_nonzero(rp.f.sum(axis=-1)) > 0
    assert rp.s["mutations"] == len(traced) * 16
    assert gpu["stats"]["stack_overflow"] == 0
    assert ch.m == 60 * 34
