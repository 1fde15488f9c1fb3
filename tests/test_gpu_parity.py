"""GPU parity: the CUDA chain step against the CPU oracle, mutation by mutation.

Exact: proposal words (hash), large-step and reverse-kernel decisions, region
visit counts i_k and histograms h_k, lambda_k after every update (the GPU's
from its own A_k, which is the exact sum of its recorded acceptance
probabilities), final chain states.  Within tolerance: path contributions
(1e-4 of the largest channel, or the path's binary32 error bound where that
is larger; a path within a few error bounds of a decision flip is excluded
and counted), acceptance probabilities (by exactly what their inputs differ
by), accept/reject decisions (excluded only when the uniform falls between
the two acceptance probabilities), A_k, and the image.  What the windows let
through is pinned per test at the counts measured on a GB300.
"""
import numpy as np
import pytest

from paper_2402_08273_gb300 import scenes as S

pytestmark = pytest.mark.gpu

TOY = S.TOY_DEFAULT


def _replay_full(oracle_mod, gpu, scene_obj, max_adopt=2, **replay_kw):
    from gpu_run import replay_full
    return replay_full(oracle_mod, gpu, scene_obj, max_adopt, **replay_kw)


def _check_counters(ch, gpu, rp, pins=None, adopted=0, max_adopted=0):
    from gpu_run import check_counters
    check_counters(ch, gpu, rp, pins, adopted, max_adopted)


# the most mutations each window may let through, measured on a GB300
PINS = {
    "toy": {"update_excluded": 2},
    "toy_weighted": {"update_excluded": 1},
    "cornell": {"f_bounded": 59, "f_excluded": 1},
}
PINS_SAMPLED = {"two_rooms": {"f_bounded": 2}}


@pytest.mark.parametrize("n_chains,target_mode", [(200, 0), (64, 1)])
def test_toy_integrand_parity(oracle_mod, n_chains, target_mode):
    from gpu_run import traced_run
    gpu = traced_run(toy=TOY, n_epochs=40, n_chains=n_chains, width=64, height=64, region_px=8,
                     max_depth=0, epoch_len=16, n_bootstrap=1 << 14, p_large=0.2,
                     target_mode=target_mode)
    ch, rp, adopted = _replay_full(oracle_mod, gpu, oracle_mod.Scene(toy=TOY), max_adopt=0)
    assert rp.s["f_excluded"] == 0
    _check_counters(ch, gpu, rp, PINS["toy"] if target_mode == 0 else PINS["toy_weighted"])
    if target_mode:
        assert np.array_equal(ch.weight, gpu["region"]["w"]), "w_k differs"
    np.testing.assert_allclose(gpu["image"], ch.image(), rtol=1e-5, atol=1e-9)
    assert abs(gpu["stats"]["bhat"] - ch.bhat) < 1e-5 * ch.bhat


def test_cornell_box_full_trajectory(oracle_mod):
    """Cornell box, 64 chains, 1e4 mutations each: every mutation replayed."""
    from gpu_run import traced_run
    gpu = traced_run(scene=S.cornell_box(), n_epochs=625, n_chains=64, width=64, height=64,
                     region_px=8, max_depth=5, epoch_len=16, n_bootstrap=1 << 16, seed=1,
                     p_large=0.3)
    ch, rp, adopted = _replay_full(oracle_mod, gpu, oracle_mod.Scene(S.cornell_box(), use_bvh=False))
    print("cornell replay:", rp.summary(), "adopted", adopted)
    _check_counters(ch, gpu, rp, PINS["cornell"], adopted, 0)
    n = rp.s["mutations"]
    assert n == 64 * 10000
    img_o = ch.image()
    rel = np.abs(gpu["image"] - img_o) / (np.abs(img_o) + 1e-3 * img_o.mean())
    assert rel.max() < 1e-3


def test_furnace_closed_form_gpu():
    from paper_2402_08273_gb300 import rmlt
    R = rmlt.Renderer()
    R.load_scene(S.furnace(rho=0.0, le=1.0))
    R.init_chains(n_chains=256, width=32, height=32, region_px=8, max_depth=3, n_bootstrap=1 << 14)
    R.step(64)
    st = R.read_stats()
    assert st["bhat"] == 1.0
    img = R.read_image()
    assert abs(img.mean() - 1.0) < 1e-6
    assert st["accepted"] + st["early_reject"] == st["mutations"] * 256
    R.close()
    R = rmlt.Renderer()
    R.load_scene(S.furnace(rho=0.5, le=1.0))
    R.init_chains(n_chains=4096, width=32, height=32, region_px=8, max_depth=3, n_bootstrap=1 << 20)
    R.step(64)
    st = R.read_stats()
    assert abs(st["bhat"] - 1.875) < 0.01 * 1.875
    img = R.read_image()
    assert abs(img.mean() - st["bhat"]) < 1e-5 * st["bhat"]


def test_two_rooms_full_size_sampled(oracle_mod):
    """Full size (512^2, 16-px regions, depth 10, 2^16 chains, 200k-triangle
    SAH BVH): 128 sampled chains replayed over two epochs from their GPU
    states; the oracle recomputes f of each state with its own BVH."""
    from oracle.replay import Replay
    from gpu_run import traced_run, oracle_params
    scene = S.two_rooms(200_000, seed=0)
    stride = 512
    gpu = traced_run(scene=scene, n_epochs=2, stride=stride, n_chains=1 << 16, width=512, height=512,
                     region_px=16, max_depth=10, epoch_len=16, n_bootstrap=1 << 20, p_large=0.3)
    p = gpu["params"]
    sc = oracle_mod.Scene(scene, use_bvh=True)
    ch = oracle_mod.Chains(sc, **oracle_params(p))
    ch.init_tables()
    traced = np.arange(0, p["n_chains"], stride)
    q0 = gpu["init"]["q"]
    for c in traced:
        ch.set_state(int(c), q0[:, c])
    rp = Replay(ch, gpu["trace"], gpu["lambdas"], stride=stride, init_f=gpu["init"]["f"])
    rp.run_sampled(2, traced)
    print("two rooms sampled replay:", rp.summary())
    assert rp.ok(), rp.summary()
    assert rp.s["mutations"] == len(traced) * 32
    for key, n in rp.counts().items():
        assert n <= PINS_SAMPLED["two_rooms"].get(key, 0), (key, n)
    st = gpu["stats"]
    assert st["stack_overflow"] == 0
    assert st["rays"] > 0
