"""The truncated-normal small-step kernel (RMLT_KERNEL_TRUNCNORM) on the GPU.

Its offsets come from binary32 erfinv, so they are not bit-identical to the
oracle's binary64 ones.  The oracle replays every mutation with the GPU's
recorded proposal words, after checking each offset against its own within
the first-order bound of that rounding, and compares the path, the
acceptance probability with the kernel's density ratio, the decision and the
region tables.  Beside that, the kernel is checked through what it must
preserve: with adaptation the toy's region histogram converges to the
closed-form region masses, the Cornell box renders the image the Kelemen
kernel renders, and the wavefront form reproduces the chain kernel bit for
bit.
"""
import numpy as np
import pytest

from paper_2402_08273_gb300 import scenes as S

pytestmark = pytest.mark.gpu
LUM = np.array([0.2126, 0.7152, 0.0722])


def _renderer(scene=None, toy=None, **params):
    from paper_2402_08273_gb300 import rmlt
    R = rmlt.Renderer()
    if toy is not None:
        R.load_toy_integrand(toy)
    else:
        R.load_scene(scene)
    R.init_chains(**params)
    return R


def test_truncnorm_toy_keeps_region_masses():
    R = _renderer(toy=S.TOY_DEFAULT, n_chains=256, width=64, height=64, region_px=8, max_depth=0,
                  n_bootstrap=1 << 14, p_large=0.1, kernel=1, lambda_init=2 * np.log(0.1))
    R.step(300 * 16)
    h = R.read_region_hist().astype(float)
    b = S.toy_region_masses(S.TOY_DEFAULT, 64, 64, 8)
    lam = R.read_region_params()["lambda"]
    assert np.ptp(lam) > 0.5
    assert 0.5 * np.abs(h / h.sum() - b / b.sum()).sum() < 0.025
    st = R.read_stats()
    assert st["early_reject"] == 0 and st["invalid_paths"] == 0


def test_truncnorm_cornell_matches_kelemen_image():
    kw = dict(n_chains=4096, width=64, height=64, region_px=8, max_depth=6, n_bootstrap=1 << 16, p_large=0.3)
    A = _renderer(S.cornell_box(), **kw)
    B = _renderer(S.cornell_box(), kernel=1, lambda_init=2 * np.log(0.05), **kw)
    A.step(512)
    B.step(512)
    la, lb = A.read_image() @ LUM, B.read_image() @ LUM
    ra = la.reshape(8, 8, 8, 8).sum(axis=(1, 3))
    rb = lb.reshape(8, 8, 8, 8).sum(axis=(1, 3))
    assert 0.5 * np.abs(ra / ra.sum() - rb / rb.sum()).sum() < 0.03
    acc = B.read_stats()["accepted"] / (4096 * 512)
    assert 0.1 < acc < 0.95


def test_truncnorm_wavefront_identical():
    from gpu_run import traced_run
    kw = dict(scene=S.two_rooms(8000, seed=4), n_epochs=3, n_chains=1500, width=96, height=64, region_px=16,
              max_depth=6, epoch_len=16, n_bootstrap=1 << 14, p_large=0.3, kernel=1, lambda_init=2 * np.log(0.05))
    a = traced_run(**kw)
    b = traced_run(tuning={"wavefront": True}, **kw)
    for name in ("f", "a", "qhash", "flags"):
        assert np.array_equal(a["trace"][name], b["trace"][name]), name
    assert np.array_equal(a["final"]["q"], b["final"]["q"])
    assert np.array_equal(a["lambdas"], b["lambdas"])


def test_truncnorm_parameter_checks():
    from paper_2402_08273_gb300 import rmlt
    R = rmlt.Renderer()
    R.load_toy_integrand(S.TOY_DEFAULT)
    with pytest.raises(rmlt.RmltError):
        R.init_chains(n_chains=64, max_depth=0, kernel=1, lambda_max=3.0)   # above 2 ln 4
    with pytest.raises(rmlt.RmltError):
        R.init_chains(n_chains=64, max_depth=0, kernel=2)


# the most mutations each window may let through, measured on a GB300
PINS = {"toy": {}, "cornell": {"f_bounded": 2}}


@pytest.mark.parametrize("case", ["toy", "cornell"])
def test_truncnorm_oracle_replay(oracle_mod, case):
    from gpu_run import check_counters, replay_full, traced_run
    if case == "toy":
        gpu = traced_run(toy=S.TOY_DEFAULT, words=True, n_epochs=30, n_chains=128, width=64, height=64, region_px=8,
                         max_depth=0, n_bootstrap=1 << 13, p_large=0.1, kernel=1, lambda_init=2 * np.log(0.1))
        osc = oracle_mod.Scene(toy=S.TOY_DEFAULT)
    else:
        gpu = traced_run(scene=S.cornell_box(), words=True, n_epochs=12, n_chains=64, width=64, height=64,
                         region_px=8, max_depth=5, n_bootstrap=1 << 13, kernel=1, lambda_init=2 * np.log(0.05))
        osc = oracle_mod.Scene(S.cornell_box(), use_bvh=False)
    ch, rp, adopted = replay_full(oracle_mod, gpu, osc)
    print("truncnorm replay:", rp.summary())
    check_counters(ch, gpu, rp, PINS[case], adopted, 0)
    assert rp.s["proposal_adopted"] > 0 and rp.s["proposal_mismatch"] == 0
    # adaptation moved the regions' scales apart, so the density ratio mattered
    assert np.ptp(gpu["region"]["lambda"]) > 0
