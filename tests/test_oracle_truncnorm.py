"""Oracle pins for the truncated-normal small-step kernel (the paper's kernel
family, Sec. 5.2, with angles mapped to torus offsets in (-1/2, 1/2)).

- offsets follow the truncated normal: a Kolmogorov-Smirnov test against
  scipy's truncated normal for several sigma, and symmetry;
- pointwise detailed balance of the state-dependent acceptance with an
  independent density (scipy.stats.truncnorm) on random pairs across regions
  of different sigma;
- stationarity with frozen distinct sigma_k: the toy's region histogram
  converges to its closed-form masses; dropping the density ratio (planted
  mistake) biases it.
"""
import math

import numpy as np
import pytest

from paper_2402_08273_gb300 import scenes as S

stats = pytest.importorskip("scipy.stats")
TOY = S.TOY_DEFAULT


@pytest.mark.parametrize("sigma", [0.003, 0.05, 0.3, 2.0])
def test_truncnorm_offsets_follow_the_distribution(oracle_mod, sigma):
    rng = np.random.default_rng(3)
    xs = rng.integers(0, 2 ** 32, 20000, dtype=np.uint64)
    d = np.array([oracle_mod.truncnorm_delta(int(x), sigma) for x in xs], dtype=np.float64) / 2 ** 32
    a = 0.5 / sigma
    ks = stats.kstest(d, stats.truncnorm(-a, a, loc=0.0, scale=sigma).cdf)
    assert ks.pvalue > 1e-3
    assert np.all(np.abs(d) < 0.5)
    # u and 1 - u give opposite offsets (up to the 24-bit grid's half step)
    assert oracle_mod.truncnorm_delta(1 << 31, sigma) == 0


def _tn_density(delta, sigma):
    a = 0.5 / sigma
    return np.prod(stats.truncnorm.pdf(delta, -a, a, loc=0.0, scale=sigma))


def test_truncnorm_detailed_balance_pointwise(oracle_mod):
    ch = oracle_mod.Chains(oracle_mod.Scene(toy=TOY), n_chains=16, width=64, height=64, region_px=32,
                           max_depth=0, n_bootstrap=1 << 10, kernel=1)
    sig = np.array([0.05, 0.2, 0.01, 0.1], np.float32)
    ch.sigma[:] = sig
    sc = ch.scene
    rng = np.random.default_rng(5)
    checked = 0
    for _ in range(6000):
        x = rng.integers(0, 2 ** 32, 2, dtype=np.uint64).astype(np.uint32)
        kx = ch.region_of(x)
        sx = float(sig[kx])
        a = 0.5 / sx
        delta = stats.truncnorm.rvs(-a, a, loc=0.0, scale=sx, size=2, random_state=rng)
        dq = np.rint(delta * 2 ** 32).astype(np.int64)
        y = ((x.astype(np.int64) + dq) % 2 ** 32).astype(np.uint32)
        dl = dq / 2 ** 32
        ky = ch.region_of(y)
        sy = float(sig[ky])
        fx, fy = sc.path_eval(x, 64, 64, 0)[0][0], sc.path_eval(y, 64, 64, 0)[0][0]
        a_xy = ch.accept_prob(x, y, fx, fy)
        a_yx = ch.accept_prob(y, x, fy, fx)
        lhs = fx * _tn_density(dl, sx) * a_xy
        rhs = fy * _tn_density(-dl, sy) * a_yx
        assert lhs == pytest.approx(rhs, rel=1e-9, abs=1e-300)
        checked += kx != ky
    assert checked > 300   # pairs across regions of different sigma


@pytest.mark.parametrize("planted", [False, True])
def test_truncnorm_frozen_regional_scales_keep_target(oracle_mod, planted):
    sig = np.array([0.05, 0.3, 0.02, 0.15])
    ch = oracle_mod.Chains(oracle_mod.Scene(toy=TOY), n_chains=256, width=64, height=64, region_px=32,
                           max_depth=0, epoch_len=16, n_bootstrap=1 << 14, p_large=0.1, kernel=1,
                           gamma_max=0.0, gamma_scale=0.0, debug_flags=int(planted))
    ch.init()
    ch.lam[:] = 2 * np.log(sig)
    ch.sigma[:] = sig.astype(np.float32)
    ch.run_epochs(200)
    h = ch.hist.astype(float)
    b = S.toy_region_masses(TOY, 64, 64, 32)
    tv = 0.5 * float(np.abs(h / h.sum() - b / b.sum()).sum())
    if planted:
        assert tv > 0.035
    else:
        assert tv < 0.02
