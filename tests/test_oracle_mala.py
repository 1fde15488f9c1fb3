"""Oracle pins for the differentiable path map and the Langevin (MALA)
strategy.

- grad log pi by forward-mode differentiation against central differences
  of the primal path map (a separate code path) on random Cornell-box paths
  of depth 10, and against the closed form on the toy integrand;
- zero gradient where f is constant (black furnace);
- MALA with a step that differs per region (tau sigma_k^2, frozen sigma_k)
  keeps the toy's closed-form region masses; dropping the proposal-density
  ratio (planted mistake) biases them.
"""
import math

import numpy as np
import pytest

from paper_2402_08273_gb300 import scenes as S

TOY = S.TOY_DEFAULT
LUM = np.array([0.2126, 0.7152, 0.0722])


def _q(rng, D):
    return rng.integers(0, 2 ** 32, D, dtype=np.uint64).astype(np.uint32)


def _shift(q, j, steps):
    out = q.copy()
    out[j] = np.uint32((int(q[j]) + steps * 256) % (1 << 32))   # u has 24 bits: one unit is 256 words
    return out


def test_gradient_matches_central_differences_cornell(oracle_mod):
    sc = oracle_mod.Scene(S.cornell_box(), use_bvh=False)
    rng = np.random.default_rng(0)
    md, D = 10, 52
    k = 16                       # h = 16 * 2^-24
    h = k / 16777216.0
    checked, worst = 0, 0.0
    for _ in range(400):
        q = _q(rng, D)
        f, g, st = sc.path_grad(q, 64, 64, md)
        f0, margin, ok, _ = sc.path_eval(q, 64, 64, md)
        np.testing.assert_allclose(f, f0, rtol=1e-12, atol=1e-14)
        if st != 1 or not ok or LUM @ f0 <= 0 or margin < 1e-3:
            continue
        fd = np.zeros(D)
        for j in range(D):
            fp = sc.path_eval(_shift(q, j, k), 64, 64, md)[0]
            fm = sc.path_eval(_shift(q, j, -k), 64, 64, md)[0]
            fd[j] = (math.log(LUM @ fp) - math.log(LUM @ fm)) / (2 * h)
        worst = max(worst, float(np.max(np.abs(fd - g)) / (np.max(np.abs(g)) + 1e-12)))
        checked += 1
    assert checked >= 60
    assert worst < 1e-4, worst


def test_gradient_toy_closed_form(oracle_mod):
    sc = oracle_mod.Scene(toy=TOY)
    rng = np.random.default_rng(1)
    p = TOY
    for _ in range(200):
        q = _q(rng, 2)
        f, g, st = sc.path_grad(q, 64, 64, 0)
        u = (q >> 8).astype(np.float64) / 16777216.0
        e = p[6] * math.exp(-((u[0] - p[7]) ** 2 + (u[1] - p[8]) ** 2) / (2 * p[9] ** 2))
        fv = p[0] + (p[1] if (p[2] <= u[0] < p[3] and p[4] <= u[1] < p[5]) else 0.0) + e
        expect = np.array([-e * (u[0] - p[7]), -e * (u[1] - p[8])]) / (p[9] ** 2 * fv)
        assert st == 1 and abs(f[0] - fv) <= 1e-12 * fv
        np.testing.assert_allclose(g, expect, rtol=1e-12, atol=1e-15)


def test_gradient_zero_where_f_is_constant(oracle_mod):
    sc = oracle_mod.Scene(S.furnace(rho=0.0, le=1.0), use_bvh=False)
    rng = np.random.default_rng(2)
    for _ in range(100):
        f, g, st = sc.path_grad(_q(rng, 17), 32, 32, 3)
        assert st == 1 and np.all(g == 0.0) and abs(LUM @ f - 1.0) < 1e-12


def _mala_toy(oracle_mod, planted, sig, epochs=200):
    ch = oracle_mod.Chains(oracle_mod.Scene(toy=TOY), n_chains=256, width=64, height=64, region_px=32,
                           max_depth=0, epoch_len=16, n_bootstrap=1 << 14, p_large=0.1, p_mala=0.6,
                           mala_tau=1e-3, mala_drift_max=0.1, gamma_max=0.0, gamma_scale=0.0,
                           debug_flags=2 if planted else 0)
    ch.init()
    ch.lam[:] = 2 * np.log(sig)
    ch.sigma[:] = np.asarray(sig, np.float32)
    ch.run_epochs(epochs)
    h = ch.hist.astype(float)
    b = S.toy_region_masses(TOY, 64, 64, 32)
    return 0.5 * float(np.abs(h / h.sum() - b / b.sum()).sum()), ch.stats()


@pytest.mark.parametrize("planted", [False, True])
def test_mala_with_regional_steps_keeps_target(oracle_mod, planted):
    tv, st = _mala_toy(oracle_mod, planted, np.array([1.0, 3.0, 0.3, 2.0]))
    assert st["mala"] > 0.5 * 256 * 200 * 16
    if planted:
        assert tv > 0.05
    else:
        assert tv < 0.015
        assert 0.3 < st["mala_accepted"] / st["mala"] < 0.9


def test_mala_needs_a_differentiable_scene(oracle_mod):
    sc = oracle_mod.Scene(S.two_rooms(2000, seed=0), use_bvh=True)   # GGX surfaces
    with pytest.raises(Exception):
        oracle_mod.Chains(sc, n_chains=16, width=32, height=32, region_px=8, max_depth=3, p_mala=0.5)


def test_mala_with_adaptation_keeps_target(oracle_mod):
    """Adaptation on (gamma as in Sec. 7.1): sigma_k, hence tau_k, keeps moving
    per region while the histogram still converges to the region masses."""
    ch = oracle_mod.Chains(oracle_mod.Scene(toy=TOY), n_chains=256, width=64, height=64, region_px=8,
                           max_depth=0, epoch_len=16, n_bootstrap=1 << 14, p_large=0.1, p_mala=0.6,
                           mala_tau=1e-3, mala_drift_max=0.1)
    ch.init()
    ch.run_epochs(300)
    h = ch.hist.astype(float)
    b = S.toy_region_masses(TOY, 64, 64, 8)
    assert np.ptp(ch.lam) > 0.5
    assert 0.5 * float(np.abs(h / h.sum() - b / b.sum()).sum()) < 0.025
