"""Pins of the CPU oracle against facts the paper and the mathematics fix.

Each test ties one part of the oracle to something other than the oracle:
brute force, a closed form, an analytic density, a special case that reduces
to the sequential algorithm printed in the paper (Alg. 1), or an invariant the
paper proves (App. B).  A negative control plants a mistake in the oracle
(through its test-only debug flag) and checks that the pin notices.
"""
import math

import numpy as np
import pytest

from paper_2402_08273_gb300 import scenes as S

TOY = S.TOY_DEFAULT


# --------------------------------------------------------------------------
# geometry: BVH closest hit / any hit == brute force
# --------------------------------------------------------------------------
def test_bvh_matches_brute_force(oracle_mod):
    scene = S.two_rooms(n_tris=20_000, seed=3)
    sc = oracle_mod.Scene(scene, use_bvh=True)
    rng = np.random.default_rng(0)
    lo = scene["verts"].min(0).astype(np.float64)
    hi = scene["verts"].max(0).astype(np.float64)
    n_hit = 0
    for _ in range(600):
        o = lo + (hi - lo) * rng.uniform(0.02, 0.98, 3)
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        h1, t1, i1, m1 = sc.closest_hit(o, d, margin=True)
        h2, t2, i2, _ = sc.closest_hit(o, d, brute=True)
        assert h1 == h2
        if h1:
            n_hit += 1
            assert abs(t1 - t2) <= 1e-12 * max(1.0, t2)
            if i1 != i2:  # only a shared edge or a coplanar tie may pick another triangle
                assert m1 < 1e-6
        tmax = rng.uniform(0.1, 5.0)
        assert sc.any_hit(o, d, 0.0, tmax) == sc.any_hit(o, d, 0.0, tmax, brute=True)
    assert n_hit > 500


def test_closest_hit_closed_form(oracle_mod):
    sc = oracle_mod.Scene(S.cornell_box(), use_bvh=False)
    # straight into the back wall z = 1 through the open face
    hit, t, tri, _ = sc.closest_hit([0.5, 0.8, -1.0], [0.0, 0.0, 1.0])
    assert hit and abs(t - 2.0) < 1e-15
    # straight down onto the floor from above the short box's footprint gap
    hit, t, tri, _ = sc.closest_hit([0.1, 0.9, 0.1], [0.0, -1.0, 0.0])
    assert hit and abs(t - 0.9) < 1e-15
    # onto the top of the tall box (y = 0.6, stored in binary32)
    hit, t, tri, _ = sc.closest_hit([0.7, 0.95, 0.7], [0.0, -1.0, 0.0])
    assert hit and abs(t - (0.95 - float(np.float32(0.6)))) < 1e-15
    # out through the open front: miss
    hit, *_ = sc.closest_hit([0.5, 0.5, 0.5], [0.0, 0.0, -1.0])
    assert not hit


# --------------------------------------------------------------------------
# light transport: white furnace closed form
# --------------------------------------------------------------------------
@pytest.mark.parametrize("rho,depth", [(0.0, 3), (0.5, 1), (0.5, 3), (0.8, 4)])
def test_furnace_path_expectation(oracle_mod, rho, depth):
    """Closed cube, every face Lambertian rho emitting Le = 1: the expected
    path contribution at every pixel is sum_{i=0..d} rho^i (emission seen
    directly plus NEE at each of the d interactions, throughput rho^b at
    interaction b).  Plain Monte Carlo of the path map over uniform u."""
    sc = oracle_mod.Scene(S.furnace(rho=rho, le=1.0), use_bvh=False)
    rng = np.random.default_rng(5)
    D = 2 + 5 * depth
    n = 1 << 15
    qs = rng.integers(0, 2 ** 32, (n, D), dtype=np.uint64).astype(np.uint32)
    f = np.array([sc.path_eval(q, 16, 16, depth)[0] for q in qs])
    expect = sum(rho ** i for i in range(depth + 1))
    assert np.array_equal(f[:, 0], f[:, 1]) and np.array_equal(f[:, 1], f[:, 2])
    if rho == 0.0:
        assert np.all(f == 1.0)
    else:
        mean, sd = f[:, 0].mean(), f[:, 0].std() / np.sqrt(n)
        assert abs(mean - expect) < 4.5 * sd, (mean, expect, sd)


@pytest.mark.parametrize("rho", [0.0, 0.5])
def test_furnace_mlt_image(oracle_mod, rho):
    """Grey furnace: f / pi is the same constant for every path, so the MLT
    estimate's screen mean equals the bootstrap normaliser b exactly, and the
    channels agree.  With rho = 0 the target is constant: b = Le exactly and
    every proposal the reverse kernel allows is accepted."""
    sc = oracle_mod.Scene(S.furnace(rho=rho, le=1.0), use_bvh=False)
    ch = oracle_mod.Chains(sc, n_chains=64, width=16, height=16, region_px=4, max_depth=3,
                           epoch_len=16, n_bootstrap=1 << 12)
    ch.init()
    ch.run_epochs(30)
    img = ch.image()
    lum = 0.2126 * img[..., 0] + 0.7152 * img[..., 1] + 0.0722 * img[..., 2]
    assert abs(lum.mean() - ch.bhat) < 1e-12 * ch.bhat
    assert np.allclose(img[..., 0], img[..., 1], rtol=1e-14) and np.allclose(img[..., 1], img[..., 2], rtol=1e-14)
    if rho == 0.0:
        assert ch.bhat == 1.0
        st = ch.stats()
        assert st["accepted"] + st["early_reject"] == st["mutations"]


# --------------------------------------------------------------------------
# adaptation: closed-form lambda trajectory on a constant target
# --------------------------------------------------------------------------
def test_lambda_trajectory_closed_form(oracle_mod):
    """Constant target (rho = 0 furnace) and one region (Global variant):
    every proposal has a = 1, so alpha_hat = 1 > alpha* at every update and
    eq. update_lambda with eq. step_size_n gives
    lambda_n = min(lambda_max, lambda_init + sum_{j=1..n} min(g_max, g_scale j^-1/2))."""
    sc = oracle_mod.Scene(S.furnace(rho=0.0, le=2.0), use_bvh=False)
    ch = oracle_mod.Chains(sc, n_chains=8, width=16, height=16, region_px=16, max_depth=2,
                           epoch_len=8, n_bootstrap=1 << 10, lambda_init=-8.0, gamma_max=1.0,
                           gamma_scale=5.0)
    ch.init()
    lam_max = ch.params.lambda_max
    expect = -8.0
    for n in range(1, 60):
        ch.run_epochs(1)
        expect = min(lam_max, expect + min(1.0, 5.0 / math.sqrt(n)))
        assert ch.lam[0] == pytest.approx(expect, abs=1e-12)
        assert ch.n_updates[0] == n + 1
    assert ch.lam[0] == lam_max
    st = ch.stats()
    assert st["accepted"] == st["mutations"]


def test_sequential_alg1_special_case(oracle_mod):
    """One chain and one mutation per epoch reduce the epoch-parallel update to
    the sequential Algorithm 1 (with the i_k >= L reading).  The test restates
    Algorithm 1's acceptance statistics, region update and state update in its
    own code, driven by the observed proposals, and compares lambda_k, n_k,
    i_k after every mutation."""
    sc = oracle_mod.Scene(toy=TOY)
    L = 10
    ch = oracle_mod.Chains(sc, n_chains=1, width=64, height=64, region_px=16, max_depth=0,
                           epoch_len=1, L=L, n_bootstrap=1 << 10, p_large=0.2, lambda_init=1.0)
    ch.init()
    m = ch.m
    lam = np.full(m, 1.0)
    nk = np.ones(m, np.int64)
    ik = np.zeros(m, np.int64)
    Ak = np.zeros(m)
    state = {"x": ch.q[0].copy()}
    seen = []

    def hook(user, chain, mut, qy, D, large, early, dec, ferr, xi, fy, a, acc):
        y = np.ctypeslib.as_array(qy, (D,)).copy()
        seen.append((bool(large), float(a[0]), bool(acc[0]), y))

    ch.set_hooks(hook, None)
    lmax = ch.params.lambda_max
    for step in range(3000):
        seen.clear()
        ch.run_epochs(1)
        large, a, acc, y = seen[0]
        k = ch.region_of(state["x"])
        if not large:                      # Alg. 1, acceptance statistics (small steps)
            Ak[k] += a
            ik[k] += 1
            if ik[k] >= L:                 # Alg. 1, region update
                ahat = Ak[k] / ik[k]
                g = min(1.0, 5.0 / math.sqrt(nk[k]))
                lam[k] = min(lmax, max(-30.0, lam[k] + g * np.sign(ahat - 0.5)))
                ik[k] = 0
                Ak[k] = 0.0
                nk[k] += 1
        if acc:                            # Alg. 1, state update
            state["x"] = y
        assert np.array_equal(ch.q[0], state["x"])
        np.testing.assert_allclose(ch.lam, lam, rtol=0, atol=1e-12)
        assert np.array_equal(ch.n_updates, nk)
        assert np.array_equal(ch.visits.astype(np.int64), ik)
    assert nk.max() > 5


# --------------------------------------------------------------------------
# stationarity: region histogram -> region mass b_k (App. B); weighted mode
# --------------------------------------------------------------------------
def _toy_chains(oracle_mod, region_px, **kw):
    sc = oracle_mod.Scene(toy=TOY)
    args = dict(n_chains=256, width=64, height=64, region_px=region_px, max_depth=0,
                epoch_len=16, n_bootstrap=1 << 14, p_large=0.1)
    args.update(kw)
    ch = oracle_mod.Chains(sc, **args)
    ch.init()
    return ch


def _tv(p, q):
    return 0.5 * float(np.abs(p - q).sum())


@pytest.mark.parametrize("planted", [False, True])
def test_frozen_regional_scales_keep_target(oracle_mod, planted):
    """Distinct frozen sigma_k per region: the state-dependent kernel with the
    reverse-kernel factor keeps pi stationary, so h_k / N -> b_k / b with the
    closed-form masses b_k.  Dropping the factor (planted mistake) biases it."""
    sig = np.array([1.0, 8.0, 0.3, 3.0])
    ch = _toy_chains(oracle_mod, 32, gamma_max=0.0, gamma_scale=0.0, debug_flags=int(planted))
    ch.lam[:] = 2 * np.log(sig)
    ch.sigma[:] = sig.astype(np.float32)
    ch.run_epochs(200)
    h = ch.hist.astype(float)
    b = S.toy_region_masses(TOY, 64, 64, 32)
    tv = _tv(h / h.sum(), b / b.sum())
    if planted:
        assert tv > 0.035
    else:
        assert tv < 0.025


def test_adaptive_histogram_matches_region_mass(oracle_mod):
    ch = _toy_chains(oracle_mod, 8)
    ch.run_epochs(200)
    h = ch.hist.astype(float)
    b = S.toy_region_masses(TOY, 64, 64, 8)
    assert _tv(h / h.sum(), b / b.sum()) < 0.025
    assert h.sum() == 256 * 200 * 16
    # f / pi has unit luminance, so the screen mean of the image is the
    # bootstrap normaliser (pinned against b in test_bootstrap_normaliser)
    img = ch.image()
    lum = 0.2126 * img[..., 0] + 0.7152 * img[..., 1] + 0.0722 * img[..., 2]
    assert abs(lum.mean() - ch.bhat) < 1e-12 * ch.bhat
    # per-region share of the image equals the region share of visits
    share = np.array([lum[j * 8:(j + 1) * 8, i * 8:(i + 1) * 8].sum()
                      for j in range(8) for i in range(8)])
    np.testing.assert_allclose(share / share.sum(), h / h.sum(), rtol=1e-9)


def test_weighted_target_flattens_histogram(oracle_mod):
    ch = _toy_chains(oracle_mod, 8, target_mode=1, p_large=0.3)
    ch.run_epochs(400)
    h = ch.hist.astype(float)
    assert _tv(h / h.sum(), np.full(64, 1 / 64)) < 0.03
    b = S.toy_region_masses(TOY, 64, 64, 8)
    assert _tv(b / b.sum(), np.full(64, 1 / 64)) > 0.5
    w = ch.weight
    assert np.corrcoef(w, b)[0, 1] > 0.98      # fixed point w_k proportional to b_k
    # the per-epoch normalised image still estimates the integral
    img = ch.image()
    lum = 0.2126 * img[..., 0] + 0.7152 * img[..., 1] + 0.0722 * img[..., 2]
    assert abs(lum.mean() - b.sum()) < 0.02 * b.sum()


def test_bootstrap_normaliser(oracle_mod):
    ch = _toy_chains(oracle_mod, 8, n_bootstrap=1 << 16)
    b = S.toy_region_masses(TOY, 64, 64, 8).sum()
    # toy f = (v, v, v): pi = l(v, v, v) = v (weights sum to 1); the spread
    # of f is measured on an independent uniform sample
    rng = np.random.default_rng(99)
    qs = rng.integers(0, 2 ** 32, (1 << 14, 2), dtype=np.uint64).astype(np.uint32)
    sd_f = np.std([ch.scene.path_eval(q, 64, 64, 0)[0][0] for q in qs])
    assert abs(ch.bhat - b) < 4.5 * sd_f / math.sqrt(1 << 16)


# --------------------------------------------------------------------------
# acceptance: pointwise detailed balance with an independent kernel density
# --------------------------------------------------------------------------
def _kelemen_density(delta, sigma, s1, s2):
    """Kelemen small step, per dimension: sign 1/2, |delta| log-uniform on
    [sigma s1, sigma s2], density 1 / (|delta| ln(s2/s1)) there."""
    a = np.abs(delta)
    inside = (a >= sigma * s1) & (a <= sigma * s2)
    return np.where(inside, 0.5 / (a * math.log(s2 / s1)), 0.0).prod()


def test_detailed_balance_pointwise(oracle_mod):
    ch = _toy_chains(oracle_mod, 32)
    sig = np.array([1.0, 2.5, 0.6, 1.3], np.float32)
    ch.sigma[:] = sig
    sc = ch.scene
    s1, s2 = 1 / 1024, 1 / 64
    rng = np.random.default_rng(11)
    checked = 0
    nonzero = 0
    for _ in range(20000):
        x = rng.integers(0, 2 ** 32, 2, dtype=np.uint64).astype(np.uint32)
        kx = ch.region_of(x)
        sx = float(sig[kx])
        mag = np.exp(rng.uniform(math.log(sx * s1), math.log(sx * s2), 2))
        sgn = rng.choice([-1, 1], 2)
        dq = np.rint(sgn * mag * 2 ** 32).astype(np.int64)
        y = ((x.astype(np.int64) + dq) % 2 ** 32).astype(np.uint32)
        ky = ch.region_of(y)
        sy = float(sig[ky])
        delta = dq / 2 ** 32
        # stay clear of the support end points, decided in binary32 by the oracle
        rel = np.concatenate([np.abs(np.abs(delta) / (sy * s1) - 1), np.abs(np.abs(delta) / (sy * s2) - 1),
                              np.abs(np.abs(delta) / (sx * s1) - 1), np.abs(np.abs(delta) / (sx * s2) - 1)])
        if rel.min() < 1e-5:
            continue
        fx = sc.path_eval(x, 64, 64, 0)[0]
        fy = sc.path_eval(y, 64, 64, 0)[0]
        px = 0.2126 * fx[0] + 0.7152 * fx[1] + 0.0722 * fx[2]
        py = 0.2126 * fy[0] + 0.7152 * fy[1] + 0.0722 * fy[2]
        a_xy = ch.accept_prob(x, y, px, py)
        a_yx = ch.accept_prob(y, x, py, px)
        lhs = px * _kelemen_density(delta, sx, s1, s2) * a_xy
        rhs = py * _kelemen_density(-delta, sy, s1, s2) * a_yx
        assert lhs == pytest.approx(rhs, rel=1e-12, abs=0.0)
        checked += 1
        nonzero += lhs > 0
    assert checked > 15000 and nonzero > 5000


# --------------------------------------------------------------------------
# invariants of the adaptation (Sec. 4.3 diminishing adaptation, containment)
# --------------------------------------------------------------------------
def test_adaptation_invariants(oracle_mod):
    sc = oracle_mod.Scene(S.cornell_box(), use_bvh=False)
    ch = oracle_mod.Chains(sc, n_chains=32, epoch_len=8, n_bootstrap=1 << 12)
    ch.init()
    lmin, lmax = ch.params.lambda_min, ch.params.lambda_max
    prev_l = ch.lam.copy()
    prev_n = ch.n_updates.copy()
    for _ in range(40):
        ch.run_epochs(1)
        lam, n = ch.lam.copy(), ch.n_updates.copy()
        step = np.abs(lam - prev_l)
        upd = n - prev_n
        assert set(np.unique(upd)) <= {0, 1}                 # at most one update per epoch
        assert np.all(step[upd == 0] == 0)
        g = np.minimum(1.0, 5.0 / np.sqrt(prev_n.astype(float)))
        assert np.all(step <= g + 1e-12)                     # |d lambda| <= gamma_n
        assert np.all((lam >= lmin) & (lam <= lmax))         # containment by clamping
        prev_l, prev_n = lam, n
    st = ch.stats()
    assert int(ch.hist.sum()) == st["mutations"] == 32 * 8 * 40
    assert st["large"] + st["small"] == st["mutations"]
