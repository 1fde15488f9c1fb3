"""Pins of three oracle parts that the Lambertian furnace cannot see.

* GGX (Walter et al. 2007), the path map's own code (`ggx_continue`,
  `bsdf_eval`), in the local frame n = z:
  - the weak white furnace (Heitz 2014): for every wo,
    int D(m) G1(wo) <wo, m>+ / <wo, n> dm = 1.  Estimated through the
    oracle's half-vector sampling (density D(m) cos theta_m), it pins the
    sampling density and the Smith masking together;
  - the sampling weight f_r cos / pdf averaged over the uniforms equals the
    directional albedo int f_r(wo, wi) cos theta_i dwi by an independent
    quadrature of the evaluated BSDF over the sphere; a planted mistake (the
    reflection Jacobian 4 <wo, m> dropped) fails it;
  - reciprocity f_r(wo, wi) = f_r(wi, wo).
* Next-event light choice in proportion to triangle area: a furnace cube whose
  faces are split into triangles of very different areas keeps the closed form
  le sum rho^i; choosing triangles uniformly (planted) is biased and fails.
* Starting states: systematic resampling of all bootstrap samples in
  proportion to pi puts the chains in region k with probability b_k / b;
  chi-square on the toy integrand against its closed-form region masses.
"""
import numpy as np
import pytest
from numpy.polynomial.legendre import leggauss

from paper_2402_08273_gb300 import scenes as S


def _wo(theta_deg):
    t = np.radians(theta_deg)
    return np.array([np.sin(t), 0.0, np.cos(t)])


def _uniform_grid(n_s=256, n_phi=256):
    """Nodes and weights on [0,1)^2 for the sampling uniforms (bu, bv): bu =
    1 - s^2 with Gauss-Legendre in s (the 1 / cos theta_m of the weights is an
    integrable 1/sqrt singularity at bu -> 1, regular in s), bv periodic
    (midpoints)."""
    x, w = leggauss(n_s)
    s = 0.5 * (x + 1.0)
    ws = 0.5 * w * 2.0 * s                    # du = 2 s ds
    bu = 1.0 - s * s
    bv = (np.arange(n_phi) + 0.5) / n_phi
    BU, BV = np.meshgrid(bu, bv, indexing="ij")
    W = np.outer(ws, np.full(n_phi, 1.0 / n_phi))
    return BU.ravel(), BV.ravel(), W.ravel()


def _albedo_quadrature(oracle_mod, alpha, F0, wo):
    """int f_r(wo, wi) cos theta_i dwi over the sphere, in spherical
    coordinates around the mirror direction of wo (the lobe's centre) with
    Gauss-Legendre panels that refine towards it; f_r = 0 below the surface."""
    r = np.array([-wo[0], -wo[1], wo[2]])
    # orthonormal frame (e1, e2, r)
    e1 = np.cross(r, [0.0, 1.0, 0.0])
    if np.linalg.norm(e1) < 1e-8:
        e1 = np.array([1.0, 0.0, 0.0])
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(r, e1)
    edges = [0.0] + [alpha * f for f in (0.01, 0.03, 0.1, 0.3, 1.0, 2.0, 4.0, 8.0, 16.0, 40.0)] + [np.pi]
    edges = sorted(set(min(e, np.pi) for e in edges))
    xg, wg = leggauss(48)
    th, wt = [], []
    for a, b in zip(edges[:-1], edges[1:]):
        th.append(0.5 * (b - a) * xg + 0.5 * (a + b))
        wt.append(0.5 * (b - a) * wg)
    th, wt = np.concatenate(th), np.concatenate(wt)
    n_phi = 720
    ph = (np.arange(n_phi) + 0.5) * 2 * np.pi / n_phi
    T, P = np.meshgrid(th, ph, indexing="ij")
    d = (np.sin(T)[..., None] * (np.cos(P)[..., None] * e1 + np.sin(P)[..., None] * e2) +
         np.cos(T)[..., None] * r).reshape(-1, 3)
    fr = oracle_mod.ggx_eval(alpha, F0, wo, d)
    cos_i = np.maximum(d[:, 2], 0.0)
    jac = (np.sin(T) * wt[:, None]).reshape(-1) * (2 * np.pi / n_phi)
    return (fr * (cos_i * jac)[:, None]).sum(axis=0)


ALPHAS = (0.02, 0.1, 0.5)
THETAS = (0.0, 30.0, 60.0, 80.0)


@pytest.mark.parametrize("alpha", ALPHAS)
@pytest.mark.parametrize("theta", THETAS)
def test_ggx_weak_white_furnace(oracle_mod, alpha, theta):
    wo = _wo(theta)
    bu, bv, W = _uniform_grid()
    _, _, m = oracle_mod.ggx_sample(alpha, [1, 1, 1], wo, bu, bv)
    co = wo[2]
    est = oracle_mod.ggx_g1(co, alpha) * np.maximum(m @ wo, 0.0) / (co * m[:, 2])
    assert abs((est * W).sum() - 1.0) < 2e-6


@pytest.mark.parametrize("alpha", ALPHAS)
@pytest.mark.parametrize("theta", THETAS)
def test_ggx_sampling_weight_matches_albedo(oracle_mod, alpha, theta):
    F0 = np.array([1.0, 0.5, 0.04])
    wo = _wo(theta)
    bu, bv, W = _uniform_grid()
    _, w, _ = oracle_mod.ggx_sample(alpha, F0, wo, bu, bv)
    est = (w * W[:, None]).sum(axis=0)
    ref = _albedo_quadrature(oracle_mod, alpha, F0, wo)
    np.testing.assert_allclose(est, ref, rtol=3e-4)
    # the planted mistake (reflection Jacobian dropped) is far outside
    _, wp, _ = oracle_mod.ggx_sample(alpha, F0, wo, bu, bv, planted=1)
    bad = (wp * W[:, None]).sum(axis=0)
    assert np.all(np.abs(bad / ref - 1.0) > 0.1)


def test_ggx_reciprocity_and_energy(oracle_mod):
    rng = np.random.default_rng(3)
    for alpha in ALPHAS:
        a = rng.normal(size=(2000, 3))
        b = rng.normal(size=(2000, 3))
        a[:, 2] = np.abs(a[:, 2])
        b[:, 2] = np.abs(b[:, 2])
        a /= np.linalg.norm(a, axis=1, keepdims=True)
        b /= np.linalg.norm(b, axis=1, keepdims=True)
        F0 = [0.9, 0.5, 0.1]
        fab = np.array([oracle_mod.ggx_eval(alpha, F0, a[i], b[i:i + 1])[0] for i in range(200)])
        fba = np.array([oracle_mod.ggx_eval(alpha, F0, b[i], a[i:i + 1])[0] for i in range(200)])
        np.testing.assert_allclose(fab, fba, rtol=1e-12, atol=0)
    # single scattering loses energy but never creates it (F0 = 1)
    for alpha in ALPHAS:
        for theta in THETAS:
            assert _albedo_quadrature(oracle_mod, alpha, [1, 1, 1], _wo(theta))[0] <= 1.0 + 2e-3


@pytest.mark.parametrize("plant", [False, True])
def test_light_choice_by_area(oracle_mod, plant):
    """Uneven furnace (triangles of areas 0.035 .. 0.47 on every face): plain
    Monte Carlo of the path map equals le sum_{i<=d} rho^i within 4.5 sigma
    with the area-proportional light choice, and misses it by more than 8
    sigma with the uniform choice planted."""
    sc = oracle_mod.Scene(S.furnace_uneven(rho=0.5, le=1.0), use_bvh=False)
    if plant:
        sc.plant_uniform_lights()
    depth = 3
    rng = np.random.default_rng(5)
    n = 1 << 15
    qs = rng.integers(0, 2 ** 32, (n, 2 + 5 * depth), dtype=np.uint64).astype(np.uint32)
    f = np.array([sc.path_eval(q, 16, 16, depth)[0][0] for q in qs])
    expect = sum(0.5 ** i for i in range(depth + 1))
    z = abs(f.mean() - expect) / (f.std() / np.sqrt(n))
    if plant:
        assert z > 8.0, z
    else:
        assert z < 4.5, z


def test_starting_states_follow_the_target(oracle_mod):
    """Chains take their start by systematic resampling of the n_bootstrap
    uniform samples in proportion to pi.  The chains' regions are then
    distributed as the region masses b_k / b of the toy integrand (closed
    form): chi-square test.  Unweighted picks of uniform samples fail the same
    test."""
    from scipy import stats
    C, K = 4096, 256
    ch = oracle_mod.Chains(oracle_mod.Scene(toy=S.TOY_DEFAULT), n_chains=C, width=32, height=32, region_px=8,
                           max_depth=0, n_bootstrap=C * K, seed=21)
    ch.init()
    masses = S.toy_region_masses(S.TOY_DEFAULT, 32, 32, 8)
    p = masses / masses.sum()
    obs = np.bincount(ch.k, minlength=len(p))
    chi2 = ((obs - C * p) ** 2 / (C * p)).sum()
    assert stats.chi2.sf(chi2, len(p) - 1) > 1e-3, chi2
    # power: one uniform sample per chain (what an unweighted pick gives)
    first = np.array([ch.region_of(_boot_sample(oracle_mod, 21, c * K, 2)) for c in range(C)])
    obs_u = np.bincount(first, minlength=len(p))
    chi2_u = ((obs_u - C * p) ** 2 / (C * p)).sum()
    assert stats.chi2.sf(chi2_u, len(p) - 1) < 1e-6, chi2_u


def _boot_sample(oracle_mod, seed, s, D):
    """Bootstrap sample s: Philox counter (s lo, s hi, 0xFFFFFFFF, 0x8000 + j), key = seed."""
    out = []
    for j in range((D + 3) // 4):
        r = oracle_mod.philox4x32_10([s & 0xFFFFFFFF, s >> 32, 0xFFFFFFFF, 0x8000 + j], [seed & 0xFFFFFFFF, seed >> 32])
        out.extend(int(x) for x in r)
    return np.array(out[:D], np.uint32)
