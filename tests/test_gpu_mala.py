"""The adjoint kernel (rmlt_path_grad), its torch.autograd.Function, and the
Langevin (MALA) strategy on the GPU.

- Config-4 check: grad log pi on the Cornell box at depth 10 for 4096 seeded
  random u against the oracle's binary64 forward-mode gradient, and against
  binary64 central differences (h = 16 * 2^-24, about 1e-6) of the oracle's
  path map on a subset; paths within 1e-4 (1e-3 for the differences) of a
  geometric decision (the oracle's margin) are excluded and counted.
- The autograd Function's backward equals the kernel's gradient.
- MALA with adaptation on the toy integrand keeps the closed-form region
  masses (the state-dependent proposal ratio is exercised by the regional
  steps tau sigma_k^2); on the Cornell box it renders the same image as the
  plain strategies; a checkpoint restores the gradients.
- The oracle replays every mutation of a Langevin run: each Langevin
  proposal is adopted from the GPU's recorded words after checking it against
  the oracle's own (binary64 Box-Muller and forward-mode gradient) within the
  first-order bound of the binary32 rounding and of the gradient's accuracy;
  the path, the acceptance with the proposal-density ratio (including the
  (D/2) ln(tau_x / tau_y) term), the decision, the region tables and the final
  states are then compared as for the other strategies.
"""
import math

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


def _points(n, D, seed):
    rng = np.random.default_rng(seed)
    return rng.integers(0, 2 ** 32, (D, n), dtype=np.uint64).astype(np.uint32)


def test_adjoint_matches_oracle_gradient_cornell_depth10(oracle_mod):
    import torch
    R = _renderer(S.cornell_box(), n_chains=64, width=64, height=64, region_px=8, max_depth=10,
                  n_bootstrap=1 << 12)
    D, n = 52, 4096
    q = _points(n, D, 11)
    logpi, grad, f = R.path_grad(torch.from_numpy(q.view(np.int32)).cuda(), want_f=True)
    torch.cuda.synchronize()
    logpi, grad, f = logpi.cpu().numpy(), grad.cpu().numpy(), f.cpu().numpy()
    sc = oracle_mod.Scene(S.cornell_box(), use_bvh=False)
    checked = excluded = 0
    rel = []
    for i in range(n):
        fo, go, st = sc.path_grad(q[:, i], 64, 64, 10)
        _, margin, ok, _ = sc.path_eval(q[:, i], 64, 64, 10)
        pio = LUM @ fo
        if st != 1 or not ok or not pio > 0:
            continue
        if margin < 1e-4:
            excluded += 1
            continue
        checked += 1
        np.testing.assert_allclose(f[:, i], fo, rtol=1e-4, atol=1e-4 * np.abs(fo).max())
        assert abs(logpi[i] - math.log(pio)) < 1e-4
        rel.append(np.abs(grad[:, i] - go).max() / max(np.abs(go).max(), 1e-6))
    rel = np.array(rel)
    print(f"checked {checked} excluded {excluded} median rel {np.median(rel):.2e} "
          f"p99 {np.quantile(rel, 0.99):.2e} max {rel.max():.2e}")
    assert checked > 1000
    assert np.median(rel) < 1e-4
    assert np.mean(rel < 2e-3) > 0.99


def test_adjoint_matches_central_differences(oracle_mod):
    import torch
    R = _renderer(S.cornell_box(), n_chains=64, width=64, height=64, region_px=8, max_depth=10,
                  n_bootstrap=1 << 12)
    D, n = 52, 256
    q = _points(n, D, 12)
    logpi, grad, _ = R.path_grad(torch.from_numpy(q.view(np.int32)).cuda())
    torch.cuda.synchronize()
    grad = grad.cpu().numpy()
    sc = oracle_mod.Scene(S.cornell_box(), use_bvh=False)
    k = 16
    h = k / 16777216.0
    worst, checked = [], 0
    for i in range(n):
        f0, margin, ok, _ = sc.path_eval(q[:, i], 64, 64, 10)
        if not ok or not LUM @ f0 > 0 or margin < 1e-3:
            continue
        fd = np.zeros(D)
        for j in range(D):
            qp, qm = q[:, i].copy(), q[:, i].copy()
            qp[j] = np.uint32((int(qp[j]) + 256 * k) % (1 << 32))
            qm[j] = np.uint32((int(qm[j]) - 256 * k) % (1 << 32))
            fp, fm = sc.path_eval(qp, 64, 64, 10)[0], sc.path_eval(qm, 64, 64, 10)[0]
            if not (LUM @ fp > 0 and LUM @ fm > 0):
                break
            fd[j] = (math.log(LUM @ fp) - math.log(LUM @ fm)) / (2 * h)
        else:
            checked += 1
            worst.append(np.abs(grad[:, i] - fd).max() / max(np.abs(fd).max(), 1e-6))
    worst = np.array(worst)
    assert checked > 40
    assert np.mean(worst < 2e-3) > 0.97, np.sort(worst)[-5:]


def test_autograd_function_uses_the_adjoint():
    import torch
    from paper_2402_08273_gb300 import rmlt
    R = _renderer(S.cornell_box(), n_chains=64, width=64, height=64, region_px=8, max_depth=6,
                  n_bootstrap=1 << 12)
    g = torch.Generator(device="cuda").manual_seed(5)
    u = torch.rand((512, R.D), device="cuda", generator=g, dtype=torch.float32).requires_grad_(True)
    lp = rmlt.path_log_pi(u, R)
    w = torch.rand(512, device="cuda", generator=g)
    (lp.clamp(min=-1e30) * w).sum().backward()
    logpi, grad, _ = R.path_grad(rmlt.u_to_words(u).t().contiguous())
    torch.cuda.synchronize()
    assert torch.equal(lp.detach(), logpi)
    expect = (w[:, None] * grad.t())
    assert torch.allclose(u.grad, expect, rtol=1e-6, atol=0)


def test_toy_gradient_closed_form():
    import torch
    R = _renderer(toy=S.TOY_DEFAULT, n_chains=64, width=64, height=64, region_px=8, max_depth=0,
                  n_bootstrap=1 << 12)
    q = _points(2048, 2, 13)
    logpi, grad, f = R.path_grad(torch.from_numpy(q.view(np.int32)).cuda(), want_f=True)
    torch.cuda.synchronize()
    p = S.TOY_DEFAULT
    u = (q >> 8).astype(np.float64) / 16777216.0
    e = p[6] * np.exp(-((u[0] - p[7]) ** 2 + (u[1] - p[8]) ** 2) / (2 * p[9] ** 2))
    box = (u[0] >= p[2]) & (u[0] < p[3]) & (u[1] >= p[4]) & (u[1] < p[5])
    fv = p[0] + np.where(box, p[1], 0.0) + e
    expect = np.stack([-e * (u[0] - p[7]), -e * (u[1] - p[8])]) / (p[9] ** 2 * fv)
    np.testing.assert_allclose(grad.cpu().numpy(), expect, rtol=1e-4, atol=1e-3)


def test_mala_toy_keeps_region_masses():
    R = _renderer(toy=S.TOY_DEFAULT, n_chains=256, width=64, height=64, region_px=8, max_depth=0,
                  n_bootstrap=1 << 14, p_large=0.1, p_mala=0.6, mala_tau=1e-3, mala_drift_max=0.1)
    R.step(200 * 16)
    st = R.read_stats()
    h = R.read_region_hist().astype(float)
    b = S.toy_region_masses(S.TOY_DEFAULT, 64, 64, 8)
    tv = 0.5 * np.abs(h / h.sum() - b / b.sum()).sum()
    lam = R.read_region_params()["lambda"]
    assert np.ptp(lam) > 0.5           # regional steps differ
    assert st["mala"] > 0.5 * 256 * 3200 and 0.1 < st["mala_accepted"] / st["mala"] < 0.95
    assert tv < 0.025, tv


def test_mala_cornell_renders_the_same_image():
    kw = dict(n_chains=4096, width=64, height=64, region_px=8, max_depth=10, n_bootstrap=1 << 16, p_large=0.3)
    A = _renderer(S.cornell_box(), **kw)
    B = _renderer(S.cornell_box(), p_mala=0.3, mala_tau=1e-3, **kw)
    A.step(512)
    B.step(512)
    st = B.read_stats()
    assert st["mala"] > 0.25 * 4096 * 512 and st["invalid_paths"] == 0
    assert 0.05 < st["mala_accepted"] / st["mala"] < 0.95
    ia, ib = A.read_image(), B.read_image()
    la, lb = ia @ LUM, ib @ LUM
    assert abs(lb.mean() - B.read_stats()["bhat"]) < 1e-9 * lb.mean()   # f / pi has unit luminance
    # region totals agree within the Monte Carlo noise of either render
    ra = la.reshape(8, 8, 8, 8).sum(axis=(1, 3))
    rb = lb.reshape(8, 8, 8, 8).sum(axis=(1, 3))
    assert 0.5 * np.abs(ra / ra.sum() - rb / rb.sum()).sum() < 0.03


def test_mala_checkpoint_resume_equals_uninterrupted(tmp_path):
    kw = dict(n_chains=512, width=64, height=64, region_px=8, max_depth=8, n_bootstrap=1 << 14, p_large=0.3,
              p_mala=0.4, mala_tau=1e-3)
    A = _renderer(S.cornell_box(), **kw)
    A.step(128)
    B = _renderer(S.cornell_box(), **kw)
    B.step(64)
    path = str(tmp_path / "m.ckpt")
    B.save(path)
    from paper_2402_08273_gb300 import rmlt
    Cn = rmlt.Renderer()
    Cn.load_scene(S.cornell_box())
    Cn.restore(path)
    Cn.step(64)
    sa, sc = A.read_chain_state(), Cn.read_chain_state()
    assert np.array_equal(sa["q"], sc["q"]) and np.array_equal(sa["f"], sc["f"])
    assert np.array_equal(A.read_region_hist(), Cn.read_region_hist())


def test_mala_rejections():
    from paper_2402_08273_gb300 import rmlt
    R = rmlt.Renderer()
    R.load_scene(S.two_rooms(3000, seed=1))   # GGX surfaces
    with pytest.raises(rmlt.RmltError):
        R.init_chains(n_chains=64, width=32, height=32, region_px=8, max_depth=3, p_mala=0.3)
    R = _renderer(S.cornell_box(), n_chains=64, max_depth=4, p_mala=0.3, n_bootstrap=1 << 12)
    R.set_tuning(wavefront=True)
    with pytest.raises(rmlt.RmltError):
        R.step(16)


# the most mutations each window may let through, measured on a GB300
PINS_REPLAY = {"toy": {}, "cornell": {"f_bounded": 4}}


@pytest.mark.parametrize("case", ["toy", "cornell"])
def test_mala_oracle_replay(oracle_mod, case):
    from gpu_run import check_counters, replay_full, traced_run
    if case == "toy":
        gpu = traced_run(toy=S.TOY_DEFAULT, words=True, n_epochs=30, n_chains=128, width=64, height=64, region_px=8,
                         max_depth=0, n_bootstrap=1 << 13, p_large=0.1, p_mala=0.5, mala_tau=1e-3,
                         mala_drift_max=0.1)
        osc = oracle_mod.Scene(toy=S.TOY_DEFAULT)
    else:
        gpu = traced_run(scene=S.cornell_box(), words=True, n_epochs=10, n_chains=64, width=64, height=64,
                         region_px=8, max_depth=5, n_bootstrap=1 << 13, p_large=0.3, p_mala=0.3, mala_tau=1e-3,
                         mala_drift_max=0.1)
        osc = oracle_mod.Scene(S.cornell_box(), use_bvh=False)
    ch, rp, adopted = replay_full(oracle_mod, gpu, osc)
    print("Langevin replay:", rp.summary())
    check_counters(ch, gpu, rp, PINS_REPLAY[case], adopted, 0)
    assert rp.s["langevin"] > 0.2 * rp.s["mutations"]
    assert rp.s["proposal_adopted"] == rp.s["langevin"] and rp.s["proposal_mismatch"] == 0
    st = gpu["stats"]
    assert st["mala"] == rp.s["langevin"] and st["mala_accepted"] > 0
