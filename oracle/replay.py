"""Mutation-by-mutation comparison of a traced GPU run with the oracle.

TEST INFRASTRUCTURE (used by the GPU parity tests and the smoke check).  It
takes the GPU's trace as plain numpy arrays and never imports the CUDA
library.

The oracle runs its own algorithm; at every mutation a hook compares the
oracle's proposal with the GPU's record:

* the proposal's 32-bit FNV-1a hash, the large-step flag and the
  early-reject flag (reverse-kernel support) must agree exactly;
* the path contribution f(y) must agree within ``f_rtol_hard`` of its
  largest channel, and within ``f_rtol`` except for a counted few (binary32
  accumulation over a long, moderately conditioned path), unless the oracle reports the path within ``margin_thr`` (scene
  relative) of a geometric decision (a triangle edge, a near tie, a grazing
  angle) -- then the mismatch is counted as excluded and the oracle continues
  with the GPU's value so the trajectories stay in step;
* the acceptance probability must agree within ``a_rtol_hard`` (``a_rtol``
  except for a counted few);
* the accept/reject decision must agree, except when the uniform lies between
  the two acceptance probabilities (or within 1e-6 of the oracle's): counted as
  excluded, and the oracle follows the GPU's decision.

At every region update the resulting lambda_k must equal the GPU's bit for
bit; a different sign of (alpha_hat - alpha*) is excluded only when
|alpha_hat - alpha*| < ``upd_thr``.
"""
from __future__ import annotations

import math

import numpy as np

FNV_OFF, FNV_PRIME = 2166136261, 16777619


def fnv32(words, n: int) -> int:
    h = FNV_OFF
    for i in range(n):
        h = ((h ^ int(words[i])) * FNV_PRIME) & 0xFFFFFFFF
    return h


def lum(f) -> float:
    return 0.2126 * f[0] + 0.7152 * f[1] + 0.0722 * f[2]


class Replay:
    def __init__(self, chains, trace: np.ndarray, lambdas: np.ndarray | None, stride: int = 1,
                 margin_thr: float = 1e-5, f_rtol: float = 1e-4, a_rtol: float = 3e-4,
                 f_rtol_hard: float = 1e-3, a_rtol_hard: float = 3e-3,
                 upd_thr: float = 1e-3, epoch0: int = 0, max_fail_log: int = 20):
        self.ch = chains
        self.E = chains.params.epoch_len
        self.stride = stride
        self.f = trace["f"].astype(np.float64)
        self.a = trace["a"].astype(np.float64)
        self.qh = trace["qhash"]
        self.flags = trace["flags"]
        self.lambdas = lambdas
        self.margin_thr, self.f_rtol, self.a_rtol, self.upd_thr = margin_thr, f_rtol, a_rtol, upd_thr
        self.f_rtol_hard, self.a_rtol_hard = f_rtol_hard, a_rtol_hard
        self.epoch0 = epoch0
        self.cur_epoch = 0
        self.max_fail_log = max_fail_log
        self.s = dict(mutations=0, q_mismatch=0, large_mismatch=0, early_mismatch=0, f_mismatch=0,
                      f_excluded=0, f_soft=0, a_soft=0, a_mismatch=0, decision_mismatch=0, decision_excluded=0,
                      near_threshold=0, update_mismatch=0, update_excluded=0, lambda_mismatch=0,
                      updates=0)
        self.f_max_rel = 0.0
        self.a_max_rel = 0.0
        self.failures: list[str] = []
        chains.set_hooks(self._mut, self._upd)

    def _fail(self, msg):
        if len(self.failures) < self.max_fail_log:
            self.failures.append(msg)

    # ---------------------------------------------------------------- hooks
    def _mut(self, user, chain, mut, qy, D, large, early, margin, xi, fy, a, acc):
        e = mut // self.E - self.epoch0
        j = mut % self.E
        if chain % self.stride:
            return
        t = chain // self.stride
        s = self.s
        s["mutations"] += 1
        flags = int(self.flags[e, t, j])
        if fnv32(qy, D) != int(self.qh[e, t, j]):
            s["q_mismatch"] += 1
            self._fail(f"chain {chain} mut {mut}: proposal hash differs")
        if bool(flags & 2) != bool(large):
            s["large_mismatch"] += 1
            self._fail(f"chain {chain} mut {mut}: large-step flag differs")
        if bool(flags & 4) != bool(early):
            s["early_mismatch"] += 1
            self._fail(f"chain {chain} mut {mut}: reverse-kernel support differs")
        fg = self.f[e, t, j]
        if not early:
            fo = (fy[0], fy[1], fy[2])
            scale = max(abs(fo[0]), abs(fo[1]), abs(fo[2]), abs(fg[0]), abs(fg[1]), abs(fg[2]))
            err = max(abs(fg[0] - fo[0]), abs(fg[1] - fo[1]), abs(fg[2] - fo[2]))
            if err > self.f_rtol * scale and err <= self.f_rtol_hard * scale and margin >= self.margin_thr:
                s["f_soft"] += 1
                self.f_max_rel = max(self.f_max_rel, err / scale)
            elif err > self.f_rtol * scale:
                if margin < self.margin_thr:
                    s["f_excluded"] += 1
                    for c3 in range(3):
                        fy[c3] = float(fg[c3])
                    qy_np = np.ctypeslib.as_array(qy, (D,)).copy()
                    a[0] = self.ch.accept_prob(self.ch.q[chain], qy_np, self.ch.pi[chain], lum(fg), large)
                    acc[0] = int(xi < a[0])
                else:
                    s["f_mismatch"] += 1
                    self._fail(f"chain {chain} mut {mut}: f oracle {fo} gpu {tuple(fg)} margin {margin:.3g}")
            elif scale > 0:
                self.f_max_rel = max(self.f_max_rel, err / scale)
        ao, ag = a[0], float(self.a[e, t, j])
        da = abs(ao - ag)
        if da > self.a_rtol_hard * max(ao, ag, 1e-30):
            s["a_mismatch"] += 1
            self._fail(f"chain {chain} mut {mut}: a oracle {ao} gpu {ag}")
        else:
            if da > self.a_rtol * max(ao, ag, 1e-30):
                s["a_soft"] += 1
            if max(ao, ag) > 0:
                self.a_max_rel = max(self.a_max_rel, da / max(ao, ag))
        if abs(xi - ao) < 1e-6:
            s["near_threshold"] += 1
        go, gg = bool(acc[0]), bool(flags & 1)
        if go != gg:
            if (xi < ag) == gg and abs(xi - ao) <= max(1e-6, 2.0 * da):
                s["decision_excluded"] += 1
            else:
                s["decision_mismatch"] += 1
                self._fail(f"chain {chain} mut {mut}: decision oracle {go} gpu {gg} xi {xi} a {ao}/{ag}")
            acc[0] = int(gg)

    def _upd(self, user, k, i_k, A_k, ahat, sign):
        if self.lambdas is None:
            return
        p = self.ch.params
        s = self.s
        s["updates"] += 1
        lam_g = float(self.lambdas[self.cur_epoch, k])
        lam_old = float(self.ch.lam[k])
        g = min(p.gamma_max, p.gamma_scale / math.sqrt(float(self.ch.n_updates[k])))

        def result(sg):
            v = lam_old + g * float(sg)
            return min(max(v, p.lambda_min), p.lambda_max)

        if result(sign[0]) == lam_g:
            return
        cands = [sg for sg in (-1, 0, 1) if result(sg) == lam_g]
        if cands and abs(ahat - p.alpha_star) < self.upd_thr:
            s["update_excluded"] += 1
        else:
            s["update_mismatch"] += 1
            self._fail(f"epoch {self.cur_epoch} region {k}: lambda oracle {result(sign[0])} gpu {lam_g} "
                       f"alpha_hat {ahat}")
        if cands:
            sign[0] = cands[0]

    # -------------------------------------------------------------- drivers
    def run_full(self, n_epochs: int):
        """All chains, epoch by epoch (the oracle's own epoch loop and region update)."""
        for e in range(n_epochs):
            self.cur_epoch = e
            self.ch.run_epochs(1)
            if self.lambdas is not None:
                lam = self.ch.lam                   # the current regions (a quadtree grows)
                bad = np.flatnonzero(lam != self.lambdas[e][:len(lam)])
                if len(bad):
                    self.s["lambda_mismatch"] += len(bad)
                    self._fail(f"epoch {e}: lambda differs in regions {bad[:8].tolist()}")
                    lam[:] = self.lambdas[e][:len(lam)]
                    self.ch.refresh_sigma()

    def run_sampled(self, n_epochs: int, traced_chains):
        """Only the traced chains; after each epoch the GPU's lambda table is
        taken over (the oracle recomputes sigma from it)."""
        for e in range(n_epochs):
            self.cur_epoch = e
            mut0 = (self.epoch0 + e) * self.E
            for c in traced_chains:
                for j in range(self.E):
                    self.ch.mutate_one(int(c), mut0 + j)
            if self.lambdas is not None:
                self.ch.lam[:] = self.lambdas[e]
                self.ch.refresh_sigma()

    def ok(self) -> bool:
        s = self.s
        return not (s["q_mismatch"] or s["large_mismatch"] or s["early_mismatch"] or s["f_mismatch"]
                    or s["a_mismatch"] or s["decision_mismatch"] or s["update_mismatch"]
                    or s["lambda_mismatch"])

    def summary(self) -> str:
        return (f"{self.s} f_max_rel={self.f_max_rel:.3g} a_max_rel={self.a_max_rel:.3g} "
                f"failures={self.failures[:5]}")


def adopt_initial_states(chains, q_gpu: np.ndarray, max_adopt: int) -> int:
    """Compare the oracle's initial states with the GPU's ([D][C] words).

    Each chain picks its start from its own bootstrap slice; a path that
    binary32 and binary64 evaluate differently (a triangle edge) can move one
    chain's pick.  Up to ``max_adopt`` such chains are given the GPU's
    starting state (the oracle recomputes f itself); returns how many."""
    q_o = chains.q
    diff = np.flatnonzero(np.any(q_o != q_gpu.T, axis=1))
    if len(diff) > max_adopt:
        raise AssertionError(f"{len(diff)} initial states differ (chains {diff[:10].tolist()})")
    for c in diff:
        chains.set_state(int(c), q_gpu[:, c])
    return len(diff)
