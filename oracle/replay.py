"""Mutation-by-mutation comparison of a traced GPU run with the oracle.

TEST INFRASTRUCTURE (used by the GPU parity tests and the smoke check).  It
takes the GPU's trace as plain numpy arrays and never imports the CUDA
library.

The oracle runs its own algorithm; at every traced mutation a hook compares
the oracle's proposal with the GPU's record.  Every window below comes from
the oracle's first-order model of what binary32 evaluation of the same path
can change (`or_path_eval_err`: unit roundoff 2^-24 propagated through the
path's positions, directions, cosines, distances and the GGX density), not
from the failures it removes:

* exact: the proposal's 32-bit FNV-1a hash, the large-step and early-reject
  (reverse-kernel support) flags;
* f(y): every channel within 1e-4 of the largest, or within `err_factor`
  times the channel's binary32 error bound where that is larger (counted as
  `f_bounded`); a path whose nearest decision (triangle edge, tie, cosine
  sign, light CDF, frame switch) lies within `dec_thr` error bounds of
  flipping may differ entirely: counted as `f_excluded`, and the oracle
  continues with the GPU's value so that the trajectories stay in step;
* a: the GPU's and the oracle's acceptance probabilities differ exactly by
  what their inputs differ by: |ln a_g - ln a_o| <= |ln(pi_y,g / pi_y,o)| +
  |ln(pi_x,g / pi_x,o)| + 32 u (the states' pi as each side computed them);
* the decision: exact, except when the uniform lies between the two
  acceptance probabilities (counted as `decision_excluded`; the oracle follows
  the GPU);
* proposals whose last bits depend on binary32 rounding (the truncated-normal
  kernel's erfinv offsets, Langevin moves) are adopted from the GPU's
  recorded words (`words`) when they lie within the first-order bound of that
  rounding around the oracle's own proposal (counted as `proposal_adopted`;
  beyond it, `proposal_mismatch`); the Langevin acceptance may further differ
  by what a relative error `EPS_G` of the drifts (the adjoint's gradient
  against the oracle's) changes in it, ln a +- EPS_G S (S from the oracle);
* the region update (Alg. 1, region update): with every chain traced, the GPU's
  A_k is rebuilt exactly from its own recorded acceptance probabilities
  (sum of round(a 2^32) over the small steps of region k), and the GPU's
  lambda_k must equal the update computed from that A_k bit for bit.  The
  oracle's own sign of (alpha_hat - alpha*) may differ only when alpha* lies
  between the two estimates (counted as `update_excluded`).
"""
from __future__ import annotations

import math

import numpy as np

FNV_OFF, FNV_PRIME = 2166136261, 16777619
U = 2.0 ** -24
# relative accuracy assumed for the adjoint kernel's gradient against the
# oracle's forward-mode gradient: twice the largest relative difference
# measured on 4096 Cornell-box paths at depth 10 (5.3e-4)
EPS_G = 1e-3


def fnv32(words, n: int) -> int:
    h = FNV_OFF
    for i in range(n):
        h = ((h ^ int(words[i])) * FNV_PRIME) & 0xFFFFFFFF
    return h


def lum(f) -> float:
    return 0.2126 * f[0] + 0.7152 * f[1] + 0.0722 * f[2]


def _log_ratio(a: float, b: float) -> float:
    if a == b:
        return 0.0
    if a <= 0.0 or b <= 0.0:
        return math.inf
    return abs(math.log(a / b))


class Replay:
    def __init__(self, chains, trace: np.ndarray, lambdas: np.ndarray | None, stride: int = 1,
                 init_f: np.ndarray | None = None, f_rtol: float = 1e-4, err_factor: float = 4.0,
                 dec_thr: float = 4.0, epoch0: int = 0, max_fail_log: int = 20, words: np.ndarray | None = None):
        """init_f: the GPU's contributions of the chains' states when the
        replay starts ([3][C] floats), for the acceptance check.  words: the
        GPU's proposal words of every record ([epoch][traced chain][mutation][D]
        u32) for the proposals the replay adopts."""
        self.ch = chains
        self.E = chains.params.epoch_len
        self.stride = stride
        self.f = trace["f"].astype(np.float64)
        self.a = trace["a"].astype(np.float64)
        self.qh = trace["qhash"]
        self.flags = trace["flags"]
        self.lambdas = lambdas
        self.f_rtol, self.err_factor, self.dec_thr = f_rtol, err_factor, dec_thr
        self.epoch0 = epoch0
        self.cur_epoch = 0
        self.max_fail_log = max_fail_log
        C = chains.C
        self.px_o = np.array(chains.pi, dtype=np.float64)
        if init_f is not None:
            f = np.asarray(init_f, np.float64)
            self.px_g = 0.2126 * f[0] + 0.7152 * f[1] + 0.0722 * f[2]
        else:
            self.px_g = self.px_o.copy()
        # the GPU's region statistics rebuilt from its trace (every chain traced)
        cap = int(chains.exchange_buffers()[1].shape[0])
        self.A_g = np.zeros(cap, dtype=object)
        self.i_g = np.zeros(cap, dtype=np.int64)
        self.words = words
        self.s = dict(mutations=0, q_mismatch=0, large_mismatch=0, early_mismatch=0, f_mismatch=0,
                      f_bounded=0, f_excluded=0, a_mismatch=0, decision_mismatch=0, decision_excluded=0,
                      update_mismatch=0, update_excluded=0, lambda_mismatch=0, visits_mismatch=0, updates=0,
                      proposal_adopted=0, proposal_mismatch=0, langevin=0, kind_mismatch=0)
        self.prop_use = 0.0      # largest proposal difference as a fraction of its bound
        self.f_max_rel = 0.0
        self.a_max_rel = 0.0
        self.bound_use = 0.0     # largest f error as a fraction of its allowed bound
        self.failures: list[str] = []
        assert len(self.px_o) == C
        chains.set_hooks(self._mut, self._upd, self._prop if words is not None else None)

    def _fail(self, msg):
        if len(self.failures) < self.max_fail_log:
            self.failures.append(msg)

    # ---------------------------------------------------------------- hooks
    def _prop(self, user, chain, mut, kind, qy, D):
        """Adopt the GPU's proposal where binary32 rounding decides its last
        bits, after checking it against the oracle's own within that rounding's
        first-order bound (in units of 2^-32 per dimension)."""
        if chain % self.stride:
            return
        e = mut // self.E - self.epoch0
        j = mut % self.E
        t = chain // self.stride
        g = self.words[e, t, j, :D].astype(np.int64)
        own = np.ctypeslib.as_array(qy, (D,)).astype(np.int64)
        truncnorm = kind == 0 and self.ch.params.kernel == 1
        if not (truncnorm or kind == 2):
            return                      # Philox words and Kelemen offsets are exact: compared by the hash
        qx = self.ch.q[chain].astype(np.int64)
        off_o = ((own - qx + 2 ** 31) % 2 ** 32) - 2 ** 31
        off_g = ((g - qx + 2 ** 31) % 2 ** 32) - 2 ** 31
        if truncnorm:
            # dl = sigma sqrt(2) erfinv(x), x = (2u - 1) Z(sigma): binary32 x errs by
            # ~6 u |x|, erfinv amplifies it by (sqrt(pi) / 2) exp(y^2), the rest ~6 u |y|
            sigma = float(self.ch.sigma[int(self.ch.k[chain])])
            y = off_o * 2.0 ** -32 / (sigma * math.sqrt(2.0))
            x = np.array([math.erf(v) for v in y])
            amp = np.exp(np.minimum(y * y, 700.0))
            tol = 4.0 * (2.0 ** 32 * sigma * math.sqrt(2.0) * (0.5 * math.sqrt(math.pi) * amp * 6 * U * np.abs(x)
                                                                 + 6 * U * np.abs(y))) + 2.0
        else:
            # step = m + sqrt(tau) z: the drift errs by EPS_G |m| (gradient); a
            # Box-Muller pair z = rho (cos, sin), rho^2 = -2 ln u1, errs by ~8 u |z|
            # plus the binary32 rounding of u1 = (x + 1/2) 2^-24 (up to u absolute),
            # which ln u1 amplifies by 1 / |ln u1| = 2 / rho^2; the sum by ~4 u |step|
            m, z, tau, _ = self.ch.last_mala()
            rho2 = np.array([z[d] ** 2 + (z[d ^ 1] ** 2 if (d ^ 1) < D else 0.0) for d in range(D)])
            ez = np.abs(z) * (8 * U + U / np.maximum(rho2, 1e-300))
            step = m + math.sqrt(tau) * z
            tol = 4.0 * 2.0 ** 32 * (EPS_G * np.abs(m) + math.sqrt(tau) * ez + 4 * U * np.abs(step)) + 2.0
        diff = np.abs(off_g - off_o)
        self.prop_use = max(self.prop_use, float(np.max(diff / tol)))
        if np.all(diff <= tol):
            self.s["proposal_adopted"] += 1
        else:
            self.s["proposal_mismatch"] += 1
            d = int(np.argmax(diff / tol))
            self._fail(f"chain {chain} mut {mut}: proposal word {d} oracle {int(own[d])} gpu {int(g[d])} "
                       f"(allowed {tol[d]:.3g})")
        np.ctypeslib.as_array(qy, (D,))[:] = self.words[e, t, j, :D]

    def _mut(self, user, chain, mut, qy, D, large, early, dec, ferr, xi, fy, a, acc):
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
        langevin = large == 2
        if bool(flags & 16) != langevin:
            s["kind_mismatch"] += 1
            self._fail(f"chain {chain} mut {mut}: Langevin flag differs")
        if langevin:
            s["langevin"] += 1
            large = 0
        if bool(flags & 2) != bool(large):
            s["large_mismatch"] += 1
            self._fail(f"chain {chain} mut {mut}: large-step flag differs")
        if bool(flags & 4) != bool(early):
            s["early_mismatch"] += 1
            self._fail(f"chain {chain} mut {mut}: reverse-kernel support differs")
        fg = self.f[e, t, j]
        kx = int(self.ch.k[chain])
        if not early:
            fo = (fy[0], fy[1], fy[2])
            scale = max(abs(fo[0]), abs(fo[1]), abs(fo[2]), abs(fg[0]), abs(fg[1]), abs(fg[2]))
            errs = [abs(fg[c] - fo[c]) for c in range(3)]
            allow = [max(self.f_rtol * scale, self.err_factor * ferr[c]) for c in range(3)]
            if scale > 0:
                self.bound_use = max(self.bound_use, max(errs[c] / allow[c] for c in range(3)))
            if all(errs[c] <= self.f_rtol * scale for c in range(3)):
                if scale > 0:
                    self.f_max_rel = max(self.f_max_rel, max(errs) / scale)
            elif all(errs[c] <= allow[c] for c in range(3)):
                s["f_bounded"] += 1
            elif dec < self.dec_thr:
                s["f_excluded"] += 1
                for c3 in range(3):
                    fy[c3] = float(fg[c3])
                qy_np = np.ctypeslib.as_array(qy, (D,)).copy()
                a[0] = self.ch.accept_prob(self.ch.q[chain], qy_np, self.ch.pi[chain], lum(fg), large)
                acc[0] = int(xi < a[0])
            else:
                s["f_mismatch"] += 1
                self._fail(f"chain {chain} mut {mut}: f oracle {fo} gpu {tuple(fg)} bound "
                           f"{tuple(ferr[c] for c in range(3))} dec {dec:.3g}")
        ao, ag = a[0], float(self.a[e, t, j])
        # the two sides' inputs: pi of the proposal and of the current state
        py_o, py_g = lum((fy[0], fy[1], fy[2])), lum(fg)
        pred = _log_ratio(py_g, py_o) + _log_ratio(self.px_g[chain], self.px_o[chain]) + 32 * U
        if langevin:
            pred += EPS_G * self.ch.last_mala()[3] + 64 * U * D
        elif self.ch.params.kernel == 1 and not large:
            pred += 8 * U * D          # the truncated normal's Z(sigma) in binary32 (erff), D times
        da = abs(ao - ag)
        amax = max(ao, ag)
        if amax > 0:
            self.a_max_rel = max(self.a_max_rel, da / amax)
        if da > amax * min(pred, 1.0) + 1e-30 and not (ao == 0.0 and ag == 0.0):
            s["a_mismatch"] += 1
            self._fail(f"chain {chain} mut {mut}: a oracle {ao} gpu {ag} (allowed {amax * pred:.3g})")
        go, gg = bool(acc[0]), bool(flags & 1)
        if go != gg:
            if min(ao, ag) <= xi <= max(ao, ag):
                s["decision_excluded"] += 1
            else:
                s["decision_mismatch"] += 1
                self._fail(f"chain {chain} mut {mut}: decision oracle {go} gpu {gg} xi {xi} a {ao}/{ag}")
            acc[0] = int(gg)
        if not large and not langevin:
            # the GPU adds round(a 2^32) of its binary32 a to A_{k(x)} (small steps)
            self.A_g[kx] += int(np.rint(np.float64(np.float32(ag)) * 4294967296.0))
            self.i_g[kx] += 1
        if acc[0]:
            self.px_g[chain] = py_g
            self.px_o[chain] = lum((fy[0], fy[1], fy[2]))

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

        def sgn(x):
            return 1 if x > p.alpha_star else (-1 if x < p.alpha_star else 0)

        if self.stride == 1:
            # the GPU's own update, from its own A_k
            if int(self.i_g[k]) != i_k:
                s["visits_mismatch"] += 1
                self._fail(f"epoch {self.cur_epoch} region {k}: i_k oracle {i_k} gpu {int(self.i_g[k])}")
            ahat_g = float(self.A_g[k]) / (4294967296.0 * float(i_k))
            sg_g = sgn(ahat_g)
            if result(sg_g) != lam_g:
                s["update_mismatch"] += 1
                self._fail(f"epoch {self.cur_epoch} region {k}: gpu lambda {lam_g} is not its own update "
                           f"{result(sg_g)} (alpha_hat {ahat_g})")
            if sg_g != sign[0]:
                if min(ahat, ahat_g) <= p.alpha_star <= max(ahat, ahat_g):
                    s["update_excluded"] += 1
                else:
                    s["update_mismatch"] += 1
                    self._fail(f"epoch {self.cur_epoch} region {k}: sign oracle {sign[0]} gpu {sg_g} "
                               f"alpha_hat {ahat}/{ahat_g}")
                sign[0] = sg_g
            self.A_g[k] = 0
            self.i_g[k] = 0
            return
        # a subset of the chains traced: the GPU's A_k is not known
        if result(sign[0]) == lam_g:
            return
        cands = [sg for sg in (-1, 0, 1) if result(sg) == lam_g]
        if cands and abs(ahat - p.alpha_star) <= self.a_max_rel:
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
            if self.stride == 1:
                # a quadtree split resets the statistics of the split regions
                # (on both sides: the final i_k are compared exactly); the
                # rebuilt counts follow, and must equal the oracle's elsewhere
                vis = self.ch.visits
                zero = vis == 0
                self.A_g[:len(vis)][zero] = 0
                self.i_g[:len(vis)][zero] = 0
                bad = np.flatnonzero(self.i_g[:len(vis)] != vis.astype(np.int64))
                if len(bad):
                    self.s["visits_mismatch"] += len(bad)
                    self._fail(f"epoch {e}: i_k differs in regions {bad[:8].tolist()}")
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

    def gpu_accsum(self) -> np.ndarray:
        """The GPU's A_k as rebuilt from its trace (every chain traced)."""
        return np.array([int(x) for x in self.A_g], dtype=np.uint64)

    def ok(self) -> bool:
        s = self.s
        return not (s["q_mismatch"] or s["large_mismatch"] or s["early_mismatch"] or s["f_mismatch"]
                    or s["a_mismatch"] or s["decision_mismatch"] or s["update_mismatch"]
                    or s["lambda_mismatch"] or s["visits_mismatch"] or s["proposal_mismatch"]
                    or s["kind_mismatch"])

    def counts(self) -> dict:
        """What the windows let through, for the pinned ceilings of each test."""
        return {k: self.s[k] for k in ("f_bounded", "f_excluded", "decision_excluded", "update_excluded")}

    def ok_proposals(self) -> bool:
        return not (self.s["proposal_mismatch"] or self.s["kind_mismatch"])

    def summary(self) -> str:
        return (f"{self.s} f_max_rel={self.f_max_rel:.3g} a_max_rel={self.a_max_rel:.3g} "
                f"bound_use={self.bound_use:.3g} prop_use={self.prop_use:.3g} failures={self.failures[:5]}")


def adopt_initial_states(chains, q_gpu: np.ndarray, max_adopt: int) -> int:
    """Compare the oracle's initial states with the GPU's ([D][C] words).

    Each chain takes the sample where the cumulative sum of pi over all
    bootstrap samples crosses its point; a path that binary32 and binary64
    evaluate differently shifts that sum by its rounding error, which can move
    a pick whose point lies that close to a sample boundary.  Up to
    ``max_adopt`` such chains are given the GPU's starting state (the oracle
    recomputes f itself); returns how many."""
    q_o = chains.q
    diff = np.flatnonzero(np.any(q_o != q_gpu.T, axis=1))
    if len(diff) > max_adopt:
        raise AssertionError(f"{len(diff)} initial states differ (chains {diff[:10].tolist()})")
    for c in diff:
        chains.set_state(int(c), q_gpu[:, c])
    return len(diff)
