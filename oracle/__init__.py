"""ctypes front end of the CPU oracle (``rmlt_oracle.c``).

TEST INFRASTRUCTURE: only the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference leg import this package.  The CUDA
library and its Python binding never import it.

The oracle is a plain binary64 restatement of Regional Adaptive Metropolis
Light Transport (Alg. 1 and Secs. 3.2, 5.2-5.4 of the paper) in primary sample
space; see the header of ``rmlt_oracle.c`` for the readings it takes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "rmlt_oracle.c"
_LIB_PATH = _HERE / "_build" / "liboracle.so"
_lib = None

CFLAGS = ["-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]


def build(force: bool = False) -> Path:
    """Compile the oracle with gcc (no FMA contraction, IEEE semantics)."""
    _LIB_PATH.parent.mkdir(exist_ok=True)
    if force or not _LIB_PATH.exists() or _LIB_PATH.stat().st_mtime < max(
            _SRC.stat().st_mtime, (_HERE / "rmlt_oracle.h").stat().st_mtime):
        tmp = _LIB_PATH.with_suffix(f".{os.getpid()}.tmp")
        subprocess.run(["gcc", *CFLAGS, str(_SRC), "-o", str(tmp), "-lm"], check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class OrParams(C.Structure):
    _fields_ = [
        ("n_chains", C.c_int32), ("width", C.c_int32), ("height", C.c_int32),
        ("region_px", C.c_int32), ("max_depth", C.c_int32), ("epoch_len", C.c_int32),
        ("L", C.c_int32), ("target_mode", C.c_int32), ("n_bootstrap", C.c_int64),
        ("seed", C.c_uint64), ("p_large", C.c_double), ("s1", C.c_double), ("s2", C.c_double),
        ("alpha_star", C.c_double), ("gamma_max", C.c_double), ("gamma_scale", C.c_double),
        ("lambda_init", C.c_double), ("lambda_min", C.c_double), ("lambda_max", C.c_double),
        ("w_floor", C.c_double), ("debug_flags", C.c_int32), ("partition", C.c_int32),
        ("qt_max_leaves", C.c_int32), ("qt_max_depth", C.c_int32), ("qt_split", C.c_int64),
        ("qt_refine", C.c_int64), ("p_mala", C.c_double), ("mala_tau", C.c_double),
        ("mala_drift_max", C.c_double), ("kernel", C.c_int32), ("dir_cells", C.c_int32),
        ("chain_first", C.c_int32), ("chains_total", C.c_int32),
    ]


MUT_HOOK = C.CFUNCTYPE(None, C.c_void_p, C.c_uint32, C.c_uint64, C.POINTER(C.c_uint32), C.c_int32,
                       C.c_int32, C.c_int32, C.c_double, C.POINTER(C.c_double), C.c_double,
                       C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_int32))
UPD_HOOK = C.CFUNCTYPE(None, C.c_void_p, C.c_int32, C.c_uint64, C.c_uint64, C.c_double,
                       C.POINTER(C.c_int32))
PROP_HOOK = C.CFUNCTYPE(None, C.c_void_p, C.c_uint32, C.c_uint64, C.c_int32, C.POINTER(C.c_uint32), C.c_int32)


def lib():
    global _lib
    if _lib is not None:
        return _lib
    L = C.CDLL(str(build()))
    P = C.POINTER
    f32p, f64p, u32p, i32p = P(C.c_float), P(C.c_double), P(C.c_uint32), P(C.c_int32)
    sig = {
        "or_philox4x32_10": (None, [u32p, u32p, u32p]),
        "or_exp2_f32": (C.c_float, [C.c_float]),
        "or_kelemen_delta": (C.c_int64, [C.c_uint32, C.c_float, C.c_float]),
        "or_truncnorm_delta": (C.c_int64, [C.c_uint32, C.c_double]),
        "or_scene_create": (C.c_void_p, [C.c_int32, f32p, C.c_int32, u32p, u32p, C.c_int32, i32p,
                                         f32p, f32p, f32p, f32p, C.c_int32]),
        "or_scene_create_toy": (C.c_void_p, [f64p]),
        "or_scene_plant_uniform_lights": (None, [C.c_void_p]),
        "or_ggx_sample_n": (None, [C.c_double, f64p, f64p, C.c_int64, f64p, f64p, C.c_int32, f64p, f64p, f64p]),
        "or_ggx_eval_n": (None, [C.c_double, f64p, f64p, C.c_int64, f64p, f64p]),
        "or_ggx_g1": (C.c_double, [C.c_double, C.c_double]),
        "or_scene_destroy": (None, [C.c_void_p]),
        "or_scene_scale": (C.c_double, [C.c_void_p]),
        "or_closest_hit": (C.c_int32, [C.c_void_p, f64p, f64p, C.c_double, C.c_double, C.c_int32,
                                       f64p, i32p, f64p]),
        "or_any_hit": (C.c_int32, [C.c_void_p, f64p, f64p, C.c_double, C.c_double, C.c_int32, f64p]),
        "or_path_eval": (C.c_int32, [C.c_void_p, C.c_int32, C.c_int32, C.c_int32, u32p, f64p, f64p,
                                     P(C.c_uint64)]),
        "or_path_eval_err": (C.c_int32, [C.c_void_p, C.c_int32, C.c_int32, C.c_int32, u32p, f64p, f64p, f64p,
                                         P(C.c_uint64)]),
        "or_ctx_create": (C.c_void_p, [C.c_void_p, P(OrParams)]),
        "or_ctx_destroy": (None, [C.c_void_p]),
        "or_set_hooks": (None, [C.c_void_p, MUT_HOOK, UPD_HOOK, C.c_void_p]),
        "or_set_prop_hook": (None, [C.c_void_p, PROP_HOOK]),
        "or_last_mala": (None, [C.c_void_p, f64p, f64p, f64p]),
        "or_init": (C.c_int32, [C.c_void_p]),
        "or_init_tables": (C.c_int32, [C.c_void_p]),
        "or_refresh_sigma": (None, [C.c_void_p]),
        "or_set_state": (C.c_int32, [C.c_void_p, C.c_uint32, u32p]),
        "or_mutate_one": (C.c_int32, [C.c_void_p, C.c_uint32, C.c_uint64]),
        "or_run_epochs": (C.c_int32, [C.c_void_p, C.c_int64]),
        "or_epoch_mutate": (C.c_int32, [C.c_void_p, P(C.c_uint64), f64p]),
        "or_epoch_update": (C.c_int32, [C.c_void_p, P(C.c_uint64), f64p]),
        "or_region_capacity": (C.c_int32, [C.c_void_p]),
        "or_read_image": (None, [C.c_void_p, f64p]),
        "or_dims": (C.c_int32, [C.c_void_p]),
        "or_regions": (C.c_int32, [C.c_void_p]),
        "or_region_of": (C.c_int32, [C.c_void_p, u32p]),
        "or_mutations_done": (C.c_uint64, [C.c_void_p]),
        "or_bhat": (C.c_double, [C.c_void_p]),
        "or_stats": (None, [C.c_void_p, P(C.c_uint64)]),
        "or_accept_prob": (C.c_double, [C.c_void_p, u32p, u32p, C.c_double, C.c_double, C.c_int32]),
        "or_quadtree": (C.c_int32, [C.c_void_p, i32p, i32p, i32p, C.c_int32]),
        "or_refine": (C.c_int32, [C.c_void_p]),
        "or_path_grad": (C.c_int32, [C.c_void_p, C.c_int32, C.c_int32, C.c_int32, u32p, f64p, f64p]),
        "or_mala_stats": (None, [C.c_void_p, P(C.c_uint64)]),
        "or_state_grad": (C.c_void_p, [C.c_void_p, C.c_uint32]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    for name in ("or_state_q", "or_state_f", "or_state_pi", "or_state_k", "or_boot_choice",
                 "or_lambda", "or_n_updates", "or_visits", "or_accsum", "or_hist", "or_hist_prev",
                 "or_weight", "or_sigma", "or_image_acc"):
        fn = getattr(L, name)
        fn.restype = C.c_void_p
        fn.argtypes = [C.c_void_p]
    _lib = L
    return L


def _ptr(a: np.ndarray, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, np.uint32)
    k = np.ascontiguousarray(key, np.uint32)
    o = np.zeros(4, np.uint32)
    lib().or_philox4x32_10(_ptr(c, C.c_uint32), _ptr(k, C.c_uint32), _ptr(o, C.c_uint32))
    return o


def exp2_f32(t: float) -> np.float32:
    return np.float32(lib().or_exp2_f32(C.c_float(t)))


def kelemen_delta(xmag: int, sigma_s2: float, log2_ratio: float) -> int:
    return int(lib().or_kelemen_delta(xmag, C.c_float(sigma_s2), C.c_float(log2_ratio)))


def truncnorm_delta(xmag: int, sigma: float) -> int:
    return int(lib().or_truncnorm_delta(xmag, float(sigma)))


def ggx_sample(alpha: float, F0, wo, bu, bv, planted: int = 0):
    """The path map's GGX continuation in the local frame n = z, for arrays of
    uniforms (bu, bv): (wi [n,3], weight [n,3], m [n,3])."""
    bu = np.ascontiguousarray(bu, np.float64).ravel()
    bv = np.ascontiguousarray(bv, np.float64).ravel()
    n = len(bu)
    F0 = np.ascontiguousarray(F0, np.float64)
    wo = np.ascontiguousarray(wo, np.float64)
    wi, w, m = np.zeros((n, 3)), np.zeros((n, 3)), np.zeros((n, 3))
    lib().or_ggx_sample_n(float(alpha), _ptr(F0, C.c_double), _ptr(wo, C.c_double), n, _ptr(bu, C.c_double),
                          _ptr(bv, C.c_double), int(planted), _ptr(wi, C.c_double), _ptr(w, C.c_double),
                          _ptr(m, C.c_double))
    return wi, w, m


def ggx_eval(alpha: float, F0, wo, wi) -> np.ndarray:
    """f_r(wo, wi) [n,3] of one GGX lobe in the local frame n = z."""
    wi = np.ascontiguousarray(wi, np.float64).reshape(-1, 3)
    F0 = np.ascontiguousarray(F0, np.float64)
    wo = np.ascontiguousarray(wo, np.float64)
    fr = np.zeros_like(wi)
    lib().or_ggx_eval_n(float(alpha), _ptr(F0, C.c_double), _ptr(wo, C.c_double), len(wi), _ptr(wi, C.c_double),
                        _ptr(fr, C.c_double))
    return fr


def ggx_g1(cos_theta: float, alpha: float) -> float:
    return float(lib().or_ggx_g1(float(cos_theta), float(alpha)))


class Scene:
    """An oracle scene built from a scene dict (see the package's scenes module)."""

    def __init__(self, scene: dict | None = None, use_bvh: bool = True, toy=None):
        L = lib()
        self.toy = toy is not None
        if toy is not None:
            self._toy = np.ascontiguousarray(toy, np.float64)
            self.h = L.or_scene_create_toy(_ptr(self._toy, C.c_double))
        else:
            self._keep = {k: np.ascontiguousarray(v) for k, v in scene.items()}
            s = self._keep
            v = np.ascontiguousarray(s["verts"], np.float32)
            t = np.ascontiguousarray(s["tris"], np.uint32)
            self._keep.update(verts=v, tris=t)
            self.h = L.or_scene_create(
                len(v), _ptr(v, C.c_float), len(t), _ptr(t, C.c_uint32),
                _ptr(np.ascontiguousarray(s["mat_id"], np.uint32), C.c_uint32), len(s["mat_type"]),
                _ptr(np.ascontiguousarray(s["mat_type"], np.int32), C.c_int32),
                _ptr(np.ascontiguousarray(s["albedo"], np.float32), C.c_float),
                _ptr(np.ascontiguousarray(s["emission"], np.float32), C.c_float),
                _ptr(np.ascontiguousarray(s["roughness"], np.float32), C.c_float),
                _ptr(np.ascontiguousarray(s["camera"], np.float32), C.c_float), int(use_bvh))
        if not self.h:
            raise ValueError("oracle rejected the scene")

    def __del__(self):
        if getattr(self, "h", None):
            lib().or_scene_destroy(self.h)
            self.h = None

    @property
    def scale(self) -> float:
        return lib().or_scene_scale(self.h)

    def plant_uniform_lights(self):
        """Tests only: a planted mistake (light triangles chosen uniformly, not by area)."""
        lib().or_scene_plant_uniform_lights(self.h)

    def closest_hit(self, o, d, tmin=0.0, tmax=float("inf"), brute=False, margin=False):
        o = np.ascontiguousarray(o, np.float64)
        d = np.ascontiguousarray(d, np.float64)
        t = C.c_double()
        tri = C.c_int32()
        m = C.c_double(float("inf"))
        hit = lib().or_closest_hit(self.h, _ptr(o, C.c_double), _ptr(d, C.c_double), tmin, tmax,
                                   int(brute), C.byref(t), C.byref(tri),
                                   C.byref(m) if margin else None)
        return bool(hit), t.value, tri.value, m.value

    def any_hit(self, o, d, tmin, tmax, brute=False):
        o = np.ascontiguousarray(o, np.float64)
        d = np.ascontiguousarray(d, np.float64)
        return bool(lib().or_any_hit(self.h, _ptr(o, C.c_double), _ptr(d, C.c_double), tmin, tmax,
                                     int(brute), None))

    def path_eval(self, q, width, height, max_depth):
        q = np.ascontiguousarray(q, np.uint32)
        f = np.zeros(3)
        m = C.c_double(float("inf"))
        cnt = np.zeros(3, np.uint64)
        ok = lib().or_path_eval(self.h, width, height, max_depth, _ptr(q, C.c_uint32),
                                _ptr(f, C.c_double), C.byref(m), _ptr(cnt, C.c_uint64))
        return f, m.value, bool(ok), int(cnt[0])

    def path_eval_err(self, q, width, height, max_depth):
        """(f, dec, ferr): the path contribution with its binary32 error model
        (decision distance in error bounds, per-channel absolute error bound)."""
        q = np.ascontiguousarray(q, np.uint32)
        f = np.zeros(3)
        e = np.zeros(3)
        dec = C.c_double(float("inf"))
        lib().or_path_eval_err(self.h, width, height, max_depth, _ptr(q, C.c_uint32), _ptr(f, C.c_double),
                               C.byref(dec), _ptr(e, C.c_double), None)
        return f, dec.value, e

    def path_grad(self, q, width, height, max_depth):
        """(f, grad log pi, status): forward-mode gradient in binary64 (status 1
        ok, 0 not differentiable here: a non-Lambertian surface or a non-finite
        path)."""
        q = np.ascontiguousarray(q, np.uint32)
        f = np.zeros(3)
        D = 2 if self.toy else 2 + 5 * max_depth
        g = np.zeros(max(D, 1))
        st = lib().or_path_grad(self.h, width, height, max_depth, _ptr(q, C.c_uint32), _ptr(f, C.c_double),
                                _ptr(g, C.c_double))
        return f, g[:D], int(st)


DEFAULT_PARAMS = dict(
    n_chains=64, width=64, height=64, region_px=8, max_depth=5, epoch_len=16, L=10,
    target_mode=0, n_bootstrap=1 << 14, seed=1, p_large=0.3, s1=1.0 / 1024.0, s2=1.0 / 64.0,
    alpha_star=0.5, gamma_max=1.0, gamma_scale=5.0, lambda_init=0.0, lambda_min=-30.0,
    lambda_max=None, w_floor=1e-3, debug_flags=0, partition=0, qt_max_leaves=4096, qt_max_depth=10,
    qt_split=5000, qt_refine=10_000_000, p_mala=0.0, mala_tau=1e-3, mala_drift_max=0.1, kernel=0,
    dir_cells=0, chain_first=0, chains_total=0,
)


def lambda_max_default(s2: float) -> float:
    """Upper clamp of lambda: sigma s2 <= 1/2, the largest offset on the torus."""
    import math
    return 2.0 * math.log(1.0 / (2.0 * s2))


def make_params(**kw) -> OrParams:
    p = dict(DEFAULT_PARAMS)
    p.update(kw)
    if p["lambda_max"] is None:
        # Kelemen: sigma s2 <= 1/2; truncated normal: sigma <= 4
        p["lambda_max"] = 2.0 * np.log(4.0) if p["kernel"] == 1 else lambda_max_default(p["s2"])
    return OrParams(**p)


class Chains:
    """The oracle's chain population (Alg. 1 over many independent chains)."""

    def __init__(self, scene: Scene, **params):
        self.scene = scene
        self.params = make_params(**params)
        self.h = lib().or_ctx_create(scene.h, C.byref(self.params))
        if not self.h:
            raise ValueError("oracle rejected the parameters")
        self.D = lib().or_dims(self.h)
        self.m = lib().or_regions(self.h)
        self.C = self.params.n_chains
        self._hooks = None

    def __del__(self):
        if getattr(self, "h", None):
            lib().or_ctx_destroy(self.h)
            self.h = None

    def _arr(self, name, ct, shape):
        addr = getattr(lib(), name)(self.h)
        n = int(np.prod(shape))
        return np.ctypeslib.as_array((ct * n).from_address(addr)).reshape(shape)

    def init(self):
        if lib().or_init(self.h) != 0:
            raise RuntimeError("or_init failed")

    def init_tables(self):
        lib().or_init_tables(self.h)

    def refresh_sigma(self):
        lib().or_refresh_sigma(self.h)

    def set_state(self, chain: int, q):
        q = np.ascontiguousarray(q, np.uint32)
        if lib().or_set_state(self.h, int(chain), _ptr(q, C.c_uint32)) != 0:
            raise ValueError("bad chain index")

    def mutate_one(self, chain: int, mut: int):
        if lib().or_mutate_one(self.h, int(chain), int(mut)) != 0:
            raise RuntimeError("or_mutate_one failed")

    def run_epochs(self, n: int):
        if lib().or_run_epochs(self.h, int(n)) != 0:
            raise RuntimeError("or_run_epochs failed")

    def exchange_buffers(self):
        """(counts, sums) arrays of one sharded epoch: [3 cap + 1] u64 and [cap] f64."""
        cap = int(lib().or_region_capacity(self.h))
        return np.zeros(3 * cap + 1, np.uint64), np.zeros(cap, np.float64)

    def epoch_mutate(self, counts: np.ndarray, sums: np.ndarray):
        """E mutations of this context's chains; what they added to the region
        tables goes to `counts` / `sums` (see or_epoch_mutate)."""
        if lib().or_epoch_mutate(self.h, _ptr(counts, C.c_uint64), _ptr(sums, C.c_double)) != 0:
            raise RuntimeError("or_epoch_mutate: not initialised, or an update is due")

    def epoch_update(self, counts: np.ndarray, sums: np.ndarray):
        """The epoch boundary from the additions summed over every context."""
        counts = np.ascontiguousarray(counts, np.uint64)
        sums = np.ascontiguousarray(sums, np.float64)
        if lib().or_epoch_update(self.h, _ptr(counts, C.c_uint64), _ptr(sums, C.c_double)) != 0:
            raise RuntimeError("or_epoch_update: or_epoch_mutate first")

    def set_hooks(self, mut_fn=None, upd_fn=None, prop_fn=None):
        mh = MUT_HOOK(mut_fn) if mut_fn else MUT_HOOK()
        uh = UPD_HOOK(upd_fn) if upd_fn else UPD_HOOK()
        ph = PROP_HOOK(prop_fn) if prop_fn else PROP_HOOK()
        self._hooks = (mh, uh, ph)
        lib().or_set_hooks(self.h, mh, uh, None)
        lib().or_set_prop_hook(self.h, ph)

    def last_mala(self):
        """(m_x [D], z [D], tau_x, S) of the last Langevin move (see or_last_mala)."""
        m = np.zeros(max(self.D, 1))
        z = np.zeros(max(self.D, 1))
        o = np.zeros(2)
        lib().or_last_mala(self.h, _ptr(m, C.c_double), _ptr(z, C.c_double), _ptr(o, C.c_double))
        return m[:self.D], z[:self.D], float(o[0]), float(o[1])

    def image(self) -> np.ndarray:
        out = np.zeros((self.params.height, self.params.width, 3))
        lib().or_read_image(self.h, _ptr(out, C.c_double))
        return out

    def accept_prob(self, qx, qy, pi_x, pi_y, large=False) -> float:
        qx = np.ascontiguousarray(qx, np.uint32)
        qy = np.ascontiguousarray(qy, np.uint32)
        return float(lib().or_accept_prob(self.h, _ptr(qx, C.c_uint32), _ptr(qy, C.c_uint32),
                                          float(pi_x), float(pi_y), int(large)))

    def quadtree(self):
        """(child [nodes,4], leaf [nodes], depth [nodes]) of the quadtree partition."""
        cap = 4 * self.params.qt_max_leaves // 3 + 8
        child = np.zeros((cap, 4), np.int32)
        leaf = np.zeros(cap, np.int32)
        depth = np.zeros(cap, np.int32)
        n = lib().or_quadtree(self.h, _ptr(child, C.c_int32), _ptr(leaf, C.c_int32), _ptr(depth, C.c_int32), cap)
        return child[:n], leaf[:n], depth[:n]

    def refine(self):
        if lib().or_refine(self.h) != 0:
            raise RuntimeError("or_refine needs an initialised quadtree context")

    @property
    def n_regions(self) -> int:
        return int(lib().or_regions(self.h))

    def region_of(self, q) -> int:
        q = np.ascontiguousarray(q, np.uint32)
        return lib().or_region_of(self.h, _ptr(q, C.c_uint32))

    @property
    def mutations_done(self) -> int:
        return int(lib().or_mutations_done(self.h))

    @property
    def bhat(self) -> float:
        return float(lib().or_bhat(self.h))

    def stats(self) -> dict:
        o = np.zeros(8, np.uint64)
        lib().or_stats(self.h, _ptr(o, C.c_uint64))
        keys = ("mutations", "accepted", "large", "small", "early_reject", "invalid", "rays", "boot")
        out = {k: int(v) for k, v in zip(keys, o)}
        m = np.zeros(2, np.uint64)
        lib().or_mala_stats(self.h, _ptr(m, C.c_uint64))
        out["mala"], out["mala_accepted"] = int(m[0]), int(m[1])
        return out

    def state_grad(self, chain: int):
        p = lib().or_state_grad(self.h, chain)
        if not p:
            return None
        return np.ctypeslib.as_array(C.cast(p, C.POINTER(C.c_double)), shape=(self.D,)).copy()

    # live views of the oracle's state arrays
    @property
    def q(self):
        return self._arr("or_state_q", C.c_uint32, (self.C, self.D))

    @property
    def f(self):
        return self._arr("or_state_f", C.c_double, (self.C, 3))

    @property
    def pi(self):
        return self._arr("or_state_pi", C.c_double, (self.C,))

    @property
    def k(self):
        return self._arr("or_state_k", C.c_int32, (self.C,))

    @property
    def boot_choice(self):
        return self._arr("or_boot_choice", C.c_int64, (self.C,))

    @property
    def lam(self):
        return self._arr("or_lambda", C.c_double, (self.n_regions,))

    @property
    def n_updates(self):
        return self._arr("or_n_updates", C.c_int64, (self.n_regions,))

    @property
    def visits(self):
        return self._arr("or_visits", C.c_uint64, (self.n_regions,))

    @property
    def accsum(self):
        return self._arr("or_accsum", C.c_uint64, (self.n_regions,))

    @property
    def hist(self):
        return self._arr("or_hist", C.c_uint64, (self.n_regions,))

    @property
    def hist_since_pass(self):
        """h_k minus its value at the last quadtree refinement pass."""
        h = self._arr("or_hist", C.c_uint64, (self.n_regions,))
        hp = self._arr("or_hist_prev", C.c_uint64, (self.n_regions,))
        return h - hp

    @property
    def weight(self):
        return self._arr("or_weight", C.c_double, (self.n_regions,))

    @property
    def sigma(self):
        return self._arr("or_sigma", C.c_float, (self.n_regions,))

    @property
    def image_acc(self):
        return self._arr("or_image_acc", C.c_double, (self.params.height, self.params.width, 3))
