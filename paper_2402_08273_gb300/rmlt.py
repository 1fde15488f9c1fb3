"""Python binding of librmlt (the C ABI in include/rmlt.h).

Argument marshalling only: every step of the method runs in the CUDA library.
PyTorch provides device memory (its caching allocator is installed as the
library's allocator) and the CUDA stream.  There is no CPU fallback: if the
library cannot be built or loaded, or no GPU is present, the calls raise.
"""
from __future__ import annotations

import ctypes as C
from pathlib import Path

import numpy as np

from . import _build

RMLT_OK = 0
STATUS = {0: "RMLT_OK", -1: "RMLT_E_INVALID_ARG", -2: "RMLT_E_INVALID_SCENE", -3: "RMLT_E_OOM",
          -4: "RMLT_E_CUDA", -5: "RMLT_E_STATE", -7: "RMLT_E_OVERFLOW", -8: "RMLT_E_IO"}
LAMBERT, GGX = 0, 1
TARGET_PLAIN, TARGET_REGION_WEIGHTED = 0, 1
KERNEL_KELEMEN, KERNEL_TRUNCNORM = 0, 1
MAX_DEPTH = 12


class RmltError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Material(C.Structure):
    _fields_ = [("type", C.c_int32), ("albedo", C.c_float * 3), ("emission", C.c_float * 3),
                ("roughness", C.c_float)]


class Camera(C.Structure):
    _fields_ = [("pos", C.c_float * 3), ("look_at", C.c_float * 3), ("up", C.c_float * 3),
                ("vfov_deg", C.c_float)]


class SceneDesc(C.Structure):
    _fields_ = [("n_verts", C.c_int32), ("verts", C.POINTER(C.c_float)), ("n_tris", C.c_int32),
                ("tris", C.POINTER(C.c_uint32)), ("mat_id", C.POINTER(C.c_uint32)),
                ("n_mats", C.c_int32), ("mats", C.POINTER(Material)), ("camera", Camera),
                ("brute_force_max", C.c_int32), ("bvh_width", C.c_int32)]


class ChainParams(C.Structure):
    _fields_ = [("n_chains", C.c_int32), ("width", C.c_int32), ("height", C.c_int32),
                ("region_px", C.c_int32), ("max_depth", C.c_int32), ("epoch_len", C.c_int32),
                ("L", C.c_int32), ("target_mode", C.c_int32), ("n_bootstrap", C.c_int64),
                ("seed", C.c_uint64), ("p_large", C.c_double), ("s1", C.c_double),
                ("s2", C.c_double), ("alpha_star", C.c_double), ("gamma_max", C.c_double),
                ("gamma_scale", C.c_double), ("lambda_init", C.c_double),
                ("lambda_min", C.c_double), ("lambda_max", C.c_double), ("w_floor", C.c_double),
                ("partition", C.c_int32), ("qt_max_leaves", C.c_int32), ("qt_max_depth", C.c_int32),
                ("qt_pad_", C.c_int32), ("qt_split", C.c_int64), ("qt_refine", C.c_int64),
                ("p_mala", C.c_double), ("mala_tau", C.c_double), ("mala_drift_max", C.c_double),
                ("kernel", C.c_int32), ("dir_cells", C.c_int32), ("chain_first", C.c_int32),
                ("chains_total", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [("mutations", C.c_uint64), ("accepted", C.c_uint64), ("large", C.c_uint64),
                ("small", C.c_uint64), ("early_reject", C.c_uint64), ("invalid_paths", C.c_uint64),
                ("rays", C.c_uint64), ("stack_overflow", C.c_uint64), ("epochs", C.c_uint64),
                ("bhat", C.c_double), ("n_regions", C.c_int32), ("dims", C.c_int32),
                ("node_visits", C.c_uint64), ("tri_tests", C.c_uint64), ("sched", C.c_uint64 * 6),
                ("cycles", C.c_uint64 * 5), ("waves", C.c_uint64), ("wave_limit_hits", C.c_uint64),
                ("mala", C.c_uint64), ("mala_accepted", C.c_uint64), ("boot_overflow", C.c_uint64),
                ("node_bytes", C.c_uint32), ("pad_", C.c_uint32)]


TRACE_DTYPE = np.dtype([("f", np.float32, 3), ("a", np.float32), ("qhash", np.uint32),
                        ("flags", np.uint32)])
assert TRACE_DTYPE.itemsize == 24

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)

# (name, restype, argtypes) of every function declared in include/rmlt.h
_P = C.POINTER
_SIGS = [
    ("rmlt_abi_version", C.c_int, []),
    ("rmlt_last_error", C.c_char_p, []),
    ("rmlt_create", C.c_int, [_P(C.c_void_p), C.c_int, C.c_void_p]),
    ("rmlt_set_allocator", C.c_int, [C.c_void_p, ALLOC_FN, FREE_FN, C.c_void_p]),
    ("rmlt_load_scene", C.c_int, [C.c_void_p, _P(SceneDesc)]),
    ("rmlt_load_toy_integrand", C.c_int, [C.c_void_p, _P(C.c_double)]),
    ("rmlt_init_chains", C.c_int, [C.c_void_p, _P(ChainParams)]),
    ("rmlt_step", C.c_int, [C.c_void_p, C.c_uint64]),
    ("rmlt_exchange_size", C.c_int, [C.c_void_p, _P(C.c_int64), _P(C.c_int64)]),
    ("rmlt_epoch_mutate", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    ("rmlt_epoch_update", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    ("rmlt_read_params", C.c_int, [C.c_void_p, _P(ChainParams)]),
    ("rmlt_set_wave_limit", C.c_int, [C.c_void_p, C.c_uint32]),
    ("rmlt_set_trace_leaf_batch", C.c_int, [C.c_void_p, C.c_int]),
    ("rmlt_set_node_format", C.c_int, [C.c_void_p, C.c_int]),
    ("rmlt_read_image", C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    ("rmlt_read_region_hist", C.c_int, [C.c_void_p, C.c_void_p]),
    ("rmlt_read_region_params", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                          C.c_void_p, C.c_void_p]),
    ("rmlt_read_chain_state", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("rmlt_read_quadtree", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32,
                                     _P(C.c_int32)]),
    ("rmlt_read_stats", C.c_int, [C.c_void_p, _P(Stats)]),
    ("rmlt_set_trace", C.c_int, [C.c_void_p, C.c_void_p, C.c_uint64, C.c_void_p, C.c_uint64,
                                 C.c_uint32]),
    ("rmlt_set_trace_words", C.c_int, [C.c_void_p, C.c_void_p, C.c_uint64]),
    ("rmlt_memory_usage", C.c_int, [C.c_void_p, _P(C.c_uint64)]),
    ("rmlt_probe_peaks", C.c_int, [C.c_int, C.c_void_p, _P(C.c_double), _P(C.c_double)]),
    ("rmlt_path_grad", C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("rmlt_read_chain_grad", C.c_int, [C.c_void_p, C.c_void_p]),
    ("rmlt_batch_create", C.c_int, [_P(C.c_void_p), _P(C.c_void_p), C.c_int]),
    ("rmlt_batch_set_order", C.c_int, [C.c_void_p, _P(C.c_int)]),
    ("rmlt_batch_set_shape", C.c_int, [C.c_void_p, C.c_int, C.c_int]),
    ("rmlt_batch_step", C.c_int, [C.c_void_p, C.c_uint64]),
    ("rmlt_batch_destroy", None, [C.c_void_p]),
    ("rmlt_set_work_counters", C.c_int, [C.c_void_p, C.c_int]),
    ("rmlt_record_paths", C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]),
    ("rmlt_walk_rays_host", C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p]),
    ("rmlt_set_tuning", C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int]),
    ("rmlt_set_wavefront", C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int]),
    ("rmlt_bootstrap_noalloc", C.c_int, [C.c_void_p, _P(ChainParams), C.c_void_p, C.c_void_p,
                                         C.c_void_p]),
    ("rmlt_save", C.c_int, [C.c_void_p, C.c_char_p]),
    ("rmlt_restore", C.c_int, [C.c_void_p, C.c_char_p]),
    ("rmlt_synchronize", C.c_int, [C.c_void_p]),
    ("rmlt_destroy", None, [C.c_void_p]),
]

_lib = None


def library_path() -> Path:
    return _build.LIB


def lib(build: bool = True):
    """Load librmlt.so (building it in-tree first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build else _build.LIB
    L = C.CDLL(str(path))
    for name, res, args in _SIGS:
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _check(st: int):
    if st != RMLT_OK:
        raise RmltError(st, lib().rmlt_last_error().decode(errors="replace"))


def default_params(**kw) -> dict:
    """Chain parameters: Sec. 7.1 values (L = 10, gamma_max = 1, gamma_scale = 5,
    lambda_min = -30, alpha* = 0.5) with Kelemen's s1 = 1/1024, s2 = 1/64.
    lambda_max = 0 lets the library choose its default."""
    p = dict(n_chains=64, width=64, height=64, region_px=8, max_depth=5, epoch_len=16, L=10,
             target_mode=TARGET_PLAIN, n_bootstrap=1 << 16, seed=1, p_large=0.3, s1=1 / 1024,
             s2=1 / 64, alpha_star=0.5, gamma_max=1.0, gamma_scale=5.0, lambda_init=0.0,
             lambda_min=-30.0, lambda_max=0.0, w_floor=1e-3, partition=0, qt_max_leaves=4096,
             qt_max_depth=10, qt_pad_=0, qt_split=5000, qt_refine=10_000_000, p_mala=0.0, mala_tau=1e-3,
             mala_drift_max=0.1, kernel=KERNEL_KELEMEN, dir_cells=0, chain_first=0, chains_total=0)
    p.update(kw)
    if p["lambda_max"] is None:
        p["lambda_max"] = 0.0
    return p


def _ptr(x):
    """Device pointer of a torch tensor, or host pointer of a numpy array."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return C.c_void_p(x.data_ptr())
    return C.c_void_p(x.ctypes.data)


class Renderer:
    """One rmlt context: a scene, a population of chains and their region tables."""

    def __init__(self, device: int = 0, stream=None, torch_allocator: bool = True):
        import torch
        if not torch.cuda.is_available():
            raise RmltError(-4, "no CUDA device: librmlt has no CPU fallback")
        self._torch = torch
        self.device = device
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        L = lib()
        h = C.c_void_p()
        _check(L.rmlt_create(C.byref(h), device, C.c_void_p(self.stream.cuda_stream)))
        self.h = h
        self._keep = []
        if torch_allocator:
            dev, strm = device, self.stream

            def _alloc(user, nbytes, stream_ptr):
                try:
                    return torch.cuda.caching_allocator_alloc(int(nbytes), dev, strm)
                except Exception:   # out of memory: the library reports RMLT_E_OOM
                    return None

            def _free(user, ptr, stream_ptr):
                torch.cuda.caching_allocator_delete(ptr)

            self._alloc_cb = ALLOC_FN(_alloc)
            self._free_cb = FREE_FN(_free)
            _check(L.rmlt_set_allocator(self.h, self._alloc_cb, self._free_cb, None))
        self.params = None
        self.D = self.m = None

    # -- lifecycle -----------------------------------------------------------
    def close(self):
        if getattr(self, "h", None):
            lib().rmlt_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- scene ---------------------------------------------------------------
    NODE_FORMATS = {"auto": 0, "float": 1, "quantised": 2}

    def load_scene(self, scene: dict, brute_force_max: int = 0, bvh_width: int = 0, node_format: str = "auto"):
        """node_format: the BVH4 node layout, "float" (128-byte nodes),
        "quantised" (64-byte nodes) or "auto" (quantised for scenes whose
        binary32 nodes and triangles exceed 48 MB)."""
        _check(lib().rmlt_set_node_format(self.h, self.NODE_FORMATS[node_format]))
        v = np.ascontiguousarray(scene["verts"], np.float32)
        t = np.ascontiguousarray(scene["tris"], np.uint32)
        mid = np.ascontiguousarray(scene["mat_id"], np.uint32)
        nm = len(scene["mat_type"])
        mats = (Material * nm)()
        for i in range(nm):
            mats[i].type = int(scene["mat_type"][i])
            for a in range(3):
                mats[i].albedo[a] = float(scene["albedo"][i][a])
                mats[i].emission[a] = float(scene["emission"][i][a])
            mats[i].roughness = float(scene["roughness"][i])
        cam = np.asarray(scene["camera"], np.float32)
        camera = Camera((C.c_float * 3)(*cam[0:3]), (C.c_float * 3)(*cam[3:6]),
                        (C.c_float * 3)(*cam[6:9]), float(cam[9]))
        desc = SceneDesc(len(v), v.ctypes.data_as(_P(C.c_float)), len(t),
                         t.ctypes.data_as(_P(C.c_uint32)), mid.ctypes.data_as(_P(C.c_uint32)), nm,
                         mats, camera, int(brute_force_max), int(bvh_width))
        _check(lib().rmlt_load_scene(self.h, C.byref(desc)))
        self.params = None

    def load_toy_integrand(self, params):
        p = np.ascontiguousarray(params, np.float64)
        _check(lib().rmlt_load_toy_integrand(self.h, p.ctypes.data_as(_P(C.c_double))))
        self.params = None

    # -- chains --------------------------------------------------------------
    def init_chains(self, **kw):
        cp = ChainParams(**default_params(**kw))
        _check(lib().rmlt_init_chains(self.h, C.byref(cp)))
        self._read_params()

    def _read_params(self):
        """The parameters in effect (defaults resolved by the library) and the sizes they fix."""
        cp = ChainParams()
        _check(lib().rmlt_read_params(self.h, C.byref(cp)))
        p = {name: getattr(cp, name) for name, _ in ChainParams._fields_}
        self.params = p
        self.D = 2 + 5 * p["max_depth"]
        nx = -(-p["width"] // p["region_px"])
        ny = -(-p["height"] // p["region_px"])
        g = p["dir_cells"] if p["dir_cells"] > 1 else 1
        self.m = p["qt_max_leaves"] if p["partition"] == 1 else nx * ny * g * g   # region table capacity

    def step(self, n_mutations: int):
        _check(lib().rmlt_step(self.h, int(n_mutations)))

    # -- sharded stepping (one epoch at a time around a sum over contexts) ---
    def exchange_buffers(self):
        """Two device tensors for rmlt_epoch_mutate / rmlt_epoch_update: the
        region counts (int64 holding u64 bits) and the per-region sums."""
        torch = self._torch
        nc, ns = C.c_int64(), C.c_int64()
        _check(lib().rmlt_exchange_size(self.h, C.byref(nc), C.byref(ns)))
        dev = torch.device("cuda", self.device)
        return (torch.zeros(nc.value, dtype=torch.int64, device=dev),
                torch.zeros(ns.value, dtype=torch.float64, device=dev))

    def epoch_mutate(self, counts, sums):
        _check(lib().rmlt_epoch_mutate(self.h, _ptr(counts), _ptr(sums)))

    def epoch_update(self, counts, sums):
        _check(lib().rmlt_epoch_update(self.h, _ptr(counts), _ptr(sums)))

    def set_trace_leaf_batch(self, leaf_batch: int = 8):
        _check(lib().rmlt_set_trace_leaf_batch(self.h, int(leaf_batch)))

    def set_wave_limit(self, waves: int = 0):
        _check(lib().rmlt_set_wave_limit(self.h, int(waves)))

    def synchronize(self):
        _check(lib().rmlt_synchronize(self.h))

    # -- read-out ------------------------------------------------------------
    def _require_chains(self):
        # before rmlt_init_chains the sizes are unknown: let the library report the state error
        if self.params is None:
            dummy = np.zeros(1, np.uint64)
            _check(lib().rmlt_read_region_hist(self.h, _ptr(dummy)))

    def read_image(self, normalized: bool = True, out=None):
        """[H, W, 3] float64: numpy (host) unless `out` is given (host array or CUDA tensor)."""
        self._require_chains()
        if out is None:
            out = np.zeros((self.params["height"], self.params["width"], 3), np.float64)
        _check(lib().rmlt_read_image(self.h, _ptr(out), int(normalized)))
        return out

    def n_regions(self) -> int:
        """Current number of regions (grows with a quadtree partition)."""
        return int(self.read_stats()["n_regions"])

    def read_quadtree(self):
        """(child [nodes,4], leaf [nodes], depth [nodes]) of the quadtree partition."""
        cap = 4 * self.params["qt_max_leaves"] // 3 + 8
        child = np.zeros((cap, 4), np.int32)
        leaf = np.zeros(cap, np.int32)
        depth = np.zeros(cap, np.int32)
        n = C.c_int32()
        _check(lib().rmlt_read_quadtree(self.h, _ptr(child), _ptr(leaf), _ptr(depth), cap, C.byref(n)))
        return child[:n.value], leaf[:n.value], depth[:n.value]

    def read_region_hist(self, out=None):
        self._require_chains()
        if out is None:
            out = np.zeros(self.n_regions(), np.uint64)
        _check(lib().rmlt_read_region_hist(self.h, _ptr(out)))
        return out

    def read_region_params(self) -> dict:
        self._require_chains()
        m = self.n_regions()
        lam = np.zeros(m)
        n = np.zeros(m, np.int64)
        i = np.zeros(m, np.uint64)
        A = np.zeros(m, np.uint64)
        w = np.zeros(m)
        _check(lib().rmlt_read_region_params(self.h, _ptr(lam), _ptr(n), _ptr(i), _ptr(A), _ptr(w)))
        return {"lambda": lam, "n": n, "i": i, "A": A, "w": w}

    def read_chain_state(self) -> dict:
        self._require_chains()
        Cn = self.params["n_chains"]
        q = np.zeros((self.D, Cn), np.uint32)
        f = np.zeros((3, Cn), np.float32)
        k = np.zeros(Cn, np.int32)
        _check(lib().rmlt_read_chain_state(self.h, _ptr(q), _ptr(f), _ptr(k)))
        return {"q": q, "f": f, "k": k}

    def read_stats(self) -> dict:
        s = Stats()
        _check(lib().rmlt_read_stats(self.h, C.byref(s)))
        d = {name: getattr(s, name) for name, _ in Stats._fields_}
        d["sched"] = list(d["sched"])
        d["cycles"] = list(d["cycles"])
        return d

    def set_tuning(self, batch_shade: int = 12, batch_setup: int = 10, large_ahead: bool = False,
                   adaptive_batch: bool = False, wavefront: bool = False):
        flags = (1 if large_ahead else 0) | (2 if adaptive_batch else 0) | (4 if wavefront else 0)
        _check(lib().rmlt_set_tuning(self.h, int(batch_shade), int(batch_setup), flags))

    def set_wavefront(self, trace_ctas_per_sm: int = 0, setup_ctas_per_sm: int = 0, refill_lanes: int = 8,
                      host_loop: bool = False, short_stack: bool = False):
        flags = (1 if host_loop else 0) | (2 if short_stack else 0)
        _check(lib().rmlt_set_wavefront(self.h, int(trace_ctas_per_sm), int(setup_ctas_per_sm),
                                        int(refill_lanes), flags))

    def read_chain_grad(self) -> np.ndarray:
        """grad log pi of the current states, [D, n_chains] (Langevin runs)."""
        self._require_chains()
        g = np.zeros((self.D, self.params["n_chains"]), np.float32)
        _check(lib().rmlt_read_chain_grad(self.h, _ptr(g)))
        return g

    def path_grad(self, q, want_f: bool = False):
        """(log pi [n], grad [D, n], f [3, n] or None) at primary-sample words
        q [D, n] (a CUDA tensor of int32 / uint32 bits), by the adjoint kernel."""
        torch = self._torch
        if not (torch.is_tensor(q) and q.is_cuda and q.dim() == 2 and q.shape[0] == self.D):
            raise RmltError(-1, f"q must be a CUDA tensor [D={self.D}, n]")
        q = q.to(torch.int32).contiguous()
        n = q.shape[1]
        dev = q.device
        logpi = torch.empty(n, dtype=torch.float32, device=dev)
        grad = torch.empty((self.D, n), dtype=torch.float32, device=dev)
        f = torch.empty((3, n), dtype=torch.float32, device=dev) if want_f else None
        with torch.cuda.stream(self.stream):
            _check(lib().rmlt_path_grad(self.h, C.c_void_p(q.data_ptr()), n,
                                        C.c_void_p(f.data_ptr() if f is not None else 0),
                                        C.c_void_p(logpi.data_ptr()), C.c_void_p(grad.data_ptr())))
        return logpi, grad, f

    def record_paths(self, q):
        """(rays [n, R, 8] float32, work [n, R, 4] uint32) on the host for the
        paths of points q (a CUDA int32 tensor [D, n]; R = 2 max_depth): every
        ray the chain kernel's path code casts, and its traversal's result and
        work (hit triangle, distance bits, nodes visited, triangles tested)."""
        torch = self._torch
        q = q.to(torch.int32).contiguous()
        n = q.shape[1]
        R = 2 * self.params["max_depth"]
        rays = torch.empty((n, R, 8), dtype=torch.float32, device=q.device)
        work = torch.empty((n, R, 4), dtype=torch.int32, device=q.device)
        _check(lib().rmlt_record_paths(self.h, _ptr(q), n, _ptr(rays), _ptr(work)))
        self.synchronize()
        return rays.cpu().numpy(), work.cpu().numpy().view(np.uint32)

    def walk_rays_host(self, rays: np.ndarray) -> np.ndarray:
        """The reference host traversal of ray records [..., 8] through the
        uploaded BVH: [..., 4] uint32 (hit triangle, distance bits, nodes, triangles)."""
        r = np.ascontiguousarray(rays, np.float32)
        n = r.size // 8
        out = np.zeros(r.shape[:-1] + (4,), np.uint32)
        _check(lib().rmlt_walk_rays_host(self.h, _ptr(r), n, _ptr(out)))
        return out

    def set_work_counters(self, enable: bool):
        _check(lib().rmlt_set_work_counters(self.h, int(enable)))

    def memory_usage(self) -> int:
        b = C.c_uint64()
        _check(lib().rmlt_memory_usage(self.h, C.byref(b)))
        return int(b.value)

    # -- test instrument -----------------------------------------------------
    def set_trace(self, records=None, lambdas=None, chain_stride: int = 1):
        """records: CUDA uint8 tensor of n * 24 bytes; lambdas: CUDA float64 tensor."""
        if records is None:
            _check(lib().rmlt_set_trace(self.h, None, 0, None, 0, 1))
            return
        cap = records.numel() * records.element_size() // TRACE_DTYPE.itemsize
        lcap = lambdas.numel() if lambdas is not None else 0
        _check(lib().rmlt_set_trace(self.h, _ptr(records), cap, _ptr(lambdas), lcap, chain_stride))

    def set_trace_words(self, words=None):
        """words: CUDA int32 tensor with room for D words per trace record (or None)."""
        _check(lib().rmlt_set_trace_words(self.h, _ptr(words), words.numel() if words is not None else 0))

    # -- checkpoint ----------------------------------------------------------
    def save(self, path):
        _check(lib().rmlt_save(self.h, str(path).encode()))

    def restore(self, path):
        _check(lib().rmlt_restore(self.h, str(path).encode()))
        self._read_params()


def u_to_words(u):
    """Primary-sample coordinates u in [0, 1) (a tensor [..]) as the 32-bit
    words the library takes (u = q 2^-32, floor), as int32 bits."""
    import torch
    q = torch.floor(u.detach().to(torch.float64) * 4294967296.0).clamp_(0, 4294967295.0).to(torch.int64)
    return torch.where(q >= 2 ** 31, q - 2 ** 32, q).to(torch.int32)


def _path_log_pi_function():
    import torch

    class PathLogPi(torch.autograd.Function):
        """log pi(u) of the path map with its gradient from the adjoint kernel
        (rmlt_path_grad): forward(u [n, D] in [0, 1), renderer) -> [n]."""

        @staticmethod
        def forward(ctx, u, renderer):
            q = u_to_words(u).t().contiguous()
            logpi, grad, _ = renderer.path_grad(q)
            renderer.stream.synchronize()
            ctx.save_for_backward(grad)
            return logpi.to(u.dtype)

        @staticmethod
        def backward(ctx, grad_out):
            (grad,) = ctx.saved_tensors
            return grad_out[:, None] * grad.t().to(grad_out.dtype), None

    return PathLogPi


_PLP = None


def path_log_pi(u, renderer):
    """Differentiable log pi(u): torch.autograd.Function around the adjoint
    kernel.  u: CUDA tensor [n, D] of primary-sample coordinates in [0, 1)."""
    global _PLP
    if _PLP is None:
        _PLP = _path_log_pi_function()
    return _PLP.apply(u, renderer)


class Batch:
    """Several renderers advanced together (rmlt_batch_*): one chain-kernel
    launch and one region-update launch per epoch cover every member."""

    def __init__(self, renderers):
        self.members = list(renderers)
        arr = (C.c_void_p * len(self.members))(*[r.h for r in self.members])
        h = C.c_void_p()
        _check(lib().rmlt_batch_create(C.byref(h), arr, len(self.members)))
        self.h = h

    def set_order(self, order):
        arr = (C.c_int * len(self.members))(*[int(i) for i in order])
        _check(lib().rmlt_batch_set_order(self.h, arr))

    def set_shape(self, ctas_per_sm: int = 4, branches: bool = False):
        _check(lib().rmlt_batch_set_shape(self.h, int(ctas_per_sm), 1 if branches else 0))

    def step(self, n_mutations: int):
        _check(lib().rmlt_batch_step(self.h, int(n_mutations)))

    def close(self):
        if getattr(self, "h", None):
            lib().rmlt_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def trace_to_numpy(records_tensor) -> np.ndarray:
    """View a trace buffer (CUDA uint8 tensor) as structured records on the host."""
    raw = records_tensor.cpu().numpy().view(np.uint8)
    return raw[: (raw.size // TRACE_DTYPE.itemsize) * TRACE_DTYPE.itemsize].view(TRACE_DTYPE)
