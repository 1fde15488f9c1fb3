"""rmlt_bootstrap_noalloc: the bootstrap for callers that cannot allocate.

Some callers cannot allocate device memory when they need starting states
(inside an allocator or arena callback, or under a framework that owns the
allocator).  rmlt_bootstrap_noalloc runs the bootstrap of rmlt_init_chains
on a fixed array inside the library and writes only to the caller's
buffers.  These tests call it through the C ABI twice in a row and compare
each result with what rmlt_init_chains produced for the same parameters:
the starting states word for word, their contributions and the normaliser b
to 1e-6 relative (the tolerance of the image and normaliser checks).
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _check(scene, **params):
    import torch
    from paper_2402_08273_gb300 import rmlt
    L = rmlt.lib()
    R = rmlt.Renderer()
    R.load_scene(scene)
    R.init_chains(**params)
    ref = R.read_chain_state()
    bhat_ref = R.read_stats()["bhat"]
    p = rmlt.default_params(**params)
    cp = rmlt.ChainParams(**p)
    D, n = 2 + 5 * p["max_depth"], p["n_chains"]
    q = torch.zeros((D, n), dtype=torch.int32, device="cuda")
    f = torch.zeros((3, n), dtype=torch.float32, device="cuda")
    for _ in range(2):
        q.fill_(-1)
        f.fill_(-1.0)
        b = C.c_double(-1.0)
        st = L.rmlt_bootstrap_noalloc(R.h, C.byref(cp), C.c_void_p(q.data_ptr()), C.c_void_p(f.data_ptr()),
                                      C.byref(b))
        assert st == 0, L.rmlt_last_error()
        assert np.array_equal(q.cpu().numpy().view(np.uint32), ref["q"])
        np.testing.assert_allclose(f.cpu().numpy(), ref["f"], rtol=1e-6, atol=0)
        assert abs(b.value - bhat_ref) <= 1e-6 * abs(bhat_ref)
    R.close()


def test_noalloc_bootstrap_brute_force_scene():
    from paper_2402_08273_gb300 import scenes
    _check(scenes.cornell_box(), n_chains=256, width=64, height=64, region_px=8, max_depth=5,
           n_bootstrap=1 << 16, seed=7)


def test_noalloc_bootstrap_bvh_scene():
    from paper_2402_08273_gb300 import scenes
    _check(scenes.two_rooms(20_000, seed=2), n_chains=1000, width=128, height=96, region_px=16,
           max_depth=6, n_bootstrap=100_000, seed=3)


def test_noalloc_rejects_sizes_above_the_fixed_scratch():
    import torch
    from paper_2402_08273_gb300 import rmlt, scenes
    L = rmlt.lib()
    R = rmlt.Renderer()
    R.load_scene(scenes.cornell_box())
    p = rmlt.default_params(n_chains=64, n_bootstrap=(1 << 18) + 64)
    cp = rmlt.ChainParams(**p)
    q = torch.zeros((27, 64), dtype=torch.int32, device="cuda")
    f = torch.zeros((3, 64), dtype=torch.float32, device="cuda")
    b = C.c_double()
    assert L.rmlt_bootstrap_noalloc(R.h, C.byref(cp), C.c_void_p(q.data_ptr()), C.c_void_p(f.data_ptr()),
                                    C.byref(b)) == -1
    assert b"fixed scratch" in L.rmlt_last_error()
    # host buffers for the states are refused
    qh = np.zeros((27, 64), np.uint32)
    cp = rmlt.ChainParams(**rmlt.default_params(n_chains=64, n_bootstrap=1 << 12))
    assert L.rmlt_bootstrap_noalloc(R.h, C.byref(cp), C.c_void_p(qh.ctypes.data), C.c_void_p(f.data_ptr()),
                                    C.byref(b)) == -1
    R.close()
