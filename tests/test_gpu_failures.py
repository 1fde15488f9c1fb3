"""Failure paths of the C ABI, exercised on the host side without any GPU
fault: an allocator that returns NULL, truncated and corrupted checkpoints,
the wavefront form's wave limit, and the library's own parameter defaults."""
import ctypes as C
import math
import struct

import numpy as np
import pytest

from paper_2402_08273_gb300 import scenes as S

pytestmark = pytest.mark.gpu


class _FlakyAllocator:
    """torch's caching allocator behind a switch that makes it return NULL."""

    def __init__(self):
        import torch
        from paper_2402_08273_gb300 import rmlt
        self.fail = False
        self.live = {}

        def alloc(user, nbytes, stream):
            if self.fail:
                return None
            t = torch.empty(int(nbytes), dtype=torch.uint8, device="cuda")
            self.live[t.data_ptr()] = t
            return t.data_ptr()

        def free(user, ptr, stream):
            self.live.pop(ptr, None)

        self.a = rmlt.ALLOC_FN(alloc)
        self.f = rmlt.FREE_FN(free)


def test_allocator_null_leaves_context_unchanged():
    from paper_2402_08273_gb300 import rmlt
    L = rmlt.lib()
    R = rmlt.Renderer(torch_allocator=False)
    fa = _FlakyAllocator()
    assert L.rmlt_set_allocator(R.h, fa.a, fa.f, None) == 0
    R.load_scene(S.cornell_box())
    R.init_chains(n_chains=64, n_bootstrap=1 << 10, seed=2)
    R.step(32)
    before = R.read_chain_state()["q"].copy()
    hist = R.read_region_hist().copy()
    fa.fail = True
    with pytest.raises(rmlt.RmltError) as e:
        R.load_scene(S.two_rooms(20_000, seed=1))
    assert e.value.status == -3
    with pytest.raises(rmlt.RmltError) as e:
        R.init_chains(n_chains=128, n_bootstrap=1 << 10, seed=3)
    assert e.value.status == -3
    # the scene and chains from before are intact and keep working
    assert np.array_equal(R.read_chain_state()["q"], before)
    assert np.array_equal(R.read_region_hist(), hist)
    fa.fail = False
    R.step(16)
    assert R.read_stats()["mutations"] == 48
    R.close()


def _fnv64(data: bytes, h: int = 1469598103934665603) -> int:
    for b in data:
        h = ((h ^ b) * 1099511628211) & 0xFFFFFFFFFFFFFFFF
    return h


def _header_size():
    from paper_2402_08273_gb300 import rmlt
    # magic 8, abi + pad 8, scene hash 8, params, mut, epochs, n_boot, since_refine, payload, checksum
    return 24 + C.sizeof(rmlt.ChainParams) + 6 * 8


def test_checkpoint_truncated_corrupted_and_bad_index(tmp_path):
    from paper_2402_08273_gb300 import rmlt
    R = rmlt.Renderer()
    R.load_scene(S.cornell_box())
    R.init_chains(n_chains=64, n_bootstrap=1 << 10, seed=4)
    R.step(32)
    path = tmp_path / "ck.bin"
    R.save(path)
    raw = path.read_bytes()
    hs = _header_size()
    # truncated: an I/O error
    (tmp_path / "trunc.bin").write_bytes(raw[:-100])
    with pytest.raises(rmlt.RmltError) as e:
        R.restore(tmp_path / "trunc.bin")
    assert e.value.status == -8
    (tmp_path / "short.bin").write_bytes(raw[:40])
    with pytest.raises(rmlt.RmltError) as e:
        R.restore(tmp_path / "short.bin")
    assert e.value.status == -8
    # one flipped bit in the payload: the checksum catches it
    bad = bytearray(raw)
    bad[hs + 1000] ^= 0x10
    (tmp_path / "flip.bin").write_bytes(bytes(bad))
    with pytest.raises(rmlt.RmltError) as e:
        R.restore(tmp_path / "flip.bin")
    assert e.value.status == -1 and "checksum" in str(e.value)
    # a region index out of range with a valid checksum: the host-side index
    # check refuses it before anything is launched
    D, Cn = R.D, 64
    k_off = hs + Cn * D * 4 + Cn * 12 + Cn * 4          # q, f, pi, then k
    bad = bytearray(raw)
    bad[k_off:k_off + 4] = struct.pack("<i", 10_000)
    bad[hs - 8:hs] = b"\0" * 8
    bad[hs - 8:hs] = struct.pack("<Q", _fnv64(bytes(bad)))
    (tmp_path / "index.bin").write_bytes(bytes(bad))
    with pytest.raises(rmlt.RmltError) as e:
        R.restore(tmp_path / "index.bin")
    assert e.value.status == -1 and "region" in str(e.value)
    # the context is unchanged after every refusal, and the intact file restores
    q = R.read_chain_state()["q"].copy()
    R.restore(path)
    assert np.array_equal(R.read_chain_state()["q"], q)
    R.step(16)
    R.close()


def test_wave_limit_reports_overflow():
    from paper_2402_08273_gb300 import rmlt
    R = rmlt.Renderer()
    R.load_scene(S.two_rooms(20_000, seed=2))
    R.set_tuning(wavefront=True)
    R.init_chains(n_chains=256, width=64, height=64, region_px=16, max_depth=6, n_bootstrap=1 << 10)
    R.step(16)
    R.synchronize()                       # the default limit is never reached
    assert R.read_stats()["wave_limit_hits"] == 0
    R.set_wave_limit(3)
    R.step(16)
    with pytest.raises(rmlt.RmltError) as e:
        R.synchronize()
    assert e.value.status == -7
    with pytest.raises(rmlt.RmltError) as e:
        R.step(16)                        # the context failed
    assert e.value.status == -5
    R.close()


def test_lambda_max_default_chosen_by_the_library():
    from paper_2402_08273_gb300 import rmlt
    R = rmlt.Renderer()
    R.load_toy_integrand(S.TOY_DEFAULT)
    for lm in (0.0, float("nan")):
        R.init_chains(n_chains=16, max_depth=0, n_bootstrap=256, s2=1 / 64, lambda_max=lm)
        assert R.params["lambda_max"] == 2.0 * math.log(32.0)
        R.init_chains(n_chains=16, max_depth=0, n_bootstrap=256, kernel=1, lambda_max=lm)
        assert R.params["lambda_max"] == 2.0 * math.log(4.0)
    R.init_chains(n_chains=16, max_depth=0, n_bootstrap=256, lambda_max=1.5)
    assert R.params["lambda_max"] == 1.5
    assert R.read_stats()["boot_overflow"] == 0
    R.close()
