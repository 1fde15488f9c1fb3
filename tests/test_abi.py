"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/rmlt.h; host-side argument checks work without a GPU."""
import ctypes as C
import re
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]


def _declared():
    text = (ROOT / "include" / "rmlt.h").read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rmlt_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("rmlt_load_scene", "rmlt_init_chains", "rmlt_step", "rmlt_read_image",
                     "rmlt_read_region_hist", "rmlt_create", "rmlt_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2402_08273_gb300 import rmlt
    L = rmlt.lib()
    missing = [n for n in _declared() if not hasattr(L, n)]
    assert not missing, missing
    # the binding covers every declared function
    bound = {name for name, _, _ in rmlt._SIGS}
    assert set(_declared()) <= bound


def test_host_side_errors_without_gpu():
    from paper_2402_08273_gb300 import rmlt
    L = rmlt.lib()
    assert L.rmlt_abi_version() == 7
    # NULL context / NULL out: argument errors, no device needed
    assert L.rmlt_create(None, 0, None) == -1
    assert L.rmlt_step(None, 1) == -1
    assert L.rmlt_set_trace(None, None, 0, None, 0, 1) == -1
    assert L.rmlt_memory_usage(None, None) == -1
    assert L.rmlt_set_wavefront(None, 0, 0, 16, 0) == -1
    assert L.rmlt_path_grad(None, None, 0, None, None, None) == -1
    assert L.rmlt_exchange_size(None, None, None) == -1
    assert L.rmlt_epoch_mutate(None, None, None) == -1
    assert L.rmlt_epoch_update(None, None, None) == -1
    assert L.rmlt_read_params(None, None) == -1
    assert L.rmlt_set_wave_limit(None, 0) == -1
    assert L.rmlt_set_trace_leaf_batch(None, 8) == -1
    assert L.rmlt_set_node_format(None, 0) == -1
    assert b"null" in L.rmlt_last_error()
    L.rmlt_destroy(None)


def test_create_without_gpu_reports_cuda_error():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2402_08273_gb300 import rmlt
    L = rmlt.lib()
    h = C.c_void_p()
    assert L.rmlt_create(C.byref(h), 0, None) == -4
    assert not h.value
    with pytest.raises(rmlt.RmltError):
        rmlt.Renderer()


def test_struct_layouts_match_header(tmp_path):
    """Every ctypes mirror has the C compiler's size and field offsets."""
    import subprocess
    from paper_2402_08273_gb300 import rmlt
    structs = {"rmlt_material": rmlt.Material, "rmlt_camera": rmlt.Camera,
               "rmlt_scene_desc": rmlt.SceneDesc, "rmlt_chain_params": rmlt.ChainParams,
               "rmlt_stats": rmlt.Stats}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "rmlt.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'printf("{cname}.{fname} %zu\\n", offsetof({cname}, {fname}));')
    lines.append('printf("rmlt_trace_record %zu\\n", sizeof(rmlt_trace_record));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", f"-I{ROOT / 'include'}", str(src), "-o", str(exe)], check=True)
    out = dict(ln.split() for ln in subprocess.run([str(exe)], capture_output=True, text=True,
                                                   check=True).stdout.splitlines())
    for cname, py in structs.items():
        assert int(out[cname]) == C.sizeof(py), cname
        for fname, _ in py._fields_:
            assert int(out[f"{cname}.{fname}"]) == getattr(py, fname).offset, (cname, fname)
    assert int(out["rmlt_trace_record"]) == rmlt.TRACE_DTYPE.itemsize
