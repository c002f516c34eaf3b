"""Host-side checks of the C ABI: the library loads without a GPU, exports
every entry point include/gpphot.h declares, and the Python structs have the
C layout (compared with a C program compiled against the header)."""
import ctypes as C
import os
import re
import subprocess

import pytest

import paper_2609_32375_gb300 as gp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gpphot.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gp_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    L = gp.load_library()
    decl = declared_functions()
    assert set(decl) == set(gp.EXPORTS)
    for name in decl:
        assert hasattr(L, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", gp.library_path()], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\sT\s(gp_\w+)", out))
    assert set(decl) <= exported


STRUCTS = {"gp_image": gp.GpImage, "gp_bkg_params": gp.GpBkgParams, "gp_bkg": gp.GpBkg,
           "gp_det_params": gp.GpDetParams, "gp_catalog": gp.GpCatalog, "gp_ap_params": gp.GpApParams,
           "gp_stats": gp.GpStats, "gp_cnn_weights": gp.GpCnnWeights, "gp_frame": gp.GpFrame,
           "gp_server_config": gp.GpServerConfig, "gp_request": gp.GpRequest, "gp_result": gp.GpResult,
           "gp_server_report": gp.GpServerReport}


def test_struct_layout_matches_header(tmp_path):
    prog = tmp_path / "layout.c"
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "gpphot.h"', "int main(void){"]
    for s, cls in STRUCTS.items():
        lines.append(f'printf("{s} %zu\\n", sizeof({s}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{s}.{f} %zu\\n", offsetof({s}, {f}));')
    lines.append("return 0;}")
    prog.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)])
    got = dict(l.split() for l in subprocess.check_output([str(exe)], text=True).splitlines())
    for s, cls in STRUCTS.items():
        assert int(got[s]) == C.sizeof(cls), s
        for f, _ in cls._fields_:
            assert int(got[f"{s}.{f}"]) == getattr(cls, f).offset, f"{s}.{f}"


def test_workspace_size_is_sane():
    L = gp.load_library()
    small = L.gp_workspace_bytes(1024, 1024, 64, 0)
    big = L.gp_workspace_bytes(12288, 12304, 256, 200000)
    assert 0 < small < big < (2 << 30)
    assert L.gp_workspace_bytes(0, 10, 64, 0) == 0


def test_status_without_device_is_an_error_not_a_fallback():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    L = gp.load_library()
    h = C.c_void_p()
    st = L.gp_ctx_create(0, 1 << 20, C.byref(h))
    assert st in (gp.GP_ERR_CUDA, gp.GP_ERR_INVALID_ARG)
    assert L.gp_last_error()
