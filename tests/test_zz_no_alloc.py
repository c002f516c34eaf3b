"""gp_background_static: the background stage for callers that cannot
allocate device memory -- for example a process whose device memory belongs
to a pool it may not bypass, or a plugin that must not allocate after
start-up.  It takes no context; its scratch is a fixed array inside the
library image.

Checks, through the C ABI:
  * two calls in a row (a uint16 and a float32 frame) give exactly the
    meshes and maps of gp_background on the same frames (the two paths share
    the clip and spline code, so the bits must agree);
  * a mesh above the scratch limit is rejected on the host;
  * in a fresh process, where this entry point is the library's first call
    on the device (the scratch address is looked up then), it gives the same
    results again.
The file name sorts last so that a run stopping at the first failure has run
every other test first.
"""
import ctypes as C
import os
import subprocess
import sys

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
gp = pytest.importorskip("paper_2609_32375_gb300")

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

FRAMES = [
    ("dense_12288x12304_u16", 1500, 1100, 21, 256),
    ("plain_1024x1024_f32", 700, 500, 22, 64),
]


def _static_background(img, mesh, maps):
    """Call gp_background_static directly through ctypes."""
    L = gp.load_library()
    H, W = img.shape
    mx, my = -(-W // mesh), -(-H // mesh)
    out = {"bkg_mesh": torch.full((my, mx), -1.0, dtype=torch.float32, device=img.device),
           "rms_mesh": torch.full((my, mx), -1.0, dtype=torch.float32, device=img.device)}
    if maps:
        out["bkg_map"] = torch.full((H, W), -1.0, dtype=torch.float32, device=img.device)
        out["rms_map"] = torch.full((H, W), -1.0, dtype=torch.float32, device=img.device)
    gi = gp.make_image(img)
    p = gp.GpBkgParams(mesh, 3, 3.0, 10)
    b = gp.GpBkg(0, 0, 0, out["bkg_mesh"].data_ptr(), out["rms_mesh"].data_ptr(),
                 out["bkg_map"].data_ptr() if maps else None, out["rms_map"].data_ptr() if maps else None)
    st = L.gp_background_static(C.byref(gi), C.byref(p), C.byref(b),
                                torch.cuda.current_stream().cuda_stream or None)
    if st != gp.GP_OK:
        raise gp.GpError(st, L.gp_last_error().decode())
    assert (b.mesh, b.mx, b.my) == (mesh, mx, my)
    return out


def _compare_with_context(static_first):
    """Run both frames through gp_background_static (two calls in a row) and
    through gp_background, and require identical outputs."""
    frames = []
    for name, w, h, seed, mesh in FRAMES:
        img, _ = synth.make_frame(synth.scaled_config(synth.CONFIGS[name], w, h), seed, cache=False)
        frames.append((torch.from_numpy(img).cuda(), mesh))
    got = [_static_background(t, mesh, maps=True) for t, mesh in frames] if static_first else None
    ctx = gp.Context(0, workspace_bytes=512 << 20)
    try:
        if got is None:
            got = [_static_background(t, mesh, maps=True) for t, mesh in frames]
        for (t, mesh), g in zip(frames, got):
            ref = ctx.gp_background(t, mesh, maps=True)
            ctx.sync()
            torch.cuda.synchronize()
            for k in ("bkg_mesh", "rms_mesh", "bkg_map", "rms_map"):
                a, b = g[k].cpu().numpy(), ref[k].cpu().numpy()
                assert np.array_equal(a, b), f"{k}: static and context paths differ"
    finally:
        ctx.close()


def test_static_background_matches_context_entry_point():
    _compare_with_context(static_first=False)


def test_static_background_rejects_meshes_above_the_limit():
    img = torch.zeros((1100, 1700), dtype=torch.uint16, device="cuda")    # 69 x 107 boxes of 16 px
    with pytest.raises(gp.GpError) as e:
        _static_background(img, 16, maps=False)
    assert e.value.status == gp.GP_ERR_INVALID_ARG
    assert "static scratch limit" in str(e.value)


def test_static_background_as_first_call_in_a_fresh_process():
    code = ("import sys; sys.path[:0] = [{root!r}, {tests!r}]; "
            "import test_zz_no_alloc as t; t._compare_with_context(static_first=True); print('fresh ok')"
            ).format(root=ROOT, tests=os.path.join(ROOT, "tests"))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, cwd=ROOT, timeout=600)
    assert r.returncode == 0 and "fresh ok" in r.stdout, r.stdout[-2000:] + r.stderr[-2000:]
