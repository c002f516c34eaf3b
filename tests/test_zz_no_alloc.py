"""gp_background_static: the background stage for callers that cannot
allocate device memory (no context, scratch inside the library image).

Checks, through the C ABI, that two calls in a row give the same meshes and
maps as gp_background on the same frames (within the parity tolerance), that
a mesh above the scratch limit is rejected on the host, and that the entry
point works in a fresh process as well as after the other tests.  The file
name sorts last so that a run stopping at the first failure has run every
other test first.
"""
import ctypes as C

import numpy as np
import pytest

import synth
from parity import assert_close

torch = pytest.importorskip("torch")
gp = pytest.importorskip("paper_2609_32375_gb300")

pytestmark = pytest.mark.gpu


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


def test_static_background_matches_context_entry_point():
    frames = [
        (synth.scaled_config(synth.CONFIGS["dense_12288x12304_u16"], 1500, 1100), 21, 256),
        (synth.scaled_config(synth.CONFIGS["plain_1024x1024_f32"], 700, 500), 22, 64),
    ]
    ctx = gp.Context(0, workspace_bytes=512 << 20)
    try:
        for cfg, seed, mesh in frames:           # two calls in a row, different frames
            img, _ = synth.make_frame(cfg, seed, cache=False)
            t = torch.from_numpy(img).cuda()
            got = _static_background(t, mesh, maps=True)
            ref = ctx.gp_background(t, mesh, maps=True)
            ctx.sync()
            torch.cuda.synchronize()
            for k in ("bkg_mesh", "rms_mesh", "bkg_map", "rms_map"):
                g, r = got[k].cpu().numpy(), ref[k].cpu().numpy()
                assert_close(k, g, r, np.abs(r) + 1e-6)
    finally:
        ctx.close()


def test_static_background_rejects_meshes_above_the_limit():
    img = torch.zeros((1100, 1700), dtype=torch.uint16, device="cuda")    # 69 x 107 boxes of 16 px
    with pytest.raises(gp.GpError) as e:
        _static_background(img, 16, maps=False)
    assert e.value.status == gp.GP_ERR_INVALID_ARG
    assert "static scratch limit" in str(e.value)
