"""Multi-threshold deblending through gp_deblend, against the oracle.

The oracle deblends its own segmentation of the frame (which must equal the
GPU's here), with nu = F / sigma and m from its own maps.  A segment whose
decisions all stay clear of their bounds -- every pixel's nu more than 1e-5
(relative) from every level, every branch sum more than 1e-5 of the
segment's sum of |m| from the contrast bound -- must come out identical,
label for label.  The rest (float32 against float64 near a bound; with 31
levels and hundreds of pixels a segment often has a pixel within 1e-5 of a
level, most of them harmless) must be valid partitions (every pixel in an
8-connected object with its canonical label), and few may differ.  The objects' catalog rows are compared with the oracle's
moments of the same objects under the plain path's tolerances, widened by
the float32 error of m = I - B (8 u sum|B|).
"""
import numpy as np
import pytest

import oracle
import synth
from parity import REL, assert_close, segment_scales

torch = pytest.importorskip("torch")
gp = pytest.importorskip("paper_2609_32375_gb300")

pytestmark = pytest.mark.gpu

U8 = 8 * 2.0 ** -24


@pytest.fixture(scope="module")
def ctx():
    c = gp.Context(0, workspace_bytes=1 << 29)
    yield c
    c.close()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("name,seed,w,h,mesh", [("dense_12288x12304_u16", 71, 900, 700, 256),
                                                ("plain_2048x2048_u16", 72, 800, 600, 128)])
def test_deblend_matches_the_oracle(ctx, name, seed, w, h, mesh):
    cfg = synth.scaled_config(synth.CONFIGS[name], w, h)
    img, _ = synth.make_frame(cfg, seed, cache=False)
    oracle.set_threads(0)
    ref = oracle.extract(img, mesh, cfg.kernel, cfg.thresh, cfg.minarea, cfg.radii, cfg.gain,
                         saturation=cfg.saturation)
    nu = np.where(ref["rms_map"] > 0, ref["F"] / np.where(ref["rms_map"] > 0, ref["rms_map"], 1.0), 0.0)
    margins = {}
    rseg, rsplit = oracle.deblend(ref["seg"], nu, ref["m"], cfg.thresh, cfg.minarea, margins=margins)
    dimg = dev(img)
    out = ctx.gp_extract(dimg, mesh, cfg.kernel, cfg.thresh, cfg.minarea, cfg.radii, cfg.gain, capacity=100000,
                         saturation=cfg.saturation)
    ctx.sync()
    seg0 = out["segmap"].cpu().numpy().view(np.uint32)
    assert np.array_equal(seg0, ref["seg"]), "the two segmentations differ before deblending"
    bkg = {"bkg_mesh": out["bkg_mesh"], "rms_mesh": out["rms_mesh"], "mesh": mesh}
    seg = out["segmap"].clone()
    db = ctx.gp_deblend(dimg, bkg, cfg.kernel, cfg.thresh, cfg.minarea, seg, out["catalog"],
                        saturation=cfg.saturation)
    ctx.sync()
    gseg = seg.cpu().numpy().view(np.uint32)
    nsplit, nobj = db["counts"].cpu().numpy().tolist()
    labels = np.unique(ref["seg"][ref["seg"] > 0])
    clear = {L for L in labels if margins[int(L)]["nu"] > 1e-5 and margins[int(L)]["flux"] > 1e-5}
    print(f"\n{name} {img.shape}: {len(labels)} segments, oracle split {rsplit}, gpu split {nsplit} "
          f"({nobj} objects); segments on a bound {len(labels) - len(clear)}")
    assert rsplit > 0
    inclear = np.isin(ref["seg"], np.array(sorted(clear), np.uint32))
    assert np.array_equal(gseg[inclear], rseg[inclear])
    differ = 0
    for L in set(labels.tolist()) - clear:
        inseg = ref["seg"] == L
        if not np.array_equal(gseg[inseg], rseg[inseg]):
            differ += 1
        for k in np.unique(gseg[inseg]):
            obj = gseg == k
            assert k != 0 and np.all(inseg[obj])
            assert oracle.label(obj.astype(np.uint8), 1)[1] == 1
            assert k == 1 + np.flatnonzero(obj.ravel())[0]
    print(f"  near a bound: {len(labels) - len(clear)}, of which differ: {differ}")
    assert differ <= max(3, len(labels) // 50)
    assert np.array_equal(gseg[ref["seg"] == 0], np.zeros(int((ref["seg"] == 0).sum()), np.uint32))
    # the objects' catalog: rows of the split segments' objects, in label order
    n = int(db["objects"]["n"].item())
    assert n == nobj
    cat = {k: v[:n].cpu().numpy() for k, v in db["objects"].items() if k != "n"}
    assert np.all(np.diff(cat["label"].astype(np.int64)) > 0)
    rc = oracle.moments(gseg, ref["m"], ref["sat"])
    pos = np.searchsorted(rc["label"], cat["label"])
    assert np.array_equal(rc["label"][pos], cat["label"])
    sub = {k: v[pos] for k, v in rc.items()}
    for k in ("npix", "xmin", "xmax", "ymin", "ymax", "flags", "xpeak", "ypeak"):
        assert np.array_equal(cat[k], sub[k]), k
    s_abs, s_dx, s_dy, s_d2 = [v[pos] for v in segment_scales(gseg, ref["m"], rc)]
    b_abs, b_dx, b_dy, b_d2 = [v[pos] for v in segment_scales(gseg, ref["bkg_map"], rc)]
    f = U8 / REL
    assert_close("flux_iso", cat["flux_iso"], sub["flux"], s_abs + f * b_abs)
    assert_close("x", cat["x"], sub["x"], s_dx + f * b_dx + 1e-3)
    assert_close("y", cat["y"], sub["y"], s_dy + f * b_dy + 1e-3)
    for k in ("x2", "y2", "xy"):
        assert_close(k, cat[k], sub[k], s_d2 + f * b_d2 + 1e-3)
    # the same call again gives the same bits
    seg2 = out["segmap"].clone()
    db2 = ctx.gp_deblend(dimg, bkg, cfg.kernel, cfg.thresh, cfg.minarea, seg2, out["catalog"],
                         saturation=cfg.saturation)
    ctx.sync()
    assert np.array_equal(seg2.cpu().numpy(), seg.cpu().numpy())
    for k in db["objects"]:
        assert torch.equal(db2["objects"][k], db["objects"][k]), k


def test_deblend_rejects_bad_parameters(ctx):
    img = dev(np.full((64, 64), 1000, np.uint16))
    out = ctx.gp_extract(img, 32, np.ones((3, 3), np.float32), 3.0, 5, (3.0,), 1.0, capacity=100)
    bkg = {"bkg_mesh": out["bkg_mesh"], "rms_mesh": out["rms_mesh"], "mesh": 32}
    for kw in ({"nthresh": 0}, {"nthresh": 65}, {"mincont": -0.1}, {"mincont": 1.5}):
        with pytest.raises(gp.GpError):
            ctx.gp_deblend(img, bkg, np.ones((3, 3), np.float32), 3.0, 5, out["segmap"], out["catalog"], **kw)
