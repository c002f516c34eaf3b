"""Parity at the full dense workload -- 12288 x 12304 uint16 (151.2 MP),
mesh 256, the 5x5 filter, k = 1.5, radii 3/6/10, and the same recipe on the
paper's 14200 x 10650 frame shape -- in the launch configuration bench.py
times: the pre-allocated Extractor, catalog capacity 400,000, no optional
maps.

The oracle runs the whole frame (its independent loops on every host core;
the results do not depend on the thread count), and every output is compared
with it:

- all mesh nodes (background and rms);
- the whole threshold mask (from a second call that also returns the byte
  mask; its map must equal the timed configuration's): every disagreement
  with the oracle lies in the near-threshold set;
- the whole segmentation map, bit for bit, against the oracle's labelling
  of the GPU's mask;
- every catalog row against the oracle's moments of the GPU's segments with
  the oracle's m, and every aperture against the oracle's sums at the GPU's
  centroids (flags exact);

and the whole output is checked for properties that hold at any size
(canonical labels, counts, ordering).
"""
import numpy as np
import pytest

import oracle
import synth
from parity import assert_close, segment_scales

torch = pytest.importorskip("torch")
gp = pytest.importorskip("paper_2609_32375_gb300")

pytestmark = pytest.mark.gpu

CAPACITY = 400_000

# the frame bench.py measures, and the paper's own 151 MP frame shape
# (14200 x 10650: ragged detection tiles and mesh boxes at full size) with
# the same source density
SHAPES = [None, (14200, 10650)]


@pytest.fixture(scope="module", params=SHAPES, ids=["12288x12304", "14200x10650"])
def run(request):
    cfg = synth.CONFIGS["dense_12288x12304_u16"]
    if request.param is not None:
        cfg = synth.scaled_config(cfg, *request.param)
    img, _ = synth.make_frame(cfg, 0)
    H, W = img.shape
    L = gp.load_library()
    ctx = gp.Context(0, workspace_bytes=L.gp_workspace_bytes(W, H, cfg.mesh, CAPACITY) + (64 << 20))
    t = torch.from_numpy(img).cuda()
    ex = gp.Extractor(ctx, (H, W), t.dtype, cfg.mesh, cfg.kernel, cfg.thresh, cfg.minarea, cfg.radii, cfg.gain,
                      CAPACITY, saturation=cfg.saturation, device="cuda")
    ex.run(t)
    ctx.sync()
    n, cat = ex.catalog_host()
    # the same frame once more, returning the byte mask as well
    full = ctx.gp_extract(t, cfg.mesh, cfg.kernel, cfg.thresh, cfg.minarea, cfg.radii, cfg.gain, capacity=CAPACITY,
                          saturation=cfg.saturation, mask_out=True)
    ctx.sync()
    out = {"n": n, "cat": cat, "seg": ex.out["segmap"],
           "bkg_mesh": ex.out["bkg_mesh"].cpu().numpy().astype(np.float64),
           "rms_mesh": ex.out["rms_mesh"].cpu().numpy().astype(np.float64),
           "mask": full["mask"].cpu().numpy(), "seg_masked_call": full["segmap"]}
    del full
    yield cfg, img, out
    del t, ex
    ctx.close()


@pytest.fixture(scope="module")
def ref(run):
    cfg, img, out = run
    oracle.set_threads(0)
    try:
        r = oracle.extract(img, cfg.mesh, cfg.kernel, cfg.thresh, cfg.minarea, cfg.radii, cfg.gain,
                           saturation=cfg.saturation)
    finally:
        oracle.set_threads(1)
    return r


def test_whole_frame_meshes(run, ref):
    cfg, img, out = run
    for k in ("bkg_mesh", "rms_mesh"):
        assert_close(k, out[k], ref[k], np.abs(ref[k]) + 1e-6)


def test_whole_frame_mask_and_segmentation(run, ref):
    cfg, img, out = run
    gmask = out["mask"]
    assert torch.equal(out["seg_masked_call"], out["seg"])      # both launch forms, one map
    diff = gmask != ref["fg"]
    print(f"\n  mask disagreements {int(diff.sum())} (near-threshold set {int(ref['near'].sum())})")
    assert not np.any(diff & ~ref["near"])
    lab, nlab = oracle.label(gmask, cfg.minarea)
    gseg = out["seg"].cpu().numpy().view(np.uint32)
    assert np.array_equal(gseg, lab)
    assert out["n"] == nlab


def test_whole_frame_catalog_and_apertures(run, ref):
    cfg, img, out = run
    gseg = out["seg"].cpu().numpy().view(np.uint32)
    m, sat = ref["m"], ref["sat"]
    rc = oracle.moments(gseg, m, sat)
    cat = out["cat"]
    n = out["n"]
    assert len(rc["label"]) == n
    assert np.array_equal(cat["label"], rc["label"])
    for k in ("npix", "xmin", "xmax", "ymin", "ymax", "flags"):
        assert np.array_equal(cat[k], rc[k]), k
    s_abs, s_dx, s_dy, s_d2 = segment_scales(gseg, m, rc)
    assert_close("flux_iso", cat["flux_iso"], rc["flux"], s_abs)
    assert_close("x", cat["x"], rc["x"], s_dx + 1e-3)
    assert_close("y", cat["y"], rc["y"], s_dy + 1e-3)
    for k in ("x2", "y2", "xy"):
        assert_close(k, cat[k], rc[k], s_d2 + 1e-3)
    # the peak: the same pixel, unless the oracle's m there ties its maximum
    # to within the float32 rounding of m (then either pixel is a peak)
    W = img.shape[1]
    gpk = m.ravel()[cat["ypeak"].astype(np.int64) * W + cat["xpeak"]]
    same = (cat["xpeak"] == rc["xpeak"]) & (cat["ypeak"] == rc["ypeak"])
    tie = np.abs(gpk - rc["peak"]) <= 1e-6 * np.abs(rc["peak"]) + 1e-3
    assert np.all(same | tie)
    assert_close("peak", cat["peak"], rc["peak"], np.abs(rc["peak"]) + 1.0)
    # apertures at the GPU's centroids
    nr = len(cfg.radii)
    rf, re, rfl = oracle.apertures(m, ref["rms_map"] ** 2, ref["bad"], sat, cat["x"], cat["y"], cfg.radii, cfg.gain)
    fa, _, _ = oracle.apertures(np.abs(m), ref["rms_map"] ** 2, ref["bad"], sat, cat["x"], cat["y"], cfg.radii, 0.0)
    assert_close("ap_flux", cat["flux"][:, :nr], rf, fa + 1e-6)
    assert_close("ap_fluxerr", cat["fluxerr"][:, :nr], re, np.abs(re) + 1e-6)
    assert np.array_equal(cat["apflags"][:, :nr].astype(np.uint32), rfl)


def test_full_frame_map_and_catalog_are_consistent(run):
    cfg, img, out = run
    H, W = img.shape
    n, cat = out["n"], out["cat"]
    seg = out["seg"].view(-1)
    assert 0 < n <= CAPACITY and len(cat["label"]) == n
    labels = cat["label"].astype(np.int64)
    assert np.all(np.diff(labels) > 0)                      # catalog in label order
    lab = torch.from_numpy(labels).cuda()
    # label = 1 + the segment's minimum index: that pixel belongs to it and opens its top row
    assert torch.equal(seg[lab - 1].to(torch.int64), lab)
    first = labels - 1
    assert np.array_equal(first // W, cat["ymin"].astype(np.int64))
    assert np.all((first % W >= cat["xmin"]) & (first % W <= cat["xmax"]))
    # every labelled pixel is counted once, and the map holds exactly the catalog's labels
    nz = seg != 0
    assert int(nz.sum()) == int(cat["npix"].astype(np.int64).sum())
    assert torch.equal(torch.unique(seg[nz]).to(torch.int64), lab)
    assert np.all(cat["npix"] >= cfg.minarea)
    # the peak pixel belongs to its segment
    pk = torch.from_numpy(cat["ypeak"].astype(np.int64) * W + cat["xpeak"].astype(np.int64)).cuda()
    assert torch.equal(seg[pk].to(torch.int64), lab)
