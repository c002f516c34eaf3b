"""Parity at the full dense workload -- 12288 x 12304 uint16, mesh 256, the
5x5 filter, k = 1.5, radii 3/6/10, and the same recipe on the paper's 14200 x
10650 frame shape -- in the launch configuration bench.py times: the pre-allocated Extractor, catalog capacity 400,000, no optional
maps.  The oracle cannot run the whole frame inside a test, so it checks
sampled outputs it computes one by one:

- mesh nodes (frame corners, the partial last column and interior nodes)
  from the clipped statistics of their 3 x 3 boxes and the median filter;
- crops at frame corners, edges and the interior: the oracle's spline maps
  (from the GPU's meshes), filter and threshold decide every pixel, and each
  segment lying wholly inside a crop must have the same label, pixels and
  catalog row, with the same apertures;

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
CW, CH = 320, 288                                  # crop size (several tiles and boxes)


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
    out = {"n": n, "cat": cat, "seg": ex.out["segmap"],
           "bkg_mesh": ex.out["bkg_mesh"].cpu().numpy().astype(np.float64),
           "rms_mesh": ex.out["rms_mesh"].cpu().numpy().astype(np.float64)}
    yield cfg, img, out
    del t, ex
    ctx.close()


def test_full_frame_mesh_nodes(run):
    cfg, img, out = run
    H, W = img.shape
    B = cfg.mesh
    Mx, My = -(-W // B), -(-H // B)
    nodes = [(0, 0), (Mx - 1, 0), (0, My - 1), (Mx - 1, My - 1), (Mx // 2, My // 2), (Mx - 1, My // 3), (7, 30)]
    for i, j in nodes:
        i0, i1, j0, j1 = max(0, i - 1), min(Mx - 1, i + 1), max(0, j - 1), min(My - 1, j + 1)
        sub = img[j0 * B:min(H, (j1 + 1) * B), i0 * B:min(W, (i1 + 1) * B)]
        st = oracle.box_stats(sub, np.zeros(sub.shape, np.uint8), B, cfg.clip_k, cfg.clip_maxiter)
        assert st["valid"].all()
        # the node's filter window lies inside this block of boxes, clipped at the mesh edge alike
        rb = oracle.median_filter(st["bkg"], cfg.filter_size)[j - j0, i - i0]
        rr = oracle.median_filter(st["rms"], cfg.filter_size)[j - j0, i - i0]
        gb, gr = out["bkg_mesh"][j, i], out["rms_mesh"][j, i]
        assert abs(gb - rb) <= 1e-5 * abs(rb) + 1e-6, (i, j, gb, rb)
        assert abs(gr - rr) <= 1e-5 * abs(rr) + 1e-6, (i, j, gr, rr)


def crop_check(cfg, img, out, x0, y0):
    """The crop [x0, x0 + CW) x [y0, y0 + CH): every pixel's decision, and the
    segments lying wholly inside it.  Returns the number of segments checked."""
    H, W = img.shape
    B = cfg.mesh
    h = len(cfg.kernel) // 2
    # a halo of h pixels where the frame goes on; at a frame edge the crop edge
    # is the frame edge and the oracle's mirror border is the frame's
    hx0, hx1 = max(0, x0 - h), min(W, x0 + CW + h)
    hy0, hy1 = max(0, y0 - h), min(H, y0 + CH + h)
    region = img[hy0:hy1, hx0:hx1].astype(np.float64)
    ys, xs = np.mgrid[hy0:hy1, hx0:hx1]
    bkg = oracle.spline_at(out["bkg_mesh"], W, H, B, xs.ravel(), ys.ravel()).reshape(region.shape)
    rms = oracle.spline_at(out["rms_mesh"], W, H, B, xs.ravel(), ys.ravel()).reshape(region.shape)
    m = region - bkg
    F = oracle.matched_filter(m, np.asarray(cfg.kernel, np.float64))
    cy, cx = y0 - hy0, x0 - hx0
    sl = (slice(cy, cy + CH), slice(cx, cx + CW))
    Fc, rc, mc = F[sl], rms[sl], m[sl]
    zero = np.zeros((CH, CW), np.uint8)
    fg = oracle.threshold(Fc, rc, zero, cfg.thresh)
    near = oracle.near_threshold(Fc, rc, cfg.thresh)
    sat = oracle.saturated(img[y0:y0 + CH, x0:x0 + CW], cfg.saturation)
    gseg = out["seg"][y0:y0 + CH, x0:x0 + CW].cpu().numpy().view(np.uint32)
    # background decided away from the threshold: no segment on the GPU either
    assert not np.any((gseg != 0) & (fg == 0) & ~near), (x0, y0)
    lab, _ = oracle.label(fg, 1)                   # crop-local canonical labels
    gidx = (np.arange(y0, y0 + CH, dtype=np.int64)[:, None] * W + np.arange(x0, x0 + CW, dtype=np.int64)[None, :])
    # components whose bounding box stays off every crop edge that is not a frame edge
    keep_seg = np.zeros((CH, CW), np.uint32)
    kept_labels = []
    checked = 0
    for c in np.unique(lab[lab != 0]):
        py, px = np.nonzero(lab == c)
        if (px.min() == 0 and x0 > 0) or (px.max() == CW - 1 and x0 + CW < W) or \
           (py.min() == 0 and y0 > 0) or (py.max() == CH - 1 and y0 + CH < H):
            continue
        # a near-threshold pixel in or next to it may flip on either side: skip it
        ya, yb, xa, xb = max(py.min() - 1, 0), py.max() + 2, max(px.min() - 1, 0), px.max() + 2
        if near[ya:yb, xa:xb].any():
            continue
        L = int(gidx[py, px].min()) + 1                # canonical label: 1 + the minimum index
        inside = lab == c
        if len(py) < cfg.minarea:
            assert np.all(gseg[inside] == 0), (x0, y0, L)
            continue
        assert np.all(gseg[inside] == L), (x0, y0, L)
        assert np.count_nonzero(gseg == L) == len(py), (x0, y0, L)
        keep_seg[inside] = c                       # the oracle's moments take labels canonical in the crop
        kept_labels.append((int(c), L))
        checked += 1
    if not kept_labels:
        return 0
    # catalog rows of those segments (oracle positions in crop coordinates);
    # crop and frame labels both follow the raster order of the first pixel
    rc_cat = oracle.moments(keep_seg, mc, sat)
    to_global = dict(kept_labels)
    glabels = np.array([to_global[int(c)] for c in rc_cat["label"]], np.uint32)
    assert np.all(np.diff(glabels.astype(np.int64)) > 0)
    cat = out["cat"]
    rows = np.searchsorted(cat["label"], glabels)
    assert np.array_equal(cat["label"][rows], glabels)
    assert np.array_equal(cat["npix"][rows], rc_cat["npix"])
    for k, off in (("xmin", x0), ("xmax", x0), ("ymin", y0), ("ymax", y0), ("xpeak", x0), ("ypeak", y0)):
        assert np.array_equal(cat[k][rows] - off, rc_cat[k]), k
    assert np.array_equal(cat["flags"][rows], rc_cat["flags"])
    s_abs, s_dx, s_dy, s_d2 = segment_scales(keep_seg, mc, rc_cat)
    assert_close("flux_iso", cat["flux_iso"][rows], rc_cat["flux"], s_abs)
    assert_close("x", cat["x"][rows] - x0, rc_cat["x"], s_dx + 1e-3)
    assert_close("y", cat["y"][rows] - y0, rc_cat["y"], s_dy + 1e-3)
    for k in ("x2", "y2", "xy"):
        assert_close(k, cat[k][rows], rc_cat[k], s_d2 + 1e-3)
    # apertures of those whose largest disc stays inside the crop (or meets only frame edges)
    rmax = max(cfg.radii) + 2.0
    gx, gy = cat["x"][rows] - x0, cat["y"][rows] - y0
    ok = ((gx >= rmax) | (x0 == 0)) & ((gx <= CW - 1 - rmax) | (x0 + CW == W)) & \
         ((gy >= rmax) | (y0 == 0)) & ((gy <= CH - 1 - rmax) | (y0 + CH == H))
    if ok.any():
        rf, re, rfl = oracle.apertures(mc, rc ** 2, zero, sat, gx[ok], gy[ok], cfg.radii, cfg.gain)
        fa, _, _ = oracle.apertures(np.abs(mc), rc ** 2, zero, sat, gx[ok], gy[ok], cfg.radii, 0.0)
        nr = len(cfg.radii)
        assert_close("ap_flux", cat["flux"][rows][ok][:, :nr], rf, fa + 1e-6)
        assert_close("ap_fluxerr", cat["fluxerr"][rows][ok][:, :nr], re, np.abs(re) + 1e-6)
        assert np.array_equal(cat["apflags"][rows][ok][:, :nr].astype(np.uint32), rfl)
    return checked


def test_full_frame_crops(run):
    cfg, img, out = run
    H, W = img.shape
    crops = [(0, 0), (W - CW, 0), (0, H - CH), (W - CW, H - CH), (6000, 5000), (3001, 8117)]
    total = sum(crop_check(cfg, img, out, x0, y0) for x0, y0 in crops)
    print(f"\nsegments checked in {len(crops)} crops of {CW} x {CH}: {total}")
    assert total > 50


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
