"""CPU oracle for the extraction path -- TEST INFRASTRUCTURE ONLY.

Plain FP64 statement of what the per-frame extraction computes (paper
Sections 3.1, 3.2 and 3.4, with the readings [R#] listed in oracle.c).  Only
tests/, the smoke check and bench.py's CPU-baseline leg import this package;
the CUDA library never does, and the two share no code.  The loops live in
oracle.c (compiled with gcc, no fast-math, no FMA contraction); the
element-wise glue between steps is plain numpy.

Parity unpinned (readings of the paper that no printed value fixes; their
arithmetic is pinned, the choice is not): the box mode rule [R4, oracle.c],
the significance nu of a source as F / sigma at its catalog peak [R24], and
the attribution of a split segment's pixels outside the seeds by growth
within the level sets [R37].
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

FLAG_SAT = 1
FLAG_CENTROID_FALLBACK = 2
FLAG_TRUNCATED = 4
FLAG_BAD = 8


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/_lib/liboracle.so (-O2, strict IEEE: no
    fast-math and no FMA contraction; OpenMP for the loops over independent
    outputs when gcc has it, else single-threaded)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        base = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fPIC", "-shared", "-ffp-contract=off",
                "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
        if subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True).returncode != 0:
            subprocess.check_call(base)
        os.replace(tmp, _LIB)
    return _LIB


def set_threads(n: int) -> int:
    """Host threads for the oracle's parallel loops (n < 1: every core);
    returns the count it will use.  The results do not depend on it."""
    return int(lib().orc_set_threads(int(n)))


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            d, i, l, u8, u32, vp = C.c_double, C.c_int, C.c_long, C.c_uint8, C.c_uint32, C.c_void_p
            L.orc_sigma_clip.argtypes = [vp, l, d, i, vp, vp, vp, vp]
            L.orc_sigma_clip.restype = i
            L.orc_mode_estimate.argtypes = [d, d, d]
            L.orc_mode_estimate.restype = d
            L.orc_box_stats.argtypes = [vp, vp, i, i, i, d, i, vp, vp, vp, vp, vp, vp]
            L.orc_fill_invalid.argtypes = [vp, vp, vp, i, i]
            L.orc_median_filter.argtypes = [vp, vp, i, i, i]
            L.orc_median_filter.restype = i
            L.orc_spline_at.argtypes = [vp, i, i, i, i, i, vp, vp, l, vp]
            L.orc_spline_map.argtypes = [vp, i, i, i, i, i, vp]
            L.orc_filter.argtypes = [vp, i, i, vp, i, i, vp]
            L.orc_filter.restype = i
            L.orc_filter_at.argtypes = [vp, i, i, vp, i, i, vp, vp, l, vp]
            L.orc_filter_at.restype = i
            L.orc_label.argtypes = [vp, i, i, i, vp]
            L.orc_label.restype = l
            L.orc_moments.argtypes = [vp, vp, vp, i, i, l] + [vp] * 16
            L.orc_moments.restype = l
            L.orc_overlap_area.argtypes = [d, d, d, d, d]
            L.orc_overlap_area.restype = d
            L.orc_apertures.argtypes = [vp, vp, vp, vp, i, i, vp, vp, l, vp, i, d, vp, vp, vp]
            L.orc_growth.argtypes = [vp, vp, vp, vp, i, i, vp, vp, l, vp, i, d, vp, vp, vp]
            L.orc_set_threads.argtypes = [i]
            L.orc_set_threads.restype = i
            _lib = L
            L.orc_set_threads(1)          # the plain single-threaded definition unless asked
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _u8(a):
    return np.ascontiguousarray(a, dtype=np.uint8)


# ---------------------------------------------------------------- pixels ---
def pixel_values(image, mask=None):
    """[R1] pixel values as exact doubles and the bad-pixel map (masked or
    NaN pixels are bad)."""
    img = np.asarray(image).astype(np.float64)
    bad = ~np.isfinite(img)
    if mask is not None:
        bad |= np.asarray(mask) != 0
    return np.where(bad, 0.0, img), bad.astype(np.uint8)


def saturated(image, saturation):
    if saturation is None or saturation <= 0:
        return np.zeros(np.shape(image), np.uint8)
    a = np.asarray(image).astype(np.float64)
    return (np.isfinite(a) & (a >= saturation)).astype(np.uint8)


# ------------------------------------------------------------ background ---
def sigma_clip(values, k=3.0, maxiter=10):
    """[R3] clipped (median, mean, std, nkept, passes) of a 1-D set."""
    v = _f64(values).copy()
    med, mean, sd = C.c_double(), C.c_double(), C.c_double()
    nk = C.c_long()
    passes = lib().orc_sigma_clip(_p(v), v.size, k, maxiter, C.byref(med), C.byref(mean),
                                  C.byref(sd), C.byref(nk))
    return med.value, mean.value, sd.value, nk.value, passes


def mode_estimate(med, mean, sd):
    return lib().orc_mode_estimate(med, mean, sd)


def box_stats(img, bad, mesh, k=3.0, maxiter=10):
    """[R2]-[R4] raw per-box statistics; dict of My x Mx arrays."""
    img, bad = _f64(img), _u8(bad)
    H, W = img.shape
    Mx, My = -(-W // mesh), -(-H // mesh)
    out = {n: np.zeros((My, Mx)) for n in ("bkg", "rms", "med", "mean")}
    valid = np.zeros((My, Mx), np.uint8)
    nk = np.zeros((My, Mx), np.int64)
    lib().orc_box_stats(_p(img), _p(bad), W, H, mesh, k, maxiter, _p(out["bkg"]), _p(out["rms"]),
                        _p(valid), _p(out["med"]), _p(out["mean"]), _p(nk))
    out["valid"] = valid
    out["nkept"] = nk
    return out


def fill_invalid(bkg, rms, valid):
    """[R5]"""
    bkg, rms, valid = _f64(bkg).copy(), _f64(rms).copy(), _u8(valid).copy()
    My, Mx = bkg.shape
    lib().orc_fill_invalid(_p(bkg), _p(rms), _p(valid), Mx, My)
    return bkg, rms


def median_filter(mesh, fsize=3):
    """[R6]"""
    a = _f64(mesh)
    out = np.zeros_like(a)
    My, Mx = a.shape
    if lib().orc_median_filter(_p(a), _p(out), Mx, My, fsize) != 0:
        raise ValueError("filter size too large")
    return out


def background_meshes(img, bad, mesh, fsize=3, k=3.0, maxiter=10):
    """Filtered background and rms meshes ([R2]-[R6])."""
    st = box_stats(img, bad, mesh, k, maxiter)
    b, r = fill_invalid(st["bkg"], st["rms"], st["valid"])
    if fsize > 1:
        b, r = median_filter(b, fsize), median_filter(r, fsize)
    return b, r, st


def spline_map(mesh_vals, W, H, B):
    """[R7] full-resolution map from a mesh."""
    a = _f64(mesh_vals)
    My, Mx = a.shape
    out = np.zeros((H, W))
    lib().orc_spline_map(_p(a), Mx, My, W, H, B, _p(out))
    return out


def spline_at(mesh_vals, W, H, B, xs, ys):
    """[R7] the map at selected pixel positions."""
    a = _f64(mesh_vals)
    My, Mx = a.shape
    xs, ys = _f64(xs), _f64(ys)
    out = np.zeros(xs.size)
    lib().orc_spline_at(_p(a), Mx, My, W, H, B, _p(xs), _p(ys), xs.size, _p(out))
    return out


# ------------------------------------------------------------- detection ---
def matched_filter(m, kernel):
    """[R8] F = normalised kernel correlated with m, mirror border."""
    m, K = _f64(m), _f64(kernel)
    H, W = m.shape
    kh, kw = K.shape
    F = np.zeros_like(m)
    if lib().orc_filter(_p(m), W, H, _p(K), kw, kh, _p(F)) != 0:
        raise ValueError("kernel sums to zero")
    return F


def matched_filter_at(m, kernel, xs, ys):
    m, K = _f64(m), _f64(kernel)
    H, W = m.shape
    kh, kw = K.shape
    xs = np.ascontiguousarray(xs, dtype=np.int64)
    ys = np.ascontiguousarray(ys, dtype=np.int64)
    out = np.zeros(xs.size)
    if lib().orc_filter_at(_p(m), W, H, _p(K), kw, kh, _p(xs), _p(ys), xs.size, _p(out)) != 0:
        raise ValueError("kernel sums to zero")
    return out


def threshold(F, rms_map, bad, k):
    """[R10] foreground mask, strict, never on bad pixels."""
    return ((F > k * rms_map) & (np.asarray(bad) == 0)).astype(np.uint8)


def near_threshold(F, rms_map, k, rel=1e-5):
    """Pixels whose decision is within rel of the threshold (set N)."""
    t = k * rms_map
    return np.abs(F - t) <= rel * np.abs(t)


def label(fg, minarea=1):
    """[R11][R12] uint32 segmentation map and number of kept components."""
    fg = _u8(fg)
    H, W = fg.shape
    seg = np.zeros((H, W), np.uint32)
    n = lib().orc_label(_p(fg), W, H, minarea, _p(seg))
    return seg, int(n)


def moments(seg, m, sat=None):
    """[R13] catalog dict in ascending label order."""
    seg = np.ascontiguousarray(seg, dtype=np.uint32)
    m = _f64(m)
    H, W = seg.shape
    sat = _u8(sat) if sat is not None else None
    ncap = int(np.count_nonzero(seg)) + 1
    f64 = lambda: np.zeros(ncap)
    i32 = lambda: np.zeros(ncap, np.int32)
    cat = dict(label=np.zeros(ncap, np.uint32), npix=np.zeros(ncap, np.int64), flux=f64(),
               x=f64(), y=f64(), x2=f64(), y2=f64(), xy=f64(), xmin=i32(), xmax=i32(),
               ymin=i32(), ymax=i32(), peak=f64(), xpeak=i32(), ypeak=i32(),
               flags=np.zeros(ncap, np.uint32))
    order = ["label", "npix", "flux", "x", "y", "x2", "y2", "xy", "xmin", "xmax", "ymin", "ymax",
             "peak", "xpeak", "ypeak", "flags"]
    n = lib().orc_moments(_p(seg), _p(m), _p(sat), W, H, ncap, *[_p(cat[k]) for k in order])
    return {k: v[:n] for k, v in cat.items()}


# ------------------------------------------------------------- apertures ---
def overlap_area(x0, x1, y0, y1, r):
    """[R14] exact area of disc(0, r) n [x0,x1] x [y0,y1]."""
    return lib().orc_overlap_area(x0, x1, y0, y1, r)


def apertures(m, var, bad, sat, xs, ys, radii, gain):
    """[R14] (flux, fluxerr, flags), each n x nr."""
    m, var, bad = _f64(m), _f64(var), _u8(bad)
    sat = _u8(sat) if sat is not None else None
    H, W = m.shape
    xs, ys = _f64(xs), _f64(ys)
    radii = _f64(radii)
    n, nr = xs.size, radii.size
    flux = np.zeros((n, nr))
    err = np.zeros((n, nr))
    flags = np.zeros((n, nr), np.uint32)
    lib().orc_apertures(_p(m), _p(var), _p(bad), _p(sat), W, H, _p(xs), _p(ys), n, _p(radii), nr,
                        float(gain), _p(flux), _p(err), _p(flags))
    return flux, err, flags


def growth_radii(fwhm):
    """[R20] the paper's integer radii, ceil(0.75 FWHM) .. ceil(5 FWHM)."""
    return np.arange(int(np.ceil(0.75 * fwhm)), int(np.ceil(5.0 * fwhm)) + 1, dtype=np.int32)


def growth(m, var, bad, sat, xs, ys, radii, gain):
    """[R20][R21] top-hat growth curves (flux, fluxerr, flags), each n x nr."""
    m, var, bad = _f64(m), _f64(var), _u8(bad)
    sat = _u8(sat) if sat is not None else None
    H, W = m.shape
    xs, ys = _f64(xs), _f64(ys)
    radii = np.ascontiguousarray(radii, dtype=np.int32)
    n, nr = xs.size, radii.size
    flux = np.zeros((n, nr))
    err = np.zeros((n, nr))
    flags = np.zeros((n, nr), np.uint32)
    lib().orc_growth(_p(m), _p(var), _p(bad), _p(sat), W, H, _p(xs), _p(ys), n, _p(radii), nr, float(gain),
                     _p(flux), _p(err), _p(flags))
    return flux, err, flags


# ------------------------------------------- optimal radius (Section 3.4) ---
# The paper searches the radius of largest S/N only for high-S/N isolated
# calibrators, fits log10 r_opt = a log10 nu + b to them (nu the detection
# significance) and gives every other source the radius of the fit.  The
# selection thresholds and the rounding onto the radius grid are readings
# [R22]-[R27].
def significance(F, rms_map, xp, yp):
    """[R24] nu = F / sigma at each source's peak pixel (0 where sigma <= 0)."""
    F, rms_map = _f64(F), _f64(rms_map)
    xp = np.asarray(xp, np.int64)
    yp = np.asarray(yp, np.int64)
    s = rms_map[yp, xp]
    return np.where(s > 0, F[yp, xp] / np.where(s > 0, s, 1.0), 0.0)


def snr_argmax(flux, fluxerr):
    """[R22][R23] S/N = flux / fluxerr per source and radius (0 where
    fluxerr <= 0) and the index of its largest value (the first on ties)."""
    flux, fluxerr = _f64(flux), _f64(fluxerr)
    snr = np.where(fluxerr > 0, flux / np.where(fluxerr > 0, fluxerr, 1.0), 0.0)
    return np.argmax(snr, axis=1).astype(np.int32), snr


def isolated(xs, ys, dmin):
    """[R25] True where no other source lies closer than dmin (all pairs)."""
    xs, ys = _f64(xs), _f64(ys)
    n = xs.size
    iso = np.ones(n, bool)
    for i0 in range(0, n, 512):
        i1 = min(n, i0 + 512)
        d2 = (xs[i0:i1, None] - xs[None, :]) ** 2 + (ys[i0:i1, None] - ys[None, :]) ** 2
        close = d2 < dmin * dmin
        close[np.arange(i1 - i0), np.arange(i0, i1)] = False
        iso[i0:i1] = ~close.any(axis=1)
    return iso


def calibrators(cat_flags, growth_flags, snr, kopt, iso, nu, snr_min):
    """[R25] unflagged (catalog and every growth radius), isolated, nu > 0 and
    S/N >= snr_min at the best radius."""
    n = len(kopt)
    best = snr[np.arange(n), kopt]
    return ((np.asarray(cat_flags) == 0) & np.all(np.asarray(growth_flags) == 0, axis=1) & iso & (nu > 0)
            & (best >= snr_min))


def power_law_fit(nu, r, sel):
    """[R26] ordinary least squares of log10 r on log10 nu over the selected
    sources, from the centred sums: a = sum (x - mx)(y - my) / sum (x - mx)^2,
    b = my - a mx.  Returns (a, b, n); a and b are NaN below 3 sources or
    when every x is the same."""
    x = np.log10(_f64(nu)[sel])
    y = np.log10(_f64(r)[sel])
    n = x.size
    if n < 3 or x.max() == x.min():
        return float("nan"), float("nan"), n
    mx, my = x.sum() / n, y.sum() / n
    dx = x - mx
    a = (dx * (y - my)).sum() / (dx * dx).sum()
    return a, my - a * mx, n


def assign_radius(nu, a, b, radii):
    """[R27] index of the grid radius nearest to r_fit = 10^(a log10 nu + b)
    (ties to the larger radius; beyond the grid, its end); the smallest
    radius where nu <= 0 or the fit failed."""
    nu = _f64(nu)
    radii = _f64(radii)
    k = np.zeros(nu.size, np.int32)
    if not (np.isfinite(a) and np.isfinite(b)):
        return k
    ok = nu > 0
    rf = 10.0 ** (a * np.log10(np.where(ok, nu, 1.0)) + b)
    d = np.abs(radii[None, :] - rf[:, None])
    last = radii.size - 1 - np.argmin(d[:, ::-1], axis=1)    # the larger radius on ties
    return np.where(ok, last, 0).astype(np.int32)


def optimal_radius(m, var, bad, sat, F, rms_map, cat, radii, gain, snr_min, d_iso):
    """The optimal-radius step: growth curves at the centroids, nu at the
    peak pixels, the best radius of every source, the calibrators, the fit,
    and each source's radius (a calibrator keeps its own best radius)."""
    radii = np.ascontiguousarray(radii, dtype=np.int32)
    flux, err, gfl = growth(m, var, bad, sat, cat["x"], cat["y"], radii, gain)
    nu = significance(F, rms_map, cat["xpeak"], cat["ypeak"])
    kopt, snr = snr_argmax(flux, err)
    iso = isolated(cat["x"], cat["y"], d_iso)
    cal = calibrators(cat["flags"], gfl, snr, kopt, iso, nu, snr_min)
    a, b, ncal = power_law_fit(nu, radii[kopt], cal)
    kas = assign_radius(nu, a, b, radii)
    kfin = np.where(cal, kopt, kas).astype(np.int32)
    i = np.arange(len(kfin))
    return dict(flux=flux, fluxerr=err, flags=gfl, nu=nu, snr=snr, kopt=kopt, iso=iso, calib=cal, a=a, b=b,
                ncal=ncal, kassign=kas, kfinal=kfin, flux_opt=flux[i, kfin], fluxerr_opt=err[i, kfin])


# --------------------------- spatially varying matched filter (Section 3.2) ---
# The second detection pass correlates m with the local PSF, a reference P0
# plus K eigenmodes e_k whose coefficients c_k vary over the frame:
# S = P0 (x) m + sum_k c_k (e_k (x) m), each term a plain correlation with a
# mirror border, weighted by its coefficient map [R28]; the maps are the
# natural cubic spline through per-tile coefficients [R29]; foreground is
# S > k sigma [R30].
def correlate(m, kernel):
    """[R28] sum over taps (u, v) of K[v, u] m(x + u - kw/2, y + v - kh/2),
    mirror border without edge repeat, the kernel used as given."""
    m, K = _f64(m), _f64(kernel)
    kh, kw = K.shape
    hy, hx = kh // 2, kw // 2
    H, W = m.shape
    pad = np.pad(m, ((hy, hy), (hx, hx)), mode="reflect")
    out = np.zeros_like(m)
    for v in range(kh):
        for u in range(kw):
            out += K[v, u] * pad[v:v + H, u:u + W]
    return out


def coefficient_maps(coef, W, H, tile):
    """[R29] per-pixel coefficient maps from K meshes of per-tile values."""
    coef = _f64(coef)
    return [spline_map(coef[k], W, H, tile) for k in range(coef.shape[0])]


def psf_filter(m, p0, modes, coef, tile):
    """[R28][R29] S = P0 (x) m + sum_k c_k * (e_k (x) m)."""
    H, W = m.shape
    S = correlate(m, p0)
    for c, e in zip(coefficient_maps(coef, W, H, tile), np.asarray(modes, np.float64)):
        S = S + c * correlate(m, e)
    return S


def detect_psf(image, mesh, p0, modes, coef, tile, thresh, minarea, mask=None, saturation=0.0,
               fsize=3, clip_k=3.0, clip_maxiter=10):
    """The second detection pass in the stage order of extract(): background
    and noise map, the spatially varying filter, threshold [R30], labelling
    and moments."""
    img, bad = pixel_values(image, mask)
    H, W = img.shape
    bkg_mesh, rms_mesh, _ = background_meshes(img, bad, mesh, fsize, clip_k, clip_maxiter)
    bkg_map = spline_map(bkg_mesh, W, H, mesh)
    rms_map = spline_map(rms_mesh, W, H, mesh)
    m = np.where(bad != 0, 0.0, img - bkg_map)
    S = psf_filter(m, p0, modes, coef, tile)
    fg = threshold(S, rms_map, bad, thresh)
    seg, n = label(fg, minarea)
    sat = saturated(image, saturation)
    cat = moments(seg, m, sat)
    return dict(bkg_mesh=bkg_mesh, rms_mesh=rms_mesh, bkg_map=bkg_map, rms_map=rms_map, m=m, bad=bad, S=S, fg=fg,
                seg=seg, cat=cat, near=near_threshold(S, rms_map, thresh))


# ----------------------------------------- cosmetic filters (Section 3.1) ---
# Two optional corrections before the background: a salt-and-pepper filter
# for random telegraph noise that replaces isolated outliers of a
# median-filtered residual [R31], and a cosmic-ray filter in the manner of
# L.A.Cosmic that flags sharp edges through a Laplacian and fills the flagged
# pixels from their neighbours [R32].  Windows have a mirror border; bad
# pixels (masked or non-finite) are left out of every window and are never
# flagged or changed.
def window_median(a, size):
    """Median of each size x size window (mirror border) over its finite
    values (the mean of the two middle ones for an even count); NaN where a
    window holds none."""
    a = _f64(a)
    h = size // 2
    pad = np.pad(a, h, mode="reflect")
    win = np.lib.stride_tricks.sliding_window_view(pad, (size, size))
    flat = win.reshape(a.shape + (size * size,))
    with np.errstate(all="ignore"):
        import warnings
        with warnings.catch_warnings():
            warnings.simplefilter("ignore", RuntimeWarning)
            return np.nanmedian(flat, axis=-1)


def _shift(a, dy, dx):
    """a(y + dy, x + dx) with a mirror border."""
    H, W = a.shape
    ys = np.array([_mirror(y + dy, H) for y in range(H)])
    xs = np.array([_mirror(x + dx, W) for x in range(W)])
    return a[np.ix_(ys, xs)]


def _mirror(i, n):
    if n == 1:
        return 0
    p = 2 * (n - 1)
    i = abs(i) % p
    return p - i if i >= n else i


def rtn_filter(image, t, mask=None):
    """[R31] r = I - med3(I); a good pixel with |r| > t whose 8 neighbours
    hold no such pixel takes med3.  Returns (corrected frame, replaced)."""
    img, bad = pixel_values(image, mask)
    a = np.where(bad != 0, np.nan, img)
    med = window_median(a, 3)
    with np.errstate(invalid="ignore"):
        out = (bad == 0) & (np.abs(a - med) > t)
    others = np.zeros(a.shape, np.int32)
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            if dy or dx:
                others += _shift(out.astype(np.int32), dy, dx)
    rep = out & (others == 0)
    return np.where(rep, med, np.where(bad != 0, np.asarray(image, np.float64), img)), rep


def cr_filter(image, gain, read_noise, sigclip=4.5, objlim=5.0, mask=None, details=False):
    """[R32] One pass: L = 4 I - (the 4 nearest neighbours), L+ = max(L, 0);
    the noise N = sqrt(max(med5(I), 0) gain + rn^2) / gain (ADU); S =
    L+ / (sqrt(20) N) (L's standard deviation for independent pixel noise N:
    4^2 + 4 x 1^2 = 20) less its 5x5 median; the fine structure F = med3(I) - med7(med3(I)),
    floored at 0.01; flagged where S > sigclip and L+ / F > objlim; a flagged
    pixel takes the median of the good unflagged pixels of its 5x5 window
    (unchanged when there are none).  Returns (corrected frame, flagged), and
    with details the two decision values (S less its median, L+ / F)."""
    img, bad = pixel_values(image, mask)
    a = np.where(bad != 0, np.nan, img)
    L = 4 * a - _shift(a, 0, -1) - _shift(a, 0, 1) - _shift(a, -1, 0) - _shift(a, 1, 0)
    Lp = np.maximum(L, 0.0)                        # NaN stays NaN
    noise = np.sqrt(np.maximum(window_median(a, 5), 0.0) * gain + read_noise * read_noise) / gain
    S = Lp / (np.sqrt(20.0) * noise)
    Sp = S - window_median(S, 5)
    m3 = window_median(a, 3)
    F = np.maximum(m3 - window_median(m3, 7), 0.01)
    with np.errstate(invalid="ignore"):
        flag = (bad == 0) & (Sp > sigclip) & (Lp / F > objlim)
    clean = np.where(flag, np.nan, a)
    fill = window_median(clean, 5)
    rep = flag & np.isfinite(fill)
    out = np.where(rep, fill, np.where(bad != 0, np.asarray(image, np.float64), img))
    if details:
        with np.errstate(invalid="ignore", divide="ignore"):
            return out, flag, dict(sp=Sp, ratio=Lp / F)
    return out, flag


# ------------------------------------------- multi-threshold deblending ---
# The paper's detection takes local maxima and does not deblend; the
# segments of the SExtractor reading are split by multi-thresholding
# [R33]-[R37]: levels of the significance nu = F / sigma between the
# threshold and the segment's peak; the branches (components) of each level
# set form a tree by containment; a branch is significant when its sum of m
# exceeds mincont times the segment's and it has minarea pixels; a branch
# with two or more significant children splits, each significant child
# being examined in turn; the other pixels go to the seeds by growth within
# the level sets, from the highest level down.
def _components(mask):
    """8-connected components of a small boolean mask: ids 1..n in raster
    order of their first pixel (0 outside)."""
    lab, _ = label(mask.astype(np.uint8), 1)
    u = np.unique(lab[lab > 0])
    ids = np.zeros(lab.shape, np.int64)
    for k, L in enumerate(u, 1):
        ids[lab == L] = k
    return ids, len(u)


def deblend_segment(nu, m, inseg, thresh, minarea, nthresh=32, mincont=0.005, margins=None):
    """One segment (the boolean map `inseg` over its bounding box, nu and m
    there): the object id of each of its pixels (0 outside; ids 1.. in the
    order of the seeds' first pixels), and the number of objects.  With a
    `margins` dict, it also records how close the decisions came to their
    bounds: the least relative distance of a pixel's nu to a level above
    the first ("nu"), and of a branch's sum of m to the contrast bound,
    relative to the segment's sum of |m| ("flux")."""
    npix = int(inseg.sum())
    total = float(m[inseg].sum())
    one = np.where(inseg, 1, 0)
    if margins is not None:
        margins.update(nu=np.inf, flux=np.inf)
    if npix < 2 * minarea or not total > 0:
        return one, 1
    numax = float(nu[inseg].max())
    if not numax > thresh:
        return one, 1
    levels = [thresh * (numax / thresh) ** (i / nthresh) for i in range(nthresh)]
    if margins is not None:
        v = nu[inseg]
        margins["nu"] = min(float(np.min(np.abs(v - t) / t)) for t in levels[1:]) if nthresh > 1 else np.inf
        sabs = float(np.abs(m[inseg]).sum())
    comp = []
    for i, t in enumerate(levels):                       # [R33][R34]
        q = inseg if i == 0 else (inseg & (nu > t))
        comp.append(_components(q)[0])

    def significant(i, c):                               # [R35]
        px = comp[i] == c
        f = float(m[px].sum())
        if margins is not None and px.sum() >= minarea:
            margins["flux"] = min(margins["flux"], abs(f - mincont * total) / sabs)
        return px.sum() >= minarea and f > mincont * total

    def children(i, c):
        if i + 1 >= nthresh:
            return []
        ids = np.unique(comp[i + 1][(comp[i] == c) & (comp[i + 1] > 0)])
        return [int(k) for k in ids]

    def objects(i, c):                                   # [R36]
        sig = [k for k in children(i, c) if significant(i + 1, k)]
        if len(sig) >= 2:
            out = []
            for k in sig:
                out += objects(i + 1, k)
            return out
        if len(sig) == 1:
            return objects(i + 1, sig[0])
        return [(i, c)]

    seeds = objects(0, 1)
    if len(seeds) < 2:
        return one, 1
    H, W = inseg.shape
    first = [int(np.flatnonzero((comp[i] == c).ravel())[0]) for i, c in seeds]
    order = np.argsort(first, kind="stable")
    own = np.zeros((H, W), np.int64)
    for k, j in enumerate(order, 1):
        i, c = seeds[j]
        own[comp[i] == c] = k
    for i in range(nthresh - 1, -1, -1):                 # [R37]
        q = inseg if i == 0 else (inseg & (nu > levels[i]))
        while True:
            big = np.iinfo(np.int64).max
            pad = np.pad(np.where(own > 0, own, big), 1, constant_values=big)
            best = np.full((H, W), big, np.int64)
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    if dy or dx:
                        best = np.minimum(best, pad[1 + dy:1 + dy + H, 1 + dx:1 + dx + W])
            grow = q & (own == 0) & (best < big)
            if not grow.any():
                break
            own = np.where(grow, best, own)
    return own, len(seeds)


def deblend(seg, nu, m, thresh, minarea, nthresh=32, mincont=0.005, margins=None):
    """The deblended segmentation map: every segment split into its objects,
    each labelled 1 + the minimum linear index of its pixels [R37].  With a
    `margins` dict: per segment label, its decision margins."""
    seg = np.asarray(seg)
    H, W = seg.shape
    out = seg.astype(np.uint32).copy()
    nsplit = 0
    for L in np.unique(seg[seg > 0]):
        ys, xs = np.nonzero(seg == L)
        y0, y1, x0, x1 = ys.min(), ys.max() + 1, xs.min(), xs.max() + 1
        inseg = seg[y0:y1, x0:x1] == L
        mg = {} if margins is not None else None
        own, n = deblend_segment(nu[y0:y1, x0:x1], m[y0:y1, x0:x1], inseg, thresh, minarea, nthresh, mincont, mg)
        if margins is not None:
            margins[int(L)] = mg
        if n < 2:
            continue
        nsplit += 1
        sub = out[y0:y1, x0:x1]
        for k in range(1, n + 1):
            py, px = np.nonzero(own == k)
            lab = 1 + min((y0 + py) * W + (x0 + px))
            sub[py, px] = lab
    return out, nsplit


# ------------------------------------------------------------ whole path ---
def extract(image, mesh, kernel, thresh, minarea, radii, gain, mask=None, saturation=0.0,
            fsize=3, clip_k=3.0, clip_maxiter=10):
    """The whole per-frame path in the paper's stage order: background and
    noise map, matched filter, threshold, labelling, moments, apertures at
    the centroids.  Returns a dict with every intermediate."""
    img, bad = pixel_values(image, mask)
    H, W = img.shape
    bkg_mesh, rms_mesh, st = background_meshes(img, bad, mesh, fsize, clip_k, clip_maxiter)
    bkg_map = spline_map(bkg_mesh, W, H, mesh)
    rms_map = spline_map(rms_mesh, W, H, mesh)
    m = np.where(bad != 0, 0.0, img - bkg_map)
    F = matched_filter(m, kernel)
    fg = threshold(F, rms_map, bad, thresh)
    seg, n = label(fg, minarea)
    sat = saturated(image, saturation)
    cat = moments(seg, m, sat)
    flux, err, apflags = apertures(m, rms_map ** 2, bad, sat, cat["x"], cat["y"], radii, gain)
    return dict(bkg_mesh=bkg_mesh, rms_mesh=rms_mesh, box=st, bkg_map=bkg_map, rms_map=rms_map,
                m=m, bad=bad, sat=sat, F=F, fg=fg, seg=seg, cat=cat, flux=flux, fluxerr=err,
                apflags=apflags, near=near_threshold(F, rms_map, thresh))
