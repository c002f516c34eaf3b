"""Seeded synthetic astronomical frames.

This module only *makes inputs*: sky, noise, Moffat stars, hot pixels and
cosmic-ray tracks, drawn from numpy's PCG64 generator so that a (config, seed)
pair gives the same frame on every machine.  It holds none of the extraction
method's arithmetic (no statistics, no filtering, no labelling, no apertures):
both the CUDA path and the CPU oracle take their inputs from here, and neither
imports the other.

The paper's 19 real frames (4.2 to 151.2 MP, 228 to 134,206 sources; the
dataset table of Section 5) are not public yet, so these frames stand in for
them with the sizes, value ranges and source densities the configurations
below state.

Moffat profile (used to render stars):
    I(r) = F (beta - 1) / (pi alpha^2 q) * (1 + r'^2 / alpha^2) ** (-beta),
    alpha = FWHM / (2 sqrt(2^(1/beta) - 1)),
with r' the elliptical radius for axis ratio q = 1 - e.
"""
from __future__ import annotations

import dataclasses
import hashlib
import os
from typing import Optional

import numpy as np

GENERATOR_VERSION = 3


def gaussian_kernel(size: int, fwhm: float) -> np.ndarray:
    """Un-normalised size x size Gaussian filter taps for a PSF of this FWHM.

    The extraction normalises the taps itself; this only supplies the input
    filter (the matched-filter kernel a user would pass)."""
    s = fwhm / (2.0 * np.sqrt(2.0 * np.log(2.0)))
    h = size // 2
    u = np.arange(-h, h + 1, dtype=np.float64)
    return np.exp(-(u[None, :] ** 2 + u[:, None] ** 2) / (2.0 * s * s)).astype(np.float32)


@dataclasses.dataclass(frozen=True)
class FrameConfig:
    """One workload: the frame recipe plus the extraction parameters."""
    name: str
    width: int
    height: int
    dtype: str                 # "f32" or "u16"
    mesh: int
    thresh: float
    minarea: int
    radii: tuple
    gain: float                # e-/ADU, also the aperture Poisson gain
    saturation: float          # <= 0: none
    nsrc: int
    sky: float
    read_noise_e: float
    fwhm: tuple                # (lo, hi): uniform per source
    ellipticity: tuple         # (lo, hi)
    flux_range: tuple          # power law dN/dF ~ F^-1.5 on this range (ADU)
    gradient: float = 0.0      # linear sky gradient across x (ADU)
    vignetting: float = 0.0    # fractional radial fall-off at the corner
    grf_std: float = 0.0       # Gaussian random field (ADU std)
    grf_corr: float = 300.0    # its correlation length (px)
    blend_frac: float = 0.0    # fraction of sources placed in close pairs
    hot_frac: float = 0.0
    n_cr: int = 0
    filter_size: int = 3       # mesh median filter
    clip_k: float = 3.0
    clip_maxiter: int = 10
    kernel_size: int = 5
    kernel_fwhm: float = 3.0
    beta: float = 2.5
    subsample: int = 3         # star rendering sub-pixel grid per axis
    stamp_radius: int = 12

    @property
    def kernel(self) -> np.ndarray:
        return gaussian_kernel(self.kernel_size, self.kernel_fwhm)

    @property
    def npix(self) -> int:
        return self.width * self.height


CONFIGS = {
    # 1 MP FP32, seed 0: 1000 ADU sky + 50 ADU gradient, Poisson + 5 ADU read
    # noise, 300 Moffat stars (beta 2.5, FWHM 3), F^-1.5 on [1e2, 1e5].
    "plain_1024x1024_f32": FrameConfig(
        name="plain_1024x1024_f32", width=1024, height=1024, dtype="f32", mesh=64,
        thresh=1.5, minarea=5, radii=(3.0, 5.0, 8.0), gain=1.0, saturation=0.0,
        nsrc=300, sky=1000.0, read_noise_e=5.0, fwhm=(3.0, 3.0), ellipticity=(0.0, 0.0),
        flux_range=(1e2, 1e5), gradient=50.0),
    # 4.2 MP uint16 CCD: 800 ADU sky, 2 % vignetting, gain 1.5, 8 e- read
    # noise, 2000 sources FWHM 2-5 with ellipticity 0-0.2, 0.05 % hot pixels,
    # 20 cosmic-ray tracks, saturation at 65535.
    "plain_2048x2048_u16": FrameConfig(
        name="plain_2048x2048_u16", width=2048, height=2048, dtype="u16", mesh=128,
        thresh=3.0, minarea=5, radii=(4.0, 8.0), gain=1.5, saturation=65535.0,
        nsrc=2000, sky=800.0, read_noise_e=8.0, fwhm=(2.0, 5.0), ellipticity=(0.0, 0.2),
        flux_range=(2e2, 2e5), vignetting=0.02, hot_frac=5e-4, n_cr=20),
    # 151.2 MP dense uint16 sCMOS: 134,000 sources, 5 % in blended pairs,
    # 2000 ADU sky + 5 % random-field nebulosity (corr. length 300 px),
    # 3 e- read noise.
    "dense_12288x12304_u16": FrameConfig(
        name="dense_12288x12304_u16", width=12288, height=12304, dtype="u16", mesh=256,
        thresh=1.5, minarea=5, radii=(3.0, 6.0, 10.0), gain=1.0, saturation=65535.0,
        nsrc=134000, sky=2000.0, read_noise_e=3.0, fwhm=(3.0, 3.0), ellipticity=(0.0, 0.0),
        flux_range=(1e2, 1e5), grf_std=100.0, grf_corr=300.0, blend_frac=0.05,
        subsample=1, stamp_radius=10),
}


def scaled_config(base: FrameConfig, width: int, height: int, nsrc: Optional[int] = None,
                  name: Optional[str] = None) -> FrameConfig:
    """The same recipe on another frame size (source density kept unless given)."""
    if nsrc is None:
        nsrc = max(1, int(round(base.nsrc * (width * height) / base.npix)))
    return dataclasses.replace(base, width=width, height=height, nsrc=nsrc,
                               name=name or f"{base.name}@{width}x{height}")


def moffat_alpha(fwhm, beta):
    return fwhm / (2.0 * np.sqrt(2.0 ** (1.0 / beta) - 1.0))


def power_law_fluxes(rng, n, lo, hi, slope=-1.5):
    """Inverse-CDF draw from dN/dF ~ F^slope on [lo, hi] (slope != -1)."""
    u = rng.random(n)
    a = slope + 1.0
    return (lo ** a + u * (hi ** a - lo ** a)) ** (1.0 / a)


def render_moffat(shape, xs, ys, fluxes, fwhm, ellip, theta, beta, radius, sub,
                  chunk=4096):
    """Add Moffat stars to a float64 image by sub-pixel sampling.

    Pixel (x, y) covers [x-1/2, x+1/2] x [y-1/2, y+1/2]; the profile is
    averaged over a sub x sub grid inside each pixel of a square stamp of
    half-side `radius` around the nearest pixel.  Light beyond the stamp is
    dropped (the truth table records the flux actually rendered)."""
    H, W = shape
    img = np.zeros(H * W, dtype=np.float64)
    rendered = np.zeros(len(xs), dtype=np.float64)
    off = np.arange(-radius, radius + 1)
    sp = (np.arange(sub) + 0.5) / sub - 0.5
    for c0 in range(0, len(xs), chunk):
        sl = slice(c0, c0 + chunk)
        x, y, f = xs[sl], ys[sl], fluxes[sl]
        al = moffat_alpha(fwhm[sl], beta)
        q = 1.0 - ellip[sl]
        ct, st = np.cos(theta[sl]), np.sin(theta[sl])
        ix = np.rint(x).astype(np.int64)
        iy = np.rint(y).astype(np.int64)
        px = ix[:, None, None] + off[None, None, :]          # (n,1,S)
        py = iy[:, None, None] + off[None, :, None]          # (n,S,1)
        acc = np.zeros((len(x), len(off), len(off)))
        for sy in sp:
            for sx in sp:
                dx = (px + sx) - x[:, None, None]
                dy = (py + sy) - y[:, None, None]
                u = dx * ct[:, None, None] + dy * st[:, None, None]
                v = (-dx * st[:, None, None] + dy * ct[:, None, None]) / q[:, None, None]
                r2 = (u * u + v * v) / (al[:, None, None] ** 2)
                acc += (1.0 + r2) ** (-beta)
        norm = f * (beta - 1.0) / (np.pi * al * al * q) / (sub * sub)
        acc *= norm[:, None, None]
        pxb = np.broadcast_to(px, acc.shape)
        pyb = np.broadcast_to(py, acc.shape)
        inside = (pxb >= 0) & (pxb < W) & (pyb >= 0) & (pyb < H)
        rendered[sl] = np.where(inside, acc, 0.0).sum(axis=(1, 2))
        lin = (pyb * W + pxb)[inside]
        img += np.bincount(lin, weights=acc[inside], minlength=H * W)
    return img.reshape(H, W), rendered


def _grf(rng, H, W, std, corr):
    """Smooth Gaussian random field: white noise on a coarse grid, Gaussian
    low-pass by FFT, bilinear upsampling, scaled to the requested std."""
    g = max(4, int(corr // 20))
    gh, gw = H // g + 2, W // g + 2
    noise = rng.standard_normal((gh, gw))
    ky = np.fft.fftfreq(gh)[:, None]
    kx = np.fft.rfftfreq(gw)[None, :]
    s = corr / g
    filt = np.exp(-2.0 * (np.pi ** 2) * (kx ** 2 + ky ** 2) * s * s)
    field = np.fft.irfft2(np.fft.rfft2(noise) * filt, s=(gh, gw))
    field *= std / field.std()
    # separable linear interpolation onto the pixel grid
    fx = (np.arange(W) + 0.5) / g
    fy = (np.arange(H) + 0.5) / g
    x0 = np.floor(fx).astype(np.int64)
    y0 = np.floor(fy).astype(np.int64)
    tx = fx - x0
    ty = fy - y0
    rows = field[:, x0] * (1 - tx) + field[:, x0 + 1] * tx          # (gh, W)
    return rows[y0, :] * (1 - ty)[:, None] + rows[y0 + 1, :] * ty[:, None]


def _cosmic_rays(rng, H, W, n):
    img = np.zeros((H, W))
    for _ in range(n):
        x0, y0 = rng.random() * W, rng.random() * H
        ang = rng.random() * np.pi
        length = rng.uniform(5, 60)
        width = int(rng.integers(1, 3))
        amp = rng.uniform(500, 2e4)
        t = np.arange(0.0, length, 0.5)
        xs = np.rint(x0 + t * np.cos(ang)).astype(np.int64)
        ys = np.rint(y0 + t * np.sin(ang)).astype(np.int64)
        steep = abs(np.sin(ang)) > 0.5          # thicken across the track
        for w in range(width):
            xx = xs + (w if steep else 0)
            yy = ys + (0 if steep else w)
            ok = (xx >= 0) & (xx < W) & (yy >= 0) & (yy < H)
            img[yy[ok], xx[ok]] = amp
    return img


def make_frame(cfg: FrameConfig, seed: int, cache: bool = True):
    """Render one frame.  Returns (image, truth): image is float32 or uint16
    (H, W) C-contiguous; truth holds the star table and the noiseless sky."""
    path = None
    if cache and cfg.npix >= 16 * 2 ** 20:
        d = os.environ.get("GPPHOT_SYNTH_CACHE", "/tmp/gpphot_synth_cache")
        key = hashlib.sha1(repr((GENERATOR_VERSION, cfg, seed)).encode()).hexdigest()[:16]
        path = os.path.join(d, f"{cfg.name}_{seed}_{key}.npz")
        if os.path.exists(path):
            z = np.load(path)
            truth = {k[6:]: z[k] for k in z.files if k.startswith("truth_")}
            return z["image"], truth
    rng = np.random.default_rng(seed)
    H, W = cfg.height, cfg.width
    n = cfg.nsrc
    npair = int(round(n * cfg.blend_frac / 2.0))
    nsingle = n - 2 * npair
    xs = rng.uniform(-0.5, W - 0.5, nsingle + npair)
    ys = rng.uniform(-0.5, H - 0.5, nsingle + npair)
    fwhm = rng.uniform(cfg.fwhm[0], cfg.fwhm[1], n)
    if npair:
        sep = rng.uniform(1.0, 2.0, npair) * fwhm[nsingle + npair:]
        ang = rng.uniform(0, 2 * np.pi, npair)
        xs = np.concatenate([xs, xs[nsingle:] + sep * np.cos(ang)])
        ys = np.concatenate([ys, ys[nsingle:] + sep * np.sin(ang)])
    fluxes = power_law_fluxes(rng, n, cfg.flux_range[0], cfg.flux_range[1])
    ellip = rng.uniform(cfg.ellipticity[0], cfg.ellipticity[1], n)
    theta = rng.uniform(0, np.pi, n)
    stars, rendered = render_moffat((H, W), xs, ys, fluxes, fwhm, ellip, theta, cfg.beta,
                                    cfg.stamp_radius, cfg.subsample)
    sky = np.full((H, W), cfg.sky)
    if cfg.gradient:
        sky += cfg.gradient * (np.arange(W) / max(W - 1, 1))[None, :]
    if cfg.vignetting:
        cx, cy = (W - 1) / 2.0, (H - 1) / 2.0
        rx = ((np.arange(W) - cx) ** 2)[None, :]
        ry = ((np.arange(H) - cy) ** 2)[:, None]
        sky *= 1.0 - cfg.vignetting * (rx + ry) / (cx * cx + cy * cy)
    if cfg.grf_std:
        sky += _grf(rng, H, W, cfg.grf_std, cfg.grf_corr)
    lam = sky + stars                                    # ADU
    electrons = rng.poisson(np.maximum(lam * cfg.gain, 0.0)).astype(np.float64)
    electrons += rng.standard_normal((H, W)) * cfg.read_noise_e
    adu = electrons / cfg.gain
    if cfg.n_cr:
        adu += _cosmic_rays(rng, H, W, cfg.n_cr)
    if cfg.hot_frac:
        nh = int(round(cfg.hot_frac * H * W))
        idx = rng.choice(H * W, nh, replace=False)
        adu.reshape(-1)[idx] = rng.uniform(5e3, 65535, nh)
    if cfg.dtype == "u16":
        image = np.clip(np.rint(adu), 0, 65535).astype(np.uint16)
    else:
        image = adu.astype(np.float32)
    truth = {"x": xs, "y": ys, "flux": fluxes, "flux_rendered": rendered, "fwhm": fwhm,
             "sky_mean": np.float64(sky.mean())}
    if path is not None:
        try:
            os.makedirs(os.path.dirname(path), exist_ok=True)
            tmp = path + f".{os.getpid()}.tmp.npz"
            np.savez(tmp, image=image, **{"truth_" + k: v for k, v in truth.items()})
            os.replace(tmp, path)
        except OSError:
            pass
    return np.ascontiguousarray(image), truth


def poisson_arrivals(rng, rate_hz: float, n: int) -> np.ndarray:
    """Arrival times (s) of a Poisson process of this rate."""
    return np.cumsum(rng.exponential(1.0 / rate_hz, n))
