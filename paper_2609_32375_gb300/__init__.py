"""GB300-native per-frame source extraction: Python binding of libgpphot.

A thin ctypes layer over the C ABI declared in include/gpphot.h.  It only
marshals arguments: torch supplies device memory and streams, every step of
the extraction runs in the library's CUDA kernels.  There is no fallback --
importing works without a GPU, but any call needs the compiled library and a
CUDA device and raises otherwise.

Entry points keep the C names (gp_background, gp_detect, gp_aperture,
gp_extract, gp_label_mask); `Context` and `Extractor` wrap them with tensor
allocation for convenience.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libgpphot.so")

GP_OK, GP_ERR_INVALID_ARG, GP_ERR_OOM, GP_ERR_CAPACITY, GP_ERR_CUDA, GP_ERR_TIMEOUT, \
    GP_ERR_NOT_IMPLEMENTED, GP_ERR_INTERNAL = range(8)
GP_U16, GP_F32 = 0, 1
GP_FLAG_SAT, GP_FLAG_CENTROID_FALLBACK, GP_FLAG_TRUNCATED, GP_FLAG_BAD = 1, 2, 4, 8
GP_GROWTH_MAX_NR, GP_GROWTH_MAX_R = 32, 255

STATUS_NAMES = {0: "GP_OK", 1: "GP_ERR_INVALID_ARG", 2: "GP_ERR_OOM", 3: "GP_ERR_CAPACITY", 4: "GP_ERR_CUDA",
                5: "GP_ERR_TIMEOUT", 6: "GP_ERR_NOT_IMPLEMENTED", 7: "GP_ERR_INTERNAL"}

EXPORTS = ("gp_ctx_create", "gp_ctx_destroy", "gp_last_error", "gp_ctx_sync", "gp_ctx_set_timing", "gp_ctx_stats",
           "gp_ctx_set_walk_limit", "gp_workspace_bytes",
           "gp_background", "gp_detect", "gp_aperture", "gp_growth", "gp_optimal_radius", "gp_detect_psf", "gp_cosmetic", "gp_deblend", "gp_extract", "gp_label_mask", "gp_background_static",
           "gp_background_learned", "gp_extract_learned", "gp_box_quantiles", "gp_cnn_conv3x3", "gp_cnn_conv3x3_wgrad",
           "gp_cnn_relu_backward", "gp_cnn_mse", "gp_cnn_pack", "gp_cnn_adamw", "gp_cnn_features", "gp_cnn_targets",
           "gp_cnn_denorm", "gp_extract_batch", "gp_server_create", "gp_server_submit", "gp_server_wait",
           "gp_server_release", "gp_server_stats", "gp_server_destroy", "gp_server_request_bytes")


class GpError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


# ------------------------------------------------------------ C structs ---
class GpImage(C.Structure):
    _fields_ = [("data", C.c_void_p), ("dtype", C.c_int), ("width", C.c_int32), ("height", C.c_int32),
                ("pitch", C.c_int64), ("mask", C.c_void_p), ("saturation", C.c_float)]


class GpBkgParams(C.Structure):
    _fields_ = [("mesh", C.c_int32), ("filter_size", C.c_int32), ("clip_k", C.c_float),
                ("clip_maxiter", C.c_int32)]


class GpBkg(C.Structure):
    _fields_ = [("mesh", C.c_int32), ("mx", C.c_int32), ("my", C.c_int32), ("bkg_mesh", C.c_void_p),
                ("rms_mesh", C.c_void_p), ("bkg_map", C.c_void_p), ("rms_map", C.c_void_p)]


class GpDetParams(C.Structure):
    _fields_ = [("kernel", C.POINTER(C.c_float)), ("kw", C.c_int32), ("kh", C.c_int32), ("thresh", C.c_float),
                ("minarea", C.c_int32), ("mask_out", C.c_void_p), ("nnear", C.c_void_p)]


class GpCatalog(C.Structure):
    _fields_ = [("capacity", C.c_int32), ("n", C.c_void_p), ("label", C.c_void_p), ("npix", C.c_void_p),
                ("flux_iso", C.c_void_p), ("x", C.c_void_p), ("y", C.c_void_p), ("x2", C.c_void_p),
                ("y2", C.c_void_p), ("xy", C.c_void_p), ("xmin", C.c_void_p), ("xmax", C.c_void_p),
                ("ymin", C.c_void_p), ("ymax", C.c_void_p), ("peak", C.c_void_p), ("xpeak", C.c_void_p),
                ("ypeak", C.c_void_p), ("flags", C.c_void_p)]


GP_NSTAGES = 7
STAGE_NAMES = ("box_stats", "mesh_spline", "threshold", "label_tiles", "tile_merge", "label_rank", "measure")


class GpStats(C.Structure):
    _fields_ = [("calls", C.c_int32), ("launches", C.c_int32), ("ms", C.c_float * GP_NSTAGES)]


class GpCnnWeights(C.Structure):
    _fields_ = [("wt", C.c_void_p * 6), ("bias", C.c_void_p * 6)]


class GpApParams(C.Structure):
    _fields_ = [("radii", C.POINTER(C.c_float)), ("nr", C.c_int32), ("gain", C.c_float)]


class GpDeblendParams(C.Structure):
    _fields_ = [("nthresh", C.c_int32), ("mincont", C.c_float)]


class GpCosmeticParams(C.Structure):
    _fields_ = [("rtn_t", C.c_float), ("cr_gain", C.c_float), ("cr_read_noise", C.c_float),
                ("cr_sigclip", C.c_float), ("cr_objlim", C.c_float)]


class GpPsfParams(C.Structure):
    _fields_ = [("p0", C.POINTER(C.c_float)), ("modes", C.POINTER(C.c_float)), ("K", C.c_int32), ("kw", C.c_int32),
                ("kh", C.c_int32), ("coef", C.c_void_p), ("tile", C.c_int32), ("thresh", C.c_float),
                ("minarea", C.c_int32)]


class GpRoptParams(C.Structure):
    _fields_ = [("radii", C.POINTER(C.c_int32)), ("nr", C.c_int32), ("gain", C.c_float), ("snr_min", C.c_float),
                ("d_iso", C.c_float)]


class GpRoptOut(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in ("flux", "fluxerr", "flags", "nu", "kopt", "calib", "kfinal", "flux_opt",
                                          "fluxerr_opt", "fit")]


GP_MAX_BATCH = 64


class GpFrame(C.Structure):
    _fields_ = [("image", GpImage), ("bkg", GpBkg), ("segmap", C.c_void_p), ("cat", GpCatalog),
                ("flux", C.c_void_p), ("fluxerr", C.c_void_p), ("apflags", C.c_void_p), ("status", C.c_void_p)]


class GpServerConfig(C.Structure):
    _fields_ = [("device", C.c_int32), ("hbm_budget", C.c_size_t), ("host_budget", C.c_size_t),
                ("slots", C.c_int32), ("batch_pixels", C.c_int64), ("max_batch", C.c_int32),
                ("bkg", GpBkgParams), ("det", GpDetParams), ("ap", GpApParams), ("net", C.c_void_p)]


class GpRequest(C.Structure):
    _fields_ = [("image", GpImage), ("capacity", C.c_int32), ("want_segmap", C.c_int32)]


class GpResult(C.Structure):
    _fields_ = [("status", C.c_int32), ("n", C.c_int32), ("cat", GpCatalog), ("flux", C.c_void_p),
                ("fluxerr", C.c_void_p), ("apflags", C.c_void_p), ("segmap", C.c_void_p), ("bkg_mesh", C.c_void_p),
                ("rms_mesh", C.c_void_p), ("mesh", C.c_int32), ("mx", C.c_int32), ("my", C.c_int32),
                ("batch", C.c_int32), ("latency_ms", C.c_double), ("queue_ms", C.c_double),
                ("h2d_ms", C.c_float), ("run_ms", C.c_float), ("d2h_ms", C.c_float)]


class GpServerReport(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("failed", C.c_int64), ("units", C.c_int64),
                ("batched_frames", C.c_int64), ("mpix", C.c_double), ("wall_s", C.c_double),
                ("p50_ms", C.c_double), ("p99_ms", C.c_double), ("mean_ms", C.c_double), ("max_ms", C.c_double),
                ("budget", C.c_size_t), ("peak_bytes", C.c_size_t), ("peak_inflight", C.c_int32)]


CATALOG_COLUMNS = (("label", "uint32"), ("npix", "int32"), ("flux_iso", "float64"), ("x", "float64"),
                   ("y", "float64"), ("x2", "float64"), ("y2", "float64"), ("xy", "float64"), ("xmin", "int32"),
                   ("xmax", "int32"), ("ymin", "int32"), ("ymax", "int32"), ("peak", "float32"),
                   ("xpeak", "int32"), ("ypeak", "int32"), ("flags", "uint32"))

_lib = None
_lib_lock = threading.Lock()


def library_path() -> str:
    return LIB_PATH


def load_library():
    """Load libgpphot.so (building it first if it is missing and nvcc is
    present).  Raises if it cannot be loaded: there is no fallback."""
    global _lib
    with _lib_lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            from . import _build
            _build.build()
        L = C.CDLL(LIB_PATH)
        vp, i32, st = C.c_void_p, C.c_int32, C.c_int
        L.gp_ctx_create.argtypes = [C.c_int, C.c_size_t, C.POINTER(C.c_void_p)]
        L.gp_ctx_create.restype = st
        L.gp_ctx_destroy.argtypes = [vp]
        L.gp_ctx_destroy.restype = None
        L.gp_last_error.argtypes = []
        L.gp_last_error.restype = C.c_char_p
        L.gp_ctx_sync.argtypes = [vp, vp]
        L.gp_ctx_sync.restype = st
        L.gp_ctx_set_timing.argtypes = [vp, i32]
        L.gp_ctx_set_timing.restype = st
        L.gp_ctx_set_walk_limit.argtypes = [vp, i32]
        L.gp_ctx_set_walk_limit.restype = st
        L.gp_ctx_stats.argtypes = [vp, C.POINTER(GpStats)]
        L.gp_ctx_stats.restype = st
        L.gp_workspace_bytes.argtypes = [i32, i32, i32, i32]
        L.gp_workspace_bytes.restype = C.c_size_t
        L.gp_background.argtypes = [vp, C.POINTER(GpImage), C.POINTER(GpBkgParams), C.POINTER(GpBkg), vp]
        L.gp_background.restype = st
        L.gp_detect.argtypes = [vp, C.POINTER(GpImage), C.POINTER(GpBkg), C.POINTER(GpDetParams), vp,
                                C.POINTER(GpCatalog), vp]
        L.gp_detect.restype = st
        L.gp_aperture.argtypes = [vp, C.POINTER(GpImage), C.POINTER(GpBkg), vp, vp, i32, C.POINTER(GpApParams),
                                  vp, vp, vp, vp]
        L.gp_aperture.restype = st
        L.gp_growth.argtypes = [vp, C.POINTER(GpImage), C.POINTER(GpBkg), vp, vp, i32, C.POINTER(C.c_int32), i32,
                                C.c_float, vp, vp, vp, vp]
        L.gp_growth.restype = st
        L.gp_optimal_radius.argtypes = [vp, C.POINTER(GpImage), C.POINTER(GpBkg), C.POINTER(GpDetParams),
                                        C.POINTER(GpCatalog), C.POINTER(GpRoptParams), C.POINTER(GpRoptOut), vp]
        L.gp_optimal_radius.restype = st
        L.gp_detect_psf.argtypes = [vp, C.POINTER(GpImage), C.POINTER(GpBkg), C.POINTER(GpPsfParams), vp,
                                    C.POINTER(GpCatalog), vp]
        L.gp_detect_psf.restype = st
        L.gp_cosmetic.argtypes = [vp, C.POINTER(GpImage), C.POINTER(GpCosmeticParams), vp, vp, vp, vp]
        L.gp_cosmetic.restype = st
        L.gp_deblend.argtypes = [vp, C.POINTER(GpImage), C.POINTER(GpBkg), C.POINTER(GpDetParams),
                                 C.POINTER(GpDeblendParams), vp, C.POINTER(GpCatalog), C.POINTER(GpCatalog), vp, vp]
        L.gp_deblend.restype = st
        L.gp_extract.argtypes = [vp, C.POINTER(GpImage), C.POINTER(GpBkgParams), C.POINTER(GpDetParams),
                                 C.POINTER(GpApParams), C.POINTER(GpBkg), vp, C.POINTER(GpCatalog), vp, vp, vp, vp]
        L.gp_extract.restype = st
        L.gp_label_mask.argtypes = [vp, vp, i32, i32, i32, vp, vp, vp]
        L.gp_label_mask.restype = st
        L.gp_background_static.argtypes = [C.POINTER(GpImage), C.POINTER(GpBkgParams), C.POINTER(GpBkg), vp]
        L.gp_background_static.restype = st
        i64, f = C.c_int64, C.c_float
        L.gp_background_learned.argtypes = [vp, C.POINTER(GpImage), C.POINTER(GpBkgParams), C.POINTER(GpCnnWeights),
                                            C.POINTER(GpBkg), vp]
        L.gp_box_quantiles.argtypes = [vp, C.POINTER(GpImage), i32, vp, vp]
        L.gp_extract_learned.argtypes = [vp, C.POINTER(GpImage), C.POINTER(GpBkgParams), C.POINTER(GpDetParams),
                                         C.POINTER(GpApParams), C.POINTER(GpCnnWeights), C.POINTER(GpBkg), vp,
                                         C.POINTER(GpCatalog), vp, vp, vp, vp]
        L.gp_cnn_conv3x3.argtypes = [vp, i32, i32, i32, i32, vp, vp, i32, i32, vp, i32, i32, vp]
        L.gp_cnn_conv3x3_wgrad.argtypes = [vp, vp, i32, i32, i32, i32, i32, i32, i32, i32, vp, vp, vp, vp, vp]
        L.gp_cnn_relu_backward.argtypes = [vp, vp, vp, i64, vp]
        L.gp_cnn_mse.argtypes = [vp, vp, i64, i32, vp, vp, i32, vp, vp]
        L.gp_cnn_pack.argtypes = [vp, vp, i32, i32, i32, i32, vp, vp, vp, vp]
        L.gp_cnn_adamw.argtypes = [vp, vp, vp, vp, i64, f, f, f, f, f, i32, vp]
        L.gp_cnn_features.argtypes = [vp, i32, i32, vp, vp, vp]
        L.gp_cnn_targets.argtypes = [vp, vp, vp, i32, i32, vp, vp]
        L.gp_cnn_denorm.argtypes = [vp, vp, i32, i32, vp, vp, vp]
        L.gp_extract_batch.argtypes = [vp, C.POINTER(GpFrame), i32, C.POINTER(GpBkgParams), C.POINTER(GpDetParams),
                                       C.POINTER(GpApParams), C.POINTER(GpCnnWeights), vp]
        L.gp_server_create.argtypes = [C.POINTER(GpServerConfig), C.POINTER(C.c_void_p)]
        L.gp_server_submit.argtypes = [vp, C.POINTER(GpRequest), C.POINTER(C.c_uint64)]
        L.gp_server_wait.argtypes = [vp, C.c_uint64, i32, C.POINTER(GpResult)]
        L.gp_server_release.argtypes = [vp, C.c_uint64]
        L.gp_server_stats.argtypes = [vp, C.POINTER(GpServerReport), i32]
        L.gp_server_destroy.argtypes = [vp]
        L.gp_server_destroy.restype = None
        L.gp_server_request_bytes.argtypes = [vp, C.POINTER(GpRequest), C.POINTER(C.c_size_t),
                                              C.POINTER(C.c_size_t)]
        for name in ("gp_extract_batch", "gp_server_create", "gp_server_submit", "gp_server_wait",
                     "gp_server_release", "gp_server_stats", "gp_server_request_bytes"):
            getattr(L, name).restype = st
        for name in ("gp_background_learned", "gp_extract_learned", "gp_box_quantiles", "gp_cnn_conv3x3", "gp_cnn_conv3x3_wgrad",
                     "gp_cnn_relu_backward", "gp_cnn_mse", "gp_cnn_pack", "gp_cnn_adamw", "gp_cnn_features",
                     "gp_cnn_targets", "gp_cnn_denorm"):
            getattr(L, name).restype = st
        _lib = L
        return L


def _check(status: int):
    if status != GP_OK:
        raise GpError(status, load_library().gp_last_error().decode(errors="replace"))


def _ptr(t) -> Optional[int]:
    return None if t is None else t.data_ptr()


def _stream_handle(stream) -> Optional[int]:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream or None


def make_image(img, mask=None, saturation: float = 0.0) -> GpImage:
    """GpImage for a 2-D CUDA tensor of uint16 or float32 (rows may be
    strided; columns must be contiguous)."""
    import torch
    if not img.is_cuda:
        raise ValueError("image must be a CUDA tensor")
    if img.dim() != 2 or img.stride(1) != 1:
        raise ValueError("image must be 2-D with contiguous rows")
    if img.dtype == torch.uint16:
        dt = GP_U16
    elif img.dtype == torch.float32:
        dt = GP_F32
    else:
        raise ValueError(f"unsupported dtype {img.dtype}")
    if mask is not None:
        if mask.dtype != torch.uint8 or not mask.is_contiguous() or tuple(mask.shape) != tuple(img.shape):
            raise ValueError("mask must be a contiguous uint8 tensor of the image's shape")
    H, W = img.shape
    return GpImage(img.data_ptr(), dt, W, H, img.stride(0), _ptr(mask), float(saturation))


def _taps(kernel):
    k = np.ascontiguousarray(np.asarray(kernel, dtype=np.float32))
    if k.ndim != 2:
        raise ValueError("kernel must be 2-D")
    return k, k.ctypes.data_as(C.POINTER(C.c_float))


def _radii(radii):
    r = np.ascontiguousarray(np.asarray(radii, dtype=np.float32).reshape(-1))
    return r, r.ctypes.data_as(C.POINTER(C.c_float))


def allocate_catalog(capacity: int, device):
    """Device tensors for a catalog of `capacity` rows and its GpCatalog."""
    import torch
    cols = {"n": torch.zeros(1, dtype=torch.int32, device=device)}
    for name, dt in CATALOG_COLUMNS:
        cols[name] = torch.zeros(max(capacity, 1), dtype=getattr(torch, dt), device=device)
    cat = GpCatalog(capacity, cols["n"].data_ptr(), *[cols[n].data_ptr() for n, _ in CATALOG_COLUMNS])
    return cols, cat


# ---------------------------------------------------------- the context ---
class Context:
    """One gp_ctx: a device and a workspace arena.  Calls on one context must
    be ordered (one stream); use one context per concurrent stream."""

    def __init__(self, device: int = 0, workspace_bytes: int = 0):
        L = load_library()
        h = C.c_void_p()
        _check(L.gp_ctx_create(int(device), int(workspace_bytes), C.byref(h)))
        self._h = h
        self.device = device

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            load_library().gp_ctx_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sync(self, stream=None):
        """Synchronise the stream and raise if the device reported an error."""
        _check(load_library().gp_ctx_sync(self._h, _stream_handle(stream)))

    def set_timing(self, enable: bool = True):
        _check(load_library().gp_ctx_set_timing(self._h, 1 if enable else 0))

    def set_walk_limit(self, steps: int = 0):
        """Bound on the steps of each union-find walk of the tile merge for
        later calls (0: the library default); see gp_ctx_set_walk_limit."""
        _check(load_library().gp_ctx_set_walk_limit(self._h, int(steps)))

    def stats(self):
        """Per-stage device milliseconds summed over the calls since the
        previous stats() (see gp_ctx_stats), the call count and the number of
        kernels the most recent call launched."""
        st = GpStats()
        _check(load_library().gp_ctx_stats(self._h, C.byref(st)))
        return {"calls": st.calls, "launches": st.launches,
                "ms": {n: float(st.ms[i]) for i, n in enumerate(STAGE_NAMES)}}

    # ------------------------------------------------------- operations ---
    def gp_background(self, img, mesh, filter_size=3, clip_k=3.0, clip_maxiter=10, mask=None, saturation=0.0,
                      maps=False, stream=None):
        import torch
        gi = make_image(img, mask, saturation)
        H, W = img.shape
        mx, my = -(-W // mesh), -(-H // mesh)
        out = {"bkg_mesh": torch.empty((my, mx), dtype=torch.float32, device=img.device),
               "rms_mesh": torch.empty((my, mx), dtype=torch.float32, device=img.device), "mesh": mesh}
        if maps:
            out["bkg_map"] = torch.empty((H, W), dtype=torch.float32, device=img.device)
            out["rms_map"] = torch.empty((H, W), dtype=torch.float32, device=img.device)
        b = GpBkg(mesh, mx, my, out["bkg_mesh"].data_ptr(), out["rms_mesh"].data_ptr(),
                  _ptr(out.get("bkg_map")), _ptr(out.get("rms_map")))
        p = GpBkgParams(mesh, filter_size, clip_k, clip_maxiter)
        _check(load_library().gp_background(self._h, C.byref(gi), C.byref(p), C.byref(b), _stream_handle(stream)))
        return out

    @staticmethod
    def _bkg_struct(bkg):
        my, mx = bkg["bkg_mesh"].shape
        return GpBkg(bkg["mesh"], mx, my, bkg["bkg_mesh"].data_ptr(), bkg["rms_mesh"].data_ptr(), None, None)

    def gp_detect(self, img, bkg, kernel, thresh, minarea, capacity, mask=None, saturation=0.0, mask_out=False,
                  count_near=False, stream=None):
        import torch
        gi = make_image(img, mask, saturation)
        H, W = img.shape
        k, kp = _taps(kernel)
        out = {"segmap": torch.empty((H, W), dtype=torch.int32, device=img.device)}
        if mask_out:
            out["mask"] = torch.empty((H, W), dtype=torch.uint8, device=img.device)
        if count_near:
            out["nnear"] = torch.zeros(1, dtype=torch.int32, device=img.device)
        dp = GpDetParams(kp, k.shape[1], k.shape[0], float(thresh), int(minarea), _ptr(out.get("mask")),
                         _ptr(out.get("nnear")))
        cols, cat = allocate_catalog(capacity, img.device)
        b = self._bkg_struct(bkg)
        _check(load_library().gp_detect(self._h, C.byref(gi), C.byref(b), C.byref(dp), out["segmap"].data_ptr(),
                                        C.byref(cat), _stream_handle(stream)))
        out["catalog"] = cols
        return out

    def gp_aperture(self, img, bkg, x, y, radii, gain=0.0, mask=None, saturation=0.0, stream=None):
        import torch
        gi = make_image(img, mask, saturation)
        r, rp = _radii(radii)
        n = int(x.numel())
        x = x.to(device=img.device, dtype=torch.float64).contiguous()
        y = y.to(device=img.device, dtype=torch.float64).contiguous()
        flux = torch.empty((max(n, 1), r.size), dtype=torch.float64, device=img.device)
        ferr = torch.empty_like(flux)
        fl = torch.empty((max(n, 1), r.size), dtype=torch.int32, device=img.device)
        ap = GpApParams(rp, r.size, float(gain))
        b = self._bkg_struct(bkg)
        _check(load_library().gp_aperture(self._h, C.byref(gi), C.byref(b), x.data_ptr(), y.data_ptr(), n,
                                          C.byref(ap), flux.data_ptr(), ferr.data_ptr(), fl.data_ptr(),
                                          _stream_handle(stream)))
        return flux[:n], ferr[:n], fl[:n]

    def gp_growth(self, img, bkg, x, y, radii, gain=0.0, mask=None, saturation=0.0, stream=None):
        """Top-hat growth curves at integer radii (strictly increasing)."""
        import torch
        gi = make_image(img, mask, saturation)
        r = np.ascontiguousarray(np.asarray(radii, dtype=np.int32).reshape(-1))
        n = int(x.numel())
        x = x.to(device=img.device, dtype=torch.float64).contiguous()
        y = y.to(device=img.device, dtype=torch.float64).contiguous()
        flux = torch.empty((max(n, 1), max(r.size, 1)), dtype=torch.float64, device=img.device)
        ferr = torch.empty_like(flux)
        fl = torch.empty((max(n, 1), max(r.size, 1)), dtype=torch.int32, device=img.device)
        b = self._bkg_struct(bkg)
        _check(load_library().gp_growth(self._h, C.byref(gi), C.byref(b), x.data_ptr(), y.data_ptr(), n,
                                        r.ctypes.data_as(C.POINTER(C.c_int32)), r.size, float(gain),
                                        flux.data_ptr(), ferr.data_ptr(), fl.data_ptr(), _stream_handle(stream)))
        return flux[:n], ferr[:n], fl[:n]

    def gp_deblend(self, img, bkg, kernel, thresh, minarea, segmap, catalog, nthresh=32, mincont=0.005,
                   obj_capacity=100000, mask=None, saturation=0.0, stream=None):
        """Multi-threshold deblending of `segmap` (modified in place) with its
        catalog `catalog` (device columns and count "n"); returns the objects'
        catalog and the counts (segments split, objects)."""
        import torch
        gi = make_image(img, mask, saturation)
        k, kp = _taps(kernel)
        dp = GpDetParams(kp, k.shape[1], k.shape[0], float(thresh), int(minarea), None, None)
        cap = int(catalog["x"].numel())
        cat = GpCatalog(cap, catalog["n"].data_ptr(), *[catalog[n].data_ptr() for n, _ in CATALOG_COLUMNS])
        cols, ocat = allocate_catalog(obj_capacity, img.device)
        counts = torch.zeros(2, dtype=torch.int32, device=img.device)
        p = GpDeblendParams(int(nthresh), float(mincont))
        b = self._bkg_struct(bkg)
        _check(load_library().gp_deblend(self._h, C.byref(gi), C.byref(b), C.byref(dp), C.byref(p), segmap.data_ptr(),
                                         C.byref(cat), C.byref(ocat), counts.data_ptr(), _stream_handle(stream)))
        return {"objects": cols, "counts": counts}

    def gp_cosmetic(self, img, rtn_t=0.0, cr_gain=0.0, cr_read_noise=0.0, cr_sigclip=4.5, cr_objlim=5.0, mask=None,
                    stream=None):
        """The cosmetic corrections (cosmic rays, then salt-and-pepper noise):
        the corrected float32 frame, per-pixel flags and the two counts."""
        import torch
        gi = make_image(img, mask, 0.0)
        H, W = img.shape
        out = {"image": torch.empty((H, W), dtype=torch.float32, device=img.device),
               "flags": torch.empty((H, W), dtype=torch.uint8, device=img.device),
               "counts": torch.zeros(2, dtype=torch.int32, device=img.device)}
        p = GpCosmeticParams(float(rtn_t), float(cr_gain), float(cr_read_noise), float(cr_sigclip), float(cr_objlim))
        _check(load_library().gp_cosmetic(self._h, C.byref(gi), C.byref(p), out["image"].data_ptr(),
                                          out["flags"].data_ptr(), out["counts"].data_ptr(), _stream_handle(stream)))
        return out

    def gp_detect_psf(self, img, bkg, p0, modes, coef, tile, thresh, minarea, capacity, mask=None, saturation=0.0,
                      stream=None):
        """The second detection pass with the spatially varying PSF
        P0 + sum_k c_k e_k; coef: device tensor [K, ceil(H/tile), ceil(W/tile)]."""
        import torch
        gi = make_image(img, mask, saturation)
        p0 = np.ascontiguousarray(np.asarray(p0, dtype=np.float32))
        kh, kw = p0.shape
        modes = np.ascontiguousarray(np.asarray(modes, dtype=np.float32).reshape(-1, kh, kw))
        K = modes.shape[0]
        if K:
            coef = coef.to(device=img.device, dtype=torch.float32).contiguous()
        H, W = img.shape
        out = {"segmap": torch.empty((H, W), dtype=torch.int32, device=img.device)}
        cols, cat = allocate_catalog(capacity, img.device)
        p = GpPsfParams(p0.ctypes.data_as(C.POINTER(C.c_float)), modes.ctypes.data_as(C.POINTER(C.c_float)), K, kw,
                        kh, coef.data_ptr() if K else None, int(tile), float(thresh), int(minarea))
        b = self._bkg_struct(bkg)
        _check(load_library().gp_detect_psf(self._h, C.byref(gi), C.byref(b), C.byref(p), out["segmap"].data_ptr(),
                                            C.byref(cat), _stream_handle(stream)))
        out["catalog"] = cols
        return out

    def gp_optimal_radius(self, img, bkg, kernel, catalog, radii, gain=0.0, snr_min=50.0, d_iso=30.0, mask=None,
                          saturation=0.0, stream=None):
        """The optimal-radius step over a catalog's rows (device columns as
        gp_extract leaves them, with its count "n")."""
        import torch
        gi = make_image(img, mask, saturation)
        k, kp = _taps(kernel)
        dp = GpDetParams(kp, k.shape[1], k.shape[0], 1.0, 1, None, None)
        cap = int(catalog["x"].numel())
        cat = GpCatalog(cap, catalog["n"].data_ptr(), *[catalog[n].data_ptr() for n, _ in CATALOG_COLUMNS])
        r = np.ascontiguousarray(np.asarray(radii, dtype=np.int32).reshape(-1))
        dev = img.device
        nr = max(r.size, 1)
        out = {"flux": torch.empty((max(cap, 1), nr), dtype=torch.float64, device=dev),
               "fluxerr": torch.empty((max(cap, 1), nr), dtype=torch.float64, device=dev),
               "flags": torch.empty((max(cap, 1), nr), dtype=torch.int32, device=dev),
               "nu": torch.empty(max(cap, 1), dtype=torch.float32, device=dev),
               "kopt": torch.empty(max(cap, 1), dtype=torch.int32, device=dev),
               "calib": torch.empty(max(cap, 1), dtype=torch.uint8, device=dev),
               "kfinal": torch.empty(max(cap, 1), dtype=torch.int32, device=dev),
               "flux_opt": torch.empty(max(cap, 1), dtype=torch.float64, device=dev),
               "fluxerr_opt": torch.empty(max(cap, 1), dtype=torch.float64, device=dev),
               "fit": torch.empty(4, dtype=torch.float64, device=dev)}
        o = GpRoptOut(*[out[n].data_ptr() for n, _ in GpRoptOut._fields_])
        p = GpRoptParams(r.ctypes.data_as(C.POINTER(C.c_int32)), r.size, float(gain), float(snr_min), float(d_iso))
        b = self._bkg_struct(bkg)
        _check(load_library().gp_optimal_radius(self._h, C.byref(gi), C.byref(b), C.byref(dp), C.byref(cat),
                                                C.byref(p), C.byref(o), _stream_handle(stream)))
        return out

    def gp_extract(self, img, mesh, kernel, thresh, minarea, radii, gain, capacity, mask=None, saturation=0.0,
                   filter_size=3, clip_k=3.0, clip_maxiter=10, maps=False, mask_out=False, count_near=False,
                   stream=None):
        ex = Extractor(self, tuple(img.shape), img.dtype, mesh, kernel, thresh, minarea, radii, gain, capacity,
                       saturation=saturation, filter_size=filter_size, clip_k=clip_k, clip_maxiter=clip_maxiter,
                       maps=maps, mask_out=mask_out, count_near=count_near, device=img.device)
        ex.run(img, mask=mask, stream=stream)
        return ex.out

    def gp_label_mask(self, mask, minarea=1, stream=None):
        import torch
        if not mask.is_cuda or mask.dtype != torch.uint8 or not mask.is_contiguous():
            raise ValueError("mask must be a contiguous uint8 CUDA tensor")
        H, W = mask.shape
        seg = torch.empty((H, W), dtype=torch.int32, device=mask.device)
        n = torch.zeros(1, dtype=torch.int32, device=mask.device)
        _check(load_library().gp_label_mask(self._h, mask.data_ptr(), W, H, int(minarea), seg.data_ptr(),
                                            n.data_ptr(), _stream_handle(stream)))
        return seg, n


class Extractor:
    """Pre-allocated outputs for repeated gp_extract calls on frames of one
    shape: `run` allocates nothing, so it can be timed or captured."""

    def __init__(self, ctx: Context, shape, dtype, mesh, kernel, thresh, minarea, radii, gain, capacity,
                 saturation=0.0, filter_size=3, clip_k=3.0, clip_maxiter=10, maps=False, mask_out=False,
                 count_near=False, device="cuda", net=None):
        import torch
        self.ctx = ctx
        self.net = net          # learned.Network: use the learned background
        H, W = shape
        self.shape = (H, W)
        mx, my = -(-W // mesh), -(-H // mesh)
        self._k, kp = _taps(kernel)
        self._r, rp = _radii(radii)
        nr = self._r.size
        self.saturation = float(saturation)
        o = {"bkg_mesh": torch.empty((my, mx), dtype=torch.float32, device=device),
             "rms_mesh": torch.empty((my, mx), dtype=torch.float32, device=device), "mesh": mesh,
             "segmap": torch.empty((H, W), dtype=torch.int32, device=device)}
        if maps:
            o["bkg_map"] = torch.empty((H, W), dtype=torch.float32, device=device)
            o["rms_map"] = torch.empty((H, W), dtype=torch.float32, device=device)
        if mask_out:
            o["mask"] = torch.empty((H, W), dtype=torch.uint8, device=device)
        if count_near:
            o["nnear"] = torch.zeros(1, dtype=torch.int32, device=device)
        cols, self._cat = allocate_catalog(capacity, device)
        o["catalog"] = cols
        o["flux"] = torch.zeros((max(capacity, 1), max(nr, 1)), dtype=torch.float64, device=device)
        o["fluxerr"] = torch.zeros_like(o["flux"])
        o["apflags"] = torch.zeros((max(capacity, 1), max(nr, 1)), dtype=torch.int32, device=device)
        self.out = o
        self._bp = GpBkgParams(mesh, filter_size, clip_k, clip_maxiter)
        self._dp = GpDetParams(kp, self._k.shape[1], self._k.shape[0], float(thresh), int(minarea),
                               _ptr(o.get("mask")), _ptr(o.get("nnear")))
        self._ap = GpApParams(rp, nr, float(gain))
        self._bkg = GpBkg(mesh, mx, my, o["bkg_mesh"].data_ptr(), o["rms_mesh"].data_ptr(), _ptr(o.get("bkg_map")),
                          _ptr(o.get("rms_map")))
        self._lib = load_library()

    def run(self, img, mask=None, stream=None):
        gi = make_image(img, mask, self.saturation)
        if self.net is None:
            _check(self._lib.gp_extract(self.ctx.handle, C.byref(gi), C.byref(self._bp), C.byref(self._dp),
                                        C.byref(self._ap), C.byref(self._bkg), self.out["segmap"].data_ptr(),
                                        C.byref(self._cat), self.out["flux"].data_ptr(),
                                        self.out["fluxerr"].data_ptr(), self.out["apflags"].data_ptr(),
                                        _stream_handle(stream)))
        else:
            w = self.net.weights()
            _check(self._lib.gp_extract_learned(self.ctx.handle, C.byref(gi), C.byref(self._bp), C.byref(self._dp),
                                                C.byref(self._ap), C.byref(w), C.byref(self._bkg),
                                                self.out["segmap"].data_ptr(), C.byref(self._cat),
                                                self.out["flux"].data_ptr(), self.out["fluxerr"].data_ptr(),
                                                self.out["apflags"].data_ptr(), _stream_handle(stream)))
        return self.out

    def catalog_host(self):
        """Copy the catalog rows that were filled to host numpy arrays."""
        n = int(self.out["catalog"]["n"].item())
        m = min(n, self._cat.capacity)
        cat = {k: v[:m].cpu().numpy() for k, v in self.out["catalog"].items() if k != "n"}
        nr = self._r.size
        cat["flux"] = self.out["flux"][:m, :nr].cpu().numpy()
        cat["fluxerr"] = self.out["fluxerr"][:m, :nr].cpu().numpy()
        cat["apflags"] = self.out["apflags"][:m, :nr].cpu().numpy()
        return n, cat


class BatchExtractor:
    """Pre-allocated outputs for gp_extract_batch over a list of frame
    shapes (one dtype): `run(images)` extracts them all in one batched call.
    `outs[f]` has the layout of Extractor.out; `status` holds each frame's
    device status word."""

    def __init__(self, ctx: Context, shapes, dtype, mesh, kernel, thresh, minarea, radii, gain, capacity,
                 saturation=0.0, filter_size=3, clip_k=3.0, clip_maxiter=10, device="cuda", net=None):
        import torch
        self.ctx = ctx
        self.net = net
        self._k, kp = _taps(kernel)
        self._r, rp = _radii(radii)
        nr = self._r.size
        self.saturation = float(saturation)
        self.shapes = [tuple(s) for s in shapes]
        n = len(self.shapes)
        if not 1 <= n <= GP_MAX_BATCH:
            raise ValueError(f"batch of {n} frames outside [1, {GP_MAX_BATCH}]")
        caps = capacity if isinstance(capacity, (list, tuple)) else [capacity] * n
        self.status = torch.zeros(n, dtype=torch.int32, device=device)
        self.outs, self._cats = [], []
        for (H, W), cap in zip(self.shapes, caps):
            mx, my = -(-W // mesh), -(-H // mesh)
            cols, cat = allocate_catalog(cap, device)
            o = {"bkg_mesh": torch.empty((my, mx), dtype=torch.float32, device=device),
                 "rms_mesh": torch.empty((my, mx), dtype=torch.float32, device=device), "mesh": mesh,
                 "segmap": torch.empty((H, W), dtype=torch.int32, device=device), "catalog": cols,
                 "flux": torch.zeros((max(cap, 1), max(nr, 1)), dtype=torch.float64, device=device)}
            o["fluxerr"] = torch.zeros_like(o["flux"])
            o["apflags"] = torch.zeros((max(cap, 1), max(nr, 1)), dtype=torch.int32, device=device)
            self.outs.append(o)
            self._cats.append(cat)
        self._bp = GpBkgParams(mesh, filter_size, clip_k, clip_maxiter)
        self._dp = GpDetParams(kp, self._k.shape[1], self._k.shape[0], float(thresh), int(minarea), None, None)
        self._ap = GpApParams(rp, nr, float(gain))
        self._frames = (GpFrame * n)()
        self._lib = load_library()

    def run(self, images, stream=None):
        if len(images) != len(self.shapes):
            raise ValueError("one image per frame shape")
        self.status.zero_()
        for f, (img, o) in enumerate(zip(images, self.outs)):
            if tuple(img.shape) != self.shapes[f]:
                raise ValueError(f"frame {f}: shape {tuple(img.shape)} != {self.shapes[f]}")
            my, mx = o["bkg_mesh"].shape
            fr = self._frames[f]
            fr.image = make_image(img, None, self.saturation)
            fr.bkg = GpBkg(o["mesh"], mx, my, o["bkg_mesh"].data_ptr(), o["rms_mesh"].data_ptr(), None, None)
            fr.segmap = o["segmap"].data_ptr()
            fr.cat = self._cats[f]
            fr.flux, fr.fluxerr, fr.apflags = o["flux"].data_ptr(), o["fluxerr"].data_ptr(), o["apflags"].data_ptr()
            fr.status = self.status.data_ptr() + 4 * f
        w = self.net.weights() if self.net is not None else None
        _check(self._lib.gp_extract_batch(self.ctx.handle, self._frames, len(self.shapes), C.byref(self._bp),
                                          C.byref(self._dp), C.byref(self._ap),
                                          C.byref(w) if w is not None else None, _stream_handle(stream)))
        return self.outs

    def catalog_host(self, f):
        o = self.outs[f]
        n = int(o["catalog"]["n"].item())
        m = min(n, self._cats[f].capacity)
        cat = {k: v[:m].cpu().numpy() for k, v in o["catalog"].items() if k != "n"}
        nr = self._r.size
        cat["flux"] = o["flux"][:m, :nr].cpu().numpy()
        cat["fluxerr"] = o["fluxerr"][:m, :nr].cpu().numpy()
        cat["apflags"] = o["apflags"][:m, :nr].cpu().numpy()
        return n, cat


def _host_image(img, mask=None, saturation=0.0):
    """GpImage for a host frame (numpy array or CPU tensor, 2-D, contiguous
    rows) and the objects that keep its memory alive."""
    keep = []
    if hasattr(img, "numpy") and not isinstance(img, np.ndarray):
        if img.is_cuda:
            raise ValueError("server requests take host frames")
        keep.append(img)
        ptr, dt, shape, stride = img.data_ptr(), str(img.dtype).replace("torch.", ""), tuple(img.shape), img.stride(0)
    else:
        a = np.asarray(img)
        if a.ndim != 2 or a.strides[1] != a.itemsize:
            a = np.ascontiguousarray(a)
        keep.append(a)
        ptr, dt, shape, stride = a.ctypes.data, str(a.dtype), a.shape, a.strides[0] // a.itemsize
    if dt not in ("uint16", "float32"):
        raise ValueError(f"unsupported dtype {dt}")
    mptr = None
    if mask is not None:
        m = np.ascontiguousarray(np.asarray(mask, dtype=np.uint8))
        if m.shape != shape:
            raise ValueError("mask shape differs from the image")
        keep.append(m)
        mptr = m.ctypes.data
    H, W = shape
    return GpImage(ptr, GP_U16 if dt == "uint16" else GP_F32, W, H, stride, mptr, float(saturation)), keep


def _np_view(ptr, n, dtype):
    dt = np.dtype(dtype)
    if n == 0 or not ptr:
        return np.zeros(0, dt)
    buf = (C.c_char * (n * dt.itemsize)).from_address(ptr)
    return np.frombuffer(buf, dtype=dt, count=n)


class Server:
    """The request server (gp_server_*): frames from host memory in,
    catalogs out, with continuous batching under a device-memory budget.

    submit() returns a ticket at once; result() waits for it, copies the
    catalog into numpy arrays and frees the server's copy."""

    def __init__(self, device=0, hbm_budget=8 << 30, host_budget=1 << 30, slots=4, batch_pixels=4 << 20,
                 max_batch=16, mesh=64, filter_size=3, clip_k=3.0, clip_maxiter=10, kernel=None, thresh=1.5,
                 minarea=5, radii=(3.0,), gain=0.0, net=None):
        L = load_library()
        self._k, kp = _taps(kernel)
        self._r, rp = _radii(radii)
        self.net = net
        self._w = net.weights() if net is not None else None
        cfg = GpServerConfig(int(device), int(hbm_budget), int(host_budget), int(slots), int(batch_pixels),
                             int(max_batch), GpBkgParams(mesh, filter_size, clip_k, clip_maxiter),
                             GpDetParams(kp, self._k.shape[1], self._k.shape[0], float(thresh), int(minarea), None,
                                         None),
                             GpApParams(rp, self._r.size, float(gain)),
                             C.cast(C.pointer(self._w), C.c_void_p) if self._w is not None else None)
        h = C.c_void_p()
        _check(L.gp_server_create(C.byref(cfg), C.byref(h)))
        self._h = h
        self._keep = {}
        self._shape = {}
        self.nr = self._r.size

    def close(self):
        if getattr(self, "_h", None):
            load_library().gp_server_destroy(self._h)
            self._h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, img, capacity, mask=None, saturation=0.0, want_segmap=False) -> int:
        gi, keep = _host_image(img, mask, saturation)
        req = GpRequest(gi, int(capacity), 1 if want_segmap else 0)
        t = C.c_uint64()
        _check(load_library().gp_server_submit(self._h, C.byref(req), C.byref(t)))
        self._keep[t.value] = keep
        self._shape[t.value] = (gi.height, gi.width, int(capacity))
        return t.value

    def request_bytes(self, img, capacity, want_segmap=False):
        """(device bytes, host bytes) the admission rule charges for this
        request alone."""
        gi, keep = _host_image(img)
        req = GpRequest(gi, int(capacity), 1 if want_segmap else 0)
        d, h = C.c_size_t(), C.c_size_t()
        _check(load_library().gp_server_request_bytes(self._h, C.byref(req), C.byref(d), C.byref(h)))
        return d.value, h.value

    def wait(self, ticket, timeout_ms=-1) -> GpResult:
        res = GpResult()
        st = load_library().gp_server_wait(self._h, C.c_uint64(ticket), int(timeout_ms), C.byref(res))
        if st == GP_ERR_TIMEOUT and res.batch == 0:
            raise GpError(st, load_library().gp_last_error().decode(errors="replace"))
        return res

    def release(self, ticket):
        _check(load_library().gp_server_release(self._h, C.c_uint64(ticket)))
        self._keep.pop(ticket, None)
        self._shape.pop(ticket, None)

    def result(self, ticket, timeout_ms=-1):
        """Wait, copy the result to numpy arrays, release.  Returns a dict:
        status, n, catalog (columns of the rows filled, with flux, fluxerr,
        apflags), bkg/rms meshes, segmap (if asked), batch, latency_ms,
        queue_ms."""
        res = self.wait(ticket, timeout_ms)
        H, W, cap = self._shape[ticket]
        m = min(max(res.n, 0), cap) if res.status in (GP_OK, GP_ERR_CAPACITY) else 0
        out = {"status": res.status, "n": res.n, "batch": res.batch, "latency_ms": res.latency_ms,
               "queue_ms": res.queue_ms, "h2d_ms": res.h2d_ms, "run_ms": res.run_ms, "d2h_ms": res.d2h_ms}
        if res.status in (GP_OK, GP_ERR_CAPACITY):
            cat = {}
            for name, dt in CATALOG_COLUMNS:
                cat[name] = _np_view(getattr(res.cat, name), m, dt).copy()
            nr = self.nr
            cat["flux"] = _np_view(res.flux, m * nr, "float64").reshape(m, nr).copy()
            cat["fluxerr"] = _np_view(res.fluxerr, m * nr, "float64").reshape(m, nr).copy()
            cat["apflags"] = _np_view(res.apflags, m * nr, "uint32").reshape(m, nr).copy()
            out["catalog"] = cat
            out["bkg_mesh"] = _np_view(res.bkg_mesh, res.mx * res.my, "float32").reshape(res.my, res.mx).copy()
            out["rms_mesh"] = _np_view(res.rms_mesh, res.mx * res.my, "float32").reshape(res.my, res.mx).copy()
            if res.segmap:
                out["segmap"] = _np_view(res.segmap, H * W, "uint32").reshape(H, W).copy()
        else:
            out["error"] = load_library().gp_last_error().decode(errors="replace")
        self.release(ticket)
        return out

    def stats(self, reset=False):
        r = GpServerReport()
        _check(load_library().gp_server_stats(self._h, C.byref(r), 1 if reset else 0))
        return {k: getattr(r, k) for k, _ in GpServerReport._fields_}
