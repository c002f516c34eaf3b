"""Learned background: training and inference driver over the C ABI.

The network (six 3x3 convolutions, 5 -> 32 -> 48 -> 48 -> 32 -> 32 -> 2)
maps one-pass per-box quantile features to the background / rms meshes.
Every layer, loss, gradient and optimiser step runs in the library's CUDA
kernels (gp_cnn_*); this module only owns the buffers and the schedule.
Targets come from the plain estimator (gp_background), which stays as the
fallback and as the reference for the network's error.

Training frames are drawn on the GPU with a seeded generator: sky level,
linear gradients, vignetting, moonlight ramps, random-field nebulosity and
500 to 20,000 Moffat stars, Poisson and read noise.  Their true sky is known,
so the held-out evaluation reports the error of both estimators against it.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import time
from dataclasses import dataclass

import numpy as np

from . import (GP_OK, GpBkg, GpBkgParams, GpCnnWeights, GpError, _check, load_library, make_image)

ARCH = (5, 32, 48, 48, 32, 32, 2)
CIP = (16, 32, 48, 48, 32, 32)      # padded input channels per layer
COP = (32, 48, 48, 32, 32, 16)      # padded output channels per layer
NSLOT = 64                          # weight-gradient partial slots
_STATE_LISTS = ("W", "b", "mW", "vW", "mb", "vb")   # per-layer tensors of the training state


def _s(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream or None


class Network:
    """Master weights (FP32) with AdamW state, and their packed BF16 forms."""

    def __init__(self, device="cuda", seed=0):
        import torch
        self.device = torch.device(device)
        g = torch.Generator(device="cpu").manual_seed(seed)
        self.W, self.b = [], []
        for l in range(6):
            ci, co = ARCH[l], ARCH[l + 1]
            std = math.sqrt(2.0 / (ci * 9)) * (0.5 if l == 5 else 1.0)
            self.W.append((torch.randn((co, ci, 3, 3), generator=g) * std).to(self.device))
            self.b.append(torch.zeros(co, device=self.device))
        self.mW = [torch.zeros_like(w) for w in self.W]
        self.vW = [torch.zeros_like(w) for w in self.W]
        self.mb = [torch.zeros_like(b) for b in self.b]
        self.vb = [torch.zeros_like(b) for b in self.b]
        self.wt = [torch.zeros((COP[l], 9 * CIP[l]), dtype=torch.bfloat16, device=self.device) for l in range(6)]
        self.wtd = [torch.zeros((CIP[l], 9 * COP[l]), dtype=torch.bfloat16, device=self.device) for l in range(6)]
        self.bias = [torch.zeros(COP[l], device=self.device) for l in range(6)]
        self.step = 0
        self._lib = load_library()
        self.pack()

    # ------------------------------------------------------------ packing ---
    def pack(self, stream=None):
        for l in range(6):
            _check(self._lib.gp_cnn_pack(self.W[l].data_ptr(), self.b[l].data_ptr(), ARCH[l], ARCH[l + 1], CIP[l],
                                         COP[l], self.wt[l].data_ptr(), self.wtd[l].data_ptr(),
                                         self.bias[l].data_ptr(), _s(stream)))

    def weights(self) -> GpCnnWeights:
        w = GpCnnWeights()
        for l in range(6):
            w.wt[l] = self.wt[l].data_ptr()
            w.bias[l] = self.bias[l].data_ptr()
        return w

    def state_dict(self):
        """Master weights, biases, AdamW moments and the step count (CPU copies)."""
        d = {k: [t.cpu() for t in getattr(self, k)] for k in _STATE_LISTS}
        d["step"] = self.step
        return d

    def load_state_dict(self, d):
        """Restores what state_dict() gave; a dict with weights only (a
        trained-weights file) leaves the AdamW moments at zero."""
        for k in _STATE_LISTS:
            if k in d:
                for dst, src in zip(getattr(self, k), d[k]):
                    dst.copy_(src)
        self.step = d.get("step", 0)
        self.pack()

    # ------------------------------------------------------------ forward ---
    def forward(self, feat, stream=None):
        """feat: bf16 [N, H, W, 16].  Returns (activations, output) with the
        activations of every layer input (bf16 NHWC) and the output float32
        [N, H, W, 2]."""
        import torch
        N, H, Wd, _ = feat.shape
        acts = [feat]
        x = feat
        for l in range(6):
            last = l == 5
            if last:
                y = torch.empty((N, H, Wd, 2), dtype=torch.float32, device=self.device)
            else:
                y = torch.empty((N, H, Wd, COP[l]), dtype=torch.bfloat16, device=self.device)
            _check(self._lib.gp_cnn_conv3x3(x.data_ptr(), N, H, Wd, CIP[l], self.wt[l].data_ptr(),
                                            self.bias[l].data_ptr(), COP[l], 0 if last else 1, y.data_ptr(),
                                            1 if last else 0, 2, _s(stream)))
            if not last:
                acts.append(y)
            x = y
        return acts, x

    # ----------------------------------------------------------- backward ---
    def backward(self, acts, out, target, stream=None):
        """MSE gradients of every layer.  Returns (loss tensor, [(dW, db)])."""
        import torch
        N, H, Wd, _ = out.shape
        npos = N * H * Wd
        nb = 256
        dy = torch.empty((N, H, Wd, COP[5]), dtype=torch.bfloat16, device=self.device)
        part = torch.empty(nb, dtype=torch.float32, device=self.device)
        loss = torch.empty(1, dtype=torch.float32, device=self.device)
        _check(self._lib.gp_cnn_mse(out.data_ptr(), target.data_ptr(), npos, COP[5], dy.data_ptr(), part.data_ptr(),
                                    nb, loss.data_ptr(), _s(stream)))
        grads = [None] * 6
        maxw = max(COP[l] * CIP[l] for l in range(6))
        partial = torch.empty(NSLOT * 9 * maxw, dtype=torch.float32, device=self.device)
        bpart = torch.empty(NSLOT * 64, dtype=torch.float32, device=self.device)
        for l in range(5, -1, -1):
            if l == 5:
                dp = dy
            else:
                dp = torch.empty_like(acts[l + 1])
                _check(self._lib.gp_cnn_relu_backward(dy.data_ptr(), acts[l + 1].data_ptr(), dp.data_ptr(),
                                                      dp.numel(), _s(stream)))
            dW = torch.empty((ARCH[l + 1], ARCH[l], 3, 3), dtype=torch.float32, device=self.device)
            db = torch.empty(ARCH[l + 1], dtype=torch.float32, device=self.device)
            _check(self._lib.gp_cnn_conv3x3_wgrad(acts[l].data_ptr(), dp.data_ptr(), N, H, Wd, CIP[l], COP[l],
                                                  ARCH[l], ARCH[l + 1], NSLOT, partial.data_ptr(),
                                                  bpart.data_ptr(), dW.data_ptr(), db.data_ptr(), _s(stream)))
            grads[l] = (dW, db)
            if l > 0:
                dx = torch.empty((N, H, Wd, CIP[l]), dtype=torch.bfloat16, device=self.device)
                zero = torch.zeros(CIP[l], dtype=torch.float32, device=self.device)
                _check(self._lib.gp_cnn_conv3x3(dp.data_ptr(), N, H, Wd, COP[l], self.wtd[l].data_ptr(),
                                                zero.data_ptr(), CIP[l], 0, dx.data_ptr(), 0, 0, _s(stream)))
                dy = dx
        return loss, grads

    def adamw(self, grads, lr=2e-3, betas=(0.9, 0.999), eps=1e-8, wd=1e-4, stream=None):
        self.step += 1
        for l in range(6):
            dW, db = grads[l]
            _check(self._lib.gp_cnn_adamw(self.W[l].data_ptr(), dW.data_ptr(), self.mW[l].data_ptr(),
                                          self.vW[l].data_ptr(), self.W[l].numel(), lr, betas[0], betas[1], eps, wd,
                                          self.step, _s(stream)))
            _check(self._lib.gp_cnn_adamw(self.b[l].data_ptr(), db.data_ptr(), self.mb[l].data_ptr(),
                                          self.vb[l].data_ptr(), self.b[l].numel(), lr, betas[0], betas[1], eps, 0.0,
                                          self.step, _s(stream)))
        self.pack(stream)

    def train_step(self, feat, target, lr=2e-3, stream=None):
        acts, out = self.forward(feat, stream)
        loss, grads = self.backward(acts, out, target, stream)
        self.adamw(grads, lr=lr, stream=stream)
        return loss


# ----------------------------------------------------------- features ---
def box_quantiles(ctx, img, mesh, stream=None):
    """[5, my, mx] float32 quantiles of one frame (one pass, gp_box_quantiles)."""
    import torch
    H, W = img.shape
    mx, my = -(-W // mesh), -(-H // mesh)
    q = torch.empty((5, my, mx), dtype=torch.float32, device=img.device)
    gi = make_image(img)
    _check(load_library().gp_box_quantiles(ctx.handle, C.byref(gi), mesh, q.data_ptr(), _s(stream)))
    return q


def features(quant, stream=None):
    """quant [N, 5, my, mx] -> (feat bf16 [N, my, mx, 16], norm [N, 2])."""
    import torch
    N, _, my, mx = quant.shape
    feat = torch.empty((N, my, mx, 16), dtype=torch.bfloat16, device=quant.device)
    norm = torch.empty((N, 2), dtype=torch.float32, device=quant.device)
    _check(load_library().gp_cnn_features(quant.contiguous().data_ptr(), N, my * mx, feat.data_ptr(),
                                          norm.data_ptr(), _s(stream)))
    return feat, norm


def targets(bkg, rms, norm, stream=None):
    """plain meshes [N, my, mx] -> normalised targets [N, my, mx, 2]."""
    import torch
    N, my, mx = bkg.shape
    t = torch.empty((N, my, mx, 2), dtype=torch.float32, device=bkg.device)
    _check(load_library().gp_cnn_targets(bkg.contiguous().data_ptr(), rms.contiguous().data_ptr(), norm.data_ptr(),
                                         my * mx, N, t.data_ptr(), _s(stream)))
    return t


def denorm(out, norm, stream=None):
    import torch
    N, my, mx, _ = out.shape
    b = torch.empty((N, my, mx), dtype=torch.float32, device=out.device)
    r = torch.empty_like(b)
    _check(load_library().gp_cnn_denorm(out.data_ptr(), norm.data_ptr(), my * mx, N, b.data_ptr(), r.data_ptr(),
                                        _s(stream)))
    return b, r


def background_learned(ctx, img, mesh, net: Network, maps=False, stream=None):
    """gp_background_learned: meshes (and maps) from the network."""
    import torch
    H, W = img.shape
    mx, my = -(-W // mesh), -(-H // mesh)
    out = {"bkg_mesh": torch.empty((my, mx), dtype=torch.float32, device=img.device),
           "rms_mesh": torch.empty((my, mx), dtype=torch.float32, device=img.device), "mesh": mesh}
    if maps:
        out["bkg_map"] = torch.empty((H, W), dtype=torch.float32, device=img.device)
        out["rms_map"] = torch.empty((H, W), dtype=torch.float32, device=img.device)
    b = GpBkg(mesh, mx, my, out["bkg_mesh"].data_ptr(), out["rms_mesh"].data_ptr(),
              out["bkg_map"].data_ptr() if maps else None, out["rms_map"].data_ptr() if maps else None)
    p = GpBkgParams(mesh, 3, 3.0, 10)
    gi = make_image(img)
    w = net.weights()
    _check(load_library().gp_background_learned(ctx.handle, C.byref(gi), C.byref(p), C.byref(w), C.byref(b),
                                                _s(stream)))
    return out


# ------------------------------------------------- training frames (GPU) ---
@dataclass
class TrainFrame:
    image: object           # float32 [H, W] CUDA tensor
    sky: object             # float32 [H, W] noiseless sky (no stars)
    var: object             # float32 [H, W] noise variance of the sky


def training_frame(seed: int, size: int = 4096, device="cuda", read_noise=5.0, stars=(500, 20000)):
    """One seeded training frame drawn on the GPU: sky with a gradient,
    vignetting, a moonlight ramp and random-field nebulosity, a number of
    Moffat stars drawn log-uniformly from `stars` (beta 2.5, FWHM 2-5 px,
    F^-1.5 fluxes on [1e2, 1e5]), Poisson and read noise."""
    import torch
    import torch.nn.functional as Fn
    g = torch.Generator(device=device).manual_seed(int(seed))
    u = lambda *shape: torch.rand(shape, generator=g, device=device)
    H = W = size
    yy = torch.linspace(-1, 1, H, device=device)[:, None]
    xx = torch.linspace(-1, 1, W, device=device)[None, :]
    sky0 = 300 + 2700 * float(u(1))
    ang = 2 * math.pi * float(u(1))
    grad = 0.2 * sky0 * float(u(1)) * (xx * math.cos(ang) + yy * math.sin(ang))
    vig = 1 - 0.15 * float(u(1)) * (xx ** 2 + yy ** 2) / 2
    ang2 = 2 * math.pi * float(u(1))
    width = 0.2 + 0.8 * float(u(1))
    ramp = 0.3 * sky0 * float(u(1)) * torch.sigmoid((xx * math.cos(ang2) + yy * math.sin(ang2)) / width * 4)
    # nebulosity: white noise on a coarse grid, Gaussian low-pass, bilinear upsampling
    corr = 100 + 700 * float(u(1))
    gs = 32
    gh = H // gs + 2
    noise = torch.randn((gh, gh), generator=g, device=device)
    k = torch.fft.fftfreq(gh, device=device)
    filt = torch.exp(-2 * math.pi ** 2 * (k[:, None] ** 2 + k[None, :] ** 2) * (corr / gs) ** 2)
    field = torch.fft.ifft2(torch.fft.fft2(noise) * filt).real
    field = field / (field.std() + 1e-12) * 0.06 * sky0 * float(u(1))
    field = Fn.interpolate(field[None, None], size=(H, W), mode="bilinear", align_corners=False)[0, 0]
    sky = (sky0 + grad + ramp + field) * vig
    # stars
    lo, hi = float(stars[0]), float(stars[1])
    nstar = int(round(math.exp(math.log(lo) + (math.log(hi) - math.log(lo)) * float(u(1)))))
    xs = u(nstar) * W
    ys = u(nstar) * H
    fl = (1e2 ** -0.5 + u(nstar) * (1e5 ** -0.5 - 1e2 ** -0.5)) ** -2.0
    fwhm = 2 + 3 * u(nstar)
    beta = 2.5
    alpha = fwhm / (2 * math.sqrt(2 ** (1 / beta) - 1))
    R = 7
    off = torch.arange(-R, R + 1, device=device)
    ix = xs.round().long()[:, None, None] + off[None, None, :]
    iy = ys.round().long()[:, None, None] + off[None, :, None]
    r2 = ((ix.float() - xs[:, None, None]) ** 2 + (iy.float() - ys[:, None, None]) ** 2) / alpha[:, None, None] ** 2
    prof = (beta - 1) / (math.pi * alpha[:, None, None] ** 2) * (1 + r2) ** (-beta) * fl[:, None, None]
    ok = (ix >= 0) & (ix < W) & (iy >= 0) & (iy < H)
    lin = (iy * W + ix).expand_as(prof)[ok]
    stars = torch.zeros(H * W, device=device).index_add_(0, lin, prof.expand_as(ok.float())[ok]).view(H, W)
    lam = (sky + stars).clamp_min(0)
    img = torch.poisson(lam, generator=g) + read_noise * torch.randn((H, W), generator=g, device=device)
    return TrainFrame(img.float().contiguous(), sky.float(), (sky + read_noise ** 2).float())


def truth_meshes(frame: TrainFrame, mesh: int):
    """Box means of the true sky and of its noise sigma."""
    import torch.nn.functional as Fn
    H, W = frame.sky.shape
    b = Fn.avg_pool2d(frame.sky[None, None], mesh, ceil_mode=True)[0, 0]
    r = Fn.avg_pool2d(frame.var.sqrt()[None, None], mesh, ceil_mode=True)[0, 0]
    return b, r


def as_u16(img):
    """A float frame rounded and clamped to the uint16 range, as a uint16 tensor
    (the integer detour keeps to casts every torch build has)."""
    import torch
    v = img.round().clamp_(0, 65535).to(torch.int32)
    return torch.where(v > 32767, v - 65536, v).to(torch.int16).view(torch.uint16)


def build_dataset(ctx, n, seed0, size=4096, mesh=64, stream=None, stars=(500, 20000), u16=False):
    """Features, normalised plain targets, norms and truth meshes of n frames
    (as uint16 frames when `u16`)."""
    import torch
    quants, pb, pr, tb, tr = [], [], [], [], []
    for i in range(n):
        fr = training_frame(seed0 + i, size, stars=stars)
        img = as_u16(fr.image) if u16 else fr.image
        quants.append(box_quantiles(ctx, img, mesh, stream))
        plain = ctx.gp_background(img, mesh, stream=stream)
        pb.append(plain["bkg_mesh"])
        pr.append(plain["rms_mesh"])
        b, r = truth_meshes(fr, mesh)
        tb.append(b)
        tr.append(r)
    q = torch.stack(quants)
    feat, norm = features(q, stream)
    pb, pr = torch.stack(pb), torch.stack(pr)
    tgt = targets(pb, pr, norm, stream)
    ctx.sync(stream)
    return {"feat": feat, "norm": norm, "target": tgt, "plain_bkg": pb, "plain_rms": pr,
            "true_bkg": torch.stack(tb), "true_rms": torch.stack(tr)}


def train(net: Network, data, epochs=60, batch=32, lr=2e-3, seed=0, log=None, checkpoint=None):
    """Minibatch AdamW on the dataset; returns the per-epoch mean losses.

    With `checkpoint` (a file path), the whole training state -- weights,
    AdamW moments, step count, finished epochs and their losses -- is written
    there after every epoch, and a run that finds the file resumes after its
    last finished epoch: the permutations of the finished epochs are drawn
    again and discarded, and the learning-rate schedule is a function of the
    epoch, so the resumed run continues exactly as the uninterrupted one."""
    import torch
    n = data["feat"].shape[0]
    g = torch.Generator(device="cpu").manual_seed(seed)
    hist = []
    start = 0
    if checkpoint and os.path.exists(checkpoint):
        rec = load_checkpoint(net, checkpoint)
        if (rec["epochs"], rec["batch"], rec["seed"], rec["n"]) != (epochs, batch, seed, n):
            raise ValueError(f"checkpoint {checkpoint} is for another schedule: {rec}")
        hist = list(rec["losses"])
        start = len(hist)
        for _ in range(start):
            torch.randperm(n, generator=g)
    for ep in range(start, epochs):
        perm = torch.randperm(n, generator=g).to(data["feat"].device)
        losses = []
        lr_e = lr * 0.5 * (1 + math.cos(math.pi * ep / epochs))
        for s in range(0, n - batch + 1, batch):
            idx = perm[s:s + batch]
            loss = net.train_step(data["feat"][idx].contiguous(), data["target"][idx].contiguous(), lr=lr_e)
            losses.append(loss)
        hist.append(float(torch.stack(losses).mean()))
        if log:
            log(f"epoch {ep} loss {hist[-1]:.5f}")
        if checkpoint:
            save_checkpoint(net, checkpoint, {"epochs": epochs, "batch": batch, "seed": seed, "n": n,
                                              "losses": hist})
    return hist


def save_checkpoint(net, path: str, rec: dict):
    """The training state of `net` and the schedule record `rec` (epochs,
    batch, seed, n, losses so far) in one .npz, replaced atomically."""
    arrays = {f"{k}{l}": t.cpu().numpy() for k in _STATE_LISTS for l, t in enumerate(getattr(net, k))}
    arrays["step"] = np.array(net.step, dtype=np.int64)
    arrays["record"] = np.frombuffer(repr(rec).encode(), dtype=np.uint8)
    tmp = path + ".tmp.npz"
    np.savez(tmp, **arrays)
    os.replace(tmp, path)


def load_checkpoint(net, path: str) -> dict:
    """Restores a save_checkpoint() file into `net`; returns its record."""
    import ast

    import torch
    z = np.load(path)
    nl = len(net.W)
    d = {k: [torch.from_numpy(z[f"{k}{l}"]) for l in range(nl)] for k in _STATE_LISTS}
    d["step"] = int(z["step"])
    net.load_state_dict(d)
    return ast.literal_eval(bytes(z["record"]).decode())


def evaluate(net: Network, data):
    """Errors of the learned and plain meshes against the true sky (in units
    of the true per-pixel noise sigma) and of the learned against the plain."""
    import torch
    acts, out = net.forward(data["feat"])
    lb, lr_ = denorm(out, data["norm"])
    torch.cuda.synchronize()
    sig = data["true_rms"]
    e_plain = ((data["plain_bkg"] - data["true_bkg"]) / sig)
    e_learn = ((lb - data["true_bkg"]) / sig)
    e_lp = ((lb - data["plain_bkg"]) / sig)
    e_rms_plain = (data["plain_rms"] - sig) / sig
    e_rms_learn = (lr_ - sig) / sig
    rmsf = lambda e: float(e.pow(2).mean().sqrt())
    return {"bkg_rmse_plain_vs_truth": rmsf(e_plain), "bkg_rmse_learned_vs_truth": rmsf(e_learn),
            "bkg_rmse_learned_vs_plain": rmsf(e_lp), "rms_relerr_plain_vs_truth": rmsf(e_rms_plain),
            "rms_relerr_learned_vs_truth": rmsf(e_rms_learn)}


def time_background(ctx, img, mesh, net, reps=20):
    """Device time per call of the plain and the learned background stage."""
    import torch
    for _ in range(3):
        ctx.gp_background(img, mesh)
        background_learned(ctx, img, mesh, net)
    torch.cuda.synchronize()
    res = {}
    for name, fn in (("plain_ms", lambda: ctx.gp_background(img, mesh)),
                     ("learned_ms", lambda: background_learned(ctx, img, mesh, net))):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        torch.cuda.synchronize()
        res[name] = a.elapsed_time(b) / reps
    return res


# --------------------------------------------------------------- weights ---
def save(net: Network, path: str, meta=None):
    arrays = {f"W{l}": net.W[l].cpu().numpy() for l in range(6)}
    arrays.update({f"b{l}": net.b[l].cpu().numpy() for l in range(6)})
    if meta:
        arrays["meta"] = np.frombuffer(repr(meta).encode(), dtype=np.uint8)
    np.savez(path, **arrays)


def meta(path: str) -> dict:
    """The training record saved with a weights file (empty if none)."""
    import ast
    z = np.load(path)
    return ast.literal_eval(bytes(z["meta"]).decode()) if "meta" in z else {}


def weights_for_mesh(mesh: int):
    """The committed weights trained at this mesh size (None if there are none)."""
    import glob
    for p in sorted(glob.glob(os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights", "*.npz"))):
        if meta(p).get("mesh") == mesh:
            return p
    return None


def load(path: str, device="cuda") -> Network:
    import torch
    z = np.load(path)
    net = Network(device=device)
    net.load_state_dict({"W": [torch.from_numpy(z[f"W{l}"]) for l in range(6)],
                         "b": [torch.from_numpy(z[f"b{l}"]) for l in range(6)]})
    return net


def main(argv=None):
    """Train the network on seeded GPU-drawn frames and report its held-out
    errors and the background stage's time against the plain estimator."""
    import argparse
    import json

    import torch

    from . import Context
    ap = argparse.ArgumentParser(description=main.__doc__)
    ap.add_argument("--frames", type=int, default=2000)
    ap.add_argument("--held", type=int, default=200)
    ap.add_argument("--size", type=int, default=4096)
    ap.add_argument("--mesh", type=int, default=64)
    ap.add_argument("--epochs", type=int, default=60)
    ap.add_argument("--batch", type=int, default=32)
    ap.add_argument("--lr", type=float, default=3e-3)
    ap.add_argument("--stars-per-mp", type=float, nargs=2, default=None, metavar=("LO", "HI"),
                    help="stars per megapixel, drawn log-uniformly (default: 500-20,000 per frame)")
    ap.add_argument("--u16", action="store_true",
                    help="round the frames to uint16 (always for meshes above 128, which the float path does not take)")
    ap.add_argument("--out", default=None, help="write the trained weights (.npz)")
    ap.add_argument("--checkpoint", default=None,
                    help="training-state file, written after every epoch; an existing one is resumed")
    a = ap.parse_args(argv)
    u16 = a.u16 or a.mesh > 128
    stars = (500, 20000) if a.stars_per_mp is None else tuple(v * a.size * a.size / 1e6 for v in a.stars_per_mp)
    ctx = Context(0, workspace_bytes=1 << 30)
    t0 = time.time()
    train_set = build_dataset(ctx, a.frames, seed0=1_000_000, size=a.size, mesh=a.mesh, stars=stars, u16=u16)
    held = build_dataset(ctx, a.held, seed0=1_000_000 + a.frames, size=a.size, mesh=a.mesh, stars=stars, u16=u16)
    t_data = time.time() - t0
    net = Network(seed=0)
    t0 = time.time()
    hist = train(net, train_set, epochs=a.epochs, batch=a.batch, lr=a.lr, checkpoint=a.checkpoint)
    torch.cuda.synchronize()
    t_train = time.time() - t0
    ev = evaluate(net, held)
    frame = training_frame(1_000_000 + a.frames + a.held, a.size, stars=stars)
    tm = time_background(ctx, as_u16(frame.image) if u16 else frame.image, a.mesh, net)
    res = {"frames": a.frames, "held_out": a.held, "size": a.size, "mesh": a.mesh, "epochs": a.epochs,
           "stars": [round(v, 1) for v in stars], "u16": u16,
           "loss_first_epoch": hist[0], "loss_last_epoch": hist[-1], "data_s": round(t_data, 1),
           "train_s": round(t_train, 1), **{k: round(v, 5) for k, v in ev.items()},
           **{k: round(v, 4) for k, v in tm.items()}}
    if a.out:
        save(net, a.out, res)
    print(json.dumps(res), flush=True)
    ctx.close()


if __name__ == "__main__":
    main()
