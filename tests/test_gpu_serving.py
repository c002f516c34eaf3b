"""Batched extraction and the request server on the GPU.

A frame's results must not depend on what it ran with: the same frame gives
bit-identical segmentation maps, catalogs, apertures and meshes whether it
runs through gp_extract alone, in a batched launch with other frames, or
through the server alone or in a mix of concurrent requests.  The chain to
the oracle is gp_extract's parity (test_gpu_parity.py).  The server's
admission must keep its device use within the budget.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
gp = pytest.importorskip("paper_2609_32375_gb300")
from paper_2609_32375_gb300 import learned  # noqa: E402

pytestmark = pytest.mark.gpu

BASE = synth.CONFIGS["plain_2048x2048_u16"]
KERNEL = synth.gaussian_kernel(5, 3.0)
RADII = (3.0, 6.0)
MESH = 64

# (width, height, seed): several tiles and boxes with ragged tails
SIZES = [(2048, 1024, 11), (1000, 777, 12), (640, 480, 13), (1500, 1100, 14), (333, 190, 15), (1280, 1280, 16)]


def make(w, h, seed, dtype="u16"):
    cfg = synth.scaled_config(BASE, w, h)
    img, _ = synth.make_frame(cfg, seed, cache=False)
    if dtype == "f32":
        img = img.astype(np.float32)
    return img


@pytest.fixture(scope="module")
def frames():
    return [make(w, h, s) for w, h, s in SIZES]


@pytest.fixture(scope="module")
def ctx():
    c = gp.Context(0, workspace_bytes=1 << 30)
    yield c
    c.close()


def single(ctx, img, capacity=20000, net=None):
    t = torch.from_numpy(img).cuda()
    ex = gp.Extractor(ctx, img.shape, t.dtype, MESH, KERNEL, 1.5, 5, RADII, 1.5, capacity, device="cuda", net=net)
    ex.run(t)
    ctx.sync()
    n, cat = ex.catalog_host()
    return {"n": n, "catalog": cat, "segmap": ex.out["segmap"].cpu().numpy(),
            "bkg_mesh": ex.out["bkg_mesh"].cpu().numpy(), "rms_mesh": ex.out["rms_mesh"].cpu().numpy()}


def same(a, b, what):
    assert a["n"] == b["n"], f"{what}: n {a['n']} != {b['n']}"
    for k in ("bkg_mesh", "rms_mesh"):
        assert np.array_equal(a[k], b[k]), f"{what}: {k}"
    if "segmap" in a and "segmap" in b:
        assert np.array_equal(a["segmap"].view(np.uint32), b["segmap"].view(np.uint32)), f"{what}: segmap"
    for k, v in a["catalog"].items():
        assert np.array_equal(v, b["catalog"][k]), f"{what}: column {k}"


def batched(ctx, imgs, capacity=20000, net=None):
    ts = [torch.from_numpy(i).cuda() for i in imgs]
    bx = gp.BatchExtractor(ctx, [i.shape for i in imgs], ts[0].dtype, MESH, KERNEL, 1.5, 5, RADII, 1.5, capacity,
                           device="cuda", net=net)
    bx.run(ts)
    ctx.sync()
    assert bx.status.cpu().numpy().tolist() == [0] * len(imgs)
    out = []
    for f in range(len(imgs)):
        n, cat = bx.catalog_host(f)
        o = bx.outs[f]
        out.append({"n": n, "catalog": cat, "segmap": o["segmap"].cpu().numpy(),
                    "bkg_mesh": o["bkg_mesh"].cpu().numpy(), "rms_mesh": o["rms_mesh"].cpu().numpy()})
    return out


# ------------------------------------------------------ batched launches ---
def test_batch_is_bit_identical_to_single_frames(ctx, frames):
    alone = [single(ctx, img) for img in frames]
    assert all(a["n"] > 10 for a in alone)
    together = batched(ctx, frames)
    for f, (a, b) in enumerate(zip(alone, together)):
        same(a, b, f"frame {f} {frames[f].shape}")
    # a different grouping and order gives the same per-frame results
    order = [3, 0, 5]
    again = batched(ctx, [frames[i] for i in order])
    for j, i in enumerate(order):
        same(alone[i], again[j], f"frame {i} regrouped")


def test_float32_batch(ctx):
    imgs = [make(700, 500, 21, "f32"), make(1024, 300, 22, "f32")]
    alone = [single(ctx, i) for i in imgs]
    for f, (a, b) in enumerate(zip(alone, batched(ctx, imgs))):
        same(a, b, f"f32 frame {f}")


def test_learned_batch_matches_single(ctx):
    net = learned.Network(seed=4)
    eq = [make(1024, 1024, 31), make(1024, 1024, 32), make(1024, 1024, 33)]    # one network pass
    mixed = [make(1024, 1024, 34), make(900, 700, 35)]                          # one pass per frame
    for imgs in (eq, mixed):
        alone = [single(ctx, i, net=net) for i in imgs]
        for f, (a, b) in enumerate(zip(alone, batched(ctx, imgs, net=net))):
            same(a, b, f"learned frame {f}")


def test_batch_rejects_mixed_dtypes_and_bad_sizes(ctx):
    a = torch.from_numpy(make(256, 256, 41)).cuda()
    b = torch.from_numpy(make(256, 256, 42, "f32")).cuda()
    bx = gp.BatchExtractor(ctx, [a.shape, b.shape], a.dtype, MESH, KERNEL, 1.5, 5, RADII, 1.5, 100)
    with pytest.raises(gp.GpError):
        bx.run([a, b])
    with pytest.raises(ValueError):
        gp.BatchExtractor(ctx, [a.shape] * (gp.GP_MAX_BATCH + 1), a.dtype, MESH, KERNEL, 1.5, 5, RADII, 1.5, 100)


# ------------------------------------------------------------ the server ---
def server(**kw):
    args = dict(device=0, hbm_budget=4 << 30, host_budget=1 << 30, slots=3, batch_pixels=2_500_000, max_batch=8,
                mesh=MESH, kernel=KERNEL, thresh=1.5, minarea=5, radii=RADII, gain=1.5)
    args.update(kw)
    return gp.Server(**args)


def pinned(img):
    t = torch.from_numpy(img).pin_memory()
    return t


def test_server_results_same_alone_and_in_the_mix(ctx, frames):
    big = make(3000, 2600, 51)                      # above batch_pixels: runs as its own unit
    imgs = frames + [big]
    ref = [single(ctx, i) for i in imgs]
    s1 = server(slots=1, max_batch=1)
    try:
        alone = []
        for img in imgs:
            t = s1.submit(pinned(img), 20000, want_segmap=True)
            r = s1.result(t)
            assert r["status"] == gp.GP_OK and r["batch"] == 1
            alone.append(r)
    finally:
        s1.close()
    for f, (a, b) in enumerate(zip(ref, alone)):
        same(a, b, f"server alone frame {f}")
    s3 = server()
    try:
        host = [pinned(i) for i in imgs]
        tickets = [s3.submit(h, 20000, want_segmap=True) for h in host + host[:3]]   # repeats mix in too
        mix = [s3.result(t) for t in tickets]
        st = s3.stats()
    finally:
        s3.close()
    for f, r in enumerate(mix):
        assert r["status"] == gp.GP_OK
        same(alone[f % len(imgs)], r, f"server mix request {f}")
    assert max(r["batch"] for r in mix) > 1, "no batching happened"
    assert st["completed"] == len(tickets) and st["failed"] == 0
    assert st["units"] < len(tickets)
    assert 0 < st["p50_ms"] <= st["p99_ms"] <= st["max_ms"]
    print({k: st[k] for k in ("units", "batched_frames", "p50_ms", "p99_ms", "peak_inflight", "peak_bytes")})


def test_server_learned_background(ctx):
    net = learned.Network(seed=5)
    imgs = [make(1024, 1024, 61), make(1024, 1024, 62), make(1024, 1024, 63), make(800, 600, 64)]
    ref = [single(ctx, i, net=net) for i in imgs]
    s = server(net=net)
    try:
        ts = [s.submit(pinned(i), 20000, want_segmap=True) for i in imgs]
        res = [s.result(t) for t in ts]
    finally:
        s.close()
    for f, (a, b) in enumerate(zip(ref, res)):
        same(a, b, f"learned server frame {f}")


def test_admission_keeps_within_the_budget():
    img = make(2048, 2048, 71)
    probe = server()
    try:
        dev_bytes, host_bytes = probe.request_bytes(img, 20000)
    finally:
        probe.close()
    assert dev_bytes > img.nbytes * 3          # pixels, segmentation map and workspace at least
    for units_fit in (1, 2):
        budget = int(dev_bytes * (units_fit + 0.5))
        s = server(hbm_budget=budget, slots=4, max_batch=1)
        try:
            h = pinned(img)
            ts = [s.submit(h, 20000) for _ in range(6)]
            res = [s.result(t) for t in ts]
            st = s.stats()
        finally:
            s.close()
        assert all(r["status"] == gp.GP_OK for r in res)
        assert len({r["n"] for r in res}) == 1
        assert st["peak_bytes"] <= budget
        assert st["peak_inflight"] <= units_fit
        print(units_fit, st["peak_inflight"], st["peak_bytes"], budget)


def test_request_larger_than_the_budget_is_refused():
    img = make(2048, 2048, 72)
    s = server(hbm_budget=16 << 20)          # below the pixels plus segmentation map alone
    try:
        with pytest.raises(gp.GpError) as e:
            s.submit(img, 20000)
        assert e.value.status == gp.GP_ERR_OOM
    finally:
        s.close()


def test_wait_timeout_capacity_and_release():
    img = make(4096, 2048, 73)
    s = server()
    try:
        h = pinned(img)
        t = s.submit(h, 20000)
        try:
            s.wait(t, timeout_ms=0)          # either already done or a timeout, never a hang
        except gp.GpError as e:
            assert e.status == gp.GP_ERR_TIMEOUT
        r = s.result(t)
        assert r["status"] == gp.GP_OK and r["n"] > 10
        with pytest.raises(gp.GpError):
            s.release(t)                     # already released
        t2 = s.submit(h, 2)                  # far fewer rows than segments
        r2 = s.result(t2)
        assert r2["status"] == gp.GP_ERR_CAPACITY and r2["n"] == r["n"]
        assert len(r2["catalog"]["label"]) == 2
        np.testing.assert_array_equal(r2["catalog"]["label"], np.sort(r2["catalog"]["label"]))
    finally:
        s.close()


def test_shutdown_with_requests_queued():
    img = make(2048, 2048, 74)
    s = server(slots=1, max_batch=1)
    h = pinned(img)
    for _ in range(8):
        s.submit(h, 20000)
    s.close()                                # finishes what is in flight, fails the rest, frees



def test_strided_host_crop_matches_contiguous_copy():
    """A request may point at a crop of a larger host frame (row pitch >
    width); the server copies it with its pitch and gives the same results as
    for a contiguous copy of the crop."""
    img = make(1500, 900, 81)
    h = pinned(img)
    crop = h[100:700, 200:1300]
    s = server()
    try:
        a = s.result(s.submit(crop, 20000, want_segmap=True))
        b = s.result(s.submit(pinned(np.ascontiguousarray(img[100:700, 200:1300])), 20000, want_segmap=True))
    finally:
        s.close()
    assert a["status"] == b["status"] == gp.GP_OK and a["n"] > 0
    same(a, b, "strided crop")


def test_requests_arriving_while_others_run():
    """Continuous batching under arrival: a first wave is submitted, and once
    the server has work on the GPU (admitted, not finished), a second thread
    submits a second wave.  The late requests are admitted while earlier
    units are still in flight (several units on the device at once), and
    every result is bit-identical to the same frame run alone."""
    import threading
    import time

    CAP = 200000
    big = [make(8192, 8192, 81)]          # one long unit: its copies (frame in, map out) and kernels take a while
    small = [make(w, h, s) for w, h, s in SIZES[:4]]
    ctx1 = gp.Context(0, workspace_bytes=2 << 30)
    try:
        ref = {id(i): single(ctx1, i, capacity=CAP) for i in big + small}
    finally:
        ctx1.close()
    s = server(hbm_budget=8 << 30, slots=3)
    try:
        # the late frames are page-locked beforehand, so their submits take
        # microseconds and land while the first wave is on the GPU
        small_host = [pinned(i) for i in small]
        wave1 = [s.submit(pinned(i), CAP, want_segmap=True) for i in big]
        # wait until the server has admitted work that has not finished
        t0 = time.time()
        while True:
            st = s.stats()
            if st["peak_inflight"] >= 1 and st["completed"] < len(wave1):
                break
            assert time.time() - t0 < 30, "the first wave never showed work in flight"
            time.sleep(0.0005)
        seen = {}

        def late():
            seen["before"] = s.stats()
            seen["tickets"] = [s.submit(h, CAP, want_segmap=True) for h in small_host]
            seen["after"] = s.stats()

        th = threading.Thread(target=late)
        th.start()
        th.join()
        assert seen["before"]["completed"] < len(wave1), "the first wave finished before the late requests came"
        res1 = [s.result(t) for t in wave1]
        res2 = [s.result(t) for t in seen["tickets"]]
        st = s.stats()
    finally:
        s.close()
    for img, r in zip(big + small, res1 + res2):
        assert r["status"] == gp.GP_OK
        same(ref[id(img)], r, "request under arrival")
    assert st["completed"] == len(big) + len(small) and st["failed"] == 0
    # the first wave is one unit: two units in flight at once means a late one ran beside it
    assert st["peak_inflight"] >= 2, "the late requests never ran beside earlier ones"
    print({k: st[k] for k in ("units", "batched_frames", "peak_inflight", "p50_ms", "p99_ms")})
