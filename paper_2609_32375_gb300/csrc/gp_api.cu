// gp_api.cu -- the C ABI (include/gpphot.h): context and workspace arena,
// host-side argument checks, and the launch sequence of each operation.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "gp_internal.cuh"
#include "gp_launch.h"
#include "gp_pipeline.h"

using namespace gp;

constexpr int RING = 256;
constexpr int NMARK = GP_NSTAGES + 1;

struct gp_ctx {
    int device;
    char* arena;
    size_t arena_bytes;
    int* dstatus;          // device status word (first bytes of the arena)
    char* base;            // first byte after the status block
    // stage timing
    int timing;
    cudaEvent_t ev[RING][NMARK];
    int ev_made;
    int nrec;              // calls recorded since the last gp_ctx_stats
    int slot;              // slot of the current call
    int launches;          // kernels launched by the current / last call
    int walk_limit;        // union-find walk bound of the tile merge (0: the library default)
    ArgStage stage;        // pinned staging of batched calls' argument records
    SideStream side;       // the crowded tiles' labelling beside the common form
    int side_made;
};

namespace {

thread_local std::string g_err;

gp_status fail(gp_status s, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

gp_status cuda_fail(cudaError_t e, const char* what)
{
    return fail(GP_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define GP_CUDA(call)                                   \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

// record the event of stage boundary k of the current call (timing on)
void mark(gp_ctx* ctx, int k, cudaStream_t st)
{
    if (ctx->timing) cudaEventRecord(ctx->ev[ctx->slot][k], st);
}

void begin_call(gp_ctx* ctx, cudaStream_t st)
{
    ctx->launches = 0;
    if (!ctx->timing) return;
    ctx->slot = ctx->nrec % RING;
    ctx->nrec++;
    mark(ctx, 0, st);
}

// mark boundaries from..to (stages the call does not run take no time)
void mark_to(gp_ctx* ctx, int from, int to, cudaStream_t st)
{
    for (int k = from; k <= to; ++k) mark(ctx, k, st);
}

constexpr size_t STATUS_BYTES = 256;

gp_status check_ctx(gp_ctx* ctx)
{
    if (!ctx) return fail(GP_ERR_INVALID_ARG, "null context");
    int dev = -1;
    GP_CUDA(cudaGetDevice(&dev));
    if (dev != ctx->device) GP_CUDA(cudaSetDevice(ctx->device));
    return GP_OK;
}

gp_status check_image(const gp_image* img)
{
    if (!img || !img->data) return fail(GP_ERR_INVALID_ARG, "null image or image data");
    if (img->dtype != GP_U16 && img->dtype != GP_F32) return fail(GP_ERR_INVALID_ARG, "dtype must be GP_U16 or GP_F32");
    if (img->width < 1 || img->height < 1) return fail(GP_ERR_INVALID_ARG, "image size %dx%d", img->width, img->height);
    if ((int64_t)img->width * img->height > 0x7fffffffll)
        return fail(GP_ERR_INVALID_ARG, "image of %lld pixels exceeds 2^31-1", (long long)img->width * img->height);
    if (img->pitch < img->width) return fail(GP_ERR_INVALID_ARG, "pitch %lld < width %d", (long long)img->pitch, img->width);
    return GP_OK;
}

Image to_image(const gp_image* img)
{
    Image im;
    im.data = img->data;
    im.pitch = img->pitch;
    im.mask = img->mask;
    im.W = img->width;
    im.H = img->height;
    im.sat = img->saturation;
    im.is_f32 = img->dtype == GP_F32;
    return im;
}

gp_status check_bkg_params(const gp_image* img, const gp_bkg_params* p)
{
    if (!p) return fail(GP_ERR_INVALID_ARG, "null background parameters");
    const int maxmesh = img->dtype == GP_U16 ? 256 : 128;
    if (p->mesh < 16 || p->mesh > maxmesh)
        return fail(GP_ERR_INVALID_ARG, "mesh %d outside [16, %d] for this dtype", p->mesh, maxmesh);
    if (p->filter_size < 1 || p->filter_size > 7 || !(p->filter_size & 1))
        return fail(GP_ERR_INVALID_ARG, "filter_size %d must be odd in [1, 7]", p->filter_size);
    if (!(p->clip_k >= 1.f) || !isfinite(p->clip_k)) return fail(GP_ERR_INVALID_ARG, "clip_k must be >= 1");
    if (p->clip_maxiter < 0 || p->clip_maxiter > 1000) return fail(GP_ERR_INVALID_ARG, "clip_maxiter out of range");
    return GP_OK;
}

gp_status check_bkg(const gp_image* img, const gp_bkg* b, bool need_meshes_only)
{
    if (!b || !b->bkg_mesh || !b->rms_mesh) return fail(GP_ERR_INVALID_ARG, "background meshes are null");
    if (b->mesh < 16) return fail(GP_ERR_INVALID_ARG, "background mesh %d < 16", b->mesh);
    const int mx = (img->width + b->mesh - 1) / b->mesh, my = (img->height + b->mesh - 1) / b->mesh;
    if (b->mx != mx || b->my != my)
        return fail(GP_ERR_INVALID_ARG, "background mesh %dx%d does not match the image (%dx%d)", b->mx, b->my, mx, my);
    (void)need_meshes_only;
    return GP_OK;
}

gp_status check_det(const gp_det_params* p, float* taps)
{
    if (!p || !p->kernel) return fail(GP_ERR_INVALID_ARG, "null detection parameters or kernel");
    if (p->kw < 1 || p->kh < 1 || !(p->kw & 1) || !(p->kh & 1) || p->kw > 2 * HMAX + 1 || p->kh > 2 * HMAX + 1)
        return fail(GP_ERR_INVALID_ARG, "kernel %dx%d must have odd sides <= %d", p->kw, p->kh, 2 * HMAX + 1);
    double s = 0;
    for (int i = 0; i < p->kw * p->kh; ++i) {
        if (!isfinite(p->kernel[i])) return fail(GP_ERR_INVALID_ARG, "kernel tap %d is not finite", i);
        s += p->kernel[i];
    }
    if (s == 0.0) return fail(GP_ERR_INVALID_ARG, "kernel taps sum to zero");
    for (int i = 0; i < p->kw * p->kh; ++i) taps[i] = (float)((double)p->kernel[i] / s);
    if (!(p->thresh > 0.f) || !isfinite(p->thresh)) return fail(GP_ERR_INVALID_ARG, "thresh must be > 0");
    if (p->minarea < 1) return fail(GP_ERR_INVALID_ARG, "minarea must be >= 1");
    return GP_OK;
}

gp_status check_ap(const gp_ap_params* p, bool allow_empty)
{
    if (!p) return fail(GP_ERR_INVALID_ARG, "null aperture parameters");
    if (p->nr < (allow_empty ? 0 : 1) || p->nr > MAX_NR) return fail(GP_ERR_INVALID_ARG, "nr %d outside [1, %d]", p->nr, MAX_NR);
    if (p->nr && !p->radii) return fail(GP_ERR_INVALID_ARG, "null radii");
    for (int k = 0; k < p->nr; ++k)
        if (!(p->radii[k] > 0.f) || p->radii[k] > 1024.f) return fail(GP_ERR_INVALID_ARG, "radius %d out of (0, 1024]", k);
    return GP_OK;
}

gp_status check_cat(const gp_catalog* c)
{
    if (!c || !c->n) return fail(GP_ERR_INVALID_ARG, "null catalog or count pointer");
    if (c->capacity < 0) return fail(GP_ERR_INVALID_ARG, "negative capacity");
    if (c->capacity > 0 && (!c->label || !c->npix || !c->flux_iso || !c->x || !c->y || !c->x2 || !c->y2 || !c->xy ||
                            !c->xmin || !c->xmax || !c->ymin || !c->ymax || !c->peak || !c->xpeak || !c->ypeak ||
                            !c->flags))
        return fail(GP_ERR_INVALID_ARG, "a catalog column is null");
    return GP_OK;
}

// spline tables of both maps from the (float) meshes in b; adds the number
// of kernels launched to *nlaunch
gp_status run_spline(Carver& cv, const gp_bkg* b, int W, int H, SplineTab* sb, SplineTab* sr, int* nlaunch,
                     cudaStream_t st)
{
    SplineWork w;
    const bool fused = mesh_fits_smem(b->mx, b->my);
    if (fused) {
        w.tab_b = cv.take<float4>((size_t)b->mx * b->my);
        w.tab_r = cv.take<float4>((size_t)b->mx * b->my);
    } else {
        carve_spline(cv, b->mx, b->my, w);
    }
    if (!cv.ok()) return GP_ERR_OOM;
    Axis ax = make_axis(W, b->mesh), ay = make_axis(H, b->mesh);
    if (fused) {
        GP_CUDA(launch_mesh_all(nullptr, nullptr, nullptr, ax, ay, 1, 1, b->bkg_mesh, b->rms_mesh, w.tab_b, w.tab_r,
                                st));
        *nlaunch += 1;
    } else {
        GP_CUDA(launch_spline_tables(b->bkg_mesh, ax, ay, w.scratch, w.tab_b, st));
        GP_CUDA(launch_spline_tables(b->rms_mesh, ax, ay, w.scratch, w.tab_r, st));
        *nlaunch += 4;
    }
    *sb = make_tab(w.tab_b, W, H, b->mesh);
    *sr = make_tab(w.tab_r, W, H, b->mesh);
    return GP_OK;
}

gp_status oom(const Carver& cv)
{
    return fail(GP_ERR_OOM, "workspace needs %zu bytes, the context arena has %zu", cv.off + STATUS_BYTES,
                cv.cap + STATUS_BYTES);
}

gp_status run_detect(gp_ctx* ctx, Carver& cv, const gp_image* img, const SplineTab& sb, const SplineTab& sr,
                     const float* taps, const gp_det_params* p, uint32_t* segmap, gp_catalog* cat,
                     const float* radii, int nr, float gain, double* flux, double* fluxerr, uint32_t* apflags,
                     cudaStream_t st)
{
    const int W = img->width, H = img->height;
    DetWork w;
    carve_det(cv, W, H, cat->capacity, w);
    if (!cv.ok()) return oom(cv);
    Image im = to_image(img);
    GP_CUDA(cudaMemsetAsync(w.zero, 0, (size_t)w.nzero * sizeof(int), st));
    if (p->nnear) GP_CUDA(cudaMemsetAsync(p->nnear, 0, sizeof(int), st));
    const DetectArgs A = detect_args(im, sb, sr, taps, p->kw, p->kh, p->thresh, p->minarea, segmap, p->mask_out,
                                     p->nnear, nullptr, w.D, w.T, w.P, w.C, ctx->dstatus);
    GP_CUDA(launch_stream_any(A, nullptr, 1, detect_grid(W, H, false), st));
    mark(ctx, 3, st);
    GP_CUDA(launch_label_any(A, nullptr, 1, st, ctx->side_made ? &ctx->side : nullptr));
    mark(ctx, 4, st);
    GP_CUDA(launch_resolve(w.T, w.P, w.C, w.D, segmap, W, H, p->minarea, ctx->walk_limit, ctx->dstatus, st));
    mark(ctx, 5, st);
    GP_CUDA(launch_rank(w.C, cat->n, cat->capacity, true, ctx->dstatus, st));
    mark(ctx, 6, st);
    GP_CUDA(launch_measure(im, sb, sr, w.C, segmap, *cat, radii, nr, gain, flux, fluxerr, apflags, st));
    mark(ctx, 7, st);
    ctx->launches += 1 + label_launches(false) + 4 + 4 + 1 + (nr > 0 ? 1 : 0);
    return GP_OK;
}

void ctx_mark(void* ud, int k, cudaStream_t st) { mark(static_cast<gp_ctx*>(ud), k, st); }

Exec ctx_exec(gp_ctx* ctx, cudaStream_t st)
{
    Exec ex;
    ex.cv = Carver{ctx->base, ctx->arena_bytes - STATUS_BYTES};
    ex.st = st;
    ex.stage = &ctx->stage;
    ex.side = ctx->side_made ? &ctx->side : nullptr;
    ex.mark = ctx_mark;
    ex.mark_ud = ctx;
    return ex;
}

// parameters shared by the frames of a call (dp, ap may be null for the
// background alone; taps already normalised by check_det)
Params make_params(const gp_bkg_params* bp, const float* taps, const gp_det_params* dp, const gp_ap_params* ap,
                   const gp_cnn_weights* net)
{
    Params P;
    memset(&P, 0, sizeof P);
    P.bp = *bp;
    if (dp) {
        for (int i = 0; i < dp->kw * dp->kh; ++i) P.taps[i] = taps[i];
        P.kw = dp->kw; P.kh = dp->kh;
        P.thresh = dp->thresh;
        P.minarea = dp->minarea;
    }
    if (ap) {
        P.nr = ap->nr;
        for (int k = 0; k < ap->nr; ++k) P.radii[k] = ap->radii[k];
        P.gain = ap->gain;
    }
    P.net = net;
    return P;
}

FrameIO frame_io(const gp_image* img, const gp_bkg* bkg, uint32_t* segmap, const gp_catalog* cat, double* flux,
                 double* fluxerr, uint32_t* apflags, const gp_det_params* dp, int* status)
{
    FrameIO F;
    memset(&F, 0, sizeof F);
    F.img = *img;
    F.bkg = *bkg;
    F.segmap = segmap;
    if (cat) F.cat = *cat;
    F.apflux = flux; F.apferr = fluxerr; F.apflags = apflags;
    if (dp) { F.mask_out = dp->mask_out; F.nnear = dp->nnear; }
    F.status = status;
    return F;
}

gp_status pipeline_result(gp_status s, const Exec& ex, gp_ctx* ctx)
{
    ctx->launches += ex.launches;
    if (s == GP_ERR_OOM)
        return fail(GP_ERR_OOM, "workspace needs %zu bytes, the context arena has %zu", ex.cv.off + STATUS_BYTES,
                    ex.cv.cap + STATUS_BYTES);
    return s;
}

gp_status check_net(const gp_cnn_weights* net);

// the background stage of one frame into bkg (clipped or learned)
gp_status background_call(gp_ctx* ctx, const gp_image* img, const gp_bkg_params* p, const gp_cnn_weights* net,
                          gp_bkg* bkg, gp_stream stream)
{
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    begin_call(ctx, st);
    Exec ex = ctx_exec(ctx, st);
    Params P = make_params(p, nullptr, nullptr, nullptr, net);
    P.walk_limit = ctx->walk_limit;
    FrameIO F = frame_io(img, bkg, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, ctx->dstatus);
    gp_status s = pipeline_result(run_background_only(ex, 1, &F, P), ex, ctx);
    bkg->mesh = F.bkg.mesh; bkg->mx = F.bkg.mx; bkg->my = F.bkg.my;
    return s;
}

gp_status extract_call(gp_ctx* ctx, const gp_image* img, const gp_bkg_params* bp, const gp_det_params* dp,
                       const gp_ap_params* ap, const gp_cnn_weights* net, gp_bkg* bkg, uint32_t* segmap,
                       gp_catalog* cat, double* flux, double* fluxerr, uint32_t* apflags, gp_stream stream)
{
    gp_status s;
    float taps[KMAX];
    if ((s = check_ctx(ctx)) != GP_OK) return s;
    if ((s = check_image(img)) != GP_OK) return s;
    if ((s = check_bkg_params(img, bp)) != GP_OK) return s;
    if (net && (s = check_net(net)) != GP_OK) return s;
    if ((s = check_det(dp, taps)) != GP_OK) return s;
    if ((s = check_ap(ap, true)) != GP_OK) return s;
    if ((s = check_cat(cat)) != GP_OK) return s;
    if (!bkg || !bkg->bkg_mesh || !bkg->rms_mesh) return fail(GP_ERR_INVALID_ARG, "null background output meshes");
    if (!segmap) return fail(GP_ERR_INVALID_ARG, "null segmap");
    if (ap->nr > 0 && cat->capacity > 0 && (!flux || !fluxerr || !apflags))
        return fail(GP_ERR_INVALID_ARG, "null aperture output array");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    begin_call(ctx, st);
    Exec ex = ctx_exec(ctx, st);
    Params P = make_params(bp, taps, dp, ap, net);
    P.walk_limit = ctx->walk_limit;
    FrameIO F = frame_io(img, bkg, segmap, cat, flux, fluxerr, apflags, dp, ctx->dstatus);
    s = pipeline_result(run_extract(ex, 1, &F, P), ex, ctx);
    bkg->mesh = F.bkg.mesh; bkg->mx = F.bkg.mx; bkg->my = F.bkg.my;
    return s;
}

}  // namespace

extern "C" {

const char* gp_last_error(void) { return g_err.c_str(); }

gp_status gp_ctx_create(int device, size_t workspace_bytes, gp_ctx** out)
{
    if (!out) return fail(GP_ERR_INVALID_ARG, "null output pointer");
    *out = nullptr;
    int n = 0;
    GP_CUDA(cudaGetDeviceCount(&n));
    if (device < 0 || device >= n) return fail(GP_ERR_INVALID_ARG, "device %d not present (%d devices)", device, n);
    GP_CUDA(cudaSetDevice(device));
    cudaDeviceProp prop;
    GP_CUDA(cudaGetDeviceProperties(&prop, device));
    if (prop.major * 10 + prop.minor < 100)
        return fail(GP_ERR_CUDA, "device %d is sm_%d%d; this library is built for sm_103a", device, prop.major, prop.minor);
    if (workspace_bytes == 0) workspace_bytes = (size_t)2 << 30;
    gp_ctx* c = new gp_ctx;
    c->device = device;
    c->timing = 0;
    c->ev_made = 0;
    c->nrec = 0;
    c->slot = 0;
    c->launches = 0;
    c->walk_limit = 0;
    c->side_made = 0;
    c->arena_bytes = workspace_bytes + STATUS_BYTES;
    cudaError_t e = cudaMalloc(&c->arena, c->arena_bytes);
    if (e != cudaSuccess) {
        delete c;
        return fail(GP_ERR_OOM, "cudaMalloc of %zu workspace bytes: %s", workspace_bytes, cudaGetErrorString(e));
    }
    c->dstatus = reinterpret_cast<int*>(c->arena);
    c->base = c->arena + STATUS_BYTES;
    e = cudaMemset(c->dstatus, 0, STATUS_BYTES);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        cudaFree(c->arena);
        delete c;
        return cuda_fail(e, "context initialisation");
    }
    // the side stream; without it the labelling forms run one after the other
    if (cudaStreamCreateWithFlags(&c->side.st, cudaStreamNonBlocking) == cudaSuccess) {
        if (cudaEventCreateWithFlags(&c->side.fork, cudaEventDisableTiming) == cudaSuccess) {
            if (cudaEventCreateWithFlags(&c->side.join, cudaEventDisableTiming) == cudaSuccess) c->side_made = 1;
            else cudaEventDestroy(c->side.fork);
        }
        if (!c->side_made) cudaStreamDestroy(c->side.st);
    }
    cudaGetLastError();
    *out = c;
    return GP_OK;
}

void gp_ctx_destroy(gp_ctx* ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    if (ctx->ev_made)
        for (int i = 0; i < RING; ++i)
            for (int k = 0; k < NMARK; ++k) cudaEventDestroy(ctx->ev[i][k]);
    ctx->stage.release();
    if (ctx->side_made) {
        cudaStreamSynchronize(ctx->side.st);
        cudaEventDestroy(ctx->side.fork);
        cudaEventDestroy(ctx->side.join);
        cudaStreamDestroy(ctx->side.st);
    }
    cudaFree(ctx->arena);
    delete ctx;
}

gp_status gp_ctx_set_timing(gp_ctx* ctx, int32_t enable)
{
    gp_status s = check_ctx(ctx);
    if (s != GP_OK) return s;
    if (enable && !ctx->ev_made) {
        for (int i = 0; i < RING; ++i)
            for (int k = 0; k < NMARK; ++k) GP_CUDA(cudaEventCreate(&ctx->ev[i][k]));
        ctx->ev_made = 1;
    }
    ctx->timing = enable ? 1 : 0;
    ctx->nrec = 0;
    return GP_OK;
}

gp_status gp_ctx_set_walk_limit(gp_ctx* ctx, int32_t steps)
{
    gp_status s = check_ctx(ctx);
    if (s != GP_OK) return s;
    if (steps < 0) return fail(GP_ERR_INVALID_ARG, "negative walk limit");
    ctx->walk_limit = steps;
    return GP_OK;
}

gp_status gp_ctx_stats(gp_ctx* ctx, gp_stats* out)
{
    gp_status s = check_ctx(ctx);
    if (s != GP_OK) return s;
    if (!out) return fail(GP_ERR_INVALID_ARG, "null stats output");
    memset(out, 0, sizeof *out);
    out->launches = ctx->launches;
    if (!ctx->ev_made) return GP_OK;
    const int n = ctx->nrec < RING ? ctx->nrec : RING;
    for (int i = 0; i < n; ++i) {
        GP_CUDA(cudaEventSynchronize(ctx->ev[i][NMARK - 1]));
        for (int k = 0; k < GP_NSTAGES; ++k) {
            float ms = 0.f;
            GP_CUDA(cudaEventElapsedTime(&ms, ctx->ev[i][k], ctx->ev[i][k + 1]));
            out->ms[k] += ms;
        }
    }
    out->calls = n;
    ctx->nrec = 0;
    return GP_OK;
}

gp_status gp_ctx_sync(gp_ctx* ctx, gp_stream stream)
{
    gp_status s = check_ctx(ctx);
    if (s != GP_OK) return s;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    GP_CUDA(cudaStreamSynchronize(st));
    int h = 0;
    GP_CUDA(cudaMemcpy(&h, ctx->dstatus, sizeof(int), cudaMemcpyDeviceToHost));
    GP_CUDA(cudaMemset(ctx->dstatus, 0, sizeof(int)));
    if (h == GP_ERR_CAPACITY) return fail(GP_ERR_CAPACITY, "more segments than catalog rows (see *cat.n)");
    if (h == GP_ERR_TIMEOUT) return fail(GP_ERR_TIMEOUT, "a bounded device-side walk gave up");
    if (h == GP_ERR_INTERNAL) return fail(GP_ERR_INTERNAL, "an internal device table overflowed; results are incomplete");
    if (h != 0) return fail((gp_status)h, "device status %d", h);
    return GP_OK;
}

size_t gp_workspace_bytes(int32_t width, int32_t height, int32_t mesh, int32_t capacity)
{
    if (width < 1 || height < 1 || mesh < 1) return 0;
    Carver cv{nullptr, 0};
    const int Mx = (width + mesh - 1) / mesh, My = (height + mesh - 1) / mesh;
    BkgWork b;
    carve_bkg(cv, Mx * My, b);
    SplineWork s;
    carve_spline(cv, Mx, My, s);
    DetWork d;
    carve_det(cv, width, height, capacity > 0 ? capacity : 0, d);
    return cv.off + STATUS_BYTES + ALIGN;
}

gp_status gp_background(gp_ctx* ctx, const gp_image* img, const gp_bkg_params* p, gp_bkg* bkg, gp_stream stream)
{
    gp_status s;
    if ((s = check_ctx(ctx)) != GP_OK) return s;
    if ((s = check_image(img)) != GP_OK) return s;
    if ((s = check_bkg_params(img, p)) != GP_OK) return s;
    if (!bkg || !bkg->bkg_mesh || !bkg->rms_mesh) return fail(GP_ERR_INVALID_ARG, "null background output meshes");
    return background_call(ctx, img, p, nullptr, bkg, stream);
}

gp_status gp_detect(gp_ctx* ctx, const gp_image* img, const gp_bkg* bkg, const gp_det_params* p, uint32_t* segmap,
                    gp_catalog* cat, gp_stream stream)
{
    gp_status s;
    float taps[(2 * HMAX + 1) * (2 * HMAX + 1)];
    if ((s = check_ctx(ctx)) != GP_OK) return s;
    if ((s = check_image(img)) != GP_OK) return s;
    if ((s = check_bkg(img, bkg, true)) != GP_OK) return s;
    if ((s = check_det(p, taps)) != GP_OK) return s;
    if ((s = check_cat(cat)) != GP_OK) return s;
    if (!segmap) return fail(GP_ERR_INVALID_ARG, "null segmap");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    Carver cv{ctx->base, ctx->arena_bytes - STATUS_BYTES};
    SplineTab sb, sr;
    begin_call(ctx, st);
    mark(ctx, 1, st);
    s = run_spline(cv, bkg, img->width, img->height, &sb, &sr, &ctx->launches, st);
    if (s == GP_ERR_OOM) return oom(cv);
    if (s != GP_OK) return s;
    mark(ctx, 2, st);
    return run_detect(ctx, cv, img, sb, sr, taps, p, segmap, cat, nullptr, 0, 0.f, nullptr, nullptr, nullptr, st);
}

gp_status gp_aperture(gp_ctx* ctx, const gp_image* img, const gp_bkg* bkg, const double* x, const double* y, int32_t n,
                      const gp_ap_params* p, double* flux, double* fluxerr, uint32_t* flags, gp_stream stream)
{
    gp_status s;
    if ((s = check_ctx(ctx)) != GP_OK) return s;
    if ((s = check_image(img)) != GP_OK) return s;
    if ((s = check_bkg(img, bkg, true)) != GP_OK) return s;
    if ((s = check_ap(p, false)) != GP_OK) return s;
    if (n < 0) return fail(GP_ERR_INVALID_ARG, "negative source count");
    if (n > 0 && (!x || !y || !flux || !fluxerr || !flags)) return fail(GP_ERR_INVALID_ARG, "null aperture array");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    Carver cv{ctx->base, ctx->arena_bytes - STATUS_BYTES};
    SplineTab sb, sr;
    begin_call(ctx, st);
    mark(ctx, 1, st);
    s = run_spline(cv, bkg, img->width, img->height, &sb, &sr, &ctx->launches, st);
    if (s == GP_ERR_OOM) return oom(cv);
    if (s != GP_OK) return s;
    mark_to(ctx, 2, GP_NSTAGES - 1, st);
    if (n > 0) {
        GP_CUDA(launch_aperture(to_image(img), sb, sr, x, y, n, p->radii, p->nr, p->gain, flux, fluxerr, flags, st));
        ctx->launches += 2;
    }
    mark(ctx, GP_NSTAGES, st);
    return GP_OK;
}

gp_status gp_growth(gp_ctx* ctx, const gp_image* img, const gp_bkg* bkg, const double* x, const double* y, int32_t n,
                    const int32_t* radii, int32_t nr, float gain, double* flux, double* fluxerr, uint32_t* flags,
                    gp_stream stream)
{
    gp_status s;
    if ((s = check_ctx(ctx)) != GP_OK) return s;
    if ((s = check_image(img)) != GP_OK) return s;
    if ((s = check_bkg(img, bkg, true)) != GP_OK) return s;
    if (!radii || nr < 1 || nr > GP_GROWTH_MAX_NR)
        return fail(GP_ERR_INVALID_ARG, "growth radii: need 1..%d of them", GP_GROWTH_MAX_NR);
    for (int k = 0; k < nr; ++k) {
        if (radii[k] < 0 || radii[k] > GP_GROWTH_MAX_R)
            return fail(GP_ERR_INVALID_ARG, "growth radius %d outside 0..%d", radii[k], GP_GROWTH_MAX_R);
        if (k > 0 && radii[k] <= radii[k - 1]) return fail(GP_ERR_INVALID_ARG, "growth radii not increasing");
    }
    if (n < 0) return fail(GP_ERR_INVALID_ARG, "negative source count");
    if (n > 0 && (!x || !y || !flux || !fluxerr || !flags)) return fail(GP_ERR_INVALID_ARG, "null growth array");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    Carver cv{ctx->base, ctx->arena_bytes - STATUS_BYTES};
    SplineTab sb, sr;
    begin_call(ctx, st);
    mark(ctx, 1, st);
    s = run_spline(cv, bkg, img->width, img->height, &sb, &sr, &ctx->launches, st);
    if (s == GP_ERR_OOM) return oom(cv);
    if (s != GP_OK) return s;
    mark_to(ctx, 2, GP_NSTAGES - 1, st);
    if (n > 0) {
        GP_CUDA(launch_growth(to_image(img), sb, sr, x, y, n, nullptr, radii, nr, gain, flux, fluxerr, flags, st));
        ctx->launches += 1;
    }
    mark(ctx, GP_NSTAGES, st);
    return GP_OK;
}

gp_status gp_deblend(gp_ctx* ctx, const gp_image* img, const gp_bkg* bkg, const gp_det_params* dp,
                     const gp_deblend_params* p, uint32_t* segmap, const gp_catalog* cat, gp_catalog* objects,
                     int32_t* counts, gp_stream stream)
{
    gp_status s;
    float taps[(2 * HMAX + 1) * (2 * HMAX + 1)];
    if ((s = check_ctx(ctx)) != GP_OK) return s;
    if ((s = check_image(img)) != GP_OK) return s;
    if ((s = check_bkg(img, bkg, true)) != GP_OK) return s;
    if ((s = check_det(dp, taps)) != GP_OK) return s;
    if ((s = check_cat(cat)) != GP_OK) return s;
    if ((s = check_cat(objects)) != GP_OK) return s;
    if (!p || !segmap || !counts) return fail(GP_ERR_INVALID_ARG, "null deblending parameters, segmap or counts");
    if (p->nthresh < 1 || p->nthresh > 64) return fail(GP_ERR_INVALID_ARG, "nthresh must be 1..64");
    if (!(p->mincont >= 0.f && p->mincont <= 1.f)) return fail(GP_ERR_INVALID_ARG, "mincont must be in [0, 1]");
    const int W = img->width, H = img->height;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    Carver cv{ctx->base, ctx->arena_bytes - STATUS_BYTES};
    SplineTab sb, sr;
    begin_call(ctx, st);
    mark(ctx, 1, st);
    s = run_spline(cv, bkg, W, H, &sb, &sr, &ctx->launches, st);
    if (s == GP_ERR_OOM) return oom(cv);
    if (s != GP_OK) return s;
    const int rows = cat->capacity > 0 ? cat->capacity : 1;
    DeblendWork w;
    w.cand = cv.take<int>(rows);
    w.cand_count = cv.take<int>(2);
    w.obj_count = w.cand_count + 1;
    w.off = cv.take<int64_t>(rows);
    w.obj_cap = objects->capacity > 0 ? objects->capacity : 1;
    w.obj = cv.take<DbObj>(w.obj_cap);
    w.scratch = cv.take<char>(0);                     // 256-byte aligned; the rest of the arena
    if (!cv.ok()) return oom(cv);
    w.scratch_bytes = (int64_t)(cv.cap - cv.off);
    mark_to(ctx, 2, GP_NSTAGES - 1, st);
    GP_CUDA(launch_deblend(to_image(img), sb, sr, taps, dp->kw, dp->kh, dp->thresh, dp->minarea, p->nthresh,
                           p->mincont, segmap, *cat, w, *objects, counts, ctx->dstatus, st));
    ctx->launches += 4;
    mark(ctx, GP_NSTAGES, st);
    return GP_OK;
}

gp_status gp_cosmetic(gp_ctx* ctx, const gp_image* img, const gp_cosmetic_params* p, float* out, uint8_t* flags,
                      int32_t* counts, gp_stream stream)
{
    gp_status s;
    if ((s = check_ctx(ctx)) != GP_OK) return s;
    if ((s = check_image(img)) != GP_OK) return s;
    if (!p || !out) return fail(GP_ERR_INVALID_ARG, "null parameters or output");
    const bool cr = p->cr_gain > 0.f, rtn = p->rtn_t > 0.f;
    if (!cr && !rtn) return fail(GP_ERR_INVALID_ARG, "both cosmetic filters are off");
    if (cr && (!(p->cr_read_noise > 0.f) || !std::isfinite(p->cr_gain) || !std::isfinite(p->cr_read_noise) ||
               !std::isfinite(p->cr_sigclip) || !std::isfinite(p->cr_objlim)))
        return fail(GP_ERR_INVALID_ARG, "cosmic-ray filter: finite parameters and read noise > 0 needed");
    if (rtn && !std::isfinite(p->rtn_t)) return fail(GP_ERR_INVALID_ARG, "salt-and-pepper threshold not finite");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    Carver cv{ctx->base, ctx->arena_bytes - STATUS_BYTES};
    const int W = img->width, H = img->height;
    float* mid = (cr && rtn) ? cv.take<float>((size_t)W * H) : nullptr;
    if (!cv.ok()) return oom(cv);
    begin_call(ctx, st);
    if (counts) GP_CUDA(cudaMemsetAsync(counts, 0, 2 * sizeof(int32_t), st));
    const Image im = to_image(img);
    if (cr) {
        GP_CUDA(launch_cr(im, p->cr_gain, p->cr_read_noise, p->cr_sigclip, p->cr_objlim, rtn ? mid : out, flags,
                          counts ? counts + 1 : nullptr, st));
        ctx->launches += 1;
    }
    if (rtn) {
        Image ir = im;
        if (cr) {
            ir.data = mid;
            ir.pitch = W;
            ir.is_f32 = 1;
        }
        const bool clean = !im.is_f32 && !im.mask;      // the cosmic-ray output of such a frame holds no NaN
        GP_CUDA(launch_rtn(ir, p->rtn_t, out, flags, cr, counts, clean, st));
        ctx->launches += 1;
    }
    mark_to(ctx, 1, GP_NSTAGES, st);
    return GP_OK;
}

gp_status gp_detect_psf(gp_ctx* ctx, const gp_image* img, const gp_bkg* bkg, const gp_psf_params* p, uint32_t* segmap,
                        gp_catalog* cat, gp_stream stream)
{
    gp_status s;
    if ((s = check_ctx(ctx)) != GP_OK) return s;
    if ((s = check_image(img)) != GP_OK) return s;
    if ((s = check_bkg(img, bkg, true)) != GP_OK) return s;
    if ((s = check_cat(cat)) != GP_OK) return s;
    if (!p || !segmap) return fail(GP_ERR_INVALID_ARG, "null PSF parameters or segmap");
    if (!p->p0 || p->K < 0 || p->K > GP_PSF_MAX_MODES || (p->K > 0 && (!p->modes || !p->coef)))
        return fail(GP_ERR_INVALID_ARG, "PSF model: need P0, and 0..%d modes with their coefficients", GP_PSF_MAX_MODES);
    if (p->kw < 1 || p->kh < 1 || !(p->kw & 1) || !(p->kh & 1) || p->kw > 2 * HMAX + 1 || p->kh > 2 * HMAX + 1)
        return fail(GP_ERR_INVALID_ARG, "PSF kernels %dx%d must have odd sides <= %d", p->kw, p->kh, 2 * HMAX + 1);
    if (p->tile < 1) return fail(GP_ERR_INVALID_ARG, "coefficient tile side must be >= 1");
    if (!(p->thresh > 0.f) || !std::isfinite(p->thresh)) return fail(GP_ERR_INVALID_ARG, "thresh must be > 0");
    if (p->minarea < 1) return fail(GP_ERR_INVALID_ARG, "minarea must be >= 1");
    for (int i = 0; i < p->kw * p->kh * (1 + p->K); ++i) {
        const float v = i < p->kw * p->kh ? p->p0[i] : p->modes[i - p->kw * p->kh];
        if (!std::isfinite(v)) return fail(GP_ERR_INVALID_ARG, "a PSF tap is not finite");
    }
    const int W = img->width, H = img->height;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    Carver cv{ctx->base, ctx->arena_bytes - STATUS_BYTES};
    SplineTab sb, sr;
    begin_call(ctx, st);
    mark(ctx, 1, st);
    s = run_spline(cv, bkg, W, H, &sb, &sr, &ctx->launches, st);
    if (s == GP_ERR_OOM) return oom(cv);
    if (s != GP_OK) return s;
    // the coefficient maps' spline tables
    const int cmx = (W + p->tile - 1) / p->tile, cmy = (H + p->tile - 1) / p->tile;
    SplineTab ct[GP_PSF_MAX_MODES];
    double* scratch = cv.take<double>(spline_scratch_doubles(cmx, cmy));
    float4* tabs = cv.take<float4>((size_t)cmx * cmy * (p->K > 0 ? p->K : 1));
    DetWork w;
    carve_det(cv, W, H, cat->capacity, w);
    if (!cv.ok()) return oom(cv);
    const Axis cax = make_axis(W, p->tile), cay = make_axis(H, p->tile);
    for (int k = 0; k < p->K; ++k) {
        float4* tab = tabs + (size_t)k * cmx * cmy;
        GP_CUDA(launch_spline_tables(p->coef + (size_t)k * cmx * cmy, cax, cay, scratch, tab, st));
        ct[k] = make_tab(tab, W, H, p->tile);
        ctx->launches += 2;
    }
    mark(ctx, 2, st);
    const Image im = to_image(img);
    GP_CUDA(cudaMemsetAsync(w.zero, 0, (size_t)w.nzero * sizeof(int), st));
    const float one = 1.f;
    const DetectArgs A = detect_args(im, sb, sr, &one, 1, 1, p->thresh, p->minarea, segmap, nullptr, nullptr, nullptr,
                                     w.D, w.T, w.P, w.C, ctx->dstatus);
    GP_CUDA(launch_psf(A, p->p0, p->modes, p->K, p->kw, p->kh, ct, st));
    mark(ctx, 3, st);
    GP_CUDA(launch_label_any(A, nullptr, 1, st, ctx->side_made ? &ctx->side : nullptr));
    mark(ctx, 4, st);
    GP_CUDA(launch_resolve(w.T, w.P, w.C, w.D, segmap, W, H, p->minarea, ctx->walk_limit, ctx->dstatus, st));
    mark(ctx, 5, st);
    GP_CUDA(launch_rank(w.C, cat->n, cat->capacity, true, ctx->dstatus, st));
    mark(ctx, 6, st);
    GP_CUDA(launch_measure(im, sb, sr, w.C, segmap, *cat, nullptr, 0, 0.f, nullptr, nullptr, nullptr, st));
    mark(ctx, 7, st);
    ctx->launches += 1 + label_launches(false) + 4 + 4 + 1;
    return GP_OK;
}

gp_status gp_optimal_radius(gp_ctx* ctx, const gp_image* img, const gp_bkg* bkg, const gp_det_params* dp,
                            const gp_catalog* cat, const gp_ropt_params* p, gp_ropt_out* out, gp_stream stream)
{
    gp_status s;
    float taps[(2 * HMAX + 1) * (2 * HMAX + 1)];
    if ((s = check_ctx(ctx)) != GP_OK) return s;
    if ((s = check_image(img)) != GP_OK) return s;
    if ((s = check_bkg(img, bkg, true)) != GP_OK) return s;
    if ((s = check_det(dp, taps)) != GP_OK) return s;
    if ((s = check_cat(cat)) != GP_OK) return s;
    if (!p || !out) return fail(GP_ERR_INVALID_ARG, "null parameters or outputs");
    if (!p->radii || p->nr < 1 || p->nr > GP_GROWTH_MAX_NR)
        return fail(GP_ERR_INVALID_ARG, "growth radii: need 1..%d of them", GP_GROWTH_MAX_NR);
    for (int k = 0; k < p->nr; ++k) {
        if (p->radii[k] < 0 || p->radii[k] > GP_GROWTH_MAX_R)
            return fail(GP_ERR_INVALID_ARG, "growth radius %d outside 0..%d", p->radii[k], GP_GROWTH_MAX_R);
        if (k > 0 && p->radii[k] <= p->radii[k - 1]) return fail(GP_ERR_INVALID_ARG, "growth radii not increasing");
    }
    if (!std::isfinite(p->snr_min) || !std::isfinite(p->d_iso) || p->d_iso < 0.f)
        return fail(GP_ERR_INVALID_ARG, "snr_min must be finite and d_iso >= 0");
    if (!out->fit || (cat->capacity > 0 && (!out->flux || !out->fluxerr || !out->flags || !out->nu || !out->kopt ||
                                             !out->calib || !out->kfinal || !out->flux_opt || !out->fluxerr_opt)))
        return fail(GP_ERR_INVALID_ARG, "null optimal-radius output");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    Carver cv{ctx->base, ctx->arena_bytes - STATUS_BYTES};
    SplineTab sb, sr;
    begin_call(ctx, st);
    mark(ctx, 1, st);
    s = run_spline(cv, bkg, img->width, img->height, &sb, &sr, &ctx->launches, st);
    if (s == GP_ERR_OOM) return oom(cv);
    if (s != GP_OK) return s;
    double cs;
    int ncx, ncy;
    iso_grid(img->width, img->height, p->d_iso, &cs, &ncx, &ncy);
    RoptWork w;
    w.count = cv.take<int>((size_t)ncx * ncy);
    w.start = cv.take<int>((size_t)ncx * ncy);
    w.fill = cv.take<int>((size_t)ncx * ncy);
    w.items = cv.take<int>(cat->capacity > 0 ? cat->capacity : 1);
    w.xy = cv.take<double2>(cat->capacity > 0 ? cat->capacity : 1);
    if (!cv.ok()) return oom(cv);
    mark_to(ctx, 2, GP_NSTAGES - 1, st);
    if (cat->capacity > 0) {
        const Image im = to_image(img);
        GP_CUDA(launch_growth(im, sb, sr, cat->x, cat->y, cat->capacity, cat->n, p->radii, p->nr, p->gain, out->flux,
                              out->fluxerr, out->flags, st));
        GP_CUDA(launch_ropt(im, sb, sr, taps, dp->kw, dp->kh, *cat, out->flux, out->fluxerr, out->flags, p->radii,
                            p->nr, p->snr_min, p->d_iso, w, out->nu, out->kopt, out->calib, out->kfinal, out->flux_opt,
                            out->fluxerr_opt, out->fit, st));
        ctx->launches += 1 + 7;
    } else {
        const double none[4] = {NAN, NAN, 0.0, 1.0};
        GP_CUDA(cudaMemcpyAsync(out->fit, none, sizeof none, cudaMemcpyHostToDevice, st));
        GP_CUDA(cudaStreamSynchronize(st));
    }
    mark(ctx, GP_NSTAGES, st);
    return GP_OK;
}

gp_status gp_extract(gp_ctx* ctx, const gp_image* img, const gp_bkg_params* bp, const gp_det_params* dp,
                     const gp_ap_params* ap, gp_bkg* bkg, uint32_t* segmap, gp_catalog* cat, double* flux,
                     double* fluxerr, uint32_t* apflags, gp_stream stream)
{
    return extract_call(ctx, img, bp, dp, ap, nullptr, bkg, segmap, cat, flux, fluxerr, apflags, stream);
}

gp_status gp_label_mask(gp_ctx* ctx, const uint8_t* mask, int32_t width, int32_t height, int32_t minarea,
                        uint32_t* segmap, int32_t* n_out, gp_stream stream)
{
    gp_status s;
    if ((s = check_ctx(ctx)) != GP_OK) return s;
    if (!mask || !segmap) return fail(GP_ERR_INVALID_ARG, "null mask or segmap");
    if (width < 1 || height < 1 || (int64_t)width * height > 0x7fffffffll)
        return fail(GP_ERR_INVALID_ARG, "image size %dx%d", width, height);
    if (minarea < 1) return fail(GP_ERR_INVALID_ARG, "minarea must be >= 1");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    Carver cv{ctx->base, ctx->arena_bytes - STATUS_BYTES};
    DetWork w;
    carve_det(cv, width, height, 0, w);
    if (!cv.ok()) return oom(cv);
    Image im{};
    im.W = width;
    im.H = height;
    SplineTab none{};
    begin_call(ctx, st);
    mark_to(ctx, 1, 2, st);
    GP_CUDA(cudaMemsetAsync(w.zero, 0, (size_t)w.nzero * sizeof(int), st));
    const DetectArgs A = detect_args(im, none, none, nullptr, 1, 1, 1.f, minarea, segmap, nullptr, nullptr, mask, w.D,
                                     w.T, w.P, w.C, ctx->dstatus);
    GP_CUDA(launch_stream_any(A, nullptr, 1, detect_grid(width, height, true), st));
    mark(ctx, 3, st);
    GP_CUDA(launch_label_any(A, nullptr, 1, st, nullptr));
    mark(ctx, 4, st);
    GP_CUDA(launch_resolve(w.T, w.P, w.C, w.D, segmap, width, height, minarea, ctx->walk_limit, ctx->dstatus, st));
    mark(ctx, 5, st);
    GP_CUDA(launch_rank(w.C, n_out, -1, false, ctx->dstatus, st));
    mark_to(ctx, 6, 7, st);
    ctx->launches += 3 + 4 + 2;
    return GP_OK;
}

}  // extern "C"

extern "C" {

gp_status gp_box_quantiles(gp_ctx* ctx, const gp_image* img, int32_t mesh, float* quant, gp_stream stream)
{
    gp_status s;
    if ((s = check_ctx(ctx)) != GP_OK) return s;
    if ((s = check_image(img)) != GP_OK) return s;
    gp_bkg_params p{mesh, 1, 3.f, 0};
    if ((s = check_bkg_params(img, &p)) != GP_OK) return s;
    if (!quant) return fail(GP_ERR_INVALID_ARG, "null quantile output");
    const int W = img->width, H = img->height;
    const int Mx = (W + mesh - 1) / mesh, My = (H + mesh - 1) / mesh;
    Carver cv{ctx->base, ctx->arena_bytes - STATUS_BYTES};
    BkgWork w;
    carve_bkg(cv, Mx * My, w);
    if (!cv.ok()) return oom(cv);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    begin_call(ctx, st);
    GP_CUDA(launch_boxstats(to_image(img), mesh, 3.0, 0, w.bkg_raw, w.rms_raw, w.valid, quant, st));
    ctx->launches += 1;
    mark_to(ctx, 1, GP_NSTAGES, st);
    return GP_OK;
}

}  // extern "C"

namespace {

gp_status check_net(const gp_cnn_weights* net)
{
    if (!net) return fail(GP_ERR_INVALID_ARG, "null network weights");
    for (int l = 0; l < GP_CNN_LAYERS; ++l)
        if (!net->wt[l] || !net->bias[l]) return fail(GP_ERR_INVALID_ARG, "null weights of layer %d", l);
    return GP_OK;
}

}  // namespace

extern "C" {

gp_status gp_background_learned(gp_ctx* ctx, const gp_image* img, const gp_bkg_params* p, const gp_cnn_weights* net,
                                gp_bkg* bkg, gp_stream stream)
{
    gp_status s;
    if ((s = check_ctx(ctx)) != GP_OK) return s;
    if ((s = check_image(img)) != GP_OK) return s;
    if ((s = check_bkg_params(img, p)) != GP_OK) return s;
    if ((s = check_net(net)) != GP_OK) return s;
    if (!bkg || !bkg->bkg_mesh || !bkg->rms_mesh) return fail(GP_ERR_INVALID_ARG, "null background output meshes");
    return background_call(ctx, img, p, net, bkg, stream);
}

gp_status gp_extract_learned(gp_ctx* ctx, const gp_image* img, const gp_bkg_params* bp, const gp_det_params* dp,
                             const gp_ap_params* ap, const gp_cnn_weights* net, gp_bkg* bkg, uint32_t* segmap,
                             gp_catalog* cat, double* flux, double* fluxerr, uint32_t* apflags, gp_stream stream)
{
    if (!net) return fail(GP_ERR_INVALID_ARG, "null network weights");
    return extract_call(ctx, img, bp, dp, ap, net, bkg, segmap, cat, flux, fluxerr, apflags, stream);
}

gp_status gp_extract_batch(gp_ctx* ctx, gp_frame* frames, int32_t n, const gp_bkg_params* bp,
                           const gp_det_params* dp, const gp_ap_params* ap, const gp_cnn_weights* net,
                           gp_stream stream)
{
    gp_status s;
    float taps[KMAX];
    if ((s = check_ctx(ctx)) != GP_OK) return s;
    if (!frames) return fail(GP_ERR_INVALID_ARG, "null frame array");
    if (n < 1 || n > GP_MAX_BATCH) return fail(GP_ERR_INVALID_ARG, "n = %d outside [1, %d]", n, GP_MAX_BATCH);
    if (net && (s = check_net(net)) != GP_OK) return s;
    if ((s = check_det(dp, taps)) != GP_OK) return s;
    if ((s = check_ap(ap, true)) != GP_OK) return s;
    for (int f = 0; f < n; ++f) {
        const gp_frame& x = frames[f];
        if ((s = check_image(&x.image)) != GP_OK) return fail(s, "frame %d: %s", f, gp_last_error());
        if (x.image.dtype != frames[0].image.dtype) return fail(GP_ERR_INVALID_ARG, "frame %d: dtype differs", f);
        if ((s = check_bkg_params(&x.image, bp)) != GP_OK) return s;
        if ((s = check_cat(&x.cat)) != GP_OK) return fail(s, "frame %d: %s", f, gp_last_error());
        if (!x.bkg.bkg_mesh || !x.bkg.rms_mesh) return fail(GP_ERR_INVALID_ARG, "frame %d: null meshes", f);
        if (!x.segmap || !x.status) return fail(GP_ERR_INVALID_ARG, "frame %d: null segmap or status", f);
        if (ap->nr > 0 && x.cat.capacity > 0 && (!x.flux || !x.fluxerr || !x.apflags))
            return fail(GP_ERR_INVALID_ARG, "frame %d: null aperture output array", f);
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (n > 1) {
        cudaError_t e = ctx->stage.init((size_t)512 << 10);
        if (e != cudaSuccess) return cuda_fail(e, "pinned argument staging");
    }
    begin_call(ctx, st);
    Exec ex = ctx_exec(ctx, st);
    Params P = make_params(bp, taps, dp, ap, net);
    P.walk_limit = ctx->walk_limit;
    std::vector<FrameIO> F(n);
    for (int f = 0; f < n; ++f) {
        const gp_frame& x = frames[f];
        F[f] = frame_io(&x.image, &x.bkg, x.segmap, &x.cat, x.flux, x.fluxerr, x.apflags, nullptr, x.status);
    }
    s = pipeline_result(run_extract(ex, n, F.data(), P), ex, ctx);
    for (int f = 0; f < n; ++f) {
        frames[f].bkg.mesh = F[f].bkg.mesh; frames[f].bkg.mx = F[f].bkg.mx; frames[f].bkg.my = F[f].bkg.my;
    }
    return s;
}

}  // extern "C"

// argument checks and gp_last_error() messages for entry points defined in
// other files
namespace gp {
void record_error(const char* msg) { g_err = msg; }
gp_status validate_image(const gp_image* img) { return check_image(img); }
gp_status validate_bkg_params(const gp_image* img, const gp_bkg_params* p) { return check_bkg_params(img, p); }
gp_status validate_det_params(const gp_det_params* p, float* taps) { return check_det(p, taps); }
gp_status validate_ap_params(const gp_ap_params* p) { return check_ap(p, true); }
gp_status validate_net(const gp_cnn_weights* net) { return check_net(net); }
}  // namespace gp
