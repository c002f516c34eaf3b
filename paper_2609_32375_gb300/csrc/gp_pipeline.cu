// gp_pipeline.cu -- workspace layout and launch sequence of the extraction
// (background, detection, measurement) over one frame or a batch of frames.
//
// A batch runs every stage as one launch over all its frames (grid y = the
// frame): per-frame argument records are built on the host, copied to the
// device in one transfer from pinned staging, and each kernel reads its
// frame's record.  A single frame passes its record by value instead, so
// gp_extract and a batch of one run the same kernels with the same
// arithmetic; a frame's results do not depend on the batch it ran in.
#include <stdio.h>
#include <string.h>

#include <algorithm>

#include "gp_pipeline.h"

namespace gp {

int piece_cap_for(int64_t npix) { return (int)std::max<int64_t>(65536, npix / 64); }

int comp_cap_for(int64_t npix, int capacity)
{
    int64_t c = std::max<int64_t>(65536, npix / 32);
    if (capacity > c) c = capacity;
    return (int)std::min<int64_t>(c, 1ll << 30);
}

// Buckets of 2^shift labels for the rank; at most 16,384 of them, so the
// one-CTA scan reads 16 counts per thread (the place step sorts within a
// bucket, about four segments on the dense 151 MP frame).
static void bucket_geometry(int64_t npix, int* shift, int* nb)
{
    int s = 0;
    while (((npix - 1) >> s) + 1 > 16384) ++s;
    *shift = s;
    *nb = (int)(((npix - 1) >> s) + 1);
}

void carve_bkg(Carver& cv, int nbox, BkgWork& w)
{
    w.bkg_raw = cv.take<double>(nbox);
    w.rms_raw = cv.take<double>(nbox);
    w.tmp_b = cv.take<double>(nbox);
    w.tmp_r = cv.take<double>(nbox);
    w.valid = cv.take<int>(nbox);
    w.tmp_v = cv.take<int>(nbox);
}

void carve_spline(Carver& cv, int Mx, int My, SplineWork& w)
{
    w.scratch = cv.take<double>(spline_scratch_doubles(Mx, My));
    w.tab_b = cv.take<float4>((size_t)Mx * My);
    w.tab_r = cv.take<float4>((size_t)Mx * My);
}

int det_zero_ints(int W, int H)
{
    int shift, nb;
    bucket_geometry((int64_t)W * H, &shift, &nb);
    return 64 + 2 * nb;
}

void carve_det(Carver& cv, int W, int H, int capacity, DetWork& w, int** zero)
{
    const int64_t npix = (int64_t)W * H;
    bucket_geometry(npix, &w.C.shift, &w.C.nb);
    w.nzero = 64 + 2 * w.C.nb;
    if (zero) {
        w.zero = *zero;
        *zero += w.nzero;
    } else {
        w.zero = cv.take<int>(w.nzero);
    }
    w.T.ntx = (W + TX - 1) / TX;
    w.T.nty = (H + TY - 1) / TY;
    const int64_t ntiles = (int64_t)w.T.ntx * w.T.nty;
    w.T.edges = cv.take<int16_t>((size_t)ntiles * EDGE_PER_TILE);
    w.T.piece_base = cv.take<int>(ntiles);
    w.T.piece_cnt = cv.take<int>(ntiles);
    w.D.bits = cv.take<uint4>((size_t)H * ((W + ST_STRIP - 1) / ST_STRIP));
    w.D.tl_list = cv.take<int>(ntiles);
    w.D.tl_count = w.zero + 16;
    w.D.dl_list = cv.take<int>(ntiles);
    w.D.dl_count = w.zero + 17;
    w.D.rl_list = cv.take<int>(ntiles);
    w.D.rl_count = w.zero + 18;
    w.P.count = w.zero + 0;
    w.P.cap = piece_cap_for(npix);
    w.P.root = cv.take<uint32_t>(w.P.cap);
    w.P.npix = cv.take<int>(w.P.cap);
    w.P.bbox = cv.take<int4>(w.P.cap);
    w.P.parent = cv.take<int>(w.P.cap);
    w.P.proot = cv.take<int>(w.P.cap);
    w.P.mom = cv.take<Moments>(w.P.cap);
    w.P.agg_min = cv.take<uint32_t>(w.P.cap);
    w.P.agg_npix = cv.take<int>(w.P.cap);
    w.P.agg_bbox = cv.take<int4>(w.P.cap);
    w.C.count = w.zero + 32;
    w.C.cap = comp_cap_for(npix, capacity);
    w.C.label = cv.take<uint32_t>(w.C.cap);
    w.C.npix = cv.take<int>(w.C.cap);
    w.C.bbox = cv.take<int4>(w.C.cap);
    w.C.flux = cv.take<double>(w.C.cap);
    w.C.xy = cv.take<double2>(w.C.cap);
    w.C.mom2 = cv.take<Mom2>(w.C.cap);
    w.C.peak = cv.take<float>(w.C.cap);
    w.C.peakL = cv.take<uint32_t>(w.C.cap);
    w.C.flags = cv.take<uint32_t>(w.C.cap);
    w.C.perm = cv.take<int>(w.C.cap);
    w.C.slots = cv.take<int>(w.C.cap);
    w.C.bcnt = w.zero + 64;
    w.C.boff = cv.take<int>(w.C.nb);
    w.C.bcur = w.zero + 64 + w.C.nb;
}

SplineTab make_tab(const float4* node, int W, int H, int mesh)
{
    SplineTab s;
    s.node = node;
    s.ax = make_axis(W, mesh);
    s.ay = make_axis(H, mesh);
    return s;
}

cudaError_t ArgStage::init(size_t nbytes)
{
    if (host && bytes >= nbytes) return cudaSuccess;
    release();
    cudaError_t e = cudaHostAlloc(reinterpret_cast<void**>(&host), nbytes, cudaHostAllocDefault);
    if (e != cudaSuccess) { host = nullptr; return e; }
    e = cudaEventCreateWithFlags(&done, cudaEventDisableTiming);
    if (e != cudaSuccess) { cudaFreeHost(host); host = nullptr; return e; }
    bytes = nbytes;
    pending = false;
    return cudaSuccess;
}

void ArgStage::release()
{
    if (done) cudaEventSynchronize(done), cudaEventDestroy(done);
    if (host) cudaFreeHost(host);
    host = nullptr;
    done = nullptr;
    bytes = 0;
    pending = false;
}

namespace {

Image to_image(const gp_image& img)
{
    Image im;
    im.data = img.data;
    im.pitch = img.pitch;
    im.mask = img.mask;
    im.W = img.width;
    im.H = img.height;
    im.sat = img.saturation;
    im.is_f32 = img.dtype == GP_F32;
    return im;
}

// device bytes of the argument records of an n-frame batch (with alignment)
size_t args_bytes(int n)
{
    const size_t per = sizeof(BoxArgs) + sizeof(MeshArgs) + sizeof(DetectArgs) + sizeof(ResolveArgs) +
                       sizeof(RankArgs) + sizeof(MeasureArgs);
    return (size_t)n * per + 8 * 64;
}

// packs argument arrays into the pinned staging, then one host-to-device copy
struct Upload {
    ArgStage* stage;
    char* dev;
    size_t off = 0;
    template <class T>
    const T* put(const T* src, int n)
    {
        off = (off + 63) & ~(size_t)63;
        memcpy(stage->host + off, src, (size_t)n * sizeof(T));
        const T* d = reinterpret_cast<const T*>(dev + off);
        off += (size_t)n * sizeof(T);
        return d;
    }
};

gp_status cuda_err(cudaError_t e, const char* what)
{
    char buf[256];
    snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
    record_error(buf);
    return GP_ERR_CUDA;
}

#define PL_CUDA(call)                                      \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_err(e_, #call); \
    } while (0)

struct FrameWork {
    int W, H, Mx, My, nbox;
    bool fused;
    BkgWork bw;
    SplineWork sw;
    float4 *tab_b, *tab_r;
    float* quant;
    int* fb_list;           // uint16 boxes left to the full-histogram kernel
    DetWork dw;
    SplineTab sb, sr;
};

const int CNN_CIN_P[GP_CNN_LAYERS] = {16, 32, 48, 48, 32, 32};
const int CNN_COUT_P[GP_CNN_LAYERS] = {32, 48, 48, 32, 32, 16};

// the network over nf frames of one mesh geometry (My x Mx), quantiles in
// quant ([nf][5][nbox]); meshes of frame f into F[f].bkg
gp_status run_network(Exec& ex, const gp_cnn_weights* net, const float* quant, int nf, int My, int Mx, float* norm,
                      uint16_t* feat, uint16_t* a0, uint16_t* a1, float* out, FrameIO* F)
{
    const int nbox = Mx * My;
    PL_CUDA(launch_cnn_features(quant, nf, nbox, feat, norm, ex.st));
    const void* in = feat;
    for (int l = 0; l < GP_CNN_LAYERS; ++l) {
        const bool last = l == GP_CNN_LAYERS - 1;
        void* o = last ? (void*)out : (void*)((l & 1) ? a1 : a0);
        PL_CUDA(launch_cnn_conv(in, nf, My, Mx, CNN_CIN_P[l], net->wt[l], net->bias[l], CNN_COUT_P[l], last ? 0 : 1,
                                o, last ? 1 : 0, 2, ex.st));
        in = o;
    }
    for (int f = 0; f < nf; ++f)
        PL_CUDA(launch_cnn_denorm(out + (size_t)f * 2 * nbox, norm + 2 * f, nbox, 1, F[f].bkg.bkg_mesh,
                                  F[f].bkg.rms_mesh, ex.st));
    ex.launches += 1 + GP_CNN_LAYERS + nf;
    return GP_OK;
}

gp_status run_frames(Exec& ex, int n, FrameIO* F, const Params& P, bool detect)
{
    const bool batched = n > 1;
    const bool learned = P.net != nullptr;
    const int B = P.bp.mesh;
    Carver& cv = ex.cv;
    std::vector<FrameWork> w(n);
    int64_t nz = 0, nbox_all = 0;
    bool same_mesh = true;
    for (int f = 0; f < n; ++f) {
        FrameWork& x = w[f];
        x.W = F[f].img.width;
        x.H = F[f].img.height;
        x.Mx = (x.W + B - 1) / B;
        x.My = (x.H + B - 1) / B;
        x.nbox = x.Mx * x.My;
        nbox_all += x.nbox;
        if (detect) nz += det_zero_ints(x.W, x.H);
        same_mesh = same_mesh && x.Mx == w[0].Mx && x.My == w[0].My;
    }
    // ---- workspace: one block cleared per call holds the box-statistics
    // fallback counts (one per frame) and the detection counters
    const bool u16 = F[0].img.dtype == GP_U16;
    const int64_t nz_all = 64 + nz;
    int* zero = cv.take<int>(nz_all);
    int* fb_count = zero;                   // [f]
    int* zc = zero + 64;
    float *quant_all = nullptr, *norm = nullptr, *out = nullptr;
    uint16_t *feat = nullptr, *a0 = nullptr, *a1 = nullptr;
    if (learned) {
        // one network pass over every frame when all share one mesh
        // geometry, else one pass per frame (buffers sized for the batch)
        quant_all = cv.take<float>((size_t)5 * nbox_all);
        norm = cv.take<float>((size_t)2 * n);
        feat = cv.take<uint16_t>((size_t)16 * nbox_all);
        a0 = cv.take<uint16_t>((size_t)48 * nbox_all);
        a1 = cv.take<uint16_t>((size_t)48 * nbox_all);
        out = cv.take<float>((size_t)2 * nbox_all);
    }
    int64_t qoff = 0;
    for (int f = 0; f < n; ++f) {
        FrameWork& x = w[f];
        carve_bkg(cv, x.nbox, x.bw);
        x.fb_list = u16 ? cv.take<int>(x.nbox) : nullptr;
        x.quant = learned ? quant_all + qoff : nullptr;
        qoff += (int64_t)5 * x.nbox;
        x.fused = mesh_fits_smem(x.Mx, x.My);
        if (x.fused) {
            x.tab_b = cv.take<float4>((size_t)x.nbox);
            x.tab_r = cv.take<float4>((size_t)x.nbox);
        } else {
            carve_spline(cv, x.Mx, x.My, x.sw);
            x.tab_b = x.sw.tab_b;
            x.tab_r = x.sw.tab_r;
        }
        if (detect) carve_det(cv, x.W, x.H, F[f].cat.capacity, x.dw, &zc);
        x.sb = make_tab(x.tab_b, x.W, x.H, B);
        x.sr = make_tab(x.tab_r, x.W, x.H, B);
    }
    char* dargs = batched ? cv.take<char>(args_bytes(n)) : nullptr;
    if (!cv.ok()) return GP_ERR_OOM;
    if (batched && (!ex.stage || !ex.stage->host || ex.stage->bytes < args_bytes(n))) {
        record_error("batched call without argument staging");
        return GP_ERR_INTERNAL;
    }

    // ---- argument records
    std::vector<BoxArgs> box(n);
    std::vector<MeshArgs> mesh;
    std::vector<DetectArgs> det(detect ? n : 0);
    std::vector<ResolveArgs> res(detect ? n : 0);
    std::vector<RankArgs> rank(detect ? n : 0);
    std::vector<MeasureArgs> meas(detect ? n : 0);
    int maxbox = 0, maxgrid = 0, maxtiles = 0;
    size_t mesh_smem = 0;
    for (int f = 0; f < n; ++f) {
        FrameWork& x = w[f];
        F[f].bkg.mesh = B;
        F[f].bkg.mx = x.Mx;
        F[f].bkg.my = x.My;
        const Image im = to_image(F[f].img);
        box[f] = box_args(im, B, learned ? 3.0 : (double)P.bp.clip_k, learned ? 0 : P.bp.clip_maxiter, x.bw.bkg_raw,
                          x.bw.rms_raw, x.bw.valid, x.quant);
        if (u16) {
            box[f].fb_list = x.fb_list;
            box[f].fb_count = fb_count + f;
        }
        maxbox = std::max(maxbox, x.nbox);
        if (x.fused) {
            mesh.push_back(mesh_args(x.bw.bkg_raw, x.bw.rms_raw, x.bw.valid, x.sb.ax, x.sb.ay, P.bp.filter_size,
                                     learned ? 1 : 0, F[f].bkg.bkg_mesh, F[f].bkg.rms_mesh, x.tab_b, x.tab_r));
            mesh_smem = std::max(mesh_smem, mesh_all_smem(x.Mx, x.My));
        }
        if (!detect) continue;
        det[f] = detect_args(im, x.sb, x.sr, P.taps, P.kw, P.kh, P.thresh, P.minarea, F[f].segmap, F[f].mask_out,
                             F[f].nnear, nullptr, x.dw.D, x.dw.T, x.dw.P, x.dw.C, F[f].status);
        res[f] = resolve_args(x.dw.T, x.dw.P, x.dw.C, x.dw.D, F[f].segmap, x.W, x.H, P.minarea, P.walk_limit,
                              F[f].status);
        rank[f] = rank_args(x.dw.C, F[f].cat.n, F[f].cat.capacity, true, F[f].status);
        meas[f] = measure_args(im, x.sb, x.sr, x.dw.C, F[f].cat, P.radii, P.nr, P.gain, F[f].apflux, F[f].apferr,
                               F[f].apflags);
        maxgrid = std::max(maxgrid, detect_grid(x.W, x.H, false));
        maxtiles = std::max(maxtiles, x.dw.T.ntx * x.dw.T.nty);
    }
    const int nfused = (int)mesh.size();
    const BoxArgs* d_box = nullptr;
    const MeshArgs* d_mesh = nullptr;
    const DetectArgs* d_det = nullptr;
    const ResolveArgs* d_res = nullptr;
    const RankArgs* d_rank = nullptr;
    const MeasureArgs* d_meas = nullptr;
    if (batched) {
        ArgStage* sg = ex.stage;
        if (sg->pending) PL_CUDA(cudaEventSynchronize(sg->done));   // the last upload has read the staging
        Upload up{sg, dargs};
        d_box = up.put(box.data(), n);
        if (nfused > 1) d_mesh = up.put(mesh.data(), nfused);
        if (detect) {
            d_det = up.put(det.data(), n);
            d_res = up.put(res.data(), n);
            d_rank = up.put(rank.data(), n);
            d_meas = up.put(meas.data(), n);
        }
        PL_CUDA(cudaMemcpyAsync(dargs, sg->host, up.off, cudaMemcpyHostToDevice, ex.st));
        PL_CUDA(cudaEventRecord(sg->done, ex.st));
        sg->pending = true;
    }

    // ---- background: per-box statistics, mesh, spline tables
    PL_CUDA(cudaMemsetAsync(zero, 0, (size_t)nz_all * sizeof(int), ex.st));
    const int is_f32 = F[0].img.dtype == GP_F32;
    PL_CUDA(launch_boxstats_any(box[0], d_box, n, maxbox, is_f32, ex.st));
    ex.launches += is_f32 ? 1 : 2;
    ex.at(1);
    if (learned) {
        if (same_mesh) {
            gp_status s = run_network(ex, P.net, quant_all, n, w[0].My, w[0].Mx, norm, feat, a0, a1, out, F);
            if (s != GP_OK) return s;
        } else {
            for (int f = 0; f < n; ++f) {
                gp_status s = run_network(ex, P.net, w[f].quant, 1, w[f].My, w[f].Mx, norm, feat, a0, a1, out, F + f);
                if (s != GP_OK) return s;
            }
        }
    }
    if (nfused > 0) {
        PL_CUDA(launch_mesh_all_any(mesh[0], d_mesh, nfused, mesh_smem, ex.st));
        ex.launches += 1;
    }
    for (int f = 0; f < n; ++f) {
        FrameWork& x = w[f];
        if (x.fused) continue;
        if (!learned) {
            PL_CUDA(launch_mesh_finalize(x.bw.bkg_raw, x.bw.rms_raw, x.bw.valid, x.bw.tmp_b, x.bw.tmp_r, x.bw.tmp_v,
                                         x.Mx, x.My, P.bp.filter_size, F[f].bkg.bkg_mesh, F[f].bkg.rms_mesh, ex.st));
            ex.launches += 1;
        }
        PL_CUDA(launch_spline_tables(F[f].bkg.bkg_mesh, x.sb.ax, x.sb.ay, x.sw.scratch, x.tab_b, ex.st));
        PL_CUDA(launch_spline_tables(F[f].bkg.rms_mesh, x.sb.ax, x.sb.ay, x.sw.scratch, x.tab_r, ex.st));
        ex.launches += 4;
    }
    for (int f = 0; f < n; ++f) {
        if (!F[f].bkg.bkg_map && !F[f].bkg.rms_map) continue;
        PL_CUDA(launch_bkg_maps(w[f].sb, w[f].sr, w[f].W, w[f].H, F[f].bkg.bkg_map, F[f].bkg.rms_map, ex.st));
        ex.launches += 1;
    }
    ex.at(2);
    if (!detect) {
        ex.at_range(3, GP_NSTAGES);
        return GP_OK;
    }

    // ---- detection, segment resolution, catalog order, measurement
    for (int f = 0; f < n; ++f)
        if (F[f].nnear) PL_CUDA(cudaMemsetAsync(F[f].nnear, 0, sizeof(int), ex.st));
    PL_CUDA(launch_stream_any(det[0], d_det, n, maxgrid, ex.st));
    ex.at(3);
    PL_CUDA(launch_label_any(det[0], d_det, n, ex.st, ex.side));
    ex.at(4);
    PL_CUDA(launch_resolve_any(res[0], d_res, n, maxtiles, ex.st));
    ex.at(5);
    PL_CUDA(launch_rank_any(rank[0], d_rank, n, ex.st));
    ex.at(6);
    PL_CUDA(launch_measure_any(meas[0], d_meas, n, ex.st));
    ex.at(7);
    ex.launches += 1 + label_launches(false) + 4 + 4 + 1 + (P.nr > 0 ? 1 : 0);
    return GP_OK;
}

}  // namespace

gp_status run_extract(Exec& ex, int n, FrameIO* F, const Params& P) { return run_frames(ex, n, F, P, true); }

gp_status run_background_only(Exec& ex, int n, FrameIO* F, const Params& P)
{
    return run_frames(ex, n, F, P, false);
}

size_t extract_workspace_bytes(int n, const int* W, const int* H, const int* capacity, int mesh, bool learned)
{
    Carver cv{nullptr, 0};
    int64_t nz = 0, nbox_all = 0;
    for (int f = 0; f < n; ++f) {
        nz += det_zero_ints(W[f], H[f]);
        nbox_all += (int64_t)((W[f] + mesh - 1) / mesh) * ((H[f] + mesh - 1) / mesh);
    }
    int* zc = cv.take<int>(64 + nz) + 64;
    if (learned) {
        cv.take<float>((size_t)5 * nbox_all);
        cv.take<float>((size_t)2 * n);
        cv.take<uint16_t>((size_t)16 * nbox_all);
        cv.take<uint16_t>((size_t)48 * nbox_all);
        cv.take<uint16_t>((size_t)48 * nbox_all);
        cv.take<float>((size_t)2 * nbox_all);
    }
    for (int f = 0; f < n; ++f) {
        const int Mx = (W[f] + mesh - 1) / mesh, My = (H[f] + mesh - 1) / mesh;
        BkgWork b;
        carve_bkg(cv, Mx * My, b);
        cv.take<int>((size_t)Mx * My);      // box fallback list
        if (mesh_fits_smem(Mx, My)) {
            cv.take<float4>((size_t)Mx * My);
            cv.take<float4>((size_t)Mx * My);
        } else {
            SplineWork s;
            carve_spline(cv, Mx, My, s);
        }
        DetWork d;
        carve_det(cv, W[f], H[f], capacity ? capacity[f] : 0, d, &zc);
    }
    if (n > 1) cv.take<char>(args_bytes(n));
    return cv.off + ALIGN;
}

}  // namespace gp
