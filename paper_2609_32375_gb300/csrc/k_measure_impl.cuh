// k_measure_impl.cuh -- device code of the catalog-row and aperture
// kernels (paper Section 3.4), shared by k_measure.cu (single-frame forms
// and the aperture entry point) and k_measure_batch.cu (batched forms), so
// the two sets of template instances compile in parallel.
#pragma once
#include <math.h>

#include "gp_internal.cuh"
#include "gp_launch.h"

namespace gp {
// integral of sqrt(r^2 - t^2) over [a, b], -r <= a <= b <= r, written with
// differences formed algebraically (no cancellation between large terms)
__device__ __forceinline__ float chord_int(float a, float b, float r2)
{
    float d = b - a;
    if (!(d > 0.f)) return 0.f;
    float ha = sqrtf(fmaxf(fmaf(-a, a, r2), 0.f));
    float hb = sqrtf(fmaxf(fmaf(-b, b, r2), 0.f));
    float s = ha + hb;
    float q = s > 0.f ? d * (a + b) / s : 0.f;      // ha - hb
    float sin_t = fmaf(d, ha, a * q);               // (b ha - a hb), r^2 sin(theta)
    float cos_t = fmaf(ha, hb, a * b);              // (ha hb + a b), r^2 cos(theta)
    float theta = atan2f(sin_t, cos_t);             // asin(b/r) - asin(a/r)
    return 0.5f * fmaf(r2, theta, fmaf(d, hb, -a * q));
}

// exact area of disc(0, r) n [x0,x1] x [y0,y1]: integrate the length of
// [y0,y1] n [-h(x), h(x)] over x, split where h(x) = |y0|, |y1|.  On each
// piece the top is y1 or the arc and the bottom y0 or the arc; rectangle parts
// add directly and only arc-bounded pieces need the arc integral.  Those are
// collected first: in a pixel that a circle of radius >= 1 crosses there are
// one or two, so the warp runs the integral once or twice per pixel instead of
// once per piece.  The roles come from squared comparisons (h^2 = r^2 - x^2).
// Every product and sum is an explicit operation (fmaf, __fmul_rn,
// __fadd_rn), so no instance of the kernels contracts it differently and a
// frame gives the same bits in a batched launch as alone.
static __device__ float disc_rect_area(float x0, float x1, float y0, float y1, float r)
{
    const float r2 = r * r;
    const float a = fmaxf(x0, -r), b = fminf(x1, r);
    if (!(a < b)) return 0.f;
    float p[6];
    p[0] = a;
    p[5] = b;
    const float c0 = fabsf(y0) < r ? sqrtf(fmaxf(fmaf(-y0, y0, r2), 0.f)) : 0.f;
    const float c1 = fabsf(y1) < r ? sqrtf(fmaxf(fmaf(-y1, y1, r2), 0.f)) : 0.f;
    p[1] = fminf(fmaxf(-c0, a), b);
    p[2] = fminf(fmaxf(c0, a), b);
    p[3] = fminf(fmaxf(-c1, a), b);
    p[4] = fminf(fmaxf(c1, a), b);
    // sort p[1..4]
#define GP_CSWAP(i, j) { float lo_ = fminf(p[i], p[j]); float hi_ = fmaxf(p[i], p[j]); p[i] = lo_; p[j] = hi_; }
    GP_CSWAP(1, 2); GP_CSWAP(3, 4); GP_CSWAP(1, 3); GP_CSWAP(2, 4); GP_CSWAP(2, 3);
#undef GP_CSWAP
    const float y02 = y0 * y0, y12 = y1 * y1;
    float area = 0.f;
    float l0 = 0.f, h0 = 0.f, k0 = 0.f, l1 = 0.f, h1 = 0.f, k1 = 0.f;   // the first two arc pieces
    int n = 0;
    // the pieces without branches: an empty piece (w = 0) adds an exact zero
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const float lo = p[k], hi = p[k + 1];
        const float w = hi - lo;                                   // >= 0: the points are sorted
        const float mid = 0.5f * (lo + hi);
        const float hm2 = fmaxf(fmaf(-mid, mid, r2), 0.f);      // h(mid)^2
        const bool top_h = y1 >= 0.f && hm2 <= y12;                // the arc is below the top edge
        const bool bot_h = y0 <= 0.f && hm2 <= y02;                // the arc is above the bottom edge
        const bool plain = !top_h && !bot_h;
        // an arc piece is empty when its top is at or below its bottom
        const bool empty = (top_h && bot_h) ? !(hm2 > 0.f) : top_h ? !(y0 < 0.f || hm2 > y02)
                                                                   : !(y1 > 0.f || hm2 > y12);
        const bool arc = w > 0.f && !plain && !empty;
        // rectangle parts: the full height of a plain piece; on an arc piece
        // the edges that the arc does not replace
        const float rect = plain ? __fmul_rn(y1 - y0, w)
                         : arc   ? __fsub_rn(top_h ? 0.f : __fmul_rn(y1, w), bot_h ? 0.f : __fmul_rn(y0, w))
                                 : 0.f;
        area = __fadd_rn(area, rect);
        const float kg = (top_h && bot_h) ? 2.f : 1.f;
        const bool s0 = arc && n == 0, s1 = arc && n == 1;
        l0 = s0 ? lo : l0; h0 = s0 ? hi : h0; k0 = s0 ? kg : k0;
        l1 = s1 ? lo : l1; h1 = s1 ? hi : h1; k1 = s1 ? kg : k1;
        if (arc && n >= 2) area = fmaf(kg, chord_int(lo, hi, r2), area);   // radii below 1 only
        n += arc ? 1 : 0;
    }
    if (n > 0) area = fmaf(k0, chord_int(l0, h0, r2), area);
    if (n > 1) area = fmaf(k1, chord_int(l1, h1, r2), area);
    return area;
}

template <bool F32>
__device__ __forceinline__ float load_px(const Image& im, int x, int y, bool& bad)
{
    float v;
    if (F32) {
        v = __ldg(reinterpret_cast<const float*>(im.data) + (int64_t)y * im.pitch + x);
        bad = !isfinite(v);
    } else {
        v = (float)__ldg(reinterpret_cast<const uint16_t*>(im.data) + (int64_t)y * im.pitch + x);
        bad = false;
    }
    if (im.mask && im.mask[(int64_t)y * im.W + x]) bad = true;
    return v;
}

// Pixels crossed by a circle wait in a per-warp queue so that the exact
// overlap area, the one expensive step, runs with every lane busy instead of
// once per row for whichever lanes meet the circle.
struct BEntry {
    float dx0, dy0, m, var;
    int kf;                 // mask of the radii crossing the pixel | bad << 8 | saturated << 9
};
constexpr int QCAP = 64;      // at most 31 waiting + 32 added by one row
constexpr int MEAS_NT = 256;

template <int NR>
__device__ __forceinline__ void flush_queue(const ApSpec& ap, BEntry* wq, int qn, DF* f, DF* v, uint32_t* fl)
{
    __syncwarp();
    const int lane = threadIdx.x & 31;
    for (int i = lane; i < qn; i += 32) {
        const BEntry e = wq[i];
        unsigned rm = e.kf & 0xffu;                  // the radii whose circle crosses the pixel
        while (rm) {
            const int k = __ffs(rm) - 1;
            rm &= rm - 1u;
            const float A = disc_rect_area(e.dx0, e.dx0 + 1.f, e.dy0, e.dy0 + 1.f, ap.r[k]);
            if (!(A > 0.f)) continue;
#pragma unroll
            for (int kk = 0; kk < NR; ++kk) {
                if (kk != k) continue;
                if (e.kf & 0x100) { fl[kk] |= GP_FLAG_BAD; continue; }
                if (e.kf & 0x200) fl[kk] |= GP_FLAG_SAT;
                df_add_prod(f[kk], A, e.m);
                df_add_prod(v[kk], A, e.var);
            }
        }
    }
    __syncwarp();
}

// Apertures around (cx, cy) for all radii; executed by one full warp.
// One lane per pixel column: the column's x-spline coefficients and the
// node-row values u_j, w_j of both maps are evaluated once per column and
// reused down the column, so each pixel costs a few FMAs for B(p) and
// sigma(p).  Pixels wholly inside a disc add directly; pixels the circle
// crosses go through the queue.  The queue order and the lane assignment are
// fixed, and lane results are combined in a fixed order, so the sums are
// reproducible.  Lane 0 writes.
template <bool F32, int NR>
__device__ void aperture_warp(const Image& im, const SplineTab& sb, const SplineTab& sr, const ApSpec& ap,
                              double cx, double cy, double* flux, double* ferr, uint32_t* aflags, BEntry* wq)
{
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int W = im.W, H = im.H;
    // The window comes from the whole and fractional parts of the position,
    // so the float64 work is one split of each coordinate (every lane issues
    // it, and float64 runs at a small fraction of the float32 rate).  With
    // cx = xi + f, a column x can meet the disc of radius rmax only if
    // xi - ceil(rmax) - 1 <= x <= xi + ceil(rmax) + 2; rows likewise.  Pixels
    // of the window beyond the disc fail the per-pixel test.  Positions far
    // outside the frame (or NaN) give an empty window.
    const bool near = fabsf((float)cx - 0.5f * (float)W) <= 0.5f * (float)W + 4096.f &&
                      fabsf((float)cy - 0.5f * (float)H) <= 0.5f * (float)H + 4096.f;
    const double xi_d = floor(near ? cx : 0.0), yi_d = floor(near ? cy : 0.0);
    const int xi = (int)xi_d, yi = (int)yi_d;
    const float xf = (float)(cx - xi_d), yf = (float)(cy - yi_d);
    const int rc = (int)ceilf(ap.rmax);
    const int xa = max(xi - rc - 1, 0), ya = max(yi - rc - 1, 0);
    int xb = min(xi + rc + 2, W - 1), yb = min(yi + rc + 2, H - 1);
    if (!near) { xb = -1; yb = -1; }
    DF f[NR > 0 ? NR : 1], v[NR > 0 ? NR : 1];
    uint32_t fl[NR > 0 ? NR : 1];
#pragma unroll
    for (int k = 0; k < NR; ++k) { f[k] = df_zero(); v[k] = df_zero(); fl[k] = 0u; }
    const float rmax2 = ap.rmax * ap.rmax;
    int qn = 0;                                      // warp-uniform queue length
    for (int xbase = xa; xbase <= xb; xbase += 32) {
        const int x = xbase + lane;
        const bool colok = x <= xb;
        const float dx0 = (float)(x - xi) - xf - 0.5f, dx1 = dx0 + 1.f;
        const float nx = fmaxf(0.f, fmaxf(dx0, -dx1));
        const float fx = fmaxf(dx0 * dx0, dx1 * dx1);
        const AxCoef ccx = axis_coef(sb.ax, (float)(colok ? x : xb));
        int jc = -1;                       // node row pair cached for this column
        float ub0 = 0, ub1 = 0, wb0 = 0, wb1 = 0, ur0 = 0, ur1 = 0, wr0 = 0, wr1 = 0;
        for (int y = ya; y <= yb; ++y) {
            const float dy0 = (float)(y - yi) - yf - 0.5f, dy1 = dy0 + 1.f;
            const float ny = fmaxf(0.f, fmaxf(dy0, -dy1));
            if (!(ny * ny < rmax2)) continue;        // a row beyond the largest disc (the whole warp)
            const float dmin2 = fmaf(nx, nx, ny * ny);
            const float dmax2 = fx + fmaxf(dy0 * dy0, dy1 * dy1);
            const bool live = colok && dmin2 < rmax2;
            bool bad = true, sat = false;
            float m = 0.f, var = 0.f;
            if (live) {
                const float val = load_px<F32>(im, x, y, bad);
                if (!bad) {
                    const AxCoef ccy = axis_coef(sb.ay, (float)y);
                    if (ccy.i != jc) {
                        const float2 b0 = row_eval(sb, ccy.i, ccx), b1 = row_eval(sb, ccy.i1, ccx);
                        const float2 r0 = row_eval(sr, ccy.i, ccx), r1 = row_eval(sr, ccy.i1, ccx);
                        ub0 = b0.x; wb0 = b0.y; ub1 = b1.x; wb1 = b1.y;
                        ur0 = r0.x; wr0 = r0.y; ur1 = r1.x; wr1 = r1.y;
                        jc = ccy.i;
                    }
                    m = val - axis_combine(ccy, ub0, ub1, wb0, wb1);
                    const float sg = axis_combine(ccy, ur0, ur1, wr0, wr1);
                    var = sg * sg;
                    sat = im.sat > 0.f && val >= im.sat;
                }
            }
            unsigned bm = 0u;                        // radii whose circle crosses this pixel
#pragma unroll
            for (int k = 0; k < NR; ++k) {
                const float r = ap.r[k], r2 = r * r;
                // rows that disc k does not reach skip it: ny depends on the row only, so the
                // branch is the same for the whole warp
                if (!(ny * ny < r2)) continue;
                const bool in = live && dmin2 < r2;
                const bool full = in && dmax2 <= r2;
                if (full) {
                    if (bad) fl[k] |= GP_FLAG_BAD;
                    else {
                        if (sat) fl[k] |= GP_FLAG_SAT;
                        df_add(f[k], m);
                        df_add(v[k], var);
                    }
                }
                if (in && !full) bm |= 1u << k;
            }
            // one queue entry per crossed pixel, for all its radii
            const bool bnd = bm != 0u;
            const unsigned bal = __ballot_sync(0xffffffffu, bnd);
            if (bnd) {
                BEntry e;
                e.dx0 = dx0; e.dy0 = dy0; e.m = m; e.var = var;
                e.kf = (int)bm | (bad ? 0x100 : 0) | (sat ? 0x200 : 0);
                wq[qn + __popc(bal & lt)] = e;
            }
            qn += __popc(bal);
            if (qn >= 32) {
                // one full round of 32 entries; the rest (< 32) moves to the front
                flush_queue<NR>(ap, wq, 32, f, v, fl);
                if (lane < qn - 32) wq[lane] = wq[lane + 32];
                __syncwarp();
                qn -= 32;
            }
        }
    }
    flush_queue<NR>(ap, wq, qn, f, v, fl);
    // Warp sums of every radius (all lanes hold them after the butterflies);
    // lane k stores radius k's raw float-float sums, and k_ap_finish turns
    // them into the flux, its error and the edge flag one (source, radius)
    // per thread, so the float64 steps issue once for 32 results.
    DF my_f = df_zero(), my_v = df_zero();
    uint32_t my_fl = 0u;
#pragma unroll
    for (int k = 0; k < NR; ++k) {
        const DF fs = df_warp_sum(f[k]);
        const DF vs = df_warp_sum(v[k]);
        uint32_t ff = fl[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ff |= __shfl_xor_sync(0xffffffffu, ff, o);
        if (lane == k) { my_f = fs; my_v = vs; my_fl = ff; }
    }
    if (lane < NR) {
        reinterpret_cast<float2*>(flux)[lane] = make_float2(my_f.hi, my_f.lo);
        reinterpret_cast<float2*>(ferr)[lane] = make_float2(my_v.hi, my_v.lo);
        aflags[lane] = my_fl;
    }
}

// Radius k's results at (cx, cy) from the raw sums in *flux and *ferr: the
// flux F, its error sqrt(V + F / gain) and the edge flag.
__device__ __forceinline__ void ap_finish(double cx, double cy, const ApSpec& ap, int k, int W, int H, double* flux,
                                          double* ferr, uint32_t* fl)
{
    const float2 fr = *reinterpret_cast<const float2*>(flux);
    const float2 vr = *reinterpret_cast<const float2*>(ferr);
    uint32_t f = *fl;
    const double r = ap.r[k];
    if (cx - r < -0.5 || cx + r > W - 0.5 || cy - r < -0.5 || cy + r > H - 0.5) f |= GP_FLAG_TRUNCATED;
    const double F = (double)fr.x + (double)fr.y;
    double V = (double)vr.x + (double)vr.y;
    if (ap.gain > 0.f && F > 0.0) V = fma(F, ap.inv_gain, V);
    // sqrt(V): a float32 estimate s0, then one Newton step in float64,
    // s0 + (V - s0^2) / (2 s0); the step is ~1e-7 s0, so a float32
    // reciprocal leaves ~1e-14 relative error
    double e = 0.0;
    if (V > 0.0) {
        const float s0f = sqrtf((float)V);
        if (s0f > 0.f) {
            const double s0 = (double)s0f;
            e = fma(fma(-s0, s0, V), (double)(0.5f / s0f), s0);
        }
    }
    *flux = F;
    *ferr = e;
    *fl = f;
}

// One warp per catalog row (segments in label order): copy the segment's
// finished moments into the row, then the apertures at its centroid.
// the frame's arguments: the kernel parameter itself for a single frame (a
// compile-time choice: hot-loop fields stay constant-bank operands), else the
// batch record of frame blockIdx.y
template <bool BATCH>
__device__ __forceinline__ const MeasureArgs& measure_frame(const MeasureArgs* __restrict__ batch,
                                                            const MeasureArgs& one)
{
    if constexpr (BATCH) return batch[blockIdx.y];
    else return one;
}

template <bool F32, int NR, bool BATCH>
__global__ void __launch_bounds__(MEAS_NT, 3) k_measure(const MeasureArgs* __restrict__ batch,
                                                     const __grid_constant__ MeasureArgs one)
{
    const MeasureArgs& A = measure_frame<BATCH>(batch, one);
    __shared__ BEntry queue[MEAS_NT / 32][QCAP];
    BEntry* wq = queue[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    const int ncomp = min(*A.C.count, A.C.cap);
    const int nrow = min(ncomp, A.capacity);
    const int W = A.im.W;
    for (int r = wid; r < nrow; r += nw) {
        const int c = A.C.perm[r];
        const double2 xy = A.C.xy[c];
        if (lane == 0) {
            const int4 bb = A.C.bbox[c];
            const Mom2 m2 = A.C.mom2[c];
            const uint32_t pL = A.C.peakL[c];
            A.label[r] = A.C.label[c];
            A.npix[r] = A.C.npix[c];
            A.flux_iso[r] = A.C.flux[c];
            A.x[r] = xy.x; A.y[r] = xy.y;
            A.x2[r] = m2.x2; A.y2[r] = m2.y2; A.xy[r] = m2.xy;
            A.xmin[r] = bb.x; A.xmax[r] = bb.y; A.ymin[r] = bb.z; A.ymax[r] = bb.w;
            A.peak[r] = A.C.peak[c];
            A.xpeak[r] = (int)(pL % (uint32_t)W); A.ypeak[r] = (int)(pL / (uint32_t)W);
            A.flags[r] = A.C.flags[c];
        }
        if constexpr (NR > 0)
            aperture_warp<F32, NR>(A.im, A.sb, A.sr, A.ap, xy.x, xy.y, A.apflux + (int64_t)r * NR,
                                   A.apferr + (int64_t)r * NR, A.apflags + (int64_t)r * NR, wq);
    }
}

template <bool F32, int NR>
__global__ void __launch_bounds__(MEAS_NT, 3) k_aperture(Image im, SplineTab sb, SplineTab sr, ApSpec ap,
                                                      const double* xs, const double* ys, int n, double* flux,
                                                      double* ferr, uint32_t* fl)
{
    __shared__ BEntry queue[MEAS_NT / 32][QCAP];
    BEntry* wq = queue[threadIdx.x >> 5];
    const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int i = wid; i < n; i += nw)
        aperture_warp<F32, NR>(im, sb, sr, ap, xs[i], ys[i], flux + (int64_t)i * NR, ferr + (int64_t)i * NR,
                               fl + (int64_t)i * NR, wq);
}

// the aperture results of the catalog rows (one (row, radius) per thread)
template <bool BATCH>
__global__ void __launch_bounds__(256) k_ap_finish_rows(const MeasureArgs* __restrict__ batch,
                                                        const __grid_constant__ MeasureArgs one)
{
    const MeasureArgs& A = measure_frame<BATCH>(batch, one);
    const int nr = A.ap.nr;
    const int nrow = min(min(*A.C.count, A.C.cap), A.capacity);
    const int64_t n = (int64_t)nrow * nr;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(i / nr), k = (int)(i - (int64_t)r * nr);
        ap_finish(A.x[r], A.y[r], A.ap, k, A.im.W, A.im.H, A.apflux + i, A.apferr + i, A.apflags + i);
    }
}

// the aperture results of a list of positions
static __global__ void __launch_bounds__(256) k_ap_finish_list(const double* xs, const double* ys, int n,
                                                        const __grid_constant__ ApSpec ap, int W,
                                                        int H, double* flux, double* ferr, uint32_t* fl)
{
    const int64_t tot = (int64_t)n * ap.nr;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot; i += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(i / ap.nr), k = (int)(i - (int64_t)j * ap.nr);
        ap_finish(xs[j], ys[j], ap, k, W, H, flux + i, ferr + i, fl + i);
    }
}

// dispatch on the number of radii (a compile-time constant in the kernels)
template <template <bool, int> class Launch, bool F32, typename... Args>
static cudaError_t dispatch_nr(int nr, Args... args)
{
    switch (nr) {
    case 0: return Launch<F32, 0>::run(args...);
    case 1: return Launch<F32, 1>::run(args...);
    case 2: return Launch<F32, 2>::run(args...);
    case 3: return Launch<F32, 3>::run(args...);
    case 4: return Launch<F32, 4>::run(args...);
    case 5: return Launch<F32, 5>::run(args...);
    case 6: return Launch<F32, 6>::run(args...);
    case 7: return Launch<F32, 7>::run(args...);
    default: return Launch<F32, 8>::run(args...);
    }
}

template <bool F32, int NR>
struct MeasureLaunch {
    static cudaError_t run(const MeasureArgs& one, dim3 g, cudaStream_t st)
    {
        k_measure<F32, NR, false><<<g, 256, 0, st>>>(nullptr, one);
        return cudaGetLastError();
    }
};

template <bool F32, int NR>
struct MeasureBatchLaunch {
    static cudaError_t run(const MeasureArgs& one, const MeasureArgs* batch, dim3 g, cudaStream_t st)
    {
        k_measure<F32, NR, true><<<g, 256, 0, st>>>(batch, one);
        return cudaGetLastError();
    }
};

// batched launch of k_measure (k_measure_batch.cu)
cudaError_t launch_measure_batched(const MeasureArgs& one, const MeasureArgs* batch, dim3 grid, cudaStream_t st);

template <bool F32, int NR>
struct ApertureLaunch {
    static cudaError_t run(Image im, SplineTab sb, SplineTab sr, ApSpec ap, const double* xs, const double* ys,
                           int n, double* flux, double* ferr, uint32_t* fl, int g, cudaStream_t st)
    {
        if (NR == 0) return cudaSuccess;
        k_aperture<F32, NR><<<g, 256, 0, st>>>(im, sb, sr, ap, xs, ys, n, flux, ferr, fl);
        k_ap_finish_list<<<g, 256, 0, st>>>(xs, ys, n, ap, im.W, im.H, flux, ferr, fl);
        return cudaGetLastError();
    }
};

}  // namespace gp
