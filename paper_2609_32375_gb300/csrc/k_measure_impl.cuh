// k_measure_impl.cuh -- device code of the catalog-row and aperture
// kernels (paper Section 3.4), shared by k_measure.cu (single-frame forms
// and the aperture entry point) and k_measure_batch.cu (batched forms), so
// the two sets of template instances compile in parallel.
#pragma once
#include <math.h>

#include "gp_internal.cuh"
#include "gp_launch.h"

namespace gp {
// square root by the hardware approximation (sqrt.approx.f32, about one ulp)
__device__ __forceinline__ float sqrt_ap(float x)
{
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// The angle atan(y / x) in [0, pi/2] for x, y >= 0, not both 0.  With
// u = min / max in [0, 1], atan(u) = u P(u^2), P the degree-8 polynomial
// that fits atan(u) / u on [0, 1] in least squares (weights iterated toward
// equal relative error; relative error below 2e-8 in exact arithmetic), and
// atan(y / x) = pi/2 - atan(x / y) above the diagonal.
__device__ __forceinline__ float atan_q1(float y, float x)
{
    const bool sw = y > x;
    const float u = __fdividef(sw ? x : y, sw ? y : x);
    const float s = u * u;
    float p = 0.002903404f;
    p = fmaf(p, s, -0.01628242f);
    p = fmaf(p, s, 0.043038424f);
    p = fmaf(p, s, -0.07533597f);
    p = fmaf(p, s, 0.10654641f);
    p = fmaf(p, s, -0.14207125f);
    p = fmaf(p, s, 0.19993053f);
    p = fmaf(p, s, -0.33333093f);
    p = fmaf(p, s, 1.0f);
    const float a = u * p;
    return sw ? 1.57079637f - a : a;
}

// integral of sqrt(r^2 - t^2) over [a, b], 0 <= a <= b <= r, written with
// differences formed algebraically (no cancellation between large terms):
// r^2 theta / 2 + (b hb - a ha) / 2 with theta = asin(b/r) - asin(a/r) from
// its sine and cosine.  The square roots, the one division and the angle use
// the fast forms above; on the host, this arithmetic against the oracle's
// float64 areas over radii 0.3-100 gives a worst absolute error of 1.5e-6
// at r = 10 and 1.5e-5 at r = 100.
__device__ __forceinline__ float chord_int(float a, float b, float r2)
{
    float d = b - a;
    if (!(d > 0.f)) return 0.f;
    float ha = sqrt_ap(fmaxf(fmaf(-a, a, r2), 0.f));
    float hb = sqrt_ap(fmaxf(fmaf(-b, b, r2), 0.f));
    float s = ha + hb;
    float q = s > 0.f ? __fdividef(d * (a + b), s) : 0.f;      // ha - hb
    float sin_t = fmaf(d, ha, a * q);               // (b ha - a hb), r^2 sin(theta)
    float cos_t = fmaf(ha, hb, a * b);              // (ha hb + a b), r^2 cos(theta)
    float theta = atan_q1(sin_t, cos_t);            // asin(b/r) - asin(a/r), in [0, pi/2]
    return 0.5f * fmaf(r2, theta, fmaf(d, hb, -a * q));
}

// exact area of disc(0, r) n [x0,x1] x [y0,y1] for a rectangle in the first
// quadrant (0 <= x0 < x1, 0 <= y0 < y1).  There the arc y = h(x) =
// sqrt(r^2 - x^2) falls monotonically: columns left of xa (h(xa) = y1) are
// covered to the full height, columns right of xb (h(xb) = y0) not at all,
// and in between to the height h(x) - y0.  So the area is one rectangle and
// one arc integral.  Every product and sum is an explicit operation (fmaf,
// __fmul_rn, __fadd_rn), so no instance of the kernels contracts it
// differently and a frame gives the same bits in a batched launch as alone.
__device__ __forceinline__ float quadrant_area(float x0, float x1, float y0, float y1, float r2)
{
    if (!(fmaf(x0, x0, __fmul_rn(y0, y0)) < r2)) return 0.f;   // the nearest corner is outside
    const float xa = sqrt_ap(fmaxf(fmaf(-y1, y1, r2), 0.f));
    const float xb = sqrt_ap(fmaxf(fmaf(-y0, y0, r2), 0.f));
    const float lo = fminf(fmaxf(xa, x0), x1);
    const float d = fmaxf(__fsub_rn(fminf(x1, xb), lo), 0.f);
    const float rect = __fmul_rn(__fsub_rn(y1, y0), __fsub_rn(lo, x0));
    return __fadd_rn(rect, fmaf(-y0, d, chord_int(lo, __fadd_rn(lo, d), r2)));
}

// One side of a pixel [a, a + 1] folded onto t >= 0: the piece [p0, p1],
// and for a pixel that straddles 0 the second piece [0, q1].
struct Fold {
    float p0, p1, q1;
    bool two;
};

__device__ __forceinline__ Fold fold_side(float a)
{
    const float b = __fadd_rn(a, 1.f);
    Fold f;
    f.two = a < 0.f && b > 0.f;
    f.p0 = a >= 0.f ? a : (b <= 0.f ? -b : 0.f);
    f.p1 = a >= 0.f ? b : (b <= 0.f ? -a : b);
    f.q1 = -a;
    return f;
}

// exact area of disc(0, r) n [dx0, dx0 + 1] x [dy0, dy0 + 1]: the pixel folded
// into the first quadrant by symmetry, a pixel on an axis split in two
__device__ __forceinline__ float pixel_area(float dx0, float dy0, float r)
{
    const float r2 = __fmul_rn(r, r);
    const Fold fx = fold_side(dx0), fy = fold_side(dy0);
    float A = quadrant_area(fx.p0, fx.p1, fy.p0, fy.p1, r2);
    if (fx.two) A = __fadd_rn(A, quadrant_area(0.f, fx.q1, fy.p0, fy.p1, r2));
    if (fy.two) A = __fadd_rn(A, quadrant_area(fx.p0, fx.p1, 0.f, fy.q1, r2));
    if (fx.two && fy.two) A = __fadd_rn(A, quadrant_area(0.f, fx.q1, 0.f, fy.q1, r2));
    return A;
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

// the flag bits a lane collects: bit k a bad pixel under disc k, bit 8 + k a
// saturated one
template <int NR>
__device__ __forceinline__ void flush_queue(const ApSpec& ap, BEntry* wq, int qn, DF* f, DF* v, uint32_t& pk)
{
    __syncwarp();
    const int lane = threadIdx.x & 31;
    for (int i = lane; i < qn; i += 32) {
        const BEntry e = wq[i];
        unsigned rm = e.kf & 0xffu;                  // the radii whose circle crosses the pixel
        while (rm) {
            const int k = __ffs(rm) - 1;
            rm &= rm - 1u;
            const float A = pixel_area(e.dx0, e.dy0, ap.r[k]);
            if (!(A > 0.f)) continue;
            if (e.kf & 0x100) { pk |= 1u << k; continue; }
            if (e.kf & 0x200) pk |= 0x100u << k;
#pragma unroll
            for (int kk = 0; kk < NR; ++kk) {
                if (kk != k) continue;
                df_add_prod(f[kk], A, e.m);
                df_add_prod(v[kk], A, e.var);
            }
        }
    }
    __syncwarp();
}

// Sums NV float-float values (a power of two) over the warp, one value per
// lane group at the end: in each of the first log2(NV) butterfly steps the
// partners split the values between them (each keeps one half and receives
// the other lane's copy of it), then the remaining steps sum the one value
// left.  Value i ends in the lanes whose bits (16, 8, ...) spell i.  The
// order of every combination is fixed, so the sums are reproducible.
template <int C, int O>
__device__ __forceinline__ void df_scatter_step(DF* v, int lane)
{
    if constexpr (O > 0) {
        const bool upper = (lane & O) != 0;
        if constexpr (C > 1) {
            constexpr int h = C / 2;
#pragma unroll
            for (int i = 0; i < h; ++i) {
                const DF send = upper ? v[i] : v[i + h];
                const DF keep = upper ? v[i + h] : v[i];
                DF recv;
                recv.hi = __shfl_xor_sync(0xffffffffu, send.hi, O);
                recv.lo = __shfl_xor_sync(0xffffffffu, send.lo, O);
                v[i] = upper ? df_merge(recv, keep) : df_merge(keep, recv);
            }
            df_scatter_step<h, O / 2>(v, lane);
        } else {
            DF w;
            w.hi = __shfl_xor_sync(0xffffffffu, v[0].hi, O);
            w.lo = __shfl_xor_sync(0xffffffffu, v[0].lo, O);
            v[0] = upper ? df_merge(w, v[0]) : df_merge(v[0], w);
            df_scatter_step<1, O / 2>(v, lane);
        }
    }
}

template <int NV>
__device__ __forceinline__ DF df_reduce_scatter(DF* v)
{
    df_scatter_step<NV, 16>(v, threadIdx.x & 31);
    return v[0];
}

// the value index df_reduce_scatter<NV> leaves in this lane: the top
// log2(NV) of the lane's five bits
template <int NV>
__device__ __forceinline__ int scatter_index(int lane)
{
    return lane / (32 / NV);
}

// Apertures around (cx, cy) for all radii; executed by one full warp.
// One lane per pixel column: the column's x-spline coefficients and the
// node-row values u_j, w_j of both maps are evaluated once per column and
// reused down the column; the y-spline coefficients of up to 32 rows are
// evaluated one row per lane and fetched by shuffle, so each pixel costs a
// few FMAs for B(p) and sigma(p).  Pixels wholly inside disc k add to a lane's
// float32 column sums (at most 32 terms, then folded into float-float sums);
// pixels the circle crosses go through the queue.  The queue order and the
// lane assignment are fixed, and lane results are combined in a fixed order,
// so the sums are reproducible.
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
    constexpr int NRA = NR > 0 ? NR : 1;
    constexpr int NV = 2 * NRA <= 2 ? 2 : 2 * NRA <= 4 ? 4 : 2 * NRA <= 8 ? 8 : 16;
    DF acc[NV];                                      // flux sums of radii 0..NR-1, then variance sums
#pragma unroll
    for (int i = 0; i < NV; ++i) acc[i] = df_zero();
    DF* f = acc;
    DF* v = acc + NRA;
    uint32_t pk = 0u;                                // bad (bit k) / saturated (bit 8 + k) under disc k
    const float rmax2 = ap.rmax * ap.rmax;
    const int nyn = sb.ay.n;
    int qn = 0;                                      // warp-uniform queue length
    for (int xbase = xa; xbase <= xb; xbase += 32) {
        const int x = xbase + lane;
        const bool colok = x <= xb;
        const int xl = colok ? x : xb;
        const float dx0 = (float)(x - xi) - xf - 0.5f, dx1 = dx0 + 1.f;
        const float nx = fmaxf(0.f, fmaxf(dx0, -dx1));
        const float fx = fmaxf(dx0 * dx0, dx1 * dx1);
        const AxCoef ccx = axis_coef(sb.ax, (float)xl);
        int jc = -1;                       // node row pair cached for this column
        float ub0 = 0, ub1 = 0, wb0 = 0, wb1 = 0, ur0 = 0, ur1 = 0, wr0 = 0, wr1 = 0;
        for (int ybase = ya; ybase <= yb; ybase += 32) {
            const AxCoef cyl = axis_coef(sb.ay, (float)min(ybase + lane, yb));   // row ybase + lane
            const int yend = min(yb, ybase + 31);
            float fs[NRA], vs[NRA];
#pragma unroll
            for (int k = 0; k < NRA; ++k) { fs[k] = 0.f; vs[k] = 0.f; }
            for (int y = ybase; y <= yend; ++y) {
                const float dy0 = (float)(y - yi) - yf - 0.5f, dy1 = dy0 + 1.f;
                const float ny = fmaxf(0.f, fmaxf(dy0, -dy1));
                if (!(ny * ny < rmax2)) continue;        // a row beyond the largest disc (the whole warp)
                const int j = y - ybase;
                AxCoef ccy;
                ccy.i = __shfl_sync(0xffffffffu, cyl.i, j);
                ccy.b = __shfl_sync(0xffffffffu, cyl.b, j);
                ccy.c0 = __shfl_sync(0xffffffffu, cyl.c0, j);
                ccy.c1 = __shfl_sync(0xffffffffu, cyl.c1, j);
                ccy.i1 = min(ccy.i + 1, nyn - 1);
                if (ccy.i != jc) {
                    const float2 b0 = row_eval(sb, ccy.i, ccx), b1 = row_eval(sb, ccy.i1, ccx);
                    const float2 r0 = row_eval(sr, ccy.i, ccx), r1 = row_eval(sr, ccy.i1, ccx);
                    ub0 = b0.x; wb0 = b0.y; ub1 = b1.x; wb1 = b1.y;
                    ur0 = r0.x; wr0 = r0.y; ur1 = r1.x; wr1 = r1.y;
                    jc = ccy.i;
                }
                const float dmin2 = fmaf(nx, nx, ny * ny);
                const float dmax2 = fx + fmaxf(dy0 * dy0, dy1 * dy1);
                const bool live = colok && dmin2 < rmax2;
                bool bad;
                const float val = load_px<F32>(im, xl, y, bad);
                const float sg = axis_combine(ccy, ur0, ur1, wr0, wr1);
                const float m = bad ? 0.f : __fsub_rn(val, axis_combine(ccy, ub0, ub1, wb0, wb1));
                const float var = bad ? 0.f : __fmul_rn(sg, sg);
                const bool sat = !bad && im.sat > 0.f && val >= im.sat;
                unsigned fm = 0u, bm = 0u;           // radii holding the pixel whole / crossing it
#pragma unroll
                for (int k = 0; k < NR; ++k) {
                    const float r2 = ap.r[k] * ap.r[k];
                    const bool full = live && dmax2 <= r2;
                    const bool in = live && dmin2 < r2;
                    fs[k] = __fadd_rn(fs[k], full ? m : 0.f);
                    vs[k] = __fadd_rn(vs[k], full ? var : 0.f);
                    fm |= full ? 1u << k : 0u;
                    bm |= (in && !full) ? 1u << k : 0u;
                }
                pk |= bad ? fm : (sat ? fm << 8 : 0u);
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
                    flush_queue<NR>(ap, wq, 32, f, v, pk);
                    if (lane < qn - 32) wq[lane] = wq[lane + 32];
                    __syncwarp();
                    qn -= 32;
                }
            }
#pragma unroll
            for (int k = 0; k < NR; ++k) {
                df_add(f[k], fs[k]);
                df_add(v[k], vs[k]);
            }
        }
    }
    flush_queue<NR>(ap, wq, qn, f, v, pk);
    // Warp sums of every radius, one value per lane group; the lane holding
    // radius k's flux sum (and the one holding its variance sum) stores the
    // raw float-float pair, and k_ap_finish turns them into the flux, its
    // error and the edge flag one (source, radius) per thread, so the
    // float64 steps issue once for 32 results.
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) pk |= __shfl_xor_sync(0xffffffffu, pk, o);
    const DF s = df_reduce_scatter<NV>(acc);
    const int idx = scatter_index<NV>(lane);
    const bool first = (lane & ((32 / NV) - 1)) == 0;     // one writer per value
    if (first && idx < NR) {
        reinterpret_cast<float2*>(flux)[idx] = make_float2(s.hi, s.lo);
        aflags[idx] = ((pk >> idx) & 1u ? GP_FLAG_BAD : 0u) | ((pk >> (8 + idx)) & 1u ? GP_FLAG_SAT : 0u);
    }
    if (first && idx >= NRA && idx < NRA + NR) reinterpret_cast<float2*>(ferr)[idx - NRA] = make_float2(s.hi, s.lo);
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

// One warp per catalog row (segments in label order): the apertures at its
// centroid (the row's other columns are written by k_ap_finish_rows).
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
    pdl_wait();
    pdl_release();
    const MeasureArgs& A = measure_frame<BATCH>(batch, one);
    __shared__ BEntry queue[MEAS_NT / 32][QCAP];
    BEntry* wq = queue[threadIdx.x >> 5];
    const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    const int ncomp = min(*A.C.count, A.C.cap);
    const int nrow = min(ncomp, A.capacity);
    for (int r = wid; r < nrow; r += nw) {
        const double2 xy = A.C.xy[A.C.perm[r]];
        if constexpr (NR > 0)
            aperture_warp<F32, NR>(A.im, A.sb, A.sr, A.ap, xy.x, xy.y, A.apflux + (int64_t)r * NR,
                                   A.apferr + (int64_t)r * NR, A.apflags + (int64_t)r * NR, wq);
    }
}

template <bool F32, int NR>
__global__ void __launch_bounds__(MEAS_NT, 3) k_aperture(Image im, SplineTab sb, SplineTab sr,
                                                      const __grid_constant__ ApSpec ap,
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

// The catalog rows in label order: thread (row, 0) copies the segment's
// finished moments into the row, and thread (row, k) finishes the aperture
// results of radius k (one (row, radius) per thread).
template <bool BATCH>
__global__ void __launch_bounds__(256) k_ap_finish_rows(const MeasureArgs* __restrict__ batch,
                                                        const __grid_constant__ MeasureArgs one)
{
    pdl_wait();
    pdl_release();
    const MeasureArgs& A = measure_frame<BATCH>(batch, one);
    const int nr = A.ap.nr, nk = nr > 0 ? nr : 1;
    const int W = A.im.W;
    const int nrow = min(min(*A.C.count, A.C.cap), A.capacity);
    const int64_t n = (int64_t)nrow * nk;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(i / nk), k = (int)(i - (int64_t)r * nk);
        const int c = A.C.perm[r];
        const double2 xy = A.C.xy[c];
        if (k == 0) {
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
        if (nr > 0) {
            const int64_t j = (int64_t)r * nr + k;
            ap_finish(xy.x, xy.y, A.ap, k, A.im.W, A.im.H, A.apflux + j, A.apferr + j, A.apflags + j);
        }
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
        launch_dep(k_measure<F32, NR, false>, g, dim3(256), 0, st, (const MeasureArgs*)nullptr, one);
        return cudaGetLastError();
    }
};

template <bool F32, int NR>
struct MeasureBatchLaunch {
    static cudaError_t run(const MeasureArgs& one, const MeasureArgs* batch, dim3 g, cudaStream_t st)
    {
        launch_dep(k_measure<F32, NR, true>, g, dim3(256), 0, st, batch, one);
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
