// k_detect.cu -- matched-filter detection and segmentation (paper Section
// 3.2, with labelled segments in place of the paper's local maxima) and the
// segment moments (its first-moment centroid, extended to second moments,
// bounding box and peak).
//
//  k_detect_tile  one CTA per 64 x 32 tile.  Stages the tile plus a filter
//                 halo in shared memory as m = I - B (the spline background
//                 evaluated from per-column node rows; 16-byte vector loads
//                 on interior tiles), correlates it with the normalised
//                 kernel (each thread slides down 8 rows of one column),
//                 thresholds F > k sigma(p), labels the tile's 8-connected
//                 components by union-find in shared memory (root = minimum
//                 index = the segment's first pixel in raster order) and
//                 accumulates each component's moment sums from the staged m
//                 (one warp per component, fixed order).  A tile without
//                 foreground writes its empty map rows and edge records and
//                 stops after thresholding.  Components that do not touch an
//                 edge shared with another tile are final here (raw sums);
//                 the others become "pieces" with partial sums, and their
//                 edge pixels are recorded for the merge.
//  k_merge        unites pieces across tile edges (lock-free union-find
//                 over piece ids, atomicMin linking).
//  k_aggregate    sums piece sizes, bounding boxes and minimum indices at
//                 each union-find root.
//  k_finalize     merges the partial moments of each multi-tile segment in
//                 tile raster order (deterministic), and rewrites the map
//                 pixels of pieces whose final label differs (other root, or
//                 below minarea) -- a sparse pass over those pieces only.
//  k_mom_finish   centroid and second moments of every segment from its raw
//                 sums, one segment per thread (the float64 steps issue once
//                 for 32 segments).
//  k_rank_*       orders segments by label (bucket counts, one scan,
//                 scatter, in-bucket rank): a deterministic catalog order.
#include <math.h>

#include "gp_internal.cuh"
#include "gp_launch.h"

namespace gp {

static_assert(TX == 64, "row masks hold one 64-pixel tile row");
constexpr int DT_NT = 256;
constexpr int ROWS_PER_THREAD = TNPIX / DT_NT;     // 8: each thread filters 8 rows of one column

// mirror without edge repeat, cheap for offsets within one reflection
__device__ __forceinline__ int mirror_fast(int i, int N)
{
    if (i < 0) i = -i;
    if (i >= N) i = 2 * (N - 1) - i;
    return (i >= 0 && i < N) ? i : mirror_idx(i, N);
}

// ------------------------------------------------ shared-memory union-find ---
__device__ __forceinline__ int sfind(volatile int* lab, int x)
{
    for (int n = 0; n < TNPIX + 1; ++n) {
        int p = lab[x];
        if (p == x) return x;
        x = p;
    }
    return x;
}

__device__ __forceinline__ void sunite(int* lab, int a, int b)
{
    for (int it = 0; it < 4 * TNPIX; ++it) {
        a = sfind(lab, a);
        b = sfind(lab, b);
        if (a == b) return;
        if (a < b) { int t = a; a = b; b = t; }
        int old = atomicMin(lab + a, b);
        if (old == a) return;
        a = old;
    }
}

// ---------------------------------------------------- global union-find ---
__device__ __forceinline__ int gfind(const int* parent, int x)
{
    for (int n = 0; n < WALK_LIMIT; ++n) {
        int p = __ldcg(parent + x);
        if (p == x) return x;
        x = p;
    }
    return -1;
}

__device__ void gunite(int* parent, int a, int b, int* status)
{
    for (int it = 0; it < WALK_LIMIT; ++it) {
        a = gfind(parent, a);
        b = gfind(parent, b);
        if (a < 0 || b < 0) break;
        if (a == b) return;
        if (a < b) { int t = a; a = b; b = t; }
        int old = atomicMin(parent + a, b);
        if (old == a) return;
        a = old;
    }
    set_status(status, GP_ERR_TIMEOUT);
}

// block-wide exclusive scan of one int per thread (DT_NT threads)
__device__ __forceinline__ int block_excl_scan(int v, int* warp_tot, int* total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int w = lane < DT_NT / 32 ? warp_tot[lane] : 0;
        int wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += t;
        }
        if (lane < DT_NT / 32) warp_tot[lane] = wi - w;
        if (lane == DT_NT / 32 - 1) *total = wi;
    }
    __syncthreads();
    int r = warp_tot[warp] + incl - v;
    __syncthreads();
    return r;
}

// ------------------------------------------------------------- moments ---
struct MomAcc {
    DF s, sx, sy, sxx, syy, sxy;
    int ux, uy, uxx, uyy, uxy;
    float peak;
    uint32_t peakL;
    uint32_t flags;
};

__device__ __forceinline__ void mom_zero(MomAcc& a)
{
    a.s = a.sx = a.sy = a.sxx = a.syy = a.sxy = df_zero();
    a.ux = a.uy = a.uxx = a.uyy = a.uxy = 0;
    a.peak = -INFINITY;
    a.peakL = 0xffffffffu;
    a.flags = 0u;
}

__device__ __forceinline__ void mom_pixel(MomAcc& a, float m, int dx, int dy, uint32_t L, bool sat)
{
    const float fx = (float)dx, fy = (float)dy;
    df_add(a.s, m);
    df_add_prod(a.sx, fx, m);
    df_add_prod(a.sy, fy, m);
    df_add_prod(a.sxx, fx * fx, m);
    df_add_prod(a.syy, fy * fy, m);
    df_add_prod(a.sxy, fx * fy, m);
    a.ux += dx; a.uy += dy;
    a.uxx += dx * dx; a.uyy += dy * dy; a.uxy += dx * dy;
    if (m > a.peak || (m == a.peak && L < a.peakL)) { a.peak = m; a.peakL = L; }
    if (sat) a.flags |= GP_FLAG_SAT;
}

__device__ __forceinline__ void mom_warp_reduce(MomAcc& a)
{
    a.s = df_warp_sum(a.s); a.sx = df_warp_sum(a.sx); a.sy = df_warp_sum(a.sy);
    a.sxx = df_warp_sum(a.sxx); a.syy = df_warp_sum(a.syy); a.sxy = df_warp_sum(a.sxy);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a.ux += __shfl_xor_sync(0xffffffffu, a.ux, o);
        a.uy += __shfl_xor_sync(0xffffffffu, a.uy, o);
        a.uxx += __shfl_xor_sync(0xffffffffu, a.uxx, o);
        a.uyy += __shfl_xor_sync(0xffffffffu, a.uyy, o);
        a.uxy += __shfl_xor_sync(0xffffffffu, a.uxy, o);
        a.flags |= __shfl_xor_sync(0xffffffffu, a.flags, o);
        float op = __shfl_xor_sync(0xffffffffu, a.peak, o);
        uint32_t oL = __shfl_xor_sync(0xffffffffu, a.peakL, o);
        if (op > a.peak || (op == a.peak && oL < a.peakL)) { a.peak = op; a.peakL = oL; }
    }
}

__device__ __forceinline__ float2 df2(DF d) { return make_float2(d.hi, d.lo); }

// finished moments of a whole segment from sums about the origin (X0, Y0)
__device__ void mom_finish(double S, double Sx, double Sy, double Sxx, double Syy, double Sxy, long long ux,
                           long long uy, long long uxx, long long uyy, long long uxy, int npix, int X0, int Y0,
                           double* flux, double2* xy, Mom2* m2, uint32_t* flags)
{
    *flux = S;
    if (S > 0.0) {
        const double iS = recip_pos(S);
        const double mx = Sx * iS, my = Sy * iS;
        *xy = make_double2(X0 + mx, Y0 + my);
        *m2 = mom2_make(Sxx * iS - mx * mx, Syy * iS - my * my, Sxy * iS - mx * my, 0.0);
    } else {
        const double in = recip_pos((double)npix);
        const double mx = (double)ux * in, my = (double)uy * in;
        *xy = make_double2(X0 + mx, Y0 + my);
        *m2 = mom2_make((double)uxx * in - mx * mx, (double)uyy * in - my * my, (double)uxy * in - mx * my, 0.0);
        *flags |= GP_FLAG_CENTROID_FALLBACK;
    }
}

// A segment's sum S = hi + lo is positive exactly when hi > -lo (a float
// comparison, exact), the same decision as (double)hi + (double)lo > 0.
__device__ __forceinline__ bool df_positive(DF d) { return d.hi > -d.lo; }

// Origin of a segment's stored sums: the corner of the detection tile that
// holds the top-left pixel of its bounding box.
__device__ __forceinline__ int2 comp_origin(int4 bb) { return make_int2(bb.x / TX * TX, bb.z / TY * TY); }

// A segment with positive sum keeps its raw float-float sums in its own
// catalog fields until k_mom_finish finishes them: flux holds S, xy holds
// (Sx, Sy), mom2 holds (Sxx, Syy, Sxy), all about comp_origin.  Finishing
// them one segment per thread issues the float64 steps once for 32 segments
// instead of once per segment on a single lane of a warp.
__device__ __forceinline__ void comp_store_raw(const Comps& C, int id, DF s, DF sx, DF sy, DF sxx, DF syy, DF sxy)
{
    reinterpret_cast<float2*>(C.flux)[id] = make_float2(s.hi, s.lo);
    reinterpret_cast<float4*>(C.xy)[id] = make_float4(sx.hi, sx.lo, sy.hi, sy.lo);
    float4* m = reinterpret_cast<float4*>(C.mom2 + id);
    m[0] = make_float4(sxx.hi, sxx.lo, syy.hi, syy.lo);
    m[1] = make_float4(sxy.hi, sxy.lo, 0.f, 0.f);
}

// ----------------------------------------------------------- tile kernel ---
// Staged columns: SMEM column c holds frame column x0 - XHALO + c (so 16-byte
// chunks of the frame land on 16-byte boundaries); staged rows: row r holds
// frame row y0 - hh + r.
struct TileSmem {
    float m[SH * SW];                 // staged pixels, then m = I - B
    int lab[TNPIX];
    uint8_t pflag[TNPIX];             // bit 0 bad, bit 1 saturated
    union {
        struct {                      // per staged column and node row (SoA)
            float ub[NJMAX * SW], wb[NJMAX * SW], ur[NJMAX * SW], wr[NJMAX * SW];
        } col;
        short rid[TNPIX];             // after thresholding: root pixel -> compact root id
    } u;
    float4 rowc[SH];                  // per staged row: (b, c0, c1, -)
    int2 rowj[SH];
    int r_npix[MAXROOT];
    int r_xmin[MAXROOT], r_xmax[MAXROOT], r_ymin[MAXROOT], r_ymax[MAXROOT];
    int r_pidx[MAXROOT];              // border flag, then local piece index
    int r_pix[MAXROOT];               // root's tile pixel
    int r_val[MAXROOT];               // value written to the map
    int r_rec[MAXROOT];               // piece id (>= 0), -2 - component id, or -1
    uint32_t rmask[2 * TY];           // foreground bits per tile row (two 32-pixel halves)
    int warp_tot[DT_NT / 32];
    int jlo, jhi, nroots, npieces, ncomps, pbase, cbase, nnear;
};

// the 64 foreground bits of tile row y (bit x = pixel x)
__device__ __forceinline__ uint64_t row_mask(const TileSmem& S, int y)
{
    return (uint64_t)S.rmask[2 * y] | ((uint64_t)S.rmask[2 * y + 1] << 32);
}

__device__ __forceinline__ float combine_row(const float4& rc, float v0, float v1, float m0, float m1)
{
    return fmaf(rc.z, m1, fmaf(rc.y, m0, fmaf(rc.x, v1 - v0, v0)));
}

// background at staged cell (ry, c)
__device__ __forceinline__ float cell_bkg(const TileSmem& S, int ry, int c)
{
    const int2 j = S.rowj[ry];
    return combine_row(S.rowc[ry], S.u.col.ub[j.x * SW + c], S.u.col.ub[j.y * SW + c], S.u.col.wb[j.x * SW + c],
                       S.u.col.wb[j.y * SW + c]);
}

// A 16-byte chunk q of the staged window (row q / nchunk, chunk q % nchunk)
// as raw bits: 8 uint16 pixels or 4 float32 pixels.  The frame's last chunk
// of a row may stop short of the vector width: those lanes repeat the last
// column (they lie outside the columns in use).
template <bool F32>
__device__ __forceinline__ uint4 load_chunk(const Image& im, int xa, int nchunk, unsigned inv_nchunk, int gy0, int q)
{
    constexpr int VEC = F32 ? 4 : 8;
    const int ry = (int)(((unsigned)q * inv_nchunk) >> 16), ch = q - ry * nchunk;
    const int64_t row = (int64_t)(gy0 + ry) * im.pitch;
    const int gx0 = xa + ch * VEC, W = im.W;
    if (gx0 + VEC <= W) {
        if (F32) {
            const float4 w = __ldg(reinterpret_cast<const float4*>(reinterpret_cast<const float*>(im.data) + row + gx0));
            return make_uint4(__float_as_uint(w.x), __float_as_uint(w.y), __float_as_uint(w.z), __float_as_uint(w.w));
        }
        return __ldg(reinterpret_cast<const uint4*>(reinterpret_cast<const uint16_t*>(im.data) + row + gx0));
    }
    uint32_t w[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        if (F32) {
            const int gx = gx0 + e < W ? gx0 + e : W - 1;
            w[e] = __float_as_uint(__ldg(reinterpret_cast<const float*>(im.data) + row + gx));
        } else {
            const int ga = gx0 + 2 * e < W ? gx0 + 2 * e : W - 1, gb = gx0 + 2 * e + 1 < W ? gx0 + 2 * e + 1 : W - 1;
            const uint16_t* px = reinterpret_cast<const uint16_t*>(im.data) + row;
            w[e] = (uint32_t)__ldg(px + ga) | ((uint32_t)__ldg(px + gb) << 16);
        }
    }
    return make_uint4(w[0], w[1], w[2], w[3]);
}

struct StageGeo {
    int xa, nchunk;
    unsigned inv_nchunk;
    int clo, chi, hh, th, tw, c_org;   // c_org: frame column of staged column 0
};

// m = I - B of one chunk from its raw bits, the spline background taken
// from the per-column node-row values (16-byte shared loads: a chunk starts
// on a 4-column boundary); columns outside the ones in use get 0.  Bad
// (non-finite) and saturated pixels of the tile are flagged.
template <bool F32>
__device__ __forceinline__ void stage_chunk(TileSmem& S, float sat, const StageGeo& g, uint4 raw, int q)
{
    constexpr int VEC = F32 ? 4 : 8;
    const int ry = (int)(((unsigned)q * g.inv_nchunk) >> 16), ch = q - ry * g.nchunk;
    const int c0 = g.xa + ch * VEC - g.c_org;
    float v[VEC];
    const uint32_t u4[4] = {raw.x, raw.y, raw.z, raw.w};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        if (F32) {
            v[e] = __uint_as_float(u4[e]);
        } else {
            v[2 * e] = (float)(u4[e] & 0xffffu);
            v[2 * e + 1] = (float)(u4[e] >> 16);
        }
    }
    const float4 rc = S.rowc[ry];
    const int2 j = S.rowj[ry];
    const int py = ry - g.hh;
    const bool row_in = py >= 0 && py < g.th;
#pragma unroll
    for (int k = 0; k < VEC / 4; ++k) {
        const int c = c0 + 4 * k;
        const float4 u0 = *reinterpret_cast<const float4*>(S.u.col.ub + j.x * SW + c);
        const float4 u1 = *reinterpret_cast<const float4*>(S.u.col.ub + j.y * SW + c);
        const float4 w0 = *reinterpret_cast<const float4*>(S.u.col.wb + j.x * SW + c);
        const float4 w1 = *reinterpret_cast<const float4*>(S.u.col.wb + j.y * SW + c);
        const float a0[4] = {u0.x, u0.y, u0.z, u0.w}, a1[4] = {u1.x, u1.y, u1.z, u1.w};
        const float b0[4] = {w0.x, w0.y, w0.z, w0.w}, b1[4] = {w1.x, w1.y, w1.z, w1.w};
        float m[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float val = v[4 * k + e];
            const int cc = c + e;
            const bool bad = F32 ? !isfinite(val) : false;
            const bool use = cc >= g.clo && cc < g.chi;
            m[e] = (bad || !use) ? 0.f : val - combine_row(rc, a0[e], a1[e], b0[e], b1[e]);
            const int px = cc - XHALO;
            if (row_in && use && px >= 0 && px < g.tw)
                S.pflag[py * TX + px] = (bad ? 1 : 0) | ((!bad && sat > 0.f && val >= sat) ? 2 : 0);
        }
        *reinterpret_cast<float4*>(S.m + ry * SW + c) = make_float4(m[0], m[1], m[2], m[3]);
    }
}

// F at 8 consecutive rows of one column: slide the kernel window down the
// column so each staged value is read once per kernel column
template <int KS>
__device__ __forceinline__ void filter_column(const TileSmem& S, const DetectArgs& A, int px, int py0, int hh,
                                              float* F)
{
    if (KS > 0) {
        constexpr int H = KS / 2;
#pragma unroll
        for (int i = 0; i < ROWS_PER_THREAD; ++i) F[i] = 0.f;
        const int c0 = px + XHALO - H;
        const int r0 = py0 + hh - H;
#pragma unroll
        for (int rr = 0; rr < ROWS_PER_THREAD + KS - 1; ++rr) {
            float v[KS > 0 ? KS : 1];
#pragma unroll
            for (int u = 0; u < KS; ++u) v[u] = S.m[(r0 + rr) * SW + c0 + u];
#pragma unroll
            for (int i = 0; i < ROWS_PER_THREAD; ++i) {
                const int kv = rr - i;
                if (kv >= 0 && kv < KS) {
#pragma unroll
                    for (int u = 0; u < KS; ++u) F[i] = fmaf(A.K[kv * KS + u], v[u], F[i]);
                }
            }
        }
    } else {
        for (int i = 0; i < ROWS_PER_THREAD; ++i) {
            float f = 0.f;
            const int r0 = py0 + i + hh - A.hy, c0 = px + XHALO - A.hx;
            for (int v = 0; v < A.kh; ++v) {
                const float* row = S.m + (r0 + v) * SW + c0;
                const float* kr = A.K + v * A.kw;
                for (int u = 0; u < A.kw; ++u) f = fmaf(kr[u], row[u], f);
            }
            F[i] = f;
        }
    }
}

// the frame's arguments: the kernel parameter itself for a single frame (a
// compile-time choice, so the taps stay in the constant bank), else the
// batch record of frame blockIdx.y
template <bool BATCH>
__device__ __forceinline__ const DetectArgs& detect_args(const DetectArgs* __restrict__ batch, const DetectArgs& one)
{
    if constexpr (BATCH) return batch[blockIdx.y];
    else return one;
}

template <bool F32, bool LABEL_ONLY, int KS, bool BATCH>
__global__ void __launch_bounds__(DT_NT) k_detect_tile(const DetectArgs* __restrict__ batch,
                                                       const __grid_constant__ DetectArgs one)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TileSmem& S = *reinterpret_cast<TileSmem*>(smem_raw);
    const DetectArgs& A = detect_args<BATCH>(batch, one);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int W = A.im.W, H = A.im.H;
    const int tile = blockIdx.x;
    const int ntx = A.T.ntx;
    if (BATCH && tile >= ntx * A.T.nty) return;
    const int tx = tile % ntx, ty = tile / ntx;
    const int x0 = tx * TX, y0 = ty * TY;
    const int tw = min(TX, W - x0), th = min(TY, H - y0);
    const int hh = LABEL_ONLY ? 0 : A.hh;

    if (!LABEL_ONLY) {
        const int srows = th + 2 * hh;
        const int clo = XHALO - hh, chi = XHALO + tw + hh;      // staged columns in use
        if (tid == 0) { S.jlo = 1 << 30; S.jhi = -1; S.nnear = 0; }
        __syncthreads();
        // spline coefficients of the staged rows (and the node rows they need)
        AxCoef cy;
        if (tid < srows) {
            const int gy = mirror_fast(y0 - hh + tid, H);
            cy = axis_coef(A.sb.ay, (float)gy);
            atomicMin(&S.jlo, cy.i);
            atomicMax(&S.jhi, cy.i1);
        }
        __syncthreads();
        const int jlo = S.jlo;
        const int nj = S.jhi - jlo + 1;
        if (nj > NJMAX) {   // excluded by the host's mesh >= 16 rule
            if (tid == 0) set_status(A.status, GP_ERR_INTERNAL);
            return;
        }
        if (tid < srows) {
            S.rowc[tid] = make_float4(cy.b, cy.c0, cy.c1, 0.f);
            S.rowj[tid] = make_int2(cy.i - jlo, cy.i1 - jlo);
        }
        // ---- stage the pixels over tile + halo (mirror border) as m = I - B
        const bool interior = x0 - hh >= 0 && x0 + tw + hh <= W && y0 - hh >= 0 && y0 + th + hh <= H;
        constexpr int VEC = F32 ? 4 : 8;          // pixels per 16-byte load
        const bool vec_ok = interior && !A.im.mask && ((((uintptr_t)A.im.data) & 15) == 0) &&
                            ((A.im.pitch % VEC) == 0);
        // 16-byte chunks covering [x0 - hh, x0 + tw + hh); frame column
        // x0 - XHALO is chunk aligned, so chunks land on 16-byte boundaries
        const int xa = (x0 - hh) & ~(VEC - 1);
        const int nchunk = (x0 + tw + hh - xa + VEC - 1) / VEC;
        // q / nchunk by multiply-shift, exact for every q < 46 * nchunk and nchunk <= 39
        const unsigned inv_nchunk = (65536u + nchunk - 1) / nchunk;
        const int nq = vec_ok ? srows * nchunk : 0;
        // this thread's first two chunks are read before the column values
        // are evaluated, so the two global-load latencies overlap
        uint4 raw0 = make_uint4(0u, 0u, 0u, 0u), raw1 = raw0;
        if (tid < nq) raw0 = load_chunk<F32>(A.im, xa, nchunk, inv_nchunk, y0 - hh, tid);
        if (tid + DT_NT < nq) raw1 = load_chunk<F32>(A.im, xa, nchunk, inv_nchunk, y0 - hh, tid + DT_NT);

        // spline values of node rows jlo.. at every staged column in use,
        // one (node row, column) pair per thread
        const int ncol = chi - clo;
        for (int q = tid; q < nj * ncol; q += DT_NT) {
            const int jj = q / ncol, c = clo + q - jj * ncol;
            const int gx = mirror_fast(x0 - XHALO + c, W);
            const AxCoef cx = axis_coef(A.sb.ax, (float)gx);
            const float2 b = row_eval(A.sb, jlo + jj, cx);
            const float2 r = row_eval(A.sr, jlo + jj, cx);
            S.u.col.ub[jj * SW + c] = b.x; S.u.col.wb[jj * SW + c] = b.y;
            S.u.col.ur[jj * SW + c] = r.x; S.u.col.wr[jj * SW + c] = r.y;
        }
        __syncthreads();

        if (vec_ok) {
            const StageGeo g{xa, nchunk, inv_nchunk, clo, chi, hh, th, tw, x0 - XHALO};
            if (tid < nq) stage_chunk<F32>(S, A.im.sat, g, raw0, tid);
            if (tid + DT_NT < nq) stage_chunk<F32>(S, A.im.sat, g, raw1, tid + DT_NT);
            for (int q = tid + 2 * DT_NT; q < nq; q += DT_NT)
                stage_chunk<F32>(S, A.im.sat, g, load_chunk<F32>(A.im, xa, nchunk, inv_nchunk, y0 - hh, q), q);
        } else {
            for (int ry = warp; ry < srows; ry += DT_NT / 32)
            for (int c = clo + lane; c < chi; c += 32) {
                const int gx = mirror_fast(x0 - XHALO + c, W), gy = mirror_fast(y0 - hh + ry, H);
                float v;
                bool bad;
                if (F32) {
                    v = __ldg(reinterpret_cast<const float*>(A.im.data) + (int64_t)gy * A.im.pitch + gx);
                    bad = !isfinite(v);
                } else {
                    v = (float)__ldg(reinterpret_cast<const uint16_t*>(A.im.data) + (int64_t)gy * A.im.pitch + gx);
                    bad = false;
                }
                if (A.im.mask && A.im.mask[(int64_t)gy * W + gx]) bad = true;
                S.m[ry * SW + c] = bad ? 0.f : v - cell_bkg(S, ry, c);
                const int py = ry - hh, px = c - XHALO;
                if (py >= 0 && py < th && px >= 0 && px < tw)
                    S.pflag[py * TX + px] = (bad ? 1 : 0) | ((!bad && A.im.sat > 0.f && v >= A.im.sat) ? 2 : 0);
            }
        }
        __syncthreads();

        // ---- matched filter and threshold: thread = one column, 8 rows
        {
            const int px = tid % TX;
            const int py0 = (tid / TX) * ROWS_PER_THREAD;
            float F[ROWS_PER_THREAD];
            filter_column<KS>(S, A, px, py0, hh, F);
            int nnear = 0;
            // the column's rms node-row values, reloaded only when the row's
            // node interval changes (the same for the whole warp)
            int jc = -1;
            float ru0 = 0.f, ru1 = 0.f, rw0 = 0.f, rw1 = 0.f;
#pragma unroll
            for (int i = 0; i < ROWS_PER_THREAD; ++i) {
                const int py = py0 + i;
                const int p = py * TX + px;
                bool fg = false;
                if (py < th && px < tw) {
                    const int2 j = S.rowj[py + hh];          // staged rows 0 .. th + 2 hh - 1 are set
                    if (j.x != jc) {
                        const int c = px + XHALO;
                        ru0 = S.u.col.ur[j.x * SW + c]; ru1 = S.u.col.ur[j.y * SW + c];
                        rw0 = S.u.col.wr[j.x * SW + c]; rw1 = S.u.col.wr[j.y * SW + c];
                        jc = j.x;
                    }
                    const float sig = combine_row(S.rowc[py + hh], ru0, ru1, rw0, rw1);
                    const float thr = A.thresh * sig;
                    fg = (F[i] > thr) && !(S.pflag[p] & 1);
                    if (fabsf(F[i] - thr) <= 1e-5f * fabsf(thr)) ++nnear;
                    if (A.mask_out) A.mask_out[(int64_t)(y0 + py) * W + x0 + px] = fg ? 1 : 0;
                }
                // the warp holds 32 consecutive pixels of this row
                const unsigned bits = __ballot_sync(0xffffffffu, fg);
                if (lane == 0) S.rmask[2 * py + (px >> 5)] = bits;
            }
            if (A.nnear) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) nnear += __shfl_xor_sync(0xffffffffu, nnear, o);
                if (lane == 0 && nnear) atomicAdd(&S.nnear, nnear);
            }
        }
        __syncthreads();
        if (A.nnear && tid == 0 && S.nnear) atomicAdd(A.nnear, S.nnear);
    } else {
        for (int p = tid; p < TNPIX; p += DT_NT) {
            const int py = p / TX, px = p - py * TX;
            const bool fg = py < th && px < tw && A.in_mask[(int64_t)(y0 + py) * W + x0 + px] != 0;
            const unsigned bits = __ballot_sync(0xffffffffu, fg);     // 32 consecutive pixels of row py
            if (lane == 0) S.rmask[2 * py + (px >> 5)] = bits;
            S.pflag[p] = 0;
        }
        __syncthreads();
    }

    // ---- a tile without foreground pixels (most tiles of a sparse field):
    // the map rows are zero, every edge record is -1 and the tile has no
    // pieces, exactly what the labelling below would write for it
    if (!__syncthreads_or(tid < 2 * TY && S.rmask[tid] != 0u)) {
        if (tid == 0) { A.T.piece_base[tile] = 0; A.T.piece_cnt[tile] = 0; }
        if (tw == TX && (W & 3) == 0 && ((((uintptr_t)A.seg) & 15) == 0)) {
            for (int p4 = tid; p4 < TNPIX / 4; p4 += DT_NT) {
                const int py = p4 / (TX / 4), px = (p4 - py * (TX / 4)) * 4;
                if (py < th) *reinterpret_cast<uint4*>(A.seg + (int64_t)(y0 + py) * W + x0 + px) = make_uint4(0u, 0u, 0u, 0u);
            }
        } else {
            for (int p = tid; p < TNPIX; p += DT_NT) {
                const int py = p / TX, px = p - py * TX;
                if (py < th && px < tw) A.seg[(int64_t)(y0 + py) * W + x0 + px] = 0u;
            }
        }
        int16_t* ed = A.T.edges + (int64_t)tile * EDGE_PER_TILE;
        for (int q = tid; q < EDGE_PER_TILE; q += DT_NT) ed[q] = -1;
        return;
    }

    // ---- tile-local labelling on horizontal runs.  Every foreground pixel
    // points at the first pixel of its run (the run's minimum index); only
    // run heads take part in the union-find.  A run is united with each run
    // of the row above that it touches (8-connectivity) at one site per
    // contact: the first column of each vertical overlap (V), and a pixel
    // whose only contact is diagonal (NW: the upper run ends at x - 1; NE:
    // it starts at x + 1).  Each overlap of a lower run R and an upper run Q
    // is one maximal interval of D & U, so V covers every overlapping pair;
    // a diagonal pair without overlap has U[x] = 0 and D[x -/+ 1] = 0 at its
    // contact, so NW / NE cover the rest.
    for (int p = tid; p < TNPIX; p += DT_NT) {
        const int py = p / TX, px = p - py * TX;
        const uint64_t M = row_mask(S, py);
        int v = -1;
        if ((M >> px) & 1ull) {
            const uint64_t z = ~M & ((1ull << px) - 1ull);        // background pixels left of px
            v = py * TX + (z ? 64 - __clzll((long long)z) : 0);
        }
        S.lab[p] = v;
    }
    __syncthreads();
    {
        const int y = tid >> 3;                 // this row against the row above
        const int xs = (tid & 7) * 8;           // 8 of its 64 columns
        if (y > 0 && y < th) {
            const uint64_t D = row_mask(S, y), U = row_mask(S, y - 1);
            const uint64_t O = D & U;
            const uint64_t V = O & ~(O << 1);
            const uint64_t NW = D & ~U & (U << 1) & ~(D << 1);
            const uint64_t NE = D & ~U & (U >> 1) & ~(D >> 1);
            uint32_t sites = (uint32_t)(((V | NW | NE) >> xs) & 0xffu);
            while (sites) {
                const int x = xs + __ffs(sites) - 1;
                sites &= sites - 1;
                const int p = y * TX + x;
                if ((V >> x) & 1ull) sunite(S.lab, p, p - TX);
                if ((NW >> x) & 1ull) sunite(S.lab, p, p - TX - 1);
                if ((NE >> x) & 1ull) sunite(S.lab, p, p - TX + 1);
            }
        }
    }
    __syncthreads();
    // roots of the run heads (thread: 8 columns of one row; heads from the
    // row mask), then every pixel through its run head
    {
        const int y = tid >> 3, xs = (tid & 7) * 8;
        const uint64_t M = row_mask(S, y);
        uint32_t heads = (uint32_t)(((M & ~(M << 1)) >> xs) & 0xffu);
        while (heads) {
            const int p = y * TX + xs + __ffs(heads) - 1;
            heads &= heads - 1;
            S.lab[p] = sfind(S.lab, p);
        }
    }
    __syncthreads();
    {
        // foreground pixels only (thread: 8 columns of one row); run heads
        // hold their roots, which this pass does not change
        const int py = tid >> 3, xs = (tid & 7) * 8;
        uint32_t fgb = (uint32_t)((row_mask(S, py) >> xs) & 0xffu);
        while (fgb) {
            const int p = py * TX + xs + __ffs(fgb) - 1;
            fgb &= fgb - 1;
            S.lab[p] = S.lab[S.lab[p]];
        }
    }
    __syncthreads();

    // ---- compact root numbering in raster (= label) order
    {
        const int p0 = tid * ROWS_PER_THREAD;
        const int4* l4 = reinterpret_cast<const int4*>(S.lab + p0);
        const int4 a = l4[0], b = l4[1];
        const int lv[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
        int cnt = 0;
#pragma unroll
        for (int e = 0; e < 8; ++e) cnt += (lv[e] == p0 + e);
        int off = block_excl_scan(cnt, S.warp_tot, &S.nroots);
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            if (lv[e] == p0 + e) {
                S.u.rid[p0 + e] = (short)off;
                S.r_pix[off] = p0 + e;
                ++off;
            }
        }
    }
    __syncthreads();
    const int nroots = S.nroots;
    for (int r = tid; r < nroots; r += DT_NT) {
        S.r_npix[r] = 0; S.r_xmin[r] = TX; S.r_xmax[r] = -1; S.r_ymin[r] = TY; S.r_ymax[r] = -1; S.r_pidx[r] = 0;
    }
    __syncthreads();
    // per-root size, bounding box and tile-border contact, one update per run
    // (thread: the run heads among 8 columns of one row)
    {
        const int py = tid >> 3, xs = (tid & 7) * 8;
        const uint64_t M = row_mask(S, py);
        uint32_t heads = (uint32_t)(((M & ~(M << 1)) >> xs) & 0xffu);
        while (heads) {
            const int px = xs + __ffs(heads) - 1;
            heads &= heads - 1;
            const uint64_t rest = ~(M >> px);                    // first background column at or after px
            const int xe = rest ? px + __ffsll((long long)rest) - 2 : 63;
            const int r = S.u.rid[S.lab[py * TX + px]];
            const bool border = (px == 0 && x0 > 0) || (xe == tw - 1 && x0 + tw < W) ||
                                (py == 0 && y0 > 0) || (py == th - 1 && y0 + th < H);
            atomicAdd(S.r_npix + r, xe - px + 1);
            atomicMin(S.r_xmin + r, px); atomicMax(S.r_xmax + r, xe);
            atomicMin(S.r_ymin + r, py); atomicMax(S.r_ymax + r, py);
            if (border) S.r_pidx[r] = 1;
        }
    }
    __syncthreads();

    // ---- decide: pieces (touch a shared tile edge), final segments, dropped
    int isp[2], isc[2];
    int pc = 0, cc = 0;
    for (int e = 0; e < 2; ++e) {
        const int r = tid * 2 + e;
        isp[e] = (r < nroots) && S.r_pidx[r];
        isc[e] = (r < nroots) && !S.r_pidx[r] && S.r_npix[r] >= A.minarea;
        pc += isp[e]; cc += isc[e];
    }
    // one scan of both counts (each at most MAXROOT < 2^16)
    const int both = block_excl_scan(pc | (cc << 16), S.warp_tot, &S.npieces);
    int poff = both & 0xffff, coff = both >> 16;
    if (tid == 0) {
        S.ncomps = S.npieces >> 16;
        S.npieces &= 0xffff;
        S.pbase = S.npieces ? atomicAdd(A.P.count, S.npieces) : 0;
        S.cbase = S.ncomps ? atomicAdd(A.C.count, S.ncomps) : 0;
        A.T.piece_base[tile] = S.pbase;
        A.T.piece_cnt[tile] = S.npieces;
    }
    __syncthreads();
    const int pbase = S.pbase, cbase = S.cbase;
    for (int e = 0; e < 2; ++e) {
        const int r = tid * 2 + e;
        if (r >= nroots) continue;
        const int p = S.r_pix[r];
        const int py = p / TX, px = p - py * TX;
        const uint32_t L = (uint32_t)(y0 + py) * (uint32_t)W + (uint32_t)(x0 + px);
        const int4 bb = make_int4(x0 + S.r_xmin[r], x0 + S.r_xmax[r], y0 + S.r_ymin[r], y0 + S.r_ymax[r]);
        const int npix = S.r_npix[r];
        int val = 0, pidx = -1, rec = -1;
        if (isp[e]) {
            const int id = pbase + poff;
            if (id < A.P.cap) {
                A.P.root[id] = L; A.P.npix[id] = npix; A.P.bbox[id] = bb; A.P.parent[id] = id;
                A.P.agg_min[id] = L; A.P.agg_npix[id] = npix; A.P.agg_bbox[id] = bb;
                pidx = poff;
                rec = id;
            } else {
                set_status(A.status, GP_ERR_INTERNAL);
            }
            val = (int)(L + 1u);
            ++poff;
        } else if (isc[e]) {
            const int id = cbase + coff;
            if (id < A.C.cap) {
                A.C.label[id] = L + 1u; A.C.npix[id] = npix; A.C.bbox[id] = bb;
                rec = -2 - id;
            } else {
                set_status(A.status, GP_ERR_INTERNAL);
            }
            val = (int)(L + 1u);
            ++coff;
        }
        S.r_val[r] = val;
        S.r_pidx[r] = pidx;
        S.r_rec[r] = rec;
    }
    __syncthreads();

    // ---- moments of each kept component from the staged m (warp per root)
    if (!LABEL_ONLY) {
        for (int r = warp; r < nroots; r += DT_NT / 32) {
            const int rec = S.r_rec[r];
            if (rec == -1) continue;
            const int rp = S.r_pix[r];
            const int bx0 = S.r_xmin[r], by0 = S.r_ymin[r];
            const int bw = S.r_xmax[r] - bx0 + 1, bh = S.r_ymax[r] - by0 + 1;
            MomAcc a;
            mom_zero(a);
            for (int q = lane; q < bw * bh; q += 32) {
                const int py = by0 + q / bw, px = bx0 + q % bw;
                const int p = py * TX + px;
                if (S.lab[p] != rp) continue;
                const float m = S.m[(py + hh) * SW + px + XHALO];
                const uint32_t L = (uint32_t)(y0 + py) * (uint32_t)W + (uint32_t)(x0 + px);
                mom_pixel(a, m, px, py, L, (S.pflag[p] & 2) != 0);
            }
            mom_warp_reduce(a);
            if (lane == 0) {
                if (rec >= 0) {
                    Moments mo;
                    mo.s = df2(a.s); mo.sx = df2(a.sx); mo.sy = df2(a.sy);
                    mo.sxx = df2(a.sxx); mo.syy = df2(a.syy); mo.sxy = df2(a.sxy);
                    mo.ux = a.ux; mo.uy = a.uy; mo.uxx = a.uxx; mo.uyy = a.uyy; mo.uxy = a.uxy;
                    mo.peak = a.peak; mo.peakL = a.peakL; mo.flags = a.flags;
                    A.P.mom[rec] = mo;
                } else {
                    const int id = -2 - rec;
                    uint32_t fl = a.flags;
                    if (df_positive(a.s)) {
                        // sums about the tile corner (x0, y0), finished by k_mom_finish
                        comp_store_raw(A.C, id, a.s, a.sx, a.sy, a.sxx, a.syy, a.sxy);
                    } else {
                        double flux;
                        double2 xy;
                        Mom2 m2;
                        mom_finish(df_value(a.s), df_value(a.sx), df_value(a.sy), df_value(a.sxx),
                                   df_value(a.syy), df_value(a.sxy), a.ux, a.uy, a.uxx, a.uyy, a.uxy, S.r_npix[r],
                                   x0, y0, &flux, &xy, &m2, &fl);
                        A.C.flux[id] = flux; A.C.xy[id] = xy; A.C.mom2[id] = m2;
                    }
                    A.C.peak[id] = a.peak; A.C.peakL[id] = a.peakL; A.C.flags[id] = fl;
                }
            }
        }
    }

    // ---- segmentation map for the tile (coalesced rows; 16-byte stores when
    // the tile is full width and rows start on 16-byte boundaries)
    if (tw == TX && (W & 3) == 0 && ((((uintptr_t)A.seg) & 15) == 0)) {
        for (int p4 = tid; p4 < TNPIX / 4; p4 += DT_NT) {
            const int py = p4 / (TX / 4), px = (p4 - py * (TX / 4)) * 4;
            if (py >= th) continue;
            const int4 l = *reinterpret_cast<const int4*>(S.lab + py * TX + px);
            uint4 v;
            v.x = l.x >= 0 ? (uint32_t)S.r_val[S.u.rid[l.x]] : 0u;
            v.y = l.y >= 0 ? (uint32_t)S.r_val[S.u.rid[l.y]] : 0u;
            v.z = l.z >= 0 ? (uint32_t)S.r_val[S.u.rid[l.z]] : 0u;
            v.w = l.w >= 0 ? (uint32_t)S.r_val[S.u.rid[l.w]] : 0u;
            *reinterpret_cast<uint4*>(A.seg + (int64_t)(y0 + py) * W + x0 + px) = v;
        }
    } else {
        for (int p = tid; p < TNPIX; p += DT_NT) {
            const int py = p / TX, px = p - py * TX;
            if (py >= th || px >= tw) continue;
            const int l = S.lab[p];
            const uint32_t v = l >= 0 ? (uint32_t)S.r_val[S.u.rid[l]] : 0u;
            A.seg[(int64_t)(y0 + py) * W + x0 + px] = v;
        }
    }
    // ---- edge records: local piece index of each edge pixel, or -1
    int16_t* ed = A.T.edges + (int64_t)tile * EDGE_PER_TILE;
    for (int q = tid; q < EDGE_PER_TILE; q += DT_NT) {
        int px, py;
        bool ok;
        if (q < TY) { py = q; px = 0; ok = py < th; }                                   // colL
        else if (q < 2 * TY) { py = q - TY; px = tw - 1; ok = py < th; }               // colR
        else if (q < 2 * TY + TX) { px = q - 2 * TY; py = 0; ok = px < tw; }           // rowT
        else { px = q - 2 * TY - TX; py = th - 1; ok = px < tw; }                      // rowB
        int16_t v = -1;
        if (ok) {
            const int l = S.lab[py * TX + px];
            if (l >= 0) v = (int16_t)S.r_pidx[S.u.rid[l]];
        }
        ed[q] = v;
    }
}

// ------------------------------------------------------------ tile merge ---
__global__ void k_merge(const ResolveArgs* __restrict__ batch, const __grid_constant__ ResolveArgs one)
{
    const ResolveArgs& R = frame_args(batch, one);
    const Tiles& T = R.T;
    const Pieces& P = R.P;
    const int W = R.W, H = R.H;
    int* status = R.status;
    const int tile = blockIdx.x;
    const int ntx = T.ntx, nty = T.nty;
    if (tile >= ntx * nty) return;
    const int tx = tile % ntx, ty = tile / ntx;
    const int tw = min(TX, W - tx * TX), th = min(TY, H - ty * TY);
    if (threadIdx.x == 0 && tx + 1 < ntx && ty + 1 < nty) {
        // anti-diagonal across this tile's bottom-right corner: bottom-left
        // pixel of the right tile and top-right pixel of the tile below
        // (independent of whether this tile has pieces)
        const int rt = tile + 1, dn = tile + ntx;
        if (T.piece_cnt[rt] > 0 && T.piece_cnt[dn] > 0) {
            const int a = T.edges[(int64_t)rt * EDGE_PER_TILE + th - 1];
            const int b = T.edges[(int64_t)dn * EDGE_PER_TILE + TY + 0];
            if (a >= 0 && b >= 0) gunite(P.parent, T.piece_base[rt] + a, T.piece_base[dn] + b, status);
        }
    }
    if (T.piece_cnt[tile] == 0) return;
    const int base = T.piece_base[tile];
    const int16_t* e = T.edges + (int64_t)tile * EDGE_PER_TILE;
    if (tx + 1 < ntx && T.piece_cnt[tile + 1] > 0) {
        const int nbase = T.piece_base[tile + 1];
        const int16_t* en = T.edges + (int64_t)(tile + 1) * EDGE_PER_TILE;
        for (int i = threadIdx.x; i < th; i += blockDim.x) {
            const int a = e[TY + i];
            if (a < 0) continue;
            for (int d = -1; d <= 1; ++d) {
                const int k = i + d;
                if (k < 0 || k >= th) continue;
                const int b = en[k];
                if (b >= 0) gunite(P.parent, base + a, nbase + b, status);
            }
        }
    }
    if (ty + 1 < nty && T.piece_cnt[tile + ntx] > 0) {
        const int nbase = T.piece_base[tile + ntx];
        const int16_t* en = T.edges + (int64_t)(tile + ntx) * EDGE_PER_TILE;
        for (int j = threadIdx.x; j < tw; j += blockDim.x) {
            const int a = e[2 * TY + TX + j];
            if (a < 0) continue;
            for (int d = -1; d <= 1; ++d) {
                const int k = j + d;
                if (k < 0 || k >= tw) continue;
                const int b = en[2 * TY + k];
                if (b >= 0) gunite(P.parent, base + a, nbase + b, status);
            }
        }
    }
    if (threadIdx.x == 0 && tx + 1 < ntx && ty + 1 < nty) {
        // bottom-right pixel of this tile and top-left pixel of the diagonal tile
        const int dr = tile + ntx + 1;
        const int a = e[TY + th - 1];
        const int b = T.edges[(int64_t)dr * EDGE_PER_TILE + 0];
        if (a >= 0 && b >= 0) gunite(P.parent, base + a, T.piece_base[dr] + b, status);
    }
}

// --------------------------------------------------------- piece resolve ---
__global__ void k_aggregate(const ResolveArgs* __restrict__ batch, const __grid_constant__ ResolveArgs one)
{
    const ResolveArgs& R = frame_args(batch, one);
    const Pieces& P = R.P;
    int* status = R.status;
    const int n = min(*P.count, P.cap);
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const int r = gfind(P.parent, p);
        P.proot[p] = r;
        if (r < 0) { set_status(status, GP_ERR_TIMEOUT); continue; }
        if (r == p) continue;
        atomicMin(P.agg_min + r, P.root[p]);
        atomicAdd(P.agg_npix + r, P.npix[p]);
        const int4 b = P.bbox[p];
        int* ab = reinterpret_cast<int*>(P.agg_bbox + r);
        atomicMin(ab + 0, b.x); atomicMax(ab + 1, b.y);
        atomicMin(ab + 2, b.z); atomicMax(ab + 3, b.w);
    }
}

// add a (hi, lo) pair times a small integer
__device__ __forceinline__ void df_add_scaled(DF& s, float2 v, float k)
{
    df_add_prod(s, k, v.x);
    s.lo = fmaf(k, v.y, s.lo);
}

__device__ __forceinline__ void df_add_pair(DF& s, float2 v)
{
    df_add(s, v.x);
    s.lo += v.y;
}

// One warp per piece.  At root pieces of kept segments: merge the partial
// moments of all the segment's pieces, visiting the tiles of the segment's
// bounding box in raster order (a fixed order, so the sums are
// reproducible) and emit the segment; a segment of a single piece is emitted
// from that piece's sums directly (the merge would add zeros to them).  Every piece whose final label differs
// from its provisional one rewrites its pixels in the map.
__global__ void k_finalize(const ResolveArgs* __restrict__ batch, const __grid_constant__ ResolveArgs one)
{
    const ResolveArgs& R = frame_args(batch, one);
    const Tiles& T = R.T;
    const Pieces& P = R.P;
    const Comps& C = R.C;
    uint32_t* seg = R.seg;
    const int W = R.W, minarea = R.minarea;
    int* status = R.status;
    const int n = min(*P.count, P.cap);
    const int lane = threadIdx.x & 31;
    const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int p = wid; p < n; p += nw) {
        const int r = P.proot[p];
        if (r < 0) continue;
        const int tot = P.agg_npix[r];
        const uint32_t fin = tot >= minarea ? P.agg_min[r] + 1u : 0u;
        if (r == p && fin && tot == P.npix[p]) {
            // a segment of this one piece: its sums, taken about the corner of
            // its one tile (the segment's origin), are already final
            if (lane == 0) {
                const Moments mo = P.mom[p];
                const int id = atomicAdd(C.count, 1);
                if (id < C.cap) {
                    DF s, sx, sy, sxx, syy, sxy;
                    s.hi = mo.s.x; s.lo = mo.s.y; sx.hi = mo.sx.x; sx.lo = mo.sx.y; sy.hi = mo.sy.x; sy.lo = mo.sy.y;
                    sxx.hi = mo.sxx.x; sxx.lo = mo.sxx.y; syy.hi = mo.syy.x; syy.lo = mo.syy.y;
                    sxy.hi = mo.sxy.x; sxy.lo = mo.sxy.y;
                    const int4 bb = P.agg_bbox[r];
                    uint32_t fl = mo.flags;
                    if (df_positive(s)) {
                        comp_store_raw(C, id, s, sx, sy, sxx, syy, sxy);     // finished by k_mom_finish
                    } else {
                        const int2 org = comp_origin(bb);
                        double flux;
                        double2 xy;
                        Mom2 m2;
                        mom_finish(df_value(s), df_value(sx), df_value(sy), df_value(sxx), df_value(syy),
                                   df_value(sxy), mo.ux, mo.uy, mo.uxx, mo.uyy, mo.uxy, tot, org.x, org.y, &flux,
                                   &xy, &m2, &fl);
                        C.flux[id] = flux; C.xy[id] = xy; C.mom2[id] = m2;
                    }
                    C.label[id] = fin; C.npix[id] = tot; C.bbox[id] = bb;
                    C.peak[id] = mo.peak; C.peakL[id] = mo.peakL; C.flags[id] = fl;
                } else {
                    set_status(status, GP_ERR_INTERNAL);
                }
            }
        } else if (r == p && fin) {
            const int4 bb = P.agg_bbox[r];
            const int2 org = comp_origin(bb);
            const int X0 = org.x, Y0 = org.y;
            const int tx0 = bb.x / TX, tx1 = bb.y / TX, ty0 = bb.z / TY, ty1 = bb.w / TY;
            const int ntw = tx1 - tx0 + 1, nt = ntw * (ty1 - ty0 + 1);
            DF s = df_zero(), sx = df_zero(), sy = df_zero(), sxx = df_zero(), syy = df_zero(), sxy = df_zero();
            long long ux = 0, uy = 0, uxx = 0, uyy = 0, uxy = 0;
            float pk = -INFINITY;
            uint32_t pkL = 0xffffffffu, fl = 0u;
            for (int k = lane; k < nt; k += 32) {
                const int t = (ty0 + k / ntw) * T.ntx + tx0 + k % ntw;
                const int b0 = T.piece_base[t], cnt = T.piece_cnt[t];
                for (int q = b0; q < b0 + cnt && q < n; ++q) {
                    if (P.proot[q] != r) continue;
                    const Moments mo = P.mom[q];
                    const uint32_t L = P.root[q];
                    const int ox = (int)(L % (uint32_t)W) / TX * TX - X0;
                    const int oy = (int)(L / (uint32_t)W) / TY * TY - Y0;
                    const float fx = (float)ox, fy = (float)oy;
                    // shift the sums from the piece's tile corner to (X0, Y0)
                    df_add_pair(s, mo.s);
                    df_add_pair(sx, mo.sx); df_add_scaled(sx, mo.s, fx);
                    df_add_pair(sy, mo.sy); df_add_scaled(sy, mo.s, fy);
                    df_add_pair(sxx, mo.sxx); df_add_scaled(sxx, mo.sx, 2.f * fx); df_add_scaled(sxx, mo.s, fx * fx);
                    df_add_pair(syy, mo.syy); df_add_scaled(syy, mo.sy, 2.f * fy); df_add_scaled(syy, mo.s, fy * fy);
                    df_add_pair(sxy, mo.sxy); df_add_scaled(sxy, mo.sy, fx); df_add_scaled(sxy, mo.sx, fy);
                    df_add_scaled(sxy, mo.s, fx * fy);
                    const long long np = P.npix[q];
                    ux += mo.ux + (long long)ox * np;
                    uy += mo.uy + (long long)oy * np;
                    uxx += mo.uxx + 2ll * ox * mo.ux + (long long)ox * ox * np;
                    uyy += mo.uyy + 2ll * oy * mo.uy + (long long)oy * oy * np;
                    uxy += mo.uxy + (long long)ox * mo.uy + (long long)oy * mo.ux + (long long)ox * oy * np;
                    if (mo.peak > pk || (mo.peak == pk && mo.peakL < pkL)) { pk = mo.peak; pkL = mo.peakL; }
                    fl |= mo.flags;
                }
            }
            s = df_warp_sum(s); sx = df_warp_sum(sx); sy = df_warp_sum(sy);
            sxx = df_warp_sum(sxx); syy = df_warp_sum(syy); sxy = df_warp_sum(sxy);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                ux += __shfl_xor_sync(0xffffffffu, ux, o);
                uy += __shfl_xor_sync(0xffffffffu, uy, o);
                uxx += __shfl_xor_sync(0xffffffffu, uxx, o);
                uyy += __shfl_xor_sync(0xffffffffu, uyy, o);
                uxy += __shfl_xor_sync(0xffffffffu, uxy, o);
                fl |= __shfl_xor_sync(0xffffffffu, fl, o);
                const float op = __shfl_xor_sync(0xffffffffu, pk, o);
                const uint32_t oL = __shfl_xor_sync(0xffffffffu, pkL, o);
                if (op > pk || (op == pk && oL < pkL)) { pk = op; pkL = oL; }
            }
            if (lane == 0) {
                const int id = atomicAdd(C.count, 1);
                if (id < C.cap) {
                    if (df_positive(s)) {
                        comp_store_raw(C, id, s, sx, sy, sxx, syy, sxy);     // finished by k_mom_finish
                    } else {
                        double flux;
                        double2 xy;
                        Mom2 m2;
                        mom_finish(df_value(s), df_value(sx), df_value(sy), df_value(sxx), df_value(syy),
                                   df_value(sxy), ux, uy, uxx, uyy, uxy, tot, X0, Y0, &flux, &xy, &m2, &fl);
                        C.flux[id] = flux; C.xy[id] = xy; C.mom2[id] = m2;
                    }
                    C.label[id] = fin; C.npix[id] = tot; C.bbox[id] = bb;
                    C.peak[id] = pk; C.peakL[id] = pkL; C.flags[id] = fl;
                } else {
                    set_status(status, GP_ERR_INTERNAL);
                }
            }
        }
        const uint32_t prov = P.root[p] + 1u;
        if (fin == prov) continue;
        const int4 b = P.bbox[p];
        const int bw = b.y - b.x + 1, bh = b.w - b.z + 1;
        for (int q = lane; q < bw * bh; q += 32) {
            const int y = b.z + q / bw, x = b.x + q % bw;
            uint32_t* sp = seg + (int64_t)y * W + x;
            if (*sp == prov) *sp = fin;
        }
    }
}

// Centroid and second moments of every segment stored with raw sums (one
// thread per segment); segments with a sum <= 0 were finished where they were
// found and carry GP_FLAG_CENTROID_FALLBACK.
__global__ void k_mom_finish(const ResolveArgs* __restrict__ batch, const __grid_constant__ ResolveArgs one)
{
    const ResolveArgs& R = frame_args(batch, one);
    const Comps& C = R.C;
    const int n = min(*C.count, C.cap);
    for (int id = blockIdx.x * blockDim.x + threadIdx.x; id < n; id += gridDim.x * blockDim.x) {
        uint32_t fl = C.flags[id];
        if (fl & GP_FLAG_CENTROID_FALLBACK) continue;
        const float2 s = reinterpret_cast<const float2*>(C.flux)[id];
        const float4 sxy = reinterpret_cast<const float4*>(C.xy)[id];
        const float4* mr = reinterpret_cast<const float4*>(C.mom2 + id);
        const float4 m0 = mr[0], m1 = mr[1];
        const int2 org = comp_origin(C.bbox[id]);
        double flux;
        double2 xy;
        Mom2 m2;
        mom_finish((double)s.x + (double)s.y, (double)sxy.x + (double)sxy.y, (double)sxy.z + (double)sxy.w,
                   (double)m0.x + (double)m0.y, (double)m0.z + (double)m0.w, (double)m1.x + (double)m1.y, 0, 0, 0,
                   0, 0, C.npix[id], org.x, org.y, &flux, &xy, &m2, &fl);
        C.flux[id] = flux; C.xy[id] = xy; C.mom2[id] = m2;
    }
}

// ------------------------------------------------------------------ rank ---
__global__ void k_rank_count(const RankArgs* __restrict__ batch, const __grid_constant__ RankArgs one)
{
    const Comps& C = frame_args(batch, one).C;
    const int n = min(*C.count, C.cap);
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x)
        atomicAdd(C.bcnt + ((C.label[c] - 1u) >> C.shift), 1);
}

constexpr int SCAN_NT = 1024;

// exclusive scan of the bucket counts in one pass of one CTA: each thread
// sums a run of consecutive buckets (16-byte loads), the block scans the run
// sums, and each thread writes its run's offsets from a second (cached) read;
// publishes the segment count
__global__ void __launch_bounds__(SCAN_NT) k_rank_scan(const RankArgs* __restrict__ batch,
                                                       const __grid_constant__ RankArgs one)
{
    const RankArgs& R = frame_args(batch, one);
    const Comps& C = R.C;
    int* n_out = R.n_out;
    const int capacity = R.capacity;
    int* status = R.status;
    __shared__ int wsum[SCAN_NT / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nb = C.nb;                                     // <= 65,536
    const int per = ((nb + SCAN_NT - 1) / SCAN_NT + 3) & ~3; // a multiple of 4 buckets per thread
    const int b0 = min(tid * per, nb), b1 = min(b0 + per, nb);
    const bool vec = (((uintptr_t)C.bcnt | (uintptr_t)C.boff) & 15) == 0;
    int tsum = 0;
    int i = b0;
    if (vec) {
#pragma unroll 4
        for (; i + 4 <= b1; i += 4) {
            const int4 q = *reinterpret_cast<const int4*>(C.bcnt + i);
            tsum += q.x + q.y + q.z + q.w;
        }
    }
    for (; i < b1; ++i) tsum += C.bcnt[i];
    int incl = tsum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const int w = wsum[lane];
        int wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += t;
        }
        wsum[lane] = wi - w;
    }
    __syncthreads();
    int excl = wsum[warp] + incl - tsum;
    i = b0;
    if (vec) {
#pragma unroll 4
        for (; i + 4 <= b1; i += 4) {
            const int4 q = *reinterpret_cast<const int4*>(C.bcnt + i);
            int4 o;
            o.x = excl; excl += q.x;
            o.y = excl; excl += q.y;
            o.z = excl; excl += q.z;
            o.w = excl; excl += q.w;
            *reinterpret_cast<int4*>(C.boff + i) = o;
        }
    }
    for (; i < b1; ++i) {
        const int v = C.bcnt[i];
        C.boff[i] = excl;
        excl += v;
    }
    if (tid == 0) {
        const int total = *C.count;
        if (total > C.cap) set_status(status, GP_ERR_INTERNAL);
        if (n_out) *n_out = total;
        if (capacity >= 0 && total > capacity) set_status(status, GP_ERR_CAPACITY);
    }
}

__global__ void k_rank_scatter(const RankArgs* __restrict__ batch, const __grid_constant__ RankArgs one)
{
    const Comps& C = frame_args(batch, one).C;
    const int n = min(*C.count, C.cap);
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        const int b = (int)((C.label[c] - 1u) >> C.shift);
        const int s = C.boff[b] + atomicAdd(C.bcur + b, 1);
        C.slots[s] = c;
    }
}

__global__ void k_rank_place(const RankArgs* __restrict__ batch, const __grid_constant__ RankArgs one)
{
    const Comps& C = frame_args(batch, one).C;
    const int n = min(*C.count, C.cap);
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        const uint32_t l = C.label[c];
        const int b = (int)((l - 1u) >> C.shift);
        const int s0 = C.boff[b], s1 = s0 + C.bcnt[b];
        int r = s0;
        for (int s = s0; s < s1; ++s) r += (C.label[C.slots[s]] < l);
        C.perm[r] = c;
    }
}

// --------------------------------------------------------------- launchers ---
template <bool F32, bool LO, int KS>
static cudaError_t launch_tile(const DetectArgs& one, const DetectArgs* batch, int nframes, int maxtiles,
                               cudaStream_t st)
{
    const size_t smem = sizeof(TileSmem);
    if (batch) {
        cudaFuncSetAttribute(k_detect_tile<F32, LO, KS, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_detect_tile<F32, LO, KS, true><<<dim3(maxtiles, nframes), DT_NT, smem, st>>>(batch, one);
    } else {
        cudaFuncSetAttribute(k_detect_tile<F32, LO, KS, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
        k_detect_tile<F32, LO, KS, false><<<maxtiles, DT_NT, smem, st>>>(nullptr, one);
    }
    return cudaGetLastError();
}

template <bool F32>
static cudaError_t launch_tile_ks(const DetectArgs& one, const DetectArgs* batch, int nframes, int maxtiles,
                                  cudaStream_t st)
{
    if (one.kw == one.kh && one.kw == 3) return launch_tile<F32, false, 3>(one, batch, nframes, maxtiles, st);
    if (one.kw == one.kh && one.kw == 5) return launch_tile<F32, false, 5>(one, batch, nframes, maxtiles, st);
    if (one.kw == one.kh && one.kw == 7) return launch_tile<F32, false, 7>(one, batch, nframes, maxtiles, st);
    return launch_tile<F32, false, 0>(one, batch, nframes, maxtiles, st);
}

DetectArgs detect_args(const Image& im, const SplineTab& sb, const SplineTab& sr, const float* taps, int kw, int kh,
                       float thresh, int minarea, uint32_t* seg, uint8_t* mask_out, int* nnear,
                       const uint8_t* in_mask, const Tiles& T, const Pieces& P, const Comps& C, int* status)
{
    DetectArgs A;
    for (int i = 0; i < KMAX; ++i) A.K[i] = (taps && i < kw * kh) ? taps[i] : 0.f;
    A.im = im; A.sb = sb; A.sr = sr;
    A.kw = kw; A.kh = kh; A.hx = kw / 2; A.hy = kh / 2; A.hh = max(kw / 2, kh / 2);
    A.thresh = thresh; A.minarea = minarea;
    A.seg = seg; A.mask_out = mask_out; A.nnear = nnear; A.in_mask = in_mask;
    A.T = T; A.P = P; A.C = C; A.status = status;
    return A;
}

// every frame of a batch shares `one`'s dtype, kernel size and mode
// (labelling a given mask or detecting); maxtiles = the largest frame's tiles
cudaError_t launch_detect_any(const DetectArgs& one, const DetectArgs* batch, int nframes, int maxtiles,
                              cudaStream_t st)
{
    if (one.in_mask) return launch_tile<false, true, 0>(one, batch, nframes, maxtiles, st);
    if (one.im.is_f32) return launch_tile_ks<true>(one, batch, nframes, maxtiles, st);
    return launch_tile_ks<false>(one, batch, nframes, maxtiles, st);
}

cudaError_t launch_detect_tiles(const Image& im, const SplineTab& sb, const SplineTab& sr, const float* taps,
                                int kw, int kh, float thresh, int minarea, uint32_t* seg, uint8_t* mask_out,
                                int* nnear, const uint8_t* in_mask, const Tiles& T, const Pieces& P, const Comps& C,
                                int* status, cudaStream_t st)
{
    const DetectArgs A = detect_args(im, sb, sr, taps, kw, kh, thresh, minarea, seg, mask_out, nnear, in_mask, T, P,
                                     C, status);
    return launch_detect_any(A, nullptr, 1, T.ntx * T.nty, st);
}

ResolveArgs resolve_args(const Tiles& T, const Pieces& P, const Comps& C, uint32_t* seg, int W, int H, int minarea,
                         int* status)
{
    ResolveArgs R;
    R.T = T; R.P = P; R.C = C; R.seg = seg; R.W = W; R.H = H; R.minarea = minarea; R.status = status;
    return R;
}

// grid of the grid-stride kernels: about 152 x 8 CTAs over the whole batch
static int stride_grid(int per_frame, int nframes)
{
    const int g = per_frame / nframes;
    return g < 16 ? 16 : g;
}

cudaError_t launch_resolve_any(const ResolveArgs& one, const ResolveArgs* batch, int nframes, int maxtiles,
                               cudaStream_t st)
{
    k_merge<<<dim3(maxtiles, nframes), 64, 0, st>>>(batch, one);
    const dim3 g(stride_grid(152 * 8, nframes), nframes);
    k_aggregate<<<g, 256, 0, st>>>(batch, one);
    k_finalize<<<g, 256, 0, st>>>(batch, one);
    k_mom_finish<<<g, 256, 0, st>>>(batch, one);
    return cudaGetLastError();
}

cudaError_t launch_resolve(const Tiles& T, const Pieces& P, const Comps& C, uint32_t* seg, int W, int H,
                           int minarea, int* status, cudaStream_t st)
{
    return launch_resolve_any(resolve_args(T, P, C, seg, W, H, minarea, status), nullptr, 1, T.ntx * T.nty, st);
}

RankArgs rank_args(const Comps& C, int* n_out, int capacity, bool place, int* status)
{
    RankArgs R;
    R.C = C; R.n_out = n_out; R.capacity = capacity; R.place = place ? 1 : 0; R.status = status;
    return R;
}

// every frame of a batch shares `one`'s place flag
cudaError_t launch_rank_any(const RankArgs& one, const RankArgs* batch, int nframes, cudaStream_t st)
{
    const dim3 g(stride_grid(152 * 4, nframes), nframes);
    k_rank_count<<<g, 256, 0, st>>>(batch, one);
    k_rank_scan<<<dim3(1, nframes), SCAN_NT, 0, st>>>(batch, one);
    if (one.place) {
        k_rank_scatter<<<g, 256, 0, st>>>(batch, one);
        k_rank_place<<<g, 256, 0, st>>>(batch, one);
    }
    return cudaGetLastError();
}

cudaError_t launch_rank(const Comps& C, int* n_out, int capacity, bool place, int* status, cudaStream_t st)
{
    return launch_rank_any(rank_args(C, n_out, capacity, place, status), nullptr, 1, st);
}

}  // namespace gp
