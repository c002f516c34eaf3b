// k_detect.cu -- segmentation of the thresholded frame (paper Section 3.2,
// with labelled segments in place of the paper's local maxima) and the
// segment moments (its first-moment centroid, extended to second moments,
// bounding box and peak).  The threshold mask comes from k_stream.cu.
//
//  k_label_tiles  one warp per 64 x 32 detection tile that holds foreground
//                 (the list k_stream appends).  Lane y takes tile row y: its
//                 64-bit row mask, its horizontal runs (numbered in raster
//                 order), and the unions of its runs with the touching runs
//                 of the row above (8-connectivity) in a per-warp union-find
//                 in shared memory whose roots are the smallest run ids (the
//                 first run, and so the minimum linear index, of each
//                 component).  Per root: pixel count and tile-edge contact
//                 (one shared atomic per run), then for each kept root, in
//                 raster order, its bounding box (warp min/max) and its
//                 moment sums over its pixels with m = I - B recomputed there
//                 (fixed order: x within a row, then a fixed butterfly over
//                 the rows).  Components that do not touch an edge shared
//                 with another tile are final here (raw sums); the others
//                 become "pieces" with partial sums, and their edge pixels
//                 are recorded for the merge.  The labels of kept
//                 components are written over the zero map.
//  k_merge        unites pieces across tile edges (lock-free union-find
//                 over piece ids, atomicMin linking), one warp per listed
//                 tile with pieces.
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
#include <string.h>

#include <algorithm>

#include "gp_internal.cuh"
#include "gp_launch.h"

namespace gp {

static_assert(TX == 64, "row masks hold one 64-pixel tile row");
static_assert(TY == 32, "a warp's lane is a tile row");

// ------------------------------------------------ shared-memory union-find ---
// over the run ids of one tile; a link always points at a smaller id
// (path halving: a run is re-pointed at its grandparent on the way, which
// stays an ancestor, so concurrent walks and links remain valid)
__device__ __forceinline__ int lfind(volatile int* par, int x)
{
    for (int n = 0; n <= MAXRUN; ++n) {
        const int p = par[x];
        if (p == x) return x;
        const int gp = par[p];
        if (gp != p) par[x] = gp;
        x = gp;
    }
    return x;
}

__device__ __forceinline__ void lunite(int* par, int a, int b)
{
    for (int it = 0; it < 4 * MAXRUN; ++it) {
        a = lfind(par, a);
        b = lfind(par, b);
        if (a == b) return;
        if (a < b) { const int t = a; a = b; b = t; }
        const int old = atomicMin(par + a, b);
        if (old == a) return;
        a = old;
    }
}

// ---------------------------------------------------- global union-find ---
// walks give up after `limit` steps (-1 / GP_ERR_TIMEOUT)
__device__ __forceinline__ int gfind(const int* parent, int x, int limit)
{
    for (int n = 0; n < limit; ++n) {
        const int p = __ldcg(parent + x);
        if (p == x) return x;
        x = p;
    }
    return -1;
}

__device__ void gunite(int* parent, int a, int b, int limit, int* status)
{
    for (int it = 0; it < limit; ++it) {
        a = gfind(parent, a, limit);
        b = gfind(parent, b, limit);
        if (a < 0 || b < 0) break;
        if (a == b) return;
        if (a < b) { const int t = a; a = b; b = t; }
        const int old = atomicMin(parent + a, b);
        if (old == a) return;
        a = old;
    }
    set_status(status, GP_ERR_TIMEOUT);
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

__device__ __forceinline__ float2 df2(DF d) { return make_float2(d.hi, d.lo); }

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

// Moments of one run (row y, columns xs..xe, tile coordinates) from its
// partial sums r0 = sum m, r1 = sum x m, r2 = sum x^2 m: the row coordinate
// enters as exact products of the sums by y and y^2, and the unweighted
// (integer) sums have closed forms.
__device__ __forceinline__ void mom_fold(MomAcc& a, DF r0, DF r1, DF r2, int xs, int xe, int y)
{
    const float fy = (float)y, fy2 = (float)(y * y);
    df_add_pair(a.s, df2(r0));
    df_add_pair(a.sx, df2(r1));
    df_add_pair(a.sxx, df2(r2));
    df_add_scaled(a.sy, df2(r0), fy);
    df_add_scaled(a.syy, df2(r0), fy2);
    df_add_scaled(a.sxy, df2(r1), fy);
    const int n = xe - xs + 1;
    const int sx = n * (xs + xe) / 2;
    const int sxx = (xe * (xe + 1) * (2 * xe + 1) - (xs - 1) * xs * (2 * xs - 1)) / 6;
    a.ux += sx; a.uy += y * n; a.uxx += sxx; a.uyy += y * y * n; a.uxy += y * sx;
}

// one pixel of a run: its partial sums, the peak (first pixel in raster
// order among equal maxima) and the saturation flag
__device__ __forceinline__ void run_pixel(DF& r0, DF& r1, DF& r2, MomAcc& a, float m, int x, uint32_t L, bool sat)
{
    const float fx = (float)x;
    df_add(r0, m);
    df_add_prod(r1, fx, m);
    df_add_prod(r2, fx * fx, m);
    if (m > a.peak || (m == a.peak && L < a.peakL)) { a.peak = m; a.peakL = L; }
    if (sat) a.flags |= GP_FLAG_SAT;
}

// sum of v over lanes base .. base + 2^levels - 1 into lane base (a fixed
// tree: reproducible); lanes outside the range hold zeros
__device__ __forceinline__ DF df_tree_sum(DF v, int levels)
{
    const int lane = threadIdx.x & 31;
    for (int o = levels > 0 ? 1 << (levels - 1) : 0; o > 0; o >>= 1) {
        DF w;
        w.hi = __shfl_down_sync(0xffffffffu, v.hi, o);
        w.lo = __shfl_down_sync(0xffffffffu, v.lo, o);
        if (lane + o < 32) v = df_merge(v, w);
    }
    return v;
}

// float -> unsigned key with the same order (+0 and -0 equal)
__device__ __forceinline__ uint32_t fkey(float f)
{
    const uint32_t b = __float_as_uint(f == 0.f ? 0.f : f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float fkey_inv(uint32_t k)
{
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// a segment's sums over the lanes (tile rows) base .. base + 2^levels - 1,
// complete in lane base
__device__ __forceinline__ void mom_rows_reduce(MomAcc& a, int levels)
{
    const uint32_t FULL = 0xffffffffu;
    a.s = df_tree_sum(a.s, levels); a.sx = df_tree_sum(a.sx, levels); a.sy = df_tree_sum(a.sy, levels);
    a.sxx = df_tree_sum(a.sxx, levels); a.syy = df_tree_sum(a.syy, levels); a.sxy = df_tree_sum(a.sxy, levels);
    a.ux = __reduce_add_sync(FULL, a.ux); a.uy = __reduce_add_sync(FULL, a.uy);
    a.uxx = __reduce_add_sync(FULL, a.uxx); a.uyy = __reduce_add_sync(FULL, a.uyy);
    a.uxy = __reduce_add_sync(FULL, a.uxy);
    a.flags = __reduce_or_sync(FULL, a.flags);
    const uint32_t k = __reduce_max_sync(FULL, fkey(a.peak));
    a.peakL = __reduce_min_sync(FULL, fkey(a.peak) == k ? a.peakL : 0xffffffffu);
    a.peak = fkey_inv(k);
}

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

// ---------------------------------------------------------- tile labelling ---
// Per-warp tables.  The common form holds up to 256 runs and 512 foreground
// pixels per tile; a tile above either is deferred to the big form, where
// every tile fits (1024 runs, 2048 pixels).
template <bool BIG>
struct LabelCfg {
    static constexpr int NW = 2;
    static constexpr int RUNS = BIG ? MAXRUN : 256;
    static constexpr int FG = BIG ? TX * TY : LT_FG;
};

// a kept segment of at most this many pixels is summed by one lane (32 such
// segments at once); larger ones by the whole warp, a lane per tile row
constexpr int LANE_SEG_MAX = 64;

template <bool BIG>
struct LabelSmem {
    static constexpr int R = LabelCfg<BIG>::RUNS, F = LabelCfg<BIG>::FG;
    int par[R];                   // union-find; after flattening, the component's root run
    int cnt[R];                   // at roots: pixels + (runs on a shared tile edge << 16)
    int val[R];                   // at roots: the map value (1 + minimum linear index), 0 when dropped
    int16_t kidx[R];              // at kept roots: the local piece index (>= 0), or -2 - the local
                                  // final-segment index; else -1
    int16_t pos[R];               // the run's row * TX + first column
    int16_t fidx[R];              // compact index of the run's first pixel
    int16_t klist[R];             // kept roots in label order
    int16_t roff[R];              // at kept roots (per-lane path): first entry of its runs in rlist
    int16_t rcnt[R];              // at kept roots (per-lane path): its runs
    int16_t rlist[R];             // runs of the per-lane segments, grouped by segment, in label order
    uint8_t len[R];               // the run's pixels - 1
    float m[F];                   // m at the tile's foreground pixels, in raster order
    uint32_t iv[F];               // the 32-bit word holding each foreground pixel's value (saturation)
};

// bits 0..15 of v to bits 0, 4, ..., 60
__device__ __forceinline__ uint64_t spread4(uint32_t v)
{
    uint64_t x = v & 0xffffu;
    x = (x | (x << 24)) & 0x000000ff000000ffull;
    x = (x | (x << 12)) & 0x000f000f000f000full;
    x = (x | (x << 6)) & 0x0303030303030303ull;
    x = (x | (x << 3)) & 0x1111111111111111ull;
    return x;
}

// bits 0..x set (x in 0..63)
__device__ __forceinline__ uint64_t upto(int x) { return (2ull << x) - 1ull; }

// last column of the run that starts at x in row mask M
__device__ __forceinline__ int run_end(uint64_t M, int x)
{
    const uint64_t rest = ~(M >> x);
    return rest ? x + __ffsll((long long)rest) - 2 : 63;
}

__device__ __forceinline__ void cp_async4(void* dst, const void* src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}

template <bool BATCH>
__device__ __forceinline__ const DetectArgs& det_frame(const DetectArgs* __restrict__ batch, const DetectArgs& one)
{
    if constexpr (BATCH) return batch[blockIdx.y];
    else return one;
}

// write the records of kept root r (lane-parallel or lane 0 of the warp path)
template <bool LABEL_ONLY, bool BIG>
__device__ __forceinline__ void emit_root(const DetectArgs& A, const LabelSmem<BIG>& S, int r, int4 bb, int pbase,
                                          int cbase, int x0, int y0, const MomAcc& a)
{
    const uint32_t L = (uint32_t)S.val[r] - 1u;
    const int npix = S.cnt[r] & 0xffff;
    if (S.kidx[r] >= 0) {
        const int id = pbase + S.kidx[r];
        if (id < A.P.cap) {
            A.P.root[id] = L; A.P.npix[id] = npix; A.P.bbox[id] = bb; A.P.parent[id] = id;
            A.P.agg_min[id] = L; A.P.agg_npix[id] = npix; A.P.agg_bbox[id] = bb;
            if (!LABEL_ONLY) {
                Moments mo;
                mo.s = df2(a.s); mo.sx = df2(a.sx); mo.sy = df2(a.sy);
                mo.sxx = df2(a.sxx); mo.syy = df2(a.syy); mo.sxy = df2(a.sxy);
                mo.ux = a.ux; mo.uy = a.uy; mo.uxx = a.uxx; mo.uyy = a.uyy; mo.uxy = a.uxy;
                mo.peak = a.peak; mo.peakL = a.peakL; mo.flags = a.flags;
                A.P.mom[id] = mo;
            }
        } else {
            set_status(A.status, GP_ERR_INTERNAL);
        }
        return;
    }
    const int id = cbase + (-2 - S.kidx[r]);
    if (id >= A.C.cap) {
        set_status(A.status, GP_ERR_INTERNAL);
        return;
    }
    A.C.label[id] = L + 1u; A.C.npix[id] = npix; A.C.bbox[id] = bb;
    if (LABEL_ONLY) return;
    uint32_t fl = a.flags;
    if (df_positive(a.s)) {
        // sums about the tile corner (x0, y0), finished by k_mom_finish
        comp_store_raw(A.C, id, a.s, a.sx, a.sy, a.sxx, a.syy, a.sxy);
    } else {
        double flux;
        double2 xy;
        Mom2 m2;
        mom_finish(df_value(a.s), df_value(a.sx), df_value(a.sy), df_value(a.sxx), df_value(a.syy), df_value(a.sxy),
                   a.ux, a.uy, a.uxx, a.uyy, a.uxy, npix, x0, y0, &flux, &xy, &m2, &fl);
        A.C.flux[id] = flux; A.C.xy[id] = xy; A.C.mom2[id] = m2;
    }
    A.C.peak[id] = a.peak; A.C.peakL[id] = a.peakL; A.C.flags[id] = fl;
}

// saturation of a foreground pixel at linear offset `lin` (elements from the
// image base): from the 32-bit word copied for it (`async`), else read here
__device__ __forceinline__ bool pix_sat(const DetectArgs& A, bool async, uint32_t word, int64_t lin)
{
    float v;
    if (A.im.is_f32) v = async ? __uint_as_float(word) : __ldg(reinterpret_cast<const float*>(A.im.data) + lin);
    else if (async) v = (float)((lin & 1) ? (word >> 16) : (word & 0xffffu));
    else v = (float)__ldg(reinterpret_cast<const uint16_t*>(A.im.data) + lin);
    return v >= A.im.sat;
}

template <bool LABEL_ONLY, bool BATCH, bool BIG>
__global__ void __launch_bounds__(32 * LabelCfg<BIG>::NW, BIG ? 4 : 11) k_label_tiles(const DetectArgs* __restrict__ batch,
                                                                        const __grid_constant__ DetectArgs one,
                                                                        int late)
{
    pdl_wait();
    pdl_release();
    using Cfg = LabelCfg<BIG>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    LabelSmem<BIG>& S = reinterpret_cast<LabelSmem<BIG>*>(smem_raw)[warp];
    const DetectArgs& A = det_frame<BATCH>(batch, one);
    const int W = A.im.W, H = A.im.H, ntx = A.T.ntx;
    // the crowded form takes the tiles the threshold pass listed, or (late)
    // the ones the common form deferred
    const int* list = BIG ? (late ? A.rl_list : A.dl_list) : A.tl_list;
    const int ntl = *(BIG ? (late ? A.rl_count : A.dl_count) : A.tl_count);
    const int nwarps = gridDim.x * Cfg::NW;
    const uint32_t FULL = 0xffffffffu;
    const bool sat_on = A.im.sat > 0.f;
    // the value words are copied asynchronously when they are 4-byte aligned
    const bool sat_async = sat_on && (A.im.is_f32 || (((uintptr_t)A.im.data) & 3) == 0);
    const int y = lane;
    // this lane's row of the mask words of tile t (zeros past the frame)
    auto mask_row = [&](int t) -> uint4 {
        if (t < 0) return make_uint4(0u, 0u, 0u, 0u);
        const int ty_ = t / ntx, tx_ = t - ty_ * ntx;
        if (ty_ * TY + y >= H) return make_uint4(0u, 0u, 0u, 0u);
        return A.bits[(int64_t)(ty_ * TY + y) * A.nstrip + (tx_ >> 1)];
    };
    // the next tile's list entry and mask row are loaded while this one is
    // labelled (both are far-memory reads)
    int it = blockIdx.x * Cfg::NW + warp;
    int tile = it < ntl ? list[it] : -1;
    uint4 wcur = mask_row(tile);
    for (; it < ntl; it += nwarps) {
        const int tile_n = it + nwarps < ntl ? list[it + nwarps] : -1;
        const int ty = tile / ntx, tx = tile - ty * ntx;
        const int x0 = tx * TX, y0 = ty * TY;
        const int tw = min(TX, W - x0), th = min(TY, H - y0);
        // ---- this lane's row mask and runs
        uint64_t M = 0ull;
        {
            const uint4 w = wcur;
            const int sh = (tx & 1) * 16;
            M = spread4(w.x >> sh) | (spread4(w.y >> sh) << 1) | (spread4(w.z >> sh) << 2) | (spread4(w.w >> sh) << 3);
        }
        const uint64_t heads = M & ~(M << 1);
        const int nr = __popcll((long long)heads), nf = __popcll((long long)M);
        int incl = nr | (nf << 16);                        // runs and pixels, both < 2^16
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += t;
        }
        const int rb = (incl & 0xffff) - nr;               // first run id of this row
        const int fb = (incl >> 16) - nf;                  // first foreground pixel of this row
        const int tot = __shfl_sync(FULL, incl, 31);
        const int NR = tot & 0xffff, NF = tot >> 16;
        if (!BIG && (NR > Cfg::RUNS || (!LABEL_ONLY && NF > Cfg::FG))) {
            // crowded: the threshold pass listed it for the crowded form when
            // it has too many foreground pixels; too many runs alone defers it
            if (lane == 0 && (LABEL_ONLY || NF <= Cfg::FG)) A.rl_list[atomicAdd(A.rl_count, 1)] = tile;
            wcur = mask_row(tile_n);
            tile = tile_n;
            continue;
        }
        // ---- m (and the value word, for saturation) of every foreground
        // pixel, copied asynchronously into the compact arrays; the streaming
        // pass left the bits of m in the map there
        if (!LABEL_ONLY && M) {
            const int64_t rowL = (int64_t)(y0 + y) * W + x0;
            const int64_t rowI = (int64_t)(y0 + y) * A.im.pitch + x0;
            uint64_t mb = M;
            for (int f = fb; mb; ++f) {
                const int x = __ffsll((long long)mb) - 1;
                mb &= mb - 1;
                cp_async4(S.m + f, A.seg + rowL + x);
                if (sat_async) {
                    const int64_t li = rowI + x;
                    const void* src = A.im.is_f32
                                          ? (const void*)(reinterpret_cast<const float*>(A.im.data) + li)
                                          : (const void*)(reinterpret_cast<const uint16_t*>(A.im.data) + (li & ~(int64_t)1));
                    cp_async4(S.iv + f, src);
                }
            }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
        {
            uint64_t hb = heads;
            int f = fb;
            for (int q = rb; hb; ++q) {
                const int x = __ffsll((long long)hb) - 1;
                hb &= hb - 1;
                const int xe = run_end(M, x);
                S.par[q] = q; S.cnt[q] = 0; S.val[q] = 0; S.kidx[q] = -1;
                S.pos[q] = (int16_t)(y * TX + x);
                S.fidx[q] = (int16_t)f;
                S.len[q] = (uint8_t)(xe - x);
                f += xe - x + 1;
            }
        }
        __syncwarp();
        // ---- unite each run with the runs of the row above it touches, at
        // one site per contact: the first column of each vertical overlap
        // (V), and a pixel whose only contact is diagonal (NW: the upper run
        // ends at x - 1; NE: it starts at x + 1).  Each overlap of a lower
        // and an upper run is one maximal interval of M & U, so V covers
        // every overlapping pair; a diagonal pair without overlap has
        // U[x] = 0 and M[x -/+ 1] = 0 at its contact, so NW / NE cover the rest.
        {
            const uint64_t Uup = __shfl_up_sync(FULL, M, 1);
            const uint64_t U = lane ? Uup : 0ull;
            const int ub = __shfl_up_sync(FULL, rb, 1);
            const uint64_t uh = U & ~(U << 1);
            const uint64_t O = M & U;
            const uint64_t V = O & ~(O << 1);
            const uint64_t NWm = M & ~U & (U << 1) & ~(M << 1);
            const uint64_t NEm = M & ~U & (U >> 1) & ~(M >> 1);
            uint64_t sites = V | NWm | NEm;
            while (sites) {
                const int x = __ffsll((long long)sites) - 1;
                sites &= sites - 1;
                const int a = rb + __popcll((long long)(heads & upto(x))) - 1;
                if ((V >> x) & 1ull) lunite(S.par, a, ub + __popcll((long long)(uh & upto(x))) - 1);
                if ((NWm >> x) & 1ull) lunite(S.par, a, ub + __popcll((long long)(uh & upto(x - 1))) - 1);
                if ((NEm >> x) & 1ull) lunite(S.par, a, ub + __popcll((long long)(uh & upto(x + 1))) - 1);
            }
        }
        __syncwarp();
        // flatten in two phases: the roots (found with path halving) go to
        // cnt first, then into par once every lane's walks are over -- a
        // halving store from a stale read can then never land on a root
        // that another lane has already written
        for (int q = rb; q < rb + nr; ++q) S.cnt[q] = lfind(S.par, q);
        __syncwarp();
        for (int q = rb; q < rb + nr; ++q) {
            S.par[q] = S.cnt[q];
            S.cnt[q] = 0;
        }
        __syncwarp();
        // ---- pixels and shared-edge contact per root, one atomic per run
        {
            uint64_t hb = heads;
            for (int q = rb; hb; ++q) {
                const int x = __ffsll((long long)hb) - 1;
                hb &= hb - 1;
                const int xe = run_end(M, x);
                const bool border = (x == 0 && x0 > 0) || (xe == tw - 1 && x0 + tw < W) || (y == 0 && y0 > 0) ||
                                    (y == th - 1 && y0 + th < H);
                atomicAdd(S.cnt + S.par[q], (xe - x + 1) + (border ? (1 << 16) : 0));
            }
        }
        const uint4 wnext = mask_row(tile_n);
        __syncwarp();
        // ---- kept roots, in label order: pieces (on a shared edge) and final
        // segments (>= minarea); local indices, map values, one id
        // reservation per kind per tile
        int np = 0, nc = 0, nk = 0;
        for (int c0 = 0; c0 < NR; c0 += 32) {
            const int k = c0 + lane;
            bool piece = false, comp = false;
            if (k < NR && S.par[k] == k) {
                const int v = S.cnt[k];
                piece = (v >> 16) != 0;
                comp = !piece && (v & 0xffff) >= A.minarea;
            }
            const uint32_t bp = __ballot_sync(FULL, piece), bc = __ballot_sync(FULL, comp);
            const uint32_t lt = (1u << lane) - 1u;
            if (piece || comp) {
                const int p = S.pos[k];
                S.val[k] = (int)((uint32_t)(y0 + p / TX) * (uint32_t)W + (uint32_t)(x0 + p % TX) + 1u);
                S.klist[nk + __popc((bp | bc) & lt)] = (int16_t)k;
                S.kidx[k] = piece ? (int16_t)(np + __popc(bp & lt)) : (int16_t)(-2 - (nc + __popc(bc & lt)));
            }
            np += __popc(bp);
            nc += __popc(bc);
            nk += __popc(bp | bc);
        }
        // id reservation (one per kind per tile), consumed after the map and
        // edge records are written
        int pbase = 0, cbase = 0;
        if (lane == 0) {
            pbase = np ? atomicAdd(A.P.count, np) : 0;
            cbase = nc ? atomicAdd(A.C.count, nc) : 0;
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
        __syncwarp();
        // ---- the map at every foreground pixel: the label of its kept
        // segment, or 0 (a dropped segment; the streaming pass left m there)
        if (y < th) {
            uint32_t* srow = A.seg + (int64_t)(y0 + y) * W + x0;
            uint64_t hb = heads;
            for (int q = rb; hb; ++q) {
                const int x = __ffsll((long long)hb) - 1;
                hb &= hb - 1;
                const uint32_t v = (uint32_t)S.val[S.par[q]];
                if (LABEL_ONLY && !v) continue;          // a given mask: the map is already 0 there
                const int xe = run_end(M, x);
                for (int xx = x; xx <= xe; ++xx) srow[xx] = v;
            }
        }
        // ---- edge records of a tile with pieces: local piece index of each
        // edge pixel, or -1
        if (np) {
            int16_t* ed = A.T.edges + (int64_t)tile * EDGE_PER_TILE;
            const uint64_t M0 = __shfl_sync(FULL, M, 0), H0 = __shfl_sync(FULL, heads, 0);
            const uint64_t MB = __shfl_sync(FULL, M, th - 1), HB = __shfl_sync(FULL, heads, th - 1);
            const int rbB = __shfl_sync(FULL, rb, th - 1);
            auto piece_at = [&](uint64_t Mr, uint64_t Hr, int rbase, int x) -> int16_t {
                if (!((Mr >> x) & 1ull)) return (int16_t)-1;
                const int16_t k = S.kidx[S.par[rbase + __popcll((long long)(Hr & upto(x))) - 1]];
                return k >= 0 ? k : (int16_t)-1;
            };
            ed[y] = y < th ? piece_at(M, heads, rb, 0) : (int16_t)-1;                 // colL
            ed[TY + y] = y < th ? piece_at(M, heads, rb, tw - 1) : (int16_t)-1;       // colR
            for (int x = lane; x < TX; x += 32) {
                ed[2 * TY + x] = x < tw ? piece_at(M0, H0, 0, x) : (int16_t)-1;       // rowT
                ed[2 * TY + TX + x] = x < tw ? piece_at(MB, HB, rbB, x) : (int16_t)-1;   // rowB
            }
        }
        if (lane == 0) {
            A.T.piece_base[tile] = pbase;
            A.T.piece_cnt[tile] = np;
        }
        pbase = __shfl_sync(FULL, pbase, 0);
        cbase = __shfl_sync(FULL, cbase, 0);
        // ---- kept segments of at most LANE_SEG_MAX pixels: one lane each (its
        // runs in label order), when the tile holds at least eight of them
        // (fewer leave most lanes idle; measured against 2, 4, 12 and 16)
        int nsmall = 0;
        for (int c0 = 0; c0 < nk; c0 += 32) {
            const int i = c0 + lane;
            nsmall += __popc(__ballot_sync(FULL, i < nk && (S.cnt[S.klist[i]] & 0xffff) <= LANE_SEG_MAX));
        }
        const bool lane_path = nsmall >= 8;
        if (lane_path) {
            // runs of each small kept segment, in label order: runs are taken
            // 32 at a time in id order; the lanes holding runs of one segment
            // find each other (match) and the first of them advances its count
            for (int c0 = 0; c0 < nk; c0 += 32) {
                const int i = c0 + lane;
                if (i < nk) S.rcnt[S.klist[i]] = 0;
            }
            for (int pass = 0; pass < 2; ++pass) {
                if (pass == 1) {
                    // offsets: the segments' runs laid out in kept-root order
                    int off = 0;
                    for (int c0 = 0; c0 < nk; c0 += 32) {
                        const int i = c0 + lane;
                        const int r = i < nk ? S.klist[i] : -1;
                        const int c = (r >= 0 && (S.cnt[r] & 0xffff) <= LANE_SEG_MAX) ? S.rcnt[r] : 0;
                        int inc = c;
#pragma unroll
                        for (int o = 1; o < 32; o <<= 1) {
                            const int t = __shfl_up_sync(FULL, inc, o);
                            if (lane >= o) inc += t;
                        }
                        if (r >= 0) { S.roff[r] = (int16_t)(off + inc - c); S.rcnt[r] = 0; }
                        off += __shfl_sync(FULL, inc, 31);
                    }
                }
                __syncwarp();
                for (int c0 = 0; c0 < NR; c0 += 32) {
                    const int q = c0 + lane;
                    const int r = q < NR ? S.par[q] : -1;
                    const bool mine = r >= 0 && S.val[r] != 0 && (S.cnt[r] & 0xffff) <= LANE_SEG_MAX;
                    const uint32_t peers = __match_any_sync(FULL, mine ? r : -1);
                    const int rank = __popc(peers & ((1u << lane) - 1u));
                    const int base = mine ? S.rcnt[r] : 0;
                    __syncwarp();
                    if (mine) {
                        if (pass == 1) S.rlist[S.roff[r] + base + rank] = (int16_t)q;
                        if (rank == 0) S.rcnt[r] = (int16_t)(base + __popc(peers));
                    }
                    __syncwarp();
                }
            }
            for (int c0 = 0; c0 < nk; c0 += 32) {
                const int i = c0 + lane;
                const int r = i < nk ? S.klist[i] : -1;
                if (r < 0 || (S.cnt[r] & 0xffff) > LANE_SEG_MAX) continue;
                MomAcc a;
                mom_zero(a);
                int bx0 = TX, bx1 = -1, by1 = -1;
                const int e0 = S.roff[r], e1 = e0 + S.rcnt[r];
                for (int e = e0; e < e1; ++e) {
                    const int q = S.rlist[e];
                    const int p = S.pos[q], ry = p / TX, rx = p % TX, n = S.len[q] + 1;
                    bx0 = min(bx0, rx); bx1 = max(bx1, rx + n - 1); by1 = ry;
                    if (!LABEL_ONLY) {
                        const int f0 = S.fidx[q];
                        const int64_t lin = (int64_t)(y0 + ry) * A.im.pitch + x0 + rx;
                        const uint32_t L0 = (uint32_t)(y0 + ry) * (uint32_t)W + (uint32_t)(x0 + rx);
                        DF r0 = df_zero(), r1 = df_zero(), r2 = df_zero();
                        for (int t = 0; t < n; ++t)
                            run_pixel(r0, r1, r2, a, S.m[f0 + t], rx + t, L0 + t,
                                      sat_on && pix_sat(A, sat_async, S.iv[f0 + t], lin + t));
                        mom_fold(a, r0, r1, r2, rx, rx + n - 1, ry);
                    }
                }
                const int ry0 = S.pos[r] / TX;
                emit_root<LABEL_ONLY, BIG>(A, S, r, make_int4(x0 + bx0, x0 + bx1, y0 + ry0, y0 + by1), pbase, cbase,
                                           x0, y0, a);
            }
        }
        // ---- the other kept segments: the whole warp, lane = tile row; the
        // sums meet in the segment's first row by a tree over its rows
        for (int i = 0; i < nk; ++i) {
            const int r = S.klist[i];
            if (lane_path && (S.cnt[r] & 0xffff) <= LANE_SEG_MAX) continue;
            int xmin = TX, xmax = -1;
            MomAcc a;
            mom_zero(a);
            uint64_t hb = heads;
            for (int q = rb; hb; ++q) {
                const int x = __ffsll((long long)hb) - 1;
                hb &= hb - 1;
                if (S.par[q] != r) continue;
                const int xe = run_end(M, x);
                xmin = min(xmin, x);
                xmax = max(xmax, xe);
                if (!LABEL_ONLY) {
                    const int f0 = S.fidx[q];
                    const int64_t lin = (int64_t)(y0 + y) * A.im.pitch + x0 + x;
                    const uint32_t L0 = (uint32_t)(y0 + y) * (uint32_t)W + (uint32_t)(x0 + x);
                    DF r0 = df_zero(), r1 = df_zero(), r2 = df_zero();
                    for (int t = 0; t <= xe - x; ++t)
                        run_pixel(r0, r1, r2, a, S.m[f0 + t], x + t, L0 + t,
                                  sat_on && pix_sat(A, sat_async, S.iv[f0 + t], lin + t));
                    mom_fold(a, r0, r1, r2, x, xe, y);
                }
            }
            const bool present = xmax >= 0;
            const int ry0 = S.pos[r] / TX;
            const int bx0 = __reduce_min_sync(FULL, xmin), bx1 = __reduce_max_sync(FULL, xmax);
            const int by1 = __reduce_max_sync(FULL, present ? y : -1);
            if (!LABEL_ONLY) {
                const int span = by1 - ry0 + 1;
                mom_rows_reduce(a, span <= 1 ? 0 : 32 - __clz(span - 1));
            }
            if (lane == ry0)
                emit_root<LABEL_ONLY, BIG>(A, S, r, make_int4(x0 + bx0, x0 + bx1, y0 + ry0, y0 + by1), pbase, cbase,
                                           x0, y0, a);
        }
        __syncwarp();
        wcur = wnext;
        tile = tile_n;
    }
}

// ------------------------------------------------------------ tile merge ---
// The contacts across one tile edge: a[i] is this tile's edge pixel i and b[k]
// the neighbour's facing pixel k (local piece indices, -1 off the foreground),
// 8-connected (k = i - 1, i, i + 1).  A pixel's contact is skipped where the
// same pair of pieces is united by its straight contact or by the straight
// contact of the pixel before (i - 1) or after (i + 1): a run of pixels along
// the edge then unites each pair of pieces once instead of up to three times
// per pixel.  (Every skipped pair is united by a straight contact that is
// itself kept or skipped only for an identical pair at a lower index.)
__device__ __forceinline__ void unite_edge(const int16_t* a, const int16_t* b, int n, int base, int nbase, int lane,
                                           int* parent, int lim, int* status)
{
    for (int i = lane; i < n; i += 32) {
        const int ai = a[i];
        if (ai < 0) continue;
        const int bi = b[i];
        const int ap = i > 0 ? a[i - 1] : -1, bp = i > 0 ? b[i - 1] : -1;
        const int an = i + 1 < n ? a[i + 1] : -1, bn = i + 1 < n ? b[i + 1] : -1;
        if (bi >= 0 && !(ap == ai && bp == bi)) gunite(parent, base + ai, nbase + bi, lim, status);
        if (bp >= 0 && bp != bi && ap != ai) gunite(parent, base + ai, nbase + bp, lim, status);
        if (bn >= 0 && bn != bi && an != ai) gunite(parent, base + ai, nbase + bn, lim, status);
    }
}

// One warp per listed tile with pieces: its right and bottom edges and its
// two lower diagonal corners against the neighbouring tiles' edge records
// (a tile without pieces records none).
__global__ void k_merge(const ResolveArgs* __restrict__ batch, const __grid_constant__ ResolveArgs one)
{
    pdl_wait();
    pdl_release();
    const ResolveArgs& R = frame_args(batch, one);
    const Tiles& T = R.T;
    const Pieces& P = R.P;
    const int W = R.W, H = R.H, lim = R.walk_limit;
    int* status = R.status;
    const int ntx = T.ntx, nty = T.nty;
    const int ntl = *R.tl_count;
    const int lane = threadIdx.x & 31;
    const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (int it = wid; it < ntl; it += nw) {
        const int tile = R.tl_list[it];
        if (T.piece_cnt[tile] == 0) continue;
        const int tx = tile % ntx, ty = tile / ntx;
        const int tw = min(TX, W - tx * TX), th = min(TY, H - ty * TY);
        const int base = T.piece_base[tile];
        const int16_t* e = T.edges + (int64_t)tile * EDGE_PER_TILE;
        if (tx + 1 < ntx && T.piece_cnt[tile + 1] > 0)      // right column against the left one of the tile right
            unite_edge(e + TY, T.edges + (int64_t)(tile + 1) * EDGE_PER_TILE, th, base, T.piece_base[tile + 1],
                       lane, P.parent, lim, status);
        if (ty + 1 < nty && T.piece_cnt[tile + ntx] > 0)    // bottom row against the top one of the tile below
            unite_edge(e + 2 * TY + TX, T.edges + (int64_t)(tile + ntx) * EDGE_PER_TILE + 2 * TY, tw, base,
                       T.piece_base[tile + ntx], lane, P.parent, lim, status);
        if (lane == 0 && ty + 1 < nty) {
            // bottom-right pixel of this tile and top-left pixel of the tile below-right
            if (tx + 1 < ntx && T.piece_cnt[tile + ntx + 1] > 0) {
                const int a = e[TY + th - 1];
                const int b = T.edges[(int64_t)(tile + ntx + 1) * EDGE_PER_TILE + 0];
                if (a >= 0 && b >= 0) gunite(P.parent, base + a, T.piece_base[tile + ntx + 1] + b, lim, status);
            }
            // bottom-left pixel of this tile and top-right pixel of the tile below-left
            if (tx > 0 && T.piece_cnt[tile + ntx - 1] > 0) {
                const int a = e[th - 1];
                const int b = T.edges[(int64_t)(tile + ntx - 1) * EDGE_PER_TILE + TY + 0];
                if (a >= 0 && b >= 0) gunite(P.parent, base + a, T.piece_base[tile + ntx - 1] + b, lim, status);
            }
        }
    }
}

// --------------------------------------------------------- piece resolve ---
__global__ void k_aggregate(const ResolveArgs* __restrict__ batch, const __grid_constant__ ResolveArgs one)
{
    pdl_wait();
    pdl_release();
    const ResolveArgs& R = frame_args(batch, one);
    const Pieces& P = R.P;
    int* status = R.status;
    const int n = min(*P.count, P.cap);
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const int r = gfind(P.parent, p, R.walk_limit);
        P.proot[p] = r;
        if (r < 0) { set_status(status, GP_ERR_TIMEOUT); continue; }
        if (r == p) continue;
        // the unions are done: pointing p at its root shortens the other
        // threads' walks through p (they read the old parent or the root)
        P.parent[p] = r;
        atomicMin(P.agg_min + r, P.root[p]);
        atomicAdd(P.agg_npix + r, P.npix[p]);
        const int4 b = P.bbox[p];
        int* ab = reinterpret_cast<int*>(P.agg_bbox + r);
        atomicMin(ab + 0, b.x); atomicMax(ab + 1, b.y);
        atomicMin(ab + 2, b.z); atomicMax(ab + 3, b.w);
    }
}

// One warp per piece.  At root pieces of kept segments: merge the partial
// moments of all the segment's pieces, visiting the tiles of the segment's
// bounding box in raster order (a fixed order, so the sums are
// reproducible) and emit the segment; a segment of a single piece is emitted
// from that piece's sums directly (the merge would add zeros to them).  Every piece whose final label differs
// from its provisional one rewrites its pixels in the map.
__global__ void __launch_bounds__(256, 4) k_finalize(const ResolveArgs* __restrict__ batch, const __grid_constant__ ResolveArgs one)
{
    pdl_wait();
    pdl_release();
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
        // the piece's box, 8 pixels per lane at a time: all loads first, then
        // the stores (a pixel of another label is never this piece's, and
        // this piece's pixels are rewritten by this warp only)
        const int4 b = P.bbox[p];
        const int bw = b.y - b.x + 1, npx = bw * (b.w - b.z + 1);
        constexpr int RW = 8;
        for (int q0 = lane; q0 < npx; q0 += 32 * RW) {
            uint32_t v[RW];
            int64_t off[RW];
#pragma unroll
            for (int j = 0; j < RW; ++j) {
                const int q = q0 + 32 * j;
                const int y = b.z + q / bw, x = b.x + q % bw;
                off[j] = (int64_t)y * W + x;
                v[j] = q < npx ? seg[off[j]] : 0u;
            }
#pragma unroll
            for (int j = 0; j < RW; ++j)
                if (v[j] == prov) seg[off[j]] = fin;
        }
    }
}

// Centroid and second moments of every segment stored with raw sums (one
// thread per segment); segments with a sum <= 0 were finished where they were
// found and carry GP_FLAG_CENTROID_FALLBACK.
__global__ void k_mom_finish(const ResolveArgs* __restrict__ batch, const __grid_constant__ ResolveArgs one)
{
    pdl_wait();
    pdl_release();
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
    pdl_wait();
    pdl_release();
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
    pdl_wait();
    pdl_release();
    const RankArgs& R = frame_args(batch, one);
    const Comps& C = R.C;
    int* n_out = R.n_out;
    const int capacity = R.capacity;
    int* status = R.status;
    __shared__ int wsum[SCAN_NT / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nb = C.nb;                                     // <= 16,384
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
    pdl_wait();
    pdl_release();
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
    pdl_wait();
    pdl_release();
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
// the normalised kernel (kh x kw) padded to ks x ks, as a sum of separable
// terms by full-pivot elimination in double: each step takes the largest
// remaining entry K[pv][pu] as pivot and removes the outer product of its
// column and row; it stops when what remains is within 1e-6 of the largest
// tap (below float32 rounding of the correlation's 25-term sums).  A
// Gaussian, or any outer product, is one term; the worst case is ks terms.
static int factor_kernel(const float* taps, int kw, int kh, int ks, float* fv, float* fh)
{
    double R[2 * HMAX + 1][2 * HMAX + 1] = {};
    const int oy = (ks - kh) / 2, ox = (ks - kw) / 2;
    double amax = 0.0;
    for (int v = 0; v < kh; ++v)
        for (int u = 0; u < kw; ++u) {
            R[v + oy][u + ox] = taps[v * kw + u];
            amax = fmax(amax, fabs((double)taps[v * kw + u]));
        }
    int r = 0;
    for (; r < ks; ++r) {
        int pv = 0, pu = 0;
        double best = -1.0;
        for (int v = 0; v < ks; ++v)
            for (int u = 0; u < ks; ++u)
                if (fabs(R[v][u]) > best) { best = fabs(R[v][u]); pv = v; pu = u; }
        if (best <= 1e-6 * amax) break;
        const double p = R[pv][pu];
        double col[2 * HMAX + 1], row[2 * HMAX + 1];
        for (int v = 0; v < ks; ++v) col[v] = R[v][pu] / p;
        for (int u = 0; u < ks; ++u) row[u] = R[pv][u];
        for (int v = 0; v < ks; ++v) {
            fv[r * ks + v] = (float)col[v];
            for (int u = 0; u < ks; ++u) R[v][u] -= col[v] * row[u];
        }
        for (int u = 0; u < ks; ++u) fh[r * ks + u] = (float)row[u];
    }
    return r;
}

DetectArgs detect_args(const Image& im, const SplineTab& sb, const SplineTab& sr, const float* taps, int kw, int kh,
                       float thresh, int minarea, uint32_t* seg, uint8_t* mask_out, int* nnear,
                       const uint8_t* in_mask, const DetMask& dm, const Tiles& T, const Pieces& P, const Comps& C,
                       int* status)
{
    DetectArgs A;
    memset(&A, 0, sizeof A);
    A.ks = stream_ks(kw, kh);
    A.nrank = taps ? factor_kernel(taps, kw, kh, A.ks, A.fv, A.fh) : 0;
    A.im = im; A.sb = sb; A.sr = sr;
    A.thresh = thresh; A.minarea = minarea;
    A.seg = seg; A.mask_out = mask_out; A.nnear = nnear; A.in_mask = in_mask;
    A.bits = dm.bits; A.nstrip = (im.W + ST_STRIP - 1) / ST_STRIP;
    A.tl_list = dm.tl_list; A.tl_count = dm.tl_count;
    A.dl_list = dm.dl_list; A.dl_count = dm.dl_count;
    A.rl_list = dm.rl_list; A.rl_count = dm.rl_count;
    A.T = T; A.P = P; A.C = C; A.status = status;
    return A;
}

// grid of the grid-stride kernels: about `per_frame` CTAs over the whole batch
static int stride_grid(int per_frame, int nframes)
{
    const int g = per_frame / nframes;
    return g < 16 ? 16 : g;
}

// the labelling kernel's persistent grids: the common form at eleven CTAs of
// two warps per SM (21 KB of shared memory and at most 88 registers each),
// the big form (crowded tiles) at four CTAs of two warps
constexpr int LT_CTAS = 152 * 11;
constexpr int LT_BIG_CTAS = 152 * 4;
constexpr int LT_LATE_CTAS = 152;         // the deferred tiles: few or none

int detect_grid(int W, int H, bool given_mask) { return given_mask ? pack_warps(W, H) : stream_ctas(W, H); }

// The crowded tiles: one warp per listed tile counts its foreground pixels
// from the packed mask (lane = tile row) and lists the tile for the crowded
// form when the common form cannot hold them.
template <bool BATCH>
__global__ void __launch_bounds__(256) k_tile_census(const DetectArgs* __restrict__ batch,
                                                     const __grid_constant__ DetectArgs one)
{
    pdl_wait();
    pdl_release();
    const DetectArgs& A = det_frame<BATCH>(batch, one);
    const int lane = threadIdx.x & 31;
    const int ntl = *A.tl_count;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int it = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; it < ntl; it += nw) {
        const int tile = A.tl_list[it];
        const int ty = tile / A.T.ntx, tx = tile - ty * A.T.ntx;
        const int y = ty * TY + lane;
        int c = 0;
        if (y < A.im.H) {
            const uint4 w = A.bits[(int64_t)y * A.nstrip + (tx >> 1)];
            const uint32_t m = (tx & 1) ? 0xffff0000u : 0x0000ffffu;
            c = __popc(w.x & m) + __popc(w.y & m) + __popc(w.z & m) + __popc(w.w & m);
        }
        c = __reduce_add_sync(0xffffffffu, c);
        if (lane == 0 && c > LT_FG) A.dl_list[atomicAdd(A.dl_count, 1)] = tile;
    }
}

template <bool LO, bool BATCH, bool BIG>
static void launch_label(const DetectArgs& one, const DetectArgs* batch, dim3 g, int late, cudaStream_t st)
{
    const size_t smem = sizeof(LabelSmem<BIG>) * LabelCfg<BIG>::NW;
    auto* fn = k_label_tiles<LO, BATCH, BIG>;
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    // all of the unified L1 / shared memory as shared memory: eleven CTAs of
    // the common form (21 KB each) per SM
    cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    launch_dep(fn, g, dim3(32 * LabelCfg<BIG>::NW), smem, st, batch, one, late);
}

// The census of the listed tiles, then the common form on `st` and the
// crowded tiles on the side stream when there is one (they touch other
// tiles' records only, so the two forms run side by side), else before it
// on `st`; then the tiles the common form deferred, on `st` once both are
// done.
template <bool LO, bool BATCH>
static cudaError_t launch_label_forms(const DetectArgs& one, const DetectArgs* batch, int nframes, cudaStream_t st,
                                      const SideStream* side)
{
    const dim3 gc(BATCH ? stride_grid(LT_CTAS, nframes) : LT_CTAS, nframes);
    const dim3 gb(BATCH ? stride_grid(LT_BIG_CTAS, nframes) : LT_BIG_CTAS, nframes);
    const dim3 gl(BATCH ? stride_grid(LT_LATE_CTAS, nframes) : LT_LATE_CTAS, nframes);
    cudaError_t e = cudaSuccess;
    if (!LO) {
        launch_dep(k_tile_census<BATCH>, gc, dim3(256), 0, st, batch, one);
        if (side) {
            if ((e = cudaEventRecord(side->fork, st)) != cudaSuccess) return e;
            if ((e = cudaStreamWaitEvent(side->st, side->fork, 0)) != cudaSuccess) return e;
            launch_label<LO, BATCH, true>(one, batch, gb, 0, side->st);
            if ((e = cudaEventRecord(side->join, side->st)) != cudaSuccess) return e;
        } else {
            launch_label<LO, BATCH, true>(one, batch, gb, 0, st);
        }
    }
    launch_label<LO, BATCH, false>(one, batch, gc, 0, st);
    if (!LO && side && (e = cudaStreamWaitEvent(st, side->join, 0)) != cudaSuccess) return e;
    launch_label<LO, BATCH, true>(one, batch, gl, 1, st);
    return cudaGetLastError();
}

int label_launches(bool given_mask) { return given_mask ? 2 : 4; }

cudaError_t launch_label_any(const DetectArgs& one, const DetectArgs* batch, int nframes, cudaStream_t st,
                             const SideStream* side)
{
    if (one.in_mask) return batch ? launch_label_forms<true, true>(one, batch, nframes, st, side)
                                  : launch_label_forms<true, false>(one, batch, nframes, st, side);
    return batch ? launch_label_forms<false, true>(one, batch, nframes, st, side)
                 : launch_label_forms<false, false>(one, batch, nframes, st, side);
}

ResolveArgs resolve_args(const Tiles& T, const Pieces& P, const Comps& C, const DetMask& dm, uint32_t* seg, int W,
                         int H, int minarea, int walk_limit, int* status)
{
    ResolveArgs R;
    R.T = T; R.P = P; R.C = C; R.seg = seg; R.tl_list = dm.tl_list; R.tl_count = dm.tl_count;
    R.W = W; R.H = H; R.minarea = minarea; R.walk_limit = walk_limit > 0 ? walk_limit : WALK_LIMIT;
    R.status = status;
    return R;
}

cudaError_t launch_resolve_any(const ResolveArgs& one, const ResolveArgs* batch, int nframes, int maxtiles,
                               cudaStream_t st)
{
    const dim3 g(stride_grid(152 * 8, nframes), nframes);
    // the merge: one warp per listed tile (latency-bound chains), up to 152 x 32 CTAs of 4 warps
    const int mcta = std::min((maxtiles + 3) / 4, 152 * 32);
    launch_dep(k_merge, dim3(std::max(1, mcta / (nframes > 1 ? 2 : 1)), nframes), dim3(128), 0, st, batch, one);
    launch_dep(k_aggregate, g, dim3(256), 0, st, batch, one);
    launch_dep(k_finalize, g, dim3(256), 0, st, batch, one);
    launch_dep(k_mom_finish, g, dim3(256), 0, st, batch, one);
    return cudaGetLastError();
}

cudaError_t launch_resolve(const Tiles& T, const Pieces& P, const Comps& C, const DetMask& dm, uint32_t* seg, int W,
                           int H, int minarea, int walk_limit, int* status, cudaStream_t st)
{
    return launch_resolve_any(resolve_args(T, P, C, dm, seg, W, H, minarea, walk_limit, status), nullptr, 1,
                              T.ntx * T.nty, st);
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
    launch_dep(k_rank_count, g, dim3(256), 0, st, batch, one);
    launch_dep(k_rank_scan, dim3(1, nframes), dim3(SCAN_NT), 0, st, batch, one);
    if (one.place) {
        launch_dep(k_rank_scatter, g, dim3(256), 0, st, batch, one);
        launch_dep(k_rank_place, g, dim3(256), 0, st, batch, one);
    }
    return cudaGetLastError();
}

cudaError_t launch_rank(const Comps& C, int* n_out, int capacity, bool place, int* status, cudaStream_t st)
{
    return launch_rank_any(rank_args(C, n_out, capacity, place, status), nullptr, 1, st);
}

}  // namespace gp
