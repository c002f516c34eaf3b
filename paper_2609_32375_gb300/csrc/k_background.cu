// k_background.cu -- local background and noise map (paper Section 3.1).
//
//  k_boxstats_u16  one CTA per mesh box: the box's uint16 values go into an
//                  exact 65,536-bin shared-memory histogram (two 16-bit
//                  counters per 32-bit word), summarised into 256 coarse bins
//                  with exact integer count / sum / sum-of-squares prefixes.
//                  The k-sigma clip then runs on the histogram, not on the
//                  pixels: each pass is two range sums and one or two order
//                  statistics, all in exact integer arithmetic.
//  k_boxstats_f32  one CTA per box (<= 16,384 pixels): values sorted in
//                  shared memory (bitonic), the clipped set is an index range
//                  of the sorted array, sums in compensated FP32.
//  k_mesh_finalize fills boxes with < 50 % good pixels from valid neighbours
//                  and median-filters both meshes (one CTA, tiny).
//  k_spline_*      second-derivative tables of the tensor-product natural
//                  spline through the box centres (FP64 tridiagonal solves).
//  k_bkg_maps      optional full-resolution B(p), sigma(p) output.
#include <float.h>
#include <math.h>

#include "gp_internal.cuh"
#include "gp_launch.h"

namespace gp {

// The box statistics of the clipped set, from which background and rms
// follow.  bkg = median if sigma == 0 or |mean - median| / sigma > 0.3, else
// the mode estimate 2.5 median - 1.5 mean; rms = sigma.
__device__ __forceinline__ void box_result(double med, double mean, double sd, double* bkg, double* rms)
{
    double b;
    if (sd == 0.0 || fabs(mean - med) > 0.3 * sd)
        b = med;
    else
        b = 2.5 * med - 1.5 * mean;
    *bkg = b;
    *rms = sd;
}

// ============================================================ uint16 box ===
constexpr int U16_NT = 1024;
constexpr int U16_WORDS = 32768;   // 65,536 16-bit counters

struct HistSums {
    unsigned long long c, s1, s2;
};

// count / sum / sum of squares of the values < v (exact integers)
// executed by one full warp; every lane returns the result
__device__ HistSums hist_prefix(const uint32_t* hist, const unsigned long long* pc, const unsigned long long* ps1,
                                const unsigned long long* ps2, uint32_t v)
{
    const int lane = threadIdx.x & 31;
    uint32_t cb = v >> 8;            // coarse bin of v (256 means "all")
    HistSums r;
    r.c = pc[cb]; r.s1 = ps1[cb]; r.s2 = ps2[cb];
    if (cb >= 256) return r;
    // fine part: values cb*256 .. v-1; lane covers 8 values (4 words)
    unsigned long long c = 0, s1 = 0, s2 = 0;
    uint32_t base = (cb << 8) + (uint32_t)lane * 8u;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        uint32_t w = hist[(base >> 1) + q];
        uint32_t v0 = base + 2u * q, v1 = v0 + 1u;
        uint32_t n0 = w & 0xffffu, n1 = w >> 16;
        if (v0 < v) { c += n0; s1 += (unsigned long long)n0 * v0; s2 += (unsigned long long)n0 * v0 * v0; }
        if (v1 < v) { c += n1; s1 += (unsigned long long)n1 * v1; s2 += (unsigned long long)n1 * v1 * v1; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        c += __shfl_xor_sync(0xffffffffu, c, o);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    r.c += c; r.s1 += s1; r.s2 += s2;
    return r;
}

// the value of global rank r (0-based, r < total count); one full warp
__device__ uint32_t hist_select(const uint32_t* hist, const unsigned long long* pc, unsigned long long r)
{
    const int lane = threadIdx.x & 31;
    // coarse bin: largest cb with pc[cb] <= r  (pc is non-decreasing, pc[0] = 0)
    // lane l checks bins 8l .. 8l+7
    int best = -1;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        int cb = lane * 8 + q;
        if (pc[cb] <= r && pc[cb + 1] > r) best = cb;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) best = max(best, __shfl_xor_sync(0xffffffffu, best, o));
    int cb = best < 0 ? 255 : best;
    unsigned long long rem = r - pc[cb];
    // fine: inclusive scan over this coarse bin's 256 counters, 8 per lane
    uint32_t base = ((uint32_t)cb << 8) + (uint32_t)lane * 8u;
    uint32_t cnt[8];
    uint32_t tot = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        uint32_t w = hist[(base >> 1) + q];
        cnt[2 * q] = w & 0xffffu;
        cnt[2 * q + 1] = w >> 16;
        tot += cnt[2 * q] + cnt[2 * q + 1];
    }
    uint32_t incl = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    uint32_t excl = incl - tot;
    // the lane whose range holds rem
    bool mine = (excl <= rem) && (rem < incl);
    uint32_t ans = 0;
    if (mine) {
        uint32_t acc = excl;
        for (int q = 0; q < 8; ++q) {
            acc += cnt[q];
            if (rem < acc) { ans = base + q; break; }
        }
    }
    unsigned ball = __ballot_sync(0xffffffffu, mine);
    int src = ball ? (__ffs(ball) - 1) : 0;
    return __shfl_sync(0xffffffffu, ans, src);
}

// queries on the full 65,536-bin histogram
struct FullHist {
    const uint32_t* hist;
    const unsigned long long *pc, *ps1, *ps2;
    bool failed = false;
    __device__ HistSums prefix(uint32_t v) { return hist_prefix(hist, pc, ps1, ps2, v); }
    __device__ uint32_t select(unsigned long long r) { return hist_select(hist, pc, r); }
};

// Iterative k-sigma clip about the median on a histogram (one full warp):
// the kept set is always the values in an integer range [a, b]; statistics
// from exact integer sums, median by rank selection.
template <class Q>
__device__ __forceinline__ void clip_histogram(Q& q, uint32_t vmin, uint32_t vmax, double k, int maxiter, double* med_o,
                                               double* mean_o, double* sd_o)
{
    uint32_t a = vmin, b = vmax;
    HistSums lo = q.prefix(a);
    HistSums hi = q.prefix(b + 1u);
    unsigned long long n = hi.c - lo.c, S1 = hi.s1 - lo.s1, S2 = hi.s2 - lo.s2;
    double med = 0, mean = 0, sd = 0;
    for (int it = 0;; ++it) {
        uint32_t m0 = q.select(lo.c + (n - 1) / 2);
        uint32_t m1 = (n & 1ull) ? m0 : q.select(lo.c + n / 2);
        med = 0.5 * ((double)m0 + (double)m1);
        const double in = recip_pos((double)n);
        mean = (double)S1 * in;
        // population variance from exact integers: (n S2 - S1^2) / n^2
        unsigned long long num = n * S2 - S1 * S1;
        sd = sqrt_pos((double)num) * in;
        if (it >= maxiter) break;
        double flo = med - k * sd, fhi = med + k * sd;
        double ca = ceil(flo), cbv = floor(fhi);
        uint32_t na = ca <= (double)a ? a : (uint32_t)ca;
        uint32_t nbv = cbv >= (double)b ? b : (cbv < 0 ? 0u : (uint32_t)cbv);
        if (nbv < na) { na = a; nbv = a; }   // cannot happen for k > 0 (median lies inside)
        HistSums nlo = q.prefix(na);
        HistSums nhi = q.prefix(nbv + 1u);
        unsigned long long nn = nhi.c - nlo.c;
        if (nn == n || q.failed) break;    // the kept set did not change (or the query failed)
        a = na; b = nbv; lo = nlo; hi = nhi;
        n = nn; S1 = nhi.s1 - nlo.s1; S2 = nhi.s2 - nlo.s2;
    }
    *med_o = med;
    *mean_o = mean;
    *sd_o = sd;
}

// rank of quantile q of n good values (features for the learned background)
__device__ __forceinline__ unsigned long long quantile_rank(float q, uint32_t n)
{
    return (unsigned long long)floor((double)q * (double)(n - 1) + 0.5);
}

__device__ void boxstats_u16_box(const BoxArgs& A, int box, uint32_t* hist);

// One CTA per box (or, with A.fb_list set, a persistent grid over the boxes
// listed there): the full 65,536-bin histogram in shared memory.
__global__ void __launch_bounds__(U16_NT, 1) k_boxstats_u16(const BoxArgs* __restrict__ batch, const __grid_constant__ BoxArgs one)
{
    pdl_wait();
    pdl_release();
    const BoxArgs& A = frame_args(batch, one);
    extern __shared__ uint32_t hist[];                    // U16_WORDS
    const bool listed = A.fb_list != nullptr;
    const int count = listed ? *A.fb_count : A.nbox;
    for (int i = blockIdx.x; i < count; i += gridDim.x) {
        __syncthreads();                                  // the previous box is done with the histogram
        boxstats_u16_box(A, listed ? A.fb_list[i] : i, hist);
    }
}

__device__ void boxstats_u16_box(const BoxArgs& A, int box, uint32_t* hist)
{
    const uint16_t* __restrict__ img = static_cast<const uint16_t*>(A.img);
    const int64_t pitch = A.pitch;
    const uint8_t* __restrict__ mask = A.mask;
    const int W = A.W, H = A.H, B = A.B, Mx = A.Mx, nbox = A.nbox;
    const double k = A.k;
    const int maxiter = A.maxiter;
    double* __restrict__ bkg_out = A.bkg;
    double* __restrict__ rms_out = A.rms;
    int* __restrict__ valid_out = A.valid;
    float* __restrict__ quant_out = A.quant;
    __shared__ unsigned long long pc[257], ps1[257], ps2[257];
    __shared__ unsigned long long cc_s[256], cs1_s[256], cs2_s[256];
    __shared__ uint32_t red_min[32], red_max[32], red_n[32];

    const int bi = box % Mx, bj = box / Mx;
    const int x0 = bi * B, x1 = min(x0 + B, W);
    const int y0 = bj * B, y1 = min(y0 + B, H);
    const int bw = x1 - x0, bh = y1 - y0;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    for (int w = tid; w < U16_WORDS; w += U16_NT) hist[w] = 0u;
    __syncthreads();

    uint32_t vmin = 0xffffffffu, vmax = 0u, ngood = 0u;
    // 8-pixel chunks along each row; rows spread over the CTA
    const int cpr = (bw + 7) >> 3;              // chunks per row
    const int nchunks = cpr * bh;
    const bool vec = ((((uintptr_t)img) & 15) == 0) && ((pitch & 7) == 0) && ((x0 & 7) == 0) && ((bw & 7) == 0) &&
                     !mask;
    auto count = [&](uint32_t u) {
        atomicAdd(&hist[u >> 1], (u & 1u) ? 65536u : 1u);
        vmin = min(vmin, u);
        vmax = max(vmax, u);
        ++ngood;
    };
    if (vec) {
        // four 16-byte loads in flight per thread before the histogram updates
        constexpr int U = 4;
        for (int c0 = tid; c0 < nchunks; c0 += U * U16_NT) {
            uint4 q[U];
#pragma unroll
            for (int k = 0; k < U; ++k) {
                const int c = c0 + k * U16_NT;
                if (c < nchunks) {
                    const int ry = c / cpr, rc = c - ry * cpr;
                    q[k] = __ldg(reinterpret_cast<const uint4*>(img + (int64_t)(y0 + ry) * pitch + x0 + rc * 8));
                }
            }
#pragma unroll
            for (int k = 0; k < U; ++k) {
                if (c0 + k * U16_NT >= nchunks) break;
                const uint32_t w4[4] = {q[k].x, q[k].y, q[k].z, q[k].w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    count(w4[e] & 0xffffu);
                    count(w4[e] >> 16);
                }
            }
        }
    } else {
        for (int c = tid; c < nchunks; c += U16_NT) {
            const int ry = c / cpr, rc = c - ry * cpr;
            const int y = y0 + ry, xs = x0 + rc * 8;
            const uint16_t* row = img + (int64_t)y * pitch;
            const int nv = min(8, x1 - xs);
            for (int e = 0; e < nv; ++e) {
                if (mask && mask[(int64_t)y * W + xs + e]) continue;
                count(__ldg(row + xs + e));
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        vmin = min(vmin, __shfl_xor_sync(0xffffffffu, vmin, o));
        vmax = max(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
        ngood += __shfl_xor_sync(0xffffffffu, ngood, o);
    }
    if (lane == 0) { red_min[warp] = vmin; red_max[warp] = vmax; red_n[warp] = ngood; }
    __syncthreads();
    if (warp == 0) {
        vmin = red_min[lane]; vmax = red_max[lane]; ngood = red_n[lane];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            vmin = min(vmin, __shfl_xor_sync(0xffffffffu, vmin, o));
            vmax = max(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
            ngood += __shfl_xor_sync(0xffffffffu, ngood, o);
        }
        if (lane == 0) { red_min[0] = vmin; red_max[0] = vmax; red_n[0] = ngood; }
    }
    __syncthreads();
    vmin = red_min[0]; vmax = red_max[0]; ngood = red_n[0];
    const bool valid = ngood > 0 && 2u * ngood >= (uint32_t)(bw * bh);

    if (ngood == 0 || vmin == vmax) {
        // empty box, or a constant one (the only case where one 16-bit
        // counter could have wrapped): statistics are immediate
        if (tid == 0) {
            double med = ngood ? (double)vmin : 0.0;
            double b, r;
            box_result(med, med, 0.0, &b, &r);
            bkg_out[box] = valid ? b : 0.0;
            rms_out[box] = valid ? r : 0.0;
            valid_out[box] = valid;
            if (quant_out)
                for (int q = 0; q < 5; ++q) quant_out[(int64_t)q * nbox + box] = (float)med;
        }
        return;
    }

    // coarse summaries: 256 bins of 256 values
    for (int cb = warp; cb < 256; cb += U16_NT / 32) {
        unsigned long long c = 0, s1 = 0, s2 = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int widx = cb * 128 + lane + 32 * q;
            uint32_t w = hist[widx];
            uint32_t v0 = (uint32_t)widx * 2u, v1 = v0 + 1u;
            uint32_t n0 = w & 0xffffu, n1 = w >> 16;
            c += n0 + n1;
            s1 += (unsigned long long)n0 * v0 + (unsigned long long)n1 * v1;
            s2 += (unsigned long long)n0 * v0 * v0 + (unsigned long long)n1 * v1 * v1;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            c += __shfl_xor_sync(0xffffffffu, c, o);
            s1 += __shfl_xor_sync(0xffffffffu, s1, o);
            s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        }
        if (lane == 0) { cc_s[cb] = c; cs1_s[cb] = s1; cs2_s[cb] = s2; }
    }
    __syncthreads();
    if (warp != 0) return;

    // exclusive prefix over the coarse bins (8 per lane)
    {
        unsigned long long c[8], s1[8], s2[8];
        unsigned long long tc = 0, t1 = 0, t2 = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            c[q] = cc_s[lane * 8 + q]; s1[q] = cs1_s[lane * 8 + q]; s2[q] = cs2_s[lane * 8 + q];
            tc += c[q]; t1 += s1[q]; t2 += s2[q];
        }
        unsigned long long ic = tc, i1 = t1, i2 = t2;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long a = __shfl_up_sync(0xffffffffu, ic, o);
            unsigned long long b = __shfl_up_sync(0xffffffffu, i1, o);
            unsigned long long d = __shfl_up_sync(0xffffffffu, i2, o);
            if (lane >= o) { ic += a; i1 += b; i2 += d; }
        }
        unsigned long long ec = ic - tc, e1 = i1 - t1, e2 = i2 - t2;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            pc[lane * 8 + q] = ec; ps1[lane * 8 + q] = e1; ps2[lane * 8 + q] = e2;
            ec += c[q]; e1 += s1[q]; e2 += s2[q];
        }
        if (lane == 31) { pc[256] = ec; ps1[256] = e1; ps2[256] = e2; }
    }
    __syncwarp();

    FullHist fq{hist, pc, ps1, ps2};
    double med, mean, sd;
    clip_histogram(fq, vmin, vmax, k, maxiter, &med, &mean, &sd);
    if (quant_out) {
        const float qs[5] = {0.10f, 0.25f, 0.50f, 0.75f, 0.90f};
        for (int q = 0; q < 5; ++q) {
            uint32_t v = fq.select(quantile_rank(qs[q], ngood));
            if (lane == 0) quant_out[(int64_t)q * nbox + box] = (float)v;
        }
    }
    if (lane == 0) {
        double bb, rr;
        box_result(med, mean, sd, &bb, &rr);
        bkg_out[box] = valid ? bb : 0.0;
        rms_out[box] = valid ? rr : 0.0;
        valid_out[box] = valid;
    }
}

// =================================================== uint16 box, window ===
// The same statistics from a 4,096-bin histogram of a window [w0, w0 + 4096)
// placed around the median of a sample of the box (every 16th row), plus
// exact count / sum / sum-of-squares aggregates of the good values below and
// above the window.  16 KB of shared memory instead of 128 KB, so several
// boxes run per SM.  The clip and the quantiles need exact per-value counts
// only where they query; a query that falls outside the window (a prefix at
// a value strictly inside (vmin, w0) or (w0 + 4096, vmax], a rank below or
// above it) marks the box, which then goes to the full-histogram kernel.
// Boxes finished here get bit-identical results: the same integer sums, the
// same ranks, the same clip loop.
constexpr int WB_NT = 128;
constexpr int NWIN = 4096;
constexpr int WCB = 64;                 // values per coarse bin of the window
constexpr int NWC = NWIN / WCB;         // 64 coarse bins

struct WinHist {
    const uint32_t* win;                        // NWIN counters
    const unsigned long long *pc, *ps1, *ps2;   // NWC + 1 prefixes; [0] = the values below the window
    uint32_t w0, vmin, vmax;
    unsigned long long tc, ts1, ts2;            // all good values
    bool failed = false;

    __device__ HistSums prefix(uint32_t v)
    {
        const int lane = threadIdx.x & 31;
        HistSums r;
        r.c = r.s1 = r.s2 = 0;
        if (v <= vmin) return r;
        if (v > vmax) { r.c = tc; r.s1 = ts1; r.s2 = ts2; return r; }
        if (v < w0 || v > w0 + NWIN) { failed = true; return r; }
        const uint32_t d = v - w0, cb = d / WCB;
        r.c = pc[cb]; r.s1 = ps1[cb]; r.s2 = ps2[cb];
        if (cb >= NWC) return r;
        unsigned long long c = 0, s1 = 0, s2 = 0;
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const uint32_t bin = cb * WCB + 2u * lane + e;
            if (bin < d) {
                const unsigned long long nb = win[bin], x = w0 + bin;
                c += nb; s1 += nb * x; s2 += nb * x * x;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            c += __shfl_xor_sync(0xffffffffu, c, o);
            s1 += __shfl_xor_sync(0xffffffffu, s1, o);
            s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        }
        r.c += c; r.s1 += s1; r.s2 += s2;
        return r;
    }

    __device__ uint32_t select(unsigned long long r)
    {
        const int lane = threadIdx.x & 31;
        if (r < pc[0] || r >= pc[NWC]) { failed = true; return w0; }
        int best = -1;
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int cb = 2 * lane + e;
            if (pc[cb] <= r && pc[cb + 1] > r) best = cb;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) best = max(best, __shfl_xor_sync(0xffffffffu, best, o));
        const int cb = best < 0 ? NWC - 1 : best;
        const unsigned long long rem = r - pc[cb];
        const uint32_t base = (uint32_t)cb * WCB + 2u * lane;
        const uint32_t n0 = win[base], n1 = win[base + 1];
        const uint32_t tot = n0 + n1;
        uint32_t incl = tot;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        const uint32_t excl = incl - tot;
        const bool mine = (excl <= rem) && (rem < incl);
        const uint32_t ans = w0 + base + ((rem < (unsigned long long)excl + n0) ? 0u : 1u);
        const unsigned ball = __ballot_sync(0xffffffffu, mine);
        const int src = ball ? (__ffs(ball) - 1) : 0;
        return __shfl_sync(0xffffffffu, ans, src);
    }
};

__global__ void __launch_bounds__(WB_NT, 8) k_boxstats_win(const BoxArgs* __restrict__ batch,
                                                        const __grid_constant__ BoxArgs one)
{
    pdl_wait();
    pdl_release();
    const BoxArgs& A = frame_args(batch, one);
    const int box = blockIdx.x;
    if (box >= A.nbox) return;
    const uint16_t* __restrict__ img = static_cast<const uint16_t*>(A.img);
    const int64_t pitch = A.pitch;
    const uint8_t* __restrict__ mask = A.mask;
    const int W = A.W, H = A.H, B = A.B, Mx = A.Mx, nbox = A.nbox;
    __shared__ uint32_t win[NWIN];
    __shared__ uint32_t samp[256];
    __shared__ unsigned long long pc[NWC + 1], ps1[NWC + 1], ps2[NWC + 1];
    __shared__ unsigned long long cc_s[NWC], cs1_s[NWC], cs2_s[NWC];
    __shared__ unsigned long long red64[6][WB_NT / 32];
    __shared__ uint32_t red_min[WB_NT / 32], red_max[WB_NT / 32], red_n[WB_NT / 32];
    __shared__ uint32_t s_w0;

    const int bi = box % Mx, bj = box / Mx;
    const int x0 = bi * B, x1 = min(x0 + B, W);
    const int y0 = bj * B, y1 = min(y0 + B, H);
    const int bw = x1 - x0, bh = y1 - y0;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int cpr = (bw + 7) >> 3;              // 8-pixel chunks per row
    const bool vec = ((((uintptr_t)img) & 15) == 0) && ((pitch & 7) == 0) && ((x0 & 7) == 0) && ((bw & 7) == 0) &&
                     !mask;

    for (int w = tid; w < NWIN; w += WB_NT) win[w] = 0u;
    for (int i = tid; i < 256; i += WB_NT) samp[i] = 0u;
    __syncthreads();

    // ---- sample (every 16th row): median coarse value -> window
    {
        const int srow = (bh + 15) >> 4;
        for (int c = tid; c < srow * cpr; c += WB_NT) {
            const int ry = (c / cpr) * 16, rc = c - (c / cpr) * cpr;
            const int y = y0 + ry, xs = x0 + rc * 8;
            const uint16_t* row = img + (int64_t)y * pitch;
            if (vec) {
                const uint4 q = __ldg(reinterpret_cast<const uint4*>(row + xs));
                const uint32_t w4[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    atomicAdd(&samp[(w4[e] & 0xffffu) >> 8], 1u);
                    atomicAdd(&samp[w4[e] >> 24], 1u);
                }
            } else {
                const int nv = min(8, x1 - xs);
                for (int e = 0; e < nv; ++e) {
                    if (mask && mask[(int64_t)y * W + xs + e]) continue;
                    atomicAdd(&samp[__ldg(row + xs + e) >> 8], 1u);
                }
            }
        }
    }
    __syncthreads();
    if (warp == 0) {
        // coarse bin holding the sample median (8 bins per lane)
        uint32_t cnt[8], tot = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q) { cnt[q] = samp[lane * 8 + q]; tot += cnt[q]; }
        uint32_t incl = tot;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        const uint32_t ns = __shfl_sync(0xffffffffu, incl, 31);
        const uint32_t rank = ns ? (ns - 1) / 2 : 0;
        uint32_t acc = incl - tot;
        int cb = -1;
        for (int q = 0; q < 8; ++q) {
            if (cb < 0 && rank < acc + cnt[q]) cb = lane * 8 + q;
            acc += cnt[q];
        }
        const bool mine = ns && cb >= 0 && (incl - tot) <= rank && rank < incl;
        const unsigned ball = __ballot_sync(0xffffffffu, mine);
        const int mcb = ball ? __shfl_sync(0xffffffffu, cb, __ffs(ball) - 1) : 0;
        if (lane == 0) {
            const int c = mcb * 256 + 128 - NWIN / 2;
            s_w0 = (uint32_t)(c < 0 ? 0 : (c > 65536 - NWIN ? 65536 - NWIN : c));
        }
    }
    __syncthreads();
    const uint32_t w0 = s_w0;

    // ---- window histogram, aggregates outside it, range and count
    uint32_t vmin = 0xffffffffu, vmax = 0u, ngood = 0u;
    uint32_t lc = 0, ls1 = 0, hc = 0, hs1 = 0;
    unsigned long long ls2 = 0, hs2 = 0;
    auto count = [&](uint32_t u) {
        vmin = min(vmin, u);
        vmax = max(vmax, u);
        ++ngood;
        const uint32_t d = u - w0;
        if (d < (uint32_t)NWIN) {
            atomicAdd(&win[d], 1u);
        } else if (u < w0) {
            ++lc; ls1 += u; ls2 += (unsigned long long)u * u;
        } else {
            ++hc; hs1 += u; hs2 += (unsigned long long)u * u;
        }
    };
    const int nchunks = cpr * bh;
    if (vec) {
        // 16-byte chunks (8 values); a thread's (row, chunk) advance by the
        // fixed step of one pass of the CTA, without a division per chunk.
        // Both values of a 32-bit word inside the window (the common case)
        // cost a subtraction and a shared atomic each; the rest go through
        // count().  The range of the window's values comes from the
        // histogram afterwards, so only values outside it update vmin/vmax.
        constexpr int U = 4;
        const int dr = WB_NT / cpr, dc = WB_NT - dr * cpr;
        int ry = tid / cpr, rc = tid - ry * cpr;
        while (ry < bh) {
            uint4 q[U];
            int nq = 0;
#pragma unroll
            for (int kk = 0; kk < U; ++kk) {
                if (ry < bh) {
                    q[kk] = __ldg(reinterpret_cast<const uint4*>(img + (int64_t)(y0 + ry) * pitch + x0 + rc * 8));
                    ++nq;
                }
                rc += dc;
                ry += dr;
                if (rc >= cpr) { rc -= cpr; ++ry; }
            }
#pragma unroll
            for (int kk = 0; kk < U; ++kk) {
                if (kk >= nq) break;
                const uint32_t w4[4] = {q[kk].x, q[kk].y, q[kk].z, q[kk].w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const uint32_t u0 = w4[e] & 0xffffu, u1 = w4[e] >> 16;
                    const uint32_t d0 = u0 - w0, d1 = u1 - w0;
                    if ((d0 | d1) < (uint32_t)NWIN) {          // NWIN is a power of two
                        atomicAdd(&win[d0], 1u);
                        atomicAdd(&win[d1], 1u);
                    } else {
                        count(u0);
                        count(u1);
                        ngood -= 2u;                           // counted per chunk below
                    }
                }
                ngood += 8u;
            }
        }
        __syncthreads();
        // the smallest and largest value held in the window
        for (int w = tid; w < NWIN; w += WB_NT)
            if (win[w]) {
                vmin = min(vmin, w0 + (uint32_t)w);
                vmax = max(vmax, w0 + (uint32_t)w);
            }
    } else {
        for (int c = tid; c < nchunks; c += WB_NT) {
            const int ry = c / cpr, rc = c - ry * cpr;
            const int y = y0 + ry, xs = x0 + rc * 8;
            const uint16_t* row = img + (int64_t)y * pitch;
            const int nv = min(8, x1 - xs);
            for (int e = 0; e < nv; ++e) {
                if (mask && mask[(int64_t)y * W + xs + e]) continue;
                count(__ldg(row + xs + e));
            }
        }
    }
    unsigned long long agg[6] = {lc, ls1, ls2, hc, hs1, hs2};
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        vmin = min(vmin, __shfl_xor_sync(0xffffffffu, vmin, o));
        vmax = max(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
        ngood += __shfl_xor_sync(0xffffffffu, ngood, o);
#pragma unroll
        for (int j = 0; j < 6; ++j) agg[j] += __shfl_xor_sync(0xffffffffu, agg[j], o);
    }
    if (lane == 0) {
        red_min[warp] = vmin; red_max[warp] = vmax; red_n[warp] = ngood;
#pragma unroll
        for (int j = 0; j < 6; ++j) red64[j][warp] = agg[j];
    }
    __syncthreads();
    vmin = 0xffffffffu; vmax = 0u; ngood = 0u;
#pragma unroll
    for (int j = 0; j < 6; ++j) agg[j] = 0;
    for (int w = 0; w < WB_NT / 32; ++w) {
        vmin = min(vmin, red_min[w]); vmax = max(vmax, red_max[w]); ngood += red_n[w];
#pragma unroll
        for (int j = 0; j < 6; ++j) agg[j] += red64[j][w];
    }
    const bool valid = ngood > 0 && 2u * ngood >= (uint32_t)(bw * bh);
    if (ngood == 0 || vmin == vmax) {
        // empty or constant box: statistics are immediate (as in the full kernel)
        if (tid == 0) {
            double med = ngood ? (double)vmin : 0.0;
            double b, r;
            box_result(med, med, 0.0, &b, &r);
            A.bkg[box] = valid ? b : 0.0;
            A.rms[box] = valid ? r : 0.0;
            A.valid[box] = valid;
            if (A.quant)
                for (int q = 0; q < 5; ++q) A.quant[(int64_t)q * nbox + box] = (float)med;
        }
        return;
    }

    // ---- coarse summaries of the window (64 bins of 64 values).  Within a
    // coarse bin the count n, sum n d and sum n d^2 of the offsets d < 64
    // from its first value fit 32 bits (n <= 65,536); the sums of v and v^2
    // follow from them exactly in 64 bits.
    for (int cb = warp; cb < NWC; cb += WB_NT / 32) {
        uint32_t c = 0, d1 = 0, d2 = 0;
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const uint32_t d = 2u * lane + e, nb = win[cb * WCB + d];
            c += nb; d1 += nb * d; d2 += nb * d * d;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            c += __shfl_xor_sync(0xffffffffu, c, o);
            d1 += __shfl_xor_sync(0xffffffffu, d1, o);
            d2 += __shfl_xor_sync(0xffffffffu, d2, o);
        }
        if (lane == 0) {
            const unsigned long long base = w0 + (uint32_t)cb * WCB;
            cc_s[cb] = c;
            cs1_s[cb] = base * c + d1;
            cs2_s[cb] = base * base * c + 2ull * base * d1 + d2;
        }
    }
    __syncthreads();
    if (warp != 0) return;
    {
        // prefixes over the coarse bins, starting from the values below the window
        unsigned long long c[2], s1[2], s2[2], tc = 0, t1 = 0, t2 = 0;
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            c[e] = cc_s[2 * lane + e]; s1[e] = cs1_s[2 * lane + e]; s2[e] = cs2_s[2 * lane + e];
            tc += c[e]; t1 += s1[e]; t2 += s2[e];
        }
        unsigned long long ic = tc, i1 = t1, i2 = t2;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long a0 = __shfl_up_sync(0xffffffffu, ic, o);
            const unsigned long long a1 = __shfl_up_sync(0xffffffffu, i1, o);
            const unsigned long long a2 = __shfl_up_sync(0xffffffffu, i2, o);
            if (lane >= o) { ic += a0; i1 += a1; i2 += a2; }
        }
        unsigned long long ec = agg[0] + ic - tc, e1 = agg[1] + i1 - t1, e2 = agg[2] + i2 - t2;
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            pc[2 * lane + e] = ec; ps1[2 * lane + e] = e1; ps2[2 * lane + e] = e2;
            ec += c[e]; e1 += s1[e]; e2 += s2[e];
        }
        if (lane == 31) { pc[NWC] = ec; ps1[NWC] = e1; ps2[NWC] = e2; }
    }
    __syncwarp();
    WinHist wq;
    wq.win = win; wq.pc = pc; wq.ps1 = ps1; wq.ps2 = ps2;
    wq.w0 = w0; wq.vmin = vmin; wq.vmax = vmax;
    wq.tc = pc[NWC] + agg[3]; wq.ts1 = ps1[NWC] + agg[4]; wq.ts2 = ps2[NWC] + agg[5];
    double med, mean, sd;
    clip_histogram(wq, vmin, vmax, A.k, A.maxiter, &med, &mean, &sd);
    float qv[5];
    if (A.quant && !wq.failed) {
        const float qs[5] = {0.10f, 0.25f, 0.50f, 0.75f, 0.90f};
        for (int q = 0; q < 5; ++q) qv[q] = (float)wq.select(quantile_rank(qs[q], ngood));
    }
    if (lane != 0) return;
    if (wq.failed) {
        A.fb_list[atomicAdd(A.fb_count, 1)] = box;
        return;
    }
    if (A.quant)
        for (int q = 0; q < 5; ++q) A.quant[(int64_t)q * nbox + box] = qv[q];
    double bb, rr;
    box_result(med, mean, sd, &bb, &rr);
    A.bkg[box] = valid ? bb : 0.0;
    A.rms[box] = valid ? rr : 0.0;
    A.valid[box] = valid;
}

// ============================================================ float32 box ===
constexpr int F32_NT = 512;

__device__ __forceinline__ DF block_df_sum(DF v, DF* red)
{
    v = df_warp_sum(v);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    DF t = lane < (int)(blockDim.x >> 5) ? red[lane] : df_zero();
    t = df_warp_sum(t);
    return t;
}

// first index in [lo, hi) with (double)v[i] >= x (v ascending)
__device__ __forceinline__ int lower_bound_d(const float* v, int lo, int hi, double x)
{
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if ((double)v[mid] < x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// first index in [lo, hi) with (double)v[i] > x
__device__ __forceinline__ int upper_bound_d(const float* v, int lo, int hi, double x)
{
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if ((double)v[mid] <= x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__global__ void __launch_bounds__(F32_NT) k_boxstats_f32(const BoxArgs* __restrict__ batch, const __grid_constant__ BoxArgs one)
{
    const BoxArgs& A = frame_args(batch, one);
    if ((int)blockIdx.x >= A.nbox) return;
    const float* __restrict__ img = static_cast<const float*>(A.img);
    const int64_t pitch = A.pitch;
    const uint8_t* __restrict__ mask = A.mask;
    const int W = A.W, H = A.H, B = A.B, Mx = A.Mx, nbox = A.nbox, npad = A.npad;
    const double k = A.k;
    const int maxiter = A.maxiter;
    double* __restrict__ bkg_out = A.bkg;
    double* __restrict__ rms_out = A.rms;
    int* __restrict__ valid_out = A.valid;
    float* __restrict__ quant_out = A.quant;
    extern __shared__ float vals[];                 // npad
    __shared__ int ngood_s;
    __shared__ DF red[32];
    const int box = blockIdx.x;
    const int bi = box % Mx, bj = box / Mx;
    const int x0 = bi * B, x1 = min(x0 + B, W);
    const int y0 = bj * B, y1 = min(y0 + B, H);
    const int bw = x1 - x0, bh = y1 - y0;
    const int tid = threadIdx.x;
    if (tid == 0) ngood_s = 0;
    __syncthreads();
    for (int p = tid; p < bw * bh; p += F32_NT) {
        int y = y0 + p / bw, x = x0 + p % bw;
        float v = __ldg(img + (int64_t)y * pitch + x);
        bool bad = !isfinite(v) || (mask && mask[(int64_t)y * W + x]);
        if (!bad) vals[atomicAdd(&ngood_s, 1)] = v;
    }
    __syncthreads();
    const int ng = ngood_s;
    for (int p = ng + tid; p < npad; p += F32_NT) vals[p] = INFINITY;
    __syncthreads();
    // bitonic sort, ascending
    for (int size = 2; size <= npad; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = tid; i < npad / 2; i += F32_NT) {
                int lo = 2 * i - (i & (stride - 1));
                int hi = lo + stride;
                bool up = ((lo & size) == 0);
                float a = vals[lo], b = vals[hi];
                if ((a > b) == up) { vals[lo] = b; vals[hi] = a; }
            }
            __syncthreads();
        }
    const bool valid = ng > 0 && 2 * ng >= bw * bh;
    if (ng == 0) {
        if (tid == 0) { bkg_out[box] = 0; rms_out[box] = 0; valid_out[box] = 0; }
        if (quant_out && tid < 5) quant_out[(int64_t)tid * nbox + box] = 0.f;
        return;
    }
    int lo = 0, hi = ng;
    double med = 0, mean = 0, sd = 0;
    for (int it = 0;; ++it) {
        int n = hi - lo;
        med = (n & 1) ? (double)vals[lo + n / 2] : 0.5 * ((double)vals[lo + n / 2 - 1] + (double)vals[lo + n / 2]);
        DF s = df_zero();
        for (int i = lo + tid; i < hi; i += F32_NT) df_add(s, vals[i]);
        s = block_df_sum(s, red);
        double S = df_value(s);
        mean = S / (double)n;
        float mh = (float)mean;
        float ml = (float)(mean - (double)mh);
        DF q = df_zero();
        for (int i = lo + tid; i < hi; i += F32_NT) {
            float d = (vals[i] - mh) - ml;
            df_add_prod(q, d, d);
        }
        q = block_df_sum(q, red);
        sd = sqrt(fmax(df_value(q), 0.0) / (double)n);
        if (it >= maxiter) break;
        double flo = med - k * sd, fhi = med + k * sd;
        int nlo = lower_bound_d(vals, lo, hi, flo);
        int nhi = upper_bound_d(vals, lo, hi, fhi);
        if (nhi - nlo == n) break;
        lo = nlo; hi = nhi;
    }
    if (tid == 0) {
        double bb, rr;
        box_result(med, mean, sd, &bb, &rr);
        bkg_out[box] = valid ? bb : 0.0;
        rms_out[box] = valid ? rr : 0.0;
        valid_out[box] = valid;
    }
    if (quant_out && tid < 5) {
        const float qs[5] = {0.10f, 0.25f, 0.50f, 0.75f, 0.90f};
        int r = (int)floor((double)qs[tid] * (double)(ng - 1) + 0.5);
        quant_out[(int64_t)tid * nbox + box] = vals[r];
    }
}

// ====================================================== mesh finalisation ===
constexpr int MF_NT = 1024;

// Fill boxes with < 50 % good pixels from the mean of their valid
// 8-neighbours (sweep after sweep), then median-filter both meshes over a
// fsize x fsize window clipped at the mesh edge.  One CTA.
__global__ void __launch_bounds__(MF_NT)
k_mesh_finalize(double* bkg, double* rms, int* valid, double* tmp_b, double* tmp_r, int* tmp_v,
                int Mx, int My, int fsize, float* bkg_out, float* rms_out)
{
    __shared__ int missing, any;
    const int nb = Mx * My, tid = threadIdx.x;
    if (tid == 0) any = 0;
    __syncthreads();
    for (int b = tid; b < nb; b += MF_NT)
        if (valid[b]) any = 1;
    __syncthreads();
    if (!any) {
        for (int b = tid; b < nb; b += MF_NT) { bkg[b] = 0; rms[b] = 0; valid[b] = 1; }
        __syncthreads();
    }
    for (int sweep = 0; sweep < Mx + My + 2; ++sweep) {
        if (tid == 0) missing = 0;
        __syncthreads();
        for (int b = tid; b < nb; b += MF_NT) {
            tmp_b[b] = bkg[b]; tmp_r[b] = rms[b]; tmp_v[b] = valid[b];
            if (valid[b]) continue;
            int i = b % Mx, j = b / Mx, c = 0;
            double sb = 0, sr = 0;
            for (int dj = -1; dj <= 1; ++dj)
                for (int di = -1; di <= 1; ++di) {
                    int ii = i + di, jj = j + dj;
                    if ((di || dj) && ii >= 0 && ii < Mx && jj >= 0 && jj < My && valid[jj * Mx + ii]) {
                        sb += bkg[jj * Mx + ii];
                        sr += rms[jj * Mx + ii];
                        ++c;
                    }
                }
            if (c) { tmp_b[b] = sb / c; tmp_r[b] = sr / c; tmp_v[b] = 1; }
            else missing = 1;
        }
        __syncthreads();
        for (int b = tid; b < nb; b += MF_NT) { bkg[b] = tmp_b[b]; rms[b] = tmp_r[b]; valid[b] = tmp_v[b]; }
        __syncthreads();
        if (!missing) break;
    }
    const int h = fsize / 2;
    for (int b = tid; b < nb; b += MF_NT) {
        int i = b % Mx, j = b / Mx;
        for (int map = 0; map < 2; ++map) {
            const double* src = map ? rms : bkg;
            double win[49];
            int c = 0;
            for (int jj = j - h; jj <= j + h; ++jj)
                for (int ii = i - h; ii <= i + h; ++ii)
                    if (ii >= 0 && ii < Mx && jj >= 0 && jj < My) {
                        double v = src[jj * Mx + ii];
                        int p = c++;
                        while (p > 0 && win[p - 1] > v) { win[p] = win[p - 1]; --p; }
                        win[p] = v;
                    }
            double med = (c & 1) ? win[c / 2] : 0.5 * (win[c / 2 - 1] + win[c / 2]);
            (map ? rms_out : bkg_out)[b] = (float)med;
        }
    }
}

// ============================================================ spline tables ===
// natural-spline second derivatives along a line of n nodes (positions from
// the axis) for values v (stride vs), written to M (stride ms); d, c are
// scratch of n doubles.  Thomas algorithm on the interior nodes.
__device__ void spline_line(const Axis& ax, const double* v, int vs, double* M, int ms, double* c, double* d)
{
    const int n = ax.n;
    for (int i = 0; i < n; ++i) M[i * ms] = 0.0;
    if (n < 3) return;
    auto pos = [&](int i) -> double {
        return (i == n - 1) ? (double)ax.tl : (double)ax.t0 + (double)i * (double)ax.B;
    };
    // rows r = 1 .. n-2: h0 M[r-1] + 2 (h0 + h1) M[r] + h1 M[r+1] = rhs
    double bprev = 0, cprev = 0, dprev = 0;
    for (int r = 1; r <= n - 2; ++r) {
        double h0 = pos(r) - pos(r - 1), h1 = pos(r + 1) - pos(r);
        double a = h0, b = 2.0 * (h0 + h1), cc = h1;
        double rhs = 6.0 * ((v[(r + 1) * vs] - v[r * vs]) / h1 - (v[r * vs] - v[(r - 1) * vs]) / h0);
        if (r > 1) {
            double w = a / bprev;
            b -= w * cprev;
            rhs -= w * dprev;
        }
        c[r] = cc; d[r] = rhs;
        bprev = b; cprev = cc; dprev = rhs;
        M[r * ms] = b;   // keep the pivot temporarily
    }
    // back substitution
    double next = 0.0;
    for (int r = n - 2; r >= 1; --r) {
        double piv = M[r * ms];
        double val = (d[r] - c[r] * next) / piv;
        M[r * ms] = val;
        next = val;
    }
}

// X: along each mesh row; Y: along each mesh column.  Each of the Mx + My
// lines has its own scratch line of Mx + My doubles in sc and sd.
__global__ void k_spline_xy(const float* mesh, Axis ax, Axis ay, double* vals, double* colv, double* X,
                            double* Y, double* scr_c, double* scr_d)
{
    const int Mx = ax.n, My = ay.n;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < My) {
        double* v = vals + (int64_t)t * Mx;
        for (int i = 0; i < Mx; ++i) v[i] = (double)mesh[t * Mx + i];
        spline_line(ax, v, 1, X + (int64_t)t * Mx, 1, scr_c + (int64_t)t * (Mx + My), scr_d + (int64_t)t * (Mx + My));
    }
    const int u = t - My;
    if (u >= 0 && u < Mx) {
        double* col = colv + (int64_t)u * My;
        for (int j = 0; j < My; ++j) col[j] = (double)mesh[j * Mx + u];
        spline_line(ay, col, 1, Y + u, Mx, scr_c + (int64_t)(My + u) * (Mx + My),
                    scr_d + (int64_t)(My + u) * (Mx + My));
    }
}

// XY: along each mesh row of Y; then pack (P, X, Y, XY) as float4
__global__ void k_spline_pack(const float* mesh, Axis ax, Axis ay, const double* X, double* Y, double* XY,
                              double* scr_c, double* scr_d, float4* tab)
{
    const int Mx = ax.n, My = ay.n;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= My) return;
    spline_line(ax, Y + (int64_t)t * Mx, 1, XY + (int64_t)t * Mx, 1, scr_c + (int64_t)t * (Mx + My),
                scr_d + (int64_t)t * (Mx + My));
    for (int i = 0; i < Mx; ++i) {
        int64_t o = (int64_t)t * Mx + i;
        tab[o] = make_float4(mesh[o], (float)X[o], (float)Y[o], (float)XY[o]);
    }
}

__global__ void k_bkg_maps(SplineTab sb, SplineTab sr, int W, int H, float* bmap, float* rmap)
{
    const int64_t n = (int64_t)W * H;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        float x = (float)(p % W), y = (float)(p / W);
        if (bmap) bmap[p] = spline_eval(sb, x, y);
        if (rmap) rmap[p] = spline_eval(sr, x, y);
    }
}

// ====================================================== fused mesh kernel ===
// One CTA does the whole mesh stage in shared memory when the mesh has at
// most MESH_SMEM_NODES nodes: invalid-box fill, median filter, and the
// spline tables of both maps.  The tridiagonal matrix of the natural spline
// depends only on the node positions, so each axis is factorised once
// (multipliers and reciprocal pivots) and every line is then solved with
// FMAs only.  FP32 throughout: the tables are stored in FP32 anyway, and the
// diagonally dominant spline system loses nothing that matters at 1e-5.
constexpr int MESH_SMEM_NODES = 4096;
constexpr int MA_NT = 1024;

// byte offset of the LU scratch in k_mesh_all's shared memory: six float
// arrays and two int arrays of n entries, rounded up to 16 bytes
__host__ __device__ __forceinline__ size_t mesh_lu_offset(int n)
{
    const size_t end = (size_t)n * (6 * sizeof(float) + 2 * sizeof(int));
    return (end + 15) & ~(size_t)15;
}

struct AxisLU {
    float* w;      // elimination multipliers  (index r = 1..n-2)
    float* ib;     // reciprocal pivots
    float* c;      // super-diagonal
    float* ih;     // 1 / interval width (n-1 entries)
};

__device__ __forceinline__ float node_pos(const Axis& a, int i)
{
    return (i == a.n - 1) ? a.tl : a.t0 + (float)i * a.B;
}

__device__ void factor_axis(const Axis& a, AxisLU L)
{
    const int n = a.n;
    for (int i = 0; i + 1 < n; ++i) L.ih[i] = 1.f / (node_pos(a, i + 1) - node_pos(a, i));
    float bprev = 0.f, cprev = 0.f;
    for (int r = 1; r <= n - 2; ++r) {
        const float h0 = node_pos(a, r) - node_pos(a, r - 1), h1 = node_pos(a, r + 1) - node_pos(a, r);
        float b = 2.f * (h0 + h1);
        float w = 0.f;
        if (r > 1) {
            w = h0 / bprev;
            b -= w * cprev;
        }
        L.w[r] = w;
        L.ib[r] = 1.f / b;
        L.c[r] = h1;
        bprev = b;
        cprev = h1;
    }
}

// second derivatives of one line (values v, stride vs) into M (stride ms)
__device__ void solve_line(const AxisLU& L, int n, const float* v, int vs, float* M, int ms)
{
    M[0] = 0.f;
    if (n >= 2) M[(n - 1) * ms] = 0.f;
    if (n < 3) return;
    float dprev = 0.f;
    for (int r = 1; r <= n - 2; ++r) {
        float d = 6.f * ((v[(r + 1) * vs] - v[r * vs]) * L.ih[r] - (v[r * vs] - v[(r - 1) * vs]) * L.ih[r - 1]);
        d = fmaf(-L.w[r], dprev, d);
        M[r * ms] = d;        // forward-eliminated right-hand side
        dprev = d;
    }
    float next = 0.f;
    for (int r = n - 2; r >= 1; --r) {
        const float val = fmaf(-L.c[r], next, M[r * ms]) * L.ib[r];
        M[r * ms] = val;
        next = val;
    }
}

// mode 0: raw box statistics -> fill, filter, write meshes, tables
// mode 1: tables only, from the float meshes given in bkg_out / rms_out
__global__ void __launch_bounds__(MA_NT) k_mesh_all(const MeshArgs* __restrict__ batch,
                                                    const __grid_constant__ MeshArgs one)
{
    pdl_wait();
    pdl_release();
    const MeshArgs& MA = frame_args(batch, one);
    const double* __restrict__ bkg_raw = MA.bkg_raw;
    const double* __restrict__ rms_raw = MA.rms_raw;
    const int* __restrict__ valid_raw = MA.valid;
    const Axis ax = MA.ax, ay = MA.ay;
    const int fsize = MA.fsize, mode = MA.mode;
    float* bkg_out = MA.bkg_mesh;
    float* rms_out = MA.rms_mesh;
    float4* tab_b = MA.tab_b;
    float4* tab_r = MA.tab_r;
    extern __shared__ __align__(16) float sh[];
    unsigned char* sh_bytes = reinterpret_cast<unsigned char*>(sh);
    // shared-memory rows are Ms = Mx | 1 wide (odd), so the row-direction
    // solves, one row per lane, hit 32 different banks
    const int Mx = ax.n, My = ay.n, n = Mx * My, tid = threadIdx.x;
    const int Ms = Mx | 1, ns = Ms * My;
    float* A0 = sh;
    float* A1 = A0 + ns;
    float* A2 = A1 + ns;
    float* A3 = A2 + ns;
    float* A4 = A3 + ns;
    float* A5 = A4 + ns;
    int* V0 = reinterpret_cast<int*>(A5 + ns);
    int* V1 = V0 + ns;
    const int nl = Mx > My ? Mx : My;
    // the LU scratch starts at the first 16-byte boundary after V1
    float* lu = reinterpret_cast<float*>(sh_bytes + mesh_lu_offset(ns));
    AxisLU Lx{lu, lu + nl, lu + 2 * nl, lu + 3 * nl};
    AxisLU Ly{lu + 4 * nl, lu + 5 * nl, lu + 6 * nl, lu + 7 * nl};
    __shared__ int missing, any;

    if (mode == 0) {
        if (tid == 0) any = 0;
        __syncthreads();
        for (int b = tid; b < n; b += MA_NT) {
            const int sb_ = (b / Mx) * Ms + b % Mx;
            A0[sb_] = (float)bkg_raw[b]; A1[sb_] = (float)rms_raw[b]; V0[sb_] = valid_raw[b];
            if (V0[sb_]) any = 1;
        }
        __syncthreads();
        if (!any) {
            for (int b = tid; b < n; b += MA_NT) {
                const int sb_ = (b / Mx) * Ms + b % Mx;
                A0[sb_] = 0.f; A1[sb_] = 0.f; V0[sb_] = 1;
            }
            __syncthreads();
        }
        // fill invalid boxes from valid 8-neighbours, sweep after sweep
        for (int sweep = 0; sweep < Mx + My + 2; ++sweep) {
            if (tid == 0) missing = 0;
            __syncthreads();
            for (int b = tid; b < n; b += MA_NT) {
                const int i = b % Mx, j = b / Mx, sb_ = j * Ms + i;
                A2[sb_] = A0[sb_]; A3[sb_] = A1[sb_]; V1[sb_] = V0[sb_];
                if (V0[sb_]) continue;
                int c = 0;
                float sb = 0.f, sr = 0.f;
                for (int dj = -1; dj <= 1; ++dj)
                    for (int di = -1; di <= 1; ++di) {
                        const int ii = i + di, jj = j + dj;
                        if ((di || dj) && ii >= 0 && ii < Mx && jj >= 0 && jj < My && V0[jj * Ms + ii]) {
                            sb += A0[jj * Ms + ii];
                            sr += A1[jj * Ms + ii];
                            ++c;
                        }
                    }
                if (c) { A2[sb_] = sb / c; A3[sb_] = sr / c; V1[sb_] = 1; }
                else missing = 1;
            }
            __syncthreads();
            const bool more = missing;
            for (int b = tid; b < n; b += MA_NT) {
                const int sb_ = (b / Mx) * Ms + b % Mx;
                A0[sb_] = A2[sb_]; A1[sb_] = A3[sb_]; V0[sb_] = V1[sb_];
            }
            __syncthreads();
            if (!more) break;
        }
        // median filter (window clipped at the mesh edge) -> float meshes;
        // meanwhile two threads factor the spline systems (first needed by
        // the solves further down)
        if (tid == MA_NT - 32) factor_axis(ax, Lx);
        if (tid == MA_NT - 64) factor_axis(ay, Ly);
        const int h = fsize / 2;
        for (int t = tid; t < 2 * n && fsize == 3; t += MA_NT) {
            // 3 x 3: the window in registers (absent cells +inf), sorted by
            // odd-even transposition; the same order statistics as below
            const int map = t / n, b = t - map * n;
            const int i = b % Mx, j = b / Mx;
            const float* src = map ? A1 : A0;
            float w[9];
            int c = 0;
#pragma unroll
            for (int dj = -1; dj <= 1; ++dj)
#pragma unroll
                for (int di = -1; di <= 1; ++di) {
                    const int ii = i + di, jj = j + dj;
                    const bool in = ii >= 0 && ii < Mx && jj >= 0 && jj < My;
                    w[(dj + 1) * 3 + di + 1] = in ? src[jj * Ms + ii] : INFINITY;
                    c += in ? 1 : 0;
                }
#pragma unroll
            for (int pass = 0; pass < 9; ++pass)
#pragma unroll
                for (int q = pass & 1; q + 1 < 9; q += 2) {
                    const float lo = fminf(w[q], w[q + 1]), hi = fmaxf(w[q], w[q + 1]);
                    w[q] = lo;
                    w[q + 1] = hi;
                }
            float m0 = w[0], m1 = w[0];
#pragma unroll
            for (int q = 1; q < 9; ++q) {
                if (q == (c - 1) / 2) m0 = w[q];
                if (q == c / 2) m1 = w[q];
            }
            (map ? rms_out : bkg_out)[b] = (c & 1) ? m1 : 0.5f * (m0 + m1);
        }
        for (int t = tid; t < 2 * n && fsize != 3; t += MA_NT) {
            const int map = t / n, b = t - map * n;
            const int i = b % Mx, j = b / Mx;
            const float* src = map ? A1 : A0;
            float win[49];
            int c = 0;
            for (int jj = j - h; jj <= j + h; ++jj)
                for (int ii = i - h; ii <= i + h; ++ii)
                    if (ii >= 0 && ii < Mx && jj >= 0 && jj < My) {
                        const float v = src[jj * Ms + ii];
                        int p = c++;
                        while (p > 0 && win[p - 1] > v) { win[p] = win[p - 1]; --p; }
                        win[p] = v;
                    }
            const float med = (c & 1) ? win[c / 2] : 0.5f * (win[c / 2 - 1] + win[c / 2]);
            (map ? rms_out : bkg_out)[b] = med;
        }
    }
    __syncthreads();
    // spline tables of both maps, from the float meshes: X (rows) and Y
    // (columns) for both maps at once, then XY (rows of Y)
    if (mode != 0) {
        if (tid == 0) factor_axis(ax, Lx);
        if (tid == 32) factor_axis(ay, Ly);
    }
    for (int b = tid; b < n; b += MA_NT) {
        const int sb_ = (b / Mx) * Ms + b % Mx;
        A4[sb_] = bkg_out[b]; A5[sb_] = rms_out[b];
    }
    __syncthreads();
    for (int t = tid; t < 2 * (My + Mx); t += MA_NT) {
        const int map = t / (My + Mx), q = t - map * (My + Mx);
        const float* P = map ? A5 : A4;
        float* X = map ? A1 : A0;
        float* Y = map ? A3 : A2;
        if (q < My) solve_line(Lx, Mx, P + q * Ms, 1, X + q * Ms, 1);
        else solve_line(Ly, My, P + (q - My), Ms, Y + (q - My), Ms);
    }
    __syncthreads();
    // XY overwrites P (no longer needed once X and Y are known)
    for (int b = tid; b < n; b += MA_NT) {
        const int sb_ = (b / Mx) * Ms + b % Mx;
        tab_b[b] = make_float4(A4[sb_], A0[sb_], A2[sb_], 0.f);
        tab_r[b] = make_float4(A5[sb_], A1[sb_], A3[sb_], 0.f);
    }
    __syncthreads();
    for (int t = tid; t < 2 * My; t += MA_NT) {
        const int map = t / My, q = t - map * My;
        solve_line(Lx, Mx, (map ? A3 : A2) + q * Ms, 1, (map ? A5 : A4) + q * Ms, 1);
    }
    __syncthreads();
    for (int b = tid; b < n; b += MA_NT) {
        const int sb_ = (b / Mx) * Ms + b % Mx;
        tab_b[b].w = A4[sb_];
        tab_r[b].w = A5[sb_];
    }
}

size_t mesh_all_smem(int Mx, int My)
{
    const size_t ns = (size_t)(Mx | 1) * My;     // odd row stride (see k_mesh_all)
    const size_t nl = Mx > My ? Mx : My;
    return mesh_lu_offset((int)ns) + 8 * nl * sizeof(float);
}

bool mesh_fits_smem(int Mx, int My)
{
    return (size_t)Mx * My <= (size_t)MESH_SMEM_NODES && mesh_all_smem(Mx, My) <= 220 * 1024;
}

MeshArgs mesh_args(const double* bkg_raw, const double* rms_raw, const int* valid, Axis ax, Axis ay, int fsize,
                   int mode, float* bkg_mesh, float* rms_mesh, float4* tab_b, float4* tab_r)
{
    MeshArgs a;
    a.bkg_raw = bkg_raw; a.rms_raw = rms_raw; a.valid = valid;
    a.ax = ax; a.ay = ay; a.fsize = fsize; a.mode = mode;
    a.bkg_mesh = bkg_mesh; a.rms_mesh = rms_mesh; a.tab_b = tab_b; a.tab_r = tab_r;
    return a;
}

// smem = the largest frame's mesh_all_smem
cudaError_t launch_mesh_all_any(const MeshArgs& one, const MeshArgs* batch, int nframes, size_t smem, cudaStream_t st)
{
    cudaFuncSetAttribute(k_mesh_all, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    launch_dep(k_mesh_all, dim3(1, nframes), dim3(MA_NT), smem, st, batch, one);
    return cudaGetLastError();
}

cudaError_t launch_mesh_all(const double* bkg_raw, const double* rms_raw, const int* valid, Axis ax, Axis ay,
                            int fsize, int mode, float* bkg_mesh, float* rms_mesh, float4* tab_b, float4* tab_r,
                            cudaStream_t st)
{
    const MeshArgs a = mesh_args(bkg_raw, rms_raw, valid, ax, ay, fsize, mode, bkg_mesh, rms_mesh, tab_b, tab_r);
    return launch_mesh_all_any(a, nullptr, 1, mesh_all_smem(ax.n, ay.n), st);
}

// --------------------------------------------------------------- launchers ---
BoxArgs box_args(const Image& im, int B, double k, int maxiter, double* bkg, double* rms, int* valid, float* quant)
{
    BoxArgs a;
    a.img = im.data; a.pitch = im.pitch; a.mask = im.mask;
    a.W = im.W; a.H = im.H; a.B = B;
    a.Mx = (im.W + B - 1) / B;
    a.nbox = a.Mx * ((im.H + B - 1) / B);
    int npad = 1;
    while (npad < B * B) npad <<= 1;
    a.npad = npad;
    a.k = k; a.maxiter = maxiter;
    a.bkg = bkg; a.rms = rms; a.valid = valid; a.quant = quant;
    a.fb_list = nullptr; a.fb_count = nullptr;
    return a;
}

// one frame (batch == nullptr) or nframes frames whose arguments are in the
// device array batch; maxbox = the largest frame's box count
cudaError_t launch_boxstats_any(const BoxArgs& one, const BoxArgs* batch, int nframes, int maxbox, int is_f32,
                                cudaStream_t st)
{
    dim3 grid(maxbox, nframes);
    if (!is_f32 && one.fb_list) {
        // windowed histograms, then the full histogram for the boxes they
        // could not finish (a persistent grid over the fallback lists)
        launch_dep(k_boxstats_win, grid, dim3(WB_NT), 0, st, batch, one);
        const size_t smem = U16_WORDS * sizeof(uint32_t);
        cudaFuncSetAttribute(k_boxstats_u16, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        launch_dep(k_boxstats_u16, dim3(maxbox < 152 ? maxbox : 152, nframes), dim3(U16_NT), smem, st, batch, one);
        return cudaGetLastError();
    }
    if (!is_f32) {
        const size_t smem = U16_WORDS * sizeof(uint32_t);
        cudaFuncSetAttribute(k_boxstats_u16, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_boxstats_u16<<<grid, U16_NT, smem, st>>>(batch, one);
    } else {
        const size_t smem = (size_t)(batch ? 16384 : one.npad) * sizeof(float);
        cudaFuncSetAttribute(k_boxstats_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_boxstats_f32<<<grid, F32_NT, smem, st>>>(batch, one);
    }
    return cudaGetLastError();
}

cudaError_t launch_boxstats(const Image& im, int B, double k, int maxiter, double* bkg, double* rms, int* valid,
                            float* quant, cudaStream_t st)
{
    const BoxArgs a = box_args(im, B, k, maxiter, bkg, rms, valid, quant);
    return launch_boxstats_any(a, nullptr, 1, a.nbox, im.is_f32, st);
}

cudaError_t launch_mesh_finalize(double* bkg, double* rms, int* valid, double* tmp_b, double* tmp_r, int* tmp_v,
                                 int Mx, int My, int fsize, float* bkg_out, float* rms_out, cudaStream_t st)
{
    k_mesh_finalize<<<1, MF_NT, 0, st>>>(bkg, rms, valid, tmp_b, tmp_r, tmp_v, Mx, My, fsize, bkg_out, rms_out);
    return cudaGetLastError();
}

cudaError_t launch_spline_tables(const float* mesh, Axis ax, Axis ay, double* scratch, float4* tab, cudaStream_t st)
{
    const int Mx = ax.n, My = ay.n;
    const int64_t nn = (int64_t)Mx * My;
    double* vals = scratch;
    double* colv = vals + nn;
    double* X = colv + nn;
    double* Y = X + nn;
    double* XY = Y + nn;
    double* sc = XY + nn;
    double* sd = sc + (int64_t)(Mx + My) * (Mx + My);
    const int nt = Mx + My;
    k_spline_xy<<<(nt + 127) / 128, 128, 0, st>>>(mesh, ax, ay, vals, colv, X, Y, sc, sd);
    k_spline_pack<<<(My + 127) / 128, 128, 0, st>>>(mesh, ax, ay, X, Y, XY, sc, sd, tab);
    return cudaGetLastError();
}

size_t spline_scratch_doubles(int Mx, int My)
{
    return (size_t)5 * Mx * My + (size_t)2 * (Mx + My) * (Mx + My);
}

cudaError_t launch_bkg_maps(const SplineTab& sb, const SplineTab& sr, int W, int H, float* bmap, float* rmap,
                            cudaStream_t st)
{
    int64_t n = (int64_t)W * H;
    int64_t nb_ = (n + 255) / 256;
    int blocks = (int)(nb_ < 152 * 16 ? nb_ : 152 * 16);
    k_bkg_maps<<<blocks, 256, 0, st>>>(sb, sr, W, H, bmap, rmap);
    return cudaGetLastError();
}

}  // namespace gp
