// k_psf.cu -- the second detection pass with a spatially varying PSF (paper
// Section 3.2): the local PSF is a reference P0 plus K eigenmodes e_k with
// coefficient maps c_k, and the matched filter splits into K + 1
// correlations,
//     S(p) = (P0 (x) m)(p) + sum_k c_k(p) (e_k (x) m)(p),
// m = I - B (bad pixels 0, mirror border), c_k the natural spline through
// per-tile coefficients; foreground where S > k sigma(p).  The pass writes
// what the streaming threshold pass writes (packed mask, the map with m at
// foreground pixels and 0 elsewhere, the list of tiles holding foreground),
// so the labelling, merge and moments that follow are the plain path's.
//
// A CTA takes one 128-column strip and one 32-row tile band.  m over the band
// and a halo of KS/2 is formed in shared memory (B from per-row and
// per-column spline coefficients); a thread takes one column and 8 rows and
// correlates them with two kernels at a time: per tap column it loads the
// 8 + KS - 1 values of its column once and applies the KS tap pairs of that
// column to its 8 rows with paired FMAs (each half rounds as one fmaf, so the
// results do not depend on the pairing).  The taps (zero-padded to KS x KS,
// centred) are kernel parameters.
#include <math.h>
#include <string.h>

#include "gp_internal.cuh"
#include "gp_launch.h"

namespace gp {

constexpr int PS_ROWS = TY;                 // rows of a CTA: one tile band
constexpr int PS_COLS = ST_STRIP;           // columns: one mask strip (two tiles)
constexpr int PS_RPT = 8;                   // rows per thread
constexpr int PS_NT = PS_COLS * (PS_ROWS / PS_RPT);   // 512 threads

// two FMAs with one rounding each, in one instruction (Blackwell's paired
// FP32 path): the lanes of a pair are independent, so the results are those
// of two fmaf
__device__ __forceinline__ float2 psf_ffma2(float2 a, float2 b, float2 c)
{
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;"
        : "=l"(d)
        : "l"(*reinterpret_cast<unsigned long long*>(&a)), "l"(*reinterpret_cast<unsigned long long*>(&b)),
          "l"(*reinterpret_cast<unsigned long long*>(&c)));
    return *reinterpret_cast<float2*>(&d);
}

constexpr int PS_NPAIR = (GP_PSF_MAX_MODES + 2) / 2;   // kernel pairs (P0 and the modes, a zero kernel last if odd)

struct PsfArgs {
    Image im;
    SplineTab sb, sr;
    SplineTab ct[GP_PSF_MAX_MODES];         // coefficient maps
    int nk;                                 // number of modes
    float thresh;
    uint32_t* seg;
    uint4* bits;
    int nstrip;
    int* tl_list;
    int* tl_count;
    Tiles T;
    float2 taps[PS_NPAIR][KMAX];             // kernels 2p and 2p + 1 of P0, then the modes, each KS x KS
};

template <bool F32, int KS>
__global__ void __launch_bounds__(PS_NT) k_psf(const __grid_constant__ PsfArgs A)
{
    constexpr int H = KS / 2, SR = PS_ROWS + KS - 1, SC = PS_COLS + KS - 1;
    constexpr int UNROLL_U = KS <= 5 ? KS : 1;     // tap columns unrolled for small kernels only (registers)
    __shared__ float ms[SR][SC];
    __shared__ float4 rowc[SR];            // b, c0, c1 of the background y-spline of each staged row
    __shared__ int2 rowj[SR];
    __shared__ float4 colc[SC];            // and of the x-spline of each staged column
    __shared__ int2 colj[SC];
    __shared__ uint8_t bads[PS_ROWS][PS_COLS];
    __shared__ uint32_t mbits[PS_ROWS][4];
    __shared__ int anyfg[2];
    const Image& im = A.im;
    const int W = im.W, Hf = im.H;
    const int X0 = blockIdx.x * PS_COLS, Y0 = blockIdx.y * PS_ROWS;
    const int t = threadIdx.x;
    for (int r = t; r < SR; r += PS_NT) {
        const AxCoef cy = axis_coef(A.sb.ay, (float)mirror_idx(Y0 - H + r, Hf));
        rowc[r] = make_float4(cy.b, cy.c0, cy.c1, 0.f);
        rowj[r] = make_int2(cy.i, cy.i1);
    }
    for (int c = t; c < SC; c += PS_NT) {
        const AxCoef cx = axis_coef(A.sb.ax, (float)mirror_idx(X0 - H + c, W));
        colc[c] = make_float4(cx.b, cx.c0, cx.c1, 0.f);
        colj[c] = make_int2(cx.i, cx.i1);
    }
    if (t < PS_ROWS * 4) mbits[t >> 2][t & 3] = 0u;
    if (t < 2) anyfg[t] = 0;
    __syncthreads();
    // ---- m over the band and its halo, one pixel per thread at a time
    // (consecutive threads take consecutive columns)
    for (int p = t; p < SR * SC; p += PS_NT) {
        const int r = p / SC, c = p - r * SC;
        const int x = mirror_idx(X0 - H + c, W), y = mirror_idx(Y0 - H + r, Hf);
        const float4 cc = colc[c], rc = rowc[r];
        const int2 jx = colj[c], jy = rowj[r];
        AxCoef cx, cy;
        cx.i = jx.x; cx.i1 = jx.y; cx.b = cc.x; cx.c0 = cc.y; cx.c1 = cc.z;
        cy.i = jy.x; cy.i1 = jy.y; cy.b = rc.x; cy.c0 = rc.y; cy.c1 = rc.z;
        const float2 b0 = row_eval(A.sb, cy.i, cx), b1 = row_eval(A.sb, cy.i1, cx);
        bool bad;
        const float v = load_px<F32>(im, x, y, bad);
        ms[r][c] = bad ? 0.f : v - axis_combine(cy, b0.x, b1.x, b0.y, b1.y);
        const int ri = r - H, ci = c - H;
        if (ri >= 0 && ri < PS_ROWS && ci >= 0 && ci < PS_COLS) bads[ri][ci] = bad ? 1 : 0;
    }
    __syncthreads();
    // ---- the K + 1 correlations of this thread's column and rows
    const int col = t % PS_COLS, r0 = (t / PS_COLS) * PS_RPT;
    const int x = X0 + col;
    const bool xin = x < W;
    const int xq = xin ? x : W - 1;
    float S[PS_RPT];
#pragma unroll
    for (int r = 0; r < PS_RPT; ++r) S[r] = 0.f;
    const int npair = (A.nk + 2) / 2;
    for (int pr = 0; pr < npair; ++pr) {
        // kernels 2 pr and 2 pr + 1 together: one paired FMA per tap and row
        float2 F2[PS_RPT];
#pragma unroll
        for (int r = 0; r < PS_RPT; ++r) F2[r] = make_float2(0.f, 0.f);
#pragma unroll UNROLL_U
        for (int u = 0; u < KS; ++u) {
            float2 w[PS_RPT + KS - 1];
#pragma unroll
            for (int q = 0; q < PS_RPT + KS - 1; ++q) {
                const float a = ms[r0 + q][col + u];
                w[q] = make_float2(a, a);
            }
#pragma unroll
            for (int v = 0; v < KS; ++v) {
                const float2 tap = A.taps[pr][v * KS + u];
#pragma unroll
                for (int r = 0; r < PS_RPT; ++r) F2[r] = psf_ffma2(tap, w[r + v], F2[r]);
            }
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int k = 2 * pr + h;
            if (k > A.nk) break;
            float F[PS_RPT];
#pragma unroll
            for (int r = 0; r < PS_RPT; ++r) F[r] = h ? F2[r].y : F2[r].x;
            if (k == 0) {
#pragma unroll
                for (int r = 0; r < PS_RPT; ++r) S[r] = F[r];
            } else {
                const SplineTab& ct = A.ct[k - 1];
                const AxCoef cx = axis_coef(ct.ax, (float)xq);
                int jc = -1;
                float u0 = 0.f, u1 = 0.f, w0 = 0.f, w1 = 0.f;
#pragma unroll
                for (int r = 0; r < PS_RPT; ++r) {
                    const int y = min(Y0 + r0 + r, Hf - 1);
                    const AxCoef cy = axis_coef(ct.ay, (float)y);
                    if (cy.i != jc) {
                        const float2 a0 = row_eval(ct, cy.i, cx), a1 = row_eval(ct, cy.i1, cx);
                        u0 = a0.x; w0 = a0.y; u1 = a1.x; w1 = a1.y;
                        jc = cy.i;
                    }
                    S[r] = fmaf(axis_combine(cy, u0, u1, w0, w1), F[r], S[r]);
                }
            }
        }
    }
    // ---- threshold, map, mask bits
    const AxCoef sx = axis_coef(A.sr.ax, (float)xq);
    uint32_t* srow = A.seg;
#pragma unroll
    for (int r = 0; r < PS_RPT; ++r) {
        const int y = Y0 + r0 + r;
        if (!xin || y >= Hf) continue;
        const AxCoef sy = axis_coef(A.sr.ay, (float)y);
        const float2 q0 = row_eval(A.sr, sy.i, sx), q1 = row_eval(A.sr, sy.i1, sx);
        const float kt = A.thresh * axis_combine(sy, q0.x, q1.x, q0.y, q1.y);
        const bool fg = !bads[r0 + r][col] && S[r] > kt;
        const float mv = ms[r0 + r + H][col + H];
        srow[(int64_t)y * W + x] = fg ? __float_as_uint(mv) : 0u;
        if (fg) {
            atomicOr(&mbits[r0 + r][col & 3], 1u << (col >> 2));
            anyfg[col >> 6] = 1;
        }
    }
    __syncthreads();
    const int strip = blockIdx.x;
    if (t < PS_ROWS && Y0 + t < Hf)
        A.bits[(int64_t)(Y0 + t) * A.nstrip + strip] = make_uint4(mbits[t][0], mbits[t][1], mbits[t][2], mbits[t][3]);
    if (t < 2) {
        const int tcol = 2 * strip + t;
        if (tcol < A.T.ntx) {
            const int tile = blockIdx.y * A.T.ntx + tcol;
            if (anyfg[t]) A.tl_list[atomicAdd(A.tl_count, 1)] = tile;
            else A.T.piece_cnt[tile] = 0;
        }
    }
}

// the padded size of a kw x kh kernel (odd, at most 15)
static int psf_ks(int kw, int kh)
{
    const int k = kw > kh ? kw : kh;
    return k <= 3 ? 3 : k <= 5 ? 5 : k <= 7 ? 7 : k <= 9 ? 9 : k <= 11 ? 11 : k <= 13 ? 13 : 15;
}

template <int KS>
static cudaError_t launch_psf_ks(const PsfArgs& A, bool f32, dim3 g, cudaStream_t st)
{
    if (f32) k_psf<true, KS><<<g, PS_NT, 0, st>>>(A);
    else k_psf<false, KS><<<g, PS_NT, 0, st>>>(A);
    return cudaGetLastError();
}

cudaError_t launch_psf(const DetectArgs& D, const float* p0, const float* modes, int nk, int kw, int kh,
                       const SplineTab* coef_tabs, cudaStream_t st)
{
    PsfArgs A;
    memset(&A, 0, sizeof A);
    A.im = D.im; A.sb = D.sb; A.sr = D.sr;
    A.nk = nk;
    for (int k = 0; k < nk; ++k) A.ct[k] = coef_tabs[k];
    A.thresh = D.thresh;
    A.seg = D.seg; A.bits = D.bits; A.nstrip = D.nstrip;
    A.tl_list = D.tl_list; A.tl_count = D.tl_count; A.T = D.T;
    const int ks = psf_ks(kw, kh), ox = (ks - kw) / 2, oy = (ks - kh) / 2;
    for (int k = 0; k <= nk; ++k) {
        const float* src = k == 0 ? p0 : modes + (size_t)(k - 1) * kw * kh;
        for (int v = 0; v < kh; ++v)
            for (int u = 0; u < kw; ++u) {
                float2& t = A.taps[k / 2][(v + oy) * ks + (u + ox)];
                if (k & 1) t.y = src[v * kw + u];
                else t.x = src[v * kw + u];
            }
    }
    const dim3 g((D.im.W + PS_COLS - 1) / PS_COLS, (D.im.H + PS_ROWS - 1) / PS_ROWS);
    const bool f32 = D.im.is_f32;
    switch (ks) {
    case 3: return launch_psf_ks<3>(A, f32, g, st);
    case 5: return launch_psf_ks<5>(A, f32, g, st);
    case 7: return launch_psf_ks<7>(A, f32, g, st);
    case 9: return launch_psf_ks<9>(A, f32, g, st);
    case 11: return launch_psf_ks<11>(A, f32, g, st);
    case 13: return launch_psf_ks<13>(A, f32, g, st);
    default: return launch_psf_ks<15>(A, f32, g, st);
    }
}

}  // namespace gp
