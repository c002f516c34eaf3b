// k_cnn.cu -- the learned background: a small convolutional network that
// maps one-pass per-box quantile features (q10, q25, q50, q75, q90) to the
// background and rms meshes, replacing the iterative clip and median filter.
// The paper has no counterpart (its background is an FFT-smoothed local
// estimate, Section 3.1); the plain estimator stays as the fallback and as
// the source of the training targets.
//
// Network: six 3x3 convolutions (zero padding, same size) with ReLU between
// them, channels 5 -> 32 -> 48 -> 48 -> 32 -> 32 -> 2.  Activations are
// NHWC bfloat16 with channels padded to a multiple of 16; weights bfloat16,
// master weights and optimiser state float32; every contraction accumulates
// in float32.
//
//  k_conv3x3   implicit GEMM on the tensor cores (mma.sync m16n8k16 bf16):
//              one CTA per 64 output positions of one row, the 3-row input
//              patch and the whole weight matrix staged in shared memory.
//              Also computes the data gradient (with flipped, transposed
//              weights).
//  k_wgrad     weight gradient dW[co][tap][ci] = sum_p dP[p][co] x[p+tap][ci]
//              as a tensor-core GEMM over positions, one partial per slot,
//              slots summed in a fixed order (reproducible).
//  others      ReLU backward, MSE loss, weight packing, AdamW, features,
//              output denormalisation.
#include <cuda_bf16.h>
#include <math.h>

#include "gp_internal.cuh"
#include "gp_launch.h"

namespace gp {

typedef __nv_bfloat16 bf16;

__device__ __forceinline__ void mma_bf16(float* c, uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                         uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t ld_u32(const bf16* p) { return *reinterpret_cast<const uint32_t*>(p); }

__device__ __forceinline__ uint32_t pack2(bf16 lo, bf16 hi)
{
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

constexpr int CONV_NT = 128;     // 4 warps x 16 positions
constexpr int CONV_TX = 64;

// ------------------------------------------------------------ forward ---
template <int CIP, int COP>
__global__ void __launch_bounds__(CONV_NT) k_conv3x3(const bf16* __restrict__ x, const bf16* __restrict__ wt,
                                                     const float* __restrict__ bias, void* __restrict__ y, int H,
                                                     int W, int relu, int out_f32, int creal)
{
    constexpr int K = 9 * CIP;
    extern __shared__ __align__(16) unsigned char sm[];
    bf16* patch = reinterpret_cast<bf16*>(sm);                       // [3][CONV_TX + 2][CIP]
    bf16* wts = patch + 3 * (CONV_TX + 2) * CIP;                     // [COP][K]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int x0 = blockIdx.x * CONV_TX, row = blockIdx.y, n = blockIdx.z;
    // stage the three input rows (zero outside the mesh), 16 bytes at a time
    constexpr int VPP = CIP / 8;                                     // 16-byte vectors per position
    for (int q = tid; q < 3 * (CONV_TX + 2) * VPP; q += CONV_NT) {
        const int v = q % VPP, pc = q / VPP;
        const int r = pc / (CONV_TX + 2), c = pc - r * (CONV_TX + 2);
        const int gy = row + r - 1, gx = x0 + c - 1;
        uint4 val = make_uint4(0, 0, 0, 0);
        if (gy >= 0 && gy < H && gx >= 0 && gx < W)
            val = *reinterpret_cast<const uint4*>(x + (((int64_t)n * H + gy) * W + gx) * CIP + v * 8);
        *reinterpret_cast<uint4*>(patch + pc * CIP + v * 8) = val;
    }
    for (int q = tid; q < COP * K / 8; q += CONV_NT)
        reinterpret_cast<uint4*>(wts)[q] = reinterpret_cast<const uint4*>(wt)[q];
    __syncthreads();

    const int g = lane >> 2, t = lane & 3;
    const int xa = warp * 16 + g, xb = xa + 8;                       // local positions of rows g, g+8
    float acc[COP / 8][4];
#pragma unroll
    for (int j = 0; j < COP / 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) {
        const int dy = tap / 3, dx = tap % 3;
        const bf16* pa = patch + (dy * (CONV_TX + 2) + xa + dx) * CIP;
        const bf16* pb = patch + (dy * (CONV_TX + 2) + xb + dx) * CIP;
#pragma unroll
        for (int cb = 0; cb < CIP / 16; ++cb) {
            const int c0 = cb * 16 + 2 * t;
            const uint32_t a0 = ld_u32(pa + c0), a1 = ld_u32(pb + c0);
            const uint32_t a2 = ld_u32(pa + c0 + 8), a3 = ld_u32(pb + c0 + 8);
            const int k0 = tap * CIP + cb * 16 + 2 * t;
#pragma unroll
            for (int j = 0; j < COP / 8; ++j) {
                const bf16* wr = wts + (j * 8 + g) * K + k0;
                mma_bf16(acc[j], a0, a1, a2, a3, ld_u32(wr), ld_u32(wr + 8));
            }
        }
    }
    // epilogue: bias, activation, store
    const int gxa = x0 + xa, gxb = x0 + xb;
#pragma unroll
    for (int j = 0; j < COP / 8; ++j) {
        const int co = j * 8 + 2 * t;
        float v0 = acc[j][0] + bias[co], v1 = acc[j][1] + bias[co + 1];
        float v2 = acc[j][2] + bias[co], v3 = acc[j][3] + bias[co + 1];
        if (relu) { v0 = fmaxf(v0, 0.f); v1 = fmaxf(v1, 0.f); v2 = fmaxf(v2, 0.f); v3 = fmaxf(v3, 0.f); }
        if (out_f32) {
            float* yo = reinterpret_cast<float*>(y);
            if (gxa < W) {
                const int64_t o = (((int64_t)n * H + row) * W + gxa) * creal;
                if (co < creal) yo[o + co] = v0;
                if (co + 1 < creal) yo[o + co + 1] = v1;
            }
            if (gxb < W) {
                const int64_t o = (((int64_t)n * H + row) * W + gxb) * creal;
                if (co < creal) yo[o + co] = v2;
                if (co + 1 < creal) yo[o + co + 1] = v3;
            }
        } else {
            bf16* yo = reinterpret_cast<bf16*>(y);
            if (gxa < W)
                *reinterpret_cast<uint32_t*>(yo + (((int64_t)n * H + row) * W + gxa) * COP + co) =
                    pack2(__float2bfloat16_rn(v0), __float2bfloat16_rn(v1));
            if (gxb < W)
                *reinterpret_cast<uint32_t*>(yo + (((int64_t)n * H + row) * W + gxb) * COP + co) =
                    pack2(__float2bfloat16_rn(v2), __float2bfloat16_rn(v3));
        }
    }
}

// ---------------------------------------------------- weight gradient ---
// Block (slot, tap): rows r = slot, slot + nslot, ... of the N*H output rows.
// GEMM per row: M = COP output channels, N = CIP input channels, K = 64
// positions.  A = dP^T (staged transposed), B = the tap-shifted input row.
template <int CIP, int COP>
__global__ void __launch_bounds__(CONV_NT) k_wgrad(const bf16* __restrict__ x, const bf16* __restrict__ dp, int NH,
                                                   int H, int W, int nslot, float* __restrict__ partial)
{
    __shared__ __align__(16) bf16 dpt[COP][CONV_TX + 8];             // dP transposed: [co][position]
    __shared__ __align__(16) bf16 xs[CONV_TX + 2][CIP];              // input row, positions -1 .. 64
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int slot = blockIdx.x, tap = blockIdx.y;
    const int dy = tap / 3, dx = tap % 3;
    const int g = lane >> 2, t = lane & 3;
    constexpr int MT = COP / 16, NT = CIP / 8, TT = MT * NT;
    constexpr int PER = (TT + 3) / 4;                                // tiles per warp
    float acc[PER][4];
#pragma unroll
    for (int i = 0; i < PER; ++i) acc[i][0] = acc[i][1] = acc[i][2] = acc[i][3] = 0.f;
    for (int r = slot; r < NH; r += nslot) {
        const int n = r / H, row = r - n * H;
        const int srow = row + dy - 1;
        for (int x0 = 0; x0 < W; x0 += CONV_TX) {
            __syncthreads();
            for (int q = tid; q < CONV_TX * COP; q += CONV_NT) {
                const int p = q / COP, co = q - p * COP;
                const int gx = x0 + p;
                dpt[co][p] = gx < W ? dp[(((int64_t)n * H + row) * W + gx) * COP + co] : __float2bfloat16_rn(0.f);
            }
            for (int q = tid; q < (CONV_TX + 2) * CIP; q += CONV_NT) {
                const int c = q / CIP, ci = q - c * CIP;
                const int gx = x0 + c - 1;
                xs[c][ci] = (srow >= 0 && srow < H && gx >= 0 && gx < W)
                                ? x[(((int64_t)n * H + srow) * W + gx) * CIP + ci]
                                : __float2bfloat16_rn(0.f);
            }
            __syncthreads();
#pragma unroll
            for (int i = 0; i < PER; ++i) {
                const int tt = warp + 4 * i;
                if (tt >= TT) break;
                const int mt = tt / NT, nt = tt - mt * NT;
#pragma unroll
                for (int ks = 0; ks < CONV_TX / 16; ++ks) {
                    const int p0 = ks * 16 + 2 * t;
                    const uint32_t a0 = ld_u32(&dpt[mt * 16 + g][p0]), a1 = ld_u32(&dpt[mt * 16 + g + 8][p0]);
                    const uint32_t a2 = ld_u32(&dpt[mt * 16 + g][p0 + 8]), a3 = ld_u32(&dpt[mt * 16 + g + 8][p0 + 8]);
                    // B(k = position, n = input channel): shifted by the tap's dx
                    const int ci = nt * 8 + g;
                    const uint32_t b0 = pack2(xs[p0 + dx][ci], xs[p0 + 1 + dx][ci]);
                    const uint32_t b1 = pack2(xs[p0 + 8 + dx][ci], xs[p0 + 9 + dx][ci]);
                    mma_bf16(acc[i], a0, a1, a2, a3, b0, b1);
                }
            }
        }
    }
    // partial[slot][tap][co][ci]
    float* out = partial + ((int64_t)slot * 9 + tap) * COP * CIP;
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int tt = warp + 4 * i;
        if (tt >= TT) break;
        const int mt = tt / NT, nt = tt - mt * NT;
        const int co = mt * 16 + g, ci = nt * 8 + 2 * t;
        out[co * CIP + ci] = acc[i][0];
        out[co * CIP + ci + 1] = acc[i][1];
        out[(co + 8) * CIP + ci] = acc[i][2];
        out[(co + 8) * CIP + ci + 1] = acc[i][3];
    }
}

// dW[co][ci][3][3] (real channels) = sum over slots in slot order; bias
// gradient likewise from per-slot partial sums of dP
__global__ void k_wgrad_reduce(const float* __restrict__ partial, int nslot, int cip, int cop, int cir, int cor,
                               float* __restrict__ dw)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int total = cor * cir * 9;
    if (i >= total) return;
    const int co = i / (cir * 9), rem = i - co * cir * 9, ci = rem / 9, tap = rem - ci * 9;
    float s = 0.f;
    for (int k = 0; k < nslot; ++k) s += partial[(((int64_t)k * 9 + tap) * cop + co) * cip + ci];
    dw[i] = s;
}

__global__ void k_bias_partial(const bf16* __restrict__ dp, int64_t npos, int cop, int nslot, float* __restrict__ part)
{
    // block = slot; thread = channel (cop <= 64); positions slot, slot + nslot, ...
    const int slot = blockIdx.x, co = threadIdx.x;
    if (co >= cop) return;
    float s = 0.f;
    for (int64_t p = slot; p < npos; p += nslot) s += __bfloat162float(dp[p * cop + co]);
    part[slot * cop + co] = s;
}

__global__ void k_bias_reduce(const float* __restrict__ part, int nslot, int cop, int cor, float* __restrict__ db)
{
    const int co = threadIdx.x;
    if (co >= cor) return;
    float s = 0.f;
    for (int k = 0; k < nslot; ++k) s += part[k * cop + co];
    db[co] = s;
}

// -------------------------------------------------------- elementwise ---
__global__ void k_relu_backward(const bf16* __restrict__ dy, const bf16* __restrict__ y, bf16* __restrict__ dp,
                                int64_t count)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        dp[i] = __bfloat162float(y[i]) > 0.f ? dy[i] : __float2bfloat16_rn(0.f);
}

// mean squared error over npos positions x 2 channels; dY (bf16, padded to
// cop channels) = 2 (pred - target) / (2 npos); per-block partial losses
__global__ void k_mse(const float* __restrict__ pred, const float* __restrict__ target, int64_t npos, int cop,
                      bf16* __restrict__ dy, float* __restrict__ part)
{
    __shared__ float red[256];
    float s = 0.f;
    const float scale = 2.f / (2.f * (float)npos);
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < npos; p += (int64_t)gridDim.x * blockDim.x) {
        for (int c = 0; c < cop; ++c) {
            float d = 0.f;
            if (c < 2) {
                d = pred[p * 2 + c] - target[p * 2 + c];
                s += d * d;
            }
            dy[p * cop + c] = __float2bfloat16_rn(scale * d);
        }
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void k_mse_reduce(const float* __restrict__ part, int nb, int64_t npos, float* __restrict__ loss)
{
    if (threadIdx.x != 0) return;
    double s = 0.0;
    for (int i = 0; i < nb; ++i) s += part[i];
    *loss = (float)(s / (2.0 * (double)npos));
}

// master W[co][ci][3][3] (real channels) -> forward wt[cop][9*cip] and the
// data-gradient weights wtd[cip][9*cop] (taps flipped, in and out swapped)
__global__ void k_pack(const float* __restrict__ W, const float* __restrict__ b, int cir, int cor, int cip, int cop,
                       bf16* __restrict__ wt, bf16* __restrict__ wtd, float* __restrict__ bias_p)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < cop * 9 * cip) {
        const int co = i / (9 * cip), k = i - co * 9 * cip, tap = k / cip, ci = k - tap * cip;
        const float v = (co < cor && ci < cir) ? W[(co * cir + ci) * 9 + tap] : 0.f;
        wt[i] = __float2bfloat16_rn(v);
        // wtd[ci][tap' * cop + co] with tap' the flipped tap
        const int tf = 8 - tap;
        wtd[(int64_t)ci * 9 * cop + tf * cop + co] = __float2bfloat16_rn(v);
    }
    if (i < cop) bias_p[i] = i < cor ? b[i] : 0.f;
}

__global__ void k_adamw(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                        float* __restrict__ v, int64_t n, float lr, float b1, float b2, float eps, float wd, float c1,
                        float c2)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float mh = mi / c1, vh = vi / c2;
        p[i] -= lr * (mh / (sqrtf(vh) + eps) + wd * p[i]);
    }
}

// ------------------------------------------------------------ features ---
// One CTA per frame: centre c = median of the box medians q50, scale
// s = median of (q75 - q25) / 1.349 (the Gaussian sigma of an interquartile
// range); features (q_k - c) / s in channels 0..4 of a 16-channel NHWC
// bf16 map; (c, s) kept for denormalising the output.
constexpr int FEAT_NT = 1024;

__device__ float block_median(float* buf, int n, int npad)
{
    for (int i = n + threadIdx.x; i < npad; i += FEAT_NT) buf[i] = INFINITY;
    __syncthreads();
    for (int size = 2; size <= npad; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < npad / 2; i += FEAT_NT) {
                const int lo = 2 * i - (i & (stride - 1)), hi = lo + stride;
                const bool up = (lo & size) == 0;
                const float a = buf[lo], b = buf[hi];
                if ((a > b) == up) { buf[lo] = b; buf[hi] = a; }
            }
            __syncthreads();
        }
    const float med = (n & 1) ? buf[n / 2] : 0.5f * (buf[n / 2 - 1] + buf[n / 2]);
    __syncthreads();
    return med;
}

__global__ void __launch_bounds__(FEAT_NT) k_features(const float* __restrict__ quant, int nbox, int npad,
                                                      bf16* __restrict__ feat, float* __restrict__ norm)
{
    extern __shared__ float buf[];
    const int f = blockIdx.x;
    const float* q = quant + (int64_t)f * 5 * nbox;                  // [5][nbox]
    for (int i = threadIdx.x; i < nbox; i += FEAT_NT) buf[i] = q[2 * nbox + i];
    const float c = block_median(buf, nbox, npad);
    for (int i = threadIdx.x; i < nbox; i += FEAT_NT) buf[i] = q[3 * nbox + i] - q[1 * nbox + i];
    float s = block_median(buf, nbox, npad) / 1.349f;
    if (!(s > 0.f)) s = 1.f;
    if (threadIdx.x == 0) { norm[2 * f] = c; norm[2 * f + 1] = s; }
    for (int i = threadIdx.x; i < nbox * 16; i += FEAT_NT) {
        const int b = i / 16, ch = i - b * 16;
        const float v = ch < 5 ? (q[ch * nbox + b] - c) / s : 0.f;
        feat[(int64_t)f * nbox * 16 + i] = __float2bfloat16_rn(v);
    }
}

// network output (N x nbox x 2, normalised) -> meshes
__global__ void k_denorm(const float* __restrict__ out, const float* __restrict__ norm, int nbox, int64_t total,
                         float* __restrict__ bkg, float* __restrict__ rms)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int f = (int)(i / nbox);
        const float c = norm[2 * f], s = norm[2 * f + 1];
        bkg[i] = c + s * out[2 * i];
        rms[i] = s * fmaxf(out[2 * i + 1], 0.f);
    }
}

// meshes -> normalised targets (training)
__global__ void k_targets(const float* __restrict__ bkg, const float* __restrict__ rms, const float* __restrict__ norm,
                          int nbox, int64_t total, float* __restrict__ tgt)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int f = (int)(i / nbox);
        const float c = norm[2 * f], s = norm[2 * f + 1];
        tgt[2 * i] = (bkg[i] - c) / s;
        tgt[2 * i + 1] = rms[i] / s;
    }
}

// --------------------------------------------------------------- launchers ---
template <int CIP, int COP>
static cudaError_t conv_launch(const void* x, int n, int h, int w, const void* wt, const float* bias, int relu,
                               void* y, int out_f32, int creal, cudaStream_t st)
{
    const size_t smem = (size_t)(3 * (CONV_TX + 2) * CIP + COP * 9 * CIP) * sizeof(bf16);
    cudaFuncSetAttribute(k_conv3x3<CIP, COP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    dim3 grid((w + CONV_TX - 1) / CONV_TX, h, n);
    k_conv3x3<CIP, COP><<<grid, CONV_NT, smem, st>>>(reinterpret_cast<const bf16*>(x),
                                                     reinterpret_cast<const bf16*>(wt), bias, y, h, w, relu, out_f32,
                                                     creal);
    return cudaGetLastError();
}

template <int CIP, int COP>
static cudaError_t wgrad_launch(const void* x, const void* dp, int n, int h, int w, int nslot, float* partial,
                                cudaStream_t st)
{
    dim3 grid(nslot, 9);
    k_wgrad<CIP, COP><<<grid, CONV_NT, 0, st>>>(reinterpret_cast<const bf16*>(x), reinterpret_cast<const bf16*>(dp),
                                                n * h, h, w, nslot, partial);
    return cudaGetLastError();
}

#define GP_CNN_PAIRS(X) X(16, 32) X(32, 48) X(48, 48) X(48, 32) X(32, 32) X(32, 16)

bool cnn_pair_supported(int cip, int cop)
{
#define GP_P(a, b) if (cip == a && cop == b) return true;
    GP_CNN_PAIRS(GP_P)
#undef GP_P
    return false;
}

cudaError_t launch_cnn_conv(const void* x, int n, int h, int w, int cip, const void* wt, const float* bias, int cop,
                            int relu, void* y, int out_f32, int creal, cudaStream_t st)
{
#define GP_P(a, b) if (cip == a && cop == b) return conv_launch<a, b>(x, n, h, w, wt, bias, relu, y, out_f32, creal, st);
    GP_CNN_PAIRS(GP_P)
#undef GP_P
    return cudaErrorInvalidValue;
}

cudaError_t launch_cnn_wgrad(const void* x, const void* dp, int n, int h, int w, int cip, int cop, int cir, int cor,
                             int nslot, float* partial, float* bpart, float* dw, float* db, cudaStream_t st)
{
    cudaError_t e = cudaErrorInvalidValue;
#define GP_P(a, b) if (cip == a && cop == b) e = wgrad_launch<a, b>(x, dp, n, h, w, nslot, partial, st);
    GP_CNN_PAIRS(GP_P)
#undef GP_P
    if (e != cudaSuccess) return e;
    const int total = cor * cir * 9;
    k_wgrad_reduce<<<(total + 255) / 256, 256, 0, st>>>(partial, nslot, cip, cop, cir, cor, dw);
    k_bias_partial<<<nslot, 64, 0, st>>>(reinterpret_cast<const bf16*>(dp), (int64_t)n * h * w, cop, nslot, bpart);
    k_bias_reduce<<<1, 64, 0, st>>>(bpart, nslot, cop, cor, db);
    return cudaGetLastError();
}

cudaError_t launch_cnn_relu_backward(const void* dy, const void* y, void* dp, int64_t count, cudaStream_t st)
{
    k_relu_backward<<<152 * 4, 256, 0, st>>>(reinterpret_cast<const bf16*>(dy), reinterpret_cast<const bf16*>(y),
                                             reinterpret_cast<bf16*>(dp), count);
    return cudaGetLastError();
}

cudaError_t launch_cnn_mse(const float* pred, const float* target, int64_t npos, int cop, void* dy, float* part,
                           int nblocks, float* loss, cudaStream_t st)
{
    k_mse<<<nblocks, 256, 0, st>>>(pred, target, npos, cop, reinterpret_cast<bf16*>(dy), part);
    k_mse_reduce<<<1, 32, 0, st>>>(part, nblocks, npos, loss);
    return cudaGetLastError();
}

cudaError_t launch_cnn_pack(const float* W, const float* b, int cir, int cor, int cip, int cop, void* wt, void* wtd,
                            float* bias_p, cudaStream_t st)
{
    const int total = cop * 9 * cip;
    k_pack<<<(total + 255) / 256, 256, 0, st>>>(W, b, cir, cor, cip, cop, reinterpret_cast<bf16*>(wt),
                                                reinterpret_cast<bf16*>(wtd), bias_p);
    return cudaGetLastError();
}

cudaError_t launch_cnn_adamw(float* p, const float* g, float* m, float* v, int64_t n, float lr, float b1, float b2,
                             float eps, float wd, int step, cudaStream_t st)
{
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    k_adamw<<<152 * 2, 256, 0, st>>>(p, g, m, v, n, lr, b1, b2, eps, wd, c1, c2);
    return cudaGetLastError();
}

cudaError_t launch_cnn_features(const float* quant, int nframes, int nbox, void* feat, float* norm, cudaStream_t st)
{
    int npad = 1;
    while (npad < nbox) npad <<= 1;
    const size_t smem = (size_t)npad * sizeof(float);
    cudaFuncSetAttribute(k_features, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_features<<<nframes, FEAT_NT, smem, st>>>(quant, nbox, npad, reinterpret_cast<bf16*>(feat), norm);
    return cudaGetLastError();
}

cudaError_t launch_cnn_denorm(const float* out, const float* norm, int nbox, int nframes, float* bkg, float* rms,
                              cudaStream_t st)
{
    const int64_t total = (int64_t)nbox * nframes;
    k_denorm<<<(int)((total + 255) / 256 < 1024 ? (total + 255) / 256 : 1024), 256, 0, st>>>(out, norm, nbox, total,
                                                                                            bkg, rms);
    return cudaGetLastError();
}

cudaError_t launch_cnn_targets(const float* bkg, const float* rms, const float* norm, int nbox, int nframes,
                               float* tgt, cudaStream_t st)
{
    const int64_t total = (int64_t)nbox * nframes;
    k_targets<<<(int)((total + 255) / 256 < 1024 ? (total + 255) / 256 : 1024), 256, 0, st>>>(bkg, rms, norm, nbox,
                                                                                             total, tgt);
    return cudaGetLastError();
}

}  // namespace gp
