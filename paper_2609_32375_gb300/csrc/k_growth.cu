// k_growth.cu -- growth curves by top-hat apertures (paper Section 3.4):
// for each source and each integer radius r of a list, the sum of m = I - B
// over the top-hat {(u, v) : u^2 + v^2 <= r^2} centred on the pixel nearest
// the source, (floor(x + 1/2), floor(y + 1/2)), with sigma^2 summed over the
// same pixels -- the value at that pixel of the frame's cross-correlation
// with the top-hat, which the paper evaluates by FFT for all pixels at once.
// Here only the sources' pixels are visited.
//
// One warp per source, a lane per column of the largest top-hat, rows in
// order.  Every pixel is added once, to the ring of radii it opens: the
// smallest r_k with r_k^2 >= u^2 + v^2 (a table over u^2 + v^2).  A lane
// keeps float-float sums for its current ring and adds them into its
// slot for that ring in shared memory when the ring changes (down a column
// the ring index falls, then rises: at most two stretches per ring).  Then
// lane k sums ring k's 32 slots in lane order, and a scan across the lanes turns
// ring sums into the growth curve (radius k = rings 0..k).  Fixed orders
// throughout: the sums are reproducible.
#include <math.h>
#include <string.h>

#include "gp_internal.cuh"
#include "gp_launch.h"

namespace gp {

constexpr int GR_NT = 128;                 // 4 warps per CTA
constexpr int GR_W = GR_NT / 32;

struct GrowthSpec {
    int nr;
    int r[GP_GROWTH_MAX_NR];
    int rmax;
    float gain;
    double inv_gain;            // 1 / gain (0 when gain <= 0)
};

// dynamic shared memory: the ring table (int8 per u^2 + v^2 up to rmax^2),
// then per warp: flux and variance slots [32 lanes][S] (float-float) and flag
// slots [32][S], S = nr rounded up to odd so that lane k reading ring k of
// every lane meets no bank conflict
template <bool F32>
__global__ void __launch_bounds__(GR_NT) k_growth(Image im, SplineTab sb, SplineTab sr,
                                                  const __grid_constant__ GrowthSpec gs, const double* __restrict__ xs,
                                                  const double* __restrict__ ys, int n, const int* __restrict__ n_dev,
                                                  double* flux, double* ferr, uint32_t* flags)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int nr = gs.nr, rmax = gs.rmax, r2max = rmax * rmax;
    int8_t* ring_of = reinterpret_cast<int8_t*>(smem);
    const size_t tab = ((size_t)r2max + 1 + 15) & ~(size_t)15;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int S = nr | 1, NS = 32 * S;
    float2* sf = reinterpret_cast<float2*>(smem + tab) + (size_t)warp * NS * 2;
    float2* sv = sf + NS;
    uint32_t* sfl = reinterpret_cast<uint32_t*>(smem + tab + (size_t)GR_W * NS * 2 * sizeof(float2)) +
                    (size_t)warp * NS;
    for (int d2 = threadIdx.x; d2 <= r2max; d2 += GR_NT) {
        int k = 0;
        while (k < nr && gs.r[k] * gs.r[k] < d2) ++k;
        ring_of[d2] = (int8_t)k;                        // k < nr: every d2 <= rmax^2 opens some radius
    }
    __syncthreads();
    const int W = im.W, H = im.H;
    const int wid = blockIdx.x * GR_W + warp, nw = gridDim.x * GR_W;
    if (n_dev) n = min(n, *n_dev);           // a device count (catalog rows), at most n
    for (int s = wid; s < n; s += nw) {
        const double cxd = floor(xs[s] + 0.5), cyd = floor(ys[s] + 0.5);
        // positions far outside the frame (or NaN) give empty sums, flagged
        const bool near = fabs(cxd - 0.5 * W) <= 0.5 * W + 4096.0 && fabs(cyd - 0.5 * H) <= 0.5 * H + 4096.0;
        const int xc = near ? (int)cxd : -(1 << 20), yc = near ? (int)cyd : -(1 << 20);
        for (int i = lane; i < NS; i += 32) {
            sf[i] = make_float2(0.f, 0.f);
            sv[i] = make_float2(0.f, 0.f);
            sfl[i] = 0u;
        }
        __syncwarp();
        for (int u0 = -rmax; u0 <= rmax; u0 += 32) {
            const int u = u0 + lane;
            const bool col = u <= rmax;
            const int x = xc + u;
            const bool xin = x >= 0 && x < W;
            const AxCoef ccx = axis_coef(sb.ax, (float)(xin ? x : 0));
            int jc = -1;
            float ub0 = 0, ub1 = 0, wb0 = 0, wb1 = 0, ur0 = 0, ur1 = 0, wr0 = 0, wr1 = 0;
            int kc = -1;
            DF cf = df_zero(), cv = df_zero();
            uint32_t cfl = 0u;
            auto flush = [&]() {
                if (kc >= 0) {
                    const int q = lane * S + kc;
                    DF a;
                    a.hi = sf[q].x; a.lo = sf[q].y;
                    a = df_merge(a, cf);
                    sf[q] = make_float2(a.hi, a.lo);
                    a.hi = sv[q].x; a.lo = sv[q].y;
                    a = df_merge(a, cv);
                    sv[q] = make_float2(a.hi, a.lo);
                    sfl[q] |= cfl;
                }
                cf = df_zero(); cv = df_zero(); cfl = 0u;
            };
            for (int v = -rmax; v <= rmax; ++v) {
                const int d2 = u * u + v * v;
                if (!col || d2 > r2max) continue;
                const int k = ring_of[d2];
                if (k != kc) {
                    flush();
                    kc = k;
                }
                const int y = yc + v;
                if (!xin || y < 0 || y >= H) {
                    cfl |= GP_FLAG_TRUNCATED;
                    continue;
                }
                bool bad;
                const float val = load_px<F32>(im, x, y, bad);
                if (bad) {
                    cfl |= GP_FLAG_BAD;
                    continue;
                }
                const AxCoef ccy = axis_coef(sb.ay, (float)y);
                if (ccy.i != jc) {
                    const float2 b0 = row_eval(sb, ccy.i, ccx), b1 = row_eval(sb, ccy.i1, ccx);
                    const float2 r0 = row_eval(sr, ccy.i, ccx), r1 = row_eval(sr, ccy.i1, ccx);
                    ub0 = b0.x; wb0 = b0.y; ub1 = b1.x; wb1 = b1.y;
                    ur0 = r0.x; wr0 = r0.y; ur1 = r1.x; wr1 = r1.y;
                    jc = ccy.i;
                }
                const float m = val - axis_combine(ccy, ub0, ub1, wb0, wb1);
                const float sg = axis_combine(ccy, ur0, ur1, wr0, wr1);
                if (im.sat > 0.f && val >= im.sat) cfl |= GP_FLAG_SAT;
                df_add(cf, m);
                df_add_prod(cv, sg, sg);
            }
            flush();
            __syncwarp();
        }
        // ring sums in lane order, then radius k = rings 0..k (a scan whose
        // combination order is fixed)
        DF rf = df_zero(), rv = df_zero();
        uint32_t rfl = 0u;
        if (lane < nr) {
            for (int l = 0; l < 32; ++l) {
                const int q = l * S + lane;
                DF a;
                a.hi = sf[q].x; a.lo = sf[q].y;
                rf = df_merge(rf, a);
                a.hi = sv[q].x; a.lo = sv[q].y;
                rv = df_merge(rv, a);
                rfl |= sfl[q];
            }
        }
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            DF pf, pv;
            pf.hi = __shfl_up_sync(0xffffffffu, rf.hi, o); pf.lo = __shfl_up_sync(0xffffffffu, rf.lo, o);
            pv.hi = __shfl_up_sync(0xffffffffu, rv.hi, o); pv.lo = __shfl_up_sync(0xffffffffu, rv.lo, o);
            const uint32_t pfl = __shfl_up_sync(0xffffffffu, rfl, o);
            if (lane >= o) {
                rf = df_merge(pf, rf);
                rv = df_merge(pv, rv);
                rfl |= pfl;
            }
        }
        if (lane < nr) {
            const double F = df_value(rf);
            double V = df_value(rv);
            if (gs.gain > 0.f && F > 0.0) V = fma(F, gs.inv_gain, V);
            const int64_t o = (int64_t)s * nr + lane;
            flux[o] = F;
            ferr[o] = V > 0.0 ? sqrt(V) : 0.0;
            flags[o] = rfl;
        }
        __syncwarp();
    }
}

size_t growth_smem_bytes(int nr, int rmax)
{
    const size_t tab = ((size_t)rmax * rmax + 1 + 15) & ~(size_t)15;
    return tab + (size_t)GR_W * (nr | 1) * 32 * (2 * sizeof(float2) + sizeof(uint32_t));
}

cudaError_t launch_growth(const Image& im, const SplineTab& sb, const SplineTab& sr, const double* xs,
                          const double* ys, int n, const int* n_dev, const int* radii, int nr, float gain,
                          double* flux, double* ferr, uint32_t* flags, cudaStream_t st)
{
    GrowthSpec gs;
    memset(&gs, 0, sizeof gs);
    gs.nr = nr;
    for (int k = 0; k < nr; ++k) gs.r[k] = radii[k];
    gs.rmax = radii[nr - 1];
    gs.gain = gain;
    gs.inv_gain = gain > 0.f ? 1.0 / (double)gain : 0.0;
    const size_t smem = growth_smem_bytes(nr, gs.rmax);
    const int grid = 152 * 4;
    if (im.is_f32) {
        cudaFuncSetAttribute(k_growth<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_growth<true><<<grid, GR_NT, smem, st>>>(im, sb, sr, gs, xs, ys, n, n_dev, flux, ferr, flags);
    } else {
        cudaFuncSetAttribute(k_growth<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_growth<false><<<grid, GR_NT, smem, st>>>(im, sb, sr, gs, xs, ys, n, n_dev, flux, ferr, flags);
    }
    return cudaGetLastError();
}

}  // namespace gp
