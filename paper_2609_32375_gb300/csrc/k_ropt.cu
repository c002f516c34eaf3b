// k_ropt.cu -- the optimal aperture radius (paper Section 3.4): the radius
// of largest S/N is searched on the growth curves of high-S/N isolated
// calibrators, log10 r_opt = a log10 nu + b is fitted to them (nu the
// detection significance), and every other source takes the radius of the
// fit.
//
//  k_ropt_nu     one thread per catalog row: nu = F / sigma at the row's peak
//                pixel (F the matched filter of m = I - B with the detection
//                kernel, mirror border, bad pixels 0) and the index of the
//                largest S/N = flux / fluxerr of its growth curve (the first
//                on ties; 0 where fluxerr <= 0).
//  k_iso_*       isolation on a grid of cells at least d_iso wide: count,
//                scan, fill, then each row looks for another centroid closer
//                than d_iso in its 3 x 3 cells, and takes the calibrator test.
//  k_ropt_fit    one CTA: least squares of log10 r on log10 nu over the
//                calibrators from centred sums, in a fixed summation order.
//  k_ropt_assign one thread per row: the calibrators keep their best radius,
//                the others take the grid radius nearest to the fit's
//                (ties to the larger).
#include <math.h>
#include <string.h>

#include <algorithm>

#include "gp_internal.cuh"
#include "gp_launch.h"

namespace gp {

constexpr int FIT_NT = 512;

struct RoptTaps {
    int kw, kh;
    float t[KMAX];
};

struct RoptRadii {
    int nr;
    int r[GP_GROWTH_MAX_NR];
};

template <bool F32>
__global__ void __launch_bounds__(256) k_ropt_nu(Image im, SplineTab sb, SplineTab sr,
                                                 const __grid_constant__ RoptTaps K, const int* __restrict__ xp,
                                                 const int* __restrict__ yp, const double* __restrict__ flux,
                                                 const double* __restrict__ ferr, int nr, const int* __restrict__ n_dev,
                                                 int cap, float* nu, int* kopt)
{
    const int n = min(*n_dev, cap);
    const int W = im.W, H = im.H, hx = K.kw / 2, hy = K.kh / 2;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int x0 = xp[i], y0 = yp[i];
        float F = 0.f;
        for (int v = 0; v < K.kh; ++v) {
            const int y = mirror_idx(y0 + v - hy, H);
            const AxCoef cy = axis_coef(sb.ay, (float)y);
            for (int u = 0; u < K.kw; ++u) {
                const int x = mirror_idx(x0 + u - hx, W);
                bool bad;
                const float val = load_px<F32>(im, x, y, bad);
                const AxCoef cx = axis_coef(sb.ax, (float)x);
                const float2 r0 = row_eval(sb, cy.i, cx), r1 = row_eval(sb, cy.i1, cx);
                const float m = bad ? 0.f : val - axis_combine(cy, r0.x, r1.x, r0.y, r1.y);
                F = fmaf(K.t[v * K.kw + u], m, F);
            }
        }
        const float s = spline_eval(sr, (float)x0, (float)y0);
        nu[i] = s > 0.f ? F / s : 0.f;
        int best = 0;
        double bs = 0.0;
        for (int k = 0; k < nr; ++k) {
            const double e = ferr[(int64_t)i * nr + k];
            const double q = e > 0.0 ? flux[(int64_t)i * nr + k] / e : 0.0;
            if (k == 0 || q > bs) { bs = q; best = k; }
        }
        kopt[i] = best;
    }
}

// cell of a centroid: the frame [-1/2, W - 1/2) in cells of side cs, clamped
__device__ __forceinline__ int iso_cell(double x, double y, double cs, int ncx, int ncy)
{
    int cx = (int)floor((x + 0.5) / cs), cy = (int)floor((y + 0.5) / cs);
    cx = cx < 0 ? 0 : (cx >= ncx ? ncx - 1 : cx);
    cy = cy < 0 ? 0 : (cy >= ncy ? ncy - 1 : cy);
    return cy * ncx + cx;
}

__global__ void __launch_bounds__(256) k_iso_count(const double* __restrict__ xs, const double* __restrict__ ys,
                                                   const int* __restrict__ n_dev, int cap, double cs, int ncx, int ncy,
                                                   int* count)
{
    const int n = min(*n_dev, cap);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        atomicAdd(count + iso_cell(xs[i], ys[i], cs, ncx, ncy), 1);
}

// exclusive scan of count into start (one CTA, chunks of 1024); fill cleared
__global__ void __launch_bounds__(1024) k_iso_scan(const int* __restrict__ count, int ncell, int* start, int* fill)
{
    __shared__ int part[32];
    __shared__ int carry;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    if (t == 0) carry = 0;
    __syncthreads();
    for (int c0 = 0; c0 < ncell; c0 += 1024) {
        const int i = c0 + t;
        const int v = i < ncell ? count[i] : 0;
        int inc = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) part[w] = inc;
        __syncthreads();
        if (w == 0) {
            int p = part[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, p, o);
                if (lane >= o) p += y;
            }
            part[lane] = p;
        }
        __syncthreads();
        const int base = carry + (w ? part[w - 1] : 0);
        if (i < ncell) {
            start[i] = base + inc - v;
            fill[i] = 0;
        }
        __syncthreads();
        if (t == 1023) carry = base + inc;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(256) k_iso_fill(const double* __restrict__ xs, const double* __restrict__ ys,
                                                  const int* __restrict__ n_dev, int cap, double cs, int ncx, int ncy,
                                                  const int* __restrict__ start, int* fill, int* items)
{
    const int n = min(*n_dev, cap);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int c = iso_cell(xs[i], ys[i], cs, ncx, ncy);
        items[start[c] + atomicAdd(fill + c, 1)] = i;
    }
}

// isolation (no other centroid closer than d_iso) and the calibrator test
__global__ void __launch_bounds__(256) k_iso_calib(const double* __restrict__ xs, const double* __restrict__ ys,
                                                   const int* __restrict__ n_dev, int cap, double cs, int ncx, int ncy,
                                                   double d_iso, const int* __restrict__ start,
                                                   const int* __restrict__ count, const int* __restrict__ items,
                                                   const uint32_t* __restrict__ cflags,
                                                   const uint32_t* __restrict__ gflags, const double* __restrict__ flux,
                                                   const double* __restrict__ ferr, const float* __restrict__ nu,
                                                   const int* __restrict__ kopt, int nr, double snr_min,
                                                   const __grid_constant__ RoptRadii rad, uint8_t* calib, double2* xy)
{
    const int n = min(*n_dev, cap);
    const double d2 = d_iso * d_iso;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double x = xs[i], y = ys[i];
        const int c = iso_cell(x, y, cs, ncx, ncy), cx = c % ncx, cy = c / ncx;
        bool iso = true;
        for (int gy = max(cy - 1, 0); gy <= min(cy + 1, ncy - 1) && iso; ++gy)
            for (int gx = max(cx - 1, 0); gx <= min(cx + 1, ncx - 1) && iso; ++gx) {
                const int g = gy * ncx + gx;
                for (int q = start[g]; q < start[g] + count[g]; ++q) {
                    const int j = items[q];
                    if (j == i) continue;
                    const double dx = xs[j] - x, dy = ys[j] - y;
                    if (dx * dx + dy * dy < d2) { iso = false; break; }
                }
            }
        bool ok = iso && cflags[i] == 0u && nu[i] > 0.f;
        for (int k = 0; k < nr && ok; ++k) ok = gflags[(int64_t)i * nr + k] == 0u;
        if (ok) {
            const int k = kopt[i];
            const double e = ferr[(int64_t)i * nr + k];
            ok = (e > 0.0 ? flux[(int64_t)i * nr + k] / e : 0.0) >= snr_min;
        }
        calib[i] = ok ? 1 : 0;
        // the fit's coordinates of a calibrator, here where every row has a
        // thread (float64 logarithms are slow; the fit is one CTA)
        if (ok) xy[i] = make_double2(log10((double)nu[i]), log10((double)rad.r[kopt[i]]));
    }
}

// sum of v over the block in a fixed order (thread partials, then a tree)
__device__ double block_sum(double v, double* red)
{
    const int t = threadIdx.x;
    red[t] = v;
    __syncthreads();
    for (int o = FIT_NT / 2; o > 0; o >>= 1) {
        if (t < o) red[t] += red[t + o];
        __syncthreads();
    }
    const double s = red[0];
    __syncthreads();
    return s;
}

__global__ void __launch_bounds__(FIT_NT) k_ropt_fit(const int* __restrict__ n_dev, int cap,
                                                    const uint8_t* __restrict__ calib,
                                                    const double2* __restrict__ xy, double* fit)
{
    __shared__ double red[FIT_NT];
    const int n = min(*n_dev, cap);
    const int t = threadIdx.x;
    double c = 0.0, sx = 0.0, sy = 0.0, xmin = INFINITY, xmax = -INFINITY;
    for (int i = t; i < n; i += FIT_NT) {
        if (!calib[i]) continue;
        const double2 q = xy[i];
        const double x = q.x, y = q.y;
        c += 1.0; sx += x; sy += y;
        xmin = fmin(xmin, x); xmax = fmax(xmax, x);
    }
    const double cnt = block_sum(c, red);
    const double Sx = block_sum(sx, red), Sy = block_sum(sy, red);
    // the spread test compares the extreme values themselves
    red[t] = xmin;
    __syncthreads();
    for (int o = FIT_NT / 2; o > 0; o >>= 1) {
        if (t < o) red[t] = fmin(red[t], red[t + o]);
        __syncthreads();
    }
    const double Xmin = red[0];
    __syncthreads();
    red[t] = xmax;
    __syncthreads();
    for (int o = FIT_NT / 2; o > 0; o >>= 1) {
        if (t < o) red[t] = fmax(red[t], red[t + o]);
        __syncthreads();
    }
    const double Xmax = red[0];
    __syncthreads();
    if (cnt < 3.0 || !(Xmax > Xmin)) {
        if (t == 0) { fit[0] = NAN; fit[1] = NAN; fit[2] = cnt; fit[3] = 1.0; }
        return;
    }
    const double mx = Sx / cnt, my = Sy / cnt;
    double sxx = 0.0, sxy = 0.0;
    for (int i = t; i < n; i += FIT_NT) {
        if (!calib[i]) continue;
        const double2 q = xy[i];
        const double dx = q.x - mx, dy = q.y - my;
        sxx = fma(dx, dx, sxx);
        sxy = fma(dx, dy, sxy);
    }
    const double Sxx = block_sum(sxx, red), Sxy = block_sum(sxy, red);
    if (t == 0) {
        const double a = Sxy / Sxx;
        fit[0] = a; fit[1] = my - a * mx; fit[2] = cnt; fit[3] = 0.0;
    }
}

__global__ void __launch_bounds__(256) k_ropt_assign(const int* __restrict__ n_dev, int cap,
                                                     const uint8_t* __restrict__ calib, const float* __restrict__ nu,
                                                     const int* __restrict__ kopt,
                                                     const __grid_constant__ RoptRadii rad,
                                                     const double* __restrict__ fit, const double* __restrict__ flux,
                                                     const double* __restrict__ ferr, int* kfinal, double* flux_opt,
                                                     double* ferr_opt)
{
    const int n = min(*n_dev, cap);
    const int nr = rad.nr;
    const double a = fit[0], b = fit[1];
    const bool ok = fit[3] == 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int k = 0;
        if (calib[i]) {
            k = kopt[i];
        } else if (ok && nu[i] > 0.f) {
            const double rf = exp10(fma(a, log10((double)nu[i]), b));
            double bd = INFINITY;
            for (int q = 0; q < nr; ++q) {
                const double d = fabs((double)rad.r[q] - rf);
                if (d <= bd) { bd = d; k = q; }      // ascending radii: ties go to the larger
            }
        }
        kfinal[i] = k;
        flux_opt[i] = flux[(int64_t)i * nr + k];
        ferr_opt[i] = ferr[(int64_t)i * nr + k];
    }
}

// cells of side cs >= d_iso, at most about 2^20 of them
void iso_grid(int W, int H, float d_iso, double* cs, int* ncx, int* ncy)
{
    double c = d_iso > 1.f ? (double)d_iso : 1.0;
    const double floor_c = ceil(sqrt((double)W * (double)H / (double)(1 << 20)));
    if (c < floor_c) c = floor_c;
    *cs = c;
    *ncx = (int)ceil((double)W / c) + 1;
    *ncy = (int)ceil((double)H / c) + 1;
}

cudaError_t launch_ropt(const Image& im, const SplineTab& sb, const SplineTab& sr, const float* taps, int kw, int kh,
                        const gp_catalog& cat, const double* flux, const double* ferr, const uint32_t* gflags,
                        const int* radii, int nr, float snr_min, float d_iso, const RoptWork& w, float* nu,
                        int* kopt, uint8_t* calib, int* kfinal, double* flux_opt, double* ferr_opt, double* fit,
                        cudaStream_t st)
{
    RoptRadii R;
    memset(&R, 0, sizeof R);
    R.nr = nr;
    for (int k = 0; k < nr; ++k) R.r[k] = radii[k];
    RoptTaps K;
    memset(&K, 0, sizeof K);
    K.kw = kw; K.kh = kh;
    for (int i = 0; i < kw * kh; ++i) K.t[i] = taps[i];
    const int cap = cat.capacity;
    const int grid = std::max(1, std::min((cap + 255) / 256, 152 * 8));
    if (im.is_f32)
        k_ropt_nu<true><<<grid, 256, 0, st>>>(im, sb, sr, K, cat.xpeak, cat.ypeak, flux, ferr, nr, cat.n, cap, nu, kopt);
    else
        k_ropt_nu<false><<<grid, 256, 0, st>>>(im, sb, sr, K, cat.xpeak, cat.ypeak, flux, ferr, nr, cat.n, cap, nu,
                                               kopt);
    double cs;
    int ncx, ncy;
    iso_grid(im.W, im.H, d_iso, &cs, &ncx, &ncy);
    const int ncell = ncx * ncy;
    cudaError_t e = cudaMemsetAsync(w.count, 0, (size_t)ncell * sizeof(int), st);
    if (e != cudaSuccess) return e;
    k_iso_count<<<grid, 256, 0, st>>>(cat.x, cat.y, cat.n, cap, cs, ncx, ncy, w.count);
    k_iso_scan<<<1, 1024, 0, st>>>(w.count, ncell, w.start, w.fill);
    k_iso_fill<<<grid, 256, 0, st>>>(cat.x, cat.y, cat.n, cap, cs, ncx, ncy, w.start, w.fill, w.items);
    k_iso_calib<<<grid, 256, 0, st>>>(cat.x, cat.y, cat.n, cap, cs, ncx, ncy, (double)d_iso, w.start, w.count, w.items,
                                      cat.flags, gflags, flux, ferr, nu, kopt, nr, (double)snr_min, R, calib, w.xy);
    k_ropt_fit<<<1, FIT_NT, 0, st>>>(cat.n, cap, calib, w.xy, fit);
    k_ropt_assign<<<grid, 256, 0, st>>>(cat.n, cap, calib, nu, kopt, R, fit, flux, ferr, kfinal, flux_opt, ferr_opt);
    return cudaGetLastError();
}

}  // namespace gp
