/*
 * oracle.c -- plain, slow, FP64 CPU statement of the per-frame extraction.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or
 * calls this file: only tests/, the smoke check and bench.py's CPU-baseline
 * leg do.  It shares no code, header or table with the CUDA library.
 *
 * What is computed follows the paper's description of the local background
 * with a per-pixel noise map (Section 3.1), of the matched-filter detection
 * with a significance threshold and first-moment centroids (Section 3.2), and
 * of aperture sums accumulated in float64 with propagated variance
 * (Section 3.4).  The paper leaves most constants open; the readings used are
 * tagged [R#] and listed with their reasons in the design notes:
 *   [R2]  mesh boxes of side B, the last one partial; centre (w-1)/2 in-box
 *   [R3]  iterative k-sigma clip about the median, population std, stop when
 *         the kept set is unchanged or after maxiter passes
 *   [R4]  box background = median if sigma==0 or |mean-median|/sigma > 0.3,
 *         else 2.5 median - 1.5 mean; box rms = sigma.  Parity unpinned: the
 *         mode rule is a reading (the SExtractor estimate); its branch choice
 *         and the symmetric case are pinned, its skewed-branch value is not
 *   [R5]  boxes with < 50 % good pixels are filled from valid neighbours
 *   [R6]  fsize x fsize median filter of each mesh, window clipped to mesh
 *   [R7]  tensor-product natural cubic spline through the box centres,
 *         linear extrapolation beyond the outer centres
 *   [R8]  filter = correlation with the kernel normalised to unit sum,
 *         mirror border without edge repeat
 *   [R10] foreground <=> F(p) > k sigma(p), strict
 *   [R11] 8-connectivity; [R12] label = 1 + min linear index, components
 *         with npix < minarea set to 0, no renumbering
 *   [R13] first and second moments of the unfiltered background-subtracted
 *         image over the segment
 *   [R14] exact disc/pixel overlap areas; error^2 = sum A sigma^2 + F/gain
 *
 * Plain algorithms throughout: sorting for medians, breadth-first flood fill
 * for labelling, direct double loops for the filter, piecewise exact
 * integration for the overlap area.
 *
 * Threads: the loops over independent outputs (boxes, map columns, filtered
 * rows, aperture sources) may run on several host threads (OpenMP, when the
 * compiler has it); each output is computed by one thread in the same
 * arithmetic order as with one, so the results do not depend on the thread
 * count.  Labelling and moments stay sequential.  orc_set_threads(1) gives
 * the plain single-threaded definition.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* threads for the loops above (n < 1: all the host's); returns the count used */
int orc_set_threads(int n)
{
#ifdef _OPENMP
    omp_set_num_threads(n >= 1 ? n : omp_get_num_procs());
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

#define ORC_FLAG_SAT 1u
#define ORC_FLAG_CENTROID_FALLBACK 2u
#define ORC_FLAG_TRUNCATED 4u
#define ORC_FLAG_BAD 8u

static int cmp_double(const void* a, const void* b)
{
    double x = *(const double*)a, y = *(const double*)b;
    return (x > y) - (x < y);
}

/* median of a sorted array: middle value, or mean of the two middle ones */
static double median_sorted(const double* v, long n)
{
    if (n <= 0) return 0.0;
    if (n & 1) return v[n / 2];
    return 0.5 * (v[n / 2 - 1] + v[n / 2]);
}

/* --------------------------------------------------------------------------
 * [R3][R4] sigma-clipped statistics of one set of values (Section 3.1 local
 * background; the sigma-clip primitive the paper also uses for the
 * reference PSF stack and the zero point).
 *
 * vals: n good values (modified: sorted in place).  Outputs the final
 * median, mean, population std and kept count.  Returns the number of clip
 * passes that removed values.
 * ------------------------------------------------------------------------ */
int orc_sigma_clip(double* vals, long n, double k, int maxiter,
                   double* med_out, double* mean_out, double* std_out, long* nkept_out)
{
    qsort(vals, (size_t)n, sizeof(double), cmp_double);
    /* the kept set stays a sorted array: clipping keeps a sub-sequence */
    double* kept = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    memcpy(kept, vals, sizeof(double) * (size_t)n);
    long nk = n;
    int passes = 0;
    double med = 0, mean = 0, sd = 0;
    for (int it = 0;; ++it) {
        med = median_sorted(kept, nk);
        double s = 0;
        for (long i = 0; i < nk; ++i) s += kept[i];
        mean = nk ? s / (double)nk : 0.0;
        double ss = 0;
        for (long i = 0; i < nk; ++i) ss += (kept[i] - mean) * (kept[i] - mean);
        sd = nk ? sqrt(ss / (double)nk) : 0.0;
        if (it >= maxiter) break;
        double lo = med - k * sd, hi = med + k * sd;
        long m = 0;
        for (long i = 0; i < nk; ++i)
            if (kept[i] >= lo && kept[i] <= hi) kept[m++] = kept[i];
        if (m == nk) break; /* unchanged: converged */
        nk = m;
        ++passes;
    }
    *med_out = med;
    *mean_out = mean;
    *std_out = sd;
    *nkept_out = nk;
    free(kept);
    return passes;
}

/* [R4] the box background from the clipped statistics */
double orc_mode_estimate(double med, double mean, double sd)
{
    if (sd == 0.0 || fabs(mean - med) / sd > 0.3) return med;
    return 2.5 * med - 1.5 * mean;
}

/* --------------------------------------------------------------------------
 * [R2][R3][R4] per-box statistics over the mesh.  img, bad: W*H row-major.
 * Outputs My*Mx arrays (row-major, My rows of Mx boxes).  valid[b] = 1 if at
 * least half the box's pixels are good.
 * ------------------------------------------------------------------------ */
int orc_box_stats(const double* img, const uint8_t* bad, int W, int H, int B,
                  double k, int maxiter, double* bkg, double* rms, uint8_t* valid,
                  double* med_out, double* mean_out, long* nkept_out)
{
    int Mx = (W + B - 1) / B, My = (H + B - 1) / B;
#pragma omp parallel
    {
    double* buf = (double*)malloc(sizeof(double) * (size_t)B * (size_t)B);
#pragma omp for schedule(dynamic, 1)
    for (int b0 = 0; b0 < Mx * My; ++b0) {
            const int j = b0 / Mx, i = b0 % Mx;
            int x0 = i * B, x1 = (i + 1) * B < W ? (i + 1) * B : W;
            int y0 = j * B, y1 = (j + 1) * B < H ? (j + 1) * B : H;
            long n = 0;
            for (int y = y0; y < y1; ++y)
                for (int x = x0; x < x1; ++x) {
                    long p = (long)y * W + x;
                    if (!bad[p]) buf[n++] = img[p];
                }
            long area = (long)(x1 - x0) * (y1 - y0);
            int b = j * Mx + i;
            double med, mean, sd;
            long nk;
            orc_sigma_clip(buf, n, k, maxiter, &med, &mean, &sd, &nk);
            valid[b] = (2 * n >= area && n > 0);
            bkg[b] = valid[b] ? orc_mode_estimate(med, mean, sd) : 0.0;
            rms[b] = valid[b] ? sd : 0.0;
            if (med_out) med_out[b] = med;
            if (mean_out) mean_out[b] = mean;
            if (nkept_out) nkept_out[b] = nk;
        }
    free(buf);
    }
    return 0;
}

/* [R5] fill invalid boxes with the mean of their valid 8-neighbours,
 * sweep after sweep, until every box is valid.  All boxes invalid: zeros. */
int orc_fill_invalid(double* bkg, double* rms, uint8_t* valid, int Mx, int My)
{
    int nb = Mx * My, any = 0;
    for (int b = 0; b < nb; ++b) any |= valid[b];
    if (!any) {
        for (int b = 0; b < nb; ++b) { bkg[b] = 0; rms[b] = 0; valid[b] = 1; }
        return 0;
    }
    uint8_t* nv = (uint8_t*)malloc((size_t)nb);
    double* nbk = (double*)malloc(sizeof(double) * (size_t)nb);
    double* nrm = (double*)malloc(sizeof(double) * (size_t)nb);
    for (;;) {
        int missing = 0;
        memcpy(nv, valid, (size_t)nb);
        memcpy(nbk, bkg, sizeof(double) * (size_t)nb);
        memcpy(nrm, rms, sizeof(double) * (size_t)nb);
        for (int j = 0; j < My; ++j)
            for (int i = 0; i < Mx; ++i) {
                int b = j * Mx + i;
                if (valid[b]) continue;
                double sb = 0, sr = 0;
                int c = 0;
                for (int dj = -1; dj <= 1; ++dj)
                    for (int di = -1; di <= 1; ++di) {
                        int ii = i + di, jj = j + dj;
                        if ((di || dj) && ii >= 0 && ii < Mx && jj >= 0 && jj < My &&
                            valid[jj * Mx + ii]) {
                            sb += bkg[jj * Mx + ii];
                            sr += rms[jj * Mx + ii];
                            ++c;
                        }
                    }
                if (c) { nbk[b] = sb / c; nrm[b] = sr / c; nv[b] = 1; }
                else missing = 1;
            }
        memcpy(valid, nv, (size_t)nb);
        memcpy(bkg, nbk, sizeof(double) * (size_t)nb);
        memcpy(rms, nrm, sizeof(double) * (size_t)nb);
        if (!missing) break;
    }
    free(nv); free(nbk); free(nrm);
    return 0;
}

/* [R6] fsize x fsize median filter, window clipped at the mesh edge */
int orc_median_filter(const double* in, double* out, int Mx, int My, int fsize)
{
    int h = fsize / 2;
    double win[64 * 64];
    if (fsize > 63) return -1;
    for (int j = 0; j < My; ++j)
        for (int i = 0; i < Mx; ++i) {
            int c = 0;
            for (int jj = j - h; jj <= j + h; ++jj)
                for (int ii = i - h; ii <= i + h; ++ii)
                    if (ii >= 0 && ii < Mx && jj >= 0 && jj < My) win[c++] = in[jj * Mx + ii];
            qsort(win, (size_t)c, sizeof(double), cmp_double);
            out[j * Mx + i] = median_sorted(win, c);
        }
    return 0;
}

/* --------------------------------------------------------------------------
 * [R7] natural cubic spline along one axis.
 * Second derivatives M (M[0] = M[n-1] = 0) from the tridiagonal system
 *   h[i-1] M[i-1] + 2 (h[i-1] + h[i]) M[i] + h[i] M[i+1]
 *       = 6 ((v[i+1]-v[i])/h[i] - (v[i]-v[i-1])/h[i-1]),
 * solved by plain forward elimination / back substitution.
 * ------------------------------------------------------------------------ */
static void spline_second_derivs(const double* t, const double* v, int n, double* M)
{
    for (int i = 0; i < n; ++i) M[i] = 0.0;
    if (n < 3) return;
    int m = n - 2;
    double* a = (double*)malloc(sizeof(double) * (size_t)m);
    double* b = (double*)malloc(sizeof(double) * (size_t)m);
    double* c = (double*)malloc(sizeof(double) * (size_t)m);
    double* d = (double*)malloc(sizeof(double) * (size_t)m);
    for (int r = 0; r < m; ++r) {
        int i = r + 1;
        double h0 = t[i] - t[i - 1], h1 = t[i + 1] - t[i];
        a[r] = h0; b[r] = 2.0 * (h0 + h1); c[r] = h1;
        d[r] = 6.0 * ((v[i + 1] - v[i]) / h1 - (v[i] - v[i - 1]) / h0);
    }
    for (int r = 1; r < m; ++r) {
        double w = a[r] / b[r - 1];
        b[r] -= w * c[r - 1];
        d[r] -= w * d[r - 1];
    }
    M[m] = d[m - 1] / b[m - 1];
    for (int r = m - 2; r >= 0; --r) M[r + 1] = (d[r] - c[r] * M[r + 2]) / b[r];
    free(a); free(b); free(c); free(d);
}

/* value of the natural spline at x; linear beyond the end nodes */
static double spline_eval(const double* t, const double* v, const double* M, int n, double x)
{
    if (n == 1) return v[0];
    if (x <= t[0]) {
        double h = t[1] - t[0];
        double s0 = (v[1] - v[0]) / h - h * (2.0 * M[0] + M[1]) / 6.0;
        return v[0] + s0 * (x - t[0]);
    }
    if (x >= t[n - 1]) {
        double h = t[n - 1] - t[n - 2];
        double s1 = (v[n - 1] - v[n - 2]) / h + h * (M[n - 2] + 2.0 * M[n - 1]) / 6.0;
        return v[n - 1] + s1 * (x - t[n - 1]);
    }
    int i = 0;
    while (i < n - 2 && x > t[i + 1]) ++i;
    double h = t[i + 1] - t[i];
    double Bc = (x - t[i]) / h, Ac = 1.0 - Bc;
    return v[i] + Bc * (v[i + 1] - v[i]) +
           h * h / 6.0 * ((Ac * Ac * Ac - Ac) * M[i] + (Bc * Bc * Bc - Bc) * M[i + 1]);
}

/* [R2] box centres along one axis */
static void box_centres(int N, int B, int nb, double* t)
{
    for (int i = 0; i < nb; ++i) {
        int w = ((i + 1) * B < N ? (i + 1) * B : N) - i * B;
        t[i] = i * B + (w - 1) / 2.0;
    }
}

/* [R7] tensor-product spline of a mesh at the pixel positions (xs[q], ys[q]):
 * spline along x through each mesh row, then along y through those values. */
int orc_spline_at(const double* mesh, int Mx, int My, int W, int H, int B,
                  const double* xs, const double* ys, long nq, double* out)
{
    double* tx = (double*)malloc(sizeof(double) * (size_t)Mx);
    double* ty = (double*)malloc(sizeof(double) * (size_t)My);
    double* Mrow = (double*)malloc(sizeof(double) * (size_t)Mx * My);
    double* u = (double*)malloc(sizeof(double) * (size_t)My);
    double* Mu = (double*)malloc(sizeof(double) * (size_t)My);
    box_centres(W, B, Mx, tx);
    box_centres(H, B, My, ty);
    for (int j = 0; j < My; ++j) spline_second_derivs(tx, mesh + (size_t)j * Mx, Mx, Mrow + (size_t)j * Mx);
    for (long q = 0; q < nq; ++q) {
        for (int j = 0; j < My; ++j)
            u[j] = spline_eval(tx, mesh + (size_t)j * Mx, Mrow + (size_t)j * Mx, Mx, xs[q]);
        spline_second_derivs(ty, u, My, Mu);
        out[q] = spline_eval(ty, u, Mu, My, ys[q]);
    }
    free(tx); free(ty); free(Mrow); free(u); free(Mu);
    return 0;
}

/* [R7] the full W*H map: one y-spline per pixel column */
int orc_spline_map(const double* mesh, int Mx, int My, int W, int H, int B, double* map)
{
    double* tx = (double*)malloc(sizeof(double) * (size_t)Mx);
    double* ty = (double*)malloc(sizeof(double) * (size_t)My);
    double* Mrow = (double*)malloc(sizeof(double) * (size_t)Mx * My);
    box_centres(W, B, Mx, tx);
    box_centres(H, B, My, ty);
    for (int j = 0; j < My; ++j) spline_second_derivs(tx, mesh + (size_t)j * Mx, Mx, Mrow + (size_t)j * Mx);
#pragma omp parallel
    {
    double* u = (double*)malloc(sizeof(double) * (size_t)My);
    double* Mu = (double*)malloc(sizeof(double) * (size_t)My);
#pragma omp for schedule(static)
    for (int x = 0; x < W; ++x) {
        for (int j = 0; j < My; ++j)
            u[j] = spline_eval(tx, mesh + (size_t)j * Mx, Mrow + (size_t)j * Mx, Mx, (double)x);
        spline_second_derivs(ty, u, My, Mu);
        for (int y = 0; y < H; ++y) map[(size_t)y * W + x] = spline_eval(ty, u, Mu, My, (double)y);
    }
    free(u); free(Mu);
    }
    free(tx); free(ty); free(Mrow);
    return 0;
}

/* [R8] mirror index without edge repeat: -1 -> 1, N -> N-2 (periodic
 * reflection so any offset lands inside; N == 1 maps everything to 0) */
static long mirror(long i, long N)
{
    if (N == 1) return 0;
    long p = 2 * (N - 1);
    i %= p;
    if (i < 0) i += p;
    return i < N ? i : p - i;
}

/* [R8] matched filter F = K (*) m, a correlation with the kernel normalised
 * to unit sum (Section 3.2).  K is kh rows of kw taps.  Returns -1 if the
 * taps sum to zero. */
int orc_filter(const double* m, int W, int H, const double* K, int kw, int kh, double* F)
{
    double s = 0;
    for (int i = 0; i < kw * kh; ++i) s += K[i];
    if (s == 0.0) return -1;
    int hx = kw / 2, hy = kh / 2;
#pragma omp parallel for schedule(static)
    for (long y = 0; y < H; ++y)
        for (long x = 0; x < W; ++x) {
            double acc = 0;
            for (int v = -hy; v <= hy; ++v)
                for (int u = -hx; u <= hx; ++u)
                    acc += (K[(v + hy) * kw + (u + hx)] / s) * m[mirror(y + v, H) * W + mirror(x + u, W)];
            F[y * W + x] = acc;
        }
    return 0;
}

/* the same filter at selected pixels only */
int orc_filter_at(const double* m, int W, int H, const double* K, int kw, int kh,
                  const long* xs, const long* ys, long nq, double* out)
{
    double s = 0;
    for (int i = 0; i < kw * kh; ++i) s += K[i];
    if (s == 0.0) return -1;
    int hx = kw / 2, hy = kh / 2;
    for (long q = 0; q < nq; ++q) {
        double acc = 0;
        for (int v = -hy; v <= hy; ++v)
            for (int u = -hx; u <= hx; ++u)
                acc += (K[(v + hy) * kw + (u + hx)] / s) * m[mirror(ys[q] + v, H) * W + mirror(xs[q] + u, W)];
        out[q] = acc;
    }
    return 0;
}

/* --------------------------------------------------------------------------
 * [R11][R12] 8-connected component labelling by breadth-first flood fill.
 * Pixels are visited in raster order, so the first pixel of a component
 * reached is its minimum linear index L and the component gets label L+1.
 * Components smaller than minarea are set back to 0.  Returns the number of
 * components kept.
 * ------------------------------------------------------------------------ */
long orc_label(const uint8_t* fg, int W, int H, int minarea, uint32_t* seg)
{
    long N = (long)W * H, kept = 0;
    long* queue = (long*)malloc(sizeof(long) * (size_t)(N > 0 ? N : 1));
    memset(seg, 0, sizeof(uint32_t) * (size_t)N);
    for (long p = 0; p < N; ++p) {
        if (!fg[p] || seg[p]) continue;
        uint32_t lab = (uint32_t)(p + 1);
        long head = 0, tail = 0;
        queue[tail++] = p;
        seg[p] = lab;
        while (head < tail) {
            long q = queue[head++];
            long qx = q % W, qy = q / W;
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    long nx = qx + dx, ny = qy + dy;
                    if ((dx || dy) && nx >= 0 && nx < W && ny >= 0 && ny < H) {
                        long r = ny * W + nx;
                        if (fg[r] && !seg[r]) { seg[r] = lab; queue[tail++] = r; }
                    }
                }
        }
        if (tail < minarea)
            for (long i = 0; i < tail; ++i) seg[queue[i]] = 0;
        else
            ++kept;
    }
    free(queue);
    return kept;
}

/* --------------------------------------------------------------------------
 * [R13] per-segment moments of the unfiltered m over each label, catalog in
 * ascending label order (Section 3.2 first-moment centroid, extended to the
 * second moments, bounding box and peak).  sat: per-pixel saturation flags
 * (nullable).  Arrays are sized ncap; returns the number of segments.
 * Two passes: sums for S and the centroid, then central second moments.
 * ------------------------------------------------------------------------ */
long orc_moments(const uint32_t* seg, const double* m, const uint8_t* sat, int W, int H, long ncap,
                 uint32_t* label, long* npix, double* flux, double* xc, double* yc,
                 double* x2, double* y2, double* xy, int* xmin, int* xmax, int* ymin, int* ymax,
                 double* peak, int* xpeak, int* ypeak, uint32_t* flags)
{
    long N = (long)W * H, nc = 0;
    /* component index stored at the label's root pixel (first in raster order) */
    long* cidx = (long*)malloc(sizeof(long) * (size_t)(N > 0 ? N : 1));
    double *sx = (double*)calloc((size_t)ncap + 1, sizeof(double));
    double *sy = (double*)calloc((size_t)ncap + 1, sizeof(double));
    double *cnt_x = (double*)calloc((size_t)ncap + 1, sizeof(double));
    double *cnt_y = (double*)calloc((size_t)ncap + 1, sizeof(double));
    for (long p = 0; p < N; ++p) {
        uint32_t l = seg[p];
        if (!l) continue;
        long root = (long)l - 1;
        long c;
        if (root == p) {
            c = nc++;
            cidx[p] = c;
            if (c < ncap) {
                label[c] = l; npix[c] = 0; flux[c] = 0; flags[c] = 0;
                xmin[c] = xmax[c] = (int)(p % W);
                ymin[c] = ymax[c] = (int)(p / W);
                peak[c] = m[p]; xpeak[c] = (int)(p % W); ypeak[c] = (int)(p / W);
            }
        } else {
            c = cidx[root];
        }
        if (c >= ncap) continue;
        int x = (int)(p % W), y = (int)(p / W);
        npix[c] += 1;
        flux[c] += m[p];
        sx[c] += x * m[p];
        sy[c] += y * m[p];
        cnt_x[c] += x;
        cnt_y[c] += y;
        if (x < xmin[c]) xmin[c] = x;
        if (x > xmax[c]) xmax[c] = x;
        if (y < ymin[c]) ymin[c] = y;
        if (y > ymax[c]) ymax[c] = y;
        if (m[p] > peak[c]) { peak[c] = m[p]; xpeak[c] = x; ypeak[c] = y; }
        if (sat && sat[p]) flags[c] |= ORC_FLAG_SAT;
    }
    long nuse = nc < ncap ? nc : ncap;
    for (long c = 0; c < nuse; ++c) {
        if (flux[c] > 0) {
            xc[c] = sx[c] / flux[c];
            yc[c] = sy[c] / flux[c];
        } else {
            xc[c] = cnt_x[c] / (double)npix[c];
            yc[c] = cnt_y[c] / (double)npix[c];
            flags[c] |= ORC_FLAG_CENTROID_FALLBACK;
        }
        x2[c] = y2[c] = xy[c] = 0;
    }
    for (long p = 0; p < N; ++p) {
        uint32_t l = seg[p];
        if (!l) continue;
        long c = cidx[(long)l - 1];
        if (c >= ncap) continue;
        double dx = (double)(p % W) - xc[c], dy = (double)(p / W) - yc[c];
        double w = (flags[c] & ORC_FLAG_CENTROID_FALLBACK) ? 1.0 : m[p];
        x2[c] += dx * dx * w;
        y2[c] += dy * dy * w;
        xy[c] += dx * dy * w;
    }
    for (long c = 0; c < nuse; ++c) {
        double d = (flags[c] & ORC_FLAG_CENTROID_FALLBACK) ? (double)npix[c] : flux[c];
        x2[c] /= d; y2[c] /= d; xy[c] /= d;
    }
    free(cidx); free(sx); free(sy); free(cnt_x); free(cnt_y);
    return nc;
}

/* --------------------------------------------------------------------------
 * [R14] exact area of the intersection of the disc x^2 + y^2 <= r^2 with the
 * rectangle [x0,x1] x [y0,y1] (coordinates relative to the disc centre).
 *
 * The area is the integral over x of the length of [y0,y1] n [-h(x), h(x)],
 * h(x) = sqrt(r^2 - x^2).  Between the break points x = +-r and the x where
 * h(x) = |y0| or |y1|, the top of that interval is y1 or h(x) and its bottom
 * y0 or -h(x) throughout, so each piece integrates in closed form with the
 * antiderivative G(t) = (t h(t) + r^2 asin(t/r)) / 2 of h.
 * ------------------------------------------------------------------------ */
static double Gint(double t, double r)
{
    if (t >= r) return 0.25 * M_PI * r * r;
    if (t <= -r) return -0.25 * M_PI * r * r;
    return 0.5 * (t * sqrt(r * r - t * t) + r * r * asin(t / r));
}

double orc_overlap_area(double x0, double x1, double y0, double y1, double r)
{
    double a = x0 > -r ? x0 : -r, b = x1 < r ? x1 : r;
    if (!(a < b) || !(y0 < y1) || r <= 0) return 0.0;
    double pts[6];
    int np = 0;
    pts[np++] = a;
    pts[np++] = b;
    double ys[2] = {y0, y1};
    double cuts[4];
    int nc = 0;
    for (int k = 0; k < 2; ++k)
        if (fabs(ys[k]) < r) {
            double c = sqrt(r * r - ys[k] * ys[k]);
            cuts[nc++] = -c;
            cuts[nc++] = c;
        }
    for (int k = 0; k < nc; ++k)
        if (cuts[k] > a && cuts[k] < b) pts[np++] = cuts[k];
    qsort(pts, (size_t)np, sizeof(double), cmp_double);
    double area = 0.0;
    for (int k = 0; k + 1 < np; ++k) {
        double p = pts[k], q = pts[k + 1];
        if (!(q > p)) continue;
        double mid = 0.5 * (p + q);
        double h = sqrt(r * r - mid * mid);
        /* non-strict: h == y1 inside a piece only happens at a tangent
         * point (y1 == r), where h <= y1 holds on the whole piece */
        int top_is_h = h <= y1, bot_is_h = -h >= y0;
        double top = top_is_h ? h : y1, bot = bot_is_h ? -h : y0;
        if (top <= bot) continue;
        double gi = Gint(q, r) - Gint(p, r);
        double itop = top_is_h ? gi : y1 * (q - p);
        double ibot = bot_is_h ? -gi : y0 * (q - p);
        area += itop - ibot;
    }
    return area;
}

/* [R14] circular-aperture sums at (xs, ys) for each radius (Section 3.4:
 * float64 sums with the variance propagated through the same aperture).
 * m: background-subtracted image (0 at bad pixels); var: sigma(p)^2; bad,
 * sat: per-pixel flags (sat nullable).  Outputs n*nr arrays (source-major).
 * Only in-frame good pixels contribute; flags record saturated or bad
 * pixels under the disc and discs that leave the frame. */
int orc_apertures(const double* m, const double* var, const uint8_t* bad, const uint8_t* sat,
                  int W, int H, const double* xs, const double* ys, long n,
                  const double* radii, int nr, double gain,
                  double* flux, double* fluxerr, uint32_t* flags)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (long s = 0; s < n; ++s)
        for (int k = 0; k < nr; ++k) {
            double cx = xs[s], cy = ys[s], r = radii[k];
            double f = 0, v = 0;
            uint32_t fl = 0;
            if (cx - r < -0.5 || cx + r > W - 0.5 || cy - r < -0.5 || cy + r > H - 0.5)
                fl |= ORC_FLAG_TRUNCATED;
            long xa = (long)floor(cx - r - 0.5), xb = (long)ceil(cx + r + 0.5);
            long ya = (long)floor(cy - r - 0.5), yb = (long)ceil(cy + r + 0.5);
            for (long y = ya; y <= yb; ++y) {
                if (y < 0 || y >= H) continue;
                for (long x = xa; x <= xb; ++x) {
                    if (x < 0 || x >= W) continue;
                    double A = orc_overlap_area(x - 0.5 - cx, x + 0.5 - cx, y - 0.5 - cy, y + 0.5 - cy, r);
                    if (A <= 0) continue;
                    long p = y * W + x;
                    if (bad[p]) { fl |= ORC_FLAG_BAD; continue; }
                    if (sat && sat[p]) fl |= ORC_FLAG_SAT;
                    f += A * m[p];
                    v += A * var[p];
                }
            }
            if (gain > 0 && f > 0) v += f / gain;
            flux[s * nr + k] = f;
            fluxerr[s * nr + k] = sqrt(v);
            flags[s * nr + k] = fl;
        }
    return 0;
}

/* --------------------------------------------------------------------------
 * [R20][R21] growth curves by top-hat correlation (Section 3.4: circular
 * apertures of integer radii, each a cross-correlation of the frame with a
 * top-hat kernel, the variance map propagated through the same kernel,
 * float64 sums).  The top-hat of radius r is the set of integer offsets
 * (u, v) with u^2 + v^2 <= r^2; the correlation is sampled at the pixel
 * nearest the source position, (floor(x + 1/2), floor(y + 1/2)).  Pixels
 * outside the frame contribute nothing (TRUNCATED), bad pixels nothing (BAD),
 * saturated ones flag the sum (SAT).  err = sqrt(sum var + max(f, 0) / gain).
 * radii: nr integers, ascending.  Outputs n*nr arrays (source-major).
 * ------------------------------------------------------------------------ */
int orc_growth(const double* m, const double* var, const uint8_t* bad, const uint8_t* sat,
               int W, int H, const double* xs, const double* ys, long n,
               const int* radii, int nr, double gain,
               double* flux, double* fluxerr, uint32_t* flags)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (long s = 0; s < n; ++s) {
        long xc = (long)floor(xs[s] + 0.5), yc = (long)floor(ys[s] + 0.5);
        for (int k = 0; k < nr; ++k) {
            long r = radii[k];
            double f = 0, v = 0;
            uint32_t fl = 0;
            for (long dv = -r; dv <= r; ++dv)
                for (long du = -r; du <= r; ++du) {
                    if (du * du + dv * dv > r * r) continue;
                    long x = xc + du, y = yc + dv;
                    if (x < 0 || x >= W || y < 0 || y >= H) { fl |= ORC_FLAG_TRUNCATED; continue; }
                    long p = y * W + x;
                    if (bad[p]) { fl |= ORC_FLAG_BAD; continue; }
                    if (sat && sat[p]) fl |= ORC_FLAG_SAT;
                    f += m[p];
                    v += var[p];
                }
            if (gain > 0 && f > 0) v += f / gain;
            flux[s * nr + k] = f;
            fluxerr[s * nr + k] = sqrt(v);
            flags[s * nr + k] = fl;
        }
    }
    return 0;
}
