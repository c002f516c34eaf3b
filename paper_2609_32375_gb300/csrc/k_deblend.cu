// k_deblend.cu -- multi-threshold deblending of the segments (the
// SExtractor reading of the detection; the paper's own detection takes local
// maxima).  For a segment S of at least 2 minarea pixels, with
// nu = F / sigma its significance:
//  - levels t_i = k (nu_max / k)^(i / N), i = 0..N-1, with k the detection
//    threshold and nu_max the segment's peak;
//  - the branches of level i are the 8-connected components of
//    {p in S : nu(p) > t_i} (level 0: S itself);
//  - a branch is significant when it has minarea pixels and its sum of m
//    exceeds mincont times the segment's (the segment's sum must be > 0);
//  - from the root up: a branch passes on to its significant children (two
//    or more: a split, each examined in turn; one: it continues there); a
//    branch without one is a seed;
//  - with two or more seeds the other pixels are attributed by growth from
//    the seeds within the level sets, from the highest level down: in rounds,
//    an unattributed pixel of the level set takes the smallest seed rank
//    among its attributed 8-neighbours (ranks in the order of the seeds'
//    first pixels); the objects are labelled 1 + their minimum linear index.
//
// One CTA per candidate segment, its bounding box in global scratch.  Sums
// of m are exact 64-bit fixed-point integers (m scaled by 2^20), the level
// sets' components come from a lock-free union-find whose roots are the
// components' minimum pixels, and the growth is synchronous, so the result
// does not depend on the order in which threads run.  The objects' catalog
// rows are formed from float64 sums in a fixed order and ranked by label.
#include <math.h>
#include <string.h>

#include <algorithm>

#include "gp_internal.cuh"
#include "gp_launch.h"

namespace gp {

constexpr int DB_NT = 512;
constexpr int DB_MAX_SEEDS = 1024;
constexpr int DB_MAX_LEVELS = 64;            // nthresh at most (checked by the API)
constexpr double DB_FIX = 1048576.0;         // 2^20

struct DeblendArgs {
    Image im;
    SplineTab sb, sr;
    int kw, kh;
    float taps[KMAX];
    float thresh;
    int minarea, nthresh;
    double mincont;
    uint32_t* seg;
    // the catalog rows of the segments
    const int* n_dev;
    int cap;
    const uint32_t* label;
    const int* npix;
    const int *xmin, *xmax, *ymin, *ymax;
    // candidates and scratch
    int* cand;
    int* cand_count;
    int64_t* off;            // [cand] first scratch byte of each candidate (-1: no room)
    char* scratch;
    // objects: staging rows, then the caller's catalog in label order
    DbObj* obj;
    int* obj_count;
    int obj_stage_cap;
    int* counts;             // [2] segments split, objects
    int* status;
};

// the scratch arrays of a candidate with area A and halo area AH
struct DbScratch {
    float* mh;      // [AH] m over the box and the filter halo
    float* nu;      // [A]  nu, -1 outside the segment
    long long* mf;  // [A]  m in fixed point
    int* lab;       // [A]  union-find of the current level
    int* act;       // [A]  active node of the pixel (-1 none)
    int* seed;      // [A]  seed id + 1 (0 none)
    long long* fs;  // [A + 1] branch sums
    int* cnt;       // [A + 1] branch pixel counts; then seed ranks
    int* sig;       // [A + 1] significant branch (root) / node with a significant child
    int* own;       // [A]  object rank (0 none)
    int* own2;      // [A]
    int* first;     // [A + 1] first pixel of each seed
};

__device__ DbScratch db_scratch(char* base, int A, int AH)
{
    DbScratch s;
    char* p = base;
    auto take = [&](size_t bytes) { char* q = p; p += (bytes + 15) & ~(size_t)15; return q; };
    s.mh = reinterpret_cast<float*>(take((size_t)AH * 4));
    s.nu = reinterpret_cast<float*>(take((size_t)A * 4));
    s.mf = reinterpret_cast<long long*>(take((size_t)A * 8));
    s.lab = reinterpret_cast<int*>(take((size_t)A * 4));
    s.act = reinterpret_cast<int*>(take((size_t)A * 4));
    s.seed = reinterpret_cast<int*>(take((size_t)A * 4));
    s.fs = reinterpret_cast<long long*>(take((size_t)(A + 1) * 8));
    s.cnt = reinterpret_cast<int*>(take((size_t)(A + 1) * 4));
    s.sig = reinterpret_cast<int*>(take((size_t)(A + 1) * 4));
    s.own = reinterpret_cast<int*>(take((size_t)A * 4));
    s.own2 = reinterpret_cast<int*>(take((size_t)A * 4));
    s.first = reinterpret_cast<int*>(take((size_t)(A + 1) * 4));
    return s;
}

__host__ __device__ inline int64_t db_scratch_bytes(int64_t A, int64_t AH)
{
    auto r = [](int64_t b) { return (b + 15) & ~(int64_t)15; };
    return r(AH * 4) + r(A * 4) + r(A * 8) + 4 * r(A * 4) + r((A + 1) * 8) + 2 * r((A + 1) * 4) + r((A + 1) * 4) +
           r(A * 4);
}

__device__ int db_find(int* lab, int x)
{
    for (int n = 0; n < (1 << 24); ++n) {
        const int p = lab[x];
        if (p == x) return x;
        const int g = lab[p];
        if (g != p) lab[x] = g;
        x = g;
    }
    return x;
}

// the root of x without writing: the flatten pass must not shorten paths,
// since a path-halving store based on a stale read could overwrite a root
// that another warp has just stored (the unions before it may halve paths)
__device__ int db_root(const int* lab, int x)
{
    for (int n = 0; n < (1 << 24); ++n) {
        const int p = lab[x];
        if (p == x) return x;
        x = p;
    }
    return x;
}

__device__ void db_unite(int* lab, int a, int b)
{
    for (int n = 0; n < (1 << 24); ++n) {
        a = db_find(lab, a);
        b = db_find(lab, b);
        if (a == b) return;
        if (a < b) { const int t = a; a = b; b = t; }
        const int old = atomicMin(lab + a, b);
        if (old == a) return;
        a = old;
    }
}

// fixed-order block reductions
__device__ double db_sum(double v, double* red)
{
    const int t = threadIdx.x;
    red[t] = v;
    __syncthreads();
    for (int o = DB_NT / 2; o > 0; o >>= 1) {
        if (t < o) red[t] += red[t + o];
        __syncthreads();
    }
    const double s = red[0];
    __syncthreads();
    return s;
}

template <bool F32>
__global__ void __launch_bounds__(DB_NT) k_deblend(const __grid_constant__ DeblendArgs A)
{
    __shared__ double red[DB_NT];
    __shared__ long long redl[DB_NT];
    __shared__ int nseed_s;
    __shared__ int seeds[DB_MAX_SEEDS];        // first pixel of each seed, then sorted
    __shared__ int seedid[DB_MAX_SEEDS];
    __shared__ unsigned olab[DB_MAX_SEEDS];    // minimum frame index of each object
    __shared__ float tlev[DB_MAX_LEVELS + 1];  // the level thresholds, rounded down to float
    __shared__ int fr_n[2];                    // growth: candidates of this round, of the next
    const int t = threadIdx.x;
    const Image& im = A.im;
    const int W = im.W, H = im.H;
    const int ncand = *A.cand_count;
    const int hx = A.kw / 2, hy = A.kh / 2;
    for (int ci = blockIdx.x; ci < ncand; ci += gridDim.x) {
        const int r = A.cand[ci];
        const uint32_t L = A.label[r];
        const int x0 = A.xmin[r], x1 = A.xmax[r], y0 = A.ymin[r], y1 = A.ymax[r];
        const int w = x1 - x0 + 1, h = y1 - y0 + 1, Ar = w * h;
        const int wh = w + 2 * hx, hh = h + 2 * hy, AH = wh * hh;
        if (A.off[ci] < 0) continue;                       // no room: left as it is (status set)
        DbScratch s = db_scratch(A.scratch + A.off[ci], Ar, AH);
        // ---- m over the box and halo, then nu and fixed-point m in the segment
        for (int q = t; q < AH; q += DB_NT) {
            const int qy = q / wh, qx = q - qy * wh;
            const int x = mirror_idx(x0 - hx + qx, W), y = mirror_idx(y0 - hy + qy, H);
            bool bad;
            const float v = load_px<F32>(im, x, y, bad);
            s.mh[q] = bad ? 0.f : v - spline_eval(A.sb, (float)x, (float)y);
        }
        __syncthreads();
        long long tot = 0;
        float numax = -INFINITY;
        for (int q = t; q < Ar; q += DB_NT) {
            const int qy = q / w, qx = q - qy * w;
            const int x = x0 + qx, y = y0 + qy;
            const bool in = A.seg[(int64_t)y * W + x] == L;
            float nu = -1.f;
            long long mf = 0;
            if (in) {
                float F = 0.f;
                for (int v = 0; v < A.kh; ++v)
                    for (int u = 0; u < A.kw; ++u) F = fmaf(A.taps[v * A.kw + u], s.mh[(qy + v) * wh + qx + u], F);
                const float sg = spline_eval(A.sr, (float)x, (float)y);
                nu = sg > 0.f ? F / sg : 0.f;
                mf = llrint((double)s.mh[(qy + hy) * wh + qx + hx] * DB_FIX);
                numax = fmaxf(numax, nu);
            }
            s.nu[q] = in ? nu : -INFINITY;
            s.mf[q] = mf;
            tot += mf;
            s.act[q] = in ? Ar : -1;              // level 0: the whole segment is node Ar
            s.seed[q] = 0;
        }
        redl[t] = tot;
        red[t] = numax;
        __syncthreads();
        for (int o = DB_NT / 2; o > 0; o >>= 1) {
            if (t < o) { redl[t] += redl[t + o]; red[t] = fmax(red[t], red[t + o]); }
            __syncthreads();
        }
        const long long total = redl[0];
        const double nu_max = red[0];
        __syncthreads();
        if (!(total > 0) || !(nu_max > (double)A.thresh)) continue;
        // a branch always holds a local maximum of nu (its largest value), so a
        // segment with fewer than two (plateaus counted per pixel) cannot split
        int nmax = 0;
        for (int q = t; q < Ar; q += DB_NT) {
            const float v = s.nu[q];
            if (v == -INFINITY) continue;
            const int qy = q / w, qx = q - qy * w;
            bool mx = true;
            for (int dy = -1; dy <= 1 && mx; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    const int yy = qy + dy, xx = qx + dx;
                    if ((dy || dx) && yy >= 0 && yy < h && xx >= 0 && xx < w && s.nu[yy * w + xx] > v) { mx = false; break; }
                }
            nmax += mx ? 1 : 0;
        }
        redl[t] = nmax;
        __syncthreads();
        for (int o = DB_NT / 2; o > 0; o >>= 1) {
            if (t < o) redl[t] += redl[t + o];
            __syncthreads();
        }
        const long long nmaxima = redl[0];
        __syncthreads();
        if (nmaxima < 2) continue;
        const double cthr = A.mincont * (double)total;
        const double lr = log(nu_max / (double)A.thresh);
        // t_i = thresh (nu_max / thresh)^(i / nthresh), once per level, in
        // float64, rounded down to float: for a float nu, nu > t_i exactly
        // when nu > rd(t_i), so every comparison below is one of floats
        for (int i = t; i <= A.nthresh; i += DB_NT)
            tlev[i] = __double2float_rd((double)A.thresh * exp(lr * (double)i / (double)A.nthresh));
        __syncthreads();
        // ---- the branch tree, one level at a time, over the list of the
        // pixels still active (own: this level's list, first: the next
        // level's).  A pixel leaves the list when it leaves the tree, and its
        // lab is then -1 for good; the nodes the listed pixels point to are
        // listed pixels themselves (a significant branch's root stays in it)
        // or node Ar.  Roots are the components' smallest pixels and the
        // sums are exact, so the list order does not matter.
        int* lst = s.own;
        int* lnx = s.first;
        if (t == 0) { fr_n[0] = 0; fr_n[1] = 0; }
        __syncthreads();
        for (int q = t; q < Ar; q += DB_NT) {
            s.lab[q] = -1;
            if (s.act[q] >= 0) lst[atomicAdd(&fr_n[0], 1)] = q;
        }
        __syncthreads();
        for (int i = 0; i + 1 < A.nthresh; ++i) {
            const float tl = tlev[i + 1];
            const int nl = fr_n[0];
            for (int k = t; k < nl; k += DB_NT) {
                const int q = lst[k];
                s.lab[q] = s.nu[q] > tl ? q : -1;
                s.fs[q] = 0; s.cnt[q] = 0; s.sig[q] = 0;
            }
            if (t == 0) { s.fs[Ar] = 0; s.cnt[Ar] = 0; s.sig[Ar] = 0; fr_n[1] = 0; }
            __syncthreads();
            for (int k = t; k < nl; k += DB_NT) {
                const int q = lst[k];
                if (s.lab[q] < 0) continue;
                const int qy = q / w, qx = q - qy * w;
                // the neighbours before q in raster order: W, NW, N, NE
                if (qx > 0 && s.lab[q - 1] >= 0) db_unite(s.lab, q, q - 1);
                if (qy > 0) {
                    const int u = q - w;
                    if (qx > 0 && s.lab[u - 1] >= 0) db_unite(s.lab, q, u - 1);
                    if (s.lab[u] >= 0) db_unite(s.lab, q, u);
                    if (qx + 1 < w && s.lab[u + 1] >= 0) db_unite(s.lab, q, u + 1);
                }
            }
            __syncthreads();
            // roots into a second array (own2 is free until the growth)
            int* root = s.own2;
            for (int k = t; k < nl; k += DB_NT) {
                const int q = lst[k];
                root[q] = s.lab[q] >= 0 ? db_root(s.lab, q) : -1;
            }
            __syncthreads();
            for (int k = t; k < nl; k += DB_NT) {
                const int q = lst[k];
                const int rt = root[q];
                if (rt < 0) continue;
                atomicAdd(reinterpret_cast<unsigned long long*>(s.fs + rt), (unsigned long long)s.mf[q]);
                atomicAdd(s.cnt + rt, 1);
            }
            __syncthreads();
            // a significant branch marks its parent node (the active node of its pixels)
            for (int k = t; k < nl; k += DB_NT) {
                const int q = lst[k];
                if (root[q] != q) continue;
                if (s.cnt[q] >= A.minarea && (double)s.fs[q] > cthr) {
                    atomicOr(s.sig + q, 1);
                    atomicOr(s.sig + s.act[q], 2);
                }
            }
            __syncthreads();
            for (int k = t; k < nl; k += DB_NT) {
                const int q = lst[k];
                const int node = s.act[q];
                if (!(s.sig[node] & 2)) {           // no significant child: the node is a seed
                    s.seed[q] = node + 1;
                    s.act[q] = -1;
                    s.lab[q] = -1;
                } else if (root[q] >= 0 && (s.sig[root[q]] & 1)) {
                    s.act[q] = root[q];
                    lnx[atomicAdd(&fr_n[1], 1)] = q;
                } else {
                    s.act[q] = -1;
                    s.lab[q] = -1;
                }
            }
            __syncthreads();
            int* tmp = lst; lst = lnx; lnx = tmp;
            if (t == 0) fr_n[0] = fr_n[1];
            __syncthreads();
            if (fr_n[0] == 0) break;
        }
        {
            const int nl = fr_n[0];
            for (int k = t; k < nl; k += DB_NT) {
                const int q = lst[k];
                s.seed[q] = s.act[q] + 1;
            }
        }
        __syncthreads();
        // ---- the seeds, in the order of their first pixels
        for (int q = t; q <= Ar; q += DB_NT) s.first[q] = INT_MAX;
        if (t == 0) nseed_s = 0;
        __syncthreads();
        for (int q = t; q < Ar; q += DB_NT)
            if (s.seed[q]) atomicMin(s.first + s.seed[q] - 1, q);
        __syncthreads();
        for (int q = t; q < Ar; q += DB_NT) {
            if (s.seed[q] && s.first[s.seed[q] - 1] == q) {
                const int k = atomicAdd(&nseed_s, 1);
                if (k < DB_MAX_SEEDS) { seeds[k] = q; seedid[k] = s.seed[q] - 1; }
            }
        }
        __syncthreads();
        const int ns = nseed_s;
        if (ns > DB_MAX_SEEDS) {
            if (t == 0) set_status(A.status, GP_ERR_CAPACITY);
            continue;
        }
        if (ns < 2) continue;
        // rank of each seed by its first pixel (first pixels are distinct)
        for (int k = t; k < ns; k += DB_NT) {
            int rk = 0;
            for (int j = 0; j < ns; ++j) rk += seeds[j] < seeds[k];
            s.cnt[seedid[k]] = rk + 1;
        }
        __syncthreads();
        // own: the object rank of each pixel (0 none); own2: the round in which
        // the pixel was assigned (seeds 0; -1 unassigned, -2 a candidate of
        // the coming round)
        for (int q = t; q < Ar; q += DB_NT) {
            const int v = s.seed[q] ? s.cnt[s.seed[q] - 1] : 0;
            s.own[q] = v;
            s.own2[q] = v > 0 ? 0 : -1;
        }
        __syncthreads();
        // ---- growth within the level sets, from the highest level down, in
        // synchronous rounds: in a round every unassigned pixel of the level
        // set with an assigned 8-neighbour takes the smallest object rank
        // among the neighbours assigned before the round.  A level's first
        // round finds its candidates by a scan of the box; after that a
        // pixel can become a candidate only through a neighbour assigned in
        // the round before (one assigned earlier would have made it one
        // already), so each later round visits the neighbours of the last
        // round's pixels only.  Lists: lab (this round's candidates), act
        // (the next round's), first (their new ranks).
        int* cur = s.own;
        int* stamp = s.own2;
        int* lc = s.lab;
        int* ln = s.act;
        int* nr = s.first;
        int round = 0;
        for (int i = A.nthresh - 1; i >= 0; --i) {
            const float tl = tlev[i];
            auto eligible = [&](int q) { return s.nu[q] > -INFINITY && (i == 0 || s.nu[q] > tl); };
            if (t == 0) { fr_n[0] = 0; fr_n[1] = 0; }
            __syncthreads();
            for (int q = t; q < Ar; q += DB_NT) {
                if (cur[q] != 0 || !eligible(q)) continue;
                const int qy = q / w, qx = q - qy * w;
                bool adj = false;
                for (int dy = -1; dy <= 1 && !adj; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        const int yy = qy + dy, xx = qx + dx;
                        if ((dy || dx) && yy >= 0 && yy < h && xx >= 0 && xx < w && cur[yy * w + xx] > 0) { adj = true; break; }
                    }
                if (adj) {
                    stamp[q] = -2;
                    lc[atomicAdd(&fr_n[0], 1)] = q;
                }
            }
            __syncthreads();
            for (;;) {
                const int nc = fr_n[0];
                if (nc == 0) break;
                ++round;
                // the new ranks, from the state before the round
                for (int k = t; k < nc; k += DB_NT) {
                    const int q = lc[k];
                    const int qy = q / w, qx = q - qy * w;
                    int best = INT_MAX;
                    for (int dy = -1; dy <= 1; ++dy)
                        for (int dx = -1; dx <= 1; ++dx) {
                            if (!dy && !dx) continue;
                            const int yy = qy + dy, xx = qx + dx;
                            if (yy < 0 || yy >= h || xx < 0 || xx >= w) continue;
                            const int o = yy * w + xx;
                            if (stamp[o] >= 0 && stamp[o] < round && cur[o] < best) best = cur[o];
                        }
                    nr[k] = best;
                }
                __syncthreads();
                for (int k = t; k < nc; k += DB_NT) {
                    const int q = lc[k];
                    cur[q] = nr[k];
                    stamp[q] = round;
                }
                if (t == 0) fr_n[1] = 0;
                __syncthreads();
                // the next round's candidates: unassigned neighbours in the level set
                for (int k = t; k < nc; k += DB_NT) {
                    const int q = lc[k];
                    const int qy = q / w, qx = q - qy * w;
                    for (int dy = -1; dy <= 1; ++dy)
                        for (int dx = -1; dx <= 1; ++dx) {
                            if (!dy && !dx) continue;
                            const int yy = qy + dy, xx = qx + dx;
                            if (yy < 0 || yy >= h || xx < 0 || xx >= w) continue;
                            const int o = yy * w + xx;
                            if (stamp[o] == -1 && eligible(o) && atomicCAS(stamp + o, -1, -2) == -1)
                                ln[atomicAdd(&fr_n[1], 1)] = o;
                        }
                }
                __syncthreads();
                int* tmp = lc; lc = ln; ln = tmp;
                if (t == 0) fr_n[0] = fr_n[1];
                __syncthreads();
            }
        }
        // ---- labels: 1 + the minimum linear index of each object
        for (int k = t; k < ns; k += DB_NT) olab[k] = 0xffffffffu;
        __syncthreads();
        for (int q = t; q < Ar; q += DB_NT) {
            const int o = cur[q];
            if (o > 0) atomicMin(olab + o - 1, (unsigned)((y0 + q / w) * W + x0 + q % w));
        }
        __syncthreads();
        for (int q = t; q < Ar; q += DB_NT) {
            const int o = cur[q];
            if (o > 0) A.seg[(int64_t)(y0 + q / w) * W + x0 + q % w] = olab[o - 1] + 1u;
        }
        // ---- each object's catalog row (float64 sums in a fixed order,
        // coordinates about the box corner)
        for (int k = 1; k <= ns; ++k) {
            double c = 0, sm = 0, sx = 0, sy = 0, sxx = 0, syy = 0, sxy = 0, ux = 0, uy = 0, uxx = 0, uyy = 0, uxy = 0;
            int bx0 = INT_MAX, bx1 = -1, by0 = INT_MAX, by1 = -1, sat = 0;
            float pk = -INFINITY;
            int pq = INT_MAX;
            for (int q = t; q < Ar; q += DB_NT) {
                if (cur[q] != k) continue;
                const int qy = q / w, qx = q - qy * w;
                const double m = (double)s.mh[(qy + hy) * wh + qx + hx];
                const double x = qx, y = qy;
                c += 1; sm += m; sx += x * m; sy += y * m; sxx += x * x * m; syy += y * y * m; sxy += x * y * m;
                ux += x; uy += y; uxx += x * x; uyy += y * y; uxy += x * y;
                bx0 = min(bx0, qx); bx1 = max(bx1, qx); by0 = min(by0, qy); by1 = max(by1, qy);
                const float mv = s.mh[(qy + hy) * wh + qx + hx];
                if (mv > pk || (mv == pk && q < pq)) { pk = mv; pq = q; }
                if (im.sat > 0.f) {
                    bool bad;
                    if (load_px<F32>(im, x0 + qx, y0 + qy, bad) >= im.sat) sat = 1;
                }
            }
            c = db_sum(c, red); sm = db_sum(sm, red); sx = db_sum(sx, red); sy = db_sum(sy, red);
            sxx = db_sum(sxx, red); syy = db_sum(syy, red); sxy = db_sum(sxy, red);
            ux = db_sum(ux, red); uy = db_sum(uy, red); uxx = db_sum(uxx, red); uyy = db_sum(uyy, red);
            uxy = db_sum(uxy, red);
            // integer and peak reductions through the shared arrays
            __shared__ int ri[4][DB_NT];
            __shared__ float rp[DB_NT];
            __shared__ int rq[DB_NT];
            ri[0][t] = bx0; ri[1][t] = -bx1; ri[2][t] = by0; ri[3][t] = -by1;
            rp[t] = pk; rq[t] = pq;
            redl[t] = sat;
            __syncthreads();
            for (int o = DB_NT / 2; o > 0; o >>= 1) {
                if (t < o) {
                    for (int j = 0; j < 4; ++j) ri[j][t] = min(ri[j][t], ri[j][t + o]);
                    if (rp[t + o] > rp[t] || (rp[t + o] == rp[t] && rq[t + o] < rq[t])) { rp[t] = rp[t + o]; rq[t] = rq[t + o]; }
                    redl[t] |= redl[t + o];
                }
                __syncthreads();
            }
            if (t == 0) {
                const int idx = atomicAdd(A.obj_count, 1);
                if (idx < A.obj_stage_cap) {
                    DbObj o;
                    o.label = olab[k - 1] + 1u;
                    o.parent = L;
                    o.npix = (int)c;
                    uint32_t fl = redl[0] ? GP_FLAG_SAT : 0u;
                    double xm, ym, x2, y2, xy;
                    if (sm > 0.0) {
                        xm = sx / sm; ym = sy / sm;
                        x2 = sxx / sm - xm * xm; y2 = syy / sm - ym * ym; xy = sxy / sm - xm * ym;
                    } else {
                        xm = ux / c; ym = uy / c;
                        x2 = uxx / c - xm * xm; y2 = uyy / c - ym * ym; xy = uxy / c - xm * ym;
                        fl |= GP_FLAG_CENTROID_FALLBACK;
                    }
                    o.flux = sm;
                    o.x = xm + x0; o.y = ym + y0; o.x2 = x2; o.y2 = y2; o.xy = xy;
                    o.xmin = x0 + ri[0][0]; o.xmax = x0 - ri[1][0]; o.ymin = y0 + ri[2][0]; o.ymax = y0 - ri[3][0];
                    o.peak = rp[0];
                    o.xpeak = x0 + rq[0] % w; o.ypeak = y0 + rq[0] / w;
                    o.flags = fl;
                    A.obj[idx] = o;
                } else {
                    set_status(A.status, GP_ERR_CAPACITY);
                }
            }
            __syncthreads();
        }
        if (t == 0) {
            atomicAdd(A.counts, 1);
            atomicAdd(A.counts + 1, ns);
        }
        __syncthreads();
    }
}

// candidates: rows with at least 2 minarea pixels, their scratch bytes
__global__ void __launch_bounds__(256) k_db_select(const int* __restrict__ n_dev, int cap,
                                                   const int* __restrict__ npix, const int* __restrict__ xmin,
                                                   const int* __restrict__ xmax, const int* __restrict__ ymin,
                                                   const int* __restrict__ ymax, int minarea, int hx, int hy,
                                                   int* cand, int* cand_count, int64_t* bytes)
{
    const int n = min(*n_dev, cap);
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        if (npix[r] < 2 * minarea) continue;
        const int64_t w = xmax[r] - xmin[r] + 1, h = ymax[r] - ymin[r] + 1;
        const int k = atomicAdd(cand_count, 1);
        cand[k] = r;
        bytes[k] = db_scratch_bytes(w * h, (w + 2 * hx) * (h + 2 * hy));
    }
}

// scratch offsets (exclusive scan of the bytes, one CTA); a candidate beyond
// the scratch gets -1 and the status records it
__global__ void __launch_bounds__(1024) k_db_offsets(const int* __restrict__ cand_count, int64_t* bytes_off,
                                                     int64_t cap_bytes, int* status)
{
    __shared__ long long part[32];
    __shared__ long long carry;
    const int t = threadIdx.x, lane = t & 31, wp = t >> 5;
    const int n = *cand_count;
    if (t == 0) carry = 0;
    __syncthreads();
    for (int c0 = 0; c0 < n; c0 += 1024) {
        const int i = c0 + t;
        const long long v = i < n ? bytes_off[i] : 0;
        long long inc = v;
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) part[wp] = inc;
        __syncthreads();
        if (wp == 0) {
            long long p = part[lane];
            for (int o = 1; o < 32; o <<= 1) {
                const long long y = __shfl_up_sync(0xffffffffu, p, o);
                if (lane >= o) p += y;
            }
            part[lane] = p;
        }
        __syncthreads();
        const long long base = carry + (wp ? part[wp - 1] : 0);
        if (i < n) {
            const long long o = base + inc - v;
            const bool fits = o + v <= cap_bytes;
            bytes_off[i] = fits ? o : -1;
            if (!fits) set_status(status, GP_ERR_CAPACITY);
        }
        __syncthreads();
        if (t == 1023) carry = base + inc;
        __syncthreads();
    }
}

// the staged object rows in label order (rank by count; labels are distinct)
__global__ void __launch_bounds__(256) k_db_place(const DbObj* __restrict__ obj, const int* __restrict__ obj_count,
                                                  int stage_cap, gp_catalog out)
{
    const int n = min(*obj_count, stage_cap);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint32_t L = obj[i].label;
        int rk = 0;
        for (int j = 0; j < n; ++j) rk += obj[j].label < L;
        if (rk >= out.capacity) continue;
        const DbObj& o = obj[i];
        out.label[rk] = o.label; out.npix[rk] = o.npix; out.flux_iso[rk] = o.flux;
        out.x[rk] = o.x; out.y[rk] = o.y; out.x2[rk] = o.x2; out.y2[rk] = o.y2; out.xy[rk] = o.xy;
        out.xmin[rk] = o.xmin; out.xmax[rk] = o.xmax; out.ymin[rk] = o.ymin; out.ymax[rk] = o.ymax;
        out.peak[rk] = o.peak; out.xpeak[rk] = o.xpeak; out.ypeak[rk] = o.ypeak; out.flags[rk] = o.flags;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *out.n = n;
}

cudaError_t launch_deblend(const Image& im, const SplineTab& sb, const SplineTab& sr, const float* taps, int kw,
                           int kh, float thresh, int minarea, int nthresh, float mincont, uint32_t* seg,
                           const gp_catalog& cat, const DeblendWork& w, const gp_catalog& objects, int* counts,
                           int* status, cudaStream_t st)
{
    DeblendArgs A;
    memset(&A, 0, sizeof A);
    A.im = im; A.sb = sb; A.sr = sr;
    A.kw = kw; A.kh = kh;
    for (int i = 0; i < kw * kh; ++i) A.taps[i] = taps[i];
    A.thresh = thresh; A.minarea = minarea; A.nthresh = nthresh; A.mincont = mincont;
    A.seg = seg;
    A.n_dev = cat.n; A.cap = cat.capacity;
    A.label = cat.label; A.npix = cat.npix;
    A.xmin = cat.xmin; A.xmax = cat.xmax; A.ymin = cat.ymin; A.ymax = cat.ymax;
    A.cand = w.cand; A.cand_count = w.cand_count; A.off = w.off;
    A.scratch = w.scratch;
    A.obj = w.obj; A.obj_count = w.obj_count; A.obj_stage_cap = w.obj_cap;
    A.counts = counts; A.status = status;
    cudaError_t e = cudaMemsetAsync(w.cand_count, 0, 2 * sizeof(int), st);   // candidates, objects
    if (e != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(counts, 0, 2 * sizeof(int), st)) != cudaSuccess) return e;
    const int grid = std::max(1, std::min((cat.capacity + 255) / 256, 152 * 8));
    k_db_select<<<grid, 256, 0, st>>>(cat.n, cat.capacity, cat.npix, cat.xmin, cat.xmax, cat.ymin, cat.ymax, minarea,
                                      kw / 2, kh / 2, w.cand, w.cand_count, w.off);
    k_db_offsets<<<1, 1024, 0, st>>>(w.cand_count, w.off, w.scratch_bytes, status);
    if (im.is_f32) k_deblend<true><<<152 * 2, DB_NT, 0, st>>>(A);
    else k_deblend<false><<<152 * 2, DB_NT, 0, st>>>(A);
    k_db_place<<<grid, 256, 0, st>>>(w.obj, w.obj_count, w.obj_cap, objects);
    return cudaGetLastError();
}

}  // namespace gp
