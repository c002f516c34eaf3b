// gp_internal.cuh -- device helpers and internal layouts of the extraction
// library (sm_103a).  Not part of the public ABI (include/gpphot.h is).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "gpphot.h"

namespace gp {

// ------------------------------------------- programmatic dependent launch ---
// A kernel launched by launch_dep may be scheduled while the kernel before it
// in the stream is finishing.  pdl_wait() blocks until that kernel has
// completed and its memory is visible; every such kernel calls it before its
// first access to global memory.  pdl_release() lets the next kernel start
// being scheduled (it still waits in its own pdl_wait()).  Both are no-ops in
// a kernel launched without the attribute.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KP, typename... A>
static inline cudaError_t launch_dep(void (*k)(KP...), dim3 g, dim3 b, size_t smem, cudaStream_t st, A&&... args)
{
    cudaLaunchConfig_t c = {};
    c.gridDim = g;
    c.blockDim = b;
    c.dynamicSmemBytes = smem;
    c.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    c.attrs = at;
    c.numAttrs = 1;
    return cudaLaunchKernelEx(&c, k, static_cast<A&&>(args)...);
}


// --------------------------------------------------- float64 reciprocals ---
// Float64 runs at a small fraction of the float32 rate on this GPU, and a
// float64 division or square root is a long instruction sequence.  These
// start from a float32 estimate and refine it with float64 Newton steps
// (two: within an ulp of the float64 result); arguments outside float32's
// range take the plain operation.

// 1 / x for x > 0
__device__ __forceinline__ double recip_pos(double x)
{
    const float xf = (float)x;
    if (!(xf > 1e-37f) || !(xf < 1e37f)) return 1.0 / x;
    double r = (double)(1.0f / xf);
    r = fma(r, fma(-x, r, 1.0), r);
    r = fma(r, fma(-x, r, 1.0), r);
    return r;
}

// sqrt(v) for v >= 0: s <- s + (v - s^2) / (2 s), with 1 / (2 s) taken
// once in float32 (the steps are tiny, so its error is squared away)
__device__ __forceinline__ double sqrt_pos(double v)
{
    const float vf = (float)v;
    if (!(vf > 1e-37f) || !(vf < 1e37f)) return v > 0.0 ? sqrt(v) : 0.0;
    const float s0f = sqrtf(vf);
    const double h = (double)(0.5f / s0f);
    double s = (double)s0f;
    s = fma(fma(-s, s, v), h, s);
    s = fma(fma(-s, s, v), h, s);
    return s;
}

// ------------------------------------------------------------ constants ---
constexpr int TX = 64;           // detection tile width  (pixels)
constexpr int TY = 32;           // detection tile height
constexpr int MAXRUN = TY * (TX / 2);   // most horizontal foreground runs a tile can hold
constexpr int HMAX = 7;          // largest filter half-size (15 x 15 taps)
constexpr int EDGE_PER_TILE = 2 * TY + 2 * TX;   // colL, colR, rowT, rowB
constexpr int MAX_NR = 8;        // most aperture radii per call

// streaming detection geometry: a lane filters 4 adjacent columns, a warp a
// 128-column strip (two detection tiles wide), a CTA ST_NW strips side by
// side over ST_RC rows; the packed foreground mask holds, per frame row and
// strip, four 32-bit words, word c bit l = column 4 l + c of the strip
constexpr int ST_CPL = 4;
// most foreground pixels of a tile that the labelling kernel's common form
// takes; a census of the listed tiles sends the ones above it to the
// crowded form
constexpr int LT_FG = 384;
constexpr int ST_STRIP = 32 * ST_CPL;

// default bound on the steps of a global union-find walk (a cycle would be a
// bug; the walk gives up, records GP_ERR_TIMEOUT and the result is flagged
// invalid); a context can lower it (gp_ctx_set_walk_limit)
constexpr int WALK_LIMIT = 1 << 22;

__device__ __forceinline__ void set_status(int* st, int code)
{
    atomicCAS(st, 0, code);  // the first error wins
}

// -------------------------------------------------------------- spline ---
// Mesh nodes along one axis: node i sits at i*B + (B-1)/2, except the last,
// which sits at the centre of the (possibly partial) last box.
struct Axis {
    int n;         // nodes
    float B;       // node spacing (box side)
    float t0;      // first node position
    float tl;      // last node position
    float hl;      // width of the last interval (tl - t[n-2])
};

// Coefficients of the natural-spline value at coordinate t, written as
//   f = v[i] + b (v[i1] - v[i]) + c0 M[i] + c1 M[i1]
// with v the node values and M their second derivatives.  Inside the node
// range this is the cubic spline; beyond the end nodes it is the linear
// continuation with the end slope (the natural spline's second derivative is
// zero there).  Written in this shifted form so that constant data give the
// constant back exactly.
struct AxCoef {
    int i, i1;
    float b, c0, c1;
};

__host__ __device__ inline Axis make_axis(int N, int B)
{
    Axis a;
    a.n = (N + B - 1) / B;
    a.B = (float)B;
    int w0 = (B < N ? B : N);
    a.t0 = 0.5f * (float)(w0 - 1);
    int wl = N - (a.n - 1) * B;
    a.tl = (float)((a.n - 1) * B) + 0.5f * (float)(wl - 1);
    a.hl = a.n > 1 ? a.tl - ((float)((a.n - 2) * B) + 0.5f * (float)(B - 1)) : 0.f;
    return a;
}

__device__ __forceinline__ AxCoef axis_coef(const Axis& a, float t)
{
    AxCoef c;
    if (a.n == 1) {
        c.i = c.i1 = 0;
        c.b = c.c0 = c.c1 = 0.f;
        return c;
    }
    if (t < a.t0) {
        float h = (a.n == 2) ? a.hl : a.B;
        float d = t - a.t0;
        c.i = 0; c.i1 = 1;
        c.b = d / h;
        c.c0 = -d * h * (1.f / 3.f);
        c.c1 = -d * h * (1.f / 6.f);
        return c;
    }
    if (t > a.tl) {
        float h = a.hl;
        float d = t - a.tl;
        c.i = a.n - 2; c.i1 = a.n - 1;
        c.b = 1.f + d / h;
        c.c0 = d * h * (1.f / 6.f);
        c.c1 = d * h * (1.f / 3.f);
        return c;
    }
    int i = (int)floorf((t - a.t0) / a.B);
    i = i < 0 ? 0 : (i > a.n - 2 ? a.n - 2 : i);
    float ti = a.t0 + (float)i * a.B;
    float h = (i == a.n - 2) ? a.hl : a.B;
    float b = (t - ti) / h;
    float aa = 1.f - b;
    float h26 = h * h * (1.f / 6.f);
    c.i = i; c.i1 = i + 1;
    c.b = b;
    c.c0 = h26 * (aa * aa * aa - aa);
    c.c1 = h26 * (b * b * b - b);
    return c;
}

__device__ __forceinline__ float axis_combine(const AxCoef& c, float v0, float v1, float m0, float m1)
{
    return fmaf(c.c1, m1, fmaf(c.c0, m0, fmaf(c.b, v1 - v0, v0)));
}

// Per-node table of one map: (P value, X = d2P/dx2 along the row,
// Y = d2P/dy2 along the column, XY = d2Y/dx2 along the row).  The value at
// (x, y) is the y-spline through u_j = x-spline(P[j], X[j]) whose node second
// derivatives are w_j = x-spline(Y[j], XY[j]) -- the tensor-product natural
// spline evaluated with precomputed derivatives.
struct SplineTab {
    const float4* node;   // [ny][nx]
    Axis ax, ay;
};

__device__ __forceinline__ float2 row_eval(const SplineTab& s, int j, const AxCoef& cx)
{
    const float4 n0 = s.node[j * s.ax.n + cx.i];
    const float4 n1 = s.node[j * s.ax.n + cx.i1];
    float2 r;
    r.x = axis_combine(cx, n0.x, n1.x, n0.y, n1.y);   // u_j(x)
    r.y = axis_combine(cx, n0.z, n1.z, n0.w, n1.w);   // w_j(x)
    return r;
}

__device__ __forceinline__ float spline_eval(const SplineTab& s, float x, float y)
{
    AxCoef cx = axis_coef(s.ax, x);
    AxCoef cy = axis_coef(s.ay, y);
    float2 r0 = row_eval(s, cy.i, cx);
    float2 r1 = row_eval(s, cy.i1, cx);
    return axis_combine(cy, r0.x, r1.x, r0.y, r1.y);
}

// ----------------------------------------------- compensated FP32 sums ---
// A float-float accumulator: hi carries the running sum, lo the rounding
// errors (TwoSum), so sums of many FP32 terms keep about 48 bits.
struct DF {
    float hi, lo;
};

__device__ __forceinline__ DF df_zero() { DF d; d.hi = 0.f; d.lo = 0.f; return d; }

__device__ __forceinline__ void df_add(DF& s, float v)
{
    float t = s.hi + v;
    float bp = t - s.hi;
    float e = (s.hi - (t - bp)) + (v - bp);
    s.hi = t;
    s.lo += e;
}

// add the exact product a*b (TwoProduct with an FMA)
__device__ __forceinline__ void df_add_prod(DF& s, float a, float b)
{
    float p = a * b;
    float e = fmaf(a, b, -p);
    df_add(s, p);
    s.lo += e;
}

__device__ __forceinline__ DF df_merge(DF a, DF b)
{
    float t = a.hi + b.hi;
    float bp = t - a.hi;
    float e = (a.hi - (t - bp)) + (b.hi - bp);
    DF r;
    r.hi = t;
    r.lo = a.lo + b.lo + e;
    return r;
}

// butterfly reduction over a full warp; every lane ends with the same value,
// the combination order is fixed, so the result is reproducible
__device__ __forceinline__ DF df_warp_sum(DF v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        DF w;
        w.hi = __shfl_xor_sync(0xffffffffu, v.hi, o);
        w.lo = __shfl_xor_sync(0xffffffffu, v.lo, o);
        // combine in lane order so both partners compute the same bits
        bool lower = (threadIdx.x & o) == 0;
        v = lower ? df_merge(v, w) : df_merge(w, v);
    }
    return v;
}

__device__ __forceinline__ double df_value(DF d) { return (double)d.hi + (double)d.lo; }

// ------------------------------------------------------------- borders ---
// mirror reflection without edge repeat (-1 -> 1, N -> N-2), periodic so any
// offset lands inside; N == 1 maps to 0
__host__ __device__ __forceinline__ int mirror_idx(int i, int N)
{
    if (N == 1) return 0;
    int p = 2 * (N - 1);
    i %= p;
    if (i < 0) i += p;
    return i < N ? i : p - i;
}

// ---------------------------------------------------- workspace layout ---
// Partial moments of the pixels of one piece of a segment, relative to an
// origin (the piece's tile corner): compensated sums of m, dx m, dy m,
// dx^2 m, dy^2 m, dx dy m; the same unweighted (integers, for segments whose
// sum is not positive); peak value and its linear index; flag bits.
struct Moments {
    float2 s, sx, sy, sxx, syy, sxy;   // (hi, lo) pairs
    int ux, uy, uxx, uyy, uxy;
    float peak;
    uint32_t peakL;
    uint32_t flags;
};

// Pieces: the parts of segments that touch a detection-tile edge shared
// with another tile; they are merged across tiles by union-find.
struct Pieces {
    int* count;           // scalar
    int cap;
    uint32_t* root;       // min linear index of the piece
    int* npix;
    int4* bbox;           // xmin, xmax, ymin, ymax (frame coordinates)
    int* parent;          // union-find over piece ids
    int* proot;           // union-find root after the merge
    uint32_t* agg_min;    // at a root piece: min linear index of the whole segment
    int* agg_npix;
    int4* agg_bbox;
    Moments* mom;         // partial moments, origin = the piece's tile corner
};

struct Mom2 {
    double x2, y2, xy, pad;
};

__host__ __device__ __forceinline__ Mom2 mom2_make(double x2, double y2, double xy, double pad)
{
    Mom2 m;
    m.x2 = x2; m.y2 = y2; m.xy = xy; m.pad = pad;
    return m;
}

// Segments that survive the minarea cut, in no particular order until ranked,
// with their finished moments
struct Comps {
    int* count;           // scalar
    int cap;
    uint32_t* label;
    int* npix;
    int4* bbox;
    double* flux;         // sum of m
    double2* xy;          // centroid
    Mom2* mom2;           // x2, y2, xy
    float* peak;
    uint32_t* peakL;
    uint32_t* flags;
    int* perm;            // rank -> component id
    int* slots;           // bucket scatter space
    int* bcnt;            // per label bucket counts
    int* boff;            // exclusive offsets
    int* bcur;            // scatter cursors
    int nb;               // number of buckets
    int shift;            // bucket = (label - 1) >> shift
};

struct Tiles {
    int ntx, nty;
    int16_t* edges;       // [ntiles][EDGE_PER_TILE] local piece index or -1
    int* piece_base;      // [ntiles] first piece id of the tile
    int* piece_cnt;       // [ntiles]
};

// the threshold mask of a frame, packed (k_stream), and the detection tiles
// that hold foreground
struct DetMask {
    uint4* bits;          // [H][ceil(W / ST_STRIP)]
    int* tl_list;         // [ntiles] appended tile indices
    int* tl_count;        // scalar, cleared per call
    int* dl_list;         // [ntiles] tiles with more than LT_FG foreground pixels (the tile census lists them)
    int* dl_count;        // scalar, cleared per call
    int* rl_list;         // [ntiles] tiles the labelling kernel's common form defers (more than its runs)
    int* rl_count;        // scalar, cleared per call
};

struct Image {
    const void* data;
    int64_t pitch;
    const uint8_t* mask;
    int W, H;
    float sat;
    int is_f32;
};

// one pixel's value and whether it is bad (masked, or NaN / Inf in an FP32
// frame); (x, y) must lie inside the frame
template <bool F32>
__device__ __forceinline__ float load_px(const Image& im, int x, int y, bool& bad)
{
    float v;
    if (F32) {
        v = __ldg(reinterpret_cast<const float*>(im.data) + (int64_t)y * im.pitch + x);
        bad = !isfinite(v);
    } else {
        v = (float)__ldg(reinterpret_cast<const uint16_t*>(im.data) + (int64_t)y * im.pitch + x);
        bad = false;
    }
    if (im.mask && im.mask[(int64_t)y * im.W + x]) bad = true;
    return v;
}

// ------------------------------------------------ per-frame arguments ---
// Every kernel of the pipeline runs either one frame, its arguments passed
// by value (`one`, a __grid_constant__ parameter, so taking its address
// makes no copy), or a batch of frames whose argument records sit in a
// device array (`batch`), one per frame: the grid's y index is the frame,
// and blocks beyond a smaller frame's extent return at once.  A batch of
// small frames thus runs each stage as a single launch.
template <class T>
__device__ __forceinline__ const T& frame_args(const T* __restrict__ batch, const T& one)
{
    return batch ? batch[blockIdx.y] : one;
}

// most frames in one batched launch
constexpr int MAX_BATCH = 64;

// per-box statistics (k_boxstats_*)
struct BoxArgs {
    const void* img;
    int64_t pitch;
    const uint8_t* mask;
    int W, H, B, Mx, nbox, npad;
    double k;
    int maxiter;
    double* bkg;
    double* rms;
    int* valid;
    float* quant;
    int* fb_list;     // uint16 boxes the windowed histogram could not finish (appended), or
    int* fb_count;    // for the full-histogram kernel, the list it works through; null: every box
};

// mesh fill, median filter and spline tables in shared memory (k_mesh_all)
struct MeshArgs {
    const double* bkg_raw;
    const double* rms_raw;
    const int* valid;
    Axis ax, ay;
    int fsize, mode;
    float* bkg_mesh;
    float* rms_mesh;
    float4* tab_b;
    float4* tab_r;
};

constexpr int KMAX = (2 * HMAX + 1) * (2 * HMAX + 1);

// detection (k_stream, k_pack_mask, k_label_tiles, k_merge)
struct DetectArgs {
    // the normalised kernel, padded to ks x ks (ks odd), as a sum of nrank
    // separable terms: K[v][u] = sum_r fv[r ks + v] fh[r ks + u]
    float fv[KMAX], fh[KMAX];
    int ks, nrank;
    Image im;
    SplineTab sb, sr;
    float thresh;
    int minarea;
    uint32_t* seg;
    uint8_t* mask_out;
    int* nnear;
    const uint8_t* in_mask;   // labelling of a given mask
    uint4* bits;              // packed foreground mask [H][nstrip]
    int nstrip;               // ceil(W / ST_STRIP)
    int* tl_list;             // detection tiles holding foreground (appended)
    int* tl_count;
    int* dl_list;             // of those, the ones with more than LT_FG foreground pixels (crowded form)
    int* dl_count;
    int* rl_list;             // of the others, the ones the common form defers (crowded form, after it)
    int* rl_count;
    Tiles T;
    Pieces P;
    Comps C;
    int* status;
};

// tile merge, piece aggregation and finalisation (k_merge, k_aggregate,
// k_finalize)
struct ResolveArgs {
    Tiles T;
    Pieces P;
    Comps C;
    uint32_t* seg;
    const int* tl_list;       // tiles holding foreground (the only ones with pieces)
    const int* tl_count;
    int W, H, minarea;
    int walk_limit;           // steps a union-find walk may take before it gives up (GP_ERR_TIMEOUT)
    int* status;
};

// label ranking (k_rank_*)
struct RankArgs {
    Comps C;
    int* n_out;
    int capacity;
    int place;
    int* status;
};

struct ApSpec {
    int nr;
    float r[MAX_NR];
    float rmax;
    float gain;
    double inv_gain;    // 1 / gain (0 when gain <= 0): Poisson variance F / gain as a product
};

// catalog rows and apertures (k_measure)
struct MeasureArgs {
    Image im;
    SplineTab sb, sr;
    Comps C;
    int capacity;
    // catalog columns
    uint32_t* label;
    int32_t* npix;
    double *flux_iso, *x, *y, *x2, *y2, *xy;
    int32_t *xmin, *xmax, *ymin, *ymax;
    float* peak;
    int32_t *xpeak, *ypeak;
    uint32_t* flags;
    ApSpec ap;
    double* apflux;
    double* apferr;
    uint32_t* apflags;
};

}  // namespace gp
