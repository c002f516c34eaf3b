// k_stream_impl.cuh -- the streaming half of detection (paper Section 3.2: the
// matched filter against a significance threshold, with the Section 3.1
// background and noise maps): one pass over the frame that evaluates the
// spline background B and noise sigma, forms m = I - B, correlates it with
// the normalised kernel, F = K (x) m, and writes
//   * the foreground F > k sigma as a packed bit mask (per frame row and
//     128-column strip, four 32-bit words: word c, bit l = column 4 l + c),
//   * the zero segmentation map (the labelling stage writes the labels of
//     the few foreground pixels afterwards),
//   * per 64 x 32 detection tile: a piece count of 0 when the tile holds no
//     foreground, else the tile's index appended to the list of tiles the
//     labelling stage visits,
//   * optionally the byte mask and the near-threshold count.
//
// Layout.  A lane owns 4 adjacent columns, a warp a 128-column strip, a CTA
// ST_NW strips side by side over ST_RC output rows.  Input rows are taken in
// groups of G (a multiple of the kernel size): each warp turns its columns of
// a group into m rows in a shared-memory ring (two halves of G rows, 528
// columns: the CTA's 512 and 8 each side, the side columns computed one per
// lane by 16 lanes of warp 0), and after one barrier per group every lane reads the
// 4 + 2h columns its outputs need and runs the separable passes: a
// horizontal dot product per rank, then a vertical one accumulated in
// registers (KS rolling output rows, so each m row is read once).  The
// kernel is applied as sum_r fv_r (x) fh_r; a Gaussian is one term.
//
// Staging of the raw pixels, two forms:
//   TMA     a thread issues cp.async.bulk.tensor.2d copies of each group's
//           rows x 528 columns into one of S shared-memory stages on an
//           mbarrier, S - 1 groups ahead; rows and columns outside the frame
//           arrive as zeros and are replaced by their mirror images in the
//           ring (the border rule of the filter).  Needs 16-byte aligned
//           rows.
//   DIRECT  each lane loads its own columns (8- or 16-byte vector loads
//           where the CTA is inside the frame and rows are aligned, else
//           element loads at mirrored coordinates), one group ahead in
//           registers.
// The ring keeps two groups.  The filter pass reads other lanes' columns only
// in the current group's rows (a warp writes the next group's rows after the
// barrier that ends every warp's pass over them); the previous group's rows
// it reads (a pixel's own m for the map) are the lane's own columns, which
// no other lane writes.
// Instances: k_stream_u16.cu and k_stream_f32.cu; launch: k_stream.cu.
#pragma once
#include <cuda.h>
#include <math.h>

#include "gp_internal.cuh"
#include "gp_launch.h"

namespace gp {

constexpr int ST_NW = 4;                        // warps (strips) per CTA
constexpr int ST_NT = 32 * ST_NW;
constexpr int ST_COLS = ST_NW * ST_STRIP;       // 512 columns per CTA
constexpr int ST_HALO = 8;                      // ring columns each side (>= HMAX, 16-byte multiple)
constexpr int ST_RW = ST_COLS + 2 * ST_HALO;    // 528 ring columns
constexpr int ST_RC = 128;                      // output rows per CTA (a multiple of TY)
constexpr int ST_BOXW = ST_RW / 3;              // 176 columns per TMA box, three boxes per row group
constexpr int ST_STAGES = 3;                    // TMA stages
constexpr int ST_WAIT_LIMIT = 1 << 22;          // bounded mbarrier polls (each try_wait also suspends)
static_assert(ST_RC % TY == 0 && ST_STRIP == 2 * TX, "a strip is two detection tiles wide");
static_assert(ST_BOXW * 3 == ST_RW && ST_BOXW % 4 == 0, "TMA boxes tile the ring row in 4-column units");

template <int KS>
struct StreamCfg {
    static constexpr int H = KS / 2;
    static constexpr int G = KS == 3 ? 6 : KS;            // input rows per group, a multiple of KS
    static constexpr int WOFF = 4 * ((H + 3) / 4);        // window start: columns left of the lane's first
    static constexpr int NV = 1 + 2 * ((H + 3) / 4);      // float4 window loads per row
    static_assert(G % KS == 0 && G > 2 * H, "slot rotation and the mirror rows need G >= KS, G % KS == 0");
};

// byte offsets of the dynamic shared memory
template <int KS>
struct StreamSmem {
    static constexpr int G = StreamCfg<KS>::G;
    static constexpr int ROWS = ST_RC + 2 * HMAX + 16;    // row table entries (>= groups * G)
    static constexpr size_t ring = 0;
    static constexpr size_t ring_bytes = sizeof(float) * 2 * G * ST_RW;
    static constexpr size_t rowc = ring + ring_bytes;
    static constexpr size_t rowj = rowc + sizeof(float4) * ROWS;
    static constexpr size_t bar = (rowj + sizeof(int2) * ROWS + 127) & ~(size_t)127;
    static constexpr size_t stage = bar + 128;
    __host__ __device__ static constexpr size_t box_bytes(int esz) { return ((size_t)ST_BOXW * G * esz + 127) & ~(size_t)127; }
    __host__ __device__ static constexpr size_t total(int esz) { return stage + (size_t)ST_STAGES * 3 * box_bytes(esz); }
};
template <int KS>
constexpr bool rows_fit()
{
    return StreamSmem<KS>::ROWS >= (ST_RC + 2 * (KS / 2) + StreamCfg<KS>::G - 1) / StreamCfg<KS>::G * StreamCfg<KS>::G;
}
static_assert(rows_fit<3>() && rows_fit<5>() && rows_fit<7>() && rows_fit<15>(), "row table covers the last group");

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity)
{
    const uint32_t a = smem_u32(bar);
    for (int i = 0; i < ST_WAIT_LIMIT; ++i) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// one group of rows, 3 boxes of 176 x G, into stage buffer `dst`
__device__ __forceinline__ void tma_issue(const CUtensorMap* map, uint64_t* bar, unsigned char* dst, size_t boxb,
                                          int x, int y, uint32_t bytes)
{
    const uint32_t b = smem_u32(bar);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(bytes) : "memory");
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        asm volatile(
            "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
            "[%4];" ::"r"(smem_u32(dst + k * boxb)),
            "l"(reinterpret_cast<uint64_t>(map)), "r"(x + k * ST_BOXW), "r"(y), "r"(b)
            : "memory");
    }
}

// raw pixels of 4 columns as floats (u16 exact)
template <bool F32>
struct Raw4;
template <>
struct Raw4<false> {
    uint2 w;
    __device__ __forceinline__ void to_float(float* v) const
    {
        v[0] = (float)(w.x & 0xffffu); v[1] = (float)(w.x >> 16);
        v[2] = (float)(w.y & 0xffffu); v[3] = (float)(w.y >> 16);
    }
};
template <>
struct Raw4<true> {
    float4 w;
    __device__ __forceinline__ void to_float(float* v) const { v[0] = w.x; v[1] = w.y; v[2] = w.z; v[3] = w.w; }
};

// 4 pixels of frame row gy starting at column x (DIRECT): one vector load
// when `vec`, else element loads at mirrored columns
template <bool F32>
__device__ __forceinline__ Raw4<F32> load4(const Image& im, int gy, int x, bool vec)
{
    Raw4<F32> r;
    const int64_t row = (int64_t)gy * im.pitch;
    if (vec) {
        if constexpr (F32) r.w = __ldg(reinterpret_cast<const float4*>(reinterpret_cast<const float*>(im.data) + row + x));
        else r.w = __ldg(reinterpret_cast<const uint2*>(reinterpret_cast<const uint16_t*>(im.data) + row + x));
        return r;
    }
    if constexpr (F32) {
        const float* p = reinterpret_cast<const float*>(im.data) + row;
        r.w = make_float4(__ldg(p + mirror_idx(x, im.W)), __ldg(p + mirror_idx(x + 1, im.W)),
                          __ldg(p + mirror_idx(x + 2, im.W)), __ldg(p + mirror_idx(x + 3, im.W)));
    } else {
        const uint16_t* p = reinterpret_cast<const uint16_t*>(im.data) + row;
        r.w = make_uint2((uint32_t)__ldg(p + mirror_idx(x, im.W)) | ((uint32_t)__ldg(p + mirror_idx(x + 1, im.W)) << 16),
                         (uint32_t)__ldg(p + mirror_idx(x + 2, im.W)) | ((uint32_t)__ldg(p + mirror_idx(x + 3, im.W)) << 16));
    }
    return r;
}

// the same 4 pixels from a TMA stage (ring column c, a multiple of 4)
template <bool F32>
__device__ __forceinline__ Raw4<F32> stage4(const unsigned char* st, size_t boxb, int s, int c)
{
    constexpr int ESZ = F32 ? 4 : 2;
    const int box = c / ST_BOXW, cc = c - box * ST_BOXW;
    const unsigned char* p = st + box * boxb + ((size_t)s * ST_BOXW + cc) * ESZ;
    Raw4<F32> r;
    if constexpr (F32) r.w = *reinterpret_cast<const float4*>(p);
    else r.w = *reinterpret_cast<const uint2*>(p);
    return r;
}

// Pairs of float32 in one 64-bit register pair, and the paired (f32x2)
// fused multiply-add / subtract: two independent float32 operations, each
// rounded like fmaf / a - b.
__device__ __forceinline__ unsigned long long f2_bits(float2 a) { return *reinterpret_cast<unsigned long long*>(&a); }
__device__ __forceinline__ float2 f2_from(unsigned long long d) { return *reinterpret_cast<float2*>(&d); }

__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c)
{
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(f2_bits(a)), "l"(f2_bits(b)), "l"(f2_bits(c)));
    return f2_from(d);
}

__device__ __forceinline__ float2 fmul2(float2 a, float2 b)
{
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2_bits(a)), "l"(f2_bits(b)));
    return f2_from(d);
}

__device__ __forceinline__ float2 fsub2(float2 a, float2 b)
{
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2_bits(a)), "l"(f2_bits(b)));
    return f2_from(d);
}

__device__ __forceinline__ float2 splat2(float a) { return make_float2(a, a); }

// spline values of one map at 4 columns for node rows (j0, j1), as pairs of
// columns (0, 1) and (2, 3): u = u_j0(x), d = u_j1(x) - u_j0(x),
// w0 = w_j0(x), w1 = w_j1(x), optionally scaled
struct Col4 {
    float2 u[2], d[2], w0[2], w1[2];
};

__device__ __forceinline__ Col4 col4_load(const SplineTab& s, int j0, int j1, int x, int W, float scale)
{
    float u[4], d[4], w0[4], w1[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const AxCoef cx = axis_coef(s.ax, (float)mirror_idx(x + e, W));
        const float2 a = row_eval(s, j0, cx);
        const float2 b = row_eval(s, j1, cx);
        u[e] = scale * a.x;
        d[e] = scale * (b.x - a.x);
        w0[e] = scale * a.y;
        w1[e] = scale * b.y;
    }
    Col4 c;
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        c.u[p] = make_float2(u[2 * p], u[2 * p + 1]);
        c.d[p] = make_float2(d[2 * p], d[2 * p + 1]);
        c.w0[p] = make_float2(w0[2 * p], w0[2 * p + 1]);
        c.w1[p] = make_float2(w1[2 * p], w1[2 * p + 1]);
    }
    return c;
}

// the map at a pair of columns of a row with coefficients rc = (b, c0, c1):
// u + b d + c0 w0 + c1 w1, in the order of axis_combine
__device__ __forceinline__ float2 col4_eval2(const Col4& c, const float4& rc, int p)
{
    return ffma2(splat2(rc.z), c.w1[p], ffma2(splat2(rc.y), c.w0[p], ffma2(splat2(rc.x), c.d[p], c.u[p])));
}

// one raw pixel of a stage buffer (ring column c) as a float
template <bool F32>
__device__ __forceinline__ float stage1(const unsigned char* st, size_t boxb, int s, int c)
{
    constexpr int ESZ = F32 ? 4 : 2;
    const int box = c / ST_BOXW, cc = c - box * ST_BOXW;
    const unsigned char* p = st + box * boxb + ((size_t)s * ST_BOXW + cc) * ESZ;
    if constexpr (F32) return *reinterpret_cast<const float*>(p);
    else return (float)*reinterpret_cast<const uint16_t*>(p);
}

// one raw pixel into a stage buffer
template <bool F32>
__device__ __forceinline__ void stage_put1(unsigned char* st, size_t boxb, int s, int c, float v)
{
    constexpr int ESZ = F32 ? 4 : 2;
    const int box = c / ST_BOXW, cc = c - box * ST_BOXW;
    unsigned char* p = st + box * boxb + ((size_t)s * ST_BOXW + cc) * ESZ;
    if constexpr (F32) *reinterpret_cast<float*>(p) = v;
    else *reinterpret_cast<uint16_t*>(p) = (uint16_t)v;
}

// one pixel of frame row gy at column x (mirrored) as a float (DIRECT)
template <bool F32>
__device__ __forceinline__ float load1(const Image& im, int gy, int x)
{
    const int64_t i = (int64_t)gy * im.pitch + mirror_idx(x, im.W);
    if constexpr (F32) return __ldg(reinterpret_cast<const float*>(im.data) + i);
    else return (float)__ldg(reinterpret_cast<const uint16_t*>(im.data) + i);
}

// the spline values of one map at one column x for node rows (j0, j1):
// (u, d, w0, w1) as in Col4
__device__ __forceinline__ float4 col1_load(const SplineTab& s, int j0, int j1, int x, int W)
{
    const AxCoef cx = axis_coef(s.ax, (float)mirror_idx(x, W));
    const float2 a = row_eval(s, j0, cx);
    const float2 b = row_eval(s, j1, cx);
    return make_float4(a.x, b.x - a.x, a.y, b.y);
}

// 4 raw pixels into a stage buffer (the TMA box layout)
template <bool F32>
__device__ __forceinline__ void stage_put4(unsigned char* st, size_t boxb, int s, int c, const Raw4<F32>& r)
{
    constexpr int ESZ = F32 ? 4 : 2;
    const int box = c / ST_BOXW, cc = c - box * ST_BOXW;
    unsigned char* p = st + box * boxb + ((size_t)s * ST_BOXW + cc) * ESZ;
    if constexpr (F32) *reinterpret_cast<float4*>(p) = r.w;
    else *reinterpret_cast<uint2*>(p) = r.w;
}


template <bool BATCH>
__device__ __forceinline__ const DetectArgs& stream_args(const DetectArgs* __restrict__ batch, const DetectArgs& one)
{
    if constexpr (BATCH) return batch[blockIdx.y];
    else return one;
}

// bad pixel (masked, or a non-finite float) at frame (x, y), x inside the frame
template <bool F32>
__device__ __forceinline__ bool bad_at(const Image& im, int x, int y)
{
    bool b = false;
    if (im.mask) b = im.mask[(int64_t)y * im.W + x] != 0;
    if constexpr (F32) b = b || !isfinite(__ldg(reinterpret_cast<const float*>(im.data) + (int64_t)y * im.pitch + x));
    return b;
}

// Staging modes of k_stream
constexpr int SM_DIRECT = 0;   // one frame, lanes load their own columns
constexpr int SM_TMA = 1;      // one frame, tensor-map copies into shared stages
constexpr int SM_BATCH = 2;    // a batch of frames (DIRECT loads), grid y = frame

// FAST: one separable term, no input mask, neither the byte mask nor the
// near-threshold count requested -- the form the pipeline runs on the
// workloads; the general form handles the rest.
template <bool F32, int KS, int MODE, bool FAST>
__global__ void __launch_bounds__(ST_NT) k_stream(const DetectArgs* __restrict__ batch,
                                                  const __grid_constant__ DetectArgs one,
                                                  const __grid_constant__ CUtensorMap tmap)
{
    pdl_wait();
    pdl_release();
    using Cfg = StreamCfg<KS>;
    using SM = StreamSmem<KS>;
    constexpr int H = Cfg::H, G = Cfg::G, NV = Cfg::NV, WOFF = Cfg::WOFF;
    constexpr int ESZ = F32 ? 4 : 2;
    constexpr bool TMA = MODE == SM_TMA, BATCH = MODE == SM_BATCH;
    // a pixel can be bad: a non-finite float, or a masked pixel (general form only)
    constexpr bool BADP = F32 || !FAST;
    // bad bits of the main columns, 4 per input row, newest lowest; an
    // output pixel's own bit sits G - 1 - s + h rows back (kernels up to
    // 7 x 7; larger ones re-read the pixel)
    constexpr bool HIST = G - 1 + H <= 15;
    extern __shared__ __align__(128) unsigned char smem[];
    float* ring = reinterpret_cast<float*>(smem + SM::ring);
    float4* rowc = reinterpret_cast<float4*>(smem + SM::rowc);
    int2* rowj = reinterpret_cast<int2*>(smem + SM::rowj);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + SM::bar);
    unsigned char* stg = smem + SM::stage;
    constexpr size_t boxb = SM::box_bytes(ESZ);

    const DetectArgs& A = stream_args<BATCH>(batch, one);
    const Image& im = A.im;
    const int W = im.W, Hf = im.H;
    const int ncx = (W + ST_COLS - 1) / ST_COLS;
    const int ncta = ncx * ((Hf + ST_RC - 1) / ST_RC);
    if (BATCH && (int)blockIdx.x >= ncta) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int X0 = (blockIdx.x % ncx) * ST_COLS, Y0 = (blockIdx.x / ncx) * ST_RC;
    const int nout = min(ST_RC, Hf - Y0);
    const int nin = nout + 2 * H;                         // input rows: frame rows Y0 - H .. Y0 + nout + H - 1
    const int ng = (nin + G - 1) / G;                     // rows past nin are computed (valid addresses) and unused
    const int xs = X0 + ST_STRIP * warp + ST_CPL * lane;  // the lane's first column
    const int slot0 = ST_HALO + ST_STRIP * warp + ST_CPL * lane;
    // lanes 0..15 of warp 0 also compute the ring's side columns, one each
    const bool hl = warp == 0 && lane < 2 * ST_HALO;
    const int hx = lane < ST_HALO ? X0 - ST_HALO + lane : X0 + ST_COLS + (lane - ST_HALO);
    const int hslot = lane < ST_HALO ? lane : ST_COLS + lane;

    // ---- row table: spline coefficients of every input row (mirrored)
    for (int k = tid; k < ng * G; k += ST_NT) {
        const AxCoef cy = axis_coef(A.sb.ay, (float)mirror_idx(Y0 - H + k, Hf));
        rowc[k] = make_float4(cy.b, cy.c0, cy.c1, 0.f);
        rowj[k] = make_int2(cy.i, cy.i1);
    }
    if (TMA && tid == 0) {
        for (int s = 0; s < ST_STAGES; ++s)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar + s)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    constexpr uint32_t gbytes = (uint32_t)(3 * ST_BOXW * G * ESZ);
    // DIRECT: vector loads when every column of the CTA (and its sides) is
    // inside the frame and rows are aligned; the loads of group g + 2 are in
    // flight during group g's filter pass and land in its stage after it
    const bool vec = !TMA && X0 - ST_HALO >= 0 && X0 + ST_COLS + ST_HALO <= W && (im.pitch % ST_CPL) == 0 &&
                     ((((uintptr_t)im.data) & (F32 ? 15 : 7)) == 0);
    Raw4<F32> raw[G];
    float hraw[G];
    auto fetch = [&](int g) {
#pragma unroll
        for (int s = 0; s < G; ++s) {
            const int gy = mirror_idx(Y0 - H + g * G + s, Hf);
            raw[s] = load4<F32>(im, gy, xs, vec);
            if (hl) hraw[s] = load1<F32>(im, gy, hx);
        }
    };
    auto put = [&](int g) {
        unsigned char* sp = stg + (g % ST_STAGES) * 3 * boxb;
#pragma unroll
        for (int s = 0; s < G; ++s) {
            stage_put4<F32>(sp, boxb, s, slot0, raw[s]);
            if (hl) stage_put1<F32>(sp, boxb, s, hslot, hraw[s]);
        }
    };
    if (!TMA) {
        fetch(0);
        put(0);
        if (ng > 1) {
            fetch(1);
            put(1);
        }
    }
    __syncthreads();
    if (TMA && tid == 0) {
        for (int s = 0; s < ST_STAGES && s < ng; ++s)
            tma_issue(&tmap, bar + s, stg + s * 3 * boxb, boxb, X0 - ST_HALO, Y0 - H + s * G, gbytes);
    }

    // per-lane spline state: background at the input rows' node interval
    // (cb; the side columns' in hcoef), k sigma at the output rows' (cs),
    // evaluated where each output row is thresholded
    Col4 cb, cs;
    float4 hcb = make_float4(0.f, 0.f, 0.f, 0.f);      // side column's background spline values
    int jb = -1, js = -1, jh = -1;
    uint64_t badh = 0;
    const int nstrip = A.nstrip;
    const int strip = xs / ST_STRIP;
    const bool strip_in = X0 + ST_STRIP * warp < W;
    const bool seg_vec = (W & 3) == 0 && ((((uintptr_t)A.seg) & 15) == 0);
    // taps of the first separable term in registers
    float th0[KS], tv0[KS];
#pragma unroll
    for (int u = 0; u < KS; ++u) { th0[u] = A.fh[u]; tv0[u] = A.fv[u]; }
    const int nrank = FAST ? 1 : A.nrank;
    float2 acc[KS][2];        // rolling output rows, columns (0, 1) and (2, 3)
#pragma unroll
    for (int q = 0; q < KS; ++q) acc[q][0] = acc[q][1] = make_float2(0.f, 0.f);
    uint32_t orw = 0u;
    int nnear = 0;
    const bool edge_l = X0 - ST_HALO < 0, edge_r = X0 + ST_COLS + ST_HALO > W;

    for (int g = 0; g < ng; ++g) {
        float* rg = ring + (g & 1) * G * ST_RW;               // this group's m rows
        const float* rp = ring + ((g + 1) & 1) * G * ST_RW;   // the previous group's
        const unsigned char* sg = stg + (g % ST_STAGES) * 3 * boxb;
        bool timed_out = false;
        if (TMA) timed_out = !mbar_wait(bar + g % ST_STAGES, (uint32_t)((g / ST_STAGES) & 1));

        // ---- m = I - B for the group's rows (a bad pixel contributes 0)
#pragma unroll 1
        for (int s = 0; s < G; ++s) {
            const int k = g * G + s;
            const int2 j = rowj[k];
            const float4 rc = rowc[k];
            if (j.x != jb) {
                cb = col4_load(A.sb, j.x, j.y, xs, W, 1.f);
                jb = j.x;
            }
            float v[4];
            stage4<F32>(sg, boxb, s, slot0).to_float(v);
            const float2 m01 = fsub2(make_float2(v[0], v[1]), col4_eval2(cb, rc, 0));
            const float2 m23 = fsub2(make_float2(v[2], v[3]), col4_eval2(cb, rc, 1));
            float m[4] = {m01.x, m01.y, m23.x, m23.y};
            if (BADP) {
                uint32_t nib = 0u;
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    bool b = F32 && !isfinite(v[e]);
                    if (!FAST && !TMA && im.mask)
                        b = b || im.mask[(int64_t)mirror_idx(Y0 - H + k, Hf) * W + mirror_idx(xs + e, W)] != 0;
                    if (b) m[e] = 0.f;
                    nib |= (uint32_t)b << e;
                }
                if (HIST) badh = (badh << 4) | nib;
            }
            *reinterpret_cast<float4*>(rg + s * ST_RW + slot0) = make_float4(m[0], m[1], m[2], m[3]);
            if (hl) {
                if (j.x != jh) {
                    hcb = col1_load(A.sb, j.x, j.y, hx, W);
                    jh = j.x;
                }
                const float hv = stage1<F32>(sg, boxb, s, hslot);
                bool b = F32 && !isfinite(hv);
                if (!FAST && !TMA && im.mask)
                    b = b || im.mask[(int64_t)mirror_idx(Y0 - H + k, Hf) * W + mirror_idx(hx, W)] != 0;
                rg[s * ST_RW + hslot] = b ? 0.f : hv - fmaf(rc.z, hcb.w, fmaf(rc.y, hcb.z, fmaf(rc.x, hcb.y, hcb.x)));
            }
        }
        if (__syncthreads_or(timed_out)) {
            if (tid == 0) set_status(A.status, GP_ERR_TIMEOUT);
            return;
        }
        if (TMA) {
            // the stage is consumed: refill it with group g + S
            if (tid == 0 && g + ST_STAGES < ng)
                tma_issue(&tmap, bar + g % ST_STAGES, stg + (g % ST_STAGES) * 3 * boxb, boxb, X0 - ST_HALO,
                          Y0 - H + (g + ST_STAGES) * G, gbytes);
            // columns outside the frame arrived as zeros: mirror images
            if (edge_l || edge_r) {
                for (int q = tid; q < G * 2 * ST_HALO; q += ST_NT) {
                    const int s = q / (2 * ST_HALO), t = q - s * 2 * ST_HALO;
                    if (g * G + s >= nin) continue;
                    // t < 8: a left side column, else a column at or beyond W inside the ring
                    const int x = t < ST_HALO ? X0 - ST_HALO + t : W + (t - ST_HALO);
                    const int c = x - X0 + ST_HALO;
                    if (x >= 0 && x < W) continue;
                    if (c < 0 || c >= ST_RW) continue;
                    rg[s * ST_RW + c] = rg[s * ST_RW + (mirror_idx(x, W) - X0 + ST_HALO)];
                }
                __syncthreads();
            }
            // rows outside the frame: copies of their mirror rows (this group or the last)
            const int r0 = Y0 - H + g * G;
            if (r0 < 0 || r0 + G > Hf) {
                for (int s = 0; s < G; ++s) {
                    const int k = g * G + s, r = r0 + s;
                    if (k >= nin || (r >= 0 && r < Hf)) continue;
                    const int ks = mirror_idx(r, Hf) - (Y0 - H);
                    const float* src = ring + ((ks / G) & 1) * G * ST_RW + (ks % G) * ST_RW;
                    for (int c = tid; c < ST_RW; c += ST_NT) rg[s * ST_RW + c] = src[c];
                }
                __syncthreads();
            }
        } else if (g + 2 < ng) {
            fetch(g + 2);
        }

        // ---- filter, threshold and emit the rows completed by this group
#pragma unroll
        for (int s = 0; s < G; ++s) {
            const int k = g * G + s;
            float win[4 * NV];
#pragma unroll
            for (int q = 0; q < NV; ++q) {
                const float4 t = *reinterpret_cast<const float4*>(rg + s * ST_RW + slot0 - WOFF + 4 * q);
                win[4 * q] = t.x; win[4 * q + 1] = t.y; win[4 * q + 2] = t.z; win[4 * q + 3] = t.w;
            }
            {
                float h[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    float t = th0[0] * win[WOFF - H + e];
#pragma unroll
                    for (int u = 1; u < KS; ++u) t = fmaf(th0[u], win[WOFF - H + e + u], t);
                    h[e] = t;
                }
                // output row k starts here with tap row 0; rows k - v take tap row v
                const float2 h01 = make_float2(h[0], h[1]), h23 = make_float2(h[2], h[3]);
                acc[s % KS][0] = fmul2(splat2(tv0[0]), h01);
                acc[s % KS][1] = fmul2(splat2(tv0[0]), h23);
#pragma unroll
                for (int v = 1; v < KS; ++v) {
                    float2* a = acc[((s - v) % KS + KS) % KS];
                    a[0] = ffma2(splat2(tv0[v]), h01, a[0]);
                    a[1] = ffma2(splat2(tv0[v]), h23, a[1]);
                }
            }
            if (!FAST) {
                for (int rk = 1; rk < nrank; ++rk) {
                    float h[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        float t = 0.f;
#pragma unroll
                        for (int u = 0; u < KS; ++u) t = fmaf(A.fh[rk * KS + u], win[WOFF - H + e + u], t);
                        h[e] = t;
                    }
#pragma unroll
                    for (int v = 0; v < KS; ++v) {
                        const float2 tv = splat2(A.fv[rk * KS + v]);
                        float2* a = acc[((s - v) % KS + KS) % KS];
                        a[0] = ffma2(tv, make_float2(h[0], h[1]), a[0]);
                        a[1] = ffma2(tv, make_float2(h[2], h[3]), a[1]);
                    }
                }
            }
            // ---- output row y = k - 2h is complete
            const int y = k - 2 * H;
            if (y < 0 || y >= nout) continue;
            const int Y = Y0 + y;
            const float F[4] = {acc[(s + 1) % KS][0].x, acc[(s + 1) % KS][0].y, acc[(s + 1) % KS][1].x,
                                acc[(s + 1) % KS][1].y};
            // k sigma of the output row
            const int2 jy = rowj[y + H];
            const float4 ry = rowc[y + H];
            if (jy.x != js) {
                cs = col4_load(A.sr, jy.x, jy.y, xs, W, A.thresh);
                js = jy.x;
            }
            const float2 t01 = col4_eval2(cs, ry, 0), t23 = col4_eval2(cs, ry, 1);
            const float tv4[4] = {t01.x, t01.y, t23.x, t23.y};
            bool fg[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float thr = tv4[e];
                const bool in = xs + e < W;
                bool b = false;
                if (BADP && in) {
                    if (HIST) b = (badh >> (4 * (G - 1 - s + H) + e)) & 1u;
                    else b = bad_at<F32>(im, xs + e, Y);
                }
                fg[e] = in && !b && F[e] > thr;
                if (!FAST && A.nnear && in && fabsf(F[e] - thr) <= 1e-5f * fabsf(thr)) ++nnear;
            }
            const uint32_t b0 = __ballot_sync(0xffffffffu, fg[0]), b1 = __ballot_sync(0xffffffffu, fg[1]);
            const uint32_t b2 = __ballot_sync(0xffffffffu, fg[2]), b3 = __ballot_sync(0xffffffffu, fg[3]);
            const uint32_t orow = b0 | b1 | b2 | b3;
            orw |= orow;
            if (strip_in) {
                if (lane == 0) A.bits[(int64_t)Y * nstrip + strip] = make_uint4(b0, b1, b2, b3);
                // the map: 0, or at foreground pixels the bits of m (the labelling
                // stage's input; it writes the labels over them)
                uint4 sv = make_uint4(0u, 0u, 0u, 0u);
                if (orow) {
                    const float4 mc = *reinterpret_cast<const float4*>(
                        (s >= H ? rg + (s - H) * ST_RW : rp + (G + s - H) * ST_RW) + slot0);
                    sv.x = fg[0] ? __float_as_uint(mc.x) : 0u;
                    sv.y = fg[1] ? __float_as_uint(mc.y) : 0u;
                    sv.z = fg[2] ? __float_as_uint(mc.z) : 0u;
                    sv.w = fg[3] ? __float_as_uint(mc.w) : 0u;
                }
                uint32_t* srow = A.seg + (int64_t)Y * W;
                if (seg_vec) {
                    if (xs < W) *reinterpret_cast<uint4*>(srow + xs) = sv;
                } else {
                    const uint32_t svv[4] = {sv.x, sv.y, sv.z, sv.w};
#pragma unroll
                    for (int e = 0; e < 4; ++e)
                        if (xs + e < W) srow[xs + e] = svv[e];
                }
                if (!FAST && A.mask_out) {
#pragma unroll
                    for (int e = 0; e < 4; ++e)
                        if (xs + e < W) A.mask_out[(int64_t)Y * W + xs + e] = fg[e] ? 1 : 0;
                }
                // the end of a detection-tile band: the strip's two tiles
                if ((Y & (TY - 1)) == TY - 1 || y == nout - 1) {
                    if (lane < 2) {
                        const int tcol = 2 * strip + lane;
                        if (tcol < A.T.ntx) {
                            const int tile = (Y / TY) * A.T.ntx + tcol;
                            if (orw & (lane ? 0xffff0000u : 0x0000ffffu)) A.tl_list[atomicAdd(A.tl_count, 1)] = tile;
                            else A.T.piece_cnt[tile] = 0;
                        }
                    }
                    orw = 0u;
                }
            }
        }
        if (!TMA && g + 2 < ng) put(g + 2);
    }
    if (!FAST && A.nnear) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) nnear += __shfl_xor_sync(0xffffffffu, nnear, o);
        if (lane == 0 && nnear) atomicAdd(A.nnear, nnear);
    }
}

template <bool F32, int KS, int MODE, bool FAST>
cudaError_t launch_stream_inst(const DetectArgs& one, const DetectArgs* batch, int nframes, int maxcta,
                               const CUtensorMap& map, cudaStream_t st)
{
    const size_t smem = StreamSmem<KS>::total(F32 ? 4 : 2);
    auto* fn = k_stream<F32, KS, MODE, FAST>;
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    launch_dep(fn, dim3(maxcta, nframes), dim3(ST_NT), smem, st, batch, one, map);
    return cudaGetLastError();
}

// the instances of one dtype (k_stream_u16.cu, k_stream_f32.cu)
template <bool F32>
cudaError_t launch_stream_dtype(const DetectArgs& one, const DetectArgs* batch, int nframes, int maxcta,
                                const CUtensorMap* map, cudaStream_t st)
{
    const bool fast = one.nrank == 1 && !one.mask_out && !one.nnear && !one.im.mask && one.ks <= 7;
    if (batch) {
        CUtensorMap m;
        memset(&m, 0, sizeof m);
        switch (one.ks) {
        case 3: return launch_stream_inst<F32, 3, SM_BATCH, false>(one, batch, nframes, maxcta, m, st);
        case 5: return launch_stream_inst<F32, 5, SM_BATCH, false>(one, batch, nframes, maxcta, m, st);
        case 7: return launch_stream_inst<F32, 7, SM_BATCH, false>(one, batch, nframes, maxcta, m, st);
        default: return launch_stream_inst<F32, 15, SM_BATCH, false>(one, batch, nframes, maxcta, m, st);
        }
    }
    const bool tma = map != nullptr;
    CUtensorMap none;
    memset(&none, 0, sizeof none);
    const CUtensorMap& m2 = tma ? *map : none;
#define GP_STREAM_CASE(KSV)                                                                                       \
    case KSV:                                                                                                     \
        if (tma) return fast ? launch_stream_inst<F32, KSV, SM_TMA, true>(one, nullptr, 1, maxcta, m2, st)         \
                             : launch_stream_inst<F32, KSV, SM_TMA, false>(one, nullptr, 1, maxcta, m2, st);       \
        return fast ? launch_stream_inst<F32, KSV, SM_DIRECT, true>(one, nullptr, 1, maxcta, m2, st)               \
                    : launch_stream_inst<F32, KSV, SM_DIRECT, false>(one, nullptr, 1, maxcta, m2, st);
    switch (one.ks) {
        GP_STREAM_CASE(3)
        GP_STREAM_CASE(5)
        GP_STREAM_CASE(7)
    default:
        if (tma) return launch_stream_inst<F32, 15, SM_TMA, false>(one, nullptr, 1, maxcta, m2, st);
        return launch_stream_inst<F32, 15, SM_DIRECT, false>(one, nullptr, 1, maxcta, m2, st);
    }
#undef GP_STREAM_CASE
}

}  // namespace gp
