// k_stream.cu -- launch of the streaming detection pass (k_stream_impl.cuh:
// spline background and noise, matched filter, threshold, packed mask, zero
// map and the list of detection tiles with foreground; paper Section 3.2 with
// the Section 3.1 maps) and its form for a caller's mask (k_pack_mask, for
// gp_label_mask).
#include <stdlib.h>
#include <string.h>

#include "k_stream_impl.cuh"

namespace gp {

cudaError_t launch_stream_u16(const DetectArgs& one, const DetectArgs* batch, int nframes, int maxcta,
                              const CUtensorMap* map, cudaStream_t st);
cudaError_t launch_stream_f32(const DetectArgs& one, const DetectArgs* batch, int nframes, int maxcta,
                              const CUtensorMap* map, cudaStream_t st);

// ------------------------------------------------------- given masks ---
// gp_label_mask: the caller's byte mask packed into the same bit layout,
// with the zero map and the tile list (one warp per strip and tile band)
template <bool BATCH>
__global__ void __launch_bounds__(128) k_pack_mask(const DetectArgs* __restrict__ batch,
                                                   const __grid_constant__ DetectArgs one)
{
    const DetectArgs& A = stream_args<BATCH>(batch, one);
    const int W = A.im.W, Hf = A.im.H;
    const int lane = threadIdx.x & 31;
    const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nty = (Hf + TY - 1) / TY;
    if (wid >= A.nstrip * nty) return;
    const int strip = wid % A.nstrip, ty = wid / A.nstrip;
    const int xs = strip * ST_STRIP + ST_CPL * lane;
    uint32_t orw = 0u;
    for (int y = ty * TY; y < min(Hf, ty * TY + TY); ++y) {
        bool fg[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const bool in = xs + e < W;
            fg[e] = in && A.in_mask[(int64_t)y * W + xs + e] != 0;
            if (in) A.seg[(int64_t)y * W + xs + e] = 0u;
        }
        const uint32_t b0 = __ballot_sync(0xffffffffu, fg[0]), b1 = __ballot_sync(0xffffffffu, fg[1]);
        const uint32_t b2 = __ballot_sync(0xffffffffu, fg[2]), b3 = __ballot_sync(0xffffffffu, fg[3]);
        orw |= b0 | b1 | b2 | b3;
        if (lane == 0) A.bits[(int64_t)y * A.nstrip + strip] = make_uint4(b0, b1, b2, b3);
    }
    if (lane < 2) {
        const int tcol = 2 * strip + lane;
        if (tcol < A.T.ntx) {
            const int tile = ty * A.T.ntx + tcol;
            if (orw & (lane ? 0xffff0000u : 0x0000ffffu)) A.tl_list[atomicAdd(A.tl_count, 1)] = tile;
            else A.T.piece_cnt[tile] = 0;
        }
    }
}

// ------------------------------------------------------------ launchers ---
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return reinterpret_cast<EncodeTiledFn>(p);
    }();
    return fn;
}

static int stream_force_direct = -1;   // GP_STREAM_DIRECT=1 in the environment: the DIRECT staging everywhere

// a tensor map of the frame for G-row groups, or false when the frame's rows
// are not 16-byte aligned (or the frame is too small for the mirror rows)
static bool make_tmap(const Image& im, int G, CUtensorMap* map)
{
    if (stream_force_direct < 0) {
        const char* e = getenv("GP_STREAM_DIRECT");
        stream_force_direct = (e && e[0] == '1') ? 1 : 0;
    }
    if (stream_force_direct) return false;
    const int esz = im.is_f32 ? 4 : 2;
    if (im.mask) return false;
    if (im.W < 2 * ST_HALO || im.H < 2 * ST_HALO) return false;
    if ((((uintptr_t)im.data) & 15) || ((im.pitch * esz) & 15)) return false;
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)im.W, (cuuint64_t)im.H};
    cuuint64_t strides[1] = {(cuuint64_t)(im.pitch * esz)};
    cuuint32_t box[2] = {(cuuint32_t)ST_BOXW, (cuuint32_t)G};
    cuuint32_t es[2] = {1, 1};
    const CUresult r = fn(map, im.is_f32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_UINT16, 2,
                          const_cast<void*>(im.data), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

int stream_ctas(int W, int H) { return ((W + ST_COLS - 1) / ST_COLS) * ((H + ST_RC - 1) / ST_RC); }

int pack_warps(int W, int H) { return ((W + ST_STRIP - 1) / ST_STRIP) * ((H + TY - 1) / TY); }

// rows per group of the streaming pass for a padded kernel size
static int stream_group_rows(int ks)
{
    switch (ks) {
    case 3: return StreamCfg<3>::G;
    case 5: return StreamCfg<5>::G;
    case 7: return StreamCfg<7>::G;
    default: return StreamCfg<15>::G;
    }
}

// the padded kernel size the streaming pass runs for a kw x kh kernel
int stream_ks(int kw, int kh)
{
    const int k = kw > kh ? kw : kh;
    return k <= 3 ? 3 : k <= 5 ? 5 : k <= 7 ? 7 : 15;
}

cudaError_t launch_stream_any(const DetectArgs& one, const DetectArgs* batch, int nframes, int maxcta,
                              cudaStream_t st)
{
    if (one.in_mask) {
        const int blocks = (maxcta + 3) / 4;   // maxcta: pack_warps() of the largest frame
        if (batch) k_pack_mask<true><<<dim3(blocks, nframes), 128, 0, st>>>(batch, one);
        else k_pack_mask<false><<<blocks, 128, 0, st>>>(nullptr, one);
        return cudaGetLastError();
    }
    CUtensorMap map;
    const bool tma = !batch && make_tmap(one.im, stream_group_rows(one.ks), &map);
    const CUtensorMap* mp = tma ? &map : nullptr;
    if (one.im.is_f32) return launch_stream_f32(one, batch, nframes, maxcta, mp, st);
    return launch_stream_u16(one, batch, nframes, maxcta, mp, st);
}

}  // namespace gp
