// gp_static.cu -- gp_background_static: the background stage (box
// statistics, mesh filling and median filter, optional full-resolution maps)
// for callers that cannot allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is not available or not
// allowed at call time -- a host process whose device memory is owned by a
// pool it must not bypass, a plugin loaded into an application that forbids
// allocations after start-up, or a latency-critical loop that must not take
// the allocator's locks.  Such callers can create no gp_ctx (its arena is
// one cudaMalloc), so this entry point takes no context: its scratch lives in
// a file-scope device array, part of the library image, which every GPU that
// loads the library holds until the process exits.
#include <math.h>
#include <stdio.h>

#include <mutex>

#include "gp_internal.cuh"
#include "gp_launch.h"

namespace {

using namespace gp;

// Largest mesh (boxes) one call may use: 3600 boxes, e.g. 60 x 60, or a
// 151 MP frame with 256-px boxes (48 x 49).
constexpr int STATIC_MAX_BOXES = 3600;
constexpr size_t RAW_BYTES = (size_t)STATIC_MAX_BOXES * sizeof(double);
constexpr size_t VALID_BYTES = ((size_t)STATIC_MAX_BOXES * sizeof(int) + 255) & ~(size_t)255;
constexpr size_t TAB_BYTES = (size_t)STATIC_MAX_BOXES * sizeof(float4);
constexpr size_t OFF_RMS = RAW_BYTES;
constexpr size_t OFF_VALID = 2 * RAW_BYTES;
constexpr size_t OFF_TAB_B = OFF_VALID + VALID_BYTES;
constexpr size_t OFF_TAB_R = OFF_TAB_B + TAB_BYTES;
constexpr size_t SCRATCH_BYTES = OFF_TAB_R + TAB_BYTES;   // about 172 KB

// the scratch: raw box background / rms (FP64), validity flags, and the two
// spline tables.  Host code must not use this name as an address; it uses
// the device address obtained below.
static __device__ __align__(256) unsigned char g_scratch[SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
void* g_addr[MAX_DEVICES];

thread_local char g_msg[256];

gp_status reject(gp_status s, const char* msg)
{
    snprintf(g_msg, sizeof g_msg, "%s", msg);
    gp::record_error(g_msg);
    return s;
}

}  // namespace

extern "C" gp_status gp_background_static(const gp_image* img, const gp_bkg_params* p, gp_bkg* bkg,
                                          gp_stream stream)
{
    if (!img || !img->data) return reject(GP_ERR_INVALID_ARG, "null image or image data");
    if (img->dtype != GP_U16 && img->dtype != GP_F32) return reject(GP_ERR_INVALID_ARG, "dtype must be GP_U16 or GP_F32");
    if (img->width < 1 || img->height < 1 || (int64_t)img->width * img->height > 0x7fffffffll)
        return reject(GP_ERR_INVALID_ARG, "image size out of range");
    if (img->pitch < img->width) return reject(GP_ERR_INVALID_ARG, "pitch < width");
    if (!p) return reject(GP_ERR_INVALID_ARG, "null background parameters");
    const int maxmesh = img->dtype == GP_U16 ? 256 : 128;
    if (p->mesh < 16 || p->mesh > maxmesh) return reject(GP_ERR_INVALID_ARG, "mesh outside [16, 256] (u16) / [16, 128] (f32)");
    if (p->filter_size < 1 || p->filter_size > 7 || !(p->filter_size & 1))
        return reject(GP_ERR_INVALID_ARG, "filter_size must be odd in [1, 7]");
    if (!(p->clip_k >= 1.f) || !isfinite(p->clip_k)) return reject(GP_ERR_INVALID_ARG, "clip_k must be >= 1");
    if (p->clip_maxiter < 0 || p->clip_maxiter > 1000) return reject(GP_ERR_INVALID_ARG, "clip_maxiter out of range");
    if (!bkg || !bkg->bkg_mesh || !bkg->rms_mesh) return reject(GP_ERR_INVALID_ARG, "null background output meshes");
    const int W = img->width, H = img->height, B = p->mesh;
    const int Mx = (W + B - 1) / B, My = (H + B - 1) / B;
    if (Mx * My > STATIC_MAX_BOXES || !mesh_fits_smem(Mx, My)) {
        char m[160];
        snprintf(m, sizeof m, "mesh of %d x %d boxes exceeds the static scratch limit of %d boxes", Mx, My,
                 STATIC_MAX_BOXES);
        return reject(GP_ERR_INVALID_ARG, m);
    }

    // device address of the scratch on the current device, looked up once
    // and kept for the process: it belongs to the device's primary context
    // (a cudaDeviceReset invalidates it)
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES)
        return reject(GP_ERR_CUDA, "no current CUDA device");
    unsigned char* base;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_addr[dev]) {
            void* a = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&a, g_scratch);
            if (e != cudaSuccess || !a) return reject(GP_ERR_CUDA, "cudaGetSymbolAddress of the static scratch failed");
            g_addr[dev] = a;
        }
        base = static_cast<unsigned char*>(g_addr[dev]);
    }

    bkg->mesh = B; bkg->mx = Mx; bkg->my = My;
    double* bkg_raw = reinterpret_cast<double*>(base);
    double* rms_raw = reinterpret_cast<double*>(base + OFF_RMS);
    int* valid = reinterpret_cast<int*>(base + OFF_VALID);
    float4* tab_b = reinterpret_cast<float4*>(base + OFF_TAB_B);
    float4* tab_r = reinterpret_cast<float4*>(base + OFF_TAB_R);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    Image im;
    im.data = img->data; im.pitch = img->pitch; im.mask = img->mask;
    im.W = W; im.H = H; im.sat = img->saturation; im.is_f32 = img->dtype == GP_F32;
    // every box of the scratch that this call reads is written first by this
    // call, so nothing needs clearing between calls
    cudaError_t e = launch_boxstats(im, B, (double)p->clip_k, p->clip_maxiter, bkg_raw, rms_raw, valid, nullptr, st);
    if (e == cudaSuccess)
        e = launch_mesh_all(bkg_raw, rms_raw, valid, make_axis(W, B), make_axis(H, B), p->filter_size, 0,
                            bkg->bkg_mesh, bkg->rms_mesh, tab_b, tab_r, st);
    if (e == cudaSuccess && (bkg->bkg_map || bkg->rms_map)) {
        SplineTab sb, sr;
        sb.node = tab_b; sb.ax = make_axis(W, B); sb.ay = make_axis(H, B);
        sr.node = tab_r; sr.ax = sb.ax; sr.ay = sb.ay;
        e = launch_bkg_maps(sb, sr, W, H, bkg->bkg_map, bkg->rms_map, st);
    }
    if (e != cudaSuccess) return reject(GP_ERR_CUDA, cudaGetErrorString(e));
    return GP_OK;
}
