// gp_pipeline.h -- the launch sequence of the extraction over one frame or a
// batch of frames, shared by the context entry points (gp_api.cu) and the
// request server (gp_server.cu).  Internal; the public ABI is include/gpphot.h.
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "gp_internal.cuh"
#include "gp_launch.h"

namespace gp {

constexpr size_t ALIGN = 256;

// bump allocator over a device region; sizes are accumulated even past the
// end so that the total requirement can be reported
struct Carver {
    char* base;
    size_t cap;
    size_t off = 0;
    template <class T>
    T* take(size_t n)
    {
        off = (off + ALIGN - 1) & ~(ALIGN - 1);
        T* p = reinterpret_cast<T*>(base + off);
        off += n * sizeof(T);
        return p;
    }
    bool ok() const { return off <= cap; }
};

struct BkgWork {
    double *bkg_raw, *rms_raw, *tmp_b, *tmp_r;
    int *valid, *tmp_v;
};

struct SplineWork {
    double* scratch;
    float4 *tab_b, *tab_r;
};

struct DetWork {
    Tiles T;
    Pieces P;
    Comps C;
    DetMask D;
    int* zero;       // counters, bucket counts and cursors: one block cleared per call
    int nzero;
};

int piece_cap_for(int64_t npix);
int comp_cap_for(int64_t npix, int capacity);
void carve_bkg(Carver& cv, int nbox, BkgWork& w);
void carve_spline(Carver& cv, int Mx, int My, SplineWork& w);
// `zero`: when non-null, the block to clear is taken from *zero (advanced);
// else it is carved here
void carve_det(Carver& cv, int W, int H, int capacity, DetWork& w, int** zero = nullptr);
int det_zero_ints(int W, int H);
SplineTab make_tab(const float4* node, int W, int H, int mesh);

// pinned host staging for the argument records of a batched call; `done`
// is recorded after the upload that last read it
struct ArgStage {
    char* host = nullptr;
    size_t bytes = 0;
    cudaEvent_t done = nullptr;
    bool pending = false;
    cudaError_t init(size_t nbytes);
    void release();
};

// where a call runs: its workspace, stream, staging, stage marks
struct Exec {
    Carver cv;
    cudaStream_t st;
    ArgStage* stage;                 // required when a call has more than one frame
    const SideStream* side = nullptr;   // for work beside `st` within the call (null: all on `st`)
    int launches = 0;                // kernels launched by the call
    // stage boundary k (0..GP_NSTAGES) reached on the stream
    void (*mark)(void* ud, int k, cudaStream_t st) = nullptr;
    void* mark_ud = nullptr;
    void at(int k) { if (mark) mark(mark_ud, k, st); }
    void at_range(int from, int to) { for (int k = from; k <= to; ++k) at(k); }
};

// one frame of a call: device inputs and outputs
struct FrameIO {
    gp_image img;
    gp_bkg bkg;                      // meshes (and optional maps) out; mesh, mx, my are set by the call
    uint32_t* segmap;
    gp_catalog cat;                  // device columns, device count
    double* apflux;
    double* apferr;
    uint32_t* apflags;
    uint8_t* mask_out;               // optional
    int* nnear;                      // optional
    int* status;                     // device status word of the frame
};

// what every frame of a call shares
struct Params {
    gp_bkg_params bp;
    float taps[KMAX];
    int kw, kh;
    float thresh;
    int minarea;
    float radii[MAX_NR];
    int nr;
    float gain;
    const gp_cnn_weights* net;       // learned background, or null for the clipped estimator
    int walk_limit;                  // bound on a union-find walk of the tile merge (0: the default)
};

// Result codes: GP_OK, GP_ERR_OOM (ex.cv ran past its end: nothing was
// launched), GP_ERR_CUDA (a launch failed: the message is recorded).
gp_status run_extract(Exec& ex, int n, FrameIO* F, const Params& P);
gp_status run_background_only(Exec& ex, int n, FrameIO* F, const Params& P);

// the context entry points' argument checks (gp_api.cu); on failure they
// record the gp_last_error() message of the calling thread
gp_status validate_image(const gp_image* img);
gp_status validate_bkg_params(const gp_image* img, const gp_bkg_params* p);
gp_status validate_det_params(const gp_det_params* p, float* taps);   // taps: normalised copy
gp_status validate_ap_params(const gp_ap_params* p);
gp_status validate_net(const gp_cnn_weights* net);

// device bytes run_extract carves for these frames (workspace only)
size_t extract_workspace_bytes(int n, const int* W, const int* H, const int* capacity, int mesh, bool learned);

}  // namespace gp
