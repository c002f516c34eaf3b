// gp_launch.h -- host-side launchers shared between the library's
// translation units (internal; the public ABI is include/gpphot.h).
#pragma once
#include <cuda_runtime.h>

#include "gp_internal.cuh"

namespace gp {

// set the thread's gp_last_error() message (gp_api.cu)
void record_error(const char* msg);

// background (k_background.cu)
cudaError_t launch_boxstats(const Image& im, int B, double k, int maxiter, double* bkg, double* rms, int* valid,
                            float* quant, cudaStream_t st);
cudaError_t launch_mesh_finalize(double* bkg, double* rms, int* valid, double* tmp_b, double* tmp_r, int* tmp_v,
                                 int Mx, int My, int fsize, float* bkg_out, float* rms_out, cudaStream_t st);
cudaError_t launch_spline_tables(const float* mesh, Axis ax, Axis ay, double* scratch, float4* tab, cudaStream_t st);
size_t spline_scratch_doubles(int Mx, int My);
bool mesh_fits_smem(int Mx, int My);
cudaError_t launch_mesh_all(const double* bkg_raw, const double* rms_raw, const int* valid, Axis ax, Axis ay,
                            int fsize, int mode, float* bkg_mesh, float* rms_mesh, float4* tab_b, float4* tab_r,
                            cudaStream_t st);
cudaError_t launch_bkg_maps(const SplineTab& sb, const SplineTab& sr, int W, int H, float* bmap, float* rmap,
                            cudaStream_t st);

// detection (k_stream.cu: threshold mask; k_detect.cu: labelling, merge, rank)
int stream_ctas(int W, int H);
int pack_warps(int W, int H);
int stream_ks(int kw, int kh);
int detect_grid(int W, int H, bool given_mask);
cudaError_t launch_stream_any(const DetectArgs& one, const DetectArgs* batch, int nframes, int maxgrid,
                              cudaStream_t st);
cudaError_t launch_resolve(const Tiles& T, const Pieces& P, const Comps& C, const DetMask& dm, uint32_t* seg, int W,
                           int H, int minarea, int walk_limit, int* status, cudaStream_t st);
cudaError_t launch_rank(const Comps& C, int* n_out, int capacity, bool place, int* status, cudaStream_t st);

// measurement (k_measure.cu)
cudaError_t launch_measure(const Image& im, const SplineTab& sb, const SplineTab& sr, const Comps& C,
                           const uint32_t* seg, const gp_catalog& cat, const float* radii, int nr, float gain,
                           double* apflux, double* apferr, uint32_t* apflags, cudaStream_t st);
cudaError_t launch_aperture(const Image& im, const SplineTab& sb, const SplineTab& sr, const double* xs,
                            const double* ys, int n, const float* radii, int nr, float gain, double* flux,
                            double* ferr, uint32_t* fl, cudaStream_t st);

// growth curves (k_growth.cu); radii strictly increasing, nr <= GP_GROWTH_MAX_NR;
// n sources, or min(n, *n_dev) when n_dev (a device count) is given
cudaError_t launch_growth(const Image& im, const SplineTab& sb, const SplineTab& sr, const double* xs,
                          const double* ys, int n, const int* n_dev, const int* radii, int nr, float gain,
                          double* flux, double* ferr, uint32_t* flags, cudaStream_t st);

// the spatially varying matched filter's threshold pass (k_psf.cu): the
// outputs of launch_stream_any for the pixel arguments of D; taps of P0 and
// the nk modes (kh*kw each), coefficient spline tables of the modes
cudaError_t launch_psf(const DetectArgs& D, const float* p0, const float* modes, int nk, int kw, int kh,
                       const SplineTab* coef_tabs, cudaStream_t st);

// cosmetic corrections (k_cosmetic.cu)
cudaError_t launch_cr(const Image& im, float gain, float rn, float sigclip, float objlim, float* out, uint8_t* flags,
                      int* count, cudaStream_t st);
// clean: the input holds no bad pixel (a uint16 frame without a mask, or the
// cosmic-ray filter's float output of one)
cudaError_t launch_rtn(const Image& im, float thr, float* out, uint8_t* flags, bool keep, int* count, bool clean,
                       cudaStream_t st);

// multi-threshold deblending (k_deblend.cu): an object's catalog row before
// the rows are put in label order, and the call's scratch
struct DbObj {
    uint32_t label, parent;
    int npix;
    double flux, x, y, x2, y2, xy;
    int xmin, xmax, ymin, ymax;
    float peak;
    int xpeak, ypeak;
    uint32_t flags;
};
struct DeblendWork {
    int* cand;             // [rows] candidate rows
    int* cand_count;       // [2] candidates, then the staged objects
    int* obj_count;        // cand_count + 1
    int64_t* off;          // [rows] bytes per candidate, then scratch offsets
    DbObj* obj;            // [obj_cap] staged object rows
    int obj_cap;
    char* scratch;
    int64_t scratch_bytes;
};
cudaError_t launch_deblend(const Image& im, const SplineTab& sb, const SplineTab& sr, const float* taps, int kw,
                           int kh, float thresh, int minarea, int nthresh, float mincont, uint32_t* seg,
                           const gp_catalog& cat, const DeblendWork& w, const gp_catalog& objects, int* counts,
                           int* status, cudaStream_t st);

// optimal aperture radius (k_ropt.cu): the growth curves of the catalog rows
// are given; scratch of the isolation grid from iso_grid()
struct RoptWork {
    int *count, *start, *fill, *items;
    double2* xy;          // [rows] (log10 nu, log10 r) of the calibrators
};
void iso_grid(int W, int H, float d_iso, double* cs, int* ncx, int* ncy);
cudaError_t launch_ropt(const Image& im, const SplineTab& sb, const SplineTab& sr, const float* taps, int kw, int kh,
                        const gp_catalog& cat, const double* flux, const double* ferr, const uint32_t* gflags,
                        const int* radii, int nr, float snr_min, float d_iso, const RoptWork& w, float* nu,
                        int* kopt, uint8_t* calib, int* kfinal, double* flux_opt, double* ferr_opt, double* fit,
                        cudaStream_t st);

// Batch-capable forms.  Each takes one frame's argument record (`one`, used
// alone when batch == nullptr) or a device array of nframes records, one per
// frame (the grid's y index); frames of one batch share what the launch
// dispatches on (dtype, filter size, number of radii, mode), taken from `one`.
BoxArgs box_args(const Image& im, int B, double k, int maxiter, double* bkg, double* rms, int* valid, float* quant);
cudaError_t launch_boxstats_any(const BoxArgs& one, const BoxArgs* batch, int nframes, int maxbox, int is_f32,
                                cudaStream_t st);
MeshArgs mesh_args(const double* bkg_raw, const double* rms_raw, const int* valid, Axis ax, Axis ay, int fsize,
                   int mode, float* bkg_mesh, float* rms_mesh, float4* tab_b, float4* tab_r);
size_t mesh_all_smem(int Mx, int My);
cudaError_t launch_mesh_all_any(const MeshArgs& one, const MeshArgs* batch, int nframes, size_t smem,
                                cudaStream_t st);
DetectArgs detect_args(const Image& im, const SplineTab& sb, const SplineTab& sr, const float* taps, int kw, int kh,
                       float thresh, int minarea, uint32_t* seg, uint8_t* mask_out, int* nnear,
                       const uint8_t* in_mask, const DetMask& dm, const Tiles& T, const Pieces& P, const Comps& C,
                       int* status);
// A second stream for work that runs beside the main stream within one
// call, with the events that fork it from and join it back to the main one.
struct SideStream {
    cudaStream_t st;
    cudaEvent_t fork, join;
};

// the detection stage: the streaming threshold pass (or the packing of a
// given mask), then the labelling of the listed tiles: the crowded tiles on
// `side` (null: on `st`) beside the common form, then the deferred ones
cudaError_t launch_label_any(const DetectArgs& one, const DetectArgs* batch, int nframes, cudaStream_t st,
                             const SideStream* side);
int label_launches(bool given_mask);
ResolveArgs resolve_args(const Tiles& T, const Pieces& P, const Comps& C, const DetMask& dm, uint32_t* seg, int W,
                         int H, int minarea, int walk_limit, int* status);
cudaError_t launch_resolve_any(const ResolveArgs& one, const ResolveArgs* batch, int nframes, int maxtiles,
                               cudaStream_t st);
RankArgs rank_args(const Comps& C, int* n_out, int capacity, bool place, int* status);
cudaError_t launch_rank_any(const RankArgs& one, const RankArgs* batch, int nframes, cudaStream_t st);
MeasureArgs measure_args(const Image& im, const SplineTab& sb, const SplineTab& sr, const Comps& C,
                         const gp_catalog& cat, const float* radii, int nr, float gain, double* apflux,
                         double* apferr, uint32_t* apflags);
cudaError_t launch_measure_any(const MeasureArgs& one, const MeasureArgs* batch, int nframes, cudaStream_t st);

}  // namespace gp

namespace gp {
// learned background network (k_cnn.cu)
bool cnn_pair_supported(int cip, int cop);
cudaError_t launch_cnn_conv(const void* x, int n, int h, int w, int cip, const void* wt, const float* bias, int cop,
                            int relu, void* y, int out_f32, int creal, cudaStream_t st);
cudaError_t launch_cnn_wgrad(const void* x, const void* dp, int n, int h, int w, int cip, int cop, int cir, int cor,
                             int nslot, float* partial, float* bpart, float* dw, float* db, cudaStream_t st);
cudaError_t launch_cnn_relu_backward(const void* dy, const void* y, void* dp, int64_t count, cudaStream_t st);
cudaError_t launch_cnn_mse(const float* pred, const float* target, int64_t npos, int cop, void* dy, float* part,
                           int nblocks, float* loss, cudaStream_t st);
cudaError_t launch_cnn_pack(const float* W, const float* b, int cir, int cor, int cip, int cop, void* wt, void* wtd,
                            float* bias_p, cudaStream_t st);
cudaError_t launch_cnn_adamw(float* p, const float* g, float* m, float* v, int64_t n, float lr, float b1, float b2,
                             float eps, float wd, int step, cudaStream_t st);
cudaError_t launch_cnn_features(const float* quant, int nframes, int nbox, void* feat, float* norm, cudaStream_t st);
cudaError_t launch_cnn_denorm(const float* out, const float* norm, int nbox, int nframes, float* bkg, float* rms,
                              cudaStream_t st);
cudaError_t launch_cnn_targets(const float* bkg, const float* rms, const float* norm, int nbox, int nframes,
                               float* tgt, cudaStream_t st);
}  // namespace gp
