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

// detection (k_detect.cu)
cudaError_t launch_detect_tiles(const Image& im, const SplineTab& sb, const SplineTab& sr, const float* taps,
                                int kw, int kh, float thresh, int minarea, uint32_t* seg, uint8_t* mask_out,
                                int* nnear, const uint8_t* in_mask, const Tiles& T, const Pieces& P, const Comps& C,
                                int* status, cudaStream_t st);
cudaError_t launch_resolve(const Tiles& T, const Pieces& P, const Comps& C, uint32_t* seg, int W, int H,
                           int minarea, int* status, cudaStream_t st);
cudaError_t launch_rank(const Comps& C, int* n_out, int capacity, bool place, int* status, cudaStream_t st);

// measurement (k_measure.cu)
cudaError_t launch_measure(const Image& im, const SplineTab& sb, const SplineTab& sr, const Comps& C,
                           const uint32_t* seg, const gp_catalog& cat, const float* radii, int nr, float gain,
                           double* apflux, double* apferr, uint32_t* apflags, cudaStream_t st);
cudaError_t launch_aperture(const Image& im, const SplineTab& sb, const SplineTab& sr, const double* xs,
                            const double* ys, int n, const float* radii, int nr, float gain, double* flux,
                            double* ferr, uint32_t* fl, cudaStream_t st);

}  // namespace gp
