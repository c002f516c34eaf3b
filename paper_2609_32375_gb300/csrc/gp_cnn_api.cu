// gp_cnn_api.cu -- C ABI of the learned background (include/gpphot.h):
// the network's layer kernels for training, the one-pass features, and the
// inference entry point gp_background_learned.
#include <math.h>
#include <stdio.h>

#include "gp_internal.cuh"
#include "gp_launch.h"

using namespace gp;

namespace {

gp_status err(gp_status s, const char* msg)
{
    record_error(msg);
    return s;
}

gp_status cuda_err(cudaError_t e)
{
    char m[200];
    snprintf(m, sizeof m, "CUDA: %s", cudaGetErrorString(e));
    return err(GP_ERR_CUDA, m);
}

#define GP_CK(call)                                         \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return cuda_err(e_);         \
    } while (0)

cudaStream_t S(gp_stream s) { return reinterpret_cast<cudaStream_t>(s); }

}  // namespace

extern "C" {

gp_status gp_cnn_conv3x3(const void* x, int32_t n, int32_t h, int32_t w, int32_t cin_p, const void* wt,
                         const float* bias, int32_t cout_p, int32_t relu, void* y, int32_t out_f32, int32_t creal,
                         gp_stream stream)
{
    if (!x || !wt || !bias || !y || n < 1 || h < 1 || w < 1) return err(GP_ERR_INVALID_ARG, "conv3x3: bad argument");
    if (!cnn_pair_supported(cin_p, cout_p)) return err(GP_ERR_INVALID_ARG, "conv3x3: unsupported channel pair");
    if (out_f32 && (creal < 1 || creal > cout_p)) return err(GP_ERR_INVALID_ARG, "conv3x3: creal out of range");
    GP_CK(launch_cnn_conv(x, n, h, w, cin_p, wt, bias, cout_p, relu, y, out_f32, creal, S(stream)));
    return GP_OK;
}

gp_status gp_cnn_conv3x3_wgrad(const void* x, const void* dp, int32_t n, int32_t h, int32_t w, int32_t cin_p,
                               int32_t cout_p, int32_t cin, int32_t cout, int32_t nslot, float* partial, float* bpart,
                               float* dw, float* db, gp_stream stream)
{
    if (!x || !dp || !partial || !bpart || !dw || !db || n < 1 || h < 1 || w < 1 || nslot < 1)
        return err(GP_ERR_INVALID_ARG, "wgrad: bad argument");
    if (!cnn_pair_supported(cin_p, cout_p) || cin > cin_p || cout > cout_p || cin < 1 || cout < 1)
        return err(GP_ERR_INVALID_ARG, "wgrad: unsupported channels");
    GP_CK(launch_cnn_wgrad(x, dp, n, h, w, cin_p, cout_p, cin, cout, nslot, partial, bpart, dw, db, S(stream)));
    return GP_OK;
}

gp_status gp_cnn_relu_backward(const void* dy, const void* y, void* dp, int64_t count, gp_stream stream)
{
    if (!dy || !y || !dp || count < 0) return err(GP_ERR_INVALID_ARG, "relu_backward: bad argument");
    GP_CK(launch_cnn_relu_backward(dy, y, dp, count, S(stream)));
    return GP_OK;
}

gp_status gp_cnn_mse(const float* pred, const float* target, int64_t npos, int32_t cout_p, void* dy, float* partial,
                     int32_t nblocks, float* loss, gp_stream stream)
{
    if (!pred || !target || !dy || !partial || !loss || npos < 1 || cout_p < 2 || nblocks < 1)
        return err(GP_ERR_INVALID_ARG, "mse: bad argument");
    GP_CK(launch_cnn_mse(pred, target, npos, cout_p, dy, partial, nblocks, loss, S(stream)));
    return GP_OK;
}

gp_status gp_cnn_pack(const float* W, const float* b, int32_t cin, int32_t cout, int32_t cin_p, int32_t cout_p,
                      void* wt, void* wtd, float* bias_p, gp_stream stream)
{
    if (!W || !b || !wt || !wtd || !bias_p || cin > cin_p || cout > cout_p || cin < 1 || cout < 1)
        return err(GP_ERR_INVALID_ARG, "pack: bad argument");
    GP_CK(launch_cnn_pack(W, b, cin, cout, cin_p, cout_p, wt, wtd, bias_p, S(stream)));
    return GP_OK;
}

gp_status gp_cnn_adamw(float* p, const float* g, float* m, float* v, int64_t n, float lr, float beta1, float beta2,
                       float eps, float weight_decay, int32_t step, gp_stream stream)
{
    if (!p || !g || !m || !v || n < 0 || step < 1) return err(GP_ERR_INVALID_ARG, "adamw: bad argument");
    GP_CK(launch_cnn_adamw(p, g, m, v, n, lr, beta1, beta2, eps, weight_decay, step, S(stream)));
    return GP_OK;
}

gp_status gp_cnn_features(const float* quant, int32_t nframes, int32_t nbox, void* feat, float* norm,
                          gp_stream stream)
{
    if (!quant || !feat || !norm || nframes < 1 || nbox < 1 || nbox > 65536)
        return err(GP_ERR_INVALID_ARG, "features: bad argument");
    GP_CK(launch_cnn_features(quant, nframes, nbox, feat, norm, S(stream)));
    return GP_OK;
}

gp_status gp_cnn_targets(const float* bkg_mesh, const float* rms_mesh, const float* norm, int32_t nbox,
                         int32_t nframes, float* target, gp_stream stream)
{
    if (!bkg_mesh || !rms_mesh || !norm || !target || nbox < 1 || nframes < 1)
        return err(GP_ERR_INVALID_ARG, "targets: bad argument");
    GP_CK(launch_cnn_targets(bkg_mesh, rms_mesh, norm, nbox, nframes, target, S(stream)));
    return GP_OK;
}

gp_status gp_cnn_denorm(const float* out, const float* norm, int32_t nbox, int32_t nframes, float* bkg_mesh,
                        float* rms_mesh, gp_stream stream)
{
    if (!out || !norm || !bkg_mesh || !rms_mesh || nbox < 1 || nframes < 1)
        return err(GP_ERR_INVALID_ARG, "denorm: bad argument");
    GP_CK(launch_cnn_denorm(out, norm, nbox, nframes, bkg_mesh, rms_mesh, S(stream)));
    return GP_OK;
}

}  // extern "C"
