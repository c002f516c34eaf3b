// k_measure_batch.cu -- the batched instances of k_measure (one launch
// over the frames of a batch, grid y = frame; see k_measure_impl.cuh).
#include "k_measure_impl.cuh"

namespace gp {

cudaError_t launch_measure_batched(const MeasureArgs& one, const MeasureArgs* batch, dim3 grid, cudaStream_t st)
{
    if (one.ap.nr > 0) {
        const cudaError_t e = one.im.is_f32 ? dispatch_nr<MeasureBatchLaunch, true>(one.ap.nr, one, batch, grid, st)
                                            : dispatch_nr<MeasureBatchLaunch, false>(one.ap.nr, one, batch, grid, st);
        if (e != cudaSuccess) return e;
    }
    launch_dep(k_ap_finish_rows<true>, grid, dim3(256), 0, st, batch, one);
    return cudaGetLastError();
}

}  // namespace gp
