// k_stream_f32.cu -- the f32 instances of the streaming detection pass
// (k_stream_impl.cuh); one translation unit per dtype so they compile in
// parallel.
#include "k_stream_impl.cuh"

namespace gp {

cudaError_t launch_stream_f32(const DetectArgs& one, const DetectArgs* batch, int nframes, int maxcta,
                             const CUtensorMap* map, cudaStream_t st)
{
    return launch_stream_dtype<true>(one, batch, nframes, maxcta, map, st);
}

}  // namespace gp
