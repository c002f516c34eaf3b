// k_stream_u16.cu -- the u16 instances of the streaming detection pass
// (k_stream_impl.cuh); one translation unit per dtype so they compile in
// parallel.
#include "k_stream_impl.cuh"

namespace gp {

cudaError_t launch_stream_u16(const DetectArgs& one, const DetectArgs* batch, int nframes, int maxcta,
                             const CUtensorMap* map, cudaStream_t st)
{
    return launch_stream_dtype<false>(one, batch, nframes, maxcta, map, st);
}

}  // namespace gp
