// Register-gather kernels for float storage, 2 chunk(s) per warp: one
// translation unit per (element type, chunk count) so the build compiles the
// instantiations in parallel.
#include "blip_register.cuh"

namespace blip {

cudaError_t launch_register_f32_c2(const EvalParams &p, int warps, int pipe, cudaStream_t stream)
{
    return reg::launch_register_vo<float, 2>(p, warps, pipe, stream);
}

}  // namespace blip
