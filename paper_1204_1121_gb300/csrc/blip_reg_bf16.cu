// Register-gather kernels for __nv_bfloat16 storage, 1 chunk(s) per warp: one
// translation unit per (element type, chunk count) so the build compiles the
// instantiations in parallel.
#include "blip_register.cuh"

namespace blip {

cudaError_t launch_register_bf16(const EvalParams &p, int warps, int pipe, cudaStream_t stream)
{
    return reg::launch_register_vo<__nv_bfloat16, 1>(p, warps, pipe, stream);
}

}  // namespace blip
