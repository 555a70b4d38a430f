// Dispatch of the register-gather evaluation kernels (kernel template in
// blip_register.cuh, instantiations in blip_reg_*.cu).
#include "blip_internal.h"

namespace blip {

cudaError_t launch_eval(const EvalParams &p, int elem, int variant, int chunks, int warps,
                        cudaStream_t stream)
{
    if (warps < 1 || warps > 16) return cudaErrorInvalidValue;
    if (variant != VAR_REGISTER && variant != VAR_REGISTER_PIPE && variant != VAR_REGISTER_ROLLED &&
        variant != VAR_REGISTER_L1 && variant != VAR_REGISTER_LOCKSTEP &&
        variant != VAR_REGISTER_PIPE3)
        return cudaErrorInvalidValue;
    if (variant == VAR_REGISTER_PIPE3 && (elem != ELEM_F32 || chunks != 1))
        return cudaErrorInvalidValue;
    const int pipe = variant == VAR_REGISTER_PIPE ? 1
                   : variant == VAR_REGISTER_ROLLED ? 2
                   : variant == VAR_REGISTER_L1 ? 3
                   : variant == VAR_REGISTER_LOCKSTEP ? 4
                   : variant == VAR_REGISTER_PIPE3 ? 5 : 0;
    switch (elem) {
    case ELEM_F32:
        if (chunks == 1) return launch_register_f32_c1(p, warps, pipe, stream);
        if (chunks == 2) return launch_register_f32_c2(p, warps, pipe, stream);
        if (chunks == 3) return launch_register_f32_c3(p, warps, pipe, stream);
        return cudaErrorInvalidValue;
    case ELEM_BF16:
        return chunks == 1 ? launch_register_bf16(p, warps, pipe, stream) : cudaErrorInvalidValue;
    case ELEM_F16:
        return chunks == 1 ? launch_register_f16(p, warps, pipe, stream) : cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace blip
