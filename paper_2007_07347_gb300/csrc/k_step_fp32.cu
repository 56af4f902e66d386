// k_step_fp32.cu -- FP32-compute instances of the fused tiled step: f stored in FP32,
// or as a bf16 or fp16 scaled deviation from the equilibrium.
#include "step_tiled.cuh"

namespace sdugks {

cudaError_t prepare_tiled_fp32(int prec)
{
    if (prec == P_FP16DEV) return prepare_tiled_p<P_FP16DEV>();
    return prec == P_BF16DEV ? prepare_tiled_p<P_BF16DEV>() : prepare_tiled_p<P_FP32>();
}

cudaError_t launch_step_tiled_fp32(int prec, const TiledMesh &m, const Coefs &c, const void *f_in, void *f_out,
                                   const double *W_in, double *W_out, cudaStream_t st)
{
    if (prec == P_BF16DEV) return launch_tiled_p<P_BF16DEV>(m, c, f_in, f_out, W_in, W_out, st);
    if (prec == P_FP16DEV) return launch_tiled_p<P_FP16DEV>(m, c, f_in, f_out, W_in, W_out, st);
    return launch_tiled_p<P_FP32>(m, c, f_in, f_out, W_in, W_out, st);
}

}  // namespace sdugks
