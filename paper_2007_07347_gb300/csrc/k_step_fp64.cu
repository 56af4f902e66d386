// k_step_fp64.cu -- FP64 instance of the fused tiled step.  Built with --fmad=false so
// that every FP64 product and sum is rounded separately, like the plain CPU
// evaluation it is checked against.
#include "step_tiled.cuh"

namespace sdugks {

cudaError_t prepare_tiled_fp64() { return prepare_tiled_p<P_FP64>(); }

cudaError_t launch_step_tiled_fp64(const TiledMesh &m, const Coefs &c, const void *f_in, void *f_out,
                                   const double *W_in, double *W_out, cudaStream_t st)
{
    return launch_tiled_p<P_FP64>(m, c, f_in, f_out, W_in, W_out, st);
}

}  // namespace sdugks
