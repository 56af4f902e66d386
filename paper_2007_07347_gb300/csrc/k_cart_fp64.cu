// k_cart_fp64.cu -- FP64 instance of the Cartesian fused step (built with --fmad=false).
#include "step_cart.cuh"

namespace sdugks {

cudaError_t prepare_cart_fp64() { return prepare_cart_p<P_FP64, 16, 16>(); }

cudaError_t launch_cart_fp64(const CartInst &m, int parity, cudaStream_t st)
{
    return launch_cart_p<P_FP64, 16, 16>(m, parity, st);
}

}  // namespace sdugks
