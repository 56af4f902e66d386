// k_cart_fp64.cu -- FP64 instance of the Cartesian fused step (built with --fmad=false).
#include "step_cart.cuh"

namespace sdugks {

cudaError_t prepare_cart_fp64() { return prepare_cart_p<P_FP64, 16, 16>(); }

cudaError_t launch_cart_fp64(const CartInst &m, const CartTma *tma, bool general, int parity, cudaStream_t st)
{
    return launch_cart_p<P_FP64, 16, 16>(m, tma, general, parity, st);
}

int occ_cart_fp64(bool tma)
{
    return tma ? occ_cart_p<P_FP64, 16, 16, CART_SPECIALISED_TMA>() : occ_cart_p<P_FP64, 16, 16, CART_SPECIALISED>();
}

}  // namespace sdugks
