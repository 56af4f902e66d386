// k_cart.cu -- FP32-compute instances of the Cartesian fused step.  The FP64
// instance is built in its own unit (k_cart_fp64.cu) with --fmad=false.
#include "step_cart.cuh"

namespace sdugks {

constexpr int CTX = 16, CTY = 16;

cudaError_t prepare_cart_fp64();
cudaError_t launch_cart_fp64(const CartInst &m, int parity, cudaStream_t st);

cudaError_t prepare_cart(int prec)
{
    if (prec == P_FP64) return prepare_cart_fp64();
    if (prec == P_BF16DEV) return prepare_cart_p<P_BF16DEV, CTX, CTY>();
    return prepare_cart_p<P_FP32, CTX, CTY>();
}

cudaError_t launch_step_cart(int prec, const CartInst &m, int parity, cudaStream_t st)
{
    if (prec == P_FP64) return launch_cart_fp64(m, parity, st);
    if (prec == P_BF16DEV) return launch_cart_p<P_BF16DEV, CTX, CTY>(m, parity, st);
    return launch_cart_p<P_FP32, CTX, CTY>(m, parity, st);
}

}  // namespace sdugks
