// k_cart.cu -- FP32-compute instances of the Cartesian fused step.  The FP64
// instance is built in its own unit (k_cart_fp64.cu) with --fmad=false.
#include "step_cart.cuh"

namespace sdugks {

// Block shapes of the FP32-compute instances: 16 x TY with TY in {16, 14, 8}
// (shape index 0, 1, 2).  FP64 uses 16 x 16 only.

cudaError_t prepare_cart_fp64();
cudaError_t launch_cart_fp64(const CartInst &m, int parity, cudaStream_t st);

template <int P> cudaError_t prepare_shapes()
{
    cudaError_t e = prepare_cart_p<P, 16, 16>();
    if (e == cudaSuccess) e = prepare_cart_p<P, 16, 14>();
    if (e == cudaSuccess) e = prepare_cart_p<P, 16, 8>();
    return e;
}

cudaError_t prepare_cart(int prec)
{
    if (prec == P_FP64) return prepare_cart_fp64();
    if (prec == P_FP16DEV) return prepare_shapes<P_FP16DEV>();
    return prec == P_BF16DEV ? prepare_shapes<P_BF16DEV>() : prepare_shapes<P_FP32>();
}

template <int P> cudaError_t launch_shape(int shape, const CartInst &m, int parity, cudaStream_t st)
{
    if (shape == 1) return launch_cart_p<P, 16, 14>(m, parity, st);
    if (shape == 2) return launch_cart_p<P, 16, 8>(m, parity, st);
    return launch_cart_p<P, 16, 16>(m, parity, st);
}

cudaError_t launch_step_cart(int prec, int shape, const CartInst &m, int parity, cudaStream_t st)
{
    if (prec == P_FP64) return launch_cart_fp64(m, parity, st);
    if (prec == P_BF16DEV) return launch_shape<P_BF16DEV>(shape, m, parity, st);
    if (prec == P_FP16DEV) return launch_shape<P_FP16DEV>(shape, m, parity, st);
    return launch_shape<P_FP32>(shape, m, parity, st);
}

template <int P, int TX, int TY> int occ_shape()
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step_cart<P, TX, TY>, cart_threads<TX, TY>(),
                                                      cart_smem<P, TX, TY>()) != cudaSuccess || n < 1)
        return 1;
    return n;
}

int cart_shape_occupancy(int prec, int shape)
{
    if (prec == P_FP64) return occ_shape<P_FP64, 16, 16>();
    if (prec == P_BF16DEV)
        return shape == 1 ? occ_shape<P_BF16DEV, 16, 14>() : shape == 2 ? occ_shape<P_BF16DEV, 16, 8>() : occ_shape<P_BF16DEV, 16, 16>();
    if (prec == P_FP16DEV)
        return shape == 1 ? occ_shape<P_FP16DEV, 16, 14>() : shape == 2 ? occ_shape<P_FP16DEV, 16, 8>() : occ_shape<P_FP16DEV, 16, 16>();
    return shape == 1 ? occ_shape<P_FP32, 16, 14>() : shape == 2 ? occ_shape<P_FP32, 16, 8>() : occ_shape<P_FP32, 16, 16>();
}

}  // namespace sdugks
