// k_cart.cu -- FP32-compute instances of the Cartesian fused step.  The FP64
// instance is built in its own unit (k_cart_fp64.cu) with --fmad=false.
#include "step_cart.cuh"

namespace sdugks {

// Block shapes of the FP32-compute instances: 16 x TY with TY in {16, 14, 8}
// (shape index 0, 1, 2).  FP64 uses 16 x 16 only.

cudaError_t prepare_cart_fp64();
cudaError_t launch_cart_fp64(const CartInst &m, const CartTma *tma, bool general, int parity, cudaStream_t st);
int occ_cart_fp64(bool tma);

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

template <int P>
cudaError_t launch_shape(int shape, const CartInst &m, const CartTma *tma, bool general, int parity, cudaStream_t st)
{
    if (shape == 1) return launch_cart_p<P, 16, 14>(m, tma, general, parity, st);
    if (shape == 2) return launch_cart_p<P, 16, 8>(m, tma, general, parity, st);
    return launch_cart_p<P, 16, 16>(m, tma, general, parity, st);
}

cudaError_t launch_step_cart(int prec, int shape, const CartInst &m, const CartTma *tma, bool general, int parity,
                             cudaStream_t st)
{
    if (prec == P_FP64) return launch_cart_fp64(m, tma, general, parity, st);
    if (prec == P_BF16DEV) return launch_shape<P_BF16DEV>(shape, m, tma, general, parity, st);
    if (prec == P_FP16DEV) return launch_shape<P_FP16DEV>(shape, m, tma, general, parity, st);
    return launch_shape<P_FP32>(shape, m, tma, general, parity, st);
}

template <int P, int TX, int TY> int occ_shape(bool tma)
{
    return tma ? occ_cart_p<P, TX, TY, CART_SPECIALISED_TMA>() : occ_cart_p<P, TX, TY, CART_SPECIALISED>();
}

int cart_shape_occupancy(int prec, int shape, bool tma)
{
    if (prec == P_FP64) return occ_cart_fp64(tma);
    if (prec == P_BF16DEV)
        return shape == 1 ? occ_shape<P_BF16DEV, 16, 14>(tma) : shape == 2 ? occ_shape<P_BF16DEV, 16, 8>(tma) : occ_shape<P_BF16DEV, 16, 16>(tma);
    if (prec == P_FP16DEV)
        return shape == 1 ? occ_shape<P_FP16DEV, 16, 14>(tma) : shape == 2 ? occ_shape<P_FP16DEV, 16, 8>(tma) : occ_shape<P_FP16DEV, 16, 16>(tma);
    return shape == 1 ? occ_shape<P_FP32, 16, 14>(tma) : shape == 2 ? occ_shape<P_FP32, 16, 8>(tma) : occ_shape<P_FP32, 16, 16>(tma);
}

// ---- tensor maps of the TMA staging

namespace {
// cuTensorMapEncodeTiled, taken from the driver through the runtime (no libcuda link)
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encoder()
{
    static const EncodeTiledFn fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return (EncodeTiledFn) nullptr;
        return reinterpret_cast<EncodeTiledFn>(p);
    }();
    return fn;
}

// (x, y, plane) view of a [planes][npad] array with rows of `pitch` elements; boxes of
// bw x by x planes elements
bool encode3(EncodeTiledFn enc, CUtensorMap &map, CUtensorMapDataType dt, size_t es, void *base, int nx, int ny,
             int planes, int64_t pitch, int64_t npad, int bw, int by)
{
    const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)planes};
    const cuuint64_t strides[2] = {(cuuint64_t)(pitch * (int64_t)es), (cuuint64_t)(npad * (int64_t)es)};
    const cuuint32_t box[3] = {(cuuint32_t)bw, (cuuint32_t)by, (cuuint32_t)planes};
    const cuuint32_t estr[3] = {1, 1, 1};
    return enc(&map, dt, 3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int P, int TY> cudaError_t make_tma_p(const CartInst &m, CartTma &out)
{
    using B = CartTmaBox<P, 16, TY>;
    using T = typename Store<P>::T;
    const EncodeTiledFn enc = encoder();
    if (!enc) return cudaErrorNotSupported;
    const CUtensorMapDataType ft = sizeof(T) == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                                                  : (sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_UINT16);
    for (int b = 0; b < 2; b++) {
        if (!encode3(enc, out.f[b], ft, sizeof(T), m.f[b], m.nx, m.ny, NQ, m.pitch, m.npad, B::BW, TY + 4) ||
            !encode3(enc, out.W[b], CU_TENSOR_MAP_DATA_TYPE_FLOAT64, sizeof(double), m.W[b], m.nx, m.ny, 3, m.pitch,
                     m.npad, B::WBW, TY + 4))
            return cudaErrorInvalidValue;
    }
    return cudaSuccess;
}

template <int P> cudaError_t make_tma_shape(int shape, const CartInst &m, CartTma &out)
{
    if (shape == 1) return make_tma_p<P, 14>(m, out);
    if (shape == 2) return make_tma_p<P, 8>(m, out);
    return make_tma_p<P, 16>(m, out);
}
}  // namespace

cudaError_t make_cart_tma(int prec, int shape, const CartInst &m, CartTma &out)
{
    if (prec == P_FP64) return make_tma_p<P_FP64, 16>(m, out);
    if (prec == P_BF16DEV) return make_tma_shape<P_BF16DEV>(shape, m, out);
    if (prec == P_FP16DEV) return make_tma_shape<P_FP16DEV>(shape, m, out);
    return make_tma_shape<P_FP32>(shape, m, out);
}

}  // namespace sdugks
