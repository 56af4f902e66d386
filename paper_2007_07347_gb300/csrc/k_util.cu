// k_util.cu -- state conversions between the caller's layout and the internal SoA
// layout, macroscopic fields, and the FP64 residual / mass reduction.
#include "d2q9.cuh"

namespace sdugks {

namespace {

constexpr int UT = 256;

// FP64 equilibrium used where a state is created from (rho, u): feq itself (FP64
// storage) or its deviation feq - w (the FP32-compute precisions, which store g = f - w).
template <int P> __device__ void feq_state(double rho, double ux, double uy, double out[NQ])
{
    if constexpr (Dev<P>::ON) feq9fd<double>(rho - 1.0, rho, ux, uy, out);
    else feq9<double>(rho, ux, uy, out);
}

// The equilibrium of the stored W in the kernels' form and compute precision (the one
// the bf16 / fp16 codecs measure their deviations from).
template <int P> __device__ void feq_of_W(double w0, double w1, double w2, typename Store<P>::R out[NQ])
{
    using R = typename Store<P>::R;
    R dr, r, x, y;
    macro_of<R>(w0, w1, w2, dr, r, x, y);
    if constexpr (Dev<P>::ON) feq9fd<R>(dr, r, x, y, out);
    else feq9<R>(r, x, y, out);
}

template <int P>
__global__ void k_init(int64_t n, int64_t npad, const int32_t *__restrict__ perm, const int32_t *__restrict__ loc,
                       const double *__restrict__ rho_in,
                       const double *__restrict__ u_in, typename Store<P>::T *__restrict__ f, double *__restrict__ W)
{
    using R = typename Store<P>::R;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = perm[q], i = loc ? loc[q] : q;
        const double rho = rho_in ? rho_in[p] : 1.0;
        const double ux = u_in ? u_in[2 * p] : 0.0, uy = u_in ? u_in[2 * p + 1] : 0.0;
        const double w0 = rho - rho_ref<P>(), w1 = rho * ux, w2 = rho * uy;
        W[i] = w0; W[npad + i] = w1; W[2 * npad + i] = w2;
        double fe[NQ];
        feq_state<P>(rho, ux, uy, fe);
        R feR[NQ];
        feq_of_W<P>(w0, w1, w2, feR);
#pragma unroll
        for (int a = 0; a < NQ; a++) f[a * npad + i] = Store<P>::enc(R(fe[a]), feR[a], a);
    }
}

template <int P>
__global__ void k_pack(int64_t n, int64_t npad, const int32_t *__restrict__ perm, const int32_t *__restrict__ loc,
                       const typename Store<P>::T *__restrict__ f,
                       const double *__restrict__ W, double *__restrict__ f_out, double *__restrict__ W_out)
{
    using R = typename Store<P>::R;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = perm[q], i = loc ? loc[q] : q;
        R fe[NQ];
        feq_of_W<P>(W[i], W[npad + i], W[2 * npad + i], fe);
        if (f_out) {
            // the kernels' form back to f (g + w in FP64 for the FP32-compute precisions)
#pragma unroll
            for (int a = 0; a < NQ; a++)
                f_out[NQ * p + a] = (double)Store<P>::dec(f[a * npad + i], fe[a], a) + (Dev<P>::ON ? wq<double>(a) : 0.0);
        }
        if (W_out) {
            W_out[3 * p] = W[i] + rho_ref<P>();
            for (int d = 1; d < 3; d++) W_out[3 * p + d] = W[d * npad + i];
        }
    }
}

template <int P>
__global__ void k_unpack(int64_t n, int64_t npad, const int32_t *__restrict__ perm, const int32_t *__restrict__ loc,
                         const double *__restrict__ f_in,
                         const double *__restrict__ W_in, typename Store<P>::T *__restrict__ f, double *__restrict__ W)
{
    using R = typename Store<P>::R;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = perm[q], i = loc ? loc[q] : q;
        const double w0 = W_in[3 * p] - rho_ref<P>();
        W[i] = w0;
        for (int d = 1; d < 3; d++) W[d * npad + i] = W_in[3 * p + d];
        R fe[NQ];
        feq_of_W<P>(w0, W_in[3 * p + 1], W_in[3 * p + 2], fe);
#pragma unroll
        for (int a = 0; a < NQ; a++)
            f[a * npad + i] = Store<P>::enc(R(f_in[NQ * p + a] - (Dev<P>::ON ? wq<double>(a) : 0.0)), fe[a], a);
    }
}

__global__ void k_macros(int64_t n, int64_t npad, const int32_t *__restrict__ perm, const int32_t *__restrict__ loc,
                         const double *__restrict__ W, double rr,
                         double *__restrict__ rho, double *__restrict__ u)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = perm[q], i = loc ? loc[q] : q;
        const double w0 = rr + W[i];
        if (rho) rho[p] = w0;
        if (u) {
            u[2 * p] = W[npad + i] / w0;
            u[2 * p + 1] = W[2 * npad + i] / w0;
        }
    }
}

// Fixed-order block sum of 4 doubles (warp shuffles, then one warp over the warps).
__device__ void block_sum4(double v[4], double *out)
{
    __shared__ double sh[UT / 32][4];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 4; k++)
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    if (lane == 0)
        for (int k = 0; k < 4; k++) sh[wid][k] = v[k];
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int k = 0; k < 4; k++) {
            double x = lane < UT / 32 ? sh[lane][k] : 0.0;
            for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
            if (lane == 0) out[k] = x;
        }
    }
}

// Residual terms per block: sum (U-U0)^2+(V-V0)^2, sum U0^2+V0^2, sum V rho, and a
// count of non-finite W; refreshes the snapshot (U0, V0) <- (U, V).  rho = rr + W[0].
__global__ void __launch_bounds__(UT) k_resid_partial(int64_t n, int64_t npad, const int32_t *__restrict__ loc,
                                                      const double *__restrict__ W, double rr,
                                                      const double *__restrict__ vol, double *__restrict__ snap,
                                                      double *__restrict__ partial)
{
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for (int64_t q = blockIdx.x * (int64_t)UT + threadIdx.x; q < n; q += (int64_t)gridDim.x * UT) {
        const int64_t i = loc ? loc[q] : q;
        const double w0 = rr + W[i], w1 = W[npad + i], w2 = W[2 * npad + i];
        const double U = w1 / w0, V = w2 / w0;
        const double U0 = snap[i], V0 = snap[npad + i];
        const double dU = U - U0, dV = V - V0;
        v[0] += dU * dU + dV * dV;
        v[1] += U0 * U0 + V0 * V0;
        v[2] += vol[i] * w0;
        v[3] += (isfinite(w0) && isfinite(w1) && isfinite(w2) && w0 != 0.0) ? 0.0 : 1.0;
        snap[i] = U;
        snap[npad + i] = V;
    }
    block_sum4(v, partial + 4 * (int64_t)blockIdx.x);
}

__global__ void __launch_bounds__(UT) k_resid_final(int nb, const double *__restrict__ partial, double *__restrict__ out)
{
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nb; b += UT)
        for (int k = 0; k < 4; k++) v[k] += partial[4 * b + k];
    block_sum4(v, out);
}

int grid_for(int64_t n) {
    int64_t b = (n + UT - 1) / UT;
    return (int)(b < 1 ? 1 : (b > 4096 ? 4096 : b));
}

}  // namespace

cudaError_t launch_init_state(int prec, int64_t n, int64_t npad, const int32_t *perm, const int32_t *loc,
                              const double *rho, const double *u, void *f, double *W, cudaStream_t st)
{
    const int g = grid_for(n);
    if (prec == P_FP64) k_init<P_FP64><<<g, UT, 0, st>>>(n, npad, perm, loc, rho, u, (double *)f, W);
    else if (prec == P_FP32) k_init<P_FP32><<<g, UT, 0, st>>>(n, npad, perm, loc, rho, u, (float *)f, W);
    else if (prec == P_FP16DEV) k_init<P_FP16DEV><<<g, UT, 0, st>>>(n, npad, perm, loc, rho, u, (__half *)f, W);
    else k_init<P_BF16DEV><<<g, UT, 0, st>>>(n, npad, perm, loc, rho, u, (__nv_bfloat16 *)f, W);
    return cudaGetLastError();
}

cudaError_t launch_pack_state(int prec, int64_t n, int64_t npad, const int32_t *perm, const int32_t *loc, const void *f,
                              const double *W, double *f_out, double *W_out, cudaStream_t st)
{
    const int g = grid_for(n);
    if (prec == P_FP64)
        k_pack<P_FP64><<<g, UT, 0, st>>>(n, npad, perm, loc, (const double *)f, W, f_out, W_out);
    else if (prec == P_FP32)
        k_pack<P_FP32><<<g, UT, 0, st>>>(n, npad, perm, loc, (const float *)f, W, f_out, W_out);
    else if (prec == P_FP16DEV)
        k_pack<P_FP16DEV><<<g, UT, 0, st>>>(n, npad, perm, loc, (const __half *)f, W, f_out, W_out);
    else
        k_pack<P_BF16DEV><<<g, UT, 0, st>>>(n, npad, perm, loc, (const __nv_bfloat16 *)f, W, f_out, W_out);
    return cudaGetLastError();
}

cudaError_t launch_unpack_state(int prec, int64_t n, int64_t npad, const int32_t *perm, const int32_t *loc,
                                const double *f_in, const double *W_in, void *f, double *W, cudaStream_t st)
{
    const int g = grid_for(n);
    if (prec == P_FP64)
        k_unpack<P_FP64><<<g, UT, 0, st>>>(n, npad, perm, loc, f_in, W_in, (double *)f, W);
    else if (prec == P_FP32)
        k_unpack<P_FP32><<<g, UT, 0, st>>>(n, npad, perm, loc, f_in, W_in, (float *)f, W);
    else if (prec == P_FP16DEV)
        k_unpack<P_FP16DEV><<<g, UT, 0, st>>>(n, npad, perm, loc, f_in, W_in, (__half *)f, W);
    else
        k_unpack<P_BF16DEV><<<g, UT, 0, st>>>(n, npad, perm, loc, f_in, W_in, (__nv_bfloat16 *)f, W);
    return cudaGetLastError();
}

cudaError_t launch_macros(int64_t n, int64_t npad, const int32_t *perm, const int32_t *loc, const double *W, double rr,
                          double *rho, double *u, cudaStream_t st)
{
    k_macros<<<grid_for(n), UT, 0, st>>>(n, npad, perm, loc, W, rr, rho, u);
    return cudaGetLastError();
}

int residual_blocks(int64_t n) {
    int64_t b = (n + 4 * UT - 1) / (4 * UT);
    return (int)(b < 1 ? 1 : (b > 1024 ? 1024 : b));
}

cudaError_t launch_residual(int64_t n, int64_t npad, const int32_t *loc, const double *W, double rr, const double *vol,
                            double *snap, double *partial, int n_blocks, double *out, cudaStream_t st)
{
    k_resid_partial<<<n_blocks, UT, 0, st>>>(n, npad, loc, W, rr, vol, snap, partial);
    k_resid_final<<<1, UT, 0, st>>>(n_blocks, partial, out);
    return cudaGetLastError();
}

}  // namespace sdugks
