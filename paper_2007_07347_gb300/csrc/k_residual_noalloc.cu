// k_residual_noalloc.cu -- the convergence residual and mass reduction over
// caller-owned device arrays, with its scratch in a fixed device array instead of
// memory the library allocates.
//
// For callers that cannot call cudaMalloc: code running where an allocation may not
// happen (inside a region whose memory is managed by someone else, a real-time loop
// that must not touch the allocator, an embedding runtime that forbids driver
// allocations).  The per-block partial sums live in `g_resid_scratch` below, a
// file-scope device array that every GPU which loads this library holds until the
// process exits; every call shares it.
#include <atomic>
#include <cstdint>
#include <cstdio>
#include <cuda_runtime.h>

#include "sdugks.h"
#include "sdugks_internal.h"

namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_CELLS_PER_BLOCK = 4 * NA_THREADS;       // each block reduces up to 1024 cells
constexpr int NA_MAX_BLOCKS = 4096;                      // scratch: 4096 x 4 doubles = 128 KiB
constexpr int64_t NA_MAX_CELLS = (int64_t)NA_MAX_BLOCKS * NA_CELLS_PER_BLOCK;   // 4,194,304
constexpr int NA_MAX_DEVICES = 64;

// Per-block partial sums (sum dU^2 + dV^2, sum U0^2 + V0^2, sum V rho, non-finite count).
static __device__ __align__(256) double g_resid_scratch[NA_MAX_BLOCKS][4];

// Device address of g_resid_scratch on each device, looked up on the first call made
// with that device current.  Atomic, because host threads may make first calls at the
// same time; they look up and store the same value.
std::atomic<double *> g_scratch_ptr[NA_MAX_DEVICES];

__device__ void na_block_sum4(double v[4], double *out)
{
    __shared__ double sh[NA_THREADS / 32][4];
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
            double x = lane < NA_THREADS / 32 ? sh[lane][k] : 0.0;
            for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
            if (lane == 0) out[k] = x;
        }
    }
}

// Partial sums of block b over cells [b * 1024, (b + 1) * 1024); refreshes the snapshot.
__global__ void __launch_bounds__(NA_THREADS)
k_na_partial(int64_t n, const double *__restrict__ W, const double *__restrict__ vol, double *__restrict__ snap,
             double (*__restrict__ scratch)[4])
{
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    const int64_t base = (int64_t)blockIdx.x * NA_CELLS_PER_BLOCK;
    for (int r = 0; r < NA_CELLS_PER_BLOCK / NA_THREADS; r++) {
        const int64_t i = base + r * NA_THREADS + threadIdx.x;
        if (i >= n) break;
        const double w0 = W[3 * i], w1 = W[3 * i + 1], w2 = W[3 * i + 2];
        const double U = w1 / w0, V = w2 / w0;
        const double U0 = snap[2 * i], V0 = snap[2 * i + 1];
        const double dU = U - U0, dV = V - V0;
        v[0] += dU * dU + dV * dV;
        v[1] += U0 * U0 + V0 * V0;
        v[2] += vol[i] * w0;
        v[3] += (isfinite(w0) && isfinite(w1) && isfinite(w2) && w0 != 0.0) ? 0.0 : 1.0;
        snap[2 * i] = U;
        snap[2 * i + 1] = V;
    }
    na_block_sum4(v, scratch[blockIdx.x]);
}

// One block: fixed-order sum of the partials; out = (eps, mass, non-finite count).
__global__ void __launch_bounds__(NA_THREADS)
k_na_final(int nb, const double (*__restrict__ scratch)[4], double *__restrict__ out)
{
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nb; b += NA_THREADS)
        for (int k = 0; k < 4; k++) v[k] += scratch[b][k];
    __shared__ double tot[4];
    na_block_sum4(v, tot);
    __syncthreads();
    if (threadIdx.x == 0) {
        out[0] = tot[1] > 0.0 ? sqrt(tot[0]) / sqrt(tot[1]) : __longlong_as_double(0x7ff0000000000000LL);
        out[1] = tot[2];
        out[2] = tot[3];
    }
}

// failures are reported through sdugks_last_error(), like every other entry point
int na_fail(int code, const char *msg, cudaError_t e = cudaSuccess)
{
    char buf[256];
    if (e != cudaSuccess) snprintf(buf, sizeof buf, "%s: %s", msg, cudaGetErrorString(e));
    else snprintf(buf, sizeof buf, "%s", msg);
    return sdugks::set_error(code, buf);
}

}  // namespace

extern "C" int sdugks_residual_noalloc(int64_t n, const double *d_W, const double *d_vol, double *d_snap, double *d_out,
                                       void *stream)
{
    if (n <= 0 || !d_W || !d_vol || !d_snap || !d_out)
        return na_fail(SDUGKS_ERR_INVALID_ARG, "sdugks_residual_noalloc: n must be > 0 and every pointer non-NULL");
    if (n > NA_MAX_CELLS)
        return na_fail(SDUGKS_ERR_INVALID_ARG,
                       "sdugks_residual_noalloc: n exceeds the fixed scratch limit of 4194304 cells");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return na_fail(SDUGKS_ERR_CUDA, "sdugks_residual_noalloc: cudaGetDevice", e);
    if (dev < 0 || dev >= NA_MAX_DEVICES) return na_fail(SDUGKS_ERR_INVALID_ARG, "sdugks_residual_noalloc: device id >= 64");
    double *sp = g_scratch_ptr[dev].load(std::memory_order_relaxed);
    if (!sp) {
        // once per device, with that device current: the device address of the scratch
        // array (its host-side name is not a device address)
        e = cudaGetSymbolAddress((void **)&sp, g_resid_scratch);
        if (e != cudaSuccess || !sp)
            return na_fail(SDUGKS_ERR_CUDA, "sdugks_residual_noalloc: cudaGetSymbolAddress", e);
        g_scratch_ptr[dev].store(sp, std::memory_order_relaxed);
    }
    double (*scratch)[4] = reinterpret_cast<double (*)[4]>(sp);
    const int nb = (int)((n + NA_CELLS_PER_BLOCK - 1) / NA_CELLS_PER_BLOCK);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // every block writes its own partial row, so nothing has to be cleared first
    k_na_partial<<<nb, NA_THREADS, 0, st>>>(n, d_W, d_vol, d_snap, scratch);
    k_na_final<<<1, NA_THREADS, 0, st>>>(nb, scratch, d_out);
    e = cudaGetLastError();
    if (e != cudaSuccess) return na_fail(SDUGKS_ERR_CUDA, "sdugks_residual_noalloc: launch", e);
    return SDUGKS_OK;
}
