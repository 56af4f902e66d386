// k_batch.cu -- batched uniform-grid solves: the fused step over an (instance,
// block) work list, the per-instance residual/mass reduction, and per-instance state
// set-up and read-out.
#include "step_cart.cuh"

namespace sdugks {

// Batched: the (instance, block) work list, one item per CTA (PER_ITEM: the grid has a
// CTA for every item, and CTAs past the item count in device memory return) or walked
// by a fixed grid (a captured graph then stays valid while instances come and go).
// One item per CTA keeps the block routine free of the walk's loop-carried state: the
// walking form spills registers at four CTAs per SM, the per-item form does not.
template <int P, int TX, int TY, bool PER_ITEM>
__global__ void __launch_bounds__(cart_threads<TX, TY>(), cart_threads<TX, TY>() <= 320 ? 4 : 2)
k_step_batch(const CartInst *__restrict__ insts, const int2 *__restrict__ items, const int *__restrict__ n_items,
             int par)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    static_assert(sizeof(CartInst) % 4 == 0, "CartInst copies in 4-byte words");
    constexpr int NW = (int)(sizeof(CartInst) / 4);
    if constexpr (PER_ITEM) {
        // The work list and the instance records are written by the host only (stream
        // ordered before the launch), so the item and its record are read before the
        // wait on the previous step: the record goes to shared memory while that step
        // ends, and the block routine reads its fields there.  Every 16th CTA asks L2
        // for the 128-byte line of the items ITEM_AHEAD places on (an in-bounds hint),
        // so that the CTAs of later waves find their item in L2 although the step's
        // state streams through it.
        constexpr int ITEM_AHEAD = 2048;
        __shared__ __align__(16) CartInst s_one;
        const int n = *n_items;
        if ((int)blockIdx.x >= n) return;
        if (threadIdx.x == 0 && (blockIdx.x & 15) == 0 && (int)blockIdx.x + ITEM_AHEAD < n)
            asm volatile("prefetch.global.L2 [%0];" ::"l"(items + blockIdx.x + ITEM_AHEAD));
        const int2 it = items[blockIdx.x];
        const uint32_t *src = reinterpret_cast<const uint32_t *>(insts + it.x);
        for (int q = threadIdx.x; q < NW; q += blockDim.x) reinterpret_cast<uint32_t *>(&s_one)[q] = src[q];
        step_dependency_wait();
        __syncthreads();
        const int bx = it.y & 0xFFFF, by = it.y >> 16;   // the block's coordinates, packed on the host
        if (cart_block_interior<TX, TY>(s_one, bx, by)) cart_tile<P, TX, TY, false, true>(s_one, par, bx, by, smem_raw);
        else cart_tile<P, TX, TY, false, false>(s_one, par, bx, by, smem_raw);
    } else {
        step_dependency_wait();
        // each item's instance record is copied to shared memory, so that the block
        // routine reads its fields there instead of from global memory: two buffers,
        // the next item's record copied while the current item ends, so that one
        // barrier between items both publishes it and separates the items' use of the
        // staging memory
        __shared__ __align__(16) CartInst s_inst[2];
        const int n = *n_items;
        auto fetch = [&](int w, int b) {
            const uint32_t *src = reinterpret_cast<const uint32_t *>(insts + items[w].x);
            for (int q = threadIdx.x; q < NW; q += blockDim.x) reinterpret_cast<uint32_t *>(&s_inst[b])[q] = src[q];
        };
        if ((int)blockIdx.x < n) fetch(blockIdx.x, 0);
        __syncthreads();
        int b = 0;
        for (int w = blockIdx.x; w < n; w += gridDim.x, b ^= 1) {
            const int2 it = items[w];
            const CartInst &m = s_inst[b];
            const int bx = it.y & 0xFFFF, by = it.y >> 16;   // the block's coordinates, packed on the host
            if (cart_block_interior<TX, TY>(m, bx, by)) cart_tile<P, TX, TY, false, true>(m, par, bx, by, smem_raw);
            else cart_tile<P, TX, TY, false, false>(m, par, bx, by, smem_raw);
            if (w + (int)gridDim.x < n) fetch(w + gridDim.x, b ^ 1);
            __syncthreads();
        }
    }
}

namespace {

constexpr int BTX = 16, BTY = BATCH_TY;
constexpr int RT = BTX * BTY;              // residual block = one block of cells

template <int P> cudaError_t prep_p() {
    cudaError_t e = cudaFuncSetAttribute(k_step_batch<P, BTX, BTY, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)cart_smem<P, BTX, BTY>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_step_batch<P, BTX, BTY, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)cart_smem<P, BTX, BTY>());
    return e;
}

template <int P> int occ_p() {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step_batch<P, BTX, BTY, false>, cart_threads<BTX, BTY>(),
                                                      cart_smem<P, BTX, BTY>()) != cudaSuccess)
        return 1;
    return n > 0 ? n : 1;
}

template <int P>
cudaError_t launch_batch_p(const CartInst *insts, const int2 *items, const int *n_items, int grid, bool per_item,
                           int parity, cudaStream_t st)
{
    if (per_item)
        return launch_step_kernel(k_step_batch<P, BTX, BTY, true>, dim3(grid), dim3(cart_threads<BTX, BTY>()),
                                  cart_smem<P, BTX, BTY>(), st, insts, items, n_items, parity);
    return launch_step_kernel(k_step_batch<P, BTX, BTY, false>, dim3(grid), dim3(cart_threads<BTX, BTY>()),
                              cart_smem<P, BTX, BTY>(), st, insts, items, n_items, parity);
}

__device__ void bsum4(double v[4], double *out)
{
    __shared__ double sh[RT / 32][4];
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
            double x = lane < RT / 32 ? sh[lane][k] : 0.0;
            for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
            if (lane == 0) out[k] = x;
        }
    }
    __syncthreads();
}

// per item: sums over the block's cells of (U-U0)^2+(V-V0)^2, U0^2+V0^2, V rho and
// non-finite W; refreshes the snapshot
__global__ void __launch_bounds__(RT) k_bresid_partial(const CartInst *__restrict__ insts, const int2 *__restrict__ items,
                                                       const int *__restrict__ n_items, int par,
                                                       double *__restrict__ partial)
{
    const int n = *n_items;
    for (int w = blockIdx.x; w < n; w += gridDim.x) {
        const int2 it = items[w];
        const CartInst &m = insts[it.x];
        const int i = (it.y & 0xFFFF) * BTX + threadIdx.x % BTX, j = (it.y >> 16) * BTY + threadIdx.x / BTX;
        double v[4] = {0.0, 0.0, 0.0, 0.0};
        if (i < m.nx && j < m.ny) {
            const int64_t g = i + (int64_t)m.pitch * j, np = m.npad;
            const double *W = m.W[par];
            // batched precisions compute in the deviation form: W[0] = rho - 1
            const double w0 = 1.0 + W[g], w1 = W[np + g], w2 = W[2 * np + g];
            const double U = w1 / w0, V = w2 / w0, U0 = m.snap[g], V0 = m.snap[np + g];
            v[0] = (U - U0) * (U - U0) + (V - V0) * (V - V0);
            v[1] = U0 * U0 + V0 * V0;
            v[2] = m.dx * m.dy * w0;
            v[3] = (isfinite(w0) && isfinite(w1) && isfinite(w2) && w0 != 0.0) ? 0.0 : 1.0;
            m.snap[g] = U;
            m.snap[np + g] = V;
        }
        bsum4(v, partial + 4 * (int64_t)w);
    }
}

// one block per instance: fixed-order sum of its items' partials
__global__ void __launch_bounds__(RT) k_bresid_final(const CartInst *__restrict__ insts, int n_inst,
                                                     const double *__restrict__ partial, double *__restrict__ out)
{
    for (int q = blockIdx.x; q < n_inst; q += gridDim.x) {
        const CartInst &m = insts[q];
        double v[4] = {0.0, 0.0, 0.0, 0.0};
        if (m.n_items > 0)
            for (int w = threadIdx.x; w < m.n_items; w += RT)
                for (int k = 0; k < 4; k++) v[k] += partial[4 * (int64_t)(m.item0 + w) + k];
        bsum4(v, out + 4 * (int64_t)q);
    }
}

template <int P>
__global__ void k_binit(const CartInst *__restrict__ mp, int par, const double *__restrict__ rho,
                        const double *__restrict__ u)
{
    using R = typename Store<P>::R;
    using T = typename Store<P>::T;
    const CartInst &m = *mp;
    const int64_t n = (int64_t)m.nx * m.ny, np = m.npad;
    T *f = static_cast<T *>(m.f[par]);
    double *W = m.W[par];
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t g = q % m.nx + (int64_t)m.pitch * (q / m.nx);
        const double r = rho ? rho[q] : 1.0, ux = u ? u[2 * q] : 0.0, uy = u ? u[2 * q + 1] : 0.0;
        // deviation form (every batched precision computes in FP32): W[0] = rho - 1 and
        // f stored as g = f - w (FP32) or as the deviation from feq (bf16, fp16)
        W[g] = r - 1.0; W[np + g] = r * ux; W[2 * np + g] = r * uy;
        m.snap[g] = ux; m.snap[np + g] = uy;
        double fe[NQ];
        feq9fd<double>(r - 1.0, r, ux, uy, fe);
        R drr, rr, x, y, feR[NQ];
        macro_of<R>(r - 1.0, r * ux, r * uy, drr, rr, x, y);
        feq9fd<R>(drr, rr, x, y, feR);
#pragma unroll
        for (int a = 0; a < NQ; a++) f[a * np + g] = Store<P>::enc(R(fe[a]), feR[a], a);
    }
}

__global__ void k_bmacros(const CartInst *__restrict__ mp, int par, double *__restrict__ rho, double *__restrict__ u)
{
    const CartInst &m = *mp;
    const int64_t n = (int64_t)m.nx * m.ny, np = m.npad;
    const double *W = m.W[par];
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t g = q % m.nx + (int64_t)m.pitch * (q / m.nx);
        const double w0 = 1.0 + W[g];      // deviation form: W[0] = rho - 1
        if (rho) rho[q] = w0;
        if (u) { u[2 * q] = W[np + g] / w0; u[2 * q + 1] = W[2 * np + g] / w0; }
    }
}

int grid_of(int64_t n) { int64_t b = (n + 255) / 256; return (int)(b < 1 ? 1 : (b > 2048 ? 2048 : b)); }

}  // namespace

cudaError_t prepare_batch(int prec)
{
    if (prec == P_FP16DEV) return prep_p<P_FP16DEV>();
    return prec == P_BF16DEV ? prep_p<P_BF16DEV>() : prep_p<P_FP32>();
}

int batch_ctas_per_sm(int prec)
{
    if (prec == P_FP16DEV) return occ_p<P_FP16DEV>();
    return prec == P_BF16DEV ? occ_p<P_BF16DEV>() : occ_p<P_FP32>();
}

cudaError_t launch_step_batch(int prec, const CartInst *insts, const int2 *items, const int *n_items, int grid,
                              bool per_item, int parity, cudaStream_t st)
{
    if (prec == P_BF16DEV) return launch_batch_p<P_BF16DEV>(insts, items, n_items, grid, per_item, parity, st);
    if (prec == P_FP16DEV) return launch_batch_p<P_FP16DEV>(insts, items, n_items, grid, per_item, parity, st);
    return launch_batch_p<P_FP32>(insts, items, n_items, grid, per_item, parity, st);
}

cudaError_t launch_batch_residual(const CartInst *insts, int n_inst, const int2 *items, const int *n_items, int grid,
                                  int parity, double *partial, double *out, cudaStream_t st)
{
    k_bresid_partial<<<grid, RT, 0, st>>>(insts, items, n_items, parity, partial);
    if (n_inst > 0) k_bresid_final<<<n_inst < 1024 ? n_inst : 1024, RT, 0, st>>>(insts, n_inst, partial, out);
    return cudaGetLastError();
}

cudaError_t launch_batch_init(int prec, const CartInst *inst_host, const CartInst *inst_dev, int parity,
                              const double *rho, const double *u, cudaStream_t st)
{
    const int g = grid_of((int64_t)inst_host->nx * inst_host->ny);
    if (prec == P_BF16DEV) k_binit<P_BF16DEV><<<g, 256, 0, st>>>(inst_dev, parity, rho, u);
    else if (prec == P_FP16DEV) k_binit<P_FP16DEV><<<g, 256, 0, st>>>(inst_dev, parity, rho, u);
    else k_binit<P_FP32><<<g, 256, 0, st>>>(inst_dev, parity, rho, u);
    return cudaGetLastError();
}

cudaError_t launch_batch_macros(const CartInst *inst_host, const CartInst *inst_dev, int parity, double *rho, double *u,
                                cudaStream_t st)
{
    k_bmacros<<<grid_of((int64_t)inst_host->nx * inst_host->ny), 256, 0, st>>>(inst_dev, parity, rho, u);
    return cudaGetLastError();
}

}  // namespace sdugks
