// k_dvm.cu -- the S-DUGKS step on a discrete velocity grid (rarefied flow, Sec. IV
// micro cavity; diffuse walls of Sec. III).
//
// The mesh is small and the velocity grid large (10^4 nodes), so the work is spread
// over velocities: one CTA per cell or per face walks all Q velocities with its
// threads, and the moments a step needs (the interface W of every face, the
// macroscopic flux of every cell) are block reductions in a fixed order.  Two launches
// per step (k_dvm_fbp only when the state is new):
//   k_dvm_fbp   per cell: fbar+ = a f + b feq(W^n)                      (Eq. fbarplus)
//   k_dvm_face  per face: characteristic reconstruction from the upwind cell with its
//               LLSR gradient evaluated on the spot (Eqs. fbpsource, fbar), interface
//               moments and Maxwellian (Eqs. Macro, Feq), f_b (Eq. f_t_n+1); walls by
//               diffuse scattering; writes xi . n l f_b per face and velocity
//   k_dvm_cell  per cell: F = sum of its faces' fluxes (Eq. MesoFlux), its moments
//               (Eq. MacroFlux) update W in FP64 (Eq. MacroUpdate), then f (Eq. fn+1)
//               and the next step's fbar+ (Eq. fbarplus with W^{n+1})
// The faces are numbered in the order of their first cell and the cell kernel takes the
// cells backwards, so each kernel first reads what the other wrote last (still in L2).
// W = (rho, rho u, rho E) per cell in FP64; f and the scratch arrays in the compute
// precision.  When nv is a multiple of 4 every thread takes 4 consecutive velocities at
// a time with 16-byte vector loads and stores (V = 4); otherwise one (V = 1).  The
// arithmetic of a velocity is the same either way.  The velocity grid is the tensor
// product of one axis' nv nodes with one weight, so every CTA stages the nv nodes in
// shared memory and reads a velocity's (x, y) from there.  The Maxwellian is that of
// Eq. Feq with exponent |xi - u|^2 / (2 R T), D = 2, sampled at the nodes and multiplied
// by the node weight.
#include "sdugks_internal.h"

#include <cuda_runtime.h>

namespace sdugks {
namespace {

// threads per CTA of the three step kernels (a CTA walks its cell's or face's
// velocities).  On the 40 x 40 x 100^2 micro cavity (GB300) 384 or 512 threads for the
// cell kernel and 512 or 1024 for fbar+ measured the same or slower than 256.  The face
// kernel (128 registers) runs four CTAs of 128 threads per SM: 14 % faster than two of
// 256, since a CTA waiting at the barrier before its second pass then holds fewer warps.
constexpr int FBP_THREADS = 256, FACE_THREADS = 128, CELL_THREADS = 256;

template <class R> struct DvmR;
template <> struct DvmR<double> {
    double a, b, c, r, dt, tie, inv1r;
    __device__ explicit DvmR(const Coefs &k) : a(k.a_plus), b(k.b_plus), c(k.c_face), r(k.r), dt(k.dt), tie(k.tie),
                                               inv1r(k.inv1r) {}
};
template <> struct DvmR<float> {
    float a, b, c, r, dt, tie, inv1r;
    __device__ explicit DvmR(const Coefs &k) : a(k.fa_plus), b(k.fb_plus), c(k.fc_face), r(k.fr), dt(k.fdt),
                                               tie(k.ftie), inv1r(k.finv1r) {}
};

// Maxwellian parameters of one state, computed once per CTA in FP64.
struct MaxP {
    double pre, ux, uy, inv2RT;
};
__device__ __forceinline__ MaxP max_params(double rho, double mx, double my, double rE)
{
    // two divisions (one thread runs this while its block waits)
    MaxP p;
    const double ir = 1.0 / rho;
    p.ux = mx * ir;
    p.uy = my * ir;
    const double RT = rE * ir - 0.5 * (p.ux * p.ux + p.uy * p.uy);
    const double iRT = 1.0 / RT;
    p.pre = rho * iRT * (0.5 / 3.14159265358979323846);
    p.inv2RT = 0.5 * iRT;
    return p;
}

// exp(-x) for the Maxwellian: FP64 exp; FP32 2^(-x log2 e) by the hardware base-2
// exponential (relative error below 2^-22), with log2 e folded into sp[3].
__device__ __forceinline__ float exp_neg(float x_log2e)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(-x_log2e));
    return y;
}
__device__ __forceinline__ double exp_neg(double x) { return exp(-x); }

// Maxwellian parameters in the compute precision: {pre, u_x, u_y, 1/(2RT)} (FP32:
// 1/(2RT) times log2 e)
template <class R> __device__ __forceinline__ void set_sp(R *sp, const MaxP &p)
{
    sp[0] = R(p.pre); sp[1] = R(p.ux); sp[2] = R(p.uy);
    sp[3] = sizeof(R) == 4 ? R(p.inv2RT * 1.4426950408889634) : R(p.inv2RT);
}

// The parameters of the state with moments (rho, rho u, rho E), in the compute
// precision.  FP64: by max_params.  FP32: the moments rounded to FP32 and the same
// formulas in FP32, so that the thread that forms them does not hold its block for the
// FP64 divisions of this GPU's narrow FP64 unit (the parameters were rounded to FP32
// before either way).
template <class R> __device__ __forceinline__ void state_sp(R *sp, double rho, double mx, double my, double rE);
template <> __device__ __forceinline__ void state_sp<double>(double *sp, double rho, double mx, double my, double rE)
{
    set_sp<double>(sp, max_params(rho, mx, my, rE));
}
template <> __device__ __forceinline__ void state_sp<float>(float *sp, double rho_d, double mx, double my, double rE)
{
    const float rho = (float)rho_d, ir = 1.0f / rho;
    const float ux = (float)mx * ir, uy = (float)my * ir;
    const float RT = (float)rE * ir - 0.5f * (ux * ux + uy * uy);
    const float iRT = 1.0f / RT;
    sp[0] = rho * iRT * (float)(0.5 / 3.14159265358979323846);
    sp[1] = ux;
    sp[2] = uy;
    sp[3] = 0.5f * iRT * 1.4426950408889634f;
}

template <class R>
__device__ __forceinline__ R maxwell(const R *sp, R x, R y, R w)
{
    const R cx = x - sp[1], cy = y - sp[2];
    return w * sp[0] * exp_neg((cx * cx + cy * cy) * sp[3]);
}

// Fixed-order block sum of NV per-thread values: warp sums by shuffles in the
// compute precision, the per-warp results of value k combined in FP64 by thread k (in
// warp order); the result in out[] on every thread.  Uses scratch[32 * NV] shared
// doubles.
template <int NV, class R>
__device__ __forceinline__ void block_sum(R v[NV], double *scratch, double out[NV])
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; k++) {
        R x = v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) scratch[k * 32 + warp] = double(x);
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        const int k = threadIdx.x;
        double t = 0.0;
        for (int w = 0; w < nw; w++) t += scratch[k * 32 + w];
        scratch[k * 32] = t;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; k++) out[k] = scratch[k * 32];
    __syncthreads();
}

// V consecutive values (V = 4: 16-byte vector accesses; the address is 16-byte aligned
// because rows start at multiples of Q values and Q is a multiple of 4).
template <class R, int V> struct VIO;
template <class R> struct VIO<R, 1> {
    static __device__ __forceinline__ void ld(const R *p, R v[1]) { v[0] = *p; }
    static __device__ __forceinline__ void st(R *p, const R v[1]) { *p = v[0]; }
};
template <> struct VIO<float, 4> {
    static __device__ __forceinline__ void ld(const float *p, float v[4]) {
        const float4 t = *reinterpret_cast<const float4 *>(p);
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    }
    static __device__ __forceinline__ void st(float *p, const float v[4]) {
        *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
    }
};
template <> struct VIO<double, 4> {
    static __device__ __forceinline__ void ld(const double *p, double v[4]) {
        const double2 a = reinterpret_cast<const double2 *>(p)[0], b = reinterpret_cast<const double2 *>(p)[1];
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
    static __device__ __forceinline__ void st(double *p, const double v[4]) {
        reinterpret_cast<double2 *>(p)[0] = make_double2(v[0], v[1]);
        reinterpret_cast<double2 *>(p)[1] = make_double2(v[2], v[3]);
    }
};

// Largest nv of the shared-memory node table (the API limit).
constexpr int MAX_NV = 1024;

// The nodes of one axis into shared memory.  They never change, so this runs before the
// wait on the previous kernel; the caller synchronises before the first use.
template <class R> __device__ __forceinline__ void load_nodes(R *vt, const DvmMesh &m)
{
    const R *g = static_cast<const R *>(m.vnode);
    for (int k = threadIdx.x; k < m.nv; k += blockDim.x) vt[k] = g[k];
}

// Where a thread's velocity groups lie on the grid.  Group starts are a fixed stride
// apart, so the grid position (j, i) of the first velocity, q = j + nv i, is stepped
// rather than divided.  With V = 4, nv is a multiple of 4: a group lies in one grid row.
struct VelWalk {
    int j, i, dj, di, nv;
    __device__ __forceinline__ VelWalk(int q0, int stride, int nv_) : nv(nv_)
    {
        j = q0 % nv_; i = q0 / nv_; dj = stride % nv_; di = stride / nv_;
    }
    __device__ __forceinline__ void next()
    {
        j += dj; i += di;
        if (j >= nv) { j -= nv; i++; }
    }
};

// (x, y) of the V velocities of a group from the node table.
template <class R, int V> struct VNodes;
template <class R> struct VNodes<R, 1> {
    static __device__ __forceinline__ void get(const R *vt, const VelWalk &w, R x[1], R y[1])
    {
        x[0] = vt[w.j]; y[0] = vt[w.i];
    }
};
template <> struct VNodes<float, 4> {
    static __device__ __forceinline__ void get(const float *vt, const VelWalk &w, float x[4], float y[4])
    {
        const float4 t = *reinterpret_cast<const float4 *>(vt + w.j);
        x[0] = t.x; x[1] = t.y; x[2] = t.z; x[3] = t.w;
        const float yy = vt[w.i];
        y[0] = yy; y[1] = yy; y[2] = yy; y[3] = yy;
    }
};
template <> struct VNodes<double, 4> {
    static __device__ __forceinline__ void get(const double *vt, const VelWalk &w, double x[4], double y[4])
    {
        const double2 a = reinterpret_cast<const double2 *>(vt + w.j)[0], b = reinterpret_cast<const double2 *>(vt + w.j)[1];
        x[0] = a.x; x[1] = a.y; x[2] = b.x; x[3] = b.y;
        const double yy = vt[w.i];
        y[0] = yy; y[1] = yy; y[2] = yy; y[3] = yy;
    }
};

// The values at q .. q+V-1 of a side's 1 + MAXF rows: rows[0] is the cell's fbar+ row,
// rows[1..4] its neighbours' (a missing neighbour repeats the cell's own row with a zero
// offset, which adds nothing); one vector load per row.
template <class R, int V>
__device__ __forceinline__ void load_rows(const R *const *rows, int q, R v[1 + MAXF][V])
{
#pragma unroll
    for (int k = 0; k < 1 + MAXF; k++) VIO<R, V>::ld(rows[k] + q, v[k]);
}

// fbar+ of a cell's velocities plus (r - xi dt) . sigma, sigma the cell's LLSR gradient,
// from the row values of load_rows.
template <class R, int V>
__device__ __forceinline__ void reconstruct_vals(const R v[1 + MAXF][V], const R *d, const R *ai, R rx, R ry,
                                                 const R *xx, const R *xy, R dt, R out[V])
{
    R bx[V], by[V];
#pragma unroll
    for (int j = 0; j < V; j++) { bx[j] = R(0); by[j] = R(0); }
#pragma unroll
    for (int sl = 0; sl < MAXF; sl++) {
        const R dx = d[2 * sl], dy = d[2 * sl + 1];
#pragma unroll
        for (int j = 0; j < V; j++) {
            const R dv = v[1 + sl][j] - v[0][j];
            bx[j] += dx * dv;
            by[j] += dy * dv;
        }
    }
#pragma unroll
    for (int j = 0; j < V; j++) {
        const R sx = ai[0] * bx[j] + ai[1] * by[j], sy = ai[1] * bx[j] + ai[2] * by[j];
        out[j] = v[0][j] + (rx - xx[j] * dt) * sx + (ry - xy[j] * dt) * sy;
    }
}

// FP32, four velocities: the same operations two velocities at a time by paired FP32
// instructions (FFMA2/FMUL2, each lane rounded as the scalar operation; differences as
// FFMA2 with -1).
template <>
__device__ __forceinline__ void reconstruct_vals<float, 4>(const float v[1 + MAXF][4], const float *d, const float *ai,
                                                           float rx, float ry, const float *xx, const float *xy,
                                                           float dt, float out[4])
{
    const float2 v01 = make_float2(v[0][0], v[0][1]), v23 = make_float2(v[0][2], v[0][3]), m1 = make_float2(-1.0f, -1.0f);
    float2 bx01 = make_float2(0.f, 0.f), bx23 = bx01, by01 = bx01, by23 = bx01;
#pragma unroll
    for (int sl = 0; sl < MAXF; sl++) {
        const float2 dx = make_float2(d[2 * sl], d[2 * sl]), dy = make_float2(d[2 * sl + 1], d[2 * sl + 1]);
        const float2 dv01 = __ffma2_rn(v01, m1, make_float2(v[1 + sl][0], v[1 + sl][1]));
        const float2 dv23 = __ffma2_rn(v23, m1, make_float2(v[1 + sl][2], v[1 + sl][3]));
        bx01 = __ffma2_rn(dx, dv01, bx01); bx23 = __ffma2_rn(dx, dv23, bx23);
        by01 = __ffma2_rn(dy, dv01, by01); by23 = __ffma2_rn(dy, dv23, by23);
    }
    const float2 a0 = make_float2(ai[0], ai[0]), a1 = make_float2(ai[1], ai[1]), a2 = make_float2(ai[2], ai[2]);
    const float2 mdt = make_float2(-dt, -dt), rx2 = make_float2(rx, rx), ry2 = make_float2(ry, ry);
    const float2 sx01 = __ffma2_rn(a1, by01, __fmul2_rn(a0, bx01)), sx23 = __ffma2_rn(a1, by23, __fmul2_rn(a0, bx23));
    const float2 sy01 = __ffma2_rn(a2, by01, __fmul2_rn(a1, bx01)), sy23 = __ffma2_rn(a2, by23, __fmul2_rn(a1, bx23));
    const float2 ex01 = __ffma2_rn(make_float2(xx[0], xx[1]), mdt, rx2), ex23 = __ffma2_rn(make_float2(xx[2], xx[3]), mdt, rx2);
    const float2 ey01 = __ffma2_rn(make_float2(xy[0], xy[1]), mdt, ry2), ey23 = __ffma2_rn(make_float2(xy[2], xy[3]), mdt, ry2);
    const float2 o01 = __ffma2_rn(ey01, sy01, __ffma2_rn(ex01, sx01, v01));
    const float2 o23 = __ffma2_rn(ey23, sy23, __ffma2_rn(ex23, sx23, v23));
    out[0] = o01.x; out[1] = o01.y; out[2] = o23.x; out[3] = o23.y;
}

template <class R, int V>
__device__ __forceinline__ void reconstruct_v(const R *const *rows, const R *d, const R *ai, int q, R rx, R ry,
                                              const R *xx, const R *xy, R dt, R out[V])
{
    R v[1 + MAXF][V];
    load_rows<R, V>(rows, q, v);
    reconstruct_vals<R, V>(v, d, ai, rx, ry, xx, xy, dt, out);
}

template <class R, int V>
__global__ void __launch_bounds__(FBP_THREADS) k_dvm_fbp(const DvmMesh m, const Coefs cf, const R *__restrict__ f,
                                                         const double *__restrict__ W, R *__restrict__ fbp)
{
    __shared__ __align__(16) R vt[MAX_NV];
    __shared__ R sp[4];
    load_nodes<R>(vt, m);
    step_dependency_wait();
    const int64_t c = blockIdx.x;
    const int Q = (int)m.Q;
    if (threadIdx.x == 0) state_sp<R>(sp, W[4 * c], W[4 * c + 1], W[4 * c + 2], W[4 * c + 3]);
    __syncthreads();
    const DvmR<R> k(cf);
    const R w = R(m.w_node);
    const R *fr = f + c * m.Q;
    R *out = fbp + c * m.Q;
    VelWalk vw(threadIdx.x * V, FBP_THREADS * V, m.nv);
#pragma unroll 2
    for (int g = threadIdx.x; g < Q / V; g += FBP_THREADS, vw.next()) {
        const int q = g * V;
        R x[V], y[V], fv[V], o[V];
        VNodes<R, V>::get(vt, vw, x, y);
        VIO<R, V>::ld(fr + q, fv);
#pragma unroll
        for (int j = 0; j < V; j++) o[j] = k.a * fv[j] + k.b * maxwell<R>(sp, x[j], y[j], w);
        VIO<R, V>::st(out + q, o);
    }
}

// The rows and LLSR data of one side of a face, in shared memory.
template <class R> struct SideData {
    const R *rows[1 + MAXF];
    R d[2 * MAXF], ai[3];
};

template <class R>
__device__ __forceinline__ void load_side(SideData<R> &sd, const DvmMesh &m, const R *fbp, int64_t cc, int sl)
{
    // called by threads sl = 0..MAXF-1 (neighbours) and sl = MAXF (the cell itself)
    if (sl < MAXF) {
        const int32_t nb = m.cell_nb[cc * MAXF + sl];
        sd.rows[1 + sl] = fbp + (nb >= 0 ? (int64_t)nb : cc) * m.Q;
        const R *d = static_cast<const R *>(m.cell_d) + (cc * MAXF + sl) * 2;
        sd.d[2 * sl] = nb >= 0 ? d[0] : R(0);
        sd.d[2 * sl + 1] = nb >= 0 ? d[1] : R(0);
        if (sl < 3) sd.ai[sl] = static_cast<const R *>(m.ainv)[cc * 3 + sl];
    } else {
        sd.rows[0] = fbp + cc * m.Q;
    }
}

// SMEM: the interface distribution of the face between the two passes over the
// velocities stays in shared memory (Q values); otherwise in the flux array itself.
template <class R, bool SMEM, int V>
__global__ void __launch_bounds__(FACE_THREADS, sizeof(R) == 4 ? 4 : 2) k_dvm_face(const DvmMesh m, const Coefs cf, double RTw,
                                                          const R *__restrict__ fbp, R *__restrict__ flux)
{
    extern __shared__ __align__(16) unsigned char dyn[];
    __shared__ __align__(16) R vt[MAX_NV];
    __shared__ double red[32 * 4];
    __shared__ R sp[4];
    __shared__ SideData<R> sd[2];
    load_nodes<R>(vt, m);
    step_dependency_wait();
    const int64_t fc = blockIdx.x;
    const int Q = (int)m.Q;
    const DvmR<R> k(cf);
    const R w = R(m.w_node);
    const R *G = static_cast<const R *>(m.face_geo) + 6 * fc;
    const R nx = G[0], ny = G[1], rox = G[2], roy = G[3], rkx = G[4], rky = G[5];
    const int64_t o = m.face_own[fc];
    const int32_t kn = m.face_nbr[fc];
    const bool interior = kn >= 0;
    if (threadIdx.x < 2 * (MAXF + 1)) {
        const int side = threadIdx.x / (MAXF + 1), sl = threadIdx.x % (MAXF + 1);
        load_side<R>(sd[side], m, fbp, side == 0 ? o : (interior ? (int64_t)kn : o), sl);
    }
    __syncthreads();
    R *out = flux + fc * m.Q;
    R *fbuf = SMEM ? reinterpret_cast<R *>(dyn) : out;

    if (interior) {
        R p0 = R(0), p1 = R(0), p2 = R(0), p3 = R(0);
        VelWalk vw(threadIdx.x * V, FACE_THREADS * V, m.nv);
        for (int gi = threadIdx.x; gi < Q / V; gi += FACE_THREADS, vw.next()) {
            const int q = gi * V;
            R x[V], y[V], s[V], fa[V], fo[V], fb[V];
            VNodes<R, V>::get(vt, vw, x, y);
            bool needA = false, needB = false;        // some velocity takes the owner's / the neighbour's side
#pragma unroll
            for (int j = 0; j < V; j++) {
                s[j] = x[j] * nx + y[j] * ny;
                needA |= !(s[j] < -k.tie);
                needB |= !(s[j] > k.tie);
                fa[j] = R(0); fo[j] = R(0);
            }
            // both sides' loads before either side's arithmetic: a warp whose lanes need
            // different sides waits for memory once
            R va[1 + MAXF][V], vb[1 + MAXF][V];
            if (needA) load_rows<R, V>(sd[0].rows, q, va);
            if (needB) load_rows<R, V>(sd[1].rows, q, vb);
            if (needA) reconstruct_vals<R, V>(va, sd[0].d, sd[0].ai, rox, roy, x, y, k.dt, fa);
            if (needB) reconstruct_vals<R, V>(vb, sd[1].d, sd[1].ai, rkx, rky, x, y, k.dt, fo);
#pragma unroll
            for (int j = 0; j < V; j++) {
                fb[j] = s[j] > k.tie ? fa[j] : (s[j] < -k.tie ? fo[j] : R(0.5) * (fa[j] + fo[j]));
                p0 += fb[j]; p1 += x[j] * fb[j]; p2 += y[j] * fb[j]; p3 += R(0.5) * (x[j] * x[j] + y[j] * y[j]) * fb[j];
            }
            VIO<R, V>::st(fbuf + q, fb);
        }
        R part[4] = {p0, p1, p2, p3};
        double Wb[4];
        block_sum<4, R>(part, red, Wb);
        if (threadIdx.x == 0) state_sp<R>(sp, Wb[0], Wb[1], Wb[2], Wb[3]);
        __syncthreads();
        VelWalk vw2(threadIdx.x * V, FACE_THREADS * V, m.nv);
        for (int gi = threadIdx.x; gi < Q / V; gi += FACE_THREADS, vw2.next()) {
            const int q = gi * V;
            R x[V], y[V], fb[V], o[V];
            VNodes<R, V>::get(vt, vw2, x, y);
            VIO<R, V>::ld(fbuf + q, fb);
#pragma unroll
            for (int j = 0; j < V; j++) {
                const R s = x[j] * nx + y[j] * ny;
                const R g = maxwell<R>(sp, x[j], y[j], w);
                o[j] = s * ((fb[j] + k.b * g) * k.c);
            }
            VIO<R, V>::st(out + q, o);
        }
    } else {
        // diffuse wall (Sec. III): entering velocities take rho_w g(u_w, R T_w), leaving
        // ones the reconstruction with the wall Maxwellian; rho_w so that no mass passes
        const int p = -1 - kn;
        const int bk = cf.bc_kind[p];
        const double uwx = bk == BK_MOVING_WALL ? cf.bc_par[p][0] : 0.0;
        const double uwy = bk == BK_MOVING_WALL ? cf.bc_par[p][1] : 0.0;
        if (threadIdx.x == 0) {
            MaxP pw;
            pw.pre = 1.0 / (2.0 * 3.14159265358979323846 * RTw); pw.ux = uwx; pw.uy = uwy; pw.inv2RT = 1.0 / (2.0 * RTw);
            set_sp<R>(sp, pw);
        }
        __syncthreads();
        R so = R(0), go = R(0), gin = R(0);
        VelWalk vw(threadIdx.x * V, FACE_THREADS * V, m.nv);
        for (int gi = threadIdx.x; gi < Q / V; gi += FACE_THREADS, vw.next()) {
            const int q = gi * V;
            R x[V], y[V], s[V], fb[V];
            VNodes<R, V>::get(vt, vw, x, y);
            bool leaving = false;                     // some velocity leaves the fluid through the wall
#pragma unroll
            for (int j = 0; j < V; j++) {
                s[j] = x[j] * nx + y[j] * ny;
                leaving |= !(s[j] < -k.tie);
                fb[j] = R(0);
            }
            if (leaving) reconstruct_v<R, V>(sd[0].rows, sd[0].d, sd[0].ai, q, rox, roy, x, y, k.dt, fb);
#pragma unroll
            for (int j = 0; j < V; j++) {
                const R g = maxwell<R>(sp, x[j], y[j], w);
                if (s[j] < -k.tie) {
                    gin += s[j] * g;
                } else {
                    so += s[j] * fb[j];
                    go += s[j] * g;
                }
            }
            if (leaving) VIO<R, V>::st(fbuf + q, fb);
        }
        R part[3] = {so, go, gin};
        double tot[3];
        block_sum<3, R>(part, red, tot);
        // every thread forms rho_w: in FP32 compute by an FP32 division (FP64 divisions
        // are slow on this GPU), from the FP64 sums rounded to FP32
        R rw;
        if constexpr (sizeof(R) == 8) rw = -k.c * tot[0] / (k.c * k.b * tot[1] + tot[2]);
        else rw = -k.c * float(tot[0]) / (k.c * k.b * float(tot[1]) + float(tot[2]));
        VelWalk vw2(threadIdx.x * V, FACE_THREADS * V, m.nv);
        for (int gi = threadIdx.x; gi < Q / V; gi += FACE_THREADS, vw2.next()) {
            const int q = gi * V;
            R x[V], y[V], fb[V], o[V];
            VNodes<R, V>::get(vt, vw2, x, y);
            VIO<R, V>::ld(fbuf + q, fb);
#pragma unroll
            for (int j = 0; j < V; j++) {
                const R s = x[j] * nx + y[j] * ny;
                const R g = maxwell<R>(sp, x[j], y[j], w);
                o[j] = s < -k.tie ? s * (rw * g) : s * ((fb[j] + k.b * (rw * g)) * k.c);
            }
            VIO<R, V>::st(out + q, o);
        }
    }
}

// Ask L2 for a row at once (a hint; the row's start and length are multiples of 16
// bytes).  Later iterations of the walk over the row then find it in L2.  At most the
// first 64 KB of a row, so that the rows of large velocity grids do not flood L2.
__device__ __forceinline__ void prefetch_row_l2(const void *p, uint32_t bytes)
{
    const uint32_t n = bytes < 65536u ? bytes : 65536u;
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(n) : "memory");
}

// SMEM: the cell's flux sum F (Q values) is kept in shared memory between the two
// passes; otherwise it is summed again from the face fluxes.  Cells are taken in
// reverse order: the face kernel writes the fluxes in cell order, so the fluxes read
// first were written last and are still in L2.
template <class R, bool SMEM, int V>
__global__ void __launch_bounds__(CELL_THREADS) k_dvm_cell(const DvmMesh m, const Coefs cf, R *__restrict__ f,
                                                          double *__restrict__ W, const R *__restrict__ flux,
                                                          R *__restrict__ fbp_next)
{
    extern __shared__ __align__(16) unsigned char dyn[];
    R *Fbuf = reinterpret_cast<R *>(dyn);
    __shared__ __align__(16) R vt[MAX_NV];
    __shared__ double red[32 * 4];
    __shared__ R sp[4];
    __shared__ const R *frow[MAXF];
    __shared__ R fsg[MAXF];
    load_nodes<R>(vt, m);
    step_dependency_wait();
    const int64_t c = m.nc - 1 - (int64_t)blockIdx.x;
    const int Q = (int)m.Q;
    const DvmR<R> k(cf);
    const R w = R(m.w_node);
    if (threadIdx.x < MAXF) {
        // the cell's faces in slot order: flux row and sign (a missing slot adds 0 x row 0)
        const int32_t v = m.cell_face[c * MAXF + threadIdx.x];
        const int32_t v0 = m.cell_face[c * MAXF];
        const int32_t id = v >= 0 ? (v & (DVM_SECOND - 1)) : (v0 & (DVM_SECOND - 1));
        frow[threadIdx.x] = flux + (int64_t)id * m.Q;
        fsg[threadIdx.x] = v < 0 ? R(0) : ((v & DVM_SECOND) ? R(-1) : R(1));
        if (V == 4 && v >= 0) prefetch_row_l2(flux + (int64_t)id * m.Q, (uint32_t)(m.Q * sizeof(R)));
    }
    __syncthreads();
    auto F_of = [&](int q, R F[V]) {
#pragma unroll
        for (int j = 0; j < V; j++) F[j] = R(0);
#pragma unroll
        for (int sl = 0; sl < MAXF; sl++) {
            R r[V];
            VIO<R, V>::ld(frow[sl] + q, r);
#pragma unroll
            for (int j = 0; j < V; j++) F[j] += fsg[sl] * r[j];
        }
    };
    R p0 = R(0), p1 = R(0), p2 = R(0), p3 = R(0);
    VelWalk vw(threadIdx.x * V, CELL_THREADS * V, m.nv);
#pragma unroll 2
    for (int gi = threadIdx.x; gi < Q / V; gi += CELL_THREADS, vw.next()) {
        const int q = gi * V;
        R x[V], y[V], F[V];
        VNodes<R, V>::get(vt, vw, x, y);
        F_of(q, F);
        if (SMEM) VIO<R, V>::st(Fbuf + q, F);
#pragma unroll
        for (int j = 0; j < V; j++) {
            p0 += F[j]; p1 += x[j] * F[j]; p2 += y[j] * F[j]; p3 += R(0.5) * (x[j] * x[j] + y[j] * y[j]) * F[j];
        }
    }
    if (V == 4 && threadIdx.x == 32) prefetch_row_l2(f + c * m.Q, (uint32_t)(m.Q * sizeof(R)));
    R part[4] = {p0, p1, p2, p3};
    double M[4];
    block_sum<4, R>(part, red, M);
    const double dtv = m.dtV[c];
    if (threadIdx.x == 0) {
        double Wn[4];
        for (int d = 0; d < 4; d++) {
            Wn[d] = W[4 * c + d] - dtv * M[d];
            W[4 * c + d] = Wn[d];
        }
        state_sp<R>(sp, Wn[0], Wn[1], Wn[2], Wn[3]);
    }
    __syncthreads();
    const R rdtv = R(dtv);
    R *fr = f + c * m.Q;
    VelWalk vw2(threadIdx.x * V, CELL_THREADS * V, m.nv);
#pragma unroll 2
    for (int gi = threadIdx.x; gi < Q / V; gi += CELL_THREADS, vw2.next()) {
        const int q = gi * V;
        R x[V], y[V], F[V], fv[V];
        VNodes<R, V>::get(vt, vw2, x, y);
        VIO<R, V>::ld(fr + q, fv);
        if (SMEM) VIO<R, V>::ld(Fbuf + q, F);
        else F_of(q, F);
        R nb[V];
#pragma unroll
        for (int j = 0; j < V; j++) {
            const R fe = maxwell<R>(sp, x[j], y[j], w);
            const R num = fv[j] - rdtv * F[j] + k.r * fe;
            fv[j] = sizeof(R) == 8 ? num / (R(1) + k.r) : num * k.inv1r;
            nb[j] = k.a * fv[j] + k.b * fe;       // the next step's fbar+ (Eq. fbarplus), as k_dvm_fbp forms it
        }
        VIO<R, V>::st(fr + q, fv);
        if (fbp_next) VIO<R, V>::st(fbp_next + c * m.Q + q, nb);
    }
}

// f = feq(W) per cell (the initial state)
template <class R>
__global__ void __launch_bounds__(DVM_THREADS) k_dvm_init(const DvmMesh m, const double *__restrict__ W,
                                                          R *__restrict__ f)
{
    __shared__ __align__(16) R vt[MAX_NV];
    __shared__ R sp[4];
    load_nodes<R>(vt, m);
    const int64_t c = blockIdx.x, Q = m.Q;
    if (threadIdx.x == 0) set_sp<R>(sp, max_params(W[4 * c], W[4 * c + 1], W[4 * c + 2], W[4 * c + 3]));
    __syncthreads();
    const R w = R(m.w_node);
    VelWalk vw(threadIdx.x, blockDim.x, m.nv);
    for (int64_t q = threadIdx.x; q < Q; q += blockDim.x, vw.next()) {
        R x[1], y[1];
        VNodes<R, 1>::get(vt, vw, x, y);
        f[c * Q + q] = maxwell<R>(sp, x[0], y[0], w);
    }
}

// Largest per-velocity buffer kept in shared memory (bytes).
constexpr size_t DVM_SMEM_MAX = 160 * 1024;

template <class R> bool dvm_use_smem(int64_t Q) { return (size_t)Q * sizeof(R) <= DVM_SMEM_MAX; }

template <class R, int V>
cudaError_t prepare_pv(int64_t Q)
{
    if (!dvm_use_smem<R>(Q)) return cudaSuccess;
    const int bytes = (int)((size_t)Q * sizeof(R));
    cudaError_t e = cudaFuncSetAttribute(k_dvm_face<R, true, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_dvm_cell<R, true, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_dvm_face<R, true, V>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_dvm_cell<R, true, V>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
    return e;
}

template <class R> cudaError_t prepare_p(int64_t Q, int nv)
{
    return nv % 4 == 0 ? prepare_pv<R, 4>(Q) : prepare_pv<R, 1>(Q);
}

template <class R, int V>
cudaError_t step_pv(const DvmMesh &m, const Coefs &c, double RTw, void *f, double *W, void *fbp, void *flux,
                    bool fbp_ready, cudaStream_t st)
{
    const dim3 cells((unsigned)m.nc), faces((unsigned)m.nf);
    const R *cf = static_cast<const R *>(f);
    R *pf = static_cast<R *>(f), *pfbp = static_cast<R *>(fbp), *pflux = static_cast<R *>(flux);
    const R *cfbp = pfbp, *cflux = pflux;
    cudaError_t e = cudaSuccess;
    if (!fbp_ready)
        e = launch_step_kernel(k_dvm_fbp<R, V>, cells, dim3(FBP_THREADS), 0, st, m, c, cf, (const double *)W, pfbp);
    if (e != cudaSuccess) return e;
    // the cell kernel leaves the next step's fbar+ in fbp (read by this step's face kernel
    // before the cell kernel starts)
    if (dvm_use_smem<R>(m.Q)) {
        const size_t bytes = (size_t)m.Q * sizeof(R);
        e = launch_step_kernel(k_dvm_face<R, true, V>, faces, dim3(FACE_THREADS), bytes, st, m, c, RTw, cfbp, pflux);
        if (e == cudaSuccess)
            e = launch_step_kernel(k_dvm_cell<R, true, V>, cells, dim3(CELL_THREADS), bytes, st, m, c, pf, W, cflux, pfbp);
    } else {
        e = launch_step_kernel(k_dvm_face<R, false, V>, faces, dim3(FACE_THREADS), 0, st, m, c, RTw, cfbp, pflux);
        if (e == cudaSuccess)
            e = launch_step_kernel(k_dvm_cell<R, false, V>, cells, dim3(CELL_THREADS), 0, st, m, c, pf, W, cflux, pfbp);
    }
    return e;
}

template <class R>
cudaError_t step_p(const DvmMesh &m, const Coefs &c, double RTw, void *f, double *W, void *fbp, void *flux,
                   bool fbp_ready, cudaStream_t st)
{
    if (m.nc <= 0) return cudaSuccess;
    return m.nv % 4 == 0 ? step_pv<R, 4>(m, c, RTw, f, W, fbp, flux, fbp_ready, st)
                         : step_pv<R, 1>(m, c, RTw, f, W, fbp, flux, fbp_ready, st);
}

}  // namespace

cudaError_t launch_dvm_step(int prec, const DvmMesh &m, const Coefs &c, double RTw, void *f, double *W, void *fbp,
                            void *flux, bool fbp_ready, cudaStream_t st)
{
    return prec == P_FP64 ? step_p<double>(m, c, RTw, f, W, fbp, flux, fbp_ready, st)
                          : step_p<float>(m, c, RTw, f, W, fbp, flux, fbp_ready, st);
}

cudaError_t prepare_dvm(int prec, int64_t Q, int nv)
{
    return prec == P_FP64 ? prepare_p<double>(Q, nv) : prepare_p<float>(Q, nv);
}

cudaError_t launch_dvm_init(int prec, const DvmMesh &m, const double *W, void *f, cudaStream_t st)
{
    if (m.nc <= 0) return cudaSuccess;
    if (prec == P_FP64) k_dvm_init<double><<<(unsigned)m.nc, DVM_THREADS, 0, st>>>(m, W, static_cast<double *>(f));
    else k_dvm_init<float><<<(unsigned)m.nc, DVM_THREADS, 0, st>>>(m, W, static_cast<float *>(f));
    return cudaGetLastError();
}

}  // namespace sdugks
