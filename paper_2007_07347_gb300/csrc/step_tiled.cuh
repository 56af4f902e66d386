// step_tiled.cuh -- fused S-DUGKS step on an unstructured quad mesh.
//
// One CTA per tile of up to TILE_MAX cells.  The tile stages in shared memory the
// transformed distribution fbar+ of its cells and of two halo rings (Eq. fbarplus),
// then the LLSR gradient of its cells and of the first ring.  Each face that touches
// a cell of the tile is then evaluated once, by one thread: the interface
// distribution is reconstructed along the characteristic from the upwind side (Eqs.
// fbpsource, fbar), its moments give the interface equilibrium (Macro at the face,
// Feq), and the interface f (Eq. f_t_n+1) times xi . n l is the face's mesoscopic
// flux, oriented from its first side to its second, kept in shared memory.  Each cell
// thread sums the fluxes of its faces in ascending face id with the sign of its side
// (Eq. MesoFlux); their moments, the macroscopic flux (Eq. MacroFlux), update the FP64
// conserved variables W^{n+1} = W^n - dt/V F_macro (Eq. MacroUpdate, the moment of
// Eq. Integration), whose equilibrium closes the implicit cell update of f (Eq.
// fn+1).  f and W ping-pong between two buffers each; nothing else is stored between
// steps.
//
// A face on the border of two tiles is evaluated by both, with the same operands in
// the same order, so both get the same flux; within a tile the two cells of a face
// add and subtract the same value, and the face fluxes cancel exactly in the sum over
// the cells.
#pragma once
#include "d2q9.cuh"

namespace sdugks {

// shared region of the face fluxes, which first holds the tile's gradient data
constexpr int TILED_FLUX_REGION = NQ * LF_MAX > (2 * MAXF + 3) * SIG_MAX ? NQ * LF_MAX : (2 * MAXF + 3) * SIG_MAX;
static_assert(SIG_MAX % 4 == 0 && (NQ * LOC_MAX + 2 * NQ * SIG_MAX) % 4 == 0, "16-byte aligned gradient planes");

template <class R> struct CoefR;
template <> struct CoefR<double> {
    double a, b, c, r, dt, tie;
    __device__ CoefR(const Coefs &k) : a(k.a_plus), b(k.b_plus), c(k.c_face), r(k.r), dt(k.dt), tie(k.tie) {}
    __device__ static double par(const Coefs &k, int p, int i) { return k.bc_par[p][i]; }
    __device__ static double drho_par(const Coefs &k, int p) { return k.bc_par[p][0] - 1.0; }
};
template <> struct CoefR<float> {
    float a, b, c, r, dt, tie;
    __device__ CoefR(const Coefs &k) : a(k.fa_plus), b(k.fb_plus), c(k.fc_face), r(k.fr), dt(k.fdt), tie(k.ftie) {}
    __device__ static float par(const Coefs &k, int p, int i) { return k.fbc_par[p][i]; }
    __device__ static float drho_par(const Coefs &k, int p) { return k.fbc_drho[p]; }
};

// fbar+ = a f^n + b feq(W^n) of one cell (Eq. fbarplus), with f^n and feq(W^n) returned.
// Asynchronous global -> shared copies (cp.async, 4 or 8 bytes) of read-only data.
template <int B> __device__ __forceinline__ void cp_async(void *smem, const void *gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    if (B == 8) asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(gmem) : "memory");
    else asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
// all committed groups but the most recent one
__device__ __forceinline__ void cp_async_wait_prior() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// FP32 compute: one FFMA2/FMUL2/FADD2 instruction does two independent FP32 operations
// (each lane rounded as the scalar operation), so the per-velocity arithmetic of the
// phases below runs two velocities at a time, paired (1,2) (3,4) (5,6) (7,8).
__device__ __forceinline__ float2 pr2(float a, float b) { return make_float2(a, b); }

// (sum v, sum xi_x v, sum xi_y v) of nine per-velocity values, paired:
// sum xi_x v = (v1 - v3) + (v5 - v7) - (v6 - v8), sum xi_y v = (v2 - v4) + (v5 - v7) + (v6 - v8)
__device__ __forceinline__ void moments9(const float v[NQ], float &m0, float &m1, float &m2)
{
    const float2 m1x2 = pr2(-1.0f, -1.0f);
    const float2 p1 = pr2(v[1], v[2]), p3 = pr2(v[3], v[4]), p5 = pr2(v[5], v[6]), p7 = pr2(v[7], v[8]);
    const float2 sum = __fadd2_rn(__fadd2_rn(p1, p3), __fadd2_rn(p5, p7));
    const float2 d13 = __ffma2_rn(p3, m1x2, p1), d57 = __ffma2_rn(p7, m1x2, p5);
    m0 = v[0] + (sum.x + sum.y);
    m1 = d13.x + (d57.x - d57.y);
    m2 = d13.y + (d57.x + d57.y);
}

// FP32 reconstruction of velocity a at a face from staged cell U (Eqs. fbpsource, fbar):
// fbar+_U + (r_U - xi_a dt) . sigma_U, with r_U = x_f - x_U = (rx, ry)
template <int a>
__device__ __forceinline__ float rec1(const float *s_fbp, const float *s_sig, int U, float rx, float ry, float dt)
{
    return s_fbp[a * LOC_MAX + U] + (rx - float(EX(a)) * dt) * s_sig[(2 * a) * SIG_MAX + U] +
           (ry - float(EY(a)) * dt) * s_sig[(2 * a + 1) * SIG_MAX + U];
}

// The interface values of the velocity pair (a, a+1) at an interior face from the
// upwind side of each (side B when the velocity leaves B, else side A); a tangential
// velocity takes the mean of both sides.
template <int a>
__device__ __forceinline__ void face_pair(float fbar[NQ], const float *s_fbp, const float *s_sig, int A, int B,
                                          float nx, float ny, float rax, float ray, float rbx, float rby, float dt,
                                          float tie)
{
    constexpr int b = a + 1;
    const float sa = xdot<float>(a, nx, ny), sb = xdot<float>(b, nx, ny);
    const bool ba = sa < -tie, bb = sb < -tie;
    const int Ua = ba ? B : A, Ub = bb ? B : A;
    const float2 cx = __fadd2_rn(pr2(ba ? rbx : rax, bb ? rbx : rax), pr2(-float(EX(a)) * dt, -float(EX(b)) * dt));
    const float2 cy = __fadd2_rn(pr2(ba ? rby : ray, bb ? rby : ray), pr2(-float(EY(a)) * dt, -float(EY(b)) * dt));
    float2 v = __ffma2_rn(cx, pr2(s_sig[(2 * a) * SIG_MAX + Ua], s_sig[(2 * b) * SIG_MAX + Ub]),
                          pr2(s_fbp[a * LOC_MAX + Ua], s_fbp[b * LOC_MAX + Ub]));
    v = __ffma2_rn(cy, pr2(s_sig[(2 * a + 1) * SIG_MAX + Ua], s_sig[(2 * b + 1) * SIG_MAX + Ub]), v);
    fbar[a] = v.x;
    fbar[b] = v.y;
    if (!ba && !(sa > tie)) fbar[a] = 0.5f * (fbar[a] + rec1<a>(s_fbp, s_sig, B, rbx, rby, dt));
    if (!bb && !(sb > tie)) fbar[b] = 0.5f * (fbar[b] + rec1<b>(s_fbp, s_sig, B, rbx, rby, dt));
}

// Diagnostic steps (m.force or m.bface set): the momentum (px, py) leaving the fluid
// through boundary face `q` (index over all local faces) of patch p, added to the
// patch total and written to the face's row.
__device__ __forceinline__ void tiled_face_momentum(const TiledMesh &m, int p, int q, double px, double py)
{
    if (m.force) {
        atomicAdd(&m.force[2 * p], px);
        atomicAdd(&m.force[2 * p + 1], py);
    }
    if (m.bface) {
        const int row = m.lf_bface[q];
        if (row >= 0) {
            m.bface[2 * row] = px;
            m.bface[2 * row + 1] = py;
        }
    }
}

// Interface velocity and equilibrium from the moments (w0, w1, w2) of the interface
// distribution: FP64, w0 = rho_b; FP32 compute (deviation form), w0 = rho_b - 1 and the
// equilibrium is returned as its deviation from w.
template <int P>
__device__ __forceinline__ void interface_feq(typename Store<P>::R w0, typename Store<P>::R w1, typename Store<P>::R w2,
                                              typename Store<P>::R &ux, typename Store<P>::R &uy,
                                              typename Store<P>::R feqb[NQ])
{
    using R = typename Store<P>::R;
    if constexpr (Dev<P>::ON) {
        const R rb = R(1) + w0;
        vel_of<R>(rb, w1, w2, ux, uy);
        feq9fd<R>(w0, rb, ux, uy, feqb);
    } else {
        vel_of<R>(w0, w1, w2, ux, uy);
        feq9f<R>(w0, ux, uy, feqb);
    }
}

// The rest equilibrium's momentum flux c_s^2 n l through a face (component nl of n l),
// which the deviation form leaves out of its face fluxes; 0 in FP64.
template <int P> __device__ __forceinline__ double ref_momentum(typename Store<P>::R nl)
{
    return Dev<P>::ON ? (1.0 / 3.0) * to_f64<typename Store<P>::R>(nl) : 0.0;
}

template <int P>
__device__ __forceinline__ void cell_fbp(const typename Store<P>::T *__restrict__ fin, const double *__restrict__ Wn,
                                         int64_t g, int64_t np, const CoefR<typename Store<P>::R> &k,
                                         typename Store<P>::R fn[NQ], typename Store<P>::R fe[NQ],
                                         typename Store<P>::R fbp[NQ])
{
    using R = typename Store<P>::R;
    R drho, rho, ux, uy;
    macro_of<R>(Wn[g], Wn[np + g], Wn[2 * np + g], drho, rho, ux, uy);
    feq9fd<R>(Dev<P>::ON ? drho : rho, rho, ux, uy, fe);      // FP32 compute: deviation form (g = f - w)
#pragma unroll
    for (int a = 0; a < NQ; a++) fn[a] = Store<P>::dec(fin[a * np + g], fe[a], a);
    if constexpr (P == P_FP64) {
#pragma unroll
        for (int a = 0; a < NQ; a++) fbp[a] = k.a * fn[a] + k.b * fe[a];
    } else {
        const float2 ka = pr2(k.a, k.a), kb = pr2(k.b, k.b);
        fbp[0] = k.a * fn[0] + k.b * fe[0];
#pragma unroll
        for (int a = 1; a < NQ; a += 2) {
            const float2 v = __ffma2_rn(ka, pr2(fn[a], fn[a + 1]), __fmul2_rn(kb, pr2(fe[a], fe[a + 1])));
            fbp[a] = v.x;
            fbp[a + 1] = v.y;
        }
    }
}

// DIAG: the diagnostic step, which also reports the momentum leaving the fluid through
// the boundary faces (m.force, m.bface); ordinary steps carry none of that code.
template <int P, bool DIAG = false>
__global__ void __launch_bounds__(TILED_THREADS, P == P_FP64 ? 1 : 4)
k_step_tiled(const TiledMesh m, const Coefs c, const typename Store<P>::T *__restrict__ fin,
             typename Store<P>::T *__restrict__ fout, const double *__restrict__ Wn, double *__restrict__ Wout)
{
    using R = typename Store<P>::R;
    using SP = Store<P>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R *s_fbp = reinterpret_cast<R *>(smem_raw);     // [NQ][LOC_MAX]
    R *s_sig = s_fbp + NQ * LOC_MAX;                 // [2 NQ][SIG_MAX]
    R *s_flux = s_sig + 2 * NQ * SIG_MAX;            // [NQ][LF_MAX]; before phase 3:
    R *s_sd = s_flux;                                //   [2 MAXF][SIG_MAX] gradient offsets of the rows
    R *s_sa = s_flux + 2 * MAXF * SIG_MAX;           //   [3][SIG_MAX] LLSR inverses
    R *s_geo = s_flux + TILED_FLUX_REGION;           // [6][LF_MAX] face geometry of the tile
    uint32_t *s_lfab = reinterpret_cast<uint32_t *>(s_geo + 6 * LF_MAX);   // [LF_MAX] face sides

    const int t = blockIdx.x, tid = threadIdx.x;
    const int c0 = m.tile_c0[t];
    const int n_int = m.tile_c0[t + 1] - c0;
    const int h0 = m.tile_h0[t];
    const int n_loc = n_int + (m.tile_h0[t + 1] - h0);
    const int n_sig = n_int + m.tile_nh1[t];
    const int s0 = m.tile_s0[t];
    const int f0 = m.tile_f0[t];
    const int n_lf = m.tile_nlf[t];
    const int64_t np = m.npad, nlf = m.n_lf;
    const CoefR<R> k(c);
    // the gradient data of the tile's rows (read-only mesh data, needed in phase 2) travels
    // to shared memory while the previous step finishes: 16-byte pieces of each of the 11
    // planes (tile_s0 and the plane stride are multiples of 4 rows)
    {
        // one 16-byte piece of each plane per thread: a tile has at most SIG_MAX / E
        // pieces per plane, fewer than the threads, so only the first warps copy
        constexpr int E = 16 / (int)sizeof(R);
        static_assert(SIG_MAX / E <= TILED_THREADS, "one piece per thread and plane");
        const int nch = (n_sig + E - 1) / E;
        if (tid < nch) {
            const R *sgd = static_cast<const R *>(m.sig_d) + s0 + tid * E;
            const R *sga = static_cast<const R *>(m.sig_ai) + s0 + tid * E;
#pragma unroll
            for (int pl = 0; pl < 2 * MAXF; pl++) cp_async16(&s_sd[pl * SIG_MAX + tid * E], sgd + pl * m.n_sig);
#pragma unroll
            for (int pl = 0; pl < 3; pl++) cp_async16(&s_sa[pl * SIG_MAX + tid * E], sga + pl * m.n_sig);
        }
        cp_async_commit();
    }
    // then the tile's face list (needed in phase 3), in 16-byte pieces: the tile's range
    // starts at a multiple of 4 faces in every face array (the pieces past its last face
    // read the range's padding)
    {
        constexpr int E = 16 / (int)sizeof(R);
        static_assert(LF_MAX % 4 == 0 && LF_MAX / E <= TILED_THREADS, "one piece per thread and plane");
        if (tid < (n_lf + 3) / 4) cp_async16(&s_lfab[tid * 4], &m.lf_ab[f0 + tid * 4]);
        if (tid < (n_lf + E - 1) / E) {
            const R *gsrc = static_cast<const R *>(m.lf_geo) + f0 + tid * E;
#pragma unroll
            for (int q = 0; q < 6; q++) cp_async16(&s_geo[q * LF_MAX + tid * E], gsrc + q * nlf);
        }
        cp_async_commit();
    }
    // the first gradient row's neighbour list
    uint2 nb0 = make_uint2(0xFFFFFFFFu, 0xFFFFFFFFu);
    if (tid < n_sig) nb0 = *reinterpret_cast<const uint2 *>(m.sig_nb + (int64_t)(s0 + tid) * MAXF);
    // cells this thread stages (read-only halo ids: looked up before the wait as well)
    const int64_t gs0 = tid < n_int ? (int64_t)c0 + tid : (tid < n_loc ? (int64_t)m.halo[h0 + tid - n_int] : 0);
    const int i1 = tid + TILED_THREADS;            // a second staged position (always a halo cell)
    const int64_t gs1 = i1 < n_loc ? (int64_t)m.halo[h0 + i1 - n_int] : 0;
    step_dependency_wait();

    // ---- phase 1: fbar+ of the tile's cells and both halo rings; a thread keeps f^n of
    // its own cell (cell tid) in registers for the update
    const bool active = tid < n_int;
    const int64_t g = c0 + tid;
    R fn[NQ];
    for (int i = tid; i < n_loc; i += TILED_THREADS) {
        const int64_t gi = i == tid ? gs0 : (i == i1 ? gs1 : (int64_t)m.halo[h0 + i - n_int]);
        R fx[NQ], fe[NQ], fb[NQ];
        cell_fbp<P>(fin, Wn, gi, np, k, fx, fe, fb);
#pragma unroll
        for (int a = 0; a < NQ; a++) s_fbp[a * LOC_MAX + i] = fb[a];
        if (i == tid) {
#pragma unroll
            for (int a = 0; a < NQ; a++) fn[a] = fx[a];
        }
    }
    cp_async_wait_prior();      // the gradient data has arrived (the face list may be in flight)
    __syncthreads();

    // ---- phase 2: LLSR gradient sigma = A^{-1} sum_k d_k (fbar+_k - fbar+_j), d = x_k - x_j
    for (int i = tid; i < n_sig; i += TILED_THREADS) {
        const uint2 nbv = i == tid ? nb0 : *reinterpret_cast<const uint2 *>(m.sig_nb + (int64_t)(s0 + i) * MAXF);
        const uint16_t nb[MAXF] = {(uint16_t)(nbv.x & 0xFFFFu), (uint16_t)(nbv.x >> 16), (uint16_t)(nbv.y & 0xFFFFu),
                                   (uint16_t)(nbv.y >> 16)};
        if constexpr (P == P_FP64) {
            R bx[NQ], by[NQ];
#pragma unroll
            for (int a = 0; a < NQ; a++) { bx[a] = R(0); by[a] = R(0); }
#pragma unroll
            for (int sl = 0; sl < MAXF; sl++) {
                const int kk = nb[sl];
                if (kk == NO_LOCAL) continue;
                const R dx = s_sd[(2 * sl) * SIG_MAX + i], dy = s_sd[(2 * sl + 1) * SIG_MAX + i];
                if (kk < SYM_X) {
#pragma unroll
                    for (int a = 0; a < NQ; a++) {
                        const R d = s_fbp[a * LOC_MAX + kk] - s_fbp[a * LOC_MAX + i];
                        bx[a] += dx * d;
                        by[a] += dy * d;
                    }
                } else {
                    // symmetry ghost: the cell's own fbar+ of the mirrored velocity (Sec. III)
                    const bool mx = kk == SYM_X;
#pragma unroll
                    for (int a = 0; a < NQ; a++) {
                        const R d = s_fbp[(mx ? MIRROR_X(a) : MIRROR_Y(a)) * LOC_MAX + i] - s_fbp[a * LOC_MAX + i];
                        bx[a] += dx * d;
                        by[a] += dy * d;
                    }
                }
            }
            const R axx = s_sa[i], axy = s_sa[SIG_MAX + i], ayy = s_sa[2 * SIG_MAX + i];
#pragma unroll
            for (int a = 0; a < NQ; a++) {
                s_sig[(2 * a) * SIG_MAX + i] = axx * bx[a] + axy * by[a];
                s_sig[(2 * a + 1) * SIG_MAX + i] = axy * bx[a] + ayy * by[a];
            }
        } else {
            // the same sums, paired; the differences f_k - f_j as FFMA2 with -1
            float fi[NQ];
#pragma unroll
            for (int a = 0; a < NQ; a++) fi[a] = s_fbp[a * LOC_MAX + i];
            const float2 m1 = pr2(-1.0f, -1.0f);
            float bx0 = 0.0f, by0 = 0.0f;
            float2 bx[4], by[4];
#pragma unroll
            for (int q = 0; q < 4; q++) { bx[q] = pr2(0.0f, 0.0f); by[q] = pr2(0.0f, 0.0f); }
#pragma unroll
            for (int sl = 0; sl < MAXF; sl++) {
                const int kk = nb[sl];
                if (kk == NO_LOCAL) continue;
                const float dx = s_sd[(2 * sl) * SIG_MAX + i], dy = s_sd[(2 * sl + 1) * SIG_MAX + i];
                float fk[NQ];
                if (kk < SYM_X) {
#pragma unroll
                    for (int a = 0; a < NQ; a++) fk[a] = s_fbp[a * LOC_MAX + kk];
                } else {
                    // symmetry ghost: the cell's own fbar+ of the mirrored velocity (Sec. III)
                    const bool mx = kk == SYM_X;
#pragma unroll
                    for (int a = 0; a < NQ; a++) fk[a] = fi[mx ? MIRROR_X(a) : MIRROR_Y(a)];
                }
                const float d0 = fk[0] - fi[0];
                bx0 += dx * d0;
                by0 += dy * d0;
                const float2 dx2 = pr2(dx, dx), dy2 = pr2(dy, dy);
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    const int a = 1 + 2 * q;
                    const float2 d = __ffma2_rn(pr2(fi[a], fi[a + 1]), m1, pr2(fk[a], fk[a + 1]));
                    bx[q] = __ffma2_rn(dx2, d, bx[q]);
                    by[q] = __ffma2_rn(dy2, d, by[q]);
                }
            }
            const float axx = s_sa[i], axy = s_sa[SIG_MAX + i], ayy = s_sa[2 * SIG_MAX + i];
            s_sig[i] = axx * bx0 + axy * by0;
            s_sig[SIG_MAX + i] = axy * bx0 + ayy * by0;
            const float2 xx = pr2(axx, axx), xy = pr2(axy, axy), yy = pr2(ayy, ayy);
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const int a = 1 + 2 * q;
                const float2 sx = __ffma2_rn(xx, bx[q], __fmul2_rn(xy, by[q]));
                const float2 sy = __ffma2_rn(xy, bx[q], __fmul2_rn(yy, by[q]));
                s_sig[(2 * a) * SIG_MAX + i] = sx.x;
                s_sig[(2 * a + 1) * SIG_MAX + i] = sy.x;
                s_sig[(2 * a + 2) * SIG_MAX + i] = sx.y;
                s_sig[(2 * a + 3) * SIG_MAX + i] = sy.y;
            }
        }
    }
    cp_async_wait_all();        // the face list has arrived
    __syncthreads();
    // inputs of the cell update, loaded now so that they arrive during the face phase
    uint16_t my_lf[MAXF] = {LF_NONE, LF_NONE, LF_NONE, LF_NONE};
    R dtv = R(0);
    double w0n = 0.0, w1n = 0.0, w2n = 0.0;
    if (active) {
#pragma unroll
        for (int sl = 0; sl < MAXF; sl++) my_lf[sl] = m.cell_lf[sl * np + g];
        dtv = static_cast<const R *>(m.dtV)[g];
        w0n = Wn[g]; w1n = Wn[np + g]; w2n = Wn[2 * np + g];
    }

    // ---- phase 3: every local face once; flux s f_b from the first side to the second
    for (int lf = tid; lf < n_lf; lf += TILED_THREADS) {
        const uint32_t ab = s_lfab[lf];
        const int A = (int)(ab & 0xFFFFu), B = (int)(ab >> 16);
        const R *G = s_geo + lf;
        const R nx = G[0], ny = G[LF_MAX], rax = G[2 * LF_MAX], ray = G[3 * LF_MAX];
        if (!(B & LF_SECOND)) {
            const R rbx = G[4 * LF_MAX], rby = G[5 * LF_MAX];
            R fbar[NQ], w0 = R(0), w1 = R(0), w2 = R(0);
            if constexpr (P == P_FP64) {
#pragma unroll
                for (int a = 0; a < NQ; a++) {
                    const R s = xdot<R>(a, nx, ny);
                    const R ex = R(EX(a)) * k.dt, ey = R(EY(a)) * k.dt;
                    // the upwind side's reconstruction only (side B when the velocity leaves
                    // it, else side A); a tangential velocity takes the mean of both sides
                    const bool from_b = s < -k.tie;
                    const int U = from_b ? B : A;
                    const R rux = from_b ? rbx : rax, ruy = from_b ? rby : ray;
                    R v = s_fbp[a * LOC_MAX + U] + (rux - ex) * s_sig[(2 * a) * SIG_MAX + U] +
                          (ruy - ey) * s_sig[(2 * a + 1) * SIG_MAX + U];
                    if (!from_b && !(s > k.tie)) {
                        const R FB = s_fbp[a * LOC_MAX + B] + (rbx - ex) * s_sig[(2 * a) * SIG_MAX + B] +
                                     (rby - ey) * s_sig[(2 * a + 1) * SIG_MAX + B];
                        v = R(0.5) * (v + FB);
                    }
                    fbar[a] = v;
                }
            } else {
                // the rest velocity is tangential to every face
                fbar[0] = 0.5f * (rec1<0>(s_fbp, s_sig, A, rax, ray, k.dt) + rec1<0>(s_fbp, s_sig, B, rbx, rby, k.dt));
                face_pair<1>(fbar, s_fbp, s_sig, A, B, nx, ny, rax, ray, rbx, rby, k.dt, k.tie);
                face_pair<3>(fbar, s_fbp, s_sig, A, B, nx, ny, rax, ray, rbx, rby, k.dt, k.tie);
                face_pair<5>(fbar, s_fbp, s_sig, A, B, nx, ny, rax, ray, rbx, rby, k.dt, k.tie);
                face_pair<7>(fbar, s_fbp, s_sig, A, B, nx, ny, rax, ray, rbx, rby, k.dt, k.tie);
            }
            if constexpr (P == P_FP64) {
#pragma unroll
                for (int a = 0; a < NQ; a++) {
                    w0 += fbar[a];
                    if (EX(a) == 1) w1 += fbar[a]; else if (EX(a) == -1) w1 -= fbar[a];
                    if (EY(a) == 1) w2 += fbar[a]; else if (EY(a) == -1) w2 -= fbar[a];
                }
            } else {
                moments9(fbar, w0, w1, w2);
            }
            R ux, uy, feqb[NQ];
            interface_feq<P>(w0, w1, w2, ux, uy, feqb);
            if constexpr (P == P_FP64) {
#pragma unroll
                for (int a = 0; a < NQ; a++) {
                    const R s = xdot<R>(a, nx, ny);
                    s_flux[a * LF_MAX + lf] = s * ((fbar[a] + k.b * feqb[a]) * k.c);
                }
            } else {
                const float2 bb = pr2(k.b, k.b), cc = pr2(k.c, k.c);
                s_flux[lf] = 0.0f * ((fbar[0] + k.b * feqb[0]) * k.c);
#pragma unroll
                for (int a = 1; a < NQ; a += 2) {
                    const float2 sv = pr2(xdot<float>(a, nx, ny), xdot<float>(a + 1, nx, ny));
                    const float2 t = __fmul2_rn(__ffma2_rn(bb, pr2(feqb[a], feqb[a + 1]), pr2(fbar[a], fbar[a + 1])), cc);
                    const float2 fl = __fmul2_rn(sv, t);
                    s_flux[a * LF_MAX + lf] = fl.x;
                    s_flux[(a + 1) * LF_MAX + lf] = fl.y;
                }
            }
        } else if (c.bc_kind[B & 0xFF] == BK_SYMMETRY) {
            // symmetry face of cell A: the far side is A's mirror ghost, whose
            // reconstruction of xi is A's own reconstruction of the mirrored velocity
            // (same fbar+, reflected gradient and offset); tangential velocities are
            // their own mirror images.  Then as on an interior face.
            const bool mx = (nx < R(0) ? -nx : nx) > (ny < R(0) ? -ny : ny);
            R rec[NQ];
#pragma unroll
            for (int a = 0; a < NQ; a++)
                rec[a] = s_fbp[a * LOC_MAX + A] + (rax - R(EX(a)) * k.dt) * s_sig[(2 * a) * SIG_MAX + A] +
                         (ray - R(EY(a)) * k.dt) * s_sig[(2 * a + 1) * SIG_MAX + A];
            R fbar[NQ], w0 = R(0), w1 = R(0), w2 = R(0);
#pragma unroll
            for (int a = 0; a < NQ; a++) {
                const R s = xdot<R>(a, nx, ny);
                fbar[a] = s < -k.tie ? (mx ? rec[MIRROR_X(a)] : rec[MIRROR_Y(a)]) : rec[a];
                w0 += fbar[a];
                if (EX(a) == 1) w1 += fbar[a]; else if (EX(a) == -1) w1 -= fbar[a];
                if (EY(a) == 1) w2 += fbar[a]; else if (EY(a) == -1) w2 -= fbar[a];
            }
            R ux, uy, feqb[NQ];
            interface_feq<P>(w0, w1, w2, ux, uy, feqb);
            R px_ = R(0), py_ = R(0);
#pragma unroll
            for (int a = 0; a < NQ; a++) {
                const R s = xdot<R>(a, nx, ny);
                const R fl = s * ((fbar[a] + k.b * feqb[a]) * k.c);
                s_flux[a * LF_MAX + lf] = fl;
                if constexpr (DIAG) {
                    px_ += R(EX(a)) * fl;
                    py_ += R(EY(a)) * fl;
                }
            }
            if constexpr (DIAG)
                tiled_face_momentum(m, B & 0xFF, f0 + lf, to_f64<R>(px_) + ref_momentum<P>(nx),
                                    to_f64<R>(py_) + ref_momentum<P>(ny));
        } else {
            // boundary face of cell A (an interior cell of the tile): Sec. III rules
            const int p = B & 0xFF;
            const int bk = c.bc_kind[p];
            const int64_t gA = (int64_t)c0 + A;
            R fnA[NQ], feqA[NQ], fbA[NQ], drhoA, rhoA, uxA, uyA;
            cell_fbp<P>(fin, Wn, gA, np, k, fnA, feqA, fbA);
            macro_of<R>(Wn[gA], Wn[np + gA], Wn[2 * np + gA], drhoA, rhoA, uxA, uyA);
            R rb = rhoA, drb = drhoA, ubx = R(0), uby = R(0);
            if (bk == BK_MOVING_WALL) { ubx = CoefR<R>::par(c, p, 0); uby = CoefR<R>::par(c, p, 1); }
            else if (bk == BK_FARFIELD) {
                rb = CoefR<R>::par(c, p, 0); drb = CoefR<R>::drho_par(c, p);
                ubx = CoefR<R>::par(c, p, 1); uby = CoefR<R>::par(c, p, 2);
            } else if (bk == BK_OUTLET) { ubx = uxA; uby = uyA; }
            R feqb[NQ];
            feq9fd<R>(Dev<P>::ON ? drb : rb, rb, ubx, uby, feqb);
            R px_ = R(0), py_ = R(0);
#pragma unroll
            for (int a = 0; a < NQ; a++) {
                const R s = xdot<R>(a, nx, ny);
                R fb;
                if (s < -k.tie) {
                    fb = feqb[a] + (fnA[a] - feqA[a]);     // non-equilibrium extrapolation
                } else {
                    const R FA = s_fbp[a * LOC_MAX + A] + (rax - R(EX(a)) * k.dt) * s_sig[(2 * a) * SIG_MAX + A] +
                                 (ray - R(EY(a)) * k.dt) * s_sig[(2 * a + 1) * SIG_MAX + A];
                    fb = (FA + k.b * feqb[a]) * k.c;
                }
                s_flux[a * LF_MAX + lf] = s * fb;
                if constexpr (DIAG) {
                    px_ += R(EX(a)) * (s * fb);
                    py_ += R(EY(a)) * (s * fb);
                }
            }
            if constexpr (DIAG)
                tiled_face_momentum(m, p, f0 + lf, to_f64<R>(px_) + ref_momentum<P>(nx),
                                    to_f64<R>(py_) + ref_momentum<P>(ny));
        }
    }
    __syncthreads();
    if (!active) return;

    // ---- mesoscopic flux of the own cell (Eq. MesoFlux), ascending face id
    R F[NQ];
#pragma unroll
    for (int a = 0; a < NQ; a++) F[a] = R(0);
#pragma unroll
    for (int sl = 0; sl < MAXF; sl++) {
        const unsigned v = my_lf[sl];
        if (v == LF_NONE) continue;
        const int lf = (int)(v & (LF_SECOND - 1u));
        if constexpr (P == P_FP64) {
            if (v & LF_SECOND) {
#pragma unroll
                for (int a = 0; a < NQ; a++) F[a] -= s_flux[a * LF_MAX + lf];
            } else {
#pragma unroll
                for (int a = 0; a < NQ; a++) F[a] += s_flux[a * LF_MAX + lf];
            }
        } else {
            // F +- flux as FFMA2 with +-1 (exactly the sum or difference)
            const float sg = (v & LF_SECOND) ? -1.0f : 1.0f;
            const float2 sg2 = pr2(sg, sg);
            F[0] = F[0] + sg * s_flux[lf];
#pragma unroll
            for (int a = 1; a < NQ; a += 2) {
                const float2 t = __ffma2_rn(pr2(s_flux[a * LF_MAX + lf], s_flux[(a + 1) * LF_MAX + lf]), sg2,
                                            pr2(F[a], F[a + 1]));
                F[a] = t.x;
                F[a + 1] = t.y;
            }
        }
    }

    // ---- macroscopic flux (moments of F) -> W^{n+1} in FP64; cell update f^{n+1} (Eq. fn+1)
    R M0 = R(0), M1 = R(0), M2 = R(0);
    if constexpr (P == P_FP64) {
#pragma unroll
        for (int a = 0; a < NQ; a++) {
            M0 += F[a];
            if (EX(a) == 1) M1 += F[a]; else if (EX(a) == -1) M1 -= F[a];
            if (EY(a) == 1) M2 += F[a]; else if (EY(a) == -1) M2 -= F[a];
        }
    } else {
        moments9(F, M0, M1, M2);
    }
    const R d0 = dtv * M0, d1 = dtv * M1, d2 = dtv * M2;
    const double W0 = w0n - to_f64<R>(d0), W1 = w1n - to_f64<R>(d1), W2 = w2n - to_f64<R>(d2);
    // FP32 compute: the FP64 sums are stored last, after the f update, which does not wait
    // for them (the FP64 unit of this GPU is narrow)
    if constexpr (P == P_FP64) {
        Wout[g] = W0;
        Wout[np + g] = W1;
        Wout[2 * np + g] = W2;
    }
    R rho1, ux1, uy1, feq1[NQ];
    if constexpr (P == P_FP64) {
        R drho1;
        macro_of<R>(W0, W1, W2, drho1, rho1, ux1, uy1);
        feq9f<R>(rho1, ux1, uy1, feq1);
    } else {
        // FP32 compute: W^{n+1} in FP32 from the FP32 copies of W^n (W[0] = rho - 1)
        const R drho1 = from_f64<R>(w0n) - d0;
        rho1 = R(1) + drho1;
        vel_of<R>(rho1, from_f64<R>(w1n) - d1, from_f64<R>(w2n) - d2, ux1, uy1);
        feq9fd<R>(drho1, rho1, ux1, uy1, feq1);
    }
    if constexpr (P == P_FP64) {
#pragma unroll
        for (int a = 0; a < NQ; a++)
            fout[a * np + g] = SP::enc((fn[a] - dtv * F[a] + k.r * feq1[a]) / (R(1) + k.r), feq1[a], a);
    } else {
        // paired: (f - dt/V F + r feq) / (1 + r)
        const float2 mdv = pr2(-dtv, -dtv), r2 = pr2(k.r, k.r), i2 = pr2(c.finv1r, c.finv1r);
        fout[g] = SP::enc((fn[0] - dtv * F[0] + k.r * feq1[0]) * c.finv1r, feq1[0], 0);
#pragma unroll
        for (int a = 1; a < NQ; a += 2) {
            const float2 t = __ffma2_rn(mdv, pr2(F[a], F[a + 1]), pr2(fn[a], fn[a + 1]));
            const float2 u = __fmul2_rn(__ffma2_rn(r2, pr2(feq1[a], feq1[a + 1]), t), i2);
            fout[a * np + g] = SP::enc(u.x, feq1[a], a);
            fout[(a + 1) * np + g] = SP::enc(u.y, feq1[a + 1], a + 1);
        }
        Wout[g] = W0;
        Wout[np + g] = W1;
        Wout[2 * np + g] = W2;
    }
}

template <int P> constexpr size_t tiled_smem() {
    return sizeof(typename Store<P>::R) * (size_t)(NQ * LOC_MAX + 2 * NQ * SIG_MAX + TILED_FLUX_REGION + 6 * LF_MAX) +
           sizeof(uint32_t) * LF_MAX;
}

template <int P, bool DIAG> cudaError_t prepare_tiled_pd() {
    cudaError_t e = cudaFuncSetAttribute(k_step_tiled<P, DIAG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)tiled_smem<P>());
    // all of the unified L1/shared array as shared memory: four FP32 tiles per SM
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_step_tiled<P, DIAG>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
    return e;
}
template <int P> cudaError_t prepare_tiled_p() {
    cudaError_t e = prepare_tiled_pd<P, false>();
    return e == cudaSuccess ? prepare_tiled_pd<P, true>() : e;
}

template <int P>
cudaError_t launch_tiled_p(const TiledMesh &m, const Coefs &c, const void *fin, void *fout, const double *Wn,
                           double *Wout, cudaStream_t st)
{
    using T = typename Store<P>::T;
    if (m.n_tiles <= 0) return cudaSuccess;
    if (m.force || m.bface)     // the diagnostic step
        return launch_step_kernel(k_step_tiled<P, true>, dim3(m.n_tiles), dim3(TILED_THREADS), tiled_smem<P>(), st, m,
                                  c, static_cast<const T *>(fin), static_cast<T *>(fout), Wn, Wout);
    return launch_step_kernel(k_step_tiled<P, false>, dim3(m.n_tiles), dim3(TILED_THREADS), tiled_smem<P>(), st, m, c,
                              static_cast<const T *>(fin), static_cast<T *>(fout), Wn, Wout);
}

}  // namespace sdugks
