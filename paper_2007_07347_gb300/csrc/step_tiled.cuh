// step_tiled.cuh -- fused S-DUGKS step on an unstructured quad mesh.
//
// One CTA per tile of up to TILE_MAX cells (one thread per interior cell).  The tile
// stages in shared memory the transformed distribution fbar+ of its cells and of
// two halo rings (Eq. fbarplus), then the LLSR gradient of its cells and of the
// first ring, then every thread reconstructs the interface distribution on the
// faces of its own cell along the characteristic (Eqs. fbpsource, fbar, Macro at the
// face, Feq, f_t_n+1) and sums the mesoscopic flux (Eq. MesoFlux).  Its moments, the
// macroscopic flux (Eq. MacroFlux), update the FP64 conserved variables
// W^{n+1} = W^n - dt/V F_macro (Eq. MacroUpdate, the moment of Eq. Integration), whose
// equilibrium then closes the implicit cell update of f (Eq. fn+1).  f and W
// ping-pong between two buffers each; nothing else is stored between steps.
//
// Face data is stored per cell and slot (normal, face centre relative to this cell
// and to the far cell), so an interior face is evaluated by the threads of both its
// cells with the same operands in the same order: both get the same interface
// values, and the face fluxes cancel exactly in the sum over the two cells.
#pragma once
#include "d2q9.cuh"

namespace sdugks {

template <class R> struct CoefR;
template <> struct CoefR<double> {
    double a, b, c, r, dt, tie;
    __device__ CoefR(const Coefs &k) : a(k.a_plus), b(k.b_plus), c(k.c_face), r(k.r), dt(k.dt), tie(k.tie) {}
    __device__ static double par(const Coefs &k, int p, int i) { return k.bc_par[p][i]; }
};
template <> struct CoefR<float> {
    float a, b, c, r, dt, tie;
    __device__ CoefR(const Coefs &k) : a(k.fa_plus), b(k.fb_plus), c(k.fc_face), r(k.fr), dt(k.fdt), tie(k.ftie) {}
    __device__ static float par(const Coefs &k, int p, int i) { return k.fbc_par[p][i]; }
};

template <int P>
__global__ void __launch_bounds__(TILE_MAX)
k_step_tiled(const TiledMesh m, const Coefs c, const typename Store<P>::T *__restrict__ fin,
             typename Store<P>::T *__restrict__ fout, const double *__restrict__ Wn, double *__restrict__ Wout)
{
    using R = typename Store<P>::R;
    using SP = Store<P>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R *s_fbp = reinterpret_cast<R *>(smem_raw);     // [NQ][LOC_MAX]
    R *s_sig = s_fbp + NQ * LOC_MAX;                 // [2 NQ][SIG_MAX]

    const int t = blockIdx.x, tid = threadIdx.x;
    const int c0 = m.tile_c0[t];
    const int n_int = m.tile_c0[t + 1] - c0;
    const int h0 = m.tile_h0[t];
    const int n_loc = n_int + (m.tile_h0[t + 1] - h0);
    const int n_sig = n_int + m.tile_nh1[t];
    const int s0 = m.tile_s0[t];
    const int64_t np = m.npad;
    const CoefR<R> k(c);
    const R *geo = static_cast<const R *>(m.sl_geo);
    const R *ainv = static_cast<const R *>(m.ainv);

    // ---- phase 1: fbar+ = a f^n + b feq(W^n) for own cells (kept in registers) and halos
    const bool active = tid < n_int;
    const int64_t g = c0 + tid;
    R fn[NQ], feqn[NQ];
    R rho_n = R(1), ux_n = R(0), uy_n = R(0);
    double w0n = 1.0, w1n = 0.0, w2n = 0.0;
    if (active) {
        w0n = Wn[g]; w1n = Wn[np + g]; w2n = Wn[2 * np + g];
        macro_of<R>(w0n, w1n, w2n, rho_n, ux_n, uy_n);
        feq9f<R>(rho_n, ux_n, uy_n, feqn);
#pragma unroll
        for (int a = 0; a < NQ; a++) {
            fn[a] = SP::dec(fin[a * np + g], feqn[a], a);
            s_fbp[a * LOC_MAX + tid] = k.a * fn[a] + k.b * feqn[a];
        }
    }
    for (int i = n_int + tid; i < n_loc; i += blockDim.x) {
        const int64_t gh = m.halo[h0 + i - n_int];
        R rho, ux, uy, fe[NQ];
        macro_of<R>(Wn[gh], Wn[np + gh], Wn[2 * np + gh], rho, ux, uy);
        feq9f<R>(rho, ux, uy, fe);
#pragma unroll
        for (int a = 0; a < NQ; a++)
            s_fbp[a * LOC_MAX + i] = k.a * SP::dec(fin[a * np + gh], fe[a], a) + k.b * fe[a];
    }
    __syncthreads();

    // ---- phase 2: LLSR gradient sigma = A^{-1} sum_k d_k (fbar+_k - fbar+_j), d = x_k - x_j
    for (int i = tid; i < n_sig; i += blockDim.x) {
        const int64_t gi = i < n_int ? (int64_t)c0 + i : (int64_t)m.halo[h0 + i - n_int];
        const uint16_t *nb = m.sig_nb + (int64_t)(s0 + i) * MAXF;
        R bx[NQ], by[NQ];
#pragma unroll
        for (int a = 0; a < NQ; a++) { bx[a] = R(0); by[a] = R(0); }
#pragma unroll
        for (int sl = 0; sl < MAXF; sl++) {
            const int kk = nb[sl];
            if (kk == NO_LOCAL) continue;
            const R *G = geo + (int64_t)(6 * sl) * np + gi;
            const R dx = G[2 * np] - G[4 * np], dy = G[3 * np] - G[5 * np];
#pragma unroll
            for (int a = 0; a < NQ; a++) {
                const R d = s_fbp[a * LOC_MAX + kk] - s_fbp[a * LOC_MAX + i];
                bx[a] += dx * d;
                by[a] += dy * d;
            }
        }
        const R axx = ainv[gi], axy = ainv[np + gi], ayy = ainv[2 * np + gi];
#pragma unroll
        for (int a = 0; a < NQ; a++) {
            s_sig[(2 * a) * SIG_MAX + i] = axx * bx[a] + axy * by[a];
            s_sig[(2 * a + 1) * SIG_MAX + i] = axy * bx[a] + ayy * by[a];
        }
    }
    __syncthreads();
    if (!active) return;

    // ---- phase 3: faces of the own cell, mesoscopic flux
    R F[NQ];
#pragma unroll
    for (int a = 0; a < NQ; a++) F[a] = R(0);
    const uint16_t *my_nb = m.sig_nb + (int64_t)(s0 + tid) * MAXF;
#pragma unroll
    for (int sl = 0; sl < MAXF; sl++) {
        const int kind = m.sl_kind[sl * np + g];
        if (kind == SK_NONE) continue;
        const R *G = geo + (int64_t)(6 * sl) * np + g;
        const R nx = G[0], ny = G[np], rmx = G[2 * np], rmy = G[3 * np];
        if (kind == SK_INTERIOR) {
            const R rox = G[4 * np], roy = G[5 * np];
            const int o = my_nb[sl];
            R fbar[NQ], w0 = R(0), w1 = R(0), w2 = R(0);
#pragma unroll
            for (int a = 0; a < NQ; a++) {
                const R s = xdot<R>(a, nx, ny);
                const R ex = R(EX(a)) * k.dt, ey = R(EY(a)) * k.dt;
                const R A = s_fbp[a * LOC_MAX + tid] + (rmx - ex) * s_sig[(2 * a) * SIG_MAX + tid] +
                            (rmy - ey) * s_sig[(2 * a + 1) * SIG_MAX + tid];
                const R B = s_fbp[a * LOC_MAX + o] + (rox - ex) * s_sig[(2 * a) * SIG_MAX + o] +
                            (roy - ey) * s_sig[(2 * a + 1) * SIG_MAX + o];
                fbar[a] = s > k.tie ? A : (s < -k.tie ? B : R(0.5) * (A + B));
                w0 += fbar[a];
                if (EX(a) == 1) w1 += fbar[a]; else if (EX(a) == -1) w1 -= fbar[a];
                if (EY(a) == 1) w2 += fbar[a]; else if (EY(a) == -1) w2 -= fbar[a];
            }
            R ux, uy, feqb[NQ];
            vel_of<R>(w0, w1, w2, ux, uy);
            feq9f<R>(w0, ux, uy, feqb);
#pragma unroll
            for (int a = 0; a < NQ; a++) {
                const R s = xdot<R>(a, nx, ny);
                F[a] += s * ((fbar[a] + k.b * feqb[a]) * k.c);
            }
        } else {
            const int p = kind;
            const int bk = c.bc_kind[p];
            R rb = rho_n, ubx = R(0), uby = R(0);
            if (bk == BK_MOVING_WALL) { ubx = CoefR<R>::par(c, p, 0); uby = CoefR<R>::par(c, p, 1); }
            else if (bk == BK_FARFIELD) { rb = CoefR<R>::par(c, p, 0); ubx = CoefR<R>::par(c, p, 1); uby = CoefR<R>::par(c, p, 2); }
            else if (bk == BK_OUTLET) { ubx = ux_n; uby = uy_n; }
            R feqb[NQ];
            feq9f<R>(rb, ubx, uby, feqb);
            R px_ = R(0), py_ = R(0);
#pragma unroll
            for (int a = 0; a < NQ; a++) {
                const R s = xdot<R>(a, nx, ny);
                R fb;
                if (s < -k.tie) {
                    fb = feqb[a] + (fn[a] - feqn[a]);     // non-equilibrium extrapolation
                } else {
                    const R A = s_fbp[a * LOC_MAX + tid] + (rmx - R(EX(a)) * k.dt) * s_sig[(2 * a) * SIG_MAX + tid] +
                                (rmy - R(EY(a)) * k.dt) * s_sig[(2 * a + 1) * SIG_MAX + tid];
                    fb = (A + k.b * feqb[a]) * k.c;
                }
                F[a] += s * fb;
                px_ += R(EX(a)) * (s * fb);
                py_ += R(EY(a)) * (s * fb);
            }
            if (m.force) {       // diagnostic steps only: momentum leaving the fluid through this patch
                atomicAdd(&m.force[2 * p], to_f64<R>(px_));
                atomicAdd(&m.force[2 * p + 1], to_f64<R>(py_));
            }
        }
    }

    // ---- macroscopic flux (moments of F) -> W^{n+1} in FP64; cell update f^{n+1} (Eq. fn+1)
    const R dtv = static_cast<const R *>(m.dtV)[g];
    R M0 = R(0), M1 = R(0), M2 = R(0);
#pragma unroll
    for (int a = 0; a < NQ; a++) {
        M0 += F[a];
        if (EX(a) == 1) M1 += F[a]; else if (EX(a) == -1) M1 -= F[a];
        if (EY(a) == 1) M2 += F[a]; else if (EY(a) == -1) M2 -= F[a];
    }
    const R d0 = dtv * M0, d1 = dtv * M1, d2 = dtv * M2;
    const double W0 = w0n - to_f64<R>(d0), W1 = w1n - to_f64<R>(d1), W2 = w2n - to_f64<R>(d2);
    Wout[g] = W0;
    Wout[np + g] = W1;
    Wout[2 * np + g] = W2;
    R rho1, ux1, uy1, feq1[NQ];
    if constexpr (P == P_FP64) {
        macro_of<R>(W0, W1, W2, rho1, ux1, uy1);
    } else {
        // FP32 compute: W^{n+1} in FP32 from the FP32 copies already at hand
        rho1 = rho_n - d0;
        vel_of<R>(rho1, from_f64<R>(w1n) - d1, from_f64<R>(w2n) - d2, ux1, uy1);
    }
    feq9f<R>(rho1, ux1, uy1, feq1);
#pragma unroll
    for (int a = 0; a < NQ; a++) {
        R fnew;
        if constexpr (P == P_FP64) fnew = (fn[a] - dtv * F[a] + k.r * feq1[a]) / (R(1) + k.r);
        else fnew = (fn[a] - dtv * F[a] + k.r * feq1[a]) * c.finv1r;
        fout[a * np + g] = SP::enc(fnew, feq1[a], a);
    }
}

template <int P> constexpr size_t tiled_smem() {
    return sizeof(typename Store<P>::R) * (size_t)(NQ * LOC_MAX + 2 * NQ * SIG_MAX);
}

template <int P> cudaError_t prepare_tiled_p() {
    return cudaFuncSetAttribute(k_step_tiled<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tiled_smem<P>());
}

template <int P>
cudaError_t launch_tiled_p(const TiledMesh &m, const Coefs &c, const void *fin, void *fout, const double *Wn,
                           double *Wout, cudaStream_t st)
{
    using T = typename Store<P>::T;
    if (m.n_tiles <= 0) return cudaSuccess;
    k_step_tiled<P><<<m.n_tiles, TILE_MAX, tiled_smem<P>(), st>>>(m, c, static_cast<const T *>(fin),
                                                                  static_cast<T *>(fout), Wn, Wout);
    return cudaGetLastError();
}

}  // namespace sdugks
