// step_tiled.cuh -- fused S-DUGKS step on an unstructured quad mesh.
//
// One CTA per tile of up to TILE_MAX cells (one thread per interior cell).  The tile
// stages in shared memory the transformed distribution fbar+ of its cells and of
// two halo rings (Eq. fbarplus), then the LLSR gradient of its cells and of the
// first ring, then every thread reconstructs the interface distribution on the
// faces of its own cell along the characteristic (Eqs. fbpsource, fbar, Macro at the
// face, Feq, f_t_n+1) and sums the mesoscopic flux (Eq. MesoFlux).  Its moments, the
// macroscopic flux (Eq. MacroFlux), are accumulated in FP64 into
// W^{n+1} = W^n - dt/V F_macro (Eq. MacroUpdate, the moment of Eq. Integration), whose
// equilibrium then closes the implicit cell update of f (Eq. fn+1).  f and W
// ping-pong between two buffers each; nothing else is stored between steps.
//
// An interior face is evaluated by the threads of both cells with identical operands
// in the same order, so both see the same interface values and the face fluxes
// cancel exactly in the sum over cells.
#pragma once
#include "d2q9.cuh"

namespace sdugks {

template <int P>
__global__ void __launch_bounds__(TILE_MAX)
k_step_tiled(const TiledMesh m, const Coefs c, const typename Store<P>::T *__restrict__ fin,
             typename Store<P>::T *__restrict__ fout, const double *__restrict__ Wn,
             double *__restrict__ Wout)
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
    const int64_t np = m.npad, fp = m.fpad;
    const R a_plus = R(c.a_plus), b_plus = R(c.b_plus), c_face = R(c.c_face), dt = R(c.dt), tie = R(c.tie);
    const R *nbd = static_cast<const R *>(m.nbd);
    const R *ainv = static_cast<const R *>(m.ainv);
    const R *nl = static_cast<const R *>(m.nl);
    const R *ro = static_cast<const R *>(m.ro);
    const R *rk = static_cast<const R *>(m.rk);

    // ---- phase 1: fbar+ = a f^n + b feq(W^n) for own cells (kept in registers) and halos
    const bool active = tid < n_int;
    const int64_t g = c0 + tid;
    R fn[NQ], feqn[NQ];
    R rho_n = R(1), ux_n = R(0), uy_n = R(0);
    if (active) {
        macro_of<R>(Wn[g], Wn[np + g], Wn[2 * np + g], rho_n, ux_n, uy_n);
        feq9<R>(rho_n, ux_n, uy_n, feqn);
#pragma unroll
        for (int a = 0; a < NQ; a++) {
            fn[a] = SP::dec(fin[a * np + g], feqn[a], a);
            s_fbp[a * LOC_MAX + tid] = a_plus * fn[a] + b_plus * feqn[a];
        }
    }
    for (int i = n_int + tid; i < n_loc; i += blockDim.x) {
        const int64_t gh = m.halo[h0 + i - n_int];
        R rho, ux, uy, fe[NQ];
        macro_of<R>(Wn[gh], Wn[np + gh], Wn[2 * np + gh], rho, ux, uy);
        feq9<R>(rho, ux, uy, fe);
#pragma unroll
        for (int a = 0; a < NQ; a++)
            s_fbp[a * LOC_MAX + i] = a_plus * SP::dec(fin[a * np + gh], fe[a], a) + b_plus * fe[a];
    }
    __syncthreads();

    // ---- phase 2: LLSR gradient sigma = A^{-1} sum_k d_k (fbar+_k - fbar+_j)
    for (int i = tid; i < n_sig; i += blockDim.x) {
        const int64_t gi = i < n_int ? (int64_t)c0 + i : (int64_t)m.halo[h0 + i - n_int];
        const uint16_t *nb = m.sig_nb + (int64_t)(s0 + i) * MAXF;
        R bx[NQ], by[NQ];
#pragma unroll
        for (int a = 0; a < NQ; a++) { bx[a] = R(0); by[a] = R(0); }
#pragma unroll
        for (int sl = 0; sl < MAXF; sl++) {
            const int k = nb[sl];
            if (k == NO_LOCAL) continue;
            const R dx = nbd[(2 * sl) * np + gi], dy = nbd[(2 * sl + 1) * np + gi];
#pragma unroll
            for (int a = 0; a < NQ; a++) {
                const R d = s_fbp[a * LOC_MAX + k] - s_fbp[a * LOC_MAX + i];
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
    for (int sl = 0; sl < MAXF; sl++) {
        const int fid = m.cface[sl * np + g];
        if (fid < 0) break;
        const int own = m.fown[fid], nbr = m.fnbr[fid];
        const bool mine = (own == (int)g);
        R nx = nl[fid], ny = nl[fp + fid];
        if (!mine) { nx = -nx; ny = -ny; }
        if (nbr >= 0) {
            const int o = m.fo_local[sl * np + g];
            R rmx = ro[fid], rmy = ro[fp + fid], rox = rk[fid], roy = rk[fp + fid];
            if (!mine) { R tx = rmx, ty = rmy; rmx = rox; rmy = roy; rox = tx; roy = ty; }
            R fbar[NQ], w0 = R(0), w1 = R(0), w2 = R(0);
#pragma unroll
            for (int a = 0; a < NQ; a++) {
                const R s = xdot<R>(a, nx, ny);
                const R ex = R(EX(a)) * dt, ey = R(EY(a)) * dt;
                const R A = s_fbp[a * LOC_MAX + tid] + (rmx - ex) * s_sig[(2 * a) * SIG_MAX + tid] +
                            (rmy - ey) * s_sig[(2 * a + 1) * SIG_MAX + tid];
                const R B = s_fbp[a * LOC_MAX + o] + (rox - ex) * s_sig[(2 * a) * SIG_MAX + o] +
                            (roy - ey) * s_sig[(2 * a + 1) * SIG_MAX + o];
                fbar[a] = s > tie ? A : (s < -tie ? B : R(0.5) * (A + B));
                w0 += fbar[a];
                if (EX(a) == 1) w1 += fbar[a]; else if (EX(a) == -1) w1 -= fbar[a];
                if (EY(a) == 1) w2 += fbar[a]; else if (EY(a) == -1) w2 -= fbar[a];
            }
            R feqb[NQ];
            feq9<R>(w0, w1 / w0, w2 / w0, feqb);
#pragma unroll
            for (int a = 0; a < NQ; a++) {
                const R s = xdot<R>(a, nx, ny);
                F[a] += s * ((fbar[a] + b_plus * feqb[a]) * c_face);
            }
        } else {
            const int p = -1 - nbr;
            const int kind = c.bc_kind[p];
            R rb = rho_n, ubx = R(0), uby = R(0);
            if (kind == BK_MOVING_WALL) { ubx = R(c.bc_par[p][0]); uby = R(c.bc_par[p][1]); }
            else if (kind == BK_FARFIELD) { rb = R(c.bc_par[p][0]); ubx = R(c.bc_par[p][1]); uby = R(c.bc_par[p][2]); }
            else if (kind == BK_OUTLET) { ubx = ux_n; uby = uy_n; }
            R feqb[NQ];
            feq9<R>(rb, ubx, uby, feqb);
            const R rmx = ro[fid], rmy = ro[fp + fid];
#pragma unroll
            for (int a = 0; a < NQ; a++) {
                const R s = xdot<R>(a, nx, ny);
                R fb;
                if (s < -tie) {
                    fb = feqb[a] + (fn[a] - feqn[a]);     // non-equilibrium extrapolation
                } else {
                    const R A = s_fbp[a * LOC_MAX + tid] + (rmx - R(EX(a)) * dt) * s_sig[(2 * a) * SIG_MAX + tid] +
                                (rmy - R(EY(a)) * dt) * s_sig[(2 * a + 1) * SIG_MAX + tid];
                    fb = (A + b_plus * feqb[a]) * c_face;
                }
                F[a] += s * fb;
            }
        }
    }

    // ---- macroscopic flux (FP64 moments of F) -> W^{n+1}; cell update f^{n+1} (Eq. fn+1)
    double M0 = 0.0, M1 = 0.0, M2 = 0.0;
#pragma unroll
    for (int a = 0; a < NQ; a++) {
        const double Fa = (double)F[a];
        M0 += Fa;
        if (EX(a) == 1) M1 += Fa; else if (EX(a) == -1) M1 -= Fa;
        if (EY(a) == 1) M2 += Fa; else if (EY(a) == -1) M2 -= Fa;
    }
    const double dtv = m.dtV[g];
    const double W0 = Wn[g] - dtv * M0, W1 = Wn[np + g] - dtv * M1, W2 = Wn[2 * np + g] - dtv * M2;
    Wout[g] = W0;
    Wout[np + g] = W1;
    Wout[2 * np + g] = W2;
    R rho1, ux1, uy1, feq1[NQ];
    macro_of<R>(W0, W1, W2, rho1, ux1, uy1);
    feq9<R>(rho1, ux1, uy1, feq1);
    const R r = R(c.r), dtvr = R(dtv);
#pragma unroll
    for (int a = 0; a < NQ; a++) {
        R fnew;
        if constexpr (P == P_FP64) fnew = (fn[a] - dtvr * F[a] + r * feq1[a]) / (R(1) + r);
        else fnew = (fn[a] - dtvr * F[a] + r * feq1[a]) * R(c.inv1r);
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
    const size_t smem = tiled_smem<P>();
    if (m.n_tiles <= 0) return cudaSuccess;
    k_step_tiled<P><<<m.n_tiles, TILE_MAX, smem, st>>>(m, c, static_cast<const T *>(fin), static_cast<T *>(fout),
                                                        Wn, Wout);
    return cudaGetLastError();
}

}  // namespace sdugks
