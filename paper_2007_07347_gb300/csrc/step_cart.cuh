// step_cart.cuh -- fused S-DUGKS step on a uniform Cartesian grid.
//
// The same update as the tiled kernel (Eqs. fbarplus, fbpsource, fbar, Macro, Feq,
// f_t_n+1, MesoFlux, MacroFlux, MacroUpdate, fn+1), specialised to nx x ny
// rectangles of one size: cell (i, j) sits at i + pitch j, a CTA owns a TX x TY
// block and stages it with a two-cell halo, the LLSR gradient reduces to central
// (or, next to a wall, one-sided) differences, and on every face the upwind side of
// each velocity is known at compile time.  No mesh arrays are read.  Each grid side
// is either one boundary patch or periodic with the opposite side.
#pragma once
#include "d2q9.cuh"
#include "step_tiled.cuh"   // CoefR

namespace sdugks {

template <int TX, int TY> struct CartShape {
    static constexpr int LX = TX + 4, LY = TY + 4;   // staged block with a two-cell halo
    static constexpr int GX = TX + 2, GY = TY + 2;   // cells whose gradient is needed
    static constexpr int NT = TX * TY;
};

template <int P, int TX, int TY> constexpr size_t cart_smem() {
    using S = CartShape<TX, TY>;
    return sizeof(typename Store<P>::R) * (size_t)(NQ * S::LX * S::LY + 2 * NQ * S::GX * S::GY);
}

// Face of the own cell in direction D (0 +x, 1 -x, 2 +y, 3 -y): returns the flux
// contribution (xi . n l) f_b for every velocity in F.
template <int D, class R>
__device__ __forceinline__ void cart_face(R F[NQ], const R *s_fbp, const R *s_sig, int lme, int loth, int gme,
                                          int goth, bool interior, int patch, const Coefs &c, const CoefR<R> &k,
                                          const R fn[NQ], const R feqn[NQ], R rho_n, R ux_n, R uy_n, R hx, R hy,
                                          int LXY, int GXY)
{
    // outward normal * length, and x_f - x_j (x_f - x_k is its negative)
    const R nx = D == 0 ? hy : (D == 1 ? -hy : R(0));
    const R ny = D == 2 ? hx : (D == 3 ? -hx : R(0));
    const R rx = D == 0 ? R(0.5) * hx : (D == 1 ? R(-0.5) * hx : R(0));
    const R ry = D == 2 ? R(0.5) * hy : (D == 3 ? R(-0.5) * hy : R(0));
    if (interior) {
        R fbar[NQ], w0 = R(0), w1 = R(0), w2 = R(0);
#pragma unroll
        for (int a = 0; a < NQ; a++) {
            // sign of xi . n, fixed per velocity and direction
            const int sg = (D < 2) ? (D == 0 ? EX(a) : -EX(a)) : (D == 2 ? EY(a) : -EY(a));
            const R ex = R(EX(a)) * k.dt, ey = R(EY(a)) * k.dt;
            R A = R(0), B = R(0);
            if (sg >= 0)
                A = s_fbp[a * LXY + lme] + (rx - ex) * s_sig[(2 * a) * GXY + gme] + (ry - ey) * s_sig[(2 * a + 1) * GXY + gme];
            if (sg <= 0)
                B = s_fbp[a * LXY + loth] + (-rx - ex) * s_sig[(2 * a) * GXY + goth] +
                    (-ry - ey) * s_sig[(2 * a + 1) * GXY + goth];
            fbar[a] = sg > 0 ? A : (sg < 0 ? B : R(0.5) * (A + B));
            w0 += fbar[a];
            if (EX(a) == 1) w1 += fbar[a]; else if (EX(a) == -1) w1 -= fbar[a];
            if (EY(a) == 1) w2 += fbar[a]; else if (EY(a) == -1) w2 -= fbar[a];
        }
        R feqb[NQ];
        feq9<R>(w0, w1 / w0, w2 / w0, feqb);
#pragma unroll
        for (int a = 0; a < NQ; a++) {
            const int sg = (D < 2) ? (D == 0 ? EX(a) : -EX(a)) : (D == 2 ? EY(a) : -EY(a));
            if (sg == 0) continue;
            const R s = xdot<R>(a, nx, ny);
            F[a] += s * ((fbar[a] + k.b * feqb[a]) * k.c);
        }
    } else {
        const int bk = c.bc_kind[patch];
        R rb = rho_n, ubx = R(0), uby = R(0);
        if (bk == BK_MOVING_WALL) { ubx = CoefR<R>::par(c, patch, 0); uby = CoefR<R>::par(c, patch, 1); }
        else if (bk == BK_FARFIELD) {
            rb = CoefR<R>::par(c, patch, 0); ubx = CoefR<R>::par(c, patch, 1); uby = CoefR<R>::par(c, patch, 2);
        } else if (bk == BK_OUTLET) { ubx = ux_n; uby = uy_n; }
        R feqb[NQ];
        feq9<R>(rb, ubx, uby, feqb);
#pragma unroll
        for (int a = 0; a < NQ; a++) {
            const int sg = (D < 2) ? (D == 0 ? EX(a) : -EX(a)) : (D == 2 ? EY(a) : -EY(a));
            if (sg == 0) continue;
            const R s = xdot<R>(a, nx, ny);
            R fb;
            if (sg < 0) {
                fb = feqb[a] + (fn[a] - feqn[a]);          // non-equilibrium extrapolation
            } else {
                const R A = s_fbp[a * LXY + lme] + (rx - R(EX(a)) * k.dt) * s_sig[(2 * a) * GXY + gme] +
                            (ry - R(EY(a)) * k.dt) * s_sig[(2 * a + 1) * GXY + gme];
                fb = (A + k.b * feqb[a]) * k.c;
            }
            F[a] += s * fb;
        }
    }
}

template <int P, int TX, int TY>
__global__ void __launch_bounds__(TX * TY)
k_step_cart(const CartMesh m, const Coefs c, const typename Store<P>::T *__restrict__ fin,
            typename Store<P>::T *__restrict__ fout, const double *__restrict__ Wn, double *__restrict__ Wout)
{
    using R = typename Store<P>::R;
    using SP = Store<P>;
    using S = CartShape<TX, TY>;
    constexpr int LXY = S::LX * S::LY, GXY = S::GX * S::GY;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R *s_fbp = reinterpret_cast<R *>(smem_raw);     // [NQ][LY][LX]
    R *s_sig = s_fbp + NQ * LXY;                     // [2 NQ][GY][GX]

    const int ntx = (m.nx + TX - 1) / TX;
    const int x0 = (blockIdx.x % ntx) * TX, y0 = (blockIdx.x / ntx) * TY;
    const int tid = threadIdx.x, ti = tid % TX, tj = tid / TX;
    const int64_t np = m.npad, pitch = m.pitch;
    const CoefR<R> k(c);
    const R hx = R(m.dx), hy = R(m.dy);

    // domain cell of a staged position (periodic sides wrap), or -1 outside
    auto cell_of = [&](int gi, int gj) -> int64_t {
        if (gi < 0 || gi >= m.nx) {
            if (!m.periodic_x) return -1;
            gi = (gi + m.nx) % m.nx;
        }
        if (gj < 0 || gj >= m.ny) {
            if (!m.periodic_y) return -1;
            gj = (gj + m.ny) % m.ny;
        }
        return gi + pitch * gj;
    };

    // ---- phase 1: fbar+ of the own cell (kept in registers) and of the halo
    const int gi = x0 + ti, gj = y0 + tj;
    const bool active = gi < m.nx && gj < m.ny;
    const int64_t g = (int64_t)gi + pitch * gj;
    const int lme = (tj + 2) * S::LX + (ti + 2);
    R fn[NQ], feqn[NQ];
    R rho_n = R(1), ux_n = R(0), uy_n = R(0);
    double w0n = 1.0, w1n = 0.0, w2n = 0.0;
    if (active) {
        w0n = Wn[g]; w1n = Wn[np + g]; w2n = Wn[2 * np + g];
        macro_of<R>(w0n, w1n, w2n, rho_n, ux_n, uy_n);
        feq9<R>(rho_n, ux_n, uy_n, feqn);
#pragma unroll
        for (int a = 0; a < NQ; a++) {
            fn[a] = SP::dec(fin[a * np + g], feqn[a], a);
            s_fbp[a * LXY + lme] = k.a * fn[a] + k.b * feqn[a];
        }
    }
    // every other staged position: the two-cell ring, and block positions without an
    // own cell (past the grid edge; they hold wrapped cells on periodic sides)
    for (int q = tid; q < LXY; q += S::NT) {
        const int li = q % S::LX, lj = q / S::LX;
        const int bi = li - 2, bj = lj - 2;
        if (bi >= 0 && bi < TX && bj >= 0 && bj < TY && x0 + bi < m.nx && y0 + bj < m.ny) continue;
        const int64_t gh = cell_of(x0 + bi, y0 + bj);
        if (gh < 0) continue;
        R rho, ux, uy, fe[NQ];
        macro_of<R>(Wn[gh], Wn[np + gh], Wn[2 * np + gh], rho, ux, uy);
        feq9<R>(rho, ux, uy, fe);
#pragma unroll
        for (int a = 0; a < NQ; a++) s_fbp[a * LXY + q] = k.a * SP::dec(fin[a * np + gh], fe[a], a) + k.b * fe[a];
    }
    __syncthreads();

    // ---- phase 2: gradient on the block and its first ring.  LLSR over the existing
    // face neighbours of a uniform grid: sigma_x = sum_k dx_k (phi_k - phi) / sum_k dx_k^2
    for (int q = tid; q < GXY; q += S::NT) {
        const int gx = q % S::GX, gy = q / S::GX;
        const int ci = x0 + gx - 1, cj = y0 + gy - 1;
        if (cell_of(ci, cj) < 0) continue;
        const bool hasE = m.periodic_x || ci + 1 < m.nx, hasW = m.periodic_x || ci - 1 >= 0;
        const bool hasN = m.periodic_y || cj + 1 < m.ny, hasS = m.periodic_y || cj - 1 >= 0;
        const int l = (gy + 1) * S::LX + (gx + 1);
        const R nxk = R((hasE ? 1 : 0) + (hasW ? 1 : 0)), nyk = R((hasN ? 1 : 0) + (hasS ? 1 : 0));
        const bool singular = nxk == R(0) || nyk == R(0);
        const R ax = singular ? R(0) : R(1) / (nxk * hx * hx), ay = singular ? R(0) : R(1) / (nyk * hy * hy);
#pragma unroll
        for (int a = 0; a < NQ; a++) {
            const R *f = s_fbp + a * LXY;
            const R p = f[l];
            R bx = R(0), by = R(0);
            if (hasE) bx += hx * (f[l + 1] - p);
            if (hasW) bx += -hx * (f[l - 1] - p);
            if (hasN) by += hy * (f[l + S::LX] - p);
            if (hasS) by += -hy * (f[l - S::LX] - p);
            s_sig[(2 * a) * GXY + q] = ax * bx;
            s_sig[(2 * a + 1) * GXY + q] = ay * by;
        }
    }
    __syncthreads();
    if (!active) return;

    // ---- phase 3: the four faces of the own cell (order -x, +x, -y, +y)
    R F[NQ];
#pragma unroll
    for (int a = 0; a < NQ; a++) F[a] = R(0);
    const int gme = (tj + 1) * S::GX + (ti + 1);
    {
        const bool in = m.periodic_x || gi - 1 >= 0;
        cart_face<1, R>(F, s_fbp, s_sig, lme, lme - 1, gme, gme - 1, in, m.side_patch[3], c, k, fn, feqn, rho_n, ux_n,
                        uy_n, hx, hy, LXY, GXY);
    }
    {
        const bool in = m.periodic_x || gi + 1 < m.nx;
        cart_face<0, R>(F, s_fbp, s_sig, lme, lme + 1, gme, gme + 1, in, m.side_patch[1], c, k, fn, feqn, rho_n, ux_n,
                        uy_n, hx, hy, LXY, GXY);
    }
    {
        const bool in = m.periodic_y || gj - 1 >= 0;
        cart_face<3, R>(F, s_fbp, s_sig, lme, lme - S::LX, gme, gme - S::GX, in, m.side_patch[0], c, k, fn, feqn, rho_n,
                        ux_n, uy_n, hx, hy, LXY, GXY);
    }
    {
        const bool in = m.periodic_y || gj + 1 < m.ny;
        cart_face<2, R>(F, s_fbp, s_sig, lme, lme + S::LX, gme, gme + S::GX, in, m.side_patch[2], c, k, fn, feqn, rho_n,
                        ux_n, uy_n, hx, hy, LXY, GXY);
    }

    // ---- macroscopic flux -> W^{n+1} (FP64); cell update f^{n+1}
    const R dtv = P == P_FP64 ? R(m.dtV) : R(m.fdtV);
    R M0 = R(0), M1 = R(0), M2 = R(0);
#pragma unroll
    for (int a = 0; a < NQ; a++) {
        M0 += F[a];
        if (EX(a) == 1) M1 += F[a]; else if (EX(a) == -1) M1 -= F[a];
        if (EY(a) == 1) M2 += F[a]; else if (EY(a) == -1) M2 -= F[a];
    }
    const R d0 = dtv * M0, d1 = dtv * M1, d2 = dtv * M2;
    const double W0 = w0n - (double)d0, W1 = w1n - (double)d1, W2 = w2n - (double)d2;
    Wout[g] = W0;
    Wout[np + g] = W1;
    Wout[2 * np + g] = W2;
    R rho1, ux1, uy1, feq1[NQ];
    if constexpr (P == P_FP64) {
        macro_of<R>(W0, W1, W2, rho1, ux1, uy1);
    } else {
        rho1 = R(w0n) - d0;
        ux1 = (R(w1n) - d1) / rho1;
        uy1 = (R(w2n) - d2) / rho1;
    }
    feq9<R>(rho1, ux1, uy1, feq1);
#pragma unroll
    for (int a = 0; a < NQ; a++) {
        R fnew;
        if constexpr (P == P_FP64) fnew = (fn[a] - dtv * F[a] + k.r * feq1[a]) / (R(1) + k.r);
        else fnew = (fn[a] - dtv * F[a] + k.r * feq1[a]) * c.finv1r;
        fout[a * np + g] = SP::enc(fnew, feq1[a], a);
    }
}

template <int P, int TX, int TY> cudaError_t prepare_cart_p() {
    return cudaFuncSetAttribute(k_step_cart<P, TX, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)cart_smem<P, TX, TY>());
}

template <int P, int TX, int TY>
cudaError_t launch_cart_p(const CartMesh &m, const Coefs &c, const void *fin, void *fout, const double *Wn, double *Wout,
                          cudaStream_t st)
{
    using T = typename Store<P>::T;
    const int ntx = (m.nx + TX - 1) / TX, nty = (m.ny + TY - 1) / TY;
    k_step_cart<P, TX, TY><<<ntx * nty, TX * TY, cart_smem<P, TX, TY>(), st>>>(
        m, c, static_cast<const T *>(fin), static_cast<T *>(fout), Wn, Wout);
    return cudaGetLastError();
}

}  // namespace sdugks
