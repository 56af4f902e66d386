// step_cart.cuh -- fused S-DUGKS step on uniform Cartesian grids.
//
// The same update as the tiled kernel (Eqs. fbarplus, fbpsource, fbar, Macro, Feq,
// f_t_n+1, MesoFlux, MacroFlux, MacroUpdate, fn+1), specialised to nx x ny
// rectangles of one size: cell (i, j) sits at i + pitch j and a CTA owns a TX x TY
// block, staged with a two-cell halo.  The LLSR gradient reduces to central (or,
// next to a wall, one-sided) differences, and on every face the upwind side of each
// velocity is known at compile time.  No mesh arrays are read.  Each grid side is one
// boundary rule or periodic with the opposite side.
//
// Phases of one block: (1) fbar+ of the block and halo into shared memory, one
// position per thread; (2) every interior face of the block once, one per thread:
// the characteristic reconstruction from the upwind cell, with that cell's LLSR
// gradient evaluated on the spot as the two-point difference it reduces to on a
// uniform grid, and the six non-zero fluxes (xi.n l f_b of the velocities that cross
// the face) into shared memory; (3) per cell: boundary faces, the flux sum, W^{n+1}
// in FP64 and f^{n+1}.  `cart_tile` does one block; `k_step_cart` runs it for every block of one
// grid (`k_step_batch`, in k_batch.cu, for every (instance, block) item of a batch).
#pragma once
#include <climits>
#include "d2q9.cuh"

namespace sdugks {

// Rows of cells or faces are dealt to warps two at a time, each half-warp one row of 16:
// rows 4g + k pair as (4g, 4g + 2) and (4g + 1, 4g + 3), so that with the staging row
// stride SX = 24 (48 = 16 mod 32 words between the two rows of a warp) every shared
// access of a warp at a common offset from its positions hits 32 distinct banks.
// Slot s of a row set: warp s / 32, half s / 16 % 2, column s % 16.
__host__ __device__ constexpr int slot_row(int s) { return 4 * (s >> 6) + ((s >> 5) & 1) + 2 * ((s >> 4) & 1); }
__host__ __device__ constexpr int row_slot(int r, int col) {
    return 32 * (2 * (r >> 2) + (r & 1)) + 16 * ((r >> 1) & 1) + col;
}
// warps that hold rows 0 .. nr-1
__host__ __device__ constexpr int row_warps(int nr) { return 2 * (nr / 4) + (nr % 4 < 2 ? nr % 4 : 2); }

template <int TX, int TY> struct CartShape {
    static_assert(TX == 16 && TY % 2 == 0 && TY <= 16, "blocks are 16 wide with an even height of at most 16");
    static constexpr int LX = TX + 4, LY = TY + 4;   // staged block with a two-cell halo
    static constexpr int SX = 24;                    // row stride of the staged planes (>= LX)
    static constexpr int PLANE = SX * LY;            // plane stride (one velocity)
    static constexpr int NT = TX * TY;
    static constexpr int WX = row_warps(TY);         // warps of the cell rows / constant-x face rows
    static constexpr int WY = row_warps(TY + 1);     // warps of the constant-y face rows
    // face slots: constant-x faces left of each block cell (32 WX slots), then the TY faces on
    // the block's right edge; constant-y faces below each block cell and above the top row
    static constexpr int NSX = 32 * WX + TY;
    static constexpr int NSY = 32 * WY;
};

// Threads per CTA: one per face slot (>= cell slots + ring positions of the staging).
template <int TX, int TY> __host__ __device__ constexpr int cart_threads() {
    using S = CartShape<TX, TY>;
    constexpr int nf = 32 * (S::WX + S::WY);
    constexpr int nl = 32 * S::WX + S::LX * S::LY - S::NT;
    return nf > nl ? nf : nl;
}

template <int P, int TX, int TY> constexpr size_t cart_smem() {
    using S = CartShape<TX, TY>;
    return sizeof(typename Store<P>::R) * (size_t)(NQ * S::PLANE + 6 * (S::NSX + S::NSY));
}

// TMA staging of an interior block: two tensor copies bring f^n and W^n of the block
// and its two-cell halo into shared memory, boxes of (x, y, plane) whose first column
// lies OFF columns left of the block so that it starts on a 16-byte boundary (x0 is a
// multiple of 16): f box BW x (TY + 4) x NQ, W box WBW x (TY + 4) x 3.  The boxes
// overlay the face-flux arrays (written only after phase 1 has read the boxes) and an
// mbarrier follows; offsets from a 128-byte aligned base.
template <class T> __host__ __device__ constexpr int tma_off() { return sizeof(T) == 8 ? 2 : (sizeof(T) == 4 ? 4 : 8); }
template <int P, int TX, int TY> struct CartTmaBox {
    using T = typename Store<P>::T;
    using R = typename Store<P>::R;
    using S = CartShape<TX, TY>;
    static constexpr int OFF = tma_off<T>(), BW = TX + 2 * OFF;
    static constexpr int WOFF = 2, WBW = TX + 4;
    static constexpr size_t F_BYTES = sizeof(T) * (size_t)NQ * S::LY * BW;
    static constexpr size_t W_BYTES = sizeof(double) * (size_t)3 * S::LY * WBW;
    static constexpr size_t FBP_BYTES = sizeof(R) * (size_t)NQ * S::PLANE;
    static constexpr size_t FLUX_BYTES = sizeof(R) * (size_t)6 * (S::NSX + S::NSY);
    static constexpr size_t F_OFF = (FBP_BYTES + 127) / 128 * 128;
    static constexpr size_t W_OFF = F_OFF + (F_BYTES + 127) / 128 * 128;
    static constexpr size_t END = (FBP_BYTES + FLUX_BYTES > W_OFF + W_BYTES) ? FBP_BYTES + FLUX_BYTES : W_OFF + W_BYTES;
    static constexpr size_t BAR_OFF = (END + 15) / 16 * 16;
    static constexpr size_t SMEM = BAR_OFF + 16 + 128;   // 128 bytes of slack align the base
    static_assert((BW * sizeof(T)) % 16 == 0 && (WBW * sizeof(double)) % 16 == 0, "TMA box rows must be 16-byte multiples");
    static_assert(BW <= 256 && WBW <= 256 && S::LY <= 256, "TMA box dimensions are at most 256");
};

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits for the phase `parity` of the mbarrier at shared address `bar` to complete;
// gives up after `limit_ns` nanoseconds and returns false (at once when limit_ns is 0).
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, uint64_t limit_ns)
{
    if (limit_ns == 0) return false;
    const uint64_t t0 = global_ns();
    for (;;) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\t"
                     "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done) : "r"(bar), "r"(parity) : "memory");
        if (done) return true;
        if (global_ns() - t0 > limit_ns) return false;
    }
}

__device__ __forceinline__ void mbar_init(uint32_t bar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// One thread: arm the barrier at `bar` for the two boxes of the block at (x0, y0) and
// start the tensor copies into dst_f / dst_w (shared addresses): the f box from
// column x0 - OFF, the W box from x0 - 2, both from row y0 - 2.
template <int P, int TX, int TY>
__device__ __forceinline__ void tma_issue_block(uint32_t bar, uint32_t dst_f, uint32_t dst_w, const CUtensorMap *tf,
                                                const CUtensorMap *tw, int x0, int y0)
{
    using B = CartTmaBox<P, TX, TY>;
    const uint32_t bytes = (uint32_t)(B::F_BYTES + B::W_BYTES);
    const int xf = x0 - B::OFF, xw = x0 - B::WOFF, y = y0 - 2;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
                 ::"r"(dst_f), "l"(reinterpret_cast<uint64_t>(tf)), "r"(xf), "r"(y), "r"(0), "r"(bar)
                 : "memory");
    asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
                 ::"r"(dst_w), "l"(reinterpret_cast<uint64_t>(tw)), "r"(xw), "r"(y), "r"(0), "r"(bar)
                 : "memory");
}

// Default wait limit of a staging copy before the block reports SDUGKS_ERR_TIMEOUT
// through the error flag (a copy normally lands within microseconds), and the limit of
// the second wait, for copies still in flight, after a block has given up.
constexpr uint64_t TMA_WAIT_NS = 200000000ull;

// Velocities crossing a face of constant x (xi_x != 0) and of constant y, in slot order.
__device__ constexpr int XSLOT_A(int k) { return k == 0 ? 1 : k == 1 ? 3 : k == 2 ? 5 : k == 3 ? 6 : k == 4 ? 7 : 8; }
__device__ constexpr int YSLOT_A(int k) { return k == 0 ? 2 : k == 1 ? 4 : k == 2 ? 5 : k == 3 ? 6 : k == 4 ? 7 : 8; }

// Step coefficients in the compute precision.
template <class R> struct CartK;
template <> struct CartK<double> {
    double a, b, c, r, dt, dtV, hx, hy, ihx, ihy;
    __device__ explicit CartK(const CartInst &m)
        : a(m.a), b(m.b), c(m.c), r(m.r), dt(m.dt), dtV(m.dtV), hx(m.dx), hy(m.dy), ihx(m.ihx), ihy(m.ihy) {}
    __device__ static double par(const CartInst &m, int side, int i) { return m.side_par[side][i]; }
    __device__ static double drho_par(const CartInst &m, int side) { return m.side_par[side][0] - 1.0; }
};
template <> struct CartK<float> {
    float a, b, c, r, dt, dtV, hx, hy, ihx, ihy;
    __device__ explicit CartK(const CartInst &m)
        : a(m.fa), b(m.fb), c(m.fc), r(m.fr), dt(m.fdt), dtV(m.fdtV), hx(m.fdx), hy(m.fdy),
          ihx(m.fihx), ihy(m.fihy) {}
    __device__ static float par(const CartInst &m, int side, int i) { return m.fside_par[side][i]; }
    __device__ static float drho_par(const CartInst &m, int side) { return m.fside_drho[side]; }
};

// LLSR gradient stencil of one staged cell on a uniform grid.  Over the face
// neighbours that exist, sum_k d_k (phi_k - phi) / sum_k d_k^2 is the central
// difference (phi_E - phi_W) / 2h when both exist and the one-sided difference
// otherwise; oE/oW/oN/oS are the staged offsets (0 for a missing neighbour) and ax, ay
// the factors 1/(2h) or 1/h.
template <class R> struct Sten {
    int oE, oW, oN, oS;
    R ax, ay;
};

// fbar+_j + (x_f - xi dt - x_j) . sigma_j for velocity a from staged cell l, with
// (px, py) = x_f - xi dt - x_j; UX / UY drop a component whose factor is zero
template <int a, bool UX, bool UY, class R>
__device__ __forceinline__ R cart_extrap(const R *s_fbp, int l, const Sten<R> &st, R px, R py, int LXY)
{
    const R *f = s_fbp + a * LXY;
    R v = f[l];
    if (UX) v += (px * st.ax) * (f[l + st.oE] - f[l + st.oW]);
    if (UY) v += (py * st.ay) * (f[l + st.oN] - f[l + st.oS]);
    return v;
}

// Interface distribution on a face between cell L (below/left) and R (above/right),
// along axis AX (0: face of constant x, 1: of constant y), from the staged fbar+ of
// the two cells and their neighbours; writes (xi . n_+ l) f_b of the six crossing
// velocities (n_+ = +x or +y).
template <int AX, class R>
__device__ __forceinline__ void cart_interior_face(R flux[6], const R *s_fbp, int lL, int lR, const Sten<R> &sL,
                                                   const Sten<R> &sR, const CartK<R> &k, int LXY)
{
    // x_f - x_L = +h/2 along the axis, x_f - x_R = -h/2
    const R hl = AX == 0 ? R(0.5) * k.hx : R(0.5) * k.hy;
    R fbar[NQ], w0 = R(0), w1 = R(0), w2 = R(0);
#define SDUGKS_FACE_ALPHA(a)                                                                        \
    {                                                                                               \
        constexpr int sg = AX == 0 ? EX(a) : EY(a);   /* sign of xi . n_+ */                        \
        const R ex = R(EX(a)) * k.dt, ey = R(EY(a)) * k.dt;                                         \
        R A = R(0), B = R(0);                                                                       \
        constexpr bool ux = AX == 0 || EX(a) != 0, uy = AX == 1 || EY(a) != 0;                     \
        if (sg >= 0) A = cart_extrap<a, ux, uy, R>(s_fbp, lL, sL, AX == 0 ? hl - ex : -ex, AX == 0 ? -ey : hl - ey, LXY); \
        if (sg <= 0) B = cart_extrap<a, ux, uy, R>(s_fbp, lR, sR, AX == 0 ? -hl - ex : -ex, AX == 0 ? -ey : -hl - ey, LXY); \
        fbar[a] = sg > 0 ? A : (sg < 0 ? B : R(0.5) * (A + B));                                     \
        w0 += fbar[a];                                                                              \
        if (EX(a) == 1) w1 += fbar[a]; else if (EX(a) == -1) w1 -= fbar[a];                         \
        if (EY(a) == 1) w2 += fbar[a]; else if (EY(a) == -1) w2 -= fbar[a];                         \
    }
    SDUGKS_FACE_ALPHA(0) SDUGKS_FACE_ALPHA(1) SDUGKS_FACE_ALPHA(2) SDUGKS_FACE_ALPHA(3) SDUGKS_FACE_ALPHA(4)
    SDUGKS_FACE_ALPHA(5) SDUGKS_FACE_ALPHA(6) SDUGKS_FACE_ALPHA(7) SDUGKS_FACE_ALPHA(8)
#undef SDUGKS_FACE_ALPHA
    R ux, uy, feqb[NQ];
    vel_of<R>(w0, w1, w2, ux, uy);
    feq9f<R>(w0, ux, uy, feqb);
    const R len = AX == 0 ? k.hy : k.hx;
#pragma unroll
    for (int q = 0; q < 6; q++) {
        const int a = AX == 0 ? XSLOT_A(q) : YSLOT_A(q);
        const int sg = AX == 0 ? EX(a) : EY(a);
        const R s = sg > 0 ? len : -len;
        flux[q] = s * ((fbar[a] + k.b * feqb[a]) * k.c);
    }
}

// FP32 specialisation of cart_interior_face with paired arithmetic: on this GPU one
// FFMA2/FMUL2 instruction does two independent FP32 operations (each rounded as the
// scalar operation), so the reconstructions are evaluated two velocities at a time,
// paired so that each pair is also a pair of the six face fluxes; the values are
// those of the scalar routine with its products and sums contracted to FMAs.
__device__ __forceinline__ float2 p2(float a, float b) { return make_float2(a, b); }

// fbar+ of velocity plane a at l plus cx (E - W) [plus cy (N - S)], for two
// (plane, position, stencil) triples at once
template <bool UX, bool UY>
__device__ __forceinline__ float2 extrap2(const float *s_fbp, int LXY, int ax_, int lx, const Sten<float> &sx,
                                          int ay_, int ly, const Sten<float> &sy, float2 cx, float2 cy)
{
    const float *fx = s_fbp + ax_ * LXY, *fy = s_fbp + ay_ * LXY;
    float2 v = p2(fx[lx], fy[ly]);
    if (UX) {
        const float2 dx = p2(fx[lx + sx.oE] - fx[lx + sx.oW], fy[ly + sy.oE] - fy[ly + sy.oW]);
        v = __ffma2_rn(cx, dx, v);
    }
    if (UY) {
        const float2 dy = p2(fx[lx + sx.oN] - fx[lx + sx.oS], fy[ly + sy.oN] - fy[ly + sy.oS]);
        v = __ffma2_rn(cy, dy, v);
    }
    return v;
}

template <int AX>
__device__ __forceinline__ void cart_interior_face_f32x2(float flux[6], const float *s_fbp, int lL, int lR,
                                                         const Sten<float> &sL, const Sten<float> &sR,
                                                         const CartK<float> &k, int LXY)
{
    const float hl = AX == 0 ? 0.5f * k.hx : 0.5f * k.hy, dt = k.dt;
    float fbar[NQ];
    float2 v01, v23, v45;     // reconstructions of the flux pairs (slots 0-1, 2-3, 4-5)
    if (AX == 0) {
        // x-face, left L / right R; x_f - x_L = (hl, 0), x_f - x_R = (-hl, 0)
        const float2 ax2 = p2(sL.ax, sR.ax), ay2 = p2(sL.ay, sR.ay);
        const float2 kb = __fmul2_rn(p2(hl - dt, -hl + dt), ax2);      // velocities with xi_x = +-1
        const float2 k0 = __fmul2_rn(p2(hl, -hl), ax2);                // xi_x = 0
        const float2 kc = __fmul2_rn(p2(-dt, -dt), ay2), kd = __fmul2_rn(p2(dt, dt), ay2);
        v01 = extrap2<true, false>(s_fbp, LXY, 1, lL, sL, 3, lR, sR, kb, kb);                       // (A1, B3)
        v23 = extrap2<true, true>(s_fbp, LXY, 5, lL, sL, 6, lR, sR, kb, kc);                        // (A5, B6)
        v45 = extrap2<true, true>(s_fbp, LXY, 7, lR, sR, 8, lL, sL, p2(kb.y, kb.x), p2(kd.y, kd.x)); // (B7, A8)
        const float2 t0 = extrap2<true, false>(s_fbp, LXY, 0, lL, sL, 0, lR, sR, k0, k0);           // (A0, B0)
        const float2 t2 = extrap2<true, true>(s_fbp, LXY, 2, lL, sL, 2, lR, sR, k0, kc);            // (A2, B2)
        const float2 t4 = extrap2<true, true>(s_fbp, LXY, 4, lL, sL, 4, lR, sR, k0, kd);            // (A4, B4)
        fbar[0] = 0.5f * (t0.x + t0.y); fbar[1] = v01.x; fbar[2] = 0.5f * (t2.x + t2.y); fbar[3] = v01.y;
        fbar[4] = 0.5f * (t4.x + t4.y); fbar[5] = v23.x; fbar[6] = v23.y; fbar[7] = v45.x; fbar[8] = v45.y;
    } else {
        // y-face, below L / above R; x_f - x_L = (0, hl), x_f - x_R = (0, -hl)
        const float2 kyb = __fmul2_rn(p2(hl - dt, -hl + dt), p2(sL.ay, sR.ay));   // (A2, B4)
        v01 = extrap2<false, true>(s_fbp, LXY, 2, lL, sL, 4, lR, sR, p2(0.f, 0.f), kyb);
        const float kyL = (hl - dt) * sL.ay, kyR = (-hl + dt) * sR.ay;
        v23 = extrap2<true, true>(s_fbp, LXY, 5, lL, sL, 6, lL, sL, __fmul2_rn(p2(-dt, dt), p2(sL.ax, sL.ax)),
                            p2(kyL, kyL));                                                      // (A5, A6)
        v45 = extrap2<true, true>(s_fbp, LXY, 7, lR, sR, 8, lR, sR, __fmul2_rn(p2(dt, -dt), p2(sR.ax, sR.ax)),
                            p2(kyR, kyR));                                                      // (B7, B8)
        const float2 ky0 = __fmul2_rn(p2(hl, -hl), p2(sL.ay, sR.ay));
        const float2 ax2 = p2(sL.ax, sR.ax);
        const float2 t0 = extrap2<false, true>(s_fbp, LXY, 0, lL, sL, 0, lR, sR, p2(0.f, 0.f), ky0);        // (A0, B0)
        const float2 t1 = extrap2<true, true>(s_fbp, LXY, 1, lL, sL, 1, lR, sR, __fmul2_rn(p2(-dt, -dt), ax2), ky0);
        const float2 t3 = extrap2<true, true>(s_fbp, LXY, 3, lL, sL, 3, lR, sR, __fmul2_rn(p2(dt, dt), ax2), ky0);
        fbar[0] = 0.5f * (t0.x + t0.y); fbar[1] = 0.5f * (t1.x + t1.y); fbar[2] = v01.x;
        fbar[3] = 0.5f * (t3.x + t3.y); fbar[4] = v01.y; fbar[5] = v23.x; fbar[6] = v23.y;
        fbar[7] = v45.x; fbar[8] = v45.y;
    }
    // moments from the pairs: with d = (f5 - f7, f6 - f8), sum xi_x f = (f1 - f3) + d.x - d.y and
    // sum xi_y f = (f2 - f4) + d.x + d.y
    const float2 d57 = __ffma2_rn(v45, p2(-1.f, -1.f), v23), s57 = __fadd2_rn(v23, v45);
    const float t13 = AX == 0 ? v01.x - v01.y : fbar[1] - fbar[3];
    const float t24 = AX == 0 ? fbar[2] - fbar[4] : v01.x - v01.y;
    const float tan2 = AX == 0 ? fbar[2] + fbar[4] : fbar[1] + fbar[3];
    const float w0 = fbar[0] + (v01.x + v01.y) + tan2 + (s57.x + s57.y);
    const float w1 = t13 + (d57.x - d57.y);
    const float w2 = t24 + (d57.x + d57.y);
    // deviation form: w0 = sum of g = rho_b - 1
    float ux, uy, feqb[NQ];
    const float rb = 1.0f + w0;
    vel_of<float>(rb, w1, w2, ux, uy);
    feq9fd<float>(w0, rb, ux, uy, feqb);
    const float len = AX == 0 ? k.hy : k.hx;
    const float2 bb = p2(k.b, k.b), cc = p2(k.c, k.c);
    // slot pairs: AX 0 -> (1,3) (5,6) (7,8); AX 1 -> (2,4) (5,6) (7,8)
    const float2 s01 = p2(len, -len);
    const float2 s23 = AX == 0 ? p2(len, -len) : p2(len, len);
    const float2 s45 = AX == 0 ? p2(-len, len) : p2(-len, -len);
    const float2 e01 = AX == 0 ? p2(feqb[1], feqb[3]) : p2(feqb[2], feqb[4]);
    const float2 f01 = __fmul2_rn(s01, __fmul2_rn(__ffma2_rn(bb, e01, v01), cc));
    const float2 f23 = __fmul2_rn(s23, __fmul2_rn(__ffma2_rn(bb, p2(feqb[5], feqb[6]), v23), cc));
    const float2 f45 = __fmul2_rn(s45, __fmul2_rn(__ffma2_rn(bb, p2(feqb[7], feqb[8]), v45), cc));
    flux[0] = f01.x; flux[1] = f01.y; flux[2] = f23.x; flux[3] = f23.y; flux[4] = f45.x; flux[5] = f45.y;
}

// Boundary face of the own cell in direction D (0 +x, 1 -x, 2 +y, 3 -y) on grid side
// `side`: adds the outward flux (xi . n l) f_b of every crossing velocity to F
// (Sec. III rules).
// Diagnostic steps: the momentum (px, py) leaving the fluid through the boundary face
// at position pos (i on the bottom and top sides, j on the left and right) of a grid
// side, added to the side's total and written to the face's row.
__device__ __forceinline__ void cart_face_momentum(const CartInst &m, int side, int pos, double px, double py)
{
    if (m.force) {
        atomicAdd(&m.force[2 * side], px);
        atomicAdd(&m.force[2 * side + 1], py);
    }
    if (m.bface) {
        const int base = side == 0 ? 0 : side == 1 ? m.nx : side == 2 ? m.nx + m.ny : 2 * m.nx + m.ny;
        const int q = m.bidx[base + pos];
        if (q >= 0) {
            m.bface[2 * q] = px;
            m.bface[2 * q + 1] = py;
        }
    }
}

template <int D, class R, bool DIAG>
__device__ __forceinline__ void cart_boundary_face(R F[NQ], const R *s_fbp, int lme, const Sten<R> &st,
                                                   const CartInst &m, int side, int pos, const CartK<R> &k,
                                                   const R fn[NQ], const R feqn[NQ], R b0_n, R ux_n, R uy_n,
                                                   int LXY)
{
    constexpr bool DEV = sizeof(R) == 4;           // FP32 compute: deviation form
    // b0_n: the cell's rho - 1 (deviation form) or rho (FP64)
    const R rho_n = DEV ? R(1) + b0_n : b0_n, drho_n = b0_n;
    const R nx = D == 0 ? k.hy : (D == 1 ? -k.hy : R(0));
    const R ny = D == 2 ? k.hx : (D == 3 ? -k.hx : R(0));
    const R rx = D == 0 ? R(0.5) * k.hx : (D == 1 ? R(-0.5) * k.hx : R(0));
    const R ry = D == 2 ? R(0.5) * k.hy : (D == 3 ? R(-0.5) * k.hy : R(0));
    const int bk = m.side_kind[side];
    R rb = rho_n, drb = drho_n, ubx = R(0), uby = R(0);
    if (bk == BK_MOVING_WALL) { ubx = CartK<R>::par(m, side, 0); uby = CartK<R>::par(m, side, 1); }
    else if (bk == BK_FARFIELD) {
        rb = CartK<R>::par(m, side, 0); drb = CartK<R>::drho_par(m, side);
        ubx = CartK<R>::par(m, side, 1); uby = CartK<R>::par(m, side, 2);
    } else if (bk == BK_OUTLET) { ubx = ux_n; uby = uy_n; }
    R feqb[NQ];
    feq9fd<R>(DEV ? drb : rb, rb, ubx, uby, feqb);
    R px_ = R(0), py_ = R(0);
#define SDUGKS_BFACE_ALPHA(a)                                                                       \
    {                                                                                               \
        constexpr int sg = (D < 2) ? (D == 0 ? EX(a) : -EX(a)) : (D == 2 ? EY(a) : -EY(a));         \
        if (sg != 0) {                                                                              \
            const R s = xdot<R>(a, nx, ny);                                                         \
            R fb;                                                                                   \
            if (sg < 0) {                                                                           \
                fb = feqb[a] + (fn[a] - feqn[a]);   /* non-equilibrium extrapolation */             \
            } else {                                                                                \
                constexpr bool ux = D < 2 || EX(a) != 0, uy = D >= 2 || EY(a) != 0;                 \
                const R A = cart_extrap<a, ux, uy, R>(s_fbp, lme, st, rx - R(EX(a)) * k.dt, ry - R(EY(a)) * k.dt, LXY); \
                fb = (A + k.b * feqb[a]) * k.c;                                                     \
            }                                                                                       \
            F[a] += s * fb;                                                                         \
            px_ += R(EX(a)) * (s * fb);                                                             \
            py_ += R(EY(a)) * (s * fb);                                                             \
        }                                                                                           \
    }
    SDUGKS_BFACE_ALPHA(0) SDUGKS_BFACE_ALPHA(1) SDUGKS_BFACE_ALPHA(2) SDUGKS_BFACE_ALPHA(3) SDUGKS_BFACE_ALPHA(4)
    SDUGKS_BFACE_ALPHA(5) SDUGKS_BFACE_ALPHA(6) SDUGKS_BFACE_ALPHA(7) SDUGKS_BFACE_ALPHA(8)
#undef SDUGKS_BFACE_ALPHA
    if (DIAG && (m.force || m.bface)) {   // diagnostic steps only; in the deviation form the
                                          // rest equilibrium's momentum flux c_s^2 n l is added back
        constexpr double third = 1.0 / 3.0;
        const double rfx = DEV ? third * (D == 0 ? m.dy : (D == 1 ? -m.dy : 0.0)) : 0.0;
        const double rfy = DEV ? third * (D == 2 ? m.dx : (D == 3 ? -m.dx : 0.0)) : 0.0;
        cart_face_momentum(m, side, pos, to_f64<R>(px_) + rfx, to_f64<R>(py_) + rfy);
    }
}

// One TX x TY block (block coordinates tbx, tby) of one grid: reads buffer `par`,
// writes buffer 1 - par.  All threads of the CTA must call it (it synchronises).
// DIAG compiles in the optional wall-force accumulation.  INTERIOR: the block and its
// two-cell halo lie inside the grid (no side, wrap or ghost within reach), so every
// stencil is the central difference and every face of a cell is interior; the
// existence tests and stencil choices are compile-time constants.  BOX (interior
// blocks only): f^n and W^n of the staged block are read from the boxes a tensor copy
// has already brought into shared memory (box_f, box_w; CartTmaBox layout) instead of
// from global memory.
template <int P, int TX, int TY, bool DIAG, bool INTERIOR, bool BOX = false>
__device__ __forceinline__ void cart_tile(const CartInst &m, int par, int tbx, int tby, unsigned char *smem_raw,
                                          const typename Store<P>::T *box_f = nullptr, const double *box_w = nullptr)
{
    static_assert(!BOX || INTERIOR, "box staging covers interior blocks");
    using R = typename Store<P>::R;
    using T = typename Store<P>::T;
    using SP = Store<P>;
    using S = CartShape<TX, TY>;
    using B = CartTmaBox<P, TX, TY>;
    constexpr int LXY = S::PLANE;
    R *s_fbp = reinterpret_cast<R *>(smem_raw);     // [NQ][LY][SX]
    R *s_fx = s_fbp + NQ * LXY;                      // [6][NSX] fluxes through faces of constant x, by slot
    R *s_fy = s_fx + 6 * S::NSX;                     // [6][NSY] constant y

    const T *__restrict__ fin = static_cast<const T *>(m.f[par]);
    T *__restrict__ fout = static_cast<T *>(m.f[1 - par]);
    const double *__restrict__ Wn = m.W[par];
    double *__restrict__ Wout = m.W[1 - par];
    const int x0 = tbx * TX, y0 = tby * TY;
    const int tid = threadIdx.x;
    const int64_t np = m.npad, pitch = m.pitch;
    const int nx = m.nx, ny = m.ny;
    const bool px = m.periodic_x != 0, py = m.periodic_y != 0;
    const CartK<R> k(m);

    // Symmetry sides (Sec. III): beyond them sit mirror ghosts of the inner cells
    // (same fbar+ for the mirrored velocity), staged like any other position, so a
    // symmetry face is an ordinary face between a cell and its ghost.
    const bool symL = !px && m.side_kind[3] == BK_SYMMETRY, symR = !px && m.side_kind[1] == BK_SYMMETRY;
    const bool symB = !py && m.side_kind[0] == BK_SYMMETRY, symT = !py && m.side_kind[2] == BK_SYMMETRY;
    // a grid column / row exists (a domain cell, a periodic image or a mirror ghost)
    // iff it lies in [xlo, xhi) x [ylo, yhi)
    const int xlo = px ? INT_MIN : (symL ? -nx : 0), xhi = px ? INT_MAX : (symR ? 2 * nx : nx);
    const int ylo = py ? INT_MIN : (symB ? -ny : 0), yhi = py ? INT_MAX : (symT ? 2 * ny : ny);
    auto has_x = [&](int ci) { return INTERIOR || (ci >= xlo && ci < xhi); };
    auto has_y = [&](int cj) { return INTERIOR || (cj >= ylo && cj < yhi); };
    // domain cell of a block-relative position (periodic sides wrap, symmetry sides
    // reflect: mir bit 0 / 1 for a reflection in x / y), or -1 outside
    auto cell_of = [&](int bi, int bj, int &mir) -> int64_t {
        int gi = x0 + bi, gj = y0 + bj;
        mir = 0;
        if (INTERIOR) return gi + pitch * gj;
        if (gi < 0 || gi >= nx) {
            if (px) gi = (gi + nx) % nx;
            else if (gi < 0 ? symL : symR) {
                gi = gi < 0 ? -1 - gi : 2 * nx - 1 - gi;
                mir |= 1;
                if (gi < 0 || gi >= nx) return -1;
            } else return -1;
        }
        if (gj < 0 || gj >= ny) {
            if (py) gj = (gj + ny) % ny;
            else if (gj < 0 ? symB : symT) {
                gj = gj < 0 ? -1 - gj : 2 * ny - 1 - gj;
                mir |= 2;
                if (gj < 0 || gj >= ny) return -1;
            } else return -1;
        }
        return gi + pitch * gj;
    };
    // gradient stencil of the staged cell at block position (bi, bj)
    auto sten = [&](int bi, int bj) {
        if (INTERIOR) return Sten<R>{1, -1, S::SX, -S::SX, R(0.5) * k.ihx, R(0.5) * k.ihy};
        const int ci = x0 + bi, cj = y0 + bj;
        const bool hE = has_x(ci + 1), hW = has_x(ci - 1);
        const bool hN = has_y(cj + 1), hS = has_y(cj - 1);
        Sten<R> st;
        st.oE = hE ? 1 : 0; st.oW = hW ? -1 : 0; st.oN = hN ? S::SX : 0; st.oS = hS ? -S::SX : 0;
        st.ax = (hE && hW) ? R(0.5) * k.ihx : k.ihx;
        st.ay = (hN && hS) ? R(0.5) * k.ihy : k.ihy;
        return st;
    };
    constexpr bool DEV = Dev<P>::ON;      // FP32 compute: g = f - w, W[0] = rho - 1
    auto macro = [&](double w0, double w1, double w2, R &drho, R &rho, R &ux, R &uy) {
        macro_of<R>(w0, w1, w2, drho, rho, ux, uy);
    };

    // ---- phase 1: fbar+ = a f^n + b feq(W^n) of every staged position, one round.
    // The cell slots (threads 0 .. 32 WX - 1) take the block (their own cell, kept in
    // registers), the next LX LY - NT threads the two-cell ring.
    const int ti = tid & 15, tj = slot_row(tid);
    const bool cell_thread = tid < 32 * S::WX && tj < TY;
    const int gi = x0 + ti, gj = y0 + tj;
    const bool active = cell_thread && gi < nx && gj < ny;
    const int64_t g = (int64_t)gi + pitch * gj;
    const int lme = (tj + 2) * S::SX + (ti + 2);
    R fn[NQ];
    R b0_n = DEV ? R(0) : R(1), ux_n = R(0), uy_n = R(0);   // b0_n: rho - 1 (deviation form) or rho (FP64)
    double w0n = 1.0 - rho_ref<P>(), w1n = 0.0, w2n = 0.0;
    {
        int64_t gs = -1;
        int ls = 0, mir = 0, li = 0, lj = 0;
        if (cell_thread) {
            ls = lme;
            li = ti + 2; lj = tj + 2;
            gs = active ? g : cell_of(ti, tj, mir);     // past the grid edge: a wrapped cell, a ghost or none
        } else if (tid >= 32 * S::WX && tid < 32 * S::WX + S::LX * S::LY - S::NT) {
            // ring position r: two rows below, two above, then two columns left and right
            const int r = tid - 32 * S::WX;
            if (r < 2 * S::LX) { li = r % S::LX; lj = r / S::LX; }
            else if (r < 4 * S::LX) { li = (r - 2 * S::LX) % S::LX; lj = S::LY - 2 + (r - 2 * S::LX) / S::LX; }
            else { const int q = r - 4 * S::LX; lj = 2 + q / 4; const int cc = q % 4; li = cc < 2 ? cc : S::LX - 4 + cc; }
            ls = lj * S::SX + li;
            gs = cell_of(li - 2, lj - 2, mir);
        }
        if (gs >= 0) {
            double a0, a1, a2;
            R rho, ux, uy, fe[NQ], fv[NQ];
            if constexpr (BOX) {
                const double *w = box_w + lj * B::WBW + li;
                a0 = w[0]; a1 = w[S::LY * B::WBW]; a2 = w[2 * S::LY * B::WBW];
                const T *fb = box_f + lj * B::BW + li + (B::OFF - 2);
#pragma unroll
                for (int a = 0; a < NQ; a++) fv[a] = SP::dec(fb[a * S::LY * B::BW], R(0), a);
            } else {
                a0 = Wn[gs]; a1 = Wn[np + gs]; a2 = Wn[2 * np + gs];
#pragma unroll
                for (int a = 0; a < NQ; a++) fv[a] = SP::dec(fin[a * np + gs], R(0), a);
            }
            R drho;
            macro(a0, a1, a2, drho, rho, ux, uy);
            feq9fd<R>(DEV ? drho : rho, rho, ux, uy, fe);
#pragma unroll
            for (int a = 0; a < NQ; a++)
                if constexpr (P == P_BF16DEV || P == P_FP16DEV) fv[a] += fe[a];       // decode the deviation
            if (mir == 0) {
                if constexpr (P == P_FP64) {
#pragma unroll
                    for (int a = 0; a < NQ; a++) s_fbp[a * LXY + ls] = k.a * fv[a] + k.b * fe[a];
                } else {
                    // paired: a f + b feq for the velocity pairs (1,2) (3,4) (5,6) (7,8)
                    const float2 kb2 = make_float2(k.b, k.b), ka2 = make_float2(k.a, k.a);
                    s_fbp[ls] = k.a * fv[0] + k.b * fe[0];
#pragma unroll
                    for (int a = 1; a < NQ; a += 2) {
                        const float2 v = __ffma2_rn(ka2, make_float2(fv[a], fv[a + 1]),
                                                    __fmul2_rn(kb2, make_float2(fe[a], fe[a + 1])));
                        s_fbp[a * LXY + ls] = v.x;
                        s_fbp[(a + 1) * LXY + ls] = v.y;
                    }
                }
            } else {
                // mirror ghost: fbar+ of the mirrored velocity
                R fb[NQ];
#pragma unroll
                for (int a = 0; a < NQ; a++) fb[a] = k.a * fv[a] + k.b * fe[a];
#pragma unroll
                for (int a = 0; a < NQ; a++)
                    s_fbp[a * LXY + ls] = mir == 1 ? fb[MIRROR_X(a)] : (mir == 2 ? fb[MIRROR_Y(a)] : fb[MIRROR_X(MIRROR_Y(a))]);
            }
            if (active) {
#pragma unroll
                for (int a = 0; a < NQ; a++) fn[a] = fv[a];
                b0_n = DEV ? drho : rho; ux_n = ux; uy_n = uy;
                w0n = a0; w1n = a1; w2n = a2;
            }
        }
    }
    __syncthreads();

    // ---- phase 2: every interior face of the block once, one per thread.  Faces of
    // constant x: slot s < 32 WX is the face left of block cell (s % 16, row of s); the TY
    // faces on the right edge take slots 32 WX + row.
    // A constant-x face between block columns fi-1 (L) and fi (R) in row fj:
    auto x_face = [&](int fi, int fj, int slot) {
        if (has_x(x0 + fi - 1) && has_x(x0 + fi) && has_y(y0 + fj)) {
            const int lL = (fj + 2) * S::SX + (fi + 1);
            R fl[6];
            if constexpr (P == P_FP64) cart_interior_face<0, R>(fl, s_fbp, lL, lL + 1, sten(fi - 1, fj), sten(fi, fj), k, LXY);
            else cart_interior_face_f32x2<0>(fl, s_fbp, lL, lL + 1, sten(fi - 1, fj), sten(fi, fj), k, LXY);
#pragma unroll
            for (int r = 0; r < 6; r++) s_fx[r * S::NSX + slot] = fl[r];
        }
    };
    // where the right-edge faces go: when TY = 2 (mod 4) the upper half of constant-x
    // warp WX - 2 holds no row, and they run there with the same code as the rest of the
    // warp; otherwise in the free upper half of the last constant-y warp
    constexpr bool EDGE_IN_X = TY % 4 == 2;
    if (tid < 32 * S::WX) {
        if (tj < TY) x_face(ti, tj, tid);
        else if (EDGE_IN_X && (tid >> 5) == S::WX - 2 && ti < TY) x_face(TX, ti, 32 * S::WX + ti);
    } else if (tid < 32 * (S::WX + S::WY)) {
        // face of constant y between block rows fj-1 (below) and fj (above), column fi
        const int qq = tid - 32 * S::WX, fi = qq & 15, fj = slot_row(qq);
        if (fj <= TY) {
            if (has_y(y0 + fj - 1) && has_y(y0 + fj) && has_x(x0 + fi)) {
                const int lB = (fj + 1) * S::SX + (fi + 2);
                R fl[6];
                if constexpr (P == P_FP64) cart_interior_face<1, R>(fl, s_fbp, lB, lB + S::SX, sten(fi, fj - 1), sten(fi, fj), k, LXY);
                else cart_interior_face_f32x2<1>(fl, s_fbp, lB, lB + S::SX, sten(fi, fj - 1), sten(fi, fj), k, LXY);
#pragma unroll
                for (int r = 0; r < 6; r++) s_fy[r * S::NSY + qq] = fl[r];
            }
        } else if (!EDGE_IN_X && (qq >> 5) == S::WY - 1 && fi < TY) {
            x_face(TX, fi, 32 * S::WX + fi);           // right edge of the block, row fi
        }
    }
    __syncthreads();

    if (active) {
        // ---- phase 3: flux sum over the own cell's faces (order -x, +x, -y, +y)
        R F[NQ];
#pragma unroll
        for (int a = 0; a < NQ; a++) F[a] = R(0);
        // face slots: left = own slot, right = next slot (or the right-edge slot of the
        // row), below / above by row_slot
        const int fW = tid, fE = ti + 1 < TX ? tid + 1 : 32 * S::WX + tj;
        const int fS = row_slot(tj, ti), fN = row_slot(tj + 1, ti);
        const bool inW = has_x(gi - 1), inE = has_x(gi + 1);
        const bool inS = has_y(gj - 1), inN = has_y(gj + 1);
        R feqn[NQ];
        if (!(inW && inE && inS && inN)) feq9fd<R>(b0_n, DEV ? R(1) + b0_n : b0_n, ux_n, uy_n, feqn);   // boundary cells only
        if (inW) {
#pragma unroll
            for (int r = 0; r < 6; r++) F[XSLOT_A(r)] -= s_fx[r * S::NSX + fW];
        } else {
            cart_boundary_face<1, R, DIAG>(F, s_fbp, lme, sten(ti, tj), m, 3, gj, k, fn, feqn, b0_n, ux_n, uy_n, LXY);
        }
        if (inE) {
#pragma unroll
            for (int r = 0; r < 6; r++) F[XSLOT_A(r)] += s_fx[r * S::NSX + fE];
        } else {
            cart_boundary_face<0, R, DIAG>(F, s_fbp, lme, sten(ti, tj), m, 1, gj, k, fn, feqn, b0_n, ux_n, uy_n, LXY);
        }
        if (inS) {
#pragma unroll
            for (int r = 0; r < 6; r++) F[YSLOT_A(r)] -= s_fy[r * S::NSY + fS];
        } else {
            cart_boundary_face<3, R, DIAG>(F, s_fbp, lme, sten(ti, tj), m, 0, gi, k, fn, feqn, b0_n, ux_n, uy_n, LXY);
        }
        if (inN) {
#pragma unroll
            for (int r = 0; r < 6; r++) F[YSLOT_A(r)] += s_fy[r * S::NSY + fN];
        } else {
            cart_boundary_face<2, R, DIAG>(F, s_fbp, lme, sten(ti, tj), m, 2, gi, k, fn, feqn, b0_n, ux_n, uy_n, LXY);
        }

        if (DIAG && (m.force || m.bface)) {
            // symmetry sides are staged as mirror ghosts, so their faces are interior
            // faces here: the momentum leaving the fluid through one is that face's flux
            // moment (fluxes are oriented along +x / +y), with the outward sign
            auto sym_face = [&](int side, int pos, const R *fl, int stride, bool y_face, R sgn) {
                R px_ = R(0), py_ = R(0);
#pragma unroll
                for (int r = 0; r < 6; r++) {
                    const int a = y_face ? YSLOT_A(r) : XSLOT_A(r);
                    px_ += R(EX(a)) * fl[r * stride];
                    py_ += R(EY(a)) * fl[r * stride];
                }
                // deviation form: plus the rest equilibrium's flux c_s^2 n l (n out of the fluid)
                const double rf = DEV ? (1.0 / 3.0) * (double)sgn * (y_face ? m.dx : m.dy) : 0.0;
                cart_face_momentum(m, side, pos, to_f64<R>(sgn * px_) + (y_face ? 0.0 : rf),
                                   to_f64<R>(sgn * py_) + (y_face ? rf : 0.0));
            };
            if (symL && gi == 0) sym_face(3, gj, s_fx + fW, S::NSX, false, R(-1));
            if (symR && gi == nx - 1) sym_face(1, gj, s_fx + fE, S::NSX, false, R(1));
            if (symB && gj == 0) sym_face(0, gi, s_fy + fS, S::NSY, true, R(-1));
            if (symT && gj == ny - 1) sym_face(2, gi, s_fy + fN, S::NSY, true, R(1));
        }

        // ---- macroscopic flux -> W^{n+1} (FP64); cell update f^{n+1} (Eq. fn+1)
        R M0 = R(0), M1 = R(0), M2 = R(0);
        if constexpr (P == P_FP64) {
#pragma unroll
            for (int a = 0; a < NQ; a++) {
                M0 += F[a];
                if (EX(a) == 1) M1 += F[a]; else if (EX(a) == -1) M1 -= F[a];
                if (EY(a) == 1) M2 += F[a]; else if (EY(a) == -1) M2 -= F[a];
            }
        } else {
            // paired: sum xi_x F = (F1 - F3) + (F5 - F7) - (F6 - F8), sum xi_y F = (F2 - F4) + (F5 - F7) + (F6 - F8)
            const float2 m1 = p2(-1.f, -1.f);
            const float2 q1 = p2(F[1], F[2]), q3 = p2(F[3], F[4]), q5 = p2(F[5], F[6]), q7 = p2(F[7], F[8]);
            const float2 sm = __fadd2_rn(__fadd2_rn(q1, q3), __fadd2_rn(q5, q7));
            const float2 d13 = __ffma2_rn(q3, m1, q1), d57 = __ffma2_rn(q7, m1, q5);
            M0 = F[0] + (sm.x + sm.y);
            M1 = d13.x + (d57.x - d57.y);
            M2 = d13.y + (d57.x + d57.y);
        }
        const R d0 = k.dtV * M0, d1 = k.dtV * M1, d2 = k.dtV * M2;
        const double W0 = w0n - to_f64<R>(d0), W1 = w1n - to_f64<R>(d1), W2 = w2n - to_f64<R>(d2);
        // FP32 compute: the FP64 sums are stored last, after the f update, which does not
        // wait for them (the FP64 unit of this GPU is narrow)
        if constexpr (P == P_FP64) {
            Wout[g] = W0;
            Wout[np + g] = W1;
            Wout[2 * np + g] = W2;
        }
        R rho1, ux1, uy1, feq1[NQ];
        if constexpr (P == P_FP64) {
            rho1 = W0;
            vel_of<R>(W0, W1, W2, ux1, uy1);
            feq9f<R>(rho1, ux1, uy1, feq1);
        } else {
            const R drho1 = b0_n - d0;
            rho1 = R(1) + drho1;
            vel_of<R>(rho1, from_f64<R>(w1n) - d1, from_f64<R>(w2n) - d2, ux1, uy1);
            feq9fd<R>(drho1, rho1, ux1, uy1, feq1);
        }
        if constexpr (P == P_FP64) {
#pragma unroll
            for (int a = 0; a < NQ; a++)
                fout[a * np + g] = SP::enc((fn[a] - k.dtV * F[a] + k.r * feq1[a]) / (R(1) + k.r), feq1[a], a);
        } else {
            // paired: (f - dt/V F + r feq) / (1 + r) for the velocity pairs
            const float2 mdv = make_float2(-k.dtV, -k.dtV), r2 = make_float2(k.r, k.r);
            const float2 i2 = make_float2(m.finv1r, m.finv1r);
            fout[g] = SP::enc((fn[0] - k.dtV * F[0] + k.r * feq1[0]) * m.finv1r, feq1[0], 0);
#pragma unroll
            for (int a = 1; a < NQ; a += 2) {
                const float2 t = __ffma2_rn(mdv, make_float2(F[a], F[a + 1]), make_float2(fn[a], fn[a + 1]));
                const float2 v = __fmul2_rn(__ffma2_rn(r2, make_float2(feq1[a], feq1[a + 1]), t), i2);
                fout[a * np + g] = SP::enc(v.x, feq1[a], a);
                fout[(a + 1) * np + g] = SP::enc(v.y, feq1[a + 1], a + 1);
            }
            Wout[g] = W0;
            Wout[np + g] = W1;
            Wout[2 * np + g] = W2;
        }
    }
}

// The block and its two-cell halo lie inside the grid.
template <int TX, int TY>
__device__ __forceinline__ bool cart_block_interior(const CartInst &m, int tbx, int tby)
{
    const int x0 = tbx * TX, y0 = tby * TY;
    return x0 >= 2 && x0 + TX + 2 <= m.nx && y0 >= 2 && y0 + TY + 2 <= m.ny;
}

// 128-byte aligned start of the dynamic shared memory (the allocation has 128 bytes of
// slack) and its shared-space address
__device__ __forceinline__ unsigned char *aligned_smem(unsigned char *raw, uint32_t &sa)
{
    const uint32_t r = (uint32_t)__cvta_generic_to_shared(raw);
    sa = (r + 127u) & ~127u;
    return raw + (sa - r);
}

// Every thread waits for the barrier phase, up to the solver's limit; false (for the
// whole CTA) if any thread gave up.  Then the error flag is set (the host treats the
// whole launch as failed) and thread 0 waits, up to TMA_WAIT_NS, for the copies to
// land, so that the CTA's shared memory is not released while a copy still writes to it;
// the other threads may exit meanwhile (the CTA's shared memory lives until its last
// thread exits).  If that second wait gives up too, nothing more can be done: the copy
// is reported but may still land after the CTA has exited.
__device__ __forceinline__ bool cta_wait_staged(const CartInst &m, uint32_t bar, uint32_t parity)
{
    const bool ok = mbar_wait_bounded(bar, parity, m.tma_wait_ns);
    if (__syncthreads_or(!ok)) {
        if (threadIdx.x == 0) {
            if (m.err) atomicExch(m.err, 1);
            mbar_wait_bounded(bar, parity, TMA_WAIT_NS);
        }
        return false;
    }
    return true;
}

// One block per CTA.  MODE (CartMode): CART_SPECIALISED runs interior blocks with the
// compile-time interior variant of cart_tile and the others with the general one;
// CART_SPECIALISED_TMA does the same with the interior blocks staged by two tensor copies
// (tf, tw: the maps of buffer par) into boxes that overlay the face-flux arrays;
// CART_GENERAL runs every block with the general variant.  One code path serves a grid
// whose blocks all run in one wave better, where the slowest (edge) blocks set the time:
// there the edge blocks' general code is not displaced by the interior variant's.
// DIAG: the diagnostic step (CART_GENERAL only), which also reports the momentum leaving
// the fluid through the boundary faces; ordinary steps carry none of that code.
enum CartMode { CART_SPECIALISED = 0, CART_SPECIALISED_TMA = 1, CART_GENERAL = 2 };

template <int P, int TX, int TY, int MODE, bool DIAG = false>
__global__ void __launch_bounds__(cart_threads<TX, TY>(), P == P_FP64 ? 1 : (cart_threads<TX, TY>() <= 320 ? 4 : 2))
k_step_cart(const CartInst m, int par, const __grid_constant__ CUtensorMap tf, const __grid_constant__ CUtensorMap tw)
{
    static_assert(!DIAG || MODE == CART_GENERAL, "diagnostic steps run every block on the general variant");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    step_dependency_wait();
    const int tbx = blockIdx.x, tby = blockIdx.y;     // a two-dimensional grid of blocks
    if (MODE != CART_GENERAL && cart_block_interior<TX, TY>(m, tbx, tby)) {
        if constexpr (MODE == CART_SPECIALISED_TMA) {
            using B = CartTmaBox<P, TX, TY>;
            uint32_t sa;
            unsigned char *sm = aligned_smem(smem_raw, sa);
            const uint32_t bar = sa + (uint32_t)B::BAR_OFF;
            if (threadIdx.x == 0) mbar_init(bar);
            __syncthreads();
            if (threadIdx.x == 0)
                tma_issue_block<P, TX, TY>(bar, sa + (uint32_t)B::F_OFF, sa + (uint32_t)B::W_OFF, &tf, &tw, tbx * TX, tby * TY);
            if (!cta_wait_staged(m, bar, 0)) return;
            cart_tile<P, TX, TY, false, true, true>(m, par, tbx, tby, sm,
                                                    reinterpret_cast<const typename Store<P>::T *>(sm + B::F_OFF),
                                                    reinterpret_cast<const double *>(sm + B::W_OFF));
        } else {
            cart_tile<P, TX, TY, false, true>(m, par, tbx, tby, smem_raw);
        }
    } else {
        cart_tile<P, TX, TY, DIAG, false>(m, par, tbx, tby, smem_raw);
    }
}

template <int P, int TX, int TY, int MODE, bool DIAG = false> constexpr size_t cart_step_smem() {
    return MODE == CART_SPECIALISED_TMA ? CartTmaBox<P, TX, TY>::SMEM : cart_smem<P, TX, TY>();
}

template <int P, int TX, int TY, int MODE, bool DIAG = false> cudaError_t prepare_mode_p() {
    return cudaFuncSetAttribute(k_step_cart<P, TX, TY, MODE, DIAG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)cart_step_smem<P, TX, TY, MODE>());
}

template <int P, int TX, int TY> cudaError_t prepare_cart_p() {
    cudaError_t e = prepare_mode_p<P, TX, TY, CART_SPECIALISED>();
    if (e == cudaSuccess) e = prepare_mode_p<P, TX, TY, CART_SPECIALISED_TMA>();
    if (e == cudaSuccess) e = prepare_mode_p<P, TX, TY, CART_GENERAL>();
    if (e == cudaSuccess) e = prepare_mode_p<P, TX, TY, CART_GENERAL, true>();
    return e;
}

// tma: the maps for TMA staging (nullptr: plain loads); general: every block on the
// general path (ignored with TMA staging).  A diagnostic step (m.force or m.bface set)
// runs the diagnostic instance, every block on the general path with plain loads.
template <int P, int TX, int TY>
cudaError_t launch_cart_p(const CartInst &m, const CartTma *tma, bool general, int par, cudaStream_t st)
{
    const int ntx = (m.nx + TX - 1) / TX, nty = (m.ny + TY - 1) / TY;
    const dim3 grid(ntx, nty), block(cart_threads<TX, TY>());
    static const CUtensorMap none0{};
    if (m.force || m.bface)
        return launch_step_kernel(k_step_cart<P, TX, TY, CART_GENERAL, true>, grid, block,
                                  cart_step_smem<P, TX, TY, CART_GENERAL>(), st, m, par, none0, none0);
    if (tma)
        return launch_step_kernel(k_step_cart<P, TX, TY, CART_SPECIALISED_TMA>, grid, block,
                                  cart_step_smem<P, TX, TY, CART_SPECIALISED_TMA>(), st, m, par, tma->f[par], tma->W[par]);
    static const CUtensorMap none{};
    if (general)
        return launch_step_kernel(k_step_cart<P, TX, TY, CART_GENERAL>, grid, block,
                                  cart_step_smem<P, TX, TY, CART_GENERAL>(), st, m, par, none, none);
    return launch_step_kernel(k_step_cart<P, TX, TY, CART_SPECIALISED>, grid, block,
                              cart_step_smem<P, TX, TY, CART_SPECIALISED>(), st, m, par, none, none);
}

template <int P, int TX, int TY, int MODE> int occ_cart_p()
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step_cart<P, TX, TY, MODE>, cart_threads<TX, TY>(),
                                                      cart_step_smem<P, TX, TY, MODE>()) != cudaSuccess || n < 1)
        return 1;
    return n;
}

}  // namespace sdugks
