// sdugks_internal.h -- launch interface between the host library (sdugks_host.cpp)
// and the CUDA translation units.  Plain structs of device pointers and sizes.
#pragma once
#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

namespace sdugks {

constexpr int NQ = 9;
constexpr int MAXF = 4;         // faces per cell (quads and triangles)
constexpr int MAXPATCH = 64;    // boundary patches
constexpr uint16_t NO_LOCAL = 0xFFFF;
// LLSR neighbour codes of a symmetry slot: the mirror image of the cell itself in a
// line of constant x (SYM_X) or constant y (SYM_Y)
constexpr uint16_t SYM_X = 0xFFFD, SYM_Y = 0xFFFE;

// Tiled kernel shape: one CTA per tile of up to TILE_MAX cells.
constexpr int TILE_MAX = 128;   // interior cells per tile
constexpr int TILED_THREADS = 256;
constexpr int LOC_MAX = 416;    // interior + two halo rings
constexpr int SIG_MAX = 272;    // interior + first halo ring (cells whose gradient is needed)
constexpr int LF_MAX = 320;     // faces with at least one interior cell of the tile

enum Prec : int32_t { P_FP64 = 0, P_FP32 = 1, P_BF16DEV = 2, P_FP16DEV = 3 };

enum BcKind : int32_t { BK_UNSET = 0, BK_PERIODIC = 1, BK_WALL = 2, BK_MOVING_WALL = 3,
                        BK_FARFIELD = 4, BK_OUTLET = 5, BK_SYMMETRY = 6 };

// Scalars of one step (host-computed in FP64 from tau and dt; FP32 copies for the
// FP32-compute kernels so that no thread converts them).
struct Coefs {
    double a_plus;   // (2 tau - dt) / (2 tau)
    double b_plus;   // dt / (2 tau)
    double c_face;   // 2 tau / (2 tau + dt)
    double r;        // dt / tau
    double inv1r;    // 1 / (1 + dt / tau)
    double dt;
    double tie;      // |xi . n l| <= tie counts as tangential
    float fa_plus, fb_plus, fc_face, fr, finv1r, fdt, ftie, fpad_;
    int32_t bc_kind[MAXPATCH];
    double bc_par[MAXPATCH][3];
    float fbc_par[MAXPATCH][3];
    float fbc_drho[MAXPATCH];     // rho_inf - 1 of far-field patches (FP32 compute works with rho - 1)
};

// Slot kinds of a cell's faces (slots in ascending face id).
constexpr uint8_t SK_NONE = 0xFE;      // cell has fewer faces than MAXF
constexpr uint8_t SK_INTERIOR = 0xFF;  // face shared with another cell (periodic pairs included)
                                       // any other value: boundary patch id

// Unstructured tiled mesh on the device.  Cells are in internal (tile-contiguous)
// order; arrays indexed by cell are padded to npad.  Each tile lists the faces that
// touch its interior cells ("local faces", evaluated once per tile), oriented from
// their first side (the face owner) to the second.
struct TiledMesh {
    int32_t n_tiles;
    int64_t n, npad;
    int64_t n_lf;             // local faces of all tiles with the padding (stride of lf_geo, a multiple of 4)
    const int32_t *tile_c0;   // [n_tiles+1] interior cell range of each tile
    const int32_t *tile_h0;   // [n_tiles+1] range into halo
    const int32_t *tile_nh1;  // [n_tiles]   cells of ring 1 (first in the tile's halo)
    const int32_t *tile_s0;   // [n_tiles+1] range into sig_nb (each tile's rows padded to a multiple of 4)
    const int32_t *tile_f0;   // [n_tiles+1] first local face of each tile, a multiple of 4 (the
                              //   ranges are padded so that each starts 16-byte aligned)
    const int32_t *tile_nlf;  // [n_tiles] local faces of each tile (the rest of its range is padding)
    const int32_t *halo;      // internal ids of ring 1 then ring 2 of each tile
    int64_t n_sig;            // gradient rows of all tiles (stride of sig_d and sig_ai)
    const uint16_t *sig_nb;   // [n_sig][MAXF] tile-local index of the cell across each slot
    const void *sig_d;        // [MAXF][2][n_sig] x_k - x_j across each slot of each gradient row
    const void *sig_ai;       // [3][n_sig] LLSR inverse (xx, xy, yy) of each gradient row
    const uint16_t *cell_lf;  // [MAXF][npad] local face of each slot, | LF_SECOND when the cell
                              //   is the face's second side; LF_NONE for no face
    const uint32_t *lf_ab;    // [n_lf] tile-local first side | second side << 16; a boundary
                              //   face's second side is LF_BOUNDARY | patch
    const void *lf_geo;       // [6][n_lf] n l from the first side to the second (2),
                              //   x_f - x_first (2), x_f - x_second (2)
    const void *dtV;          // [npad] dt / V (compute precision)
    const double *vol;        // [npad] V
    double *force;            // nullptr, or [MAXPATCH][2]: momentum flux out of the fluid per boundary patch
    const int32_t *lf_bface;  // [n_lf] boundary-face row of each local face (-1: interior or periodic)
    double *bface;            // nullptr, or [n_bfaces][2]: momentum flux out of the fluid per boundary face
};
constexpr uint16_t LF_SECOND = 0x8000, LF_NONE = 0xFFFF;
constexpr uint32_t LF_BOUNDARY = 0xC000;

// One uniform-grid solve as the Cartesian kernels see it: nx x ny rectangles
// dx x dy, cell (i, j) at i + pitch j; side boundary rules; step coefficients; and
// its ping-pong state f[2] ([NQ][npad]), W[2] ([3][npad] FP64).  Buffer p holds
// t_n when the launch parity is p.
struct CartInst {
    int32_t nx, ny, pitch, periodic_x, periodic_y;
    int32_t side_kind[4];     // BK_* of the bottom, right, top, left side (unused if periodic)
    int32_t item0, n_items;   // batched runs: this instance's range in the work list
    int64_t npad;             // >= pitch * ny, multiple of 32
    double dx, dy, dtV;       // dtV = dt / (dx dy)
    double ihx, ihy;          // 1 / dx, 1 / dy
    double a, b, c, r, dt;    // (2tau-dt)/2tau, dt/2tau, 2tau/(2tau+dt), dt/tau, dt
    double side_par[4][3];
    float fdx, fdy, fdtV, fa, fb, fc, fr, finv1r, fdt, fihx, fihy;
    float fside_par[4][3];
    float fside_drho[4];      // rho_inf - 1 of far-field sides (FP32 compute works with rho - 1)
    void *f[2];
    double *W[2];
    double *snap;             // [2][npad] residual snapshot (U0, V0)
    double *force;            // nullptr, or [4][2]: momentum flux out of the fluid per grid side
    int32_t *err;             // nullptr, or a device flag set to 1 when a bounded staging wait gave up
    uint64_t tma_wait_ns;     // TMA staging: wait limit of a block's copies (0: give up at once)
    const int32_t *bidx;      // [2 (nx + ny)] boundary-face row of each side face: bottom (by i), right
                              //   (by j), top (by i), left (by j); -1 on periodic sides
    double *bface;            // nullptr, or [n_bfaces][2]: momentum flux out of the fluid per boundary face
};

// Device state of one solver, ping-pong: f [2][NQ][npad] (element type by
// precision), W [2][3][npad] FP64.
struct State {
    void *f[2];
    double *W[2];
};

// fused step kernels (k_step_fp64.cu, k_step_fp32.cu); prepare_* sets the kernel
// attributes on the current device and is called once per solver creation
cudaError_t prepare_tiled_fp64();
cudaError_t launch_step_tiled_fp64(const TiledMesh &m, const Coefs &c, const void *f_in, void *f_out,
                                   const double *W_in, double *W_out, cudaStream_t st);
cudaError_t prepare_tiled_fp32(int prec);
cudaError_t prepare_cart(int prec);
// block shapes of the Cartesian kernel: 0 = 16x16, 1 = 16x14, 2 = 16x8 (FP64: 16x16 only)
constexpr int CART_SHAPES = 3;
// block of the batched kernel: 16 x BATCH_TY cells per (instance, block) work item (the
// 16x8 shape fits four CTAs per SM, the fastest shape of the single-solve kernel on
// grids of many waves)
constexpr int BATCH_TY = 8;
constexpr int CART_TY[CART_SHAPES] = {16, 14, 8};
// Tensor maps of one Cartesian state for the TMA staging of interior blocks:
// f[b] views f buffer b as (x, y, velocity), W[b] views W buffer b as (x, y, component);
// the boxes are the block with its two-cell halo, widened in x to 16-byte boundaries.
struct CartTma {
    CUtensorMap f[2], W[2];
};
cudaError_t make_cart_tma(int prec, int shape, const CartInst &m, CartTma &out);
// tma: nullptr stages every block with plain loads; general: every block on the general
// code path (no interior variant; ignored with TMA staging)
cudaError_t launch_step_cart(int prec, int shape, const CartInst &m, const CartTma *tma, bool general, int parity,
                             cudaStream_t st);
int cart_shape_occupancy(int prec, int shape, bool tma);   // resident CTAs per SM
// batched: every (instance, tile) item of the list, one per CTA (per_item: grid >= the
// item count) or grid-stride over a fixed grid
cudaError_t prepare_batch(int prec);
cudaError_t launch_step_batch(int prec, const CartInst *insts, const int2 *items, const int *n_items, int grid,
                              bool per_item, int parity, cudaStream_t st);
int batch_ctas_per_sm(int prec);
// batched residual: partial [max_items][4] per tile, out [n_inst][4] = (num, den, mass, non-finite)
cudaError_t launch_batch_residual(const CartInst *insts, int n_inst, const int2 *items, const int *n_items, int grid,
                                  int parity, double *partial, double *out, cudaStream_t st);
cudaError_t launch_batch_init(int prec, const CartInst *inst_host, const CartInst *inst_dev, int parity,
                              const double *rho, const double *u, cudaStream_t st);
cudaError_t launch_batch_macros(const CartInst *inst_host, const CartInst *inst_dev, int parity, double *rho, double *u,
                                cudaStream_t st);
cudaError_t launch_step_tiled_fp32(int prec, const TiledMesh &m, const Coefs &c, const void *f_in, void *f_out,
                                   const double *W_in, double *W_out, cudaStream_t st);

// Programmatic dependent launch of the step kernels: each step kernel lets the next
// launch in its stream be scheduled as soon as all of its CTAs are running
// (griddepcontrol.launch_dependents) and, before it touches memory that a step
// writes, waits until the previous grid has completed and its writes are visible
// (griddepcontrol.wait; a no-op when the launch did not allow an early start); what
// only the host writes (mesh data, work items) may be read before the wait.  The
// next step's CTAs therefore take the SM slots the moment the current step's CTAs
// retire, instead of after the launch latency.
#ifdef __CUDACC__
__device__ __forceinline__ void step_dependency_wait()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

template <class... P, class... A>
cudaError_t launch_step_kernel(void (*kernel)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, A &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<A &&>(args)...);
}
#endif

// Rarefied solver on a discrete velocity grid (Q nodes): any face-based mesh, f and
// the scratch arrays cell- (or face-) major with the Q velocities contiguous.
struct DvmMesh {
    int64_t nc, nf, Q;
    const int32_t *cell_face;  // [nc][MAXF] face id, | DVM_SECOND when the cell is the face's
                               //   second side; -1 for no face
    const int32_t *cell_nb;    // [nc][MAXF] LLSR neighbour (periodic partners included), -1 none
    const void *cell_d;        // [nc][MAXF][2] x_k - x_j (compute precision)
    const void *ainv;          // [nc][3] LLSR inverse (xx, xy, yy)
    const double *dtV;         // [nc] dt / V
    const int32_t *face_own, *face_nbr;   // face_nbr: cell, or -1 - patch
    const void *face_geo;      // [nf][6] n l (first -> second side), x_f - x_first, x_f - x_second
    // velocity q = j + nv i (x fastest) sits at (vnode[j], vnode[i]) with weight w_node
    const void *vnode;         // [nv] nodes of one axis (compute precision)
    int32_t nv;
    double w_node;
};
constexpr int32_t DVM_SECOND = int32_t(0x40000000);
constexpr int DVM_THREADS = 256;
// one step; fbp_ready: fbp already holds this step's fbar+ (left there by the previous
// step's cell kernel), else it is formed first.  The step leaves the next step's fbar+ in fbp.
cudaError_t launch_dvm_step(int prec, const DvmMesh &m, const Coefs &c, double RTw, void *f, double *W, void *fbp,
                            void *flux, bool fbp_ready, cudaStream_t st);
cudaError_t launch_dvm_init(int prec, const DvmMesh &m, const double *W, void *f, cudaStream_t st);
cudaError_t prepare_dvm(int prec, int64_t Q, int nv);   // kernel attributes on the current device

// state conversions between the caller's cell-major FP64 layout (user cell order)
// and the internal SoA layout: the q-th listed cell is user cell perm[q] stored at
// internal offset loc[q] (loc == nullptr: offset q).
cudaError_t launch_init_state(int prec, int64_t n, int64_t npad, const int32_t *perm, const int32_t *loc,
                              const double *rho, const double *u, void *f, double *W, cudaStream_t st);
cudaError_t launch_pack_state(int prec, int64_t n, int64_t npad, const int32_t *perm, const int32_t *loc, const void *f,
                              const double *W, double *f_out, double *W_out, cudaStream_t st);
cudaError_t launch_unpack_state(int prec, int64_t n, int64_t npad, const int32_t *perm, const int32_t *loc,
                                const double *f_in, const double *W_in, void *f, double *W, cudaStream_t st);
// rr: the density the stored W[0] is measured from (rho = rr + W[0]; 0 for FP64, 1 for
// the FP32-compute precisions)
cudaError_t launch_macros(int64_t n, int64_t npad, const int32_t *perm, const int32_t *loc, const double *W, double rr,
                          double *rho, double *u, cudaStream_t st);
// residual over the listed cells: snap [2][npad] (U0, V0); partial [blocks][4];
// out[4] = (num, den, mass, non-finite count)
cudaError_t launch_residual(int64_t n, int64_t npad, const int32_t *loc, const double *W, double rr, const double *vol,
                            double *snap, double *partial, int n_blocks, double *out, cudaStream_t st);
inline double rho_ref_of(int prec) { return prec == P_FP64 ? 0.0 : 1.0; }
int residual_blocks(int64_t n);

// records msg as the calling thread's sdugks_last_error() and returns code
int set_error(int code, const char *msg);

}  // namespace sdugks
