// sdugks_host.cpp -- host side of libsdugks: mesh geometry and validation, periodic
// pairing, LLSR normal matrices, the tile partition with its halo rings, device
// upload, stepping (with captured CUDA graphs) and the C-ABI of include/sdugks.h.
#include "sdugks.h"
#include "sdugks_internal.h"

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <numeric>
#include <string>
#include <tuple>
#include <vector>

using namespace sdugks;

// ------------------------------------------------------------------ errors

static thread_local std::string g_err;

static int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

int sdugks::set_error(int code, const char *msg)
{
    g_err = msg;
    return code;
}

#define CUDA_TRY(expr)                                                                           \
    do {                                                                                         \
        cudaError_t e_ = (expr);                                                                 \
        if (e_ != cudaSuccess)                                                                   \
            return fail(e_ == cudaErrorMemoryAllocation ? SDUGKS_ERR_OOM : SDUGKS_ERR_CUDA,       \
                        "%s: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__, __LINE__);     \
    } while (0)

// ------------------------------------------------------------------ mesh

struct sdugks_mesh {
    int64_t np = 0, nf = 0, nc = 0;
    std::vector<double> xy;
    std::vector<int64_t> fpts, own, nbr;
    int32_t npatch = 0;
    std::array<int32_t, MAXPATCH> bc_kind{};
    std::array<std::array<double, 3>, MAXPATCH> bc_par{};
    // geometry (FP64)
    std::vector<double> vol, xc, xf, nl;   // nl: out of the owner
    std::vector<int64_t> cs, cl;           // cell -> faces
};

// Area and centroid from the outward face normals (divergence theorem on straight
// edges: V = 1/2 sum x_f . n l; int x dA = sum n_x l (x0^2 + x0 x1 + x1^2) / 6).
static int build_geometry(sdugks_mesh &m)
{
    const int64_t nc = m.nc, nf = m.nf;
    m.cs.assign(nc + 1, 0);
    for (int64_t f = 0; f < nf; f++) {
        m.cs[m.own[f] + 1]++;
        if (m.nbr[f] >= 0) m.cs[m.nbr[f] + 1]++;
    }
    for (int64_t c = 0; c < nc; c++) m.cs[c + 1] += m.cs[c];
    m.cl.assign(m.cs[nc], 0);
    {
        std::vector<int64_t> fill(nc, 0);
        for (int64_t f = 0; f < nf; f++) {
            m.cl[m.cs[m.own[f]] + fill[m.own[f]]++] = f;
            if (m.nbr[f] >= 0) m.cl[m.cs[m.nbr[f]] + fill[m.nbr[f]]++] = f;
        }
    }
    // vertex mean of each cell (inside a convex cell) for orienting the normals
    std::vector<double> vm(2 * nc, 0.0);
    for (int64_t c = 0; c < nc; c++) {
        const int64_t k = m.cs[c + 1] - m.cs[c];
        if (k < 3 || k > MAXF) return fail(SDUGKS_ERR_INVALID_MESH, "cell %lld has %lld faces (3 or 4 supported)",
                                           (long long)c, (long long)k);
        for (int64_t e = m.cs[c]; e < m.cs[c + 1]; e++) {
            const int64_t f = m.cl[e];
            for (int q = 0; q < 2; q++) {
                vm[2 * c] += m.xy[2 * m.fpts[2 * f + q]];
                vm[2 * c + 1] += m.xy[2 * m.fpts[2 * f + q] + 1];
            }
        }
        vm[2 * c] /= 2.0 * k;
        vm[2 * c + 1] /= 2.0 * k;
    }
    m.xf.assign(2 * nf, 0.0);
    m.nl.assign(2 * nf, 0.0);
    for (int64_t f = 0; f < nf; f++) {
        const double x0 = m.xy[2 * m.fpts[2 * f]], y0 = m.xy[2 * m.fpts[2 * f] + 1];
        const double x1 = m.xy[2 * m.fpts[2 * f + 1]], y1 = m.xy[2 * m.fpts[2 * f + 1] + 1];
        double nx = y1 - y0, ny = x0 - x1;
        const double mx = 0.5 * (x0 + x1), my = 0.5 * (y0 + y1);
        if ((mx - vm[2 * m.own[f]]) * nx + (my - vm[2 * m.own[f] + 1]) * ny < 0.0) { nx = -nx; ny = -ny; }
        if (nx == 0.0 && ny == 0.0) return fail(SDUGKS_ERR_INVALID_MESH, "face %lld has zero length", (long long)f);
        m.xf[2 * f] = mx; m.xf[2 * f + 1] = my;
        m.nl[2 * f] = nx; m.nl[2 * f + 1] = ny;
    }
    // the sums run in coordinates relative to the cell's vertex mean, so that cells
    // far from the origin keep their digits
    m.vol.assign(nc, 0.0);
    m.xc.assign(2 * nc, 0.0);
    for (int64_t c = 0; c < nc; c++) {
        const double ox = vm[2 * c], oy = vm[2 * c + 1];
        double v2 = 0, ix = 0, iy = 0, sx = 0, sy = 0, per = 0;
        for (int64_t e = m.cs[c]; e < m.cs[c + 1]; e++) {
            const int64_t f = m.cl[e];
            const double sg = m.own[f] == c ? 1.0 : -1.0;
            const double nx = sg * m.nl[2 * f], ny = sg * m.nl[2 * f + 1];
            const double x0 = m.xy[2 * m.fpts[2 * f]] - ox, y0 = m.xy[2 * m.fpts[2 * f] + 1] - oy;
            const double x1 = m.xy[2 * m.fpts[2 * f + 1]] - ox, y1 = m.xy[2 * m.fpts[2 * f + 1] + 1] - oy;
            v2 += 0.5 * ((x0 + x1) * nx + (y0 + y1) * ny);
            ix += nx * (x0 * x0 + x0 * x1 + x1 * x1);
            iy += ny * (y0 * y0 + y0 * y1 + y1 * y1);
            sx += nx; sy += ny;
            per += std::hypot(nx, ny);
        }
        const double V = 0.5 * v2;
        if (!(V > 0.0)) return fail(SDUGKS_ERR_INVALID_MESH, "cell %lld has area %g", (long long)c, V);
        if (std::hypot(sx, sy) > 1e-12 * per)
            return fail(SDUGKS_ERR_INVALID_MESH, "cell %lld is not closed (|sum n l| = %g)", (long long)c, std::hypot(sx, sy));
        m.vol[c] = V;
        m.xc[2 * c] = ox + ix / (6.0 * V);
        m.xc[2 * c + 1] = oy + iy / (6.0 * V);
    }
    return SDUGKS_OK;
}

extern "C" int sdugks_mesh_create(int64_t n_points, const double *xy, int64_t n_faces, const int64_t *face_pts,
                                  const int64_t *owner, const int64_t *neighbour, int64_t n_cells, sdugks_mesh **out)
{
    if (!out) return fail(SDUGKS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n_points <= 0 || n_faces <= 0 || n_cells <= 0 || !xy || !face_pts || !owner || !neighbour)
        return fail(SDUGKS_ERR_INVALID_ARG, "empty mesh or NULL array");
    if (n_cells > INT32_MAX / 2 || n_faces > INT32_MAX / 2)
        return fail(SDUGKS_ERR_INVALID_ARG, "mesh too large (%lld cells, %lld faces)", (long long)n_cells, (long long)n_faces);
    sdugks_mesh *m = new (std::nothrow) sdugks_mesh;
    if (!m) return fail(SDUGKS_ERR_OOM, "host allocation failed");
    try {
        m->np = n_points; m->nf = n_faces; m->nc = n_cells;
        m->xy.assign(xy, xy + 2 * n_points);
        m->fpts.assign(face_pts, face_pts + 2 * n_faces);
        m->own.assign(owner, owner + n_faces);
        m->nbr.assign(neighbour, neighbour + n_faces);
    } catch (...) {
        delete m;
        return fail(SDUGKS_ERR_OOM, "host allocation failed");
    }
    for (int64_t k = 0; k < 2 * n_points; k++)
        if (!std::isfinite(m->xy[k])) { delete m; return fail(SDUGKS_ERR_INVALID_MESH, "non-finite point coordinate"); }
    int32_t npatch = 0;
    for (int64_t f = 0; f < n_faces; f++) {
        const int64_t p0 = m->fpts[2 * f], p1 = m->fpts[2 * f + 1];
        if (p0 < 0 || p0 >= n_points || p1 < 0 || p1 >= n_points || p0 == p1) {
            delete m;
            return fail(SDUGKS_ERR_INVALID_MESH, "face %lld has bad points (%lld, %lld)", (long long)f, (long long)p0, (long long)p1);
        }
        const int64_t o = m->own[f], k = m->nbr[f];
        if (o < 0 || o >= n_cells || k >= n_cells || k == o) {
            delete m;
            return fail(SDUGKS_ERR_INVALID_MESH, "face %lld has bad owner/neighbour (%lld, %lld)", (long long)f, (long long)o, (long long)k);
        }
        if (k < 0) {
            const int64_t p = -1 - k;
            if (p >= MAXPATCH) { delete m; return fail(SDUGKS_ERR_INVALID_MESH, "patch %lld >= %d", (long long)p, MAXPATCH); }
            npatch = std::max<int32_t>(npatch, (int32_t)p + 1);
        }
    }
    m->npatch = npatch;
    int rc = build_geometry(*m);
    if (rc) { delete m; return rc; }
    *out = m;
    return SDUGKS_OK;
}

extern "C" int sdugks_set_bc(sdugks_mesh *m, int32_t patch, int32_t kind, const double *params)
{
    if (!m) return fail(SDUGKS_ERR_INVALID_ARG, "mesh is NULL");
    if (patch < 0 || patch >= MAXPATCH) return fail(SDUGKS_ERR_INVALID_ARG, "patch %d out of range", patch);
    if (kind < SDUGKS_BC_PERIODIC || kind > SDUGKS_BC_SYMMETRY) return fail(SDUGKS_ERR_INVALID_ARG, "unknown kind %d", kind);
    const bool need = kind == SDUGKS_BC_PERIODIC || kind == SDUGKS_BC_MOVING_WALL || kind == SDUGKS_BC_FARFIELD;
    if (need && !params) return fail(SDUGKS_ERR_INVALID_ARG, "kind %d needs params", kind);
    for (int k = 0; k < 3; k++) {
        const double v = params ? params[k] : 0.0;
        if (!std::isfinite(v)) return fail(SDUGKS_ERR_INVALID_ARG, "non-finite boundary parameter");
        m->bc_par[patch][k] = v;
    }
    if (kind == SDUGKS_BC_FARFIELD && !(params[0] > 0)) return fail(SDUGKS_ERR_INVALID_ARG, "far-field density must be > 0");
    m->bc_kind[patch] = kind;
    return SDUGKS_OK;
}

extern "C" int sdugks_mesh_cfl_dt(const sdugks_mesh *m, double cfl, double *dt)
{
    if (!m || !dt || !(cfl > 0)) return fail(SDUGKS_ERR_INVALID_ARG, "bad argument");
    double dmin = INFINITY;
    for (int64_t c = 0; c < m->nc; c++) {
        double lmax = 0;
        for (int64_t e = m->cs[c]; e < m->cs[c + 1]; e++) {
            const int64_t f = m->cl[e];
            lmax = std::max(lmax, std::hypot(m->nl[2 * f], m->nl[2 * f + 1]));
        }
        dmin = std::min(dmin, m->vol[c] / lmax);
    }
    *dt = cfl * dmin / std::sqrt(2.0);
    return SDUGKS_OK;
}

extern "C" int sdugks_mesh_sizes(const sdugks_mesh *m, int64_t *n_cells, int64_t *n_faces, int32_t *n_patches)
{
    if (!m) return fail(SDUGKS_ERR_INVALID_ARG, "mesh is NULL");
    if (n_cells) *n_cells = m->nc;
    if (n_faces) *n_faces = m->nf;
    if (n_patches) *n_patches = m->npatch;
    return SDUGKS_OK;
}

extern "C" void sdugks_mesh_destroy(sdugks_mesh *m) { delete m; }

// ------------------------------------------------------------------ solver build

namespace {

// Faces after periodic pairs are merged into interior faces.
struct Faces {
    int64_t nf = 0;
    std::vector<int64_t> own, nbr;        // nbr: cell or -1 - patch
    std::vector<double> nl, ro, rk;       // [nf][2]
    std::vector<int64_t> orig;            // the caller's id of each merged face
};

// Row of each caller face in the per-boundary-face outputs (sdugks_step_boundary_flux):
// the faces on non-periodic patches, in the caller's face order; -1 for the others.
// Returns the number of rows.
int64_t boundary_rows(const sdugks_mesh &m, std::vector<int64_t> &row)
{
    row.assign(m.nf, -1);
    int64_t n = 0;
    for (int64_t f = 0; f < m.nf; f++)
        if (m.nbr[f] < 0 && m.bc_kind[-1 - m.nbr[f]] != SDUGKS_BC_PERIODIC) row[f] = n++;
    return n;
}

int merge_periodic(const sdugks_mesh &m, Faces &F)
{
    const int64_t nf = m.nf;
    std::vector<int64_t> partner(nf, -1);
    for (int32_t p = 0; p < m.npatch; p++) {
        if (m.bc_kind[p] != SDUGKS_BC_PERIODIC) continue;
        const int32_t q = (int32_t)m.bc_par[p][0];
        if (q < 0 || q >= MAXPATCH || q == p || m.bc_kind[q] != SDUGKS_BC_PERIODIC)
            return fail(SDUGKS_ERR_BAD_BC, "periodic patch %d names partner %d which is not periodic", p, q);
        if ((int32_t)m.bc_par[q][0] != p) return fail(SDUGKS_ERR_BAD_BC, "periodic patches %d and %d are not partners of each other", p, q);
        const double sx = m.bc_par[p][1], sy = m.bc_par[p][2];
        if (std::hypot(sx + m.bc_par[q][1], sy + m.bc_par[q][2]) > 1e-9 * std::max(1.0, std::hypot(sx, sy)))
            return fail(SDUGKS_ERR_BAD_BC, "periodic shifts of patches %d and %d do not cancel", p, q);
        // faces of q sorted along their centres for matching
        std::vector<int64_t> fq;
        for (int64_t g = 0; g < nf; g++)
            if (m.nbr[g] == -1 - q) fq.push_back(g);
        std::sort(fq.begin(), fq.end(), [&](int64_t a, int64_t b) {
            return m.xf[2 * a] != m.xf[2 * b] ? m.xf[2 * a] < m.xf[2 * b] : m.xf[2 * a + 1] < m.xf[2 * b + 1];
        });
        for (int64_t f = 0; f < nf; f++) {
            if (m.nbr[f] != -1 - p) continue;
            const double len = std::hypot(m.nl[2 * f], m.nl[2 * f + 1]);
            const double tx = m.xf[2 * f] + sx, ty = m.xf[2 * f + 1] + sy, tol = 1e-9 * len;
            auto it = std::lower_bound(fq.begin(), fq.end(), tx - tol, [&](int64_t g, double v) { return m.xf[2 * g] < v; });
            int64_t hit = -1;
            for (; it != fq.end() && m.xf[2 * *it] <= tx + tol; ++it)
                if (std::hypot(m.xf[2 * *it] - tx, m.xf[2 * *it + 1] - ty) <= tol) { hit = *it; break; }
            if (hit < 0) return fail(SDUGKS_ERR_BAD_BC, "periodic face %lld of patch %d has no partner on patch %d", (long long)f, p, q);
            partner[f] = hit;
        }
    }
    std::vector<int64_t> newid(nf, -1);
    for (int64_t f = 0; f < nf; f++) {
        if (m.nbr[f] < 0) {
            const int32_t p = (int32_t)(-1 - m.nbr[f]);
            if (m.bc_kind[p] == SDUGKS_BC_UNSET) return fail(SDUGKS_ERR_BAD_BC, "boundary patch %d has no boundary condition", p);
            if (m.bc_kind[p] == SDUGKS_BC_PERIODIC) {
                const int64_t g = partner[f];
                if (partner[g] != f) return fail(SDUGKS_ERR_BAD_BC, "periodic faces %lld and %lld do not pair both ways", (long long)f, (long long)g);
                if (g < f) continue;      // the pair is kept once, at the lower face id
            }
        }
        newid[f] = F.nf++;
    }
    F.own.resize(F.nf); F.nbr.resize(F.nf); F.orig.resize(F.nf);
    F.nl.resize(2 * F.nf); F.ro.resize(2 * F.nf); F.rk.resize(2 * F.nf);
    for (int64_t f = 0; f < nf; f++) {
        const int64_t k = newid[f];
        if (k < 0) continue;
        const int64_t o = m.own[f];
        F.own[k] = o;
        F.orig[k] = f;
        F.nl[2 * k] = m.nl[2 * f]; F.nl[2 * k + 1] = m.nl[2 * f + 1];
        F.ro[2 * k] = m.xf[2 * f] - m.xc[2 * o]; F.ro[2 * k + 1] = m.xf[2 * f + 1] - m.xc[2 * o + 1];
        if (m.nbr[f] >= 0) {
            const int64_t nb = m.nbr[f];
            F.nbr[k] = nb;
            F.rk[2 * k] = m.xf[2 * f] - m.xc[2 * nb]; F.rk[2 * k + 1] = m.xf[2 * f + 1] - m.xc[2 * nb + 1];
        } else if (partner[f] >= 0) {
            const int64_t g = partner[f], nb = m.own[g];
            F.nbr[k] = nb;
            // the same face seen from the far cell: its own copy of the face centre
            F.rk[2 * k] = m.xf[2 * g] - m.xc[2 * nb]; F.rk[2 * k + 1] = m.xf[2 * g + 1] - m.xc[2 * nb + 1];
        } else {
            F.nbr[k] = m.nbr[f];
            F.rk[2 * k] = 0.0; F.rk[2 * k + 1] = 0.0;
        }
    }
    return SDUGKS_OK;
}

// Recursive coordinate bisection of the cell centroids into tiles of <= cap cells.
void rcb(const std::vector<double> &xc, std::vector<int32_t> &ids, size_t lo, size_t hi, size_t cap,
         std::vector<std::pair<size_t, size_t>> &tiles)
{
    if (hi - lo <= cap) { tiles.push_back({lo, hi}); return; }
    double mn[2] = {INFINITY, INFINITY}, mx[2] = {-INFINITY, -INFINITY};
    for (size_t i = lo; i < hi; i++)
        for (int d = 0; d < 2; d++) {
            mn[d] = std::min(mn[d], xc[2 * ids[i] + d]);
            mx[d] = std::max(mx[d], xc[2 * ids[i] + d]);
        }
    const int ax = (mx[0] - mn[0] >= mx[1] - mn[1]) ? 0 : 1;
    // split so the left part is a whole number of full tiles where possible
    const size_t n = hi - lo, ntile = (n + cap - 1) / cap;
    const size_t mid = lo + ((ntile / 2) * n + ntile / 2) / ntile;
    std::nth_element(ids.begin() + lo, ids.begin() + mid, ids.begin() + hi, [&](int32_t a, int32_t b) {
        const double va = xc[2 * a + ax], vb = xc[2 * b + ax];
        if (va != vb) return va < vb;
        const double wa = xc[2 * a + 1 - ax], wb = xc[2 * b + 1 - ax];
        return wa != wb ? wa < wb : a < b;
    });
    rcb(xc, ids, lo, mid, cap, tiles);
    rcb(xc, ids, mid, hi, cap, tiles);
}

struct Arena {
    char *base = nullptr;
    size_t used = 0, cap = 0;
    template <class T> T *take(size_t count) {
        size_t off = (used + 255) & ~size_t(255);
        used = off + count * sizeof(T);
        return base ? reinterpret_cast<T *>(base + off) : nullptr;
    }
};

}  // namespace

struct sdugks_solver {
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    sdugks_params p{};
    Coefs coefs{};
    int64_t n = 0, npad = 0, nf = 0;
    int32_t n_tiles = 0;
    int64_t halo_cells = 0;
    int32_t kernel = SDUGKS_KERNEL_TILED;
    TiledMesh tm{};
    // device buffers
    char *dmem = nullptr;
    size_t dbytes = 0;
    int32_t *perm = nullptr;        // q-th listed cell -> user id
    int32_t *loc = nullptr;         // q-th listed cell -> internal offset (nullptr: q)
    CartInst ci{};
    int cart_shape = 0;             // Cartesian block shape (CART_TY)
    CartTma *tma = nullptr;         // Cartesian: tensor maps of the TMA staging (nullptr: plain loads)
    bool cart_general = false;      // Cartesian: every block on the general code path (one-wave grids)
    double *vol = nullptr, *snap = nullptr, *partial = nullptr, *red = nullptr;
    State st{};
    int n_red_blocks = 1;
    double *staging = nullptr;      // [n][15] FP64, allocated on first use
    double *h_red = nullptr;        // pinned [5]: red[0..3], then the error flag (int32 in red[4])
    bool initialised = false;
    int cur = 0;                    // buffer (f and W) holding the state at t_n
    int64_t steps_done = 0;
    cudaGraphExec_t graph = nullptr;
    int graph_len = 0;
    cudaGraphExec_t tail[31] = {};  // graphs of 2^k steps (k >= 1, 2^k < graph_len) for the remainders
    double mesh_bytes = 0.0;
    double *d_force = nullptr;      // [MAXPATCH][2] (allocated on first force step)
    int64_t n_bfaces = 0;           // rows of the per-boundary-face outputs
    double *d_bface = nullptr;      // [n_bfaces][2] (allocated on first per-face flux step)
    int32_t side_patch[4] = {-1, -1, -1, -1};   // Cartesian: patch of each grid side
};

static int prepare(int prec, int kernel)
{
    if (kernel == SDUGKS_KERNEL_CARTESIAN) return (int)prepare_cart(prec);
    return prec == P_FP64 ? (int)prepare_tiled_fp64() : (int)prepare_tiled_fp32(prec);
}

static cudaError_t launch_one(sdugks_solver *s, cudaStream_t st)
{
    const int a = s->cur;
    cudaError_t e;
    if (s->kernel == SDUGKS_KERNEL_CARTESIAN)
        e = launch_step_cart(s->p.precision, s->cart_shape, s->ci, s->tma, s->cart_general, a, st);
    else if (s->p.precision == P_FP64)
        e = launch_step_tiled_fp64(s->tm, s->coefs, s->st.f[a], s->st.f[1 - a], s->st.W[a], s->st.W[1 - a], st);
    else
        e = launch_step_tiled_fp32(s->p.precision, s->tm, s->coefs, s->st.f[a], s->st.f[1 - a], s->st.W[a],
                                   s->st.W[1 - a], st);
    s->cur = 1 - a;
    return e;
}

static void fill_coefs(Coefs &c, const sdugks_mesh &m, double tau, double dt)
{
    c.a_plus = (2.0 * tau - dt) / (2.0 * tau);
    c.b_plus = dt / (2.0 * tau);
    c.c_face = 2.0 * tau / (2.0 * tau + dt);
    c.r = dt / tau;
    c.inv1r = 1.0 / (1.0 + dt / tau);
    c.dt = dt;
    c.tie = 1e-12;
    c.fa_plus = (float)c.a_plus; c.fb_plus = (float)c.b_plus; c.fc_face = (float)c.c_face; c.fr = (float)c.r;
    c.finv1r = (float)c.inv1r; c.fdt = (float)c.dt; c.ftie = (float)c.tie; c.fpad_ = 0.0f;
    for (int q = 0; q < MAXPATCH; q++) {
        c.bc_kind[q] = m.bc_kind[q];
        for (int d = 0; d < 3; d++) {
            c.bc_par[q][d] = m.bc_par[q][d];
            c.fbc_par[q][d] = (float)m.bc_par[q][d];
        }
        c.fbc_drho[q] = (float)(m.bc_par[q][0] - 1.0);
    }
}

namespace {

// A mesh recognised as a uniform nx x ny grid of dx x dy rectangles.
struct CartGrid {
    int32_t nx = 0, ny = 0;
    double dx = 0, dy = 0;
    int32_t side_patch[4] = {-1, -1, -1, -1};   // bottom, right, top, left
    bool px = false, py = false;
    std::vector<int32_t> ci, cj;                  // lattice position of each user cell
    std::string why;
};

bool detect_cart(const sdugks_mesh &m, CartGrid &g)
{
    double dx = -1, dy = -1;
    for (int64_t f = 0; f < m.nf; f++) {
        const double nx = m.nl[2 * f], ny = m.nl[2 * f + 1], len = std::hypot(nx, ny);
        double *h;
        if (std::fabs(ny) <= 1e-12 * len) h = &dy;          // face of constant x, length dy
        else if (std::fabs(nx) <= 1e-12 * len) h = &dx;     // face of constant y, length dx
        else { g.why = "a face is not axis-aligned"; return false; }
        if (*h < 0) *h = len;
        else if (std::fabs(*h - len) > 1e-12 * len) { g.why = "faces of different lengths"; return false; }
    }
    if (dx <= 0 || dy <= 0) { g.why = "no faces in one direction"; return false; }
    for (int64_t c = 0; c < m.nc; c++)
        if (m.cs[c + 1] - m.cs[c] != 4) { g.why = "a cell without four faces"; return false; }
    double x0 = INFINITY, y0 = INFINITY;
    for (int64_t p = 0; p < m.np; p++) { x0 = std::min(x0, m.xy[2 * p]); y0 = std::min(y0, m.xy[2 * p + 1]); }
    g.ci.resize(m.nc); g.cj.resize(m.nc);
    int64_t mi = 0, mj = 0;
    for (int64_t c = 0; c < m.nc; c++) {
        const double fi = (m.xc[2 * c] - x0) / dx - 0.5, fj = (m.xc[2 * c + 1] - y0) / dy - 0.5;
        const long long i = std::llround(fi), j = std::llround(fj);
        if (std::fabs(fi - i) > 1e-6 || std::fabs(fj - j) > 1e-6 || i < 0 || j < 0 || i > INT32_MAX / 4 || j > INT32_MAX / 4) {
            g.why = "cell centres are not on a lattice";
            return false;
        }
        g.ci[c] = (int32_t)i; g.cj[c] = (int32_t)j;
        mi = std::max<int64_t>(mi, i); mj = std::max<int64_t>(mj, j);
    }
    const int64_t nx = mi + 1, ny = mj + 1;
    if (nx * ny != m.nc || nx < 2 || ny < 2) { g.why = "cells do not fill an nx x ny grid (nx, ny >= 2)"; return false; }
    // the kernel's grid of blocks is two-dimensional: at most 65535 rows of blocks of >= 8 rows
    if (ny > 8 * 65535) { g.why = "more than 524,280 rows of cells"; return false; }
    {
        std::vector<char> seen(m.nc, 0);
        for (int64_t c = 0; c < m.nc; c++) {
            char &v = seen[g.ci[c] + nx * g.cj[c]];
            if (v) { g.why = "two cells on one lattice site"; return false; }
            v = 1;
        }
    }
    for (int64_t f = 0; f < m.nf; f++) {
        const int64_t o = m.own[f], k = m.nbr[f];
        const double nx_ = m.nl[2 * f], ny_ = m.nl[2 * f + 1];
        const int sx = std::fabs(nx_) > std::fabs(ny_) ? (nx_ > 0 ? 1 : -1) : 0;
        const int sy = sx == 0 ? (ny_ > 0 ? 1 : -1) : 0;
        if (k >= 0) {
            if (g.ci[k] - g.ci[o] != sx || g.cj[k] - g.cj[o] != sy) { g.why = "an interior face joins non-adjacent cells"; return false; }
            continue;
        }
        int side;
        if (sx == 1 && g.ci[o] == nx - 1) side = 1;
        else if (sx == -1 && g.ci[o] == 0) side = 3;
        else if (sy == 1 && g.cj[o] == ny - 1) side = 2;
        else if (sy == -1 && g.cj[o] == 0) side = 0;
        else { g.why = "a boundary face inside the grid"; return false; }
        const int32_t patch = (int32_t)(-1 - k);
        if (g.side_patch[side] < 0) g.side_patch[side] = patch;
        else if (g.side_patch[side] != patch) { g.why = "one grid side carries two patches"; return false; }
    }
    // periodic sides must pair left/right and bottom/top with the grid period as shift
    const double W = nx * dx, H = ny * dy;
    const int opp[4] = {2, 3, 0, 1};
    const double shx[4] = {0, -W, 0, W}, shy[4] = {H, 0, -H, 0};
    for (int side = 0; side < 4; side++) {
        const int32_t p = g.side_patch[side];
        if (p < 0) { g.why = "a grid side has no boundary faces"; return false; }
        const bool per = m.bc_kind[p] == SDUGKS_BC_PERIODIC;
        if (!per) continue;
        if ((int32_t)m.bc_par[p][0] != g.side_patch[opp[side]] ||
            std::fabs(m.bc_par[p][1] - shx[side]) > 1e-9 * dx || std::fabs(m.bc_par[p][2] - shy[side]) > 1e-9 * dy) {
            g.why = "a periodic side does not pair with the opposite side";
            return false;
        }
    }
    auto periodic = [&](int side) { return m.bc_kind[g.side_patch[side]] == SDUGKS_BC_PERIODIC; };
    g.px = periodic(1) && periodic(3);
    g.py = periodic(0) && periodic(2);
    if (periodic(1) != periodic(3) || periodic(0) != periodic(2)) { g.why = "one-sided periodic grid"; return false; }
    for (int side = 0; side < 4; side++)
        for (int other = 0; other < 4; other++)
            if (other != side && g.side_patch[other] == g.side_patch[side] && periodic(side)) {
                g.why = "a periodic patch on two sides"; return false;
            }
    g.nx = (int32_t)nx; g.ny = (int32_t)ny; g.dx = dx; g.dy = dy;
    return true;
}

}  // namespace

// Grid, side rules and coefficients of a uniform-grid solve (state pointers are set
// by the caller).
static void fill_cart_inst(CartInst &ci, const sdugks_mesh &m, const CartGrid &g, double tau, double dt, int32_t pitch,
                           int64_t npad)
{
    std::memset(&ci, 0, sizeof ci);
    ci.nx = g.nx; ci.ny = g.ny; ci.pitch = pitch; ci.periodic_x = g.px; ci.periodic_y = g.py;
    for (int k = 0; k < 4; k++) {
        const int32_t p = g.side_patch[k];
        ci.side_kind[k] = m.bc_kind[p];
        for (int d = 0; d < 3; d++) {
            ci.side_par[k][d] = m.bc_par[p][d];
            ci.fside_par[k][d] = (float)m.bc_par[p][d];
        }
        ci.fside_drho[k] = (float)(m.bc_par[p][0] - 1.0);
    }
    ci.npad = npad;
    ci.dx = g.dx; ci.dy = g.dy; ci.dtV = dt / (g.dx * g.dy);
    ci.a = (2.0 * tau - dt) / (2.0 * tau);
    ci.b = dt / (2.0 * tau);
    ci.c = 2.0 * tau / (2.0 * tau + dt);
    ci.r = dt / tau;
    ci.dt = dt;
    ci.ihx = 1.0 / g.dx; ci.ihy = 1.0 / g.dy;
    ci.fdx = (float)ci.dx; ci.fdy = (float)ci.dy; ci.fdtV = (float)ci.dtV;
    ci.fihx = (float)ci.ihx; ci.fihy = (float)ci.ihy;
    ci.fa = (float)ci.a; ci.fb = (float)ci.b; ci.fc = (float)ci.c; ci.fr = (float)ci.r;
    ci.finv1r = (float)(1.0 / (1.0 + dt / tau));
    ci.fdt = (float)dt;
}

static int create_cart(const sdugks_mesh &m, const CartGrid &g, const sdugks_params *prm, void *stream, sdugks_solver **out)
{
    const int64_t n = m.nc;
    const int32_t pitch = (g.nx + 31) / 32 * 32;
    const int64_t npad = ((int64_t)pitch * g.ny + 31) / 32 * 32;
    const int prec = prm->precision;
    const size_t fs = prec == P_FP64 ? 8 : (prec == P_FP32 ? 4 : 2);
    sdugks_solver *s = new (std::nothrow) sdugks_solver;
    if (!s) return fail(SDUGKS_ERR_OOM, "host allocation failed");
    s->p = *prm;
    if (s->p.graph_steps == 0) s->p.graph_steps = 64;
    if (s->p.graph_steps > 0) s->p.graph_steps = std::max(2, s->p.graph_steps / 2 * 2);
    s->stream = static_cast<cudaStream_t>(stream);
    s->n = n; s->npad = npad; s->nf = m.nf;
    s->kernel = SDUGKS_KERNEL_CARTESIAN;
    constexpr int TX = 16, TY = 16;
    s->n_tiles = ((g.nx + TX - 1) / TX) * ((g.ny + TY - 1) / TY);
    s->halo_cells = (int64_t)s->n_tiles * ((TX + 4) * (TY + 4) - TX * TY);
    s->n_red_blocks = residual_blocks(n);
    s->mesh_bytes = 0.0;
    fill_cart_inst(s->ci, m, g, prm->tau, prm->dt, pitch, npad);
    for (int k = 0; k < 4; k++) s->side_patch[k] = g.side_patch[k];
    auto layout = [&](Arena &A) {
        s->perm = A.take<int32_t>(n);
        s->loc = A.take<int32_t>(n);
        s->vol = A.take<double>(npad);
        s->snap = A.take<double>(2 * npad);
        s->partial = A.take<double>(4 * (size_t)s->n_red_blocks);
        s->red = A.take<double>(5);
        s->ci.bidx = A.take<int32_t>(2 * ((size_t)g.nx + g.ny));
        for (int b = 0; b < 2; b++) s->st.f[b] = A.take<char>(NQ * npad * fs);
        for (int b = 0; b < 2; b++) s->st.W[b] = A.take<double>(3 * npad);
    };
    Arena A0;
    layout(A0);
    s->dbytes = A0.used + 256;
    cudaError_t e = cudaGetDevice(&s->device);
    if (e == cudaSuccess) e = cudaMalloc(&s->dmem, s->dbytes);
    if (e != cudaSuccess) {
        delete s;
        return fail(e == cudaErrorMemoryAllocation ? SDUGKS_ERR_OOM : SDUGKS_ERR_CUDA, "cudaMalloc(%zu): %s", A0.used,
                    cudaGetErrorString(e));
    }
    Arena A{s->dmem, 0, s->dbytes};
    layout(A);
    // boundary-face row of each side face, by side and position along the side
    std::vector<int32_t> bidx(2 * ((size_t)g.nx + g.ny), -1);
    {
        std::vector<int64_t> row;
        s->n_bfaces = boundary_rows(m, row);
        for (int64_t f = 0; f < m.nf; f++) {
            if (row[f] < 0) continue;
            const int64_t o = m.own[f];
            const double nx_ = m.nl[2 * f], ny_ = m.nl[2 * f + 1];
            size_t q;
            if (std::fabs(nx_) > std::fabs(ny_)) q = nx_ > 0 ? (size_t)g.nx + g.cj[o] : 2 * (size_t)g.nx + g.ny + g.cj[o];
            else q = ny_ > 0 ? (size_t)g.nx + g.ny + g.ci[o] : (size_t)g.ci[o];
            bidx[q] = (int32_t)row[f];
        }
    }
    for (int b = 0; b < 2; b++) { s->ci.f[b] = s->st.f[b]; s->ci.W[b] = s->st.W[b]; }
    s->ci.snap = s->snap;
    s->ci.err = reinterpret_cast<int32_t *>(s->red + 4);
    s->ci.tma_wait_ns = prm->tma_wait_us == 0 ? 200000000ull
                        : prm->tma_wait_us < 0 ? 0ull : 1000ull * (uint64_t)prm->tma_wait_us;
    std::vector<int32_t> perm(n), loc(n);
    std::vector<double> vol(npad, 1.0);
    for (int64_t c = 0; c < n; c++) {
        perm[c] = (int32_t)c;
        loc[c] = g.ci[c] + pitch * g.cj[c];
        vol[loc[c]] = m.vol[c];
    }
    int rc2 = SDUGKS_OK;
    auto chk = [&](cudaError_t ee, const char *what) {
        if (ee != cudaSuccess && rc2 == SDUGKS_OK) rc2 = fail(SDUGKS_ERR_CUDA, "%s: %s", what, cudaGetErrorString(ee));
    };
    chk(cudaMemset(s->dmem, 0, s->dbytes), "memset");
    chk(cudaMemcpy(s->perm, perm.data(), n * 4, cudaMemcpyHostToDevice), "upload perm");
    chk(cudaMemcpy(s->loc, loc.data(), n * 4, cudaMemcpyHostToDevice), "upload loc");
    chk(cudaMemcpy(s->vol, vol.data(), npad * 8, cudaMemcpyHostToDevice), "upload vol");
    chk(cudaMemcpy(const_cast<int32_t *>(s->ci.bidx), bidx.data(), bidx.size() * 4, cudaMemcpyHostToDevice),
        "upload boundary rows");
    chk(cudaMallocHost(&s->h_red, 5 * sizeof(double)), "cudaMallocHost");
    chk(cudaStreamCreateWithFlags(&s->cap_stream, cudaStreamNonBlocking), "cudaStreamCreate");
    chk((cudaError_t)prepare(prec, SDUGKS_KERNEL_CARTESIAN), "kernel attributes");
    if (rc2) { sdugks_solver_destroy(s); return rc2; }
    fill_coefs(s->coefs, m, prm->tau, prm->dt);
    // Block shape: tile_cells 256/224/128 picks 16x16/16x14/16x8; 0 picks by a cost
    // model: waves of resident blocks (rounded up) times the work one SM does per
    // wave (resident blocks x staged positions plus faces of a block), with the
    // shapes that fit four blocks per SM credited 1.21x for hiding latency better (the
    // ratio measured on GB300 between the 16x8 and 16x16 shapes on a 1024^2 grid).
    // The choice depends only on the grid size and the device, never on timings.
    const bool use_tma = prm->staging == SDUGKS_STAGING_TMA;
    {
        int n_sm = 1;
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, s->device);
        s->cart_shape = 0;
        if (prec != P_FP64) {
            double best = 1e300;
            for (int sh = 0; sh < CART_SHAPES; sh++) {
                const int ty = CART_TY[sh];
                if (prm->tile_cells && prm->tile_cells != 16 * ty) continue;
                const int occ = std::max(1, cart_shape_occupancy(prec, sh, use_tma));
                const int64_t tiles = (int64_t)((g.nx + 15) / 16) * ((g.ny + ty - 1) / ty);
                const int64_t slots = (int64_t)n_sm * occ;
                const double work = (20.0 * (ty + 4) + 17.0 * ty + 16.0 * (ty + 1));
                const double eff = occ >= 4 ? 1.21 : 1.0;
                const double cost = (double)((tiles + slots - 1) / slots) * occ * work / eff;
                if (cost < best - 1e-9) { best = cost; s->cart_shape = sh; }
            }
        }
        const int ty = CART_TY[s->cart_shape];
        s->n_tiles = ((g.nx + 15) / 16) * ((g.ny + ty - 1) / ty);
        s->halo_cells = (int64_t)s->n_tiles * (20 * (ty + 4) - 16 * ty);
        // all blocks in one wave: the slowest (edge) block sets the step time, and one
        // code path for every block measured faster (GB300, 256^2: 126.4 k against 120.3 k
        // MLUPS; 512^2, four waves: 150.1 k against 160.1 k with the interior variant)
        s->cart_general = !use_tma &&
                          s->n_tiles <= (int64_t)n_sm * std::max(1, cart_shape_occupancy(prec, s->cart_shape, false));
    }
    // interior blocks staged by tensor copies; the maps hold the fixed addresses of the
    // two state buffers
    if (use_tma) {
        s->tma = new (std::nothrow) CartTma;
        if (!s->tma) { sdugks_solver_destroy(s); return fail(SDUGKS_ERR_OOM, "host allocation failed"); }
        const cudaError_t te = make_cart_tma(prec, s->cart_shape, s->ci, *s->tma);
        if (te != cudaSuccess) {
            sdugks_solver_destroy(s);
            return fail(SDUGKS_ERR_CUDA, "tensor maps of the Cartesian state: %s", cudaGetErrorString(te));
        }
    }
    *out = s;
    return SDUGKS_OK;
}

extern "C" int sdugks_solver_create(const sdugks_mesh *m, const sdugks_params *prm, void *stream, sdugks_solver **out)
{
    if (!out) return fail(SDUGKS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!m || !prm) return fail(SDUGKS_ERR_INVALID_ARG, "mesh or params is NULL");
    if (!(prm->tau > 0) || !(prm->dt > 0) || !std::isfinite(prm->tau) || !std::isfinite(prm->dt))
        return fail(SDUGKS_ERR_INVALID_ARG, "tau and dt must be finite and > 0");
    if (prm->precision < SDUGKS_FP64 || prm->precision > SDUGKS_FP32_FP16DEV)
        return fail(SDUGKS_ERR_INVALID_ARG, "unknown precision %d", prm->precision);
    if (prm->kernel < SDUGKS_KERNEL_AUTO || prm->kernel > SDUGKS_KERNEL_CARTESIAN)
        return fail(SDUGKS_ERR_INVALID_ARG, "unknown kernel %d", prm->kernel);
    if (prm->staging != SDUGKS_STAGING_LOADS && prm->staging != SDUGKS_STAGING_TMA)
        return fail(SDUGKS_ERR_INVALID_ARG, "unknown staging %d", prm->staging);

    Faces F;
    int rc = merge_periodic(*m, F);
    if (rc) return rc;
    const int64_t n = m->nc;
    if (prm->kernel != SDUGKS_KERNEL_TILED) {
        CartGrid cg;
        if (detect_cart(*m, cg)) {
            const int t = prm->tile_cells;
            if (t != 0 && !(prm->precision != SDUGKS_FP64 && (t == 256 || t == 224 || t == 128)) &&
                !(prm->precision == SDUGKS_FP64 && t == 256))
                return fail(SDUGKS_ERR_INVALID_ARG, "Cartesian kernel: tile_cells must be 0, 256, 224 or 128 (FP64: 0 or 256)");
            return create_cart(*m, cg, prm, stream, out);
        }
        if (prm->kernel == SDUGKS_KERNEL_CARTESIAN)
            return fail(SDUGKS_ERR_INVALID_ARG, "not a uniform Cartesian grid: %s", cg.why.c_str());
    }
    if (prm->staging == SDUGKS_STAGING_TMA)
        return fail(SDUGKS_ERR_INVALID_ARG, "TMA staging needs the Cartesian kernel (a uniform grid)");
    if (prm->tile_cells != 0 && (prm->tile_cells < 16 || prm->tile_cells > TILE_MAX))
        return fail(SDUGKS_ERR_INVALID_ARG, "tile_cells must be 0 or in [16, %d]", TILE_MAX);

    // cell -> faces over the merged faces; slots in ascending merged face id, which
    // keeps the caller's face order, so per-cell sums do not depend on the tiling
    std::vector<std::array<int64_t, MAXF>> slots(n);
    std::vector<int> nslot(n, 0);
    for (int64_t f = 0; f < F.nf; f++) {
        if (F.own[f] == F.nbr[f])
            return fail(SDUGKS_ERR_INVALID_MESH, "periodic pair joins cell %lld to itself", (long long)F.own[f]);
        for (int side = 0; side < 2; side++) {
            const int64_t c = side == 0 ? F.own[f] : F.nbr[f];
            if (c < 0) continue;
            if (nslot[c] >= MAXF) return fail(SDUGKS_ERR_INVALID_MESH, "cell %lld has more than %d faces", (long long)c, MAXF);
            slots[c][nslot[c]++] = f;
        }
    }
    // per cell and slot: n l out of the cell, x_f - x_j, x_f - x_k; LLSR inverse from
    // d = x_k - x_j = (x_f - x_j) - (x_f - x_k)
    std::vector<double> sgeo((size_t)n * MAXF * 6, 0.0), ainv(3 * n, 0.0);
    std::vector<uint8_t> skind((size_t)n * MAXF, SK_NONE);
    for (int64_t c = 0; c < n; c++) {
        double axx = 0, axy = 0, ayy = 0;
        for (int sl = 0; sl < nslot[c]; sl++) {
            const int64_t f = slots[c][sl];
            double *G = &sgeo[((size_t)c * MAXF + sl) * 6];
            const bool mine = F.own[f] == c;
            const double sg = mine ? 1.0 : -1.0;
            G[0] = sg * F.nl[2 * f]; G[1] = sg * F.nl[2 * f + 1];
            const double *rme = mine ? &F.ro[2 * f] : &F.rk[2 * f];
            const double *rot = mine ? &F.rk[2 * f] : &F.ro[2 * f];
            G[2] = rme[0]; G[3] = rme[1];
            if (F.nbr[f] >= 0) {
                skind[(size_t)c * MAXF + sl] = SK_INTERIOR;
                G[4] = rot[0]; G[5] = rot[1];
                const double dx = rme[0] - rot[0], dy = rme[1] - rot[1];
                axx += dx * dx; axy += dx * dy; ayy += dy * dy;
            } else {
                const int p = (int)(-1 - F.nbr[f]);
                skind[(size_t)c * MAXF + sl] = (uint8_t)p;
                if (m->bc_kind[p] == SDUGKS_BC_SYMMETRY) {
                    // the mirror ghost: x_f - x_g is x_f - x_j reflected in the face line,
                    // and the ghost is an LLSR neighbour at d = x_g - x_j
                    const double ax = std::fabs(G[0]), ay = std::fabs(G[1]);
                    if (ay > 1e-12 * ax && ax > 1e-12 * ay)
                        return fail(SDUGKS_ERR_BAD_BC, "symmetry face %lld is not a line of constant x or y", (long long)f);
                    const bool nx_axis = ax > ay;
                    G[4] = nx_axis ? -rme[0] : rme[0];
                    G[5] = nx_axis ? rme[1] : -rme[1];
                    const double dx = rme[0] - G[4], dy = rme[1] - G[5];
                    axx += dx * dx; axy += dx * dy; ayy += dy * dy;
                }
            }
        }
        const double det = axx * ayy - axy * axy, tr = axx + ayy;
        if (det > 1e-14 * tr * tr) {
            ainv[3 * c] = ayy / det; ainv[3 * c + 1] = -axy / det; ainv[3 * c + 2] = axx / det;
        }
    }

    // ---- tiles: RCB, then halo rings; tiles whose halo overflows are split again
    const size_t cap0 = prm->tile_cells ? (size_t)prm->tile_cells : (size_t)TILE_MAX;
    std::vector<int32_t> ids(n);
    std::iota(ids.begin(), ids.end(), 0);
    std::vector<std::pair<size_t, size_t>> tiles;
    rcb(m->xc, ids, 0, (size_t)n, cap0, tiles);

    auto other_of = [&](int64_t c, int sl) -> int64_t {
        const int64_t f = slots[c][sl];
        if (F.nbr[f] < 0) return -1;
        return F.own[f] == c ? F.nbr[f] : F.own[f];
    };
    std::vector<int32_t> stamp(n, -1), local(n, 0), fstamp(F.nf, -1);
    struct TileHalo { std::vector<int32_t> r1, r2; };
    std::vector<TileHalo> halos;
    std::vector<std::pair<size_t, size_t>> final_tiles;
    int32_t tag = 0;
    for (size_t ti = 0; ti < tiles.size(); ti++) {
        const auto [lo, hi] = tiles[ti];
        tag++;
        for (size_t i = lo; i < hi; i++) stamp[ids[i]] = tag;
        TileHalo h;
        size_t n_faces = 0;
        for (size_t i = lo; i < hi; i++)
            for (int sl = 0; sl < nslot[ids[i]]; sl++) {
                const int64_t kc = other_of(ids[i], sl);
                if (kc >= 0 && stamp[kc] != tag) { stamp[kc] = tag; h.r1.push_back((int32_t)kc); }
                const int64_t f = slots[ids[i]][sl];
                if (fstamp[f] != tag) { fstamp[f] = tag; n_faces++; }
            }
        for (int32_t c1 : h.r1)
            for (int sl = 0; sl < nslot[c1]; sl++) {
                const int64_t kc = other_of(c1, sl);
                if (kc >= 0 && stamp[kc] != tag) { stamp[kc] = tag; h.r2.push_back((int32_t)kc); }
            }
        const size_t nint = hi - lo;
        if (nint + h.r1.size() + h.r2.size() > (size_t)LOC_MAX || nint + h.r1.size() > (size_t)SIG_MAX ||
            n_faces > (size_t)LF_MAX) {
            if (nint <= 8) return fail(SDUGKS_ERR_INVALID_MESH, "halo of a %zu-cell tile does not fit", nint);
            std::vector<std::pair<size_t, size_t>> sub;
            rcb(m->xc, ids, lo, hi, (nint + 1) / 2, sub);
            tiles.insert(tiles.begin() + ti + 1, sub.begin(), sub.end());
            continue;
        }
        final_tiles.push_back(tiles[ti]);
        halos.push_back(std::move(h));
    }
    const int32_t nt = (int32_t)final_tiles.size();
    // within a tile, cells along a Morton curve of their centroids (16 bits per axis over
    // the tile's bounding box): faces, which are listed in the order of their cells,
    // then read nearby local indices from one warp to the next lane
    for (const auto &t : final_tiles) {
        double mn[2] = {INFINITY, INFINITY}, mx[2] = {-INFINITY, -INFINITY};
        for (size_t i = t.first; i < t.second; i++)
            for (int d = 0; d < 2; d++) {
                mn[d] = std::min(mn[d], m->xc[2 * ids[i] + d]);
                mx[d] = std::max(mx[d], m->xc[2 * ids[i] + d]);
            }
        auto key = [&](int32_t c) {
            uint32_t q[2];
            for (int d = 0; d < 2; d++) {
                const double w = mx[d] - mn[d];
                const double u = w > 0 ? (m->xc[2 * c + d] - mn[d]) / w : 0.0;
                q[d] = (uint32_t)std::min(65535.0, std::max(0.0, std::floor(u * 65536.0)));
            }
            uint64_t k = 0;
            for (int b = 15; b >= 0; b--) k = (k << 2) | (((q[1] >> b) & 1u) << 1) | ((q[0] >> b) & 1u);
            return k;
        };
        std::sort(ids.begin() + t.first, ids.begin() + t.second, [&](int32_t a, int32_t b) {
            const uint64_t ka = key(a), kb = key(b);
            return ka != kb ? ka < kb : a < b;
        });
    }
    // internal order: tiles in RCB order
    std::vector<int32_t> perm(n), iperm(n);
    {
        int64_t q = 0;
        for (auto &t : final_tiles)
            for (size_t i = t.first; i < t.second; i++) perm[q++] = ids[i];
        for (int64_t i = 0; i < n; i++) iperm[perm[i]] = (int32_t)i;
    }

    const int64_t npad = (n + 31) / 32 * 32;
    std::vector<int32_t> tile_c0(nt + 1), tile_h0(nt + 1), tile_nh1(nt), tile_s0(nt + 1), tile_f0(nt + 1), tile_nlf(nt), halo;
    int64_t lf_total = 0;            // local faces of all tiles without the padding
    std::vector<uint16_t> sig_nb, cell_lf((size_t)MAXF * npad, LF_NONE);
    std::vector<int32_t> sig_cell;   // internal cell of each gradient row
    std::vector<uint32_t> lf_ab;
    std::vector<int32_t> lf_bface;  // boundary-face row of each local face (-1: none)
    std::vector<int64_t> brow;
    const int64_t n_bfaces = boundary_rows(*m, brow);
    std::vector<double> lf_geo;   // [n_lf][6], transposed at upload
    std::vector<uint8_t> islk((size_t)MAXF * npad, SK_NONE);
    std::vector<double> iainv(3 * npad, 0.0), ivol(npad, 1.0), idtv(npad, 0.0);
    // x_k - x_j across each interior slot, formed in the compute precision from the
    // two face-centre offsets as they are stored for the kernel
    const int prec = prm->precision;
    const size_t rs = prec == P_FP64 ? sizeof(double) : sizeof(float);
    std::vector<char> isld((size_t)MAXF * 2 * npad * rs, 0);
    for (int64_t i = 0; i < n; i++) {
        const int64_t c = perm[i];
        for (int sl = 0; sl < MAXF; sl++) {
            const uint8_t kd = skind[(size_t)c * MAXF + sl];
            islk[(size_t)sl * npad + i] = kd;
            if (kd != SK_INTERIOR && !(kd < MAXPATCH && m->bc_kind[kd] == SDUGKS_BC_SYMMETRY)) continue;
            const double *G = &sgeo[((size_t)c * MAXF + sl) * 6];
            for (int q = 0; q < 2; q++) {
                const size_t at = ((size_t)(2 * sl + q) * npad + i) * rs;
                if (prec == P_FP64) {
                    const double v = G[2 + q] - G[4 + q];
                    std::memcpy(&isld[at], &v, rs);
                } else {
                    const float v = (float)G[2 + q] - (float)G[4 + q];
                    std::memcpy(&isld[at], &v, rs);
                }
            }
        }
        for (int d = 0; d < 3; d++) iainv[d * npad + i] = ainv[3 * c + d];
        ivol[i] = m->vol[c];
        idtv[i] = prm->dt / m->vol[c];
    }
    int64_t halo_total = 0, sig_total = 0;
    std::vector<int32_t> flocal(F.nf, 0);
    {
        int32_t c0 = 0, hoff = 0, soff = 0;
        for (int32_t t = 0; t < nt; t++) {
            const int32_t nint = (int32_t)(final_tiles[t].second - final_tiles[t].first);
            tile_c0[t] = c0; tile_h0[t] = hoff; tile_s0[t] = soff;
            std::vector<int32_t> r1, r2;
            for (int32_t c : halos[t].r1) r1.push_back(iperm[c]);
            for (int32_t c : halos[t].r2) r2.push_back(iperm[c]);
            std::sort(r1.begin(), r1.end());
            std::sort(r2.begin(), r2.end());
            tile_nh1[t] = (int32_t)r1.size();
            // local numbering: interior, ring 1, ring 2
            for (int32_t i = 0; i < nint; i++) local[c0 + i] = i;
            for (size_t q = 0; q < r1.size(); q++) local[r1[q]] = nint + (int32_t)q;
            for (size_t q = 0; q < r2.size(); q++) local[r2[q]] = nint + (int32_t)(r1.size() + q);
            halo.insert(halo.end(), r1.begin(), r1.end());
            halo.insert(halo.end(), r2.begin(), r2.end());
            auto push_sig = [&](int32_t i) {
                std::array<uint16_t, MAXF> row;
                row.fill(NO_LOCAL);
                const int64_t c = perm[i];
                for (int sl = 0; sl < nslot[c]; sl++) {
                    const int64_t kc = other_of(c, sl);
                    if (kc >= 0) row[sl] = (uint16_t)local[iperm[kc]];
                    const uint8_t kd = skind[(size_t)c * MAXF + sl];
                    if (kd != SK_INTERIOR && m->bc_kind[kd] == SDUGKS_BC_SYMMETRY) {
                        const double *G = &sgeo[((size_t)c * MAXF + sl) * 6];
                        row[sl] = std::fabs(G[0]) > std::fabs(G[1]) ? SYM_X : SYM_Y;
                    }
                }
                sig_nb.insert(sig_nb.end(), row.begin(), row.end());
                sig_cell.push_back(i);
            };
            for (int32_t i = 0; i < nint; i++) push_sig(c0 + i);
            for (int32_t c : r1) push_sig(c);
            // pad the tile's rows to a multiple of 4 so that every tile's gradient data
            // starts 16-byte aligned (the kernel copies it in 16-byte pieces)
            const int32_t nsig_t = nint + (int32_t)r1.size(), npad_t = (nsig_t + 3) / 4 * 4;
            for (int32_t q = nsig_t; q < npad_t; q++) {
                for (int sl = 0; sl < MAXF; sl++) sig_nb.push_back(NO_LOCAL);
                sig_cell.push_back(-1);
            }
            // local faces, in order of first appearance over the tile's cells and slots;
            // oriented from the merged face's owner to its neighbour (or boundary)
            tile_f0[t] = (int32_t)lf_ab.size();
            for (int32_t i = 0; i < nint; i++) {
                const int64_t c = perm[c0 + i];
                for (int sl = 0; sl < nslot[c]; sl++) {
                    const int64_t f = slots[c][sl];
                    if (fstamp[f] != -2 - t) {
                        fstamp[f] = -2 - t;
                        flocal[f] = (int32_t)lf_ab.size() - tile_f0[t];
                        const uint32_t a = (uint32_t)local[iperm[F.own[f]]];
                        const uint32_t b = F.nbr[f] >= 0 ? (uint32_t)local[iperm[F.nbr[f]]]
                                                         : (LF_BOUNDARY | (uint32_t)(-1 - F.nbr[f]));
                        lf_ab.push_back(a | (b << 16));
                        lf_bface.push_back(F.nbr[f] >= 0 ? -1 : (int32_t)brow[F.orig[f]]);
                        const double q6[6] = {F.nl[2 * f], F.nl[2 * f + 1], F.ro[2 * f], F.ro[2 * f + 1],
                                              F.rk[2 * f], F.rk[2 * f + 1]};
                        lf_geo.insert(lf_geo.end(), q6, q6 + 6);
                    }
                    const bool second = F.own[f] != c;
                    cell_lf[(size_t)sl * npad + c0 + i] = (uint16_t)(flocal[f] | (second ? LF_SECOND : 0));
                }
            }
            // the next tile's faces start at a multiple of 4 (16-byte pieces of every
            // face array); padding entries are never read as faces
            tile_nlf[t] = (int32_t)lf_ab.size() - tile_f0[t];
            lf_total += tile_nlf[t];
            while (lf_ab.size() % 4 != 0) {
                lf_ab.push_back(0u);
                lf_bface.push_back(-1);
                lf_geo.insert(lf_geo.end(), 6, 0.0);
            }
            c0 += nint;
            hoff += (int32_t)(r1.size() + r2.size());
            soff += (nint + (int32_t)r1.size() + 3) / 4 * 4;
            halo_total += (int64_t)(r1.size() + r2.size());
            sig_total += nint + (int64_t)r1.size();
        }
        tile_c0[nt] = c0; tile_h0[nt] = hoff; tile_s0[nt] = soff; tile_f0[nt] = (int32_t)lf_ab.size();
    }

    // ---- every index the kernel dereferences is checked here, on the host
    for (int32_t t = 0; t < nt; t++) {
        const int32_t nint = tile_c0[t + 1] - tile_c0[t];
        const int32_t nloc = nint + (tile_h0[t + 1] - tile_h0[t]);
        const int32_t nsig = nint + tile_nh1[t];
        if (nint < 1 || nint > TILE_MAX || nloc > LOC_MAX || nsig > SIG_MAX || tile_s0[t] % 4 != 0 ||
            tile_s0[t + 1] - tile_s0[t] != (nsig + 3) / 4 * 4)
            return fail(SDUGKS_ERR_INVALID_MESH, "internal: tile %d sizes out of range", t);
        for (int32_t q = tile_h0[t]; q < tile_h0[t + 1]; q++)
            if (halo[q] < 0 || halo[q] >= n) return fail(SDUGKS_ERR_INVALID_MESH, "internal: halo id out of range");
        for (int32_t i = 0; i < nsig; i++) {
            const int32_t g = i < nint ? tile_c0[t] + i : halo[tile_h0[t] + i - nint];
            for (int sl = 0; sl < MAXF; sl++) {
                const uint16_t v = sig_nb[((size_t)tile_s0[t] + i) * MAXF + sl];
                const uint8_t kd = islk[(size_t)sl * npad + g];
                const bool sym = kd != SK_INTERIOR && kd != SK_NONE && kd < MAXPATCH &&
                                 m->bc_kind[kd] == SDUGKS_BC_SYMMETRY;
                if (sym != (v == SYM_X || v == SYM_Y))
                    return fail(SDUGKS_ERR_INVALID_MESH, "internal: symmetry slot without its mirror code");
                if (!sym && v != NO_LOCAL && v >= nloc)
                    return fail(SDUGKS_ERR_INVALID_MESH, "internal: gradient neighbour outside the tile's cells");
                if ((kd == SK_INTERIOR) != (!sym && v != NO_LOCAL))
                    return fail(SDUGKS_ERR_INVALID_MESH, "internal: slot kind and neighbour disagree");
                if (i < nint && kd == SK_INTERIOR && v >= nsig)
                    return fail(SDUGKS_ERR_INVALID_MESH, "internal: face neighbour outside ring 1");
            }
        }
        const int32_t nlf = tile_nlf[t];
        if (nlf < 1 || nlf > LF_MAX || tile_f0[t] % 4 != 0 || tile_f0[t + 1] - tile_f0[t] != (nlf + 3) / 4 * 4)
            return fail(SDUGKS_ERR_INVALID_MESH, "internal: tile %d face count out of range", t);
        for (int32_t q = tile_f0[t]; q < tile_f0[t] + nlf; q++) {
            const uint32_t a = lf_ab[q] & 0xFFFFu, b = lf_ab[q] >> 16;
            if ((b & LF_SECOND) == 0) {
                if (a >= (uint32_t)nsig || b >= (uint32_t)nsig || (a >= (uint32_t)nint && b >= (uint32_t)nint))
                    return fail(SDUGKS_ERR_INVALID_MESH, "internal: face sides outside the tile's gradient cells");
            } else {
                const uint32_t p = b & 0xFFu;
                if ((b & ~0xFFu) != LF_BOUNDARY || a >= (uint32_t)nint || p >= MAXPATCH ||
                    m->bc_kind[p] == SDUGKS_BC_UNSET || m->bc_kind[p] == SDUGKS_BC_PERIODIC)
                    return fail(SDUGKS_ERR_BAD_BC, "internal: boundary face without a usable condition");
            }
        }
        for (int32_t i = 0; i < nint; i++)
            for (int sl = 0; sl < MAXF; sl++) {
                const uint16_t v = cell_lf[(size_t)sl * npad + tile_c0[t] + i];
                const bool none = islk[(size_t)sl * npad + tile_c0[t] + i] == SK_NONE;
                if (none != (v == LF_NONE)) return fail(SDUGKS_ERR_INVALID_MESH, "internal: slot without its face");
                if (none) continue;
                const int32_t lf = v & (LF_SECOND - 1);
                if (lf >= nlf) return fail(SDUGKS_ERR_INVALID_MESH, "internal: local face out of range");
                const uint32_t ab = lf_ab[tile_f0[t] + lf];
                const uint32_t side = (v & LF_SECOND) ? ab >> 16 : ab & 0xFFFFu;
                if (side != (uint32_t)i) return fail(SDUGKS_ERR_INVALID_MESH, "internal: face side is not the cell");
            }
    }

    // ---- device allocation (one arena) and upload
    sdugks_solver *s = new (std::nothrow) sdugks_solver;
    if (!s) return fail(SDUGKS_ERR_OOM, "host allocation failed");
    s->p = *prm;
    if (s->p.graph_steps == 0) s->p.graph_steps = 64;
    if (s->p.graph_steps > 0) s->p.graph_steps = std::max(2, s->p.graph_steps / 2 * 2);
    s->n_bfaces = n_bfaces;
    s->stream = static_cast<cudaStream_t>(stream);
    s->n = n; s->npad = npad; s->nf = F.nf; s->n_tiles = nt; s->halo_cells = halo_total;
    s->kernel = SDUGKS_KERNEL_TILED;
    const size_t fs = prec == P_FP64 ? 8 : (prec == P_FP32 ? 4 : 2);
    s->n_red_blocks = residual_blocks(n);

    auto layout = [&](Arena &A) {
        s->perm = A.take<int32_t>(npad);
        s->vol = A.take<double>(npad);
        s->snap = A.take<double>(2 * npad);
        s->partial = A.take<double>(4 * (size_t)s->n_red_blocks);
        s->red = A.take<double>(5);
        for (int b = 0; b < 2; b++) s->st.f[b] = A.take<char>(NQ * npad * fs);
        for (int b = 0; b < 2; b++) s->st.W[b] = A.take<double>(3 * npad);
        s->tm.tile_c0 = A.take<int32_t>(nt + 1);
        s->tm.tile_h0 = A.take<int32_t>(nt + 1);
        s->tm.tile_nh1 = A.take<int32_t>(nt);
        s->tm.tile_s0 = A.take<int32_t>(nt + 1);
        s->tm.halo = A.take<int32_t>(std::max<size_t>(1, halo.size()));
        s->tm.sig_nb = A.take<uint16_t>(sig_nb.size());
        s->tm.tile_f0 = A.take<int32_t>(nt + 1);
        s->tm.tile_nlf = A.take<int32_t>(nt);
        s->tm.sig_d = A.take<char>((size_t)MAXF * 2 * sig_cell.size() * rs);
        s->tm.sig_ai = A.take<char>((size_t)3 * sig_cell.size() * rs);
        s->tm.cell_lf = A.take<uint16_t>(cell_lf.size());
        s->tm.lf_ab = A.take<uint32_t>(lf_ab.size());
        s->tm.lf_bface = A.take<int32_t>(lf_bface.size());
        s->tm.lf_geo = A.take<char>(lf_geo.size() * rs);
        s->tm.dtV = A.take<char>(npad * rs);
        s->tm.vol = s->vol;
    };
    Arena A0;
    layout(A0);
    s->dbytes = A0.used + 256;
    cudaError_t e = cudaGetDevice(&s->device);
    if (e == cudaSuccess) e = cudaMalloc(&s->dmem, s->dbytes);
    if (e != cudaSuccess) {
        delete s;
        return fail(e == cudaErrorMemoryAllocation ? SDUGKS_ERR_OOM : SDUGKS_ERR_CUDA, "cudaMalloc(%zu): %s",
                    A0.used, cudaGetErrorString(e));
    }
    Arena A{s->dmem, 0, s->dbytes};
    layout(A);
    s->tm.n_tiles = nt; s->tm.n = n; s->tm.npad = npad; s->tm.n_lf = (int64_t)lf_ab.size();

    auto conv = [&](const std::vector<double> &v) {
        std::vector<char> o(v.size() * rs);
        if (prec == P_FP64) std::memcpy(o.data(), v.data(), o.size());
        else {
            float *q = reinterpret_cast<float *>(o.data());
            for (size_t i = 0; i < v.size(); i++) q[i] = (float)v[i];
        }
        return o;
    };
    std::vector<int32_t> permpad(npad, 0);
    std::copy(perm.begin(), perm.end(), permpad.begin());
    auto up = [&](const void *dst, const void *src, size_t bytes) {
        return cudaMemcpy(const_cast<void *>(dst), src, bytes, cudaMemcpyHostToDevice);
    };
    std::vector<double> lgeo_t(lf_geo.size());
    {
        const size_t nlf = lf_ab.size();
        for (size_t q = 0; q < nlf; q++)
            for (int d = 0; d < 6; d++) lgeo_t[d * nlf + q] = lf_geo[q * 6 + d];
    }
    const std::vector<char> ggeo = conv(lgeo_t), gdtv = conv(idtv);
    // gradient data per row (tile cells and ring 1 of every tile), SoA over the rows
    const size_t nrow = sig_cell.size();
    std::vector<char> gsd((size_t)MAXF * 2 * nrow * rs), gsa((size_t)3 * nrow * rs);
    {
        const std::vector<char> gainv = conv(iainv);
        for (size_t r = 0; r < nrow; r++) {
            if (sig_cell[r] < 0) continue;             // padding row: zeros
            const size_t i = (size_t)sig_cell[r];
            for (int k = 0; k < 2 * MAXF; k++)
                std::memcpy(&gsd[((size_t)k * nrow + r) * rs], &isld[((size_t)k * npad + i) * rs], rs);
            for (int k = 0; k < 3; k++)
                std::memcpy(&gsa[((size_t)k * nrow + r) * rs], &gainv[((size_t)k * npad + i) * rs], rs);
        }
    }
    s->tm.n_sig = (int64_t)nrow;
    int rc2 = SDUGKS_OK;
    auto chk = [&](cudaError_t ee, const char *what) {
        if (ee != cudaSuccess && rc2 == SDUGKS_OK) rc2 = fail(SDUGKS_ERR_CUDA, "%s: %s", what, cudaGetErrorString(ee));
    };
    chk(cudaMemset(s->dmem, 0, s->dbytes), "memset");
    chk(up(s->perm, permpad.data(), npad * 4), "upload perm");
    chk(up(s->vol, ivol.data(), npad * 8), "upload vol");
    chk(up(s->tm.tile_c0, tile_c0.data(), (nt + 1) * 4), "upload tiles");
    chk(up(s->tm.tile_h0, tile_h0.data(), (nt + 1) * 4), "upload tiles");
    chk(up(s->tm.tile_nh1, tile_nh1.data(), nt * 4), "upload tiles");
    chk(up(s->tm.tile_s0, tile_s0.data(), (nt + 1) * 4), "upload tiles");
    if (!halo.empty()) chk(up(s->tm.halo, halo.data(), halo.size() * 4), "upload halo");
    chk(up(s->tm.sig_nb, sig_nb.data(), sig_nb.size() * 2), "upload sig_nb");
    chk(up(s->tm.tile_f0, tile_f0.data(), (nt + 1) * 4), "upload tiles");
    chk(up(s->tm.tile_nlf, tile_nlf.data(), nt * 4), "upload tiles");
    chk(up(s->tm.sig_d, gsd.data(), gsd.size()), "upload gradient offsets");
    chk(up(s->tm.sig_ai, gsa.data(), gsa.size()), "upload LLSR inverse");
    chk(up(s->tm.cell_lf, cell_lf.data(), cell_lf.size() * 2), "upload cell faces");
    chk(up(s->tm.lf_ab, lf_ab.data(), lf_ab.size() * 4), "upload face sides");
    chk(up(s->tm.lf_bface, lf_bface.data(), lf_bface.size() * 4), "upload boundary rows");
    chk(up(s->tm.lf_geo, ggeo.data(), ggeo.size()), "upload face geometry");
    chk(up(s->tm.dtV, gdtv.data(), gdtv.size()), "upload dtV");
    chk(cudaMallocHost(&s->h_red, 5 * sizeof(double)), "cudaMallocHost");
    chk(cudaStreamCreateWithFlags(&s->cap_stream, cudaStreamNonBlocking), "cudaStreamCreate");
    chk((cudaError_t)prepare(prec, SDUGKS_KERNEL_TILED), "kernel attributes");
    if (rc2) { sdugks_solver_destroy(s); return rc2; }

    fill_coefs(s->coefs, *m, prm->tau, prm->dt);
    // mesh bytes the tiled kernel reads per interior cell and step: the slot list of
    // its own cell, the tile's local faces (sides and 6 geometry values), gradient
    // data (d vectors, inverse, neighbour indices) of interior and ring-1 cells, halo
    // ids and dt/V
    {
        const double sigc = (double)sig_total / n, lfc = (double)lf_total / n;
        s->mesh_bytes = MAXF * 2 + lfc * (4 + 6 * rs) + sigc * (MAXF * (2 + 2 * rs) + 3 * rs) +
                        (double)halo_total / n * 4 + rs;
    }
    *out = s;
    return SDUGKS_OK;
}

static int ensure_staging(sdugks_solver *s)
{
    if (s->staging) return SDUGKS_OK;
    CUDA_TRY(cudaSetDevice(s->device));
    CUDA_TRY(cudaMalloc(&s->staging, sizeof(double) * 12 * (size_t)std::max<int64_t>(s->n, 1)));
    return SDUGKS_OK;
}

static int snapshot(sdugks_solver *s, double *eps, double *mass)
{
    CUDA_TRY(launch_residual(s->n, s->npad, s->loc, s->st.W[s->cur], rho_ref_of(s->p.precision), s->vol, s->snap,
                             s->partial, s->n_red_blocks, s->red,
                             s->stream));
    CUDA_TRY(cudaMemcpyAsync(s->h_red, s->red, 5 * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    CUDA_TRY(cudaStreamSynchronize(s->stream));
    int32_t err_flag;
    std::memcpy(&err_flag, &s->h_red[4], sizeof err_flag);
    if (err_flag != 0) {
        // blocks of some launch since the last check skipped their update: no result of
        // the state is usable until init or set_state; the flag is cleared for that
        s->initialised = false;
        CUDA_TRY(cudaMemsetAsync(s->red + 4, 0, sizeof(int32_t), s->stream));
        CUDA_TRY(cudaStreamSynchronize(s->stream));
        return fail(SDUGKS_ERR_TIMEOUT, "a TMA staging copy of the Cartesian step did not complete within its wait "
                                        "limit; the state is invalid until init or set_state");
    }
    const double num = s->h_red[0], den = s->h_red[1];
    if (mass) *mass = s->h_red[2];
    if (s->h_red[3] != 0.0) {
        if (eps) *eps = NAN;
        return fail(SDUGKS_ERR_DIVERGED, "%g cells hold non-finite or zero-density W after %lld steps", s->h_red[3],
                    (long long)s->steps_done);
    }
    if (eps) *eps = den > 0.0 ? std::sqrt(num) / std::sqrt(den) : INFINITY;
    return SDUGKS_OK;
}

extern "C" int sdugks_init(sdugks_solver *s, const double *rho, const double *u)
{
    if (!s) return fail(SDUGKS_ERR_INVALID_ARG, "solver is NULL");
    CUDA_TRY(cudaSetDevice(s->device));
    int rc = ensure_staging(s);
    if (rc) return rc;
    double *d_rho = rho ? s->staging : nullptr;
    double *d_u = u ? s->staging + s->n : nullptr;
    if (rho) CUDA_TRY(cudaMemcpyAsync(d_rho, rho, sizeof(double) * s->n, cudaMemcpyHostToDevice, s->stream));
    if (u) CUDA_TRY(cudaMemcpyAsync(d_u, u, sizeof(double) * 2 * s->n, cudaMemcpyHostToDevice, s->stream));
    s->cur = 0; s->steps_done = 0;
    CUDA_TRY(launch_init_state(s->p.precision, s->n, s->npad, s->perm, s->loc, d_rho, d_u, s->st.f[0], s->st.W[0], s->stream));
    CUDA_TRY(cudaMemsetAsync(s->red + 4, 0, sizeof(int32_t), s->stream));   // a new state: no failed launch
    s->initialised = true;
    return snapshot(s, nullptr, nullptr);
}

// A graph of L (even) steps captured from buffer phase 0; it leaves the phase unchanged.
static int capture_steps(sdugks_solver *s, int L, cudaGraphExec_t *out)
{
    const int cur0 = s->cur;
    s->cur = 0;
    cudaGraph_t g = nullptr;
    CUDA_TRY(cudaStreamBeginCapture(s->cap_stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < L && e == cudaSuccess; k++) e = launch_one(s, s->cap_stream);
    cudaError_t e2 = cudaStreamEndCapture(s->cap_stream, &g);
    s->cur = cur0;
    CUDA_TRY(e);
    CUDA_TRY(e2);
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    CUDA_TRY(e);
    return SDUGKS_OK;
}

static int ensure_graph(sdugks_solver *s)
{
    if (s->graph) return SDUGKS_OK;
    int rc = capture_steps(s, s->p.graph_steps, &s->graph);
    if (rc) return rc;
    s->graph_len = s->p.graph_steps;
    return SDUGKS_OK;
}

extern "C" int sdugks_step(sdugks_solver *s, int64_t n)
{
    if (!s) return fail(SDUGKS_ERR_INVALID_ARG, "solver is NULL");
    if (n < 0) return fail(SDUGKS_ERR_INVALID_ARG, "negative step count");
    if (!s->initialised) return fail(SDUGKS_ERR_STATE, "step before init or set_state");
    CUDA_TRY(cudaSetDevice(s->device));
    int64_t left = n;
    const int G = s->p.graph_steps;
    if (G > 0 && left >= 2 * G) {
        while (left > 0 && s->cur != 0) {
            CUDA_TRY(launch_one(s, s->stream));
            s->steps_done++; left--;
        }
        int rc = ensure_graph(s);
        if (rc) return rc;
        while (left >= G) {
            CUDA_TRY(cudaGraphLaunch(s->graph, s->stream));
            s->steps_done += G; left -= G;
            // a graph of G (even) steps leaves the buffer phase unchanged
        }
        // the remainder in graphs of 2^k steps (each captured at its first use): a
        // replayed step costs about 10 % less than a launch of its own
        for (int k = 30; k >= 1; k--) {
            const int64_t L = int64_t(1) << k;
            if (L >= G || left < L) continue;
            if (!s->tail[k]) {
                rc = capture_steps(s, (int)L, &s->tail[k]);
                if (rc) return rc;
            }
            CUDA_TRY(cudaGraphLaunch(s->tail[k], s->stream));
            s->steps_done += L; left -= L;
        }
    }
    while (left > 0) {
        CUDA_TRY(launch_one(s, s->stream));
        s->steps_done++; left--;
    }
    return SDUGKS_OK;
}

extern "C" int sdugks_step_boundary_flux(sdugks_solver *s, double *force, double *face_flux)
{
    if (!s) return fail(SDUGKS_ERR_INVALID_ARG, "solver is NULL");
    if (!s->initialised) return fail(SDUGKS_ERR_STATE, "step before init or set_state");
    CUDA_TRY(cudaSetDevice(s->device));
    if (force && !s->d_force) CUDA_TRY(cudaMalloc(&s->d_force, sizeof(double) * 2 * MAXPATCH));
    if (face_flux && s->n_bfaces > 0 && !s->d_bface)
        CUDA_TRY(cudaMalloc(&s->d_bface, sizeof(double) * 2 * (size_t)s->n_bfaces));
    double *d_force = force ? s->d_force : nullptr;
    double *d_bface = face_flux && s->n_bfaces > 0 ? s->d_bface : nullptr;
    if (d_force) CUDA_TRY(cudaMemsetAsync(d_force, 0, sizeof(double) * 2 * MAXPATCH, s->stream));
    cudaError_t e;
    if (s->kernel == SDUGKS_KERNEL_CARTESIAN) {
        CartInst ci = s->ci;
        ci.force = d_force;                    // per grid side
        ci.bface = d_bface;
        e = launch_step_cart(s->p.precision, s->cart_shape, ci, s->tma, s->cart_general, s->cur, s->stream);
    } else {
        TiledMesh tm = s->tm;
        tm.force = d_force;                    // per patch
        tm.bface = d_bface;
        const int a = s->cur;
        e = s->p.precision == P_FP64
                ? launch_step_tiled_fp64(tm, s->coefs, s->st.f[a], s->st.f[1 - a], s->st.W[a], s->st.W[1 - a], s->stream)
                : launch_step_tiled_fp32(s->p.precision, tm, s->coefs, s->st.f[a], s->st.f[1 - a], s->st.W[a],
                                         s->st.W[1 - a], s->stream);
    }
    CUDA_TRY(e);
    s->cur = 1 - s->cur;
    s->steps_done++;
    double h[2 * MAXPATCH];
    if (d_force) CUDA_TRY(cudaMemcpyAsync(h, d_force, sizeof h, cudaMemcpyDeviceToHost, s->stream));
    if (d_bface)
        CUDA_TRY(cudaMemcpyAsync(face_flux, d_bface, sizeof(double) * 2 * (size_t)s->n_bfaces, cudaMemcpyDeviceToHost,
                                 s->stream));
    CUDA_TRY(cudaStreamSynchronize(s->stream));
    if (force) {
        for (int q = 0; q < 2 * MAXPATCH; q++) force[q] = 0.0;
        if (s->kernel == SDUGKS_KERNEL_CARTESIAN) {
            for (int side = 0; side < 4; side++) {
                const int p = s->side_patch[side];
                if (p < 0 || s->coefs.bc_kind[p] == SDUGKS_BC_PERIODIC) continue;
                force[2 * p] += h[2 * side];
                force[2 * p + 1] += h[2 * side + 1];
            }
        } else {
            for (int q = 0; q < 2 * MAXPATCH; q++) force[q] = h[q];
        }
    }
    return SDUGKS_OK;
}

extern "C" int sdugks_step_forces(sdugks_solver *s, double *force)
{
    if (!s || !force) return fail(SDUGKS_ERR_INVALID_ARG, "NULL argument");
    return sdugks_step_boundary_flux(s, force, nullptr);
}

extern "C" int sdugks_get_macros_device(sdugks_solver *s, double *d_rho, double *d_u)
{
    if (!s) return fail(SDUGKS_ERR_INVALID_ARG, "solver is NULL");
    if (!s->initialised) return fail(SDUGKS_ERR_STATE, "get_macros before init");
    CUDA_TRY(cudaSetDevice(s->device));
    CUDA_TRY(launch_macros(s->n, s->npad, s->perm, s->loc, s->st.W[s->cur], rho_ref_of(s->p.precision), d_rho, d_u,
                           s->stream));
    return SDUGKS_OK;
}

extern "C" int sdugks_get_macros(sdugks_solver *s, double *rho, double *u)
{
    if (!s) return fail(SDUGKS_ERR_INVALID_ARG, "solver is NULL");
    if (!s->initialised) return fail(SDUGKS_ERR_STATE, "get_macros before init");
    CUDA_TRY(cudaSetDevice(s->device));
    int rc = ensure_staging(s);
    if (rc) return rc;
    CUDA_TRY(launch_macros(s->n, s->npad, s->perm, s->loc, s->st.W[s->cur], rho_ref_of(s->p.precision), s->staging,
                           s->staging + s->n, s->stream));
    if (rho) CUDA_TRY(cudaMemcpyAsync(rho, s->staging, sizeof(double) * s->n, cudaMemcpyDeviceToHost, s->stream));
    if (u) CUDA_TRY(cudaMemcpyAsync(u, s->staging + s->n, sizeof(double) * 2 * s->n, cudaMemcpyDeviceToHost, s->stream));
    CUDA_TRY(cudaStreamSynchronize(s->stream));
    return SDUGKS_OK;
}

extern "C" int sdugks_residual(sdugks_solver *s, double *eps, double *mass)
{
    if (!s) return fail(SDUGKS_ERR_INVALID_ARG, "solver is NULL");
    if (!s->initialised) return fail(SDUGKS_ERR_STATE, "residual before init");
    CUDA_TRY(cudaSetDevice(s->device));
    return snapshot(s, eps, mass);
}

extern "C" int sdugks_get_state(sdugks_solver *s, double *f, double *W)
{
    if (!s) return fail(SDUGKS_ERR_INVALID_ARG, "solver is NULL");
    if (!s->initialised) return fail(SDUGKS_ERR_STATE, "get_state before init");
    CUDA_TRY(cudaSetDevice(s->device));
    int rc = ensure_staging(s);
    if (rc) return rc;
    double *df = s->staging, *dW = s->staging + 9 * s->n;
    CUDA_TRY(launch_pack_state(s->p.precision, s->n, s->npad, s->perm, s->loc, s->st.f[s->cur], s->st.W[s->cur], df, dW,
                               s->stream));
    if (f) CUDA_TRY(cudaMemcpyAsync(f, df, sizeof(double) * 9 * s->n, cudaMemcpyDeviceToHost, s->stream));
    if (W) CUDA_TRY(cudaMemcpyAsync(W, dW, sizeof(double) * 3 * s->n, cudaMemcpyDeviceToHost, s->stream));
    CUDA_TRY(cudaStreamSynchronize(s->stream));
    return SDUGKS_OK;
}

extern "C" int sdugks_set_state(sdugks_solver *s, const double *f, const double *W)
{
    if (!s) return fail(SDUGKS_ERR_INVALID_ARG, "solver is NULL");
    if (!f || !W) return fail(SDUGKS_ERR_INVALID_ARG, "f and W are required");
    CUDA_TRY(cudaSetDevice(s->device));
    int rc = ensure_staging(s);
    if (rc) return rc;
    double *df = s->staging, *dW = s->staging + 9 * s->n;
    CUDA_TRY(cudaMemcpyAsync(df, f, sizeof(double) * 9 * s->n, cudaMemcpyHostToDevice, s->stream));
    CUDA_TRY(cudaMemcpyAsync(dW, W, sizeof(double) * 3 * s->n, cudaMemcpyHostToDevice, s->stream));
    s->cur = 0; s->steps_done = 0;
    CUDA_TRY(launch_unpack_state(s->p.precision, s->n, s->npad, s->perm, s->loc, df, dW, s->st.f[0], s->st.W[0], s->stream));
    CUDA_TRY(cudaMemsetAsync(s->red + 4, 0, sizeof(int32_t), s->stream));   // a new state: no failed launch
    s->initialised = true;
    return snapshot(s, nullptr, nullptr);
}

namespace {
// Header of a raw checkpoint: the state is only meaningful to a solver of the same
// layout (precision, cell count and padding, kernel, tile size).
struct RawHeader {
    uint32_t magic;
    int32_t precision;
    int64_t n, npad;
    int32_t kernel, tile_cells;
};
constexpr uint32_t RAW_MAGIC = 0x31474453u;   // "SDG1"

size_t raw_f_bytes(const sdugks_solver *s)
{
    const size_t fs = s->p.precision == P_FP64 ? 8 : (s->p.precision == P_FP32 ? 4 : 2);
    return (size_t)NQ * (size_t)s->npad * fs;
}
RawHeader raw_header(const sdugks_solver *s)
{
    RawHeader h{};
    h.magic = RAW_MAGIC;
    h.precision = s->p.precision;
    h.n = s->n;
    h.npad = s->npad;
    h.kernel = s->kernel;
    h.tile_cells = s->kernel == SDUGKS_KERNEL_CARTESIAN ? 16 * CART_TY[s->cart_shape] : s->p.tile_cells;
    return h;
}
}  // namespace

extern "C" int sdugks_get_state_raw(sdugks_solver *s, void *buf, int64_t *bytes)
{
    if (!s || !bytes) return fail(SDUGKS_ERR_INVALID_ARG, "NULL argument");
    const size_t fb = raw_f_bytes(s), wb = sizeof(double) * 3 * (size_t)s->npad;
    const size_t total = sizeof(RawHeader) + fb + wb;
    if (!buf) { *bytes = (int64_t)total; return SDUGKS_OK; }
    if (*bytes < (int64_t)total) return fail(SDUGKS_ERR_INVALID_ARG, "raw state needs %zu bytes", total);
    if (!s->initialised) return fail(SDUGKS_ERR_STATE, "get_state_raw before init");
    CUDA_TRY(cudaSetDevice(s->device));
    const RawHeader h = raw_header(s);
    char *c = static_cast<char *>(buf);
    std::memcpy(c, &h, sizeof h);
    CUDA_TRY(cudaMemcpyAsync(c + sizeof h, s->st.f[s->cur], fb, cudaMemcpyDeviceToHost, s->stream));
    CUDA_TRY(cudaMemcpyAsync(c + sizeof h + fb, s->st.W[s->cur], wb, cudaMemcpyDeviceToHost, s->stream));
    CUDA_TRY(cudaStreamSynchronize(s->stream));
    *bytes = (int64_t)total;
    return SDUGKS_OK;
}

extern "C" int sdugks_set_state_raw(sdugks_solver *s, const void *buf, int64_t bytes)
{
    if (!s || !buf) return fail(SDUGKS_ERR_INVALID_ARG, "NULL argument");
    const size_t fb = raw_f_bytes(s), wb = sizeof(double) * 3 * (size_t)s->npad;
    const size_t total = sizeof(RawHeader) + fb + wb;
    if (bytes != (int64_t)total) return fail(SDUGKS_ERR_INVALID_ARG, "raw state of %lld bytes, this solver's is %zu",
                                             (long long)bytes, total);
    RawHeader h;
    std::memcpy(&h, buf, sizeof h);
    const RawHeader mine = raw_header(s);
    if (std::memcmp(&h, &mine, sizeof h) != 0)
        return fail(SDUGKS_ERR_INVALID_ARG, "raw state was taken from a solver of another layout");
    CUDA_TRY(cudaSetDevice(s->device));
    const char *c = static_cast<const char *>(buf);
    s->cur = 0; s->steps_done = 0;
    CUDA_TRY(cudaMemcpyAsync(s->st.f[0], c + sizeof h, fb, cudaMemcpyHostToDevice, s->stream));
    CUDA_TRY(cudaMemcpyAsync(s->st.W[0], c + sizeof h + fb, wb, cudaMemcpyHostToDevice, s->stream));
    CUDA_TRY(cudaMemsetAsync(s->red + 4, 0, sizeof(int32_t), s->stream));   // a new state: no failed launch
    s->initialised = true;
    return snapshot(s, nullptr, nullptr);
}

extern "C" int sdugks_solver_info(const sdugks_solver *s, sdugks_info *o)
{
    if (!s || !o) return fail(SDUGKS_ERR_INVALID_ARG, "NULL argument");
    std::memset(o, 0, sizeof *o);
    o->n_cells = s->n;
    o->n_faces = s->nf;
    o->n_tiles = s->n_tiles;
    o->halo_cells = s->halo_cells;
    o->steps_done = s->steps_done;
    o->device_bytes = (int64_t)s->dbytes + (s->staging ? (int64_t)(12 * sizeof(double) * s->n) : 0);
    const double fb = s->p.precision == P_FP64 ? 8 : (s->p.precision == P_FP32 ? 4 : 2);
    o->state_bytes_per_cell_step = 2 * NQ * fb + 2 * 3 * 8;   // f and W (FP64) read and written once
    o->mesh_bytes_per_cell_step = s->mesh_bytes;
    o->kernel = s->kernel;
    o->precision = s->p.precision;
    o->tile_cells = s->kernel == SDUGKS_KERNEL_CARTESIAN ? 16 * CART_TY[s->cart_shape] : (s->p.tile_cells ? s->p.tile_cells : TILE_MAX);
    o->nx = s->kernel == SDUGKS_KERNEL_CARTESIAN ? s->ci.nx : 0;
    o->ny = s->kernel == SDUGKS_KERNEL_CARTESIAN ? s->ci.ny : 0;
    o->staging = s->tma ? SDUGKS_STAGING_TMA : SDUGKS_STAGING_LOADS;
    o->n_boundary_faces = s->n_bfaces;
    o->one_code_path = s->cart_general ? 1 : 0;
    return SDUGKS_OK;
}

extern "C" void sdugks_solver_destroy(sdugks_solver *s)
{
    if (!s) return;
    cudaSetDevice(s->device);
    if (s->graph) cudaGraphExecDestroy(s->graph);
    for (cudaGraphExec_t t : s->tail)
        if (t) cudaGraphExecDestroy(t);
    if (s->cap_stream) cudaStreamDestroy(s->cap_stream);
    if (s->staging) cudaFree(s->staging);
    if (s->d_bface) cudaFree(s->d_bface);
    if (s->d_force) cudaFree(s->d_force);
    if (s->h_red) cudaFreeHost(s->h_red);
    if (s->dmem) cudaFree(s->dmem);
    delete s->tma;
    delete s;
}

// ------------------------------------------------------------------ autotuner

namespace {

// Fingerprint of a mesh and its boundary rules (FNV-1a over the caller's arrays): two
// solves of the same mesh share a tuning result whatever their tau and dt, which do
// not change the work of a step.
uint64_t mesh_fingerprint(const sdugks_mesh &m)
{
    uint64_t h = 1469598103934665603ull;
    auto mix = [&](const void *p, size_t n) {
        const unsigned char *c = static_cast<const unsigned char *>(p);
        for (size_t i = 0; i < n; i++) { h ^= c[i]; h *= 1099511628211ull; }
    };
    mix(&m.nc, sizeof m.nc);
    mix(&m.nf, sizeof m.nf);
    mix(m.xy.data(), m.xy.size() * sizeof(double));
    mix(m.own.data(), m.own.size() * sizeof(int64_t));
    mix(m.nbr.data(), m.nbr.size() * sizeof(int64_t));
    mix(m.bc_kind.data(), sizeof m.bc_kind);
    return h;
}

using TuneKey = std::tuple<int, uint64_t, int32_t, int32_t>;   // device, mesh, precision, kernel request
std::mutex g_tune_mu;
std::map<TuneKey, std::pair<sdugks_params, double>> g_tune_cache;

// Per-step time of one candidate: a solver with these parameters, at rest, one graph of
// warm-up, then `steps` steps (rounded up to whole graphs) between two events.
int time_candidate(const sdugks_mesh *m, const sdugks_params &p, int64_t steps, cudaStream_t st, double *ns)
{
    sdugks_solver *s = nullptr;
    int rc = sdugks_solver_create(m, &p, st, &s);
    if (rc) return rc;
    rc = sdugks_init(s, nullptr, nullptr);
    const int64_t G = s->p.graph_steps > 0 ? 2 * (int64_t)s->p.graph_steps : 2;
    const int64_t n = std::max<int64_t>(G, (steps + G - 1) / G * G);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float ms = 0.0f;
    if (!rc) rc = sdugks_step(s, G);
    if (!rc && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
        rc = fail(SDUGKS_ERR_CUDA, "autotune: cudaEventCreate");
    if (!rc && cudaEventRecord(e0, st) != cudaSuccess) rc = fail(SDUGKS_ERR_CUDA, "autotune: cudaEventRecord");
    if (!rc) rc = sdugks_step(s, n);
    if (!rc && cudaEventRecord(e1, st) != cudaSuccess) rc = fail(SDUGKS_ERR_CUDA, "autotune: cudaEventRecord");
    if (!rc) {
        cudaError_t e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) rc = fail(SDUGKS_ERR_CUDA, "autotune: %s", cudaGetErrorString(e));
    }
    if (!rc) {
        double eps = 0.0;
        rc = sdugks_residual(s, &eps, nullptr);      // a candidate that failed (TIMEOUT, DIVERGED) is not taken
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    sdugks_solver_destroy(s);
    if (!rc) *ns = 1e6 * (double)ms / (double)n;
    return rc;
}

}  // namespace

extern "C" int sdugks_autotune(const sdugks_mesh *m, const sdugks_params *base, int64_t steps, void *stream,
                               sdugks_params *best, sdugks_tune_info *info)
{
    if (!m || !base || !best || steps <= 0) return fail(SDUGKS_ERR_INVALID_ARG, "bad argument");
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    const TuneKey key{dev, mesh_fingerprint(*m), base->precision, base->kernel};
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            *best = *base;
            best->tile_cells = it->second.first.tile_cells;
            best->graph_steps = it->second.first.graph_steps;
            best->staging = it->second.first.staging;
            if (info) { std::memset(info, 0, sizeof *info); info->ns_per_step = it->second.second; info->from_cache = 1; }
            return SDUGKS_OK;
        }
    }
    // which kernel the solve takes decides the search space
    sdugks_params p0 = *base;
    p0.tile_cells = 0; p0.graph_steps = 0; p0.staging = SDUGKS_STAGING_LOADS;
    int32_t kernel = 0;
    {
        sdugks_solver *s = nullptr;
        int rc = sdugks_solver_create(m, &p0, stream, &s);
        if (rc) return rc;
        kernel = s->kernel;
        sdugks_solver_destroy(s);
    }
    std::vector<int32_t> tiles, stagings{SDUGKS_STAGING_LOADS};
    if (kernel == SDUGKS_KERNEL_CARTESIAN) {
        stagings.push_back(SDUGKS_STAGING_TMA);
        if (base->precision == P_FP64) tiles = {0};
        else tiles = {256, 224, 128};
    } else {
        tiles = {64, 96, 108, 120, 128};
    }
    const int32_t graphs[3] = {32, 64, 128};
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    double best_ns = 1e300;
    sdugks_params win = p0;
    int32_t n_cand = 0;
    for (int32_t t : tiles)
        for (int32_t sg : stagings)
            for (int32_t g : graphs) {
                sdugks_params p = p0;
                p.kernel = kernel;
                p.tile_cells = t;
                p.staging = sg;
                p.graph_steps = g;
                double ns = 0.0;
                const int rc = time_candidate(m, p, steps, st, &ns);
                if (rc == SDUGKS_ERR_OOM || rc == SDUGKS_ERR_CUDA) return rc;
                if (rc) continue;                    // a combination this mesh does not take
                n_cand++;
                if (ns < best_ns) { best_ns = ns; win = p; }
            }
    if (n_cand == 0) return fail(SDUGKS_ERR_INVALID_ARG, "autotune: no candidate configuration runs on this mesh");
    *best = *base;
    best->kernel = base->kernel;
    best->tile_cells = win.tile_cells;
    best->graph_steps = win.graph_steps;
    best->staging = win.staging;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[key] = {*best, best_ns};
    }
    if (info) {
        std::memset(info, 0, sizeof *info);
        info->ns_per_step = best_ns;
        info->candidates = n_cand;
        info->from_cache = 0;
        info->kernel = kernel;
    }
    return SDUGKS_OK;
}

extern "C" void sdugks_autotune_clear(void)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache.clear();
}

extern "C" const char *sdugks_last_error(void) { return g_err.c_str(); }

extern "C" const char *sdugks_version(void) { return "sdugks 0.1 sm_103a"; }

// ------------------------------------------------------------------ batched solves

namespace {

// First-fit allocator over [0, cap) in 256-byte units, with coalescing on free.
class PoolAlloc {
  public:
    explicit PoolAlloc(size_t cap = 0) { reset(cap); }
    void reset(size_t cap) { free_.clear(); if (cap) free_.push_back({0, cap}); cap_ = cap; used_ = 0; }
    bool alloc(size_t bytes, size_t &off) {
        bytes = (bytes + 255) & ~size_t(255);
        for (size_t k = 0; k < free_.size(); k++) {
            if (free_[k].second < bytes) continue;
            off = free_[k].first;
            free_[k].first += bytes;
            free_[k].second -= bytes;
            if (free_[k].second == 0) free_.erase(free_.begin() + k);
            used_ += bytes;
            return true;
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        bytes = (bytes + 255) & ~size_t(255);
        auto it = std::lower_bound(free_.begin(), free_.end(), std::make_pair(off, size_t(0)));
        it = free_.insert(it, {off, bytes});
        // merge with the next and the previous block
        if (it + 1 != free_.end() && it->first + it->second == (it + 1)->first) {
            it->second += (it + 1)->second;
            free_.erase(it + 1);
        }
        if (it != free_.begin() && (it - 1)->first + (it - 1)->second == it->first) {
            (it - 1)->second += it->second;
            free_.erase(it);
        }
        used_ -= bytes;
    }
    size_t used() const { return used_; }
    size_t cap() const { return cap_; }

  private:
    std::vector<std::pair<size_t, size_t>> free_;   // (offset, size), sorted by offset
    size_t cap_ = 0, used_ = 0;
};

struct BatchInst {
    int64_t id;
    CartInst ci;
    size_t off, bytes;
    int64_t admitted_at;            // batch step at admission
    int64_t ntiles;
    std::vector<int64_t> lattice;   // caller's cell c -> lattice position i + nx j
};

int64_t cart_npad(int32_t pitch, int32_t ny) { return ((int64_t)pitch * ny + 31) / 32 * 32; }

size_t inst_bytes(int prec, int64_t npad)
{
    const size_t fs = (prec == P_BF16DEV || prec == P_FP16DEV) ? 2 : 4;
    auto up = [](size_t x) { return (x + 255) & ~size_t(255); };
    return 2 * up(NQ * npad * fs) + 2 * up(3 * npad * 8) + up(2 * npad * 8);
}

}  // namespace

struct sdugks_batch {
    int device = 0;
    cudaStream_t stream = nullptr, cap_stream = nullptr;
    int32_t prec = P_FP32;
    int32_t max_inst = 0;
    char *pool = nullptr;
    PoolAlloc alloc;
    std::vector<BatchInst> inst;        // active instances, in work-list order
    int64_t next_id = 1;
    int64_t steps = 0;
    int cur = 0;
    // device tables (fixed addresses, sized for max_inst and max_items)
    CartInst *d_inst = nullptr;
    int2 *d_items = nullptr;
    int *d_nitems = nullptr;
    double *d_partial = nullptr, *d_out = nullptr;
    double *h_out = nullptr;            // pinned [max_inst][4]
    double *d_stage = nullptr;          // [max_cells_one][3] staging for add/get
    int64_t stage_cells = 0;
    int64_t max_items = 0, n_items = 0;
    int grid = 0, ctas_per_sm = 1, n_sm = 1;   // grid: CTAs of the walking form
    bool per_item = true;                       // one CTA per work item (the grid follows the list)
    int graph_steps = 64;
    cudaGraphExec_t graph = nullptr;
    int64_t graph_items = -1;                   // the item count the graph's per-item grids were sized for
};

// CTAs of a step launch: one per work item (at least one), or the walking form's grid
static int batch_launch_grid(const sdugks_batch *b)
{
    return b->per_item ? (int)(b->n_items > 0 ? b->n_items : 1) : b->grid;
}

static int batch_upload_tables(sdugks_batch *b)
{
    std::vector<CartInst> h;
    std::vector<int2> items;
    h.reserve(b->inst.size());
    for (size_t q = 0; q < b->inst.size(); q++) {
        CartInst ci = b->inst[q].ci;
        ci.item0 = (int32_t)items.size();
        ci.n_items = (int32_t)b->inst[q].ntiles;
        // item: (instance, block x | block y << 16)
        const int ntx = (ci.nx + 15) / 16;
        for (int64_t t = 0; t < b->inst[q].ntiles; t++)
            items.push_back(make_int2((int)q, (int)(t % ntx) | ((int)(t / ntx) << 16)));
        b->inst[q].ci.item0 = ci.item0;
        b->inst[q].ci.n_items = ci.n_items;
        h.push_back(ci);
    }
    if ((int64_t)items.size() > b->max_items) return fail(SDUGKS_ERR_FULL, "batch work list full");
    b->n_items = (int64_t)items.size();
    const int ni = (int)b->n_items;
    if (!h.empty()) CUDA_TRY(cudaMemcpyAsync(b->d_inst, h.data(), h.size() * sizeof(CartInst), cudaMemcpyHostToDevice, b->stream));
    if (!items.empty()) CUDA_TRY(cudaMemcpyAsync(b->d_items, items.data(), items.size() * sizeof(int2), cudaMemcpyHostToDevice, b->stream));
    CUDA_TRY(cudaMemcpyAsync(b->d_nitems, &ni, sizeof(int), cudaMemcpyHostToDevice, b->stream));
    CUDA_TRY(cudaStreamSynchronize(b->stream));   // the host vectors go out of scope
    // a graph of per-item launches has grids of the old item count (destroyed after the
    // synchronisation, so no launch of it is still running)
    if (b->graph && b->per_item && b->graph_items != b->n_items) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    return SDUGKS_OK;
}

extern "C" int sdugks_batch_create(int64_t pool_bytes, int32_t precision, int32_t max_instances, void *stream,
                                   sdugks_batch **out)
{
    if (!out) return fail(SDUGKS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (pool_bytes <= 0 || max_instances <= 0 || max_instances > (1 << 20))
        return fail(SDUGKS_ERR_INVALID_ARG, "pool_bytes must be > 0 and max_instances in [1, 2^20]");
    if (precision != SDUGKS_FP32 && precision != SDUGKS_FP32_BF16DEV && precision != SDUGKS_FP32_FP16DEV)
        return fail(SDUGKS_ERR_INVALID_ARG, "batches run in FP32 or FP32_BF16DEV");
    sdugks_batch *b = new (std::nothrow) sdugks_batch;
    if (!b) return fail(SDUGKS_ERR_OOM, "host allocation failed");
    b->prec = precision;
    b->max_inst = max_instances;
    b->stream = static_cast<cudaStream_t>(stream);
    // the work list can hold one item per 64 pool cells plus one per instance
    b->max_items = pool_bytes / (64 * 100) + max_instances + 1024;
    auto cleanup = [&](int rc) { sdugks_batch_destroy(b); return rc; };
    cudaError_t e = cudaGetDevice(&b->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->n_sm, cudaDevAttrMultiProcessorCount, b->device);
    if (e == cudaSuccess) e = cudaMalloc(&b->pool, (size_t)pool_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_inst, sizeof(CartInst) * (size_t)max_instances);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_items, sizeof(int2) * (size_t)b->max_items);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_nitems, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_partial, sizeof(double) * 4 * (size_t)b->max_items);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_out, sizeof(double) * 4 * (size_t)max_instances);
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_out, sizeof(double) * 4 * (size_t)max_instances);
    if (e == cudaSuccess) e = cudaMemset(b->d_nitems, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = prepare_batch(precision);
    if (e != cudaSuccess)
        return cleanup(fail(e == cudaErrorMemoryAllocation ? SDUGKS_ERR_OOM : SDUGKS_ERR_CUDA, "batch create: %s",
                            cudaGetErrorString(e)));
    b->alloc.reset((size_t)pool_bytes);
    b->ctas_per_sm = batch_ctas_per_sm(precision);
    b->grid = b->n_sm * b->ctas_per_sm;
    *out = b;
    return SDUGKS_OK;
}

extern "C" int sdugks_batch_footprint(const sdugks_batch *b, const sdugks_mesh *m, int64_t *bytes)
{
    if (!b || !m || !bytes) return fail(SDUGKS_ERR_INVALID_ARG, "NULL argument");
    CartGrid g;
    if (!detect_cart(*m, g)) return fail(SDUGKS_ERR_INVALID_ARG, "not a uniform Cartesian grid: %s", g.why.c_str());
    const int32_t pitch = (g.nx + 31) / 32 * 32;
    *bytes = (int64_t)inst_bytes(b->prec, cart_npad(pitch, g.ny));
    return SDUGKS_OK;
}

extern "C" int sdugks_batch_add(sdugks_batch *b, const sdugks_mesh *m, double tau, double dt, const double *rho,
                                const double *u, int64_t *id)
{
    if (!b || !m || !id) return fail(SDUGKS_ERR_INVALID_ARG, "NULL argument");
    if (!(tau > 0) || !(dt > 0) || !std::isfinite(tau) || !std::isfinite(dt))
        return fail(SDUGKS_ERR_INVALID_ARG, "tau and dt must be finite and > 0");
    Faces F;
    int rc = merge_periodic(*m, F);       // boundary table checks
    if (rc) return rc;
    CartGrid g;
    if (!detect_cart(*m, g)) return fail(SDUGKS_ERR_INVALID_ARG, "not a uniform Cartesian grid: %s", g.why.c_str());
    if ((int32_t)b->inst.size() >= b->max_inst) return fail(SDUGKS_ERR_FULL, "batch instance table full");
    if ((g.nx + 15) / 16 > 0xFFFF || (g.ny + BATCH_TY - 1) / BATCH_TY > 0x7FFF)
        return fail(SDUGKS_ERR_INVALID_ARG, "grid of %d x %d cells too large for a batch instance", g.nx, g.ny);
    const int32_t pitch = (g.nx + 31) / 32 * 32;
    const int64_t npad = cart_npad(pitch, g.ny);
    const size_t bytes = inst_bytes(b->prec, npad);
    size_t off = 0;
    if (!b->alloc.alloc(bytes, off)) return fail(SDUGKS_ERR_FULL, "batch pool has no room for %zu bytes", bytes);
    CUDA_TRY(cudaSetDevice(b->device));
    BatchInst bi;
    bi.id = b->next_id++;
    bi.off = off;
    bi.bytes = bytes;
    bi.admitted_at = b->steps;
    bi.ntiles = (int64_t)((g.nx + 15) / 16) * ((g.ny + BATCH_TY - 1) / BATCH_TY);
    fill_cart_inst(bi.ci, *m, g, tau, dt, pitch, npad);
    {
        auto up = [](size_t x) { return (x + 255) & ~size_t(255); };
        const size_t fs = (b->prec == P_BF16DEV || b->prec == P_FP16DEV) ? 2 : 4;
        char *p = b->pool + off;
        for (int k = 0; k < 2; k++) { bi.ci.f[k] = p; p += up(NQ * npad * fs); }
        for (int k = 0; k < 2; k++) { bi.ci.W[k] = reinterpret_cast<double *>(p); p += up(3 * npad * 8); }
        bi.ci.snap = reinterpret_cast<double *>(p);
    }
    // initial state into the current buffer, through a staging slot of the instance table
    const int64_t n = (int64_t)g.nx * g.ny;
    if (b->stage_cells < n) {
        if (b->d_stage) cudaFree(b->d_stage);
        b->d_stage = nullptr;
        b->stage_cells = 0;
        cudaError_t e = cudaMalloc(&b->d_stage, sizeof(double) * 3 * (size_t)n);
        if (e != cudaSuccess) { b->alloc.release(off, bytes); return fail(SDUGKS_ERR_OOM, "batch staging: %s", cudaGetErrorString(e)); }
        b->stage_cells = n;
    }
    // user cell c -> lattice position; the staging arrays are in lattice order i + nx j
    bi.lattice.resize(n);
    for (int64_t c = 0; c < n; c++) bi.lattice[c] = g.ci[c] + (int64_t)g.nx * g.cj[c];
    std::vector<double> r_l, u_l;
    if (rho || u) {
        r_l.assign(n, 1.0);
        u_l.assign(2 * n, 0.0);
        for (int64_t c = 0; c < n; c++) {
            const int64_t q = bi.lattice[c];
            if (rho) r_l[q] = rho[c];
            if (u) { u_l[2 * q] = u[2 * c]; u_l[2 * q + 1] = u[2 * c + 1]; }
        }
    }
    CartInst *slot = b->d_inst + b->inst.size();        // the new instance's table entry
    CUDA_TRY(cudaMemcpyAsync(slot, &bi.ci, sizeof(CartInst), cudaMemcpyHostToDevice, b->stream));
    double *dr = nullptr, *du = nullptr;
    if (rho) { dr = b->d_stage; CUDA_TRY(cudaMemcpyAsync(dr, r_l.data(), sizeof(double) * n, cudaMemcpyHostToDevice, b->stream)); }
    if (u) { du = b->d_stage + n; CUDA_TRY(cudaMemcpyAsync(du, u_l.data(), sizeof(double) * 2 * n, cudaMemcpyHostToDevice, b->stream)); }
    CUDA_TRY(launch_batch_init(b->prec, &bi.ci, slot, b->cur, dr, du, b->stream));
    CUDA_TRY(cudaStreamSynchronize(b->stream));
    b->inst.push_back(std::move(bi));
    rc = batch_upload_tables(b);
    if (rc) { b->inst.pop_back(); b->alloc.release(off, bytes); return rc; }
    *id = b->inst.back().id;
    return SDUGKS_OK;
}

static int batch_find(const sdugks_batch *b, int64_t id)
{
    for (size_t q = 0; q < b->inst.size(); q++)
        if (b->inst[q].id == id) return (int)q;
    return -1;
}

extern "C" int sdugks_batch_remove(sdugks_batch *b, int64_t id)
{
    if (!b) return fail(SDUGKS_ERR_INVALID_ARG, "batch is NULL");
    const int q = batch_find(b, id);
    if (q < 0) return fail(SDUGKS_ERR_INVALID_ARG, "no instance %lld in the batch", (long long)id);
    CUDA_TRY(cudaSetDevice(b->device));
    CUDA_TRY(cudaStreamSynchronize(b->stream));        // no step may still read its memory
    b->alloc.release(b->inst[q].off, b->inst[q].bytes);
    b->inst.erase(b->inst.begin() + q);
    return batch_upload_tables(b);
}

static int batch_ensure_graph(sdugks_batch *b)
{
    if (b->graph) return SDUGKS_OK;
    cudaGraph_t g = nullptr;
    CUDA_TRY(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    const int grid = batch_launch_grid(b);
    for (int k = 0; k < b->graph_steps && e == cudaSuccess; k++)
        e = launch_step_batch(b->prec, b->d_inst, b->d_items, b->d_nitems, grid, b->per_item, k & 1, b->cap_stream);
    cudaError_t e2 = cudaStreamEndCapture(b->cap_stream, &g);
    CUDA_TRY(e);
    CUDA_TRY(e2);
    e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    CUDA_TRY(e);
    b->graph_items = b->n_items;
    return SDUGKS_OK;
}

extern "C" int sdugks_batch_step(sdugks_batch *b, int64_t n)
{
    if (!b) return fail(SDUGKS_ERR_INVALID_ARG, "batch is NULL");
    if (n < 0) return fail(SDUGKS_ERR_INVALID_ARG, "negative step count");
    CUDA_TRY(cudaSetDevice(b->device));
    int64_t left = n;
    if (left >= 2 * b->graph_steps) {
        if (b->cur != 0) {
            CUDA_TRY(launch_step_batch(b->prec, b->d_inst, b->d_items, b->d_nitems, batch_launch_grid(b),
                                       b->per_item, b->cur, b->stream));
            b->cur ^= 1; b->steps++; left--;
        }
        int rc = batch_ensure_graph(b);
        if (rc) return rc;
        while (left >= b->graph_steps) {
            CUDA_TRY(cudaGraphLaunch(b->graph, b->stream));
            b->steps += b->graph_steps; left -= b->graph_steps;
        }
    }
    while (left > 0) {
        CUDA_TRY(launch_step_batch(b->prec, b->d_inst, b->d_items, b->d_nitems, batch_launch_grid(b), b->per_item,
                                   b->cur, b->stream));
        b->cur ^= 1; b->steps++; left--;
    }
    return SDUGKS_OK;
}

extern "C" int sdugks_batch_residual(sdugks_batch *b, int64_t *ids, double *eps, double *mass, int64_t *steps,
                                     int64_t *count)
{
    if (!b) return fail(SDUGKS_ERR_INVALID_ARG, "batch is NULL");
    CUDA_TRY(cudaSetDevice(b->device));
    const int ni = (int)b->inst.size();
    if (count) *count = ni;
    if (ni == 0) return SDUGKS_OK;
    CUDA_TRY(launch_batch_residual(b->d_inst, ni, b->d_items, b->d_nitems, b->grid, b->cur, b->d_partial, b->d_out,
                                   b->stream));
    CUDA_TRY(cudaMemcpyAsync(b->h_out, b->d_out, sizeof(double) * 4 * ni, cudaMemcpyDeviceToHost, b->stream));
    CUDA_TRY(cudaStreamSynchronize(b->stream));
    for (int q = 0; q < ni; q++) {
        const double *o = b->h_out + 4 * q;
        if (ids) ids[q] = b->inst[q].id;
        if (eps) eps[q] = o[3] != 0.0 ? NAN : (o[1] > 0.0 ? std::sqrt(o[0]) / std::sqrt(o[1]) : INFINITY);
        if (mass) mass[q] = o[2];
        if (steps) steps[q] = b->steps - b->inst[q].admitted_at;
    }
    return SDUGKS_OK;
}

extern "C" int sdugks_batch_get_macros(sdugks_batch *b, int64_t id, double *rho, double *u)
{
    if (!b) return fail(SDUGKS_ERR_INVALID_ARG, "batch is NULL");
    const int q = batch_find(b, id);
    if (q < 0) return fail(SDUGKS_ERR_INVALID_ARG, "no instance %lld in the batch", (long long)id);
    CUDA_TRY(cudaSetDevice(b->device));
    const CartInst &ci = b->inst[q].ci;
    const int64_t n = (int64_t)ci.nx * ci.ny;
    if (b->stage_cells < n) return fail(SDUGKS_ERR_STATE, "internal: staging smaller than an instance");
    CUDA_TRY(launch_batch_macros(&ci, b->d_inst + q, b->cur, b->d_stage, b->d_stage + n, b->stream));
    std::vector<double> r(n), v(2 * n);
    CUDA_TRY(cudaMemcpyAsync(r.data(), b->d_stage, sizeof(double) * n, cudaMemcpyDeviceToHost, b->stream));
    CUDA_TRY(cudaMemcpyAsync(v.data(), b->d_stage + n, sizeof(double) * 2 * n, cudaMemcpyDeviceToHost, b->stream));
    CUDA_TRY(cudaStreamSynchronize(b->stream));
    const std::vector<int64_t> &lat = b->inst[q].lattice;       // back to the caller's cell order
    for (int64_t c = 0; c < n; c++) {
        if (rho) rho[c] = r[lat[c]];
        if (u) { u[2 * c] = v[2 * lat[c]]; u[2 * c + 1] = v[2 * lat[c] + 1]; }
    }
    return SDUGKS_OK;
}

extern "C" int sdugks_batch_autotune(sdugks_batch *b, int64_t steps)
{
    if (!b || steps <= 0) return fail(SDUGKS_ERR_INVALID_ARG, "bad argument");
    if (b->inst.empty()) return fail(SDUGKS_ERR_STATE, "autotune needs admitted instances");
    CUDA_TRY(cudaSetDevice(b->device));
    cudaEvent_t e0, e1;
    CUDA_TRY(cudaEventCreate(&e0));
    CUDA_TRY(cudaEventCreate(&e1));
    // candidates: one CTA per item (mult 0), then the walking form at 1, 2 and 4 times
    // the resident CTAs
    const int base = b->n_sm * b->ctas_per_sm;
    const int item_grid = (int)(b->n_items > 0 ? b->n_items : 1);
    int best = 0;
    float best_ms = 1e30f;
    for (int mult : {0, 1, 2, 4}) {
        const bool per_item = mult == 0;
        const int grid = per_item ? item_grid : base * mult;
        // steps in pairs so that the buffer parity is unchanged
        for (int64_t k = 0; k < 2; k++)
            launch_step_batch(b->prec, b->d_inst, b->d_items, b->d_nitems, grid, per_item, (b->cur + k) & 1, b->stream);
        cudaEventRecord(e0, b->stream);
        for (int64_t k = 0; k < 2 * steps; k++)
            launch_step_batch(b->prec, b->d_inst, b->d_items, b->d_nitems, grid, per_item, (b->cur + k) & 1, b->stream);
        cudaEventRecord(e1, b->stream);
        cudaError_t e = cudaEventSynchronize(e1);
        float ms = 0;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) { cudaEventDestroy(e0); cudaEventDestroy(e1); return fail(SDUGKS_ERR_CUDA, "autotune: %s", cudaGetErrorString(e)); }
        b->steps += 2 + 2 * steps;
        if (ms < best_ms) { best_ms = ms; best = mult; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const bool per_item = best == 0;
    const int grid = per_item ? b->grid : base * best;
    if (per_item != b->per_item || grid != b->grid) {
        b->per_item = per_item;
        b->grid = grid;
        if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
    }
    return SDUGKS_OK;
}

extern "C" int sdugks_batch_info(const sdugks_batch *b, sdugks_batch_status *o)
{
    if (!b || !o) return fail(SDUGKS_ERR_INVALID_ARG, "NULL argument");
    std::memset(o, 0, sizeof *o);
    o->instances = (int64_t)b->inst.size();
    for (const auto &i : b->inst) o->cells += (int64_t)i.ci.nx * i.ci.ny;
    o->items = b->n_items;
    o->pool_bytes = (int64_t)b->alloc.cap();
    o->pool_used = (int64_t)b->alloc.used();
    o->steps = b->steps;
    o->grid = batch_launch_grid(b);
    o->ctas_per_sm = b->ctas_per_sm;
    o->graph_steps = b->graph_steps;
    o->precision = b->prec;
    o->per_item = b->per_item ? 1 : 0;
    return SDUGKS_OK;
}

extern "C" void sdugks_batch_destroy(sdugks_batch *b)
{
    if (!b) return;
    cudaSetDevice(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    cudaFree(b->pool);
    cudaFree(b->d_inst);
    cudaFree(b->d_items);
    cudaFree(b->d_nitems);
    cudaFree(b->d_partial);
    cudaFree(b->d_out);
    cudaFree(b->d_stage);
    if (b->h_out) cudaFreeHost(b->h_out);
    delete b;
}

// ------------------------------------------------------------------ rarefied (discrete velocity grid)

struct sdugks_dvm {
    sdugks_dvm_params p{};
    int prec = P_FP32;
    int device = 0;
    cudaStream_t stream = nullptr, cap_stream = nullptr;
    int64_t n = 0, nf = 0, Q = 0;
    size_t rs = 4, dbytes = 0;
    char *dmem = nullptr;
    DvmMesh dm{};
    Coefs coefs{};
    void *f = nullptr, *fbp = nullptr, *flux = nullptr;
    double *W = nullptr;
    cudaGraphExec_t graph = nullptr;
    int graph_len = 0;
    bool initialised = false;
    bool fbp_ready = false;         // fbp holds fbar+ of the current state (left by the last step)
};

extern "C" int sdugks_dvm_create(const sdugks_mesh *m, const sdugks_dvm_params *prm, void *stream, sdugks_dvm **out)
{
    if (!out) return fail(SDUGKS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!m || !prm) return fail(SDUGKS_ERR_INVALID_ARG, "mesh or params is NULL");
    if (prm->nv < 2 || prm->nv > 1024) return fail(SDUGKS_ERR_INVALID_ARG, "nv must be in [2, 1024]");
    if (!(prm->vmax > 0) || !(prm->RT_wall > 0) || !(prm->tau > 0) || !(prm->dt > 0) || !std::isfinite(prm->vmax) ||
        !std::isfinite(prm->RT_wall) || !std::isfinite(prm->tau) || !std::isfinite(prm->dt))
        return fail(SDUGKS_ERR_INVALID_ARG, "vmax, RT_wall, tau and dt must be finite and > 0");
    if (prm->precision != SDUGKS_FP64 && prm->precision != SDUGKS_FP32)
        return fail(SDUGKS_ERR_INVALID_ARG, "precision must be FP64 or FP32");
    for (int64_t f = 0; f < m->nf; f++) {
        if (m->nbr[f] >= 0) continue;
        const int k = m->bc_kind[-1 - m->nbr[f]];
        if (k != SDUGKS_BC_PERIODIC && k != SDUGKS_BC_WALL && k != SDUGKS_BC_MOVING_WALL)
            return fail(SDUGKS_ERR_BAD_BC, "rarefied solver: boundary kind %d (only periodic and diffuse walls)", k);
    }
    Faces F;
    int rc = merge_periodic(*m, F);
    if (rc) return rc;
    const int64_t n = m->nc, nf = F.nf, Q = (int64_t)prm->nv * prm->nv;
    for (int64_t f = 0; f < nf; f++)
        if (F.own[f] == F.nbr[f]) return fail(SDUGKS_ERR_INVALID_MESH, "periodic pair joins a cell to itself");
    {
        // faces in the order of their first cell: the face kernel then writes the fluxes
        // in cell order, and the cell kernel, which walks the cells backwards, first reads
        // the fluxes written last (still in L2)
        std::vector<int64_t> ord(nf);
        std::iota(ord.begin(), ord.end(), int64_t(0));
        std::stable_sort(ord.begin(), ord.end(), [&](int64_t a, int64_t b) { return F.own[a] < F.own[b]; });
        Faces G;
        G.nf = nf;
        G.own.resize(nf); G.nbr.resize(nf); G.nl.resize(2 * nf); G.ro.resize(2 * nf); G.rk.resize(2 * nf);
        for (int64_t i = 0; i < nf; i++) {
            const int64_t f = ord[i];
            G.own[i] = F.own[f]; G.nbr[i] = F.nbr[f];
            for (int d = 0; d < 2; d++) {
                G.nl[2 * i + d] = F.nl[2 * f + d]; G.ro[2 * i + d] = F.ro[2 * f + d]; G.rk[2 * i + d] = F.rk[2 * f + d];
            }
        }
        F = std::move(G);
    }

    // cell slots in ascending merged face id; LLSR neighbours, offsets and inverse
    std::vector<int32_t> cface((size_t)n * MAXF, -1), cnb((size_t)n * MAXF, -1);
    std::vector<double> cd((size_t)n * MAXF * 2, 0.0), ainv((size_t)n * 3, 0.0), dtv(n);
    std::vector<int> ns(n, 0);
    for (int64_t f = 0; f < nf; f++)
        for (int side = 0; side < 2; side++) {
            const int64_t c = side == 0 ? F.own[f] : F.nbr[f];
            if (c < 0) continue;
            if (ns[c] >= MAXF) return fail(SDUGKS_ERR_INVALID_MESH, "cell %lld has more than %d faces", (long long)c, MAXF);
            const int sl = ns[c]++;
            cface[(size_t)c * MAXF + sl] = (int32_t)f | (side ? DVM_SECOND : 0);
            const int64_t k = side == 0 ? F.nbr[f] : F.own[f];
            if (k >= 0) {
                cnb[(size_t)c * MAXF + sl] = (int32_t)k;
                const double *rme = side == 0 ? &F.ro[2 * f] : &F.rk[2 * f];
                const double *rot = side == 0 ? &F.rk[2 * f] : &F.ro[2 * f];
                cd[((size_t)c * MAXF + sl) * 2] = rme[0] - rot[0];
                cd[((size_t)c * MAXF + sl) * 2 + 1] = rme[1] - rot[1];
            }
        }
    for (int64_t c = 0; c < n; c++) {
        double axx = 0, axy = 0, ayy = 0;
        for (int sl = 0; sl < MAXF; sl++) {
            if (cnb[(size_t)c * MAXF + sl] < 0) continue;
            const double dx = cd[((size_t)c * MAXF + sl) * 2], dy = cd[((size_t)c * MAXF + sl) * 2 + 1];
            axx += dx * dx; axy += dx * dy; ayy += dy * dy;
        }
        const double det = axx * ayy - axy * axy, tr = axx + ayy;
        if (det > 1e-14 * tr * tr) {
            ainv[3 * c] = ayy / det; ainv[3 * c + 1] = -axy / det; ainv[3 * c + 2] = axx / det;
        }
        dtv[c] = prm->dt / m->vol[c];
    }
    std::vector<double> fgeo((size_t)nf * 6);
    std::vector<int32_t> fown(nf), fnbr(nf);
    for (int64_t f = 0; f < nf; f++) {
        fown[f] = (int32_t)F.own[f];
        fnbr[f] = (int32_t)F.nbr[f];
        const double g6[6] = {F.nl[2 * f], F.nl[2 * f + 1], F.ro[2 * f], F.ro[2 * f + 1], F.rk[2 * f], F.rk[2 * f + 1]};
        std::copy(g6, g6 + 6, &fgeo[(size_t)f * 6]);
    }
    // velocity nodes: midpoints of a uniform nv x nv partition of [-vmax, vmax]^2; node
    // q = j + nv i (x fastest) is (vn[j], vn[i]) with weight h^2
    const double h = 2.0 * prm->vmax / prm->nv;
    std::vector<double> vn(prm->nv);
    for (int j = 0; j < prm->nv; j++) vn[j] = -prm->vmax + (j + 0.5) * h;

    sdugks_dvm *d = new (std::nothrow) sdugks_dvm;
    if (!d) return fail(SDUGKS_ERR_OOM, "host allocation failed");
    d->p = *prm;
    if (d->p.graph_steps == 0) d->p.graph_steps = 32;
    d->prec = prm->precision;
    d->rs = d->prec == P_FP64 ? 8 : 4;
    d->stream = static_cast<cudaStream_t>(stream);
    d->n = n; d->nf = nf; d->Q = Q;
    const size_t rs = d->rs;
    auto layout = [&](Arena &A) {
        d->f = A.take<char>((size_t)n * Q * rs);
        d->fbp = A.take<char>((size_t)n * Q * rs);
        d->flux = A.take<char>((size_t)nf * Q * rs);
        d->W = A.take<double>((size_t)n * 4);
        d->dm.cell_face = A.take<int32_t>(cface.size());
        d->dm.cell_nb = A.take<int32_t>(cnb.size());
        d->dm.cell_d = A.take<char>(cd.size() * rs);
        d->dm.ainv = A.take<char>(ainv.size() * rs);
        d->dm.dtV = A.take<double>(n);
        d->dm.face_own = A.take<int32_t>(nf);
        d->dm.face_nbr = A.take<int32_t>(nf);
        d->dm.face_geo = A.take<char>(fgeo.size() * rs);
        d->dm.vnode = A.take<char>(vn.size() * rs);
    };
    Arena A0;
    layout(A0);
    d->dbytes = A0.used + 256;
    cudaError_t e = cudaGetDevice(&d->device);
    if (e == cudaSuccess) e = cudaMalloc(&d->dmem, d->dbytes);
    if (e != cudaSuccess) {
        delete d;
        return fail(e == cudaErrorMemoryAllocation ? SDUGKS_ERR_OOM : SDUGKS_ERR_CUDA, "cudaMalloc(%zu): %s",
                    A0.used, cudaGetErrorString(e));
    }
    Arena A{d->dmem, 0, d->dbytes};
    layout(A);
    d->dm.nc = n; d->dm.nf = nf; d->dm.Q = Q;
    d->dm.nv = prm->nv;
    d->dm.w_node = h * h;
    auto conv = [&](const std::vector<double> &v) {
        std::vector<char> o(v.size() * rs);
        if (rs == 8) std::memcpy(o.data(), v.data(), o.size());
        else {
            float *q = reinterpret_cast<float *>(o.data());
            for (size_t i = 0; i < v.size(); i++) q[i] = (float)v[i];
        }
        return o;
    };
    int rc2 = SDUGKS_OK;
    auto up = [&](const void *dst, const void *src, size_t bytes, const char *what) {
        const cudaError_t ee = cudaMemcpy(const_cast<void *>(dst), src, bytes, cudaMemcpyHostToDevice);
        if (ee != cudaSuccess && rc2 == SDUGKS_OK) rc2 = fail(SDUGKS_ERR_CUDA, "%s: %s", what, cudaGetErrorString(ee));
    };
    const auto gcd = conv(cd), gai = conv(ainv), gfg = conv(fgeo), gvn = conv(vn);
    up(d->dm.cell_face, cface.data(), cface.size() * 4, "upload cell faces");
    up(d->dm.cell_nb, cnb.data(), cnb.size() * 4, "upload neighbours");
    up(d->dm.cell_d, gcd.data(), gcd.size(), "upload offsets");
    up(d->dm.ainv, gai.data(), gai.size(), "upload LLSR inverse");
    up(d->dm.dtV, dtv.data(), dtv.size() * 8, "upload dt/V");
    up(d->dm.face_own, fown.data(), fown.size() * 4, "upload owners");
    up(d->dm.face_nbr, fnbr.data(), fnbr.size() * 4, "upload neighbours");
    up(d->dm.face_geo, gfg.data(), gfg.size(), "upload face geometry");
    up(d->dm.vnode, gvn.data(), gvn.size(), "upload velocity nodes");
    if (rc2 == SDUGKS_OK) {
        cudaError_t ee = cudaStreamCreateWithFlags(&d->cap_stream, cudaStreamNonBlocking);
        if (ee == cudaSuccess) ee = prepare_dvm(d->prec, Q, prm->nv);
        if (ee != cudaSuccess) rc2 = fail(SDUGKS_ERR_CUDA, "stream / kernel attributes: %s", cudaGetErrorString(ee));
    }
    if (rc2) { sdugks_dvm_destroy(d); return rc2; }
    fill_coefs(d->coefs, *m, prm->tau, prm->dt);
    *out = d;
    return SDUGKS_OK;
}

extern "C" int sdugks_dvm_init(sdugks_dvm *d, const double *rho, const double *u, const double *RT)
{
    if (!d) return fail(SDUGKS_ERR_INVALID_ARG, "solver is NULL");
    std::vector<double> W((size_t)d->n * 4);
    for (int64_t c = 0; c < d->n; c++) {
        const double r = rho ? rho[c] : 1.0, ux = u ? u[2 * c] : 0.0, uy = u ? u[2 * c + 1] : 0.0;
        const double t = RT ? RT[c] : d->p.RT_wall;
        if (!(r > 0) || !(t > 0) || !std::isfinite(ux) || !std::isfinite(uy))
            return fail(SDUGKS_ERR_INVALID_ARG, "initial state of cell %lld: rho and RT must be > 0", (long long)c);
        W[4 * c] = r; W[4 * c + 1] = r * ux; W[4 * c + 2] = r * uy; W[4 * c + 3] = r * (0.5 * (ux * ux + uy * uy) + t);
    }
    CUDA_TRY(cudaSetDevice(d->device));
    CUDA_TRY(cudaMemcpyAsync(d->W, W.data(), W.size() * 8, cudaMemcpyHostToDevice, d->stream));
    CUDA_TRY(launch_dvm_init(d->prec, d->dm, d->W, d->f, d->stream));
    CUDA_TRY(cudaStreamSynchronize(d->stream));
    d->initialised = true;
    d->fbp_ready = false;
    return SDUGKS_OK;
}

static int dvm_ensure_graph(sdugks_dvm *d)
{
    if (d->graph) return SDUGKS_OK;
    const int G = d->p.graph_steps;
    cudaGraph_t g = nullptr;
    CUDA_TRY(cudaStreamBeginCapture(d->cap_stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < G && e == cudaSuccess; k++)     // replayed only once fbp is ready
        e = launch_dvm_step(d->prec, d->dm, d->coefs, d->p.RT_wall, d->f, d->W, d->fbp, d->flux, true, d->cap_stream);
    cudaError_t e2 = cudaStreamEndCapture(d->cap_stream, &g);
    CUDA_TRY(e);
    CUDA_TRY(e2);
    e = cudaGraphInstantiate(&d->graph, g, 0);
    cudaGraphDestroy(g);
    CUDA_TRY(e);
    d->graph_len = G;
    return SDUGKS_OK;
}

extern "C" int sdugks_dvm_step(sdugks_dvm *d, int64_t n)
{
    if (!d) return fail(SDUGKS_ERR_INVALID_ARG, "solver is NULL");
    if (n < 0) return fail(SDUGKS_ERR_INVALID_ARG, "negative step count");
    if (!d->initialised) return fail(SDUGKS_ERR_STATE, "step before init");
    CUDA_TRY(cudaSetDevice(d->device));
    int64_t left = n;
    const int G = d->p.graph_steps;
    if (left > 0 && !d->fbp_ready) {
        CUDA_TRY(launch_dvm_step(d->prec, d->dm, d->coefs, d->p.RT_wall, d->f, d->W, d->fbp, d->flux, false, d->stream));
        d->fbp_ready = true;
        left--;
    }
    if (G > 0 && left >= G) {
        int rc = dvm_ensure_graph(d);
        if (rc) return rc;
        for (; left >= G; left -= G) CUDA_TRY(cudaGraphLaunch(d->graph, d->stream));
    }
    for (; left > 0; left--)
        CUDA_TRY(launch_dvm_step(d->prec, d->dm, d->coefs, d->p.RT_wall, d->f, d->W, d->fbp, d->flux, true, d->stream));
    return SDUGKS_OK;
}

extern "C" int sdugks_dvm_get_macros(sdugks_dvm *d, double *rho, double *u, double *RT)
{
    if (!d) return fail(SDUGKS_ERR_INVALID_ARG, "solver is NULL");
    std::vector<double> W((size_t)d->n * 4);
    CUDA_TRY(cudaSetDevice(d->device));
    CUDA_TRY(cudaMemcpyAsync(W.data(), d->W, W.size() * 8, cudaMemcpyDeviceToHost, d->stream));
    CUDA_TRY(cudaStreamSynchronize(d->stream));
    for (int64_t c = 0; c < d->n; c++) {
        const double r = W[4 * c], ux = W[4 * c + 1] / r, uy = W[4 * c + 2] / r;
        if (rho) rho[c] = r;
        if (u) { u[2 * c] = ux; u[2 * c + 1] = uy; }
        if (RT) RT[c] = W[4 * c + 3] / r - 0.5 * (ux * ux + uy * uy);
    }
    return SDUGKS_OK;
}

extern "C" int sdugks_dvm_get_state(sdugks_dvm *d, double *f, double *W)
{
    if (!d) return fail(SDUGKS_ERR_INVALID_ARG, "solver is NULL");
    CUDA_TRY(cudaSetDevice(d->device));
    if (W) CUDA_TRY(cudaMemcpyAsync(W, d->W, (size_t)d->n * 4 * 8, cudaMemcpyDeviceToHost, d->stream));
    if (f) {
        const size_t cnt = (size_t)d->n * d->Q;
        if (d->prec == P_FP64) {
            CUDA_TRY(cudaMemcpyAsync(f, d->f, cnt * 8, cudaMemcpyDeviceToHost, d->stream));
        } else {
            std::vector<float> tmp(cnt);
            CUDA_TRY(cudaMemcpyAsync(tmp.data(), d->f, cnt * 4, cudaMemcpyDeviceToHost, d->stream));
            CUDA_TRY(cudaStreamSynchronize(d->stream));
            for (size_t i = 0; i < cnt; i++) f[i] = tmp[i];
        }
    }
    CUDA_TRY(cudaStreamSynchronize(d->stream));
    return SDUGKS_OK;
}

extern "C" int sdugks_dvm_sizes(const sdugks_dvm *d, int64_t *n_cells, int64_t *n_faces, int64_t *n_velocities,
                                int64_t *device_bytes)
{
    if (!d) return fail(SDUGKS_ERR_INVALID_ARG, "solver is NULL");
    if (n_cells) *n_cells = d->n;
    if (n_faces) *n_faces = d->nf;
    if (n_velocities) *n_velocities = d->Q;
    if (device_bytes) *device_bytes = (int64_t)d->dbytes;
    return SDUGKS_OK;
}

extern "C" void sdugks_dvm_destroy(sdugks_dvm *d)
{
    if (!d) return;
    cudaSetDevice(d->device);
    if (d->graph) cudaGraphExecDestroy(d->graph);
    if (d->cap_stream) cudaStreamDestroy(d->cap_stream);
    if (d->dmem) cudaFree(d->dmem);
    delete d;
}
