/*
 * sdugks_oracle.c -- TEST INFRASTRUCTURE, not part of the product.
 *
 * A plain, slow, FP64 CPU restatement of one time step of the simplified discrete
 * unified gas kinetic scheme (S-DUGKS, arXiv:2007.07347, Sec. II) on a face-based
 * finite-volume quad mesh, with the boundary conditions of Sec. III.  Only the test
 * suite, the package's smoke check and the CPU-baseline leg of the benchmark load it.
 * It shares no code with the CUDA library and includes none of its headers.
 *
 * Every function cites the passage it follows.  Each one is pinned by a CPU test
 * against something other than itself (closed forms, invariants, special cases, an
 * exact-rational hand stepper on tiny meshes); see the test files under tests/.
 *
 * Readings of points the paper leaves open (velocity set, time level of the macro
 * flux, upwind choice, boundary Maxwellian, residual) are the ones listed next to
 * the functions below.
 *
 * Layouts (all host, caller-owned, row-major):
 *   xy[n_points][2], face_pts[n_faces][2], owner[n_faces], neighbour[n_faces]
 *   (neighbour < 0 means boundary patch -1-neighbour),
 *   bc_kind[n_patches], bc_par[n_patches][3],
 *   f[n_cells][9], W[n_cells][3] = (rho, rho*u_x, rho*u_y).
 */
#define _GNU_SOURCE
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NQ 9

enum { OR_OK = 0, OR_ERR_ARG = -1, OR_ERR_MESH = -2, OR_ERR_BC = -3, OR_ERR_NOMEM = -4 };
enum { KIND_UNSET = 0, KIND_PERIODIC = 1, KIND_WALL = 2, KIND_MOVING_WALL = 3,
       KIND_FARFIELD = 4, KIND_OUTLET = 5, KIND_SYMMETRY = 6 };

/* D2Q9 velocity set and weights (reading A1: the paper names no set; the continuum
 * cases use the nine-velocity lattice with c = 1, c_s^2 = 1/3).
 * Order: rest, +x, +y, -x, -y, (+,+), (-,+), (-,-), (+,-). */
static const double XI[NQ][2] = {{0, 0}, {1, 0}, {0, 1}, {-1, 0}, {0, -1},
                                 {1, 1}, {-1, 1}, {-1, -1}, {1, -1}};
static const double WGT[NQ] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0,
                               1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const double CS2 = 1.0 / 3.0;
/* Mirror images of the velocities in a line of constant x (xi_x -> -xi_x) and of
 * constant y (xi_y -> -xi_y), by index. */
static const int MIRROR_X[NQ] = {0, 3, 2, 1, 4, 6, 5, 8, 7};
static const int MIRROR_Y[NQ] = {0, 1, 4, 3, 2, 8, 7, 6, 5};
/* Tangential tie: |xi . n l| <= TIE counts as neither inflow nor outflow. */
static const double TIE = 1e-12;

/* ------------------------------------------------------------------ equilibrium */

/* Eq. Feq (Sec. II) truncated to second order in u (Hermite form on D2Q9):
 * f_eq = w rho [1 + (xi.u)/c_s^2 + (xi.u)^2/(2 c_s^4) - |u|^2/(2 c_s^2)]. */
static void feq_of(double rho, double ux, double uy, double out[NQ])
{
    double uu = ux * ux + uy * uy;
    for (int a = 0; a < NQ; a++) {
        double eu = XI[a][0] * ux + XI[a][1] * uy;
        out[a] = WGT[a] * rho * (1.0 + eu / CS2 + (eu * eu) / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
    }
}

/* Equilibrium from the conserved variables W = (rho, rho u). */
static void feq_of_W(const double W[3], double out[NQ])
{
    feq_of(W[0], W[1] / W[0], W[2] / W[0], out);
}

int oracle_feq(double rho, double ux, double uy, double *out9)
{
    if (!out9) return OR_ERR_ARG;
    feq_of(rho, ux, uy, out9);
    return OR_OK;
}

/* ------------------------------------------------------------------------- mesh */

typedef struct {
    int64_t nc, nf, np;
    const double *xy;
    const int64_t *fpts, *own, *nbr;
    int npatch;
    const int32_t *bck;
    const double *bcp;
    /* derived */
    double *xf;     /* [nf][2] face midpoint                                       */
    double *nl;     /* [nf][2] unit normal times length, pointing out of the owner */
    double *vol;    /* [nc] cell area                                              */
    double *xc;     /* [nc][2] cell centroid                                       */
    int64_t *ghost; /* [nf] periodic faces: the cell on the far side; symmetry
                       faces: the owner (the ghost is its mirror image); else -1    */
    double *gpos;   /* [nf][2] position of that (ghost) cell seen from this side    */
    int *mir;       /* [nf] symmetry faces: 1 = mirror in x (normal along x),
                       2 = mirror in y; 0 for every other face                      */
    int64_t *cs, *cl; /* cell -> faces, ascending face id                          */
    double *ainv;   /* [nc][3] inverse of the LLSR normal matrix: xx, xy, yy       */
} omesh;

static void omesh_free(omesh *m)
{
    free(m->xf); free(m->nl); free(m->vol); free(m->xc); free(m->ghost); free(m->gpos);
    free(m->mir); free(m->cs); free(m->cl); free(m->ainv);
    memset(m, 0, sizeof(*m));
}

/* Polygon area and centroid of one cell from its faces (shoelace).  The faces are
 * chained end to end into a closed vertex loop first (reading A11: the cell
 * centre is the polygon centroid). */
static int cell_polygon(const omesh *m, int64_t c, double *area, double cen[2])
{
    int64_t n = m->cs[c + 1] - m->cs[c];
    if (n < 3 || n > 64) return OR_ERR_MESH;
    int64_t loop[65];
    int used[64] = {0};
    const int64_t *fl = m->cl + m->cs[c];
    loop[0] = m->fpts[2 * fl[0]];
    loop[1] = m->fpts[2 * fl[0] + 1];
    used[0] = 1;
    for (int64_t k = 2; k <= n; k++) {
        int64_t tail = loop[k - 1], next = -1;
        for (int64_t e = 0; e < n; e++) {
            if (used[e]) continue;
            int64_t p0 = m->fpts[2 * fl[e]], p1 = m->fpts[2 * fl[e] + 1];
            if (p0 == tail) next = p1;
            else if (p1 == tail) next = p0;
            else continue;
            used[e] = 1;
            break;
        }
        if (next < 0) return OR_ERR_MESH;
        loop[k] = next;
    }
    if (loop[n] != loop[0]) return OR_ERR_MESH;
    /* shoelace in coordinates relative to the first vertex (the same sums, without
     * the cancellation of large absolute coordinates) */
    const double ox = m->xy[2 * loop[0]], oy = m->xy[2 * loop[0] + 1];
    double a2 = 0, cx = 0, cy = 0;
    for (int64_t k = 0; k < n; k++) {
        double x0 = m->xy[2 * loop[k]] - ox, y0 = m->xy[2 * loop[k] + 1] - oy;
        double x1 = m->xy[2 * loop[k + 1]] - ox, y1 = m->xy[2 * loop[k + 1] + 1] - oy;
        double cr = x0 * y1 - x1 * y0;
        a2 += cr;
        cx += (x0 + x1) * cr;
        cy += (y0 + y1) * cr;
    }
    if (a2 == 0.0) return OR_ERR_MESH;
    cen[0] = ox + cx / (3.0 * a2);
    cen[1] = oy + cy / (3.0 * a2);
    *area = fabs(0.5 * a2);
    return OR_OK;
}

/* Geometry, periodic pairing (Sec. III, periodic boundary: the ghost cell of a
 * periodic face is the inner cell of the partner patch) and the LLSR normal matrix
 * of Sec. II (2x2, over the face neighbours of each cell; reading A6). */
static int omesh_build(omesh *m, int64_t np, const double *xy, int64_t nf, const int64_t *fpts,
                       const int64_t *own, const int64_t *nbr, int64_t nc, int npatch,
                       const int32_t *bck, const double *bcp)
{
    memset(m, 0, sizeof(*m));
    if (np <= 0 || nf <= 0 || nc <= 0 || !xy || !fpts || !own || !nbr) return OR_ERR_ARG;
    m->np = np; m->nf = nf; m->nc = nc; m->xy = xy; m->fpts = fpts; m->own = own; m->nbr = nbr;
    m->npatch = npatch; m->bck = bck; m->bcp = bcp;
    m->xf = malloc(sizeof(double) * 2 * nf);
    m->nl = malloc(sizeof(double) * 2 * nf);
    m->vol = malloc(sizeof(double) * nc);
    m->xc = malloc(sizeof(double) * 2 * nc);
    m->ghost = malloc(sizeof(int64_t) * nf);
    m->gpos = calloc(2 * nf, sizeof(double));
    m->mir = calloc(nf, sizeof(int));
    m->cs = calloc(nc + 1, sizeof(int64_t));
    m->cl = malloc(sizeof(int64_t) * 2 * nf);
    m->ainv = calloc(3 * nc, sizeof(double));
    if (!m->xf || !m->nl || !m->vol || !m->xc || !m->ghost || !m->gpos || !m->mir || !m->cs || !m->cl ||
        !m->ainv) {
        omesh_free(m);
        return OR_ERR_NOMEM;
    }
    /* cell -> face lists in ascending face id */
    for (int64_t f = 0; f < nf; f++) {
        if (own[f] < 0 || own[f] >= nc || nbr[f] >= nc || nbr[f] == own[f]) { omesh_free(m); return OR_ERR_MESH; }
        if (fpts[2 * f] < 0 || fpts[2 * f] >= np || fpts[2 * f + 1] < 0 || fpts[2 * f + 1] >= np ||
            fpts[2 * f] == fpts[2 * f + 1]) { omesh_free(m); return OR_ERR_MESH; }
        if (nbr[f] < 0 && (-1 - nbr[f]) >= npatch) { omesh_free(m); return OR_ERR_BC; }
        m->cs[own[f] + 1]++;
        if (nbr[f] >= 0) m->cs[nbr[f] + 1]++;
    }
    for (int64_t c = 0; c < nc; c++) m->cs[c + 1] += m->cs[c];
    {
        int64_t *fill = calloc(nc, sizeof(int64_t));
        if (!fill) { omesh_free(m); return OR_ERR_NOMEM; }
        for (int64_t f = 0; f < nf; f++) {
            m->cl[m->cs[own[f]] + fill[own[f]]++] = f;
            if (nbr[f] >= 0) m->cl[m->cs[nbr[f]] + fill[nbr[f]]++] = f;
        }
        free(fill);
    }
    for (int64_t c = 0; c < nc; c++) {
        int rc = cell_polygon(m, c, &m->vol[c], &m->xc[2 * c]);
        if (rc) { omesh_free(m); return rc; }
    }
    /* face midpoint and normal*length, turned to point away from the owner centroid */
    for (int64_t f = 0; f < nf; f++) {
        double x0 = xy[2 * fpts[2 * f]], y0 = xy[2 * fpts[2 * f] + 1];
        double x1 = xy[2 * fpts[2 * f + 1]], y1 = xy[2 * fpts[2 * f + 1] + 1];
        double mx = 0.5 * (x0 + x1), my = 0.5 * (y0 + y1);
        double nx = y1 - y0, ny = -(x1 - x0);
        const double *c = &m->xc[2 * own[f]];
        if ((mx - c[0]) * nx + (my - c[1]) * ny < 0) { nx = -nx; ny = -ny; }
        m->xf[2 * f] = mx; m->xf[2 * f + 1] = my;
        m->nl[2 * f] = nx; m->nl[2 * f + 1] = ny;
        m->ghost[f] = -1;
    }
    /* every boundary face needs a boundary condition */
    for (int64_t f = 0; f < nf; f++) {
        if (nbr[f] >= 0) continue;
        int p = (int)(-1 - nbr[f]);
        if (!bck || bck[p] == KIND_UNSET) { omesh_free(m); return OR_ERR_BC; }
    }
    /* periodic pairing by face centre + shift (brute force) */
    for (int64_t f = 0; f < nf; f++) {
        if (nbr[f] >= 0) continue;
        int p = (int)(-1 - nbr[f]);
        if (bck[p] != KIND_PERIODIC) continue;
        int q = (int)bcp[3 * p];
        if (q < 0 || q >= npatch || bck[q] != KIND_PERIODIC) { omesh_free(m); return OR_ERR_BC; }
        double sx = bcp[3 * p + 1], sy = bcp[3 * p + 2];
        double len = hypot(m->nl[2 * f], m->nl[2 * f + 1]);
        double tx = m->xf[2 * f] + sx, ty = m->xf[2 * f + 1] + sy;
        int64_t hit = -1;
        for (int64_t g = 0; g < nf; g++) {
            if (nbr[g] != -1 - q) continue;
            if (hypot(m->xf[2 * g] - tx, m->xf[2 * g + 1] - ty) <= 1e-9 * len) { hit = g; break; }
        }
        if (hit < 0) { omesh_free(m); return OR_ERR_BC; }
        int64_t other = own[hit];
        m->ghost[f] = other;
        m->gpos[2 * f] = m->xc[2 * other] - sx;
        m->gpos[2 * f + 1] = m->xc[2 * other + 1] - sy;
    }
    /* Symmetric boundary (Sec. III): a ghost cell mirrors the owner in the face line,
     * x_g = x_o + 2 ((x_f - x_o) . N) N, with the owner's density and the mirrored
     * velocity.  Mirrored velocities must be lattice velocities, so the face must be
     * a line of constant x or constant y. */
    for (int64_t f = 0; f < nf; f++) {
        if (nbr[f] >= 0) continue;
        int p = (int)(-1 - nbr[f]);
        if (bck[p] != KIND_SYMMETRY) continue;
        double len = hypot(m->nl[2 * f], m->nl[2 * f + 1]);
        double Nx = m->nl[2 * f] / len, Ny = m->nl[2 * f + 1] / len;
        if (fabs(Ny) <= 1e-12) m->mir[f] = 1;
        else if (fabs(Nx) <= 1e-12) m->mir[f] = 2;
        else { omesh_free(m); return OR_ERR_BC; }
        const double *xo = &m->xc[2 * own[f]];
        double dn = (m->xf[2 * f] - xo[0]) * Nx + (m->xf[2 * f + 1] - xo[1]) * Ny;
        m->ghost[f] = own[f];
        m->gpos[2 * f] = xo[0] + 2.0 * dn * Nx;
        m->gpos[2 * f + 1] = xo[1] + 2.0 * dn * Ny;
    }
    /* LLSR normal matrix sum_k d d^T and its inverse (Cramer) */
    for (int64_t c = 0; c < nc; c++) {
        double axx = 0, axy = 0, ayy = 0;
        for (int64_t e = m->cs[c]; e < m->cs[c + 1]; e++) {
            int64_t f = m->cl[e];
            double px, py;
            if (nbr[f] >= 0) {
                int64_t k = own[f] == c ? nbr[f] : own[f];
                px = m->xc[2 * k]; py = m->xc[2 * k + 1];
            } else if (m->ghost[f] >= 0) {
                px = m->gpos[2 * f]; py = m->gpos[2 * f + 1];
            } else {
                continue;            /* plain boundary faces add no LLSR term */
            }
            double dx = px - m->xc[2 * c], dy = py - m->xc[2 * c + 1];
            axx += dx * dx; axy += dx * dy; ayy += dy * dy;
        }
        double det = axx * ayy - axy * axy;
        double tr = axx + ayy;
        if (!(det > 1e-14 * tr * tr)) {        /* degenerate stencil: zero gradient */
            m->ainv[3 * c] = m->ainv[3 * c + 1] = m->ainv[3 * c + 2] = 0.0;
        } else {
            m->ainv[3 * c] = ayy / det;
            m->ainv[3 * c + 1] = -axy / det;
            m->ainv[3 * c + 2] = axx / det;
        }
    }
    return OR_OK;
}

/* Geometry as the oracle sees it (for the pins): vol[nc], xc[nc][2], ainv[nc][3],
 * nl[nf][2], xf[nf][2], ghost[nf]. */
int oracle_geometry(int64_t np, const double *xy, int64_t nf, const int64_t *fpts,
                    const int64_t *own, const int64_t *nbr, int64_t nc, int npatch,
                    const int32_t *bck, const double *bcp,
                    double *vol, double *xc, double *ainv, double *nl, double *xf, int64_t *ghost)
{
    omesh m;
    int rc = omesh_build(&m, np, xy, nf, fpts, own, nbr, nc, npatch, bck, bcp);
    if (rc) return rc;
    if (vol) memcpy(vol, m.vol, sizeof(double) * nc);
    if (xc) memcpy(xc, m.xc, sizeof(double) * 2 * nc);
    if (ainv) memcpy(ainv, m.ainv, sizeof(double) * 3 * nc);
    if (nl) memcpy(nl, m.nl, sizeof(double) * 2 * nf);
    if (xf) memcpy(xf, m.xf, sizeof(double) * 2 * nf);
    if (ghost) memcpy(ghost, m.ghost, sizeof(int64_t) * nf);
    omesh_free(&m);
    return OR_OK;
}

/* LLSR gradient of Sec. II for nv interleaved scalar fields phi[nc][nv]:
 * sigma_j = A_j^{-1} sum_k (x_k - x_j)(phi_k - phi_j), k over face neighbours
 * (periodic images at their shifted positions).  out: grad[nc][nv][2]. */
static void llsr(const omesh *m, const double *phi, int nv, double *grad)
{
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < m->nc; c++) {
        for (int v = 0; v < nv; v++) {
            double bx = 0, by = 0;
            for (int64_t e = m->cs[c]; e < m->cs[c + 1]; e++) {
                int64_t f = m->cl[e], k;
                double px, py;
                if (m->nbr[f] >= 0) {
                    k = m->own[f] == c ? m->nbr[f] : m->own[f];
                    px = m->xc[2 * k]; py = m->xc[2 * k + 1];
                } else if (m->ghost[f] >= 0) {
                    k = m->ghost[f];
                    px = m->gpos[2 * f]; py = m->gpos[2 * f + 1];
                } else {
                    continue;
                }
                /* a symmetry ghost holds the owner's value of the mirrored velocity
                 * (nv == NQ: the nine velocity fields; a single field mirrors to itself) */
                int vk = v;
                if (m->mir[f] && nv == NQ) vk = m->mir[f] == 1 ? MIRROR_X[v] : MIRROR_Y[v];
                double dphi = phi[k * nv + vk] - phi[c * nv + v];
                bx += (px - m->xc[2 * c]) * dphi;
                by += (py - m->xc[2 * c + 1]) * dphi;
            }
            const double *ai = &m->ainv[3 * c];
            grad[(c * nv + v) * 2 + 0] = ai[0] * bx + ai[1] * by;
            grad[(c * nv + v) * 2 + 1] = ai[1] * bx + ai[2] * by;
        }
    }
}

int oracle_gradient(int64_t np, const double *xy, int64_t nf, const int64_t *fpts,
                    const int64_t *own, const int64_t *nbr, int64_t nc, int npatch,
                    const int32_t *bck, const double *bcp, const double *phi, double *grad)
{
    omesh m;
    int rc = omesh_build(&m, np, xy, nf, fpts, own, nbr, nc, npatch, bck, bcp);
    if (rc) return rc;
    llsr(&m, phi, 1, grad);
    omesh_free(&m);
    return OR_OK;
}

/* --------------------------------------------------------------------- the step */

/* Boundary values (rho_b, u_b) of Sec. III for patch kind on the owner cell with
 * conserved variables Wo at t_n (reading A7: "in" is the owner cell, time t_n). */
static void boundary_macros(int kind, const double *par, const double Wo[3], double *rho,
                            double *ux, double *uy)
{
    switch (kind) {
    case KIND_WALL:           /* no-slip wall at rest: rho from inside, u = 0 */
        *rho = Wo[0]; *ux = 0.0; *uy = 0.0; break;
    case KIND_MOVING_WALL:    /* no-slip wall: rho from inside, u = u_wall */
        *rho = Wo[0]; *ux = par[0]; *uy = par[1]; break;
    case KIND_FARFIELD:       /* inlet / free stream: rho_inf, u_inf */
        *rho = par[0]; *ux = par[1]; *uy = par[2]; break;
    default:                  /* outlet: rho and u of the inner cell */
        *rho = Wo[0]; *ux = Wo[1] / Wo[0]; *uy = Wo[2] / Wo[0]; break;
    }
}

typedef struct {
    double *feqn, *fbp, *sig, *fb, *F;
} owork;

/* One S-DUGKS step, the eleven steps of Sec. II.  State at t_n: f (cell-centred
 * distribution) and W (conserved variables).
 * Reading A3 of the macroscopic flux in Eq. MacroUpdate: Eq. MacroUpdate is the
 * moment psi = (1, xi) of Eq. Integration, whose flux is F_meso^{n+1}, so the
 * macroscopic flux is the moment of the mesoscopic flux of this same step, built
 * from the interface distribution f(x_b, t_{n+1}) of step 7.  It is therefore
 * evaluated with step 8 and applied in step 9.  (A lagged reading that uses the
 * previous step's interface distribution diverges on the cavity at dt = 10 tau,
 * where the paper reports converged runs.) */
static void one_step(const omesh *m, double tau, double dt, double *f, double *W, owork *w)
{
    const int64_t nc = m->nc, nf = m->nf;
    const double a_plus = (2.0 * tau - dt) / (2.0 * tau);  /* Eq. fbarplus */
    const double b_plus = dt / (2.0 * tau);
    const double c_face = 2.0 * tau / (2.0 * tau + dt);    /* Eq. f_t_n+1 */

    /* Step 2, Eq. fbarplus at the cell centre: fbar+ = (2tau-dt)/(2tau) f + dt/(2tau) feq(W^n). */
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < nc; j++) {
        feq_of_W(&W[3 * j], &w->feqn[NQ * j]);
        for (int a = 0; a < NQ; a++)
            w->fbp[NQ * j + a] = a_plus * f[NQ * j + a] + b_plus * w->feqn[NQ * j + a];
    }

    /* Step 3, LLSR gradient of fbar+ for every velocity. */
    llsr(m, w->fbp, NQ, w->sig);

    /* Steps 3-7 at every face. */
#pragma omp parallel for schedule(static)
    for (int64_t fc = 0; fc < nf; fc++) {
        int64_t o = m->own[fc], k = m->nbr[fc];
        const double *n = &m->nl[2 * fc], *xb = &m->xf[2 * fc];
        double *fbf = &w->fb[NQ * fc];
        int64_t kk = k >= 0 ? k : m->ghost[fc];
        if (kk >= 0) {
            /* interior (or periodic) face: upwind characteristic reconstruction */
            const double *xk = k >= 0 ? &m->xc[2 * k] : &m->gpos[2 * fc];
            const double *xo = &m->xc[2 * o];
            const int mir = k >= 0 ? 0 : m->mir[fc];
            double fbar[NQ], Wb[3] = {0, 0, 0}, feqb[NQ];
            for (int a = 0; a < NQ; a++) {
                double s = XI[a][0] * n[0] + XI[a][1] * n[1];
                /* Eq. fbpsource: fbar+(x_b - xi dt) = fbar+_u + (x_b - xi dt - x_u) . sigma_u */
                double px = xb[0] - XI[a][0] * dt, py = xb[1] - XI[a][1] * dt;
                double from_o = w->fbp[NQ * o + a] + (px - xo[0]) * w->sig[2 * (NQ * o + a)] +
                                (py - xo[1]) * w->sig[2 * (NQ * o + a) + 1];
                /* far cell: a real cell, a periodic image, or the mirror ghost, whose
                 * fbar+ and gradient are the owner's for the mirrored velocity with the
                 * gradient reflected (Sec. III, symmetric boundary) */
                int ak = a;
                double gsx = 1.0, gsy = 1.0;
                if (mir == 1) { ak = MIRROR_X[a]; gsx = -1.0; }
                else if (mir == 2) { ak = MIRROR_Y[a]; gsy = -1.0; }
                double from_k = w->fbp[NQ * kk + ak] + (px - xk[0]) * (gsx * w->sig[2 * (NQ * kk + ak)]) +
                                (py - xk[1]) * (gsy * w->sig[2 * (NQ * kk + ak) + 1]);
                /* reading A5: upwind by the sign of xi.n, mean of both when tangential */
                if (s > TIE) fbar[a] = from_o;
                else if (s < -TIE) fbar[a] = from_k;
                else fbar[a] = 0.5 * (from_o + from_k);
                /* Eq. fbar: fbar(x_b, t_{n+1}) = fbar+(x_b - xi dt, t_n).
                 * Step 5, Eq. Macro: interface W from the moments of fbar (the collision
                 * term conserves mass and momentum, so fbar has the moments of f). */
                Wb[0] += fbar[a];
                Wb[1] += XI[a][0] * fbar[a];
                Wb[2] += XI[a][1] * fbar[a];
            }
            feq_of_W(Wb, feqb);                 /* step 6 */
            for (int a = 0; a < NQ; a++)        /* step 7, Eq. f_t_n+1 */
                fbf[a] = (fbar[a] + b_plus * feqb[a]) * c_face;
        } else {
            int p = (int)(-1 - k);
            int kind = m->bck[p];
            double rb, ubx, uby, feqb[NQ];
            boundary_macros(kind, &m->bcp[3 * p], &W[3 * o], &rb, &ubx, &uby);
            feq_of(rb, ubx, uby, feqb);         /* Maxwellian of the boundary macros */
            const double *xo = &m->xc[2 * o];
            for (int a = 0; a < NQ; a++) {
                double s = XI[a][0] * n[0] + XI[a][1] * n[1];
                if (s < -TIE) {
                    /* Sec. III, xi.N < 0: non-equilibrium extrapolation
                     * f_b = feq_b + (f_in - feq_in), inner values at t_n */
                    fbf[a] = feqb[a] + (f[NQ * o + a] - w->feqn[NQ * o + a]);
                } else {
                    /* xi.N >= 0: interpolate from the inner field (Eqs. fbpsource, fbar,
                     * f_t_n+1) with the boundary Maxwellian (reading A8) */
                    double px = xb[0] - XI[a][0] * dt, py = xb[1] - XI[a][1] * dt;
                    double fbar = w->fbp[NQ * o + a] + (px - xo[0]) * w->sig[2 * (NQ * o + a)] +
                                  (py - xo[1]) * w->sig[2 * (NQ * o + a) + 1];
                    fbf[a] = (fbar + b_plus * feqb[a]) * c_face;
                }
            }
        }
    }

    /* Step 8, Eq. MesoFlux: F_j = sum over faces (xi . n_out) l f_b, ascending face id. */
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < nc; j++) {
        double Fj[NQ] = {0};
        for (int64_t e = m->cs[j]; e < m->cs[j + 1]; e++) {
            int64_t fc = m->cl[e];
            double sg = (m->own[fc] == j) ? 1.0 : -1.0;
            for (int a = 0; a < NQ; a++) {
                double s = XI[a][0] * m->nl[2 * fc] + XI[a][1] * m->nl[2 * fc + 1];
                Fj[a] += sg * s * w->fb[NQ * fc + a];
            }
        }
        for (int a = 0; a < NQ; a++) w->F[NQ * j + a] = Fj[a];
    }

    /* Steps 1 and 9 (Eqs. MacroFlux, MacroUpdate), 10 and 11 (Eq. fn+1). */
    const double r = dt / tau;
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < nc; j++) {
        double Mj[3] = {0, 0, 0}, feq1[NQ];
        for (int a = 0; a < NQ; a++) {          /* macroscopic flux: moments psi = (1, xi) */
            double Fa = w->F[NQ * j + a];
            Mj[0] += Fa;
            Mj[1] += XI[a][0] * Fa;
            Mj[2] += XI[a][1] * Fa;
        }
        for (int d = 0; d < 3; d++) W[3 * j + d] = W[3 * j + d] - dt / m->vol[j] * Mj[d];   /* step 9 */
        feq_of_W(&W[3 * j], feq1);                                                          /* step 10 */
        for (int a = 0; a < NQ; a++)                                                        /* step 11 */
            f[NQ * j + a] = (f[NQ * j + a] - dt / m->vol[j] * w->F[NQ * j + a] + r * feq1[a]) / (1.0 + r);
    }
}

/* Momentum that leaves the fluid through each boundary face in the step just taken
 * (the forces of Sec. IV: C_d and C_l are the wall patch's sums over 0.5 rho U^2 D):
 * the psi = xi moment of the face's term of Eq. MesoFlux,
 *   F_f = sum_a xi_a (xi_a . n_f l_f) f_b,a,
 * with n_f l_f out of the fluid and f_b the interface distribution of step 7 of that
 * step.  Every face with a neighbour < 0 whose patch is not periodic gets one row, in
 * ascending face id: out[2 i], out[2 i + 1] for the i-th such face. */
static void boundary_flux(const omesh *m, const double *fb, double *out)
{
    int64_t i = 0;
    for (int64_t fc = 0; fc < m->nf; fc++) {
        if (m->nbr[fc] >= 0 || m->bck[-1 - m->nbr[fc]] == KIND_PERIODIC) continue;
        double px = 0.0, py = 0.0;
        for (int a = 0; a < NQ; a++) {
            double s = XI[a][0] * m->nl[2 * fc] + XI[a][1] * m->nl[2 * fc + 1];
            px += XI[a][0] * s * fb[NQ * fc + a];
            py += XI[a][1] * s * fb[NQ * fc + a];
        }
        out[2 * i] = px;
        out[2 * i + 1] = py;
        i++;
    }
}

/* Run n_steps steps in place on (f, W); if bflux is given (n_steps >= 1), also the
 * boundary momentum flux of the last step (boundary_flux). */
static int run_steps(int64_t np, const double *xy, int64_t nf, const int64_t *fpts, const int64_t *own,
                     const int64_t *nbr, int64_t nc, int npatch, const int32_t *bck, const double *bcp,
                     double tau, double dt, int64_t n_steps, double *f, double *W, double *bflux);

int oracle_run(int64_t np, const double *xy, int64_t nf, const int64_t *fpts, const int64_t *own,
               const int64_t *nbr, int64_t nc, int npatch, const int32_t *bck, const double *bcp,
               double tau, double dt, int64_t n_steps, double *f, double *W)
{
    return run_steps(np, xy, nf, fpts, own, nbr, nc, npatch, bck, bcp, tau, dt, n_steps, f, W, NULL);
}

int oracle_run_flux(int64_t np, const double *xy, int64_t nf, const int64_t *fpts, const int64_t *own,
                    const int64_t *nbr, int64_t nc, int npatch, const int32_t *bck, const double *bcp,
                    double tau, double dt, int64_t n_steps, double *f, double *W, double *bflux)
{
    if (n_steps < 1 || !bflux) return OR_ERR_ARG;
    return run_steps(np, xy, nf, fpts, own, nbr, nc, npatch, bck, bcp, tau, dt, n_steps, f, W, bflux);
}

static int run_steps(int64_t np, const double *xy, int64_t nf, const int64_t *fpts, const int64_t *own,
                     const int64_t *nbr, int64_t nc, int npatch, const int32_t *bck, const double *bcp,
                     double tau, double dt, int64_t n_steps, double *f, double *W, double *bflux)
{
    if (!(tau > 0) || !(dt > 0) || n_steps < 0 || !f || !W) return OR_ERR_ARG;
    omesh m;
    int rc = omesh_build(&m, np, xy, nf, fpts, own, nbr, nc, npatch, bck, bcp);
    if (rc) return rc;
    owork w;
    w.feqn = malloc(sizeof(double) * NQ * nc);
    w.fbp = malloc(sizeof(double) * NQ * nc);
    w.sig = malloc(sizeof(double) * 2 * NQ * nc);
    w.fb = malloc(sizeof(double) * NQ * nf);
    w.F = malloc(sizeof(double) * NQ * nc);
    if (!w.feqn || !w.fbp || !w.sig || !w.fb || !w.F) rc = OR_ERR_NOMEM;
    for (int64_t s = 0; s < n_steps && !rc; s++) one_step(&m, tau, dt, f, W, &w);
    if (!rc && bflux) boundary_flux(&m, w.fb, bflux);
    free(w.feqn); free(w.fbp); free(w.sig); free(w.fb); free(w.F);
    omesh_free(&m);
    return rc;
}

/* Initial state: W = (rho, rho u), f = feq(W). */
int oracle_init(int64_t nc, const double *rho, const double *u, double *f, double *W)
{
    if (nc <= 0 || !rho || !u || !f || !W) return OR_ERR_ARG;
    for (int64_t j = 0; j < nc; j++) {
        W[3 * j] = rho[j];
        W[3 * j + 1] = rho[j] * u[2 * j];
        W[3 * j + 2] = rho[j] * u[2 * j + 1];
        feq_of(rho[j], u[2 * j], u[2 * j + 1], &f[NQ * j]);
    }
    return OR_OK;
}

/* Convergence residual of Sec. IV (lid-driven cavity):
 * eps = sqrt(sum[(U-U0)^2 + (V-V0)^2]) / sqrt(sum[U0^2 + V0^2]), U = rho u_x / rho
 * from W, (U0, V0) from the earlier snapshot Ws.  A zero denominator gives +inf
 * (reading A12).  Also returns the mass sum_j V_j rho_j when vol is given. */
int oracle_residual(int64_t nc, const double *W, const double *Ws, const double *vol,
                    double *eps, double *mass)
{
    if (nc <= 0 || !W || !Ws || !eps) return OR_ERR_ARG;
    double num = 0, den = 0, ms = 0;
    for (int64_t j = 0; j < nc; j++) {
        double U = W[3 * j + 1] / W[3 * j], V = W[3 * j + 2] / W[3 * j];
        double U0 = Ws[3 * j + 1] / Ws[3 * j], V0 = Ws[3 * j + 2] / Ws[3 * j];
        num += (U - U0) * (U - U0) + (V - V0) * (V - V0);
        den += U0 * U0 + V0 * V0;
        if (vol) ms += vol[j] * W[3 * j];
    }
    *eps = den > 0 ? sqrt(num) / sqrt(den) : INFINITY;
    if (mass) *mass = ms;
    return OR_OK;
}

/* ===================================================================== rarefied
 * The same scheme on a discrete velocity grid for rarefied flow (Sec. IV, micro
 * cavity): Q velocities xi_q with quadrature weights w_q; the state is the
 * weighted distribution f_q = w_q f(xi_q) (so moments are plain sums), and
 * W = (rho, rho u, rho E) with psi = (1, xi, xi^2/2) of Eq. Macro.  Readings:
 *  - the velocity grid: nv x nv nodes at the midpoints of a uniform partition of
 *    [-vmax, vmax]^2, weights (2 vmax / nv)^2 (midpoint rule);
 *  - the equilibrium: the Maxwellian of Eq. Feq with the exponent written as
 *    |xi - u|^2 / (2 R T) in D = 2 dimensions, sampled at the nodes;
 *  - the temperature from W: R T = (rho E - rho |u|^2 / 2) / rho (two translational
 *    degrees of freedom);
 *  - the relaxation time tau is a constant of the run;
 *  - walls scatter diffusely (Sec. III, diffuse boundary): velocities entering the
 *    gas (xi . N < 0) take the wall Maxwellian rho_w g(xi; u_w, R T_w) (Eq. 6001);
 *    velocities leaving it take the characteristic reconstruction from the inner
 *    cell with the wall Maxwellian as interface equilibrium (as reading A8); rho_w
 *    makes the wall pass no mass (the balance of Eq. 6002, solved in closed form
 *    because the outgoing values depend linearly on rho_w).
 * Periodic faces work as in the continuum scheme; other boundary kinds are
 * rejected. */

int oracle_dvm_grid(int nv, double vmax, double *xi, double *w)
{
    if (nv <= 0 || !(vmax > 0) || !xi || !w) return OR_ERR_ARG;
    const double h = 2.0 * vmax / nv;
    for (int i = 0; i < nv; i++)          /* q = i + nv * j: x fastest */
        for (int j = 0; j < nv; j++) {
            const int q = j + nv * i;
            xi[2 * q] = -vmax + (j + 0.5) * h;
            xi[2 * q + 1] = -vmax + (i + 0.5) * h;
            w[q] = h * h;
        }
    return OR_OK;
}

/* Weighted Maxwellian of Eq. Feq (D = 2) at every node. */
static void dvm_maxwell(double rho, double ux, double uy, double RT, int Q, const double *xi, const double *w,
                        double *out)
{
    const double pre = rho / (2.0 * M_PI * RT);
    for (int q = 0; q < Q; q++) {
        double cx = xi[2 * q] - ux, cy = xi[2 * q + 1] - uy;
        out[q] = w[q] * pre * exp(-(cx * cx + cy * cy) / (2.0 * RT));
    }
}

static void dvm_maxwell_W(const double W[4], int Q, const double *xi, const double *w, double *out)
{
    double rho = W[0], ux = W[1] / rho, uy = W[2] / rho;
    double RT = W[3] / rho - 0.5 * (ux * ux + uy * uy);
    dvm_maxwell(rho, ux, uy, RT, Q, xi, w, out);
}

/* Moments psi = (1, xi, xi^2/2) of a weighted distribution. */
static void dvm_moments(int Q, const double *xi, const double *g, double W[4])
{
    W[0] = W[1] = W[2] = W[3] = 0.0;
    for (int q = 0; q < Q; q++) {
        double x = xi[2 * q], y = xi[2 * q + 1];
        W[0] += g[q];
        W[1] += x * g[q];
        W[2] += y * g[q];
        W[3] += 0.5 * (x * x + y * y) * g[q];
    }
}

int oracle_dvm_maxwell(double rho, double ux, double uy, double RT, int Q, const double *xi, const double *w,
                       double *out)
{
    if (Q <= 0 || !(rho > 0) || !(RT > 0) || !xi || !w || !out) return OR_ERR_ARG;
    dvm_maxwell(rho, ux, uy, RT, Q, xi, w, out);
    return OR_OK;
}

/* Initial state W = (rho, rho u, rho (|u|^2/2 + R T)) and f = feq(W) (as the continuum
 * scheme starts from f = feq(W^0)). */
int oracle_dvm_init(int64_t nc, int Q, const double *xi, const double *w, const double *rho, const double *u,
                    const double *RT, double *f, double *W)
{
    if (nc <= 0 || Q <= 0 || !xi || !w || !rho || !u || !RT || !f || !W) return OR_ERR_ARG;
    for (int64_t j = 0; j < nc; j++) {
        double ux = u[2 * j], uy = u[2 * j + 1];
        W[4 * j] = rho[j];
        W[4 * j + 1] = rho[j] * ux;
        W[4 * j + 2] = rho[j] * uy;
        W[4 * j + 3] = rho[j] * (0.5 * (ux * ux + uy * uy) + RT[j]);
        dvm_maxwell_W(&W[4 * j], Q, xi, w, &f[(size_t)Q * j]);
    }
    return OR_OK;
}

typedef struct {
    double *fbp, *sig, *fb, *F;
} dwork;

/* One step of the scheme (Sec. II, steps in the paper's order, as in one_step) on
 * the velocity grid; RTw is the wall temperature R T_w. */
static void dvm_step(const omesh *m, int Q, const double *xi, const double *w, double RTw, double tau, double dt,
                     double *f, double *W, dwork *k)
{
    const int64_t nc = m->nc, nf = m->nf;
    const double a_plus = (2.0 * tau - dt) / (2.0 * tau);
    const double b_plus = dt / (2.0 * tau);
    const double c_face = 2.0 * tau / (2.0 * tau + dt);

    /* step 2, Eq. fbarplus */
#pragma omp parallel
    {
        double *fe = malloc(sizeof(double) * Q);
#pragma omp for schedule(static)
        for (int64_t j = 0; j < nc; j++) {
            dvm_maxwell_W(&W[4 * j], Q, xi, w, fe);
            for (int q = 0; q < Q; q++)
                k->fbp[(size_t)Q * j + q] = a_plus * f[(size_t)Q * j + q] + b_plus * fe[q];
        }
        free(fe);
    }
    /* step 3, LLSR gradient of every velocity's fbar+ */
    llsr(m, k->fbp, Q, k->sig);

    /* steps 3-7 at every face */
#pragma omp parallel
    {
        double *fbar = malloc(sizeof(double) * Q), *g = malloc(sizeof(double) * Q);
#pragma omp for schedule(static)
        for (int64_t fc = 0; fc < nf; fc++) {
            int64_t o = m->own[fc], kc = m->nbr[fc];
            const double *n = &m->nl[2 * fc], *xb = &m->xf[2 * fc];
            const double *xo = &m->xc[2 * o];
            double *fbf = &k->fb[(size_t)Q * fc];
            int64_t kk = kc >= 0 ? kc : m->ghost[fc];
            if (kk >= 0) {
                const double *xk = kc >= 0 ? &m->xc[2 * kc] : &m->gpos[2 * fc];
                for (int q = 0; q < Q; q++) {
                    double s = xi[2 * q] * n[0] + xi[2 * q + 1] * n[1];
                    double px = xb[0] - xi[2 * q] * dt, py = xb[1] - xi[2 * q + 1] * dt;
                    const double *so = &k->sig[2 * ((size_t)Q * o + q)], *sk = &k->sig[2 * ((size_t)Q * kk + q)];
                    double from_o = k->fbp[(size_t)Q * o + q] + (px - xo[0]) * so[0] + (py - xo[1]) * so[1];
                    double from_k = k->fbp[(size_t)Q * kk + q] + (px - xk[0]) * sk[0] + (py - xk[1]) * sk[1];
                    fbar[q] = s > TIE ? from_o : (s < -TIE ? from_k : 0.5 * (from_o + from_k));
                }
                double Wb[4];
                dvm_moments(Q, xi, fbar, Wb);               /* step 5 */
                dvm_maxwell_W(Wb, Q, xi, w, g);             /* step 6 */
                for (int q = 0; q < Q; q++) fbf[q] = (fbar[q] + b_plus * g[q]) * c_face;   /* step 7 */
            } else {
                int p = (int)(-1 - kc);
                double uwx = 0.0, uwy = 0.0;
                if (m->bck[p] == KIND_MOVING_WALL) { uwx = m->bcp[3 * p]; uwy = m->bcp[3 * p + 1]; }
                dvm_maxwell(1.0, uwx, uwy, RTw, Q, xi, w, g);
                double S_out = 0.0, G_out = 0.0, G_in = 0.0;
                for (int q = 0; q < Q; q++) {
                    double s = xi[2 * q] * n[0] + xi[2 * q + 1] * n[1];
                    if (s < -TIE) {
                        G_in += s * g[q];
                    } else {
                        double px = xb[0] - xi[2 * q] * dt, py = xb[1] - xi[2 * q + 1] * dt;
                        const double *so = &k->sig[2 * ((size_t)Q * o + q)];
                        fbar[q] = k->fbp[(size_t)Q * o + q] + (px - xo[0]) * so[0] + (py - xo[1]) * so[1];
                        S_out += s * fbar[q];
                        G_out += s * g[q];
                    }
                }
                double rho_w = -c_face * S_out / (c_face * b_plus * G_out + G_in);
                for (int q = 0; q < Q; q++) {
                    double s = xi[2 * q] * n[0] + xi[2 * q + 1] * n[1];
                    fbf[q] = s < -TIE ? rho_w * g[q] : (fbar[q] + b_plus * rho_w * g[q]) * c_face;
                }
            }
        }
        free(fbar); free(g);
    }

    /* step 8 and steps 1, 9-11 per cell */
    const double r = dt / tau;
#pragma omp parallel
    {
        double *Fj = malloc(sizeof(double) * Q), *fe = malloc(sizeof(double) * Q);
#pragma omp for schedule(static)
        for (int64_t j = 0; j < nc; j++) {
            for (int q = 0; q < Q; q++) Fj[q] = 0.0;
            for (int64_t e = m->cs[j]; e < m->cs[j + 1]; e++) {
                int64_t fc = m->cl[e];
                double sg = (m->own[fc] == j) ? 1.0 : -1.0;
                for (int q = 0; q < Q; q++) {
                    double s = xi[2 * q] * m->nl[2 * fc] + xi[2 * q + 1] * m->nl[2 * fc + 1];
                    Fj[q] += sg * s * k->fb[(size_t)Q * fc + q];
                }
            }
            double Mj[4];
            dvm_moments(Q, xi, Fj, Mj);
            for (int d = 0; d < 4; d++) W[4 * j + d] -= dt / m->vol[j] * Mj[d];
            dvm_maxwell_W(&W[4 * j], Q, xi, w, fe);
            for (int q = 0; q < Q; q++)
                f[(size_t)Q * j + q] = (f[(size_t)Q * j + q] - dt / m->vol[j] * Fj[q] + r * fe[q]) / (1.0 + r);
        }
        free(Fj); free(fe);
    }
}

int oracle_dvm_run(int64_t np, const double *xy, int64_t nf, const int64_t *fpts, const int64_t *own,
                   const int64_t *nbr, int64_t nc, int npatch, const int32_t *bck, const double *bcp,
                   int Q, const double *xi, const double *w, double RTw, double tau, double dt, int64_t n_steps,
                   double *f, double *W)
{
    if (Q <= 0 || !xi || !w || !(RTw > 0) || !(tau > 0) || !(dt > 0) || n_steps < 0 || !f || !W) return OR_ERR_ARG;
    omesh m;
    int rc = omesh_build(&m, np, xy, nf, fpts, own, nbr, nc, npatch, bck, bcp);
    if (rc) return rc;
    for (int64_t fc = 0; fc < nf && !rc; fc++) {
        if (nbr[fc] >= 0) continue;
        int kd = bck[-1 - nbr[fc]];
        if (kd != KIND_PERIODIC && kd != KIND_WALL && kd != KIND_MOVING_WALL) rc = OR_ERR_BC;
    }
    dwork k;
    k.fbp = malloc(sizeof(double) * Q * nc);
    k.sig = malloc(sizeof(double) * 2 * Q * nc);
    k.fb = malloc(sizeof(double) * Q * nf);
    k.F = NULL;
    if (!k.fbp || !k.sig || !k.fb) rc = rc ? rc : OR_ERR_NOMEM;
    for (int64_t s = 0; s < n_steps && !rc; s++) dvm_step(&m, Q, xi, w, RTw, tau, dt, f, W, &k);
    free(k.fbp); free(k.sig); free(k.fb);
    omesh_free(&m);
    return rc;
}

int oracle_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}
