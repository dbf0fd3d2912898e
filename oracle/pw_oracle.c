/*
 * pw_oracle.c -- plain FP64 CPU oracle of the Piacsek-Williams (PW) advection
 * source terms su, sv, sw for the wind fields u, v, w (paper section 3.1: the
 * "energy conserving scheme by Piacsek and Williams" that the hybrid model
 * offloads; section 2.1: the advection component is the longest running part of
 * the dynamics group; section 3: each dynamics component adds into source terms).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link or call this
 * file: only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline and
 * reference legs use it.  It shares no code, header, table or constant with the
 * CUDA library.
 *
 * Layout: interior arrays only, [nx][ny][nz] with k fastest.  Periodicity in i and
 * j is taken by modulo indexing (no halo arrays).  The grid is an Arakawa C-grid:
 *   u(i,j,k) at (x_{i+1/2}, y_j,       zn_k)
 *   v(i,j,k) at (x_i,       y_{j+1/2}, zn_k)
 *   w(i,j,k) at (x_i,       y_j,       zf_k), zf_k being the TOP face of cell k.
 * The ground face w(-1) is 0 by definition and the lid face w(nz-1) is 0 by
 * definition: the value stored there is never read, and every term it would
 * multiply is dropped.  sw(nz-1) = 0.
 *
 * The paper names the scheme but prints no equations; the discrete operator below
 * is the second-order centred skew-symmetric (energy conserving) PW form on this
 * grid, with horizontal coefficients tcx = 0.25/dx, tcy = 0.25/dy and the
 * anelastic vertical coefficients tzc1/tzc2 (u, v levels) and tzd1/tzd2 (w levels).
 *
 * The end of the file holds the second scheme the paper names, the
 * positivity-preserving ULTIMATE-QUICKEST flux-form advection of a scalar
 * (section 3.1), in the reading written out there.
 *
 * Floating point: FP64, built with -ffp-contract=off so that each source is the
 * literal left-to-right evaluation of its formula.  OpenMP (when enabled) only
 * splits the independent outer i loop of full-field sweeps; reductions are
 * sequential, so results do not depend on the thread count.
 */
#include <math.h>
#include <stddef.h>
#include <string.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* threads                                                                  */
/* ------------------------------------------------------------------------ */
int pwo_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* A1: vertical grid and coefficients                                       */
/* ------------------------------------------------------------------------ */
/*
 * dz(k): the given spacing, or by default a geometric stretch from 10 m at the
 * ground to 40 m at the top, dz(k) = 10 * 4^(k/(nz-1)) (10 m when nz = 1).
 * zf(k) = sum_{m<=k} dz(m)   (top face of cell k, ground at z = 0)
 * zn(k) = zf(k) - dz(k)/2    (cell centre)
 * dzn(k) = zn(k+1) - zn(k)   (k < nz-1; the w cell around face k), dzn(nz-1) = 0
 * rho_n(k) = rho0 exp(-zn(k)/H), rho_w(k) = rho0 exp(-zf(k)/H) unless given;
 * the ground face density rho_w(-1) is rho0.
 * tzc1(k) = 0.25 rho_w(k-1) / (rho_n(k) dz(k))
 * tzc2(k) = 0.25 rho_w(k)   / (rho_n(k) dz(k))
 * tzd1(k) = 0.25 rho_n(k)   / (rho_w(k) dzn(k))     k < nz-1, else 0
 * tzd2(k) = 0.25 rho_n(k+1) / (rho_w(k) dzn(k))     k < nz-1, else 0
 * Each output array has nz entries.  Returns 0, or -1 on a bad argument.
 */
int pwo_coeffs(int nz, const double *dz_in, const double *rhon_in, const double *rhow_in,
               double rho0, double H,
               double *dz, double *zf, double *zn, double *dzn,
               double *rhon, double *rhow,
               double *tzc1, double *tzc2, double *tzd1, double *tzd2)
{
    if (nz < 1 || H == 0.0) return -1;
    for (int k = 0; k < nz; k++) {
        if (dz_in) dz[k] = dz_in[k];
        else if (nz == 1) dz[k] = 10.0;
        else dz[k] = 10.0 * pow(4.0, (double)k / (double)(nz - 1));
        if (!(dz[k] > 0.0)) return -1;
    }
    double z = 0.0;
    for (int k = 0; k < nz; k++) {
        z = z + dz[k];
        zf[k] = z;
        zn[k] = zf[k] - 0.5 * dz[k];
    }
    for (int k = 0; k < nz; k++) dzn[k] = (k < nz - 1) ? zn[k + 1] - zn[k] : 0.0;
    for (int k = 0; k < nz; k++) {
        rhon[k] = rhon_in ? rhon_in[k] : rho0 * exp(-zn[k] / H);
        rhow[k] = rhow_in ? rhow_in[k] : rho0 * exp(-zf[k] / H);
    }
    for (int k = 0; k < nz; k++) {
        double rw_below = (k == 0) ? rho0 : rhow[k - 1];
        tzc1[k] = 0.25 * rw_below / (rhon[k] * dz[k]);
        tzc2[k] = 0.25 * rhow[k] / (rhon[k] * dz[k]);
        if (k < nz - 1) {
            tzd1[k] = 0.25 * rhon[k] / (rhow[k] * dzn[k]);
            tzd2[k] = 0.25 * rhon[k + 1] / (rhow[k] * dzn[k]);
        } else {
            tzd1[k] = 0.0;
            tzd2[k] = 0.0;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* the operator                                                             */
/* ------------------------------------------------------------------------ */
typedef struct {
    long nx, ny, nz;
    double tcx, tcy;
    const double *tzc1, *tzc2, *tzd1, *tzd2;
} pwo_grid;

static long wrap(long a, long n) { a %= n; return a < 0 ? a + n : a; }

/* periodic in i and j; k must be in range (callers guarantee it) */
static double at(const pwo_grid *g, const double *f, long i, long j, long k)
{
    return f[((size_t)wrap(i, g->nx) * (size_t)g->ny + (size_t)wrap(j, g->ny)) * (size_t)g->nz + (size_t)k];
}

/*
 * The three stencils, written with the advecting velocities (u, v, w) and the
 * advected field phi separate, so that su = src_u(u,v,w; phi=u) and so on.  Each
 * term is c * phi_neighbour * (sum of the two advecting velocities on the face).
 * *cond receives the sum over the twelve elementary products |c| |phi| |a|.
 */
static double src_u(const pwo_grid *g, const double *u, const double *v, const double *w,
                     const double *p, long i, long j, long k, double *cond)
{
    long nz = g->nz;
    double s, c;
    s = g->tcx * (at(g, p, i - 1, j, k) * (at(g, u, i - 1, j, k) + at(g, u, i, j, k))
                - at(g, p, i + 1, j, k) * (at(g, u, i, j, k) + at(g, u, i + 1, j, k)));
    c = fabs(g->tcx) * (fabs(at(g, p, i - 1, j, k)) * (fabs(at(g, u, i - 1, j, k)) + fabs(at(g, u, i, j, k)))
                      + fabs(at(g, p, i + 1, j, k)) * (fabs(at(g, u, i, j, k)) + fabs(at(g, u, i + 1, j, k))));
    s = s + g->tcy * (at(g, p, i, j - 1, k) * (at(g, v, i, j - 1, k) + at(g, v, i + 1, j - 1, k))
                    - at(g, p, i, j + 1, k) * (at(g, v, i, j, k) + at(g, v, i + 1, j, k)));
    c = c + fabs(g->tcy) * (fabs(at(g, p, i, j - 1, k)) * (fabs(at(g, v, i, j - 1, k)) + fabs(at(g, v, i + 1, j - 1, k)))
                          + fabs(at(g, p, i, j + 1, k)) * (fabs(at(g, v, i, j, k)) + fabs(at(g, v, i + 1, j, k))));
    if (k > 0) {            /* the face below cell 0 is the ground: w = 0 there */
        s = s + g->tzc1[k] * at(g, p, i, j, k - 1) * (at(g, w, i, j, k - 1) + at(g, w, i + 1, j, k - 1));
        c = c + fabs(g->tzc1[k]) * fabs(at(g, p, i, j, k - 1)) * (fabs(at(g, w, i, j, k - 1)) + fabs(at(g, w, i + 1, j, k - 1)));
    }
    if (k < nz - 1) {       /* the face above cell nz-1 is the lid: w = 0 there */
        s = s - g->tzc2[k] * at(g, p, i, j, k + 1) * (at(g, w, i, j, k) + at(g, w, i + 1, j, k));
        c = c + fabs(g->tzc2[k]) * fabs(at(g, p, i, j, k + 1)) * (fabs(at(g, w, i, j, k)) + fabs(at(g, w, i + 1, j, k)));
    }
    if (cond) *cond = c;
    return s;
}

static double src_v(const pwo_grid *g, const double *u, const double *v, const double *w,
                    const double *p, long i, long j, long k, double *cond)
{
    long nz = g->nz;
    double s, c;
    s = g->tcx * (at(g, p, i - 1, j, k) * (at(g, u, i - 1, j, k) + at(g, u, i - 1, j + 1, k))
                - at(g, p, i + 1, j, k) * (at(g, u, i, j, k) + at(g, u, i, j + 1, k)));
    c = fabs(g->tcx) * (fabs(at(g, p, i - 1, j, k)) * (fabs(at(g, u, i - 1, j, k)) + fabs(at(g, u, i - 1, j + 1, k)))
                      + fabs(at(g, p, i + 1, j, k)) * (fabs(at(g, u, i, j, k)) + fabs(at(g, u, i, j + 1, k))));
    s = s + g->tcy * (at(g, p, i, j - 1, k) * (at(g, v, i, j - 1, k) + at(g, v, i, j, k))
                    - at(g, p, i, j + 1, k) * (at(g, v, i, j, k) + at(g, v, i, j + 1, k)));
    c = c + fabs(g->tcy) * (fabs(at(g, p, i, j - 1, k)) * (fabs(at(g, v, i, j - 1, k)) + fabs(at(g, v, i, j, k)))
                          + fabs(at(g, p, i, j + 1, k)) * (fabs(at(g, v, i, j, k)) + fabs(at(g, v, i, j + 1, k))));
    if (k > 0) {
        s = s + g->tzc1[k] * at(g, p, i, j, k - 1) * (at(g, w, i, j, k - 1) + at(g, w, i, j + 1, k - 1));
        c = c + fabs(g->tzc1[k]) * fabs(at(g, p, i, j, k - 1)) * (fabs(at(g, w, i, j, k - 1)) + fabs(at(g, w, i, j + 1, k - 1)));
    }
    if (k < nz - 1) {
        s = s - g->tzc2[k] * at(g, p, i, j, k + 1) * (at(g, w, i, j, k) + at(g, w, i, j + 1, k));
        c = c + fabs(g->tzc2[k]) * fabs(at(g, p, i, j, k + 1)) * (fabs(at(g, w, i, j, k)) + fabs(at(g, w, i, j + 1, k)));
    }
    if (cond) *cond = c;
    return s;
}

/* w lives on faces 0..nz-2 (nz-1 is the lid); sw(nz-1) = 0 */
static double src_w(const pwo_grid *g, const double *u, const double *v, const double *w,
                    const double *p, long i, long j, long k, double *cond)
{
    long nz = g->nz;
    double s, c;
    if (k >= nz - 1) {
        if (cond) *cond = 0.0;
        return 0.0;
    }
    s = g->tcx * (at(g, p, i - 1, j, k) * (at(g, u, i - 1, j, k) + at(g, u, i - 1, j, k + 1))
                - at(g, p, i + 1, j, k) * (at(g, u, i, j, k) + at(g, u, i, j, k + 1)));
    c = fabs(g->tcx) * (fabs(at(g, p, i - 1, j, k)) * (fabs(at(g, u, i - 1, j, k)) + fabs(at(g, u, i - 1, j, k + 1)))
                      + fabs(at(g, p, i + 1, j, k)) * (fabs(at(g, u, i, j, k)) + fabs(at(g, u, i, j, k + 1))));
    s = s + g->tcy * (at(g, p, i, j - 1, k) * (at(g, v, i, j - 1, k) + at(g, v, i, j - 1, k + 1))
                    - at(g, p, i, j + 1, k) * (at(g, v, i, j, k) + at(g, v, i, j, k + 1)));
    c = c + fabs(g->tcy) * (fabs(at(g, p, i, j - 1, k)) * (fabs(at(g, v, i, j - 1, k)) + fabs(at(g, v, i, j - 1, k + 1)))
                          + fabs(at(g, p, i, j + 1, k)) * (fabs(at(g, v, i, j, k)) + fabs(at(g, v, i, j, k + 1))));
    if (k > 0) {            /* phi(k-1) with k-1 >= 0; phi(-1) is the ground face, 0 */
        s = s + g->tzd1[k] * at(g, p, i, j, k - 1) * (at(g, w, i, j, k - 1) + at(g, w, i, j, k));
        c = c + fabs(g->tzd1[k]) * fabs(at(g, p, i, j, k - 1)) * (fabs(at(g, w, i, j, k - 1)) + fabs(at(g, w, i, j, k)));
    }
    if (k + 1 < nz - 1) {   /* phi(k+1) is the lid when k+1 = nz-1: 0 */
        s = s - g->tzd2[k] * at(g, p, i, j, k + 1) * (at(g, w, i, j, k) + at(g, w, i, j, k + 1));
        c = c + fabs(g->tzd2[k]) * fabs(at(g, p, i, j, k + 1)) * (fabs(at(g, w, i, j, k)) + fabs(at(g, w, i, j, k + 1)));
    }
    if (cond) *cond = c;
    return s;
}

static void fill_grid(pwo_grid *g, int nx, int ny, int nz, double tcx, double tcy,
                      const double *tzc1, const double *tzc2, const double *tzd1, const double *tzd2)
{
    g->nx = nx; g->ny = ny; g->nz = nz; g->tcx = tcx; g->tcy = tcy;
    g->tzc1 = tzc1; g->tzc2 = tzc2; g->tzd1 = tzd1; g->tzd2 = tzd2;
}

/*
 * General bilinear form B(adv; phi): which = 0, 1, 2 selects the u-, v- or
 * w-grid stencil; (u, v, w) advect; phi is advected.  out and cond (optional)
 * are [nx][ny][nz].
 */
void pwo_src(int which, int nx, int ny, int nz, double tcx, double tcy,
             const double *tzc1, const double *tzc2, const double *tzd1, const double *tzd2,
             const double *u, const double *v, const double *w, const double *phi,
             double *out, double *cond)
{
    pwo_grid g;
    fill_grid(&g, nx, ny, nz, tcx, tcy, tzc1, tzc2, tzd1, tzd2);
    long i;
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (i = 0; i < nx; i++)
        for (long j = 0; j < ny; j++)
            for (long k = 0; k < nz; k++) {
                size_t m = ((size_t)i * ny + j) * nz + k;
                double c = 0.0;
                double s = which == 0 ? src_u(&g, u, v, w, phi, i, j, k, &c)
                         : which == 1 ? src_v(&g, u, v, w, phi, i, j, k, &c)
                                      : src_w(&g, u, v, w, phi, i, j, k, &c);
                out[m] = s;
                if (cond) cond[m] = c;
            }
}

/* su, sv, sw = S(u, v, w): each wind component advected by the wind itself */
void pwo_advect(int nx, int ny, int nz, double tcx, double tcy,
                const double *tzc1, const double *tzc2, const double *tzd1, const double *tzd2,
                const double *u, const double *v, const double *w,
                double *su, double *sv, double *sw, double *cu, double *cv, double *cw)
{
    pwo_src(0, nx, ny, nz, tcx, tcy, tzc1, tzc2, tzd1, tzd2, u, v, w, u, su, cu);
    pwo_src(1, nx, ny, nz, tcx, tcy, tzc1, tzc2, tzd1, tzd2, u, v, w, v, sv, cv);
    pwo_src(2, nx, ny, nz, tcx, tcy, tzc1, tzc2, tzd1, tzd2, u, v, w, w, sw, cw);
}

/* S at a list of points only: pts holds n triples (i, j, k); out/cond hold 3n
 * values ordered (su, sv, sw) per point.  For spot checks on large fields. */
void pwo_advect_points(int nx, int ny, int nz, double tcx, double tcy,
                       const double *tzc1, const double *tzc2, const double *tzd1, const double *tzd2,
                       const double *u, const double *v, const double *w,
                       long n, const long *pts, double *out, double *cond)
{
    pwo_grid g;
    fill_grid(&g, nx, ny, nz, tcx, tcy, tzc1, tzc2, tzd1, tzd2);
    for (long p = 0; p < n; p++) {
        long i = pts[3 * p], j = pts[3 * p + 1], k = pts[3 * p + 2];
        double c0, c1, c2;
        out[3 * p + 0] = src_u(&g, u, v, w, u, i, j, k, &c0);
        out[3 * p + 1] = src_v(&g, u, v, w, v, i, j, k, &c1);
        out[3 * p + 2] = src_w(&g, u, v, w, w, i, j, k, &c2);
        if (cond) { cond[3 * p] = c0; cond[3 * p + 1] = c1; cond[3 * p + 2] = c2; }
    }
}

/* ------------------------------------------------------------------------ */
/* adjoint: transpose of the Jacobian of S at (u, v, w)                     */
/* ------------------------------------------------------------------------ */
/*
 * Written independently of the forward functions, from a table of the same
 * terms: every source term is  sign * coef * phi(P) * (a(Q1) + a(Q2)),  with phi
 * the advected component and a the advecting one.  Its derivative sends
 *   y * sign * coef * (a(Q1) + a(Q2))  to the gradient of phi at P, and
 *   y * sign * coef * phi(P)           to the gradient of a at Q1 and at Q2,
 * where y is the incoming gradient of that source at the output point.  The
 * gradient is scattered with periodic wrap, so what the forward reads through a
 * halo copy lands on the interior point it copies.
 */
enum { CX, CY, C1, C2, D1, D2 };
typedef struct {
    int src;            /* 0: su, 1: sv, 2: sw (phi is the same component) */
    int coef;           /* CX tcx, CY tcy, C1 tzc1, C2 tzc2, D1 tzd1, D2 tzd2 */
    int sign;           /* +1 or -1 */
    int pi, pj, pk;     /* offset of phi */
    int a;              /* advecting component: 0 u, 1 v, 2 w */
    int q1i, q1j, q1k, q2i, q2j, q2k;
    int kcond;          /* 0 always; 1 needs k > 0; 2 needs k < nz-1; 3 needs k+1 < nz-1 */
} pwo_term;

static const pwo_term TERMS[18] = {
    /* su */
    {0, CX, +1, -1, 0, 0, 0, -1, 0, 0, 0, 0, 0, 0},
    {0, CX, -1, +1, 0, 0, 0, 0, 0, 0, +1, 0, 0, 0},
    {0, CY, +1, 0, -1, 0, 1, 0, -1, 0, +1, -1, 0, 0},
    {0, CY, -1, 0, +1, 0, 1, 0, 0, 0, +1, 0, 0, 0},
    {0, C1, +1, 0, 0, -1, 2, 0, 0, -1, +1, 0, -1, 1},
    {0, C2, -1, 0, 0, +1, 2, 0, 0, 0, +1, 0, 0, 2},
    /* sv */
    {1, CX, +1, -1, 0, 0, 0, -1, 0, 0, -1, +1, 0, 0},
    {1, CX, -1, +1, 0, 0, 0, 0, 0, 0, 0, +1, 0, 0},
    {1, CY, +1, 0, -1, 0, 1, 0, -1, 0, 0, 0, 0, 0},
    {1, CY, -1, 0, +1, 0, 1, 0, 0, 0, 0, +1, 0, 0},
    {1, C1, +1, 0, 0, -1, 2, 0, 0, -1, 0, +1, -1, 1},
    {1, C2, -1, 0, 0, +1, 2, 0, 0, 0, 0, +1, 0, 2},
    /* sw (only rows k < nz-1 exist) */
    {2, CX, +1, -1, 0, 0, 0, -1, 0, 0, -1, 0, +1, 0},
    {2, CX, -1, +1, 0, 0, 0, 0, 0, 0, 0, 0, +1, 0},
    {2, CY, +1, 0, -1, 0, 1, 0, -1, 0, 0, -1, +1, 0},
    {2, CY, -1, 0, +1, 0, 1, 0, 0, 0, 0, 0, +1, 0},
    {2, D1, +1, 0, 0, -1, 2, 0, 0, -1, 0, 0, 0, 1},
    {2, D2, -1, 0, 0, +1, 2, 0, 0, 0, 0, 0, +1, 3},
};

static size_t pidx(const pwo_grid *g, long i, long j, long k)
{
    return ((size_t)wrap(i, g->nx) * (size_t)g->ny + (size_t)wrap(j, g->ny)) * (size_t)g->nz + (size_t)k;
}

void pwo_adjoint_mode(int nx, int ny, int nz, double tcx, double tcy,
                      const double *tzc1, const double *tzc2, const double *tzd1, const double *tzd2,
                      const double *u, const double *v, const double *w,
                      const double *gsu, const double *gsv, const double *gsw,
                      double *gu, double *gv, double *gw, int beta, int abs_mode);

/*
 * gu, gv, gw = J(u,v,w)^T (gsu, gsv, gsw).  If beta is 0 the outputs are
 * overwritten, otherwise added to.  Sequential (scatter) so the summation order
 * is fixed.
 */
void pwo_adjoint(int nx, int ny, int nz, double tcx, double tcy,
                 const double *tzc1, const double *tzc2, const double *tzd1, const double *tzd2,
                 const double *u, const double *v, const double *w,
                 const double *gsu, const double *gsv, const double *gsw,
                 double *gu, double *gv, double *gw, int beta)
{
    pwo_adjoint_mode(nx, ny, nz, tcx, tcy, tzc1, tzc2, tzd1, tzd2, u, v, w, gsu, gsv, gsw,
                     gu, gv, gw, beta, 0);
}

/* Same scatter with every contribution replaced by its absolute value
 * (abs_mode = 1): the per-point condition sums of the gradient, used to scale
 * tolerances of reduced-precision gradients. */
void pwo_adjoint_mode(int nx, int ny, int nz, double tcx, double tcy,
                      const double *tzc1, const double *tzc2, const double *tzd1, const double *tzd2,
                      const double *u, const double *v, const double *w,
                      const double *gsu, const double *gsv, const double *gsw,
                      double *gu, double *gv, double *gw, int beta, int abs_mode)
{
    pwo_grid g;
    fill_grid(&g, nx, ny, nz, tcx, tcy, tzc1, tzc2, tzd1, tzd2);
    size_t n = (size_t)nx * ny * nz;
    if (!beta) {
        memset(gu, 0, n * sizeof(double));
        memset(gv, 0, n * sizeof(double));
        memset(gw, 0, n * sizeof(double));
    }
    const double *fld[3] = {u, v, w};
    const double *ys[3] = {gsu, gsv, gsw};
    double *gs[3] = {gu, gv, gw};
    for (long i = 0; i < nx; i++)
        for (long j = 0; j < ny; j++)
            for (long k = 0; k < nz; k++)
                for (int t = 0; t < 18; t++) {
                    const pwo_term *T = &TERMS[t];
                    if (T->src == 2 && k >= nz - 1) continue;
                    if (T->kcond == 1 && !(k > 0)) continue;
                    if (T->kcond == 2 && !(k < nz - 1)) continue;
                    if (T->kcond == 3 && !(k + 1 < nz - 1)) continue;
                    double coef = T->coef == CX ? tcx : T->coef == CY ? tcy
                                : T->coef == C1 ? tzc1[k] : T->coef == C2 ? tzc2[k]
                                : T->coef == D1 ? tzd1[k] : tzd2[k];
                    double y = ys[T->src][pidx(&g, i, j, k)];
                    size_t P = pidx(&g, i + T->pi, j + T->pj, k + T->pk);
                    size_t Q1 = pidx(&g, i + T->q1i, j + T->q1j, k + T->q1k);
                    size_t Q2 = pidx(&g, i + T->q2i, j + T->q2j, k + T->q2k);
                    const double *a = fld[T->a];
                    double phi = fld[T->src][P];
                    double sc = T->sign * coef * y;
                    if (abs_mode) {
                        gs[T->src][P] += fabs(sc) * (fabs(a[Q1]) + fabs(a[Q2]));
                        gs[T->a][Q1] += fabs(sc * phi);
                        gs[T->a][Q2] += fabs(sc * phi);
                        continue;
                    }
                    gs[T->src][P] += sc * (a[Q1] + a[Q2]);
                    gs[T->a][Q1] += sc * phi;
                    gs[T->a][Q2] += sc * phi;
                }
}

/* ------------------------------------------------------------------------ */
/* A5: conservation diagnostics                                             */
/* ------------------------------------------------------------------------ */
/*
 * Weights: W = rho_n(k) dz(k) on the u and v levels, W = rho_w(k) dzn(k) on the
 * w faces k < nz-1 (the lid face carries no weight).  For each component
 * phi in (u, v, w) with source S:
 *   out[4c+0] = sum W phi S        out[4c+1] = sum W |phi S|
 *   out[4c+2] = sum W S            out[4c+3] = sum W |S|
 * so R_E = out[4c]/out[4c+1] and R_M = out[4c+2]/out[4c+3].  Sequential sums.
 */
void pwo_residual_sums(int nx, int ny, int nz, const double *rhon, const double *dz,
                       const double *rhow, const double *dzn,
                       const double *u, const double *v, const double *w,
                       const double *su, const double *sv, const double *sw, double *out)
{
    const double *f[3] = {u, v, w};
    const double *s[3] = {su, sv, sw};
    for (int c = 0; c < 3; c++) {
        double a = 0.0, b = 0.0, m = 0.0, n = 0.0;
        for (long i = 0; i < nx; i++)
            for (long j = 0; j < ny; j++)
                for (long k = 0; k < nz; k++) {
                    double W;
                    if (c < 2) W = rhon[k] * dz[k];
                    else W = (k < nz - 1) ? rhow[k] * dzn[k] : 0.0;
                    size_t idx = ((size_t)i * ny + j) * nz + k;
                    double ps = f[c][idx] * s[c][idx];
                    a = a + W * ps;
                    b = b + W * fabs(ps);
                    m = m + W * s[c][idx];
                    n = n + W * fabs(s[c][idx]);
                }
        out[4 * c + 0] = a; out[4 * c + 1] = b; out[4 * c + 2] = m; out[4 * c + 3] = n;
    }
}

/*
 * Discrete divergence of the advecting face sums seen by each stencil, used for
 * the momentum identity  sum W S_phi = sum W phi D_phi  (summation by parts):
 * for a stencil c [A_{m-1/2} phi_{m-1} - A_{m+1/2} phi_{m+1}] per direction,
 * D(m) = c_+ A_{m+1/2} - c_- A_{m-1/2} with the same face sums A and the
 * coefficient of each face (tzc2/tzc1, tzd2/tzd1 vertically; faces at the
 * ground or lid carry A = 0).  which = 0, 1, 2 for the u, v, w grids.
 */
void pwo_face_divergence(int which, int nx, int ny, int nz, double tcx, double tcy,
                         const double *tzc1, const double *tzc2, const double *tzd1, const double *tzd2,
                         const double *u, const double *v, const double *w, double *out)
{
    pwo_grid g;
    fill_grid(&g, nx, ny, nz, tcx, tcy, tzc1, tzc2, tzd1, tzd2);
    for (long i = 0; i < nx; i++)
        for (long j = 0; j < ny; j++)
            for (long k = 0; k < nz; k++) {
                double Axm, Axp, Aym, Ayp, Azm = 0.0, Azp = 0.0, cm, cp;
                if (which == 0) {
                    Axm = at(&g, u, i - 1, j, k) + at(&g, u, i, j, k);
                    Axp = at(&g, u, i, j, k) + at(&g, u, i + 1, j, k);
                    Aym = at(&g, v, i, j - 1, k) + at(&g, v, i + 1, j - 1, k);
                    Ayp = at(&g, v, i, j, k) + at(&g, v, i + 1, j, k);
                    if (k > 0) Azm = at(&g, w, i, j, k - 1) + at(&g, w, i + 1, j, k - 1);
                    if (k < nz - 1) Azp = at(&g, w, i, j, k) + at(&g, w, i + 1, j, k);
                    cm = tzc1[k]; cp = tzc2[k];
                } else if (which == 1) {
                    Axm = at(&g, u, i - 1, j, k) + at(&g, u, i - 1, j + 1, k);
                    Axp = at(&g, u, i, j, k) + at(&g, u, i, j + 1, k);
                    Aym = at(&g, v, i, j - 1, k) + at(&g, v, i, j, k);
                    Ayp = at(&g, v, i, j, k) + at(&g, v, i, j + 1, k);
                    if (k > 0) Azm = at(&g, w, i, j, k - 1) + at(&g, w, i, j + 1, k - 1);
                    if (k < nz - 1) Azp = at(&g, w, i, j, k) + at(&g, w, i, j + 1, k);
                    cm = tzc1[k]; cp = tzc2[k];
                } else {
                    size_t m = ((size_t)i * ny + j) * nz + k;
                    if (k >= nz - 1) { out[m] = 0.0; continue; }
                    Axm = at(&g, u, i - 1, j, k) + at(&g, u, i - 1, j, k + 1);
                    Axp = at(&g, u, i, j, k) + at(&g, u, i, j, k + 1);
                    Aym = at(&g, v, i, j - 1, k) + at(&g, v, i, j - 1, k + 1);
                    Ayp = at(&g, v, i, j, k) + at(&g, v, i, j, k + 1);
                    /* the w cell around face k has faces at zn(k) and zn(k+1) */
                    if (k > 0) Azm = at(&g, w, i, j, k - 1) + at(&g, w, i, j, k);
                    if (k + 1 < nz - 1) Azp = at(&g, w, i, j, k) + at(&g, w, i, j, k + 1);
                    cm = tzd1[k]; cp = tzd2[k];
                }
                size_t m = ((size_t)i * ny + j) * nz + k;
                out[m] = tcx * (Axp - Axm) + tcy * (Ayp - Aym) + (cp * Azp - cm * Azm);
            }
}

/* ------------------------------------------------------------------------ */
/* forward Euler: x <- x + dt S(x), nsteps times (in place)                 */
/* ------------------------------------------------------------------------ */
int pwo_euler(int nx, int ny, int nz, double tcx, double tcy,
              const double *tzc1, const double *tzc2, const double *tzd1, const double *tzd2,
              double *u, double *v, double *w, double dt, int nsteps)
{
    size_t n = (size_t)nx * ny * nz;
    double *s = (double *)malloc(3 * n * sizeof(double));
    if (!s) return -1;
    for (int t = 0; t < nsteps; t++) {
        pwo_advect(nx, ny, nz, tcx, tcy, tzc1, tzc2, tzd1, tzd2, u, v, w,
                   s, s + n, s + 2 * n, NULL, NULL, NULL);
        for (size_t m = 0; m < n; m++) {
            u[m] = u[m] + dt * s[m];
            v[m] = v[m] + dt * s[n + m];
            w[m] = w[m] + dt * s[2 * n + m];
        }
    }
    free(s);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* scalars: theta and the moisture / tracer fields q                        */
/* ------------------------------------------------------------------------ */
/*
 * Section 3 of the paper: the advection kernels serve every advected field;
 * u, v and w are shared between them, and theta and the q fields are the
 * further fields the device may be asked to advect.  A scalar phi sits at the
 * cell centre (x_i, y_j, zn_k), so the six faces of its cell carry the wind
 * components themselves: u(i-1,j,k) west and u(i,j,k) east, v(i,j-1,k) south
 * and v(i,j,k) north, w(i,j,k-1) at the bottom (the ground when k = 0: w = 0)
 * and w(i,j,k) at the top (the lid when k = nz-1: w = 0).  The PW skew form
 * with these face velocities taken as they are (no averaging, so the
 * coefficients are 0.5 where the momentum stencils have 0.25):
 *   s = hx [u(i-1) phi(i-1) - u(i) phi(i+1)] + hy [v(j-1) phi(j-1) - v(j) phi(j+1)]
 *     + hz1(k) w(k-1) phi(k-1) - hz2(k) w(k) phi(k+1)
 *   hx = 0.5/dx, hy = 0.5/dy,
 *   hz1(k) = 0.5 rho_w(k-1) / (rho_n(k) dz(k)),  hz2(k) = 0.5 rho_w(k) / (rho_n(k) dz(k)),
 * with rho_w(-1) = rho0 (the ground face).
 */
void pwo_scalar_coeffs(int nz, const double *dz, const double *rhon, const double *rhow, double rho0,
                       double *hz1, double *hz2)
{
    for (int k = 0; k < nz; k++) {
        double rho_face_below = (k == 0) ? rho0 : rhow[k - 1];
        hz1[k] = 0.5 * rho_face_below / (rhon[k] * dz[k]);
        hz2[k] = 0.5 * rhow[k] / (rhon[k] * dz[k]);
    }
}

static double src_scalar(const pwo_grid *g, const double *hz1, const double *hz2,
                         const double *u, const double *v, const double *w, const double *p,
                         long i, long j, long k, double *cond)
{
    long nz = g->nz;
    double s, c;
    s = g->tcx * (at(g, u, i - 1, j, k) * at(g, p, i - 1, j, k) - at(g, u, i, j, k) * at(g, p, i + 1, j, k));
    c = fabs(g->tcx) * (fabs(at(g, u, i - 1, j, k)) * fabs(at(g, p, i - 1, j, k))
                      + fabs(at(g, u, i, j, k)) * fabs(at(g, p, i + 1, j, k)));
    s = s + g->tcy * (at(g, v, i, j - 1, k) * at(g, p, i, j - 1, k) - at(g, v, i, j, k) * at(g, p, i, j + 1, k));
    c = c + fabs(g->tcy) * (fabs(at(g, v, i, j - 1, k)) * fabs(at(g, p, i, j - 1, k))
                          + fabs(at(g, v, i, j, k)) * fabs(at(g, p, i, j + 1, k)));
    if (k > 0) {            /* bottom face of cell 0 is the ground: w = 0 */
        s = s + hz1[k] * at(g, w, i, j, k - 1) * at(g, p, i, j, k - 1);
        c = c + fabs(hz1[k]) * fabs(at(g, w, i, j, k - 1)) * fabs(at(g, p, i, j, k - 1));
    }
    if (k < nz - 1) {       /* top face of cell nz-1 is the lid: w = 0 */
        s = s - hz2[k] * at(g, w, i, j, k) * at(g, p, i, j, k + 1);
        c = c + fabs(hz2[k]) * fabs(at(g, w, i, j, k)) * fabs(at(g, p, i, j, k + 1));
    }
    if (cond) *cond = c;
    return s;
}

/* s (and optionally cond) = the PW source of the scalar phi advected by (u, v, w) */
void pwo_scalar_src(int nx, int ny, int nz, double hx, double hy, const double *hz1, const double *hz2,
                    const double *u, const double *v, const double *w, const double *phi,
                    double *out, double *cond)
{
    pwo_grid g;
    fill_grid(&g, nx, ny, nz, hx, hy, NULL, NULL, NULL, NULL);
    long i;
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (i = 0; i < nx; i++)
        for (long j = 0; j < ny; j++)
            for (long k = 0; k < nz; k++) {
                size_t m = ((size_t)i * ny + j) * nz + k;
                double c = 0.0;
                out[m] = src_scalar(&g, hz1, hz2, u, v, w, phi, i, j, k, &c);
                if (cond) cond[m] = c;
            }
}

/* the scalar source at a list of points (n triples i, j, k) */
void pwo_scalar_points(int nx, int ny, int nz, double hx, double hy, const double *hz1, const double *hz2,
                       const double *u, const double *v, const double *w, const double *phi,
                       long n, const long *pts, double *out, double *cond)
{
    pwo_grid g;
    fill_grid(&g, nx, ny, nz, hx, hy, NULL, NULL, NULL, NULL);
    for (long p = 0; p < n; p++) {
        double c = 0.0;
        out[p] = src_scalar(&g, hz1, hz2, u, v, w, phi, pts[3 * p], pts[3 * p + 1], pts[3 * p + 2], &c);
        if (cond) cond[p] = c;
    }
}

/* ------------------------------------------------------------------------ */
/* (f)4: the positivity-preserving scheme, ULTIMATE-limited QUICKEST         */
/* ------------------------------------------------------------------------ */
/*
 * Section 3.1 (and section 4) names MONC's second advection scheme: Leonard et
 * al.'s ULTIMATE scheme, positivity preserving, column fluxes feeding the next
 * column, about sixteen times the PW work.  The paper writes none of it out;
 * the reading taken here is the published scheme of that name, in flux form on
 * the same C-grid, the three directions summed from the same state:
 *
 *   s = (u(i-1) f_x(i-1) - u(i) f_x(i)) / dx + (v(j-1) f_y(j-1) - v(j) f_y(j)) / dy
 *     + fz1(k) w(k-1) f_z(k-1) - fz2(k) w(k) f_z(k)
 *   fz1(k) = rho_w(k-1) / (rho_n(k) dz(k)),  fz2(k) = rho_w(k) / (rho_n(k) dz(k)),
 *
 * f_x(i) the face value of phi on the face between cells i and i+1 (where u(i)
 * sits), f_y(j) and f_z(k) likewise; the ground face w(-1) and the lid w(nz-1)
 * carry no flux (their terms are dropped, the stored lid value is never read).
 *
 * Face value, for a face with velocity a between the lower cell L and the
 * upper cell R.  The flow direction names the cells: a >= 0: C = L (upwind),
 * D = R (downwind), U = L - 1 (far upwind); a < 0: C = R, D = L, U = R + 1.
 * The Courant number is c = |a| dt / h_C with h_C the width of cell C along the
 * face normal (dx, dy, or dz(C)).
 *  - QUICKEST (Leonard 1979): the mean, over the fluid that crosses the face
 *    in one step, of the parabola whose cell averages are phi_U, phi_C, phi_D:
 *      q = (phi_C + phi_D)/2 - c (phi_D - phi_C)/2 - (1 - c^2)/6 (phi_D - 2 phi_C + phi_U)
 *  - ULTIMATE (Leonard 1991), in the normalised variable
 *    t(x) = (x - phi_U) / (phi_D - phi_U): where phi_C lies strictly between
 *    phi_U and phi_D, t(f) = t(q) held to [t(phi_C), min(1, t(phi_C) / c)]
 *    (the upper end taken first); where it does not, f = phi_C.
 *  - a face whose U cell would lie below the ground or above the lid takes
 *    f = phi_C (first-order upwind).
 * For constant a and c <= 1 in one dimension this makes the step
 * phi + dt s total-variation diminishing; at c = 1 it is an exact shift by one
 * cell; on the cell averages of a quadratic that the limiter leaves alone it is
 * exact.
 *
 * The condition sum of a point is the sum over its six faces of
 * |coefficient a| (|phi_U| + |phi_C| + |phi_D|) (only |phi_C| where the face is
 * first order): the scale of the rounding error of any evaluation order.
 */
static double quickest(double pu, double pc, double pd, double c)
{
    return 0.5 * (pc + pd) - 0.5 * c * (pd - pc) - (1.0 - c * c) / 6.0 * (pd - 2.0 * pc + pu);
}

static double ultimate(double pu, double pc, double pd, double c)
{
    int monotone = (pu < pc && pc < pd) || (pd < pc && pc < pu);
    if (!monotone) return pc;
    double del = pd - pu;
    double tc = (pc - pu) / del;
    double tf = (quickest(pu, pc, pd, c) - pu) / del;
    double top = (c > tc) ? tc / c : 1.0;   /* min(1, tc / c) */
    if (tf > top) tf = top;
    if (tf < tc) tf = tc;
    return pu + tf * del;
}

/* the face value between cells L and R; pl2, pr2 are the cells beyond them
   (L - 1 and R + 1), have_l2 / have_r2 whether those exist; *mag gets the
   face's error scale |phi_U| + |phi_C| + |phi_D| */
static double tvd_face(double a, double c, double pl2, double pl, double pr, double pr2,
                       int have_l2, int have_r2, double *mag)
{
    if (a >= 0.0) {
        if (!have_l2) {
            *mag = fabs(pl);
            return pl;
        }
        *mag = fabs(pl2) + fabs(pl) + fabs(pr);
        return ultimate(pl2, pl, pr, c);
    }
    if (!have_r2) {
        *mag = fabs(pr);
        return pr;
    }
    *mag = fabs(pr2) + fabs(pr) + fabs(pl);
    return ultimate(pr2, pr, pl, c);
}

/* fz1, fz2 of the flux form; fz1(0) and fz2(nz-1) are 0 (ground, lid) */
void pwo_tvd_coeffs(int nz, const double *dz, const double *rhon, const double *rhow,
                    double *fz1, double *fz2)
{
    for (int k = 0; k < nz; k++) {
        fz1[k] = (k > 0) ? rhow[k - 1] / (rhon[k] * dz[k]) : 0.0;
        fz2[k] = (k < nz - 1) ? rhow[k] / (rhon[k] * dz[k]) : 0.0;
    }
}

typedef struct {
    long nx, ny, nz;
    double dx, dy, dt;
    const double *dz, *fz1, *fz2;
} pwo_tvd_grid;

static double tat(const pwo_tvd_grid *g, const double *f, long i, long j, long k)
{
    return f[((size_t)wrap(i, g->nx) * (size_t)g->ny + (size_t)wrap(j, g->ny)) * (size_t)g->nz + (size_t)k];
}

/* face values of phi on the six faces of cell (i, j, k) */
static double src_tvd(const pwo_tvd_grid *g, const double *u, const double *v, const double *w,
                      const double *p, long i, long j, long k, double *cond)
{
    long nz = g->nz;
    double a, c, f, m, s = 0.0, cs = 0.0;

    /* x: west face (u(i-1), cells i-1 | i) and east face (u(i), cells i | i+1) */
    a = tat(g, u, i - 1, j, k);
    c = fabs(a) * g->dt / g->dx;
    f = tvd_face(a, c, tat(g, p, i - 2, j, k), tat(g, p, i - 1, j, k), tat(g, p, i, j, k),
                 tat(g, p, i + 1, j, k), 1, 1, &m);
    s = s + a * f / g->dx;
    cs = cs + fabs(a) * m / g->dx;
    a = tat(g, u, i, j, k);
    c = fabs(a) * g->dt / g->dx;
    f = tvd_face(a, c, tat(g, p, i - 1, j, k), tat(g, p, i, j, k), tat(g, p, i + 1, j, k),
                 tat(g, p, i + 2, j, k), 1, 1, &m);
    s = s - a * f / g->dx;
    cs = cs + fabs(a) * m / g->dx;

    /* y: south face (v(j-1)) and north face (v(j)) */
    a = tat(g, v, i, j - 1, k);
    c = fabs(a) * g->dt / g->dy;
    f = tvd_face(a, c, tat(g, p, i, j - 2, k), tat(g, p, i, j - 1, k), tat(g, p, i, j, k),
                 tat(g, p, i, j + 1, k), 1, 1, &m);
    s = s + a * f / g->dy;
    cs = cs + fabs(a) * m / g->dy;
    a = tat(g, v, i, j, k);
    c = fabs(a) * g->dt / g->dy;
    f = tvd_face(a, c, tat(g, p, i, j - 1, k), tat(g, p, i, j, k), tat(g, p, i, j + 1, k),
                 tat(g, p, i, j + 2, k), 1, 1, &m);
    s = s - a * f / g->dy;
    cs = cs + fabs(a) * m / g->dy;

    /* z: bottom face w(k-1) (cells k-1 | k; none at the ground) and top face
       w(k) (cells k | k+1; none at the lid) */
    if (k > 0) {
        a = tat(g, w, i, j, k - 1);
        c = fabs(a) * g->dt / g->dz[a >= 0.0 ? k - 1 : k];
        f = tvd_face(a, c, k >= 2 ? tat(g, p, i, j, k - 2) : 0.0, tat(g, p, i, j, k - 1), tat(g, p, i, j, k),
                     k + 1 < nz ? tat(g, p, i, j, k + 1) : 0.0, k >= 2, k + 1 < nz, &m);
        s = s + g->fz1[k] * a * f;
        cs = cs + fabs(g->fz1[k] * a) * m;
    }
    if (k < nz - 1) {
        a = tat(g, w, i, j, k);
        c = fabs(a) * g->dt / g->dz[a >= 0.0 ? k : k + 1];
        f = tvd_face(a, c, k >= 1 ? tat(g, p, i, j, k - 1) : 0.0, tat(g, p, i, j, k), tat(g, p, i, j, k + 1),
                     k + 2 < nz ? tat(g, p, i, j, k + 2) : 0.0, k >= 1, k + 2 < nz, &m);
        s = s - g->fz2[k] * a * f;
        cs = cs + fabs(g->fz2[k] * a) * m;
    }
    if (cond) *cond = cs;
    return s;
}

static void fill_tvd_grid(pwo_tvd_grid *g, int nx, int ny, int nz, double dx, double dy, double dt,
                          const double *dz, const double *fz1, const double *fz2)
{
    g->nx = nx;
    g->ny = ny;
    g->nz = nz;
    g->dx = dx;
    g->dy = dy;
    g->dt = dt;
    g->dz = dz;
    g->fz1 = fz1;
    g->fz2 = fz2;
}

/* s (and optionally cond) = the ULTIMATE-QUICKEST source of phi advected by
   (u, v, w) over one step dt */
void pwo_tvd_src(int nx, int ny, int nz, double dx, double dy, double dt, const double *dz,
                 const double *fz1, const double *fz2, const double *u, const double *v, const double *w,
                 const double *phi, double *out, double *cond)
{
    pwo_tvd_grid g;
    fill_tvd_grid(&g, nx, ny, nz, dx, dy, dt, dz, fz1, fz2);
    long i;
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (i = 0; i < nx; i++)
        for (long j = 0; j < ny; j++)
            for (long k = 0; k < nz; k++) {
                size_t m = ((size_t)i * ny + j) * nz + k;
                double c = 0.0;
                out[m] = src_tvd(&g, u, v, w, phi, i, j, k, &c);
                if (cond) cond[m] = c;
            }
}

/* the same at a list of points (n triples i, j, k) */
void pwo_tvd_points(int nx, int ny, int nz, double dx, double dy, double dt, const double *dz,
                    const double *fz1, const double *fz2, const double *u, const double *v, const double *w,
                    const double *phi, long n, const long *pts, double *out, double *cond)
{
    pwo_tvd_grid g;
    fill_tvd_grid(&g, nx, ny, nz, dx, dy, dt, dz, fz1, fz2);
    for (long p = 0; p < n; p++) {
        double c = 0.0;
        out[p] = src_tvd(&g, u, v, w, phi, pts[3 * p], pts[3 * p + 1], pts[3 * p + 2], &c);
        if (cond) cond[p] = c;
    }
}
