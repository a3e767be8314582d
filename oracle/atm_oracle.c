/*
 * atm_oracle.c -- plain CPU oracle for the ATM linked-cell method
 * (arXiv 2510.21230).  TEST INFRASTRUCTURE ONLY: loaded by the tests, the
 * smoke check and the benchmark's CPU-baseline leg, never by the library.
 *
 * Everything is FP64 and written for readability, not speed.  Build with
 * -ffp-contract=off so that every product and sum is rounded exactly as
 * written (the truncation decisions are compared bit for bit).
 *
 * Conventions (section 2 of the paper): r_ab = r_a - r_b, the three squared
 * side lengths of a triplet are a = r_ij^2, b = r_ik^2, c = r_jk^2.
 * Interpretations of points the paper leaves open are stated where they are
 * used: strict "<" at the cutoff, the product test taken on the sorted
 * squared sides, base-frame cell shifts for distances inside a traversal.
 */
#include "atm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Potentials                                                               */
/* ------------------------------------------------------------------------ */

/* Eq. atm, with the angles removed through the law of cosines:
 *   u = nu * [ 1/(r_ij^3 r_ik^3 r_jk^3)
 *            + 3 (-a+b+c)(a-b+c)(a+b-c) / (8 r_ij^5 r_ik^5 r_jk^5) ]            */
double orc_atm_u(double a, double b, double c, double nu)
{
    double s = a * b * c;          /* (r_ij r_ik r_jk)^2 */
    double rt = sqrt(s);           /*  r_ij r_ik r_jk    */
    double A = -a + b + c, B = a - b + c, C = a + b - c;
    return nu * (1.0 / (s * rt) + 3.0 * A * B * C / (8.0 * s * s * rt));
}

/* du/da, du/db, du/dc of the expression above, differentiated term by term:
 *   u = nu [ s^(-3/2) + 3/8 P s^(-5/2) ],  s = abc,  P = A B C,
 *   du/da = nu [ -3/2 s^(-5/2) bc + 3/8 ( dP/da s^(-5/2) - 5/2 P s^(-7/2) bc ) ]
 * with dP/da = -BC + AC + AB, dP/db = BC - AC + AB, dP/dc = BC + AC - AB.   */
void orc_atm_du_dsq(double a, double b, double c, double nu, double out[3])
{
    double s = a * b * c, rt = sqrt(s);
    double s52 = s * s * rt, s72 = s52 * s;
    double A = -a + b + c, B = a - b + c, C = a + b - c;
    double P = A * B * C;
    double Pa = -B * C + A * C + A * B;
    double Pb = B * C - A * C + A * B;
    double Pc = B * C + A * C - A * B;
    out[0] = nu * (-1.5 * b * c / s52 + 0.375 * (Pa / s52 - 2.5 * P * b * c / s72));
    out[1] = nu * (-1.5 * a * c / s52 + 0.375 * (Pb / s52 - 2.5 * P * a * c / s72));
    out[2] = nu * (-1.5 * a * b / s52 + 0.375 * (Pc / s52 - 2.5 * P * a * b / s72));
}

/* Eq. ATMGradient: the paper's eleven-term closed form of du/dr_ij. */
double orc_atm_dudr_paper(double rij, double rik, double rjk, double nu)
{
    double x = rij, y = rik, z = rjk;
    double t = 0.0;
    t += -1.0 / (pow(x, 4) * pow(y, 3) * pow(z, 3));
    t += -1.0 / (8.0 * pow(y, 5) * pow(z, 5));
    t += 5.0 * y / (8.0 * pow(x, 6) * pow(z, 5));
    t += 5.0 * z / (8.0 * pow(x, 6) * pow(y, 5));
    t += -1.0 / (8.0 * pow(x, 2) * pow(y, 3) * pow(z, 5));
    t += -1.0 / (8.0 * pow(x, 2) * pow(y, 5) * pow(z, 3));
    t += -3.0 / (8.0 * pow(x, 4) * y * pow(z, 5));
    t += -3.0 / (8.0 * pow(x, 4) * pow(y, 5) * z);
    t += -5.0 / (8.0 * pow(x, 6) * y * pow(z, 3));
    t += -5.0 / (8.0 * pow(x, 6) * pow(y, 3) * z);
    t += 6.0 / (8.0 * pow(x, 4) * pow(y, 3) * pow(z, 3));
    return 3.0 * nu * t;
}

/* ------------------------------------------------------------------------ */
/* Linked cells (section 3: cell edge >= r_c, lexicographic cell order)     */
/* ------------------------------------------------------------------------ */

typedef struct {
    double L[3], rc, nu, eps, sig;
    int shift;
    int nc[3];
    double w[3];
    int64_t ncell;
} grid_t;

int orc_cell_grid(const double* prm, int32_t ncell[3], double w[3])
{
    for (int d = 0; d < 3; d++) {
        double L = prm[d], rc = prm[3];
        if (!(L > 0.0) || !(rc > 0.0) || !isfinite(L) || !isfinite(rc)) return 1;
        /* largest k with L/k >= rc, decided on the rounded quotient */
        double k = floor(L / rc);
        if (k < 1.0) k = 1.0;
        while (L / (k + 1.0) >= rc) k += 1.0;
        while (k > 0.0 && L / k < rc) k -= 1.0;
        if (k < 3.0) return 2;
        if (k > 1.0e6) return 1;
        ncell[d] = (int32_t)k;
        w[d] = L / k;
    }
    return 0;
}

static int grid_init(const double* prm, grid_t* g)
{
    int32_t nc[3];
    double w[3];
    int st = orc_cell_grid(prm, nc, w);
    if (st) return st;
    for (int d = 0; d < 3; d++) {
        g->L[d] = prm[d];
        g->nc[d] = nc[d];
        g->w[d] = w[d];
    }
    g->rc = prm[3];
    g->nu = prm[4];
    g->eps = prm[5];
    g->sig = prm[6];
    g->shift = prm[7] != 0.0;
    g->ncell = (int64_t)nc[0] * nc[1] * nc[2];
    return 0;
}

/* periodic wrap into [0, L): t = x - L floor(x/L); a result that rounds to
 * L (or below 0) is folded back, and one that still equals L becomes 0 */
static double wrap1(double x, double L)
{
    double t = x - floor(x / L) * L;
    if (t < 0.0) t += L;
    if (t >= L) t = 0.0;
    return t;
}

/* cell coordinate along one axis and the cell-local coordinate in [0, w] */
static int bin1(double t, double w, int n, double* loc)
{
    int c = (int)floor(t / w);
    if (c > n - 1) c = n - 1;
    if (c < 0) c = 0;
    double l = t - (double)c * w;
    if (l < 0.0) l = 0.0;
    if (l > w) l = w;
    *loc = l;
    return c;
}

typedef struct {
    grid_t g;
    int64_t n;
    double* xw;      /* wrapped, original order, SoA */
    int32_t* cell;   /* original order */
    int32_t* start;  /* ncell + 1 */
    int32_t* perm;   /* sorted -> original */
    double* xl;      /* sorted local coordinates, SoA */
    float* xl32;
} cells_t;

static void cells_free(cells_t* c)
{
    free(c->xw);
    free(c->cell);
    free(c->start);
    free(c->perm);
    free(c->xl);
    free(c->xl32);
}

static int cells_make(const double* prm, int64_t n, const double* x, cells_t* c)
{
    memset(c, 0, sizeof(*c));
    if (n < 0) return 1;
    int st = grid_init(prm, &c->g);
    if (st) return st;
    for (int64_t i = 0; i < 3 * n; i++)
        if (!isfinite(x[i])) return 1;
    grid_t* g = &c->g;
    c->n = n;
    size_t nn = (size_t)(n > 0 ? n : 1);
    c->xw = malloc(sizeof(double) * 3 * nn);
    c->cell = malloc(sizeof(int32_t) * nn);
    c->start = calloc((size_t)g->ncell + 1, sizeof(int32_t));
    c->perm = malloc(sizeof(int32_t) * nn);
    c->xl = malloc(sizeof(double) * 3 * nn);
    c->xl32 = malloc(sizeof(float) * 3 * nn);
    double* loc = malloc(sizeof(double) * 3 * nn);
    if (!c->xw || !c->cell || !c->start || !c->perm || !c->xl || !c->xl32 || !loc) {
        free(loc);
        cells_free(c);
        return 1;
    }
    /* A1: wrap, bin, cell id (z-major lexicographic) */
    for (int64_t i = 0; i < n; i++) {
        int cc[3];
        for (int d = 0; d < 3; d++) {
            double t = wrap1(x[d * n + i], g->L[d]);
            c->xw[d * n + i] = t;
            cc[d] = bin1(t, g->w[d], g->nc[d], &loc[d * n + i]);
        }
        c->cell[i] = (cc[2] * g->nc[1] + cc[1]) * g->nc[0] + cc[0];
    }
    /* A2: counting sort, stable in the original index */
    for (int64_t i = 0; i < n; i++) c->start[c->cell[i] + 1]++;
    for (int64_t q = 0; q < g->ncell; q++) c->start[q + 1] += c->start[q];
    int32_t* fill = malloc(sizeof(int32_t) * (size_t)g->ncell);
    memcpy(fill, c->start, sizeof(int32_t) * (size_t)g->ncell);
    for (int64_t i = 0; i < n; i++) {
        int32_t s = fill[c->cell[i]]++;
        c->perm[s] = (int32_t)i;
        for (int d = 0; d < 3; d++) {
            c->xl[d * n + s] = loc[d * n + i];
            c->xl32[d * n + s] = (float)loc[d * n + i];
        }
    }
    free(fill);
    free(loc);
    return 0;
}

int orc_build_cells(const double* prm, int64_t n, const double* x, double* xw,
                    int32_t* cell_of, int32_t* cell_start, int32_t* perm,
                    double* xl, float* xl32)
{
    cells_t c;
    int st = cells_make(prm, n, x, &c);
    if (st) return st;
    if (xw) memcpy(xw, c.xw, sizeof(double) * 3 * n);
    if (cell_of) memcpy(cell_of, c.cell, sizeof(int32_t) * n);
    if (cell_start) memcpy(cell_start, c.start, sizeof(int32_t) * (c.g.ncell + 1));
    if (perm) memcpy(perm, c.perm, sizeof(int32_t) * n);
    if (xl) memcpy(xl, c.xl, sizeof(double) * 3 * n);
    if (xl32) memcpy(xl32, c.xl32, sizeof(float) * 3 * n);
    cells_free(&c);
    return 0;
}

/* neighbour cell of cell id b at offset off (periodic) */
static int64_t nb_cell(const grid_t* g, int64_t b, const int off[3])
{
    int cx = (int)(b % g->nc[0]);
    int cy = (int)((b / g->nc[0]) % g->nc[1]);
    int cz = (int)(b / ((int64_t)g->nc[0] * g->nc[1]));
    cx = (cx + off[0] + g->nc[0]) % g->nc[0];
    cy = (cy + off[1] + g->nc[1]) % g->nc[1];
    cz = (cz + off[2] + g->nc[2]) % g->nc[2];
    return ((int64_t)cz * g->nc[1] + cy) * g->nc[0] + cx;
}

/* ------------------------------------------------------------------------ */
/* One traversal evaluation context                                         */
/* ------------------------------------------------------------------------ */

typedef struct {
    const cells_t* c;
    int trunc, prec;
    double rc2, rc6;       /* FP64 thresholds */
    float rc2f, rc6f;      /* FP32 thresholds */
    float wf[3];           /* FP32 cell edges */
    double* f;             /* forces, sorted order, SoA */
    double e, w;
    uint64_t ncand, nint;
} ev_t;

static void ev_init(ev_t* ev, const cells_t* c, int trunc, int prec, double* f)
{
    memset(ev, 0, sizeof(*ev));
    ev->c = c;
    ev->trunc = trunc;
    ev->prec = prec;
    ev->rc2 = c->g.rc * c->g.rc;
    ev->rc6 = ev->rc2 * ev->rc2 * ev->rc2;
    float rcf = (float)c->g.rc;
    ev->rc2f = rcf * rcf;
    ev->rc6f = ev->rc2f * ev->rc2f * ev->rc2f;
    for (int d = 0; d < 3; d++) ev->wf[d] = (float)c->g.w[d];
    ev->f = f;
}

/* displacement q - p (p sits in the cell at offset op, q at oq, both offsets
 * in cells relative to one base cell) and its square, FP64:
 *   d = (xl_q - xl_p) + (oq - op) w                                          */
static double dsq64(const ev_t* ev, int64_t p, const int op[3], int64_t q, const int oq[3],
                    double d[3])
{
    const cells_t* c = ev->c;
    for (int k = 0; k < 3; k++)
        d[k] = (c->xl[k * c->n + q] - c->xl[k * c->n + p]) + (double)(oq[k] - op[k]) * c->g.w[k];
    return (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
}

/* the same in FP32 on the FP32 local coordinates */
static float dsq32(const ev_t* ev, int64_t p, const int op[3], int64_t q, const int oq[3])
{
    const cells_t* c = ev->c;
    float d[3];
    for (int k = 0; k < 3; k++)
        d[k] = (c->xl32[k * c->n + q] - c->xl32[k * c->n + p]) + (float)(oq[k] - op[k]) * ev->wf[k];
    return (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
}

/* truncation tests (section 2): interacting iff every side < r_c (pair), or
 * r_ij r_ik r_jk < r_c^3 (product), evaluated as (p*q)*r < r_c^6 on the
 * squared sides sorted ascending so that the rounding does not depend on the
 * order in which a traversal names the three molecules.                     */
static int keep64(const ev_t* ev, double a, double b, double c)
{
    if (ev->trunc == ORC_PAIR) return a < ev->rc2 && b < ev->rc2 && c < ev->rc2;
    double t;
    if (a > b) { t = a; a = b; b = t; }
    if (b > c) { t = b; b = c; c = t; }
    if (a > b) { t = a; a = b; b = t; }
    return (a * b) * c < ev->rc6;
}

static int keep32(const ev_t* ev, float a, float b, float c)
{
    if (ev->trunc == ORC_PAIR) return a < ev->rc2f && b < ev->rc2f && c < ev->rc2f;
    float t;
    if (a > b) { t = a; a = b; b = t; }
    if (b > c) { t = b; b = c; c = t; }
    if (a > b) { t = a; a = b; b = t; }
    return (a * b) * c < ev->rc6f;
}

/* pair-rule pre-test of one side; it only skips work the full test below
 * would reject anyway */
static int side_ok(const ev_t* ev, int64_t p, const int op[3], int64_t q, const int oq[3])
{
    if (ev->trunc != ORC_PAIR) return 1;
    if (ev->prec == ORC_FP32) return dsq32(ev, p, op, q, oq) < ev->rc2f;
    double d[3];
    return dsq64(ev, p, op, q, oq, d) < ev->rc2;
}

/* One candidate triplet (i, j, k).  Newton's third law (Eq. forcepairs and
 * Eq. newton3rdlaw): with g_ij = 2 du/da (r_j - r_i) etc.,
 *   F_i = g_ij + g_ik,  F_j = -g_ij + g_jk,  F_k = -g_ik - g_jk.
 * owner_only (3c01): only F_i is written and u/3, W/3 are added per visit.
 * W = r_ij . F_i(j)k + r_ik . F_i(k)j + r_jk . F_j(k)i (Eq. P_3).            */
static void triplet(ev_t* ev, int64_t i, const int oi[3], int64_t j, const int oj[3],
                    int64_t k, const int ok[3], int owner_only)
{
    ev->ncand++;
    if (ev->prec == ORC_FP32) {
        float a32 = dsq32(ev, i, oi, j, oj);
        float b32 = dsq32(ev, i, oi, k, ok);
        float c32 = dsq32(ev, j, oj, k, ok);
        if (!keep32(ev, a32, b32, c32)) return;
    }
    double dij[3], dik[3], djk[3];
    double a = dsq64(ev, i, oi, j, oj, dij);
    double b = dsq64(ev, i, oi, k, ok, dik);
    double c = dsq64(ev, j, oj, k, ok, djk);
    if (ev->prec == ORC_FP64 && !keep64(ev, a, b, c)) return;
    ev->nint++;
    double du[3];
    orc_atm_du_dsq(a, b, c, ev->c->g.nu, du);
    double u = orc_atm_u(a, b, c, ev->c->g.nu);
    double W = 0.0;
    int64_t n = ev->c->n;
    for (int d = 0; d < 3; d++) {
        double gij = 2.0 * du[0] * dij[d];
        double gik = 2.0 * du[1] * dik[d];
        double gjk = 2.0 * du[2] * djk[d];
        ev->f[d * n + i] += gij + gik;
        if (!owner_only) {
            ev->f[d * n + j] += -gij + gjk;
            ev->f[d * n + k] += -gik - gjk;
        }
        /* r_ab = -(d_ab) */
        W += -(dij[d] * gij + dik[d] * gik + djk[d] * gjk);
    }
    if (owner_only) {
        ev->e += u / 3.0;
        ev->w += W / 3.0;
    } else {
        ev->e += u;
        ev->w += W;
    }
}

static const int ZERO3[3] = {0, 0, 0};

/* the 13 forward neighbour offsets: (dz, dy, dx) lexicographically > 0 */
static void forward13(int off[13][3])
{
    int m = 0;
    for (int dz = -1; dz <= 1; dz++)
        for (int dy = -1; dy <= 1; dy++)
            for (int dx = -1; dx <= 1; dx++) {
                int fwd = dz > 0 || (dz == 0 && (dy > 0 || (dy == 0 && dx > 0)));
                if (fwd) {
                    off[m][0] = dx;
                    off[m][1] = dy;
                    off[m][2] = dz;
                    m++;
                }
            }
}

/* ---- 3c01: for i in C_b, all pairs {j, k} of the 27-cell neighbourhood,
 *      forces on i only (section 4, 3c01 traversal) ---------------------- */
static void unit_3c01(ev_t* ev, int64_t b)
{
    const cells_t* c = ev->c;
    int off[27][3];
    int64_t cid[27];
    int m = 0;
    for (int dz = -1; dz <= 1; dz++)
        for (int dy = -1; dy <= 1; dy++)
            for (int dx = -1; dx <= 1; dx++) {
                off[m][0] = dx;
                off[m][1] = dy;
                off[m][2] = dz;
                cid[m] = nb_cell(&c->g, b, off[m]);
                m++;
            }
    for (int64_t i = c->start[b]; i < c->start[b + 1]; i++) {
        for (int s1 = 0; s1 < 27; s1++) {
            for (int64_t j = c->start[cid[s1]]; j < c->start[cid[s1] + 1]; j++) {
                if (j == i) continue;
                int pj = side_ok(ev, i, ZERO3, j, off[s1]);
                for (int s2 = s1; s2 < 27; s2++) {
                    int64_t k0 = (s2 == s1) ? j + 1 : c->start[cid[s2]];
                    for (int64_t k = k0; k < c->start[cid[s2] + 1]; k++) {
                        if (k == i) continue;
                        if (pj)
                            triplet(ev, i, ZERO3, j, off[s1], k, off[s2], 1);
                        else
                            ev->ncand++;
                    }
                }
            }
        }
    }
}

/* ---- 3cw, the wide owner traversal (not in the paper; it measures what the
 *      paper's traversals miss under the product rule): for i in C_b, every
 *      pair {j, k} of molecules of the 5^3 neighbourhood within R_w = 2 min(w)
 *      of i (within r_c under the pair rule, where no longer side can
 *      interact), kept if the third side is shorter than R_w too and the
 *      truncation test holds; forces on i only, u/3 and W/3 per visit.  It
 *      finds every triplet with all sides shorter than R_w, which under the
 *      product rule is every interacting triplet once the closest pair is at
 *      least r_min apart with (r_min + sqrt(r_min^2 + 4 r_c^3 / r_min)) / 2
 *      <= R_w (the longest side L of a triplet with shortest side r_min obeys
 *      r_min (L - r_min) L < r_c^3).  Needs at least 5 cells per axis.
 *      Candidates: the partner pairs of every owner. */
static void unit_3cw(ev_t* ev, int64_t b, int64_t* plist, int* poff)
{
    const cells_t* c = ev->c;
    double wmin = c->g.w[0];
    for (int d = 1; d < 3; d++) wmin = c->g.w[d] < wmin ? c->g.w[d] : wmin;
    const double rw2 = (2.0 * wmin) * (2.0 * wmin);
    const float rw2f = (float)rw2;
    /* partner radius: R_w, or r_c under the pair rule */
    const double pr2 = ev->trunc == ORC_PAIR ? ev->rc2 : rw2;
    const float pr2f = ev->trunc == ORC_PAIR ? ev->rc2f : rw2f;
    int off[125][3];
    int64_t cid[125];
    int m = 0;
    for (int dz = -2; dz <= 2; dz++)
        for (int dy = -2; dy <= 2; dy++)
            for (int dx = -2; dx <= 2; dx++) {
                off[m][0] = dx;
                off[m][1] = dy;
                off[m][2] = dz;
                cid[m] = nb_cell(&c->g, b, off[m]);
                m++;
            }
    for (int64_t i = c->start[b]; i < c->start[b + 1]; i++) {
        /* partners of i: within R_w */
        int64_t np = 0;
        for (int s = 0; s < 125; s++)
            for (int64_t j = c->start[cid[s]]; j < c->start[cid[s] + 1]; j++) {
                if (j == i) continue;
                int in;
                if (ev->prec == ORC_FP32) {
                    in = dsq32(ev, i, ZERO3, j, off[s]) < pr2f;
                } else {
                    double d[3];
                    in = dsq64(ev, i, ZERO3, j, off[s], d) < pr2;
                }
                if (in) {
                    plist[np] = j;
                    poff[np] = s;
                    np++;
                }
            }
        for (int64_t kk = 1; kk < np; kk++)
            for (int64_t jj = 0; jj < kk; jj++) {
                const int64_t j = plist[jj], k = plist[kk];
                const int* oj = off[poff[jj]];
                const int* ok = off[poff[kk]];
                ev->ncand++;
                double dij[3], dik[3], djk[3];
                if (ev->prec == ORC_FP32) {
                    float a32 = dsq32(ev, i, ZERO3, j, oj);
                    float b32 = dsq32(ev, i, ZERO3, k, ok);
                    float c32 = dsq32(ev, j, oj, k, ok);
                    if (!(c32 < rw2f) || !keep32(ev, a32, b32, c32)) continue;
                }
                double a = dsq64(ev, i, ZERO3, j, oj, dij);
                double bb = dsq64(ev, i, ZERO3, k, ok, dik);
                double cc = dsq64(ev, j, oj, k, ok, djk);
                if (ev->prec == ORC_FP64 && (!(cc < rw2) || !keep64(ev, a, bb, cc))) continue;
                ev->nint++;
                double du[3];
                orc_atm_du_dsq(a, bb, cc, c->g.nu, du);
                double u = orc_atm_u(a, bb, cc, c->g.nu);
                double W = 0.0;
                const int64_t n = c->n;
                for (int d = 0; d < 3; d++) {
                    double gij = 2.0 * du[0] * dij[d];
                    double gik = 2.0 * du[1] * dik[d];
                    double gjk = 2.0 * du[2] * djk[d];
                    ev->f[d * n + i] += gij + gik;
                    W += -(dij[d] * gij + dik[d] * gik + djk[d] * gjk);
                }
                ev->e += u / 3.0;
                ev->w += W / 3.0;
            }
    }
}

/* ---- every task holds the base cell: <C_b>, <C_b, C_n1> and
 *      <C_b, C_n1, C_n2> with C_n1 before C_n2 in the partner list -------- */
static void unit_based(ev_t* ev, int64_t b, const int (*po)[3], int np)
{
    const cells_t* c = ev->c;
    int64_t cid[13];
    for (int q = 0; q < np; q++) cid[q] = nb_cell(&c->g, b, po[q]);
    int64_t b0 = c->start[b], b1 = c->start[b + 1];
    /* <C_b>: i < j < k inside the base cell */
    for (int64_t i = b0; i < b1; i++)
        for (int64_t j = i + 1; j < b1; j++) {
            int pj = side_ok(ev, i, ZERO3, j, ZERO3);
            for (int64_t k = j + 1; k < b1; k++) {
                if (pj) triplet(ev, i, ZERO3, j, ZERO3, k, ZERO3, 0);
                else ev->ncand++;
            }
        }
    for (int q = 0; q < np; q++) {
        int64_t n0 = c->start[cid[q]], n1 = c->start[cid[q] + 1];
        /* <C_b, C_n1>: two in C_b and one in C_n1, then one in C_b and two in C_n1 */
        for (int64_t i = b0; i < b1; i++)
            for (int64_t j = i + 1; j < b1; j++) {
                int pj = side_ok(ev, i, ZERO3, j, ZERO3);
                for (int64_t k = n0; k < n1; k++) {
                    if (pj) triplet(ev, i, ZERO3, j, ZERO3, k, po[q], 0);
                    else ev->ncand++;
                }
            }
        for (int64_t i = b0; i < b1; i++)
            for (int64_t j = n0; j < n1; j++) {
                int pj = side_ok(ev, i, ZERO3, j, po[q]);
                for (int64_t k = j + 1; k < n1; k++) {
                    if (pj) triplet(ev, i, ZERO3, j, po[q], k, po[q], 0);
                    else ev->ncand++;
                }
            }
    }
    /* <C_b, C_n1, C_n2>: C_n2 after C_n1 in the partner list */
    for (int q1 = 0; q1 < np; q1++)
        for (int q2 = q1 + 1; q2 < np; q2++) {
            int64_t j0 = c->start[cid[q1]], j1 = c->start[cid[q1] + 1];
            int64_t k0 = c->start[cid[q2]], k1 = c->start[cid[q2] + 1];
            for (int64_t i = b0; i < b1; i++)
                for (int64_t j = j0; j < j1; j++) {
                    int pj = side_ok(ev, i, ZERO3, j, po[q1]);
                    for (int64_t k = k0; k < k1; k++) {
                        if (pj) triplet(ev, i, ZERO3, j, po[q1], k, po[q2], 0);
                        else ev->ncand++;
                    }
                }
        }
}

/* ---- 3c18: base cell, its 13 forward neighbours and every pair of them
 *      (Algorithm 1 with forward neighbours only, section 4) ------------ */
static void unit_3c18(ev_t* ev, int64_t b)
{
    int fw[13][3];
    forward13(fw);
    unit_based(ev, b, (const int (*)[3])fw, 13);
}

/* ---- 3c08 as the text describes it (section 4, Fig. c08traversal): the
 *      procedure of 3c18 with the partners restricted to the 2x2x2 block in
 *      front of the base cell (offsets in {0,1}^3 other than 0, in slot
 *      order x + 2y + 4z), so every task holds the block's corner cell.  A
 *      cell triple of the block that misses the corner (e.g. the three
 *      face neighbours of the corner) belongs to no task: the omitted
 *      interactions the paper mentions. ------------------------------------ */
static void unit_3c08a(ev_t* ev, int64_t b)
{
    int blk[7][3];
    for (int s = 1; s < 8; s++) {
        blk[s - 1][0] = s & 1;
        blk[s - 1][1] = (s >> 1) & 1;
        blk[s - 1][2] = (s >> 2) & 1;
    }
    unit_based(ev, b, (const int (*)[3])blk, 7);
}

/* ---- 3c08: the 2x2x2 block anchored at the base cell; every cell multiset
 *      of the block whose bounding box starts at the anchor, i.e. whose
 *      slot bit patterns (x + 2y + 4z) have an empty common AND ---------- */
static void unit_3c08(ev_t* ev, int64_t b)
{
    const cells_t* c = ev->c;
    int off[8][3];
    int64_t cid[8], s0[8], s1[8];
    for (int s = 0; s < 8; s++) {
        off[s][0] = s & 1;
        off[s][1] = (s >> 1) & 1;
        off[s][2] = (s >> 2) & 1;
        cid[s] = nb_cell(&c->g, b, off[s]);
        s0[s] = c->start[cid[s]];
        s1[s] = c->start[cid[s] + 1];
    }
    /* one cell: the anchor */
    for (int64_t i = s0[0]; i < s1[0]; i++)
        for (int64_t j = i + 1; j < s1[0]; j++) {
            int pj = side_ok(ev, i, off[0], j, off[0]);
            for (int64_t k = j + 1; k < s1[0]; k++) {
                if (pj) triplet(ev, i, off[0], j, off[0], k, off[0], 0);
                else ev->ncand++;
            }
        }
    /* two cells */
    for (int s = 0; s < 8; s++)
        for (int t = s + 1; t < 8; t++) {
            if ((s & t) != 0) continue;
            for (int64_t i = s0[s]; i < s1[s]; i++)
                for (int64_t j = i + 1; j < s1[s]; j++) {
                    int pj = side_ok(ev, i, off[s], j, off[s]);
                    for (int64_t k = s0[t]; k < s1[t]; k++) {
                        if (pj) triplet(ev, i, off[s], j, off[s], k, off[t], 0);
                        else ev->ncand++;
                    }
                }
            for (int64_t i = s0[s]; i < s1[s]; i++)
                for (int64_t j = s0[t]; j < s1[t]; j++) {
                    int pj = side_ok(ev, i, off[s], j, off[t]);
                    for (int64_t k = j + 1; k < s1[t]; k++) {
                        if (pj) triplet(ev, i, off[s], j, off[t], k, off[t], 0);
                        else ev->ncand++;
                    }
                }
        }
    /* three cells */
    for (int s = 0; s < 8; s++)
        for (int t = s + 1; t < 8; t++)
            for (int u = t + 1; u < 8; u++) {
                if ((s & t & u) != 0) continue;
                for (int64_t i = s0[s]; i < s1[s]; i++)
                    for (int64_t j = s0[t]; j < s1[t]; j++) {
                        int pj = side_ok(ev, i, off[s], j, off[t]);
                        for (int64_t k = s0[u]; k < s1[u]; k++) {
                            if (pj) triplet(ev, i, off[s], j, off[t], k, off[u], 0);
                            else ev->ncand++;
                        }
                    }
            }
}

static int atm_cells_impl(const double* prm, int64_t n, const double* x, int trav, int trunc,
                          int prec, int64_t unit_lo, int64_t unit_hi, const int64_t* units,
                          int64_t nunits, double* f, double* ew, uint64_t* cnt)
{
    if (trav < 0 || trav > 4 || trunc < 0 || trunc > 1 || prec < 0 || prec > 1) return 1;
    cells_t c;
    int st = cells_make(prm, n, x, &c);
    if (st) return st;
    if (trav == ORC_3CW && (c.g.nc[0] < 5 || c.g.nc[1] < 5 || c.g.nc[2] < 5)) {
        cells_free(&c);
        return 2;
    }
    int64_t lo = unit_lo < 0 ? 0 : unit_lo;
    int64_t hi = (unit_hi < 0 || unit_hi > c.g.ncell) ? c.g.ncell : unit_hi;
    if (units) {
        for (int64_t q = 0; q < nunits; q++)
            if (units[q] < 0 || units[q] >= c.g.ncell) {
                cells_free(&c);
                return 1;
            }
        lo = 0;
        hi = nunits;
    }
    double* fs = calloc((size_t)(3 * (n > 0 ? n : 1)), sizeof(double));
    double e = 0.0, w = 0.0;
    uint64_t ncand = 0, nint = 0;
#pragma omp parallel
    {
        double* fl = calloc((size_t)(3 * (n > 0 ? n : 1)), sizeof(double));
        int64_t* plist = trav == ORC_3CW ? malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1)) : NULL;
        int* poff = trav == ORC_3CW ? malloc(sizeof(int) * (size_t)(n > 0 ? n : 1)) : NULL;
        ev_t ev;
        ev_init(&ev, &c, trunc, prec, fl);
#pragma omp for schedule(dynamic, 4)
        for (int64_t q = lo; q < hi; q++) {
            int64_t u = units ? units[q] : q;
            if (trav == ORC_3C01) unit_3c01(&ev, u);
            else if (trav == ORC_3C18) unit_3c18(&ev, u);
            else if (trav == ORC_3C08) unit_3c08(&ev, u);
            else if (trav == ORC_3C08A) unit_3c08a(&ev, u);
            else unit_3cw(&ev, u, plist, poff);
        }
        free(plist);
        free(poff);
#pragma omp critical
        {
            for (int64_t q = 0; q < 3 * n; q++) fs[q] += fl[q];
            e += ev.e;
            w += ev.w;
            ncand += ev.ncand;
            nint += ev.nint;
        }
        free(fl);
    }
    /* back to the original order */
    if (f)
        for (int64_t s = 0; s < n; s++)
            for (int d = 0; d < 3; d++) f[d * n + c.perm[s]] = fs[d * n + s];
    if (ew) {
        ew[0] = e;
        ew[1] = w;
    }
    if (cnt) {
        cnt[0] = ncand;
        cnt[1] = nint;
    }
    free(fs);
    cells_free(&c);
    return 0;
}

int orc_atm_cells(const double* prm, int64_t n, const double* x, int trav, int trunc,
                  int prec, int64_t unit_lo, int64_t unit_hi,
                  double* f, double* ew, uint64_t* cnt)
{
    return atm_cells_impl(prm, n, x, trav, trunc, prec, unit_lo, unit_hi, NULL, 0, f, ew, cnt);
}

int orc_atm_cells_units(const double* prm, int64_t n, const double* x, int trav, int trunc,
                        int prec, const int64_t* units, int64_t nunits,
                        double* f, double* ew, uint64_t* cnt)
{
    if (!units && nunits > 0) return 1;
    return atm_cells_impl(prm, n, x, trav, trunc, prec, 0, 0, units, nunits, f, ew, cnt);
}

/* ------------------------------------------------------------------------ */
/* Brute force with the minimum-image convention                            */
/* ------------------------------------------------------------------------ */

/* minimum-image displacement along one axis: t - rint(t/L) L */
static double min_image(double t, double L)
{
    return t - rint(t / L) * L;
}

static double bf_dsq(const double* xw, int64_t n, const double* L, int64_t p, int64_t q,
                     double d[3])
{
    for (int k = 0; k < 3; k++) d[k] = min_image(xw[k * n + q] - xw[k * n + p], L[k]);
    return (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
}

/* wrapped cell offset of q relative to p along each axis; returns 0 if the
 * cells are not equal-or-adjacent (offset outside {-1, 0, 1}^3) */
static int cell_offset(const grid_t* g, int32_t cp, int32_t cq, int o[3])
{
    int p3[3] = {cp % g->nc[0], (cp / g->nc[0]) % g->nc[1], cp / (g->nc[0] * g->nc[1])};
    int q3[3] = {cq % g->nc[0], (cq / g->nc[0]) % g->nc[1], cq / (g->nc[0] * g->nc[1])};
    for (int d = 0; d < 3; d++) {
        int m = ((q3[d] - p3[d]) % g->nc[d] + g->nc[d]) % g->nc[d];
        if (m == 0) o[d] = 0;
        else if (m == 1) o[d] = 1;
        else if (m == g->nc[d] - 1) o[d] = -1;
        else return 0;
    }
    return 1;
}

static int is_forward(const int o[3])
{
    return o[2] > 0 || (o[2] == 0 && (o[1] > 0 || (o[1] == 0 && o[0] > 0)));
}

/* 3c18 visits an unordered cell triple once iff some member cell sees the
 * other two as itself or as forward neighbours */
static int member_3c18(const grid_t* g, int32_t ci, int32_t cj, int32_t ck)
{
    int32_t cs[3] = {ci, cj, ck};
    for (int x = 0; x < 3; x++) {
        int ok = 1;
        for (int y = 0; y < 3 && ok; y++) {
            if (y == x || cs[y] == cs[x]) continue;
            int o[3];
            if (!cell_offset(g, cs[x], cs[y], o) || !is_forward(o)) ok = 0;
        }
        if (ok) return 1;
    }
    return 0;
}

/* 3c08 visits a cell multiset iff it fits in one 2x2x2 block: along every
 * axis the distinct coordinates are one value, or two cyclically adjacent */
static int member_3c08(const grid_t* g, int32_t ci, int32_t cj, int32_t ck)
{
    int32_t cs[3] = {ci, cj, ck};
    for (int d = 0; d < 3; d++) {
        int v[3];
        for (int m = 0; m < 3; m++) {
            int32_t q = cs[m];
            v[m] = d == 0 ? q % g->nc[0] : d == 1 ? (q / g->nc[0]) % g->nc[1]
                                                  : q / (g->nc[0] * g->nc[1]);
        }
        int u[3], nu = 0;
        for (int m = 0; m < 3; m++) {
            int seen = 0;
            for (int r = 0; r < nu; r++) seen |= u[r] == v[m];
            if (!seen) u[nu++] = v[m];
        }
        if (nu == 3) return 0;
        if (nu == 2) {
            int diff = ((u[1] - u[0]) % g->nc[d] + g->nc[d]) % g->nc[d];
            if (diff != 1 && diff != g->nc[d] - 1) return 0;
        }
    }
    return 1;
}

/* the corner-anchored 3c08 visits a cell multiset iff it fits in one 2x2x2
 * block and that block's corner (the smallest coordinate along every axis,
 * cyclically) is one of its cells */
static int member_3c08a(const grid_t* g, int32_t ci, int32_t cj, int32_t ck)
{
    if (!member_3c08(g, ci, cj, ck)) return 0;
    int32_t cs[3] = {ci, cj, ck};
    int v[3][3], lo[3];
    for (int m = 0; m < 3; m++) {
        v[m][0] = cs[m] % g->nc[0];
        v[m][1] = (cs[m] / g->nc[0]) % g->nc[1];
        v[m][2] = cs[m] / (g->nc[0] * g->nc[1]);
    }
    for (int d = 0; d < 3; d++) {
        /* two distinct values are cyclic neighbours: the lower one is the one
         * whose successor is the other */
        lo[d] = v[0][d];
        for (int m = 1; m < 3; m++)
            if (v[m][d] != lo[d] && (v[m][d] + 1) % g->nc[d] == lo[d]) lo[d] = v[m][d];
    }
    for (int m = 0; m < 3; m++)
        if (v[m][0] == lo[0] && v[m][1] == lo[1] && v[m][2] == lo[2]) return 1;
    return 0;
}

static int bf_keep(double rc2, double rc6, int trunc, double a, double b, double c)
{
    if (trunc == ORC_PAIR) return a < rc2 && b < rc2 && c < rc2;
    double t;
    if (a > b) { t = a; a = b; b = t; }
    if (b > c) { t = b; b = c; c = t; }
    if (a > b) { t = a; a = b; b = t; }
    return (a * b) * c < rc6;
}

int orc_atm_brute(const double* prm, int64_t n, const double* x, int trunc, int member,
                  double* f, double* ew, uint64_t* cnt)
{
    if (trunc < 0 || trunc > 1 || member < -1 || member > 4) return 1;
    cells_t c;
    int st = cells_make(prm, n, x, &c);
    if (st) return st;
    const grid_t* g = &c.g;
    double rc2 = g->rc * g->rc, rc6 = rc2 * rc2 * rc2;
    double wmin = g->w[0];
    for (int d = 1; d < 3; d++) wmin = g->w[d] < wmin ? g->w[d] : wmin;
    const double rw2 = (2.0 * wmin) * (2.0 * wmin);  /* 3cw: every side shorter than R_w */
    double e = 0.0, w = 0.0;
    uint64_t nint = 0;
    double* F = calloc((size_t)(3 * (n > 0 ? n : 1)), sizeof(double));
    for (int64_t i = 0; i < n; i++)
        for (int64_t j = 0; j < n; j++)
            for (int64_t k = j + 1; k < n; k++) {
                if (j == i || k == i) continue;
                int owner = member == ORC_3C01;
                if (!owner && !(i < j)) continue;  /* unordered i<j<k */
                if (member == ORC_3C01) {
                    int o[3];
                    if (!cell_offset(g, c.cell[i], c.cell[j], o)) continue;
                    if (!cell_offset(g, c.cell[i], c.cell[k], o)) continue;
                } else if (member == ORC_3C18) {
                    if (!member_3c18(g, c.cell[i], c.cell[j], c.cell[k])) continue;
                } else if (member == ORC_3C08) {
                    if (!member_3c08(g, c.cell[i], c.cell[j], c.cell[k])) continue;
                } else if (member == ORC_3C08A) {
                    if (!member_3c08a(g, c.cell[i], c.cell[j], c.cell[k])) continue;
                }
                double dij[3], dik[3], djk[3];
                double a = bf_dsq(c.xw, n, g->L, i, j, dij);
                double b = bf_dsq(c.xw, n, g->L, i, k, dik);
                double cc = bf_dsq(c.xw, n, g->L, j, k, djk);
                if (!bf_keep(rc2, rc6, trunc, a, b, cc)) continue;
                if (member == ORC_3CW && !(a < rw2 && b < rw2 && cc < rw2)) continue;
                nint++;
                double du[3];
                orc_atm_du_dsq(a, b, cc, g->nu, du);
                double u = orc_atm_u(a, b, cc, g->nu);
                double W = 0.0;
                for (int d = 0; d < 3; d++) {
                    double gij = 2.0 * du[0] * dij[d];
                    double gik = 2.0 * du[1] * dik[d];
                    double gjk = 2.0 * du[2] * djk[d];
                    F[d * n + i] += gij + gik;
                    if (!owner) {
                        F[d * n + j] += -gij + gjk;
                        F[d * n + k] += -gik - gjk;
                    }
                    W += -(dij[d] * gij + dik[d] * gik + djk[d] * gjk);
                }
                e += owner ? u / 3.0 : u;
                w += owner ? W / 3.0 : W;
            }
    if (f) memcpy(f, F, sizeof(double) * 3 * n);
    if (ew) {
        ew[0] = e;
        ew[1] = w;
    }
    if (cnt) cnt[0] = nint;
    free(F);
    cells_free(&c);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Lennard-Jones pairs (section 5): u = 4 eps [(sig/r)^12 - (sig/r)^6]      */
/* ------------------------------------------------------------------------ */

/* energy and the scalar fw = -(du/dr)/r (so F_i = fw * r_ij) of one pair */
static double lj_pair(const grid_t* g, double a, double* fw)
{
    double s = g->sig * g->sig / a;
    double s3 = s * s * s, s6 = s3 * s3;
    double u = 4.0 * g->eps * (s6 - s3);
    if (g->shift) {
        double sc = g->sig * g->sig / (g->rc * g->rc);
        double sc3 = sc * sc * sc;
        u -= 4.0 * g->eps * (sc3 * sc3 - sc3);
    }
    *fw = (48.0 * g->eps * s6 - 24.0 * g->eps * s3) / a;
    return u;
}

int orc_lj_brute(const double* prm, int64_t n, const double* x, double* f, double* ew,
                 uint64_t* cnt)
{
    cells_t c;
    int st = cells_make(prm, n, x, &c);
    if (st) return st;
    const grid_t* g = &c.g;
    double rc2 = g->rc * g->rc, e = 0.0, w = 0.0;
    uint64_t nint = 0;
    double* F = calloc((size_t)(3 * (n > 0 ? n : 1)), sizeof(double));
    for (int64_t i = 0; i < n; i++)
        for (int64_t j = i + 1; j < n; j++) {
            double d[3];
            double a = bf_dsq(c.xw, n, g->L, i, j, d);
            if (!(a < rc2)) continue;
            nint++;
            double fw;
            e += lj_pair(g, a, &fw);
            w += fw * a;
            for (int k = 0; k < 3; k++) {
                F[k * n + i] -= fw * d[k];
                F[k * n + j] += fw * d[k];
            }
        }
    if (f) memcpy(f, F, sizeof(double) * 3 * n);
    if (ew) {
        ew[0] = e;
        ew[1] = w;
    }
    if (cnt) cnt[0] = nint;
    free(F);
    cells_free(&c);
    return 0;
}

int orc_lj_cells(const double* prm, int64_t n, const double* x, int prec,
                 double* f, double* ew, uint64_t* cnt)
{
    if (prec < 0 || prec > 1) return 1;
    cells_t c;
    int st = cells_make(prm, n, x, &c);
    if (st) return st;
    ev_t ev;
    double* fs = calloc((size_t)(3 * (n > 0 ? n : 1)), sizeof(double));
    ev_init(&ev, &c, ORC_PAIR, prec, fs);
    const grid_t* g = &c.g;
    int fw13[13][3];
    forward13(fw13);
    for (int64_t b = 0; b < g->ncell; b++) {
        int64_t b0 = c.start[b], b1 = c.start[b + 1];
        for (int q = -1; q < 13; q++) {
            const int* o = q < 0 ? ZERO3 : fw13[q];
            int64_t nc = q < 0 ? b : nb_cell(g, b, o);
            for (int64_t i = b0; i < b1; i++)
                for (int64_t j = (q < 0 ? i + 1 : c.start[nc]); j < c.start[nc + 1]; j++) {
                    ev.ncand++;
                    if (!side_ok(&ev, i, ZERO3, j, o)) continue;
                    double d[3];
                    double a = dsq64(&ev, i, ZERO3, j, o, d);
                    if (prec == ORC_FP64 && !(a < ev.rc2)) continue;
                    ev.nint++;
                    double fwv;
                    ev.e += lj_pair(g, a, &fwv);
                    ev.w += fwv * a;
                    for (int k = 0; k < 3; k++) {
                        fs[k * n + i] -= fwv * d[k];
                        fs[k * n + j] += fwv * d[k];
                    }
                }
        }
    }
    if (f)
        for (int64_t s = 0; s < n; s++)
            for (int d = 0; d < 3; d++) f[d * n + c.perm[s]] = fs[d * n + s];
    if (ew) {
        ew[0] = ev.e;
        ew[1] = ev.w;
    }
    if (cnt) {
        cnt[0] = ev.ncand;
        cnt[1] = ev.nint;
    }
    free(fs);
    cells_free(&c);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Observables of the validation runs (section 5)                           */
/* ------------------------------------------------------------------------ */

/* pair-distance histogram behind the radial distribution functions of the
 * single-phase runs (section 5.1, Fig. rdfs): every pair once (own cell and
 * the 13 forward neighbour cells), r = sqrt of the FP64 canonical squared
 * distance, bin floor(r / (r_max / nbins)) for r < r_max; r_max must not
 * exceed the smallest cell edge, so the cell loop misses no pair            */
int orc_rdf(const double* prm, int64_t n, const double* x, double rmax, int nbins,
            uint64_t* counts)
{
    if (nbins < 1 || !(rmax > 0.0) || !isfinite(rmax) || !counts) return 1;
    cells_t c;
    int st = cells_make(prm, n, x, &c);
    if (st) return st;
    const grid_t* g = &c.g;
    for (int d = 0; d < 3; d++)
        if (rmax > g->w[d]) {
            cells_free(&c);
            return 1;
        }
    ev_t ev;
    ev_init(&ev, &c, ORC_PAIR, ORC_FP64, NULL);
    const double dr = rmax / (double)nbins, rmax2 = rmax * rmax;
    int fw13[13][3];
    forward13(fw13);
    for (int b = 0; b < nbins; b++) counts[b] = 0;
    for (int64_t b = 0; b < g->ncell; b++) {
        int64_t b0 = c.start[b], b1 = c.start[b + 1];
        for (int q = -1; q < 13; q++) {
            const int* o = q < 0 ? ZERO3 : fw13[q];
            int64_t nc = q < 0 ? b : nb_cell(g, b, o);
            for (int64_t i = b0; i < b1; i++)
                for (int64_t j = (q < 0 ? i + 1 : c.start[nc]); j < c.start[nc + 1]; j++) {
                    double d[3];
                    double a = dsq64(&ev, i, ZERO3, j, o, d);
                    if (!(a < rmax2)) continue;
                    int k = (int)(sqrt(a) / dr);
                    if (k > nbins - 1) k = nbins - 1;
                    counts[k]++;
                }
        }
    }
    cells_free(&c);
    return 0;
}

/* velocity rescaling for the NVT runs of section 5.1 (no thermostat is
 * named; reading: the kinetic temperature T = 2K / (3n - 3) is set to the
 * target by scaling every velocity by one factor): v *= sqrt(T0 / T) */
int orc_rescale(int64_t n, double* v, double t0)
{
    if (n < 0 || !v || !(t0 >= 0.0)) return 1;
    if (n < 2) return 0;
    double k = 0.0;
    for (int64_t i = 0; i < n; i++)
        for (int d = 0; d < 3; d++) k += 0.5 * v[d * n + i] * v[d * n + i];
    if (!(k > 0.0)) return 0;
    double t = 2.0 * k / (3.0 * (double)n - 3.0);
    double lam = sqrt(t0 / t);
    for (int64_t i = 0; i < 3 * n; i++) v[i] *= lam;
    return 0;
}

/* LJ 12-6 pair energy and its derivative du/dr at distance r */
static void lj_u_du(double r, double eps, double sig, double* u, double* du)
{
    double s6 = pow(sig / r, 6.0), s12 = s6 * s6;
    *u = 4.0 * eps * (s12 - s6);
    *du = 4.0 * eps * (-12.0 * s12 + 6.0 * s6) / r;
}

/* long-range corrections of the truncated LJ pair terms of a homogeneous
 * fluid (section 5.1 applies them to E2 and P2; g(r) = 1 beyond r_c):
 *   E_tail = 2 pi N rho  int_{r_c}^inf r^2 u(r) dr
 *   P_tail = -2/3 pi rho^2 int_{r_c}^inf r^3 u'(r) dr,   rho = N / V,
 * both integrals taken numerically (composite Simpson, `intervals` even) in
 * s = r_c / r on (0, 1], where dr = r_c / s^2 ds and both integrands vanish
 * at s = 0                                                                  */
int orc_lj_tail(const double* prm, int64_t n, int intervals, double* out)
{
    if (n < 0 || intervals < 2 || (intervals & 1) || !out) return 1;
    const double V = prm[0] * prm[1] * prm[2], rc = prm[3], eps = prm[5], sig = prm[6];
    if (!(V > 0.0) || !(rc > 0.0) || !(sig > 0.0)) return 1;
    const double pi = 3.14159265358979323846, rho = (double)n / V;
    double ie = 0.0, ip = 0.0;
    for (int k = 0; k <= intervals; k++) {
        double s = (double)k / intervals, fe = 0.0, fp = 0.0;
        if (k > 0) {
            double r = rc / s, u, du, jac = rc / (s * s);
            lj_u_du(r, eps, sig, &u, &du);
            fe = r * r * u * jac;
            fp = r * r * r * du * jac;
        }
        double wgt = (k == 0 || k == intervals) ? 1.0 : ((k & 1) ? 4.0 : 2.0);
        ie += wgt * fe;
        ip += wgt * fp;
    }
    ie *= 1.0 / (3.0 * intervals);
    ip *= 1.0 / (3.0 * intervals);
    out[0] = 2.0 * pi * (double)n * rho * ie;
    out[1] = -2.0 / 3.0 * pi * rho * rho * ip;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Velocity-Verlet NVE (unit mass; the paper's integrator is not named)     */
/* ------------------------------------------------------------------------ */

static int total_force(const double* prm, int64_t n, const double* x, int trav, int trunc,
                       int prec, double* f, double* rec)
{
    double* f3 = malloc(sizeof(double) * 3 * (n > 0 ? n : 1));
    double ew2[2], ew3[2];
    uint64_t c2[2], c3[2];
    int st = orc_lj_cells(prm, n, x, prec, f, ew2, c2);
    if (!st) st = orc_atm_cells(prm, n, x, trav, trunc, prec, 0, -1, f3, ew3, c3);
    if (!st)
        for (int64_t q = 0; q < 3 * n; q++) f[q] += f3[q];
    free(f3);
    rec[0] = ew2[0];
    rec[1] = ew3[0];
    rec[3] = ew2[1] + ew3[1];
    return st;
}

int orc_md_run(const double* prm, int64_t n, double* x, double* v, int nsteps, double dt,
               int trav, int trunc, int prec, double* f, double* energies)
{
    if (nsteps < 0) return 1;
    for (int64_t i = 0; i < n; i++)
        for (int d = 0; d < 3; d++) x[d * n + i] = wrap1(x[d * n + i], prm[d]);
    int st = total_force(prm, n, x, trav, trunc, prec, f, energies);
    if (st) return st;
    for (int s = 0; s <= nsteps; s++) {
        if (s > 0) {
            for (int64_t q = 0; q < 3 * n; q++) v[q] += 0.5 * dt * f[q];
            for (int64_t i = 0; i < n; i++)
                for (int d = 0; d < 3; d++)
                    x[d * n + i] = wrap1(x[d * n + i] + dt * v[d * n + i], prm[d]);
            st = total_force(prm, n, x, trav, trunc, prec, f, energies + 4 * s);
            if (st) return st;
            for (int64_t q = 0; q < 3 * n; q++) v[q] += 0.5 * dt * f[q];
        }
        double k = 0.0;
        for (int64_t q = 0; q < 3 * n; q++) k += 0.5 * v[q] * v[q];
        energies[4 * s + 2] = k;
    }
    return 0;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
