/*
 * atm_oracle.h -- CPU oracle for the Axilrod-Teller-Muto (ATM) linked-cell
 * three-body method of "Linked Cell Traversal Algorithms for Three-Body
 * Interactions in Molecular Dynamics" (arXiv 2510.21230).
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, obviously-correct FP64
 * restatement of the method.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it.  It shares no code, header,
 * table or constant with the CUDA library and neither side includes the
 * other.
 *
 * Parameter vector `prm` (8 doubles) used by every entry point:
 *   prm[0..2] box edge lengths L_x, L_y, L_z (periodic, origin at 0)
 *   prm[3]    cutoff radius r_c (pairs and triplets)
 *   prm[4]    ATM strength nu
 *   prm[5]    Lennard-Jones epsilon
 *   prm[6]    Lennard-Jones sigma
 *   prm[7]    1.0 = shift the LJ energy to zero at r_c, 0.0 = plain truncation
 *
 * Arrays of 3-vectors are "SoA": x[0..n), then y[0..n), then z[0..n).
 * Return value: 0 on success, 1 invalid argument, 2 box smaller than three
 * cells along some axis.
 */
#ifndef ATM_ORACLE_H
#define ATM_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* traversal, truncation and precision selectors */
enum { ORC_3C01 = 0, ORC_3C18 = 1, ORC_3C08 = 2, ORC_3CW = 3, ORC_3C08A = 4 };
enum { ORC_PAIR = 0, ORC_PRODUCT = 1 };
enum { ORC_FP64 = 0, ORC_FP32 = 1 };
/* brute-force membership filters: all triples, or the triples a traversal visits */
enum { ORC_MEMBER_ALL = -1 };

/* ATM energy of one triplet from squared side lengths a=r_ij^2, b=r_ik^2, c=r_jk^2 (Eq. atm). */
double orc_atm_u(double a, double b, double c, double nu);
/* partial derivatives du/da, du/db, du/dc of the same expression. */
void orc_atm_du_dsq(double a, double b, double c, double nu, double out[3]);
/* du/dr_ij as printed in the paper's eleven-term gradient (Eq. ATMGradient). */
double orc_atm_dudr_paper(double rij, double rik, double rjk, double nu);

/* Linked-cell grid along each axis: n_d = largest k with L_d/k >= r_c, w_d = L_d/n_d. */
int orc_cell_grid(const double* prm, int32_t ncell[3], double w[3]);

/*
 * Build the linked cells (wrap, bin, stable counting sort).
 *   xw        [3n] wrapped positions, original order
 *   cell_of   [n]  cell id of each molecule, original order (z-major: (cz*ny+cy)*nx+cx)
 *   cell_start[ncell+1]
 *   perm      [n]  sorted slot -> original index (sorted by (cell, original index))
 *   xl        [3n] FP64 cell-local coordinates in sorted order
 *   xl32      [3n] FP32 cell-local coordinates in sorted order
 * Any output pointer may be NULL.
 */
int orc_build_cells(const double* prm, int64_t n, const double* x, double* xw,
                    int32_t* cell_of, int32_t* cell_start, int32_t* perm,
                    double* xl, float* xl32);

/*
 * Brute-force O(N^3) ATM over all i<j<k with the minimum-image convention.
 * member = ORC_MEMBER_ALL, or a traversal id: keep only the triplets that
 * traversal visits (3c01 keeps owner visits and adds u/3 per visit).
 * f[3n] ATM forces (original order), ew[2] = {E3, W3}, cnt[1] = interacting visits.
 */
int orc_atm_brute(const double* prm, int64_t n, const double* x, int trunc, int member,
                  double* f, double* ew, uint64_t* cnt);

/*
 * Linked-cell ATM with traversal trav in {3c01, 3c18, 3c08}, truncation trunc
 * and decision precision prec.  With prec = ORC_FP32 the truncation decision is
 * taken in FP32 on FP32 cell-local coordinates; energies and forces of the
 * kept triplets are still evaluated in FP64.  Units (base cells / block anchors)
 * [unit_lo, unit_hi) are processed (unit_hi < 0: all).
 * f[3n] ATM forces (original order), ew[2] = {E3, W3},
 * cnt[2] = {candidate triplets traversed, interacting triplets (3c01: visits)}.
 */
int orc_atm_cells(const double* prm, int64_t n, const double* x, int trav, int trunc,
                  int prec, int64_t unit_lo, int64_t unit_hi,
                  double* f, double* ew, uint64_t* cnt);

/* The same over an explicit list of units (each unit id in [0, ncell)). */
int orc_atm_cells_units(const double* prm, int64_t n, const double* x, int trav, int trunc,
                        int prec, const int64_t* units, int64_t nunits,
                        double* f, double* ew, uint64_t* cnt);

/* Brute-force LJ over all pairs (minimum image). ew = {E2, W2}, cnt[1] = pairs within r_c. */
int orc_lj_brute(const double* prm, int64_t n, const double* x, double* f, double* ew,
                 uint64_t* cnt);

/* Linked-cell LJ over the half shell (base cell + 13 forward neighbours).
 * cnt[2] = {candidate pairs, pairs within r_c}. */
int orc_lj_cells(const double* prm, int64_t n, const double* x, int prec,
                 double* f, double* ew, uint64_t* cnt);

/*
 * Velocity-Verlet NVE run with LJ + ATM forces (linked cells).
 * x[3n], v[3n] in/out (x returned wrapped), f[3n] out (total force at the end).
 * energies[4*nsteps+4]: per record {E2, E3, Ekin, W2+W3}; record 0 is the
 * start state, record s the state after step s.
 */
int orc_md_run(const double* prm, int64_t n, double* x, double* v, int nsteps, double dt,
               int trav, int trunc, int prec, double* f, double* energies);

/* Pair-distance histogram (every pair once, linked cells, FP64 canonical
 * distance): counts[nbins], bin floor(r / (r_max / nbins)), r < r_max,
 * r_max at most the smallest cell edge. */
int orc_rdf(const double* prm, int64_t n, const double* x, double rmax, int nbins,
            uint64_t* counts);

/* Velocity rescaling to kinetic temperature t0 (T = 2K / (3n - 3)), in place. */
int orc_rescale(int64_t n, double* v, double t0);

/* LJ long-range corrections of a homogeneous fluid by numerical quadrature:
 * out = {E_tail (total), P_tail}. */
int orc_lj_tail(const double* prm, int64_t n, int intervals, double* out);

/* number of OpenMP threads the oracle uses (1 without OpenMP) */
int orc_num_threads(void);

#ifdef __cplusplus
}
#endif
#endif
