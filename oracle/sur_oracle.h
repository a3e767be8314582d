/*
 * sur_oracle.h -- plain FP64 oracle of the learned three-body force surrogate.
 * TEST INFRASTRUCTURE ONLY (see sur_oracle.c).
 *
 * The surrogate is not part of the paper; it replaces the ATM triplet sum of
 * Section 2 (Eq. atm / Eq. forcepairs) by a per-molecule model:
 *   descriptors D_i (32 rotation invariants of the neighbourhood r < r_c),
 *   16 equivariant vectors v_m(i): the four vector channels
 *   p_a = sum_j phi_a(r_ij) rhat_ij and the twelve products T_a p_b of the
 *   three quadrupole channels with them,
 *   an MLP 32 -> 64 -> 64 -> 16 (SiLU) giving weights w_m(i),
 *   F_i = sum_m w_m(i) v_m(i).
 *
 * Parameter vector layout (SUR_NP doubles), all matrices row-major with the
 * input index first:  W1[32][64], b1[64], W2[64][64], b2[64], W3[64][16], b3[16].
 */
#ifndef SUR_ORACLE_H
#define SUR_ORACLE_H

#include <stdint.h>

#define SUR_ND 32
#define SUR_NH 64
#define SUR_NO 16
#define SUR_NV 48
#define SUR_NP (SUR_ND * SUR_NH + SUR_NH + SUR_NH * SUR_NH + SUR_NH + SUR_NH * SUR_NO + SUR_NO)

#ifdef __cplusplus
extern "C" {
#endif

/* radial centres / widths of the descriptor basis for cutoff rc:
 * mu_g[16], eta_g (Gaussian radial channels), mu_v[4], eta_v (vector channels) */
void orc_sur_basis(double rc, double* mu_g, double* eta_g, double* mu_v, double* eta_v);

/* smooth cutoff 0.5 (cos(pi r / rc) + 1) for r < rc, else 0 */
double orc_sur_fcut(double r, double rc);

/* descriptors D[nrows][32] and vectors V[nrows][48] of the molecules rows[],
 * by brute force over all other molecules (minimum image); prm as the ATM
 * oracle: [Lx, Ly, Lz, rc, ...]; x SoA [3][n].  Returns 0, or -1 if rc <= 0.8
 * or a box side is below 2 rc. */
int orc_sur_descriptors(const double* prm, const double* x, int64_t n, const int64_t* rows,
                        int64_t nrows, double* D, double* V);

/* round to the nearest bfloat16 value (8 significant bits, ties to even) */
double orc_bf16(double x);

/* MLP forward for n rows: normalised input xn = (D - mean) / scale, outputs
 * w[n][16] and F[n][3] = sum_m w_m v_m.  bf16 != 0 rounds xn, the three weight
 * matrices and the two hidden activations to bfloat16 (biases and sums stay
 * FP64). */
void orc_sur_mlp(const double* P, const double* mean, const double* scale, int64_t n,
                 const double* D, const double* V, int bf16, double* w, double* F);

/* loss L = sum_i |F_i - Fref_i|^2 / (3 n sigma2) and its gradient dL/dP */
void orc_sur_loss_grad(const double* P, const double* mean, const double* scale, int64_t n,
                       const double* D, const double* V, const double* Fref, double sigma2,
                       double* loss, double* grad);

/* one Adam step (Kingma & Ba, Algorithm 1) with step number t >= 1, in place */
void orc_sur_adam(double* P, double* m, double* v, const double* g, int64_t np, int64_t t,
                  double lr, double beta1, double beta2, double eps);

/* per-column mean and population standard deviation of D[n][32] (a column
 * whose deviation is below 1e-12 gets scale 1), and the mean squared force
 * component sigma2 = sum |F|^2 / (3 n) */
void orc_sur_stats(int64_t n, const double* D, const double* F, double* mean, double* scale,
                   double* sigma2);

#ifdef __cplusplus
}
#endif
#endif
