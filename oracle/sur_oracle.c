/*
 * sur_oracle.c -- plain FP64 oracle of the learned three-body force surrogate.
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * benchmark's CPU legs, never by the library.
 *
 * The paper computes the ATM forces exactly (Section 2); the surrogate is a
 * cheaper per-molecule model of the same force, defined here:
 *
 *   neighbours j of i: minimum-image distance r = |r_j - r_i| < r_c,
 *   rhat = (r_j - r_i) / r, smooth cutoff f_c(r) = (cos(pi r / r_c) + 1) / 2;
 *   radial channels   G_k   = sum_j exp(-eta_g (r - mu_k)^2) f_c(r),  k < 16,
 *                     mu_k  = 0.8 + k (r_c - 0.8) / 15,  eta_g = 1 / (2 dk^2),
 *                     dk    = (r_c - 0.8) / 15;
 *   vector channels   phi_a = exp(-eta_v (r - nu_a)^2) f_c(r),  a < 4,
 *                     nu_a  = 0.8 + (a + 1/2) (r_c - 0.8) / 4,  eta_v = 1 / (2 da^2),
 *                     da    = (r_c - 0.8) / 4;
 *                     p_a   = sum_j phi_a rhat,
 *                     T_a   = sum_j phi_a (rhat rhat^T - I / 3)   (a < 3);
 *   descriptors D = [G_0..G_15,
 *                    p_a . p_b for (a, b) = 00 01 02 03 11 12 13 22 23 33,
 *                    tr(T_a T_b) for (a, b) = 00 01 02 11 12 22];
 *   equivariant vectors (16): v_m = p_m (m < 4) and v_{4 + 4a + b} = T_a p_b
 *                     (a < 3, b < 4), the quadrupole channels applied to the
 *                     vector channels (they carry the angular correlation of
 *                     two neighbours that a triplet force depends on);
 *   MLP: xn = (D - mean) / scale, h1 = silu(xn W1 + b1), h2 = silu(h1 W2 + b2),
 *        w = h2 W3 + b3 (16 outputs), silu(z) = z / (1 + exp(-z));
 *   force F_i = sum_m w_m v_m.
 *
 * Everything is FP64 and written for reading, not speed.
 */
#include "sur_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define SUR_R0 0.8
#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* offsets of the parameter blocks */
#define OFF_W1 0
#define OFF_B1 (OFF_W1 + SUR_ND * SUR_NH)
#define OFF_W2 (OFF_B1 + SUR_NH)
#define OFF_B2 (OFF_W2 + SUR_NH * SUR_NH)
#define OFF_W3 (OFF_B2 + SUR_NH)
#define OFF_B3 (OFF_W3 + SUR_NH * SUR_NO)

void orc_sur_basis(double rc, double* mu_g, double* eta_g, double* mu_v, double* eta_v)
{
    double dk = (rc - SUR_R0) / 15.0, da = (rc - SUR_R0) / 4.0;
    for (int k = 0; k < 16; k++) mu_g[k] = SUR_R0 + k * dk;
    *eta_g = 1.0 / (2.0 * dk * dk);
    for (int a = 0; a < 4; a++) mu_v[a] = SUR_R0 + (a + 0.5) * da;
    *eta_v = 1.0 / (2.0 * da * da);
}

double orc_sur_fcut(double r, double rc)
{
    return r < rc ? 0.5 * (cos(M_PI * r / rc) + 1.0) : 0.0;
}

static double wrap(double x, double L)
{
    double y = x - floor(x / L) * L;
    return y >= L ? 0.0 : y;
}

int orc_sur_descriptors(const double* prm, const double* x, int64_t n, const int64_t* rows,
                        int64_t nrows, double* D, double* V)
{
    const double* L = prm;
    const double rc = prm[3];
    if (!(rc > SUR_R0) || L[0] < 2 * rc || L[1] < 2 * rc || L[2] < 2 * rc) return -1;
    double mu_g[16], eta_g, mu_v[4], eta_v;
    orc_sur_basis(rc, mu_g, &eta_g, mu_v, &eta_v);
    static const int PA[10] = {0, 0, 0, 0, 1, 1, 1, 2, 2, 3};
    static const int PB[10] = {0, 1, 2, 3, 1, 2, 3, 2, 3, 3};
    static const int TA[6] = {0, 0, 0, 1, 1, 2};
    static const int TB[6] = {0, 1, 2, 1, 2, 2};
    for (int64_t q = 0; q < nrows; q++) {
        int64_t i = rows[q];
        double G[16] = {0}, p[4][3] = {{0}}, T[3][3][3] = {{{0}}};
        for (int64_t j = 0; j < n; j++) {
            if (j == i) continue;
            double d[3];
            for (int k = 0; k < 3; k++) {
                double t = wrap(x[k * n + j], L[k]) - wrap(x[k * n + i], L[k]);
                d[k] = t - rint(t / L[k]) * L[k];
            }
            double r2 = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
            if (!(r2 < rc * rc)) continue;
            double r = sqrt(r2);
            double u[3] = {d[0] / r, d[1] / r, d[2] / r};
            double fc = orc_sur_fcut(r, rc);
            for (int k = 0; k < 16; k++) G[k] += exp(-eta_g * (r - mu_g[k]) * (r - mu_g[k])) * fc;
            for (int a = 0; a < 4; a++) {
                double phi = exp(-eta_v * (r - mu_v[a]) * (r - mu_v[a])) * fc;
                for (int k = 0; k < 3; k++) p[a][k] += phi * u[k];
                if (a < 3)
                    for (int s = 0; s < 3; s++)
                        for (int t = 0; t < 3; t++)
                            T[a][s][t] += phi * (u[s] * u[t] - (s == t ? 1.0 / 3.0 : 0.0));
            }
        }
        double* Dq = D + q * SUR_ND;
        for (int k = 0; k < 16; k++) Dq[k] = G[k];
        for (int e = 0; e < 10; e++) {
            const double* pa = p[PA[e]];
            const double* pb = p[PB[e]];
            Dq[16 + e] = pa[0] * pb[0] + pa[1] * pb[1] + pa[2] * pb[2];
        }
        for (int e = 0; e < 6; e++) {
            double tr = 0.0;
            for (int s = 0; s < 3; s++)
                for (int t = 0; t < 3; t++) tr += T[TA[e]][s][t] * T[TB[e]][t][s];
            Dq[26 + e] = tr;
        }
        double* Vq = V + q * SUR_NV;
        for (int m = 0; m < 4; m++)
            for (int k = 0; k < 3; k++) Vq[3 * m + k] = p[m][k];
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 4; b++)
                for (int k = 0; k < 3; k++) {
                    double tp = 0.0;
                    for (int t = 0; t < 3; t++) tp += T[a][k][t] * p[b][t];
                    Vq[3 * (4 + 4 * a + b) + k] = tp;
                }
    }
    return 0;
}

double orc_bf16(double x)
{
    if (x == 0.0 || !isfinite(x)) return x;
    int e;
    frexp(x, &e);                        /* x = f 2^e, 0.5 <= |f| < 1 */
    double m = ldexp(x, 8 - e);          /* 8 significant bits left of the point */
    double rm = nearbyint(m);            /* ties to even in the default mode */
    return ldexp(rm, e - 8);
}

static double silu(double z) { return z / (1.0 + exp(-z)); }

/* d silu / dz = s (1 + z (1 - s)), s = 1 / (1 + exp(-z)) */
static double dsilu(double z)
{
    double s = 1.0 / (1.0 + exp(-z));
    return s * (1.0 + z * (1.0 - s));
}

/* forward pass of one row; keeps the pre-activations for the backward pass */
static void forward_row(const double* P, const double* mean, const double* scale,
                        const double* Drow, int bf16, double* xn, double* z1, double* h1,
                        double* z2, double* h2, double* w)
{
    for (int k = 0; k < SUR_ND; k++) {
        xn[k] = (Drow[k] - mean[k]) / scale[k];
        if (bf16) xn[k] = orc_bf16(xn[k]);
    }
    for (int j = 0; j < SUR_NH; j++) {
        double s = 0.0;
        for (int k = 0; k < SUR_ND; k++) {
            double wt = P[OFF_W1 + k * SUR_NH + j];
            s += xn[k] * (bf16 ? orc_bf16(wt) : wt);
        }
        z1[j] = s + P[OFF_B1 + j];
        h1[j] = silu(z1[j]);
        if (bf16) h1[j] = orc_bf16(h1[j]);
    }
    for (int j = 0; j < SUR_NH; j++) {
        double s = 0.0;
        for (int k = 0; k < SUR_NH; k++) {
            double wt = P[OFF_W2 + k * SUR_NH + j];
            s += h1[k] * (bf16 ? orc_bf16(wt) : wt);
        }
        z2[j] = s + P[OFF_B2 + j];
        h2[j] = silu(z2[j]);
        if (bf16) h2[j] = orc_bf16(h2[j]);
    }
    for (int m = 0; m < SUR_NO; m++) {
        double s = 0.0;
        for (int k = 0; k < SUR_NH; k++) {
            double wt = P[OFF_W3 + k * SUR_NO + m];
            s += h2[k] * (bf16 ? orc_bf16(wt) : wt);
        }
        w[m] = s + P[OFF_B3 + m];
    }
}

void orc_sur_mlp(const double* P, const double* mean, const double* scale, int64_t n,
                 const double* D, const double* V, int bf16, double* w, double* F)
{
    double xn[SUR_ND], z1[SUR_NH], h1[SUR_NH], z2[SUR_NH], h2[SUR_NH];
    for (int64_t i = 0; i < n; i++) {
        double* wi = w + SUR_NO * i;
        forward_row(P, mean, scale, D + i * SUR_ND, bf16, xn, z1, h1, z2, h2, wi);
        for (int c = 0; c < 3; c++) {
            double f = 0.0;
            for (int m = 0; m < SUR_NO; m++) f += wi[m] * V[i * SUR_NV + 3 * m + c];
            F[3 * i + c] = f;
        }
    }
}

void orc_sur_loss_grad(const double* P, const double* mean, const double* scale, int64_t n,
                       const double* D, const double* V, const double* Fref, double sigma2,
                       double* loss, double* grad)
{
    double xn[SUR_ND], z1[SUR_NH], h1[SUR_NH], z2[SUR_NH], h2[SUR_NH], w[SUR_NO];
    double dw[SUR_NO], dz2[SUR_NH], dz1[SUR_NH];
    memset(grad, 0, SUR_NP * sizeof(double));
    double L = 0.0;
    const double norm = 1.0 / (3.0 * (double)n * sigma2);
    for (int64_t i = 0; i < n; i++) {
        forward_row(P, mean, scale, D + i * SUR_ND, 0, xn, z1, h1, z2, h2, w);
        const double* Vi = V + i * SUR_NV;
        double r[3];
        for (int c = 0; c < 3; c++) {
            double f = 0.0;
            for (int m = 0; m < SUR_NO; m++) f += w[m] * Vi[3 * m + c];
            r[c] = f - Fref[3 * i + c];
            L += r[c] * r[c] * norm;
        }
        /* dL/dw_m = sum_c 2 r_c v_mc / (3 n sigma2) */
        for (int m = 0; m < SUR_NO; m++) {
            dw[m] = 0.0;
            for (int c = 0; c < 3; c++) dw[m] += 2.0 * norm * r[c] * Vi[3 * m + c];
        }
        /* output layer */
        for (int m = 0; m < SUR_NO; m++) {
            grad[OFF_B3 + m] += dw[m];
            for (int k = 0; k < SUR_NH; k++) grad[OFF_W3 + k * SUR_NO + m] += h2[k] * dw[m];
        }
        /* second hidden layer */
        for (int k = 0; k < SUR_NH; k++) {
            double dh = 0.0;
            for (int m = 0; m < SUR_NO; m++) dh += P[OFF_W3 + k * SUR_NO + m] * dw[m];
            dz2[k] = dh * dsilu(z2[k]);
        }
        for (int j = 0; j < SUR_NH; j++) {
            grad[OFF_B2 + j] += dz2[j];
            for (int k = 0; k < SUR_NH; k++) grad[OFF_W2 + k * SUR_NH + j] += h1[k] * dz2[j];
        }
        /* first hidden layer */
        for (int k = 0; k < SUR_NH; k++) {
            double dh = 0.0;
            for (int j = 0; j < SUR_NH; j++) dh += P[OFF_W2 + k * SUR_NH + j] * dz2[j];
            dz1[k] = dh * dsilu(z1[k]);
        }
        for (int j = 0; j < SUR_NH; j++) {
            grad[OFF_B1 + j] += dz1[j];
            for (int k = 0; k < SUR_ND; k++) grad[OFF_W1 + k * SUR_NH + j] += xn[k] * dz1[j];
        }
    }
    *loss = L;
}

void orc_sur_adam(double* P, double* m, double* v, const double* g, int64_t np, int64_t t,
                  double lr, double beta1, double beta2, double eps)
{
    double c1 = 1.0 - pow(beta1, (double)t), c2 = 1.0 - pow(beta2, (double)t);
    for (int64_t k = 0; k < np; k++) {
        m[k] = beta1 * m[k] + (1.0 - beta1) * g[k];
        v[k] = beta2 * v[k] + (1.0 - beta2) * g[k] * g[k];
        double mh = m[k] / c1, vh = v[k] / c2;
        P[k] -= lr * mh / (sqrt(vh) + eps);
    }
}

void orc_sur_stats(int64_t n, const double* D, const double* F, double* mean, double* scale,
                   double* sigma2)
{
    for (int k = 0; k < SUR_ND; k++) {
        double s = 0.0;
        for (int64_t i = 0; i < n; i++) s += D[i * SUR_ND + k];
        double mu = n > 0 ? s / (double)n : 0.0;
        double q = 0.0;
        for (int64_t i = 0; i < n; i++) q += (D[i * SUR_ND + k] - mu) * (D[i * SUR_ND + k] - mu);
        double sd = n > 0 ? sqrt(q / (double)n) : 0.0;
        mean[k] = mu;
        scale[k] = sd < 1e-12 ? 1.0 : sd;
    }
    double f2 = 0.0;
    for (int64_t i = 0; i < 3 * n; i++) f2 += F[i] * F[i];
    *sigma2 = n > 0 ? f2 / (3.0 * (double)n) : 0.0;
}
