/*
 * mlp_oracle.c -- FP64 reference of the learned ionization-rate surrogate.
 * TEST INFRASTRUCTURE ONLY (see md_oracle.c).
 *
 * The surrogate is not from the paper: it stands in for the per-ion rate
 * evaluation of Sec. II (nu_total = nu_ofi + nu_ci).  Definition:
 *   features  f = ((log10(F / F0) + 1.4) / 1.5,  z / 8,
 *                  (log10 max(n_e, 1e15) - 19.5) / 4.5,
 *                  (log10(max(T_e, 0.1) / Ip) + 0.2) / 3)
 *             with F = max(|E|, 1e-6) in atomic units of field, Ip the
 *             ionization energy of charge state z and F0 = (2 Ip / E_h)^(3/2)
 *             (the field scale of the tunnel exponent), so that the field and
 *             temperature enter relative to the scales of the rate of the
 *             charge state at hand;
 *   network   h1 = silu(W1 f + b1)    (64)
 *             h2 = silu(W2 h1 + b2)   (64)
 *             y  = W3 h2 + b3          (8)
 *   output    y_k approximates (log10(nu_k + 1e-12) + 6) / 6 for the
 *             transition k -> k+1; the ion of charge z uses y_z and
 *             nu = max(10^(6 y - 6) - 1e-12, 0).  The 1e-12 per unit time
 *             floor (P < 1e-13 per pass: such rates never ionize) keeps the
 *             fitted range to 13 decades, and adding it rather than clipping
 *             keeps the target smooth.
 *   loss      mean over samples of (y_{z_s} - target_s)^2.
 * Parameters, one flat array: W1[64][4], b1[64], W2[64][64], b2[64],
 * W3[8][64], b3[8] (5000 values, rows = outputs).
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

#define NI 4
#define NH 64
#define NO 8
#define OFF_W1 0
#define OFF_B1 (OFF_W1 + NH * NI)
#define OFF_W2 (OFF_B1 + NH)
#define OFF_B2 (OFF_W2 + NH * NH)
#define OFF_W3 (OFF_B2 + NH)
#define OFF_B3 (OFF_W3 + NO * NH)
#define NPARAM (OFF_B3 + NO)

int mo_nparam(void) { return NPARAM; }

/* |E| in the paper's unit a = eE/(m_e omega c) -> atomic units of field:
 * E = a m_e c omega / e = a (m_e c^2 / e) k, divided by the atomic field. */
#define MO_ME_C2_EV 510998.95          /* electron rest energy, eV */
#define MO_HARTREE_EV 27.211386245988  /* Hartree energy, eV */
#define MO_FIELD_AU 5.14220674763e11   /* atomic unit of field, V/m */
#define MO_PI 3.14159265358979323846

void mo_features(double e_mag, int z, double ne, double te, double ip_ev, double lambda_um,
                 double f[4])
{
    double k = 2.0 * MO_PI / (lambda_um * 1e-6);
    double F = fmax(e_mag, 1e-6) * MO_ME_C2_EV * k / MO_FIELD_AU;
    double F0 = pow(2.0 * ip_ev / MO_HARTREE_EV, 1.5);
    f[0] = (log10(F / F0) + 1.4) / 1.5;
    f[1] = z / 8.0;
    f[2] = (log10(fmax(ne, 1e15)) - 19.5) / 4.5;
    f[3] = (log10(fmax(te, 0.1) / ip_ev) + 0.2) / 3.0;
}

double mo_target(double nu) { return (log10(fmax(nu, 0.0) + 1e-12) + 6.0) / 6.0; }

double mo_rate_from_output(double y) { return fmax(pow(10.0, 6.0 * y - 6.0) - 1e-12, 0.0); }

static double silu(double a) { return a / (1.0 + exp(-a)); }

/* d silu / da = s (1 + a (1 - s)), s = sigmoid(a) */
static double dsilu(double a)
{
    double s = 1.0 / (1.0 + exp(-a));
    return s * (1.0 + a * (1.0 - s));
}

/* Forward pass of n samples f[n][4] -> y[n][8]. */
void mo_forward(const double *p, int n, const double *f, double *y)
{
    for (int s = 0; s < n; ++s) {
        double h1[NH], h2[NH];
        for (int j = 0; j < NH; ++j) {
            double a = p[OFF_B1 + j];
            for (int k = 0; k < NI; ++k) a += p[OFF_W1 + j * NI + k] * f[s * NI + k];
            h1[j] = silu(a);
        }
        for (int j = 0; j < NH; ++j) {
            double a = p[OFF_B2 + j];
            for (int k = 0; k < NH; ++k) a += p[OFF_W2 + j * NH + k] * h1[k];
            h2[j] = silu(a);
        }
        for (int j = 0; j < NO; ++j) {
            double a = p[OFF_B3 + j];
            for (int k = 0; k < NH; ++k) a += p[OFF_W3 + j * NH + k] * h2[k];
            y[s * NO + j] = a;
        }
    }
}

/* Loss (mean squared error of the selected outputs) and its gradient with
 * respect to every parameter, by reverse-mode differentiation of the forward
 * pass (chain rule written out layer by layer).  grad has NPARAM entries. */
double mo_loss_grad(const double *p, int n, const double *f, const int32_t *z,
                    const double *target, double *grad)
{
    memset(grad, 0, sizeof(double) * NPARAM);
    double loss = 0.0;
    for (int s = 0; s < n; ++s) {
        double a1[NH], h1[NH], a2[NH], h2[NH], y[NO];
        const double *x = f + s * NI;
        for (int j = 0; j < NH; ++j) {
            double a = p[OFF_B1 + j];
            for (int k = 0; k < NI; ++k) a += p[OFF_W1 + j * NI + k] * x[k];
            a1[j] = a;
            h1[j] = silu(a);
        }
        for (int j = 0; j < NH; ++j) {
            double a = p[OFF_B2 + j];
            for (int k = 0; k < NH; ++k) a += p[OFF_W2 + j * NH + k] * h1[k];
            a2[j] = a;
            h2[j] = silu(a);
        }
        for (int j = 0; j < NO; ++j) {
            double a = p[OFF_B3 + j];
            for (int k = 0; k < NH; ++k) a += p[OFF_W3 + j * NH + k] * h2[k];
            y[j] = a;
        }
        int zs = z[s];
        double r = y[zs] - target[s];
        loss += r * r;
        double dy[NO] = {0};
        dy[zs] = 2.0 * r / n;
        double dh2[NH] = {0};
        for (int j = 0; j < NO; ++j) {
            if (dy[j] == 0.0) continue;
            grad[OFF_B3 + j] += dy[j];
            for (int k = 0; k < NH; ++k) {
                grad[OFF_W3 + j * NH + k] += dy[j] * h2[k];
                dh2[k] += dy[j] * p[OFF_W3 + j * NH + k];
            }
        }
        double da2[NH], dh1[NH] = {0};
        for (int j = 0; j < NH; ++j) da2[j] = dh2[j] * dsilu(a2[j]);
        for (int j = 0; j < NH; ++j) {
            grad[OFF_B2 + j] += da2[j];
            for (int k = 0; k < NH; ++k) {
                grad[OFF_W2 + j * NH + k] += da2[j] * h1[k];
                dh1[k] += da2[j] * p[OFF_W2 + j * NH + k];
            }
        }
        for (int j = 0; j < NH; ++j) {
            double da1 = dh1[j] * dsilu(a1[j]);
            grad[OFF_B1 + j] += da1;
            for (int k = 0; k < NI; ++k) grad[OFF_W1 + j * NI + k] += da1 * x[k];
        }
    }
    return loss / n;
}
