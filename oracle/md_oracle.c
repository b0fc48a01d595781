/*
 * md_oracle.c -- plain, slow, FP64 CPU oracle of the laser-cluster MD hot path
 * (Holkundkar, "Parallel Implementation of 3D Molecular Dynamic Simulation for
 * Laser-Cluster Interaction", arXiv:1307.3711, Sec. II).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library calls, links or
 * includes this file; only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark load it.  It shares no source with the CUDA path.
 *
 * Everything is in the paper's dimensionless units (Sec. II): time in 1/omega,
 * length in 1/k, velocity in c, u = gamma*beta, field a = eE/(m_e omega c),
 * b = eB/(m_e omega), charge in e, mass in m_e, energy in m_e c^2.
 *
 * Readings of points on which the paper is silent (each one is listed with its
 * reason in the design notes of the repository):
 *  - Coulomb constant: the field of charge Q at distance r is K_C Q / r^2 with
 *    K_C = r_e k = 2 pi r_e / lambda (follows from the definition of a and of
 *    the length unit 1/k in Sec. II).
 *  - Softening: Plummer form, force ~ d / (r^2 + eps^2)^{3/2}, potential
 *    ~ 1 / sqrt(r^2 + eps^2); the self term is excluded.
 *  - Step order: field E^n at x^n, laser at t_n = t0 + n dt, relativistic Boris
 *    kick u^{n-1/2} -> u^{n+1/2}, drift x^{n+1} = x^n + dt u^{n+1/2}/gamma.
 *    The first step starts from u^{-1/2} = u^0 (no back-kick).
 *  - Envelope of Eq. 3: the printed formula mixes I and a0; the constant 2.77 is
 *    4 ln 2, the intensity-FWHM constant, so the field envelope is
 *    exp[-2 ln2 (t - 2 tau)^2 / tau^2] (intensity FWHM = tau, peak at 2 tau).
 *  - Linear polarisation: no phase makes a sine vanish, so the E_y and B_x
 *    amplitudes are set to zero (Eqs. 5 and 7); circular uses phi_E = 3pi/2,
 *    phi_B = pi/2 with both amplitudes a0.
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846
#define OR_ME_C2_EV 510998.95  /* electron rest energy, eV */
/* classical electron radius in metres (CODATA 2018) */
#define OR_R_E 2.8179403262e-15

/* ------------------------------------------------------------------ units */

/* K_C = r_e k = 2 pi r_e / lambda; Sec. II defines a = eE/(m_e omega c) and
 * length in units of 1/k, so a Coulomb field eQ/(4 pi eps0 r^2) becomes
 * K_C Q / r'^2 with r' = k r. */
double or_coulomb_constant(double lambda_um)
{
    return 2.0 * OR_PI * OR_R_E / (lambda_um * 1.0e-6);
}

/* Eq. 2: a0 = sqrt(I0 lambda^2 / 1.366e18), I0 in W/cm^2, lambda in micron. */
double or_a0_from_intensity(double intensity_wcm2, double lambda_um)
{
    return sqrt(intensity_wcm2 * lambda_um * lambda_um / 1.366e18);
}

/* Eq. 1: N_atoms = (R0 / R_W)^3. */
double or_n_atoms(double r0, double r_w)
{
    double q = r0 / r_w;
    return q * q * q;
}

/* --------------------------------------------------------------- laser */

enum { OR_ENV_GAUSS = 0, OR_ENV_SIN2 = 1, OR_ENV_LITERAL_EQ3 = 2, OR_ENV_FLAT = 3 };

/* Temporal envelope of the field amplitude (Eq. 3 and its readings).
 *  GAUSS:       exp[-2 ln2 (t - 2 tau)^2 / tau^2]  (intensity FWHM = tau)
 *  SIN2:        sin^2(pi t / T) on [0, T], 0 outside (tau holds T)
 *  LITERAL_EQ3: exp[-2.77 (t - 2 tau)^2 / tau^2] applied to the field
 *  FLAT:        1 (continuous wave; used by tests) */
double or_envelope(double t, int kind, double tau)
{
    switch (kind) {
    case OR_ENV_GAUSS: {
        double s = (t - 2.0 * tau) / tau;
        return exp(-2.0 * log(2.0) * s * s);
    }
    case OR_ENV_SIN2: {
        if (t < 0.0 || t > tau) return 0.0;
        double s = sin(OR_PI * t / tau);
        return s * s;
    }
    case OR_ENV_LITERAL_EQ3: {
        double s = (t - 2.0 * tau) / tau;
        return exp(-2.77 * s * s);
    }
    default:
        return 1.0;
    }
}

/* Eqs. 4-9 in the dipole approximation (Sec. II: only the temporal variation
 * of the field is kept).  pol = 0 linear, 1 circular; b0 = a0. */
void or_laser_fields(double t, double a0, int pol, int env, double tau,
                     double a[3], double b[3])
{
    double amp = a0 * or_envelope(t, env, tau);
    double c = pol ? 1.0 : 0.0;
    double phi_e = 1.5 * OR_PI, phi_b = 0.5 * OR_PI;
    a[0] = amp * sin(t);
    a[1] = c * amp * sin(t + phi_e);
    a[2] = 0.0;
    b[0] = c * amp * sin(t + phi_b);
    b[1] = amp * sin(t);
    b[2] = 0.0;
}

/* ------------------------------------------------------ Coulomb direct sum */

/* Field (and optionally potential) at nt targets from ns sources:
 *   E_i   = K_C sum_{j != i} Q_j (x_i - x_j) / (|x_i - x_j|^2 + eps^2)^{3/2}
 *   phi_i = K_C sum_{j != i} Q_j / sqrt(|x_i - x_j|^2 + eps^2)
 * Q_j = w_j z_j is the macro charge.  self_idx[i] is the source index that is
 * target i itself (excluded), or -1.  Plain sequential sum over j for each i;
 * nthreads > 1 spreads the targets over OpenMP threads (the paper's own
 * decomposition, Sec. II last paragraph) without changing any target's sum. */
void or_coulomb_field(int nt, const double *xt, const int64_t *self_idx,
                      int ns, const double *xs, const double *qs,
                      double eps, double kc, double *e_out, double *phi_out,
                      int nthreads)
{
    double eps2 = eps * eps;
    int i;
#ifdef _OPENMP
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads)
#endif
    for (i = 0; i < nt; ++i) {
        double xi = xt[3 * i], yi = xt[3 * i + 1], zi = xt[3 * i + 2];
        int64_t self = self_idx ? self_idx[i] : -1;
        double ex = 0.0, ey = 0.0, ez = 0.0, ph = 0.0;
        for (int j = 0; j < ns; ++j) {
            if ((int64_t)j == self || qs[j] == 0.0) continue;
            double dx = xi - xs[3 * j];
            double dy = yi - xs[3 * j + 1];
            double dz = zi - xs[3 * j + 2];
            double r2 = dx * dx + dy * dy + dz * dz + eps2;
            double r = sqrt(r2);
            double inv_r3 = 1.0 / (r2 * r);
            ex += qs[j] * dx * inv_r3;
            ey += qs[j] * dy * inv_r3;
            ez += qs[j] * dz * inv_r3;
            ph += qs[j] / r;
        }
        e_out[3 * i] = kc * ex;
        e_out[3 * i + 1] = kc * ey;
        e_out[3 * i + 2] = kc * ez;
        if (phi_out) phi_out[i] = kc * ph;
    }
}

/* The same sum with minimum-image displacements in a periodic cube of side
 * box (the "optional minimum-image forces" of a periodic boundary, Sec. II,
 * boundary paragraph): each component of x_i - x_j is reduced to the nearest
 * periodic image, d - box * nearbyint(d / box) (ties to even), before the
 * softened pair term is formed.  box <= 0 gives the open sum. */
void or_coulomb_field_mi(int nt, const double *xt, const int64_t *self_idx,
                         int ns, const double *xs, const double *qs,
                         double eps, double kc, double box, double *e_out,
                         double *phi_out, int nthreads)
{
    double eps2 = eps * eps;
    int i;
#ifdef _OPENMP
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads)
#endif
    for (i = 0; i < nt; ++i) {
        double xi = xt[3 * i], yi = xt[3 * i + 1], zi = xt[3 * i + 2];
        int64_t self = self_idx ? self_idx[i] : -1;
        double ex = 0.0, ey = 0.0, ez = 0.0, ph = 0.0;
        for (int j = 0; j < ns; ++j) {
            if (qs[j] == 0.0 || (int64_t)j == self) continue;
            double d[3] = {xi - xs[3 * j], yi - xs[3 * j + 1], zi - xs[3 * j + 2]};
            if (box > 0.0)
                for (int k = 0; k < 3; ++k) d[k] -= box * nearbyint(d[k] / box);
            double rm2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2] + eps2;
            double rm = sqrt(rm2);
            double inv_rm3 = 1.0 / (rm2 * rm);
            ex += qs[j] * d[0] * inv_rm3;
            ey += qs[j] * d[1] * inv_rm3;
            ez += qs[j] * d[2] * inv_rm3;
            ph += qs[j] / rm;
        }
        e_out[3 * i] = kc * ex;
        e_out[3 * i + 1] = kc * ey;
        e_out[3 * i + 2] = kc * ez;
        if (phi_out) phi_out[i] = kc * ph;
    }
}

/* --------------------------------------------------------------- Boris */

/* One relativistic Boris kick (Sec. II, "standard Boris leap frog"):
 * half electric kick, rotation about B with tan(theta/2) = h|B|/gamma,
 * second half electric kick.  h = (q/m) dt / 2.  u is updated in place. */
void or_boris_kick(double u[3], const double e[3], const double b[3],
                   double qm, double dt)
{
    double h = 0.5 * dt * qm;
    double um[3] = {u[0] + h * e[0], u[1] + h * e[1], u[2] + h * e[2]};
    double g = sqrt(1.0 + um[0] * um[0] + um[1] * um[1] + um[2] * um[2]);
    double tv[3] = {h * b[0] / g, h * b[1] / g, h * b[2] / g};
    double t2 = tv[0] * tv[0] + tv[1] * tv[1] + tv[2] * tv[2];
    double sv[3] = {2.0 * tv[0] / (1.0 + t2), 2.0 * tv[1] / (1.0 + t2),
                    2.0 * tv[2] / (1.0 + t2)};
    double up[3] = {um[0] + (um[1] * tv[2] - um[2] * tv[1]),
                    um[1] + (um[2] * tv[0] - um[0] * tv[2]),
                    um[2] + (um[0] * tv[1] - um[1] * tv[0])};
    double pl[3] = {um[0] + (up[1] * sv[2] - up[2] * sv[1]),
                    um[1] + (up[2] * sv[0] - up[0] * sv[2]),
                    um[2] + (up[0] * sv[1] - up[1] * sv[0])};
    u[0] = pl[0] + h * e[0];
    u[1] = pl[1] + h * e[1];
    u[2] = pl[2] + h * e[2];
}

/* Drift x^{n+1} = x^n + dt u^{n+1/2} / gamma^{n+1/2}. */
void or_drift(double x[3], const double u[3], double dt)
{
    double g = sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    x[0] += dt * u[0] / g;
    x[1] += dt * u[1] / g;
    x[2] += dt * u[2] / g;
}

/* Boundary handling after the drift (Sec. II): 0 open, 1 periodic on the cube
 * of side L = R_IC centred on the cluster (positions wrapped into
 * [-L/2, L/2), no image forces), 2 mixed = periodic while t < t_switch, open
 * afterwards. */
static void or_boundary(double x[3], int mode, double box, double t, double t_switch)
{
    if (mode == 0) return;
    if (mode == 2 && t >= t_switch) return;
    for (int k = 0; k < 3; ++k) {
        double h = 0.5 * box;
        x[k] = x[k] - box * floor((x[k] + h) / box);
    }
}

typedef struct {
    double a0, tau, t0, dt, eps, kc, box, t_switch;
    int pol, env, boundary;
    int min_image; /* 1: minimum-image forces while the boundary is periodic */
} or_params;

/* The Coulomb field of a step at time t: minimum-image while the boundary is
 * periodic (mode 1, or mode 2 before t_switch) and min_image is set. */
static void or_step_field(int n, const double *x, const int64_t *self_idx, const double *q,
                          const or_params *p, double t, double *e, double *phi, int nthreads)
{
    int periodic = p->boundary == 1 || (p->boundary == 2 && t < p->t_switch);
    if (p->min_image && periodic)
        or_coulomb_field_mi(n, x, self_idx, n, x, q, p->eps, p->kc, p->box, e, phi, nthreads);
    else
        or_coulomb_field(n, x, self_idx, n, x, q, p->eps, p->kc, e, phi, nthreads);
}

/* nsteps full MD steps (Sec. II) on n particles, starting at step index
 * step0 (t_n = t0 + n dt).  x, u: [n][3] in/out; qm = z/m; q = w z (macro
 * charge, the source strength); active[i] = 0 excludes particle i from the
 * push, and an inactive particle must carry q = 0 so that it is no source.
 * Scratch: e [n][3], self_idx [n]. */
void or_md_steps(int n, double *x, double *u, const double *qm, const double *q,
                 const uint8_t *active, const or_params *p, int64_t step0,
                 int nsteps, double *e, int64_t *self_idx, int nthreads)
{
    for (int i = 0; i < n; ++i) self_idx[i] = i;
    for (int s = 0; s < nsteps; ++s) {
        int64_t step = step0 + s;
        double t = p->t0 + (double)step * p->dt;
        double a[3], b[3];
        or_laser_fields(t, p->a0, p->pol, p->env, p->tau, a, b);
        or_step_field(n, x, self_idx, q, p, t, e, NULL, nthreads);
        for (int i = 0; i < n; ++i) {
            if (!active[i]) continue;
            double et[3] = {e[3 * i] + a[0], e[3 * i + 1] + a[1], e[3 * i + 2] + a[2]};
            or_boris_kick(&u[3 * i], et, b, qm[i], p->dt);
            or_drift(&x[3 * i], &u[3 * i], p->dt);
            or_boundary(&x[3 * i], p->boundary, p->box, t + p->dt, p->t_switch);
        }
    }
}

/* Diagnostics at integer time t_n for the state (x^n, u^{n-1/2}):
 *   u^n = (u^{n-1/2} + u^{n+1/2}) / 2 with u^{n+1/2} the kick of this step,
 *   KE  = sum w m (gamma(u^n) - 1),   PE = 1/2 sum_i Q_i phi_i,
 *   P   = sum w m u^n.
 * wm = w * m.  out[0..7] = KE, KE of ions (z >= 0), KE of electrons (z < 0),
 * PE, Px, Py, Pz, number of active particles. */
void or_diagnostics(int n, const double *x, const double *u, const double *qm,
                    const double *q, const double *wm, const int32_t *z,
                    const uint8_t *active, const or_params *p, int64_t step,
                    double *e, double *phi, int64_t *self_idx, double *out,
                    int nthreads)
{
    double t = p->t0 + (double)step * p->dt;
    double a[3], b[3];
    for (int i = 0; i < n; ++i) self_idx[i] = i;
    or_laser_fields(t, p->a0, p->pol, p->env, p->tau, a, b);
    or_step_field(n, x, self_idx, q, p, t, e, phi, nthreads);
    double ke = 0, kei = 0, kee = 0, pe = 0, px = 0, py = 0, pz = 0, na = 0;
    for (int i = 0; i < n; ++i) {
        if (!active[i]) continue;
        double et[3] = {e[3 * i] + a[0], e[3 * i + 1] + a[1], e[3 * i + 2] + a[2]};
        double un[3] = {u[3 * i], u[3 * i + 1], u[3 * i + 2]};
        or_boris_kick(un, et, b, qm[i], p->dt);
        double um[3] = {0.5 * (u[3 * i] + un[0]), 0.5 * (u[3 * i + 1] + un[1]),
                        0.5 * (u[3 * i + 2] + un[2])};
        double uu = um[0] * um[0] + um[1] * um[1] + um[2] * um[2];
        /* gamma - 1 = uu / (gamma + 1), free of cancellation */
        double k = wm[i] * uu / (sqrt(1.0 + uu) + 1.0);
        ke += k;
        if (z[i] < 0) kee += k; else kei += k;
        pe += 0.5 * q[i] * phi[i];
        px += wm[i] * um[0];
        py += wm[i] * um[1];
        pz += wm[i] * um[2];
        na += 1.0;
    }
    out[0] = ke; out[1] = kei; out[2] = kee; out[3] = pe;
    out[4] = px; out[5] = py; out[6] = pz; out[7] = na;
}

/* ------------------------------------------------- directional detectors */

/* Ion energy detectors on a sphere of radius R around `center` (the IEDF of
 * Sec. III, Fig. 3, read at a fixed radius): an ion (active, z >= 1) that
 * first crosses the sphere outward during a step, |x^n - c| < R <= |x^{n+1} - c|,
 * is recorded once with its kinetic energy (gamma - 1) m c^2 at u^{n+1/2}.
 * Detectors: 0 = +x, 1 = -x, 2 = +y, 3 = -y (the ion's direction
 * (x^{n+1} - c)/|x^{n+1} - c| within the cone of half-angle theta around the
 * axis: component >= cos(theta) |x^{n+1} - c|), 4 = all directions.
 * Histogram hist[5][nbins + 1]: bin floor(E nbins / e_max) for E < e_max,
 * bin nbins for E >= e_max (eV).  crossed[i] marks recorded ions.
 * Floating point is evaluated in the order written (no contraction). */
static double or_ke_ev(const double u[3], double mass)
{
    double uu = (u[0] * u[0] + u[1] * u[1]) + u[2] * u[2];
    return (uu / (sqrt(1.0 + uu) + 1.0)) * mass * OR_ME_C2_EV;
}

static int or_energy_bin(double ke, double e_max, int nbins)
{
    if (!(ke < e_max)) return nbins;
    int b = (int)floor(ke * (double)nbins / e_max);
    return b < 0 ? 0 : (b >= nbins ? nbins - 1 : b);
}

void or_detect(int n, const double *x_prev, const double *x_next, const double *u,
               const double *mass, const int32_t *z, const uint8_t *active,
               const double center[3], double radius, double cos_cone, double e_max_ev,
               int nbins, uint8_t *crossed, uint64_t *hist)
{
    double R2 = radius * radius;
    for (int i = 0; i < n; ++i) {
        if (!active[i] || z[i] < 1 || crossed[i]) continue;
        double a0 = x_prev[3 * i] - center[0], a1 = x_prev[3 * i + 1] - center[1],
               a2 = x_prev[3 * i + 2] - center[2];
        double b0 = x_next[3 * i] - center[0], b1 = x_next[3 * i + 1] - center[1],
               b2 = x_next[3 * i + 2] - center[2];
        double rp2 = (a0 * a0 + a1 * a1) + a2 * a2;
        double rn2 = (b0 * b0 + b1 * b1) + b2 * b2;
        if (!(rp2 < R2 && rn2 >= R2)) continue;
        crossed[i] = 1;
        int bin = or_energy_bin(or_ke_ev(&u[3 * i], mass[i]), e_max_ev, nbins);
        double c = cos_cone * sqrt(rn2);
        hist[4 * (nbins + 1) + bin] += 1;
        if (b0 >= c) hist[0 * (nbins + 1) + bin] += 1;
        if (-b0 >= c) hist[1 * (nbins + 1) + bin] += 1;
        if (b1 >= c) hist[2 * (nbins + 1) + bin] += 1;
        if (-b1 >= c) hist[3 * (nbins + 1) + bin] += 1;
    }
}

/* Energy histogram hist[nbins + 1] of the ions (active, z >= 1) not yet
 * recorded by the detectors, at momentum u (the rest of the total IEDF). */
void or_iedf_inside(int n, const double *u, const double *mass, const int32_t *z,
                    const uint8_t *active, const uint8_t *crossed, double e_max_ev, int nbins,
                    uint64_t *hist)
{
    for (int i = 0; i < n; ++i) {
        if (!active[i] || z[i] < 1 || crossed[i]) continue;
        hist[or_energy_bin(or_ke_ev(&u[3 * i], mass[i]), e_max_ev, nbins)] += 1;
    }
}

