/*
 * ionize_oracle.c -- FP64 CPU oracle of the Monte-Carlo ionization step of the
 * laser-cluster MD method (Holkundkar, arXiv:1307.3711, Sec. II, ionization
 * paragraph).  TEST INFRASTRUCTURE ONLY (see md_oracle.c).
 *
 * The paper names the rates but prints neither formulas nor constants: optical
 * field ionization by the ADK tunnelling formula (Ammosov, Delone, Krainov,
 * Sov. Phys. JETP 64, 1191 (1986)), collisional ionization by fitted rates
 * (Voronov) or Lotz's formula.  Readings taken here (listed in the design
 * notes): the static ADK rate with l* = n* - 1 and l = m = 0; Lotz's
 * single-shell cross section sigma = a q ln(E/P)/(E P), a = 4.5e-14 cm^2 eV^2,
 * Maxwell-averaged in closed form, used for argon as well (the Voronov fit
 * coefficients are not available); local electron density and temperature
 * from the electrons within r_loc of the ion.  Ionization potentials and
 * outer-shell occupations are inputs (a species table), not constants here.
 *
 *   nu_total = nu_ofi + nu_ci,  P = 1 - exp(-nu_total dt_ion),
 *   alpha in (0, 1] from Philox4x32-10 keyed on (seed) with counter
 *   (ion id, step lo, step hi, 0); the ion ionizes if alpha < P.
 *
 * Parity unpinned: the ADK rate away from n* = 1.  The tests fix it where
 * n* = 1 (l* = 0, both Gamma factors of C^2 equal 1): Landau's exact hydrogen
 * rate, and its Coulomb scaling to hydrogen-like ions of any nuclear charge
 * (Ip = Z^2/2), which fixes the Ip and F0 dependence.  Nothing in reach fixes
 * the l* and Gamma terms of C^2 for n* != 1 (planted slips there pass every
 * test), and the species data are unpinned as well, so the absolute rates of
 * multi-electron ions rest on the formula as written above.
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>

#define IO_PI 3.14159265358979323846
#define IO_EULER_GAMMA 0.57721566490153286061
#define IO_HARTREE_EV 27.211386245988        /* Hartree energy in eV */
#define IO_FIELD_AU 5.14220674763e11         /* atomic unit of field, V/m */
#define IO_TIME_AU 2.4188843265857e-17       /* atomic unit of time, s */
#define IO_ME_C2_EV 510998.95                /* electron rest energy, eV */
#define IO_C 299792458.0                     /* m/s */
#define IO_E_CHARGE 1.602176634e-19          /* C */
#define IO_ME 9.1093837015e-31               /* kg */
#define IO_LOTZ_A 4.5e-14                    /* cm^2 eV^2 */

/* ---------------------------------------------------------------- Philox */

/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of
 * (L, R) -> two 32x32->64 multiplications by 0xD2511F53 and 0xCD9E8D57, the
 * high halves xored with the other counter words and the round key, the key
 * bumped by the Weyl constants 0x9E3779B9, 0xBB67AE85 between rounds. */
void io_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        if (r < 9) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform in (0, 1]: (w + 1) 2^-32 (the alpha of Sec. II, 0 < alpha <= 1). */
double io_uniform_open0(uint32_t w)
{
    return ((double)w + 1.0) * (1.0 / 4294967296.0);
}

/* ------------------------------------------------------------------ E1 */

/* Exponential integral E1(x) = int_x^inf e^-t / t dt, x > 0: power series
 * -gamma - ln x - sum_k (-x)^k / (k k!) for x <= 1, the continued fraction
 * e^-x / (x + 1/(1 + 1/(x + 2/(1 + 2/(x + ...))))) (modified Lentz) above. */
double io_e1(double x)
{
    if (!(x > 0.0)) return INFINITY;
    if (x <= 1.0) {
        double sum = 0.0, term = 1.0;
        for (int k = 1; k < 60; ++k) {
            term *= -x / k;
            double add = -term / k;
            sum += add;
            if (fabs(add) < 1e-18 * fabs(sum)) break;
        }
        return -IO_EULER_GAMMA - log(x) + sum;
    }
    /* continued fraction in the even form x + 1 - 1^2/(x + 3 - 2^2/(x + 5 - ...)) */
    const double tiny = 1e-300;
    double b = x + 1.0, c = 1.0 / tiny, d = 1.0 / b, h = d;
    for (int i = 1; i < 300; ++i) {
        double a = -(double)i * i;
        b += 2.0;
        d = 1.0 / (a * d + b);
        c = b + a / c;
        double del = c * d;
        h *= del;
        if (fabs(del - 1.0) < 1e-16) break;
    }
    return h * exp(-x);
}

/* ----------------------------------------------------------------- rates */

/* Static ADK tunnelling rate in atomic units for field strength F (a.u.),
 * ionization potential Ip (a.u.) and residual charge Z (charge after
 * ionization): n* = Z / sqrt(2 Ip), l* = n* - 1, l = m = 0,
 *   C^2 = 2^{2n*} / (n* Gamma(n* + l* + 1) Gamma(n* - l*)),
 *   w = C^2 Ip (2 F0 / F)^{2n* - 1} exp(-2 F0 / (3 F)),  F0 = (2 Ip)^{3/2}. */
double io_adk_rate_au(double F, double ip, double Z)
{
    if (!(F > 0.0)) return 0.0;
    double ns = Z / sqrt(2.0 * ip);
    double ls = ns - 1.0;
    double c2 = pow(2.0, 2.0 * ns) / (ns * tgamma(ns + ls + 1.0) * tgamma(ns - ls));
    double F0 = pow(2.0 * ip, 1.5);
    return c2 * ip * pow(2.0 * F0 / F, 2.0 * ns - 1.0) * exp(-2.0 * F0 / (3.0 * F));
}

/* Lotz rate coefficient <sigma v> in cm^3/s for a shell of q electrons bound
 * by P (eV) at electron temperature T (eV): with sigma = a q ln(E/P)/(E P),
 *   <sigma v> = sqrt(8 / (pi m_e)) a q E1(P/T) / (P sqrt(T)). */
double io_lotz_rate_cgs(double P, double T, double q)
{
    if (!(T > 0.0) || !(q > 0.0)) return 0.0;
    double v_th = sqrt(8.0 * IO_E_CHARGE / (IO_PI * IO_ME)) * 100.0; /* cm/s per sqrt(eV) */
    return v_th * IO_LOTZ_A * q * io_e1(P / T) / (P * sqrt(T));
}

/* Total rate per unit dimensionless time (1/omega) of an ion of charge
 * state z (z < zmax) in a field of magnitude |a| (laser + Coulomb, paper
 * units), with local electron density ne (cm^-3) and temperature Te (eV).
 * ip_ev[z], q_outer[z]: potential and outer electrons of the z -> z+1 step. */
double io_rate_total(double a_mag, int z, double ne, double te, const double *ip_ev,
                     const double *q_outer, double lambda_um)
{
    double lam = lambda_um * 1e-6;
    double k = 2.0 * IO_PI / lam;
    double omega = IO_C * k;
    double e_si = a_mag * IO_ME_C2_EV * k;                 /* V/m */
    double F = e_si / IO_FIELD_AU;
    double ip = ip_ev[z] / IO_HARTREE_EV;
    double w_ofi = io_adk_rate_au(F, ip, (double)(z + 1)) / IO_TIME_AU;   /* 1/s */
    double w_ci = ne > 0.0 ? ne * io_lotz_rate_cgs(ip_ev[z], te, q_outer[z]) : 0.0;
    return (w_ofi + w_ci) / omega;
}

/* ------------------------------------------------ local electron moments */

/* For each target (ion) position, the electrons (q < 0) within r_loc:
 * ne = sum w / (4/3 pi r_loc^3) converted to cm^-3, and the temperature
 * Te = (m_e c^2 / 3) (<|u|^2> - |<u>|^2) in eV (non-relativistic, weights w,
 * local mean frame); 0 when no electron is in range. */
void io_local_moments(int nt, const double *xt, int ns, const double *xs, const double *us,
                      const double *ws, const int32_t *zs, const uint8_t *active_s,
                      double r_loc, double lambda_um, double *ne, double *te)
{
    double k = 2.0 * IO_PI / (lambda_um * 1e-6);
    double vol_cm3 = (4.0 / 3.0) * IO_PI * pow(r_loc / k, 3) * 1e6;
    double r2max = r_loc * r_loc;
    for (int i = 0; i < nt; ++i) {
        double sw = 0, sux = 0, suy = 0, suz = 0, su2 = 0;
        for (int j = 0; j < ns; ++j) {
            if (!active_s[j] || zs[j] >= 0) continue;
            double dx = xs[3 * j] - xt[3 * i];
            double dy = xs[3 * j + 1] - xt[3 * i + 1];
            double dz = xs[3 * j + 2] - xt[3 * i + 2];
            if (dx * dx + dy * dy + dz * dz >= r2max) continue;
            double w = ws[j];
            double ux = us[3 * j], uy = us[3 * j + 1], uz = us[3 * j + 2];
            sw += w;
            sux += w * ux; suy += w * uy; suz += w * uz;
            su2 += w * (ux * ux + uy * uy + uz * uz);
        }
        if (sw > 0.0) {
            double mx = sux / sw, my = suy / sw, mz = suz / sw;
            double var = su2 / sw - (mx * mx + my * my + mz * mz);
            ne[i] = sw / vol_cm3;
            te[i] = var > 0.0 ? IO_ME_C2_EV * var / 3.0 : 0.0;
        } else {
            ne[i] = 0.0;
            te[i] = 0.0;
        }
    }
}

/* The same moments with minimum-image distances in a periodic cube of side
 * box (box <= 0: open): an electron counts if its nearest periodic image is
 * within r_loc of the ion. */
void io_local_moments_box(int nt, const double *xt, int ns, const double *xs, const double *us,
                          const double *ws, const int32_t *zs, const uint8_t *active_s,
                          double r_loc, double lambda_um, double box, double *ne, double *te)
{
    double kw = 2.0 * IO_PI / (lambda_um * 1e-6);
    double vol = (4.0 / 3.0) * IO_PI * pow(r_loc / kw, 3) * 1e6;
    double rl2 = r_loc * r_loc;
    for (int i = 0; i < nt; ++i) {
        double s_w = 0, s_x = 0, s_y = 0, s_z = 0, s_2 = 0;
        for (int j = 0; j < ns; ++j) {
            if (!active_s[j] || zs[j] >= 0) continue;
            double d[3];
            for (int c = 0; c < 3; ++c) {
                d[c] = xs[3 * j + c] - xt[3 * i + c];
                if (box > 0.0) d[c] -= box * nearbyint(d[c] / box);
            }
            if (d[0] * d[0] + d[1] * d[1] + d[2] * d[2] >= rl2) continue;
            double wj = ws[j];
            double vx = us[3 * j], vy = us[3 * j + 1], vz = us[3 * j + 2];
            s_w += wj;
            s_x += wj * vx; s_y += wj * vy; s_z += wj * vz;
            s_2 += wj * (vx * vx + vy * vy + vz * vz);
        }
        if (s_w > 0.0) {
            double ax = s_x / s_w, ay = s_y / s_w, az = s_z / s_w;
            double v2 = s_2 / s_w - (ax * ax + ay * ay + az * az);
            ne[i] = s_w / vol;
            te[i] = v2 > 0.0 ? IO_ME_C2_EV * v2 / 3.0 : 0.0;
        } else {
            ne[i] = 0.0;
            te[i] = 0.0;
        }
    }
}

/* ------------------------------------------------------------- decision */

/* Monte-Carlo decision for n ions with ids id[] (Philox counter word 0),
 * charge states z[], field magnitude a_mag[], ne[], te[] at step `step`.
 * An ion with z < zmax ionizes if alpha < 1 - exp(-nu dt_ion); then
 * fired[i] = 1, z[i] += 1 and offset[3i..] is the new electron's position
 * relative to the ion: uniform in the ball of radius r_create, from Philox
 * words 1-3 (cos(theta) = 2 u1 - 1, phi = 2 pi u2, r = r_create u3^{1/3},
 * u_k = (w_k + 0.5) 2^-32).  prob[i] receives P. */
void io_decide(int n, const int64_t *id, int32_t *z, const double *a_mag, const double *ne,
               const double *te, const double *ip_ev, const double *q_outer, int zmax,
               double lambda_um, double dt_ion, uint64_t seed, int64_t step, double r_create,
               uint8_t *fired, double *offset, double *prob)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int i = 0; i < n; ++i) {
        fired[i] = 0;
        offset[3 * i] = offset[3 * i + 1] = offset[3 * i + 2] = 0.0;
        prob[i] = 0.0;
        if (z[i] < 0 || z[i] >= zmax) continue;
        double nu = io_rate_total(a_mag[i], z[i], ne[i], te[i], ip_ev, q_outer, lambda_um);
        double P = -expm1(-nu * dt_ion);
        prob[i] = P;
        uint32_t ctr[4] = {(uint32_t)id[i], (uint32_t)step, (uint32_t)((uint64_t)step >> 32), 0u};
        uint32_t w[4];
        io_philox4x32_10(ctr, key, w);
        double alpha = io_uniform_open0(w[0]);
        if (alpha < P) {
            fired[i] = 1;
            z[i] += 1;
            double u1 = ((double)w[1] + 0.5) * (1.0 / 4294967296.0);
            double u2 = ((double)w[2] + 0.5) * (1.0 / 4294967296.0);
            double u3 = ((double)w[3] + 0.5) * (1.0 / 4294967296.0);
            double ct = 2.0 * u1 - 1.0, st = sqrt(fmax(0.0, 1.0 - ct * ct));
            double ph = 2.0 * IO_PI * u2, r = r_create * cbrt(u3);
            offset[3 * i] = r * st * cos(ph);
            offset[3 * i + 1] = r * st * sin(ph);
            offset[3 * i + 2] = r * ct;
        }
    }
}
