/*
 * generate_oracle.c -- FP64 CPU oracle of the seeded generation of a
 * cluster's particle records (Holkundkar, arXiv:1307.3711, Sec. II: the atoms
 * of a cluster of radius R0 are placed at random inside the sphere; Eq. 1
 * lumps N_atoms / N_macro real atoms into one macro-particle of weight w).
 * TEST INFRASTRUCTURE ONLY (see md_oracle.c).
 *
 * The paper says only "randomly" for the placement and gives no initial
 * velocities; the readings taken here (and by the library's generator, whose
 * code is separate) are:
 *   - records in the order ions, electrons, inactive electron slots;
 *   - position of an ion or electron: uniform in the ball of radius r0 about
 *     `center`, by rejection from the cube [-1, 1]^3: attempt a draws
 *     Philox4x32-10 with key (seed lo, seed hi) and counter
 *     (record lo, record hi, a, 0x67656E01); s_k = (w_k + 1/2) 2^-31 - 1 for
 *     k = 0, 1, 2 (exact in FP64); accepted when (s0 s0 + s1 s1) + s2 s2 < 1,
 *     each operation rounded to nearest; x_k = center_k + r0 s_k.  After 64
 *     rejected attempts (probability 2e-21 per record) the record sits at the
 *     centre;
 *   - momentum: a non-relativistic Maxwellian at temperature kT (eV),
 *     u_k = sigma n_k, sigma = sqrt(kT / (m m_e c^2)), with normal deviates
 *     from Box-Muller on the words of counter (record lo, record hi, 0,
 *     0x67656E02): n0, n1 = rho (cos, sin)(2 pi v1), rho = sqrt(-2 ln v0),
 *     v0 = (w0 + 1) 2^-32 in (0, 1], v1 = (w1 + 1/2) 2^-32; n2 = sqrt(-2 ln v2)
 *     cos(2 pi v3) from words 2 and 3 likewise; kT = 0 gives u = 0;
 *   - charge z = ion_charge (ions), -1 (electrons), 0 (slots); mass ion_mass
 *     (ions), 1 (electrons and slots); weight w for every record; slots sit
 *     at the centre with u = 0.
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>

#define GO_PI 3.14159265358979323846
#define GO_ME_C2_EV 510998.95
#define GO_TAG_POSITION 0x67656E01u
#define GO_TAG_MOMENTUM 0x67656E02u
#define GO_MAX_ATTEMPTS 64

void io_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]);

/* Point of record `rec` uniform in the unit ball (s[3]), by rejection. */
static void go_unit_ball(uint64_t seed, int64_t rec, double s[3])
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (uint32_t a = 0; a < GO_MAX_ATTEMPTS; ++a) {
        uint32_t ctr[4] = {(uint32_t)rec, (uint32_t)((uint64_t)rec >> 32), a, GO_TAG_POSITION};
        uint32_t w[4];
        io_philox4x32_10(ctr, key, w);
        double c[3];
        for (int k = 0; k < 3; ++k) c[k] = ((double)w[k] + 0.5) * (1.0 / 2147483648.0) - 1.0;
        double r2 = c[0] * c[0] + c[1] * c[1];
        r2 = r2 + c[2] * c[2];
        if (r2 < 1.0) {
            s[0] = c[0];
            s[1] = c[1];
            s[2] = c[2];
            return;
        }
    }
    s[0] = s[1] = s[2] = 0.0;
}

/* Three standard normal deviates of record `rec` (Box-Muller). */
static void go_normals(uint64_t seed, int64_t rec, double n[3])
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t ctr[4] = {(uint32_t)rec, (uint32_t)((uint64_t)rec >> 32), 0u, GO_TAG_MOMENTUM};
    uint32_t w[4];
    io_philox4x32_10(ctr, key, w);
    double v0 = ((double)w[0] + 1.0) * (1.0 / 4294967296.0);
    double v1 = ((double)w[1] + 0.5) * (1.0 / 4294967296.0);
    double v2 = ((double)w[2] + 1.0) * (1.0 / 4294967296.0);
    double v3 = ((double)w[3] + 0.5) * (1.0 / 4294967296.0);
    double rho = sqrt(-2.0 * log(v0));
    n[0] = rho * cos(2.0 * GO_PI * v1);
    n[1] = rho * sin(2.0 * GO_PI * v1);
    n[2] = sqrt(-2.0 * log(v2)) * cos(2.0 * GO_PI * v3);
}

/* Records of one cluster (n_ions + n_electrons + n_slots of them) into the
 * host arrays x[n][3], u[n][3], z[n], mass[n], w[n], kind[n] (kind 0 ion,
 * 1 electron, 2 inactive). */
void or_generate_cluster(double r0, const double center[3], double ion_mass, double weight,
                         double kt_e_ev, double kt_i_ev, int64_t n_ions, int64_t n_electrons,
                         int64_t n_slots, int32_t ion_charge, uint64_t seed, double *x, double *u,
                         int32_t *z, double *mass, double *w, uint8_t *kind)
{
    const int64_t n = n_ions + n_electrons + n_slots;
    const double sig_i = kt_i_ev > 0.0 ? sqrt(kt_i_ev / (ion_mass * GO_ME_C2_EV)) : 0.0;
    const double sig_e = kt_e_ev > 0.0 ? sqrt(kt_e_ev / (1.0 * GO_ME_C2_EV)) : 0.0;
    for (int64_t i = 0; i < n; ++i) {
        const int k = i < n_ions ? 0 : (i < n_ions + n_electrons ? 1 : 2);
        kind[i] = (uint8_t)k;
        z[i] = k == 0 ? ion_charge : (k == 1 ? -1 : 0);
        mass[i] = k == 0 ? ion_mass : 1.0;
        w[i] = weight;
        double s[3] = {0.0, 0.0, 0.0};
        if (k != 2) go_unit_ball(seed, i, s);
        for (int c = 0; c < 3; ++c) x[3 * i + c] = center[c] + r0 * s[c];
        const double sig = k == 0 ? sig_i : (k == 1 ? sig_e : 0.0);
        double g[3] = {0.0, 0.0, 0.0};
        if (sig > 0.0) go_normals(seed, i, g);
        for (int c = 0; c < 3; ++c) u[3 * i + c] = sig * g[c];
    }
}
