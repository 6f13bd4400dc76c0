/*
 * oracle.c -- FP64 CPU oracle of the Langevin nanoparticle-aggregation step
 * (arXiv 2501.04456, a Langevin-dynamics model of nanoparticle aggregation in
 * an evaporating droplet).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
 * GPU library is checked against.  Only the test suite, the smoke check and
 * the CPU-baseline leg of the benchmark load it; the product library never
 * links, includes or calls it, and it shares no code, header or table with
 * the CUDA sources.
 *
 * Every function is written as the plain definition of what it computes, in
 * IEEE double precision, with no blocking, fusion or reordering: one loop per
 * sum, j in ascending order.  Build with -ffp-contract=off so that no
 * multiply-add is fused (results are then identical on x86-64 and aarch64).
 *
 * The paper states its forces in words only (Sec. 2.1 and the six-step loop of
 * Sec. 2.2); the formulas below are the textbook forms it names, with every
 * reading the paper leaves open stated at the function that takes it.
 *
 * Parity status of each function (what pins it is in tests/test_oracle_pins.py):
 *   or_philox4x32_10 ........ pinned (cuRAND host generator, statistics)
 *   or_normals .............. pinned (moments, chi-square of the normal CDF)
 *   or_mix_tables ........... pinned (closed forms)
 *   or_pair_forces .......... pinned (two-body closed forms, Newton III, Gauss)
 *   or_external_forces ...... pinned (closed forms)
 *   or_radius ............... pinned (closed form)
 *   or_run .................. pinned (free-particle MSD, equipartition, drift,
 *                             brute-force tiny-N step, resume)
 *   or_pair_hist / or_rdf ... pinned (uniform-ball chord law, FCC shells)
 *   or_boxcount ............. pinned (lattices of dimension 1, 2, 3)
 *   or_rg ................... pinned (solid ball R_g, fractal equation)
 *   or_radial_hist .......... pinned (uniform ball -> flat profile)
 *   or_surface_count ........ pinned (hand-placed NPs on both sides of the band edges)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAX_TYPES 8

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 counter-based generator, written from its published
 * definition (J. K. Salmon, M. A. Moraes, R. O. Dror, D. E. Shaw, "Parallel
 * random numbers: as easy as 1, 2, 3", SC'11).  One round maps the counter
 * (c0,c1,c2,c3) with round key (k0,k1) through two 32x32->64 multiplications:
 *   (hi0,lo0) = M0*c0, (hi1,lo1) = M1*c2,
 *   out = (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0);
 * the key is bumped by the Weyl constants between rounds.  Ten rounds.      */
static const uint32_t OR_PHILOX_M0 = 0xD2511F53u;
static const uint32_t OR_PHILOX_M1 = 0xCD9E8D57u;
static const uint32_t OR_PHILOX_W0 = 0x9E3779B9u;
static const uint32_t OR_PHILOX_W1 = 0xBB67AE85u;

void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2],
                      uint32_t out[4])
{
    uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += OR_PHILOX_W0;
            k1 += OR_PHILOX_W1;
        }
        uint64_t p0 = (uint64_t)OR_PHILOX_M0 * (uint64_t)c[0];
        uint64_t p1 = (uint64_t)OR_PHILOX_M1 * (uint64_t)c[2];
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c[1] ^ k0;
        uint32_t n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
    }
    out[0] = c[0];
    out[1] = c[1];
    out[2] = c[2];
    out[3] = c[3];
}

/* Raw stream for tests: block b uses counter (ctr0 + b, ctr1, ctr2, ctr3)
 * with the 32-bit carry of ctr0+b propagated into ctr1. */
void or_philox_blocks(uint64_t seed, const uint32_t ctr[4], int64_t n_blocks,
                      uint32_t *out /* 4*n_blocks */)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int64_t b = 0; b < n_blocks; ++b) {
        uint64_t lo = (uint64_t)ctr[0] + (uint64_t)b;
        uint32_t c[4] = {(uint32_t)lo, ctr[1] + (uint32_t)(lo >> 32), ctr[2], ctr[3]};
        or_philox4x32_10(c, key, out + 4 * b);
    }
}

/* Noise convention of this library: the key is the 64-bit seed (low word,
 * high word); the counter is (particle index, step low word, step high word,
 * purpose).  Uniforms are u = (k + 1/2) 2^-32 in (0,1); three standard normals
 * come from the Box-Muller transform (G. E. P. Box, M. E. Muller, 1958):
 *   n0 = sqrt(-2 ln u0) cos(2 pi u1), n1 = sqrt(-2 ln u0) sin(2 pi u1),
 *   n2 = sqrt(-2 ln u2) cos(2 pi u3).                                       */
static void or_normals3(uint64_t seed, uint64_t i, int64_t step, uint32_t purpose,
                        double out[3])
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint64_t s = (uint64_t)step;
    uint32_t ctr[4] = {(uint32_t)i, (uint32_t)s, (uint32_t)(s >> 32), purpose};
    uint32_t r[4];
    or_philox4x32_10(ctr, key, r);
    const double two_m32 = 1.0 / 4294967296.0;
    double u0 = ((double)r[0] + 0.5) * two_m32;
    double u1 = ((double)r[1] + 0.5) * two_m32;
    double u2 = ((double)r[2] + 0.5) * two_m32;
    double u3 = ((double)r[3] + 0.5) * two_m32;
    const double two_pi = 6.283185307179586476925286766559;
    double rho1 = sqrt(-2.0 * log(u0));
    double rho2 = sqrt(-2.0 * log(u2));
    out[0] = rho1 * cos(two_pi * u1);
    out[1] = rho1 * sin(two_pi * u1);
    out[2] = rho2 * cos(two_pi * u3);
}

void or_normals(uint64_t seed, int64_t step, uint32_t purpose, int64_t n,
                double *out /* n*3 */)
{
    for (int64_t i = 0; i < n; ++i)
        or_normals3(seed, (uint64_t)i, step, purpose, out + 3 * i);
}

/* ------------------------------------------------------------------------ */
/* Per type-pair interaction table (Sec. 2.1: the like and unlike type pairs
 * each have their own interaction parameters; Table 1 prints an epsilon
 * matrix).  Default mixing is Lorentz-Berthelot: sigma_ab = (sigma_a +
 * sigma_b)/2, eps_ab = sqrt(eps_a eps_b); an explicit T x T epsilon matrix
 * replaces the eps rule.  The LJ cutoff is lj_cut * sigma_ab.              */
void or_mix_tables(int T, const double *sigma, const double *eps,
                   const double *eps_override /* T*T or NULL */, double lj_cut,
                   double *sig_ab, double *eps_ab, double *rc_ab)
{
    for (int a = 0; a < T; ++a)
        for (int b = 0; b < T; ++b) {
            double s = 0.5 * (sigma[a] + sigma[b]);
            sig_ab[a * T + b] = s;
            eps_ab[a * T + b] = eps_override ? eps_override[a * T + b]
                                             : sqrt(eps[a] * eps[b]);
            rc_ab[a * T + b] = lj_cut * s;
        }
}

/* ------------------------------------------------------------------------ */
/* Pair forces, step (ii) of the loop in Sec. 2.2.  For every selected i:
 *   F_i = sum_{j != i} [ C q_i q_j r_ij / r^3
 *                       + 24 eps_ij (2 (s/r)^12 - (s/r)^6) r_ij / r^2 * [r < rc_ij] ]
 * with r_ij = x_i - x_j, s = sigma_ij, C = Bjerrum length (energy unit kT = 1).
 * LJ is truncated and not shifted (Sec. 2.2 step ii).  Coulomb is summed over
 * all pairs (no truncation) when rcc_ab is NULL; otherwise the Coulomb term of
 * a pair counts only for r < rcc_ab (truncated, not shifted: the paper's
 * "pure" Coulomb with the interaction range of step i).  x is row-major n x 3.
 * sel (length n_sel) picks the rows to evaluate; NULL means rows 0..n_sel-1.
 * F is n_sel x 3.                                                           */
void or_pair_forces(int64_t n, const double *x, const int32_t *type, int T,
                    const double *sig_ab, const double *eps_ab, const double *rc_ab,
                    const double *rcc_ab, const double *charge, double bjerrum, int lj_on,
                    int coul_on, int64_t n_sel, const int64_t *sel, double *F)
{
    if (!lj_on && !coul_on) { /* every term of the sum is zero */
        memset(F, 0, sizeof(double) * 3 * (size_t)n_sel);
        return;
    }
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t s = 0; s < n_sel; ++s) {
        int64_t i = sel ? sel[s] : s;
        int ti = type[i];
        double fx = 0.0, fy = 0.0, fz = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i)
                continue;
            int tj = type[j];
            double dx = x[3 * i + 0] - x[3 * j + 0];
            double dy = x[3 * i + 1] - x[3 * j + 1];
            double dz = x[3 * i + 2] - x[3 * j + 2];
            double r2 = dx * dx + dy * dy + dz * dz;
            double r = sqrt(r2);
            double f = 0.0; /* force / |r_ij| times 1/r, i.e. F = f * r_ij */
            if (coul_on && (!rcc_ab || r < rcc_ab[ti * T + tj]))
                f += bjerrum * charge[ti] * charge[tj] / (r2 * r);
            if (lj_on) {
                int p = ti * T + tj;
                if (r < rc_ab[p]) {
                    double sr = sig_ab[p] / r;
                    double sr6 = sr * sr * sr * sr * sr * sr;
                    f += 24.0 * eps_ab[p] * (2.0 * sr6 * sr6 - sr6) / r2;
                }
            }
            fx += f * dx;
            fy += f * dy;
            fz += f * dz;
        }
        F[3 * s + 0] = fx;
        F[3 * s + 1] = fy;
        F[3 * s + 2] = fz;
    }
}

/* ------------------------------------------------------------------------ */
/* Droplet radius, step (iii): the radius-square law R(t)^2 = R0^2 - k t
 * (k > 0 evaporation, k < 0 condensation, k = 0 stationary), clamped at 0.  */
double or_radius(double R0, double k_evap, double t)
{
    double R2 = R0 * R0 - k_evap * t;
    return R2 > 0.0 ? sqrt(R2) : 0.0;
}

/* Simulation parameters of the oracle (its own definition; the GPU library
 * declares its own structure and the test harness fills both).            */
typedef struct {
    int32_t n_types;
    int32_t rot_mode;   /* 0 none, 1 about z, 2 isotropic */
    int32_t lj_on;
    int32_t coul_on;
    int32_t wall_on;    /* 0 off, 1 beyond the equilibrium point, 2 within the band only */
    int32_t integrator; /* 0 BAOAB Langevin, 1 overdamped (Brownian), 2 printed step vi */
    uint64_t seed;
    double dt, kT, R0, k_evap, g, omega, bjerrum, lj_cut;
    double sigma[OR_MAX_TYPES];
    double eps[OR_MAX_TYPES];
    double mass[OR_MAX_TYPES];
    double charge[OR_MAX_TYPES];
    double gamma[OR_MAX_TYPES];  /* friction rate, 1/time */
    double k_wall[OR_MAX_TYPES]; /* interface spring constant */
    double eps_override[OR_MAX_TYPES * OR_MAX_TYPES];
    int32_t has_eps_override;
    int32_t pad_;
    double v_kick;      /* integrator 2: magnitude of the random velocity per step */
    double coul_cut;    /* > 0: Coulomb truncated (not shifted) at coul_cut * sigma_ab */
} or_params_t;

/* External forces on one particle at time t (steps iv and v):
 *  - interface wall (Sec. 2.1: a spring whose equilibrium point lies one NP
 *    radius inside the surface; spring constant per type).  With
 *    s = |x| - (R(t) - sigma/2), a particle with s > 0 feels -k_wall s x/|x|.
 *    Reading taken (wall_on = 1): the spring acts on every particle beyond its
 *    equilibrium point, with no outer limit (the literal band (-r, r) of step
 *    iv would let particles that the moving interface outruns escape).
 *    wall_on = 2 is the band as printed: the spring acts only for
 *    -r < |x| - R < r, i.e. 0 < s < sigma.
 *  - gravity -m g z^ (Sec. 1.2, step v; buoyancy folded into g).
 *  - centrifugal m w^2 (x, y, 0) for rotation about z, or m w^2 x for the
 *    isotropic tumbling of Sec. 1.2.                                        */
void or_external_forces(const or_params_t *p, int64_t n, const double *x,
                        const int32_t *type, double t, double *F /* n*3, added */)
{
    double R = or_radius(p->R0, p->k_evap, t);
    for (int64_t i = 0; i < n; ++i) {
        int ti = type[i];
        const double *xi = x + 3 * i;
        double m = p->mass[ti];
        if (p->wall_on) {
            double r = sqrt(xi[0] * xi[0] + xi[1] * xi[1] + xi[2] * xi[2]);
            double s = r - (R - 0.5 * p->sigma[ti]);
            int in_band = p->wall_on != 2 || s < p->sigma[ti];
            if (s > 0.0 && r > 0.0 && in_band) {
                double f = -p->k_wall[ti] * s / r;
                F[3 * i + 0] += f * xi[0];
                F[3 * i + 1] += f * xi[1];
                F[3 * i + 2] += f * xi[2];
            }
        }
        F[3 * i + 2] += -m * p->g;
        double w2 = p->omega * p->omega;
        if (p->rot_mode == 1) {
            F[3 * i + 0] += m * w2 * xi[0];
            F[3 * i + 1] += m * w2 * xi[1];
        } else if (p->rot_mode == 2) {
            F[3 * i + 0] += m * w2 * xi[0];
            F[3 * i + 1] += m * w2 * xi[1];
            F[3 * i + 2] += m * w2 * xi[2];
        }
    }
}

/* Total force at (x, t): pair forces of every particle plus external ones.  */
void or_total_forces(const or_params_t *p, int64_t n, const double *x,
                     const int32_t *type, double t, double *F)
{
    double sig_ab[OR_MAX_TYPES * OR_MAX_TYPES], eps_ab[OR_MAX_TYPES * OR_MAX_TYPES],
        rc_ab[OR_MAX_TYPES * OR_MAX_TYPES];
    or_mix_tables(p->n_types, p->sigma, p->eps,
                  p->has_eps_override ? p->eps_override : NULL, p->lj_cut, sig_ab,
                  eps_ab, rc_ab);
    double rcc_ab[OR_MAX_TYPES * OR_MAX_TYPES];
    for (int k = 0; k < p->n_types * p->n_types; ++k)
        rcc_ab[k] = p->coul_cut * sig_ab[k];
    or_pair_forces(n, x, type, p->n_types, sig_ab, eps_ab, rc_ab,
                   p->coul_cut > 0.0 ? rcc_ab : NULL, p->charge, p->bjerrum, p->lj_on,
                   p->coul_on, n, NULL, F);
    or_external_forces(p, n, x, type, t, F);
}

/* ------------------------------------------------------------------------ */
/* Time integration, step (vi).  The paper adds a fixed-magnitude random
 * vector to the velocity and has no temperature; the reading taken here is a
 * fluctuation-dissipation-consistent Langevin thermostat so that
 * equipartition and the free-particle MSD hold:
 *   BAOAB splitting (B. Leimkuhler, C. Matthews, 2013), per step n:
 *     v += dt/2 F(x_n, t_n)/m;  x += dt/2 v;
 *     v  = c1 v + sqrt((1 - c1^2) kT/m) xi_n,  c1 = exp(-gamma dt);
 *     x += dt/2 v;  F <- F(x_{n+1}, t_{n+1});  v += dt/2 F/m.
 *   Overdamped mode (Brownian dynamics, Euler-Maruyama):
 *     x += F(x_n, t_n) dt/(m gamma) + sqrt(2 kT dt/(m gamma)) xi_n.
 *   Printed mode (integrator 2, step vi as the paper states it):
 *     v += dt (F(x_n, t_n)/m - gamma v);  v += v_kick xi_n/|xi_n|;  x += dt v.
 * xi_n are the three normals of particle i at step n, purpose 0.  In the
 * overdamped mode velocities are not a state and v is left unchanged.
 * x, v (n x 3) are updated in place from step `step0` for n_steps steps;
 * F (n x 3) receives the total force at the final positions and time.     */
void or_run(const or_params_t *p, int64_t n, double *x, double *v,
            const int32_t *type, int64_t step0, int64_t n_steps, double *F)
{
    double *xi = (double *)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    memset(F, 0, sizeof(double) * 3 * (size_t)n);
    or_total_forces(p, n, x, type, (double)step0 * p->dt, F);
    for (int64_t k = 0; k < n_steps; ++k) {
        int64_t step = step0 + k;
        double dt = p->dt;
        or_normals(p->seed, step, 0u, n, xi);
        for (int64_t i = 0; i < n; ++i) {
            int ti = type[i];
            double m = p->mass[ti], gam = p->gamma[ti];
            if (p->integrator == 0) {
                double c1 = exp(-gam * dt);
                double sd = sqrt((1.0 - c1 * c1) * p->kT / m);
                for (int d = 0; d < 3; ++d) {
                    double vi = v[3 * i + d] + 0.5 * dt * F[3 * i + d] / m;
                    double xv = x[3 * i + d] + 0.5 * dt * vi;
                    vi = c1 * vi + sd * xi[3 * i + d];
                    xv = xv + 0.5 * dt * vi;
                    v[3 * i + d] = vi;
                    x[3 * i + d] = xv;
                }
            } else if (p->integrator == 1) {
                double mob = 1.0 / (m * gam);
                double sd = sqrt(2.0 * p->kT * dt * mob);
                for (int d = 0; d < 3; ++d)
                    x[3 * i + d] += F[3 * i + d] * dt * mob + sd * xi[3 * i + d];
            } else {
                /* step (vi) as printed: the force with the drag -m gamma v
                 * changes the velocity, a random velocity of fixed magnitude
                 * v_kick along the unit vector n/|n| of this step's normals is
                 * added, and the position moves with the new velocity.     */
                const double *nrm = xi + 3 * i;
                double len = sqrt(nrm[0] * nrm[0] + nrm[1] * nrm[1] + nrm[2] * nrm[2]);
                double a = len > 0.0 ? p->v_kick / len : 0.0;
                for (int d = 0; d < 3; ++d) {
                    double vi = v[3 * i + d] + dt * (F[3 * i + d] / m - gam * v[3 * i + d]);
                    vi += a * nrm[d];
                    v[3 * i + d] = vi;
                    x[3 * i + d] += dt * vi;
                }
            }
        }
        memset(F, 0, sizeof(double) * 3 * (size_t)n);
        or_total_forces(p, n, x, type, (double)(step + 1) * p->dt, F);
        if (p->integrator == 0) {
            for (int64_t i = 0; i < n; ++i) {
                double m = p->mass[type[i]];
                for (int d = 0; d < 3; ++d)
                    v[3 * i + d] += 0.5 * p->dt * F[3 * i + d] / m;
            }
        }
    }
    free(xi);
}

/* ------------------------------------------------------------------------ */
/* Statistics (Sec. 3 post-processing).                                      */

/* Pair-distance histogram over ordered pairs i != j: bin b = floor(r/dr),
 * dr = r_max/n_bins, counted when b < n_bins.  r is computed in double as
 * sqrt(dx*dx + dy*dy + dz*dz) from double positions.  counts is int64[n_bins]. */
void or_pair_hist(int64_t n, const double *x, double r_max, int n_bins,
                  int64_t *counts)
{
    double dr = r_max / (double)n_bins;
    memset(counts, 0, sizeof(int64_t) * (size_t)n_bins);
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < n; ++j) {
            if (j == i)
                continue;
            double dx = x[3 * i + 0] - x[3 * j + 0];
            double dy = x[3 * i + 1] - x[3 * j + 1];
            double dz = x[3 * i + 2] - x[3 * j + 2];
            double r = sqrt(dx * dx + dy * dy + dz * dz);
            double b = floor(r / dr);
            if (b < (double)n_bins)
                counts[(int64_t)b] += 1;
        }
}

/* Radial distribution function of Sec. 3.2:
 *   g(r) = sum_i (psi_i(r)/N) / ((N-1) dV_r / V),
 * psi_i(r) the number of particles in the shell [r_b, r_b + dr) around i,
 * dV_r = 4 pi/3 (r_{b+1}^3 - r_b^3).  Reading taken: V is the current droplet
 * volume 4 pi R^3 / 3.                                                       */
void or_rdf(int64_t n, const double *x, double r_max, int n_bins, double R,
            int64_t *counts, double *g)
{
    or_pair_hist(n, x, r_max, n_bins, counts);
    double dr = r_max / (double)n_bins;
    const double pi = 3.14159265358979323846264338327950;
    double V = 4.0 / 3.0 * pi * R * R * R;
    for (int b = 0; b < n_bins; ++b) {
        double r0 = b * dr, r1 = (b + 1) * dr;
        double dV = 4.0 / 3.0 * pi * (r1 * r1 * r1 - r0 * r0 * r0);
        g[b] = ((double)counts[b] / (double)n) / ((double)(n - 1) * dV / V);
    }
}

/* N_surf, the number of NPs at the droplet surface (Sec. 1, where the
 * scattered intensity grows with N_surf^2): NP i counts when its centre lies in
 * the band (-r_i, r_i) about the surface of radius R, the band of Sec. 2.2
 * step (iv):  | |x_i| - R | < r_i,  r_i = sigma_{type i} / 2.               */
int64_t or_surface_count(int64_t n, const double *x, const int32_t *type, const double *sigma,
                         double R)
{
    int64_t count = 0;
    for (int64_t i = 0; i < n; ++i) {
        double r = sqrt(x[3 * i] * x[3 * i] + x[3 * i + 1] * x[3 * i + 1] +
                        x[3 * i + 2] * x[3 * i + 2]);
        if (fabs(r - R) < 0.5 * sigma[type[i]])
            ++count;
    }
    return count;
}

/* Radial concentration about the droplet centre, Sec. 3.2:
 *   C(r_o) = (psi(r_o)/N) / (dV/V),  psi = number of particles with |x| in
 * the shell [r_b, r_b + dr), dr = r_max/n_bins, V = 4 pi R^3/3.            */
void or_radial_hist(int64_t n, const double *x, double r_max, int n_bins, double R,
                    int64_t *counts, double *C)
{
    double dr = r_max / (double)n_bins;
    memset(counts, 0, sizeof(int64_t) * (size_t)n_bins);
    for (int64_t i = 0; i < n; ++i) {
        double r = sqrt(x[3 * i] * x[3 * i] + x[3 * i + 1] * x[3 * i + 1] +
                        x[3 * i + 2] * x[3 * i + 2]);
        double b = floor(r / dr);
        if (b < (double)n_bins)
            counts[(int64_t)b] += 1;
    }
    const double pi = 3.14159265358979323846264338327950;
    double V = 4.0 / 3.0 * pi * R * R * R;
    for (int b = 0; b < n_bins; ++b) {
        double r0 = b * dr, r1 = (b + 1) * dr;
        double dV = 4.0 / 3.0 * pi * (r1 * r1 * r1 - r0 * r0 * r0);
        C[b] = ((double)counts[b] / (double)n) / (dV / V);
    }
}

/* Radius of gyration about the centre of mass (Eqs. Rg and r0 of Sec. 3.1),
 * each NP weighted equally, and the fractal dimension solved from the
 * fractal equation N = k_f (2 R_g / d)^D_f (Eq. N), k_f = 1.593:
 *   D_f = ln(N / k_f) / ln(2 R_g / d).
 * d is the NP diameter; for several sizes the number-mean diameter is used
 * (reading taken: the paper's equation assumes identical NPs).            */
void or_rg(int64_t n, const double *x, double d_mean, double k_f, double *Rg,
           double *Df, double *r0)
{
    double c[3] = {0.0, 0.0, 0.0};
    for (int64_t i = 0; i < n; ++i)
        for (int d = 0; d < 3; ++d)
            c[d] += x[3 * i + d];
    for (int d = 0; d < 3; ++d)
        c[d] /= (double)n;
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i)
        for (int d = 0; d < 3; ++d) {
            double e = c[d] - x[3 * i + d];
            s += e * e;
        }
    double rg = sqrt(s / (double)n);
    *Rg = rg;
    *Df = log((double)n / k_f) / log(2.0 * rg / d_mean);
    if (r0) {
        r0[0] = c[0];
        r0[1] = c[1];
        r0[2] = c[2];
    }
}

/* Box counting (the box-counting estimate of the mass fractal dimension):
 * origin o = componentwise minimum of the NP centres; for box edge
 * eps_k = d 2^k, k = 0..n_scales-1, N_box(eps_k) is the number of distinct
 * integer triples floor((x - o)/eps_k) that hold at least one centre.
 * nbox is int64[n_scales].  Counting distinct triples is done by sorting
 * the triples, the plainest exact method.                                   */
static int or_cmp_triple(const void *a, const void *b)
{
    const int64_t *u = (const int64_t *)a, *w = (const int64_t *)b;
    for (int d = 0; d < 3; ++d) {
        if (u[d] < w[d])
            return -1;
        if (u[d] > w[d])
            return 1;
    }
    return 0;
}

void or_boxcount(int64_t n, const double *x, double d, int n_scales, int64_t *nbox)
{
    double o[3] = {x[0], x[1], x[2]};
    for (int64_t i = 1; i < n; ++i)
        for (int k = 0; k < 3; ++k)
            if (x[3 * i + k] < o[k])
                o[k] = x[3 * i + k];
    int64_t *t = (int64_t *)malloc(sizeof(int64_t) * 3 * (size_t)(n > 0 ? n : 1));
    for (int s = 0; s < n_scales; ++s) {
        double eps = d * ldexp(1.0, s);
        for (int64_t i = 0; i < n; ++i)
            for (int k = 0; k < 3; ++k)
                t[3 * i + k] = (int64_t)floor((x[3 * i + k] - o[k]) / eps);
        qsort(t, (size_t)n, sizeof(int64_t) * 3, or_cmp_triple);
        int64_t distinct = n > 0 ? 1 : 0;
        for (int64_t i = 1; i < n; ++i)
            if (or_cmp_triple(t + 3 * i, t + 3 * (i - 1)) != 0)
                ++distinct;
        nbox[s] = distinct;
    }
    free(t);
}

/* Least-squares slope of y on x over m points (ordinary least squares).     */
double or_lsq_slope(int m, const double *xs, const double *ys)
{
    double mx = 0.0, my = 0.0;
    for (int k = 0; k < m; ++k) {
        mx += xs[k];
        my += ys[k];
    }
    mx /= m;
    my /= m;
    double sxy = 0.0, sxx = 0.0;
    for (int k = 0; k < m; ++k) {
        sxy += (xs[k] - mx) * (ys[k] - my);
        sxx += (xs[k] - mx) * (xs[k] - mx);
    }
    return sxy / sxx;
}

/* Box-counting fractal dimension.  Scales eps_k = d 2^k for k = 0, 1, ...
 * while eps_k <= 2 R_g (at most max_scales); D_f is minus the least-squares
 * slope of ln N_box against ln eps over k >= 1 (k = 0 is left out: at the
 * NP diameter nearly every NP has a box of its own and the count saturates).
 * Returns the number of scales counted (written to nbox); D_f is NaN when
 * fewer than two scales enter the fit.                                      */
int or_boxcount_df(int64_t n, const double *x, double d, double Rg, int max_scales,
                   int64_t *nbox, double *Df)
{
    int ns = 0;
    while (ns < max_scales && d * ldexp(1.0, ns) <= 2.0 * Rg)
        ++ns;
    or_boxcount(n, x, d, ns, nbox);
    if (ns - 1 < 2) {
        *Df = NAN;
        return ns;
    }
    double xs[64], ys[64];
    int m = 0;
    for (int k = 1; k < ns && m < 64; ++k, ++m) {
        xs[m] = log(d * ldexp(1.0, k));
        ys[m] = log((double)nbox[k]);
    }
    *Df = -or_lsq_slope(m, xs, ys);
    return ns;
}
