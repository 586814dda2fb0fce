/*
 * mpr_oracle.c -- plain FP64 CPU oracle of the MPR gap-filling method.
 *
 * TEST INFRASTRUCTURE ONLY: called by the tests, the smoke check and the benchmark's CPU-baseline
 * leg, never by the CUDA library. No blocking, fusion or reordering: every step is written in the
 * order the method states it, one site at a time, so that it can be read against the paper.
 *
 * Sources of each step:
 *   Hamiltonian H = -J sum_<ij> cos[q(phi_i - phi_j)], J = 1 ........ Eq. 2 (Sec. 2)
 *   conditional MC, only prediction spins move; hybrid algorithm;
 *   temperature as the single inferred parameter; averaging of
 *   equilibrium configurations into predictions ...................... Sec. 2
 *   specific energy e = <H>/L^2 ....................................... Sec. 2
 *   counter-based random numbers: Philox-4x32-10 ...................... Salmon et al., SC'11
 * Points on which the paper is silent (the mapping formula, open boundaries, the Metropolis
 * proposal, the over-relaxation reflection for q < 1, the tuning procedure; and the options built
 * on them: energy-slope equilibration, bounded proposals with an adapted width, tuning by heating
 * and by the unconditional energy curve) follow the readings recorded in the design notes; each
 * is restated at the function that uses it.
 */
#include "mpr_oracle.h"

#include <math.h>
#include <stddef.h>
#include <stdlib.h>

static const double TWO_PI = 6.283185307179586476925286766559;

/* ------------------------------------------------------------------------------------------ */
/* Philox (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11).  */
/* Four W-bit words per counter. One round multiplies words 0 and 2 by the two round           */
/* multipliers, keeping both halves of each double-width product; the high halves are mixed     */
/* with words 1 and 3 and the two key words, and the words are permuted. Between rounds the     */
/* key words advance by the two Weyl constants (golden ratio and sqrt(3) - 1).                  */
/* ------------------------------------------------------------------------------------------ */

static void mulhilo(int W, uint64_t a, uint64_t b, uint64_t* hi, uint64_t* lo)
{
    if (W == 32) {
        uint64_t p = (a & 0xffffffffu) * (b & 0xffffffffu);
        *hi = p >> 32;
        *lo = p & 0xffffffffu;
    } else {
        unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
        *hi = (uint64_t)(p >> 64);
        *lo = (uint64_t)p;
    }
}

void mpro_philox(int W, int rounds, const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4])
{
    uint64_t M0, M1, C0, C1, mask;
    if (W == 32) {
        M0 = 0xD2511F53u; M1 = 0xCD9E8D57u;
        C0 = 0x9E3779B9u; C1 = 0xBB67AE85u;
        mask = 0xffffffffu;
    } else {
        M0 = 0xD2E7470EE14C6C93ull; M1 = 0xCA5A826395121157ull;
        C0 = 0x9E3779B97F4A7C15ull; C1 = 0xBB67AE8584CAA73Bull;
        mask = ~0ull;
    }
    uint64_t x0 = ctr[0] & mask, x1 = ctr[1] & mask, x2 = ctr[2] & mask, x3 = ctr[3] & mask;
    uint64_t k0 = key[0] & mask, k1 = key[1] & mask;
    for (int r = 0; r < rounds; ++r) {
        if (r > 0) {
            k0 = (k0 + C0) & mask;
            k1 = (k1 + C1) & mask;
        }
        uint64_t hi0, lo0, hi1, lo1;
        mulhilo(W, M0, x0, &hi0, &lo0);
        mulhilo(W, M1, x2, &hi1, &lo1);
        uint64_t y0 = hi1 ^ x1 ^ k0;
        uint64_t y1 = lo1;
        uint64_t y2 = hi0 ^ x3 ^ k1;
        uint64_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

void mpro_philox_n(int W, int rounds, int n, const uint64_t* ctr, const uint64_t key[2],
                   uint64_t* out)
{
    for (int i = 0; i < n; ++i) mpro_philox(W, rounds, ctr + 4 * (size_t)i, key, out + 4 * (size_t)i);
}

/* Counter layout (one Philox-4x32-10 call serves two same-colour sites of a row):
 *   ctr = (x >> 2, y, sweep, problem << 8 | tag << 1 | colour), key = (seed_lo, seed_hi);
 *   the site takes words 2t and 2t+1 with t = (x >> 1) & 1: the first word drives the
 *   Metropolis proposal (or the initial angle), the second the acceptance test. */
void mpro_site_words(const mpro_cfg* cfg, int x, int y, uint32_t sweep, int tag,
                     uint32_t* w_prop, uint32_t* w_acc)
{
    int c = (x + y) & 1;
    int t = (x >> 1) & 1;
    uint64_t ctr[4], key[2], out[4];
    ctr[0] = (uint64_t)(x >> 2);
    ctr[1] = (uint64_t)y;
    ctr[2] = (uint64_t)sweep;
    ctr[3] = ((uint64_t)cfg->problem << 8) | ((uint64_t)tag << 1) | (uint64_t)c;
    key[0] = cfg->seed & 0xffffffffu;
    key[1] = cfg->seed >> 32;
    mpro_philox(32, 10, ctr, key, out);
    *w_prop = (uint32_t)out[2 * t];
    *w_acc = (uint32_t)out[2 * t + 1];
}

/* Uniform in [0, 1): all 32 bits for the FP64 function setting, the top 23 bits for FP32. */
double mpro_uniform(const mpro_cfg* cfg, uint32_t w)
{
    if (cfg->ubits == 32)
        return (double)w * (1.0 / 4294967296.0);
    return (double)(w >> 9) * (1.0 / 8388608.0);
}

/* The two Metropolis uniforms of site (x, y) at a sweep: proposal and acceptance, in [0, 1).
 *
 * FP64 function setting (ubits = 32): the site's two words from mpro_site_words (tag 0), all 32
 * bits of each.
 *
 * FP32 function setting (ubits = 23): each uniform has 23 bits, so one Philox-4x32-10 call (128
 * bits) can serve more than two sites. Reading: three calls serve a group of eight same-colour
 * sites, the four half-lattice columns j = 4g .. 4g + 3 (j = x >> 1) of the two rows 2h and
 * 2h + 1; call m (m = 0, 1, 2) has counter (g, h, sweep, problem << 8 | m << 2 | colour) and
 * key = seed, and gives the words W[4m] .. W[4m + 3]. In the group's first row, the one with
 * y + colour even, site i = j & 3 takes the top 23 bits of W[2i] for its proposal and of
 * W[2i + 1] for its acceptance. In the second row site i takes the top 23 bits of W[8 + i] for
 * its proposal, and for its acceptance the 23 bits
 *     b[3i] | b[3i + 1] << 8 | (b[3i + 2] & 127) << 16,   b[k] = W[k] & 255,
 * built from the low bytes, which the top-23-bit fields never touch. No bit of the 384 serves two
 * uniforms. */
void mpro_site_uniforms(const mpro_cfg* cfg, int x, int y, uint32_t sweep, double* u_prop,
                        double* u_acc)
{
    if (cfg->ubits == 32) {
        uint32_t wp, wa;
        mpro_site_words(cfg, x, y, sweep, 0, &wp, &wa);
        *u_prop = mpro_uniform(cfg, wp);
        *u_acc = mpro_uniform(cfg, wa);
        return;
    }
    const int c = (x + y) & 1;
    const int j = x >> 1;
    const int g = j >> 2, i = j & 3;
    const int second_row = (y + c) & 1;
    uint64_t W[12], key[2];
    key[0] = cfg->seed & 0xffffffffu;
    key[1] = cfg->seed >> 32;
    for (int m = 0; m < 3; ++m) {
        uint64_t ctr[4];
        ctr[0] = (uint64_t)g;
        ctr[1] = (uint64_t)(y >> 1);
        ctr[2] = (uint64_t)sweep;
        ctr[3] = ((uint64_t)cfg->problem << 8) | ((uint64_t)m << 2) | (uint64_t)c;
        mpro_philox(32, 10, ctr, key, W + 4 * m);
    }
    uint64_t mp, ma;
    if (!second_row) {
        mp = W[2 * i] >> 9;
        ma = W[2 * i + 1] >> 9;
    } else {
        mp = W[8 + i] >> 9;
        ma = (W[3 * i] & 255u) | ((W[3 * i + 1] & 255u) << 8) | ((W[3 * i + 2] & 127u) << 16);
    }
    *u_prop = (double)mp * (1.0 / 8388608.0);
    *u_acc = (double)ma * (1.0 / 8388608.0);
}

/* ------------------------------------------------------------------------------------------ */
/* Data -> spins (Sec. 2: the measured data are mapped onto spins).                            */
/* Reading: phi = 2*pi*(z - zmin)/(zmax - zmin), zmin/zmax over the measured values only.      */
/* ------------------------------------------------------------------------------------------ */

int mpro_map(int N, const double* z, const uint8_t* mask, double* phi, double* zmin, double* zmax)
{
    int n_meas = 0;
    double lo = INFINITY, hi = -INFINITY;
    for (int s = 0; s < N; ++s) {
        if (!mask[s]) continue;
        ++n_meas;
        if (z[s] < lo) lo = z[s];
        if (z[s] > hi) hi = z[s];
    }
    if (n_meas < 2 || !(hi > lo)) return 2;
    for (int s = 0; s < N; ++s) {
        if (mask[s]) {
            double t = (z[s] - lo) / (hi - lo);
            phi[s] = TWO_PI * t;
        } else {
            phi[s] = 0.0;
        }
    }
    *zmin = lo;
    *zmax = hi;
    return 0;
}

/* Reading: prediction spins start from independent uniform angles ("hot" start). */
void mpro_init(const mpro_cfg* cfg, const uint8_t* mask, double* phi)
{
    for (int y = 0; y < cfg->Ly; ++y)
        for (int x = 0; x < cfg->Lx; ++x) {
            int s = y * cfg->Lx + x;
            if (mask[s]) continue;
            uint32_t wp, wa;
            mpro_site_words(cfg, x, y, 0u, 1, &wp, &wa);
            phi[s] = TWO_PI * mpro_uniform(cfg, wp);
        }
}

/* ------------------------------------------------------------------------------------------ */
/* Hybrid move of one prediction site (Sec. 2: conditional MC with the hybrid algorithm).      */
/* ------------------------------------------------------------------------------------------ */

/* Local field of site (x, y): h = sum over its neighbours j of (cos q phi_j, sin q phi_j), so that
 * the part of Eq. 2 that involves phi_s is E_s(phi) = -(hx cos q phi + hy sin q phi). */
static void local_field(const mpro_cfg* cfg, const double* phi, int x, int y, double* hx, double* hy)
{
    const int Lx = cfg->Lx, Ly = cfg->Ly;
    const double q = cfg->q;
    double sx = 0.0, sy = 0.0;
    if (x > 0)      { double a = q * phi[y * Lx + x - 1];   sx += cos(a); sy += sin(a); }
    if (x < Lx - 1) { double a = q * phi[y * Lx + x + 1];   sx += cos(a); sy += sin(a); }
    if (y > 0)      { double a = q * phi[(y - 1) * Lx + x]; sx += cos(a); sy += sin(a); }
    if (y < Ly - 1) { double a = q * phi[(y + 1) * Lx + x]; sx += cos(a); sy += sin(a); }
    *hx = sx;
    *hy = sy;
}

static double site_energy(double q, double hx, double hy, double f)
{
    return -(hx * cos(q * f) + hy * sin(q * f));
}

/* Over-relaxation. Reading: reflect q*phi about the direction theta of the local field,
 * psi = 2*theta - q*phi, which keeps E_s = -|h| cos(q*phi - theta) unchanged; take the
 * representative r of psi modulo 2*pi in [0, 2*pi) and accept it when r <= 2*pi*q, i.e. when the
 * new angle r/q lies in [0, 2*pi]; otherwise (and when h = 0) the angle stays. With q = 1 every r
 * is accepted and the move is the planar-rotator reflection phi -> 2*theta - phi (mod 2*pi). */
double mpro_overrelax(double q, double hx, double hy, double f, double* or_margin)
{
    if (hx == 0.0 && hy == 0.0) {
        if (or_margin) *or_margin = INFINITY;
        return f;
    }
    double theta = atan2(hy, hx);
    double psi = 2.0 * theta - q * f;
    double r = psi - TWO_PI * floor(psi / TWO_PI);
    double width = TWO_PI * q;
    if (or_margin) {
        double m = r < TWO_PI - r ? r : TWO_PI - r;
        double d = fabs(r - width);
        *or_margin = m < d ? m : d;
    }
    if (r <= width) return r / q;
    return f;
}

double mpro_update_site(const mpro_cfg* cfg, const double* phi, const uint8_t* mask, int x, int y,
                        double T, uint32_t sweep, double* met_margin, double* or_margin,
                        int* accepted)
{
    const double q = cfg->q;
    const int s = y * cfg->Lx + x;
    (void)mask;
    double hx, hy;
    local_field(cfg, phi, x, y, &hx, &hy);

    /* Metropolis. Reading: the proposal is an independent uniform angle on [0, 2*pi); the
     * move is accepted when dE <= 0 or u < exp(-dE/T) (strict). Option (cfg->width > 0): a
     * proposal f + w*(2u - 1) uniform on the segment of half-width w around f (symmetric, so the
     * same acceptance rule holds), rejected when it leaves the state space [0, 2*pi). */
    double u_prop, u_acc;
    mpro_site_uniforms(cfg, x, y, sweep, &u_prop, &u_acc);
    double f = phi[s];
    const int bounded = cfg->width > 0.0;
    double f_prop = bounded ? f + cfg->width * (2.0 * u_prop - 1.0) : TWO_PI * u_prop;
    const int inside = !bounded || (f_prop >= 0.0 && f_prop < TWO_PI);
    double dE = site_energy(q, hx, hy, f_prop) - site_energy(q, hx, hy, f);
    double p_acc = (dE <= 0.0) ? 1.0 : exp(-dE / T);
    int accept = inside && ((dE <= 0.0) || (u_acc < p_acc));
    if (met_margin) {
        *met_margin = fabs(u_acc - p_acc);
        if (bounded) {
            const double edge = fmin(fabs(f_prop), fabs(TWO_PI - f_prop));
            if (edge < *met_margin) *met_margin = edge;
        }
    }
    if (accepted) *accepted = accept;
    double f1 = accept ? f_prop : f;

    return mpro_overrelax(q, hx, hy, f1, or_margin);
}

int64_t mpro_half_sweep(const mpro_cfg* cfg, double* phi, const uint8_t* mask, double T,
                        uint32_t sweep, int colour, double* met_margin, double* or_margin)
{
    const int Lx = cfg->Lx, Ly = cfg->Ly;
    int64_t n_acc = 0;
    /* A site reads only neighbours of the other colour, so the sites of one colour can be
     * overwritten in place. */
    for (int y = 0; y < Ly; ++y)
        for (int x = 0; x < Lx; ++x) {
            if (((x + y) & 1) != colour) continue;
            int s = y * Lx + x;
            if (mask[s]) continue;
            double mm, om;
            int acc;
            double f = mpro_update_site(cfg, phi, mask, x, y, T, sweep, &mm, &om, &acc);
            phi[s] = f;
            n_acc += acc;
            if (met_margin) met_margin[s] = mm;
            if (or_margin) or_margin[s] = om;
        }
    return n_acc;
}

int64_t mpro_sweep(const mpro_cfg* cfg, double* phi, const uint8_t* mask, double T, uint32_t sweep,
                   double* met_margin, double* or_margin)
{
    const int N = cfg->Lx * cfg->Ly;
    if (met_margin)
        for (int s = 0; s < N; ++s) met_margin[s] = INFINITY;
    if (or_margin)
        for (int s = 0; s < N; ++s) or_margin[s] = INFINITY;
    /* red sites first, then black */
    int64_t n = mpro_half_sweep(cfg, phi, mask, T, sweep, 0, met_margin, or_margin);
    return n + mpro_half_sweep(cfg, phi, mask, T, sweep, 1, met_margin, or_margin);
}

/* ------------------------------------------------------------------------------------------ */
/* Energies (Eq. 2; Sec. 2 defines the specific energy e = <H>/L^2). Reading: the tuning      */
/* compares energies per bond, e_b = H / N_b, N_b = Lx(Ly-1) + Ly(Lx-1).                       */
/* ------------------------------------------------------------------------------------------ */

double mpro_energy_bond(const mpro_cfg* cfg, const double* phi)
{
    const int Lx = cfg->Lx, Ly = cfg->Ly;
    const double q = cfg->q;
    double sum = 0.0;
    long nb = 0;
    for (int y = 0; y < Ly; ++y)
        for (int x = 0; x < Lx; ++x) {
            int s = y * Lx + x;
            if (x + 1 < Lx) { sum += cos(q * (phi[s] - phi[s + 1]));  ++nb; }
            if (y + 1 < Ly) { sum += cos(q * (phi[s] - phi[s + Lx])); ++nb; }
        }
    return -sum / (double)nb;
}

int mpro_energy_sample(const mpro_cfg* cfg, const double* phi, const uint8_t* mask,
                       double* e_s, int64_t* n_pairs)
{
    const int Lx = cfg->Lx, Ly = cfg->Ly;
    const double q = cfg->q;
    double sum = 0.0;
    int64_t n = 0;
    for (int y = 0; y < Ly; ++y)
        for (int x = 0; x < Lx; ++x) {
            int s = y * Lx + x;
            if (!mask[s]) continue;
            if (x + 1 < Lx && mask[s + 1])  { sum += cos(q * (phi[s] - phi[s + 1]));  ++n; }
            if (y + 1 < Ly && mask[s + Lx]) { sum += cos(q * (phi[s] - phi[s + Lx])); ++n; }
        }
    *n_pairs = n;
    if (n == 0) return 3;
    *e_s = -sum / (double)n;
    return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* Equilibration and sampling (Sec. 2: averaging over configurations in equilibrium).          */
/* Reading: the arithmetic mean of phi over every sampling sweep.                              */
/* ------------------------------------------------------------------------------------------ */

void mpro_run(const mpro_cfg* cfg, double* phi, const uint8_t* mask, double T, uint32_t sweep0,
              int nsweeps, double* acc, double* energies)
{
    const int N = cfg->Lx * cfg->Ly;
    for (int k = 0; k < nsweeps; ++k) {
        mpro_sweep(cfg, phi, mask, T, sweep0 + (uint32_t)k, NULL, NULL);
        if (energies) energies[k] = mpro_energy_bond(cfg, phi);
        if (acc)
            for (int s = 0; s < N; ++s)
                if (!mask[s]) acc[s] += phi[s];
    }
}

/* ------------------------------------------------------------------------------------------ */
/* Bounded proposals with an adapted width. A reading, not the paper's (its proposal is not     */
/* stated): after every sweep the width follows the sweep's acceptance fraction a of Metropolis */
/* proposals toward a target, w <- w * exp(a - target), kept in [1e-3, 2*pi]. Adapting makes    */
/* the chain time-inhomogeneous, so it belongs to equilibration; the width is then held fixed.  */
/* ------------------------------------------------------------------------------------------ */

void mpro_run_adapt(mpro_cfg* cfg, double* phi, const uint8_t* mask, double T, uint32_t sweep0,
                    int nsweeps, double target, double* widths)
{
    const int N = cfg->Lx * cfg->Ly;
    int64_t n_pred = 0;
    for (int s = 0; s < N; ++s) n_pred += mask[s] == 0;
    for (int k = 0; k < nsweeps; ++k) {
        if (widths) widths[k] = cfg->width;
        const int64_t n_acc = mpro_sweep(cfg, phi, mask, T, sweep0 + (uint32_t)k, NULL, NULL);
        const double a = n_pred > 0 ? (double)n_acc / (double)n_pred : target;
        double w = cfg->width * exp(a - target);
        if (w < 1e-3) w = 1e-3;
        if (w > TWO_PI) w = TWO_PI;
        cfg->width = w;
    }
}

/* ------------------------------------------------------------------------------------------ */
/* Equilibration with an energy-slope stop. A reading, not the paper's: Sec. 2 averages          */
/* configurations "in equilibrium" without saying how equilibrium is recognised. The energy of  */
/* the chain drifts while it relaxes; equilibrium is declared when two consecutive chunks of    */
/* sweeps have means that agree within z standard errors of their difference.                   */
/* ------------------------------------------------------------------------------------------ */

int mpro_equilibrate(const mpro_cfg* cfg, double* phi, const uint8_t* mask, double T,
                     uint32_t* sweep, int chunk, int max_sweeps, double z)
{
    if (chunk < 2) return 0;
    double* e = (double*)malloc(sizeof(double) * (size_t)chunk);
    double prev_mean = 0.0, prev_var = 0.0;
    int done = 0;
    for (int k = 0; done + chunk <= max_sweeps; ++k) {
        mpro_run(cfg, phi, mask, T, *sweep, chunk, NULL, e);
        *sweep += (uint32_t)chunk;
        done += chunk;
        double mean = 0.0;
        for (int i = 0; i < chunk; ++i) mean += e[i];
        mean /= (double)chunk;
        double var = 0.0;
        for (int i = 0; i < chunk; ++i) var += (e[i] - mean) * (e[i] - mean);
        var /= (double)(chunk - 1);
        if (k > 0 && fabs(mean - prev_mean) <= z * sqrt((var + prev_var) / (double)chunk)) break;
        prev_mean = mean;
        prev_var = var;
    }
    free(e);
    return done;
}

/* ------------------------------------------------------------------------------------------ */
/* Temperature tuning (Sec. 2: the temperature is the only parameter and is inferred from the   */
/* data). Reading: find T whose equilibrium bond energy of the conditional lattice equals the   */
/* sample's, by bisection in log T; e_b(T) is non-decreasing because d<H>/dT = Var(H)/T^2.      */
/* Each probe continues the chain of the previous one.                                          */
/* ------------------------------------------------------------------------------------------ */

static double probe(const mpro_cfg* cfg, double* phi, const uint8_t* mask, uint32_t* sweep,
                    const mpro_tune_cfg* t, double T)
{
    mpro_run(cfg, phi, mask, T, *sweep, t->n_eq, NULL, NULL);
    *sweep += (uint32_t)t->n_eq;
    double* e = (double*)malloc(sizeof(double) * (size_t)(t->n_meas > 0 ? t->n_meas : 1));
    mpro_run(cfg, phi, mask, T, *sweep, t->n_meas, NULL, e);
    *sweep += (uint32_t)t->n_meas;
    double sum = 0.0;
    for (int k = 0; k < t->n_meas; ++k) sum += e[k];
    free(e);
    return sum / (double)t->n_meas;
}

int mpro_tune(const mpro_cfg* cfg, double* phi, const uint8_t* mask, double e_s, uint32_t* sweep,
              const mpro_tune_cfg* t, double* T_out, double* trace_T, double* trace_e,
              int* n_probes)
{
    const double tol = t->rel_tol * fabs(e_s);
    double lo = log(t->T_lo), hi = log(t->T_hi);
    int np = 0;
    int status = 0;
    double T, e;

    T = t->T_lo;
    e = probe(cfg, phi, mask, sweep, t, T);
    if (trace_T) { trace_T[np] = T; trace_e[np] = e; }
    ++np;
    if (fabs(e - e_s) <= tol || e_s < e) { *T_out = T; goto done; }

    T = t->T_hi;
    e = probe(cfg, phi, mask, sweep, t, T);
    if (trace_T) { trace_T[np] = T; trace_e[np] = e; }
    ++np;
    if (fabs(e - e_s) <= tol) { *T_out = T; goto done; }
    if (e_s > e) { *T_out = T; status = 4; goto done; }

    for (;;) {
        if (np >= t->max_probes) { *T_out = exp(0.5 * (lo + hi)); status = 4; goto done; }
        double mid = 0.5 * (lo + hi);
        T = exp(mid);
        e = probe(cfg, phi, mask, sweep, t, T);
        if (trace_T) { trace_T[np] = T; trace_e[np] = e; }
        ++np;
        if (fabs(e - e_s) <= tol) { *T_out = T; goto done; }
        if (e < e_s) lo = mid; else hi = mid;
        if (hi - lo < log(t->ratio_tol)) { *T_out = exp(0.5 * (lo + hi)); goto done; }
    }
done:
    if (n_probes) *n_probes = np;
    return status;
}

/* ------------------------------------------------------------------------------------------ */
/* Alternative tunings. Readings, not the paper's (Sec. 2 says only that the temperature is     */
/* inferred from the incomplete data).                                                          */
/* ------------------------------------------------------------------------------------------ */

/* Heating: probe T_lo, then raise T by `factor` per probe (the chain carries over, so each probe
 * starts from the equilibrium of the cooler one) until e_b(T) reaches e_s; the last two
 * temperatures bracket the crossing, which bisection in log T then refines with the stopping
 * rules of mpro_tune. No crossing up to T_hi: status 4 with T = T_hi. */
int mpro_tune_heating(const mpro_cfg* cfg, double* phi, const uint8_t* mask, double e_s,
                      uint32_t* sweep, const mpro_tune_cfg* t, double factor, double* T_out,
                      double* trace_T, double* trace_e, int* n_probes)
{
    const double tol = t->rel_tol * fabs(e_s);
    int np = 0;
    int status = 0;
    double T = t->T_lo, e, lo, hi;

    e = probe(cfg, phi, mask, sweep, t, T);
    if (trace_T) { trace_T[np] = T; trace_e[np] = e; }
    ++np;
    if (fabs(e - e_s) <= tol || e_s < e) { *T_out = T; goto done; }

    /* heat until the energy passes e_s */
    for (;;) {
        if (T >= t->T_hi) { *T_out = T; status = 4; goto done; }
        if (np >= t->max_probes) { *T_out = T; status = 4; goto done; }
        double Tn = T * factor;
        if (Tn > t->T_hi) Tn = t->T_hi;
        e = probe(cfg, phi, mask, sweep, t, Tn);
        if (trace_T) { trace_T[np] = Tn; trace_e[np] = e; }
        ++np;
        if (fabs(e - e_s) <= tol) { *T_out = Tn; goto done; }
        if (e > e_s) { lo = log(T); hi = log(Tn); break; }
        T = Tn;
    }

    /* bisection inside the bracket */
    for (;;) {
        if (hi - lo < log(t->ratio_tol)) { *T_out = exp(0.5 * (lo + hi)); goto done; }
        if (np >= t->max_probes) { *T_out = exp(0.5 * (lo + hi)); status = 4; goto done; }
        double mid = 0.5 * (lo + hi);
        T = exp(mid);
        e = probe(cfg, phi, mask, sweep, t, T);
        if (trace_T) { trace_T[np] = T; trace_e[np] = e; }
        ++np;
        if (fabs(e - e_s) <= tol) { *T_out = T; goto done; }
        if (e < e_s) lo = mid; else hi = mid;
    }
done:
    if (n_probes) *n_probes = np;
    return status;
}

/* Energy curve of the unconditional model: every site free, uniform start (mpro_init), then for
 * each temperature in turn n_eq sweeps and the mean e_b over n_meas sweeps, the chain carrying
 * over from one temperature to the next. The sweep counter starts at *sweep and advances. */
void mpro_energy_curve(const mpro_cfg* cfg, const double* T, int n, const mpro_tune_cfg* t,
                       uint32_t* sweep, double* e_out)
{
    const int N = cfg->Lx * cfg->Ly;
    uint8_t* mask = (uint8_t*)calloc((size_t)N, 1);
    double* phi = (double*)calloc((size_t)N, sizeof(double));
    mpro_init(cfg, mask, phi);
    for (int i = 0; i < n; ++i) e_out[i] = probe(cfg, phi, mask, sweep, t, T[i]);
    free(phi);
    free(mask);
}

/* Inverse of a tabulated curve e(T), T ascending: the temperature where the piecewise-linear
 * interpolant in log T first reaches e_s. e_s at or below e[0]: T[0]; above every e[i]: T[n-1]
 * with status 4. */
int mpro_invert_curve(const double* T, const double* e, int n, double e_s, double* T_out)
{
    if (e_s <= e[0]) { *T_out = T[0]; return 0; }
    for (int i = 1; i < n; ++i) {
        if (e[i] >= e_s) {   /* here e[i-1] < e_s <= e[i] */
            const double f = (e_s - e[i - 1]) / (e[i] - e[i - 1]);
            *T_out = exp(log(T[i - 1]) + f * (log(T[i]) - log(T[i - 1])));
            return 0;
        }
    }
    *T_out = T[n - 1];
    return 4;
}

/* ------------------------------------------------------------------------------------------ */
/* Prediction: mean angle mapped back to the data scale (inverse of the mapping above).        */
/* ------------------------------------------------------------------------------------------ */

void mpro_predict(int N, const double* acc, int nsamples, const double* z, const uint8_t* mask,
                  double zmin, double zmax, double* zhat)
{
    for (int s = 0; s < N; ++s) {
        if (mask[s]) {
            zhat[s] = z[s];
        } else {
            double phibar = acc[s] / (double)nsamples;
            zhat[s] = zmin + (zmax - zmin) * (phibar / TWO_PI);
        }
    }
}
