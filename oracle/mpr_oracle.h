/*
 * mpr_oracle.h -- plain FP64 CPU oracle of the modified planar rotator (MPR) gap-filling
 * method (Lach, Borovsky, Zukovic, "Numerical Precision Effects on GPU Simulation of Massive
 * Spatial Data, Based on the Modified Planar Rotator Model", Sec. 2, Eq. 2).
 *
 * TEST INFRASTRUCTURE ONLY. This oracle exists to check the CUDA library against the method's
 * definition. Only the tests, the smoke check and the CPU-baseline leg of the benchmark may call
 * it. It shares no code with the CUDA path and the CUDA path never calls it.
 *
 * Every function works on one problem held as plain row-major arrays:
 *   site s = y*Lx + x, 0 <= x < Lx, 0 <= y < Ly, colour c(s) = (x + y) & 1 (0 = red),
 *   phi[s]  spin angle in [0, 2*pi] (FP64),
 *   mask[s] 1 = measured (frozen), 0 = prediction site,
 *   open boundaries: neighbours (x+-1, y), (x, y+-1) inside the grid only.
 * Return codes follow the library's status codes (0 ok, 2 degenerate data, 3 no measured pair,
 * 4 tuning did not converge).
 */
#ifndef MPR_ORACLE_H
#define MPR_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int Lx, Ly;          /* lattice size */
    double q;            /* exponent of Eq. 2, q in (0, 1/2]; q = 1 is the planar rotator of Eq. 1 */
    uint64_t seed;       /* Philox key (low word, high word) */
    uint32_t problem;    /* problem id, part of the Philox counter */
    int ubits;           /* uniform resolution: 32 -> u = w*2^-32, 23 -> 23-bit uniforms
                            (initial angles: (w>>9)*2^-23; Metropolis: mpro_site_uniforms) */
    double width;        /* Metropolis proposal: 0 -> uniform angle on [0, 2*pi); w > 0 ->
                            phi + w*(2u - 1), rejected outside [0, 2*pi) */
} mpro_cfg;

typedef struct {
    int n_eq;            /* sweeps to equilibrate at each probe temperature */
    int n_meas;          /* sweeps whose bond energy is averaged at each probe */
    double T_lo, T_hi;   /* bracket of the reduced temperature */
    double rel_tol;      /* stop when |e_b - e_s| <= rel_tol * |e_s| */
    double ratio_tol;    /* or when T_hi / T_lo < ratio_tol */
    int max_probes;
} mpro_tune_cfg;

/* Philox-NxW-R of Salmon et al. (SC'11), N = 4, W = 32 or 64. Counter, key and output are held
 * in 64-bit words; with W = 32 only the low 32 bits are used and produced. */
void mpro_philox(int W, int rounds, const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]);
/* The block function on n counters (ctr and out: n x 4 words, row-major). */
void mpro_philox_n(int W, int rounds, int n, const uint64_t* ctr, const uint64_t key[2],
                   uint64_t* out);

/* The two 32-bit random words of site (x, y) at the given sweep and tag (0 Metropolis, 1 init). */
void mpro_site_words(const mpro_cfg* cfg, int x, int y, uint32_t sweep, int tag,
                     uint32_t* w_prop, uint32_t* w_acc);
double mpro_uniform(const mpro_cfg* cfg, uint32_t w);
/* The Metropolis uniforms (proposal, acceptance) of site (x, y) at a sweep: from the site's two
 * words with ubits = 32; with ubits = 23 from three Philox calls per group of eight same-colour
 * sites (four half-lattice columns x two rows), 23 bits each (layout in mpr_oracle.c). */
void mpro_site_uniforms(const mpro_cfg* cfg, int x, int y, uint32_t sweep, double* u_prop,
                        double* u_acc);

/* Data -> spin mapping over the measured values; returns 2 on < 2 measured sites or zmax == zmin. */
int mpro_map(int N, const double* z, const uint8_t* mask, double* phi, double* zmin, double* zmax);
/* Initial angles of the prediction sites: phi = 2*pi*u, u from the init stream at sweep 0. */
void mpro_init(const mpro_cfg* cfg, const uint8_t* mask, double* phi);

/* Energy-conserving over-relaxation of angle f in the local field (hx, hy); or_margin (may be
 * NULL) receives the distance of the reflected angle to the ends of its admissible interval. */
double mpro_overrelax(double q, double hx, double hy, double f, double* or_margin);

/* One hybrid move (Metropolis, then over-relaxation) of prediction site (x, y) against the
 * current neighbour angles; returns the new angle. met_margin = |u_acc - min(1, exp(-dE/T))|
 * (bounded proposals: also the distance of the proposal to the ends of [0, 2*pi)), or_margin =
 * distance of the reflected angle to the ends of its admissible interval; accepted (may be NULL)
 * = 1 when the Metropolis proposal was accepted. */
double mpro_update_site(const mpro_cfg* cfg, const double* phi, const uint8_t* mask, int x, int y,
                        double T, uint32_t sweep, double* met_margin, double* or_margin,
                        int* accepted);
/* The prediction sites of one colour (0 red, 1 black); margins as for mpro_sweep, written only at
 * the sites it updates. Returns the accepted Metropolis proposals. */
int64_t mpro_half_sweep(const mpro_cfg* cfg, double* phi, const uint8_t* mask, double T,
                        uint32_t sweep, int colour, double* met_margin, double* or_margin);
/* One hybrid sweep: all red prediction sites, then all black ones. The margin arrays (N, may be
 * NULL) receive each updated site's margins; other entries are set to +inf. Returns the accepted
 * Metropolis proposals. */
int64_t mpro_sweep(const mpro_cfg* cfg, double* phi, const uint8_t* mask, double T, uint32_t sweep,
                   double* met_margin, double* or_margin);
/* Bounded proposals with an adapted width (an option, see mpr_oracle.c): nsweeps sweeps; after
 * each, width <- clamp(width * exp(a - target), width_min, 2*pi) with a the sweep's accepted
 * fraction of Metropolis proposals. cfg->width is the starting width and receives the final one;
 * widths (nsweeps, may be NULL) records the width each sweep used. */
void mpro_run_adapt(mpro_cfg* cfg, double* phi, const uint8_t* mask, double T, uint32_t sweep0,
                    int nsweeps, double target, double* widths);

/* e_b = -(1/N_b) sum over nearest-neighbour bonds of cos[q(phi_i - phi_j)]. */
double mpro_energy_bond(const mpro_cfg* cfg, const double* phi);
/* Per-bond energy over measured-measured bonds; returns 3 when there is no such bond. */
int mpro_energy_sample(const mpro_cfg* cfg, const double* phi, const uint8_t* mask,
                       double* e_s, int64_t* n_pairs);

/* nsweeps hybrid sweeps with indices sweep0 .. sweep0+nsweeps-1. acc (N, may be NULL) gains the
 * angle of every prediction site after every sweep; energies (nsweeps, may be NULL) receives e_b
 * after every sweep. */
void mpro_run(const mpro_cfg* cfg, double* phi, const uint8_t* mask, double T, uint32_t sweep0,
              int nsweeps, double* acc, double* energies);

/* Temperature tuning by bisection in log T; *sweep is the next sweep index and advances by the
 * sweeps used. trace_T / trace_e (max_probes entries, may be NULL) record the probes. */
int mpro_tune(const mpro_cfg* cfg, double* phi, const uint8_t* mask, double e_s, uint32_t* sweep,
              const mpro_tune_cfg* tcfg, double* T_out, double* trace_T, double* trace_e,
              int* n_probes);

/* Alternative tunings (readings): heating from T_lo by `factor` per probe until e_b crosses e_s,
 * then bisection; the energy curve of the unconditional lattice; inversion of a tabulated curve. */
int mpro_tune_heating(const mpro_cfg* cfg, double* phi, const uint8_t* mask, double e_s,
                      uint32_t* sweep, const mpro_tune_cfg* t, double factor, double* T_out,
                      double* trace_T, double* trace_e, int* n_probes);
void mpro_energy_curve(const mpro_cfg* cfg, const double* T, int n, const mpro_tune_cfg* t,
                       uint32_t* sweep, double* e_out);
int mpro_invert_curve(const double* T, const double* e, int n, double e_s, double* T_out);

/* Equilibration with an energy-slope stop (an option: the paper fixes no equilibration rule):
 * sweeps in chunks of `chunk` (>= 2), e_b recorded after every sweep; after the second and every
 * later chunk, stop when the chunk's mean differs from the previous chunk's by at most z standard
 * errors of the difference, sqrt((s_k^2 + s_{k-1}^2) / chunk), s^2 the chunk's sample variance:
 * no drift the chunk can resolve. At most max_sweeps sweeps (whole chunks). Returns the sweeps
 * run; *sweep advances by them. */
int mpro_equilibrate(const mpro_cfg* cfg, double* phi, const uint8_t* mask, double T,
                     uint32_t* sweep, int chunk, int max_sweeps, double z);

/* zhat = z on measured sites, zmin + (zmax - zmin) * (acc/nsamples) / (2*pi) elsewhere. */
void mpro_predict(int N, const double* acc, int nsamples, const double* z, const uint8_t* mask,
                  double zmin, double zmax, double* zhat);

#ifdef __cplusplus
}
#endif
#endif
