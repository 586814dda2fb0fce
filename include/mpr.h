/*
 * mpr.h -- C ABI of libmpr: GPU (sm_103a) gap filling of 2-D gridded data with the modified
 * planar rotator (MPR) model (Lach, Borovsky, Zukovic, "Numerical Precision Effects on GPU
 * Simulation of Massive Spatial Data, Based on the Modified Planar Rotator Model").
 *
 * The method (Sec. 2): measured values are mapped onto spin angles that stay frozen; the spins of
 * the prediction sites evolve by conditional Monte Carlo with the hybrid algorithm (Metropolis +
 * energy-conserving over-relaxation) under H = -J sum_<ij> cos[q(phi_i - phi_j)] (Eq. 2, J = 1,
 * q = 1/2 by default); the reduced temperature is the only parameter and is inferred from the
 * data; predictions are averages of equilibrium configurations mapped back to the data scale.
 * Precision settings follow the paper's three axes (Sec. 2): spin storage X_S, energy X_E and
 * functions X_F, plus 16-bit spin storage (the paper's stated future work, Sec. 3).
 *
 * Conventions
 *   - Grids are Lx x Ly, row-major, site s = y*Lx + x. Boundaries are open.
 *   - Every call returns an mpr_status; nothing aborts or throws across the ABI. Arguments are
 *     validated before any device work. mpr_last_error() gives a message for the calling thread.
 *   - A handle is used by one host thread at a time. All device work of a handle is ordered on
 *     its stream (default: the legacy default stream; see mpr_set_stream).
 *   - "host" pointers are ordinary CPU memory (pinned memory makes the copies faster); "dev"
 *     pointers are device memory of the current CUDA device, e.g. from torch. The library copies
 *     inputs; the caller keeps ownership of every pointer it passes.
 *   - The library allocates the device memory of a handle at creation (from its stream-ordered
 *     pool, see mpr_trim_memory; batches with cudaMalloc) and frees it in mpr_destroy.
 */
#ifndef MPR_H
#define MPR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mpr_ctx* mpr_handle;

typedef enum {
    MPR_OK = 0,
    MPR_ERR_INVALID_ARG = 1,      /* bad size, NULL pointer, option out of range, NaN data  */
    MPR_ERR_DEGENERATE = 2,       /* fewer than 2 measured sites, or zmax == zmin           */
    MPR_ERR_NO_PAIRS = 3,         /* no two measured sites are neighbours: e_s undefined    */
    MPR_ERR_TUNE_NO_CONVERGE = 4, /* sample energy above the bracket's top, or probes out   */
    MPR_ERR_CUDA = 5,             /* a CUDA runtime call failed                              */
    MPR_ERR_OOM = 6,              /* device allocation failed                                */
    MPR_ERR_DEVICE_TIMEOUT = 7,   /* a bounded device-side wait ran out (batched kernel)    */
    MPR_ERR_STATE = 8             /* call out of order, e.g. predict before any sample       */
} mpr_status;

/* Spin storage X_S (Sec. 2: DP or SP spin variables; 16-bit storage is the future work of Sec. 3). */
typedef enum { MPR_STORE_F64 = 0, MPR_STORE_F32 = 1, MPR_STORE_F16 = 2, MPR_STORE_BF16 = 3 } mpr_store;
/* Energy X_E and function X_F precision (Sec. 2): D = FP64, S = FP32 (functions: hardware
 * intrinsics __sinf/__cosf/__expf, as the paper uses for all SP function evaluations).
 * H (functions only, FP16 spin storage only; FP16 arithmetic is the paper's future work, Sec. 3):
 * as S, except that the over-relaxation's doubled field angle is computed in FP16 (half2)
 * arithmetic from the FP32 field rounded to FP16 (error at most about 3.4e-3 rad on the doubled
 * angle: 2.4e-3 from the FP16 polynomial and result, 1e-3 from the rounded components), so an
 * over-relaxed angle moves by up to about 7e-3 rad more than with S; the Metropolis energy
 * difference, the acceptance test and the angle wraps stay FP32. Uniform proposals only. */
typedef enum { MPR_PREC_D = 0, MPR_PREC_S = 1, MPR_PREC_H = 2 } mpr_prec;
/* Running sums of the sampled angles: FP64, or FP32 with Kahan compensation. */
typedef enum { MPR_ACC_F64 = 0, MPR_ACC_KAHAN_F32 = 1 } mpr_acc;

typedef struct {
    uint64_t seed;     /* Philox-4x32-10 key (Salmon et al., SC'11); counters are (site, sweep) */
    double q;          /* exponent of Eq. 2, 0 < q <= 1; 0 selects the default 1/2              */
    int store;         /* mpr_store  (X_S)                                                      */
    int energy;        /* mpr_prec   (X_E): the energy reduction                                */
    int func;          /* mpr_prec   (X_F): sin/cos/exp/atan2 and the update arithmetic         */
    int acc;           /* mpr_acc: prediction accumulators                                      */
} mpr_options;

/* Temperature tuning (Sec. 2: the reduced temperature is inferred from the incomplete data):
 * bisection in log T on [T_lo, T_hi] for the T whose equilibrium bond energy of the conditional
 * lattice equals the sample's, e_b(T) = e_s. Each probe runs n_eq sweeps, then averages e_b over
 * n_meas sweeps; it stops when |e_b - e_s| <= rel_tol*|e_s| or T_hi/T_lo < ratio_tol. */
typedef struct {
    int n_eq;          /* default 200 */
    int n_meas;        /* default 50  */
    double T_lo;       /* default 1e-3 */
    double T_hi;       /* default 10   */
    double rel_tol;    /* default 1e-3 */
    double ratio_tol;  /* default 1.001 */
    int max_probes;    /* default 30, at most 64 */
} mpr_tuning;

typedef struct {
    int Lx, Ly;
    int64_t n_sites, n_pred, n_bonds, n_sample_pairs;
    double zmin, zmax;         /* range of the measured values                               */
    double e_sample;           /* e_s: per-bond energy of the measured-measured bonds         */
    double T;                  /* current temperature (tuned or set), 0 if none               */
    uint32_t sweep;            /* index of the next sweep (Philox counter)                    */
    int n_samples;             /* sampling sweeps accumulated so far                          */
    int n_probes;              /* probes of the last tuning                                   */
    double e_bond_mean;        /* mean e_b over the sampling sweeps of the last mpr_run       */
    uint64_t site_updates;     /* prediction-site hybrid moves done since creation            */
    size_t device_bytes;       /* device memory held by the handle                            */
    uint64_t kernel_launches;  /* kernels launched by the handle since creation               */
    double prof_sweep_ms;      /* with profiling on: device time of the pure sweep segments   */
    uint64_t prof_sweep_launches; /* ... and the number of sweep-kernel launches they hold    */
    int sweep_kernel;          /* FP32-function sweeps: 0 = one tile per block, 1 = TMA-fed   */
                               /* persistent kernel; -1 = not chosen yet, or FP64 functions   */
} mpr_info;

/* mpr_create: copies the host grid (values: Lx*Ly doubles, ignored where mask == 0 and may be
 * NaN there; mask: Lx*Ly bytes, nonzero = measured/frozen), maps the measured values onto angles
 * phi = 2*pi*(z - zmin)/(zmax - zmin) (Sec. 2: the data are mapped onto spins), draws uniform
 * initial angles for the prediction sites and computes the sample energy e_s. Default options:
 * seed 0, q = 1/2, FP32 spins, FP64 energy, FP32 intrinsic functions, FP64 accumulators.
 * Errors: INVALID_ARG (Lx or Ly < 2, N > 2^31 - 1, NULL pointer, NaN/inf at a measured site),
 * DEGENERATE, NO_PAIRS, OOM, CUDA. *out is NULL on error. */
mpr_status mpr_create(int Lx, int Ly, const double* values, const unsigned char* mask,
                      mpr_handle* out);
/* Same, from device buffers, with all work on `stream` (a cudaStream_t, NULL = legacy default),
 * which becomes the handle's stream. */
mpr_status mpr_create_dev(int Lx, int Ly, const double* values_dev, const unsigned char* mask_dev,
                          void* stream, mpr_handle* out);
/* Waits for the handle's queued work, then releases its device and pinned host memory (to the
 * pool). NULL is ignored. */
void mpr_destroy(mpr_handle h);
/* Device memory of handles comes from one stream-ordered pool per device that the library owns;
 * up to 8 GiB of freed memory stays cached there for the next handles (no driver call, no
 * device-wide synchronisation at creation or destruction). This returns every cached byte to
 * the driver (handles alive keep theirs). */
mpr_status mpr_trim_memory(void);

/* Replaces the options and restarts the chain: the spins are re-initialised, the sweep counter,
 * the samples and the temperature are cleared. */
mpr_status mpr_set_options(mpr_handle h, const mpr_options* opt);
mpr_status mpr_get_options(mpr_handle h, mpr_options* opt);
/* Waits for the work queued on the old stream, then orders all later work on `stream`. */
mpr_status mpr_set_stream(mpr_handle h, void* stream);
/* INVALID_ARG for n_eq < 0, n_meas < 1, T_lo <= 0, T_hi <= T_lo, rel_tol < 0, ratio_tol <= 1 or
 * max_probes outside [2, 64]. */
mpr_status mpr_set_tuning(mpr_handle h, const mpr_tuning* t);

/* Runs the tuning from the current state (the chain continues through the probes) and sets the
 * handle's temperature. TUNE_NO_CONVERGE still sets T (to T_hi, or the last bracket midpoint). */
mpr_status mpr_tune_temperature(mpr_handle h, double* T_out);
mpr_status mpr_set_temperature(mpr_handle h, double T);   /* T > 0; bypasses the tuning */

/* Alternative tunings (readings of Sec. 2, which says only that T is inferred from the data).
 *
 * Heating: probe T_lo, then T *= factor per probe (clamped to T_hi; the chain carries over, so
 * every probe starts from the cooler probe's equilibrium) until e_b(T) passes e_s, then bisection
 * in log T inside the last bracket with the stopping rules of mpr_tune_temperature. e_s at or
 * below e_b(T_lo): T_lo. No crossing up to T_hi, or max_probes reached: TUNE_NO_CONVERGE with T
 * set to the last temperature (or bracket midpoint). factor in (1, 100], else INVALID_ARG. */
mpr_status mpr_tune_heating(mpr_handle h, double factor, double* T_out);
/* Energy curve of the unconditional model: an Lx x Ly lattice with every site free (no data),
 * uniform random start, options `opt` (NULL: defaults; seed, q, precision), then for each T[i] in
 * turn n_eq sweeps and the mean bond energy e_b over n_meas sweeps (from `tuning`; NULL:
 * defaults), the chain carrying over between temperatures. e_out: n doubles (host). Runs on the
 * legacy default stream and synchronises; allocates and frees its own device memory. */
mpr_status mpr_energy_curve(int Lx, int Ly, const mpr_options* opt, const mpr_tuning* tuning,
                            const double* T, int n, double* e_out);
/* Sets T from a tabulated curve e(T) (host arrays, n >= 2, T increasing): the temperature where
 * the piecewise-linear interpolant in log T first reaches the handle's e_s. e_s at or below e[0]:
 * T[0]; above every e[i]: T[n-1] with TUNE_NO_CONVERGE. No sweeps run. */
mpr_status mpr_tune_from_curve(mpr_handle h, const double* T, const double* e, int n,
                               double* T_out);

/* equil sweeps, then samples sweeps after each of which every prediction angle is added to its
 * accumulator (Sec. 2: averaging over configurations in equilibrium). One hybrid sweep updates
 * all red prediction sites, then all black ones; each update is a Metropolis move with a uniform
 * proposal followed by one over-relaxation move. May be called repeatedly; the sweep counter
 * and the accumulators carry over. STATE if no temperature is set. */
mpr_status mpr_run(mpr_handle h, int equil, int samples);

/* mpr_run with the length of the equilibration decided from the energy: sweeps in chunks of
 * `chunk` (>= 2) with the bond energy e_b recorded after every sweep; after the second and every
 * later chunk, equilibration ends when the chunk's mean e_b differs from the previous chunk's by
 * at most 2 standard errors of the difference (sqrt((s_k^2 + s_{k-1}^2) / chunk), s^2 the chunks'
 * sample variances), i.e. once the energy shows no drift a chunk can resolve, or after max_equil
 * sweeps (whole chunks). Then `samples` accumulated sweeps as in mpr_run. The paper averages
 * configurations "in equilibrium" without a rule for recognising it; this is one. *equil_done
 * (may be NULL) receives the equilibration sweeps run. STATE if no temperature is set. */
mpr_status mpr_run_auto(mpr_handle h, int chunk, int max_equil, int samples, int* equil_done);

/* Prediction zhat = zmin + (zmax - zmin) * mean(phi) / (2*pi) at prediction sites, the measured
 * value elsewhere; out holds Lx*Ly doubles, row-major. STATE if no sample was taken. */
mpr_status mpr_predict(mpr_handle h, double* out);
mpr_status mpr_predict_dev(mpr_handle h, double* out_dev);

/* e_bond = -(1/N_b) sum_<ij> cos[q(phi_i - phi_j)] of the current state, N_b = Lx(Ly-1)+Ly(Lx-1)
 * (Eq. 2; Sec. 2 defines the specific energy e = <H>/L^2 = e_bond*N_b/N), computed in FP64;
 * e_sample = e_s. Either pointer may be NULL. */
mpr_status mpr_energy(mpr_handle h, double* e_bond, double* e_sample);
mpr_status mpr_get_info(mpr_handle h, mpr_info* info);
/* on != 0: bracket every run of sweeps without energy or sample work (equilibration) with CUDA
 * events on the handle's stream and accumulate their device time into prof_sweep_ms. */
mpr_status mpr_set_profiling(mpr_handle h, int on);

/* Sweep kernel of the FP32-function setups; both compute identical states, bit for bit.
 * kind 0: one tile (128 half-lattice columns x 32 rows) per block, staged with ordinary loads.
 * kind 1: persistent blocks over 128 x 32 tiles; the TMA unit copies the next tile's boxes into
 *         shared memory (cp.async.bulk.tensor, mbarrier with a bounded wait) while the block
 *         updates the current one. Needs a lattice at least two tiles wide (Lx > 256) and 34 rows.
 * kind -1 (default): automatic. The first run of at least 12 sweeps without energy or sample
 *         work (an equilibration, or a tuning probe's) times 5 sweeps of each kernel after one
 *         warm-up sweep each, as ordinary sweeps of the chain, and keeps kind 1 only if it is
 *         more than 2 % faster.
 * INVALID_ARG if kind is not -1, 0 or 1, or kind 1 is unavailable for the handle. A forced kind
 * stays across mpr_set_options while it remains available; an automatic choice is redone. */
mpr_status mpr_set_sweep_kernel(mpr_handle h, int kind);

/* Metropolis proposal of the handle's sweeps. The paper's hybrid step (Sec. 2) is read as an
 * independent uniform proposal on [0, 2 pi), the default (width = 0). width in (0, 2 pi] selects
 * the bounded proposal phi' = phi + width (2u - 1), u uniform on [0, 1) from the same Philox
 * word, rejected when phi' leaves [0, 2 pi); the acceptance rule is unchanged (the proposal is
 * symmetric). target in (0, 1) adapts the width after every sweep that does not sample:
 * w <- w exp(a - target), a = the sweep's accepted proposals / n_pred, w kept in [1e-3, 2 pi]; the
 * width then stays fixed while sampling (target = 0: fixed width). The width lives on the
 * device; both FP32 and FP64 function setups support it, the FP32 ones through sweep kernel
 * kind 0 only (mpr_get_info reports kind 0 while it is on). The setting and the adapted width
 * stay across mpr_set_options and mpr_set_state (a checkpoint that must resume the same chain
 * saves the width from mpr_get_proposal and sets it again with target 0 or its old target).
 * Batched handles draw uniform proposals. Synchronises the handle's stream.
 * INVALID_ARG for width outside [0, 2 pi] or target outside [0, 1). */
mpr_status mpr_set_proposal(mpr_handle h, double width, double target);
/* Current half-width of the bounded proposal (0 when proposals are uniform); synchronises. */
mpr_status mpr_get_proposal(mpr_handle h, double* width);

/* Test hook for the bounded wait of the TMA kernel: in the next pass that runs with kind 1, block
 * 0 issues no copy for its first tile, so its mbarrier wait runs out after timeout_s (0 < timeout_s
 * <= 10); the block records MPR_ERR_DEVICE_TIMEOUT and returns, the other blocks finish, nothing
 * faults or hangs, and the call that synchronises next (e.g. mpr_run) returns
 * MPR_ERR_DEVICE_TIMEOUT. That pass leaves the tiles of block 0 unchanged (the chain deviates);
 * the handle stays usable. INVALID_ARG if the handle cannot run kind 1. */
mpr_status mpr_inject_tma_stall(mpr_handle h, double timeout_s);

/* State access for checkpoints and tests: angles as Lx*Ly doubles, row-major, host memory.
 * mpr_set_state writes the prediction sites only (rounded to the storage type), leaves the
 * frozen sites as mapped, and sets the next sweep index. */
mpr_status mpr_get_state(mpr_handle h, double* angles, uint32_t* sweep);
mpr_status mpr_set_state(mpr_handle h, const double* angles, uint32_t sweep);

/* Philox-4x32-10 (Salmon et al., SC'11) as used by the sweeps: n counters of 4 words each
 * (ctr_dev, device, 4n uint32) under key (seed_lo, seed_hi) -> 4n words in out_dev. */
mpr_status mpr_philox4x32_10_dev(const uint32_t* ctr_dev, uint32_t* out_dev, int n, uint64_t seed,
                                 void* stream);

/* ---------------------------------------------------------------------------------------------
 * Batches: many independent problems of uneven size and sparsity in one persistent launch.
 * Every problem runs the method of Sec. 2 (tuning, equilibration, sampling) with its own data,
 * mask and temperature; problem i draws its random numbers from the Philox stream with problem id
 * i (so problem 0 of a batch follows the same chain as a single handle with the same options).
 * The batch computes with FP32 functions (opt->func must be MPR_PREC_S); storage, energy and
 * accumulator precision are free. The whole fill is ONE launch: by default a CUDA graph whose
 * device-side while loop repeats a red pass, a black pass (one block per tile of every unfinished
 * problem) and a finish kernel until every problem is done; or one persistent cooperative kernel
 * whose blocks meet at grid barriers between colour passes. A barrier wait is bounded (2 s by
 * default) and a wait that runs out ends the launch with MPR_ERR_DEVICE_TIMEOUT (the batch is then
 * unusable).
 * --------------------------------------------------------------------------------------------- */
typedef struct mpr_batch_ctx* mpr_batch;

/* n problems; problem i has an Lx[i] x Ly[i] grid with host arrays values[i] and mask[i] as in
 * mpr_create. opt may be NULL (defaults of mpr_create). Errors name the offending problem. */
mpr_status mpr_batch_create(int n, const int* Lx, const int* Ly, const double* const* values,
                            const unsigned char* const* mask, const mpr_options* opt,
                            mpr_batch* out);
void mpr_batch_destroy(mpr_batch b);
mpr_status mpr_batch_set_stream(mpr_batch b, void* stream);
mpr_status mpr_batch_set_tuning(mpr_batch b, const mpr_tuning* t);
/* Launch shape: the tile in half-lattice entries, tile_rows x tile_cols = 8, 16 or 32 x 128, or
 * 16 or 32 x 64 (64-column tiles waste less of narrow problems; default 32 x 128), blocks per SM
 * (persistent modes; 0 = occupancy limit) and mode: 0 = one persistent cooperative kernel (blocks
 * walk the tiles, grid barriers between colour passes), 1 = the same kernel as a one-node CUDA
 * graph, 2 (default) = one CUDA graph whose device-side while loop repeats a red pass, a black
 * pass (one block per tile) and a finish kernel until every problem is done. */
mpr_status mpr_batch_set_launch(mpr_batch b, int tile_rows, int tile_cols, int blocks_per_sm,
                                int use_graph);
/* Autotuner: times `sweeps` sweeps of every tile shape and mode (persistent modes at every
 * residency) on a copy of the batch state (the chains are left as they were), keeps the fastest,
 * and caches it for batches of the same signature. Any output pointer may be NULL. */
mpr_status mpr_batch_autotune(mpr_batch b, int sweeps, int* tile_rows_out, int* tile_cols_out,
                              int* blocks_per_sm_out);
/* One launch: with T == NULL every problem is tuned first (as mpr_tune_temperature), else T[i]
 * is used; then equil sweeps and samples accumulated sweeps (as mpr_run). T_out[i] and
 * status_out[i] (either may be NULL) receive each problem's temperature and tuning status.
 * Returns MPR_ERR_TUNE_NO_CONVERGE if any problem's tuning did not converge (results are still
 * produced), MPR_ERR_DEVICE_TIMEOUT if a grid-barrier wait ran out. */
mpr_status mpr_batch_fill(mpr_batch b, const double* T, int equil, int samples, double* T_out,
                          int* status_out);
mpr_status mpr_batch_predict(mpr_batch b, int i, double* out);          /* host, Lx*Ly doubles */
mpr_status mpr_batch_get_state(mpr_batch b, int i, double* angles, uint32_t* sweep);
/* Problem i's info as mpr_get_info gives a handle's; e_bond_mean is the mean over the sampling
 * sweeps of the latest fill that sampled, n_samples counts the sampling sweeps of every fill. */
mpr_status mpr_batch_get_info(mpr_batch b, int i, mpr_info* info);
/* The last fill's launch: iterations (sweeps of the longest-running problem), device time in ms
 * (CUDA events on the batch's stream), and the launch shape and mode it used. Any pointer may be
 * NULL. */
mpr_status mpr_batch_get_stats(mpr_batch b, int* iterations, double* fill_ms, int* tile_rows,
                               int* tile_cols, int* blocks_per_sm, int* mode);
/* Fault injection for tests of the timeout path: the next fill expects `extra_arrivals` more
 * blocks at every grid barrier than exist (so the first barrier cannot complete) and waits at most
 * timeout_s seconds. Nothing faults or hangs: the launch ends and reports MPR_ERR_DEVICE_TIMEOUT. */
mpr_status mpr_batch_inject_barrier_fault(mpr_batch b, int extra_arrivals, double timeout_s);

/* mpr_bond_energy_noalloc: e_bond = -(1/N_b) sum_<ij> cos[q(phi_i - phi_j)] of a state the caller
 * holds on the device, computed without allocating any device memory. The paper has no
 * counterpart; this entry point exists for callers that cannot call cudaMalloc -- code under a
 * fixed device-memory budget or a custom allocator that owns the device, real-time loops that must
 * not take allocator locks or synchronise.
 *   angles_dev: Lx*Ly doubles, row-major, device memory (every site, frozen or not).
 *   e_bond_dev: one double in device memory, written on `stream` (a cudaStream_t, NULL = legacy
 *               default stream); the call returns once the work is queued.
 * Limit: Lx*Ly <= 2^28 sites (16384 x 16384); larger grids return MPR_ERR_INVALID_ARG. The scratch
 * is a fixed 32 KiB array inside the library that every GPU loading the library holds until the
 * process exits. The first call on a device looks up that array's device address in the current
 * (primary) context of the device and caches it per device for the life of the process (so make
 * that first call before any stream capture that should contain later calls). The cache is not
 * refreshed: after cudaDeviceReset on a device, which destroys that context, the cached address is
 * stale, and this entry point must not be called on that device again in the same process.
 * All calls share the array: calls
 * that overlap on the GPU (e.g. on two streams) race and must be ordered by the caller.
 * No cudaMalloc, cudaFree or other allocating call is made. */
mpr_status mpr_bond_energy_noalloc(int Lx, int Ly, const double* angles_dev, double q,
                                   double* e_bond_dev, void* stream);

const char* mpr_status_string(mpr_status s);
const char* mpr_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* MPR_H */
