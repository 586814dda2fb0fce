// mpr_batch.h -- device structures shared by the batched persistent kernel (mpr_batch.cu) and
// its host driver (mpr_batch_api.cu). Not part of the public ABI.
#pragma once

#include "mpr_internal.h"

namespace mpr {
namespace batch {

enum Phase : int { kProbeEquil = 0, kProbeMeasure = 1, kRunEquil = 2, kRunSample = 3, kDone = 4 };

// Per-problem state that the kernel changes: the tuning state machine and the run counters.
struct Dyn {
    int phase;                  // Phase
    int step;                   // sweeps done in the current phase
    int np;                     // probes finished
    int kind;                   // probe kind: 0 = T_lo, 1 = T_hi, 2 = bisection midpoint
    int status;                 // MPR_OK or MPR_ERR_TUNE_NO_CONVERGE
    int nsamples;               // sampling sweeps accumulated (every fill)
    int nfill;                  // sampling sweeps of the latest fill that sampled
    unsigned sweep;             // Philox sweep index of the next sweep
    float invTf;                // 1/T in FP32 for the tile kernel
    double T;                   // temperature of the current probe / of the run
    double lo, hi, mid;         // bisection bracket in log T, current midpoint
    double esum;                // sum of e_b over the measured sweeps of the current probe
    double esamp;               // sum of e_b over the sampling sweeps of the latest fill that
                                // sampled (its mean is the problem's e_bond_mean, as a single
                                // handle reports the mean over its latest run with samples)
    unsigned long long site_updates;
};

struct Prob {
    // layout (fixed at creation)
    int Lx, Ly, Lxh, pitch, mpitch;
    int ntx, nty, ntiles, tile_base;
    long long ang_off[2];       // element offsets into the angle pool (storage type)
    long long mb_off[2];        // word offsets into the mask-bit pool
    long long acc_off[2];       // element offsets into the accumulator pool(s)
    long long Np;               // prediction sites
    double Nb;                  // bonds
    double e_s;                 // sample energy
    unsigned tiles_done;        // black tiles finished in this sweep (arrival counter)
    int tail;                   // 128-column tiles: 0, or the width (64 or 32) of the narrower
                                // tile code that runs the last tile column (it holds at most
                                // that many columns)
    Dyn d;
};

struct Ctl {
    unsigned bar_count;         // grid barrier arrivals
    unsigned bar_gen;           // grid barrier generation
    int err;                    // 0, or MPR_ERR_DEVICE_TIMEOUT after a barrier wait ran out
    int n_active;               // problems not yet done
    long long timeout_ns;       // limit of one barrier wait
    int bar_extra;              // fault injection: arrivals expected beyond the grid (0 normally)
    int pad_;
    unsigned work[2];           // next tile of the red / black pass (reset at the pass's barrier)
    int list_sel;               // which of the two tile lists is current
    int n_list;                 // tiles in the current list (tiles of unfinished problems)
    int changed;                // a problem finished in this sweep: compact the list
    int iters;                  // iterations (sweeps) the launch ran
};

struct Args {
    Prob* prob;
    int nprob;
    const int* tile_prob;       // global tile index -> problem
    int2* lists;                // two tile lists of ntiles (tile, problem) entries: the current
                                // one holds the tiles of unfinished problems, largest first
    int ntiles;
    void* ang;
    uint32_t* mb;
    double* acc;                // FP64 accumulator pool (acc_kind 0)
    float* acc_hi;              // Kahan pools (acc_kind 1)
    float* acc_lo;
    int* part32;                // 16-bit storage with acc_kind 0: exact int32 partials of the
                                // sampled angles (units of 2^-24), folded into acc every 16
                                // samples and after the last; null otherwise
    void* epart;                // one energy partial per tile
    Ctl* ctl;
    int n_eq, n_meas, max_probes;
    int equil, samples;
    int energy_f32, acc_kind;
    int max_iters;
    double T_lo, T_hi, rel_tol, log_ratio;
    uint32_t seed_lo, seed_hi;
    double q;
    float qf;
};

// Tile shapes of the batched kernels: half-lattice columns and rows per thread; the tile height
// is 8 warps x (128 / cols) x rows per thread (a warp step covers one 128-column row or two
// 64-column rows). Index = the shape id used by the launch functions below.
struct Shape {
    int cols, rpt;
};
constexpr int kShapes = 5;
constexpr Shape kShape[kShapes] = {{128, 1}, {128, 2}, {128, 4}, {64, 1}, {64, 2}};
constexpr int shape_rows(int s) { return 8 * (128 / kShape[s].cols) * kShape[s].rpt; }
constexpr int shape_cols(int s) { return kShape[s].cols; }

// The kernels of one storage type and tile shape: graph-mode pass kernel, persistent kernel, and
// their dynamic shared memory; pass_qhalf is the pass kernel compiled for q = 1/2 (16-bit
// storages only, else null). One function per storage type (mpr_batch_<type>.cu).
struct Kernels {
    const void* pass;
    const void* persistent;
    size_t smem;
    const void* pass_qhalf;
};
Kernels kernels_f16(int shape);
Kernels kernels_bf16(int shape);
Kernels kernels_f32(int shape);
Kernels kernels_f64(int shape);

}  // namespace batch

cudaError_t batch_occupancy(int store, int shape, int* blocks_per_sm);
// keys: the batch's Philox round keys (philox_sched of its seed; only k[] is read), a kernel
// parameter of every tile kernel.
cudaError_t batch_launch(int store, int shape, int grid, const batch::Args* args_dev,
                         const PhiloxSched& keys, cudaStream_t st, bool use_graph);
// Graph mode: an executable graph whose device-side while loop runs red pass, black pass and the
// finish kernel until no problem is active (or max_iters). max_tiles = blocks of a pass kernel.
// qhalf: the batch's q is 1/2 (the pass kernels compiled for it, where the storage has them).
// The black pass and the finish kernel hang on programmatic edges (each may start while its
// predecessor's last blocks run, and waits for it before reading its results); where the
// runtime refuses such edges, plain ones.
cudaError_t batch_graph_build(int store, int shape, int max_tiles, bool qhalf,
                              const batch::Args* args_dev, const PhiloxSched& keys,
                              cudaGraphExec_t* out);

}  // namespace mpr
