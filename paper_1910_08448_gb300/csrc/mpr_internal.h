// mpr_internal.h -- host-side interface between the translation units of libmpr (kernel
// launchers and the layout they share). Not part of the public ABI.
#pragma once

#include <cuda.h>   // CUtensorMap
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stddef.h>
#include <stdint.h>

#include "mpr_device.cuh"   // PhiloxSched

namespace mpr {

// NVTX range for the lifetime of a scope (visible in Nsight tools; costs nothing without one).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// Device layout of one problem. The lattice is split by colour c = (x + y) & 1 into two
// half-lattices of Ly rows x pitch columns; site (x, y) of colour c sits at column j = x >> 1 of
// row y (x = 2j + ((y + c) & 1)). Column j of a row exists when x < Lx; the rest is padding.
// mbits[c] holds one bit per half-lattice entry (1 = measured/frozen or padding, 0 = update).
struct Layout {
    int Lx, Ly;
    int Lxh;        // ceil(Lx / 2)
    int pitch;      // entries per half-lattice row (multiple of 128)
    int mpitch;     // 32-bit mask words per row = pitch / 32
};

enum Store : int { kF64 = 0, kF32 = 1, kF16 = 2, kBF16 = 3 };

struct Precision {
    int store;      // Store
    int energy;     // 0 = FP64, 1 = FP32
    int func;       // 0 = FP64, 1 = FP32 intrinsics, 2 = FP16 arithmetic where safe (FP16 spins)
    int acc;        // 0 = FP64, 1 = Kahan FP32
};

inline size_t store_bytes(int store) { return store == kF64 ? 8 : store == kF32 ? 4 : 2; }

enum SweepFlags : int { kSample = 1, kMeasure = 2, kEnergyF32 = 4 };

// One colour half-sweep of one problem.
struct SweepArgs {
    void* own;                 // half-lattice of the colour being updated
    const void* other;         // the other colour
    const uint32_t* mbits;     // mask words of the colour being updated
    double* acc;               // FP64 accumulators of the colour (kSample, acc = FP64)
    float* acc_hi;             // Kahan sum / compensation (kSample, acc = Kahan FP32)
    float* acc_lo;
    int* part32;               // FP16 spins with FP64 accumulators: exact fixed-point partial sums
                               // (units of 2^-24) of up to 16 samples, folded into acc by the
                               // handle; NULL: samples go straight to acc
    void* epart;               // per-block energy partials (kMeasure on colour 1), E type
    int Lx, Ly, Lxh, pitch, mpitch;
    int colour;
    int flags;
    uint32_t seed_lo, seed_hi, sweep, problem;
    double q, T, invT;
    float qf, invTf;           // the same in FP32 for the FP32-function kernel (no FP64 on device)
    float nl2eTf;              // -log2(e) * invTf as one FP32 product: exp(-dE/T) = 2^(dE * nl2eTf)
    int* err;                  // device error word (MPR_ERR_DEVICE_TIMEOUT) or NULL
    long long wait_ns;         // limit of one device-side wait (TMA kernel)
    int stall_test;            // test hook: block 0 of the TMA kernel issues no copy for its
                               // first tile, so its wait runs out (see mpr_inject_tma_stall)
    PhiloxSched ph;            // Philox schedule of this pass (FP32-function single-problem kernels)
    const double* width;       // bounded Metropolis proposals: device address of the half-width
                               // (NULL: uniform proposals)
    unsigned long long* accepted;  // bounded proposals: accepted proposals of the pass's
                                   // prediction sites are added here (NULL: not counted)
    int nsplit;                // one-tile-per-block FP32 kernel, plain passes: the last nsplit
                               // tiles run as two half-height tiles each (0: none)
    int late;                  // same kernel, plain passes with 16-bit spins: 1 = load each own
                               // row just before its update (the state is resident in L2), 0 =
                               // load all own rows before the staging
};

// TMA descriptors of one problem's half-lattices for the TMA-fed FP32 sweep kernel: per colour c
// the staging box of the other-colour role, the own-values box and the mask-word box.
struct TmaMaps {
    CUtensorMap other[2];
    CUtensorMap own[2];
    CUtensorMap mask[2];
    bool ok = false;
};

// Launchers (all asynchronous on `st`); each returns the launch's cudaError_t.
// FP64-function setups (X_F = D): generic kernel; FP32-function setups: the FP32 kernel.
int sweep_blocks(const Layout& L, const Precision& p);
cudaError_t launch_sweep(const Precision& p, const SweepArgs& a, cudaStream_t st);
int sweep_f32_blocks(const Layout& L);
// Resident blocks per SM of the plain pass of the one-tile-per-block FP32 kernel.
int sweep_f32_plain_occupancy(const Precision& p);
cudaError_t launch_sweep_f32(const Precision& p, const SweepArgs& a, cudaStream_t st);
cudaError_t launch_sweep_f32_prop(const Precision& p, const SweepArgs& a, cudaStream_t st);
// FP16-function setting (func 2, FP16 spins, uniform proposals only).
cudaError_t launch_sweep_f32_half(const Precision& p, const SweepArgs& a, cudaStream_t st);
// TMA kernel: maps for the layout and storage (false when the lattice is too small for its boxes,
// or the driver has no tensor maps; the one-tile-per-block kernel then runs); the launch of a
// plain pass (no kMeasure, no kSample) on nsm SMs.
bool make_sweep_maps(const Layout& L, int store, void* const ang[2], uint32_t* const mb[2],
                     TmaMaps* out);
cudaError_t launch_sweep_f32_tma(const Precision& p, const SweepArgs& a, const TmaMaps& m, int nsm,
                                 cudaStream_t st);

cudaError_t launch_minmax(const double* z, const unsigned char* mask, long long N, double* part,
                          int nblk, double* out4, cudaStream_t st);
cudaError_t launch_init(const Layout& L, const Precision& p, const double* z,
                        const unsigned char* mask, const double* range, void* ang0, void* ang1,
                        uint32_t* mb0, uint32_t* mb1, uint64_t seed, uint32_t problem,
                        cudaStream_t st);
cudaError_t launch_sample_energy(const Layout& L, const double* z, const unsigned char* mask,
                                 const double* range, double q, double* part_sum,
                                 long long* part_cnt, int nblk, double* out2, cudaStream_t st);
int sample_energy_blocks(const Layout& L);
cudaError_t launch_energy_fp64(const Layout& L, const Precision& p, const void* ang0,
                               const void* ang1, double q, double* part, int nblk, double* out,
                               cudaStream_t st);
int energy_blocks(const Layout& L);
cudaError_t launch_reduce(const Precision& p, const void* part, int n, double* out,
                          cudaStream_t st);
cudaError_t launch_predict(const Layout& L, const Precision& p, const double* z,
                           const unsigned char* mask, const double* range, const double* acc0,
                           const double* acc1, const float* hi0, const float* lo0,
                           const float* hi1, const float* lo1, int nsamples, double* out,
                           cudaStream_t st);
cudaError_t launch_get_state(const Layout& L, const Precision& p, const void* ang0,
                             const void* ang1, double* out, cudaStream_t st);
cudaError_t launch_set_state(const Layout& L, const Precision& p, const double* in,
                             const unsigned char* mask, void* ang0, void* ang1, cudaStream_t st);
cudaError_t launch_philox(const uint32_t* ctr, uint32_t* out, int n, uint64_t seed,
                          cudaStream_t st);
// acc[i] += part[i] * 2^-24 and part[i] = 0 for i < n (fixed-point partial sums of FP16 spins).
cudaError_t launch_fold_partials(double* acc, int* part, size_t n, cudaStream_t st);
// One step of the proposal-width adaptation (bounded proposals): reads and clears *count.
cudaError_t launch_adapt_width(double* width, unsigned long long* count, long long n_pred,
                               double target, cudaStream_t st);

// Sets the message returned by mpr_last_error() on the calling thread.
void set_last_error(const char* msg);

}  // namespace mpr
