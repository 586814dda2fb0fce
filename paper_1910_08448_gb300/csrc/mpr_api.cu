// mpr_api.cu -- host driver and C ABI of libmpr (declared in include/mpr.h).
//
// The handle owns the device state of one gap-filling problem: the data z and mask, the two
// colour half-lattices of spin angles in the storage precision, the frozen-site bits, the
// prediction accumulators and the reduction partials. The host side only validates, sequences
// kernels on the handle's stream and runs the temperature bisection (Sec. 2: the temperature is
// the single parameter inferred from the data) on scalars read back from the device.
#include "mpr.h"
#include "mpr_internal.h"

#include <cuda_runtime.h>

#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <new>
#include <string>
#include <vector>

using namespace mpr;

namespace {

thread_local std::string g_err;

mpr_status fail(mpr_status s, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
mpr_status fail(mpr_status s, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

#define CU(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) {                                                              \
            if (e_ == cudaErrorMemoryAllocation)                                              \
                return fail(MPR_ERR_OOM, "%s: %s", #call, cudaGetErrorString(e_));            \
            return fail(MPR_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_));               \
        }                                                                                     \
    } while (0)

#define CHECK(st)                                                                             \
    do {                                                                                      \
        mpr_status s_ = (st);                                                                 \
        if (s_ != MPR_OK) return s_;                                                          \
    } while (0)

mpr_options default_options()
{
    mpr_options o;
    o.seed = 0;
    o.q = 0.5;
    o.store = MPR_STORE_F32;
    o.energy = MPR_PREC_D;
    o.func = MPR_PREC_S;
    o.acc = MPR_ACC_F64;
    return o;
}

mpr_tuning default_tuning()
{
    mpr_tuning t;
    t.n_eq = 200;
    t.n_meas = 50;
    t.T_lo = 1e-3;
    t.T_hi = 10.0;
    t.rel_tol = 1e-3;
    t.ratio_tol = 1.001;
    t.max_probes = 30;
    return t;
}

}  // namespace

struct mpr_ctx {
    int device = 0;
    Layout L{};
    Precision prec{};
    mpr_options opt{};
    mpr_tuning tune{};
    cudaStream_t stream = nullptr;
    long long N = 0, Np = 0, Nb = 0, Nss = 0;
    double zmin = 0, zmax = 0, e_s = 0, T = 0;
    bool have_T = false;
    bool free_lattice = false;           // every site free (energy curve of the unconditional model)
    uint32_t sweep = 0;
    int nsamples = 0, n_probes = 0;
    double e_bond_mean = NAN;
    uint64_t site_updates = 0;
    size_t bytes = 0;
    uint64_t launches = 0;

    // optional CUDA-event timing of pure sweep segments
    bool prof = false, prof_pending = false;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    double prof_ms = 0.0;
    uint64_t prof_launches = 0, prof_pending_launches = 0;

    // device memory
    double* z = nullptr;                 // N, row-major
    unsigned char* mask = nullptr;       // N, row-major
    void* ang[2] = {nullptr, nullptr};   // colour half-lattices, Ly x pitch, storage type
    uint32_t* mb[2] = {nullptr, nullptr};
    double* acc[2] = {nullptr, nullptr};
    float* acc_hi[2] = {nullptr, nullptr};
    float* acc_lo[2] = {nullptr, nullptr};
    int* part32[2] = {nullptr, nullptr};   // FP16 spins + FP64 sums: fixed-point partial sums
    int pending32 = 0;                     // samples in part32 not yet folded into acc
    void* part = nullptr;                // reduction partials
    size_t part_bytes = 0;
    double* scal = nullptr;              // 16 device scalars
    double* eseries = nullptr;           // raw bond sums of measured sweeps
    int eseries_cap = 0;
    double* tmpN = nullptr;              // N doubles for state transfer / prediction
    double* host = nullptr;              // pinned host staging (16 doubles)

    // TMA descriptors of the half-lattices (FP32-function sweeps of lattices wider than a tile)
    TmaMaps tma{};
    int nsm = 0;                         // SMs of the device
    int sweep_force = -1;                // mpr_set_sweep_kernel: -1 automatic, 0, 1
    long long stall_ns = 0;              // mpr_inject_tma_stall: wait limit of the next TMA pass
    int sweep_kind = -1;                 // automatic choice (-1 until made)
    int nsplit = 0;                      // plain passes of the tile kernel: last tiles split in two
    int late = 0;                        // plain passes of the tile kernel, 16-bit spins: own rows
                                         // loaded at their update (the state fits the L2)
    // bounded Metropolis proposals (mpr_set_proposal): the half-width lives on the device in
    // scal[14], the acceptance counter of the adaptation in scal[13]
    bool prop_on = false;
    double prop_target = 0.0;            // target acceptance fraction; 0: fixed width
    cudaEvent_t cal[4] = {nullptr, nullptr, nullptr, nullptr};   // timing of the choice
};

constexpr int kCalSweeps = 5;            // timed sweeps per kernel in the automatic choice

// Device error word of the handle: the last of the 16 device scalars (zeroed at creation).
inline int* dev_err(mpr_ctx* h) { return reinterpret_cast<int*>(h->scal + 15); }
inline int* host_err(mpr_ctx* h) { return reinterpret_cast<int*>(h->host + 15); }
// Accepted bounded proposals of the current sweep (device scalar 13, as an integer).
inline unsigned long long* prop_count(mpr_ctx* h)
{
    return reinterpret_cast<unsigned long long*>(h->scal + 13);
}

namespace {

// Device memory of the handles: one stream-ordered pool per device, owned by the library. Freed
// blocks stay in the pool up to kPoolKeepBytes (returned to the driver beyond that at the next
// synchronisation), so a handle created after another one of similar size allocates without a
// driver call or a device-wide synchronisation; mpr_trim_memory returns everything.
constexpr uint64_t kPoolKeepBytes = 8ull << 30;
constexpr int kMaxDevices = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pool[kMaxDevices] = {};

cudaError_t handle_pool(int device, cudaMemPool_t* out)
{
    if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_pool_mu);
    if (!g_pool[device]) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = device;
        cudaMemPool_t pool = nullptr;
        cudaError_t e = cudaMemPoolCreate(&pool, &props);
        if (e != cudaSuccess) return e;
        uint64_t keep = kPoolKeepBytes;
        e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        if (e != cudaSuccess) {
            cudaMemPoolDestroy(pool);
            return e;
        }
        g_pool[device] = pool;
    }
    *out = g_pool[device];
    return cudaSuccess;
}

template <typename T>
mpr_status dalloc(mpr_ctx* h, T** p, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    void* q = nullptr;
    cudaMemPool_t pool = nullptr;
    cudaError_t e = handle_pool(h->device, &pool);
    if (e == cudaSuccess) e = cudaMallocFromPoolAsync(&q, bytes, pool, h->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? MPR_ERR_OOM : MPR_ERR_CUDA,
                    "device allocation (%zu bytes): %s", bytes, cudaGetErrorString(e));
    }
    *p = static_cast<T*>(q);
    h->bytes += bytes;
    return MPR_OK;
}

// Stream-ordered: the block returns to the pool after the work queued before it on the stream.
template <typename T>
void dfree(mpr_ctx* h, T** p, size_t bytes)
{
    if (*p) {
        cudaFreeAsync(*p, h->stream);
        h->bytes -= bytes ? bytes : 16;
    }
    *p = nullptr;
}

size_t ang_bytes(const mpr_ctx* h) { return (size_t)h->L.Ly * h->L.pitch * store_bytes(h->prec.store); }
size_t mb_bytes(const mpr_ctx* h) { return (size_t)h->L.Ly * h->L.mpitch * 4; }
size_t accd_bytes(const mpr_ctx* h) { return (size_t)h->L.Ly * h->L.pitch * 8; }
size_t accf_bytes(const mpr_ctx* h) { return (size_t)h->L.Ly * h->L.pitch * 4; }

void free_state(mpr_ctx* h)
{
    for (int c = 0; c < 2; ++c) {
        dfree(h, &h->ang[c], ang_bytes(h));
        dfree(h, &h->mb[c], mb_bytes(h));
        dfree(h, &h->acc[c], accd_bytes(h));
        dfree(h, &h->acc_hi[c], accf_bytes(h));
        dfree(h, &h->acc_lo[c], accf_bytes(h));
        dfree(h, &h->part32[c], accf_bytes(h));
    }
}

void free_all(mpr_ctx* h)
{
    free_state(h);
    dfree(h, &h->z, (size_t)h->N * 8);
    dfree(h, &h->mask, (size_t)h->N);
    dfree(h, &h->part, h->part_bytes);
    dfree(h, &h->scal, 16 * 8);
    dfree(h, &h->eseries, (size_t)h->eseries_cap * 8);
    dfree(h, &h->tmpN, (size_t)h->N * 8);
    if (h->host) cudaFreeHost(h->host);
    h->host = nullptr;
    if (h->ev0) cudaEventDestroy(h->ev0);
    if (h->ev1) cudaEventDestroy(h->ev1);
    h->ev0 = h->ev1 = nullptr;
    for (cudaEvent_t& e : h->cal) {
        if (e) cudaEventDestroy(e);
        e = nullptr;
    }
}

mpr_status harvest_profile(mpr_ctx* h)
{
    if (!h->prof_pending) return MPR_OK;
    CU(cudaEventSynchronize(h->ev1));
    float ms = 0.f;
    CU(cudaEventElapsedTime(&ms, h->ev0, h->ev1));
    h->prof_ms += ms;
    h->prof_launches += h->prof_pending_launches;
    h->prof_pending = false;
    return MPR_OK;
}

// Waits for the handle's stream; reports a device-side wait that ran out (MPR_ERR_DEVICE_TIMEOUT)
// since the previous check, then clears the error word.
mpr_status sync(mpr_ctx* h)
{
    CU(cudaMemcpyAsync(host_err(h), dev_err(h), sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    if (*host_err(h) != 0) {
        const int e = *host_err(h);
        *host_err(h) = 0;
        CU(cudaMemsetAsync(dev_err(h), 0, sizeof(int), h->stream));
        CU(cudaStreamSynchronize(h->stream));
        return fail(e == MPR_ERR_DEVICE_TIMEOUT ? MPR_ERR_DEVICE_TIMEOUT : MPR_ERR_CUDA,
                    "a device-side wait for a TMA copy ran out");
    }
    return harvest_profile(h);
}

mpr_status validate_options(const mpr_options* o)
{
    if (!o) return fail(MPR_ERR_INVALID_ARG, "options pointer is NULL");
    if (o->store < 0 || o->store > 3) return fail(MPR_ERR_INVALID_ARG, "store %d out of range", o->store);
    if (o->energy < 0 || o->energy > 1) return fail(MPR_ERR_INVALID_ARG, "energy %d out of range", o->energy);
    if (o->func < 0 || o->func > 2) return fail(MPR_ERR_INVALID_ARG, "func %d out of range", o->func);
    if (o->func == MPR_PREC_H && o->store != MPR_STORE_F16)
        return fail(MPR_ERR_INVALID_ARG, "FP16 functions (func = H) need FP16 spin storage");
    if (o->acc < 0 || o->acc > 1) return fail(MPR_ERR_INVALID_ARG, "acc %d out of range", o->acc);
    if (!(o->q >= 0.0 && o->q <= 1.0)) return fail(MPR_ERR_INVALID_ARG, "q = %g outside (0, 1]", o->q);
    return MPR_OK;
}

// Allocates the precision-dependent state, maps the data, draws the initial angles and computes
// e_s (which depends on q). Clears the chain: sweep counter, samples, temperature.
mpr_status init_state(mpr_ctx* h)
{
    free_state(h);
    const Precision& p = h->prec;
    for (int c = 0; c < 2; ++c) {
        CHECK(dalloc(h, &h->ang[c], ang_bytes(h)));
        CHECK(dalloc(h, &h->mb[c], mb_bytes(h)));
        if (p.acc == 0) {
            CHECK(dalloc(h, &h->acc[c], accd_bytes(h)));
            CU(cudaMemsetAsync(h->acc[c], 0, accd_bytes(h), h->stream));
            if (p.store == kF16 && p.func >= 1) {   // exact fixed-point partials (tile kernel)
                CHECK(dalloc(h, &h->part32[c], accf_bytes(h)));
                CU(cudaMemsetAsync(h->part32[c], 0, accf_bytes(h), h->stream));
            }
        } else {
            CHECK(dalloc(h, &h->acc_hi[c], accf_bytes(h)));
            CHECK(dalloc(h, &h->acc_lo[c], accf_bytes(h)));
            CU(cudaMemsetAsync(h->acc_hi[c], 0, accf_bytes(h), h->stream));
            CU(cudaMemsetAsync(h->acc_lo[c], 0, accf_bytes(h), h->stream));
        }
    }
    // Last wave of the tile kernel's plain passes: with T tiles and S resident blocks on the
    // device, the last T mod S tiles would run as a partial wave; when twice that many blocks
    // still fit one wave (and no tile column is narrow), they run as half-height tiles. Only for
    // lattices of fewer than four waves, where the partial one is a large share of the pass
    // (4096^2: 2048 tiles on 608 blocks, 2 % faster; at 8192^2 it measured 1 % slower).
    h->nsplit = 0;
    if (p.func != 0 && h->L.Lxh % 128 == 0) {
        const int slots = sweep_f32_plain_occupancy(p) * h->nsm;
        const int nt = sweep_f32_blocks(h->L);
        const int rem = slots > 0 ? nt % slots : 0;
        if (rem > 0 && 2 * rem <= slots && nt < 4 * slots) h->nsplit = rem;
    }
    // Own rows of a plain pass with 16-bit spins: loaded at each row's update when both colours
    // fit comfortably in the 129 MB L2 (4096^2: 33.5 MB; 1.8 % faster there), else all before
    // the staging (8192^2: 134 MB, where the late loads measured 1.6 % slower).
    h->late = (p.func != 0 && (p.store == kF16 || p.store == kBF16) &&
               2 * ang_bytes(h) <= ((size_t)48 << 20)) ? 1 : 0;
    // TMA maps for the FP32-function kernel (false: the lattice is too narrow for its boxes)
    h->tma = TmaMaps{};
    if (p.func == 1) make_sweep_maps(h->L, p.store, h->ang, h->mb, &h->tma);
    h->sweep_kind = -1;   // the storage type may have changed: choose again
    if (h->sweep_force == 1 && !h->tma.ok) h->sweep_force = -1;
    CU(launch_init(h->L, p, h->z, h->mask, h->scal, h->ang[0], h->ang[1], h->mb[0], h->mb[1],
                   h->opt.seed, 0u, h->stream));
    h->launches += 3;   // init + sample energy (2)
    const int nb = sample_energy_blocks(h->L);
    double* psum = static_cast<double*>(h->part);
    long long* pcnt = reinterpret_cast<long long*>(psum + nb);
    CU(launch_sample_energy(h->L, h->z, h->mask, h->scal, h->opt.q, psum, pcnt, nb, h->scal + 4,
                            h->stream));
    CU(cudaMemcpyAsync(h->host, h->scal + 4, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CHECK(sync(h));
    h->e_s = h->host[0];
    h->Nss = (long long)h->host[1];
    h->sweep = 0;
    h->nsamples = 0;
    h->pending32 = 0;
    h->have_T = false;
    h->T = 0.0;
    h->n_probes = 0;
    h->e_bond_mean = NAN;
    if (h->Nss == 0 && !h->free_lattice)
        return fail(MPR_ERR_NO_PAIRS, "no two measured sites are nearest neighbours");
    return MPR_OK;
}

// free_lattice: no data (values and mask ignored); every site is free, as in the unconditional
// model whose energy curve mpr_energy_curve records.
mpr_status create_common(int Lx, int Ly, const double* values, const unsigned char* mask,
                         bool on_device, cudaStream_t stream, mpr_handle* out,
                         bool free_lattice = false)
{
    if (!out) return fail(MPR_ERR_INVALID_ARG, "out pointer is NULL");
    *out = nullptr;
    if (!free_lattice && (!values || !mask)) return fail(MPR_ERR_INVALID_ARG, "values or mask is NULL");
    if (Lx < 2 || Ly < 2) return fail(MPR_ERR_INVALID_ARG, "grid %d x %d: both sides must be >= 2", Lx, Ly);
    if ((long long)Lx * Ly > 2147483647LL)
        return fail(MPR_ERR_INVALID_ARG, "grid %d x %d exceeds 2^31 - 1 sites", Lx, Ly);
    mpr_ctx* h = new (std::nothrow) mpr_ctx();
    if (!h) return fail(MPR_ERR_OOM, "host allocation failed");
    h->stream = stream;
    h->free_lattice = free_lattice;
    h->opt = default_options();
    h->tune = default_tuning();
    h->prec = Precision{h->opt.store, h->opt.energy, h->opt.func, h->opt.acc};
    h->L.Lx = Lx;
    h->L.Ly = Ly;
    h->L.Lxh = (Lx + 1) / 2;
    h->L.pitch = (h->L.Lxh + 127) / 128 * 128;
    h->L.mpitch = h->L.pitch / 32;
    h->N = (long long)Lx * Ly;
    h->Nb = (long long)Lx * (Ly - 1) + (long long)Ly * (Lx - 1);
    auto bail = [&](mpr_status s) {
        std::string keep = g_err;
        free_all(h);
        delete h;
        g_err = keep;
        return s;
    };
    mpr_status s;
    if (cudaGetDevice(&h->device) != cudaSuccess) return bail(fail(MPR_ERR_CUDA, "no CUDA device"));
    if (cudaMallocHost(&h->host, 16 * sizeof(double)) != cudaSuccess)
        return bail(fail(MPR_ERR_OOM, "pinned host allocation failed"));
    const int nmm = 256;
    {
        const int sb = sweep_blocks(h->L, h->prec), sf = sweep_f32_blocks(h->L);
        size_t need = (size_t)std::max(sb, sf) * 8;
        size_t a = (size_t)sample_energy_blocks(h->L) * 16;
        size_t b = (size_t)energy_blocks(h->L) * 8;
        size_t c = (size_t)nmm * 32;
        for (size_t v : {a, b, c}) need = need > v ? need : v;
        h->part_bytes = need;
    }
    if ((s = dalloc(h, &h->part, h->part_bytes)) != MPR_OK) return bail(s);
    if ((s = dalloc(h, &h->scal, 16 * 8)) != MPR_OK) return bail(s);
    if (cudaMemsetAsync(h->scal, 0, 16 * 8, stream) != cudaSuccess ||
        cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess)
        return bail(fail(MPR_ERR_CUDA, "device query failed"));
    h->host[15] = 0.0;
    if ((s = dalloc(h, &h->z, (size_t)h->N * 8)) != MPR_OK) return bail(s);
    if ((s = dalloc(h, &h->mask, (size_t)h->N)) != MPR_OK) return bail(s);
    if (free_lattice) {
        if (cudaMemsetAsync(h->z, 0, (size_t)h->N * 8, stream) != cudaSuccess ||
            cudaMemsetAsync(h->mask, 0, (size_t)h->N, stream) != cudaSuccess)
            return bail(fail(MPR_ERR_CUDA, "lattice setup failed"));
        h->zmin = 0.0;
        h->zmax = 0.0;
        h->Np = h->N;
        if ((s = init_state(h)) != MPR_OK) return bail(s);
        *out = h;
        return MPR_OK;
    }
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (cudaMemcpyAsync(h->z, values, (size_t)h->N * 8, kind, stream) != cudaSuccess ||
        cudaMemcpyAsync(h->mask, mask, (size_t)h->N, kind, stream) != cudaSuccess)
        return bail(fail(MPR_ERR_CUDA, "input copy failed: %s", cudaGetErrorString(cudaGetLastError())));
    if (launch_minmax(h->z, h->mask, h->N, static_cast<double*>(h->part), nmm, h->scal, stream) != cudaSuccess ||
        cudaMemcpyAsync(h->host, h->scal, 4 * sizeof(double), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess)
        return bail(fail(MPR_ERR_CUDA, "range reduction failed: %s", cudaGetErrorString(cudaGetLastError())));
    const double lo = h->host[0], hi = h->host[1], nmeas = h->host[2], bad = h->host[3];
    if (bad > 0) return bail(fail(MPR_ERR_INVALID_ARG, "%.0f measured values are NaN or infinite", bad));
    if (nmeas < 2 || !(hi > lo))
        return bail(fail(MPR_ERR_DEGENERATE, "%.0f measured sites, range [%g, %g]", nmeas, lo, hi));
    h->zmin = lo;
    h->zmax = hi;
    h->Np = h->N - (long long)nmeas;
    h->launches += 2;   // range reduction
    if ((s = init_state(h)) != MPR_OK) return bail(s);
    *out = h;
    return MPR_OK;
}

mpr_status ensure_eseries(mpr_ctx* h, int n)
{
    if (n <= h->eseries_cap) return MPR_OK;
    dfree(h, &h->eseries, (size_t)h->eseries_cap * 8);
    h->eseries_cap = 0;
    CHECK(dalloc(h, &h->eseries, (size_t)n * 8));
    h->eseries_cap = n;
    return MPR_OK;
}

// Adds the fixed-point partial sums (units of 2^-24) into the FP64 sums and clears them; every add
// is exact, so the sums equal those of adding each sample to FP64 directly.
mpr_status fold_partials(mpr_ctx* h)
{
    if (!h->part32[0] || h->pending32 == 0) return MPR_OK;
    const size_t n = (size_t)h->L.Ly * h->L.pitch;
    for (int c = 0; c < 2; ++c) CU(launch_fold_partials(h->acc[c], h->part32[c], n, h->stream));
    h->launches += 2;
    h->pending32 = 0;
    return MPR_OK;
}

// n hybrid sweeps at temperature T; with kMeasure the raw bond sum of sweep k lands in
// eseries[k]. Every launch goes to the handle's stream; nothing here synchronises, except the
// one-time choice of the FP32 sweep kernel (sweep_kind), which waits for its timing events.
//
// Kernel choice: the TMA kernel (kind 1) and the one-tile-per-block kernel (kind 0) change the
// state identically, but their energy partials come from tiles of different heights, so passes
// with the fused energy (kMeasure) always run kind 0: energies stay bit-identical whatever kind
// the plain passes use.
mpr_status sweeps(mpr_ctx* h, int n, double T, int flags)
{
    if (n <= 0) return MPR_OK;
    if (flags & kMeasure) CHECK(ensure_eseries(h, n));
    SweepArgs a{};
    a.Lx = h->L.Lx;
    a.Ly = h->L.Ly;
    a.Lxh = h->L.Lxh;
    a.pitch = h->L.pitch;
    a.mpitch = h->L.mpitch;
    a.flags = flags | (h->prec.energy == 1 ? kEnergyF32 : 0);
    a.seed_lo = (uint32_t)h->opt.seed;
    a.seed_hi = (uint32_t)(h->opt.seed >> 32);
    a.problem = 0;
    a.q = h->opt.q;
    a.T = T;
    a.invT = 1.0 / T;
    a.qf = (float)h->opt.q;
    a.invTf = (float)(1.0 / T);
    a.nl2eTf = -1.4426950408889634f * a.invTf;   // FP32 product, as the batched kernels form it
    a.epart = h->part;
    a.err = dev_err(h);
    a.wait_ns = 2000000000LL;   // 2 s: a TMA copy lands in microseconds
    a.stall_test = 0;
    a.nsplit = (flags == 0) ? h->nsplit : 0;   // plain passes of the tile kernel only
    a.late = h->late;   // read by the plain-pass launches only (the red pass of a measured sweep too)
    // bounded proposals; the width adapts after every sweep that does not sample
    const bool adapt = h->prop_on && h->prop_target > 0.0 && !(flags & kSample);
    a.width = h->prop_on ? h->scal + 14 : nullptr;
    a.accepted = adapt ? prop_count(h) : nullptr;
    const bool f32 = h->prec.func != 0;   // FP32 (or FP16) functions: the tile kernels
    const int nblk = f32 ? sweep_f32_blocks(h->L) : sweep_blocks(h->L, h->prec);
    const bool timed = h->prof && flags == 0;
    if (timed) {
        CHECK(harvest_profile(h));
        CU(cudaEventRecord(h->ev0, h->stream));
    }
    // one hybrid sweep (both colour passes) with kernel kind (0/1; ignored for FP64 functions)
    auto one = [&](int k, int kind) -> mpr_status {
        a.sweep = h->sweep;
        for (int c = 0; c < 2; ++c) {
            a.colour = c;
            a.ph = philox_sched(a.sweep, a.problem, kTagMetropolis, (uint32_t)c, a.seed_lo, a.seed_hi);
            a.own = h->ang[c];
            a.other = h->ang[c ^ 1];
            a.mbits = h->mb[c];
            a.acc = h->acc[c];
            a.acc_hi = h->acc_hi[c];
            a.part32 = h->part32[c];
            a.acc_lo = h->acc_lo[c];
            if (kind == 1 && h->stall_ns > 0) {   // injected stall: this launch only
                SweepArgs s = a;
                s.stall_test = 1;
                s.wait_ns = h->stall_ns;
                h->stall_ns = 0;
                CU(launch_sweep_f32_tma(h->prec, s, h->tma, h->nsm, h->stream));
                continue;
            }
            CU(!f32 ? launch_sweep(h->prec, a, h->stream)
                    : kind == 1 ? launch_sweep_f32_tma(h->prec, a, h->tma, h->nsm, h->stream)
                                : launch_sweep_f32(h->prec, a, h->stream));
        }
        if (flags & kMeasure) CU(launch_reduce(h->prec, h->part, nblk, h->eseries + k, h->stream));
        if (adapt) CU(launch_adapt_width(h->scal + 14, prop_count(h), h->Np, h->prop_target, h->stream));
        h->launches += ((flags & kMeasure) ? 3 : 2) + (adapt ? 1 : 0);
        // int32 partials hold at most 16 samples: fold them into the FP64 sums then
        if ((flags & kSample) && h->part32[0] && ++h->pending32 == 16) CHECK(fold_partials(h));
        ++h->sweep;
        h->site_updates += (uint64_t)h->Np;
        return MPR_OK;
    };
    // the TMA kernel draws uniform proposals only
    const bool tma_ok = f32 && h->tma.ok && !(flags & kMeasure) && !h->prop_on;
    int k = 0;
    if (tma_ok && h->sweep_force < 0 && h->sweep_kind < 0 && flags == 0 && n >= 2 * (1 + kCalSweeps)) {
        // automatic choice: one warm-up and kCalSweeps timed sweeps of each kernel, as ordinary
        // sweeps of the chain (both kernels give the same states), then the faster one
        if (!h->cal[0])
            for (cudaEvent_t& e : h->cal) CU(cudaEventCreate(&e));
        float ms[2] = {0.f, 0.f};
        for (int kind = 0; kind < 2; ++kind) {
            CHECK(one(k++, kind));
            CU(cudaEventRecord(h->cal[2 * kind], h->stream));
            for (int i = 0; i < kCalSweeps; ++i) CHECK(one(k++, kind));
            CU(cudaEventRecord(h->cal[2 * kind + 1], h->stream));
        }
        CU(cudaEventSynchronize(h->cal[3]));
        for (int kind = 0; kind < 2; ++kind)
            CU(cudaEventElapsedTime(&ms[kind], h->cal[2 * kind], h->cal[2 * kind + 1]));
        h->sweep_kind = ms[1] < 0.98f * ms[0] ? 1 : 0;   // the TMA kernel only when clearly faster
    }
    const int kind = !tma_ok ? 0 : h->sweep_force >= 0 ? h->sweep_force : (h->sweep_kind > 0 ? 1 : 0);
    for (; k < n; ++k) CHECK(one(k, kind));
    if (timed) {
        CU(cudaEventRecord(h->ev1, h->stream));
        h->prof_pending = true;
        h->prof_pending_launches = 2ull * (uint64_t)n;
    }
    return MPR_OK;
}

// Mean over n measured sweeps of e_b = -raw/N_b, summed in sweep order on the host (FP64).
mpr_status mean_energy(mpr_ctx* h, int n, double* mean)
{
    std::vector<double> raw((size_t)n);
    CU(cudaMemcpyAsync(raw.data(), h->eseries, (size_t)n * 8, cudaMemcpyDeviceToHost, h->stream));
    CHECK(sync(h));
    double s = 0.0;
    for (int k = 0; k < n; ++k) s += -raw[(size_t)k] / (double)h->Nb;
    *mean = s / (double)n;
    return MPR_OK;
}

// e_b = -raw/N_b of the n measured sweeps of the last run, in sweep order.
mpr_status energy_series(mpr_ctx* h, int n, double* e)
{
    CU(cudaMemcpyAsync(e, h->eseries, (size_t)n * 8, cudaMemcpyDeviceToHost, h->stream));
    CHECK(sync(h));
    for (int k = 0; k < n; ++k) e[k] = -e[k] / (double)h->Nb;
    return MPR_OK;
}

mpr_status probe(mpr_ctx* h, double T, double* e)
{
    CHECK(sweeps(h, h->tune.n_eq, T, 0));
    CHECK(sweeps(h, h->tune.n_meas, T, kMeasure));
    return mean_energy(h, h->tune.n_meas, e);
}

}  // namespace

extern "C" {

mpr_status mpr_create(int Lx, int Ly, const double* values, const unsigned char* mask, mpr_handle* out)
{
    NvtxRange r("mpr_create");
    return create_common(Lx, Ly, values, mask, false, nullptr, out);
}

mpr_status mpr_create_dev(int Lx, int Ly, const double* values_dev, const unsigned char* mask_dev,
                          void* stream, mpr_handle* out)
{
    return create_common(Lx, Ly, values_dev, mask_dev, true, static_cast<cudaStream_t>(stream), out);
}

void mpr_destroy(mpr_handle h)
{
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    free_all(h);
    cudaStreamSynchronize(h->stream);   // the frees are stream-ordered: complete them here
    delete h;
}

mpr_status mpr_trim_memory(void)
{
    std::lock_guard<std::mutex> lock(g_pool_mu);
    for (cudaMemPool_t pool : g_pool) {
        if (!pool) continue;
        const cudaError_t e = cudaMemPoolTrimTo(pool, 0);
        if (e != cudaSuccess) return fail(MPR_ERR_CUDA, "cudaMemPoolTrimTo: %s", cudaGetErrorString(e));
    }
    return MPR_OK;
}

mpr_status mpr_set_options(mpr_handle h, const mpr_options* opt)
{
    if (!h) return fail(MPR_ERR_INVALID_ARG, "handle is NULL");
    CHECK(validate_options(opt));
    if (opt->func == MPR_PREC_H && h->prop_on)
        return fail(MPR_ERR_INVALID_ARG, "FP16 functions run uniform proposals only");
    free_state(h);   // sizes depend on the old precision
    h->opt = *opt;
    if (h->opt.q == 0.0) h->opt.q = 0.5;
    h->prec = Precision{opt->store, opt->energy, opt->func, opt->acc};
    return init_state(h);
}

mpr_status mpr_get_options(mpr_handle h, mpr_options* opt)
{
    if (!h || !opt) return fail(MPR_ERR_INVALID_ARG, "NULL argument");
    *opt = h->opt;
    return MPR_OK;
}

mpr_status mpr_set_stream(mpr_handle h, void* stream)
{
    if (!h) return fail(MPR_ERR_INVALID_ARG, "handle is NULL");
    CHECK(sync(h));
    h->stream = static_cast<cudaStream_t>(stream);
    return MPR_OK;
}

mpr_status mpr_set_tuning(mpr_handle h, const mpr_tuning* t)
{
    if (!h || !t) return fail(MPR_ERR_INVALID_ARG, "NULL argument");
    if (t->n_eq < 0 || t->n_meas < 1 || !(t->T_lo > 0) || !(t->T_hi > t->T_lo) ||
        !(t->rel_tol >= 0) || !(t->ratio_tol > 1.0) || t->max_probes < 2 || t->max_probes > 64)
        return fail(MPR_ERR_INVALID_ARG, "tuning parameters out of range");
    h->tune = *t;
    return MPR_OK;
}

mpr_status mpr_tune_temperature(mpr_handle h, double* T_out)
{
    NvtxRange r("mpr_tune_temperature");
    if (!h) return fail(MPR_ERR_INVALID_ARG, "handle is NULL");
    const mpr_tuning& t = h->tune;
    const double e_s = h->e_s;
    const double tol = t.rel_tol * fabs(e_s);
    double lo = log(t.T_lo), hi = log(t.T_hi);
    int np = 0;
    mpr_status status = MPR_OK;
    double T, e;

    T = t.T_lo;
    CHECK(probe(h, T, &e));
    ++np;
    if (fabs(e - e_s) <= tol || e_s < e) goto done;

    T = t.T_hi;
    CHECK(probe(h, T, &e));
    ++np;
    if (fabs(e - e_s) <= tol) goto done;
    if (e_s > e) {
        status = fail(MPR_ERR_TUNE_NO_CONVERGE, "sample energy %.6f above e_b(T_hi) = %.6f", e_s, e);
        goto done;
    }
    for (;;) {
        if (np >= t.max_probes) {
            T = exp(0.5 * (lo + hi));
            status = fail(MPR_ERR_TUNE_NO_CONVERGE, "no convergence in %d probes", np);
            goto done;
        }
        const double mid = 0.5 * (lo + hi);
        T = exp(mid);
        CHECK(probe(h, T, &e));
        ++np;
        if (fabs(e - e_s) <= tol) goto done;
        if (e < e_s) lo = mid; else hi = mid;
        if (hi - lo < log(t.ratio_tol)) {
            T = exp(0.5 * (lo + hi));
            goto done;
        }
    }
done:
    h->T = T;
    h->have_T = true;
    h->n_probes = np;
    if (T_out) *T_out = T;
    return status;
}

mpr_status mpr_tune_heating(mpr_handle h, double factor, double* T_out)
{
    NvtxRange r("mpr_tune_heating");
    if (!h) return fail(MPR_ERR_INVALID_ARG, "handle is NULL");
    if (!(factor > 1.0) || !(factor <= 100.0))
        return fail(MPR_ERR_INVALID_ARG, "heating factor %g outside (1, 100]", factor);
    if (h->free_lattice) return fail(MPR_ERR_STATE, "the lattice has no measured data");
    const mpr_tuning& t = h->tune;
    const double e_s = h->e_s;
    const double tol = t.rel_tol * fabs(e_s);
    int np = 0;
    mpr_status status = MPR_OK;
    double T = t.T_lo, e, lo = 0.0, hi = 0.0;

    CHECK(probe(h, T, &e));
    ++np;
    if (fabs(e - e_s) <= tol || e_s < e) goto done;
    // heat until the energy passes e_s (the chain carries over from probe to probe)
    for (;;) {
        if (T >= t.T_hi) {
            status = fail(MPR_ERR_TUNE_NO_CONVERGE, "sample energy %.6f above e_b(T_hi) = %.6f", e_s, e);
            goto done;
        }
        if (np >= t.max_probes) {
            status = fail(MPR_ERR_TUNE_NO_CONVERGE, "no crossing in %d probes", np);
            goto done;
        }
        const double Tn = std::min(T * factor, t.T_hi);
        CHECK(probe(h, Tn, &e));
        ++np;
        if (fabs(e - e_s) <= tol) {
            T = Tn;
            goto done;
        }
        if (e > e_s) {
            lo = log(T);
            hi = log(Tn);
            break;
        }
        T = Tn;
    }
    // bisection in log T inside the last bracket
    for (;;) {
        if (hi - lo < log(t.ratio_tol)) {
            T = exp(0.5 * (lo + hi));
            goto done;
        }
        if (np >= t.max_probes) {
            T = exp(0.5 * (lo + hi));
            status = fail(MPR_ERR_TUNE_NO_CONVERGE, "no convergence in %d probes", np);
            goto done;
        }
        const double mid = 0.5 * (lo + hi);
        T = exp(mid);
        CHECK(probe(h, T, &e));
        ++np;
        if (fabs(e - e_s) <= tol) goto done;
        if (e < e_s) lo = mid; else hi = mid;
    }
done:
    h->T = T;
    h->have_T = true;
    h->n_probes = np;
    if (T_out) *T_out = T;
    return status;
}

mpr_status mpr_energy_curve(int Lx, int Ly, const mpr_options* opt, const mpr_tuning* tuning,
                            const double* T, int n, double* e_out)
{
    NvtxRange r("mpr_energy_curve");
    if (!T || !e_out || n < 1) return fail(MPR_ERR_INVALID_ARG, "NULL argument or n < 1");
    for (int i = 0; i < n; ++i)
        if (!(T[i] > 0.0) || !isfinite(T[i]))
            return fail(MPR_ERR_INVALID_ARG, "temperature %d (%g) must be > 0", i, T[i]);
    mpr_handle h = nullptr;
    CHECK(create_common(Lx, Ly, nullptr, nullptr, false, nullptr, &h, true));
    mpr_status s = opt ? mpr_set_options(h, opt) : MPR_OK;
    if (s == MPR_OK && tuning) s = mpr_set_tuning(h, tuning);
    for (int i = 0; i < n && s == MPR_OK; ++i) s = probe(h, T[i], &e_out[i]);
    std::string keep = g_err;
    mpr_destroy(h);
    g_err = keep;
    return s;
}

mpr_status mpr_tune_from_curve(mpr_handle h, const double* T, const double* e, int n, double* T_out)
{
    if (!h || !T || !e) return fail(MPR_ERR_INVALID_ARG, "NULL argument");
    if (n < 2) return fail(MPR_ERR_INVALID_ARG, "the curve needs at least 2 points (n = %d)", n);
    for (int i = 0; i < n; ++i) {
        if (!(T[i] > 0.0) || !isfinite(T[i]) || !isfinite(e[i]) || (i > 0 && !(T[i] > T[i - 1])))
            return fail(MPR_ERR_INVALID_ARG, "point %d: T must be positive and increasing, e finite", i);
    }
    if (h->free_lattice) return fail(MPR_ERR_STATE, "the lattice has no measured data");
    const double e_s = h->e_s;
    mpr_status status = MPR_OK;
    double Tc = T[n - 1];
    if (e_s <= e[0]) {
        Tc = T[0];
    } else {
        int i = 1;
        while (i < n && e[i] < e_s) ++i;
        if (i < n) {   // e[i - 1] < e_s <= e[i]: linear in log T
            const double f = (e_s - e[i - 1]) / (e[i] - e[i - 1]);
            Tc = exp(log(T[i - 1]) + f * (log(T[i]) - log(T[i - 1])));
        } else {
            status = fail(MPR_ERR_TUNE_NO_CONVERGE, "sample energy %.6f above the curve's top %.6f",
                          e_s, e[n - 1]);
        }
    }
    h->T = Tc;
    h->have_T = true;
    h->n_probes = 0;
    if (T_out) *T_out = Tc;
    return status;
}

mpr_status mpr_set_temperature(mpr_handle h, double T)
{
    if (!h) return fail(MPR_ERR_INVALID_ARG, "handle is NULL");
    if (!(T > 0.0) || !isfinite(T)) return fail(MPR_ERR_INVALID_ARG, "temperature %g must be > 0", T);
    h->T = T;
    h->have_T = true;
    return MPR_OK;
}

mpr_status mpr_run(mpr_handle h, int equil, int samples)
{
    NvtxRange r("mpr_run");
    if (!h) return fail(MPR_ERR_INVALID_ARG, "handle is NULL");
    if (equil < 0 || samples < 0) return fail(MPR_ERR_INVALID_ARG, "negative sweep count");
    if (!h->have_T) return fail(MPR_ERR_STATE, "no temperature: tune or set it first");
    CHECK(sweeps(h, equil, h->T, 0));
    if (samples > 0) {
        CHECK(sweeps(h, samples, h->T, kSample | kMeasure));
        h->nsamples += samples;
        CHECK(mean_energy(h, samples, &h->e_bond_mean));
    } else {
        CHECK(sync(h));
    }
    return MPR_OK;
}

// Energy-slope equilibration: chunks of measured sweeps until two consecutive chunk means agree
// within kSlopeZ standard errors of their difference (the same rule as the oracle's
// mpro_equilibrate), then the sampling sweeps of mpr_run.
constexpr double kSlopeZ = 2.0;

mpr_status mpr_run_auto(mpr_handle h, int chunk, int max_equil, int samples, int* equil_done)
{
    NvtxRange r("mpr_run_auto");
    if (!h) return fail(MPR_ERR_INVALID_ARG, "handle is NULL");
    if (chunk < 2 || max_equil < 0 || samples < 0)
        return fail(MPR_ERR_INVALID_ARG, "chunk %d must be >= 2, sweep counts >= 0", chunk);
    if (!h->have_T) return fail(MPR_ERR_STATE, "no temperature: tune or set it first");
    std::vector<double> e((size_t)chunk);
    double prev_mean = 0.0, prev_var = 0.0;
    int done = 0;
    for (int k = 0; done + chunk <= max_equil; ++k) {
        CHECK(sweeps(h, chunk, h->T, kMeasure));
        CHECK(energy_series(h, chunk, e.data()));
        done += chunk;
        double mean = 0.0;
        for (int i = 0; i < chunk; ++i) mean += e[(size_t)i];
        mean /= (double)chunk;
        double var = 0.0;
        for (int i = 0; i < chunk; ++i) var += (e[(size_t)i] - mean) * (e[(size_t)i] - mean);
        var /= (double)(chunk - 1);
        if (k > 0 && fabs(mean - prev_mean) <= kSlopeZ * sqrt((var + prev_var) / (double)chunk)) break;
        prev_mean = mean;
        prev_var = var;
    }
    if (equil_done) *equil_done = done;
    if (samples > 0) {
        CHECK(sweeps(h, samples, h->T, kSample | kMeasure));
        h->nsamples += samples;
        CHECK(mean_energy(h, samples, &h->e_bond_mean));
    } else {
        CHECK(sync(h));
    }
    return MPR_OK;
}

static mpr_status predict_to(mpr_handle h, double* out_dev)
{
    CHECK(fold_partials(h));
    CU(launch_predict(h->L, h->prec, h->z, h->mask, h->scal, h->acc[0], h->acc[1], h->acc_hi[0],
                      h->acc_lo[0], h->acc_hi[1], h->acc_lo[1], h->nsamples, out_dev, h->stream));
    h->launches += 1;
    return MPR_OK;
}

mpr_status mpr_predict(mpr_handle h, double* out)
{
    NvtxRange r("mpr_predict");
    if (!h || !out) return fail(MPR_ERR_INVALID_ARG, "NULL argument");
    if (h->nsamples == 0) return fail(MPR_ERR_STATE, "no samples taken yet");
    if (!h->tmpN) CHECK(dalloc(h, &h->tmpN, (size_t)h->N * 8));
    CHECK(predict_to(h, h->tmpN));
    CU(cudaMemcpyAsync(out, h->tmpN, (size_t)h->N * 8, cudaMemcpyDeviceToHost, h->stream));
    return sync(h);
}

mpr_status mpr_predict_dev(mpr_handle h, double* out_dev)
{
    if (!h || !out_dev) return fail(MPR_ERR_INVALID_ARG, "NULL argument");
    if (h->nsamples == 0) return fail(MPR_ERR_STATE, "no samples taken yet");
    CHECK(predict_to(h, out_dev));
    return sync(h);
}

mpr_status mpr_energy(mpr_handle h, double* e_bond, double* e_sample)
{
    if (!h) return fail(MPR_ERR_INVALID_ARG, "handle is NULL");
    if (e_bond) {
        const int nb = energy_blocks(h->L);
        CU(launch_energy_fp64(h->L, h->prec, h->ang[0], h->ang[1], h->opt.q,
                              static_cast<double*>(h->part), nb, h->scal + 8, h->stream));
        h->launches += 2;
        CU(cudaMemcpyAsync(h->host + 8, h->scal + 8, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        CHECK(sync(h));
        *e_bond = -h->host[8] / (double)h->Nb;
    }
    if (e_sample) *e_sample = h->e_s;
    return MPR_OK;
}

mpr_status mpr_get_info(mpr_handle h, mpr_info* info)
{
    if (!h || !info) return fail(MPR_ERR_INVALID_ARG, "NULL argument");
    info->Lx = h->L.Lx;
    info->Ly = h->L.Ly;
    info->n_sites = h->N;
    info->n_pred = h->Np;
    info->n_bonds = h->Nb;
    info->n_sample_pairs = h->Nss;
    info->zmin = h->zmin;
    info->zmax = h->zmax;
    info->e_sample = h->e_s;
    info->T = h->have_T ? h->T : 0.0;
    info->sweep = h->sweep;
    info->n_samples = h->nsamples;
    info->n_probes = h->n_probes;
    info->e_bond_mean = h->e_bond_mean;
    info->site_updates = h->site_updates;
    info->device_bytes = h->bytes;
    info->kernel_launches = h->launches;
    info->prof_sweep_ms = h->prof_ms;
    info->prof_sweep_launches = h->prof_launches;
    info->sweep_kernel = h->prec.func == 0 ? -1
                         : (!h->tma.ok || h->prop_on) ? 0
                         : h->sweep_force >= 0 ? h->sweep_force : h->sweep_kind;
    return MPR_OK;
}

mpr_status mpr_inject_tma_stall(mpr_handle h, double timeout_s)
{
    if (!h) return fail(MPR_ERR_INVALID_ARG, "handle is NULL");
    if (!(h->prec.func == 1 && h->tma.ok))
        return fail(MPR_ERR_INVALID_ARG, "the handle cannot run the TMA sweep kernel");
    if (!(timeout_s > 0.0) || timeout_s > 10.0)
        return fail(MPR_ERR_INVALID_ARG, "timeout %g s outside (0, 10]", timeout_s);
    h->stall_ns = (long long)(timeout_s * 1e9);
    return MPR_OK;
}

mpr_status mpr_set_proposal(mpr_handle h, double width, double target)
{
    if (!h) return fail(MPR_ERR_INVALID_ARG, "handle is NULL");
    if (!(width >= 0.0) || width > 6.283185307179586)
        return fail(MPR_ERR_INVALID_ARG, "proposal half-width %g outside [0, 2 pi]", width);
    if (!(target >= 0.0) || target >= 1.0)
        return fail(MPR_ERR_INVALID_ARG, "target acceptance %g outside [0, 1)", target);
    if (width > 0.0 && h->prec.func == MPR_PREC_H)
        return fail(MPR_ERR_INVALID_ARG, "FP16 functions run uniform proposals only");
    CHECK(sync(h));
    h->prop_on = width > 0.0;
    h->prop_target = h->prop_on ? target : 0.0;
    h->host[14] = width;
    CU(cudaMemcpyAsync(h->scal + 14, h->host + 14, sizeof(double), cudaMemcpyHostToDevice, h->stream));
    CU(cudaMemsetAsync(prop_count(h), 0, sizeof(unsigned long long), h->stream));
    return sync(h);
}

mpr_status mpr_get_proposal(mpr_handle h, double* width)
{
    if (!h || !width) return fail(MPR_ERR_INVALID_ARG, "NULL argument");
    if (!h->prop_on) {
        CHECK(sync(h));
        *width = 0.0;
        return MPR_OK;
    }
    CU(cudaMemcpyAsync(h->host + 14, h->scal + 14, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CHECK(sync(h));
    *width = h->host[14];
    return MPR_OK;
}

mpr_status mpr_set_sweep_kernel(mpr_handle h, int kind)
{
    if (!h) return fail(MPR_ERR_INVALID_ARG, "handle is NULL");
    if (kind < -1 || kind > 1) return fail(MPR_ERR_INVALID_ARG, "sweep kernel %d: use -1, 0 or 1", kind);
    if (kind == 1 && !(h->prec.func == 1 && h->tma.ok))
        return fail(MPR_ERR_INVALID_ARG,
                    "the TMA sweep kernel needs FP32 functions and a lattice of Lx > 256, Ly >= 34");
    h->sweep_force = kind;
    return MPR_OK;
}

mpr_status mpr_set_profiling(mpr_handle h, int on)
{
    if (!h) return fail(MPR_ERR_INVALID_ARG, "handle is NULL");
    CHECK(sync(h));
    if (on && !h->ev0) {
        CU(cudaEventCreate(&h->ev0));
        CU(cudaEventCreate(&h->ev1));
    }
    h->prof = on != 0;
    return MPR_OK;
}

mpr_status mpr_get_state(mpr_handle h, double* angles, uint32_t* sweep)
{
    if (!h || !angles) return fail(MPR_ERR_INVALID_ARG, "NULL argument");
    if (!h->tmpN) CHECK(dalloc(h, &h->tmpN, (size_t)h->N * 8));
    CU(launch_get_state(h->L, h->prec, h->ang[0], h->ang[1], h->tmpN, h->stream));
    h->launches += 1;
    CU(cudaMemcpyAsync(angles, h->tmpN, (size_t)h->N * 8, cudaMemcpyDeviceToHost, h->stream));
    CHECK(sync(h));
    if (sweep) *sweep = h->sweep;
    return MPR_OK;
}

mpr_status mpr_set_state(mpr_handle h, const double* angles, uint32_t sweep)
{
    if (!h || !angles) return fail(MPR_ERR_INVALID_ARG, "NULL argument");
    if (!h->tmpN) CHECK(dalloc(h, &h->tmpN, (size_t)h->N * 8));
    CU(cudaMemcpyAsync(h->tmpN, angles, (size_t)h->N * 8, cudaMemcpyHostToDevice, h->stream));
    CU(launch_set_state(h->L, h->prec, h->tmpN, h->mask, h->ang[0], h->ang[1], h->stream));
    h->launches += 1;
    CHECK(sync(h));
    h->sweep = sweep;
    return MPR_OK;
}

mpr_status mpr_philox4x32_10_dev(const uint32_t* ctr_dev, uint32_t* out_dev, int n, uint64_t seed,
                                 void* stream)
{
    if (n < 0 || (n > 0 && (!ctr_dev || !out_dev)))
        return fail(MPR_ERR_INVALID_ARG, "bad Philox arguments");
    CU(launch_philox(ctr_dev, out_dev, n, seed, static_cast<cudaStream_t>(stream)));
    CU(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
    return MPR_OK;
}

const char* mpr_status_string(mpr_status s)
{
    switch (s) {
    case MPR_OK: return "ok";
    case MPR_ERR_INVALID_ARG: return "invalid argument";
    case MPR_ERR_DEGENERATE: return "degenerate data";
    case MPR_ERR_NO_PAIRS: return "no measured nearest-neighbour pair";
    case MPR_ERR_TUNE_NO_CONVERGE: return "temperature tuning did not converge";
    case MPR_ERR_CUDA: return "CUDA error";
    case MPR_ERR_OOM: return "out of device memory";
    case MPR_ERR_DEVICE_TIMEOUT: return "device-side wait timed out";
    case MPR_ERR_STATE: return "call out of order";
    }
    return "unknown status";
}

const char* mpr_last_error(void) { return g_err.c_str(); }

}  // extern "C"

void mpr::set_last_error(const char* msg) { g_err = msg; }
