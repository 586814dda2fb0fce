// mpr_batch_api.cu -- host driver and C ABI of the batched persistent path (include/mpr.h,
// "batches"). Creates the pooled device state of many independent problems, builds the tile list
// for a launch shape, runs the whole batch (tuning, equilibration, sampling) as one cooperative
// launch, and picks the launch shape by timing the candidates on the batch itself (autotuner).
#include "mpr.h"
#include "mpr_batch.h"

#include <cuda_runtime.h>

#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

using namespace mpr;
using batch::Prob;

namespace {

mpr_status bfail(mpr_status s, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
mpr_status bfail(mpr_status s, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    set_last_error(buf);
    return s;
}

#define BCU(call)                                                                             \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) {                                                              \
            return bfail(e_ == cudaErrorMemoryAllocation ? MPR_ERR_OOM : MPR_ERR_CUDA,        \
                         "%s: %s", #call, cudaGetErrorString(e_));                            \
        }                                                                                     \
    } while (0)

#define BCHECK(st)                                                                            \
    do {                                                                                      \
        mpr_status s_ = (st);                                                                 \
        if (s_ != MPR_OK) return s_;                                                          \
    } while (0)

// Launch shapes chosen by the autotuner, per batch signature, for the life of the process.
std::mutex g_tune_mu;
std::map<std::tuple<int, long long, int, int>, std::tuple<int, int, int>> g_tune_cache;

}  // namespace

struct mpr_batch_ctx {
    int n = 0;
    int device = 0, sms = 0;
    Precision prec{};
    mpr_options opt{};
    mpr_tuning tune{};
    cudaStream_t stream = nullptr;
    bool broken = false;
    int shape = 2, bps = 0, use_graph = 2;   // launch shape (tile shape id of batch::kShape,
                                             // blocks per SM) and mode: 0/1 persistent kernel
                                             // (direct / one-node graph), 2 graph with a
                                             // device-side while loop
    cudaGraphExec_t gexec[batch::kShapes] = {};   // graph-mode executables per tile shape
    int gexec_tiles[batch::kShapes] = {};
    bool gexec_qhalf[batch::kShapes] = {};
    int tiled_shape = -1;                    // tile shape of the current tile list
    int bar_extra = 0;
    double timeout_s = 2.0;
    int last_iters = 0;                      // iterations of the last fill's launch
    float last_ms = 0.f;                     // device time of the last fill's launch
    size_t bytes = 0;
    uint64_t launches = 0;

    std::vector<Prob> P;                     // host mirror of the device problem table
    std::vector<double> zmin, zmax;
    std::vector<long long> N, Nss, z_off;
    std::vector<int> tile_prob;
    std::vector<int> order;                  // all tiles, largest first
    std::vector<int2> list;                  // (tile, problem) of the problems a fill starts with
    int2* d_lists = nullptr;                 // the two device tile lists
    int ntiles = 0;
    batch::Args* dArgs = nullptr;            // device copy of the launch arguments

    // device
    Prob* dP = nullptr;
    batch::Ctl* ctl = nullptr;
    int* d_tile_prob = nullptr;
    int tile_cap = 0;
    void* ang = nullptr;
    uint32_t* mb = nullptr;
    double* acc = nullptr;
    float* acc_hi = nullptr;
    float* acc_lo = nullptr;
    int* part32 = nullptr;                   // int32 sample partials (16-bit storage, FP64 sums)
    void* epart = nullptr;
    double* zpool = nullptr;
    unsigned char* mpool = nullptr;
    double* range = nullptr;                 // 2 per problem
    double* scal = nullptr;                  // 8 per problem
    double* part = nullptr;                  // reduction scratch of the set-up kernels
    size_t part_bytes = 0;
    double* tmp = nullptr;                   // largest N doubles
    long long maxN = 0;
    long long ang_elems = 0, mb_words = 0, acc_elems = 0, z_elems = 0;
};

namespace {

template <typename T>
mpr_status balloc(mpr_batch_ctx* b, T** p, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    void* q = nullptr;
    const cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return bfail(e == cudaErrorMemoryAllocation ? MPR_ERR_OOM : MPR_ERR_CUDA,
                     "cudaMalloc(%zu bytes): %s", bytes, cudaGetErrorString(e));
    }
    *p = static_cast<T*>(q);
    b->bytes += bytes;
    return MPR_OK;
}

void bfree_all(mpr_batch_ctx* b)
{
    for (auto& g : b->gexec)
        if (g) cudaGraphExecDestroy(g);
    void* ptrs[] = {b->d_lists, b->dArgs, b->dP, b->ctl, b->d_tile_prob, b->ang, b->mb, b->acc, b->acc_hi, b->acc_lo, b->part32,
                    b->epart, b->zpool, b->mpool, b->range, b->scal, b->part, b->tmp};
    for (void* p : ptrs)
        if (p) cudaFree(p);
}

Layout layout_of(const Prob& p)
{
    Layout L;
    L.Lx = p.Lx;
    L.Ly = p.Ly;
    L.Lxh = p.Lxh;
    L.pitch = p.pitch;
    L.mpitch = p.mpitch;
    return L;
}

// Tile list for a tile shape: problem by problem, row-major tiles; then the order in which the
// blocks take them: by the number of lattice entries they cover, largest first.
mpr_status build_tiles(mpr_batch_ctx* b, int shape)
{
    if (b->tiled_shape == shape) return MPR_OK;
    const int TY = batch::shape_rows(shape), TJ = batch::shape_cols(shape);
    // 128-column shapes with an even row count per thread run a last tile column of at most 64
    // columns as a 64-column tile, and with a row count per thread divisible by 4 one of at most
    // 32 columns as a 32-column tile (see do_tile)
    const bool tail = TJ == 128 && batch::kShape[shape].rpt % 2 == 0;
    const bool tail32 = TJ == 128 && batch::kShape[shape].rpt % 4 == 0;
    b->tile_prob.clear();
    std::vector<long long> cost;
    for (int i = 0; i < b->n; ++i) {
        Prob& p = b->P[(size_t)i];
        p.ntx = (p.Lxh + TJ - 1) / TJ;
        p.nty = (p.Ly + TY - 1) / TY;
        p.ntiles = p.ntx * p.nty;
        const int rem = p.Lxh - (p.ntx - 1) * TJ;   // columns of the last tile column
        p.tail = tail32 && rem <= 32 ? 32 : (tail && rem <= 64 ? 64 : 0);
        p.tile_base = (int)b->tile_prob.size();
        for (int t = 0; t < p.ntiles; ++t) {
            b->tile_prob.push_back(i);
            const int tx = t % p.ntx, ty = t / p.ntx;
            const long long w = std::min(TJ, p.Lxh - tx * TJ), h = std::min(TY, p.Ly - ty * TY);
            // cost of a tile: the lattice entries its block sweeps (a tail tile: its width)
            const long long wt = (p.tail && tx == p.ntx - 1) ? std::min((long long)p.tail, w) : w;
            cost.push_back(wt * h);
        }
    }
    b->ntiles = (int)b->tile_prob.size();
    std::vector<int> order((size_t)b->ntiles);
    for (int t = 0; t < b->ntiles; ++t) order[(size_t)t] = t;
    std::stable_sort(order.begin(), order.end(),
                     [&](int x, int y) { return cost[(size_t)x] > cost[(size_t)y]; });
    b->order = order;
    if (b->ntiles > b->tile_cap) {
        if (b->d_tile_prob) cudaFree(b->d_tile_prob);
        if (b->d_lists) cudaFree(b->d_lists);
        if (b->epart) cudaFree(b->epart);
        b->d_tile_prob = nullptr;
        b->d_lists = nullptr;
        b->epart = nullptr;
        BCHECK(balloc(b, &b->d_tile_prob, (size_t)b->ntiles * sizeof(int)));
        BCHECK(balloc(b, &b->d_lists, 2 * (size_t)b->ntiles * sizeof(int2)));
        BCHECK(balloc(b, &b->epart, (size_t)b->ntiles * sizeof(double)));
        b->tile_cap = b->ntiles;
    }
    BCU(cudaMemcpyAsync(b->d_tile_prob, b->tile_prob.data(), (size_t)b->ntiles * sizeof(int),
                        cudaMemcpyHostToDevice, b->stream));
    b->tiled_shape = shape;
    return MPR_OK;
}

mpr_status default_shape(mpr_batch_ctx* b)
{
    if (b->bps > 0) return MPR_OK;
    int occ = 0;
    BCU(batch_occupancy(b->prec.store, b->shape, &occ));
    if (occ < 1) return bfail(MPR_ERR_CUDA, "batched kernel cannot be resident on an SM");
    b->bps = occ;
    return MPR_OK;
}

// One cooperative launch: the whole batch to completion (or a device-side timeout).
mpr_status launch_fill(mpr_batch_ctx* b, bool tune, int equil, int samples, float* ms_out)
{
    BCHECK(default_shape(b));
    BCHECK(build_tiles(b, b->shape));
    int occ = 0;
    BCU(batch_occupancy(b->prec.store, b->shape, &occ));
    const int bps = b->bps < occ ? b->bps : occ;
    const int grid = b->sms * bps;
    int active = 0;
    for (int i = 0; i < b->n; ++i) active += b->P[(size_t)i].d.phase != batch::kDone;
    BCU(cudaMemcpyAsync(b->dP, b->P.data(), sizeof(Prob) * (size_t)b->n, cudaMemcpyHostToDevice,
                        b->stream));
    b->list.clear();
    for (int t : b->order) {
        const int p = b->tile_prob[(size_t)t];
        if (b->P[(size_t)p].d.phase != batch::kDone) b->list.push_back(make_int2(t, p));
    }
    if (!b->list.empty())
        BCU(cudaMemcpyAsync(b->d_lists, b->list.data(), b->list.size() * sizeof(int2),
                            cudaMemcpyHostToDevice, b->stream));
    batch::Ctl c{};
    c.n_active = active;
    c.list_sel = 0;
    c.n_list = (int)b->list.size();
    c.timeout_ns = (long long)(b->timeout_s * 1e9);
    c.bar_extra = b->bar_extra;
    BCU(cudaMemcpyAsync(b->ctl, &c, sizeof c, cudaMemcpyHostToDevice, b->stream));
    batch::Args A{};
    A.prob = b->dP;
    A.nprob = b->n;
    A.tile_prob = b->d_tile_prob;
    A.lists = b->d_lists;
    A.ntiles = b->ntiles;
    A.ang = b->ang;
    A.mb = b->mb;
    A.acc = b->acc;
    A.acc_hi = b->acc_hi;
    A.acc_lo = b->acc_lo;
    A.part32 = b->part32;
    A.epart = b->epart;
    A.ctl = b->ctl;
    A.n_eq = b->tune.n_eq;
    A.n_meas = b->tune.n_meas;
    A.max_probes = b->tune.max_probes;
    A.equil = equil;
    A.samples = samples;
    A.energy_f32 = b->prec.energy == 1;
    A.acc_kind = b->prec.acc;
    A.max_iters = (tune ? b->tune.max_probes * (b->tune.n_eq + b->tune.n_meas) : 0) + equil + samples + 2;
    A.T_lo = b->tune.T_lo;
    A.T_hi = b->tune.T_hi;
    A.rel_tol = b->tune.rel_tol;
    A.log_ratio = log(b->tune.ratio_tol);
    A.seed_lo = (uint32_t)b->opt.seed;
    A.seed_hi = (uint32_t)(b->opt.seed >> 32);
    A.q = b->opt.q;
    A.qf = (float)b->opt.q;
    // round keys of the batch's seed for the tile kernels' parameter (counter parts unused)
    const PhiloxSched keys = philox_sched(0u, 0u, kTagMetropolis, 0u, A.seed_lo, A.seed_hi);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    BCU(cudaEventCreate(&e0));
    BCU(cudaEventCreate(&e1));
    BCU(cudaEventRecord(e0, b->stream));
    if (active > 0) {
        if (!b->dArgs) BCHECK(balloc(b, &b->dArgs, sizeof(batch::Args)));
        BCU(cudaMemcpyAsync(b->dArgs, &A, sizeof A, cudaMemcpyHostToDevice, b->stream));
        if (b->use_graph == 2) {
            cudaGraphExec_t& ge = b->gexec[b->shape];
            const bool qhalf = A.qf == 0.5f;
            if (ge && (b->gexec_tiles[b->shape] != b->ntiles || b->gexec_qhalf[b->shape] != qhalf)) {
                cudaGraphExecDestroy(ge);
                ge = nullptr;
            }
            if (!ge) {
                BCU(batch_graph_build(b->prec.store, b->shape, b->ntiles, qhalf, b->dArgs, keys, &ge));
                b->gexec_tiles[b->shape] = b->ntiles;
                b->gexec_qhalf[b->shape] = qhalf;
            }
            BCU(cudaGraphLaunch(ge, b->stream));
        } else {
            BCU(batch_launch(b->prec.store, b->shape, grid, b->dArgs, keys, b->stream,
                             b->use_graph != 0));
        }
        b->launches += 1;
    }
    BCU(cudaEventRecord(e1, b->stream));
    BCU(cudaMemcpyAsync(&c, b->ctl, sizeof c, cudaMemcpyDeviceToHost, b->stream));
    BCU(cudaMemcpyAsync(b->P.data(), b->dP, sizeof(Prob) * (size_t)b->n, cudaMemcpyDeviceToHost,
                        b->stream));
    BCU(cudaStreamSynchronize(b->stream));
    BCU(cudaEventElapsedTime(&b->last_ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (ms_out) *ms_out = b->last_ms;
    b->last_iters = c.iters;
    b->bar_extra = 0;
    if (c.err) {
        b->broken = true;
        return bfail(MPR_ERR_DEVICE_TIMEOUT,
                     "a grid-barrier wait of the batched kernel ran out (%.3f s limit); the batch "
                     "state is undefined, destroy it", b->timeout_s);
    }
    for (int i = 0; i < b->n; ++i)
        if (b->P[(size_t)i].d.phase != batch::kDone)
            return bfail(MPR_ERR_STATE, "problem %d did not finish within the iteration bound", i);
    return MPR_OK;
}

void prepare_fill(mpr_batch_ctx* b, const double* T)
{
    for (int i = 0; i < b->n; ++i) {
        batch::Dyn& d = b->P[(size_t)i].d;
        d.invTf = (float)(1.0 / (T ? T[i] : b->tune.T_lo));
        d.status = MPR_OK;
        d.esum = 0.0;
        d.step = 0;
        d.lo = log(b->tune.T_lo);
        d.hi = log(b->tune.T_hi);
        d.mid = 0.0;
        d.np = 0;
        if (T) {
            d.T = T[i];
            d.kind = 0;
            d.phase = batch::kRunEquil;   // adjusted by the caller when equil == 0
        } else {
            d.kind = 0;
            d.T = b->tune.T_lo;
            d.phase = b->tune.n_eq > 0 ? batch::kProbeEquil : batch::kProbeMeasure;
        }
    }
}

}  // namespace

extern "C" {

mpr_status mpr_batch_create(int n, const int* Lx, const int* Ly, const double* const* values,
                            const unsigned char* const* mask, const mpr_options* opt,
                            mpr_batch* out)
{
    if (!out) return bfail(MPR_ERR_INVALID_ARG, "out pointer is NULL");
    *out = nullptr;
    if (n < 1 || !Lx || !Ly || !values || !mask)
        return bfail(MPR_ERR_INVALID_ARG, "need n >= 1 and non-NULL size, value and mask arrays");
    for (int i = 0; i < n; ++i) {
        if (Lx[i] < 2 || Ly[i] < 2 || (long long)Lx[i] * Ly[i] > 2147483647LL || !values[i] || !mask[i])
            return bfail(MPR_ERR_INVALID_ARG, "problem %d: bad size %d x %d or NULL data", i, Lx[i], Ly[i]);
    }
    mpr_options o;
    if (opt) {
        o = *opt;
    } else {
        memset(&o, 0, sizeof o);
        o.q = 0.5;
        o.store = MPR_STORE_F32;
        o.energy = MPR_PREC_D;
        o.func = MPR_PREC_S;
        o.acc = MPR_ACC_F64;
    }
    if (o.q == 0.0) o.q = 0.5;
    if (!(o.q > 0.0 && o.q <= 1.0) || o.store < 0 || o.store > 3 || o.energy < 0 || o.energy > 1 ||
        o.acc < 0 || o.acc > 1)
        return bfail(MPR_ERR_INVALID_ARG, "options out of range");
    if (o.func != MPR_PREC_S)
        return bfail(MPR_ERR_INVALID_ARG, "the batched path computes with FP32 functions (func = S)");
    mpr_batch_ctx* b = new (std::nothrow) mpr_batch_ctx();
    if (!b) return bfail(MPR_ERR_OOM, "host allocation failed");
    auto bail = [&](mpr_status s) {
        bfree_all(b);
        delete b;
        return s;
    };
    b->n = n;
    b->opt = o;
    b->prec = Precision{o.store, o.energy, o.func, o.acc};
    b->tune = mpr_tuning{200, 50, 1e-3, 10.0, 1e-3, 1.001, 30};
    if (cudaGetDevice(&b->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device) != cudaSuccess)
        return bail(bfail(MPR_ERR_CUDA, "no CUDA device"));
    int coop = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, b->device);
    if (!coop) return bail(bfail(MPR_ERR_CUDA, "device does not support cooperative launches"));

    // layout of every problem in the pools
    b->P.resize((size_t)n);
    b->zmin.resize((size_t)n);
    b->zmax.resize((size_t)n);
    b->N.resize((size_t)n);
    b->Nss.resize((size_t)n);
    b->z_off.resize((size_t)n);
    const size_t sb = store_bytes(o.store);
    for (int i = 0; i < n; ++i) {
        Prob& p = b->P[(size_t)i];
        memset(&p, 0, sizeof p);
        p.Lx = Lx[i];
        p.Ly = Ly[i];
        p.Lxh = (Lx[i] + 1) / 2;
        p.pitch = (p.Lxh + 127) / 128 * 128;
        p.mpitch = p.pitch / 32;
        for (int c = 0; c < 2; ++c) {
            p.ang_off[c] = b->ang_elems;
            b->ang_elems += (long long)p.Ly * p.pitch;
            p.mb_off[c] = b->mb_words;
            b->mb_words += (long long)p.Ly * p.mpitch;
            p.acc_off[c] = b->acc_elems;
            b->acc_elems += (long long)p.Ly * p.pitch;
        }
        b->N[(size_t)i] = (long long)Lx[i] * Ly[i];
        b->z_off[(size_t)i] = b->z_elems;
        b->z_elems += b->N[(size_t)i];
        if (b->N[(size_t)i] > b->maxN) b->maxN = b->N[(size_t)i];
        p.Nb = (double)Lx[i] * (Ly[i] - 1) + (double)Ly[i] * (Lx[i] - 1);
    }
    mpr_status s;
    b->part_bytes = 1024 * 16;
    if ((s = balloc(b, &b->dP, sizeof(Prob) * (size_t)n)) != MPR_OK ||
        (s = balloc(b, &b->ctl, sizeof(batch::Ctl))) != MPR_OK ||
        (s = balloc(b, &b->ang, (size_t)b->ang_elems * sb)) != MPR_OK ||
        (s = balloc(b, &b->mb, (size_t)b->mb_words * 4)) != MPR_OK ||
        (s = balloc(b, &b->zpool, (size_t)b->z_elems * 8)) != MPR_OK ||
        (s = balloc(b, &b->mpool, (size_t)b->z_elems)) != MPR_OK ||
        (s = balloc(b, &b->range, (size_t)n * 2 * 8)) != MPR_OK ||
        (s = balloc(b, &b->scal, (size_t)n * 8 * 8)) != MPR_OK ||
        (s = balloc(b, &b->part, b->part_bytes)) != MPR_OK ||
        (s = balloc(b, &b->tmp, (size_t)b->maxN * 8)) != MPR_OK)
        return bail(s);
    if (o.acc == MPR_ACC_F64) {
        if ((s = balloc(b, &b->acc, (size_t)b->acc_elems * 8)) != MPR_OK) return bail(s);
        if (cudaMemset(b->acc, 0, (size_t)b->acc_elems * 8) != cudaSuccess)
            return bail(bfail(MPR_ERR_CUDA, "memset failed"));
        if (o.store == MPR_STORE_F16) {   // exact fixed-point sample partials (FP16 values)
            if ((s = balloc(b, &b->part32, (size_t)b->acc_elems * 4)) != MPR_OK) return bail(s);
            if (cudaMemset(b->part32, 0, (size_t)b->acc_elems * 4) != cudaSuccess)
                return bail(bfail(MPR_ERR_CUDA, "memset failed"));
        }
    } else {
        if ((s = balloc(b, &b->acc_hi, (size_t)b->acc_elems * 4)) != MPR_OK ||
            (s = balloc(b, &b->acc_lo, (size_t)b->acc_elems * 4)) != MPR_OK)
            return bail(s);
        if (cudaMemset(b->acc_hi, 0, (size_t)b->acc_elems * 4) != cudaSuccess ||
            cudaMemset(b->acc_lo, 0, (size_t)b->acc_elems * 4) != cudaSuccess)
            return bail(bfail(MPR_ERR_CUDA, "memset failed"));
    }
    // inputs, range of every problem
    for (int i = 0; i < n; ++i) {
        const long long Ni = b->N[(size_t)i];
        double* z = b->zpool + b->z_off[(size_t)i];
        unsigned char* m = b->mpool + b->z_off[(size_t)i];
        if (cudaMemcpyAsync(z, values[i], (size_t)Ni * 8, cudaMemcpyHostToDevice, b->stream) != cudaSuccess ||
            cudaMemcpyAsync(m, mask[i], (size_t)Ni, cudaMemcpyHostToDevice, b->stream) != cudaSuccess ||
            launch_minmax(z, m, Ni, b->part, 256, b->scal + 8 * i, b->stream) != cudaSuccess)
            return bail(bfail(MPR_ERR_CUDA, "problem %d: input copy or range failed", i));
        b->launches += 2;
        // the range feeds the mapping and the prediction of this problem
        if (cudaMemcpyAsync(b->range + 2 * i, b->scal + 8 * i, 16, cudaMemcpyDeviceToDevice,
                            b->stream) != cudaSuccess)
            return bail(bfail(MPR_ERR_CUDA, "range copy failed"));
    }
    std::vector<double> sc((size_t)n * 8);
    if (cudaMemcpyAsync(sc.data(), b->scal, sc.size() * 8, cudaMemcpyDeviceToHost, b->stream) != cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess)
        return bail(bfail(MPR_ERR_CUDA, "range read-back failed"));
    for (int i = 0; i < n; ++i) {
        const double lo = sc[8 * (size_t)i], hi = sc[8 * (size_t)i + 1];
        const double nm = sc[8 * (size_t)i + 2], bad = sc[8 * (size_t)i + 3];
        if (bad > 0) return bail(bfail(MPR_ERR_INVALID_ARG, "problem %d: %.0f measured values are NaN or infinite", i, bad));
        if (nm < 2 || !(hi > lo)) return bail(bfail(MPR_ERR_DEGENERATE, "problem %d: degenerate data", i));
        b->zmin[(size_t)i] = lo;
        b->zmax[(size_t)i] = hi;
        b->P[(size_t)i].Np = b->N[(size_t)i] - (long long)nm;
    }
    // mapping + initial angles (Philox problem id = index), sample energy
    for (int i = 0; i < n; ++i) {
        Prob& p = b->P[(size_t)i];
        const Layout L = layout_of(p);
        double* z = b->zpool + b->z_off[(size_t)i];
        unsigned char* m = b->mpool + b->z_off[(size_t)i];
        char* ang = static_cast<char*>(b->ang);
        if (launch_init(L, b->prec, z, m, b->range + 2 * i, ang + (size_t)p.ang_off[0] * sb,
                        ang + (size_t)p.ang_off[1] * sb, b->mb + p.mb_off[0], b->mb + p.mb_off[1],
                        o.seed, (uint32_t)i, b->stream) != cudaSuccess)
            return bail(bfail(MPR_ERR_CUDA, "problem %d: init failed", i));
        const int nb = sample_energy_blocks(L) < 512 ? sample_energy_blocks(L) : 512;
        if (launch_sample_energy(L, z, m, b->range + 2 * i, o.q, b->part,
                                 reinterpret_cast<long long*>(b->part + 512), nb, b->scal + 8 * i + 4,
                                 b->stream) != cudaSuccess)
            return bail(bfail(MPR_ERR_CUDA, "problem %d: sample energy failed", i));
        b->launches += 3;
    }
    if (cudaMemcpyAsync(sc.data(), b->scal, sc.size() * 8, cudaMemcpyDeviceToHost, b->stream) != cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess)
        return bail(bfail(MPR_ERR_CUDA, "sample energy read-back failed"));
    for (int i = 0; i < n; ++i) {
        b->P[(size_t)i].e_s = sc[8 * (size_t)i + 4];
        b->Nss[(size_t)i] = (long long)sc[8 * (size_t)i + 5];
        if (b->Nss[(size_t)i] == 0)
            return bail(bfail(MPR_ERR_NO_PAIRS, "problem %d: no two measured sites are neighbours", i));
        b->P[(size_t)i].d.phase = batch::kDone;
    }
    *out = b;
    return MPR_OK;
}

void mpr_batch_destroy(mpr_batch b)
{
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    bfree_all(b);
    delete b;
}

mpr_status mpr_batch_set_stream(mpr_batch b, void* stream)
{
    if (!b) return bfail(MPR_ERR_INVALID_ARG, "batch is NULL");
    BCU(cudaStreamSynchronize(b->stream));
    b->stream = static_cast<cudaStream_t>(stream);
    b->tiled_shape = -1;   // re-upload the tile list on the new stream
    return MPR_OK;
}

mpr_status mpr_batch_set_tuning(mpr_batch b, const mpr_tuning* t)
{
    if (!b || !t) return bfail(MPR_ERR_INVALID_ARG, "NULL argument");
    if (t->n_eq < 0 || t->n_meas < 1 || !(t->T_lo > 0) || !(t->T_hi > t->T_lo) ||
        !(t->rel_tol >= 0) || !(t->ratio_tol > 1.0) || t->max_probes < 2 || t->max_probes > 64)
        return bfail(MPR_ERR_INVALID_ARG, "tuning parameters out of range");
    b->tune = *t;
    return MPR_OK;
}

mpr_status mpr_batch_set_launch(mpr_batch b, int tile_rows, int tile_cols, int blocks_per_sm,
                                int use_graph)
{
    if (!b) return bfail(MPR_ERR_INVALID_ARG, "batch is NULL");
    int shape = -1;
    for (int s = 0; s < batch::kShapes; ++s)
        if (batch::shape_rows(s) == tile_rows && batch::shape_cols(s) == tile_cols) shape = s;
    if (shape < 0)
        return bfail(MPR_ERR_INVALID_ARG,
                     "tile %d x %d: use 8, 16 or 32 rows x 128 columns, or 16 or 32 rows x 64 columns",
                     tile_rows, tile_cols);
    int occ = 0;
    BCU(batch_occupancy(b->prec.store, shape, &occ));
    if (blocks_per_sm < 0 || blocks_per_sm > occ)
        return bfail(MPR_ERR_INVALID_ARG, "blocks per SM must be in [0, %d] (0 = occupancy limit)", occ);
    if (use_graph < 0 || use_graph > 2) return bfail(MPR_ERR_INVALID_ARG, "mode must be 0, 1 or 2");
    b->shape = shape;
    b->bps = blocks_per_sm;
    b->use_graph = use_graph;
    return MPR_OK;
}

mpr_status mpr_batch_fill(mpr_batch b, const double* T, int equil, int samples, double* T_out,
                          int* status_out)
{
    NvtxRange r("mpr_batch_fill");
    if (!b) return bfail(MPR_ERR_INVALID_ARG, "batch is NULL");
    if (b->broken) return bfail(MPR_ERR_STATE, "the batch was left undefined by a device timeout");
    if (equil < 0 || samples < 0) return bfail(MPR_ERR_INVALID_ARG, "negative sweep count");
    if (T)
        for (int i = 0; i < b->n; ++i)
            if (!(T[i] > 0.0) || !isfinite(T[i]))
                return bfail(MPR_ERR_INVALID_ARG, "problem %d: temperature %g must be > 0", i, T[i]);
    prepare_fill(b, T);
    for (int i = 0; i < b->n; ++i) {
        batch::Dyn& d = b->P[(size_t)i].d;
        if (T) d.phase = equil > 0 ? batch::kRunEquil : (samples > 0 ? batch::kRunSample : batch::kDone);
        if (samples > 0) {   // this fill's samples give the mean bond energy
            d.esamp = 0.0;
            d.nfill = 0;
        }
    }
    BCHECK(launch_fill(b, T == nullptr, equil, samples, nullptr));
    int worst = MPR_OK;
    for (int i = 0; i < b->n; ++i) {
        const batch::Dyn& d = b->P[(size_t)i].d;
        if (T_out) T_out[i] = d.T;
        if (status_out) status_out[i] = d.status;
        if (d.status != MPR_OK) worst = d.status;
    }
    if (worst != MPR_OK)
        return bfail((mpr_status)worst, "the tuning of at least one problem did not converge");
    return MPR_OK;
}

mpr_status mpr_batch_autotune(mpr_batch b, int sweeps, int* tile_rows_out, int* tile_cols_out,
                              int* blocks_per_sm_out)
{
    if (!b) return bfail(MPR_ERR_INVALID_ARG, "batch is NULL");
    if (b->broken) return bfail(MPR_ERR_STATE, "the batch was left undefined by a device timeout");
    if (sweeps < 1) sweeps = 10;
    long long total = 0;
    for (long long v : b->N) total += v;
    const auto key = std::make_tuple(b->n, total, b->prec.store, b->prec.energy);
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            b->shape = std::get<0>(it->second);
            b->bps = std::get<1>(it->second);
            b->use_graph = std::get<2>(it->second);
            if (tile_rows_out) *tile_rows_out = batch::shape_rows(b->shape);
            if (tile_cols_out) *tile_cols_out = batch::shape_cols(b->shape);
            if (blocks_per_sm_out) *blocks_per_sm_out = b->bps;
            return MPR_OK;
        }
    }
    // time every candidate on a copy of the state, then put the state back
    const size_t ang_bytes = (size_t)b->ang_elems * store_bytes(b->prec.store);
    void* saved = nullptr;
    BCU(cudaMalloc(&saved, ang_bytes));
    BCU(cudaMemcpyAsync(saved, b->ang, ang_bytes, cudaMemcpyDeviceToDevice, b->stream));
    const std::vector<Prob> keep = b->P;
    std::vector<double> T((size_t)b->n);
    for (int i = 0; i < b->n; ++i) T[(size_t)i] = keep[(size_t)i].d.T > 0 ? keep[(size_t)i].d.T : 0.5;
    float best = 1e30f;
    int best_shape = b->shape, best_bps = b->bps, best_mode = b->use_graph;
    mpr_status st = MPR_OK;
    for (int r = 0; r < batch::kShapes; ++r) {
        // graph mode (one block per tile, device-side loop)
        b->shape = r;
        b->bps = 0;
        b->use_graph = 2;
        prepare_fill(b, T.data());
        float ms = 0.f;
        st = launch_fill(b, false, sweeps, 0, &ms);
        if (st != MPR_OK) break;
        if (ms < best) {
            best = ms;
            best_shape = r;
            best_bps = 0;
            best_mode = 2;
        }
        // persistent cooperative kernel at every residency
        int occ = 0;
        if (batch_occupancy(b->prec.store, r, &occ) != cudaSuccess) continue;
        for (int bps = 1; bps <= occ; ++bps) {
            b->shape = r;
            b->bps = bps;
            b->use_graph = 0;
            prepare_fill(b, T.data());
            st = launch_fill(b, false, sweeps, 0, &ms);
            if (st != MPR_OK) break;
            if (ms < best) {
                best = ms;
                best_shape = r;
                best_bps = bps;
                best_mode = 0;
            }
        }
        if (st != MPR_OK) break;
    }
    cudaMemcpyAsync(b->ang, saved, ang_bytes, cudaMemcpyDeviceToDevice, b->stream);
    cudaStreamSynchronize(b->stream);
    cudaFree(saved);
    b->P = keep;
    b->tiled_shape = -1;   // the restored table holds an older tile layout: rebuild on next fill
    if (st != MPR_OK) return st;
    b->shape = best_shape;
    b->bps = best_bps;
    b->use_graph = best_mode;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune_cache[key] = std::make_tuple(best_shape, best_bps, best_mode);
    }
    if (tile_rows_out) *tile_rows_out = batch::shape_rows(best_shape);
    if (tile_cols_out) *tile_cols_out = batch::shape_cols(best_shape);
    if (blocks_per_sm_out) *blocks_per_sm_out = best_bps;
    return MPR_OK;
}

mpr_status mpr_batch_predict(mpr_batch b, int i, double* out)
{
    if (!b || !out || i < 0 || i >= b->n) return bfail(MPR_ERR_INVALID_ARG, "bad batch, index or output");
    const Prob& p = b->P[(size_t)i];
    if (p.d.nsamples == 0) return bfail(MPR_ERR_STATE, "problem %d has no samples", i);
    const Layout L = layout_of(p);
    const double* z = b->zpool + b->z_off[(size_t)i];
    const unsigned char* m = b->mpool + b->z_off[(size_t)i];
    const bool f64 = b->acc != nullptr;
    BCU(launch_predict(L, b->prec, z, m, b->range + 2 * i, f64 ? b->acc + p.acc_off[0] : nullptr,
                       f64 ? b->acc + p.acc_off[1] : nullptr,
                       f64 ? nullptr : b->acc_hi + p.acc_off[0], f64 ? nullptr : b->acc_lo + p.acc_off[0],
                       f64 ? nullptr : b->acc_hi + p.acc_off[1], f64 ? nullptr : b->acc_lo + p.acc_off[1],
                       p.d.nsamples, b->tmp, b->stream));
    b->launches += 1;
    BCU(cudaMemcpyAsync(out, b->tmp, (size_t)b->N[(size_t)i] * 8, cudaMemcpyDeviceToHost, b->stream));
    BCU(cudaStreamSynchronize(b->stream));
    return MPR_OK;
}

mpr_status mpr_batch_get_state(mpr_batch b, int i, double* angles, uint32_t* sweep)
{
    if (!b || !angles || i < 0 || i >= b->n) return bfail(MPR_ERR_INVALID_ARG, "bad batch, index or output");
    const Prob& p = b->P[(size_t)i];
    const size_t sb = store_bytes(b->prec.store);
    const char* ang = static_cast<const char*>(b->ang);
    BCU(launch_get_state(layout_of(p), b->prec, ang + (size_t)p.ang_off[0] * sb,
                         ang + (size_t)p.ang_off[1] * sb, b->tmp, b->stream));
    b->launches += 1;
    BCU(cudaMemcpyAsync(angles, b->tmp, (size_t)b->N[(size_t)i] * 8, cudaMemcpyDeviceToHost, b->stream));
    BCU(cudaStreamSynchronize(b->stream));
    if (sweep) *sweep = p.d.sweep;
    return MPR_OK;
}

mpr_status mpr_batch_get_info(mpr_batch b, int i, mpr_info* info)
{
    if (!b || !info || i < 0 || i >= b->n) return bfail(MPR_ERR_INVALID_ARG, "bad batch, index or output");
    const Prob& p = b->P[(size_t)i];
    memset(info, 0, sizeof *info);
    info->Lx = p.Lx;
    info->Ly = p.Ly;
    info->n_sites = b->N[(size_t)i];
    info->n_pred = p.Np;
    info->n_bonds = (int64_t)p.Nb;
    info->n_sample_pairs = b->Nss[(size_t)i];
    info->zmin = b->zmin[(size_t)i];
    info->zmax = b->zmax[(size_t)i];
    info->e_sample = p.e_s;
    info->T = p.d.T;
    info->sweep = p.d.sweep;
    info->n_samples = p.d.nsamples;
    info->n_probes = p.d.np;
    info->e_bond_mean = p.d.nfill > 0 ? p.d.esamp / (double)p.d.nfill : NAN;
    info->site_updates = p.d.site_updates;
    info->device_bytes = b->bytes;
    info->kernel_launches = b->launches;
    info->sweep_kernel = 0;   // batch tiles are staged with ordinary loads
    return MPR_OK;
}

mpr_status mpr_batch_get_stats(mpr_batch b, int* iterations, double* fill_ms, int* tile_rows,
                               int* tile_cols, int* blocks_per_sm, int* mode)
{
    if (!b) return bfail(MPR_ERR_INVALID_ARG, "batch is NULL");
    if (mode) *mode = b->use_graph;
    if (iterations) *iterations = b->last_iters;
    if (fill_ms) *fill_ms = (double)b->last_ms;
    if (tile_rows) *tile_rows = batch::shape_rows(b->shape);
    if (tile_cols) *tile_cols = batch::shape_cols(b->shape);
    if (blocks_per_sm) *blocks_per_sm = b->bps;
    return MPR_OK;
}

mpr_status mpr_batch_inject_barrier_fault(mpr_batch b, int extra_arrivals, double timeout_s)
{
    if (!b) return bfail(MPR_ERR_INVALID_ARG, "batch is NULL");
    if (extra_arrivals < 0 || !(timeout_s > 0.0) || timeout_s > 60.0)
        return bfail(MPR_ERR_INVALID_ARG, "extra arrivals >= 0, timeout in (0, 60] s");
    b->bar_extra = extra_arrivals;
    b->timeout_s = timeout_s;
    return MPR_OK;
}

}  // extern "C"
