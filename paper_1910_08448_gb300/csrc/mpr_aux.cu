// mpr_aux.cu -- the non-sweep kernels of libmpr: range of the measured data, data -> spin
// mapping with the initial angles and the frozen-site bits, sample energy e_s, FP64 bond energy
// of a state, deterministic fixed-order reductions, prediction and state transfer.
//
// Every reduction writes per-block partials and sums them in a fixed order in a second kernel,
// so results do not depend on scheduling (no floating-point atomics).
#include "mpr_device.cuh"
#include "mpr_internal.h"

#include <math.h>

namespace mpr {
namespace {

constexpr int kThreads = 256;

// --------------------------------------------------------------------------------------------
// Range of the measured values: partial (min, max, count, non-finite count) per block.
// --------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) minmax_kernel(const double* __restrict__ z,
                                                          const unsigned char* __restrict__ mask,
                                                          long long N, double* __restrict__ part)
{
    double lo = INFINITY, hi = -INFINITY, n = 0.0, bad = 0.0;
    for (long long s = blockIdx.x * (long long)kThreads + threadIdx.x; s < N;
         s += (long long)gridDim.x * kThreads) {
        if (!mask[s]) continue;
        const double v = z[s];
        if (!isfinite(v)) { bad += 1.0; continue; }
        lo = fmin(lo, v);
        hi = fmax(hi, v);
        n += 1.0;
    }
    __shared__ double sh[4][kThreads];
    sh[0][threadIdx.x] = lo;
    sh[1][threadIdx.x] = hi;
    sh[2][threadIdx.x] = n;
    sh[3][threadIdx.x] = bad;
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            sh[0][threadIdx.x] = fmin(sh[0][threadIdx.x], sh[0][threadIdx.x + w]);
            sh[1][threadIdx.x] = fmax(sh[1][threadIdx.x], sh[1][threadIdx.x + w]);
            sh[2][threadIdx.x] += sh[2][threadIdx.x + w];
            sh[3][threadIdx.x] += sh[3][threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int k = 0; k < 4; ++k) part[4 * blockIdx.x + k] = sh[k][0];
}

__global__ void minmax_final(const double* __restrict__ part, int nblk, double* __restrict__ out)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double lo = INFINITY, hi = -INFINITY, n = 0.0, bad = 0.0;
    for (int b = 0; b < nblk; ++b) {
        lo = fmin(lo, part[4 * b]);
        hi = fmax(hi, part[4 * b + 1]);
        n += part[4 * b + 2];
        bad += part[4 * b + 3];
    }
    out[0] = lo;
    out[1] = hi;
    out[2] = n;
    out[3] = bad;
}

// --------------------------------------------------------------------------------------------
// Mapping phi = 2*pi*(z - zmin)/(zmax - zmin) on measured sites, uniform initial angles on the
// prediction sites (init stream, sweep 0), packed by colour; one warp ballot per mask word.
// --------------------------------------------------------------------------------------------
template <typename S>
__global__ void __launch_bounds__(kThreads) init_kernel(Layout L, const double* __restrict__ z,
                                                        const unsigned char* __restrict__ mask,
                                                        const double* __restrict__ range,
                                                        S* __restrict__ ang0, S* __restrict__ ang1,
                                                        uint32_t* __restrict__ mb0,
                                                        uint32_t* __restrict__ mb1, uint32_t seed_lo,
                                                        uint32_t seed_hi, uint32_t problem,
                                                        int fp32_uniform)
{
    const int j = blockIdx.x * kThreads + threadIdx.x;
    if (j >= L.pitch) return;   // pitch is a multiple of 32: whole warps leave together
    const int c = blockIdx.z;
    for (int y = blockIdx.y; y < L.Ly; y += gridDim.y) {   // rows beyond the 65535 grid limit
        const int x = 2 * j + ((y + c) & 1);
        S* ang = c ? ang1 : ang0;
        uint32_t* mb = c ? mb1 : mb0;
        const size_t idx = (size_t)y * L.pitch + j;
        bool frozen = true;   // padding counts as frozen: never updated
        if (x < L.Lx) {
            const size_t s = (size_t)y * L.Lx + x;
            double phi;
            if (mask[s]) {
                const double lo = range[0], hi = range[1];
                const double t = (z[s] - lo) / (hi - lo);
                phi = kTwoPi * t;
            } else {
                frozen = false;
                const uint4 w = pair_words((uint32_t)(j >> 1), (uint32_t)y, 0u, problem, kTagInit,
                                           (uint32_t)c, seed_lo, seed_hi);
                const uint32_t wp = (j & 1) ? w.z : w.x;
                const double u = fp32_uniform ? (double)uniform_f(wp) : uniform_d(wp);
                phi = kTwoPi * u;
            }
            ang[idx] = store_from<S>(phi);
        } else {
            ang[idx] = store_from<S>(0.0);
        }
        const uint32_t bits = __ballot_sync(0xffffffffu, frozen);
        if ((threadIdx.x & 31) == 0) mb[(size_t)y * L.mpitch + (j >> 5)] = bits;
    }
}

// --------------------------------------------------------------------------------------------
// Sample energy: sum of cos[q(phi_i - phi_j)] over measured-measured bonds, in FP64 from the
// mapped values, and the number of such bonds.
// --------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) sample_energy_kernel(Layout L,
                                                                 const double* __restrict__ z,
                                                                 const unsigned char* __restrict__ mask,
                                                                 const double* __restrict__ range,
                                                                 double q, double* __restrict__ psum,
                                                                 long long* __restrict__ pcnt)
{
    const long long N = (long long)L.Lx * L.Ly;
    const double lo = range[0], hi = range[1];
    double sum = 0.0;
    long long cnt = 0;
    for (long long s = blockIdx.x * (long long)kThreads + threadIdx.x; s < N;
         s += (long long)gridDim.x * kThreads) {
        if (!mask[s]) continue;
        const int y = (int)(s / L.Lx), x = (int)(s - (long long)y * L.Lx);
        const double ps = kTwoPi * ((z[s] - lo) / (hi - lo));
        if (x + 1 < L.Lx && mask[s + 1]) {
            const double pr = kTwoPi * ((z[s + 1] - lo) / (hi - lo));
            sum += cos(q * (ps - pr));
            ++cnt;
        }
        if (y + 1 < L.Ly && mask[s + L.Lx]) {
            const double pd = kTwoPi * ((z[s + L.Lx] - lo) / (hi - lo));
            sum += cos(q * (ps - pd));
            ++cnt;
        }
    }
    __shared__ double ss[kThreads];
    __shared__ long long sc[kThreads];
    ss[threadIdx.x] = sum;
    sc[threadIdx.x] = cnt;
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            ss[threadIdx.x] += ss[threadIdx.x + w];
            sc[threadIdx.x] += sc[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        psum[blockIdx.x] = ss[0];
        pcnt[blockIdx.x] = sc[0];
    }
}

__global__ void sample_energy_final(const double* __restrict__ psum, const long long* __restrict__ pcnt,
                                    int nblk, double* __restrict__ out)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double s = 0.0;
    long long n = 0;
    for (int b = 0; b < nblk; ++b) {
        s += psum[b];
        n += pcnt[b];
    }
    out[0] = n > 0 ? -s / (double)n : 0.0;
    out[1] = (double)n;
}

// --------------------------------------------------------------------------------------------
// FP64 bond energy of the current state: every bond joins a red and a black site, so the bond
// sum is the sum over black sites b of (cos q phi_b, sin q phi_b) . h_b.
// --------------------------------------------------------------------------------------------
template <typename S>
__global__ void __launch_bounds__(kThreads) energy_kernel(Layout L, const S* __restrict__ red,
                                                          const S* __restrict__ black, double q,
                                                          double* __restrict__ part)
{
    const long long n = (long long)L.Ly * L.Lxh;
    double sum = 0.0;
    for (long long e = blockIdx.x * (long long)kThreads + threadIdx.x; e < n;
         e += (long long)gridDim.x * kThreads) {
        const int y = (int)(e / L.Lxh), j = (int)(e - (long long)y * L.Lxh);
        const int o = (y + 1) & 1;   // black: x = 2j + ((y + 1) & 1)
        const int x = 2 * j + o;
        if (x >= L.Lx) continue;
        double hx = 0.0, hy = 0.0, sn, cs;
        if (x > 0) { sincos(q * load_as<double>(red[(size_t)y * L.pitch + j + o - 1]), &sn, &cs); hx += cs; hy += sn; }
        if (x + 1 < L.Lx) { sincos(q * load_as<double>(red[(size_t)y * L.pitch + j + o]), &sn, &cs); hx += cs; hy += sn; }
        if (y > 0) { sincos(q * load_as<double>(red[(size_t)(y - 1) * L.pitch + j]), &sn, &cs); hx += cs; hy += sn; }
        if (y + 1 < L.Ly) { sincos(q * load_as<double>(red[(size_t)(y + 1) * L.pitch + j]), &sn, &cs); hx += cs; hy += sn; }
        sincos(q * load_as<double>(black[(size_t)y * L.pitch + j]), &sn, &cs);
        sum += cs * hx + sn * hy;
    }
    __shared__ double ss[kThreads];
    ss[threadIdx.x] = sum;
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) ss[threadIdx.x] += ss[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = ss[0];
}

// Fixed-order sum of n partials: thread t adds entries t, t + 256, ... then a tree in shared memory.
template <typename E>
__global__ void __launch_bounds__(kThreads) reduce_kernel(const E* __restrict__ part, int n,
                                                          double* __restrict__ out)
{
    __shared__ E ss[kThreads];
    E s = (E)0;
    for (int i = threadIdx.x; i < n; i += kThreads) s += part[i];
    ss[threadIdx.x] = s;
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) ss[threadIdx.x] += ss[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = (double)ss[0];
}

// --------------------------------------------------------------------------------------------
// Prediction zhat = zmin + (zmax - zmin) * (mean phi / 2*pi) on prediction sites, z elsewhere.
// --------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) predict_kernel(Layout L, const double* __restrict__ z,
                                                           const unsigned char* __restrict__ mask,
                                                           const double* __restrict__ range,
                                                           const double* __restrict__ acc0,
                                                           const double* __restrict__ acc1,
                                                           const float* __restrict__ hi0,
                                                           const float* __restrict__ lo0,
                                                           const float* __restrict__ hi1,
                                                           const float* __restrict__ lo1,
                                                           int nsamples, double* __restrict__ out)
{
    const long long N = (long long)L.Lx * L.Ly;
    const long long s = blockIdx.x * (long long)kThreads + threadIdx.x;
    if (s >= N) return;
    if (mask[s]) {
        out[s] = z[s];
        return;
    }
    const int y = (int)(s / L.Lx), x = (int)(s - (long long)y * L.Lx);
    const int c = (x + y) & 1;
    const size_t idx = (size_t)y * L.pitch + (x >> 1);
    double v;
    if (acc0) {
        v = c ? acc1[idx] : acc0[idx];
    } else {
        const float h = c ? hi1[idx] : hi0[idx];
        const float l = c ? lo1[idx] : lo0[idx];
        v = (double)h - (double)l;
    }
    const double lo = range[0], hi = range[1];
    const double phibar = v / (double)nsamples;
    out[s] = __dadd_rn(lo, __dmul_rn(hi - lo, phibar / kTwoPi));
}

// --------------------------------------------------------------------------------------------
// State transfer between the packed colour layout and a row-major FP64 grid.
// --------------------------------------------------------------------------------------------
template <typename S>
__global__ void __launch_bounds__(kThreads) get_state_kernel(Layout L, const S* __restrict__ a0,
                                                             const S* __restrict__ a1,
                                                             double* __restrict__ out)
{
    const long long N = (long long)L.Lx * L.Ly;
    const long long s = blockIdx.x * (long long)kThreads + threadIdx.x;
    if (s >= N) return;
    const int y = (int)(s / L.Lx), x = (int)(s - (long long)y * L.Lx);
    const size_t idx = (size_t)y * L.pitch + (x >> 1);
    out[s] = load_as<double>(((x + y) & 1) ? a1[idx] : a0[idx]);
}

template <typename S>
__global__ void __launch_bounds__(kThreads) set_state_kernel(Layout L, const double* __restrict__ in,
                                                             const unsigned char* __restrict__ mask,
                                                             S* __restrict__ a0, S* __restrict__ a1)
{
    const long long N = (long long)L.Lx * L.Ly;
    const long long s = blockIdx.x * (long long)kThreads + threadIdx.x;
    if (s >= N || mask[s]) return;
    const int y = (int)(s / L.Lx), x = (int)(s - (long long)y * L.Lx);
    const size_t idx = (size_t)y * L.pitch + (x >> 1);
    (((x + y) & 1) ? a1 : a0)[idx] = store_from<S>(in[s]);
}

__global__ void philox_kernel(const uint32_t* __restrict__ ctr, uint32_t* __restrict__ out, int n,
                              uint32_t k0, uint32_t k1)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint4 c = reinterpret_cast<const uint4*>(ctr)[i];
    reinterpret_cast<uint4*>(out)[i] = philox4x32_10(c, k0, k1);
}

// Width of the bounded Metropolis proposals after one sweep: w <- w exp(a - target), with a the
// sweep's acceptance fraction over the n_pred prediction sites, kept in [1e-3, 2 pi]; the
// counter restarts at 0 for the next sweep.
// Launched as a programmatic dependent launch between two sweeps: it waits for the black pass it
// follows, then lets the next red pass be scheduled at once (that pass still waits for this
// kernel's completion before it reads the width).
__global__ void adapt_width_kernel(double* __restrict__ width, unsigned long long* __restrict__ count,
                                   long long n_pred, double target)
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;");
    const double acc = n_pred > 0 ? (double)*count / (double)n_pred : target;
    *width = fmin(fmax(*width * exp(acc - target), 1e-3), 6.283185307179586);
    *count = 0ull;
}

inline int grid_for(long long n) { return (int)((n + kThreads - 1) / kThreads); }

// Folds fixed-point partial sums of sampled FP16 angles (units of 2^-24) into the FP64 sums:
// exact, as both are integer multiples of 2^-24 far below 2^53 units.
__global__ void __launch_bounds__(kThreads) fold_partials_kernel(double* __restrict__ acc,
                                                                 int* __restrict__ part,
                                                                 long long n)
{
    const long long i = blockIdx.x * (long long)kThreads + threadIdx.x;
    if (i >= n) return;
    const int v = part[i];
    if (v) {
        acc[i] += (double)v * 0x1.0p-24;
        part[i] = 0;
    }
}

template <typename Fn>
cudaError_t dispatch_store(int store, Fn&& f)
{
    switch (store) {
    case kF64: return f(double{});
    case kF32: return f(float{});
    case kF16: return f(__half{});
    case kBF16: return f(__nv_bfloat16{});
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_minmax(const double* z, const unsigned char* mask, long long N, double* part,
                          int nblk, double* out4, cudaStream_t st)
{
    minmax_kernel<<<nblk, kThreads, 0, st>>>(z, mask, N, part);
    minmax_final<<<1, 32, 0, st>>>(part, nblk, out4);
    return cudaGetLastError();
}

cudaError_t launch_init(const Layout& L, const Precision& p, const double* z,
                        const unsigned char* mask, const double* range, void* ang0, void* ang1,
                        uint32_t* mb0, uint32_t* mb1, uint64_t seed, uint32_t problem,
                        cudaStream_t st)
{
    const dim3 grid((L.pitch + kThreads - 1) / kThreads, L.Ly < 65535 ? L.Ly : 65535, 2);
    const uint32_t klo = (uint32_t)seed, khi = (uint32_t)(seed >> 32);
    return dispatch_store(p.store, [&](auto tag) {
        using S = decltype(tag);
        init_kernel<S><<<grid, kThreads, 0, st>>>(L, z, mask, range, static_cast<S*>(ang0),
                                                  static_cast<S*>(ang1), mb0, mb1, klo, khi,
                                                  problem, p.func);
        return cudaGetLastError();
    });
}

int sample_energy_blocks(const Layout& L)
{
    const long long n = (long long)L.Lx * L.Ly;
    const long long b = (n + kThreads - 1) / kThreads;
    return (int)(b < 1024 ? b : 1024);
}

cudaError_t launch_sample_energy(const Layout& L, const double* z, const unsigned char* mask,
                                 const double* range, double q, double* part_sum,
                                 long long* part_cnt, int nblk, double* out2, cudaStream_t st)
{
    sample_energy_kernel<<<nblk, kThreads, 0, st>>>(L, z, mask, range, q, part_sum, part_cnt);
    sample_energy_final<<<1, 32, 0, st>>>(part_sum, part_cnt, nblk, out2);
    return cudaGetLastError();
}

int energy_blocks(const Layout& L)
{
    const long long n = (long long)L.Ly * L.Lxh;
    const long long b = (n + kThreads - 1) / kThreads;
    return (int)(b < 1024 ? b : 1024);
}

cudaError_t launch_energy_fp64(const Layout& L, const Precision& p, const void* ang0,
                               const void* ang1, double q, double* part, int nblk, double* out,
                               cudaStream_t st)
{
    return dispatch_store(p.store, [&](auto tag) {
        using S = decltype(tag);
        energy_kernel<S><<<nblk, kThreads, 0, st>>>(L, static_cast<const S*>(ang0),
                                                    static_cast<const S*>(ang1), q, part);
        reduce_kernel<double><<<1, kThreads, 0, st>>>(part, nblk, out);
        return cudaGetLastError();
    });
}

cudaError_t launch_reduce(const Precision& p, const void* part, int n, double* out, cudaStream_t st)
{
    if (p.energy == 0)
        reduce_kernel<double><<<1, kThreads, 0, st>>>(static_cast<const double*>(part), n, out);
    else
        reduce_kernel<float><<<1, kThreads, 0, st>>>(static_cast<const float*>(part), n, out);
    return cudaGetLastError();
}

cudaError_t launch_predict(const Layout& L, const Precision&, const double* z,
                           const unsigned char* mask, const double* range, const double* acc0,
                           const double* acc1, const float* hi0, const float* lo0,
                           const float* hi1, const float* lo1, int nsamples, double* out,
                           cudaStream_t st)
{
    const long long N = (long long)L.Lx * L.Ly;
    predict_kernel<<<grid_for(N), kThreads, 0, st>>>(L, z, mask, range, acc0, acc1, hi0, lo0, hi1,
                                                     lo1, nsamples, out);
    return cudaGetLastError();
}

cudaError_t launch_get_state(const Layout& L, const Precision& p, const void* ang0,
                             const void* ang1, double* out, cudaStream_t st)
{
    const long long N = (long long)L.Lx * L.Ly;
    return dispatch_store(p.store, [&](auto tag) {
        using S = decltype(tag);
        get_state_kernel<S><<<grid_for(N), kThreads, 0, st>>>(L, static_cast<const S*>(ang0),
                                                             static_cast<const S*>(ang1), out);
        return cudaGetLastError();
    });
}

cudaError_t launch_set_state(const Layout& L, const Precision& p, const double* in,
                             const unsigned char* mask, void* ang0, void* ang1, cudaStream_t st)
{
    const long long N = (long long)L.Lx * L.Ly;
    return dispatch_store(p.store, [&](auto tag) {
        using S = decltype(tag);
        set_state_kernel<S><<<grid_for(N), kThreads, 0, st>>>(L, in, mask, static_cast<S*>(ang0),
                                                             static_cast<S*>(ang1));
        return cudaGetLastError();
    });
}

cudaError_t launch_adapt_width(double* width, unsigned long long* count, long long n_pred,
                               double target, cudaStream_t st)
{
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(1);
    cfg.blockDim = dim3(1);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, adapt_width_kernel, width, count, n_pred, target);
}

cudaError_t launch_fold_partials(double* acc, int* part, size_t n, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    fold_partials_kernel<<<grid_for((long long)n), kThreads, 0, st>>>(acc, part, (long long)n);
    return cudaGetLastError();
}

cudaError_t launch_philox(const uint32_t* ctr, uint32_t* out, int n, uint64_t seed, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    philox_kernel<<<grid_for(n), kThreads, 0, st>>>(ctr, out, n, (uint32_t)seed,
                                                   (uint32_t)(seed >> 32));
    return cudaGetLastError();
}

}  // namespace mpr
