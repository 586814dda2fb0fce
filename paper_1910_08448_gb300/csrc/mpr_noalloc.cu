// mpr_noalloc.cu -- mpr_bond_energy_noalloc: the bond energy of a caller-held state with no device
// allocation at all.
//
// Some callers cannot call cudaMalloc: code that works under a strict device-memory budget or a
// custom allocator that owns the whole device, and real-time loops that must not take the
// allocator's locks or synchronise. Every other entry point of this library allocates its scratch
// (reduction partials) inside a handle. This one keeps its scratch in a fixed array compiled into
// the library instead, so a call only launches kernels.
//
// Cost of that choice: the array below (32 KiB of FP64 partials) exists on every GPU that loads
// the library, for the life of the process, and all calls share it.
#include "mpr.h"
#include "mpr_internal.h"

#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>

#include <mutex>

namespace {

constexpr int kThreads = 256;
constexpr long long kSitesPerBlock = 65536;   // one partial sum per 65536 sites
constexpr int kMaxBlocks = 4096;              // -> at most 2^28 sites (16384 x 16384)
constexpr int kMaxDevices = 64;

// The scratch: one partial sum per block of the first pass. Every block of a call writes its own
// slot before the second pass reads it, so nothing has to be cleared between calls. Calls that
// overlap on the GPU (for example on two streams) use the same slots and race.
static __device__ __align__(256) double g_bond_partials[kMaxBlocks];

// First pass: block b sums cos[q(phi_s - phi_right)] and cos[q(phi_s - phi_down)] over the sites
// s of [b * 65536, (b + 1) * 65536) in row-major order (Eq. 2, open boundaries).
__global__ void __launch_bounds__(kThreads) bond_partials(int Lx, int Ly,
                                                          const double* __restrict__ phi, double q,
                                                          double* __restrict__ part)
{
    const long long N = (long long)Lx * Ly;
    const long long base = (long long)blockIdx.x * kSitesPerBlock;
    const long long end = base + kSitesPerBlock < N ? base + kSitesPerBlock : N;
    double sum = 0.0;
    for (long long s = base + threadIdx.x; s < end; s += kThreads) {
        const int y = (int)(s / Lx), x = (int)(s - (long long)y * Lx);
        const double f = phi[s];
        if (x + 1 < Lx) sum += cos(q * (f - phi[s + 1]));
        if (y + 1 < Ly) sum += cos(q * (f - phi[s + Lx]));
    }
    __shared__ double sh[kThreads];
    sh[threadIdx.x] = sum;
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// Second pass, one block: fixed-order sum of the partials, e_b = -sum / N_b.
__global__ void __launch_bounds__(kThreads) bond_final(const double* __restrict__ part, int nblk,
                                                       double n_bonds, double* __restrict__ out)
{
    __shared__ double sh[kThreads];
    double s = 0.0;
    for (int i = threadIdx.x; i < nblk; i += kThreads) s += part[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = -sh[0] / n_bonds;
}

// Device address of g_bond_partials per device. In host code the array's name only stands for
// the symbol, so the address is looked up once per device, with that device current, and cached
// for the life of the process. It belongs to the device's primary context: after a
// cudaDeviceReset of that device the cached address is stale (see include/mpr.h).
std::mutex g_mu;
double* g_addr[kMaxDevices] = {};

mpr_status err(mpr_status s, const char* msg)
{
    mpr::set_last_error(msg);
    return s;
}

}  // namespace

extern "C" mpr_status mpr_bond_energy_noalloc(int Lx, int Ly, const double* angles_dev, double q,
                                              double* e_bond_dev, void* stream)
{
    if (!angles_dev || !e_bond_dev) return err(MPR_ERR_INVALID_ARG, "angles or output pointer is NULL");
    if (Lx < 2 || Ly < 2) return err(MPR_ERR_INVALID_ARG, "both sides of the grid must be >= 2");
    if (!(q > 0.0 && q <= 1.0)) return err(MPR_ERR_INVALID_ARG, "q must lie in (0, 1]");
    const long long N = (long long)Lx * Ly;
    if (N > kSitesPerBlock * kMaxBlocks) {
        char buf[160];
        snprintf(buf, sizeof buf,
                 "grid of %lld sites exceeds the %lld sites (2^28) that the fixed scratch of "
                 "mpr_bond_energy_noalloc covers",
                 N, kSitesPerBlock * kMaxBlocks);
        return err(MPR_ERR_INVALID_ARG, buf);
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return err(MPR_ERR_CUDA, "no usable current CUDA device");
    double* part = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_addr[dev]) {
            void* p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_bond_partials);
            if (e != cudaSuccess || !p) {
                char buf[160];
                snprintf(buf, sizeof buf, "cudaGetSymbolAddress(g_bond_partials): %s",
                         cudaGetErrorString(e));
                return err(MPR_ERR_CUDA, buf);
            }
            g_addr[dev] = static_cast<double*>(p);
        }
        part = g_addr[dev];
    }
    const int nblk = (int)((N + kSitesPerBlock - 1) / kSitesPerBlock);
    const double n_bonds = (double)Lx * (Ly - 1) + (double)Ly * (Lx - 1);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    bond_partials<<<nblk, kThreads, 0, st>>>(Lx, Ly, angles_dev, q, part);
    bond_final<<<1, kThreads, 0, st>>>(part, nblk, n_bonds, e_bond_dev);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        char buf[160];
        snprintf(buf, sizeof buf, "bond energy launch: %s", cudaGetErrorString(e));
        return err(MPR_ERR_CUDA, buf);
    }
    return MPR_OK;
}
