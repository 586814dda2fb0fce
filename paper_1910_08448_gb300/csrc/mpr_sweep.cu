// mpr_sweep.cu -- one colour half-sweep of the conditional hybrid Monte Carlo (Sec. 2): for every
// prediction site of the colour, one Metropolis move with a uniform proposal followed by one
// energy-conserving over-relaxation move under Eq. 2; measured sites stay frozen. Fused into the
// same pass: the accumulation of the sampled angles (Sec. 2: averaging over configurations in
// equilibrium) and, on the black pass, the bond-energy partial sums (Sec. 2: e = <H>/L^2).
//
// Precision axes (Sec. 2): S = spin storage (X_S, plus FP16/BF16), F = function and update
// arithmetic (X_F), E = energy accumulation (X_E).
#include "mpr_device.cuh"
#include "mpr_internal.h"

namespace mpr {
namespace {

constexpr int kTJ = 64;      // half-lattice columns per tile: 32 lanes x one site pair
constexpr int kWarps = 8;    // 256 threads; each warp owns R rows of the tile

template <typename F> struct Wrap;
template <> struct Wrap<double> {
    // representative of psi modulo 2*pi in [0, 2*pi), as the method states it
    static __device__ __forceinline__ double rep(double psi) { return psi - kTwoPi * floor(psi / kTwoPi); }
};
template <> struct Wrap<float> {
    static __device__ __forceinline__ float rep(float psi)
    {
        return psi - kTwoPiF * floorf(psi * 0.159154943091895335768883763373f);
    }
};

template <typename S, typename F, typename E, int R>
__global__ void __launch_bounds__(256) sweep_kernel(const SweepArgs a)
{
    using F2 = typename Vec2<F>::type;
    using M = Math<F>;
    constexpr int TY = kWarps * R;
    constexpr int SW = kTJ + 2;
    __shared__ F2 nb[TY + 2][SW];
    __shared__ E wsum[kWarps];

    const int c = a.colour, cb = c ^ 1;
    // one tile per block, tiles row-major over a 1-D grid (no limit on the number of tile rows)
    const int ntx = (a.Lxh + kTJ - 1) / kTJ;
    const int j0 = (int)(blockIdx.x % ntx) * kTJ;
    const int y0 = (int)(blockIdx.x / ntx) * TY;
    const S* __restrict__ other = static_cast<const S*>(a.other);
    S* __restrict__ own = static_cast<S*>(a.own);
    const F q = (F)a.q;
    const int tid = threadIdx.y * 32 + threadIdx.x;

    // Stage the other colour's unit vectors (cos q*phi, sin q*phi) with a one-site halo. Entries
    // outside the lattice stay (0, 0): that is the open boundary.
    for (int e = tid; e < (TY + 2) * SW; e += 256) {
        const int r = e / SW, cc = e - r * SW;
        const int y = y0 - 1 + r, j = j0 - 1 + cc;
        F2 v;
        v.x = (F)0;
        v.y = (F)0;
        if (y >= 0 && y < a.Ly && j >= 0 && 2 * j + ((y + cb) & 1) < a.Lx) {
            F s, co;
            M::sincos_(q * load_as<F>(other[(size_t)y * a.pitch + j]), &s, &co);
            v.x = co;
            v.y = s;
        }
        nb[r][cc] = v;
    }
    __syncthreads();

    const bool measure = (a.flags & kMeasure) && c == 1;
    const bool sample = (a.flags & kSample) != 0;
    const F T = (F)a.T, invT = (F)a.invT;
    const F two_pi = M::two_pi();
    const F width = two_pi * q;
    const bool bounded = a.width != nullptr;
    const F pw = bounded ? (F)*a.width : (F)0;   // bounded proposals: half-width
    int n_acc = 0;
    E eacc = (E)0;

    for (int rr = 0; rr < R; ++rr) {
        const int ly = threadIdx.y * R + rr;
        const int y = y0 + ly;
        if (y >= a.Ly) break;
        const int jp = j0 + 2 * threadIdx.x;
        const int o = (y + c) & 1;
        const uint32_t mw = a.mbits[(size_t)y * a.mpitch + (jp >> 5)];
        bool ex[2], upd[2];
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            const int j = jp + t;
            ex[t] = 2 * j + o < a.Lx;
            upd[t] = ex[t] && !((mw >> (j & 31)) & 1u);
        }
        uint4 w = make_uint4(0u, 0u, 0u, 0u);
        if (upd[0] || upd[1])
            w = pair_words((uint32_t)(jp >> 1), (uint32_t)y, a.sweep, a.problem, kTagMetropolis,
                           (uint32_t)c, a.seed_lo, a.seed_hi);
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            if (!ex[t]) continue;
            const int j = jp + t, lj = j - j0;
            // local field h = sum of the neighbours' unit vectors (left, right, up, down)
            const F2 lf = nb[ly + 1][lj + o], rt = nb[ly + 1][lj + o + 1];
            const F2 up = nb[ly][lj + 1], dn = nb[ly + 2][lj + 1];
            const F hx = ((lf.x + rt.x) + up.x) + dn.x;
            const F hy = ((lf.y + rt.y) + up.y) + dn.y;
            const size_t idx = (size_t)y * a.pitch + j;
            F f = load_as<F>(own[idx]);
            if (upd[t]) {
                const uint32_t wp = t ? w.z : w.x, wa = t ? w.w : w.y;
                const F u_prop = M::uniform(wp), u_acc = M::uniform(wa);
                // Metropolis: uniform proposal (or bounded: f + pw (2u - 1), rejected outside
                // [0, 2 pi)), accept if dE <= 0 or u < exp(-dE/T)
                const F fp = bounded ? f + pw * ((F)2 * u_prop - (F)1) : two_pi * u_prop;
                const bool inside = !bounded || (fp >= (F)0 && fp < two_pi);
                F s0, c0, sp, cp;
                M::sincos_(q * f, &s0, &c0);
                M::sincos_(q * fp, &sp, &cp);
                const F dE = (-(hx * cp + hy * sp)) - (-(hx * c0 + hy * s0));
                bool accept = dE <= (F)0;
                if (!accept) accept = u_acc < M::exp_neg_over(dE, T, invT);
                accept = accept && inside;
                n_acc += accept ? 1 : 0;
                const F f1 = accept ? fp : f;
                // over-relaxation: reflect q*phi about arg(h); keep it if it lands in [0, 2*pi*q]
                F fn = f1;
                if (hx != (F)0 || hy != (F)0) {
                    const F th = M::atan2_(hy, hx);
                    const F r = Wrap<F>::rep((F)2 * th - q * f1);
                    if (r <= width) fn = r / q;
                }
                const S st = store_from<S>(fn);
                own[idx] = st;
                f = load_as<F>(st);
                if (sample) {
                    if (a.acc) {
                        a.acc[idx] += (double)f;
                    } else {
                        // Kahan: hi carries the sum, lo the (negated) lost low-order part
                        const float v = (float)f;
                        const float hi = a.acc_hi[idx], lo = a.acc_lo[idx];
                        const float yv = v - lo;
                        const float tt = hi + yv;
                        a.acc_lo[idx] = (tt - hi) - yv;
                        a.acc_hi[idx] = tt;
                    }
                }
            }
            if (measure) {
                // every bond joins a red and a black site: sum over black sites of u_b . h_b
                F s, co;
                M::sincos_(q * f, &s, &co);
                eacc += (E)(co * hx + s * hy);
            }
        }
    }

    if (a.accepted) {
#pragma unroll
        for (int off = 16; off; off >>= 1) n_acc += __shfl_xor_sync(0xffffffffu, n_acc, off);
        if (threadIdx.x == 0 && n_acc) atomicAdd(a.accepted, (unsigned long long)n_acc);
    }
    if (measure) {
#pragma unroll
        for (int off = 16; off; off >>= 1) eacc += __shfl_xor_sync(0xffffffffu, eacc, off);
        if (threadIdx.x == 0) wsum[threadIdx.y] = eacc;
        __syncthreads();
        if (tid == 0) {
            E s = (E)0;
            for (int i = 0; i < kWarps; ++i) s += wsum[i];
            static_cast<E*>(a.epart)[blockIdx.x] = s;
        }
    }
}

constexpr int kRows = 2;

template <typename S, typename F, typename E>
cudaError_t launch_typed(const SweepArgs& a, cudaStream_t st)
{
    const dim3 grid(((a.Lxh + kTJ - 1) / kTJ) * ((a.Ly + kWarps * kRows - 1) / (kWarps * kRows)));
    sweep_kernel<S, F, E, kRows><<<grid, dim3(32, kWarps), 0, st>>>(a);
    return cudaGetLastError();
}

template <typename S>
cudaError_t launch_store(const Precision& p, const SweepArgs& a, cudaStream_t st)
{
    if (p.func == 0) {
        return p.energy == 0 ? launch_typed<S, double, double>(a, st)
                             : launch_typed<S, double, float>(a, st);
    }
    return p.energy == 0 ? launch_typed<S, float, double>(a, st)
                         : launch_typed<S, float, float>(a, st);
}

}  // namespace

int sweep_blocks(const Layout& L, const Precision&)
{
    return ((L.Lxh + kTJ - 1) / kTJ) * ((L.Ly + kWarps * kRows - 1) / (kWarps * kRows));
}

cudaError_t launch_sweep(const Precision& p, const SweepArgs& a, cudaStream_t st)
{
    switch (p.store) {
    case kF64: return launch_store<double>(p, a, st);
    case kF32: return launch_store<float>(p, a, st);
    case kF16: return launch_store<__half>(p, a, st);
    case kBF16: return launch_store<__nv_bfloat16>(p, a, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace mpr
