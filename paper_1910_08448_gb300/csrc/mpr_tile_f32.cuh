// mpr_tile_f32.cuh -- one tile of a colour half-sweep for the FP32 function setting (X_F = S,
// Sec. 2): Metropolis + over-relaxation of every prediction site of one colour in the tile, FP32
// update arithmetic with the hardware intrinsics __sincosf / __expf, any spin storage type.
// Used by the single-problem kernel (one tile per block) and the batched persistent kernel
// (many tiles of many problems per block).
//
// Tile: 128 half-lattice columns x (8 warps x R rows). A thread owns 4 consecutive columns of a
// row (two same-colour site pairs -> two Philox calls), loaded and stored as one vector. The other
// colour's tile and its one-site halo are staged in shared memory as unit vectors
// (cos q*phi, sin q*phi), computed once per site and read by its four neighbours; column j of the
// tile sits at shared column j - j0 + 2, so each lane's four interior entries are 16-B aligned.
#pragma once

#include "mpr_device.cuh"
#include "mpr_internal.h"

namespace mpr {
namespace f32 {

constexpr int kTJ = 128;     // half-lattice columns per tile
constexpr int kWarps = 8;    // 256 threads, blockDim = (32, 8)

// atan2 in FP32: reduce to a = min(|x|,|y|)/max(|x|,|y|) in [0, 1], evaluate atan(a) = a*P(a^2),
// then map the octant back. P is a degree-7 polynomial in a^2 fitted for this library by Lawson's
// iteratively reweighted least squares (a minimax method) to atan on [0, 1]: max error 3.8e-8 rad,
// below the FP32 spacing of angles near pi/4. The quotient uses the approximate FP32 division.
__device__ __forceinline__ float atan2_fast(float y, float x)
{
    const float ax = fabsf(x), ay = fabsf(y);
    const float mx = fmaxf(ax, ay), mn = fminf(ax, ay);
    const float a = __fdividef(mn, mx);
    const float s = a * a;
    float p = -0.004054565913975239f;
    p = fmaf(p, s, 0.021862953901290894f);
    p = fmaf(p, s, -0.0559123195707798f);
    p = fmaf(p, s, 0.0964219719171524f);
    p = fmaf(p, s, -0.1390862911939621f);
    p = fmaf(p, s, 0.19946566224098206f);
    p = fmaf(p, s, -0.33329859375953674f);
    p = fmaf(p, s, 0.9999993443489075f);
    float t = a * p;
    t = (ay > ax) ? 1.57079632679489662f - t : t;
    t = (x < 0.0f) ? 3.14159265358979324f - t : t;
    return (y < 0.0f) ? -t : t;
}

template <typename S> struct Raw4;
template <> struct Raw4<__half> { using T = uint2; };
template <> struct Raw4<__nv_bfloat16> { using T = uint2; };
template <> struct Raw4<float> { using T = float4; };
struct alignas(16) Doubles4 { double x[4]; };
template <> struct Raw4<double> { using T = Doubles4; };

template <typename S> union Pack4 {
    typename Raw4<S>::T v;
    S s[4];
};

template <typename S>
__device__ __forceinline__ void load4(const S* p, Pack4<S>& out)
{
    if constexpr (sizeof(S) == 8) {
        const double2* q = reinterpret_cast<const double2*>(p);
        const double2 a = q[0], b = q[1];
        out.s[0] = a.x; out.s[1] = a.y; out.s[2] = b.x; out.s[3] = b.y;
    } else {
        out.v = *reinterpret_cast<const typename Raw4<S>::T*>(p);
    }
}

template <typename S>
__device__ __forceinline__ void store4(S* p, const Pack4<S>& in)
{
    if constexpr (sizeof(S) == 8) {
        double2* q = reinterpret_cast<double2*>(p);
        q[0] = make_double2(in.s[0], in.s[1]);
        q[1] = make_double2(in.s[2], in.s[3]);
    } else {
        *reinterpret_cast<typename Raw4<S>::T*>(p) = in.v;
    }
}

template <int R> struct TileSmem {
    float2 nb[kWarps * R + 2][kTJ + 4];
    double wsum_d[kWarps];
    float wsum_f[kWarps];
};

template <int R> __host__ __device__ constexpr int tile_rows() { return kWarps * R; }

// One tile (tile column tx, tile row ty) of colour a.colour. SAMPLE: 0 none, 1 FP64 accumulators,
// 2 Kahan FP32 accumulators. With MEASURE (black pass) the tile's sum of u_b . h_b over its
// existing black sites is written by thread (0, 0) to *eslot (double, or float with kEnergyF32).
// Begins with a block barrier, so a block may call it for several tiles in a row.
template <typename S, int R, bool MEASURE, int SAMPLE>
__device__ __forceinline__ void sweep_tile(const SweepArgs& a, int tx, int ty, TileSmem<R>& sm,
                                           void* eslot)
{
    constexpr int TY = kWarps * R;
    const int c = a.colour, cb = c ^ 1;
    const int j0 = tx * kTJ;
    const int y0 = ty * TY;
    const int lane = threadIdx.x, warp = threadIdx.y;
    const S* __restrict__ other = static_cast<const S*>(a.other);
    S* __restrict__ own = static_cast<S*>(a.own);
    const float q = (float)a.q;

    __syncthreads();   // the previous tile's readers are done with sm
    // ---- stage the other colour (rows y0-1 .. y0+TY, columns j0-1 .. j0+TJ) ----
    for (int r = warp; r < TY + 2; r += kWarps) {
        const int y = y0 - 1 + r;
        const bool row_ok = y >= 0 && y < a.Ly;
        const int ob = (y + cb) & 1;
        {   // interior: 4 consecutive columns per lane, one vector load
            const int j = j0 + 4 * lane;
            float2 v[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) v[k] = make_float2(0.f, 0.f);
            if (row_ok) {
                Pack4<S> pk;
                load4(other + (size_t)y * a.pitch + j, pk);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    if (2 * (j + k) + ob < a.Lx) {
                        float sn, cs;
                        __sincosf(q * load_as<float>(pk.s[k]), &sn, &cs);
                        v[k] = make_float2(cs, sn);
                    }
                }
            }
            float4* dst = reinterpret_cast<float4*>(&sm.nb[r][2 + 4 * lane]);
            dst[0] = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
            dst[1] = make_float4(v[2].x, v[2].y, v[3].x, v[3].y);
        }
        if (lane < 2) {   // halo columns j0 - 1 and j0 + TJ
            const int j = lane == 0 ? j0 - 1 : j0 + kTJ;
            const int cc = lane == 0 ? 1 : kTJ + 2;
            float2 v = make_float2(0.f, 0.f);
            if (row_ok && j >= 0 && 2 * j + ob < a.Lx) {
                float sn, cs;
                __sincosf(q * load_as<float>(other[(size_t)y * a.pitch + j]), &sn, &cs);
                v = make_float2(cs, sn);
            }
            sm.nb[r][cc] = v;
        }
    }
    __syncthreads();

    const float invT = (float)a.invT;
    const float two_pi = kTwoPiF;
    const float width = two_pi * q;
    const float inv_q = 1.0f / q;
    double e_d = 0.0;
    float e_f = 0.0f;

    for (int rr = 0; rr < R; ++rr) {
        const int ly = warp * R + rr;
        const int y = y0 + ly;
        if (y >= a.Ly) break;
        const int o = (y + c) & 1;
        const int jb = j0 + 4 * lane;           // first of this thread's 4 columns
        const int lj = 4 * lane;
        const size_t idx = (size_t)y * a.pitch + jb;
        const uint32_t bits = (a.mbits[(size_t)y * a.mpitch + (jb >> 5)] >> (jb & 31)) & 0xFu;
        bool ex[4], upd[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            ex[k] = 2 * (jb + k) + o < a.Lx;
            upd[k] = ex[k] && !((bits >> k) & 1u);
        }
        if (!MEASURE && !(upd[0] || upd[1] || upd[2] || upd[3])) continue;
        Pack4<S> pk;
        load4(own + idx, pk);
        uint4 w[2];
#pragma unroll
        for (int pr = 0; pr < 2; ++pr) {
            w[pr] = make_uint4(0u, 0u, 0u, 0u);
            if (upd[2 * pr] || upd[2 * pr + 1])
                w[pr] = pair_words((uint32_t)((jb >> 1) + pr), (uint32_t)y, a.sweep, a.problem,
                                   kTagMetropolis, (uint32_t)c, a.seed_lo, a.seed_hi);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            // local field h = sum of the neighbours' unit vectors (left, right, up, down)
            const float2 lf = sm.nb[ly + 1][lj + k + o + 1], rt = sm.nb[ly + 1][lj + k + o + 2];
            const float2 up = sm.nb[ly][lj + k + 2], dn = sm.nb[ly + 2][lj + k + 2];
            const float hx = ((lf.x + rt.x) + up.x) + dn.x;
            const float hy = ((lf.y + rt.y) + up.y) + dn.y;
            float f = load_as<float>(pk.s[k]);
            if (upd[k]) {
                const uint32_t wp = (k & 1) ? w[k >> 1].z : w[k >> 1].x;
                const uint32_t wa = (k & 1) ? w[k >> 1].w : w[k >> 1].y;
                const float u_prop = uniform_f(wp), u_acc = uniform_f(wa);
                // Metropolis: uniform proposal, accept if dE <= 0 or u < exp(-dE/T)
                const float fp = two_pi * u_prop;
                float s0, c0, sp, cp;
                __sincosf(q * f, &s0, &c0);
                __sincosf(q * fp, &sp, &cp);
                // dE = E(fp) - E(f), E(phi) = -(hx cos q*phi + hy sin q*phi)
                const float dE = hx * (c0 - cp) + hy * (s0 - sp);
                const bool accept = dE <= 0.0f || u_acc < __expf(-dE * invT);
                const float f1 = accept ? fp : f;
                // over-relaxation: reflect q*phi about arg(h); keep it if it lands in [0, 2*pi*q]
                float fn = f1;
                if (hx != 0.0f || hy != 0.0f) {
                    float r = 2.0f * atan2_fast(hy, hx) - q * f1;   // in [-2pi(1+q), 2pi]
                    r = r < 0.0f ? r + two_pi : r;
                    r = r < 0.0f ? r + two_pi : r;
                    fn = r <= width ? r * inv_q : f1;
                }
                pk.s[k] = store_from<S>(fn);
                f = load_as<float>(pk.s[k]);
                if (SAMPLE == 1) {
                    a.acc[idx + k] += (double)f;
                } else if (SAMPLE == 2) {
                    // Kahan: hi carries the sum, lo the (negated) lost low-order part
                    const float hi = a.acc_hi[idx + k], lo = a.acc_lo[idx + k];
                    const float yv = f - lo;
                    const float tt = hi + yv;
                    a.acc_lo[idx + k] = (tt - hi) - yv;
                    a.acc_hi[idx + k] = tt;
                }
            }
            if (MEASURE && ex[k]) {
                // every bond joins a red and a black site: sum over black sites of u_b . h_b
                float sn, cs;
                __sincosf(q * f, &sn, &cs);
                const float e = cs * hx + sn * hy;
                if (a.flags & kEnergyF32) e_f += e; else e_d += (double)e;
            }
        }
        if (upd[0] || upd[1] || upd[2] || upd[3]) store4(own + idx, pk);
    }

    if (MEASURE) {
#pragma unroll
        for (int off = 16; off; off >>= 1) {
            e_d += __shfl_xor_sync(0xffffffffu, e_d, off);
            e_f += __shfl_xor_sync(0xffffffffu, e_f, off);
        }
        if (lane == 0) {
            sm.wsum_d[warp] = e_d;
            sm.wsum_f[warp] = e_f;
        }
        __syncthreads();
        if (warp == 0 && lane == 0) {
            if (a.flags & kEnergyF32) {
                float s = 0.0f;
                for (int i = 0; i < kWarps; ++i) s += sm.wsum_f[i];
                *static_cast<float*>(eslot) = s;
            } else {
                double s = 0.0;
                for (int i = 0; i < kWarps; ++i) s += sm.wsum_d[i];
                *static_cast<double*>(eslot) = s;
            }
        }
    }
}

}  // namespace f32
}  // namespace mpr
