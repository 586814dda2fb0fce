// mpr_tile_f32.cuh -- one tile of a colour half-sweep for the FP32 function setting (X_F = S,
// Sec. 2): Metropolis + over-relaxation of every prediction site of one colour in the tile, FP32
// update arithmetic with the hardware intrinsics __sincosf / __expf, any spin storage type.
// Used by the single-problem kernel (one tile per block) and the batched persistent kernel
// (many tiles of many problems per block).
//
// Tile: 128 half-lattice columns x (8 warps x R rows). A thread owns 4 consecutive columns of a
// row (two same-colour site pairs -> two Philox calls), loaded and stored as one vector. The other
// colour's tile and its one-site halo are staged in shared memory as unit vectors
// (cos q*phi, sin q*phi), computed once per site and read by its four neighbours.
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

// Shared tile of the other colour as structure of arrays: column j of the tile at index
// j - j0 + 4 (halo columns at 3 and kTJ + 4), so a lane's four interior columns form one aligned
// 16-byte vector and a warp's vector accesses touch consecutive banks.
constexpr int kSW = kTJ + 8;
template <int R> struct TileSmem {
    float cs[kWarps * R + 2][kSW];
    float sn[kWarps * R + 2][kSW];
    double wsum_d[kWarps];
    float wsum_f[kWarps];
};

template <int R> __host__ __device__ constexpr int tile_rows() { return kWarps * R; }

// 2^x on the MUFU (hand-written PTX: ex2.approx.ftz.f32)
__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Stages the other colour's rows y0-1 .. y0+TY and columns j0-1 .. j0+TJ of a tile as unit vectors
// (cos q*phi, sin q*phi); entries outside the lattice are (0, 0) (open boundaries). All loads are
// issued before the sin/cos work. CHECK = false when the caller knows every entry exists.
template <typename S, int R, bool CHECK>
__device__ __forceinline__ void stage(const SweepArgs& a, const S* __restrict__ other, int y0,
                                      int j0, int jb, int lj, int cb, float q, TileSmem<R>& sm)
{
    constexpr int TY = kWarps * R;
    constexpr int NR = (TY + 2 + kWarps - 1) / kWarps;   // staged rows per warp
    const int lane = threadIdx.x, warp = threadIdx.y;
    Pack4<S> st[NR];
    S halo[NR];
#pragma unroll
    for (int i = 0; i < NR; ++i) {
        const int r = warp + i * kWarps;
        const int y = y0 - 1 + r;
        if (r < TY + 2 && (!CHECK || (y >= 0 && y < a.Ly))) {
            load4(other + (size_t)y * a.pitch + jb, st[i]);
            if (lane < 2) {
                const int j = lane == 0 ? j0 - 1 : j0 + kTJ;
                if (!CHECK || (j >= 0 && 2 * j + ((y + cb) & 1) < a.Lx))
                    halo[i] = other[(size_t)y * a.pitch + j];
            }
        }
    }
#pragma unroll
    for (int i = 0; i < NR; ++i) {
        const int r = warp + i * kWarps;
        if (r >= TY + 2) break;
        const int y = y0 - 1 + r;
        const bool row_ok = !CHECK || (y >= 0 && y < a.Ly);
        const int ob = (y + cb) & 1;
        float vc[4], vs[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            vc[k] = 0.0f;
            vs[k] = 0.0f;
            if (!CHECK || (row_ok && 2 * (jb + k) + ob < a.Lx))
                __sincosf(q * load_as<float>(st[i].s[k]), &vs[k], &vc[k]);
        }
        *reinterpret_cast<float4*>(&sm.cs[r][4 + lj]) = make_float4(vc[0], vc[1], vc[2], vc[3]);
        *reinterpret_cast<float4*>(&sm.sn[r][4 + lj]) = make_float4(vs[0], vs[1], vs[2], vs[3]);
        if (lane < 2) {   // halo columns j0 - 1 (index 3) and j0 + TJ (index kTJ + 4)
            const int j = lane == 0 ? j0 - 1 : j0 + kTJ;
            const int cc = lane == 0 ? 3 : kTJ + 4;
            float hc = 0.0f, hs = 0.0f;
            if (!CHECK || (row_ok && j >= 0 && 2 * j + ob < a.Lx))
                __sincosf(q * load_as<float>(halo[i]), &hs, &hc);
            sm.cs[r][cc] = hc;
            sm.sn[r][cc] = hs;
        }
    }
}

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
    const float q = a.qf;
    const int jb = j0 + 4 * lane;             // first of this thread's 4 columns
    const int lj = 4 * lane;

    // ---- own rows: values and frozen bits, loaded before the staging so their latency overlaps
    Pack4<S> mine[R];
    uint32_t bits[R];
#pragma unroll
    for (int rr = 0; rr < R; ++rr) {
        const int y = y0 + warp * R + rr;
        bits[rr] = 0xFu;
        if (y < a.Ly) {
            load4(own + (size_t)y * a.pitch + jb, mine[rr]);
            bits[rr] = (a.mbits[(size_t)y * a.mpitch + (jb >> 5)] >> (jb & 31)) & 0xFu;
        }
    }

    __syncthreads();   // the previous tile's readers are done with sm
    // ---- stage the other colour (rows y0-1 .. y0+TY, columns j0-1 .. j0+TJ). Tiles whose halo
    // lies inside the lattice (nearly all) skip the per-entry bounds checks.
    const bool interior = y0 >= 1 && y0 + TY < a.Ly && j0 >= 1 && 2 * (j0 + kTJ) + 1 < a.Lx;
    if (interior) stage<S, R, false>(a, other, y0, j0, jb, lj, cb, q, sm);
    else stage<S, R, true>(a, other, y0, j0, jb, lj, cb, q, sm);
    __syncthreads();

    const float nl2e_invT = -1.4426950408889634f * a.invTf;   // exp(-dE/T) = 2^(dE * nl2e_invT)
    const float two_pi = kTwoPiF;
    const float width = two_pi * q;
    const float inv_q = 1.0f / q;
    double e_d = 0.0;
    float e_f = 0.0f;

#pragma unroll
    for (int rr = 0; rr < R; ++rr) {
        const int ly = warp * R + rr;
        const int y = y0 + ly;
        if (y >= a.Ly) break;
        const int o = (y + c) & 1;
        const size_t idx = (size_t)y * a.pitch + jb;
        bool ex[4], upd[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            ex[k] = 2 * (jb + k) + o < a.Lx;
            upd[k] = ex[k] && !((bits[rr] >> k) & 1u);
        }
        Pack4<S>& pk = mine[rr];
        // both Philox calls of the row, whether or not their sites update: no branch per site
        uint4 w[2];
#pragma unroll
        for (int pr = 0; pr < 2; ++pr)
            w[pr] = pair_words((uint32_t)((jb >> 1) + pr), (uint32_t)y, a.sweep, a.problem,
                               kTagMetropolis, (uint32_t)c, a.seed_lo, a.seed_hi);
        // neighbours: up/down rows at the same columns, the middle row at columns j+o-1, j+o
        const float4 uc = *reinterpret_cast<const float4*>(&sm.cs[ly][4 + lj]);
        const float4 us = *reinterpret_cast<const float4*>(&sm.sn[ly][4 + lj]);
        const float4 dc = *reinterpret_cast<const float4*>(&sm.cs[ly + 2][4 + lj]);
        const float4 ds = *reinterpret_cast<const float4*>(&sm.sn[ly + 2][4 + lj]);
        const float4 mc4 = *reinterpret_cast<const float4*>(&sm.cs[ly + 1][4 + lj]);
        const float4 ms4 = *reinterpret_cast<const float4*>(&sm.sn[ly + 1][4 + lj]);
        const float ec = o ? sm.cs[ly + 1][8 + lj] : sm.cs[ly + 1][3 + lj];
        const float es = o ? sm.sn[ly + 1][8 + lj] : sm.sn[ly + 1][3 + lj];
        // middle row values m[0..4] = columns j+o-1 .. j+o+3 (site k: left m[k], right m[k+1])
        const float mcv[5] = {o ? mc4.x : ec, o ? mc4.y : mc4.x, o ? mc4.z : mc4.y, o ? mc4.w : mc4.z, o ? ec : mc4.w};
        const float msv[5] = {o ? ms4.x : es, o ? ms4.y : ms4.x, o ? ms4.z : ms4.y, o ? ms4.w : ms4.z, o ? es : ms4.w};
        const float ucv[4] = {uc.x, uc.y, uc.z, uc.w}, usv[4] = {us.x, us.y, us.z, us.w};
        const float dcv[4] = {dc.x, dc.y, dc.z, dc.w}, dsv[4] = {ds.x, ds.y, ds.z, ds.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            // local field h = sum of the neighbours' unit vectors (left, right, up, down)
            const float hx = ((mcv[k] + mcv[k + 1]) + ucv[k]) + dcv[k];
            const float hy = ((msv[k] + msv[k + 1]) + usv[k]) + dsv[k];
            float f = load_as<float>(pk.s[k]);
            {
                // every site runs the move; frozen sites and padding discard the result below
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
                const bool accept = dE <= 0.0f || u_acc < ex2_approx(dE * nl2e_invT);
                const float f1 = accept ? fp : f;
                // over-relaxation: reflect q*phi about arg(h); keep it if it lands in [0, 2*pi*q].
                // h = 0 gives 0/0 = NaN in atan2_fast, every comparison below is false and the
                // angle stays, as the move requires.
                float r = 2.0f * atan2_fast(hy, hx) - q * f1;   // in [-2pi(1+q), 2pi]
                r = r < 0.0f ? r + two_pi : r;
                r = r < 0.0f ? r + two_pi : r;
                const float fn = r <= width ? r * inv_q : f1;
                const S stored = store_from<S>(fn);
                pk.s[k] = upd[k] ? stored : pk.s[k];
                f = upd[k] ? load_as<float>(stored) : f;
            }
            if (SAMPLE == 1) {
                if (upd[k]) a.acc[idx + k] += (double)f;
            } else if (SAMPLE == 2) {
                if (upd[k]) {
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
        store4(own + idx, pk);   // unchanged entries are written back with their own bits
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
