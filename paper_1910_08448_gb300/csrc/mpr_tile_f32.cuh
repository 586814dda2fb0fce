// mpr_tile_f32.cuh -- one tile of a colour half-sweep for the FP32 function setting (X_F = S,
// Sec. 2): Metropolis + over-relaxation of every prediction site of one colour in the tile, FP32
// update arithmetic with the hardware intrinsics __sincosf / __expf, any spin storage type.
// Used by the single-problem kernel (one tile per block) and the batched persistent kernel
// (many tiles of many problems per block).
//
// Tile: TJ half-lattice columns (128, or 64 for narrow lattices) x TY rows. A thread owns 4
// consecutive columns of a row (two same-colour site pairs -> two Philox calls), loaded and stored
// as one vector; a warp step covers one 128-column row or two 64-column rows, and each thread
// handles R rows, so TY = 8 warps x (128 / TJ) x R. The other colour's tile and its one-site halo
// are staged in shared memory as unit vectors (cos q*phi, sin q*phi), computed once per site and
// read by its four neighbours.
#pragma once

#include "mpr_device.cuh"
#include "mpr_internal.h"

namespace mpr {
namespace f32 {

constexpr int kTJ = 128;     // half-lattice columns per tile (single-problem kernels)
constexpr int kWarps = 8;    // 256 threads, blockDim = (32, 8)

// Lanes of a warp per tile row (TJ / 4) and tile rows per warp step.
template <int TJ> struct Lanes {
    static_assert(TJ == 128 || TJ == 64 || TJ == 32, "tile width");
    static constexpr int kPerRow = TJ / 4;
    static constexpr int kRows = 32 / kPerRow;
};

// Twice atan2(y, x) modulo 2*pi, in FP32, as an angle in [-pi, pi] (the over-relaxation needs the
// doubled angle only modulo 2*pi). Reduce to a = min(|x|,|y|)/max(|x|,|y|) in [0, 1] and evaluate
// 2 atan(a) = a*P(a^2); P is a polynomial in a^2 fitted for this library by Lawson's iteratively
// reweighted least squares (a minimax method) to atan on [0, 1], here with every coefficient
// doubled (exact: Horner's rounding commutes with the factor 2). SHORT (16-bit spin storage): 6
// coefficients, max error 1.7e-6 rad (3.5e-6 on the doubled angle in FP32, three orders below the
// storage's 2^-8 rad spacing near 2 pi); otherwise 8 coefficients, max error 3.8e-8 rad.
// In the first quadrant the doubled angle is 2t (|y| <= |x|) or pi - 2t; reflecting into the other
// quadrants maps it to its negative modulo 2 pi (x < 0: 2(pi - t1) = -2 t1; y < 0: -2 t1), so the
// sign of the result is the sign of x*y, applied by flipping the sign bit. The quotient uses the
// approximate FP32 division; x = y = 0 gives NaN.
template <bool SHORT>
__device__ __forceinline__ float atan2_doubled(float y, float x)
{
    const float ax = fabsf(x), ay = fabsf(y);
    const float mx = fmaxf(ax, ay), mn = fminf(ax, ay);
    const float a = __fdividef(mn, mx);
    const float s = a * a;
    float p;
    if constexpr (SHORT) {
        p = -0.023438263684511185f;
        p = fmaf(p, s, 0.10529468208551407f);
        p = fmaf(p, s, -0.23285295069217682f);
        p = fmaf(p, s, 0.38708075881004333f);
        p = fmaf(p, s, -0.6652456521987915f);
        p = fmaf(p, s, 1.9999544620513916f);
    } else {
        p = -0.008109131827950478f;
        p = fmaf(p, s, 0.04372590780258179f);
        p = fmaf(p, s, -0.1118246391415596f);
        p = fmaf(p, s, 0.1928439438343048f);
        p = fmaf(p, s, -0.2781725823879242f);
        p = fmaf(p, s, 0.3989313244819641f);
        p = fmaf(p, s, -0.6665971875190735f);
        p = fmaf(p, s, 1.999998688697815f);
    }
    float t2 = a * p;
    t2 = (ay > ax) ? 3.14159265358979324f - t2 : t2;
    const uint32_t sgn = (__float_as_uint(x) ^ __float_as_uint(y)) & 0x80000000u;
    return __uint_as_float(__float_as_uint(t2) ^ sgn);
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

template <int R, int TJ = kTJ> __host__ __device__ constexpr int tile_rows()
{
    return kWarps * Lanes<TJ>::kRows * R;
}

// Shared tile of the other colour as structure of arrays: column j of the tile at index
// j - j0 + 4 (halo columns at 3 and TJ + 4), so a lane's four interior columns form one aligned
// 16-byte vector and a warp's vector accesses touch consecutive banks.
template <int R, int TJ = kTJ> struct TileSmem {
    float cs[tile_rows<R, TJ>() + 2][TJ + 8];
    float sn[tile_rows<R, TJ>() + 2][TJ + 8];
    double wsum_d[kWarps];
    float wsum_f[kWarps];
};


// 2^x on the MUFU (hand-written PTX: ex2.approx.ftz.f32)
__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Converts one staged row r (tile row y = y0 - 1 + r, parity ob of its columns) of the other
// colour to unit vectors (cos q*phi, sin q*phi) in sm: the thread's four columns from st, the halo
// column j0 - 1 (first lane of the row) or j0 + TJ (second lane) from halo. Entries outside the
// lattice become (0, 0) (open boundaries); CHECK = false when the caller knows every entry exists.
template <typename S, int R, bool CHECK, int TJ>
__device__ __forceinline__ void unit_row(const SweepArgs& a, int r, int y, int j0, int jb, int lj,
                                         int ob, float q, const Pack4<S>& st, S halo,
                                         TileSmem<R, TJ>& sm)
{
    const int lc = threadIdx.x % Lanes<TJ>::kPerRow;   // lane within the row
    const bool row_ok = !CHECK || (y >= 0 && y < a.Ly);
    float vc[4], vs[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        vc[k] = 0.0f;
        vs[k] = 0.0f;
        if (!CHECK || (row_ok && 2 * (jb + k) + ob < a.Lx))
            __sincosf(q * load_as<float>(st.s[k]), &vs[k], &vc[k]);
    }
    *reinterpret_cast<float4*>(&sm.cs[r][4 + lj]) = make_float4(vc[0], vc[1], vc[2], vc[3]);
    *reinterpret_cast<float4*>(&sm.sn[r][4 + lj]) = make_float4(vs[0], vs[1], vs[2], vs[3]);
    if (lc < 2) {   // halo columns j0 - 1 (index 3) and j0 + TJ (index TJ + 4)
        const int j = lc == 0 ? j0 - 1 : j0 + TJ;
        const int cc = lc == 0 ? 3 : TJ + 4;
        float hc = 0.0f, hs = 0.0f;
        if (!CHECK || (row_ok && j >= 0 && 2 * j + ob < a.Lx))
            __sincosf(q * load_as<float>(halo), &hs, &hc);
        sm.cs[r][cc] = hc;
        sm.sn[r][cc] = hs;
    }
}

// Stages the other colour's rows y0-1 .. y0+TY and columns j0-1 .. j0+TJ of a tile from global
// memory as unit vectors. All loads are issued before the sin/cos work.
template <typename S, int R, bool CHECK, int TJ>
__device__ __forceinline__ void stage(const SweepArgs& a, const S* __restrict__ other, int y0,
                                      int j0, int jb, int lj, int cb, float q, TileSmem<R, TJ>& sm)
{
    constexpr int TY = tile_rows<R, TJ>();
    constexpr int HW = Lanes<TJ>::kRows;
    constexpr int NR = (TY + 2 + kWarps * HW - 1) / (kWarps * HW);   // staged rows per thread
    const int warp = threadIdx.y;
    const int lc = threadIdx.x % Lanes<TJ>::kPerRow, lr = threadIdx.x / Lanes<TJ>::kPerRow;
    Pack4<S> st[NR];
    S halo[NR];
#pragma unroll
    for (int i = 0; i < NR; ++i) {
        const int r = (warp + i * kWarps) * HW + lr;
        const int y = y0 - 1 + r;
        if (r < TY + 2 && (!CHECK || (y >= 0 && y < a.Ly))) {
            load4(other + (size_t)y * a.pitch + jb, st[i]);
            if (lc < 2) {
                const int j = lc == 0 ? j0 - 1 : j0 + TJ;
                if (!CHECK || (j >= 0 && 2 * j + ((y + cb) & 1) < a.Lx))
                    halo[i] = other[(size_t)y * a.pitch + j];
            }
        }
    }
#pragma unroll
    for (int i = 0; i < NR; ++i) {
        const int r = (warp + i * kWarps) * HW + lr;
        if (r >= TY + 2) break;
        const int y = y0 - 1 + r;
        unit_row<S, R, CHECK>(a, r, y, j0, jb, lj, (y + cb) & 1, q, st[i], halo[i], sm);
    }
}

// Two FP32 results rounded to a 16-bit storage type by one paired conversion (each half rounds
// exactly as a single conversion would), packed low = a, high = b.
template <typename S> __device__ __forceinline__ uint32_t pack2(float a, float b);
template <> __device__ __forceinline__ uint32_t pack2<__half>(float a, float b)
{
    const __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&h);
}
template <> __device__ __forceinline__ uint32_t pack2<__nv_bfloat16>(float a, float b)
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&h);
}

// Metropolis + over-relaxation of the thread's four columns jb .. jb+3 of tile row ly (lattice
// row y < Ly) of colour a.colour, reading the staged neighbours in sm; pk holds the four stored
// values (updated in place and written back as one vector), bits their frozen bits. SAMPLE: 0
// none, 1 FP64 accumulators, 2 Kahan FP32 accumulators. MEASURE adds u_b . h_b of the row's
// existing (black) sites to e_d or e_f (SAMPLE 3: fixed-point int32 partial sums of FP16
// spins, see below). SCHED: Philox words from the precomputed schedule a.ph
// (a kernel parameter) instead of the seed. OPAR: the row's column offset o = (y + colour) & 1
// when the caller knows it at compile time (0 or 1), else -1. PROP: bounded proposals
// f + pw (2u - 1), rejected outside [0, 2 pi); n_acc counts the accepted ones of updated sites.
// W1: the caller knows q <= 1/2, so the reflected angle needs one 2 pi wrap, not two.
template <typename S, int R, bool MEASURE, int SAMPLE, bool SCHED, int OPAR, bool PROP, bool W1,
          int TJ>
__device__ __forceinline__ void update_row(const SweepArgs& a, int y, int ly, int jb, int lj,
                                           Pack4<S>& pk, uint32_t bits, const TileSmem<R, TJ>& sm,
                                           double& e_d, float& e_f, float pw, int& n_acc)
{
    const int c = a.colour;
    S* __restrict__ own = static_cast<S*>(a.own);
    const float q = a.qf;
    const float nl2e_invT = -1.4426950408889634f * a.invTf;   // exp(-dE/T) = 2^(dE * nl2e_invT)
    const float two_pi = kTwoPiF;
    const float width = two_pi * q;
    const float inv_q = 1.0f / q;
    const int o = OPAR >= 0 ? OPAR : ((y + c) & 1);
    const size_t idx = (size_t)y * a.pitch + jb;
    // entries past the row's end carry frozen bits (padding), so the bit alone decides an update;
    // existence matters only for the energy sum
    bool ex[4], upd[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        ex[k] = 2 * (jb + k) + o < a.Lx;
        upd[k] = !((bits >> k) & 1u);
    }
    // local fields h = sum of the neighbours' unit vectors (left, right, up, down), all four sites
    // first: the neighbour vectors are dead before the moves start
    float hx[4], hy[4];
    {
        // up/down rows at the same columns, the middle row at columns j+o-1, j+o
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
            hx[k] = ((mcv[k] + mcv[k + 1]) + ucv[k]) + dcv[k];
            hy[k] = ((msv[k] + msv[k + 1]) + usv[k]) + dsv[k];
        }
    }
    uint4 w;
    float fn_even = 0.0f;
    float ev[4] = {0.0f, 0.0f, 0.0f, 0.0f};   // MEASURE: u_b . h_b of the row's sites
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        // one Philox call per site pair, whether or not its sites update: no branch per site
        if ((k & 1) == 0) {
            const uint32_t jpair = (uint32_t)((jb >> 1) + (k >> 1));
            if constexpr (SCHED)
                w = pair_words(jpair, (uint32_t)y, a.ph);
            else
                w = pair_words(jpair, (uint32_t)y, a.sweep, a.problem, kTagMetropolis,
                               (uint32_t)c, a.seed_lo, a.seed_hi);
        }
        const float hxk = hx[k], hyk = hy[k];
        float f = load_as<float>(pk.s[k]);
        {
            // every site runs the move; frozen sites and padding discard the result below
            const uint32_t wp = (k & 1) ? w.z : w.x;
            const uint32_t wa = (k & 1) ? w.w : w.y;
            const float u_acc = uniform_f(wa);
            // Metropolis: uniform proposal fp = 2 pi u (or bounded: f + pw (2u - 1), inside
            // [0, 2 pi) only), accept if dE <= 0 or u_acc < exp(-dE/T)
            float fp;
            bool inside = true;
            if constexpr (PROP) {
                fp = fmaf(2.0f * pw, uniform_f(wp), f - pw);
                inside = fp >= 0.0f && fp < two_pi;
            } else {
                fp = fmaf(two_pi, one_plus_uniform_f(wp), -two_pi);
            }
            float s0, c0, sp, cp;
            __sincosf(q * f, &s0, &c0);
            __sincosf(q * fp, &sp, &cp);
            // dE = E(fp) - E(f), E(phi) = -(hx cos q*phi + hy sin q*phi)
            const float dE = hxk * (c0 - cp) + hyk * (s0 - sp);
            const bool accept = inside && (dE <= 0.0f || u_acc < ex2_approx(dE * nl2e_invT));
            if constexpr (PROP) n_acc += (accept && upd[k]) ? 1 : 0;
            const float f1 = accept ? fp : f;
            // over-relaxation: reflect q*phi about arg(h); keep it if it lands in [0, 2*pi*q].
            // h = 0 gives NaN in atan2_doubled, every comparison below is false and the angle
            // stays, as the move requires.
            float r = atan2_doubled<sizeof(S) == 2>(hyk, hxk) - q * f1;   // in [-pi - 2 pi q, pi]
            // r < 0 ? r + 2 pi : r, twice, on the FMA pipe: the saturated product is 1 for every
            // negative normal r and 0 for r >= 0 and NaN; the FMA then adds 2 pi or 0 with the
            // rounding of a plain add. (A nonzero r is never subnormal: its two terms are 0 or at
            // least ~1e-8 in magnitude.)
            // (with q <= 1/2, r >= -2 pi and the first wrap already lands in [0, 2 pi); the second
            // would add 0, so W1 drops it without changing a bit)
            r = fmaf(two_pi, __saturatef(r * -0x1.0p126f), r);
            if constexpr (!W1) r = fmaf(two_pi, __saturatef(r * -0x1.0p126f), r);
            const float fn = r <= width ? r * inv_q : f1;
            if constexpr (sizeof(S) == 2) {
                // 16-bit storage: the pair's two results rounded by one conversion and merged into
                // the pair's 32-bit word under the update mask
                if ((k & 1) == 0) {
                    fn_even = fn;
                } else {
                    const uint32_t m = (upd[k - 1] ? 0x0000FFFFu : 0u) | (upd[k] ? 0xFFFF0000u : 0u);
                    const uint32_t packed = pack2<S>(fn_even, fn);
                    if (k == 1) pk.v.x = (packed & m) | (pk.v.x & ~m);
                    else pk.v.y = (packed & m) | (pk.v.y & ~m);
                }
                if (SAMPLE || MEASURE) f = upd[k] ? load_as<float>(store_from<S>(fn)) : f;
            } else {
                const S stored = store_from<S>(fn);
                pk.s[k] = upd[k] ? stored : pk.s[k];
                f = upd[k] ? load_as<float>(stored) : f;
            }
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
        } else if (SAMPLE == 3) {
            // FP16 spins, FP64 sums: f is an FP16 value, an integer multiple of 2^-24 below
            // 2^3, so f * 2^24 converts to an int exactly and 16 of them fit an int32; the
            // handle folds the partial into the FP64 sum, where every add is exact (the sum stays
            // a multiple of 2^-24 below 2^29): the same bits as adding f itself, with a 4-byte
            // read and write per sample instead of 8-byte ones
            if (upd[k]) a.part32[idx + k] += __float2int_rn(f * 16777216.0f);
        }
        if (MEASURE && ex[k]) {
            // every bond joins a red and a black site: sum over black sites of u_b . h_b
            float sn, cs;
            __sincosf(q * f, &sn, &cs);
            ev[k] = cs * hxk + sn * hyk;
        }
    }
    if (MEASURE) {
        // the row's four FP32 terms pairwise in FP32 (two roundings of the size of the terms'
        // own), then into the thread's FP64 (or FP32) sum: one FP64 add per row instead of four,
        // on a part whose FP64 rate is a small fraction of its FP32 rate
        const float er = (ev[0] + ev[1]) + (ev[2] + ev[3]);
        if (a.flags & kEnergyF32) e_f += er; else e_d += (double)er;
    }
    store4(own + idx, pk);   // unchanged entries are written back with their own bits
}

// The tile's energy partial: warp shuffles, then the warps in order, written by thread (0, 0) to
// *eslot (double, or float with kEnergyF32). Contains a block barrier.
template <int R, int TJ>
__device__ __forceinline__ void tile_energy(const SweepArgs& a, double e_d, float e_f,
                                            TileSmem<R, TJ>& sm, void* eslot)
{
    const int lane = threadIdx.x, warp = threadIdx.y;
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

// Row order of a thread's R rows. With even R (and tile origins at even rows) the thread's rows
// start at an even tile row, so its row rr has o = (rr + colour) & 1, and visiting rr = i ^ colour
// makes o = i & 1 a compile-time constant of the unrolled loop over i. Odd R keeps the natural
// order, o at run time.
template <int R> __device__ __forceinline__ int row_of(int i, int c) { return (R % 2 == 0) ? (i ^ c) : i; }

// update_row of the i-th row in the order row_of(), with o fixed at compile time for even R (the
// branch on i & 1 disappears when the caller's loop over i is unrolled).
template <typename S, int R, bool MEASURE, int SAMPLE, bool SCHED, bool PROP, bool W1, int TJ>
__device__ __forceinline__ void update_row_i(int i, const SweepArgs& a, int y, int ly, int jb,
                                             int lj, Pack4<S>& pk, uint32_t bits,
                                             const TileSmem<R, TJ>& sm, double& e_d, float& e_f,
                                             float pw, int& n_acc)
{
    if constexpr (R % 2 == 0) {
        if (i & 1)
            update_row<S, R, MEASURE, SAMPLE, SCHED, 1, PROP, W1>(a, y, ly, jb, lj, pk, bits, sm, e_d,
                                                              e_f, pw, n_acc);
        else
            update_row<S, R, MEASURE, SAMPLE, SCHED, 0, PROP, W1>(a, y, ly, jb, lj, pk, bits, sm, e_d,
                                                              e_f, pw, n_acc);
    } else {
        update_row<S, R, MEASURE, SAMPLE, SCHED, -1, PROP, W1>(a, y, ly, jb, lj, pk, bits, sm, e_d, e_f,
                                                           pw, n_acc);
    }
}

// Adds the block's accepted bounded proposals to *counter: warp sums, then one atomic per block
// (every block of a pass adds to the same word, so fewer atomics means less serialisation at L2).
// Called by every thread of the block.
__device__ __forceinline__ void count_accepted(int n_acc, unsigned long long* counter)
{
    __shared__ int s_acc[kWarps];
#pragma unroll
    for (int off = 16; off; off >>= 1) n_acc += __shfl_xor_sync(0xffffffffu, n_acc, off);
    if (threadIdx.x == 0) s_acc[threadIdx.y] = n_acc;
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        int t = 0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) t += s_acc[w];
        if (t) atomicAdd(counter, (unsigned long long)t);
    }
}

// One tile (tile column tx, tile row ty) of colour a.colour, staged from global memory. With
// MEASURE (black pass) the tile's sum of u_b . h_b over its existing black sites is written to
// *eslot. Begins with a block barrier, so a block may call it for several tiles in a row.
// PDL (programmatic dependent launch, one tile per block): the block reads its own colour's values
// and bits, then waits for the previous kernel (the other colour's pass), then lets the next
// kernel in the stream start launching. The own colour was last written two passes back, which
// has completed: the previous pass's blocks released this pass only after their own wait.
// Everything the previous pass may write (the other colour, accumulators, energy partials) is
// touched only after the wait.
// PROP: bounded proposals of half-width *a.width; accepted ones counted into *a.accepted.
// W1: the caller has checked q <= 1/2 (one 2 pi wrap of the reflected angle suffices).
template <typename S, int R, bool MEASURE, int SAMPLE, bool SCHED, bool PDL = false,
          bool PROP = false, int TJ = kTJ, bool W1 = false>
__device__ __forceinline__ void sweep_tile(const SweepArgs& a, int tx, int ty, TileSmem<R, TJ>& sm,
                                           void* eslot)
{
    constexpr int TY = tile_rows<R, TJ>();
    const int c = a.colour, cb = c ^ 1;
    const int j0 = tx * TJ;
    const int y0 = ty * TY;
    const int warp = threadIdx.y;
    const int lc = threadIdx.x % Lanes<TJ>::kPerRow, lr = threadIdx.x / Lanes<TJ>::kPerRow;
    const int row0 = (warp * Lanes<TJ>::kRows + lr) * R;   // first of this thread's R tile rows
    const S* __restrict__ other = static_cast<const S*>(a.other);
    const S* __restrict__ own = static_cast<const S*>(a.own);
    const int lj = 4 * lc;
    const int jb = j0 + lj;                   // first of this thread's 4 columns

    // ---- own rows: values and frozen bits, loaded before the staging so their latency overlaps
    Pack4<S> mine[R];   // in the order row_of()
    uint32_t bits[R];
#pragma unroll
    for (int i = 0; i < R; ++i) {
        const int y = y0 + row0 + row_of<R>(i, c);
        bits[i] = 0xFu;
        if (y < a.Ly) {
            load4(own + (size_t)y * a.pitch + jb, mine[i]);
            bits[i] = (a.mbits[(size_t)y * a.mpitch + (jb >> 5)] >> (jb & 31)) & 0xFu;
        }
    }

    if (PDL) {
        asm volatile("griddepcontrol.wait;" ::: "memory");   // the previous pass is complete
        asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    }
    __syncthreads();   // the previous tile's readers are done with sm
    // ---- stage the other colour (rows y0-1 .. y0+TY, columns j0-1 .. j0+TJ). Tiles whose halo
    // lies inside the lattice (nearly all) skip the per-entry bounds checks.
    const bool interior = y0 >= 1 && y0 + TY < a.Ly && j0 >= 1 && 2 * (j0 + TJ) + 1 < a.Lx;
    if (interior) stage<S, R, false>(a, other, y0, j0, jb, lj, cb, a.qf, sm);
    else stage<S, R, true>(a, other, y0, j0, jb, lj, cb, a.qf, sm);
    __syncthreads();

    double e_d = 0.0;
    float e_f = 0.0f;
    const float pw = PROP ? (float)*a.width : 0.0f;   // written before this pass (stream order)
    int n_acc = 0;
#pragma unroll
    for (int i = 0; i < R; ++i) {
        const int ly = row0 + row_of<R>(i, c);
        const int y = y0 + ly;
        if (y < a.Ly)
            update_row_i<S, R, MEASURE, SAMPLE, SCHED, PROP, W1>(i, a, y, ly, jb, lj, mine[i], bits[i],
                                                             sm, e_d, e_f, pw, n_acc);
    }
    if (PROP && a.accepted) count_accepted(n_acc, a.accepted);
    if (MEASURE) tile_energy(a, e_d, e_f, sm, eslot);
}

}  // namespace f32
}  // namespace mpr
