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

// Two FP32 lanes per instruction (Blackwell's packed FP32 arithmetic: __ffma2_rn, __fadd2_rn,
// __fmul2_rn). Each lane rounds exactly as the scalar FP32 operation would, so a pair of sites
// computed in float2 gets the same bits as the two sites computed one by one; the kernel is
// bound by instruction issue, and a packed instruction issues once for both sites.
__device__ __forceinline__ float2 splat(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
// a - b with one rounding (the product b * -1 is exact)
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, splat(-1.0f), a); }

// 1 / x on the MUFU (hand-written PTX: rcp.approx.ftz.f32)
__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// atan2_doubled of two sites at once: the same reduction and polynomial, the multiplies and the
// polynomial in float2. The quotient is min * rcp(max) (approximate reciprocal on the MUFU); both
// lanes NaN-propagate as the scalar version does when x = y = 0.
template <bool SHORT>
__device__ __forceinline__ float2 atan2_doubled2(float2 y, float2 x)
{
    const float ax0 = fabsf(x.x), ay0 = fabsf(y.x), ax1 = fabsf(x.y), ay1 = fabsf(y.y);
    const float2 mx = make_float2(fmaxf(ax0, ay0), fmaxf(ax1, ay1));
    const float2 mn = make_float2(fminf(ax0, ay0), fminf(ax1, ay1));
    const float2 a = mul2(mn, make_float2(rcp_approx(mx.x), rcp_approx(mx.y)));
    const float2 s = mul2(a, a);
    float2 p;
    if constexpr (SHORT) {
        p = splat(-0.023438263684511185f);
        p = fma2(p, s, splat(0.10529468208551407f));
        p = fma2(p, s, splat(-0.23285295069217682f));
        p = fma2(p, s, splat(0.38708075881004333f));
        p = fma2(p, s, splat(-0.6652456521987915f));
        p = fma2(p, s, splat(1.9999544620513916f));
    } else {
        p = splat(-0.008109131827950478f);
        p = fma2(p, s, splat(0.04372590780258179f));
        p = fma2(p, s, splat(-0.1118246391415596f));
        p = fma2(p, s, splat(0.1928439438343048f));
        p = fma2(p, s, splat(-0.2781725823879242f));
        p = fma2(p, s, splat(0.3989313244819641f));
        p = fma2(p, s, splat(-0.6665971875190735f));
        p = fma2(p, s, splat(1.999998688697815f));
    }
    const float2 t2 = mul2(a, p);
    const float2 u = sub2(splat(3.14159265358979324f), t2);
    const float r0 = ay0 > ax0 ? u.x : t2.x, r1 = ay1 > ax1 ? u.y : t2.y;
    // the sign of x*y (a product that underflows keeps its sign; r0, r1 >= 0 or NaN)
    const float2 xy = mul2(x, y);
    return make_float2(copysignf(r0, xy.x), copysignf(r1, xy.y));
}

// atan2_doubled2 in the FP16-function setting (X_F = H: FP16 arithmetic where it is safe, the
// paper's future work of Sec. 3): the field is rounded to FP16, and the ratio of its smaller to
// its larger component and the polynomial run in half2 arithmetic, both sites per instruction.
// The polynomial has 3 coefficients (a*P(a^2) ~ 2 atan(a) on [0, 1], fitted for this library by
// Lawson's iteratively reweighted least squares, rounded to FP16): 1.2e-3 rad minimax, 2.4e-3 rad
// evaluated in FP16, near the FP16 spacing of the result (9.8e-4 on [1, 2)). PTX has no FP16
// reciprocal, so the larger component's reciprocal is the FP32 one. The fold pi - 2t and the
// sign stay in FP32: pi (and 2 pi in the later wraps) rounded to FP16 would shift every
// reflection that uses it by about 1e-3 rad in the same direction.
__device__ __forceinline__ float2 atan2_doubled_h2(float2 y, float2 x)
{
    const __half2 xh = __float22half2_rn(x), yh = __float22half2_rn(y);
    const __half2 axh = __habs2(xh), ayh = __habs2(yh);
    const __half2 mx = __hmax2(axh, ayh), mn = __hmin2(axh, ayh);
    const float2 mxf = __half22float2(mx);
    const __half2 a = __hmul2(mn, __floats2half2_rn(rcp_approx(mxf.x), rcp_approx(mxf.y)));
    const __half2 s = __hmul2(a, a);
    __half2 p = __hfma2(__float2half2_rn(0.15869140625f), s, __float2half2_rn(-0.5771484375f));
    p = __hfma2(p, s, __float2half2_rn(1.990234375f));
    const float2 t2 = __half22float2(__hmul2(a, p));
    const float2 u = sub2(splat(3.14159265358979324f), t2);
    const float2 ax = __half22float2(axh), ay = __half22float2(ayh);
    const float r0 = ay.x > ax.x ? u.x : t2.x, r1 = ay.y > ax.y ? u.y : t2.y;
    const float2 xy = mul2(x, y);
    return make_float2(copysignf(r0, xy.x), copysignf(r1, xy.y));
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
// colour to unit vectors (cos q*phi, sin q*phi) in sm: the thread's four columns from st and, with
// HALO, the halo column j0 - 1 (first lane of the row) or j0 + TJ (second lane) from halo. Entries
// outside the lattice become (0, 0) (open boundaries); CHECK = false when the caller knows every
// entry exists.
template <typename S, int R, bool CHECK, int TJ, bool HALO = true>
__device__ __forceinline__ void unit_row(const SweepArgs& a, int r, int y, int j0, int jb, int lj,
                                         int ob, float q, const Pack4<S>& st, S halo,
                                         TileSmem<R, TJ>& sm)
{
    const int lc = threadIdx.x % Lanes<TJ>::kPerRow;   // lane within the row
    const bool row_ok = !CHECK || (y >= 0 && y < a.Ly);
    float vc[4], vs[4];
    if constexpr (!CHECK) {
        // q * phi of the four entries as two float2 products
        const float2 a01 = mul2(splat(q), make_float2(load_as<float>(st.s[0]), load_as<float>(st.s[1])));
        const float2 a23 = mul2(splat(q), make_float2(load_as<float>(st.s[2]), load_as<float>(st.s[3])));
        __sincosf(a01.x, &vs[0], &vc[0]);
        __sincosf(a01.y, &vs[1], &vc[1]);
        __sincosf(a23.x, &vs[2], &vc[2]);
        __sincosf(a23.y, &vs[3], &vc[3]);
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            vc[k] = 0.0f;
            vs[k] = 0.0f;
            if (row_ok && 2 * (jb + k) + ob < a.Lx)
                __sincosf(q * load_as<float>(st.s[k]), &vs[k], &vc[k]);
        }
    }
    *reinterpret_cast<float4*>(&sm.cs[r][4 + lj]) = make_float4(vc[0], vc[1], vc[2], vc[3]);
    *reinterpret_cast<float4*>(&sm.sn[r][4 + lj]) = make_float4(vs[0], vs[1], vs[2], vs[3]);
    if (HALO && lc < 2) {   // halo columns j0 - 1 (index 3) and j0 + TJ (index TJ + 4)
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
// memory as unit vectors. All loads are issued before the sin/cos work. The work is spread evenly
// over the block: staged rows 0 .. TY-1 as 4-entry vectors (the same number per warp), the last
// two rows (TY, TY+1) one entry per thread, and the 2 (TY + 2) halo entries (columns j0 - 1 and
// j0 + TJ) one per thread of the block's first threads, so no warp converts a row more than the
// others and none runs a halo branch with two of its lanes.
template <typename S, int R, bool CHECK, int TJ>
__device__ __forceinline__ void stage(const SweepArgs& a, const S* __restrict__ other, int y0,
                                      int j0, int jb, int lj, int cb, float q, TileSmem<R, TJ>& sm)
{
    constexpr int TY = tile_rows<R, TJ>();
    constexpr int HW = Lanes<TJ>::kRows;
    static_assert(TY % (kWarps * HW) == 0, "vector rows split evenly over the warps");
    constexpr int NR = TY / (kWarps * HW);   // vector rows per thread
    constexpr int NH = 2 * (TY + 2);         // halo entries
    constexpr int NE = 2 * TJ;               // entries of the last two rows
    static_assert(NH <= 32 * kWarps && NE <= 32 * kWarps, "one entry per thread");
    const int warp = threadIdx.y;
    const int lr = threadIdx.x / Lanes<TJ>::kPerRow;
    const int tid = warp * 32 + threadIdx.x;
    Pack4<S> st[NR];
    // this thread's halo entry: row hr = tid / 2, column j0 - 1 (tid even) or j0 + TJ (odd)
    const int hr = tid >> 1, hj = (tid & 1) ? j0 + TJ : j0 - 1;
    const int hy = y0 - 1 + hr;
    const bool hok = tid < NH && (!CHECK || (hy >= 0 && hy < a.Ly && hj >= 0 &&
                                             2 * hj + ((hy + cb) & 1) < a.Lx));
    // this thread's entry of the last two rows: row er = TY + tid / TJ, column j0 + tid % TJ
    const int er = TY + tid / TJ, ej = j0 + tid % TJ;
    const int ey = y0 - 1 + er;
    const bool eok = tid < NE && (!CHECK || (ey < a.Ly && 2 * ej + ((ey + cb) & 1) < a.Lx));
    S hv{}, evl{};
    if (hok) hv = other[(size_t)hy * a.pitch + hj];
    if (eok) evl = other[(size_t)ey * a.pitch + ej];
#pragma unroll
    for (int i = 0; i < NR; ++i) {
        const int r = (warp + i * kWarps) * HW + lr;
        const int y = y0 - 1 + r;
        if (!CHECK || (y >= 0 && y < a.Ly)) load4(other + (size_t)y * a.pitch + jb, st[i]);
    }
#pragma unroll
    for (int i = 0; i < NR; ++i) {
        const int r = (warp + i * kWarps) * HW + lr;
        const int y = y0 - 1 + r;
        unit_row<S, R, CHECK, TJ, false>(a, r, y, j0, jb, lj, (y + cb) & 1, q, st[i], S{}, sm);
    }
    if (tid < NE) {
        float ec = 0.0f, es = 0.0f;
        if (eok) __sincosf(q * load_as<float>(evl), &es, &ec);
        sm.cs[er][4 + tid % TJ] = ec;
        sm.sn[er][4 + tid % TJ] = es;
    }
    if (tid < NH) {
        float hc = 0.0f, hs = 0.0f;
        if (hok) __sincosf(q * load_as<float>(hv), &hs, &hc);
        const int cc = (tid & 1) ? TJ + 4 : 3;
        sm.cs[hr][cc] = hc;
        sm.sn[hr][cc] = hs;
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

// Metropolis random numbers of the FP32-function setting. Every uniform has 23 bits, so three
// Philox-4x32-10 calls (384 bits) serve a group of eight same-colour sites: the thread's four
// half-lattice columns jb .. jb+3 (g = jb >> 2) in the two rows 2h, 2h + 1 (h = y >> 1); call
// sub (0, 1, 2) has counter (g, h, sweep, problem << 8 | sub << 2 | colour). The group's first
// row is the one with y + colour even (the thread visits it first, see row_of). In the first row
// the site pair t uses call t like the two-site layout: sites 2t, 2t + 1 take the top 23 bits of
// words (x, y) and (z, w) for proposal and acceptance. In the second row site i takes the top 23
// bits of word i of call 2 for its proposal, and its acceptance from the calls' low bytes (which
// no top-23-bit field touches): site i gets bytes 3i, 3i+1, 3i+2 of the twelve words' low bytes
// in call order, 23 bits of them. GroupCarry holds the first row's low bytes for the second row.
struct GroupCarry {
    uint32_t a0, a1;   // second-row sites 0, 1: bytes (W0, W1, W2), (W3, W4, W5) low bytes
    uint32_t p2;       // site 2: bytes W6, W7 (W8 comes from call 2)
    uint32_t w3;       // call 0's last word until call 1 completes a1
};

template <bool SCHED>
__device__ __forceinline__ uint4 group_call(const SweepArgs& a, uint32_t g, uint32_t h, uint32_t sub)
{
    if constexpr (SCHED)
        return pair_words(g, h, a.ph, sub);
    else
        return pair_words(g, h, a.sweep, a.problem, kTagMetropolis, (uint32_t)a.colour, a.seed_lo,
                          a.seed_hi, sub);
}

// the low bytes of (x, y) in bytes 0, 1 of the result
__device__ __forceinline__ uint32_t low2(uint32_t x, uint32_t y) { return __byte_perm(x, y, 0x0040u); }
// bytes 0, 1 of p and the low byte of z in bytes 0, 1, 2
__device__ __forceinline__ uint32_t low3(uint32_t p, uint32_t z) { return __byte_perm(p, z, 0x0410u); }

// The first row's low bytes, from its two calls (or from recomputed calls when that row lies
// outside the lattice).
__device__ __forceinline__ void carry_call0(GroupCarry& gc, const uint4& w)
{
    gc.a0 = low3(low2(w.x, w.y), w.z);
    gc.w3 = w.w;
}
__device__ __forceinline__ void carry_call1(GroupCarry& gc, const uint4& w)
{
    gc.a1 = low3(low2(gc.w3, w.x), w.y);
    gc.p2 = low2(w.z, w.w);
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
// QM: 0 any q; 1 the caller knows q <= 1/2, so the reflected angle needs one 2 pi wrap, not two;
// 2 q = 1/2 (the paper's value) at compile time: q*phi of the accepted angle is the proposal's
// or the old angle's product (both computed for the energy), and r/q is r + r (exact).
template <typename S, int R, bool MEASURE, int SAMPLE, bool SCHED, int OPAR, bool PROP, int QM,
          int TJ, int ROW, bool HM>
__device__ __forceinline__ void update_row(const SweepArgs& a, int y, int ly, int jb, int lj,
                                           Pack4<S>& pk, uint32_t bits, const TileSmem<R, TJ>& sm,
                                           double& e_d, float& e_f, float pw, int& n_acc,
                                           GroupCarry& gc)
{
    const int c = a.colour;
    S* __restrict__ own = static_cast<S*>(a.own);
    constexpr bool QH = QM == 2;
    const float q = QH ? 0.5f : a.qf;
    // exp(-dE/T) = 2^(dE * nl2e): nl2e = -log2(e) * (1/T), the FP32 product formed by the caller
    const float nl2e = a.nl2eTf;
    const float two_pi = kTwoPiF;
    const float width = QH ? 3.14159265358979324f : two_pi * q;
    const float inv_q = QH ? 2.0f : 1.0f / q;
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
    // local fields h = sum of the neighbours' unit vectors (left, right, up, down), sites 2t and
    // 2t + 1 in lanes x and y of hx2[t], hy2[t]; all four sites first: the neighbour vectors are
    // dead before the moves start. Order of the sums: ((left + right) + up) + down.
    float2 hx2[2], hy2[2];
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
        hx2[0] = add2(add2(make_float2(mcv[0] + mcv[1], mcv[1] + mcv[2]), make_float2(uc.x, uc.y)),
                      make_float2(dc.x, dc.y));
        hx2[1] = add2(add2(make_float2(mcv[2] + mcv[3], mcv[3] + mcv[4]), make_float2(uc.z, uc.w)),
                      make_float2(dc.z, dc.w));
        hy2[0] = add2(add2(make_float2(msv[0] + msv[1], msv[1] + msv[2]), make_float2(us.x, us.y)),
                      make_float2(ds.x, ds.y));
        hy2[1] = add2(add2(make_float2(msv[2] + msv[3], msv[3] + msv[4]), make_float2(us.z, us.w)),
                      make_float2(ds.z, ds.w));
    }
    float ev[4] = {0.0f, 0.0f, 0.0f, 0.0f};   // MEASURE: u_b . h_b of the row's sites
    float fsamp[4];                            // SAMPLE: the row's sampled angles (0: frozen)
    // Random numbers (see GroupCarry), whether or not the sites update: no branch per site.
    // ROW 0: first row of the group; 1: second row (gc from the first); 2: the thread's only row
    // of the group (odd rows per thread: the group's other row belongs to another thread), whose
    // role follows from y + colour.
    const uint32_t g = (uint32_t)(jb >> 2), h = (uint32_t)(y >> 1);
    uint4 w2 = make_uint4(0u, 0u, 0u, 0u);
    uint4 wl0 = w2, wl1 = w2;
    bool second = ROW == 1;
    if constexpr (ROW == 2 || ROW == 0) {
        if constexpr (ROW == 2) second = ((y + c) & 1) != 0;
        wl0 = group_call<SCHED>(a, g, h, 0u);
        wl1 = group_call<SCHED>(a, g, h, 1u);
        carry_call0(gc, wl0);
        carry_call1(gc, wl1);
    }
    if constexpr (ROW != 0) w2 = group_call<SCHED>(a, g, h, 2u);
    const uint32_t a2 = low3(gc.p2, w2.x), a3 = low3(low2(w2.y, w2.z), w2.w);
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        const int k0 = 2 * t, k1 = 2 * t + 1;   // the pair's sites (lanes x and y)
        // 1 + u of the pair's proposal (op) and acceptance (oa) uniforms
        float2 op, oa;
        {
            uint4 w;
            if constexpr (ROW == 0 || ROW == 2) {
                w = t == 0 ? wl0 : wl1;
            }
            const float2 op_f = make_float2(one_plus_uniform_f(w.x), one_plus_uniform_f(w.z));
            const float2 oa_f = make_float2(one_plus_uniform_f(w.y), one_plus_uniform_f(w.w));
            const float2 op_s = t == 0 ? make_float2(one_plus_uniform_f(w2.x), one_plus_uniform_f(w2.y))
                                       : make_float2(one_plus_uniform_f(w2.z), one_plus_uniform_f(w2.w));
            const float2 oa_s = t == 0 ? make_float2(one_plus_low23_f(gc.a0), one_plus_low23_f(gc.a1))
                                       : make_float2(one_plus_low23_f(a2), one_plus_low23_f(a3));
            if constexpr (ROW == 0) {
                op = op_f;
                oa = oa_f;
            } else if constexpr (ROW == 1) {
                op = op_s;
                oa = oa_s;
            } else {
                op = second ? op_s : op_f;
                oa = second ? oa_s : oa_f;
            }
        }
        const float2 hx = hx2[t], hy = hy2[t];
        const float2 f = make_float2(load_as<float>(pk.s[k0]), load_as<float>(pk.s[k1]));
        // every site runs the move; a frozen site (or padding) rejects both moves, so its result
        // is its own value
        // Metropolis: uniform proposal fp = 2 pi u (or bounded: f + pw (2u - 1), inside
        // [0, 2 pi) only), accept if dE <= 0 or u_acc < exp(-dE/T). The first word of a site
        // drives its proposal, the second its acceptance.
        const float2 u_acc = add2(oa, splat(-1.0f));
        float2 fp;
        bool inside0 = true, inside1 = true;
        if constexpr (PROP) {
            const float2 u_p = add2(op, splat(-1.0f));
            fp = fma2(splat(2.0f * pw), u_p, add2(f, splat(-pw)));
            inside0 = (fp.x >= 0.0f) & (fp.x < two_pi);
            inside1 = (fp.y >= 0.0f) & (fp.y < two_pi);
        } else if constexpr (!QH) {
            fp = fma2(splat(two_pi), op, splat(-two_pi));
        }
        // q * phi of the old angle and of the proposal. With q = 1/2 and uniform proposals,
        // q * fp = pi * (1 + u) - pi rounded once, and fp = 2 * (q * fp) exactly: the same bits as
        // fp = 2 pi (1 + u) - 2 pi rounded once, then halved.
        const float2 qf = mul2(splat(q), f);
        float2 qp;
        if constexpr (QH && !PROP) {
            qp = fma2(splat(3.14159265358979324f), op, splat(-3.14159265358979324f));
            fp = add2(qp, qp);
        } else {
            qp = mul2(splat(q), fp);
        }
        float2 s0, c0, sp, cp;
        __sincosf(qf.x, &s0.x, &c0.x);
        __sincosf(qf.y, &s0.y, &c0.y);
        __sincosf(qp.x, &sp.x, &cp.x);
        __sincosf(qp.y, &sp.y, &cp.y);
        // dE = E(fp) - E(f), E(phi) = -(hx cos q*phi + hy sin q*phi)
        const float2 dE = fma2(hx, sub2(c0, cp), mul2(hy, sub2(s0, sp)));
        const float2 ea = make_float2(dE.x * nl2e, dE.y * nl2e);
        // both exponentials always (no branch per site); the decisions combine without
        // short-circuit evaluation
        const float e0 = ex2_approx(ea.x), e1 = ex2_approx(ea.y);
        const bool acc0 = upd[k0] & inside0 & ((dE.x <= 0.0f) | (u_acc.x < e0));
        const bool acc1 = upd[k1] & inside1 & ((dE.y <= 0.0f) | (u_acc.y < e1));
        if constexpr (PROP) n_acc += (acc0 ? 1 : 0) + (acc1 ? 1 : 0);
        const float2 f1 = make_float2(acc0 ? fp.x : f.x, acc1 ? fp.y : f.y);
        // over-relaxation: reflect q*phi about arg(h); keep it if it lands in [0, 2*pi*q].
        // h = 0 gives NaN in atan2_doubled2, every comparison below is false and the angle
        // stays, as the move requires.
        float2 r;   // in [-pi - 2 pi q, pi]
        if constexpr (QH) {
            const float2 qf1 = make_float2(acc0 ? qp.x : qf.x, acc1 ? qp.y : qf.y);   // q * f1, exact
            r = sub2(HM ? atan2_doubled_h2(hy, hx) : atan2_doubled2<sizeof(S) == 2>(hy, hx), qf1);
        } else {
            r = fma2(splat(-q), f1,
                     HM ? atan2_doubled_h2(hy, hx) : atan2_doubled2<sizeof(S) == 2>(hy, hx));
        }
        // r < 0 ? r + 2 pi : r, twice: the saturated product is 1 for every negative normal r
        // and 0 for r >= 0 and NaN; the FMA then adds 2 pi or 0 with the rounding of a plain
        // add. (A nonzero r is never subnormal: its two terms are 0 or at least ~1e-8 in
        // magnitude.) With q <= 1/2, r >= -2 pi and the first wrap already lands in [0, 2 pi);
        // the second would add 0, so QM > 0 drops it without changing a bit.
        r = fma2(splat(two_pi), make_float2(__saturatef(r.x * -0x1.0p126f),
                                            __saturatef(r.y * -0x1.0p126f)), r);
        if constexpr (QM == 0)
            r = fma2(splat(two_pi), make_float2(__saturatef(r.x * -0x1.0p126f),
                                                __saturatef(r.y * -0x1.0p126f)), r);
        const float2 rq = QH ? add2(r, r) : mul2(r, splat(inv_q));
        float2 fn = make_float2(upd[k0] & (r.x <= width) ? rq.x : f1.x,
                                upd[k1] & (r.y <= width) ? rq.y : f1.y);
        if constexpr (sizeof(S) == 2) {
            // 16-bit storage: the pair's two results rounded by one paired conversion; a frozen
            // site's own value converts back to its stored bits exactly
            const uint32_t packed = pack2<S>(fn.x, fn.y);
            if (t == 0) pk.v.x = packed; else pk.v.y = packed;
            if (SAMPLE || MEASURE) {
                Pack4<S> back;
                back.v.x = packed;
                fn = make_float2(load_as<float>(back.s[0]), load_as<float>(back.s[1]));
            }
        } else if constexpr (sizeof(S) == 4) {
            pk.s[k0] = fn.x;   // exact for a frozen site
            pk.s[k1] = fn.y;
        } else {
            // FP64 storage: a frozen site's FP64 value is not an FP32 value; keep it
            if (upd[k0]) pk.s[k0] = store_from<S>(fn.x);
            if (upd[k1]) pk.s[k1] = store_from<S>(fn.y);
            fn = make_float2(load_as<float>(pk.s[k0]), load_as<float>(pk.s[k1]));
        }
        // the site's angle after the move, as stored (SAMPLE and MEASURE use it); a frozen site
        // (or padding) contributes 0 to the sums below, which leaves them unchanged
        fsamp[k0] = upd[k0] ? fn.x : 0.0f;
        fsamp[k1] = upd[k1] ? fn.y : 0.0f;
        if (MEASURE) {
            // every bond joins a red and a black site: sum over black sites of u_b . h_b
            const float2 qn = mul2(splat(q), fn);
            float2 sn, cs;
            __sincosf(qn.x, &sn.x, &cs.x);
            __sincosf(qn.y, &sn.y, &cs.y);
            const float2 e2 = fma2(cs, hx, mul2(sn, hy));
            ev[k0] = ex[k0] ? e2.x : 0.0f;
            ev[k1] = ex[k1] ? e2.y : 0.0f;
        }
    }
    // Sampling: the row's four sums updated by one vector read and write (the thread's columns
    // are 4-aligned, rows 128-aligned); frozen sites add 0.
    if constexpr (SAMPLE == 1) {
        double2* p = reinterpret_cast<double2*>(a.acc + idx);
        double2 s0 = p[0], s1 = p[1];
        s0.x += (double)fsamp[0];
        s0.y += (double)fsamp[1];
        s1.x += (double)fsamp[2];
        s1.y += (double)fsamp[3];
        p[0] = s0;
        p[1] = s1;
    } else if constexpr (SAMPLE == 2) {
        // Kahan: hi carries the sum, lo the (negated) lost low-order part
        float4* ph = reinterpret_cast<float4*>(a.acc_hi + idx);
        float4* pl = reinterpret_cast<float4*>(a.acc_lo + idx);
        const float4 h4 = *ph, l4 = *pl;
        const float hv[4] = {h4.x, h4.y, h4.z, h4.w}, lv[4] = {l4.x, l4.y, l4.z, l4.w};
        float nh[4], nl[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float yv = fsamp[k] - lv[k];
            const float tt = hv[k] + yv;
            nl[k] = (tt - hv[k]) - yv;
            nh[k] = tt;
        }
        *ph = make_float4(nh[0], nh[1], nh[2], nh[3]);
        *pl = make_float4(nl[0], nl[1], nl[2], nl[3]);
    } else if constexpr (SAMPLE == 3) {
        // FP16 spins, FP64 sums: f is an FP16 value, an integer multiple of 2^-24 below 2^3, so
        // f * 2^24 converts to an int exactly and 16 of them fit an int32; the handle folds the
        // partial into the FP64 sum, where every add is exact (the sum stays a multiple of 2^-24
        // below 2^29): the same bits as adding f itself, with a 4-byte read and write per sample
        // instead of 8-byte ones
        int4* p = reinterpret_cast<int4*>(a.part32 + idx);
        int4 v = *p;
        v.x += __float2int_rn(fsamp[0] * 16777216.0f);
        v.y += __float2int_rn(fsamp[1] * 16777216.0f);
        v.z += __float2int_rn(fsamp[2] * 16777216.0f);
        v.w += __float2int_rn(fsamp[3] * 16777216.0f);
        *p = v;
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
// With even R, i even is the first row of its Philox group (see GroupCarry) and i odd the second;
// with odd R each row computes its group's three calls itself.
template <typename S, int R, bool MEASURE, int SAMPLE, bool SCHED, bool PROP, int QM, int TJ,
          bool HM = false>
__device__ __forceinline__ void update_row_i(int i, const SweepArgs& a, int y, int ly, int jb,
                                             int lj, Pack4<S>& pk, uint32_t bits,
                                             const TileSmem<R, TJ>& sm, double& e_d, float& e_f,
                                             float pw, int& n_acc, GroupCarry& gc)
{
    if constexpr (R % 2 == 0) {
        if (i & 1)
            update_row<S, R, MEASURE, SAMPLE, SCHED, 1, PROP, QM, TJ, 1, HM>(a, y, ly, jb, lj, pk, bits,
                                                                       sm, e_d, e_f, pw, n_acc, gc);
        else
            update_row<S, R, MEASURE, SAMPLE, SCHED, 0, PROP, QM, TJ, 0, HM>(a, y, ly, jb, lj, pk, bits,
                                                                       sm, e_d, e_f, pw, n_acc, gc);
    } else {
        update_row<S, R, MEASURE, SAMPLE, SCHED, -1, PROP, QM, TJ, 2, HM>(a, y, ly, jb, lj, pk, bits, sm,
                                                                    e_d, e_f, pw, n_acc, gc);
    }
}

// A thread's first row of a Philox group lies outside the lattice (odd Ly) while its second row
// exists: the second row still needs the first row's low bytes.
template <bool SCHED>
__device__ __forceinline__ void group_carry_only(const SweepArgs& a, int y, int jb, GroupCarry& gc)
{
    const uint32_t g = (uint32_t)(jb >> 2), h = (uint32_t)(y >> 1);
    carry_call0(gc, group_call<SCHED>(a, g, h, 0u));
    carry_call1(gc, group_call<SCHED>(a, g, h, 1u));
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
// *eslot. A block that runs several tiles in a row passes a block barrier between them (the
// staging overwrites sm; the batched persistent kernel has one after every tile).
// PDL (programmatic dependent launch, one tile per block): the block reads its own colour's values
// and bits, then waits for the previous kernel (the other colour's pass), then lets the next
// kernel in the stream start launching. The own colour was last written two passes back, which
// has completed: the previous pass's blocks released this pass only after their own wait.
// Everything the previous pass may write (the other colour, accumulators, energy partials) is
// touched only after the wait.
// PROP: bounded proposals of half-width *a.width; accepted ones counted into *a.accepted.
// QM: 1 the caller has checked q <= 1/2 (one 2 pi wrap of the reflected angle suffices); 2 q = 1/2.
// HM: FP16-function setting (the field's doubled angle in half2 arithmetic, atan2_doubled_h2).
// LATE: each own row's values and bits are loaded just before the row's update instead of all
// before the staging: fewer live registers, the better choice when the state sits in L2 (the
// loads are short) and the worse one when they come from DRAM (the host decides).
template <typename S, int R, bool MEASURE, int SAMPLE, bool SCHED, bool PDL = false,
          bool PROP = false, int TJ = kTJ, int QM = 0, bool HM = false, bool LATE = false>
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
    // (LATE: at each row's update)
    Pack4<S> mine[LATE ? 1 : R];   // in the order row_of()
    uint32_t bits[LATE ? 1 : R];
    if constexpr (!LATE) {
#pragma unroll
        for (int i = 0; i < R; ++i) {
            const int y = y0 + row0 + row_of<R>(i, c);
            bits[i] = 0xFu;
            if (y < a.Ly) {
                load4(own + (size_t)y * a.pitch + jb, mine[i]);
                bits[i] = (a.mbits[(size_t)y * a.mpitch + (jb >> 5)] >> (jb & 31)) & 0xFu;
            }
        }
    }

    if (PDL) {
        asm volatile("griddepcontrol.wait;" ::: "memory");   // the previous pass is complete
        asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    }
    // ---- stage the other colour (rows y0-1 .. y0+TY, columns j0-1 .. j0+TJ). Tiles whose halo
    // lies inside the lattice (nearly all) skip the per-entry bounds checks.
    const bool interior = y0 >= 1 && y0 + TY < a.Ly && j0 >= 1 && 2 * (j0 + TJ) + 1 < a.Lx;
    const float qs = QM == 2 ? 0.5f : a.qf;
    if (interior) stage<S, R, false>(a, other, y0, j0, jb, lj, cb, qs, sm);
    else stage<S, R, true>(a, other, y0, j0, jb, lj, cb, qs, sm);
    __syncthreads();

    double e_d = 0.0;
    float e_f = 0.0f;
    const float pw = PROP ? (float)*a.width : 0.0f;   // written before this pass (stream order)
    int n_acc = 0;
    GroupCarry gc{0u, 0u, 0u, 0u};
#pragma unroll
    for (int i = 0; i < R; ++i) {
        const int ly = row0 + row_of<R>(i, c);
        const int y = y0 + ly;
        if (R % 2 == 0 && (i & 1) && y < a.Ly && y0 + row0 + row_of<R>(i - 1, c) >= a.Ly)
            group_carry_only<SCHED>(a, y, jb, gc);
        if (y < a.Ly) {
            const int k = LATE ? 0 : i;
            if constexpr (LATE) {
                load4(own + (size_t)y * a.pitch + jb, mine[0]);
                bits[0] = (a.mbits[(size_t)y * a.mpitch + (jb >> 5)] >> (jb & 31)) & 0xFu;
            }
            update_row_i<S, R, MEASURE, SAMPLE, SCHED, PROP, QM, TJ, HM>(i, a, y, ly, jb, lj, mine[k], bits[k],
                                                             sm, e_d, e_f, pw, n_acc, gc);
        }
    }
    if (PROP && a.accepted) count_accepted(n_acc, a.accepted);
    if (MEASURE) tile_energy(a, e_d, e_f, sm, eslot);
}

}  // namespace f32
}  // namespace mpr
