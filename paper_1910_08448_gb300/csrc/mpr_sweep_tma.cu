// mpr_sweep_tma.cu -- single-problem colour half-sweep for the FP32 function setting, sweep kernel
// kind 1, plain passes: persistent blocks (as many per SM as the shared memory allows: 4 with
// 16-bit spins) walk 128 x 32 tiles u = blockIdx.x, blockIdx.x + gridDim.x, ...; while a block
// updates tile u, the TMA unit copies the next tile's three boxes (other colour with halo, own
// values, own frozen bits) into shared memory, completing on one mbarrier, so the staging step is
// pure sin/cos work. When the tiles left after the whole rounds of the grid fit one round as
// halves, they run as half-height units, so the last round takes half as long. Blocks that walk
// equal tiles stay in step with each other (all convert, then all update); the handle keeps this
// kernel only where its own timing finds it faster than kind 0 (mpr_sweep_f32.cu). Also the
// tensor maps (cuTensorMapEncodeTiled through the runtime's driver entry point).
#include "mpr.h"
#include "mpr_tile_f32.cuh"
#include "mpr_tma.cuh"

#include <cudaTypedefs.h>   // PFN_cuTensorMapEncodeTiled

namespace mpr {
namespace {

using namespace f32;

constexpr int kTmaRows = 4;   // rows per thread of the TMA kernel's tiles (128 x 32)

// Shared memory of the TMA kernel: the boxes the TMA unit writes (other colour rows y0-1 ..
// y0+TY over columns j0-HL .. j0+TJ+HL-1; own rows; own mask words), the unit-vector tile, and
// the barrier the copies complete on.
template <typename S, int R> struct TmaSmem {
    static constexpr int TY = kWarps * R;
    static constexpr int HL = 16 / (int)sizeof(S);   // one 16-byte chunk left and right of the tile
    static constexpr int BW = kTJ + 2 * HL;
    static constexpr int MW = kTJ / 32;              // mask words per tile row
    static constexpr uint32_t kBytes =
        (uint32_t)(sizeof(S) * ((TY + 2) * BW + TY * kTJ) + 4 * TY * MW);
    alignas(128) S other[TY + 2][BW];
    alignas(128) S own[TY][kTJ];
    alignas(128) uint32_t mbits[TY][MW];
    alignas(16) TileSmem<R> t;
    uint64_t bar;
    int ok;
};

// Unit vectors of the other colour from the TMA box (see stage() for the global-memory form), for
// a tile of RT rows per thread (RT = R, or R / 2 for a half-height tile, which uses the box's
// first TY / 2 + 2 rows). As in stage(), the work is spread evenly: rows 0 .. TYT-1 as 4-entry
// vectors (RT per warp, the halo entries by lanes 0 and 1), the last two rows one entry per
// thread and their four halo entries by threads 0 .. 3.
template <typename S, int R, int RT, bool CHECK>
__device__ __forceinline__ void convert(const SweepArgs& a, const TmaSmem<S, R>& sm, int y0,
                                        int j0, int jb, int lj, int cb, float q, TileSmem<RT>& t)
{
    using Sm = TmaSmem<S, R>;
    constexpr int TYT = kWarps * RT;
    static_assert(2 * kTJ == 32 * kWarps, "one entry of the last two rows per thread");
    const int lane = threadIdx.x, warp = threadIdx.y;
    const int tid = warp * 32 + lane;
#pragma unroll
    for (int i = 0; i < RT; ++i) {
        const int r = warp + i * kWarps;
        const int y = y0 - 1 + r;
        Pack4<S> st;
        load4(&sm.other[r][Sm::HL + lj], st);
        const S halo = sm.other[r][lane == 0 ? Sm::HL - 1 : Sm::HL + kTJ];
        unit_row<S, RT, CHECK>(a, r, y, j0, jb, lj, (y + cb) & 1, q, st, halo, t);
    }
    {
        const int er = TYT + tid / kTJ, ec = tid % kTJ;
        const int ey = y0 - 1 + er;
        float vc = 0.0f, vs = 0.0f;
        if (!CHECK || (ey < a.Ly && 2 * (j0 + ec) + ((ey + cb) & 1) < a.Lx))
            __sincosf(q * load_as<float>(sm.other[er][Sm::HL + ec]), &vs, &vc);
        t.cs[er][4 + ec] = vc;
        t.sn[er][4 + ec] = vs;
    }
    if (tid < 4) {
        const int hr = TYT + (tid >> 1), side = tid & 1;
        const int hy = y0 - 1 + hr, hj = side ? j0 + kTJ : j0 - 1;
        float hc = 0.0f, hs = 0.0f;
        if (!CHECK || (hy < a.Ly && hj >= 0 && 2 * hj + ((hy + cb) & 1) < a.Lx))
            __sincosf(q * load_as<float>(sm.other[hr][side ? Sm::HL + kTJ : Sm::HL - 1]), &hs, &hc);
        t.cs[hr][side ? kTJ + 4 : 3] = hc;
        t.sn[hr][side ? kTJ + 4 : 3] = hs;
    }
}

// Origin of work unit u of a pass: units below nfull are whole tiles in row-major order; unit
// nfull + k is half k & 1 (the upper or lower TY / 2 rows) of tile nfull + (k >> 1).
struct Unit {
    int j0, y0;
    bool half;
};
__device__ __forceinline__ Unit unit_of(int u, int nfull, int ntx, int TY)
{
    if (u < nfull) return {(u % ntx) * kTJ, (u / ntx) * TY, false};
    const int k = u - nfull, t = nfull + (k >> 1);
    return {(t % ntx) * kTJ, (t / ntx) * TY + (k & 1) * (TY / 2), true};
}

// One work unit of RT rows per thread whose boxes have landed: own values and bits to registers,
// unit vectors of the other colour, a block barrier, the next unit's copies (leader, next >= 0),
// then the update of the unit's rows.
template <typename S, int R, int RT, int QM, typename Issue>
__device__ __forceinline__ void tma_unit(const SweepArgs& a, TmaSmem<S, R>& sm, int j0, int y0,
                                         int next, bool leader, Issue&& issue)
{
    constexpr int TYT = kWarps * RT;
    TileSmem<RT>& t = *reinterpret_cast<TileSmem<RT>*>(&sm.t);
    const int lane = threadIdx.x, warp = threadIdx.y;
    const int lj = 4 * lane, jb = j0 + lj;
    const int cb = a.colour ^ 1;
    Pack4<S> mine[RT];
    uint32_t bits[RT];
#pragma unroll
    for (int i = 0; i < RT; ++i) {   // rows in the order row_of()
        const int ly = warp * RT + row_of<RT>(i, a.colour);
        load4(&sm.own[ly][lj], mine[i]);
        bits[i] = (sm.mbits[ly][lane >> 3] >> (lj & 31)) & 0xFu;
    }
    const bool interior = y0 >= 1 && y0 + TYT < a.Ly && j0 >= 1 && 2 * (j0 + kTJ) + 1 < a.Lx;
    const float qs = QM == 2 ? 0.5f : a.qf;
    if (interior) convert<S, R, RT, false>(a, sm, y0, j0, jb, lj, cb, qs, t);
    else convert<S, R, RT, true>(a, sm, y0, j0, jb, lj, cb, qs, t);
    __syncthreads();   // unit vectors complete; the boxes are free for the next unit
    if (leader && next >= 0) {
        tma::fence_proxy_async();
        issue(next);
    }

    double e_d = 0.0;   // unused: no energy in plain passes
    float e_f = 0.0f;
    int n_acc = 0;      // unused: uniform proposals only
    GroupCarry gc{0u, 0u, 0u, 0u};
#pragma unroll
    for (int i = 0; i < RT; ++i) {
        const int ly = warp * RT + row_of<RT>(i, a.colour);
        const int y = y0 + ly;
        if (RT % 2 == 0 && (i & 1) && y < a.Ly && y0 + warp * RT + row_of<RT>(i - 1, a.colour) >= a.Ly)
            group_carry_only<true>(a, y, jb, gc);
        if (y < a.Ly)
            update_row_i<S, RT, false, 0, true, false, QM>(i, a, y, ly, jb, lj, mine[i], bits[i], t,
                                                          e_d, e_f, 0.0f, n_acc, gc);
    }
}

// Plain passes only (no fused energy, no sampling): the handle runs those passes with
// sweep_f32_kernel, whose per-tile energy partials it reduces. QM as in sweep_tile (2: q = 1/2 at
// compile time, the 16-bit storages only). Blocks per SM as the shared memory allows: 4 with
// 16-bit spins (64 registers), 3 with FP32 and 2 with FP64 spins.
// Launched as a programmatic dependent launch: the leader issues the first tile's own-colour and
// mask copies (the own colour was last written two passes back, which has completed), every
// thread waits for the previous pass, the next pass is released, and only then is the other
// colour copied; results are written after the block barrier that follows.
template <typename S, int R, int QM>
__global__ void __launch_bounds__(256, sizeof(S) == 2 ? 4 : (sizeof(S) == 4 ? 3 : 2))
    sweep_f32_tma_kernel(const SweepArgs a, const __grid_constant__ CUtensorMap m_other,
                         const __grid_constant__ CUtensorMap m_own,
                         const __grid_constant__ CUtensorMap m_mask)
{
    using Sm = TmaSmem<S, R>;
    constexpr int TY = Sm::TY;
    extern __shared__ __align__(128) unsigned char dsm[];
    Sm& sm = *reinterpret_cast<Sm*>(dsm);
    const bool leader = threadIdx.x == 0 && threadIdx.y == 0;
    const int ntx = (a.Lxh + kTJ - 1) / kTJ;
    const int ntiles = ntx * ((a.Ly + TY - 1) / TY);
    const int nfull = ntiles - a.nsplit;          // the last nsplit tiles run as two halves each
    const int nunits = nfull + 2 * a.nsplit;

    // one thread issues the three copies of unit u (full-height boxes also for a half tile);
    // x offsets are multiples of 16 bytes
    auto issue = [&](int u) {
        const Unit w = unit_of(u, nfull, ntx, TY);
        tma::arrive_expect_tx(&sm.bar, Sm::kBytes);
        tma::load_2d(&sm.other[0][0], &m_other, &sm.bar, w.j0 - Sm::HL, w.y0 - 1);
        tma::load_2d(&sm.own[0][0], &m_own, &sm.bar, w.j0, w.y0);
        tma::load_2d(&sm.mbits[0][0], &m_mask, &sm.bar, w.j0 / 32, w.y0);
    };
    // the leader waits for unit `it`'s copies; a wait that runs out records the error, waits once
    // more for the copy in flight, and stops the block at the next barrier
    auto await = [&](uint32_t it) {
        if (!tma::wait(&sm.bar, it & 1u, a.wait_ns)) {
            if (a.err) atomicExch(a.err, (int)MPR_ERR_DEVICE_TIMEOUT);
            tma::wait(&sm.bar, it & 1u, a.wait_ns);
            sm.ok = 0;
        }
    };

    int u = blockIdx.x;
    const bool first = leader && u < nunits && !(a.stall_test && blockIdx.x == 0);
    if (leader) {
        sm.ok = 1;
        tma::mbar_init(&sm.bar, 1);
    }
    if (first) {
        const Unit w = unit_of(u, nfull, ntx, TY);
        tma::arrive_expect_tx(&sm.bar, Sm::kBytes);
        tma::load_2d(&sm.own[0][0], &m_own, &sm.bar, w.j0, w.y0);
        tma::load_2d(&sm.mbits[0][0], &m_mask, &sm.bar, w.j0 / 32, w.y0);
    }
    asm volatile("griddepcontrol.wait;" ::: "memory");   // the previous pass is complete
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    if (leader && u < nunits) {
        if (first) {
            const Unit w = unit_of(u, nfull, ntx, TY);
            tma::load_2d(&sm.other[0][0], &m_other, &sm.bar, w.j0 - Sm::HL, w.y0 - 1);
        }
        await(0);
    }
    __syncthreads();
    for (uint32_t it = 0; u < nunits; ++it) {
        if (!sm.ok) return;   // uniform: read after a block barrier
        const Unit w = unit_of(u, nfull, ntx, TY);
        const int un = u + (int)gridDim.x;
        const int next = un < nunits ? un : -1;
        if (R % 2 == 0 && w.half) tma_unit<S, R, R / 2, QM>(a, sm, w.j0, w.y0, next, leader, issue);
        else tma_unit<S, R, R, QM>(a, sm, w.j0, w.y0, next, leader, issue);
        if (leader && next >= 0) await(it + 1);
        __syncthreads();   // the unit vectors' readers are done; sm.ok is current
        u = un;
    }
}

template <typename S, int QM>
cudaError_t go_tma_q(const SweepArgs& a, const TmaMaps& m, int nsm, cudaStream_t st)
{
    using Sm = TmaSmem<S, kTmaRows>;
    auto kern = sweep_f32_tma_kernel<S, kTmaRows, QM>;
    // per instantiation, once: shared-memory opt-in and the resident blocks per SM
    static const int bps = [&] {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Sm));
        cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, 256, sizeof(Sm)) != cudaSuccess)
            n = 1;
        return n < 1 ? 1 : n;
    }();
    const int ntiles = ((a.Lxh + kTJ - 1) / kTJ) * ((a.Ly + Sm::TY - 1) / Sm::TY);
    const int slots = nsm * bps;
    // last round: when the tiles left over after whole rounds of the grid, split into halves,
    // still fit one round, they run as half-height units (that round takes half as long)
    SweepArgs b = a;
    const int rem = ntiles % slots;
    b.nsplit = (ntiles > slots && rem > 0 && 2 * rem <= slots) ? rem : 0;
    const int nunits = ntiles + b.nsplit;
    const int grid = nunits < slots ? nunits : slots;
    const int c = a.colour;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(32, kWarps);
    cfg.dynamicSmemBytes = sizeof(Sm);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, b, m.other[c ^ 1], m.own[c], m.mask[c]);
}

template <typename S>
cudaError_t go_tma(const SweepArgs& a, const TmaMaps& m, int nsm, cudaStream_t st)
{
    if (a.flags & (kMeasure | kSample)) return cudaErrorInvalidValue;   // plain passes only
    if constexpr (sizeof(S) == 2) {
        if (a.qf == 0.5f) return go_tma_q<S, 2>(a, m, nsm, st);
    }
    return go_tma_q<S, 0>(a, m, nsm, st);
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                             &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            f = nullptr;
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    }();
    return fn;
}

// 2-D map over a row-major [rows][cols] array with a row stride of cols elements.
bool encode(CUtensorMap* m, CUtensorMapDataType dt, size_t esize, void* base, int cols, int rows,
            int box_x, int box_y)
{
    auto fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)cols * esize};
    const cuuint32_t box[2] = {(cuuint32_t)box_x, (cuuint32_t)box_y};
    const cuuint32_t estr[2] = {1, 1};
    return fn(m, dt, 2, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <typename S>
bool make_maps_typed(const Layout& L, CUtensorMapDataType dt, void* const ang[2],
                     uint32_t* const mb[2], TmaMaps* out)
{
    using Sm = TmaSmem<S, kTmaRows>;
    // the boxes must fit inside the arrays: at least two tile columns and TY + 2 rows
    if (L.pitch < Sm::BW || L.Ly < Sm::TY + 2) return false;
    for (int c = 0; c < 2; ++c) {
        if (!encode(&out->other[c], dt, sizeof(S), ang[c], L.pitch, L.Ly, Sm::BW, Sm::TY + 2) ||
            !encode(&out->own[c], dt, sizeof(S), ang[c], L.pitch, L.Ly, kTJ, Sm::TY) ||
            !encode(&out->mask[c], CU_TENSOR_MAP_DATA_TYPE_UINT32, 4, mb[c], L.mpitch, L.Ly,
                    Sm::MW, Sm::TY))
            return false;
    }
    return true;
}

}  // namespace

bool make_sweep_maps(const Layout& L, int store, void* const ang[2], uint32_t* const mb[2],
                     TmaMaps* out)
{
    bool ok = false;
    switch (store) {
    case kF64: ok = make_maps_typed<double>(L, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, ang, mb, out); break;
    case kF32: ok = make_maps_typed<float>(L, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, ang, mb, out); break;
    case kF16: ok = make_maps_typed<__half>(L, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, ang, mb, out); break;
    case kBF16: ok = make_maps_typed<__nv_bfloat16>(L, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, ang, mb, out); break;
    default: break;
    }
    out->ok = ok;
    return ok;
}

cudaError_t launch_sweep_f32_tma(const Precision& p, const SweepArgs& a, const TmaMaps& m, int nsm,
                                 cudaStream_t st)
{
    switch (p.store) {
    case kF64: return go_tma<double>(a, m, nsm, st);
    case kF32: return go_tma<float>(a, m, nsm, st);
    case kF16: return go_tma<__half>(a, m, nsm, st);
    case kBF16: return go_tma<__nv_bfloat16>(a, m, nsm, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace mpr
