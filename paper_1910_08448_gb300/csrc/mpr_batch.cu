// mpr_batch.cu -- host side of the batched kernels: the kernel table of a storage type and tile
// shape, occupancy, the persistent launch (direct or as a one-node graph) and the graph-mode
// executable with its device-side while loop; and the finish kernel of graph mode.
#include "mpr_batch_kernels.cuh"

namespace mpr {
namespace batch {

__global__ void __launch_bounds__(256) finish_kernel(const Args* __restrict__ A,
                                                     cudaGraphConditionalHandle loop)
{
    __shared__ int s_scan[256];
    Ctl* ctl = A->ctl;
    const bool t0 = threadIdx.x == 0 && threadIdx.y == 0;
    if (__ldcg(&ctl->changed)) {   // a problem finished in this sweep: shrink the tile list
        const int sel = __ldcg(&ctl->list_sel);
        compact_list(A, A->lists + (size_t)sel * A->ntiles, __ldcg(&ctl->n_list),
                     A->lists + (size_t)(sel ^ 1) * A->ntiles, &ctl->n_list, s_scan);
        if (t0) {
            ctl->list_sel = sel ^ 1;
            ctl->changed = 0;
        }
    }
    if (t0) {
        const int it = ctl->iters + 1;
        ctl->iters = it;
        __threadfence();
        cudaGraphSetConditional(loop, (__ldcg(&ctl->n_active) > 0 && it < A->max_iters) ? 1u : 0u);
    }
}

}  // namespace batch

namespace {

batch::Kernels kernels_for(int store, int shape)
{
    if (shape < 0 || shape >= batch::kShapes) return batch::Kernels{nullptr, nullptr, 0};
    switch (store) {
    case kF64: return batch::kernels_f64(shape);
    case kF32: return batch::kernels_f32(shape);
    case kF16: return batch::kernels_f16(shape);
    case kBF16: return batch::kernels_bf16(shape);
    default: return batch::Kernels{nullptr, nullptr, 0};
    }
}

}  // namespace

cudaError_t batch_occupancy(int store, int shape, int* blocks_per_sm)
{
    const batch::Kernels k = kernels_for(store, shape);
    if (!k.persistent) return cudaErrorInvalidValue;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k.persistent, 256, k.smem);
}

cudaError_t batch_launch(int store, int shape, int grid, const batch::Args* args_dev,
                         const PhiloxSched& keys, cudaStream_t st, bool use_graph)
{
    const batch::Kernels kk = kernels_for(store, shape);
    const void* k = kk.persistent;
    if (!k) return cudaErrorInvalidValue;
    void* params[] = {const_cast<batch::Args**>(&args_dev), const_cast<PhiloxSched*>(&keys)};
    if (!use_graph)
        return cudaLaunchCooperativeKernel(k, dim3(grid), dim3(32, f32::kWarps), params, kk.smem, st);
    // the same launch as a one-node CUDA graph with a cooperative kernel node
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    cudaKernelNodeParams kp{};
    kp.func = const_cast<void*>(k);
    kp.gridDim = dim3(grid);
    kp.blockDim = dim3(32, f32::kWarps);
    kp.sharedMemBytes = (unsigned)kk.smem;
    kp.kernelParams = params;
    cudaError_t e = cudaGraphCreate(&g, 0);
    cudaGraphNode_t node;
    if (e == cudaSuccess) e = cudaGraphAddKernelNode(&node, g, nullptr, 0, &kp);
    if (e == cudaSuccess) {
        cudaLaunchAttributeValue v{};
        v.cooperative = 1;
        e = cudaGraphKernelNodeSetAttribute(node, cudaLaunchAttributeCooperative, &v);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&ge, g, 0);
    if (e == cudaSuccess) e = cudaGraphLaunch(ge, st);
    if (ge) cudaGraphExecDestroy(ge);
    if (g) cudaGraphDestroy(g);
    return e;
}

cudaError_t batch_graph_build(int store, int shape, int max_tiles, const batch::Args* args_dev,
                              const PhiloxSched& keys, cudaGraphExec_t* out)
{
    const batch::Kernels kk = kernels_for(store, shape);
    const void* pass = kk.pass;
    if (!pass || max_tiles < 1) return cudaErrorInvalidValue;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaGraphCreate(&g, 0);
    if (e != cudaSuccess) return e;
    cudaGraphConditionalHandle loop;
    e = cudaGraphConditionalHandleCreate(&loop, g, 1u, cudaGraphCondAssignDefault);
    cudaGraphNode_t wnode;
    cudaGraph_t body = nullptr;
    if (e == cudaSuccess) {
        cudaGraphNodeParams cp{};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = loop;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        e = cudaGraphAddNode(&wnode, g, nullptr, nullptr, 0, &cp);
        if (e == cudaSuccess) body = cp.conditional.phGraph_out[0];
    }
    const int red = 0, black = 1;
    cudaGraphNode_t n_red, n_black, n_fin;
    if (e == cudaSuccess) {
        void* params[] = {const_cast<batch::Args**>(&args_dev), const_cast<int*>(&red),
                          const_cast<PhiloxSched*>(&keys)};
        cudaKernelNodeParams kp{};
        kp.func = const_cast<void*>(pass);
        kp.gridDim = dim3(max_tiles);
        kp.blockDim = dim3(32, f32::kWarps);
        kp.sharedMemBytes = (unsigned)kk.smem;
        kp.kernelParams = params;
        e = cudaGraphAddKernelNode(&n_red, body, nullptr, 0, &kp);
        if (e == cudaSuccess) {
            void* params_b[] = {const_cast<batch::Args**>(&args_dev), const_cast<int*>(&black),
                                const_cast<PhiloxSched*>(&keys)};
            kp.kernelParams = params_b;
            e = cudaGraphAddKernelNode(&n_black, body, &n_red, 1, &kp);
        }
    }
    if (e == cudaSuccess) {
        void* params[] = {const_cast<batch::Args**>(&args_dev), &loop};
        cudaKernelNodeParams kp{};
        kp.func = reinterpret_cast<void*>(&batch::finish_kernel);
        kp.gridDim = dim3(1);
        kp.blockDim = dim3(32, f32::kWarps);
        kp.sharedMemBytes = 0;
        kp.kernelParams = params;
        e = cudaGraphAddKernelNode(&n_fin, body, &n_black, 1, &kp);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    return e;
}

}  // namespace mpr
