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
    // the black pass (a programmatic edge) has completed: its bookkeeping is visible
    asm volatile("griddepcontrol.wait;" ::: "memory");
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
    if (shape < 0 || shape >= batch::kShapes) return batch::Kernels{nullptr, nullptr, 0, nullptr};
    switch (store) {
    case kF64: return batch::kernels_f64(shape);
    case kF32: return batch::kernels_f32(shape);
    case kF16: return batch::kernels_f16(shape);
    case kBF16: return batch::kernels_bf16(shape);
    default: return batch::Kernels{nullptr, nullptr, 0, nullptr};
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

namespace {

// A kernel node of `body` after `dep` (none if null); programmatic: the node may launch once
// every block of `dep` has released it (griddepcontrol.launch_dependents) or exited.
cudaError_t add_kernel(cudaGraphNode_t* node, cudaGraph_t body, const cudaGraphNode_t* dep,
                       bool programmatic, const void* func, int grid, size_t smem, void** params)
{
    cudaGraphNodeParams np{};
    np.type = cudaGraphNodeTypeKernel;
    np.kernel.func = const_cast<void*>(func);
    np.kernel.gridDim = dim3(grid);
    np.kernel.blockDim = dim3(32, f32::kWarps);
    np.kernel.sharedMemBytes = (unsigned)smem;
    np.kernel.kernelParams = params;
    cudaGraphEdgeData ed{};
    if (programmatic) {
        ed.from_port = cudaGraphKernelNodePortProgrammatic;
        ed.type = cudaGraphDependencyTypeProgrammatic;
    }
    return cudaGraphAddNode(node, body, dep, dep ? &ed : nullptr, dep ? 1 : 0, &np);
}

cudaError_t graph_build(const void* pass, size_t smem, int max_tiles, bool programmatic,
                        const batch::Args* args_dev, const PhiloxSched& keys, cudaGraphExec_t* out)
{
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
    void* params_r[] = {const_cast<batch::Args**>(&args_dev), const_cast<int*>(&red),
                        const_cast<PhiloxSched*>(&keys)};
    void* params_b[] = {const_cast<batch::Args**>(&args_dev), const_cast<int*>(&black),
                        const_cast<PhiloxSched*>(&keys)};
    void* params_f[] = {const_cast<batch::Args**>(&args_dev), &loop};
    cudaGraphNode_t n_red, n_black, n_fin;
    if (e == cudaSuccess) e = add_kernel(&n_red, body, nullptr, false, pass, max_tiles, smem, params_r);
    if (e == cudaSuccess)
        e = add_kernel(&n_black, body, &n_red, programmatic, pass, max_tiles, smem, params_b);
    if (e == cudaSuccess)
        e = add_kernel(&n_fin, body, &n_black, programmatic,
                       reinterpret_cast<const void*>(&batch::finish_kernel), 1, 0, params_f);
    if (e == cudaSuccess) e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    return e;
}

}  // namespace

cudaError_t batch_graph_build(int store, int shape, int max_tiles, bool qhalf,
                              const batch::Args* args_dev, const PhiloxSched& keys,
                              cudaGraphExec_t* out)
{
    const batch::Kernels kk = kernels_for(store, shape);
    const void* pass = (qhalf && kk.pass_qhalf) ? kk.pass_qhalf : kk.pass;
    if (!pass || max_tiles < 1) return cudaErrorInvalidValue;
    if (graph_build(pass, kk.smem, max_tiles, true, args_dev, keys, out) == cudaSuccess)
        return cudaSuccess;
    cudaGetLastError();   // the runtime refused the programmatic edges: plain ones
    return graph_build(pass, kk.smem, max_tiles, false, args_dev, keys, out);
}

}  // namespace mpr
