// mufu_rate.cu -- throughput of the special-function unit (MUFU) instructions the FP32 sweep uses:
// sin.approx, cos.approx, ex2.approx and rcp.approx (the reciprocal inside the FP32 quotient), in
// operations per second on device 0. Measurement infrastructure for the roofline of bench.py (the
// peaks file holds no MUFU figure): every thread runs 8 independent chains of one operation each,
// with finite, normal operands throughout, on 8 resident blocks per SM, after a warm-up that
// brings the clocks up; the best of three timed runs counts. Prints one JSON object.
#include <cstdio>
#include <cuda_runtime.h>

namespace {

template <int OP>
__global__ void __launch_bounds__(256) chains(float* out, int iters)
{
    float a[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = 0.25f + 0.001f * (float)((threadIdx.x + i) & 63);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            float y;
            if (OP == 0) asm volatile("sin.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(a[i]));
            if (OP == 1) asm volatile("cos.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(a[i]));
            if (OP == 2) asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(a[i]));
            if (OP == 3) asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(a[i]));
            // every operand stays a finite normal number in the range the sweep uses. sin and
            // cos feed their result straight back (the iterates stay in (0, 1)); ex2 feeds back
            // -2y, so 2^a converges to 1/2 with a in [-2.4, 0) and never reaches a special
            // operand (inf, 0 or a subnormal, which the unit may pass through at another rate);
            // rcp gets one dependent FMA (the iterate settles near 0.84), so no two reciprocals
            // can be folded into one another. sin and cos, like the sweep's, carry the one
            // multiply of their range scaling
            a[i] = OP == 3 ? y * 0.5f + 0.25f : (OP == 2 ? -2.0f * y : y);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i) s += a[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <int OP>
double rate(float* out, int blocks, int iters, cudaEvent_t e0, cudaEvent_t e1)
{
    double best = 0.0;
    for (int rep = 0; rep < 4; ++rep) {   // the first run warms up; keep the fastest
        cudaEventRecord(e0);
        chains<OP><<<blocks, 256>>>(out, iters);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double r = (double)blocks * 256 * iters * 8 / (ms * 1e-3);
        if (rep > 0 && r > best) best = r;
    }
    return best;
}

}  // namespace

int main()
{
    int nsm = 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, 0) != cudaSuccess) {
        printf("{\"error\": \"no CUDA device\"}\n");
        return 1;
    }
    const int blocks = nsm * 8, iters = 2048;
    float* out = nullptr;
    if (cudaMalloc(&out, sizeof(float) * blocks * 256) != cudaSuccess) {
        printf("{\"error\": \"cudaMalloc failed\"}\n");
        return 1;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // bring the clocks up first: about 0.2 s of the sin kernel
    for (int i = 0; i < 100; ++i) chains<0><<<blocks, 256>>>(out, iters);
    cudaDeviceSynchronize();
    const double r_sin = rate<0>(out, blocks, iters, e0, e1);
    const double r_cos = rate<1>(out, blocks, iters, e0, e1);
    const double r_ex2 = rate<2>(out, blocks, iters, e0, e1);
    const double r_rcp = rate<3>(out, blocks, iters, e0, e1);
    const cudaError_t err = cudaGetLastError();
    cudaFree(out);
    if (err != cudaSuccess) {
        printf("{\"error\": \"%s\"}\n", cudaGetErrorString(err));
        return 1;
    }
    printf("{\"sms\": %d, \"sin_per_s\": %.6e, \"cos_per_s\": %.6e, \"ex2_per_s\": %.6e, "
           "\"rcp_per_s\": %.6e}\n", nsm, r_sin, r_cos, r_ex2, r_rcp);
    return 0;
}
