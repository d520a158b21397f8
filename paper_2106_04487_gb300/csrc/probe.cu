// Pipe-rate probe: the lane-operation throughput of the arithmetic pipes that bound the near and
// far kernels (FP32 FMA, packed FP32x2 FMA, and the MUFU approximations ex2 / rsqrt / sqrt / rcp),
// measured with CUDA events on a grid that fills every SM.  It is the measured denominator of the
// kernels' ALU rooflines, not part of the product.
#include "fkt_internal.h"
#include "ptx.cuh"

namespace fkt {
namespace {

constexpr int kChains = 8;  // independent dependency chains per thread

template <int OP>
__global__ void __launch_bounds__(256) probe_kernel(int64_t iters, float seed, float* out) {
    float v[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = seed + 1e-3f * (threadIdx.x + c);
    float2 w[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) w[c] = make_float2(v[c], v[c] + 0.5f);
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) {
            if (OP == 0) v[c] = fmaf(v[c], 0.999f, 1e-4f);                      // FP32 FMA
            else if (OP == 1) v[c] = ptx::ex2(-v[c]);                            // MUFU ex2
            else if (OP == 2) v[c] = ptx::rsqrt_approx(v[c] + 1.0f);             // MUFU rsqrt (+ FADD)
            else if (OP == 3) v[c] = ptx::sqrt_approx(v[c]);                     // MUFU sqrt
            else if (OP == 4) v[c] = ptx::rcp_approx(v[c] + 1.0f);               // MUFU rcp (+ FADD)
            else w[c] = __ffma2_rn(w[c], make_float2(0.999f, 0.999f), make_float2(1e-4f, 1e-4f));  // FFMA2
        }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += OP == 5 ? w[c].x + w[c].y : v[c];
    if (s == 12345.678f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;  // keeps the loop alive
}

template <int OP>
int run_probe(int64_t iters, int blocks, float* buf, cudaEvent_t e0, cudaEvent_t e1, float* ms) {
    probe_kernel<OP><<<blocks, 256>>>(iters / 8, 0.5f, buf);  // warm-up
    FKT_CUDA_TRY(cudaEventRecord(e0));
    probe_kernel<OP><<<blocks, 256>>>(iters, 0.5f, buf);
    FKT_CUDA_TRY(cudaEventRecord(e1));
    FKT_CUDA_TRY(cudaEventSynchronize(e1));
    FKT_CUDA_TRY(cudaGetLastError());
    FKT_CUDA_TRY(cudaEventElapsedTime(ms, e0, e1));
    return FKT_OK;
}

}  // namespace
}  // namespace fkt

extern "C" int fkt_probe_pipe_rate(int op, int64_t iters, double* lane_ops_per_second) {
    using namespace fkt;
    if (op < 0 || op > 5 || iters < 1 || iters > (int64_t)1 << 32 || !lane_ops_per_second) return FKT_ERR_INVALID_ARG;
    int dev = 0, nsm = 0;
    FKT_CUDA_TRY(cudaGetDevice(&dev));
    FKT_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = nsm * 8;  // 2048 threads per SM
    float* buf = nullptr;
    FKT_CUDA_TRY(cudaMalloc(&buf, sizeof(float) * blocks * 256));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float ms = 0.f;
    int rc = FKT_ERR_INVALID_ARG;
    switch (op) {
    case 0: rc = run_probe<0>(iters, blocks, buf, e0, e1, &ms); break;
    case 1: rc = run_probe<1>(iters, blocks, buf, e0, e1, &ms); break;
    case 2: rc = run_probe<2>(iters, blocks, buf, e0, e1, &ms); break;
    case 3: rc = run_probe<3>(iters, blocks, buf, e0, e1, &ms); break;
    case 4: rc = run_probe<4>(iters, blocks, buf, e0, e1, &ms); break;
    default: rc = run_probe<5>(iters, blocks, buf, e0, e1, &ms); break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(buf);
    if (rc) return rc;
    const double lanes = (double)blocks * 256.0 * (double)iters * kChains * (op == 5 ? 2.0 : 1.0);
    *lane_ops_per_second = lanes / (ms * 1e-3);
    return FKT_OK;
}
