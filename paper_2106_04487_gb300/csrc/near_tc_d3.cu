#include <algorithm>

// Tensor-core near-field kernel instantiations for d = 3 (one translation unit per dimension).
#include "near_tc2.cuh"

namespace fkt {

__global__ void near_image_kernel(int64_t nnodes, const int32_t* __restrict__ nd_leaf,
                                  const int32_t* __restrict__ nd_begin, const int32_t* __restrict__ nd_end,
                                  const int32_t* __restrict__ nd_img, const float4* __restrict__ rec, int rec_f4,
                                  float* __restrict__ img) {
    constexpr int GF = kNearGroupFloats;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    const float* rf = reinterpret_cast<const float*>(rec);
    const int64_t rs = 4 * (int64_t)rec_f4;  // floats per record
    for (int64_t nd = blockIdx.x; nd < nnodes; nd += gridDim.x) {
        if (!nd_leaf[nd]) continue;
        const int b = nd_begin[nd], n = nd_end[nd] - b;
        const int ng = (n + 7) / 8 * 2;
        float* base = img + (int64_t)(nd_img[nd] / 4) * GF;
        for (int g = warp; g < ng; g += nwarps) {
            float* gp = base + (int64_t)g * GF;
            uint32_t h[4], l[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int k = 4 * g + i;
                const float v = k < n ? rf[(int64_t)(b + k) * rs + 4 + lane] : 0.f;
                split_tf32(v, h[i], l[i]);
            }
            *reinterpret_cast<uint4*>(gp + 4 * lane) = make_uint4(h[0], h[1], h[2], h[3]);
            *reinterpret_cast<uint4*>(gp + 128 + 4 * lane) = make_uint4(l[0], l[1], l[2], l[3]);
            if (lane < 16) {
                const int comp = lane >> 2, k = 4 * g + (lane & 3);
                gp[256 + lane] = k < n ? -rf[(int64_t)(b + k) * rs + comp] : 0.f;
            }
        }
    }
}

void launch_near_image(int64_t nnodes, const int32_t* nd_leaf, const int32_t* nd_begin, const int32_t* nd_end,
                       const int32_t* nd_img, const float4* rec, int rec_f4, float* img, cudaStream_t st) {
    if (nnodes <= 0) return;
    const unsigned g = (unsigned)std::min<int64_t>(nnodes, 152 * 16);
    near_image_kernel<<<g, 256, 0, st>>>(nnodes, nd_leaf, nd_begin, nd_end, nd_img, rec, rec_f4, img);
}

void launch_near_tc_d3(int kind, unsigned grid, cudaStream_t st, const MvmArgs& a, const KernelParams& kp) {
    launch_near_tc_dim<3>(kind, grid, st, a, kp);
}

void launch_near_tc2_d3(int kind, unsigned grid, cudaStream_t st, const MvmArgs& a, const KernelParams& kp,
                         unsigned* wmax) {
    cudaMemsetAsync(wmax, 0, sizeof(unsigned) * 32, st);
    const unsigned g = (unsigned)std::min<int64_t>((a.N + 255) / 256, 152 * 4);
    near_wscale_kernel<3><<<g, 256, 0, st>>>(a.N, a.rec, a.rec_f4, 4, a.nr, wmax);
    launch_near_tc2_dim<3>(kind, grid, st, a, kp, wmax);
}

}  // namespace fkt
