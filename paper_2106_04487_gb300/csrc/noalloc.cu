// fkt_mvm_noalloc: the FKT product with its per-call work buffers carved out of one
// statically declared device array instead of cudaMalloc'd plan buffers (for callers that
// cannot allocate; see include/fkt.h).  The kernels and their order are those of fkt_mvm.
#include <mutex>

#include "fkt_internal.h"

namespace fkt {

namespace {

constexpr size_t kScratchFloats = FKT_NOALLOC_SCRATCH_BYTES / sizeof(float);

// The scratch itself.  In host code this name is only a stand-in for the device array:
// kernels must be given the address that cudaGetSymbolAddress returns for the current device.
static __device__ __align__(256) float g_noalloc_scratch[kScratchFloats];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
float* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch on the plan's device, looked up once per device.  That device
// must be the current one: the symbol lookup and the kernels both act on the current device, so
// a call made while another device is current is rejected instead of handing the plan's kernels
// another device's address.
int scratch_for_plan_device(const fkt_plan_s* P, float** out) {
    int dev = 0;
    FKT_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != P->device) return FKT_ERR_INVALID_ARG;
    if (dev < 0 || dev >= kMaxDevices) return FKT_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return FKT_ERR_CUDA;
        }
        g_scratch_ptr[dev] = static_cast<float*>(p);
    }
    *out = g_scratch_ptr[dev];
    return FKT_OK;
}

}  // namespace
}  // namespace fkt

extern "C" int fkt_mvm_noalloc(fkt_plan_t plan, const float* w, float* y, int nrhs) {
    using namespace fkt;
    if (!plan || !w || !y || nrhs < 1 || nrhs > kMaxRhs || w == y) return FKT_ERR_INVALID_ARG;
    size_t f[kMvmBufs];
    mvm_buffer_floats(plan, nrhs, f);   // each part is already a multiple of 64 floats (256 bytes)
    size_t total = 0;
    for (size_t v : f) total += v;
    if (total > kScratchFloats) return FKT_ERR_SCRATCH_LIMIT;
    float* base = nullptr;
    int rc = scratch_for_plan_device(plan, &base);
    if (rc) return rc;
    float* q = base;
    MvmBuffers B{};
    B.rec = reinterpret_cast<float4*>(q);
    B.ynear = (q += f[0]);
    B.mult = (q += f[1]);
    B.part = (q += f[2]);
    B.image = reinterpret_cast<unsigned char*>(q += f[3]);
    B.yfar = (q += f[4]);
    B.nimg = (q += f[5]);
    return run_mvm(plan, B, w, y, nrhs, false);
}
