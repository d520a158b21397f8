// fkt_mvm_noalloc: the FKT product with its per-call work buffers carved out of one
// statically declared device array instead of cudaMalloc'd plan buffers (for callers that
// cannot allocate; see include/fkt.h).  The kernels and their order are those of fkt_mvm.
#include <mutex>

#include "far_dispatch.cuh"
#include "mvm_kernels.cuh"

namespace fkt {

int mvm_launch_s2m(int d, int p, int nrb, const FarLaunch& L);
int mvm_launch_far(int d, int p, int nrb, const FarLaunch& L);
void mvm_launch_near(int d, int nrb, int kind, unsigned grid, cudaStream_t st, const MvmArgs& a,
                     const KernelParams& kp);
MvmArgs mvm_base_args(fkt_plan_s* P);

namespace {

constexpr size_t kScratchFloats = FKT_NOALLOC_SCRATCH_BYTES / sizeof(float);

// The scratch itself.  In host code this name is only a stand-in for the device array:
// kernels must be given the address that cudaGetSymbolAddress returns for the current device.
static __device__ __align__(256) float g_noalloc_scratch[kScratchFloats];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
float* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch on the current device, looked up once per device.
int scratch_for_current_device(float** out) {
    int dev = 0;
    FKT_CUDA_TRY(cudaGetDevice(&dev));
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

size_t round256(size_t nfloats) { return (nfloats + 63) / 64 * 64; }

}  // namespace
}  // namespace fkt

extern "C" int fkt_mvm_noalloc(fkt_plan_t plan, const float* w, float* y, int nrhs) {
    using namespace fkt;
    if (!plan || !w || !y || nrhs < 1 || nrhs > kMaxRhs || w == y) return FKT_ERR_INVALID_ARG;
    fkt_plan_s* P = plan;
    const int nrb = nrhs == 1 ? 1 : 8;
    const int groups = (nrhs + nrb - 1) / nrb;
    const size_t cap = (size_t)nrb * groups;
    const size_t N = (size_t)P->N, NT = (size_t)P->nterms;
    const size_t items = P->n_s2m_items > 0 ? (size_t)P->n_s2m_items : 1;
    const size_t nodes = P->nnodes > 0 ? (size_t)P->nnodes : 1;
    const size_t n_ws = round256(cap * N), n_yn = round256(cap * N);
    const size_t n_mult = round256(cap * NT * nodes), n_part = round256(cap * NT * items);
    if (n_ws + n_yn + n_mult + n_part > kScratchFloats) return FKT_ERR_SCRATCH_LIMIT;
    float* base = nullptr;
    int rc = scratch_for_current_device(&base);
    if (rc) return rc;
    float* ws = base;
    float* ynear = ws + n_ws;
    float* mult = ynear + n_yn;
    float* part = mult + n_mult;
    cudaStream_t st = P->stream, st2 = P->stream2;
    for (int g = 0; g < groups; ++g) {
        const int nr = nrhs - g * nrb < nrb ? nrhs - g * nrb : nrb;
        MvmArgs a = mvm_base_args(P);
        a.ws = ws + (size_t)g * nrb * N;
        a.ynear = ynear + (size_t)g * nrb * N;
        a.mult = mult + (size_t)g * nrb * NT * nodes;
        a.part = part + (size_t)g * nrb * NT * items;
        a.y = y + (size_t)g * nrb * N;
        a.nr = nr;
        const float* wg = w + (size_t)g * nrb * N;
        const unsigned pg = (unsigned)((N + 255) / 256);
        if (nrb == 1) permute_kernel<1><<<pg, 256, 0, st>>>((int64_t)N, P->perm, wg, nr, ws + (size_t)g * nrb * N);
        else permute_kernel<8><<<pg, 256, 0, st>>>((int64_t)N, P->perm, wg, nr, ws + (size_t)g * nrb * N);
        FKT_CUDA_TRY(cudaGetLastError());
        FKT_CUDA_TRY(cudaEventRecord(P->ev[1], st));
        FKT_CUDA_TRY(cudaStreamWaitEvent(st2, P->ev[1], 0));
        FarLaunch L{&a, &P->kp, &P->tabs, P->nblocks, P->n_s2m_items, P->nnodes, st, st2};
        rc = mvm_launch_s2m(P->d, P->p, nrb, L);
        if (rc) return rc;
        FKT_CUDA_TRY(cudaEventRecord(P->ev[4], st2));
        mvm_launch_near(P->d, nrb, P->kernel.kind, (unsigned)P->nblocks, st, a, P->kp);
        FKT_CUDA_TRY(cudaGetLastError());
        FKT_CUDA_TRY(cudaStreamWaitEvent(st, P->ev[4], 0));
        rc = mvm_launch_far(P->d, P->p, nrb, L);
        if (rc) return rc;
    }
    return FKT_OK;
}
