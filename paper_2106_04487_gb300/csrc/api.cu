// C ABI entry points (include/fkt.h).
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <chrono>
#include <new>
#include <vector>

#include "fkt_internal.h"

namespace {

bool is_device_pointer(const void* p) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

void free_plan(fkt_plan_s* P) {
    if (!P) return;
    void* bufs[] = {P->xs, P->perm, P->codes, P->nd_begin, P->nd_end, P->nd_level, P->nd_leaf, P->nd_child,
                    P->nd_centre, P->nd_rho2, P->nd_cf, P->nd_scale, P->nd_used, P->blk_range, P->far_off,
                    P->near_off, P->far_ent, P->near_ent, P->masks, P->s2m_items, P->s2m_node_items,
                    P->s2m_item_off, P->rec, P->ynear, P->yfar, P->mult, P->s2m_part, P->tc_image, P->hbuf_w, P->hbuf_y,
                    P->d_err, P->d_wmax, P->dense_off, P->dense_ent, P->nd_img, P->nimg};
    for (void* b : bufs)
        if (b) cudaFree(b);
    fkt::free_learn(P);
    fkt::free_solve(P);
    fkt::free_batch_arrays(P);
    fkt::free_shard(P);
    for (auto& e : P->ev)
        if (e) cudaEventDestroy(e);
    if (P->stream2) cudaStreamDestroy(P->stream2);
    delete P;
}

int valid_kernel(const fkt_kernel& k) {
    if (k.kind < FKT_GAUSSIAN || k.kind > FKT_LAPLACE) return 0;
    if (!(k.lengthscale > 0.0) || !isfinite(k.lengthscale)) return 0;
    if (!isfinite(k.scale)) return 0;
    if (k.kind == FKT_RATQUAD && (!(k.alpha > 0.0) || !isfinite(k.alpha))) return 0;
    return 1;
}

}  // namespace

namespace fkt {

// The radial compression that is exact for the kernel: the Laplace kernel in d = 3, whose degree-k
// radial parts have rank 1 (Table 3), keeps only its j = k terms.
bool radial_compression_exact(int d, int kind) { return d == 3 && kind == FKT_LAPLACE; }

// Switch the expansion layout and size; the per-call work buffers depend on it, so they are freed
// and regrown by the next product.
void set_radial_compression(fkt_plan_s* P, bool on) {
    long long nt = 1;  // binom(p + d, d): every radial term
    for (int i = 1; i <= P->d; ++i) nt = nt * (P->p + i) / i;
    const int want = on ? (P->p + 1) * (P->p + 1) : (int)nt;  // j = k only: sum_k (2k + 1)
    if (P->diag == on && P->nterms == want) return;
    P->diag = on;
    P->nterms = want;
    P->stats.nterms = want;
    for (void** b : {(void**)&P->rec, (void**)&P->ynear, (void**)&P->yfar, (void**)&P->mult, (void**)&P->s2m_part,
                     (void**)&P->tc_image}) {
        cudaFree(*b);
        *b = nullptr;
    }
    P->cap_rhs = 0;
    P->cap_tc = 0;
}

}  // namespace fkt

extern "C" {

const char* fkt_error_string(int status) {
    switch (status) {
    case FKT_OK: return "ok";
    case FKT_ERR_INVALID_ARG: return "invalid argument";
    case FKT_ERR_CUDA: return "CUDA error";
    case FKT_ERR_OOM: return "out of device memory";
    case FKT_ERR_NOT_CONVERGED: return "solver did not converge";
    case FKT_ERR_TIMEOUT: return "device-side wait timed out";
    case FKT_ERR_UNSUPPORTED: return "unsupported request";
    case FKT_ERR_INTERNAL: return "internal consistency check failed";
    case FKT_ERR_SCRATCH_LIMIT: return "request exceeds the fixed scratch of fkt_mvm_noalloc";
    default: return "unknown status";
    }
}

int fkt_plan(const float* points, int64_t N, int d, fkt_kernel kernel, int p, int leaf_size, double theta,
             void* cuda_stream, fkt_plan_t* out) {
    if (out) *out = nullptr;
    if (!out || !points || N < 1 || N > 0x7fffffffLL || d < 2 || d > 4 || !valid_kernel(kernel)) return FKT_ERR_INVALID_ARG;
    if (p < 0 || p > (d <= 3 ? fkt::kMaxP3 : fkt::kMaxP4)) return FKT_ERR_INVALID_ARG;
    if (leaf_size < 1 || leaf_size > 4096 || !(theta > 0.0 && theta < 1.0)) return FKT_ERR_INVALID_ARG;
    if (!is_device_pointer(points)) return FKT_ERR_INVALID_ARG;
    auto t0 = std::chrono::steady_clock::now();
    fkt_plan_s* P = new (std::nothrow) fkt_plan_s();
    if (!P) return FKT_ERR_OOM;
    P->N = N;
    P->d = d;
    P->p = p;
    P->leaf_size = leaf_size;
    P->theta = theta;
    P->kernel = kernel;
    P->kp = fkt::make_kernel_params(kernel);
    P->stream = (cudaStream_t)cuda_stream;
    if (cudaGetDevice(&P->device) != cudaSuccess) { free_plan(P); return FKT_ERR_CUDA; }
    int rc = fkt::build_far_tables(d, p, &P->tabs);
    if (rc) { free_plan(P); return rc; }
    fkt::set_radial_compression(P, fkt::radial_compression_exact(d, kernel.kind));
    if (fkt::create_far_stream(&P->stream2) != FKT_OK) { free_plan(P); return FKT_ERR_CUDA; }
    for (auto& e : P->ev)
        if (cudaEventCreate(&e) != cudaSuccess) { free_plan(P); return FKT_ERR_CUDA; }
    if (cudaMalloc(&P->d_err, sizeof(int)) != cudaSuccess || cudaMemsetAsync(P->d_err, 0, sizeof(int), P->stream) != cudaSuccess ||
        cudaMalloc(&P->d_wmax, sizeof(unsigned) * 32) != cudaSuccess) {
        free_plan(P);
        return FKT_ERR_OOM;
    }
    rc = fkt::build_tree(P, points);
    if (!rc) rc = fkt::build_lists(P);
    if (!rc) rc = fkt::build_near_image_index(P);
    if (!rc && cudaStreamSynchronize(P->stream) != cudaSuccess) rc = FKT_ERR_CUDA;
    if (rc) { free_plan(P); return rc; }
    fkt_stats& s = P->stats;
    s.N = N;
    s.d = d;
    s.p = p;
    s.nterms = P->nterms;
    s.leaf_size = leaf_size;
    s.depth = P->depth;
    s.nodes = P->nnodes;
    s.leaves = P->nleaves;
    s.target_blocks = P->nblocks;
    s.far_entries = P->nfar;
    s.near_entries = P->nnear;
    s.masks = P->nmasks;
    s.plan_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    *out = P;
    return FKT_OK;
}

int fkt_mvm(fkt_plan_t plan, const float* w, float* y, int nrhs) {
    if (!plan || !w || !y || nrhs < 1 || nrhs > fkt::kMaxRhs || w == y) return FKT_ERR_INVALID_ARG;
    return fkt::launch_mvm(plan, w, y, nrhs);
}

int fkt_mvm_host(fkt_plan_t plan, const float* w_host, float* y_host, int nrhs) {
    if (!plan || !w_host || !y_host || nrhs < 1 || nrhs > fkt::kMaxRhs) return FKT_ERR_INVALID_ARG;
    fkt_plan_s* P = plan;
    const size_t bytes = sizeof(float) * (size_t)nrhs * P->N;
    // device staging buffers, sized for the largest nrhs seen so far
    if (P->hbuf_cap < nrhs) {
        cudaFree(P->hbuf_w);
        cudaFree(P->hbuf_y);
        P->hbuf_w = P->hbuf_y = nullptr;
        P->hbuf_cap = 0;
        FKT_CUDA_TRY(cudaMalloc(&P->hbuf_w, bytes));
        FKT_CUDA_TRY(cudaMalloc(&P->hbuf_y, bytes));
        P->hbuf_cap = nrhs;
    }
    FKT_CUDA_TRY(cudaMemcpyAsync(P->hbuf_w, w_host, bytes, cudaMemcpyHostToDevice, P->stream));
    int rc = fkt::launch_mvm(P, P->hbuf_w, P->hbuf_y, nrhs);
    if (rc) return rc;
    FKT_CUDA_TRY(cudaMemcpyAsync(y_host, P->hbuf_y, bytes, cudaMemcpyDeviceToHost, P->stream));
    FKT_CUDA_TRY(cudaStreamSynchronize(P->stream));
    return FKT_OK;
}

int fkt_dense_mvm(fkt_plan_t plan, const float* w, float* y, int nrhs) {
    if (!plan || !w || !y || nrhs < 1 || nrhs > fkt::kMaxRhs || w == y) return FKT_ERR_INVALID_ARG;
    if (plan->nprob) return FKT_ERR_UNSUPPORTED;
    return fkt::launch_dense(plan, w, y, nrhs);
}

int fkt_precond_setup(fkt_plan_t plan, double sigma2) {
    if (!plan || !(sigma2 > 0.0) || !isfinite(sigma2)) return FKT_ERR_INVALID_ARG;
    return fkt::precond_setup(plan, sigma2);
}

int fkt_precond_apply(fkt_plan_t plan, const float* r, float* z, int nrhs) {
    if (!plan || !r || !z || r == z || nrhs < 1 || nrhs > fkt::kMaxRhs) return FKT_ERR_INVALID_ARG;
    return fkt::precond_apply(plan, r, nullptr, z, nrhs);
}

int fkt_solve(fkt_plan_t plan, double sigma2, const float* b, float* x, int nrhs, double tol, int max_iter,
              fkt_solve_info* info) {
    if (info) memset(info, 0, sizeof(*info));
    if (!plan || !b || !x || b == x || nrhs < 1 || nrhs > fkt::kMaxRhs || !(sigma2 > 0.0) || !isfinite(sigma2) ||
        !(tol > 0.0 && tol < 1.0) || max_iter < 1)
        return FKT_ERR_INVALID_ARG;
    return fkt::solve(plan, sigma2, b, x, nullptr, nrhs, tol, max_iter, info);
}

int fkt_solve_f64(fkt_plan_t plan, double sigma2, const float* b, double* x, int nrhs, double tol, int max_iter,
                  fkt_solve_info* info) {
    if (info) memset(info, 0, sizeof(*info));
    if (!plan || !b || !x || (const void*)b == (const void*)x || nrhs < 1 || nrhs > fkt::kMaxRhs ||
        !(sigma2 > 0.0) || !isfinite(sigma2) || !(tol > 0.0 && tol < 1.0) || max_iter < 1)
        return FKT_ERR_INVALID_ARG;
    return fkt::solve(plan, sigma2, b, nullptr, x, nrhs, tol, max_iter, info);
}

int fkt_precond_learn(fkt_plan_t plan, double sigma2, const fkt_learn_opts* opts, fkt_learn_info* info) {
    if (info) memset(info, 0, sizeof(*info));
    if (!plan || !(sigma2 > 0.0) || !isfinite(sigma2)) return FKT_ERR_INVALID_ARG;
    return fkt::precond_learn(plan, sigma2, opts, info);
}

int fkt_learn_params(fkt_plan_t plan, float* params, int* nparams) {
    if (!plan || !nparams) return FKT_ERR_INVALID_ARG;
    return fkt::learn_params(plan, params, nparams);
}

int fkt_learn_eval(fkt_plan_t plan, const float* params, double* loss, float* grad) {
    if (!plan || !params) return FKT_ERR_INVALID_ARG;
    return fkt::learn_eval(plan, params, loss, grad);
}

int fkt_learn_teacher(fkt_plan_t plan, int64_t* blocks, float* D) {
    if (!plan) return FKT_ERR_INVALID_ARG;
    return fkt::learn_teacher(plan, blocks, D);
}

int fkt_set_option(fkt_plan_t plan, const char* key, const char* value) {
    if (!plan || !key || !value) return FKT_ERR_INVALID_ARG;
    if (!strcmp(key, "timing")) {
        if (!strcmp(value, "0")) plan->timing = false;
        else if (!strcmp(value, "1")) plan->timing = true;
        else return FKT_ERR_INVALID_ARG;
        return FKT_OK;
    }
    if (!strcmp(key, "preconditioner")) {
        if (!strcmp(value, "none")) plan->pc_mode = 0;
        else if (!strcmp(value, "block_jacobi")) plan->pc_mode = 1;
        else if (!strcmp(value, "learned")) plan->pc_mode = 2;
        else return FKT_ERR_INVALID_ARG;
        return FKT_OK;
    }
    if (!strcmp(key, "coarse_rank") || !strcmp(key, "coarse_seed")) {
        char* end = nullptr;
        const unsigned long long v = strtoull(value, &end, 10);
        if (!*value || *end || value[0] == '-') return FKT_ERR_INVALID_ARG;
        if (key[7] == 'r') {
            if (v > 256) return FKT_ERR_INVALID_ARG;
            plan->coarse_rank = (int)v;
        } else {
            plan->coarse_seed = (uint64_t)v;
        }
        return FKT_OK;
    }
    if (!strcmp(key, "radial_compression")) {
        if (!strcmp(value, "off")) fkt::set_radial_compression(plan, false);
        else if (!strcmp(value, "auto")) fkt::set_radial_compression(plan, fkt::radial_compression_exact(plan->d, plan->kernel.kind) && !plan->nprob);
        else return FKT_ERR_INVALID_ARG;
        return FKT_OK;
    }
    if (!strcmp(key, "far_kernel")) {
        if (!strcmp(value, "pairs")) plan->far_kernel = 0;
        else if (!strcmp(value, "single")) plan->far_kernel = 1;
        else if (!strcmp(value, "held")) plan->far_kernel = 2;
        else return FKT_ERR_INVALID_ARG;
        return FKT_OK;
    }
    if (!strcmp(key, "wait_limit_cycles")) {
        if (!strcmp(value, "default")) {
            plan->wait_cycles = fkt::kWaitCycles;
            return FKT_OK;
        }
        char* end = nullptr;
        const long long v = strtoll(value, &end, 10);
        if (!end || *end || end == value || v < 0 || v > fkt::kWaitCycles) return FKT_ERR_INVALID_ARG;
        plan->wait_cycles = v;
        return FKT_OK;
    }
    if (!strcmp(key, "near_targets_per_thread")) {
        if (!strcmp(value, "2")) plan->near_tpt = 2;
        else if (!strcmp(value, "4")) plan->near_tpt = 4;
        else return FKT_ERR_INVALID_ARG;
        return FKT_OK;
    }
    if (!strcmp(key, "near_precision")) {
        if (!strcmp(value, "fp32")) plan->near_precision = fkt::NEAR_FP32;
        else if (!strcmp(value, "tf32x3")) plan->near_precision = fkt::NEAR_TF32X3;
        else if (!strcmp(value, "f16x3")) plan->near_precision = fkt::NEAR_F16X3;
        else return FKT_ERR_INVALID_ARG;
        return FKT_OK;
    }
    if (!strcmp(key, "far_precision")) {
        if (!strcmp(value, "fp32")) plan->far_precision = fkt::FAR_FP32;
        else if (!strcmp(value, "tf32")) plan->far_precision = fkt::FAR_TF32;
        else if (!strcmp(value, "bf16")) plan->far_precision = fkt::FAR_BF16;
        else if (!strcmp(value, "bf16x3")) plan->far_precision = fkt::FAR_BF16X3;
        else return FKT_ERR_INVALID_ARG;
        return FKT_OK;
    }
    return FKT_ERR_INVALID_ARG;
}

int fkt_plan_stats(fkt_plan_t plan, fkt_stats* out) {
    if (!plan || !out) return FKT_ERR_INVALID_ARG;
    *out = plan->stats;
    return FKT_OK;
}

int fkt_plan_tree(fkt_plan_t plan, int64_t* perm, int64_t* begin, int64_t* end, int32_t* level, int32_t* leaf,
                  int64_t* child, double* centre, double* rho2) {
    if (!plan) return FKT_ERR_INVALID_ARG;
    fkt_plan_s* P = plan;
    FKT_CUDA_TRY(cudaStreamSynchronize(P->stream));
    const int64_t nn = P->nnodes, N = P->N;
    std::vector<int32_t> t32;
    if (perm) {
        t32.resize(N);
        FKT_CUDA_TRY(cudaMemcpy(t32.data(), P->perm, 4 * N, cudaMemcpyDeviceToHost));
        for (int64_t i = 0; i < N; ++i) perm[i] = t32[i];
    }
    auto cp64 = [&](int64_t* dst, const int32_t* src, int64_t n) -> int {
        t32.resize(n);
        FKT_CUDA_TRY(cudaMemcpy(t32.data(), src, 4 * n, cudaMemcpyDeviceToHost));
        for (int64_t i = 0; i < n; ++i) dst[i] = t32[i];
        return FKT_OK;
    };
    int rc;
    if (begin && (rc = cp64(begin, P->nd_begin, nn))) return rc;
    if (end && (rc = cp64(end, P->nd_end, nn))) return rc;
    if (child && (rc = cp64(child, P->nd_child, 2 * nn))) return rc;
    if (level) FKT_CUDA_TRY(cudaMemcpy(level, P->nd_level, 4 * nn, cudaMemcpyDeviceToHost));
    if (leaf) FKT_CUDA_TRY(cudaMemcpy(leaf, P->nd_leaf, 4 * nn, cudaMemcpyDeviceToHost));
    if (rho2) FKT_CUDA_TRY(cudaMemcpy(rho2, P->nd_rho2, 8 * nn, cudaMemcpyDeviceToHost));
    if (centre) {
        std::vector<double> c4(4 * nn);
        FKT_CUDA_TRY(cudaMemcpy(c4.data(), P->nd_centre, 8 * 4 * nn, cudaMemcpyDeviceToHost));
        for (int64_t i = 0; i < nn; ++i)
            for (int a = 0; a < P->d; ++a) centre[i * P->d + a] = c4[4 * i + a];
    }
    return FKT_OK;
}

int fkt_plan_lists(fkt_plan_t plan, int64_t* block_range, int64_t* far_off, int32_t* far_node, int32_t* far_mask,
                   int64_t* near_off, int32_t* near_leaf, int32_t* near_mask, uint32_t* masks) {
    if (!plan) return FKT_ERR_INVALID_ARG;
    fkt_plan_s* P = plan;
    FKT_CUDA_TRY(cudaStreamSynchronize(P->stream));
    const int64_t nb = P->nblocks;
    if (block_range) {
        std::vector<int2> v(nb);
        FKT_CUDA_TRY(cudaMemcpy(v.data(), P->blk_range, sizeof(int2) * nb, cudaMemcpyDeviceToHost));
        for (int64_t i = 0; i < nb; ++i) { block_range[2 * i] = v[i].x; block_range[2 * i + 1] = v[i].y; }
    }
    if (far_off) FKT_CUDA_TRY(cudaMemcpy(far_off, P->far_off, 8 * (nb + 1), cudaMemcpyDeviceToHost));
    if (near_off) FKT_CUDA_TRY(cudaMemcpy(near_off, P->near_off, 8 * (nb + 1), cudaMemcpyDeviceToHost));
    auto split = [&](const int2* src, int64_t n, int32_t* a, int32_t* b) -> int {
        std::vector<int2> v(n);
        if (n) FKT_CUDA_TRY(cudaMemcpy(v.data(), src, sizeof(int2) * n, cudaMemcpyDeviceToHost));
        for (int64_t i = 0; i < n; ++i) {
            if (a) a[i] = v[i].x;
            if (b) b[i] = v[i].y;
        }
        return FKT_OK;
    };
    int rc;
    if ((far_node || far_mask) && (rc = split(P->far_ent, P->nfar, far_node, far_mask))) return rc;
    if ((near_leaf || near_mask) && (rc = split(P->near_ent, P->nnear, near_leaf, near_mask))) return rc;
    if (masks && P->nmasks)
        FKT_CUDA_TRY(cudaMemcpy(masks, P->masks, sizeof(uint32_t) * fkt::kMaskWords * P->nmasks, cudaMemcpyDeviceToHost));
    return FKT_OK;
}

int fkt_shard_partition(int64_t nblocks, const double* work, int nranks, int64_t* bounds) {
    if (nranks < 1 || nranks > 4096) return FKT_ERR_INVALID_ARG;
    return fkt::shard_partition(nblocks, work, nranks, bounds);
}

int fkt_shard_set(fkt_plan_t plan, int nranks, int rank) {
    if (!plan || nranks < 1 || nranks > 4096 || rank < 0 || rank >= nranks) return FKT_ERR_INVALID_ARG;
    return fkt::shard_set(plan, nranks, rank);
}

int fkt_shard_block_work(fkt_plan_t plan, double* work) {
    if (!plan || !work) return FKT_ERR_INVALID_ARG;
    if (plan->nprob) return FKT_ERR_UNSUPPORTED;
    std::vector<double> w;
    int rc = fkt::shard_block_work(plan, w);
    if (rc) return rc;
    std::copy(w.begin(), w.end(), work);
    return FKT_OK;
}

int fkt_shard_info(fkt_plan_t plan, int nrhs, int64_t* block_lo, int64_t* block_hi, int64_t* target_lo,
                   int64_t* target_hi, int64_t* mult_floats) {
    if (!plan || plan->sh_nranks == 0 || nrhs < 1 || nrhs > 32) return FKT_ERR_INVALID_ARG;
    if (block_lo) *block_lo = plan->sh_b0;
    if (block_hi) *block_hi = plan->sh_b1;
    if (target_lo) *target_lo = plan->sh_t0;
    if (target_hi) *target_hi = plan->sh_t1;
    if (mult_floats) *mult_floats = (int64_t)fkt::shard_mult_floats(plan, nrhs);
    return FKT_OK;
}

int fkt_mvm_shard_begin(fkt_plan_t plan, const float* w, float* mult, int nrhs) {
    if (!plan || !w || !mult || plan->sh_nranks == 0 || nrhs < 1 || nrhs > 32) return FKT_ERR_INVALID_ARG;
    return fkt::shard_begin(plan, w, mult, nrhs);
}

int fkt_mvm_shard_end(fkt_plan_t plan, const float* mult, float* y, int nrhs) {
    if (!plan || !mult || !y || plan->sh_nranks == 0 || nrhs < 1 || nrhs > 32) return FKT_ERR_INVALID_ARG;
    return fkt::shard_end(plan, mult, y, nrhs);
}

int fkt_check(fkt_plan_t plan) {
    if (!plan) return FKT_ERR_INVALID_ARG;
    FKT_CUDA_TRY(cudaStreamSynchronize(plan->stream));
    FKT_CUDA_TRY(cudaStreamSynchronize(plan->stream2));
    int h = 0;
    FKT_CUDA_TRY(cudaMemcpy(&h, plan->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (h) {
        FKT_CUDA_TRY(cudaMemset(plan->d_err, 0, sizeof(int)));
        return FKT_ERR_TIMEOUT;
    }
    return FKT_OK;
}

void fkt_destroy(fkt_plan_t plan) {
    if (!plan) return;
    cudaStreamSynchronize(plan->stream);
    cudaStreamSynchronize(plan->stream2);
    free_plan(plan);
}

}  // extern "C"
