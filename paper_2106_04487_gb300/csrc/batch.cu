// Batches of independent problems (the batching form): every problem gets its own tree, lists
// and expansion (same d, p, theta), then all plans are merged into one arena -- points, nodes,
// target blocks, interaction lists, masks and s2m work items concatenated with offsets -- so that
// each stage of the product runs as one launch over the whole batch.  Per-problem kernel
// parameters are looked up per target block; near-field blocks are grouped by kernel kind and
// ordered largest-first, far-field blocks by their number of far entries.  The whole batched
// product is captured once as a CUDA graph and replayed.  A leaf-size autotuner times candidate
// plans on the device.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <map>
#include <string>
#include <numeric>
#include <vector>

#include "fkt_internal.h"

namespace fkt {
namespace {

__global__ void add_i32_kernel(int32_t* dst, const int32_t* src, int64_t n, int32_t add, int keep_negative) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t v = src[i];
    dst[i] = (keep_negative && v < 0) ? v : v + add;
}
__global__ void add_i64_kernel(int64_t* dst, const int64_t* src, int64_t n, int64_t add) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) dst[i] = src[i] + add;
}
__global__ void add_int2_kernel(int2* dst, const int2* src, int64_t n, int32_t ax, int32_t ay, int keep_negative_y) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int2 v = src[i];
    dst[i] = make_int2(v.x + ax, (keep_negative_y && v.y < 0) ? v.y : v.y + ay);
}
__global__ void add_int4_kernel(int4* dst, const int4* src, int64_t n, int32_t ax, int32_t ayz) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int4 v = src[i];
    dst[i] = make_int4(v.x + ax, v.y + ayz, v.z + ayz, v.w);
}
__global__ void fill_i32_kernel(int32_t* dst, int64_t n, int32_t v) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) dst[i] = v;
}
__global__ void fill_f32_kernel(float* dst, int64_t n, float v) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) dst[i] = v;
}

unsigned g256(int64_t n) { return (unsigned)std::max<int64_t>((n + 255) / 256, 1); }

template <typename T>
int dmalloc(T** p, int64_t n) {
    FKT_CUDA_TRY(cudaMalloc((void**)p, sizeof(T) * (size_t)std::max<int64_t>(n, 1)));
    return FKT_OK;
}

template <typename T>
int d2h(std::vector<T>& v, const T* src, int64_t n) {
    v.resize((size_t)n);
    if (n) FKT_CUDA_TRY(cudaMemcpy(v.data(), src, sizeof(T) * (size_t)n, cudaMemcpyDeviceToHost));
    return FKT_OK;
}

}  // namespace

int free_batch_arrays(fkt_plan_s* P) {
    cudaFree(P->kps);
    cudaFree(P->blk_prob);
    cudaFree(P->pt_sig);
    cudaFree(P->far_list);
    for (int32_t* l : P->kind_list) cudaFree(l);
    P->kind_list.clear();
    if (P->graph) cudaGraphExecDestroy(P->graph);
    P->graph = nullptr;
    return FKT_OK;
}

// Merge already built single-problem plans into B (a fresh plan struct).
static int merge_plans(std::vector<fkt_plan_s*>& plans, fkt_plan_s* B) {
    const int np = (int)plans.size();
    cudaStream_t st = B->stream;
    int64_t NP = 0, NN = 0, NB = 0, NF = 0, NE = 0, NM = 0, NI = 0;
    std::vector<int64_t> pt(np + 1), nd(np + 1), bk(np + 1), fe(np + 1), ne(np + 1), mk(np + 1), it(np + 1);
    for (int i = 0; i < np; ++i) {
        pt[i] = NP; nd[i] = NN; bk[i] = NB; fe[i] = NF; ne[i] = NE; mk[i] = NM; it[i] = NI;
        NP += plans[i]->N; NN += plans[i]->nnodes; NB += plans[i]->nblocks; NF += plans[i]->nfar;
        NE += plans[i]->nnear; NM += plans[i]->nmasks; NI += plans[i]->n_s2m_items;
    }
    pt[np] = NP; nd[np] = NN; bk[np] = NB; fe[np] = NF; ne[np] = NE; mk[np] = NM; it[np] = NI;
    if (NP > 0x7fffffffLL) return FKT_ERR_INVALID_ARG;
    int rc;
    if ((rc = dmalloc(&B->xs, NP)) || (rc = dmalloc(&B->perm, NP)) || (rc = dmalloc(&B->nd_begin, NN)) ||
        (rc = dmalloc(&B->nd_end, NN)) || (rc = dmalloc(&B->nd_level, NN)) || (rc = dmalloc(&B->nd_leaf, NN)) ||
        (rc = dmalloc(&B->nd_child, 2 * NN)) || (rc = dmalloc(&B->nd_centre, 4 * NN)) || (rc = dmalloc(&B->nd_rho2, NN)) ||
        (rc = dmalloc(&B->nd_cf, NN)) || (rc = dmalloc(&B->nd_scale, NN)) || (rc = dmalloc(&B->nd_used, NN)) ||
        (rc = dmalloc(&B->blk_range, NB)) || (rc = dmalloc(&B->far_off, NB + 1)) || (rc = dmalloc(&B->near_off, NB + 1)) ||
        (rc = dmalloc(&B->far_ent, NF + 1)) || (rc = dmalloc(&B->near_ent, NE + 1)) ||
        (rc = dmalloc(&B->masks, kMaskWords * (NM + 1))) || (rc = dmalloc(&B->s2m_items, NI + 1)) ||
        (rc = dmalloc(&B->s2m_item_off, NN + 1)) || (rc = dmalloc(&B->blk_prob, NB)) || (rc = dmalloc(&B->pt_sig, NP)) ||
        (rc = dmalloc(&B->kps, np)))
        return rc;
    std::vector<KernelParams> kps(np);
    for (int i = 0; i < np; ++i) {
        fkt_plan_s* Q = plans[i];
        kps[i] = Q->kp;
        const int64_t n = Q->N, nn = Q->nnodes, nb = Q->nblocks;
        FKT_CUDA_TRY(cudaMemcpyAsync(B->xs + pt[i], Q->xs, sizeof(float4) * n, cudaMemcpyDeviceToDevice, st));
        add_i32_kernel<<<g256(n), 256, 0, st>>>(B->perm + pt[i], Q->perm, n, (int32_t)pt[i], 0);
        add_i32_kernel<<<g256(nn), 256, 0, st>>>(B->nd_begin + nd[i], Q->nd_begin, nn, (int32_t)pt[i], 0);
        add_i32_kernel<<<g256(nn), 256, 0, st>>>(B->nd_end + nd[i], Q->nd_end, nn, (int32_t)pt[i], 0);
        add_i32_kernel<<<g256(2 * nn), 256, 0, st>>>(B->nd_child + 2 * nd[i], Q->nd_child, 2 * nn, (int32_t)nd[i], 1);
        FKT_CUDA_TRY(cudaMemcpyAsync(B->nd_level + nd[i], Q->nd_level, 4 * nn, cudaMemcpyDeviceToDevice, st));
        FKT_CUDA_TRY(cudaMemcpyAsync(B->nd_leaf + nd[i], Q->nd_leaf, 4 * nn, cudaMemcpyDeviceToDevice, st));
        FKT_CUDA_TRY(cudaMemcpyAsync(B->nd_centre + 4 * nd[i], Q->nd_centre, 32 * nn, cudaMemcpyDeviceToDevice, st));
        FKT_CUDA_TRY(cudaMemcpyAsync(B->nd_rho2 + nd[i], Q->nd_rho2, 8 * nn, cudaMemcpyDeviceToDevice, st));
        FKT_CUDA_TRY(cudaMemcpyAsync(B->nd_cf + nd[i], Q->nd_cf, 16 * nn, cudaMemcpyDeviceToDevice, st));
        FKT_CUDA_TRY(cudaMemcpyAsync(B->nd_scale + nd[i], Q->nd_scale, 4 * nn, cudaMemcpyDeviceToDevice, st));
        FKT_CUDA_TRY(cudaMemcpyAsync(B->nd_used + nd[i], Q->nd_used, 4 * nn, cudaMemcpyDeviceToDevice, st));
        add_int2_kernel<<<g256(nb), 256, 0, st>>>(B->blk_range + bk[i], Q->blk_range, nb, (int32_t)pt[i], (int32_t)pt[i], 0);
        add_i64_kernel<<<g256(nb), 256, 0, st>>>(B->far_off + bk[i], Q->far_off, nb, fe[i]);
        add_i64_kernel<<<g256(nb), 256, 0, st>>>(B->near_off + bk[i], Q->near_off, nb, ne[i]);
        if (Q->nfar)
            add_int2_kernel<<<g256(Q->nfar), 256, 0, st>>>(B->far_ent + fe[i], Q->far_ent, Q->nfar, (int32_t)nd[i], (int32_t)mk[i], 1);
        if (Q->nnear)
            add_int2_kernel<<<g256(Q->nnear), 256, 0, st>>>(B->near_ent + ne[i], Q->near_ent, Q->nnear, (int32_t)nd[i], (int32_t)mk[i], 1);
        if (Q->nmasks)
            FKT_CUDA_TRY(cudaMemcpyAsync(B->masks + kMaskWords * mk[i], Q->masks, 4 * kMaskWords * Q->nmasks,
                                         cudaMemcpyDeviceToDevice, st));
        if (Q->n_s2m_items)
            add_int4_kernel<<<g256(Q->n_s2m_items), 256, 0, st>>>(B->s2m_items + it[i], Q->s2m_items, Q->n_s2m_items,
                                                                  (int32_t)nd[i], (int32_t)pt[i]);
        add_i64_kernel<<<g256(nn), 256, 0, st>>>(B->s2m_item_off + nd[i], Q->s2m_item_off, nn, it[i]);
        fill_i32_kernel<<<g256(nb), 256, 0, st>>>(B->blk_prob + bk[i], nb, i);
        fill_f32_kernel<<<g256(n), 256, 0, st>>>(B->pt_sig + pt[i], n, Q->kp.sig);
        FKT_CUDA_TRY(cudaGetLastError());
    }
    const int64_t tails[3] = {NF, NE, NI};
    FKT_CUDA_TRY(cudaMemcpyAsync(B->far_off + NB, &tails[0], 8, cudaMemcpyHostToDevice, st));
    FKT_CUDA_TRY(cudaMemcpyAsync(B->near_off + NB, &tails[1], 8, cudaMemcpyHostToDevice, st));
    FKT_CUDA_TRY(cudaMemcpyAsync(B->s2m_item_off + NN, &tails[2], 8, cudaMemcpyHostToDevice, st));
    FKT_CUDA_TRY(cudaMemcpyAsync(B->kps, kps.data(), sizeof(KernelParams) * np, cudaMemcpyHostToDevice, st));
    FKT_CUDA_TRY(cudaStreamSynchronize(st));
    B->N = NP;
    B->nnodes = NN;
    B->nblocks = NB;
    B->nfar = NF;
    B->nnear = NE;
    B->nmasks = NM;
    B->n_s2m_items = NI;
    B->nprob = np;
    B->prob_off = pt;
    // work lists: near blocks grouped by kernel kind, most near sources first; far blocks by entries
    std::vector<int64_t> hnoff, hfoff;
    std::vector<int2> hnent;
    std::vector<int32_t> hb, he;
    if ((rc = d2h(hnoff, B->near_off, NB + 1)) || (rc = d2h(hfoff, B->far_off, NB + 1)) ||
        (rc = d2h(hnent, B->near_ent, NE)) || (rc = d2h(hb, B->nd_begin, NN)) || (rc = d2h(he, B->nd_end, NN)))
        return rc;
    std::vector<int64_t> near_cost(NB, 0);
    std::vector<int32_t> prob_of(NB);
    for (int i = 0; i < np; ++i)
        for (int64_t b = bk[i]; b < bk[i + 1]; ++b) prob_of[b] = i;
    for (int64_t b = 0; b < NB; ++b)
        for (int64_t e = hnoff[b]; e < hnoff[b + 1]; ++e) near_cost[b] += he[hnent[e].x] - hb[hnent[e].x];
    std::map<int, std::vector<int32_t>> by_kind;
    for (int64_t b = 0; b < NB; ++b) by_kind[kps[prob_of[b]].kind].push_back((int32_t)b);
    for (auto& kv : by_kind) {
        auto& v = kv.second;
        std::stable_sort(v.begin(), v.end(), [&](int32_t x, int32_t y) { return near_cost[x] > near_cost[y]; });
        int32_t* d = nullptr;
        if ((rc = dmalloc(&d, (int64_t)v.size()))) return rc;
        FKT_CUDA_TRY(cudaMemcpy(d, v.data(), 4 * v.size(), cudaMemcpyHostToDevice));
        B->kind_of_list.push_back(kv.first);
        B->kind_list.push_back(d);
        B->kind_list_n.push_back((int64_t)v.size());
    }
    std::vector<int32_t> fl(NB);
    std::iota(fl.begin(), fl.end(), 0);
    std::stable_sort(fl.begin(), fl.end(), [&](int32_t x, int32_t y) {
        return hfoff[x + 1] - hfoff[x] > hfoff[y + 1] - hfoff[y];
    });
    if ((rc = dmalloc(&B->far_list, NB))) return rc;
    FKT_CUDA_TRY(cudaMemcpy(B->far_list, fl.data(), 4 * NB, cudaMemcpyHostToDevice));
    // totals
    fkt_stats& s = B->stats;
    s.N = NP; s.d = B->d; s.p = B->p; s.nterms = B->nterms; s.leaf_size = B->leaf_size;
    s.nodes = NN; s.target_blocks = NB; s.far_entries = NF; s.near_entries = NE; s.masks = NM;
    for (auto* Q : plans) {
        s.depth = std::max(s.depth, Q->stats.depth);
        s.leaves += Q->stats.leaves;
        s.far_pairs += Q->stats.far_pairs;
        s.near_pairs += Q->stats.near_pairs;
        s.s2m_pairs += Q->stats.s2m_pairs;
        s.s2m_nodes += Q->stats.s2m_nodes;
    }
    return FKT_OK;
}

}  // namespace fkt

struct fkt_batch_s {
    fkt_plan_s* merged = nullptr;
    std::vector<int> leaf_of;          // leaf size chosen for each problem
    cudaStream_t user = nullptr;       // the caller's stream
    cudaStream_t own = nullptr;        // the batch's stream (graphs cannot be captured on the legacy stream)
    cudaEvent_t in = nullptr, out = nullptr;
};

namespace {

void free_plan_all(fkt_plan_s* P) { fkt_destroy(P); }

double time_mvm_ms(fkt_plan_s* P, int nrhs, int reps) {
    float *w = nullptr, *y = nullptr;
    const size_t n = (size_t)nrhs * P->N;
    if (cudaMalloc(&w, 4 * n) != cudaSuccess) return 1e30;
    if (cudaMalloc(&y, 4 * n) != cudaSuccess) { cudaFree(w); return 1e30; }
    cudaMemsetAsync(w, 0, 4 * n, P->stream);
    double best = 1e30;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    for (int r = 0; r < reps + 1; ++r) {
        cudaEventRecord(a, P->stream);
        if (fkt_mvm(P, w, y, nrhs) != FKT_OK) { best = 1e30; break; }
        cudaEventRecord(b, P->stream);
        cudaEventSynchronize(b);
        float ms = 0;
        cudaEventElapsedTime(&ms, a, b);
        if (r > 0) best = std::min(best, (double)ms);  // first run is a warm-up
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(w);
    cudaFree(y);
    return best;
}

}  // namespace

extern "C" {

int fkt_autotune_leaf(const float* points, int64_t N, int d, fkt_kernel kernel, int p, double theta, int nrhs,
                      const int* candidates, int ncand, void* cuda_stream, int* best_leaf, double* best_ms) {
    if (!points || !candidates || ncand < 1 || !best_leaf || nrhs < 1 || nrhs > fkt::kMaxRhs) return FKT_ERR_INVALID_ARG;
    double best = 1e30;
    int arg = -1;
    for (int c = 0; c < ncand; ++c) {
        fkt_plan_t P = nullptr;
        int rc = fkt_plan(points, N, d, kernel, p, candidates[c], theta, cuda_stream, &P);
        if (rc) return rc;
        const double ms = time_mvm_ms(P, nrhs, 3);
        fkt_destroy(P);
        if (ms < best) { best = ms; arg = candidates[c]; }
    }
    if (arg < 0) return FKT_ERR_CUDA;
    *best_leaf = arg;
    if (best_ms) *best_ms = best;
    return FKT_OK;
}

int fkt_batch_plan(int nprob, const fkt_problem* probs, int d, int p, int leaf_size, double theta, void* cuda_stream,
                   fkt_batch_t* out) {
    if (out) *out = nullptr;
    if (!out || !probs || nprob < 1 || (d != 3 && d != 4) || leaf_size < 0 || leaf_size > 4096) return FKT_ERR_INVALID_ARG;
    auto t0 = std::chrono::steady_clock::now();
    fkt_batch_s* Bt = new fkt_batch_s();
    Bt->leaf_of.resize(nprob);
    // leaf size: given, or autotuned once per size class (powers of 2 of N) on its largest problem
    if (leaf_size > 0) {
        for (int i = 0; i < nprob; ++i) Bt->leaf_of[i] = leaf_size;
    } else {
        std::map<int, int> rep;  // class -> problem with the largest N
        for (int i = 0; i < nprob; ++i) {
            const int cls = (int)floor(log2((double)std::max<int64_t>(probs[i].N, 1)));
            auto f = rep.find(cls);
            if (f == rep.end() || probs[f->second].N < probs[i].N) rep[cls] = i;
        }
        std::map<int, int> tuned;
        const int cand[4] = {64, 128, 256, 512};
        for (auto& kv : rep) {
            const fkt_problem& q = probs[kv.second];
            int best = 256;
            int rc = fkt_autotune_leaf(q.points, q.N, d, q.kernel, p, theta, 8, cand, 4, cuda_stream, &best, nullptr);
            if (rc) { delete Bt; return rc; }
            tuned[kv.first] = best;
        }
        for (int i = 0; i < nprob; ++i)
            Bt->leaf_of[i] = tuned[(int)floor(log2((double)std::max<int64_t>(probs[i].N, 1)))];
    }
    std::vector<fkt_plan_s*> plans(nprob, nullptr);
    int rc = FKT_OK;
    for (int i = 0; i < nprob && !rc; ++i) {
        rc = fkt_plan(probs[i].points, probs[i].N, d, probs[i].kernel, p, Bt->leaf_of[i], theta, cuda_stream, &plans[i]);
        // one expansion layout for all problems of the batch: the full one
        if (!rc) fkt::set_radial_compression(plans[i], false);
    }
    fkt_plan_s* M = nullptr;
    if (!rc) {
        M = new fkt_plan_s();
        M->d = d;
        M->p = p;
        M->theta = theta;
        M->leaf_size = leaf_size;
        M->nterms = plans[0]->nterms;
        M->tabs = plans[0]->tabs;
        M->kernel = probs[0].kernel;
        M->kp = plans[0]->kp;
        M->stream = (cudaStream_t)cuda_stream;
        M->device = plans[0]->device;
        if (fkt::create_far_stream(&M->stream2) != FKT_OK) rc = FKT_ERR_CUDA;
        for (auto& e : M->ev)
            if (!rc && cudaEventCreate(&e) != cudaSuccess) rc = FKT_ERR_CUDA;
        if (!rc && (cudaMalloc(&M->d_err, sizeof(int)) != cudaSuccess || cudaMemset(M->d_err, 0, sizeof(int)) != cudaSuccess ||
                    cudaMalloc(&M->d_wmax, sizeof(unsigned) * 32) != cudaSuccess))
            rc = FKT_ERR_OOM;
        if (!rc) rc = fkt::merge_plans(plans, M);
        if (!rc) rc = fkt::build_near_image_index(M);
    }
    for (auto* Q : plans)
        if (Q) free_plan_all(Q);
    if (rc) {
        if (M) fkt_destroy(M);
        delete Bt;
        return rc;
    }
    M->stats.plan_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    Bt->merged = M;
    Bt->user = (cudaStream_t)cuda_stream;
    if (cudaStreamCreateWithFlags(&Bt->own, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&Bt->in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&Bt->out, cudaEventDisableTiming) != cudaSuccess) {
        fkt_batch_destroy(Bt);
        return FKT_ERR_CUDA;
    }
    M->stream = Bt->own;
    *out = Bt;
    return FKT_OK;
}

static int batch_mvm_on_own_stream(fkt_batch_t batch, const float* w, float* y, int nrhs);

int fkt_batch_mvm(fkt_batch_t batch, const float* w, float* y, int nrhs) {
    if (!batch || !w || !y || w == y || nrhs < 1 || nrhs > fkt::kMaxRhs) return FKT_ERR_INVALID_ARG;
    // the batch's stream waits for the caller's work, and the caller's stream for the batch's
    FKT_CUDA_TRY(cudaEventRecord(batch->in, batch->user));
    FKT_CUDA_TRY(cudaStreamWaitEvent(batch->own, batch->in, 0));
    const int rc = batch_mvm_on_own_stream(batch, w, y, nrhs);
    FKT_CUDA_TRY(cudaEventRecord(batch->out, batch->own));
    FKT_CUDA_TRY(cudaStreamWaitEvent(batch->user, batch->out, 0));
    return rc;
}

static int batch_mvm_on_own_stream(fkt_batch_t batch, const float* w, float* y, int nrhs) {
    fkt_plan_s* P = batch->merged;
    if (P->graph && P->graph_w == w && P->graph_y == y && P->graph_nrhs == nrhs) {
        FKT_CUDA_TRY(cudaGraphLaunch(P->graph, P->stream));
        return FKT_OK;
    }
    // first product with these buffers: run it directly (sizes the work buffers and sets kernel
    // attributes), then capture the same sequence of launches as a graph for the next calls
    const bool timing = P->timing;
    P->timing = false;  // event timing synchronises the host, which a captured graph cannot do
    int rc = fkt::launch_mvm(P, w, y, nrhs);
    if (rc) { P->timing = timing; return rc; }
    if (P->graph) {
        cudaGraphExecDestroy(P->graph);
        P->graph = nullptr;
    }
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(P->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) { P->timing = timing; return FKT_ERR_CUDA; }
    rc = fkt::launch_mvm(P, w, y, nrhs);
    e = cudaStreamEndCapture(P->stream, &g);
    P->timing = timing;
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return FKT_ERR_CUDA;
    e = cudaGraphInstantiate(&P->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        P->graph = nullptr;
        return FKT_ERR_CUDA;
    }
    P->graph_w = w;
    P->graph_y = y;
    P->graph_nrhs = nrhs;
    return FKT_OK;
}

int fkt_batch_set_option(fkt_batch_t batch, const char* key, const char* value) {
    if (!batch) return FKT_ERR_INVALID_ARG;
    int rc = fkt_set_option(batch->merged, key, value);
    if (!rc && batch->merged->graph) {  // options change the launch sequence: capture again
        cudaGraphExecDestroy(batch->merged->graph);
        batch->merged->graph = nullptr;
    }
    return rc;
}

int fkt_batch_info(fkt_batch_t batch, int64_t* offsets, int32_t* leaf_sizes, fkt_stats* total) {
    if (!batch) return FKT_ERR_INVALID_ARG;
    fkt_plan_s* P = batch->merged;
    if (offsets)
        for (int i = 0; i <= P->nprob; ++i) offsets[i] = P->prob_off[i];
    if (leaf_sizes)
        for (int i = 0; i < P->nprob; ++i) leaf_sizes[i] = batch->leaf_of[i];
    if (total) *total = P->stats;
    return FKT_OK;
}

int fkt_batch_check(fkt_batch_t batch) { return batch ? fkt_check(batch->merged) : FKT_ERR_INVALID_ARG; }

int fkt_batch_autotune(fkt_batch_t batch, int nrhs, char* chosen, int len) {
    if (!batch || nrhs < 1 || nrhs > fkt::kMaxRhs || (chosen && len < 1)) return FKT_ERR_INVALID_ARG;
    fkt_plan_s* P = batch->merged;
    // kernel variants of equal accuracy (CTA shapes, per-thread work, operand paths), by axis
    struct Axis { const char* key; std::vector<const char*> values; };
    std::vector<Axis> axes;
    if (P->d == 3 && (P->far_precision == fkt::FAR_BF16 || P->far_precision == fkt::FAR_BF16X3))
        axes.push_back({"far_kernel", {"single", "held", "pairs"}});
    if (nrhs > 16) axes.push_back({"near_precision", {"fp32", "tf32x3", "f16x3"}});
    if (nrhs == 1) axes.push_back({"near_targets_per_thread", {"2", "4"}});
    std::string out;
    for (const Axis& ax : axes) {  // one axis at a time, each at the fastest of its values
        double best = 1e30;
        const char* arg = nullptr;
        for (const char* v : ax.values) {
            int rc = fkt_set_option(P, ax.key, v);
            if (rc) return rc;
            const double ms = time_mvm_ms(P, nrhs, 3);
            if (ms < best) { best = ms; arg = v; }
        }
        if (!arg) return FKT_ERR_CUDA;
        int rc = fkt_set_option(P, ax.key, arg);
        if (rc) return rc;
        out += std::string(out.empty() ? "" : ";") + ax.key + "=" + arg;
    }
    if (P->graph) {  // options change the launch sequence: capture again on the next product
        cudaGraphExecDestroy(P->graph);
        P->graph = nullptr;
    }
    if (chosen) {
        const size_t n = std::min(out.size(), (size_t)len - 1);
        memcpy(chosen, out.data(), n);
        chosen[n] = 0;
    }
    return FKT_OK;
}

void fkt_batch_destroy(fkt_batch_t batch) {
    if (!batch) return;
    if (batch->own) cudaStreamSynchronize(batch->own);
    fkt_destroy(batch->merged);
    if (batch->in) cudaEventDestroy(batch->in);
    if (batch->out) cudaEventDestroy(batch->out);
    if (batch->own) cudaStreamDestroy(batch->own);
    delete batch;
}

}  // extern "C"
