// Host orchestration of one FKT matrix-vector product (Algorithm 1) on the GPU:
//   permute w -> [s2m -> s2m_reduce] (second stream)  ||  near field (plan stream)
//   -> far field + combine + scatter to the caller's order.
// Right-hand sides are processed in passes of up to 32: one permute and one near-field launch
// per pass (the kernel value of a pair serves every right-hand side of the pass), s2m and the
// float32 far field per group of 8 (or 1 for a single right-hand side), the tensor-core far
// field once per pass.
#include <climits>
#include <vector>
#include <algorithm>

#include "mvm_kernels.cuh"
#include "far_dispatch.cuh"
#include "far_tc.cuh"

namespace fkt {

#define FKT_DECL_RANGE(D, A, B)                                         \
    int launch_s2m_d##D##_p##A##_##B(int p, int nrb, const FarLaunch& L); \
    int launch_far_d##D##_p##A##_##B(int p, int nrb, const FarLaunch& L);
FKT_DECL_RANGE(3, 0, 4)
FKT_DECL_RANGE(3, 5, 6)
FKT_DECL_RANGE(3, 7, 8)
FKT_DECL_RANGE(3, 9, 10)
FKT_DECL_RANGE(4, 0, 4)
FKT_DECL_RANGE(4, 5, 6)
FKT_DECL_RANGE(4, 7, 8)
#undef FKT_DECL_RANGE
int launch_s2m_d2_p0_10(int p, int nrb, const FarLaunch& L);
int launch_far_d2_p0_10(int p, int nrb, const FarLaunch& L);
int launch_s2m_diag_p0_5(int p, int nrb, const FarLaunch& L);
int launch_far_diag_p0_5(int p, int nrb, const FarLaunch& L);
int launch_s2m_diag_p6_10(int p, int nrb, const FarLaunch& L);
int launch_far_diag_p6_10(int p, int nrb, const FarLaunch& L);
int launch_tc_diag_p0_6(int p, int prec, bool far, const TcLaunch& L);
int launch_tc_diag_p7_10(int p, int prec, bool far, const TcLaunch& L);

void launch_near_d3(int nw, int tpt, int kind, unsigned grid, cudaStream_t st, const MvmArgs& a, const KernelParams& kp);
void launch_near_d4(int nw, int tpt, int kind, unsigned grid, cudaStream_t st, const MvmArgs& a, const KernelParams& kp);
void launch_near_image(int64_t nnodes, const int32_t* nd_leaf, const int32_t* nd_begin, const int32_t* nd_end,
                       const int32_t* nd_img, const float4* rec, int rec_f4, float* img, cudaStream_t st);
void launch_near_tc_d3(int kind, unsigned grid, cudaStream_t st, const MvmArgs& a, const KernelParams& kp);
void launch_near_tc_d4(int kind, unsigned grid, cudaStream_t st, const MvmArgs& a, const KernelParams& kp);
void launch_near_tc2_d3(int kind, unsigned grid, cudaStream_t st, const MvmArgs& a, const KernelParams& kp, unsigned* wmax);
void launch_near_tc2_d4(int kind, unsigned grid, cudaStream_t st, const MvmArgs& a, const KernelParams& kp, unsigned* wmax);

int launch_tc_d3_p0_6(int p, int prec, bool far, const TcLaunch& L);
int launch_tc_d3_p7_10(int p, int prec, bool far, const TcLaunch& L);
int launch_tc_d4_p0_5(int p, int prec, bool far, const TcLaunch& L);
int launch_tc_d4_p6_8(int p, int prec, bool far, const TcLaunch& L);

// d: the layout code (2, 3, 4, or kDiag3 for the compressed d = 3 layout).  The tensor-core
// far field is built for d = 3 and 4.
static int launch_tc_any(int d, int p, int prec, bool far, const TcLaunch& L) {
    if (d == 2) return FKT_ERR_UNSUPPORTED;
    if (d == kDiag3) return p <= 6 ? launch_tc_diag_p0_6(p, prec, far, L) : launch_tc_diag_p7_10(p, prec, far, L);
    if (d == 3) return p <= 6 ? launch_tc_d3_p0_6(p, prec, far, L) : launch_tc_d3_p7_10(p, prec, far, L);
    return p <= 5 ? launch_tc_d4_p0_5(p, prec, far, L) : launch_tc_d4_p6_8(p, prec, far, L);
}

// Layout code of the plan's expansion (fkt_kernels.cuh): the compressed d = 3 layout when the
// radial compression is on, otherwise the dimension.
static int layout_code(const fkt_plan_s* P) { return P->diag ? kDiag3 : P->d; }

static int tc_prec_of(int far_precision) {
    return far_precision == FAR_BF16 ? TC_BF16 : far_precision == FAR_BF16X3 ? TC_BF16X3 : TC_TF32;
}

static int launch_s2m_any(int d, int p, int nrb, const FarLaunch& L) {
    if (d == 2) return launch_s2m_d2_p0_10(p, nrb, L);
    if (d == kDiag3) return p <= 5 ? launch_s2m_diag_p0_5(p, nrb, L) : launch_s2m_diag_p6_10(p, nrb, L);
    if (d == 3) {
        if (p <= 4) return launch_s2m_d3_p0_4(p, nrb, L);
        if (p <= 6) return launch_s2m_d3_p5_6(p, nrb, L);
        if (p <= 8) return launch_s2m_d3_p7_8(p, nrb, L);
        return launch_s2m_d3_p9_10(p, nrb, L);
    }
    if (p <= 4) return launch_s2m_d4_p0_4(p, nrb, L);
    if (p <= 6) return launch_s2m_d4_p5_6(p, nrb, L);
    return launch_s2m_d4_p7_8(p, nrb, L);
}

static int launch_far_any(int d, int p, int nrb, const FarLaunch& L) {
    if (d == 2) return launch_far_d2_p0_10(p, nrb, L);
    if (d == kDiag3) return p <= 5 ? launch_far_diag_p0_5(p, nrb, L) : launch_far_diag_p6_10(p, nrb, L);
    if (d == 3) {
        if (p <= 4) return launch_far_d3_p0_4(p, nrb, L);
        if (p <= 6) return launch_far_d3_p5_6(p, nrb, L);
        if (p <= 8) return launch_far_d3_p7_8(p, nrb, L);
        return launch_far_d3_p9_10(p, nrb, L);
    }
    if (p <= 4) return launch_far_d4_p0_4(p, nrb, L);
    if (p <= 6) return launch_far_d4_p5_6(p, nrb, L);
    return launch_far_d4_p7_8(p, nrb, L);
}

namespace {

// Near field launch: nw right-hand sides per pass (1, 8, 16, 32); targets per thread tpt = 2 or 4
// (4 only for one right-hand side); tc: the 32-wide pass on the tensor cores -- tc = 1 TF32 hi/lo
// operands, tc = 2 FP16 hi/lo operands with double buffering (wmax: 32 words of device scratch for
// the weights' per-right-hand-side scale), which the 1/r kernel leaves for TF32 (its values are
// unbounded).
// d = 2 runs the d = 3 near kernels: its points carry zero third and fourth coordinates.
void launch_near(int d, int nw, int tpt, int tc, int kind, unsigned grid, cudaStream_t st, const MvmArgs& a,
                 const KernelParams& kp, unsigned* wmax) {
    if (d == 2) d = 3;
    if (tc && nw == 32) {
        if (tc == 2 && kind != FKT_LAPLACE && wmax) {
            if (d == 3) launch_near_tc2_d3(kind, grid, st, a, kp, wmax);
            else launch_near_tc2_d4(kind, grid, st, a, kp, wmax);
        } else if (d == 3) {
            launch_near_tc_d3(kind, grid, st, a, kp);
        } else {
            launch_near_tc_d4(kind, grid, st, a, kp);
        }
        return;
    }
    if (d == 3) launch_near_d3(nw, tpt, kind, grid, st, a, kp);
    else launch_near_d4(nw, tpt, kind, grid, st, a, kp);
}

template <int D>
void launch_permute_dim(int nw, unsigned grid, cudaStream_t st, int64_t N, const int32_t* perm, const float4* xs,
                        const float* w, int nr, float sig, const float* pt_sig, float4* rec) {
    switch (nw) {
    case 1: permute_kernel<D, 1><<<grid, 256, 0, st>>>(N, perm, xs, w, nr, sig, pt_sig, rec); break;
    case 4: permute_kernel<D, 4><<<grid, 256, 0, st>>>(N, perm, xs, w, nr, sig, pt_sig, rec); break;
    case 8: permute_kernel<D, 8><<<grid, 256, 0, st>>>(N, perm, xs, w, nr, sig, pt_sig, rec); break;
    case 16: permute_kernel<D, 16><<<grid, 256, 0, st>>>(N, perm, xs, w, nr, sig, pt_sig, rec); break;
    default: permute_kernel<D, 32><<<grid, 256, 0, st>>>(N, perm, xs, w, nr, sig, pt_sig, rec); break;
    }
}

void launch_permute(int d, int nw, unsigned grid, cudaStream_t st, int64_t N, const int32_t* perm, const float4* xs,
                    const float* w, int nr, float sig, const float* pt_sig, float4* rec) {
    if (d <= 3) launch_permute_dim<3>(nw, grid, st, N, perm, xs, w, nr, sig, pt_sig, rec);
    else launch_permute_dim<4>(nw, grid, st, N, perm, xs, w, nr, sig, pt_sig, rec);
}

MvmArgs base_args(fkt_plan_s* P) {
    MvmArgs a{};
    a.N = P->N;
    a.xs = P->xs;
    a.perm = P->perm;
    a.blk = P->blk_range;
    a.far_off = P->far_off;
    a.far_ent = P->far_ent;
    a.near_off = P->near_off;
    a.near_ent = P->near_ent;
    a.masks = P->masks;
    a.nd_begin = P->nd_begin;
    a.nd_end = P->nd_end;
    a.nd_cf = P->nd_cf;
    a.nd_scale = P->nd_scale;
    a.s2m_items = P->s2m_items;
    a.s2m_item_off = P->s2m_item_off;
    a.nd_img = P->nd_img;
    a.nnodes = P->nnodes;
    a.err = P->d_err;
    a.kps = P->kps;
    a.blk_prob = P->blk_prob;
    a.blk_list = nullptr;
    a.pt_sig = P->pt_sig;
    a.wait_cycles = P->wait_cycles;
    a.near_split = 1;
    a.far_split = 1;
    return a;
}

size_t round64(size_t n) { return (n + 63) / 64 * 64; }

// y[r][perm[i]] = ys[r][i] + yadd[r][i] for the sorted targets i0 <= i < i1 only.
__global__ void unpermute_range_kernel(int64_t i0, int64_t i1, int64_t N, int nr, const int32_t* __restrict__ perm,
                                       const float* __restrict__ ys, const float* __restrict__ yadd,
                                       float* __restrict__ y) {
    const int64_t i = i0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= i1) return;
    const int64_t o = perm[i];
    for (int r = 0; r < nr; ++r) y[r * N + o] = ys[r * N + i] + yadd[r * N + i];
}

__global__ void dense_lists_kernel(int64_t nblocks, int64_t* off, int2* ent) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < nblocks) ent[i] = make_int2(0, -1);  // the root holds every point
    if (i <= nblocks) off[i] = i;
}

}  // namespace

// Near field of every target block: one launch, or for a batch one launch per kernel kind over
// that kind's blocks (largest first, so uneven problems balance across the SMs).  exact: keep
// the float32 CUDA-core kernels whatever near_precision says (the exact dense product).
static int near_tc_mode(const fkt_plan_s* P, bool exact) {
    if (exact) return 0;
    return P->near_precision == NEAR_TF32X3 ? 1 : P->near_precision == NEAR_F16X3 ? 2 : 0;
}

// Whether a near stage of nw-wide passes runs the TF32 tensor-core kernel, which reads the pass's
// near-field image (the FP16 kernel leaves the 1/r kernel to it).
static bool near_uses_image(const fkt_plan_s* P, int tc, int nw) {
    if (nw != 32 || tc == 0) return false;
    if (tc == 1) return true;
    if (P->nprob == 0) return P->kernel.kind == FKT_LAPLACE;
    for (int k : P->kind_of_list)
        if (k == FKT_LAPLACE) return true;
    return false;
}

// The pass's near-field image from its source records (a.rec), when the near stage reads it.
static void pack_near_image(fkt_plan_s* P, const MvmArgs& a, int tc, int nw, cudaStream_t st) {
    if (!near_uses_image(P, tc, nw)) return;
    launch_near_image(P->nnodes, P->nd_leaf, P->nd_begin, P->nd_end, P->nd_img, a.rec, a.rec_f4,
                      const_cast<float*>(a.nimg), st);
}

// CTAs per target block of the single-right-hand-side near field of a single problem: small
// problems have too few target blocks to fill the GPU (152 SMs, ~8 CTAs each), so each block's
// near entries are dealt to up to 8 CTAs, each writing its own partial row.
static int near_parts(const fkt_plan_s* P) {
    if (P->nprob != 0 || P->nblocks <= 0) return 1;
    const int64_t want = 152 * 8;
    return (int)std::min<int64_t>(8, std::max<int64_t>(1, (want + P->nblocks - 1) / P->nblocks));
}

void launch_near_stage(fkt_plan_s* P, MvmArgs& a, int nrb, int tpt, cudaStream_t st, bool exact) {
    const int tc = near_tc_mode(P, exact);
    pack_near_image(P, a, tc, nrb, st);
    if (P->nprob == 0) {
        a.blk_list = nullptr;
        a.near_split = (nrb == 1 && !exact) ? near_parts(P) : 1;
        launch_near(P->d, nrb, tpt, tc, P->kernel.kind, (unsigned)(P->nblocks * a.near_split), st, a, P->kp,
                    P->d_wmax);
        a.near_split = 1;
        return;
    }
    for (size_t i = 0; i < P->kind_list.size(); ++i) {
        if (P->kind_list_n[i] == 0) continue;
        a.blk_list = P->kind_list[i];
        launch_near(P->d, nrb, tpt, tc, P->kind_of_list[i], (unsigned)P->kind_list_n[i], st, a, P->kp, P->d_wmax);
    }
    a.blk_list = P->far_list;  // the far stage that follows walks all blocks, most work first
}

// Right-hand sides per s2m / float32 far-field group: 1 for a single right-hand side on the
// float32 far path, 8 otherwise (the tensor-core far field always consumes groups of 8).
static int rhs_block(const fkt_plan_s* P, int nrhs) { return (nrhs == 1 && P->far_precision == FAR_FP32) ? 1 : 8; }

// Right-hand sides per near-field pass of npass (<= kPass) right-hand sides.
static int near_width(int nrb, int npass) {
    return nrb == 1 ? 1 : npass <= 4 ? 4 : npass <= 8 ? 8 : npass <= 16 ? 16 : 32;
}

constexpr int kPass = 32;  // right-hand sides per pass (= the tensor-core far field's N)
static_assert(kPass == kTcN, "a pass feeds one tensor-core far-field launch");

void mvm_buffer_floats(const fkt_plan_s* P, int nrhs, size_t out[kMvmBufs]) {
    const int nrb = rhs_block(P, nrhs);
    const int nw = near_width(nrb, std::min(nrhs, kPass));
    const size_t groups = (size_t)(nrhs + nrb - 1) / nrb;
    const size_t N = (size_t)P->N, NT = (size_t)P->nterms;
    const size_t nodes = std::max<int64_t>(P->nnodes, 1), items = std::max<int64_t>(P->n_s2m_items, 1);
    out[0] = round64(N * 4 * (size_t)rec_f4(P->d, nw));  // records of one pass (reused by every pass)
    out[1] = round64(groups * nrb * N * (nrb == 1 ? near_parts(P) : 1));  // near result (partial rows)
    out[2] = round64(groups * nrb * NT * nodes);         // multipoles
    out[3] = round64(groups * nrb * NT * items);         // s2m partials
    out[4] = P->far_precision == FAR_FP32 ? 0
             : round64(nodes * (size_t)tc_b_bytes(P->nterms, tc_prec_of(P->far_precision)) / 4);
    out[5] = round64(groups * nrb * N * (nrb == 1 ? near_parts(P) : 1));  // far result (partial rows)
    out[6] = near_uses_image(P, near_tc_mode(P, false), nw)  // near-field image of one pass
                 ? round64((size_t)(P->img_pos / 4) * kNearGroupFloats)
                 : 0;
}

int ensure_rhs_capacity(fkt_plan_s* P, int nrhs) {
    const int nrb = rhs_block(P, nrhs);
    const int cap = nrb == 1 ? 1 : (nrhs + 7) / 8 * 8;
    size_t f[kMvmBufs];
    mvm_buffer_floats(P, cap, f);
    if (cap > P->cap_rhs) {
        cudaFree(P->rec);
        cudaFree(P->ynear);
        cudaFree(P->yfar);
        cudaFree(P->mult);
        cudaFree(P->s2m_part);
        P->rec = nullptr;
        P->ynear = P->yfar = P->mult = P->s2m_part = nullptr;
        P->cap_rhs = 0;
        FKT_CUDA_TRY(cudaMalloc(&P->rec, sizeof(float) * f[0]));
        FKT_CUDA_TRY(cudaMalloc(&P->ynear, sizeof(float) * f[1]));
        FKT_CUDA_TRY(cudaMalloc(&P->mult, sizeof(float) * f[2]));
        FKT_CUDA_TRY(cudaMalloc(&P->s2m_part, sizeof(float) * f[3]));
        FKT_CUDA_TRY(cudaMalloc(&P->yfar, sizeof(float) * f[5]));
        P->cap_rhs = cap;
    }
    if (f[6] > P->cap_nimg) {
        cudaFree(P->nimg);
        P->nimg = nullptr;
        P->cap_nimg = 0;
        FKT_CUDA_TRY(cudaMalloc(&P->nimg, sizeof(float) * f[6]));
        P->cap_nimg = f[6];
    }
    if (f[4] && P->cap_tc != P->far_precision + 1) {
        cudaFree(P->tc_image);
        P->tc_image = nullptr;
        P->cap_tc = 0;
        FKT_CUDA_TRY(cudaMalloc(&P->tc_image, sizeof(float) * f[4]));
        P->cap_tc = P->far_precision + 1;
    }
    return FKT_OK;
}

// Stage times of the last product from the plan's events: 0 start, 7 end (plan stream);
// 2-3 s2m and 8-9 far field (second stream); 5-6 near field (plan stream).  The near and far
// stages run concurrently.  With more than one pass each interval spans from the first pass's
// launch to the last one's end.
static int finish_timing(fkt_plan_s* P) {
    FKT_CUDA_TRY(cudaEventRecord(P->ev[7], P->stream));
    FKT_CUDA_TRY(cudaEventSynchronize(P->ev[7]));
    float t_tot = 0, t_s2m = 0, t_near = 0, t_far = 0;
    cudaEventElapsedTime(&t_tot, P->ev[0], P->ev[7]);
    cudaEventElapsedTime(&t_s2m, P->ev[2], P->ev[3]);
    cudaEventElapsedTime(&t_near, P->ev[5], P->ev[6]);
    cudaEventElapsedTime(&t_far, P->ev[8], P->ev[9]);
    P->stats.last_total_ms = t_tot;
    P->stats.last_s2m_ms = t_s2m;
    P->stats.last_near_ms = t_near;
    P->stats.last_far_ms = t_far;
    return FKT_OK;
}

// One product on the plan's stream with the given work buffers.  Per pass of up to 32
// right-hand sides:
//   plan stream:    permute -> near field (whole pass) -----------------> wait -> unpermute(near + far)
//   second stream:            s2m + reduce per group -> far field (float32 per group, or pack +
//                             one tensor-core launch) -> event
// The near and far fields are independent until the final sum, so they share the SMs.  Passes
// reuse one record buffer: the next pass's permute is ordered after this pass's unpermute on the
// plan stream, which itself waited for this pass's s2m and far field.
int run_mvm(fkt_plan_s* P, const MvmBuffers& B, const float* w, float* y, int nrhs, bool timing) {
    const bool tc = P->far_precision != FAR_FP32;
    const int nrb = rhs_block(P, nrhs);
    cudaStream_t st = P->stream, st2 = P->stream2;
    const int64_t N = P->N;
    const size_t NT = (size_t)P->nterms;
    const size_t nodes = std::max<int64_t>(P->nnodes, 1), items = std::max<int64_t>(P->n_s2m_items, 1);
    const unsigned pgrid = (unsigned)((N + 255) / 256);
    if (timing) FKT_CUDA_TRY(cudaEventRecord(P->ev[0], st));
    for (int r0 = 0; r0 < nrhs; r0 += kPass) {
        const int npass = std::min(kPass, nrhs - r0);
        const int nw = near_width(nrb, npass);
        const int g0 = r0 / nrb, ng = (npass + nrb - 1) / nrb;
        const bool first = r0 == 0;
        MvmArgs a = base_args(P);
        a.rec = B.rec;
        a.rec_f4 = rec_f4(P->d, nw);
        a.nimg = B.nimg;
        launch_permute(P->d, nw, pgrid, st, N, P->perm, P->xs, w + (size_t)r0 * N, npass, P->kp.sig, P->pt_sig, B.rec);
        FKT_CUDA_TRY(cudaGetLastError());
        // fork: s2m and the far field on the second stream, the near field on the plan stream
        FKT_CUDA_TRY(cudaEventRecord(P->ev[1], st));
        FKT_CUDA_TRY(cudaStreamWaitEvent(st2, P->ev[1], 0));
        if (timing && first) FKT_CUDA_TRY(cudaEventRecord(P->ev[2], st2));
        for (int gi = 0; gi < ng; ++gi) {
            const int g = g0 + gi;
            MvmArgs ag = a;
            ag.woff = rec_woff(P->d, nw) + gi * nrb;
            ag.mult = B.mult + (size_t)g * nrb * NT * nodes;
            ag.part = B.part + (size_t)g * nrb * NT * items;
            ag.nr = std::min(nrb, nrhs - g * nrb);
            FarLaunch L{&ag, &P->kp, &P->tabs, P->nblocks, P->n_s2m_items, P->nnodes, st2, st2};
            int rc = launch_s2m_any(layout_code(P), P->p, nrb, L);
            if (rc) return rc;
        }
        if (timing) FKT_CUDA_TRY(cudaEventRecord(P->ev[3], st2));
        if (timing && first) FKT_CUDA_TRY(cudaEventRecord(P->ev[8], st2));
        MvmArgs af = a;
        af.blk_list = P->nprob ? P->far_list : nullptr;  // most work first
        if (!tc) {
            for (int gi = 0; gi < ng; ++gi) {
                const int g = g0 + gi;
                MvmArgs ag = af;
                ag.mult = B.mult + (size_t)g * nrb * NT * nodes;
                ag.yfar = B.yfar + (size_t)g * nrb * N;
                ag.nr = std::min(nrb, nrhs - g * nrb);
                ag.far_split = nrb == 1 ? near_parts(P) : 1;  // partial rows, summed by unpermute
                FarLaunch L{&ag, &P->kp, &P->tabs, P->nblocks * ag.far_split, P->n_s2m_items, P->nnodes, st2, st2};
                int rc = launch_far_any(layout_code(P), P->p, nrb, L);
                if (rc) return rc;
            }
        } else {
            af.mult = B.mult + (size_t)g0 * 8 * NT * nodes;
            af.yfar = B.yfar + (size_t)r0 * N;
            TcLaunch T{&af, &P->kp, &P->tabs, P->nblocks, P->nnodes, (int64_t)(8 * NT * nodes), npass, B.image, st2, st2,
                       P->far_kernel};
            int rc = launch_tc_any(layout_code(P), P->p, tc_prec_of(P->far_precision), false, T);  // pack
            if (rc) return rc;
            rc = launch_tc_any(layout_code(P), P->p, tc_prec_of(P->far_precision), true, T);
            if (rc) return rc;
        }
        if (timing) FKT_CUDA_TRY(cudaEventRecord(P->ev[9], st2));
        FKT_CUDA_TRY(cudaEventRecord(P->ev[4], st2));
        // near field of the whole pass on the plan stream
        if (timing && first) FKT_CUDA_TRY(cudaEventRecord(P->ev[5], st));
        a.ynear = B.ynear + (size_t)r0 * N;
        a.nr = npass;
        launch_near_stage(P, a, nw, P->near_tpt, st);
        FKT_CUDA_TRY(cudaGetLastError());
        if (timing) FKT_CUDA_TRY(cudaEventRecord(P->ev[6], st));
        // join, then near + far back to the caller's order
        FKT_CUDA_TRY(cudaStreamWaitEvent(st, P->ev[4], 0));
        if (nw == 1 && near_parts(P) > 1) {  // one right-hand side, near field in partial rows
            unpermute_parts_kernel<><<<pgrid, 256, 0, st>>>(N, near_parts(P), P->perm, B.ynear, B.yfar, y);
        } else {
            unpermute_kernel<><<<pgrid, 256, 0, st>>>(N, npass, P->perm, B.ynear + (size_t)r0 * N,
                                                       B.yfar + (size_t)r0 * N, y + (size_t)r0 * N);
        }
        FKT_CUDA_TRY(cudaGetLastError());
    }
    if (timing) return finish_timing(P);
    return FKT_OK;
}

// ---------------------------------------------------------------- sharded product
// Floats of the multipole array that the ranks sum between the two phases: every group of 8
// right-hand sides of one pass, [group][nodes][nterms][8].
size_t shard_mult_floats(const fkt_plan_s* P, int nrhs) {
    const size_t groups = (size_t)(nrhs + 7) / 8;
    return groups * 8 * (size_t)P->nterms * (size_t)std::max<int64_t>(P->nnodes, 1);
}

// Phase 1 on this rank: source records of every point (the near field reads any source), then
// the partial multipoles of the rank's own sources into mult (zeroed first; nodes without such
// sources stay zero).  One pass: 1 <= nrhs <= 32.
int shard_begin(fkt_plan_s* P, const float* w, float* mult, int nrhs) {
    const int cap = std::max(8, (nrhs + 7) / 8 * 8);
    int rc = ensure_rhs_capacity(P, cap);
    if (rc) return rc;
    cudaStream_t st = P->stream;
    const int64_t N = P->N;
    const size_t NT = (size_t)P->nterms, nodes = std::max<int64_t>(P->nnodes, 1);
    const int nrb = 8, nw = near_width(nrb, nrhs), ng = (nrhs + nrb - 1) / nrb;
    launch_permute(P->d, nw, (unsigned)((N + 255) / 256), st, N, P->perm, P->xs, w, nrhs, P->kp.sig, P->pt_sig, P->rec);
    FKT_CUDA_TRY(cudaGetLastError());
    FKT_CUDA_TRY(cudaMemsetAsync(mult, 0, sizeof(float) * shard_mult_floats(P, nrhs), st));
    MvmArgs a = base_args(P);
    a.rec = P->rec;
    a.rec_f4 = rec_f4(P->d, nw);
    a.s2m_items = P->sh_items;
    a.s2m_item_off = P->sh_item_off;
    for (int g = 0; g < ng; ++g) {
        MvmArgs ag = a;
        ag.woff = rec_woff(P->d, nw) + g * nrb;
        ag.mult = mult + (size_t)g * nrb * NT * nodes;
        ag.part = P->s2m_part + (size_t)g * nrb * NT * std::max<int64_t>(P->n_s2m_items, 1);
        ag.nr = std::min(nrb, nrhs - g * nrb);
        FarLaunch L{&ag, &P->kp, &P->tabs, P->nblocks, P->sh_nitems, P->nnodes, st, st};
        if ((rc = launch_s2m_any(layout_code(P), P->p, nrb, L))) return rc;
    }
    return FKT_OK;
}

// Phase 2 on this rank, after the multipoles were summed over all ranks: far and near field of
// the rank's target blocks, written to y (caller order) for the rank's targets only.  Uses the
// source records of phase 1.
int shard_end(fkt_plan_s* P, const float* mult, float* y, int nrhs) {
    const bool tc = P->far_precision != FAR_FP32;
    cudaStream_t st = P->stream;
    const int64_t N = P->N, nb = P->sh_b1 - P->sh_b0;
    const size_t NT = (size_t)P->nterms, nodes = std::max<int64_t>(P->nnodes, 1);
    const int nrb = 8, nw = near_width(nrb, nrhs), ng = (nrhs + nrb - 1) / nrb;
    if (nb == 0) return FKT_OK;
    MvmArgs a = base_args(P);
    a.rec = P->rec;
    a.rec_f4 = rec_f4(P->d, nw);
    a.blk_list = P->sh_blocks;
    if (!tc) {
        for (int g = 0; g < ng; ++g) {
            MvmArgs ag = a;
            ag.mult = const_cast<float*>(mult) + (size_t)g * nrb * NT * nodes;
            ag.yfar = P->yfar + (size_t)g * nrb * N;
            ag.nr = std::min(nrb, nrhs - g * nrb);
            FarLaunch L{&ag, &P->kp, &P->tabs, nb, P->n_s2m_items, P->nnodes, st, st};
            int rc = launch_far_any(layout_code(P), P->p, nrb, L);
            if (rc) return rc;
        }
    } else {
        MvmArgs af = a;
        af.mult = const_cast<float*>(mult);
        af.yfar = P->yfar;
        TcLaunch T{&af, &P->kp, &P->tabs, nb, P->nnodes, (int64_t)(8 * NT * nodes), nrhs, P->tc_image, st, st,
                   P->far_kernel};
        int rc = launch_tc_any(layout_code(P), P->p, tc_prec_of(P->far_precision), false, T);  // pack every used node
        if (!rc) rc = launch_tc_any(layout_code(P), P->p, tc_prec_of(P->far_precision), true, T);
        if (rc) return rc;
    }
    a.ynear = P->ynear;
    a.nr = nrhs;
    a.nimg = P->nimg;
    pack_near_image(P, a, near_tc_mode(P, false), nw, st);
    launch_near(P->d, nw, P->near_tpt, near_tc_mode(P, false), P->kernel.kind, (unsigned)nb, st, a, P->kp, P->d_wmax);
    FKT_CUDA_TRY(cudaGetLastError());
    const int64_t nt = P->sh_t1 - P->sh_t0;
    unpermute_range_kernel<<<(unsigned)((nt + 255) / 256), 256, 0, st>>>(P->sh_t0, P->sh_t1, N, nrhs, P->perm, P->ynear,
                                                                         P->yfar, y);
    FKT_CUDA_TRY(cudaGetLastError());
    return FKT_OK;
}

int build_near_image_index(fkt_plan_s* P) {
    const int64_t nn = P->nnodes;
    cudaFree(P->nd_img);
    P->nd_img = nullptr;
    P->img_pos = 0;
    if (nn <= 0) return FKT_OK;
    std::vector<int32_t> leaf(nn), b(nn), e(nn), img(nn, -1);
    FKT_CUDA_TRY(cudaMemcpyAsync(leaf.data(), P->nd_leaf, 4 * nn, cudaMemcpyDeviceToHost, P->stream));
    FKT_CUDA_TRY(cudaMemcpyAsync(b.data(), P->nd_begin, 4 * nn, cudaMemcpyDeviceToHost, P->stream));
    FKT_CUDA_TRY(cudaMemcpyAsync(e.data(), P->nd_end, 4 * nn, cudaMemcpyDeviceToHost, P->stream));
    FKT_CUDA_TRY(cudaStreamSynchronize(P->stream));
    int64_t pos = 0;
    for (int64_t i = 0; i < nn; ++i) {
        if (!leaf[i]) continue;
        img[i] = (int32_t)pos;
        pos += (int64_t)(e[i] - b[i] + 7) / 8 * 8;
        if (pos > INT32_MAX) return FKT_ERR_INVALID_ARG;
    }
    FKT_CUDA_TRY(cudaMalloc(&P->nd_img, 4 * nn));
    FKT_CUDA_TRY(cudaMemcpyAsync(P->nd_img, img.data(), 4 * nn, cudaMemcpyHostToDevice, P->stream));
    FKT_CUDA_TRY(cudaStreamSynchronize(P->stream));
    P->img_pos = pos;
    return FKT_OK;
}

int create_far_stream(cudaStream_t* s) {
    FKT_CUDA_TRY(cudaStreamCreateWithFlags(s, cudaStreamNonBlocking));
    return FKT_OK;
}

int launch_mvm(fkt_plan_s* P, const float* w, float* y, int nrhs) {
    int rc = ensure_rhs_capacity(P, nrhs);
    if (rc) return rc;
    MvmBuffers B{P->rec, P->ynear, P->mult, P->s2m_part, P->tc_image, P->yfar, P->nimg};
    return run_mvm(P, B, w, y, nrhs, P->timing);
}

// Exact product: the near kernel with one entry per target block -- the root, which holds every point.
int launch_dense(fkt_plan_s* P, const float* w, float* y, int nrhs) {
    int rc = ensure_rhs_capacity(P, nrhs);
    if (rc) return rc;
    cudaStream_t st = P->stream;
    if (!P->dense_off) {
        FKT_CUDA_TRY(cudaMalloc(&P->dense_off, sizeof(int64_t) * (P->nblocks + 1)));
        FKT_CUDA_TRY(cudaMalloc(&P->dense_ent, sizeof(int2) * P->nblocks));
        dense_lists_kernel<<<(unsigned)((P->nblocks + 256) / 256), 256, 0, st>>>(P->nblocks, P->dense_off, P->dense_ent);
        FKT_CUDA_TRY(cudaGetLastError());
    }
    const int nrb = rhs_block(P, nrhs);
    const int64_t N = P->N;
    const unsigned pg = (unsigned)((N + 255) / 256);
    for (int r0 = 0; r0 < nrhs; r0 += kPass) {
        const int npass = std::min(kPass, nrhs - r0);
        const int nw = near_width(nrb, npass);
        MvmArgs a = base_args(P);
        a.near_off = P->dense_off;
        a.near_ent = P->dense_ent;
        a.rec = P->rec;
        a.rec_f4 = rec_f4(P->d, nw);
        a.ynear = P->ynear + (size_t)r0 * N;
        a.nr = npass;
        launch_permute(P->d, nw, pg, st, N, P->perm, P->xs, w + (size_t)r0 * N, npass, P->kp.sig, P->pt_sig, P->rec);
        launch_near_stage(P, a, nw, P->near_tpt, st, true);
        unpermute_kernel<><<<pg, 256, 0, st>>>(N, npass, P->perm, a.ynear, nullptr, y + (size_t)r0 * N);
        FKT_CUDA_TRY(cudaGetLastError());
    }
    return FKT_OK;
}

}  // namespace fkt
