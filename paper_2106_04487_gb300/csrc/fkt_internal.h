// Internal declarations of the GB300 FKT library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/fkt.h"

namespace fkt {

constexpr int kMaxP3 = 10;        // largest order for d = 3
constexpr int kMaxP4 = 8;         // largest order for d = 4
constexpr int kTB = 128;          // targets per target block (one CTA)
constexpr int kMaskWords = kTB / 32;
constexpr int kMaxRhs = 64;
constexpr int kMaxTerms = 495;    // binom(8+4, 4); binom(10+3, 3) = 286
constexpr long long kWaitCycles = 2000000000;  // ~1 s at 2 GHz: a device-side wait this long is a fault
// Near-field image of a 32-wide pass on the tensor cores: per leaf, its sources in groups of 4
// (the leaf starting at a multiple of 8 image positions, zero-padded to a multiple of 8), each
// group 272 floats: the TF32 hi parts of the 4 x 32 weights in the MMA's K-major core-matrix
// order (right-hand side n, source k: float 4n + k), the lo parts the same way, then the
// negated, kernel-scaled coordinates -x[4], -y[4], -z[4], -u[4].
constexpr int kNearGroupFloats = 272;
constexpr int kNearGroupBytes = 4 * kNearGroupFloats;     // 1088: the MMA's leading-dimension offset
constexpr int kNearChunkBytes = 8 * kNearGroupBytes;      // one 32-source chunk

// Far-field coefficient tables handed to the kernels by value (they land in the
// constant bank).  Index conventions:
//   radial pairs (k, j), j = k, k+2, ..., <= p, enumerated k-major: kj index q
//   That[q][m] = m! * Tbar_{k,j,m} for m <= j   (Theorem 3.1 with the m! of the
//   scaled derivatives folded in, see tables.cpp)
//   Legendre-type recurrence coefficients of the normalised solid harmonics (d = 3)
//   and of the extra Gegenbauer chain level (d = 4).
struct FarTables {
    float That[36][11];      // radial pairs up to p = 10: 36 pairs, m <= 10
    float hA[11][11];        // d=3: Pi_l^m = hA[l][m] z Pi_{l-1}^m - hB[l][m] r2 Pi_{l-2}^m
    float hB[11][11];
    float hSeed[11];         // Pi_m^m
    float gA[9][9];          // d=4 chain level: Q_n^{(l)} = gA[l][n] x4 Q_{n-1} - gB[l][n] r2 Q_{n-2}
    float gB[9][9];
    float gSeed[9];          // normalisation of the chain level per l (Q_0^{(l)})
};

struct KernelParams {
    int kind;
    float ell, alpha, scale;
    float c1;                // kind-specific: 1/(2l^2), 1/l, sqrt3/l, sqrt5/l, 1/l^2, 1/(2 a l^2)
    float c2;                // c1 * log2(e) for the exponential kernels (argument of ex2)
    float sig;               // near-field coordinate scale: distances in the kernel's own units
};

enum FarPrecision { FAR_FP32 = 0, FAR_TF32 = 1, FAR_BF16 = 2, FAR_BF16X3 = 3 };
enum NearPrecision { NEAR_FP32 = 0, NEAR_TF32X3 = 1, NEAR_F16X3 = 2 };

}  // namespace fkt

struct fkt_plan_s {
    // problem
    int64_t N = 0;
    int d = 3, p = 0, leaf_size = 0, nterms = 0;
    double theta = 0.5;
    fkt_kernel kernel{};
    fkt::KernelParams kp{};
    fkt::FarTables tabs{};
    cudaStream_t stream = nullptr;
    int device = 0;                // CUDA device that was current at fkt_plan (the plan's memory lives there)
    long long wait_cycles = fkt::kWaitCycles;  // limit of the tensor-core kernels' pipeline waits (option)
    bool timing = false;
    int far_precision = fkt::FAR_FP32;
    int near_tpt = 2;              // near-field targets per thread (2 or 4)
    int near_precision = fkt::NEAR_FP32;  // near-field contraction of 32-wide passes
    int far_kernel = 1;            // tensor-core far field, d = 3 BF16 forms: 0 = two entries per thread, 1 = one
    bool diag = false;             // radial compression: only the j = k terms (Laplace kernel, d = 3)
    // bounding cube
    double lo[4] = {0, 0, 0, 0};
    double L = 1.0;
    int B = 21;
    // sorted points: float4 (x, y, z, u) per point, u = 0 for d = 3
    float4* xs = nullptr;
    int32_t* perm = nullptr;       // sorted -> original
    uint64_t* codes = nullptr;
    // tree, breadth-first
    int64_t nnodes = 0, nleaves = 0;
    int depth = 0;
    int32_t* nd_begin = nullptr;
    int32_t* nd_end = nullptr;
    int32_t* nd_level = nullptr;
    int32_t* nd_leaf = nullptr;
    int32_t* nd_child = nullptr;   // [nodes][2]
    double* nd_centre = nullptr;   // [nodes][4]
    double* nd_rho2 = nullptr;
    float4* nd_cf = nullptr;       // float32 centre (x, y, z, u)
    float* nd_scale = nullptr;     // s2m/m2t length scale of the node
    int32_t* nd_used = nullptr;    // 1 if some target uses the node's coefficients
    // target blocks and lists
    int64_t nblocks = 0, nfar = 0, nnear = 0, nmasks = 0;
    int2* blk_range = nullptr;     // [lo, hi) sorted targets
    int64_t* far_off = nullptr;    // [nblocks+1]
    int64_t* near_off = nullptr;
    int2* far_ent = nullptr;       // (node, mask)
    int2* near_ent = nullptr;      // (leaf, mask)
    uint32_t* masks = nullptr;     // [nmasks][kMaskWords]
    // s2m work items (node, first point, last point)
    int64_t n_s2m_items = 0;
    int4* s2m_items = nullptr;     // (node, begin, end, unused)
    int32_t* s2m_node_items = nullptr; // per used node: [first item, last item) -> via offsets
    int64_t* s2m_item_off = nullptr;   // [nodes+1] item offsets per node (nodes without items: empty)
    // per-MVM scratch (grown on demand)
    int cap_rhs = 0;
    float4* rec = nullptr;         // source records (point + weights) in tree order, per group
    float* ynear = nullptr;        // near-field result, sorted [nrhs][N]
    float* yfar = nullptr;         // far-field result, sorted [nrhs][N]
    float* mult = nullptr;         // multipoles [nodes][nterms][nrhs]
    float* s2m_part = nullptr;     // per-item partial multipoles [items][nterms][nrhs]
    unsigned char* tc_image = nullptr;  // packed tensor-core operands of the multipoles
    int cap_tc = 0;                // far_precision the image was sized for (0: none)
    int32_t* nd_img = nullptr;     // per node: image position of a leaf's first source (-1: not a leaf)
    int64_t img_pos = 0;           // image positions of all leaves (each leaf padded to a multiple of 8)
    float* nimg = nullptr;         // near-field image of one 32-wide pass (tensor-core near field)
    size_t cap_nimg = 0;           // floats allocated for it
    float* hbuf_w = nullptr;       // device staging for fkt_mvm_host
    float* hbuf_y = nullptr;
    int hbuf_cap = 0;              // right-hand sides the staging buffers hold
    int* d_err = nullptr;          // device error word (bounded waits that ran out)
    unsigned* d_wmax = nullptr;    // device [32]: largest |w| per right-hand side of a pass (FP16 near field)
    int64_t* dense_off = nullptr;  // one-entry lists (the root) per target block, for fkt_dense_mvm
    int2* dense_ent = nullptr;
    // block-Jacobi preconditioner: inverse of K(X_b, X_b) + sigma2 I per target block
    double pc_sigma2 = -1.0;       // sigma2 the inverses were built for (< 0: none)
    int pc_mode = 1;               // 0: no preconditioner (z = r), 1: block-Jacobi, 2: learned correction
    void* learn = nullptr;         // learned-correction state (learn.cu)
    float* pc_learned = nullptr;   // [blocks][kTB][kTB]: A_bb^{-1} + beta^2 V_b V_b^T
    double pc_learned_sigma2 = -1.0;
    float* pc_inv = nullptr;       // [blocks][kTB][kTB], symmetric
    // CG work space (grown on demand)
    int cg_cap = 0;
    double* cg_x = nullptr;        // [nrhs][N] float64 iterate
    double* cg_r = nullptr;        // [nrhs][N] float64 residual
    float* cg_p = nullptr;         // [nrhs][N] search direction
    float* cg_q = nullptr;         // [nrhs][N] (Ktilde + sigma2 I) p
    float* cg_z = nullptr;         // [nrhs][N] preconditioned residual
    double* cg_s = nullptr;        // scalars: [8][kMaxRhs]
    // two-level coarse correction of the preconditioner (coarse.cu)
    int coarse_rank = 0;           // R random Fourier features (0: off)
    uint64_t coarse_seed = 1;
    void* coarse = nullptr;        // coarse-space state
    cudaStream_t stream2 = nullptr;
    cudaEvent_t ev[10] = {};
    // batch of independent problems merged into one plan (empty for a single problem)
    int nprob = 0;
    std::vector<int64_t> prob_off;          // first point of each problem, nprob + 1 entries
    fkt::KernelParams* kps = nullptr;       // device, per problem
    int32_t* blk_prob = nullptr;            // device, per target block
    float* pt_sig = nullptr;                // device, per point: near-field coordinate scale
    std::vector<int> kind_of_list;          // kernel kind of each near work list
    std::vector<int32_t*> kind_list;        // device: target blocks of that kind, largest first
    std::vector<int64_t> kind_list_n;
    int32_t* far_list = nullptr;            // device: all target blocks, most far entries first
    // CUDA graph of the last batched product (replayed while w, y, nrhs stay the same)
    cudaGraphExec_t graph = nullptr;
    const void* graph_w = nullptr;
    const void* graph_y = nullptr;
    int graph_nrhs = 0;
    // target-sharded product (shard.cu): this rank's share of the partition
    int sh_nranks = 0, sh_rank = 0;             // 0 ranks: no share selected
    int64_t sh_b0 = 0, sh_b1 = 0;               // target blocks [b0, b1) in target order
    int32_t* sh_blocks = nullptr;               // device: their block indices
    int64_t sh_t0 = 0, sh_t1 = 0;               // sorted targets (= owned sources) [t0, t1)
    int4* sh_items = nullptr;                   // device: the s2m items cut to [t0, t1)
    int64_t* sh_item_off = nullptr;             // device: [nodes + 1] item offsets per node
    int64_t sh_nitems = 0;
    // stats
    fkt_stats stats{};
};

namespace fkt {

// api.cu
bool radial_compression_exact(int d, int kind);
void set_radial_compression(fkt_plan_s* P, bool on);

// tables.cpp
int build_far_tables(int d, int p, FarTables* out);
KernelParams make_kernel_params(const fkt_kernel& k);

// tree.cu / lists.cu
int build_tree(fkt_plan_s* P, const float* points);
int build_lists(fkt_plan_s* P);

struct MvmArgs;

// mvm.cu
// Work buffers of one MVM call (fkt_mvm: plan-owned; fkt_mvm_noalloc: the static scratch).
struct MvmBuffers {
    float4* rec;
    float* ynear;          // near-field result, tree order
    float* mult;
    float* part;
    unsigned char* image;  // tensor-core operand image of the multipoles (far_precision != fp32)
    float* yfar;           // far-field result, tree order
    float* nimg;           // near-field image of one pass (32-wide passes on the TF32 tensor-core kernel)
};
constexpr int kMvmBufs = 7;
// Floats each buffer needs for nrhs right-hand sides (each rounded up to 64 floats), in the
// order rec, ynear, mult, part, image, yfar, nimg.
void mvm_buffer_floats(const fkt_plan_s* P, int nrhs, size_t out[kMvmBufs]);
int run_mvm(fkt_plan_s* P, const MvmBuffers& B, const float* w, float* y, int nrhs, bool timing);
int launch_mvm(fkt_plan_s* P, const float* w, float* y, int nrhs);
int launch_dense(fkt_plan_s* P, const float* w, float* y, int nrhs);
int ensure_rhs_capacity(fkt_plan_s* P, int nrhs);
// nd_img and img_pos from the tree (host scan over the leaves); once per plan or merged batch.
int build_near_image_index(fkt_plan_s* P);

// The plan's second stream (s2m and the far field), non-blocking.  (A higher priority for it
// makes the far field overlap the near field but gives no net speed-up: both stages compete for
// the same SM resources.)
int create_far_stream(cudaStream_t* s);

// stage launch helpers shared with batch.cu
void launch_near_stage(fkt_plan_s* P, MvmArgs& a, int nrb, int tpt, cudaStream_t st, bool exact = false);
int free_batch_arrays(fkt_plan_s* P);

// shard.cu
int shard_partition(int64_t nblocks, const double* work, int nranks, int64_t* bounds);
int shard_set(fkt_plan_s* P, int nranks, int rank);
int shard_block_work(fkt_plan_s* P, std::vector<double>& work, std::vector<int32_t>* order = nullptr);
void free_shard(fkt_plan_s* P);
// mvm.cu: the two phases of the sharded product (one pass of <= 32 right-hand sides)
size_t shard_mult_floats(const fkt_plan_s* P, int nrhs);
int shard_begin(fkt_plan_s* P, const float* w, float* mult, int nrhs);
int shard_end(fkt_plan_s* P, const float* mult, float* y, int nrhs);

// solve.cu
int precond_setup(fkt_plan_s* P, double sigma2);
int precond_build(fkt_plan_s* P, double sigma2, const float* addV, int R, const float* addT, float* out);
int precond_apply(fkt_plan_s* P, const float* r, const double* r64, float* z, int nrhs);
int solve(fkt_plan_s* P, double sigma2, const float* b, float* x, double* x64, int nrhs, double tol, int max_iter,
          fkt_solve_info* info);
void free_solve(fkt_plan_s* P);

// coarse.cu
int spectral_sample(const fkt_kernel& k, int d, int R, uint64_t seed, double* omega, double* phase);
int coarse_setup(fkt_plan_s* P, double sigma2);
int coarse_apply(fkt_plan_s* P, const double* r64, float* z, int nrhs);
void free_coarse(fkt_plan_s* P);

// learn.cu
int precond_learn(fkt_plan_s* P, double sigma2, const fkt_learn_opts* opts, fkt_learn_info* info);
int learn_params(fkt_plan_s* P, float* out, int* nparams);
int learn_eval(fkt_plan_s* P, const float* params, double* loss, float* grad);
int learn_teacher(fkt_plan_s* P, int64_t* blocks, float* D);
void free_learn(fkt_plan_s* P);

}  // namespace fkt

#define FKT_CUDA_TRY(expr)                                        \
    do {                                                          \
        cudaError_t e__ = (expr);                                 \
        if (e__ != cudaSuccess) {                                 \
            return e__ == cudaErrorMemoryAllocation ? FKT_ERR_OOM \
                                                    : FKT_ERR_CUDA; \
        }                                                         \
    } while (0)
