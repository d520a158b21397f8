// GPU tree build (Sec. 3.1): bounding cube, Morton codes, radix sort, level-synchronous
// midpoint splits, node centres and radii.
//
// Contract (identical decisions on any IEEE machine): lo = min x, L = max extent
// (1 if zero), B = floor(63/d) bits per axis, q_a = min(floor((x_a - lo_a) * (2^B/L)),
// 2^B - 1) in float64 with explicit round-to-nearest operations; codes interleave the
// bits from the top, axis 0 first; stable sort by (code, index); a node at level l
// with more than leaf_size points splits at code bit l (counted from the top), which
// halves the box along axis l mod d (rules (a) and (b) of Sec. 3.1: halving, aspect
// ratio <= 2); empty children are dropped; a node is a leaf iff it holds <= leaf_size
// points or l = d*B.  Centre = box midpoint, radius rho = max |x - c| over the node's
// points (the numerator of eq. accparam).
#include <cub/cub.cuh>

#include <vector>

#include "fkt_internal.h"

namespace fkt {
namespace {

__device__ __forceinline__ unsigned int f2ord(float f) {
    unsigned int u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__host__ __device__ __forceinline__ float ord2f(unsigned int o) {
#ifdef __CUDA_ARCH__
    return __uint_as_float((o & 0x80000000u) ? (o & 0x7fffffffu) : ~o);
#else
    unsigned int u = (o & 0x80000000u) ? (o & 0x7fffffffu) : ~o;
    float f;
    memcpy(&f, &u, 4);
    return f;
#endif
}

// mins[a], maxs[a] as order-preserving uints; bad counts non-finite coordinates.
__global__ void bbox_kernel(const float* __restrict__ pts, int64_t N, int d, unsigned int* mins,
                            unsigned int* maxs, unsigned int* bad) {
    unsigned int mn[4] = {0xffffffffu, 0xffffffffu, 0xffffffffu, 0xffffffffu};
    unsigned int mx[4] = {0, 0, 0, 0};
    unsigned int nb = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        for (int a = 0; a < d; ++a) {
            float v = pts[i * d + a];
            if (!isfinite(v)) { ++nb; continue; }
            unsigned int o = f2ord(v);
            mn[a] = min(mn[a], o);
            mx[a] = max(mx[a], o);
        }
    }
    for (int a = 0; a < d; ++a) {
        for (int off = 16; off; off >>= 1) {
            mn[a] = min(mn[a], __shfl_xor_sync(0xffffffffu, mn[a], off));
            mx[a] = max(mx[a], __shfl_xor_sync(0xffffffffu, mx[a], off));
        }
    }
    for (int off = 16; off; off >>= 1) nb += __shfl_xor_sync(0xffffffffu, nb, off);
    if ((threadIdx.x & 31) == 0) {
        for (int a = 0; a < d; ++a) {
            atomicMin(&mins[a], mn[a]);
            atomicMax(&maxs[a], mx[a]);
        }
        if (nb) atomicAdd(bad, nb);
    }
}

__global__ void morton_kernel(const float* __restrict__ pts, int64_t N, int d, int B, double lo0, double lo1,
                              double lo2, double lo3, double scale, uint64_t* codes, int32_t* idx) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double lo[4] = {lo0, lo1, lo2, lo3};
    const uint64_t qmax = (1ull << B) - 1;
    uint64_t q[4] = {0, 0, 0, 0};
    for (int a = 0; a < d; ++a) {
        double t = floor(__dmul_rn(__dsub_rn((double)pts[i * d + a], lo[a]), scale));
        q[a] = (t >= (double)qmax) ? qmax : (uint64_t)t;
    }
    uint64_t code = 0;
    for (int bit = B - 1; bit >= 0; --bit)
        for (int a = 0; a < d; ++a) code = (code << 1) | ((q[a] >> bit) & 1ull);
    codes[i] = code;
    idx[i] = (int32_t)i;
}

__global__ void gather_points_kernel(const float* __restrict__ pts, int64_t N, int d, const int32_t* __restrict__ perm,
                                     float4* xs) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    int64_t j = perm[i];
    float v[4] = {0, 0, 0, 0};
    for (int a = 0; a < d; ++a) v[a] = pts[j * d + a];
    xs[i] = make_float4(v[0], v[1], v[2], v[3]);
}

// For each node of the current level: decide leaf / split and find the split point.
__global__ void split_kernel(const int32_t* __restrict__ begin, const int32_t* __restrict__ end, int64_t n, int level,
                             int maxlevel, int leaf_size, const uint64_t* __restrict__ codes, int32_t* mid,
                             int32_t* nchild) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t b = begin[i], e = end[i];
    if (e - b <= leaf_size || level >= maxlevel) {
        nchild[i] = 0;
        mid[i] = b;
        return;
    }
    int bitpos = maxlevel - 1 - level;
    // first index in [b, e) whose split bit is 1 (bits are sorted within the node)
    int32_t lo = b, hi = e;
    while (lo < hi) {
        int32_t m = lo + (hi - lo) / 2;
        if ((codes[m] >> bitpos) & 1ull) hi = m; else lo = m + 1;
    }
    mid[i] = lo;
    nchild[i] = (lo > b) + (lo < e);
}

__global__ void emit_children_kernel(const int32_t* __restrict__ begin, const int32_t* __restrict__ end, int64_t n,
                                     const int32_t* __restrict__ mid, const int32_t* __restrict__ nchild,
                                     const int32_t* __restrict__ off, int64_t next_base, int32_t* nbegin,
                                     int32_t* nend, int32_t* child, int32_t* leaf) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t c0 = -1, c1 = -1;
    int32_t o = off[i];
    int32_t b = begin[i], e = end[i], m = mid[i];
    if (nchild[i] > 0) {
        int k = 0;
        if (m > b) { nbegin[o + k] = b; nend[o + k] = m; c0 = (int32_t)(next_base + o + k); ++k; }
        if (m < e) {
            nbegin[o + k] = m; nend[o + k] = e;
            int32_t id = (int32_t)(next_base + o + k);
            if (c0 < 0) c0 = id; else c1 = id;
        }
    }
    child[2 * i] = c0;
    child[2 * i + 1] = c1;
    leaf[i] = nchild[i] == 0;
}

// Centre of each node from the code of its first point; one CTA per node computes rho2.
__global__ void geometry_kernel(const int32_t* __restrict__ begin, const int32_t* __restrict__ end,
                                const int32_t* __restrict__ level, int64_t nnodes, const uint64_t* __restrict__ codes,
                                const float4* __restrict__ xs, int d, int B, double lo0, double lo1, double lo2,
                                double lo3, double L, double* centre, double* rho2, float4* cf, float* scale) {
    int64_t nd = blockIdx.x;
    if (nd >= nnodes) return;
    __shared__ double c[4];
    __shared__ double red[32];
    const double lo[4] = {lo0, lo1, lo2, lo3};
    int32_t b = begin[nd], e = end[nd], lev = level[nd];
    if (threadIdx.x >= d && threadIdx.x < 4) c[threadIdx.x] = 0.0;  // unused axes (d < 4)
    if (threadIdx.x < d) {
        int a = threadIdx.x;
        uint64_t code = codes[b];
        uint64_t q = 0;
        for (int bit = B - 1; bit >= 0; --bit) {
            int pos = (B - 1 - bit) * d + a;
            q = (q << 1) | ((code >> (d * B - 1 - pos)) & 1ull);
        }
        int na = lev > a ? (lev - a + d - 1) / d : 0;
        uint64_t width = 1ull << (B - na);
        uint64_t qlo = (q >> (B - na)) << (B - na);
        double frac = (double)(2 * qlo + width) * ldexp(1.0, -(B + 1));
        c[a] = __dadd_rn(lo[a], __dmul_rn(L, frac));
    }
    __syncthreads();
    double m = 0.0;
    for (int32_t s = b + threadIdx.x; s < e; s += blockDim.x) {
        float4 x = xs[s];
        double dx = __dsub_rn((double)x.x, c[0]);
        double acc = __dmul_rn(dx, dx);
        dx = __dsub_rn((double)x.y, c[1]);
        acc = __dadd_rn(acc, __dmul_rn(dx, dx));
        dx = __dsub_rn((double)x.z, c[2]);
        acc = __dadd_rn(acc, __dmul_rn(dx, dx));
        if (d == 4) {
            dx = __dsub_rn((double)x.w, c[3]);
            acc = __dadd_rn(acc, __dmul_rn(dx, dx));
        }
        m = fmax(m, acc);
    }
    for (int off = 16; off; off >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, red[w]);
        rho2[nd] = m;
        for (int a = 0; a < 4; ++a) centre[nd * 4 + a] = a < d ? c[a] : 0.0;
        cf[nd] = make_float4((float)c[0], (float)c[1], (float)c[2], d == 4 ? (float)c[3] : 0.f);
        double r = sqrt(m);
        scale[nd] = r > 0.0 ? (float)r : 1.0f;
    }
}

template <typename T>
int dalloc(T** p, size_t n) {
    FKT_CUDA_TRY(cudaMalloc((void**)p, sizeof(T) * (n ? n : 1)));
    return FKT_OK;
}

}  // namespace

int build_tree(fkt_plan_s* P, const float* points) {
    const int64_t N = P->N;
    const int d = P->d;
    cudaStream_t st = P->stream;
    const int B = 63 / d;
    P->B = B;
    // ---- bounding cube and finiteness
    unsigned int* red = nullptr;
    FKT_CUDA_TRY(cudaMalloc(&red, sizeof(unsigned int) * 9));
    std::vector<unsigned int> init(9, 0);
    for (int a = 0; a < 4; ++a) init[a] = 0xffffffffu;
    FKT_CUDA_TRY(cudaMemcpyAsync(red, init.data(), sizeof(unsigned int) * 9, cudaMemcpyHostToDevice, st));
    int grid = (int)std::min<int64_t>((N + 255) / 256, 152 * 8);
    bbox_kernel<<<grid, 256, 0, st>>>(points, N, d, red, red + 4, red + 8);
    FKT_CUDA_TRY(cudaGetLastError());
    unsigned int hred[9];
    FKT_CUDA_TRY(cudaMemcpyAsync(hred, red, sizeof(hred), cudaMemcpyDeviceToHost, st));
    FKT_CUDA_TRY(cudaStreamSynchronize(st));
    cudaFree(red);
    if (hred[8] != 0) return FKT_ERR_INVALID_ARG;
    double L = 0.0;
    for (int a = 0; a < d; ++a) {
        double lo = (double)ord2f(hred[a]);
        double hi = (double)ord2f(hred[4 + a]);
        P->lo[a] = lo;
        if (hi - lo > L) L = hi - lo;
    }
    if (L == 0.0) L = 1.0;
    P->L = L;
    const double scale = ldexp(1.0, B) / L;
    // ---- Morton codes + stable radix sort by (code, index)
    uint64_t* codes_in = nullptr;
    int32_t* idx_in = nullptr;
    int rc;
    if ((rc = dalloc(&codes_in, N)) || (rc = dalloc(&idx_in, N)) || (rc = dalloc(&P->codes, N)) ||
        (rc = dalloc(&P->perm, N)) || (rc = dalloc(&P->xs, N)))
        return rc;
    morton_kernel<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(points, N, d, B, P->lo[0], P->lo[1], P->lo[2], P->lo[3],
                                                               scale, codes_in, idx_in);
    FKT_CUDA_TRY(cudaGetLastError());
    size_t tmp_bytes = 0;
    cub::DeviceRadixSort::SortPairs(nullptr, tmp_bytes, codes_in, P->codes, idx_in, P->perm, (int)N, 0, d * B, st);
    void* tmp = nullptr;
    FKT_CUDA_TRY(cudaMalloc(&tmp, tmp_bytes));
    FKT_CUDA_TRY(cub::DeviceRadixSort::SortPairs(tmp, tmp_bytes, codes_in, P->codes, idx_in, P->perm, (int)N, 0, d * B,
                                                 st));
    gather_points_kernel<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(points, N, d, P->perm, P->xs);
    FKT_CUDA_TRY(cudaGetLastError());
    FKT_CUDA_TRY(cudaStreamSynchronize(st));
    cudaFree(tmp);
    cudaFree(codes_in);
    cudaFree(idx_in);
    // ---- level-synchronous splits
    const int maxlevel = d * B;
    struct Level { int32_t *begin, *end, *child, *leaf; int64_t n; };
    std::vector<Level> levels;
    Level cur{};
    cur.n = 1;
    if ((rc = dalloc(&cur.begin, 1)) || (rc = dalloc(&cur.end, 1))) return rc;
    int32_t root[2] = {0, (int32_t)N};
    FKT_CUDA_TRY(cudaMemcpyAsync(cur.begin, &root[0], 4, cudaMemcpyHostToDevice, st));
    FKT_CUDA_TRY(cudaMemcpyAsync(cur.end, &root[1], 4, cudaMemcpyHostToDevice, st));
    int64_t base = 0;
    for (int level = 0;; ++level) {
        int64_t n = cur.n;
        int32_t *mid, *nchild, *off;
        if ((rc = dalloc(&mid, n)) || (rc = dalloc(&nchild, n)) || (rc = dalloc(&off, n + 1)) ||
            (rc = dalloc(&cur.child, 2 * n)) || (rc = dalloc(&cur.leaf, n)))
            return rc;
        unsigned g = (unsigned)((n + 255) / 256);
        split_kernel<<<g, 256, 0, st>>>(cur.begin, cur.end, n, level, maxlevel, P->leaf_size, P->codes, mid, nchild);
        FKT_CUDA_TRY(cudaGetLastError());
        // exclusive scan of the child counts; the total is off[n-1] + nchild[n-1]
        void* stmp = nullptr;
        size_t sb = 0;
        cub::DeviceScan::ExclusiveSum(nullptr, sb, nchild, off, (int)n, st);
        FKT_CUDA_TRY(cudaMalloc(&stmp, sb));
        FKT_CUDA_TRY(cub::DeviceScan::ExclusiveSum(stmp, sb, nchild, off, (int)n, st));
        int32_t last_off = 0, last_cnt = 0;
        FKT_CUDA_TRY(cudaMemcpyAsync(&last_off, off + n - 1, 4, cudaMemcpyDeviceToHost, st));
        FKT_CUDA_TRY(cudaMemcpyAsync(&last_cnt, nchild + n - 1, 4, cudaMemcpyDeviceToHost, st));
        FKT_CUDA_TRY(cudaStreamSynchronize(st));
        cudaFree(stmp);
        int64_t nnext = (int64_t)last_off + last_cnt;
        Level nxt{};
        nxt.n = nnext;
        if (nnext > 0 && ((rc = dalloc(&nxt.begin, nnext)) || (rc = dalloc(&nxt.end, nnext)))) return rc;
        emit_children_kernel<<<g, 256, 0, st>>>(cur.begin, cur.end, n, mid, nchild, off, base + n, nxt.begin, nxt.end,
                                                 cur.child, cur.leaf);
        FKT_CUDA_TRY(cudaGetLastError());
        FKT_CUDA_TRY(cudaStreamSynchronize(st));
        cudaFree(mid);
        cudaFree(nchild);
        cudaFree(off);
        levels.push_back(cur);
        base += n;
        if (nnext == 0) break;
        cur = nxt;
    }
    // ---- concatenate levels (breadth-first order)
    const int64_t nn = base;
    P->nnodes = nn;
    P->depth = (int)levels.size() - 1;
    if ((rc = dalloc(&P->nd_begin, nn)) || (rc = dalloc(&P->nd_end, nn)) || (rc = dalloc(&P->nd_level, nn)) ||
        (rc = dalloc(&P->nd_leaf, nn)) || (rc = dalloc(&P->nd_child, 2 * nn)) || (rc = dalloc(&P->nd_centre, 4 * nn)) ||
        (rc = dalloc(&P->nd_rho2, nn)) || (rc = dalloc(&P->nd_cf, nn)) || (rc = dalloc(&P->nd_scale, nn)) ||
        (rc = dalloc(&P->nd_used, nn)))
        return rc;
    int64_t o = 0;
    std::vector<int32_t> hlev(nn);
    for (size_t l = 0; l < levels.size(); ++l) {
        Level& v = levels[l];
        FKT_CUDA_TRY(cudaMemcpyAsync(P->nd_begin + o, v.begin, 4 * v.n, cudaMemcpyDeviceToDevice, st));
        FKT_CUDA_TRY(cudaMemcpyAsync(P->nd_end + o, v.end, 4 * v.n, cudaMemcpyDeviceToDevice, st));
        FKT_CUDA_TRY(cudaMemcpyAsync(P->nd_leaf + o, v.leaf, 4 * v.n, cudaMemcpyDeviceToDevice, st));
        FKT_CUDA_TRY(cudaMemcpyAsync(P->nd_child + 2 * o, v.child, 8 * v.n, cudaMemcpyDeviceToDevice, st));
        for (int64_t i = 0; i < v.n; ++i) hlev[o + i] = (int32_t)l;
        o += v.n;
    }
    FKT_CUDA_TRY(cudaMemcpyAsync(P->nd_level, hlev.data(), 4 * nn, cudaMemcpyHostToDevice, st));
    FKT_CUDA_TRY(cudaMemsetAsync(P->nd_used, 0, 4 * nn, st));
    FKT_CUDA_TRY(cudaStreamSynchronize(st));
    for (auto& v : levels) {
        cudaFree(v.begin);
        cudaFree(v.end);
        cudaFree(v.child);
        cudaFree(v.leaf);
    }
    geometry_kernel<<<(unsigned)nn, 256, 0, st>>>(P->nd_begin, P->nd_end, P->nd_level, nn, P->codes, P->xs, d, B,
                                                  P->lo[0], P->lo[1], P->lo[2], P->lo[3], P->L, P->nd_centre,
                                                  P->nd_rho2, P->nd_cf, P->nd_scale);
    FKT_CUDA_TRY(cudaGetLastError());
    std::vector<int32_t> hleaf(nn);
    FKT_CUDA_TRY(cudaMemcpyAsync(hleaf.data(), P->nd_leaf, 4 * nn, cudaMemcpyDeviceToHost, st));
    FKT_CUDA_TRY(cudaStreamSynchronize(st));
    int64_t nl = 0;
    for (int64_t i = 0; i < nn; ++i) nl += hleaf[i] != 0;
    P->nleaves = nl;
    return FKT_OK;
}

}  // namespace fkt
