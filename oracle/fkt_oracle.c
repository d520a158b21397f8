/*
 * CPU FP64 oracle of the Fast Kernel Transform (FKT) matrix-vector product.
 *
 * TEST INFRASTRUCTURE ONLY: this file is built into liborc_fkt.so, which only
 * tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may load.
 * It shares no code with the GPU library (paper_2106_04487_gb300/csrc).
 *
 * Plain, slow and step by step, in the order of the paper:
 *   - eq. nbody (Sec. 3):            z_i = sum_j K(|r_i - r_j|) y_j      -> orc_dense
 *   - Sec. 3.1:                      binary space partitioning tree       -> build_tree
 *   - eq. accparam (Sec. 3.1):       far iff max_{r' in b}|r'-c_b| / |r-c_b| < theta
 *   - Algorithm 1 (Sec. 3.2):        z[far] += m2t * (s2m * y[node]);  z[near] += K(near, leaf) y[leaf]
 *   - Theorem 3.1 / eq. finaltrunc:  K(|r'-r|) ~ sum_{k<=p} sum_h Y_k^h(r) Y_k^h(r') K_p^(k)(r', r)
 *   - eq. kdef:                      K_p^(k)(r', r) = sum_{j=k,k+2..<=p} r'^j sum_{m=0}^j K^(m)(r) r^(m-j) Tbar_{k,j,m}
 *   - Sec. A.1:                      Gegenbauer recurrence and the addition theorem
 *   - Sec. B.1:                      K^(m) by Taylor-mode automatic differentiation
 *
 * The table Tbar is an input (exact rationals from oracle/tables.py, rounded
 * once to double).  The harmonic basis of degree k is the zonal construction
 * Ytilde_k(u) = L_k^{-1} [C_k^alpha(u . v_i)]_i with G_k = [C_k^alpha(v_i . v_j)] = L_k L_k^T
 * for D_k = |H_k| given unit vectors v_i; it satisfies
 * sum_h Ytilde_kh(u) Ytilde_kh(v) = C_k^alpha(u . v), so Tbar is used without
 * the normalisation Z_k (which the paper never gives).  In d = 2 (alpha = 0) the zonal
 * function of degree k is the Chebyshev T_k and the table is built for it.
 *
 * Tree contract (midpoint splits cycling the axes, Sec. 3.1 rules (a), (b)): bounding cube lo = min x, L = max extent;
 * q_a = min(floor((x_a - lo_a) * (2^B / L)), 2^B - 1) with B = floor(63/d);
 * Morton code interleaving bits from the top, axis 0 first; stable sort by
 * (code, index); a node at level l with more than leaf_size points splits at
 * code bit l (axis l mod d, box midpoint); empty children are dropped; a node
 * is a leaf iff it holds <= leaf_size points or l = d*B.  Centre = box
 * midpoint lo + L * (2 q_lo + width) / 2^(B+1); rho2 = max |x_s - c|^2.
 * All FP64 arithmetic here must be compiled with -ffp-contract=off so the
 * tree and the far decisions are reproducible bit for bit.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAXP 32
#define ORC_MAXD 8

enum { ORC_GAUSSIAN = 0, ORC_EXPONENTIAL = 1, ORC_MATERN32 = 2, ORC_MATERN52 = 3,
       ORC_CAUCHY = 4, ORC_RATQUAD = 5, ORC_LAPLACE = 6 };

typedef struct { int kind; double ell, alpha, scale; } okernel;

static okernel mk_kernel(const double* kp) {
    okernel k;
    k.kind = (int)kp[0];
    k.ell = kp[1];
    k.alpha = kp[2];
    k.scale = kp[3];
    return k;
}

static int kernel_singular(const okernel* k) { return k->kind == ORC_LAPLACE; }

/* Kernel values (Table 1 of the paper, plus the Gaussian, Matern-5/2 and
 * Laplace kernels of the workloads; Cauchy 1/(1 + r^2/l^2), rational quadratic
 * (1 + r^2/(2 a l^2))^(-a)). */
static double kernel_value(const okernel* k, double r) {
    double s = k->scale, l = k->ell;
    switch (k->kind) {
    case ORC_GAUSSIAN: return s * exp(-(r * r) / (2.0 * l * l));
    case ORC_EXPONENTIAL: return s * exp(-r / l);
    case ORC_MATERN32: { double t = sqrt(3.0) * r / l; return s * (1.0 + t) * exp(-t); }
    case ORC_MATERN52: { double t = sqrt(5.0) * r / l; return s * (1.0 + t + t * t / 3.0) * exp(-t); }
    case ORC_CAUCHY: return s / (1.0 + (r * r) / (l * l));
    case ORC_RATQUAD: return s * pow(1.0 + (r * r) / (2.0 * k->alpha * l * l), -k->alpha);
    case ORC_LAPLACE: return s / r;
    }
    return NAN;
}

/* ---- truncated Taylor series ("jets") in one variable, orders 0..n ---- */
typedef struct { int n; double c[ORC_MAXP + 1]; } jet;

static jet jconst(int n, double v) { jet a; memset(&a, 0, sizeof a); a.n = n; a.c[0] = v; return a; }
static jet jvar(int n, double r) { jet a = jconst(n, r); if (n >= 1) a.c[1] = 1.0; return a; }
static jet jadd(jet a, jet b) { for (int i = 0; i <= a.n; ++i) a.c[i] += b.c[i]; return a; }
static jet jscale(jet a, double s) { for (int i = 0; i <= a.n; ++i) a.c[i] *= s; return a; }
static jet jaddc(jet a, double v) { a.c[0] += v; return a; }
static jet jmul(jet a, jet b) {
    jet o = jconst(a.n, 0.0);
    for (int i = 0; i <= a.n; ++i)
        for (int j = 0; j + i <= a.n; ++j) o.c[i + j] += a.c[i] * b.c[j];
    return o;
}
/* 1/a: a * q = 1 */
static jet jrecip(jet a) {
    jet q = jconst(a.n, 0.0);
    q.c[0] = 1.0 / a.c[0];
    for (int m = 1; m <= a.n; ++m) {
        double s = 0.0;
        for (int i = 1; i <= m; ++i) s += a.c[i] * q.c[m - i];
        q.c[m] = -s / a.c[0];
    }
    return q;
}
/* exp(a): e' = a' e  =>  m e_m = sum_{i=1}^m i a_i e_{m-i} */
static jet jexp(jet a) {
    jet e = jconst(a.n, 0.0);
    e.c[0] = exp(a.c[0]);
    for (int m = 1; m <= a.n; ++m) {
        double s = 0.0;
        for (int i = 1; i <= m; ++i) s += i * a.c[i] * e.c[m - i];
        e.c[m] = s / m;
    }
    return e;
}
/* log(a): a l' = a'  =>  a_0 m l_m = m a_m - sum_{i=1}^{m-1} i l_i a_{m-i} */
static jet jlog(jet a) {
    jet l = jconst(a.n, 0.0);
    l.c[0] = log(a.c[0]);
    for (int m = 1; m <= a.n; ++m) {
        double s = m * a.c[m];
        for (int i = 1; i < m; ++i) s -= i * l.c[i] * a.c[m - i];
        l.c[m] = s / (m * a.c[0]);
    }
    return l;
}
static jet jpow(jet a, double beta) { return jexp(jscale(jlog(a), beta)); }

/* Taylor coefficients of tau -> K(r + tau), orders 0..n (Taylor-mode AD, Sec. B.1). */
static jet kernel_jet(const okernel* k, double r, int n) {
    jet x = jvar(n, r), out;
    double l = k->ell;
    switch (k->kind) {
    case ORC_GAUSSIAN: out = jexp(jscale(jmul(x, x), -1.0 / (2.0 * l * l))); break;
    case ORC_EXPONENTIAL: out = jexp(jscale(x, -1.0 / l)); break;
    case ORC_MATERN32: { jet t = jscale(x, sqrt(3.0) / l); out = jmul(jaddc(t, 1.0), jexp(jscale(t, -1.0))); break; }
    case ORC_MATERN52: {
        jet t = jscale(x, sqrt(5.0) / l);
        jet poly = jaddc(jadd(t, jscale(jmul(t, t), 1.0 / 3.0)), 1.0);
        out = jmul(poly, jexp(jscale(t, -1.0)));
        break;
    }
    case ORC_CAUCHY: out = jrecip(jaddc(jscale(jmul(x, x), 1.0 / (l * l)), 1.0)); break;
    case ORC_RATQUAD: out = jpow(jaddc(jscale(jmul(x, x), 1.0 / (2.0 * k->alpha * l * l)), 1.0), -k->alpha); break;
    case ORC_LAPLACE: out = jrecip(x); break;
    default: out = jconst(n, NAN);
    }
    return jscale(out, k->scale);
}

/* K^(m)(r) for m = 0..n */
static void kernel_derivs(const okernel* k, double r, int n, double* out) {
    jet j = kernel_jet(k, r, n);
    double f = 1.0;
    for (int m = 0; m <= n; ++m) {
        if (m > 0) f *= m;
        out[m] = j.c[m] * f;
    }
}

/* Zonal functions of degree 0..n at x: Gegenbauer C_n^alpha (Sec. A.1 recurrence); for
 * alpha = 0 (d = 2), where C_n^0 vanishes for n >= 1, the Chebyshev T_n, the limit of
 * C_n^alpha / alpha up to the factor 2/n that the d = 2 coefficient tables absorb. */
static void gegenbauer(double alpha, int n, double x, double* C) {
    C[0] = 1.0;
    if (alpha == 0.0) {
        if (n >= 1) C[1] = x;
        for (int m = 2; m <= n; ++m) C[m] = 2.0 * x * C[m - 1] - C[m - 2];
        return;
    }
    if (n >= 1) C[1] = 2.0 * alpha * x;
    for (int m = 2; m <= n; ++m)
        C[m] = (2.0 * x * (m + alpha - 1.0) * C[m - 1] - (m + 2.0 * alpha - 2.0) * C[m - 2]) / m;
}

static double dot(const double* a, const double* b, int d) {
    double s = 0.0;
    for (int i = 0; i < d; ++i) s += a[i] * b[i];
    return s;
}

/* ---------------------------- expansion basis ---------------------------- */
typedef struct {
    int d, p;
    double alpha;
    int Dk[ORC_MAXP + 1];     /* |H_k| */
    int voff[ORC_MAXP + 1];   /* offset of the k-th block of zonal points (in points) */
    double* v;                /* zonal points, unit vectors, [sum Dk][d] */
    double* L;                /* Cholesky factors, block k at loff[k], Dk x Dk row-major */
    int loff[ORC_MAXP + 1];
    double* T;                /* Tbar[k][j][m], (p+1)^3 */
    int nterms;               /* sum_k Dk * (number of j) */
    int toff[ORC_MAXP + 1];   /* offset of degree k in a multipole vector; layout [k][i][jj] */
    int nj[ORC_MAXP + 1];     /* number of j values for degree k: floor((p-k)/2)+1 */
} obasis;

static double Tb(const obasis* b, int k, int j, int m) {
    int P = b->p + 1;
    return b->T[(k * P + j) * P + m];
}

/* Build the zonal-Gram basis; returns NULL if a Gram matrix is not positive definite. */
void* orc_basis_new(int d, int p, const double* Tbar, const int* Dk, const double* zonal_pts) {
    if (d < 2 || d > ORC_MAXD || p < 0 || p > ORC_MAXP) return NULL;
    obasis* b = (obasis*)calloc(1, sizeof(obasis));
    b->d = d;
    b->p = p;
    b->alpha = d / 2.0 - 1.0;
    int nv = 0, nl = 0, nt = 0;
    for (int k = 0; k <= p; ++k) {
        b->Dk[k] = Dk[k];
        b->voff[k] = nv;
        b->loff[k] = nl;
        b->toff[k] = nt;
        b->nj[k] = (p - k) / 2 + 1;
        nv += Dk[k];
        nl += Dk[k] * Dk[k];
        nt += Dk[k] * b->nj[k];
    }
    b->nterms = nt;
    b->v = (double*)malloc(sizeof(double) * nv * d);
    memcpy(b->v, zonal_pts, sizeof(double) * nv * d);
    b->L = (double*)calloc(nl, sizeof(double));
    b->T = (double*)malloc(sizeof(double) * (p + 1) * (p + 1) * (p + 1));
    memcpy(b->T, Tbar, sizeof(double) * (p + 1) * (p + 1) * (p + 1));
    double C[ORC_MAXP + 1];
    for (int k = 0; k <= p; ++k) {
        int D = Dk[k];
        double* L = b->L + b->loff[k];
        const double* V = b->v + (size_t)b->voff[k] * d;
        /* G_ij = C_k(v_i . v_j), then plain Cholesky G = L L^T */
        for (int i = 0; i < D; ++i)
            for (int j = 0; j <= i; ++j) {
                gegenbauer(b->alpha, k, dot(V + i * d, V + j * d, d), C);
                L[i * D + j] = C[k];
            }
        for (int j = 0; j < D; ++j) {
            double s = L[j * D + j];
            for (int t = 0; t < j; ++t) s -= L[j * D + t] * L[j * D + t];
            if (!(s > 0.0)) { free(b->v); free(b->L); free(b->T); free(b); return NULL; }
            L[j * D + j] = sqrt(s);
            for (int i = j + 1; i < D; ++i) {
                double u = L[i * D + j];
                for (int t = 0; t < j; ++t) u -= L[i * D + t] * L[j * D + t];
                L[i * D + j] = u / L[j * D + j];
            }
        }
    }
    return b;
}

void orc_basis_free(void* h) {
    obasis* b = (obasis*)h;
    if (!b) return;
    free(b->v);
    free(b->L);
    free(b->T);
    free(b);
}

int orc_basis_nterms(void* h) { return ((obasis*)h)->nterms; }

/* Ytilde_k(u) = L_k^{-1} [C_k(u . v_i)]_i by forward substitution; u a unit vector. */
static void harmonics_k(const obasis* b, int k, const double* u, double* Y) {
    int D = b->Dk[k], d = b->d;
    const double* L = b->L + b->loff[k];
    const double* V = b->v + (size_t)b->voff[k] * d;
    double C[ORC_MAXP + 1];
    for (int i = 0; i < D; ++i) {
        gegenbauer(b->alpha, k, dot(u, V + i * d, d), C);
        double s = C[k];
        for (int t = 0; t < i; ++t) s -= L[i * D + t] * Y[t];
        Y[i] = s / L[i * D + i];
    }
}

/* Harmonic values of all degrees k <= p at unit vector u, concatenated. */
void orc_harmonics(void* h, const double* u, double* out) {
    obasis* b = (obasis*)h;
    int off = 0;
    for (int k = 0; k <= b->p; ++k) {
        harmonics_k(b, k, u, out + off);
        off += b->Dk[k];
    }
}

/* Source side (s2m) of one point: adds w * r'^j * Ytilde_kh(x'/r') to M[k][h][jj]. */
static void s2m_point(const obasis* b, const double* xp, const double* w, int nrhs, double* M) {
    int d = b->d, p = b->p, nt = b->nterms;
    double rp = sqrt(dot(xp, xp, d));
    if (rp == 0.0) { /* only k = 0, j = 0 survives (0^0 = 1) */
        double Y0[1];
        double u[ORC_MAXD] = {1.0};
        harmonics_k(b, 0, u, Y0);
        for (int q = 0; q < nrhs; ++q) M[(size_t)q * nt + b->toff[0]] += w[q] * Y0[0];
        return;
    }
    double u[ORC_MAXD], rpow[ORC_MAXP + 1];
    for (int a = 0; a < d; ++a) u[a] = xp[a] / rp;
    rpow[0] = 1.0;
    for (int j = 1; j <= p; ++j) rpow[j] = rpow[j - 1] * rp;
    double* Y = (double*)malloc(sizeof(double) * (b->Dk[p] + 1));
    for (int k = 0; k <= p; ++k) {
        harmonics_k(b, k, u, Y);
        for (int i = 0; i < b->Dk[k]; ++i)
            for (int jj = 0; jj < b->nj[k]; ++jj) {
                double basis = rpow[k + 2 * jj] * Y[i];
                size_t t = (size_t)b->toff[k] + (size_t)i * b->nj[k] + jj;
                for (int q = 0; q < nrhs; ++q) M[(size_t)q * nt + t] += w[q] * basis;
            }
    }
    free(Y);
}

/* Target side (m2t) of one (target, node) pair: z[q] += sum Ytilde_kh(x/r) g_kj(r) M[k][h][jj],
 * g_kj(r) = r^{-j} sum_{m=0}^{j} K^(m)(r) r^m Tbar_{k,j,m}  (eq. kdef, truncated at p). */
static void m2t_point(const obasis* b, const okernel* ker, const double* x, const double* M, int nrhs, double* z) {
    int d = b->d, p = b->p, nt = b->nterms;
    double r = sqrt(dot(x, x, d));
    double u[ORC_MAXD], Kd[ORC_MAXP + 1], rpow[2 * ORC_MAXP + 2];
    for (int a = 0; a < d; ++a) u[a] = x[a] / r;
    kernel_derivs(ker, r, p, Kd);
    rpow[0] = 1.0;
    for (int i = 1; i <= p; ++i) rpow[i] = rpow[i - 1] * r;
    double* Y = (double*)malloc(sizeof(double) * (b->Dk[p] + 1));
    for (int k = 0; k <= p; ++k) {
        harmonics_k(b, k, u, Y);
        for (int jj = 0; jj < b->nj[k]; ++jj) {
            int j = k + 2 * jj;
            double g = 0.0;
            for (int m = 0; m <= j; ++m) g += Kd[m] * rpow[m] * Tb(b, k, j, m);
            g /= rpow[j];
            for (int i = 0; i < b->Dk[k]; ++i) {
                size_t t = (size_t)b->toff[k] + (size_t)i * b->nj[k] + jj;
                for (int q = 0; q < nrhs; ++q) z[q] += Y[i] * g * M[(size_t)q * nt + t];
            }
        }
    }
    free(Y);
}

/* Truncated expansion of K(|x - x'|) for n pairs (x = target rel. centre, x' = source rel. centre),
 * through the factorised s2m/m2t form with one unit weight. */
void orc_expansion_pairs(void* h, const double* kp, const double* X, const double* XP, int64_t n, double* out) {
    obasis* b = (obasis*)h;
    okernel ker = mk_kernel(kp);
    #pragma omp parallel
    {
        double* M = (double*)malloc(sizeof(double) * b->nterms);
        #pragma omp for schedule(static)
        for (int64_t i = 0; i < n; ++i) {
            memset(M, 0, sizeof(double) * b->nterms);
            double one = 1.0, z = 0.0;
            s2m_point(b, XP + i * b->d, &one, 1, M);
            m2t_point(b, &ker, X + i * b->d, M, 1, &z);
            out[i] = z;
        }
        free(M);
    }
}

/* Same truncated expansion through the Gegenbauer form (addition theorem applied,
 * no harmonic basis): sum_k C_k(cos g) sum_j r'^j g_kj(r). */
void orc_expansion_pairs_gegenbauer(int d, int p, const double* Tbar, const double* kp,
                                    const double* X, const double* XP, int64_t n, double* out) {
    okernel ker = mk_kernel(kp);
    double alpha = d / 2.0 - 1.0;
    int P = p + 1;
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        const double* x = X + i * d;
        const double* xp = XP + i * d;
        double r = sqrt(dot(x, x, d)), rp = sqrt(dot(xp, xp, d));
        double cg = (rp > 0.0) ? dot(x, xp, d) / (r * rp) : 0.0;
        double Kd[ORC_MAXP + 1], C[ORC_MAXP + 1];
        kernel_derivs(&ker, r, p, Kd);
        gegenbauer(alpha, p, cg, C);
        double z = 0.0;
        for (int k = 0; k <= p; ++k)
            for (int j = k; j <= p; j += 2) {
                double g = 0.0;
                for (int m = 0; m <= j; ++m) g += Kd[m] * pow(r, m - j) * Tbar[(k * P + j) * P + m];
                z += C[k] * pow(rp, j) * g;
            }
        out[i] = z;
    }
}

/* Exported scalar helpers for the pins. */
double orc_kernel_value(const double* kp, double r) { okernel k = mk_kernel(kp); return kernel_value(&k, r); }
void orc_kernel_derivs(const double* kp, double r, int n, double* out) { okernel k = mk_kernel(kp); kernel_derivs(&k, r, n, out); }
void orc_gegenbauer(double alpha, int n, double x, double* out) { gegenbauer(alpha, n, x, out); }

/* ------------------------------ dense MVM ------------------------------- */
/* z[q][t] = sum_s K(|x_t - x_s|) w[q][s] over all sources (eq. nbody); a singular
 * kernel skips r = 0 pairs (eq. nbody includes j = i; 1/r is singular there). Targets are indices into X. */
int orc_dense(const float* X, int64_t N, int d, const double* kp, const double* W, int nrhs,
              const int64_t* targets, int64_t nt, double* out) {
    okernel ker = mk_kernel(kp);
    int sing = kernel_singular(&ker);
    #pragma omp parallel for schedule(dynamic, 16)
    for (int64_t ti = 0; ti < nt; ++ti) {
        int64_t t = targets[ti];
        double acc[64];
        for (int q = 0; q < nrhs; ++q) acc[q] = 0.0;
        for (int64_t s = 0; s < N; ++s) {
            double r2 = 0.0;
            for (int a = 0; a < d; ++a) {
                double dx = (double)X[t * d + a] - (double)X[s * d + a];
                r2 += dx * dx;
            }
            if (sing && r2 == 0.0) continue;
            double kv = kernel_value(&ker, sqrt(r2));
            for (int q = 0; q < nrhs; ++q) acc[q] += kv * W[(size_t)q * N + s];
        }
        for (int q = 0; q < nrhs; ++q) out[(size_t)q * nt + ti] = acc[q];
    }
    return 0;
}

/* ---------------------------------- tree --------------------------------- */
typedef struct {
    int64_t begin, end;
    int level, leaf;
    int64_t child[2];
    double c[ORC_MAXD];
    double rho2;
} onode;

typedef struct {
    int d, p, leaf_size, B;
    int64_t N;
    double theta, theta2;
    okernel ker;
    obasis* basis;
    double lo[ORC_MAXD], L;
    float* X;        /* sorted points [N][d] */
    int64_t* perm;   /* sorted position -> original index */
    uint64_t* code;  /* sorted codes */
    onode* nodes;
    int64_t nnodes, cap;
    double* W;       /* sorted weights [nrhs][N] */
    int nrhs;
    double* M;       /* multipoles [node][nrhs][nterms] */
} ofkt;

typedef struct { uint64_t code; int64_t idx; } keyidx;

static int cmp_keyidx(const void* a, const void* b) {
    const keyidx* x = (const keyidx*)a;
    const keyidx* y = (const keyidx*)b;
    if (x->code != y->code) return x->code < y->code ? -1 : 1;
    if (x->idx != y->idx) return x->idx < y->idx ? -1 : 1;
    return 0;
}

static double dist2(const float* x, const double* c, int d) {
    double s = 0.0;
    for (int a = 0; a < d; ++a) {
        double dx = (double)x[a] - c[a];
        s = s + dx * dx;
    }
    return s;
}

static int64_t push_node(ofkt* f, int64_t begin, int64_t end, int level) {
    if (f->nnodes == f->cap) {
        f->cap = f->cap ? 2 * f->cap : 1024;
        f->nodes = (onode*)realloc(f->nodes, sizeof(onode) * f->cap);
    }
    onode* n = &f->nodes[f->nnodes];
    memset(n, 0, sizeof *n);
    n->begin = begin;
    n->end = end;
    n->level = level;
    n->child[0] = n->child[1] = -1;
    return f->nnodes++;
}

/* quantised coordinate of axis a of a Morton code */
static uint64_t code_axis(uint64_t code, int a, int d, int B) {
    uint64_t q = 0;
    for (int bit = B - 1; bit >= 0; --bit) {
        int pos = (B - 1 - bit) * d + a;           /* position from the top (0 = MSB of the d*B-bit code) */
        uint64_t v = (code >> (d * B - 1 - pos)) & 1u;
        q = (q << 1) | v;
    }
    return q;
}

static void node_geometry(ofkt* f, onode* n) {
    int d = f->d, B = f->B;
    uint64_t c0 = f->code[n->begin];
    for (int a = 0; a < d; ++a) {
        int na = (n->level > a) ? (n->level - a + d - 1) / d : 0; /* splits applied to axis a */
        uint64_t q = code_axis(c0, a, d, B);
        uint64_t width = (uint64_t)1 << (B - na);
        uint64_t qlo = (q >> (B - na)) << (B - na);
        double frac = (double)(2 * qlo + width) * ldexp(1.0, -(B + 1));
        n->c[a] = f->lo[a] + f->L * frac;
    }
    double r2 = 0.0;
    for (int64_t s = n->begin; s < n->end; ++s) {
        double v = dist2(f->X + s * d, n->c, d);
        if (v > r2) r2 = v;
    }
    n->rho2 = r2;
}

static void build_tree(ofkt* f) {
    int d = f->d, B = f->B;
    int64_t N = f->N;
    int maxlevel = d * B;
    int64_t root = push_node(f, 0, N, 0);
    (void)root;
    for (int64_t i = 0; i < f->nnodes; ++i) { /* breadth-first: the array grows as we go */
        onode n = f->nodes[i];
        int64_t cnt = n.end - n.begin;
        if (cnt <= f->leaf_size || n.level >= maxlevel) { f->nodes[i].leaf = 1; continue; }
        int bitpos = maxlevel - 1 - n.level; /* code bit (from the LSB) that splits this node */
        int64_t mid = n.begin;
        while (mid < n.end && ((f->code[mid] >> bitpos) & 1u) == 0) ++mid;
        /* push_node may reallocate the node array: take the index first, then store it */
        int nc = 0;
        if (mid > n.begin) { int64_t c = push_node(f, n.begin, mid, n.level + 1); f->nodes[i].child[nc++] = c; }
        if (mid < n.end) { int64_t c = push_node(f, mid, n.end, n.level + 1); f->nodes[i].child[nc++] = c; }
    }
    for (int64_t i = 0; i < f->nnodes; ++i) node_geometry(f, &f->nodes[i]);
}

void* orc_fkt_new(const float* X, int64_t N, int d, const double* kp, int p, int leaf_size,
                  double theta, void* basis) {
    if (N < 1 || d < 2 || d > ORC_MAXD || leaf_size < 1 || !(theta > 0.0 && theta < 1.0) || !basis) return NULL;
    ofkt* f = (ofkt*)calloc(1, sizeof(ofkt));
    f->d = d;
    f->p = p;
    f->N = N;
    f->leaf_size = leaf_size;
    f->B = 63 / d;
    f->theta = theta;
    f->theta2 = theta * theta;
    f->ker = mk_kernel(kp);
    f->basis = (obasis*)basis;
    /* bounding cube */
    double mx[ORC_MAXD];
    for (int a = 0; a < d; ++a) { f->lo[a] = X[a]; mx[a] = X[a]; }
    for (int64_t i = 1; i < N; ++i)
        for (int a = 0; a < d; ++a) {
            double v = X[i * d + a];
            if (v < f->lo[a]) f->lo[a] = v;
            if (v > mx[a]) mx[a] = v;
        }
    f->L = 0.0;
    for (int a = 0; a < d; ++a) if (mx[a] - f->lo[a] > f->L) f->L = mx[a] - f->lo[a];
    if (f->L == 0.0) f->L = 1.0;
    /* Morton codes */
    int B = f->B;
    double scale = ldexp(1.0, B) / f->L;
    uint64_t qmax = ((uint64_t)1 << B) - 1;
    keyidx* ki = (keyidx*)malloc(sizeof(keyidx) * N);
    for (int64_t i = 0; i < N; ++i) {
        uint64_t q[ORC_MAXD];
        for (int a = 0; a < d; ++a) {
            double t = floor(((double)X[i * d + a] - f->lo[a]) * scale);
            q[a] = (t >= (double)qmax) ? qmax : (uint64_t)t;
        }
        uint64_t code = 0;
        for (int bit = B - 1; bit >= 0; --bit)
            for (int a = 0; a < d; ++a) code = (code << 1) | ((q[a] >> bit) & 1u);
        ki[i].code = code;
        ki[i].idx = i;
    }
    qsort(ki, N, sizeof(keyidx), cmp_keyidx);
    f->X = (float*)malloc(sizeof(float) * N * d);
    f->perm = (int64_t*)malloc(sizeof(int64_t) * N);
    f->code = (uint64_t*)malloc(sizeof(uint64_t) * N);
    for (int64_t i = 0; i < N; ++i) {
        f->perm[i] = ki[i].idx;
        f->code[i] = ki[i].code;
        memcpy(f->X + i * d, X + ki[i].idx * d, sizeof(float) * d);
    }
    free(ki);
    build_tree(f);
    return f;
}

void orc_fkt_free(void* h) {
    ofkt* f = (ofkt*)h;
    if (!f) return;
    free(f->X); free(f->perm); free(f->code); free(f->nodes); free(f->W); free(f->M);
    free(f);
}

int64_t orc_fkt_num_nodes(void* h) { return ((ofkt*)h)->nnodes; }

/* Tree export: begin, end, level, leaf flag, children, centres [n][d], rho2. */
void orc_fkt_nodes(void* h, int64_t* begin, int64_t* end, int32_t* level, int32_t* leaf,
                   int64_t* child, double* centre, double* rho2) {
    ofkt* f = (ofkt*)h;
    for (int64_t i = 0; i < f->nnodes; ++i) {
        onode* n = &f->nodes[i];
        begin[i] = n->begin; end[i] = n->end; level[i] = n->level; leaf[i] = n->leaf;
        child[2 * i] = n->child[0]; child[2 * i + 1] = n->child[1];
        for (int a = 0; a < f->d; ++a) centre[i * f->d + a] = n->c[a];
        rho2[i] = n->rho2;
    }
}

void orc_fkt_perm(void* h, int64_t* perm, uint64_t* codes, double* lo_L) {
    ofkt* f = (ofkt*)h;
    memcpy(perm, f->perm, sizeof(int64_t) * f->N);
    memcpy(codes, f->code, sizeof(uint64_t) * f->N);
    for (int a = 0; a < f->d; ++a) lo_L[a] = f->lo[a];
    lo_L[f->d] = f->L;
}

/* The far-field acceptance criterion (eq. accparam) for a point and a node:
 * rho_b / |x - c_b| < theta, evaluated as rho_b^2 < theta^2 |x - c_b|^2. */
static int is_far(const ofkt* f, const float* x, const onode* n) {
    double d2 = dist2(x, n->c, f->d);
    return n->rho2 < f->theta2 * d2;
}

/* s2m for every node: M_b = sum_{s in b} w_s * basis(x_s - c_b)  (Algorithm 1, source2mult). */
int orc_fkt_s2m(void* h, const double* W, int nrhs) {
    ofkt* f = (ofkt*)h;
    int d = f->d, nt = f->basis->nterms;
    if (nrhs < 1 || nrhs > 64) return -1;
    free(f->W);
    free(f->M);
    f->nrhs = nrhs;
    f->W = (double*)malloc(sizeof(double) * nrhs * f->N);
    for (int q = 0; q < nrhs; ++q)
        for (int64_t i = 0; i < f->N; ++i) f->W[(size_t)q * f->N + i] = W[(size_t)q * f->N + f->perm[i]];
    f->M = (double*)calloc((size_t)f->nnodes * nrhs * nt, sizeof(double));
    #pragma omp parallel
    {
        double w[64];
        #pragma omp for schedule(dynamic, 1)
        for (int64_t b = 1; b < f->nnodes; ++b) { /* the root is never far from any of its own points */
            onode* n = &f->nodes[b];
            double* M = f->M + (size_t)b * nrhs * nt;
            for (int64_t s = n->begin; s < n->end; ++s) {
                double xp[ORC_MAXD];
                for (int a = 0; a < d; ++a) xp[a] = (double)f->X[s * d + a] - n->c[a];
                for (int q = 0; q < nrhs; ++q) w[q] = f->W[(size_t)q * f->N + s];
                s2m_point(f->basis, xp, w, nrhs, M);
            }
        }
    }
    return 0;
}

/* Per-target traversal: far -> m2t and stop; leaf -> dense near block; else children. */
static void traverse(const ofkt* f, int64_t t, int64_t b, double* z) {
    const onode* n = &f->nodes[b];
    const float* xt = f->X + t * f->d;
    int d = f->d, nt = f->basis->nterms, nrhs = f->nrhs;
    if (is_far(f, xt, n)) {
        double x[ORC_MAXD];
        for (int a = 0; a < d; ++a) x[a] = (double)xt[a] - n->c[a];
        m2t_point(f->basis, &f->ker, x, f->M + (size_t)b * nrhs * nt, nrhs, z);
        return;
    }
    if (n->leaf) {
        int sing = kernel_singular(&f->ker);
        for (int64_t s = n->begin; s < n->end; ++s) {
            double r2 = 0.0;
            for (int a = 0; a < d; ++a) {
                double dx = (double)xt[a] - (double)f->X[s * d + a];
                r2 += dx * dx;
            }
            if (sing && r2 == 0.0) continue;
            double kv = kernel_value(&f->ker, sqrt(r2));
            for (int q = 0; q < nrhs; ++q) z[q] += kv * f->W[(size_t)q * f->N + s];
        }
        return;
    }
    for (int c = 0; c < 2; ++c)
        if (n->child[c] >= 0) traverse(f, t, n->child[c], z);
}

/* z = Ktilde w at the given ORIGINAL target indices; out is [nrhs][nt]. Needs orc_fkt_s2m first. */
int orc_fkt_eval(void* h, const int64_t* targets, int64_t nt, double* out) {
    ofkt* f = (ofkt*)h;
    if (!f->M) return -1;
    int64_t* inv = (int64_t*)malloc(sizeof(int64_t) * f->N);
    for (int64_t i = 0; i < f->N; ++i) inv[f->perm[i]] = i;
    int nrhs = f->nrhs;
    #pragma omp parallel for schedule(dynamic, 8)
    for (int64_t ti = 0; ti < nt; ++ti) {
        double z[64];
        for (int q = 0; q < nrhs; ++q) z[q] = 0.0;
        traverse(f, inv[targets[ti]], 0, z);
        for (int q = 0; q < nrhs; ++q) out[(size_t)q * nt + ti] = z[q];
    }
    free(inv);
    return 0;
}

/* The multipoles of the last orc_fkt_s2m ([node][nrhs][nterms], count = nodes * nrhs * nterms
 * doubles), read out or replaced (accessors only: a test sums per-rank partial multipoles and
 * evaluates with the sum).  Return -1 on a count mismatch or before orc_fkt_s2m. */
int orc_fkt_get_multipoles(void* h, double* out, int64_t count) {
    ofkt* f = (ofkt*)h;
    if (!f->M || count != f->nnodes * (int64_t)f->nrhs * f->basis->nterms) return -1;
    memcpy(out, f->M, sizeof(double) * (size_t)count);
    return 0;
}
int orc_fkt_set_multipoles(void* h, const double* in, int64_t count) {
    ofkt* f = (ofkt*)h;
    if (!f->M || count != f->nnodes * (int64_t)f->nrhs * f->basis->nterms) return -1;
    memcpy(f->M, in, sizeof(double) * (size_t)count);
    return 0;
}

/* Interaction lists of one target (original index): far nodes and near leaves. */
static void lists_rec(const ofkt* f, int64_t t, int64_t b, int64_t* far, int64_t* nf, int64_t* near, int64_t* nn) {
    const onode* n = &f->nodes[b];
    if (is_far(f, f->X + t * f->d, n)) { far[(*nf)++] = b; return; }
    if (n->leaf) { near[(*nn)++] = b; return; }
    for (int c = 0; c < 2; ++c)
        if (n->child[c] >= 0) lists_rec(f, t, n->child[c], far, nf, near, nn);
}

void orc_fkt_target_lists(void* h, int64_t t_orig, int64_t* far, int64_t* nfar, int64_t* near, int64_t* nnear) {
    ofkt* f = (ofkt*)h;
    int64_t t = 0;
    for (int64_t i = 0; i < f->N; ++i) if (f->perm[i] == t_orig) { t = i; break; }
    *nfar = 0;
    *nnear = 0;
    lists_rec(f, t, 0, far, nfar, near, nnear);
}

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
