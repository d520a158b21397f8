// Host float64 tables of the generalized multipole expansion (Theorem 3.1).
//
// The radial coefficients are built by composing power series rather than
// from the closed forms of the appendix:
//   K(r sqrt(1+e)) = K(r (1 + s(e))),  s(e) = sqrt(1+e) - 1,
//   K(r (1 + t))   = sum_m J_m t^m,    J_m = K^(m)(r) r^m / m!,
// so the coefficient of e^n is sum_m J_m [e^n] s(e)^m (this is Lemma A.2 with
// the m!/n! scaling absorbed).  With e = (r'/r)^2 - 2 (r'/r) cos g (Sec. 3.3),
// e^n = sum_i binom(n, i) (-2)^i cos^i g (r'/r)^(2n-i), and cos^i g is expanded
// in Gegenbauer polynomials by inverting the triangular matrix of their
// monomial coefficients (the identity of eq. coschange).  Collecting
// C_k(cos g) (r'/r)^j J_m gives
//   That_{k,j,m} = sum_n [e^n] s^m * binom(n, 2n-j) (-2)^(2n-j) A_{k,2n-j}  (= m! Tbar_{k,j,m}).
//
// In d = 2 (alpha = 0, where C_k^alpha vanishes for k >= 1) the zonal functions are the
// Chebyshev T_k instead (the limit C_k^alpha / alpha -> (2/k) T_k, the 2/k folded into the
// change of basis), found the same way from the monomial coefficients of T_k.
//
// The harmonic bases are real solid harmonics normalised so that
// sum_h Y_kh(u) Y_kh(v) = C_k^alpha(u.v) (T_k(u.v) in d = 2) for unit u, v (addition theorem, Sec. A.1):
//   d = 2: Re and Im of (x + i y)^k (one function, 1, at k = 0);
//   d = 3: Pi_l^m(z, r^2) (x + i y)^m with Pi_l^m = N_lm r^(l-m) P_l^(m)(z/r),
//          N_lm = sqrt((2 - [m=0]) (l-m)! / (l+m)!)   (Schmidt semi-normalised);
//   d = 4: nu_kl Q_(k-l)^(l+1)(x4, r^2) S^(3)_lm(x1, x2, x3) with the Gegenbauer
//          chain factor Q_n^(lam) = r^n C_n^lam(x4 / r) and nu_kl from the
//          Gegenbauer norms (Funk-Hecke normalisation).
#include <math.h>
#include <string.h>

#include <vector>

#include "fkt_internal.h"

namespace fkt {
namespace {

typedef long double ld;

ld lfact(int n) {
    ld f = 1;
    for (int i = 2; i <= n; ++i) f *= i;
    return f;
}

ld lbinom(int n, int k) {
    if (k < 0 || k > n) return 0;
    ld b = 1;
    for (int i = 1; i <= k; ++i) b = b * (n - k + i) / i;
    return b;
}

// [e^n] s(e)^m for n, m <= P, s(e) = sqrt(1+e) - 1.
std::vector<std::vector<ld>> sqrt_shift_powers(int P) {
    std::vector<ld> s(P + 1, 0);
    // sqrt(1+e) = sum_i binom(1/2, i) e^i
    ld c = 1;
    for (int i = 1; i <= P; ++i) {
        c = c * (0.5L - (i - 1)) / i;
        s[i] = c;
    }
    std::vector<std::vector<ld>> pw(P + 1, std::vector<ld>(P + 1, 0));
    pw[0][0] = 1;
    for (int m = 1; m <= P; ++m)
        for (int n = 0; n <= P; ++n) {
            ld acc = 0;
            for (int i = 1; i <= n; ++i) acc += s[i] * pw[m - 1][n - i];
            pw[m][n] = acc;
        }
    return pw;  // pw[m][n]
}

// A[k][i]: x^i = sum_k A[k][i] C_k^alpha(x), by inverting the Gegenbauer coefficient matrix;
// with chebyshev set, x^i = sum_k A[k][i] T_k(x) from the Chebyshev coefficient matrix.
std::vector<std::vector<ld>> cos_power_to_gegenbauer(int P, ld alpha, bool chebyshev = false) {
    std::vector<std::vector<ld>> g(P + 1, std::vector<ld>(P + 1, 0));  // g[k][t]: C_k = sum_t g[k][t] x^t
    g[0][0] = 1;
    if (P >= 1) g[1][1] = chebyshev ? 1 : 2 * alpha;
    for (int k = 2; k <= P; ++k)
        for (int t = 0; t <= k; ++t) {
            if (chebyshev) {  // T_k = 2 x T_{k-1} - T_{k-2}
                g[k][t] = -g[k - 2][t] + (t >= 1 ? 2 * g[k - 1][t - 1] : 0);
                continue;
            }
            ld v = -(k + 2 * alpha - 2) * g[k - 2][t];
            if (t >= 1) v += 2 * (k + alpha - 1) * g[k - 1][t - 1];
            g[k][t] = v / k;
        }
    // Solve sum_k A[k][i] g[k][t] = [i == t]: for fixed i this is an upper-triangular system in k.
    std::vector<std::vector<ld>> A(P + 1, std::vector<ld>(P + 1, 0));
    for (int i = 0; i <= P; ++i)
        for (int t = i; t >= 0; --t) {
            ld rhs = (t == i) ? 1 : 0;
            for (int k = t + 1; k <= i; ++k) rhs -= A[k][i] * g[k][t];
            A[t][i] = rhs / g[t][t];
        }
    return A;
}

ld gegenbauer_norm2(int n, ld lam) {
    // int_{-1}^{1} C_n^lam(t)^2 (1-t^2)^(lam-1/2) dt = pi 2^(1-2 lam) Gamma(n+2 lam) / (n! (n+lam) Gamma(lam)^2)
    return (ld)M_PI * powl(2.0L, 1 - 2 * lam) * tgammal(n + 2 * lam) / (lfact(n) * (n + lam) * tgammal(lam) * tgammal(lam));
}

// Host mirror of the device harmonics, used only for the self-check below.
void host_harmonics(int d, int p, const FarTables& T, const double* x, std::vector<double>* out) {
    out->clear();
    if (d == 2) {
        double c = 1, s = 0;  // (x + i y)^k
        out->push_back(1.0);
        for (int k = 1; k <= p; ++k) {
            const double cn = x[0] * c - x[1] * s, sn = x[0] * s + x[1] * c;
            c = cn;
            s = sn;
            out->push_back(c);
            out->push_back(s);
        }
        return;
    }
    double r2_3 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
    double r2 = r2_3 + (d == 4 ? x[3] * x[3] : 0.0);
    std::vector<std::vector<double>> Pi(p + 1, std::vector<double>(p + 1, 0));
    std::vector<double> C(p + 1), S(p + 1);
    C[0] = 1;
    S[0] = 0;
    for (int m = 1; m <= p; ++m) {
        C[m] = x[0] * C[m - 1] - x[1] * S[m - 1];
        S[m] = x[0] * S[m - 1] + x[1] * C[m - 1];
    }
    for (int m = 0; m <= p; ++m) {
        Pi[m][m] = T.hSeed[m];
        if (m + 1 <= p) Pi[m + 1][m] = T.hA[m + 1][m] * x[2] * Pi[m][m];
        for (int l = m + 2; l <= p; ++l) Pi[l][m] = T.hA[l][m] * x[2] * Pi[l - 1][m] - T.hB[l][m] * r2_3 * Pi[l - 2][m];
    }
    auto s3 = [&](int l, std::vector<double>* v) {
        v->push_back(Pi[l][0]);
        for (int m = 1; m <= l; ++m) {
            v->push_back(Pi[l][m] * C[m]);
            v->push_back(Pi[l][m] * S[m]);
        }
    };
    if (d == 3) {
        for (int k = 0; k <= p; ++k) s3(k, out);
        return;
    }
    for (int k = 0; k <= p; ++k)
        for (int l = 0; l <= k; ++l) {
            int n = k - l;
            std::vector<double> Q(n + 1);
            Q[0] = T.gSeed[l];
            if (n >= 1) Q[1] = T.gA[l][1] * x[3] * Q[0];
            for (int t = 2; t <= n; ++t) Q[t] = T.gA[l][t] * x[3] * Q[t - 1] - T.gB[l][t] * r2 * Q[t - 2];
            std::vector<double> v;
            s3(l, &v);
            for (double y : v) out->push_back(Q[n] * y);
        }
}

}  // namespace

int build_far_tables(int d, int p, FarTables* out) {
    if (d < 2 || d > 4) return FKT_ERR_INVALID_ARG;
    if (p < 0 || p > (d <= 3 ? kMaxP3 : kMaxP4)) return FKT_ERR_INVALID_ARG;
    memset(out, 0, sizeof(*out));
    const int P = (d <= 3) ? kMaxP3 : kMaxP4;  // fill the whole table; kernels read what they need
    const ld alpha = d / 2.0L - 1.0L;
    auto pw = sqrt_shift_powers(P);
    auto A = cos_power_to_gegenbauer(P, alpha, d == 2);
    int q = 0;
    for (int k = 0; k <= p; ++k)
        for (int j = k; j <= p; j += 2, ++q)
            for (int m = 0; m <= j; ++m) {
                ld acc = 0;
                for (int n = (j + 1) / 2; n <= j; ++n) {
                    int i = 2 * n - j;
                    if (i < k || (i - k) % 2) continue;
                    acc += pw[m][n] * lbinom(n, i) * powl(-2.0L, i) * A[k][i];
                }
                out->That[q][m] = (float)acc;
            }
    // d = 3 normalised associated-Legendre recurrences
    auto N = [](int l, int m) { return sqrtl((m == 0 ? 1.0L : 2.0L) * lfact(l - m) / lfact(l + m)); };
    for (int m = 0; m <= kMaxP3; ++m) {
        ld df = 1;
        for (int t = 2 * m - 1; t > 1; t -= 2) df *= t;
        out->hSeed[m] = (float)(N(m, m) * df);
        for (int l = m + 1; l <= kMaxP3; ++l) {
            out->hA[l][m] = (float)((ld)(2 * l - 1) / (l - m) * N(l, m) / N(l - 1, m));
            if (l >= m + 2) out->hB[l][m] = (float)((ld)(l + m - 1) / (l - m) * N(l, m) / N(l - 2, m));
        }
    }
    // d = 4 Gegenbauer chain level, lam = l + 1
    for (int l = 0; l <= kMaxP4; ++l) {
        ld lam = l + 1;
        auto nu = [&](int n) {
            int k = l + n;
            ld lamk = 2 * (ld)M_PI * (ld)M_PI / (k + 1);           // |S^3| C_k^1(1) / dim H_k
            ld nh = gegenbauer_norm2(n, lam) * 4 * (ld)M_PI / (2 * l + 1);
            return sqrtl(lamk / nh);
        };
        out->gSeed[l] = (float)nu(0);
        for (int n = 1; l + n <= kMaxP4; ++n) {
            out->gA[l][n] = (float)(nu(n) / nu(n - 1) * 2 * (n + lam - 1) / n);
            if (n >= 2) out->gB[l][n] = (float)(nu(n) / nu(n - 2) * (n + 2 * lam - 2) / n);
        }
    }
    // Self-check of the addition theorem on two fixed unit vectors.
    {
        double u[4] = {0.3, -0.5, 0.7, 0.2}, v[4] = {-0.6, 0.1, 0.4, -0.5};
        double nu = 0, nv = 0, uv = 0;
        for (int a = 0; a < d; ++a) { nu += u[a] * u[a]; nv += v[a] * v[a]; }
        for (int a = 0; a < d; ++a) { u[a] /= sqrt(nu); v[a] /= sqrt(nv); uv += u[a] * v[a]; }
        std::vector<double> Yu, Yv;
        host_harmonics(d, p, *out, u, &Yu);
        host_harmonics(d, p, *out, v, &Yv);
        double Cm2 = 1, Cm1 = (d == 2) ? uv : 2 * (double)alpha * uv;
        size_t off = 0;
        for (int k = 0; k <= p; ++k) {
            double Ck = (k == 0) ? 1.0 : (k == 1) ? Cm1
                      : (d == 2) ? 2 * uv * Cm1 - Cm2
                                 : ((2 * uv * (k + (double)alpha - 1) * Cm1 - (k + 2 * (double)alpha - 2) * Cm2) / k);
            if (k >= 2) { Cm2 = Cm1; Cm1 = Ck; }
            size_t D = (d == 2) ? (size_t)(k == 0 ? 1 : 2) : (d == 3) ? (size_t)(2 * k + 1) : (size_t)((k + 1) * (k + 1));
            double s = 0;
            for (size_t h = 0; h < D; ++h) s += Yu[off + h] * Yv[off + h];
            off += D;
            if (fabs(s - Ck) > 1e-4 * (1 + fabs(Ck))) return FKT_ERR_INTERNAL;
        }
    }
    return FKT_OK;
}

KernelParams make_kernel_params(const fkt_kernel& k) {
    KernelParams p{};
    p.kind = k.kind;
    p.ell = (float)k.lengthscale;
    p.alpha = (float)k.alpha;
    p.scale = (float)k.scale;
    double l = k.lengthscale;
    p.sig = 1.0f;
    switch (k.kind) {
    case FKT_GAUSSIAN:
        p.c1 = (float)(1.0 / (2.0 * l * l));
        p.c2 = (float)(M_LOG2E / (2.0 * l * l));
        p.sig = (float)sqrt(M_LOG2E / (2.0 * l * l));
        break;
    case FKT_EXPONENTIAL: p.c1 = (float)(1.0 / l); p.c2 = (float)(M_LOG2E / l); p.sig = p.c2; break;
    case FKT_MATERN32: p.c1 = (float)(sqrt(3.0) / l); p.c2 = (float)(M_LOG2E * sqrt(3.0) / l); p.sig = p.c2; break;
    case FKT_MATERN52: p.c1 = (float)(sqrt(5.0) / l); p.c2 = (float)(M_LOG2E * sqrt(5.0) / l); p.sig = p.c2; break;
    case FKT_CAUCHY: p.c1 = (float)(1.0 / (l * l)); p.sig = (float)(1.0 / l); break;
    case FKT_RATQUAD: p.c1 = (float)(1.0 / (2.0 * k.alpha * l * l)); p.sig = (float)sqrt(p.c1); break;
    default: break;
    }
    return p;
}

}  // namespace fkt
