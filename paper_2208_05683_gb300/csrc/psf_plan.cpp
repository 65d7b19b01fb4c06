// psf_plan.cpp -- host planner of the filtered PS scheme.
//
// From the coefficients, the tolerance and the norms z_i = ||Z^i||_1
// (i <= 10), compute the truncation length N (Eq. 34), the PS split q, b, g
// (Eq. 6), the truncation bound, and the filtering-norm-thresholds zeta_k
// (baby steps) and sigma_j (giant steps) of Eqs. (24)-(28) and (36).
//
// Floating-point conventions: plain IEEE FP64, this file is compiled with
// contraction off; every sum runs left to right in ascending index order as
// written in the paper; z_i = alpha_10^i above i = 10 (Lemma 1) uses pow().
// With stride 2 the scheme runs on W = Z^2 (even or odd series, the caller
// passes the substituted coefficients and tolerance) and z_i of W is z_{2i}.
#include "psf_plan.h"

#include <cmath>

namespace psf {

namespace {

constexpr int kNormest = 10;  // Eq. (37): exact norms up to ||Z^10||

// Eq. (6); s > 0 overrides q (clamped to N - 1)
void split(int N, int s, int& q, int& b, int& g) {
    if (N <= 1) {
        q = 0;
        b = 1;
        g = 0;
        return;
    }
    if (s > 0) {
        q = s < N - 1 ? s : N - 1;
    } else {
        q = 0;
        while ((long long)(q + 1) * (q + 1) <= (long long)(N - 1)) ++q;  // floor(sqrt(N-1))
    }
    b = (N + q - 1) / q;
    g = (N - q * (b - 1) == 1) ? 1 : 0;
}

// sum_{i=m}^{M-1} |a_i| z_i, zero coefficients skipped
double tail_sum(const std::vector<double>& a, const std::vector<double>& z, int m) {
    double s = 0.0;
    for (size_t i = (size_t)m; i < a.size(); ++i)
        if (a[i] != 0.0) s += std::fabs(a[i]) * z[i];
    return s;
}

}  // namespace

int make_plan(const std::vector<double>& a, double tol, bool poly, bool submult, int s,
              const double* norms, Plan& p, int stride) {
    const int M = (int)a.size();
    const int upto = M > kNormest + 1 ? M : kNormest + 1;
    const int zlen = stride * upto;
    std::vector<double>& zz = p.zz;  // Eq. (37) for Z itself
    zz.assign((size_t)zlen + 1, 0.0);
    if (submult) {
        zz[0] = 1.0;
        for (int i = 1; i <= zlen; ++i) zz[(size_t)i] = std::pow(norms[1], (double)i);
        p.alpha10 = norms[1];
    } else {
        double alpha = 0.0;
        for (int k = 5; k <= kNormest; ++k) {
            double r = std::pow(norms[k], 1.0 / k);
            if (k == 5 || r > alpha) alpha = r;
        }
        p.alpha10 = alpha;
        for (int i = 0; i <= zlen; ++i) zz[(size_t)i] = i <= kNormest ? norms[i] : std::pow(alpha, (double)i);
    }
    // the matrix whose powers the scheme forms: Z (stride 1) or W = Z^2
    // (stride 2), whose ||W^i|| = ||Z^{2i}|| is bounded by z_{2i}
    p.z.assign((size_t)upto + 1, 0.0);
    for (int i = 0; i <= upto; ++i) p.z[(size_t)i] = zz[(size_t)(stride * i)];

    if (poly) {
        p.N = M;
        p.trunc = 0.0;
        p.budget = tol;
    } else {
        int N = -1;
        for (int m = 1; m <= M; ++m)
            if (tail_sum(a, p.z, m) <= 0.5 * tol) {
                N = m;
                break;
            }
        if (N < 0 || N == M) return 1;  // not converged within the supplied terms
        p.N = N;
        p.trunc = tail_sum(a, p.z, N);
        p.budget = tol - p.trunc;
    }
    split(p.N, s, p.q, p.b, p.g);
    const int N = p.N, q = p.q, b = p.b, g = p.g;
    p.products = N <= 2 ? 0 : q + b - 2 - g;
    p.zeta.assign((size_t)q + 2, 0.0);
    p.sigma.assign((size_t)b + 1, 0.0);
    p.d.assign((size_t)q + 2, 0.0);
    if (N < 2) return 0;

    auto coef = [&](int idx) { return (idx < N && idx < M) ? a[(size_t)idx] : 0.0; };
    const int Mp = q + b - 2 - g;
    const std::vector<double>& z = p.z;

    // Eq. (25): ||B_i|| <= sum_j |a_{iq+j}| z_j
    std::vector<double> nB((size_t)b, 0.0), nS((size_t)b, 0.0);
    for (int i = 0; i < b; ++i) {
        double acc = 0.0;
        for (int j = 0; j < q; ++j) acc += std::fabs(coef(i * q + j)) * z[(size_t)j];
        nB[(size_t)i] = acc;
    }
    // Eq. (26)
    nS[0] = nB[(size_t)b - 1];
    for (int i = 1; i < b; ++i) nS[(size_t)i] = nB[(size_t)(b - 1 - i)] + z[(size_t)q] * nS[(size_t)i - 1];

    // Eq. (21): beta_{i,k} = sum_{l=k}^{q-1} |a_{iq+l}| z_{l-k}
    auto beta = [&](int i, int k) {
        double acc = 0.0;
        for (int l = k; l < q; ++l) acc += std::fabs(coef(i * q + l)) * z[(size_t)(l - k)];
        return acc;
    };
    // Eq. (24) and (28)/(36)
    for (int k = 2; k <= q; ++k) {
        double acc = 0.0;
        for (int j = 0; j < b; ++j) {
            double sprev = j >= 1 ? nS[(size_t)j - 1] : 0.0;
            acc += z[(size_t)(q * (b - 1 - j))] * (beta(b - 1 - j, k) + z[(size_t)(q - k)] * sprev);
        }
        p.d[(size_t)k] = acc;
        double den = acc * Mp;
        p.zeta[(size_t)k] = den != 0.0 ? p.budget / den : INFINITY;
    }
    for (int j = 1 + g; j < b; ++j) {
        double den = z[(size_t)(q * (b - 1 - j))] * Mp;
        p.sigma[(size_t)j] = den != 0.0 ? p.budget / den : INFINITY;
    }
    return 0;
}

int split_even_odd(const std::vector<double>& a, std::vector<double>& c, bool& odd) {
    bool even_nz = false, odd_nz = false;
    for (size_t i = 0; i < a.size(); ++i)
        if (a[i] != 0.0) (i % 2 ? odd_nz : even_nz) = true;
    if (even_nz && odd_nz) return 1;
    odd = odd_nz;
    c.clear();
    for (size_t i = odd ? 1 : 0; i < a.size(); i += 2) c.push_back(a[i]);
    return 0;
}

}  // namespace psf
