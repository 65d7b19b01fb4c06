// psf_plan.h -- host planner of the filtered PS scheme (Eqs. 5-6, 24-28,
// 34-37 and Lemma 1).  No CUDA dependency.
#pragma once

#include <vector>

namespace psf {

struct Plan {
    int N = 0, q = 0, b = 1, g = 0, products = 0;
    double alpha10 = 0.0, trunc = 0.0, budget = 0.0;
    std::vector<double> z;      // z_0 .. z_max of the matrix the scheme forms powers of
    std::vector<double> zz;     // Eq. (37) for Z itself (equal to z unless stride 2)
    std::vector<double> zeta;   // index k = 2..q
    std::vector<double> sigma;  // index j = 1+g..b-1
    std::vector<double> d;      // d_k (Eq. 24)
};

// Returns 0 on success, 1 if no truncation length exists within the supplied
// coefficients (series mode).  `norms` holds z_0..z_10 (or z_0, z_1 when
// submult).  stride 2 plans the series of the substituted coefficients in
// W = Z^2: z_i of W is z_{2i} of Z.
int make_plan(const std::vector<double>& a, double tol, bool poly, bool submult, int s,
              const double* norms, Plan& p, int stride = 1);

// W = Z^2 substitution: c_k = a_{2k} (even series) or a_{2k+1} (odd series).
// Returns 0 and sets odd, or 1 when both parities have nonzero coefficients;
// all-zero coefficients count as even.
int split_even_odd(const std::vector<double>& a, std::vector<double>& c, bool& odd);

}  // namespace psf
