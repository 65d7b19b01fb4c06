// psf_plan.h -- host planner of the filtered PS scheme (Eqs. 5-6, 24-28,
// 34-37 and Lemma 1).  No CUDA dependency.
#pragma once

#include <vector>

namespace psf {

struct Plan {
    int N = 0, q = 0, b = 1, g = 0, products = 0;
    double alpha10 = 0.0, trunc = 0.0, budget = 0.0;
    std::vector<double> z;      // z_0 .. z_max
    std::vector<double> zeta;   // index k = 2..q
    std::vector<double> sigma;  // index j = 1+g..b-1
    std::vector<double> d;      // d_k (Eq. 24)
};

// Returns 0 on success, 1 if no truncation length exists within the supplied
// coefficients (series mode).  `norms` holds z_0..z_10 (or z_0, z_1 when
// submult).
int make_plan(const std::vector<double>& a, double tol, bool poly, bool submult, int s,
              const double* norms, Plan& p);

}  // namespace psf
