#pragma once

#include <vector>

namespace hhg {

// Least-squares pseudo-inverse A+ = R^{-1} Q^T of a full-rank m x n matrix
// (m >= n, row-major) by Householder QR; returns n x m row-major.
std::vector<double> lsq_pinv(const std::vector<double>& A, int m, int n);

}  // namespace hhg
