// Host-side FP64 spherical-harmonic coupling matrices and small symmetric eigen-solver.
#pragma once
#include <algorithm>
#include <vector>

namespace sap {

struct Mat {  // dense row-major n x n
  int n = 0;
  std::vector<double> a;
  Mat() = default;
  explicit Mat(int n_);
  double& operator()(int i, int j) { return a[(size_t)i * n + j]; }
  double operator()(int i, int j) const { return a[(size_t)i * n + j]; }
};

Mat matmul(const Mat& x, const Mat& y);
Mat transpose(const Mat& x);

struct SHTables {
  int lmax = 0, n = 0;
  Mat A[3], Om[3], E[3], AA[3][3], F[3][3], C, Ux, Uz;
};

int sh_index(int l, int m, int s);
void sh_lms(int lmax, std::vector<int>& L, std::vector<int>& M, std::vector<int>& S);
SHTables build_sh_tables(int lmax);

// Connected components of the symmetric sparsity pattern of a matrix.
std::vector<std::vector<int>> connected_blocks(const Mat& pattern);
// Eigen-decomposition x = W diag(lam) W^T, computed independently on each block.
void sym_eig_blocks(const Mat& x, const std::vector<std::vector<int>>& blocks, Mat& W, std::vector<double>& lam);

}  // namespace sap
