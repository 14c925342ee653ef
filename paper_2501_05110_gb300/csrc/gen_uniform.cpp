// Build-time generator for the uniform-coefficient kernel (uniform.cu).
//
// When every term coefficient of a problem is one number (a spatial box with uniform U, B, nu; no
// momentum axis), the operator is a sum of Kronecker products: a combined reaction matrix
// R = sum_t c_t K_t, per-axis advection matrices beta_a = U_a 1 + V A^a and their upwind
// matrices |beta_a| (Sec. 2.2, Eq. definitions-advection-reaction-eq; Eq. definition-upwind-flux).
// Their sparsity depends on l_max alone.  This program computes the patterns from the library's
// own coupling tables (sh_tables.cpp, the same code the set-up runs) and writes, for every l_max
// the kernel is built for, straight-line device functions in which every nonzero is one fused
// multiply-add with register operands at compile-time indices and the value read from the kernel's
// parameter block, visiting the columns in turn (one input value live at a time); plus host tables of the (row, column) pairs in the same order, which the set-up
// uses to pack the values and to check that a problem's matrices fit the patterns.
//
// Patterns: R = Om^x u Om^y u Om^z u diagonal; beta_a = A^a u diagonal; |beta_a| = the pattern of
// W_a |Lambda| W_a^T for the eigenvectors W_a of A^a (rotated from W_x as the set-up does) u diagonal.
// Usage: gen_uniform <output file> <l_max> [<l_max> ...]
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <string>
#include <utility>
#include <vector>

#include "sh_tables.h"

using namespace sap;

namespace {

struct Pat {
  std::vector<int> r, c;
};

double max_abs(const Mat& m) {
  double s = 0.0;
  for (double v : m.a) s = std::max(s, std::fabs(v));
  return s;
}

// entries of m above 1e-14 of its largest entry, in row-major order, with the diagonal added
Pat pattern(const std::vector<const Mat*>& ms, int n) {
  std::vector<char> on((size_t)n * n, 0);
  for (const Mat* m : ms) {
    const double cut = 1e-14 * max_abs(*m);
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j)
        if (std::fabs((*m)(i, j)) > cut) on[(size_t)i * n + j] = 1;
  }
  for (int i = 0; i < n; ++i) on[(size_t)i * n + i] = 1;
  Pat p;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      if (on[(size_t)i * n + j]) {
        p.r.push_back(i);
        p.c.push_back(j);
      }
  return p;
}

Mat abs_of(const Mat& W, const std::vector<double>& lam) {
  const int n = W.n;
  Mat out(n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int k = 0; k < n; ++k) s += W(i, k) * std::fabs(lam[k]) * W(j, k);
      out(i, j) = s;
    }
  return out;
}

void emit_host_table(FILE* f, const char* name, const Pat& p) {
  std::fprintf(f, "  static constexpr unsigned char %s[%zu][2] = {", name, p.r.size());
  for (size_t k = 0; k < p.r.size(); ++k) std::fprintf(f, "%s{%d,%d}", k ? "," : "", p.r[k], p.c[k]);
  std::fprintf(f, "};\n");
}

// Column-major emission: the values v[k] keep the row-major order of the pattern (the packing
// order), the code visits the columns in turn so that one column value is live at a time besides the
// accumulators.  col(c) is a callable the kernel passes (it forms the column value from shared memory).
std::vector<std::vector<std::pair<int, size_t>>> by_column(const Pat& p, int n) {
  std::vector<std::vector<std::pair<int, size_t>>> cols(n);
  for (size_t k = 0; k < p.r.size(); ++k) cols[p.c[k]].push_back({p.r[k], k});
  return cols;
}

// acc[r] += v[k] * col(c) for every nonzero k
void emit_matvec(FILE* f, const std::string& fname, const Pat& p, int n) {
  std::fprintf(f,
               "  template <typename T, typename Col>\n  static __device__ __forceinline__ void %s(const T* __restrict__ v, "
               "Col&& col, T (&acc)[%d]) {\n",
               fname.c_str(), n);
  const auto cols = by_column(p, n);
  for (int c = 0; c < n; ++c) {
    if (cols[c].empty()) continue;
    std::fprintf(f, "    { const T xc = col(%d);", c);
    for (auto& e : cols[c]) std::fprintf(f, " acc[%d] = fma(v[%zu], xc, acc[%d]);", e.first, e.second, e.first);
    std::fprintf(f, " }\n");
  }
  std::fprintf(f, "  }\n");
}

// out[r] = sum_k vb[k] S[c] + sum_k va[k] D[c] with sd(c, S_c, D_c) forming column c's pair
void emit_flux(FILE* f, const std::string& fname, const Pat& pb, const Pat& pa, int n) {
  std::fprintf(f,
               "  template <typename T, typename SD>\n  static __device__ __forceinline__ void %s(const T* __restrict__ vb, "
               "const T* __restrict__ va, SD&& sd, T* __restrict__ out) {\n    T J[%d];\n",
               fname.c_str(), n);
  std::fprintf(f, "#pragma unroll\n    for (int r = 0; r < %d; ++r) J[r] = T(0);\n", n);
  const auto cb = by_column(pb, n), ca = by_column(pa, n);
  for (int c = 0; c < n; ++c) {
    std::fprintf(f, "    { T sc, dc; sd(%d, sc, dc);", c);
    for (auto& e : cb[c]) std::fprintf(f, " J[%d] = fma(vb[%zu], sc, J[%d]);", e.first, e.second, e.first);
    for (auto& e : ca[c]) std::fprintf(f, " J[%d] = fma(va[%zu], dc, J[%d]);", e.first, e.second, e.first);
    std::fprintf(f, " }\n");
  }
  std::fprintf(f, "#pragma unroll\n    for (int r = 0; r < %d; ++r) out[r] = J[r];\n  }\n", n);
}

}  // namespace

int main(int argc, char** argv) {
  if (argc < 3) {
    std::fprintf(stderr, "usage: %s <output> <l_max> [...]\n", argv[0]);
    return 2;
  }
  FILE* f = std::fopen(argv[1], "w");
  if (!f) {
    std::perror(argv[1]);
    return 1;
  }
  std::fprintf(f, "// generated by gen_uniform.cpp from the library's coupling tables; do not edit\n#pragma once\n\n");
  std::vector<int> lmaxes;
  for (int i = 2; i < argc; ++i) lmaxes.push_back(std::atoi(argv[i]));
  for (int L : lmaxes) {
    const SHTables Tb = build_sh_tables(L);
    const int n = Tb.n;
    Mat Wx;
    std::vector<double> lam;
    sym_eig_blocks(Tb.A[0], connected_blocks(Tb.A[0]), Wx, lam);
    Mat Wa[3];
    Wa[0] = Wx;
    Wa[1] = matmul(transpose(Tb.Uz), Wx);
    Wa[2] = matmul(transpose(Tb.Ux), Wa[1]);
    const Pat pr = pattern({&Tb.Om[0], &Tb.Om[1], &Tb.Om[2]}, n);
    Pat pb[3], pa[3];
    for (int a = 0; a < 3; ++a) {
      pb[a] = pattern({&Tb.A[a]}, n);
      const Mat ab = abs_of(Wa[a], lam);
      pa[a] = pattern({&ab}, n);
    }
    std::fprintf(f, "template <> struct UniK<%d> {\n", L);
    std::fprintf(f, "  static constexpr int n = %d, nR = %zu, nB0 = %zu, nB1 = %zu, nB2 = %zu, nA0 = %zu, nA1 = %zu, nA2 = %zu;\n",
                 n, pr.r.size(), pb[0].r.size(), pb[1].r.size(), pb[2].r.size(), pa[0].r.size(), pa[1].r.size(),
                 pa[2].r.size());
    emit_host_table(f, "patR", pr);
    for (int a = 0; a < 3; ++a) {
      emit_host_table(f, ("patB" + std::to_string(a)).c_str(), pb[a]);
      emit_host_table(f, ("patA" + std::to_string(a)).c_str(), pa[a]);
    }
    // the diagonal of R (the point-Jacobi diagonal of the reaction part)
    std::fprintf(f, "  template <typename T>\n  static __device__ __forceinline__ void Rdiag(const T* __restrict__ v, T (&d)[%d]) {\n", n);
    for (size_t k = 0; k < pr.r.size(); ++k)
      if (pr.r[k] == pr.c[k]) std::fprintf(f, "    d[%d] = v[%zu];\n", pr.r[k], k);
    std::fprintf(f, "  }\n");
    emit_matvec(f, "R", pr, n);
    for (int a = 0; a < 3; ++a) {
      emit_matvec(f, "B" + std::to_string(a), pb[a], n);
      emit_flux(f, "flux" + std::to_string(a), pb[a], pa[a], n);
    }
    std::fprintf(f, "};\n");
    std::fprintf(f, "\n");
  }
  std::fclose(f);
  return 0;
}
