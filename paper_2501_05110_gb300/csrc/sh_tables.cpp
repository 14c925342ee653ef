// Spherical-harmonic coupling matrices of the (l,m,s) system, built on the host in FP64.
//
// Route (independent of any quadrature): the closed forms of A^x and Omega^x (Sec. 2.1,
// Eq. representation-matrix-Ax / -Omegax), the rotation elements exp(pi/2 Omega^z)
// (Eq. representation-matrix-Uz with Eq. complex-rotation) and exp(pi/2 Omega^x), and the
// rotation relations A^y = e^{-pi/2 Om^z} A^x e^{pi/2 Om^z}, A^z = e^{-pi/2 Om^x} A^y e^{pi/2 Om^x}
// (same for Omega) of Eq. real-direction-op-matrices-and-rotations.  All matrices are built for
// L = lmax + 1, multiplied there and cut to n x n (Sec. 2.1, last paragraph).
//
// Readings: the element formula printed for exp(pi/2 Omega^x) is the exponential with the
// opposite sign, exp(-pi/2 Omega^x), of the printed Omega^x; this file uses the exponential of the
// printed Omega^x, i.e. the transpose of the printed element formula.  The sum in
// Eq. complex-rotation runs over every k for which all factorial arguments are non-negative.
#include "sh_tables.h"

#include <cmath>
#include <cstdlib>
#include <vector>

namespace sap {

int sh_index(int l, int m, int s) { return l * (l + 1) + (s == 1 ? 1 : -1) * m; }

void sh_lms(int lmax, std::vector<int>& L, std::vector<int>& M, std::vector<int>& S) {
  int n = (lmax + 1) * (lmax + 1);
  L.assign(n, 0); M.assign(n, 0); S.assign(n, 0);
  for (int l = 0; l <= lmax; ++l)
    for (int m = 0; m <= l; ++m)
      for (int s = 0; s <= (m == 0 ? 0 : 1); ++s) {
        int j = sh_index(l, m, s);
        L[j] = l; M[j] = m; S[j] = s;
      }
}

static double fact(int k) {
  double r = 1.0;
  for (int i = 2; i <= k; ++i) r *= i;
  return r;
}

// u(l,m',l,m) of Eq. complex-rotation (the l' = l part).
static double u_rot(int l, int mp, int m) {
  double tot = 0.0;
  for (int k = 0; k <= 2 * l + 1; ++k) {
    int a1 = l - mp - k, a2 = l - m - k, a3 = mp + m + k;
    if (a1 < 0 || a2 < 0 || a3 < 0) continue;
    double num = std::sqrt(fact(l + mp) * fact(l - mp) * fact(l + m) * fact(l - m));
    tot += ((k & 1) ? -1.0 : 1.0) * num / (fact(k) * fact(a1) * fact(a2) * fact(a3));
  }
  return (((l - mp) & 1) ? -1.0 : 1.0) / std::ldexp(1.0, l) * tot;
}

Mat::Mat(int n_) : n(n_), a((size_t)n_ * n_, 0.0) {}

Mat matmul(const Mat& x, const Mat& y) {
  Mat r(x.n);
  for (int i = 0; i < x.n; ++i)
    for (int k = 0; k < x.n; ++k) {
      double v = x(i, k);
      if (v == 0.0) continue;
      for (int j = 0; j < x.n; ++j) r(i, j) += v * y(k, j);
    }
  return r;
}

Mat transpose(const Mat& x) {
  Mat r(x.n);
  for (int i = 0; i < x.n; ++i)
    for (int j = 0; j < x.n; ++j) r(i, j) = x(j, i);
  return r;
}

static Mat truncate(const Mat& x, int n) {
  Mat r(n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double v = x(i, j);
      r(i, j) = std::fabs(v) < 1e-12 ? 0.0 : v;  // exact entries are 0 or O(1)
    }
  return r;
}

SHTables build_sh_tables(int lmax) {
  const int Lx = lmax + 1;
  const int nL = (Lx + 1) * (Lx + 1);
  std::vector<int> Ls, Ms, Ss;
  sh_lms(Lx, Ls, Ms, Ss);
  Mat Ax(nL), Omx(nL), Ux(nL), Uz(nL);
  for (int i = 0; i < nL; ++i)
    for (int j = 0; j < nL; ++j) {
      int lp = Ls[i], mp = Ms[i], sp = Ss[i], l = Ls[j], m = Ms[j], s = Ss[j];
      if (mp == m && sp == s) {
        if (lp == l + 1) Ax(i, j) = std::sqrt(double((l + m + 1) * (l - m + 1)) / double((2 * l + 3) * (2 * l + 1)));
        if (lp == l - 1) Ax(i, j) = std::sqrt(double((l + m) * (l - m)) / double((2 * l + 1) * (2 * l - 1)));
      }
      if (lp == l && mp == m) {
        double v = 0.0;
        if (sp == 0 && s == 1) v += m / std::sqrt(1.0 + (mp == 0));
        if (sp == 1 && s == 0) v -= m / std::sqrt(1.0 + (m == 0));
        Omx(i, j) = v;
        // exp(pi/2 Omega^x): on each (l,m) pair the generator is m [[0,1],[-1,0]] in (s'=0,1)x(s=0,1),
        // whose exponential is [[cos, sin],[-sin, cos]](m pi/2); m = 0 gives 1.
        double c = std::cos(0.5 * M_PI * m), sn = std::sin(0.5 * M_PI * m);
        if (m == 0) {
          Ux(i, j) = 1.0;
        } else {
          if (sp == 0 && s == 0) Ux(i, j) = c;
          if (sp == 1 && s == 1) Ux(i, j) = c;
          if (sp == 0 && s == 1) Ux(i, j) = sn;
          if (sp == 1 && s == 0) Ux(i, j) = -sn;
        }
      }
      if (lp == l) {
        double upm = u_rot(l, mp, m);
        double umm = u_rot(l, mp, -m);
        double sgn = (m & 1) ? -1.0 : 1.0;
        if (sp == 0 && s == 0) Uz(i, j) = (upm + sgn * umm) / std::sqrt((1.0 + (mp == 0)) * (1.0 + (m == 0)));
        if (sp == 1 && s == 1) Uz(i, j) = upm - sgn * umm;
      }
    }
  Mat UzT = transpose(Uz), UxT = transpose(Ux);
  Mat A[3], Om[3];
  A[0] = Ax;
  Om[0] = Omx;
  A[1] = matmul(UzT, matmul(Ax, Uz));
  Om[1] = matmul(UzT, matmul(Omx, Uz));
  A[2] = matmul(UxT, matmul(A[1], Ux));
  Om[2] = matmul(UxT, matmul(Om[1], Ux));
  SHTables T;
  T.lmax = lmax;
  T.n = (lmax + 1) * (lmax + 1);
  const int n = T.n;
  // E^a = eps_abc A^b Om^c ; AA^{ab} = A^a A^b ; F^{ab} = A^a E^b  (all at L, then cut)
  Mat E[3] = {Mat(nL), Mat(nL), Mat(nL)};
  for (int a = 0; a < 3; ++a) {
    int b = (a + 1) % 3, c = (a + 2) % 3;
    Mat p1 = matmul(A[b], Om[c]), p2 = matmul(A[c], Om[b]);
    for (size_t q = 0; q < p1.a.size(); ++q) E[a].a[q] = p1.a[q] - p2.a[q];
  }
  for (int a = 0; a < 3; ++a) {
    T.A[a] = truncate(A[a], n);
    T.Om[a] = truncate(Om[a], n);
    T.E[a] = truncate(E[a], n);
    for (int b = 0; b < 3; ++b) {
      T.AA[a][b] = truncate(matmul(A[a], A[b]), n);
      T.F[a][b] = truncate(matmul(A[a], E[b]), n);
    }
  }
  T.C = Mat(n);
  std::vector<int> l2, m2, s2;
  sh_lms(lmax, l2, m2, s2);
  for (int i = 0; i < n; ++i) T.C(i, i) = 0.5 * l2[i] * (l2[i] + 1);
  T.Uz = truncate(Uz, n);  // rotations preserve l, so the cut is exact
  T.Ux = truncate(Ux, n);
  return T;
}

// ------------------------------------------------------------------------------------------------
// symmetric eigen-decomposition (cyclic Jacobi), per connected block of the sparsity pattern
// ------------------------------------------------------------------------------------------------
static void jacobi_dense(int m, std::vector<double>& a, std::vector<double>& v, std::vector<double>& w) {
  v.assign((size_t)m * m, 0.0);
  for (int i = 0; i < m; ++i) v[(size_t)i * m + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) {
        double x = a[(size_t)i * m + j] * a[(size_t)i * m + j];
        tot += x;
        if (i != j) off += x;
      }
    if (off <= 1e-32 * tot || off == 0.0) break;
    for (int p = 0; p < m; ++p)
      for (int q = p + 1; q < m; ++q) {
        double apq = a[(size_t)p * m + q];
        if (std::fabs(apq) < 1e-300) continue;
        double app = a[(size_t)p * m + p], aqq = a[(size_t)q * m + q];
        double theta = 0.5 * (aqq - app) / apq;
        double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < m; ++k) {  // A <- A J  (columns p, q)
          double akp = a[(size_t)k * m + p], akq = a[(size_t)k * m + q];
          a[(size_t)k * m + p] = c * akp - s * akq;
          a[(size_t)k * m + q] = s * akp + c * akq;
        }
        for (int k = 0; k < m; ++k) {  // A <- J^T A (rows p, q)
          double apk = a[(size_t)p * m + k], aqk = a[(size_t)q * m + k];
          a[(size_t)p * m + k] = c * apk - s * aqk;
          a[(size_t)q * m + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < m; ++k) {
          double vkp = v[(size_t)k * m + p], vkq = v[(size_t)k * m + q];
          v[(size_t)k * m + p] = c * vkp - s * vkq;
          v[(size_t)k * m + q] = s * vkp + c * vkq;
        }
      }
  }
  w.resize(m);
  for (int i = 0; i < m; ++i) w[i] = a[(size_t)i * m + i];
}

std::vector<std::vector<int>> connected_blocks(const Mat& pattern) {
  const int n = pattern.n;
  std::vector<int> comp(n, -1);
  std::vector<std::vector<int>> out;
  for (int s = 0; s < n; ++s) {
    if (comp[s] >= 0) continue;
    std::vector<int> stack{s}, members;
    comp[s] = (int)out.size();
    while (!stack.empty()) {
      int i = stack.back();
      stack.pop_back();
      members.push_back(i);
      for (int j = 0; j < n; ++j)
        if (comp[j] < 0 && (pattern(i, j) != 0.0 || pattern(j, i) != 0.0)) {
          comp[j] = comp[s];
          stack.push_back(j);
        }
    }
    std::sort(members.begin(), members.end());
    out.push_back(members);
  }
  return out;
}

void sym_eig_blocks(const Mat& x, const std::vector<std::vector<int>>& blocks, Mat& W, std::vector<double>& lam) {
  const int n = x.n;
  W = Mat(n);
  lam.assign(n, 0.0);
  std::vector<double> a, v, w;
  for (const auto& b : blocks) {
    int m = (int)b.size();
    a.assign((size_t)m * m, 0.0);
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) a[(size_t)i * m + j] = 0.5 * (x(b[i], b[j]) + x(b[j], b[i]));
    jacobi_dense(m, a, v, w);
    // eigenvector k of the block goes to column b[k] of W
    for (int k = 0; k < m; ++k) {
      lam[b[k]] = w[k];
      for (int i = 0; i < m; ++i) W(b[i], b[k]) = v[(size_t)i * m + k];
    }
  }
}

}  // namespace sap
