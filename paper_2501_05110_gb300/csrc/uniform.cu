// Operator apply for problems whose term coefficients are all uniform (a spatial box with uniform
// U, B, nu and no momentum axis; tensor-product cells with k = 2): one thread per node.
//
// With uniform coefficients the discrete operator of Eq. definition-mass-and-dg-matrix is a sum of
// Kronecker products of (l,m,s) coupling matrices with 1-D nodal matrices (Sec. 2.2,
// Eq. definitions-advection-reaction-eq; upwind flux, Eq. definition-upwind-flux):
//   M^-1 D x = R x - sum_a (1/h_a) (beta_a (x) S_a) x + sum_a (1/h_a) lift_a [ beta_a {x} + |beta_a| [x] ]
// with R = sum_t c_t K_t the combined reaction matrix, beta_a = U_a 1 + V A^a and |beta_a| its
// upwind matrix.  The thread of node i keeps the n coefficients of its node in registers; every
// nonzero of R, beta_a, |beta_a| is one FMA whose value comes from the parameter block (the
// sparsity patterns are compiled in, see gen_uniform.cpp).  Phases of one block (C cells):
//   1. stage the block's cells in shared memory (coalesced);
//   2. upwind fluxes: 54 tasks per cell (3 axes x 2 faces x 9 face points), one per axis for 18 of
//      each cell's 27 threads, each forming the traces of the n rows from its own cell (shared memory)
//      and the neighbour (global), then J = beta_a (f_lo + f_hi) + |beta_a| (f_lo - f_hi) into
//      shared memory;
//   3. per node: reaction R x; per axis the volume term -(1/h) beta_a (S x along the axis) and the
//      lift of both faces' J; the fused epilogue (mass inverse is the nodal scaling already in L and S).
// The result equals the row kernel's (apply_rows.cu) up to the order of the sums.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>

#include "kernels_common.cuh"
#include "sap_internal.h"

namespace sap {

template <int L>
struct UniK;
#include "uniform_patterns.inc"  // generated at build time by gen_uniform

namespace {

// threads per block at most (27 per cell) and blocks per SM the registers are sized for: FP32
// 8 cells, three blocks per SM; FP64 4 cells, four blocks per SM
template <typename T>
struct UniLaunch {
  static constexpr int max_threads = sizeof(T) == 8 ? 108 : 216;
  static constexpr int min_blocks = sizeof(T) == 8 ? 4 : 3;
};

template <typename T, int L>
struct UniParams {
  using K = UniK<L>;
  T vR[K::nR];
  T vB0[K::nB0], vB1[K::nB1], vB2[K::nB2];
  T vA0[K::nA0], vA1[K::nA1], vA2[K::nA2];
  T dR[K::n];  // diagonal of R (the point-Jacobi diagonal of the reaction part)
  T S[3][3], B0[3], B1[3], L0[3], L1[3];
  const int* cell_nb;  // [ncell][6]
  const T* cell_invh;  // [ncell][3]
  const T* s000;       // [ncell * 27] or null (uniform s_uni)
  T s_uni;
  int ncell;
  int bc_lo[3], bc_hi[3];
  int active[3];
};

// node index of face point fp (the two other axes) and position j along axis a, k = 2 (3 nodes)
__device__ __forceinline__ int unode(int fp, int j, int a) {
  if (a == 0) return j + fp * 3;
  if (a == 1) return (fp % 3) + j * 3 + (fp / 3) * 9;
  return fp + j * 9;
}
// face point of node i for axis a (node i with its a-index removed)
__device__ __forceinline__ int ufp(int i, int a) {
  if (a == 0) return i / 3;
  if (a == 1) return (i % 3) + 3 * (i / 9);
  return i % 9;
}
// L2 prefetch of [p, p + bytes) by one bulk copy-engine request, trimmed to 16-byte boundaries (the
// rule of cp.async.bulk); a hint only: nothing is read into the SM
__device__ __forceinline__ void prefetch_l2(const void* p, size_t bytes) {
  const uintptr_t a = (reinterpret_cast<uintptr_t>(p) + 15) & ~uintptr_t(15);
  const uintptr_t e = (reinterpret_cast<uintptr_t>(p) + bytes) & ~uintptr_t(15);
  if (e > a) asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a), "r"(unsigned(e - a)) : "memory");
}

// w[j] selected by a runtime j in {0,1,2} without indexing the parameter block
template <typename T>
__device__ __forceinline__ T sel3(const T (&w)[3], int j) {
  return j == 0 ? w[0] : (j == 1 ? w[1] : w[2]);
}

// one upwind-flux task: face (a, s) of local cell lc2 at face point fp
template <typename T, int L, int A>
__device__ __forceinline__ void flux_task(const UniParams<T, L>& P, const T* __restrict__ x, const T* __restrict__ X,
                                          T* __restrict__ F, int cell0, int lc2, int s, int fp) {
  using K = UniK<L>;
  constexpr int n = K::n, NL = 27;
  const int per_cell = n * NL;
  const int c2 = cell0 + lc2;
  const int nb = __ldg(P.cell_nb + c2 * 6 + 2 * A + s);
  const bool cont = nb < 0 && (s ? P.bc_hi[A] : P.bc_lo[A]) == SAP_BC_CONTINUOUS;
  // own trace at this face (B0 lower, B1 upper); the neighbour's trace at the shared face is its
  // upper one (B1) across the lower face and its lower one (B0) across the upper face
  T wo[3], wn[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    wo[q] = s ? P.B1[q] : P.B0[q];
    wn[q] = s ? P.B0[q] : P.B1[q];
  }
  const T* Xo = X + lc2 * per_cell;
  const T* xn = x + (size_t)(nb >= 0 ? nb : c2) * per_cell;  // a missing neighbour reads the own cell
  int nd[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) nd[q] = unode(fp, q, A);
  // column c of the flux: the traces of row c on both sides of the face
  auto sd = [&](int c, T& sc, T& dc) {
    T uo = T(0), un = T(0);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      uo = fma(wo[q], Xo[c * NL + nd[q]], uo);
      un = fma(wn[q], __ldg(xn + c * NL + nd[q]), un);
    }
    if (nb < 0) un = cont ? uo : T(0);
    const T flo = s ? uo : un, fhi = s ? un : uo;
    sc = flo + fhi;
    dc = flo - fhi;
  };
  T* out = F + ((lc2 * 6 + 2 * A + s) * 9 + fp) * n;
  if constexpr (A == 0) K::flux0(P.vB0, P.vA0, sd, out);
  else if constexpr (A == 1) K::flux1(P.vB1, P.vA1, sd, out);
  else K::flux2(P.vB2, P.vA2, sd, out);
}

// volume term and lift of axis A at node i of local cell lc
template <typename T, int L, int A>
__device__ __forceinline__ void node_axis(const UniParams<T, L>& P, const T* __restrict__ Xc, const T* __restrict__ Fc,
                                          int cell, int i, T (&acc)[UniK<L>::n]) {
  using K = UniK<L>;
  constexpr int n = K::n, NL = 27;
  if (!P.active[A]) return;  // uniform over the grid
  const T invh = __ldg(P.cell_invh + cell * 3 + A);
  const int ia = A == 0 ? i % 3 : (A == 1 ? (i / 3) % 3 : i / 9);
  const int fp = ufp(i, A);
  T sw[3];
  {
    const T s0[3] = {P.S[0][0], P.S[0][1], P.S[0][2]};
    const T s1[3] = {P.S[1][0], P.S[1][1], P.S[1][2]};
    const T s2[3] = {P.S[2][0], P.S[2][1], P.S[2][2]};
#pragma unroll
    for (int q = 0; q < 3; ++q) sw[q] = -invh * (ia == 0 ? s0[q] : (ia == 1 ? s1[q] : s2[q]));
  }
  int nd[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) nd[q] = unode(fp, q, A);
  // acc += beta_a z with z = -(1/h) (S x)(node i) along the axis, one column at a time
  auto zf = [&](int c) {
    T v = T(0);
#pragma unroll
    for (int q = 0; q < 3; ++q) v = fma(sw[q], Xc[c * NL + nd[q]], v);
    return v;
  };
  if constexpr (A == 0) K::B0(P.vB0, zf, acc);
  else if constexpr (A == 1) K::B1(P.vB1, zf, acc);
  else K::B2(P.vB2, zf, acc);
  // lift: lower face -L0[ia] J/2h, upper face +L1[ia] J/2h
  const T wl = -T(0.5) * invh * sel3(P.L0, ia), wu = T(0.5) * invh * sel3(P.L1, ia);
  const T* J0 = Fc + ((2 * A) * 9 + fp) * n;
  const T* J1 = Fc + ((2 * A + 1) * 9 + fp) * n;
#pragma unroll
  for (int r = 0; r < n; ++r) acc[r] = fma(wl, J0[r], fma(wu, J1[r], acc[r]));
}

template <typename T, int L>
__global__ void __launch_bounds__(UniLaunch<T>::max_threads, UniLaunch<T>::min_blocks) uniform_kernel(const __grid_constant__ UniParams<T, L> P,
                                                                 const T* __restrict__ x, const Epi<T> E, int C) {
  using K = UniK<L>;
  constexpr int n = K::n, NL = 27;
  if (E.skip && *E.skip) return;  // uniform over the grid
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int per_cell = n * NL;
  T* X = reinterpret_cast<T*>(smem_raw);  // [C][n][27]: the block's cells in their global order
  T* F = X + C * per_cell;                // [C][6 faces][9 face points][n]: J of every face point
  const int cell0 = blockIdx.x * C;
  const int Cv = min(C, P.ncell - cell0);
  const int tid = threadIdx.x;
  const int lc = tid / NL, i = tid - lc * NL;
  const bool valid = lc < Cv;
  const int cell = cell0 + (valid ? lc : 0);
  if (E.erk && E.y0 && tid == 0) {  // the RK4 epilogue reads the FP64 state and accumulator of these cells
    const size_t off = (size_t)cell0 * per_cell, bytes = (size_t)Cv * per_cell * sizeof(double);
    prefetch_l2(E.y0 + off, bytes);
    if (E.erk >= 2) prefetch_l2(E.acc + off, bytes);
  }
  {
    const T* xb = x + (size_t)cell0 * per_cell;
    for (int e = tid; e < Cv * per_cell; e += blockDim.x) X[e] = __ldg(xb + e);
  }
  __syncthreads();
  // upwind fluxes: thread t < 18 Cv takes (local cell, side, face point) = t and does that task for the
  // three axes in turn, so all warps run the same axis's code at a time
  if (tid < 18 * Cv) {
    const int lc2 = tid / 18, sp = tid - lc2 * 18, s = sp / 9, fp = sp - s * 9;
    if (P.active[0]) flux_task<T, L, 0>(P, x, X, F, cell0, lc2, s, fp);
    if (P.active[1]) flux_task<T, L, 1>(P, x, X, F, cell0, lc2, s, fp);
    if (P.active[2]) flux_task<T, L, 2>(P, x, X, F, cell0, lc2, s, fp);
  }
  __syncthreads();
  const T* Xc = X + lc * per_cell;
  T* Fc = F + lc * 6 * 9 * n;
  T acc[n];
  if (valid) {
#pragma unroll
    for (int r = 0; r < n; ++r) acc[r] = T(0);
    K::R(P.vR, [&](int c) { return Xc[c * NL + i]; }, acc);
    node_axis<T, L, 0>(P, Xc, Fc, cell, i, acc);
    node_axis<T, L, 1>(P, Xc, Fc, cell, i, acc);
    node_axis<T, L, 2>(P, Xc, Fc, cell, i, acc);
  }
  __syncthreads();  // every thread has read the fluxes: the cell's flux area takes the results
  if (!valid) return;  // no barrier follows
  // epilogue through shared memory (each thread reads back only what it wrote) in a loop over the
  // rows: one copy of the epilogue's code instead of n
#pragma unroll
  for (int r = 0; r < n; ++r) Fc[r * NL + i] = acc[r];
  const T src = P.s000 ? __ldg(P.s000 + (size_t)cell * NL + i) : P.s_uni;
  const size_t dof = (size_t)cell * per_cell + i;
#pragma unroll 1
  for (int r = 0; r < n; ++r)
    epi_write(E, dof + (size_t)r * NL, Xc[r * NL + i], Fc[r * NL + i], r == 0 ? src : T(0), P.dR[r]);
}

}  // namespace

// ------------------------------------------------------------------------------------------------
// host side: packing the combined matrices, launch
// ------------------------------------------------------------------------------------------------
namespace {

// values of dense m (n x n, row major) at the pattern's (row, column) pairs; false if m has a
// nonzero outside the pattern
template <size_t NZ>
bool pack_pattern(const std::vector<double>& m, int n, const unsigned char (&pat)[NZ][2], std::vector<double>& out) {
  std::vector<char> in((size_t)n * n, 0);
  for (size_t k = 0; k < NZ; ++k) {
    in[(size_t)pat[k][0] * n + pat[k][1]] = 1;
    out.push_back(m[(size_t)pat[k][0] * n + pat[k][1]]);
  }
  for (size_t e = 0; e < (size_t)n * n; ++e)
    if (!in[e] && m[e] != 0.0) return false;
  return true;
}

template <int L>
bool pack_l(const UniDense& u, std::vector<double>& vals) {
  using K = UniK<L>;
  if (u.n != K::n) return false;
  vals.clear();
  bool ok = pack_pattern(u.R, K::n, K::patR, vals);
  ok = ok && pack_pattern(u.B[0], K::n, K::patB0, vals) && pack_pattern(u.B[1], K::n, K::patB1, vals) &&
       pack_pattern(u.B[2], K::n, K::patB2, vals);
  ok = ok && pack_pattern(u.A[0], K::n, K::patA0, vals) && pack_pattern(u.A[1], K::n, K::patA1, vals) &&
       pack_pattern(u.A[2], K::n, K::patA2, vals);
  return ok;
}

template <typename T, int L>
UniParams<T, L> make_params(const OpParams<T>& P) {
  using K = UniK<L>;
  UniParams<T, L> U;
  std::memset(&U, 0, sizeof(U));
  const T* v = static_cast<const T*>(P.uni);
  auto take = [&](T* dst, int cnt) {
    std::memcpy(dst, v, sizeof(T) * cnt);
    v += cnt;
  };
  take(U.vR, K::nR);
  take(U.vB0, K::nB0);
  take(U.vB1, K::nB1);
  take(U.vB2, K::nB2);
  take(U.vA0, K::nA0);
  take(U.vA1, K::nA1);
  take(U.vA2, K::nA2);
  for (int k = 0; k < K::nR; ++k)
    if (K::patR[k][0] == K::patR[k][1]) U.dR[K::patR[k][0]] = U.vR[k];
  for (int j = 0; j < 3; ++j) {
    for (int q = 0; q < 3; ++q) U.S[j][q] = P.S[j][q];
    U.B0[j] = P.B0[j];
    U.B1[j] = P.B1[j];
    U.L0[j] = P.L0[j];
    U.L1[j] = P.L1[j];
  }
  U.cell_nb = P.cell_nb;
  U.cell_invh = P.cell_invh;
  U.s000 = P.s000;
  U.s_uni = P.s_uni;
  U.ncell = P.ncell;
  for (int a = 0; a < 3; ++a) {
    U.bc_lo[a] = P.ax[a].bc_lo;
    U.bc_hi[a] = P.ax[a].bc_hi;
    U.active[a] = P.ax[a].active;
  }
  return U;
}

// cells per block: 27 threads each; shared memory (n x 27 values + 54 n fluxes) x cells
template <typename T, int L>
void uni_config(const OpParams<T>& P, int* cells, size_t* smem) {
  constexpr int n = UniK<L>::n;
  // default from a sweep on the 48^3 box at l_max = 5 (FP32: 1.35 ms at 6 cells, 1.38 at 8 and at 3,
  // 1.51 at 1; FP64: 16.0 ms at 3 cells, 16.8 at 4): three blocks per SM fit the shared memory
  const int cmax = UniLaunch<T>::max_threads / 27;
  const int C = P.uni_cells > 0 ? std::min(P.uni_cells, cmax) : (sizeof(T) == 8 ? 3 : 6);
  *cells = C;
  *smem = (size_t)C * (n * 27 + 54 * n) * sizeof(T);
}

constexpr size_t kUniSmemMax = 200 * 1024;

template <typename T, int L>
cudaError_t launch_l(const OpParams<T>& P, const T* x, const Epi<T>& e, cudaStream_t s) {
  static DeviceMask opted{};
  if (cudaError_t err = smem_opt_in(uniform_kernel<T, L>, (int)kUniSmemMax, opted); err != cudaSuccess) return err;
  int C;
  size_t smem;
  uni_config<T, L>(P, &C, &smem);
  if (smem > kUniSmemMax) return cudaErrorInvalidConfiguration;
  const UniParams<T, L> U = make_params<T, L>(P);
  const int blocks = (P.ncell + C - 1) / C;
  uniform_kernel<T, L><<<blocks, 27 * C, smem, s>>>(U, x, e, C);
  note_launch();
  return cudaGetLastError();
}

}  // namespace

bool uni_supported(int lmax) { return lmax >= 1 && lmax <= 5; }

namespace {
// floating-point operations of one cell (an FMA counts 2): reaction, per axis the derivative along
// the axis, beta_a, the lifts and the 18 face tasks (traces of both sides, sum and difference,
// beta_a and |beta_a|)
template <int L>
double flops_l(const int* active) {
  using K = UniK<L>;
  constexpr int n = K::n;
  const int nb[3] = {K::nB0, K::nB1, K::nB2}, na[3] = {K::nA0, K::nA1, K::nA2};
  double f = 2.0 * 27 * K::nR;
  for (int a = 0; a < 3; ++a) {
    if (!active[a]) continue;
    f += 27.0 * (2.0 * 3 * n + 2.0 * nb[a] + 2.0 * 2 * n);
    f += 18.0 * (2.0 * 6 * n + 2.0 * n + 2.0 * (nb[a] + na[a]));
  }
  return f;
}
}  // namespace

double uni_flops_per_cell(int lmax, const int* active) {
  switch (lmax) {
    case 1: return flops_l<1>(active);
    case 2: return flops_l<2>(active);
    case 3: return flops_l<3>(active);
    case 4: return flops_l<4>(active);
    case 5: return flops_l<5>(active);
    default: return 0.0;
  }
}

bool uni_pack(const UniDense& u, std::vector<double>& vals) {
  switch (u.lmax) {
    case 1: return pack_l<1>(u, vals);
    case 2: return pack_l<2>(u, vals);
    case 3: return pack_l<3>(u, vals);
    case 4: return pack_l<4>(u, vals);
    case 5: return pack_l<5>(u, vals);
    default: return false;
  }
}

template <typename T>
cudaError_t launch_uniform(const OpParams<T>& P, const T* x, const Epi<T>& e, cudaStream_t s) {
  switch (P.uni_L) {
    case 1: return launch_l<T, 1>(P, x, e, s);
    case 2: return launch_l<T, 2>(P, x, e, s);
    case 3: return launch_l<T, 3>(P, x, e, s);
    case 4: return launch_l<T, 4>(P, x, e, s);
    case 5: return launch_l<T, 5>(P, x, e, s);
    default: return cudaErrorInvalidConfiguration;
  }
}

template cudaError_t launch_uniform<double>(const OpParams<double>&, const double*, const Epi<double>&, cudaStream_t);
template cudaError_t launch_uniform<float>(const OpParams<float>&, const float*, const Epi<float>&, cudaStream_t);

}  // namespace sap
