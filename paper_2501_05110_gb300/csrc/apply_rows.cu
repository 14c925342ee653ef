// Row-per-thread dG operator apply for the compiled shapes (D, q) = (1, 3), (2, 2), (3, 3).
//
// Same operator as the cell-node kernel in operator.cu (Sec. 3: volume term, upwind face flux with
// |beta| = W |Lambda| W^T, diagonal mass matrix of the Gauss-collocated basis), organised so that the
// sparse (l,m,s) couplings cost one table load per nonzero instead of one per nonzero and node:
//
//   thread (cell c, coefficient row r) holds row r of the result at all q^D nodes of the cell in
//   registers.  A coupling matrix K contributes  out[r][:] += coef * sum_k K[r][c_k] f[c_k][:]:  one
//   (column, value) pair from the ELL table, one vectorised shared-memory load of row c_k and q^D
//   fused multiply-adds.  The volume derivative along each axis and the face lifts are unrolled over
//   the nodes with compile-time indices.
//
// Phases of one block (C cells, C n threads):
//   P0  stage the cells' values in shared memory (coalesced), coefficient tables per node / face point
//   P1  reaction terms and the volume term  -sum_a (1/h_a) S (beta^a f)  per row
//   P2  per axis: traces of both faces from the own cell (shared memory) and the two neighbours
//       (global, coalesced over face points), S = f_lo + f_hi and D = f_lo - f_hi per row and point;
//       then per row: J = 1/2 sum_t c_t K_t S + 1/2 |beta| D  and the lift into the row's nodes
//   P3  the row results go through shared memory to a coalesced epilogue (the same fused epilogue as
//       the cell-node kernel: CN right-hand side, Jacobi scaling, ERK stage bookkeeping).
//
// Every global load uses an address inside its allocation also where a guard discards the value
// (a missing neighbour reads the own cell, a point without a momentum-face slot reads slot 0).
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>

#include "kernels_common.cuh"

namespace sap {

namespace {

__host__ __device__ constexpr int ipow(int b, int e) { return e == 0 ? 1 : b * ipow(b, e - 1); }

template <typename T, int D, int Q>
struct Shape {
  static constexpr int NL = ipow(Q, D);       // nodes per cell
  static constexpr int NF = ipow(Q, D - 1);   // points per face
  static constexpr int VEC = 16 / (int)sizeof(T);
  static constexpr int NLP = (NL + VEC - 1) / VEC * VEC;  // padded row strides (16-byte rows)
  static constexpr int NFP = (NF + VEC - 1) / VEC * VEC;
  static constexpr int MAXT = (sizeof(T) == 8 && D == 3) ? 256 : 512;  // threads per block
};

// f(integral_constant<A>) for A = A0 .. A1-1 (axis loops with compile-time axis)
template <int A0, int A1, typename F>
__device__ __forceinline__ void static_for(F&& f) {
  if constexpr (A0 < A1) {
    f(std::integral_constant<int, A0>{});
    static_for<A0 + 1, A1>(f);
  }
}

// node index from a face point (axis a removed) and the position j along a
template <int Q>
__device__ __forceinline__ int node_of(int fp, int j, int a) {
  if (a == 0) return j + fp * Q;
  if (a == 1) return (fp % Q) + j * Q + (fp / Q) * Q * Q;
  return (fp % (Q * Q)) + j * Q * Q + (fp / (Q * Q)) * Q * Q * Q;
}

// a / d for 0 <= a < 2^16 and 1 <= d <= 2^16: multiply by ceil(2^32 / d) and keep the high word
// (the rounding error a (ceil(2^32/d) - 2^32/d) / 2^32 < 2^-16 <= 1/d cannot reach the next integer)
struct FastDiv {
  unsigned m;
  int d;
  __device__ explicit FastDiv(int d_) : m(d_ > 1 ? 0xFFFFFFFFu / unsigned(d_) + 1u : 0u), d(d_) {}
  __device__ __forceinline__ int operator()(int a) const { return d > 1 ? int(__umulhi(unsigned(a), m)) : a; }
};

__device__ __forceinline__ void ell_get(const void* base, int idx, int& c, float& v) {
  const int2 e = __ldg(reinterpret_cast<const int2*>(base) + idx);
  c = e.x;
  v = __int_as_float(e.y);
}
__device__ __forceinline__ void ell_get(const void* base, int idx, int& c, double& v) {
  const int4 e = __ldg(reinterpret_cast<const int4*>(base) + idx);
  c = e.x;
  v = __hiloint2double(e.w, e.z);
}

// NP consecutive values from 16-byte aligned shared memory
template <int NP>
__device__ __forceinline__ void ldv(const float* p, float (&v)[NP]) {
#pragma unroll
  for (int k = 0; k < NP / 4; ++k) {
    const float4 w = reinterpret_cast<const float4*>(p)[k];
    v[4 * k] = w.x;
    v[4 * k + 1] = w.y;
    v[4 * k + 2] = w.z;
    v[4 * k + 3] = w.w;
  }
}
template <int NP>
__device__ __forceinline__ void ldv(const double* p, double (&v)[NP]) {
#pragma unroll
  for (int k = 0; k < NP / 2; ++k) {
    const double2 w = reinterpret_cast<const double2*>(p)[k];
    v[2 * k] = w.x;
    v[2 * k + 1] = w.y;
  }
}

// acc[:] += sum_k K[r][c_k] rows[c_k][:]   (rows: [n][NP] in shared memory; K = I for MAT_I)
template <typename T, int N, int NP>
__device__ __forceinline__ void ell_apply(const Bank<T>& B, int mat, int r, int n, const T* rows, T (&acc)[N]) {
  if (mat == MAT_I) {
    T v[NP];
    ldv<NP>(rows + r * NP, v);
#pragma unroll
    for (int i = 0; i < N; ++i) acc[i] += v[i];
    return;
  }
  const int w = B.ell_w[mat];
  int idx = B.ell_off[mat] + r;
#pragma unroll 2
  for (int k = 0; k < w; ++k, idx += n) {
    int c;
    T v;
    ell_get(B.ell, idx, c, v);
    T f[NP];
    ldv<NP>(rows + c * NP, f);
#pragma unroll
    for (int i = 0; i < N; ++i) acc[i] += v * f[i];
  }
}

// the same with every entry multiplied by s
template <typename T, int N, int NP>
__device__ __forceinline__ void ell_apply_scaled(const Bank<T>& B, int mat, int r, int n, const T* rows, T s,
                                                 T (&acc)[N]) {
  if (mat == MAT_I) {
    T v[NP];
    ldv<NP>(rows + r * NP, v);
#pragma unroll
    for (int i = 0; i < N; ++i) acc[i] += s * v[i];
    return;
  }
  const int w = B.ell_w[mat];
  int idx = B.ell_off[mat] + r;
#pragma unroll 2
  for (int k = 0; k < w; ++k, idx += n) {
    int c;
    T v;
    ell_get(B.ell, idx, c, v);
    v *= s;
    T f[NP];
    ldv<NP>(rows + c * NP, f);
#pragma unroll
    for (int i = 0; i < N; ++i) acc[i] += v * f[i];
  }
}

// acc[:] += coef[:] .* (K rows)[r][:], with a single coefficient when it is the same at every node
template <typename T, int N, int NP>
__device__ __forceinline__ void term_apply(const Bank<T>& B, int mat, bool uni, const T* coef, int r, int n,
                                           const T* rows, T (&acc)[N]) {
  if (uni) {
    ell_apply_scaled<T, N, NP>(B, mat, r, n, rows, coef[0], acc);
    return;
  }
  T tmp[N];
#pragma unroll
  for (int i = 0; i < N; ++i) tmp[i] = T(0);
  ell_apply<T, N, NP>(B, mat, r, n, rows, tmp);
  T cv[NP];
  ldv<NP>(coef, cv);
#pragma unroll
  for (int i = 0; i < N; ++i) acc[i] += cv[i] * tmp[i];
}

template <typename T>
__host__ __device__ inline void term_counts(const OpParams<T>& P, int* nvt, int* nadvmax, bool* eigen) {
  int v = P.nreact, m = 0;
  bool e = false;
  for (int a = 0; a < P.D; ++a) {
    v += P.ax[a].nadv;
    m = P.ax[a].nadv > m ? P.ax[a].nadv : m;
    if (P.ax[a].active && P.ax[a].route == ABS_EIGEN) e = true;
  }
  *nvt = v;
  *nadvmax = m;
  *eigen = e;
}

// shared-memory elements of T for C cells (the carve of rows_body)
template <typename T, int D, int Q>
__host__ __device__ inline int rows_smem_elems(const OpParams<T>& P, int C) {
  using S = Shape<T, D, Q>;
  int nvt, nadvmax;
  bool eigen;
  term_counts(P, &nvt, &nadvmax, &eigen);
  const int n = P.n;
  const int fsz = C * n * S::NFP;
  const int acc = (C * n * S::NL + S::VEC - 1) / S::VEC * S::VEC;
  const int freg = (eigen ? 6 : 4) * fsz > acc ? (eigen ? 6 : 4) * fsz : acc;
  // + per cell: a 64-bit mask of the volume / reaction terms and one mask per face of the advection
  // terms whose coefficient is nonzero somewhere in the cell
  const int masks = (C * (2 + 2 * D) * 4 + (int)sizeof(T) - 1) / (int)sizeof(T);
  return C * n * S::NLP + freg + C * nvt * S::NLP + C * 2 * D * nadvmax * S::NFP + masks;
}

// Coefficient of term tt (reaction terms first, then the advection terms axis by axis) at node ii of
// cell c2: scale x spatial field at the node's spatial point x momentum factor at its momentum node
// (x nu for the collision term).
template <typename T, int D, int Q>
__device__ __forceinline__ T node_coef(const OpParams<T>& P, int c2, int tt, int ii) {
  using S = Shape<T, D, Q>;
  constexpr int NL = S::NL, NF = S::NF;
  const int has_mom = P.has_mom;
  const int qdx = has_mom ? NF : NL;
  const Term* tm;
  if (tt < P.nreact) {
    tm = &P.react[tt];
  } else {
    int a = 0, off = P.nreact;
    while (a + 1 < D && tt >= off + P.ax[a].nadv) off += P.ax[a++].nadv;
    tm = &P.ax[a].adv[tt - off];
  }
  const int scell = __ldg(P.cell_scell + c2), pcell = __ldg(P.cell_pcell + c2);
  const int sp = scell * qdx + (has_mom ? ii % NF : ii);
  const int pn = has_mom ? pcell * Q + ii / NF : 0;
  T c = T(tm->scale) * spatial_factor(P, tm->sf, sp) * mom_node(P, tm->mf, pn);
  if (tm->nu) c *= P.nu ? P.nu[(size_t)c2 * NL + ii] : P.nu_uni;
  return c;
}

// Coefficient of advection term tt of axis f / 2 on face f of cell c2 at face point fp (0 for an
// inactive axis or a term index beyond the axis's terms).
template <typename T, int D, int Q>
__device__ __forceinline__ T face_coef(const OpParams<T>& P, int c2, int f, int tt, int fp) {
  using S = Shape<T, D, Q>;
  constexpr int NL = S::NL, NF = S::NF;
  const int has_mom = P.has_mom;
  const int qdx = has_mom ? NF : NL;
  const int qsp = has_mom ? NF / Q : NF;
  const int a = f >> 1, side = f & 1;
  const AxisInfo& A = P.ax[a];
  if (!A.active || tt >= A.nadv) return T(0);
  const int scell = __ldg(P.cell_scell + c2), pcell = __ldg(P.cell_pcell + c2);
  const Term& tm = A.adv[tt];
  T c = T(tm.scale);
  if (A.kind <= SAP_AXIS_Z) {
    // spatial face: U_a at the spatial face point, momentum factor at the point's p
    const int fsp = has_mom ? fp % qsp : fp;
    if (tm.sf == SF_U + a) {
      const int fb = __ldg(P.scell_face + scell * 2 * P.dx + 2 * a + side);
      c *= P.uface_is_uni[a] ? P.uface_uni[a] : P.uface[a][fb + fsp];
    } else {
      c *= spatial_factor(P, tm.sf, scell * qdx);  // only SF_ONE occurs here
    }
    c *= mom_node(P, tm.mf, has_mom ? pcell * Q + fp / qsp : 0);
  } else {
    // momentum face: spatial factor at the spatial node (fp), momentum at the face
    c *= spatial_factor(P, tm.sf, scell * qdx + fp);
    c *= mom_face(P, tm.mf, pcell + side);
  }
  return c;
}

// TRANS = false: y = L x.  TRANS = true: y = L^T x, the transpose of the nodal operator, term by term:
// transposed couplings; volume -(1/h) beta^a (S^T x along the axis); faces g = (lift-weighted traces
// of x from both cells, each with its own 1/h), then beta+ g distributed to the lower cell (its upper
// face) and beta- g to the upper cell, beta+- = (beta +- |beta|)/2 (beta at a continuous boundary).
template <typename T, int D, int Q, bool TRANS>
__device__ __forceinline__ void rows_body(const OpParams<T>& P, const T* __restrict__ x, const Epi<T>& E, int C,
                                          int cell0, int64_t doff, unsigned char* smem_raw) {
  using S = Shape<T, D, Q>;
  constexpr int NL = S::NL, NF = S::NF, NLP = S::NLP, NFP = S::NFP, NFACE = 2 * D;
  if (E.skip && *E.skip) return;  // uniform over the grid
  T* sm = reinterpret_cast<T*>(smem_raw);
  x += doff;
  const int n = P.n;
  const int per_cell = n * NL;
  const int nthr = C * n;
  const int tid = threadIdx.x;
  const FastDiv divn(n);
  const int lc = divn(tid);  // thread = lc n + r: cell lc of the block, coefficient row r
  const int r = tid - lc * n;
  const int Cv = min(C, P.ncell - cell0);
  const bool valid = lc < Cv;
  const int cell = cell0 + (valid ? lc : 0);  // an existing cell also for idle threads (table reads)
  const int has_mom = P.has_mom;
  int nvt, nadvmax;
  bool eigen;
  term_counts(P, &nvt, &nadvmax, &eigen);
  int adv_off[D];
  {
    int o = P.nreact;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      adv_off[a] = o;
      o += P.ax[a].nadv;
    }
  }
  // shared memory carve (rows_smem_elems)
  const int fsz = C * n * NFP;
  const int accsz = (C * n * NL + S::VEC - 1) / S::VEC * S::VEC;
  const int freg = (eigen ? 6 : 4) * fsz > accsz ? (eigen ? 6 : 4) * fsz : accsz;
  T* Fs = sm;                      // [C][n][NLP]   cell values
  T* FR = Fs + C * n * NLP;        // face buffers S0 D0 S1 D1 (Y0 Y1), later the row results
  T* CV = FR + freg;               // [C][nvt][NLP] node coefficients of every term
  T* CF = CV + C * nvt * NLP;      // [C][2D][nadvmax][NFP] face coefficients of the advection terms
  // [C][2 + 2D]: bit tt of words 0-1: term tt (reaction, then advection by axis) has a nonzero node
  // coefficient in the cell; bit t of word 2 + f: advection term t has a nonzero coefficient on face f.
  // A term that is zero on the whole cell adds nothing and is skipped (shock cells away from the
  // velocity gradient, where the momentum terms' FP32 coefficients underflow to zero).  FP32 only:
  // FP64 coefficients of these terms stay nonzero and the bookkeeping would cost more than it saves.
  constexpr bool kMask = sizeof(T) == 4;
  constexpr int MKS = 2 + NFACE;
  unsigned* MK = reinterpret_cast<unsigned*>(CF + C * NFACE * nadvmax * NFP);
  // P0 reads the coefficients from the per-cell tables built at sap_set_fields when they exist
  const bool tab = P.cvtab != nullptr;  // uniform over the grid
  if (kMask && !tab) {
    for (int k = tid; k < C * MKS; k += blockDim.x) MK[k] = 0u;
    __syncthreads();
  }
  const int qdx = has_mom ? NF : NL;           // spatial nodes per cell

  // ---- P0 ---------------------------------------------------------------------------------------
  {
    const int64_t base = (int64_t)cell0 * per_cell;
    for (int e = tid; e < Cv * per_cell; e += blockDim.x) {
      const int R = e / NL;
      Fs[R * NLP + (e - R * NL)] = x[base + e];
    }
    if (tab) {
      const T* cvt = P.cvtab + (size_t)cell0 * nvt * NL;
      for (int w = tid; w < Cv * nvt * NL; w += blockDim.x) {
        const int q1 = w / NL;
        CV[q1 * NLP + (w - q1 * NL)] = __ldg(cvt + w);
      }
      const T* cft = P.cftab + (size_t)cell0 * NFACE * nadvmax * NF;
      for (int w = tid; w < Cv * NFACE * nadvmax * NF; w += blockDim.x) {
        const int q1 = w / NF;
        CF[q1 * NFP + (w - q1 * NF)] = __ldg(cft + w);
      }
      if constexpr (kMask)
        for (int k = tid; k < C * MKS; k += blockDim.x) MK[k] = k < Cv * MKS ? __ldg(P.mktab + (size_t)cell0 * MKS + k) : 0u;
    } else {
      const FastDiv divt(nvt);
      for (int w = tid; w < Cv * nvt * NL; w += blockDim.x) {
        const int q1 = w / NL, ii = w - q1 * NL;  // q1 = lc2 nvt + tt
        const int lc2 = divt(q1), tt = q1 - lc2 * nvt;
        const T c = node_coef<T, D, Q>(P, cell0 + lc2, tt, ii);
        CV[q1 * NLP + ii] = c;
        if (kMask && c != T(0)) {
          unsigned* m = MK + lc2 * MKS + (tt >> 5);
          const unsigned bit = 1u << (tt & 31);
          if (!(*m & bit)) atomicOr(m, bit);
        }
      }
      if (nadvmax > 0) {
        const FastDiv diva(nadvmax);
        for (int w = tid; w < Cv * NFACE * nadvmax * NF; w += blockDim.x) {
          const int q1 = w / NF, fp = w - q1 * NF;  // q1 = (lc2 NFACE + f) nadvmax + tt
          const int q2 = diva(q1), tt = q1 - q2 * nadvmax;
          const int lc2 = q2 / NFACE, f = q2 - lc2 * NFACE;
          const AxisInfo& A = P.ax[f >> 1];
          if (!A.active || tt >= A.nadv) continue;
          const T c = face_coef<T, D, Q>(P, cell0 + lc2, f, tt, fp);
          CF[q1 * NFP + fp] = c;
          if (kMask && c != T(0)) {
            unsigned* m = MK + lc2 * MKS + 2 + f;
            if (!(*m & (1u << tt))) atomicOr(m, 1u << tt);
          }
        }
      }
    }
  }
  __syncthreads();

  // ---- P1: reaction and volume terms --------------------------------------------------------------
  T acc[NL];
#pragma unroll
  for (int i = 0; i < NL; ++i) acc[i] = T(0);
  const T* Fc = Fs + lc * n * NLP;
  const T* CVc = CV + lc * nvt * NLP;
  const unsigned mlo = kMask ? MK[lc * MKS] : ~0u, mhi = kMask ? MK[lc * MKS + 1] : ~0u;
  auto live = [&](int tt) { return ((tt < 32 ? mlo >> tt : mhi >> (tt - 32)) & 1u) != 0u; };
  if (valid) {
    for (int t = 0; t < P.nreact; ++t) {
      if (((P.react_zero >> t) & 1u) || !live(t)) continue;  // zero coefficient (everywhere, or in the cell)
      term_apply<T, NL, NLP>(P.bank, TRANS ? P.react[t].matT : P.react[t].mat, (P.react_uni >> t) & 1u, CVc + t * NLP,
                             r, n, Fc, acc);
    }
  }
  if constexpr (TRANS) {
    // volume: z = S^T x along the axis for every row (shared memory), then -(1/h) sum_t c_t K_t^T z
    static_for<0, D>([&](auto ac) {
      constexpr int a = decltype(ac)::value;
      const AxisInfo& A = P.ax[a];
      if (!A.active) return;  // uniform over the block
      constexpr int qa = ipow(Q, a);
      T* Z = FR;  // [C][n][NLP], free until the faces
      if (valid) {
        T z[NLP];
#pragma unroll
        for (int i = 0; i < NLP; ++i) z[i] = T(0);
#pragma unroll
        for (int i = 0; i < NL; ++i) {
          const int ia = (i / qa) % Q;
          const int b = i - ia * qa;
#pragma unroll
          for (int qq = 0; qq < Q; ++qq) z[i] += P.S[qq][ia] * Fc[r * NLP + b + qq * qa];
        }
#pragma unroll
        for (int i = 0; i < NLP; ++i) Z[(lc * n + r) * NLP + i] = z[i];
      }
      __syncthreads();
      if (valid) {
        T g[NL];
#pragma unroll
        for (int i = 0; i < NL; ++i) g[i] = T(0);
        for (int t = 0; t < A.nadv; ++t) {
          if (((P.adv_zero[a] >> t) & 1u) || !live(adv_off[a] + t)) continue;
          term_apply<T, NL, NLP>(P.bank, A.adv[t].matT, (P.adv_uni[a] >> t) & 1u, CVc + (adv_off[a] + t) * NLP, r, n,
                                 Z + lc * n * NLP, g);
        }
        const T invh = __ldg(P.cell_invh + cell * D + a);
#pragma unroll
        for (int i = 0; i < NL; ++i) acc[i] -= invh * g[i];
      }
      __syncthreads();  // Z is reused by the next axis and the faces
    });
  } else if (valid) {
    static_for<0, D>([&](auto ac) {
      constexpr int a = decltype(ac)::value;
      const AxisInfo& A = P.ax[a];
      if (!A.active) return;
      T g[NL];
#pragma unroll
      for (int i = 0; i < NL; ++i) g[i] = T(0);
      for (int t = 0; t < A.nadv; ++t) {
        if (((P.adv_zero[a] >> t) & 1u) || !live(adv_off[a] + t)) continue;
        term_apply<T, NL, NLP>(P.bank, A.adv[t].mat, (P.adv_uni[a] >> t) & 1u, CVc + (adv_off[a] + t) * NLP, r, n,
                               Fc, g);
      }
      const T invh = __ldg(P.cell_invh + cell * D + a);
      constexpr int qa = ipow(Q, a);
#pragma unroll
      for (int i = 0; i < NL; ++i) {
        const int ia = (i / qa) % Q;
        const int b = i - ia * qa;
        T ds = T(0);
#pragma unroll
        for (int qq = 0; qq < Q; ++qq) ds += P.S[ia][qq] * g[b + qq * qa];
        acc[i] -= invh * ds;
      }
    });
  }

  // ---- P2: faces, one axis at a time ---------------------------------------------------------------
  static_for<0, D>([&](auto ac) {
    constexpr int a = decltype(ac)::value;
    const AxisInfo& A = P.ax[a];
    if (!A.active) return;  // uniform over the block
    T* S0 = FR;
    T* D0 = FR + fsz;
    T* S1 = FR + 2 * fsz;
    T* D1 = FR + 3 * fsz;
    T* Y0 = FR + 4 * fsz;
    T* Y1 = FR + 5 * fsz;
    // P2a: traces.  Item (row R = lc2 n + c, point fp), fp fastest: neighbour reads are coalesced.
    if (tid < nthr) {
#pragma unroll
      for (int k = 0; k < NF; ++k) {
        const int it = tid + k * nthr;
        const int R = it / NF, fp = it - R * NF;
        const int lc2 = divn(R), c = R - lc2 * n;
        if (lc2 >= Cv) continue;
        const int c2 = cell0 + lc2;
        const T* own = Fs + R * NLP;
        T tr0 = T(0), tr1 = T(0);
#pragma unroll
        for (int j = 0; j < Q; ++j) {
          const T v = own[node_of<Q>(fp, j, a)];
          tr0 += P.B0[j] * v;
          tr1 += P.B1[j] * v;
        }
        const int nbl = __ldg(P.cell_nb + c2 * NFACE + 2 * a);
        const int nbh = __ldg(P.cell_nb + c2 * NFACE + 2 * a + 1);
        // a missing neighbour (boundary) reads the own cell and the value is replaced below
        const T* xl = x + (size_t)(nbl >= 0 ? nbl : c2) * per_cell + c * NL;
        const T* xh = x + (size_t)(nbh >= 0 ? nbh : c2) * per_cell + c * NL;
        if constexpr (TRANS) {
          // g = lift-weighted traces of both cells at the face, each with its own 1/h:
          // lower face g = (1/h_lo) L1^T x_lo - (1/h) L0^T x, upper face g = (1/h) L1^T x - (1/h_hi) L0^T x_hi
          T ol = T(0), oh = T(0), gl = T(0), gh = T(0);
#pragma unroll
          for (int j = 0; j < Q; ++j) {
            const T v = own[node_of<Q>(fp, j, a)];
            ol += P.L0[j] * v;
            oh += P.L1[j] * v;
            gl += P.L1[j] * __ldg(xl + node_of<Q>(fp, j, a));
            gh += P.L0[j] * __ldg(xh + node_of<Q>(fp, j, a));
          }
          const T ih = __ldg(P.cell_invh + c2 * D + a);
          const T ihl = nbl >= 0 ? __ldg(P.cell_invh + nbl * D + a) : T(0);  // a missing side adds nothing
          const T ihh = nbh >= 0 ? __ldg(P.cell_invh + nbh * D + a) : T(0);
          S0[R * NFP + fp] = ihl * gl - ih * ol;
          S1[R * NFP + fp] = ih * oh - ihh * gh;
          (void)tr0;
          (void)tr1;
        } else {
          T tl = T(0), th = T(0);
#pragma unroll
          for (int j = 0; j < Q; ++j) {
            tl += P.B1[j] * __ldg(xl + node_of<Q>(fp, j, a));
            th += P.B0[j] * __ldg(xh + node_of<Q>(fp, j, a));
          }
          if (nbl < 0) tl = A.bc_lo == SAP_BC_CONTINUOUS ? tr0 : T(0);
          if (nbh < 0) th = A.bc_hi == SAP_BC_CONTINUOUS ? tr1 : T(0);
          // lower face: f_lo = lower neighbour, f_hi = own; upper face: f_lo = own, f_hi = upper neighbour
          S0[R * NFP + fp] = tl + tr0;
          D0[R * NFP + fp] = tl - tr0;
          S1[R * NFP + fp] = tr1 + th;
          D1[R * NFP + fp] = tr1 - th;
        }
      }
    }
    __syncthreads();
    const int roff = lc * n * NFP;
    if (A.route == ABS_EIGEN) {  // Y = |c0 + lam c1| W^T D  (beta = c0 I + c1 A at the face point)
      if (valid) {
        const T lr = __ldg(P.lam + r);
#pragma unroll
        for (int s = 0; s < 2; ++s) {
          T tmp[NF];
#pragma unroll
          for (int fp = 0; fp < NF; ++fp) tmp[fp] = T(0);
          ell_apply<T, NF, NFP>(P.bank, A.WTmat, r, n, (TRANS ? (s ? S1 : S0) : (s ? D1 : D0)) + roff, tmp);
          const T* c0 = CF + ((lc * NFACE + 2 * a + s) * nadvmax) * NFP;
          const T* c1 = c0 + NFP;
          T* Ys = (s ? Y1 : Y0) + roff + r * NFP;
          if (A.llf) {  // alpha = max over the eigenvalues of |c0 + lam c1|, at an extreme eigenvalue
#pragma unroll
            for (int fp = 0; fp < NF; ++fp)
              Ys[fp] = fmax(fabs(c0[fp] + T(A.lam_lo) * c1[fp]), fabs(c0[fp] + T(A.lam_hi) * c1[fp])) * tmp[fp];
          } else {
#pragma unroll
            for (int fp = 0; fp < NF; ++fp) Ys[fp] = fabs(c0[fp] + lr * c1[fp]) * tmp[fp];
          }
        }
      }
      __syncthreads();
    }
    if (valid) {
      const T h2 = T(0.5) * __ldg(P.cell_invh + cell * D + a);
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const int f = 2 * a + s;
        const T* Ss = (s ? S1 : S0) + roff;
        const T* Ds = TRANS ? Ss : (s ? D1 : D0) + roff;  // the transpose applies |beta| to g as well
        T J[NF];
#pragma unroll
        for (int fp = 0; fp < NF; ++fp) J[fp] = T(0);
        const unsigned fmask = kMask ? MK[lc * MKS + 2 + f] : ~0u;
        for (int t = 0; t < A.nadv; ++t) {
          if (((P.adv_zero[a] >> t) & 1u) || !((fmask >> t) & 1u)) continue;
          T tmp[NF];
#pragma unroll
          for (int fp = 0; fp < NF; ++fp) tmp[fp] = T(0);
          ell_apply<T, NF, NFP>(P.bank, TRANS ? A.adv[t].matT : A.adv[t].mat, r, n, Ss, tmp);
          T cv[NFP];
          ldv<NFP>(CF + ((lc * NFACE + f) * nadvmax + t) * NFP, cv);
#pragma unroll
          for (int fp = 0; fp < NF; ++fp) J[fp] += cv[fp] * tmp[fp];
        }
        T Jc[NF];  // the central part alone (the transpose at a continuous boundary uses all of beta)
        if constexpr (TRANS) {
#pragma unroll
          for (int fp = 0; fp < NF; ++fp) {
            Jc[fp] = J[fp];
            J[fp] = T(0);
          }
        }
        if (A.route == ABS_CONST) {
          ell_apply<T, NF, NFP>(P.bank, A.absmat, r, n, Ds, J);
        } else if (A.route == ABS_EIGEN) {
          ell_apply<T, NF, NFP>(P.bank, A.Wmat, r, n, (s ? Y1 : Y0) + roff, J);
        } else if (P.pabs_ell) {  // ABS_POINT: |beta^p| tabulated per (spatial node, momentum face)
          const int scell = __ldg(P.cell_scell + cell), pcell = __ldg(P.cell_pcell + cell);
          int slot[NF];
          bool any_slot = false;
#pragma unroll
          for (int fp = 0; fp < NF; ++fp) {
            slot[fp] = __ldg(P.pslot + scell * qdx + fp);
            any_slot |= slot[fp] >= 0;
          }
          // a cell none of whose points has a slot (|beta^p| negligible there) adds nothing: skip
          // the loop (most cells of a shock lie away from the velocity gradient)
          const int w = any_slot ? P.bank.ell_w[A.absmat] : 0;
          int idx = P.bank.ell_off[A.absmat] + r;
          const int pf = pcell + s;
          for (int k = 0; k < w; ++k, idx += n) {
            int c;
            T unused;
            ell_get(P.bank.ell, idx, c, unused);
            T dv[NFP];
            ldv<NFP>(Ds + c * NFP, dv);
#pragma unroll
            for (int fp = 0; fp < NF; ++fp) {
              // points without a slot read slot 0 and add nothing
              const int sl = slot[fp] >= 0 ? slot[fp] : 0;
              const T v = __ldg(P.pabs_ell + (((size_t)sl * P.npface + pf) * w + k) * n + r);
              J[fp] += slot[fp] >= 0 ? v * dv[fp] : T(0);
            }
          }
        }
        if constexpr (TRANS) {
          // J = beta+ g (upper face) or beta- g (lower face), beta at a continuous boundary; the
          // traces B distribute it into the nodes (the 1/h are inside g)
          const int nb = __ldg(P.cell_nb + cell * NFACE + f);
          const bool cont = nb < 0 && (s ? A.bc_hi : A.bc_lo) == SAP_BC_CONTINUOUS;
          const T sg = s ? T(0.5) : T(-0.5);
#pragma unroll
          for (int fp = 0; fp < NF; ++fp) {
            const T jt = cont ? Jc[fp] : T(0.5) * Jc[fp] + sg * J[fp];
#pragma unroll
            for (int j = 0; j < Q; ++j) acc[node_of<Q>(fp, j, a)] += (s ? P.B1[j] : P.B0[j]) * jt;
          }
        } else {
          (void)Jc;
          // lift: lower face -L0[j] J, upper face +L1[j] J, times 1/h (the 1/2 of the flux folded in)
#pragma unroll
          for (int fp = 0; fp < NF; ++fp)
#pragma unroll
            for (int j = 0; j < Q; ++j) acc[node_of<Q>(fp, j, a)] += h2 * (s ? P.L1[j] : -P.L0[j]) * J[fp];
        }
      }
    }
    __syncthreads();  // the next axis (or P3) reuses the face buffers
  });

  // ---- P3: row results through shared memory to a coalesced epilogue ------------------------------
  T* Ab = FR;  // [C n][NL], the global order of the block's DoFs
  if (valid) {
#pragma unroll
    for (int i = 0; i < NL; ++i) Ab[tid * NL + i] = acc[i];
  }
  __syncthreads();
  const bool need_rd = E.jacobi || E.out32 || E.outj;
  const size_t dbase = (size_t)doff + (size_t)cell0 * per_cell;
  for (int e = tid; e < Cv * per_cell; e += blockDim.x) {
    const int R = e / NL, i = e - R * NL;
    const int lc2 = divn(R), c = R - lc2 * n;
    T s = T(0);
    if (c == 0) s = P.s000 ? P.s000[(size_t)(cell0 + lc2) * NL + i] : P.s_uni;
    T rd = T(0);
    if (need_rd) {
      if (P.rdtab) {
        rd = __ldg(P.rdtab + (size_t)cell0 * per_cell + e);
      } else {
        for (int t = 0; t < P.nreact; ++t)
          rd += CV[(lc2 * nvt + t) * NLP + i] * csr_diag(P.bank, P.react[t].mat, c, n);
      }
    }
    epi_write(E, dbase + e, Fs[R * NLP + i], Ab[e], s, rd);
  }
}

template <typename T, int D, int Q, bool TRANS>
__global__ void __launch_bounds__(Shape<T, D, Q>::MAXT) rows_kernel(const __grid_constant__ OpParams<T> P,
                                                                   const T* __restrict__ x, const Epi<T> E, int C) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  rows_body<T, D, Q, TRANS>(P, x, E, C, blockIdx.x * C, 0, smem_raw);
}

// Batched: block b works on instance blocks[b].x, cells [blocks[b].y, + cpb[inst]); the instance's
// parameter block is staged in shared memory; blocks of inactive instances return.
template <typename T, int D, int Q>
__global__ void __launch_bounds__(Shape<T, D, Q>::MAXT) rows_kernel_batched(
    const OpParams<T>* __restrict__ Pall, const int64_t* __restrict__ doffs, const int* __restrict__ cpbs,
    const int2* __restrict__ blocks, const int* __restrict__ active, const T* __restrict__ x, const Epi<T> E) {
  __shared__ __align__(16) unsigned char pbuf[sizeof(OpParams<T>)];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int2 bb = blocks[blockIdx.x];
  if (active && !active[bb.x]) return;  // uniform over the block
  const int* src = reinterpret_cast<const int*>(Pall + bb.x);
  int* dst = reinterpret_cast<int*>(pbuf);
  for (int k = threadIdx.x; k < (int)(sizeof(OpParams<T>) / sizeof(int)); k += blockDim.x) dst[k] = src[k];
  __syncthreads();
  rows_body<T, D, Q, false>(*reinterpret_cast<const OpParams<T>*>(pbuf), x, E, cpbs[bb.x], bb.y, doffs[bb.x], smem_raw);
}

// Per-cell coefficient tables of the row kernel (built once per sap_set_fields): the node
// coefficients [cell][term][node], the face coefficients [cell][face][term][point] and the masks of
// the terms that are nonzero somewhere in the cell (FP32 contexts; mktab zeroed by the caller).
template <typename T, int D, int Q>
__global__ void coef_tables_kernel(const __grid_constant__ OpParams<T> P, T* __restrict__ cvtab, T* __restrict__ cftab,
                                   unsigned* __restrict__ mktab, T* __restrict__ rdtab, int nvt, int nadvmax) {
  using S = Shape<T, D, Q>;
  constexpr int NL = S::NL, NF = S::NF, NFACE = 2 * D, MKS = 2 + NFACE;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t ncv = (int64_t)P.ncell * nvt * NL;
  for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < ncv; w += stride) {
    const int64_t q1 = w / NL;
    const int ii = (int)(w - q1 * NL);
    const int c2 = (int)(q1 / nvt), tt = (int)(q1 - (int64_t)c2 * nvt);
    const T c = node_coef<T, D, Q>(P, c2, tt, ii);
    cvtab[w] = c;
    if (mktab && c != T(0)) atomicOr(mktab + (size_t)c2 * MKS + (tt >> 5), 1u << (tt & 31));
  }
  const int64_t ncf = (int64_t)P.ncell * NFACE * nadvmax * NF;
  for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < ncf; w += stride) {
    const int64_t q1 = w / NF;
    const int fp = (int)(w - q1 * NF);
    const int64_t q2 = q1 / nadvmax;
    const int tt = (int)(q1 - q2 * nadvmax);
    const int c2 = (int)(q2 / NFACE), f = (int)(q2 - (int64_t)c2 * NFACE);
    const T c = face_coef<T, D, Q>(P, c2, f, tt, fp);
    cftab[w] = c;
    if (mktab && c != T(0)) atomicOr(mktab + (size_t)c2 * MKS + 2 + f, 1u << tt);
  }
  // the reaction diagonal at every DoF (the point-Jacobi diagonal): sum_t c_t(node) K_t[r][r]
  if (rdtab) {
    const int n = P.n;
    const int64_t N = (int64_t)P.ncell * n * NL;
    for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < N; w += stride) {
      const int64_t R = w / NL;
      const int ii = (int)(w - R * NL);
      const int c2 = (int)(R / n), r = (int)(R - (int64_t)c2 * n);
      T d = T(0);
      for (int t = 0; t < P.nreact; ++t) d += node_coef<T, D, Q>(P, c2, t, ii) * csr_diag(P.bank, P.react[t].mat, r, n);
      rdtab[w] = d;
    }
  }
}

template <typename T, int D, int Q>
cudaError_t coef_tables_shape(OpParams<T>& P, std::vector<DevBuf>& owner, bool with_diag) {
  int nvt, nadvmax;
  bool eigen;
  term_counts(P, &nvt, &nadvmax, &eigen);
  using S = Shape<T, D, Q>;
  const size_t ncv = (size_t)P.ncell * nvt * S::NL, ncf = (size_t)P.ncell * 2 * D * nadvmax * S::NF;
  const size_t nmk = sizeof(T) == 4 ? (size_t)P.ncell * (2 + 2 * D) : 0;
  void* pv = nullptr;
  void* pf = nullptr;
  void* pm = nullptr;
  void* pd = nullptr;
  const size_t nd = with_diag ? (size_t)P.ncell * P.n * S::NL : 0;
  cudaError_t err = cudaMalloc(&pv, sizeof(T) * std::max<size_t>(ncv, 1));
  if (err == cudaSuccess) err = cudaMalloc(&pf, sizeof(T) * std::max<size_t>(ncf, 1));
  if (err == cudaSuccess && nmk) err = cudaMalloc(&pm, sizeof(unsigned) * nmk);
  if (err == cudaSuccess && nd) err = cudaMalloc(&pd, sizeof(T) * nd);
  if (pv) owner.push_back(DevBuf{pv, sizeof(T) * std::max<size_t>(ncv, 1)});
  if (pf) owner.push_back(DevBuf{pf, sizeof(T) * std::max<size_t>(ncf, 1)});
  if (pm) owner.push_back(DevBuf{pm, sizeof(unsigned) * nmk});
  if (pd) owner.push_back(DevBuf{pd, sizeof(T) * nd});
  if (err != cudaSuccess) return err;
  if (nmk && (err = cudaMemset(pm, 0, sizeof(unsigned) * nmk)) != cudaSuccess) return err;
  coef_tables_kernel<T, D, Q><<<1024, 256>>>(P, static_cast<T*>(pv), static_cast<T*>(pf), static_cast<unsigned*>(pm),
                                             static_cast<T*>(pd), nvt, nadvmax);
  note_launch();
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  P.cvtab = static_cast<const T*>(pv);
  P.cftab = static_cast<const T*>(pf);
  P.mktab = static_cast<const unsigned*>(pm);
  P.rdtab = static_cast<const T*>(pd);
  return cudaSuccess;
}

constexpr size_t kRowsSmemMax = 160 * 1024;

template <typename T, int D, int Q>
void rows_config_shape(const OpParams<T>& P, int target, int* cells, size_t* smem) {
  const int maxt = Shape<T, D, Q>::MAXT;
  int C = std::max(1, std::min(target, maxt) / P.n);
  // two blocks per SM where the shared memory allows it
  while (C > 1 && (size_t)rows_smem_elems<T, D, Q>(P, C) * sizeof(T) > 100 * 1024) --C;
  *cells = C;
  *smem = (size_t)rows_smem_elems<T, D, Q>(P, C) * sizeof(T);
}

template <typename T, int D, int Q, bool TRANS>
cudaError_t launch_rows_shape(const OpParams<T>& P, const T* x, const Epi<T>& e, cudaStream_t s) {
  static DeviceMask opted{};
  if (cudaError_t err = smem_opt_in(rows_kernel<T, D, Q, TRANS>, (int)kRowsSmemMax, opted); err != cudaSuccess)
    return err;
  int C;
  size_t smem;
  // threads per block measured best on GB300: FP64 rows need many registers (3-D: ~190), so
  // smaller blocks let more of them share an SM (box 32^3: 5.67 ms at 128 against 6.50 ms at 256;
  // shock: 177 us at 192 against 183 us at 256); FP32: 256
  const int target = sizeof(T) == 8 ? (D == 3 ? 128 : 192) : 256;
  rows_config_shape<T, D, Q>(P, target, &C, &smem);
  if (smem > kRowsSmemMax || C * P.n > Shape<T, D, Q>::MAXT) return cudaErrorInvalidConfiguration;
  const int blocks = (P.ncell + C - 1) / C;
  rows_kernel<T, D, Q, TRANS><<<blocks, C * P.n, smem, s>>>(P, x, e, C);
  note_launch();
  return cudaGetLastError();
}

template <typename T, int D, int Q>
cudaError_t opt_in_rows_batched_shape() {
  static DeviceMask opted{};
  return smem_opt_in(rows_kernel_batched<T, D, Q>, (int)kRowsSmemMax, opted);
}

template <typename T, int D, int Q>
cudaError_t launch_rows_batched_shape(const BatchDev<T>& B, const int* active, const T* x, const Epi<T>& e,
                                      cudaStream_t s) {
  if (cudaError_t err = opt_in_rows_batched_shape<T, D, Q>(); err != cudaSuccess) return err;
  if (B.smem > kRowsSmemMax || B.threads > Shape<T, D, Q>::MAXT) return cudaErrorInvalidConfiguration;
  rows_kernel_batched<T, D, Q><<<B.nblocks, B.threads, B.smem, s>>>(B.P, B.doff, B.cpb, B.blocks, active, x, e);
  note_launch();
  return cudaGetLastError();
}

}  // namespace

bool rows_supported(int D, int q) { return (D == 1 && q == 3) || (D == 2 && q == 2) || (D == 3 && q == 3); }

template <typename T>
void rows_config(const OpParams<T>& P, int target, int* cells, size_t* smem) {
  if (P.D == 1 && P.q == 3) return rows_config_shape<T, 1, 3>(P, target, cells, smem);
  if (P.D == 2 && P.q == 2) return rows_config_shape<T, 2, 2>(P, target, cells, smem);
  if (P.D == 3 && P.q == 3) return rows_config_shape<T, 3, 3>(P, target, cells, smem);
  *cells = 0;
  *smem = 0;
}

template <typename T>
cudaError_t launch_rows(const OpParams<T>& P, const T* x, const Epi<T>& e, cudaStream_t s) {
  if (P.D == 1 && P.q == 3) return launch_rows_shape<T, 1, 3, false>(P, x, e, s);
  if (P.D == 2 && P.q == 2) return launch_rows_shape<T, 2, 2, false>(P, x, e, s);
  if (P.D == 3 && P.q == 3) return launch_rows_shape<T, 3, 3, false>(P, x, e, s);
  return cudaErrorInvalidConfiguration;
}

template <typename T>
cudaError_t build_coef_tables(OpParams<T>& P, std::vector<DevBuf>& owner, bool with_diag) {
  P.cvtab = nullptr;
  P.cftab = nullptr;
  P.mktab = nullptr;
  P.rdtab = nullptr;
  if (P.D == 1 && P.q == 3) return coef_tables_shape<T, 1, 3>(P, owner, with_diag);
  if (P.D == 2 && P.q == 2) return coef_tables_shape<T, 2, 2>(P, owner, with_diag);
  if (P.D == 3 && P.q == 3) return coef_tables_shape<T, 3, 3>(P, owner, with_diag);
  return cudaSuccess;  // other shapes run the cell-node kernel, which computes its coefficients
}

template <typename T>
cudaError_t launch_rows_transposed(const OpParams<T>& P, const T* x, const Epi<T>& e, cudaStream_t s) {
  if (P.D == 1 && P.q == 3) return launch_rows_shape<T, 1, 3, true>(P, x, e, s);
  if (P.D == 2 && P.q == 2) return launch_rows_shape<T, 2, 2, true>(P, x, e, s);
  if (P.D == 3 && P.q == 3) return launch_rows_shape<T, 3, 3, true>(P, x, e, s);
  return cudaErrorInvalidConfiguration;
}

template <typename T>
cudaError_t launch_rows_batched(const BatchDev<T>& B, const int* active, const T* x, const Epi<T>& e, cudaStream_t s) {
  if (B.shape_d == 1 && B.shape_q == 3) return launch_rows_batched_shape<T, 1, 3>(B, active, x, e, s);
  if (B.shape_d == 2 && B.shape_q == 2) return launch_rows_batched_shape<T, 2, 2>(B, active, x, e, s);
  if (B.shape_d == 3 && B.shape_q == 3) return launch_rows_batched_shape<T, 3, 3>(B, active, x, e, s);
  return cudaErrorInvalidConfiguration;
}

template <typename T>
cudaError_t prepare_rows_batched(const BatchDev<T>& B) {
  if (B.shape_d == 1 && B.shape_q == 3) return opt_in_rows_batched_shape<T, 1, 3>();
  if (B.shape_d == 2 && B.shape_q == 2) return opt_in_rows_batched_shape<T, 2, 2>();
  if (B.shape_d == 3 && B.shape_q == 3) return opt_in_rows_batched_shape<T, 3, 3>();
  return cudaErrorInvalidConfiguration;
}

template cudaError_t prepare_rows_batched<double>(const BatchDev<double>&);
template cudaError_t prepare_rows_batched<float>(const BatchDev<float>&);
template void rows_config<double>(const OpParams<double>&, int, int*, size_t*);
template void rows_config<float>(const OpParams<float>&, int, int*, size_t*);
template cudaError_t launch_rows<double>(const OpParams<double>&, const double*, const Epi<double>&, cudaStream_t);
template cudaError_t launch_rows<float>(const OpParams<float>&, const float*, const Epi<float>&, cudaStream_t);
template cudaError_t build_coef_tables<double>(OpParams<double>&, std::vector<DevBuf>&, bool);
template cudaError_t build_coef_tables<float>(OpParams<float>&, std::vector<DevBuf>&, bool);
template cudaError_t launch_rows_transposed<double>(const OpParams<double>&, const double*, const Epi<double>&,
                                                    cudaStream_t);
template cudaError_t launch_rows_transposed<float>(const OpParams<float>&, const float*, const Epi<float>&,
                                                   cudaStream_t);
template cudaError_t launch_rows_batched<double>(const BatchDev<double>&, const int*, const double*,
                                                 const Epi<double>&, cudaStream_t);
template cudaError_t launch_rows_batched<float>(const BatchDev<float>&, const int*, const float*, const Epi<float>&,
                                                cudaStream_t);

}  // namespace sap
