// CUDA kernels of the dG operator apply, fused ERK4 stages and the Crank--Nicolson / GMRES solve.
//
// Operator (Sec. 3, Eq. linear-system-degrees-of-freedom, Eq. definition-mass-and-dg-matrix) in the
// Gauss-collocated nodal basis, where the mass matrix is diagonal:
//   (M^-1 D f)(i) = (R - div beta) f (i)
//                 - sum_a (1/h_a) sum_q S[i_a][q] (beta^a f)(.., q, ..)            volume term
//                 + sum_a (1/h_a) [ L1[i_a] J_a,up(i) - L0[i_a] J_a,dn(i) ]          face lifts
// with S[i][q] = w_q l_i'(x_q) / w_i, L0/L1 = l_i(0 or 1) / w_i, and the upwind flux
//   J = 1/2 beta (f_lo + f_hi) + 1/2 |beta| (f_lo - f_hi),   |beta| = W |Lambda| W^T,
// which equals W (Lambda+ W^T f_lo + Lambda- W^T f_hi) (Eq. definition-upwind-flux).  Boundary faces
// replace the missing side by 0 (zero inflow, Eq. definition-boundary-flux) or by the inner trace
// (continuous, Eq. continuous-bc); periodic faces use the wrapped neighbour.
//
// One thread block handles `cpb` cells; one thread per (cell, coefficient j, node).  Neighbour
// traces are read straight from global memory (L2), the cell's own data is staged in shared memory.
// The sparse (l,m,s) couplings are applied from CSR tables held in global memory (read through the
// read-only cache); their coefficients are formed per node from spatial fields and the momentum.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <atomic>
#include <mutex>
#include <type_traits>
#include <string>
#include <vector>

#include "kernels_common.cuh"

namespace sap {

// kernels launched by this host thread (for the launch counts reported in sap_solver_stats)
static thread_local int64_t g_launches = 0;
int64_t launch_count() { return g_launches; }
void note_launch() { ++g_launches; }

void cn_graphs_release(sap_ctx* c) {
  for (auto& gg : c->cn_graphs)
    if (gg.exec) cudaGraphExecDestroy(gg.exec);
  c->cn_graphs.clear();
}

template <typename T>
__device__ __forceinline__ T csr_row(const Bank<T>& B, int mat, int r, const T* x, int stride) {
  if (mat == MAT_I) return x[r * stride];
  const int* rp = B.rp + B.rp_off[mat];
  T acc0 = T(0), acc1 = T(0);
  int k = __ldg(rp + r);
  const int e = __ldg(rp + r + 1);
  for (; k + 1 < e; k += 2) {  // two independent chains hide the load latency
    const int c0 = __ldg(B.col + k), c1 = __ldg(B.col + k + 1);
    const T v0 = __ldg(B.val + k), v1 = __ldg(B.val + k + 1);
    acc0 += v0 * x[c0 * stride];
    acc1 += v1 * x[c1 * stride];
  }
  if (k < e) acc0 += __ldg(B.val + k) * x[__ldg(B.col + k) * stride];
  return acc0 + acc1;
}

// node index from a face point (axis a removed) and the position j along a
__device__ __forceinline__ int face_node(int fp, int j, int a, const int* qpow) {
  const int lo = fp % qpow[a];
  const int hi = fp / qpow[a];
  return lo + j * qpow[a] + hi * qpow[a + 1];
}

constexpr int EMAX = 6;  // face entries per thread: ceil(2 D / q) <= 6

// Body of the apply for the cells [cell0, cell0 + cpb) of one problem whose state starts at element
// `doff` of every state-sized vector (0 for a single problem, the instance offset in a batch).
// DT, QT: compile-time number of axes and nodes per axis (0: taken from P at run time).
template <typename T, int DT, int QT>
__device__ __forceinline__ void apply_body(const OpParams<T>& P, const T* __restrict__ x, const Epi<T>& E, int cpb,
                                           int cell_stride, int cell0, int64_t doff, unsigned char* smem_raw) {
  if (E.skip && *E.skip) return;  // uniform over the grid
  T* sm = reinterpret_cast<T*>(smem_raw);
  x += doff;
  const int n = P.n;
  const int D = DT ? DT : P.D;
  const int q = QT ? QT : P.q;
  const int nloc = DT ? qpow_of(q, D) : P.nloc;
  const int nfp = DT ? qpow_of(q, D - 1) : P.nfp;
  const int has_mom = P.has_mom;
  const int per_cell = n * nloc;
  const int nf = 2 * D;
  const int lc = threadIdx.x / per_cell;
  const int t = threadIdx.x - lc * per_cell;
  const int r = t / nloc, i = t - r * nloc;
  const int cell = cell0 + lc;
  const bool valid = (lc < cpb) && (cell < P.ncell);
  int nvt = P.nreact;
  int adv_off[MAXD];
#pragma unroll
  for (int a = 0; a < MAXD; ++a) {
    if (a < D) {
      adv_off[a] = nvt;
      nvt += P.ax[a].nadv;
    }
  }
  const int szT = nf * n * nfp;
  T* F = sm + (size_t)(lc < cpb ? lc : 0) * cell_stride;
  T* Jf = F + per_cell;
  T* Tr = Jf + szT;
  T* Tn = Tr + szT;
  T* W1 = Tn + szT;
  T* G = Tr;  // aliases Tr/Tn/W1 once the face fluxes are done
  const int region = (3 * szT > D * per_cell) ? 3 * szT : D * per_cell;
  T* CV = Tr + region;
  T* CF = CV + nvt * nloc;
  const int scell = valid ? P.cell_scell[cell] : 0;
  const int pcell = valid ? P.cell_pcell[cell] : 0;
  const int qdx = has_mom ? nfp : nloc;            // spatial nodes per cell
  const int qsp = has_mom ? (DT ? qpow_of(q, D - 2) : P.qdx / q) : nfp;  // spatial points per spatial face
  // this thread's face entries w = t + e * per_cell, decomposed once: face f, coefficient, face point
  int fe[EMAX], re[EMAX], pe[EMAX], nbe[EMAX];
  int ne = 0;
#pragma unroll
  for (int e = 0; e < EMAX; ++e) {
    const int w = t + e * per_cell;
    fe[e] = 0; re[e] = 0; pe[e] = 0; nbe[e] = -1;
    if (w < szT) {
      fe[e] = w / (n * nfp);
      const int rem = w - fe[e] * n * nfp;
      re[e] = rem / nfp;
      pe[e] = rem - re[e] * nfp;
      nbe[e] = valid ? P.cell_nb[cell * nf + fe[e]] : -1;
      ne = e + 1;
    }
  }

  // ---- phase 1: stage own data, coefficient tables, neighbour traces ---------------------------
  if (valid) {
    F[t] = x[(size_t)cell * per_cell + t];
    for (int w = t; w < nvt * nloc; w += per_cell) {
      const int tt = w / nloc, ii = w - tt * nloc;
      const Term* tm;
      if (tt < P.nreact) {
        tm = &P.react[tt];
      } else {
        int a = 0;
        while (a + 1 < D && tt >= adv_off[a + 1]) ++a;
        tm = &P.ax[a].adv[tt - adv_off[a]];
      }
      const int sp = scell * qdx + (has_mom ? ii % nfp : ii);
      const int pn = has_mom ? pcell * q + ii / nfp : 0;
      T c = T(tm->scale) * spatial_factor(P, tm->sf, sp) * mom_node(P, tm->mf, pn);
      if (tm->nu) c *= P.nu ? P.nu[(size_t)cell * nloc + ii] : P.nu_uni;
      CV[w] = c;
    }
    // face coefficients of the advection terms at every face point
    for (int w = t; w < nf * MAXADV * nfp; w += per_cell) {
      const int f = w / (MAXADV * nfp);
      const int rem = w - f * MAXADV * nfp;
      const int tt = rem / nfp;
      const int fp = rem - tt * nfp;
      const int a = f >> 1, side = f & 1;
      const AxisInfo& A = P.ax[a];
      if (!A.active || tt >= A.nadv) continue;
      const Term& tm = A.adv[tt];
      T c = T(tm.scale);
      if (A.kind <= SAP_AXIS_Z) {
        // spatial face: U_a at the spatial face point, momentum factor at the node's p
        const int fsp = has_mom ? fp % qsp : fp;
        if (tm.sf == SF_U + a) {
          const int base = P.scell_face[scell * 2 * P.dx + 2 * a + side];
          c *= P.uface_is_uni[a] ? P.uface_uni[a] : P.uface[a][base + fsp];
        } else {
          c *= spatial_factor(P, tm.sf, scell * qdx);  // only SF_ONE occurs here
        }
        c *= mom_node(P, tm.mf, has_mom ? pcell * q + fp / qsp : 0);
      } else {
        // momentum face: spatial factor at the spatial node (fp), momentum at the face
        c *= spatial_factor(P, tm.sf, scell * qdx + fp);
        c *= mom_face(P, tm.mf, pcell + side);
      }
      CF[w] = c;
    }
    // neighbour traces
#pragma unroll
    for (int e = 0; e < EMAX; ++e) {
      if (e >= ne) break;
      const int w = t + e * per_cell;
      const int f = fe[e], a = f >> 1, side = f & 1;
      T v = T(0);
      if (nbe[e] >= 0 && P.ax[a].active) {
        const T* xn = x + ((size_t)nbe[e] * n + re[e]) * nloc;
        for (int j = 0; j < q; ++j) v += (side == 0 ? P.B1[j] : P.B0[j]) * __ldg(xn + face_node_q(pe[e], j, a, q));
      }
      Tn[w] = v;
    }
  }
  __syncthreads();
  // ---- phase 2: own traces ------------------------------------------------------------------------
  if (valid) {
#pragma unroll
    for (int e = 0; e < EMAX; ++e) {
      if (e >= ne) break;
      const int w = t + e * per_cell;
      const int f = fe[e], a = f >> 1, side = f & 1;
      const T* Fr = F + re[e] * nloc;
      T v = T(0);
      for (int j = 0; j < q; ++j) v += (side == 0 ? P.B0[j] : P.B1[j]) * Fr[face_node_q(pe[e], j, a, q)];
      Tr[w] = v;
    }
  }
  __syncthreads();
  // ---- phase 3a: boundary substitution; Tr <- f_lo + f_hi, Tn <- f_lo - f_hi -----------------------
  if (valid) {
#pragma unroll
    for (int e = 0; e < EMAX; ++e) {
      if (e >= ne) break;
      const int w = t + e * per_cell;
      const int f = fe[e], a = f >> 1, side = f & 1;
      if (!P.ax[a].active) continue;
      const T own = Tr[w];
      T oth = Tn[w];
      if (nbe[e] < 0) {
        const int bc = side == 0 ? P.ax[a].bc_lo : P.ax[a].bc_hi;
        oth = (bc == SAP_BC_CONTINUOUS) ? own : T(0);
      }
      const T flo = side == 0 ? oth : own;
      const T fhi = side == 0 ? own : oth;
      Tr[w] = flo + fhi;
      Tn[w] = flo - fhi;
    }
  }
  __syncthreads();
  // ---- phase 3b: J = 1/2 beta S + 1/2 |beta| Dd  (eigen route: first half W^T Dd into W1) ------------
  if (valid) {
#pragma unroll
    for (int e = 0; e < EMAX; ++e) {
      if (e >= ne) break;
      const int w = t + e * per_cell;
      const int f = fe[e], rr = re[e], fp = pe[e];
      const int a = f >> 1;
      const AxisInfo& A = P.ax[a];
      if (!A.active) continue;
      const T* Sb = Tr + f * n * nfp + fp;
      const T* Db = Tn + f * n * nfp + fp;
      T acc = T(0);
      for (int tt = 0; tt < A.nadv; ++tt) acc += CF[(f * MAXADV + tt) * nfp + fp] * csr_row(P.bank, A.adv[tt].mat, rr, Sb, nfp);
      if (A.route == ABS_CONST) {
        acc += csr_row(P.bank, A.absmat, rr, Db, nfp);
        Jf[w] = T(0.5) * acc;
      } else if (A.route == ABS_POINT) {
        const int side = f & 1;
        const int sp = scell * qdx + fp;
        const int slot = __ldg(P.pslot + sp);
        if (slot >= 0) {
          const int* rp = P.bank.rp + P.bank.rp_off[A.absmat];
          const int nnzp = __ldg(rp + n) - __ldg(rp);
          const T* vals = P.pabs + ((size_t)slot * P.npface + pcell + side) * nnzp - __ldg(rp);
          T s2 = T(0);
          for (int k = __ldg(rp + rr); k < __ldg(rp + rr + 1); ++k) s2 += __ldg(vals + k) * Db[__ldg(P.bank.col + k) * nfp];
          acc += s2;
        }
        Jf[w] = T(0.5) * acc;
      } else {  // ABS_EIGEN
        Jf[w] = T(0.5) * acc;
        const T c0 = CF[(f * MAXADV + 0) * nfp + fp];
        const T c1 = CF[(f * MAXADV + 1) * nfp + fp];
        const T ab = A.llf ? fmax(fabs(c0 + T(A.lam_lo) * c1), fabs(c0 + T(A.lam_hi) * c1)) : fabs(c0 + P.lam[rr] * c1);
        W1[w] = ab * csr_row(P.bank, A.WTmat, rr, Db, nfp);
      }
    }
  }
  __syncthreads();
  if (valid) {
#pragma unroll
    for (int e = 0; e < EMAX; ++e) {
      if (e >= ne) break;
      const int w = t + e * per_cell;
      const int f = fe[e];
      const AxisInfo& A = P.ax[f >> 1];
      if (!A.active || A.route != ABS_EIGEN) continue;
      Jf[w] += T(0.5) * csr_row(P.bank, A.Wmat, re[e], W1 + f * n * nfp + pe[e], nfp);
    }
  }
  __syncthreads();
  // ---- phase 3c: volume advection g^a = beta^a f at the nodes (G aliases the face scratch) -------------
  if (valid) {
#pragma unroll
    for (int a = 0; a < MAXD; ++a) {
      if (a >= D) break;
      const AxisInfo& A = P.ax[a];
      if (!A.active) continue;
      T g = T(0);
      for (int tt = 0; tt < A.nadv; ++tt) g += CV[(adv_off[a] + tt) * nloc + i] * csr_row(P.bank, A.adv[tt].mat, r, F + i, nloc);
      G[a * per_cell + t] = g;
    }
  }
  __syncthreads();
  if (!valid) return;
  // ---- phase 4: assemble M^-1 D f at (r, i) -------------------------------------------------------
  T acc = T(0);
  T rdiag = T(0);
  for (int tt = 0; tt < P.nreact; ++tt) {
    const T c = CV[tt * nloc + i];
    acc += c * csr_row(P.bank, P.react[tt].mat, r, F + i, nloc);
    if (E.jacobi || E.out32 || E.outj) rdiag += c * csr_diag(P.bank, P.react[tt].mat, r, n);
  }
#pragma unroll
  for (int a = 0; a < MAXD; ++a) {
    if (a >= D) break;
    if (!P.ax[a].active) continue;
    const int qa = qpow_of(q, a), qa1 = qa * q;
    const T invh = P.cell_invh[cell * D + a];
    const int ia = (i / qa) % q;
    const int base = i - ia * qa;
    const T* Ga = G + a * per_cell + r * nloc + base;
    T ds = T(0);
    for (int qq = 0; qq < q; ++qq) ds += P.S[ia][qq] * Ga[qq * qa];
    const int fp = (i % qa) + (i / qa1) * qa;
    const T jup = Jf[((2 * a + 1) * n + r) * nfp + fp];
    const T jdn = Jf[((2 * a) * n + r) * nfp + fp];
    acc += invh * (P.L1[ia] * jup - P.L0[ia] * jdn - ds);
  }
  T s = T(0);
  if (r == 0) s = P.s000 ? P.s000[(size_t)cell * nloc + i] : P.s_uni;
  epi_write(E, (size_t)doff + (size_t)cell * per_cell + t, F[t], acc, s, rdiag);
}

// Transposed operator L^T = (M^-1 D)^T in the nodal basis (discrete adjoint).  Term by term:
//   reaction  (R - div beta)^T per node (transposed couplings);
//   volume    -(1/h_a) beta^a (S^T y along lines)          (beta^a symmetric);
//   faces     per face g = E_lo^T y_lo - E_hi^T y_hi  (lift-weighted traces, E = lift of the forward
//             operator), then the lo side receives T_lo^T beta+ g and the hi side T_hi^T beta- g,
//             beta+- = (beta +- |beta|)/2; a missing side contributes 0 to g; a continuous
//             boundary uses beta instead of beta+-.
template <typename T>
__device__ __forceinline__ void applyT_body(const OpParams<T>& P, const T* __restrict__ x, const Epi<T>& E, int cpb,
                                            int cell_stride, int cell0, int64_t doff, unsigned char* smem_raw) {
  if (E.skip && *E.skip) return;  // uniform over the grid
  T* sm = reinterpret_cast<T*>(smem_raw);
  x += doff;
  const int n = P.n, nloc = P.nloc, nfp = P.nfp, D = P.D, q = P.q;
  const int per_cell = n * nloc;
  const int nf = 2 * D;
  const int lc = threadIdx.x / per_cell;
  const int t = threadIdx.x - lc * per_cell;
  const int r = t / nloc, i = t - r * nloc;
  const int cell = cell0 + lc;
  const bool valid = (lc < cpb) && (cell < P.ncell);
  int qpow[MAXD + 2];
  qpow[0] = 1;
#pragma unroll
  for (int a = 1; a < MAXD + 2; ++a) qpow[a] = qpow[a - 1] * q;
  int nvt = P.nreact;
  int adv_off[MAXD];
  for (int a = 0; a < D; ++a) {
    adv_off[a] = nvt;
    nvt += P.ax[a].nadv;
  }
  const int szT = nf * n * nfp;
  T* F = sm + (size_t)(lc < cpb ? lc : 0) * cell_stride;
  T* Jf = F + per_cell;
  T* Tr = Jf + szT;
  T* Tn = Tr + szT;
  T* W1 = Tn + szT;
  T* G = Tr;
  const int region = (3 * szT > D * per_cell) ? 3 * szT : D * per_cell;
  T* CV = Tr + region;
  T* CF = CV + nvt * nloc;
  const int scell = valid ? P.cell_scell[cell] : 0;
  const int pcell = valid ? P.cell_pcell[cell] : 0;
  if (valid) {
    F[t] = x[(size_t)cell * per_cell + t];
    for (int w = t; w < nvt * nloc; w += per_cell) {
      const int tt = w / nloc, ii = w - tt * nloc;
      const Term* tm;
      if (tt < P.nreact) {
        tm = &P.react[tt];
      } else {
        int a = 0;
        while (a + 1 < D && tt >= adv_off[a + 1]) ++a;
        tm = &P.ax[a].adv[tt - adv_off[a]];
      }
      const int sp = scell * P.qdx + ii % P.qdx;
      T c = T(tm->scale) * spatial_factor(P, tm->sf, sp) * mom_node(P, tm->mf, pcell * q + ii / P.qdx);
      if (tm->nu) c *= P.nu ? P.nu[(size_t)cell * nloc + ii] : P.nu_uni;
      CV[w] = c;
    }
    for (int w = t; w < nf * MAXADV * nfp; w += per_cell) {
      const int f = w / (MAXADV * nfp);
      const int tt = (w / nfp) % MAXADV;
      const int fp = w % nfp;
      const int a = f >> 1, side = f & 1;
      const AxisInfo& A = P.ax[a];
      if (!A.active || tt >= A.nadv) continue;
      const Term& tm = A.adv[tt];
      T c = T(tm.scale);
      if (A.kind <= SAP_AXIS_Z) {
        const int qsp = P.qdx / q;
        const int fsp = fp % qsp;
        if (tm.sf == SF_U + a) {
          const int base = P.scell_face[scell * 2 * P.dx + 2 * a + side];
          c *= P.uface_is_uni[a] ? P.uface_uni[a] : P.uface[a][base + fsp];
        } else {
          c *= spatial_factor(P, tm.sf, scell * P.qdx);
        }
        c *= mom_node(P, tm.mf, pcell * q + fp / qsp);
      } else {
        c *= spatial_factor(P, tm.sf, scell * P.qdx + fp);
        c *= mom_face(P, tm.mf, pcell + side);
      }
      CF[w] = c;
    }
    // neighbour lift-weighted traces: lower face -> +E_lo^T y_nb (nb is lo), upper -> -E_hi^T y_nb
    for (int w = t; w < szT; w += per_cell) {
      const int f = w / (n * nfp);
      const int rr = (w / nfp) % n;
      const int fp = w % nfp;
      const int a = f >> 1, side = f & 1;
      const int nb = P.cell_nb[cell * nf + f];
      T v = T(0);
      if (nb >= 0 && P.ax[a].active) {
        const T ihn = P.cell_invh[nb * D + a];
        const T* xn = x + ((size_t)nb * n + rr) * nloc;
        for (int j = 0; j < q; ++j) v += (side == 0 ? P.L1[j] : -P.L0[j]) * __ldg(xn + face_node(fp, j, a, qpow));
        v *= ihn;
      }
      Tn[w] = v;
    }
  }
  __syncthreads();
  if (valid) {
    // own lift-weighted traces: lower face (I am hi) -> -E_hi^T y, upper face (I am lo) -> +E_lo^T y
    const T* ihm = P.cell_invh + cell * D;
    for (int w = t; w < szT; w += per_cell) {
      const int f = w / (n * nfp);
      const int rr = (w / nfp) % n;
      const int fp = w % nfp;
      const int a = f >> 1, side = f & 1;
      T v = T(0);
      const T* Fr = F + rr * nloc;
      for (int j = 0; j < q; ++j) v += (side == 0 ? -P.L0[j] : P.L1[j]) * Fr[face_node(fp, j, a, qpow)];
      Tr[w] = v * ihm[a];
    }
  }
  __syncthreads();
  if (valid) {
    // g = own + neighbour part (a boundary has no neighbour part)
    for (int w = t; w < szT; w += per_cell) {
      const int f = w / (n * nfp);
      const int a = f >> 1;
      if (!P.ax[a].active) continue;
      Tr[w] += Tn[w];
    }
  }
  __syncthreads();
  // K g with K = beta+ (upper face), beta- (lower face), beta (continuous boundary)
  if (valid) {
    for (int w = t; w < szT; w += per_cell) {
      const int f = w / (n * nfp);
      const int rr = (w / nfp) % n;
      const int fp = w % nfp;
      const int a = f >> 1, side = f & 1;
      const AxisInfo& A = P.ax[a];
      if (!A.active) continue;
      const int nb = P.cell_nb[cell * nf + f];
      const int bc = side == 0 ? A.bc_lo : A.bc_hi;
      const bool cont = (nb < 0) && (bc == SAP_BC_CONTINUOUS);
      const T sgn = side == 1 ? T(1) : T(-1);
      const T* Gb = Tr + f * n * nfp + fp;
      T acc = T(0);
      for (int tt = 0; tt < A.nadv; ++tt) acc += CF[(f * MAXADV + tt) * nfp + fp] * csr_row(P.bank, A.adv[tt].mat, rr, Gb, nfp);
      if (cont) {
        Jf[w] = acc;
        if (A.route == ABS_EIGEN) W1[w] = T(0);
        continue;
      }
      if (A.route == ABS_CONST) {
        Jf[w] = T(0.5) * (acc + sgn * csr_row(P.bank, A.absmat, rr, Gb, nfp));
      } else if (A.route == ABS_POINT) {
        const int sp = scell * P.qdx + fp;
        const int slot = __ldg(P.pslot + sp);
        T s2 = T(0);
        if (slot >= 0) {
          const int* rp = P.bank.rp + P.bank.rp_off[A.absmat];
          const int nnzp = __ldg(rp + n) - __ldg(rp);
          const T* vals = P.pabs + ((size_t)slot * P.npface + pcell + side) * nnzp - __ldg(rp);
          for (int k = __ldg(rp + rr); k < __ldg(rp + rr + 1); ++k) s2 += __ldg(vals + k) * Gb[__ldg(P.bank.col + k) * nfp];
        }
        Jf[w] = T(0.5) * (acc + sgn * s2);
      } else {
        Jf[w] = T(0.5) * acc;
        const T c0 = CF[(f * MAXADV + 0) * nfp + fp];
        const T c1 = CF[(f * MAXADV + 1) * nfp + fp];
        const T ab = A.llf ? fmax(fabs(c0 + T(A.lam_lo) * c1), fabs(c0 + T(A.lam_hi) * c1)) : fabs(c0 + P.lam[rr] * c1);
        W1[w] = sgn * ab * csr_row(P.bank, A.WTmat, rr, Gb, nfp);
      }
    }
  }
  __syncthreads();
  if (valid) {
    for (int w = t; w < szT; w += per_cell) {
      const int f = w / (n * nfp);
      const int rr = (w / nfp) % n;
      const int fp = w % nfp;
      const AxisInfo& A = P.ax[f >> 1];
      if (!A.active || A.route != ABS_EIGEN) continue;
      Jf[w] += T(0.5) * csr_row(P.bank, A.Wmat, rr, W1 + f * n * nfp + fp, nfp);
    }
  }
  __syncthreads();
  // volume: z_a = S^T y along lines (G aliases the face scratch)
  if (valid) {
    for (int a = 0; a < D; ++a) {
      if (!P.ax[a].active) continue;
      const int ia = (i / qpow[a]) % q;
      const int base = i - ia * qpow[a];
      const T* Fa = F + r * nloc + base;
      T z = T(0);
      for (int qq = 0; qq < q; ++qq) z += P.S[qq][ia] * Fa[qq * qpow[a]];
      G[a * per_cell + t] = z;
    }
  }
  __syncthreads();
  if (!valid) return;
  T acc = T(0);
  T rdiag = T(0);
  for (int tt = 0; tt < P.nreact; ++tt) {
    const T c = CV[tt * nloc + i];
    acc += c * csr_row(P.bank, P.react[tt].matT, r, F + i, nloc);
    if (E.jacobi || E.out32 || E.outj) rdiag += c * csr_diag(P.bank, P.react[tt].mat, r, n);
  }
  for (int a = 0; a < D; ++a) {
    if (!P.ax[a].active) continue;
    const T invh = P.cell_invh[cell * D + a];
    T g = T(0);
    for (int tt = 0; tt < P.ax[a].nadv; ++tt)
      g += CV[(adv_off[a] + tt) * nloc + i] * csr_row(P.bank, P.ax[a].adv[tt].mat, r, G + a * per_cell + i, nloc);
    const int ia = (i / qpow[a]) % q;
    const int fp = (i % qpow[a]) + (i / qpow[a + 1]) * qpow[a];
    const T jup = Jf[((2 * a + 1) * n + r) * nfp + fp];
    const T jdn = Jf[((2 * a) * n + r) * nfp + fp];
    acc += P.B1[ia] * jup + P.B0[ia] * jdn - invh * g;
  }
  const size_t dof = (size_t)doff + (size_t)cell * per_cell + t;
  T o = E.ax * F[t] + E.bl * acc;
  if (E.bvec) o += E.wb * __ldg(E.bvec + dof);
  if (E.out32) E.out32[dof] = float(o * jacobi_scale(E.cj, rdiag));
  if (E.out2) {
    const T o2 = E.ax2 * F[t] + E.bl2 * acc;
    E.out2[dof] = o2;
    if (E.outj) E.outj[dof] = o2 * jacobi_scale(E.cj, rdiag);
  } else if (E.outj) {
    E.outj[dof] = o * jacobi_scale(E.cj, rdiag);
  }
  if (E.jacobi) o *= jacobi_scale(E.cj, rdiag);
  if (E.axpost != T(0)) o += E.axpost * F[t];
  if (E.xs) o *= T(*E.xs);
  if (E.out) E.out[dof] = o;
}

template <typename T>
__global__ void __launch_bounds__(1024) applyT_kernel(const __grid_constant__ OpParams<T> P, const T* __restrict__ x, const Epi<T> E,
                                                      int cpb, int cell_stride) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  applyT_body<T>(P, x, E, cpb, cell_stride, blockIdx.x * cpb, 0, smem_raw);
}

template <typename T, int DT, int QT>
__global__ void __launch_bounds__(1024) apply_kernel(const __grid_constant__ OpParams<T> P, const T* __restrict__ x, const Epi<T> E,
                                                     int cpb, int cell_stride) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  apply_body<T, DT, QT>(P, x, E, cpb, cell_stride, blockIdx.x * cpb, 0, smem_raw);
}

// Batched apply: block b works on instance blocks[b].x, cells [blocks[b].y, + cpb[inst]).  The
// instance's parameter block is staged in shared memory; blocks of inactive instances return.
template <typename T, int DT, int QT>
__global__ void __launch_bounds__(1024) apply_kernel_batched(const OpParams<T>* __restrict__ Pall,
                                                             const int64_t* __restrict__ doffs,
                                                             const int* __restrict__ cpbs,
                                                             const int* __restrict__ strides,
                                                             const int2* __restrict__ blocks,
                                                             const int* __restrict__ active,
                                                             const T* __restrict__ x, const Epi<T> E) {
  __shared__ __align__(16) unsigned char pbuf[sizeof(OpParams<T>)];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int2 bb = blocks[blockIdx.x];
  if (active && !active[bb.x]) return;  // uniform over the block: no barrier is skipped by part of it
  const int* src = reinterpret_cast<const int*>(Pall + bb.x);
  int* dst = reinterpret_cast<int*>(pbuf);
  for (int k = threadIdx.x; k < (int)(sizeof(OpParams<T>) / sizeof(int)); k += blockDim.x) dst[k] = src[k];
  __syncthreads();
  apply_body<T, DT, QT>(*reinterpret_cast<const OpParams<T>*>(pbuf), x, E, cpbs[bb.x], strides[bb.x], bb.y, doffs[bb.x],
                        smem_raw);
}

int apply_cells_per_block(int n, int nloc) {
  const int per = n * nloc;
  int cpb = std::max(1, 256 / per);
  while (cpb > 1 && cpb * per > 1024) --cpb;
  return cpb;
}

template <typename T>
static int cell_stride_elems(const OpParams<T>& P);
int apply_cell_stride(const OpParams<double>& P) { return cell_stride_elems(P); }

template <typename T>
static int cell_stride_elems(const OpParams<T>& P) {
  int nvt = P.nreact;
  for (int a = 0; a < P.D; ++a) nvt += P.ax[a].nadv;
  const int per = P.n * P.nloc;
  const int szT = 2 * P.D * P.n * P.nfp;
  int s = per + szT + std::max(3 * szT, P.D * per) + nvt * P.nloc + 2 * P.D * MAXADV * P.nfp;
  return (s + 1) & ~1;  // keep 16-byte alignment of each cell's block for doubles
}

template <typename T, int DT, int QT>
static cudaError_t launch_apply_shape(const OpParams<T>& P, const T* x, const Epi<T>& e, cudaStream_t s, int cpb,
                                      int stride, size_t smem) {
  static DeviceMask opted{};
  if (cudaError_t err = smem_opt_in(apply_kernel<T, DT, QT>, 200 * 1024, opted); err != cudaSuccess) return err;
  const int blocks = (P.ncell + cpb - 1) / cpb;
  apply_kernel<T, DT, QT><<<blocks, cpb * P.n * P.nloc, smem, s>>>(P, x, e, cpb, stride);
  ++g_launches;
  return cudaGetLastError();
}

// The shapes (D, q) compiled for the row-per-thread kernel (apply_rows.cu) run there; every other
// shape runs the generic cell-node kernel.
template <typename T>
static cudaError_t launch_apply(const OpParams<T>& P, const T* x, const Epi<T>& e, cudaStream_t s) {
  if (P.uni_L >= 0) return launch_uniform<T>(P, x, e, s);
  if (rows_supported(P.D, P.q)) return launch_rows<T>(P, x, e, s);
  const int per = P.n * P.nloc;
  if (per > 1024) return cudaErrorInvalidConfiguration;  // n (k+1)^D must fit one thread block
  const int cpb = apply_cells_per_block(P.n, P.nloc);
  const int stride = cell_stride_elems(P);
  const size_t smem = (size_t)cpb * stride * sizeof(T);
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  return launch_apply_shape<T, 0, 0>(P, x, e, s, cpb, stride, smem);
}

template <typename T>
static cudaError_t launch_applyT(const OpParams<T>& P, const T* x, const Epi<T>& e, cudaStream_t s) {
  if (rows_supported(P.D, P.q)) return launch_rows_transposed<T>(P, x, e, s);
  const int per = P.n * P.nloc;
  if (per > 1024) return cudaErrorInvalidConfiguration;
  const int cpb = apply_cells_per_block(P.n, P.nloc);
  const int stride = cell_stride_elems(P);
  const size_t smem = (size_t)cpb * stride * sizeof(T);
  static DeviceMask opted{};  // one per instantiation (T)
  if (cudaError_t err = smem_opt_in(applyT_kernel<T>, 200 * 1024, opted); err != cudaSuccess) return err;
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  const int blocks = (P.ncell + cpb - 1) / cpb;
  applyT_kernel<T><<<blocks, cpb * per, smem, s>>>(P, x, e, cpb, stride);
  ++g_launches;
  return cudaGetLastError();
}

template <typename T>
static Epi<T> epi_plain(T* out, T ax, T bl, T gs) {
  Epi<T> e{};
  e.out = out;
  e.ax = ax;
  e.bl = bl;
  e.gs = gs;
  return e;
}

cudaError_t launch_apply64(const OpParams<double>& p, const double* x, double* y, int mode, cudaStream_t s) {
  if (mode == SAP_APPLY_T) return launch_applyT<double>(p, x, epi_plain<double>(y, 0, 1, 0), s);
  return launch_apply<double>(p, x, mode == SAP_APPLY_RHS ? epi_plain<double>(y, 0, -1, 1) : epi_plain<double>(y, 0, 1, 0), s);
}
cudaError_t launch_apply32(const OpParams<float>& p, const float* x, float* y, int mode, cudaStream_t s) {
  if (mode == SAP_APPLY_T) return launch_applyT<float>(p, x, epi_plain<float>(y, 0, 1, 0), s);
  return launch_apply<float>(p, x, mode == SAP_APPLY_RHS ? epi_plain<float>(y, 0, -1, 1) : epi_plain<float>(y, 0, 1, 0), s);
}

// ------------------------------------------------------------------------------------------------
// ERK4 (classical) with fused stages
// ------------------------------------------------------------------------------------------------
template <typename T>
__global__ void cast_kernel(const double* __restrict__ a, T* __restrict__ b, int64_t N) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x) b[k] = T(a[k]);
}

template <typename T>
static cudaError_t erk_impl(sap_ctx* c, const OpParams<T>& P, T* ya, T* yb, double* acc, double* state, double dt,
                            int nsteps, cudaStream_t s) {
  // stage inputs Y1 = y, Y2 = y + dt/2 k1, Y3 = y + dt/2 k2, Y4 = y + dt k3; y' = y + dt/6 (k1 + 2k2 + 2k3 + k4)
  const T* stage_in0 = nullptr;
  cudaError_t err = cudaSuccess;
  for (int it = 0; it < nsteps; ++it) {
    if (sizeof(T) == 8) {
      stage_in0 = reinterpret_cast<const T*>(state);
    } else {
      cast_kernel<T><<<1024, 256, 0, s>>>(state, ya, c->N);
  ++g_launches;
      stage_in0 = ya;
    }
    Epi<T> e{};
    e.acc = acc;
    e.y0 = state;
    // stage 1
    e.erk = 1; e.bdt = dt / 6.0; e.adt = 0.5 * dt; e.ynext = (sizeof(T) == 8) ? ya : yb;
    if ((err = launch_apply<T>(P, stage_in0, e, s)) != cudaSuccess) return err;
    const T* in2 = e.ynext;
    T* out2 = (in2 == ya) ? yb : ya;
    e.erk = 2; e.bdt = dt / 3.0; e.adt = 0.5 * dt; e.ynext = out2;
    if ((err = launch_apply<T>(P, in2, e, s)) != cudaSuccess) return err;
    const T* in3 = out2;
    T* out3 = (in3 == ya) ? yb : ya;
    e.erk = 2; e.bdt = dt / 3.0; e.adt = dt; e.ynext = out3;
    if ((err = launch_apply<T>(P, in3, e, s)) != cudaSuccess) return err;
    e.erk = 3; e.bdt = dt / 6.0; e.ynext = nullptr; e.state = state;
    if ((err = launch_apply<T>(P, out3, e, s)) != cudaSuccess) return err;
  }
  return cudaSuccess;
}

// ------------------------------------------------------------------------------------------------
// RK4 without allocation: stage buffers in a file-scope device array (see sap_step_erk_noalloc)
// ------------------------------------------------------------------------------------------------
static __device__ __align__(256) unsigned char g_noalloc_scratch[24 * (size_t)SAP_NOALLOC_MAX_DOFS];

sap_status erk_steps_noalloc(sap_ctx* c, double* state, double dt, int nsteps, cudaStream_t s) {
  if (c->N > SAP_NOALLOC_MAX_DOFS) {
    c->err = "sap_step_erk_noalloc: N = " + std::to_string(c->N) + " exceeds SAP_NOALLOC_MAX_DOFS = " +
             std::to_string((long long)SAP_NOALLOC_MAX_DOFS);
    return SAP_EINVAL;
  }
  // host code cannot use the array's name as a device address: look it up once per device
  static std::mutex mu;
  static void* addr[128] = {nullptr};
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess || dev < 0 || dev >= 128) {
    c->err = "sap_step_erk_noalloc: cudaGetDevice failed";
    return SAP_ECUDA;
  }
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
      err = cudaGetSymbolAddress(&addr[dev], g_noalloc_scratch);
      if (err != cudaSuccess) {
        addr[dev] = nullptr;
        c->err = std::string("sap_step_erk_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(err);
        return SAP_ECUDA;
      }
    }
    base = addr[dev];
  }
  const size_t N = (size_t)c->N;
  if (c->prec == SAP_PREC_FP64) {
    double* ya = static_cast<double*>(base);
    err = erk_impl<double>(c, c->p64, ya, ya + N, ya + 2 * N, state, dt, nsteps, s);
  } else {
    float* ya = static_cast<float*>(base);
    double* acc = reinterpret_cast<double*>(ya + 2 * N);  // byte offset 8N: 8-byte aligned
    err = erk_impl<float>(c, c->p32, ya, ya + N, acc, state, dt, nsteps, s);
  }
  if (err != cudaSuccess) {
    c->err = std::string("erk_noalloc: ") + cudaGetErrorString(err);
    return SAP_ECUDA;
  }
  return SAP_OK;
}

sap_status erk_steps(sap_ctx* c, double* state, double dt, int nsteps, cudaStream_t s) {
  cudaError_t err;
  if (c->prec == SAP_PREC_FP64) {
    err = erk_impl<double>(c, c->p64, c->ws64, c->ws64 + c->N, c->ws64 + 2 * c->N, state, dt, nsteps, s);
  } else {
    err = erk_impl<float>(c, c->p32, c->ws32, c->ws32 + c->N, c->ws64, state, dt, nsteps, s);
  }
  if (err != cudaSuccess) {
    c->err = std::string("erk: ") + cudaGetErrorString(err);
    return SAP_ECUDA;
  }
  return SAP_OK;
}

// ------------------------------------------------------------------------------------------------
// Krylov kernels: multi-dot, update, norms (FP64 sums)
// ------------------------------------------------------------------------------------------------
constexpr int KRY_THREADS = 256;
constexpr int KRY_MAXV = 32;

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// The batched Krylov kernels work on chunks of KRY_CHUNK entries, one thread block per chunk; the
// single-problem passes take one wave of blocks and stage their ranges in sub-chunks of at most
// KRY_CHUNK entries.  The partial-sum scratch holds one slot per chunk.
constexpr int KRY_CHUNK = 2048;

// x (FP64) += sum_i y[i] V_i
template <typename TV>
__global__ void combine_kernel(const TV* __restrict__ V, int64_t ldv, int m, const double* __restrict__ y,
                               double* __restrict__ x, int64_t N) {
  __shared__ double ys[KRY_MAXV];
  if (threadIdx.x < m) ys[threadIdx.x] = y[threadIdx.x];
  __syncthreads();
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x) {
    double v = x[k];
    for (int i = 0; i < m; ++i) v += ys[i] * double(__ldg(V + i * ldv + k));
    x[k] = v;
  }
}

}  // namespace sap

// ------------------------------------------------------------------------------------------------
// Crank--Nicolson step, restarted GMRES with left point-Jacobi preconditioning (FP64)
// ------------------------------------------------------------------------------------------------
namespace sap {

// partial[i][chunk], i <= KRY_MAXV (the dots of w with up to KRY_MAXV basis vectors and w . w)
int64_t krylov_scratch_doubles(int64_t N) {
  const int64_t nchunks = (N + KRY_CHUNK - 1) / KRY_CHUNK;
  return (KRY_MAXV + 1) * nchunks;
}

int64_t krylov_batch_scratch_doubles(const std::vector<int64_t>& Ns) {
  int64_t nchunks = 0;
  for (int64_t n : Ns) nchunks += (n + KRY_CHUNK - 1) / KRY_CHUNK;
  return (KRY_MAXV + 1) * nchunks + (int64_t)Ns.size() * 4 * KRY_MAXV;
}

// ------------------------------------------------------------------------------------------------
// Device-controlled Arnoldi (single problem, FP64): reductions are finished by the last block of
// each kernel (atomic ticket, fixed summation order, no waiting), the Gram--Schmidt decision, the
// Givens rotations and the convergence test run on one device thread, and kernels after
// convergence exit at once.  The host enqueues iterations in groups and synchronises per group.
// ------------------------------------------------------------------------------------------------
struct GmresDev {
  double H[KRY_MAXV * (KRY_MAXV + 1)];  // H[i * KRY_MAXV + j]
  double g[KRY_MAXV + 1], cs[KRY_MAXV], sn[KRY_MAXV];
  double h1[KRY_MAXV + 1], h2[KRY_MAXV + 1];
  double vs[KRY_MAXV + 1];  // the basis is stored unnormalised: v_i = vs[i] * V_i
  double nrm, inv_norm, target, beta;
  double misc[8];
  int done, reorth, jdone, m;
  unsigned int counter;
};

__device__ void gmres_finalize_column(GmresDev* G, int j) {
  const int M = KRY_MAXV;
  const double hn = sqrt(G->nrm);
  // the Arnoldi vectors are built from the shifted operator P^-1 A - 1 (same Krylov space, better
  // conditioned Gram--Schmidt); the Hessenberg matrix of P^-1 A has the shift back on its diagonal
  G->H[j * M + j] += 1.0;
  G->H[(j + 1) * M + j] = hn;
  for (int i = 0; i < j; ++i) {
    const double a0 = G->H[i * M + j], a1 = G->H[(i + 1) * M + j];
    G->H[i * M + j] = G->cs[i] * a0 + G->sn[i] * a1;
    G->H[(i + 1) * M + j] = -G->sn[i] * a0 + G->cs[i] * a1;
  }
  const double a0 = G->H[j * M + j], a1 = G->H[(j + 1) * M + j];
  const double den = hypot(a0, a1);
  G->cs[j] = den > 0 ? a0 / den : 1.0;
  G->sn[j] = den > 0 ? a1 / den : 0.0;
  G->H[j * M + j] = den;
  G->H[(j + 1) * M + j] = 0.0;
  G->g[j + 1] = -G->sn[j] * G->g[j];
  G->g[j] = G->cs[j] * G->g[j];
  G->inv_norm = hn > 0 ? 1.0 / hn : 0.0;
  G->vs[j + 1] = G->inv_norm;  // V_{j+1} holds the orthogonalised w, of norm hn
  G->jdone = j + 1;
  if (fabs(G->g[j + 1]) <= G->target || hn == 0.0 || j + 1 >= G->m) G->done = 1;
}

__device__ __forceinline__ bool kry_skip(const int* done, const int* need) {
  return (done && *done) || (need && !*need);
}

// dots of w with V_0..V_{m-1} (+ w.w) over chunks; the last block sums the partials in chunk order.
// 16 warps per block, one basis vector per warp at a time, paired loads when the layout allows.
constexpr int LB_THREADS = 512;
// Double-float arithmetic on the FP32 units for the FP32 Krylov vectors of the precision form.  On
// GB300 an FP64 instruction costs ~64 FP32 ones; the orthogonalisation keeps FP64-class accuracy
// with exact products (p + pe = a b via FMA) and compensated sums (TwoSum): (s, c) carries a sum
// with ~2^-48 relative error, converted to FP64 once per lane.
// (The _rn intrinsics keep every rounding step as written: no contraction into FMAs.)
__device__ __forceinline__ void df_fma(float& s, float& c, float a, float b) {
  const float p = __fmul_rn(a, b);
  const float pe = fmaf(a, b, -p);
  const float t = __fadd_rn(s, p);
  const float bp = __fsub_rn(t, s);
  const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(p, bp));
  s = t;
  c = __fadd_rn(c, __fadd_rn(err, pe));
}

// V_i . w over one chunk by one warp, FP32 vectors, double-float sums (ws: the chunk of w in FP32)
__device__ __forceinline__ double dot_chunk_df(const float* __restrict__ a, const float* ws, int len, int lane,
                                               bool pairs) {
  // four compensated sums: the dependent chain of each is a quarter as long
  float s0 = 0.0f, c0 = 0.0f, s1 = 0.0f, c1 = 0.0f, s2 = 0.0f, c2 = 0.0f, s3 = 0.0f, c3 = 0.0f;
  int k = lane;
  if (pairs) {
    const float2* a2 = reinterpret_cast<const float2*>(a);
    const int np = len >> 1;
    int p = lane;
    for (; p + 32 < np; p += 64) {
      const float2 x = __ldg(a2 + p), y = __ldg(a2 + p + 32);
      df_fma(s0, c0, x.x, ws[2 * p]);
      df_fma(s1, c1, x.y, ws[2 * p + 1]);
      df_fma(s2, c2, y.x, ws[2 * p + 64]);
      df_fma(s3, c3, y.y, ws[2 * p + 65]);
    }
    for (; p < np; p += 32) {
      const float2 x = __ldg(a2 + p);
      df_fma(s0, c0, x.x, ws[2 * p]);
      df_fma(s1, c1, x.y, ws[2 * p + 1]);
    }
    k = 2 * np + lane;
  }
  for (; k < len; k += 32) df_fma(s0, c0, __ldg(a + k), ws[k]);
  return ((double(s0) + double(c0)) + (double(s1) + double(c1))) + ((double(s2) + double(c2)) + (double(s3) + double(c3)));
}

// V_i . w over one chunk by one warp, FP32 vectors with a and ws 16-byte aligned: four 16-byte loads
// per lane in flight (sixteen entries), the same four compensated sums as dot_chunk_df
__device__ __forceinline__ double dot_chunk_df4(const float* __restrict__ a, const float* ws, int len, int lane) {
  float s0 = 0.0f, c0 = 0.0f, s1 = 0.0f, c1 = 0.0f, s2 = 0.0f, c2 = 0.0f, s3 = 0.0f, c3 = 0.0f;
  const float4* a4 = reinterpret_cast<const float4*>(a);
  const float4* w4 = reinterpret_cast<const float4*>(ws);
  const int nq = len >> 2;
  int q = lane;
  for (; q + 96 < nq; q += 128) {
    const float4 x0 = __ldg(a4 + q), x1 = __ldg(a4 + q + 32), x2 = __ldg(a4 + q + 64), x3 = __ldg(a4 + q + 96);
    const float4 y0 = w4[q], y1 = w4[q + 32], y2 = w4[q + 64], y3 = w4[q + 96];
    df_fma(s0, c0, x0.x, y0.x);
    df_fma(s1, c1, x0.y, y0.y);
    df_fma(s2, c2, x0.z, y0.z);
    df_fma(s3, c3, x0.w, y0.w);
    df_fma(s0, c0, x1.x, y1.x);
    df_fma(s1, c1, x1.y, y1.y);
    df_fma(s2, c2, x1.z, y1.z);
    df_fma(s3, c3, x1.w, y1.w);
    df_fma(s0, c0, x2.x, y2.x);
    df_fma(s1, c1, x2.y, y2.y);
    df_fma(s2, c2, x2.z, y2.z);
    df_fma(s3, c3, x2.w, y2.w);
    df_fma(s0, c0, x3.x, y3.x);
    df_fma(s1, c1, x3.y, y3.y);
    df_fma(s2, c2, x3.z, y3.z);
    df_fma(s3, c3, x3.w, y3.w);
  }
  for (; q < nq; q += 32) {
    const float4 x = __ldg(a4 + q), y = w4[q];
    df_fma(s0, c0, x.x, y.x);
    df_fma(s1, c1, x.y, y.y);
    df_fma(s2, c2, x.z, y.z);
    df_fma(s3, c3, x.w, y.w);
  }
  for (int k = 4 * nq + lane; k < len; k += 32) df_fma(s0, c0, __ldg(a + k), ws[k]);
  return ((double(s0) + double(c0)) + (double(s1) + double(c1))) + ((double(s2) + double(c2)) + (double(s3) + double(c3)));
}

// w . w over one chunk by one warp, double-float sums
__device__ __forceinline__ double dot_self_df(const float* ws, int len, int lane) {
  float s = 0.0f, c = 0.0f;
  for (int k = lane; k < len; k += 32) df_fma(s, c, ws[k], ws[k]);
  return double(s) + double(c);
}

// x (FP64) += sum_{i<m} y[i] V_i for FP32 basis vectors: the sum in double-float on the FP32 units
// (y split into FP32 hi + lo parts, exact products, compensated sums), then one FP64 add per entry.
// The FP64 form of this loop (combine_kernel) is bound by the FP64 pipe.
__global__ void combine_df_kernel(const float* __restrict__ V, int64_t ldv, int m, const double* __restrict__ y,
                                  double* __restrict__ x, int64_t N) {
  __shared__ float yh[KRY_MAXV], yl[KRY_MAXV];
  if (threadIdx.x < m) {
    const double v = y[threadIdx.x];
    yh[threadIdx.x] = float(v);
    yl[threadIdx.x] = float(v - double(float(v)));
  }
  __syncthreads();
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x) {
    float s = 0.0f, c = 0.0f;
#pragma unroll 4
    for (int i = 0; i < m; ++i) {
      const float v = __ldg(V + i * ldv + k);
      df_fma(s, c, yh[i], v);
      c = fmaf(yl[i], v, c);
    }
    x[k] += double(s) + double(c);
  }
}

// w_k - sum_{i<m} h_i V_i[k] in double-float (h split into FP32 hi + lo parts), rounded to FP32
__device__ __forceinline__ float update_df(float wk, const float* __restrict__ vp, int64_t ldv, int m,
                                           const float* hh, const float* hl) {
  float s = wk, c = 0.0f;
#pragma unroll 4
  for (int i = 0; i < m; ++i) {
    const float v = __ldg(vp + i * ldv);
    df_fma(s, c, -hh[i], v);
    c = fmaf(-hl[i], v, c);
  }
  return s + c;
}

// w_k -= sum_i h_i V_i[k] for the chunk's elements k, four elements per thread at a time with the
// basis vectors outermost (four independent loads per vector in flight); each element's arithmetic is
// that of update_df.  Adds |w'|^2 to (ns, nc).
__device__ __forceinline__ void update_chunk_df(float* __restrict__ w, const float* __restrict__ V, int64_t k0,
                                                int len, int64_t ldv, int m, const float* hh, const float* hl,
                                                int nthreads, float& ns, float& nc) {
  int k = threadIdx.x;
  for (; k + 3 * nthreads < len; k += 4 * nthreads) {
    float s[4], c[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      s[q] = w[k0 + k + q * nthreads];
      c[q] = 0.0f;
    }
    const float* vp = V + k0 + k;
#pragma unroll 2
    for (int i = 0; i < m; ++i) {
      float v[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) v[q] = __ldg(vp + i * ldv + q * nthreads);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        df_fma(s[q], c[q], -hh[i], v[q]);
        c[q] = fmaf(-hl[i], v[q], c[q]);
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float vs = s[q] + c[q];
      w[k0 + k + q * nthreads] = vs;
      df_fma(ns, nc, vs, vs);
    }
  }
  for (; k < len; k += nthreads) {
    const float vs = update_df(w[k0 + k], V + k0 + k, ldv, m, hh, hl);
    w[k0 + k] = vs;
    df_fma(ns, nc, vs, vs);
  }
}

template <typename TV>
__device__ __forceinline__ double dot_chunk(const TV* __restrict__ a, const double* ws, int len, int lane, bool pairs) {
  double acc0 = 0.0, acc1 = 0.0, acc2 = 0.0, acc3 = 0.0;
  int k = 0;
  if (pairs) {
    using TV2 = typename std::conditional<sizeof(TV) == 8, double2, float2>::type;
    const TV2* a2 = reinterpret_cast<const TV2*>(a);
    const int np = len >> 1;
    int p = lane;
    // four pairs per lane and step: eight loads in flight per warp (the loop is latency-bound)
    for (; p + 96 < np; p += 128) {
      const TV2 u = __ldg(a2 + p), v = __ldg(a2 + p + 32), u2 = __ldg(a2 + p + 64), v2 = __ldg(a2 + p + 96);
      acc0 += double(u.x) * ws[2 * p];
      acc1 += double(u.y) * ws[2 * p + 1];
      acc2 += double(v.x) * ws[2 * p + 64];
      acc3 += double(v.y) * ws[2 * p + 65];
      acc0 += double(u2.x) * ws[2 * p + 128];
      acc1 += double(u2.y) * ws[2 * p + 129];
      acc2 += double(v2.x) * ws[2 * p + 192];
      acc3 += double(v2.y) * ws[2 * p + 193];
    }
    for (; p + 32 < np; p += 64) {
      const TV2 u = __ldg(a2 + p), v = __ldg(a2 + p + 32);
      acc0 += double(u.x) * ws[2 * p];
      acc1 += double(u.y) * ws[2 * p + 1];
      acc2 += double(v.x) * ws[2 * p + 64];
      acc3 += double(v.y) * ws[2 * p + 65];
    }
    for (; p < np; p += 32) {
      const TV2 u = __ldg(a2 + p);
      acc0 += double(u.x) * ws[2 * p];
      acc1 += double(u.y) * ws[2 * p + 1];
    }
    k = 2 * np + lane;
  } else {
    k = lane;
  }
  for (; k < len; k += 32) acc0 += double(__ldg(a + k)) * ws[k];
  return (acc0 + acc1) + (acc2 + acc3);
}

// Launch shape of the single-problem Krylov kernels: one wave of blocks (the kernel's occupancy
// times the SM count), block b on the contiguous range [b per, (b+1) per) of `unit`-entry units.  A
// grid of fixed-size chunks left a partial second wave (512 chunks of a 2^20-entry vector on 456
// resident blocks).  The grid never exceeds the chunk count the partial-sum scratch is sized for.
struct KryShape {
  int grid;
  int64_t per;
};

static KryShape kry_shape(int64_t N, int unit, int wave) {
  const int64_t nchunks = std::max<int64_t>(1, (N + KRY_CHUNK - 1) / KRY_CHUNK);
  const int64_t nu = std::max<int64_t>(1, (N + unit - 1) / unit);
  int64_t g = std::min<int64_t>(nchunks, wave > 0 ? wave : nchunks);
  const int64_t per = (nu + g - 1) / g;
  g = (nu + per - 1) / per;  // every block has units
  return {(int)g, per};
}

// blocks of LB_THREADS threads of `kernel` resident at once on the current device, cached per
// device ordinal and kernel slot (0 when the query fails: kry_shape then uses one block per chunk)
constexpr int KRY_WAVE_SLOTS = 4;  // multidot FP64, FP32; update FP64, FP32
template <typename K>
static int kry_wave(K kernel, int slot) {
  static std::atomic<int> cache[KRY_WAVE_SLOTS][128];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  const bool cached = dev >= 0 && dev < 128 && slot >= 0 && slot < KRY_WAVE_SLOTS;
  if (cached) {
    const int v = cache[slot][dev].load(std::memory_order_relaxed);
    if (v > 0) return v;
  }
  int nsm = 0, bps = 0;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kernel, LB_THREADS, 0) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  const int v = std::max(1, nsm) * std::max(1, bps);
  if (cached) cache[slot][dev].store(v, std::memory_order_relaxed);
  return v;
}

// dots of w with V_0..V_{m-1} (+ w.w): block b takes the range [b per, (b+1) per) (per a multiple of 64,
// so V_i + k0 stays 16-byte aligned when ldv is even for FP64, a multiple of 4 for FP32), staged
// through shared memory in equal sub-chunks of at most KRY_CHUNK entries.  One basis vector per warp,
// streamed with four 16-byte loads per lane in flight, its partial sum kept per lane across the
// sub-chunks; w.w is summed by every
// thread while it stages w.  The last block sums the blocks' partials in block order.  out[i] for
// i < m is the dot with V_i, out[m] (with_ww) is w.w.  (Measured on 2^20 entries against a variant
// that keeps all basis vectors' sums per lane over 16-byte units: as fast up to 8 vectors, faster
// beyond, in FP64 and FP32.)
template <typename TV>
__global__ void __launch_bounds__(LB_THREADS) multidot_lb_kernel(const TV* __restrict__ V, int64_t ldv, int m,
                                                                 const TV* __restrict__ w, int64_t N, int64_t per,
                                                                 int with_ww, double* __restrict__ partial,
                                                                 unsigned int* counter, double* out,
                                                                 const double* vs, const int* done,
                                                                 const int* need) {
  if (kry_skip(done, need)) return;
  constexpr int NW = LB_THREADS / 32;
  constexpr int NQ = (KRY_MAXV + NW - 1) / NW;  // basis vectors per warp
  __shared__ unsigned int ticket;
  __shared__ double red[NW];
  const int nb = gridDim.x;
  const int64_t beg = (int64_t)blockIdx.x * per;
  const int64_t end = beg + per < N ? beg + per : N;
  const int64_t nsub = (per + KRY_CHUNK - 1) / KRY_CHUNK;
  const int64_t sub = ((per + nsub - 1) / nsub + 63) / 64 * 64;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool pairs = ((ldv & 1) == 0);
  const bool quads = ((ldv & 3) == 0);  // FP32: V_i + k0 16-byte aligned (k0 is a multiple of 64)
  double acc[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) acc[q] = 0.0;
  double ww = 0.0;
  if constexpr (sizeof(TV) == 4) {
    __shared__ __align__(16) float wsf[KRY_CHUNK];
    float ss = 0.0f, sc = 0.0f;
    for (int64_t k0 = beg; k0 < end; k0 += sub) {
      const int len = (int)(end - k0 < sub ? end - k0 : sub);
      __syncthreads();  // the previous sub-chunk's reads of wsf are done
      for (int k = threadIdx.x; k < len; k += LB_THREADS) {
        const float wv = w[k0 + k];
        wsf[k] = wv;
        df_fma(ss, sc, wv, wv);
      }
      __syncthreads();
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        const int i = warp + q * NW;
        if (i < m)
          acc[q] += quads ? dot_chunk_df4(V + i * ldv + k0, wsf, len, lane)
                          : dot_chunk_df(V + i * ldv + k0, wsf, len, lane, pairs);
      }
    }
    ww = double(ss) + double(sc);
  } else {
    __shared__ double ws[KRY_CHUNK];
    for (int64_t k0 = beg; k0 < end; k0 += sub) {
      const int len = (int)(end - k0 < sub ? end - k0 : sub);
      __syncthreads();
      for (int k = threadIdx.x; k < len; k += LB_THREADS) {
        const double wv = double(w[k0 + k]);
        ws[k] = wv;
        ww += wv * wv;
      }
      __syncthreads();
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        const int i = warp + q * NW;
        if (i < m) acc[q] += dot_chunk<TV>(V + i * ldv + k0, ws, len, lane, pairs);
      }
    }
  }
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const int i = warp + q * NW;
    if (i < m) {  // warp-uniform
      const double v = warp_sum(acc[q]);
      if (lane == 0) partial[(size_t)i * nb + blockIdx.x] = v;
    }
  }
  if (with_ww) {
    ww = warp_sum(ww);
    if (lane == 0) red[warp] = ww;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int q = 0; q < NW; ++q) t += red[q];
      partial[(size_t)m * nb + blockIdx.x] = t;
    }
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) ticket = atomicAdd(counter, 1u);
  __syncthreads();
  if (ticket != (unsigned)(nb - 1)) return;
  __threadfence();
  const int mt = m + (with_ww ? 1 : 0);
  for (int i = warp; i < mt; i += NW) {
    double v0 = 0.0, v1 = 0.0;
    int c = lane;
    for (; c + 32 < nb; c += 64) {
      v0 += __ldcg(partial + (size_t)i * nb + c);
      v1 += __ldcg(partial + (size_t)i * nb + c + 32);
    }
    for (; c < nb; c += 32) v0 += __ldcg(partial + (size_t)i * nb + c);
    const double v = warp_sum(v0 + v1);
    if (lane == 0) out[i] = vs && i < m ? vs[i] * v : v;
  }
  if (threadIdx.x == 0) *counter = 0u;
}

// w -= V h; |w|^2 finished by the last block, which then runs the Arnoldi control (pass 1: decide on
// re-orthogonalisation or finalise the column; pass 2: add the second coefficients and finalise)
template <typename TV>
__global__ void __launch_bounds__(LB_THREADS) update_lb_kernel(const TV* __restrict__ V, int64_t ldv, int j,
                                                                TV* __restrict__ w, int64_t N, int64_t per,
                                                                double* __restrict__ partial, GmresDev* G,
                                                                int pass) {
  if (kry_skip(&G->done, pass == 2 ? &G->reorth : nullptr)) return;
  const int m = j + 1;
  const int nb = gridDim.x;
  __shared__ double hs[KRY_MAXV];
  __shared__ double red[LB_THREADS / 32];
  __shared__ unsigned int ticket;
  const double* h = pass == 1 ? G->h1 : G->h2;
  if (threadIdx.x < m) hs[threadIdx.x] = h[threadIdx.x] * G->vs[threadIdx.x];  // w -= sum h_i v_i
  __syncthreads();
  const int64_t k0 = (int64_t)blockIdx.x * per;  // the block's range [k0, k0 + len)
  const int len = (int)((N - k0) < per ? (N - k0) : per);
  double nrm = 0.0;
  if constexpr (sizeof(TV) == 4) {
    __shared__ float hh[KRY_MAXV], hl[KRY_MAXV];
    if (threadIdx.x < m) {
      hh[threadIdx.x] = float(hs[threadIdx.x]);
      hl[threadIdx.x] = float(hs[threadIdx.x] - double(float(hs[threadIdx.x])));
    }
    __syncthreads();
    float ns = 0.0f, nc = 0.0f;
    update_chunk_df(reinterpret_cast<float*>(w), reinterpret_cast<const float*>(V), k0, len, ldv, m, hh, hl,
                    LB_THREADS, ns, nc);
    nrm = double(ns) + double(nc);
  } else {
    // four elements per thread at a time, the basis vectors outermost: four independent loads per
    // vector in flight (the loop is latency-bound)
    int k = threadIdx.x;
    for (; k + 3 * LB_THREADS < len; k += 4 * LB_THREADS) {
      double v0 = double(w[k0 + k]), v1 = double(w[k0 + k + LB_THREADS]);
      double v2 = double(w[k0 + k + 2 * LB_THREADS]), v3 = double(w[k0 + k + 3 * LB_THREADS]);
      const TV* vp = V + k0 + k;
#pragma unroll 2
      for (int i = 0; i < m; ++i) {
        const TV* vi = vp + i * ldv;
        const double hi = hs[i];
        v0 -= hi * double(__ldg(vi));
        v1 -= hi * double(__ldg(vi + LB_THREADS));
        v2 -= hi * double(__ldg(vi + 2 * LB_THREADS));
        v3 -= hi * double(__ldg(vi + 3 * LB_THREADS));
      }
      const TV s0 = TV(v0), s1 = TV(v1), s2 = TV(v2), s3 = TV(v3);
      w[k0 + k] = s0;
      w[k0 + k + LB_THREADS] = s1;
      w[k0 + k + 2 * LB_THREADS] = s2;
      w[k0 + k + 3 * LB_THREADS] = s3;
      nrm += double(s0) * double(s0) + double(s1) * double(s1) + double(s2) * double(s2) + double(s3) * double(s3);
    }
    for (; k < len; k += LB_THREADS) {
      double v = double(w[k0 + k]);
      const TV* vp = V + k0 + k;
#pragma unroll 4
      for (int i = 0; i < m; ++i) v -= hs[i] * double(__ldg(vp + i * ldv));
      const TV vs = TV(v);
      w[k0 + k] = vs;
      nrm += double(vs) * double(vs);
    }
  }
  nrm = warp_sum(nrm);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = nrm;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < LB_THREADS / 32; ++q) t += red[q];
    partial[blockIdx.x] = t;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) ticket = atomicAdd(&G->counter, 1u);
  __syncthreads();
  if (ticket != (unsigned)(nb - 1)) return;
  __threadfence();
  const int lane = threadIdx.x & 31;
  if (threadIdx.x < 32) {
    double v0 = 0.0, v1 = 0.0;
    int c = lane;
    for (; c + 32 < nb; c += 64) {
      v0 += __ldcg(partial + c);
      v1 += __ldcg(partial + c + 32);
    }
    for (; c < nb; c += 32) v0 += __ldcg(partial + c);
    double v = warp_sum(v0 + v1);
    if (lane == 0) {
      G->counter = 0u;
      G->nrm = v;
      const int M = KRY_MAXV;
      if (pass == 1) {
        for (int i = 0; i <= j; ++i) G->H[i * M + j] = G->h1[i];
        if (v < 0.5 * G->h1[j + 1]) {
          G->reorth = 1;  // |w'| < |w| / sqrt(2): second Gram--Schmidt pass
        } else {
          G->reorth = 0;
          gmres_finalize_column(G, j);
        }
      } else {
        for (int i = 0; i <= j; ++i) G->H[i * M + j] += G->h2[i];
        G->reorth = 0;
        gmres_finalize_column(G, j);
      }
    }
  }
}

// the multi-dot of w with m basis vectors (+ w.w) over one wave of blocks
template <typename TV>
static void launch_multidot(const TV* V, int64_t ldv, int m, const TV* w, int64_t N, int with_ww, double* partial,
                            unsigned int* counter, double* out, const double* vs, const int* done, const int* need,
                            cudaStream_t s) {
  const KryShape sh = kry_shape(N, 64, kry_wave(multidot_lb_kernel<TV>, sizeof(TV) == 8 ? 0 : 1));
  multidot_lb_kernel<TV><<<sh.grid, LB_THREADS, 0, s>>>(V, ldv, m, w, N, sh.per * 64, with_ww, partial, counter, out,
                                                         vs, done, need);
}

// w -= V h (pass 1 or 2) over one wave of blocks, ranges in multiples of 64 entries
template <typename TV>
static void launch_update(const TV* V, int64_t N, int j, TV* w, double* partial, GmresDev* G, int pass,
                          cudaStream_t s) {
  const KryShape sh = kry_shape(N, 64, kry_wave(update_lb_kernel<TV>, sizeof(TV) == 8 ? 2 : 3));
  update_lb_kernel<TV><<<sh.grid, LB_THREADS, 0, s>>>(V, N, j, w, N, sh.per * 64, partial, G, pass);
}

// the occupancy queries of the pass kernels, run outside any stream capture (gmres_cycle)
template <typename TV>
static void kry_warm() {
  kry_wave(multidot_lb_kernel<TV>, sizeof(TV) == 8 ? 0 : 1);
  kry_wave(update_lb_kernel<TV>, sizeof(TV) == 8 ? 2 : 3);
}

// y = R^-1 g by back substitution over the jdone columns of the rotated Hessenberg matrix, then the
// combination coefficients y_i vs_i of the stored (unnormalised) basis vectors, into h2 (one thread:
// at most KRY_MAXV unknowns)
__global__ void gmres_solve_kernel(GmresDev* G) {
  if (threadIdx.x != 0) return;
  const int jd = G->jdone;
  double* y = G->h2;
  for (int i = jd - 1; i >= 0; --i) {
    double v = G->g[i];
    for (int k = i + 1; k < jd; ++k) v -= G->H[i * KRY_MAXV + k] * y[k];
    y[i] = v / G->H[i * KRY_MAXV + i];
  }
  for (int i = 0; i < jd; ++i) y[i] *= G->vs[i];  // x += sum y_i v_i = sum (y_i vs_i) V_i
}

size_t gmres_control_bytes() { return sizeof(GmresDev); }

// x <- 2 x - prev, prev <- old x
__global__ void extrapolate_kernel(double* __restrict__ x, double* __restrict__ prev, int64_t N) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x) {
    const double v = x[k];
    x[k] = 2.0 * v - prev[k];
    prev[k] = v;
  }
}

// G->misc[slot] = |v|^2 (one launch; its last block finishes the sum)
template <typename TV>
static void norm2_dev(sap_ctx* c, const TV* v, int slot, cudaStream_t s) {
  const int64_t N = c->N;
  GmresDev* G = reinterpret_cast<GmresDev*>(c->gdev);
  launch_multidot<TV>(nullptr, N, 0, v, N, 1, c->small, &G->counter, &G->misc[slot], nullptr, nullptr, nullptr, s);
  ++g_launches;
}

static cudaError_t fetch_misc(sap_ctx* c, cudaStream_t s) {
  GmresDev* G = reinterpret_cast<GmresDev*>(c->gdev);
  GmresDev* Gh = reinterpret_cast<GmresDev*>(c->gdev_host);
  cudaMemcpyAsync(Gh->misc, G->misc, sizeof(double) * 8, cudaMemcpyDeviceToHost, s);
  return cudaStreamSynchronize(s);
}

// Arnoldi iterations j0 .. j0+cnt-1 of the device-controlled GMRES on P^-1 A - 1 (TRANS: on
// P^-1 A^T - 1), A = 1 + dt/2 L, P its point-Jacobi diagonal (also that of A^T): apply,
// Gram--Schmidt with selective second pass, normalisation; launches after convergence return at
// once.  The group ends with the copy of the flags to the host.
template <typename TV, bool TRANS>
static cudaError_t enqueue_arnoldi(sap_ctx* c, const OpParams<TV>& PV, TV* V, double half, int j0, int cnt,
                                   cudaStream_t cs) {
  const int64_t N = c->N;
  double* partial = c->small;
  GmresDev* G = reinterpret_cast<GmresDev*>(c->gdev);
  GmresDev* Gh = reinterpret_cast<GmresDev*>(c->gdev_host);
  for (int j = j0; j < j0 + cnt; ++j) {
    TV* w = V + (size_t)(j + 1) * N;
    Epi<TV> e{};
    e.out = w; e.ax = TV(1); e.bl = TV(half); e.jacobi = 1; e.cj = TV(half); e.skip = &G->done;
    e.axpost = TV(-1);
    e.xs = &G->vs[j];  // the apply of v_j = vs[j] V_j
    cudaError_t e1;
    if constexpr (TRANS) e1 = launch_applyT<TV>(PV, V + (size_t)j * N, e, cs);
    else e1 = launch_apply<TV>(PV, V + (size_t)j * N, e, cs);
    if (e1 != cudaSuccess) return e1;
    launch_multidot<TV>(V, N, j + 1, w, N, 1, partial, &G->counter, G->h1, G->vs, &G->done, nullptr, cs);
    launch_update<TV>(V, N, j, w, partial, G, 1, cs);
    launch_multidot<TV>(V, N, j + 1, w, N, 0, partial, &G->counter, G->h2, G->vs, &G->done, &G->reorth, cs);
    launch_update<TV>(V, N, j, w, partial, G, 2, cs);
    g_launches += 4;
  }
  cudaMemcpyAsync(&Gh->done, &G->done, sizeof(int) * 4, cudaMemcpyDeviceToHost, cs);
  return cudaGetLastError();
}

// A group's launches as a CUDA graph (one launch instead of 6 per iteration), captured once on a
// private stream for this operator (forward or transposed), dt, field set and workspace; nullptr
// (direct launches) if capture fails.
template <typename TV, bool TRANS>
static cudaGraphExec_t arnoldi_graph(sap_ctx* c, const OpParams<TV>& PV, TV* V, double alpha, int j0, int cnt) {
  const int kind = TRANS ? 1 : 0;
  const void* ws = static_cast<const void*>(V);
  if (!c->cn_graphs.empty()) {
    const auto& g0 = c->cn_graphs.front();
    if (g0.alpha != alpha || g0.fields_version != c->fields_version || g0.ws != ws) cn_graphs_release(c);
  }
  for (const auto& gg : c->cn_graphs)
    if (gg.kind == kind && gg.j0 == j0 && gg.cnt == cnt) return gg.exec;
  if (!c->cap_stream && cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    c->cap_stream = nullptr;
    cudaGetLastError();
    return nullptr;
  }
  const int64_t l0 = g_launches;
  cudaGraph_t graph = nullptr;
  if (cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  const cudaError_t e1 = enqueue_arnoldi<TV, TRANS>(c, PV, V, alpha, j0, cnt, c->cap_stream);
  const cudaError_t e2 = cudaStreamEndCapture(c->cap_stream, &graph);
  g_launches = l0;
  cudaGraphExec_t ex = nullptr;
  if (e1 != cudaSuccess || e2 != cudaSuccess || !graph || cudaGraphInstantiate(&ex, graph, 0) != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return nullptr;
  }
  cudaGraphDestroy(graph);
  sap_ctx::CnGraph gg;
  gg.exec = ex; gg.kind = kind; gg.j0 = j0; gg.cnt = cnt; gg.fields_version = c->fields_version; gg.alpha = alpha;
  gg.ws = ws;
  c->cn_graphs.push_back(gg);
  return ex;
}

// One restart cycle of the device-controlled GMRES, from V_0 = P^-1 r of norm beta (not yet
// normalised): groups of Arnoldi iterations until the device flags convergence (|g_{j+1}| <= target)
// or the cycle length mlen, then y = R^-1 g by back substitution on the host and x += V y.
// *jd = the cycle's iterations.
template <typename TV, bool TRANS>
static cudaError_t gmres_cycle(sap_ctx* c, const OpParams<TV>& PV, TV* V, double alpha, double beta, double target,
                               int mlen, double* x, cudaStream_t s, int* jd, int cyc) {
  const int64_t N = c->N;
  GmresDev* G = reinterpret_cast<GmresDev*>(c->gdev);
  GmresDev* Gh = reinterpret_cast<GmresDev*>(c->gdev_host);
  // iterations enqueued between host checks: the first group as long as the last converged cycle
  // (iterations after convergence still launch and return at once), then groups of `group`
  const int group = 6, later = 3;
  int dummy = 0;
  int& hint = cyc >= 0 && cyc < 4 ? c->gm_hint[TRANS ? 1 : 0][cyc] : dummy;
  cudaError_t err = cudaSuccess;
  *jd = 0;
  kry_warm<TV>();  // the occupancy queries run here, not inside a graph capture
  Gh->g[0] = beta;
  Gh->beta = beta;
  Gh->inv_norm = 1.0 / beta;
  Gh->vs[0] = 1.0 / beta;  // V_0 = P^-1 r stays as it is: v_0 = V_0 / beta
  Gh->target = target;
  Gh->done = 0;
  Gh->reorth = 0;
  Gh->jdone = 0;
  Gh->m = mlen;
  if ((err = cudaMemcpyAsync(&G->g[0], &Gh->g[0], sizeof(double), cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return err;
  if ((err = cudaMemcpyAsync(&G->inv_norm, &Gh->inv_norm, sizeof(double) * 4, cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return err;
  if ((err = cudaMemcpyAsync(&G->done, &Gh->done, sizeof(int) * 4, cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return err;
  if ((err = cudaMemcpyAsync(&G->vs[0], &Gh->vs[0], sizeof(double), cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return err;
  for (int j0 = 0; j0 < mlen;) {
    const int want = j0 == 0 ? (hint > 0 ? hint : group) : (hint > 0 ? later : group);
    const int cnt = std::min(want, mlen - j0);
    cudaGraphExec_t ex = arnoldi_graph<TV, TRANS>(c, PV, V, alpha, j0, cnt);
    if (ex) {
      err = cudaGraphLaunch(ex, s);
      g_launches += 5 * cnt;
    } else {
      err = enqueue_arnoldi<TV, TRANS>(c, PV, V, alpha, j0, cnt, s);
    }
    if (err != cudaSuccess) return err;
    if ((err = cudaStreamSynchronize(s)) != cudaSuccess) return err;
    j0 += cnt;
    if (Gh->done) break;
  }
  const int jdone = Gh->jdone;
  // a cycle that converged before its length sets the next first group
  if (jdone > 0 && jdone < mlen) hint = std::min(jdone, KRY_MAXV - 1);
  // y = R^-1 g on the device (no copy of H to the host and back), then x += V y
  gmres_solve_kernel<<<1, 32, 0, s>>>(G);
  ++g_launches;
  if constexpr (sizeof(TV) == 4) combine_df_kernel<<<1024, KRY_THREADS, 0, s>>>(V, N, jdone, G->h2, x, N);
  else combine_kernel<TV><<<1024, KRY_THREADS, 0, s>>>(V, N, jdone, G->h2, x, N);
  ++g_launches;
  *jd = jdone;
  return cudaGetLastError();
}

// TV = double: FP64 operator and Krylov vectors (the plain path).  TV = float: precision form: the
// Arnoldi process applies the FP32 operator to FP32 vectors (double-float accumulation in dots and
// updates) inside the FP64 residual / refinement loop, each cycle asking for no more than the FP32
// operator can deliver (1e-6).
template <typename TV>
static sap_status cn_steps_t(sap_ctx* c, double* state, double dt, double theta, int nsteps, double tol, int restart,
                             int maxit, sap_solver_stats* st, cudaStream_t s) {
  const int64_t N = c->N;
  const int m = restart;
  constexpr bool f64 = sizeof(TV) == 8;
  TV* V = f64 ? reinterpret_cast<TV*>(c->ws64) : reinterpret_cast<TV*>(c->ws32);  // (m+1) vectors
  double* b = f64 ? c->ws64 + (size_t)(m + 1) * N : c->ws64;
  double* tmp = b + N;
  double* prev = c->ws64 + (size_t)(c->ws64_count - 1) * N;  // state before the last step
  const OpParams<TV>& PV = *reinterpret_cast<const OpParams<TV>*>(f64 ? (const void*)&c->p64 : (const void*)&c->p32);
  GmresDev* Gh = reinterpret_cast<GmresDev*>(c->gdev_host);
  const OpParams<double>& P = c->p64;
  // theta-method: A = 1 + alpha L, B = 1 - brhs L (alpha = theta dt, brhs = (1 - theta) dt)
  const double alpha = theta * dt, brhs = (1.0 - theta) * dt;
  int64_t total_its = 0;
  const int64_t launches0 = g_launches;
  int max_its = 0;
  double last_rel = 0.0;
  cudaError_t err = cudaSuccess;
  auto jcopy = [&](Epi<double>& e) {  // Jacobi-scaled copy of the residual into V_0
    if constexpr (f64) e.outj = reinterpret_cast<double*>(V);
    else e.out32 = reinterpret_cast<float*>(V);
    e.cj = alpha;
  };
#define CK(x)                               \
  do {                                      \
    err = (x);                              \
    if (err != cudaSuccess) goto cuda_fail; \
  } while (0)
  for (int step = 0; step < nsteps; ++step) {
    // one apply gives b = zeta - dt/2 L zeta + dt s (Eq. system-matrix-rhs), the residual of the
    // initial guess zeta, r = b - A zeta = dt (s - L zeta), and its Jacobi-scaled copy in V_0
    const bool extrap = c->cn_prev_valid && c->cn_prev_ptr == state && c->cn_prev_dt == dt && c->cn_prev_theta == theta;
    if (!extrap) {
      Epi<double> e{};
      e.out = b; e.ax = 1.0; e.bl = -brhs; e.gs = dt;
      e.out2 = tmp; e.ax2 = 0.0; e.bl2 = -dt; e.gs2 = dt;
      jcopy(e);
      CK(launch_apply<double>(P, state, e, s));
      CK(cudaMemcpyAsync(prev, state, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
    } else {
      // initial guess 2 zeta^(n-1) - zeta^(n-2) (linear extrapolation; only the iteration count
      // depends on it), then r = b - A x0 and its Jacobi-scaled copy
      Epi<double> e{};
      e.out = b; e.ax = 1.0; e.bl = -brhs; e.gs = dt;
      CK(launch_apply<double>(P, state, e, s));
      extrapolate_kernel<<<1024, KRY_THREADS, 0, s>>>(state, prev, N);
      ++g_launches;
      Epi<double> e2{};
      e2.out = tmp; e2.bvec = b; e2.wb = 1.0; e2.ax = -1.0; e2.bl = -alpha;
      jcopy(e2);
      CK(launch_apply<double>(P, state, e2, s));
    }
    c->cn_prev_valid = true;
    c->cn_prev_ptr = state;
    c->cn_prev_dt = dt;
    c->cn_prev_theta = theta;
    norm2_dev<double>(c, b, 0, s);
    norm2_dev<double>(c, tmp, 1, s);
    norm2_dev<TV>(c, V, 2, s);
    CK(fetch_misc(c, s));
    const double bnorm = std::sqrt(Gh->misc[0]);
    double rel = bnorm > 0 ? std::sqrt(Gh->misc[1]) / bnorm : 0.0;
    double beta = std::sqrt(Gh->misc[2]);
    int its = 0;
    if (bnorm == 0.0) {
      CK(cudaMemsetAsync(state, 0, sizeof(double) * N, s));
      continue;
    }
    if (!std::isfinite(bnorm)) rel = bnorm;  // reported as not converged below
    for (int cyc = 0; !(rel <= tol) && its < maxit && std::isfinite(rel); ++cyc) {
      const double target = f64 ? 0.5 * beta * (tol / rel) : beta * std::max(0.5 * tol / rel, 1e-6);
      int jd = 0;
      CK((gmres_cycle<TV, false>(c, PV, V, alpha, beta, target, std::min(m, maxit - its), state, s, &jd, cyc)));
      its += jd;
      // true residual r = b - A zeta and its Jacobi-scaled copy (start of a further cycle)
      {
        Epi<double> e{};
        e.out = tmp; e.bvec = b; e.wb = 1.0; e.ax = -1.0; e.bl = -alpha;
        jcopy(e);
        CK(launch_apply<double>(P, state, e, s));
      }
      norm2_dev<double>(c, tmp, 1, s);
      norm2_dev<TV>(c, V, 2, s);
      CK(fetch_misc(c, s));
      rel = std::sqrt(Gh->misc[1]) / bnorm;
      beta = std::sqrt(Gh->misc[2]);
      if (jd == 0) break;
    }
    total_its += its;
    max_its = std::max(max_its, its);
    last_rel = rel;
    if (!(rel <= tol)) {  // also catches a NaN residual
      c->err = "cn: GMRES did not reach the tolerance within maxit";
      if (st) {
        st->steps = step + 1; st->iterations = total_its; st->max_iterations = max_its; st->last_rel_residual = rel;
        st->kernel_launches = g_launches - launches0;
      }
      return SAP_ENOCONV;
    }
  }
  if (st) {
    st->steps = nsteps; st->iterations = total_its; st->max_iterations = max_its; st->last_rel_residual = last_rel;
    st->kernel_launches = g_launches - launches0;
  }
  return SAP_OK;
cuda_fail:
  c->err = std::string("cn: ") + cudaGetErrorString(err);
  return SAP_ECUDA;
#undef CK
}

sap_status cn_steps(sap_ctx* c, double* state, double dt, double theta, int nsteps, double tol, int restart,
                    int maxit, sap_solver_stats* st, cudaStream_t s) {
  return c->prec == SAP_PREC_FP64 ? cn_steps_t<double>(c, state, dt, theta, nsteps, tol, restart, maxit, st, s)
                                  : cn_steps_t<float>(c, state, dt, theta, nsteps, tol, restart, maxit, st, s);
}




// ================================================================================================
// Batches of independent problems (one launch per operator apply over all instances)
// ================================================================================================
template <typename T, int DT, int QT>
static cudaError_t launch_apply_batched_shape(const BatchDev<T>& B, const int* active, const T* x, const Epi<T>& e,
                                              cudaStream_t s) {
  static DeviceMask opted{};
  if (cudaError_t err = smem_opt_in(apply_kernel_batched<T, DT, QT>, 200 * 1024, opted); err != cudaSuccess)
    return err;
  apply_kernel_batched<T, DT, QT><<<B.nblocks, B.threads, B.smem, s>>>(B.P, B.doff, B.cpb, B.stride, B.blocks, active, x, e);
  ++g_launches;
  return cudaGetLastError();
}

// dynamic shared-memory limit of the batched apply kernel that runs B, set once per device
template <typename T>
static cudaError_t prepare_batched(const BatchDev<T>& B) {
  if (B.rows) return prepare_rows_batched<T>(B);
  static DeviceMask opted{};
  return smem_opt_in(apply_kernel_batched<T, 0, 0>, 200 * 1024, opted);
}
template <typename T>
static cudaError_t prepare_batched(const std::vector<BatchDev<T>>& Bs) {
  for (const auto& B : Bs)
    if (cudaError_t err = prepare_batched<T>(B); err != cudaSuccess) return err;
  return cudaSuccess;
}

template <typename T>
static cudaError_t launch_apply_batched(const BatchDev<T>& B, const int* active, const T* x, const Epi<T>& e,
                                        cudaStream_t s);

// one launch per group of instances with the same expansion order (each with its own tile shape)
template <typename T>
static cudaError_t launch_apply_batched(const std::vector<BatchDev<T>>& Bs, const int* active, const T* x,
                                        const Epi<T>& e, cudaStream_t s) {
  for (const auto& B : Bs) {
    if (B.nblocks == 0) continue;
    if (cudaError_t err = launch_apply_batched<T>(B, active, x, e, s); err != cudaSuccess) return err;
  }
  return cudaSuccess;
}

template <typename T>
static cudaError_t launch_apply_batched(const BatchDev<T>& B, const int* active, const T* x, const Epi<T>& e,
                                        cudaStream_t s) {
  if (B.smem > 200 * 1024 || B.threads > 1024 || B.threads < 1) return cudaErrorInvalidConfiguration;
  if (B.rows) return launch_rows_batched<T>(B, active, x, e, s);
  return launch_apply_batched_shape<T, 0, 0>(B, active, x, e, s);
}

// per-instance Krylov kernels: block b works on chunk b of instance chunks.inst[b]
template <typename TV>
__global__ void __launch_bounds__(KRY_THREADS) multidot_b_kernel(const TV* __restrict__ V, int64_t ldv, int m,
                                                                 const TV* __restrict__ w, int with_ww,
                                                                 BatchChunks C, const int* __restrict__ active,
                                                                 double* __restrict__ partial) {
  const int inst = C.inst[blockIdx.x];
  if (!active[inst]) return;
  const int64_t k0 = C.k0[blockIdx.x];
  const int len = C.len[blockIdx.x];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int mt = m + (with_ww ? 1 : 0);
  const bool pairs = ((ldv & 1) == 0) && ((k0 & 1) == 0);  // V_i + k0 stays 2-element aligned
  if constexpr (sizeof(TV) == 4) {
    __shared__ float wsf[KRY_CHUNK];
    for (int k = threadIdx.x; k < len; k += KRY_THREADS) wsf[k] = w[k0 + k];
    __syncthreads();
    for (int i = warp; i < mt; i += KRY_THREADS / 32) {
      double acc = i < m ? dot_chunk_df(V + i * ldv + k0, wsf, len, lane, pairs) : dot_self_df(wsf, len, lane);
      acc = warp_sum(acc);
      if (lane == 0) partial[(size_t)i * C.nchunks + blockIdx.x] = acc;
    }
  } else {
    __shared__ double ws[KRY_CHUNK];
    for (int k = threadIdx.x; k < len; k += KRY_THREADS) ws[k] = double(w[k0 + k]);
    __syncthreads();
    for (int i = warp; i < mt; i += KRY_THREADS / 32) {
      double acc;
      if (i < m) {
        acc = dot_chunk<TV>(V + i * ldv + k0, ws, len, lane, pairs);
      } else {
        acc = 0.0;
        for (int k = lane; k < len; k += 32) acc += ws[k] * ws[k];
      }
      acc = warp_sum(acc);
      if (lane == 0) partial[(size_t)i * C.nchunks + blockIdx.x] = acc;
    }
  }
}

// out[inst*stride + i] = sum over the instance's chunks of partial[i][chunk]; block = instance
__global__ void reduce_b_kernel(const double* __restrict__ partial, BatchChunks C, const int* __restrict__ active,
                                int m, double* __restrict__ out, int stride) {
  const int inst = blockIdx.x;
  if (!active[inst]) return;
  const int lane = threadIdx.x & 31, i = threadIdx.x >> 5;
  if (i >= m) return;
  const int c0 = C.first[inst], cn = C.count[inst];
  double v = 0.0;
  for (int c = lane; c < cn; c += 32) v += partial[(size_t)i * C.nchunks + c0 + c];
  v = warp_sum(v);
  if (lane == 0) out[(size_t)inst * stride + i] = v;
}

template <typename TV>
__global__ void __launch_bounds__(KRY_THREADS) update_b_kernel(const TV* __restrict__ V, int64_t ldv, int m,
                                                               const double* __restrict__ h, int hstride,
                                                               TV* __restrict__ w, BatchChunks C,
                                                               const int* __restrict__ active,
                                                               double* __restrict__ partial) {
  __shared__ double hs[KRY_MAXV];
  __shared__ double red[KRY_THREADS / 32];
  const int inst = C.inst[blockIdx.x];
  if (!active[inst]) return;
  if (threadIdx.x < m) hs[threadIdx.x] = h[(size_t)inst * hstride + threadIdx.x];
  __syncthreads();
  const int64_t k0 = C.k0[blockIdx.x];
  const int len = C.len[blockIdx.x];
  double nrm = 0.0;
  if constexpr (sizeof(TV) == 4) {
    __shared__ float hh[KRY_MAXV], hl[KRY_MAXV];
    if (threadIdx.x < m) {
      hh[threadIdx.x] = float(hs[threadIdx.x]);
      hl[threadIdx.x] = float(hs[threadIdx.x] - double(float(hs[threadIdx.x])));
    }
    __syncthreads();
    float ns = 0.0f, nc = 0.0f;
    update_chunk_df(reinterpret_cast<float*>(w), reinterpret_cast<const float*>(V), k0, len, ldv, m, hh, hl,
                    KRY_THREADS, ns, nc);
    nrm = double(ns) + double(nc);
  } else {
    for (int k = threadIdx.x; k < len; k += KRY_THREADS) {
      double v = double(w[k0 + k]);
      const TV* vp = V + k0 + k;
#pragma unroll 4
      for (int i = 0; i < m; ++i) v -= hs[i] * double(__ldg(vp + i * ldv));
      const TV vs = TV(v);
      w[k0 + k] = vs;
      nrm += double(vs) * double(vs);
    }
  }
  nrm = warp_sum(nrm);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = nrm;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < KRY_THREADS / 32; ++q) t += red[q];
    partial[blockIdx.x] = t;
  }
}

// y = x / sqrt(a[inst*stride]) on the active instances
template <typename TV>
__global__ void scale_b_kernel(const TV* x, TV* y, const double* __restrict__ a, int stride,
                               BatchChunks C, const int* __restrict__ active) {
  const int inst = C.inst[blockIdx.x];
  if (!active[inst]) return;
  const double av = a[(size_t)inst * stride];
  if (!(av > 0.0)) return;
  const double f = 1.0 / sqrt(av);
  const int64_t k0 = C.k0[blockIdx.x];
  const int len = C.len[blockIdx.x];  // in a register: the stores to y cannot change it
#pragma unroll 4
  for (int k = threadIdx.x; k < len; k += blockDim.x) y[k0 + k] = TV(f * double(x[k0 + k]));
}

// x (FP64) += sum_{i < mi[inst]} y[inst*stride + i] V_i
template <typename TV>
__global__ void combine_b_kernel(const TV* __restrict__ V, int64_t ldv, const int* __restrict__ mi,
                                 const double* __restrict__ y, int stride, double* __restrict__ x, BatchChunks C) {
  const int inst = C.inst[blockIdx.x];
  const int m = mi[inst];
  if (m <= 0) return;
  __shared__ double ys[KRY_MAXV];
  if (threadIdx.x < m) ys[threadIdx.x] = y[(size_t)inst * stride + threadIdx.x];
  __syncthreads();
  const int64_t k0 = C.k0[blockIdx.x];
  const int len = C.len[blockIdx.x];
  for (int k = threadIdx.x; k < len; k += blockDim.x) {
    double v = x[k0 + k];
    const TV* vp = V + k0 + k;
#pragma unroll 4
    for (int i = 0; i < m; ++i) v += ys[i] * double(__ldg(vp + i * ldv));
    x[k0 + k] = v;
  }
}

// zero the vectors of masked instances
template <typename T>
__global__ void zero_b_kernel(T* __restrict__ x, BatchChunks C, const int* __restrict__ mask) {
  const int inst = C.inst[blockIdx.x];
  if (!mask[inst]) return;
  const int64_t k0 = C.k0[blockIdx.x];
  const int len = C.len[blockIdx.x];
  for (int k = threadIdx.x; k < len; k += blockDim.x) x[k0 + k] = T(0);
}

template <typename V>
static void* dev_upload(sap_ctx* c, const std::vector<V>& h) {
  void* p = nullptr;
  const size_t bytes = std::max<size_t>(1, h.size()) * sizeof(V);
  if (cudaMalloc(&p, bytes) != cudaSuccess) throw std::string("cudaMalloc failed");
  if (!h.empty() && cudaMemcpy(p, h.data(), h.size() * sizeof(V), cudaMemcpyHostToDevice) != cudaSuccess)
    throw std::string("cudaMemcpy failed");
  c->batch_bufs.push_back({p, bytes});
  return p;
}

// Tables of a batch for the thread-block targets target[i] of every instance (the row kernel picks
// an instance's cells per block from its target and its n).
static void batch_tables(sap_ctx* c, const std::vector<int>& target) {
  for (auto& b : c->batch_bufs) cudaFree(b.p);
  c->batch_bufs.clear();
  const int ni = (int)c->sub.size();
  std::vector<OpParams<double>> P64(ni);
  std::vector<OpParams<float>> P32(ni);
  std::vector<int64_t> doff(ni);
  int sd = c->sub[0]->D, sq = c->sub[0]->q;
  for (auto* sc : c->sub)
    if (sc->D != sd || sc->q != sq) sd = sq = 0;
  const bool rows = sd > 0 && rows_supported(sd, sq);
  for (int i = 0; i < ni; ++i) {
    P64[i] = c->sub[i]->p64;
    P32[i] = c->sub[i]->p32;
    doff[i] = c->inst_off[i];
  }
  // instances are grouped by expansion order: each group is one launch with its own block size
  c->batch_class.assign(ni, 0);
  std::vector<int> lclass;
  for (int i = 0; i < ni; ++i) {
    const int l = c->sub[i]->desc.lmax;
    auto it = std::find(lclass.begin(), lclass.end(), l);
    c->batch_class[i] = (int)(it - lclass.begin());
    if (it == lclass.end()) lclass.push_back(l);
  }
  const int ncls = (int)lclass.size();
  // cells per block, block lists (per group), block sizes and shared memory for one precision
  auto plan = [&](auto tag, const auto& Pv, std::vector<int>& cpb, std::vector<int>& stride,
                  std::vector<std::vector<int2>>& blocks, std::vector<int>& threads, std::vector<size_t>& smem) {
    using T = decltype(tag);
    cpb.assign(ni, 1);
    stride.assign(ni, 0);
    blocks.assign(ncls, {});
    threads.assign(ncls, 1);
    smem.assign(ncls, 0);
    for (int i = 0; i < ni; ++i) {
      sap_ctx* sc = c->sub[i];
      const int g = c->batch_class[i];
      size_t sm = 0;
      if (rows) {
        rows_config<T>(Pv[i], target[i], &cpb[i], &sm);
        threads[g] = std::max(threads[g], cpb[i] * sc->n);
      } else {
        const int per = sc->n * sc->nloc;
        if (per > 1024) throw std::string("an instance has n (k+1)^D > 1024");
        cpb[i] = std::max(1, std::min(target[i], 1024) / per);
        stride[i] = cell_stride_elems(sc->p64);
        threads[g] = std::max(threads[g], cpb[i] * per);
        sm = (size_t)cpb[i] * stride[i] * sizeof(T);
      }
      smem[g] = std::max(smem[g], sm);
      for (int c0 = 0; c0 < sc->ncell; c0 += cpb[i]) blocks[g].push_back(make_int2(i, c0));
    }
  };
  std::vector<int> cpb64, cpb32, st64, st32, th64, th32;
  std::vector<std::vector<int2>> bl64, bl32;
  std::vector<size_t> sm64, sm32;
  plan(double{}, P64, cpb64, st64, bl64, th64, sm64);
  plan(float{}, P32, cpb32, st32, bl32, th32, sm32);
  std::vector<int> cinst, clen, cfirst(ni), ccount(ni);
  std::vector<int64_t> ck0;
  for (int i = 0; i < ni; ++i) {
    cfirst[i] = (int)cinst.size();
    const int64_t Ni = c->sub[i]->N;
    for (int64_t k = 0; k < Ni; k += KRY_CHUNK) {
      cinst.push_back(i);
      ck0.push_back(c->inst_off[i] + k);
      clen.push_back((int)std::min<int64_t>(KRY_CHUNK, Ni - k));
    }
    ccount[i] = (int)cinst.size() - cfirst[i];
  }
  const int64_t* d_doff = (const int64_t*)dev_upload(c, doff);
  const auto* dP64 = (const OpParams<double>*)dev_upload(c, P64);
  const auto* dP32 = (const OpParams<float>*)dev_upload(c, P32);
  const int* dcpb64 = (const int*)dev_upload(c, cpb64);
  const int* dcpb32 = (const int*)dev_upload(c, cpb32);
  const int* dst64 = (const int*)dev_upload(c, st64);
  const int* dst32 = (const int*)dev_upload(c, st32);
  c->b64.clear();
  c->b32.clear();
  for (int g = 0; g < ncls; ++g) {
    c->b64.push_back(BatchDev<double>{dP64, d_doff, dcpb64, dst64, (const int2*)dev_upload(c, bl64[g]),
                                      (int)bl64[g].size(), th64[g], sm64[g], sd, sq, rows ? 1 : 0});
    c->b32.push_back(BatchDev<float>{dP32, d_doff, dcpb32, dst32, (const int2*)dev_upload(c, bl32[g]),
                                     (int)bl32[g].size(), th32[g], sm32[g], sd, sq, rows ? 1 : 0});
  }
  c->chunks = BatchChunks{(const int*)dev_upload(c, cinst), (const int64_t*)dev_upload(c, ck0),
                          (const int*)dev_upload(c, clen), (const int*)dev_upload(c, cfirst),
                          (const int*)dev_upload(c, ccount), (int)cinst.size()};
  c->h_active.assign(3 * ni, 1);  // activity mask, combine lengths, zero mask
  c->d_active = (int*)dev_upload(c, c->h_active);
}

// Builds the batch tables.  On the first call the tile shape is autotuned per expansion order: for
// every candidate thread-block target the batched apply is timed with only the instances of one
// l_max active (the others' blocks return at once), and each l_max keeps its fastest target, i.e. its
// own cells per block.
sap_status batch_prepare(sap_ctx* c, cudaStream_t s) {
  int version = 0;
  for (auto* sc : c->sub) {
    if (!sc->fields_set) {
      c->err = "batch: fields not set on every instance";
      return SAP_EINVAL;
    }
    version += sc->fields_version;
  }
  if (version == c->batch_built_version) return SAP_OK;
  const int ni = (int)c->sub.size();
  try {
    if (!c->batch_tuned) {
      const size_t w = c->prec == SAP_PREC_FP64 ? 8 : 4;
      void *x = nullptr, *y = nullptr;
      if (cudaMalloc(&x, w * c->N) != cudaSuccess || cudaMalloc(&y, w * c->N) != cudaSuccess) {
        if (x) cudaFree(x);
        c->err = "batch: autotune allocation failed";
        return SAP_ENOMEM;
      }
      cudaMemsetAsync(x, 0, w * c->N, s);
      std::vector<int> lclass;  // distinct expansion orders
      for (auto* sc : c->sub)
        if (std::find(lclass.begin(), lclass.end(), sc->desc.lmax) == lclass.end()) lclass.push_back(sc->desc.lmax);
      const int cand[4] = {64, 128, 256, 512};
      std::vector<float> best(lclass.size(), 1e30f);
      std::vector<int> best_t(lclass.size(), 256);
      cudaEvent_t e0, e1;
      cudaEventCreate(&e0);
      cudaEventCreate(&e1);
      for (int target : cand) {
        batch_tables(c, std::vector<int>(ni, target));
        // the groups are launched one by one, so each is timed on its own launch
        for (size_t L = 0; L < lclass.size(); ++L) {
          const int g = c->batch_class[std::find_if(c->sub.begin(), c->sub.end(),
                                                    [&](sap_ctx* sc) { return sc->desc.lmax == lclass[L]; }) -
                                       c->sub.begin()];
          const int64_t l0 = g_launches;
          for (int rep = 0; rep < 4; ++rep) {
            if (rep == 1) cudaEventRecord(e0, s);
            cudaError_t err = c->prec == SAP_PREC_FP64
                                  ? launch_apply_batched<double>(c->b64[g], c->d_active, (const double*)x,
                                                                 Epi<double>{(double*)y, nullptr, 0, 0, 1, 0}, s)
                                  : launch_apply_batched<float>(c->b32[g], c->d_active, (const float*)x,
                                                                Epi<float>{(float*)y, nullptr, 0, 0, 1, 0}, s);
            if (err != cudaSuccess) break;
          }
          g_launches = l0;
          cudaEventRecord(e1, s);
          cudaEventSynchronize(e1);
          float ms = 1e30f;
          if (cudaGetLastError() == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
          if (ms < best[L]) {
            best[L] = ms;
            best_t[L] = target;
          }
        }
      }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      cudaStreamSynchronize(s);
      cudaFree(x);
      cudaFree(y);
      c->batch_targets.assign(ni, 256);
      for (int i = 0; i < ni; ++i)
        for (size_t L = 0; L < lclass.size(); ++L)
          if (c->sub[i]->desc.lmax == lclass[L]) c->batch_targets[i] = best_t[L];
      c->batch_tuned = true;
    }
    batch_tables(c, c->batch_targets);
  } catch (const std::string& e) {
    c->err = "batch: " + e;
    return SAP_ENOMEM;
  }
  c->batch_built_version = version;
  return SAP_OK;
}

sap_status batch_apply(sap_ctx* c, const void* x, void* y, int mode, cudaStream_t s) {
  sap_status st = batch_prepare(c, s);
  if (st != SAP_OK) return st;
  cudaError_t err;
  if (c->prec == SAP_PREC_FP64) {
    Epi<double> e = mode == SAP_APPLY_RHS ? epi_plain<double>((double*)y, 0, -1, 1) : epi_plain<double>((double*)y, 0, 1, 0);
    err = launch_apply_batched<double>(c->b64, c->d_active, (const double*)x, e, s);
  } else {
    Epi<float> e = mode == SAP_APPLY_RHS ? epi_plain<float>((float*)y, 0, -1, 1) : epi_plain<float>((float*)y, 0, 1, 0);
    err = launch_apply_batched<float>(c->b32, c->d_active, (const float*)x, e, s);
  }
  if (err != cudaSuccess) {
    c->err = std::string("batch apply: ") + cudaGetErrorString(err);
    return SAP_ECUDA;
  }
  return SAP_OK;
}

sap_status batch_erk(sap_ctx* c, double* state, double dt, int nsteps, cudaStream_t s) {
  sap_status st = batch_prepare(c, s);
  if (st != SAP_OK) return st;
  cudaError_t err = cudaSuccess;
  const int64_t N = c->N;
  auto run = [&](auto tag, const auto& B, auto* ya, auto* yb, double* acc) -> cudaError_t {
    using T = decltype(tag);
    for (int it = 0; it < nsteps; ++it) {
      const T* in0;
      if (sizeof(T) == 8) {
        in0 = reinterpret_cast<const T*>(state);
      } else {
        cast_kernel<T><<<1024, 256, 0, s>>>(state, ya, N);
        ++g_launches;
        in0 = ya;
      }
      Epi<T> e{};
      e.acc = acc;
      e.y0 = state;
      e.erk = 1; e.bdt = dt / 6.0; e.adt = 0.5 * dt; e.ynext = (sizeof(T) == 8) ? ya : yb;
      cudaError_t r = launch_apply_batched<T>(B, c->d_active, in0, e, s);
      if (r != cudaSuccess) return r;
      const T* in2 = e.ynext;
      T* out2 = (in2 == ya) ? yb : ya;
      e.erk = 2; e.bdt = dt / 3.0; e.adt = 0.5 * dt; e.ynext = out2;
      if ((r = launch_apply_batched<T>(B, c->d_active, in2, e, s)) != cudaSuccess) return r;
      const T* in3 = out2;
      T* out3 = (in3 == ya) ? yb : ya;
      e.erk = 2; e.bdt = dt / 3.0; e.adt = dt; e.ynext = out3;
      if ((r = launch_apply_batched<T>(B, c->d_active, in3, e, s)) != cudaSuccess) return r;
      e.erk = 3; e.bdt = dt / 6.0; e.ynext = nullptr; e.state = state;
      if ((r = launch_apply_batched<T>(B, c->d_active, out3, e, s)) != cudaSuccess) return r;
    }
    return cudaSuccess;
  };
  if (c->prec == SAP_PREC_FP64) err = run(double{}, c->b64, c->ws64, c->ws64 + N, c->ws64 + 2 * N);
  else err = run(float{}, c->b32, c->ws32, c->ws32 + N, c->ws64);
  if (err != cudaSuccess) {
    c->err = std::string("batch erk: ") + cudaGetErrorString(err);
    return SAP_ECUDA;
  }
  return SAP_OK;
}

// ------------------------------------------------------------------------------------------------
// Batched CN with per-instance GMRES control on the device, one CUDA-graph launch per step
// ------------------------------------------------------------------------------------------------
// Every instance runs its own restarted GMRES (own Krylov space, Hessenberg matrix, Givens rotations,
// convergence test).  The decisions the host used to take between launches (re-orthogonalisation,
// column finalisation, convergence, restart targets, back substitution) are taken by control kernels
// with one thread per instance, which write the per-instance masks that the batched kernels read, so
// a whole CN step is a fixed sequence of launches: it is captured once as a CUDA graph (per state
// buffer, dt, fields, workspace, initial-guess variant) and replayed with one launch per step.
// Launches that find every instance finished return at once.  The host reads the per-instance
// status once after the graph; instances that need more refinement cycles (rare) get one-cycle
// continuation graphs.
enum { BS_SOLVING = 0, BS_DONE = 1, BS_ZERO = 2, BS_STOPPED = 3 };

struct BCtl {
  double H[KRY_MAXV * (KRY_MAXV + 1)];  // H[i * KRY_MAXV + j]
  double g[KRY_MAXV + 1], cs[KRY_MAXV], sn[KRY_MAXV];
  double bnorm, rel, target;
  int its, status, jdone, pad;
};

struct BStat {  // per-instance status copied to the host after each graph
  double rel;
  int its, status;
};

struct BMasks {  // device masks read by the batched kernels, written by the control kernels
  int* act;      // instance still solving this step
  int* inner;    // instance active in the current Arnoldi iteration
  int* reo;      // instance needs the second Gram--Schmidt pass in this iteration
  int* mi;       // basis vectors to combine into the solution (0: none)
  int* zero;     // right side is zero: the state is set to zero
};

__global__ void bctl_init(BCtl* ctl, BMasks M, int ni) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ni; i += gridDim.x * blockDim.x) {
    ctl[i].its = 0;
    ctl[i].status = BS_SOLVING;
    ctl[i].rel = 0.0;
    M.act[i] = 1;
    M.inner[i] = 0;
    M.reo[i] = 0;
    M.mi[i] = 0;
    M.zero[i] = 0;
  }
}

// ||b|| from the dots (region 1, index 0); a zero right side finishes the instance at zero
__global__ void bctl_bnorm(BCtl* ctl, BMasks M, const double* dsc, int SS, int ni) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ni; i += gridDim.x * blockDim.x) {
    const double bn = sqrt(dsc[(size_t)i * SS + KRY_MAXV]);
    ctl[i].bnorm = bn;
    const bool z = bn == 0.0;
    M.zero[i] = z;
    M.act[i] = !z && isfinite(bn);
    if (z) ctl[i].status = BS_ZERO;
    if (!isfinite(bn)) {  // reported as not converged
      ctl[i].status = BS_STOPPED;
      ctl[i].rel = bn;
    }
  }
}

// true relative residual from the dots of r (region 1, index 0): converged, stopped or go on
__global__ void bctl_residual(BCtl* ctl, BMasks M, const double* dsc, int SS, int ni, double tol, int maxit) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ni; i += gridDim.x * blockDim.x) {
    if (!M.act[i]) continue;
    const double rel = sqrt(dsc[(size_t)i * SS + KRY_MAXV]) / ctl[i].bnorm;
    ctl[i].rel = rel;
    if (rel <= tol) {
      ctl[i].status = BS_DONE;
      M.act[i] = 0;
    } else if (ctl[i].its >= maxit || !isfinite(rel)) {
      ctl[i].status = BS_STOPPED;
      M.act[i] = 0;
    }
  }
}

// start of an Arnoldi cycle: beta = |P^-1 r| (region 1), g = beta e_1, the cycle's target
__global__ void bctl_beta(BCtl* ctl, BMasks M, const double* dsc, int SS, int ni, double tol, double floor_rel) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ni; i += gridDim.x * blockDim.x) {
    M.inner[i] = M.act[i];
    M.mi[i] = 0;
    if (!M.act[i]) continue;
    BCtl& C = ctl[i];
    const double beta = sqrt(dsc[(size_t)i * SS + KRY_MAXV]);
    for (int k = 0; k <= KRY_MAXV; ++k) C.g[k] = 0.0;
    C.g[0] = beta;
    C.jdone = 0;
    C.target = beta * fmax(0.5 * tol / C.rel, floor_rel);
    if (!(beta > 0.0)) M.inner[i] = 0;
  }
}

// after the first Gram--Schmidt pass of column j: h (region 0, j+1 values) into H; second pass when
// |w'| < |w| / sqrt(2) (|w|^2 at region 0 index j+1, |w'|^2 at region 1 index 0)
__global__ void bctl_reo(BCtl* ctl, BMasks M, const double* dsc, int SS, int ni, int j) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ni; i += gridDim.x * blockDim.x) {
    M.reo[i] = 0;
    if (!M.inner[i]) continue;
    const double* h = dsc + (size_t)i * SS;
    for (int k = 0; k <= j; ++k) ctl[i].H[k * KRY_MAXV + j] = h[k];
    M.reo[i] = h[KRY_MAXV] < 0.5 * h[j + 1];
  }
}

// after the second pass: its coefficients (region 2) added to column j
__global__ void bctl_addh2(BCtl* ctl, BMasks M, const double* dsc, int SS, int ni, int j) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ni; i += gridDim.x * blockDim.x) {
    if (!M.reo[i]) continue;
    const double* h2 = dsc + (size_t)i * SS + 2 * KRY_MAXV;
    for (int k = 0; k <= j; ++k) ctl[i].H[k * KRY_MAXV + j] += h2[k];
  }
}

// column j finalised: subdiagonal |w| (region 1), previous rotations, new rotation, residual
// estimate |g_{j+1}|; the instance leaves the cycle when it meets its target or maxit
__global__ void bctl_finalize(BCtl* ctl, BMasks M, const double* dsc, int SS, int ni, int j, int maxit) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ni; i += gridDim.x * blockDim.x) {
    if (!M.inner[i]) continue;
    BCtl& C = ctl[i];
    const int MM = KRY_MAXV;
    const double hn = sqrt(dsc[(size_t)i * SS + KRY_MAXV]);
    C.H[(j + 1) * MM + j] = hn;
    for (int k = 0; k < j; ++k) {
      const double a0 = C.H[k * MM + j], a1 = C.H[(k + 1) * MM + j];
      C.H[k * MM + j] = C.cs[k] * a0 + C.sn[k] * a1;
      C.H[(k + 1) * MM + j] = -C.sn[k] * a0 + C.cs[k] * a1;
    }
    const double a0 = C.H[j * MM + j], a1 = C.H[(j + 1) * MM + j];
    const double den = hypot(a0, a1);
    C.cs[j] = den > 0 ? a0 / den : 1.0;
    C.sn[j] = den > 0 ? a1 / den : 0.0;
    C.H[j * MM + j] = den;
    C.H[(j + 1) * MM + j] = 0.0;
    C.g[j + 1] = -C.sn[j] * C.g[j];
    C.g[j] = C.cs[j] * C.g[j];
    C.its += 1;
    C.jdone = j + 1;
    if (fabs(C.g[j + 1]) <= C.target || hn == 0.0 || C.its >= maxit) M.inner[i] = 0;
  }
}

// end of a cycle: y = R^-1 g (region 3) and the number of basis vectors to combine
__global__ void bctl_solve(BCtl* ctl, BMasks M, double* dsc, int SS, int ni) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ni; i += gridDim.x * blockDim.x) {
    M.mi[i] = 0;
    if (!M.act[i]) continue;
    BCtl& C = ctl[i];
    const int jd = C.jdone;
    double* y = dsc + (size_t)i * SS + 3 * KRY_MAXV;
    for (int k = jd - 1; k >= 0; --k) {
      double v = C.g[k];
      for (int l = k + 1; l < jd; ++l) v -= C.H[k * KRY_MAXV + l] * y[l];
      y[k] = v / C.H[k * KRY_MAXV + k];
    }
    M.mi[i] = jd;
  }
}

__global__ void bctl_status(const BCtl* ctl, BStat* out, int ni) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ni; i += gridDim.x * blockDim.x) {
    out[i].rel = ctl[i].rel;
    out[i].its = ctl[i].its;
    out[i].status = ctl[i].status;
  }
}

template <typename TV>
struct BatchGraphArgs {
  double* state;
  double *b, *r, *prev;
  TV* V;
  double dt;
  double tol;
  int m, maxit;
};

// the launches of one refinement cycle (Arnoldi from the prepared V_0, solution update, new
// residual and decision), or of the start of a step (right side, initial guess, first residual)
template <typename TV>
static cudaError_t batch_enqueue(sap_ctx* c, const BatchGraphArgs<TV>& A, int what, int extrap, cudaStream_t s) {
  const int64_t N = c->N;
  const int ni = (int)c->sub.size();
  const BatchChunks& C = c->chunks;
  double* partial = c->small;
  const int SS = 4 * KRY_MAXV;
  double* dsc = c->small + (size_t)(KRY_MAXV + 1) * C.nchunks;
  BCtl* ctl = reinterpret_cast<BCtl*>(c->bctl);
  BMasks M{c->bmask, c->bmask + ni, c->bmask + 2 * ni, c->bmask + 3 * ni, c->bmask + 4 * ni};
  const double half = 0.5 * A.dt;
  const int cb = (ni + 127) / 128;
  cudaError_t err = cudaSuccess;
  auto dots = [&](const TV* Vb, int mm, const TV* w, int ww, int region, const int* mask) {
    multidot_b_kernel<TV><<<C.nchunks, KRY_THREADS, 0, s>>>(Vb, N, mm, w, ww, C, mask, partial);
    reduce_b_kernel<<<ni, 32 * (mm + ww), 0, s>>>(partial, C, mask, mm + ww, dsc + region * KRY_MAXV, SS);
    g_launches += 2;
  };
  auto dots64 = [&](const double* w, const int* mask) {
    multidot_b_kernel<double><<<C.nchunks, KRY_THREADS, 0, s>>>(nullptr, N, 0, w, 1, C, mask, partial);
    reduce_b_kernel<<<ni, 32, 0, s>>>(partial, C, mask, 1, dsc + KRY_MAXV, SS);
    g_launches += 2;
  };
  auto update = [&](int mm, int hregion, TV* w, const int* mask) {
    update_b_kernel<TV><<<C.nchunks, KRY_THREADS, 0, s>>>(A.V, N, mm, dsc + hregion * KRY_MAXV, SS, w, C, mask, partial);
    reduce_b_kernel<<<ni, 32, 0, s>>>(partial, C, mask, 1, dsc + KRY_MAXV, SS);
    g_launches += 2;
  };
  auto residual = [&]() -> cudaError_t {
    // r = b - A zeta in FP64 and the inner right side V_0 = P^-1 r
    Epi<double> e{};
    e.out = A.r; e.bvec = A.b; e.wb = 1.0; e.ax = -1.0; e.bl = -half; e.cj = half;
    if (sizeof(TV) == 4) e.out32 = reinterpret_cast<float*>(A.V);
    else e.outj = reinterpret_cast<double*>(A.V);
    cudaError_t e1 = launch_apply_batched<double>(c->b64, M.act, A.state, e, s);
    if (e1 != cudaSuccess) return e1;
    dots64(A.r, M.act);
    bctl_residual<<<cb, 128, 0, s>>>(ctl, M, dsc, SS, ni, A.tol, A.maxit);
    ++g_launches;
    return cudaGetLastError();
  };
  if (what == 0) {  // start of a step; initial guess zeta^(n-1)
    (void)extrap;
    bctl_init<<<cb, 128, 0, s>>>(ctl, M, ni);
    ++g_launches;
    // one FP64 apply gives the right side b = zeta - dt/2 L zeta + dt s and the first residual
    // r = b - A zeta = dt (s - L zeta), with its Jacobi-scaled copy as the inner right side V_0
    Epi<double> e{};
    e.out = A.b; e.ax = 1.0; e.bl = -half; e.gs = A.dt;
    e.out2 = A.r; e.ax2 = 0.0; e.bl2 = -A.dt; e.gs2 = A.dt; e.cj = half;
    if (sizeof(TV) == 4) e.out32 = reinterpret_cast<float*>(A.V);
    else e.outj = reinterpret_cast<double*>(A.V);
    if ((err = launch_apply_batched<double>(c->b64, M.act, A.state, e, s)) != cudaSuccess) return err;
    dots64(A.b, M.act);
    bctl_bnorm<<<cb, 128, 0, s>>>(ctl, M, dsc, SS, ni);
    // instances with b = 0 take zeta = 0, so their residual is 0
    zero_b_kernel<double><<<C.nchunks, KRY_THREADS, 0, s>>>(A.state, C, M.zero);
    zero_b_kernel<double><<<C.nchunks, KRY_THREADS, 0, s>>>(A.r, C, M.zero);
    zero_b_kernel<TV><<<C.nchunks, KRY_THREADS, 0, s>>>(A.V, C, M.zero);
    g_launches += 4;
    dots64(A.r, M.act);
    bctl_residual<<<cb, 128, 0, s>>>(ctl, M, dsc, SS, ni, A.tol, A.maxit);
    ++g_launches;
    return cudaGetLastError();
  }
  // one refinement cycle
  dots(nullptr, 0, A.V, 1, 1, M.act);
  bctl_beta<<<cb, 128, 0, s>>>(ctl, M, dsc, SS, ni, A.tol, sizeof(TV) == 8 ? 0.0 : 1e-6);
  scale_b_kernel<TV><<<C.nchunks, KRY_THREADS, 0, s>>>(A.V, A.V, dsc + KRY_MAXV, SS, C, M.inner);
  g_launches += 2;
  for (int j = 0; j < A.m; ++j) {
    TV* w = A.V + (size_t)(j + 1) * N;
    Epi<TV> e{};
    e.out = w; e.ax = TV(1); e.bl = TV(half); e.jacobi = 1; e.cj = TV(half);
    if constexpr (sizeof(TV) == 8) err = launch_apply_batched<double>(c->b64, M.inner, A.V + (size_t)j * N, e, s);
    else err = launch_apply_batched<float>(c->b32, M.inner, A.V + (size_t)j * N, e, s);
    if (err != cudaSuccess) return err;
    dots(A.V, j + 1, w, 1, 0, M.inner);
    update(j + 1, 0, w, M.inner);
    bctl_reo<<<cb, 128, 0, s>>>(ctl, M, dsc, SS, ni, j);
    ++g_launches;
    dots(A.V, j + 1, w, 0, 2, M.reo);
    update(j + 1, 2, w, M.reo);
    bctl_addh2<<<cb, 128, 0, s>>>(ctl, M, dsc, SS, ni, j);
    scale_b_kernel<TV><<<C.nchunks, KRY_THREADS, 0, s>>>(w, w, dsc + KRY_MAXV, SS, C, M.inner);
    bctl_finalize<<<cb, 128, 0, s>>>(ctl, M, dsc, SS, ni, j, A.maxit);
    g_launches += 3;
  }
  bctl_solve<<<cb, 128, 0, s>>>(ctl, M, dsc, SS, ni);
  combine_b_kernel<TV><<<C.nchunks, KRY_THREADS, 0, s>>>(A.V, N, M.mi, dsc + 3 * KRY_MAXV, SS, A.state, C);
  g_launches += 2;
  return residual();
}

// refinement cycles in the graph that starts a step (two cover the FP32 form at 1e-10: each cycle
// asks the FP32 solve for at most a 1e-6 reduction)
constexpr int kBatchStartCycles = 2;

template <typename TV>
static sap_status batch_cn_graph(sap_ctx* c, double* state, double dt, int nsteps, double tol, int m, int maxit,
                                 sap_solver_stats* st, cudaStream_t s) {
  // kernel attributes (dynamic shared-memory limits) are set before any capture
  if (cudaError_t e0 = prepare_batched<double>(c->b64); e0 != cudaSuccess) {
    c->err = std::string("batch cn: ") + cudaGetErrorString(e0);
    return SAP_ECUDA;
  }
  if (cudaError_t e0 = prepare_batched<TV>(*reinterpret_cast<const std::vector<BatchDev<TV>>*>(
          sizeof(TV) == 8 ? (const void*)&c->b64 : (const void*)&c->b32));
      e0 != cudaSuccess) {
    c->err = std::string("batch cn: ") + cudaGetErrorString(e0);
    return SAP_ECUDA;
  }
  const int64_t N = c->N;
  const int ni = (int)c->sub.size();
  BatchGraphArgs<TV> A{};
  A.state = state;
  A.b = c->ws64;
  A.r = c->ws64 + N;
  A.V = (sizeof(TV) == 8) ? reinterpret_cast<TV*>(c->ws64 + 2 * N) : reinterpret_cast<TV*>(c->ws32);
  A.prev = (sizeof(TV) == 8) ? c->ws64 + (size_t)(m + 3) * N : c->ws64 + 2 * N;
  A.dt = dt;
  A.tol = tol;
  A.m = m;
  A.maxit = maxit;
  cudaError_t err = cudaSuccess;
  if (!c->bctl) {
    if (cudaMalloc(&c->bctl, sizeof(BCtl) * ni) != cudaSuccess ||
        cudaMalloc(&c->bmask, sizeof(int) * 5 * ni) != cudaSuccess ||
        cudaMalloc(&c->bstat, sizeof(BStat) * ni) != cudaSuccess ||
        cudaMallocHost(&c->bstat_host, sizeof(BStat) * ni) != cudaSuccess) {
      c->err = "batch cn: allocation of the control blocks failed";
      return SAP_ENOMEM;
    }
  }
  BStat* hst = reinterpret_cast<BStat*>(c->bstat_host);
  // graphs are kept per (kind, extrapolation) for the current state buffer, dt, tolerances, fields and
  // workspace
  const void* ws = static_cast<const void*>(A.V);
  auto key_ok = [&](const sap_ctx::BGraph& g) {
    return g.state == state && g.dt == dt && g.tol == tol && g.m == m && g.maxit == maxit && g.ws == ws &&
           g.version == c->batch_built_version;
  };
  if (!c->bgraphs.empty() && !key_ok(c->bgraphs.front())) {
    for (auto& g : c->bgraphs)
      if (g.exec) cudaGraphExecDestroy(g.exec);
    c->bgraphs.clear();
  }
  auto get_graph = [&](int kind, int extrap, int64_t* nl) -> cudaGraphExec_t {
    for (const auto& g : c->bgraphs)
      if (g.kind == kind && g.extrap == extrap) {
        *nl = g.launches;
        return g.exec;
      }
    if (!c->cap_stream && cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
      c->cap_stream = nullptr;
      cudaGetLastError();
      return nullptr;
    }
    const int64_t l0 = g_launches;
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    cudaError_t e1 = cudaSuccess;
    if (kind == 0) {
      e1 = batch_enqueue<TV>(c, A, 0, extrap, c->cap_stream);
      for (int k = 0; k < kBatchStartCycles && e1 == cudaSuccess; ++k) e1 = batch_enqueue<TV>(c, A, 1, 0, c->cap_stream);
    } else {
      e1 = batch_enqueue<TV>(c, A, 1, 0, c->cap_stream);
    }
    if (e1 == cudaSuccess) {
      bctl_status<<<(ni + 127) / 128, 128, 0, c->cap_stream>>>(reinterpret_cast<BCtl*>(c->bctl),
                                                               reinterpret_cast<BStat*>(c->bstat), ni);
      ++g_launches;
      e1 = cudaMemcpyAsync(c->bstat_host, c->bstat, sizeof(BStat) * ni, cudaMemcpyDeviceToHost, c->cap_stream);
    }
    const cudaError_t e2 = cudaStreamEndCapture(c->cap_stream, &graph);
    const int64_t launched = g_launches - l0;
    g_launches = l0;
    cudaGraphExec_t ex = nullptr;
    if (e1 != cudaSuccess || e2 != cudaSuccess || !graph || cudaGraphInstantiate(&ex, graph, 0) != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      return nullptr;
    }
    cudaGraphDestroy(graph);
    sap_ctx::BGraph g;
    g.exec = ex; g.kind = kind; g.extrap = extrap; g.state = state; g.dt = dt; g.tol = tol; g.m = m;
    g.maxit = maxit; g.ws = ws; g.version = c->batch_built_version; g.launches = launched;
    c->bgraphs.push_back(g);
    *nl = launched;
    return ex;
  };
  int64_t total_its = 0;
  int max_its = 0;
  double worst_rel = 0.0;
  const int64_t launches0 = g_launches;
  for (int step = 0; step < nsteps; ++step) {
    // the batched precision form starts from zeta^(n-1): an extrapolated guess did not lower the
    // iteration counts (the first refinement cycle stops at a 1e-6 reduction anyway), and without it
    // one FP64 apply yields both the right side and the first residual
    const int extrap = 0;
    int64_t nl = 0;
    cudaGraphExec_t ex = get_graph(0, extrap, &nl);
    if (!ex) {
      c->err = "batch cn: CUDA graph capture of the step failed";
      return SAP_ECUDA;
    }
    if ((err = cudaGraphLaunch(ex, s)) != cudaSuccess) goto cuda_fail;
    g_launches += nl;
    c->cn_prev_valid = true;
    c->cn_prev_ptr = state;
    c->cn_prev_dt = dt;
    c->cn_prev_theta = 0.5;
    if ((err = cudaStreamSynchronize(s)) != cudaSuccess) goto cuda_fail;
    for (;;) {  // continuation cycles for instances still solving under maxit
      bool more = false;
      for (int i = 0; i < ni; ++i) more = more || hst[i].status == BS_SOLVING;
      if (!more) break;
      cudaGraphExec_t exc = get_graph(1, 0, &nl);
      if (!exc) {
        c->err = "batch cn: CUDA graph capture of a refinement cycle failed";
        return SAP_ECUDA;
      }
      if ((err = cudaGraphLaunch(exc, s)) != cudaSuccess) goto cuda_fail;
      g_launches += nl;
      if ((err = cudaStreamSynchronize(s)) != cudaSuccess) goto cuda_fail;
    }
    for (int i = 0; i < ni; ++i) {
      total_its += hst[i].its;
      max_its = std::max(max_its, hst[i].its);
      if (hst[i].status != BS_ZERO) worst_rel = std::max(worst_rel, hst[i].rel);
    }
    for (int i = 0; i < ni; ++i) {
      if (hst[i].status == BS_STOPPED) {
        c->err = "batch cn: GMRES did not reach the tolerance within maxit on instance " + std::to_string(i);
        if (st) {
          st->steps = step + 1; st->iterations = total_its; st->max_iterations = max_its;
          st->last_rel_residual = worst_rel; st->kernel_launches = g_launches - launches0;
        }
        c->cn_prev_valid = false;
        return SAP_ENOCONV;
      }
    }
  }
  if (st) {
    st->steps = nsteps; st->iterations = total_its; st->max_iterations = max_its;
    st->last_rel_residual = worst_rel; st->kernel_launches = g_launches - launches0;
  }
  return SAP_OK;
cuda_fail:
  c->err = std::string("batch cn: ") + cudaGetErrorString(err);
  return SAP_ECUDA;
}

sap_status batch_cn(sap_ctx* c, double* state, double dt, int nsteps, double tol, int restart, int maxit,
                    sap_solver_stats* st, cudaStream_t s) {
  sap_status ps = batch_prepare(c, s);
  if (ps != SAP_OK) return ps;
  return c->prec == SAP_PREC_FP64 ? batch_cn_graph<double>(c, state, dt, nsteps, tol, restart, maxit, st, s)
                                  : batch_cn_graph<float>(c, state, dt, nsteps, tol, restart, maxit, st, s);
}


// ================================================================================================
// Discrete adjoint of the Crank--Nicolson step
// ================================================================================================
// l(l+1)/2 of expansion coefficient r (l = floor(sqrt(r))): the collision rate per unit nu
__device__ __forceinline__ double coll_rate(int r) {
  int l = (int)sqrt((double)r);
  while ((l + 1) * (l + 1) <= r) ++l;
  while (l * l > r) --l;
  return 0.5 * l * (l + 1);
}

// grad[node] += coef * sum_r mu[r,node] * l_r(l_r+1)/2 * (zp + zn)[r,node]
__global__ void grad_nu_kernel(const double* __restrict__ mu, const double* __restrict__ zp,
                               const double* __restrict__ zn, int n, int nloc, int64_t npv, double coef,
                               double* __restrict__ grad) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < npv; p += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cell = p / nloc;
    const int i = (int)(p - cell * nloc);
    double acc = 0.0;
    for (int r = 1; r < n; ++r) {
      const size_t k = ((size_t)cell * n + r) * nloc + i;
      acc += coll_rate(r) * mu[k] * (zp[k] + zn[k]);
    }
    grad[p] += coef * acc;
  }
}

// One reverse step: A^T mu = lambda (A = 1 + dt/2 L) by the device-controlled GMRES on P^-1 A^T from
// the initial guess lambda, the same iteration groups (graph-replayed) as the forward solve; then
// lambda <- B^T mu (B = 1 - dt/2 L) and the nu gradient of the collision term.
sap_status adjoint_cn_step(sap_ctx* c, const double* zp, const double* zn, double* lambda, double dt, double tol,
                           int m, int maxit, double* mu_out, double* grad_nu, sap_solver_stats* st, cudaStream_t s) {
  const int64_t N = c->N;
  double* V = c->ws64;                       // (m+1) vectors
  double* b = V + (size_t)(m + 1) * N;       // right side (copy of lambda)
  double* tmp = b + N;
  double* mu = tmp + N;                      // solution
  GmresDev* Gh = reinterpret_cast<GmresDev*>(c->gdev_host);
  const OpParams<double>& P = c->p64;
  const double half = 0.5 * dt;
  const int64_t launches0 = g_launches;
  int its = 0;
  double rel = 0.0;
  cudaError_t err = cudaSuccess;
#define CK(x)                               \
  do {                                      \
    err = (x);                              \
    if (err != cudaSuccess) goto cuda_fail; \
  } while (0)
  CK(cudaMemcpyAsync(b, lambda, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(mu, lambda, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));  // initial guess
  norm2_dev<double>(c, b, 0, s);
  CK(fetch_misc(c, s));
  {
    const double bnorm = std::sqrt(Gh->misc[0]);
    if (bnorm == 0.0) {
      CK(cudaMemsetAsync(mu, 0, sizeof(double) * N, s));
    } else {
      for (int cyc = 0;; ++cyc) {
        {  // r = b - A^T mu and its Jacobi-scaled copy in V_0
          Epi<double> e{};
          e.out = tmp; e.bvec = b; e.wb = 1.0; e.ax = -1.0; e.bl = -half; e.outj = V; e.cj = half;
          CK(launch_applyT<double>(P, mu, e, s));
        }
        norm2_dev<double>(c, tmp, 1, s);
        norm2_dev<double>(c, V, 2, s);
        CK(fetch_misc(c, s));
        rel = std::sqrt(Gh->misc[1]) / bnorm;
        const double beta = std::sqrt(Gh->misc[2]);
        if (rel <= tol || its >= maxit || !std::isfinite(rel)) break;
        int jd = 0;
        CK((gmres_cycle<double, true>(c, P, V, half, beta, 0.5 * beta * (tol / rel), std::min(m, maxit - its), mu, s,
                                      &jd, cyc)));
        its += jd;
        if (jd == 0) break;
      }
    }
  }
  if (!(rel <= tol)) {  // also catches a NaN residual
    c->err = "adjoint cn: GMRES did not reach the tolerance within maxit";
    if (st) {
      st->steps = 1; st->iterations = its; st->max_iterations = its; st->last_rel_residual = rel;
      st->kernel_launches = g_launches - launches0;
    }
    return SAP_ENOCONV;
  }
  {  // lambda <- B^T mu = mu - dt/2 L^T mu
    Epi<double> e{};
    e.out = lambda; e.ax = 1.0; e.bl = -half;
    CK(launch_applyT<double>(P, mu, e, s));
  }
  if (grad_nu && (c->desc.terms & SAP_TERM_COLL)) {
    grad_nu_kernel<<<1024, 256, 0, s>>>(mu, zp, zn, c->n, c->nloc, (int64_t)c->npv, -half, grad_nu);
    ++g_launches;
  }
  if (mu_out) CK(cudaMemcpyAsync(mu_out, mu, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
  CK(cudaStreamSynchronize(s));
  if (st) {
    st->steps = 1; st->iterations = its; st->max_iterations = its; st->last_rel_residual = rel;
    st->kernel_launches = g_launches - launches0;
  }
  return SAP_OK;
cuda_fail:
  c->err = std::string("adjoint cn: ") + cudaGetErrorString(err);
  return SAP_ECUDA;
#undef CK
}


// ================================================================================================
// Discrete adjoint of the RK4 step
// ================================================================================================
// grad[node] += coef * sum_r l_r(l_r+1)/2 * sum_i kb_i[r,node] Y_i[r,node] over the four stages
__global__ void grad_nu_erk_kernel(const double* __restrict__ y, const double* __restrict__ S, int64_t N, int n,
                                   int nloc, int64_t npv, double coef, double* __restrict__ grad) {
  const double* Y2 = S;
  const double* Y3 = S + N;
  const double* Y4 = S + 2 * N;
  const double* kb1 = S + 3 * N;
  const double* kb2 = S + 4 * N;
  const double* kb3 = S + 5 * N;
  const double* kb4 = S + 6 * N;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < npv; p += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cell = p / nloc;
    const int i = (int)(p - cell * nloc);
    double acc = 0.0;
    for (int r = 1; r < n; ++r) {
      const size_t k = ((size_t)cell * n + r) * nloc + i;
      acc += coll_rate(r) * (kb1[k] * y[k] + kb2[k] * Y2[k] + kb3[k] * Y3[k] + kb4[k] * Y4[k]);
    }
    grad[p] += coef * acc;
  }
}

// kb4 = c4 lam, ksum = kb1 + kb2 + kb3 + kb4
__global__ void erk_adj_sum_kernel(const double* __restrict__ kb1, const double* __restrict__ kb2,
                                   const double* __restrict__ kb3, const double* __restrict__ lam, double c4,
                                   double* __restrict__ kb4, double* __restrict__ ksum, int64_t N) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x) {
    const double k4 = c4 * lam[k];
    kb4[k] = k4;
    ksum[k] = (kb1[k] + kb2[k]) + (kb3[k] + k4);
  }
}

// One reverse step of classical RK4 on zeta' = s - L zeta (L = M^-1 D).  The stage inputs
// Y_1 = y, Y_2 = y + dt/2 k_1, Y_3 = y + dt/2 k_2, Y_4 = y + dt k_3 (k_i = s - L Y_i) are recomputed
// from y; the stage adjoints, in reverse order, are
//   kb4 = dt/6 lam,  kb3 = dt/3 lam - dt L^T kb4,  kb2 = dt/3 lam - dt/2 L^T kb3,
//   kb1 = dt/6 lam - dt/2 L^T kb2,
// and lam <- lam - L^T (kb1 + kb2 + kb3 + kb4).  A parameter theta adds sum_i kb_i . dF/dtheta(Y_i);
// for nu that is -sum_i kb_i . (dL/dnu) Y_i, pointwise in the nodal basis.
// S (7 N): Y2, Y3, Y4, kb1, kb2, kb3, kb4 (the caller's buffer or the workspace).
sap_status adjoint_erk_step(sap_ctx* c, const double* y, double* lambda, double dt, double* grad_nu, double* stages,
                            sap_solver_stats* st, cudaStream_t s) {
  const int64_t N = c->N;
  double* S = stages ? stages : c->ws64;
  double* Y2 = S;
  double* Y3 = S + N;
  double* Y4 = S + 2 * N;
  double* kb1 = S + 3 * N;
  double* kb2 = S + 4 * N;
  double* kb3 = S + 5 * N;
  double* kb4 = S + 6 * N;
  double* ksum = c->ws64 + 7 * N;
  const OpParams<double>& P = c->p64;
  const int64_t launches0 = g_launches;
  cudaError_t err = cudaSuccess;
#define CK(x)                               \
  do {                                      \
    err = (x);                              \
    if (err != cudaSuccess) goto cuda_fail; \
  } while (0)
  {  // stage inputs of the forward step
    Epi<double> e2{};
    e2.out = Y2; e2.ax = 1.0; e2.bl = -0.5 * dt; e2.gs = 0.5 * dt;
    CK(launch_apply<double>(P, y, e2, s));
    Epi<double> e3{};
    e3.out = Y3; e3.bvec = y; e3.wb = 1.0; e3.bl = -0.5 * dt; e3.gs = 0.5 * dt;
    CK(launch_apply<double>(P, Y2, e3, s));
    Epi<double> e4{};
    e4.out = Y4; e4.bvec = y; e4.wb = 1.0; e4.bl = -dt; e4.gs = dt;
    CK(launch_apply<double>(P, Y3, e4, s));
  }
  {  // stage adjoints (kb4 = dt/6 lam enters kb3 directly)
    Epi<double> a3{};
    a3.out = kb3; a3.ax = dt / 3.0; a3.bl = -dt * dt / 6.0;
    CK(launch_applyT<double>(P, lambda, a3, s));
    Epi<double> a2{};
    a2.out = kb2; a2.bvec = lambda; a2.wb = dt / 3.0; a2.bl = -0.5 * dt;
    CK(launch_applyT<double>(P, kb3, a2, s));
    Epi<double> a1{};
    a1.out = kb1; a1.bvec = lambda; a1.wb = dt / 6.0; a1.bl = -0.5 * dt;
    CK(launch_applyT<double>(P, kb2, a1, s));
  }
  erk_adj_sum_kernel<<<1024, 256, 0, s>>>(kb1, kb2, kb3, lambda, dt / 6.0, kb4, ksum, N);
  ++g_launches;
  if (grad_nu && (c->desc.terms & SAP_TERM_COLL)) {
    grad_nu_erk_kernel<<<1024, 256, 0, s>>>(y, S, N, c->n, c->nloc, (int64_t)c->npv, -1.0, grad_nu);
    ++g_launches;
  }
  {  // lam <- lam - L^T (kb1 + kb2 + kb3 + kb4); each entry of lam is read, then written, by one thread
    Epi<double> e{};
    e.out = lambda; e.bvec = lambda; e.wb = 1.0; e.bl = -1.0;
    CK(launch_applyT<double>(P, ksum, e, s));
  }
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  if (st) {
    st->steps = 1; st->iterations = 0; st->max_iterations = 0; st->last_rel_residual = 0.0;
    st->kernel_launches = g_launches - launches0;
  }
  return SAP_OK;
cuda_fail:
  c->err = std::string("adjoint erk: ") + cudaGetErrorString(err);
  return SAP_ECUDA;
#undef CK
}

// ================================================================================================
// Adjoint step with field gradients (sap_adjoint_step)
// ================================================================================================
// CN: the adjoint solve of adjoint_cn_step leaves mu in the workspace; the fields enter through
// -dt/2 mu^T L' (zeta_prev + zeta_next) + dt mu^T s'.  RK4: adjoint_erk_step leaves the stage inputs
// and stage adjoints in the workspace; the fields enter through sum_i kb_i^T (s' - L' Y_i).
sap_status adjoint_fields_step(sap_ctx* c, int scheme, const double* zp, const double* zn, double* lambda, double dt,
                               double tol, int m, int maxit, const sap_field_grads& g, sap_solver_stats* st,
                               cudaStream_t s) {
  const int64_t N = c->N;
  const bool spatial = g.U || g.gradU || g.DUDt || g.Bw || g.Uface[0] || g.Uface[1] || g.Uface[2];
  const int64_t launches0 = g_launches;
  sap_status rs;
  cudaError_t err = cudaSuccess;
  if (scheme == SAP_SCHEME_CN) {
    rs = adjoint_cn_step(c, zp, zn, lambda, dt, tol, m, maxit, nullptr, g.nu, st, s);
    if (rs != SAP_OK) return rs;
    const double* mu = c->ws64 + (size_t)(m + 3) * N;
    double* w = c->ws64 + (size_t)(m + 2) * N;
    if (spatial) {
      if ((err = launch_add2(zp, zn, w, N, s)) != cudaSuccess) goto fail;
      if ((err = cudaMemsetAsync(c->gpart, 0, sizeof(double) * (size_t)c->ncell * c->gt.ps, s)) != cudaSuccess)
        goto fail;
      if ((err = launch_coef_adjoint(c->p64, c->gt, mu, w, c->gpart, s)) != cudaSuccess) goto fail;
      if ((err = launch_grad_reduce(c->p64, c->gt, c->gpart, c->nscell, c->npc, -0.5 * dt, g, s)) != cudaSuccess)
        goto fail;
    }
    if (g.s000 && (c->desc.terms & SAP_TERM_SRC))
      if ((err = launch_grad_src(mu, N, 1, c->n, c->nloc, c->npv, dt, g.s000, s)) != cudaSuccess) goto fail;
  } else {
    rs = adjoint_erk_step(c, zp, lambda, dt, g.nu, nullptr, st, s);
    if (rs != SAP_OK) return rs;
    const double* S = c->ws64;  // Y2, Y3, Y4, kb1, kb2, kb3, kb4
    if (spatial) {
      if ((err = cudaMemsetAsync(c->gpart, 0, sizeof(double) * (size_t)c->ncell * c->gt.ps, s)) != cudaSuccess)
        goto fail;
      const double* Y[4] = {zp, S, S + N, S + 2 * N};
      for (int i = 0; i < 4; ++i)
        if ((err = launch_coef_adjoint(c->p64, c->gt, S + (size_t)(3 + i) * N, Y[i], c->gpart, s)) != cudaSuccess)
          goto fail;
      if ((err = launch_grad_reduce(c->p64, c->gt, c->gpart, c->nscell, c->npc, -1.0, g, s)) != cudaSuccess) goto fail;
    }
    if (g.s000 && (c->desc.terms & SAP_TERM_SRC))
      if ((err = launch_grad_src(S + 3 * N, N, 4, c->n, c->nloc, c->npv, 1.0, g.s000, s)) != cudaSuccess) goto fail;
  }
  if ((err = cudaStreamSynchronize(s)) != cudaSuccess) goto fail;
  if (st) st->kernel_launches = g_launches - launches0;
  return SAP_OK;
fail:
  c->err = std::string("adjoint fields: ") + cudaGetErrorString(err);
  return SAP_ECUDA;
}

}  // namespace sap
