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
#include <mutex>
#include <string>
#include <vector>

#include "sap_internal.h"

namespace sap {

// kernels launched by this host thread (for the launch counts reported in sap_solver_stats)
static thread_local int64_t g_launches = 0;
int64_t launch_count() { return g_launches; }

// ------------------------------------------------------------------------------------------------
// epilogue: out = d .* (wb*b + ax*x + bl*(Lx) + gs*s), and/or ERK bookkeeping
// ------------------------------------------------------------------------------------------------
template <typename T>
struct Epi {
  T* out;               // may be null
  const T* bvec;        // optional
  T wb, ax, bl, gs;
  int jacobi;           // multiply out by 1 / (1 + cj * diag(R - div beta))
  T cj;
  // ERK stage (k = s - Lx):  acc += bdt k ; ynext = y0 + adt k ; final: state = acc + bdt k
  double* acc;
  const double* y0;
  T* ynext;
  double adt, bdt;
  int erk;              // 0 none, 1 first stage (acc = y0 + bdt k), 2 middle, 3 last (y0 <- acc + bdt k)
  double* state;        // for erk == 3
};

template <typename T>
__device__ __forceinline__ T csr_row(const Bank<T>& B, int mat, int r, const T* x, int stride) {
  if (mat == MAT_I) return x[r * stride];
  const int* rp = B.rp + B.rp_off[mat];
  T acc = T(0);
  const int e = __ldg(rp + r + 1);
  for (int k = __ldg(rp + r); k < e; ++k) acc += __ldg(B.val + k) * x[__ldg(B.col + k) * stride];
  return acc;
}

template <typename T>
__device__ __forceinline__ T csr_diag(const Bank<T>& B, int mat, int r) {
  if (mat == MAT_I) return T(1);
  const int* rp = B.rp + B.rp_off[mat];
  for (int k = __ldg(rp + r); k < __ldg(rp + r + 1); ++k)
    if (__ldg(B.col + k) == r) return __ldg(B.val + k);
  return T(0);
}

// momentum factors (p, gamma m, V, 1/V, ...) are tabulated on the host per momentum node and face
template <typename T>
__device__ __forceinline__ T mom_node(const OpParams<T>& P, int mf, int pn) {
  return mf == MF_ONE ? T(1) : __ldg(P.mfn + (size_t)mf * P.npn + pn);
}
template <typename T>
__device__ __forceinline__ T mom_face(const OpParams<T>& P, int mf, int pf) {
  return mf == MF_ONE ? T(1) : __ldg(P.mff + (size_t)mf * P.npface + pf);
}

template <typename T>
__device__ __forceinline__ T spatial_factor(const OpParams<T>& P, int sf, int sp) {
  if (sf == SF_ONE) return T(1);
  if (P.sf_is_uni[sf]) return P.sf_uni[sf];
  return __ldg(P.sfield + (size_t)sf * P.nsv + sp);
}

// node index from a face point (axis a removed) and the position j along a
__device__ __forceinline__ int face_node(int fp, int j, int a, const int* qpow) {
  const int lo = fp % qpow[a];
  const int hi = fp / qpow[a];
  return lo + j * qpow[a] + hi * qpow[a + 1];
}

template <typename T>
__global__ void __launch_bounds__(1024) apply_kernel(const OpParams<T> P, const T* __restrict__ x, const Epi<T> E,
                                                     int cpb, int cell_stride) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int n = P.n, nloc = P.nloc, nfp = P.nfp, D = P.D, q = P.q;
  const int per_cell = n * nloc;
  const int nf = 2 * D;
  const int lc = threadIdx.x / per_cell;
  const int t = threadIdx.x - lc * per_cell;
  const int r = t / nloc, i = t - r * nloc;
  const int cell = blockIdx.x * cpb + lc;
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
  T* G = Tr;  // aliases Tr/Tn/W1 once the face fluxes are done
  const int region = (3 * szT > D * per_cell) ? 3 * szT : D * per_cell;
  T* CV = Tr + region;
  T* CF = CV + nvt * nloc;

  const int scell = valid ? P.cell_scell[cell] : 0;
  const int pcell = valid ? P.cell_pcell[cell] : 0;

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
      const int sp = scell * P.qdx + ii % P.qdx;
      T c = T(tm->scale) * spatial_factor(P, tm->sf, sp) * mom_node(P, tm->mf, pcell * q + ii / P.qdx);
      if (tm->nu) c *= P.nu ? __ldg(P.nu + (size_t)cell * nloc + ii) : P.nu_uni;
      CV[w] = c;
    }
    // face coefficients of the advection terms at every face point
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
        // spatial face: U_a at the spatial face point, momentum factor at the node's p
        const int qsp = P.qdx / q;  // spatial face points per spatial face
        const int fsp = fp % qsp;
        if (tm.sf == SF_U + a) {
          const int base = P.scell_face[scell * 2 * P.dx + 2 * a + side];
          c *= P.uface_is_uni[a] ? P.uface_uni[a] : __ldg(P.uface[a] + base + fsp);
        } else {
          c *= spatial_factor(P, tm.sf, scell * P.qdx);  // only SF_ONE occurs here
        }
        c *= mom_node(P, tm.mf, pcell * q + fp / qsp);
      } else {
        // momentum face: spatial factor at the spatial node (fp), momentum at the face
        c *= spatial_factor(P, tm.sf, scell * P.qdx + fp);
        c *= mom_face(P, tm.mf, pcell + side);
      }
      CF[w] = c;
    }
    // neighbour traces
    for (int w = t; w < szT; w += per_cell) {
      const int f = w / (n * nfp);
      const int rr = (w / nfp) % n;
      const int fp = w % nfp;
      const int a = f >> 1, side = f & 1;
      const int nb = P.cell_nb[cell * nf + f];
      T v = T(0);
      if (nb >= 0 && P.ax[a].active) {
        const T* xn = x + ((size_t)nb * n + rr) * nloc;
        for (int j = 0; j < q; ++j) v += (side == 0 ? P.B1[j] : P.B0[j]) * __ldg(xn + face_node(fp, j, a, qpow));
      }
      Tn[w] = v;
    }
  }
  __syncthreads();
  // ---- phase 2: own traces ------------------------------------------------------------------------
  if (valid) {
    for (int w = t; w < szT; w += per_cell) {
      const int f = w / (n * nfp);
      const int rr = (w / nfp) % n;
      const int fp = w % nfp;
      const int a = f >> 1, side = f & 1;
      T v = T(0);
      const T* Fr = F + rr * nloc;
      for (int j = 0; j < q; ++j) v += (side == 0 ? P.B0[j] : P.B1[j]) * Fr[face_node(fp, j, a, qpow)];
      Tr[w] = v;
    }
  }
  __syncthreads();
  // ---- phase 3a: boundary substitution; Tr <- f_lo + f_hi, Tn <- f_lo - f_hi -----------------------
  if (valid) {
    for (int w = t; w < szT; w += per_cell) {
      const int f = w / (n * nfp);
      const int a = f >> 1, side = f & 1;
      if (!P.ax[a].active) continue;
      const int nb = P.cell_nb[cell * nf + f];
      const T own = Tr[w];
      T oth = Tn[w];
      if (nb < 0) {
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
    for (int w = t; w < szT; w += per_cell) {
      const int f = w / (n * nfp);
      const int rr = (w / nfp) % n;
      const int fp = w % nfp;
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
        const int sp = scell * P.qdx + fp;
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
        W1[w] = fabs(c0 + P.lam[rr] * c1) * csr_row(P.bank, A.WTmat, rr, Db, nfp);
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
  // ---- phase 3c: volume advection g^a = beta^a f at the nodes (G aliases the face scratch) -------------
  if (valid) {
    for (int a = 0; a < D; ++a) {
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
    if (E.jacobi) rdiag += c * csr_diag(P.bank, P.react[tt].mat, r);
  }
  for (int a = 0; a < D; ++a) {
    if (!P.ax[a].active) continue;
    const T invh = P.cell_invh[cell * D + a];
    const int ia = (i / qpow[a]) % q;
    const int base = i - ia * qpow[a];
    const T* Ga = G + a * per_cell + r * nloc + base;
    T ds = T(0);
    for (int qq = 0; qq < q; ++qq) ds += P.S[ia][qq] * Ga[qq * qpow[a]];
    const int fp = (i % qpow[a]) + (i / qpow[a + 1]) * qpow[a];
    const T jup = Jf[((2 * a + 1) * n + r) * nfp + fp];
    const T jdn = Jf[((2 * a) * n + r) * nfp + fp];
    acc += invh * (P.L1[ia] * jup - P.L0[ia] * jdn - ds);
  }
  const size_t dof = (size_t)cell * per_cell + t;
  T s = T(0);
  if (r == 0) s = P.s000 ? __ldg(P.s000 + (size_t)cell * nloc + i) : P.s_uni;
  if (E.erk) {
    const double k = double(s) - double(acc);
    if (E.erk == 1) {
      E.acc[dof] = E.y0[dof] + E.bdt * k;
    } else if (E.erk == 2) {
      E.acc[dof] += E.bdt * k;
    } else {
      E.state[dof] = E.acc[dof] + E.bdt * k;
    }
    if (E.ynext) E.ynext[dof] = T(E.y0[dof] + E.adt * k);
    return;
  }
  T o = E.ax * F[t] + E.bl * acc + E.gs * s;
  if (E.bvec) o += E.wb * __ldg(E.bvec + dof);
  if (E.jacobi) o /= (T(1) + E.cj * rdiag);
  E.out[dof] = o;
}

int apply_cells_per_block(int n, int nloc) {
  const int per = n * nloc;
  int cpb = std::max(1, 256 / per);
  while (cpb > 1 && cpb * per > 1024) --cpb;
  return cpb;
}

template <typename T>
static int cell_stride_elems(const OpParams<T>& P) {
  int nvt = P.nreact;
  for (int a = 0; a < P.D; ++a) nvt += P.ax[a].nadv;
  const int per = P.n * P.nloc;
  const int szT = 2 * P.D * P.n * P.nfp;
  int s = per + szT + std::max(3 * szT, P.D * per) + nvt * P.nloc + 2 * P.D * MAXADV * P.nfp;
  return (s + 1) & ~1;  // keep 16-byte alignment of each cell's block for doubles
}

template <typename T>
static cudaError_t launch_apply(const OpParams<T>& P, const T* x, const Epi<T>& e, cudaStream_t s) {
  const int per = P.n * P.nloc;
  if (per > 1024) return cudaErrorInvalidConfiguration;  // n (k+1)^D must fit one thread block
  const int cpb = apply_cells_per_block(P.n, P.nloc);
  const int stride = cell_stride_elems(P);
  const size_t smem = (size_t)cpb * stride * sizeof(T);
  static bool attr_set[2] = {false, false};
  const int idx = sizeof(T) == 8 ? 0 : 1;
  if (!attr_set[idx]) {
    cudaError_t err = cudaFuncSetAttribute(apply_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (err != cudaSuccess) return err;
    attr_set[idx] = true;
  }
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  const int blocks = (P.ncell + cpb - 1) / cpb;
  apply_kernel<T><<<blocks, cpb * per, smem, s>>>(P, x, e, cpb, stride);
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
  return launch_apply<double>(p, x, mode == SAP_APPLY_RHS ? epi_plain<double>(y, 0, -1, 1) : epi_plain<double>(y, 0, 1, 0), s);
}
cudaError_t launch_apply32(const OpParams<float>& p, const float* x, float* y, int mode, cudaStream_t s) {
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
// Krylov kernels (FP64): multi-dot, update, norms
// ------------------------------------------------------------------------------------------------
constexpr int KRY_THREADS = 256;
constexpr int KRY_MAXV = 32;

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Dot products of w with V_0..V_{m-1} (V_i = V + i*ldv) and, if `with_ww`, of w with itself.
// Block b handles the chunk [b*KRY_CHUNK, (b+1)*KRY_CHUNK): it stages w in shared memory once, then
// warp v sums V_i . w for i = v, v+8, ... ; partial[i][b] = the chunk's value (fixed order).
constexpr int KRY_CHUNK = 2048;
__global__ void __launch_bounds__(KRY_THREADS) multidot_kernel(const double* __restrict__ V, int64_t ldv, int m,
                                                               const double* __restrict__ w, int64_t N, int with_ww,
                                                               double* __restrict__ partial, int nchunks) {
  __shared__ double ws[KRY_CHUNK];
  const int64_t k0 = (int64_t)blockIdx.x * KRY_CHUNK;
  const int len = (int)((N - k0) < KRY_CHUNK ? (N - k0) : KRY_CHUNK);
  for (int k = threadIdx.x; k < len; k += KRY_THREADS) ws[k] = w[k0 + k];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int mt = m + (with_ww ? 1 : 0);
  for (int i = warp; i < mt; i += KRY_THREADS / 32) {
    const double* a = (i < m) ? V + i * ldv + k0 : nullptr;
    double acc = 0.0;
    if (a) {
      for (int k = lane; k < len; k += 32) acc += __ldg(a + k) * ws[k];
    } else {
      for (int k = lane; k < len; k += 32) acc += ws[k] * ws[k];
    }
    acc = warp_sum(acc);
    if (lane == 0) partial[(size_t)i * nchunks + blockIdx.x] = acc;
  }
}

// out[i] = sum_c partial[i][c], i < m: warp i strides over the chunks, then a fixed-order shuffle
// reduction (deterministic for a given N).
__global__ void reduce_partials_kernel(const double* __restrict__ partial, int nchunks, int m, double* __restrict__ out) {
  const int lane = threadIdx.x & 31, i = threadIdx.x >> 5;
  if (i >= m) return;
  double v = 0.0;
  for (int c = lane; c < nchunks; c += 32) v += partial[(size_t)i * nchunks + c];
  v = warp_sum(v);
  if (lane == 0) out[i] = v;
}

// w -= sum_i h[i] V_i ; partial[b] = this block's sum of the updated w^2 (block-strided chunks)
__global__ void __launch_bounds__(KRY_THREADS) update_kernel(const double* __restrict__ V, int64_t ldv, int m,
                                                             const double* __restrict__ h, double* __restrict__ w,
                                                             int64_t N, double* __restrict__ partial, int nchunks) {
  __shared__ double hs[KRY_MAXV];
  __shared__ double red[KRY_THREADS / 32];
  if (threadIdx.x < m) hs[threadIdx.x] = h[threadIdx.x];
  __syncthreads();
  const int64_t k0 = (int64_t)blockIdx.x * KRY_CHUNK;
  const int64_t k1 = (k0 + KRY_CHUNK < N) ? k0 + KRY_CHUNK : N;
  double nrm = 0.0;
  for (int64_t k = k0 + threadIdx.x; k < k1; k += KRY_THREADS) {
    double v = w[k];
    for (int i = 0; i < m; ++i) v -= hs[i] * __ldg(V + i * ldv + k);
    w[k] = v;
    nrm += v * v;
  }
  nrm = warp_sum(nrm);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = nrm;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < KRY_THREADS / 32; ++q) t += red[q];
    partial[blockIdx.x] = t;
  }
  (void)nchunks;
}

// y = a*x with a = 1/a_dev[0] (invert = 1), 1/sqrt(a_dev[0]) (invert = 2) or a_dev[0]
__global__ void scale_kernel(const double* __restrict__ x, double* __restrict__ y, const double* __restrict__ a_dev,
                             int invert, int64_t N) {
  const double a = invert == 1 ? 1.0 / a_dev[0] : (invert == 2 ? 1.0 / sqrt(a_dev[0]) : a_dev[0]);
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x) y[k] = a * x[k];
}

// x += sum_i y[i] V_i
__global__ void combine_kernel(const double* __restrict__ V, int64_t ldv, int m, const double* __restrict__ y,
                               double* __restrict__ x, int64_t N) {
  __shared__ double ys[KRY_MAXV];
  if (threadIdx.x < m) ys[threadIdx.x] = y[threadIdx.x];
  __syncthreads();
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x) {
    double v = x[k];
    for (int i = 0; i < m; ++i) v += ys[i] * __ldg(V + i * ldv + k);
    x[k] = v;
  }
}

}  // namespace sap

// ------------------------------------------------------------------------------------------------
// Crank--Nicolson step, restarted GMRES with left point-Jacobi preconditioning (FP64)
// ------------------------------------------------------------------------------------------------
namespace sap {

struct KrylovCtx {
  sap_ctx* c;
  cudaStream_t s;
  int nchunks;
  double* partial;   // [KRY_MAXV + 1][nchunks]
  double* dsc;       // device scalars [8 * KRY_MAXV]
  double* hsc;       // pinned host mirror [8 * KRY_MAXV]
};

// dsc_out[i] = V_i . w for i < m, and dsc_out[m] = w . w if with_ww
static void dots(KrylovCtx& K, const double* V, int m, const double* w, int with_ww, double* dsc_out) {
  const int64_t N = K.c->N;
  multidot_kernel<<<K.nchunks, KRY_THREADS, 0, K.s>>>(V, N, m, w, N, with_ww, K.partial, K.nchunks);
  ++g_launches;
  reduce_partials_kernel<<<1, 32 * (m + with_ww), 0, K.s>>>(K.partial, K.nchunks, m + with_ww, dsc_out);
  ++g_launches;
}

// w -= V h (m vectors), then dsc_out[0] = |w|^2
static void update(KrylovCtx& K, const double* V, int m, const double* h, double* w, double* dsc_out) {
  const int64_t N = K.c->N;
  update_kernel<<<K.nchunks, KRY_THREADS, 0, K.s>>>(V, N, m, h, w, N, K.partial, K.nchunks);
  ++g_launches;
  reduce_partials_kernel<<<1, 32, 0, K.s>>>(K.partial, K.nchunks, 1, dsc_out);
  ++g_launches;
}

static cudaError_t fetch(KrylovCtx& K, int first, int count) {
  cudaMemcpyAsync(K.hsc + first, K.dsc + first, sizeof(double) * count, cudaMemcpyDeviceToHost, K.s);
  return cudaStreamSynchronize(K.s);
}

int64_t krylov_scratch_doubles(int64_t N) {
  const int64_t nchunks = (N + KRY_CHUNK - 1) / KRY_CHUNK;
  return (KRY_MAXV + 1) * nchunks + 8 * KRY_MAXV;
}

sap_status cn_steps(sap_ctx* c, double* state, double dt, int nsteps, double tol, int restart, int maxit,
                    sap_solver_stats* st, cudaStream_t s) {
  const int64_t N = c->N;
  const int m = restart;
  double* V = c->ws64;                       // (m+1) vectors
  double* b = V + (size_t)(m + 1) * N;
  double* tmp = b + N;
  const int nchunks = (int)((N + KRY_CHUNK - 1) / KRY_CHUNK);
  KrylovCtx K{c, s, nchunks, c->small, c->small + (size_t)(KRY_MAXV + 1) * nchunks, c->small_host};
  double* const d_h1 = K.dsc;                  // [0, 32): first Gram-Schmidt coefficients (+ |w|^2 at j+1)
  double* const d_nrm = K.dsc + KRY_MAXV;      // [32]: |w|^2 after the update
  double* const d_h2 = K.dsc + 2 * KRY_MAXV;   // [64, 96): re-orthogonalisation coefficients
  double* const d_y = K.dsc + 3 * KRY_MAXV;    // [96, 128): least-squares solution
  const OpParams<double>& P = c->p64;
  const double half = 0.5 * dt;
  std::vector<double> H((size_t)(m + 1) * m), g(m + 1), cs(m), sn(m), y(m);
  int64_t total_its = 0;
  const int64_t launches0 = g_launches;
  int max_its = 0;
  double last_rel = 0.0;
  cudaError_t err = cudaSuccess;
#define CK(x)                                           \
  do {                                                  \
    err = (x);                                          \
    if (err != cudaSuccess) goto cuda_fail;             \
  } while (0)
  for (int step = 0; step < nsteps; ++step) {
    // b = zeta - dt/2 M^-1 D zeta + dt M^-1 h   (Eq. system-matrix-rhs, theta = 1/2)
    {
      Epi<double> e{};
      e.out = b; e.ax = 1.0; e.bl = -half; e.gs = dt;
      CK(launch_apply<double>(P, state, e, s));
    }
    dots(K, nullptr, 0, b, 1, d_nrm);
    CK(fetch(K, KRY_MAXV, 1));
    const double bnorm = std::sqrt(K.hsc[KRY_MAXV]);
    int its = 0;
    double rel = 0.0;
    if (bnorm == 0.0) {
      CK(cudaMemsetAsync(state, 0, sizeof(double) * N, s));
      last_rel = 0.0;
      continue;
    }
    for (;;) {
      // true residual r = b - (zeta + dt/2 M^-1 D zeta)
      {
        Epi<double> e{};
        e.out = tmp; e.bvec = b; e.wb = 1.0; e.ax = -1.0; e.bl = -half;
        CK(launch_apply<double>(P, state, e, s));
      }
      dots(K, nullptr, 0, tmp, 1, d_nrm);
      CK(fetch(K, KRY_MAXV, 1));
      rel = std::sqrt(K.hsc[KRY_MAXV]) / bnorm;
      if (rel <= tol || its >= maxit) break;
      // preconditioned residual v0 = P^-1 r, normalised
      {
        Epi<double> e{};
        e.out = V; e.bvec = b; e.wb = 1.0; e.ax = -1.0; e.bl = -half; e.jacobi = 1; e.cj = half;
        CK(launch_apply<double>(P, state, e, s));
      }
      dots(K, nullptr, 0, V, 1, d_nrm);
      scale_kernel<<<1024, KRY_THREADS, 0, s>>>(V, V, d_nrm, 2, N);
      ++g_launches;
      CK(fetch(K, KRY_MAXV, 1));
      const double beta = std::sqrt(K.hsc[KRY_MAXV]);
      std::fill(g.begin(), g.end(), 0.0);
      g[0] = beta;
      // inner target on the preconditioned residual, scaled to the true-residual goal
      const double target = 0.5 * beta * (tol / rel);
      int jdone = 0;
      for (int j = 0; j < m && its < maxit; ++j) {
        double* w = V + (size_t)(j + 1) * N;
        {
          Epi<double> e{};
          e.out = w; e.ax = 1.0; e.bl = half; e.jacobi = 1; e.cj = half;
          CK(launch_apply<double>(P, V + (size_t)j * N, e, s));
        }
        // classical Gram--Schmidt with selective re-orthogonalisation (|w'| < |w|/sqrt(2))
        dots(K, V, j + 1, w, 1, d_h1);
        update(K, V, j + 1, d_h1, w, d_nrm);
        CK(fetch(K, 0, KRY_MAXV + 1));
        for (int i2 = 0; i2 <= j; ++i2) H[(size_t)i2 * m + j] = K.hsc[i2];
        const double wn0 = std::sqrt(K.hsc[j + 1]);
        double wn = std::sqrt(K.hsc[KRY_MAXV]);
        if (wn < 0.7071067811865476 * wn0) {
          dots(K, V, j + 1, w, 0, d_h2);
          update(K, V, j + 1, d_h2, w, d_nrm);
          CK(fetch(K, 2 * KRY_MAXV, j + 1));
          CK(fetch(K, KRY_MAXV, 1));
          for (int i2 = 0; i2 <= j; ++i2) H[(size_t)i2 * m + j] += K.hsc[2 * KRY_MAXV + i2];
          wn = std::sqrt(K.hsc[KRY_MAXV]);
        }
        H[(size_t)(j + 1) * m + j] = wn;
        if (wn > 0.0) {
          scale_kernel<<<1024, KRY_THREADS, 0, s>>>(w, w, d_nrm, 2, N);
          ++g_launches;
        }
        for (int i2 = 0; i2 < j; ++i2) {
          const double a0 = H[(size_t)i2 * m + j], a1 = H[(size_t)(i2 + 1) * m + j];
          H[(size_t)i2 * m + j] = cs[i2] * a0 + sn[i2] * a1;
          H[(size_t)(i2 + 1) * m + j] = -sn[i2] * a0 + cs[i2] * a1;
        }
        const double a0 = H[(size_t)j * m + j], a1 = H[(size_t)(j + 1) * m + j];
        const double den = std::hypot(a0, a1);
        cs[j] = den > 0 ? a0 / den : 1.0;
        sn[j] = den > 0 ? a1 / den : 0.0;
        H[(size_t)j * m + j] = den;
        H[(size_t)(j + 1) * m + j] = 0.0;
        g[j + 1] = -sn[j] * g[j];
        g[j] = cs[j] * g[j];
        ++its;
        jdone = j + 1;
        if (std::fabs(g[j + 1]) <= target || wn == 0.0) break;
      }
      // y = H^-1 g ; zeta += V y
      for (int i2 = jdone - 1; i2 >= 0; --i2) {
        double v = g[i2];
        for (int k2 = i2 + 1; k2 < jdone; ++k2) v -= H[(size_t)i2 * m + k2] * y[k2];
        y[i2] = v / H[(size_t)i2 * m + i2];
      }
      for (int i2 = 0; i2 < jdone; ++i2) K.hsc[3 * KRY_MAXV + i2] = y[i2];
      CK(cudaMemcpyAsync(d_y, K.hsc + 3 * KRY_MAXV, sizeof(double) * jdone, cudaMemcpyHostToDevice, s));
      combine_kernel<<<1024, KRY_THREADS, 0, s>>>(V, N, jdone, d_y, state, N);
      ++g_launches;
      CK(cudaGetLastError());
    }
    total_its += its;
    max_its = std::max(max_its, its);
    last_rel = rel;
    if (rel > tol) {
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

}  // namespace sap
