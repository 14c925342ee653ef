// Field gradients of the discrete adjoint steps: sigma * d/d(field) [ g^T L(fields) w ] at every point
// where a field is sampled (L = M^-1 D of Eq. definition-mass-and-dg-matrix, nodal basis).
//
// In the CN adjoint (Eq. theta-method transposed) a field enters through -dt/2 mu^T L'(zeta_prev +
// zeta_next); in the RK4 adjoint through -sum_i kb_i^T L' Y_i (Sec. 3.4 stages).  Both are of the form
// sigma g^T (dL/dtheta) w.  L is linear in every coefficient of its term tables (Eq.
// definitions-advection-reaction-eq: volume terms, face central terms), except through the upwind
// matrices |beta| of Eq. definition-upwind-flux, whose derivative is taken by the Daleckii--Krein
// formula d|beta|[dB] = W (Gamma o (W^T dB W)) W^T, Gamma_ij = (|l_i| - |l_j|) / (l_i - l_j)
// (sign(l_i) for equal signs; 0 where both eigenvalues vanish: the zero subgradient at the kink).
//
//   coef_adjoint_kernel   one block per cell: the derivative with respect to every term coefficient
//                         at the cell's nodes and face points, chained to the spatial field
//                         components (partials per cell, summed over the cell's momentum nodes)
//   grad_sf_reduce_kernel sums the per-cell partials over the momentum cells of each spatial cell
//                         into dJ/dU, dJ/d gradU, dJ/d DU/Dt, dJ/dB at the spatial points
//   grad_uface_kernel     the same for U_a at the spatial face points (one pass per face side)
//   grad_src_kernel       dJ/ds_000 at the phase-space nodes (row 0 of the source is s_000)
#include <cuda_runtime.h>

#include "kernels_common.cuh"

namespace sap {

void note_launch();

namespace {

__device__ __forceinline__ double sgn(double v) { return v > 0.0 ? 1.0 : (v < 0.0 ? -1.0 : 0.0); }

// (K x)[r] at node i for a bank matrix K (CSR), x = [n][stride] in shared memory
__device__ __forceinline__ double csr_row_apply(const Bank<double>& B, int mat, int r, const double* x, int stride,
                                                int i) {
  if (mat == MAT_I) return x[r * stride + i];
  const int* rp = B.rp + B.rp_off[mat];
  double s = 0.0;
  for (int k = rp[r]; k < rp[r + 1]; ++k) s += B.val[k] * x[B.col[k] * stride + i];
  return s;
}

// node index from a face point (axis a removed) and the position j along a
__device__ __forceinline__ int fnode(int fp, int j, int a, int q) {
  if (a == 0) return j + fp * q;
  if (a == 1) return (fp % q) + j * q + (fp / q) * q * q;
  return (fp % (q * q)) + j * q * q + (fp / (q * q)) * q * q * q;
}

}  // namespace

// Dynamic shared memory of coef_adjoint_kernel (doubles): w, g, ghat, tmp [n nloc]; S, D, ell, u, v
// [n nfp]; node and face-point values [nloc]; the cell's partials [ps].
int coef_adjoint_smem_doubles(const OpParams<double>& P, const GradTables& G) {
  return 4 * P.n * P.nloc + 5 * P.n * P.nfp + P.nloc + G.ps;
}

__global__ void __launch_bounds__(256) coef_adjoint_kernel(const __grid_constant__ OpParams<double> P,
                                                           const __grid_constant__ GradTables G,
                                                           const double* __restrict__ g,
                                                           const double* __restrict__ w,
                                                           double* __restrict__ part) {
  extern __shared__ __align__(16) double sm[];
  const int n = P.n, nloc = P.nloc, nfp = P.nfp, q = P.q, D = P.D;
  const int NL = n * nloc, NF = n * nfp;
  const int cell = blockIdx.x;
  const int tid = threadIdx.x, nt = blockDim.x;
  double* ws = sm;             // [n][nloc] w of the cell
  double* gs = ws + NL;        // [n][nloc] g of the cell
  double* gh = gs + NL;        // [n][nloc] g contracted with the derivative matrix along an axis
  double* tmp = gh + NL;       // [n][nloc] products before the sum over rows
  double* fS = tmp + NL;       // [n][nfp] face: f_lo + f_hi
  double* fD = fS + NF;        // [n][nfp] face: f_lo - f_hi
  double* fl = fD + NF;        // [n][nfp] face: lifted adjoint weight ell
  double* fu = fl + NF;        // [n][nfp] face: W^T ell, later products before the sum over rows
  double* fv = fu + NF;        // [n][nfp] face: W^T (f_lo - f_hi)
  double* nv = fv + NF;        // [nloc] per-node (or per-face-point) values
  double* pc = nv + nloc;      // [ps] partials of this cell
  const size_t base = (size_t)cell * NL;
  for (int e = tid; e < NL; e += nt) {
    ws[e] = w[base + e];
    gs[e] = g[base + e];
  }
  for (int k = tid; k < G.ps; k += nt) pc[k] = 0.0;
  __syncthreads();
  const int has_mom = P.has_mom;
  const int qdx = P.qdx;
  const int scell = P.cell_scell[cell], pcell = P.cell_pcell[cell];
  const int np_per_s = nloc / qdx;  // momentum nodes per spatial node of the cell (1 without momentum)

  // sum the per-node values nv[i] (scaled already) into the partial of component ci at the spatial
  // node of i, in a fixed order (momentum node index ascending)
  auto to_snodes = [&](int ci) {
    __syncthreads();
    for (int sn = tid; sn < qdx; sn += nt) {
      double s = 0.0;
      for (int jp = 0; jp < np_per_s; ++jp) s += nv[sn + qdx * jp];
      pc[ci * qdx + sn] += s;
    }
    __syncthreads();
  };
  auto pnode_of = [&](int i) { return has_mom ? pcell * q + i / qdx : 0; };

  // ---- reaction terms: d/dc_t(i) = sum_r g[r][i] (K_t w)[r][i] ---------------------------------
  for (int t = 0; t < P.nreact; ++t) {
    const Term tm = P.react[t];
    if (tm.sf == SF_ONE) continue;
    const int ci = G.sf_comp[tm.sf];
    if (ci < 0) continue;
    for (int e = tid; e < NL; e += nt) {
      const int r = e / nloc, i = e - r * nloc;
      tmp[e] = gs[e] * csr_row_apply(P.bank, tm.mat, r, ws, nloc, i);
    }
    __syncthreads();
    for (int i = tid; i < nloc; i += nt) {
      double s = 0.0;
      for (int r = 0; r < n; ++r) s += tmp[r * nloc + i];
      double f = tm.scale * mom_node(P, tm.mf, pnode_of(i));
      if (tm.nu) f *= P.nu ? P.nu[(size_t)cell * nloc + i] : P.nu_uni;
      nv[i] = f * s;
    }
    to_snodes(ci);
  }

  // ---- volume advection along each axis: acc[i] -= invh sum_j S_a[i_a][j_a] (beta^a w)[j] ------------
  for (int a = 0; a < D; ++a) {
    const AxisInfo& A = P.ax[a];
    if (!A.active) continue;
    int qa = 1;
    for (int b = 0; b < a; ++b) qa *= q;
    const double invh = P.cell_invh[cell * D + a];
    // gh[r][j] = sum_{i_a} g[r][i(i_a, rest of j)] S[i_a][j_a]
    for (int e = tid; e < NL; e += nt) {
      const int r = e / nloc, j = e - r * nloc;
      const int ja = (j / qa) % q, b0 = j - ja * qa;
      double s = 0.0;
      for (int ia = 0; ia < q; ++ia) s += gs[r * nloc + b0 + ia * qa] * P.S[ia][ja];
      gh[e] = s;
    }
    __syncthreads();
    for (int t = 0; t < A.nadv; ++t) {
      const Term tm = A.adv[t];
      if (tm.sf == SF_ONE) continue;
      const int ci = G.sf_comp[tm.sf];
      if (ci < 0) continue;
      for (int e = tid; e < NL; e += nt) {
        const int r = e / nloc, i = e - r * nloc;
        tmp[e] = gh[e] * csr_row_apply(P.bank, tm.mat, r, ws, nloc, i);
      }
      __syncthreads();
      for (int i = tid; i < nloc; i += nt) {
        double s = 0.0;
        for (int r = 0; r < n; ++r) s += tmp[r * nloc + i];
        nv[i] = -invh * tm.scale * mom_node(P, tm.mf, pnode_of(i)) * s;
      }
      to_snodes(ci);
    }
  }

  // ---- faces: J = sum_t c_t K_t S + |beta| D, lifted with h2 (+-L) into both cells ------------------
  const int qsp = G.qsp;
  for (int a = 0; a < D; ++a) {
    const AxisInfo& A = P.ax[a];
    if (!A.active) continue;
    const bool spatial = A.kind <= SAP_AXIS_Z;
    const double h2 = 0.5 * P.cell_invh[cell * D + a];
    for (int s = 0; s < 2; ++s) {
      const int nb = P.cell_nb[cell * 2 * D + 2 * a + s];
      const int bc = s ? A.bc_hi : A.bc_lo;
      for (int e = tid; e < NF; e += nt) {
        const int r = e / nfp, fp = e - r * nfp;
        double tr = 0.0, tn = 0.0, l = 0.0;
        for (int j = 0; j < q; ++j) {
          const int nd = fnode(fp, j, a, q);
          tr += (s ? P.B1[j] : P.B0[j]) * ws[r * nloc + nd];
          l += (s ? P.L1[j] : -P.L0[j]) * gs[r * nloc + nd];
        }
        if (nb >= 0) {
          const double* xn = w + (size_t)nb * NL + r * nloc;
          for (int j = 0; j < q; ++j) tn += (s ? P.B0[j] : P.B1[j]) * xn[fnode(fp, j, a, q)];
        } else {
          tn = bc == SAP_BC_CONTINUOUS ? tr : 0.0;
        }
        // lower face (s = 0): f_lo = neighbour, f_hi = own; upper face (s = 1): f_lo = own
        fS[e] = tr + tn;
        fD[e] = s ? tr - tn : tn - tr;
        fl[e] = h2 * l;
      }
      __syncthreads();
      // central part: d/dCF_t(fp) = sum_r ell[r][fp] (K_t S)[r][fp]
      for (int t = 0; t < A.nadv; ++t) {
        const Term tm = A.adv[t];
        if (tm.sf == SF_ONE) continue;
        const int ci = spatial ? -1 : G.sf_comp[tm.sf];
        if (!spatial && ci < 0) continue;
        for (int e = tid; e < NF; e += nt) {
          const int r = e / nfp, fp = e - r * nfp;
          fu[e] = fl[e] * csr_row_apply(P.bank, tm.mat, r, fS, nfp, fp);
        }
        __syncthreads();
        for (int fp = tid; fp < nfp; fp += nt) {
          double sm2 = 0.0;
          for (int r = 0; r < n; ++r) sm2 += fu[r * nfp + fp];
          if (spatial) {  // CF = scale U_a(face point) mf(p node): gradient to U_a at the face point
            nv[fp] = tm.scale * mom_node(P, tm.mf, has_mom ? pcell * q + fp / qsp : 0) * sm2;
          } else {        // CF = scale sf(spatial node fp) mf(p face)
            nv[fp] = tm.scale * mom_face(P, tm.mf, pcell + s) * sm2;
          }
        }
        __syncthreads();
        if (spatial) {
          for (int fs = tid; fs < qsp; fs += nt) {
            double acc = 0.0;
            for (int jp = 0; jp < nfp / qsp; ++jp) acc += nv[fs + qsp * jp];
            pc[G.face_off + (2 * a + s) * qsp + fs] += acc;
          }
        } else {
          for (int fp = tid; fp < nfp; fp += nt) pc[ci * qdx + fp] += nv[fp];
        }
        __syncthreads();
      }
      // upwind part
      if (spatial) {
        // |beta| = W |c0 + lam c1| W^T with c0 = CF_0 (U_a), c1 = CF_1 (V): d/dc0 = sum_k u_k sgn v_k
        const Term t0 = A.adv[0], t1 = A.adv[1];
        for (int e = tid; e < NF; e += nt) {
          const int k = e / nfp, fp = e - k * nfp;
          fu[e] = csr_row_apply(P.bank, A.WTmat, k, fl, nfp, fp);
          fv[e] = csr_row_apply(P.bank, A.WTmat, k, fD, nfp, fp);
        }
        __syncthreads();
        const int fb = P.scell_face[scell * 2 * P.dx + 2 * a + s];
        for (int fp = tid; fp < nfp; fp += nt) {
          const int fs = has_mom ? fp % qsp : fp;
          const int pn = has_mom ? pcell * q + fp / qsp : 0;
          const double ua = P.uface_is_uni[a] ? P.uface_uni[a] : P.uface[a][fb + fs];
          const double m0 = t0.scale * mom_node(P, t0.mf, pn);
          const double c0 = m0 * ua;
          const double c1 = t1.scale * mom_node(P, t1.mf, pn);
          double sm2 = 0.0;
          for (int k = 0; k < n; ++k) sm2 += fu[k * nfp + fp] * sgn(c0 + P.lam[k] * c1) * fv[k * nfp + fp];
          nv[fp] = m0 * sm2;
        }
        __syncthreads();
        for (int fs = tid; fs < qsp; fs += nt) {
          double acc = 0.0;
          for (int jp = 0; jp < nfp / qsp; ++jp) acc += nv[fs + qsp * jp];
          pc[G.face_off + (2 * a + s) * qsp + fs] += acc;
        }
        __syncthreads();
      } else if (A.route == ABS_POINT && G.pd_w > 0) {
        // |beta^p| per (spatial node, momentum face): d/dc_t = ell^T P_t D, P_t = d|beta^p|[K_t]
        const int pf = pcell + s;
        const int wpat = G.pd_w;
        for (int t = 0; t < A.nadv; ++t) {
          const Term tm = A.adv[t];
          const double* pd = G.pd[t];
          if (!pd || tm.sf == SF_ONE) continue;
          const int ci = G.sf_comp[tm.sf];
          if (ci < 0) continue;
          for (int e = tid; e < NF; e += nt) {
            const int r = e / nfp, fp = e - r * nfp;
            const int slot = P.pslot[scell * qdx + fp];
            double acc = 0.0;
            if (slot >= 0) {
              const double* pe = pd + (((size_t)slot * P.npface + pf) * wpat) * n + r;
              int idx = P.bank.ell_off[A.absmat] + r;
              for (int k = 0; k < wpat; ++k, idx += n) {
                const int c = reinterpret_cast<const int4*>(P.bank.ell)[idx].x;
                acc += pe[(size_t)k * n] * fD[c * nfp + fp];
              }
            }
            fu[e] = fl[e] * acc;
          }
          __syncthreads();
          for (int fp = tid; fp < nfp; fp += nt) {
            double sm2 = 0.0;
            for (int r = 0; r < n; ++r) sm2 += fu[r * nfp + fp];
            pc[ci * qdx + fp] += tm.scale * mom_face(P, tm.mf, pf) * sm2;
          }
          __syncthreads();
        }
      }
      __syncthreads();
    }
  }
  __syncthreads();
  for (int k = tid; k < G.ps; k += nt) part[(size_t)cell * G.ps + k] += pc[k];
}

// dJ/d(spatial field component) at spatial point sp: sigma * sum over the momentum cells
__global__ void grad_sf_reduce_kernel(const GradTables G, const double* __restrict__ part, int nscell, int qdx,
                                      int npc, double sigma, double* U, double* gradU, double* DUDt, double* Bw) {
  const int total = G.ncomp * nscell * qdx;
  for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < total; it += gridDim.x * blockDim.x) {
    const int ci = it / (nscell * qdx);
    const int sp = it - ci * nscell * qdx;
    const int scell = sp / qdx, sn = sp - scell * qdx;
    double s = 0.0;
    for (int pcl = 0; pcl < npc; ++pcl) s += part[(size_t)(scell + nscell * pcl) * G.ps + ci * qdx + sn];
    const int k = G.comp_sf[ci];
    double* dst = nullptr;
    if (k >= SF_U && k < SF_U + 3) dst = U ? U + (size_t)sp * 3 + (k - SF_U) : nullptr;
    else if (k >= SF_G && k < SF_G + 9) dst = gradU ? gradU + (size_t)sp * 9 + (k - SF_G) : nullptr;
    else if (k >= SF_DU && k < SF_DU + 3) dst = DUDt ? DUDt + (size_t)sp * 3 + (k - SF_DU) : nullptr;
    else if (k >= SF_B && k < SF_B + 3) dst = Bw ? Bw + (size_t)sp * 3 + (k - SF_B) : nullptr;
    if (dst) *dst += sigma * s;
  }
}

// dJ/dU_a at the spatial face points from the face side `side` of every spatial cell (each face
// point is the lower face of one spatial cell and the upper face of one: one pass per side)
__global__ void grad_uface_kernel(const GradTables G, const double* __restrict__ part, const int* __restrict__ sface,
                                  int nscell, int dx, int qsp, int npc, int a, int side, double sigma,
                                  double* __restrict__ out) {
  const int total = nscell * qsp;
  for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < total; it += gridDim.x * blockDim.x) {
    const int scell = it / qsp, fs = it - scell * qsp;
    double s = 0.0;
    for (int pcl = 0; pcl < npc; ++pcl)
      s += part[(size_t)(scell + nscell * pcl) * G.ps + G.face_off + (2 * a + side) * qsp + fs];
    out[sface[scell * 2 * dx + 2 * a + side] + fs] += sigma * s;
  }
}

// grad[node] += coef * sum_{v < nv} g_v[row 0 of the node]  (the source s_000 enters row 0 only)
__global__ void grad_src_kernel(const double* __restrict__ g, int64_t N, int nvec, int n, int nloc, int64_t npv,
                                double coef, double* __restrict__ grad) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < npv; p += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cell = p / nloc;
    const int i = (int)(p - cell * nloc);
    double s = 0.0;
    for (int v = 0; v < nvec; ++v) s += g[(size_t)v * N + (size_t)cell * n * nloc + i];
    grad[p] += coef * s;
  }
}

// w = a + b
__global__ void add2_kernel(const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ w,
                            int64_t N) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x)
    w[k] = a[k] + b[k];
}

cudaError_t launch_coef_adjoint(const OpParams<double>& P, const GradTables& G, const double* g, const double* w,
                                double* part, cudaStream_t s) {
  static DeviceMask opted{};
  const size_t smem = sizeof(double) * (size_t)coef_adjoint_smem_doubles(P, G);
  if (smem > 200 * 1024) return cudaErrorInvalidConfiguration;
  if (cudaError_t err = smem_opt_in(coef_adjoint_kernel, 200 * 1024, opted); err != cudaSuccess) return err;
  coef_adjoint_kernel<<<P.ncell, 128, smem, s>>>(P, G, g, w, part);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_grad_reduce(const OpParams<double>& P, const GradTables& G, const double* part, int nscell,
                               int npc, double sigma, const sap_field_grads& out, cudaStream_t s) {
  if (G.ncomp > 0 && (out.U || out.gradU || out.DUDt || out.Bw)) {
    grad_sf_reduce_kernel<<<256, 256, 0, s>>>(G, part, nscell, P.qdx, npc, sigma, out.U, out.gradU, out.DUDt, out.Bw);
    note_launch();
  }
  for (int a = 0; a < P.dx; ++a) {
    if (!out.Uface[a] || !P.ax[a].active) continue;
    for (int side = 0; side < 2; ++side) {
      grad_uface_kernel<<<256, 256, 0, s>>>(G, part, P.scell_face, nscell, P.dx, G.qsp, npc, a, side, sigma,
                                            out.Uface[a]);
      note_launch();
    }
  }
  return cudaGetLastError();
}

cudaError_t launch_grad_src(const double* g, int64_t N, int nvec, int n, int nloc, int64_t npv, double coef,
                            double* grad, cudaStream_t s) {
  grad_src_kernel<<<1024, 256, 0, s>>>(g, N, nvec, n, nloc, npv, coef, grad);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_add2(const double* a, const double* b, double* w, int64_t N, cudaStream_t s) {
  add2_kernel<<<1024, 256, 0, s>>>(a, b, w, N);
  note_launch();
  return cudaGetLastError();
}

}  // namespace sap
