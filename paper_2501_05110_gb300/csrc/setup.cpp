// Host set-up and the C ABI entry points of sap.h.
//
// Builds everything the kernels read: the Gauss rule and 1-D Lagrange tables, mesh connectivity,
// the coupling matrices (sh_tables.cpp), the advection / reaction term lists of Sec. 2.2
// (Eq. definitions-advection-reaction-eq) with their coefficient factors, and the face upwind data:
// the eigen-pairs of A^x computed once and rotated for y and z (Sec. 3.2), and the eigen-pairs of
// beta^p at every momentum-face point (Sec. 3.2, Eq. beta-p).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <exception>
#include <map>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "sap_internal.h"

using namespace sap;

static std::string g_create_error;

// Every entry point returns a status: host exceptions (allocation failures of host containers and
// the like) become status codes here instead of crossing the C boundary.  Errors of a call without
// a handle go to the creation-error text.
template <typename F>
static sap_status guarded(sap_ctx* c, const char* what, F&& body) {
  auto note = [&](const std::string& msg) {
    try {
      (c ? c->err : g_create_error) = std::string(what) + ": " + msg;
    } catch (...) {
    }
  };
  try {
    return body();
  } catch (const std::bad_alloc&) {
    note("host allocation failed");
    return SAP_ENOMEM;
  } catch (const std::exception& e) {
    note(e.what());
    return SAP_EINVAL;
  } catch (const std::string& e) {
    note(e);
    return SAP_EINVAL;
  }
}

// ------------------------------------------------------------------------------------------------
// 1-D Gauss--Legendre rule on [0,1] (Newton on the three-term recurrence) and Lagrange tables
// ------------------------------------------------------------------------------------------------
static void gauss_legendre01(int q, std::vector<double>& x, std::vector<double>& w) {
  x.resize(q);
  w.resize(q);
  for (int i = 0; i < q; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (q + 0.5)), dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = 0.0;
      for (int j = 1; j <= q; ++j) {
        double p2 = p1;
        p1 = p0;
        p0 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p2) / j;
      }
      dp = q * (z * p0 - p1) / (z * z - 1.0);
      double dz = p0 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    // recompute derivative at the converged root
    double p0 = 1.0, p1 = 0.0;
    for (int j = 1; j <= q; ++j) {
      double p2 = p1;
      p1 = p0;
      p0 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p2) / j;
    }
    dp = q * (z * p0 - p1) / (z * z - 1.0);
    x[q - 1 - i] = 0.5 * (z + 1.0);
    w[q - 1 - i] = 1.0 / ((1.0 - z * z) * dp * dp);  // 2/((1-z^2)p'^2) halved for [0,1]
  }
}

static double lagr(const std::vector<double>& nd, int i, double t) {
  double v = 1.0;
  for (size_t j = 0; j < nd.size(); ++j)
    if ((int)j != i) v *= (t - nd[j]) / (nd[i] - nd[j]);
  return v;
}

static double dlagr(const std::vector<double>& nd, int i, double t) {
  double s = 0.0;
  for (size_t k = 0; k < nd.size(); ++k) {
    if ((int)k == i) continue;
    double v = 1.0 / (nd[i] - nd[k]);
    for (size_t j = 0; j < nd.size(); ++j)
      if ((int)j != i && j != k) v *= (t - nd[j]) / (nd[i] - nd[j]);
    s += v;
  }
  return s;
}

// ------------------------------------------------------------------------------------------------
// device memory helpers
// ------------------------------------------------------------------------------------------------
template <typename V>
static void* upload(sap_ctx* c, const std::vector<V>& h, std::vector<DevBuf>& owner) {
  if (h.empty()) return nullptr;
  void* p = nullptr;
  size_t bytes = h.size() * sizeof(V);
  if (cudaMalloc(&p, bytes) != cudaSuccess) throw std::string("cudaMalloc failed");
  if (cudaMemcpy(p, h.data(), bytes, cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(p);
    throw std::string("cudaMemcpy failed");
  }
  owner.push_back({p, bytes});
  return p;
}

template <typename V>
static std::vector<float> to_f32(const std::vector<V>& v) {
  return std::vector<float>(v.begin(), v.end());
}

// The forward apply's kernel (sap_set_apply_kernel): the node kernel where the problem fits it and
// it is not switched off, else the row kernel.
static void apply_kernel_choice(sap_ctx* c) {
  const bool uni = c->apply_kernel == SAP_KERNEL_AUTO && c->uni_avail >= 0;
  c->p64.uni_L = c->p32.uni_L = uni ? c->uni_avail : -1;
  c->p64.uni = uni ? static_cast<const void*>(c->uni_v64.data()) : nullptr;
  c->p32.uni = uni ? static_cast<const void*>(c->uni_v32.data()) : nullptr;
  c->p64.uni_cells = c->p32.uni_cells = c->uni_cells;
}

static void free_bufs(std::vector<DevBuf>& v) {
  for (auto& b : v) cudaFree(b.p);
  v.clear();
}

// ------------------------------------------------------------------------------------------------
// create
// ------------------------------------------------------------------------------------------------
static bool is_spatial(int k) { return k >= SAP_AXIS_X && k <= SAP_AXIS_Z; }

static std::string validate(const sap_desc* d) {
  if (!d) return "null descriptor";
  if (d->ndim < 1 || d->ndim > 3) return "ndim must be 1..3";
  int dx = 0;
  for (int a = 0; a < d->ndim; ++a) {
    int k = d->axis_kind[a];
    if (is_spatial(k)) {
      if (k != a) return "spatial axes must be x, y, z in this order starting at axis 0";
      ++dx;
    } else if (k == SAP_AXIS_P || k == SAP_AXIS_LNP) {
      if (a != d->ndim - 1) return "the momentum axis must be the last axis";
    } else {
      return "unknown axis kind";
    }
    if (d->ncells[a] < 1) return "ncells must be >= 1";
    if (!d->edges[a]) return "missing edges";
    for (int i = 0; i < d->ncells[a]; ++i)
      if (!(d->edges[a][i + 1] > d->edges[a][i])) return "edges must increase strictly";
    if (k == SAP_AXIS_P && !(d->edges[a][0] > 0)) return "linear momentum axis must have p > 0";
    bool plo = d->bc_lo[a] == SAP_BC_PERIODIC, phi = d->bc_hi[a] == SAP_BC_PERIODIC;
    if (plo != phi) return "periodic must be set on both ends of an axis";
    for (int bc : {d->bc_lo[a], d->bc_hi[a]})
      if (bc < 0 || bc > 2) return "unknown boundary condition";
  }
  if (dx == 0 && d->ndim > 1) return "a momentum-only problem must be one-dimensional";
  bool mom = !is_spatial(d->axis_kind[d->ndim - 1]);
  if ((d->terms & SAP_TERM_MOM) && !mom) return "momentum terms need a momentum axis";
  if (d->lmax < 0 || d->lmax > 11) return "lmax must be 0..11";
  if (d->degree < 0 || d->degree > MAXQ - 1) return "degree must be 0..5";
  if (!mom && !(d->V > 0)) return "particle speed V must be > 0 without a momentum axis";
  return "";
}

static double mom_factor_h(int mf, double p, bool has_mom, double Vm) {
  if (mf == MF_ONE) return 1.0;
  if (!has_mom) return mf == MF_V ? Vm : (mf == MF_INV_V ? 1.0 / Vm : 1.0);
  double gm = std::sqrt(1.0 + p * p);
  switch (mf) {
    case MF_P: return p;
    case MF_GM: return gm;
    case MF_V: return p / gm;
    case MF_INV_V: return gm / p;
    case MF_INV_GM: return 1.0 / gm;
    case MF_INV_P: return 1.0 / p;
    case MF_INV_GMP: return 1.0 / (gm * p);
    case MF_GM_OVER_P: return gm / p;
  }
  return 1.0;
}

template <typename T>
static void fill_1d_tables(sap_ctx* c, OpParams<T>& P) {
  const int q = c->q;
  for (int i = 0; i < q; ++i) {
    P.B0[i] = T(lagr(c->xg, i, 0.0));
    P.B1[i] = T(lagr(c->xg, i, 1.0));
    P.L0[i] = T(lagr(c->xg, i, 0.0) / c->wg[i]);
    P.L1[i] = T(lagr(c->xg, i, 1.0) / c->wg[i]);
    for (int k = 0; k < q; ++k) P.S[i][k] = T(c->wg[k] * dlagr(c->xg, i, c->xg[k]) / c->wg[i]);
  }
}

extern "C" sap_status sap_create(const sap_desc* desc, int prec, sap_handle* out) {
  return guarded(nullptr, "sap_create", [&]() -> sap_status {
    if (!out) {
      g_create_error = "null output handle";
      return SAP_EINVAL;
    }
    *out = nullptr;
    std::string v = validate(desc);
    if (!v.empty()) {
      g_create_error = v;
      return SAP_EINVAL;
    }
    if (prec != SAP_PREC_FP64 && prec != SAP_PREC_FP32) {
      g_create_error = "unknown precision";
      return SAP_EINVAL;
    }
    sap_ctx* c = new sap_ctx();
    try {
      c->desc = *desc;
      c->prec = prec;
      c->D = desc->ndim;
      c->q = desc->degree + 1;
      c->n = (desc->lmax + 1) * (desc->lmax + 1);
      c->nloc = 1;
      for (int a = 0; a < c->D; ++a) c->nloc *= c->q;
      c->nfp = c->nloc / c->q;
      c->has_mom = !is_spatial(desc->axis_kind[c->D - 1]);
      c->dx = c->D - c->has_mom;
      c->qdx = 1;
      for (int a = 0; a < c->dx; ++a) c->qdx *= c->q;
      c->ncell = 1;
      for (int a = 0; a < c->D; ++a) {
        c->nc[a] = desc->ncells[a];
        c->ncell *= desc->ncells[a];
        c->edges[a].assign(desc->edges[a], desc->edges[a] + desc->ncells[a] + 1);
        c->desc.edges[a] = c->edges[a].data();
      }
      c->N = (int64_t)c->ncell * c->n * c->nloc;
      c->nscell = 1;
      for (int a = 0; a < c->dx; ++a) c->nscell *= c->nc[a];
      c->npc = c->has_mom ? c->nc[c->D - 1] : 1;
      c->nsv = c->nscell * c->qdx;
      c->npv = c->ncell * c->nloc;
      gauss_legendre01(c->q, c->xg, c->wg);
      c->T = build_sh_tables(desc->lmax);
      // momentum node and face values
      if (c->has_mom) {
        const int a = c->D - 1;
        const bool lg = desc->axis_kind[a] == SAP_AXIS_LNP;
        for (int pc = 0; pc < c->npc; ++pc)
          for (int j = 0; j < c->q; ++j) {
            double crd = c->edges[a][pc] + (c->edges[a][pc + 1] - c->edges[a][pc]) * c->xg[j];
            c->pnode.push_back(lg ? std::exp(crd) : crd);
          }
        for (int f = 0; f <= c->npc; ++f) c->pface.push_back(lg ? std::exp(c->edges[a][f]) : c->edges[a][f]);
      } else {
        c->pnode.assign(c->q, 1.0);
        c->pface.assign(2, 1.0);
      }
      // mesh connectivity
      std::vector<int> nb((size_t)c->ncell * 2 * c->D), scell(c->ncell), pcell(c->ncell);
      std::vector<double> invh((size_t)c->ncell * c->D);
      for (int cell = 0; cell < c->ncell; ++cell) {
        int idx[3] = {0, 0, 0}, rest = cell, stride[3];
        int st = 1;
        for (int a = 0; a < c->D; ++a) {
          idx[a] = rest % c->nc[a];
          rest /= c->nc[a];
          stride[a] = st;
          st *= c->nc[a];
        }
        for (int a = 0; a < c->D; ++a) {
          invh[(size_t)cell * c->D + a] = 1.0 / (c->edges[a][idx[a] + 1] - c->edges[a][idx[a]]);
          bool per = desc->bc_lo[a] == SAP_BC_PERIODIC;
          int lo = idx[a] > 0 ? cell - stride[a] : (per ? cell + (c->nc[a] - 1) * stride[a] : -1);
          int hi = idx[a] < c->nc[a] - 1 ? cell + stride[a] : (per ? cell - (c->nc[a] - 1) * stride[a] : -1);
          nb[(size_t)cell * 2 * c->D + 2 * a] = lo;
          nb[(size_t)cell * 2 * c->D + 2 * a + 1] = hi;
        }
        int sc = 0, sst = 1;
        for (int a = 0; a < c->dx; ++a) {
          sc += idx[a] * sst;
          sst *= c->nc[a];
        }
        scell[cell] = sc;
        pcell[cell] = c->has_mom ? idx[c->D - 1] : 0;
      }
      // spatial face point bases: faces along spatial axis a, ordered (face position, tangential
      // spatial cell with lower axes fastest, tangential spatial node)
      const int qt = c->qdx / c->q;  // tangential spatial nodes per face
      c->scell_face_h.assign((size_t)c->nscell * 2 * std::max(c->dx, 1), 0);
      for (int a = 0; a < c->dx; ++a) {
        int ntang = c->nscell / c->nc[a];
        c->nsf[a] = (c->nc[a] + 1) * ntang * qt;
        for (int sc = 0; sc < c->nscell; ++sc) {
          int idx[3] = {0, 0, 0}, rest = sc;
          for (int b = 0; b < c->dx; ++b) {
            idx[b] = rest % c->nc[b];
            rest /= c->nc[b];
          }
          int tc = 0, tst = 1;
          for (int b = 0; b < c->dx; ++b) {
            if (b == a) continue;
            tc += idx[b] * tst;
            tst *= c->nc[b];
          }
          bool per = desc->bc_lo[a] == SAP_BC_PERIODIC;
          int flo = (idx[a] == 0 && per) ? c->nc[a] : idx[a];
          int fhi = idx[a] + 1;
          c->scell_face_h[(size_t)sc * 2 * c->dx + 2 * a] = (flo * ntang + tc) * qt;
          c->scell_face_h[(size_t)sc * 2 * c->dx + 2 * a + 1] = (fhi * ntang + tc) * qt;
        }
      }
      // A^x blocks for the eigen route
      c->Ablocks = connected_blocks(c->T.A[0]);
      // device mesh tables (both precisions share the integer tables)
      auto& own = c->owned;
      int* d_nb = (int*)upload(c, nb, own);
      int* d_sc = (int*)upload(c, scell, own);
      int* d_pc = (int*)upload(c, pcell, own);
      int* d_sf = (int*)upload(c, c->scell_face_h, own);
      double* d_ih64 = (double*)upload(c, invh, own);
      float* d_ih32 = (float*)upload(c, to_f32(invh), own);
      double* d_pn64 = (double*)upload(c, c->pnode, own);
      float* d_pn32 = (float*)upload(c, to_f32(c->pnode), own);
      double* d_pf64 = (double*)upload(c, c->pface, own);
      float* d_pf32 = (float*)upload(c, to_f32(c->pface), own);
      // momentum factor tables (MF_*) at nodes and faces
      const int npn = (int)c->pnode.size(), npf = (int)c->pface.size();
      std::vector<double> mfn((size_t)MF_COUNT * npn), mff((size_t)MF_COUNT * npf);
      for (int mf = 0; mf < MF_COUNT; ++mf) {
        for (int i = 0; i < npn; ++i) mfn[(size_t)mf * npn + i] = mom_factor_h(mf, c->pnode[i], c->has_mom, desc->V);
        for (int i = 0; i < npf; ++i) mff[(size_t)mf * npf + i] = mom_factor_h(mf, c->pface[i], c->has_mom, desc->V);
      }
      double* d_mfn64 = (double*)upload(c, mfn, own);
      float* d_mfn32 = (float*)upload(c, to_f32(mfn), own);
      double* d_mff64 = (double*)upload(c, mff, own);
      float* d_mff32 = (float*)upload(c, to_f32(mff), own);
      auto base = [&](auto& P, auto* ih, auto* pn, auto* pf, auto* mn, auto* mfc) {
        P.D = c->D; P.dx = c->dx; P.q = c->q; P.nloc = c->nloc; P.nfp = c->nfp; P.n = c->n;
        P.ncell = c->ncell; P.has_mom = c->has_mom; P.qdx = c->qdx;
        for (int a = 0; a < 3; ++a) P.nc[a] = c->nc[a];
        P.cell_nb = d_nb; P.cell_scell = d_sc; P.cell_pcell = d_pc; P.scell_face = d_sf;
        P.cell_invh = ih; P.pnode = pn; P.pface = pf; P.npface = npf; P.mfn = mn; P.mff = mfc; P.npn = npn;
        P.nsv = c->nsv;
        P.Vmono = c->has_mom ? 1 : desc->V;
        fill_1d_tables(c, P);
      };
      base(c->p64, d_ih64, d_pn64, d_pf64, d_mfn64, d_mff64);
      base(c->p32, d_ih32, d_pn32, d_pf32, d_mfn32, d_mff32);
      // block partial sums of the Krylov reductions
      if (cudaMalloc(&c->small, sizeof(double) * krylov_scratch_doubles(c->N)) != cudaSuccess) throw std::string("cudaMalloc failed");
      if (cudaMalloc(&c->gdev, gmres_control_bytes()) != cudaSuccess ||
          cudaMemset(c->gdev, 0, gmres_control_bytes()) != cudaSuccess)
        throw std::string("cudaMalloc failed");
      if (cudaMallocHost(&c->gdev_host, gmres_control_bytes()) != cudaSuccess) throw std::string("cudaMallocHost failed");
      std::memset(c->gdev_host, 0, gmres_control_bytes());
    } catch (const std::string& e) {
      g_create_error = "sap_create: " + e;
      sap_destroy(c);
      return SAP_ENOMEM;
    } catch (const std::exception& e) {
      sap_destroy(c);
      throw;  // reported by the guard
    }
    *out = c;
    return SAP_OK;
  });
}

extern "C" sap_status sap_create_batch(int ninst, const sap_desc* descs, int prec, sap_handle* out) {
  return guarded(nullptr, "sap_create_batch", [&]() -> sap_status {
    if (!out || !descs || ninst < 1) {
      g_create_error = "sap_create_batch: bad arguments";
      return SAP_EINVAL;
    }
    *out = nullptr;
    sap_ctx* c = new sap_ctx();
    c->prec = prec;
    std::vector<int64_t> Ns;
    for (int i = 0; i < ninst; ++i) {
      sap_handle sub = nullptr;
      sap_status st = sap_create(&descs[i], prec, &sub);
      if (st != SAP_OK) {
        g_create_error = "sap_create_batch: instance " + std::to_string(i) + ": " + g_create_error;
        for (auto* s2 : c->sub) {
          s2->parent = nullptr;
          sap_destroy(s2);
        }
        delete c;
        return st;
      }
      sub->parent = c;
      c->inst_off.push_back(c->N);
      c->N += sub->N;
      Ns.push_back(sub->N);
      c->sub.push_back(sub);
    }
    if (cudaMalloc(&c->small, sizeof(double) * krylov_batch_scratch_doubles(Ns)) != cudaSuccess) {
      g_create_error = "sap_create_batch: allocation failed";
      sap_destroy(c);
      return SAP_ENOMEM;
    }
    *out = c;
    return SAP_OK;
  });
}

extern "C" sap_status sap_batch_instance(sap_handle c, int inst, sap_handle* sub, int64_t* offset) {
  if (!c || c->sub.empty() || inst < 0 || inst >= (int)c->sub.size()) return SAP_EINVAL;
  if (sub) *sub = c->sub[inst];
  if (offset) *offset = c->inst_off[inst];
  return SAP_OK;
}

// ------------------------------------------------------------------------------------------------
// points
// ------------------------------------------------------------------------------------------------
extern "C" sap_status sap_field_points(sap_handle c, int which, double* coords, int64_t* count) {
  return guarded(c, "sap_field_points", [&]() -> sap_status {
    if (!c || !count) return SAP_EINVAL;
    const int q = c->q;
    std::vector<double> out;
    if (which == SAP_PTS_SPATIAL) {
      *count = c->nsv;
      if (!coords) return SAP_OK;
      for (int sc = 0; sc < c->nscell; ++sc) {
        int idx[3] = {0, 0, 0}, rest = sc;
        for (int a = 0; a < c->dx; ++a) {
          idx[a] = rest % c->nc[a];
          rest /= c->nc[a];
        }
        for (int nd = 0; nd < c->qdx; ++nd) {
          int r2 = nd;
          for (int a = 0; a < c->dx; ++a) {
            int j = r2 % q;
            r2 /= q;
            double lo = c->edges[a][idx[a]], h = c->edges[a][idx[a] + 1] - lo;
            coords[((size_t)sc * c->qdx + nd) * c->dx + a] = lo + h * c->xg[j];
          }
        }
      }
      return SAP_OK;
    }
    if (which >= SAP_PTS_FACE_X && which <= SAP_PTS_FACE_Z) {
      int a = which - SAP_PTS_FACE_X;
      if (a >= c->dx) {
        *count = 0;
        return SAP_OK;
      }
      *count = c->nsf[a];
      if (!coords) return SAP_OK;
      const int qt = c->qdx / q;
      const int ntang = c->nscell / c->nc[a];
      for (int f = 0; f <= c->nc[a]; ++f)
        for (int tc = 0; tc < ntang; ++tc) {
          int tidx[3] = {0, 0, 0}, rest = tc;
          for (int b = 0; b < c->dx; ++b) {
            if (b == a) continue;
            tidx[b] = rest % c->nc[b];
            rest /= c->nc[b];
          }
          for (int nd = 0; nd < qt; ++nd) {
            size_t pidx = ((size_t)f * ntang + tc) * qt + nd;
            int r2 = nd;
            for (int b = 0; b < c->dx; ++b) {
              double v;
              if (b == a) {
                v = c->edges[a][f];
              } else {
                int j = r2 % q;
                r2 /= q;
                double lo = c->edges[b][tidx[b]], h = c->edges[b][tidx[b] + 1] - lo;
                v = lo + h * c->xg[j];
              }
              coords[pidx * c->dx + b] = v;
            }
          }
        }
      return SAP_OK;
    }
    if (which == SAP_PTS_PHASE) {
      *count = c->npv;
      if (!coords) return SAP_OK;
      for (int cell = 0; cell < c->ncell; ++cell) {
        int idx[3] = {0, 0, 0}, rest = cell;
        for (int a = 0; a < c->D; ++a) {
          idx[a] = rest % c->nc[a];
          rest /= c->nc[a];
        }
        for (int nd = 0; nd < c->nloc; ++nd) {
          int r2 = nd;
          for (int a = 0; a < c->D; ++a) {
            int j = r2 % q;
            r2 /= q;
            double lo = c->edges[a][idx[a]], h = c->edges[a][idx[a] + 1] - lo;
            coords[((size_t)cell * c->nloc + nd) * c->D + a] = lo + h * c->xg[j];
          }
        }
      }
      return SAP_OK;
    }
    return SAP_EINVAL;
  });
}

// ------------------------------------------------------------------------------------------------
// fields -> term lists, matrix bank, face upwind data
// ------------------------------------------------------------------------------------------------
struct HostCSR {
  std::vector<int> rp, col;
  std::vector<double> val;
};

static HostCSR to_csr(const Mat& m, double drop = 0.0) {
  HostCSR h;
  h.rp.push_back(0);
  for (int i = 0; i < m.n; ++i) {
    for (int j = 0; j < m.n; ++j)
      if (std::fabs(m(i, j)) > drop) {
        h.col.push_back(j);
        h.val.push_back(m(i, j));
      }
    h.rp.push_back((int)h.col.size());
  }
  return h;
}

// body(i, scratch) for i = 0 .. count-1 on the host's cores (each i on one thread; `scratch` is a
// per-thread buffer).  Used for the per-point eigen-decompositions of the momentum-face set-up.
template <typename F>
static void parallel_for(int count, F&& body) {
  const unsigned hw = std::thread::hardware_concurrency();
  const int nt = (int)std::min<unsigned>(hw ? hw : 1u, 64u);
  if (nt < 2 || count < 4 * nt) {
    std::vector<double> scratch;
    for (int i = 0; i < count; ++i) body(i, scratch);
    return;
  }
  std::atomic<int> next{0};
  std::atomic<bool> failed{false};
  auto run = [&]() {
    std::vector<double> scratch;
    try {
      for (;;) {
        const int i0 = next.fetch_add(8);
        if (i0 >= count) break;
        for (int i = i0; i < std::min(count, i0 + 8); ++i) body(i, scratch);
      }
    } catch (...) {
      failed = true;
    }
  };
  std::vector<std::thread> th;
  for (int k = 1; k < nt; ++k) {
    try {
      th.emplace_back(run);
    } catch (...) {
      break;  // fewer threads: the remaining work is shared by those that started
    }
  }
  run();
  for (auto& t : th) t.join();
  if (failed) throw std::bad_alloc();
}

// Inputs of the momentum-face upwind data (kept after sap_set_fields for the derivative tables of the
// adjoint): the block pattern of beta^p, each advection term scattered into it, the fields.
struct MomFaceSrc {
  int axis = -1;
  HostCSR pat;                                                 // dense within each block
  std::vector<std::vector<int>> blocks;
  std::vector<std::vector<std::pair<int, double>>> tpos;       // per term: (pattern position, value)
  int nadv = 0;
  Term adv[MAXADV];
  std::vector<double> sf;                                      // [SF_NCOMP][nsv]
  double V = 1.0;
  bool has_mom = false;
  std::vector<int> pslot;
  int nslot = 0;
  // beta^p (Eq. beta-p; the ln p form through the term factors) at spatial node sp and momentum p,
  // on the block pattern
  void beta_at(int sp, double p, int nsv, std::vector<double>& pv) const {
    pv.assign(pat.col.size(), 0.0);
    for (int t = 0; t < nadv; ++t) {
      const Term& tm = adv[t];
      const double cf = tm.scale * (tm.sf == SF_ONE ? 1.0 : sf[(size_t)tm.sf * nsv + sp]) *
                        mom_factor_h(tm.mf, p, has_mom, V);
      for (const auto& pr : tpos[t]) pv[pr.first] += cf * pr.second;
    }
  }
};

struct FieldStore {  // per-context field-dependent device buffers and host inputs
  std::vector<DevBuf> bufs;
  MomFaceSrc mom;
  std::vector<DevBuf> gbufs;  // derivative tables of the adjoint's field gradients
};
static std::map<sap_ctx*, FieldStore> g_fields;

struct BankBuilder {
  std::vector<HostCSR> mats;
  std::map<std::string, int> ids;
  int add(const std::string& key, const Mat& m) {
    auto it = ids.find(key);
    if (it != ids.end()) return it->second;
    mats.push_back(to_csr(m));
    ids[key] = (int)mats.size() - 1;
    return ids[key];
  }
  int add_csr(const std::string& key, const HostCSR& h) {
    mats.push_back(h);
    ids[key] = (int)mats.size() - 1;
    return ids[key];
  }
};

template <typename T>
static void set_bank(OpParams<T>& P, const BankBuilder& B, sap_ctx* c, std::vector<DevBuf>& own) {
  std::vector<int> rp, col;
  std::vector<double> val;
  if (B.mats.size() > 96) throw std::string("too many matrices");
  for (size_t m = 0; m < B.mats.size(); ++m) {
    P.bank.rp_off[m] = (int)rp.size();
    int off = (int)col.size();
    for (int v : B.mats[m].rp) rp.push_back(v + off);
    col.insert(col.end(), B.mats[m].col.begin(), B.mats[m].col.end());
    val.insert(val.end(), B.mats[m].val.begin(), B.mats[m].val.end());
  }
  if (col.empty()) {
    col.push_back(0);
    val.push_back(0.0);
  }
  if (rp.empty()) rp.push_back(0);
  c->bank_nnz.clear();
  for (size_t m = 0; m < B.mats.size(); ++m) c->bank_nnz.push_back((double)B.mats[m].col.size());
  std::vector<double> dgv(std::max<size_t>(c->n, B.mats.size() * c->n), 0.0);  // >= n: see csr_diag
  for (size_t m = 0; m < B.mats.size(); ++m)
    for (int i = 0; i < c->n; ++i)
      for (int k = B.mats[m].rp[i]; k < B.mats[m].rp[i + 1]; ++k)
        if (B.mats[m].col[k] == i) dgv[m * c->n + i] = B.mats[m].val[k];
  if (sizeof(T) == 8) P.bank.dg = (const T*)upload(c, dgv, own);
  else P.bank.dg = (const T*)upload(c, to_f32(dgv), own);
  // ELL copy: slot k of row r at ell_off[m] + k n + r; rows shorter than the widest are padded (r, 0)
  std::vector<EllEntry<T>> ell;
  for (size_t m = 0; m < B.mats.size(); ++m) {
    const HostCSR& h = B.mats[m];
    int w = 0;
    for (int i = 0; i < c->n; ++i) w = std::max(w, h.rp[i + 1] - h.rp[i]);
    P.bank.ell_off[m] = (int)ell.size();
    P.bank.ell_w[m] = w;
    for (int k = 0; k < w; ++k)
      for (int i = 0; i < c->n; ++i) {
        EllEntry<T> e{};
        const bool in = h.rp[i] + k < h.rp[i + 1];
        e.col = in ? h.col[h.rp[i] + k] : i;
        e.val = in ? T(h.val[h.rp[i] + k]) : T(0);
        ell.push_back(e);
      }
  }
  // n spare entries at the end: a load of slot 0 of an empty last matrix stays inside the table
  for (int i = 0; i < c->n; ++i) ell.push_back(EllEntry<T>{i, T(0)});
  P.bank.ell = upload(c, ell, own);
  P.bank.rp = (const int*)upload(c, rp, own);
  P.bank.col = (const int*)upload(c, col, own);
  if (sizeof(T) == 8) P.bank.val = (const T*)upload(c, val, own);
  else P.bank.val = (const T*)upload(c, to_f32(val), own);
}

extern "C" sap_status sap_set_fields(sap_handle c, const double* U, const double* gradU, const double* DUDt,
                                     const double* Bw, const double* const Uface[3], const double* nu,
                                     const double* s000) {
  return guarded(c, "sap_set_fields", [&]() -> sap_status {
    if (!c) return SAP_EINVAL;
    try {
      FieldStore& fs = g_fields[c];
      // the old field buffers go now: until this call succeeds the context has no fields, so no
      // compute call can read a freed buffer after a failure part-way
      c->fields_set = false;
      free_bufs(fs.bufs);
      // tables that lived in those buffers
      c->p64.cvtab = nullptr; c->p64.cftab = nullptr; c->p64.mktab = nullptr; c->p64.rdtab = nullptr;
      c->p32.cvtab = nullptr; c->p32.cftab = nullptr; c->p32.mktab = nullptr; c->p32.rdtab = nullptr;
      free_bufs(fs.gbufs);
      fs.mom = MomFaceSrc{};
      const sap_desc& d = c->desc;
      const int n = c->n, nsv = c->nsv;
      const unsigned terms = d.terms;
      // spatial field components [SF_NCOMP][nsv]
      std::vector<double> sf((size_t)SF_NCOMP * nsv, 0.0);
      for (int p = 0; p < nsv; ++p) {
        for (int a = 0; a < 3; ++a) {
          if (U) sf[(size_t)(SF_U + a) * nsv + p] = U[(size_t)p * 3 + a];
          if (DUDt) sf[(size_t)(SF_DU + a) * nsv + p] = DUDt[(size_t)p * 3 + a];
          if (Bw) sf[(size_t)(SF_B + a) * nsv + p] = Bw[(size_t)p * 3 + a];
          for (int b = 0; b < 3; ++b)
            if (gradU) sf[(size_t)(SF_G + 3 * a + b) * nsv + p] = gradU[(size_t)p * 9 + 3 * a + b];
        }
      }
      bool nonzero[SF_NCOMP], uni[SF_NCOMP];
      double uval[SF_NCOMP];
      for (int k = 0; k < SF_NCOMP; ++k) {
        nonzero[k] = false;
        uni[k] = true;
        uval[k] = nsv ? sf[(size_t)k * nsv] : 0.0;
        for (int p = 0; p < nsv; ++p) {
          double v = sf[(size_t)k * nsv + p];
          if (v != 0.0) nonzero[k] = true;
          if (v != uval[k]) uni[k] = false;
        }
      }
      // the FP32 row kernel skips, per cell, terms whose coefficient is zero at all its nodes: the
      // fraction of spatial cells where each component's FP32 value vanishes (cost model)
      for (int k = 0; k < SF_NCOMP; ++k) {
        int z = 0;
        for (int sc = 0; sc < c->nscell; ++sc) {
          bool all0 = true;
          for (int j2 = 0; j2 < c->qdx && all0; ++j2) all0 = float(sf[(size_t)k * nsv + (size_t)sc * c->qdx + j2]) == 0.0f;
          z += all0 ? 1 : 0;
        }
        c->sf_zero_frac32[k] = c->nscell ? double(z) / c->nscell : 0.0;
      }
      const bool has_mom = c->has_mom;
      const bool lnp = has_mom && d.axis_kind[c->D - 1] == SAP_AXIS_LNP;
      BankBuilder B;
      const SHTables& Tb = c->T;
      auto A_id = [&](int a) { return B.add("A" + std::to_string(a), Tb.A[a]); };
      auto AA_id = [&](int a, int b) { return B.add("AA" + std::to_string(a) + std::to_string(b), Tb.AA[a][b]); };
      std::vector<Term> react;
      auto add_term = [&](std::vector<Term>& v, int mat, int sfc, int mf, int nuf, double sc) {
        int matT = MAT_I;
        if (mat != MAT_I) {
          std::string key;
          for (auto& kv : B.ids)
            if (kv.second == mat) key = kv.first;
          Mat m(n);
          const HostCSR& h = B.mats[mat];
          for (int i = 0; i < n; ++i)
            for (int k = h.rp[i]; k < h.rp[i + 1]; ++k) m(h.col[k], i) = h.val[k];
          matT = B.add(key + "^T", m);
        }
        v.push_back(Term{mat, matT, sfc, mf, nuf, sc});
      };
      // reaction matrix R - div(beta)  (Eq. definitions-advection-reaction-eq, Eq. linear-system-...)
      if (terms & SAP_TERM_MOM) {
        for (int a = 0; a < 3; ++a)
          if (nonzero[SF_DU + a]) add_term(react, B.add("E" + std::to_string(a), Tb.E[a]), SF_DU + a, MF_INV_V, 0, 1.0);
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b)
            if (nonzero[SF_G + 3 * a + b])
              add_term(react, B.add("F" + std::to_string(a) + std::to_string(b), Tb.F[a][b]), SF_G + 3 * a + b, MF_ONE, 0, 1.0);
      }
      if (terms & SAP_TERM_ROT)
        for (int a = 0; a < 3; ++a)
          if (nonzero[SF_B + a])
            add_term(react, B.add("Om" + std::to_string(a), Tb.Om[a]), SF_B + a, has_mom ? MF_INV_GM : MF_ONE, 0, -1.0);
      if (terms & SAP_TERM_COLL) add_term(react, B.add("C", Tb.C), SF_ONE, MF_ONE, 1, 1.0);
      if (terms & SAP_TERM_ADV)
        for (int a = 0; a < c->dx; ++a)
          if (nonzero[SF_G + 3 * a + a]) add_term(react, MAT_I, SF_G + 3 * a + a, MF_ONE, 0, -1.0);
      if ((terms & SAP_TERM_MOM) && has_mom) {
        if (!lnp) {  // -d/dp beta^p = +V DU_a A^a + dU_b/dx^a A^a A^b
          for (int a = 0; a < 3; ++a)
            if (nonzero[SF_DU + a]) add_term(react, A_id(a), SF_DU + a, MF_V, 0, 1.0);
          for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
              if (nonzero[SF_G + 3 * a + b]) add_term(react, AA_id(a, b), SF_G + 3 * a + b, MF_ONE, 0, 1.0);
        } else {  // -p d/dp (beta^p/p) = -DU_a A^a / (gamma m p)
          for (int a = 0; a < 3; ++a)
            if (nonzero[SF_DU + a]) add_term(react, A_id(a), SF_DU + a, MF_INV_GMP, 0, -1.0);
        }
      }
      if ((int)react.size() > MAXTERMS) throw std::string("too many reaction terms");
      // advection terms per axis
      AxisInfo ax[MAXD];
      std::memset(ax, 0, sizeof(ax));
      for (int a = 0; a < c->D; ++a) {
        AxisInfo& A = ax[a];
        A.kind = d.axis_kind[a];
        A.bc_lo = d.bc_lo[a];
        A.bc_hi = d.bc_hi[a];
        std::vector<Term> adv;
        if (is_spatial(A.kind)) {
          if (terms & SAP_TERM_ADV) {
            adv.push_back(Term{MAT_I, MAT_I, SF_U + a, MF_ONE, 0, 1.0});
            adv.push_back(Term{A_id(a), A_id(a), SF_ONE, MF_V, 0, 1.0});
          }
        } else if (terms & SAP_TERM_MOM) {
          for (int b = 0; b < 3; ++b)
            if (nonzero[SF_DU + b]) adv.push_back(Term{A_id(b), A_id(b), SF_DU + b, lnp ? MF_GM_OVER_P : MF_GM, 0, -1.0});
          for (int b = 0; b < 3; ++b)
            for (int e = 0; e < 3; ++e)
              if (nonzero[SF_G + 3 * b + e]) adv.push_back(Term{AA_id(b, e), AA_id(b, e), SF_G + 3 * b + e, lnp ? MF_ONE : MF_P, 0, -1.0});
        }
        if ((int)adv.size() > MAXADV) throw std::string("too many advection terms");
        A.nadv = (int)adv.size();
        for (int t = 0; t < A.nadv; ++t) A.adv[t] = adv[t];
        A.active = A.nadv > 0;
      }
      // eigen-pairs of A^x once, rotated for y and z (Sec. 3.2)
      Mat Wx;
      std::vector<double> lam;
      sym_eig_blocks(Tb.A[0], c->Ablocks, Wx, lam);
      for (int a = 0; a < c->D; ++a) {
        ax[a].llf = c->flux == SAP_FLUX_LLF;
        ax[a].lam_lo = *std::min_element(lam.begin(), lam.end());
        ax[a].lam_hi = *std::max_element(lam.begin(), lam.end());
      }
      Mat Wa[3];
      Wa[0] = Wx;
      Wa[1] = matmul(transpose(Tb.Uz), Wx);
      Wa[2] = matmul(transpose(Tb.Ux), Wa[1]);
      for (int a = 0; a < 3; ++a)
        for (auto& v : Wa[a].a)
          if (std::fabs(v) < 1e-14) v = 0.0;
      // face |beta| data
      std::vector<double> uface_vals[3];
      bool uface_uni[3] = {true, true, true};
      double uface_u[3] = {0, 0, 0};
      for (int a = 0; a < c->dx; ++a) {
        if (Uface && Uface[a]) uface_vals[a].assign(Uface[a], Uface[a] + c->nsf[a]);
        else uface_vals[a].assign(c->nsf[a], 0.0);
        uface_u[a] = uface_vals[a].empty() ? 0.0 : uface_vals[a][0];
        for (double v : uface_vals[a])
          if (v != uface_u[a]) uface_uni[a] = false;
      }
      std::vector<int> pslot(nsv, -1);
      std::vector<double> pabs;
      int npface = c->npc + 1;
      for (int a = 0; a < c->D; ++a) {
        AxisInfo& A = ax[a];
        if (!A.active) continue;
        if (is_spatial(A.kind)) {
          if (uface_uni[a] && !has_mom) {  // constant beta: |beta| = W |U + lam V| W^T as one matrix
            A.route = ABS_CONST;
            // entries below 1e-14 of the largest |eigenvalue| are rounding residue of the
            // back-transformation (they vanish by symmetry); the cut is relative, so a small U or V
            // keeps every real entry
            double bmax = 0.0;
            for (int k = 0; k < n; ++k) bmax = std::max(bmax, std::fabs(uface_u[a] + lam[k] * d.V));
            Mat Ab(n);
            if (c->flux == SAP_FLUX_LLF) {  // alpha I with alpha = the largest |eigenvalue|
              for (int i = 0; i < n; ++i) Ab(i, i) = bmax;
            } else {
              for (int i = 0; i < n; ++i)
                for (int j = 0; j < n; ++j) {
                  double s = 0.0;
                  for (int k = 0; k < n; ++k) s += Wa[a](i, k) * std::fabs(uface_u[a] + lam[k] * d.V) * Wa[a](j, k);
                  Ab(i, j) = std::fabs(s) <= 1e-14 * bmax ? 0.0 : s;
                }
            }
            A.absmat = B.add("abs" + std::to_string(a), Ab);
            // eigenvectors also here: the adjoint differentiates |beta| with respect to U_a
            A.Wmat = B.add("W" + std::to_string(a), Wa[a]);
            A.WTmat = B.add("WT" + std::to_string(a), transpose(Wa[a]));
          } else {
            A.route = ABS_EIGEN;
            A.Wmat = B.add("W" + std::to_string(a), Wa[a]);
            A.WTmat = B.add("WT" + std::to_string(a), transpose(Wa[a]));
          }
        } else {
          // momentum faces: eigen-decomposition of beta^p at every (spatial node, p face) point
          A.route = ABS_POINT;
          Mat pat(n);
          for (int t = 0; t < A.nadv; ++t) {
            const HostCSR& h = B.mats[A.adv[t].mat];
            for (int i = 0; i < n; ++i)
              for (int k = h.rp[i]; k < h.rp[i + 1]; ++k) pat(i, h.col[k]) = 1.0;
          }
          MomFaceSrc& M = fs.mom;
          M = MomFaceSrc{};
          M.axis = a;
          M.blocks = connected_blocks(pat);
          Mat full(n);  // block pattern: dense within each block
          for (auto& b : M.blocks)
            for (int i : b)
              for (int j : b) full(i, j) = 1.0;
          M.pat = to_csr(full);
          A.absmat = B.add_csr("pabs_pattern", M.pat);
          // each term's entries scattered into the block pattern once
          M.tpos.assign(A.nadv, {});
          for (int t = 0; t < A.nadv; ++t) {
            const HostCSR& h = B.mats[A.adv[t].mat];
            for (int i = 0; i < n; ++i)
              for (int k = h.rp[i]; k < h.rp[i + 1]; ++k) {
                const int j = h.col[k];
                int pos = -1;
                for (int e = M.pat.rp[i]; e < M.pat.rp[i + 1]; ++e)
                  if (M.pat.col[e] == j) pos = e;
                M.tpos[t].push_back({pos, h.val[k]});
              }
          }
          M.nadv = A.nadv;
          for (int t = 0; t < A.nadv; ++t) M.adv[t] = A.adv[t];
          M.sf = sf;
          M.V = d.V;
          M.has_mom = has_mom;
          // points where |beta^p| stays below 1e-15 of its largest value carry no upwinding term
          // beyond FP64 rounding of the largest momentum flux; they are skipped
          std::vector<double> pmax(nsv, 0.0);
          parallel_for(nsv, [&](int sp, std::vector<double>& pv) {
            for (int f = 0; f < npface; ++f) {
              M.beta_at(sp, c->pface[f], nsv, pv);
              for (double v : pv) pmax[sp] = std::max(pmax[sp], std::fabs(v));
            }
          });
          double gmax = 0.0;
          for (double v : pmax) gmax = std::max(gmax, v);
          int nslot = 0;
          for (int sp = 0; sp < nsv; ++sp)
            if (gmax > 0.0 && pmax[sp] > 1e-15 * gmax) pslot[sp] = nslot++;
          M.pslot = pslot;
          {  // the row kernel skips the |beta^p| loop in cells without a tabulated point
            int with = 0;
            for (int sc = 0; sc < c->nscell; ++sc) {
              bool any = false;
              for (int j = 0; j < c->qdx; ++j) any = any || pslot[(size_t)sc * c->qdx + j] >= 0;
              with += any ? 1 : 0;
            }
            c->pslot_cell_frac = c->nscell ? double(with) / c->nscell : 1.0;
          }
          M.nslot = nslot;
          const int nnzp = (int)M.pat.col.size();
          const bool llf = c->flux == SAP_FLUX_LLF;
          pabs.assign((size_t)nslot * npface * nnzp, 0.0);
          parallel_for(nsv, [&](int sp, std::vector<double>& pv) {
            if (pslot[sp] < 0) return;
            Mat bm(n), Wb;
            std::vector<double> lb;
            for (int f = 0; f < npface; ++f) {
              M.beta_at(sp, c->pface[f], nsv, pv);
              for (int i = 0; i < n; ++i)
                for (int e = M.pat.rp[i]; e < M.pat.rp[i + 1]; ++e) bm(i, M.pat.col[e]) = pv[e];
              sym_eig_blocks(bm, M.blocks, Wb, lb);
              double* dst = &pabs[((size_t)pslot[sp] * npface + f) * nnzp];
              if (llf) {  // alpha I on the pattern, alpha = the largest |eigenvalue| at the point
                double alpha = 0.0;
                for (int e = 0; e < n; ++e) alpha = std::max(alpha, std::fabs(lb[e]));
                for (int i = 0; i < n; ++i)
                  for (int k = M.pat.rp[i]; k < M.pat.rp[i + 1]; ++k) dst[k] = M.pat.col[k] == i ? alpha : 0.0;
                continue;
              }
              for (int i = 0; i < n; ++i)
                for (int k = M.pat.rp[i]; k < M.pat.rp[i + 1]; ++k) {
                  const int j = M.pat.col[k];
                  double s2 = 0.0;
                  for (int e = 0; e < n; ++e) s2 += Wb(i, e) * std::fabs(lb[e]) * Wb(j, e);
                  dst[k] = s2;
                }
            }
          });
        }
      }
      // upload: bank, fields, term lists
      std::vector<double> sf_nonuni;  // [SF_NCOMP][nsv], only used for non-uniform components
      sf_nonuni = sf;
      std::vector<double> nu_v, s_v;
      bool nu_uni = true, s_uni = true;
      double nu_u = nu ? nu[0] : 0.0, s_u = s000 ? s000[0] : 0.0;
      if (nu)
        for (int p = 0; p < c->npv; ++p)
          if (nu[p] != nu_u) { nu_uni = false; break; }
      if (s000)
        for (int p = 0; p < c->npv; ++p)
          if (s000[p] != s_u) { s_uni = false; break; }
      if (!(terms & SAP_TERM_SRC)) { s_uni = true; s_u = 0.0; }
      if (!nu_uni) nu_v.assign(nu, nu + c->npv);
      if (!s_uni) s_v.assign(s000, s000 + c->npv);
      auto fill = [&](auto& P, auto tag) {
        using T = decltype(tag);
        set_bank<T>(P, B, c, fs.bufs);
        P.nreact = (int)react.size();
        for (int t = 0; t < P.nreact; ++t) P.react[t] = react[t];
        for (int a = 0; a < MAXD; ++a) P.ax[a] = ax[a];
        bool any_nonuni = false;
        for (int k = 0; k < SF_NCOMP; ++k) {
          P.sf_is_uni[k] = uni[k];
          P.sf_uni[k] = T(uval[k]);
          if (!uni[k]) any_nonuni = true;
        }
        if (any_nonuni) {
          if (sizeof(T) == 8) P.sfield = (const T*)upload(c, sf_nonuni, fs.bufs);
          else P.sfield = (const T*)upload(c, to_f32(sf_nonuni), fs.bufs);
        } else {
          P.sfield = nullptr;
        }
        for (int a = 0; a < MAXD; ++a) {
          P.uface_is_uni[a] = a < c->dx ? uface_uni[a] : 1;
          P.uface_uni[a] = T(a < c->dx ? uface_u[a] : 0.0);
          P.uface[a] = nullptr;
          if (a < c->dx && !uface_uni[a]) {
            if (sizeof(T) == 8) P.uface[a] = (const T*)upload(c, uface_vals[a], fs.bufs);
            else P.uface[a] = (const T*)upload(c, to_f32(uface_vals[a]), fs.bufs);
          }
        }
        P.nu_uni = T(nu_u);
        P.nu = nullptr;
        if (!nu_uni) P.nu = (sizeof(T) == 8) ? (const T*)upload(c, nu_v, fs.bufs) : (const T*)upload(c, to_f32(nu_v), fs.bufs);
        P.s_uni = T(s_u);
        P.s000 = nullptr;
        if (!s_uni) P.s000 = (sizeof(T) == 8) ? (const T*)upload(c, s_v, fs.bufs) : (const T*)upload(c, to_f32(s_v), fs.bufs);
        P.pslot = (const int*)upload(c, pslot, fs.bufs);
        if (!pabs.empty())
          P.pabs = (sizeof(T) == 8) ? (const T*)upload(c, pabs, fs.bufs) : (const T*)upload(c, to_f32(pabs), fs.bufs);
        else
          P.pabs = nullptr;
        P.lam = (sizeof(T) == 8) ? (const T*)upload(c, lam, fs.bufs) : (const T*)upload(c, to_f32(lam), fs.bufs);
        // the momentum-face |beta| values again in the ELL order of their pattern matrix
        P.pabs_ell = nullptr;
        for (int a = 0; a < c->D; ++a) {
          const AxisInfo& A = ax[a];
          if (!A.active || A.route != ABS_POINT || pabs.empty()) continue;
          const HostCSR& pc = B.mats[A.absmat];
          const int w = P.bank.ell_w[A.absmat];
          const int nnzp = (int)pc.col.size();
          const size_t npts = pabs.size() / nnzp;  // slots x momentum faces
          std::vector<double> pe(npts * w * n, 0.0);
          for (size_t sp = 0; sp < npts; ++sp)
            for (int i = 0; i < n; ++i)
              for (int k = 0; pc.rp[i] + k < pc.rp[i + 1]; ++k) pe[(sp * w + k) * n + i] = pabs[sp * nnzp + pc.rp[i] + k];
          P.pabs_ell = (sizeof(T) == 8) ? (const T*)upload(c, pe, fs.bufs) : (const T*)upload(c, to_f32(pe), fs.bufs);
        }
        // terms whose coefficient is one number for the whole problem
        auto term_uni = [&](const Term& tm) {
          return (tm.sf == SF_ONE || uni[tm.sf]) && (tm.mf == MF_ONE || !has_mom) && (!tm.nu || nu_uni);
        };
        P.react_uni = 0u;
        for (int t = 0; t < P.nreact; ++t)
          if (term_uni(P.react[t])) P.react_uni |= 1u << t;
        for (int a = 0; a < MAXD; ++a) {
          P.adv_uni[a] = 0u;
          for (int t = 0; t < P.ax[a].nadv; ++t)
            if (term_uni(P.ax[a].adv[t])) P.adv_uni[a] |= 1u << t;
        }
        // terms whose coefficient is zero everywhere (the spatial advection U_a I with U_a = 0)
        auto term_zero = [&](const Term& tm) {
          return (tm.sf != SF_ONE && uni[tm.sf] && uval[tm.sf] == 0.0) || (tm.nu && nu_uni && nu_u == 0.0);
        };
        P.react_zero = 0u;
        for (int t = 0; t < P.nreact; ++t)
          if (term_zero(P.react[t])) P.react_zero |= 1u << t;
        for (int a = 0; a < MAXD; ++a) {
          P.adv_zero[a] = 0u;
          for (int t = 0; t < P.ax[a].nadv; ++t) {
            const Term& tm = P.ax[a].adv[t];
            // a spatial face coefficient of U_a uses the face values, so both must vanish
            const bool face_ok = !(tm.sf == SF_U + a && a < c->dx) || (uface_uni[a] && uface_u[a] == 0.0);
            if (term_zero(tm) && face_ok) P.adv_zero[a] |= 1u << t;
          }
        }
      };
      fill(c->p64, double{});
      fill(c->p32, float{});
      // the uniform-coefficient kernel: a spatial 3-D problem with k = 2 whose every term coefficient
      // is one number and whose faces use the constant upwind matrix
      c->uni_avail = -1;
      c->uni_v64.clear();
      c->uni_v32.clear();
      if (c->D == 3 && c->dx == 3 && !has_mom && c->q == 3 && uni_supported(c->T.lmax)) {
        const double p0 = c->pnode.empty() ? 1.0 : c->pnode[0];
        auto coef = [&](const Term& tm) {
          return tm.scale * (tm.sf == SF_ONE ? 1.0 : uval[tm.sf]) * mom_factor_h(tm.mf, p0, false, d.V) *
                 (tm.nu ? nu_u : 1.0);
        };
        auto add_dense = [&](std::vector<double>& m, int mat, double cv) {
          if (mat == MAT_I) {
            for (int i = 0; i < n; ++i) m[(size_t)i * n + i] += cv;
            return;
          }
          const HostCSR& h = B.mats[mat];
          for (int i = 0; i < n; ++i)
            for (int k = h.rp[i]; k < h.rp[i + 1]; ++k) m[(size_t)i * n + h.col[k]] += cv * h.val[k];
        };
        UniDense u;
        u.lmax = c->T.lmax;
        u.n = n;
        u.R.assign((size_t)n * n, 0.0);
        bool ok = nu_uni;
        const OpParams<double>& P = c->p64;
        for (int t = 0; t < P.nreact && ok; ++t) {
          if ((P.react_zero >> t) & 1u) continue;
          if (!((P.react_uni >> t) & 1u)) ok = false;
          else add_dense(u.R, P.react[t].mat, coef(P.react[t]));
        }
        for (int a = 0; a < 3 && ok; ++a) {
          u.B[a].assign((size_t)n * n, 0.0);
          u.A[a].assign((size_t)n * n, 0.0);
          const AxisInfo& A = P.ax[a];
          if (!A.active) continue;
          if (A.route != ABS_CONST || !uface_uni[a]) ok = false;
          for (int t = 0; t < A.nadv && ok; ++t) {
            const Term& tm = A.adv[t];
            if ((P.adv_zero[a] >> t) & 1u) continue;
            if (!((P.adv_uni[a] >> t) & 1u)) { ok = false; break; }
            // the face coefficient of U_a is the face value: it must equal the node value
            if (tm.sf == SF_U + a && uface_u[a] != uval[tm.sf]) { ok = false; break; }
            add_dense(u.B[a], tm.mat, coef(tm));
          }
          if (ok) add_dense(u.A[a], A.absmat, 1.0);
        }
        std::vector<double> vals;
        if (ok && uni_pack(u, vals)) {
          c->uni_v64 = vals;
          c->uni_v32 = to_f32(vals);
          c->uni_avail = u.lmax;
        }
      }
      apply_kernel_choice(c);
      // the row kernel's per-cell coefficient tables (not for problems the node kernel runs: their
      // transposed applies compute the coefficients in the kernel)
      if (c->uni_avail < 0) {
        // the Jacobi diagonal per DoF: FP64 always (the Krylov matvecs of FP64 contexts, the
        // Jacobi-scaled FP32 copy of the FP64 residual in FP32 contexts), FP32 for FP32 contexts
        cudaError_t te = build_coef_tables<double>(c->p64, fs.bufs, true);
        if (te == cudaSuccess) te = build_coef_tables<float>(c->p32, fs.bufs, c->prec == SAP_PREC_FP32);
        if (te == cudaSuccess) te = cudaDeviceSynchronize();
        if (te != cudaSuccess) throw std::string("coefficient tables: ") + cudaGetErrorString(te);
      }
      c->fields_set = true;
      c->fields_version += 1;
      c->cn_prev_valid = false;
    } catch (const std::string& e) {
      c->err = "sap_set_fields: " + e;
      return SAP_ENOMEM;
    }
    return SAP_OK;
  });
}

extern "C" sap_status sap_set_flux(sap_handle c, int flux) {
  if (!c || (flux != SAP_FLUX_UPWIND && flux != SAP_FLUX_LLF)) return SAP_EINVAL;
  if (!c->sub.empty()) {
    c->err = "sap_set_flux: set the flux of a batch through its instance handles";
    return SAP_EINVAL;
  }
  if (flux != c->flux) {
    c->flux = flux;
    c->fields_set = false;  // the face tables depend on the flux: the fields must be set again
  }
  return SAP_OK;
}

extern "C" sap_status sap_set_apply_kernel(sap_handle c, int kernel, int cells_per_block) {
  if (!c || (kernel != SAP_KERNEL_AUTO && kernel != SAP_KERNEL_ROWS) || cells_per_block < 0) return SAP_EINVAL;
  if (!c->sub.empty()) {
    c->err = "sap_set_apply_kernel: a batch runs the row kernel";
    return SAP_EINVAL;
  }
  c->apply_kernel = kernel;
  c->uni_cells = cells_per_block;
  apply_kernel_choice(c);
  c->fields_version += 1;  // graphs captured with the previous kernel are captured again
  return SAP_OK;
}

extern "C" sap_status sap_apply_kernel_in_use(sap_handle c, int* uniform) {
  if (!c || !uniform) return SAP_EINVAL;
  if (!c->fields_set) {
    c->err = "sap_apply_kernel_in_use: fields not set";
    return SAP_EINVAL;
  }
  *uniform = c->p64.uni_L >= 0 ? 1 : 0;
  return SAP_OK;
}

extern "C" sap_status sap_set_fields_device(sap_handle c, const double* U, const double* gradU, const double* DUDt,
                                            const double* Bw, const double* const Uface[3], const double* nu,
                                            const double* s000, sap_stream stream) {
  return guarded(c, "sap_set_fields_device", [&]() -> sap_status {
    if (!c) return SAP_EINVAL;
    if (!c->sub.empty()) {
      c->err = "sap_set_fields_device: set the fields of a batch through its instance handles";
      return SAP_EINVAL;
    }
    const cudaStream_t s = (cudaStream_t)stream;
    // the term tables and the momentum-face eigen data are built on the host: read the fields back
    // on the caller's stream (ordered after whatever produced them), then build as sap_set_fields
    std::vector<double> hU, hG, hDU, hB, hF[3], hnu, hs;
    cudaError_t err = cudaSuccess;
    auto fetch = [&](const double* d, size_t count, std::vector<double>& h) -> const double* {
      if (!d) return nullptr;
      h.resize(std::max<size_t>(count, 1));
      if (count && err == cudaSuccess) err = cudaMemcpyAsync(h.data(), d, sizeof(double) * count, cudaMemcpyDeviceToHost, s);
      return h.data();
    };
    const size_t nsv = (size_t)c->nsv, npv = (size_t)c->npv;
    const double* pU = fetch(U, nsv * 3, hU);
    const double* pG = fetch(gradU, nsv * 9, hG);
    const double* pDU = fetch(DUDt, nsv * 3, hDU);
    const double* pB = fetch(Bw, nsv * 3, hB);
    const double* pF[3] = {nullptr, nullptr, nullptr};
    for (int a = 0; a < 3; ++a)
      if (Uface && a < c->dx) pF[a] = fetch(Uface[a], (size_t)c->nsf[a], hF[a]);
    const double* pnu = fetch(nu, npv, hnu);
    const double* ps = fetch(s000, npv, hs);
    if (err == cudaSuccess) err = cudaStreamSynchronize(s);
    if (err != cudaSuccess) {
      c->err = std::string("sap_set_fields_device: copy of the fields: ") + cudaGetErrorString(err);
      return SAP_ECUDA;
    }
    return sap_set_fields(c, pU, pG, pDU, pB, pF, pnu, ps);
  });
}

// ------------------------------------------------------------------------------------------------
// compute entry points
// ------------------------------------------------------------------------------------------------
extern "C" sap_status sap_num_dofs(sap_handle c, int64_t* n) {
  if (!c || !n) return SAP_EINVAL;
  *n = c->N;
  return SAP_OK;
}

static bool ensure_ws64(sap_ctx* c, int count) {
  if (c->ws64_count >= count) return true;
  c->cn_prev_valid = false;
  if (c->ws64) cudaFree(c->ws64);
  c->ws64 = nullptr;
  c->ws64_count = 0;
  if (cudaMalloc(&c->ws64, sizeof(double) * (size_t)count * c->N) != cudaSuccess) return false;
  c->ws64_count = count;
  return true;
}

static bool ensure_ws32(sap_ctx* c, int count) {
  if (c->ws32_count >= count) return true;
  if (c->ws32) cudaFree(c->ws32);
  c->ws32 = nullptr;
  c->ws32_count = 0;
  if (cudaMalloc(&c->ws32, sizeof(float) * (size_t)count * c->N) != cudaSuccess) return false;
  c->ws32_count = count;
  return true;
}

extern "C" sap_status sap_apply_operator(sap_handle c, const void* x, void* y, int mode, sap_stream stream) {
  return guarded(c, "sap_apply_operator", [&]() -> sap_status {
    if (!c || !x || !y || x == y) return SAP_EINVAL;
    if (!c->sub.empty()) {
      if (mode != SAP_APPLY_D && mode != SAP_APPLY_RHS) return SAP_EUNSUPPORTED;
      return batch_apply(c, x, y, mode, (cudaStream_t)stream);
    }
    if (!c->fields_set) {
      c->err = "fields not set";
      return SAP_EINVAL;
    }
    if (mode != SAP_APPLY_D && mode != SAP_APPLY_RHS && mode != SAP_APPLY_T) {
      c->err = "unsupported apply mode";
      return SAP_EUNSUPPORTED;
    }
    cudaError_t e = c->prec == SAP_PREC_FP64
                        ? launch_apply64(c->p64, (const double*)x, (double*)y, mode, (cudaStream_t)stream)
                        : launch_apply32(c->p32, (const float*)x, (float*)y, mode, (cudaStream_t)stream);
    if (e != cudaSuccess) {
      c->err = std::string("apply: ") + cudaGetErrorString(e);
      return SAP_ECUDA;
    }
    return SAP_OK;
  });
}

extern "C" sap_status sap_step_erk(sap_handle c, double* state, double dt, int nsteps, sap_stream stream) {
  return guarded(c, "sap_step_erk", [&]() -> sap_status {
    if (!c || !state || nsteps < 0) return SAP_EINVAL;
    c->cn_prev_valid = false;  // the RK4 stage buffers share the workspace
    if (!c->sub.empty()) {
      if (c->prec == SAP_PREC_FP64 ? !ensure_ws64(c, 3) : (!ensure_ws32(c, 2) || !ensure_ws64(c, 1))) {
        c->err = "erk: workspace allocation failed";
        return SAP_ENOMEM;
      }
      return batch_erk(c, state, dt, nsteps, (cudaStream_t)stream);
    }
    if (!c->fields_set) {
      c->err = "fields not set";
      return SAP_EINVAL;
    }
    if (c->prec == SAP_PREC_FP64 ? !ensure_ws64(c, 3) : (!ensure_ws32(c, 2) || !ensure_ws64(c, 1))) {
      c->err = "erk: workspace allocation failed";
      return SAP_ENOMEM;
    }
    return erk_steps(c, state, dt, nsteps, (cudaStream_t)stream);
  });
}

extern "C" sap_status sap_step_erk_noalloc(sap_handle c, double* state, double dt, int nsteps, sap_stream stream) {
  return guarded(c, "sap_step_erk_noalloc", [&]() -> sap_status {
    if (!c || !state || nsteps < 0) return SAP_EINVAL;
    if (!c->sub.empty()) {
      c->err = "sap_step_erk_noalloc: batch handles are not supported (use sap_step_erk)";
      return SAP_EUNSUPPORTED;
    }
    // as in sap_step_erk: a following CN step starts from the plain previous state
    c->cn_prev_valid = false;
    if (!c->fields_set) {
      c->err = "fields not set";
      return SAP_EINVAL;
    }
    return erk_steps_noalloc(c, state, dt, nsteps, (cudaStream_t)stream);
  });
}

static sap_status step_theta(sap_handle c, double* state, double dt, double theta, int nsteps, double tol, int restart,
                             int maxit, sap_solver_stats* stats, sap_stream stream) {
  if (!c || !state || nsteps < 0 || restart < 1 || restart > 31 || maxit < 1 || !(tol > 0) || !(theta >= 0.0) ||
      !(theta <= 1.0) || !std::isfinite(dt))
    return SAP_EINVAL;
  if (!c->sub.empty()) {
    if (theta != 0.5) {
      c->err = "batch: Crank--Nicolson (theta = 1/2) only";
      return SAP_EUNSUPPORTED;
    }
    // FP64: b, r, the Krylov basis and the initial-guess history; FP32: FP32 basis, FP64 b, r, history
    const int need64 = c->prec == SAP_PREC_FP64 ? restart + 4 : 3;
    if (c->ws64_count < need64) c->cn_prev_valid = false;  // the history lives in the workspace
    const bool ok = c->prec == SAP_PREC_FP64 ? ensure_ws64(c, need64) : (ensure_ws32(c, restart + 1) && ensure_ws64(c, need64));
    if (!ok) {
      c->err = "cn: workspace allocation failed";
      return SAP_ENOMEM;
    }
    return batch_cn(c, state, dt, nsteps, tol, restart, maxit, stats, (cudaStream_t)stream);
  }
  if (!c->fields_set) {
    c->err = "fields not set";
    return SAP_EINVAL;
  }
  if (c->prec == SAP_PREC_FP32) {
    if (c->ws64_count < 3) c->cn_prev_valid = false;
    if (!ensure_ws32(c, restart + 1) || !ensure_ws64(c, 3)) {
      c->err = "cn: workspace allocation failed";
      return SAP_ENOMEM;
    }
    return cn_steps(c, state, dt, theta, nsteps, tol, restart, maxit, stats, (cudaStream_t)stream);
  }
  if (c->ws64_count < restart + 4) c->cn_prev_valid = false;  // the history lives in the workspace
  if (!ensure_ws64(c, restart + 4)) {
    c->err = "cn: workspace allocation failed";
    return SAP_ENOMEM;
  }
  return cn_steps(c, state, dt, theta, nsteps, tol, restart, maxit, stats, (cudaStream_t)stream);
}

extern "C" sap_status sap_step_cn(sap_handle c, double* state, double dt, int nsteps, double tol, int restart,
                                  int maxit, sap_solver_stats* stats, sap_stream stream) {
  return guarded(c, "sap_step_cn", [&]() -> sap_status {
    return step_theta(c, state, dt, 0.5, nsteps, tol, restart, maxit, stats, stream);
  });
}

extern "C" sap_status sap_step_theta(sap_handle c, double* state, double dt, double theta, int nsteps, double tol,
                                     int restart, int maxit, sap_solver_stats* stats, sap_stream stream) {
  return guarded(c, "sap_step_theta", [&]() -> sap_status {
    return step_theta(c, state, dt, theta, nsteps, tol, restart, maxit, stats, stream);
  });
}

extern "C" sap_status sap_apply_cost(sap_handle c, double* flops, double* bytes) {
  return guarded(c, "sap_apply_cost", [&]() -> sap_status {
    if (!c || !flops || !bytes) return SAP_EINVAL;
    if (!c->sub.empty()) {
      double f = 0, b = 0;
      for (auto* s2 : c->sub) {
        double f1, b1;
        sap_status st = sap_apply_cost(s2, &f1, &b1);
        if (st != SAP_OK) return st;
        f += f1;
        b += b1;
      }
      *flops = f;
      *bytes = b;
      return SAP_OK;
    }
    if (!c->fields_set) return SAP_EINVAL;
    const OpParams<double>& P = c->p64;
    *bytes = 2.0 * (double)c->N * (c->prec == SAP_PREC_FP64 ? 8.0 : 4.0);
    if (P.uni_L >= 0) {  // the node kernel: its own count
      const int active[3] = {P.ax[0].active, P.ax[1].active, P.ax[2].active};
      *flops = uni_flops_per_cell(P.uni_L, active) * c->ncell;
      return SAP_OK;
    }
    const int n = c->n, nloc = c->nloc, nfp = c->nfp, q = c->q, D = c->D;
    auto nnz_row_avg = [&](int mat) -> double {
      if (mat == MAT_I) return 1.0;
      const std::vector<int>* rp = nullptr;
      (void)rp;
      return c->bank_nnz[mat] / double(n);
    };
    double per_cell = 0.0;
    int nvt = P.nreact;
    for (int a = 0; a < D; ++a) nvt += P.ax[a].nadv;
    per_cell += 4.0 * nvt * nloc;                       // coefficient tables
    const double faces = 2.0 * D * n * nfp;            // face entries per cell
    per_cell += 2.0 * faces * 2.0 * q;                  // own + neighbour traces
    per_cell += 2.0 * faces;                            // sum / difference
    // share of the cells in which a term is applied: none for a term that is zero everywhere; in FP32,
    // not in cells where its spatial field component is zero at every node
    auto share = [&](const Term& tm, bool zero) -> double {
      if (zero) return 0.0;
      if (c->prec == SAP_PREC_FP32 && tm.sf != SF_ONE) return 1.0 - c->sf_zero_frac32[tm.sf];
      return 1.0;
    };
    for (int a = 0; a < D; ++a) {
      const AxisInfo& A = P.ax[a];
      if (!A.active) continue;
      const double fe = 2.0 * n * nfp;  // this axis' face entries per cell
      double f = 1.0;
      for (int t = 0; t < A.nadv; ++t)
        f += share(A.adv[t], (P.adv_zero[a] >> t) & 1u) * (2.0 * nnz_row_avg(A.adv[t].mat) + 2.0);
      if (A.route == ABS_EIGEN) f += 2.0 * nnz_row_avg(A.WTmat) + 3.0 + 2.0 * nnz_row_avg(A.Wmat) + 2.0;
      else if (A.route == ABS_POINT) f += c->pslot_cell_frac * (2.0 * nnz_row_avg(A.absmat)) + 1.0;
      else f += 2.0 * nnz_row_avg(A.absmat) + 1.0;
      per_cell += fe * f;
      double v = 0.0;  // volume advection per DoF
      for (int t = 0; t < A.nadv; ++t)
        v += share(A.adv[t], (P.adv_zero[a] >> t) & 1u) * (2.0 * nnz_row_avg(A.adv[t].mat) + 2.0);
      v += 2.0 * q + 6.0;  // derivative and lifts
      per_cell += v * n * nloc;
    }
    double rx = 0.0;
    for (int t = 0; t < P.nreact; ++t)
      rx += share(P.react[t], (P.react_zero >> t) & 1u) * (2.0 * nnz_row_avg(P.react[t].mat) + 2.0);
    per_cell += (rx + 4.0) * n * nloc;
    *flops = per_cell * c->ncell;
    return SAP_OK;
  });
}

extern "C" sap_status sap_adjoint_step_cn(sap_handle c, const double* zeta_prev, const double* zeta_next,
                                          double* lambda, double dt, double tol, int restart, int maxit,
                                          double* mu_out, double* grad_nu, sap_solver_stats* stats,
                                          sap_stream stream) {
  return guarded(c, "sap_adjoint_step_cn", [&]() -> sap_status {
    if (!c || !zeta_prev || !zeta_next || !lambda || restart < 1 || restart > 31 || maxit < 1 || !(tol > 0))
      return SAP_EINVAL;
    if (!c->sub.empty() || c->prec != SAP_PREC_FP64) {
      c->err = "adjoint: FP64 single-problem contexts only";
      return SAP_EUNSUPPORTED;
    }
    if (!c->fields_set) {
      c->err = "fields not set";
      return SAP_EINVAL;
    }
    if (!ensure_ws64(c, restart + 4)) {
      c->err = "adjoint: workspace allocation failed";
      return SAP_ENOMEM;
    }
    c->cn_prev_valid = false;  // the adjoint solve shares the workspace
    return adjoint_cn_step(c, zeta_prev, zeta_next, lambda, dt, tol, restart, maxit, mu_out, grad_nu, stats,
                           (cudaStream_t)stream);
  });
}

extern "C" sap_status sap_adjoint_step_erk(sap_handle c, const double* zeta_prev, double* lambda, double dt,
                                           double* grad_nu, double* stages_out, sap_solver_stats* stats,
                                           sap_stream stream) {
  return guarded(c, "sap_adjoint_step_erk", [&]() -> sap_status {
    if (!c || !zeta_prev || !lambda || !std::isfinite(dt)) return SAP_EINVAL;
    if (!c->sub.empty() || c->prec != SAP_PREC_FP64) {
      c->err = "adjoint: FP64 single-problem contexts only";
      return SAP_EUNSUPPORTED;
    }
    if (!c->fields_set) {
      c->err = "fields not set";
      return SAP_EINVAL;
    }
    if (!ensure_ws64(c, 8)) {
      c->err = "adjoint: workspace allocation failed";
      return SAP_ENOMEM;
    }
    c->cn_prev_valid = false;  // the adjoint step shares the workspace
    return adjoint_erk_step(c, zeta_prev, lambda, dt, grad_nu, stages_out, stats, (cudaStream_t)stream);
  });
}

// Gradient tables for the current fields (see GradTables): the compact list of spatial field
// components, and for the momentum axis the Daleckii--Krein derivatives of |beta^p| along each
// advection term, P_t = W (Gamma o (W^T K_t W)) W^T per block of the pattern, at every kept
// (spatial node, momentum face) point.
static double dk_gamma(double x, double y) {
  if (x > 0.0 && y > 0.0) return 1.0;
  if (x < 0.0 && y < 0.0) return -1.0;
  if (x == y) return 0.0;  // both zero: zero subgradient
  return (std::fabs(x) - std::fabs(y)) / (x - y);
}

static void build_grad_tables(sap_ctx* c) {
  FieldStore& fs = g_fields[c];
  free_bufs(fs.gbufs);
  GradTables G;
  std::memset(&G, 0, sizeof(G));
  const OpParams<double>& P = c->p64;
  for (int k = 0; k < SF_NCOMP; ++k) G.sf_comp[k] = -1;
  auto use = [&](const Term& t) {
    if (t.sf != SF_ONE && G.sf_comp[t.sf] < 0) {
      G.sf_comp[t.sf] = G.ncomp;
      G.comp_sf[G.ncomp++] = t.sf;
    }
  };
  for (int t = 0; t < P.nreact; ++t) use(P.react[t]);
  for (int a = 0; a < c->D; ++a)
    for (int t = 0; t < P.ax[a].nadv; ++t) use(P.ax[a].adv[t]);
  G.qsp = 1;
  for (int a = 1; a < c->dx; ++a) G.qsp *= c->q;
  G.face_off = G.ncomp * c->qdx;
  G.ps = G.face_off + 2 * c->dx * G.qsp;
  const MomFaceSrc& M = fs.mom;
  if (M.axis >= 0 && M.nslot > 0) {
    const AxisInfo& A = P.ax[M.axis];
    const int n = c->n, nsv = c->nsv, npface = c->npc + 1;
    const int w = P.bank.ell_w[A.absmat];
    const int nnzp = (int)M.pat.col.size();
    std::vector<int> loc(n, 0);
    for (const auto& b : M.blocks)
      for (int i = 0; i < (int)b.size(); ++i) loc[b[i]] = i;
    G.pd_w = w;
    for (int t = 0; t < A.nadv; ++t) {
      if (A.adv[t].sf == SF_ONE) continue;
      std::vector<double> Kp(nnzp, 0.0);  // K_t on the pattern
      for (const auto& pr : M.tpos[t]) Kp[pr.first] += pr.second;
      std::vector<double> pe((size_t)M.nslot * npface * w * n, 0.0);
      parallel_for(nsv, [&](int sp, std::vector<double>& pv) {
        const int slot = M.pslot[sp];
        if (slot < 0) return;
        Mat bm(n), W;
        std::vector<double> lb, Kb, X, T2;
        for (int f = 0; f < npface; ++f) {
          M.beta_at(sp, c->pface[f], nsv, pv);
          for (int i = 0; i < n; ++i)
            for (int e = M.pat.rp[i]; e < M.pat.rp[i + 1]; ++e) bm(i, M.pat.col[e]) = pv[e];
          sym_eig_blocks(bm, M.blocks, W, lb);
          double* dst = &pe[((size_t)slot * npface + f) * w * n];
          for (const auto& b : M.blocks) {
            const int m = (int)b.size();
            Kb.assign((size_t)m * m, 0.0);
            for (int i = 0; i < m; ++i)
              for (int e = M.pat.rp[b[i]]; e < M.pat.rp[b[i] + 1]; ++e) Kb[(size_t)i * m + loc[M.pat.col[e]]] = Kp[e];
            // X = W_b^T K_b W_b, then Gamma o X, then P_b = W_b X W_b^T
            T2.assign((size_t)m * m, 0.0);
            for (int i = 0; i < m; ++i)
              for (int k = 0; k < m; ++k) {
                double v = 0.0;
                for (int j = 0; j < m; ++j) v += Kb[(size_t)i * m + j] * W(b[j], b[k]);
                T2[(size_t)i * m + k] = v;  // (K_b W_b)[i][k]
              }
            X.assign((size_t)m * m, 0.0);
            for (int k = 0; k < m; ++k)
              for (int l = 0; l < m; ++l) {
                double v = 0.0;
                for (int i = 0; i < m; ++i) v += W(b[i], b[k]) * T2[(size_t)i * m + l];
                X[(size_t)k * m + l] = v * dk_gamma(lb[b[k]], lb[b[l]]);
              }
            for (int i = 0; i < m; ++i)
              for (int l = 0; l < m; ++l) {
                double v = 0.0;
                for (int k = 0; k < m; ++k) v += W(b[i], b[k]) * X[(size_t)k * m + l];
                T2[(size_t)i * m + l] = v;  // (W_b X)[i][l]
              }
            for (int i = 0; i < m; ++i) {
              const int r = b[i];
              for (int e = M.pat.rp[r]; e < M.pat.rp[r + 1]; ++e) {
                const int j = loc[M.pat.col[e]];
                double v = 0.0;
                for (int l = 0; l < m; ++l) v += T2[(size_t)i * m + l] * W(b[j], b[l]);
                dst[(size_t)(e - M.pat.rp[r]) * n + r] = v;  // ELL slot e - rp[r] of row r
              }
            }
          }
        }
      });
      G.pd[t] = (const double*)upload(c, pe, fs.gbufs);
    }
  }
  c->gt = G;
  c->gt_version = c->fields_version;
}

extern "C" sap_status sap_adjoint_step(sap_handle c, int scheme, const double* zeta_prev, const double* zeta_next,
                                       double* lambda, double dt, double tol, int restart, int maxit,
                                       const sap_field_grads* grads, sap_solver_stats* stats, sap_stream stream) {
  return guarded(c, "sap_adjoint_step", [&]() -> sap_status {
    if (!c || !zeta_prev || !lambda || !std::isfinite(dt) || (scheme != SAP_SCHEME_CN && scheme != SAP_SCHEME_ERK4))
      return SAP_EINVAL;
    if (scheme == SAP_SCHEME_CN && (!zeta_next || restart < 1 || restart > 31 || maxit < 1 || !(tol > 0)))
      return SAP_EINVAL;
    if (!c->sub.empty() || c->prec != SAP_PREC_FP64) {
      c->err = "adjoint: FP64 single-problem contexts only";
      return SAP_EUNSUPPORTED;
    }
    if (!c->fields_set) {
      c->err = "fields not set";
      return SAP_EINVAL;
    }
    if (c->flux != SAP_FLUX_UPWIND && grads &&
        (grads->U || grads->gradU || grads->DUDt || grads->Bw || grads->Uface[0] || grads->Uface[1] || grads->Uface[2])) {
      c->err = "adjoint: field gradients of the local Lax--Friedrichs flux are not formed";
      return SAP_EUNSUPPORTED;
    }
    const int need = scheme == SAP_SCHEME_CN ? restart + 4 : 8;
    if (!ensure_ws64(c, need)) {
      c->err = "adjoint: workspace allocation failed";
      return SAP_ENOMEM;
    }
    c->cn_prev_valid = false;  // the adjoint shares the workspace
    sap_field_grads g{};
    if (grads) g = *grads;
    const bool spatial = g.U || g.gradU || g.DUDt || g.Bw || g.Uface[0] || g.Uface[1] || g.Uface[2];
    if (spatial) {
      if (c->gt_version != c->fields_version) {
        try {
          build_grad_tables(c);
        } catch (const std::string& e) {
          c->err = "adjoint: gradient tables: " + e;
          return SAP_ENOMEM;
        }
      }
      if (coef_adjoint_smem_doubles(c->p64, c->gt) * sizeof(double) > 200 * 1024) {
        c->err = "adjoint: a cell is too large for the field-gradient kernel";
        return SAP_EUNSUPPORTED;
      }
      const size_t cnt = (size_t)c->ncell * c->gt.ps;
      if (c->gpart_count < cnt) {
        if (c->gpart) cudaFree(c->gpart);
  for (auto& g : c->bgraphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  if (c->bctl) cudaFree(c->bctl);
  if (c->bmask) cudaFree(c->bmask);
  if (c->bstat) cudaFree(c->bstat);
  if (c->bstat_host) cudaFreeHost(c->bstat_host);
        c->gpart = nullptr;
        c->gpart_count = 0;
        if (cudaMalloc(&c->gpart, sizeof(double) * std::max<size_t>(cnt, 1)) != cudaSuccess) {
          c->err = "adjoint: allocation of the gradient partials failed";
          return SAP_ENOMEM;
        }
        c->gpart_count = cnt;
      }
    }
    return adjoint_fields_step(c, scheme, zeta_prev, zeta_next, lambda, dt, tol, restart, maxit, g, stats,
                               (cudaStream_t)stream);
  });
}

extern "C" sap_status sap_destroy(sap_handle c) {
  if (!c) return SAP_OK;
  if (c->parent) return SAP_EINVAL;  // sub-handles belong to their batch
  for (auto* s2 : c->sub) {
    s2->parent = nullptr;
    sap_destroy(s2);
  }
  c->sub.clear();
  for (auto& b : c->batch_bufs) cudaFree(b.p);
  c->batch_bufs.clear();
  free_bufs(c->owned);
  auto it = g_fields.find(c);
  if (it != g_fields.end()) {
    free_bufs(it->second.bufs);
    free_bufs(it->second.gbufs);
    g_fields.erase(it);
  }
  if (c->gpart) cudaFree(c->gpart);
  if (c->ws64) cudaFree(c->ws64);
  if (c->ws32) cudaFree(c->ws32);
  if (c->small) cudaFree(c->small);
  if (c->gdev) cudaFree(c->gdev);
  if (c->gdev_host) cudaFreeHost(c->gdev_host);
  cn_graphs_release(c);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  delete c;
  return SAP_OK;
}

extern "C" const char* sap_last_error(sap_handle c) {
  if (!c) return g_create_error.c_str();
  return c->err.c_str();
}

extern "C" sap_status sap_coupling_matrix(int lmax, int which, int a, int b, double* out) {
  return guarded(nullptr, "sap_coupling_matrix", [&]() -> sap_status {
    if (lmax < 0 || lmax > 11 || !out || a < 0 || a > 2 || b < 0 || b > 2) return SAP_EINVAL;
    SHTables T = build_sh_tables(lmax);
    const Mat* m = nullptr;
    switch (which) {
      case 0: m = &T.A[a]; break;
      case 1: m = &T.Om[a]; break;
      case 2: m = &T.C; break;
      case 3: m = &T.AA[a][b]; break;
      case 4: m = &T.E[a]; break;
      case 5: m = &T.F[a][b]; break;
      default: return SAP_EINVAL;
    }
    std::memcpy(out, m->a.data(), sizeof(double) * m->a.size());
    return SAP_OK;
  });
}
