// Internal data structures shared by the host set-up (setup.cpp) and the CUDA kernels (operator.cu).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/sap.h"
#include "sh_tables.h"

namespace sap {

constexpr int MAXD = 3;
constexpr int MAXQ = 6;          // dG degree <= 5
constexpr int MAXTERMS = 28;     // reaction terms
constexpr int MAXADV = 12;       // advection terms per axis
constexpr int MAT_I = -1;        // identity "matrix"

// spatial field components stored per spatial volume point
enum : int { SF_ONE = -1, SF_U = 0, SF_G = 3, SF_DU = 12, SF_B = 15, SF_NCOMP = 18 };
// momentum factors, functions of the momentum p at a node or face
enum : int { MF_ONE = 0, MF_P, MF_GM, MF_V, MF_INV_V, MF_INV_GM, MF_INV_P, MF_INV_GMP, MF_GM_OVER_P, MF_COUNT };

struct Term {
  int mat;      // matrix id in the bank, or MAT_I
  int matT;     // id of the transposed matrix (for the transposed operator), or MAT_I
  int sf;       // spatial factor component or SF_ONE
  int mf;       // momentum factor
  int nu;       // 1: multiply by nu at the phase-space node
  double scale;
};

enum : int { ABS_CONST = 0, ABS_EIGEN = 1, ABS_POINT = 2 };

struct AxisInfo {
  int kind, bc_lo, bc_hi;
  int active;                 // 0: no advection along this axis
  int nadv;
  Term adv[MAXADV];           // beta^alpha = sum_t coef_t K_t
  int route;                  // how |beta| is applied on faces
  int absmat;                 // ABS_CONST: |beta| matrix id; ABS_POINT: pattern matrix id
  int Wmat, WTmat;            // ABS_EIGEN: eigenvectors W and W^T (bank ids)
  // ABS_EIGEN: beta = c0 I + c1 A with c0 = adv[0] coefficient, c1 = adv[1] coefficient at the face
  int llf;                    // local Lax--Friedrichs flux: |beta| replaced by alpha I, alpha = max |eig|
  double lam_lo, lam_hi;      // smallest and largest eigenvalue of A^a (alpha of the eigen route)
};

// Device-side CSR bank of n x n matrices (rowptr per matrix: n+1 entries at rp_off[m]).
template <typename T>
struct Bank {
  const int* rp;   // concatenated row pointers (absolute offsets into col/val)
  const int* col;
  const T* val;
  const T* dg;     // [nmat][n] diagonal of every matrix (at least n entries)
  int rp_off[96];
  // the same matrices in ELL form for the row-per-thread kernels: matrix m, row r, slot k < ell_w[m]
  // is entry ell_off[m] + k n + r, a (column, value) pair (EllEntry<T>); short rows are padded with
  // (r, 0), and n spare entries follow the last matrix
  const void* ell;
  int ell_off[96];
  int ell_w[96];
};

// One ELL entry: the column and the value, loaded together (8 bytes in FP32, 16 in FP64).
template <typename T>
struct alignas(2 * sizeof(T)) EllEntry {
  int col;
  T val;
};

template <typename T>
struct OpParams {
  int D, dx, q, nloc, nfp, n, ncell, has_mom;
  int qdx;                         // q^dx: spatial nodes per cell
  int nc[MAXD];
  AxisInfo ax[MAXD];
  int nreact;
  Term react[MAXTERMS];
  Bank<T> bank;
  T S[MAXQ][MAXQ];                 // S[i][q] = w_q l_i'(x_q) / w_i  on [0,1]
  T B0[MAXQ], B1[MAXQ];            // l_i(0), l_i(1)
  T L0[MAXQ], L1[MAXQ];            // l_i(0)/w_i, l_i(1)/w_i
  // mesh
  const int* cell_nb;              // [ncell][2D]: neighbour across face 2a+side, -1 at a boundary
  const T* cell_invh;              // [ncell][D]
  const int* cell_scell;           // [ncell] spatial cell
  const int* cell_pcell;           // [ncell] momentum cell (0 without momentum)
  const int* scell_face;           // [nscell][2*dx] first spatial-face point of each face of the cell
  // fields
  const T* sfield;                 // [SF_NCOMP][nsv] (components not uniform)
  int nsv;
  T sf_uni[SF_NCOMP];
  int sf_is_uni[SF_NCOMP];
  const T* uface[MAXD];            // [nsf_a]
  T uface_uni[MAXD];
  int uface_is_uni[MAXD];
  const T* nu;                     // [npv] or null (uniform nu_uni)
  T nu_uni;
  const T* s000;                   // [npv] or null (uniform s_uni)
  T s_uni;
  const T* pnode;                  // [npc*q] momentum p at nodes
  const T* pface;                  // [npc+1] momentum p at faces
  const T* mfn;                    // [MF_COUNT][npc*q] momentum factors at nodes
  const T* mff;                    // [MF_COUNT][npc+1] momentum factors at faces
  int npn;                         // npc*q
  T Vmono;
  // momentum-face |beta| per point
  const int* pslot;                // [nsv] slot or -1
  const T* pabs;                   // [slot][npc+1][nnz(pattern)]
  const T* pabs_ell;               // [slot][npc+1][ell_w(pattern)][n]: the same values in ELL order
  int npface;
  const T* lam;                    // eigenvalues of A^a (same for a = x, y, z), n entries
  // bit t set: the coefficient of reaction term t (of advection term t of axis a) is the same at
  // every node of every cell
  unsigned react_uni;
  unsigned adv_uni[MAXD];
  // bit t set: the coefficient of the term is identically zero (a uniform field component that is
  // zero, such as U = 0): the apply kernels skip it
  unsigned react_zero;
  unsigned adv_zero[MAXD];
  // uniform-coefficient kernel (uniform.cu): l_max of the compiled patterns it runs with, or -1;
  // the packed values of R, beta_a, |beta_a| (host memory owned by the context); cells per block
  // (0: the default)
  int uni_L = -1;
  const void* uni = nullptr;
  int uni_cells = 0;
  // row kernel: per-cell coefficient tables built at sap_set_fields (null: computed in the kernel):
  // node coefficients [cell][term][node], face coefficients [cell][face][term][point], and (FP32)
  // masks [cell][2 + 2D] of the terms nonzero somewhere in the cell
  const T* cvtab = nullptr;
  const T* cftab = nullptr;
  const unsigned* mktab = nullptr;
  const T* rdtab = nullptr;  // reaction diagonal per DoF (the point-Jacobi diagonal), or null
};

// Tables of the field-gradient kernels of the adjoint (adjoint_fields.cu): the spatial field
// components that enter some term (compact numbering), the per-cell partial layout, and for the
// momentum axis the Daleckii--Krein derivatives P_t = d|beta^p|[K_t] of the upwind matrix along each
// advection term, per (slot, momentum face) in the ELL order of the block pattern.
struct GradTables {
  int ncomp;                 // spatial field components with a gradient
  int comp_sf[SF_NCOMP];     // compact index -> SF component
  int sf_comp[SF_NCOMP];     // SF component -> compact index or -1
  int ps;                    // partials per cell: ncomp * qdx (spatial nodes) + 2 dx qsp (face points)
  int face_off;              // first face partial
  int qsp;                   // spatial points per spatial face
  const double* pd[MAXADV];  // [slot][momentum face][pd_w][n] per momentum advection term (or null)
  int pd_w;                  // ELL width of the block pattern (0: no momentum-face tables)
};

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

// Device tables for a batch of independent problems run by one launch per operator apply.
template <typename T>
struct BatchDev {
  const OpParams<T>* P = nullptr;     // [ninst] parameter blocks (device)
  const int64_t* doff = nullptr;      // [ninst] first DoF of each instance in the state vectors
  const int* cpb = nullptr;           // [ninst] cells per thread block
  const int* stride = nullptr;        // [ninst] shared-memory elements per cell
  const int2* blocks = nullptr;       // [nblocks] (instance, first cell)
  int nblocks = 0, threads = 0;
  size_t smem = 0;
  int shape_d = 0, shape_q = 0;       // common (D, q) of all instances, 0 if they differ
  int rows = 0;                       // 1: the row-per-thread kernel runs the batch
};

// Chunking of the concatenated state for the per-instance Krylov reductions: chunks never cross an
// instance boundary.
struct BatchChunks {
  const int* inst = nullptr;          // [nchunks] instance of the chunk
  const int64_t* k0 = nullptr;        // [nchunks] first element
  const int* len = nullptr;           // [nchunks] length (<= KRY_CHUNK)
  const int* first = nullptr;         // [ninst] first chunk of the instance
  const int* count = nullptr;         // [ninst] number of chunks of the instance
  int nchunks = 0;
};

}  // namespace sap

// The context (opaque to callers).
struct sap_ctx {
  sap_desc desc;
  int prec = SAP_PREC_FP64;
  int D = 0, dx = 0, q = 0, nloc = 0, nfp = 0, n = 0, ncell = 0, has_mom = 0, qdx = 0, nscell = 0;
  int nc[3] = {1, 1, 1};
  int64_t N = 0;
  int nsv = 0, npv = 0, nsf[3] = {0, 0, 0}, npc = 1;
  std::vector<double> edges[3];
  sap::SHTables T;
  std::vector<double> xg, wg;                  // Gauss rule on [0,1]
  std::vector<double> pnode, pface;            // momentum values
  std::vector<int> scell_face_h;               // [nscell][2dx]
  int uni_avail = -1;                          // l_max of the node kernel's patterns if the problem fits, else -1
  int apply_kernel = SAP_KERNEL_AUTO;          // sap_set_apply_kernel
  int uni_cells = 0;
  std::vector<double> uni_v64;                 // packed values of the uniform-coefficient kernel
  std::vector<float> uni_v32;
  sap::OpParams<double> p64{};
  sap::OpParams<float> p32{};
  std::vector<sap::DevBuf> owned;              // device allocations
  std::vector<std::vector<int>> Ablocks;       // (m,s) blocks of A^x
  bool fields_set = false;
  std::string err;
  // workspaces (FP64 state-sized vectors; FP32 where noted)
  double* ws64 = nullptr;
  int ws64_count = 0;
  float* ws32 = nullptr;
  int ws32_count = 0;
  double* small = nullptr;                     // block partial sums of the Krylov reductions (+ batch scalars)
  void* gdev = nullptr;                        // device Arnoldi control block
  void* gdev_host = nullptr;                   // pinned mirror
  int krylov_restart = 0;
  // CN initial-guess history: the state before the last step, valid for the buffer and dt it was
  // taken with (any other call starts from the plain previous state)
  const double* cn_prev_ptr = nullptr;
  double cn_prev_dt = 0.0, cn_prev_theta = 0.5;
  bool cn_prev_valid = false;
  // Arnoldi iterations of the last converged GMRES cycle with the same position in its solve (first,
  // second, ... cycle; forward and transposed operator): the size of the first group of iterations
  // enqueued for the next such cycle (0: fixed groups)
  int gm_hint[2][4] = {};
  std::vector<double> bank_nnz;                // nnz per bank matrix (cost model)
  double pslot_cell_frac = 1.0;                // spatial cells with a tabulated |beta^p| point (cost model)
  double sf_zero_frac32[sap::SF_NCOMP] = {};        // spatial cells where a field component is 0 in FP32 (cost model)
  int64_t launches = 0;                        // kernels launched by the current call
  // batches: a batch handle owns one sub-context per instance and runs them with batched launches
  std::vector<sap_ctx*> sub;
  std::vector<int64_t> inst_off;
  int fields_version = 0;                      // bumped by sap_set_fields
  int batch_built_version = -1;                // sum of the sub versions the batch tables were built for
  std::vector<int> batch_targets;              // autotuned thread-block target of every instance (per l_max)
  bool batch_tuned = false;
  std::vector<sap::DevBuf> batch_bufs;
  std::vector<sap::BatchDev<double>> b64;      // one launch per group of instances with the same l_max
  std::vector<sap::BatchDev<float>> b32;
  std::vector<int> batch_class;                // group of every instance
  sap::BatchChunks chunks;
  int* d_active = nullptr;                     // [ninst] device activity mask
  std::vector<int> h_active;
  sap_ctx* parent = nullptr;                   // set on the sub-contexts of a batch
  // CUDA graphs of the GMRES iteration groups of sap_step_cn (kind 0) and of the adjoint step (kind 1),
  // replayed while the configuration they were captured for (alpha, fields, workspace, group) holds
  struct CnGraph {
    cudaGraphExec_t exec = nullptr;
    int kind = 0, j0 = -1, cnt = 0, fields_version = -1;
    double alpha = 0.0;  // the captured operator A = 1 + alpha L
    const void* ws = nullptr;
  };
  std::vector<CnGraph> cn_graphs;
  cudaStream_t cap_stream = nullptr;           // private stream for the captures
  int flux = SAP_FLUX_UPWIND;                  // numerical flux of the faces (sap_set_flux)
  // batched CN: per-instance GMRES control blocks, masks and status (device, pinned mirror) and the
  // CUDA graphs of a step and of a continuation cycle
  void* bctl = nullptr;
  int* bmask = nullptr;
  void* bstat = nullptr;
  void* bstat_host = nullptr;
  struct BGraph {
    cudaGraphExec_t exec = nullptr;
    int kind = 0, extrap = 0, m = 0, maxit = 0, version = -1;
    const double* state = nullptr;
    double dt = 0.0, tol = 0.0;
    const void* ws = nullptr;
    int64_t launches = 0;
  };
  std::vector<BGraph> bgraphs;
  // field gradients of the adjoint: tables (built on first use for the current fields) and the
  // per-cell partials
  sap::GradTables gt{};
  int gt_version = -1;
  double* gpart = nullptr;
  size_t gpart_count = 0;
};

namespace sap {
// kernels / launchers implemented in operator.cu
cudaError_t launch_apply64(const OpParams<double>& p, const double* x, double* y, int mode, cudaStream_t s);
cudaError_t launch_apply32(const OpParams<float>& p, const float* x, float* y, int mode, cudaStream_t s);
sap_status erk_steps(sap_ctx* c, double* state, double dt, int nsteps, cudaStream_t s);
sap_status erk_steps_noalloc(sap_ctx* c, double* state, double dt, int nsteps, cudaStream_t s);
sap_status cn_steps(sap_ctx* c, double* state, double dt, double theta, int nsteps, double tol, int restart,
                    int maxit, sap_solver_stats* st, cudaStream_t s);
sap_status adjoint_cn_step(sap_ctx* c, const double* zp, const double* zn, double* lambda, double dt, double tol,
                           int m, int maxit, double* mu_out, double* grad_nu, sap_solver_stats* st, cudaStream_t s);
sap_status adjoint_erk_step(sap_ctx* c, const double* y, double* lambda, double dt, double* grad_nu, double* stages,
                            sap_solver_stats* st, cudaStream_t s);
int apply_cells_per_block(int n, int nloc);
// row-per-thread apply (apply_rows.cu) for the compiled shapes (D, q) = (1, 3), (2, 2), (3, 3)
bool rows_supported(int D, int q);

// Combined dense matrices (n x n, row major, FP64) of a problem whose term coefficients are all
// uniform: R = sum of the reaction terms, B[a] = sum of the advection terms of axis a, A[a] = the
// upwind matrix |beta_a| of axis a.
struct UniDense {
  int lmax = 0, n = 0;
  std::vector<double> R, B[3], A[3];
};
bool uni_supported(int lmax);
// floating-point operations of the node kernel per cell (axes with active[a] != 0)
double uni_flops_per_cell(int lmax, const int* active);
// the values at the compiled patterns' positions (R, B0..2, A0..2 in turn); false if l_max is not
// compiled or a matrix has a nonzero outside its pattern
bool uni_pack(const UniDense& u, std::vector<double>& vals);

template <typename T>
struct Epi;
template <typename T>
cudaError_t launch_uniform(const OpParams<T>& P, const T* x, const Epi<T>& e, cudaStream_t s);
template <typename T>
cudaError_t launch_rows(const OpParams<T>& P, const T* x, const Epi<T>& e, cudaStream_t s);
// build the row kernel's coefficient tables of P (device buffers appended to `owner`); with_diag: also
// the per-DoF reaction diagonal the Jacobi epilogues read
template <typename T>
cudaError_t build_coef_tables(OpParams<T>& P, std::vector<DevBuf>& owner, bool with_diag);
template <typename T>
cudaError_t launch_rows_transposed(const OpParams<T>& P, const T* x, const Epi<T>& e, cudaStream_t s);
// cells per block and dynamic shared memory (bytes) of the row kernel for a problem
template <typename T>
void rows_config(const OpParams<T>& P, int target_threads, int* cells, size_t* smem);
template <typename T>
cudaError_t launch_rows_batched(const BatchDev<T>& B, const int* active, const T* x, const Epi<T>& e, cudaStream_t s);
template <typename T>
cudaError_t prepare_rows_batched(const BatchDev<T>& B);  // shared-memory limit of the batched row kernel
int apply_cell_stride(const OpParams<double>& P);
sap_status batch_prepare(sap_ctx* c, cudaStream_t s);
sap_status batch_apply(sap_ctx* c, const void* x, void* y, int mode, cudaStream_t s);
sap_status batch_cn(sap_ctx* c, double* state, double dt, int nsteps, double tol, int restart, int maxit,
                    sap_solver_stats* st, cudaStream_t s);
sap_status batch_erk(sap_ctx* c, double* state, double dt, int nsteps, cudaStream_t s);
// field gradients of the adjoint (adjoint_fields.cu)
int coef_adjoint_smem_doubles(const OpParams<double>& P, const GradTables& G);
cudaError_t launch_coef_adjoint(const OpParams<double>& P, const GradTables& G, const double* g, const double* w,
                                double* part, cudaStream_t s);
cudaError_t launch_grad_reduce(const OpParams<double>& P, const GradTables& G, const double* part, int nscell,
                               int npc, double sigma, const sap_field_grads& out, cudaStream_t s);
cudaError_t launch_grad_src(const double* g, int64_t N, int nvec, int n, int nloc, int64_t npv, double coef,
                            double* grad, cudaStream_t s);
cudaError_t launch_add2(const double* a, const double* b, double* w, int64_t N, cudaStream_t s);
sap_status adjoint_fields_step(sap_ctx* c, int scheme, const double* zp, const double* zn, double* lambda, double dt,
                               double tol, int m, int maxit, const sap_field_grads& g, sap_solver_stats* st,
                               cudaStream_t s);
int64_t launch_count();
void cn_graphs_release(sap_ctx* c);  // destroys the cached CN graphs and the capture stream
int64_t krylov_scratch_doubles(int64_t N);
size_t gmres_control_bytes();
int64_t krylov_batch_scratch_doubles(const std::vector<int64_t>& Ns);
}  // namespace sap
