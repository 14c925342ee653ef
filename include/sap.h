/*
 * sap.h -- C ABI of the GB300 library for the discontinuous-Galerkin spherical-harmonic
 * Vlasov--Fokker--Planck operator of arXiv:2501.05110 ("Sapphire++").
 *
 * The library discretises the advection--reaction system
 *     d_t f + (beta . grad~) f + R f = s                              (Sec. 2.2, Eq. well-posed-...)
 * for the n = (lmax+1)^2 expansion coefficients f_lms (Sec. 2.1) with a dG method on a
 * tensor-product mesh of the reduced phase space xi = (x[, y[, z]][, p or ln p]) (Sec. 3):
 * broken Q^k space, upwind numerical flux J = W (L+ W^T f1 + L- W^T f2) (Eq. definition-upwind-flux),
 * zero-inflow / continuous / periodic boundaries (Eq. definition-boundary-flux, Eq. continuous-bc),
 * and advances M zeta' + D zeta = h (Eq. matrix-formulation-system-odes) with explicit RK4 or the
 * Crank--Nicolson theta-method solved by restarted GMRES (Eq. theta-method, Eq. system-matrix-rhs).
 *
 * Conventions used by every entry point:
 *  - Status: every call returns sap_status and never aborts; sap_last_error() gives text for the
 *    last failure on that handle.  Asynchronous CUDA errors surface as SAP_ECUDA at the next call
 *    that synchronises.
 *  - Ownership: the caller owns every buffer it passes (state vectors, field arrays); the library
 *    owns its tables and workspaces, released by sap_destroy().  Host arrays passed to setup calls
 *    are copied before the call returns.
 *  - State layout (device, canonical): index = ((cell * n + j) * (k+1)^D + node), cells
 *    lexicographic with axis 0 fastest, j the paper's index map j(l,m,s) = l(l+1) + (-1)^(s+1) m
 *    (Eq. ordering-expansion-coefficients), nodes the tensor Gauss--Legendre points of the cell
 *    (axis 0 fastest).  Values are nodal values of f_h at those points.  In this basis the mass
 *    matrix is diagonal and the initial projection (Eq. zeta-initial-condition) is evaluation of
 *    f^0 at the nodes.
 *  - Streams: compute entry points take a cudaStream_t (0 = legacy default stream) and are
 *    asynchronous with respect to the host unless stated otherwise.
 *  - Thread safety: one handle must not be used from two host threads at once.  Different
 *    handles may be used from different threads and on different devices (each handle lives on
 *    the device that was current at sap_create; make that device current for its calls).
 *  - Aliasing: device buffers passed to one call must not overlap unless the call says so (a
 *    vector updated in place, such as `state` or `lambda`, is one buffer).
 */
#ifndef SAP_H
#define SAP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sap_ctx* sap_handle;
typedef struct CUstream_st* sap_stream; /* same object as cudaStream_t */

typedef enum {
  SAP_OK = 0,
  SAP_EINVAL = 1,        /* invalid argument or descriptor */
  SAP_ENOMEM = 2,        /* device or host allocation failed */
  SAP_ECUDA = 3,         /* a CUDA call failed (text in sap_last_error) */
  SAP_ENOCONV = 4,       /* the iterative solve did not reach the tolerance within maxit */
  SAP_ETIMEOUT = 5,      /* a bounded device-side wait gave up */
  SAP_EUNSUPPORTED = 6   /* valid request outside what this build implements */
} sap_status;

/* axis kinds: spatial axes come first in x, y, z order, the momentum axis (if any) last */
enum { SAP_AXIS_X = 0, SAP_AXIS_Y = 1, SAP_AXIS_Z = 2, SAP_AXIS_P = 3, SAP_AXIS_LNP = 4 };
/* boundary conditions per axis end (Sec. 2.2; Eq. definition-boundary-flux; Eq. continuous-bc) */
enum { SAP_BC_PERIODIC = 0, SAP_BC_ZERO_INFLOW = 1, SAP_BC_CONTINUOUS = 2 };
/* term toggles (Eq. vfp-terms-names): spatial advection, momentum, rotation, collision, source */
enum { SAP_TERM_ADV = 1, SAP_TERM_MOM = 2, SAP_TERM_ROT = 4, SAP_TERM_COLL = 8, SAP_TERM_SRC = 16 };
/* arithmetic of the operator apply: FP64 throughout, or FP32 apply with FP64 state/Krylov */
enum { SAP_PREC_FP64 = 0, SAP_PREC_FP32 = 1 };
/* apply modes */
enum { SAP_APPLY_D = 0,        /* y = M^-1 D x                       */
       SAP_APPLY_RHS = 1,      /* y = M^-1 (h - D x)  (ERK right side) */
       SAP_APPLY_T = 2 };      /* y = (M^-1 D)^T x: transpose of the nodal operator (discrete adjoint) */
/* numerical flux on the faces (sap_set_flux) */
enum { SAP_FLUX_UPWIND = 0,    /* J = W (L+ W^T f_lo + L- W^T f_hi)  (Eq. definition-upwind-flux)        */
       SAP_FLUX_LLF = 1 };     /* local Lax--Friedrichs: J = 1/2 beta (f_lo + f_hi) + 1/2 alpha (f_lo - f_hi),
                                  alpha = largest |eigenvalue| of n.beta at the face point                */
/* operator-apply kernel choice (sap_set_apply_kernel) */
enum { SAP_KERNEL_AUTO = 0,    /* the node kernel for uniform-coefficient 3-D k = 2 problems, else the row kernel */
       SAP_KERNEL_ROWS = 1 };  /* always the row kernel (or the cell-node kernel for shapes it lacks)        */
/* point sets reported by sap_field_points */
enum { SAP_PTS_SPATIAL = 0,    /* spatial volume points (nsv x dim_x), fields U, gradU, DUDt, B   */
       SAP_PTS_FACE_X = 1,     /* spatial face points normal to x (nsf x dim_x), field U_x         */
       SAP_PTS_FACE_Y = 2,     /*   ... normal to y, field U_y                                     */
       SAP_PTS_FACE_Z = 3,     /*   ... normal to z, field U_z                                     */
       SAP_PTS_PHASE = 4 };    /* phase-space volume points = nodes (N/n x D), fields nu, s_000    */

typedef struct {
  int ndim;                 /* D = number of reduced phase-space axes, 1..3 (Sec. 4, footnote)    */
  int axis_kind[3];         /* SAP_AXIS_*                                                         */
  int ncells[3];            /* cells per axis, >= 1                                               */
  const double* edges[3];   /* host, ncells[a]+1 strictly increasing edges (graded meshes allowed) */
  int bc_lo[3], bc_hi[3];   /* SAP_BC_*; periodic must be set on both ends                         */
  int lmax;                 /* expansion order, 0..11; n = (lmax+1)^2 (Sec. 2.1)                  */
  int degree;               /* dG degree k >= 0 (Sec. 3.1), k <= 5                                 */
  double V;                 /* particle speed, used only without a momentum axis                  */
  unsigned terms;           /* OR of SAP_TERM_*                                                    */
} sap_desc;

typedef struct {
  int steps;                /* CN steps taken                                                      */
  int64_t iterations;       /* total GMRES iterations over all steps                               */
  int max_iterations;       /* most iterations in one step                                         */
  double last_rel_residual; /* true relative residual ||b - A x|| / ||b|| of the last step         */
  int64_t kernel_launches;  /* CUDA kernels this call launched (operator applies + Krylov kernels)  */
} sap_solver_stats;

/* Create a context for one problem (Sec. 2-3).  Builds the coupling matrices A^a, Omega^a, C and
 * their products at L = lmax+1 (Sec. 2.1), the eigen-pairs of A^x once and their rotations for y, z
 * (Sec. 3.2, "eigenvectors once"), the Gauss rules and the mesh tables, and allocates device
 * workspaces on the current CUDA device.  `prec` is SAP_PREC_*.  Fields must be set with
 * sap_set_fields before any compute call.  Errors: SAP_EINVAL (bad descriptor), SAP_ENOMEM,
 * SAP_ECUDA.  On failure *out is NULL. */
sap_status sap_create(const sap_desc* desc, int prec, sap_handle* out);

/* Create a batch of `ninst` independent problems (one descriptor each; different lmax, degree,
 * meshes and fields allowed) that run together: every operator apply is one kernel launch over all
 * instances.  sap_step_cn runs one restarted GMRES per instance (own Krylov space, Hessenberg matrix,
 * Givens rotations and convergence test) with the control on the device: a CN step is one CUDA-graph
 * launch (captured on first use for the state buffer, dt, tolerances and fields), finished instances
 * cost nothing in later launches, and the host reads the per-instance status once per step.  The
 * batch state is the concatenation of the instances' canonical states (offsets from
 * sap_batch_instance).  The tile shape (cells per thread block) is autotuned per expansion order on
 * the first compute call by timing the batched apply of each l_max class.  sap_apply_operator,
 * sap_step_erk and sap_step_cn accept the batch handle.  Fields are set per instance through the
 * sub-handles of sap_batch_instance.  Errors as sap_create. */
sap_status sap_create_batch(int ninst, const sap_desc* descs, int prec, sap_handle* out);

/* Sub-handle of instance `inst` of a batch (for sap_field_points, sap_set_fields, sap_num_dofs; owned
 * by the batch, not to be destroyed) and the instance's first element in the batch state. */
sap_status sap_batch_instance(sap_handle batch, int inst, sap_handle* sub, int64_t* offset);

/* Number of points and their coordinates for a point set (SAP_PTS_*).  If `coords` is NULL only
 * *count is written; otherwise `coords` (host) receives count x dim coordinates, dim = number of
 * spatial axes (momentum coordinates are p, not ln p, for SAP_PTS_PHASE's momentum column when the
 * axis is SAP_AXIS_LNP: the column holds ln p as the mesh coordinate).  Errors: SAP_EINVAL. */
sap_status sap_field_points(sap_handle h, int which, double* coords, int64_t* count);

/* Set the prescribed fields, sampled at the points of sap_field_points (host arrays, copied):
 *  U[nsv*3], gradU[nsv*9] with gradU[p*9 + 3a + b] = dU_b/dx^a, DUDt[nsv*3] (material derivative of
 *  the flow), Bw[nsv*3] = B with a momentum axis (omega = qB/(gamma m), q = m = c = 1, Tab. 1) or
 *  omega directly without one; Uface[a][nsf_a] = U_a at the spatial face points normal to spatial
 *  axis a (NULL for absent axes); nu[npv] (scattering frequency) and s000[npv] (isotropic source,
 *  s = s000 Y_000) at the phase-space nodes.  Any pointer may be NULL when the corresponding terms
 *  are off.  Builds the per-face upwind data, including the eigen-decomposition of beta^p at every
 *  momentum-face point (Sec. 3.2, Eq. beta-p).  Synchronous.  Errors: SAP_EINVAL, SAP_ENOMEM,
 *  SAP_ECUDA. */
sap_status sap_set_fields(sap_handle h, const double* U, const double* gradU, const double* DUDt,
                          const double* Bw, const double* const Uface[3], const double* nu,
                          const double* s000);

/* sap_set_fields with the field arrays in device memory (same shapes and layouts; any pointer may be
 * NULL): the arrays are read on `stream`, after the work already queued there (for instance the
 * kernels that produced them), with one synchronisation of that stream; then the term tables and the
 * momentum-face eigen data are built as in sap_set_fields.  The device arrays may be reused or freed
 * once the call returns.  Errors: SAP_EINVAL (also for a batch handle: set the fields of its
 * instances), SAP_ENOMEM, SAP_ECUDA. */
sap_status sap_set_fields_device(sap_handle h, const double* U, const double* gradU, const double* DUDt,
                                 const double* Bw, const double* const Uface[3], const double* nu,
                                 const double* s000, sap_stream stream);

/* Choose the numerical flux of the faces (SAP_FLUX_*; the default is the upwind flux of Eq.
 * definition-upwind-flux; the paper names the local Lax--Friedrichs flux as the alternative, Sec. 3.2).
 * Boundaries keep their definitions with the flux's split: zero inflow takes the outgoing half
 * 1/2 (beta +- alpha) of the chosen flux, continuous takes beta.  Takes effect at the next
 * sap_set_fields; changing it clears the fields, which must be set again.  sap_adjoint_step does not
 * differentiate the LLF flux (alpha is a maximum over eigenvalues) and returns SAP_EUNSUPPORTED for it.
 * Errors: SAP_EINVAL. */
sap_status sap_set_flux(sap_handle h, int flux);

/* Choose the kernel of the forward operator apply (y = M^-1 D x and the fused RK4 / CN forms; the
 * transposed apply always runs the row kernel).  SAP_KERNEL_AUTO (the default) runs, for a spatial
 * 3-D problem with k = 2 and l_max <= 5 whose every term coefficient is one number (uniform U, B and
 * nu; constant upwind matrices), the node kernel: one thread per node with the combined coupling
 * matrices R = sum_t c_t K_t, beta_a and |beta_a| applied as compiled sparse patterns (the operator of
 * Eq. definition-mass-and-dg-matrix written as sums of Kronecker products).  Other problems run the
 * row kernel.  SAP_KERNEL_ROWS forces the row kernel.  cells_per_block > 0 sets the node kernel's
 * cells per block (clamped to 8 in FP32, 4 in FP64); 0 keeps the default (the largest).  Both kernels
 * compute the same operator; results differ by the order of the sums.  Takes effect at the next apply
 * or step (CUDA graphs captured before the call are captured again).  Errors: SAP_EINVAL (null
 * handle, unknown kernel, negative cells, a batch handle). */
sap_status sap_set_apply_kernel(sap_handle h, int kernel, int cells_per_block);
/* The kernel the forward apply runs now: 1 the node kernel (uniform coefficients), 0 the row kernel
 * or the cell-node kernel.  Errors: SAP_EINVAL (null handle or pointer, fields not set). */
sap_status sap_apply_kernel_in_use(sap_handle h, int* uniform);

/* Number of degrees of freedom N = ncells * n * (k+1)^D (Sec. 3.1). */
sap_status sap_num_dofs(sap_handle h, int64_t* n);

/* Apply the semi-discrete operator (Eq. definition-mass-and-dg-matrix) to a device vector x,
 * writing device vector y (x != y, both canonical layout, N elements of the context's precision:
 * double for SAP_PREC_FP64, float for SAP_PREC_FP32).  mode SAP_APPLY_D: y = M^-1 D x;
 * SAP_APPLY_RHS: y = M^-1 (h - D x); SAP_APPLY_T: y = (M^-1 D)^T x, the transpose of the nodal
 * operator, built term by term (transposed couplings, S^T along lines, face lifts and traces
 * exchanged, upwind splits beta+/beta- per side).  Asynchronous on `stream`.
 * Errors: SAP_EINVAL, SAP_ECUDA. */
sap_status sap_apply_operator(sap_handle h, const void* x, void* y, int mode, sap_stream stream);

/* Advance the FP64 device state (canonical layout, N doubles, in place) by `nsteps` classical RK4
 * steps of size dt on zeta' = M^-1 (h - D zeta) (Sec. 3.4).  With SAP_PREC_FP32 the stage
 * derivatives are computed in FP32 and accumulated into the FP64 state.  Asynchronous.
 * Errors: SAP_EINVAL, SAP_ECUDA. */
sap_status sap_step_erk(sap_handle h, double* state, double dt, int nsteps, sap_stream stream);

/* Advance the FP64 device state by `nsteps` Crank--Nicolson steps (theta = 1/2, Eq. theta-method):
 * (1 + dt/2 M^-1 D) zeta^n = (1 - dt/2 M^-1 D) zeta^(n-1) + dt M^-1 h, each solved by restarted
 * GMRES(restart) with point-Jacobi preconditioning to ||b - A zeta|| <= tol ||b|| (2-norm,
 * canonical nodal vector), at most maxit iterations per step.  With SAP_PREC_FP32 the inner GMRES
 * applies the operator in FP32 to FP32 Krylov vectors, orthogonalised with FP64-class accuracy
 * (exact FP32 products and compensated sums, ~2^-48 relative), and an FP64 residual/refinement loop
 * restores the tolerance.
 * Synchronous (reads the convergence status each restart).  `stats` may be NULL.
 * Errors: SAP_EINVAL, SAP_ENOCONV (state holds the last iterate), SAP_ECUDA. */
sap_status sap_step_cn(sap_handle h, double* state, double dt, int nsteps, double tol, int restart,
                       int maxit, sap_solver_stats* stats, sap_stream stream);

/* Advance the FP64 device state by `nsteps` steps of the theta-method (Eq. theta-method):
 * (1 + theta dt M^-1 D) zeta^n = (1 - (1 - theta) dt M^-1 D) zeta^(n-1) + dt M^-1 h, theta in [0, 1]
 * (0: forward Euler, 1: backward Euler, 1/2: Crank--Nicolson, the same as sap_step_cn), solved as in
 * sap_step_cn (for theta = 0 the system matrix is the identity and GMRES ends after one iteration).
 * Synchronous.  Errors: SAP_EINVAL (theta outside [0, 1], bad arguments), SAP_ENOCONV, SAP_ECUDA,
 * SAP_EUNSUPPORTED (batch handles with theta != 1/2). */
sap_status sap_step_theta(sap_handle h, double* state, double dt, double theta, int nsteps, double tol, int restart,
                          int maxit, sap_solver_stats* stats, sap_stream stream);

/* One step of the discrete adjoint of the Crank--Nicolson step (Eq. theta-method, theta = 1/2).
 * The forward step maps zeta_prev to zeta_next through A zeta_next = B zeta_prev + dt M^-1 h with
 * A = 1 + dt/2 M^-1 D, B = 1 - dt/2 M^-1 D.  On entry `lambda` (device, N doubles) holds dJ/dzeta_next;
 * the call solves A^T mu = lambda by restarted GMRES on the transposed operator (Jacobi, tolerance
 * `tol` on the true relative residual), overwrites lambda with B^T mu = dJ/dzeta_prev, writes mu to
 * `mu_out` when it is not NULL (for derivatives the caller forms itself), and, when `grad_nu` is not
 * NULL, adds dJ/dnu at every phase-space node: -dt/2 sum_j mu_j l_j(l_j+1)/2 (zeta_prev+zeta_next)_j
 * (the collision term nu C of Eq. definitions-advection-reaction-eq is pointwise in the nodal basis).
 * zeta_prev / zeta_next are the forward states (device).  Synchronous.  `stats` may be NULL.
 * Errors: SAP_EINVAL, SAP_ENOCONV, SAP_ECUDA, SAP_EUNSUPPORTED (batch handles, FP32 contexts). */
sap_status sap_adjoint_step_cn(sap_handle h, const double* zeta_prev, const double* zeta_next, double* lambda,
                               double dt, double tol, int restart, int maxit, double* mu_out, double* grad_nu,
                               sap_solver_stats* stats, sap_stream stream);

/* One step of the discrete adjoint of the classical RK4 step of sap_step_erk (Sec. 3.4, last
 * paragraph) on zeta' = s - L zeta, L = M^-1 D.  On entry `lambda` (device, N doubles) holds
 * dJ/dzeta_next for the step that starts from `zeta_prev` (device, N doubles); on return it holds
 * dJ/dzeta_prev.  The call recomputes the stage inputs Y_1 = zeta_prev, Y_2 = Y_1 + dt/2 k_1,
 * Y_3 = Y_1 + dt/2 k_2, Y_4 = Y_1 + dt k_3 (k_i = s - L Y_i), forms the stage adjoints in reverse
 * order, kb_4 = dt/6 lambda, kb_3 = dt/3 lambda - dt L^T kb_4, kb_2 = dt/3 lambda - dt/2 L^T kb_3,
 * kb_1 = dt/6 lambda - dt/2 L^T kb_2, and sets lambda <- lambda - L^T (kb_1 + kb_2 + kb_3 + kb_4).
 * When `grad_nu` (device, one double per phase-space node) is not NULL it adds dJ/dnu there:
 * -sum_i sum_j kb_i,j l_j(l_j+1)/2 Y_i,j (the collision term is pointwise in the nodal basis).
 * When `stages_out` (device, 7 N doubles, caller-owned) is not NULL the call keeps Y_2, Y_3, Y_4,
 * kb_1, kb_2, kb_3, kb_4 there, in that order, for derivatives the caller forms itself (a parameter
 * theta adds sum_i kb_i . dF/dtheta(Y_i)).  Synchronous.  `stats` may be NULL.
 * Errors: SAP_EINVAL, SAP_ENOMEM, SAP_ECUDA, SAP_EUNSUPPORTED (batch handles, FP32 contexts). */
sap_status sap_adjoint_step_erk(sap_handle h, const double* zeta_prev, double* lambda, double dt, double* grad_nu,
                                double* stages_out, sap_solver_stats* stats, sap_stream stream);

/* Time-stepping schemes of sap_adjoint_step */
enum { SAP_SCHEME_ERK4 = 0, SAP_SCHEME_CN = 1 };

/* Gradient accumulators of sap_adjoint_step: device arrays (caller-owned, FP64) with the shapes and
 * layouts of the field arrays of sap_set_fields; each call ADDS its contribution.  Any pointer may
 * be NULL (that gradient is not formed). */
typedef struct {
  double* U;          /* [nsv * 3]   dJ/dU_a at the spatial points                                  */
  double* gradU;      /* [nsv * 9]   dJ/d(dU_b/dx^a), index p*9 + 3a + b                             */
  double* DUDt;       /* [nsv * 3]   dJ/d(DU_a/Dt)                                                   */
  double* Bw;         /* [nsv * 3]   dJ/dB_a (momentum axis) or dJ/domega_a (no momentum axis)       */
  double* Uface[3];   /* [nsf_a]     dJ/dU_a at the spatial face points normal to axis a             */
  double* nu;         /* [npv]       dJ/dnu at the phase-space nodes                                 */
  double* s000;       /* [npv]       dJ/ds_000 at the phase-space nodes                              */
} sap_field_grads;

/* One step of the discrete adjoint of sap_step_cn (scheme SAP_SCHEME_CN: theta = 1/2 of Eq.
 * theta-method, solved as in sap_adjoint_step_cn) or of sap_step_erk (SAP_SCHEME_ERK4: the stage
 * adjoints of sap_adjoint_step_erk), with the gradients of J with respect to every prescribed field
 * at the points where it is sampled.  On entry `lambda` (device, N doubles) holds dJ/dzeta_next;
 * on return dJ/dzeta_prev.  zeta_prev (and, for CN, zeta_next) are the forward states (device).
 * A field theta enters the CN step through -dt/2 mu^T (dL/dtheta)(zeta_prev + zeta_next) + dt mu^T
 * ds/dtheta (mu = A^-T lambda) and the RK4 step through sum_i kb_i^T (ds/dtheta - (dL/dtheta) Y_i),
 * L = M^-1 D (Eq. definition-mass-and-dg-matrix).  dL/dtheta is exact: L is linear in the
 * coefficients of its volume and face terms (Eq. definitions-advection-reaction-eq, Eq.
 * definition-upwind-flux); the upwind matrices |beta| are differentiated by the Daleckii--Krein
 * formula d|beta|[dB] = W (Gamma o (W^T dB W)) W^T with Gamma_ij = (|l_i| - |l_j|)/(l_i - l_j) (sign
 * for equal signs, 0 where both eigenvalues vanish: the zero subgradient at the kink of |.|).
 * Gradients are formed for the field components that are non-zero somewhere at sap_set_fields (the
 * components whose terms the operator contains); a component that is identically zero there adds
 * nothing.  Points where |beta^p| was dropped as negligible add nothing to the momentum-face part.
 * The first call after sap_set_fields builds the derivative tables of |beta^p| on the host.
 * Synchronous.  tol, restart, maxit: the adjoint GMRES of the CN scheme (ignored for RK4).
 * Errors: SAP_EINVAL, SAP_ENOCONV, SAP_ENOMEM, SAP_ECUDA, SAP_EUNSUPPORTED (batch handles, FP32
 * contexts, a cell too large for the gradient kernel's shared memory). */
sap_status sap_adjoint_step(sap_handle h, int scheme, const double* zeta_prev, const double* zeta_next,
                            double* lambda, double dt, double tol, int restart, int maxit,
                            const sap_field_grads* grads, sap_solver_stats* stats, sap_stream stream);

/* Largest N (degrees of freedom) that sap_step_erk_noalloc accepts. */
#define SAP_NOALLOC_MAX_DOFS 262144

/* Same RK4 steps as sap_step_erk, but without allocating device memory.  The paper has no
 * counterpart: this is an interface for callers that cannot allocate, for instance code that
 * captures the step into a CUDA graph with a global-mode stream capture (where cudaMalloc is not
 * allowed), a framework whose own allocator must account for every byte of device memory, or a
 * loop that cannot absorb the device-wide synchronisation of cudaMalloc/cudaFree.
 * The stage buffers (two stage inputs and the accumulator, at most 24 bytes per DoF) live in one
 * fixed array of 24 * SAP_NOALLOC_MAX_DOFS bytes (6 MiB) that every GPU which loads the library
 * holds until the process exits.  The first call on each device looks up that array's device
 * address (cudaGetSymbolAddress) with the device current; make that first call before any stream
 * capture.  The address is kept for the life of the process: after cudaDeviceReset (or any other
 * teardown of the device's primary context) the library must not be used on that device again.
 * Every call shares the one array and it keeps the last call's contents; each step writes every
 * scratch value before reading it, so nothing needs clearing.  Calls that overlap on the GPU (other
 * streams, threads or handles on the same device) race on the array.  Like sap_step_erk, the call
 * ends the CN initial-guess history of the handle (the next sap_step_cn starts from the plain
 * previous state).
 * Errors: SAP_EINVAL (N > SAP_NOALLOC_MAX_DOFS, fields not set, bad arguments), SAP_EUNSUPPORTED
 * (batch handles: use sap_step_erk), SAP_ECUDA. */
sap_status sap_step_erk_noalloc(sap_handle h, double* state, double dt, int nsteps, sap_stream stream);

/* Algorithmic cost of one sap_apply_operator call on this context: `flops` = floating-point
 * operations (an FMA counts 2) summed from the kernel's term tables (coefficient set-up, traces,
 * upwind fluxes, volume terms, lifts; for the node kernel its own count from the compiled patterns:
 * reaction, derivative along each axis, beta_a, lifts, traces, beta_a and |beta_a| at the faces) of the
 * kernel the forward apply runs now (sap_apply_kernel_in_use); `bytes` = 2 N w (read x, write y; w = word size of the
 * context's precision).  Host-only.  Errors: SAP_EINVAL (fields not set). */
sap_status sap_apply_cost(sap_handle h, double* flops, double* bytes);

/* Measured fused-multiply-add throughput of the current device in precision `prec` (SAP_PREC_FP64 or
 * SAP_PREC_FP32), in flop/s (an FMA counts 2): eight independent FMA chains per thread on every SM,
 * timed with CUDA events over five launches after a warm-up.  The arithmetic roof of the operator
 * apply, which is above the ridge point in both precisions.  The paper has no counterpart
 * (measurement).  Synchronous; allocates a small output buffer.  Errors: SAP_EINVAL, SAP_ECUDA. */
sap_status sap_probe_fma(int prec, double* flops_per_s);

/* Destroy a context and free its device memory.  NULL is accepted. */
sap_status sap_destroy(sap_handle h);

/* Text of the last error on `h` (or of the last failed sap_create when h is NULL). */
const char* sap_last_error(sap_handle h);

/* Host-only: copy the library's n x n coupling matrix `which` for expansion order lmax into `out`
 * (row-major, n*n doubles).  which: 0 A^a, 1 Omega^a, 2 C, 3 A^a A^b, 4 E^a = eps_abc A^b Om^c,
 * 5 F^ab = A^a E^b (a, b in 0..2 select components; products formed at L = lmax+1, Sec. 2.1).
 * Needs no GPU.  Errors: SAP_EINVAL. */
sap_status sap_coupling_matrix(int lmax, int which, int a, int b, double* out);

#ifdef __cplusplus
}
#endif
#endif /* SAP_H */
