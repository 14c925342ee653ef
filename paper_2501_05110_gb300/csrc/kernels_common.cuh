// Device-side pieces shared by the operator kernels: the fused epilogue, coefficient helpers and
// node indexing of the tensor-product Gauss points.
#pragma once
#include <cuda_runtime.h>

#include <atomic>

#include "sap_internal.h"

namespace sap {

void note_launch();  // counts a kernel launch of this host thread (sap_solver_stats.kernel_launches)

// Devices whose kernel attributes the library tracks (ordinals 0 .. kMaxDevices-1).
constexpr int kMaxDevices = 256;

// One bit per device ordinal: the devices on which a kernel's attribute has been set.
struct DeviceMask {
  std::atomic<unsigned long long> w[kMaxDevices / 64];
};

// Raise `kernel`'s dynamic shared-memory limit to `bytes` on the current device.  The attribute is
// per device, so `done` (one per call site) records the devices already set.  Device ordinals
// beyond kMaxDevices are refused (cudaErrorInvalidDevice) instead of sharing another device's bit.
template <typename K>
inline cudaError_t smem_opt_in(K kernel, int bytes, DeviceMask& done) {
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  const unsigned long long bit = 1ull << (dev & 63);
  std::atomic<unsigned long long>& word = done.w[dev >> 6];
  if (word.load(std::memory_order_acquire) & bit) return cudaSuccess;
  err = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (err == cudaSuccess) word.fetch_or(bit, std::memory_order_acq_rel);
  return err;
}

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
  float* out32;         // optional: FP32 copy of out / (1 + cj * diag(R - div beta)), before `jacobi`
  T* out2;              // optional second output out2 = ax2*x + bl2*(Lx) + gs2*s
  T ax2, bl2, gs2;
  T* outj;              // optional: out2 (or out when out2 is null) / (1 + cj * diag(R - div beta))
  T axpost;             // added after the Jacobi scaling: out += axpost * x
  const int* skip;      // when non-null and *skip != 0 the launch does nothing
  const double* xs;     // when non-null, out (only) is multiplied by *xs: the apply of the vector *xs * x
  // ERK stage (k = s - Lx):  acc += bdt k ; ynext = y0 + adt k ; final: state = acc + bdt k
  double* acc;
  const double* y0;
  T* ynext;
  double adt, bdt;
  int erk;              // 0 none, 1 first stage (acc = y0 + bdt k), 2 middle, 3 last (y0 <- acc + bdt k)
  double* state;        // for erk == 3
};

// Loads never form an address outside an allocation, also on a path that a guard rules out: the
// guard selects the value after the load, or the load is a plain one that stays under its guard.
template <typename T>
__device__ __forceinline__ T csr_diag(const Bank<T>& B, int mat, int r, int n) {
  const T d = __ldg(B.dg + (mat < 0 ? 0 : mat) * n + r);  // the table has at least n entries
  return mat == MAT_I ? T(1) : d;
}

// 1 / (1 + cj d): the point-Jacobi scale; a preconditioner needs no FP64 division, so the reciprocal
// is taken in FP32 (the same fixed diagonal at every application)
template <typename T>
__device__ __forceinline__ T jacobi_scale(T cj, T rdiag) {
  return T(__frcp_rn(float(T(1) + cj * rdiag)));
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
  return P.sfield[(size_t)sf * P.nsv + sp];
}

// Index helpers: node index from a face point (axis a removed) and the position j along a; with
// a compile-time q the divisions become multiply-shifts.
__device__ __forceinline__ int face_node_q(int fp, int j, int a, int q) {
  if (a == 0) return j + fp * q;
  if (a == 1) return (fp % q) + j * q + (fp / q) * q * q;
  return (fp % (q * q)) + j * q * q + (fp / (q * q)) * q * q * q;
}
__device__ __forceinline__ int qpow_of(int q, int a) { return a == 0 ? 1 : (a == 1 ? q : (a == 2 ? q * q : q * q * q)); }

// Epilogue at one DoF: f = input value, acc = (M^-1 D f) at the DoF, s = source (row 0 only),
// rdiag = diagonal of the reaction operator at the DoF (used by the Jacobi outputs only).
template <typename T>
__device__ __forceinline__ void epi_write(const Epi<T>& E, size_t dof, T f, T acc, T s, T rdiag) {
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
  T o = E.ax * f + E.bl * acc + E.gs * s;
  if (E.bvec) o += E.wb * E.bvec[dof];
  if (E.out2) {
    const T o2 = E.ax2 * f + E.bl2 * acc + E.gs2 * s;
    E.out2[dof] = o2;
    if (E.outj) E.outj[dof] = o2 * jacobi_scale(E.cj, rdiag);
    if (E.out32) E.out32[dof] = float(o2 * jacobi_scale(E.cj, rdiag));
  } else {
    if (E.outj) E.outj[dof] = o * jacobi_scale(E.cj, rdiag);
    if (E.out32) E.out32[dof] = float(o * jacobi_scale(E.cj, rdiag));
  }
  if (E.jacobi) o *= jacobi_scale(E.cj, rdiag);
  if (E.axpost != T(0)) o += E.axpost * f;
  if (E.xs) o *= T(*E.xs);
  if (E.out) E.out[dof] = o;
}

}  // namespace sap
