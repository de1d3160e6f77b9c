// hydro_step_mixed.cuh -- the per-sub-grid hydro step in mixed precision:
// one persistent launch over a batch of ghost-filled sub-grids, each read
// from the padded state and its dU/dt written out.  Two decompositions of a
// sub-grid with the same arithmetic: the row sweep (hydro_mixed_body.cuh,
// which also carries the learned indicator) and the plane sweep
// (hydro_mixed_planes.cuh).  Instantiated without the spin feedback in
// hydro_step_mixed.cu and with it in hydro_step_mixed_spin.cu.
#pragma once
#include "hydro_mixed_planes.cuh"

namespace hyd {

// Padded state in, dU/dt and amax out, for the 8^3 tiles of NN^3 sub-grids
// (Tile).  Holds a reference to the kernel's parameters, so its pointers
// stay in the parameter bank (no registers).
template <int NN>
struct StepIo {
  using T = Tile<NN>;
  static constexpr bool kPrims = false;
  const StepArgs64& A;
  using Sub = T;
  __device__ __forceinline__ Sub begin(int u) const { return T(u); }
  __device__ __forceinline__ int sidx(const Sub& q) const { return q.s; }
  __device__ __forceinline__ int offx(const Sub& q) const { return q.o[0]; }
  __device__ __forceinline__ int offy(const Sub& q) const { return q.o[1]; }
  __device__ __forceinline__ void load(const Sub& q, int c, double u[F]) const { load_fields(q, c, 0, F, u); }
  __device__ __forceinline__ void load_fields(const Sub& q, int c, int f0, int nf, double* u) const {
    const double* __restrict__ Us = A.U + (size_t)q.s * F * T::kS3 + (size_t)f0 * T::kS3 + q.pad(c);
#pragma unroll
    for (int k = 0; k < nf; ++k) u[k] = __ldg(Us + (size_t)k * T::kS3);
  }
  // only the fields the sources read (rho, s, z_x, z_y)
  __device__ __forceinline__ void own(const Sub& q, int, int uc, double u[F]) const {
    const double* __restrict__ Us = A.U + (size_t)q.s * F * T::kS3 + q.pad(uc);
#pragma unroll
    for (int k = 0; k < F; ++k) u[k] = (k <= SZ || k == ZX || k == ZY) ? __ldg(Us + (size_t)k * T::kS3) : 0.0;
  }
  __device__ __forceinline__ void store(const Sub& q, int c, int, const double du[F], const double*) const {
    double* dU = A.dUdt + (size_t)q.s * F * T::kN3 + q.cell(c);
#pragma unroll
    for (int k = 0; k < F; ++k) dU[(size_t)k * T::kN3] = du[k];
  }
  __device__ __forceinline__ void grav(const Sub& q, int c, double& gx, double& gy, double& gz) const {
    const double* gs = A.g + (size_t)q.s * 3 * T::kN3 + q.cell(c);
    gx = gs[0];
    gy = gs[T::kN3];
    gz = gs[2 * T::kN3];
  }
  __device__ __forceinline__ void face(const Sub& q, int f, int k, int pc, int pb, double v) const {
    if (q.outer(f)) A.face_flux[q.face(f, k, pc, pb)] = v;
  }
  __device__ __forceinline__ void amax(const Sub& q, double m) const {
    if (T::kTiles == 1)
      A.amax[q.s] = m;
    else
      atomic_max_nonneg(A.amax + q.s, m);  // cleared before the launch
  }
};

// kGate: the learned smoothness indicator is on (A.gate); the kernel without
// it carries none of the indicator's registers.  kContact: contact
// steepening (A.P.contact).  kSpin: the spin feedback (A.P.spin), which the
// other instances carry none of.
template <bool kGate, bool kContact = false, int NN = N, bool kSpin = false>
__global__ void __launch_bounds__(kThreadsMx, 2) hydro_step_mixed_kernel(StepArgs64 A) {
  extern __shared__ __align__(128) float Qf[];  // [F][S3] FP32 primitives, then [2][S3] smooth flags
  __shared__ float red[kThreadsMx / 32];
  double* __restrict__ D = A.scratch + (size_t)blockIdx.x * kScratchPerSub;
  const RowMap R = row_map(threadIdx.x);
  const StepIo<NN> io{A};
  const int units = A.n_sub * Tile<NN>::kTiles;
  for (int u = blockIdx.x; u < units; u += gridDim.x) mixed_subgrid<kGate, kContact, kSpin>(A, io, u, R, Qf, red, D);
}

// The plane sweep: one CTA of kThreadsPl threads per SM (no indicator).
template <bool kContact, int NN = N, bool kSpin = false>
__global__ void __launch_bounds__(kThreadsPl, 1) hydro_step_mixed_planes_kernel(StepArgs64 A) {
  extern __shared__ __align__(128) unsigned char sm[];
  const StepIo<NN> io{A};
  const int units = A.n_sub * Tile<NN>::kTiles;
  for (int u = blockIdx.x; u < units; u += gridDim.x) mixed_subgrid_planes<kContact, kSpin>(A, io, u, sm);
}


template <int NN, bool kSpin>
static cudaError_t mixed_attrs() {
  const int rows = (int)kMixedSmemBytes, planes = (int)kPlaneSmemBytes;
  const cudaFuncAttribute at = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e = cudaFuncSetAttribute(hydro_step_mixed_kernel<false, false, NN, kSpin>, at, rows);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(hydro_step_mixed_kernel<true, false, NN, kSpin>, at, rows);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(hydro_step_mixed_kernel<false, true, NN, kSpin>, at, rows);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(hydro_step_mixed_kernel<true, true, NN, kSpin>, at, rows);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(hydro_step_mixed_planes_kernel<false, NN, kSpin>, at, planes);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(hydro_step_mixed_planes_kernel<true, NN, kSpin>, at, planes);
  return e;
}

template <int NN, bool kSpin>
static void launch_mixed_nn(const StepArgs64& A, int grid, int planes, cudaStream_t st) {
  if (planes && !A.gate) {
    if (A.P.contact)
      hydro_step_mixed_planes_kernel<true, NN, kSpin><<<grid, kThreadsPl, kPlaneSmemBytes, st>>>(A);
    else
      hydro_step_mixed_planes_kernel<false, NN, kSpin><<<grid, kThreadsPl, kPlaneSmemBytes, st>>>(A);
  } else if (A.gate) {
    if (A.P.contact)
      hydro_step_mixed_kernel<true, true, NN, kSpin><<<grid, kThreadsMx, kMixedSmemBytes, st>>>(A);
    else
      hydro_step_mixed_kernel<true, false, NN, kSpin><<<grid, kThreadsMx, kMixedSmemBytes, st>>>(A);
  } else if (A.P.contact) {
    hydro_step_mixed_kernel<false, true, NN, kSpin><<<grid, kThreadsMx, kMixedSmemBytes, st>>>(A);
  } else {
    hydro_step_mixed_kernel<false, false, NN, kSpin><<<grid, kThreadsMx, kMixedSmemBytes, st>>>(A);
  }
}

}  // namespace hyd
