// hydro_step_mixed.cu -- the per-sub-grid hydro step in mixed precision:
// one persistent launch over a batch of ghost-filled sub-grids, each read
// from the padded state and its dU/dt written out.  Two decompositions of a
// sub-grid with the same arithmetic: the row sweep (hydro_mixed_body.cuh,
// which also carries the learned indicator) and the plane sweep
// (hydro_mixed_planes.cuh).
#include "hydro_mixed_planes.cuh"

namespace hyd {

// Padded state in, dU/dt and amax out.  Holds a reference to the kernel's
// parameters, so its pointers stay in the parameter bank (no registers).
struct StepIo {
  const StepArgs64& A;
  struct Sub {
    int s;
  };
  __device__ __forceinline__ Sub begin(int s) const { return Sub{s}; }
  __device__ __forceinline__ void load(const Sub& q, int c, double u[F]) const {
    const double* __restrict__ Us = A.U + (size_t)q.s * F * S3;
#pragma unroll
    for (int k = 0; k < F; ++k) u[k] = __ldg(Us + (size_t)k * S3 + c);
  }
  __device__ __forceinline__ void load_fields(const Sub& q, int c, int f0, int nf, double* u) const {
    const double* __restrict__ Us = A.U + (size_t)q.s * F * S3 + (size_t)f0 * S3 + c;
#pragma unroll
    for (int k = 0; k < nf; ++k) u[k] = __ldg(Us + (size_t)k * S3);
  }
  // only the fields the sources read (rho, s, z_x, z_y)
  __device__ __forceinline__ void own(const Sub& q, int, int uc, double u[F]) const {
    const double* __restrict__ Us = A.U + (size_t)q.s * F * S3;
#pragma unroll
    for (int k = 0; k < F; ++k) u[k] = (k <= SZ || k == ZX || k == ZY) ? __ldg(Us + (size_t)k * S3 + uc) : 0.0;
  }
  __device__ __forceinline__ void store(const Sub& q, int c, int, const double du[F], const double*) const {
    double* dU = A.dUdt + (size_t)q.s * F * N3;
#pragma unroll
    for (int k = 0; k < F; ++k) dU[k * N3 + c] = du[k];
  }
  __device__ __forceinline__ void amax(const Sub& q, double m) const { A.amax[q.s] = m; }
};

// kGate: the learned smoothness indicator is on (A.gate); the kernel without
// it carries none of the indicator's registers.  kContact: contact
// steepening (A.P.contact; not combined with the indicator).
template <bool kGate, bool kContact = false>
__global__ void __launch_bounds__(kThreadsMx, 2) hydro_step_mixed_kernel(StepArgs64 A) {
  extern __shared__ __align__(128) float Qf[];  // [F][S3] FP32 primitives, then [2][S3] smooth flags
  __shared__ float red[kThreadsMx / 32];
  double* __restrict__ D = A.scratch + (size_t)blockIdx.x * kScratchPerSub;
  const RowMap R = row_map(threadIdx.x);
  const StepIo io{A};
  for (int s = blockIdx.x; s < A.n_sub; s += gridDim.x) mixed_subgrid<kGate, kContact>(A, io, s, R, Qf, red, D);
}

// The plane sweep: one CTA of kThreadsPl threads per SM (no indicator).
template <bool kContact>
__global__ void __launch_bounds__(kThreadsPl, 1) hydro_step_mixed_planes_kernel(StepArgs64 A) {
  extern __shared__ __align__(128) unsigned char sm[];
  const StepIo io{A};
  for (int s = blockIdx.x; s < A.n_sub; s += gridDim.x) mixed_subgrid_planes<kContact>(A, io, s, sm);
}

size_t step_mixed_smem_bytes() { return kMixedSmemBytes; }

// Opt in to the kernels' dynamic shared memory once per device (no
// allocation; call before any stream capture).
cudaError_t prepare_step_mixed() {
  static unsigned long long done = 0;
  return once_per_device(&done, [] {
    cudaError_t e = cudaFuncSetAttribute(hydro_step_mixed_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)step_mixed_smem_bytes());
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(hydro_step_mixed_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)step_mixed_smem_bytes());
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(hydro_step_mixed_kernel<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)step_mixed_smem_bytes());
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(hydro_step_mixed_planes_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)kPlaneSmemBytes);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(hydro_step_mixed_planes_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)kPlaneSmemBytes);
    return e;
  });
}

// planes: the plane-sweep decomposition (grid: CTAs, at most one per SM);
// the learned indicator always runs in the row sweep.
cudaError_t launch_step_mixed(const StepArgs64& A, int grid, int planes, cudaStream_t st) {
  cudaError_t e = prepare_step_mixed();
  if (e != cudaSuccess) return e;
  if (planes && !A.gate) {
    if (A.P.contact)
      hydro_step_mixed_planes_kernel<true><<<grid, kThreadsPl, kPlaneSmemBytes, st>>>(A);
    else
      hydro_step_mixed_planes_kernel<false><<<grid, kThreadsPl, kPlaneSmemBytes, st>>>(A);
  } else if (A.gate) {
    hydro_step_mixed_kernel<true><<<grid, kThreadsMx, step_mixed_smem_bytes(), st>>>(A);
  } else if (A.P.contact) {
    hydro_step_mixed_kernel<false, true><<<grid, kThreadsMx, step_mixed_smem_bytes(), st>>>(A);
  } else {
    hydro_step_mixed_kernel<false><<<grid, kThreadsMx, step_mixed_smem_bytes(), st>>>(A);
  }
  return cudaGetLastError();
}

}  // namespace hyd
