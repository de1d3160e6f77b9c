// hydro_step_mixed_amr.cu -- the mixed-precision row sweep over the leaves of
// an adaptive mesh (8^3 leaves) with a tile loader that reads each ghost cell
// where it lives, so that the ghost fill need not copy or restrict
// (hydro_fill_ghosts_amr_lean):
//   - held by a leaf of the same level (the leaf itself included, where the
//     outflow boundary clamps the position into it): that leaf's interior
//     cell;
//   - over a refined position: the restriction image of the finer leaf
//     holding its eight children (hydro_amr_restrict_kernel);
//   - inside a coarser leaf: the leaf's own ghost cell, which the
//     prolongation wrote.
// Each is the value the two-pass fill would have written into that ghost
// cell, so dU/dt, amax and the boundary faces are those of hydro_step after
// hydro_fill_ghosts_amr, bit for bit.
#include "hydro_amr.cuh"
#include "hydro_step_mixed.cuh"

namespace hyd {

struct AmrStepIo {
  using T = Tile<N>;
  static constexpr bool kPrims = false;
  const StepArgs64& A;
  const AMRArgs& M;
  struct Sub {
    T t;
    LevelRef L, Lf;   // the tables of the leaf's level and the next finer one
    int bx, by, bz;   // the global cell (at that level) of its first interior cell
  };
  // s: the leaf (one tile per 8^3 leaf)
  __device__ __forceinline__ Sub begin(int s) const {
    const T t(s);
    const int l = M.leaf_level[t.s];
    return Sub{t, level_ref(M, l), level_ref(M, l + 1), M.leaf_ijk[3 * t.s] * N, M.leaf_ijk[3 * t.s + 1] * N,
               M.leaf_ijk[3 * t.s + 2] * N};
  }
  __device__ __forceinline__ int sidx(const Sub& q) const { return q.t.s; }
  __device__ __forceinline__ int offx(const Sub& q) const { return q.t.o[0]; }
  __device__ __forceinline__ int offy(const Sub& q) const { return q.t.o[1]; }
  __device__ __forceinline__ void load(const Sub& q, int c, double u[F]) const { load_fields(q, c, 0, F, u); }
  __device__ __forceinline__ void load_fields(const Sub& q, int c, int f0, int nf, double* u) const {
    const int lx = c % S - G, ly = (c / S) % S - G, lz = c / (S * S) - G;
    const double* p = A.U + (size_t)q.t.s * F * S3 + c;
    size_t st = S3;
    if (!((unsigned)lx < (unsigned)N && (unsigned)ly < (unsigned)N && (unsigned)lz < (unsigned)N)) {
      const int n = N * q.L.n;
      size_t sd;
      const double* r = amr_source<N>(M, q.L, q.Lf, bc_amr(q.bx + lx, n, M.bc), bc_amr(q.by + ly, n, M.bc),
                                      bc_amr(q.bz + lz, n, M.bc), sd);
      if (r) {
        p = r;
        st = sd;
      }
    }
#pragma unroll
    for (int k = 0; k < nf; ++k) u[k] = __ldg(p + (size_t)(f0 + k) * st);
  }
  // only the fields the sources read (rho, s, z_x, z_y)
  __device__ __forceinline__ void own(const Sub& q, int, int uc, double u[F]) const {
    const double* __restrict__ Us = A.U + (size_t)q.t.s * F * S3 + uc;
#pragma unroll
    for (int k = 0; k < F; ++k) u[k] = (k <= SZ || k == ZX || k == ZY) ? __ldg(Us + (size_t)k * S3) : 0.0;
  }
  __device__ __forceinline__ void store(const Sub& q, int c, int, const double du[F], const double*) const {
    double* dU = A.dUdt + (size_t)q.t.s * F * N3 + c;
#pragma unroll
    for (int k = 0; k < F; ++k) dU[(size_t)k * N3] = du[k];
  }
  __device__ __forceinline__ void grav(const Sub& q, int c, double& gx, double& gy, double& gz) const {
    const double* gs = A.g + (size_t)q.t.s * 3 * N3 + c;
    gx = gs[0];
    gy = gs[N3];
    gz = gs[2 * N3];
  }
  __device__ __forceinline__ void face(const Sub& q, int f, int k, int pc, int pb, double v) const {
    A.face_flux[q.t.face(f, k, pc, pb)] = v;
  }
  __device__ __forceinline__ void amax(const Sub& q, double m) const { A.amax[q.t.s] = m; }
};

// kGate: the learned smoothness indicator is on (A.gate).
template <bool kGate>
__global__ void __launch_bounds__(kThreadsMx, 2) hydro_step_mixed_amr_kernel(StepArgs64 A, AMRArgs M) {
  extern __shared__ __align__(128) float Qf[];  // [F][S3] FP32 primitives, then [2][S3] smooth flags
  __shared__ float red[kThreadsMx / 32];
  double* __restrict__ D = A.scratch + (size_t)blockIdx.x * kScratchPerSub;
  const RowMap R = row_map(threadIdx.x);
  const AmrStepIo io{A, M};
  for (int u = blockIdx.x; u < A.n_sub; u += gridDim.x) {
    const int s = leaf_at(M, u);  // the same for the whole CTA
    if (s >= 0) mixed_subgrid<kGate>(A, io, s, R, Qf, red, D);
  }
}

cudaError_t prepare_step_mixed_amr() {
  static unsigned long long done = 0;
  return once_per_device(&done, [] {
    const cudaFuncAttribute at = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaError_t e = cudaFuncSetAttribute(hydro_step_mixed_amr_kernel<false>, at, (int)kMixedSmemBytes);
    return e == cudaSuccess ? cudaFuncSetAttribute(hydro_step_mixed_amr_kernel<true>, at, (int)kMixedSmemBytes) : e;
  });
}

// grid: persistent CTAs (two per SM by default, as the row sweep of
// hydro_step); the leaves' dU/dt, amax and boundary faces (A.face_flux).
cudaError_t launch_step_mixed_amr(const StepArgs64& A, const AMRArgs& M, int grid, cudaStream_t st) {
  cudaError_t e = prepare_step_mixed_amr();
  if (e != cudaSuccess) return e;
  if (A.gate)
    hydro_step_mixed_amr_kernel<true><<<grid, kThreadsMx, kMixedSmemBytes, st>>>(A, M);
  else
    hydro_step_mixed_amr_kernel<false><<<grid, kThreadsMx, kMixedSmemBytes, st>>>(A, M);
  return cudaGetLastError();
}

}  // namespace hyd
