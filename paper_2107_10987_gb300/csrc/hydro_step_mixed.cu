// hydro_step_mixed.cu -- the mixed-precision step kernels without the spin
// feedback, their shared-memory opt-in and the dispatch (with the spin
// feedback: hydro_step_mixed_spin.cu).
#include "hydro_step_mixed.cuh"

namespace hyd {

void launch_step_mixed_spin(const StepArgs64& A, int grid, int planes, int nn, cudaStream_t st);
cudaError_t prepare_step_mixed_spin();
cudaError_t prepare_step_mixed_amr();

size_t step_mixed_smem_bytes() { return kMixedSmemBytes; }

// Opt in to the kernels' dynamic shared memory once per device, with and
// without the spin feedback and for the adaptive mesh's direct loader (no
// allocation; call before any stream capture).
cudaError_t prepare_step_mixed() {
  static unsigned long long done = 0;
  cudaError_t e = once_per_device(&done, [] {
    cudaError_t r = mixed_attrs<8, false>();
    return r == cudaSuccess ? mixed_attrs<16, false>() : r;
  });
  if (e == cudaSuccess) e = prepare_step_mixed_spin();
  return e == cudaSuccess ? prepare_step_mixed_amr() : e;
}

// planes: the plane-sweep decomposition (grid: CTAs, at most one per SM);
// the learned indicator always runs in the row sweep.  nn: the sub-grids'
// edge (8 or 16); the persistent CTAs loop over A.n_sub * (nn/8)^3 tiles,
// and with 16^3 sub-grids the amax of a sub-grid is the atomic maximum over
// its tiles, cleared here first.
cudaError_t launch_step_mixed(const StepArgs64& A, int grid, int planes, int nn, cudaStream_t st) {
  cudaError_t e = prepare_step_mixed();
  if (e != cudaSuccess) return e;
  if (nn == 16) {
    e = cudaMemsetAsync(A.amax, 0, (size_t)A.n_sub * sizeof(double), st);
    if (e != cudaSuccess) return e;
  }
  if (A.P.spin)
    launch_step_mixed_spin(A, grid, planes, nn, st);
  else if (nn == 16)
    launch_mixed_nn<16, false>(A, grid, planes, st);
  else
    launch_mixed_nn<8, false>(A, grid, planes, st);
  return cudaGetLastError();
}

}  // namespace hyd
