// hydro_step_mixed_spin.cu -- the mixed-precision step kernels with the spin
// feedback (hydro_mode_t.spin): a translation unit of their own, so that the
// plain instances carry none of it and both compile in parallel.
#include "hydro_step_mixed.cuh"

namespace hyd {

cudaError_t prepare_step_mixed_spin() {
  static unsigned long long done = 0;
  return once_per_device(&done, [] {
    cudaError_t e = mixed_attrs<8, true>();
    return e == cudaSuccess ? mixed_attrs<16, true>() : e;
  });
}

// As launch_step_mixed (the 16^3 amax cleared by the caller).
void launch_step_mixed_spin(const StepArgs64& A, int grid, int planes, int nn, cudaStream_t st) {
  if (nn == 16)
    launch_mixed_nn<16, true>(A, grid, planes, st);
  else
    launch_mixed_nn<8, true>(A, grid, planes, st);
}

}  // namespace hyd
