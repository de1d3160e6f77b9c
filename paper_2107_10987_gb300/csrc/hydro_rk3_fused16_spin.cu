// hydro_rk3_fused16_spin.cu -- the fused RK3 step's instances with the spin
// feedback for 16^3 sub-grids.
#include "hydro_rk3_fused.cuh"

namespace hyd {

cudaError_t prepare_rk3_fused16_spin(int num_sms, int planes, int* max_grid) {
  return prepare_fused_nn<16, true>(num_sms, planes, max_grid);
}

cudaError_t launch_rk3_fused16_spin(const StepArgs64& S, double* Y, double* U2, float* prims, double* dt_out,
                                    unsigned* sync, int nbx, int nby, int nbz, int bc, double cfl, double eta2,
                                    double gamma, int num_sms, int planes, cudaStream_t st) {
  return launch_fused_nn<16, true>(S, Y, U2, prims, dt_out, sync, nbx, nby, nbz, bc, cfl, eta2, gamma, num_sms,
                                   planes, st);
}

}  // namespace hyd
