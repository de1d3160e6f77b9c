// hydro_rk3_fused_spin.cu -- the fused RK3 step's instances with the spin
// feedback (hydro_mode_t.spin) for 8^3 sub-grids, and the dispatch by size
// (translation units of their own, so that the plain instances carry none
// of it and everything compiles in parallel).
#include "hydro_rk3_fused.cuh"

namespace hyd {

cudaError_t prepare_rk3_fused16_spin(int num_sms, int planes, int* max_grid);
cudaError_t launch_rk3_fused16_spin(const StepArgs64& S, double* Y, double* U2, float* prims, double* dt_out,
                                    unsigned* sync, int nbx, int nby, int nbz, int bc, double cfl, double eta2,
                                    double gamma, int num_sms, int planes, cudaStream_t st);

cudaError_t prepare_rk3_fused_spin(int num_sms, int planes, int nn, int* max_grid) {
  return nn == 16 ? prepare_rk3_fused16_spin(num_sms, planes, max_grid)
                  : prepare_fused_nn<8, true>(num_sms, planes, max_grid);
}

cudaError_t launch_rk3_fused_spin(const StepArgs64& S, double* Y, double* U2, float* prims, double* dt_out,
                                  unsigned* sync, int nbx, int nby, int nbz, int bc, double cfl, double eta2,
                                  double gamma, int num_sms, int planes, int nn, cudaStream_t st) {
  if (nn == 16)
    return launch_rk3_fused16_spin(S, Y, U2, prims, dt_out, sync, nbx, nby, nbz, bc, cfl, eta2, gamma, num_sms,
                                   planes, st);
  return launch_fused_nn<8, true>(S, Y, U2, prims, dt_out, sync, nbx, nby, nbz, bc, cfl, eta2, gamma, num_sms,
                                  planes, st);
}

}  // namespace hyd
