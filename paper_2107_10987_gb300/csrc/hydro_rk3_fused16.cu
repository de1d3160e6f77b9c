// hydro_rk3_fused16.cu -- the fused RK3 step for 16^3 sub-grids (each work
// unit an 8^3 octant tile; a translation unit of its own so that the two
// sizes compile in parallel).
#include "hydro_rk3_fused.cuh"

namespace hyd {

cudaError_t prepare_rk3_fused16(int num_sms, int planes, int* max_grid) {
  return prepare_fused_nn<16>(num_sms, planes, max_grid);
}

cudaError_t launch_rk3_fused16(const StepArgs64& S, double* Y, double* U2, float* prims, double* dt_out,
                               unsigned* sync, int nbx, int nby, int nbz, int bc, double cfl, double eta2,
                               double gamma, int num_sms, int planes, cudaStream_t st) {
  return launch_fused_nn<16>(S, Y, U2, prims, dt_out, sync, nbx, nby, nbz, bc, cfl, eta2, gamma, num_sms, planes,
                             st);
}

}  // namespace hyd
