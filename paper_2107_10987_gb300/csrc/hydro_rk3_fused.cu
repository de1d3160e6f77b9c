// hydro_rk3_fused.cu -- the fused RK3 step for 8^3 sub-grids, the dispatch
// by sub-grid size, and the self-test of its bounded wait.
#include "hydro_rk3_fused.cuh"

namespace hyd {

cudaError_t launch_rk3_fused16(const StepArgs64& S, double* Y, double* U2, float* prims, double* dt_out,
                               unsigned* sync, int nbx, int nby, int nbz, int bc, double cfl, double eta2,
                               double gamma, int num_sms, int planes, cudaStream_t st);
cudaError_t prepare_rk3_fused16(int num_sms, int planes, int* max_grid);
cudaError_t launch_rk3_fused_spin(const StepArgs64& S, double* Y, double* U2, float* prims, double* dt_out,
                                  unsigned* sync, int nbx, int nby, int nbz, int bc, double cfl, double eta2,
                                  double gamma, int num_sms, int planes, int nn, cudaStream_t st);
cudaError_t prepare_rk3_fused_spin(int num_sms, int planes, int nn, int* max_grid);

// Self-test of the bounded wait: thread 0 waits on a flag that nothing sets
// (flag[0], abort flag[1], both zero) and reports the expiry in the status
// word, as the fused step does.
__global__ void hydro_wait_selftest_kernel(const unsigned* flag, unsigned* status, long long limit_ns) {
  if (threadIdx.x == 0 && !wait_geq(flag, 1u, flag + 1, limit_ns)) atomicOr(status, 2u);
}

cudaError_t launch_wait_selftest(unsigned* words, unsigned* status, long long limit_ns, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(words, 0, 2 * sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  hydro_wait_selftest_kernel<<<1, 32, 0, st>>>(words, status, limit_ns);
  return cudaGetLastError();
}

size_t rk3_fused_sync_words(int n_sub) { return (size_t)kSyncHead + 2 * (size_t)n_sub; }

// Both the plain instances and those with the spin feedback (once per
// device), so that a capture finds either ready; *max_grid for the plain ones.
cudaError_t prepare_rk3_fused(int num_sms, int planes, int nn, int* max_grid) {
  int spin_grid = 0;
  cudaError_t e = prepare_rk3_fused_spin(num_sms, planes, nn, &spin_grid);
  if (e != cudaSuccess) return e;
  return nn == 16 ? prepare_rk3_fused16(num_sms, planes, max_grid) : prepare_fused_nn<8>(num_sms, planes, max_grid);
}

// nn: the sub-grids' edge (8 or 16).
cudaError_t launch_rk3_fused(const StepArgs64& S, double* Y, double* U2, float* prims, double* dt_out,
                             unsigned* sync, int nbx, int nby, int nbz, int bc, double cfl, double eta2,
                             double gamma, int num_sms, int planes, int nn, cudaStream_t st) {
  if (S.P.spin)
    return launch_rk3_fused_spin(S, Y, U2, prims, dt_out, sync, nbx, nby, nbz, bc, cfl, eta2, gamma, num_sms,
                                 planes, nn, st);
  if (nn == 16)
    return launch_rk3_fused16(S, Y, U2, prims, dt_out, sync, nbx, nby, nbz, bc, cfl, eta2, gamma, num_sms,
                              planes, st);
  return launch_fused_nn<8>(S, Y, U2, prims, dt_out, sync, nbx, nby, nbz, bc, cfl, eta2, gamma, num_sms, planes,
                            st);
}

}  // namespace hyd
