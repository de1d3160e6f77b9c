// hydro_step_mixed.cu -- the per-sub-grid hydro step in mixed precision.
//
// Same sweep as the FP64 step (see hydro_step_fp64.cu): PPM on the 13 lines
// through each cell, Kurganov-Tadmor fluxes at the 9 points of every face,
// Simpson face sums, divergence, sources, amax.  Precision split:
//   FP64: the dual-energy internal-energy recovery eps_E = E - |s|^2/(2 rho)
//         and its selection (cancellation between E and the kinetic energy),
//         the per-axis flux differences F(i+1/2) - F(i-1/2) (exact in FP64
//         from FP32 face sums), the divergence accumulation, the sources and
//         the output dU/dt;
//   FP32: primitives in shared memory, PPM, the point fluxes, signal speeds
//         and the face quadrature.
// The primitives are half the size of the FP64 stage, so two CTAs share an
// SM: while one converts its next sub-grid (HBM/L2-bound loads), the other
// sweeps (FP32-bound).  The conversion reads the FP64 state with coalesced
// loads and writes FP32 primitives: a bulk TMA copy cannot convert, and an
// FP64 staging buffer would not fit beside the FP32 primitives of two CTAs.
#include "hydro_mixed.cuh"

namespace hyd {

constexpr int kThreadsMx = NROW;  // 192

// kGate: the learned smoothness indicator is on (A.gate); the kernel without
// it carries none of the indicator's registers.
template <bool kGate>
__global__ void __launch_bounds__(kThreadsMx, 2) hydro_step_mixed_kernel(StepArgs64 A) {
  extern __shared__ __align__(128) float Qf[];  // [F][S3] FP32 primitives, then [S3] smooth flags
  uint8_t* smooth = reinterpret_cast<uint8_t*>(Qf + F * S3);
  __shared__ float red[kThreadsMx / 32];
  const int tid = threadIdx.x;
  double* __restrict__ D = A.scratch + (size_t)blockIdx.x * kScratchPerSub;
  const StepParamsF PF{(float)A.P.gamma, (float)A.P.gm1, (float)A.P.omega};

  const int a = tid / (N * N);
  const int r = tid % (N * N);
  const int pb = r % N, pc = r / N;
  const int b = (a == 0) ? 1 : 0;
  const int cx = (a == 2) ? 1 : 2;
  const int sa = axis_stride(a), sb = axis_stride(b), sc = axis_stride(cx);

  for (int s = blockIdx.x; s < A.n_sub; s += gridDim.x) {
    // ---- 1-2. load the FP64 state, recover primitives, store FP32 -------
    const double* __restrict__ Us = A.U + (size_t)s * F * S3;
    bool bad = false;
    for (int c = tid; c < S3; c += kThreadsMx) {
      double u[F];
#pragma unroll
      for (int k = 0; k < F; ++k) u[k] = __ldg(Us + (size_t)k * S3 + c);
      float q[F];
      bad |= !prims_mixed(u, A.P.eta1, PF.gamma, q);
#pragma unroll
      for (int k = 0; k < F; ++k) Qf[k * S3 + c] = q[k];
    }
    if (bad) atomicOr(A.status, 1u);
    __syncthreads();

    // ---- 2b. learned smoothness indicator (gate_phase) ---------------------
    if (kGate)
      gate_phase<float, kThreadsMx>(Qf, PF.gm1, A.gate_w, A.gate_logit_thr, A.gate_zero_smooth, smooth, smooth + S3);

    // ---- 3. row sweep in FP32 --------------------------------------------
    const double hd = A.h[s];
    const float h = (float)hd, half_h = 0.5f * h;
    const double o[3] = {A.origin[3 * s + 0], A.origin[3 * s + 1], A.origin[3 * s + 2]};
    float amax = 0.f;
    float plus[9][F];
    // the previous face's FP32 sums (their FP64 values are these converted: exact)
    float fprev[F], trprev[3];
    const int c0 = ((axis_comp(2, a, b, 0, pb, pc) + G) * S + (axis_comp(1, a, b, 0, pb, pc) + G)) * S +
                   (axis_comp(0, a, b, 0, pb, pc) + G);
#pragma unroll 1
    for (int j = -1; j <= N; ++j) {
      const int cj = c0 + j * sa;
      float fsum[F], tl[3], tr[3];
#pragma unroll
      for (int k = 0; k < F; ++k) fsum[k] = 0.f;
      tl[0] = tl[1] = tl[2] = 0.f;
      tr[0] = tr[1] = tr[2] = 0.f;
      // cell-centre coordinates of the left cell j - 1 (FP64 -> FP32 once)
      const float xc = (float)(o[0] + hd * (axis_comp(0, a, b, j - 1, pb, pc) + 0.5)),
                  yc = (float)(o[1] + hd * (axis_comp(1, a, b, j - 1, pb, pc) + 0.5));
#pragma unroll 1
      for (int p = 0; p <= 4; ++p) {
        const int t1 = p / 3 - 1, t2 = p % 3 - 1;
        float qpA[F], qmA[F], qpB[F], qmB[F];
        if (kGate && smooth[cj]) {
          line10u(Qf, cj, sa + t1 * sb + t2 * sc, qpA, qmA);
          if (p != 4) line10u(Qf, cj, sa - t1 * sb - t2 * sc, qpB, qmB);
        } else {
          line10f(Qf, cj, sa + t1 * sb + t2 * sc, qpA, qmA);
          if (p != 4) line10f(Qf, cj, sa - t1 * sb - t2 * sc, qpB, qmB);
        }
        if (j >= 0) {
#pragma unroll 1
          for (int side = 0; side < 2; ++side) {
            if (p == 4 && side == 1) continue;
            const int u1 = side ? t1 : -t1, u2 = side ? t2 : -t2;
            const int pt = (u1 + 1) * 3 + (u2 + 1);
            const int d0 = axis_comp(0, a, b, 1, u1, u2), d1 = axis_comp(1, a, b, 1, u1, u2),
                      d2 = axis_comp(2, a, b, 1, u1, u2);
            const float xq = xc + half_h * d0;
            const float yq = yc + half_h * d1;
            const float rl[3] = {half_h * d0, half_h * d1, half_h * d2};
            const float rr[3] = {a == 0 ? -half_h : rl[0], a == 1 ? -half_h : rl[1], a == 2 ? -half_h : rl[2]};
            const float w = (u1 == 0 && u2 == 0) ? (16.f / 36.f) : (u1 == 0 || u2 == 0) ? (4.f / 36.f) : (1.f / 36.f);
            point32(plus[pt], side ? qmB : qmA, a, xq, yq, w, rl, rr, PF, fsum, tl, tr, amax);
          }
        }
#pragma unroll
        for (int k = 0; k < F; ++k) {
          plus[p][k] = qpA[k];
          if (p != 4) plus[8 - p][k] = qpB[k];
        }
      }
      if (j >= 0) {
        // face j-1/2 is complete: its sums in FP64 (each converted once); the
        // a-difference of cell j-1 is exact in FP64
        double fd[F], tld[3];
#pragma unroll
        for (int k = 0; k < F; ++k) fd[k] = (double)fsum[k];
#pragma unroll
        for (int m = 0; m < 3; ++m) tld[m] = (double)tl[m];
        if (j >= 1) {
          const int cell = (axis_comp(2, a, b, j - 1, pb, pc) * N + axis_comp(1, a, b, j - 1, pb, pc)) * N +
                           axis_comp(0, a, b, j - 1, pb, pc);
          double* Da = D + (size_t)a * DQ * N3 + cell;
#pragma unroll
          for (int k = 0; k < F; ++k) Da[k * N3] = fd[k] - (double)fprev[k];
#pragma unroll
          for (int m = 0; m < 3; ++m) Da[(F + m) * N3] = tld[m] - (double)trprev[m];
        }
#pragma unroll
        for (int k = 0; k < F; ++k) fprev[k] = fsum[k];
#pragma unroll
        for (int m = 0; m < 3; ++m) trprev[m] = tr[m];
        if (A.face_flux && (j == 0 || j == N)) {
          // sub-grid boundary face: sums and the torque about the interior cell
          const int f = 2 * a + (j == N ? 1 : 0);
#pragma unroll
          for (int k = 0; k < F; ++k) A.face_flux[face_index(s, f, k, pc, pb)] = fd[k];
#pragma unroll
          for (int m = 0; m < 3; ++m) A.face_flux[face_index(s, f, F + m, pc, pb)] = (j == N) ? tld[m] : (double)trprev[m];
        }
      }
    }
#pragma unroll
    for (int o2 = 16; o2 > 0; o2 >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o2));
    if ((tid & 31) == 0) red[tid >> 5] = amax;
    __syncthreads();

    // ---- 4. divergence + sources in FP64 --------------------------------
    const double inv_h = 1.0 / hd;
    const double om = A.P.omega;
    double* dU = A.dUdt + (size_t)s * F * N3;
    for (int c = tid; c < N3; c += kThreadsMx) {
      const int x = c % N, y = (c / N) % N, z = c / (N * N);
      const int uc = ((z + G) * S + (y + G)) * S + (x + G);
      double du[F];
#pragma unroll
      for (int k = 0; k < F; ++k) {
        const double div = (D[(0 * DQ + k) * N3 + c] + D[(1 * DQ + k) * N3 + c]) + D[(2 * DQ + k) * N3 + c];
        du[k] = -(div * inv_h);
      }
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        const double tq =
            (D[(0 * DQ + F + m) * N3 + c] + D[(1 * DQ + F + m) * N3 + c]) + D[(2 * DQ + F + m) * N3 + c];
        du[ZX + m] = du[ZX + m] - tq * inv_h;
      }
      const double sx = Us[SX * S3 + uc], sy = Us[SY * S3 + uc], sz = Us[SZ * S3 + uc];
      du[SX] = du[SX] + om * sy;
      du[SY] = du[SY] - om * sx;
      du[ZX] = du[ZX] + om * Us[ZY * S3 + uc];
      du[ZY] = du[ZY] - om * Us[ZX * S3 + uc];
      {
        // spin source w(x_c) x s, w = -omega z_hat x x_c: removes the torque
        // that the frame part s w_n of the momentum flux leaves in the face
        // torques, so that sum (x_c x s + z)_z is conserved for omega != 0
        const double xc = __dadd_rn(o[0], __dmul_rn(hd, x + 0.5));
        const double yc = __dadd_rn(o[1], __dmul_rn(hd, y + 0.5));
        const double wx = om * yc, wy = -(om * xc);
        du[ZX] = du[ZX] + wy * sz;
        du[ZY] = du[ZY] - wx * sz;
        du[ZZ] = du[ZZ] + (wx * sy - wy * sx);
      }
      if (A.g) {
        const double* gs = A.g + (size_t)s * 3 * N3;
        const double gx = gs[c], gy = gs[N3 + c], gz = gs[2 * N3 + c];
        const double rho = Us[RHO * S3 + uc];
        du[SX] = du[SX] + rho * gx;
        du[SY] = du[SY] + rho * gy;
        du[SZ] = du[SZ] + rho * gz;
        du[EGAS] = du[EGAS] + ((sx * gx + sy * gy) + sz * gz);
      }
#pragma unroll
      for (int k = 0; k < F; ++k) dU[k * N3 + c] = du[k];
    }
    if (tid == 0) {
      float m = red[0];
#pragma unroll
      for (int w = 1; w < kThreadsMx / 32; ++w) m = fmaxf(m, red[w]);
      A.amax[s] = (double)m;
    }
    __syncthreads();
  }
}

size_t step_mixed_smem_bytes() { return (size_t)F * S3 * sizeof(float) + 2 * S3; }

// Opt in to the kernel's dynamic shared memory once per process (no
// allocation; call before any stream capture).
cudaError_t prepare_step_mixed() {
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(hydro_step_mixed_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)step_mixed_smem_bytes());
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(hydro_step_mixed_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)step_mixed_smem_bytes());
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  return cudaSuccess;
}

cudaError_t launch_step_mixed(const StepArgs64& A, int grid, cudaStream_t st) {
  cudaError_t e = prepare_step_mixed();
  if (e != cudaSuccess) return e;
  if (A.gate)
    hydro_step_mixed_kernel<true><<<grid, kThreadsMx, step_mixed_smem_bytes(), st>>>(A);
  else
    hydro_step_mixed_kernel<false><<<grid, kThreadsMx, step_mixed_smem_bytes(), st>>>(A);
  return cudaGetLastError();
}

}  // namespace hyd
