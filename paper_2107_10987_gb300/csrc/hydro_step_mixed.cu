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
#include "hydro_common.cuh"

namespace hyd {

__device__ __forceinline__ float slope32(float a, float b) {
  const float m = fminf(fminf(2.f * fabsf(a), 2.f * fabsf(b)), 0.5f * fabsf(a + b));
  return (a * b <= 0.f) ? 0.f : copysignf(m, b);
}

// PPM on one line in FP32 (branch-free form of the same limiter).
__device__ __forceinline__ void ppm32(float s0, float s1, float s2, float s3, float s4, float& qp, float& qm) {
  const float sixth = 1.f / 6.f;
  const float D0 = slope32(s1 - s0, s2 - s1), D1 = slope32(s2 - s1, s3 - s2), D2 = slope32(s3 - s2, s4 - s3);
  const float p = 0.5f * (s2 + s3) - (D2 - D1) * sixth;
  const float m = 0.5f * (s1 + s2) - (D1 - D0) * sixth;
  const bool ext = (p - s2) * (s2 - m) <= 0.f;
  const float dq = p - m;
  const float lhs = dq * (s2 - 0.5f * (p + m));
  const float rhs = dq * dq * sixth;
  const float m2 = (lhs > rhs) ? 3.f * s2 - 2.f * p : m;
  const float p2 = (lhs < -rhs) ? 3.f * s2 - 2.f * m : p;
  qp = ext ? s2 : p2;
  qm = ext ? s2 : m2;
}

__device__ __forceinline__ void line10f(const float* __restrict__ Q, int c, int st, float qp[F], float qm[F]) {
#pragma unroll
  for (int k = 0; k < F; ++k) {
    const float* q = Q + k * S3 + c;
    ppm32(q[-2 * st], q[-st], q[0], q[st], q[2 * st], qp[k], qm[k]);
  }
}

struct StepParamsF {
  float gamma, gm1, omega;
};

__device__ __forceinline__ void side32(const float q[F], int a, float xq, float yq, const StepParamsF& P, float U[F],
                                       float Fl[F], float& spd) {
  const float rho = q[RHO], vx = q[1], vy = q[2], vz = q[3], eps = q[4];
  const float ek = (0.5f * rho) * (vx * vx + vy * vy + vz * vz);
  const float E = eps + ek;
  const float p = P.gm1 * eps;
  const float c2 = __fdividef(P.gamma * p, rho);
  const float c = c2 * rsqrtf(c2);
  const float ux = vx + P.omega * yq, uy = vy - P.omega * xq;
  const float un = (a == 0) ? ux : (a == 1) ? uy : vz;
  const float va = (a == 0) ? vx : (a == 1) ? vy : vz;
  U[RHO] = rho;
  U[SX] = rho * vx;
  U[SY] = rho * vy;
  U[SZ] = rho * vz;
  U[EGAS] = E;
#pragma unroll
  for (int k = TAU; k < F; ++k) U[k] = q[k];
#pragma unroll
  for (int k = 0; k < F; ++k) Fl[k] = U[k] * un;
  Fl[SX + a] += p;
  Fl[EGAS] += p * va;
  spd = fabsf(un) + c;
}

__device__ __forceinline__ void point32(const float qL[F], const float qR[F], int a, float xq, float yq, float w,
                                        const float rl[3], const float rr[3], const StepParamsF& P, float fsum[F],
                                        float tl[3], float tr[3], float& amax) {
  float UL[F], FL[F], UR[F], FR[F], sL, sR;
  side32(qL, a, xq, yq, P, UL, FL, sL);
  side32(qR, a, xq, yq, P, UR, FR, sR);
  const float aq = fmaxf(sL, sR);
  amax = fmaxf(amax, aq);
  float Fq[F];
#pragma unroll
  for (int k = 0; k < F; ++k) {
    Fq[k] = 0.5f * (FL[k] + FR[k]) - (0.5f * aq) * (UR[k] - UL[k]);
    fsum[k] += w * Fq[k];
  }
  const float fx = Fq[SX], fy = Fq[SY], fz = Fq[SZ];
  tl[0] += w * (rl[1] * fz - rl[2] * fy);
  tl[1] += w * (rl[2] * fx - rl[0] * fz);
  tl[2] += w * (rl[0] * fy - rl[1] * fx);
  tr[0] += w * (rr[1] * fz - rr[2] * fy);
  tr[1] += w * (rr[2] * fx - rr[0] * fz);
  tr[2] += w * (rr[0] * fy - rr[1] * fx);
}

constexpr int kThreadsMx = NROW;  // 192

__global__ void __launch_bounds__(kThreadsMx, 2) hydro_step_mixed_kernel(StepArgs64 A) {
  extern __shared__ __align__(128) float Qf[];  // [F][S3] FP32 primitives
  __shared__ float red[kThreadsMx / 32];
  const int tid = threadIdx.x;
  double* __restrict__ D = A.scratch + (size_t)blockIdx.x * kScratchPerSub;
  const StepParamsF PF{(float)A.P.gamma, (float)A.P.gm1, (float)A.P.omega};

  const int a = tid / (N * N);
  const int r = tid % (N * N);
  const int pb = r % N, pc = r / N;
  const int b = (a == 0) ? 1 : 0;
  const int cx = (a == 2) ? 1 : 2;
  const int st[3] = {1, S, S * S};
  const int sa = st[a], sb = st[b], sc = st[cx];

  for (int s = blockIdx.x; s < A.n_sub; s += gridDim.x) {
    // ---- 1-2. load the FP64 state, recover primitives, store FP32 -------
    const double* __restrict__ Us = A.U + (size_t)s * F * S3;
    bool bad = false;
    for (int c = tid; c < S3; c += kThreadsMx) {
      double u[F];
#pragma unroll
      for (int k = 0; k < F; ++k) u[k] = __ldg(Us + (size_t)k * S3 + c);
      const double rho = u[RHO];
      // 1/rho: FP32 reciprocal refined by one Newton step in FP64 (rel. err ~1e-14)
      const double r0 = (double)__frcp_rn((float)rho);
      const double ri = r0 * fma(-rho, r0, 2.0);
      const double s2 = fma(u[SZ], u[SZ], fma(u[SY], u[SY], u[SX] * u[SX]));
      const double ek = 0.5 * s2 * ri;
      const double eE = u[EGAS] - ek;  // FP64: the cancellation the dual energy guards
      const float rif = (float)ri;
      const float eps = (eE > A.P.eta1 * u[EGAS]) ? (float)eE : __powf((float)u[TAU], PF.gamma);
      Qf[RHO * S3 + c] = (float)rho;
      Qf[SX * S3 + c] = (float)u[SX] * rif;
      Qf[SY * S3 + c] = (float)u[SY] * rif;
      Qf[SZ * S3 + c] = (float)u[SZ] * rif;
      Qf[EGAS * S3 + c] = eps;
#pragma unroll
      for (int k = TAU; k < F; ++k) Qf[k * S3 + c] = (float)u[k];
      bad |= !(rho > 0.0) || !(eps > 0.f);
    }
    if (bad) atomicOr(A.status, 1u);
    __syncthreads();

    // ---- 3. row sweep in FP32 --------------------------------------------
    const double hd = A.h[s];
    const float h = (float)hd, half_h = 0.5f * h;
    const double o[3] = {A.origin[3 * s + 0], A.origin[3 * s + 1], A.origin[3 * s + 2]};
    float amax = 0.f;
    float plus[9][F];
    float fprev[F], trprev[3];
    int coord0[3];
    coord0[a] = 0;
    coord0[b] = pb;
    coord0[cx] = pc;
    const int c0 = ((coord0[2] + G) * S + (coord0[1] + G)) * S + (coord0[0] + G);
#pragma unroll 1
    for (int j = -1; j <= N; ++j) {
      const int cj = c0 + j * sa;
      float fsum[F], tl[3], tr[3];
#pragma unroll
      for (int k = 0; k < F; ++k) fsum[k] = 0.f;
      tl[0] = tl[1] = tl[2] = 0.f;
      tr[0] = tr[1] = tr[2] = 0.f;
      int ci[3];
      ci[a] = j - 1;
      ci[b] = pb;
      ci[cx] = pc;
      // cell-centre coordinates of the left cell (FP64 -> FP32 once)
      const float xc = (float)(o[0] + hd * (ci[0] + 0.5)), yc = (float)(o[1] + hd * (ci[1] + 0.5));
#pragma unroll 1
      for (int p = 0; p <= 4; ++p) {
        const int t1 = p / 3 - 1, t2 = p % 3 - 1;
        float qpA[F], qmA[F], qpB[F], qmB[F];
        line10f(Qf, cj, sa + t1 * sb + t2 * sc, qpA, qmA);
        if (p != 4) line10f(Qf, cj, sa - t1 * sb - t2 * sc, qpB, qmB);
        if (j >= 0) {
#pragma unroll 1
          for (int side = 0; side < 2; ++side) {
            if (p == 4 && side == 1) continue;
            const int u1 = side ? t1 : -t1, u2 = side ? t2 : -t2;
            const int pt = (u1 + 1) * 3 + (u2 + 1);
            int d[3];
            d[a] = 1;
            d[b] = u1;
            d[cx] = u2;
            const float xq = xc + half_h * d[0];
            const float yq = yc + half_h * d[1];
            const float rl[3] = {half_h * d[0], half_h * d[1], half_h * d[2]};
            float rr[3] = {rl[0], rl[1], rl[2]};
            rr[a] = -half_h;
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
      if (j >= 1) {
        const int i = j - 1;
        int cc[3];
        cc[a] = i;
        cc[b] = pb;
        cc[cx] = pc;
        const int cell = (cc[2] * N + cc[1]) * N + cc[0];
        double* Da = D + (size_t)a * DQ * N3 + cell;
#pragma unroll
        for (int k = 0; k < F; ++k) Da[k * N3] = (double)fsum[k] - (double)fprev[k];
#pragma unroll
        for (int m = 0; m < 3; ++m) Da[(F + m) * N3] = (double)tl[m] - (double)trprev[m];
      }
      if (j >= 0) {
#pragma unroll
        for (int k = 0; k < F; ++k) fprev[k] = fsum[k];
        trprev[0] = tr[0];
        trprev[1] = tr[1];
        trprev[2] = tr[2];
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

size_t step_mixed_smem_bytes() { return (size_t)F * S3 * sizeof(float); }

// Opt in to the kernel's dynamic shared memory once per process (no
// allocation; call before any stream capture).
cudaError_t prepare_step_mixed() {
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(hydro_step_mixed_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)step_mixed_smem_bytes());
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  return cudaSuccess;
}

cudaError_t launch_step_mixed(const StepArgs64& A, int grid, cudaStream_t st) {
  cudaError_t e = prepare_step_mixed();
  if (e != cudaSuccess) return e;
  hydro_step_mixed_kernel<<<grid, kThreadsMx, step_mixed_smem_bytes(), st>>>(A);
  return cudaGetLastError();
}

}  // namespace hyd
