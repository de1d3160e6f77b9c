// hydro_mixed.cuh -- FP32 device functions of the mixed-precision path,
// shared by the step kernel and the smoothness-indicator kernels.
#pragma once
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

// Unlimited interface value towards +d (the 4-point formula the PPM
// interface value reduces to when no limiter acts): used on cells the
// learned indicator marks smooth.
__device__ __forceinline__ void unlimited32(float s0, float s1, float s2, float s3, float s4, float& qp, float& qm) {
  qp = (7.f / 12.f) * (s2 + s3) - (1.f / 12.f) * (s1 + s4);
  qm = (7.f / 12.f) * (s1 + s2) - (1.f / 12.f) * (s0 + s3);
}

// Lines of a cell the indicator marks smooth: the unlimited formula for all
// fields but the spin, which stays limited.
__device__ __forceinline__ void line10u(const float* __restrict__ Q, int c, int st, float qp[F], float qm[F]) {
#pragma unroll
  for (int k = 0; k < F; ++k) {
    const float* q = Q + k * S3 + c;
    if (k == ZX || k == ZY || k == ZZ)
      ppm32(q[-2 * st], q[-st], q[0], q[st], q[2 * st], qp[k], qm[k]);
    else
      unlimited32(q[-2 * st], q[-st], q[0], q[st], q[2 * st], qp[k], qm[k]);
  }
}

// Primitive recovery of one cell for the mixed form: eps_E = E - |s|^2/(2 rho)
// and its dual-energy selection in FP64, everything else rounded to FP32.
// Returns false for a non-physical cell.
__device__ __forceinline__ bool prims_mixed(const double u[F], double eta1, float gamma, float q[F]) {
  const double rho = u[RHO];
  const double r0 = (double)__frcp_rn((float)rho);
  const double ri = r0 * fma(-rho, r0, 2.0);
  const double s2 = fma(u[SZ], u[SZ], fma(u[SY], u[SY], u[SX] * u[SX]));
  const double eE = u[EGAS] - 0.5 * s2 * ri;
  const float rif = (float)ri;
  const float eps = (eE > eta1 * u[EGAS]) ? (float)eE : __powf((float)u[TAU], gamma);
  q[RHO] = (float)rho;
  q[SX] = (float)u[SX] * rif;
  q[SY] = (float)u[SY] * rif;
  q[SZ] = (float)u[SZ] * rif;
  q[EGAS] = eps;
#pragma unroll
  for (int k = TAU; k < F; ++k) q[k] = (float)u[k];
  return (rho > 0.0) && (eps > 0.f);
}

// Indicator features of cell c (54: density then pressure over the 3x3x3
// neighbourhood in (z, y, x) order): (q_k - q_c) / (|q_k| + |q_c|).
__device__ __forceinline__ void gate_features(const float* __restrict__ Q, int c, float gm1, float x[54]) {
  const float rc = Q[RHO * S3 + c], pc = gm1 * Q[EGAS * S3 + c];
  int j = 0;
#pragma unroll
  for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx, ++j) {
        const int ck = c + (dz * S + dy) * S + dx;
        const float rk = Q[RHO * S3 + ck], pk = gm1 * Q[EGAS * S3 + ck];
        x[j] = __fdividef(rk - rc, fabsf(rk) + fabsf(rc));
        x[27 + j] = __fdividef(pk - pc, fabsf(pk) + fabsf(pc));
      }
}

// Indicator network: 54 -> 32 (ReLU) -> 32 (ReLU) -> 1 (logit).  Parameters
// packed W1[32][54], b1[32], W2[32][32], b2[32], w3[32], b3.
constexpr int kGateIn = 54, kGateH = 32;
constexpr int kGateParams = kGateH * kGateIn + kGateH + kGateH * kGateH + kGateH + kGateH + 1;  // 2849

template <class W>
__device__ __forceinline__ float gate_logit(const W& w, const float x[54]) {
  float h1[kGateH];
#pragma unroll
  for (int j = 0; j < kGateH; ++j) {
    float z = w(kGateH * kGateIn + j);
#pragma unroll
    for (int i = 0; i < kGateIn; ++i) z = fmaf(w(j * kGateIn + i), x[i], z);
    h1[j] = fmaxf(z, 0.f);
  }
  const int o2 = kGateH * kGateIn + kGateH;
  float out = w(o2 + kGateH * kGateH + kGateH + kGateH);
#pragma unroll 4
  for (int j = 0; j < kGateH; ++j) {
    float z = w(o2 + kGateH * kGateH + j);
#pragma unroll
    for (int i = 0; i < kGateH; ++i) z = fmaf(w(o2 + j * kGateH + i), h1[i], z);
    out = fmaf(w(o2 + kGateH * kGateH + kGateH + j), fmaxf(z, 0.f), out);
  }
  return out;
}

}  // namespace hyd
