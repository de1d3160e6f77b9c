// hydro_mixed.cuh -- FP32 device functions of the mixed-precision path,
// shared by the step kernel and the smoothness-indicator kernels.
#pragma once
#include <cuda_bf16.h>

#include "hydro_common.cuh"

namespace hyd {

// ---- PPM on one line, FP32 ------------------------------------------------
// Every operation below is written out as an explicitly rounded or fused
// intrinsic, for two reasons: every kernel that inlines these functions then
// computes the same bits (the compiler has no contraction left to choose),
// and the line operator is exactly symmetric under reversal of the line --
// ppm32 on (s4, s3, s2, s1, s0) returns (qm, qp) of ppm32 on (s0, ..., s4)
// bit for bit -- so a line may be evaluated in either orientation.
// (Negation, |x|, min, 2x and x/2 are exact; a + b, a - b, a*b and fma round
// symmetrically.)

// MC slope of two one-sided differences: 0 where they differ in sign, else
// the sign of b times min(2|a|, 2|b|, |a + b|/2).
__device__ __forceinline__ float slope32(float a, float b) {
  const float m = fminf(__fmul_rn(2.f, fminf(fabsf(a), fabsf(b))), __fmul_rn(0.5f, fabsf(__fadd_rn(a, b))));
  return (__fmul_rn(a, b) <= 0.f) ? 0.f : copysignf(m, b);
}

// PPM on one line in FP32 (branch-free form of the limiter).  kSteep: the
// contact-steepening blend with weight eta before the fix-ups (as ppm64).
template <bool kSteep = false>
__device__ __forceinline__ void ppm32(float s0, float s1, float s2, float s3, float s4, float& qp, float& qm,
                                      float eta = 0.f) {
  const float sixth = 1.f / 6.f;
  const float d0 = __fsub_rn(s1, s0), d1 = __fsub_rn(s2, s1), d2 = __fsub_rn(s3, s2), d3 = __fsub_rn(s4, s3);
  const float D0 = slope32(d0, d1), D1 = slope32(d1, d2), D2 = slope32(d2, d3);
  float p = __fmaf_rn(-sixth, __fsub_rn(D2, D1), __fmul_rn(0.5f, __fadd_rn(s2, s3)));
  float m = __fmaf_rn(-sixth, __fsub_rn(D1, D0), __fmul_rn(0.5f, __fadd_rn(s1, s2)));
  if (kSteep) {
    const float keep = __fsub_rn(1.f, eta);
    p = __fmaf_rn(eta, __fmaf_rn(-0.5f, D2, s3), __fmul_rn(keep, p));
    m = __fmaf_rn(eta, __fmaf_rn(0.5f, D0, s1), __fmul_rn(keep, m));
  }
  const bool ext = __fmul_rn(__fsub_rn(p, s2), __fsub_rn(s2, m)) <= 0.f;
  const float dq = __fsub_rn(p, m);
  const float lhs = __fmul_rn(dq, __fmaf_rn(-0.5f, __fadd_rn(p, m), s2));
  const float rhs = __fmul_rn(__fmul_rn(dq, dq), sixth);
  const float s2x3 = __fmul_rn(3.f, s2);
  const float m2 = (lhs > rhs) ? __fmaf_rn(-2.f, p, s2x3) : m;
  const float p2 = (lhs < -rhs) ? __fmaf_rn(-2.f, m, s2x3) : p;
  qp = ext ? s2 : p2;
  qm = ext ? s2 : m2;
}

// ---- Two lanes per instruction ---------------------------------------------
// Blackwell's packed FP32 add, multiply and fma (FADD2/FMUL2/FFMA2) round
// each of their two lanes exactly as the scalar intrinsics do.  The step
// kernels are bound by instruction issue, so the hot arithmetic below runs
// two independent evaluations per instruction -- two fields of one line, or
// the same quantities at two quadrature points -- and gives, lane by lane,
// the bits of the scalar form.  a - b is fma(b, -1, a): one rounding of the
// exact a - b, as the scalar subtraction.  Minima, |x|, comparisons and
// selects have no packed form and run per lane.
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, f2(-1.f), a); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 abs2(float2 a) { return f2(fabsf(a.x), fabsf(a.y)); }

// slope32 on two lanes.
__device__ __forceinline__ float2 slope32x2(float2 a, float2 b) {
  const float2 t = mul2(f2(2.f), f2(fminf(fabsf(a.x), fabsf(b.x)), fminf(fabsf(a.y), fabsf(b.y))));
  const float2 u = mul2(f2(0.5f), abs2(add2(a, b)));
  const float2 ab = mul2(a, b);
  return f2(ab.x <= 0.f ? 0.f : copysignf(fminf(t.x, u.x), b.x), ab.y <= 0.f ? 0.f : copysignf(fminf(t.y, u.y), b.y));
}

// ppm32 on two lanes (two fields of a line, or two lines); eta per lane.
template <bool kSteep = false>
__device__ __forceinline__ void ppm32x2(float2 s0, float2 s1, float2 s2, float2 s3, float2 s4, float2& qp, float2& qm,
                                        float2 eta = make_float2(0.f, 0.f)) {
  const float2 msixth = f2(-(1.f / 6.f)), half = f2(0.5f);
  const float2 d0 = sub2(s1, s0), d1 = sub2(s2, s1), d2 = sub2(s3, s2), d3 = sub2(s4, s3);
  const float2 D0 = slope32x2(d0, d1), D1 = slope32x2(d1, d2), D2 = slope32x2(d2, d3);
  float2 p = fma2(msixth, sub2(D2, D1), mul2(half, add2(s2, s3)));
  float2 m = fma2(msixth, sub2(D1, D0), mul2(half, add2(s1, s2)));
  if (kSteep) {
    const float2 keep = sub2(f2(1.f), eta);
    p = fma2(eta, fma2(f2(-0.5f), D2, s3), mul2(keep, p));
    m = fma2(eta, fma2(half, D0, s1), mul2(keep, m));
  }
  const float2 e = mul2(sub2(p, s2), sub2(s2, m));
  const float2 dq = sub2(p, m);
  const float2 lhs = mul2(dq, fma2(f2(-0.5f), add2(p, m), s2));
  const float2 rhs = mul2(mul2(dq, dq), f2(1.f / 6.f));
  const float2 s2x3 = mul2(f2(3.f), s2);
  const float2 mc = fma2(f2(-2.f), p, s2x3), pc = fma2(f2(-2.f), m, s2x3);
  qp.x = e.x <= 0.f ? s2.x : (lhs.x < -rhs.x ? pc.x : p.x);
  qp.y = e.y <= 0.f ? s2.y : (lhs.y < -rhs.y ? pc.y : p.y);
  qm.x = e.x <= 0.f ? s2.x : (lhs.x > rhs.x ? mc.x : m.x);
  qm.y = e.y <= 0.f ? s2.y : (lhs.y > rhs.y ? mc.y : m.y);
}

// The five samples of fields fa and fb along a line (stride st through cell
// c of the padded FP32 array Q), as pairs.
struct Samples2 {
  float2 s[5];
};
__device__ __forceinline__ Samples2 samples2(const float* __restrict__ Q, int c, int st, int fa, int fb) {
  const float* qa = Q + fa * S3 + c;
  const float* qb = Q + fb * S3 + c;
  Samples2 r;
#pragma unroll
  for (int m = 0; m < 5; ++m) r.s[m] = f2(qa[(m - 2) * st], qb[(m - 2) * st]);
  return r;
}

__device__ __forceinline__ void line10f(const float* __restrict__ Q, int c, int st, float qp[F], float qm[F]) {
#pragma unroll
  for (int k = 0; k < F; k += 2) {
    const Samples2 v = samples2(Q, c, st, k, k + 1);
    float2 p, m;
    ppm32x2(v.s[0], v.s[1], v.s[2], v.s[3], v.s[4], p, m);
    qp[k] = p.x;
    qp[k + 1] = p.y;
    qm[k] = m.x;
    qm[k + 1] = m.y;
  }
}

// Contact-steepening weight of one line in FP32 (contact_eta64's definition;
// symmetric under reversal of the line).
__device__ __forceinline__ float contact_eta32(float a0, float a1, float a2, float a3, float a4) {
  const float d2m = __fsub_rn(__fadd_rn(a0, a2), __fmul_rn(2.f, a1)),
              d2p = __fsub_rn(__fadd_rn(a2, a4), __fmul_rn(2.f, a3));
  const float jump = __fsub_rn(a3, a1);
  const float et = __fdiv_rn(__fsub_rn(d2m, d2p), __fmul_rn(6.f, jump));
  const bool off = __fmul_rn(d2m, d2p) > 0.f || fabsf(jump) <= __fmul_rn(0.01f, fminf(fabsf(a3), fabsf(a1)));
  return off ? 0.f : fminf(fmaxf(__fmul_rn(20.f, __fsub_rn(et, 0.05f)), 0.f), 1.f);
}

// The gas-dynamics contact test of a line over its two neighbours (density
// r0, r1 and pressure p0, p1; gamma_k0 = gamma K0): the density jump is a
// contact unless gamma K0 |drho|/min(rho) < |dp|/min(p), taken multiplied
// through by the two positive minima: gamma K0 |drho| min(p) < |dp| min(rho).
// Symmetric.
__device__ __forceinline__ bool contact_line32(float r0, float r1, float p0, float p1, float gamma_k0) {
  const float drho = fabsf(__fsub_rn(r1, r0)), dp = fabsf(__fsub_rn(p1, p0));
  return !(__fmul_rn(__fmul_rn(gamma_k0, drho), fminf(p0, p1)) < __fmul_rn(dp, fminf(r0, r1)));
}

// line10f with contact steepening of the density and species lines (the
// gas-dynamics contact test of line10c over the two neighbours; gamma_k0 =
// gamma K0, gm1 = gamma - 1).
__device__ __forceinline__ void line10fc(const float* __restrict__ Q, int c, int st, float gamma_k0, float gm1,
                                         float qp[F], float qm[F]) {
  static_assert(RHO == 0 && SP0 == F - 1, "the steepened fields are the first and the last");
  const bool contact = contact_line32(Q[RHO * S3 + c - st], Q[RHO * S3 + c + st],
                                      __fmul_rn(gm1, Q[EGAS * S3 + c - st]), __fmul_rn(gm1, Q[EGAS * S3 + c + st]),
                                      gamma_k0);
  {
    // density and species, steepened, as one pair
    const Samples2 v = samples2(Q, c, st, RHO, SP0);
    const float2 eta = contact ? f2(contact_eta32(v.s[0].x, v.s[1].x, v.s[2].x, v.s[3].x, v.s[4].x),
                                    contact_eta32(v.s[0].y, v.s[1].y, v.s[2].y, v.s[3].y, v.s[4].y))
                               : f2(0.f);
    float2 p, m;
    ppm32x2<true>(v.s[0], v.s[1], v.s[2], v.s[3], v.s[4], p, m, eta);
    qp[RHO] = p.x;
    qp[SP0] = p.y;
    qm[RHO] = m.x;
    qm[SP0] = m.y;
  }
#pragma unroll
  for (int k = 1; k < F - 1; k += 2) {
    const Samples2 v = samples2(Q, c, st, k, k + 1);
    float2 p, m;
    ppm32x2(v.s[0], v.s[1], v.s[2], v.s[3], v.s[4], p, m);
    qp[k] = p.x;
    qp[k + 1] = p.y;
    qm[k] = m.x;
    qm[k + 1] = m.y;
  }
}

struct StepParamsF {
  float gamma, gm1, omega;
  int spin;   // the spin feedback (spin_dv32) on (the kernels take it as a template parameter)
  float k3h;  // its 3 / h, (float)(3 / h) of the sub-grid's FP64 h
};

// Spin feedback at a cell's point x_c + (h/2) d, FP32: the velocity there of
// the cell's rigid rotation omega = z / I, I = rho h^2 / 6 (a uniform cube
// about its centre), (3 / (rho h)) z x d, from the cell's FP32 primitives
// rho, eps and z (gg1 = gamma (gamma - 1)); subsonic as spin_dv64 (the
// factor scaled where the corner speed would exceed the sound speed); z x d
// by sign selection (d in {-1, 0, 1}^3), so the increment at x_c - (h/2) d
// is exactly the negative and a line walked either way gets the same values.
// Every operation explicitly rounded.
__device__ __forceinline__ float spin_pick32(int d, float x) { return d == 0 ? 0.f : (d > 0 ? x : -x); }
__device__ __forceinline__ void spin_dv32(float rho, float eps, float zx, float zy, float zz, float k3h, float gg1,
                                          int dx, int dy, int dz, float dv[3]) {
  float k = __fdiv_rn(k3h, rho);
  const float z2 = __fadd_rn(__fadd_rn(__fmul_rn(zx, zx), __fmul_rn(zy, zy)), __fmul_rn(zz, zz));
  const float rc2 = __fmul_rn(gg1, eps);
  if (rc2 < __fmul_rn(__fmul_rn(3.f, __fmul_rn(k3h, k)), z2))
    k = rc2 > 0.f ? __fsqrt_rn(__fdiv_rn(rc2, __fmul_rn(__fmul_rn(3.f, rho), z2))) : 0.f;
  dv[0] = __fmul_rn(k, __fsub_rn(spin_pick32(dz, zy), spin_pick32(dy, zz)));
  dv[1] = __fmul_rn(k, __fsub_rn(spin_pick32(dx, zz), spin_pick32(dz, zx)));
  dv[2] = __fmul_rn(k, __fsub_rn(spin_pick32(dy, zx), spin_pick32(dx, zy)));
}

// ---- Kurganov-Tadmor flux at quadrature points, FP32 ------------------------
// Two points per call, in the two lanes (A, B) of every packed operation; a
// single point runs with both lanes equal.
//
// A side's state at the points: density, velocity, energy E = eps +
// rho|v|^2/2, pressure p = (gamma-1) eps, the rotating-frame advection
// velocity normal to the face (u = v - omega z_hat x x_q) and |u_n| + c.
struct Side32x2 {
  float2 rho, vx, vy, vz, E, p, un, va, spd;
};
template <class QA, class QB>
__device__ __forceinline__ Side32x2 side32x2(const QA& qa, const QB& qb, int a, float2 xq, float2 yq,
                                             const StepParamsF& P) {
  Side32x2 s;
  s.rho = f2(qa(RHO), qb(RHO));
  s.vx = f2(qa(SX), qb(SX));
  s.vy = f2(qa(SY), qb(SY));
  s.vz = f2(qa(SZ), qb(SZ));
  const float2 eps = f2(qa(EGAS), qb(EGAS));
  const float2 v2 = fma2(s.vz, s.vz, fma2(s.vy, s.vy, mul2(s.vx, s.vx)));
  s.E = fma2(mul2(f2(0.5f), s.rho), v2, eps);
  s.p = mul2(f2(P.gm1), eps);
  const float2 gp = mul2(f2(P.gamma), s.p);
  const float2 c2 = f2(__fdividef(gp.x, s.rho.x), __fdividef(gp.y, s.rho.y));
  const float2 c = mul2(c2, f2(rsqrtf(c2.x), rsqrtf(c2.y)));
  const float2 ux = fma2(f2(P.omega), yq, s.vx), uy = fma2(f2(-P.omega), xq, s.vy);
  s.un = (a == 0) ? ux : (a == 1) ? uy : s.vz;
  s.va = (a == 0) ? s.vx : (a == 1) ? s.vy : s.vz;
  s.spd = add2(abs2(s.un), c);
  return s;
}

// Conserved component k of a side (qk: the reconstructed value of field k,
// used for the advected scalars).
__device__ __forceinline__ float2 cons32x2(float2 qk, const Side32x2& s, int k) {
  if (k == RHO) return s.rho;
  if (k <= SZ) return mul2(s.rho, k == SX ? s.vx : (k == SY ? s.vy : s.vz));
  if (k == EGAS) return s.E;
  return qk;
}

// Two quadrature points A, B of a face of axis a (kTwo = false: A only,
// with both lanes equal), added to a face group's sums in the order A, B:
// the point fluxes 2 F_q = (F_L + F_R) - a_q (U_R - U_L) with a_q =
// max(|u_n| + c) of the two sides and F_L + F_R = U_L u_nL + U_R u_nR (+ the
// pressure terms: p_L + p_R in the normal momentum, p_L v_aL + p_R v_aR in
// the energy) as two fused steps, G[k] += (w/2) (2 F_q[k]), and the momentum-
// flux torque about the left cell centre, TL += (w h/4) d x (2 F_s) (the
// lever is (h/2) d), each a fused step; amax takes a_q.  qlA(k), qrA(k),
// qlB(k), qrB(k): the reconstructed primitives of the two sides of A and B
// (read when needed); xq, yq, d per lane; hwA = wA/2, hwB = wB/2 and hqA =
// wA h/4, hqB = wB h/4 (exact halvings of the weights w and w h/2, so each
// sum gets the same value as with the weights applied to F_q).  d is in
// {-1, 0, 1}, so each cross-product component is one rounding of an exact
// difference of exact products.  The torque about the right centre follows
// per face (right_torque32).
template <bool kTwo, class QLA, class QRA, class QLB, class QRB>
__device__ __forceinline__ void point_pair32(const QLA& qlA, const QRA& qrA, const QLB& qlB, const QRB& qrB, int a,
                                             float2 xq, float2 yq, const float2 dL[3], const StepParamsF& P,
                                             float hwA, float hqA, float hwB, float hqB, float G[F], float TL[3],
                                             float& amax) {
  const Side32x2 L = side32x2(qlA, qlB, a, xq, yq, P);
  const Side32x2 R = side32x2(qrA, qrB, a, xq, yq, P);
  const float2 aq = f2(fmaxf(L.spd.x, R.spd.x), fmaxf(L.spd.y, R.spd.y));
  amax = fmaxf(amax, kTwo ? fmaxf(aq.x, aq.y) : aq.x);
  const float2 naq = mul2(f2(-1.f), aq);
  const float2 pp = add2(L.p, R.p);
  const float2 pw = fma2(L.p, L.va, mul2(R.p, R.va));
  float2 fs[3];
#pragma unroll
  for (int k = 0; k < F; ++k) {
    const float2 uL = cons32x2(k >= TAU ? f2(qlA(k), qlB(k)) : f2(0.f), L, k);
    const float2 uR = cons32x2(k >= TAU ? f2(qrA(k), qrB(k)) : f2(0.f), R, k);
    float2 sum;
    if (k == EGAS)
      sum = fma2(uL, L.un, fma2(uR, R.un, pw));
    else if (k >= SX && k <= SZ)
      sum = fma2(uL, L.un, fma2(uR, R.un, k - SX == a ? pp : f2(0.f)));
    else
      sum = fma2(uL, L.un, mul2(uR, R.un));
    const float2 fq2 = fma2(naq, sub2(uR, uL), sum);
    G[k] = __fmaf_rn(hwA, fq2.x, G[k]);
    if (kTwo) G[k] = __fmaf_rn(hwB, fq2.y, G[k]);
    if (k >= SX && k <= SZ) fs[k - SX] = fq2;
  }
  const float2 mL[3] = {mul2(f2(-1.f), dL[0]), mul2(f2(-1.f), dL[1]), mul2(f2(-1.f), dL[2])};
  const float2 cl[3] = {fma2(dL[1], fs[2], mul2(mL[2], fs[1])), fma2(dL[2], fs[0], mul2(mL[0], fs[2])),
                        fma2(dL[0], fs[1], mul2(mL[1], fs[0]))};
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    TL[m] = __fmaf_rn(hqA, cl[m].x, TL[m]);
    if (kTwo) TL[m] = __fmaf_rn(hqB, cl[m].y, TL[m]);
  }
}

// A face's momentum-flux torque about the right cell centre (x_L + h e_a)
// from the one about the left centre, tl, and the face's momentum sums
// S[SX..SZ]: tr = tl - h e_a x S, one fused step per nonzero component.
__device__ __forceinline__ void right_torque32(int a, float h, const float S[F], const float tl[3], float tr[3]) {
  // (e_a x S) components: a = 0: (0, -Sz, Sy); a = 1: (Sz, 0, -Sx); a = 2: (-Sy, Sx, 0)
  tr[0] = a == 0 ? tl[0] : __fmaf_rn(a == 1 ? -h : h, a == 1 ? S[SZ] : S[SY], tl[0]);
  tr[1] = a == 1 ? tl[1] : __fmaf_rn(a == 0 ? h : -h, a == 0 ? S[SZ] : S[SX], tl[1]);
  tr[2] = a == 2 ? tl[2] : __fmaf_rn(a == 0 ? -h : h, a == 0 ? S[SY] : S[SX], tl[2]);
}

// The 9 points of a face in their summation order: point n has offsets
// (u1, u2) along the face's two transverse axes b < c,
//   (1,1), (-1,-1), (1,0), (-1,0), (1,-1), (-1,1), (0,1), (0,-1), (0,0),
// summed in three groups, points 0-3, 4-5 and 6-8, as (G0 + G1) + G2, each
// group a fused chain from zero.  The points go in mirrored pairs (2p, 2p+1)
// and the centre, and no group ends inside a pair.  With one point per face
// (the old module) only the last, the centre, with weight 1.  (u + 1 packed
// two bits per point.)
__host__ __device__ constexpr bool face_group_ends(int n) { return n == 3 || n == 5 || n == 8; }
__device__ __forceinline__ int face_u1(int n) { return ((86562 >> (2 * n)) & 3) - 1; }
__device__ __forceinline__ int face_u2(int n) { return ((75858 >> (2 * n)) & 3) - 1; }
// Newton-Cotes (Simpson) weight of a point, (1,4,1)x(1,4,1)/36, or 1 with
// one point per face.
__device__ __forceinline__ float face_w(int u1, int u2, int face_points) {
  return face_points == 1 ? 1.f : (u1 == 0 && u2 == 0) ? (16.f / 36.f) : (u1 == 0 || u2 == 0) ? (4.f / 36.f) : (1.f / 36.f);
}

// Unlimited interface value towards +d (the 4-point formula the PPM
// interface value reduces to when no limiter acts): used on cells the
// learned indicator marks smooth.
__device__ __forceinline__ void unlimited32(float s0, float s1, float s2, float s3, float s4, float& qp, float& qm) {
  const float a = 7.f / 12.f, b = 1.f / 12.f;
  qp = __fmaf_rn(a, __fadd_rn(s2, s3), -__fmul_rn(b, __fadd_rn(s1, s4)));
  qm = __fmaf_rn(a, __fadd_rn(s1, s2), -__fmul_rn(b, __fadd_rn(s0, s3)));
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
constexpr int kGateB1 = kGateH * kGateIn, kGateW2 = kGateB1 + kGateH, kGateB2 = kGateW2 + kGateH * kGateH,
              kGateW3 = kGateB2 + kGateH, kGateB3 = kGateW3 + kGateH;

__device__ __forceinline__ float bf16r(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

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

// The deployed (inference) form of the network: the inputs and the first
// hidden layer rounded to BF16, products and sums in FP32 -- the arithmetic
// of the tensor-core evaluation in the step kernel (BF16 operands, FP32
// accumulation), here written sequentially.  Parameters already rounded.
template <class W>
__device__ __forceinline__ float gate_logit_infer(const W& w, const float x[54]) {
  float h1[kGateH];
#pragma unroll
  for (int j = 0; j < kGateH; ++j) {
    float z = w(kGateB1 + j);
#pragma unroll
    for (int i = 0; i < kGateIn; ++i) z = fmaf(w(j * kGateIn + i), bf16r(x[i]), z);
    h1[j] = bf16r(fmaxf(z, 0.f));
  }
  float out = w(kGateB3);
#pragma unroll 4
  for (int j = 0; j < kGateH; ++j) {
    float z = w(kGateB2 + j);
#pragma unroll
    for (int i = 0; i < kGateH; ++i) z = fmaf(w(kGateW2 + j * kGateH + i), h1[i], z);
    out = fmaf(w(kGateW3 + j), fmaxf(z, 0.f), out);
  }
  return out;
}

// ---- the indicator on the tensor cores (mma.sync m16n8k16, BF16 in, FP32 out)
// A warp evaluates the network for a tile of 16 cells: A = features [16 x 64]
// (54 used), B = W1^T [64 x 32], then A = the first hidden layer [16 x 32],
// B = W2^T [32 x 32].  Fragments (lane = 4 g + t): A holds rows g and g + 8,
// columns 2t, 2t+1, 2t+8, 2t+9 of a 16-column step; B holds rows 2t, 2t+1,
// 2t+8, 2t+9 of column g; the FP32 accumulator holds rows g, g + 8 and
// columns 2t, 2t+1 of an 8-column tile -- so the first layer's accumulators,
// rounded to BF16, are the second layer's A fragments in place.
__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ __forceinline__ void mma_bf16_16816(float d[4], const uint32_t a[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Weight fragments of one lane (BF16 pairs), loaded once per sub-grid.
struct GateFrags {
  uint32_t w1[4][4][2];  // [k-step][n-tile][reg]
  uint32_t w2[2][4][2];
  float b1[4][2], b2[4][2], w3[4][2], b3;
};

__device__ __forceinline__ void gate_load_frags(const float* __restrict__ w, int lane, GateFrags& f) {
  const int g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int nt = 0; nt < 4; ++nt) {
    const int n = 8 * nt + g;
#pragma unroll
    for (int ks = 0; ks < 4; ++ks) {
      const int k0 = 16 * ks + 2 * t;
      auto W1 = [&](int k) { return k < kGateIn ? __ldg(w + n * kGateIn + k) : 0.f; };
      f.w1[ks][nt][0] = pack_bf16x2(W1(k0), W1(k0 + 1));
      f.w1[ks][nt][1] = pack_bf16x2(W1(k0 + 8), W1(k0 + 9));
    }
#pragma unroll
    for (int ks = 0; ks < 2; ++ks) {
      const int k0 = 16 * ks + 2 * t;
      f.w2[ks][nt][0] = pack_bf16x2(__ldg(w + kGateW2 + n * kGateH + k0), __ldg(w + kGateW2 + n * kGateH + k0 + 1));
      f.w2[ks][nt][1] =
          pack_bf16x2(__ldg(w + kGateW2 + n * kGateH + k0 + 8), __ldg(w + kGateW2 + n * kGateH + k0 + 9));
    }
    const int c0 = 8 * nt + 2 * t;
    f.b1[nt][0] = __ldg(w + kGateB1 + c0);
    f.b1[nt][1] = __ldg(w + kGateB1 + c0 + 1);
    f.b2[nt][0] = __ldg(w + kGateB2 + c0);
    f.b2[nt][1] = __ldg(w + kGateB2 + c0 + 1);
    f.w3[nt][0] = __ldg(w + kGateW3 + c0);
    f.w3[nt][1] = __ldg(w + kGateW3 + c0 + 1);
  }
  f.b3 = __ldg(w + kGateB3);
}

// Shared-memory offset of the j-th feature's neighbour: density (j < 27) or
// internal energy (27 <= j < 54) of neighbour k_j (z, y, x order) relative
// to the cell's density slot; the padding columns 54..63 point at the cell.
struct GateOffsets {
  int off[64];
};
__host__ __device__ constexpr GateOffsets make_gate_offsets() {
  GateOffsets t{};
  for (int j = 0; j < 64; ++j) {
    const int jj = j < 27 ? j : j - 27;
    const int nb = ((jj / 9 - 1) * S + ((jj / 3) % 3 - 1)) * S + (jj % 3 - 1);
    t.off[j] = j < 27 ? nb : (j < kGateIn ? (EGAS - RHO) * S3 + nb : 0);
  }
  return t;
}
__constant__ const GateOffsets c_gate_off = make_gate_offsets();

// One indicator feature (index j of 54) of the cell at padded index c:
// (q(c + k_j) - q(c)) / (|q(c + k_j)| + |q(c)|), q = density (j < 27) or
// pressure (gm1 * eps), k_j the j-th neighbour in (z, y, x) order.
template <class T>
__device__ __forceinline__ float gate_feature(const T* __restrict__ Q, int c, float rc, float pc, float gm1, int j) {
  const float v = (float)Q[RHO * S3 + c + c_gate_off.off[j]];
  const float qk = j < 27 ? v : gm1 * v;
  const float qc = j < 27 ? rc : pc;
  return __fdividef(qk - qc, fabsf(qk) + fabsf(qc));
}

// Logits of the two cells (rows g and g + 8 of the tile) held by this lane's
// group; cells c0, c1 are padded indices of the primitives Q (FP32, or FP64
// read in FP32: the features are defined in FP32).  zero0/zero1: whether
// every feature of the cell is zero (a uniform neighbourhood).
template <class T>
__device__ __forceinline__ void gate_tile_mma(const T* __restrict__ Q, float gm1, int c0, int c1,
                                              const GateFrags& f, int lane, float& logit0, float& logit1,
                                              bool& zero0, bool& zero1) {
  const int t = lane & 3;
  const float r0 = (float)Q[RHO * S3 + c0], p0 = gm1 * (float)Q[EGAS * S3 + c0];
  const float r1 = (float)Q[RHO * S3 + c1], p1 = gm1 * (float)Q[EGAS * S3 + c1];
  uint32_t a[4][4];
  bool nz0 = false, nz1 = false;
#pragma unroll
  for (int ks = 0; ks < 4; ++ks) {
    float v0[4], v1[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int j = 16 * ks + 2 * t + (e & 1) + ((e >> 1) << 3);  // columns 2t, 2t+1, 2t+8, 2t+9
      v0[e] = j < kGateIn ? gate_feature(Q, c0, r0, p0, gm1, j) : 0.f;
      v1[e] = j < kGateIn ? gate_feature(Q, c1, r1, p1, gm1, j) : 0.f;
      nz0 |= v0[e] != 0.f;
      nz1 |= v1[e] != 0.f;
    }
    a[ks][0] = pack_bf16x2(v0[0], v0[1]);
    a[ks][1] = pack_bf16x2(v1[0], v1[1]);
    a[ks][2] = pack_bf16x2(v0[2], v0[3]);
    a[ks][3] = pack_bf16x2(v1[2], v1[3]);
  }
  nz0 |= __shfl_xor_sync(0xffffffffu, nz0, 1);
  nz0 |= __shfl_xor_sync(0xffffffffu, nz0, 2);
  nz1 |= __shfl_xor_sync(0xffffffffu, nz1, 1);
  nz1 |= __shfl_xor_sync(0xffffffffu, nz1, 2);
  zero0 = !nz0;
  zero1 = !nz1;
  logit0 = logit1 = 0.f;
  if (!__any_sync(0xffffffffu, nz0 || nz1)) return;  // a uniform tile: the caller uses the zero-feature decision
  float acc[4][4];
#pragma unroll
  for (int nt = 0; nt < 4; ++nt) {
    acc[nt][0] = acc[nt][2] = f.b1[nt][0];
    acc[nt][1] = acc[nt][3] = f.b1[nt][1];
#pragma unroll
    for (int ks = 0; ks < 4; ++ks) mma_bf16_16816(acc[nt], a[ks], f.w1[ks][nt][0], f.w1[ks][nt][1]);
  }
  uint32_t h[2][4];
#pragma unroll
  for (int ks = 0; ks < 2; ++ks) {
    h[ks][0] = pack_bf16x2(fmaxf(acc[2 * ks][0], 0.f), fmaxf(acc[2 * ks][1], 0.f));
    h[ks][1] = pack_bf16x2(fmaxf(acc[2 * ks][2], 0.f), fmaxf(acc[2 * ks][3], 0.f));
    h[ks][2] = pack_bf16x2(fmaxf(acc[2 * ks + 1][0], 0.f), fmaxf(acc[2 * ks + 1][1], 0.f));
    h[ks][3] = pack_bf16x2(fmaxf(acc[2 * ks + 1][2], 0.f), fmaxf(acc[2 * ks + 1][3], 0.f));
  }
  float s0 = 0.f, s1 = 0.f;
#pragma unroll
  for (int nt = 0; nt < 4; ++nt) {
    float d[4] = {f.b2[nt][0], f.b2[nt][1], f.b2[nt][0], f.b2[nt][1]};
#pragma unroll
    for (int ks = 0; ks < 2; ++ks) mma_bf16_16816(d, h[ks], f.w2[ks][nt][0], f.w2[ks][nt][1]);
    s0 = fmaf(f.w3[nt][0], fmaxf(d[0], 0.f), s0);
    s0 = fmaf(f.w3[nt][1], fmaxf(d[1], 0.f), s0);
    s1 = fmaf(f.w3[nt][0], fmaxf(d[2], 0.f), s1);
    s1 = fmaf(f.w3[nt][1], fmaxf(d[3], 0.f), s1);
  }
  // the group's four lanes hold eight columns each: fixed-order sum
  s0 += __shfl_xor_sync(0xffffffffu, s0, 1);
  s0 += __shfl_xor_sync(0xffffffffu, s0, 2);
  s1 += __shfl_xor_sync(0xffffffffu, s1, 1);
  s1 += __shfl_xor_sync(0xffffffffu, s1, 2);
  logit0 = s0 + f.b3;
  logit1 = s1 + f.b3;
}

// The indicator's decision for every reconstructed cell of a sub-grid whose
// primitives Q (FP32 or FP64) are in shared memory: predict on the 12^3 block
// of cells [-2, N+1]^3, 16 cells per warp-wide tensor-core tile (a cell whose
// 3x3x3 neighbourhood is uniform has all features 0 and takes the network's
// decision at 0, computed once with the parameters; a tile of such cells
// skips the MMAs; a sub-grid whose padded density and internal energy are
// uniform skips the network altogether), then a reconstructed cell (in
// [-1, N]^3) is smooth only if every cell of its 3x3x3 block is predicted
// smooth: the 5-point stencils along the 13 lines reach two cells out,
// beyond one cell's 3x3x3 features.  smooth and pred: [S3] bytes each.
// Called by all threads of the block; ends with a block barrier.
template <class T, int kThreads>
__device__ __forceinline__ void gate_phase(const T* __restrict__ Q, float gm1, const float* __restrict__ gate_w,
                                           float logit_thr, int zero_smooth, uint8_t* smooth, uint8_t* pred) {
  const int tid = threadIdx.x;
  const T r0 = Q[RHO * S3], e0 = Q[EGAS * S3];
  bool same = true;
  for (int c = tid; c < S3; c += kThreads) same &= (Q[RHO * S3 + c] == r0) & (Q[EGAS * S3 + c] == e0);
  if (__syncthreads_and(same)) {
    for (int c = tid; c < S3; c += kThreads) smooth[c] = (uint8_t)zero_smooth;
    __syncthreads();
    return;
  }
  const int lane = tid & 31;
  GateFrags gf;
  gate_load_frags(gate_w, lane, gf);
  constexpr int kBlock = (N + 4) * (N + 4) * (N + 4);  // 1728 = 108 tiles of 16
  for (int tile = tid >> 5; tile < kBlock / 16; tile += kThreads / 32) {
    int cc[2];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int i = 16 * tile + (lane >> 2) + 8 * r;
      const int x = i % (N + 4) - 2, y = (i / (N + 4)) % (N + 4) - 2, z = i / ((N + 4) * (N + 4)) - 2;
      cc[r] = ((z + G) * S + (y + G)) * S + (x + G);
    }
    float l0, l1;
    bool z0, z1;
    gate_tile_mma(Q, gm1, cc[0], cc[1], gf, lane, l0, l1, z0, z1);
    if ((lane & 3) == 0) {
      pred[cc[0]] = (z0 ? zero_smooth : (l0 < logit_thr)) ? 1 : 0;
      pred[cc[1]] = (z1 ? zero_smooth : (l1 < logit_thr)) ? 1 : 0;
    }
  }
  __syncthreads();
  for (int i = tid; i < (N + 2) * (N + 2) * (N + 2); i += kThreads) {
    const int x = i % (N + 2) - 1, y = (i / (N + 2)) % (N + 2) - 1, z = i / ((N + 2) * (N + 2)) - 1;
    const int c = ((z + G) * S + (y + G)) * S + (x + G);
    uint8_t all = 1;
#pragma unroll
    for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
      for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx) all &= pred[c + (dz * S + dy) * S + dx];
    smooth[c] = all;
  }
  __syncthreads();
}

}  // namespace hyd
