// hydro_fp64.cuh -- FP64 arithmetic of the plain method shared by the FP64
// step kernels: the MC-limited PPM reconstruction (Colella & Woodward 1984)
// in explicitly rounded operations in the oracle's order, contact
// steepening, the indicator's unlimited reconstruction, and the
// Kurganov-Tadmor point flux with its torques (Sec. III-B).
#pragma once
#include "hydro_common.cuh"

namespace hyd {

// Smaller of two non-negative doubles: their bit patterns order like their
// values, so an integer minimum gives fmin's result on the integer pipes
// (GB300 issues FP64 at 1/64 of the FP32 rate).
__device__ __forceinline__ double min_nonneg(double x, double y) {
  const long long a = __double_as_longlong(x), b = __double_as_longlong(y);
  return __longlong_as_double(a < b ? a : b);
}

__device__ __forceinline__ double max_nonneg(double x, double y) {
  const long long a = __double_as_longlong(x), b = __double_as_longlong(y);
  return __longlong_as_double(a > b ? a : b);
}

// An integer that orders like the double (for non-NaN values; -0 sorts just
// below +0).  x > y with y >= +0, and x < -y with y >= +0 (-y <= -0), give the
// IEEE results through these keys: the two cases where the key order and
// IEEE disagree, -0 against +0, then both answer false as IEEE does.
__device__ __forceinline__ long long order_key(double x) {
  const long long b = __double_as_longlong(x);
  return b >= 0 ? b : (b ^ 0x7fffffffffffffffLL);
}

// 2x for a finite double x >= 0, exactly: a normal x gains one in the
// exponent field, a subnormal x (exponent field 0) doubles its pattern, which
// carries into the exponent field where 2x is normal.
__device__ __forceinline__ double twice_nonneg(double x) {
  const long long b = __double_as_longlong(x);
  return __longlong_as_double(b < (1LL << 52) ? b + b : b + (1LL << 52));
}

// x <= 0 for a non-NaN double: +0 has the bit pattern 0 and every value with
// the sign bit set (-0 and the negatives) is negative as a signed integer.
__device__ __forceinline__ bool nonpositive(double x) { return __double_as_longlong(x) <= 0LL; }

// x / 2 exactly as the FP64 product 0.5 x rounds it (to nearest, ties to
// even), on the integer pipes: with the exponent field at least 2 the result
// is normal and the field drops by one (infinities and NaNs pass unchanged);
// below that the magnitude's bit pattern is the significand with its
// implicit bit (field 1) or without (zero, subnormals), and half of it,
// rounded to even, is the result's pattern (a carry into bit 52 is the
// smallest normal, correctly encoded).
__device__ __forceinline__ double half64(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned long long sign = b & 0x8000000000000000ull, mag = b ^ sign;
  unsigned long long r;
  if (mag >= (2ull << 52))
    r = mag < (0x7ffull << 52) ? mag - (1ull << 52) : mag;
  else
    r = (mag >> 1) + (mag & (mag >> 1) & 1ull);
  return __longlong_as_double((long long)(r | sign));
}

// MC-limited slope of sample j from delta_{j-1} = a and delta_j = b:
// 0 if a b <= 0, else sgn(b) min(2|a|, 2|b|, |a + b|/2).  The product test is
// the FP64 product, compared on its bit pattern; min(2|a|, 2|b|) =
// 2 min(|a|, |b|) exactly, the minima of non-negative values are taken and
// the doubling and halving done on the bit patterns, and with a b > 0 the
// sign of the result is the sign bit of b: the same bits as the FP64
// multiplications, fmin and comparisons, with 2 instead of 9 FP64
// instructions.  (An integer form of the product test, exact but for a
// fallback near the underflow threshold, measured slower.)
__device__ __forceinline__ double slope64(double a, double b) {
  if (nonpositive(rmul(a, b))) return 0.0;
  const double m = min_nonneg(twice_nonneg(min_nonneg(fabs(a), fabs(b))), half64(fabs(radd(a, b))));
  const long long sign = __double_as_longlong(b) & (long long)0x8000000000000000ull;
  return __longlong_as_double(__double_as_longlong(m) | sign);
}

// The unlimited PPM interface value between samples sa and sb (in the line's
// order) from their limited slopes Da, Db: (sa + sb)/2 - (Db - Da)/6.  The
// +d value of a cell and the -d value of its +d neighbour are the same
// number, so a sweep along the line may compute it once for both.
__device__ __forceinline__ double ppm_iface64(double sa, double sb, double Da, double Db) {
  const double sixth = 1.0 / 6.0;
  return rsub(half64(radd(sa, sb)), rmul(rsub(Db, Da), sixth));
}

// Contact steepening of the interface values p (+d) and m (-d) of the
// centre sample s2 with weight eta > 0, from its neighbours s1, s3 and their
// slopes D0, D2.
__device__ __forceinline__ void ppm_steep64(double s1, double s3, double D0, double D2, double eta, double& p,
                                            double& m) {
  const double keep = rsub(1.0, eta);
  p = radd(rmul(keep, p), rmul(eta, rsub(s3, half64(D2))));
  m = radd(rmul(keep, m), rmul(eta, radd(s1, half64(D0))));
}

// The monotonicity fix-ups of PPM on the interface values p (+d) and m (-d)
// of the cell value s2: a local extremum flattens the cell, an interface
// value that would put the parabola's extremum inside the cell is moved to
// 3 s2 - 2 (the other one).
__device__ __forceinline__ void ppm_limit64(double s2, double& p, double& m) {
  const double sixth = 1.0 / 6.0;
  if (nonpositive(rmul(rsub(p, s2), rsub(s2, m)))) {
    p = s2;
    m = s2;
  } else {
    const double dq = rsub(p, m);
    const double lhs = rmul(dq, rsub(s2, half64(radd(p, m))));
    const double rhs = rmul(rmul(dq, dq), sixth);  // >= +0
    const long long kl = order_key(lhs);
    if (kl > order_key(rhs)) {
      m = rsub(rmul(3.0, s2), rmul(2.0, p));
    } else if (kl < order_key(-rhs)) {
      p = rsub(rmul(3.0, s2), rmul(2.0, m));
    }
  }
}

// PPM on the five samples s0..s4 of one line: qp = value at the +d end of the
// centre cell, qm = value at its -d end (limited, monotonised).  kSteep: blend
// both interface values with the neighbours' limited extrapolations by the
// contact-steepening weight eta before the fix-ups (Colella & Woodward 1984):
//   qp <- (1-eta) qp + eta (s3 - D2/2),  qm <- (1-eta) qm + eta (s1 + D0/2).
template <bool kSteep = false>
__device__ __forceinline__ void ppm64(double s0, double s1, double s2, double s3, double s4, double& qp,
                                      double& qm, double eta = 0.0) {
  const double d0 = rsub(s1, s0), d1 = rsub(s2, s1), d2 = rsub(s3, s2), d3 = rsub(s4, s3);
  const double D0 = slope64(d0, d1), D1 = slope64(d1, d2), D2 = slope64(d2, d3);
  double p = ppm_iface64(s2, s3, D1, D2);
  double m = ppm_iface64(s1, s2, D0, D1);
  if (kSteep && eta > 0.0) ppm_steep64(s1, s3, D0, D2, eta, p, m);
  ppm_limit64(s2, p, m);
  qp = p;
  qm = m;
}

// All ten primitives along the line through smem cell index c with stride st.
__device__ __forceinline__ void line10(const double* __restrict__ Q, int c, int st, double qp[F], double qm[F]) {
#pragma unroll
  for (int k = 0; k < F; ++k) {
    const double* q = Q + k * S3 + c;
    ppm64(q[-2 * st], q[-st], q[0], q[st], q[2 * st], qp[k], qm[k]);
  }
}

// Contact-steepening weight of one line from the five samples a0..a4 of the
// steepened field (Colella & Woodward 1984 discontinuity detection; their
// constants eps = 0.01, eta1 = 20, eta2 = 0.05): second differences
// d- = (a0 + a2) - 2 a1 and d+ = (a2 + a4) - 2 a3; no weight without an
// inflection (d- d+ > 0) or with a jump a3 - a1 of at most eps min(|a3|, |a1|);
// else eta~ = -(d+ - d-) / (6 (a3 - a1)) and eta = max(0, min(20 (eta~ - 0.05), 1)).
// Every operation explicitly rounded, in the oracle's order, and the minima
// and maxima as the same comparisons: the oracle's bits.
__device__ __forceinline__ double contact_eta64(double a0, double a1, double a2, double a3, double a4) {
  const double d2m = rsub(radd(a0, a2), rmul(2.0, a1));
  const double d2p = rsub(radd(a2, a4), rmul(2.0, a3));
  if (rmul(d2m, d2p) > 0.0) return 0.0;
  const double jump = rsub(a3, a1);
  const double f3 = fabs(a3), f1 = fabs(a1);
  if (fabs(jump) <= rmul(0.01, f3 < f1 ? f3 : f1)) return 0.0;
  const double et = -rsub(d2p, d2m) / rmul(6.0, jump);
  const double v = rmul(20.0, rsub(et, 0.05));
  const double m = v < 1.0 ? v : 1.0;
  return 0.0 > m ? 0.0 : m;
}

// Whether the line through smem cell c with stride st crosses a contact, not
// a shock: Colella & Woodward's gas-dynamics test over the cell's two
// neighbours on the line (K0 = 0.1), multiplied through by the two positive
// minima (no division):
//   gamma K0 |rho+ - rho-| min(p) >= |p+ - p-| min(rho),  p = (gamma-1) eps.
__device__ __forceinline__ bool contact_line64(const double* __restrict__ Q, int c, int st, const StepParams& P) {
  const double r0 = Q[RHO * S3 + c - st], r1 = Q[RHO * S3 + c + st];
  const double p0 = rmul(P.gm1, Q[EGAS * S3 + c - st]), p1 = rmul(P.gm1, Q[EGAS * S3 + c + st]);
  const double drho = fabs(rsub(r1, r0)), dp = fabs(rsub(p1, p0));
  return !(rmul(rmul(rmul(P.gamma, 0.1), drho), p0 < p1 ? p0 : p1) < rmul(dp, r0 < r1 ? r0 : r1));
}

// line10 with contact steepening of the density and species lines where the
// line crosses a contact.
__device__ __forceinline__ void line10c(const double* __restrict__ Q, int c, int st, const StepParams& P,
                                        double qp[F], double qm[F]) {
  const bool contact = contact_line64(Q, c, st, P);
#pragma unroll
  for (int k = 0; k < F; ++k) {
    const double* q = Q + k * S3 + c;
    if (k == RHO || k >= SP0) {
      const double eta = contact ? contact_eta64(q[-2 * st], q[-st], q[0], q[st], q[2 * st]) : 0.0;
      ppm64<true>(q[-2 * st], q[-st], q[0], q[st], q[2 * st], qp[k], qm[k], eta);
    } else {
      ppm64(q[-2 * st], q[-st], q[0], q[st], q[2 * st], qp[k], qm[k]);
    }
  }
}

// Lines of a cell the learned indicator marks smooth: the unlimited 4-point
// interface values q+ = 7/12 (q0 + q1) - 1/12 (q-1 + q2) towards +d (and the
// mirror towards -d) for every field but the spin, which stays limited.
__device__ __forceinline__ void line10u(const double* __restrict__ Q, int c, int st, double qp[F], double qm[F]) {
  const double c7 = 7.0 / 12.0, c1 = 1.0 / 12.0;
#pragma unroll
  for (int k = 0; k < F; ++k) {
    const double* q = Q + k * S3 + c;
    if (k == ZX || k == ZY || k == ZZ) {
      ppm64(q[-2 * st], q[-st], q[0], q[st], q[2 * st], qp[k], qm[k]);
    } else {
      qp[k] = rsub(rmul(c7, radd(q[0], q[st])), rmul(c1, radd(q[-st], q[2 * st])));
      qm[k] = rsub(rmul(c7, radd(q[0], q[-st])), rmul(c1, radd(q[st], q[-2 * st])));
    }
  }
}

// Physical side state at a quadrature point: conserved U, the normal
// velocity u_n and the a-component v_a of v, the pressure p and the signal
// speed |u_n| + c.  u = v - omega z_hat x x_q (rotating frame), so u_n is one
// FMA of the selected components (exactly v_z along z).
__device__ __forceinline__ void side64(const double q[F], int a, double xq, double yq, const StepParams& P,
                                       double U[F], double& un, double& va, double& p, double& spd) {
  const double rho = q[RHO], vx = q[1], vy = q[2], vz = q[3], eps = q[4];
  const double ek = half64(rho) * ((vx * vx + vy * vy) + vz * vz);
  p = P.gm1 * eps;
  // c = sqrt(gamma p / rho) = gamma p / sqrt(gamma p rho): one reciprocal
  // square root instead of a division and a square root (a few ulps from the
  // correctly rounded value); c = 0 where p <= 0 (a non-physical state)
  const double gp = P.gamma * p;
  const double c = (__double_as_longlong(gp) <= 0LL) ? 0.0 : gp * rsqrt(gp * rho);
  va = (a == 0) ? vx : (a == 1) ? vy : vz;
  const double om = (a == 0) ? P.omega : (a == 1) ? -P.omega : 0.0;
  const double r = (a == 0) ? yq : (a == 1) ? xq : 0.0;
  un = fma(om, r, va);
  U[RHO] = rho;
  U[SX] = rho * vx;
  U[SY] = rho * vy;
  U[SZ] = rho * vz;
  U[EGAS] = eps + ek;
#pragma unroll
  for (int k = TAU; k < F; ++k) U[k] = q[k];
  spd = fabs(un) + c;
}

// d x g for an integer vector d with components in {-1, 0, 1}: each term is
// +-g_i or zero, taken by sign selection, so one FP64 subtraction per
// component.
__device__ __forceinline__ double signed_pick(int d, double x) { return d == 0 ? 0.0 : (d > 0 ? x : -x); }

// Spin feedback at a cell's point x_c + (h/2) d: the velocity there of the
// cell's rigid rotation omega = z / I, I = rho h^2 / 6 (a uniform cube about
// its centre), omega x (h/2) d = (3 / (rho h)) z x d, for the cell's
// primitives rho, eps and z and k3h = 3 / h, gg1 = gamma (gamma - 1).  The
// rotation is subsonic: where its corner speed sqrt(3) (3 / (rho h)) |z|
// exceeds the sound speed c = sqrt(gg1 eps / rho), the factor 3 / (rho h) is
// replaced by the one that reaches c there, c / (sqrt(3) |z|) (none for
// eps <= 0).  The test compares rho c^2 with rho times the corner speed
// squared, so that only a capped cell divides again.  z x d by sign
// selection (d in {-1, 0, 1}^3), so the increment at x_c - (h/2) d is
// exactly the negative.  Explicitly rounded (no contraction), so that every
// kernel that adds it gets the same bits.
__device__ __forceinline__ void spin_dv64(double rho, double eps, double zx, double zy, double zz, double k3h,
                                          double gg1, int dx, int dy, int dz, double dv[3]) {
  double k = k3h / rho;
  const double z2 = radd(radd(rmul(zx, zx), rmul(zy, zy)), rmul(zz, zz));
  const double rc2 = rmul(gg1, eps);
  if (rc2 < rmul(rmul(3.0, rmul(k3h, k)), z2)) k = rc2 > 0.0 ? sqrt(rc2 / rmul(rmul(3.0, rho), z2)) : 0.0;
  dv[0] = rmul(k, rsub(signed_pick(dz, zy), signed_pick(dy, zz)));
  dv[1] = rmul(k, rsub(signed_pick(dx, zz), signed_pick(dz, zx)));
  dv[2] = rmul(k, rsub(signed_pick(dy, zx), signed_pick(dx, zy)));
}

// Kurganov-Tadmor flux at one point with half its Simpson weight hw = w/2:
//   w F_q = hw (F_L + F_R) - hw a_q (U_R - U_L),  F = U u_n (+ p e_a, + p v_a),
// accumulated per field into the face sum (F_L + F_R as two fused products,
// the weight folded into the fused accumulation).  The point lies at
// x_L + (h/2) d from the left cell's centre (integer d, d_a = 1); the torque
// sum T accumulates d x (w F_q) of the momentum flux, so that the face's
// torque about the left centre is (h/2) T and about the right centre (at
// x_L + h e_a) (h/2) T - h e_a x (sum of w F_q).
__device__ __forceinline__ void point64(const double qL[F], const double qR[F], int a, double xq, double yq,
                                        double hw, int d0, int d1, int d2, const StepParams& P, double fsum[F],
                                        double T[3], double& amax) {
  double UL[F], UR[F], unL, unR, vaL, vaR, pL, pR, sL, sR;
  side64(qL, a, xq, yq, P, UL, unL, vaL, pL, sL);
  side64(qR, a, xq, yq, P, UR, unR, vaR, pR, sR);
  const double aq = max_nonneg(sL, sR);  // signal speeds are >= 0
  amax = max_nonneg(amax, aq);
  const double hwa = hw * aq;
  const double pp = pL + pR;
  double g[3];
#pragma unroll
  for (int k = 0; k < F; ++k) {
    // the pressure terms of F_L + F_R: p in the normal momentum, p v_a in the energy
    double extra = 0.0;
    if (k == SX || k == SY || k == SZ) extra = (a == k - SX) ? pp : 0.0;
    if (k == EGAS) extra = fma(pL, vaL, pR * vaR);
    const double sum = fma(UL[k], unL, fma(UR[k], unR, extra));
    const double dif = UR[k] - UL[k];
    if (k == SX || k == SY || k == SZ) {
      const double gk = fma(hw, sum, -(hwa * dif));
      g[k - SX] = gk;
      fsum[k] += gk;
    } else {
      fsum[k] = fma(hw, sum, fma(-hwa, dif, fsum[k]));
    }
  }
  T[0] += signed_pick(d1, g[2]) - signed_pick(d2, g[1]);
  T[1] += signed_pick(d2, g[0]) - signed_pick(d0, g[2]);
  T[2] += signed_pick(d0, g[1]) - signed_pick(d1, g[0]);
}

// The face's torques about the left and right cell centres from point64's
// torque sum T and face sum fsum: tl = (h/2) T, tr = (h/2) (T - 2 e_a x m)
// with m the momentum part of fsum.
__device__ __forceinline__ void face_torques64(const double T[3], const double fsum[F], int a, double half_h,
                                               double tl[3], double tr[3]) {
  const double mx = fsum[SX], my = fsum[SY], mz = fsum[SZ];
  // e_a x m
  const double ex = (a == 0) ? 0.0 : (a == 1) ? mz : -my;
  const double ey = (a == 0) ? -mz : (a == 1) ? 0.0 : mx;
  const double ez = (a == 0) ? my : (a == 1) ? -mx : 0.0;
  tl[0] = half_h * T[0];
  tl[1] = half_h * T[1];
  tl[2] = half_h * T[2];
  tr[0] = half_h * (T[0] - (ex + ex));
  tr[1] = half_h * (T[1] - (ey + ey));
  tr[2] = half_h * (T[2] - (ez + ez));
}

}  // namespace hyd
