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

// MC-limited slope of sample j from delta_{j-1} = a and delta_j = b:
// 0 if a b <= 0, else sgn(b) min(2|a|, 2|b|, |a + b|/2).  The product test is
// the FP64 product, compared on its bit pattern; min(2|a|, 2|b|) =
// 2 min(|a|, |b|) exactly, the minima of non-negative values are taken and
// the doubling done on the bit patterns, and with a b > 0 the sign of the
// result is the sign bit of b: the same bits as the FP64 multiplications,
// fmin and comparisons, with 3 instead of 9 FP64 instructions.
__device__ __forceinline__ double slope64(double a, double b) {
  if (nonpositive(rmul(a, b))) return 0.0;
  const double m = min_nonneg(twice_nonneg(min_nonneg(fabs(a), fabs(b))), rmul(0.5, fabs(radd(a, b))));
  const long long sign = __double_as_longlong(b) & (long long)0x8000000000000000ull;
  return __longlong_as_double(__double_as_longlong(m) | sign);
}

// The unlimited PPM interface value between samples sa and sb (in the line's
// order) from their limited slopes Da, Db: (sa + sb)/2 - (Db - Da)/6.  The
// +d value of a cell and the -d value of its +d neighbour are the same
// number, so a sweep along the line may compute it once for both.
__device__ __forceinline__ double ppm_iface64(double sa, double sb, double Da, double Db) {
  const double sixth = 1.0 / 6.0;
  return rsub(rmul(0.5, radd(sa, sb)), rmul(rsub(Db, Da), sixth));
}

// Contact steepening of the interface values p (+d) and m (-d) of the
// centre sample s2 with weight eta > 0, from its neighbours s1, s3 and their
// slopes D0, D2.
__device__ __forceinline__ void ppm_steep64(double s1, double s3, double D0, double D2, double eta, double& p,
                                            double& m) {
  const double keep = rsub(1.0, eta);
  p = radd(rmul(keep, p), rmul(eta, rsub(s3, rmul(0.5, D2))));
  m = radd(rmul(keep, m), rmul(eta, radd(s1, rmul(0.5, D0))));
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
    const double lhs = rmul(dq, rsub(s2, rmul(0.5, radd(p, m))));
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

// Physical side state at a quadrature point: conserved U, flux F along axis a,
// signal speed |u_n| + c.  u = v - omega z_hat x x_q (rotating frame).
__device__ __forceinline__ void side64(const double q[F], int a, double xq, double yq, const StepParams& P,
                                       double U[F], double Fl[F], double& spd) {
  const double rho = q[RHO], vx = q[1], vy = q[2], vz = q[3], eps = q[4];
  const double ek = (0.5 * rho) * ((vx * vx + vy * vy) + vz * vz);
  const double E = eps + ek;
  const double p = P.gm1 * eps;
  // c = sqrt(gamma p / rho) = gamma p / sqrt(gamma p rho): one reciprocal
  // square root instead of a division and a square root (a few ulps from the
  // correctly rounded value); c = 0 where p <= 0 (a non-physical state)
  const double gp = P.gamma * p;
  const double c = (__double_as_longlong(gp) <= 0LL) ? 0.0 : gp * rsqrt(gp * rho);
  const double ux = vx + P.omega * yq, uy = vy - P.omega * xq;
  const double un = (a == 0) ? ux : (a == 1) ? uy : vz;
  const double va = (a == 0) ? vx : (a == 1) ? vy : vz;
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
  spd = fabs(un) + c;
}

// Kurganov-Tadmor flux at one point, accumulated with weight w into the face
// sum and into the torques about the left (rl) and right (rr) cell centres.
__device__ __forceinline__ void point64(const double qL[F], const double qR[F], int a, double xq, double yq,
                                        double w, const double rl[3], const double rr[3], const StepParams& P,
                                        double fsum[F], double tl[3], double tr[3], double& amax) {
  double UL[F], FL[F], UR[F], FR[F], sL, sR;
  side64(qL, a, xq, yq, P, UL, FL, sL);
  side64(qR, a, xq, yq, P, UR, FR, sR);
  const double aq = max_nonneg(sL, sR);  // signal speeds are >= 0
  amax = max_nonneg(amax, aq);
  double Fq[F];
#pragma unroll
  for (int k = 0; k < F; ++k) {
    Fq[k] = 0.5 * (FL[k] + FR[k]) - (0.5 * aq) * (UR[k] - UL[k]);
    fsum[k] += w * Fq[k];
  }
  const double fx = Fq[SX], fy = Fq[SY], fz = Fq[SZ];
  tl[0] += w * (rl[1] * fz - rl[2] * fy);
  tl[1] += w * (rl[2] * fx - rl[0] * fz);
  tl[2] += w * (rl[0] * fy - rl[1] * fx);
  tr[0] += w * (rr[1] * fz - rr[2] * fy);
  tr[1] += w * (rr[2] * fx - rr[0] * fz);
  tr[2] += w * (rr[0] * fy - rr[1] * fx);
}

}  // namespace hyd
