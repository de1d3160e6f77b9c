// hydro_oracle.cpp -- plain, slow FP64 CPU oracle of the per-sub-grid hydro step.
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call
// this file: only the tests, the smoke check and the benchmark's CPU-baseline
// leg do.  It shares no code, header, table or constant with the CUDA library.
//
// What it computes (arXiv 2107.10987, Sec. III-B "Octo-Tiger's Hydro
// Implementation", and the rotating frame of Sec. I):
//   * cell averages of the evolved fields (rho, s, E, tau, z, species) on an
//     N^3 sub-grid with a 3-deep ghost layer;
//   * primitives with the dual-energy selection of Bryan et al. (1995);
//   * PPM (Colella & Woodward 1984) along the 13 lines through cell centres,
//     giving left/right values at the 26 face, edge and vertex points, with
//     the optional contact-discontinuity steepening of that paper;
//   * the Kurganov-Tadmor (2000) central flux at the 9 points of each face;
//   * the Newton-Cotes (Simpson) face sum and the flux divergence;
//   * rotating-frame, gravity and spin-torque sources;
//   * the maximum signal speed over all quadrature points (CFL);
//   * the SSP-RK3 stage update with the dual-energy tracer resync.
//   * optionally, the spin's feedback into the velocity at the quadrature
//     points (spin_feedback: parity unpinned beyond its checks).
// Where the paper defers a detail to the Octo-Tiger method paper, the reading
// taken is stated at the line that uses it.  Every function is templated on
// the scalar type so that an operation-counting type yields the exact number
// of floating-point operations of the method.
//
// Build: g++ -O2 -std=c++17 -ffp-contract=off -fopenmp -shared -fPIC
// (-ffp-contract=off: every a*b+c below is two rounded operations, as written).

#include <cmath>
#include <cstdint>
#include <cstring>
#include <type_traits>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace orc {

// ----------------------------------------------------------------------------
// Operation-counting scalar.  Each arithmetic operator, comparison, min/max,
// sqrt and pow increments a per-thread counter; abs and negation are counted
// separately (they are sign-bit operations).
struct Ops {
  long add = 0, mul = 0, div = 0, sqrt = 0, pow = 0, cmp = 0, minmax = 0, sgn = 0;
  long total() const { return add + mul + div + sqrt + pow + cmp + minmax; }
};
static thread_local Ops g_ops;
// operations spent inside PPM line evaluations, and the number of evaluations
static thread_local long g_ppm_ops = 0, g_ppm_calls = 0;

struct CD {
  double v;
  CD(double x = 0.0) : v(x) {}
};
inline CD operator+(CD a, CD b) { g_ops.add++; return CD(a.v + b.v); }
inline CD operator-(CD a, CD b) { g_ops.add++; return CD(a.v - b.v); }
inline CD operator*(CD a, CD b) { g_ops.mul++; return CD(a.v * b.v); }
inline CD operator/(CD a, CD b) { g_ops.div++; return CD(a.v / b.v); }
inline CD operator-(CD a) { g_ops.sgn++; return CD(-a.v); }
inline bool operator<(CD a, CD b) { g_ops.cmp++; return a.v < b.v; }
inline bool operator>(CD a, CD b) { g_ops.cmp++; return a.v > b.v; }
inline bool operator<=(CD a, CD b) { g_ops.cmp++; return a.v <= b.v; }
inline CD& operator+=(CD& a, CD b) { a = a + b; return a; }
inline CD& operator-=(CD& a, CD b) { a = a - b; return a; }
inline CD sqrt_(CD a) { g_ops.sqrt++; return CD(std::sqrt(a.v)); }
inline CD pow_(CD a, CD b) { g_ops.pow++; return CD(std::pow(a.v, b.v)); }
inline CD abs_(CD a) { g_ops.sgn++; return CD(std::fabs(a.v)); }
inline CD min_(CD a, CD b) { g_ops.minmax++; return CD(a.v < b.v ? a.v : b.v); }
inline CD max_(CD a, CD b) { g_ops.minmax++; return CD(a.v > b.v ? a.v : b.v); }
inline double val(CD a) { return a.v; }

inline double sqrt_(double a) { return std::sqrt(a); }
inline double pow_(double a, double b) { return std::pow(a, b); }
inline double abs_(double a) { return std::fabs(a); }
inline double min_(double a, double b) { return a < b ? a : b; }
inline double max_(double a, double b) { return a > b ? a : b; }
inline double val(double a) { return a; }

// ----------------------------------------------------------------------------
// Field order of the evolved state (cell averages, per unit volume):
//   0 rho, 1..3 s (momentum), 4 E (gas energy), 5 tau (entropy tracer),
//   6..8 z (spin angular momentum), 9.. species partial densities.
// Primitive order (what PPM reconstructs):
//   0 rho, 1..3 v = s/rho, 4 eps (internal energy density), 5 tau, 6..8 z,
//   9.. species.  Reading: the paper reconstructs "the evolution variables";
//   velocity and internal energy replace momentum and total energy so that
//   the face states are physical, tau/z/species are reconstructed as given.
enum { RHO = 0, SX = 1, SY = 2, SZ = 3, EGAS = 4, TAU = 5, ZX = 6, ZY = 7, ZZ = 8, SP0 = 9 };
static const int kMaxF = 16;

struct Params {
  double gamma;   // ratio of specific heats
  double omega;   // frame angular velocity about +z
  double eta1;    // dual-energy selection threshold (Bryan et al. 1995)
  double eta2;    // dual-energy tracer-resync threshold (Bryan et al. 1995)
  int N;          // interior cells per sub-grid edge
  int G;          // ghost depth (3 for the 5-point stencil)
  int nf;         // number of fields = 9 + species
  int face_points;  // 9: flux at the 9 points of each face, Simpson sum (the new module);
                    // 1: flux at the face centre only (the old module, Sec. III-B)
  int contact;      // 1: PPM contact-discontinuity detection and steepening of the
                    // density and species lines (optional in Sec. III-B); 0: off
  int spin;         // 1: the spin of a cell feeds back into the velocity
                    // reconstructed at its quadrature points (spin_feedback); 0: off
};

// Primitive recovery of one cell (Sec. III-B; dual energy after Bryan 1995).
// eps = E - rho|v|^2/2 unless that is below eta1*E, where the tracer gives
// eps = tau^gamma (tau is the entropy tracer, a per-volume density).
template <class T>
void primitives(const Params& P, const T* u, T* q) {
  const T rho = u[RHO];
  const T vx = u[SX] / rho, vy = u[SY] / rho, vz = u[SZ] / rho;
  const T ek = (T(0.5) * rho) * ((vx * vx + vy * vy) + vz * vz);
  const T eE = u[EGAS] - ek;
  const T eps = (eE > T(P.eta1) * u[EGAS]) ? eE : pow_(u[TAU], T(P.gamma));
  q[RHO] = rho;
  q[1] = vx; q[2] = vy; q[3] = vz;
  q[4] = eps;
  for (int k = TAU; k < P.nf; ++k) q[k] = u[k];
}

// PPM on one line (Colella & Woodward 1984, as cited in Sec. III-B): the five
// samples s[0..4] = q(i-2d) .. q(i+2d) give qp = value of cell i at its end
// towards +d and qm = value at its end towards -d.
//   delta_j = q_{j+1} - q_j
//   Delta_j = 0 if delta_j*delta_{j-1} <= 0, else
//             sgn(delta_j) min(2|delta_{j-1}|, 2|delta_j|, |delta_{j-1}+delta_j|/2)
//   qp = (q0+q1)/2 - (Delta_1-Delta_0)/6,  qm = (q_{-1}+q0)/2 - (Delta_0-Delta_{-1})/6
// then, with a steepening weight eta > 0 (contact_eta below), the blend of
// both values with the limited-slope extrapolations from the neighbours
// (Colella & Woodward 1984, discontinuity detection):
//   qp <- (1-eta) qp + eta (q1 - Delta_1/2),  qm <- (1-eta) qm + eta (q-1 + Delta_-1/2),
// then the monotonicity fix-ups, in this order: local extremum -> flatten;
// overshoot towards -d -> qm = 3q0-2qp; overshoot towards +d -> qp = 3q0-2qm.
// With uq (non-null), also returns the unlimited pair uq[0] = towards +d,
// uq[1] = towards -d, from central slopes Delta_j = (delta_{j-1}+delta_j)/2
// and no fix-ups (what the limiter would leave untouched).
template <class T>
void ppm_line(const T s[5], T& qp, T& qm, T* uq = nullptr, T eta = T(0.0)) {
  const T sixth = T(1.0 / 6.0);
  T dl[4];
  for (int j = 0; j < 4; ++j) dl[j] = s[j + 1] - s[j];  // delta_{j-2}
  T D[3];                                               // Delta_{-1}, Delta_0, Delta_1
  for (int k = 0; k < 3; ++k) {
    const T a = dl[k], b = dl[k + 1];  // delta_{j-1}, delta_j
    if (a * b <= T(0.0)) {
      D[k] = T(0.0);
    } else {
      const T m = min_(min_(T(2.0) * abs_(a), T(2.0) * abs_(b)), T(0.5) * abs_(a + b));
      D[k] = (b > T(0.0)) ? m : -m;
    }
  }
  const T q0 = s[2];
  qp = T(0.5) * (q0 + s[3]) - (D[2] - D[1]) * sixth;
  qm = T(0.5) * (s[1] + q0) - (D[1] - D[0]) * sixth;
  if (val(eta) > 0.0) {  // (not a counted comparison: eta is 0 with steepening off)
    const T keep = T(1.0) - eta;
    qp = keep * qp + eta * (s[3] - T(0.5) * D[2]);
    qm = keep * qm + eta * (s[1] + T(0.5) * D[0]);
  }
  if ((qp - q0) * (q0 - qm) <= T(0.0)) {
    qp = q0;
    qm = q0;
  } else {
    const T dq = qp - qm;
    const T lhs = dq * (q0 - T(0.5) * (qp + qm));
    const T rhs = (dq * dq) * sixth;
    if (lhs > rhs) {
      qm = T(3.0) * q0 - T(2.0) * qp;
    } else if (lhs < -rhs) {
      qp = T(3.0) * q0 - T(2.0) * qm;
    }
  }
  if (!uq) return;
  T Du[3];
  for (int k = 0; k < 3; ++k) Du[k] = T(0.5) * (dl[k] + dl[k + 1]);
  uq[0] = T(0.5) * (q0 + s[3]) - (Du[2] - Du[1]) * sixth;
  uq[1] = T(0.5) * (s[1] + q0) - (Du[1] - Du[0]) * sixth;
}

// Steepening weight of one line (Colella & Woodward 1984, discontinuity
// detection, with their constants eps = 0.01, eta1 = 20, eta2 = 0.05, and
// their contact criterion for gas dynamics with K0 = 0.1).  a[0..4] are the
// five samples of the steepened field, rho/p the density and pressure of the
// two neighbours on the same line (index 0: towards -d, 1: towards +d).
//   The jump must be a contact, not a shock: the relative density jump,
//   times gamma K0, at least the relative pressure jump,
//     gamma K0 |rho_1 - rho_0| / min(rho) >= |p_1 - p_0| / min(p),
//   taken multiplied through by the two (positive) minima:
//     gamma K0 |rho_1 - rho_0| min(p) >= |p_1 - p_0| min(rho).
//   With the second differences d2_m = (a_-2 + a_0) - 2a_-1 and
//   d2_p = (a_0 + a_2) - 2a_1 (the 1/(6 h^2) of the nonuniform form cancels;
//   each is summed symmetrically, so that a reversed line rounds alike):
//     eta~ = 0 if d2_m d2_p > 0 (no inflection at the cell), or if
//            |a_1 - a_-1| <= eps min(|a_1|, |a_-1|) (no jump to speak of),
//     else eta~ = -(d2_p - d2_m) / (6 (a_1 - a_-1));
//     eta = max(0, min(eta1 (eta~ - eta2), 1)).
// The formula is free of the spacing, so it serves the diagonal lines as it
// serves the axes.
template <class T>
T contact_eta(const Params& P, const T a[5], const T rho[2], const T p[2]) {
  const T K0 = T(0.1), eps = T(0.01), eta1 = T(20.0), eta2 = T(0.05);
  const T drho = abs_(rho[1] - rho[0]), dp = abs_(p[1] - p[0]);
  if (((T(P.gamma) * K0) * drho) * min_(p[0], p[1]) < dp * min_(rho[0], rho[1])) return T(0.0);
  const T d2m = (a[0] + a[2]) - T(2.0) * a[1];
  const T d2p = (a[2] + a[4]) - T(2.0) * a[3];
  if (T(0.0) < d2m * d2p) return T(0.0);
  const T jump = a[3] - a[1];
  if (abs_(jump) <= eps * min_(abs_(a[3]), abs_(a[1]))) return T(0.0);
  const T et = -(d2p - d2m) / (T(6.0) * jump);
  return max_(T(0.0), min_(eta1 * (et - eta2), T(1.0)));
}
inline bool steepened_field(int k) { return k == RHO || k >= SP0; }

// Significant limiter activity (the learned indicator's label): on a line
// of field k through a cell, the limited pair differs from the unlimited one
// by more than 1e-4 of the field's scale at the cell: |q0| for density,
// internal energy, tracer and species, |vx|+|vy|+|vz|+c for velocities.
// The spin fields are always limited and never labelled.  (Differences below
// that are rounding-level noise, e.g. numerical precursors ahead of a shock.)
static const double kLabelTol = 1e-4;
inline bool spin_field(int k) { return k == ZX || k == ZY || k == ZZ; }

// Physical state on one side of a quadrature point x_q on a face with normal
// axis a.  The frame rotates about +z at omega; momentum and energy are the
// inertial ones expressed in the rotating frame (reading), so the advection
// velocity is u = v - omega z_hat x x_q and the pressure work uses v.
//   s = rho v, E = eps + rho|v|^2/2, p = (gamma-1) eps, c = sqrt(gamma p/rho)
//   F = (rho u_n, s u_n + p e_a, E u_n + p v_a, tau u_n, z u_n, species u_n)
template <class T>
void side_state(const Params& P, const T* q, int a, const T xq[3], T* U, T* F, T& speed) {
  const T rho = q[RHO], vx = q[1], vy = q[2], vz = q[3], eps = q[4];
  const T ek = (T(0.5) * rho) * ((vx * vx + vy * vy) + vz * vz);
  const T E = eps + ek;
  const T p = T(P.gamma - 1.0) * eps;
  const T c = sqrt_((T(P.gamma) * p) / rho);
  const T om = T(P.omega);
  const T u[3] = {vx + om * xq[1], vy - om * xq[0], vz};
  const T v[3] = {vx, vy, vz};
  const T un = u[a];
  U[RHO] = rho;
  U[SX] = rho * vx; U[SY] = rho * vy; U[SZ] = rho * vz;
  U[EGAS] = E;
  for (int k = TAU; k < P.nf; ++k) U[k] = q[k];
  for (int k = 0; k < P.nf; ++k) F[k] = U[k] * un;
  F[SX + a] = F[SX + a] + p;
  F[EGAS] = F[EGAS] + p * v[a];
  speed = abs_(un) + c;
}

// Kurganov-Tadmor central flux at one quadrature point (Sec. III-B, citing
// Kurganov & Tadmor 2000), with the symmetric local speed
// a_q = max(|u_n,L| + c_L, |u_n,R| + c_R):
//   F_q = (F_L + F_R)/2 - a_q (U_R - U_L)/2.
template <class T>
void point_flux(const Params& P, const T* qL, const T* qR, int a, const T xq[3], T* Fq, T& aq) {
  T UL[kMaxF], FL[kMaxF], UR[kMaxF], FR[kMaxF], sL, sR;
  side_state(P, qL, a, xq, UL, FL, sL);
  side_state(P, qR, a, xq, UR, FR, sR);
  aq = max_(sL, sR);
  for (int k = 0; k < P.nf; ++k)
    Fq[k] = T(0.5) * (FL[k] + FR[k]) - (T(0.5) * aq) * (UR[k] - UL[k]);
}

// Spin feedback into the reconstructed velocity.  PARITY UNPINNED beyond the
// checks in tests/test_oracle_spin.py (the reduction to the plain method at
// z = 0, conservation, the rigid-rotation moment of inertia, dissipation of a
// uniform spin, the sound-speed bound): the paper names the rotating-frame
// and spin treatment of the hydro module but defers its definition to the
// Octo-Tiger method paper.
// Reading, in the manner of Despres & Labourasse (2015): the spin angular
// momentum density z of a cell (its angular momentum about its own centre,
// per unit volume) is carried as a rigid rotation of the cell's material,
// omega = z / I with I = rho h^2 / 6 the moment of inertia per unit volume of
// a uniform cube of side h about an axis through its centre, and the
// velocity reconstructed at a point x_q of the cell's surface gains that
// rotation's velocity omega x (x_q - x_c).  The rotation is taken as
// subsonic: where its fastest point, a corner at |omega| h sqrt(3) / 2,
// would outrun the cell's sound speed c = sqrt(gamma (gamma-1) eps / rho),
// omega is scaled down to reach c there (c = 0 for eps <= 0).  rho, eps and
// z are the cell's primitives (Q at stored cell index c).
template <class T>
void spin_feedback(const Params& P, const std::vector<T>& Q, long c, double h, const T xq[3], const T xc[3], T* q) {
  const int S = P.N + 2 * P.G;
  const long S3 = (long)S * S * S;
  const T rho = Q[RHO * S3 + c], eps = Q[EGAS * S3 + c];
  const T I = (rho * T(h * h)) / T(6.0);
  T om[3] = {Q[ZX * S3 + c] / I, Q[ZY * S3 + c] / I, Q[ZZ * S3 + c] / I};
  const T wabs = sqrt_((om[0] * om[0] + om[1] * om[1]) + om[2] * om[2]);
  const T vcorner = wabs * T(0.5 * h * std::sqrt(3.0));
  const T cs2 = (T(P.gamma * (P.gamma - 1.0)) * eps) / rho;
  const T cs = T(0.0) < cs2 ? sqrt_(cs2) : T(0.0);
  if (cs < vcorner) {
    const T theta = cs / vcorner;
    for (int m = 0; m < 3; ++m) om[m] = theta * om[m];
  }
  const T r[3] = {xq[0] - xc[0], xq[1] - xc[1], xq[2] - xc[2]};
  q[1] = q[1] + (om[1] * r[2] - om[2] * r[1]);
  q[2] = q[2] + (om[2] * r[0] - om[0] * r[2]);
  q[3] = q[3] + (om[0] * r[1] - om[1] * r[0]);
}

// Newton-Cotes (Simpson) weights on the 3x3 face points: (1,4,1)x(1,4,1)/36.
// Reading of the paper's "Newtonian quadrature" for 3 points per direction.
inline double nc_weight(int t1, int t2) {
  static const double w1[3] = {1.0, 4.0, 1.0};
  return (w1[t1 + 1] * w1[t2 + 1]) / 36.0;
}

// Primitives on every stored cell of a ghost-padded sub-grid:
// U [nf][S^3] -> Q [nf][S^3].
template <class T>
void primitives_subgrid(const Params& P, const T* U, std::vector<T>& Q) {
  const int S = P.N + 2 * P.G, nf = P.nf;
  const long S3 = (long)S * S * S;
  Q.assign((size_t)nf * S3, T(0.0));
  T u[kMaxF] = {}, q[kMaxF] = {};
  for (long c = 0; c < S3; ++c) {
    for (int k = 0; k < nf; ++k) u[k] = U[k * S3 + c];
    primitives(P, u, q);
    for (int k = 0; k < nf; ++k) Q[k * S3 + c] = q[k];
  }
}

// Unlimited interface value of the centre cell towards +d on five samples:
// the 4-point formula 7/12 (q0 + q1) - 1/12 (q-1 + q2) (what the PPM
// interface value is when no limiter acts).  Used for cells that the learned
// smoothness indicator marks as smooth.
template <class T>
T unlimited_plus(const T s[5]) {
  return T(7.0 / 12.0) * (s[2] + s[3]) - T(1.0 / 12.0) * (s[1] + s[4]);
}

// Reconstructed value R_i[d] of cell i = (x,y,z) (interior coordinates, may
// be -1 or N on a face-adjacent ghost) at its point x_c + (h/2) d, for every
// primitive: PPM along the line of cell centres i + m d, m = -2..2 (with
// `unlimited`, the 4-point formula for all fields but the spin).  With
// want_flag, returns 1 when the limiter acted significantly on the line.
template <class T>
int recon_point(const Params& P, const std::vector<T>& Q, int x, int y, int z, const int d[3], T* out,
                bool want_flag, bool unlimited = false) {
  const int S = P.N + 2 * P.G, G = P.G;
  const long S3 = (long)S * S * S;
  auto at = [&](int xx, int yy, int zz) -> long { return ((long)(zz + G) * S + (yy + G)) * S + (xx + G); };
  const long c = at(x, y, z);
  double vscale = 0.0;
  if (want_flag) {
    const double rho = val(Q[RHO * S3 + c]), eps = val(Q[4 * S3 + c]);
    vscale = std::fabs(val(Q[1 * S3 + c])) + std::fabs(val(Q[2 * S3 + c])) + std::fabs(val(Q[3 * S3 + c])) +
             std::sqrt(P.gamma * (P.gamma - 1.0) * eps / rho);
  }
  // density and pressure of the two neighbours on the line (contact test)
  T nrho[2] = {T(0.0), T(0.0)}, np_[2] = {T(0.0), T(0.0)};
  if (P.contact && !unlimited) {
    for (int e = 0; e < 2; ++e) {
      const int m = 2 * e - 1;
      const long cn = at(x + m * d[0], y + m * d[1], z + m * d[2]);
      nrho[e] = Q[RHO * S3 + cn];
      np_[e] = T(P.gamma - 1.0) * Q[4 * S3 + cn];
    }
  }
  int fl = 0;
  for (int k = 0; k < P.nf; ++k) {
    T s5[5];
    for (int m = -2; m <= 2; ++m) s5[m + 2] = Q[k * S3 + at(x + m * d[0], y + m * d[1], z + m * d[2])];
    T qp, qm;
    if (unlimited && !spin_field(k)) {
      out[k] = unlimited_plus(s5);
      continue;
    }
    const T eta = (P.contact && steepened_field(k)) ? contact_eta(P, s5, nrho, np_) : T(0.0);
    if (want_flag && !spin_field(k)) {
      T uq[2];
      ppm_line(s5, qp, qm, uq, eta);
      const double scale = (k >= 1 && k <= 3) ? vscale : std::fabs(val(s5[2]));
      const double diff = std::max(std::fabs(val(qp) - val(uq[0])), std::fabs(val(qm) - val(uq[1])));
      if (diff > kLabelTol * scale) fl = 1;
    } else if constexpr (std::is_same<T, CD>::value) {
      const long before = g_ops.total();
      ppm_line(s5, qp, qm, (T*)nullptr, eta);
      g_ppm_ops += g_ops.total() - before;
      g_ppm_calls += 1;
    } else {
      ppm_line(s5, qp, qm, (T*)nullptr, eta);
    }
    out[k] = qp;
  }
  return fl;
}

// One sub-grid, one stage of the semi-discrete operator.
//   U      [nf][S][S][S] cell averages with ghosts filled, S = N + 2G, x fastest
//   origin lower corner of the interior block; h cell width
//   g      optional gravitational acceleration [3][N][N][N] (nullptr: none)
//   dUdt   [nf][N][N][N]
//   amax   max signal speed over every quadrature point of every face of the
//          N^3 interior cells (sub-grid boundary faces included)
//   limflag optional [N][N][N]: 1 where the limiter acted significantly on a
//          line through the cell (the indicator's label, see kLabelTol)
//   smooth  optional [S][S][S]: cells whose lines use the unlimited formula
//          (all fields but the spin, which stays limited)
//   face_flux optional [6][nf+3][N][N]: the sub-grid's boundary faces (slot
//          2a lower, 2a+1 upper face of axis a), per face cell [c][b] (b < c
//          the transverse axes) the face sums and the torque about the
//          adjacent interior cell
template <class T>
void step_subgrid(const Params& P, const T* U, const double origin[3], double h, const T* g, T* dUdt,
                  T* amax, uint8_t* limflag, const uint8_t* smooth = nullptr, T* face_flux = nullptr) {
  const int N = P.N, G = P.G, S = N + 2 * G, nf = P.nf;
  const long S3 = (long)S * S * S;
  auto at = [&](int x, int y, int z) -> long { return ((long)(z + G) * S + (y + G)) * S + (x + G); };

  // 1. primitives on every stored cell
  std::vector<T> Q;
  primitives_subgrid(P, U, Q);

  // 2. reconstructed value of cell (x,y,z) at its point towards direction d
  std::vector<uint8_t> fired((size_t)N * N * N, 0);
  auto recon = [&](int x, int y, int z, const int d[3], T* out) {
    const bool un = smooth && smooth[at(x, y, z)];
    const int fl = recon_point(P, Q, x, y, z, d, out, limflag != nullptr, un);
    if (fl && x >= 0 && x < N && y >= 0 && y < N && z >= 0 && z < N) fired[((long)z * N + y) * N + x] = 1;
  };

  // 3-4. face fluxes: Fbar[a][k] on the a+ face of cell i for i_a in [-1,N-1]
  // and the other two indices in [0,N-1]; torque sums of the two cells.
  const int NF1 = N + 1;
  auto fidx = [&](int a, int x, int y, int z) -> long {
    // face a+ of cell (x,y,z); store with the a-index shifted by +1
    int c[3] = {x, y, z};
    c[a] += 1;
    return ((long)a * NF1 * NF1 * NF1 + ((long)c[2] * NF1 + c[1]) * NF1 + c[0]);
  };
  const long nface = 3L * NF1 * NF1 * NF1;
  std::vector<T> Fbar((size_t)nface * nf), TqL((size_t)nface * 3), TqR((size_t)nface * 3);
  T am = T(0.0);
  bool first = true;
  const T half_h = T(0.5 * h);
  for (int a = 0; a < 3; ++a) {
    const int b = (a == 0) ? 1 : 0;       // first transverse axis
    const int cax = (a == 2) ? 1 : 2;     // second transverse axis
    int lo[3] = {0, 0, 0}, hi[3] = {N, N, N};
    lo[a] = -1;
    hi[a] = N;
    for (int z = lo[2]; z < hi[2]; ++z)
      for (int y = lo[1]; y < hi[1]; ++y)
        for (int x = lo[0]; x < hi[0]; ++x) {
          const int ci[3] = {x, y, z};
          int cr[3] = {x, y, z};
          cr[a] += 1;
          T fsum[kMaxF];
          for (int k = 0; k < nf; ++k) fsum[k] = T(0.0);
          T tl[3] = {T(0.0), T(0.0), T(0.0)}, tr[3] = {T(0.0), T(0.0), T(0.0)};
          for (int t1 = -1; t1 <= 1; ++t1)
            for (int t2 = -1; t2 <= 1; ++t2) {
              if (P.face_points == 1 && (t1 != 0 || t2 != 0)) continue;
              int d[3];
              d[a] = 1;
              d[b] = t1;
              d[cax] = t2;
              int dr[3] = {d[0], d[1], d[2]};
              dr[a] -= 2;  // the same point seen from the right-hand cell
              T xq[3];
              for (int m = 0; m < 3; ++m)
                xq[m] = T(origin[m]) + T(h) * (T(ci[m] + 0.5) + T(0.5 * d[m]));
              T qL[kMaxF], qR[kMaxF], Fq[kMaxF], aq;
              recon(ci[0], ci[1], ci[2], d, qL);
              recon(cr[0], cr[1], cr[2], dr, qR);
              if (P.spin) {
                T xl[3], xr[3];
                for (int m = 0; m < 3; ++m) {
                  xl[m] = T(origin[m]) + T(h) * T(ci[m] + 0.5);
                  xr[m] = T(origin[m]) + T(h) * T(cr[m] + 0.5);
                }
                spin_feedback(P, Q, at(ci[0], ci[1], ci[2]), h, xq, xl, qL);
                spin_feedback(P, Q, at(cr[0], cr[1], cr[2]), h, xq, xr, qR);
              }
              point_flux(P, qL, qR, a, xq, Fq, aq);
              if (first) { am = aq; first = false; }
              else am = max_(am, aq);
              const T w = T(P.face_points == 1 ? 1.0 : nc_weight(t1, t2));
              for (int k = 0; k < nf; ++k) fsum[k] = fsum[k] + w * Fq[k];
              // torque of the momentum flux about each cell centre:
              // (x_q - x_c) x F_s with x_q - x_c = (h/2) d (left), (h/2)(d-2e_a) (right)
              const T Fs[3] = {Fq[SX], Fq[SY], Fq[SZ]};
              T rl[3], rr[3];
              for (int m = 0; m < 3; ++m) { rl[m] = half_h * T(d[m]); rr[m] = half_h * T(dr[m]); }
              const T cl[3] = {rl[1] * Fs[2] - rl[2] * Fs[1], rl[2] * Fs[0] - rl[0] * Fs[2],
                               rl[0] * Fs[1] - rl[1] * Fs[0]};
              const T cr2[3] = {rr[1] * Fs[2] - rr[2] * Fs[1], rr[2] * Fs[0] - rr[0] * Fs[2],
                                rr[0] * Fs[1] - rr[1] * Fs[0]};
              for (int m = 0; m < 3; ++m) {
                tl[m] = tl[m] + w * cl[m];
                tr[m] = tr[m] + w * cr2[m];
              }
            }
          const long f = fidx(a, x, y, z);
          for (int k = 0; k < nf; ++k) Fbar[f * nf + k] = fsum[k];
          for (int m = 0; m < 3; ++m) { TqL[f * 3 + m] = tl[m]; TqR[f * 3 + m] = tr[m]; }
        }
  }

  if (face_flux) {
    const int q = nf + 3;
    for (int a = 0; a < 3; ++a) {
      const int b = (a == 0) ? 1 : 0, cax = (a == 2) ? 1 : 2;
      for (int side = 0; side < 2; ++side) {
        const int f = 2 * a + side;
        for (int pc = 0; pc < N; ++pc)
          for (int pb = 0; pb < N; ++pb) {
            int ci[3];
            ci[a] = side ? N - 1 : -1;
            ci[b] = pb;
            ci[cax] = pc;
            const long fi = fidx(a, ci[0], ci[1], ci[2]);
            T* out = face_flux + (long)f * q * N * N + (long)pc * N + pb;
            for (int k = 0; k < nf; ++k) out[(long)k * N * N] = Fbar[fi * nf + k];
            for (int m = 0; m < 3; ++m)
              out[(long)(nf + m) * N * N] = side ? TqL[fi * 3 + m] : TqR[fi * 3 + m];
          }
      }
    }
  }

  // 4-5. divergence and sources on the interior cells:
  //   dU/dt = -(1/h) sum_a (Fbar_{a,i+1/2} - Fbar_{a,i-1/2})
  //   spin:  dz/dt gets -(1/h) sum over faces of sigma * torque (sigma = +1 on
  //          the a+ face, -1 on the a- face), so that sum(x_c x s + z) is
  //          conserved by the fluxes alone.
  //   frame: ds/dt += -omega z_hat x s = (omega s_y, -omega s_x, 0); the same
  //          rotation of components applies to the spin vector z (reading).
  //          The face torques above take the momentum flux s u_n with the grid
  //          velocity w = -omega z_hat x x = (omega y, -omega x, 0) inside u;
  //          the part s w_n is not a symmetric stress, and its torque belongs
  //          to the change of frame, not to an exchange between orbital and
  //          spin angular momentum.  dz/dt += w(x_c) x s removes it (for a
  //          uniform stream exactly), so that sum (x_c x s + z)_z h^3, which
  //          the frame source on s alone changes by
  //          -omega sum (x_c s_x + y_c s_y) h^3, is conserved for omega != 0
  //          as it is in the continuum (reading).
  //   gravity (optional): ds/dt += rho g, dE/dt += s.g.
  const T inv_h = T(1.0 / h);
  const T om = T(P.omega);
  const long N3 = (long)N * N * N;
  for (int z = 0; z < N; ++z)
    for (int y = 0; y < N; ++y)
      for (int x = 0; x < N; ++x) {
        const int ci[3] = {x, y, z};
        long fp[3], fm[3];
        for (int a = 0; a < 3; ++a) {
          int cm[3] = {x, y, z};
          cm[a] -= 1;
          fp[a] = fidx(a, ci[0], ci[1], ci[2]);
          fm[a] = fidx(a, cm[0], cm[1], cm[2]);
        }
        const long c = ((long)z * N + y) * N + x;
        T du[kMaxF];
        for (int k = 0; k < nf; ++k) {
          const T div = ((Fbar[fp[0] * nf + k] - Fbar[fm[0] * nf + k]) +
                         (Fbar[fp[1] * nf + k] - Fbar[fm[1] * nf + k])) +
                        (Fbar[fp[2] * nf + k] - Fbar[fm[2] * nf + k]);
          du[k] = -(div * inv_h);
        }
        for (int m = 0; m < 3; ++m) {
          const T tq = ((TqL[fp[0] * 3 + m] - TqR[fm[0] * 3 + m]) + (TqL[fp[1] * 3 + m] - TqR[fm[1] * 3 + m])) +
                       (TqL[fp[2] * 3 + m] - TqR[fm[2] * 3 + m]);
          du[ZX + m] = du[ZX + m] - tq * inv_h;
        }
        const long uc = at(x, y, z);
        const T rho = U[RHO * S3 + uc];
        const T s[3] = {U[SX * S3 + uc], U[SY * S3 + uc], U[SZ * S3 + uc]};
        const T zz[3] = {U[ZX * S3 + uc], U[ZY * S3 + uc], U[ZZ * S3 + uc]};
        du[SX] = du[SX] + om * s[1];
        du[SY] = du[SY] - om * s[0];
        du[ZX] = du[ZX] + om * zz[1];
        du[ZY] = du[ZY] - om * zz[0];
        {
          const T xc = T(origin[0]) + T(h) * T(x + 0.5), yc = T(origin[1]) + T(h) * T(y + 0.5);
          const T wx = om * yc, wy = -(om * xc);  // w_z = 0
          du[ZX] = du[ZX] + wy * s[2];
          du[ZY] = du[ZY] - wx * s[2];
          du[ZZ] = du[ZZ] + (wx * s[1] - wy * s[0]);
        }
        if (g) {
          const T gv[3] = {g[0 * N3 + c], g[1 * N3 + c], g[2 * N3 + c]};
          for (int m = 0; m < 3; ++m) du[SX + m] = du[SX + m] + rho * gv[m];
          du[EGAS] = du[EGAS] + ((s[0] * gv[0] + s[1] * gv[1]) + s[2] * gv[2]);
        }
        for (int k = 0; k < nf; ++k) dUdt[k * N3 + c] = du[k];
        if (limflag) limflag[c] = fired[c];
      }
  *amax = am;
}

}  // namespace orc

namespace orc {

// SSP-RK3 stage update of the interior cells (3 hydro iterations per step,
// Sec. IV-A), followed by the dual-energy tracer resync (Bryan et al. 1995):
//   stage k: U <- alpha_k U0 + beta_k (U + dt dU/dt),
//            (alpha, beta) = (0, 1), (3/4, 1/4), (1/3, 2/3)
//   then, where eps_E = E - |s|^2/(2 rho) exceeds eta2 E: tau <- eps_E^(1/gamma).
// U and U0 are ghost-padded [nf][S][S][S]; dUdt is [nf][N][N][N].
template <class T>
void update_subgrid(const Params& P, T* U, const T* U0, const T* dUdt, double dt, int stage) {
  static const double alpha[3] = {0.0, 0.75, 1.0 / 3.0};
  static const double beta[3] = {1.0, 0.25, 2.0 / 3.0};
  const int N = P.N, G = P.G, S = N + 2 * G, nf = P.nf;
  const long S3 = (long)S * S * S, N3 = (long)N * N * N;
  const T a = T(alpha[stage]), b = T(beta[stage]), tdt = T(dt);
  for (int z = 0; z < N; ++z)
    for (int y = 0; y < N; ++y)
      for (int x = 0; x < N; ++x) {
        const long uc = ((long)(z + G) * S + (y + G)) * S + (x + G);
        const long c = ((long)z * N + y) * N + x;
        T u[kMaxF];
        for (int k = 0; k < nf; ++k) {
          const T t = U[k * S3 + uc] + tdt * dUdt[k * N3 + c];
          u[k] = a * U0[k * S3 + uc] + b * t;
        }
        const T rho = u[RHO];
        const T vx = u[SX] / rho, vy = u[SY] / rho, vz = u[SZ] / rho;
        const T ek = (T(0.5) * rho) * ((vx * vx + vy * vy) + vz * vz);
        const T eE = u[EGAS] - ek;
        if (eE > T(P.eta2) * u[EGAS]) u[TAU] = pow_(eE, T(1.0 / P.gamma));
        for (int k = 0; k < nf; ++k) U[k * S3 + uc] = u[k];
      }
}

}  // namespace orc

// ============================================================================
// C entry points (ctypes).  All arrays are host FP64, caller-owned.
extern "C" {

struct orc_params {
  double gamma, omega, eta1, eta2;
  int N, G, nf, face_points, contact, spin;
};

static orc::Params to_p(const orc_params* p) {
  orc::Params P;
  P.gamma = p->gamma; P.omega = p->omega; P.eta1 = p->eta1; P.eta2 = p->eta2;
  P.N = p->N; P.G = p->G; P.nf = p->nf;
  P.face_points = p->face_points == 1 ? 1 : 9;
  P.contact = p->contact ? 1 : 0;
  P.spin = p->spin ? 1 : 0;
  return P;
}

// One stage of the semi-discrete operator on n_sub sub-grids.
//   U [n_sub][nf][S^3], origin [n_sub][3], h [n_sub], g nullable [n_sub][3][N^3]
//   dUdt [n_sub][nf][N^3], amax [n_sub], limflag nullable [n_sub][N^3]
// nthreads <= 0 uses the OpenMP default.
int orc_step(const orc_params* p, int n_sub, const double* U, const double* origin, const double* h,
             const double* g, double* dUdt, double* amax, uint8_t* limflag, double* face_flux, int nthreads) {
  const orc::Params P = to_p(p);
  if (P.nf > orc::kMaxF || P.nf < 10 || P.N < 1 || P.G != 3 || n_sub < 0) return -1;
  const int S = P.N + 2 * P.G;
  const long S3 = (long)S * S * S, N3 = (long)P.N * P.N * P.N;
#ifdef _OPENMP
  const int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
#endif
  for (int s = 0; s < n_sub; ++s) {
    orc::step_subgrid<double>(P, U + (long)s * P.nf * S3, origin + 3L * s, h[s], g ? g + 3L * s * N3 : nullptr,
                              dUdt + (long)s * P.nf * N3, amax + s, limflag ? limflag + (long)s * N3 : nullptr,
                              nullptr, face_flux ? face_flux + (long)s * 6 * (P.nf + 3) * P.N * P.N : nullptr);
  }
  (void)nthreads;
  return 0;
}

// orc_step with a per-cell smoothness mask [n_sub][S^3] (1: unlimited lines).
int orc_step_masked(const orc_params* p, int n_sub, const double* U, const double* origin, const double* h,
                    const double* g, double* dUdt, double* amax, const uint8_t* smooth, int nthreads) {
  const orc::Params P = to_p(p);
  if (P.nf > orc::kMaxF || P.nf < 10 || P.N < 1 || P.G != 3 || n_sub < 0 || !smooth) return -1;
  const int S = P.N + 2 * P.G;
  const long S3 = (long)S * S * S, N3 = (long)P.N * P.N * P.N;
#ifdef _OPENMP
  const int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
#endif
  for (int s = 0; s < n_sub; ++s) {
    orc::step_subgrid<double>(P, U + (long)s * P.nf * S3, origin + 3L * s, h[s], g ? g + 3L * s * N3 : nullptr,
                              dUdt + (long)s * P.nf * N3, amax + s, nullptr, smooth + (long)s * S3);
  }
  (void)nthreads;
  return 0;
}

// RK3 stage update, in place on the interior of U (ghosts untouched).
int orc_update(const orc_params* p, int n_sub, double* U, const double* U0, const double* dUdt, double dt,
               int stage) {
  const orc::Params P = to_p(p);
  if (stage < 0 || stage > 2 || P.nf > orc::kMaxF) return -1;
  const int S = P.N + 2 * P.G;
  const long S3 = (long)S * S * S, N3 = (long)P.N * P.N * P.N;
  for (int s = 0; s < n_sub; ++s)
    orc::update_subgrid<double>(P, U + (long)s * P.nf * S3, U0 + (long)s * P.nf * S3, dUdt + (long)s * P.nf * N3,
                                dt, stage);
  return 0;
}

// Primitive recovery of one cell (nf values in, nf values out).
void orc_primitives(const orc_params* p, const double* u, double* q) {
  const orc::Params P = to_p(p);
  orc::primitives<double>(P, u, q);
}

// PPM on one line of five samples; returns 1 when the limited pair differs
// from the unlimited (central-slope, no fix-up) pair.
int orc_ppm_line(const double* s5, double* qp, double* qm) {
  double uq[2];
  orc::ppm_line<double>(s5, *qp, *qm, uq);
  return (*qp != uq[0] || *qm != uq[1]) ? 1 : 0;
}

// PPM on one line with a given steepening weight eta (no unlimited pair).
void orc_ppm_line_eta(const double* s5, double eta, double* qp, double* qm) {
  orc::ppm_line<double>(s5, *qp, *qm, nullptr, eta);
}

// Steepening weight of one line: a5 the steepened field's five samples,
// rho2/p2 the density and pressure of the neighbours (-d, +d).
double orc_contact_eta(const orc_params* p, const double* a5, const double* rho2, const double* p2) {
  const orc::Params P = to_p(p);
  return orc::contact_eta<double>(P, a5, rho2, p2);
}

// The spin feedback's velocity increment at offset r from the centre of a
// cell of density rho, internal energy density eps, spin density z[3] and
// width h (spin_feedback on a one-cell array).
void orc_spin_velocity(const orc_params* p, double rho, double eps, const double* z, double h, const double* r,
                       double* dv) {
  orc::Params P = to_p(p);
  P.N = 1;
  P.G = 0;
  std::vector<double> Q(orc::kMaxF, 0.0);
  double q[orc::kMaxF] = {};
  Q[orc::RHO] = rho;
  Q[orc::EGAS] = eps;
  Q[orc::ZX] = z[0];
  Q[orc::ZY] = z[1];
  Q[orc::ZZ] = z[2];
  const double xc[3] = {0.0, 0.0, 0.0};
  orc::spin_feedback<double>(P, Q, 0, h, r, xc, q);
  dv[0] = q[1];
  dv[1] = q[2];
  dv[2] = q[3];
}

// Central flux at one quadrature point from primitive states qL, qR.
void orc_point_flux(const orc_params* p, const double* qL, const double* qR, int axis, const double* xq,
                    double* Fq, double* aq) {
  const orc::Params P = to_p(p);
  orc::point_flux<double>(P, qL, qR, axis, xq, Fq, *aq);
}

// Reconstructed values R_i[d] for a list of (cell, direction) requests on
// one ghost-padded sub-grid: cells/dirs [n][3] (interior coordinates),
// out [n][nf], flags [n] (limiter changed a value on that line).
void orc_face_values(const orc_params* p, const double* U, int n, const int* cells, const int* dirs, double* out,
                     int* flags) {
  const orc::Params P = to_p(p);
  std::vector<double> Q;
  orc::primitives_subgrid<double>(P, U, Q);
  for (int i = 0; i < n; ++i) {
    const int d[3] = {dirs[3 * i], dirs[3 * i + 1], dirs[3 * i + 2]};
    const int f = orc::recon_point<double>(P, Q, cells[3 * i], cells[3 * i + 1], cells[3 * i + 2], d,
                                           out + (long)i * P.nf, true);
    if (flags) flags[i] = f;
  }
}

// Operation count of one sub-grid stage (step) and of one update, through the
// counting scalar: out[0..7] = add, mul, div, sqrt, pow, cmp, minmax, sgn for
// the step; out[8..15] the same for the update; out[16] = operations inside
// PPM line evaluations of the step, out[17] = number of those evaluations.
void orc_count_ops(const orc_params* p, const double* U, const double* origin, double h, long* out) {
  const orc::Params P = to_p(p);
  const int S = P.N + 2 * P.G;
  const long S3 = (long)S * S * S, N3 = (long)P.N * P.N * P.N;
  std::vector<orc::CD> Uc((size_t)P.nf * S3), dU((size_t)P.nf * N3);
  for (size_t i = 0; i < Uc.size(); ++i) Uc[i] = orc::CD(U[i]);
  orc::CD am;
  orc::g_ops = orc::Ops();
  orc::g_ppm_ops = 0;
  orc::g_ppm_calls = 0;
  orc::step_subgrid<orc::CD>(P, Uc.data(), origin, h, nullptr, dU.data(), &am, nullptr);
  const orc::Ops a = orc::g_ops;
  out[16] = orc::g_ppm_ops;
  out[17] = orc::g_ppm_calls;
  std::vector<orc::CD> U0 = Uc;
  orc::g_ops = orc::Ops();
  orc::update_subgrid<orc::CD>(P, Uc.data(), U0.data(), dU.data(), 1e-6, 1);
  const orc::Ops b = orc::g_ops;
  const orc::Ops* o[2] = {&a, &b};
  for (int i = 0; i < 2; ++i) {
    out[8 * i + 0] = o[i]->add; out[8 * i + 1] = o[i]->mul; out[8 * i + 2] = o[i]->div;
    out[8 * i + 3] = o[i]->sqrt; out[8 * i + 4] = o[i]->pow; out[8 * i + 5] = o[i]->cmp;
    out[8 * i + 6] = o[i]->minmax; out[8 * i + 7] = o[i]->sgn;
  }
}

}  // extern "C"
