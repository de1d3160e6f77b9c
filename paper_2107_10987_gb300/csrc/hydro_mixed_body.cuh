// hydro_mixed_body.cuh -- one sub-grid of the mixed-precision hydro step.
// The body is shared by the step kernel (hydro_step_mixed.cu) and the fused
// uniform-mesh RK3 step (hydro_rk3_fused.cu).  They differ only in where the
// sub-grid's state comes from and where its results go (the Io policy below).
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
#pragma once
#include <type_traits>
#include "hydro_mixed.cuh"

namespace hyd {

constexpr int kThreadsMx = NROW;  // 192

// Dynamic shared memory of one CTA: FP32 primitives [F][S3], then two
// [S3] byte arrays of smooth flags (learned indicator), then the FP32 cell-
// centre coordinates x_c, y_c of the reconstructed cells (sub_coords).
constexpr size_t kMixedSmemBytes = (size_t)F * S3 * sizeof(float) + 2 * S3 + 2 * (N + 2) * sizeof(float);

// The FP32 x and y cell-centre coordinates of the cells -1 .. N of a tile
// (cell offsets offx, offy in its sub-grid), x_c = fl(o + h (off + i + 1/2))
// (an FP64 fma rounded once to FP32), coord[a * (N + 2) + i + 1]: computed
// once per tile instead of at every quadrature point (the FP64 pipe is 1/64
// of the FP32 rate).  Threads 0 .. 2(N+2)-1 write; the caller's next barrier
// publishes them.
__device__ __forceinline__ void sub_coords(float* coord, double hd, double ox, double oy, int offx, int offy) {
  const int t = threadIdx.x;
  if (t < 2 * (N + 2)) {
    const bool y = t >= N + 2;
    coord[t] = (float)fma(hd, (t % (N + 2) - 1 + (y ? offy : offx)) + 0.5, y ? oy : ox);
  }
}

// This thread's row: axis a, transverse axes b < cx at positions pb, pc.
// Warp w of the axis takes pb in [4w, 4w+4) x pc in [0, 8).  With the cell
// strides (1, 14, 196) every FP32 stencil load of a warp then spans 32
// (y rows) or 16 (x and z rows) distinct banks: 1- or 2-way conflicts,
// against 2- to 4-way with pb running fastest over the warp.
struct RowMap {
  int a, b, cx, pb, pc, sa, sb, sc;
};
__device__ __forceinline__ RowMap row_map(int tid) {
  static_assert(N == 8 && S == 14, "row-to-warp map assumes 8^3 interiors with 3-cell ghosts");
  RowMap R;
  R.a = tid / (N * N);
  const int r = tid % (N * N);
  R.pb = ((r >> 5) << 2) | (r & 3);
  R.pc = (r & 31) >> 2;
  R.b = (R.a == 0) ? 1 : 0;
  R.cx = (R.a == 2) ? 1 : 2;
  R.sa = axis_stride(R.a);
  R.sb = axis_stride(R.b);
  R.sc = axis_stride(R.cx);
  return R;
}

// The end of one interior cell (x, y, z) of a tile (its compact index c and
// padded index uc are the tile's; offx, offy: the tile's cell offsets in its
// sub-grid): dU/dt from its per-axis differences of face sums,
// D_a[q] = Fbar_a(i+1/2) - Fbar_a(i-1/2) for the F fluxes and the torque
// differences for q >= F (FP64), summed as (D_x + D_y) + D_z: s01(q) gives
// D_x + D_y, d2(q) gives D_z.  Then the rotating-frame, spin and gravity
// sources, and io.store.  Every operation is explicitly rounded or fused,
// so that both sub-grid decompositions and every kernel give the same bits.
template <class Io, class S01, class D2>
__device__ __forceinline__ void finish_cell(const StepArgs64& A, const Io& io, const typename Io::Sub& sub,
                                            int offx, int offy, int x, int y, int z, const S01& s01, const D2& d2,
                                            double hd, double inv_h, const double o[3]) {
  const int c = (z * N + y) * N + x;
  const int uc = ((z + G) * S + (y + G)) * S + (x + G);
  const double om = A.P.omega;
  double du[F];
#pragma unroll
  for (int k = 0; k < F; ++k) du[k] = -__dmul_rn(__dadd_rn(s01(k), d2(k)), inv_h);
#pragma unroll
  for (int m = 0; m < 3; ++m) du[ZX + m] = __dsub_rn(du[ZX + m], __dmul_rn(__dadd_rn(s01(F + m), d2(F + m)), inv_h));
  // The sources' products and sums are written as explicit FMAs and
  // rounded operations, so that every kernel instance rounds them alike.
  double uin[F];
  io.own(sub, c, uc, uin);
  const double sx = uin[SX], sy = uin[SY], sz = uin[SZ];
  du[SX] = fma(om, sy, du[SX]);
  du[SY] = fma(-om, sx, du[SY]);
  du[ZX] = fma(om, uin[ZY], du[ZX]);
  du[ZY] = fma(-om, uin[ZX], du[ZY]);
  {
    // spin source w(x_c) x s, w = -omega z_hat x x_c: removes the torque
    // that the frame part s w_n of the momentum flux leaves in the face
    // torques, so that sum (x_c x s + z)_z is conserved for omega != 0
    const double xc = __dadd_rn(o[0], __dmul_rn(hd, (x + offx) + 0.5));
    const double yc = __dadd_rn(o[1], __dmul_rn(hd, (y + offy) + 0.5));
    const double wx = __dmul_rn(om, yc), wy = -__dmul_rn(om, xc);
    du[ZX] = fma(wy, sz, du[ZX]);
    du[ZY] = fma(-wx, sz, du[ZY]);
    du[ZZ] = __dadd_rn(du[ZZ], fma(wx, sy, -__dmul_rn(wy, sx)));
  }
  if (A.g) {
    double gx, gy, gz;
    io.grav(sub, c, gx, gy, gz);
    const double rho = uin[RHO];
    du[SX] = fma(rho, gx, du[SX]);
    du[SY] = fma(rho, gy, du[SY]);
    du[SZ] = fma(rho, gz, du[SZ]);
    du[EGAS] = __dadd_rn(du[EGAS], fma(sz, gz, fma(sy, gy, __dmul_rn(sx, gx))));
  }
  io.store(sub, c, uc, du, uin);
}

// One 8^3 tile (a sub-grid, or an octant of a 16^3 sub-grid) of work unit s.
// Io supplies the state and takes the results; all cell indices are the
// tile's own (padded 14^3, interior 8^3):
//   typename Io::Sub io.begin(s)                    per-unit context
//   io.sidx(sub), io.offx(sub), io.offy(sub)  the sub-grid (for h, origin)
//                             and the tile's x and y cell offsets in it
//   io.load(sub, c, u)        conserved state u[F] of padded cell c
//   Io::kPrims, io.load_prims(sub, c, q)  if kPrims: the FP32 primitives
//                             q[F] of padded cell c instead (prims_mixed of
//                             its state, non-physical cells reported by the
//                             producer)
//   io.own(sub, c, uc, u)     conserved state of interior cell c (padded index uc)
//   io.store(sub, c, uc, du, u)  dU/dt of interior cell c; u is its state from own()
//   io.grav(sub, c, gx, gy, gz)  gravity at interior cell c
//   io.face(sub, f, q, pc, pb, v)  boundary-face value (tile face f)
//   io.amax(sub, m)           the tile's maximum signal speed (thread 0)
// Qf: the CTA's dynamic shared memory; red: [kThreadsMx / 32] floats of
// shared memory; D: the CTA's scratch (kScratchPerSub doubles).  Ends with
// a barrier, so the next sub-grid may reuse all of them.
// kContact: contact steepening of the density and species lines (line10fc).
template <bool kGate, bool kContact = false, bool kSpin = false, class Io>
__device__ __forceinline__ void mixed_subgrid(const StepArgs64& A, const Io& io, int s, const RowMap& R, float* Qf,
                                              float* red, double* __restrict__ D) {
  uint8_t* smooth = reinterpret_cast<uint8_t*>(Qf + F * S3);
  float* coord = reinterpret_cast<float*>(smooth + 2 * S3);
  const int tid = threadIdx.x;
  const int a = R.a, b = R.b, pb = R.pb, pc = R.pc, sa = R.sa, sb = R.sb, sc = R.sc;
  const typename Io::Sub sub = io.begin(s);
  const int si = io.sidx(sub), offx = io.offx(sub), offy = io.offy(sub);
  const double hd = A.h[si];
  const StepParamsF PF{(float)A.P.gamma, (float)A.P.gm1, (float)A.P.omega, kSpin ? 1 : 0,
                       kSpin ? (float)(3.0 / hd) : 0.f};
  const double o[3] = {A.origin[3 * si + 0], A.origin[3 * si + 1], A.origin[3 * si + 2]};
  sub_coords(coord, hd, o[0], o[1], offx, offy);

  // ---- 1-2. load the FP64 state, recover primitives, store FP32 ---------
  // (an Io with kPrims supplies the primitives, recovered once per cell by
  // whoever produced the state, and reports non-physical cells itself)
  bool bad = false;
  for (int c = tid; c < S3; c += kThreadsMx) {
    float q[F];
    if constexpr (Io::kPrims) {
      io.load_prims(sub, c, q);
    } else {
      double u[F];
      io.load(sub, c, u);
      bad |= !prims_mixed(u, A.P.eta1, PF.gamma, q);
    }
#pragma unroll
    for (int k = 0; k < F; ++k) Qf[k * S3 + c] = q[k];
  }
  if (bad) atomicOr(A.status, 1u);
  __syncthreads();

  // ---- 2b. learned smoothness indicator (gate_phase) ---------------------
  if (kGate)
    gate_phase<float, kThreadsMx>(Qf, PF.gm1, A.gate_w, A.gate_logit_thr, A.gate_zero_smooth, smooth, smooth + S3);

  // ---- 3. row sweep in FP32 --------------------------------------------
  const float h = (float)hd, half_h = 0.5f * h;
  float amax = 0.f;
  float plus[9][F];
  // the previous face's sums and right-cell torques, converted to FP64 once
  // (exact conversions of the FP32 sums)
  double fprev[F], trprev[3];
  const int c0 = ((axis_comp(2, a, b, 0, pb, pc) + G) * S + (axis_comp(1, a, b, 0, pb, pc) + G)) * S +
                 (axis_comp(0, a, b, 0, pb, pc) + G);
  const int npt = A.P.face_points;
#pragma unroll 1
  for (int j = -1; j <= N; ++j) {
    const int cj = c0 + j * sa;
    // face j-1/2: completed groups S (fluxes, left-cell torques) and the
    // group being summed, G
    float Sf[F], Stl[3], Gf[F], Gtl[3];
    bool first = true;
#pragma unroll
    for (int k = 0; k < F; ++k) Gf[k] = 0.f;
#pragma unroll
    for (int m = 0; m < 3; ++m) Gtl[m] = 0.f;
    // cell-centre coordinates of the left cell j - 1 (FP64 -> FP32 once; an
    // explicit FMA, so that every kernel instance rounds them alike)
    const float xc = coord[axis_comp(0, a, b, j - 1, pb, pc) + 1],
                yc = coord[(N + 2) + axis_comp(1, a, b, j - 1, pb, pc) + 1];
    // the 9 face points as 4 mirrored pairs and the centre (p = 4); with one
    // flux point per face (the old module) only the centre.  Pair p's two
    // points are points 2p and 2p + 1 of the face's summation order.
    // pair p (kTwo) or the centre p = 4: its lines through cell j, the face
    // points they give with the previous cell's plus-states, and the new
    // plus-states
    auto pair_step = [&](int p, auto two) {
      constexpr bool kTwo = decltype(two)::value;
      const int t1 = p / 3 - 1, t2 = p % 3 - 1;
      float qpA[F], qmA[F], qpB[F], qmB[F];
      if (kGate && smooth[cj]) {
        line10u(Qf, cj, sa + t1 * sb + t2 * sc, qpA, qmA);
        if (kTwo) line10u(Qf, cj, sa - t1 * sb - t2 * sc, qpB, qmB);
      } else if (kContact) {
        const float gk0 = __fmul_rn(PF.gamma, 0.1f);
        line10fc(Qf, cj, sa + t1 * sb + t2 * sc, gk0, PF.gm1, qpA, qmA);
        if (kTwo) line10fc(Qf, cj, sa - t1 * sb - t2 * sc, gk0, PF.gm1, qpB, qmB);
      } else {
        line10f(Qf, cj, sa + t1 * sb + t2 * sc, qpA, qmA);
        if (kTwo) line10f(Qf, cj, sa - t1 * sb - t2 * sc, qpB, qmB);
      }
      if constexpr (kSpin) {
        // the cell's spin fed back into the velocity at both ends of both
        // lines (spin_dv32; the plane sweep's values, bit for bit)
        const float rc = Qf[RHO * S3 + cj], ec = Qf[EGAS * S3 + cj], zx = Qf[ZX * S3 + cj],
                    zy = Qf[ZY * S3 + cj], zz = Qf[ZZ * S3 + cj], gg1 = __fmul_rn(PF.gamma, PF.gm1);
        float dv[3];
        spin_dv32(rc, ec, zx, zy, zz, PF.k3h, gg1, axis_comp(0, a, b, 1, t1, t2), axis_comp(1, a, b, 1, t1, t2),
                  axis_comp(2, a, b, 1, t1, t2), dv);
#pragma unroll
        for (int m = 0; m < 3; ++m) {
          qpA[1 + m] = __fadd_rn(qpA[1 + m], dv[m]);
          qmA[1 + m] = __fsub_rn(qmA[1 + m], dv[m]);
        }
        if (kTwo) {
          spin_dv32(rc, ec, zx, zy, zz, PF.k3h, gg1, axis_comp(0, a, b, 1, -t1, -t2),
                    axis_comp(1, a, b, 1, -t1, -t2), axis_comp(2, a, b, 1, -t1, -t2), dv);
#pragma unroll
          for (int m = 0; m < 3; ++m) {
            qpB[1 + m] = __fadd_rn(qpB[1 + m], dv[m]);
            qmB[1 + m] = __fsub_rn(qmB[1 + m], dv[m]);
          }
        }
      }
      if (j >= 0) {
        // the pair's two points (n = 2p, 2p + 1) in the two lanes; the centre
        // in both
        const int nA = 2 * p, nB = kTwo ? nA + 1 : nA;
        const int u1A = face_u1(nA), u2A = face_u2(nA), u1B = face_u1(nB), u2B = face_u2(nB);
        const int ptA = (u1A + 1) * 3 + (u2A + 1), ptB = (u1B + 1) * 3 + (u2B + 1);
        float2 dL[3];
#pragma unroll
        for (int m = 0; m < 3; ++m)
          dL[m] = f2((float)axis_comp(m, a, b, 1, u1A, u2A), (float)axis_comp(m, a, b, 1, u1B, u2B));
        const float2 xq = fma2(f2(half_h), dL[0], f2(xc)), yq = fma2(f2(half_h), dL[1], f2(yc));
        const float wA = face_w(u1A, u2A, npt), wB = face_w(u1B, u2B, npt);
        point_pair32<kTwo>([&](int k) { return plus[ptA][k]; }, [&](int k) { return qmA[k]; },
                           [&](int k) { return plus[ptB][k]; }, [&](int k) { return kTwo ? qmB[k] : qmA[k]; }, a,
                           xq, yq, dL, PF, 0.5f * wA, 0.5f * __fmul_rn(wA, half_h), 0.5f * wB,
                           0.5f * __fmul_rn(wB, half_h), Gf, Gtl, amax);
        // a group is complete after points 3, 5 and 8 (face_group_ends, never
        // inside a pair): S = G0, then (S + G1), then (S + G2)
        if (face_group_ends(nB)) {
#pragma unroll
          for (int k = 0; k < F; ++k) {
            Sf[k] = first ? Gf[k] : __fadd_rn(Sf[k], Gf[k]);
            Gf[k] = 0.f;
          }
#pragma unroll
          for (int m = 0; m < 3; ++m) {
            Stl[m] = first ? Gtl[m] : __fadd_rn(Stl[m], Gtl[m]);
            Gtl[m] = 0.f;
          }
          first = false;
        }
      }
#pragma unroll
      for (int k = 0; k < F; ++k) {
        plus[p][k] = qpA[k];
        if (kTwo) plus[8 - p][k] = qpB[k];
      }
    };
#pragma unroll 1
    for (int p = npt == 1 ? 4 : 0; p < 4; ++p) pair_step(p, std::integral_constant<bool, true>{});
    pair_step(4, std::integral_constant<bool, false>{});
    if (j >= 0) {
      // face j-1/2 is complete: its sums in FP64 (each converted once); the
      // a-difference of cell j-1 is exact in FP64
      double fd[F], tld[3];
      float Str[3];
      right_torque32(a, h, Sf, Stl, Str);
#pragma unroll
      for (int k = 0; k < F; ++k) fd[k] = (double)Sf[k];
#pragma unroll
      for (int m = 0; m < 3; ++m) tld[m] = (double)Stl[m];
      if (j >= 1) {
        const int cell = (axis_comp(2, a, b, j - 1, pb, pc) * N + axis_comp(1, a, b, j - 1, pb, pc)) * N +
                         axis_comp(0, a, b, j - 1, pb, pc);
        double* Da = D + (size_t)a * DQ * N3 + cell;
#pragma unroll
        for (int k = 0; k < F; ++k) Da[k * N3] = __dsub_rn(fd[k], fprev[k]);
#pragma unroll
        for (int m = 0; m < 3; ++m) Da[(F + m) * N3] = __dsub_rn(tld[m], trprev[m]);
      }
#pragma unroll
      for (int k = 0; k < F; ++k) fprev[k] = fd[k];
#pragma unroll
      for (int m = 0; m < 3; ++m) trprev[m] = (double)Str[m];
      if (A.face_flux && (j == 0 || j == N)) {
        // tile boundary face: sums and the torque about the interior cell
        const int f = 2 * a + (j == N ? 1 : 0);
#pragma unroll
        for (int k = 0; k < F; ++k) io.face(sub, f, k, pc, pb, fd[k]);
#pragma unroll
        for (int m = 0; m < 3; ++m) io.face(sub, f, F + m, pc, pb, j == N ? tld[m] : trprev[m]);
      }
    }
  }
#pragma unroll
  for (int o2 = 16; o2 > 0; o2 >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o2));
  if ((tid & 31) == 0) red[tid >> 5] = amax;
  __syncthreads();

  // ---- 4. divergence + sources in FP64 --------------------------------
  const double inv_h = 1.0 / hd;
  for (int c = tid; c < N3; c += kThreadsMx) {
    const int x = c % N, y = (c / N) % N, z = c / (N * N);
    finish_cell(
        A, io, sub, offx, offy, x, y, z,
        [&](int q) { return __dadd_rn(D[(0 * DQ + q) * N3 + c], D[(1 * DQ + q) * N3 + c]); },
        [&](int q) { return D[(2 * DQ + q) * N3 + c]; }, hd, inv_h, o);
  }
  if (tid == 0) {
    float m = red[0];
#pragma unroll
    for (int w = 1; w < kThreadsMx / 32; ++w) m = fmaxf(m, red[w]);
    io.amax(sub, (double)m);
  }
  __syncthreads();
}

}  // namespace hyd
