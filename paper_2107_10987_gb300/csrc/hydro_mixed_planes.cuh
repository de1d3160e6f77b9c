// hydro_mixed_planes.cuh -- one sub-grid of the mixed-precision hydro step as
// a plane sweep: each of the 13 lines through a cell is reconstructed once.
//
// The row sweep (hydro_mixed_body.cuh) gives every thread one row of cells
// along one axis and reconstructs, at each cell of the row, the 9 lines that
// cross its faces of that axis: the edge lines of a cell are evaluated in two
// axis sweeps and the vertex lines in three, 27 line evaluations per cell for
// 13 distinct lines.  Here one CTA of kThreadsPl threads sweeps the sub-grid
// plane by plane along z (k = -1 .. N), each step in three phases separated
// by two barriers:
//   A  reconstruct plane k: the 13 lines of its interior cells, the 9 lines
//      of the face-adjacent ghost cells around it (x = -1, N and y = -1, N)
//      and, on the planes k = -1 and N, the 9 lines that cross the z-faces;
//      both interface values of every line go to shared memory (R), the
//      values towards +z into one of two z-buffers (Zp) that the next step
//      reads;
//   B  the fluxes of the x- and y-faces of plane k and of the z-faces between
//      planes k-1 and k, three threads per face (the face's three groups
//      of points, combined by warp shuffles in the fixed order), into face-sum
//      buffers (converted to FP64 once per face); meanwhile the primitives of
//      plane k+3 are converted from the FP64 staging buffer that phase A
//      filled from global memory, and two of the warps that have no face
//      finish plane k-2: its z-differences, the divergence and the sources,
//      and its dU/dt is stored (finish_cell);
//   C  per cell of plane k, the FP64 x- and y-differences of face sums.
// The primitives live in a ring of six FP32 planes (the five planes a line
// of plane k reaches, and the one being converted), so the CTA holds about
// 190 KB of shared memory instead of the whole padded sub-grid and runs 21
// warps on its SM; the per-axis flux differences never leave the SM.
//
// The arithmetic is the row sweep's own: the same ppm32x2 on the same samples
// (exactly symmetric under reversal of a line, so the orientation in which a
// line is evaluated does not matter; each lane rounds alike whichever field
// or line shares its instruction), the same point_pair32 on the same pairs
// in the same order, the same grouping of
// each face sum, the same FP64 differences and finish_cell.  The two
// decompositions therefore give the same bits.
#pragma once
#include <type_traits>

#include "hydro_mixed_body.cuh"

namespace hyd {

// 24 warps, one CTA per SM.  (The register file is shared out per scheduler:
// 21 warps would be charged as 24, at the same 80 registers a thread.)
constexpr int kThreadsPl = 768;
constexpr int kWarpsPl = kThreadsPl / 32;
constexpr int kPl = S * S;                // 196 cells of a padded plane
constexpr int kRing = 6;                  // primitive planes held
constexpr int kRowR = N * N + 1;          // interior cells of a plane, padded for the banks
constexpr int kRowB = N + 1;              // face-adjacent ghost cells along a side, padded
constexpr int kNFaceXY = 2 * (N + 1) * N; // x- and y-faces of a plane (144)
// Phase B: 10 faces per warp, the 208 faces of a plane on warps 0 .. 20;
// warps 21 and 22 finish an earlier plane meanwhile.
constexpr int kFinishT0 = 21 * 32;
static_assert((kNFaceXY + N * N + 9) / 10 <= kFinishT0 / 32 && kFinishT0 + N * N <= kThreadsPl, "phase B warps");

// Shared-memory layout of one CTA (offsets in bytes).
struct PlaneSmem {
  static constexpr size_t stage = 0;                                            // double [F][kPl]
  static constexpr size_t s01 = stage + sizeof(double) * F * kPl;               // double [2][DQ][64]
  static constexpr size_t ring = s01 + sizeof(double) * 2 * DQ * N * N;         // float [kRing][F][kPl]
  static constexpr size_t rint = ring + sizeof(float) * kRing * F * kPl;        // float [17][F][kRowR]
  static constexpr size_t zp = rint + sizeof(float) * 17 * F * kRowR;           // float [2][9][F][kRowR]
  static constexpr size_t rbnd = zp + sizeof(float) * 2 * 9 * F * kRowR;        // float [4][9][F][kRowB]
  static constexpr size_t fs = rbnd + sizeof(float) * 4 * 9 * F * kRowB;        // double [16][kNFaceXY]
  static constexpr size_t zs = fs + sizeof(double) * 16 * kNFaceXY;             // double [3][16][64]
  static constexpr size_t coord = zs + sizeof(double) * 3 * 16 * N * N;         // float [2][N + 2]
  static constexpr size_t red = coord + sizeof(float) * 2 * (N + 2);            // float [kWarpsPl]
  static constexpr size_t total = red + sizeof(float) * kWarpsPl;
};
constexpr size_t kPlaneSmemBytes = PlaneSmem::total;
static_assert(kPlaneSmemBytes <= 227 * 1024, "plane sweep shared memory");

// Direction code of d in {-1,0,1}^3: (dz+1)*9 + (dy+1)*3 + (dx+1); 13 is 0.
__device__ __forceinline__ int dcode(int dx, int dy, int dz) { return (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1); }

// Where R[d] of interior cell `cell` (y*8 + x) of plane k lives: directions
// towards +z (code >= 18) in the z-buffer of the plane's parity, the other
// 17 in rint.  Returns the address of field 0; fields are kRowR apart.
__device__ __forceinline__ float* r_int_slot(float* rint, float* zp, int code, int k, int cell) {
  if (code >= 18) return zp + ((size_t)((k & 1) * 9 + code - 18) * F) * kRowR + cell;
  return rint + ((size_t)(code < 13 ? code : code - 1) * F) * kRowR + cell;
}
// R[d] of a face-adjacent ghost cell of side sd (0: x = -1, 1: x = N, 2:
// y = -1, 3: y = N) at position pos along the side; the side's 9 directions
// point into the sub-grid: (+-1, u1, u2) for x sides, (u1, +-1, u2) for y
// sides, bi = (u2+1)*3 + (u1+1).
__device__ __forceinline__ float* r_bnd_slot(float* rbnd, int sd, int bi, int pos) {
  return rbnd + ((size_t)(sd * 9 + bi) * F) * kRowB + pos;
}

// Reconstruct one line of the cell at padded plane coordinates (ix, iy) of
// padded plane zp along (dx, dy, dz), for the five fields f0 .. f0 + 4 (f0 =
// 0 or 5): both interface values of each, to dp (towards +d) and dm (towards
// -d; nullptr: not needed), field stride fst (dp, dm address field 0).
// Samples from the primitive ring.  kContact as line10fc.
template <bool kContact, bool kSpin>
__device__ __forceinline__ void plane_line(const float* __restrict__ ring, int ix, int iy, int zp, int dx, int dy,
                                           int dz, int f0, float* dp, float* dm, int fst, const StepParamsF& PF) {
  int off[5];
#pragma unroll
  for (int m = 0; m < 5; ++m)
    off[m] = ((zp + (m - 2) * dz) % kRing) * (F * kPl) + (iy + (m - 2) * dy) * S + (ix + (m - 2) * dx);
  bool contact = false;
  if (kContact)
    contact = contact_line32(ring[off[1] + RHO * kPl], ring[off[3] + RHO * kPl],
                             __fmul_rn(PF.gm1, ring[off[1] + EGAS * kPl]),
                             __fmul_rn(PF.gm1, ring[off[3] + EGAS * kPl]), __fmul_rn(PF.gamma, 0.1f));
  // the five samples of fields fa and fb as pairs
  auto samples = [&](int fa, int fb, float2 v[5]) {
#pragma unroll
    for (int m = 0; m < 5; ++m) v[m] = f2(ring[off[m] + fa * kPl], ring[off[m] + fb * kPl]);
  };
  auto put = [&](int f, float qp, float qm) {
    dp[f * fst] = qp;
    if (dm) dm[f * fst] = qm;
  };
  // fields 0 .. 4: the density alone (the steepened field), then (1, 2) and
  // (3, 4); fields 5 .. 9: (5, 6), (7, 8), then the species alone
  static_assert(RHO == 0 && SP0 == F - 1 && F == 10, "field split of a half line");
  const int fs = f0 == 0 ? RHO : SP0;
  {
    float2 v[5], qp, qm;
    samples(fs, fs, v);
    const float eta = (kContact && contact) ? contact_eta32(v[0].x, v[1].x, v[2].x, v[3].x, v[4].x) : 0.f;
    if (kContact)
      ppm32x2<true>(v[0], v[1], v[2], v[3], v[4], qp, qm, f2(eta));
    else
      ppm32x2(v[0], v[1], v[2], v[3], v[4], qp, qm);
    put(fs, qp.x, qm.x);
  }
  // the cell's spin fed back into the velocity at both ends (spin_dv32; the
  // row sweep's values, bit for bit)
  float dv[3] = {0.f, 0.f, 0.f};
  const bool spin = kSpin && f0 == 0;
  if (spin)
    spin_dv32(ring[off[2] + RHO * kPl], ring[off[2] + EGAS * kPl], ring[off[2] + ZX * kPl], ring[off[2] + ZY * kPl],
              ring[off[2] + ZZ * kPl], PF.k3h, __fmul_rn(PF.gamma, PF.gm1), dx, dy, dz, dv);
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int fa = (f0 == 0 ? 1 : 5) + 2 * i;
    float2 v[5], qp, qm;
    samples(fa, fa + 1, v);
    ppm32x2(v[0], v[1], v[2], v[3], v[4], qp, qm);
    if (spin) {
      // fields 1, 2 (i = 0) and 3 (i = 1) are the velocity
      qp.x = __fadd_rn(qp.x, dv[2 * i]);
      qm.x = __fsub_rn(qm.x, dv[2 * i]);
      if (i == 0) {
        qp.y = __fadd_rn(qp.y, dv[1]);
        qm.y = __fsub_rn(qm.y, dv[1]);
      }
    }
    put(fa, qp.x, qm.x);
    put(fa + 1, qp.y, qm.y);
  }
}

// One 8^3 tile (work unit s) as a plane sweep; Io as for mixed_subgrid, plus
//   io.load_fields(sub, c, f0, nf, u)   fields f0 .. f0+nf-1 of padded cell c
// (nf <= 5).  sm: the CTA's dynamic shared memory (kPlaneSmemBytes).  Ends
// with a barrier.  Must be called by all kThreadsPl threads.
template <bool kContact, bool kSpin, class Io>
__device__ __forceinline__ void mixed_subgrid_planes(const StepArgs64& A, const Io& io, int s, unsigned char* sm) {
  double* stage = reinterpret_cast<double*>(sm + PlaneSmem::stage);
  double* s01 = reinterpret_cast<double*>(sm + PlaneSmem::s01);
  float* ring = reinterpret_cast<float*>(sm + PlaneSmem::ring);
  float* rint = reinterpret_cast<float*>(sm + PlaneSmem::rint);
  float* zp = reinterpret_cast<float*>(sm + PlaneSmem::zp);
  float* rbnd = reinterpret_cast<float*>(sm + PlaneSmem::rbnd);
  double* fsum = reinterpret_cast<double*>(sm + PlaneSmem::fs);
  double* zsum = reinterpret_cast<double*>(sm + PlaneSmem::zs);
  float* coord = reinterpret_cast<float*>(sm + PlaneSmem::coord);
  float* red = reinterpret_cast<float*>(sm + PlaneSmem::red);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const typename Io::Sub sub = io.begin(s);
  const int si = io.sidx(sub), offx = io.offx(sub), offy = io.offy(sub);
  const double hd = A.h[si];
  const StepParamsF PF{(float)A.P.gamma, (float)A.P.gm1, (float)A.P.omega, kSpin ? 1 : 0,
                       kSpin ? (float)(3.0 / hd) : 0.f};
  const float h = (float)hd, half_h = 0.5f * h;
  const double o[3] = {A.origin[3 * si + 0], A.origin[3 * si + 1], A.origin[3 * si + 2]};
  const double inv_h = 1.0 / hd;
  const int npt = A.P.face_points;
  float amax = 0.f;
  bool bad = false;

  // primitives of one padded cell into the ring (cell q of padded plane z)
  auto convert = [&](const double* u, int z, int q) {
    float pq[F];
    bad |= !prims_mixed(u, A.P.eta1, PF.gamma, pq);
    float* dst = ring + (size_t)(z % kRing) * F * kPl + q;
#pragma unroll
    for (int f = 0; f < F; ++f) dst[f * kPl] = pq[f];
  };

  sub_coords(coord, hd, o[0], o[1], offx, offy);

  // dU/dt of plane p (its z-differences from the face sums of p - 1/2 and
  // p + 1/2, the x- plus y-differences from phase C, finish_cell), on the
  // 64 threads t0 .. t0 + 63
  auto finish_plane = [&](int p, int t0) {
    const int c2 = tid - t0;
    if (c2 < 0 || c2 >= N * N) return;
    const double* a01 = s01 + (size_t)(p & 1) * DQ * N * N + c2;
    const double* zu = zsum + (size_t)((p + 1) % 3) * 16 * N * N + c2;  // face p+1/2: upper face of p
    const double* zl = zsum + (size_t)(p % 3) * 16 * N * N + c2;        // face p-1/2: lower face of p
    finish_cell(
        A, io, sub, offx, offy, c2 % N, c2 / N, p, [&](int q) { return a01[q * N * N]; },
        [&](int q) { return __dsub_rn(zu[q * N * N], zl[(q < F ? q : q + 3) * N * N]); }, hd, inv_h, o);
  };

  // ---- planes 0..4 of the padded sub-grid, straight into the ring --------
  for (int e = tid; e < 5 * kPl; e += kThreadsPl) {
    double u[F];
    io.load_fields(sub, e, 0, 5, u);
    io.load_fields(sub, e, 5, 5, u + 5);
    convert(u, e / kPl, e % kPl);
  }
  __syncthreads();

  // this thread's share of the prefetch of the next padded plane: 5 fields
  // of one cell
  const bool pf_on = tid < 2 * kPl;
  const int pf_q = tid % kPl, pf_f0 = (tid / kPl) * 5;

#pragma unroll 1
  for (int k = -1; k <= N; ++k) {
    const int zpk = k + G;  // padded index of plane k
    double pf[5];
    const bool pf_do = pf_on && k + 6 < S;  // padded plane k + 6 = plane k + 3
    if (pf_do) io.load_fields(sub, (k + 6) * kPl + pf_q, pf_f0, 5, pf);

    // ---- A: reconstruct plane k ------------------------------------------
    // work items: a line of one cell for five of its fields (f0 = 0 or 5)
    if (k >= 0 && k < N) {
      constexpr int kLines = 13 * N * N + 4 * 9 * N;  // 1120
      for (int i = tid; i < 2 * kLines; i += kThreadsPl) {
        const int f0 = i < kLines ? 0 : 5, li = i < kLines ? i : i - kLines;
        if (li < 13 * N * N) {
          // line L of interior cell (x, y): canonical direction code 14 + L
          const int L = li / (N * N), cell = li % (N * N), x = cell % N, y = cell / N;
          const int code = 14 + L, dx = code % 3 - 1, dy = (code / 3) % 3 - 1, dz = code / 9 - 1;
          float* dp = r_int_slot(rint, zp, code, k, cell);
          float* dm = r_int_slot(rint, zp, 26 - code, k, cell);
          plane_line<kContact, kSpin>(ring, x + G, y + G, zpk, dx, dy, dz, f0, dp, dm, kRowR, PF);
        } else {
          // face-adjacent ghost cell: the 9 lines into the sub-grid
          const int j = li - 13 * N * N, sd = j / (9 * N), bi = (j % (9 * N)) / N, pos = j % N;
          const int u1 = bi % 3 - 1, u2 = bi / 3 - 1;
          int x, y, dx, dy;
          if (sd < 2) {
            x = sd == 0 ? -1 : N;
            y = pos;
            dx = sd == 0 ? 1 : -1;
            dy = u1;
          } else {
            x = pos;
            y = sd == 2 ? -1 : N;
            dx = u1;
            dy = sd == 2 ? 1 : -1;
          }
          plane_line<kContact, kSpin>(ring, x + G, y + G, zpk, dx, dy, u2, f0, r_bnd_slot(rbnd, sd, bi, pos), nullptr,
                               kRowB, PF);
        }
      }
    } else {
      // k = -1: the lines towards +z; k = N: towards -z (interior columns)
      constexpr int kLines = 9 * N * N;
      for (int i = tid; i < 2 * kLines; i += kThreadsPl) {
        const int f0 = i < kLines ? 0 : 5, li = i < kLines ? i : i - kLines;
        const int zi = li / (N * N), cell = li % (N * N), x = cell % N, y = cell / N;
        const int dx = zi % 3 - 1, dy = zi / 3 - 1, dz = k < 0 ? 1 : -1;
        float* dp = r_int_slot(rint, zp, dcode(dx, dy, dz), k, cell);
        plane_line<kContact, kSpin>(ring, x + G, y + G, zpk, dx, dy, dz, f0, dp, nullptr, kRowR, PF);
      }
    }
    if (pf_do) {
#pragma unroll
      for (int f = 0; f < 5; ++f) stage[(pf_f0 + f) * kPl + pf_q] = pf[f];
    }
    __syncthreads();

    // ---- B: face fluxes; conversion of padded plane k + 6 ------------------
    if (k >= 0) {
      const int slot = warp * 10 + lane / 3, g = lane % 3;
      // x- and y-faces of plane k (k < N), z-faces between k-1 and k
      const bool zface = slot >= kNFaceXY;
      const bool active = lane < 30 && slot < kNFaceXY + N * N && (k < N || zface);
      float Gf[F], Gtl[3];
#pragma unroll
      for (int q = 0; q < F; ++q) Gf[q] = 0.f;
#pragma unroll
      for (int m = 0; m < 3; ++m) Gtl[m] = 0.f;
      int a = 0, fx = 0, fy = 0;  // face axis; the left cell's (x, y) in plane k (or k-1 for z-faces)
      if (active) {
        if (slot < N * (N + 1)) {
          a = 0;
          fy = slot / (N + 1);
          fx = slot % (N + 1) - 1;
        } else if (!zface) {
          a = 1;
          const int t = slot - N * (N + 1);
          fx = t / (N + 1);
          fy = t % (N + 1) - 1;
        } else {
          a = 2;
          const int t = slot - kNFaceXY;
          fx = t % N;
          fy = t / N;
        }
        // left-cell centre in FP32 (the row sweep's values)
        const float xc = coord[fx + 1], yc = coord[(N + 2) + fy + 1];
        // point n of the face: its directions dL, dR (as small integers) and
        // where its left value R_left[dL] and right value R_right[dR] live
        struct Pt {
          const float* pl;
          const float* pr;
          int sl, sr, dl[3], dr[3], u1, u2;
        };
        auto geom = [&](int n) {
          Pt t;
          t.u1 = face_u1(n);
          t.u2 = face_u2(n);
          const int u1 = t.u1, u2 = t.u2;
          // d along (a, b, c) = (1, u1, u2), b < c the transverse axes
          t.dl[0] = a == 0 ? 1 : u1;
          t.dl[1] = a == 1 ? 1 : (a == 0 ? u1 : u2);
          t.dl[2] = a == 2 ? 1 : u2;
#pragma unroll
          for (int m = 0; m < 3; ++m) t.dr[m] = m == a ? -1 : t.dl[m];
          const int cl = dcode(t.dl[0], t.dl[1], t.dl[2]), cr = dcode(t.dr[0], t.dr[1], t.dr[2]);
          t.sl = t.sr = kRowR;
          if (a == 0) {
            const int bi = (u2 + 1) * 3 + (u1 + 1);
            if (fx < 0) {
              t.pl = r_bnd_slot(rbnd, 0, bi, fy);
              t.sl = kRowB;
            } else {
              t.pl = r_int_slot(rint, zp, cl, k, fy * N + fx);
            }
            if (fx + 1 >= N) {
              t.pr = r_bnd_slot(rbnd, 1, bi, fy);
              t.sr = kRowB;
            } else {
              t.pr = r_int_slot(rint, zp, cr, k, fy * N + fx + 1);
            }
          } else if (a == 1) {
            const int bi = (u2 + 1) * 3 + (u1 + 1);
            if (fy < 0) {
              t.pl = r_bnd_slot(rbnd, 2, bi, fx);
              t.sl = kRowB;
            } else {
              t.pl = r_int_slot(rint, zp, cl, k, fy * N + fx);
            }
            if (fy + 1 >= N) {
              t.pr = r_bnd_slot(rbnd, 3, bi, fx);
              t.sr = kRowB;
            } else {
              t.pr = r_int_slot(rint, zp, cr, k, (fy + 1) * N + fx);
            }
          } else {
            t.pl = r_int_slot(rint, zp, cl, k - 1, fy * N + fx);
            t.pr = r_int_slot(rint, zp, cr, k, fy * N + fx);
          }
          return t;
        };
        // the lane's group (face_group_ends): g = 0 the pairs (0, 1) and (2,
        // 3), g = 1 the pair (4, 5), g = 2 the pair (6, 7) and the centre 8 in
        // both lanes (with one flux point per face only the centre)
        // points n and n + 1 in the two lanes (kTwo), or n alone
        auto points = [&](auto two, int n) {
          constexpr bool kTwo = decltype(two)::value;
          const Pt tA = geom(n), tB = kTwo ? geom(n + 1) : tA;
          float2 dL[3];
#pragma unroll
          for (int m = 0; m < 3; ++m) dL[m] = f2((float)tA.dl[m], (float)tB.dl[m]);
          const float2 xq = fma2(f2(half_h), dL[0], f2(xc)), yq = fma2(f2(half_h), dL[1], f2(yc));
          const float wA = face_w(tA.u1, tA.u2, npt), wB = face_w(tB.u1, tB.u2, npt);
          point_pair32<kTwo>([&](int q) { return tA.pl[q * tA.sl]; }, [&](int q) { return tA.pr[q * tA.sr]; },
                             [&](int q) { return tB.pl[q * tB.sl]; }, [&](int q) { return tB.pr[q * tB.sr]; }, a,
                             xq, yq, dL, PF, 0.5f * wA, 0.5f * __fmul_rn(wA, half_h), 0.5f * wB,
                             0.5f * __fmul_rn(wB, half_h), Gf, Gtl, amax);
        };
        // the lane's group (face_group_ends): g = 0 the pairs (0, 1) and (2,
        // 3), g = 1 the pair (4, 5), g = 2 the pair (6, 7) and the centre 8
        // (with one flux point per face only the centre)
        static_assert(face_group_ends(3) && face_group_ends(5) && face_group_ends(8), "lane groups");
        using Two = std::integral_constant<bool, true>;
        using One = std::integral_constant<bool, false>;
        if (npt != 1) points(Two{}, g == 0 ? 0 : 2 * g + 2);  // 0, 4, 6
        if (npt != 1 && g == 0) points(Two{}, 2);
        if (g == 2) points(One{}, 8);
      }
      // the face's three groups, (G0 + G1) + G2, on the lane of group 0
      float out[16];
#pragma unroll
      for (int q = 0; q < F + 3; ++q) {
        const float v = q < F ? Gf[q] : Gtl[q - F];
        const float v1 = __shfl_down_sync(0xffffffffu, v, 1), v2 = __shfl_down_sync(0xffffffffu, v, 2);
        out[q] = npt == 1 ? v2 : __fadd_rn(__fadd_rn(v, v1), v2);
      }
      // the torque about the right cell centre from the face's sums
      right_torque32(a, h, out, out + F, out + F + 3);
      if (active && g == 0) {
        double* dst = zface ? zsum + (size_t)(k % 3) * 16 * N * N + (slot - kNFaceXY) : fsum + slot;
        const int dstride = zface ? N * N : kNFaceXY;
#pragma unroll
        for (int q = 0; q < 16; ++q) dst[q * dstride] = (double)out[q];
        if (A.face_flux) {
          // sub-grid boundary faces: sums and the torque about the interior cell
          int f = -1, pc = 0, pb = 0;
          bool upper = false;
          if (a == 0 && (fx < 0 || fx + 1 >= N)) {
            f = fx < 0 ? 0 : 1;
            upper = fx >= 0;
            pc = k;
            pb = fy;
          } else if (a == 1 && (fy < 0 || fy + 1 >= N)) {
            f = fy < 0 ? 2 : 3;
            upper = fy >= 0;
            pc = k;
            pb = fx;
          } else if (a == 2 && (k == 0 || k == N)) {
            f = k == 0 ? 4 : 5;
            upper = k == N;
            pc = fy;
            pb = fx;
          }
          if (f >= 0) {
#pragma unroll
            for (int q = 0; q < F; ++q) io.face(sub, f, q, pc, pb, dst[q * dstride]);
#pragma unroll
            for (int m = 0; m < 3; ++m) io.face(sub, f, F + m, pc, pb, dst[(upper ? F + m : F + 3 + m) * dstride]);
          }
        }
      }
    }
    // plane k - 2 is complete (its upper z-face was summed in the last
    // step): two warps that have no face finish it
    if (k >= 2) finish_plane(k - 2, kFinishT0);
    if (k + 6 < S) {
      // the staged padded plane k + 6 into the ring
      for (int q = tid; q < kPl; q += kThreadsPl) {
        double u[F];
#pragma unroll
        for (int f = 0; f < F; ++f) u[f] = stage[f * kPl + q];
        convert(u, k + 6, q);
      }
    }
    __syncthreads();

    // ---- C: the x- plus y-differences of face sums of plane k -------------
    if (k >= 0 && k < N) {
      for (int t = tid; t < DQ * N * N; t += kThreadsPl) {
        const int q = t / (N * N), cell = t % (N * N), x = cell % N, y = cell / N;
        // upper face: its fluxes and left-cell torques (q); lower face: its
        // fluxes and right-cell torques (ql)
        const int ql = q < F ? q : q + 3;
        const int xl = y * (N + 1) + x, yl = N * (N + 1) + x * (N + 1) + y;  // lower x- and y-face slots
        const double d0 = __dsub_rn(fsum[q * kNFaceXY + xl + 1], fsum[ql * kNFaceXY + xl]);
        const double d1 = __dsub_rn(fsum[q * kNFaceXY + yl + 1], fsum[ql * kNFaceXY + yl]);
        s01[(size_t)(k & 1) * DQ * N * N + q * N * N + cell] = __dadd_rn(d0, d1);
      }
    }
  }
  // the last plane, after the last z-faces
  finish_plane(N - 1, 0);

  // ---- amax and the status ------------------------------------------------
#pragma unroll
  for (int o2 = 16; o2 > 0; o2 >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o2));
  if (lane == 0) red[warp] = amax;
  if (bad) atomicOr(A.status, 1u);
  __syncthreads();
  if (tid == 0) {
    float m = red[0];
#pragma unroll
    for (int w = 1; w < kWarpsPl; ++w) m = fmaxf(m, red[w]);
    io.amax(sub, (double)m);
  }
  __syncthreads();
}

}  // namespace hyd
