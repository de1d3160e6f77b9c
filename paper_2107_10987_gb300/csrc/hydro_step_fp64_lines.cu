// hydro_step_fp64_lines.cu -- the per-sub-grid hydro step in FP64 with every
// PPM line evaluated once per cell.
//
// The same method, arithmetic and face-sum order as hydro_step_fp64.cu (and
// the same bits), organised around the 13 line directions of Sec. III-B
// instead of the three axis sweeps.  A face point lies on the surface of its
// two cells: the face centres use the axis lines, the edge midpoints (shared
// by two faces of a cell) the 6 edge lines and the corners (shared by three
// faces) the 4 vertex lines, so an axis sweep that reconstructs its own 9
// lines per cell evaluates 27 line-fields per cell where 13 are unique.
// One persistent CTA of 192 threads per SM loops over 8^3 tiles:
//   1. bulk TMA copies stage the ghost-padded state into shared memory (the
//      next tile's copies are issued as soon as phase 3 no longer reads it,
//      so they overlap phases 4 and 5); primitives replace it in place;
//   2. (learned smoothness indicator, optional) its per-cell decisions;
//   3. lines: one work item per (field group, run), a run being a maximal segment
//      of consecutive cells along one of the 13 directions d among the cells
//      that need that line (the interior, and the face-adjacent ghost cells
//      of the faces whose normal component of d is nonzero).  The item walks
//      its run with a sliding window, so that the differences, the MC slopes
//      and the unlimited interface value between two cells of the run are
//      computed once for both cells (PPM's interface value at x + d/2 is one
//      number for the cell x and its neighbour x + d), then applies the
//      per-cell steepening and monotonicity fix-ups and stores both
//      interface values of the cell in a per-CTA buffer in global memory
//      (26 values per field and cell, read back from L2 or DRAM in phase 4);
//   4. faces: 192 threads, one per (axis, transverse row), sweep their row's
//      9 faces in the order of hydro_step_fp64.cu and sum the 9 Kurganov-
//      Tadmor point fluxes with the Simpson weights from the stored values;
//      per-axis flux differences go to the step scratch;
//   5. divergence, sources and dU/dt as in hydro_step_fp64.cu.
// Runs are listed once per device, longest first, so that the lanes of a
// warp mostly walk runs of equal length.  The walk's arithmetic is ppm64's,
// operation for operation, on the same operands (the reversed line gives
// the mirrored values bit for bit), so the stored values are those the axis
// sweeps compute.
#include <algorithm>
#include <vector>

#include "hydro.h"
#include "hydro_common.cuh"
#include "hydro_fp64.cuh"
#include "hydro_mixed.cuh"

namespace hyd {

constexpr int kLThreads = NROW;  // 192
constexpr long kLWaitPolls = 1L << 24;

// The line-end buffer of one CTA: for each of the 26 (direction, end) slots
// and each cell of the 10^3 box of interior cells and their face-adjacent
// ghost layer, a record of the 10 fields padded to 12 doubles (three 32-byte
// sectors, each written whole by one thread: fields 0-3, 4-7, 8-9 and two
// zeros): [slot][box cell][kRec] doubles.
constexpr int kBox = (N + 2) * (N + 2) * (N + 2);  // 1000
constexpr int kRec = 12;
constexpr size_t kLinesPerCta = (size_t)26 * kBox * kRec;

// Directions d with components in {-1, 0, 1}, the first nonzero one
// positive; index 9 dx + 3 dy + dz - 1 in [0, 13).  Slot 2 dd + 0 holds the
// value at x + d/2 of cell x, slot 2 dd + 1 the value at x - d/2.
__host__ __device__ constexpr int dir_index(int dx, int dy, int dz) { return 9 * dx + 3 * dy + dz - 1; }

// Slot of the value at x + w/2 for a nonzero w with components in {-1, 0, 1}.
__device__ __forceinline__ int end_slot(int wx, int wy, int wz) {
  const int sg = wx != 0 ? wx : (wy != 0 ? wy : wz);
  return 2 * dir_index(sg * wx, sg * wy, sg * wz) + (sg > 0 ? 0 : 1);
}

// Run list: one 32-bit word per run, bits 0-11 the shared-memory index of its
// first cell (14^3 layout), 12-21 that cell's box index, 22-25 its length
// (1..10), 26-31 the direction's components plus one (2 bits each, x first).
constexpr int kMaxRuns = 2048;
__device__ uint32_t g_line_runs[kMaxRuns];

// Whether box cell (x, y, z) in [-1, N]^3 needs the line along d: interior
// cells need all 13, a ghost cell only the lines that reach its one face
// (exactly one coordinate outside [0, N), and d nonzero along that axis).
static bool needs_line(int x, int y, int z, int dx, int dy, int dz) {
  const int c[3] = {x, y, z}, d[3] = {dx, dy, dz};
  int out = 0;
  for (int i = 0; i < 3; ++i) {
    if (c[i] < -1 || c[i] > N) return false;
    if (c[i] < 0 || c[i] >= N) {
      if (d[i] == 0) return false;
      ++out;
    }
  }
  return out <= 1;
}

// The runs of all 13 directions, the axis lines' first (they alone serve the
// single-point face flux), each group longest first.
static std::vector<uint32_t> build_line_runs(int* n_axis) {
  struct R {
    int len, axis;
    uint32_t word;
  };
  std::vector<R> runs;
  for (int dx = -1; dx <= 1; ++dx)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dz = -1; dz <= 1; ++dz) {
        const int sg = dx != 0 ? dx : (dy != 0 ? dy : dz);
        if (sg <= 0) continue;  // the zero vector and the reversed directions
        const int axis = (dx != 0) + (dy != 0) + (dz != 0) == 1;
        for (int z = -1; z <= N; ++z)
          for (int y = -1; y <= N; ++y)
            for (int x = -1; x <= N; ++x) {
              if (!needs_line(x, y, z, dx, dy, dz) || needs_line(x - dx, y - dy, z - dz, dx, dy, dz)) continue;
              int len = 0;
              while (needs_line(x + len * dx, y + len * dy, z + len * dz, dx, dy, dz)) ++len;
              const uint32_t smem = (uint32_t)(((z + G) * S + (y + G)) * S + (x + G));
              const uint32_t box = (uint32_t)(((z + 1) * (N + 2) + (y + 1)) * (N + 2) + (x + 1));
              const uint32_t dirs = (uint32_t)(dx + 1) | ((uint32_t)(dy + 1) << 2) | ((uint32_t)(dz + 1) << 4);
              runs.push_back({len, axis, smem | (box << 12) | ((uint32_t)len << 22) | (dirs << 26)});
            }
      }
  std::stable_sort(runs.begin(), runs.end(), [](const R& p, const R& q) {
    if (p.axis != q.axis) return p.axis > q.axis;
    return p.len > q.len;
  });
  std::vector<uint32_t> words;
  *n_axis = 0;
  for (const R& r : runs) {
    words.push_back(r.word);
    *n_axis += r.axis;
  }
  return words;
}

static int g_runs_total = 0, g_runs_axis = 0;

// One work item of phase 3: fields k0 .. k0 + NG - 1 along run word e.  The
// window holds, per field, the samples S(i-2..i+2) of cell i of the run, the
// differences and MC slopes around it and the interface value Q(i - 1/2);
// each step loads one sample per field and forms one difference, one slope
// and one interface value (ppm64's operations on the same operands), then
// the cell's fix-ups, and stores the group's 32-byte sector of both records
// of the cell.
template <bool kGate, bool kContact, int NG>
__device__ __forceinline__ void line_run(const double* __restrict__ Q, const uint8_t* __restrict__ smooth,
                                         const StepParams& P, double* __restrict__ R, uint32_t e, int k0,
                                         double k3h) {
  const int c0 = (int)(e & 0xfffu), b0 = (int)((e >> 12) & 0x3ffu), n = (int)((e >> 22) & 0xfu);
  const int dx = (int)((e >> 26) & 3u) - 1, dy = (int)((e >> 28) & 3u) - 1, dz = (int)(e >> 30) - 1;
  const int sv = dx + S * dy + S * S * dz;                             // shared-memory stride along d
  const int bv = (dx + (N + 2) * dy + (N + 2) * (N + 2) * dz) * kRec;  // line-buffer stride along d
  double* Rp = R + ((size_t)(2 * dir_index(dx, dy, dz)) * kBox + b0) * kRec + k0;
  double* Rm = Rp + (size_t)kBox * kRec;
  const double* q = Q + k0 * S3 + c0;
  // the group's steepened field (rho in group 0, the species in group 2)
  const bool steep_group = kContact && (k0 == RHO || k0 + NG > SP0);
  double sm2[NG], sm1[NG], s0[NG], s1[NG], dr[NG], Dm[NG], Dc[NG], qm[NG];
#pragma unroll
  for (int f = 0; f < NG; ++f) {
    const double* qf = q + f * S3;
    sm2[f] = qf[-2 * sv];
    sm1[f] = qf[-sv];
    s0[f] = qf[0];
    s1[f] = qf[sv];
    const double dl = rsub(s0[f], sm1[f]);
    Dm[f] = slope64(rsub(sm1[f], sm2[f]), dl);  // slope at cell i - 1
    dr[f] = rsub(s1[f], s0[f]);
    Dc[f] = slope64(dl, dr[f]);  // slope at cell i
    qm[f] = ppm_iface64(sm1[f], s0[f], Dm[f], Dc[f]);  // interface value at i - 1/2
  }
#pragma unroll 1
  for (int i = 0; i < n; ++i) {
    const int ci = c0 + i * sv;
    const bool smooth_i = kGate && smooth[ci];
    const bool contact = steep_group && !smooth_i && contact_line64(Q, ci, sv, P);
    double p[NG], m[NG];
#pragma unroll
    for (int f = 0; f < NG; ++f) {
      const int k = k0 + f;
      const double s2 = q[f * S3 + (i + 2) * sv];
      const double d2 = rsub(s2, s1[f]);
      const double Dp = slope64(dr[f], d2);  // slope at cell i + 1
      const double qp = ppm_iface64(s0[f], s1[f], Dc[f], Dp);
      p[f] = qp;
      m[f] = qm[f];
      if (kGate && smooth_i && !(k == ZX || k == ZY || k == ZZ)) {
        // the indicator's unlimited 4-point values (line10u)
        const double c7 = 7.0 / 12.0, c1 = 1.0 / 12.0;
        p[f] = rsub(rmul(c7, radd(s0[f], s1[f])), rmul(c1, radd(sm1[f], s2)));
        m[f] = rsub(rmul(c7, radd(s0[f], sm1[f])), rmul(c1, radd(s1[f], sm2[f])));
      } else {
        if (kContact && contact && (k == RHO || k == SP0)) {
          const double eta = contact_eta64(sm2[f], sm1[f], s0[f], s1[f], s2);
          if (eta > 0.0) ppm_steep64(sm1[f], s1[f], Dm[f], Dp, eta, p[f], m[f]);
        }
        ppm_limit64(s0[f], p[f], m[f]);
      }
      sm2[f] = sm1[f];
      sm1[f] = s0[f];
      s0[f] = s1[f];
      s1[f] = s2;
      dr[f] = d2;
      Dm[f] = Dc[f];
      Dc[f] = Dp;
      qm[f] = qp;
    }
    if (NG == 4 && k0 == 0 && P.spin) {
      // the cell's spin fed back into the velocity at both ends (spin_dv64)
      double dv[3];
      spin_dv64(Q[RHO * S3 + ci], Q[EGAS * S3 + ci], Q[ZX * S3 + ci], Q[ZY * S3 + ci], Q[ZZ * S3 + ci], k3h,
                rmul(P.gamma, P.gm1), dx, dy, dz, dv);
#pragma unroll
      for (int m3 = 0; m3 < 3; ++m3) {
        p[(1 + m3) % NG] = radd(p[(1 + m3) % NG], dv[m3]);
        m[(1 + m3) % NG] = rsub(m[(1 + m3) % NG], dv[m3]);
      }
    }
    double2* wp = reinterpret_cast<double2*>(Rp + i * bv);
    double2* wm = reinterpret_cast<double2*>(Rm + i * bv);
    wp[0] = make_double2(p[0], p[1]);
    wm[0] = make_double2(m[0], m[1]);
    if (NG == 4) {
      wp[1] = make_double2(p[NG > 2 ? 2 : 0], p[NG > 3 ? 3 : 0]);
      wm[1] = make_double2(m[NG > 2 ? 2 : 0], m[NG > 3 ? 3 : 0]);
    } else {
      wp[1] = make_double2(0.0, 0.0);
      wm[1] = make_double2(0.0, 0.0);
    }
  }
}

// kGate, kContact, NN: as for hydro_step_fp64_kernel.  A.lines: the per-CTA
// line-end buffers (kLinesPerCta doubles per CTA); n_runs: the runs of
// g_line_runs that phase 3 walks (the axis runs alone for the single-point
// face flux).
template <bool kGate, bool kContact = false, int NN = N>
__global__ void __launch_bounds__(kLThreads, 1) hydro_step_fp64_lines_kernel(StepArgs64 A, int n_runs) {
  using T = Tile<NN>;
  extern __shared__ __align__(128) double Q[];  // [F][S3], then the indicator's flags
  uint8_t* smooth = reinterpret_cast<uint8_t*>(Q + F * S3);
  __shared__ __align__(8) uint64_t bar;
  __shared__ double red[kLThreads / 32];
  __shared__ int bail;
  const int tid = threadIdx.x;
  double* __restrict__ D = A.scratch + (size_t)blockIdx.x * kScratchPerSub;
  double* R = A.lines + (size_t)blockIdx.x * kLinesPerCta;
  const int n_units = A.n_sub * T::kTiles;

  // the row of phases 4 and 5: axis a, transverse axes b < c at pb, pc (the
  // warp map of hydro_step_fp64_kernel)
  static_assert(N == 8 && S == 14, "row-to-warp map assumes 8^3 interiors with 3-cell ghosts");
  const int a = tid / (N * N);
  const int r = tid % (N * N);
  const int pb = ((r >> 5) << 2) | (r & 3), pc = (r & 31) >> 2;
  const int b = (a == 0) ? 1 : 0;

  // bulk copies of tile u into Q, completing on bar (warp 0; as in
  // hydro_step_fp64_kernel)
  auto stage = [&](int u) {
    if (tid < 32) {
      const T tile(u);
      if (tid == 0) {
        fence_proxy_async();
        mbar_expect_tx(&bar, (uint32_t)(F * S3 * sizeof(double)));
      }
      __syncwarp();
      const double* src = A.U + (size_t)tile.s * F * T::kS3;
      if (NN == N) {
        if (tid == 0)
#pragma unroll 1
          for (int k = 0; k < F; ++k) bulk_g2s(Q + k * S3, src + (size_t)k * S3, S3 * sizeof(double), &bar);
      } else {
#pragma unroll 1
        for (int w = tid; w < F * S * S; w += 32) {
          const int k = w / (S * S), z = (w / S) % S, y = w % S;
          bulk_g2s(Q + k * S3 + (z * S + y) * S, src + (size_t)k * T::kS3 + tile.pad(0, y, z), S * sizeof(double),
                   &bar);
        }
      }
    }
  };

  if (tid == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
    bail = 0;
  }
  __syncthreads();
  if ((int)blockIdx.x < n_units) stage(blockIdx.x);

  uint32_t phase = 0;
  for (int u = blockIdx.x; u < n_units; u += gridDim.x) {
    const T tile(u);
    const int s = tile.s;
    if (!mbar_wait_bounded(&bar, phase, kLWaitPolls)) {
      atomicOr(A.status, 2u);
      bail = 1;
    }
    phase ^= 1u;
    __syncthreads();
    if (bail) break;

    // ---- 1. primitives in place (hydro_step_fp64_kernel's arithmetic) ----
    bool bad = false;
    for (int c = tid; c < S3; c += kLThreads) {
      const double rho = Q[RHO * S3 + c];
      const double vx = Q[SX * S3 + c] / rho, vy = Q[SY * S3 + c] / rho, vz = Q[SZ * S3 + c] / rho;
      const double E = Q[EGAS * S3 + c];
      const double ek = rmul(rmul(0.5, rho), radd(radd(rmul(vx, vx), rmul(vy, vy)), rmul(vz, vz)));
      const double eE = rsub(E, ek);
      const double eps = (eE > rmul(A.P.eta1, E)) ? eE : pow(Q[TAU * S3 + c], A.P.gamma);
      Q[SX * S3 + c] = vx;
      Q[SY * S3 + c] = vy;
      Q[SZ * S3 + c] = vz;
      Q[EGAS * S3 + c] = eps;
      bad |= !(rho > 0.0) || !(eps > 0.0);
    }
    if (bad) atomicOr(A.status, 1u);
    __syncthreads();

    // ---- 2. learned smoothness indicator -----------------------------------
    if (kGate)
      gate_phase<double, kLThreads>(Q, (float)A.P.gm1, A.gate_w, A.gate_logit_thr, A.gate_zero_smooth, smooth,
                                    smooth + S3);

    // ---- 3. every line once: (field group, run) items, group-major ----------
    {
      const double k3h = 3.0 / A.h[s];  // the spin feedback's 3 / h
      const int n_items = 3 * n_runs;
#pragma unroll 1
      for (int it = tid; it < n_items; it += kLThreads) {
        const int g = it / n_runs;
        const uint32_t e = g_line_runs[it - g * n_runs];
        if (g < 2)
          line_run<kGate, kContact, 4>(Q, smooth, A.P, R, e, 4 * g, k3h);
        else
          line_run<kGate, kContact, 2>(Q, smooth, A.P, R, e, 8, k3h);
      }
    }
    // the last reads of Q for this tile are done: order them before the bulk
    // copies of the next tile, which overlap phases 4 and 5
    fence_proxy_async();
    __syncthreads();  // also: the line ends are visible to the whole CTA
    if (u + (int)gridDim.x < n_units) stage(u + gridDim.x);

    // ---- 4. face sweep of the row from the stored line ends ------------------
    const int ox = tile.o[0], oy = tile.o[1];
    const double h = A.h[s];
    const double half_h = 0.5 * h;
    const double o[3] = {A.origin[3 * s + 0], A.origin[3 * s + 1], A.origin[3 * s + 2]};
    double amax = 0.0;
    double fprev[F], trprev[3];
    // box index of the row's cell at a-index 0, and the box stride along a
    const int box0 = ((axis_comp(2, a, b, 0, pb, pc) + 1) * (N + 2) + (axis_comp(1, a, b, 0, pb, pc) + 1)) * (N + 2) +
                     (axis_comp(0, a, b, 0, pb, pc) + 1);
    const int ba = a == 0 ? 1 : (a == 1 ? N + 2 : (N + 2) * (N + 2));
    // The points of a face in the summation order of hydro_step_fp64_kernel:
    // q = 2p + side for the mirrored pairs p = 0..3 (side 0: the point
    // (-t1,-t2), side 1: (t1,t2), with (t1,t2) = (p/3 - 1, p%3 - 1)), then the
    // centre q = 8; the single-point face flux takes the centre alone.
    const int q0 = A.P.face_points == 1 ? 8 : 0;
    auto offsets = [](int qq, int& u1, int& u2) {
      const int pp = qq >> 1, t1 = pp / 3 - 1, t2 = pp % 3 - 1;
      u1 = (qq & 1) ? t1 : -t1;
      u2 = (qq & 1) ? t2 : -t2;
    };
    // the states at point qq of face jj - 1/2: the value at x + w/2 of cell
    // jj - 1, w = e_a + u1 e_b + u2 e_c (left), and at x + w'/2 of cell jj,
    // w' = w - 2 e_a (right)
    auto fetch = [&](int jj, int qq, double(&L)[F], double(&Rr)[F]) {
      int u1, u2;
      offsets(qq, u1, u2);
      const int d0 = axis_comp(0, a, b, 1, u1, u2), d1 = axis_comp(1, a, b, 1, u1, u2),
                d2 = axis_comp(2, a, b, 1, u1, u2);
      const int sl = end_slot(d0, d1, d2);
      const int sr = end_slot(a == 0 ? -1 : d0, a == 1 ? -1 : d1, a == 2 ? -1 : d2);
      const double2* pl = reinterpret_cast<const double2*>(R + ((size_t)sl * kBox + box0 + (jj - 1) * ba) * kRec);
      const double2* pr = reinterpret_cast<const double2*>(R + ((size_t)sr * kBox + box0 + jj * ba) * kRec);
#pragma unroll
      for (int k = 0; k < F / 2; ++k) {
        const double2 vl = pl[k], vr = pr[k];
        L[2 * k] = vl.x;
        L[2 * k + 1] = vl.y;
        Rr[2 * k] = vr.x;
        Rr[2 * k + 1] = vr.y;
      }
    };
    // one point ahead: the next point's states load while this one computes
    double nL[F], nR[F];
    fetch(0, q0, nL, nR);
#pragma unroll 1
    for (int j = 0; j <= N; ++j) {
      // face j - 1/2 between the cells j - 1 (left) and j (right) along a
      double fsum[F], T[3];
#pragma unroll
      for (int k = 0; k < F; ++k) fsum[k] = 0.0;
      T[0] = T[1] = T[2] = 0.0;
      const int ci0 = axis_comp(0, a, b, j - 1, pb, pc) + ox, ci1 = axis_comp(1, a, b, j - 1, pb, pc) + oy;
#pragma unroll 1
      for (int qq = q0; qq <= 8; ++qq) {
        double qL[F], qR[F];
#pragma unroll
        for (int k = 0; k < F; ++k) {
          qL[k] = nL[k];
          qR[k] = nR[k];
        }
        if (qq < 8)
          fetch(j, qq + 1, nL, nR);
        else if (j < N)
          fetch(j + 1, q0, nL, nR);
        int u1, u2;
        offsets(qq, u1, u2);
        const int d0 = axis_comp(0, a, b, 1, u1, u2), d1 = axis_comp(1, a, b, 1, u1, u2),
                  d2 = axis_comp(2, a, b, 1, u1, u2);
        const double xq = o[0] + h * ((ci0 + 0.5) + 0.5 * d0);
        const double yq = o[1] + h * ((ci1 + 0.5) + 0.5 * d1);
        // half the Simpson weight (1, 4, 1) x (1, 4, 1) / 36 of the point; 1/2
        // for the single-point face flux
        const double hw = A.P.face_points == 1 ? 0.5
                         : (u1 == 0 && u2 == 0) ? (8.0 / 36.0) : (u1 == 0 || u2 == 0) ? (2.0 / 36.0) : (0.5 / 36.0);
        point64(qL, qR, a, xq, yq, hw, d0, d1, d2, A.P, fsum, T, amax);
      }
      double tl[3], tr[3];
      face_torques64(T, fsum, a, half_h, tl, tr);
      if (j >= 1) {
        // interior cell i = j-1 along a: differences of its two a-faces
        const int i = j - 1;
        const int cell = (axis_comp(2, a, b, i, pb, pc) * N + axis_comp(1, a, b, i, pb, pc)) * N +
                         axis_comp(0, a, b, i, pb, pc);
        double* Da = D + (size_t)a * DQ * N3 + cell;
#pragma unroll
        for (int k = 0; k < F; ++k) Da[k * N3] = fsum[k] - fprev[k];
#pragma unroll
        for (int m = 0; m < 3; ++m) Da[(F + m) * N3] = tl[m] - trprev[m];
      }
#pragma unroll
      for (int k = 0; k < F; ++k) fprev[k] = fsum[k];
      trprev[0] = tr[0];
      trprev[1] = tr[1];
      trprev[2] = tr[2];
      if (A.face_flux && (j == 0 || j == N) && tile.outer(2 * a + (j == N ? 1 : 0))) {
        // sub-grid boundary face: sums and the torque about the interior cell
        const int f = 2 * a + (j == N ? 1 : 0);
#pragma unroll
        for (int k = 0; k < F; ++k) A.face_flux[tile.face(f, k, pc, pb)] = fsum[k];
#pragma unroll
        for (int m = 0; m < 3; ++m) A.face_flux[tile.face(f, F + m, pc, pb)] = (j == N) ? tl[m] : tr[m];
      }
    }
    amax = warp_max(amax);
    if ((tid & 31) == 0) red[tid >> 5] = amax;
    __syncthreads();  // also: scratch writes visible, line-end reads finished

    // ---- 5. divergence + sources, one thread per interior cell -----------
    const double inv_h = 1.0 / h;
    const double om = A.P.omega;
    const double* Us = A.U + (size_t)s * F * T::kS3;
    double* dU = A.dUdt + (size_t)s * F * T::kN3;
    for (int c = tid; c < N3; c += kLThreads) {
      const int x = c % N, y = (c / N) % N, z = c / (N * N);
      const int uc = tile.pad(x + G, y + G, z + G);  // in the sub-grid's padded array
      const int cs = tile.cell(c);                   // in its compact NN^3 array
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
      const double sx = Us[SX * T::kS3 + uc], sy = Us[SY * T::kS3 + uc], sz = Us[SZ * T::kS3 + uc];
      du[SX] = du[SX] + om * sy;
      du[SY] = du[SY] - om * sx;
      du[ZX] = du[ZX] + om * Us[ZY * T::kS3 + uc];
      du[ZY] = du[ZY] - om * Us[ZX * T::kS3 + uc];
      {
        // spin source w(x_c) x s, w = -omega z_hat x x_c: removes the torque
        // that the frame part s w_n of the momentum flux leaves in the face
        // torques, so that sum (x_c x s + z)_z is conserved for omega != 0
        const double xc = __dadd_rn(o[0], __dmul_rn(h, (x + ox) + 0.5));
        const double yc = __dadd_rn(o[1], __dmul_rn(h, (y + oy) + 0.5));
        const double wx = om * yc, wy = -(om * xc);
        du[ZX] = du[ZX] + wy * sz;
        du[ZY] = du[ZY] - wx * sz;
        du[ZZ] = du[ZZ] + (wx * sy - wy * sx);
      }
      if (A.g) {
        const double* gs = A.g + (size_t)s * 3 * T::kN3 + cs;
        const double gx = gs[0], gy = gs[T::kN3], gz = gs[2 * T::kN3];
        const double rho = Us[RHO * T::kS3 + uc];
        du[SX] = du[SX] + rho * gx;
        du[SY] = du[SY] + rho * gy;
        du[SZ] = du[SZ] + rho * gz;
        du[EGAS] = du[EGAS] + ((sx * gx + sy * gy) + sz * gz);
      }
#pragma unroll
      for (int k = 0; k < F; ++k) dU[k * T::kN3 + cs] = du[k];
    }
    if (tid == 0) {
      double m = red[0];
#pragma unroll
      for (int w = 1; w < kLThreads / 32; ++w) m = fmax(m, red[w]);
      if (T::kTiles == 1)
        A.amax[s] = m;
      else
        atomic_max_nonneg(A.amax + s, m);  // cleared before the launch
    }
    __syncthreads();  // scratch, line ends and red reused by the next tile
  }
  __syncthreads();
  if (tid == 0) mbar_inval(&bar);
}

size_t step_fp64_lines_smem_bytes(bool gate) { return (size_t)F * S3 * sizeof(double) + (gate ? 2 * S3 : 0); }

template <int NN>
static cudaError_t fp64_lines_attrs() {
  cudaError_t e = cudaSuccess;
  const void* fns[4] = {(const void*)hydro_step_fp64_lines_kernel<false, false, NN>,
                        (const void*)hydro_step_fp64_lines_kernel<true, false, NN>,
                        (const void*)hydro_step_fp64_lines_kernel<false, true, NN>,
                        (const void*)hydro_step_fp64_lines_kernel<true, true, NN>};
  for (int i = 0; i < 4 && e == cudaSuccess; ++i)
    e = cudaFuncSetAttribute(fns[i], cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)step_fp64_lines_smem_bytes(i & 1));
  return e;
}

// Once per device: the shared-memory opt-in and the run list (no
// allocation; call before any stream capture).
cudaError_t prepare_step_fp64_lines() {
  static unsigned long long done = 0;
  return once_per_device(&done, [] {
    cudaError_t e = fp64_lines_attrs<8>();
    if (e == cudaSuccess) e = fp64_lines_attrs<16>();
    if (e != cudaSuccess) return e;
    int n_axis = 0;
    const std::vector<uint32_t> runs = build_line_runs(&n_axis);
    if (runs.size() > (size_t)kMaxRuns) return cudaErrorInvalidValue;
    e = cudaMemcpyToSymbol(g_line_runs, runs.data(), runs.size() * sizeof(uint32_t));
    if (e == cudaSuccess) {
      g_runs_total = (int)runs.size();
      g_runs_axis = n_axis;
    }
    return e;
  });
}

size_t step_fp64_lines_per_cta() { return kLinesPerCta; }

template <int NN>
static void launch_fp64_lines_nn(const StepArgs64& A, int grid, int n_runs, cudaStream_t st) {
  const size_t sm1 = step_fp64_lines_smem_bytes(true), sm0 = step_fp64_lines_smem_bytes(false);
  if (A.gate && A.P.contact)
    hydro_step_fp64_lines_kernel<true, true, NN><<<grid, kLThreads, sm1, st>>>(A, n_runs);
  else if (A.gate)
    hydro_step_fp64_lines_kernel<true, false, NN><<<grid, kLThreads, sm1, st>>>(A, n_runs);
  else if (A.P.contact)
    hydro_step_fp64_lines_kernel<false, true, NN><<<grid, kLThreads, sm0, st>>>(A, n_runs);
  else
    hydro_step_fp64_lines_kernel<false, false, NN><<<grid, kLThreads, sm0, st>>>(A, n_runs);
}

// The FP64 step with every line once: grid persistent CTAs over the
// A.n_sub * (nn/8)^3 tiles; A.lines holds grid * step_fp64_lines_per_cta()
// doubles.  With 16^3 sub-grids the amax of a sub-grid is the atomic maximum
// over its tiles, cleared here first.
cudaError_t launch_step_fp64_lines(const StepArgs64& A, int grid, int nn, cudaStream_t st) {
  cudaError_t e = prepare_step_fp64_lines();
  if (e != cudaSuccess) return e;
  if (!A.lines) return cudaErrorInvalidValue;
  const int n_runs = A.P.face_points == 1 ? g_runs_axis : g_runs_total;
  if (nn == 16) {
    e = cudaMemsetAsync(A.amax, 0, (size_t)A.n_sub * sizeof(double), st);
    if (e != cudaSuccess) return e;
    launch_fp64_lines_nn<16>(A, grid, n_runs, st);
  } else {
    launch_fp64_lines_nn<8>(A, grid, n_runs, st);
  }
  return cudaGetLastError();
}

}  // namespace hyd

namespace hyd {

__global__ void selftest_arith_kernel(const double* __restrict__ x, const double* __restrict__ y, int n,
                                      double* __restrict__ out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double a = x[i], b = y[i];
    out[2 * i] = half64(a);
    out[2 * i + 1] = slope64(a, b);
  }
}

}  // namespace hyd

extern "C" int hydro_selftest_arith(const double* x, const double* y, int n, double* out, void* stream) {
  if (n < 0 || (n > 0 && (!x || !y || !out))) return HYDRO_EINVAL;
  if (n == 0) return HYDRO_OK;
  const int grid = (n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024;
  hyd::selftest_arith_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(x, y, n, out);
  return cudaGetLastError() == cudaSuccess ? HYDRO_OK : HYDRO_ECUDA;
}
