// hydro_step_fp64.cu -- the per-sub-grid hydro step in FP64 (the plain method).
//
// One persistent CTA per SM loops over sub-grids.  For each sub-grid:
//   1. the ghost-padded state (10 fields x 14^3 doubles, 219,520 B) is staged
//      into shared memory by bulk TMA copies completing on an mbarrier;
//   2. primitives (rho, v, eps with the dual-energy selection, tau, z,
//      species) replace the conserved values in place (Sec. III-B, Bryan 1995);
//   3. 192 threads, one per (axis a, transverse row), sweep their row along a.
//      At each cell j they run PPM (Colella & Woodward 1984) on the 9 lines
//      d = e_a + t1 e_b + t2 e_c; the line's +d end is the left state of face
//      j+1/2 at point (t1,t2), its -d end the right state of face j-1/2 at
//      point (-t1,-t2).  The left states are carried to the next cell, so every
//      line is evaluated once per axis and both of its ends are used.  At each
//      face the 9 Kurganov-Tadmor point fluxes are summed with the Simpson
//      weights (1,4,1)x(1,4,1)/36, together with the torques of the momentum
//      flux about both cell centres;
//   4. per-axis flux differences go to a per-CTA scratch buffer in global
//      memory (L2-resident); one thread per interior cell then forms the
//      divergence in a fixed order, adds the rotating-frame, gravity and spin
//      sources and writes dU/dt;
//   5. the maximum signal speed is reduced by warp shuffles, then across warps.
// The PPM and primitive arithmetic uses explicitly rounded operations (no FMA
// contraction) so that every limiter branch is decided on exactly the values
// the FP64 oracle sees; the flux arithmetic may contract.
#include "hydro_common.cuh"
#include "hydro_fp64.cuh"
#include "hydro_mixed.cuh"

namespace hyd {

constexpr int kThreads64 = NROW;  // 192
constexpr long kWaitPolls = 1L << 24;

// kGate: the learned smoothness indicator is on (A.gate): its decisions per
// reconstructed cell follow the primitives in shared memory ([S3] bytes of
// flags and [S3] of predictions after the state).  kContact: contact
// steepening (A.P.contact; with the indicator, only the cells it does not
// mark smooth are steepened).  NN: the
// sub-grids' edge (8, or 16: each 8^3 octant tile is a work unit staged from
// its 14^3 window of the 22^3 array, Tile<NN>).
template <bool kGate, bool kContact = false, int NN = N>
__global__ void __launch_bounds__(kThreads64, 1) hydro_step_fp64_kernel(StepArgs64 A) {
  using T = Tile<NN>;
  extern __shared__ __align__(128) double Q[];  // [F][S3], then the indicator's flags
  uint8_t* smooth = reinterpret_cast<uint8_t*>(Q + F * S3);
  __shared__ __align__(8) uint64_t bar;
  __shared__ double red[kThreads64 / 32];
  __shared__ int bail;
  const int tid = threadIdx.x;
  double* __restrict__ D = A.scratch + (size_t)blockIdx.x * kScratchPerSub;

  if (tid == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
    bail = 0;
  }
  __syncthreads();

  // this thread's row: axis a, transverse axes b < c at positions pb, pc.
  // Warp w of the axis takes pb in [4w, 4w+4) x pc in [0, 8): with the cell
  // strides (1, 14, 196) each half-warp's FP64 stencil loads then fall on 16
  // (y rows) or 8 (x and z rows) distinct bank pairs, against 8 for all axes
  // with pb running fastest.
  static_assert(N == 8 && S == 14, "row-to-warp map assumes 8^3 interiors with 3-cell ghosts");
  const int a = tid / (N * N);
  const int r = tid % (N * N);
  const int pb = ((r >> 5) << 2) | (r & 3), pc = (r & 31) >> 2;
  const int b = (a == 0) ? 1 : 0;
  const int cx = (a == 2) ? 1 : 2;
  const int sa = axis_stride(a), sb = axis_stride(b), sc = axis_stride(cx);

  uint32_t phase = 0;
  for (int u = blockIdx.x; u < A.n_sub * T::kTiles; u += gridDim.x) {
    const T tile(u);
    const int s = tile.s;
    // ---- 1. stage the tile into shared memory (bulk TMA) ----------------
    // 8^3 sub-grid: one copy per field of its contiguous padded block; 16^3
    // octant: one copy per (field, z, y) row of its 14^3 window (112 bytes,
    // 16-byte aligned: the octant offsets are 0 or 8 cells), issued by the
    // 32 lanes of warp 0 after lane 0 has announced the total.
    if (tid < 32) {
      if (tid == 0) {
        fence_proxy_async();
        mbar_expect_tx(&bar, (uint32_t)(F * S3 * sizeof(double)));
      }
      __syncwarp();
      const double* src = A.U + (size_t)s * F * T::kS3;
      if (NN == N) {
        if (tid == 0)
#pragma unroll 1
          for (int k = 0; k < F; ++k) bulk_g2s(Q + k * S3, src + (size_t)k * S3, S3 * sizeof(double), &bar);
      } else {
#pragma unroll 1
        for (int r = tid; r < F * S * S; r += 32) {
          const int k = r / (S * S), z = (r / S) % S, y = r % S;
          bulk_g2s(Q + k * S3 + (z * S + y) * S, src + (size_t)k * T::kS3 + tile.pad(0, y, z), S * sizeof(double),
                   &bar);
        }
      }
    }
    if (!mbar_wait_bounded(&bar, phase, kWaitPolls)) {
      atomicOr(A.status, 2u);
      bail = 1;
    }
    phase ^= 1u;
    __syncthreads();
    if (bail) break;

    // ---- 2. primitives in place ----------------------------------------
    bool bad = false;
    for (int c = tid; c < S3; c += kThreads64) {
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

    // ---- 2b. learned smoothness indicator (gate_phase; features in FP32) ----
    if (kGate)
      gate_phase<double, kThreads64>(Q, (float)A.P.gm1, A.gate_w, A.gate_logit_thr, A.gate_zero_smooth, smooth,
                                     smooth + S3);

    // ---- 3. row sweep ------------------------------------------------------
    const int ox = tile.o[0], oy = tile.o[1];
    const double h = A.h[s];
    const double half_h = 0.5 * h;
    const double o[3] = {A.origin[3 * s + 0], A.origin[3 * s + 1], A.origin[3 * s + 2]};
    double amax = 0.0;
    double plus[9][F];
    double fprev[F], trprev[3];
    // smem index of the row's cell at a-index j
    const int c0 = ((axis_comp(2, a, b, 0, pb, pc) + G) * S + (axis_comp(1, a, b, 0, pb, pc) + G)) * S +
                   (axis_comp(0, a, b, 0, pb, pc) + G);
#pragma unroll 1
    for (int j = -1; j <= N; ++j) {
      const int cj = c0 + j * sa;
      double fsum[F], T[3];
#pragma unroll
      for (int k = 0; k < F; ++k) fsum[k] = 0.0;
      T[0] = T[1] = T[2] = 0.0;
      // left cell of face j-1/2 is (j-1) along a
      const int ci0 = axis_comp(0, a, b, j - 1, pb, pc) + ox, ci1 = axis_comp(1, a, b, j - 1, pb, pc) + oy;
      // the 9 face points as 4 mirrored pairs and the centre (p = 4); with one
      // flux point per face (the old module) only the centre
#pragma unroll 1
      for (int p = A.P.face_points == 1 ? 4 : 0; p <= 4; ++p) {
        const int t1 = p / 3 - 1, t2 = p % 3 - 1;  // point p; its mirror 8-p has (-t1,-t2)
        double qpA[F], qmA[F], qpB[F], qmB[F];
        if (kGate && smooth[cj]) {
          line10u(Q, cj, sa + t1 * sb + t2 * sc, qpA, qmA);
          if (p != 4) line10u(Q, cj, sa - t1 * sb - t2 * sc, qpB, qmB);
        } else if (kContact) {
          line10c(Q, cj, sa + t1 * sb + t2 * sc, A.P, qpA, qmA);
          if (p != 4) line10c(Q, cj, sa - t1 * sb - t2 * sc, A.P, qpB, qmB);
        } else {
          line10(Q, cj, sa + t1 * sb + t2 * sc, qpA, qmA);
          if (p != 4) line10(Q, cj, sa - t1 * sb - t2 * sc, qpB, qmB);
        }
        if (A.P.spin) {
          // the cell's spin fed back into the velocity at both ends of both
          // lines (spin_dv64; the lines kernel's values, bit for bit)
          const double k3h = 3.0 / h;
          double dv[3];
          const double gg1 = rmul(A.P.gamma, A.P.gm1);
          spin_dv64(Q[RHO * S3 + cj], Q[EGAS * S3 + cj], Q[ZX * S3 + cj], Q[ZY * S3 + cj], Q[ZZ * S3 + cj], k3h,
                    gg1, axis_comp(0, a, b, 1, t1, t2), axis_comp(1, a, b, 1, t1, t2), axis_comp(2, a, b, 1, t1, t2),
                    dv);
#pragma unroll
          for (int m = 0; m < 3; ++m) {
            qpA[1 + m] = radd(qpA[1 + m], dv[m]);
            qmA[1 + m] = rsub(qmA[1 + m], dv[m]);
          }
          if (p != 4) {
            spin_dv64(Q[RHO * S3 + cj], Q[EGAS * S3 + cj], Q[ZX * S3 + cj], Q[ZY * S3 + cj], Q[ZZ * S3 + cj], k3h,
                      gg1, axis_comp(0, a, b, 1, -t1, -t2), axis_comp(1, a, b, 1, -t1, -t2),
                      axis_comp(2, a, b, 1, -t1, -t2), dv);
#pragma unroll
            for (int m = 0; m < 3; ++m) {
              qpB[1 + m] = radd(qpB[1 + m], dv[m]);
              qmB[1 + m] = rsub(qmB[1 + m], dv[m]);
            }
          }
        }
        if (j >= 0) {
#pragma unroll 1
          for (int side = 0; side < 2; ++side) {
            if (p == 4 && side == 1) continue;
            // side 0: point 8-p (offsets -t1,-t2) with right state qmA;
            // side 1: point p (offsets t1,t2) with right state qmB.
            const int u1 = side ? t1 : -t1, u2 = side ? t2 : -t2;
            const int pt = (u1 + 1) * 3 + (u2 + 1);
            const int d0 = axis_comp(0, a, b, 1, u1, u2), d1 = axis_comp(1, a, b, 1, u1, u2),
                      d2 = axis_comp(2, a, b, 1, u1, u2);
            const double xq = o[0] + h * ((ci0 + 0.5) + 0.5 * d0);
            const double yq = o[1] + h * ((ci1 + 0.5) + 0.5 * d1);
            // half the Simpson weight (1, 4, 1) x (1, 4, 1) / 36 of the point; 1/2
            // for the single-point face flux
            const double hw = A.P.face_points == 1 ? 0.5
                             : (u1 == 0 && u2 == 0) ? (8.0 / 36.0) : (u1 == 0 || u2 == 0) ? (2.0 / 36.0) : (0.5 / 36.0);
            point64(plus[pt], side ? qmB : qmA, a, xq, yq, hw, d0, d1, d2, A.P, fsum, T, amax);
          }
        }
#pragma unroll
        for (int k = 0; k < F; ++k) {
          plus[p][k] = qpA[k];
          if (p != 4) plus[8 - p][k] = qpB[k];
        }
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
      if (j >= 0) {
#pragma unroll
        for (int k = 0; k < F; ++k) fprev[k] = fsum[k];
        trprev[0] = tr[0];
        trprev[1] = tr[1];
        trprev[2] = tr[2];
      }
      if (A.face_flux && (j == 0 || j == N) && tile.outer(2 * a + (j == N ? 1 : 0))) {
        // sub-grid boundary face: sums and the torque about the interior cell
        const int f = 2 * a + (j == N ? 1 : 0);
#pragma unroll
        for (int k = 0; k < F; ++k) A.face_flux[tile.face(f, k, pc, pb)] = fsum[k];
#pragma unroll
        for (int m = 0; m < 3; ++m) A.face_flux[tile.face(f, F + m, pc, pb)] = (j == N) ? tl[m] : tr[m];
      }
    }
    // block-wide amax; order the generic-proxy shared-memory accesses of this
    // sub-grid before the next bulk copy overwrites the buffer
    fence_proxy_async();
    amax = warp_max(amax);
    if ((tid & 31) == 0) red[tid >> 5] = amax;
    __syncthreads();  // also: scratch writes visible, shared Q reads finished

    // ---- 4. divergence + sources, one thread per interior cell -----------
    const double inv_h = 1.0 / h;
    const double om = A.P.omega;
    const double* Us = A.U + (size_t)s * F * T::kS3;
    double* dU = A.dUdt + (size_t)s * F * T::kN3;
    for (int c = tid; c < N3; c += kThreads64) {
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
      for (int w = 1; w < kThreads64 / 32; ++w) m = fmax(m, red[w]);
      if (T::kTiles == 1)
        A.amax[s] = m;
      else
        atomic_max_nonneg(A.amax + s, m);  // cleared before the launch
    }
    __syncthreads();  // scratch and red reused by the next sub-grid
  }
  __syncthreads();
  if (tid == 0) mbar_inval(&bar);
}

size_t step_fp64_smem_bytes(bool gate = false) { return (size_t)F * S3 * sizeof(double) + (gate ? 2 * S3 : 0); }

// Opt in to the kernel's dynamic shared memory once per device (no
// allocation; call before any stream capture).
template <int NN>
static cudaError_t fp64_attrs() {
  cudaError_t e = cudaFuncSetAttribute(hydro_step_fp64_kernel<false, false, NN>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)step_fp64_smem_bytes(false));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(hydro_step_fp64_kernel<true, false, NN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)step_fp64_smem_bytes(true));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(hydro_step_fp64_kernel<false, true, NN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)step_fp64_smem_bytes(false));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(hydro_step_fp64_kernel<true, true, NN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)step_fp64_smem_bytes(true));
  return e;
}

cudaError_t prepare_step_fp64() {
  static unsigned long long done = 0;
  return once_per_device(&done, [] {
    cudaError_t e = fp64_attrs<8>();
    return e == cudaSuccess ? fp64_attrs<16>() : e;
  });
}

template <int NN>
static void launch_fp64_nn(const StepArgs64& A, int grid, cudaStream_t st) {
  if (A.gate && A.P.contact)
    hydro_step_fp64_kernel<true, true, NN><<<grid, kThreads64, step_fp64_smem_bytes(true), st>>>(A);
  else if (A.gate)
    hydro_step_fp64_kernel<true, false, NN><<<grid, kThreads64, step_fp64_smem_bytes(true), st>>>(A);
  else if (A.P.contact)
    hydro_step_fp64_kernel<false, true, NN><<<grid, kThreads64, step_fp64_smem_bytes(false), st>>>(A);
  else
    hydro_step_fp64_kernel<false, false, NN><<<grid, kThreads64, step_fp64_smem_bytes(false), st>>>(A);
}

// nn: the sub-grids' edge (8 or 16); grid: persistent CTAs over the
// A.n_sub * (nn/8)^3 tiles.  With 16^3 sub-grids the amax of a sub-grid is
// the atomic maximum over its tiles, cleared here first.
cudaError_t launch_step_fp64(const StepArgs64& A, int grid, int nn, cudaStream_t st) {
  cudaError_t e = prepare_step_fp64();
  if (e != cudaSuccess) return e;
  if (nn == 16) {
    e = cudaMemsetAsync(A.amax, 0, (size_t)A.n_sub * sizeof(double), st);
    if (e != cudaSuccess) return e;
    launch_fp64_nn<16>(A, grid, st);
  } else {
    launch_fp64_nn<8>(A, grid, st);
  }
  return cudaGetLastError();
}

}  // namespace hyd
