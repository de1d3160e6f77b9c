// hydro_rk3_fused.cuh -- the fused RK3 step's kernel and host templates,
// instantiated for 8^3 sub-grids in hydro_rk3_fused.cu and for 16^3 ones in
// hydro_rk3_fused16.cu.
//
// One whole SSP-RK3 time step (three hydro iterations,
// Sec. IV-A.2) of a uniform mesh in mixed precision, as one persistent
// cooperative launch.
//
// The separate-launch step (hydro_graph.cu) runs per stage a ghost fill, the
// step kernel and the update, with the whole mesh finishing each launch
// before the next starts.  Here, state X -> Y:
//   stage 0  every sub-grid: dU0 = L(X), amax (static schedule);
//            one grid-wide barrier; dt = cfl min h/amax (every CTA); each
//            CTA writes U1 = X + dt dU0 (with the tracer resync) of its
//            stage-0 sub-grids into the interiors of Y and publishes them;
//   stage 1  sub-grid s reads U1 and writes U2 = 3/4 X + 1/4 (U1 + dt L(U1))
//            to an interior-only scratch and publishes it;
//   stage 2  sub-grid s reads U2 and writes U3 = 1/3 X + 2/3 (U2 + dt L(U2))
//            into the interiors of Y.
// Ghost cells are read straight from the neighbouring sub-grids' interiors
// through the boundary map of hydro_fill_ghosts_uniform, so no ghost layer
// is written and no separate update runs.  Stage-1 and stage-2 sub-grids come
// from one work counter, all stage-1 ones first; a sub-grid waits until its
// 27 neighbours (itself included) have published its input (U1, U2).  U3
// overwrites U1 in Y only after every reader of that U1 (the neighbours'
// stage 1) has published.  The waits end: every CTA writes its U1 before it
// takes a unit, so a stage-1 unit waits only for CTAs that are not waiting,
// and a stage-2 unit waits only for stage-1 units, all taken before it by
// resident CTAs.  Each wait is still bounded in time and polls and reports
// HYDRO_ST_TIMEOUT.
//
// The row sweep reads the FP32 primitives of its windows (prims_mixed of
// the FP64 state) from a buffer that the producer of each state fills, once
// per cell: a pass over X's interiors before stage 0 (with one more grid
// barrier), the U1 writes and the stage-1 stores.  The separate launches
// recover them in every padded cell of every window, from the same FP64
// values, so the bits are the same; the conversions and the dual-energy
// recovery in FP64 drop from 2,744 to 512 per sub-grid and stage.
//
// With 16^3 sub-grids a work unit is one of a sub-grid's eight 8^3 octant
// tiles (Tile), and a sub-grid's U1 or U2 counts as published once all
// eight tiles have added theirs to its flag.
//
// The per-cell arithmetic is the separate-launch step's own (the same
// sub-grid body and rk3_cell with the same operands), so the interiors of Y
// and dt equal its results bit for bit.  The ghost layers of Y are not
// written, and dUdt holds the first stage's rates.
#pragma once
#include "hydro_mixed_planes.cuh"

namespace hyd {

struct FusedArgs {
  StepArgs64 S;         // U = X (padded), dUdt = dU0 [n][F][N3], amax, scratch, status, ...
  double* Y;            // padded output state (interiors written)
  double* U2;           // [n][F][N3] second-stage state
  double* dt_out;       // the step's dt
  unsigned* sync;       // zero at launch: [0] barrier arrivals, [1] work counter, [2] abort,
                        // [kSyncHead + s] U2 of sub-grid s published, [kSyncHead + n + s] its U1
  int nbx, nby, nbz, bc;
  double cfl, eta2, inv_gamma;
  double alpha[3], beta[3];  // the stage coefficients of the update kernel
  long long wait_ns;    // bound of every wait
  float* P[2];          // FP32 primitives of the stage inputs, [n][F][NN^3] each (row
                        // sweep only; NULL otherwise): P[0] holds X's, then U2's;
                        // P[1] holds U1's
};
constexpr int kSyncHead = 4;

// Where the state of a tile (an 8^3 sub-grid, or an octant of a 16^3 one:
// Tile) comes from, per stage (see above).
// The FP32 primitives of one cell's state u (prims_mixed) into P at
// compact cell ci of sub-grid s (NN^3 = n3 cells); a non-physical cell sets
// the status bit.
__device__ __forceinline__ void store_prims(const FusedArgs& A, float* P, int s, int ci, const double u[F], int n3) {
  float q[F];
  if (!prims_mixed(u, A.S.P.eta1, (float)A.S.P.gamma, q)) atomicOr(A.S.status, 1u);
  float* p = P + (size_t)s * F * n3 + ci;
#pragma unroll
  for (int k = 0; k < F; ++k) p[(size_t)k * n3] = q[k];
}

// kPrims: the row sweep reads the FP32 primitives of its window from P
// (recovered once per cell by the tile that produced the state) instead of
// recovering them from the FP64 state of every padded cell.
template <int NN, bool kPrimsIn = false>
struct FusedIo {
  using T = Tile<NN>;
  static constexpr bool kPrims = kPrimsIn;
  const FusedArgs& A;
  int stage;
  double dt;
  struct Sub {
    T t;
    int kx, ky, kz;  // the sub-grid's position in the mesh
  };
  __device__ __forceinline__ Sub begin(int u) const {
    const T t(u);
    return Sub{t, t.s % A.nbx, (t.s / A.nbx) % A.nby, t.s / (A.nbx * A.nby)};
  }
  __device__ __forceinline__ int sidx(const Sub& q) const { return q.t.s; }
  __device__ __forceinline__ int offx(const Sub& q) const { return q.t.o[0]; }
  __device__ __forceinline__ int offy(const Sub& q) const { return q.t.o[1]; }
  __device__ __forceinline__ void grav(const Sub& q, int c, double& gx, double& gy, double& gz) const {
    const double* gs = A.S.g + (size_t)q.t.s * 3 * T::kN3 + q.t.cell(c);
    gx = gs[0];
    gy = gs[T::kN3];
    gz = gs[2 * T::kN3];
  }
  // the fused step exports no boundary faces (uniform meshes only)
  __device__ __forceinline__ void face(const Sub&, int, int, int, int, double) const {}
  // Stage input state of interior cell (os; oi compact, op padded index of
  // the sub-grid): fields f0 .. f0 + nf - 1 into u[0 .. nf-1].
  __device__ __forceinline__ void state(int os, int oi, int op, double* u, int f0 = 0, int nf = F) const {
    if (stage == 0) {
      const double* __restrict__ x = A.S.U + (size_t)os * F * T::kS3 + op;
#pragma unroll
      for (int k = 0; k < nf; ++k) u[k] = __ldg(x + (size_t)(f0 + k) * T::kS3);
    } else if (stage == 1) {
      const double* q = A.Y + (size_t)os * F * T::kS3 + op;
#pragma unroll
      for (int k = 0; k < nf; ++k) u[k] = __ldcg(q + (size_t)(f0 + k) * T::kS3);
    } else {
      const double* q = A.U2 + (size_t)os * F * T::kN3 + oi;
#pragma unroll
      for (int k = 0; k < nf; ++k) u[k] = __ldcg(q + (size_t)(f0 + k) * T::kN3);
    }
  }
  // Padded cell c of the tile: its source sub-grid and cell under the
  // uniform mesh's boundary map, fields f0 .. f0 + nf - 1.
  __device__ __forceinline__ void load_fields(const Sub& q, int c, int f0, int nf, double* u) const {
    const int nx = A.nbx * NN, ny = A.nby * NN, nz = A.nbz * NN;
    const int gx = bc_map(q.kx * NN + q.t.o[0] + c % S - G, nx, A.bc);
    const int gy = bc_map(q.ky * NN + q.t.o[1] + (c / S) % S - G, ny, A.bc);
    const int gz = bc_map(q.kz * NN + q.t.o[2] + c / (S * S) - G, nz, A.bc);
    const int os = ((gz / NN) * A.nby + (gy / NN)) * A.nbx + (gx / NN);
    const int ix = gx & (NN - 1), iy = gy & (NN - 1), iz = gz & (NN - 1);
    state(os, (iz * NN + iy) * NN + ix, ((iz + G) * T::kS + (iy + G)) * T::kS + (ix + G), u, f0, nf);
  }
  __device__ __forceinline__ void load(const Sub& q, int c, double u[F]) const { load_fields(q, c, 0, F, u); }
  // The primitives of padded cell c of the tile (kPrims): from the stage
  // input's primitive buffer, at the source cell of the boundary map.
  __device__ __forceinline__ void load_prims(const Sub& q, int c, float* u) const {
    const int nx = A.nbx * NN, ny = A.nby * NN, nz = A.nbz * NN;
    const int gx = bc_map(q.kx * NN + q.t.o[0] + c % S - G, nx, A.bc);
    const int gy = bc_map(q.ky * NN + q.t.o[1] + (c / S) % S - G, ny, A.bc);
    const int gz = bc_map(q.kz * NN + q.t.o[2] + c / (S * S) - G, nz, A.bc);
    const int os = ((gz / NN) * A.nby + (gy / NN)) * A.nbx + (gx / NN);
    const int ix = gx & (NN - 1), iy = gy & (NN - 1), iz = gz & (NN - 1);
    const float* p = A.P[stage == 1 ? 1 : 0] + (size_t)os * F * T::kN3 + (iz * NN + iy) * NN + ix;
#pragma unroll
    for (int k = 0; k < F; ++k) u[k] = __ldcg(p + (size_t)k * T::kN3);
  }
  __device__ __forceinline__ void own(const Sub& q, int c, int uc, double u[F]) const {
    state(q.t.s, q.t.cell(c), q.t.pad(uc), u);
  }
  __device__ __forceinline__ void store(const Sub& q, int c, int uc, const double du[F], const double u[F]) const {
    const int s = q.t.s, ci = q.t.cell(c), pi = q.t.pad(uc);
    if (stage == 0) {
      double* r = A.S.dUdt + (size_t)s * F * T::kN3 + ci;
#pragma unroll
      for (int k = 0; k < F; ++k) r[(size_t)k * T::kN3] = du[k];
      return;
    }
    const double* __restrict__ x = A.S.U + (size_t)s * F * T::kS3 + pi;
    double xv[F], un[F];
#pragma unroll
    for (int k = 0; k < F; ++k) xv[k] = __ldg(x + (size_t)k * T::kS3);
    rk3_cell<true>(u, xv, du, dt, A.alpha[stage], A.beta[stage], A.eta2, A.inv_gamma, un);
    if (stage == 1) {
      double* o = A.U2 + (size_t)s * F * T::kN3 + ci;
#pragma unroll
      for (int k = 0; k < F; ++k) o[(size_t)k * T::kN3] = un[k];
      if (kPrims) store_prims(A, A.P[0], s, ci, un, T::kN3);  // U2's, for stage 2
    } else {
      double* o = A.Y + (size_t)s * F * T::kS3 + pi;
#pragma unroll
      for (int k = 0; k < F; ++k) o[(size_t)k * T::kS3] = un[k];
    }
  }
  __device__ __forceinline__ void amax(const Sub& q, double m) const {
    if (stage != 0) return;
    if (T::kTiles == 1)
      A.S.amax[q.t.s] = m;
    else
      atomic_max_nonneg(A.S.amax + q.t.s, m);  // cleared before the launch
  }
};

// ---- bounded inter-CTA waits ---------------------------------------------
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Wait until *p >= target.  Gives up (false) after limit_ns of polling, after
// 2^26 polls whatever the clock says, or as soon as *abort is set.
static __device__ bool wait_geq(const unsigned* p, unsigned target, const unsigned* abort, long long limit_ns) {
  if (ld_acquire(p) >= target) return true;
  const unsigned long long t0 = global_ns();
  for (long i = 0; i < (1l << 26); ++i) {
    __nanosleep(128);
    if (ld_acquire(p) >= target) return true;
    if (ld_acquire(abort) != 0u) return false;
    if ((long long)(global_ns() - t0) > limit_ns) return false;
  }
  return false;
}

// Threads 0..26 wait until flags[] of the 27 neighbours of sub-grid s (under
// the boundary map, s itself included) reach target (the sub-grid's tile
// count: each tile adds one when its part is published); on a timeout the
// launch is aborted.  Returns, to every thread, whether all were reached.
static __device__ bool wait_neighbours(const FusedArgs& A, const unsigned* flags, int s, unsigned target,
                                const unsigned* abort, int* sh_ok) {
  const int tid = threadIdx.x;
  if (tid == 0) *sh_ok = 1;
  __syncthreads();
  if (tid < 27) {
    const int kx = s % A.nbx, ky = (s / A.nbx) % A.nby, kz = s / (A.nbx * A.nby);
    int nx = kx + tid % 3 - 1, ny = ky + (tid / 3) % 3 - 1, nz = kz + tid / 9 - 1;
    if (A.bc == 0) {
      nx = (nx + A.nbx) % A.nbx;
      ny = (ny + A.nby) % A.nby;
      nz = (nz + A.nbz) % A.nbz;
    } else {
      nx = min(max(nx, 0), A.nbx - 1);
      ny = min(max(ny, 0), A.nby - 1);
      nz = min(max(nz, 0), A.nbz - 1);
    }
    if (!wait_geq(flags + (nz * A.nby + ny) * A.nbx + nx, target, abort, A.wait_ns)) {
      atomicOr(A.S.status, 2u);
      atomicExch(const_cast<unsigned*>(abort), 1u);
      *sh_ok = 0;
    }
  }
  __syncthreads();
  return *sh_ok != 0;
}

// The sub-grid bodies the fused step can run, with their launch shapes: the
// row sweep (two CTAs of kThreadsMx threads per SM, per-CTA scratch of flux
// differences; with or without the learned indicator and contact
// steepening) and the plane sweep (one CTA of kThreadsPl threads per SM).
template <bool kGate, bool kContact, bool kSpin = false>
struct RowBody {
  static constexpr int kThreads = kThreadsMx, kMinBlocks = 2;
  static constexpr bool kPrims = true;  // reads its windows' primitives from FusedArgs::P
  static constexpr size_t kRed = (kMixedSmemBytes + 15) / 16 * 16;
  static constexpr size_t kSmem = kRed + sizeof(float) * (kThreadsMx / 32);
  RowMap R;
  float* Qf;
  float* red;
  double* D;
  __device__ RowBody(const StepArgs64& S, unsigned char* sm)
      : R(row_map(threadIdx.x)), Qf(reinterpret_cast<float*>(sm)), red(reinterpret_cast<float*>(sm + kRed)),
        D(S.scratch + (size_t)blockIdx.x * kScratchPerSub) {}
  template <class Io>
  __device__ __forceinline__ void run(const StepArgs64& S, const Io& io, int s) const {
    mixed_subgrid<kGate, kContact, kSpin>(S, io, s, R, Qf, red, D);
  }
};
template <bool kContact, bool kSpin = false>
struct PlaneBody {
  static constexpr int kThreads = kThreadsPl, kMinBlocks = 1;
  static constexpr bool kPrims = false;
  static constexpr size_t kSmem = kPlaneSmemBytes;
  unsigned char* sm;
  __device__ PlaneBody(const StepArgs64&, unsigned char* p) : sm(p) {}
  template <class Io>
  __device__ __forceinline__ void run(const StepArgs64& S, const Io& io, int s) const {
    mixed_subgrid_planes<kContact, kSpin>(S, io, s, sm);
  }
};

template <class Body, int NN>
__global__ void __launch_bounds__(Body::kThreads, Body::kMinBlocks) hydro_rk3_fused_kernel(FusedArgs A) {
  using T = Tile<NN>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ double dred[Body::kThreads / 32];
  __shared__ int sh_unit, sh_ok;
  const int tid = threadIdx.x;
  const int n = A.S.n_sub;
  const int units = n * T::kTiles;  // work units: tiles
  const Body body(A.S, smem_raw);
  unsigned* arrive = A.sync;
  unsigned* counter = A.sync + 1;
  unsigned* abort = A.sync + 2;
  unsigned* published = A.sync + kSyncHead;    // U2 tiles done, per sub-grid
  unsigned* published1 = published + n;        // U1 tiles done, per sub-grid

  using Io = FusedIo<NN, Body::kPrims>;
  // grid-wide barrier number k (1, 2, ...): every CTA arrives once per barrier
  auto grid_sync = [&](unsigned k) {
    if (tid == 0) {
      __threadfence();
      atomicAdd(arrive, 1u);
      const bool ok = wait_geq(arrive, k * gridDim.x, abort, A.wait_ns);
      if (!ok) {
        atomicOr(A.S.status, 2u);
        atomicExch(abort, 1u);
      }
      sh_ok = ok;
    }
    __syncthreads();
    return sh_ok != 0;
  };
  unsigned barriers = 0;

  // ---- the primitives of X's interiors (row sweep), once per cell --------
  if (Body::kPrims) {
    for (int u = blockIdx.x; u < units; u += gridDim.x) {
      const T t(u);
      const double* __restrict__ x = A.S.U + (size_t)t.s * F * T::kS3;
      for (int c = tid; c < N3; c += Body::kThreads) {
        const int uc = t.pad((((c >> 6) + G) * S + (((c >> 3) & (N - 1)) + G)) * S + ((c & (N - 1)) + G));
        double xv[F];
#pragma unroll
        for (int k = 0; k < F; ++k) xv[k] = __ldg(x + (size_t)k * T::kS3 + uc);
        store_prims(A, A.P[0], t.s, t.cell(c), xv, T::kN3);
      }
    }
    if (!grid_sync(++barriers)) return;
  }

  // ---- stage 0 --------------------------------------------------------
  {
    const Io io{A, 0, 0.0};
    for (int u = blockIdx.x; u < units; u += gridDim.x) body.run(A.S, io, u);
  }

  // ---- grid-wide barrier, then dt (the reduction of hydro_dt_kernel) ----
  if (!grid_sync(++barriers)) return;
  double m = INFINITY;
  for (int i = tid; i < n; i += Body::kThreads) m = fmin(m, A.S.h[i] / __ldcg(A.S.amax + i));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmin(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((tid & 31) == 0) dred[tid >> 5] = m;
  __syncthreads();
  m = dred[0];
#pragma unroll
  for (int w = 1; w < Body::kThreads / 32; ++w) m = fmin(m, dred[w]);
  const double dt = A.cfl * m;
  if (blockIdx.x == 0 && tid == 0) *A.dt_out = dt;

  // ---- U1 of this CTA's stage-0 tiles, into the interiors of Y ---------
  for (int u = blockIdx.x; u < units; u += gridDim.x) {
    const T t(u);
    const double* __restrict__ x = A.S.U + (size_t)t.s * F * T::kS3;
    const double* r = A.S.dUdt + (size_t)t.s * F * T::kN3;
    double* y = A.Y + (size_t)t.s * F * T::kS3;
    for (int c = tid; c < N3; c += Body::kThreads) {
      const int uc = t.pad((((c >> 6) + G) * S + (((c >> 3) & (N - 1)) + G)) * S + ((c & (N - 1)) + G));
      const int ci = t.cell(c);
      double xv[F], rv[F], u1[F];
#pragma unroll
      for (int k = 0; k < F; ++k) {
        xv[k] = __ldg(x + (size_t)k * T::kS3 + uc);
        rv[k] = r[(size_t)k * T::kN3 + ci];
      }
      rk3_cell<true>(xv, xv, rv, dt, A.alpha[0], A.beta[0], A.eta2, A.inv_gamma, u1);
#pragma unroll
      for (int k = 0; k < F; ++k) y[(size_t)k * T::kS3 + uc] = u1[k];
      if (Body::kPrims) store_prims(A, A.P[1], t.s, ci, u1, T::kN3);
    }
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      atomicAdd(published1 + t.s, 1u);
    }
  }

  // ---- stages 1 and 2 from one work counter ---------------------------
  for (;;) {
    if (tid == 0) {
      int u = (int)atomicAdd(counter, 1u);
      if (ld_acquire(abort) != 0u) u = 2 * units;
      sh_unit = u;
    }
    __syncthreads();
    const int u = sh_unit;
    if (u >= 2 * units) break;
    const int stage = u < units ? 1 : 2;
    const int tu = stage == 1 ? u : u - units;
    const int s = tu / T::kTiles;
    if (!wait_neighbours(A, stage == 1 ? published1 : published, s, (unsigned)T::kTiles, abort, &sh_ok)) break;
    body.run(A.S, Io{A, stage, dt}, tu);  // ends with a barrier
    if (stage == 1 && tid == 0) {
      __threadfence();
      atomicAdd(published + s, 1u);
    }
  }
}

// The fused kernel instances: the row sweep plain, with the learned
// indicator, with contact steepening, with both; the plane sweep plain and
// with contact steepening (the indicator runs in the row sweep only).
template <class Body, int NN>
static cudaError_t fused_attr(int* per_sm) {
  cudaError_t e = cudaFuncSetAttribute(hydro_rk3_fused_kernel<Body, NN>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Body::kSmem);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, hydro_rk3_fused_kernel<Body, NN>, Body::kThreads,
                                                      Body::kSmem);
  return e;
}

// Opt in to the dynamic shared memory (once per device); the most CTAs of
// the decomposition's kernels that can be resident at once (the cooperative
// launch's limit).
template <int NN, bool kSpin = false>
static cudaError_t prepare_fused_nn(int num_sms, int planes, int* max_grid) {
  static unsigned long long done = 0;
  static int per_sm_dev[64][2];
  cudaError_t e = once_per_device(&done, [] {
    int dev = 0, p[6] = {0, 0, 0, 0, 0, 0};
    cudaError_t r = cudaGetDevice(&dev);
    if (r == cudaSuccess) r = fused_attr<RowBody<false, false, kSpin>, NN>(&p[0]);
    if (r == cudaSuccess) r = fused_attr<RowBody<true, false, kSpin>, NN>(&p[1]);
    if (r == cudaSuccess) r = fused_attr<RowBody<false, true, kSpin>, NN>(&p[2]);
    if (r == cudaSuccess) r = fused_attr<PlaneBody<false, kSpin>, NN>(&p[3]);
    if (r == cudaSuccess) r = fused_attr<PlaneBody<true, kSpin>, NN>(&p[4]);
    if (r == cudaSuccess) r = fused_attr<RowBody<true, true, kSpin>, NN>(&p[5]);
    if (r != cudaSuccess) return r;
    int rows = p[0] < p[1] ? p[0] : p[1];
    rows = rows < p[2] ? rows : p[2];
    rows = rows < p[5] ? rows : p[5];
    if (rows > 2) rows = 2;
    int pl = p[3] < p[4] ? p[3] : p[4];
    if (pl > 1) pl = 1;
    if (rows < 1 || pl < 1) return cudaErrorInvalidConfiguration;
    per_sm_dev[dev][0] = rows;
    per_sm_dev[dev][1] = pl;
    return cudaSuccess;
  });
  if (e != cudaSuccess) return e;
  int dev = 0;
  e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  *max_grid = per_sm_dev[dev][planes ? 1 : 0] * num_sms;
  return cudaSuccess;
}

template <class Body, int NN>
static cudaError_t launch_fused(const FusedArgs& A, int max_grid, cudaStream_t st) {
  const int units = A.S.n_sub * Tile<NN>::kTiles;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(units < max_grid ? units : max_grid));
  cfg.blockDim = dim3(Body::kThreads);
  cfg.dynamicSmemBytes = Body::kSmem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, hydro_rk3_fused_kernel<Body, NN>, A);
}

// One fused RK3 step of a mesh of NN^3 sub-grids; sync must hold
// rk3_fused_sync_words(n_sub) words, and with 16^3 sub-grids amax is the
// atomic maximum over each sub-grid's tiles: both are cleared here.  prims:
// 2 n_sub F NN^3 floats of scratch for the row sweep's primitives.  planes:
// the plane-sweep body (no learned indicator); otherwise the row sweep.
// kSpin: the instances with the spin feedback (hydro_mode_t.spin), which the
// others carry none of.
template <int NN, bool kSpin = false>
static cudaError_t launch_fused_nn(const StepArgs64& S, double* Y, double* U2, float* prims, double* dt_out,
                                   unsigned* sync, int nbx, int nby, int nbz, int bc, double cfl, double eta2,
                                   double gamma, int num_sms, int planes, cudaStream_t st) {
  int max_grid = 0;
  cudaError_t e = prepare_fused_nn<NN, kSpin>(num_sms, planes, &max_grid);
  if (e != cudaSuccess) return e;
  FusedArgs A;
  A.S = S;
  A.Y = Y;
  A.U2 = U2;
  A.P[0] = prims;
  A.P[1] = prims + (size_t)S.n_sub * F * Tile<NN>::kN3;
  A.dt_out = dt_out;
  A.sync = sync;
  A.nbx = nbx;
  A.nby = nby;
  A.nbz = nbz;
  A.bc = bc;
  A.cfl = cfl;
  A.eta2 = eta2;
  A.inv_gamma = 1.0 / gamma;
  const double alpha[3] = {0.0, 0.75, 1.0 / 3.0}, beta[3] = {1.0, 0.25, 2.0 / 3.0};
  for (int k = 0; k < 3; ++k) {
    A.alpha[k] = alpha[k];
    A.beta[k] = beta[k];
  }
  // a second plus 20 us per tile: far above any stage's duration
  A.wait_ns = 1000000000ll + 20000ll * (long long)S.n_sub * Tile<NN>::kTiles;
  e = cudaMemsetAsync(sync, 0, ((size_t)kSyncHead + 2 * (size_t)S.n_sub) * sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  if (Tile<NN>::kTiles > 1) {
    e = cudaMemsetAsync(S.amax, 0, (size_t)S.n_sub * sizeof(double), st);
    if (e != cudaSuccess) return e;
  }
  if (planes && !S.gate)
    return S.P.contact ? launch_fused<PlaneBody<true, kSpin>, NN>(A, max_grid, st)
                       : launch_fused<PlaneBody<false, kSpin>, NN>(A, max_grid, st);
  if (S.gate && S.P.contact) return launch_fused<RowBody<true, true, kSpin>, NN>(A, max_grid, st);
  if (S.gate) return launch_fused<RowBody<true, false, kSpin>, NN>(A, max_grid, st);
  if (S.P.contact) return launch_fused<RowBody<false, true, kSpin>, NN>(A, max_grid, st);
  return launch_fused<RowBody<false, false, kSpin>, NN>(A, max_grid, st);
}

}  // namespace hyd
