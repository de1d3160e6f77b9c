// hydro_common.cuh -- layout constants and device helpers shared by the
// kernels of the GB300 hydro library (sm_103a).
#pragma once
#include <cstdint>
#include <mutex>

#include <cuda_runtime.h>

namespace hyd {

// Sub-grid geometry (Sec. III-B: 8^3 cells per leaf sub-grid by default; a
// 5-cell PPM stencil on the face-adjacent ghost row needs 3 ghost layers).
constexpr int N = 8;
constexpr int G = 3;
constexpr int S = N + 2 * G;         // 14 stored cells per edge
constexpr int S3 = S * S * S;        // 2744
constexpr int N3 = N * N * N;        // 512
constexpr int F = 10;                // rho, s(3), E, tau, z(3), one species
constexpr int NROW = 3 * N * N;      // 192 rows: 3 axes x 8 x 8 transverse positions

// Field slots of the conserved state and of the reconstructed primitives
// (rho, v(3), eps, tau, z(3), species share the slots).
enum { RHO = 0, SX = 1, SY = 2, SZ = 3, EGAS = 4, TAU = 5, ZX = 6, ZY = 7, ZZ = 8, SP0 = 9 };

// Per-axis scratch of one sub-grid: for each axis a and interior cell the 10
// flux differences Fbar(i+1/2) - Fbar(i-1/2) and the 3 torque differences.
constexpr int DQ = F + 3;
constexpr size_t kScratchPerSub = (size_t)3 * DQ * N3;  // doubles

// Boundary-face export of one sub-grid face (axis a, side): the 10 face-
// averaged fluxes and the 3 torque components about the adjacent interior
// cell, on the N x N face cells indexed [c][b] (b < c the transverse axes).
// Face slot f = 2a for the lower face, 2a + 1 for the upper face.
__device__ __forceinline__ size_t face_index(int s, int f, int q, int pc, int pb) {
  return ((((size_t)s * 6 + f) * DQ + q) * N + pc) * N + pb;
}

// ---- sub-grid layouts and their 8^3 tiles ----------------------------------
// A sub-grid has NN^3 interior cells (NN = 8, the paper's default, or 16)
// and G ghost layers, stored [F][NN+2G]^3.  The step kernels work on 8^3
// tiles: the whole sub-grid (NN = 8), or one of the eight octants of a 16^3
// sub-grid, whose 14^3 window of the padded array -- the octant and its
// G-deep surround of neighbouring octants' interior cells and ghost cells --
// is a padded 8^3 sub-grid in place.  Work unit u = s * kTiles + octant,
// octant = (oz * 2 + oy) * 2 + ox.
template <int NN>
struct Tile {
  static_assert(NN == 8 || NN == 16, "8^3 or 16^3 sub-grids");
  static constexpr int kN = NN, kS = NN + 2 * G, kS3 = kS * kS * kS, kN3 = NN * NN * NN;
  static constexpr int kTiles = (NN / N) * (NN / N) * (NN / N);
  int s;     // the sub-grid
  int o[3];  // the tile's cell offsets in the sub-grid (0, or N for the upper octants)
  __device__ __forceinline__ explicit Tile(int u) {
    s = u / kTiles;
    const int t = u % kTiles;
    o[0] = (t & 1) * N;
    o[1] = ((t >> 1) & 1) * N;
    o[2] = ((t >> 2) & 1) * N;
  }
  // index in the sub-grid's padded array of tile-padded cell (x, y, z) in [0, S)^3
  __device__ __forceinline__ int pad(int x, int y, int z) const {
    return ((z + o[2]) * kS + (y + o[1])) * kS + (x + o[0]);
  }
  __device__ __forceinline__ int pad(int c) const {
    return NN == N ? c : pad(c % S, (c / S) % S, c / (S * S));
  }
  // index in the sub-grid's compact NN^3 array of tile interior cell c (an 8^3 index)
  __device__ __forceinline__ int cell(int c) const {
    return NN == N ? c : (((c / (N * N)) + o[2]) * kN + ((c / N) % N + o[1])) * kN + (c % N + o[0]);
  }
  // whether face slot f (2a: lower, 2a + 1: upper face of axis a) of the tile
  // is a face of the sub-grid
  __device__ __forceinline__ bool outer(int f) const {
    return (f & 1) ? o[f >> 1] + N == kN : o[f >> 1] == 0;
  }
  // index of boundary-face value q of sub-grid face f at the tile's face cell
  // (pc, pb) (b < c the face's transverse axes): [n][6][DQ][NN][NN]
  __device__ __forceinline__ size_t face(int f, int q, int pc, int pb) const {
    const int a = f >> 1, b = a == 0 ? 1 : 0, c = a == 2 ? 1 : 2;
    return ((((size_t)s * 6 + f) * DQ + q) * kN + (pc + o[c])) * kN + (pb + o[b]);
  }
};

// Largest of the non-negative doubles in *p and v, atomically (IEEE order of
// non-negative doubles is the order of their bit patterns): the amax of a
// sub-grid whose tiles run on different CTAs.  The result does not depend on
// the order of the updates.
__device__ __forceinline__ void atomic_max_nonneg(double* p, double v) {
  atomicMax(reinterpret_cast<unsigned long long*>(p), (unsigned long long)__double_as_longlong(v));
}

struct StepParams {
  double gamma, gm1, omega, eta1;
  int face_points;  // 9: Simpson sum of the 9 face points; 1: the face centre only
  int contact;      // 1: PPM contact steepening of the density and species lines
  int spin;         // 1: a cell's spin feeds back into the velocity at its points (spin_dv64)
};

// Arguments of the step kernels (device pointers; layouts as in hydro.h).
struct StepArgs64 {
  const double* U;
  const double* origin;
  const double* h;
  const double* g;
  double* dUdt;
  double* amax;
  double* face_flux;  // optional [n_sub][6][DQ][N][N] boundary-face sums (null: none)
  double* scratch;  // per-CTA scratch, kScratchPerSub doubles per CTA
  double* lines;    // FP64 step with every line once: per-CTA line ends (null for the other kernels)
  unsigned* status;
  int n_sub;
  StepParams P;
  int gate;               // mixed form: use the learned smoothness indicator
  const float* gate_w;    // its BF16-rounded parameters (device, kGateParams floats)
  float gate_logit_thr;   // cells with indicator logit below this are smooth
  int gate_zero_smooth;   // the decision for all-zero features (uniform neighbourhood)
};

// Component i (0 = x, 1 = y, 2 = z) of a vector given by its components va,
// vb, vc along a row sweep's axes a, b, c (a permutation of 0, 1, 2): a
// select, so that no small array is indexed by the runtime axis (which
// would place it in local memory).
template <class T>
__device__ __forceinline__ T axis_comp(int i, int a, int b, T va, T vb, T vc) {
  return i == a ? va : (i == b ? vb : vc);
}
__device__ __forceinline__ int axis_stride(int i) { return i == 0 ? 1 : (i == 1 ? S : S * S); }

// ---- FP64 arithmetic that the compiler may not contract into FMA --------
__device__ __forceinline__ double radd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double rsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double rmul(double a, double b) { return __dmul_rn(a, b); }

// ---- SSP-RK3 stage combination of one cell (Sec. IV-A.2) ----------------
//   u <- alpha U0 + beta (U + dt dU/dt), (alpha, beta) = (0,1), (3/4,1/4), (1/3,2/3)
//   then tau <- eps_E^(1/gamma) where eps_E = E - |s|^2/(2 rho) > eta2 E
//   (tracer resync of the dual-energy formalism, Bryan et al. 1995).
// One definition for every kernel that applies a stage, so that the separate
// update kernel and the fused RK3 step give the same bits.
// FP64 form: explicitly rounded operations (the oracle's values).  Mixed
// form: FMA allowed, 1/rho from an FP32 reciprocal refined by a Newton step,
// the tracer power in FP32 like the rest of the tracer's arithmetic there.
template <bool kMixed>
__device__ __forceinline__ void rk3_cell(const double U[F], const double U0[F], const double R[F], double dt,
                                         double alpha, double beta, double eta2, double inv_gamma, double u[F]) {
#pragma unroll
  for (int k = 0; k < F; ++k) {
    if (kMixed) {
      u[k] = fma(alpha, U0[k], beta * fma(dt, R[k], U[k]));
    } else {
      const double t = radd(U[k], rmul(dt, R[k]));
      u[k] = radd(rmul(alpha, U0[k]), rmul(beta, t));
    }
  }
  const double rho = u[RHO];
  if (kMixed) {
    const double r0 = (double)__frcp_rn((float)rho);
    const double ri = r0 * fma(-rho, r0, 2.0);
    const double s2 = fma(u[SZ], u[SZ], fma(u[SY], u[SY], u[SX] * u[SX]));
    const double eE = u[EGAS] - 0.5 * s2 * ri;
    if (eE > eta2 * u[EGAS]) u[TAU] = (double)__powf((float)eE, (float)inv_gamma);
  } else {
    const double vx = u[SX] / rho, vy = u[SY] / rho, vz = u[SZ] / rho;
    const double ek = rmul(rmul(0.5, rho), radd(radd(rmul(vx, vx), rmul(vy, vy)), rmul(vz, vz)));
    const double eE = rsub(u[EGAS], ek);
    if (eE > rmul(eta2, u[EGAS])) u[TAU] = pow(eE, inv_gamma);
  }
}

// Uniform-mesh boundary map of one global cell coordinate (n cells along the
// axis, |overshoot| <= G < n): periodic wraps, outflow clamps to the nearest
// interior cell (zero gradient).
__device__ __forceinline__ int bc_map(int gpos, int n, int bc) {
  if (bc == 0) return gpos < 0 ? gpos + n : (gpos >= n ? gpos - n : gpos);
  return gpos < 0 ? 0 : (gpos >= n ? n - 1 : gpos);
}

// ---- mbarrier + bulk (TMA) copy, inline PTX -----------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
// Bulk global->shared copy completing on an mbarrier (size and both
// addresses multiples of 16 bytes).
__device__ __forceinline__ void bulk_g2s(void* dst_smem, const void* src_gmem, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst_smem)),
      "l"(src_gmem), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: gives up after max_iter polls (each poll itself suspends for
// a hardware-chosen time) and returns false.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, long max_iter) {
  for (long i = 0; i < max_iter; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// ---- host: once-per-device set-up -------------------------------------
// Function attributes (the dynamic shared-memory opt-in) belong to each
// device's context, so a set-up step runs once per device: bit d of *mask
// records that fn() succeeded with device d current.  Serialised by one
// process-wide mutex.
inline std::mutex& device_setup_mutex() {
  static std::mutex m;
  return m;
}
template <class Fn>
cudaError_t once_per_device(unsigned long long* mask, Fn fn) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(device_setup_mutex());
  if (*mask & (1ull << dev)) return cudaSuccess;
  e = fn();
  if (e == cudaSuccess) *mask |= 1ull << dev;
  return e;
}

}  // namespace hyd
