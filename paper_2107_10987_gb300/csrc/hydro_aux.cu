// hydro_aux.cu -- the kernels around the step: SSP-RK3 stage update with the
// dual-energy tracer resync, CFL time step, uniform-mesh ghost fill and the
// global conservation sums.
#include "hydro_common.cuh"

namespace hyd {

// ---------------------------------------------------------------------------
// RK3 stage update (three hydro iterations per time step, Sec. IV-A.2) of
// the interior cells: the stage combination and tracer resync of rk3_cell,
// FP64 or mixed form.  Out of place when Uout != U (the interior of Uout is
// written, U untouched).
struct UpdateArgs {
  const double* U;
  double* Uout;
  const double* U0;
  const double* dUdt;
  const double* dt_dev;
  double dt;
  double alpha, beta, eta2, inv_gamma;
  int n_sub;
};

// NN: the sub-grids' edge (8 or 16).
template <bool kMixed, int NN>
__global__ void __launch_bounds__(256) hydro_update_kernel(UpdateArgs A) {
  constexpr int LS = NN + 2 * G, LS3 = LS * LS * LS, LN3 = NN * NN * NN;
  const double dt = A.dt_dev ? *A.dt_dev : A.dt;
  for (int s = blockIdx.x; s < A.n_sub; s += gridDim.x) {
    const size_t ub = (size_t)s * F * LS3, db = (size_t)s * F * LN3;
    for (int c = threadIdx.x; c < LN3; c += blockDim.x) {
      const int x = c % NN, y = (c / NN) % NN, z = c / (NN * NN);
      const size_t uc = ub + ((z + G) * LS + (y + G)) * LS + (x + G);
      const size_t dc = db + c;
      double U[F], U0[F], R[F], u[F];
#pragma unroll
      for (int k = 0; k < F; ++k) {
        U[k] = A.U[uc + (size_t)k * LS3];
        U0[k] = A.U0[uc + (size_t)k * LS3];
        R[k] = A.dUdt[dc + (size_t)k * LN3];
      }
      rk3_cell<kMixed>(U, U0, R, dt, A.alpha, A.beta, A.eta2, A.inv_gamma, u);
#pragma unroll
      for (int k = 0; k < F; ++k) A.Uout[uc + (size_t)k * LS3] = u[k];
    }
  }
}

cudaError_t launch_update(const double* U, double* Uout, const double* U0, const double* dUdt, double dt,
                          const double* dt_dev, int stage, double eta2, double gamma, int n_sub, bool mixed,
                          int num_sms, int nn, cudaStream_t st) {
  static const double alpha[3] = {0.0, 0.75, 1.0 / 3.0};
  static const double beta[3] = {1.0, 0.25, 2.0 / 3.0};
  UpdateArgs A{U, Uout, U0, dUdt, dt_dev, dt, alpha[stage], beta[stage], eta2, 1.0 / gamma, n_sub};
  const int cap = num_sms * 8;
  const int blocks = n_sub < cap ? n_sub : cap;
  if (nn == 16) {
    if (mixed)
      hydro_update_kernel<true, 16><<<blocks, 256, 0, st>>>(A);
    else
      hydro_update_kernel<false, 16><<<blocks, 256, 0, st>>>(A);
  } else {
    if (mixed)
      hydro_update_kernel<true, 8><<<blocks, 256, 0, st>>>(A);
    else
      hydro_update_kernel<false, 8><<<blocks, 256, 0, st>>>(A);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// CFL time step: dt = cfl * min_s h[s] / amax[s], one block, fixed order.
__global__ void __launch_bounds__(1024) hydro_dt_kernel(const double* amax, const double* h, int n, double cfl,
                                                       double* out) {
  __shared__ double red[32];
  double m = INFINITY;
  for (int i = threadIdx.x; i < n; i += blockDim.x) m = fmin(m, h[i] / amax[i]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmin(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : INFINITY;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmin(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) *out = cfl * m;
  }
}

cudaError_t launch_dt(const double* amax, const double* h, int n, double cfl, double* out, cudaStream_t st) {
  hydro_dt_kernel<<<1, 1024, 0, st>>>(amax, h, n, cfl, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Uniform-mesh ghost fill: a ghost cell copies the cell at the same global
// position; outside the domain the position wraps (periodic) or is clamped
// to the nearest interior cell (outflow, zero gradient).  One block per
// sub-grid, one thread per ghost cell (all ten fields).
struct GhostArgs {
  double* U;
  int nbx, nby, nbz, bc, n_sub;
};


// The kernel reads only interior cells and writes only ghost cells, so the
// two sets never overlap: all loads of a batch of cells are issued before
// their stores (through the read-only path), instead of one dependent
// load-store pair per field.
constexpr int kGhostBatch = 2;

template <int NN>
__global__ void __launch_bounds__(256) hydro_ghost_uniform_kernel(GhostArgs A) {
  constexpr int LS = NN + 2 * G, LS3 = LS * LS * LS;
  const int nx = A.nbx * NN, ny = A.nby * NN, nz = A.nbz * NN;
  for (int s = blockIdx.x; s < A.n_sub; s += gridDim.x) {
    const int kx = s % A.nbx, ky = (s / A.nbx) % A.nby, kz = s / (A.nbx * A.nby);
    double* dst = A.U + (size_t)s * F * LS3;
    for (int c0 = threadIdx.x; c0 < LS3; c0 += kGhostBatch * blockDim.x) {
      double v[kGhostBatch][F];
      bool ghost[kGhostBatch];
#pragma unroll
      for (int j = 0; j < kGhostBatch; ++j) {
        const int c = c0 + j * blockDim.x;
        const int lx = c % LS - G, ly = (c / LS) % LS - G, lz = c / (LS * LS) - G;
        ghost[j] =
            c < LS3 && !((unsigned)lx < (unsigned)NN && (unsigned)ly < (unsigned)NN && (unsigned)lz < (unsigned)NN);
        if (ghost[j]) {
          const int gx = bc_map(kx * NN + lx, nx, A.bc), gy = bc_map(ky * NN + ly, ny, A.bc);
          const int gz = bc_map(kz * NN + lz, nz, A.bc);
          const int os = ((gz / NN) * A.nby + (gy / NN)) * A.nbx + (gx / NN);
          const int oc = (((gz % NN) + G) * LS + ((gy % NN) + G)) * LS + ((gx % NN) + G);
          const double* src = A.U + (size_t)os * F * LS3 + oc;
#pragma unroll
          for (int k = 0; k < F; ++k) v[j][k] = __ldg(src + (size_t)k * LS3);
        }
      }
#pragma unroll
      for (int j = 0; j < kGhostBatch; ++j)
        if (ghost[j])
#pragma unroll
          for (int k = 0; k < F; ++k) dst[(size_t)k * LS3 + c0 + j * blockDim.x] = v[j][k];
    }
  }
}

// ---------------------------------------------------------------------------
// Interior copies between the compact layout [n_sub][F][N][N][N] and the
// ghost-padded state: one thread per two neighbouring cells along x (one
// 16-byte access on the compact side).
template <bool kScatter, int NN>
__global__ void __launch_bounds__(256) hydro_interior_kernel(double* U, double* I, long long pairs) {
  constexpr int LS = NN + 2 * G, LS3 = LS * LS * LS, LN3 = NN * NN * NN;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < pairs;
       i += (long long)gridDim.x * blockDim.x) {
    const long long e = 2 * i;  // compact element index, x even
    const int c = (int)(e % LN3);
    const long long sk = e / LN3;  // s * F + field
    const int x = c % NN, y = (c / NN) % NN, z = c / (NN * NN);
    double* u = U + sk * LS3 + ((z + G) * LS + (y + G)) * LS + (x + G);
    double2* q = reinterpret_cast<double2*>(I + e);
    if (kScatter) {
      const double2 v = *q;
      u[0] = v.x;
      u[1] = v.y;
    } else {
      *q = make_double2(u[0], u[1]);
    }
  }
}

cudaError_t launch_interior(double* U, double* I, int n_sub, bool scatter, int num_sms, int nn, cudaStream_t st) {
  const long long pairs = (long long)n_sub * F * nn * nn * nn / 2;
  const long long want = (pairs + 255) / 256;
  const int blocks = (int)(want < (long long)num_sms * 16 ? want : (long long)num_sms * 16);
  if (nn == 16) {
    if (scatter)
      hydro_interior_kernel<true, 16><<<blocks, 256, 0, st>>>(U, I, pairs);
    else
      hydro_interior_kernel<false, 16><<<blocks, 256, 0, st>>>(U, I, pairs);
  } else {
    if (scatter)
      hydro_interior_kernel<true, 8><<<blocks, 256, 0, st>>>(U, I, pairs);
    else
      hydro_interior_kernel<false, 8><<<blocks, 256, 0, st>>>(U, I, pairs);
  }
  return cudaGetLastError();
}

cudaError_t launch_ghost_uniform(double* U, int nbx, int nby, int nbz, int bc, int num_sms, int nn,
                                 cudaStream_t st) {
  const int n_sub = nbx * nby * nbz;
  GhostArgs A{U, nbx, nby, nbz, bc, n_sub};
  const int cap = num_sms * 8;
  if (nn == 16)
    hydro_ghost_uniform_kernel<16><<<n_sub < cap ? n_sub : cap, 256, 0, st>>>(A);
  else
    hydro_ghost_uniform_kernel<8><<<n_sub < cap ? n_sub : cap, 256, 0, st>>>(A);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Conservation sums: per sub-grid partials (one block each, fixed tree), then
// one block over the partials in a fixed order.
constexpr int NSUM = F + 1;

template <int NN>
__global__ void __launch_bounds__(256) hydro_sums_partial_kernel(const double* U, const double* origin,
                                                                 const double* h, int n_sub, double* part) {
  constexpr int LS = NN + 2 * G, LS3 = LS * LS * LS, LN3 = NN * NN * NN;
  __shared__ double red[NSUM][256];
  const int s = blockIdx.x;
  if (s >= n_sub) return;
  const double hs = h[s];
  const double vol = hs * hs * hs;
  double acc[NSUM];
#pragma unroll
  for (int k = 0; k < NSUM; ++k) acc[k] = 0.0;
  for (int c = threadIdx.x; c < LN3; c += blockDim.x) {
    const int x = c % NN, y = (c / NN) % NN, z = c / (NN * NN);
    const long uc = (size_t)s * F * LS3 + ((z + G) * LS + (y + G)) * LS + (x + G);
#pragma unroll
    for (int k = 0; k < F; ++k) acc[k] += U[uc + (long)k * LS3];
    const double xc = origin[3 * s] + (x + 0.5) * hs, yc = origin[3 * s + 1] + (y + 0.5) * hs;
    acc[F] += (xc * U[uc + SY * LS3] - yc * U[uc + SX * LS3]) + U[uc + ZZ * LS3];
  }
#pragma unroll
  for (int k = 0; k < NSUM; ++k) red[k][threadIdx.x] = acc[k];
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
#pragma unroll
      for (int k = 0; k < NSUM; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < NSUM) part[(size_t)s * NSUM + threadIdx.x] = red[threadIdx.x][0] * vol;
}

__global__ void __launch_bounds__(256) hydro_sums_final_kernel(const double* part, int n_sub, double* sums) {
  __shared__ double red[NSUM][256];
  double acc[NSUM];
#pragma unroll
  for (int k = 0; k < NSUM; ++k) acc[k] = 0.0;
  for (int s = threadIdx.x; s < n_sub; s += blockDim.x)
#pragma unroll
    for (int k = 0; k < NSUM; ++k) acc[k] += part[(size_t)s * NSUM + k];
#pragma unroll
  for (int k = 0; k < NSUM; ++k) red[k][threadIdx.x] = acc[k];
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
#pragma unroll
      for (int k = 0; k < NSUM; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < NSUM) sums[threadIdx.x] = red[threadIdx.x][0];
}

cudaError_t launch_sums(const double* U, const double* origin, const double* h, int n_sub, double* part,
                        double* sums, int nn, cudaStream_t st) {
  if (nn == 16)
    hydro_sums_partial_kernel<16><<<n_sub, 256, 0, st>>>(U, origin, h, n_sub, part);
  else
    hydro_sums_partial_kernel<8><<<n_sub, 256, 0, st>>>(U, origin, h, n_sub, part);
  hydro_sums_final_kernel<<<1, 256, 0, st>>>(part, n_sub, sums);
  return cudaGetLastError();
}

}  // namespace hyd
