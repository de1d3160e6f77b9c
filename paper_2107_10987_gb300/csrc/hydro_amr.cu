// hydro_amr.cu -- ghost fill and coarse-fine flux correction on an adaptive
// octree of 8^3 sub-grids (2:1 balanced across faces, edges and vertices).
//
// Leaves are found through dense per-level tables (hydro_amr_t): at level l
// entry ((k 2^l) + j) 2^l + i is the leaf index at that sub-grid position,
// -1 where the position is refined, -2 where it lies inside a coarser leaf.
//
// Ghost fill, two launches: (1) a ghost cell held by a same-level leaf is
// copied, one over a refined position is the mean of its 8 finer cells
// (taken in (dz, dy, dx) order and summed pairwise, ((a0+a1)+(a2+a3)) +
// ((a4+a5)+(a6+a7)), times 1/8, which keeps a uniform state exact); (2) one inside a coarser leaf is
// prolonged from the coarse cell with minmod-limited slopes, conservative
// (offsets -1/4, +1/4 of a coarse cell).  Outside the domain the position is
// clamped (outflow) or wrapped (periodic) first.  The second launch reads
// only cells the first one wrote or interiors (2:1 balance keeps every
// coarse cell and its neighbours used by a prolongation in leaves of the
// same or a finer level).
//
// Flux correction: a coarse boundary cell whose face borders finer leaves
// takes the mean of the 4 fine sub-face fluxes instead of its own, and the
// mean of the fine torques moved to its centre, T(x_C) = T(x_f) + (x_f - x_C)
// x F_s.  Both operations use explicitly rounded arithmetic so that the FP64
// oracle's values are reproduced.
#include "hydro.h"
#include "hydro_common.cuh"
#include "hydro_ctx.h"

namespace hyd {

struct AMRArgs {
  double* U;
  const int* table;
  const int* leaf_level;
  const int* leaf_ijk;
  int lmin, lmax, bc, n_sub;
  unsigned* status;
};

__device__ __forceinline__ long level_offset(int l, int lmin) {
  // sum_{m = lmin}^{l-1} 8^m
  long off = 0;
  for (int m = lmin; m < l; ++m) off += 1L << (3 * m);
  return off;
}

__device__ __forceinline__ int lookup(const AMRArgs& A, int l, int gx, int gy, int gz) {
  if (l < A.lmin || l > A.lmax) return -3;
  const int n = 1 << l;
  return A.table[level_offset(l, A.lmin) + ((long)(gz >> 3) * n + (gy >> 3)) * n + (gx >> 3)];
}

__device__ __forceinline__ int bc_amr(int g, int n, int bc) {
  if (bc == 0) return g < 0 ? g + n : (g >= n ? g - n : g);
  return g < 0 ? 0 : (g >= n ? n - 1 : g);
}

template <int kPass>
__global__ void __launch_bounds__(256) hydro_ghost_amr_kernel(AMRArgs A) {
  for (int s = blockIdx.x; s < A.n_sub; s += gridDim.x) {
    const int l = A.leaf_level[s];
    const int bx = A.leaf_ijk[3 * s] * N, by = A.leaf_ijk[3 * s + 1] * N, bz = A.leaf_ijk[3 * s + 2] * N;
    const int ncell = N << l;
    double* dst = A.U + (size_t)s * F * S3;
    for (int c = threadIdx.x; c < S3; c += blockDim.x) {
      const int lx = c % S - G, ly = (c / S) % S - G, lz = c / (S * S) - G;
      if ((unsigned)lx < (unsigned)N && (unsigned)ly < (unsigned)N && (unsigned)lz < (unsigned)N) continue;
      const int gx = bc_amr(bx + lx, ncell, A.bc), gy = bc_amr(by + ly, ncell, A.bc), gz = bc_amr(bz + lz, ncell, A.bc);
      const int t = lookup(A, l, gx, gy, gz);
      if (kPass == 1) {
        if (t >= 0) {
          const double* src = A.U + (size_t)t * F * S3 + (((gz & 7) + G) * S + ((gy & 7) + G)) * S + ((gx & 7) + G);
#pragma unroll
          for (int k = 0; k < F; ++k) dst[(size_t)k * S3 + c] = src[(size_t)k * S3];
        } else if (t == -1) {
          const double* kid[8];
          bool ok = true;
          for (int d = 0; d < 8; ++d) {
            const int fx = 2 * gx + (d & 1), fy = 2 * gy + ((d >> 1) & 1), fz = 2 * gz + (d >> 2);
            const int tf = lookup(A, l + 1, fx, fy, fz);
            ok &= tf >= 0;
            kid[d] = A.U + (size_t)(tf < 0 ? s : tf) * F * S3 + (((fz & 7) + G) * S + ((fy & 7) + G)) * S +
                     ((fx & 7) + G);
          }
          if (!ok) atomicOr(A.status, 4u);
#pragma unroll
          for (int k = 0; k < F; ++k) {
            const size_t o = (size_t)k * S3;
            const double acc = radd(radd(radd(kid[0][o], kid[1][o]), radd(kid[2][o], kid[3][o])),
                                    radd(radd(kid[4][o], kid[5][o]), radd(kid[6][o], kid[7][o])));
            dst[o + c] = rmul(acc, 0.125);
          }
        }
      } else if (t == -2) {
        const int cx = gx >> 1, cy = gy >> 1, cz = gz >> 1;
        const int tc = lookup(A, l - 1, cx, cy, cz);
        if (tc < 0) {
          atomicOr(A.status, 4u);
          continue;
        }
        const double* C = A.U + (size_t)tc * F * S3 + (((cz & 7) + G) * S + ((cy & 7) + G)) * S + ((cx & 7) + G);
        const double off[3] = {(gx & 1) ? 0.25 : -0.25, (gy & 1) ? 0.25 : -0.25, (gz & 1) ? 0.25 : -0.25};
        const int st[3] = {1, S, S * S};
#pragma unroll
        for (int k = 0; k < F; ++k) {
          const double* q = C + (size_t)k * S3;
          double v = q[0];
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            const double dp = rsub(q[st[d]], q[0]), dm = rsub(q[0], q[-st[d]]);
            const double mm = (rmul(dp, dm) <= 0.0) ? 0.0 : (fabs(dp) < fabs(dm) ? dp : dm);
            v = radd(v, rmul(mm, off[d]));
          }
          dst[(size_t)k * S3 + c] = v;
        }
      }
    }
  }
}

// One thread per interior cell of a leaf; the cell's faces on the leaf
// boundary that border finer leaves are corrected in the order x-, x+, y-, ...
__global__ void __launch_bounds__(256) hydro_flux_correct_kernel(AMRArgs A, const double* h, const double* faces,
                                                                 double* dUdt) {
  for (int s = blockIdx.x; s < A.n_sub; s += gridDim.x) {
    const int l = A.leaf_level[s];
    const int ijk[3] = {A.leaf_ijk[3 * s], A.leaf_ijk[3 * s + 1], A.leaf_ijk[3 * s + 2]};
    const int n = 1 << l;
    const double hc = h[s];
    for (int cell = threadIdx.x; cell < N3; cell += blockDim.x) {
      const int cl[3] = {cell & 7, (cell >> 3) & 7, cell >> 6};
      double du[F];
      bool touched = false;
      for (int a = 0; a < 3; ++a) {
        const int b = (a == 0) ? 1 : 0, c = (a == 2) ? 1 : 2;
        for (int side = 0; side < 2; ++side) {
          if (cl[a] != (side ? N - 1 : 0)) continue;
          int nb[3] = {ijk[0], ijk[1], ijk[2]};
          nb[a] += side ? 1 : -1;
          if (nb[a] < 0 || nb[a] >= n) {
            if (A.bc != 0) continue;
            nb[a] = (nb[a] + n) % n;
          }
          if (lookup(A, l, nb[0] * N, nb[1] * N, nb[2] * N) != -1) continue;
          if (!touched) {
#pragma unroll
            for (int k = 0; k < F; ++k) du[k] = dUdt[((size_t)s * F + k) * N3 + cell];
            touched = true;
          }
          const double sgn = side ? 1.0 : -1.0;
          const int pb = cl[b], pc = cl[c];
          double fsum[F], tsum[3] = {0.0, 0.0, 0.0};
#pragma unroll
          for (int k = 0; k < F; ++k) fsum[k] = 0.0;
          bool ok = true;
          for (int dc = 0; dc < 2; ++dc)
            for (int db = 0; db < 2; ++db) {
              int gf[3];
              gf[a] = side ? (ijk[a] + 1) * 2 * N : ijk[a] * 2 * N - 1;
              gf[b] = 2 * (ijk[b] * N + pb) + db;
              gf[c] = 2 * (ijk[c] * N + pc) + dc;
              const int nf = N << (l + 1);
              if (gf[a] < 0 || gf[a] >= nf) gf[a] = (gf[a] + nf) % nf;  // periodic wrap
              const int o = lookup(A, l + 1, gf[0], gf[1], gf[2]);
              if (o < 0) {
                ok = false;
                continue;
              }
              const int loc[3] = {gf[0] & 7, gf[1] & 7, gf[2] & 7};
              const double* ff = faces + face_index(o, 2 * a + (side ? 0 : 1), 0, loc[c], loc[b]);
              const size_t qs = (size_t)N * N;  // stride between quantities
              double r[3];
              r[a] = rmul(0.75 * sgn, hc);
              r[b] = rmul(db ? 0.25 : -0.25, hc);
              r[c] = rmul(dc ? 0.25 : -0.25, hc);
              const double Fx = ff[SX * qs], Fy = ff[SY * qs], Fz = ff[SZ * qs];
              const double tor[3] = {rsub(rmul(r[1], Fz), rmul(r[2], Fy)), rsub(rmul(r[2], Fx), rmul(r[0], Fz)),
                                     rsub(rmul(r[0], Fy), rmul(r[1], Fx))};
#pragma unroll
              for (int k = 0; k < F; ++k) fsum[k] = radd(fsum[k], ff[k * qs]);
#pragma unroll
              for (int m = 0; m < 3; ++m) tsum[m] = radd(tsum[m], radd(ff[(F + m) * qs], tor[m]));
            }
          if (!ok) {
            atomicOr(A.status, 4u);
            continue;
          }
          const double* own = faces + face_index(s, 2 * a + side, 0, pc, pb);
          const size_t qs = (size_t)N * N;
          const double coef = -(sgn / hc);
          double corr[F];
#pragma unroll
          for (int k = 0; k < F; ++k) corr[k] = rmul(coef, rsub(rmul(fsum[k], 0.25), own[k * qs]));
#pragma unroll
          for (int m = 0; m < 3; ++m)
            corr[ZX + m] = radd(corr[ZX + m], rmul(coef, rsub(rmul(tsum[m], 0.25), own[(F + m) * qs])));
#pragma unroll
          for (int k = 0; k < F; ++k) du[k] = radd(du[k], corr[k]);
        }
      }
      if (touched) {
#pragma unroll
        for (int k = 0; k < F; ++k) dUdt[((size_t)s * F + k) * N3 + cell] = du[k];
      }
    }
  }
}

}  // namespace hyd

static hyd::AMRArgs amr_args(hydro_ctx_t* c, const hydro_batch_t* B, const hydro_amr_t* M) {
  hyd::AMRArgs A;
  A.U = B->U;
  A.table = M->table;
  A.leaf_level = M->leaf_level;
  A.leaf_ijk = M->leaf_ijk;
  A.lmin = M->lmin;
  A.lmax = M->lmax;
  A.bc = M->bc;
  A.n_sub = B->n_sub;
  A.status = c->status;
  return A;
}

static bool amr_ok(const hydro_amr_t* M) {
  return M && M->table && M->leaf_level && M->leaf_ijk && M->lmin >= 0 && M->lmax >= M->lmin && M->lmax <= 10 &&
         (M->bc == HYDRO_BC_PERIODIC || M->bc == HYDRO_BC_OUTFLOW);
}

int hydro_ctx_prepare(hydro_ctx* c, int n_sub);

extern "C" {

int hydro_fill_ghosts_amr(hydro_ctx_t* c, const hydro_batch_t* B, const hydro_amr_t* M, void* stream) {
  if (!c || !B || B->n_sub < 0 || !amr_ok(M)) return HYDRO_EINVAL;
  if (B->n_sub == 0) return HYDRO_OK;
  if (!B->U) return HYDRO_EINVAL;
  int rc = hydro_ctx_prepare(c, 0);
  if (rc) return rc;
  hyd::AMRArgs A = amr_args(c, B, M);
  const int cap = c->num_sms * 8;
  const int grid = B->n_sub < cap ? B->n_sub : cap;
  cudaStream_t st = (cudaStream_t)stream;
  hyd::hydro_ghost_amr_kernel<1><<<grid, 256, 0, st>>>(A);
  hyd::hydro_ghost_amr_kernel<2><<<grid, 256, 0, st>>>(A);
  return cudaGetLastError() == cudaSuccess ? HYDRO_OK : HYDRO_ECUDA;
}

int hydro_flux_correct_amr(hydro_ctx_t* c, const hydro_batch_t* B, const hydro_amr_t* M, const double* face_flux,
                           double* dUdt, void* stream) {
  if (!c || !B || B->n_sub < 0 || !amr_ok(M)) return HYDRO_EINVAL;
  if (B->n_sub == 0) return HYDRO_OK;
  if (!B->h || !face_flux || !dUdt) return HYDRO_EINVAL;
  int rc = hydro_ctx_prepare(c, 0);
  if (rc) return rc;
  hyd::AMRArgs A = amr_args(c, B, M);
  const int cap = c->num_sms * 8;
  const int grid = B->n_sub < cap ? B->n_sub : cap;
  hyd::hydro_flux_correct_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(A, B->h, face_flux, dUdt);
  return cudaGetLastError() == cudaSuccess ? HYDRO_OK : HYDRO_ECUDA;
}

}  // extern "C"
