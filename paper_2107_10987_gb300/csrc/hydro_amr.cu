// hydro_amr.cu -- ghost fill and coarse-fine flux correction on an adaptive
// octree of NN^3 sub-grids, NN = 8 or 16 (2:1 balanced across faces, edges
// and vertices).
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
#include "hydro_amr.cuh"
#include "hydro_ctx.h"

namespace hyd {

// Boundary-face value [s][f][q][pc][pb] of leaves of NN^3 cells.
template <int NN>
__device__ __forceinline__ size_t face_index_nn(int s, int f, int q, int pc, int pb) {
  return ((((size_t)s * 6 + f) * DQ + q) * NN + pc) * NN + pb;
}

// Position of a ghost cell's sub-grid relative to a base position, after the
// boundary map: in lo..lo+span-1 (periodic wrap-around mapped back).
__device__ __forceinline__ int rel_pos(int p, int base, int n, int bc, int lo, int span) {
  int r = p - base;
  if (bc == 0) {
    if (r > lo + span - 1) r -= n;
    else if (r < lo) r += n;
  }
  return r;
}

// Pass 1: same-level copies and restrictions.  A leaf's ghost cells (G < N)
// lie in the 26 positions around it at its level, and the finer cells of a
// restricted ghost cell in the 4^3 positions 2p-1 .. 2p+2 one level down: the
// table entries of both sets are read once per leaf into shared memory.
// Pass 1 reads interior cells only and writes ghost cells only, so each
// thread takes four ghost cells at a time and issues all their loads (read-
// only path) before their stores.
constexpr int kAmrBatch = 4;

template <int NN>
__global__ void __launch_bounds__(256) hydro_ghost_amr_kernel(AMRArgs A) {
  constexpr int LS = NN + 2 * G, LS3 = LS * LS * LS, LN3 = NN * NN * NN, LM = NN - 1, LSH = NN == 8 ? 3 : 4;
  __shared__ int nb[27];   // level l:   relative position (-1..1)^3
  __shared__ int nbf[64];  // level l+1: relative position (-1..2)^3 from 2p
  const int tid = threadIdx.x;
  for (int u = blockIdx.x; u < A.n_sub; u += gridDim.x) {
    const int s = leaf_at(A, u);
    if (s < 0) continue;
    const int l = A.leaf_level[s];
    const int pi[3] = {A.leaf_ijk[3 * s], A.leaf_ijk[3 * s + 1], A.leaf_ijk[3 * s + 2]};
    const int n = 1 << l, ncell = NN << l;
    __syncthreads();  // the previous leaf's tables are no longer read
    if (tid < 27) {
      const int q[3] = {pi[0] + tid % 3 - 1, pi[1] + (tid / 3) % 3 - 1, pi[2] + tid / 9 - 1};
      int w[3];
      bool inside = true;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        w[d] = (A.bc == 0) ? (q[d] + n) % n : q[d];
        inside &= (w[d] >= 0 && w[d] < n);
      }
      nb[tid] = inside ? A.table[level_offset(l, A.lmin) + ((long)w[2] * n + w[1]) * n + w[0]] : -3;
    } else if (tid >= 64 && tid < 128) {
      const int i = tid - 64, nf = 2 * n;
      const int q[3] = {2 * pi[0] + i % 4 - 1, 2 * pi[1] + (i / 4) % 4 - 1, 2 * pi[2] + i / 16 - 1};
      int w[3];
      bool inside = l < A.lmax;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        w[d] = (A.bc == 0) ? (q[d] + nf) % nf : q[d];
        inside &= (w[d] >= 0 && w[d] < nf);
      }
      nbf[i] = inside ? A.table[level_offset(l + 1, A.lmin) + ((long)w[2] * nf + w[1]) * nf + w[0]] : -3;
    }
    __syncthreads();
    double* dst = A.U + (size_t)s * F * LS3;
    for (int c0 = tid; c0 < LS3; c0 += kAmrBatch * blockDim.x) {
      double v[kAmrBatch][F];
      bool put[kAmrBatch];
#pragma unroll
      for (int j = 0; j < kAmrBatch; ++j) {
        const int c = c0 + j * blockDim.x;
        const int lx = c % LS - G, ly = (c / LS) % LS - G, lz = c / (LS * LS) - G;
        put[j] = c < LS3 && !((unsigned)lx < (unsigned)NN && (unsigned)ly < (unsigned)NN && (unsigned)lz < (unsigned)NN);
        if (!put[j]) continue;
        const int g[3] = {bc_amr(pi[0] * NN + lx, ncell, A.bc), bc_amr(pi[1] * NN + ly, ncell, A.bc),
                          bc_amr(pi[2] * NN + lz, ncell, A.bc)};
        const int r[3] = {rel_pos(g[0] >> LSH, pi[0], n, A.bc, -1, 3), rel_pos(g[1] >> LSH, pi[1], n, A.bc, -1, 3),
                          rel_pos(g[2] >> LSH, pi[2], n, A.bc, -1, 3)};
        const int t = nb[((r[2] + 1) * 3 + (r[1] + 1)) * 3 + (r[0] + 1)];
        if (t >= 0) {
          const double* src =
              A.U + (size_t)t * F * LS3 + (((g[2] & LM) + G) * LS + ((g[1] & LM) + G)) * LS + ((g[0] & LM) + G);
#pragma unroll
          for (int k = 0; k < F; ++k) v[j][k] = __ldg(src + (size_t)k * LS3);
        } else if (t == -1) {
          const double* kid[8];
          bool ok = true;
#pragma unroll
          for (int d = 0; d < 8; ++d) {
            const int f[3] = {2 * g[0] + (d & 1), 2 * g[1] + ((d >> 1) & 1), 2 * g[2] + (d >> 2)};
            const int rf[3] = {rel_pos(f[0] >> LSH, 2 * pi[0], 2 * n, A.bc, -1, 4),
                               rel_pos(f[1] >> LSH, 2 * pi[1], 2 * n, A.bc, -1, 4),
                               rel_pos(f[2] >> LSH, 2 * pi[2], 2 * n, A.bc, -1, 4)};
            const int tf = nbf[((rf[2] + 1) * 4 + (rf[1] + 1)) * 4 + (rf[0] + 1)];
            ok &= tf >= 0;
            kid[d] = A.U + (size_t)(tf < 0 ? s : tf) * F * LS3 + (((f[2] & LM) + G) * LS + ((f[1] & LM) + G)) * LS +
                     ((f[0] & LM) + G);
          }
          if (!ok) atomicOr(A.status, 4u);
#pragma unroll
          for (int k = 0; k < F; ++k) {
            const size_t o = (size_t)k * LS3;
            const double acc = radd(radd(radd(__ldg(kid[0] + o), __ldg(kid[1] + o)), radd(__ldg(kid[2] + o), __ldg(kid[3] + o))),
                                    radd(radd(__ldg(kid[4] + o), __ldg(kid[5] + o)), radd(__ldg(kid[6] + o), __ldg(kid[7] + o))));
            v[j][k] = rmul(acc, 0.125);
          }
        } else {
          put[j] = false;  // inside a coarser leaf: pass 2
        }
      }
#pragma unroll
      for (int j = 0; j < kAmrBatch; ++j)
        if (put[j])
#pragma unroll
          for (int k = 0; k < F; ++k) dst[(size_t)k * LS3 + c0 + j * blockDim.x] = v[j][k];
    }
  }
}

// minmod(dp, dm) = 0 if dp dm <= 0, else the one of smaller magnitude: the
// FP64 product's sign and the magnitudes compared on their bit patterns
// (exact equivalents of the FP64 comparisons; GB300 issues FP64 at 1/64 of
// the FP32 rate).
__device__ __forceinline__ double minmod64(double dp, double dm) {
  const long long bp = __double_as_longlong(dp), bm = __double_as_longlong(dm);
  const long long a = bp & 0x7fffffffffffffffLL, b = bm & 0x7fffffffffffffffLL;
  // dp dm <= 0 when either is zero or the signs differ; with equal signs the
  // product is positive unless it underflows to zero, which needs an operand
  // below the normal range or |dp| |dm| < 2^-1074, i.e. biased exponents
  // summing below 972: only then is the FP64 product itself consulted.
  if (a == 0 || b == 0 || (bp ^ bm) < 0) return 0.0;
  const int ep = (int)(a >> 52), em = (int)(b >> 52);
  if ((ep == 0 || em == 0 || ep + em < 972) && __double_as_longlong(rmul(dp, dm)) <= 0LL) return 0.0;
  return a < b ? dp : dm;
}

// x * 0.25 exactly: a normal x whose quarter is still normal has its
// exponent lowered by two; zeros, denormal results, inf and NaN take the
// FP64 product.
__device__ __forceinline__ double quarter64(double x) {
  const long long bx = __double_as_longlong(x);
  const int e = (int)((bx >> 52) & 0x7ff);
  if (e > 2 && e < 0x7ff) return __longlong_as_double(bx - (2LL << 52));
  return rmul(x, 0.25);
}

// The six face neighbours of coarse cell C (global cell Cw of level lc, Cp
// its padded pointer in its leaf), minus and plus along x, y, z: pointer to
// field 0 and field stride.  Without kDirect every neighbour is read from
// the coarse leaf's padded array, whose ghost cells the first pass filled;
// with kDirect a neighbour outside the coarse leaf's interior is read where
// it lives (amr_source: a same-level leaf's interior or a finer leaf's
// restriction image), which are the values the first pass would copy there.
template <int NN, bool kDirect>
__device__ __forceinline__ void coarse_stencil(const AMRArgs& A, LevelRef Lc, LevelRef Lcf, const int Cw[3],
                                               const double* Cp, const double* nbp[6], int nbs[6]) {
  constexpr int LS = NN + 2 * G, LS3 = LS * LS * LS, LM = NN - 1;
  const int st[3] = {1, LS, LS * LS};
#pragma unroll
  for (int d = 0; d < 3; ++d)
#pragma unroll
    for (int sg = 0; sg < 2; ++sg) {
      const int j = 2 * d + sg, step = sg ? 1 : -1;
      nbp[j] = Cp + step * st[d];
      nbs[j] = LS3;
      if (kDirect) {
        const int loc = (Cw[d] & LM) + step;
        if (loc < 0 || loc > LM) {
          int g[3] = {Cw[0], Cw[1], Cw[2]};
          g[d] = bc_amr(Cw[d] + step, NN * Lc.n, A.bc);
          size_t sd;
          const double* p = amr_source<NN>(A, Lc, Lcf, g[0], g[1], g[2], sd);
          if (p) {
            nbp[j] = p;
            nbs[j] = (int)sd;
          }
        }
      }
    }
}

// Prolongation of one fine ghost cell from coarse cell C (padded pointer to
// field 0, face neighbours from coarse_stencil): U_C + s_x o_x + s_y o_y +
// s_z o_z, all ten fields.
template <int NN>
__device__ __forceinline__ void prolong_cell(const double* C, const double* const nbp[6], const int nbs[6],
                                             const double off[3], double* dst) {
  constexpr int LS = NN + 2 * G, LS3 = LS * LS * LS;
#pragma unroll
  for (int k = 0; k < F; ++k) {
    const double c = C[(size_t)k * LS3];
    double v = c;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const double dp = rsub(nbp[2 * d + 1][(size_t)k * nbs[2 * d + 1]], c);
      const double dm = rsub(c, nbp[2 * d][(size_t)k * nbs[2 * d]]);
      v = radd(v, rmul(minmod64(dp, dm), off[d]));
    }
    dst[(size_t)k * LS3] = v;
  }
}

// Pass 2: ghost cells inside coarser leaves.  One thread per coarse cell of
// the 8^3 coarse block covering the leaf's padded region computes the ten
// fields' minmod slopes once and writes every child that is one of the
// leaf's ghost cells (the same values as prolonging child by child).  Ghost
// cells outside the domain (outflow: clamped positions) are prolonged one by
// one afterwards.  kDirect: the coarse cells' neighbours are read where they
// live (coarse_stencil), so that the first pass need not run.
template <int NN, bool kDirect>
__global__ void __launch_bounds__(256) hydro_ghost_amr_prolong_kernel(AMRArgs A) {
  constexpr int LS = NN + 2 * G, LS3 = LS * LS * LS, LM = NN - 1;
  // the coarse block covering the leaf's padded region: NN/2 + 4 cells an axis
  constexpr int LB = NN / 2 + 4;
  __shared__ int coarser;  // some neighbour position of the leaf lies inside a coarser leaf
  // the coarse cells of the block that have children to prolong (block index,
  // coarse leaf), gathered first so that each warp's lanes all have work
  __shared__ int nwork;
  __shared__ int2 work[LB * LB * LB];
  for (int u = blockIdx.x; u < A.n_sub; u += gridDim.x) {
    const int s = leaf_at(A, u);
    if (s < 0) continue;
    const int l = A.leaf_level[s];
    if (l <= A.lmin) continue;  // no coarser leaves
    // Every ghost cell of the leaf lies, after the boundary map, in one of
    // the 27 positions around it at its level; a leaf none of whose positions
    // is inside a coarser leaf (most of them) has nothing to prolong.
    __syncthreads();  // the previous leaf's flag and work list are no longer read
    if (threadIdx.x == 0) {
      coarser = 0;
      nwork = 0;
    }
    __syncthreads();
    if (threadIdx.x < 27) {
      const int n = 1 << l, t = threadIdx.x;
      const int q[3] = {A.leaf_ijk[3 * s] + t % 3 - 1, A.leaf_ijk[3 * s + 1] + (t / 3) % 3 - 1,
                        A.leaf_ijk[3 * s + 2] + t / 9 - 1};
      int w[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) w[d] = bc_amr(q[d], n, A.bc);
      if (A.table[level_offset(l, A.lmin) + ((long)w[2] * n + w[1]) * n + w[0]] == -2) coarser = 1;
    }
    __syncthreads();
    if (!coarser) continue;
    const int b[3] = {A.leaf_ijk[3 * s] * NN, A.leaf_ijk[3 * s + 1] * NN, A.leaf_ijk[3 * s + 2] * NN};
    const int ncell = NN << l, nc = ncell >> 1;
    const LevelRef Lc = level_ref(A, l - 1), Lcf = level_ref(A, l);  // the coarse level and this one
    double* dstb = A.U + (size_t)s * F * LS3;
    // coarse cell i of the block: its global cell C (Cw after the boundary
    // map) and the mask of its children that are ghost cells of this leaf
    // (padded range, not interior); 0 outside the domain (outflow)
    auto coarse_cell = [&](int i, int C[3], int Cw[3]) {
      const int ii[3] = {i % LB, (i / LB) % LB, i / (LB * LB)};
      bool out = false;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        C[d] = (b[d] >> 1) - 2 + ii[d];
        Cw[d] = C[d];
        if (C[d] < 0 || C[d] >= nc) {
          if (A.bc == 0) Cw[d] = C[d] < 0 ? C[d] + nc : C[d] - nc;
          else out = true;
        }
      }
      int mask = 0;
#pragma unroll
      for (int dch = 0; dch < 8; ++dch) {
        const int f[3] = {2 * C[0] + (dch & 1) - b[0], 2 * C[1] + ((dch >> 1) & 1) - b[1], 2 * C[2] + (dch >> 2) - b[2]};
        const bool in = f[0] >= -G && f[0] < NN + G && f[1] >= -G && f[1] < NN + G && f[2] >= -G && f[2] < NN + G;
        const bool interior = (unsigned)f[0] < (unsigned)NN && (unsigned)f[1] < (unsigned)NN && (unsigned)f[2] < (unsigned)NN;
        if (in && !interior) mask |= 1 << dch;
      }
      return out ? 0 : mask;
    };
    for (int i = threadIdx.x; i < LB * LB * LB; i += blockDim.x) {
      int C[3], Cw[3];
      if (!coarse_cell(i, C, Cw)) continue;
      const int tc = lookup_at<NN>(A, Lc, Cw[0], Cw[1], Cw[2]);
      if (tc == -2) atomicOr(A.status, 4u);  // two levels coarser: not 2:1 balanced
      if (tc < 0) continue;                  // refined at level l-1: held at this level or finer
      work[atomicAdd(&nwork, 1)] = make_int2(i, tc);
    }
    __syncthreads();
    const int nw = nwork;
    for (int j = threadIdx.x; j < nw; j += blockDim.x) {
      const int2 wk = work[j];
      const int tc = wk.y;
      int C[3], Cw[3];
      const int mask = coarse_cell(wk.x, C, Cw);
      const double* Cp =
          A.U + (size_t)tc * F * LS3 + (((Cw[2] & LM) + G) * LS + ((Cw[1] & LM) + G)) * LS + ((Cw[0] & LM) + G);
      const double* nbp[6];
      int nbs[6];
      coarse_stencil<NN, kDirect>(A, Lc, Lcf, Cw, Cp, nbp, nbs);
      // per field: the quarter slopes t_d = s_d / 4 once (the child offsets are
      // +-1/4, and -(s/4) = s * (-1/4) exactly), then the children's values
      // ((c +- t_x) +- t_y) +- t_z as a tree of partial sums -- the same
      // additions, in the same order, as prolonging child by child
      const int need_x = ((mask & 0x55) ? 1 : 0) | ((mask & 0xaa) ? 2 : 0);  // children with x offset -, +
      double* dst0 = dstb + ((2 * C[2] - b[2] + G) * LS + (2 * C[1] - b[1] + G)) * LS + (2 * C[0] - b[0] + G);
#pragma unroll 1
      for (int k = 0; k < F; ++k) {
        const double c = Cp[(size_t)k * LS3];
        double qp[3], qm[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          qp[d] = nbp[2 * d + 1][(size_t)k * nbs[2 * d + 1]];
          qm[d] = nbp[2 * d][(size_t)k * nbs[2 * d]];
        }
        // A coarse cell whose six neighbours have its bits (finite, not -0:
        // a uniform region) has the slopes c - c = +0, and every child is
        // ((c -+ 0) -+ 0) -+ 0 = c exactly: stored without the FP64 work.
        const long long cb = __double_as_longlong(c);
        bool flat = ((cb >> 52) & 0x7ff) != 0x7ff && cb != (long long)0x8000000000000000ULL;
#pragma unroll
        for (int d = 0; d < 3; ++d)
          flat = flat && __double_as_longlong(qp[d]) == cb && __double_as_longlong(qm[d]) == cb;
        if (flat) {
#pragma unroll
          for (int dch = 0; dch < 8; ++dch)
            if (mask & (1 << dch))
              dst0[(size_t)k * LS3 + ((dch >> 2) * LS + ((dch >> 1) & 1)) * LS + (dch & 1)] = c;
          continue;
        }
        double t[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) t[d] = quarter64(minmod64(rsub(qp[d], c), rsub(c, qm[d])));
        double vx[2];
        if (need_x & 1) vx[0] = radd(c, -t[0]);
        if (need_x & 2) vx[1] = radd(c, t[0]);
#pragma unroll
        for (int iy = 0; iy < 2; ++iy) {
          if (!(mask & (0x33 << (2 * iy)))) continue;  // children 2iy, 2iy+1, 2iy+4, 2iy+5
#pragma unroll
          for (int ix = 0; ix < 2; ++ix) {
            const int m2 = (1 << (ix + 2 * iy)) | (1 << (ix + 2 * iy + 4));  // the two children below/above in z
            if (!(mask & m2)) continue;
            const double vxy = radd(vx[ix], iy ? t[1] : -t[1]);
#pragma unroll
            for (int iz = 0; iz < 2; ++iz) {
              const int dch = ix + 2 * iy + 4 * iz;
              if (!(mask & (1 << dch))) continue;
              dst0[(size_t)k * LS3 + (iz * LS + iy) * LS + ix] = radd(vxy, iz ? t[2] : -t[2]);
            }
          }
        }
      }
    }
    if (A.bc == 0) continue;
    // outflow: ghost cells outside the domain, clamped, one by one
    for (int c = threadIdx.x; c < LS3; c += blockDim.x) {
      const int lx = c % LS - G, ly = (c / LS) % LS - G, lz = c / (LS * LS) - G;
      const int gx = b[0] + lx, gy = b[1] + ly, gz = b[2] + lz;
      if (gx >= 0 && gx < ncell && gy >= 0 && gy < ncell && gz >= 0 && gz < ncell) continue;
      const int cx = bc_amr(gx, ncell, 1), cy = bc_amr(gy, ncell, 1), cz = bc_amr(gz, ncell, 1);
      if (lookup_at<NN>(A, Lcf, cx, cy, cz) != -2) continue;
      const int px = cx >> 1, py = cy >> 1, pz = cz >> 1;
      const int tc = lookup_at<NN>(A, Lc, px, py, pz);
      if (tc < 0) {
        atomicOr(A.status, 4u);
        continue;
      }
      const double* Cp = A.U + (size_t)tc * F * LS3 + (((pz & LM) + G) * LS + ((py & LM) + G)) * LS + ((px & LM) + G);
      const int Cw[3] = {px, py, pz};
      const double* nbp[6];
      int nbs[6];
      coarse_stencil<NN, kDirect>(A, Lc, Lcf, Cw, Cp, nbp, nbs);
      const double off[3] = {(cx & 1) ? 0.25 : -0.25, (cy & 1) ? 0.25 : -0.25, (cz & 1) ? 0.25 : -0.25};
      prolong_cell<NN>(Cp, nbp, nbs, off, dstb + c);
    }
  }
}

// Each leaf's restriction image: image cell (i, j, k) of field f is the mean
// of the leaf's cells (2i + dx, 2j + dy, 2k + dz), in the first pass's order
// and rounding (children at d = dx + 2 dy + 4 dz, summed pairwise, times
// 1/8), so it equals the value that pass writes into a coarser leaf's ghost
// cell over this leaf.
template <int NN>
__global__ void __launch_bounds__(256) hydro_amr_restrict_kernel(const double* __restrict__ U,
                                                                 double* __restrict__ img, int n_sub) {
  constexpr int LS = NN + 2 * G, LS3 = LS * LS * LS, H2 = NN / 2, I3 = img_cells<NN>();
  for (int s = blockIdx.x; s < n_sub; s += gridDim.x) {
    for (int e = threadIdx.x; e < F * I3; e += blockDim.x) {
      const int k = e / I3, i = e % I3;
      const int x = i % H2, y = (i / H2) % H2, z = i / (H2 * H2);
      const double* p = U + ((size_t)s * F + k) * LS3 + ((2 * z + G) * LS + (2 * y + G)) * LS + (2 * x + G);
      const double a0 = __ldg(p), a1 = __ldg(p + 1), a2 = __ldg(p + LS), a3 = __ldg(p + LS + 1);
      const double a4 = __ldg(p + LS * LS), a5 = __ldg(p + LS * LS + 1), a6 = __ldg(p + LS * LS + LS),
                   a7 = __ldg(p + LS * LS + LS + 1);
      img[((size_t)s * F + k) * I3 + i] =
          rmul(radd(radd(radd(a0, a1), radd(a2, a3)), radd(radd(a4, a5), radd(a6, a7))), 0.125);
    }
  }
}

// Coarse-fine flux correction of a leaf, in parts shared by the separate
// kernel and the update of the adaptive RK3 sequence.
//
// leaf_finer: the leaf's six face neighbours looked up once (bit 2a + side
// of the result: refined at the leaf's level) and, for such faces, the four
// finer leaves across each (fine[2a + side][2 qc + qb], qb and qc the halves
// of the face along its transverse axes b < c).  Every thread of the block
// calls it (it synchronises) and gets the same result.
template <int NN>
__device__ __forceinline__ int leaf_finer(const AMRArgs& A, int l, const int ijk[3], int* finer, int (*fine)[4]) {
  const int n = 1 << l;
  __syncthreads();  // the previous leaf's tables are no longer read
  if (threadIdx.x == 0) *finer = 0;
  __syncthreads();
  if (threadIdx.x < 6 && l < A.lmax) {
    const int a = threadIdx.x >> 1, side = threadIdx.x & 1;
    int nb[3] = {ijk[0], ijk[1], ijk[2]};
    nb[a] += side ? 1 : -1;
    bool in = true;
    if (nb[a] < 0 || nb[a] >= n) {
      if (A.bc != 0) in = false;
      else nb[a] = (nb[a] + n) % n;
    }
    if (in && lookup<NN>(A, l, nb[0] * NN, nb[1] * NN, nb[2] * NN) == -1) atomicOr(finer, 1 << threadIdx.x);
  }
  __syncthreads();
  const int fl = *finer;
  if (!fl) return 0;
  if (threadIdx.x < 24) {
    const int j = threadIdx.x >> 2, a = j >> 1, side = j & 1, qb = threadIdx.x & 1, qc = (threadIdx.x >> 1) & 1;
    const int b = (a == 0) ? 1 : 0, c = (a == 2) ? 1 : 2;
    int o = -3;
    if (fl & (1 << j)) {
      const int nf = 2 * n;
      int pf[3];
      pf[a] = side ? 2 * (ijk[a] + 1) : 2 * ijk[a] - 1;
      if (pf[a] < 0 || pf[a] >= nf) pf[a] = (pf[a] + nf) % nf;  // periodic wrap
      pf[b] = 2 * ijk[b] + qb;
      pf[c] = 2 * ijk[c] + qc;
      o = lookup<NN>(A, l + 1, pf[0] * NN, pf[1] * NN, pf[2] * NN);
    }
    fine[j][threadIdx.x & 3] = o;
  }
  __syncthreads();
  return fl;
}

// Whether interior cell `cell` lies on a leaf face flagged in fl.
template <int NN>
__device__ __forceinline__ bool on_finer_face(int cell, int fl) {
  const int cl[3] = {cell % NN, (cell / NN) % NN, cell / (NN * NN)};
  bool on = false;
#pragma unroll
  for (int a = 0; a < 3; ++a)
    on |= (((fl >> (2 * a)) & 1) && cl[a] == 0) || (((fl >> (2 * a + 1)) & 1) && cl[a] == NN - 1);
  return on;
}

// The corrections of interior cell `cell` of leaf s (cell width hc), added
// to its rates du in the order x-, x+, y-, y+, z-, z+: a face bordering finer
// leaves takes the mean of the 4 fine sub-face fluxes instead of its own,
// and the mean of the fine torques moved to the cell centre,
// T(x_C) = T(x_f) + (x_f - x_C) x F_s.
template <int NN>
__device__ __forceinline__ void correct_cell(const AMRArgs& A, const double* faces, int s, const int ijk[3],
                                             double hc, int fl, const int (*fine)[4], int cell, double du[F]) {
  constexpr int LM = NN - 1, H2 = NN / 2;
  const int cl[3] = {cell % NN, (cell / NN) % NN, cell / (NN * NN)};
  for (int a = 0; a < 3; ++a) {
    const int b = (a == 0) ? 1 : 0, c = (a == 2) ? 1 : 2;
    for (int side = 0; side < 2; ++side) {
      if (cl[a] != (side ? NN - 1 : 0)) continue;
      if (!(fl & (1 << (2 * a + side)))) continue;
      const double sgn = side ? 1.0 : -1.0;
      const int pb = cl[b], pc = cl[c];
      double fsum[F], tsum[3] = {0.0, 0.0, 0.0};
#pragma unroll
      for (int k = 0; k < F; ++k) fsum[k] = 0.0;
      // the fine leaf across this half of the face: the same for the four
      // sub-faces of the cell
      const int o = fine[2 * a + side][2 * (pc / H2) + pb / H2];
      if (o < 0) {
        atomicOr(A.status, 4u);
        continue;
      }
#pragma unroll
      for (int dc = 0; dc < 2; ++dc)
#pragma unroll
        for (int db = 0; db < 2; ++db) {
          int gf[3];
          gf[a] = side ? (ijk[a] + 1) * 2 * NN : ijk[a] * 2 * NN - 1;
          gf[b] = 2 * (ijk[b] * NN + pb) + db;
          gf[c] = 2 * (ijk[c] * NN + pc) + dc;
          const int loc[3] = {gf[0] & LM, gf[1] & LM, gf[2] & LM};
          const double* ff = faces + face_index_nn<NN>(o, 2 * a + (side ? 0 : 1), 0, loc[c], loc[b]);
          const size_t qs = (size_t)NN * NN;  // stride between quantities
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
      const double* own = faces + face_index_nn<NN>(s, 2 * a + side, 0, pc, pb);
      const size_t qs = (size_t)NN * NN;
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
}

// Each leaf's finer-neighbour table, as leaf_finer leaves it in shared
// memory: entry 0 the flags, entry 1 + 4 (2a + side) + 2 qc + qb the finer
// leaf across that half of a flagged face (-3 for faces not flagged).  Eight
// lanes per leaf, one per face (lanes 6 and 7 idle); the flags are the
// group's ballot.
template <int NN>
__global__ void __launch_bounds__(256) hydro_amr_finer_kernel(AMRArgs A) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int s = t >> 3, j = t & 7;
  bool refined = false;
  int o[4] = {-3, -3, -3, -3};
  if (s < A.n_sub && j < 6) {
    const int l = A.leaf_level[s], n = 1 << l;
    const int ijk[3] = {A.leaf_ijk[3 * s], A.leaf_ijk[3 * s + 1], A.leaf_ijk[3 * s + 2]};
    const int a = j >> 1, side = j & 1, b = (a == 0) ? 1 : 0, c = (a == 2) ? 1 : 2;
    int nb[3] = {ijk[0], ijk[1], ijk[2]};
    nb[a] += side ? 1 : -1;
    bool in = l < A.lmax;
    if (nb[a] < 0 || nb[a] >= n) {
      if (A.bc != 0) in = false;
      else nb[a] = (nb[a] + n) % n;
    }
    refined = in && lookup<NN>(A, l, nb[0] * NN, nb[1] * NN, nb[2] * NN) == -1;
    if (refined) {
      const int nf = 2 * n;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        int pf[3];
        pf[a] = side ? 2 * (ijk[a] + 1) : 2 * ijk[a] - 1;
        if (pf[a] < 0 || pf[a] >= nf) pf[a] = (pf[a] + nf) % nf;  // periodic wrap
        pf[b] = 2 * ijk[b] + (q & 1);
        pf[c] = 2 * ijk[c] + (q >> 1);
        o[q] = lookup<NN>(A, l + 1, pf[0] * NN, pf[1] * NN, pf[2] * NN);
      }
    }
  }
  const unsigned m = __ballot_sync(0xffffffffu, refined);
  if (s < A.n_sub) {
    int* e = A.finer_tab + (size_t)s * kFinerTab;
    if (j == 0) e[0] = (int)((m >> (threadIdx.x & 24)) & 0x3fu);
    if (j < 6)
#pragma unroll
      for (int q = 0; q < 4; ++q) e[1 + 4 * j + q] = o[q];
  }
}

// One thread per interior cell of a leaf; a leaf with no finer face
// neighbour, most of a mesh, is left at once.  kTable: the leaf's flags and
// finer leaves come from A.finer_tab (hydro_amr_finer_kernel) instead of
// being looked up here.
template <int NN, bool kTable>
__global__ void __launch_bounds__(256) hydro_flux_correct_kernel(AMRArgs A, const double* h, const double* faces,
                                                                 double* dUdt) {
  constexpr int LN3 = NN * NN * NN;
  __shared__ int finer;
  __shared__ int fine_s[6][4];
  for (int u = blockIdx.x; u < A.n_sub; u += gridDim.x) {
    const int s = leaf_at(A, u);
    if (s < 0) continue;
    const int ijk[3] = {A.leaf_ijk[3 * s], A.leaf_ijk[3 * s + 1], A.leaf_ijk[3 * s + 2]};
    int fl;
    const int(*fine)[4];
    if (kTable) {
      const int* ft = A.finer_tab + (size_t)s * kFinerTab;
      fl = __ldg(ft);
      fine = reinterpret_cast<const int(*)[4]>(ft + 1);
    } else {
      fl = leaf_finer<NN>(A, A.leaf_level[s], ijk, &finer, fine_s);
      fine = fine_s;
    }
    if (!fl) continue;
    const double hc = h[s];
    for (int cell = threadIdx.x; cell < LN3; cell += blockDim.x) {
      if (!on_finer_face<NN>(cell, fl)) continue;
      double du[F];
#pragma unroll
      for (int k = 0; k < F; ++k) du[k] = dUdt[((size_t)s * F + k) * LN3 + cell];
      correct_cell<NN>(A, faces, s, ijk, hc, fl, fine, cell, du);
#pragma unroll
      for (int k = 0; k < F; ++k) dUdt[((size_t)s * F + k) * LN3 + cell] = du[k];
    }
  }
}

// The update of the adaptive RK3 sequence with direct neighbour reads (8^3
// leaves): per leaf, in the mesh's order, the SSP-RK3 stage update of every
// interior cell (rk3_cell, as hydro_update) from A.U and U0 into Uout, and
// with kImage the new state's restriction image (as
// hydro_amr_restrict_kernel) for the next stage's fill: the same bits as
// the separate launches, without reading the new state back.
template <bool kMixed, bool kImage>
__global__ void __launch_bounds__(256) hydro_update_amr_kernel(AMRArgs A, const double* dUdt, const double* U0,
                                                               double* Uout, const double* dt_dev, double alpha,
                                                               double beta, double eta2, double inv_gamma) {
  constexpr int NN = 8, LS = NN + 2 * G, LS3 = LS * LS * LS, LN3 = NN * NN * NN, H2 = NN / 2,
                I3 = img_cells<NN>();
  __shared__ double img_s[kImage ? F * LN3 : 1];  // the leaf's new state, for its image
  const double dt = *dt_dev;
  for (int u = blockIdx.x; u < A.n_sub; u += gridDim.x) {
    const int s = leaf_at(A, u);
    if (s < 0) continue;
    const size_t ub = (size_t)s * F * LS3, db = (size_t)s * F * LN3;
    for (int cell = threadIdx.x; cell < LN3; cell += blockDim.x) {
      const int x = cell % NN, y = (cell / NN) % NN, z = cell / (NN * NN);
      const size_t uc = ub + ((z + G) * LS + (y + G)) * LS + (x + G), dc = db + cell;
      double Uc[F], U0c[F], R[F], un[F];
#pragma unroll
      for (int k = 0; k < F; ++k) {
        Uc[k] = A.U[uc + (size_t)k * LS3];
        U0c[k] = U0[uc + (size_t)k * LS3];
        R[k] = dUdt[dc + (size_t)k * LN3];
      }
      rk3_cell<kMixed>(Uc, U0c, R, dt, alpha, beta, eta2, inv_gamma, un);
#pragma unroll
      for (int k = 0; k < F; ++k) Uout[uc + (size_t)k * LS3] = un[k];
      if (kImage) {
#pragma unroll
        for (int k = 0; k < F; ++k) img_s[k * LN3 + cell] = un[k];
      }
    }
    if (kImage) {
      __syncthreads();
      for (int e = threadIdx.x; e < F * I3; e += blockDim.x) {
        const int k = e / I3, i = e % I3;
        const int x = i % H2, y = (i / H2) % H2, z = i / (H2 * H2);
        const double* p = img_s + k * LN3 + ((2 * z) * NN + 2 * y) * NN + 2 * x;
        const double a0 = p[0], a1 = p[1], a2 = p[NN], a3 = p[NN + 1];
        const double a4 = p[NN * NN], a5 = p[NN * NN + 1], a6 = p[NN * NN + NN], a7 = p[NN * NN + NN + 1];
        A.image[((size_t)s * F + k) * I3 + i] =
            rmul(radd(radd(radd(a0, a1), radd(a2, a3)), radd(radd(a4, a5), radd(a6, a7))), 0.125);
      }
      __syncthreads();  // img_s is free for the next leaf
    }
  }
}

}  // namespace hyd

hyd::AMRArgs hydro_amr_args(hydro_ctx_t* c, const hydro_batch_t* B, const hydro_amr_t* M) {
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
  A.image = c->amr_img;
  A.order = M->order;
  A.finer_tab = reinterpret_cast<int*>(c->amr_finer);
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
  hyd::AMRArgs A = hydro_amr_args(c, B, M);
  const int cap = c->num_sms * 8;
  const int grid = B->n_sub < cap ? B->n_sub : cap;
  cudaStream_t st = (cudaStream_t)stream;
  if (c->N == 16) {
    hyd::hydro_ghost_amr_kernel<16><<<grid, 256, 0, st>>>(A);
    hyd::hydro_ghost_amr_prolong_kernel<16, false><<<grid, 256, 0, st>>>(A);
  } else {
    hyd::hydro_ghost_amr_kernel<8><<<grid, 256, 0, st>>>(A);
    hyd::hydro_ghost_amr_prolong_kernel<8, false><<<grid, 256, 0, st>>>(A);
  }
  return cudaGetLastError() == cudaSuccess ? HYDRO_OK : HYDRO_ECUDA;
}

int hydro_flux_correct_amr(hydro_ctx_t* c, const hydro_batch_t* B, const hydro_amr_t* M, const double* face_flux,
                           double* dUdt, void* stream) {
  if (!c || !B || B->n_sub < 0 || !amr_ok(M)) return HYDRO_EINVAL;
  if (B->n_sub == 0) return HYDRO_OK;
  if (!B->h || !face_flux || !dUdt) return HYDRO_EINVAL;
  int rc = hydro_ctx_prepare(c, 0);
  if (rc) return rc;
  hyd::AMRArgs A = hydro_amr_args(c, B, M);
  const int cap = c->num_sms * 8;
  const int grid = B->n_sub < cap ? B->n_sub : cap;
  if (c->N == 16)
    hyd::hydro_flux_correct_kernel<16, false><<<grid, 256, 0, (cudaStream_t)stream>>>(A, B->h, face_flux, dUdt);
  else
    hyd::hydro_flux_correct_kernel<8, false><<<grid, 256, 0, (cudaStream_t)stream>>>(A, B->h, face_flux, dUdt);
  return cudaGetLastError() == cudaSuccess ? HYDRO_OK : HYDRO_ECUDA;
}

}  // extern "C"

// The lean fill of the adaptive RK3 sequence (8^3 leaves; the step's loader
// reads same-level and finer neighbours itself): every leaf's restriction
// image and finer-neighbour table (with restrict_first; otherwise the
// previous stage's update wrote the images for this state), then the ghost cells inside coarser leaves, prolonged
// from coarse cells whose neighbours are read where they live.  Ghost cells
// held by same-level or finer leaves are left as they were.  The image
// buffer (hydro_ctx_prepare_amr) must hold n_sub leaves.
int hydro_fill_ghosts_amr_lean(hydro_ctx_t* c, const hydro_batch_t* B, const hydro_amr_t* M, bool restrict_first,
                               cudaStream_t st) {
  if (!c || !B || B->n_sub < 0 || !amr_ok(M) || c->N != 8) return HYDRO_EINVAL;
  if (B->n_sub == 0) return HYDRO_OK;
  if (!B->U || !c->amr_img || c->amr_img_bytes < (size_t)B->n_sub * hyd::F * hyd::img_cells<8>() * sizeof(double))
    return HYDRO_EINVAL;
  if (!c->amr_finer || c->amr_finer_bytes < (size_t)B->n_sub * hyd::kFinerTab * sizeof(int)) return HYDRO_EINVAL;
  hyd::AMRArgs A = hydro_amr_args(c, B, M);
  const int cap = c->num_sms * 8;
  const int grid = B->n_sub < cap ? B->n_sub : cap;
  if (restrict_first) {
    hyd::hydro_amr_restrict_kernel<8><<<grid, 256, 0, st>>>(B->U, c->amr_img, B->n_sub);
    hyd::hydro_amr_finer_kernel<8><<<(8 * B->n_sub + 255) / 256, 256, 0, st>>>(A);
  }
  hyd::hydro_ghost_amr_prolong_kernel<8, true><<<grid, 256, 0, st>>>(A);
  return cudaGetLastError() == cudaSuccess ? HYDRO_OK : HYDRO_ECUDA;
}

// The coarse-fine flux correction (from the finer-neighbour tables of the
// lean fill) and the SSP-RK3 stage update of the adaptive RK3 sequence
// (hydro_update_amr_kernel): B->U the stage's state, U0 the step's initial
// state, Uout the new state (B->U in place after the first stage), dt on
// the device; with image the new state's restriction images for the next
// stage's lean fill.
int hydro_update_amr_lean(hydro_ctx_t* c, const hydro_batch_t* B, const hydro_amr_t* M, const double* U0,
                          double* dUdt, const double* face_flux, const double* dt_dev, int stage, double* Uout,
                          bool image, cudaStream_t st) {
  if (!c || !B || B->n_sub < 0 || !amr_ok(M) || c->N != 8 || stage < 0 || stage > 2) return HYDRO_EINVAL;
  if (B->n_sub == 0) return HYDRO_OK;
  if (!B->U || !B->h || !U0 || !dUdt || !face_flux || !dt_dev || !Uout) return HYDRO_EINVAL;
  if (!c->amr_finer || c->amr_finer_bytes < (size_t)B->n_sub * hyd::kFinerTab * sizeof(int)) return HYDRO_EINVAL;
  if (image && (!c->amr_img ||
                c->amr_img_bytes < (size_t)B->n_sub * hyd::F * hyd::img_cells<8>() * sizeof(double)))
    return HYDRO_EINVAL;
  static const double alpha[3] = {0.0, 0.75, 1.0 / 3.0};
  static const double beta[3] = {1.0, 0.25, 2.0 / 3.0};
  hyd::AMRArgs A = hydro_amr_args(c, B, M);
  const int cap = c->num_sms * 8;
  const int grid = B->n_sub < cap ? B->n_sub : cap;
  const bool mixed = c->mode.precision == HYDRO_PREC_MIXED;
  const double eta2 = c->mode.de_eta2, ig = 1.0 / c->gamma;
  const double al = alpha[stage], be = beta[stage];
  hyd::hydro_flux_correct_kernel<8, true><<<grid, 256, 0, st>>>(A, B->h, face_flux, dUdt);
  if (mixed && image)
    hyd::hydro_update_amr_kernel<true, true><<<grid, 256, 0, st>>>(A, dUdt, U0, Uout, dt_dev, al, be, eta2, ig);
  else if (mixed)
    hyd::hydro_update_amr_kernel<true, false><<<grid, 256, 0, st>>>(A, dUdt, U0, Uout, dt_dev, al, be, eta2, ig);
  else if (image)
    hyd::hydro_update_amr_kernel<false, true><<<grid, 256, 0, st>>>(A, dUdt, U0, Uout, dt_dev, al, be, eta2, ig);
  else
    hyd::hydro_update_amr_kernel<false, false><<<grid, 256, 0, st>>>(A, dUdt, U0, Uout, dt_dev, al, be, eta2, ig);
  return cudaGetLastError() == cudaSuccess ? HYDRO_OK : HYDRO_ECUDA;
}
