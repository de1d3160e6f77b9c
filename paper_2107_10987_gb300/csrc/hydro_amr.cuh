// hydro_amr.cuh -- octree lookups shared by the adaptive-mesh kernels: the
// ghost fill and flux correction (hydro_amr.cu) and the mixed step whose
// tile loader reads a leaf's same-level and finer neighbours directly
// (hydro_step_mixed_amr.cu).
//
// Leaves are found through dense per-level tables (hydro_amr_t): at level l
// entry ((k 2^l) + j) 2^l + i is the leaf index at that sub-grid position,
// -1 where the position is refined, -2 where it lies inside a coarser leaf.
#pragma once
#include "hydro_common.cuh"

namespace hyd {

struct AMRArgs {
  double* U;
  const int* table;
  const int* leaf_level;
  const int* leaf_ijk;
  int lmin, lmax, bc, n_sub;
  unsigned* status;
  // [n_sub][F][(NN/2)^3]: each leaf's restriction image (the means of its
  // 2^3 cell blocks, written by hydro_amr_restrict_kernel), or null
  double* image;
  const int* order;  // the order in which kernels take the leaves, or null
  // [n_sub][kFinerTab]: per leaf, the faces that border finer leaves (bits
  // 2a + side) and the four finer leaves across each (hydro_amr_finer_kernel),
  // or null
  int* finer_tab;
};

constexpr int kFinerTab = 25;

// The leaf that work unit u (0 <= u < n_sub) takes, or -1 (with status bit
// 4) for an order entry outside the leaves.
__device__ __forceinline__ int leaf_at(const AMRArgs& A, int u) {
  if (!A.order) return u;
  const int s = __ldg(A.order + u);
  if ((unsigned)s < (unsigned)A.n_sub) return s;
  if (threadIdx.x == 0) atomicOr(A.status, 4u);
  return -1;
}

__device__ __forceinline__ long level_offset(int l, int lmin) {
  // sum_{m = lmin}^{l-1} 8^m
  long off = 0;
  for (int m = lmin; m < l; ++m) off += 1L << (3 * m);
  return off;
}

// One level's part of the tables: its offset and its sub-grid positions per
// axis (n = 0: a level the mesh does not have).
struct LevelRef {
  long off;
  int n;
};

__device__ __forceinline__ LevelRef level_ref(const AMRArgs& A, int l) {
  if (l < A.lmin || l > A.lmax) return LevelRef{0, 0};
  return LevelRef{level_offset(l, A.lmin), 1 << l};
}

// The leaf (or -1 / -2) holding global cell (gx, gy, gz) >= 0 of level L,
// for leaves of NN^3 cells; -3 for a level the mesh does not have.
template <int NN>
__device__ __forceinline__ int lookup_at(const AMRArgs& A, LevelRef L, int gx, int gy, int gz) {
  if (L.n == 0) return -3;
  const unsigned px = (unsigned)gx / NN, py = (unsigned)gy / NN, pz = (unsigned)gz / NN;
  return __ldg(A.table + L.off + ((long)pz * L.n + py) * L.n + px);
}

template <int NN>
__device__ __forceinline__ int lookup(const AMRArgs& A, int l, int gx, int gy, int gz) {
  return lookup_at<NN>(A, level_ref(A, l), gx, gy, gz);
}

// The boundary map of a global cell coordinate of a level with n cells
// along the axis: periodic wraps, outflow clamps.
__device__ __forceinline__ int bc_amr(int g, int n, int bc) {
  if (bc == 0) return g < 0 ? g + n : (g >= n ? g - n : g);
  return g < 0 ? 0 : (g >= n ? n - 1 : g);
}

// Cells of a leaf's restriction image.
template <int NN>
__host__ __device__ constexpr int img_cells() {
  return (NN / 2) * (NN / 2) * (NN / 2);
}

// Where the value of boundary-mapped global cell (gx, gy, gz) of level l
// lives, as the ghost fill's first pass would copy or restrict it into a
// ghost cell: the interior cell of the level-l leaf holding it, or, where
// the position is refined, the image cell of the level-(l+1) leaf holding
// its eight children (the same sum in the same order).  Returns the pointer
// to field 0 and sets the field stride; null where the position lies inside
// a coarser leaf (filled by the prolongation), and null with status bit 4
// where the octree is not 2:1 balanced there.
// L and Lf: the tables of levels l and l + 1.
template <int NN>
__device__ __forceinline__ const double* amr_source(const AMRArgs& A, LevelRef L, LevelRef Lf, int gx, int gy,
                                                    int gz, size_t& stride) {
  constexpr int LS = NN + 2 * G, LS3 = LS * LS * LS, LM = NN - 1, H2 = NN / 2;
  const int t = lookup_at<NN>(A, L, gx, gy, gz);
  if (t >= 0) {
    stride = LS3;
    return A.U + (size_t)t * F * LS3 + (((gz & LM) + G) * LS + ((gy & LM) + G)) * LS + ((gx & LM) + G);
  }
  if (t == -1) {
    const int tf = lookup_at<NN>(A, Lf, 2 * gx, 2 * gy, 2 * gz);
    if (tf >= 0) {
      stride = img_cells<NN>();
      return A.image + (size_t)tf * F * img_cells<NN>() + ((gz & (H2 - 1)) * H2 + (gy & (H2 - 1))) * H2 +
             (gx & (H2 - 1));
    }
  }
  if (t != -2) atomicOr(A.status, 4u);
  return nullptr;
}

}  // namespace hyd
