// hydro_ctx.h -- the context behind the opaque hydro_ctx_t of include/hydro.h.
#pragma once
#include <cstddef>
#include <vector>

#include <cuda_runtime.h>

#include "hydro.h"

struct hydro_ctx {
  int N, G, n_species, F;
  double gamma, omega;
  hydro_mode_t mode;
  int device;
  int num_sms;
  int slots_tuned[2];    // persistent CTAs chosen by hydro_autotune_step or hydro_set_launch (0: default), [fp64, mixed]
  int decomp;            // mixed-precision sub-grid decomposition, HYDRO_DECOMP_* (AUTO: planes)
  unsigned* status;      // device word
  double* scratch;       // step scratch
  size_t scratch_bytes;
  double* lines;         // FP64 step: per-CTA line ends
  size_t lines_bytes;
  double* part;          // conservation partials
  size_t part_bytes;
  int gate_on;           // learned smoothness indicator active (mixed mode)
  double gate_logit_thr; // smooth where the indicator's logit is below this
  int gate_zero_smooth;  // decision for all-zero features, set with the parameters
  float* gate_w;         // BF16-rounded indicator parameters (device)
  double* u2;            // fused RK3 step: second-stage state [n_sub][F][N^3]
  size_t u2_bytes;
  double* prims;         // fused RK3 step: 2 x [n_sub][F][N^3] FP32 primitives (float words)
  size_t prims_bytes;
  double* sync;          // fused RK3 step: barrier, work counter and per-sub-grid flags (unsigned words)
  size_t sync_bytes;
  double* amr_img;       // adaptive RK3 step: each leaf's restriction image [n_sub][F][(N/2)^3]
  size_t amr_img_bytes;
  double* amr_finer;     // adaptive RK3 step: each leaf's finer-neighbour table (int words)
  size_t amr_finer_bytes;
  // Once a CUDA graph has been captured on the context, a work buffer that
  // has to grow keeps its old allocation here (graphs hold its address)
  // until hydro_destroy.
  bool had_graph;
  std::vector<void*> retired;
};

// Allocate the context's status word and the step scratch for a batch of
// n_sub sub-grids, and opt the step kernels in to their shared memory, so
// that later launches allocate nothing (needed before a stream capture).
int hydro_ctx_prepare(hydro_ctx* c, int n_sub);

// Enqueue the fused RK3 time step (hydro_rk3_desc_t.fused) of a uniform mesh,
// allocating its buffers on first use (hydro_ctx_prepare_fused before a
// capture).
int hydro_ctx_prepare_fused(hydro_ctx* c, int n_sub);
// The adaptive RK3 sequence with direct neighbour reads: whether this
// context's step takes it (mixed precision, 8^3 leaves, row sweep, no
// contact steepening or spin feedback), its image buffer for n_sub leaves
// (allocated before a stream capture), its lean ghost fill, its step, and
// its flux correction with the stage update.
bool hydro_amr_direct_ok(const hydro_ctx* c);
int hydro_ctx_prepare_amr(hydro_ctx* c, int n_sub);
int hydro_fill_ghosts_amr_lean(hydro_ctx* c, const hydro_batch_t* B, const hydro_amr_t* M, bool restrict_first,
                               cudaStream_t st);
int hydro_update_amr_lean(hydro_ctx* c, const hydro_batch_t* B, const hydro_amr_t* M, const double* U0,
                          double* dUdt, const double* face_flux, const double* dt_dev, int stage, double* Uout,
                          bool image, cudaStream_t st);
int hydro_step_amr_direct(hydro_ctx* c, const hydro_batch_t* B, const hydro_amr_t* M, double* dUdt, double* amax,
                          double* face_flux, cudaStream_t st);
int hydro_rk3_fused_enqueue(hydro_ctx* c, const hydro_rk3_desc_t* d, int parity, cudaStream_t st);
