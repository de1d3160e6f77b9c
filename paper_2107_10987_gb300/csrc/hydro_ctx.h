// hydro_ctx.h -- the context behind the opaque hydro_ctx_t of include/hydro.h.
#pragma once
#include <cstddef>

#include "hydro.h"

struct hydro_ctx {
  int N, G, n_species, F;
  double gamma, omega;
  hydro_mode_t mode;
  int device;
  int num_sms;
  int slots_tuned[2];    // persistent CTAs chosen by hydro_autotune_step (0: default), [fp64, mixed]
  unsigned* status;      // device word
  double* scratch;       // step scratch
  size_t scratch_bytes;
  double* part;          // conservation partials
  size_t part_bytes;
  int gate_on;           // learned smoothness indicator active (mixed mode)
  double gate_logit_thr; // smooth where the indicator's logit is below this
  int gate_zero_smooth;  // decision for all-zero features, set with the parameters
  float* gate_w;         // BF16-rounded indicator parameters (device)
};

// Allocate the context's status word and the step scratch for a batch of
// n_sub sub-grids, and opt the step kernels in to their shared memory, so
// that later launches allocate nothing (needed before a stream capture).
int hydro_ctx_prepare(hydro_ctx* c, int n_sub);
