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
  unsigned* status;      // device word
  double* scratch;       // step scratch
  size_t scratch_bytes;
  double* part;          // conservation partials
  size_t part_bytes;
};
