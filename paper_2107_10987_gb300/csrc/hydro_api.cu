// hydro_api.cu -- the C ABI (include/hydro.h): context, argument checks,
// scratch management and dispatch to the kernels.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include "hydro.h"
#include "hydro_amr.cuh"
#include "hydro_common.cuh"
#include "hydro_ctx.h"

namespace hyd {
cudaError_t launch_step_mixed_amr(const StepArgs64& A, const AMRArgs& M, int grid, cudaStream_t st);
cudaError_t launch_step_fp64_lines(const StepArgs64& A, int grid, int nn, cudaStream_t st);
cudaError_t prepare_step_fp64_lines();
size_t step_fp64_lines_per_cta();
cudaError_t launch_step_mixed(const StepArgs64& A, int grid, int planes, int nn, cudaStream_t st);
cudaError_t prepare_step_fp64();
cudaError_t prepare_step_mixed();
cudaError_t launch_update(const double* U, double* Uout, const double* U0, const double* dUdt, double dt,
                          const double* dt_dev, int stage, double eta2, double gamma, int n_sub, bool mixed,
                          int num_sms, int nn, cudaStream_t st);
cudaError_t launch_dt(const double* amax, const double* h, int n, double cfl, double* out, cudaStream_t st);
cudaError_t launch_ghost_uniform(double* U, int nbx, int nby, int nbz, int bc, int num_sms, int nn,
                                 cudaStream_t st);
cudaError_t launch_interior(double* U, double* I, int n_sub, bool scatter, int num_sms, int nn, cudaStream_t st);
cudaError_t launch_rk3_fused(const StepArgs64& S, double* Y, double* U2, float* prims, double* dt_out,
                             unsigned* sync, int nbx, int nby, int nbz, int bc, double cfl, double eta2,
                             double gamma, int num_sms, int planes, int nn, cudaStream_t st);
cudaError_t prepare_rk3_fused(int num_sms, int planes, int nn, int* max_grid);
size_t rk3_fused_sync_words(int n_sub);
cudaError_t launch_wait_selftest(unsigned* words, unsigned* status, long long limit_ns, cudaStream_t st);
cudaError_t launch_sums(const double* U, const double* origin, const double* h, int n_sub, double* part,
                        double* sums, int nn, cudaStream_t st);
}  // namespace hyd


static thread_local char g_cuda_err[256] = "no CUDA error";

static int cuda_fail(cudaError_t e, const char* where) {
  snprintf(g_cuda_err, sizeof g_cuda_err, "%s: %s", where, cudaGetErrorString(e));
  return HYDRO_ECUDA;
}

static bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// Cells of a padded sub-grid of the context's layout, and the 8^3 tiles the
// step kernels process for n_sub sub-grids (one per 8^3 sub-grid, eight
// octants per 16^3 sub-grid).
static size_t padded_cells(const hydro_ctx* c) {
  const size_t s = (size_t)c->N + 2 * hyd::G;
  return s * s * s;
}
static int step_units(const hydro_ctx* c, int n_sub) {
  const int t = c->N / hyd::N;
  return n_sub * t * t * t;
}

static int ensure_status(hydro_ctx* c) {
  if (c->status) return HYDRO_OK;
  cudaError_t e = cudaMalloc(&c->status, sizeof(unsigned));
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(status)");
  e = cudaMemset(c->status, 0, sizeof(unsigned));
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemset(status)");
  return HYDRO_OK;
}

// Grow one of the context's work buffers to `need` bytes (no-op if it is
// large enough).  The old allocation is freed, or, once a graph has been
// captured on the context, kept until hydro_destroy: a graph replays with
// the addresses it was captured with.
static int ensure_buf(hydro_ctx* c, double** buf, size_t* have, size_t need, const char* what) {
  if (*have >= need) return HYDRO_OK;
  if (*buf && c->had_graph) {
    try {
      c->retired.push_back(*buf);
    } catch (...) {
      return HYDRO_ENOMEM;
    }
  } else if (*buf) {
    cudaFree(*buf);
  }
  *buf = nullptr;
  *have = 0;
  cudaError_t e = cudaMalloc(buf, need);
  if (e != cudaSuccess) {
    cuda_fail(e, what);
    return HYDRO_ENOMEM;
  }
  *have = need;
  return HYDRO_OK;
}

// The sub-grid decomposition a step of this context runs: the row sweep
// unless the plane sweep was chosen (by hydro_set_launch or the autotuner;
// mixed precision without the learned indicator only).
static int eff_decomp(const hydro_ctx* c) {
  if (c->mode.precision != HYDRO_PREC_MIXED || c->gate_on) return HYDRO_DECOMP_ROWS;
  return c->decomp == HYDRO_DECOMP_PLANES ? HYDRO_DECOMP_PLANES : HYDRO_DECOMP_ROWS;
}

static int step_slots(const hydro_ctx* c, bool mixed) {
  // persistent CTAs: one per SM for FP64 (219 KB of shared memory each) and
  // for the plane sweep (190 KB, 672 threads), two per SM for the mixed row
  // sweep (110 KB each), unless the autotuner or the caller chose another
  if (c->slots_tuned[mixed ? 1 : 0] > 0) return c->slots_tuned[mixed ? 1 : 0];
  if (!mixed || eff_decomp(c) == HYDRO_DECOMP_PLANES) return c->num_sms;
  return 2 * c->num_sms;
}

// The FP64 step's per-CTA line-end buffers for its persistent grid over
// `units` tiles (2.08 MB per CTA).
static int ensure_lines(hydro_ctx* c, int units) {
  const int slots = step_slots(c, false);
  const int grid = units < slots ? units : slots;
  return ensure_buf(c, &c->lines, &c->lines_bytes, (size_t)grid * hyd::step_fp64_lines_per_cta() * sizeof(double),
                    "cudaMalloc(FP64 line ends)");
}

static hyd::StepArgs64 step_args(const hydro_ctx* c, const hydro_batch_t* B, double* dUdt, double* amax,
                                 double* face_flux) {
  hyd::StepArgs64 A;
  A.U = B->U;
  A.origin = B->origin;
  A.h = B->h;
  A.g = B->g;
  A.dUdt = dUdt;
  A.amax = amax;
  A.face_flux = face_flux;
  A.scratch = c->scratch;
  A.lines = c->lines;
  A.status = c->status;
  A.n_sub = B->n_sub;
  A.P.gamma = c->gamma;
  A.P.gm1 = c->gamma - 1.0;
  A.P.omega = c->omega;
  A.P.eta1 = c->mode.de_eta1;
  A.P.face_points = c->mode.flux_points == 1 ? 1 : 9;
  A.P.contact = c->mode.contact ? 1 : 0;
  A.P.spin = c->mode.spin ? 1 : 0;
  A.gate = c->gate_on ? 1 : 0;
  A.gate_w = c->gate_w;
  A.gate_logit_thr = (float)c->gate_logit_thr;
  A.gate_zero_smooth = c->gate_zero_smooth;
  return A;
}

int hydro_ctx_prepare_fused(hydro_ctx* c, int n_sub) {
  int rc = hydro_ctx_prepare(c, n_sub);
  if (rc) return rc;
  rc = ensure_buf(c, &c->u2, &c->u2_bytes, (size_t)n_sub * hyd::F * c->N * c->N * c->N * sizeof(double),
                  "cudaMalloc(fused second-stage state)");
  if (rc) return rc;
  rc = ensure_buf(c, &c->prims, &c->prims_bytes, 2 * (size_t)n_sub * hyd::F * c->N * c->N * c->N * sizeof(float),
                  "cudaMalloc(fused primitives)");
  if (rc) return rc;
  const size_t words = hyd::rk3_fused_sync_words(n_sub);
  rc = ensure_buf(c, &c->sync, &c->sync_bytes, (words * sizeof(unsigned) + 7) / 8 * 8, "cudaMalloc(fused sync words)");
  if (rc) return rc;
  int max_grid = 0;
  cudaError_t e = hyd::prepare_rk3_fused(c->num_sms, 0, c->N, &max_grid);
  if (e != cudaSuccess) return cuda_fail(e, "hydro_ctx_prepare_fused");
  return HYDRO_OK;
}

int hydro_rk3_fused_enqueue(hydro_ctx* c, const hydro_rk3_desc_t* d, int parity, cudaStream_t st) {
  if (d->amr || c->mode.precision != HYDRO_PREC_MIXED) return HYDRO_EUNSUP;
  if (d->bc != HYDRO_BC_PERIODIC && d->bc != HYDRO_BC_OUTFLOW) return HYDRO_EINVAL;
  if (!aligned16(d->a.U) || !aligned16(d->U_b) || !aligned16(d->dUdt)) return HYDRO_EINVAL;
  int rc = hydro_ctx_prepare_fused(c, d->a.n_sub);
  if (rc) return rc;
  hydro_batch_t X = d->a;
  double* Y = d->U_b;
  if (parity) {
    X.U = d->U_b;
    Y = d->a.U;
  }
  const hyd::StepArgs64 S = step_args(c, &X, d->dUdt, d->amax, nullptr);
  const double cfl = d->cfl > 0.0 ? d->cfl : c->mode.cfl;
  cudaError_t e = hyd::launch_rk3_fused(S, Y, c->u2, reinterpret_cast<float*>(c->prims), d->dt,
                                        reinterpret_cast<unsigned*>(c->sync), d->nbx, d->nby,
                                        d->nbz, d->bc, cfl, c->mode.de_eta2, c->gamma, c->num_sms,
                                        eff_decomp(c) == HYDRO_DECOMP_PLANES, c->N, st);
  if (e != cudaSuccess) return cuda_fail(e, "hydro_rk3_step (fused)");
  return HYDRO_OK;
}

extern "C" int hydro_selftest_wait(hydro_ctx_t* c, double seconds, void* stream) {
  if (!c || !(seconds > 0.0 && seconds <= 1.0)) return HYDRO_EINVAL;
  int rc = hydro_ctx_prepare_fused(c, 1);
  if (rc) return rc;
  cudaError_t e = hyd::launch_wait_selftest(reinterpret_cast<unsigned*>(c->sync), c->status,
                                            (long long)(seconds * 1e9), (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "hydro_selftest_wait");
  return HYDRO_OK;
}

int hydro_ctx_prepare(hydro_ctx* c, int n_sub) {
  int rc = ensure_status(c);
  if (rc) return rc;
  const int slots = 2 * c->num_sms;  // the most any launch uses
  const int units = step_units(c, n_sub);
  const int grid = units < slots ? units : slots;
  rc = ensure_buf(c, &c->scratch, &c->scratch_bytes, (size_t)grid * hyd::kScratchPerSub * sizeof(double),
                  "cudaMalloc(step scratch)");
  if (rc) return rc;
  if (c->mode.precision == HYDRO_PREC_FP64) {
    rc = ensure_lines(c, units);
    if (rc) return rc;
  }
  cudaError_t e = hyd::prepare_step_fp64();
  if (e == cudaSuccess) e = hyd::prepare_step_fp64_lines();
  if (e == cudaSuccess) e = hyd::prepare_step_mixed();
  if (e != cudaSuccess) return cuda_fail(e, "hydro_ctx_prepare");
  return HYDRO_OK;
}

bool hydro_amr_direct_ok(const hydro_ctx* c) {
  return c->N == hyd::N && c->mode.precision == HYDRO_PREC_MIXED && !c->mode.contact && !c->mode.spin &&
         eff_decomp(c) == HYDRO_DECOMP_ROWS;
}

int hydro_ctx_prepare_amr(hydro_ctx* c, int n_sub) {
  int rc = hydro_ctx_prepare(c, n_sub);
  if (rc) return rc;
  rc = ensure_buf(c, &c->amr_img, &c->amr_img_bytes,
                  (size_t)n_sub * hyd::F * (hyd::N / 2) * (hyd::N / 2) * (hyd::N / 2) * sizeof(double),
                  "cudaMalloc(restriction images)");
  if (rc) return rc;
  return ensure_buf(c, &c->amr_finer, &c->amr_finer_bytes, ((size_t)n_sub * hyd::kFinerTab * sizeof(int) + 7) & ~7ul,
                    "cudaMalloc(finer-neighbour tables)");
}

hyd::AMRArgs hydro_amr_args(hydro_ctx_t* c, const hydro_batch_t* B, const hydro_amr_t* M);

// The mixed row sweep over the leaves of an adaptive mesh, its loader
// reading same-level neighbours' interiors and finer neighbours' restriction
// images itself (hydro_fill_ghosts_amr_lean before it): the same dU/dt,
// amax and boundary faces, bit for bit, as hydro_step after the full fill.
int hydro_step_amr_direct(hydro_ctx* c, const hydro_batch_t* B, const hydro_amr_t* M, double* dUdt, double* amax,
                          double* face_flux, cudaStream_t st) {
  if (!c || !B || !M || B->n_sub < 0 || !hydro_amr_direct_ok(c)) return HYDRO_EINVAL;
  if (B->n_sub == 0) return HYDRO_OK;
  if (!B->U || !B->origin || !B->h || !dUdt || !amax || !face_flux) return HYDRO_EINVAL;
  if (!aligned16(B->U) || !aligned16(dUdt)) return HYDRO_EINVAL;
  int rc = hydro_ctx_prepare_amr(c, B->n_sub);
  if (rc) return rc;
  const int slots = step_slots(c, true);
  const int grid = B->n_sub < slots ? B->n_sub : slots;
  rc = ensure_buf(c, &c->scratch, &c->scratch_bytes, (size_t)grid * hyd::kScratchPerSub * sizeof(double),
                  "cudaMalloc(step scratch)");
  if (rc) return rc;
  const hyd::StepArgs64 A = step_args(c, B, dUdt, amax, face_flux);
  const hyd::AMRArgs Am = hydro_amr_args(c, B, M);
  const cudaError_t e = hyd::launch_step_mixed_amr(A, Am, grid, st);
  if (e != cudaSuccess) return cuda_fail(e, "hydro_step_amr_direct");
  return HYDRO_OK;
}

extern "C" {

int hydro_create(const hydro_layout_t* L, double gamma, double omega, hydro_ctx_t** out) {
  if (!L || !out) return HYDRO_EINVAL;
  *out = nullptr;
  if ((L->N != 8 && L->N != 16) || L->ghost != hyd::G || L->n_species < 1) return HYDRO_EINVAL;
  if (L->n_species != 1) return HYDRO_EUNSUP;
  if (!(gamma > 1.0) || !std::isfinite(gamma) || !std::isfinite(omega)) return HYDRO_EINVAL;
  hydro_ctx* c = new (std::nothrow) hydro_ctx();
  if (!c) return HYDRO_ENOMEM;
  c->N = L->N;
  c->G = L->ghost;
  c->n_species = L->n_species;
  c->F = 9 + L->n_species;
  c->gamma = gamma;
  c->omega = omega;
  c->mode.precision = HYDRO_PREC_FP64;
  c->mode.cfl = 0.4;
  c->mode.de_eta1 = 1e-3;
  c->mode.de_eta2 = 0.1;
  c->mode.flux_points = 9;
  c->mode.contact = 0;
  c->mode.spin = 0;
  cudaError_t e = cudaGetDevice(&c->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
  if (e != cudaSuccess) {
    delete c;
    return cuda_fail(e, "hydro_create");
  }
  *out = c;
  return HYDRO_OK;
}

int hydro_set_mode(hydro_ctx_t* c, const hydro_mode_t* m) {
  if (!c || !m) return HYDRO_EINVAL;
  if (m->precision != HYDRO_PREC_FP64 && m->precision != HYDRO_PREC_MIXED) return HYDRO_EINVAL;
  if (!(m->cfl > 0.0 && m->cfl <= 1.0) || !(m->de_eta1 > 0.0 && m->de_eta1 <= 1.0) ||
      !(m->de_eta2 > 0.0 && m->de_eta2 <= 1.0))
    return HYDRO_EINVAL;
  if (m->flux_points != 0 && m->flux_points != 1 && m->flux_points != 9) return HYDRO_EINVAL;
  if (m->contact != 0 && m->contact != 1) return HYDRO_EINVAL;
  if (m->spin != 0 && m->spin != 1) return HYDRO_EINVAL;
  c->mode = *m;
  if (c->mode.flux_points == 0) c->mode.flux_points = 9;
  return HYDRO_OK;
}

int hydro_step(hydro_ctx_t* c, const hydro_batch_t* B, double dt, double* dUdt, double* amax, double* face_flux,
               void* stream) {
  if (!c || !B) return HYDRO_EINVAL;
  if (B->n_sub < 0 || !std::isfinite(dt) || dt < 0.0) return HYDRO_EINVAL;
  if (B->n_sub == 0) return HYDRO_OK;
  if (!B->U || !B->origin || !B->h || !dUdt || !amax) return HYDRO_EINVAL;
  if (!aligned16(B->U) || !aligned16(dUdt)) return HYDRO_EINVAL;
  const bool mixed = c->mode.precision == HYDRO_PREC_MIXED;
  int rc = ensure_status(c);
  if (rc) return rc;
  const int slots = step_slots(c, mixed);
  const int units = step_units(c, B->n_sub);
  const int grid = units < slots ? units : slots;
  rc = ensure_buf(c, &c->scratch, &c->scratch_bytes, (size_t)grid * hyd::kScratchPerSub * sizeof(double),
                  "cudaMalloc(step scratch)");
  if (rc) return rc;
  if (!mixed) {
    rc = ensure_lines(c, units);
    if (rc) return rc;
  }
  const hyd::StepArgs64 A = step_args(c, B, dUdt, amax, face_flux);
  cudaError_t e = mixed ? hyd::launch_step_mixed(A, grid, eff_decomp(c) == HYDRO_DECOMP_PLANES, c->N,
                                                  (cudaStream_t)stream)
                        : hyd::launch_step_fp64_lines(A, grid, c->N, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "hydro_step");
  return HYDRO_OK;
}

int hydro_autotune_step(hydro_ctx_t* c, const hydro_batch_t* B, double* dUdt, double* amax, int* slots_out,
                        void* stream) {
  if (!c || !B || B->n_sub <= 0 || !dUdt || !amax) return HYDRO_EINVAL;
  const bool mixed = c->mode.precision == HYDRO_PREC_MIXED;
  const int idx = mixed ? 1 : 0;
  int rc = hydro_ctx_prepare(c, B->n_sub);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t ee = cudaEventCreate(&e0);
  if (ee == cudaSuccess) ee = cudaEventCreate(&e1);
  if (ee != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return cuda_fail(ee, "hydro_autotune_step");
  }
  // candidates (decomposition, persistent CTAs), three timed launches each
  // after one warm-up:
  //   row sweep: whole rounds of the batch over 1, 1.5 and 2 CTAs per SM
  //     (mixed) or 1 (FP64), and the smallest grid with the same number of
  //     rounds as the largest;
  //   plane sweep (mixed without the indicator): 1 CTA per SM and the
  //     smallest grid with the same number of rounds.
  struct Cand {
    int decomp, ctas;
  };
  Cand cand[8];
  int nc = 0;
  const bool planes_ok = mixed && !c->gate_on;
  {
    const int maxs = mixed ? 2 * c->num_sms : c->num_sms;
    const int per[3] = {c->num_sms, (3 * c->num_sms) / 2, 2 * c->num_sms};
    for (int i = 0; i < 3; ++i)
      if (per[i] <= maxs) cand[nc++] = {HYDRO_DECOMP_ROWS, per[i]};
    const int units = step_units(c, B->n_sub);
    const int rounds = (units + maxs - 1) / maxs;
    cand[nc++] = {HYDRO_DECOMP_ROWS, (units + rounds - 1) / rounds};
  }
  if (planes_ok) {
    const int maxs = c->num_sms;
    cand[nc++] = {HYDRO_DECOMP_PLANES, maxs};
    const int units = step_units(c, B->n_sub);
    const int rounds = (units + maxs - 1) / maxs;
    cand[nc++] = {HYDRO_DECOMP_PLANES, (units + rounds - 1) / rounds};
  }
  const int decomp0 = c->decomp;
  float best = 1e30f;
  Cand best_c = cand[0];
  for (int i = 0; i < nc && rc == HYDRO_OK; ++i) {
    c->decomp = cand[i].decomp;
    c->slots_tuned[idx] = cand[i].ctas;
    rc = hydro_step(c, B, 0.0, dUdt, amax, nullptr, stream);
    if (rc) break;
    cudaEventRecord(e0, st);
    for (int r = 0; r < 3 && rc == HYDRO_OK; ++r) rc = hydro_step(c, B, 0.0, dUdt, amax, nullptr, stream);
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess) rc = HYDRO_ECUDA;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rc == HYDRO_OK && ms < best) {
      best = ms;
      best_c = cand[i];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc == HYDRO_OK) {
    c->decomp = mixed ? best_c.decomp : decomp0;
    c->slots_tuned[idx] = best_c.ctas;
  } else {
    c->decomp = decomp0;
    c->slots_tuned[idx] = 0;
  }
  if (slots_out) *slots_out = c->slots_tuned[idx];
  return rc;
}

int hydro_set_launch(hydro_ctx_t* c, int decomposition, int ctas) {
  if (!c || ctas < 0) return HYDRO_EINVAL;
  if (decomposition != HYDRO_DECOMP_AUTO && decomposition != HYDRO_DECOMP_ROWS &&
      decomposition != HYDRO_DECOMP_PLANES)
    return HYDRO_EINVAL;
  const bool mixed = c->mode.precision == HYDRO_PREC_MIXED;
  if (!mixed && decomposition == HYDRO_DECOMP_PLANES) return HYDRO_EUNSUP;
  if (mixed) c->decomp = decomposition;
  c->slots_tuned[mixed ? 1 : 0] = ctas;
  return HYDRO_OK;
}

int hydro_get_launch(const hydro_ctx_t* c, int* decomposition, int* ctas) {
  if (!c) return HYDRO_EINVAL;
  const bool mixed = c->mode.precision == HYDRO_PREC_MIXED;
  if (decomposition) *decomposition = eff_decomp(c);
  if (ctas) *ctas = step_slots(c, mixed);
  return HYDRO_OK;
}

int hydro_update(hydro_ctx_t* c, const hydro_batch_t* B, const double* U0, const double* dUdt, double dt,
                 const double* dt_dev, int stage, double* U_out, void* stream) {
  if (!c || !B) return HYDRO_EINVAL;
  if (stage < 0 || stage > 2 || B->n_sub < 0) return HYDRO_EINVAL;
  if (!dt_dev && (!std::isfinite(dt) || dt < 0.0)) return HYDRO_EINVAL;
  if (B->n_sub == 0) return HYDRO_OK;
  if (!B->U || !U0 || !dUdt) return HYDRO_EINVAL;
  double* out = U_out ? U_out : B->U;
  if (out != B->U) {
    // out of place: the two state buffers may not overlap
    const size_t bytes = (size_t)B->n_sub * hyd::F * padded_cells(c) * sizeof(double);
    const char *a = (const char*)B->U, *b = (const char*)out;
    if (a < b + bytes && b < a + bytes) return HYDRO_EINVAL;
  }
  cudaError_t e = hyd::launch_update(B->U, out, U0, dUdt, dt, dt_dev, stage, c->mode.de_eta2, c->gamma, B->n_sub,
                                     c->mode.precision == HYDRO_PREC_MIXED, c->num_sms, c->N, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "hydro_update");
  return HYDRO_OK;
}

int hydro_dt(hydro_ctx_t* c, const double* amax, const double* h, int n_sub, double cfl, double* dt_out,
             void* stream) {
  if (!c || !amax || !h || !dt_out || n_sub <= 0) return HYDRO_EINVAL;
  if (!(cfl > 0.0)) cfl = c->mode.cfl;
  cudaError_t e = hyd::launch_dt(amax, h, n_sub, cfl, dt_out, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "hydro_dt");
  return HYDRO_OK;
}

int hydro_fill_ghosts_uniform(hydro_ctx_t* c, const hydro_batch_t* B, int nbx, int nby, int nbz, int bc,
                              void* stream) {
  if (!c || !B || !B->U) return HYDRO_EINVAL;
  if (nbx <= 0 || nby <= 0 || nbz <= 0 || (long)nbx * nby * nbz != B->n_sub) return HYDRO_EINVAL;
  if (bc != HYDRO_BC_PERIODIC && bc != HYDRO_BC_OUTFLOW) return HYDRO_EINVAL;
  cudaError_t e = hyd::launch_ghost_uniform(B->U, nbx, nby, nbz, bc, c->num_sms, c->N, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "hydro_fill_ghosts_uniform");
  return HYDRO_OK;
}

// The address at which a kernel reaches buffer p: device or managed memory as
// is; page-locked host memory through its device mapping (with unified
// addressing every cudaHostAlloc'd or registered buffer has one, and the
// kernel's loads and stores then cross the host link directly); null for
// pageable host memory, which no kernel may touch.
static double* device_view(const double* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();  // clear the sticky-free error of the query
    return nullptr;
  }
  switch (at.type) {
    case cudaMemoryTypeDevice:
    case cudaMemoryTypeManaged:
      return const_cast<double*>(p);
    case cudaMemoryTypeHost:
      return static_cast<double*>(at.devicePointer);
    default:
      return nullptr;
  }
}

static int interior_copy(hydro_ctx_t* c, const hydro_batch_t* B, const double* I, bool scatter, void* stream) {
  if (!c || !B || B->n_sub < 0) return HYDRO_EINVAL;
  if (B->n_sub == 0) return HYDRO_OK;
  if (!B->U || !I) return HYDRO_EINVAL;
  double* Id = device_view(I);
  if (!Id || !aligned16(Id)) return HYDRO_EINVAL;
  cudaError_t e = hyd::launch_interior(B->U, Id, B->n_sub, scatter, c->num_sms, c->N, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, scatter ? "hydro_scatter_interior" : "hydro_gather_interior");
  return HYDRO_OK;
}

int hydro_scatter_interior(hydro_ctx_t* c, const hydro_batch_t* B, const double* interior, void* stream) {
  return interior_copy(c, B, interior, true, stream);
}

int hydro_gather_interior(hydro_ctx_t* c, const hydro_batch_t* B, double* interior, void* stream) {
  return interior_copy(c, B, interior, false, stream);
}

int hydro_conserved_sums(hydro_ctx_t* c, const hydro_batch_t* B, double* sums, void* stream) {
  if (!c || !B || !sums || B->n_sub <= 0 || !B->U || !B->origin || !B->h) return HYDRO_EINVAL;
  int rc = ensure_buf(c, &c->part, &c->part_bytes, (size_t)B->n_sub * (hyd::F + 1) * sizeof(double),
                      "cudaMalloc(sum partials)");
  if (rc) return rc;
  cudaError_t e = hyd::launch_sums(B->U, B->origin, B->h, B->n_sub, c->part, sums, c->N, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "hydro_conserved_sums");
  return HYDRO_OK;
}

int hydro_status(hydro_ctx_t* c, uint32_t* flags) {
  if (!c || !flags) return HYDRO_EINVAL;
  *flags = 0;
  if (!c->status) return HYDRO_OK;
  unsigned v = 0;
  cudaError_t e = cudaMemcpy(&v, c->status, sizeof v, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "hydro_status");
  e = cudaMemset(c->status, 0, sizeof(unsigned));
  if (e != cudaSuccess) return cuda_fail(e, "hydro_status");
  *flags = v;
  return HYDRO_OK;
}

const char* hydro_strerror(int code) {
  switch (code) {
    case HYDRO_OK: return "success";
    case HYDRO_EINVAL: return "invalid argument (layout, size, pointer, alignment or value)";
    case HYDRO_ECUDA: return "CUDA error (see hydro_last_cuda_error)";
    case HYDRO_ENOMEM: return "device scratch allocation failed";
    case HYDRO_EUNSUP: return "unsupported configuration";
    case HYDRO_ERANGE: return "batch larger than the fixed scratch of hydro_step_static (HYDRO_STATIC_MAX_SUB)";
    default: return "unknown error code";
  }
}

const char* hydro_last_cuda_error(void) { return g_cuda_err; }

void hydro_destroy(hydro_ctx_t* c) {
  if (!c) return;
  if (c->status) cudaFree(c->status);
  if (c->scratch) cudaFree(c->scratch);
  if (c->lines) cudaFree(c->lines);
  if (c->part) cudaFree(c->part);
  if (c->gate_w) cudaFree(c->gate_w);
  if (c->u2) cudaFree(c->u2);
  if (c->prims) cudaFree(c->prims);
  if (c->sync) cudaFree(c->sync);
  if (c->amr_img) cudaFree(c->amr_img);
  if (c->amr_finer) cudaFree(c->amr_finer);
  for (void* p : c->retired) cudaFree(p);
  delete c;
}

}  // extern "C"
