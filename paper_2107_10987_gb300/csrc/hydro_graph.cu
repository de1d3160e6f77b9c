// hydro_graph.cu -- a whole RK3 time step of a mesh (uniform, or adaptive with
// its two-pass ghost fill and coarse-fine flux correction) as a sequence of
// launches on one stream, and the same sequence captured once into CUDA
// graphs that are replayed step after step.
//
// One time step (three hydro iterations, Sec. IV-A.2), state X -> Y (the
// fused form, one persistent launch for a uniform mesh in mixed precision,
// is in hydro_rk3_fused.cu):
//   ghost(X); step(X) -> dU, amax; dt = cfl min h/amax; Y = X + dt dU
//   ghost(Y); step(Y);            Y = 3/4 X + 1/4 (Y + dt dU)
//   ghost(Y); step(Y);            Y = 1/3 X + 2/3 (Y + dt dU)
// The first update writes the second buffer, so the step's initial state X
// is kept without a copy; the next step runs Y -> X.  Two graphs (X->Y and
// Y->X) are instantiated and replayed alternately.
// On an adaptive mesh in mixed precision (8^3 leaves, row sweep, no contact
// steepening or spin feedback) the ghost fill is the lean one and the step
// reads same-level and finer neighbours itself (hydro_step_mixed_amr.cu):
// the same values, bit for bit, without copying them into ghost cells.
#include <cmath>
#include <new>

#include "hydro.h"
#include "hydro_common.cuh"
#include "hydro_ctx.h"

struct hydro_graph {
  hydro_ctx_t* ctx;
  hydro_rk3_desc_t d;
  cudaStream_t cap;
  cudaGraph_t graph[2];
  cudaGraphExec_t exec[2];
  int parity;  // 0: current state in d.a.U, 1: in d.U_b
};

static int rk3_enqueue(hydro_ctx_t* ctx, const hydro_rk3_desc_t* d, int parity, cudaStream_t st) {
  if (d->fused) return hydro_rk3_fused_enqueue(ctx, d, parity, st);
  hydro_batch_t X = d->a, Y = d->a;
  if (parity) X.U = d->U_b;
  else Y.U = d->U_b;
  int rc;
  for (int k = 0; k < 3; ++k) {
    const hydro_batch_t* B = (k == 0) ? &X : &Y;
    if (d->amr && hydro_amr_direct_ok(ctx)) {
      // the first stage restricts its state; the updates of the first two
      // write the next state's restriction images
      if ((rc = hydro_ctx_prepare_amr(ctx, B->n_sub))) return rc;
      if ((rc = hydro_fill_ghosts_amr_lean(ctx, B, d->amr, k == 0, st))) return rc;
      if ((rc = hydro_step_amr_direct(ctx, B, d->amr, d->dUdt, d->amax, d->face_flux, st))) return rc;
      if (k == 0 && (rc = hydro_dt(ctx, d->amax, d->a.h, d->a.n_sub, d->cfl, d->dt, st))) return rc;
      if ((rc = hydro_update_amr_lean(ctx, B, d->amr, X.U, d->dUdt, d->face_flux, d->dt, k,
                                      k == 0 ? Y.U : B->U, k < 2, st)))
        return rc;
      continue;
    } else if (d->amr) {
      if ((rc = hydro_fill_ghosts_amr(ctx, B, d->amr, st))) return rc;
      if ((rc = hydro_step(ctx, B, 0.0, d->dUdt, d->amax, d->face_flux, st))) return rc;
      if ((rc = hydro_flux_correct_amr(ctx, B, d->amr, d->face_flux, d->dUdt, st))) return rc;
    } else {
      if ((rc = hydro_fill_ghosts_uniform(ctx, B, d->nbx, d->nby, d->nbz, d->bc, st))) return rc;
      if ((rc = hydro_step(ctx, B, 0.0, d->dUdt, d->amax, nullptr, st))) return rc;
    }
    if (k == 0 && (rc = hydro_dt(ctx, d->amax, d->a.h, d->a.n_sub, d->cfl, d->dt, st))) return rc;
    if ((rc = hydro_update(ctx, B, X.U, d->dUdt, 0.0, d->dt, k, k == 0 ? Y.U : nullptr, st))) return rc;
  }
  return HYDRO_OK;
}

static bool desc_ok(const hydro_ctx_t* ctx, const hydro_rk3_desc_t* d) {
  if (!(d && d->a.U && d->U_b && d->a.origin && d->a.h && d->dUdt && d->amax && d->dt && d->a.n_sub > 0))
    return false;
  // the two state buffers may not overlap: each stage reads one and writes the other
  const size_t sp = (size_t)ctx->N + 2 * hyd::G;
  const size_t bytes = (size_t)d->a.n_sub * hyd::F * sp * sp * sp * sizeof(double);
  const char *a = (const char*)d->a.U, *b = (const char*)d->U_b;
  if (a < b + bytes && b < a + bytes) return false;
  if (d->amr) return d->face_flux != nullptr;
  return (long)d->nbx * d->nby * d->nbz == d->a.n_sub;
}

extern "C" {

int hydro_rk3_step(hydro_ctx_t* ctx, const hydro_rk3_desc_t* d, int parity, void* stream) {
  if (!ctx || !desc_ok(ctx, d) || (parity != 0 && parity != 1)) return HYDRO_EINVAL;
  return rk3_enqueue(ctx, d, parity, (cudaStream_t)stream);
}

int hydro_rk3_graph_create(hydro_ctx_t* ctx, const hydro_rk3_desc_t* d, hydro_graph_t** out) {
  if (!ctx || !out || !desc_ok(ctx, d)) return HYDRO_EINVAL;
  *out = nullptr;
  hydro_graph* g = new (std::nothrow) hydro_graph();
  if (!g) return HYDRO_ENOMEM;
  g->ctx = ctx;
  g->d = *d;
  cudaError_t e = cudaStreamCreateWithFlags(&g->cap, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    delete g;
    return HYDRO_ECUDA;
  }
  // everything the launches need is allocated before the capture
  int rc = d->fused ? hydro_ctx_prepare_fused(ctx, d->a.n_sub)
           : (d->amr && hydro_amr_direct_ok(ctx)) ? hydro_ctx_prepare_amr(ctx, d->a.n_sub)
                                                   : hydro_ctx_prepare(ctx, d->a.n_sub);
  for (int p = 0; p < 2 && rc == HYDRO_OK; ++p) {
    if (cudaStreamBeginCapture(g->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      rc = HYDRO_ECUDA;
      break;
    }
    const int r2 = rk3_enqueue(ctx, d, p, g->cap);
    cudaGraph_t gr = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(g->cap, &gr);
    if (r2 != HYDRO_OK || e2 != cudaSuccess) {
      if (gr) cudaGraphDestroy(gr);
      rc = r2 != HYDRO_OK ? r2 : HYDRO_ECUDA;
      break;
    }
    g->graph[p] = gr;
    if (cudaGraphInstantiate(&g->exec[p], gr, 0) != cudaSuccess) rc = HYDRO_ECUDA;
  }
  if (rc != HYDRO_OK) {
    hydro_rk3_graph_destroy(g);
    return rc;
  }
  g->parity = 0;
  ctx->had_graph = true;  // from now on the context keeps grown-out buffers
  *out = g;
  return HYDRO_OK;
}

int hydro_rk3_graph_launch(hydro_graph_t* g, void* stream) {
  if (!g) return HYDRO_EINVAL;
  if (cudaGraphLaunch(g->exec[g->parity], (cudaStream_t)stream) != cudaSuccess) return HYDRO_ECUDA;
  g->parity ^= 1;
  return HYDRO_OK;
}

int hydro_rk3_graph_state(const hydro_graph_t* g) { return g ? g->parity : HYDRO_EINVAL; }

void hydro_rk3_graph_destroy(hydro_graph_t* g) {
  if (!g) return;
  for (int p = 0; p < 2; ++p) {
    if (g->exec[p]) cudaGraphExecDestroy(g->exec[p]);
    if (g->graph[p]) cudaGraphDestroy(g->graph[p]);
  }
  if (g->cap) cudaStreamDestroy(g->cap);
  delete g;
}

}  // extern "C"
