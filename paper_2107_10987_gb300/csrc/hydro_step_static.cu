// hydro_step_static.cu -- hydro_step without any device allocation.
//
// Some callers cannot call cudaMalloc: a host code that hands all device
// memory to its own pool allocator and forbids allocations behind its back,
// or a time-stepping loop that cannot afford the device-wide synchronisation
// a cudaMalloc may imply.  hydro_step_static runs the same FP64 step kernel
// as hydro_step, but its per-sub-grid scratch lives in a fixed array of this
// library's device code instead of a buffer the context allocates.
//
// The array holds HYDRO_STATIC_MAX_SUB sub-grid slots of kScratchPerSub
// doubles (192 x 159,744 B = 30.7 MB on every GPU that loads the library,
// kept until the process exits).  A call with more sub-grids is rejected
// with HYDRO_ERANGE; callers split larger batches.  Every call uses the same
// array and leaves its contents behind: the kernel writes every scratch
// element it reads before reading it, so nothing needs clearing, but two
// calls whose kernels overlap on the GPU (different streams, no ordering
// between them) race on the array and give wrong results.
//
// Set-up: the first call on a device, with that device current, loads the
// device code and looks the array's address up with cudaGetSymbolAddress
// (the host-side name of the array is only a stand-in, not a device
// address).  Make that first call before any stream capture.
#include <cmath>
#include <mutex>

#include "hydro.h"
#include "hydro_common.cuh"
#include "hydro_ctx.h"

namespace hyd {
cudaError_t launch_step_fp64(const StepArgs64& A, int grid, int nn, cudaStream_t st);
}

namespace {

static __device__ __align__(256) double g_step_scratch[(size_t)HYDRO_STATIC_MAX_SUB * hyd::kScratchPerSub];
static __device__ __align__(256) unsigned g_step_status[1];

constexpr int kMaxDevices = 64;
struct DeviceAddrs {
  bool ready;
  double* scratch;
  unsigned* status;
};
DeviceAddrs g_addrs[kMaxDevices];
std::mutex g_mu;

int addrs_for_current_device(DeviceAddrs* out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return HYDRO_ECUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  DeviceAddrs& a = g_addrs[dev];
  if (!a.ready) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_step_scratch);
    if (e != cudaSuccess) return HYDRO_ECUDA;
    a.scratch = static_cast<double*>(p);
    e = cudaGetSymbolAddress(&p, g_step_status);
    if (e != cudaSuccess) return HYDRO_ECUDA;
    a.status = static_cast<unsigned*>(p);
    a.ready = true;
  }
  *out = a;
  return HYDRO_OK;
}

}  // namespace

// Declared in hydro.h; see there for the contract.
extern "C" int hydro_step_static(hydro_ctx_t* c, const hydro_batch_t* B, double dt, double* dUdt, double* amax,
                                 uint32_t* status, void* stream) {
  if (!c || !B) return HYDRO_EINVAL;
  if (B->n_sub < 0 || !std::isfinite(dt) || dt < 0.0) return HYDRO_EINVAL;
  if (B->n_sub > HYDRO_STATIC_MAX_SUB) return HYDRO_ERANGE;
  if (B->n_sub == 0) return HYDRO_OK;
  if (!B->U || !B->origin || !B->h || !dUdt || !amax) return HYDRO_EINVAL;
  if ((((uintptr_t)B->U) & 15u) || (((uintptr_t)dUdt) & 15u)) return HYDRO_EINVAL;
  if (c->mode.precision != HYDRO_PREC_FP64 || c->N != hyd::N) return HYDRO_EUNSUP;
  DeviceAddrs a;
  int rc = addrs_for_current_device(&a);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  unsigned* word = status ? reinterpret_cast<unsigned*>(status) : a.status;
  // the status bits of this call start at zero
  if (cudaMemsetAsync(word, 0, sizeof(unsigned), st) != cudaSuccess) return HYDRO_ECUDA;
  hyd::StepArgs64 A;
  A.U = B->U;
  A.origin = B->origin;
  A.h = B->h;
  A.g = B->g;
  A.dUdt = dUdt;
  A.amax = amax;
  A.face_flux = nullptr;
  A.scratch = a.scratch;  // one slot per CTA, one CTA per sub-grid
  A.lines = nullptr;      // the axis-sweep kernel keeps its lines on chip
  A.status = word;
  A.n_sub = B->n_sub;
  A.P.gamma = c->gamma;
  A.P.gm1 = c->gamma - 1.0;
  A.P.omega = c->omega;
  A.P.eta1 = c->mode.de_eta1;
  A.P.face_points = c->mode.flux_points == 1 ? 1 : 9;
  A.P.spin = c->mode.spin ? 1 : 0;
  A.P.contact = c->mode.contact ? 1 : 0;
  // the learned indicator as the context has it (its parameters are the
  // context's own device copy, made by hydro_set_indicator)
  A.gate = c->gate_on ? 1 : 0;
  A.gate_w = c->gate_w;
  A.gate_logit_thr = (float)c->gate_logit_thr;
  A.gate_zero_smooth = c->gate_zero_smooth;
  if (hyd::launch_step_fp64(A, B->n_sub, hyd::N, st) != cudaSuccess) return HYDRO_ECUDA;
  return HYDRO_OK;
}
