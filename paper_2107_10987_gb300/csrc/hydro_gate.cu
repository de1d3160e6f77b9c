// hydro_gate.cu -- the learned smoothness indicator: training data from the
// method itself (features and limiter-activity labels per cell), and the
// forward, backward and Adam kernels that train the network on the GPU.
//
// Network: 54 -> 32 (ReLU) -> 32 (ReLU) -> 1 (sigmoid).  The master
// parameters are FP32; every forward and backward pass uses them rounded to
// BF16 (the storage precision of the deployed indicator) and accumulates in
// FP32.  Loss: class-weighted binary cross-entropy, mean over the samples.
#include <cuda_bf16.h>

#include <cstdint>

#include "hydro.h"
#include "hydro_ctx.h"
#include "hydro_mixed.cuh"

namespace hyd {

// Significant limiter activity on one line of one field: the limited pair
// differs from the central-slope pair (Delta_j = (delta_{j-1}+delta_j)/2, no
// fix-ups) by more than 1e-4 of the field's scale at the cell.
constexpr float kLabelTol = 1e-4f;

__device__ __forceinline__ bool ppm32_significant(float s0, float s1, float s2, float s3, float s4, float scale) {
  float qp, qm;
  ppm32(s0, s1, s2, s3, s4, qp, qm);
  const float sixth = 1.f / 6.f;
  const float d0 = s1 - s0, d1 = s2 - s1, d2 = s3 - s2, d3 = s4 - s3;
  const float C0 = 0.5f * (d0 + d1), C1 = 0.5f * (d1 + d2), C2 = 0.5f * (d2 + d3);
  const float pu = 0.5f * (s2 + s3) - (C2 - C1) * sixth;
  const float mu = 0.5f * (s1 + s2) - (C1 - C0) * sixth;
  return fmaxf(fabsf(qp - pu), fabsf(qm - mu)) > kLabelTol * scale;
}

struct GateDataArgs {
  const double* U;
  float* X;       // [n_sub*N3][54] or null
  uint8_t* y;     // [n_sub*N3] or null
  int n_sub;
  double eta1;
  float gamma, gm1;
};

__global__ void __launch_bounds__(256, 2) hydro_gate_data_kernel(GateDataArgs A) {
  extern __shared__ __align__(128) float Qf[];
  for (int s = blockIdx.x; s < A.n_sub; s += gridDim.x) {
    const double* Us = A.U + (size_t)s * F * S3;
    for (int c = threadIdx.x; c < S3; c += blockDim.x) {
      double u[F];
#pragma unroll
      for (int k = 0; k < F; ++k) u[k] = __ldg(Us + (size_t)k * S3 + c);
      float q[F];
      prims_mixed(u, A.eta1, A.gamma, q);
#pragma unroll
      for (int k = 0; k < F; ++k) Qf[k * S3 + c] = q[k];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < N3; i += blockDim.x) {
      const int x = i & (N - 1), yy = (i >> 3) & (N - 1), z = i >> 6;
      const int c = ((z + G) * S + (yy + G)) * S + (x + G);
      const size_t cell = (size_t)s * N3 + i;
      if (A.X) {
        float f[54];
        gate_features(Qf, c, A.gm1, f);
#pragma unroll
        for (int k = 0; k < 54; ++k) A.X[cell * 54 + k] = f[k];
      }
      if (A.y) {
        bool fired = false;
        // scales: |q0| for density, eps, tau, species; |v| + c for velocity
        const float rho0 = Qf[RHO * S3 + c], eps0 = Qf[EGAS * S3 + c];
        const float vs = fabsf(Qf[SX * S3 + c]) + fabsf(Qf[SY * S3 + c]) + fabsf(Qf[SZ * S3 + c]) +
                         sqrtf(A.gamma * A.gm1 * eps0 / rho0);
        // the 13 lines through the cell: d with first non-zero component > 0
#pragma unroll 1
        for (int dz = 0; dz <= 1; ++dz)
#pragma unroll 1
          for (int dy = -1; dy <= 1; ++dy)
#pragma unroll 1
            for (int dx = -1; dx <= 1; ++dx) {
              if (dz == 0 && (dy < 0 || (dy == 0 && dx <= 0))) continue;
              const int st = (dz * S + dy) * S + dx;
#pragma unroll
              for (int k = 0; k < F; ++k) {
                if (k == ZX || k == ZY || k == ZZ) continue;  // spin: always limited, never labelled
                const float* q = Qf + k * S3 + c;
                const float scale = (k >= SX && k <= SZ) ? vs : fabsf(q[0]);
                fired |= ppm32_significant(q[-2 * st], q[-st], q[0], q[st], q[2 * st], scale);
              }
            }
        A.y[cell] = fired ? 1 : 0;
      }
    }
    __syncthreads();
  }
}

// ---- MLP training ----------------------------------------------------------
constexpr int kTile = 128;

struct SmemW {
  const float* w;
  __device__ float operator()(int i) const { return w[i]; }
};

// Forward only, in the deployed form (BF16 inputs and first hidden layer,
// FP32 accumulation; gate_logit_infer): out[i] = sigmoid(logit(x_i)).
__global__ void __launch_bounds__(kTile) hydro_mlp_forward_kernel(const float* params, const float* X, int n,
                                                                  float* out) {
  __shared__ float w[kGateParams];
  for (int i = threadIdx.x; i < kGateParams; i += blockDim.x) w[i] = bf16r(params[i]);
  __syncthreads();
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    float x[54];
#pragma unroll
    for (int k = 0; k < 54; ++k) x[k] = X[(size_t)t * 54 + k];
    const float z = gate_logit_infer(SmemW{w}, x);
    out[t] = 1.f / (1.f + __expf(-z));
  }
}

// Loss and gradient of one tile of kTile samples; per-tile partial sums
// (kGateParams gradient entries, then the loss) in a fixed order.
__global__ void __launch_bounds__(kTile) hydro_mlp_grad_kernel(const float* params, const float* X, const float* y,
                                                               int n, float w1, float w0, float inv_n,
                                                               float* partial) {
  extern __shared__ __align__(16) float sm[];
  float* w = sm;                               // kGateParams
  float* xs = w + kGateParams + 3;             // [kTile][54]
  float* h1s = xs + kTile * kGateIn;           // [kTile][32]
  float* h2s = h1s + kTile * kGateH;           // [kTile][32]
  float* g1s = h2s + kTile * kGateH;           // dL/dz1 [kTile][32]
  float* g2s = g1s + kTile * kGateH;           // dL/dz2 [kTile][32]
  float* g3s = g2s + kTile * kGateH;           // dL/dz3 [kTile]
  float* ls = g3s + kTile;                     // loss terms [kTile]
  for (int i = threadIdx.x; i < kGateParams; i += blockDim.x) w[i] = bf16r(params[i]);
  __syncthreads();
  const int t = threadIdx.x;
  const int sidx = blockIdx.x * kTile + t;
  const int oW2 = kGateH * kGateIn + kGateH, ob2 = oW2 + kGateH * kGateH, ow3 = ob2 + kGateH, ob3 = ow3 + kGateH;
  {
    float x[54];
    const bool live = sidx < n;
#pragma unroll
    for (int k = 0; k < 54; ++k) {
      x[k] = live ? X[(size_t)sidx * 54 + k] : 0.f;
      xs[t * kGateIn + k] = x[k];
    }
    float z1[kGateH], h1[kGateH], z2[kGateH];
#pragma unroll
    for (int j = 0; j < kGateH; ++j) {
      float z = w[kGateH * kGateIn + j];
#pragma unroll
      for (int i = 0; i < kGateIn; ++i) z = fmaf(w[j * kGateIn + i], x[i], z);
      z1[j] = z;
      h1[j] = fmaxf(z, 0.f);
      h1s[t * kGateH + j] = h1[j];
    }
    float z3 = w[ob3];
#pragma unroll
    for (int j = 0; j < kGateH; ++j) {
      float z = w[ob2 + j];
#pragma unroll
      for (int i = 0; i < kGateH; ++i) z = fmaf(w[oW2 + j * kGateH + i], h1[i], z);
      z2[j] = z;
      const float h2 = fmaxf(z, 0.f);
      h2s[t * kGateH + j] = h2;
      z3 = fmaf(w[ow3 + j], h2, z3);
    }
    const float out = 1.f / (1.f + __expf(-z3));
    const float yy = live ? y[sidx] : 0.f;
    // -[w1 y log(out) + w0 (1-y) log(1-out)] with log(out) = -softplus(-z3)
    const float sp_neg = fmaxf(-z3, 0.f) + log1pf(__expf(-fabsf(z3)));  // softplus(-z3)
    const float sp_pos = sp_neg + z3;                                   // softplus(z3)
    ls[t] = live ? (w1 * yy * sp_neg + w0 * (1.f - yy) * sp_pos) * inv_n : 0.f;
    const float g3 = live ? (w1 * yy * (out - 1.f) + w0 * (1.f - yy) * out) * inv_n : 0.f;
    g3s[t] = g3;
    float gh1[kGateH];
#pragma unroll
    for (int i = 0; i < kGateH; ++i) gh1[i] = 0.f;
#pragma unroll
    for (int j = 0; j < kGateH; ++j) {
      const float g2 = (z2[j] > 0.f) ? g3 * w[ow3 + j] : 0.f;
      g2s[t * kGateH + j] = g2;
#pragma unroll
      for (int i = 0; i < kGateH; ++i) gh1[i] = fmaf(g2, w[oW2 + j * kGateH + i], gh1[i]);
    }
#pragma unroll
    for (int i = 0; i < kGateH; ++i) g1s[t * kGateH + i] = (z1[i] > 0.f) ? gh1[i] : 0.f;
  }
  __syncthreads();
  // weight gradients: sums over the tile's samples in index order
  float* out = partial + (size_t)blockIdx.x * (kGateParams + 1);
  for (int p = threadIdx.x; p < kGateParams + 1; p += blockDim.x) {
    float acc = 0.f;
    if (p < kGateH * kGateIn) {
      const int j = p / kGateIn, i = p % kGateIn;
      for (int s = 0; s < kTile; ++s) acc = fmaf(g1s[s * kGateH + j], xs[s * kGateIn + i], acc);
    } else if (p < oW2) {
      const int j = p - kGateH * kGateIn;
      for (int s = 0; s < kTile; ++s) acc += g1s[s * kGateH + j];
    } else if (p < ob2) {
      const int j = (p - oW2) / kGateH, i = (p - oW2) % kGateH;
      for (int s = 0; s < kTile; ++s) acc = fmaf(g2s[s * kGateH + j], h1s[s * kGateH + i], acc);
    } else if (p < ow3) {
      const int j = p - ob2;
      for (int s = 0; s < kTile; ++s) acc += g2s[s * kGateH + j];
    } else if (p < ob3) {
      const int j = p - ow3;
      for (int s = 0; s < kTile; ++s) acc = fmaf(g3s[s], h2s[s * kGateH + j], acc);
    } else if (p == ob3) {
      for (int s = 0; s < kTile; ++s) acc += g3s[s];
    } else {
      for (int s = 0; s < kTile; ++s) acc += ls[s];
    }
    out[p] = acc;
  }
}

__global__ void hydro_mlp_reduce_kernel(const float* partial, int n_tiles, float* grad, float* loss) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p > kGateParams) return;
  float acc = 0.f;
  for (int b = 0; b < n_tiles; ++b) acc += partial[(size_t)b * (kGateParams + 1) + p];
  if (p < kGateParams) grad[p] = acc;
  else if (loss) *loss = acc;
}

__global__ void hydro_mlp_adam_kernel(float* params, float* m, float* v, const float* grad, float lr, float bc1,
                                      float bc2) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= kGateParams) return;
  const float g = grad[p];
  const float mm = 0.9f * m[p] + 0.1f * g, vv = 0.999f * v[p] + 0.001f * g * g;
  m[p] = mm;
  v[p] = vv;
  params[p] -= lr * (mm / bc1) / (sqrtf(vv / bc2) + 1e-8f);
}

// Logit of the network at all-zero features (parameters already rounded).
__global__ void hydro_gate_zero_kernel(const float* w, float* out) {
  float x[54];
#pragma unroll
  for (int k = 0; k < 54; ++k) x[k] = 0.f;
  out[0] = gate_logit_infer(SmemW{w}, x);
}

__global__ void hydro_bf16_round_kernel(const float* in, float* out, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = bf16r(in[i]);
}

size_t mlp_grad_smem() {
  return sizeof(float) * (kGateParams + 3 + kTile * kGateIn + 4 * kTile * kGateH + 2 * kTile);
}

}  // namespace hyd

extern "C" {

int hydro_gate_data(hydro_ctx_t* c, const hydro_batch_t* B, float* X, uint8_t* y, void* stream) {
  if (!c || !B || B->n_sub < 0 || (!X && !y)) return HYDRO_EINVAL;
  if (c->N != hyd::N) return HYDRO_EUNSUP;
  if (B->n_sub == 0) return HYDRO_OK;
  if (!B->U) return HYDRO_EINVAL;
  const size_t smem = (size_t)hyd::F * hyd::S3 * sizeof(float);
  static unsigned long long attr = 0;
  if (hyd::once_per_device(&attr, [smem] {
        return cudaFuncSetAttribute(hyd::hydro_gate_data_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem);
      }) != cudaSuccess)
    return HYDRO_ECUDA;
  hyd::GateDataArgs A{B->U, X, y, B->n_sub, c->mode.de_eta1, (float)c->gamma, (float)(c->gamma - 1.0)};
  const int grid = B->n_sub < 2 * c->num_sms ? B->n_sub : 2 * c->num_sms;
  hyd::hydro_gate_data_kernel<<<grid, 256, smem, (cudaStream_t)stream>>>(A);
  return cudaGetLastError() == cudaSuccess ? HYDRO_OK : HYDRO_ECUDA;
}

int hydro_mlp_forward(const float* params, const float* X, int n, float* out, void* stream) {
  if (!params || n < 0 || (n > 0 && (!X || !out))) return HYDRO_EINVAL;
  if (n == 0) return HYDRO_OK;
  int blocks = (n + hyd::kTile - 1) / hyd::kTile;
  if (blocks > 4096) blocks = 4096;
  hyd::hydro_mlp_forward_kernel<<<blocks, hyd::kTile, 0, (cudaStream_t)stream>>>(params, X, n, out);
  return cudaGetLastError() == cudaSuccess ? HYDRO_OK : HYDRO_ECUDA;
}

size_t hydro_mlp_work_bytes(int n) {
  const size_t tiles = (size_t)((n > 0 ? n : 0) + hyd::kTile - 1) / hyd::kTile;
  return tiles * (hyd::kGateParams + 1) * sizeof(float);
}

int hydro_mlp_loss_grad(const float* params, const float* X, const float* y, int n, float w1, float w0, float* grad,
                        float* loss, void* work_v, size_t work_bytes, void* stream) {
  float* work = static_cast<float*>(work_v);
  if (!params || !X || !y || !grad || !work || n <= 0) return HYDRO_EINVAL;
  if (work_bytes < hydro_mlp_work_bytes(n)) return HYDRO_EINVAL;
  static unsigned long long attr = 0;
  if (hyd::once_per_device(&attr, [] {
        return cudaFuncSetAttribute(hyd::hydro_mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)hyd::mlp_grad_smem());
      }) != cudaSuccess)
    return HYDRO_ECUDA;
  const int tiles = (n + hyd::kTile - 1) / hyd::kTile;
  cudaStream_t st = (cudaStream_t)stream;
  hyd::hydro_mlp_grad_kernel<<<tiles, hyd::kTile, hyd::mlp_grad_smem(), st>>>(params, X, y, n, w1, w0, 1.f / n,
                                                                             work);
  hyd::hydro_mlp_reduce_kernel<<<(hyd::kGateParams + 1 + 255) / 256, 256, 0, st>>>(work, tiles, grad, loss);
  return cudaGetLastError() == cudaSuccess ? HYDRO_OK : HYDRO_ECUDA;
}

int hydro_mlp_adam(float* params, float* m, float* v, const float* grad, int t, float lr, void* stream) {
  if (!params || !m || !v || !grad || t < 1 || !(lr > 0.f)) return HYDRO_EINVAL;
  const float bc1 = 1.f - powf(0.9f, (float)t), bc2 = 1.f - powf(0.999f, (float)t);
  hyd::hydro_mlp_adam_kernel<<<(hyd::kGateParams + 255) / 256, 256, 0, (cudaStream_t)stream>>>(params, m, v, grad, lr,
                                                                                               bc1, bc2);
  return cudaGetLastError() == cudaSuccess ? HYDRO_OK : HYDRO_ECUDA;
}

int hydro_set_indicator(hydro_ctx_t* c, const float* params, double threshold, void* stream) {
  if (!c) return HYDRO_EINVAL;
  if (!params) {
    c->gate_on = 0;
    return HYDRO_OK;
  }
  if (!(threshold > 0.0 && threshold < 1.0)) return HYDRO_EINVAL;
  int rc = HYDRO_OK;
  if (!c->gate_w) {
    if (cudaMalloc(&c->gate_w, hyd::kGateParams * sizeof(float)) != cudaSuccess) return HYDRO_ENOMEM;
  }
  cudaStream_t st = (cudaStream_t)stream;
  hyd::hydro_bf16_round_kernel<<<(hyd::kGateParams + 255) / 256, 256, 0, st>>>(params, c->gate_w, hyd::kGateParams);
  if (cudaGetLastError() != cudaSuccess) rc = HYDRO_ECUDA;
  if (rc == HYDRO_OK) {
    // the network's decision at all-zero features (a uniform neighbourhood),
    // evaluated once with the same rounded parameters and arithmetic
    float* d_zero = nullptr;
    float h_zero = 1.f;
    if (cudaMalloc(&d_zero, 2 * sizeof(float)) != cudaSuccess) return HYDRO_ENOMEM;
    hyd::hydro_gate_zero_kernel<<<1, 1, 0, st>>>(c->gate_w, d_zero);
    if (cudaMemcpyAsync(&h_zero, d_zero, sizeof(float), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      rc = HYDRO_ECUDA;
    cudaFree(d_zero);
    if (rc != HYDRO_OK) return rc;
    c->gate_logit_thr = log(threshold / (1.0 - threshold));
    c->gate_zero_smooth = (h_zero < (float)c->gate_logit_thr) ? 1 : 0;
    c->gate_on = 1;
  }
  return rc;
}

}  // extern "C"
