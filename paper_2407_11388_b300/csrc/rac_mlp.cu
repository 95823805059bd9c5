// Training and stand-alone inference of the active-block predictor (an MLP
// 8 -> 64 -> 64 -> 1, see rac_mlp.cuh) on the GPU.
//
// Loss: binary cross entropy of the logit z against the label y (1 = the
// evaluation of that (slab, state) pair removed a value), positive samples
// weighted by pos_weight:  l = w(y) (softplus(z) - y z),  w(1) = pos_weight,
// w(0) = 1; the batch loss is the mean over its samples.
//
// Backward pass: the BF16 rounding of the inputs and of the first hidden
// layer is treated as the identity (straight-through), so dW2 = d2 h1~^T and
// dW1 = d1 x~^T use the rounded operands the forward pass multiplied.
//
// Kernels: mlp_fwd_bwd (one thread per sample: forward, then the deltas of
// every layer, stored feature-major), mlp_grad_reduce (one thread per
// parameter: the sum over the batch, FP32), mlp_adam (FP32 master weights,
// BF16 copy for inference), mlp_predict_scalar / mlp_predict_tc (logits).
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <random>
#include <vector>

#include "rac_internal.h"
#include "rac_mlp.cuh"

using namespace rac;

struct rac_predictor {
  int device = 0;
  float *master = nullptr;           // FP32 parameters
  __nv_bfloat16 *w = nullptr;        // BF16 copy that inference reads
  float *m = nullptr, *v = nullptr;  // Adam moments
  float *grad = nullptr;
  float *loss = nullptr;
  uint32_t *pack = nullptr;          // fragment-packed BF16 copy for the warp-wide routine
  int64_t step = 0;
  // per-batch scratch, feature-major [rows][cap]
  float *xr = nullptr, *h1 = nullptr, *d1 = nullptr, *h2 = nullptr, *d2 = nullptr, *dz = nullptr;
  int64_t cap = 0;
};

namespace {

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Sample n of the batch is row idx of X / Y: idx = n when seed == 0, else a
// uniform draw from [0, N) (minibatch sampling with replacement).
__global__ void mlp_fwd_bwd(const __nv_bfloat16 *w, const float *X, const float *Y, int64_t N,
                            int64_t nb, uint64_t seed, float pos_weight, float inv_n, float *XR,
                            float *H1, float *D1, float *H2, float *D2, float *DZ, float *loss) {
  const int64_t n = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (n >= nb) return;
  const int64_t idx = seed ? int64_t(mix64(seed ^ uint64_t(n)) % uint64_t(N)) : n;
  float x[kMlpIn], xr[kMlpIn], h1[kMlpHidden], h2[kMlpHidden];
#pragma unroll
  for (int j = 0; j < kMlpIn; ++j) x[j] = X[idx * kMlpIn + j];
  const float z = mlp_forward(w, x, xr, h1, h2);
  const float y = Y[idx];
  const float wy = y > 0.5f ? pos_weight : 1.0f;
  // softplus(z) - y z, written stably
  const float l = fmaxf(z, 0.0f) + log1pf(expf(-fabsf(z))) - y * z;
  atomicAdd(loss, wy * l * inv_n);
  const float p = 1.0f / (1.0f + expf(-z));
  const float dz = wy * (p - y) * inv_n;
  DZ[n] = dz;
#pragma unroll
  for (int j = 0; j < kMlpIn; ++j) XR[j * nb + n] = xr[j];
  float g1[kMlpHidden];
  for (int j = 0; j < kMlpHidden; ++j) g1[j] = 0.0f;
  for (int i = 0; i < kMlpHidden; ++i) {
    const float d2 = h2[i] > 0.0f ? dz * mlp_w(w, kMlpW3 + i) : 0.0f;
    D2[i * nb + n] = d2;
    H2[i * nb + n] = h2[i];
    if (d2 != 0.0f)
      for (int j = 0; j < kMlpHidden; ++j) g1[j] = fmaf(d2, mlp_w(w, kMlpW2 + i * kMlpHidden + j), g1[j]);
  }
  for (int j = 0; j < kMlpHidden; ++j) {
    D1[j * nb + n] = h1[j] > 0.0f ? g1[j] : 0.0f;
    H1[j * nb + n] = h1[j];
  }
}

// grad[p] = sum over the batch of parameter p's per-sample contribution (the
// 1 / batch factor is already in dz).
__global__ void mlp_grad_reduce(const float *XR, const float *H1, const float *D1, const float *H2,
                                const float *D2, const float *DZ, int64_t nb, float *grad) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= kMlpParams) return;
  const float *a = nullptr, *b = nullptr;  // grad = sum a[n] * (b ? b[n] : 1)
  if (p < kMlpB1) {
    a = D1 + (p / kMlpIn) * nb;
    b = XR + (p % kMlpIn) * nb;
  } else if (p < kMlpW2) {
    a = D1 + (p - kMlpB1) * nb;
  } else if (p < kMlpB2) {
    a = D2 + ((p - kMlpW2) / kMlpHidden) * nb;
    b = H1 + ((p - kMlpW2) % kMlpHidden) * nb;
  } else if (p < kMlpW3) {
    a = D2 + (p - kMlpB2) * nb;
  } else if (p < kMlpB3) {
    a = DZ;
    b = H2 + (p - kMlpW3) * nb;
  } else {
    a = DZ;
  }
  float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
  int64_t n = 0;
  if (b) {
    for (; n + 4 <= nb; n += 4) {
      s0 = fmaf(a[n], b[n], s0);
      s1 = fmaf(a[n + 1], b[n + 1], s1);
      s2 = fmaf(a[n + 2], b[n + 2], s2);
      s3 = fmaf(a[n + 3], b[n + 3], s3);
    }
    for (; n < nb; ++n) s0 = fmaf(a[n], b[n], s0);
  } else {
    for (; n + 4 <= nb; n += 4) {
      s0 += a[n];
      s1 += a[n + 1];
      s2 += a[n + 2];
      s3 += a[n + 3];
    }
    for (; n < nb; ++n) s0 += a[n];
  }
  grad[p] = (s0 + s1) + (s2 + s3);
}

__global__ void mlp_adam(float *master, __nv_bfloat16 *w, float *m, float *v, const float *grad,
                         float lr, float b1, float b2, float eps, float c1, float c2) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= kMlpParams) return;
  const float g = grad[p];
  const float mp = b1 * m[p] + (1.0f - b1) * g;
  const float vp = b2 * v[p] + (1.0f - b2) * g * g;
  m[p] = mp;
  v[p] = vp;
  const float x = master[p] - lr * (mp / c1) / (sqrtf(vp / c2) + eps);
  master[p] = x;
  w[p] = __float2bfloat16(x);
}

__global__ void mlp_to_bf16(const float *master, __nv_bfloat16 *w) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < kMlpParams) w[p] = __float2bfloat16(master[p]);
}

// The fragment-packed copy (rac_mlp.cuh): thread (lane, j) writes word j of
// the lane; one more thread writes b3.
__global__ void mlp_pack(const __nv_bfloat16 *w, uint32_t *pack) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < 32 * 96) {
    const int lane = i / 96, j = i % 96;
    int i0, i1;
    mlp_pack_word(lane, j, i0, i1);
    const uint32_t lo = __bfloat16_as_ushort(w[i0]), hi = __bfloat16_as_ushort(w[i1]);
    pack[((j / 4) * 32 + lane) * 4 + (j % 4)] = lo | (hi << 16);
  } else if (i == 32 * 96) {
    reinterpret_cast<float *>(pack)[kPackChunks * 32 * 4] = __bfloat162float(w[kMlpB3]);
  }
}

__global__ void mlp_predict_scalar(const __nv_bfloat16 *w, const float *X, int64_t N, float *Z) {
  const int64_t n = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float x[kMlpIn], xr[kMlpIn], h1[kMlpHidden], h2[kMlpHidden];
  for (int j = 0; j < kMlpIn; ++j) x[j] = X[n * kMlpIn + j];
  Z[n] = mlp_forward(w, x, xr, h1, h2);
}

// The sweep kernel's inference routine on a plain array: warp q scores
// samples 32 q .. 32 q + 31 (missing samples get zero features).
__global__ void mlp_predict_tc(const uint4 *pack, const float *X, int64_t N, float *Z) {
  const int64_t n = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  float f[kMlpIn];
#pragma unroll
  for (int j = 0; j < kMlpIn; ++j) f[j] = n < N ? X[n * kMlpIn + j] : 0.0f;
  // the upper M tile only when one of this warp's samples 16..31 exists
  const bool upper = __any_sync(0xFFFFFFFFu, n < N && (threadIdx.x & 31) >= 16);
  const float z = mlp_warp_logits(pack, f, upper);
  if (n < N) Z[n] = z;
}

void repack(rac_predictor *p) {
  mlp_pack<<<(32 * 96 + 1 + 127) / 128, 128>>>(p->w, p->pack);
}

void pred_free_scratch(rac_predictor *p) {
  float *s[] = {p->xr, p->h1, p->d1, p->h2, p->d2, p->dz};
  for (float *q : s) cudaFree(q);
  p->xr = p->h1 = p->d1 = p->h2 = p->d2 = p->dz = nullptr;
  p->cap = 0;
}

void pred_free(rac_predictor *p) {
  if (!p) return;
  pred_free_scratch(p);
  void *ptrs[] = {p->master, p->w, p->m, p->v, p->grad, p->loss, p->pack};
  for (void *q : ptrs) cudaFree(q);
  delete p;
}

rac_status ensure_scratch(rac_predictor *p, int64_t nb) {
  if (p->cap >= nb) return RAC_OK;
  pred_free_scratch(p);
  const size_t hb = size_t(nb) * kMlpHidden * sizeof(float);
  if (cudaMalloc(&p->xr, size_t(nb) * kMlpIn * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&p->h1, hb) != cudaSuccess || cudaMalloc(&p->d1, hb) != cudaSuccess ||
      cudaMalloc(&p->h2, hb) != cudaSuccess || cudaMalloc(&p->d2, hb) != cudaSuccess ||
      cudaMalloc(&p->dz, size_t(nb) * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    pred_free_scratch(p);
    set_error("device allocation for predictor training failed");
    return RAC_ENOMEM;
  }
  p->cap = nb;
  return RAC_OK;
}

bool check_pred_device(const rac_predictor *p) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != p->device) {
    set_error("the current CUDA device is not the predictor's device");
    return false;
  }
  return true;
}

// one batch: forward + backward + gradient reduction (into p->grad)
void batch_gradient(rac_predictor *p, const float *X, const float *Y, int64_t N, int64_t nb,
                    uint64_t seed, float pos_weight) {
  mlp_fwd_bwd<<<unsigned((nb + 127) / 128), 128>>>(p->w, X, Y, N, nb, seed, pos_weight,
                                                   1.0f / float(nb), p->xr, p->h1, p->d1, p->h2,
                                                   p->d2, p->dz, p->loss);
  mlp_grad_reduce<<<(kMlpParams + 127) / 128, 128>>>(p->xr, p->h1, p->d1, p->h2, p->d2, p->dz,
                                                     nb, p->grad);
}

}  // namespace

namespace rac {
const uint4 *predictor_pack(const rac_predictor *p) {
  return p ? reinterpret_cast<const uint4 *>(p->pack) : nullptr;
}
int predictor_device(const rac_predictor *p) { return p ? p->device : -1; }
}  // namespace rac

extern "C" {

int32_t rac_predictor_num_params(void) { return kMlpParams; }

rac_status rac_predictor_create(uint64_t seed, rac_predictor **out) try {
  set_error("");
  if (!out) {
    set_error("out is NULL");
    return RAC_EINVAL;
  }
  *out = nullptr;
  rac_predictor *p = new (std::nothrow) rac_predictor();
  if (!p) {
    set_error("out of host memory");
    return RAC_ENOMEM;
  }
  cudaError_t e = cudaGetDevice(&p->device);
  if (e != cudaSuccess) {
    delete p;
    return cuda_fail(e, "cudaGetDevice");
  }
  // He initialisation from a seeded host generator; biases zero
  std::vector<float> init(kMlpParams, 0.0f);
  std::mt19937_64 rng(seed);
  std::normal_distribution<float> nd(0.0f, 1.0f);
  for (int i = 0; i < kMlpHidden * kMlpIn; ++i) init[kMlpW1 + i] = nd(rng) * std::sqrt(2.0f / kMlpIn);
  for (int i = 0; i < kMlpHidden * kMlpHidden; ++i)
    init[kMlpW2 + i] = nd(rng) * std::sqrt(2.0f / kMlpHidden);
  for (int i = 0; i < kMlpHidden; ++i) init[kMlpW3 + i] = nd(rng) * std::sqrt(1.0f / kMlpHidden);
  const size_t pb = kMlpParams * sizeof(float);
  if (cudaMalloc(&p->master, pb) != cudaSuccess ||
      cudaMalloc(&p->w, kMlpParams * sizeof(__nv_bfloat16)) != cudaSuccess ||
      cudaMalloc(&p->m, pb) != cudaSuccess || cudaMalloc(&p->v, pb) != cudaSuccess ||
      cudaMalloc(&p->grad, pb) != cudaSuccess || cudaMalloc(&p->loss, sizeof(float)) != cudaSuccess ||
      cudaMalloc(&p->pack, kPackWords * sizeof(uint32_t)) != cudaSuccess) {
    cudaGetLastError();
    pred_free(p);
    set_error("device allocation of the predictor failed");
    return RAC_ENOMEM;
  }
  e = cudaMemcpy(p->master, init.data(), pb, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(p->m, 0, pb);
  if (e == cudaSuccess) e = cudaMemset(p->v, 0, pb);
  if (e == cudaSuccess) {
    mlp_to_bf16<<<(kMlpParams + 255) / 256, 256>>>(p->master, p->w);
    repack(p);
    e = cudaDeviceSynchronize();
  }
  if (e != cudaSuccess) {
    pred_free(p);
    return cuda_fail(e, "predictor initialisation");
  }
  *out = p;
  return RAC_OK;
} RAC_CATCH_STATUS

void rac_predictor_destroy(rac_predictor *p) { pred_free(p); }

rac_status rac_predictor_set_weights(rac_predictor *p, const float *params) try {
  set_error("");
  if (!p || !params) {
    set_error("NULL argument");
    return RAC_EINVAL;
  }
  if (!check_pred_device(p)) return RAC_EINVAL;
  cudaError_t e = cudaMemcpy(p->master, params, kMlpParams * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(p->m, 0, kMlpParams * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(p->v, 0, kMlpParams * sizeof(float));
  if (e == cudaSuccess) {
    p->step = 0;
    mlp_to_bf16<<<(kMlpParams + 255) / 256, 256>>>(p->master, p->w);
    repack(p);
    e = cudaDeviceSynchronize();
  }
  return e == cudaSuccess ? RAC_OK : cuda_fail(e, "rac_predictor_set_weights");
} RAC_CATCH_STATUS

rac_status rac_predictor_get_weights(const rac_predictor *p, float *params, int32_t bf16) try {
  set_error("");
  if (!p || !params) {
    set_error("NULL argument");
    return RAC_EINVAL;
  }
  if (!check_pred_device(p)) return RAC_EINVAL;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess && !bf16) {
    e = cudaMemcpy(params, p->master, kMlpParams * sizeof(float), cudaMemcpyDeviceToHost);
  } else if (e == cudaSuccess) {
    std::vector<__nv_bfloat16> h(kMlpParams);
    e = cudaMemcpy(h.data(), p->w, kMlpParams * sizeof(__nv_bfloat16), cudaMemcpyDeviceToHost);
    for (int i = 0; e == cudaSuccess && i < kMlpParams; ++i) params[i] = __bfloat162float(h[i]);
  }
  return e == cudaSuccess ? RAC_OK : cuda_fail(e, "rac_predictor_get_weights");
} RAC_CATCH_STATUS

rac_status rac_predictor_gradient(rac_predictor *p, const float *X, const float *Y, int64_t N,
                                  float pos_weight, float *grad_out, float *loss_out) try {
  set_error("");
  if (!p || !X || !Y || N <= 0 || !(pos_weight > 0.0f)) {
    set_error("NULL argument, empty batch or pos_weight <= 0");
    return RAC_EINVAL;
  }
  if (!check_pred_device(p)) return RAC_EINVAL;
  rac_status rc = ensure_scratch(p, N);
  if (rc != RAC_OK) return rc;
  cudaError_t e = cudaMemset(p->loss, 0, sizeof(float));
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemset");
  batch_gradient(p, X, Y, N, N, 0, pos_weight);
  e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "predictor gradient");
  if (grad_out) e = cudaMemcpy(grad_out, p->grad, kMlpParams * sizeof(float), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && loss_out) e = cudaMemcpy(loss_out, p->loss, sizeof(float), cudaMemcpyDeviceToHost);
  return e == cudaSuccess ? RAC_OK : cuda_fail(e, "copy of the gradient");
} RAC_CATCH_STATUS

rac_status rac_predictor_train(rac_predictor *p, const float *X, const float *Y, int64_t N,
                               int32_t steps, int32_t batch, float lr, float pos_weight,
                               uint64_t seed, float *loss_out) try {
  set_error("");
  if (!p || !X || !Y || N <= 0 || steps < 0 || batch <= 0 || !(lr > 0.0f) ||
      !(pos_weight > 0.0f)) {
    set_error("bad training arguments");
    return RAC_EINVAL;
  }
  if (!check_pred_device(p)) return RAC_EINVAL;
  rac_status rc = ensure_scratch(p, batch);
  if (rc != RAC_OK) return rc;
  const float b1 = 0.9f, b2 = 0.999f;
  for (int32_t it = 0; it < steps; ++it) {
    cudaMemsetAsync(p->loss, 0, sizeof(float));
    // a distinct, non-zero sampling seed per step
    const uint64_t step_seed =
        ((seed + 1ull) * 0x2545F4914F6CDD1Dull) ^ ((uint64_t(p->step) + 1ull) * 0x9E3779B97F4A7C15ull);
    batch_gradient(p, X, Y, N, batch, step_seed | 1ull, pos_weight);
    ++p->step;
    const float c1 = 1.0f - std::pow(b1, float(p->step));
    const float c2 = 1.0f - std::pow(b2, float(p->step));
    mlp_adam<<<(kMlpParams + 127) / 128, 128>>>(p->master, p->w, p->m, p->v, p->grad, lr, b1, b2,
                                                1e-8f, c1, c2);
  }
  repack(p);
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "predictor training");
  if (loss_out) {
    e = cudaMemcpy(loss_out, p->loss, sizeof(float), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "copy of the loss");
  }
  return RAC_OK;
} RAC_CATCH_STATUS

rac_status rac_predictor_predict(const rac_predictor *p, const float *X, int64_t N, float *Z,
                                 int32_t tensor_cores) try {
  set_error("");
  if (!p || N < 0 || (N > 0 && (!X || !Z))) {
    set_error("NULL argument or negative count");
    return RAC_EINVAL;
  }
  if (!check_pred_device(p)) return RAC_EINVAL;
  if (N == 0) return RAC_OK;
  if (tensor_cores)
    mlp_predict_tc<<<unsigned((N + 127) / 128), 128>>>(reinterpret_cast<const uint4 *>(p->pack), X,
                                                       N, Z);
  else
    mlp_predict_scalar<<<unsigned((N + 127) / 128), 128>>>(p->w, X, N, Z);
  cudaError_t e = cudaDeviceSynchronize();
  return e == cudaSuccess ? RAC_OK : cuda_fail(e, "predictor inference");
} RAC_CATCH_STATUS

}  // extern "C"
