// Training of the learned predictor on the GPU (not in the paper).
//
// Samples come from the encoder (12 floats per reference slot: 8 features, 3
// target displacements, valid flag).  The valid ones are compacted in order
// (flags, scan, scatter).  One SGD step on a batch of B samples:
//   mlp_grad_kernel    blocks of 128 samples: forward (the inference's fmaf
//                      order) and backward per sample, kept in shared memory;
//                      then the block's gradient, every parameter summed over
//                      its samples in ascending order
//   mlp_reduce_kernel  sum of the block gradients in ascending block order
//   mlp_sgd_kernel     params -= lr * gradient
// Every sum has a fixed order, so training is deterministic.
// Loss: (1/B) sum_i sum_a (o_ia - y_ia)^2.
#include "codec.cuh"

using namespace tera;

namespace {

constexpr int kGB = 128;       // samples per gradient block
constexpr int kDense = 11;     // dense sample: 8 features + 3 targets

__global__ void sample_flags_kernel(const float* __restrict__ samples, u64 n, u32* __restrict__ flags) {
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (u64)gridDim.x * blockDim.x)
    flags[i] = samples[i * kSampleFloats + 11] != 0.0f ? 1u : 0u;
}

__global__ void sample_compact_kernel(const float* __restrict__ samples, u64 n,
                                      const u32* __restrict__ flags, const u32* __restrict__ pos,
                                      float* __restrict__ dense) {
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (u64)gridDim.x * blockDim.x) {
    if (!flags[i]) continue;
    const float* s = samples + i * kSampleFloats;
    float* d = dense + (u64)pos[i] * kDense;
    for (int k = 0; k < kDense; ++k) d[k] = s[k];
  }
}

// rows padded by one float: a thread walks its own row without bank conflicts
struct GradSmem {
  float x[kGB][kMlpIn + 1];
  float a1[kGB][kMlpH + 1];
  float a2[kGB][kMlpH + 1];
  float g1[kGB][kMlpH + 1];
  float g2[kGB][kMlpH + 1];
  float go[kGB][4];
};

__global__ void __launch_bounds__(kGB)
    mlp_grad_kernel(const float* __restrict__ dense, u64 nv, u64 start, u32 batch,
                    const float* __restrict__ params, float* __restrict__ partial) {
  extern __shared__ __align__(16) float smem[];
  float* W = smem;
  GradSmem& S = *reinterpret_cast<GradSmem*>(smem + ((kMlpParams + 3) & ~3));
  for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x) W[i] = params[i];
  __syncthreads();
  const int t = threadIdx.x;
  const u64 i = (u64)blockIdx.x * kGB + t;
  if (i < batch && nv > 0) {
    const float* d = dense + ((start + i) % nv) * kDense;
    float f[kMlpIn], y[kMlpOut];
#pragma unroll
    for (int k = 0; k < kMlpIn; ++k) f[k] = d[k];
#pragma unroll
    for (int a = 0; a < kMlpOut; ++a) y[a] = d[kMlpIn + a];
#pragma unroll
    for (int k = 0; k < kMlpIn; ++k) S.x[t][k] = f[k];
    // forward, as mlp_infer
    for (int j = 0; j < kMlpH; ++j) {
      float acc = W[kMlpB1 + j];
#pragma unroll
      for (int k = 0; k < kMlpIn; ++k) acc = __fmaf_rn(W[kMlpW1 + j * kMlpIn + k], f[k], acc);
      S.a1[t][j] = acc > 0.0f ? acc : 0.0f;
    }
    float o[kMlpOut] = {W[kMlpB3 + 0], W[kMlpB3 + 1], W[kMlpB3 + 2]};
    for (int j = 0; j < kMlpH; ++j) {
      float acc = W[kMlpB2 + j];
      for (int k = 0; k < kMlpH; ++k) acc = __fmaf_rn(W[kMlpW2 + j * kMlpH + k], S.a1[t][k], acc);
      const float h2 = acc > 0.0f ? acc : 0.0f;
      S.a2[t][j] = h2;
#pragma unroll
      for (int a = 0; a < kMlpOut; ++a) o[a] = __fmaf_rn(W[kMlpW3 + a * kMlpH + j], h2, o[a]);
    }
    // backward
    const float scale = __fdiv_rn(2.0f, (float)batch);
    float go[kMlpOut];
#pragma unroll
    for (int a = 0; a < kMlpOut; ++a) {
      go[a] = __fmul_rn(__fsub_rn(o[a], y[a]), scale);
      S.go[t][a] = go[a];
    }
    S.go[t][3] = 0.0f;
    for (int k = 0; k < kMlpH; ++k) {
      float acc = 0.0f;
#pragma unroll
      for (int a = 0; a < kMlpOut; ++a) acc = __fmaf_rn(go[a], W[kMlpW3 + a * kMlpH + k], acc);
      S.g2[t][k] = S.a2[t][k] > 0.0f ? acc : 0.0f;
    }
    for (int k = 0; k < kMlpH; ++k) {
      float acc = 0.0f;
      for (int j = 0; j < kMlpH; ++j) acc = __fmaf_rn(S.g2[t][j], W[kMlpW2 + j * kMlpH + k], acc);
      S.g1[t][k] = S.a1[t][k] > 0.0f ? acc : 0.0f;
    }
  } else {
    for (int k = 0; k < kMlpIn; ++k) S.x[t][k] = 0.0f;
    for (int k = 0; k < kMlpH; ++k) S.a1[t][k] = S.a2[t][k] = S.g1[t][k] = S.g2[t][k] = 0.0f;
    for (int a = 0; a < 4; ++a) S.go[t][a] = 0.0f;
  }
  __syncthreads();
  // the block's gradient: every parameter summed over samples s = 0..127 in order
  float* out = partial + (u64)blockIdx.x * kMlpParams;
  for (int q = threadIdx.x; q < kMlpParams; q += blockDim.x) {
    float acc = 0.0f;
    if (q < kMlpB1) {
      const int j = q / kMlpIn, k = q % kMlpIn;
      for (int s = 0; s < kGB; ++s) acc = __fmaf_rn(S.g1[s][j], S.x[s][k], acc);
    } else if (q < kMlpW2) {
      const int j = q - kMlpB1;
      for (int s = 0; s < kGB; ++s) acc = __fadd_rn(acc, S.g1[s][j]);
    } else if (q < kMlpB2) {
      const int j = (q - kMlpW2) / kMlpH, k = (q - kMlpW2) % kMlpH;
      for (int s = 0; s < kGB; ++s) acc = __fmaf_rn(S.g2[s][j], S.a1[s][k], acc);
    } else if (q < kMlpW3) {
      const int j = q - kMlpB2;
      for (int s = 0; s < kGB; ++s) acc = __fadd_rn(acc, S.g2[s][j]);
    } else if (q < kMlpB3) {
      const int a = (q - kMlpW3) / kMlpH, k = (q - kMlpW3) % kMlpH;
      for (int s = 0; s < kGB; ++s) acc = __fmaf_rn(S.go[s][a], S.a2[s][k], acc);
    } else {
      const int a = q - kMlpB3;
      for (int s = 0; s < kGB; ++s) acc = __fadd_rn(acc, S.go[s][a]);
    }
    out[q] = acc;
  }
}

__global__ void mlp_reduce_kernel(const float* __restrict__ partial, u32 nblocks,
                                  float* __restrict__ grad) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < kMlpParams; q += gridDim.x * blockDim.x) {
    float acc = 0.0f;
    for (u32 b = 0; b < nblocks; ++b) acc = __fadd_rn(acc, partial[(u64)b * kMlpParams + q]);
    grad[q] = acc;
  }
}

// One block: params -= lr * c * grad, c = min(1, clip / |grad|) when clip > 0
// (global-norm clipping; the norm is summed in a fixed order).
__global__ void mlp_sgd_kernel(float* __restrict__ params, const float* __restrict__ grad, float lr,
                               float clip) {
  __shared__ float part[256];
  float ss = 0.0f;
  for (int q = threadIdx.x; q < kMlpParams; q += blockDim.x) ss = __fmaf_rn(grad[q], grad[q], ss);
  part[threadIdx.x] = ss;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) part[threadIdx.x] = __fadd_rn(part[threadIdx.x], part[threadIdx.x + s]);
    __syncthreads();
  }
  const float norm = __fsqrt_rn(part[0]);
  const float c = (clip > 0.0f && norm > clip) ? __fdiv_rn(clip, norm) : 1.0f;
  const float step = __fmul_rn(lr, c);
  for (int q = threadIdx.x; q < kMlpParams; q += blockDim.x)
    params[q] = __fsub_rn(params[q], __fmul_rn(step, grad[q]));
}

constexpr size_t kGradSmem = sizeof(float) * ((kMlpParams + 3) & ~3) + sizeof(GradSmem);

// Scratch layout in ctx->mlp_scratch (floats): dense [n * 11] | flags [n+1] (u32)
// | pos [n+1] (u32) | partial [blocks * 4931] | grad [4931]
tera_status prepare(tera_ctx* ctx, u64 n, u32 max_blocks, float** dense, u32** flags, u32** pos,
                    float** partial, float** grad) {
  const u64 need = n * kDense + 2 * (n + 1) + (u64)max_blocks * kMlpParams + kMlpParams + 64;
  if (!ctx->mlp_scratch || ctx->mlp_scratch_cap < need) {
    cudaDeviceSynchronize();
    if (ctx->mlp_scratch) cudaFree(ctx->mlp_scratch);
    ctx->mlp_scratch = nullptr;
    if (cudaMalloc(reinterpret_cast<void**>(&ctx->mlp_scratch), sizeof(float) * need) != cudaSuccess) {
      cudaGetLastError();
      ctx->mlp_scratch_cap = 0;
      return TERA_ENOMEM;
    }
    ctx->mlp_scratch_cap = need;
  }
  float* b = ctx->mlp_scratch;
  *dense = b;
  *flags = reinterpret_cast<u32*>(b + n * kDense);
  *pos = *flags + (n + 1);
  *partial = reinterpret_cast<float*>(*pos + (n + 1));
  *grad = *partial + (u64)max_blocks * kMlpParams;
  static bool configured = false;
  if (!configured) {
    cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kGradSmem);
    configured = true;
  }
  return TERA_OK;
}

tera_status compact(tera_ctx* ctx, const float* samples, u64 n, float* dense, u32* flags,
                    u32* pos, u64* nv, cudaStream_t s) {
  const unsigned g = (unsigned)((n + 255) / 256 < 65535 ? (n + 255) / 256 + 1 : 65535);
  prof_begin(ctx, s);
  sample_flags_kernel<<<g, 256, 0, s>>>(samples, n, flags);
  tera_status st = check_launch(ctx, "sample_flags_kernel", s);
  if (st != TERA_OK) return st;
  if ((st = scan_u32(ctx, flags, nullptr, pos, n, s)) != TERA_OK) return st;
  prof_begin(ctx, s);
  sample_compact_kernel<<<g, 256, 0, s>>>(samples, n, flags, pos, dense);
  if ((st = check_launch(ctx, "sample_compact_kernel", s)) != TERA_OK) return st;
  u32 h = 0;
  if (cudaMemcpyAsync(&h, pos + n, sizeof(u32), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return TERA_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return TERA_ECUDA;
  *nv = h;
  return TERA_OK;
}

tera_status grad_step(tera_ctx* ctx, const float* dense, u64 nv, u64 start, u32 batch,
                      const float* params, float* partial, float* grad, cudaStream_t s) {
  const u32 nb = (batch + kGB - 1) / kGB;
  prof_begin(ctx, s);
  mlp_grad_kernel<<<nb, kGB, kGradSmem, s>>>(dense, nv, start, batch, params, partial);
  tera_status st = check_launch(ctx, "mlp_grad_kernel", s);
  if (st != TERA_OK) return st;
  prof_begin(ctx, s);
  mlp_reduce_kernel<<<(kMlpParams + 255) / 256, 256, 0, s>>>(partial, nb, grad);
  return check_launch(ctx, "mlp_reduce_kernel", s);
}

}  // namespace

extern "C" tera_status tera_mlp_grad(tera_ctx* ctx, const float* samples, uint64_t n,
                                     const float* params, float* grad, uint64_t* n_valid,
                                     void* stream) {
  TERA_CALL_RANGE("tera_mlp_grad");
  if (!ctx || !samples || !params || !grad || n == 0 || n > 0xFFFFFFF0ull) return TERA_EINVAL;
  cudaSetDevice(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  const u32 max_blocks = (u32)((n + kGB - 1) / kGB);
  float *dense, *partial, *g;
  u32 *flags, *pos;
  tera_status st = prepare(ctx, n, max_blocks, &dense, &flags, &pos, &partial, &g);
  if (st != TERA_OK) return st;
  u64 nv = 0;
  if ((st = compact(ctx, samples, n, dense, flags, pos, &nv, s)) != TERA_OK) return st;
  if (n_valid) *n_valid = nv;
  if (nv == 0) return TERA_EINVAL;
  return grad_step(ctx, dense, nv, 0, (u32)nv, params, partial, grad, s);
}

extern "C" tera_status tera_mlp_train(tera_ctx* ctx, const float* samples, uint64_t n,
                                      float* params, int steps, int batch, float lr, float clip,
                                      uint64_t* n_valid, void* stream) {
  TERA_CALL_RANGE("tera_mlp_train");
  if (!ctx || !samples || !params || n == 0 || n > 0xFFFFFFF0ull || steps < 0 || batch < 1 ||
      batch > (1 << 24))
    return TERA_EINVAL;
  cudaSetDevice(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  const u32 max_blocks = (u32)((batch + kGB - 1) / kGB);
  float *dense, *partial, *g;
  u32 *flags, *pos;
  tera_status st = prepare(ctx, n, max_blocks, &dense, &flags, &pos, &partial, &g);
  if (st != TERA_OK) return st;
  u64 nv = 0;
  if ((st = compact(ctx, samples, n, dense, flags, pos, &nv, s)) != TERA_OK) return st;
  if (n_valid) *n_valid = nv;
  if (nv == 0) return TERA_EINVAL;
  const u32 b = (u32)batch;
  for (int k = 0; k < steps; ++k) {
    const u64 start = ((u64)k * b) % nv;
    if ((st = grad_step(ctx, dense, nv, start, b, params, partial, g, s)) != TERA_OK) return st;
    prof_begin(ctx, s);
    mlp_sgd_kernel<<<1, 256, 0, s>>>(params, g, lr, clip);
    if ((st = check_launch(ctx, "mlp_sgd_kernel", s)) != TERA_OK) return st;
  }
  return TERA_OK;
}
