// The learned ranker: an MLP 96 -> 256 -> 256 -> 1 that scores access pairs
// of a bound kernel so that likely races are checked first.  BF16 operands,
// FP32 accumulation (mma.sync m16n8k16 on the tensor cores), FP32 master
// weights, AdamW, weighted binary cross-entropy on the logits.  Nothing here
// changes a verdict: the ranker only orders the exact checks.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <string>

#include "hgrd_host.h"

namespace hgrd {
namespace {

constexpr int IN = HGRD_MLP_IN, HID = HGRD_MLP_HIDDEN;
// parameter offsets (floats) inside the flat parameter vector
constexpr size_t O_W1 = 0, O_B1 = O_W1 + (size_t)HID * IN, O_W2 = O_B1 + HID, O_B2 = O_W2 + (size_t)HID * HID,
                 O_W3 = O_B2 + HID, O_B3 = O_W3 + HID, NPARAM = O_B3 + 1;
static_assert(NPARAM == HGRD_MLP_PARAMS, "parameter count");

// model buffer: params | grads | adam m | adam v (fp32), then bf16 params
struct Model {
  float *p, *g, *m, *v;
  __nv_bfloat16* pb;
};
size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
Model model_of(void* base) {
  char* c = (char*)base;
  const size_t f = align256(NPARAM * 4);
  Model M;
  M.p = (float*)c;
  M.g = (float*)(c + f);
  M.m = (float*)(c + 2 * f);
  M.v = (float*)(c + 3 * f);
  M.pb = (__nv_bfloat16*)(c + 4 * f);
  return M;
}
size_t model_bytes() { return 4 * align256(NPARAM * 4) + align256(NPARAM * 2); }

// activations for a batch of n samples
struct Acts {
  __nv_bfloat16 *x, *h1, *h2, *dh2, *dh1;
  float *z, *dz, *loss;
};
Acts acts_of(void* base, uint32_t n) {
  char* c = (char*)base;
  size_t off = 0;
  auto take = [&](size_t b) {
    char* r = c + off;
    off = align256(off + b);
    return r;
  };
  Acts A;
  A.x = (__nv_bfloat16*)take((size_t)n * IN * 2);
  A.h1 = (__nv_bfloat16*)take((size_t)n * HID * 2);
  A.h2 = (__nv_bfloat16*)take((size_t)n * HID * 2);
  A.dh2 = (__nv_bfloat16*)take((size_t)n * HID * 2);
  A.dh1 = (__nv_bfloat16*)take((size_t)n * HID * 2);
  A.z = (float*)take((size_t)n * 4);
  A.dz = (float*)take((size_t)n * 4);
  A.loss = (float*)take(256);
  return A;
}
size_t acts_bytes(uint32_t n) {
  return align256((size_t)n * IN * 2) + 4 * align256((size_t)n * HID * 2) + 2 * align256((size_t)n * 4) + 256;
}

// ---------------------------------------------------------------- GEMM
// C[M x N] = A[M x K] * B[K x N]; element access by layout:
//   A row-major: A[m*lda + k], column-major: A[k*lda + m]
//   B row-major: B[k*ldb + n], column-major: B[n*ldb + k]
enum { EP_BIAS_RELU = 0, EP_MASK = 1, EP_ATOMIC = 2 };
constexpr int GT = 64, GK = 16;

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

template <bool A_ROW, bool B_ROW, int EP>
__global__ void __launch_bounds__(128) gemm_kernel(const __nv_bfloat16* __restrict__ A, int lda,
                                                   const __nv_bfloat16* __restrict__ B, int ldb, int M, int N, int K,
                                                   int kchunk, const float* __restrict__ bias,
                                                   const __nv_bfloat16* __restrict__ mask,
                                                   __nv_bfloat16* __restrict__ outb, float* __restrict__ outf, int ldc) {
  __shared__ __nv_bfloat16 As[GT][GK + 8];
  __shared__ __nv_bfloat16 Bs[GK][GT + 8];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int m0 = blockIdx.y * GT, n0 = blockIdx.x * GT;
  const int k_begin = blockIdx.z * kchunk;
  const int k_end = min(K, k_begin + kchunk);
  const int g = lane >> 2, t = lane & 3;
  float acc[8][4];
#pragma unroll
  for (int j = 0; j < 8; ++j)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[j][q] = 0.f;
  const __nv_bfloat16 zero = __float2bfloat16(0.f);
  for (int k0 = k_begin; k0 < k_end; k0 += GK) {
    for (int e = tid; e < GT * GK; e += 128) {
      const int mm = e / GK, kk = e % GK;
      const int gm = m0 + mm, gk = k0 + kk;
      __nv_bfloat16 v = zero;
      if (gm < M && gk < k_end) v = A_ROW ? A[(size_t)gm * lda + gk] : A[(size_t)gk * lda + gm];
      As[mm][kk] = v;
      const int kk2 = e / GT, nn = e % GT;
      const int gn = n0 + nn, gk2 = k0 + kk2;
      __nv_bfloat16 w = zero;
      if (gn < N && gk2 < k_end) w = B_ROW ? B[(size_t)gk2 * ldb + gn] : B[(size_t)gn * ldb + gk2];
      Bs[kk2][nn] = w;
    }
    __syncthreads();
    const int r = warp * 16;
    const uint32_t a0 = pack2(As[r + g][2 * t], As[r + g][2 * t + 1]);
    const uint32_t a1 = pack2(As[r + g + 8][2 * t], As[r + g + 8][2 * t + 1]);
    const uint32_t a2 = pack2(As[r + g][2 * t + 8], As[r + g][2 * t + 9]);
    const uint32_t a3 = pack2(As[r + g + 8][2 * t + 8], As[r + g + 8][2 * t + 9]);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int c = j * 8 + g;
      const uint32_t b0 = pack2(Bs[2 * t][c], Bs[2 * t + 1][c]);
      const uint32_t b1 = pack2(Bs[2 * t + 8][c], Bs[2 * t + 9][c]);
      asm volatile(
          "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
          "{%0,%1,%2,%3};\n"
          : "+f"(acc[j][0]), "+f"(acc[j][1]), "+f"(acc[j][2]), "+f"(acc[j][3])
          : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
    }
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < 8; ++j)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int row = m0 + warp * 16 + g + (q >= 2 ? 8 : 0);
      const int col = n0 + j * 8 + 2 * t + (q & 1);
      if (row >= M || col >= N) continue;
      float v = acc[j][q];
      const size_t o = (size_t)row * ldc + col;
      if (EP == EP_BIAS_RELU) {
        v += bias[col];
        outb[o] = __float2bfloat16(v > 0.f ? v : 0.f);
      } else if (EP == EP_MASK) {
        outb[o] = __float2bfloat16(__bfloat162float(mask[o]) > 0.f ? v : 0.f);
      } else {
        atomicAdd(&outf[o], v);
      }
    }
}

template <bool A_ROW, bool B_ROW, int EP>
cudaError_t gemm(cudaStream_t s, const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb, int M, int N,
                 int K, const float* bias, const __nv_bfloat16* mask, __nv_bfloat16* outb, float* outf, int ldc,
                 int splits = 1) {
  int kchunk = (K + splits - 1) / splits;
  kchunk = ((kchunk + GK - 1) / GK) * GK;
  const int zs = (K + kchunk - 1) / kchunk;
  dim3 grid((N + GT - 1) / GT, (M + GT - 1) / GT, zs);
  gemm_kernel<A_ROW, B_ROW, EP><<<grid, 128, 0, s>>>(A, lda, B, ldb, M, N, K, kchunk, bias, mask, outb, outf, ldc);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- small kernels
__global__ void to_bf16_kernel(const float* __restrict__ in, __nv_bfloat16* __restrict__ out, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = __float2bfloat16(in[i]);
}

// counter-based uniform(-b, b) from SplitMix64 of (seed, index)
__device__ __forceinline__ float uniform_pm(uint64_t seed, uint64_t i, float b) {
  uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  const float u = (float)(z >> 40) * (1.0f / 16777216.0f);
  return (2.f * u - 1.f) * b;
}

__global__ void init_kernel(float* p, float* m, float* v, float* g, uint64_t seed) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < NPARAM; i += (size_t)gridDim.x * blockDim.x) {
    float x = 0.f;
    if (i < O_B1) x = uniform_pm(seed, i, rsqrtf((float)IN));
    else if (i >= O_W2 && i < O_B2) x = uniform_pm(seed, i, rsqrtf((float)HID));
    else if (i >= O_W3 && i < O_B3) x = uniform_pm(seed, i, rsqrtf((float)HID));
    p[i] = x;
    m[i] = v[i] = g[i] = 0.f;
  }
}

// logit, loss and dlogit of each sample; one warp per sample
__global__ void head_forward_kernel(const __nv_bfloat16* __restrict__ h2, const float* __restrict__ p, uint32_t n,
                                    float* __restrict__ z, const float* __restrict__ y, const float* __restrict__ w,
                                    float inv_wsum, float* __restrict__ dz, float* __restrict__ loss) {
  const int lane = threadIdx.x & 31;
  const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  float lsum = 0.f;
  for (uint64_t i = gw; i < n; i += nw) {
    float s = 0.f;
    for (int j = lane; j < HID; j += 32) s += __bfloat162float(h2[i * HID + j]) * p[O_W3 + j];
    for (int o = 16; o; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) {
      const float zz = s + p[O_B3];
      z[i] = zz;
      if (y) {
        const float wi = w ? w[i] : 1.f;
        const float sig = 1.f / (1.f + expf(-zz));
        dz[i] = wi * (sig - y[i]) * inv_wsum;
        lsum += wi * (fmaxf(zz, 0.f) - zz * y[i] + log1pf(expf(-fabsf(zz))));
      }
    }
  }
  if (y && lane == 0 && lsum != 0.f) atomicAdd(loss, lsum * inv_wsum);
}

// dh2 = dz * w3 where h2 > 0; grads of w3 and b3
__global__ void head_backward_kernel(const __nv_bfloat16* __restrict__ h2, const float* __restrict__ p,
                                     const float* __restrict__ dz, uint32_t n, __nv_bfloat16* __restrict__ dh2,
                                     float* __restrict__ g) {
  const int j = threadIdx.x;  // hidden unit, blockDim = HID
  float gw = 0.f, gb = 0.f;
  for (uint64_t i = blockIdx.x; i < n; i += gridDim.x) {
    const float d = dz[i];
    const float h = __bfloat162float(h2[i * HID + j]);
    dh2[i * HID + j] = __float2bfloat16(h > 0.f ? d * p[O_W3 + j] : 0.f);
    gw += d * h;
    gb += d;
  }
  atomicAdd(&g[O_W3 + j], gw);
  if (j == 0) atomicAdd(&g[O_B3], gb);
}

// column sums of a [n x HID] bf16 matrix into the bias gradient
__global__ void bias_grad_kernel(const __nv_bfloat16* __restrict__ d, uint32_t n, float* __restrict__ gb) {
  const int j = threadIdx.x;
  float s = 0.f;
  for (uint64_t i = blockIdx.x; i < n; i += gridDim.x) s += __bfloat162float(d[i * HID + j]);
  atomicAdd(&gb[j], s);
}

__global__ void adamw_kernel(float* p, const float* g, float* m, float* v, __nv_bfloat16* pb, float lr, float wd,
                             float b1c, float b2c) {
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < NPARAM; i += (size_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float upd = (mi / b1c) / (sqrtf(vi / b2c) + eps);
    const float pi = p[i] - lr * (upd + wd * p[i]);
    p[i] = pi;
    pb[i] = __float2bfloat16(pi);
  }
}

#define MK(x)                                                                                  \
  do {                                                                                         \
    cudaError_t e_ = (x);                                                                      \
    if (e_ != cudaSuccess) return fail(HGRD_EDEVICE, std::string("CUDA: ") + cudaGetErrorString(e_)); \
  } while (0)

int forward(const Model& M, const Acts& A, const float* d_x, uint32_t n, cudaStream_t s) {
  const size_t nx = (size_t)n * IN;
  to_bf16_kernel<<<(unsigned)std::min<size_t>((nx + 255) / 256, 4096), 256, 0, s>>>(d_x, A.x, nx);
  MK(cudaGetLastError());
  // h1 = relu(x W1^T + b1): B(k, n) = W1[n][k] (column-major K x N with ldb = IN)
  MK((gemm<true, false, EP_BIAS_RELU>(s, A.x, IN, M.pb + O_W1, IN, (int)n, HID, IN, M.p + O_B1, nullptr, A.h1,
                                       nullptr, HID)));
  MK((gemm<true, false, EP_BIAS_RELU>(s, A.h1, HID, M.pb + O_W2, HID, (int)n, HID, HID, M.p + O_B2, nullptr, A.h2,
                                       nullptr, HID)));
  return HGRD_OK;
}

}  // namespace
}  // namespace hgrd

using namespace hgrd;

extern "C" {

size_t hgrd_mlp_model_bytes(void) { return model_bytes(); }
size_t hgrd_mlp_workspace_bytes(uint32_t batch) { return acts_bytes(batch); }

int hgrd_mlp_init(void* d_model, uint64_t seed, void* stream) {
  if (!d_model) return fail(HGRD_EINVAL, "null model");
  Model M = model_of(d_model);
  cudaStream_t s = (cudaStream_t)stream;
  init_kernel<<<128, 256, 0, s>>>(M.p, M.m, M.v, M.g, seed);
  MK(cudaGetLastError());
  to_bf16_kernel<<<128, 256, 0, s>>>(M.p, M.pb, NPARAM);
  MK(cudaGetLastError());
  return HGRD_OK;
}

int hgrd_mlp_predict(const void* d_model, const float* d_x, uint32_t n, float* d_logits, void* d_ws, size_t ws_bytes,
                     void* stream) {
  if (!d_model || !d_x || !d_logits || !d_ws) return fail(HGRD_EINVAL, "null argument");
  if (ws_bytes < acts_bytes(n)) return fail(HGRD_ENOMEM, "MLP workspace too small");
  if (n == 0) return HGRD_OK;
  Model M = model_of((void*)d_model);
  Acts A = acts_of(d_ws, n);
  cudaStream_t s = (cudaStream_t)stream;
  int rc = forward(M, A, d_x, n, s);
  if (rc) return rc;
  head_forward_kernel<<<(n + 7) / 8, 256, 0, s>>>(A.h2, M.p, n, d_logits, nullptr, nullptr, 0.f, nullptr, nullptr);
  MK(cudaGetLastError());
  return HGRD_OK;
}

int hgrd_mlp_grad(void* d_model, const float* d_x, const float* d_y, const float* d_w, float wsum, uint32_t n,
                  void* d_ws, size_t ws_bytes, void* stream) {
  if (!d_model || !d_x || !d_y || !d_ws) return fail(HGRD_EINVAL, "null argument");
  if (ws_bytes < acts_bytes(n)) return fail(HGRD_ENOMEM, "MLP workspace too small");
  if (n == 0 || !(wsum > 0)) return fail(HGRD_EINVAL, "empty batch");
  Model M = model_of(d_model);
  Acts A = acts_of(d_ws, n);
  cudaStream_t s = (cudaStream_t)stream;
  int rc = forward(M, A, d_x, n, s);
  if (rc) return rc;
  MK(cudaMemsetAsync(M.g, 0, NPARAM * 4, s));
  MK(cudaMemsetAsync(A.loss, 0, 4, s));
  head_forward_kernel<<<(n + 7) / 8, 256, 0, s>>>(A.h2, M.p, n, A.z, d_y, d_w, 1.f / wsum, A.dz, A.loss);
  MK(cudaGetLastError());
  head_backward_kernel<<<std::min<uint32_t>(n, 1024), HID, 0, s>>>(A.h2, M.p, A.dz, n, A.dh2, M.g);
  MK(cudaGetLastError());
  bias_grad_kernel<<<std::min<uint32_t>(n, 1024), HID, 0, s>>>(A.dh2, n, M.g + O_B2);
  MK(cudaGetLastError());
  const int splits = (int)std::max<uint32_t>(1, std::min<uint32_t>(64, n / 256));
  // dW2 = dh2^T h1: A(m, k) = dh2[k][m] (column-major, lda = HID), B(k, n) = h1[k][n]
  MK((gemm<false, true, EP_ATOMIC>(s, A.dh2, HID, A.h1, HID, HID, HID, (int)n, nullptr, nullptr, nullptr,
                                    M.g + O_W2, HID, splits)));
  // dh1 = (dh2 W2) where h1 > 0: B(k, n) = W2[k][n]
  MK((gemm<true, true, EP_MASK>(s, A.dh2, HID, M.pb + O_W2, HID, (int)n, HID, HID, nullptr, A.h1, A.dh1, nullptr,
                                 HID)));
  bias_grad_kernel<<<std::min<uint32_t>(n, 1024), HID, 0, s>>>(A.dh1, n, M.g + O_B1);
  MK(cudaGetLastError());
  // dW1 = dh1^T x
  MK((gemm<false, true, EP_ATOMIC>(s, A.dh1, HID, A.x, IN, HID, IN, (int)n, nullptr, nullptr, nullptr, M.g + O_W1,
                                    IN, splits)));
  return HGRD_OK;
}

int hgrd_mlp_train_step(void* d_model, const float* d_x, const float* d_y, const float* d_w, float wsum, uint32_t n,
                        float lr, float weight_decay, uint32_t step, void* d_ws, size_t ws_bytes, void* stream,
                        float* d_loss) {
  int rc = hgrd_mlp_grad(d_model, d_x, d_y, d_w, wsum, n, d_ws, ws_bytes, stream);
  if (rc) return rc;
  Model M = model_of(d_model);
  Acts A = acts_of(d_ws, n);
  cudaStream_t s = (cudaStream_t)stream;
  const float t = (float)(step + 1);
  adamw_kernel<<<128, 256, 0, s>>>(M.p, M.g, M.m, M.v, M.pb, lr, weight_decay, 1.f - powf(0.9f, t),
                                   1.f - powf(0.999f, t));
  MK(cudaGetLastError());
  if (d_loss) MK(cudaMemcpyAsync(d_loss, A.loss, 4, cudaMemcpyDeviceToDevice, s));
  return HGRD_OK;
}

int hgrd_mlp_params(const void* d_model, float** d_params, float** d_grads) {
  if (!d_model) return fail(HGRD_EINVAL, "null model");
  Model M = model_of((void*)d_model);
  if (d_params) *d_params = M.p;
  if (d_grads) *d_grads = M.g;
  return HGRD_OK;
}

int hgrd_mlp_sync_bf16(void* d_model, void* stream) {
  Model M = model_of(d_model);
  to_bf16_kernel<<<128, 256, 0, (cudaStream_t)stream>>>(M.p, M.pb, NPARAM);
  MK(cudaGetLastError());
  return HGRD_OK;
}

}  // extern "C"
