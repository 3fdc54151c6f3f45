// dg_mlp.cu -- the quadrature-proposal network: 24 -> 128 -> 128 -> 84,
// tanh hidden layers, linear output; bfloat16 operands with FP32
// accumulation (mma.sync m16n8k16), FP32 master weights and Adam.
//
// Forward:  H1 = tanh(X W1 + b1), H2 = tanh(H1 W2 + b2), O = H2 W3 + b3.
// Loss:     (1/2n) sum |O - T|^2.
// Backward: D = (O - T)/n;  gW3 = H2^T D, gb3 = colsum D;
//           G2 = (D W3^T) (1 - H2^2);  gW2 = H1^T G2, gb2 = colsum G2;
//           G1 = (G2 W2^T) (1 - H1^2); gW1 = X^T G1, gb1 = colsum G1.
// Every product is one call of the strided GEMM below.
#include <cuda_bf16.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <random>
#include <vector>

#include "../../include/dg.h"
#include "dg_internal.h"

namespace dg {

namespace {

constexpr int NIN = 24, NH = 128, NO = 84;
constexpr size_t OFF_W1 = 0, OFF_B1 = OFF_W1 + NIN * NH, OFF_W2 = OFF_B1 + NH, OFF_B2 = OFF_W2 + NH * NH;
constexpr size_t OFF_W3 = OFF_B2 + NH, OFF_B3 = OFF_W3 + NH * NO, NPARAM = OFF_B3 + NO;

__device__ __forceinline__ uint32_t pack_bf16(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  const uint32_t l = __bfloat16_as_ushort(lo), h = __bfloat16_as_ushort(hi);
  return l | (h << 16);
}

// C(m, n) = sum_k A(m, k) B(k, n); A(m, k) = A[m*sam + k*sak], B(k, n) = B[k*sbk + n*sbn].
// Epilogue: v = acc (+ bias[n]); act 1: v = tanh(v); act 2: v *= 1 - H(m, n)^2
// (H fp32 with row stride ldh).  Stores fp32 (Cf, ldc) and/or bf16 (Cb, ldcb).
// Each warp computes a 16 x 32 tile; 4 warps per CTA cover 64 x 32.
__global__ void __launch_bounds__(128)
    gemm_bf16_kernel(int M, int N, int K, const __nv_bfloat16* __restrict__ A, int sam, int sak,
                     const __nv_bfloat16* __restrict__ B, int sbk, int sbn, const float* __restrict__ bias, int act,
                     const float* __restrict__ H, int ldh, float* __restrict__ Cf, int ldc,
                     __nv_bfloat16* __restrict__ Cb, int ldcb) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, t = lane & 3;
  const int m0 = blockIdx.y * 64 + warp * 16;
  const int n0 = blockIdx.x * 32;
  const __nv_bfloat16 z = __float2bfloat16_rn(0.f);
  auto ga = [&](int m, int k) { return (m < M && k < K) ? A[(size_t)m * sam + (size_t)k * sak] : z; };
  auto gb = [&](int k, int n) { return (k < K && n < N) ? B[(size_t)k * sbk + (size_t)n * sbn] : z; };
  float c[4][4];
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int i = 0; i < 4; ++i) c[j][i] = 0.f;
  for (int k0 = 0; k0 < K; k0 += 16) {
    const uint32_t a0 = pack_bf16(ga(m0 + g, k0 + 2 * t), ga(m0 + g, k0 + 2 * t + 1));
    const uint32_t a1 = pack_bf16(ga(m0 + g + 8, k0 + 2 * t), ga(m0 + g + 8, k0 + 2 * t + 1));
    const uint32_t a2 = pack_bf16(ga(m0 + g, k0 + 2 * t + 8), ga(m0 + g, k0 + 2 * t + 9));
    const uint32_t a3 = pack_bf16(ga(m0 + g + 8, k0 + 2 * t + 8), ga(m0 + g + 8, k0 + 2 * t + 9));
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + 8 * j + g;
      const uint32_t b0 = pack_bf16(gb(k0 + 2 * t, n), gb(k0 + 2 * t + 1, n));
      const uint32_t b1 = pack_bf16(gb(k0 + 2 * t + 8, n), gb(k0 + 2 * t + 9, n));
      asm volatile(
          "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
          "{%0,%1,%2,%3};\n"
          : "+f"(c[j][0]), "+f"(c[j][1]), "+f"(c[j][2]), "+f"(c[j][3])
          : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
    }
  }
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int m = m0 + g + (i >= 2 ? 8 : 0);
      const int n = n0 + 8 * j + 2 * t + (i & 1);
      if (m >= M || n >= N) continue;
      float v = c[j][i];
      if (bias) v += bias[n];
      if (act == 1) v = tanhf(v);
      if (act == 2) {
        const float h = H[(size_t)m * ldh + n];
        v *= 1.f - h * h;
      }
      if (Cf) Cf[(size_t)m * ldc + n] = v;
      if (Cb) Cb[(size_t)m * ldcb + n] = __float2bfloat16_rn(v);
    }
}

void gemm(cudaStream_t st, int M, int N, int K, const __nv_bfloat16* A, int sam, int sak, const __nv_bfloat16* B,
          int sbk, int sbn, const float* bias, int act, const float* H, int ldh, float* Cf, int ldc, __nv_bfloat16* Cb,
          int ldcb) {
  dim3 grid((N + 31) / 32, (M + 63) / 64);
  gemm_bf16_kernel<<<grid, 128, 0, st>>>(M, N, K, A, sam, sak, B, sbk, sbn, bias, act, H, ldh, Cf, ldc, Cb, ldcb);
}

// D = (O - T)/n (fp32 and bf16), per-row squared error for the loss
__global__ void loss_grad_kernel(int n, const float* __restrict__ O, const float* __restrict__ T,
                                 float* __restrict__ D, __nv_bfloat16* __restrict__ Db, float* __restrict__ rowerr) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  float s = 0.f;
  for (int j = 0; j < NO; ++j) {
    const float d = O[(size_t)r * NO + j] - T[(size_t)r * NO + j];
    s += d * d;
    D[(size_t)r * NO + j] = d / n;
    Db[(size_t)r * NO + j] = __float2bfloat16_rn(d / n);
  }
  rowerr[r] = s;
}

// column sums of G [n x c] into out (fixed order: deterministic)
__global__ void colsum_kernel(int n, int c, const float* __restrict__ G, float* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= c) return;
  float s = 0.f;
  for (int r = 0; r < n; ++r) s += G[(size_t)r * c + j];
  out[j] = s;
}

__global__ void sum_kernel(int n, const float* __restrict__ v, float scale, float* __restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += v[i];
  *out = (float)(s * scale);
}

// Adam on the fp32 master parameters, then their bf16 copies
__global__ void adam_kernel(int np, float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m1,
                            float* __restrict__ m2, float lr, float b1, float b2, float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= np) return;
  const float gi = g[i];
  const float a = b1 * m1[i] + (1.f - b1) * gi;
  const float b = b2 * m2[i] + (1.f - b2) * gi * gi;
  m1[i] = a;
  m2[i] = b;
  p[i] -= lr * (a / c1) / (sqrtf(b / c2) + eps);
}

__global__ void to_bf16_kernel(int n, const float* __restrict__ a, __nv_bfloat16* __restrict__ b) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = __float2bfloat16_rn(a[i]);
}

}  // namespace

}  // namespace dg

using namespace dg;

struct dg_mlp {
  int device = 0;
  float* p = nullptr;  // fp32 master parameters [NPARAM]
  float* g = nullptr;  // gradients
  float* m1 = nullptr;
  float* m2 = nullptr;
  __nv_bfloat16* pb = nullptr;  // bf16 copy of the parameters
  int64_t step = 0;
  // activations for a batch of up to cap rows
  int cap = 0;
  float *h1 = nullptr, *h2 = nullptr, *o = nullptr, *d = nullptr, *g2 = nullptr, *g1 = nullptr, *rowerr = nullptr;
  __nv_bfloat16 *h1b = nullptr, *h2b = nullptr, *db = nullptr, *g2b = nullptr, *g1b = nullptr;
  ~dg_mlp() {
    void* ptrs[] = {p, g, m1, m2, pb, h1, h2, o, d, g2, g1, rowerr, h1b, h2b, db, g2b, g1b};
    for (void* q : ptrs)
      if (q) cudaFree(q);
  }
};

namespace {

int mlp_fail(int code, const char* msg) { return dg_fail_msg(code, msg); }

int ensure_cap(dg_mlp* net, int n) {
  if (n <= net->cap) return DG_OK;
  void** fl[] = {(void**)&net->h1, (void**)&net->h2, (void**)&net->o, (void**)&net->d, (void**)&net->g2,
                 (void**)&net->g1, (void**)&net->rowerr};
  size_t fs[] = {(size_t)NH, (size_t)NH, (size_t)NO, (size_t)NO, (size_t)NH, (size_t)NH, 1};
  for (int i = 0; i < 7; ++i) {
    if (*fl[i]) cudaFree(*fl[i]);
    *fl[i] = nullptr;
    if (cudaMalloc(fl[i], sizeof(float) * fs[i] * n) != cudaSuccess) return mlp_fail(DG_ERR_OOM, "network buffers");
  }
  void** bl[] = {(void**)&net->h1b, (void**)&net->h2b, (void**)&net->db, (void**)&net->g2b, (void**)&net->g1b};
  size_t bs[] = {(size_t)NH, (size_t)NH, (size_t)NO, (size_t)NH, (size_t)NH};
  for (int i = 0; i < 5; ++i) {
    if (*bl[i]) cudaFree(*bl[i]);
    *bl[i] = nullptr;
    if (cudaMalloc(bl[i], 2 * bs[i] * n) != cudaSuccess) return mlp_fail(DG_ERR_OOM, "network buffers");
  }
  net->cap = n;
  return DG_OK;
}

void forward(dg_mlp* net, const __nv_bfloat16* X, int n, float* out, cudaStream_t st) {
  const __nv_bfloat16* W = net->pb;
  const float* P = net->p;
  // H1 = tanh(X W1 + b1): W1 stored [24 x 128] row-major
  gemm(st, n, NH, NIN, X, NIN, 1, W + OFF_W1, NH, 1, P + OFF_B1, 1, nullptr, 0, net->h1, NH, net->h1b, NH);
  gemm(st, n, NH, NH, net->h1b, NH, 1, W + OFF_W2, NH, 1, P + OFF_B2, 1, nullptr, 0, net->h2, NH, net->h2b, NH);
  gemm(st, n, NO, NH, net->h2b, NH, 1, W + OFF_W3, NO, 1, P + OFF_B3, 0, nullptr, 0, out, NO, nullptr, 0);
}

void backward(dg_mlp* net, const __nv_bfloat16* X, const float* T, int n, float* loss, cudaStream_t st) {
  const __nv_bfloat16* W = net->pb;
  float* G = net->g;
  loss_grad_kernel<<<(n + 127) / 128, 128, 0, st>>>(n, net->o, T, net->d, net->db, net->rowerr);
  if (loss) sum_kernel<<<1, 32, 0, st>>>(n, net->rowerr, 0.5f / n, loss);
  // gW3 = H2^T D  (A(m=i, k=s) = H2[s][i])
  gemm(st, NH, NO, n, net->h2b, 1, NH, net->db, NO, 1, nullptr, 0, nullptr, 0, G + OFF_W3, NO, nullptr, 0);
  colsum_kernel<<<1, 128, 0, st>>>(n, NO, net->d, G + OFF_B3);
  // G2 = (D W3^T) (1 - H2^2): B(k=j, n=i) = W3[i][j]
  gemm(st, n, NH, NO, net->db, NO, 1, W + OFF_W3, 1, NO, nullptr, 2, net->h2, NH, net->g2, NH, net->g2b, NH);
  gemm(st, NH, NH, n, net->h1b, 1, NH, net->g2b, NH, 1, nullptr, 0, nullptr, 0, G + OFF_W2, NH, nullptr, 0);
  colsum_kernel<<<1, 128, 0, st>>>(n, NH, net->g2, G + OFF_B2);
  gemm(st, n, NH, NH, net->g2b, NH, 1, W + OFF_W2, 1, NH, nullptr, 2, net->h1, NH, net->g1, NH, net->g1b, NH);
  gemm(st, NIN, NH, n, X, 1, NIN, net->g1b, NH, 1, nullptr, 0, nullptr, 0, G + OFF_W1, NH, nullptr, 0);
  colsum_kernel<<<1, 128, 0, st>>>(n, NH, net->g1, G + OFF_B1);
}

void refresh_bf16(dg_mlp* net, cudaStream_t st) {
  to_bf16_kernel<<<(int)((NPARAM + 255) / 256), 256, 0, st>>>((int)NPARAM, net->p, net->pb);
}

}  // namespace

extern "C" {

int dg_mlp_create(dg_ctx* ctx, int seed, dg_mlp** out) {
  (void)ctx;
  if (!out) return mlp_fail(DG_ERR_ARG, "dg_mlp_create: null output");
  *out = nullptr;
  dg_mlp* net = new (std::nothrow) dg_mlp();
  if (!net) return mlp_fail(DG_ERR_OOM, "out of host memory");
  float** fp[] = {&net->p, &net->g, &net->m1, &net->m2};
  for (float** q : fp)
    if (cudaMalloc(q, sizeof(float) * NPARAM) != cudaSuccess) {
      delete net;
      return mlp_fail(DG_ERR_OOM, "network parameters");
    }
  if (cudaMalloc(&net->pb, 2 * NPARAM) != cudaSuccess) {
    delete net;
    return mlp_fail(DG_ERR_OOM, "network parameters");
  }
  // Xavier-uniform weights, zero biases, from a seeded generator
  std::vector<float> h(NPARAM, 0.f);
  std::mt19937_64 rng((uint64_t)seed * 0x9E3779B97F4A7C15ull + 1);
  auto fill = [&](size_t off, int fi, int fo) {
    const double lim = std::sqrt(6.0 / (fi + fo));
    std::uniform_real_distribution<double> u(-lim, lim);
    for (size_t i = 0; i < (size_t)fi * fo; ++i) h[off + i] = (float)u(rng);
  };
  fill(OFF_W1, NIN, NH);
  fill(OFF_W2, NH, NH);
  fill(OFF_W3, NH, NO);
  if (cudaMemcpy(net->p, h.data(), sizeof(float) * NPARAM, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(net->m1, 0, sizeof(float) * NPARAM) != cudaSuccess ||
      cudaMemset(net->m2, 0, sizeof(float) * NPARAM) != cudaSuccess) {
    delete net;
    return mlp_fail(DG_ERR_CUDA, "network initialisation");
  }
  refresh_bf16(net, nullptr);
  if (cudaDeviceSynchronize() != cudaSuccess) {
    delete net;
    return mlp_fail(DG_ERR_CUDA, "network initialisation");
  }
  *out = net;
  return DG_OK;
}

int dg_mlp_free(dg_mlp* net) {
  delete net;
  return DG_OK;
}

int64_t dg_mlp_num_params(void) { return (int64_t)NPARAM; }

int dg_mlp_get_params(const dg_mlp* net, float* host, int64_t* step) {
  if (!net || !host) return mlp_fail(DG_ERR_ARG, "dg_mlp_get_params: null argument");
  if (cudaMemcpy(host, net->p, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost) != cudaSuccess)
    return mlp_fail(DG_ERR_CUDA, "dg_mlp_get_params: copy failed");
  if (step) *step = net->step;
  return DG_OK;
}

int dg_mlp_set_params(dg_mlp* net, const float* host, int64_t step) {
  if (!net || !host) return mlp_fail(DG_ERR_ARG, "dg_mlp_set_params: null argument");
  if (cudaMemcpy(net->p, host, sizeof(float) * NPARAM, cudaMemcpyHostToDevice) != cudaSuccess)
    return mlp_fail(DG_ERR_CUDA, "dg_mlp_set_params: copy failed");
  net->step = step;
  refresh_bf16(net, nullptr);
  return DG_OK;
}

int dg_mlp_get_state(const dg_mlp* net, float* m1, float* m2) {
  if (!net) return mlp_fail(DG_ERR_ARG, "dg_mlp_get_state: null network");
  if ((m1 && cudaMemcpy(m1, net->m1, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost) != cudaSuccess) ||
      (m2 && cudaMemcpy(m2, net->m2, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost) != cudaSuccess))
    return mlp_fail(DG_ERR_CUDA, "dg_mlp_get_state: copy failed");
  return DG_OK;
}

int dg_mlp_set_state(dg_mlp* net, const float* m1, const float* m2) {
  if (!net) return mlp_fail(DG_ERR_ARG, "dg_mlp_set_state: null network");
  if ((m1 && cudaMemcpy(net->m1, m1, sizeof(float) * NPARAM, cudaMemcpyHostToDevice) != cudaSuccess) ||
      (m2 && cudaMemcpy(net->m2, m2, sizeof(float) * NPARAM, cudaMemcpyHostToDevice) != cudaSuccess))
    return mlp_fail(DG_ERR_CUDA, "dg_mlp_set_state: copy failed");
  return DG_OK;
}

int dg_mlp_forward(dg_ctx* ctx, dg_mlp* net, const void* x_bf16, int n, float* out) {
  if (!ctx || !net || !x_bf16 || !out || n <= 0) return mlp_fail(DG_ERR_ARG, "dg_mlp_forward: bad argument");
  int rc = ensure_cap(net, n);
  if (rc != DG_OK) return rc;
  cudaStream_t st = dg_ctx_stream(ctx);
  forward(net, static_cast<const __nv_bfloat16*>(x_bf16), n, out, st);
  return cudaGetLastError() == cudaSuccess ? DG_OK : mlp_fail(DG_ERR_CUDA, "dg_mlp_forward: launch failed");
}

int dg_mlp_grad(dg_ctx* ctx, dg_mlp* net, const void* x_bf16, const float* target, int n, float* grad,
                float* loss) {
  if (!ctx || !net || !x_bf16 || !target || n <= 0) return mlp_fail(DG_ERR_ARG, "dg_mlp_grad: bad argument");
  int rc = ensure_cap(net, n);
  if (rc != DG_OK) return rc;
  cudaStream_t st = dg_ctx_stream(ctx);
  const __nv_bfloat16* X = static_cast<const __nv_bfloat16*>(x_bf16);
  forward(net, X, n, net->o, st);
  backward(net, X, target, n, loss, st);
  if (grad) cudaMemcpyAsync(grad, net->g, sizeof(float) * NPARAM, cudaMemcpyDeviceToDevice, st);
  return cudaGetLastError() == cudaSuccess ? DG_OK : mlp_fail(DG_ERR_CUDA, "dg_mlp_grad: launch failed");
}

int dg_mlp_train_step(dg_ctx* ctx, dg_mlp* net, const void* x_bf16, const float* target, int n, float lr,
                      float* loss) {
  int rc = dg_mlp_grad(ctx, net, x_bf16, target, n, nullptr, loss);
  if (rc != DG_OK) return rc;
  cudaStream_t st = dg_ctx_stream(ctx);
  net->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - (float)std::pow((double)b1, (double)net->step);
  const float c2 = 1.f - (float)std::pow((double)b2, (double)net->step);
  adam_kernel<<<(int)((NPARAM + 255) / 256), 256, 0, st>>>((int)NPARAM, net->p, net->g, net->m1, net->m2, lr, b1,
                                                           b2, 1e-8f, c1, c2);
  refresh_bf16(net, st);
  return cudaGetLastError() == cudaSuccess ? DG_OK : mlp_fail(DG_ERR_CUDA, "dg_mlp_train_step: launch failed");
}

// Checkpoint file (little-endian, as the host writes it):
//   "DGMLPCK1" | u32 version = 1 | u32 NPARAM | i64 step | u64 seed |
//   i64 cursor | f32 params[NPARAM] | f32 m1[NPARAM] | f32 m2[NPARAM] |
//   u64 FNV-1a of every byte before it.
// Written to "<path>.tmp" and renamed over path, so a reader never sees a
// half-written checkpoint.
namespace {
constexpr char kCkMagic[8] = {'D', 'G', 'M', 'L', 'P', 'C', 'K', '1'};
struct CkHead {
  char magic[8];
  uint32_t version, nparam;
  int64_t step;
  uint64_t seed;
  int64_t cursor;
};
uint64_t fnv1a(uint64_t h, const void* data, size_t n) {
  const unsigned char* b = static_cast<const unsigned char*>(data);
  for (size_t i = 0; i < n; ++i) {
    h ^= b[i];
    h *= 1099511628211ull;
  }
  return h;
}
constexpr uint64_t kFnvBasis = 14695981039346656037ull;
}  // namespace

int dg_mlp_save(dg_ctx* ctx, const dg_mlp* net, const char* path, uint64_t seed, int64_t cursor) {
  if (!ctx || !net || !path) return mlp_fail(DG_ERR_ARG, "dg_mlp_save: null argument");
  if (cudaStreamSynchronize(dg_ctx_stream(ctx)) != cudaSuccess) return mlp_fail(DG_ERR_CUDA, "dg_mlp_save: stream failed");
  std::vector<float> buf((size_t)3 * NPARAM);
  if (cudaMemcpy(buf.data(), net->p, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(buf.data() + NPARAM, net->m1, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(buf.data() + 2 * NPARAM, net->m2, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost) != cudaSuccess)
    return mlp_fail(DG_ERR_CUDA, "dg_mlp_save: copy failed");
  CkHead h{};
  std::memcpy(h.magic, kCkMagic, 8);
  h.version = 1;
  h.nparam = (uint32_t)NPARAM;
  h.step = net->step;
  h.seed = seed;
  h.cursor = cursor;
  uint64_t sum = fnv1a(kFnvBasis, &h, sizeof h);
  sum = fnv1a(sum, buf.data(), sizeof(float) * buf.size());
  const std::string tmp = std::string(path) + ".tmp";
  FILE* f = std::fopen(tmp.c_str(), "wb");
  if (!f) return mlp_fail(DG_ERR_ARG, "dg_mlp_save: cannot open the file for writing");
  const bool ok = std::fwrite(&h, sizeof h, 1, f) == 1 && std::fwrite(buf.data(), sizeof(float), buf.size(), f) == buf.size() &&
                  std::fwrite(&sum, sizeof sum, 1, f) == 1;
  if (std::fclose(f) != 0 || !ok) {
    std::remove(tmp.c_str());
    return mlp_fail(DG_ERR_ARG, "dg_mlp_save: write failed");
  }
  if (std::rename(tmp.c_str(), path) != 0) {
    std::remove(tmp.c_str());
    return mlp_fail(DG_ERR_ARG, "dg_mlp_save: rename failed");
  }
  return DG_OK;
}

int dg_mlp_load(dg_ctx* ctx, dg_mlp* net, const char* path, uint64_t* seed, int64_t* cursor) {
  if (!ctx || !net || !path) return mlp_fail(DG_ERR_ARG, "dg_mlp_load: null argument");
  FILE* f = std::fopen(path, "rb");
  if (!f) return mlp_fail(DG_ERR_ARG, "dg_mlp_load: cannot open the file");
  CkHead h{};
  std::vector<float> buf((size_t)3 * NPARAM);
  uint64_t sum = 0;
  const bool ok = std::fread(&h, sizeof h, 1, f) == 1 && std::memcmp(h.magic, kCkMagic, 8) == 0 && h.version == 1 &&
                  h.nparam == (uint32_t)NPARAM && std::fread(buf.data(), sizeof(float), buf.size(), f) == buf.size() &&
                  std::fread(&sum, sizeof sum, 1, f) == 1;
  std::fclose(f);
  if (!ok) return mlp_fail(DG_ERR_ARG, "dg_mlp_load: not a checkpoint of this network");
  uint64_t chk = fnv1a(kFnvBasis, &h, sizeof h);
  chk = fnv1a(chk, buf.data(), sizeof(float) * buf.size());
  if (chk != sum) return mlp_fail(DG_ERR_ARG, "dg_mlp_load: checksum mismatch");
  cudaStream_t st = dg_ctx_stream(ctx);
  if (cudaStreamSynchronize(st) != cudaSuccess ||
      cudaMemcpy(net->p, buf.data(), sizeof(float) * NPARAM, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(net->m1, buf.data() + NPARAM, sizeof(float) * NPARAM, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(net->m2, buf.data() + 2 * NPARAM, sizeof(float) * NPARAM, cudaMemcpyHostToDevice) != cudaSuccess)
    return mlp_fail(DG_ERR_CUDA, "dg_mlp_load: copy failed");
  net->step = h.step;
  refresh_bf16(net, nullptr);
  if (cudaDeviceSynchronize() != cudaSuccess) return mlp_fail(DG_ERR_CUDA, "dg_mlp_load: refresh failed");
  if (seed) *seed = h.seed;
  if (cursor) *cursor = h.cursor;
  return DG_OK;
}

}  // extern "C"
