// Learned starting density for the SCF (not in the paper, which leaves the
// starting density open): a multilayer perceptron over atom-centred
// Gaussian descriptors, trained and evaluated on the GPU with BF16 operands
// on the tensor cores (tcgen05, FP32 accumulation) and FP32/FP64 elementwise
// work.
//
// Model (per grid point x, P = N points of the context's grid):
//   d_k(x) = log(1 + sum_J sum_images exp(-|x - R_J|^2 / w_k^2) / m_k),
//            m_k = natoms pi^{3/2} w_k^3 / Omega   (the sum's cell mean)
//   h1 = tanh(W1 d + b1), h2 = tanh(W2 h1 + b2), h3 = tanh(W3 h2 + b3)
//   y = softplus(w4 . h3 + b4),  rho = Ne y / (sum_x y dV)
// Loss against a self-consistent density rho*: L = sum_x (rho - rho*)^2 dV.
//
// Layouts (row-major, K contiguous, as the tcgen05 GEMM takes them):
//   point-major BF16 activations  [P][K]   A operand of the next layer
//   feature-major BF16 copies     [K][ldP] B / A operands of the weight
//                                          gradients (K = points)
//   weights BF16 [out][in] and their transposes [in][out]
// A layer is one GEMM (M = P, N = 128, K = 64 or 128) whose FP32 output is
// written feature-major; one elementwise kernel adds the bias, applies tanh
// and writes both BF16 layouts (a 32-point x 128-feature tile transposed in
// shared memory).  Backward: dW_l = dZ_l^T H_{l-1} (M = 128, N = in, K = P,
// split-K with FP64 atomics), dH_{l-1} = dZ_l W_l (M = P, N = in, K = 128).
// The features are zero-padded from n_features to 64 columns (one K stage).
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>
#include <vector>

#include "sq3_internal.cuh"
#include "tc_gemm.cuh"

namespace sq3 {

constexpr int MLP_H = 128;    // hidden units
constexpr int MLP_FP = 64;    // padded feature columns
constexpr int MLP_MAXF = 16;  // most descriptor widths
constexpr int MLP_RED = 304;  // blocks of the fixed-order reductions

}  // namespace sq3

// Handle of one model bound to a context (its device, stream and grid).
struct sq3_mlp {
  sq3_ctx* ctx = nullptr;
  // the context's device and stream, kept so that the model can be
  // released after its context
  int device = 0;
  cudaStream_t stream = nullptr;
  int F = 0;                         // descriptor widths
  double widths[16] = {};
  long long P = 0, ldP = 0;          // grid points, padded to 8
  int natoms = 0;
  double omega = 0;
  // parameters: FP32 master, FP64 gradient, Adam moments (same layout:
  // W1 [H][F], b1, W2 [H][H], b2, W3, b3, w4 [H], b4)
  int nparam = 0;
  float* prm = nullptr;
  double* grad = nullptr;
  float* adam_m = nullptr;
  float* adam_v = nullptr;
  long long t = 0;
  // BF16 weights: W1 [H][FP], W2 [H][H], W3 [H][H]; transposes W2t, W3t
  __nv_bfloat16 *w1b = nullptr, *w2b = nullptr, *w3b = nullptr, *w2t = nullptr, *w3t = nullptr;
  // per-point buffers (sized for P)
  double* desc = nullptr;            // F x P descriptors (FP64)
  __nv_bfloat16 *xp = nullptr, *xf = nullptr;          // features [P][FP], [FP][ldP]
  float* z32 = nullptr;                                // GEMM output [H][ldP]
  float* h32[3] = {};                                  // activations [H][ldP]
  __nv_bfloat16* hp[3] = {};                           // [P][H]
  __nv_bfloat16* hf[3] = {};                           // [H][ldP]
  __nv_bfloat16 *dzp = nullptr, *dzf = nullptr;        // gradient of a layer input
  float* y = nullptr;                                  // softplus output
  float* sg = nullptr;                                 // its derivative
  double* red = nullptr;                               // reduction partials + scalars
  bool bufs = false;
};

namespace sq3 {
namespace {

struct Offs { int W1, b1, W2, b2, W3, b3, w4, b4, n; };
__host__ __device__ inline Offs offsets(int F) {
  Offs o;
  o.W1 = 0;
  o.b1 = o.W1 + MLP_H * F;
  o.W2 = o.b1 + MLP_H;
  o.b2 = o.W2 + MLP_H * MLP_H;
  o.W3 = o.b2 + MLP_H;
  o.b3 = o.W3 + MLP_H * MLP_H;
  o.w4 = o.b3 + MLP_H;
  o.b4 = o.w4 + MLP_H;
  o.n = o.b4 + 1;
  return o;
}

// BF16 weights (and transposes) from the FP32 master copy.
__global__ void weights_bf16_kernel(const float* __restrict__ prm, int F, __nv_bfloat16* w1b,
                                    __nv_bfloat16* w2b, __nv_bfloat16* w3b, __nv_bfloat16* w2t,
                                    __nv_bfloat16* w3t) {
  const Offs o = offsets(F);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < MLP_H * MLP_FP) {
    const int r = i / MLP_FP, c = i % MLP_FP;
    w1b[i] = __float2bfloat16_rn(c < F ? prm[o.W1 + r * F + c] : 0.f);
  }
  if (i < MLP_H * MLP_H) {
    const int r = i / MLP_H, c = i % MLP_H;
    const float a = prm[o.W2 + i], b = prm[o.W3 + i];
    w2b[i] = __float2bfloat16_rn(a);
    w3b[i] = __float2bfloat16_rn(b);
    w2t[c * MLP_H + r] = __float2bfloat16_rn(a);
    w3t[c * MLP_H + r] = __float2bfloat16_rn(b);
  }
}

// Compressed descriptors log(1 + d / m) -> BF16 features in both layouts
// (zero beyond F).
__global__ void features_kernel(const double* __restrict__ desc, int F, long long P,
                                long long ldP, const double* __restrict__ scale,
                                __nv_bfloat16* xp, __nv_bfloat16* xf) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < ldP;
       p += (long long)gridDim.x * blockDim.x) {
    __align__(16) __nv_bfloat16 row[MLP_FP];
#pragma unroll
    for (int k = 0; k < MLP_FP; ++k) {
      const float v = (k < F && p < P) ? (float)log1p(desc[(size_t)k * P + p] * scale[k]) : 0.f;
      row[k] = __float2bfloat16_rn(v);
      xf[(size_t)k * ldP + p] = row[k];
    }
    if (p < P) {
      uint4* dst = reinterpret_cast<uint4*>(xp + (size_t)p * MLP_FP);
#pragma unroll
      for (int q = 0; q < MLP_FP / 8; ++q) dst[q] = reinterpret_cast<const uint4*>(row)[q];
    }
  }
}

// h = tanh(z + b) for a tile of 32 points x 128 features: z and h FP32
// feature-major; h also as BF16 feature-major and (through shared memory)
// point-major.
__global__ void __launch_bounds__(256) act_kernel(const float* __restrict__ z,
                                                  const float* __restrict__ bias, long long P,
                                                  long long ldP, float* h32, __nv_bfloat16* hf,
                                                  __nv_bfloat16* hp) {
  __shared__ __align__(16) __nv_bfloat16 tile[32][MLP_H + 8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long p0 = (long long)blockIdx.x * 32;
  const long long p = p0 + lane;
  for (int f = warp; f < MLP_H; f += 8) {
    float v = 0.f;
    if (p < P) {
      v = tanhf(z[(size_t)f * ldP + p] + bias[f]);
      h32[(size_t)f * ldP + p] = v;
    }
    const __nv_bfloat16 b = __float2bfloat16_rn(v);
    if (p < ldP) hf[(size_t)f * ldP + p] = b;
    tile[lane][f] = b;
  }
  __syncthreads();
  // 32 rows x 16 chunks of 16 bytes
  for (int e = threadIdx.x; e < 32 * (MLP_H / 8); e += blockDim.x) {
    const int r = e / (MLP_H / 8), q = e % (MLP_H / 8);
    if (p0 + r < P)
      reinterpret_cast<uint4*>(hp + (size_t)(p0 + r) * MLP_H)[q] =
          *reinterpret_cast<const uint4*>(&tile[r][q * 8]);
  }
}

// Output layer: z4 = w4 . h3 + b4, y = softplus(z4), sg = sigmoid(z4);
// per-block sums of y in part[blockIdx.x].
__global__ void __launch_bounds__(256) out_kernel(const float* __restrict__ h3,
                                                  const float* __restrict__ prm, int F,
                                                  long long P, long long ldP, float* y, float* sg,
                                                  double* part) {
  __shared__ float w4[MLP_H];
  __shared__ double sh[8];
  const Offs o = offsets(F);
  for (int i = threadIdx.x; i < MLP_H; i += blockDim.x) w4[i] = prm[o.w4 + i];
  __syncthreads();
  const float b4 = prm[o.b4];
  double s = 0.0;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < P;
       p += (long long)gridDim.x * blockDim.x) {
    float z = b4;
#pragma unroll 8
    for (int f = 0; f < MLP_H; ++f) z = fmaf(w4[f], h3[(size_t)f * ldP + p], z);
    // softplus and sigmoid without overflow
    const float e = expf(-fabsf(z));
    const float yv = fmaxf(z, 0.f) + log1pf(e);
    y[p] = yv;
    sg[p] = z >= 0.f ? 1.f / (1.f + e) : e / (1.f + e);
    s += yv;
  }
  for (int k = 16; k > 0; k >>= 1) s += __shfl_xor_sync(0xffffffffu, s, k);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += sh[w];
    part[blockIdx.x] = t;
  }
}

// rho = Ne y / S, S = sum y dV from the ordered partials (S into scal[0]).
__global__ void normalise_kernel(const float* __restrict__ y, long long P, const double* part,
                                 double dV, double Ne, double* rho, double* scal) {
  __shared__ double S;
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int b = 0; b < MLP_RED; ++b) t += part[b];
    S = t * dV;
    if (blockIdx.x == 0) scal[0] = S;
  }
  __syncthreads();
  const double f = Ne / S;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < P;
       p += (long long)gridDim.x * blockDim.x)
    rho[p] = f * (double)y[p];
}

// Loss and the sum A = sum_p g_p y_p with g = 2 (rho - rho*) dV: per-block
// partials part[2 b], part[2 b + 1].
__global__ void __launch_bounds__(256) loss_kernel(const double* __restrict__ rho,
                                                   const double* __restrict__ ref,
                                                   const float* __restrict__ y, long long P,
                                                   double dV, double* part) {
  __shared__ double sl[8], sa[8];
  double l = 0.0, a = 0.0;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < P;
       p += (long long)gridDim.x * blockDim.x) {
    const double r = rho[p] - ref[p];
    l += r * r * dV;
    a += 2.0 * r * dV * (double)y[p];
  }
  for (int k = 16; k > 0; k >>= 1) {
    l += __shfl_xor_sync(0xffffffffu, l, k);
    a += __shfl_xor_sync(0xffffffffu, a, k);
  }
  if ((threadIdx.x & 31) == 0) { sl[threadIdx.x >> 5] = l; sa[threadIdx.x >> 5] = a; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tl = 0.0, ta = 0.0;
    for (int w = 0; w < 8; ++w) { tl += sl[w]; ta += sa[w]; }
    part[2 * blockIdx.x] = tl;
    part[2 * blockIdx.x + 1] = ta;
  }
}

__global__ void loss_finish_kernel(const double* part, double* scal) {
  if (threadIdx.x != 0) return;
  double l = 0.0, a = 0.0;
  for (int b = 0; b < MLP_RED; ++b) { l += part[2 * b]; a += part[2 * b + 1]; }
  scal[1] = l;
  scal[2] = a;
}

// Backward through the normalisation, the softplus and the output layer
// for a tile of 32 points: dz4 = (Ne/S)(g - dV A / S) sigmoid(z4);
// gradients of w4 and b4 (FP64 atomics of block sums) and
// dz3 = dz4 w4 (1 - h3^2) in both BF16 layouts, plus its bias gradient.
__global__ void __launch_bounds__(256) out_backward_kernel(
    const double* __restrict__ rho, const double* __restrict__ ref, const float* __restrict__ sg,
    const float* __restrict__ h3, const float* __restrict__ prm, int F, long long P,
    long long ldP, double dV, double Ne, const double* scal, double* grad, __nv_bfloat16* dzf,
    __nv_bfloat16* dzp) {
  __shared__ float dz4[32];
  __shared__ __align__(16) __nv_bfloat16 tile[32][MLP_H + 8];
  const Offs o = offsets(F);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long p0 = (long long)blockIdx.x * 32;
  const long long p = p0 + lane;
  if (warp == 0) {
    const double S = scal[0], A = scal[2];
    double d = 0.0;
    if (p < P) {
      const double g = 2.0 * (rho[p] - ref[p]) * dV;
      d = (Ne / S) * (g - dV * A / S) * (double)sg[p];
    }
    dz4[lane] = (float)d;
    double s = d;
    for (int k = 16; k > 0; k >>= 1) s += __shfl_xor_sync(0xffffffffu, s, k);
    if (lane == 0) atomicAdd(grad + o.b4, s);
  }
  __syncthreads();
  for (int f = warp; f < MLP_H; f += 8) {
    float hv = 0.f, dz = 0.f;
    if (p < P) {
      hv = h3[(size_t)f * ldP + p];
      dz = dz4[lane] * prm[o.w4 + f] * (1.f - hv * hv);
    }
    double gw = (double)dz4[lane] * hv, gb = dz;
    for (int k = 16; k > 0; k >>= 1) {
      gw += __shfl_xor_sync(0xffffffffu, gw, k);
      gb += __shfl_xor_sync(0xffffffffu, gb, k);
    }
    if (lane == 0) {
      atomicAdd(grad + o.w4 + f, gw);
      atomicAdd(grad + o.b3 + f, gb);
    }
    const __nv_bfloat16 b = __float2bfloat16_rn(dz);
    if (p < ldP) dzf[(size_t)f * ldP + p] = b;
    tile[lane][f] = b;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < 32 * (MLP_H / 8); e += blockDim.x) {
    const int r = e / (MLP_H / 8), q = e % (MLP_H / 8);
    if (p0 + r < P)
      reinterpret_cast<uint4*>(dzp + (size_t)(p0 + r) * MLP_H)[q] =
          *reinterpret_cast<const uint4*>(&tile[r][q * 8]);
  }
}

// dz = dh (1 - h^2) for a hidden layer (dh FP32 feature-major from the
// GEMM), in both BF16 layouts, and its bias gradient.
__global__ void __launch_bounds__(256) act_backward_kernel(const float* __restrict__ dh,
                                                           const float* __restrict__ h,
                                                           long long P, long long ldP,
                                                           double* gbias, __nv_bfloat16* dzf,
                                                           __nv_bfloat16* dzp) {
  __shared__ __align__(16) __nv_bfloat16 tile[32][MLP_H + 8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long p0 = (long long)blockIdx.x * 32;
  const long long p = p0 + lane;
  for (int f = warp; f < MLP_H; f += 8) {
    float dz = 0.f;
    if (p < P) {
      const float hv = h[(size_t)f * ldP + p];
      dz = dh[(size_t)f * ldP + p] * (1.f - hv * hv);
    }
    double gb = dz;
    for (int k = 16; k > 0; k >>= 1) gb += __shfl_xor_sync(0xffffffffu, gb, k);
    if (lane == 0) atomicAdd(gbias + f, gb);
    const __nv_bfloat16 b = __float2bfloat16_rn(dz);
    if (p < ldP) dzf[(size_t)f * ldP + p] = b;
    tile[lane][f] = b;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < 32 * (MLP_H / 8); e += blockDim.x) {
    const int r = e / (MLP_H / 8), q = e % (MLP_H / 8);
    if (p0 + r < P)
      reinterpret_cast<uint4*>(dzp + (size_t)(p0 + r) * MLP_H)[q] =
          *reinterpret_cast<const uint4*>(&tile[r][q * 8]);
  }
}

// Weight gradient of a layer from the GEMM's FP64 column-major output
// C(out, in) (ldc = 128): grad[W][out][in] (in < n_in).
__global__ void collect_wgrad_kernel(const double* __restrict__ C, int n_in, double* gW) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= MLP_H * n_in) return;
  const int r = i / n_in, c = i % n_in;
  gW[i] += C[r + (size_t)c * MLP_H];
}

// Adam on every parameter (FP32 master copy, FP64 gradient).
__global__ void adam_kernel(float* prm, const double* __restrict__ g, float* m, float* v, int n,
                            float lr, float b1, float b2, float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = (float)g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  prm[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

template <typename T>
int alloc(T** p, size_t n) {
  if (cudaMalloc((void**)p, n * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return SQ3_ENOMEM;
  }
  return SQ3_OK;
}

void free_buffers(sq3_mlp* m) {
  void* ps[] = {m->desc, m->xp, m->xf, m->z32, m->h32[0], m->h32[1], m->h32[2], m->hp[0],
                m->hp[1], m->hp[2], m->hf[0], m->hf[1], m->hf[2], m->dzp, m->dzf, m->y, m->sg,
                m->red};
  for (void* p : ps) if (p) cudaFree(p);
  m->desc = nullptr; m->xp = m->xf = nullptr; m->z32 = nullptr;
  for (int l = 0; l < 3; ++l) { m->h32[l] = nullptr; m->hp[l] = m->hf[l] = nullptr; }
  m->dzp = m->dzf = nullptr; m->y = m->sg = nullptr; m->red = nullptr;
  m->bufs = false;
}

int ensure_buffers(sq3_mlp* m) {
  const sq3_ctx* c = m->ctx;
  const long long P = c->grid.N;
  if (m->bufs && m->P == P) return SQ3_OK;
  free_buffers(m);
  m->P = P;
  m->ldP = (P + 7) / 8 * 8;
  const size_t ldP = (size_t)m->ldP;
  int rc = SQ3_OK;
  rc = rc ? rc : alloc(&m->desc, (size_t)m->F * P);
  rc = rc ? rc : alloc(&m->xp, (size_t)P * MLP_FP);
  rc = rc ? rc : alloc(&m->xf, (size_t)MLP_FP * ldP);
  rc = rc ? rc : alloc(&m->z32, (size_t)MLP_H * ldP);
  for (int l = 0; l < 3; ++l) {
    rc = rc ? rc : alloc(&m->h32[l], (size_t)MLP_H * ldP);
    rc = rc ? rc : alloc(&m->hp[l], (size_t)P * MLP_H);
    rc = rc ? rc : alloc(&m->hf[l], (size_t)MLP_H * ldP);
  }
  rc = rc ? rc : alloc(&m->dzp, (size_t)P * MLP_H);
  rc = rc ? rc : alloc(&m->dzf, (size_t)MLP_H * ldP);
  rc = rc ? rc : alloc(&m->y, (size_t)P);
  rc = rc ? rc : alloc(&m->sg, (size_t)P);
  rc = rc ? rc : alloc(&m->red, (size_t)2 * MLP_RED + MLP_H * MLP_H + 8);
  if (rc) { free_buffers(m); return rc; }
  m->bufs = true;
  return SQ3_OK;
}

Operand op(const __nv_bfloat16* base, long long rows, int K, long long ld) {
  Operand o;
  o.base = base;
  o.rows = (int)rows;
  o.K = K;
  o.ld = ld;
  o.piece_stride = ((long long)rows * ld + 7) / 8 * 8;
  o.pieces = 1;
  return o;
}

// C32 (feature-major, ldc = ldP) = A (P x K point-major) B^T (B: 128 x K).
int layer_gemm(sq3_mlp* m, const __nv_bfloat16* A, int K, const __nv_bfloat16* B, float* C32) {
  Products pr{};
  pr.n = 1;
  TcParams p{};
  p.C32 = C32;
  p.ldc = m->ldP;
  p.alpha = 1.f;
  return tc_gemm(m->ctx, op(A, m->P, K, K), op(B, MLP_H, K, K), pr, p, EPI_TC_STORE, 1,
                 m->ctx->stream);
}

// C64 (128 x n_in, column-major, ldc 128) += A^T B over the points: A the
// layer's input gradient dz feature-major [128][ldP], B the layer input
// feature-major [n_rows][ldP].
int wgrad_gemm(sq3_mlp* m, const __nv_bfloat16* dzf, const __nv_bfloat16* xf, int n_rows,
               double* C64) {
  Products pr{};
  pr.n = 1;
  TcParams p{};
  p.C64 = C64;
  p.ldc = MLP_H;
  const long long K = m->P;
  int splits = (int)std::min<long long>(152, std::max<long long>(1, K / 512));
  return tc_gemm(m->ctx, op(dzf, MLP_H, (int)K, m->ldP), op(xf, n_rows, (int)K, m->ldP), pr, p,
                 EPI_TC_ATOMIC, splits, m->ctx->stream);
}

int forward(sq3_mlp* m, double Ne, double* rho) {
  sq3_ctx* c = m->ctx;
  cudaStream_t st = c->stream;
  const Offs o = offsets(m->F);
  const long long P = m->P, ldP = m->ldP;
  const unsigned tiles = (unsigned)((ldP + 31) / 32);
  const __nv_bfloat16* in = m->xp;
  int K = MLP_FP;
  const __nv_bfloat16* W[3] = {m->w1b, m->w2b, m->w3b};
  const int boff[3] = {o.b1, o.b2, o.b3};
  for (int l = 0; l < 3; ++l) {
    int rc = layer_gemm(m, in, K, W[l], m->z32);
    if (rc) return rc;
    act_kernel<<<tiles, 256, 0, st>>>(m->z32, m->prm + boff[l], P, ldP, m->h32[l], m->hf[l],
                                      m->hp[l]);
    in = m->hp[l];
    K = MLP_H;
  }
  double* part = m->red;
  double* scal = m->red + 2 * MLP_RED + MLP_H * MLP_H;
  out_kernel<<<MLP_RED, 256, 0, st>>>(m->h32[2], m->prm, m->F, P, ldP, m->y, m->sg, part);
  const unsigned nb = (unsigned)std::min<long long>((P + 255) / 256, 152LL * 8);
  normalise_kernel<<<nb, 256, 0, st>>>(m->y, P, part, c->dV, Ne, rho, scal);
  return cuda_err(cudaGetLastError());
}

// Loss and gradient (into m->grad, zeroed first) for the current features;
// rho: device scratch of P doubles receiving the prediction.
int backward(sq3_mlp* m, const double* ref, double Ne, double* rho) {
  sq3_ctx* c = m->ctx;
  cudaStream_t st = c->stream;
  const Offs o = offsets(m->F);
  const long long P = m->P, ldP = m->ldP;
  int rc = forward(m, Ne, rho);
  if (rc) return rc;
  double* part = m->red;
  double* C64 = m->red + 2 * MLP_RED;
  double* scal = C64 + MLP_H * MLP_H;
  loss_kernel<<<MLP_RED, 256, 0, st>>>(rho, ref, m->y, P, c->dV, part);
  loss_finish_kernel<<<1, 32, 0, st>>>(part, scal);
  rc = cuda_err(cudaMemsetAsync(m->grad, 0, (size_t)m->nparam * sizeof(double), st));
  if (rc) return rc;
  const unsigned tiles = (unsigned)((ldP + 31) / 32);
  out_backward_kernel<<<tiles, 256, 0, st>>>(rho, ref, m->sg, m->h32[2], m->prm, m->F, P, ldP,
                                             c->dV, Ne, scal, m->grad, m->dzf, m->dzp);
  // layers 3, 2, 1: weight gradient, then (l > 1) the gradient of the input
  const __nv_bfloat16* Wt[3] = {nullptr, m->w2t, m->w3t};
  const int woff[3] = {o.W1, o.W2, o.W3};
  const int boff[3] = {o.b1, o.b2, o.b3};
  for (int l = 2; l >= 0; --l) {
    const __nv_bfloat16* xin = l == 0 ? m->xf : m->hf[l - 1];
    const int nin = l == 0 ? m->F : MLP_H;
    rc = cuda_err(cudaMemsetAsync(C64, 0, (size_t)MLP_H * MLP_H * sizeof(double), st));
    if (rc) return rc;
    rc = wgrad_gemm(m, m->dzf, xin, l == 0 ? MLP_FP : MLP_H, C64);
    if (rc) return rc;
    collect_wgrad_kernel<<<(MLP_H * nin + 255) / 256, 256, 0, st>>>(C64, nin, m->grad + woff[l]);
    if (l == 0) break;
    // dH_{l-1} = dZ_l W_l (z32 as scratch), then dZ_{l-1}
    rc = layer_gemm(m, m->dzp, MLP_H, Wt[l], m->z32);
    if (rc) return rc;
    act_backward_kernel<<<tiles, 256, 0, st>>>(m->z32, m->h32[l - 1], P, ldP,
                                               m->grad + boff[l - 1], m->dzf, m->dzp);
  }
  return cuda_err(cudaGetLastError());
}

int refresh_weights(sq3_mlp* m) {
  weights_bf16_kernel<<<(MLP_H * MLP_H + 255) / 256, 256, 0, m->ctx->stream>>>(
      m->prm, m->F, m->w1b, m->w2b, m->w3b, m->w2t, m->w3t);
  return cuda_err(cudaGetLastError());
}

}  // namespace
}  // namespace sq3

using namespace sq3;

extern "C" {

int sq3_mlp_create(sq3_ctx* c, int n_features, const double* widths, int seed, sq3_mlp** out) {
  if (!out) return SQ3_EINVAL;
  *out = nullptr;
  if (!c || !widths || n_features < 1 || n_features > MLP_MAXF) return SQ3_EINVAL;
  for (int k = 0; k < n_features; ++k)
    if (!(widths[k] > 0) || !isfinite(widths[k])) return SQ3_EINVAL;
  if (!c->grid_ok) return SQ3_ENOTSETUP;
  cudaSetDevice(c->device);
  sq3_mlp* m = new sq3_mlp();
  m->ctx = c;
  m->device = c->device;
  m->stream = c->stream;
  m->F = n_features;
  for (int k = 0; k < n_features; ++k) m->widths[k] = widths[k];
  const Offs o = offsets(n_features);
  m->nparam = o.n;
  int rc = SQ3_OK;
  rc = rc ? rc : alloc(&m->prm, (size_t)o.n);
  rc = rc ? rc : alloc(&m->grad, (size_t)o.n);
  rc = rc ? rc : alloc(&m->adam_m, (size_t)o.n);
  rc = rc ? rc : alloc(&m->adam_v, (size_t)o.n);
  rc = rc ? rc : alloc(&m->w1b, (size_t)MLP_H * MLP_FP);
  rc = rc ? rc : alloc(&m->w2b, (size_t)MLP_H * MLP_H);
  rc = rc ? rc : alloc(&m->w3b, (size_t)MLP_H * MLP_H);
  rc = rc ? rc : alloc(&m->w2t, (size_t)MLP_H * MLP_H);
  rc = rc ? rc : alloc(&m->w3t, (size_t)MLP_H * MLP_H);
  if (rc) { sq3_mlp_destroy(m); return rc; }
  // seeded initial weights (a counter-based hash of (seed, index) mapped to
  // N(0, 1) by Box-Muller), scaled by 1/sqrt(fan_in); biases zero
  std::vector<float> h(o.n, 0.f);
  auto normal = [&](unsigned long long i) {
    auto mix = [](unsigned long long x) {
      x += 0x9E3779B97F4A7C15ull;
      x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
      x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
      return x ^ (x >> 31);
    };
    const unsigned long long a = mix(((unsigned long long)seed << 32) ^ (2 * i));
    const unsigned long long b = mix(((unsigned long long)seed << 32) ^ (2 * i + 1));
    const double u1 = ((a >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    const double u2 = ((b >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    return sqrt(-2.0 * log(u1)) * cos(2.0 * 3.14159265358979323846 * u2);
  };
  for (int i = 0; i < MLP_H * n_features; ++i) h[o.W1 + i] = (float)(normal(o.W1 + i) / sqrt((double)n_features));
  for (int i = 0; i < MLP_H * MLP_H; ++i) {
    h[o.W2 + i] = (float)(normal(o.W2 + i) / sqrt((double)MLP_H));
    h[o.W3 + i] = (float)(normal(o.W3 + i) / sqrt((double)MLP_H));
  }
  for (int i = 0; i < MLP_H; ++i) h[o.w4 + i] = (float)(normal(o.w4 + i) / sqrt((double)MLP_H));
  rc = sq3_mlp_set_params(m, h.data());
  if (rc) { sq3_mlp_destroy(m); return rc; }
  *out = m;
  return SQ3_OK;
}

void sq3_mlp_destroy(sq3_mlp* m) {
  if (!m) return;
  cudaSetDevice(m->device);
  cudaStreamSynchronize(m->stream);
  free_buffers(m);
  void* ps[] = {m->prm, m->grad, m->adam_m, m->adam_v, m->w1b, m->w2b, m->w3b, m->w2t, m->w3t};
  for (void* p : ps) if (p) cudaFree(p);
  delete m;
}

int sq3_mlp_num_params(const sq3_mlp* m) { return m ? m->nparam : SQ3_EINVAL; }

int sq3_mlp_set_params(sq3_mlp* m, const float* params) {
  if (!m || !params) return SQ3_EINVAL;
  for (int i = 0; i < m->nparam; ++i)
    if (!isfinite(params[i])) return SQ3_EINVAL;
  sq3_ctx* c = m->ctx;
  cudaSetDevice(c->device);
  int rc = cuda_err(cudaMemcpyAsync(m->prm, params, (size_t)m->nparam * sizeof(float),
                                    cudaMemcpyHostToDevice, c->stream));
  if (rc == SQ3_OK)
    rc = cuda_err(cudaMemsetAsync(m->adam_m, 0, (size_t)m->nparam * sizeof(float), c->stream));
  if (rc == SQ3_OK)
    rc = cuda_err(cudaMemsetAsync(m->adam_v, 0, (size_t)m->nparam * sizeof(float), c->stream));
  if (rc) return rc;
  m->t = 0;
  rc = refresh_weights(m);
  if (rc) return rc;
  return cuda_err(cudaStreamSynchronize(c->stream));
}

int sq3_mlp_get_params(sq3_mlp* m, float* params) {
  if (!m || !params) return SQ3_EINVAL;
  sq3_ctx* c = m->ctx;
  cudaSetDevice(c->device);
  int rc = cuda_err(cudaMemcpyAsync(params, m->prm, (size_t)m->nparam * sizeof(float),
                                    cudaMemcpyDeviceToHost, c->stream));
  if (rc) return rc;
  return cuda_err(cudaStreamSynchronize(c->stream));
}

int sq3_mlp_features(sq3_mlp* m, int natoms, const double* pos) {
  if (!m || natoms < 1 || !pos) return SQ3_EINVAL;
  sq3_ctx* c = m->ctx;
  if (!c->grid_ok) return SQ3_ENOTSETUP;
  cudaSetDevice(c->device);
  int rc = ensure_buffers(m);
  if (rc) return rc;
  const double omega = c->Lx * c->Ly * c->Lz;
  double scale[MLP_MAXF];
  for (int k = 0; k < m->F; ++k) {
    const double w = m->widths[k];
    rc = sq3_atom_gaussians(c, natoms, pos, nullptr, w, 0, 0.0, m->desc + (size_t)k * m->P,
                            nullptr);
    if (rc) return rc;
    scale[k] = omega / (natoms * pow(3.14159265358979323846, 1.5) * w * w * w);
  }
  double* dscale = m->red;
  rc = cuda_err(cudaMemcpyAsync(dscale, scale, m->F * sizeof(double), cudaMemcpyHostToDevice,
                                c->stream));
  if (rc) return rc;
  const unsigned nb = (unsigned)std::min<long long>((m->ldP + 255) / 256, 152LL * 8);
  features_kernel<<<nb, 256, 0, c->stream>>>(m->desc, m->F, m->P, m->ldP, dscale, m->xp, m->xf);
  rc = cuda_err(cudaGetLastError());
  if (rc) return rc;
  rc = cuda_err(cudaStreamSynchronize(c->stream));
  if (rc) return rc;
  m->natoms = natoms;
  return check_device_status(c);
}

int sq3_mlp_predict(sq3_mlp* m, double Ne, double* rho) {
  if (!m || !rho || !(Ne > 0)) return SQ3_EINVAL;
  if (!m->bufs || m->natoms == 0 || m->P != m->ctx->grid.N) return SQ3_ENOTSETUP;
  sq3_ctx* c = m->ctx;
  cudaSetDevice(c->device);
  int rc = forward(m, Ne, rho);
  if (rc) return rc;
  check_finite(rho, m->P, c->dev_status, c->stream);
  rc = cuda_err(cudaStreamSynchronize(c->stream));
  if (rc) return rc;
  return check_device_status(c);
}

int sq3_mlp_gradient(sq3_mlp* m, const double* rho_ref, double Ne, double* rho_scratch,
                     double* loss, double* grad) {
  if (!m || !rho_ref || !rho_scratch || !(Ne > 0)) return SQ3_EINVAL;
  if (!m->bufs || m->natoms == 0 || m->P != m->ctx->grid.N) return SQ3_ENOTSETUP;
  sq3_ctx* c = m->ctx;
  cudaSetDevice(c->device);
  int rc = backward(m, rho_ref, Ne, rho_scratch);
  if (rc) return rc;
  double* scal = m->red + 2 * MLP_RED + MLP_H * MLP_H;
  rc = cuda_err(cudaMemcpyAsync(c->host_scal + 48, scal + 1, sizeof(double),
                                cudaMemcpyDeviceToHost, c->stream));
  if (rc == SQ3_OK && grad)
    rc = cuda_err(cudaMemcpyAsync(grad, m->grad, (size_t)m->nparam * sizeof(double),
                                  cudaMemcpyDeviceToHost, c->stream));
  if (rc) return rc;
  rc = cuda_err(cudaStreamSynchronize(c->stream));
  if (rc) return rc;
  rc = check_device_status(c);
  if (rc) return rc;
  if (loss) *loss = c->host_scal[48];
  return isfinite(c->host_scal[48]) ? SQ3_OK : SQ3_ENONFINITE;
}

int sq3_mlp_train_step(sq3_mlp* m, const double* rho_ref, double Ne, double lr,
                       double* rho_scratch, double* loss) {
  if (!(lr > 0) || !isfinite(lr)) return SQ3_EINVAL;
  int rc = sq3_mlp_gradient(m, rho_ref, Ne, rho_scratch, loss, nullptr);
  if (rc) return rc;
  sq3_ctx* c = m->ctx;
  m->t += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = (float)(1.0 - pow(0.9, (double)m->t));
  const float c2 = (float)(1.0 - pow(0.999, (double)m->t));
  adam_kernel<<<(m->nparam + 255) / 256, 256, 0, c->stream>>>(m->prm, m->grad, m->adam_m,
                                                              m->adam_v, m->nparam, (float)lr,
                                                              b1, b2, 1e-8f, c1, c2);
  rc = refresh_weights(m);
  if (rc) return rc;
  return cuda_err(cudaStreamSynchronize(c->stream));
}

}  // extern "C"
