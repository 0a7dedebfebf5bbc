// FP32 dense linear algebra for the mixed-precision Cholesky QR (Sec. 4:
// the filtered block is orthonormalised before the projection).
//
// * Deviation Cholesky.  The second Cholesky QR pass factors the Gram
//   matrix G = I + E of a block that is already nearly orthonormal.  The
//   factor is carried as L = I + F and every operation works on E and F
//   only: a pivot is 1 + t with t the running deviation, its square root
//   is 1 + f with f = t / (1 + sqrt(1 + t)), and the trailing updates
//   subtract products of off-diagonal entries, which are small.  Rounding
//   errors are then relative to |E| instead of |G| = 1, so FP32 gives the
//   factor to about 1e-7 |E| absolute, which FP64 on G could not beat.
// * Triangular inverse W = L^{-1} (lower), for L plain or L = I + F (then
//   W = I + H and H is returned), by blocked recursive doubling: the
//   64 x 64 diagonal blocks are inverted in shared memory, then for block
//   sizes s = 64, 128, ... every pair of neighbouring inverted blocks is
//   joined with W_21 = -W_22 L_21 W_11 (two FP32 GEMMs per level, all pairs
//   of a level in one batched launch).
// * A small FP32 GEMM (64 x 64 tiles, 4 x 4 per thread) with the epilogue
//   C = alpha A B + beta C + gamma D, batched by blockIdx.z with strides.
#include <math.h>

#include "sq3_internal.cuh"

namespace sq3 {

namespace l32 {

constexpr int NB = 64;

// ---------------------------------------------------------------------------
// GEMM: C(m,n) = alpha sum_k A(m,k) B(k,n) + beta C(m,n) + gamma D(m,n)
// A(m,k) = A[m + k lda]; B(k,n) = B[k + n ldb] (bt = false) or B[n + k ldb]
// (bt = true); C, D column-major.  tri = 3: only tiles on or below the
// diagonal.  Batch z offsets every pointer by z times its stride.
// ---------------------------------------------------------------------------
struct G32 {
  int M, N, K;
  const float* A; long long lda, sA;
  const float* B; long long ldb, sB; bool bt;
  float* C; long long ldc, sC;
  const float* D; long long ldd, sD;
  float alpha, beta, gamma;
  int tri;
};

constexpr int BM = 64, BN = 64, BK = 16;

template <bool BT>
__global__ void __launch_bounds__(256) gemm32_kernel(G32 g) {
  __shared__ float As[BK][BM + 4];
  __shared__ float Bs[BK][BN + 4];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  if (g.tri == 3 && n0 >= m0 + BM) return;
  const long long z = blockIdx.z;
  const float* A = g.A + z * g.sA;
  const float* B = g.B + z * g.sB;
  float* C = g.C + z * g.sC;
  const float* D = g.D ? g.D + z * g.sD : nullptr;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  for (int k0 = 0; k0 < g.K; k0 += BK) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int m = tid & 63, k = (tid >> 6) + 4 * r;
      const int gm = m0 + m, gk = k0 + k;
      As[k][m] = (gm < g.M && gk < g.K) ? A[gm + (long long)gk * g.lda] : 0.f;
      if (BT) {
        const int n = tid & 63, kb = (tid >> 6) + 4 * r;
        const int gn = n0 + n, gkb = k0 + kb;
        Bs[kb][n] = (gn < g.N && gkb < g.K) ? B[gn + (long long)gkb * g.ldb] : 0.f;
      } else {
        const int kb = tid & 15, n = (tid >> 4) + 16 * r;
        const int gn = n0 + n, gkb = k0 + kb;
        Bs[kb][n] = (gn < g.N && gkb < g.K) ? B[gkb + (long long)gn * g.ldb] : 0.f;
      }
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + ty + 16 * i;
    if (m >= g.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tx + 16 * j;
      if (n >= g.N) continue;
      float* c = C + m + (long long)n * g.ldc;
      float v = g.alpha * acc[i][j];
      if (g.beta != 0.f) v += g.beta * *c;
      if (D != nullptr) v += g.gamma * D[m + (long long)n * g.ldd];
      *c = v;
    }
  }
}

static void gemm32(const G32& g, int batch, cudaStream_t st) {
  if (g.M <= 0 || g.N <= 0 || batch <= 0) return;
  dim3 grid((g.N + BN - 1) / BN, (g.M + BM - 1) / BM, batch);
  if (g.bt) gemm32_kernel<true><<<grid, 256, 0, st>>>(g);
  else gemm32_kernel<false><<<grid, 256, 0, st>>>(g);
}

// ---------------------------------------------------------------------------
// deviation Cholesky
// ---------------------------------------------------------------------------
// E = S - I in FP32 (S column-major FP64, n x n).
__global__ void deviation_kernel(const double* __restrict__ S, int n, float* E) {
  const long long tot = (long long)n * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e % n), j = (int)(e / n);
    E[e] = (float)(S[e] - (i == j ? 1.0 : 0.0));
  }
}

// Diagonal block (k0, k0) of size kb: on entry the running deviation of the
// Schur complement, on exit F (f_jj on the diagonal, l_ij below).  A pivot
// 1 + t that is not above 1e-3 or not finite sets DEV_NOTPD.
__global__ void __launch_bounds__(256)
potrf_dev_kernel(float* E, int n, int k0, int kb, int* status) {
  __shared__ float A[NB][NB + 1];
  __shared__ float lsh[NB];
  for (int e = threadIdx.x; e < kb * kb; e += blockDim.x) {
    const int i = e % kb, j = e / kb;
    A[i][j] = E[(k0 + i) + (long long)(k0 + j) * n];
  }
  __syncthreads();
  for (int j = 0; j < kb; ++j) {
    const float t = A[j][j];
    float l = sqrtf(1.f + t);
    float f = t / (1.f + l);
    if (!(1.f + t > 1e-3f) || !isfinite(t)) {
      if (threadIdx.x == 0) atomicCAS(status, 0, DEV_NOTPD);
      l = 1.f;
      f = 0.f;
    }
    const float inv = 1.f / l;
    for (int i = j + threadIdx.x; i < kb; i += blockDim.x) {
      const float v = (i == j) ? f : A[i][j] * inv;
      E[(k0 + i) + (long long)(k0 + j) * n] = v;
      if (i > j) lsh[i] = v;
    }
    __syncthreads();
    // trailing lower triangle: thread (row r, column group cg) updates
    // A[r][c] for c = j+1+cg, j+5+cg, .. <= r; the updates of a thread are
    // independent (no chain of shared-memory round trips per column)
    {
      const int r = threadIdx.x & (NB - 1), cg = threadIdx.x / NB;
      if (r > j && r < kb) {
        const float lr = lsh[r];
#pragma unroll 4
        for (int c = j + 1 + cg; c <= r; c += 256 / NB) A[r][c] -= lr * lsh[c];
      }
    }
    __syncthreads();
  }
}

// L21 = E21 (I + F11)^{-T}: each thread solves one row of the panel below,
// right-looking: once x_c is known it is subtracted from every later entry
// (independent FMAs), so the dependent chain is one multiply per column
// instead of a dot product per column; each entry still receives its terms
// in increasing column order.  The pivots' reciprocals are formed once.
__global__ void __launch_bounds__(128)
trsm_dev_kernel(float* E, int n, int k0, int kb) {
  __shared__ float L[NB][NB + 1];
  __shared__ float rinv[NB];
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    const int i = e % NB, j = e / NB;
    L[i][j] = (i < kb && j <= i) ? E[(k0 + i) + (long long)(k0 + j) * n] : 0.f;
  }
  for (int c = threadIdx.x; c < kb; c += blockDim.x)
    rinv[c] = 1.f / (1.f + E[(k0 + c) + (long long)(k0 + c) * n]);
  __syncthreads();
  const int i = k0 + kb + blockIdx.x * blockDim.x + threadIdx.x;
  const bool ok = i < n;
  float x[NB];
#pragma unroll
  for (int c = 0; c < NB; ++c) x[c] = (ok && c < kb) ? E[i + (long long)(k0 + c) * n] : 0.f;
#pragma unroll
  for (int c = 0; c < NB; ++c) {
    if (c < kb) {
      x[c] *= rinv[c];
#pragma unroll
      for (int j = c + 1; j < NB; ++j) x[j] -= x[c] * L[j][c];
    }
  }
  if (ok) {
#pragma unroll
    for (int c = 0; c < NB; ++c)
      if (c < kb) E[i + (long long)(k0 + c) * n] = x[c];
  }
}

// ---------------------------------------------------------------------------
// triangular inverse
// ---------------------------------------------------------------------------
// Inverse of each diagonal NB-block of the lower-triangular L (or of I + F
// when dev, returning H with W = I + H); thread j computes column j.  The
// upper part of every diagonal block of W is written as zero.
__global__ void __launch_bounds__(NB)
tri_inv_diag_kernel(const float* __restrict__ L, int n, float* W, bool dev) {
  __shared__ float Lb[NB][NB + 1];
  __shared__ float Wb[NB][NB + 1];
  const int k0 = blockIdx.x * NB;
  const int kb = min(NB, n - k0);
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    const int i = e % NB, j = e / NB;
    Lb[i][j] = (i < kb && j < kb && i >= j) ? L[(k0 + i) + (long long)(k0 + j) * n] : 0.f;
  }
  __syncthreads();
  const int j = threadIdx.x;
  if (j < kb) {
    // diagonal: w_jj = 1 / l_jj, or h_jj = -f_jj / (1 + f_jj)
    const float djj = dev ? 1.f + Lb[j][j] : Lb[j][j];
    const float wjj = 1.f / djj;
    Wb[j][j] = dev ? -Lb[j][j] / djj : wjj;
    for (int i = j + 1; i < kb; ++i) {
      // w_ij = -(sum_{k=j}^{i-1} l_ik w_kj) / l_ii with l_ik = f_ik (k < i)
      float s = Lb[i][j] * wjj;
      for (int k = j + 1; k < i; ++k) s += Lb[i][k] * Wb[k][j];
      const float dii = dev ? 1.f + Lb[i][i] : Lb[i][i];
      Wb[i][j] = -s / dii;
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < kb * kb; e += blockDim.x) {
    const int i = e % kb, c = e / kb;
    W[(k0 + i) + (long long)(k0 + c) * n] = (i >= c) ? Wb[i][c] : 0.f;
  }
}

// Strictly upper part of W beyond the diagonal blocks is zero; W21 blocks
// are filled level by level.
__global__ void zero_upper_kernel(float* W, int n) {
  const long long tot = (long long)n * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e % n), j = (int)(e / n);
    if (i < j) W[e] = 0.f;
  }
}

// W = L^{-1} (lower, column-major n x n).  tmp: at least n * n / 2 floats.
// Returns the number of kernel launches.
static int tri_inverse(const float* L, float* W, int n, bool dev, float* tmp,
                       cudaStream_t st) {
  int launches = 2;
  const unsigned zg = (unsigned)(((long long)n * n + 255) / 256 > 152 * 16
                                     ? 152 * 16
                                     : ((long long)n * n + 255) / 256);
  zero_upper_kernel<<<zg, 256, 0, st>>>(W, n);
  tri_inv_diag_kernel<<<(n + NB - 1) / NB, NB, 0, st>>>(L, n, W, dev);
  for (int s = NB; s < n; s *= 2) {
    const int full = n / (2 * s);                 // pairs with |B2| = s
    const int r_last = full * 2 * s;              // a ragged pair starts here
    const int b2_last = n - r_last - s;           // its |B2| (<= 0: none)
    for (int part = 0; part < 2; ++part) {
      const int batch = part == 0 ? full : (b2_last > 0 ? 1 : 0);
      if (batch == 0) continue;
      const int r0 = part == 0 ? 0 : r_last;
      const int m2 = part == 0 ? s : b2_last;
      const long long stride = 2LL * s * (1 + n);
      const long long off11 = r0 + (long long)r0 * n;
      const long long off21 = (r0 + s) + (long long)r0 * n;
      const long long off22 = (r0 + s) + (long long)(r0 + s) * n;
      // T = L21 W11 (dev: L21 + L21 H11), m2 x s, ld m2, one per pair
      G32 a{};
      a.M = m2; a.N = s; a.K = s;
      a.A = L + off21; a.lda = n; a.sA = stride;
      a.B = W + off11; a.ldb = n; a.sB = stride; a.bt = false;
      a.C = tmp; a.ldc = m2; a.sC = (long long)m2 * s;
      a.D = dev ? L + off21 : nullptr; a.ldd = n; a.sD = stride;
      a.alpha = 1.f; a.beta = 0.f; a.gamma = 1.f;
      gemm32(a, batch, st);
      // W21 = -W22 T (dev: -(T + H22 T))
      G32 b{};
      b.M = m2; b.N = s; b.K = m2;
      b.A = W + off22; b.lda = n; b.sA = stride;
      b.B = tmp; b.ldb = m2; b.sB = (long long)m2 * s; b.bt = false;
      b.C = W + off21; b.ldc = n; b.sC = stride;
      b.D = dev ? tmp : nullptr; b.ldd = m2; b.sD = (long long)m2 * s;
      b.alpha = -1.f; b.beta = 0.f; b.gamma = -1.f;
      gemm32(b, batch, st);
      launches += 2;
    }
  }
  return launches;
}

// Rinv = W^T as an upper-triangular column-major FP32 matrix; with dev the
// identity is added back (W = I + H).
__global__ void transpose_add_identity_kernel(const float* __restrict__ W, int n, bool dev,
                                              float* Rinv) {
  __shared__ float tile[32][33];
  const int i0 = blockIdx.x * 32, j0 = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 8
  for (int r = ty; r < 32; r += 8) {
    const int i = i0 + tx, j = j0 + r;
    tile[r][tx] = (i < n && j < n) ? W[i + (long long)j * n] : 0.f;
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int i = j0 + tx, j = i0 + r;          // Rinv(i, j) = W(j, i)
    if (i < n && j < n) Rinv[i + (long long)j * n] = tile[tx][r] + ((dev && i == j) ? 1.f : 0.f);
  }
}

__global__ void f64_to_f32_kernel(const double* __restrict__ A, long long tot, float* B) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x)
    B[e] = (float)A[e];
}

}  // namespace l32

using namespace l32;

static unsigned grid_n2(long long tot) {
  long long g = (tot + 255) / 256;
  if (g > 152 * 16) g = 152 * 16;
  return (unsigned)(g < 1 ? 1 : g);
}

// dinv[i] = 1 / sqrt(S_ii) (0 if S_ii is not positive)
__global__ void diag_rsqrt_kernel(const double* __restrict__ S, int n, float* dinv) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const double d = S[i + (long long)i * n];
    dinv[i] = d > 0.0 ? (float)(1.0 / sqrt(d)) : 0.f;
  }
}

// E = D^{-1} S D^{-1} - I with D = diag(S)^{1/2}: the deviation of the
// unit-diagonal scaled Gram matrix
__global__ void scaled_deviation_kernel(const double* __restrict__ S, int n,
                                        const float* __restrict__ dinv, float* E) {
  const long long tot = (long long)n * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e % n), j = (int)(e / n);
    E[e] = (float)(S[e] * (double)dinv[i] * (double)dinv[j] - (i == j ? 1.0 : 0.0));
  }
}

// out = sum_ij (S_ij - delta_ij)^2 (one CTA)
// |S - I|_F^2: block b sums the squares of the columns b, b + DN_BLOCKS, ..
// into part[b]; deviation_norm_finish_kernel adds the DN_BLOCKS partial sums
// in order (the result does not depend on the order in which blocks run).
constexpr int DN_BLOCKS = 32;
__global__ void __launch_bounds__(1024) deviation_norm_kernel(const double* __restrict__ S, int n,
                                                              double* part) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (int j = blockIdx.x; j < n; j += gridDim.x) {
    const double* col = S + (long long)j * n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const double d = col[i] - (i == j ? 1.0 : 0.0);
      acc += d * d;
    }
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    part[blockIdx.x] = t;
  }
}

__global__ void deviation_norm_finish_kernel(const double* part, double* out) {
  double t = 0.0;
  for (int b = 0; b < DN_BLOCKS; ++b) t += part[b];
  *out = t;
}

// R(i, :) *= dinv[i]
__global__ void scale_rows_kernel(float* R, int n, const float* __restrict__ dinv) {
  const long long tot = (long long)n * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x)
    R[e] *= dinv[(int)(e % n)];
}

static void deviation_factor(sq3_ctx* ctx, float* F, int n, cudaStream_t st) {
  for (int k0 = 0; k0 < n; k0 += NB) {
    const int kb = (n - k0 < NB) ? n - k0 : NB;
    potrf_dev_kernel<<<1, 256, 0, st>>>(F, n, k0, kb, ctx->dev_status);
    const int m2 = n - k0 - kb;
    if (m2 <= 0) continue;
    trsm_dev_kernel<<<(m2 + 127) / 128, 128, 0, st>>>(F, n, k0, kb);
    G32 g{};
    g.M = m2; g.N = m2; g.K = kb;
    g.A = F + (k0 + kb) + (long long)k0 * n; g.lda = n;
    g.B = F + (k0 + kb) + (long long)k0 * n; g.ldb = n; g.bt = true;
    g.C = F + (k0 + kb) + (long long)(k0 + kb) * n; g.ldc = n;
    g.alpha = -1.f; g.beta = 1.f; g.gamma = 0.f;
    g.tri = 3;
    gemm32(g, 1, st);
  }
}

int scaled_deviation_cholesky_f32(sq3_ctx* ctx, const double* S, float* F, float* dinv, int n,
                                  cudaStream_t st) {
  diag_rsqrt_kernel<<<(n + 255) / 256, 256, 0, st>>>(S, n, dinv);
  scaled_deviation_kernel<<<grid_n2((long long)n * n), 256, 0, st>>>(S, n, dinv, F);
  deviation_factor(ctx, F, n, st);
  return cuda_err(cudaGetLastError());
}

void deviation_norm_f64(const double* S, int n, double* out, double* part, cudaStream_t st) {
  deviation_norm_kernel<<<DN_BLOCKS, 1024, 0, st>>>(S, n, part);
  deviation_norm_finish_kernel<<<1, 1, 0, st>>>(part, out);
}

void scale_rows_f32(float* R, int n, const float* dinv, cudaStream_t st) {
  scale_rows_kernel<<<grid_n2((long long)n * n), 256, 0, st>>>(R, n, dinv);
}

int deviation_cholesky_f32(sq3_ctx* ctx, const double* S, float* F, int n, cudaStream_t st) {
  deviation_kernel<<<grid_n2((long long)n * n), 256, 0, st>>>(S, n, F);
  deviation_factor(ctx, F, n, st);
  return cuda_err(cudaGetLastError());
}

int rinv_from_lower_f32(const float* L, int n, bool dev, float* W, float* tmp, float* Rinv,
                        cudaStream_t st, bool add_identity) {
  const int launches = tri_inverse(L, W, n, dev, tmp, st);
  dim3 grid((n + 31) / 32, (n + 31) / 32);
  transpose_add_identity_kernel<<<grid, dim3(32, 8), 0, st>>>(W, n, dev && add_identity, Rinv);
  return launches + 1;
}

void convert_f64_to_f32(const double* A, long long tot, float* B, cudaStream_t st) {
  f64_to_f32_kernel<<<grid_n2(tot), 256, 0, st>>>(A, tot, B);
}

}  // namespace sq3
