// Mixed-precision path: FP32 block X, BF16-split tcgen05 GEMMs with FP32
// accumulation, FP64 Cholesky / Fermi level / energies / reductions.
//
// Steps (Sec. 4 of the paper, same order as the FP64 path):
//   orthonormalise   S = X^T X (tcgen05, FP64 accumulation across K-splits),
//                    FP64 Cholesky, R^{-1}, X <- X R^{-1} (tcgen05); applied
//                    twice (Cholesky QR 2); when the first Cholesky meets a
//                    non-positive pivot the pass is repeated on S + s I
//                    (shifted Cholesky QR) before the two plain passes.
//   project          H X by the FP32 stencil, Hs = X^T (H X) (tcgen05)
//   kernel           Hhat and T_j in FP32 with BF16-split products, traces
//                    and the Fermi-level multisection in FP64, Ds summed in
//                    FP64 from FP32 products
//   density          X Ds (tcgen05) with the FP64 row-dot epilogue
// The split of an FP32 value x into bf16 pieces is x_0 = bf16(x),
// x_1 = bf16(x - x_0), x_2 = bf16(x - x_0 - x_1), all round-to-nearest-even.
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>
#include <utility>
#include <vector>

#include "sq3_internal.cuh"
#include "tc_gemm.cuh"

namespace sq3 {

static inline long long pad8(long long x) { return (x + 7) / 8 * 8; }

template <typename T>
__device__ __forceinline__ void split3(T xv, __nv_bfloat16* out, long long e,
                                       long long ps, int pieces) {
  const float x = (float)xv;
  const __nv_bfloat16 h = __float2bfloat16_rn(x);
  out[e] = h;
  if (pieces > 1) {
    const float r = x - __bfloat162float(h);
    const __nv_bfloat16 l = __float2bfloat16_rn(r);
    out[e + ps] = l;
    if (pieces > 2) out[e + 2 * ps] = __float2bfloat16_rn(r - __bfloat162float(l));
  }
}

// Column-major rows x cols source (leading dimension lds) -> pieces with the
// source column as operand row: out[q][c * ld + r].
template <typename T>
__global__ void split_cols_kernel(const T* __restrict__ src, long long lds, int rows,
                                  int cols, __nv_bfloat16* out, long long ld,
                                  long long ps, int pieces) {
  const long long tot = (long long)rows * cols;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const long long c = e / rows, r = e - c * rows;
    split3(src[r + c * lds], out, c * ld + r, ps, pieces);
  }
}

// Pieces of the upper-triangular B = 2 triu(D, 1) + diag(D) of a symmetric
// Ns x Ns matrix D, in the layout of split_cols_kernel.  For symmetric D,
// x D x^T = x B x^T, so the row-dot of the density needs only this B.
__global__ void split_upper_twice_kernel(const double* __restrict__ D, int Ns,
                                         __nv_bfloat16* out, long long ld, long long ps,
                                         int pieces) {
  const long long tot = (long long)Ns * Ns;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const long long c = e / Ns, r = e - c * Ns;
    const double d = D[e];
    split3(r < c ? 2.0 * d : (r == c ? d : 0.0), out, c * ld + r, ps, pieces);
  }
}

// Same layout for an FP32 source, four consecutive rows per thread (16-byte
// load, 8-byte stores per piece) on a 2-D grid (rows x columns), so no
// 64-bit division per element.
__global__ void split_cols_f32x4_kernel(const float* __restrict__ src, long long lds,
                                        int rows, __nv_bfloat16* out, long long ld,
                                        long long ps, int pieces) {
  const long long c = blockIdx.y;
  const long long r = ((long long)blockIdx.x * blockDim.x + threadIdx.x) * 4;
  if (r >= rows) return;
  const float* sp = src + c * lds + r;
  const long long e = c * ld + r;
  if (r + 4 <= rows) {
    const float4 x = *reinterpret_cast<const float4*>(sp);
    const float xs[4] = {x.x, x.y, x.z, x.w};
    __nv_bfloat16 h[3][4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      h[0][i] = __float2bfloat16_rn(xs[i]);
      const float r1 = xs[i] - __bfloat162float(h[0][i]);
      h[1][i] = __float2bfloat16_rn(r1);
      h[2][i] = __float2bfloat16_rn(r1 - __bfloat162float(h[1][i]));
    }
    // unrolled over the three pieces (a loop bounded by `pieces` alone would
    // index h dynamically and put it in local memory)
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      if (q >= pieces) break;
      uint2 pk;
      pk.x = (uint32_t)__bfloat16_as_ushort(h[q][0]) |
             ((uint32_t)__bfloat16_as_ushort(h[q][1]) << 16);
      pk.y = (uint32_t)__bfloat16_as_ushort(h[q][2]) |
             ((uint32_t)__bfloat16_as_ushort(h[q][3]) << 16);
      *reinterpret_cast<uint2*>(out + e + q * ps) = pk;
    }
  } else {
    for (long long t = r; t < rows; ++t) split3(src[c * lds + t], out, c * ld + t, ps, pieces);
  }
}

// Column-major rows x cols source -> pieces with the source ROW as operand
// row: out[q][r * ld + c] (a transpose through shared memory).
__global__ void split_rows_kernel(const float* __restrict__ src, long long lds, int rows,
                                  int cols, __nv_bfloat16* out, long long ld,
                                  long long ps, int pieces) {
  __shared__ float tile[32][33];
  const long long r0 = (long long)blockIdx.x * 32;
  const int c0 = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  for (int j = ty; j < 32; j += 8) {
    const long long r = r0 + tx;
    const int c = c0 + j;
    tile[j][tx] = (r < rows && c < cols) ? src[r + (long long)c * lds] : 0.f;
  }
  __syncthreads();
  for (int j = ty; j < 32; j += 8) {
    const long long r = r0 + j;
    const int c = c0 + tx;
    if (r < rows && c < cols) split3(tile[tx][j], out, r * ld + c, ps, pieces);
  }
}

// Same result for an FP32 source whose rows are a multiple of 4, transposed
// in registers: a lane loads a 4-row x 4-column block (four 16-byte column
// reads; two lanes cover a 32-byte sector) and writes, for each of its 4
// rows, its 4 columns as one 8-byte vector per piece (16 lanes write 128
// contiguous bytes of a row).  A warp covers 8 rows x 64 columns, a CTA 64
// rows x 64 columns (128-row CTAs were measured slower).  No shared memory:
// the shared-memory transpose issued about 2.6 load/store instructions per
// element, this form one.
__global__ void __launch_bounds__(256)
split_rows_reg_kernel(const float* __restrict__ src, long long lds, int rows, int cols,
                      __nv_bfloat16* out, long long ld, long long ps) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int vq = lane & 15, pq = lane >> 4;          // column quad, row quad
  const long long r0 = (long long)blockIdx.x * 64 + warp * 8 + pq * 4;
  const int c0 = blockIdx.y * 64 + vq * 4;
  if (r0 >= rows || c0 >= cols) return;
  float x[4][4];                                     // x[column][row]
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (c0 + j < cols) v = *reinterpret_cast<const float4*>(src + r0 + (long long)(c0 + j) * lds);
    x[j][0] = v.x;
    x[j][1] = v.y;
    x[j][2] = v.z;
    x[j][3] = v.w;
  }
  const int nc = cols - c0;                          // columns of this lane (4 unless the tail)
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    __nv_bfloat16 h[3][4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      h[0][j] = __float2bfloat16_rn(x[j][i]);
      const float r1 = x[j][i] - __bfloat162float(h[0][j]);
      h[1][j] = __float2bfloat16_rn(r1);
      h[2][j] = __float2bfloat16_rn(r1 - __bfloat162float(h[1][j]));
    }
    __nv_bfloat16* o = out + (r0 + i) * ld + c0;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      if (nc >= 4) {
        uint2 w;
        w.x = (uint32_t)__bfloat16_as_ushort(h[q][0]) |
              ((uint32_t)__bfloat16_as_ushort(h[q][1]) << 16);
        w.y = (uint32_t)__bfloat16_as_ushort(h[q][2]) |
              ((uint32_t)__bfloat16_as_ushort(h[q][3]) << 16);
        *reinterpret_cast<uint2*>(o + q * ps) = w;
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (j < nc) o[q * ps + j] = h[q][j];
      }
    }
  }
}

__global__ void hhat_f32_kernel(const double* __restrict__ Hs, int n, const double* bounds,
                                float* T0, float* T1, double* moments) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e == 0) moments[0] = (double)n;
  if (e >= (long long)n * n) return;
  const int i = (int)(e % n), j = (int)(e / n);
  const double h = (Hs[e] - (i == j ? bounds[0] : 0.0)) / bounds[1];
  T1[e] = (float)h;
  T0[e] = (i == j) ? 1.f : 0.f;
}

__global__ void trace_f32_kernel(const float* __restrict__ A, int n, double* out) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += A[i + (long long)i * n];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    *out = t;
  }
}


__global__ void add_shift_kernel(double* S, int n, double rel) {
  // S += rel * (trace(S)/n) I, computed from the diagonal in one CTA
  __shared__ double sh[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += S[i + (long long)i * n];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
  const double shift = rel * t / n;
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) S[i + (long long)i * n] += shift;
}

// ---------------------------------------------------------------------------
// piece buffers inside ctx->wsSplit
// ---------------------------------------------------------------------------
struct MixedBuffers {
  __nv_bfloat16* colX;   // X as K-major over the grid: rows = vectors
  __nv_bfloat16* colY;   // second block (H X) in the same layout
  __nv_bfloat16* rowX;   // X as K-major over vectors: rows = grid points
  __nv_bfloat16* rowX2;  // a second one (written by X R^-1 for the next pass)
  __nv_bfloat16* matA;   // Ns x Ns operands
  __nv_bfloat16* matB;
  __nv_bfloat16* matC;
  long long ldN, ldS, psN, psS;
};

static int mixed_buffers(sq3_ctx* ctx, int Ns, MixedBuffers* b) {
  const long long N = ctx->grid.N;
  b->ldN = pad8(N);
  b->ldS = pad8(Ns);
  b->psN = (long long)Ns * b->ldN;          // colX: Ns rows of ldN
  const long long psR = N * b->ldS;         // rowX: N rows of ldS
  b->psS = (long long)Ns * b->ldS;
  const size_t need = (size_t)MIXED_PIECES * (2 * b->psN + 2 * psR + 3 * b->psS) * 2 + 4096;
  int rc = ensure(&ctx->wsSplit, &ctx->wsSplit_bytes, need);
  if (rc) return rc;
  __nv_bfloat16* p = (__nv_bfloat16*)ctx->wsSplit;
  b->colX = p; p += MIXED_PIECES * b->psN;
  b->colY = p; p += MIXED_PIECES * b->psN;
  b->rowX = p; p += MIXED_PIECES * psR;
  b->rowX2 = p; p += MIXED_PIECES * psR;
  b->matA = p; p += MIXED_PIECES * b->psS;
  b->matB = p; p += MIXED_PIECES * b->psS;
  b->matC = p;
  return SQ3_OK;
}

static Products products(int pieces) {
  Products pr{};
  if (pieces == 1) {
    pr.n = 1;                           // x0 y0 only
  } else if (pieces == 3) {
    // terms down to 2^-16 relative: x0y0, x0y1, x1y0, x0y2, x1y1, x2y0
    const int a[6] = {2, 1, 0, 1, 0, 0}, b[6] = {0, 1, 2, 0, 1, 0};
    pr.n = 6;
    for (int i = 0; i < 6; ++i) { pr.a[i] = a[i]; pr.b[i] = b[i]; }
  } else {
    const int a[3] = {1, 0, 0}, b[3] = {0, 1, 0};
    pr.n = 3;
    for (int i = 0; i < 3; ++i) { pr.a[i] = a[i]; pr.b[i] = b[i]; }
  }
  return pr;
}

static unsigned grid_for(long long tot) {
  long long g = (tot + 255) / 256;
  if (g > 152 * 32) g = 152 * 32;
  return (unsigned)(g < 1 ? 1 : g);
}

static void split_block_cols(sq3_ctx* ctx, const float* X, int Ns, __nv_bfloat16* out,
                             const MixedBuffers& b) {
  Prof p(ctx, ST_SPLIT);
  const long long N = ctx->grid.N;
  if (N % 4 == 0) {      // 16-byte aligned columns
    dim3 grid((unsigned)((N / 4 + 255) / 256), Ns);
    split_cols_f32x4_kernel<<<grid, 256, 0, ctx->stream>>>(X, N, (int)N, out, b.ldN, b.psN,
                                                            MIXED_PIECES);
  } else {
    split_cols_kernel<float><<<grid_for(N * Ns), 256, 0, ctx->stream>>>(
        X, N, (int)N, Ns, out, b.ldN, b.psN, MIXED_PIECES);
  }
}

static void split_block_rows(sq3_ctx* ctx, const float* X, int Ns, const MixedBuffers& b,
                             __nv_bfloat16* out = nullptr) {
  Prof p(ctx, ST_SPLIT);
  const long long N = ctx->grid.N;
  if (!out) out = b.rowX;
  if (N % 4 == 0 && b.ldS % 8 == 0 && MIXED_PIECES == 3) {
    // 16-byte column reads; rows of the pieces are 16-byte aligned (ldS % 8)
    dim3 grid((unsigned)((N + 63) / 64), (Ns + 63) / 64);
    split_rows_reg_kernel<<<grid, 256, 0, ctx->stream>>>(X, N, (int)N, Ns, out, b.ldS,
                                                         N * b.ldS);
    return;
  }
  dim3 grid((unsigned)((N + 31) / 32), (Ns + 31) / 32);
  split_rows_kernel<<<grid, dim3(32, 8), 0, ctx->stream>>>(X, N, (int)N, Ns, out, b.ldS,
                                                           N * b.ldS, MIXED_PIECES);
}

template <typename T>
static void split_matrix(sq3_ctx* ctx, const T* A, int Ns, __nv_bfloat16* out,
                         const MixedBuffers& b) {
  Prof p(ctx, ST_SPLIT);
  split_cols_kernel<T><<<grid_for((long long)Ns * Ns), 256, 0, ctx->stream>>>(
      A, Ns, Ns, Ns, out, b.ldS, b.psS, MIXED_PIECES);
}

static Operand op_cols(const __nv_bfloat16* base, int Ns, long long N, const MixedBuffers& b) {
  return Operand{base, Ns, (int)N, b.ldN, b.psN, MIXED_PIECES};
}
static Operand op_rows(const MixedBuffers& b, long long N, int Ns,
                       const __nv_bfloat16* base = nullptr, int pieces = MIXED_PIECES) {
  return Operand{base ? base : b.rowX, (int)N, Ns, b.ldS, N * b.ldS, pieces};
}
static Operand op_mat(const __nv_bfloat16* base, int Ns, const MixedBuffers& b,
                      int pieces = MIXED_PIECES) {
  return Operand{base, Ns, Ns, b.ldS, b.psS, pieces};
}

// Split-K factor for `tiles` output tiles: each CTA keeps >= 4096 of K, and
// the CTA count is chosen close to a whole number of waves over the 152 SMs
// (one 197 KB CTA per SM).
static int splits_for(int tiles, long long K) {
  long long maxs = K / 4096;
  if (maxs < 1) maxs = 1;
  if (maxs > 64) maxs = 64;
  int best = 1;
  double best_eff = -1.0;
  for (int s = 1; s <= maxs; ++s) {
    const long long ctas = (long long)tiles * s;
    const long long waves = (ctas + 151) / 152;
    const double eff = (double)ctas / (double)(waves * 152);
    if (ctas >= 152 && eff >= 0.95) return s;
    if (eff > best_eff) { best_eff = eff; best = s; }
  }
  return best;
}

// S = A^T B over the grid for two split blocks (upper tiles, mirrored).
static int gram_mixed(sq3_ctx* ctx, const __nv_bfloat16* a, const __nv_bfloat16* bb,
                      int Ns, double* S, const MixedBuffers& b, int stage) {
  const long long N = ctx->grid.N;
  int rc;
  {
    Prof p(ctx, stage);
    cudaMemsetAsync(S, 0, (size_t)Ns * Ns * sizeof(double), ctx->stream);
    TcParams t{};
    t.tri = 1;
    t.C64 = S;
    t.ldc = Ns;
    const int nt = (Ns + 127) / 128;
    rc = tc_gemm(ctx, op_cols(a, Ns, N, b), op_cols(bb, Ns, N, b), products(MIXED_PIECES), t,
                 EPI_TC_ATOMIC, splits_for(nt * (nt + 1) / 2, N), ctx->stream);
  }
  if (rc) return rc;
  mirror_upper_f64(S, Ns, ctx->stream);
  return SQ3_OK;
}

__global__ void add_shift_maxdiag_kernel(double* S, int n, double rel) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s = fmax(s, S[i + (long long)i * n]);
  for (int o = 16; o > 0; o >>= 1) s = fmax(s, __shfl_xor_sync(0xffffffffu, s, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = fmax(t, sh[w]);
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) S[i + (long long)i * n] += rel * t;
}

// Cholesky QR 2 in mixed precision.  If the first Cholesky meets a
// non-positive pivot (the Gram matrix of an ill-conditioned filtered block
// carries rounding errors near its smallest eigenvalues), that pass is
// redone on S + s I with s = 1e-6 max_i S_ii (shifted Cholesky QR, Fukaya et
// al. 2020), after which two plain passes follow.
// Precision of the factors: a pass on the filtered block factors S in FP64
// and inverts the factor in FP32 (its error, about cond(R) 6e-8, only
// leaves the block slightly non-orthonormal, which the last pass removes);
// the last pass factors S = I + E of the nearly orthonormal block by the
// deviation Cholesky and inverts I + F in the same form, both FP32 with
// errors relative to |E|.  Should the deviation Cholesky meet a pivot below
// 1e-3 the last pass falls back to the FP64 factor.
int orthonormalise_mixed(sq3_ctx* ctx, float* X, int Ns) {
  const long long N = ctx->grid.N;
  MixedBuffers b;
  int rc = mixed_buffers(ctx, Ns, &b);
  if (rc) return rc;
  rc = ensure((void**)&ctx->wsMat, &ctx->wsMat_bytes,
              ((size_t)2 * Ns * Ns + Ns) * sizeof(double));
  if (rc) return rc;
  const size_t nn = (size_t)Ns * Ns;
  rc = ensure((void**)&ctx->wsLin32, &ctx->wsLin32_bytes,
              (3 * nn + nn / 2 + (size_t)Ns + 64) * sizeof(float));
  if (rc) return rc;
  double* S = ctx->wsMat;
  double* Rinv = S + nn;
  double* diag = Rinv + nn;
  float* F32 = ctx->wsLin32;          // factor (FP32)
  float* W32 = F32 + nn;              // inverse of the factor
  float* R32 = W32 + nn;              // R^{-1} = W^T
  float* tmp32 = R32 + nn;            // n * n / 2
  float* dinv32 = tmp32 + nn / 2 + 32;   // Ns: 1 / sqrt(S_ii)
  double* devnorm = ctx->dev_scal + 16;  // |S - I|_F^2 of the last pass
  double* devpart = ctx->dev_scal + 24;  // its 32 block sums (slots 24 .. 55)
  bool shift_now = false, shifted = false, extra = false;
  int plain_left = 2;
  // pieces of the last pass's product X + X (R^-1 - I), 0: the plain X R^-1
  int dev_pieces = 0;
  // the pieces of X for the next pass, written by the X R^-1 product of the
  // pass before (colX for the Gram, rows for the next X R^-1)
  bool have_pieces = false;
  __nv_bfloat16* rowA = b.rowX;       // rows of the current X
  __nv_bfloat16* rowB = b.rowX2;      // rows of the next X
  ctx->pieces_X = nullptr;
  ctx->hx_X = nullptr;                // X changes: a kept H X is stale
  while (plain_left > 0) {
    dev_pieces = 0;
    if (!have_pieces) split_block_cols(ctx, X, Ns, b.colX, b);
    rc = gram_mixed(ctx, b.colX, b.colX, Ns, S, b, ST_GRAM);
    if (rc) return rc;
    const bool last = plain_left == 1 && !shift_now;
    bool have_r32 = false, again = false;
    if (last) {
      {
        const int panels = (Ns + 63) / 64;
        Prof p(ctx, ST_CHOL, 3 * panels);
        deviation_norm_f64(S, Ns, devnorm, devpart, ctx->stream);
        cudaMemcpyAsync(ctx->host_scal + 16, devnorm, sizeof(double), cudaMemcpyDeviceToHost,
                        ctx->stream);
        rc = deviation_cholesky_f32(ctx, S, F32, Ns, ctx->stream);
      }
      if (rc) return rc;
      rc = check_device_status(ctx);
      // a block still far from orthonormal (|X^T X - I|_F > 0.3) gets one
      // more pass: the orthogonality a pass leaves grows with cond(X)^2
      again = !extra && ctx->host_scal[16] > 0.09;
      // The product of the final pass as X + X G with G = R^-1 - I, whose
      // norm is about |E|_F / 2: the piece products left out (order k in
      // the BF16 pieces, 2^-9k relative each) then cost at most about
      // 2 2^-9k |G| per element, so one piece of each operand suffices when
      // |E|_F <= 1.6e-5 and two (three products) when |E|_F <= 2.6e-3, both
      // within 3e-8; a larger deviation takes the full product.
      dev_pieces = 0;
      if (!again) {
        const double e2 = ctx->host_scal[16];
        if (e2 <= 2.5e-10) dev_pieces = 1;
        else if (e2 <= 6.8e-6) dev_pieces = 2;
      }
      if (rc == SQ3_OK) {
        Prof p(ctx, ST_TRINV);
        p.launches = rinv_from_lower_f32(F32, Ns, true, W32, tmp32, R32, ctx->stream,
                                         dev_pieces == 0);
        have_r32 = true;
      } else if (rc != SQ3_ENOTPD) {
        return rc;
      }
    } else if (!shift_now) {
      // the filtered block: the unit-diagonal scaled Gram matrix factored by
      // the FP32 deviation Cholesky (any upper-triangular factor keeps the
      // column space; the last pass restores orthonormality); a pivot below
      // 1e-3 falls back to the FP64 factor below
      {
        const int panels = (Ns + 63) / 64;
        Prof p(ctx, ST_CHOL, 3 * panels);
        rc = scaled_deviation_cholesky_f32(ctx, S, F32, dinv32, Ns, ctx->stream);
      }
      if (rc) return rc;
      rc = check_device_status(ctx);
      if (rc == SQ3_OK) {
        Prof p(ctx, ST_TRINV);
        p.launches = rinv_from_lower_f32(F32, Ns, true, W32, tmp32, R32, ctx->stream) + 1;
        scale_rows_f32(R32, Ns, dinv32, ctx->stream);
        have_r32 = true;
      } else if (rc != SQ3_ENOTPD) {
        return rc;
      }
    }
    if (!have_r32) {
      dev_pieces = 0;                   // the FP64 fallback: the full product
      if (shift_now) {
        Prof p(ctx, ST_CHOL);
        add_shift_maxdiag_kernel<<<1, 1024, 0, ctx->stream>>>(S, Ns, 1e-6);
      }
      {
        const int panels = (Ns + 63) / 64;
        Prof p(ctx, ST_CHOL, 3 * panels - 1);
        rc = cholesky_lower_f64(ctx, S, Ns, diag, ctx->stream);
      }
      if (rc) return rc;
      rc = check_device_status(ctx);
      if (rc == SQ3_ENOTPD && !shifted && !last) {
        shifted = shift_now = true;
        continue;                        // X unchanged: its pieces stay valid
      }
      if (rc) return rc;
      if (last) {
        // fallback of the last pass: the FP64 inverse of the FP64 factor
        Prof p(ctx, ST_TRINV);
        tri_inverse_transpose_f64(S, Rinv, Ns, diag, ctx->stream);
      } else {
        Prof p(ctx, ST_TRINV);
        convert_f64_to_f32(S, (long long)nn, F32, ctx->stream);
        p.launches = 1 + rinv_from_lower_f32(F32, Ns, false, W32, tmp32, R32, ctx->stream);
        have_r32 = true;
      }
    }
    if (have_r32) split_matrix<float>(ctx, R32, Ns, b.matA, b);
    else split_matrix<double>(ctx, Rinv, Ns, b.matA, b);
    if (!have_pieces) split_block_rows(ctx, X, Ns, b, rowA);
    // another pass follows this one: its inputs' pieces come from this product
    const bool follows = shift_now || again || plain_left > 1;
    // the final product also writes the pieces of the result for the
    // projection and the density, when the SCF driver will reuse them
    const bool keep = !follows && ctx->reuse_pieces;
    {
      // the product reads X only through its pieces, so it overwrites X
      Prof p(ctx, ST_XRINV);
      TcParams t{};
      t.tri = 2;
      t.C32 = X;
      t.ldc = N;
      t.alpha = 1.f;
      if (follows || keep) {
        t.colP = b.colX;
        t.col_ld = b.ldN;
        t.col_ps = b.psN;
        t.rowP = rowB;
        t.row_ld = b.ldS;
        t.row_ps = N * b.ldS;
      }
      const int pieces = dev_pieces > 0 ? dev_pieces : MIXED_PIECES;
      if (dev_pieces > 0) {
        t.beta = 1.f;                     // X <- X + X (R^-1 - I), in place
        // the correction is |G| ~ 1e-5 of X: its FP32 accumulation over the
        // whole K range of a tile costs far less than FP32 rounding of X
        t.one_partial = 1;
      }
      rc = tc_gemm(ctx, op_rows(b, N, Ns, rowA, pieces), op_mat(b.matA, Ns, b, pieces),
                   products(pieces), t, EPI_TC_STORE, 1, ctx->stream);
    }
    if (rc) return rc;
    have_pieces = follows;
    if (keep) {
      ctx->pieces_X = X;
      ctx->pieces_Ns = Ns;
      ctx->pieces_rows = rowB;
    }
    if (follows) std::swap(rowA, rowB);
    if (shift_now) shift_now = false;
    else if (again) extra = true;       // the last pass once more
    else --plain_left;
  }
  return check_device_status(ctx);
}

// The pieces of X kept by the last Cholesky QR are still those of X.
static bool pieces_of(const sq3_ctx* ctx, const float* X, int Ns) {
  return ctx->reuse_pieces && ctx->pieces_X == X && ctx->pieces_Ns == Ns &&
         ctx->pieces_rows != nullptr;
}

int project_mixed(sq3_ctx* ctx, const float* X, int Ns, double* Hs) {
  const long long N = ctx->grid.N;
  MixedBuffers b;
  int rc = mixed_buffers(ctx, Ns, &b);
  if (rc) return rc;
  rc = ensure(&ctx->wsX, &ctx->wsX_bytes, (size_t)N * Ns * sizeof(float));
  if (rc) return rc;
  float* HX = (float*)ctx->wsX;
  ctx->hx_X = nullptr;
  rc = hamiltonian_apply_f32(ctx, X, HX, Ns);
  if (rc) return rc;
  if (ctx->reuse_pieces) {
    // keep H X (in wsX) and its potential for the next filter of this X
    if (!ctx->Vf_hx && cudaMalloc((void**)&ctx->Vf_hx, (size_t)N * sizeof(float)) != cudaSuccess) {
      cudaGetLastError();
      ctx->Vf_hx = nullptr;
    }
    if (ctx->Vf_hx) {
      cudaMemcpyAsync(ctx->Vf_hx, ctx->Vf, (size_t)N * sizeof(float), cudaMemcpyDeviceToDevice,
                      ctx->stream);
      ctx->hx_X = X;
      ctx->hx_Ns = Ns;
    }
  }
  if (!pieces_of(ctx, X, Ns)) split_block_cols(ctx, X, Ns, b.colX, b);
  split_block_cols(ctx, HX, Ns, b.colY, b);
  return gram_mixed(ctx, b.colX, b.colY, Ns, Hs, b, ST_HS_GEMM);
}

// Recurrence of Eq. (ThreeTermRecurrenceRelation) on the tensor cores; fills
// the FP32 T_j array for j = 0 .. h (h + 1 slots) and the moments m_0 .. m_h
// (FP64 traces).
int cheb_recurrence_mixed(sq3_ctx* ctx, const double* Hs, int Ns, int h,
                          const double* bounds, double* mom, float* T) {
  MixedBuffers b;
  int rc = mixed_buffers(ctx, Ns, &b);
  if (rc) return rc;
  const long long nn = (long long)Ns * Ns;
  {
    Prof p(ctx, ST_CHEB_GEMM, 2);
    hhat_f32_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, ctx->stream>>>(
        Hs, Ns, bounds, T, T + nn, mom);
    trace_f32_kernel<<<1, 1024, 0, ctx->stream>>>(T + nn, Ns, mom + 1);
  }
  split_matrix<float>(ctx, T + nn, Ns, b.matA, b);          // Hhat (A operand)
  {
    Prof p(ctx, ST_SPLIT);
    cudaMemcpyAsync(b.matB, b.matA, (size_t)MIXED_PIECES * b.psS * 2,
                    cudaMemcpyDeviceToDevice, ctx->stream);  // T_1 pieces
  }
  __nv_bfloat16* cur = b.matB;
  __nv_bfloat16* nxt = b.matC;
  Prof p(ctx, ST_CHEB_GEMM, h > 1 ? h - 1 : 0);
  for (int j = 1; j < h; ++j) {
    TcParams t{};
    t.C32 = T + (long long)(j + 1) * nn;
    t.ldc = Ns;
    t.Tprev = T + (long long)(j - 1) * nn;
    t.Bnext = nxt;
    t.ld_next = b.ldS;
    t.next_piece_stride = b.psS;
    t.next_pieces = MIXED_PIECES;
    t.trace = mom + j + 1;
    t.tri = 1;           // T_{j+1} is symmetric: upper tiles, each stored with its mirror
    rc = tc_gemm(ctx, op_mat(b.matA, Ns, b), op_mat(cur, Ns, b), products(MIXED_PIECES), t,
                 EPI_TC_CHEB, 1, ctx->stream);
    if (rc) return rc;
    __nv_bfloat16* tmp = cur; cur = nxt; nxt = tmp;
  }
  return SQ3_OK;
}

// m_{h+k} = tr(T_{h+k}) = 2 tr(T_h T_k) - m_{h-k} for k = 1 .. npl - h, by
// the product identity T_h T_k = (T_{h+k} + T_{h-k}) / 2; T_h and T_k are
// symmetric, so tr(T_h T_k) = sum_e T_h[e] T_k[e].  Block (k, s) sums the
// s-th of MT_SPLITS slices of the elements into part[(k-1) MT_SPLITS + s];
// moments_tail_finish_kernel adds the slices in order.
constexpr int MT_SPLITS = 16;
__global__ void __launch_bounds__(256)
moments_tail_kernel(const float* __restrict__ T, long long nn, int h, double* part) {
  __shared__ double sh[8];
  const int k = blockIdx.x + 1;
  const float* Th = T + (long long)h * nn;
  const float* Tk = T + (long long)k * nn;
  const long long chunk = (nn + MT_SPLITS - 1) / MT_SPLITS;
  const long long e0 = blockIdx.y * chunk;
  const long long e1 = e0 + chunk < nn ? e0 + chunk : nn;
  // FP32 products of the FP32 matrices in runs of 16 (FMA), each run folded
  // into the FP64 sum: GB300 issues few FP64 FMAs per SM, and the entries
  // are FP32 already
  double s = 0.0;
  long long e = e0 + threadIdx.x;
  while (e < e1) {
    float r = 0.f;
#pragma unroll 4
    for (int i = 0; i < 16 && e < e1; ++i, e += blockDim.x) r = fmaf(Th[e], Tk[e], r);
    s += (double)r;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += sh[w];
    part[(long long)(k - 1) * MT_SPLITS + blockIdx.y] = t;
  }
}

__global__ void moments_tail_finish_kernel(const double* part, int h, int K, double* mom) {
  for (int k = 1 + blockIdx.x * blockDim.x + threadIdx.x; k <= K; k += gridDim.x * blockDim.x) {
    double t = 0.0;
    for (int s = 0; s < MT_SPLITS; ++s) t += part[(long long)(k - 1) * MT_SPLITS + s];
    mom[h + k] = 2.0 * t - mom[h - k];
  }
}

size_t moments_tail_part_words(int npl, int h) {
  return npl > h ? (size_t)(npl - h) * MT_SPLITS : 0;
}

int moments_tail_mixed(sq3_ctx* ctx, const float* T, int Ns, int npl, int h, double* mom,
                       double* part) {
  if (npl <= h) return SQ3_OK;
  const int K = npl - h;
  moments_tail_kernel<<<dim3(K, MT_SPLITS), 256, 0, ctx->stream>>>(T, (long long)Ns * Ns, h,
                                                                   part);
  moments_tail_finish_kernel<<<(K + 255) / 256, 256, 0, ctx->stream>>>(part, h, K, mom);
  return cuda_err(cudaGetLastError());
}

// D = sum'_{j<=h} c_j T_j - sum_{k=1}^{npl-h} c_{h+k} T_{h-k} and
// A2 = 2 sum_{k=1}^{npl-h} c_{h+k} T_k (FP32), so that Ds = D + T_h A2.  The
// two sums over T_0 .. T_h are folded into one weight per T_t,
// w_t = c_t - c_{2h-t} [h - t <= npl - h] (w_0 with c_0 / 2; T_0 = I is
// stored), so each T_t is read once.  The terms are FP32 products of the
// FP32 T_t (weights rounded to FP32) summed in runs of 8 and each run
// folded into an FP64 sum: GB300 issues few FP64 FMAs per SM, and the T_t
// carry FP32 accuracy already.
__global__ void __launch_bounds__(256)
d_split_kernel(const float* __restrict__ T, long long nn, int npl, int h,
               const double* __restrict__ coef, double* D, float* A2) {
  __shared__ float w[SQ3_MAX_NPL + 1];
  __shared__ float ca[SQ3_MAX_NPL + 1];
  const int K = npl - h;
  for (int t = threadIdx.x; t <= h; t += blockDim.x) {
    double v = (t == 0 ? 0.5 : 1.0) * coef[t];
    if (t < h && h - t <= K) v -= coef[2 * h - t];
    w[t] = (float)v;
    ca[t] = (t >= 1 && t <= K) ? (float)coef[h + t] : 0.f;
  }
  __syncthreads();
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= nn) return;
  double d = 0.0, a = 0.0;
  for (int t0 = 0; t0 <= h; t0 += 8) {
    float dr = 0.f, ar = 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int t = t0 + i;
      if (t <= h) {
        const float x = T[(long long)t * nn + e];
        dr = fmaf(w[t], x, dr);
        ar = fmaf(ca[t], x, ar);
      }
    }
    d += (double)dr;
    a += (double)ar;
  }
  D[e] = d;
  A2[e] = (float)(2.0 * a);
}

// Ds = sum'_{j<=npl} c_j T_j from T_0 .. T_h (Eq. (ChebyshevExpansion)),
// with the terms j > h folded into one tensor-core product T_h A2.
int accumulate_d_mixed(sq3_ctx* ctx, const float* T, int Ns, int npl, int h,
                       const double* coef, double* D, float* A2) {
  const long long nn = (long long)Ns * Ns;
  MixedBuffers b;
  int rc = mixed_buffers(ctx, Ns, &b);
  if (rc) return rc;
  {
    Prof p(ctx, ST_D_ACCUM);
    d_split_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, ctx->stream>>>(
        T, nn, npl, h, coef, D, A2);
  }
  if (npl <= h) return cuda_err(cudaGetLastError());
  split_matrix<float>(ctx, T + (long long)h * nn, Ns, b.matA, b);   // T_h
  split_matrix<float>(ctx, A2, Ns, b.matB, b);                      // A2
  Prof p(ctx, ST_D_ACCUM);
  TcParams t{};
  t.C64 = D;
  t.ldc = Ns;
  t.tri = 1;             // T_h A2 is symmetric (both are polynomials of Hhat)
  rc = tc_gemm(ctx, op_mat(b.matA, Ns, b), op_mat(b.matB, Ns, b), products(MIXED_PIECES), t,
               EPI_TC_ATOMIC, 1, ctx->stream);
  if (rc) return rc;
  mirror_upper_f64(D, Ns, ctx->stream);
  return cuda_err(cudaGetLastError());
}

int density_mixed(sq3_ctx* ctx, const float* X, const double* D, int Ns, double* rho) {
  const long long N = ctx->grid.N;
  MixedBuffers b;
  int rc = mixed_buffers(ctx, Ns, &b);
  if (rc) return rc;
  {
    // x Ds x^T with Ds symmetric: the upper-triangular form halves the product
    Prof p(ctx, ST_SPLIT);
    split_upper_twice_kernel<<<grid_for((long long)Ns * Ns), 256, 0, ctx->stream>>>(
        D, Ns, b.matA, b.ldS, b.psS, MIXED_PIECES);
  }
  const __nv_bfloat16* rows = b.rowX;
  if (pieces_of(ctx, X, Ns)) rows = (const __nv_bfloat16*)ctx->pieces_rows;
  else split_block_rows(ctx, X, Ns, b);
  Prof p(ctx, ST_RHO);
  cudaMemsetAsync(rho, 0, (size_t)N * sizeof(double), ctx->stream);
  TcParams t{};
  t.X = X;
  t.ldx = N;
  t.rho = rho;
  t.rho_alpha = 2.0 / ctx->dV;
  t.tri = 2;                                         // B upper triangular
  return tc_gemm(ctx, op_rows(b, N, Ns, rows), op_mat(b.matA, Ns, b), products(MIXED_PIECES), t,
                 EPI_TC_RHO, 1, ctx->stream);
}

// ---------------------------------------------------------------------------
// Paterson-Stockmeyer evaluation of the expansion on the tensor cores (the
// mixed path's form of foe.cu's FP64 one; the same identities):
//   baby steps    T_0 .. T_s by the recurrence in Hhat
//   giant steps   G_q = T_q(Y) = T_{qs}, Y = T_s: G_{q+1} = 2 Y G_q - G_{q-1}
//   moments       m_{qs+r} = 2 <G_q, T_r> - m_{qs-r}
//   kernel        Ds = sum_q A_q T_q(Y), A_q = sum_{r<s} alpha_{qr} T_r, by
//                 Clenshaw's recurrence b_q = A_q + 2 Y b_{q+1} - b_{q+2},
//                 Ds = A_0 + Y b_1 - b_2.
// Matrices in FP32, every product a tcgen05 GEMM of BF16 pieces with the
// Chebyshev epilogue (C = 2 acc - P, its pieces for the next product, its
// trace); (s - 1) + (Q - 1) + Q products instead of the recurrence's
// ceil(npl / 2).  Workspace W (FP32 matrices, then doubles):
//   T_0 .. T_s | G_2 .. G_Q | b[3] | P | part | alpha | work | trace scratch
//   | pointers to G_0 .. G_Q
// ---------------------------------------------------------------------------
struct PsMixed {
  float* baby;
  float* giant;
  float* b[3];
  float* P;
  double* part;
  double* alpha;
  double* work;
  double* scratch;
  const float** gptr;
};

static PsMixed ps_mixed_ws(void* W, long long nn, int s, int Q) {
  PsMixed w;
  float* f = (float*)W;
  w.baby = f; f += (long long)(s + 1) * nn;
  w.giant = f; f += (long long)std::max(Q - 1, 0) * nn;
  for (int k = 0; k < 3; ++k) { w.b[k] = f; f += nn; }
  w.P = f; f += nn;
  double* d = (double*)(((uintptr_t)f + 15) & ~(uintptr_t)15);
  w.part = d; d += (size_t)std::max(Q, 1) * s * PS_FROB_BLOCKS;
  w.alpha = d; d += (size_t)(Q + 1) * s;
  w.work = d; d += (size_t)(Q + 1) * s;
  w.scratch = d; d += 2;
  w.gptr = (const float**)d;
  return w;
}

size_t ps_mixed_bytes(int Ns, int s, int Q) {
  const long long nn = (long long)Ns * Ns;
  const size_t mats = (size_t)(s + 1) + (size_t)std::max(Q - 1, 0) + 4;
  return mats * nn * sizeof(float) + 16 +
         ((size_t)std::max(Q, 1) * s * PS_FROB_BLOCKS + 2 * (size_t)(Q + 1) * s + 2) *
             sizeof(double) +
         (size_t)(Q + 2) * sizeof(float*);
}

// part[pair PS_FROB_BLOCKS + b]: block b's share of <G_q, T_r>, pair =
// (q - 1)(s - 1) + (r - 1); FP32 products in runs of 16 folded into FP64.
__global__ void __launch_bounds__(256)
ps_frob_f32_kernel(const float* const* __restrict__ gq, const float* __restrict__ T,
                   long long nn, int s, double* part) {
  __shared__ double sh[8];
  const int pair = blockIdx.x / PS_FROB_BLOCKS, blk = blockIdx.x % PS_FROB_BLOCKS;
  const int q = pair / (s - 1) + 1, r = pair % (s - 1) + 1;
  const float* A = gq[q];
  const float* B = T + (long long)r * nn;
  const long long stride = (long long)PS_FROB_BLOCKS * blockDim.x;
  double acc = 0.0;
  long long e = (long long)blk * blockDim.x + threadIdx.x;
  while (e < nn) {
    float run = 0.f;
    for (int i = 0; i < 16 && e < nn; ++i, e += stride) run = fmaf(A[e], B[e], run);
    acc += (double)run;
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

// out = ea E + eb Bm + as sum_{r<s} alpha[r] T_r, into FP32 out32 or FP64
// out64 (one of them); the sum over r in FP32 runs of 8 folded into FP64.
constexpr int PS_MAX_S = 64;
__global__ void __launch_bounds__(256)
ps_combine_f32_kernel(float* out32, double* out64, const float* E, double ea, const float* Bm,
                      double eb, double as, const float* __restrict__ T, long long nn, int s,
                      const double* __restrict__ alpha) {
  __shared__ float al[PS_MAX_S];
  for (int r = threadIdx.x; r < s; r += blockDim.x) al[r] = (float)alpha[r];
  __syncthreads();
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nn;
       e += (long long)gridDim.x * blockDim.x) {
    double v = 0.0;
    for (int r0 = 0; r0 < s; r0 += 8) {
      float run = 0.f;
#pragma unroll
      for (int i = 0; i < 8; ++i)
        if (r0 + i < s) run = fmaf(al[r0 + i], T[(long long)(r0 + i) * nn + e], run);
      v += (double)run;
    }
    v *= as;
    if (E) v += ea * (double)E[e];
    if (Bm) v += eb * (double)Bm[e];
    if (out64) out64[e] = v;
    else out32[e] = (float)v;
  }
}

// C = 2 Y B - P on the tensor cores (symmetric operands that commute: upper
// tiles, mirrored), with the pieces of C into Cp and its trace into tr.
static int ps_product(sq3_ctx* ctx, const MixedBuffers& b, const __nv_bfloat16* Yp,
                      const __nv_bfloat16* Bp, const float* P, float* C, __nv_bfloat16* Cp,
                      double* tr, int Ns) {
  TcParams t{};
  t.C32 = C;
  t.ldc = Ns;
  t.Tprev = P;
  t.Bnext = Cp;
  t.ld_next = b.ldS;
  t.next_piece_stride = b.psS;
  t.next_pieces = MIXED_PIECES;
  t.trace = tr;
  t.tri = 1;
  return tc_gemm(ctx, op_mat(Yp, Ns, b), op_mat(Bp, Ns, b), products(MIXED_PIECES), t,
                 EPI_TC_CHEB, 1, ctx->stream);
}

int ps_moments_mixed(sq3_ctx* ctx, const double* Hs, int Ns, int npl, int s, int Q,
                     const double* bounds, double* mom, void* W) {
  if (s < 2 || s > PS_MAX_S) return SQ3_EINVAL;
  MixedBuffers b;
  int rc = mixed_buffers(ctx, Ns, &b);
  if (rc) return rc;
  cudaStream_t st = ctx->stream;
  const long long nn = (long long)Ns * Ns;
  const PsMixed w = ps_mixed_ws(W, nn, s, Q);
  const int sb = std::min(s, npl);            // baby steps needed for the moments
  {
    Prof p(ctx, ST_CHEB_GEMM, 2);
    hhat_f32_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, st>>>(Hs, Ns, bounds, w.baby,
                                                                  w.baby + nn, mom);
    trace_f32_kernel<<<1, 1024, 0, st>>>(w.baby + nn, Ns, mom + 1);
  }
  split_matrix<float>(ctx, w.baby + nn, Ns, b.matA, b);          // Hhat
  __nv_bfloat16* cur = b.matB;
  __nv_bfloat16* nxt = b.matC;
  {
    Prof p(ctx, ST_SPLIT);
    cudaMemcpyAsync(cur, b.matA, (size_t)MIXED_PIECES * b.psS * 2, cudaMemcpyDeviceToDevice,
                    st);                                          // T_1
  }
  {
    Prof p(ctx, ST_CHEB_GEMM, std::max(sb - 1, 0));
    for (int j = 1; j < sb; ++j) {
      rc = ps_product(ctx, b, b.matA, cur, w.baby + (long long)(j - 1) * nn,
                      w.baby + (long long)(j + 1) * nn, nxt, mom + j + 1, Ns);
      if (rc) return rc;
      std::swap(cur, nxt);
    }
  }
  if (Q < 1) return cuda_err(cudaGetLastError());
  // giant steps in Y = T_s (its pieces in matA from here on)
  const float* Y = w.baby + (long long)s * nn;
  split_matrix<float>(ctx, Y, Ns, b.matA, b);
  std::vector<const float*> g(Q + 1);
  g[0] = w.baby;
  g[1] = Y;
  for (int q = 2; q <= Q; ++q) g[q] = w.giant + (long long)(q - 2) * nn;
  {
    Prof p(ctx, ST_SPLIT);
    cudaMemcpyAsync(cur, b.matA, (size_t)MIXED_PIECES * b.psS * 2, cudaMemcpyDeviceToDevice,
                    st);                                          // G_1 = Y
  }
  {
    Prof p(ctx, ST_CHEB_GEMM, std::max(Q - 1, 0));
    for (int q = 1; q < Q; ++q) {
      rc = ps_product(ctx, b, b.matA, cur, g[q - 1], const_cast<float*>(g[q + 1]), nxt,
                      mom + (long long)(q + 1) * s, Ns);
      if (rc) return rc;
      std::swap(cur, nxt);
    }
  }
  rc = cuda_err(cudaMemcpyAsync(w.gptr, g.data(), (Q + 1) * sizeof(float*),
                                cudaMemcpyHostToDevice, st));
  if (rc) return rc;
  {
    Prof p(ctx, ST_CHEB_GEMM, 2);
    ps_frob_f32_kernel<<<Q * (s - 1) * PS_FROB_BLOCKS, 256, 0, st>>>(w.gptr, w.baby, nn, s,
                                                                     w.part);
    ps_moments_finish(w.part, s, Q, npl, mom, st);
  }
  // the host vector g is read by the copy above: wait for it before it goes
  return cuda_err(cudaStreamSynchronize(st));
}

int ps_kernel_mixed(sq3_ctx* ctx, int Ns, int npl, int s, int Q, const double* coef, void* W,
                    double* D) {
  MixedBuffers b;
  int rc = mixed_buffers(ctx, Ns, &b);
  if (rc) return rc;
  cudaStream_t st = ctx->stream;
  const long long nn = (long long)Ns * Ns;
  const PsMixed w = ps_mixed_ws(W, nn, s, Q);
  const int sb = std::min(s, npl + 1);        // T_0 .. T_{sb-1} carry the A_q
  const unsigned blocks = (unsigned)std::min<long long>((nn + 255) / 256, 152LL * 8);
  Prof pd(ctx, ST_D_ACCUM, 2 + 2 * Q);
  ps_alpha(coef, npl, s, Q, w.work, w.alpha, st);
  if (Q == 0) {
    ps_combine_f32_kernel<<<blocks, 256, 0, st>>>(nullptr, D, nullptr, 0.0, nullptr, 0.0, 1.0,
                                                  w.baby, nn, sb, w.alpha);
    return cuda_err(cudaGetLastError());
  }
  split_matrix<float>(ctx, w.baby + (long long)s * nn, Ns, b.matA, b);   // Y = T_s
  float* bq1 = w.b[0];      // b_{q+1}
  float* bq2 = w.b[1];      // b_{q+2}
  float* bq = w.b[2];
  cudaMemsetAsync(bq2, 0, nn * sizeof(float), st);
  // b_Q = A_Q
  ps_combine_f32_kernel<<<blocks, 256, 0, st>>>(bq1, nullptr, nullptr, 0.0, nullptr, 0.0, 1.0,
                                                w.baby, nn, s, w.alpha + (size_t)Q * s);
  split_matrix<float>(ctx, bq1, Ns, b.matB, b);
  __nv_bfloat16* cur = b.matB;
  __nv_bfloat16* nxt = b.matC;
  for (int q = Q - 1; q >= 1; --q) {
    // b_q = 2 Y b_{q+1} - P with P = b_{q+2} - A_q
    ps_combine_f32_kernel<<<blocks, 256, 0, st>>>(w.P, nullptr, bq2, 1.0, nullptr, 0.0, -1.0,
                                                  w.baby, nn, s, w.alpha + (size_t)q * s);
    rc = ps_product(ctx, b, b.matA, cur, w.P, bq, nxt, w.scratch, Ns);
    if (rc) return rc;
    std::swap(cur, nxt);
    float* t = bq2;
    bq2 = bq1;
    bq1 = bq;
    bq = t;
  }
  // Ds = A_0 + Y b_1 - b_2 = (2 Y b_1 - b_2) / 2 - b_2 / 2 + A_0
  rc = ps_product(ctx, b, b.matA, cur, bq2, bq, nxt, w.scratch, Ns);
  if (rc) return rc;
  ps_combine_f32_kernel<<<blocks, 256, 0, st>>>(nullptr, D, bq, 0.5, bq2, -0.5, 1.0, w.baby, nn,
                                                sb, w.alpha);
  return cuda_err(cudaGetLastError());
}

}  // namespace sq3
