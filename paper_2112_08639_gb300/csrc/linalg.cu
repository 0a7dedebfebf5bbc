// Dense FP64 linear algebra on the device for the orthonormalisation and
// spectral-bound steps.
//
// * Blocked right-looking Cholesky S = L L^T (64-wide panels: one-CTA panel
//   factorisation, row-parallel triangular solve for the panel below, GEMM
//   update of the trailing matrix).  Used for Cholesky QR, the
//   orthonormalisation that follows the Chebyshev filter (Sec. 4).
// * R^{-1} = L^{-T} by column-parallel forward substitution.
// * Lanczos extremal eigenvalue estimates of Hs for chi and xi of
//   Eq. (ChebyshevExpansion) (the paper takes them from lambda_1 and
//   lambda_Ns of Hs without saying how they are obtained).
#include <math.h>

#include <mutex>

#include "sq3_internal.cuh"

namespace sq3 {

constexpr int CH_NB = 64;

__device__ inline void set_status(int* st, int code) {
  atomicCAS(st, 0, code);
}

__global__ void copy_diag_kernel(const double* S, int n, double* d) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) d[i] = S[i + (long long)i * n];
}

// Factor the kb x kb diagonal block at (k0, k0) of the column-major n x n S.
// A pivot that is not above 1e-13 times the original diagonal entry diag0
// (numerically rank-deficient X) or is not finite sets DEV_NOTPD.  The
// shared block A keeps the running Schur complement; step j reads column j
// of A, writes column j of the factor straight to S and updates the trailing
// part of A, so one barrier per column suffices.
__global__ void __launch_bounds__(256)
potrf_diag_kernel(double* S, int n, int k0, int kb, const double* diag0,
                  int* status) {
  __shared__ double A[CH_NB][CH_NB + 1];
  __shared__ double d0[CH_NB];
  for (int e = threadIdx.x; e < kb * kb; e += blockDim.x) {
    int i = e % kb, j = e / kb;
    A[i][j] = S[(k0 + i) + (long long)(k0 + j) * n];
  }
  for (int i = threadIdx.x; i < kb; i += blockDim.x) d0[i] = diag0[k0 + i];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nw = blockDim.x >> 5;
  for (int j = 0; j < kb; ++j) {
    double d = A[j][j];
    if (!(d > 1e-13 * d0[j]) || !isfinite(d)) {
      if (threadIdx.x == 0) set_status(status, DEV_NOTPD);
      d = 1.0;
    }
    // one square root and one division per column; the rest multiplies
    const double sd = sqrt(d), rsd = 1.0 / sd, inv = rsd * rsd;
    for (int i = j + threadIdx.x; i < kb; i += blockDim.x)
      S[(k0 + i) + (long long)(k0 + j) * n] = (i == j) ? sd : A[i][j] * rsd;
    // trailing lower triangle: warp w takes columns l = j+1+w, j+1+w+nw, ..,
    // its lanes the rows i >= l (no index division)
    for (int l = j + 1 + warp; l < kb; l += nw) {
      const double alj = A[l][j] * inv;
      for (int i = l + lane; i < kb; i += 32) A[i][l] -= A[i][j] * alj;
    }
    __syncthreads();
  }
}

// L21 = S21 L11^{-T}: each thread solves one row of the panel below the
// diagonal block by forward substitution.
__global__ void __launch_bounds__(128)
trsm_panel_kernel(double* S, int n, int k0, int kb) {
  __shared__ double L[CH_NB][CH_NB + 1];
  for (int e = threadIdx.x; e < kb * kb; e += blockDim.x) {
    int i = e % kb, j = e / kb;
    L[i][j] = (i >= j) ? S[(k0 + i) + (long long)(k0 + j) * n] : 0.0;
  }
  __syncthreads();
  const int i = k0 + kb + blockIdx.x * blockDim.x + threadIdx.x;
  const bool ok = i < n;
  double x[CH_NB];
#pragma unroll
  for (int c = 0; c < CH_NB; ++c)
    x[c] = (ok && c < kb) ? S[i + (long long)(k0 + c) * n] : 0.0;
#pragma unroll
  for (int c = 0; c < CH_NB; ++c) {
    if (c < kb) {
      double s = x[c];
#pragma unroll
      for (int j = 0; j < c; ++j) s -= x[j] * L[c][j];
      x[c] = s / L[c][c];
    }
  }
  if (ok) {
#pragma unroll
    for (int c = 0; c < CH_NB; ++c)
      if (c < kb) S[i + (long long)(k0 + c) * n] = x[c];
  }
}

int cholesky_lower_f64(sq3_ctx* ctx, double* S, int n, double* diag_ws,
                       cudaStream_t st) {
  copy_diag_kernel<<<(n + 255) / 256, 256, 0, st>>>(S, n, diag_ws);
  for (int k0 = 0; k0 < n; k0 += CH_NB) {
    const int kb = (n - k0 < CH_NB) ? n - k0 : CH_NB;
    potrf_diag_kernel<<<1, 256, 0, st>>>(S, n, k0, kb, diag_ws,
                                         ctx->dev_status);
    const int m2 = n - k0 - kb;
    if (m2 <= 0) continue;
    trsm_panel_kernel<<<(m2 + 127) / 128, 128, 0, st>>>(S, n, k0, kb);
    GemmArgs g{};
    g.M = m2; g.N = m2; g.K = kb;
    g.A = S + (k0 + kb) + (long long)k0 * n; g.lda = n; g.a_kcontig = false;
    g.B = S + (k0 + kb) + (long long)k0 * n; g.ldb = n; g.b_kcontig = false;
    g.C = S + (k0 + kb) + (long long)(k0 + kb) * n; g.ldc = n;
    g.alpha = -1.0; g.beta = 1.0; g.splits = 1;
    g.tri = 3;                 // later panels read only the lower triangle
    gemm_f64(g, EPI_STORE, st);
  }
  return cuda_err(cudaGetLastError());
}

// Column j of W = L^{-1} by forward substitution, written as row j of
// Rinv = W^T (column-major, upper triangular).
__global__ void __launch_bounds__(256)
tri_inv_kernel(const double* __restrict__ L, double* Rinv, int n) {
  extern __shared__ double r[];
  const int j = blockIdx.x;
  for (int i = threadIdx.x; i < n; i += blockDim.x) r[i] = (i == j) ? 1.0 : 0.0;
  __syncthreads();
  for (int i = j; i < n; ++i) {
    const double wi = r[i] / L[i + (long long)i * n];
    __syncthreads();
    if (threadIdx.x == 0) r[i] = wi;
    for (int k = i + 1 + threadIdx.x; k < n; k += blockDim.x)
      r[k] -= L[k + (long long)i * n] * wi;
    __syncthreads();
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    Rinv[j + (long long)i * n] = (i >= j) ? r[i] : 0.0;
}

// Same result with TRI_WPB columns per CTA, one warp each, walking the rows
// i together: column i of L (below the diagonal) is copied into shared
// memory once per step for all the CTA's columns, and 1/L_ii comes from a
// precomputed array, so a step costs one coalesced column read and two
// block barriers.
constexpr int TRI_WPB = 8;
__global__ void __launch_bounds__(32 * TRI_WPB)
tri_inv_block_kernel(const double* __restrict__ L, const double* __restrict__ inv_diag,
                     double* Rinv, int n) {
  extern __shared__ double sm[];
  double* lc = sm;                          // n : current column of L
  double* rw = sm + n;                      // TRI_WPB x n
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int j0 = blockIdx.x * TRI_WPB;
  const int j = j0 + warp;
  double* r = rw + (size_t)warp * n;
  for (int i = lane; i < n; i += 32) r[i] = (i == j) ? 1.0 : 0.0;
  for (int i = j0; i < n; ++i) {
    __syncthreads();                        // previous column consumed
    for (int k = i + 1 + threadIdx.x; k < n; k += blockDim.x) lc[k] = L[k + (long long)i * n];
    __syncthreads();
    if (j < n && i >= j) {
      const double wi = r[i] * inv_diag[i];
      __syncwarp();
      if (lane == 0) r[i] = wi;
      for (int k = i + 1 + lane; k < n; k += 32) r[k] -= lc[k] * wi;
    }
  }
  __syncthreads();
  if (j < n)
    for (int i = lane; i < n; i += 32) Rinv[j + (long long)i * n] = (i >= j) ? r[i] : 0.0;
}

__global__ void inv_diag_kernel(const double* L, int n, double* d) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) d[i] = 1.0 / L[i + (long long)i * n];
}

void tri_inverse_transpose_f64(const double* L, double* Rinv, int n,
                               double* diag_ws, cudaStream_t st) {
  const size_t wsm = (size_t)(TRI_WPB + 1) * n * sizeof(double);
  if (wsm <= 200 * 1024) {
    if (wsm > 48 * 1024)
      cudaFuncSetAttribute(tri_inv_block_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)wsm);
    inv_diag_kernel<<<(n + 255) / 256, 256, 0, st>>>(L, n, diag_ws);
    tri_inv_block_kernel<<<(n + TRI_WPB - 1) / TRI_WPB, 32 * TRI_WPB, wsm, st>>>(
        L, diag_ws, Rinv, n);
    return;
  }
  size_t smem = (size_t)n * sizeof(double);
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(tri_inv_kernel,
                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
  tri_inv_kernel<<<n, 256, smem, st>>>(L, Rinv, n);
}

__global__ void symmetrize_kernel(double* A, int n) {
  long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= (long long)n * n) return;
  int i = (int)(e % n), j = (int)(e / n);
  if (i < j) {
    double a = A[i + (long long)j * n], b = A[j + (long long)i * n];
    double s = 0.5 * (a + b);
    A[i + (long long)j * n] = s;
    A[j + (long long)i * n] = s;
  }
}

__global__ void mirror_upper_kernel(double* A, int n) {
  long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= (long long)n * n) return;
  int i = (int)(e % n), j = (int)(e / n);
  if (i > j) A[e] = A[j + (long long)i * n];
}

void mirror_upper_f64(double* A, int n, cudaStream_t st) {
  long long tot = (long long)n * n;
  mirror_upper_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(A, n);
}

void symmetrize_f64(double* A, int n, cudaStream_t st) {
  long long tot = (long long)n * n;
  symmetrize_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(A, n);
}

// ---------------------------------------------------------------------------
// Lanczos with full reorthogonalisation on the symmetric Hs.
// work layout: V[(steps+1) * n] | w[n] | alpha[steps] | beta[steps] | k[1]
// ---------------------------------------------------------------------------
__device__ inline double hash_unit(unsigned i) {
  unsigned h = i * 2654435761u + 0x9e3779b9u;
  h ^= h >> 16; h *= 0x85ebca6bu; h ^= h >> 13; h *= 0xc2b2ae35u; h ^= h >> 16;
  return (double)h / 4294967296.0 - 0.5;
}

__device__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double s = 0.0;
  const int nw = (blockDim.x + 31) >> 5;
  for (int w = 0; w < nw; ++w) s += sh[w];
  return s;
}

__global__ void __launch_bounds__(1024)
lanczos_init_kernel(double* V, int n, double* kcount) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double v = hash_unit((unsigned)i) + 0.25;
    V[i] = v;
    s += v * v;
  }
  s = block_sum(s, sh);
  const double inv = 1.0 / sqrt(s);
  for (int i = threadIdx.x; i < n; i += blockDim.x) V[i] *= inv;
  if (threadIdx.x == 0) kcount[0] = 0.0;
}

// One Lanczos step j is five grid-wide launches over the n components
// (LZ_T per block): w = Hs v_j with alpha_j = v_j^T w; the three-term
// update with the first reorthogonalisation pass's projections; two
// classical Gram-Schmidt passes against v_0 .. v_j (all projections of a
// pass computed at once); beta_j and v_{j+1}.  Each block writes its
// partial sums to its own slot and the next launch adds the slots in a
// fixed order, so the result does not depend on the order in which blocks
// run.  Every kernel returns at once after termination (kcount < j).
constexpr int LZ_T = 256;
constexpr int LZ_MAXQ = 64;                          // basis vectors (steps) at most

struct LzParts {
  double* alpha;                                     // [gr]   symv blocks
  double* h1;                                        // [gv][LZ_MAXQ]
  double* h2;                                        // [gv][LZ_MAXQ]
  double* b2;                                        // [gv]
};

// Sum of the m values p[0], p[stride], ... by the whole block (fixed order).
__device__ double block_sum_parts(const double* p, int m, long long stride, double* sh) {
  double s = 0.0;
  for (int k = threadIdx.x; k < m; k += blockDim.x) s += p[k * stride];
  return block_sum(s, sh);
}

// w = Hs v: one warp per output row (Hs symmetric, so row i = column i);
// the block's share of alpha = v^T w into its slot.
__global__ void __launch_bounds__(LZ_T)
symv_alpha_kernel(const double* __restrict__ Hs, const double* __restrict__ v,
                  double* w, int n, const double* kcount, int j, double* apart) {
  __shared__ double sh[LZ_T / 32];
  if (kcount[0] < j) return;  // Lanczos already terminated
  const int row = (blockIdx.x * LZ_T + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  double s = 0.0;
  if (row < n) {
    const double* col = Hs + (long long)row * n;
    for (int k = lane; k < n; k += 32) s += col[k] * v[k];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  }
  if (lane == 0) {
    if (row < n) w[row] = s;
    sh[threadIdx.x >> 5] = row < n ? s * v[row] : 0.0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0;
    for (int k = 0; k < LZ_T / 32; ++k) a += sh[k];
    apart[blockIdx.x] = a;
  }
}

// The block's partial sums of d_q (q = 0 .. nq-1, one value per thread each)
// into out[blockIdx.x * LZ_MAXQ + q].
__device__ void block_dots(const double* V, long long n, int i, double t, int nq, double* out) {
  __shared__ double sh[LZ_MAXQ][LZ_T / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int q = 0; q < nq; ++q) {
    double d = i < n ? V[(long long)q * n + i] * t : 0.0;
    for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
    if (lane == 0) sh[q][wid] = d;
  }
  __syncthreads();
  if (threadIdx.x < nq) {
    double d = 0.0;
    for (int k = 0; k < LZ_T / 32; ++k) d += sh[threadIdx.x][k];
    out[(long long)blockIdx.x * LZ_MAXQ + threadIdx.x] = d;
  }
}

// w -= alpha_j v_j + beta_{j-1} v_{j-1}; projections of the result on v_0..v_j.
__global__ void __launch_bounds__(LZ_T)
lanczos_three_term_kernel(const double* V, double* w, const double* beta, int n, int j,
                          const double* kcount, LzParts P, int gr) {
  __shared__ double sh[32];
  if (kcount[0] < j) return;
  const double a = block_sum_parts(P.alpha, gr, 1, sh);
  const int i = blockIdx.x * LZ_T + threadIdx.x;
  double t = 0.0;
  if (i < n) {
    t = w[i] - a * V[(long long)j * n + i];
    if (j > 0) t -= beta[j - 1] * V[(long long)(j - 1) * n + i];
    w[i] = t;
  }
  block_dots(V, n, i, t, j + 1, P.h1);
}

// One Gram-Schmidt pass with the projections summed from the blocks' slots
// (hin): w -= sum_q h_q v_q; then the projections of the result (hout), or
// after the last pass the block's share of |w|^2.
__global__ void __launch_bounds__(LZ_T)
lanczos_reorth_kernel(const double* V, double* w, int n, int j, const double* kcount,
                      const double* hin, double* hout, double* b2part, int gv) {
  __shared__ double hs[LZ_MAXQ];
  __shared__ double sh[LZ_T / 32];
  if (kcount[0] < j) return;
  if (threadIdx.x <= j) {
    double h = 0.0;
    for (int k = 0; k < gv; ++k) h += hin[(long long)k * LZ_MAXQ + threadIdx.x];
    hs[threadIdx.x] = h;
  }
  __syncthreads();
  const int i = blockIdx.x * LZ_T + threadIdx.x;
  double t = 0.0;
  if (i < n) {
    t = w[i];
    for (int q = 0; q <= j; ++q) t -= hs[q] * V[(long long)q * n + i];
    w[i] = t;
  }
  if (hout) {
    block_dots(V, n, i, t, j + 1, hout);
    return;
  }
  double b = t * t;
  for (int o = 16; o > 0; o >>= 1) b += __shfl_xor_sync(0xffffffffu, b, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = b;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < LZ_T / 32; ++k) s += sh[k];
    b2part[blockIdx.x] = s;
  }
}

// beta_j = |w|, the termination test, v_{j+1} = w / beta_j; block 0 records
// alpha_j, beta_j and the step count.
__global__ void __launch_bounds__(LZ_T)
lanczos_next_kernel(double* V, const double* w, double* alpha, double* beta, double* kcount,
                    int n, int j, LzParts P, int gr, int gv) {
  __shared__ double sh[32];
  if (kcount[0] < j) return;
  const double a = block_sum_parts(P.alpha, gr, 1, sh);
  const double b = sqrt(block_sum_parts(P.b2, gv, 1, sh));
  const double scale = fabs(a) + b;
  const bool stop = b <= 1e-12 * (scale > 0 ? scale : 1.0) || j + 1 >= n;
  const int i = blockIdx.x * LZ_T + threadIdx.x;
  if (!stop && i < n) V[(long long)(j + 1) * n + i] = w[i] / b;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    alpha[j] = a;
    beta[j] = b;
    kcount[0] = stop ? -(double)(j + 1) : (double)(j + 1);
  }
}

// Number of eigenvalues of the k x k tridiagonal (alpha, beta) below x.
__device__ int sturm_count(const double* al, const double* be, int k, double x) {
  int cnt = 0;
  double d = al[0] - x;
  if (d < 0) ++cnt;
  for (int i = 1; i < k; ++i) {
    if (d == 0.0) d = 1e-300;
    d = al[i] - x - be[i - 1] * be[i - 1] / d;
    if (d < 0) ++cnt;
  }
  return cnt;
}

// |last component| of the normalised eigenvector of T for eigenvalue th.
__device__ double last_component(const double* al, const double* be, int k,
                                 double th) {
  if (k == 1) return 1.0;
  double sp = 0.0, s = 1.0, nrm2 = 1.0;
  for (int i = 0; i < k - 1; ++i) {
    double bi = be[i] != 0.0 ? be[i] : 1e-300;
    double sn = ((th - al[i]) * s - (i > 0 ? be[i - 1] * sp : 0.0)) / bi;
    sp = s; s = sn;
    nrm2 += s * s;
    if (nrm2 > 1e200) { sp *= 1e-100; s *= 1e-100; nrm2 *= 1e-200; }
  }
  double r = fabs(s) / sqrt(nrm2);
  return r > 1.0 ? 1.0 : r;
}

// Extremal eigenvalue of the tridiagonal by multisection: 32 lanes test 32
// interior points per round, shrinking the bracket 33-fold.  `target` is the
// number of eigenvalues that must lie below the returned point's right end:
// 1 for the smallest, k for the largest.
__device__ double multisect(const double* al, const double* be, int k, double lo,
                            double hi, int target) {
  const int lane = threadIdx.x & 31;
  for (int it = 0; it < 40; ++it) {
    const double x = lo + (hi - lo) * (lane + 1) / 33.0;
    const bool ge = sturm_count(al, be, k, x) >= target;
    const unsigned m = __ballot_sync(0xffffffffu, ge);
    const int first = m ? __ffs(m) - 1 : 32;       // first lane with count >= target
    const double nlo = first == 0 ? lo : lo + (hi - lo) * first / 33.0;
    const double nhi = first == 32 ? hi : lo + (hi - lo) * (first + 1) / 33.0;
    if (!(nhi - nlo < hi - lo)) break;
    lo = nlo; hi = nhi;
  }
  return 0.5 * (lo + hi);
}

__global__ void lanczos_finish_kernel(const double* alpha, const double* beta,
                                      const double* kcount, double* bounds) {
  const bool terminated = kcount[0] < 0;
  const int k = (int)fabs(kcount[0]);
  double lo = 1e300, hi = -1e300;
  for (int i = 0; i < k; ++i) {
    double r = (i > 0 ? fabs(beta[i - 1]) : 0.0) + (i < k - 1 ? fabs(beta[i]) : 0.0);
    lo = fmin(lo, alpha[i] - r);
    hi = fmax(hi, alpha[i] + r);
  }
  const double tmin = multisect(alpha, beta, k, lo, hi, 1);
  const double tmax = multisect(alpha, beta, k, lo, hi, k);
  if (threadIdx.x != 0) return;
  double bk = terminated ? 0.0 : fabs(beta[k - 1]);
  double rmin = bk * last_component(alpha, beta, k, tmin);
  double rmax = bk * last_component(alpha, beta, k, tmax);
  double l1 = tmin - rmin, l2 = tmax + rmax;
  double chi = 0.5 * (l1 + l2);
  double xi = 0.5 * (l2 - l1) * 1.001;
  double floor_xi = 1e-6 * fmax(fabs(chi), 1.0);
  if (!(xi > floor_xi)) xi = floor_xi;
  bounds[0] = chi;
  bounds[1] = xi;
}

void lanczos_bounds_f64(sq3_ctx* ctx, const double* Hs, int n, int steps,
                        double* d_bounds, double* work, cudaStream_t st) {
  (void)ctx;
  if (steps > n) steps = n;
  if (steps > LZ_MAXQ) steps = LZ_MAXQ;
  double* V = work;
  double* w = V + (long long)(steps + 1) * n;
  double* alpha = w + n;
  double* beta = alpha + steps;
  double* kc = beta + steps;
  const int gv = (n + LZ_T - 1) / LZ_T;
  const int gr = (int)(((long long)n * 32 + LZ_T - 1) / LZ_T);
  LzParts P;
  P.alpha = kc + 8;
  P.h1 = P.alpha + gr;
  P.h2 = P.h1 + (long long)gv * LZ_MAXQ;
  P.b2 = P.h2 + (long long)gv * LZ_MAXQ;
  lanczos_init_kernel<<<1, 1024, 0, st>>>(V, n, kc);
  for (int j = 0; j < steps; ++j) {
    symv_alpha_kernel<<<gr, LZ_T, 0, st>>>(Hs, V + (long long)j * n, w, n, kc, j, P.alpha);
    lanczos_three_term_kernel<<<gv, LZ_T, 0, st>>>(V, w, beta, n, j, kc, P, gr);
    lanczos_reorth_kernel<<<gv, LZ_T, 0, st>>>(V, w, n, j, kc, P.h1, P.h2, P.b2, gv);
    lanczos_reorth_kernel<<<gv, LZ_T, 0, st>>>(V, w, n, j, kc, P.h2, nullptr, P.b2, gv);
    lanczos_next_kernel<<<gv, LZ_T, 0, st>>>(V, w, alpha, beta, kc, n, j, P, gr, gv);
  }
  lanczos_finish_kernel<<<1, 32, 0, st>>>(alpha, beta, kc, d_bounds);
}

}  // namespace sq3

// ---------------------------------------------------------------------------
// Allocation-free variant of the spectral bounds (see sq3_lanczos_bounds_noalloc
// in sq3.h).  Its scratch is this file-scope device array, sized for
// Ns <= SQ3_NOALLOC_MAX_NS and the fixed 40 Lanczos steps.
// ---------------------------------------------------------------------------
namespace sq3 {
namespace {
constexpr int kNoAllocSteps = 40;
constexpr size_t kNoAllocWords = lanczos_work_words(SQ3_NOALLOC_MAX_NS, kNoAllocSteps);
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocWords];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
// per device: the address of the array and the id of the CUDA context it
// was looked up in.  A device reset or a new primary context loads the
// module again at another address, so the cache is keyed on the context.
double* g_noalloc_addr[kMaxDevices] = {nullptr};
unsigned long long g_noalloc_ctx[kMaxDevices] = {0};

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

// Id of the calling thread's current CUDA context (0 if it cannot be read).
unsigned long long current_context_id() {
  static CtxGetCurrentFn get_cur = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static bool looked_up = false;
  if (!looked_up) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_cur = (CtxGetCurrentFn)p;
    p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_id = (CtxGetIdFn)p;
    looked_up = true;
  }
  CUcontext c = nullptr;
  unsigned long long id = 0;
  if (!get_cur || !get_id || get_cur(&c) != CUDA_SUCCESS || !c || get_id(c, &id) != CUDA_SUCCESS)
    return 0;
  return id;
}
}  // namespace

}  // namespace sq3

extern "C" int sq3_lanczos_bounds_noalloc(const double* Hs, int Ns, double* bounds,
                                          void* cuda_stream) {
  using namespace sq3;
  if (!Hs || !bounds || Ns < 1) return SQ3_EINVAL;
  if (Ns > SQ3_NOALLOC_MAX_NS) return SQ3_EINVAL;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return SQ3_ECUDA;
  }
  // an error left by earlier, unrelated asynchronous work is not this
  // call's: clear it so that the check after the launches sees only ours
  cudaGetLastError();
  double* scratch = nullptr;
  {
    // first call on this device (and after its context changed): look up
    // the device address of the array with the device current (the
    // host-side name is only a stand-in)
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    const unsigned long long cid = current_context_id();
    if (!g_noalloc_addr[dev] || cid == 0 || cid != g_noalloc_ctx[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        g_noalloc_addr[dev] = nullptr;
        return SQ3_ECUDA;
      }
      g_noalloc_addr[dev] = (double*)p;
      g_noalloc_ctx[dev] = cid;
    }
    scratch = g_noalloc_addr[dev];
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const int steps = Ns < kNoAllocSteps ? Ns : kNoAllocSteps;
  // every scratch word the kernels read is written earlier in the same call
  // (the basis, the step counter, alpha, beta and each step's block partial
  // sums), so nothing is cleared here
  lanczos_bounds_f64(nullptr, Hs, Ns, steps, bounds, scratch, st);
  if (cudaGetLastError() != cudaSuccess) return SQ3_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    return SQ3_ECUDA;
  }
  return SQ3_OK;
}
