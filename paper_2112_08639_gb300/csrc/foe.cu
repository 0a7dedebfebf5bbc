// Chebyshev Fermi-operator expansion of the density kernel (Sec. 4).
//
//   Hhat = (Hs - chi I)/xi                              Eq. (ChebyshevExpansion)
//   T_0 = I, T_1 = Hhat, T_{j+1} = 2 Hhat T_j - T_{j-1}  Eq. (ThreeTermRecurrenceRelation)
//   m_j = sum_n e_n^T t^j_n = tr T_j                     Eq. (FermiLevelCalc)
//   c_j(mu) = (2/pi) int g(xi l + chi) T_j(l) / sqrt(1 - l^2) dl
//                                                        Eq. (ChebyshevCoeff)
//   mu: 2 sum'_j c_j(mu) m_j = Ne ;  Ds = sum'_j c_j T_j
//   E_band = 2 sum'_j d_j m_j ;  E_ent = 2 sigma sum'_j e_j m_j
//
// The integral is evaluated by Chebyshev-Gauss quadrature on M nodes
// theta_k = (k + 1/2) pi / M, M = max(1024, 8 (npl + 1)).  With that rule the
// electron count is a double sum over j and k; this implementation sums over
// j first, w_k = sum'_j m_j T_j(cos theta_k) (independent of mu), so every
// evaluation of the count costs M Fermi evaluations and one block
// reduction; mu is found by a multisection that evaluates 63 counts per
// round, one block each, all on the GPU in FP64.  All T_j are kept (they fit in HBM for the sizes used), so
// Ds is a weighted sum of stored matrices instead of a second recurrence.
#include <math.h>

#include <algorithm>
#include <vector>

#include "sq3_internal.cuh"

namespace sq3 {

__global__ void hhat_kernel(const double* __restrict__ Hs, double* T0,
                            double* T1, int n, const double* bounds,
                            double* moments, int npl) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long tot = (long long)n * n;
  if (e == 0) moments[0] = (double)n;
  if (e >= tot) return;
  const int i = (int)(e % n), j = (int)(e / n);
  const double chi = bounds[0], xi = bounds[1];
  const double h = (Hs[e] - (i == j ? chi : 0.0)) / xi;
  T1[e] = h;
  T0[e] = (i == j) ? 1.0 : 0.0;
}

__global__ void trace_kernel(const double* __restrict__ A, int n, double* out) {
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

__device__ inline double fermi_dev(double eps, double mu, double sigma) {
  // 1 / (1 + exp(x)), x = (eps - mu)/sigma, without overflow
  const double x = (eps - mu) / sigma;
  if (x > 0) {
    const double t = exp(-x);
    return t / (1.0 + t);
  }
  return 1.0 / (1.0 + exp(x));
}

// g ln g + (1-g) ln(1-g), even in x; evaluated at t = -|x|.
__device__ inline double entropy_dev(double eps, double mu, double sigma) {
  const double t = -fabs((eps - mu) / sigma);
  const double et = exp(t);
  return -log1p(et) + t * et / (1.0 + et);
}

__device__ double bsum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
  return s;
}

// The Fermi level by multisection on the electron count of Eq.
// (FermiLevelCalc), N(mu) = 2 (2/M) sum_k g(xi x_k + chi; mu) w_k with the
// moment-weighted node sums w_k = sum'_j m_j T_j(x_k).  fermi_prep_kernel
// (one CTA) forms x_k and w_k, checks the moments and the initial bracket;
// each round fermi_count_kernel evaluates N at FL_POINTS interior points of
// the bracket, one block per point, and fermi_bracket_kernel keeps the
// sub-interval where N crosses Ne (the bracket shrinks FL_POINTS + 1 fold
// per round; rounds stop once it no longer shrinks).  fermi_values_kernel
// then writes mu and the three functions at the nodes.  Every count is one
// block's sum in a fixed order, so mu does not depend on scheduling.
// fl[0..M) = w_k, fl[M..2M) = x_k, fl[2M] = lo, fl[2M+1] = hi,
// fl[2M+2] = done flag, fl[2M+3 ..] = the round's counts.
constexpr int FL_POINTS = 63;
constexpr int FL_ROUNDS = 12;

__device__ double fermi_count(const double* fl, int M, double chi, double xi, double mu,
                              double sigma, double* sh) {
  const double* wq = fl;
  const double* xk = fl + M;
  double s = 0.0;
  for (int k = threadIdx.x; k < M; k += blockDim.x)
    s += fermi_dev(xi * xk[k] + chi, mu, sigma) * wq[k];
  return 2.0 * (2.0 / M) * bsum(s, sh);
}

__global__ void __launch_bounds__(1024)
fermi_prep_kernel(const double* __restrict__ moments, int npl, int M, double sigma, double Ne,
                  int n, const double* bounds, double* fl, int* status) {
  __shared__ double sh[32];
  const double chi = bounds[0], xi = bounds[1];
  // moment sanity: |tr T_j| <= n unless the spectrum left [-1, 1]
  for (int j = threadIdx.x; j <= npl; j += blockDim.x) {
    const double mj = moments[j];
    if (!isfinite(mj)) atomicCAS(status, 0, DEV_NONFINITE);
    else if (fabs(mj) > n * (1.0 + 1e-6)) atomicCAS(status, 0, DEV_NOCONV);
  }
  for (int k = threadIdx.x; k < M; k += blockDim.x) {
    const double x = cospi((2.0 * k + 1.0) / (2.0 * M));
    fl[M + k] = x;
    double tp = 1.0, t = x;                  // T_0, T_1 at x
    double acc = 0.5 * moments[0] + (npl >= 1 ? moments[1] * x : 0.0);
    for (int j = 2; j <= npl; ++j) {
      const double tn = 2.0 * x * t - tp;
      tp = t; t = tn;
      acc += moments[j] * t;
    }
    fl[k] = acc;
  }
  __syncthreads();
  const double lo = chi - xi - 40.0 * sigma, hi = chi + xi + 40.0 * sigma;
  const double clo = fermi_count(fl, M, chi, xi, lo, sigma, sh);
  const double chi_ = fermi_count(fl, M, chi, xi, hi, sigma, sh);
  if (threadIdx.x == 0) {
    if (!(clo < Ne && chi_ > Ne)) atomicCAS(status, 0, DEV_NOCONV);
    fl[2 * M] = lo;
    fl[2 * M + 1] = hi;
    fl[2 * M + 2] = 0.0;
  }
}

__global__ void __launch_bounds__(256)
fermi_count_kernel(int M, double sigma, const double* bounds, double* fl) {
  __shared__ double sh[32];
  if (fl[2 * M + 2] != 0.0) return;          // converged in an earlier round
  const double lo = fl[2 * M], hi = fl[2 * M + 1];
  const double mu = lo + (hi - lo) * (blockIdx.x + 1) / (FL_POINTS + 1.0);
  const double c = fermi_count(fl, M, bounds[0], bounds[1], mu, sigma, sh);
  if (threadIdx.x == 0) fl[2 * M + 3 + blockIdx.x] = c;
}

__global__ void fermi_bracket_kernel(int M, double Ne, double* fl) {
  if (fl[2 * M + 2] != 0.0) return;
  const double lo = fl[2 * M], hi = fl[2 * M + 1];
  int first = FL_POINTS;                      // first point with N >= Ne
  for (int b = 0; b < FL_POINTS; ++b)
    if (fl[2 * M + 3 + b] >= Ne) { first = b; break; }
  const double nlo = first == 0 ? lo : lo + (hi - lo) * first / (FL_POINTS + 1.0);
  const double nhi = first == FL_POINTS ? hi : lo + (hi - lo) * (first + 1) / (FL_POINTS + 1.0);
  if (!(nhi - nlo < hi - lo) || !(nlo < nhi)) {
    fl[2 * M + 2] = 1.0;                      // no longer shrinks
    return;
  }
  fl[2 * M] = nlo;
  fl[2 * M + 1] = nhi;
}

// out[0] = mu, out[3] = chi, out[4] = xi; fvals[0..3M) = g, eps g, entropy.
__global__ void __launch_bounds__(256)
fermi_values_kernel(int M, double sigma, const double* bounds, const double* fl,
                    double* fvals, double* out, int* status) {
  const double chi = bounds[0], xi = bounds[1];
  const double mu = 0.5 * (fl[2 * M] + fl[2 * M + 1]);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < M; k += gridDim.x * blockDim.x) {
    const double eps = xi * fl[M + k] + chi;
    const double g = fermi_dev(eps, mu, sigma);
    fvals[k] = g;
    fvals[M + k] = eps * g;
    fvals[2 * M + k] = entropy_dev(eps, mu, sigma);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    out[0] = mu;
    out[3] = chi;
    out[4] = xi;
    if (!isfinite(mu)) atomicCAS(status, 0, DEV_NONFINITE);
  }
}

// One warp per degree j: c_j, d_j, e_j = (2/M) sum_k f(x_k) cos(j theta_k)
// for the three functions, with cos(j theta_k) = cospi(j (2k+1) / (2M))
// evaluated after reducing the integer j (2k+1) modulo 4M.  Writes c_j and
// the primed products with the moments into terms[3][npl+1].
__global__ void __launch_bounds__(256)
cheb_coeff_kernel(const double* __restrict__ fvals, const double* __restrict__ moments,
                  int npl, int M, double* coef, double* terms) {
  const int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (j > npl) return;
  double a = 0.0, b = 0.0, c = 0.0;
  const long long fourM = 4LL * M;
  for (int k = lane; k < M; k += 32) {
    const long long q = ((long long)j * (2 * k + 1)) % fourM;
    const double cj = cospi((double)q / (2.0 * M));
    a += fvals[k] * cj;
    b += fvals[M + k] * cj;
    c += fvals[2 * M + k] * cj;
  }
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
    c += __shfl_xor_sync(0xffffffffu, c, o);
  }
  if (lane == 0) {
    a *= 2.0 / M; b *= 2.0 / M; c *= 2.0 / M;
    coef[j] = a;
    const double wgt = (j == 0) ? 0.5 : 1.0;
    terms[j] = wgt * a * moments[j];
    terms[(npl + 1) + j] = wgt * b * moments[j];
    terms[2 * (npl + 1) + j] = wgt * c * moments[j];
  }
}

// In-order sums of the primed series: out[1] = E_band, out[2] = E_ent,
// out[5] = 2 sum'_j c_j m_j.
__global__ void fermi_finish_kernel(const double* __restrict__ terms, int npl, double sigma,
                                    double* out, int* status) {
  if (threadIdx.x != 0) return;
  double sc = 0.0, sd = 0.0, se = 0.0;
  for (int j = 0; j <= npl; ++j) {
    sc += terms[j];
    sd += terms[(npl + 1) + j];
    se += terms[2 * (npl + 1) + j];
  }
  out[1] = 2.0 * sd;
  out[2] = 2.0 * sigma * se;
  out[5] = 2.0 * sc;
  if (!isfinite(sd) || !isfinite(se) || !isfinite(sc)) atomicCAS(status, 0, DEV_NONFINITE);
}

// Ds = c_0/2 I + sum_{j>=1} c_j T_j over the stored T_j.
__global__ void accumulate_d_kernel(const double* __restrict__ T, long long nn,
                                    int n, int npl,
                                    const double* __restrict__ coef,
                                    double* D) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= nn) return;
  const int i = (int)(e % n), j = (int)(e / n);
  double s = (i == j) ? 0.5 * coef[0] : 0.0;
  for (int t = 1; t <= npl; ++t) s += coef[t] * T[(long long)t * nn + e];
  D[e] = s;
}

// ---------------------------------------------------------------------------
// Paterson-Stockmeyer evaluation (FP64): the same polynomial of Hhat,
// reordered so that it takes O(sqrt(npl)) matrix products instead of npl.
// With s baby steps T_0 .. T_s and Y = T_s, every T_{qs} = T_q(Y) (the
// Chebyshev composition identity T_q(T_s(x)) = T_{qs}(x)):
//   giant steps   G_{q+1} = 2 Y G_q - G_{q-1}, G_0 = I, G_1 = Y
//   moments       m_{qs+r} = 2 tr(G_q T_r) - m_{qs-r}   (T_a T_b =
//                 (T_{a+b} + T_{|a-b|}) / 2; tr(G_q T_r) is a Frobenius
//                 product of symmetric matrices, no further product)
//   kernel        sum'_j c_j T_j = sum_{q=0}^{Q} A_q T_q(Y),
//                 A_q = sum_{r<s} alpha_{q,r} T_r, the alpha found top-down
//                 (T_r T_{qs} = (T_{qs+r} + T_{qs-r}) / 2), and the outer
//                 sum by Clenshaw's recurrence in Y:
//                 b_q = A_q + 2 Y b_{q+1} - b_{q+2},  Ds = A_0 + Y b_1 - b_2.
// Products: (s - 1) + (Q - 1) + Q with Q = floor(npl / s), s = ceil(sqrt(2 npl)).
// ---------------------------------------------------------------------------

// part[(pair) * PS_FROB_BLOCKS + b]: block sums of <G_q, T_r>, pair =
// (q - 1) (s - 1) + (r - 1); G_q at gq[q], T_r at T + r nn.
__global__ void __launch_bounds__(256) ps_frob_kernel(const double* const* __restrict__ gq,
                                                      const double* __restrict__ T, long long nn,
                                                      int s, double* part) {
  __shared__ double sh[8];
  const int pair = blockIdx.x / PS_FROB_BLOCKS, blk = blockIdx.x % PS_FROB_BLOCKS;
  const int q = pair / (s - 1) + 1, r = pair % (s - 1) + 1;
  const double* A = gq[q];
  const double* B = T + (long long)r * nn;
  double acc = 0.0;
  for (long long e = (long long)blk * blockDim.x + threadIdx.x; e < nn;
       e += (long long)PS_FROB_BLOCKS * blockDim.x)
    acc += A[e] * B[e];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    part[blockIdx.x] = t;
  }
}

// m_{qs + r} = 2 <G_q, T_r> - m_{qs - r}, in increasing q (one thread).
__global__ void ps_moments_kernel(const double* __restrict__ part, int s, int Q, int npl,
                                  double* mom) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int q = 1; q <= Q; ++q)
    for (int r = 1; r < s; ++r) {
      const int j = q * s + r;
      if (j > npl) continue;
      const int pair = (q - 1) * (s - 1) + (r - 1);
      double f = 0.0;
      for (int b = 0; b < PS_FROB_BLOCKS; ++b) f += part[pair * PS_FROB_BLOCKS + b];
      mom[j] = 2.0 * f - mom[q * s - r];
    }
}

// alpha[q s + r] from the coefficients c_j (c_0 halved), top-down; w: work
// of (Q + 1) s doubles (one thread).
__global__ void ps_alpha_kernel(const double* __restrict__ coef, int npl, int s, int Q,
                                double* w, double* alpha) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int top = (Q + 1) * s;
  for (int j = 0; j < top; ++j) w[j] = j <= npl ? (j == 0 ? 0.5 * coef[0] : coef[j]) : 0.0;
  for (int q = Q; q >= 1; --q) {
    alpha[q * s] = w[q * s];
    for (int r = 1; r < s; ++r) {
      alpha[q * s + r] = 2.0 * w[q * s + r];
      w[q * s - r] -= w[q * s + r];
    }
  }
  for (int r = 0; r < s; ++r) alpha[r] = w[r];
}

// out = ea E + eb Bm + sum_{r<s} alpha[r] T_r (E, Bm may be null; out may
// alias E).
__global__ void __launch_bounds__(256) ps_combine_kernel(double* out, const double* E, double ea,
                                                         const double* __restrict__ Bm, double eb,
                                                         const double* __restrict__ T, long long nn,
                                                         int s, const double* __restrict__ alpha) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nn;
       e += (long long)gridDim.x * blockDim.x) {
    double v = 0.0;
    for (int r = 0; r < s; ++r) v += alpha[r] * T[(long long)r * nn + e];
    if (E) v += ea * E[e];
    if (Bm) v += eb * Bm[e];
    out[e] = v;
  }
}

// Pointers into the Paterson-Stockmeyer workspace (T = ctx->wsT).
struct PsWs {
  double* baby;        // T_0 .. T_s
  double* giant;       // G_2 .. G_Q
  double* b[3];        // Clenshaw buffers
  double* part;        // Frobenius partials
  double* alpha;       // (Q + 1) s
  double* work;        // (Q + 1) s
  double** gptr;       // device pointers G_0 .. G_Q (Q + 2 slots)
};
static PsWs ps_ws(double* T, long long nn, int s, int Q) {
  PsWs w;
  w.baby = T;
  w.giant = T + (long long)(s + 1) * nn;
  double* p = w.giant + (long long)std::max(Q - 1, 0) * nn;
  for (int k = 0; k < 3; ++k) { w.b[k] = p; p += nn; }
  w.part = p; p += (size_t)Q * s * PS_FROB_BLOCKS;
  w.alpha = p; p += (size_t)(Q + 1) * s;
  w.work = p; p += (size_t)(Q + 1) * s;
  w.gptr = reinterpret_cast<double**>(p);
  return w;
}
// C = 2 A B - P (FP64 GEMM with the Chebyshev epilogue), trace of C into tr
static void cheb_product(const double* A, const double* B, const double* P, double* C, int Ns,
                         double* tr, cudaStream_t st) {
  GemmArgs g{};
  g.M = Ns; g.N = Ns; g.K = Ns;
  g.A = A; g.lda = Ns; g.a_kcontig = false;
  g.B = B; g.ldb = Ns; g.b_kcontig = true;
  g.C = C; g.ldc = Ns;
  g.P = P; g.ldp = Ns;
  g.trace = tr;
  g.alpha = 1.0; g.splits = 1;
  gemm_f64(g, EPI_CHEB, st);
}

// Moments m_0 .. m_npl by baby steps, giant steps and Frobenius products.
int ps_moments_f64(sq3_ctx* ctx, const double* Hs, int Ns, int npl, int s, int Q,
                   const double* bounds, double* mom, double* T) {
  cudaStream_t st = ctx->stream;
  const long long nn = (long long)Ns * Ns;
  const PsWs w = ps_ws(T, nn, s, Q);
  const int sb = std::min(s, npl);            // baby steps actually needed
  {
    Prof p(ctx, ST_CHEB_GEMM, 2);
    hhat_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, st>>>(Hs, w.baby, w.baby + nn, Ns,
                                                              bounds, mom, npl);
    trace_kernel<<<1, 1024, 0, st>>>(w.baby + nn, Ns, mom + 1);
  }
  {
    Prof p(ctx, ST_CHEB_GEMM, std::max(sb - 1, 0));
    for (int j = 1; j < sb; ++j)
      cheb_product(w.baby + nn, w.baby + (long long)j * nn, w.baby + (long long)(j - 1) * nn,
                   w.baby + (long long)(j + 1) * nn, Ns, mom + j + 1, st);
  }
  if (Q < 1) return cuda_err(cudaGetLastError());
  // giant steps G_q = T_{qs}: G_{q+1} = 2 Y G_q - G_{q-1}, Y = T_s
  const double* Y = w.baby + (long long)s * nn;
  std::vector<double*> g(Q + 1);
  g[0] = w.baby;
  g[1] = const_cast<double*>(Y);
  for (int q = 2; q <= Q; ++q) g[q] = w.giant + (long long)(q - 2) * nn;
  {
    Prof p(ctx, ST_CHEB_GEMM, std::max(Q - 1, 0));
    for (int q = 1; q < Q; ++q)
      cheb_product(Y, g[q], g[q - 1], g[q + 1], Ns, mom + (q + 1) * s, st);
  }
  int rc = cuda_err(cudaMemcpyAsync(w.gptr, g.data(), (Q + 1) * sizeof(double*),
                                    cudaMemcpyHostToDevice, st));
  if (rc) return rc;
  {
    Prof p(ctx, ST_CHEB_GEMM, 2);
    ps_frob_kernel<<<Q * (s - 1) * PS_FROB_BLOCKS, 256, 0, st>>>(
        const_cast<const double* const*>(w.gptr), w.baby, nn, s, w.part);
    ps_moments_kernel<<<1, 32, 0, st>>>(w.part, s, Q, npl, mom);
  }
  // the host vector g is only read by the copy above, which the stream
  // orders before any later use; wait for it before g goes out of scope
  return cuda_err(cudaStreamSynchronize(st));
}

// Ds = sum'_j c_j T_j by the Clenshaw recurrence in Y = T_s.
int ps_kernel_f64(sq3_ctx* ctx, int Ns, int npl, int s, int Q, const double* coef, double* T,
                  double* D) {
  cudaStream_t st = ctx->stream;
  const long long nn = (long long)Ns * Ns;
  const PsWs w = ps_ws(T, nn, s, Q);
  const int sb = std::min(s, npl + 1);       // baby steps T_0 .. T_{sb-1} hold A_q
  const unsigned blocks = (unsigned)std::min<long long>((nn + 255) / 256, 152LL * 8);
  Prof pd(ctx, ST_D_ACCUM, 2 + 2 * Q);
  ps_alpha_kernel<<<1, 32, 0, st>>>(coef, npl, s, Q, w.work, w.alpha);
  if (Q == 0) {
    ps_combine_kernel<<<blocks, 256, 0, st>>>(D, nullptr, 0.0, nullptr, 0.0, w.baby, nn, sb,
                                              w.alpha);
    return cuda_err(cudaGetLastError());
  }
  const double* Y = w.baby + (long long)s * nn;
  double* bq1 = w.b[0];     // b_{q+1}
  double* bq2 = w.b[1];     // b_{q+2}
  double* bq = w.b[2];
  cudaMemsetAsync(bq2, 0, nn * sizeof(double), st);
  // b_Q = A_Q
  ps_combine_kernel<<<blocks, 256, 0, st>>>(bq1, nullptr, 0.0, nullptr, 0.0, w.baby, nn, s,
                                            w.alpha + (size_t)Q * s);
  for (int q = Q - 1; q >= 1; --q) {
    // b_q = A_q + 2 Y b_{q+1} - b_{q+2}
    cheb_product(Y, bq1, bq2, bq, Ns, nullptr, st);
    ps_combine_kernel<<<blocks, 256, 0, st>>>(bq, bq, 1.0, nullptr, 0.0, w.baby, nn, s,
                                              w.alpha + (size_t)q * s);
    double* t = bq2;
    bq2 = bq1;
    bq1 = bq;
    bq = t;
  }
  // Ds = A_0 + Y b_1 - b_2 = (2 Y b_1 - b_2) / 2 - b_2 / 2 + A_0
  cheb_product(Y, bq1, bq2, bq, Ns, nullptr, st);
  ps_combine_kernel<<<blocks, 256, 0, st>>>(D, bq, 0.5, bq2, -0.5, w.baby, nn, s, w.alpha);
  return cuda_err(cudaGetLastError());
}

void ps_moments_finish(const double* part, int s, int Q, int npl, double* mom,
                       cudaStream_t st) {
  ps_moments_kernel<<<1, 32, 0, st>>>(part, s, Q, npl, mom);
}

void ps_alpha(const double* coef, int npl, int s, int Q, double* work, double* alpha,
              cudaStream_t st) {
  ps_alpha_kernel<<<1, 32, 0, st>>>(coef, npl, s, Q, work, alpha);
}

int ps_layout(int npl, int* s_out, int* Q_out) {
  int s = (int)ceil(sqrt(2.0 * npl));
  if (s < 2) s = 2;
  *s_out = s;
  *Q_out = npl / s;
  return 0;
}

int density_kernel_from_hs(sq3_ctx* ctx, const double* Hs, int Ns, int npl,
                           double sigma, double Ne, const double* bounds_in,
                           double* D, double* out_host, bool mixed, double fermi_tol,
                           int eval_mode, int* npl_used) {
  cudaStream_t st = ctx->stream;
  const long long nn = (long long)Ns * Ns;
  // workspace: T_0..T_npl (FP64), or in the mixed path T_0..T_h (FP32) and
  // one more Ns x Ns FP32 matrix; Lanczos work
  // The mixed path runs the recurrence to h = ceil(npl / 2) only: the
  // moments and the terms of Ds above h follow from the product identity
  // T_h T_k = (T_{h+k} + T_{h-k}) / 2 (one more tensor-core product).
  const int lsteps = Ns < 40 ? Ns : 40;
  size_t need_m = lanczos_work_words((size_t)Ns, (size_t)lsteps) * sizeof(double);
  int rc = ensure((void**)&ctx->wsMat, &ctx->wsMat_bytes, need_m);
  if (rc) return rc;
  double* bounds = ctx->dev_scal;                  // chi, xi
  double* outd = ctx->dev_scal + 8;                // 6 outputs
  double* mom = ctx->dev_scal + 64;                // moments m_0..m_npl
  double* coef = ctx->dev_scal + 64 + SQ3_MAX_NPL + 1;  // c_0..c_npl
  if (bounds_in) {
    rc = cuda_err(cudaMemcpyAsync(bounds, bounds_in, 2 * sizeof(double),
                                  cudaMemcpyHostToDevice, st));
    if (rc) return rc;
  } else {
    Prof p(ctx, ST_LANCZOS, 5 * lsteps + 2);
    lanczos_bounds_f64(ctx, Hs, Ns, lsteps, bounds, ctx->wsMat, st);
  }
  if (npl < 1) {
    // degree from the tolerance and the spectral half-width (the Bernstein
    // ellipse rule of sq3_fermi_degree)
    double xi = 0.0;
    if (bounds_in) {
      xi = bounds_in[1];
    } else {
      rc = cuda_err(cudaMemcpyAsync(ctx->host_scal + 40, bounds + 1, sizeof(double),
                                    cudaMemcpyDeviceToHost, st));
      if (rc == SQ3_OK) rc = cuda_err(cudaStreamSynchronize(st));
      if (rc) return rc;
      xi = ctx->host_scal[40];
    }
    if (!(xi > 0) || !isfinite(xi)) return SQ3_ENONFINITE;
    npl = sq3_fermi_degree(sigma, xi, fermi_tol);
    if (npl < 1) return SQ3_EINVAL;
    if (npl > SQ3_MAX_NPL) npl = SQ3_MAX_NPL;
  }
  if (npl > SQ3_MAX_NPL) return SQ3_EINVAL;
  if (npl_used) *npl_used = npl;
  const bool ps = eval_mode == 1;
  int ps_s = 0, ps_Q = 0;
  ps_layout(npl, &ps_s, &ps_Q);
  const int h = mixed ? (npl + 1) / 2 : npl;
  // (mixed: then the block sums of the moment tail, 8-byte aligned)
  const size_t tail_off = (((size_t)(h + 2) * nn * sizeof(float) + 7) / 8) * 8;
  // Paterson-Stockmeyer: T_0..T_s, G_2..G_Q, three Clenshaw buffers, the
  // Frobenius partials, alpha and its work, and the giant-step pointers
  const size_t ps_mats = (size_t)(ps_s + 1) + (size_t)std::max(ps_Q - 1, 0) + 3;
  const size_t ps_words = ps_mats * nn + (size_t)ps_Q * ps_s * PS_FROB_BLOCKS +
                          2 * (size_t)(ps_Q + 1) * ps_s + (size_t)(ps_Q + 2);
  size_t need_T = (mixed && ps) ? ps_mixed_bytes(Ns, ps_s, ps_Q)
                  : mixed ? tail_off + moments_tail_part_words(npl, h) * sizeof(double)
                          : (ps ? ps_words : (size_t)(npl + 1) * nn) * sizeof(double);
  rc = ensure((void**)&ctx->wsT, &ctx->wsT_bytes, need_T);
  if (rc) return rc;
  rc = cuda_err(cudaMemsetAsync(mom, 0, (size_t)(npl + 1) * sizeof(double), st));
  if (rc) return rc;
  double* T = ctx->wsT;
  if (mixed && ps) {
    rc = ps_moments_mixed(ctx, Hs, Ns, npl, ps_s, ps_Q, bounds, mom, ctx->wsT);
    if (rc) return rc;
  } else if (mixed) {
    rc = cheb_recurrence_mixed(ctx, Hs, Ns, h, bounds, mom, (float*)ctx->wsT);
    if (rc) return rc;
    {
      Prof p(ctx, ST_CHEB_GEMM, npl > h ? 2 : 0);
      rc = moments_tail_mixed(ctx, (const float*)ctx->wsT, Ns, npl, h, mom,
                              (double*)((char*)ctx->wsT + tail_off));
    }
    if (rc) return rc;
  } else if (ps) {
    rc = ps_moments_f64(ctx, Hs, Ns, npl, ps_s, ps_Q, bounds, mom, T);
    if (rc) return rc;
  } else {
  {
    Prof p(ctx, ST_CHEB_GEMM, 2);
    hhat_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, st>>>(
        Hs, T, T + nn, Ns, bounds, mom, npl);
    trace_kernel<<<1, 1024, 0, st>>>(T + nn, Ns, mom + 1);
  }
  {
  Prof prec(ctx, ST_CHEB_GEMM, npl - 1);
  for (int j = 1; j < npl; ++j) {
    GemmArgs g{};
    g.M = Ns; g.N = Ns; g.K = Ns;
    g.A = T + nn; g.lda = Ns; g.a_kcontig = false;             // Hhat
    g.B = T + (long long)j * nn; g.ldb = Ns; g.b_kcontig = true;  // T_j
    g.C = T + (long long)(j + 1) * nn; g.ldc = Ns;
    g.P = T + (long long)(j - 1) * nn; g.ldp = Ns;
    g.trace = mom + j + 1;
    g.alpha = 1.0; g.splits = 1;
    gemm_f64(g, EPI_CHEB, st);
  }
  }
  }
  const int M = (8 * (npl + 1) > 1024) ? 8 * (npl + 1) : 1024;
  rc = ensure((void**)&ctx->wsFoe, &ctx->wsFoe_bytes,
              ((size_t)5 * M + 3 * (npl + 1) + 3 + FL_POINTS) * sizeof(double));
  if (rc) return rc;
  double* fvals = ctx->wsFoe;
  double* terms = fvals + 3 * M;
  double* fl = terms + 3 * (npl + 1);
  {
    Prof p(ctx, ST_FERMI, 4 + 2 * FL_ROUNDS);
    fermi_prep_kernel<<<1, 1024, 0, st>>>(mom, npl, M, sigma, Ne, Ns, bounds, fl,
                                          ctx->dev_status);
    for (int r = 0; r < FL_ROUNDS; ++r) {
      fermi_count_kernel<<<FL_POINTS, 256, 0, st>>>(M, sigma, bounds, fl);
      fermi_bracket_kernel<<<1, 1, 0, st>>>(M, Ne, fl);
    }
    fermi_values_kernel<<<(M + 255) / 256, 256, 0, st>>>(M, sigma, bounds, fl, fvals, outd,
                                                         ctx->dev_status);
    cheb_coeff_kernel<<<(npl + 1 + 7) / 8, 256, 0, st>>>(fvals, mom, npl, M, coef,
                                                         terms);
    fermi_finish_kernel<<<1, 32, 0, st>>>(terms, npl, sigma, outd, ctx->dev_status);
  }
  if (D != nullptr && mixed && ps) {
    rc = ps_kernel_mixed(ctx, Ns, npl, ps_s, ps_Q, coef, ctx->wsT, D);
    if (rc) return rc;
  } else if (D != nullptr && mixed) {
    rc = accumulate_d_mixed(ctx, (const float*)ctx->wsT, Ns, npl, h, coef, D,
                            (float*)ctx->wsT + (size_t)(h + 1) * nn);
    if (rc) return rc;
  } else if (D != nullptr && ps) {
    rc = ps_kernel_f64(ctx, Ns, npl, ps_s, ps_Q, coef, T, D);
    if (rc) return rc;
  } else if (D != nullptr) {
    Prof pd(ctx, ST_D_ACCUM);
    accumulate_d_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, st>>>(
        T, nn, Ns, npl, coef, D);
  }
  if (D != nullptr) check_finite(D, nn, ctx->dev_status, st);
  rc = cuda_err(cudaGetLastError());
  if (rc) return rc;
  rc = cuda_err(cudaMemcpyAsync(ctx->host_scal, outd, 6 * sizeof(double),
                                cudaMemcpyDeviceToHost, st));
  if (rc) return rc;
  rc = check_device_status(ctx);
  if (rc) return rc;
  for (int i = 0; i < 6; ++i) {
    if (!isfinite(ctx->host_scal[i])) return SQ3_ENONFINITE;
    out_host[i] = ctx->host_scal[i];
  }
  return SQ3_OK;
}

}  // namespace sq3
