// C ABI entry points of libsq3: context, set-up, and the host-side ordering
// of the kernels of one SQ3 iteration (Sec. 4 of the paper).  Every step of
// the computation runs in this library's CUDA kernels; the host code here
// only validates arguments, sizes workspace and enqueues launches.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <array>
#include <vector>

#include "async_copy.cuh"
#include "sq3_internal.cuh"

namespace sq3 {

// Name of the last CUDA error seen by this host thread (reported by
// sq3_last_cuda_error).
static thread_local const char* g_last_cuda_error = "none";

int cuda_err(cudaError_t e) {
  if (e == cudaSuccess) return SQ3_OK;
  g_last_cuda_error = cudaGetErrorName(e);
  return SQ3_ECUDA;
}

int ensure(void** p, size_t* have, size_t need) {
  if (need <= *have && *p != nullptr) return SQ3_OK;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *have = 0;
  if (need == 0) return SQ3_OK;
  if (cudaMalloc(p, need) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return SQ3_ENOMEM;
  }
  *have = need;
  return SQ3_OK;
}

int check_device_status(sq3_ctx* ctx) {
  int h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, ctx->dev_status, sizeof(int),
                                  cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return SQ3_ECUDA;
  if (h != DEV_OK) {
    cudaMemsetAsync(ctx->dev_status, 0, sizeof(int), ctx->stream);
    cudaStreamSynchronize(ctx->stream);
    switch (h) {
      case DEV_NOTPD: return SQ3_ENOTPD;
      case DEV_NOCONV: return SQ3_ENOCONV;
      case DEV_NONFINITE: return SQ3_ENONFINITE;
      case DEV_TIMEOUT: return SQ3_ETIMEOUT;
      default: return SQ3_ECUDA;
    }
  }
  return SQ3_OK;
}

Prof::Prof(sq3_ctx* c, int st, int n) : ctx(c), stage(st), launches(n) {
  if (!ctx->prof) return;
  auto get = [&]() {
    cudaEvent_t e;
    if (!ctx->prof_pool.empty()) { e = ctx->prof_pool.back(); ctx->prof_pool.pop_back(); }
    else cudaEventCreate(&e);
    return e;
  };
  a = get();
  b = get();
  cudaEventRecord(a, ctx->stream);
}

Prof::~Prof() {
  if (!a) return;
  cudaEventRecord(b, ctx->stream);
  ctx->prof_recs.push_back({stage, launches, a, b});
}

// Central second-derivative weights of order 2n (Fornberg closed form).
static void fd_weights(int order, double* w) {
  const int n = order / 2;
  auto fact = [](int k) { double f = 1; for (int i = 2; i <= k; ++i) f *= i; return f; };
  w[0] = 0.0;
  for (int p = 1; p <= n; ++p) {
    w[p] = 2.0 * ((p % 2) ? 1.0 : -1.0) * fact(n) * fact(n) /
           ((double)p * p * fact(n - p) * fact(n + p));
    w[0] -= 2.0 / ((double)p * p);
  }
}

__global__ void to_float_kernel(const double* a, float* b, long long n) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

// Sets DEV_NONFINITE when any of the n values is NaN or infinite.
__global__ void check_finite_kernel(const double* __restrict__ a, long long n, int* status) {
  bool bad = false;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    bad |= !isfinite(a[i]);
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicCAS(status, DEV_OK, DEV_NONFINITE);
}

void check_finite(const double* a, long long n, int* status, cudaStream_t st) {
  if (n <= 0) return;
  const long long blocks = std::min<long long>((n + 255) / 256, 152LL * 8);
  check_finite_kernel<<<(unsigned)blocks, 256, 0, st>>>(a, n, status);
}

// Smallest and largest value of a (n > 0) in a fixed reduction order:
// per-block pairs into part[2 * blockIdx.x], then one block folds them into
// out[0] = min, out[1] = max.  Non-finite values set DEV_NONFINITE.
constexpr int MM_BLOCKS = 304;
__global__ void __launch_bounds__(256) minmax_part_kernel(const double* __restrict__ a,
                                                          long long n, double* part,
                                                          int* status) {
  __shared__ double smin[8], smax[8];
  double lo = INFINITY, hi = -INFINITY;
  bool bad = false;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double v = a[i];
    bad |= !isfinite(v);
    lo = fmin(lo, v);
    hi = fmax(hi, v);
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicCAS(status, DEV_OK, DEV_NONFINITE);
  for (int o = 16; o > 0; o >>= 1) {
    lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  if ((threadIdx.x & 31) == 0) { smin[threadIdx.x >> 5] = lo; smax[threadIdx.x >> 5] = hi; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) { lo = fmin(lo, smin[w]); hi = fmax(hi, smax[w]); }
    lo = fmin(lo, smin[0]);
    hi = fmax(hi, smax[0]);
    part[2 * blockIdx.x] = lo;
    part[2 * blockIdx.x + 1] = hi;
  }
}

__global__ void minmax_finish_kernel(const double* part, int nb, double* out) {
  if (threadIdx.x != 0) return;
  double lo = INFINITY, hi = -INFINITY;
  for (int b = 0; b < nb; ++b) { lo = fmin(lo, part[2 * b]); hi = fmax(hi, part[2 * b + 1]); }
  out[0] = lo;
  out[1] = hi;
}

// out[0..1] = min, max of the n device values (part: 2 * MM_BLOCKS doubles
// of device scratch).
void minmax(const double* a, long long n, double* part, double* out, int* status,
            cudaStream_t st) {
  minmax_part_kernel<<<MM_BLOCKS, 256, 0, st>>>(a, n, part, status);
  minmax_finish_kernel<<<1, 32, 0, st>>>(part, MM_BLOCKS, out);
}

static void free_projectors(Projectors& P) {
  void* ptrs[] = {P.gamma,       P.nb_ball_ptr, P.nb_slot_pid, P.nb_pt_ptr, P.nb_pt_lb,
                  P.nb_pt_val,   P.nb_pt_valf, P.nb_bl_ptr,  P.nb_bl_pt,
                  P.nb_bl_val,   P.nb_bl_valf, P.fq_ptr,     P.fq_idx,
                  P.fq_val,      P.fq_valf};
  for (void* p : ptrs) if (p) cudaFree(p);
  P = Projectors{};
}

template <typename T>
static int upload(T** dst, const T* src, size_t n) {
  if (n == 0) { *dst = nullptr; return SQ3_OK; }
  if (cudaMalloc((void**)dst, n * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    *dst = nullptr;
    return SQ3_ENOMEM;
  }
  return cuda_err(cudaMemcpy(*dst, src, n * sizeof(T), cudaMemcpyHostToDevice));
}


// Two gC workspaces (current and next step) for the nonlocal projections.
static int gc_buffer(sq3_ctx* ctx, int Ns, void** out, void** out2 = nullptr) {
  *out = nullptr;
  if (out2) *out2 = nullptr;
  if (ctx->proj.n_proj == 0) return SQ3_OK;
  const size_t one = (size_t)ctx->proj.n_proj * Ns * sizeof(double);
  int rc = ensure((void**)&ctx->wsProj, &ctx->wsProj_bytes, 2 * one);
  *out = ctx->wsProj;
  if (out2) *out2 = (char*)ctx->wsProj + one;
  return rc;
}

template <typename T>
static int hamiltonian_apply_t(sq3_ctx* ctx, const T* X, T* Y, int Ns) {
  void* gC;
  int rc = gc_buffer(ctx, Ns, &gC);
  if (rc) return rc;
  if (ctx->proj.n_proj) {
    // projections of X by the nonlocal pass in projection-only mode
    Prof p(ctx, ST_NL_PROJECT);
    cudaMemsetAsync(gC, 0, (size_t)ctx->proj.n_proj * Ns * sizeof(T), ctx->stream);
    rc = launch_nl_pass<T>(ctx, const_cast<T*>(X), nullptr, (T*)gC, Ns, 0.0, ctx->stream);
    if (rc) return rc;
  }
  {
    Prof p(ctx, ST_STENCIL);
    launch_cheb_step<T>(ctx, X, nullptr, Y, Ns, 1.0, 0.0, 0.0, ctx->stream);
  }
  if (ctx->proj.n_proj) {
    Prof p(ctx, ST_NL_PASS);
    rc = launch_nl_pass<T>(ctx, Y, (const T*)gC, nullptr, Ns, 1.0, ctx->stream);
    if (rc) return rc;
  }
  return cuda_err(cudaGetLastError());
}

// W = sc1 (W + (Vf - Vf_hx - c) X) over N x Ns (column v at v N), W holding
// H X applied with the potential Vf_hx: the first filter step from a kept
// H X.  Block row y: vector y; 16-byte vectors when N is a multiple of 4.
__global__ void filter_first_from_hx_kernel(float* W, const float* __restrict__ X,
                                            const float* __restrict__ V,
                                            const float* __restrict__ Vhx, long long N,
                                            float sc1, float c) {
  const long long off = (long long)blockIdx.y * N;
  if ((N & 3) == 0) {
    const long long n4 = N / 4;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n4;
         i += (long long)gridDim.x * blockDim.x) {
      float4 w = reinterpret_cast<float4*>(W + off)[i];
      const float4 x = reinterpret_cast<const float4*>(X + off)[i];
      const float4 v = reinterpret_cast<const float4*>(V)[i];
      const float4 h = reinterpret_cast<const float4*>(Vhx)[i];
      w.x = sc1 * (w.x + ((v.x - h.x) - c) * x.x);
      w.y = sc1 * (w.y + ((v.y - h.y) - c) * x.y);
      w.z = sc1 * (w.z + ((v.z - h.z) - c) * x.z);
      w.w = sc1 * (w.w + ((v.w - h.w) - c) * x.w);
      reinterpret_cast<float4*>(W + off)[i] = w;
    }
  } else {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < N;
         k += (long long)gridDim.x * blockDim.x)
      W[off + k] = sc1 * (W[off + k] + ((V[k] - Vhx[k]) - c) * X[off + k]);
  }
}

static void filter_first_from_hx(sq3_ctx* ctx, float* W, const float* X, int Ns, double sc1,
                                 double c) {
  const long long N = ctx->grid.N;
  const long long per = (N % 4 == 0) ? N / 4 : N;
  const unsigned bx = (unsigned)std::min<long long>((per + 255) / 256, 64);
  filter_first_from_hx_kernel<<<dim3(bx, Ns), 256, 0, ctx->stream>>>(W, X, ctx->Vf, ctx->Vf_hx,
                                                                      N, (float)sc1, (float)c);
}

int hamiltonian_apply_f32(sq3_ctx* ctx, const float* X, float* Y, int Ns) {
  return hamiltonian_apply_t<float>(ctx, X, Y, Ns);
}

// Scaled three-term recurrence of the Chebyshev filter (Zhou et al. 2006):
// with x = (t - c)/e and rho_k = T_k((a0 - c)/e), Y_k = T_k(x) X / rho_k obeys
// Y_1 = (s_1/e)(H - c) X and Y_{k+1} = (2 s_{k+1}/e)(H - c) Y_k
// - s_k s_{k+1} Y_{k-1} with s_1 = e/(a0 - c), s_{k+1} = 1/(2/s_1 - s_k).
template <typename T>
static int cheb_filter_t(sq3_ctx* ctx, T* X, int Ns, int m, double a,
                         double b, double a0) {
  ctx->pieces_X = nullptr;                 // X changes: its kept pieces are stale
  // H X kept by the driver's last projection of this same X (mixed path)
  const bool from_hx = sizeof(T) == 4 && ctx->reuse_pieces && ctx->hx_X == (const void*)X &&
                       ctx->hx_Ns == Ns && ctx->Vf_hx != nullptr && ctx->wsX != nullptr &&
                       ctx->wsX_bytes >= (size_t)ctx->grid.N * Ns * sizeof(T);
  ctx->hx_X = nullptr;
  const size_t blk = (size_t)ctx->grid.N * Ns * sizeof(T);
  int rc = ensure(&ctx->wsX, &ctx->wsX_bytes, blk);
  if (rc) return rc;
  void *gA, *gB;
  rc = gc_buffer(ctx, Ns, &gA, &gB);
  if (rc) return rc;
  T* gC = (T*)gA;        // projections gamma c^T of the current iterate
  T* gN = (T*)gB;        // projections of the step's output
  const size_t gbytes = (size_t)ctx->proj.n_proj * Ns * sizeof(T);
  T* W = (T*)ctx->wsX;
  const double e = 0.5 * (b - a), c = 0.5 * (b + a);
  const double s1 = e / (a0 - c);
  const double tau = 2.0 / s1;
  double s = s1;
  T* cur = W;      // holds Y_1 after the first step
  T* prev = X;     // holds Y_0
  const bool nl = ctx->proj.n_proj > 0;
  // one step: local stencil into `out`, then the nonlocal pass in place,
  // which also accumulates the projections of the result for the next step
  int nrc = SQ3_OK;
  auto step = [&](const T* yk, const T* ykm1, T* out, double sc1, double sc2,
                  bool want_next) {
    {
      Prof p(ctx, ST_STENCIL);
      launch_cheb_step<T>(ctx, yk, ykm1, out, Ns, sc1, c, sc2, ctx->stream);
    }
    if (nl && nrc == SQ3_OK) {
      Prof p(ctx, ST_NL_PASS);
      if (want_next) cudaMemsetAsync(gN, 0, gbytes, ctx->stream);
      nrc = launch_nl_pass<T>(ctx, out, gC, want_next ? gN : nullptr, Ns, sc1, ctx->stream);
    }
  };
  if (from_hx) {
    // Y_1 = (s1/e)(H X - c X) from the kept H X: W = (s1/e)(W + (V - V_hx - c) X),
    // then the projections of Y_1 for the second step
    {
      Prof p(ctx, ST_STENCIL);
      filter_first_from_hx(ctx, (float*)W, (const float*)X, Ns, s1 / e, c);
    }
    if (nl && m > 1) {
      Prof p(ctx, ST_NL_PROJECT);
      cudaMemsetAsync(gN, 0, gbytes, ctx->stream);
      nrc = launch_nl_pass<T>(ctx, W, nullptr, gN, Ns, 0.0, ctx->stream);
    }
  } else {
    if (nl) {
      // projections of the input block (projection-only nonlocal pass)
      Prof p(ctx, ST_NL_PROJECT);
      cudaMemsetAsync(gC, 0, gbytes, ctx->stream);
      nrc = launch_nl_pass<T>(ctx, X, nullptr, gC, Ns, 0.0, ctx->stream);
    }
    step(X, nullptr, W, s1 / e, 0.0, m > 1);
  }
  for (int k = 2; k <= m; ++k) {
    const double sn = 1.0 / (tau - s);
    if (nl) std::swap(gC, gN);
    // Y_k overwrites Y_{k-2} in place (each element reads only its yprev)
    step(cur, prev, prev, 2.0 * sn / e, -s * sn, k < m);
    std::swap(cur, prev);
    s = sn;
  }
  if (nrc) return nrc;
  if (cur != X) {
    Prof p(ctx, ST_COPY, 0);
    rc = cuda_err(cudaMemcpyAsync(X, cur, blk, cudaMemcpyDeviceToDevice,
                                  ctx->stream));
  }
  if (rc) return rc;
  return cuda_err(cudaGetLastError());
}

static int splitk_for(int tiles, long long K) {
  int want = (4 * 152 + tiles - 1) / tiles;
  long long maxs = K / 512;
  if (maxs < 1) maxs = 1;
  if (want > maxs) want = (int)maxs;
  return want < 1 ? 1 : want;
}

// S = A^T B for N x Ns column-major blocks A, B (FP64).
static void gram_f64(sq3_ctx* ctx, const double* A, const double* B, int Ns,
                     double* S, int stage) {
  Prof p(ctx, stage);
  const long long N = ctx->grid.N;
  cudaMemsetAsync(S, 0, (size_t)Ns * Ns * sizeof(double), ctx->stream);
  GemmArgs g{};
  g.M = Ns; g.N = Ns; g.K = (int)N;
  g.A = A; g.lda = N; g.a_kcontig = true;
  g.B = B; g.ldb = N; g.b_kcontig = true;
  g.C = S; g.ldc = Ns; g.alpha = 1.0;
  const int nt = (Ns + 63) / 64;
  g.splits = splitk_for(nt * (nt + 1) / 2, N);
  g.tri = 1;                       // S is symmetric: upper tiles only
  gemm_f64(g, EPI_ATOMIC, ctx->stream);
  mirror_upper_f64(S, Ns, ctx->stream);
}

static int orthonormalise_f64(sq3_ctx* ctx, double* X, int Ns) {
  const long long N = ctx->grid.N;
  const size_t blk = (size_t)N * Ns * sizeof(double);
  int rc = ensure(&ctx->wsX, &ctx->wsX_bytes, blk);
  if (rc) return rc;
  rc = ensure((void**)&ctx->wsMat, &ctx->wsMat_bytes,
              ((size_t)2 * Ns * Ns + Ns) * sizeof(double));
  if (rc) return rc;
  double* S = ctx->wsMat;
  double* Rinv = ctx->wsMat + (size_t)Ns * Ns;
  double* diag = Rinv + (size_t)Ns * Ns;
  gram_f64(ctx, X, X, Ns, S, ST_GRAM);
  {
    const int panels = (Ns + 63) / 64;
    Prof p(ctx, ST_CHOL, 3 * panels - 1);
    rc = cholesky_lower_f64(ctx, S, Ns, diag, ctx->stream);
  }
  if (rc) return rc;
  {
    Prof p(ctx, ST_TRINV);
    tri_inverse_transpose_f64(S, Rinv, Ns, diag, ctx->stream);
  }
  GemmArgs g{};
  g.M = (int)N; g.N = Ns; g.K = Ns;
  g.A = X; g.lda = N; g.a_kcontig = false;
  g.B = Rinv; g.ldb = Ns; g.b_kcontig = true;
  g.C = (double*)ctx->wsX; g.ldc = N; g.alpha = 1.0; g.beta = 0.0;
  g.splits = 1;
  g.tri = 2;                       // R^{-1} is upper triangular
  {
    Prof p(ctx, ST_XRINV);
    gemm_f64(g, EPI_STORE, ctx->stream);
  }
  {
    Prof p(ctx, ST_COPY, 0);
    rc = cuda_err(cudaMemcpyAsync(X, ctx->wsX, blk, cudaMemcpyDeviceToDevice,
                                  ctx->stream));
  }
  if (rc) return rc;
  rc = cuda_err(cudaGetLastError());
  if (rc) return rc;
  return check_device_status(ctx);
}

static int project_f64(sq3_ctx* ctx, const double* X, int Ns, double* Hs) {
  const size_t blk = (size_t)ctx->grid.N * Ns * sizeof(double);
  int rc = ensure(&ctx->wsX, &ctx->wsX_bytes, blk);
  if (rc) return rc;
  rc = hamiltonian_apply_t<double>(ctx, X, (double*)ctx->wsX, Ns);
  if (rc) return rc;
  // upper triangle of X^T (H X), mirrored: H is symmetric
  gram_f64(ctx, X, (const double*)ctx->wsX, Ns, Hs, ST_HS_GEMM);
  return cuda_err(cudaGetLastError());
}

static int density_f64(sq3_ctx* ctx, const double* X, const double* D, int Ns,
                       double* rho) {
  const long long N = ctx->grid.N;
  cudaMemsetAsync(rho, 0, (size_t)N * sizeof(double), ctx->stream);
  GemmArgs g{};
  g.M = (int)N; g.N = Ns; g.K = Ns;
  g.A = X; g.lda = N; g.a_kcontig = false;
  g.B = D; g.ldb = Ns; g.b_kcontig = true;
  g.X = X; g.ldx = N; g.rho = rho;
  g.alpha = 2.0 / ctx->dV;
  g.splits = 1;
  Prof p(ctx, ST_RHO);
  gemm_f64(g, EPI_RHO, ctx->stream);
  return cuda_err(cudaGetLastError());
}

static int finish(sq3_ctx* ctx, int rc) {
  if (rc) {
    cudaStreamSynchronize(ctx->stream);
    cudaGetLastError();
    return rc;
  }
  rc = cuda_err(cudaGetLastError());
  if (rc) return rc;
  return check_device_status(ctx);
}

static bool ready(const sq3_ctx* ctx) { return ctx && ctx->grid_ok && ctx->pot_ok; }

}  // namespace sq3

using namespace sq3;

extern "C" {

const char* sq3_version(void) { return "sq3-gb300 0.1 (sm_103a)"; }

const char* sq3_last_cuda_error(void) { return g_last_cuda_error; }

int sq3_fermi_degree(double sigma, double xi, double tol) {
  if (!(sigma > 0) || !(xi > 0) || !(tol > 0) || !(tol < 1) || !isfinite(sigma) ||
      !isfinite(xi))
    return SQ3_EINVAL;
  const double a = 3.14159265358979323846 * sigma / xi;
  const double lr = log(a + sqrt(1.0 + a * a));   // ln rho > 0
  const double n = ceil(log(1.0 / tol) / lr);
  if (!(n < 2147483647.0)) return SQ3_EINVAL;
  return n < 1.0 ? 1 : (int)n;
}

const char* sq3_status_string(int s) {
  switch (s) {
    case SQ3_OK: return "ok";
    case SQ3_EINVAL: return "invalid argument";
    case SQ3_ENOTSETUP: return "grid or potential not set";
    case SQ3_ECUDA: return "CUDA error";
    case SQ3_ENOTPD: return "Cholesky pivot not positive (X^T X not positive definite)";
    case SQ3_ENOCONV: return "Fermi-level bracket or spectral bound check failed";
    case SQ3_ETIMEOUT: return "bounded device wait timed out";
    case SQ3_ENONFINITE: return "non-finite value detected";
    case SQ3_ENOMEM: return "workspace allocation failed";
    default: return "unknown status";
  }
}

int sq3_create(sq3_ctx** out, int device, void* cuda_stream) {
  if (!out) return SQ3_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return device < 0 ? SQ3_EINVAL : SQ3_ECUDA;
  }
  if (cudaSetDevice(device) != cudaSuccess) return SQ3_ECUDA;
  sq3_ctx* c = new sq3_ctx();
  c->device = device;
  c->stream = (cudaStream_t)cuda_stream;
  if (cudaMalloc((void**)&c->dev_status, sizeof(int)) != cudaSuccess ||
      cudaMalloc((void**)&c->dev_scal, SQ3_DEV_SCAL * sizeof(double)) != cudaSuccess ||
      cudaMallocHost((void**)&c->host_scal, 64 * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    sq3_destroy(c);
    return SQ3_ECUDA;
  }
  cudaMemset(c->dev_status, 0, sizeof(int));
  cudaMemset(c->dev_scal, 0, SQ3_DEV_SCAL * sizeof(double));
  *out = c;
  return SQ3_OK;
}

void sq3_destroy(sq3_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  else cudaDeviceSynchronize();
  free_projectors(c->proj);
  for (auto& r : c->prof_recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
  for (auto e : c->prof_pool) cudaEventDestroy(e);
  if (c->copy_stream) cudaStreamSynchronize(c->copy_stream);
  for (auto e : c->upload_ev) if (e) cudaEventDestroy(e);
  if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
  if (c->Vf_hx) cudaFree(c->Vf_hx);
  void* ptrs[] = {c->V, c->Vf, c->dev_status, c->dev_scal, c->wsX, c->wsX2,
                  c->wsMat, c->wsT, c->wsProj, c->wsSplit, c->wsFoe, c->wsLin32,
                  c->scfTab, c->wsScf, c->wsMix, c->wsDrv, c->wsAtoms};
  for (void* p : ptrs) if (p) cudaFree(p);
  if (c->host_scal) cudaFreeHost(c->host_scal);
  delete c;
}

int sq3_setup_grid(sq3_ctx* c, int nx, int ny, int nz, double Lx, double Ly,
                   double Lz, int fd_order) {
  if (!c || fd_order < 2 || fd_order > 2 * SQ3_MAX_FD_RADIUS || fd_order % 2)
    return SQ3_EINVAL;
  c->hx_X = nullptr;
  if (c->Vf_hx) {                          // sized for the previous grid
    cudaSetDevice(c->device);
    cudaFree(c->Vf_hx);
    c->Vf_hx = nullptr;
  }
  const int R = fd_order / 2;
  if (nx < R || ny < R || nz < R || nx > 512 ||
      !(Lx > 0) || !(Ly > 0) || !(Lz > 0))
    return SQ3_EINVAL;
  cudaSetDevice(c->device);
  Grid g{};
  g.nx = nx; g.ny = ny; g.nz = nz;
  g.N = (long long)nx * ny * nz;
  g.hx = Lx / nx; g.hy = Ly / ny; g.hz = Lz / nz;
  g.radius = R;
  fd_weights(fd_order, g.w);
  c->grid = g;
  c->Lx = Lx; c->Ly = Ly; c->Lz = Lz;
  c->dV = g.hx * g.hy * g.hz;
  c->grid_ok = true;
  c->pot_ok = false;
  c->scf_tab_ok = false;
  c->mix.ready = false;
  if (c->V) cudaFree(c->V);
  if (c->Vf) cudaFree(c->Vf);
  c->V = nullptr; c->Vf = nullptr;
  free_projectors(c->proj);
  return SQ3_OK;
}

int sq3_set_potential(sq3_ctx* c, const double* V) {
  if (!c || !c->grid_ok) return SQ3_ENOTSETUP;
  if (!V) return SQ3_EINVAL;
  cudaSetDevice(c->device);
  const long long N = c->grid.N;
  if (!c->V) {
    if (cudaMalloc((void**)&c->V, N * sizeof(double)) != cudaSuccess ||
        cudaMalloc((void**)&c->Vf, N * sizeof(float)) != cudaSuccess) {
      cudaGetLastError();
      return SQ3_ENOMEM;
    }
  }
  int rc = cuda_err(cudaMemcpyAsync(c->V, V, N * sizeof(double),
                                    cudaMemcpyDeviceToDevice, c->stream));
  if (rc) return rc;
  to_float_kernel<<<(unsigned)((N + 255) / 256), 256, 0, c->stream>>>(c->V, c->Vf, N);
  // range of the potential (the Chebyshev filter's spectral bounds use it)
  // and a check that every value is finite
  double* part = c->dev_scal + SQ3_SCAL_MISC;
  double* mm = part + 2 * MM_BLOCKS;
  minmax(c->V, N, part, mm, c->dev_status, c->stream);
  rc = cuda_err(cudaMemcpyAsync(c->host_scal + 62, mm, 2 * sizeof(double),
                                cudaMemcpyDeviceToHost, c->stream));
  if (rc) return finish(c, rc);
  rc = finish(c, 0);
  c->pot_ok = rc == SQ3_OK;
  if (rc) return rc;
  c->v_min = c->host_scal[62];
  c->v_max = c->host_scal[63];
  return SQ3_OK;
}

// The CSR projector table's own checks (indices inside the grid of N
// points, ptr monotone from 0, every value and energy finite).
static int check_projector_table(long long N, int n_proj, const int* ptr, const int* idx,
                                 const double* val, const double* gamma) {
  if (n_proj < 0) return SQ3_EINVAL;
  if (n_proj == 0) return SQ3_OK;
  if (!ptr || !idx || !val || !gamma || ptr[0] != 0) return SQ3_EINVAL;
  for (int p = 0; p < n_proj; ++p)
    if (ptr[p + 1] < ptr[p] || !isfinite(gamma[p])) return SQ3_EINVAL;
  for (long long e = 0; e < (long long)ptr[n_proj]; ++e)
    if (idx[e] < 0 || idx[e] >= N || !isfinite(val[e])) return SQ3_EINVAL;
  return SQ3_OK;
}

int sq3_projector_table_info(int nx, int ny, int nz, double dV, int n_proj, const int* ptr,
                             const int* idx, const double* val, const double* gamma, int* info,
                             double* bounds) {
  if (nx < 1 || ny < 1 || nz < 1 || !(dV > 0) || !info || !bounds) return SQ3_EINVAL;
  const long long N = (long long)nx * ny * nz;
  int rc = check_projector_table(N, n_proj, ptr, idx, val, gamma);
  if (rc) return rc;
  for (int i = 0; i < 6; ++i) info[i] = 0;
  bounds[0] = bounds[1] = 0.0;
  if (n_proj == 0) return SQ3_OK;
  ProjectorHostTables T;
  projector_host_tables(nx, ny, nz, dV, n_proj, ptr, idx, val, gamma, T);
  info[0] = (int)T.bp0.size();
  info[1] = (int)T.qlb.size();
  info[2] = (int)(T.sptr.size() - 1);
  info[3] = T.max_brick_balls;
  info[4] = T.max_brick_entries;
  info[5] = (int)nl_pass_smem_bytes(4, 16, 3, T.max_brick_balls, T.max_brick_entries);
  bounds[0] = T.vnl_lo;
  bounds[1] = T.vnl_hi;
  return SQ3_OK;
}

int sq3_set_projectors(sq3_ctx* c, int n_proj, const int* ptr, const int* idx,
                       const double* val, const double* gamma) {
  if (!c || !c->grid_ok) return SQ3_ENOTSETUP;
  if (n_proj < 0) return SQ3_EINVAL;
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  const long long N = c->grid.N;
  // a rejected table leaves the context's projectors as they were
  if (check_projector_table(N, n_proj, ptr, idx, val, gamma)) return SQ3_EINVAL;
  free_projectors(c->proj);
  c->hx_X = nullptr;
  if (n_proj == 0) return SQ3_OK;
  ProjectorHostTables T;
  projector_host_tables(c->grid.nx, c->grid.ny, c->grid.nz, c->dV, n_proj, ptr, idx, val,
                        gamma, T);
  Projectors P;
  P.n_proj = n_proj;
  P.n_ball = (int)T.bp0.size();
  P.vnl_lo = T.vnl_lo;
  P.vnl_hi = T.vnl_hi;
  P.max_brick_balls = T.max_brick_balls;
  P.max_brick_entries = T.max_brick_entries;
  int rc = SQ3_OK;
  // shared memory of the nonlocal pass, FP64 variant (two boxes of 8
  // vectors, two coefficient buffers, both entry orders, barriers, alignment)
  if (nl_pass_smem_bytes(8, 8, 2, T.max_brick_balls, T.max_brick_entries) > 227 * 1024)
    rc = SQ3_EINVAL;
  rc = rc ? rc : upload(&P.gamma, gamma, (size_t)n_proj);
  rc = rc ? rc : upload(&P.nb_ball_ptr, T.sptr.data(), T.sptr.size());
  rc = rc ? rc : upload(&P.nb_slot_pid, T.spid.data(), T.spid.size());
  rc = rc ? rc : upload(&P.nb_pt_ptr, T.qptr.data(), T.qptr.size());
  rc = rc ? rc : upload(&P.nb_pt_lb, T.qlb.data(), T.qlb.size());
  rc = rc ? rc : upload(&P.nb_pt_val, T.qval.data(), T.qval.size());
  rc = rc ? rc : upload(&P.nb_bl_ptr, T.zptr.data(), T.zptr.size());
  rc = rc ? rc : upload(&P.nb_bl_pt, T.zpt.data(), T.zpt.size());
  rc = rc ? rc : upload(&P.nb_bl_val, T.zval.data(), T.zval.size());
  // FP32 copies of the values, converted on the device
  for (int w = 0; w < 2 && rc == SQ3_OK; ++w) {
    const double* src = w ? P.nb_bl_val : P.nb_pt_val;
    float** dst = w ? &P.nb_bl_valf : &P.nb_pt_valf;
    const long long n = (long long)(w ? T.zval.size() : T.qval.size());
    if (n == 0) continue;
    if (cudaMalloc((void**)dst, (size_t)n * sizeof(float)) != cudaSuccess) {
      cudaGetLastError();
      *dst = nullptr;
      rc = SQ3_ENOMEM;
      break;
    }
    to_float_kernel<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(src, *dst, n);
  }
  if (rc == SQ3_OK) rc = cuda_err(cudaStreamSynchronize(c->stream));
  P.h_bptr = std::move(T.bptr);
  P.h_bidx = std::move(T.bidx);
  P.h_bp0 = std::move(T.bp0);
  P.h_bnp = std::move(T.bnp);
  P.h_boff = std::move(T.boff);
  P.h_bval = std::move(T.bval);
  P.h_gamma.assign(gamma, gamma + n_proj);
  c->proj = std::move(P);
  if (rc) { free_projectors(c->proj); return rc; }
  return SQ3_OK;
}

int sq3_hamiltonian_apply(sq3_ctx* c, const void* X, void* Y, int Ns,
                          sq3_prec prec) {
  if (!ready(c)) return SQ3_ENOTSETUP;
  if (!X || !Y || Ns <= 0 || X == Y || Ns > 65535) return SQ3_EINVAL;
  cudaSetDevice(c->device);
  int rc;
  if (prec == SQ3_FP64) rc = hamiltonian_apply_t<double>(c, (const double*)X, (double*)Y, Ns);
  else if (prec == SQ3_MIXED) rc = hamiltonian_apply_t<float>(c, (const float*)X, (float*)Y, Ns);
  else return SQ3_EINVAL;
  return finish(c, rc);
}

int sq3_cheb_filter(sq3_ctx* c, void* X, int Ns, int degree, double a,
                    double b, double a0, sq3_prec prec) {
  if (!ready(c)) return SQ3_ENOTSETUP;
  if (!X || Ns <= 0 || Ns > 65535 || degree < 1 || !(a0 < a) || !(a < b))
    return SQ3_EINVAL;
  cudaSetDevice(c->device);
  int rc;
  if (prec == SQ3_FP64) rc = cheb_filter_t<double>(c, (double*)X, Ns, degree, a, b, a0);
  else if (prec == SQ3_MIXED) rc = cheb_filter_t<float>(c, (float*)X, Ns, degree, a, b, a0);
  else return SQ3_EINVAL;
  return finish(c, rc);
}

namespace sq3 {
// One CTA waits on an mbarrier that nothing completes, through the same
// bounded wait (ac::mbar_wait, about one second) that the library's kernels
// use for their TMA and tensor-core barriers; when it runs out the kernel
// records DEV_TIMEOUT and returns.
__global__ void timeout_selftest_kernel(int* status) {
  __shared__ __align__(8) uint64_t bar;
  const uint32_t b = ac::smem_u32(&bar);
  if (threadIdx.x == 0) {
    ac::mbar_init(b, 1);
    ac::mbar_init_fence();
  }
  __syncthreads();
  if (threadIdx.x == 0 && !ac::mbar_wait(b, 0)) atomicCAS(status, DEV_OK, DEV_TIMEOUT);
}
}  // namespace sq3

int sq3_selftest_timeout(sq3_ctx* c) {
  if (!c) return SQ3_EINVAL;
  cudaSetDevice(c->device);
  timeout_selftest_kernel<<<1, 32, 0, c->stream>>>(c->dev_status);
  const int rc = cuda_err(cudaGetLastError());
  if (rc) return rc;
  // SQ3_ETIMEOUT when the wait ran out as it should; the status word is
  // cleared by the check, so the context stays usable
  return check_device_status(c);
}

int sq3_cheb_filter_from_host(sq3_ctx* c, const void* X_host, void* X, int Ns, int degree,
                              double a, double b, double a0, sq3_prec prec) {
  if (c) c->pieces_X = nullptr;
  if (!ready(c)) return SQ3_ENOTSETUP;
  if (!X_host || !X || Ns <= 0 || Ns > 65535 || degree < 1 || !(a0 < a) || !(a < b))
    return SQ3_EINVAL;
  if (prec != SQ3_FP64 && prec != SQ3_MIXED) return SQ3_EINVAL;
  cudaSetDevice(c->device);
  if (!c->copy_stream) {
    if (cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking) != cudaSuccess) {
      c->copy_stream = nullptr;
      cudaGetLastError();
      return SQ3_ECUDA;
    }
    for (auto& e : c->upload_ev)
      if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
        e = nullptr;
        cudaGetLastError();
        return SQ3_ECUDA;
      }
  }
  // every vector is filtered on its own (the filter is p_m(H) applied column
  // by column), so a chunk of the vectors is filtered as soon as its upload
  // has landed while the rest is still being copied.  Two chunks: the first
  // eighth of the vectors, whose filtering (m stencil and nonlocal steps)
  // outlasts the copy of the other seven eighths, then those in one piece,
  // which keeps the filter's launches as large as possible (a nonlocal pass
  // over few vectors stages its brick tables for fewer vector groups).
  const size_t es = prec == SQ3_FP64 ? sizeof(double) : sizeof(float);
  const size_t vbytes = (size_t)c->grid.N * es;
  const int cut = (Ns + 7) / 8;
  const int v0s[SQ3_UPLOAD_CHUNKS] = {0, cut};
  const int nvs[SQ3_UPLOAD_CHUNKS] = {cut, Ns - cut};
  int rc = SQ3_OK;
  for (int k = 0; k < SQ3_UPLOAD_CHUNKS && nvs[k] > 0 && rc == SQ3_OK; ++k) {
    const int v0 = v0s[k], nv = nvs[k];
    rc = cuda_err(cudaMemcpyAsync((char*)X + v0 * vbytes, (const char*)X_host + v0 * vbytes,
                                  nv * vbytes, cudaMemcpyHostToDevice, c->copy_stream));
    if (rc == SQ3_OK) rc = cuda_err(cudaEventRecord(c->upload_ev[k], c->copy_stream));
  }
  for (int k = 0; k < SQ3_UPLOAD_CHUNKS && nvs[k] > 0 && rc == SQ3_OK; ++k) {
    const int v0 = v0s[k], nv = nvs[k];
    rc = cuda_err(cudaStreamWaitEvent(c->stream, c->upload_ev[k], 0));
    if (rc) break;
    if (prec == SQ3_FP64)
      rc = cheb_filter_t<double>(c, (double*)X + (size_t)v0 * c->grid.N, nv, degree, a, b, a0);
    else
      rc = cheb_filter_t<float>(c, (float*)X + (size_t)v0 * c->grid.N, nv, degree, a, b, a0);
  }
  // no copy of this call is left in flight when it returns
  if (cudaStreamSynchronize(c->copy_stream) != cudaSuccess && rc == SQ3_OK) rc = SQ3_ECUDA;
  return finish(c, rc);
}

int sq3_orthonormalise(sq3_ctx* c, void* X, int Ns, sq3_prec prec) {
  if (!ready(c)) return SQ3_ENOTSETUP;
  if (!X || Ns <= 0 || Ns > c->grid.N) return SQ3_EINVAL;
  cudaSetDevice(c->device);
  int rc;
  if (prec == SQ3_FP64) rc = orthonormalise_f64(c, (double*)X, Ns);
  else if (prec == SQ3_MIXED) rc = orthonormalise_mixed(c, (float*)X, Ns);
  else return SQ3_EINVAL;
  return finish(c, rc);
}

int sq3_project(sq3_ctx* c, const void* X, int Ns, sq3_prec prec, double* Hs) {
  if (!ready(c)) return SQ3_ENOTSETUP;
  if (!X || !Hs || Ns <= 0 || Ns > 65535) return SQ3_EINVAL;
  cudaSetDevice(c->device);
  int rc;
  if (prec == SQ3_FP64) rc = project_f64(c, (const double*)X, Ns, Hs);
  else if (prec == SQ3_MIXED) rc = project_mixed(c, (const float*)X, Ns, Hs);
  else return SQ3_EINVAL;
  return finish(c, rc);
}

int sq3_kernel_from_hs(sq3_ctx* c, const double* Hs, int Ns, int npl,
                       double kT, double Ne, sq3_prec prec,
                       const double* bounds_in, double* D, double* out) {
  if (npl < 1) return SQ3_EINVAL;
  return sq3_kernel_from_hs_ex(c, Hs, Ns, npl, 0.0, SQ3_EVAL_RECURRENCE, kT, Ne, prec,
                               bounds_in, D, out, nullptr);
}

int sq3_kernel_from_hs_ex(sq3_ctx* c, const double* Hs, int Ns, int npl, double fermi_tol,
                          int eval_mode, double kT, double Ne, sq3_prec prec,
                          const double* bounds_in, double* D, double* out, int* npl_used) {
  if (!c) return SQ3_EINVAL;
  if (!Hs || !out || Ns <= 0 || npl > SQ3_MAX_NPL || !(kT > 0) ||
      !(Ne > 0) || !(Ne < 2.0 * Ns))
    return SQ3_EINVAL;
  if (npl < 1 && !(fermi_tol > 0 && fermi_tol < 1)) return SQ3_EINVAL;
  if (eval_mode != SQ3_EVAL_RECURRENCE && eval_mode != SQ3_EVAL_PATERSON_STOCKMEYER)
    return SQ3_EINVAL;
  if (bounds_in && !(bounds_in[1] > 0)) return SQ3_EINVAL;
  if (prec != SQ3_FP64 && prec != SQ3_MIXED) return SQ3_EINVAL;
  cudaSetDevice(c->device);
  int used = 0;
  int rc = density_kernel_from_hs(c, Hs, Ns, npl, kT, Ne, bounds_in, D, out,
                                  prec == SQ3_MIXED, fermi_tol, eval_mode, &used);
  if (npl_used) *npl_used = used;
  return finish(c, rc);
}

int sq3_density_kernel(sq3_ctx* c, const void* X, int Ns, int npl, double kT,
                       double Ne, sq3_prec prec, const double* bounds_in,
                       double* Hs_out, double* D, double* out) {
  if (!ready(c)) return SQ3_ENOTSETUP;
  if (!X || !out || Ns <= 0) return SQ3_EINVAL;
  cudaSetDevice(c->device);
  double* Hs = Hs_out;
  int rc;
  if (!Hs) {
    rc = ensure(&c->wsX2, &c->wsX2_bytes, (size_t)Ns * Ns * sizeof(double));
    if (rc) return rc;
    Hs = (double*)c->wsX2;
  }
  rc = sq3_project(c, X, Ns, prec, Hs);
  if (rc) return rc;
  return sq3_kernel_from_hs(c, Hs, Ns, npl, kT, Ne, prec, bounds_in, D, out);
}

int sq3_profile_enable(sq3_ctx* c, int enable) {
  if (!c) return SQ3_EINVAL;
  c->prof = enable != 0;
  return SQ3_OK;
}

int sq3_profile_read(sq3_ctx* c, double* ms, long long* launches, int n) {
  if (!c) return SQ3_EINVAL;
  cudaSetDevice(c->device);
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return SQ3_ECUDA;
  std::vector<double> t(ST_COUNT, 0.0);
  std::vector<long long> l(ST_COUNT, 0);
  for (auto& r : c->prof_recs) {
    float x = 0.f;
    cudaEventElapsedTime(&x, r.a, r.b);
    t[r.stage] += x;
    l[r.stage] += r.launches;
    c->prof_pool.push_back(r.a);
    c->prof_pool.push_back(r.b);
  }
  c->prof_recs.clear();
  for (int s = 0; s < n && s < ST_COUNT; ++s) {
    if (ms) ms[s] = t[s];
    if (launches) launches[s] = l[s];
  }
  return ST_COUNT;
}

int sq3_density(sq3_ctx* c, const void* X, const double* D, int Ns,
                sq3_prec prec, double* rho) {
  if (!ready(c)) return SQ3_ENOTSETUP;
  if (!X || !D || !rho || Ns <= 0 || Ns > 65535) return SQ3_EINVAL;
  cudaSetDevice(c->device);
  int rc;
  if (prec == SQ3_FP64) rc = density_f64(c, (const double*)X, D, Ns, rho);
  else if (prec == SQ3_MIXED) rc = density_mixed(c, (const float*)X, D, Ns, rho);
  else return SQ3_EINVAL;
  // a NaN or infinity anywhere in X or D reaches rho: report it
  if (rc == SQ3_OK) check_finite(rho, c->grid.N, c->dev_status, c->stream);
  return finish(c, rc);
}

}  // extern "C"
