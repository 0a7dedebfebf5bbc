// The self-consistent-field pieces around the fixed-potential iteration:
// the electrostatic potential of the total charge (Sec. 2, Eq. (poisson)),
// the LDA exchange-correlation potential (Sec. 2), the effective potential
// V_eff = phi + V_xc of Eq. (KSeqn), the free energy of
// Eq. (FreeEnergy:NewForm), and the Kerker preconditioner of the density
// mixing that Sec. 5 cites.
//
// Poisson.  The grid Laplacian L_h is the same central finite-difference
// operator as in the Hamiltonian.  It is a sum of three 1-D circulant
// operators, each diagonal in the real orthonormal Fourier basis of its axis
// (columns 1/sqrt(n), sqrt(2/n) cos(2 pi f k / n), sqrt(2/n) sin(2 pi f k / n),
// and (-1)^k / sqrt(n) for even n), with eigenvalue -s(theta_f) / h^2,
// s(theta) = -w_0 - 2 sum_p w_p cos(p theta).  So -L_h phi = 4 pi (rho + b)
// is solved exactly by three forward basis changes (one per axis), a
// division by (s_x + s_y + s_z) / (4 pi) per mode with the zero mode set to
// zero (the total charge is zero; phi has zero mean), and three inverse
// basis changes.  Each basis change is a contraction of length n along one
// axis; the whole solve is 6 n FMAs per point, far below the cost of the
// rest of an iteration, so the kernels read their operands through the
// cache instead of staging them.
//
// Determinism: every sum (the basis changes, the per-block partial energies
// and their final sum) runs in a fixed order, so repeated calls agree bit
// for bit.
#include <math.h>

#include <algorithm>
#include <vector>

#include "sq3_internal.cuh"

namespace sq3 {

namespace {

constexpr int XC_BLOCKS = 304;   // fixed partial-sum blocks (2 per SM)
constexpr int XC_THREADS = 256;
constexpr double RHO_FLOOR = 1e-14;
constexpr double PI = 3.14159265358979323846;

// Perdew-Wang 1992 correlation of the spin-unpolarised electron gas
// (A, alpha1, beta1..beta4, p = 1).
constexpr double PW_A = 0.031091;
constexpr double PW_ALPHA1 = 0.21370;
constexpr double PW_B1 = 7.5957, PW_B2 = 3.5876, PW_B3 = 1.6382, PW_B4 = 0.49294;

// Spectral scalings applied after the forward basis changes.
enum ModeScale : int {
  SCALE_POISSON = 0,   // 4 pi / (lam_x + lam_y + lam_z), zero mode 0
  SCALE_KERKER = 1,    // g2 / (g2 + k0^2), g2 = G_x^2 + G_y^2 + G_z^2
};

// Column m of the real Fourier basis of n points: its integer frequency f
// and whether it is the sine of the pair.
struct Col { int f; bool sine; };
inline Col column(int n, int m) {
  if (m == 0) return {0, false};
  if (n % 2 == 0 && m == n - 1) return {n / 2, false};
  return {(m + 1) / 2, (m % 2) == 0};
}

// Q[k * n + m] = column m at point k; lam[m] = s(theta_f) / h^2 (the FD
// eigenvalue, sign flipped); g2[m] = (2 pi f / L)^2 (continuum).
void basis_tables(int n, double h, double L, int R, const double* w, double* Q,
                  double* lam, double* g2) {
  for (int m = 0; m < n; ++m) {
    const Col c = column(n, m);
    const double scale = (c.f == 0 || 2 * c.f == n) ? 1.0 / sqrt((double)n)
                                                    : sqrt(2.0 / (double)n);
    for (int k = 0; k < n; ++k) {
      const double arg = 2.0 * PI * (double)(((long long)c.f * k) % n) / (double)n;
      Q[(size_t)k * n + m] = scale * (c.sine ? sin(arg) : cos(arg));
    }
    double s = -w[0];
    for (int p = 1; p <= R; ++p)
      s -= 2.0 * w[p] * cos(2.0 * PI * (double)(((long long)p * c.f) % n) / (double)n);
    lam[m] = s / (h * h);
    const double g = 2.0 * PI * (double)c.f / L;
    g2[m] = g * g;
  }
}

// Table layout: Qx | Qy | Qz | lam_x | lam_y | lam_z | g2_x | g2_y | g2_z.
struct TabPtrs {
  const double *Qx, *Qy, *Qz, *lx, *ly, *lz, *gx, *gy, *gz;
};

size_t table_words(const Grid& g) {
  return (size_t)g.nx * g.nx + (size_t)g.ny * g.ny + (size_t)g.nz * g.nz +
         3 * (size_t)(g.nx + g.ny + g.nz);
}

TabPtrs table_ptrs(const Grid& g, const double* t) {
  TabPtrs p;
  p.Qx = t; t += (size_t)g.nx * g.nx;
  p.Qy = t; t += (size_t)g.ny * g.ny;
  p.Qz = t; t += (size_t)g.nz * g.nz;
  p.lx = t; t += g.nx;
  p.ly = t; t += g.ny;
  p.lz = t; t += g.nz;
  p.gx = t; t += g.nx;
  p.gy = t; t += g.ny;
  p.gz = t;
  return p;
}

int ensure_tables(sq3_ctx* ctx) {
  if (ctx->scf_tab_ok) return SQ3_OK;
  const Grid& g = ctx->grid;
  const size_t words = table_words(g);
  std::vector<double> h(words);
  double* t = h.data();
  double* Qx = t; t += (size_t)g.nx * g.nx;
  double* Qy = t; t += (size_t)g.ny * g.ny;
  double* Qz = t; t += (size_t)g.nz * g.nz;
  double* lx = t; t += g.nx;
  double* ly = t; t += g.ny;
  double* lz = t; t += g.nz;
  double* gx = t; t += g.nx;
  double* gy = t; t += g.ny;
  double* gz = t;
  basis_tables(g.nx, g.hx, ctx->Lx, g.radius, g.w, Qx, lx, gx);
  basis_tables(g.ny, g.hy, ctx->Ly, g.radius, g.w, Qy, ly, gy);
  basis_tables(g.nz, g.hz, ctx->Lz, g.radius, g.w, Qz, lz, gz);
  int rc = ensure((void**)&ctx->scfTab, &ctx->scfTab_bytes, words * sizeof(double));
  if (rc) return rc;
  rc = cuda_err(cudaMemcpy(ctx->scfTab, h.data(), words * sizeof(double),
                           cudaMemcpyHostToDevice));
  if (rc) return rc;
  ctx->scf_tab_ok = true;
  return SQ3_OK;
}

// Scratch: two N-point buffers, the per-block partial sums and 4 results.
int scf_scratch(sq3_ctx* ctx, double** A, double** B, double** part, double** res) {
  const size_t N = (size_t)ctx->grid.N;
  const size_t words = 2 * N + 3 * XC_BLOCKS + 4;
  int rc = ensure((void**)&ctx->wsScf, &ctx->wsScf_bytes, words * sizeof(double));
  if (rc) return rc;
  *A = ctx->wsScf;
  *B = *A + N;
  *part = *B + N;
  *res = *part + 3 * XC_BLOCKS;
  return SQ3_OK;
}

// One basis change along an axis of length n and stride sa (grid order
// [z][y][x], x fastest).  Forward (FWD): out(c) = sum_k Q[k][c] in(k);
// inverse: out(c) = sum_m Q[c][m] in(m).  in2, when given, is added to in
// (the total charge rho + b).  With `scale` >= 0 the output is multiplied by
// the mode's spectral factor (ModeScale), which needs all three coordinates.
template <bool FWD>
__global__ void __launch_bounds__(256)
axis_transform_kernel(const double* __restrict__ in, const double* __restrict__ in2,
                      double* __restrict__ out, const double* __restrict__ Q, int n,
                      long long sa, long long N, int nx, int ny, int scale, TabPtrs tp,
                      double k0sq) {
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < N;
       idx += (long long)gridDim.x * blockDim.x) {
    const int c = (int)((idx / sa) % n);
    const long long base = idx - (long long)c * sa;
    double acc = 0.0;
    if (in2) {
      for (int k = 0; k < n; ++k) {
        const double q = FWD ? __ldg(Q + (size_t)k * n + c) : __ldg(Q + (size_t)c * n + k);
        const long long p = base + (long long)k * sa;
        acc = fma(q, __ldg(in + p) + __ldg(in2 + p), acc);
      }
    } else {
      for (int k = 0; k < n; ++k) {
        const double q = FWD ? __ldg(Q + (size_t)k * n + c) : __ldg(Q + (size_t)c * n + k);
        acc = fma(q, __ldg(in + base + (long long)k * sa), acc);
      }
    }
    if (scale >= 0) {
      const int i = (int)(idx % nx);
      const int j = (int)((idx / nx) % ny);
      const int l = (int)(idx / ((long long)nx * ny));
      if (scale == SCALE_POISSON) {
        const double den = tp.lx[i] + tp.ly[j] + tp.lz[l];
        acc = (i == 0 && j == 0 && l == 0) ? 0.0 : acc * (4.0 * PI / den);
      } else {
        const double g2 = tp.gx[i] + tp.gy[j] + tp.gz[l];
        acc = (i == 0 && j == 0 && l == 0) ? 0.0 : acc * (g2 / (g2 + k0sq));
      }
    }
    out[idx] = acc;
  }
}

unsigned transform_blocks(long long N) {
  long long b = (N + 255) / 256;
  return (unsigned)(b < 65535LL * 64 ? b : 65535LL * 64);
}

// dst = forward basis changes, spectral factor, inverse basis changes of
// (src + src2).  A and B are N-point scratch; dst may alias src or src2
// (they are read by the first basis change only) but not A or B.
void spectral_apply(sq3_ctx* ctx, const double* src, const double* src2, double* dst,
                    int scale, double k0sq, double* A, double* B) {
  const Grid& g = ctx->grid;
  const TabPtrs tp = table_ptrs(g, ctx->scfTab);
  const long long N = g.N, sx = 1, sy = g.nx, sz = (long long)g.nx * g.ny;
  const unsigned blocks = transform_blocks(N);
  cudaStream_t st = ctx->stream;
  axis_transform_kernel<true><<<blocks, 256, 0, st>>>(src, src2, A, tp.Qx, g.nx, sx, N, g.nx,
                                                      g.ny, -1, tp, k0sq);
  axis_transform_kernel<true><<<blocks, 256, 0, st>>>(A, nullptr, B, tp.Qy, g.ny, sy, N, g.nx,
                                                      g.ny, -1, tp, k0sq);
  axis_transform_kernel<true><<<blocks, 256, 0, st>>>(B, nullptr, A, tp.Qz, g.nz, sz, N, g.nx,
                                                      g.ny, scale, tp, k0sq);
  axis_transform_kernel<false><<<blocks, 256, 0, st>>>(A, nullptr, B, tp.Qz, g.nz, sz, N, g.nx,
                                                       g.ny, -1, tp, k0sq);
  axis_transform_kernel<false><<<blocks, 256, 0, st>>>(B, nullptr, A, tp.Qy, g.ny, sy, N, g.nx,
                                                       g.ny, -1, tp, k0sq);
  axis_transform_kernel<false><<<blocks, 256, 0, st>>>(A, nullptr, dst, tp.Qx, g.nx, sx, N,
                                                       g.nx, g.ny, -1, tp, k0sq);
}

// LDA per point (Slater exchange + PW92 correlation), rho clamped below at
// RHO_FLOOR: energy per electron and potential.
__device__ __forceinline__ void lda_point(double rho, double& exc, double& vxc) {
  const double r = fmax(rho, RHO_FLOOR);
  const double ex = -0.75 * cbrt(3.0 * r / PI);
  const double vx = (4.0 / 3.0) * ex;
  const double rs = cbrt(3.0 / (4.0 * PI * r));
  const double sq = sqrt(rs);
  const double q0 = -2.0 * PW_A * (1.0 + PW_ALPHA1 * rs);
  const double q1 = 2.0 * PW_A * (PW_B1 * sq + PW_B2 * rs + PW_B3 * rs * sq + PW_B4 * rs * rs);
  const double q1p = PW_A * (PW_B1 / sq + 2.0 * PW_B2 + 3.0 * PW_B3 * sq + 4.0 * PW_B4 * rs);
  const double lg = log1p(1.0 / q1);
  const double ec = q0 * lg;
  const double dec = -2.0 * PW_A * PW_ALPHA1 * lg - q0 * q1p / (q1 * q1 + q1);
  exc = ex + ec;
  vxc = vx + ec - rs * dec / 3.0;
}

// Per point: V_xc, optional veff = phi + V_xc, and the block's partial sums
// of eps_xc rho, V_xc rho and (b - rho) phi (b may be null).  Fixed grid of
// XC_BLOCKS blocks; the block sum is a fixed-order tree.
__global__ void __launch_bounds__(XC_THREADS)
xc_kernel(const double* rho, const double* b, const double* phi, double* veff, long long N,
          double* __restrict__ part) {
  // veff may alias rho (each point is read before it is written, by the
  // same thread), so these pointers carry no __restrict__
  __shared__ double sh[3][XC_THREADS];
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  for (long long i = blockIdx.x * (long long)XC_THREADS + threadIdx.x; i < N;
       i += (long long)XC_BLOCKS * XC_THREADS) {
    const double r = rho[i];
    const double p = phi[i];
    double exc, vxc;
    lda_point(r, exc, vxc);
    if (veff) veff[i] = p + vxc;
    s0 = fma(exc, r, s0);
    s1 = fma(vxc, r, s1);
    s2 = fma((b ? b[i] : 0.0) - r, p, s2);
  }
  sh[0][threadIdx.x] = s0;
  sh[1][threadIdx.x] = s1;
  sh[2][threadIdx.x] = s2;
  __syncthreads();
  for (int w = XC_THREADS / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int t = 0; t < 3; ++t) sh[t][threadIdx.x] += sh[t][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < 3) part[3 * blockIdx.x + threadIdx.x] = sh[threadIdx.x][0];
}

// res[0] = E_xc, res[1] = int V_xc rho, res[2] = 1/2 int (b - rho) phi.
__global__ void xc_finish_kernel(const double* __restrict__ part, double dV,
                                 double* __restrict__ res) {
  const int t = threadIdx.x;
  if (t >= 3) return;
  double s = 0.0;
  for (int k = 0; k < XC_BLOCKS; ++k) s += part[3 * k + t];
  res[t] = (t == 2 ? 0.5 : 1.0) * s * dV;
}

int check_grid(const sq3_ctx* ctx) {
  if (!ctx) return SQ3_EINVAL;
  if (!ctx->grid_ok) return SQ3_ENOTSETUP;
  return SQ3_OK;
}

// phi of (rho + b) into dst, then the LDA terms (and veff when given).
int potential_and_terms(sq3_ctx* ctx, const double* rho, const double* b, double* phi_dst,
                        double* veff, double terms[3]) {
  cudaSetDevice(ctx->device);
  int rc = ensure_tables(ctx);
  if (rc) return rc;
  double *A, *B, *part, *res;
  rc = scf_scratch(ctx, &A, &B, &part, &res);
  if (rc) return rc;
  // the last inverse basis change reads A only, so B may receive phi
  double* phi = phi_dst ? phi_dst : B;
  spectral_apply(ctx, rho, b, phi, SCALE_POISSON, 0.0, A, B);
  xc_kernel<<<XC_BLOCKS, XC_THREADS, 0, ctx->stream>>>(rho, b, phi, veff, ctx->grid.N, part);
  xc_finish_kernel<<<1, 32, 0, ctx->stream>>>(part, ctx->dV, res);
  rc = cuda_err(cudaGetLastError());
  if (rc) return rc;
  rc = cuda_err(cudaMemcpyAsync(terms, res, 3 * sizeof(double), cudaMemcpyDeviceToHost,
                                ctx->stream));
  if (rc) return rc;
  rc = cuda_err(cudaStreamSynchronize(ctx->stream));
  if (rc) return rc;
  for (int t = 0; t < 3; ++t)
    if (!isfinite(terms[t])) return SQ3_ENONFINITE;
  return check_device_status(ctx);
}


// ---- Periodic Pulay mixing of the density (the mixing Sec. 5 cites) ----
//
// State (per context, reset by sq3_mixer_setup and sq3_setup_grid): the
// previous input and residual, and a ring of up to MIX_MAXH differences
// dX_a = x_k - x_{k-1}, dF_a = f_k - f_{k-1} (f = x_out - x_in).  Every
// period-th step the next input is x_bar + beta K f_bar with
// x_bar = x - DX c, f_bar = f - DF c and c the least-squares solution of
// DF c ~ f; the other steps mix linearly, x + beta K f.  K is the Kerker
// preconditioner (identity when k0 <= 0).  c solves the normal equations
// (DF^T DF) c = DF^T f by a Cholesky factorisation that drops a column whose
// pivot falls below 1e-12 of its diagonal (a difference that depends
// linearly on the earlier ones); with a full-rank history that is the
// least-squares solution, and with a deficient one it is still a
// least-squares solution (the same f_bar).

constexpr int MIX_MAXH = 8;
constexpr int MIX_NPAIR = MIX_MAXH * (MIX_MAXH + 1) / 2;
constexpr int MIX_NQ = MIX_NPAIR + MIX_MAXH;    // Gram entries + right-hand side
constexpr int MIX_BLOCKS = 304;

struct MixPtrs {
  const double* dX[MIX_MAXH];
  const double* dF[MIX_MAXH];
  int m;
};

// f = x_out - x_in; with a previous step, dX[slot] = x_in - x_prev and
// dF[slot] = f - f_prev; then x_prev = x_in, f_prev = f.  Point-wise, each
// point read before it is written by the same thread (no __restrict__:
// callers may pass aliased inputs).
__global__ void mix_prepare_kernel(const double* x_in, const double* x_out, double* xp,
                                   double* fp, double* dX, double* dF, long long N) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    const double xi = x_in[i];
    const double f = x_out[i] - xi;
    if (dX) {
      dX[i] = xi - xp[i];
      dF[i] = f - fp[i];
    }
    xp[i] = xi;
    fp[i] = f;
  }
}

// Per-block partial sums of dF_a . dF_b (a <= b) and dF_a . f.
__global__ void __launch_bounds__(256)
mix_dots_kernel(MixPtrs mp, const double* __restrict__ f, long long N,
                double* __restrict__ part) {
  double acc[MIX_NQ];
#pragma unroll
  for (int q = 0; q < MIX_NQ; ++q) acc[q] = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    double v[MIX_MAXH];
#pragma unroll
    for (int a = 0; a < MIX_MAXH; ++a) v[a] = a < mp.m ? mp.dF[a][i] : 0.0;
    const double fi = f[i];
    int q = 0;
#pragma unroll
    for (int a = 0; a < MIX_MAXH; ++a)
#pragma unroll
      for (int b = a; b < MIX_MAXH; ++b) {
        acc[q] = fma(v[a], v[b], acc[q]);
        ++q;
      }
#pragma unroll
    for (int a = 0; a < MIX_MAXH; ++a) acc[MIX_NPAIR + a] = fma(v[a], fi, acc[MIX_NPAIR + a]);
  }
  __shared__ double sh[8][MIX_NQ];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < MIX_NQ; ++q) {
    double x = acc[q];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) sh[warp][q] = x;
  }
  __syncthreads();
  if (threadIdx.x < MIX_NQ) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += sh[w][threadIdx.x];
    part[(size_t)blockIdx.x * MIX_NQ + threadIdx.x] = s;
  }
}

// Sums the partials in block order, then one thread solves the m x m
// normal equations; c[a] = 0 for a dropped column.
__global__ void mix_solve_kernel(const double* __restrict__ part, int m,
                                 double* __restrict__ c) {
  __shared__ double tot[MIX_NQ];
  const int t = threadIdx.x;
  if (t < MIX_NQ) {
    double s = 0.0;
    for (int k = 0; k < MIX_BLOCKS; ++k) s += part[(size_t)k * MIX_NQ + t];
    tot[t] = s;
  }
  __syncthreads();
  if (t != 0) return;
  double G[MIX_MAXH][MIX_MAXH], r[MIX_MAXH], L[MIX_MAXH][MIX_MAXH], y[MIX_MAXH];
  bool keep[MIX_MAXH];
  int q = 0;
  for (int a = 0; a < MIX_MAXH; ++a)
    for (int b = a; b < MIX_MAXH; ++b, ++q) G[a][b] = G[b][a] = tot[q];
  for (int a = 0; a < MIX_MAXH; ++a) r[a] = tot[MIX_NPAIR + a];
  for (int j = 0; j < m; ++j) {
    double d = G[j][j];
    for (int k = 0; k < j; ++k) if (keep[k]) d -= L[j][k] * L[j][k];
    keep[j] = d > 1e-12 * G[j][j] && G[j][j] > 0.0;
    const double ljj = keep[j] ? sqrt(d) : 0.0;
    L[j][j] = ljj;
    for (int i = j + 1; i < m; ++i) {
      double v = G[i][j];
      for (int k = 0; k < j; ++k) if (keep[k]) v -= L[i][k] * L[j][k];
      L[i][j] = keep[j] ? v / ljj : 0.0;
    }
  }
  for (int i = 0; i < m; ++i) {
    double v = r[i];
    for (int k = 0; k < i; ++k) if (keep[k]) v -= L[i][k] * y[k];
    y[i] = keep[i] ? v / L[i][i] : 0.0;
  }
  for (int i = m - 1; i >= 0; --i) {
    double v = y[i];
    for (int k = i + 1; k < m; ++k) if (keep[k]) v -= L[k][i] * c[k];
    c[i] = keep[i] ? v / L[i][i] : 0.0;
  }
}

// x_bar = x_in - sum_a c_a dX_a, f_bar = f - sum_a c_a dF_a (c == null: the
// linear step, x_bar = x_in, f_bar = f).  Without a preconditioner the next
// input x_bar + beta f_bar is written; with one, x_bar goes to x_next and
// f_bar to fbar for the Kerker step.
__global__ void mix_combine_kernel(MixPtrs mp, const double* c, const double* x_in,
                                   const double* f, double* x_next, double* fbar,
                                   double beta, long long N) {
  double cc[MIX_MAXH];
#pragma unroll
  for (int a = 0; a < MIX_MAXH; ++a) cc[a] = (c && a < mp.m) ? c[a] : 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    double xb = x_in[i], fb = f[i];
#pragma unroll
    for (int a = 0; a < MIX_MAXH; ++a)
      if (a < mp.m && c) {
        xb = fma(-cc[a], mp.dX[a][i], xb);
        fb = fma(-cc[a], mp.dF[a][i], fb);
      }
    if (fbar) {
      x_next[i] = xb;
      fbar[i] = fb;
    } else {
      x_next[i] = fma(beta, fb, xb);
    }
  }
}

__global__ void axpy_kernel(double* y, const double* __restrict__ x, double a, long long N) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = fma(a, x[i], y[i]);
}

// Mixer buffers: x_prev | f_prev | f_bar | dX ring (h) | dF ring (h) |
// partials | c.
int mixer_buffers(sq3_ctx* ctx) {
  const size_t N = (size_t)ctx->grid.N;
  const size_t words = (3 + 2 * (size_t)ctx->mix.h) * N + (size_t)MIX_BLOCKS * MIX_NQ + MIX_MAXH;
  return ensure((void**)&ctx->wsMix, &ctx->wsMix_bytes, words * sizeof(double));
}

int mixer_step(sq3_ctx* ctx, const double* x_in, const double* x_out, double* x_next) {
  auto& M = ctx->mix;
  const long long N = ctx->grid.N;
  double* xp = ctx->wsMix;
  double* fp = xp + N;
  double* fbar = fp + N;
  double* dXr = fbar + N;
  double* dFr = dXr + (size_t)M.h * N;
  double* part = dFr + (size_t)M.h * N;
  double* cbuf = part + (size_t)MIX_BLOCKS * MIX_NQ;
  cudaStream_t st = ctx->stream;
  const unsigned blocks = (unsigned)std::min<long long>((N + 255) / 256, 152LL * 8);
  const bool precond = M.k0 > 0.0;
  double *A = nullptr, *B = nullptr;
  if (precond) {
    // workspace first (sq3_mixer_setup already holds it): a failure here
    // leaves the mixer's state untouched
    int rc = ensure_tables(ctx);
    if (rc) return rc;
    double *p2, *res;
    rc = scf_scratch(ctx, &A, &B, &p2, &res);
    if (rc) return rc;
  }
  // ring slot of the new difference (the oldest is overwritten when full)
  int slot = -1;
  if (M.have_prev) {
    if (M.m < M.h) slot = (M.head + M.m) % M.h;
    else slot = M.head;
  }
  mix_prepare_kernel<<<blocks, 256, 0, st>>>(
      x_in, x_out, xp, fp, slot >= 0 ? dXr + (size_t)slot * N : nullptr,
      slot >= 0 ? dFr + (size_t)slot * N : nullptr, N);
  if (slot >= 0) {
    if (M.m < M.h) ++M.m;
    else M.head = (M.head + 1) % M.h;
  }
  M.have_prev = true;
  ++M.k;
  MixPtrs mp{};
  mp.m = M.m;
  for (int a = 0; a < M.m; ++a) {
    const int ph = (M.head + a) % M.h;   // logical order: oldest first
    mp.dX[a] = dXr + (size_t)ph * N;
    mp.dF[a] = dFr + (size_t)ph * N;
  }
  const bool pulay = M.m > 0 && M.k % M.period == 0;
  if (pulay) {
    mix_dots_kernel<<<MIX_BLOCKS, 256, 0, st>>>(mp, fp, N, part);
    mix_solve_kernel<<<1, 64, 0, st>>>(part, M.m, cbuf);
  } else {
    mp.m = 0;
  }
  mix_combine_kernel<<<blocks, 256, 0, st>>>(mp, pulay ? cbuf : nullptr, x_in, fp, x_next,
                                             precond ? fbar : nullptr, M.beta, N);
  if (precond) {
    spectral_apply(ctx, fbar, nullptr, fbar, SCALE_KERKER, M.k0 * M.k0, A, B);
    axpy_kernel<<<blocks, 256, 0, st>>>(x_next, fbar, M.beta, N);
  }
  return cuda_err(cudaGetLastError());
}

}  // namespace

}  // namespace sq3

using namespace sq3;

extern "C" {

int sq3_poisson(sq3_ctx* c, const double* rho, const double* b, double* phi) {
  int rc = check_grid(c);
  if (rc) return rc;
  if (!rho || !phi) return SQ3_EINVAL;
  cudaSetDevice(c->device);
  rc = ensure_tables(c);
  if (rc) return rc;
  double *A, *B, *part, *res;
  rc = scf_scratch(c, &A, &B, &part, &res);
  if (rc) return rc;
  spectral_apply(c, rho, b, phi, SCALE_POISSON, 0.0, A, B);
  rc = cuda_err(cudaGetLastError());
  if (rc) return rc;
  rc = cuda_err(cudaStreamSynchronize(c->stream));
  if (rc) return rc;
  return check_device_status(c);
}

int sq3_mixer_setup(sq3_ctx* c, int history, int period, double beta, double k0) {
  int rc = check_grid(c);
  if (rc) return rc;
  if (history < 1 || history > MIX_MAXH || period < 1 || !(beta > 0) || !isfinite(beta) ||
      !isfinite(k0))
    return SQ3_EINVAL;
  cudaSetDevice(c->device);
  c->mix = sq3_ctx::MixState{};
  c->mix.h = history;
  c->mix.period = period;
  c->mix.beta = beta;
  c->mix.k0 = k0 > 0 ? k0 : 0.0;
  rc = mixer_buffers(c);
  if (rc) return rc;
  if (c->mix.k0 > 0.0) {          // the Kerker step's tables and scratch
    rc = ensure_tables(c);
    if (rc) return rc;
    double *A, *B, *part, *res;
    rc = scf_scratch(c, &A, &B, &part, &res);
    if (rc) return rc;
  }
  c->mix.ready = true;
  return SQ3_OK;
}

int sq3_mixer_step(sq3_ctx* c, const double* x_in, const double* x_out, double* x_next) {
  int rc = check_grid(c);
  if (rc) return rc;
  if (!c->mix.ready) return SQ3_ENOTSETUP;
  if (!x_in || !x_out || !x_next) return SQ3_EINVAL;
  cudaSetDevice(c->device);
  rc = mixer_step(c, x_in, x_out, x_next);
  if (rc) return rc;
  rc = cuda_err(cudaStreamSynchronize(c->stream));
  if (rc) return rc;
  return check_device_status(c);
}

int sq3_kerker(sq3_ctx* c, const double* r, double* out, double k0) {
  int rc = check_grid(c);
  if (rc) return rc;
  if (!r || !out || !(k0 > 0) || !isfinite(k0)) return SQ3_EINVAL;
  cudaSetDevice(c->device);
  rc = ensure_tables(c);
  if (rc) return rc;
  double *A, *B, *part, *res;
  rc = scf_scratch(c, &A, &B, &part, &res);
  if (rc) return rc;
  spectral_apply(c, r, nullptr, out, SCALE_KERKER, k0 * k0, A, B);
  rc = cuda_err(cudaGetLastError());
  if (rc) return rc;
  rc = cuda_err(cudaStreamSynchronize(c->stream));
  if (rc) return rc;
  return check_device_status(c);
}

int sq3_effective_potential(sq3_ctx* c, const double* rho, const double* b, double* veff,
                            double* phi, double* terms) {
  int rc = check_grid(c);
  if (rc) return rc;
  if (!rho || !veff) return SQ3_EINVAL;
  if (phi && (phi == rho || phi == b || phi == veff)) return SQ3_EINVAL;
  double t[3];
  rc = potential_and_terms(c, rho, b, phi, veff, t);
  if (rc) return rc;
  if (terms)
    for (int k = 0; k < 3; ++k) terms[k] = t[k];
  return SQ3_OK;
}

int sq3_free_energy(sq3_ctx* c, const double* rho, const double* b, double e_band,
                    double e_ent, double e_self, double* out) {
  int rc = check_grid(c);
  if (rc) return rc;
  if (!rho || !b || !out) return SQ3_EINVAL;
  double t[3];
  rc = potential_and_terms(c, rho, b, nullptr, nullptr, t);
  if (rc) return rc;
  out[0] = e_band + t[0] - t[1] + t[2] - e_self + e_ent;
  out[1] = t[0];
  out[2] = t[1];
  out[3] = t[2];
  return SQ3_OK;
}

}  // extern "C"
