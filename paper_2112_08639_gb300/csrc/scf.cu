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
