// Native self-consistent-field driver: the SCF loop of Sec. 2 with the
// fixed-potential SQ3 iteration of Sec. 4 inside each SCF iteration and the
// density mixing Sec. 5 cites, run by the library from one call.
//
// Per SCF iteration (the paper's algorithm order):
//   V_eff = phi[rho_in + b] + V_xc[rho_in]         sq3_effective_potential
//   spectral bounds of H (closed form, below)      filter's upper bound b_up
//   passes x { X <- p_m(H) X ; Cholesky QR }       sq3_cheb_filter, sq3_orthonormalise
//   Hs = X^T H X ; Lanczos bounds (chi, xi)        sq3_project, lanczos_bounds_f64
//   Ds, mu, E_band, E_ent                          sq3_kernel_from_hs
//   rho_out = 2 rowdot(X, X Ds) / dV               sq3_density
//   err = sum |rho_out - rho_in| dV / Ne           (device reduction)
//   F of rho_out                                   sq3_free_energy
//   rho_in <- Pulay/Kerker mix(rho_in, rho_out)    sq3_mixer_step
// until err < tol.  The filter's damped interval for the next iteration is
// [lambda_max(Hs), b_up] with a0 = lambda_min(Hs) (the Ritz bounds of the
// Lanczos step; Zhou et al.'s choice, which the paper's CheFSI follows).
//
// Upper bound of the spectrum of H = -1/2 L_h + V + V_nl (rigorous, no
// iteration): the FD kinetic operator's largest eigenvalue is
// 1/2 sum_axes max_f s(2 pi f / n) / h^2 over the grid's own frequencies
// (s the FD symbol), V contributes max V, and V_nl its Gershgorin bound
// (computed by sq3_set_projectors); the lower bound likewise with 0,
// min V and the lower Gershgorin bound.
#include <math.h>

#include <chrono>
#include <vector>

#include "sq3_internal.cuh"

namespace sq3 {
namespace {

constexpr int L1_BLOCKS = 304;

// Per-block sums of |a - b| into part (fixed order: reproducible).
__global__ void __launch_bounds__(256) l1_diff_kernel(const double* __restrict__ a,
                                                      const double* __restrict__ b, long long n,
                                                      double* part) {
  __shared__ double sh[8];
  double s = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    s += fabs(a[i] - b[i]);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    part[blockIdx.x] = t;
  }
}

__global__ void l1_finish_kernel(const double* part, int nb, double scale, double* out) {
  if (threadIdx.x != 0) return;
  double t = 0.0;
  for (int k = 0; k < nb; ++k) t += part[k];
  out[0] = t * scale;
}

// Largest eigenvalue of the 1-D periodic FD second-derivative operator
// (sign flipped, h = 1) over the n grid frequencies: max_f s(2 pi f / n).
double fd_symbol_max(const Grid& g, int n) {
  double best = 0.0;
  for (int f = 0; f <= n / 2; ++f) {
    double s = -g.w[0];
    for (int p = 1; p <= g.radius; ++p)
      s -= 2.0 * g.w[p] * cos(2.0 * 3.14159265358979323846 * (double)((long long)p * f % n) / n);
    if (s > best) best = s;
  }
  return best;
}

}  // namespace

// Bounds [lo, hi] of the spectrum of the context's H (grid, potential and
// projectors set).
void hamiltonian_bounds(const sq3_ctx* c, double* lo, double* hi) {
  const Grid& g = c->grid;
  const double tmax = 0.5 * (fd_symbol_max(g, g.nx) / (g.hx * g.hx) +
                             fd_symbol_max(g, g.ny) / (g.hy * g.hy) +
                             fd_symbol_max(g, g.nz) / (g.hz * g.hz));
  *lo = c->v_min + c->proj.vnl_lo;
  *hi = tmax + c->v_max + c->proj.vnl_hi;
}

}  // namespace sq3

using namespace sq3;

extern "C" {

int sq3_hamiltonian_bounds(sq3_ctx* c, double* out) {
  if (!c || !out) return SQ3_EINVAL;
  if (!c->grid_ok || !c->pot_ok) return SQ3_ENOTSETUP;
  hamiltonian_bounds(c, &out[0], &out[1]);
  return SQ3_OK;
}

int sq3_scf_solve(sq3_ctx* c, const sq3_scf_params* p, const double* b, double* rho,
                  void* X, sq3_prec prec, double* D, sq3_scf_result* res, double* history) {
  if (!c || !p || !res) return SQ3_EINVAL;
  if (!c->grid_ok) return SQ3_ENOTSETUP;
  if (!b || !rho || !X) return SQ3_EINVAL;
  if (prec != SQ3_FP64 && prec != SQ3_MIXED) return SQ3_EINVAL;
  const int Ns = p->Ns;
  if (Ns <= 0 || Ns > 65535 || p->degree < 1 || p->max_iter < 1 || p->first_passes < 1 ||
      p->passes < 1 || !(p->kT > 0) || !(p->Ne > 0) || !(p->Ne < 2.0 * Ns) || !(p->tol > 0) ||
      p->npl > SQ3_MAX_NPL || (p->npl < 1 && !(p->fermi_tol > 0 && p->fermi_tol < 1)) ||
      !isfinite(p->e_self) || !isfinite(p->cut_shift) || p->cut_shift < 0 ||
      (p->kernel_eval != SQ3_EVAL_RECURRENCE && p->kernel_eval != SQ3_EVAL_PATERSON_STOCKMEYER))
    return SQ3_EINVAL;
  cudaSetDevice(c->device);
  // the driver alone knows that X is unchanged between its Cholesky QR, the
  // projection and the density: only inside it are the kept pieces reused
  struct ReuseGuard {
    sq3_ctx* c;
    explicit ReuseGuard(sq3_ctx* cc) : c(cc) {
      c->reuse_pieces = true;
      c->pieces_X = nullptr;
      c->hx_X = nullptr;
    }
    ~ReuseGuard() {
      c->reuse_pieces = false;
      c->pieces_X = nullptr;
      c->hx_X = nullptr;
    }
  } reuse_guard(c);
  *res = sq3_scf_result{};
  const long long N = c->grid.N;
  const size_t nn = (size_t)Ns * Ns;
  // driver workspace: rho_out, veff (N each), Hs, D when the caller passes
  // none (Ns^2 each), Lanczos work
  const int lsteps = Ns < 40 ? Ns : 40;
  const size_t lz_words = lanczos_work_words((size_t)Ns, (size_t)lsteps);
  const size_t words = 2 * (size_t)N + 2 * nn + lz_words + L1_BLOCKS + 8;
  int rc = ensure((void**)&c->wsDrv, &c->wsDrv_bytes, words * sizeof(double));
  if (rc) return rc;
  double* rho_out = c->wsDrv;
  double* veff = rho_out + N;
  double* Hs = veff + N;
  double* Dw = Hs + nn;
  double* lz = Dw + nn;
  double* part = lz + lz_words;
  double* scal = part + L1_BLOCKS;     // err, bounds (chi, xi)
  if (!D) D = Dw;
  rc = sq3_mixer_setup(c, p->mix_history, p->mix_period, p->mix_beta, p->kerker_k0);
  if (rc) return rc;

  double a = 0, a0 = 0;
  bool have_bounds = p->xi0 > 0;
  if (have_bounds) {
    a0 = p->chi0 - p->xi0;
    a = p->chi0 + p->xi0 + p->cut_shift;
  }
  double out[6] = {0}, fe[4] = {0};
  int npl_it = p->npl;
  for (int it = 0; it < p->max_iter; ++it) {
    const auto t0 = std::chrono::steady_clock::now();
    rc = sq3_effective_potential(c, rho, b, veff, nullptr, nullptr);
    if (rc) return rc;
    rc = sq3_set_potential(c, veff);
    if (rc) return rc;
    double lo, hi;
    hamiltonian_bounds(c, &lo, &hi);
    if (!have_bounds) {
      // first iteration from an arbitrary block: the damped interval starts
      // 5 % of the spectral width above the lower bound
      a0 = lo;
      a = lo + (p->filter_cut > 0 ? p->filter_cut : 0.05) * (hi - lo);
      have_bounds = true;
    }
    if (!(a < hi)) a = 0.5 * (a0 + hi);
    if (!(a0 < a)) a0 = a - 1e-3 * (hi - lo);
    const int npass = it == 0 ? p->first_passes : p->passes;
    for (int ps = 0; ps < npass; ++ps) {
      rc = sq3_cheb_filter(c, X, Ns, p->degree, a, hi, a0, prec);
      if (rc) return rc;
      rc = sq3_orthonormalise(c, X, Ns, prec);
      if (rc) return rc;
      if (ps + 1 < npass) {
        // refine the damped interval from the Ritz bounds of the new block
        rc = sq3_project(c, X, Ns, prec, Hs);
        if (rc) return rc;
        lanczos_bounds_f64(c, Hs, Ns, lsteps, scal + 1, lz, c->stream);
        rc = cuda_err(cudaMemcpyAsync(c->host_scal + 56, scal + 1, 2 * sizeof(double),
                                      cudaMemcpyDeviceToHost, c->stream));
        if (rc == SQ3_OK) rc = cuda_err(cudaStreamSynchronize(c->stream));
        if (rc) return rc;
        const double chi = c->host_scal[56], xi = c->host_scal[57];
        if (!isfinite(chi) || !isfinite(xi)) return SQ3_ENONFINITE;
        a0 = chi - xi;
        a = chi + xi + p->cut_shift;
        if (!(a < hi)) a = 0.5 * (a0 + hi);
      }
    }
    rc = sq3_project(c, X, Ns, prec, Hs);
    if (rc) return rc;
    lanczos_bounds_f64(c, Hs, Ns, lsteps, scal + 1, lz, c->stream);
    rc = cuda_err(cudaMemcpyAsync(c->host_scal + 56, scal + 1, 2 * sizeof(double),
                                  cudaMemcpyDeviceToHost, c->stream));
    if (rc == SQ3_OK) rc = cuda_err(cudaStreamSynchronize(c->stream));
    if (rc) return rc;
    const double bnd[2] = {c->host_scal[56], c->host_scal[57]};
    if (!isfinite(bnd[0]) || !(bnd[1] > 0)) return SQ3_ENONFINITE;
    rc = sq3_kernel_from_hs_ex(c, Hs, Ns, p->npl, p->fermi_tol, p->kernel_eval, p->kT, p->Ne,
                               prec, bnd, D, out, &npl_it);
    if (rc) return rc;
    rc = sq3_density(c, X, D, Ns, prec, rho_out);
    if (rc) return rc;
    l1_diff_kernel<<<L1_BLOCKS, 256, 0, c->stream>>>(rho_out, rho, N, part);
    l1_finish_kernel<<<1, 32, 0, c->stream>>>(part, L1_BLOCKS, c->dV / p->Ne, scal);
    rc = cuda_err(cudaMemcpyAsync(c->host_scal + 58, scal, sizeof(double),
                                  cudaMemcpyDeviceToHost, c->stream));
    if (rc == SQ3_OK) rc = cuda_err(cudaStreamSynchronize(c->stream));
    if (rc) return rc;
    const double err = c->host_scal[58];
    if (!isfinite(err)) return SQ3_ENONFINITE;
    rc = sq3_free_energy(c, rho_out, b, out[1], out[2], p->e_self, fe);
    if (rc) return rc;
    a0 = bnd[0] - bnd[1];
    a = bnd[0] + bnd[1] + p->cut_shift;
    res->iterations = it + 1;
    res->npl_last = npl_it;
    res->F = fe[0];
    res->e_band = out[1];
    res->e_ent = out[2];
    res->mu = out[0];
    res->e_xc = fe[1];
    res->vxc_rho = fe[2];
    res->e_es = fe[3];
    res->err = err;
    res->chi = bnd[0];
    res->xi = bnd[1];
    res->b_up = hi;
    const bool done = err < p->tol;
    if (!done) {
      rc = sq3_mixer_step(c, rho, rho_out, rho);
      if (rc) return rc;
    } else {
      rc = cuda_err(cudaMemcpyAsync(rho, rho_out, (size_t)N * sizeof(double),
                                    cudaMemcpyDeviceToDevice, c->stream));
      if (rc == SQ3_OK) rc = cuda_err(cudaStreamSynchronize(c->stream));
      if (rc) return rc;
    }
    const double ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (history) {
      double* h = history + (size_t)it * SQ3_SCF_HIST;
      h[0] = err; h[1] = out[0]; h[2] = out[1]; h[3] = out[2]; h[4] = fe[0];
      h[5] = npl_it; h[6] = ms; h[7] = bnd[0]; h[8] = bnd[1];
    }
    if (done) {
      res->converged = 1;
      return SQ3_OK;
    }
  }
  return SQ3_ENOCONV;
}

}  // extern "C"
