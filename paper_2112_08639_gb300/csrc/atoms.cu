// Atom-centred Gaussians on the periodic grid: the Gaussian pseudocharges
// b of the electrostatics (Sec. 2, Eq. (poisson): the nuclei's charge
// smeared into b, whose potential is the local pseudopotential), the
// atomic-superposition starting density, and the radial descriptors of the
// learned starting density.  All three are sums over atoms J and their
// periodic images of q_J exp(-|x - R_J|^2 / w^2) / (pi^{3/2} w^3) (or the
// same without the normalisation), which factorise by axis:
//   out(i, j, l) = sum_J q_J gx_J(i) gy_J(j) gz_J(l),
//   g_J(i) = sum_images exp(-(x_i - R_J - m L)^2 / w^2).
// The 1-D image sums are tabulated on the host (natoms x (nx + ny + nz)
// values) and the 3-D sum runs on the device, one thread per grid point.
#include <math.h>

#include <algorithm>
#include <vector>

#include "sq3_internal.cuh"

namespace sq3 {
namespace {

constexpr int AG_BLOCKS = 304;
constexpr double PI = 3.14159265358979323846;

// Image sum of exp(-(x - r0 - m L)^2 / w^2) at x = k L / n, k < n, over the
// images whose distance is below 28 w (exp(-784) underflows to 0); with
// `deriv` the x-derivative -2 (x - r0 - m L) / w^2 exp(...) instead.
void image_sum_1d(int n, double L, double r0, double w, bool deriv, double* g) {
  const double h = L / n;
  const double reach = 28.0 * w;
  const int mlo = (int)floor((-reach - r0) / L) - 1, mhi = (int)ceil((L + reach - r0) / L) + 1;
  for (int k = 0; k < n; ++k) {
    double s = 0.0;
    for (int m = mlo; m <= mhi; ++m) {
      const double d = k * h - r0 - m * L;
      if (fabs(d) > reach) continue;
      const double e = exp(-d * d / (w * w));
      s += deriv ? (-2.0 * d / (w * w)) * e : e;
    }
    g[k] = s;
  }
}

__global__ void __launch_bounds__(256) gauss_sum_kernel(int nx, int ny, int nz, int natoms,
                                                        const double* __restrict__ tab,
                                                        const double* __restrict__ q,
                                                        double norm, double* out) {
  const long long N = (long long)nx * ny * nz;
  const double* gx = tab;
  const double* gy = gx + (size_t)natoms * nx;
  const double* gz = gy + (size_t)natoms * ny;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < N;
       k += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(k % nx), j = (int)((k / nx) % ny), l = (int)(k / ((long long)nx * ny));
    double s = 0.0;
    for (int J = 0; J < natoms; ++J)
      s += q[J] * gx[(size_t)J * nx + i] * gy[(size_t)J * ny + j] * gz[(size_t)J * nz + l];
    out[k] = norm * s;
  }
}

__global__ void __launch_bounds__(256) sum_part_kernel(const double* __restrict__ a, long long n,
                                                       double* part) {
  __shared__ double sh[8];
  double s = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    s += a[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    part[blockIdx.x] = t;
  }
}

// out *= total / (sum(out) dV) with the sum from the ordered partials;
// res[0] receives sum(out) dV before the scaling.
__global__ void rescale_kernel(double* out, long long n, const double* part, int nb, double dV,
                               double total, double* res) {
  __shared__ double sc;
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int b = 0; b < nb; ++b) t += part[b];
    t *= dV;
    if (blockIdx.x == 0) res[0] = t;
    sc = (total != 0.0 && t != 0.0) ? total / t : 1.0;
  }
  __syncthreads();
  const double f = sc;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[i] *= f;
}

}  // namespace

// Host tables of the 1-D image sums (values, or derivatives when deriv) for
// every atom: gx | gy | gz, natoms x n each.
void atom_tables(const sq3_ctx* c, int natoms, const double* pos, double w, bool deriv,
                 std::vector<double>& tab) {
  const Grid& g = c->grid;
  tab.assign((size_t)natoms * (g.nx + g.ny + g.nz), 0.0);
  double* gx = tab.data();
  double* gy = gx + (size_t)natoms * g.nx;
  double* gz = gy + (size_t)natoms * g.ny;
  for (int J = 0; J < natoms; ++J) {
    image_sum_1d(g.nx, c->Lx, pos[3 * J + 0], w, deriv, gx + (size_t)J * g.nx);
    image_sum_1d(g.ny, c->Ly, pos[3 * J + 1], w, deriv, gy + (size_t)J * g.ny);
    image_sum_1d(g.nz, c->Lz, pos[3 * J + 2], w, deriv, gz + (size_t)J * g.nz);
  }
}

}  // namespace sq3

using namespace sq3;

extern "C" int sq3_atom_gaussians(sq3_ctx* c, int natoms, const double* pos, const double* q,
                                  double width, int normalised, double total, double* out,
                                  double* sum_out) {
  if (!c) return SQ3_EINVAL;
  if (!c->grid_ok) return SQ3_ENOTSETUP;
  if (natoms < 1 || !pos || !out || !(width > 0) || !isfinite(width) || !isfinite(total))
    return SQ3_EINVAL;
  for (int k = 0; k < 3 * natoms; ++k)
    if (!isfinite(pos[k])) return SQ3_EINVAL;
  cudaSetDevice(c->device);
  std::vector<double> tab;
  atom_tables(c, natoms, pos, width, false, tab);
  std::vector<double> qh(natoms, 1.0);
  if (q)
    for (int J = 0; J < natoms; ++J) {
      if (!isfinite(q[J])) return SQ3_EINVAL;
      qh[J] = q[J];
    }
  const size_t words = tab.size() + natoms + AG_BLOCKS + 2;
  int rc = ensure((void**)&c->wsAtoms, &c->wsAtoms_bytes, words * sizeof(double));
  if (rc) return rc;
  double* dtab = c->wsAtoms;
  double* dq = dtab + tab.size();
  double* part = dq + natoms;
  double* res = part + AG_BLOCKS;
  rc = cuda_err(cudaMemcpyAsync(dtab, tab.data(), tab.size() * sizeof(double),
                                cudaMemcpyHostToDevice, c->stream));
  if (rc == SQ3_OK)
    rc = cuda_err(cudaMemcpyAsync(dq, qh.data(), natoms * sizeof(double), cudaMemcpyHostToDevice,
                                  c->stream));
  if (rc) return rc;
  const Grid& g = c->grid;
  const double norm = normalised ? 1.0 / (pow(PI, 1.5) * width * width * width) : 1.0;
  const long long N = g.N;
  const unsigned blocks = (unsigned)std::min<long long>((N + 255) / 256, 152LL * 16);
  gauss_sum_kernel<<<blocks, 256, 0, c->stream>>>(g.nx, g.ny, g.nz, natoms, dtab, dq, norm, out);
  sum_part_kernel<<<AG_BLOCKS, 256, 0, c->stream>>>(out, N, part);
  rescale_kernel<<<blocks, 256, 0, c->stream>>>(out, N, part, AG_BLOCKS, c->dV, total, res);
  rc = cuda_err(cudaGetLastError());
  if (rc) return rc;
  rc = cuda_err(cudaMemcpyAsync(c->host_scal + 60, res, sizeof(double), cudaMemcpyDeviceToHost,
                                c->stream));
  if (rc) return rc;
  check_finite(out, N, c->dev_status, c->stream);
  rc = check_device_status(c);
  if (rc) return rc;
  if (sum_out) *sum_out = c->host_scal[60];
  return SQ3_OK;
}

// Velocity-Verlet halves on host arrays (the QMD of Sec. 5 moves the nuclei
// on the forces of Eq. (force:NewForm)); see sq3.h.
extern "C" int sq3_verlet(int natoms, const double* masses, double dt, double* R, double* V,
                          const double* F, int phase, double ke_target) {
  if (natoms < 1 || !masses || !V || !F || !(dt > 0) || !isfinite(dt) || (phase != 0 && phase != 1) ||
      (phase == 0 && !R) || !isfinite(ke_target))
    return SQ3_EINVAL;
  for (int I = 0; I < natoms; ++I)
    if (!(masses[I] > 0)) return SQ3_EINVAL;
  for (int I = 0; I < natoms; ++I)
    for (int a = 0; a < 3; ++a) {
      V[3 * I + a] += 0.5 * dt * F[3 * I + a] / masses[I];
      if (phase == 0) R[3 * I + a] += dt * V[3 * I + a];
    }
  if (phase == 1 && ke_target > 0) {
    double ke = 0.0;
    for (int I = 0; I < natoms; ++I)
      for (int a = 0; a < 3; ++a) ke += 0.5 * masses[I] * V[3 * I + a] * V[3 * I + a];
    if (ke > 0) {
      const double f = sqrt(ke_target / ke);
      for (int k = 0; k < 3 * natoms; ++k) V[k] *= f;
    }
  }
  return SQ3_OK;
}

namespace sq3 {
namespace {
// out = max(prev + a - b, 0), per-block sums of out in part
__global__ void __launch_bounds__(256) extrapolate_kernel(const double* __restrict__ prev,
                                                         const double* __restrict__ a,
                                                         const double* __restrict__ b, long long n,
                                                         double* out, double* part) {
  __shared__ double sh[8];
  double s = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double v = fmax(prev[i] + a[i] - b[i], 0.0);
    out[i] = v;
    s += v;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += sh[w];
    part[blockIdx.x] = t;
  }
}
}  // namespace
}  // namespace sq3

extern "C" int sq3_extrapolate_density(sq3_ctx* c, const double* prev, const double* a,
                                       const double* b, double Ne, double* out) {
  if (!c) return SQ3_EINVAL;
  if (!c->grid_ok) return SQ3_ENOTSETUP;
  if (!prev || !a || !b || !out || !(Ne > 0) || !isfinite(Ne)) return SQ3_EINVAL;
  cudaSetDevice(c->device);
  const size_t words = AG_BLOCKS + 2;
  int rc = ensure((void**)&c->wsAtoms, &c->wsAtoms_bytes, words * sizeof(double));
  if (rc) return rc;
  double* part = c->wsAtoms;
  double* res = part + AG_BLOCKS;
  const long long N = c->grid.N;
  const unsigned blocks = (unsigned)std::min<long long>((N + 255) / 256, 152LL * 16);
  extrapolate_kernel<<<AG_BLOCKS, 256, 0, c->stream>>>(prev, a, b, N, out, part);
  rescale_kernel<<<blocks, 256, 0, c->stream>>>(out, N, part, AG_BLOCKS, c->dV, Ne, res);
  rc = cuda_err(cudaGetLastError());
  if (rc) return rc;
  check_finite(out, N, c->dev_status, c->stream);
  return check_device_status(c);
}
