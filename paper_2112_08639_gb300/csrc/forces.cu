// Hellmann-Feynman forces on the nuclei, Eq. (force:NewForm) (Sec. 3;
// Eq. (ON:forces) in Sec. 2):
//
//   f_I = sum_{I'} int grad b_{I'} phi dx + f_sc
//         - 4 sum_i sum_p gamma_p (int phi_i chi_p)(int grad phi~_i chi_p),
//
// I' running over atom I and its periodic images, phi the electrostatic
// potential of rho + b, phi~_i = sum_j phi_j (Ds)_ji, p over the projectors
// of atom I.  With Gaussian pseudocharges E_self is a constant and E_c = 0,
// so f_sc = 0.
//
// Local term.  b_I = s q exp(-|x - R_I|^2 / rc^2) / (pi^{3/2} rc^3) summed
// over images factorises by axis, so grad_x b_I(i, j, l) = s q norm
// dgx(i) gy(j) gz(l) with the 1-D image sums g and their derivatives dg
// (s: the rescaling that makes sum b dV = -Ne).  One CTA per atom reduces
// sum_k grad b_I(k) phi(k) dV over the grid.
//
// Nonlocal term.  On the grid (Euclidean vectors u_i, c_p = chi_p sqrt(dV))
// it is -4 sum gamma_p (c_p . u_i)(c_p . grad_h u~_i) with grad_h the
// central FD first derivative of the Laplacian's order.  grad_h is
// antisymmetric on the periodic grid (sum f grad_h g = -sum (grad_h f) g),
// so c_p . grad_h u~_i = -(grad_h c_p) . u~_i and, with u~ = U Ds,
//   f_I,a = 4 sum_p gamma_p P_p^T Ds Q_pa,
//   P_p = U^T c_p,  Q_pa = U^T grad_{h,a} c_p,
// which needs the FD gradient of the sparse projectors only, not of the
// N x Ns block.  The projectors of a ball (one atom) and their gradients
// are tabulated per grid point of the ball dilated by the stencil radius
// (16 values: 4 projectors x {c, d/dx, d/dy, d/dz}); one kernel forms
// P and Q for every ball and vector (a 16 x 64 tile of T^T U per CTA,
// the table and the gathered rows of U staged in shared memory), an FP64
// GEMM forms R = Ds Q, and a last kernel the dot products gamma P . R.
#include <math.h>

#include <algorithm>
#include <vector>

#include "sq3_internal.cuh"

namespace sq3 {
namespace {

constexpr double PI = 3.14159265358979323846;
constexpr int FQ_VALS = 16;   // 4 projectors x {c, grad_x c, grad_y c, grad_z c}
constexpr int FQ_PTS = 64;    // points per staged chunk
constexpr int FQ_VEC = 64;    // vectors per CTA

// One CTA per atom: out[3 I + a] = scale * sum_k dG_a(k) phi(k), with
// dG_x = dgx gy gz, dG_y = gx dgy gz, dG_z = gx gy dgz.
__global__ void __launch_bounds__(256) local_force_kernel(int nx, int ny, int nz, int natoms,
                                                          const double* __restrict__ g,
                                                          const double* __restrict__ dg,
                                                          const double* __restrict__ phi,
                                                          double scale, double* out) {
  __shared__ double sh[3][8];
  const int I = blockIdx.x;
  const double* gx = g + (size_t)I * nx;
  const double* gy = g + (size_t)natoms * nx + (size_t)I * ny;
  const double* gz = g + (size_t)natoms * (nx + ny) + (size_t)I * nz;
  const double* dx = dg + (size_t)I * nx;
  const double* dy = dg + (size_t)natoms * nx + (size_t)I * ny;
  const double* dz = dg + (size_t)natoms * (nx + ny) + (size_t)I * nz;
  const long long N = (long long)nx * ny * nz;
  double fx = 0.0, fy = 0.0, fz = 0.0;
  for (long long k = threadIdx.x; k < N; k += blockDim.x) {
    const int i = (int)(k % nx), j = (int)((k / nx) % ny), l = (int)(k / ((long long)nx * ny));
    const double p = phi[k];
    const double a = gy[j] * gz[l], b = gx[i] * gz[l], c = gx[i] * gy[j];
    fx += dx[i] * a * p;
    fy += dy[j] * b * p;
    fz += dz[l] * c * p;
  }
  for (int o = 16; o > 0; o >>= 1) {
    fx += __shfl_xor_sync(0xffffffffu, fx, o);
    fy += __shfl_xor_sync(0xffffffffu, fy, o);
    fz += __shfl_xor_sync(0xffffffffu, fz, o);
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) { sh[0][w] = fx; sh[1][w] = fy; sh[2][w] = fz; }
  __syncthreads();
  if (threadIdx.x < 3) {
    double t = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += sh[threadIdx.x][q];
    out[3 * I + threadIdx.x] = scale * t;
  }
}

// PQ[(ball slot 16 B + m) * Ns + v] = sum_rows T[row][m] U[idx[row]][v] for
// the ball's rows; grid (balls, ceil(Ns / 64)); 256 threads, each four
// (m, v) outputs of the 16 x 64 tile.
template <typename T>
__global__ void __launch_bounds__(256) ball_project_kernel(const int* __restrict__ rptr,
                                                           const int* __restrict__ ridx,
                                                           const T* __restrict__ rval,
                                                           const T* __restrict__ U, long long N,
                                                           int Ns, double* PQ) {
  __shared__ T tv[FQ_PTS][FQ_VALS];
  __shared__ T tu[FQ_PTS][FQ_VEC + 1];
  const int B = blockIdx.x;
  const int v0 = blockIdx.y * FQ_VEC;
  const int r0 = rptr[B], r1 = rptr[B + 1];
  const int tid = threadIdx.x;
  // outputs of this thread: m = tid / 16, vectors (tid % 16) + 16 c, c < 4
  const int m = tid >> 4, vq = tid & 15;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int c0 = r0; c0 < r1; c0 += FQ_PTS) {
    const int nr = min(FQ_PTS, r1 - c0);
    for (int e = tid; e < FQ_PTS * FQ_VALS; e += blockDim.x) {
      const int r = e / FQ_VALS, q = e % FQ_VALS;
      tv[r][q] = r < nr ? rval[(size_t)(c0 + r) * FQ_VALS + q] : T(0);
    }
    // U rows at the chunk's points: lanes along the points (consecutive
    // grid indices along x), warps along the vectors
    for (int e = tid; e < FQ_PTS * FQ_VEC; e += blockDim.x) {
      const int r = e % FQ_PTS, v = e / FQ_PTS;
      T val = T(0);
      if (r < nr && v0 + v < Ns) val = U[(size_t)(v0 + v) * N + ridx[c0 + r]];
      tu[r][v] = val;
    }
    __syncthreads();
    for (int r = 0; r < nr; ++r) {
      const double t = (double)tv[r][m];
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[c] += t * (double)tu[r][vq + 16 * c];
    }
    __syncthreads();
  }
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int v = v0 + vq + 16 * c;
    if (v < Ns) PQ[((size_t)B * FQ_VALS + m) * Ns + v] = acc[c];
  }
}

// R[(slot * 16 + m) * Ns + i] = sum_j Ds[i][j] PQ[(slot * 16 + m) * Ns + j]
// for the gradient columns m >= 4 (Ds symmetric); one CTA per (ball slot,
// m), a thread per i, Ds read by rows (column i of the symmetric Ds is row i).
__global__ void __launch_bounds__(256) ds_apply_kernel(const double* __restrict__ Ds, int Ns,
                                                       const double* __restrict__ PQ, double* R) {
  extern __shared__ double q[];
  const int slot = blockIdx.x, m = 4 + blockIdx.y;
  const double* src = PQ + ((size_t)slot * FQ_VALS + m) * Ns;
  for (int j = threadIdx.x; j < Ns; j += blockDim.x) q[j] = src[j];
  __syncthreads();
  for (int i = blockIdx.z * blockDim.x + threadIdx.x; i < Ns; i += gridDim.z * blockDim.x) {
    const double* row = Ds + (size_t)i;         // column-major: Ds[i + j Ns]
    double s = 0.0;
    for (int j = 0; j < Ns; ++j) s += row[(size_t)j * Ns] * q[j];
    R[((size_t)slot * FQ_VALS + m) * Ns + i] = s;
  }
}

// out[slot * 12 + 3 q + a] = sum_i P[slot][q][i] R[slot][4 + 4 a + q][i]:
// one warp per (slot, q, a).
__global__ void nl_dot_kernel(const double* __restrict__ PQ, const double* __restrict__ R,
                              int Ns, int nslots, double* out) {
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (w >= nslots * 12) return;
  const int slot = w / 12, q = (w % 12) / 3, a = w % 3;
  const double* p = PQ + ((size_t)slot * FQ_VALS + q) * Ns;
  const double* r = R + ((size_t)slot * FQ_VALS + 4 + 4 * a + q) * Ns;
  double s = 0.0;
  for (int i = lane; i < Ns; i += 32) s += p[i] * r[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) out[w] = s;
}

// Central FD first-derivative weights of order 2n (Fornberg's closed form):
// f' ~ sum_p a_p (f(x + p h) - f(x - p h)) / h,
// a_p = (-1)^(p+1) (n!)^2 / (p (n - p)! (n + p)!).
void fd_first_weights(int n, double* a) {
  auto fact = [](int k) { double f = 1; for (int i = 2; i <= k; ++i) f *= i; return f; };
  for (int p = 1; p <= n; ++p)
    a[p] = ((p % 2) ? 1.0 : -1.0) * fact(n) * fact(n) / (p * fact(n - p) * fact(n + p));
}

// Build the per-ball tables of c and grad_h c on the host and upload them.
int build_force_tables(sq3_ctx* c) {
  Projectors& P = c->proj;
  if (P.fq_ok) return SQ3_OK;
  const Grid& g = c->grid;
  const int R = g.radius;
  double a[SQ3_MAX_FD_RADIUS + 1] = {0};
  fd_first_weights(R, a);
  const double ih[3] = {1.0 / g.hx, 1.0 / g.hy, 1.0 / g.hz};
  const long long N = g.N;
  const int nb = P.n_ball;
  std::vector<int> slot(N, -1), touched, rptr{0}, ridx;
  std::vector<double> rval;
  int maxrows = 0;
  for (int B = 0; B < nb; ++B) {
    const int len = P.h_bptr[B + 1] - P.h_bptr[B];
    const size_t base = rval.size() / FQ_VALS;
    touched.clear();
    auto row_of = [&](long long k) -> double* {
      int& s = slot[k];
      if (s < 0) {
        s = (int)touched.size();
        touched.push_back((int)k);
        rval.resize(rval.size() + FQ_VALS, 0.0);
      }
      return &rval[(base + s) * FQ_VALS];
    };
    for (int e = 0; e < len; ++e) {
      const long long k = P.h_bidx[P.h_bptr[B] + e];
      const int i = (int)(k % g.nx), j = (int)((k / g.nx) % g.ny),
                l = (int)(k / ((long long)g.nx * g.ny));
      double v[4] = {0, 0, 0, 0};
      for (int q = 0; q < P.h_bnp[B]; ++q) v[q] = P.h_bval[(size_t)P.h_boff[B] + (size_t)q * len + e];
      double* r0 = row_of(k);
      for (int q = 0; q < 4; ++q) r0[q] += v[q];
      // c(k) contributes +a_s v / h at k - s e_a and -a_s v / h at k + s e_a
      for (int ax = 0; ax < 3; ++ax) {
        const int n = ax == 0 ? g.nx : (ax == 1 ? g.ny : g.nz);
        const int pos = ax == 0 ? i : (ax == 1 ? j : l);
        const long long stride = ax == 0 ? 1 : (ax == 1 ? g.nx : (long long)g.nx * g.ny);
        for (int s = 1; s <= R; ++s) {
          const double w = a[s] * ih[ax];
          const long long km = k + (long long)(((pos - s) % n + n) % n - pos) * stride;
          const long long kp = k + (long long)(((pos + s) % n) - pos) * stride;
          double* rm = row_of(km);
          for (int q = 0; q < 4; ++q) rm[4 + 4 * ax + q] += w * v[q];
          double* rp = row_of(kp);
          for (int q = 0; q < 4; ++q) rp[4 + 4 * ax + q] -= w * v[q];
        }
      }
    }
    // rows of this ball in grid order (coalesced gathers), then reset slots
    std::vector<int> order(touched.size());
    for (size_t t = 0; t < order.size(); ++t) order[t] = (int)t;
    std::sort(order.begin(), order.end(), [&](int x, int y) { return touched[x] < touched[y]; });
    std::vector<double> sorted(order.size() * FQ_VALS);
    for (size_t t = 0; t < order.size(); ++t) {
      ridx.push_back(touched[order[t]]);
      for (int q = 0; q < FQ_VALS; ++q)
        sorted[t * FQ_VALS + q] = rval[(base + order[t]) * FQ_VALS + q];
    }
    std::copy(sorted.begin(), sorted.end(), rval.begin() + base * FQ_VALS);
    for (int k : touched) slot[k] = -1;
    rptr.push_back((int)ridx.size());
    maxrows = std::max(maxrows, (int)touched.size());
  }
  std::vector<float> rvalf(rval.begin(), rval.end());
  auto up = [&](void** dst, const void* src, size_t bytes) -> int {
    if (cudaMalloc(dst, bytes) != cudaSuccess) {
      cudaGetLastError();
      *dst = nullptr;
      return SQ3_ENOMEM;
    }
    return cuda_err(cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice));
  };
  int rc = SQ3_OK;
  rc = rc ? rc : up((void**)&P.fq_ptr, rptr.data(), rptr.size() * sizeof(int));
  rc = rc ? rc : up((void**)&P.fq_idx, ridx.data(), ridx.size() * sizeof(int));
  rc = rc ? rc : up((void**)&P.fq_val, rval.data(), rval.size() * sizeof(double));
  rc = rc ? rc : up((void**)&P.fq_valf, rvalf.data(), rvalf.size() * sizeof(float));
  if (rc) return rc;
  P.fq_max_rows = maxrows;
  P.fq_ok = true;
  return SQ3_OK;
}

}  // namespace
}  // namespace sq3

using namespace sq3;

extern "C" int sq3_forces(sq3_ctx* c, int natoms, const double* pos, double Z, double rc,
                          double Ne, const double* phi, const void* X, const double* D, int Ns,
                          sq3_prec prec, const int* atom_of, double* forces, double* parts) {
  if (!c) return SQ3_EINVAL;
  if (!c->grid_ok) return SQ3_ENOTSETUP;
  if (natoms < 1 || !pos || !phi || !forces || !(rc > 0) || !isfinite(Z) || !(Ne > 0))
    return SQ3_EINVAL;
  if (prec != SQ3_FP64 && prec != SQ3_MIXED) return SQ3_EINVAL;
  const int np = c->proj.n_proj;
  if (np > 0 && (!X || !D || !atom_of || Ns < 1 || Ns > 65535)) return SQ3_EINVAL;
  for (int p = 0; p < np; ++p)
    if (atom_of[p] < 0 || atom_of[p] >= natoms) return SQ3_EINVAL;
  for (int k = 0; k < 3 * natoms; ++k)
    if (!isfinite(pos[k])) return SQ3_EINVAL;
  cudaSetDevice(c->device);
  const Grid& g = c->grid;
  cudaStream_t st = c->stream;
  // local term: image-sum tables of the Gaussians and their derivatives
  std::vector<double> gt, dgt;
  atom_tables(c, natoms, pos, rc, false, gt);
  atom_tables(c, natoms, pos, rc, true, dgt);
  // the rescaling of b: sum b dV = -Ne, the unscaled sum being separable
  const double norm = -Z / (pow(PI, 1.5) * rc * rc * rc);
  double total = 0.0;
  for (int J = 0; J < natoms; ++J) {
    double sx = 0, sy = 0, sz = 0;
    for (int i = 0; i < g.nx; ++i) sx += gt[(size_t)J * g.nx + i];
    for (int j = 0; j < g.ny; ++j) sy += gt[(size_t)natoms * g.nx + (size_t)J * g.ny + j];
    for (int l = 0; l < g.nz; ++l) sz += gt[(size_t)natoms * (g.nx + g.ny) + (size_t)J * g.nz + l];
    total += sx * sy * sz;
  }
  total *= norm * c->dV;
  const double scale = (-Ne / total) * norm * c->dV;
  const size_t tw = gt.size();
  size_t words = 2 * tw + 3 * (size_t)natoms;
  const int nslots = c->proj.n_ball;
  if (np > 0) words += 2 * (size_t)nslots * FQ_VALS * Ns + (size_t)nslots * 12;
  int rc2 = ensure((void**)&c->wsAtoms, &c->wsAtoms_bytes, words * sizeof(double));
  if (rc2) return rc2;
  double* dg_ = c->wsAtoms;
  double* ddg = dg_ + tw;
  double* floc = ddg + tw;
  double* PQ = floc + 3 * (size_t)natoms;
  double* Rm = PQ + (size_t)nslots * FQ_VALS * Ns;
  double* dots = Rm + (size_t)nslots * FQ_VALS * Ns;
  int r = cuda_err(cudaMemcpyAsync(dg_, gt.data(), tw * sizeof(double), cudaMemcpyHostToDevice, st));
  if (r == SQ3_OK)
    r = cuda_err(cudaMemcpyAsync(ddg, dgt.data(), tw * sizeof(double), cudaMemcpyHostToDevice, st));
  if (r) return r;
  local_force_kernel<<<natoms, 256, 0, st>>>(g.nx, g.ny, g.nz, natoms, dg_, ddg, phi, scale, floc);
  std::vector<double> fl(3 * (size_t)natoms), dh;
  if (np > 0) {
    r = build_force_tables(c);
    if (r) return r;
    const Projectors& P = c->proj;
    dim3 grid(nslots, (Ns + FQ_VEC - 1) / FQ_VEC);
    if (prec == SQ3_FP64)
      ball_project_kernel<double><<<grid, 256, 0, st>>>(P.fq_ptr, P.fq_idx, P.fq_val,
                                                        (const double*)X, g.N, Ns, PQ);
    else
      ball_project_kernel<float><<<grid, 256, 0, st>>>(P.fq_ptr, P.fq_idx, P.fq_valf,
                                                       (const float*)X, g.N, Ns, PQ);
    const size_t smem = (size_t)Ns * sizeof(double);
    if (smem > 227 * 1024) return SQ3_EINVAL;
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(ds_apply_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
      return cuda_err(cudaGetLastError());
    const int zb = std::max(1, std::min(8, (Ns + 255) / 256));
    ds_apply_kernel<<<dim3(nslots, 12, zb), 256, smem, st>>>(D, Ns, PQ, Rm);
    nl_dot_kernel<<<(nslots * 12 * 32 + 255) / 256, 256, 0, st>>>(PQ, Rm, Ns, nslots, dots);
    dh.resize((size_t)nslots * 12);
    r = cuda_err(cudaGetLastError());
    if (r) return r;
    r = cuda_err(cudaMemcpyAsync(dh.data(), dots, dh.size() * sizeof(double),
                                 cudaMemcpyDeviceToHost, st));
    if (r) return r;
  }
  r = cuda_err(cudaMemcpyAsync(fl.data(), floc, fl.size() * sizeof(double),
                               cudaMemcpyDeviceToHost, st));
  if (r == SQ3_OK) r = cuda_err(cudaGetLastError());
  if (r == SQ3_OK) r = cuda_err(cudaStreamSynchronize(st));
  if (r) return r;
  r = check_device_status(c);
  if (r) return r;
  std::vector<double> fnl(3 * (size_t)natoms, 0.0);
  for (int B = 0; B < nslots; ++B)
    for (int q = 0; q < c->proj.h_bnp[B]; ++q) {
      const int p = c->proj.h_bp0[B] + q;
      for (int ax = 0; ax < 3; ++ax)
        fnl[3 * (size_t)atom_of[p] + ax] += 4.0 * c->proj.h_gamma[p] * dh[(size_t)B * 12 + 3 * q + ax];
    }
  for (int k = 0; k < 3 * natoms; ++k) {
    forces[k] = fl[k] + fnl[k];
    if (parts) { parts[2 * k] = fl[k]; parts[2 * k + 1] = fnl[k]; }
    if (!isfinite(forces[k])) return SQ3_ENONFINITE;
  }
  return SQ3_OK;
}
