// Batched Chebyshev filtering of many independent cells (not in the paper:
// throughput for many uneven cells on one GPU).  Every cell has its own
// periodic grid, FP32 potential and FP32 block of Ns vectors; the whole
// filter of every cell runs in ONE persistent launch: the CTAs (a multiple
// of the SM count) take work items from a device counter, an item being one
// vector of one cell, which the CTA takes through all of the cell's filter
// steps.  Each step marches the vector's row tiles along z of the local
// Hamiltonian step
//   out = s1 (H y - c y) + s2 yprev,   H = -1/2 L_12 + V,
// with the single-cell FP32 ring stencil's tiling, rings and register
// queue; the taps are summed per axis with the twelfth-order weights as
// compile-time constants and then scaled by the cell's -1/2 / h^2, so a cell
// carries five scalars instead of 19 coefficients (equal to the single-cell
// step up to FP32 rounding).  A vector's filter needs nothing from other
// vectors, so its steps follow each other inside one CTA with no grid-wide
// synchronisation, and its two live iterates stay in L2 from step to step.
// The launch is captured once into a CUDA graph and replayed; the per-cell
// recurrence coefficients live in a device table that the host refreshes
// before each replay, so new filter bounds need no new capture.  The tile
// height and the number of resident CTAs are picked by a small autotuner
// that times each candidate on the batch itself.
//
// Work items are claimed with one atomicAdd each; nothing waits on another
// CTA, so there is no spin-wait anywhere in this file.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "async_copy.cuh"
#include "sq3_internal.cuh"

namespace sq3 {
namespace {

constexpr int BR = 6;              // stencil radius (12th order)
constexpr int BVW = 4;             // floats per thread along x
constexpr int BPAD = 8;            // wrapped columns per side (R rounded up to VW)
constexpr int BA = 4;              // planes in flight
constexpr int BTHREADS = 256;
constexpr int BKC = 3;             // precomputed window copies per thread
constexpr int BMAX_CELLS = 256;
constexpr int BMAX_STEPS = 256;

struct BCell {
  int nx, ny, nz, TY, TX, Wd, tiles;   // row tiles per vector
  int Ns, m;
  long long N;
  const float* V;
  float* buf[2];                       // [0] the cell's block X, [1] work block
  float kdiag;                         // -1/2 w_0 (1/hx^2 + 1/hy^2 + 1/hz^2)
  float hx2, hy2, hz2;                 // -1/2 / h^2 per axis
  float c;                             // filter centre
};

// Per (step, cell): recurrence scalars and which buffers take which role.
struct BStep {
  float s1, s2;
  int y, prev, out;                    // buffer ids (-1: no yprev)
};

// Second-derivative weights w_1..w_R of order 2R (R = 6), the closed form
// 2 (-1)^(p+1) (R!)^2 / (p^2 (R-p)! (R+p)!), as compile-time constants: the
// taps of every cell are w_p times its -1/2 / h^2, so a cell carries only its
// three spacings.
__host__ __device__ constexpr double bfact(int k) { return k <= 1 ? 1.0 : k * bfact(k - 1); }
__host__ __device__ constexpr float bw(int p) {
  return (float)(2.0 * ((p % 2) ? 1.0 : -1.0) * bfact(BR) * bfact(BR) /
                 ((double)p * p * bfact(BR - p) * bfact(BR + p)));
}

// w_p as an immediate for an index that unrolling makes constant
__device__ __forceinline__ float bwc(int p) {
  constexpr float w1 = bw(1), w2 = bw(2), w3 = bw(3), w4 = bw(4), w5 = bw(5), w6 = bw(6);
  switch (p) {
    case 1: return w1;
    case 2: return w2;
    case 3: return w3;
    case 4: return w4;
    case 5: return w5;
    default: return w6;
  }
}

__host__ __device__ inline int bwidth(int nx) {
  // row stride congruent to nx modulo the 128-byte bank cycle (32 floats)
  return nx + 2 * BPAD + ((32 - (2 * BPAD) % 32) % 32);
}

// One item = one vector of one cell through ALL its filter steps: the CTA
// marches the vector's row tiles along z for step 1, then step 2, ..., so a
// step reads what the same CTA wrote in the step before (visible after the
// CTA barrier; every read of the block goes to L2, none through L1) and a
// vector's two live iterates (2 N words) stay in L2 between steps instead of
// streaming through HBM once per step.  Items are claimed largest cell
// first (the host orders them), so the small ones fill the tail.
__global__ void __launch_bounds__(BTHREADS, 2)
batch_filter_kernel(const BCell* __restrict__ cells, const BStep* __restrict__ steps,
                    const long long* __restrict__ item0, const int* __restrict__ cell_of,
                    int ncells, long long total, unsigned long long* counter) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ long long s_item;
  const int tid = threadIdx.x;
  const int nthr = blockDim.x;       // >= the largest tile's thread count
  for (;;) {
    if (tid == 0) s_item = (long long)atomicAdd(counter, 1ull);
    __syncthreads();
    const long long it = s_item;
    __syncthreads();
    if (it >= total) return;
    // position of the item's cell in the claim order (binary search of the
    // prefix sums), then the cell
    int lo = 0, hi = ncells - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (item0[mid] <= it) lo = mid; else hi = mid - 1;
    }
    const int ci = cell_of[lo];
    const BCell& C = cells[ci];
    const long long vec = it - item0[lo];
    const int nx = C.nx, ny = C.ny, nz = C.nz, TY = C.TY, TX = C.TX, Wd = C.Wd;
    const float kdiag = C.kdiag, kc = C.c, hx2 = C.hx2, hy2 = C.hy2, hz2 = C.hz2;
    const int nact = TX * TY;                         // threads with points
    const bool act = tid < nact;
    const int tx = act ? tid % TX : 0, ty = act ? tid / TX : 0;
    const int x0 = tx * BVW;
    const int plane = nx * ny;
    const float* V = C.V;
    const int rows = TY + 2 * BR;
    const int wsz = rows * Wd;
    const int csz = TY * nx;
    float* win = reinterpret_cast<float*>(smem_raw);
    float* cen = win + (BA + 1) * wsz;
    const int rv = TX + 2 * (BPAD / BVW);            // 16-byte vectors per window row
    const int cofs = ty * nx + x0;
    for (int k = 0; k < C.m; ++k) {
      const BStep S = steps[(size_t)k * ncells + ci];
      const float* yv = C.buf[S.y] + vec * C.N;
      const float* pv = S.prev >= 0 ? C.buf[S.prev] + vec * C.N : nullptr;
      float* ov = C.buf[S.out] + vec * C.N;
      for (int tile = 0; tile < C.tiles; ++tile) {
        const int y0 = tile * TY;
        const int col = (y0 + ty) * nx + x0;
        // this thread's window copies (row, 16-byte vector), the same for
        // every plane of the tile: the first BKC precomputed, any beyond
        // (rows longer than BKC x blockDim vectors) on the fly
        auto wcopy = [&](int q, int& src, int& dst) {
          const int r = q / rv, v = q - r * rv;
          int gy = (y0 - BR + r) % ny;
          gy += (gy < 0) ? ny : 0;
          int sx = v * BVW - BPAD;
          sx += (sx < 0) ? nx : 0;
          sx -= (sx >= nx) ? nx : 0;
          src = gy * nx + sx;
          dst = r * Wd + v * BVW;
        };
        int wsrc[BKC], wdst[BKC];
#pragma unroll
        for (int j = 0; j < BKC; ++j) {
          const int q = tid + j * nthr;
          wsrc[j] = -1;
          wdst[j] = 0;
          if (q < rows * rv) wcopy(q, wsrc[j], wdst[j]);
        }
        // entry `e`: window of plane e, centre of plane e + R, V and yprev of e
        auto issue = [&](int e) {
          if (e < nz) {
            const int sl = e % (BA + 1);
            float* w = win + sl * wsz;
            const float* src = yv + (long long)e * plane;
#pragma unroll
            for (int j = 0; j < BKC; ++j)
              if (wsrc[j] >= 0) ac::cp_async16(w + wdst[j], src + wsrc[j]);
            for (int q = tid + BKC * nthr; q < rows * rv; q += nthr) {
              int a, b;
              wcopy(q, a, b);
              ac::cp_async16(w + b, src + a);
            }
            if (act) {
              float* ce = cen + sl * 3 * csz;
              int zq = e + BR;
              zq -= (zq >= nz) ? nz : 0;
              zq -= (zq >= nz) ? nz : 0;
              ac::cp_async16(ce + cofs, yv + (long long)zq * plane + col);
              ac::cp_async16(ce + csz + cofs, V + (long long)e * plane + col);
              if (pv) ac::cp_async16(ce + 2 * csz + cofs, pv + (long long)e * plane + col);
            }
          }
          ac::cp_async_commit();
        };
        // z-neighbour ring: plane z + j - R in q[(z + j) % BQ], the z loop
        // unrolled BQ-fold so every index is a compile-time constant; loaded
        // from L2 (the block changes during the launch)
        constexpr int BQ = 2 * BR + 1;
        float4 q[BQ];
        if (act) {
#pragma unroll
          for (int j = 0; j < 2 * BR; ++j) {
            int zz = j - BR;
            zz += (zz < 0) ? nz : 0;
            zz -= (zz >= nz) ? nz : 0;
            q[j] = __ldcg(reinterpret_cast<const float4*>(yv + (long long)zz * plane + col));
          }
        }
#pragma unroll
        for (int e = 0; e < BA; ++e) issue(e);
        for (int z0 = 0; z0 < nz; z0 += BQ) {
#pragma unroll
          for (int u = 0; u < BQ; ++u) {
            const int z = z0 + u;
            if (z >= nz) break;
            ac::cp_async_wait<BA - 1>();
            __syncthreads();
            issue(z + BA);
            if (act) {
              const int sl = z % (BA + 1);
              const float* ce = cen + sl * 3 * csz;
              q[(u + 2 * BR) % BQ] = *reinterpret_cast<const float4*>(ce + cofs);
              const float4 vz = *reinterpret_cast<const float4*>(ce + csz + cofs);
              const float4 yp = pv ? *reinterpret_cast<const float4*>(ce + 2 * csz + cofs)
                                   : make_float4(0.f, 0.f, 0.f, 0.f);
              const float* row = win + sl * wsz + (ty + BR) * Wd + BPAD + x0;
              float xw[BVW + 2 * BPAD];
#pragma unroll
              for (int j = 0; j < (BVW + 2 * BPAD) / BVW; ++j) {
                const float4 t = (j == BPAD / BVW)
                                     ? q[(u + BR) % BQ]
                                     : *reinterpret_cast<const float4*>(row - BPAD + j * BVW);
                xw[j * 4 + 0] = t.x; xw[j * 4 + 1] = t.y; xw[j * 4 + 2] = t.z; xw[j * 4 + 3] = t.w;
              }
              const float* vzp = reinterpret_cast<const float*>(&vz);
              const float* qc = reinterpret_cast<const float*>(&q[(u + BR) % BQ]);
              // the taps summed per axis with the compile-time weights, then
              // scaled by the cell's spacings
              float sx[BVW], sy[BVW], sz[BVW];
#pragma unroll
              for (int i = 0; i < BVW; ++i) sx[i] = sy[i] = sz[i] = 0.f;
#pragma unroll
              for (int p = 1; p <= BR; ++p) {
                const float4 up = *reinterpret_cast<const float4*>(row + p * Wd);
                const float4 dn = *reinterpret_cast<const float4*>(row - p * Wd);
                const float* upp = reinterpret_cast<const float*>(&up);
                const float* dnp = reinterpret_cast<const float*>(&dn);
                const float* zp = reinterpret_cast<const float*>(&q[(u + BR + p) % BQ]);
                const float* zm = reinterpret_cast<const float*>(&q[(u + BR - p) % BQ]);
                const float wp = bwc(p);
#pragma unroll
                for (int i = 0; i < BVW; ++i) {
                  sx[i] += wp * (xw[BPAD + i + p] + xw[BPAD + i - p]);
                  sy[i] += wp * (upp[i] + dnp[i]);
                  sz[i] += wp * (zp[i] + zm[i]);
                }
              }
              const float* ypp = reinterpret_cast<const float*>(&yp);
              float4 o;
              float* op = reinterpret_cast<float*>(&o);
#pragma unroll
              for (int i = 0; i < BVW; ++i) {
                const float acc = (kdiag + vzp[i] - kc) * qc[i] + hx2 * sx[i] + hy2 * sy[i] +
                                  hz2 * sz[i];
                op[i] = S.s1 * acc + S.s2 * ypp[i];
              }
              *reinterpret_cast<float4*>(ov + (long long)z * plane + col) = o;
            }
          }
        }
        ac::cp_async_wait<0>();
        __syncthreads();     // the ring is reused; the step's writes are visible
      }
    }
    // after an odd number of steps Y_m sits in the work block: copy the
    // vector back into the cell's block
    if (C.m % 2 == 1) {
      const float4* src = reinterpret_cast<const float4*>(C.buf[1] + vec * C.N);
      float4* dst = reinterpret_cast<float4*>(C.buf[0] + vec * C.N);
      for (long long i = tid; i < C.N / 4; i += nthr) dst[i] = __ldcg(src + i);
    }
    __syncthreads();
  }
}

}  // namespace
}  // namespace sq3

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct sq3_batch {
  int device = 0;
  cudaStream_t stream = nullptr;
  std::vector<sq3::BCell> cells;        // host copies (pointers are device)
  std::vector<double> a, b, a0;         // filter bounds per cell
  std::vector<void*> owned;             // work blocks and FP32 potentials
  // device tables
  sq3::BCell* d_cells = nullptr;        // the cells' descriptors
  sq3::BStep* d_steps = nullptr;        // m_max x ncells
  long long* d_item0 = nullptr;         // ncells + 1 prefix sums, claim order
  int* d_cell_of = nullptr;             // claim order -> cell
  unsigned long long* d_counter = nullptr;  // the item counter
  std::vector<sq3::BStep> h_steps;
  std::vector<long long> h_item0;       // ncells + 1
  std::vector<int> h_cell_of;           // ncells
  long long h_total = 0;                // items (vectors of all cells)
  int m_max = 0;
  // launch shape (autotuned) and the captured graph
  int ctas_per_sm = 1;
  int sms = 152;
  size_t smem = 0;
  bool dirty = true;                    // tables or shape changed: re-capture
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool tuned = false;
};

namespace sq3 {
namespace {

void fd_weights12(double* w) {
  const int n = BR;
  auto fact = [](int k) { double f = 1; for (int i = 2; i <= k; ++i) f *= i; return f; };
  w[0] = 0.0;
  for (int p = 1; p <= n; ++p) {
    w[p] = 2.0 * ((p % 2) ? 1.0 : -1.0) * fact(n) * fact(n) /
           ((double)p * p * fact(n - p) * fact(n + p));
    w[0] -= 2.0 / ((double)p * p);
  }
}

__global__ void batch_f32_kernel(const double* a, float* b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}

size_t cell_smem(const BCell& c) {
  return (size_t)(BA + 1) * ((size_t)(c.TY + 2 * BR) * c.Wd + 3 * (size_t)c.TY * c.nx) *
         sizeof(float);
}

// Step tables for the current bounds: the scaled three-term recurrence of
// the Chebyshev filter (as sq3_cheb_filter), with step 1 writing the work
// block and step k >= 2 writing over Y_{k-2}.
void build_steps(sq3_batch* B) {
  const int nc = (int)B->cells.size();
  B->m_max = 0;
  for (auto& c : B->cells) B->m_max = std::max(B->m_max, c.m);
  B->h_steps.assign((size_t)B->m_max * nc, BStep{0.f, 0.f, 0, -1, 1});
  for (int ci = 0; ci < nc; ++ci) {
    BCell& c = B->cells[ci];
    const double e = 0.5 * (B->b[ci] - B->a[ci]), ctr = 0.5 * (B->b[ci] + B->a[ci]);
    c.c = (float)ctr;
    const double s1 = e / (B->a0[ci] - ctr), tau = 2.0 / s1;
    double s = s1;
    int cur = 1, prev = 0;       // after step 1: Y_1 in the work block, Y_0 in X
    B->h_steps[ci] = BStep{(float)(s1 / e), 0.f, 0, -1, 1};
    for (int k = 2; k <= c.m; ++k) {
      const double sn = 1.0 / (tau - s);
      B->h_steps[(size_t)(k - 1) * nc + ci] =
          BStep{(float)(2.0 * sn / e), (float)(-s * sn), cur, prev, prev};
      std::swap(cur, prev);
      s = sn;
    }
  }
  // items: the vectors of every cell, cells in decreasing order of grid
  // size (the largest items are claimed first)
  B->h_cell_of.resize(nc);
  for (int ci = 0; ci < nc; ++ci) B->h_cell_of[ci] = ci;
  std::stable_sort(B->h_cell_of.begin(), B->h_cell_of.end(), [&](int u, int v) {
    return B->cells[u].N * B->cells[u].m > B->cells[v].N * B->cells[v].m;
  });
  B->h_item0.assign(nc + 1, 0);
  for (int j = 0; j < nc; ++j)
    B->h_item0[j + 1] = B->h_item0[j] + B->cells[B->h_cell_of[j]].Ns;
  B->h_total = B->h_item0[nc];
}

void free_graph(sq3_batch* B) {
  if (B->exec) cudaGraphExecDestroy(B->exec);
  if (B->graph) cudaGraphDestroy(B->graph);
  B->exec = nullptr;
  B->graph = nullptr;
}

void free_tables(sq3_batch* B) {
  void* ps[] = {B->d_cells, B->d_steps, B->d_item0, B->d_cell_of, B->d_counter};
  for (void* p : ps) if (p) cudaFree(p);
  B->d_cells = nullptr; B->d_steps = nullptr; B->d_item0 = nullptr; B->d_cell_of = nullptr;
  B->d_counter = nullptr;
}

int upload_tables(sq3_batch* B) {
  free_tables(B);
  const int nc = (int)B->cells.size();
  auto put = [&](void** d, const void* h, size_t bytes) -> int {
    if (cudaMalloc(d, bytes) != cudaSuccess) { cudaGetLastError(); *d = nullptr; return SQ3_ENOMEM; }
    return cuda_err(cudaMemcpy(*d, h, bytes, cudaMemcpyHostToDevice));
  };
  int rc = put((void**)&B->d_cells, B->cells.data(), nc * sizeof(BCell));
  if (!rc) rc = put((void**)&B->d_steps, B->h_steps.data(), B->h_steps.size() * sizeof(BStep));
  if (!rc) rc = put((void**)&B->d_item0, B->h_item0.data(), B->h_item0.size() * sizeof(long long));
  if (!rc) rc = put((void**)&B->d_cell_of, B->h_cell_of.data(), B->h_cell_of.size() * sizeof(int));
  if (!rc && cudaMalloc((void**)&B->d_counter, sizeof(unsigned long long)) != cudaSuccess) {
    cudaGetLastError();
    rc = SQ3_ENOMEM;
  }
  return rc;
}

// Threads per CTA: the largest tile's threads (TX TY), rounded up to whole
// warps; the narrower cells' tiles leave the rest idle.
int batch_threads(const sq3_batch* B) {
  int t = 32;
  for (auto& c : B->cells) t = std::max(t, c.TX * c.TY);
  return std::min(BTHREADS, (t + 31) / 32 * 32);
}

// Enqueue the whole filter: a counter reset and one persistent launch that
// takes every vector of every cell through all of its steps.
int enqueue(sq3_batch* B, cudaStream_t st) {
  const int nc = (int)B->cells.size();
  auto k = batch_filter_kernel;
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)B->smem) !=
      cudaSuccess)
    return cuda_err(cudaGetLastError());
  int rc = cuda_err(cudaMemsetAsync(B->d_counter, 0, sizeof(unsigned long long), st));
  if (rc) return rc;
  const unsigned grid = (unsigned)(B->sms * B->ctas_per_sm);
  k<<<grid, batch_threads(B), B->smem, st>>>(B->d_cells, B->d_steps, B->d_item0, B->d_cell_of, nc,
                                     B->h_total, B->d_counter);
  return cuda_err(cudaGetLastError());
}

int capture(sq3_batch* B) {
  free_graph(B);
  cudaStream_t cs;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess)
    return cuda_err(cudaGetLastError());
  int rc = cuda_err(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  if (rc == SQ3_OK) {
    const int erc = enqueue(B, cs);
    cudaGraph_t g = nullptr;
    rc = cuda_err(cudaStreamEndCapture(cs, &g));
    if (rc == SQ3_OK && erc) rc = erc;
    if (rc == SQ3_OK) {
      B->graph = g;
      rc = cuda_err(cudaGraphInstantiate(&B->exec, g, 0));
    } else if (g) {
      cudaGraphDestroy(g);
    }
  }
  cudaStreamDestroy(cs);
  return rc;
}

}  // namespace
}  // namespace sq3

using namespace sq3;

extern "C" {

int sq3_batch_create(int device, void* cuda_stream, sq3_batch** out) {
  if (!out) return SQ3_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return device < 0 ? SQ3_EINVAL : SQ3_ECUDA;
  }
  if (cudaSetDevice(device) != cudaSuccess) return SQ3_ECUDA;
  sq3_batch* B = new sq3_batch();
  B->device = device;
  B->stream = (cudaStream_t)cuda_stream;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) == cudaSuccess && sms > 0)
    B->sms = sms;
  cudaGetLastError();
  *out = B;
  return SQ3_OK;
}

void sq3_batch_destroy(sq3_batch* B) {
  if (!B) return;
  cudaSetDevice(B->device);
  cudaStreamSynchronize(B->stream);
  free_graph(B);
  free_tables(B);
  for (void* p : B->owned) cudaFree(p);
  delete B;
}

int sq3_batch_add_cell(sq3_batch* B, int nx, int ny, int nz, double Lx, double Ly, double Lz,
                       const double* V, float* X, int Ns, int degree) {
  if (!B || !V || !X || Ns < 1 || degree < 1 || degree > BMAX_STEPS) return SQ3_EINVAL;
  if ((int)B->cells.size() >= BMAX_CELLS) return SQ3_EINVAL;
  if (nx % BVW || nx < 2 * BPAD || ny < BR || nz < BR || nx > 512 || !(Lx > 0) || !(Ly > 0) ||
      !(Lz > 0) || ((uintptr_t)X & 15))
    return SQ3_EINVAL;
  cudaSetDevice(B->device);
  BCell c{};
  c.nx = nx; c.ny = ny; c.nz = nz;
  c.TX = nx / BVW;
  c.Wd = bwidth(nx);
  c.N = (long long)nx * ny * nz;
  c.Ns = Ns;
  c.m = degree;
  // tile height: the largest divisor of ny with TX TY <= 256 whose window
  // copies fit the block (the autotuner may lower it)
  c.TY = 0;
  for (int t = 1; t <= ny; ++t)
    if (ny % t == 0 && c.TX * t <= BTHREADS) c.TY = t;
  if (c.TY == 0) return SQ3_EINVAL;
  c.tiles = ny / c.TY;
  double w[BR + 1];
  fd_weights12(w);
  const double ix = 1.0 / ((Lx / nx) * (Lx / nx)), iy = 1.0 / ((Ly / ny) * (Ly / ny)),
               iz = 1.0 / ((Lz / nz) * (Lz / nz));
  c.kdiag = (float)(-0.5 * w[0] * (ix + iy + iz));
  c.hx2 = (float)(-0.5 * ix);
  c.hy2 = (float)(-0.5 * iy);
  c.hz2 = (float)(-0.5 * iz);
  float* Vf = nullptr;
  float* W = nullptr;
  if (cudaMalloc((void**)&Vf, c.N * sizeof(float)) != cudaSuccess ||
      cudaMalloc((void**)&W, (size_t)c.N * Ns * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    if (Vf) cudaFree(Vf);
    return SQ3_ENOMEM;
  }
  B->owned.push_back(Vf);
  B->owned.push_back(W);
  batch_f32_kernel<<<(unsigned)std::min<long long>((c.N + 255) / 256, 1216), 256, 0,
                     B->stream>>>(V, Vf, c.N);
  int rc = cuda_err(cudaGetLastError());
  if (rc) return rc;
  rc = cuda_err(cudaStreamSynchronize(B->stream));
  if (rc) return rc;
  c.V = Vf;
  c.buf[0] = X;
  c.buf[1] = W;
  B->cells.push_back(c);
  B->a.push_back(0.0);
  B->b.push_back(1.0);
  B->a0.push_back(-1.0);
  B->dirty = true;
  B->tuned = false;
  return (int)B->cells.size() - 1;
}

int sq3_batch_set_bounds(sq3_batch* B, int cell, double a, double b, double a0) {
  if (!B || cell < 0 || cell >= (int)B->cells.size() || !(a0 < a) || !(a < b)) return SQ3_EINVAL;
  B->a[cell] = a;
  B->b[cell] = b;
  B->a0[cell] = a0;
  return SQ3_OK;
}

// Shared memory for a tile-height choice applied to every cell.
static size_t batch_smem(sq3_batch* B) {
  size_t s = 0;
  for (auto& c : B->cells) s = std::max(s, cell_smem(c));
  return s;
}

int sq3_batch_filter(sq3_batch* B) {
  if (!B || B->cells.empty()) return SQ3_EINVAL;
  cudaSetDevice(B->device);
  build_steps(B);
  B->smem = batch_smem(B);
  if (B->smem > 227 * 1024) return SQ3_EINVAL;
  int rc = SQ3_OK;
  if (B->dirty || !B->exec) {
    rc = upload_tables(B);
    if (rc) return rc;
    rc = capture(B);
    if (rc) return rc;
    B->dirty = false;
  } else {
    // new bounds only: refresh the step table in place (the graph reads it)
    rc = cuda_err(cudaMemcpyAsync(B->d_steps, B->h_steps.data(),
                                  B->h_steps.size() * sizeof(BStep), cudaMemcpyHostToDevice,
                                  B->stream));
    if (rc) return rc;
    rc = cuda_err(cudaMemcpyAsync(B->d_cells, B->cells.data(), B->cells.size() * sizeof(BCell),
                                  cudaMemcpyHostToDevice, B->stream));
    if (rc) return rc;
  }
  rc = cuda_err(cudaGraphLaunch(B->exec, B->stream));
  if (rc) return rc;
  return cuda_err(cudaStreamSynchronize(B->stream));
}

int sq3_batch_autotune(sq3_batch* B, int* best_ctas, int* best_ty_scale) {
  if (!B || B->cells.empty()) return SQ3_EINVAL;
  cudaSetDevice(B->device);
  // candidates: 1 or 2 resident CTAs per SM, and the cells' tile heights
  // as chosen or halved (smaller tiles: more items, less shared memory)
  std::vector<int> ty0;
  for (auto& c : B->cells) ty0.push_back(c.TY);
  // the trial runs filter the blocks in place: keep a copy to put back
  std::vector<float*> keep(B->cells.size(), nullptr);
  for (size_t i = 0; i < B->cells.size(); ++i) {
    const BCell& c = B->cells[i];
    const size_t bytes = (size_t)c.N * c.Ns * sizeof(float);
    if (cudaMalloc((void**)&keep[i], bytes) != cudaSuccess) {
      cudaGetLastError();
      for (float* k : keep) if (k) cudaFree(k);
      return SQ3_ENOMEM;
    }
    cudaMemcpyAsync(keep[i], c.buf[0], bytes, cudaMemcpyDeviceToDevice, B->stream);
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  int bc = 1, bs = 1;
  int rc = SQ3_OK;
  for (int scale : {1, 2}) {
    bool ok = true;
    for (size_t i = 0; i < B->cells.size(); ++i) {
      BCell& c = B->cells[i];
      int t = ty0[i];
      if (scale == 2) {
        if (t % 2 || t / 2 < 1 || c.ny % (t / 2)) { ok = false; }
        else t = t / 2;
      }
      c.TY = t;
      c.tiles = c.ny / t;
    }
    if (!ok) continue;
    for (int ctas : {1, 2}) {
      B->ctas_per_sm = ctas;
      B->dirty = true;
      if (batch_smem(B) * ctas > 228 * 1024) continue;
      rc = sq3_batch_filter(B);            // builds the graph and warms it up
      if (rc) break;
      cudaEventRecord(e0, B->stream);
      rc = cuda_err(cudaGraphLaunch(B->exec, B->stream));
      cudaEventRecord(e1, B->stream);
      if (rc == SQ3_OK) rc = cuda_err(cudaEventSynchronize(e1));
      if (rc) break;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) { best = ms; bc = ctas; bs = scale; }
    }
    if (rc) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  for (size_t i = 0; i < B->cells.size(); ++i) {
    const BCell& c = B->cells[i];
    cudaMemcpyAsync(c.buf[0], keep[i], (size_t)c.N * c.Ns * sizeof(float),
                    cudaMemcpyDeviceToDevice, B->stream);
  }
  if (cudaStreamSynchronize(B->stream) != cudaSuccess && rc == SQ3_OK) rc = SQ3_ECUDA;
  for (float* k : keep) cudaFree(k);
  // apply the winner
  for (size_t i = 0; i < B->cells.size(); ++i) {
    BCell& c = B->cells[i];
    c.TY = bs == 2 ? ty0[i] / 2 : ty0[i];
    c.tiles = c.ny / c.TY;
  }
  B->ctas_per_sm = bc;
  B->dirty = true;
  B->tuned = true;
  if (best_ctas) *best_ctas = bc;
  if (best_ty_scale) *best_ty_scale = bs;
  return rc;
}

}  // extern "C"
