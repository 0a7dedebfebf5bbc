// Hamiltonian apply and Chebyshev-filter step on a periodic grid.
//
// H y = -1/2 Lap y + V y + sum_p gamma_p c_p (c_p^T y)   (Sec. 2, Eq. (KSeqn),
// Eq. (nonlocaloperator)), with Lap the central finite-difference Laplacian of
// order 2R (R <= 6; the paper uses twelfth order, Sec. 5).  One launch
// computes, for every vector of a block,
//
//     out = s1 * (H y - c y) + s2 * yprev,
//
// which covers both a plain apply (s1 = 1, c = 0, s2 = 0) and one step of the
// scaled Chebyshev filter recurrence.
//
// Layout: a CTA owns TY full x-rows of one vector and marches along z.  The
// 2R+1 z-neighbours of each (x, y) column live in a register queue; the
// current z-plane of the CTA's rows plus R halo rows above and below (wrapped
// periodically) is staged in shared memory, so x- and y-taps read shared
// memory and the x wrap costs nothing.  Every element of y is loaded from
// global memory once per CTA for the queue plus once for each neighbouring
// tile's y-halo; yprev, V and out stream once.  The nonlocal term is added
// from a per-point table of (projector, c_p[k]) and the precomputed
// coefficients gC = gamma (c^T y) of the same vector.
#include <stdint.h>
#include <type_traits>
#include <stdlib.h>

#include "async_copy.cuh"
#include "sq3_internal.cuh"

namespace sq3 {

using namespace ac;

template <typename T>
struct StepCoef {
  T diag;                      // -1/2 w0 (1/hx^2 + 1/hy^2 + 1/hz^2)
  T ax[SQ3_MAX_FD_RADIUS + 1]; // -1/2 w_p / hx^2
  T ay[SQ3_MAX_FD_RADIUS + 1];
  T az[SQ3_MAX_FD_RADIUS + 1];
};

// VB vectors per CTA share the (x, y) tile: the potential and the index
// arithmetic are loaded once for all VB.  Shared-memory rows carry R wrapped
// columns on each side, so the x-taps need no index wrap.  The next plane's
// register-queue entry and yprev are loaded one iteration ahead.  This is
// the general form (any row length); the vectorised forms below take rows
// whose length is a multiple of the 16-byte vector width.
template <typename T, int R, int VB>
__global__ void __launch_bounds__(512, 1)
cheb_step_kernel(int nx, int ny, int nz, int Ns, int TY, StepCoef<T> k,
                 const T* __restrict__ y, const T* yprev, T* out,
                 const T* __restrict__ V, T s1, T c, T s2) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int rows = TY + 2 * R;
  const int W = nx + 2 * R;                          // padded row width
  T* sm = reinterpret_cast<T*>(smem_raw);           // VB planes, rows x W each
  const int tid = threadIdx.x;
  const int x = tid % nx;
  const int ty = tid / nx;
  const int y0 = blockIdx.x * TY;
  const int yy = y0 + ty;
  const bool active = (ty < TY) && (yy < ny);
  const int plane = nx * ny;
  const long long N = (long long)plane * nz;
  const int v0 = blockIdx.y * VB;
  const int nv = min(VB, Ns - v0);
  const int col = yy * nx + x;
  const T* yb[VB];
  T* ob[VB];
  const T* pb[VB];
#pragma unroll
  for (int v = 0; v < VB; ++v) {
    const int vv = (v < nv) ? v0 + v : v0;
    yb[v] = y + (long long)vv * N;
    ob[v] = out + (long long)vv * N;
    pb[v] = (yprev != nullptr) ? yprev + (long long)vv * N : nullptr;
  }

  T q[VB][2 * R + 1];
  T ypn[VB], la[VB];
#pragma unroll
  for (int v = 0; v < VB; ++v) {
#pragma unroll
    for (int i = 0; i < 2 * R + 1; ++i) q[v][i] = T(0);
    ypn[v] = T(0);
    la[v] = T(0);
  }
  if (active) {
#pragma unroll
    for (int v = 0; v < VB; ++v) {
#pragma unroll
      for (int i = 1; i < 2 * R + 1; ++i) {
        int zz = i - 1 - R;                          // planes -R .. R-1
        zz += (zz < 0) ? nz : 0;
        zz -= (zz >= nz) ? nz : 0;
        q[v][i] = __ldg(yb[v] + zz * plane + col);
      }
      // first look-ahead: plane R for the queue, plane 0 of yprev
      la[v] = __ldg(yb[v] + (R % nz) * plane + col);
      if (s2 != T(0)) ypn[v] = pb[v][col];
    }
  }

  for (int z = 0; z < nz; ++z) {
    const int gidx = z * plane + col;
    T yp[VB];
#pragma unroll
    for (int v = 0; v < VB; ++v) {
      // la[v] holds the look-ahead value for plane z + R
#pragma unroll
      for (int i = 0; i < 2 * R; ++i) q[v][i] = q[v][i + 1];
      q[v][2 * R] = la[v];
      yp[v] = ypn[v];
    }
    T vz = T(0);
    if (active) {
      // look-ahead loads for the next iteration
      if (z + 1 < nz) {
        int zl = z + 1 + R;
        zl -= (zl >= nz) ? nz : 0;
        zl -= (zl >= nz) ? nz : 0;
#pragma unroll
        for (int v = 0; v < VB; ++v) {
          la[v] = __ldg(yb[v] + zl * plane + col);
          if (s2 != T(0)) ypn[v] = pb[v][gidx + plane];
        }
      }
      vz = __ldg(V + gidx);
    }

    __syncthreads();  // previous plane fully consumed
#pragma unroll
    for (int v = 0; v < VB; ++v) {
      T* smv = sm + (size_t)v * rows * W;
      if (active) {
        T* row = smv + (ty + R) * W + R;
        const T u = q[v][R];
        row[x] = u;
        if (x < R) row[nx + x] = u;                  // wrapped right halo
        if (x >= nx - R) row[x - nx] = u;            // wrapped left halo
      }
      const T* pz = yb[v] + z * plane;
      for (int e = tid; e < 2 * R * nx; e += blockDim.x) {
        const int r = e / nx, xx = e - r * nx;
        const int srow = (r < R) ? r : (r + TY);
        int gy = y0 - R + srow;
        gy %= ny;
        gy += (gy < 0) ? ny : 0;
        const T u = __ldg(pz + gy * nx + xx);
        T* row = smv + srow * W + R;
        row[xx] = u;
        if (xx < R) row[nx + xx] = u;
        if (xx >= nx - R) row[xx - nx] = u;
      }
      for (int e = tid; e < TY * nx; e += blockDim.x) {   // rows past ny (tiny grids)
        const int r = e / nx, xx = e - r * nx;
        if (y0 + r >= ny) {
          const T u = __ldg(pz + ((y0 + r) % ny) * nx + xx);
          T* row = smv + (r + R) * W + R;
          row[xx] = u;
          if (xx < R) row[nx + xx] = u;
          if (xx >= nx - R) row[xx - nx] = u;
        }
      }
    }
    __syncthreads();

    if (active) {
      T acc[VB];
#pragma unroll
      for (int v = 0; v < VB; ++v) {
        const T* row = sm + (size_t)v * rows * W + (ty + R) * W + R + x;
        const T u = q[v][R];
        T a = (k.diag + vz - c) * u;
#pragma unroll
        for (int p = 1; p <= R; ++p) {
          a += k.ax[p] * (row[p] + row[-p]);
          a += k.ay[p] * (row[p * W] + row[-p * W]);
          a += k.az[p] * (q[v][R + p] + q[v][R - p]);
        }
        acc[v] = a;
      }
#pragma unroll
      for (int v = 0; v < VB; ++v)
        if (v < nv) ob[v][gidx] = s1 * acc[v] + s2 * yp[v];
    }
  }
}

// ---------------------------------------------------------------------------
// Vectorised variant for rows whose length is a multiple of the 16-byte
// vector width VW (4 floats or 2 doubles).  Each thread owns VW consecutive
// points of one row: global loads and stores are 16-byte vectors, the
// x-taps come from one contiguous run of VW + 2 PAD shared-memory values,
// each y-tap is one 16-byte shared load serving VW points, and the
// register queue holds 16-byte vectors.  Blocks are ordered row-tile-fastest
// so that the tiles of one vector run together and read each other's halo
// rows from L2.  The nonlocal term is added by the nonlocal pass afterwards.
// ---------------------------------------------------------------------------
template <typename T> struct Vec16;
template <> struct Vec16<float> { using type = float4; static constexpr int W = 4; };
template <> struct Vec16<double> { using type = double2; static constexpr int W = 2; };

template <typename T, int R>
__global__ void __launch_bounds__(256, 2)
cheb_step_vec_kernel(int nx, int ny, int nz, int TY, StepCoef<T> k,
                     const T* __restrict__ y, const T* yprev, T* out,
                     const T* __restrict__ V, T s1, T c, T s2) {
  using VT = typename Vec16<T>::type;
  constexpr int VW = Vec16<T>::W;
  constexpr int PAD = ((R + VW - 1) / VW) * VW;
  constexpr int HS = 2;                                // halo slots per thread
  constexpr int XW = VW + 2 * PAD;                     // x-window length
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int TX = nx / VW;
  const int Wd = nx + 2 * PAD;
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int tid = threadIdx.x;
  const int tx = tid % TX, ty = tid / TX;
  const int x0 = tx * VW;
  const long long vec = blockIdx.y;
  const int y0 = blockIdx.x * TY;
  const int yy = y0 + ty;
  const int plane = nx * ny;
  const long long N = (long long)plane * nz;
  const T* yv = y + vec * N;
  T* ov = out + vec * N;
  const T* pv = (yprev != nullptr) ? yprev + vec * N : nullptr;
  const int col = yy * nx + x0;

  // halo rows of a plane (2R rows x TX vectors) spread over the threads
  int hsrc[HS], hdst[HS];
  const int nhalo = 2 * R * TX;
#pragma unroll
  for (int sl = 0; sl < HS; ++sl) {
    const int e = tid + sl * blockDim.x;
    hsrc[sl] = -1;
    hdst[sl] = 0;
    if (e < nhalo) {
      const int r = e / TX, hx = e - r * TX;
      const int srow = (r < R) ? r : r + TY;
      int gy = (y0 - R + srow) % ny;
      gy += (gy < 0) ? ny : 0;
      hsrc[sl] = gy * nx + hx * VW;
      hdst[sl] = srow * Wd + PAD + hx * VW;
    }
  }
  const bool padr = x0 < PAD;             // also feeds the right pad
  const bool padl = x0 >= nx - PAD;       // also feeds the left pad

  VT q[2 * R + 1];
  VT la, ypn;
#pragma unroll
  for (int i = 1; i < 2 * R + 1; ++i) {
    int zz = i - 1 - R;
    zz += (zz < 0) ? nz : 0;
    zz -= (zz >= nz) ? nz : 0;
    q[i] = *reinterpret_cast<const VT*>(yv + zz * plane + col);
  }
  la = *reinterpret_cast<const VT*>(yv + (R % nz) * plane + col);
  if (s2 != T(0)) ypn = *reinterpret_cast<const VT*>(pv + col);
  else ypn = VT{};

  for (int z = 0; z < nz; ++z) {
#pragma unroll
    for (int i = 0; i < 2 * R; ++i) q[i] = q[i + 1];
    q[2 * R] = la;
    const VT yp = ypn;
    const int gz = z * plane;
    if (z + 1 < nz) {
      int zl = z + 1 + R;
      zl -= (zl >= nz) ? nz : 0;
      zl -= (zl >= nz) ? nz : 0;
      la = __ldg(reinterpret_cast<const VT*>(yv + zl * plane + col));
      if (s2 != T(0)) ypn = *reinterpret_cast<const VT*>(pv + gz + plane + col);
    }
    const VT vz = __ldg(reinterpret_cast<const VT*>(V + gz + col));
    VT hv[HS];
#pragma unroll
    for (int sl = 0; sl < HS; ++sl)
      if (hsrc[sl] >= 0) hv[sl] = __ldg(reinterpret_cast<const VT*>(yv + gz + hsrc[sl]));

    __syncthreads();   // previous plane consumed
    {
      T* d = sm + (ty + R) * Wd + PAD + x0;
      *reinterpret_cast<VT*>(d) = q[R];
      if (padr) *reinterpret_cast<VT*>(d + nx) = q[R];
      if (padl) *reinterpret_cast<VT*>(d - nx) = q[R];
    }
#pragma unroll
    for (int sl = 0; sl < HS; ++sl) {
      if (hsrc[sl] >= 0) {
        T* d = sm + hdst[sl];
        const int hx0 = hsrc[sl] % nx;
        *reinterpret_cast<VT*>(d) = hv[sl];
        if (hx0 < PAD) *reinterpret_cast<VT*>(d + nx) = hv[sl];
        if (hx0 >= nx - PAD) *reinterpret_cast<VT*>(d - nx) = hv[sl];
      }
    }
    __syncthreads();

    const T* row = sm + (ty + R) * Wd + PAD + x0;
    T xw[XW];
#pragma unroll
    for (int j = 0; j < XW / VW; ++j) {
      const VT t = *reinterpret_cast<const VT*>(row - PAD + j * VW);
      const T* tp = reinterpret_cast<const T*>(&t);
#pragma unroll
      for (int i = 0; i < VW; ++i) xw[j * VW + i] = tp[i];
    }
    T acc[VW];
    const T* vzp = reinterpret_cast<const T*>(&vz);
    const T* qc = reinterpret_cast<const T*>(&q[R]);
#pragma unroll
    for (int i = 0; i < VW; ++i) acc[i] = (k.diag + vzp[i] - c) * qc[i];
#pragma unroll
    for (int p = 1; p <= R; ++p) {
      const VT up = *reinterpret_cast<const VT*>(row + p * Wd);
      const VT dn = *reinterpret_cast<const VT*>(row - p * Wd);
      const T* upp = reinterpret_cast<const T*>(&up);
      const T* dnp = reinterpret_cast<const T*>(&dn);
      const T* zp = reinterpret_cast<const T*>(&q[R + p]);
      const T* zm = reinterpret_cast<const T*>(&q[R - p]);
#pragma unroll
      for (int i = 0; i < VW; ++i) {
        acc[i] += k.ax[p] * (xw[PAD + i + p] + xw[PAD + i - p]);
        acc[i] += k.ay[p] * (upp[i] + dnp[i]);
        acc[i] += k.az[p] * (zp[i] + zm[i]);
      }
    }
    VT o;
    T* op = reinterpret_cast<T*>(&o);
    const T* ypp = reinterpret_cast<const T*>(&yp);
#pragma unroll
    for (int i = 0; i < VW; ++i) op[i] = s1 * acc[i] + s2 * ypp[i];
    *reinterpret_cast<VT*>(ov + gz + col) = o;
  }
}

// Row stride of the ring's window: the row plus PAD wrapped columns per
// side, padded so that the stride is congruent to nx modulo the 128-byte
// bank cycle; a warp whose threads straddle two rows then maps onto banks as
// if the rows were contiguous (no bank conflicts between its quarter-warps).
template <typename T>
__host__ __device__ inline int ring_row_width(int nx, int pad) {
  const int cyc = 128 / (int)sizeof(T);
  return nx + 2 * pad + ((cyc - (2 * pad) % cyc) % cyc);
}

// Pipelined form of the vectorised step.  The same tile and register queue,
// but every plane's inputs arrive by asynchronous copies issued A planes
// ahead into a ring of A + 1 shared-memory entries, so each thread keeps
// several planes of loads in flight without holding them in registers:
//   window ring : y plane z, TY + 2R rows with PAD wrapped columns per side
//                 (the x- and y-taps);
//   centre ring : y plane z + R on the CTA's own rows (the queue's new
//                 entry), V and yprev of plane z.
// The centre copy is the first touch of each element; the window copy of
// the same rows R planes later hits L2.  One barrier per plane.
template <typename T, int R, int A>
__global__ void __launch_bounds__(256, 2)
cheb_step_ring_kernel(int nx, int ny, int nz, int TY, StepCoef<T> k,
                      const T* __restrict__ y, const T* yprev, T* out,
                      const T* __restrict__ V, T s1, T c, T s2) {
  using VT = typename Vec16<T>::type;
  constexpr int VW = Vec16<T>::W;
  constexpr int PAD = ((R + VW - 1) / VW) * VW;
  constexpr int PV = PAD / VW;
  constexpr int XW = VW + 2 * PAD;
  constexpr int KC = 4;                  // window copies per thread per plane
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int TX = nx / VW;
  const int Wd = ring_row_width<T>(nx, PAD);
  const int rows = TY + 2 * R;
  const int wsz = rows * Wd;             // one window entry
  const int csz = TY * nx;               // one centre array
  T* win = reinterpret_cast<T*>(smem_raw);
  T* cen = win + (A + 1) * wsz;          // (A + 1) entries of 3 centre arrays
  const int nthr = blockDim.x;
  const int tid = threadIdx.x;
  const int tx = tid % TX, ty = tid / TX;
  const int x0 = tx * VW;
  const long long vec = blockIdx.y;
  const int y0 = blockIdx.x * TY;
  const int plane = nx * ny;
  const long long N = (long long)plane * nz;
  const T* yv = y + vec * N;
  T* ov = out + vec * N;
  const T* pv = (s2 != T(0)) ? yprev + vec * N : nullptr;
  const int col = (y0 + ty) * nx + x0;
  const int cofs = ty * nx + x0;

  // this thread's share of a window: (row, 16-byte vector) pairs
  const int rv = TX + 2 * PV;
  int wsrc[KC], wdst[KC];
#pragma unroll
  for (int j = 0; j < KC; ++j) {
    const int e = tid + j * nthr;
    wsrc[j] = -1;
    wdst[j] = 0;
    if (e < rows * rv) {
      const int r = e / rv, v = e - r * rv;
      int gy = (y0 - R + r) % ny;
      gy += (gy < 0) ? ny : 0;
      int sx = v * VW - PAD;
      sx += (sx < 0) ? nx : 0;
      sx -= (sx >= nx) ? nx : 0;
      wsrc[j] = gy * nx + sx;
      wdst[j] = r * Wd + v * VW;
    }
  }
  // entry `it`: window of plane it, centre of plane it + R, V and yprev of it
  auto issue = [&](int it) {
    if (it < nz) {
      const int sl = it % (A + 1);
      T* w = win + sl * wsz;
      const T* src = yv + (long long)it * plane;
#pragma unroll
      for (int j = 0; j < KC; ++j)
        if (wsrc[j] >= 0) cp_async16(w + wdst[j], src + wsrc[j]);
      T* ce = cen + sl * 3 * csz;
      int zq = it + R;
      zq -= (zq >= nz) ? nz : 0;
      zq -= (zq >= nz) ? nz : 0;
      cp_async16(ce + cofs, yv + (long long)zq * plane + col);
      cp_async16(ce + csz + cofs, V + (long long)it * plane + col);
      if (pv) cp_async16(ce + 2 * csz + cofs, pv + (long long)it * plane + col);
    }
    cp_async_commit();
  };

  // The 2R+1 z-neighbours live in a register ring: plane z + j - R is in
  // q[(z + j) % Q], Q = 2R + 1.  The z loop is unrolled Q-fold so that every
  // ring index is a compile-time constant: the new entry overwrites the
  // slot of the plane that just left the window and no register moves.
  constexpr int Q = 2 * R + 1;
  VT q[Q];
#pragma unroll
  for (int j = 0; j < 2 * R; ++j) {
    int zz = j - R;
    zz += (zz < 0) ? nz : 0;
    zz -= (zz >= nz) ? nz : 0;
    q[j] = __ldg(reinterpret_cast<const VT*>(yv + (long long)zz * plane + col));
  }
#pragma unroll
  for (int it = 0; it < A; ++it) issue(it);

  for (int z0 = 0; z0 < nz; z0 += Q) {
#pragma unroll
    for (int u = 0; u < Q; ++u) {
      const int z = z0 + u;
      if (z >= nz) break;                  // the same for every thread
      cp_async_wait<A - 1>();
      __syncthreads();     // entry z landed for all; entry z - 1 fully consumed
      issue(z + A);        // reuses the slot of entry z - 1
      const int sl = z % (A + 1);
      const T* ce = cen + sl * 3 * csz;
      q[(u + 2 * R) % Q] = *reinterpret_cast<const VT*>(ce + cofs);
      const VT vz = *reinterpret_cast<const VT*>(ce + csz + cofs);
      const VT yp = pv ? *reinterpret_cast<const VT*>(ce + 2 * csz + cofs) : VT{};
      const T* row = win + sl * wsz + (ty + R) * Wd + PAD + x0;
      // the x-window; its centre vector is the queue's centre entry
      T xw[XW];
#pragma unroll
      for (int j = 0; j < XW / VW; ++j) {
        const VT t = (j == PV) ? q[(u + R) % Q] : *reinterpret_cast<const VT*>(row - PAD + j * VW);
        const T* tp = reinterpret_cast<const T*>(&t);
#pragma unroll
        for (int i = 0; i < VW; ++i) xw[j * VW + i] = tp[i];
      }
      T acc[VW];
      const T* vzp = reinterpret_cast<const T*>(&vz);
      const T* qc = reinterpret_cast<const T*>(&q[(u + R) % Q]);
#pragma unroll
      for (int i = 0; i < VW; ++i) acc[i] = (k.diag + vzp[i] - c) * qc[i];
#pragma unroll
      for (int p = 1; p <= R; ++p) {
        const VT up = *reinterpret_cast<const VT*>(row + p * Wd);
        const VT dn = *reinterpret_cast<const VT*>(row - p * Wd);
        const T* upp = reinterpret_cast<const T*>(&up);
        const T* dnp = reinterpret_cast<const T*>(&dn);
        const T* zp = reinterpret_cast<const T*>(&q[(u + R + p) % Q]);
        const T* zm = reinterpret_cast<const T*>(&q[(u + R - p) % Q]);
#pragma unroll
        for (int i = 0; i < VW; ++i) {
          acc[i] += k.ax[p] * (xw[PAD + i + p] + xw[PAD + i - p]);
          acc[i] += k.ay[p] * (upp[i] + dnp[i]);
          acc[i] += k.az[p] * (zp[i] + zm[i]);
        }
      }
      VT o;
      T* op = reinterpret_cast<T*>(&o);
      const T* ypp = reinterpret_cast<const T*>(&yp);
#pragma unroll
      for (int i = 0; i < VW; ++i) op[i] = s1 * acc[i] + s2 * ypp[i];
      *reinterpret_cast<VT*>(ov + (long long)z * plane + col) = o;
    }
  }
  cp_async_wait<0>();
}

static int pick_ty(int nx, int ny, int target) {
  int best = 1;
  for (int t = 1; t <= ny; ++t)
    if (ny % t == 0 && nx * t <= target) best = t;
  if (nx * best < 128) {  // tiny rows: allow a ragged last tile
    best = target / nx;
    if (best > ny) best = ny;
    if (best < 1) best = 1;
  }
  return best;
}

static int stencil_vb(int esize) { return esize == 8 ? 1 : 2; }

template <typename T, int R, int VB>
static void launch_rv(const sq3_ctx* ctx, const T* y, const T* yprev, T* out,
                      int Ns, double s1, double c, double s2, cudaStream_t st) {
  const Grid& g = ctx->grid;
  StepCoef<T> k{};
  double ix = 1.0 / (g.hx * g.hx), iy = 1.0 / (g.hy * g.hy),
         iz = 1.0 / (g.hz * g.hz);
  k.diag = T(-0.5 * g.w[0] * (ix + iy + iz));
  for (int p = 1; p <= R; ++p) {
    k.ax[p] = T(-0.5 * g.w[p] * ix);
    k.ay[p] = T(-0.5 * g.w[p] * iy);
    k.az[p] = T(-0.5 * g.w[p] * iz);
  }
  const int TY = pick_ty(g.nx, g.ny, 512);
  dim3 grid((g.ny + TY - 1) / TY, (Ns + VB - 1) / VB);
  dim3 block(g.nx * TY);
  size_t smem = (size_t)VB * (TY + 2 * R) * (g.nx + 2 * R) * sizeof(T);
  const T* V;
  if constexpr (sizeof(T) == 8) V = reinterpret_cast<const T*>(ctx->V);
  else V = reinterpret_cast<const T*>(ctx->Vf);
  auto kern = cheb_step_kernel<T, R, VB>;
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  kern<<<grid, block, smem, st>>>(g.nx, g.ny, g.nz, Ns, TY, k, y, yprev, out, V, T(s1),
                                  T(c), T(s2));
}

// Vectorised launch when the grid allows it; returns false otherwise.
template <typename T, int R>
static bool launch_vec(const sq3_ctx* ctx, const T* y, const T* yprev, T* out,
                       int Ns, double s1, double c, double s2, cudaStream_t st) {
  constexpr int VW = Vec16<T>::W;
  constexpr int PAD = ((R + VW - 1) / VW) * VW;
  const Grid& g = ctx->grid;
  if (g.nx % VW || g.nx < PAD) return false;
  // 16-byte vector accesses need 16-byte aligned blocks
  if (((uintptr_t)y | (uintptr_t)out | (uintptr_t)(yprev ? yprev : y)) & 15) return false;
  const int TX = g.nx / VW;
  int TY = 0;
  for (int t = 1; t <= g.ny; ++t)
    if (g.ny % t == 0 && TX * t <= 256 && 2 * TX * t >= 2 * R * TX) TY = t;
  if (TY == 0) return false;
  StepCoef<T> k{};
  const double ix = 1.0 / (g.hx * g.hx), iy = 1.0 / (g.hy * g.hy),
               iz = 1.0 / (g.hz * g.hz);
  k.diag = T(-0.5 * g.w[0] * (ix + iy + iz));
  for (int p = 1; p <= R; ++p) {
    k.ax[p] = T(-0.5 * g.w[p] * ix);
    k.ay[p] = T(-0.5 * g.w[p] * iy);
    k.az[p] = T(-0.5 * g.w[p] * iz);
  }
  const T* V;
  if constexpr (sizeof(T) == 8) V = reinterpret_cast<const T*>(ctx->V);
  else V = reinterpret_cast<const T*>(ctx->Vf);
  const int rv = TX + 2 * (PAD / VW);
  if ((TY + 2 * R) * rv <= 4 * TX * TY) {
    constexpr int A = 4;
    const size_t rs = (size_t)(A + 1) *
                      ((size_t)(TY + 2 * R) * ring_row_width<T>(g.nx, PAD) +
                       3 * (size_t)TY * g.nx) *
                      sizeof(T);
    if (rs <= 227 * 1024) {
      auto kr = cheb_step_ring_kernel<T, R, A>;
      if (rs > 48 * 1024)
        cudaFuncSetAttribute(kr, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rs);
      dim3 grid(g.ny / TY, Ns);
      kr<<<grid, TX * TY, rs, st>>>(g.nx, g.ny, g.nz, TY, k, y, yprev, out, V,
                                    T(s1), T(c), T(s2));
      return true;
    }
  }
  size_t smem = (size_t)(TY + 2 * R) * (g.nx + 2 * PAD) * sizeof(T);
  auto kern = cheb_step_vec_kernel<T, R>;
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  dim3 grid(g.ny / TY, Ns);    // the row tiles of one vector run together
  kern<<<grid, TX * TY, smem, st>>>(g.nx, g.ny, g.nz, TY, k, y, yprev, out, V,
                                    T(s1), T(c), T(s2));
  return true;
}

template <typename T, int R>
static void launch_r(const sq3_ctx* ctx, const T* y, const T* yprev, T* out,
                     int Ns, double s1, double c, double s2, cudaStream_t st) {
  if (launch_vec<T, R>(ctx, y, yprev, out, Ns, s1, c, s2, st)) return;
  switch (stencil_vb(sizeof(T))) {
    case 1: launch_rv<T, R, 1>(ctx, y, yprev, out, Ns, s1, c, s2, st); break;
    case 2: launch_rv<T, R, 2>(ctx, y, yprev, out, Ns, s1, c, s2, st); break;
    default: launch_rv<T, R, 4>(ctx, y, yprev, out, Ns, s1, c, s2, st); break;
  }
}

template <typename T>
void launch_cheb_step(const sq3_ctx* ctx, const T* y, const T* yprev, T* out,
                      int Ns, double s1, double c, double s2, cudaStream_t st) {
  switch (ctx->grid.radius) {
    case 1: launch_r<T, 1>(ctx, y, yprev, out, Ns, s1, c, s2, st); break;
    case 2: launch_r<T, 2>(ctx, y, yprev, out, Ns, s1, c, s2, st); break;
    case 3: launch_r<T, 3>(ctx, y, yprev, out, Ns, s1, c, s2, st); break;
    case 4: launch_r<T, 4>(ctx, y, yprev, out, Ns, s1, c, s2, st); break;
    case 5: launch_r<T, 5>(ctx, y, yprev, out, Ns, s1, c, s2, st); break;
    default: launch_r<T, 6>(ctx, y, yprev, out, Ns, s1, c, s2, st); break;
  }
}

// ---------------------------------------------------------------------------
// Nonlocal pass, in place on the output of a local stencil step:
//   out_v[k] += s1 sum_p c_p[k] gC[p][v]                      (apply)
//   gC_next[p][v] += gamma_p sum_k c_p[k] out_v[k]            (projection)
// (gC is projector-major: gC[p * Ns + v].)  A CTA owns one 8 x 8 x NL_BZ
// brick of grid points and a run of vector groups of VB vectors.  The
// projectors are handled per ball: the <= 4 projectors of an atom share its
// points, so one (point, ball) entry carries four values and one load of a
// point's value feeds four projectors.  The brick's entries are staged in
// shared memory once, in two orders (by point for the apply, by ball for
// the projection).  Each group's values, a VB x NL_BZ x 8 x 8 box of the
// block, arrive by one 4-D TMA load into a ring of NBUF buffers (issued
// NBUF groups ahead); the group's coefficients gC arrive by cp.async.
//   phase 1: a lane applies the term to two points for half of the
//            vectors in shared memory and keeps a point-major copy of the
//            results for phase 2; the box goes back to global memory with
//            one TMA store;
//   phase 2: a warp takes a ball, its lanes eight entry slots and four
//            16-byte quarters of the vectors, the slots folded by three
//            shuffle rounds; one atomic per (projector, vector) and ball.
// The box store writes unchanged points back unchanged; elements outside
// the grid or beyond Ns are zero-filled on load and skipped on store.
// ---------------------------------------------------------------------------
struct alignas(16) Dbl4 { double x, y, z, w; };

size_t nl_pass_smem_bytes(int es, int VB, int NBUF, int max_balls, int max_entries) {
  return 128 + (size_t)NBUF * VB * NL_BRICK_PTS * es +
         (size_t)NL_BRICK_PTS * (VB + 16 / es) * es +
         (size_t)NBUF * max_balls * (4 * (VB + 4) + 16 / es) * es +
         (size_t)2 * max_entries * 4 * es +
         (size_t)2 * max_entries * sizeof(short) + 8 + (size_t)NBUF * 8 +
         (size_t)4 * max_balls * (es + sizeof(int)) + (size_t)(max_balls + 1) * sizeof(int);
}

template <typename T, int VB, int NBUF, int MINB>
__global__ void __launch_bounds__(NL_BRICK_PTS, MINB)
nl_brick_kernel(const __grid_constant__ CUtensorMap omap, int nx, int ny, int Ns,
                int groups_per_cta, const T* __restrict__ gC, T* gC_next, T s1,
                const int* __restrict__ ball_ptr, const int* __restrict__ slot_pid,
                const int* __restrict__ pt_ptr, const short* __restrict__ pt_lb,
                const T* __restrict__ pt_val, const int* __restrict__ bl_ptr,
                const short* __restrict__ bl_pt, const T* __restrict__ bl_val,
                const double* __restrict__ gamma, int max_entries, int max_balls,
                int* status) {
  using T4 = typename std::conditional<sizeof(T) == 4, float4, Dbl4>::type;
  constexpr int PTS = NL_BRICK_PTS;
  constexpr int GS = VB + 4;                         // padded row of gloc
  // a ball's four rows, padded by 16 bytes so that the blocks of different
  // balls start on different banks (phase 1 gathers rows of several balls)
  constexpr int BST = 4 * GS + 16 / (int)sizeof(T);
  // the updated values of the current group again, point-major (row of VB
  // values padded by 16 bytes), so phase 2 reads a point with 16-byte loads
  constexpr int YT = VB + 16 / (int)sizeof(T);
  using V16 = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
  constexpr int EV = 16 / (int)sizeof(T);           // elements per 16-byte vector
  constexpr int BOX = VB * PTS;                      // elements of one box
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int b = blockIdx.x;
  const int s0 = ball_ptr[b], nlb = ball_ptr[b + 1] - s0;
  if (nlb == 0) return;                              // brick outside every ball
  const int ngroups = (Ns + VB - 1) / VB;
  const int g0 = blockIdx.y * groups_per_cta;
  const int g1 = min(ngroups, g0 + groups_per_cta);
  if (g0 >= g1) return;
  // TMA boxes start on a 128-byte boundary (the launch adds 128 bytes)
  unsigned char* sbase = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  T* ybuf = reinterpret_cast<T*>(sbase);             // NBUF boxes
  T* ytr = ybuf + NBUF * BOX;                        // PTS x YT: a point's VB values
  T* gloc = ytr + PTS * YT;                          // NBUF x max_balls x BST
  T* qval = gloc + (size_t)NBUF * max_balls * BST;   // point-major values (x4)
  T* zval = qval + (size_t)4 * max_entries;             // ball-major values (x4)
  short* qlb = reinterpret_cast<short*>(zval + (size_t)4 * max_entries);
  short* zpt = qlb + max_entries;
  uint64_t* bars = reinterpret_cast<uint64_t*>(
      (reinterpret_cast<uintptr_t>(zpt + max_entries) + 7) & ~uintptr_t(7));
  // the brick's per-ball metadata, read in every group: projector ids and
  // energies of the ball slots, ball-major entry ranges
  T* s_gam = reinterpret_cast<T*>(bars + NBUF);
  int* s_pid = reinterpret_cast<int*>(s_gam + 4 * max_balls);
  int* s_bptr = s_pid + 4 * max_balls;
  __shared__ int abort_flag;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nbx = (nx + 7) / 8, nby = (ny + 7) / 8;
  const int bx = b % nbx, by = (b / nbx) % nby, bz = b / (nbx * nby);
  const int eb = pt_ptr[b * PTS];
  const int ne = pt_ptr[(b + 1) * PTS] - eb;
  // phase 1 lanes: a pair of points (x, y, z) and (x, y + 2, z) of the
  // warp's 8 x 4 slab, and one half of the group's vectors
  constexpr int VH = VB / 2;
  const int pp = lane & 15, vh = lane >> 4;
  const int p1 = warp * 32 + pp, p2 = p1 + 16;
  const int ea0 = pt_ptr[b * PTS + p1] - eb, ea1 = pt_ptr[b * PTS + p1 + 1] - eb;
  const int eb0 = pt_ptr[b * PTS + p2] - eb, eb1 = pt_ptr[b * PTS + p2 + 1] - eb;
  const int fb = bl_ptr[s0];
  const int nrows = 4 * nlb;
  const uint32_t bar0 = smem_u32(bars);
  for (int i = tid; i < 4 * nlb; i += PTS) {
    const int pid = slot_pid[4 * s0 + i];
    s_pid[i] = pid;
    s_gam[i] = pid >= 0 ? T(gamma[pid]) : T(0);
  }
  for (int i = tid; i <= nlb; i += PTS) s_bptr[i] = bl_ptr[s0 + i] - fb;
  if (tid == 0) {
    abort_flag = 0;
#pragma unroll
    for (int i = 0; i < NBUF; ++i) mbar_init(bar0 + 8 * i, 1);
    mbar_init_fence();
  }
  __syncthreads();
  auto issue_box = [&](int g) {                      // thread 0
    const int bi = (g - g0) % NBUF;
    mbar_expect_tx(bar0 + 8 * bi, BOX * (uint32_t)sizeof(T));
    tma_load_4d(smem_u32(ybuf + bi * BOX), &omap, bar0 + 8 * bi, bx * 8, by * 8,
                bz * NL_BZ, g * VB);
  };
  // gC == nullptr: projection only (no apply, the box is not written back)
  const bool apply = gC != nullptr;
  auto issue_gloc = [&](int g) {                     // all threads, one commit group
    if (apply && g < g1) {
      T* gl = gloc + (size_t)((g - g0) % NBUF) * max_balls * BST;
      for (int i = tid; i < nrows * VB; i += PTS) {
        const int r = i / VB, v = i - r * VB;
        const int vg = g * VB + v;
        const int pid = s_pid[r];
        const bool ok = pid >= 0 && vg < Ns;
        const T* src = gC + (ok ? (long long)pid * Ns + vg : 0);
        cp_async_zfill<(int)sizeof(T)>(gl + (r >> 2) * BST + (r & 3) * GS + v, src,
                                       ok ? (int)sizeof(T) : 0);
      }
    }
    cp_async_commit();
  };
  if (tid == 0)
    for (int g = g0; g < g1 && g < g0 + NBUF; ++g) issue_box(g);
#pragma unroll
  for (int i = 0; i < NBUF; ++i) issue_gloc(g0 + i);
  {
    const T4* qv = reinterpret_cast<const T4*>(pt_val) + eb;
    const T4* zv = reinterpret_cast<const T4*>(bl_val) + fb;
    for (int e = tid; e < ne; e += PTS) {
      reinterpret_cast<T4*>(qval)[e] = qv[e];
      reinterpret_cast<T4*>(zval)[e] = zv[e];
      qlb[e] = pt_lb[eb + e];
      zpt[e] = bl_pt[fb + e];
    }
  }
  int g = g0;
  for (; g < g1; ++g) {
    const int j = g - g0, bi = j % NBUF;
    cp_async_wait<NBUF - 1>();                       // this thread's gloc copies of g
    if (!mbar_wait(bar0 + 8 * bi, (uint32_t)((j / NBUF) & 1))) {
      atomicCAS(status, DEV_OK, DEV_TIMEOUT);
      abort_flag = 1;
    }
    __syncthreads();
    if (abort_flag) break;
    T* yb = ybuf + bi * BOX;
    const T* gl = gloc + (size_t)bi * max_balls * BST;
    // phase 1: apply, four projectors per entry.  A lane sums two points
    // for half of the vectors, so each coefficient row it loads serves both
    // points.  The warp walks the brick's balls in one order (a point's
    // entries are sorted by ball), so the coefficient rows it reads are the
    // same for all lanes of a half (shared-memory broadcasts); balls no lane
    // of the warp touches are skipped.
    {
      T acc1[VH], acc2[VH];
#pragma unroll
      for (int v = 0; v < VH; ++v) acc1[v] = acc2[v] = T(0);
      int ea = ea0, ebb = eb0;
      for (int lb = 0; apply && lb < nlb; ++lb) {
        const bool h1 = ea < ea1 && qlb[ea] == lb;
        const bool h2 = ebb < eb1 && qlb[ebb] == lb;
        if (!__any_sync(0xffffffffu, h1 || h2)) continue;
        T4 c1 = reinterpret_cast<const T4*>(qval)[h1 ? ea : 0];
        T4 c2 = reinterpret_cast<const T4*>(qval)[h2 ? ebb : 0];
        if (!h1) c1.x = c1.y = c1.z = c1.w = T(0);
        if (!h2) c2.x = c2.y = c2.z = c2.w = T(0);
        ea += h1 ? 1 : 0;
        ebb += h2 ? 1 : 0;
        const T* row = gl + lb * BST + vh * VH;
        const T cq1[4] = {c1.x, c1.y, c1.z, c1.w};
        const T cq2[4] = {c2.x, c2.y, c2.z, c2.w};
        // coefficient rows as 16-byte vectors (BST, GS and VH times the
        // element size are multiples of 16, so every piece is 16-byte aligned)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const V16* rq = reinterpret_cast<const V16*>(row + q * GS);
#pragma unroll
          for (int j = 0; j < VH / EV; ++j) {
            const V16 w = rq[j];
            const T* wp = reinterpret_cast<const T*>(&w);
#pragma unroll
            for (int i = 0; i < EV; ++i) {
              acc1[j * EV + i] += cq1[q] * wp[i];
              acc2[j * EV + i] += cq2[q] * wp[i];
            }
          }
        }
      }
      // update and point-major copy; the two halves of the warp take the two
      // points in opposite order, so one access covers 32 distinct banks
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const bool second = (k ^ vh) != 0;
        const int p = second ? p2 : p1;
        if (second ? eb1 > eb0 : ea1 > ea0) {
          T yv[VH];
#pragma unroll
          for (int i = 0; i < VH; ++i) {
            const int v = vh * VH + i;
            yv[i] = yb[v * PTS + p] + s1 * (second ? acc2[i] : acc1[i]);
            if (apply) yb[v * PTS + p] = yv[i];
          }
          V16* yt = reinterpret_cast<V16*>(ytr + p * YT + vh * VH);
#pragma unroll
          for (int j = 0; j < VH / EV; ++j) yt[j] = *reinterpret_cast<const V16*>(yv + j * EV);
        }
      }
    }
    fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0 && apply) {
      tma_store_4d(&omap, smem_u32(yb), bx * 8, by * 8, bz * NL_BZ, g * VB);
      bulk_commit();
    }
    // phase 2: projection of the updated values, one warp per ball (a brick
    // has about 6 balls for 8 warps; halves of balls were measured slower:
    // twice the folds and atomics for the same longest warp).  A lane
    // serves one of NSL entry slots and one 16-byte quarter of the group's
    // vectors: NSL entries are read per step, each slot sums 4 projectors x EV
    // vectors, and the slots are folded at the end (three shuffle rounds).
    if (gC_next != nullptr) {
      constexpr int NQ = VB / EV;                    // 16-byte quarters of a point row
      constexpr int NSL = 32 / NQ;                   // entry slots per warp
      constexpr int NA = 4 * EV;                     // sums per lane
      constexpr int NR = NA / NSL;                   // sums per lane after the fold
      static_assert(NQ == 4 && NR * NSL == NA, "four quarters, eight slots");
      const int qd = lane % NQ, sl = lane / NQ;
      for (int lb = warp; lb < nlb; lb += PTS / 32) {
        const int f0 = s_bptr[lb], f1 = s_bptr[lb + 1];
        T a[NA];
#pragma unroll
        for (int i = 0; i < NA; ++i) a[i] = T(0);
        for (int f = f0 + sl; f < f1; f += NSL) {
          const T4 c = reinterpret_cast<const T4*>(zval)[f];
          const V16 w = reinterpret_cast<const V16*>(ytr + zpt[f] * YT)[qd];
          const T* wp = reinterpret_cast<const T*>(&w);
#pragma unroll
          for (int i = 0; i < EV; ++i) {
            a[i] += c.x * wp[i];
            a[EV + i] += c.y * wp[i];
            a[2 * EV + i] += c.z * wp[i];
            a[3 * EV + i] += c.w * wp[i];
          }
        }
        // fold over the slots (lane bits above the quarter index): after
        // round k a lane keeps the half of its sums selected by its slot bit
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const int m = 16 >> k;
          const int half = NA >> (k + 1);
          const bool up = (lane & m) != 0;
#pragma unroll
          for (int i = 0; i < NA / 2; ++i) {
            if (i < half) {
              const T send = up ? a[i] : a[i + half];
              const T keep = up ? a[i + half] : a[i];
              a[i] = keep + __shfl_xor_sync(0xffffffffu, send, m);
            }
          }
        }
        // the lane now holds the sums of a[sl * NR + i] (projector idx / EV,
        // vector qd * EV + idx % EV)
#pragma unroll
        for (int i = 0; i < NR; ++i) {
          const int idx = sl * NR + i;
          const int q = idx / EV, v = qd * EV + idx % EV;
          const int pid = s_pid[4 * lb + q];
          const int vg = g * VB + v;
          if (pid >= 0 && vg < Ns && a[i] != T(0))
            atomicAdd(gC_next + (long long)pid * Ns + vg, s_gam[4 * lb + q] * a[i]);
        }
      }
    }
    __syncthreads();                                 // box and coefficients consumed
    if (tid == 0 && g + NBUF < g1) {
      bulk_wait_read0();                             // the store has read the box
      issue_box(g + NBUF);
    }
    issue_gloc(g + NBUF);
  }
  // drain: loads still in flight after an abort, then every store
  if (tid == 0) {
    for (int h = g; h < g1 && h < g + NBUF; ++h) {
      const int j = h - g0;
      if (h > g || abort_flag) mbar_wait(bar0 + 8 * (j % NBUF), (uint32_t)((j / NBUF) & 1));
    }
    bulk_wait0();
  }
  cp_async_wait<0>();
}

template <typename T, int VB, int NBUF, int MINB>
static int launch_brick(const sq3_ctx* ctx, T* out, const T* gC, T* gC_next, int Ns,
                        double s1, cudaStream_t st) {
  const Projectors& P = ctx->proj;
  const Grid& g = ctx->grid;
  const size_t es = sizeof(T);
  const size_t smem =
      nl_pass_smem_bytes((int)es, VB, NBUF, P.max_brick_balls, P.max_brick_entries);
  if (smem > 227 * 1024) return SQ3_EINVAL;
  CUtensorMap map;
  const unsigned long long dims[4] = {(unsigned long long)g.nx, (unsigned long long)g.ny,
                                      (unsigned long long)g.nz, (unsigned long long)Ns};
  const unsigned long long strides[3] = {(unsigned long long)g.nx * es,
                                         (unsigned long long)g.nx * g.ny * es,
                                         (unsigned long long)g.N * es};
  const unsigned box[4] = {8, 8, NL_BZ, VB};
  int rc = encode_tensor_map(&map, sizeof(T) == 8, 4, out, dims, strides, box);
  if (rc) return rc;
  const int nb = ((g.nx + 7) / 8) * ((g.ny + 7) / 8) * ((g.nz + NL_BZ - 1) / NL_BZ);
  const int ngroups = (Ns + VB - 1) / VB;
  // runs of groups: several CTAs per SM-slot in total, each run long enough
  // to amortise staging the brick's tables (few groups: runs of up to 8)
  int per = (ngroups + 7) / 8;
  if (ngroups < 32) per = ngroups < 8 ? ngroups : 8;
  const int nruns = (ngroups + per - 1) / per;
  auto kern = nl_brick_kernel<T, VB, NBUF, MINB>;
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const T* qv;
  const T* zv;
  if constexpr (sizeof(T) == 8) {
    qv = reinterpret_cast<const T*>(P.nb_pt_val);
    zv = reinterpret_cast<const T*>(P.nb_bl_val);
  } else {
    qv = reinterpret_cast<const T*>(P.nb_pt_valf);
    zv = reinterpret_cast<const T*>(P.nb_bl_valf);
  }
  kern<<<dim3(nb, nruns), NL_BRICK_PTS, smem, st>>>(
      map, g.nx, g.ny, Ns, per, gC, gC_next, T(s1), P.nb_ball_ptr, P.nb_slot_pid,
      P.nb_pt_ptr, P.nb_pt_lb, qv, P.nb_bl_ptr, P.nb_bl_pt, zv, P.gamma,
      P.max_brick_entries, P.max_brick_balls, ctx->dev_status);
  return SQ3_OK;
}

template <typename T>
int launch_nl_pass(const sq3_ctx* ctx, T* out, const T* gC, T* gC_next, int Ns,
                   double s1, cudaStream_t st) {
  if (ctx->proj.n_proj == 0) return SQ3_OK;
  if ((uintptr_t)out & 15) return SQ3_EINVAL;        // TMA base alignment
  if constexpr (sizeof(T) == 8) return launch_brick<T, 8, 2, 2>(ctx, out, gC, gC_next, Ns, s1, st);
  else return launch_brick<T, 16, 3, 2>(ctx, out, gC, gC_next, Ns, s1, st);
}

template int launch_nl_pass<double>(const sq3_ctx*, double*, const double*, double*, int,
                                    double, cudaStream_t);
template int launch_nl_pass<float>(const sq3_ctx*, float*, const float*, float*, int,
                                   double, cudaStream_t);

template void launch_cheb_step<double>(const sq3_ctx*, const double*, const double*, double*,
                                       int, double, double, double, cudaStream_t);
template void launch_cheb_step<float>(const sq3_ctx*, const float*, const float*, float*, int,
                                      double, double, double, cudaStream_t);

}  // namespace sq3
