// FP64 GEMM with fused epilogues for the plain-FP64 path.
//
// C(m,n) = sum_k A(m,k) B(k,n) on 64 x 64 x 16 tiles, 256 threads, 4 x 4
// outputs per thread, register-prefetched tile loads.  Used for the Gram
// matrix X^T X (Sec. 4, orthonormalisation), X R^{-1}, the projection
// X^T (H X) (Sec. 3, Eq. (DsHsRelation)), the Chebyshev recurrence
// T_{j+1} = 2 Hhat T_j - T_{j-1} with the trace for the moments (Sec. 4,
// Eq. (ThreeTermRecurrenceRelation), Eq. (FermiLevelCalc)) and X Ds with the
// density row-dot (Sec. 3, Eq. (phi_tilde), Eq. (density:NewForm)).
// GB300 has no FP64 tensor-core kind in tcgen05, so this path runs on the
// FP64 FMA pipe.
#include "sq3_internal.cuh"

namespace sq3 {

constexpr int BM = 64, BN = 64, BK = 16;

template <bool AK, bool BKc, int EPI>
__global__ void __launch_bounds__(256)
gemm_f64_kernel(GemmArgs g) {
  __shared__ double As[2][BK][BM + 1];
  __shared__ double Bs[2][BK][BN + 1];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  if (g.tri == 1 && n0 + BN <= m0) return;       // tile strictly below diagonal
  if (g.tri == 3 && n0 >= m0 + BM) return;       // tile strictly above diagonal
  const int Keff = (g.tri == 2) ? min(g.K, n0 + BN) : g.K;
  int kchunk = (Keff + g.splits - 1) / g.splits;
  kchunk = (kchunk + BK - 1) / BK * BK;
  const int kbeg = blockIdx.z * kchunk;
  const int kend = min(Keff, kbeg + kchunk);

  double ra[4], rb[4];
  auto load = [&](int k0) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int m, k;
      if (AK) { k = tid & 15; m = (tid >> 4) + 16 * r; }
      else { m = tid & 63; k = (tid >> 6) + 4 * r; }
      int gm = m0 + m, gk = k0 + k;
      double v = 0.0;
      if (gm < g.M && gk < kend)
        v = AK ? g.A[(long long)gm * g.lda + gk] : g.A[gm + (long long)gk * g.lda];
      ra[r] = v;
      int n, kb;
      if (BKc) { kb = tid & 15; n = (tid >> 4) + 16 * r; }
      else { n = tid & 63; kb = (tid >> 6) + 4 * r; }
      int gn = n0 + n, gkb = k0 + kb;
      double w = 0.0;
      if (gn < g.N && gkb < kend)
        w = BKc ? g.B[gkb + (long long)gn * g.ldb] : g.B[(long long)gkb * g.ldb + gn];
      rb[r] = w;
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int m, k;
      if (AK) { k = tid & 15; m = (tid >> 4) + 16 * r; }
      else { m = tid & 63; k = (tid >> 6) + 4 * r; }
      As[buf][k][m] = ra[r];
      int n, kb;
      if (BKc) { kb = tid & 15; n = (tid >> 4) + 16 * r; }
      else { n = tid & 63; kb = (tid >> 6) + 4 * r; }
      Bs[buf][kb][n] = rb[r];
    }
  };

  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

  if (kbeg < kend) {
    load(kbeg);
    store(0);
    __syncthreads();
    int buf = 0;
    for (int k0 = kbeg; k0 < kend; k0 += BK) {
      const bool more = k0 + BK < kend;
      if (more) load(k0 + BK);
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        double a[4], b[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = As[buf][kk][ty + 16 * i];
#pragma unroll
        for (int j = 0; j < 4; ++j) b[j] = Bs[buf][kk][tx + 16 * j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
      }
      if (more) {
        store(buf ^ 1);
        __syncthreads();
        buf ^= 1;
      }
    }
  }

  if constexpr (EPI == EPI_RHO) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int m = m0 + ty + 16 * i;
      double s = 0.0;
      if (m < g.M) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int n = n0 + tx + 16 * j;
          if (n < g.N) s += g.X[m + (long long)n * g.ldx] * acc[i][j];
        }
      }
      for (int o = 8; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (tx == 0 && m < g.M) atomicAdd(g.rho + m, g.alpha * s);
    }
  } else {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int m = m0 + ty + 16 * i;
      if (m >= g.M) continue;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int n = n0 + tx + 16 * j;
        if (n >= g.N) continue;
        double* c = g.C + m + (long long)n * g.ldc;
        if (EPI == EPI_STORE) {
          double v = g.alpha * acc[i][j];
          if (g.beta != 0.0) v += g.beta * *c;
          *c = v;
        } else if (EPI == EPI_ATOMIC) {
          atomicAdd(c, g.alpha * acc[i][j]);
        } else {  // EPI_CHEB
          const double v = 2.0 * acc[i][j] - g.P[m + (long long)n * g.ldp];
          *c = v;
          if (m == n && g.trace != nullptr) atomicAdd(g.trace, v);
        }
      }
    }
  }
}

template <int EPI>
static void dispatch(const GemmArgs& g, dim3 grid, cudaStream_t st) {
  if (g.a_kcontig) {
    if (g.b_kcontig) gemm_f64_kernel<true, true, EPI><<<grid, 256, 0, st>>>(g);
    else gemm_f64_kernel<true, false, EPI><<<grid, 256, 0, st>>>(g);
  } else {
    if (g.b_kcontig) gemm_f64_kernel<false, true, EPI><<<grid, 256, 0, st>>>(g);
    else gemm_f64_kernel<false, false, EPI><<<grid, 256, 0, st>>>(g);
  }
}

void gemm_f64(const GemmArgs& g0, Epi epi, cudaStream_t st) {
  GemmArgs g = g0;
  if (g.splits < 1) g.splits = 1;
  if (g.M <= 0 || g.N <= 0) return;
  dim3 grid((g.N + BN - 1) / BN, (g.M + BM - 1) / BM, g.splits);
  switch (epi) {
    case EPI_STORE: dispatch<EPI_STORE>(g, grid, st); break;
    case EPI_ATOMIC: dispatch<EPI_ATOMIC>(g, grid, st); break;
    case EPI_CHEB: dispatch<EPI_CHEB>(g, grid, st); break;
    case EPI_RHO: dispatch<EPI_RHO>(g, grid, st); break;
  }
}

}  // namespace sq3
