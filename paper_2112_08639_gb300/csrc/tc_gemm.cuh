// Interface of the tcgen05 BF16-split GEMM (tc_gemm.cu).
#pragma once

#include <cuda_bf16.h>

#include "sq3_internal.cuh"

namespace sq3 {

// A K-major operand of `pieces` bf16 pieces: element (row r, k, piece q) at
// base[q * piece_stride + r * ld + k].  ld and piece_stride are multiples of
// 8 elements (16 bytes, the TMA stride rule); rows and K may be ragged.
struct Operand {
  const __nv_bfloat16* base;
  int rows, K;
  long long ld, piece_stride;
  int pieces;
};

// Which piece products are summed: A_{a[i]} B_{b[i]}, i < n (n <= 6).
struct Products {
  int n;
  int a[6], b[6];
};

enum { EPI_TC_ATOMIC = 0, EPI_TC_STORE = 1, EPI_TC_CHEB = 2, EPI_TC_RHO = 3 };

struct TcParams {
  int M, N, K;
  int nprod;
  int prod_a[6], prod_b[6];
  int tri;               // 1: upper output tiles only; 2: B upper triangular
  int one_partial;       // 1: the whole K range of a tile in one TMEM accumulator
  int splits;            // K splits (set by tc_gemm)
  int* status;
  // outputs (column-major with leading dimension ldc)
  double* C64;           // EPI_TC_ATOMIC
  float* C32;            // EPI_TC_STORE, EPI_TC_CHEB (T_{j+1})
  long long ldc;
  float alpha;           // EPI_TC_STORE: C = alpha acc (+ beta C, read first,
  float beta;            //   when beta != 0; C may then be updated in place)
  // EPI_TC_CHEB
  const float* Tprev;
  __nv_bfloat16* Bnext;  // pieces of T_{j+1}, row n at Bnext[n*ld_next + m]
  long long ld_next, next_piece_stride;
  int next_pieces;
  double* trace;
  // EPI_TC_STORE, optional: the three BF16 pieces of the stored values in
  // two layouts, colP[q*col_ps + n*col_ld + m] and rowP[q*row_ps + m*row_ld + n]
  __nv_bfloat16* colP;
  long long col_ld, col_ps;
  __nv_bfloat16* rowP;
  long long row_ld, row_ps;
  // EPI_TC_RHO: rho[m] += rho_alpha * sum_n X[m + n*ldx] acc(m, n)
  const float* X;
  long long ldx;
  double* rho;
  double rho_alpha;
};

int tc_gemm(sq3_ctx* ctx, const Operand& A, const Operand& B, const Products& pr,
            TcParams p, int epi, int splits, cudaStream_t st);

}  // namespace sq3
