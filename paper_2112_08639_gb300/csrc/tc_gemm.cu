// tcgen05 (5th-generation tensor core) GEMM on BF16 split operands for the
// mixed-precision path.
//
// Every FP32 operand x is carried as P bf16 pieces, x ~ x_0 + x_1 (+ x_2),
// x_0 = bf16(x), x_1 = bf16(x - x_0), x_2 = bf16(x - x_0 - x_1) (round to
// nearest even).  A product A B is then a short sum of piece products
// sum_(p,q) A_p B_q, each issued as tcgen05.mma kind::f16 with BF16 inputs
// and FP32 accumulation in tensor memory (TMEM).
//
// Tile: 128 x 128 output, K stepped by 64 per shared-memory stage (one
// 128-byte swizzle row of bf16).  Operands are K-major; each stage holds all
// pieces of a 128 x 64 A tile and a 128 x 64 B tile, loaded by one 3-D TMA
// copy per operand with 128-byte swizzle; two stages (three pieces, 96 KB
// each) let the copies of one stage run while the tensor core works on the
// other.  One thread issues the TMA copies and another the MMAs, so a refill
// never waits behind an MMA issue.  The accumulator (128 lanes x 128 FP32
// columns) is read back by sixteen warps with tcgen05.ld (each warp on the
// 32 lanes its index allows) and
// fed to a fused epilogue:
//   EPI_TC_ATOMIC  C(m,n) += acc (FP64 atomics; split-K Gram and X^T (H X))
//   EPI_TC_STORE   C(m,n)  = alpha acc (+ beta C(m,n)) (FP32)
//   EPI_TC_CHEB    T_{j+1} = 2 acc - T_{j-1}; stores T_{j+1} (FP32), its bf16
//                  pieces for the next product, and its trace
//   EPI_TC_RHO     rho(m) += alpha sum_n X(m,n) acc(m,n)   (FP64 atomics)
// Every mbarrier wait is bounded (about one second of wall time); on
// timeout the kernel records DEV_TIMEOUT, drains its outstanding copies with
// the same bound, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include "async_copy.cuh"
#include "sq3_internal.cuh"
#include "tc_gemm.cuh"

namespace sq3 {

namespace tc {

constexpr int BM = 128, BN = 128;
// K per smem stage: one 128-byte swizzle row of bf16.  Measured against
// 64-byte rows (K = 32, four stages): the TMA copies of 128-byte rows move
// twice the bytes per row, and the Gram product ran 1.6x faster with them.
constexpr int BK = 64;
constexpr int ROW_BYTES = BK * 2;                 // bytes of one K row of a tile
constexpr int KPP = 128 / BK;                     // stages per TMEM partial (128 of K)
constexpr int TILE_BYTES = 128 * BK * 2;          // one piece of a 128 x 64 tile
constexpr int SMEM_BUDGET = 196608;               // bytes of tile stages
using namespace ac;

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle (one
// 64-element bf16 row per 128 bytes), 8-row groups 1024 bytes apart (SBO),
// version 1, base offset 0 (tiles start on 1024-byte boundaries).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFF) >> 4);
  d |= (uint64_t)1 << 16;                 // leading byte offset (unused, swizzled K-major)
  d |= (uint64_t)((8 * ROW_BYTES) >> 4) << 32;   // stride byte offset: 8-row groups
  d |= (uint64_t)1 << 46;                 // descriptor version
  d |= (uint64_t)2 << 61;                 // 128-byte swizzle
  return d;
}

// Instruction descriptor, kind::f16: D FP32, A and B BF16, both K-major,
// N = BN, M = BM.
__host__ __device__ constexpr uint32_t idesc_bf16() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
         ((uint32_t)(BM >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b,
                                         uint32_t idesc, uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(accum));
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          bar)
      : "memory");
}

// tcgen05.ld of 8 columns without the wait (pair with tmem_wait_ld)
__device__ __forceinline__ void tmem_ld8_nw(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
        "=r"(r[6]), "=r"(r[7])
      : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_st8(uint32_t taddr, const float* v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr),
      "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
      "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
      "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7]))
      : "memory");
}

__device__ __forceinline__ void tmem_wait_st() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void split_store(float t, __nv_bfloat16* out, long long e,
                                            long long piece_stride, int pieces) {
  __nv_bfloat16 h = __float2bfloat16_rn(t);
  out[e] = h;
  if (pieces > 1) {
    const float r1 = t - __bfloat162float(h);
    const __nv_bfloat16 l = __float2bfloat16_rn(r1);
    out[e + piece_stride] = l;
    if (pieces > 2) out[e + 2 * piece_stride] = __float2bfloat16_rn(r1 - __bfloat162float(l));
  }
}

// The three BF16 pieces of 8 consecutive values of a row (row r of a piece
// array at base + r * ld): one 16-byte store per piece when all 8 are inside
// the row and 16-byte aligned, element stores for the first nvalid otherwise.
__device__ __forceinline__ void store_row_pieces(const float (&v)[8], __nv_bfloat16* base,
                                                 long long piece_stride, int nvalid,
                                                 bool aligned16) {
  if (nvalid >= 8 && aligned16) {
    __align__(16) __nv_bfloat16 pc[3][8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      pc[0][i] = __float2bfloat16_rn(v[i]);
      const float r1 = v[i] - __bfloat162float(pc[0][i]);
      pc[1][i] = __float2bfloat16_rn(r1);
      pc[2][i] = __float2bfloat16_rn(r1 - __bfloat162float(pc[1][i]));
    }
#pragma unroll
    for (int q = 0; q < 3; ++q)
      *reinterpret_cast<uint4*>(base + q * piece_stride) = *reinterpret_cast<const uint4*>(pc[q]);
  } else {
#pragma unroll
    for (int i = 0; i < 8; ++i)
      if (i < nvalid) split_store(v[i], base, i, piece_stride, 3);
  }
}

// Persistent CTAs (one per SM) walk the output tiles t = blockIdx.x +
// i gridDim.x; the TMA producer and the MMA issuer run through the stages
// of successive tiles back to back, so the next tile's copies and MMAs
// overlap the previous tile's epilogue and no CTA launch separates tiles
// (per-CTA timestamps of a one-tile-per-CTA form showed about 25 us between
// one CTA's end and the next CTA's start on an SM).
// Thread roles (576 threads): warp 0 allocates TMEM and its lane 0 issues
// the TMA copies (refilling a stage as soon as its MMAs complete); lane 0 of
// warp 1 issues the MMAs; warps 2..17 accumulate and run the epilogue.  Each
// K-block (KPP stages, 128 of K) of piece products goes into a fresh TMEM
// accumulator (two of them, alternating), so the tensor core never adds into
// a long running sum (unless one_partial: a product whose result is a small
// correction, where the whole K range of a tile goes into one accumulator);
// the accumulation warps add every finished K-block
// partial into a Kahan-compensated FP32 sum that is kept in TMEM as well
// (columns 2 BN .. 4 BN: sum and compensation; an 18-warp CTA has at most
// 96 registers per thread).  Warp w owns lanes 32 (w % 4) .. + 31, the lanes
// it may access, and columns 32 h .. 32 h + 31 with h = (w - 2) / 4.  The
// K-block partial is the sum of at most 8 nprod tensor-core steps started
// from zero, which bounds the accumulation error of the result by about
// that many half-ulps of a K-block partial instead of half an ulp per step
// of the whole K loop.  tcgen05.ld/st are warp-collective (.sync.aligned):
// every condition around them is warp-uniform.
constexpr int ACC_WARPS = 16;
constexpr int THREADS = 64 + 32 * ACC_WARPS;
constexpr int ACC_COLS = BN / (ACC_WARPS / 4);   // columns per accumulation thread
constexpr int STG_BYTES = ACC_WARPS * 32 * ACC_COLS * 2;   // row-piece staging
static_assert(ACC_COLS == 32, "four 16-byte chunks per staged row");

template <int PA, int PB, int EPI>
__global__ void __launch_bounds__(THREADS, 1)
tc_gemm_kernel(const __grid_constant__ CUtensorMap mapA,
               const __grid_constant__ CUtensorMap mapB, TcParams p) {
  constexpr int STAGE_BYTES = (PA + PB) * TILE_BYTES;
  constexpr int STAGES = SMEM_BUDGET / STAGE_BYTES;
  // every K-block partial goes into an FP32 sum in registers; products whose
  // K is a block dimension (Ns: a few tens of partials per tile) use that sum
  // as it is, the split-K Gram products over the grid fold it every GROUPP
  // partials into a Kahan-compensated sum kept in TMEM
  constexpr bool REG = EPI != EPI_TC_ATOMIC;
  constexpr int GROUPP = 16;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // full[s], empty[s] for the smem stages; accf[b], acce[b] for the two
  // TMEM accumulators; done for the MMA issuer's last commit
  __shared__ __align__(8) uint64_t bars[2 * STAGES + 5];
  __shared__ uint32_t tmem_slot;
  __shared__ int failed;
  __shared__ int n_issued, n_consumed;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntN = (p.N + BN - 1) / BN, ntM = (p.M + BM - 1) / BM;
  // tiles of one K split: all of them, or (tri = 1, symmetric output) the
  // upper ones nt >= mt only, enumerated row by row
  const int per_split = (p.tri == 1) ? ntM * (2 * ntN - ntM + 1) / 2 : ntN * ntM;
  const int total = per_split * p.splits;
  // tile t (K split slowest; within it N tile fastest): output corner, K range
  auto decode = [&](int t, int& m0, int& n0, int& kbeg, int& nk) {
    const int kz = t / per_split;
    int u = t - kz * per_split, mt = 0, nt;
    if (p.tri == 1) {
      while (u >= ntN - mt) { u -= ntN - mt; ++mt; }
      nt = mt + u;
    } else {
      nt = u % ntN;
      mt = u / ntN;
    }
    m0 = mt * BM;
    n0 = nt * BN;
    const int Keff = (p.tri == 2) ? min(p.K, n0 + BN) : p.K;
    int kchunk = (Keff + p.splits - 1) / p.splits;
    kchunk = (kchunk + BK - 1) / BK * BK;
    kbeg = kz * kchunk;
    const int kend = min(Keff, kbeg + kchunk);
    nk = (kend > kbeg) ? (kend - kbeg + BK - 1) / BK : 0;
  };

  const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
  const uint32_t full0 = smem_u32(&bars[0]);
  const uint32_t empty0 = smem_u32(&bars[STAGES]);
  const uint32_t accf0 = smem_u32(&bars[2 * STAGES]);
  const uint32_t acce0 = smem_u32(&bars[2 * STAGES + 2]);
  const uint32_t done0 = smem_u32(&bars[2 * STAGES + 4]);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(4 * BN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(accf0 + 8 * b, 1);
      mbar_init(acce0 + 8 * b, ACC_WARPS);
    }
    mbar_init(done0, 1);
    failed = 0;
    n_issued = 0;
    n_consumed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  volatile int* vfailed = &failed;

  if (warp == 0 && lane == 0) {
    // ------------------------------ TMA producer ------------------------------
    // g counts stages over all of this CTA's tiles
    int g = 0;
    for (int t = blockIdx.x; t < total && !*vfailed; t += gridDim.x) {
      int m0, n0, kbeg, nk;
      decode(t, m0, n0, kbeg, nk);
      for (int kb = 0; kb < nk; ++kb, ++g) {
        const int s = g % STAGES;
        if (g >= STAGES && !mbar_wait(empty0 + 8 * s, (uint32_t)(((g / STAGES) - 1) & 1))) {
          atomicExch(&failed, 1);
          atomicCAS(p.status, 0, DEV_TIMEOUT);
          break;
        }
        if (*vfailed) break;
        const uint32_t sa = base + s * STAGE_BYTES;
        const uint32_t fb = full0 + 8 * s;
        mbar_expect_tx(fb, STAGE_BYTES);
        tma_load_3d(sa, &mapA, fb, kbeg + kb * BK, m0, 0);
        tma_load_3d(sa + PA * TILE_BYTES, &mapB, fb, kbeg + kb * BK, n0, 0);
      }
    }
    n_issued = g;
  } else if (warp == 1 && lane == 0) {
    // ------------------------------- MMA issuer -------------------------------
    const uint32_t idesc = idesc_bf16();
    // piece offsets of the products in registers (a dynamically indexed
    // parameter array would be read from local memory on every MMA issue)
    uint32_t offa[6], offb[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      offa[q] = (uint32_t)((q < p.nprod ? p.prod_a[q] : 0) * TILE_BYTES);
      offb[q] = (uint32_t)((q < p.nprod ? p.prod_b[q] : 0) * TILE_BYTES);
    }
    bool ok = true;
    int g = 0, part = 0;        // stages and K-block partials over all tiles
    for (int t = blockIdx.x; t < total && ok; t += gridDim.x) {
      int m0, n0, kbeg, nk;
      decode(t, m0, n0, kbeg, nk);
      for (int kb = 0; kb < nk; ++kb, ++g) {
        const int s = g % STAGES;
        const int buf = part & 1;
        const bool first = p.one_partial ? kb == 0 : (kb % KPP) == 0;
        const bool last = p.one_partial ? kb == nk - 1 : ((kb % KPP) == KPP - 1 || kb == nk - 1);
        // the accumulator used two partials ago must have been drained
        if (first && part >= 2 && !mbar_wait(acce0 + 8 * buf, ((part - 2) >> 1) & 1)) {
          ok = false;
          break;
        }
        if (!mbar_wait(full0 + 8 * s, (g / STAGES) & 1)) { ok = false; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t sa = base + s * STAGE_BYTES;
        const uint32_t sb = sa + PA * TILE_BYTES;
        const uint32_t td = tmem + (uint32_t)(buf * BN);
#pragma unroll
        for (int q = 0; q < 6; ++q) {
          if (q < p.nprod) {
            const uint32_t pa = sa + offa[q];
            const uint32_t pb = sb + offb[q];
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk)
              mma_bf16(td, smem_desc(pa + kk * 32), smem_desc(pb + kk * 32), idesc,
                       (!first || q > 0 || kk > 0) ? 1u : 0u);
          }
        }
        mma_commit(empty0 + 8 * s);      // smem stage free once these MMAs finish
        if (last) {
          mma_commit(accf0 + 8 * buf);   // partial of up to KPP stages ready
          ++part;
        }
      }
      if (*vfailed) ok = false;
    }
    if (!ok) {
      atomicExch(&failed, 1);
      atomicCAS(p.status, 0, DEV_TIMEOUT);
    }
    n_consumed = g;
    // every MMA issued here completes before TMEM is released
    mma_commit(done0);
    mbar_wait(done0, 0);
  } else if (warp >= 2) {
    // -------------------- accumulation and epilogue, per tile --------------------
    const int q4 = warp & 3, half = (warp - 2) >> 2;
    const uint32_t trow = tmem + ((uint32_t)(q4 * 32) << 16);
    const uint32_t tsum = trow + (uint32_t)(2 * BN + half * ACC_COLS);
    const uint32_t tcmp = trow + (uint32_t)(3 * BN + half * ACC_COLS);
    // this warp's staging rows for the row-major pieces (EPI_TC_STORE): 32
    // rows x ACC_COLS bf16 past the tile stages
    __nv_bfloat16* stg = reinterpret_cast<__nv_bfloat16*>(
        smem_raw + (base - smem_u32(smem_raw)) + STAGES * STAGE_BYTES +
        (warp - 2) * 32 * ACC_COLS * 2);
    int part = 0;
    bool alive = true;
    for (int t = blockIdx.x; t < total && alive; t += gridDim.x) {
      int m0, n0, kbeg, nk;
      decode(t, m0, n0, kbeg, nk);
      const int ngrp = p.one_partial ? (nk > 0 ? 1 : 0) : (nk + KPP - 1) / KPP;
      bool have = ngrp > 0;
      float ksum[ACC_COLS];
#pragma unroll
      for (int i = 0; i < ACC_COLS; ++i) ksum[i] = 0.f;
      for (int kg = 0; kg < ngrp; ++kg, ++part) {
        const int buf = part & 1;
        // one verdict per warp: the TMEM accesses below are warp-collective
        const bool landed =
            __all_sync(0xffffffffu, mbar_wait(accf0 + 8 * buf, (part >> 1) & 1));
        if (!landed) {
          have = false;
          alive = false;
          atomicExch(&failed, 1);
          atomicCAS(p.status, 0, DEV_TIMEOUT);
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t ta = trow + (uint32_t)(buf * BN + half * ACC_COLS);
        // the partial into the FP32 register sum, one TMEM load per 8 columns
        // (two chunks in flight per wait)
#pragma unroll
        for (int c = 0; c < ACC_COLS / 8; c += 2) {
          uint32_t rv[2][8];
          tmem_ld8_nw(ta + c * 8, rv[0]);
          tmem_ld8_nw(ta + (c + 1) * 8, rv[1]);
          tmem_wait_ld();
#pragma unroll
          for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int i = 0; i < 8; ++i) ksum[(c + h) * 8 + i] += __uint_as_float(rv[h][i]);
        }
        if (!REG && ((kg + 1) % GROUPP == 0 || kg == ngrp - 1)) {
          // long K: every GROUPP partials the register sum is added into a
          // Kahan-compensated sum kept in TMEM, then restarts from zero
          const bool first_fold = kg < GROUPP;
#pragma unroll
          for (int c = 0; c < ACC_COLS / 8; ++c) {
            float sm[8], cm[8];
            if (first_fold) {
#pragma unroll
              for (int i = 0; i < 8; ++i) {
                sm[i] = ksum[c * 8 + i];
                cm[i] = 0.f;
              }
            } else {
              uint32_t rs[8], rc[8];
              tmem_ld8_nw(tsum + c * 8, rs);
              tmem_ld8_nw(tcmp + c * 8, rc);
              tmem_wait_ld();
#pragma unroll
              for (int i = 0; i < 8; ++i) {
                const float s0 = __uint_as_float(rs[i]);
                const float yk = ksum[c * 8 + i] - __uint_as_float(rc[i]);
                const float tt = s0 + yk;
                cm[i] = (tt - s0) - yk;
                sm[i] = tt;
              }
            }
            tmem_st8(tsum + c * 8, sm);
            tmem_st8(tcmp + c * 8, cm);
#pragma unroll
            for (int i = 0; i < 8; ++i) ksum[c * 8 + i] = 0.f;
          }
          tmem_wait_st();
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0)
          asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(acce0 + 8 * buf)
                       : "memory");
      }
      if (__any_sync(0xffffffffu, *vfailed != 0)) {
        have = false;
        alive = false;
      }
      // epilogue of this tile (the MMAs of the next tile proceed meanwhile);
      // warp-uniform condition around the TMEM loads, rows past M skip only
      // the stores
      const int m = m0 + q4 * 32 + lane;
      const bool mrow = m < p.M;
      double rsum = 0.0;
      // EPI_TC_STORE with beta reads C back: its values are loaded a chunk
      // of 8 columns ahead as independent loads (one at a time between the
      // stores, each waited for a full memory latency; the one-piece
      // correction product of the last Cholesky QR pass took twice as long)
      const bool rdc = EPI == EPI_TC_STORE && p.beta != 0.f;
      float cnext[8];
      auto load_old = [&](int c, float (&o)[8]) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int n = n0 + half * ACC_COLS + c * 8 + i;
          o[i] = (mrow && n < p.N) ? p.C32[(long long)m + (long long)n * p.ldc] : 0.f;
        }
      };
      if (rdc) load_old(0, cnext);
      if (have || EPI == EPI_TC_STORE || EPI == EPI_TC_CHEB) {
#pragma unroll
        for (int c = 0; c < ACC_COLS / 8; ++c) {
          float cold[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) cold[i] = rdc ? cnext[i] : 0.f;
          if (rdc && c + 1 < ACC_COLS / 8) load_old(c + 1, cnext);
          float sm[8], cm[8];
          if (REG) {
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              sm[i] = ksum[c * 8 + i];
              cm[i] = 0.f;
            }
          } else if (have) {
            uint32_t rs[8], rc[8];
            tmem_ld8_nw(tsum + c * 8, rs);
            tmem_ld8_nw(tcmp + c * 8, rc);
            tmem_wait_ld();
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              sm[i] = __uint_as_float(rs[i]);
              cm[i] = __uint_as_float(rc[i]);
            }
          }
          if (!mrow) continue;
          // The FP32 epilogues (REG: cm = 0) compute in FP32: one fma
          // rounds the exact alpha acc + beta C or 2 acc - T_{j-1} once, as
          // the FP64 forms did (the FP64 pipe, a small fraction of the FP32
          // rate on this part, had bound the X R^-1 products); the row-dot
          // adds 8 FP32 products per FP64 addition.
          float tvs[8];
          float rpart = 0.f;
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const int n = n0 + half * ACC_COLS + c * 8 + i;
            tvs[i] = 0.f;
            if (n >= p.N) continue;
            const long long e = (long long)m + (long long)n * p.ldc;
            if (EPI == EPI_TC_ATOMIC) {
              const double acc = have ? (double)sm[i] - (double)cm[i] : 0.0;
              atomicAdd(p.C64 + e, acc);
            } else if (EPI == EPI_TC_STORE) {
              const float acc = have ? sm[i] : 0.f;
              const float v = p.beta != 0.f ? fmaf(p.alpha, acc, p.beta * cold[i])
                                            : p.alpha * acc;
              p.C32[e] = v;
              tvs[i] = v;
              if (p.colP) split_store(v, p.colP, (long long)n * p.col_ld + m, p.col_ps, 3);
            } else if (EPI == EPI_TC_CHEB) {
              const float acc = have ? sm[i] : 0.f;
              const float tv = fmaf(2.f, acc, -p.Tprev[e]);
              tvs[i] = tv;
              p.C32[e] = tv;
              split_store(tv, p.Bnext, (long long)n * p.ld_next + m, p.next_piece_stride,
                          p.next_pieces);
              if (m == n) atomicAdd(p.trace, (double)tv);
            } else {  // EPI_TC_RHO
              const float acc = have ? sm[i] : 0.f;
              rpart = fmaf(p.X[(long long)m + (long long)n * p.ldx], acc, rpart);
            }
          }
          if (EPI == EPI_TC_RHO) rsum += (double)rpart;
          if (EPI == EPI_TC_CHEB && p.tri == 1 && n0 != m0) {
            // symmetric T_{j+1} from its upper tiles: the mirror of an
            // off-diagonal tile, row m of it holding this lane's 8 columns
            const int nb = n0 + half * ACC_COLS + c * 8;
            float* cm32 = p.C32 + (long long)m * p.ldc + nb;
            if (nb + 8 <= p.N && (p.ldc & 3) == 0) {
              reinterpret_cast<float4*>(cm32)[0] = make_float4(tvs[0], tvs[1], tvs[2], tvs[3]);
              reinterpret_cast<float4*>(cm32)[1] = make_float4(tvs[4], tvs[5], tvs[6], tvs[7]);
            } else {
#pragma unroll
              for (int i = 0; i < 8; ++i)
                if (nb + i < p.N) cm32[i] = tvs[i];
            }
            store_row_pieces(tvs, p.Bnext + (long long)m * p.ld_next + nb, p.next_piece_stride,
                             p.N - nb, (p.ld_next & 7) == 0);
          }
          if (EPI == EPI_TC_STORE) {
#pragma unroll
            for (int i = 0; i < 8; ++i) ksum[c * 8 + i] = tvs[i];   // kept for the row pieces
          }
        }
      }
      if (EPI == EPI_TC_STORE && p.rowP) {
        // The pieces of the tile's rows, row-major: a lane's 32 values (its
        // row, this warp's columns) go to the warp's staging rows in shared
        // memory (16-byte chunks swizzled by row, conflict-free both ways),
        // then four lanes store one row's 64 bytes, so every store writes 8
        // rows x 64 contiguous bytes instead of 32 rows x 16.  Piece q is
        // bf16 of what pieces 0 .. q-1 left (ksum keeps the rest).
        const int nb0 = n0 + half * ACC_COLS;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
#pragma unroll
          for (int c = 0; c < ACC_COLS / 8; ++c) {
            __align__(16) __nv_bfloat16 pc[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              const float x = ksum[c * 8 + i];
              pc[i] = __float2bfloat16_rn(x);
              ksum[c * 8 + i] = x - __bfloat162float(pc[i]);
            }
            *reinterpret_cast<uint4*>(stg + lane * ACC_COLS + 8 * (c ^ ((lane >> 1) & 3))) =
                *reinterpret_cast<const uint4*>(pc);
          }
          __syncwarp();
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const int r = 8 * i + (lane >> 2), cc = lane & 3;
            const int mr = m0 + q4 * 32 + r, nb = nb0 + cc * 8;
            const uint4 val =
                *reinterpret_cast<const uint4*>(stg + r * ACC_COLS + 8 * (cc ^ ((r >> 1) & 3)));
            if (mr < p.M && nb < p.N) {
              __nv_bfloat16* dst = p.rowP + q * p.row_ps + (long long)mr * p.row_ld + nb;
              if (nb + 8 <= p.N && (p.row_ld & 7) == 0) {
                *reinterpret_cast<uint4*>(dst) = val;
              } else {
                const __nv_bfloat16* e = reinterpret_cast<const __nv_bfloat16*>(&val);
#pragma unroll
                for (int k = 0; k < 8; ++k)
                  if (nb + k < p.N) dst[k] = e[k];
              }
            }
          }
          __syncwarp();
        }
      }
      if (EPI == EPI_TC_RHO && have && mrow) atomicAdd(p.rho + m, p.rho_alpha * rsum);
    }
  }

  __syncthreads();
  if (failed && threadIdx.x == 0) {
    // copies issued but never consumed: wait (bounded) until they land
    for (int g = n_consumed; g < n_issued; ++g)
      mbar_wait(full0 + 8 * (g % STAGES), (g / STAGES) & 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(4 * BN));
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion,
                                  CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                         cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  }
  return fn;
}

static int make_map(CUtensorMap* map, const Operand& o, int box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return SQ3_ECUDA;
  if (((uintptr_t)o.base & 15) || (o.ld * 2) % 16 || (o.piece_stride * 2) % 16)
    return SQ3_EINVAL;
  cuuint64_t dims[3] = {(cuuint64_t)o.K, (cuuint64_t)o.rows, (cuuint64_t)o.pieces};
  cuuint64_t strides[2] = {(cuuint64_t)o.ld * 2, (cuuint64_t)o.piece_stride * 2};
  cuuint32_t box[3] = {(cuuint32_t)BK, (cuuint32_t)box_rows, (cuuint32_t)o.pieces};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, (void*)o.base, dims, strides,
                  box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? SQ3_OK : SQ3_ECUDA;
}

}  // namespace tc

int encode_tensor_map(CUtensorMap* map, bool fp64, int rank, void* base,
                      const unsigned long long* dims, const unsigned long long* strides,
                      const unsigned* box) {
  tc::EncodeTiledFn fn = tc::encode_fn();
  if (!fn) return SQ3_ECUDA;
  if (rank < 1 || rank > 5 || ((uintptr_t)base & 15)) return SQ3_EINVAL;
  cuuint64_t d[5], st[4];
  cuuint32_t bx[5], es[5];
  for (int i = 0; i < rank; ++i) {
    d[i] = dims[i];
    bx[i] = box[i];
    es[i] = 1;
  }
  for (int i = 0; i + 1 < rank; ++i) {
    if (strides[i] % 16) return SQ3_EINVAL;
    st[i] = strides[i];
  }
  CUresult r = fn(map, fp64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                  (cuuint32_t)rank, base, d, st, bx, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? SQ3_OK : SQ3_ECUDA;
}

namespace tc {

template <int PA, int PB, int EPI>
static int launch_t(const CUtensorMap& a, const CUtensorMap& b, const TcParams& p,
                    dim3 grid, cudaStream_t st) {
  constexpr int STAGE_BYTES = (PA + PB) * TILE_BYTES;
  constexpr int STAGES = SMEM_BUDGET / STAGE_BYTES;
  // + the accumulation warps' staging rows of EPI_TC_STORE
  const int smem = STAGES * STAGE_BYTES + 1024 + (EPI == EPI_TC_STORE ? STG_BYTES : 0);
  auto k = tc_gemm_kernel<PA, PB, EPI>;
  // per launch (about a microsecond), so that every device the process uses
  // has the attribute set
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
    return SQ3_ECUDA;
  k<<<grid, THREADS, smem, st>>>(a, b, p);
  return cuda_err(cudaGetLastError());
}

template <int EPI>
static int launch_e(int PA, int PB, const CUtensorMap& a, const CUtensorMap& b,
                    const TcParams& p, dim3 grid, cudaStream_t st) {
  if constexpr (EPI == EPI_TC_STORE || EPI == EPI_TC_ATOMIC)
    if (PA == 1 && PB == 1) return launch_t<1, 1, EPI>(a, b, p, grid, st);
  if (PA == 2 && PB == 2) return launch_t<2, 2, EPI>(a, b, p, grid, st);
  if (PA == 3 && PB == 3) return launch_t<3, 3, EPI>(a, b, p, grid, st);
  return SQ3_EINVAL;
}

}  // namespace tc

int tc_gemm(sq3_ctx* ctx, const Operand& A, const Operand& B, const Products& pr,
            TcParams p, int epi, int splits, cudaStream_t st) {
  using namespace tc;
  if (A.K != B.K || A.pieces != B.pieces || pr.n < 1 || pr.n > 6) return SQ3_EINVAL;
  for (int i = 0; i < pr.n; ++i) {
    if (pr.a[i] >= A.pieces || pr.b[i] >= B.pieces) return SQ3_EINVAL;
    p.prod_a[i] = pr.a[i];
    p.prod_b[i] = pr.b[i];
  }
  p.nprod = pr.n;
  p.M = A.rows;
  p.N = B.rows;
  p.K = A.K;
  p.status = ctx->dev_status;
  CUtensorMap ma, mb;
  int rc = make_map(&ma, A, BM);
  if (rc) return rc;
  rc = make_map(&mb, B, BN);
  if (rc) return rc;
  if (splits < 1) splits = 1;
  p.splits = splits;
  // persistent CTAs, one per SM, each walking tiles t = blockIdx.x + i gridDim.x
  const long long tN = (p.N + BN - 1) / BN, tM = (p.M + BM - 1) / BM;
  if (p.tri == 1 && tN < tM) return SQ3_EINVAL;   // upper tiles need N >= M
  const long long tiles = (p.tri == 1 ? tM * (2 * tN - tM + 1) / 2 : tN * tM) * splits;
  if (tiles > (1LL << 30)) return SQ3_EINVAL;
  int dev = 0, sms = 0;                            // the current device's SM count
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      sms < 1) {
    cudaGetLastError();
    sms = 152;
  }
  dim3 grid((unsigned)(tiles < sms ? tiles : sms));
  switch (epi) {
    case EPI_TC_ATOMIC: return launch_e<EPI_TC_ATOMIC>(A.pieces, B.pieces, ma, mb, p, grid, st);
    case EPI_TC_STORE: return launch_e<EPI_TC_STORE>(A.pieces, B.pieces, ma, mb, p, grid, st);
    case EPI_TC_CHEB: return launch_e<EPI_TC_CHEB>(A.pieces, B.pieces, ma, mb, p, grid, st);
    case EPI_TC_RHO: return launch_e<EPI_TC_RHO>(A.pieces, B.pieces, ma, mb, p, grid, st);
  }
  return SQ3_EINVAL;
}

}  // namespace sq3
