// Host-side tables of the Kleinman-Bylander projectors (Sec. 2, Eq.
// (nonlocaloperator): V_nl = sum_p gamma_p c_p c_p^T): the projectors grouped
// into balls (the lm components of one atom share their grid points), the
// per-brick tables of the nonlocal pass, and Gershgorin bounds of V_nl.  No
// device work happens here; sq3_set_projectors uploads the result.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <thread>
#include <vector>

#include "sq3_internal.cuh"

namespace sq3 {

// Host threads for the table loops (at most 16).
static int table_threads() {
  return std::max(1, std::min((int)std::thread::hardware_concurrency(), 16));
}

// f(i, w) for i in [0, n) on table_threads() host threads, in chunks taken
// from a shared counter; w < table_threads() numbers the worker, so f may use
// scratch indexed by w.  f writes only state owned by i or by w.
template <typename F>
static void parallel_for(long long n, long long chunk, F f) {
  const int nt = (int)std::min<long long>(table_threads(), (n + chunk - 1) / chunk);
  std::atomic<long long> next(0);
  auto work = [&](int w) {
    for (;;) {
      const long long i0 = next.fetch_add(chunk);
      if (i0 >= n) return;
      const long long i1 = std::min(n, i0 + chunk);
      for (long long i = i0; i < i1; ++i) f(i, w);
    }
  };
  if (nt <= 1) { work(0); return; }
  std::vector<std::thread> pool;
  for (int t = 1; t < nt; ++t) pool.emplace_back(work, t);
  work(0);
  for (auto& th : pool) th.join();
}

void projector_host_tables(int nx, int ny, int nz, double dV, int n_proj, const int* ptr,
                           const int* idx, const double* val, const double* gamma,
                           ProjectorHostTables& T) {
  const long long N = (long long)nx * ny * nz;
  // canonical lists: each projector's indices ascending, a repeated index
  // merged into one entry whose value is the sum (the operator is the same;
  // the nonlocal pass takes at most one entry per point and ball)
  std::vector<int> cptr_v, cidx_v;
  std::vector<double> cval_v;
  {
    bool canonical = true;
    for (int p = 0; p < n_proj && canonical; ++p)
      for (int e = ptr[p] + 1; e < ptr[p + 1]; ++e)
        if (idx[e] <= idx[e - 1]) { canonical = false; break; }
    if (!canonical) {
      cptr_v.assign(1, 0);
      std::vector<std::pair<int, double>> ent;
      for (int p = 0; p < n_proj; ++p) {
        ent.clear();
        for (int e = ptr[p]; e < ptr[p + 1]; ++e) ent.push_back({idx[e], val[e]});
        std::stable_sort(ent.begin(), ent.end(),
                         [](const std::pair<int, double>& u, const std::pair<int, double>& w) {
                           return u.first < w.first;
                         });
        for (size_t i = 0; i < ent.size(); ++i) {
          if (i > 0 && ent[i].first == ent[i - 1].first) cval_v.back() += ent[i].second;
          else { cidx_v.push_back(ent[i].first); cval_v.push_back(ent[i].second); }
        }
        cptr_v.push_back((int)cidx_v.size());
      }
      ptr = cptr_v.data();
      idx = cidx_v.data();
      val = cval_v.data();
    }
  }
  const double sq = sqrt(dV);
  // balls: runs of consecutive projectors (<= 4) with identical index lists
  std::vector<int>& bptr = T.bptr;
  std::vector<int>& bidx = T.bidx;
  std::vector<int>& bp0 = T.bp0;
  std::vector<int>& bnp = T.bnp;
  std::vector<int>& boff = T.boff;
  std::vector<double>& bval = T.bval;
  bptr.assign(1, 0);
  bidx.clear(); bp0.clear(); bnp.clear(); boff.clear(); bval.clear();
  bidx.reserve(ptr[n_proj]);
  bval.reserve(ptr[n_proj]);
  for (int p = 0; p < n_proj;) {
    int q = p + 1;
    const int len = ptr[p + 1] - ptr[p];
    while (q < n_proj && q - p < 4 && ptr[q + 1] - ptr[q] == len &&
           memcmp(idx + ptr[q], idx + ptr[p], sizeof(int) * len) == 0)
      ++q;
    bp0.push_back(p);
    bnp.push_back(q - p);
    boff.push_back((int)bval.size());
    bidx.insert(bidx.end(), idx + ptr[p], idx + ptr[p] + len);
    for (int r = p; r < q; ++r)
      for (int e = 0; e < len; ++e) bval.push_back(val[ptr[r] + e] * sq);
    bptr.push_back((int)bidx.size());
    p = q;
  }
  const int nballs = (int)bp0.size();
  const int nent = bptr[nballs];
  // point -> (ball, position in the ball's point list), balls ascending
  std::vector<int> kptr(N + 1, 0);
  for (int e = 0; e < nent; ++e) kptr[bidx[e] + 1]++;
  for (long long k = 0; k < N; ++k) kptr[k + 1] += kptr[k];
  std::vector<int> kball(nent), kpos(nent);
  {
    std::vector<int> kfill(kptr.begin(), kptr.end() - 1);
    for (int B = 0; B < nballs; ++B)
      for (int e = bptr[B]; e < bptr[B + 1]; ++e) {
        const int k = bidx[e];
        kball[kfill[k]] = B;
        kpos[kfill[k]] = e - bptr[B];
        kfill[k]++;
      }
  }
  auto ball_val4 = [&](int B, int pos, double* v4) {
    const int len = bptr[B + 1] - bptr[B];
    for (int q = 0; q < 4; ++q)
      v4[q] = (q < bnp[B]) ? bval[(size_t)boff[B] + (size_t)q * len + pos] : 0.0;
  };
  // Gershgorin bounds of V_nl: its nonzero eigenvalues are those of
  // Gamma S, S_pq = c_p . c_q the overlaps of the projectors.  Row block B
  // of S is summed over B's points, against every ball sharing the point;
  // `where` maps a neighbouring ball to its slot in the row block.
  {
    std::vector<double> blo(nballs, 0.0), bhi(nballs, 0.0);
    std::vector<std::vector<int>> where_w(table_threads());
    parallel_for(nballs, 4, [&](long long Bl, int w) {
      std::vector<int>& where = where_w[w];
      if ((int)where.size() != nballs) where.assign(nballs, -1);
      const int B = (int)Bl;
      std::vector<int> nbrs;
      std::vector<std::array<double, 16>> blk;
      double v4a[4], v4b[4];
      for (int e = bptr[B]; e < bptr[B + 1]; ++e) {
        const int k = bidx[e];
        ball_val4(B, e - bptr[B], v4a);
        for (int j = kptr[k]; j < kptr[k + 1]; ++j) {
          const int C = kball[j];
          int s = where[C];
          if (s < 0) {
            s = where[C] = (int)nbrs.size();
            nbrs.push_back(C);
            blk.push_back({});
          }
          ball_val4(C, kpos[j], v4b);
          double* o = blk[s].data();
          for (int q = 0; q < 4; ++q)
            for (int r = 0; r < 4; ++r) o[4 * q + r] += v4a[q] * v4b[r];
        }
      }
      double lo = 0.0, hi = 0.0;
      for (int q = 0; q < bnp[B]; ++q) {
        const int pq = bp0[B] + q;
        double diag = 0.0, rad = 0.0;
        for (size_t s = 0; s < nbrs.size(); ++s)
          for (int r = 0; r < bnp[nbrs[s]]; ++r) {
            const double v = gamma[pq] * blk[s][4 * q + r];
            if (nbrs[s] == B && r == q) diag = v;
            else rad += fabs(v);
          }
        lo = std::min(lo, diag - rad);
        hi = std::max(hi, diag + rad);
      }
      for (int C : nbrs) where[C] = -1;
      blo[B] = lo;
      bhi[B] = hi;
    });
    T.vnl_lo = *std::min_element(blo.begin(), blo.end());
    T.vnl_hi = *std::max_element(bhi.begin(), bhi.end());
  }
  // brick tables of the nonlocal pass (8 x 8 x NL_BZ bricks, x fastest)
  const int nbx = (nx + 7) / 8, nby = (ny + 7) / 8, nbz = (nz + NL_BZ - 1) / NL_BZ;
  const long long nb = (long long)nbx * nby * nbz;
  auto brick_point = [&](long long b, int t) -> long long {
    const int bx = (int)(b % nbx), by = (int)((b / nbx) % nby),
              bz = (int)(b / ((long long)nbx * nby));
    const int ix = bx * 8 + (t & 7), iy = by * 8 + ((t >> 3) & 7), iz = bz * NL_BZ + (t >> 6);
    if (ix >= nx || iy >= ny || iz >= nz) return -1;
    return (long long)ix + (long long)nx * (iy + (long long)ny * iz);
  };
  // pass 1: each brick's balls (ascending) and number of entries
  std::vector<std::vector<int>> bids(nb);
  std::vector<int> bne(nb);
  parallel_for(nb, 8, [&](long long b, int) {
    std::vector<int>& ids = bids[b];
    int ne = 0;
    for (int t = 0; t < NL_BRICK_PTS; ++t) {
      const long long k = brick_point(b, t);
      if (k < 0) continue;
      ne += kptr[k + 1] - kptr[k];
      for (int j = kptr[k]; j < kptr[k + 1]; ++j) ids.push_back(kball[j]);
    }
    std::sort(ids.begin(), ids.end());
    ids.erase(std::unique(ids.begin(), ids.end()), ids.end());
    bne[b] = ne;
  });
  // offsets of each brick's entries and ball slots
  std::vector<long long> eoff(nb + 1, 0), soff(nb + 1, 0);
  int maxb = 0, maxe = 0;
  for (long long b = 0; b < nb; ++b) {
    eoff[b + 1] = eoff[b] + bne[b];
    soff[b + 1] = soff[b] + (long long)bids[b].size();
    maxb = std::max(maxb, (int)bids[b].size());
    maxe = std::max(maxe, bne[b]);
  }
  const long long ntot = eoff[nb], nslots = soff[nb];
  T.qptr.assign((size_t)nb * NL_BRICK_PTS + 1, 0);
  T.qlb.assign(ntot, 0);
  T.qval.assign((size_t)4 * ntot, 0.0);
  T.zpt.assign(ntot, 0);
  T.zval.assign((size_t)4 * ntot, 0.0);
  T.spid.assign((size_t)4 * nslots, -1);
  T.zptr.assign(nslots + 1, 0);
  T.sptr.assign(nb + 1, 0);
  for (long long b = 0; b <= nb; ++b) T.sptr[b] = (int)soff[b];
  // pass 2: fill each brick's range.  Point-major entries: a point's
  // entries in ascending ball order (kball is filled ball by ball), which the
  // apply's walk over the balls relies on; ball-major entries: per local
  // ball, its points in ascending order (a counting sort of the same entries)
  parallel_for(nb, 8, [&](long long b, int) {
    const std::vector<int>& ids = bids[b];
    const int nl = (int)ids.size();
    auto local = [&](int B) {
      return (int)(std::lower_bound(ids.begin(), ids.end(), B) - ids.begin());
    };
    std::vector<int> lcount(nl, 0);
    long long e = eoff[b];
    for (int t = 0; t < NL_BRICK_PTS; ++t) {
      const long long k = brick_point(b, t);
      if (k >= 0)
        for (int j = kptr[k]; j < kptr[k + 1]; ++j, ++e) {
          const int lb = local(kball[j]);
          T.qlb[e] = (short)lb;
          ball_val4(kball[j], kpos[j], &T.qval[(size_t)4 * e]);
          lcount[lb]++;
        }
      T.qptr[(size_t)b * NL_BRICK_PTS + t + 1] = (int)e;
    }
    std::vector<long long> fill(nl + 1, eoff[b]);
    for (int l = 0; l < nl; ++l) fill[l + 1] = fill[l] + lcount[l];
    for (int l = 0; l < nl; ++l) {
      const int B = ids[l];
      const long long s = soff[b] + l;
      for (int q = 0; q < 4; ++q) T.spid[(size_t)4 * s + q] = q < bnp[B] ? bp0[B] + q : -1;
      T.zptr[s + 1] = (int)fill[l + 1];
    }
    for (int t = 0; t < NL_BRICK_PTS; ++t) {
      const long long k = brick_point(b, t);
      if (k < 0) continue;
      for (int j = kptr[k]; j < kptr[k + 1]; ++j) {
        const long long f = fill[local(kball[j])]++;
        T.zpt[f] = (short)t;
        ball_val4(kball[j], kpos[j], &T.zval[(size_t)4 * f]);
      }
    }
  });
  T.max_brick_balls = maxb;
  T.max_brick_entries = maxe;
}

}  // namespace sq3
