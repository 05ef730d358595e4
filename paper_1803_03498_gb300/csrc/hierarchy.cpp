// Hierarchy builder: the tuples n in N^M with |n| <= D of Eq. (Nmatrices) and the "+"/"-" links of
// section "HEOM formalism" (arXiv 1803.03498), built with the combinatorial number system.
//
// A tuple of level L is a stars-and-bars word with L stars and M-1 bars; bar j (1-based) sits at
// b_j = (j - 1) + n_1 + ... + n_j.  Inside a level the tuples are numbered by the colexicographic
// rank sum_j C(b_j, j); levels are stacked in increasing L, so u = C(M + L - 1, M) + rank.
// Tuples are generated in rank order by the colex successor of the bar set, and the links by the
// rank of the shifted bars: n + e_l moves bars j >= l up by one, n - e_l moves them down by one.
#include "hierarchy.h"

#include <algorithm>
#include <array>
#include <atomic>
#include <thread>

#include "../../include/heom.h"

namespace heom {

int64_t binom(int a, int b) {
  if (b < 0 || a < 0 || b > a) return 0;
  b = std::min(b, a - b);
  // exact multiplicative formula with __int128 intermediates
  __int128 r = 1;
  for (int i = 1; i <= b; ++i) {
    r = r * (a - b + i) / i;
    if (r > ((__int128)1 << 62)) return -1;
  }
  return (int64_t)r;
}

int host_threads() {
  const unsigned hc = std::thread::hardware_concurrency();
  return (int)std::max(1u, std::min(hc == 0 ? 1u : hc, 32u));
}

int build_hierarchy(int M, int D, Hierarchy *h, std::string *err) {
  if (M < 1 || M > 255 || D < 0 || D > 255) {
    *err = "heom_build_hierarchy: need 1 <= n_modes <= 255 and 0 <= depth <= 255";
    return HEOM_E_ARG;
  }
  int64_t total = binom(M + D, D);
  if (total < 0 || total > INT32_MAX) {
    *err = "heom_build_hierarchy: C(n_modes + depth, depth) exceeds 2^31 - 1 ADOs";
    return HEOM_E_OVERFLOW;
  }
  // binomial table C[a][j] for a <= M + D, j <= M (all <= total, so no overflow)
  const int A = M + D + 1;
  std::vector<int64_t> C((size_t)A * (M + 1), 0);
  for (int a = 0; a < A; ++a)
    for (int j = 0; j <= M && j <= a; ++j) C[(size_t)a * (M + 1) + j] = binom(a, j);
  auto Cb = [&](int a, int j) -> int64_t { return (a < j || a < 0) ? 0 : C[(size_t)a * (M + 1) + j]; };

  try {
    h->M = M;
    h->D = D;
    h->n = total;
    h->level_off.assign(D + 2, 0);
    for (int L = 0; L <= D + 1; ++L) h->level_off[L] = (L == 0) ? 0 : Cb(M + L - 1, M);
    h->tuples.assign((size_t)total * M, 0);
    h->plus.assign((size_t)total * M, -1);
    h->minus.assign((size_t)total * M, -1);
  } catch (...) {
    *err = "heom_build_hierarchy: host allocation failed";
    return HEOM_E_NOMEM;
  }

  const int nb = M - 1;  // number of bars
  // Ranks [r0, r1) of level L: the tuples from their bar positions, and the +/- tables by the rank
  // formula.  Items are independent, so ranges of a level are built on several host threads.
  auto build_range = [&](int L, int64_t r0, int64_t r1) {
    std::vector<int> b(std::max(nb, 1));  // bar positions, 0-based slot j-1 holds b_j
    std::vector<int64_t> pre(M + 1), sup(M + 2), sdn(M + 2);
    // colex unrank of r0: from the top bar down, the largest position x below the bar above with
    // C(x, j) <= the rank left
    int64_t rem = r0;
    int above = L + M - 1;  // one past the largest slot
    for (int j = nb; j >= 1; --j) {
      int x = above - 1;
      while (Cb(x, j) > rem) --x;
      b[j - 1] = x;
      rem -= Cb(x, j);
      above = x;
    }
    for (int64_t r = r0; r < r1; ++r) {
      const int64_t u = h->level_off[L] + r;
      uint8_t *t = &h->tuples[(size_t)u * M];
      // tuple from bars
      if (nb == 0) {
        t[0] = (uint8_t)L;
      } else {
        t[0] = (uint8_t)b[0];
        for (int j = 1; j < nb; ++j) t[j] = (uint8_t)(b[j] - b[j - 1] - 1);
        t[M - 1] = (uint8_t)(L + M - 2 - b[nb - 1]);
      }
      // prefix sums of C(b_j, j) and suffix sums of C(b_j +- 1, j)  (j 1-based)
      pre[0] = 0;
      for (int j = 1; j <= nb; ++j) pre[j] = pre[j - 1] + Cb(b[j - 1], j);
      sup[nb + 1] = 0;
      sdn[nb + 1] = 0;
      for (int j = nb; j >= 1; --j) {
        sup[j] = sup[j + 1] + Cb(b[j - 1] + 1, j);
        sdn[j] = sdn[j + 1] + Cb(b[j - 1] - 1, j);
      }
      for (int l = 1; l <= M; ++l) {  // mode l (1-based) moves bars j >= l
        const int jl = std::min(l, nb + 1);
        if (L + 1 <= D) {
          int64_t rp = pre[jl - 1] + sup[jl];
          h->plus[(size_t)u * M + (l - 1)] = (int32_t)(h->level_off[L + 1] + rp);
        }
        if (t[l - 1] >= 1) {
          int64_t rm = pre[jl - 1] + sdn[jl];
          h->minus[(size_t)u * M + (l - 1)] = (int32_t)(h->level_off[L - 1] + rm);
        }
      }
      // colex successor: raise the lowest bar that can move, reset the ones below it
      if (nb > 0 && r + 1 < r1) {
        int j = 0;
        while (j < nb - 1 && b[j] + 1 == b[j + 1]) ++j;
        ++b[j];
        for (int i = 0; i < j; ++i) b[i] = i;
      }
    }
  };
  // work items: ranges of at most kChunk ranks of one level
  constexpr int64_t kChunk = 1 << 15;
  std::vector<std::array<int64_t, 3>> items;
  for (int L = 0; L <= D; ++L) {
    const int64_t cnt = h->level_off[L + 1] - h->level_off[L];
    for (int64_t r0 = 0; r0 < cnt; r0 += kChunk) items.push_back({L, r0, std::min(cnt, r0 + kChunk)});
  }
  const int nthr = (int)std::min<int64_t>((int64_t)items.size(), host_threads());
  if (nthr <= 1) {
    for (const auto &it : items) build_range((int)it[0], it[1], it[2]);
  } else {
    std::atomic<size_t> next{0};
    std::atomic<bool> failed{false};
    std::vector<std::thread> pool;
    for (int i = 0; i < nthr; ++i)
      pool.emplace_back([&] {
        try {
          for (size_t k = next++; k < items.size(); k = next++) build_range((int)items[k][0], items[k][1], items[k][2]);
        } catch (...) {
          failed = true;
        }
      });
    for (auto &th : pool) th.join();
    if (failed) {
      *err = "heom_build_hierarchy: host allocation failed";
      return HEOM_E_NOMEM;
    }
  }
  // every ADO below depth D has all M "+" links, and "-" links pair with them one to one
  h->n_links = 2 * (int64_t)M * h->level_off[D];
  return HEOM_OK;
}

}  // namespace heom
