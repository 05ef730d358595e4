// Host-side HEOM hierarchy: multi-indices with |n| <= D, their numbering and +/- links.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace heom {

struct Hierarchy {
  int M = 0;                       // modes (the paper's W = B * K)
  int D = 0;                       // depth
  int64_t n = 0;                   // C(M + D, D)
  std::vector<int64_t> level_off;  // [D + 2], first u of each level, then n
  std::vector<uint8_t> tuples;     // [n][M]
  std::vector<int32_t> plus;       // [n][M], -1 if |n| = D
  std::vector<int32_t> minus;      // [n][M], -1 if n_l = 0
  int64_t n_links = 0;             // valid entries of plus and minus together
};

// Returns 0 or a negative HEOM_E_* code with *err filled.
int build_hierarchy(int M, int D, Hierarchy *h, std::string *err);

// Host threads for the parallel loops of the builder and of run set-up (hardware threads, at most 32).
int host_threads();

// C(a, b) with overflow detection (returns -1 when above 2^62).
int64_t binom(int a, int b);

}  // namespace heom
