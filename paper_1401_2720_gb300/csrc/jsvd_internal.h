// Internal declarations shared by the library's translation units.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace jsvd {

// Block p-strategy tables (Sec. 3).  Pairs are 0-based, p < q, stored
// p-step by p-step: out[2*(s*(n/2)+i)] = p, out[2*(s*(n/2)+i)+1] = q.
// Returns 0, or a JSVD_* status / -2 for an order the family cannot build.
int build_pstrategy(int strategy, int n, std::vector<int> &out);

// Smallest even order >= n that build_pstrategy accepts for `strategy`.
int admissible_order(int strategy, int n);

}  // namespace jsvd
