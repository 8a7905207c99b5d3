// Parallel pivot strategies (Sec. 3 of the paper) for the block level and the
// inner level of the sweep.  Host code, run once per (strategy, order) and
// cached by the caller.
//
//   modulus   Sameh's modulus ordering of odd order N = n-1, completed to
//             even order by pairing the index idle in p-step s with index N.
//   R|| / C|| the p-strategy closest (Def. 3.1) to the row- / column-cyclic
//             order: for n = 2^k * o (o odd) the closest p-strategy of order
//             2o is found by a lexicographic depth-first search over perfect
//             matchings with backtracking (Alg. 3.1), and then doubled k-1
//             times by the block expansion of Alg. 3.2.
//   reverse   the sweep's pair sequence read backwards.
#include <algorithm>
#include <cstdint>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "jsvd.h"
#include "jsvd_internal.h"

namespace jsvd {
namespace {

using Step = std::vector<std::pair<int, int>>;
using Strat = std::vector<Step>;

constexpr int kMaxSearchOrder = 24;  // largest order 2o searched by Alg. 3.1

Strat modulus_strategy(int n) {
    const int N = n - 1;  // odd
    Strat st(N);
    for (int s = 0; s < N; ++s) {
        Step step;
        for (int i = 0; i < N; ++i) {
            int j = ((s - i) % N + N) % N;  // i + j == s (mod N)
            if (i < j) step.emplace_back(i, j);
            else if (i == j) step.emplace_back(i, N);  // the idle index meets N
        }
        std::sort(step.begin(), step.end());
        st[s] = std::move(step);
    }
    return st;
}

// Alg. 3.1 at a small even order n: vertices are positions in the sequential
// order; a p-step is a set of n/2 pairwise disjoint unused pairs, tried in
// increasing lexicographic order of its sorted positions.
class ClosestSearch {
  public:
    ClosestSearch(bool row, int n) : n_(n), t_(n / 2) {
        if (row) {
            for (int i = 0; i < n; ++i)
                for (int j = i + 1; j < n; ++j) seq_.emplace_back(i, j);
        } else {
            for (int j = 1; j < n; ++j)
                for (int i = 0; i < j; ++i) seq_.emplace_back(i, j);
        }
        used_.assign(seq_.size(), 0);
    }

    bool run(Strat &out) {
        steps_.clear();
        if (!next_step(0)) return false;
        out.clear();
        for (auto &s : steps_) {
            Step st;
            for (int pos : s) st.push_back(seq_[pos]);
            out.push_back(st);
        }
        return true;
    }

  private:
    // Place p-step number `depth`; true once all n-1 p-steps are placed.
    bool next_step(int depth) {
        if (depth == n_ - 1) return true;
        std::vector<int> chosen;
        chosen.reserve(t_);
        return extend(depth, 0, 0u, chosen);
    }

    // Every index not in `covered` must still be reachable by some unused
    // pair at a position >= start whose other end is also uncovered.
    bool coverable(int start, uint32_t covered) const {
        const uint32_t all = (n_ == 32) ? 0xffffffffu : ((1u << n_) - 1u);
        uint32_t need = all & ~covered, reach = 0;
        if (!need) return true;
        for (size_t pos = start; pos < seq_.size(); ++pos) {
            if (used_[pos]) continue;
            uint32_t a = 1u << seq_[pos].first, b = 1u << seq_[pos].second;
            if ((covered & a) || (covered & b)) continue;
            reach |= a | b;
            if ((reach & need) == need) return true;
        }
        return false;
    }

    bool extend(int depth, int start, uint32_t covered, std::vector<int> &chosen) {
        if ((int)chosen.size() == t_) {
            for (int pos : chosen) used_[pos] = 1;
            steps_.push_back(chosen);
            if (next_step(depth + 1)) return true;
            steps_.pop_back();
            for (int pos : chosen) used_[pos] = 0;
            return false;
        }
        for (size_t pos = start; pos < seq_.size(); ++pos) {
            if (used_[pos]) continue;
            uint32_t a = 1u << seq_[pos].first, b = 1u << seq_[pos].second;
            if ((covered & a) || (covered & b)) continue;
            chosen.push_back((int)pos);
            if (coverable((int)pos + 1, covered | a | b) &&
                extend(depth, (int)pos + 1, covered | a | b, chosen))
                return true;
            chosen.pop_back();
        }
        return false;
    }

    int n_, t_;
    std::vector<std::pair<int, int>> seq_;
    std::vector<char> used_;
    std::vector<std::vector<int>> steps_;
};

// Alg. 3.2: order n -> order 2n.
Strat expand(const Strat &in, bool row) {
    const int n = (int)in.size() + 1;
    Strat out;
    Step first;
    for (int k = 0; k < n; ++k) first.emplace_back(2 * k, 2 * k + 1);
    out.push_back(first);
    for (int i = 2; i <= 2 * n - 1; ++i) {
        const Step &src = in[i / 2 - 1];
        Step st;
        for (auto [p, q] : src) {
            if (i % 2 == 0) {
                st.emplace_back(2 * p, 2 * q);          // NW
                st.emplace_back(2 * p + 1, 2 * q + 1);  // SE
            } else {
                std::pair<int, int> ne(2 * p, 2 * q + 1), sw(2 * p + 1, 2 * q);
                if (row) { st.push_back(ne); st.push_back(sw); }
                else     { st.push_back(sw); st.push_back(ne); }
            }
        }
        out.push_back(st);
    }
    return out;
}

int odd_part(int n, int *twos) {
    int k = 0;
    while (n % 2 == 0 && n > 0) { n /= 2; ++k; }
    if (twos) *twos = k;
    return n;
}

std::mutex g_mu;
std::map<std::pair<int, int>, Strat> g_base;  // (row?, 2o) -> closest strategy

bool closest(bool row, int n, Strat &out) {
    int k = 0;
    int o = odd_part(n, &k);
    int base = 2 * o;
    if (base > kMaxSearchOrder) return false;
    Strat s;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto key = std::make_pair(row ? 1 : 0, base);
        auto it = g_base.find(key);
        if (it == g_base.end()) {
            ClosestSearch search(row, base);
            Strat found;
            if (!search.run(found)) return false;
            it = g_base.emplace(key, found).first;
        }
        s = it->second;
    }
    for (int i = 1; i < k; ++i) s = expand(s, row);
    out = std::move(s);
    return true;
}

}  // namespace

int admissible_order(int strategy, int n) {
    if (n < 2) n = 2;
    if (n % 2) ++n;
    if (strategy == JSVD_STRAT_MODULUS) return n;
    while (2 * odd_part(n, nullptr) > kMaxSearchOrder) n += 2;
    return n;
}

int build_pstrategy(int strategy, int n, std::vector<int> &out) {
    if (n < 2 || n % 2) return -2;
    Strat s;
    switch (strategy) {
        case JSVD_STRAT_MODULUS: s = modulus_strategy(n); break;
        case JSVD_STRAT_ROW:
        case JSVD_STRAT_ROW_REV:
            if (!closest(true, n, s)) return -2;
            break;
        case JSVD_STRAT_COL:
        case JSVD_STRAT_COL_REV:
            if (!closest(false, n, s)) return -2;
            break;
        default: return -1;
    }
    if (strategy == JSVD_STRAT_ROW_REV || strategy == JSVD_STRAT_COL_REV) {
        std::reverse(s.begin(), s.end());
        for (auto &st : s) std::reverse(st.begin(), st.end());
    }
    out.clear();
    out.reserve((size_t)(n - 1) * n);
    for (auto &st : s)
        for (auto [p, q] : st) { out.push_back(p); out.push_back(q); }
    return 0;
}

}  // namespace jsvd

extern "C" int jsvd_pivot_table(int strategy, int nblocks, int *out_pairs) {
    if (!out_pairs) return -3;
    std::vector<int> v;
    int rc = jsvd::build_pstrategy(strategy, nblocks, v);
    if (rc) return rc;
    std::copy(v.begin(), v.end(), out_pairs);
    return 0;
}
