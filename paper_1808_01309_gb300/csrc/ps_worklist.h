// Host-side ordering of the ensemble's shared launches (plain C++, no CUDA):
// the work list of the persistent launch and the member groups of the
// batched launches.  ps_ensemble.cu builds both from these functions; the
// CPU tests compile this header alone and check the orders' invariants.
#pragma once
#include <algorithm>
#include <vector>

namespace ps {

// One pass instance in a member's own sequence (its passes in execution
// order: per step and RK stage z-inverse, y-inverse, x, y-forward,
// z-forward, update; plus the energy sum after a z-inverse).
struct WlItem {
  int ntiles;  // tiles of the pass instance (> 0)
  int per;     // tiles per ticket (> 0)
  bool chain;  // false: the member's later passes do not wait for it (the energy sum)
};

// Its place in the launch's global list.
struct WlSlot {
  int member, item;  // which member's which item
  long long tick0;   // first ticket
  int dep;           // global index of the pass instance it waits for, or -1
  int need;          // that pass instance's tile count (0 if none)
};

// Members' skew in levels: 0 for all (order 0, 1), or the position in `ord`
// modulo 6 (order 2: the members' pass sequences are staggered over the six
// passes of a stage).
inline std::vector<int> wl_skew(const std::vector<int>& ord, int order) {
  std::vector<int> skew(ord.size(), 0);
  if (order == 2)
    for (size_t k = 0; k < ord.size(); ++k) skew[ord[k]] = (int)(k % 6);
  return skew;
}

// Global work list, level by level: at level L member ord[k] contributes its
// item L - skew[ord[k]] (if it has one).  Each pass instance waits for the
// member's previous chained one, which sits earlier in the list and so owns
// lower tickets: a CTA only ever waits for tickets handed out before its own.
// Returns the total ticket count.
inline long long wl_schedule(const std::vector<std::vector<WlItem>>& seq, const std::vector<int>& ord,
                             const std::vector<int>& skew, std::vector<WlSlot>* out) {
  out->clear();
  size_t longest = 0;
  for (size_t i = 0; i < seq.size(); ++i) longest = std::max(longest, seq[i].size() + (size_t)skew[i]);
  std::vector<int> last(seq.size(), -1);
  long long tick = 0;
  for (size_t lev = 0; lev < longest; ++lev)
    for (int i : ord) {
      const long long idx = (long long)lev - skew[i];
      if (idx < 0 || idx >= (long long)seq[i].size()) continue;
      const WlItem& it = seq[i][idx];
      WlSlot s;
      s.member = i;
      s.item = (int)idx;
      s.tick0 = tick;
      s.dep = last[i];
      s.need = last[i] >= 0 ? seq[i][(*out)[last[i]].item].ntiles : 0;
      tick += (it.ntiles + it.per - 1) / it.per;
      if (it.chain) last[i] = (int)out->size();
      out->push_back(s);
    }
  return tick;
}

// Members sharing the batched launches: greedily, the first member not yet
// placed and the following members of its class (cls[j] == cls[i]), at most
// `cap` per group, in member order.
inline std::vector<std::vector<int>> wl_batches(const std::vector<int>& cls, int cap) {
  cap = std::max(1, cap);
  std::vector<std::vector<int>> groups;
  std::vector<bool> done(cls.size(), false);
  for (size_t i = 0; i < cls.size(); ++i) {
    if (done[i]) continue;
    std::vector<int> g;
    for (size_t j = i; j < cls.size() && (int)g.size() < cap; ++j)
      if (!done[j] && cls[j] == cls[i]) {
        g.push_back((int)j);
        done[j] = true;
      }
    groups.push_back(g);
  }
  return groups;
}

}  // namespace ps
