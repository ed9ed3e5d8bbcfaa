// Runs the ensemble's host-side ordering functions (ps_worklist.h) on a spec
// read from standard input and prints their results, for tests/test_worklist.py.
//
// Input:  m order cap
//         per member: count, then count triples "ntiles per chain"
//         ord (m integers), cls (m integers)
// Output: "skew" + m integers
//         "slot member item tick0 dep need" per pass instance
//         "tickets T"
//         "group" + members, per batched group
#include <cstdio>
#include <vector>

#include "ps_worklist.h"

int main() {
  int m = 0, order = 0, cap = 0;
  if (std::scanf("%d %d %d", &m, &order, &cap) != 3 || m < 0) return 2;
  std::vector<std::vector<ps::WlItem>> seq(m);
  for (int i = 0; i < m; ++i) {
    int c = 0;
    if (std::scanf("%d", &c) != 1 || c < 0) return 2;
    for (int k = 0; k < c; ++k) {
      int nt = 0, per = 0, chain = 0;
      if (std::scanf("%d %d %d", &nt, &per, &chain) != 3) return 2;
      seq[i].push_back(ps::WlItem{nt, per, chain != 0});
    }
  }
  std::vector<int> ord(m), cls(m);
  for (int i = 0; i < m; ++i)
    if (std::scanf("%d", &ord[i]) != 1) return 2;
  for (int i = 0; i < m; ++i)
    if (std::scanf("%d", &cls[i]) != 1) return 2;
  const std::vector<int> skew = ps::wl_skew(ord, order);
  std::printf("skew");
  for (int s : skew) std::printf(" %d", s);
  std::printf("\n");
  std::vector<ps::WlSlot> slots;
  const long long t = ps::wl_schedule(seq, ord, skew, &slots);
  for (const ps::WlSlot& s : slots)
    std::printf("slot %d %d %lld %d %d\n", s.member, s.item, s.tick0, s.dep, s.need);
  std::printf("tickets %lld\n", t);
  for (const std::vector<int>& g : ps::wl_batches(cls, cap)) {
    std::printf("group");
    for (int j : g) std::printf(" %d", j);
    std::printf("\n");
  }
  return 0;
}
