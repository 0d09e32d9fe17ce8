// Runs the library's topology code (csrc/topology.h) on a scene read from
// stdin and prints what it found, for tests/test_topology.py to check.
// Input: M K, then M fixed flags, then K lines "body_a body_b type".
// Output lines: "chain 0|1", "chain_border ...", "chain_jorder ...",
// "ring 0|1", "ring_border ...", "ring_jorder ...", "tree 0|1", and for a
// forest "tree_border", "tree_jorder", "tree_lvl", "tree_parent",
// "tree_pjoint", "tree_pside", "tree_cfirst", "tree_ccount", "tree_roots".
#include <cstdio>
#include <vector>

#include "topology.h"

using namespace mabd;

template <class T>
static void put(const char *name, const std::vector<T> &v) {
  std::printf("%s", name);
  for (const T &x : v) std::printf(" %d", (int)x);
  std::printf("\n");
}

int main() {
  int M = 0, K = 0;
  if (std::scanf("%d %d", &M, &K) != 2) return 2;
  std::vector<uint8_t> fixed(M);
  for (int j = 0; j < M; ++j) {
    int f = 0;
    if (std::scanf("%d", &f) != 1) return 2;
    fixed[j] = (uint8_t)f;
  }
  std::vector<int64_t> ja(K), jb(K);
  std::vector<int> jt(K);
  for (int k = 0; k < K; ++k) {
    long long a = 0, b = 0;
    int t = 0;
    if (std::scanf("%lld %lld %d", &a, &b, &t) != 3) return 2;
    ja[k] = a;
    jb[k] = b;
    jt[k] = t;
  }
  const Graph g = build_graph(fixed, ja, jb, jt);
  std::vector<int32_t> border, jorder;
  const bool chain = K > 0 && chain_order(g, border, jorder);
  std::printf("chain %d\n", chain ? 1 : 0);
  if (chain) {
    put("chain_border", border);
    put("chain_jorder", jorder);
  }
  TreeOrder t;
  const bool tree = K > 0 && tree_order(g, t);
  std::printf("tree %d\n", tree ? 1 : 0);
  if (tree) {
    put("tree_border", t.border);
    put("tree_jorder", t.jorder);
    put("tree_lvl", t.lvl_off);
    put("tree_parent", t.parent);
    put("tree_pjoint", t.pjoint);
    put("tree_pside", t.pside);
    put("tree_cfirst", t.cfirst);
    put("tree_ccount", t.ccount);
    put("tree_rootjoint", t.root_joint);
    put("tree_rootside", t.root_side);
    std::printf("tree_nroots %d\n", t.nroots);
  }
  border.clear();
  jorder.clear();
  const bool ring = K > 0 && !chain && !tree && ring_order(g, border, jorder);
  std::printf("ring %d\n", ring ? 1 : 0);
  if (ring) {
    put("ring_border", border);
    put("ring_jorder", jorder);
  }
  return 0;
}
