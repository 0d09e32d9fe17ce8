// Topology of a scene's joint graph (host code, no CUDA): which solver fits
// it and the orders the solvers need.  A chain's joints ordered along the
// path (Sec. 5.2, Eq. chain-btd), a single closed loop's bodies along the
// cycle with the breaker last (Sec. 5.4), a forest's bodies breadth-first
// over all roots so that each level and each body's children are ranges
// (Sec. 5.3).
#pragma once
#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <vector>

namespace mabd {

struct Graph {
  int M = 0, K = 0;
  std::vector<char> free_body;
  std::vector<int> fa, fb;                     // free ends of each joint (-1 if none)
  std::vector<std::vector<int>> inc;           // free body -> incident joints
  std::vector<int> jtype;                      // joint types
  std::vector<int> ja;                         // body a of each joint (user id)
};

// fixed[j]: body j never moves; ja, jb, jt: each joint's bodies (jb may be
// -1, the world) and type
inline Graph build_graph(const std::vector<uint8_t> &fixed, const std::vector<int64_t> &ja,
                         const std::vector<int64_t> &jb, const std::vector<int> &jt) {
  Graph g;
  g.M = (int)fixed.size();
  g.K = (int)ja.size();
  g.free_body.resize(g.M);
  for (int j = 0; j < g.M; ++j) g.free_body[j] = fixed[j] ? 0 : 1;
  g.fa.resize(g.K);
  g.fb.resize(g.K);
  g.ja.resize(g.K);
  g.inc.resize(g.M);
  g.jtype.resize(g.K);
  for (int k = 0; k < g.K; ++k) {
    g.jtype[k] = jt[k];
    int a = (int)ja[k], b = (int)jb[k];
    g.ja[k] = a;
    g.fa[k] = g.free_body[a] ? a : -1;
    g.fb[k] = (b >= 0 && g.free_body[b]) ? b : -1;
    if (g.fa[k] >= 0) g.inc[a].push_back(k);
    if (g.fb[k] >= 0) g.inc[b].push_back(k);
  }
  return g;
}

inline int other_end(const Graph &g, int k, int j) { return g.fa[k] == j ? g.fb[k] : g.fa[k]; }

// A chain: the free bodies form one path through joints between free bodies,
// and ordering the joints along it puts every two joints that share a body
// next to each other (so the dual is block tridiagonal, Eq. chain-btd).
inline bool chain_order(const Graph &g, std::vector<int32_t> &border, std::vector<int32_t> &jorder) {
  int nfree = 0, nint = 0;
  for (int j = 0; j < g.M; ++j) nfree += g.free_body[j];
  for (int k = 0; k < g.K; ++k) nint += (g.fa[k] >= 0 && g.fb[k] >= 0);
  if (nfree == 0 || g.K == 0 || nint != nfree - 1) return false;
  int start = -1;
  for (int j = 0; j < g.M; ++j) {
    if (!g.free_body[j]) continue;
    int deg = 0;
    for (int k : g.inc[j]) deg += other_end(g, k, j) >= 0;
    if (deg > 2) return false;
    if (deg <= 1 && start < 0) start = j;
  }
  if (start < 0) return false;
  std::vector<char> used(g.K, 0);
  border.clear();
  jorder.clear();
  int cur = start, prevk = -1;
  while (cur >= 0) {
    border.push_back(cur);
    std::vector<int> side;
    for (int k : g.inc[cur])
      if (other_end(g, k, cur) < 0) side.push_back(k);
    std::sort(side.begin(), side.end());
    for (int k : side) {
      jorder.push_back(k);
      used[k] = 1;
    }
    int next = -1, nk = -1;
    for (int k : g.inc[cur])
      if (k != prevk && !used[k] && other_end(g, k, cur) >= 0) {
        nk = k;
        next = other_end(g, k, cur);
      }
    if (nk >= 0) {
      jorder.push_back(nk);
      used[nk] = 1;
    }
    prevk = nk;
    cur = next;
    if ((int)border.size() > nfree) return false;
  }
  if ((int)border.size() != nfree || (int)jorder.size() != g.K) return false;
  std::vector<int> pos(g.K);
  for (int i = 0; i < g.K; ++i) pos[jorder[i]] = i;
  for (int j = 0; j < g.M; ++j) {
    if (!g.free_body[j]) continue;
    if (g.inc[j].size() > 2) return false;
    if (g.inc[j].size() == 2 && std::abs(pos[g.inc[j][0]] - pos[g.inc[j][1]]) != 1) return false;
  }
  for (int j = 0; j < g.M; ++j)
    if (!g.free_body[j]) border.push_back(j);
  return true;
}

// A single closed loop (Sec. 5.4, Case III): every joint joins two free
// bodies, every free body has exactly two joints, and they form one cycle of
// at least three bodies.  Bodies follow the cycle; joint p joins bodies p and
// p + 1 for p < K - 1, and the last joint (the loop breaker) closes the loop
// between bodies K - 1 and 0.  The breaker is a ball joint when there is one
// (its rows count the right-hand-side passes of the Schur complement).
inline bool ring_order(const Graph &g, std::vector<int32_t> &border, std::vector<int32_t> &jorder) {
  int nfree = 0;
  for (int j = 0; j < g.M; ++j) nfree += g.free_body[j];
  if (g.K < 3 || g.K != nfree) return false;
  for (int k = 0; k < g.K; ++k)
    if (g.fa[k] < 0 || g.fb[k] < 0) return false;
  for (int j = 0; j < g.M; ++j)
    if (g.free_body[j] && g.inc[j].size() != 2) return false;
  int kb = 0;  // the breaker: the first ball joint, else joint 0
  for (int k = 0; k < g.K; ++k)
    if (g.jtype[k] == 0) {
      kb = k;
      break;
    }
  border.clear();
  jorder.clear();
  const int start = g.fb[kb];
  int cur = start, prevk = kb;
  for (int step = 0; step < g.K; ++step) {
    border.push_back(cur);
    const int k = g.inc[cur][0] == prevk ? g.inc[cur][1] : g.inc[cur][0];
    jorder.push_back(k);
    prevk = k;
    cur = other_end(g, k, cur);
  }
  if (cur != start || jorder.back() != kb || (int)border.size() != nfree) return false;
  std::vector<char> seen(g.M, 0);
  for (int j : border) {
    if (seen[j]) return false;
    seen[j] = 1;
  }
  for (int j = 0; j < g.M; ++j)
    if (!g.free_body[j]) border.push_back(j);
  return true;
}

// A forest: joints between free bodies form a forest and one-sided joints
// (to the world or a fixed body) sit on at most one body of each component,
// which becomes its root (at most two such joints, Sec. 5.3).  Bodies are
// ordered breadth-first over all roots at once, so each level is a range and
// the children of a body are a range; joints follow their body.
struct TreeOrder {
  std::vector<int32_t> border, jorder, lvl_off, parent, pjoint, cfirst, ccount, root_id;
  std::vector<int8_t> pside;
  std::vector<int32_t> root_joint;  // [2][nroots] user joint ids
  std::vector<int8_t> root_side;
  int nroots = 0;
};

inline bool tree_order(const Graph &g, TreeOrder &t) {
  const int M = g.M;
  std::vector<int> comp(M, -1), roots;
  int ncomp = 0;
  for (int s = 0; s < M; ++s) {
    if (!g.free_body[s] || comp[s] >= 0) continue;
    std::vector<int> q{s};
    comp[s] = ncomp;
    int root = -1, nroot_cand = 0;
    long edges2 = 0;
    for (size_t h = 0; h < q.size(); ++h) {
      int j = q[h];
      int nside = 0;
      for (int k : g.inc[j]) {
        int o = other_end(g, k, j);
        if (o < 0) {
          ++nside;
          continue;
        }
        ++edges2;
        if (comp[o] < 0) {
          comp[o] = ncomp;
          q.push_back(o);
        }
      }
      if (nside > 0) {
        ++nroot_cand;
        root = j;
        if (nside > 2) return false;
      }
    }
    if (edges2 != 2L * ((long)q.size() - 1) || nroot_cand > 1) return false;
    roots.push_back(root >= 0 ? root : s);
    ++ncomp;
  }
  t.nroots = (int)roots.size();
  t.border.clear();
  t.lvl_off.assign(1, 0);
  std::vector<int> depth(M, -1), par(M, -1), pj(M, -1);
  std::vector<int> frontier = roots;
  for (int r : roots) depth[r] = 0;
  // children of a free body, excluding its parent (for the level ordering)
  auto nkids = [&](int j) {
    int c = 0;
    for (int k : g.inc[j]) {
      int o = other_end(g, k, j);
      if (o >= 0 && o != par[j]) ++c;
    }
    return c;
  };
  (void)nkids;
  while (!frontier.empty()) {
    std::vector<int> next;
    for (int j : frontier) {
      t.border.push_back(j);
      std::vector<int> ks;
      for (int k : g.inc[j]) {
        int o = other_end(g, k, j);
        if (o >= 0 && o != par[j]) ks.push_back(k);
      }
      std::sort(ks.begin(), ks.end());
      for (int k : ks) {
        int o = other_end(g, k, j);
        if (depth[o] >= 0) return false;
        depth[o] = depth[j] + 1;
        par[o] = j;
        pj[o] = k;
        next.push_back(o);
      }
    }
    t.lvl_off.push_back((int32_t)t.border.size());
    frontier.swap(next);
  }
  const int nfree = (int)t.border.size();
  for (int j = 0; j < M; ++j)
    if (!g.free_body[j]) t.border.push_back(j);
  std::vector<int> pos(M);
  for (int i = 0; i < M; ++i) pos[t.border[i]] = i;
  // joints in body order: a root's one-sided joints, else the parent joint
  t.jorder.clear();
  t.root_joint.assign(2 * (size_t)std::max(t.nroots, 1), -1);
  t.root_side.assign(2 * (size_t)std::max(t.nroots, 1), 0);
  t.parent.assign(M, -1);
  t.pjoint.assign(M, -1);
  t.pside.assign(M, 0);
  t.cfirst.assign(M, 0);
  t.ccount.assign(M, 0);
  t.root_id.assign(M, -1);
  int rid = 0;
  for (int i = 0; i < nfree; ++i) {
    const int j = t.border[i];
    if (par[j] < 0) {
      t.root_id[i] = rid;
      int w = 0;
      std::vector<int> side;
      for (int k : g.inc[j])
        if (other_end(g, k, j) < 0) side.push_back(k);
      std::sort(side.begin(), side.end());
      for (int k : side) {
        t.root_joint[(size_t)w * t.nroots + rid] = k;
        t.root_side[(size_t)w * t.nroots + rid] = g.ja[k] == j ? 0 : 1;
        ++w;
        t.jorder.push_back(k);
      }
      ++rid;
    } else {
      t.parent[i] = pos[par[j]];
      t.pjoint[i] = pj[j];  // user id
      t.pside[i] = g.ja[pj[j]] == j ? 0 : 1;
      t.jorder.push_back(pj[j]);
    }
  }
  if ((int)t.jorder.size() != g.K) return false;
  for (int i = nfree - 1; i >= 0; --i) {
    const int p = t.parent[i];
    if (p < 0) continue;
    t.ccount[p] += 1;
    t.cfirst[p] = i;  // children of a body are contiguous; the smallest index wins
  }
  return true;
}

}  // namespace mabd
