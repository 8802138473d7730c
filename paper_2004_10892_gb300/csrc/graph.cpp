// graph.cpp -- planner graph algorithms (see graph.hpp for the paper mapping).
#include "graph.hpp"

#include <algorithm>
#include <stdexcept>

namespace tnq {

static inline int popc(uint64_t x) { return __builtin_popcountll(x); }

Graph::Graph(int n_) : n(n_), words((n_ + 63) / 64), bits((size_t)n_ * ((n_ + 63) / 64), 0ull) {}

void Graph::add_edge(int a, int b) {
  if (a == b) return;  // self-loops carry no edge (Section II.A)
  row(a)[b >> 6] |= 1ull << (b & 63);
  row(b)[a >> 6] |= 1ull << (a & 63);
}

int Graph::degree(int v) const {
  int d = 0;
  for (int w = 0; w < words; ++w) d += popc(row(v)[w]);
  return d;
}

int TreeDecomposition::max_bag() const {
  int m = 0;
  for (auto& b : bags) m = std::max<int>(m, (int)b.size());
  return m;
}

uint64_t splitmix64_next(uint64_t* state) {
  uint64_t z = (*state += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

void delete_vertex(Graph& g, int v) {
  for (int w = 0; w < g.n; ++w) g.row(w)[v >> 6] &= ~(1ull << (v & 63));
  std::fill(g.row(v), g.row(v) + g.words, 0ull);
}

// Elimination state: a working copy of the adjacency plus the alive set.
namespace {
struct Elim {
  Graph g;
  std::vector<uint64_t> alive;
  explicit Elim(const Graph& g0) : g(g0), alive(g0.words, 0ull) {}
  void set_alive(int v) { alive[v >> 6] |= 1ull << (v & 63); }
  bool is_alive(int v) const { return (alive[v >> 6] >> (v & 63)) & 1ull; }
  // N(u) among alive vertices (u itself excluded).
  void nbrs(int u, std::vector<uint64_t>& out) const {
    out.resize(g.words);
    const uint64_t* r = g.row(u);
    for (int w = 0; w < g.words; ++w) out[w] = r[w] & alive[w];
    out[u >> 6] &= ~(1ull << (u & 63));
  }
  // Removes u: its alive neighbourhood becomes a clique (Eq. 2 step).
  void eliminate(int u, const std::vector<uint64_t>& N) {
    for (int w = 0; w < g.words; ++w) {
      uint64_t m = N[w];
      while (m) {
        int a = w * 64 + __builtin_ctzll(m);
        m &= m - 1;
        uint64_t* ra = g.row(a);
        for (int x = 0; x < g.words; ++x) ra[x] |= N[x];
        ra[a >> 6] &= ~(1ull << (a & 63));
      }
    }
    alive[u >> 6] &= ~(1ull << (u & 63));
  }
};

std::vector<int> bits_to_list(const std::vector<uint64_t>& b) {
  std::vector<int> out;
  for (size_t w = 0; w < b.size(); ++w) {
    uint64_t m = b[w];
    while (m) {
      out.push_back((int)(w * 64 + __builtin_ctzll(m)));
      m &= m - 1;
    }
  }
  return out;
}
}  // namespace

std::vector<int> greedy_order(const Graph& g0, int method, uint64_t* rng) {
  Elim E(g0);
  for (int v = 0; v < g0.n; ++v) E.set_alive(v);
  std::vector<int> order;
  order.reserve(g0.n);
  std::vector<uint64_t> N, best_N;
  std::vector<int> ties;
  for (int step = 0; step < g0.n; ++step) {
    int best = -1;
    long best_fill = -1, best_deg = -1;
    ties.clear();
    for (int v = 0; v < g0.n; ++v) {
      if (!E.is_alive(v)) continue;
      E.nbrs(v, N);
      long d = 0;
      for (int w = 0; w < g0.words; ++w) d += popc(N[w]);
      long fill = 0;
      if (method == ORDER_MIN_FILL) {
        // missing edges among N(v): sum over a in N(v) of (d - 1 - |N(a) & N(v)|), halved
        for (int w = 0; w < g0.words; ++w) {
          uint64_t m = N[w];
          while (m) {
            int a = w * 64 + __builtin_ctzll(m);
            m &= m - 1;
            const uint64_t* ra = E.g.row(a);
            long common = 0;
            for (int x = 0; x < g0.words; ++x) common += popc(ra[x] & N[x]);
            fill += d - 1 - common;
          }
        }
        fill /= 2;
      }
      bool better, tie;
      if (best < 0) {
        better = true;
        tie = false;
      } else if (method == ORDER_MIN_FILL) {
        better = fill < best_fill || (fill == best_fill && d < best_deg);
        tie = fill == best_fill && d == best_deg;
      } else {
        better = d < best_deg;
        tie = d == best_deg;
      }
      if (better) {
        best = v;
        best_fill = fill;
        best_deg = d;
        ties.assign(1, v);
      } else if (tie) {
        ties.push_back(v);
      }
    }
    if (rng && ties.size() > 1) best = ties[splitmix64_next(rng) % ties.size()];
    E.nbrs(best, N);
    E.eliminate(best, N);
    order.push_back(best);
  }
  return order;
}

int treewidth_of_order(const Graph& g0, const std::vector<int>& order, std::vector<int>* bag_sizes) {
  Elim E(g0);
  for (int v : order) E.set_alive(v);
  int tau = 1;
  std::vector<uint64_t> N;
  if (bag_sizes) bag_sizes->clear();
  for (int u : order) {
    E.nbrs(u, N);
    int d = 0;
    for (int w = 0; w < g0.words; ++w) d += popc(N[w]);
    tau = std::max(tau, d);
    if (bag_sizes) bag_sizes->push_back(d + 1);
    E.eliminate(u, N);
  }
  return tau;
}

std::vector<std::vector<int>> elimination_bags(const Graph& g0, const std::vector<int>& order) {
  Elim E(g0);
  for (int v : order) E.set_alive(v);
  std::vector<std::vector<int>> bags;
  std::vector<uint64_t> N;
  for (int u : order) {
    E.nbrs(u, N);
    std::vector<int> b = bits_to_list(N);
    b.push_back(u);
    std::sort(b.begin(), b.end());
    bags.push_back(std::move(b));
    E.eliminate(u, N);
  }
  return bags;
}

// Contracts tree edges whose end bags are nested until every bag is maximal.
static void td_make_maximal(TreeDecomposition& td) {
  const int nb = (int)td.bags.size();
  std::vector<char> dead(nb, 0);
  bool changed = true;
  while (changed) {
    changed = false;
    for (int c = 0; c < nb; ++c) {
      if (dead[c]) continue;
      int p = td.parent[c];
      if (p < 0) continue;
      const auto& bc = td.bags[c];
      const auto& bp = td.bags[p];
      if (std::includes(bp.begin(), bp.end(), bc.begin(), bc.end())) {
        // c is redundant: its children move to p
        for (int x = 0; x < nb; ++x)
          if (!dead[x] && td.parent[x] == c) td.parent[x] = p;
        dead[c] = 1;
        changed = true;
      } else if (std::includes(bc.begin(), bc.end(), bp.begin(), bp.end())) {
        // p is redundant: c takes its place
        for (int x = 0; x < nb; ++x)
          if (!dead[x] && x != c && td.parent[x] == p) td.parent[x] = c;
        td.parent[c] = td.parent[p];
        dead[p] = 1;
        changed = true;
      }
    }
  }
  // compact
  std::vector<int> remap(nb, -1);
  TreeDecomposition out;
  for (int b = 0; b < nb; ++b)
    if (!dead[b]) {
      remap[b] = (int)out.bags.size();
      out.bags.push_back(td.bags[b]);
    }
  out.parent.assign(out.bags.size(), -1);
  for (int b = 0; b < nb; ++b)
    if (!dead[b] && td.parent[b] >= 0) out.parent[remap[b]] = remap[td.parent[b]];
  td = std::move(out);
}

TreeDecomposition tree_decomposition(const Graph& g0, const std::vector<int>& order) {
  // Bag of step i is {u_i} U N(u_i); its parent is the step of the neighbour
  // eliminated first (that neighbour's bag holds all of N(u_i)). Roots of
  // separate components are chained to the last root so the result is a tree.
  TreeDecomposition td;
  td.bags = elimination_bags(g0, order);
  const int n = (int)order.size();
  std::vector<int> step_of(g0.n, -1);
  for (int i = 0; i < n; ++i) step_of[order[i]] = i;
  td.parent.assign(n, -1);
  for (int i = 0; i < n; ++i) {
    int best = -1;
    for (int v : td.bags[i])
      if (v != order[i] && (best < 0 || step_of[v] < best)) best = step_of[v];
    td.parent[i] = best;
  }
  int last_root = -1;
  for (int i = n - 1; i >= 0; --i)
    if (td.parent[i] < 0) {
      if (last_root < 0) last_root = i;
      else td.parent[i] = last_root;
    }
  td_make_maximal(td);
  return td;
}

void td_remove_vertex(TreeDecomposition& td, int v) {
  for (auto& b : td.bags) {
    auto it = std::lower_bound(b.begin(), b.end(), v);
    if (it != b.end() && *it == v) b.erase(it);
  }
  td_make_maximal(td);
}

std::vector<TrimCandidate> tree_trimming_candidates(const TreeDecomposition& td) {
  const int M = td.max_bag();
  std::vector<int> cand;
  for (auto& b : td.bags)
    if ((int)b.size() == M) cand.insert(cand.end(), b.begin(), b.end());
  std::sort(cand.begin(), cand.end());
  cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
  std::vector<TrimCandidate> out;
  for (int v : cand) {
    TrimCandidate c{v, 0, 0};
    for (auto& b : td.bags)
      if (std::binary_search(b.begin(), b.end(), v)) {
        c.length += 1;
        c.weight += (int)b.size();
      }
    out.push_back(c);
  }
  return out;
}

// Picks among `ties` (all equally good) the earliest order position, or a
// seeded random one.
static int break_tie(const std::vector<int>& ties, const std::vector<int>& pos, uint64_t* rng) {
  if (ties.empty()) return -1;
  if (rng) return ties[splitmix64_next(rng) % ties.size()];
  int best = ties[0];
  for (int v : ties)
    if (pos[v] < pos[best]) best = v;
  return best;
}

int score_tree_trimming(const TreeDecomposition& td, const std::vector<int>& pos, uint64_t* rng) {
  auto cands = tree_trimming_candidates(td);
  int bl = -1, bw = -1;
  for (auto& c : cands) {
    if (pos[c.v] < 0) continue;
    if (c.length > bl || (c.length == bl && c.weight > bw)) {
      bl = c.length;
      bw = c.weight;
    }
  }
  std::vector<int> ties;
  for (auto& c : cands)
    if (pos[c.v] >= 0 && c.length == bl && c.weight == bw) ties.push_back(c.v);
  return break_tie(ties, pos, rng);
}

int score_degree(const Graph& g, const std::vector<int>& order, const std::vector<int>& pos,
                 uint64_t* rng) {
  int bd = -1;
  for (int v : order) bd = std::max(bd, g.degree(v));
  std::vector<int> ties;
  for (int v : order)
    if (g.degree(v) == bd) ties.push_back(v);
  return break_tie(ties, pos, rng);
}

std::vector<double> betweenness(const Graph& g, const std::vector<int>& verts) {
  // Brandes' algorithm (J. Math. Sociol. 25, 2001) for an unweighted graph:
  // per source s one BFS counts the shortest paths sigma[v]; walking the BFS
  // order backwards accumulates the dependency
  //   delta[v] = sum over successors w of sigma[v] / sigma[w] * (1 + delta[w]),
  // and CB[w] += delta[w] for w != s. Every unordered pair is met from both
  // ends, hence the final halving.
  const int n = g.n;
  std::vector<std::vector<int>> adj(n);
  for (int v : verts)
    for (int w : verts)
      if (w != v && g.has(v, w)) adj[v].push_back(w);
  std::vector<double> cb(n, 0.0), sigma(n, 0.0), delta(n, 0.0);
  std::vector<int> dist(n, -1), bfs;
  bfs.reserve(verts.size());
  for (int s : verts) {
    for (int v : verts) {
      sigma[v] = 0.0;
      delta[v] = 0.0;
      dist[v] = -1;
    }
    bfs.clear();
    sigma[s] = 1.0;
    dist[s] = 0;
    bfs.push_back(s);
    for (size_t head = 0; head < bfs.size(); ++head) {
      const int v = bfs[head];
      for (int w : adj[v]) {
        if (dist[w] < 0) {
          dist[w] = dist[v] + 1;
          bfs.push_back(w);
        }
        if (dist[w] == dist[v] + 1) sigma[w] += sigma[v];
      }
    }
    for (size_t i = bfs.size(); i-- > 0;) {
      const int w = bfs[i];
      for (int v : adj[w])
        if (dist[v] == dist[w] - 1) delta[v] += sigma[v] / sigma[w] * (1.0 + delta[w]);
      if (w != s) cb[w] += delta[w];
    }
  }
  for (double& c : cb) c *= 0.5;
  return cb;
}

int score_betweenness(const Graph& g, const std::vector<int>& order, const std::vector<int>& pos,
                      uint64_t* rng) {
  const std::vector<double> cb = betweenness(g, order);
  double best = -1.0;
  for (int v : order) best = std::max(best, cb[v]);
  std::vector<int> ties;  // equal up to the rounding of the accumulated fractions
  for (int v : order)
    if (cb[v] >= best - 1e-9 * std::max(1.0, best)) ties.push_back(v);
  return break_tie(ties, pos, rng);
}

int score_direct(const Graph& g, const std::vector<int>& order, const std::vector<int>& pos,
                 uint64_t* rng) {
  // Algorithm 3 (read with u deleted in the trial and the best gain kept):
  // try deleting every u, keep the largest treewidth reduction.
  const int tau = treewidth_of_order(g, order);
  int best_gain = -1;
  std::vector<int> ties;
  std::vector<int> reduced;
  reduced.reserve(order.size());
  for (int u : order) {
    reduced.clear();
    for (int v : order)
      if (v != u) reduced.push_back(v);
    int gain = tau - treewidth_of_order(g, reduced);
    if (gain > best_gain) {
      best_gain = gain;
      ties.clear();
    }
    if (gain == best_gain) ties.push_back(u);
  }
  return break_tie(ties, pos, rng);
}

static int max_bag_of(const Graph& g, const std::vector<int>& order) {
  std::vector<int> sizes;
  treewidth_of_order(g, order, &sizes);
  int m = 0;
  for (int s : sizes) m = std::max(m, s);
  return m;
}

DeletionResult greedy_deletion(const Graph& g0, const std::vector<int>& order0, int slicer, int min_p,
                               int max_p, int max_bag, uint64_t seed, bool td_rebuild,
                               ProposerFn proposer, void* proposer_ctx, int reorder_every, int order_method) {
  DeletionResult R;
  Graph g = g0;
  std::vector<int> order = order0;
  std::vector<int> pos(g0.n, -1);
  for (size_t i = 0; i < order.size(); ++i) pos[order[i]] = (int)i;
  uint64_t rng_state = seed;
  uint64_t* rng = seed ? &rng_state : nullptr;
  TreeDecomposition td = tree_decomposition(g, order);
  int p = 0;
  while (!order.empty()) {
    if (p >= max_p) break;
    if (p >= min_p && max_bag > 0 && max_bag_of(g, order) <= max_bag) break;
    int u = -1;
    switch (slicer) {
      case SLICER_DEGREE: u = score_degree(g, order, pos, rng); break;
      case SLICER_DIRECT: u = score_direct(g, order, pos, rng); break;
      case SLICER_BETWEENNESS: u = score_betweenness(g, order, pos, rng); break;
      case SLICER_LEARNED:
        if (proposer) u = proposer(proposer_ctx, g, order, td, p);
        if (u < 0 || u >= g.n || pos[u] < 0) u = score_tree_trimming(td, pos, rng);  // fallback
        break;
      default: u = score_tree_trimming(td, pos, rng); break;
    }
    if (u < 0) break;
    delete_vertex(g, u);
    order.erase(std::find(order.begin(), order.end(), u));
    R.mu.push_back(u);
    const bool reorder = reorder_every > 0 && (int)R.mu.size() % reorder_every == 0;
    if (reorder) {  // fresh greedy order of the reduced graph (deleted vertices are isolated: drop them),
                    // kept unless its treewidth is larger than that of the inherited order
      std::vector<char> keep(g.n, 0);
      for (int v : order) keep[v] = 1;
      std::vector<int> fresh;
      for (int v : greedy_order(g, order_method))
        if (keep[v]) fresh.push_back(v);
      if (treewidth_of_order(g, fresh) <= treewidth_of_order(g, order)) order = fresh;
    }
    std::fill(pos.begin(), pos.end(), -1);
    for (size_t i = 0; i < order.size(); ++i) pos[order[i]] = (int)i;
    if (td_rebuild || reorder) td = tree_decomposition(g, order);
    else td_remove_vertex(td, u);
    R.tau_after.push_back(treewidth_of_order(g, order));
    ++p;
  }
  R.reduced_order = order;
  return R;
}

}  // namespace tnq
