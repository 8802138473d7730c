// graph.hpp -- host-side graph algorithms of the planner (Sections II.B-II.C,
// III, Appendix A): greedy elimination orders, treewidth of an order
// (Algorithm 1), tree decomposition of an order (Algorithm 4), the greedy
// mu-treewidth deletion of Algorithm 2 with the degree, direct-reduction
// (Algorithm 3) and tree-trimming (Section III.B) scores.
#pragma once
#include <cstdint>
#include <vector>

namespace tnq {

// Simple undirected graph on vertices 0..n-1 as adjacency bitsets.
struct Graph {
  int n = 0;
  int words = 0;
  std::vector<uint64_t> bits;  // n * words

  Graph() = default;
  explicit Graph(int n_);
  void add_edge(int a, int b);
  bool has(int a, int b) const { return (row(a)[b >> 6] >> (b & 63)) & 1ull; }
  const uint64_t* row(int v) const { return bits.data() + (size_t)v * words; }
  uint64_t* row(int v) { return bits.data() + (size_t)v * words; }
  int degree(int v) const;
};

// A tree decomposition: bags (sorted vertex lists) and a parent per bag (-1 = root).
struct TreeDecomposition {
  std::vector<std::vector<int>> bags;
  std::vector<int> parent;
  int max_bag() const;
};

enum OrderMethod { ORDER_MIN_FILL = 0, ORDER_MIN_DEGREE = 1 };
enum Slicer { SLICER_TREE_TRIMMING = 0, SLICER_DEGREE = 1, SLICER_DIRECT = 2, SLICER_LEARNED = 3,
              SLICER_BETWEENNESS = 4 };

// Greedy elimination order (min-fill: fewest fill edges, then lowest degree;
// min-degree). Ties go to the lowest vertex id, or to a seeded random choice
// when rng != nullptr.
std::vector<int> greedy_order(const Graph& g, int method, uint64_t* rng = nullptr);

// Algorithm 1: simulates the elimination of `order` (vertices absent from the
// order are treated as deleted) and returns the largest neighbourhood seen,
// starting from 1. If bag_sizes is given it receives |N(u)|+1 per step.
int treewidth_of_order(const Graph& g, const std::vector<int>& order,
                       std::vector<int>* bag_sizes = nullptr);

// Neighbourhoods met during the elimination: bag of step i = {order[i]} U N(order[i]).
std::vector<std::vector<int>> elimination_bags(const Graph& g, const std::vector<int>& order);

// Algorithm 4 (Appendix A): tree decomposition of the elimination order with
// only maximal cliques kept.
TreeDecomposition tree_decomposition(const Graph& g, const std::vector<int>& order);

// Removes vertex v from every bag and merges bags that became subsets of a
// tree neighbour (the TD stays valid for the graph without v).
void td_remove_vertex(TreeDecomposition& td, int v);

// Score functions of Algorithm 2; each returns the vertex to delete (degree,
// direct and betweenness are recomputed on the reduced graph at every step).
// `pos[v]` = position of v in the current order (-1 if deleted); ties go to the
// earliest position, or to a seeded random choice when rng_state != nullptr.
int score_tree_trimming(const TreeDecomposition& td, const std::vector<int>& pos, uint64_t* rng_state);
int score_degree(const Graph& g, const std::vector<int>& order, const std::vector<int>& pos,
                 uint64_t* rng_state);
int score_direct(const Graph& g, const std::vector<int>& order, const std::vector<int>& pos,
                 uint64_t* rng_state);
// Betweenness centrality (Section III.A): the number of shortest paths between
// pairs of the listed vertices that pass through each vertex (Brandes'
// algorithm; a pair with several shortest paths counts fractionally).
std::vector<double> betweenness(const Graph& g, const std::vector<int>& verts);
int score_betweenness(const Graph& g, const std::vector<int>& order, const std::vector<int>& pos,
                      uint64_t* rng_state);

// Tree-trimming candidates with their (length, weight) as the learned proposer's features.
struct TrimCandidate {
  int v;
  int length;   // number of bags containing v
  int weight;   // sum of the sizes of those bags
};
std::vector<TrimCandidate> tree_trimming_candidates(const TreeDecomposition& td);

// Graph with vertex v removed (same vertex numbering, v isolated).
void delete_vertex(Graph& g, int v);

struct DeletionResult {
  std::vector<int> mu;               // deleted vertices in order
  std::vector<int> tau_after;        // treewidth of the reduced order after each deletion
  std::vector<int> reduced_order;    // pi~ = pi minus mu
};

// Callback used by the learned slicer (p = vertices deleted so far): returns a
// vertex or -1 to fall back.
typedef int (*ProposerFn)(void* ctx, const Graph& g, const std::vector<int>& order,
                          const TreeDecomposition& td, int p);

// Algorithm 2. Deletes vertices until p >= min_p and (largest bag <= max_bag, or
// p == max_p). max_bag <= 0 means no bag limit.
// reorder_every > 0: after every reorder_every deletions the order is
// recomputed by the greedy heuristic `order_method` on the reduced graph (kept
// unless its treewidth exceeds that of the inherited order) and the TD rebuilt
// from it: the optional recomputation step of Algorithm 2, with the greedy
// orderer in place of an exact tree-decomposition solver.
DeletionResult greedy_deletion(const Graph& g, const std::vector<int>& order, int slicer, int min_p,
                               int max_p, int max_bag, uint64_t seed, bool td_rebuild,
                               ProposerFn proposer = nullptr, void* proposer_ctx = nullptr,
                               int reorder_every = 0, int order_method = ORDER_MIN_FILL);

uint64_t splitmix64_next(uint64_t* state);

}  // namespace tnq
