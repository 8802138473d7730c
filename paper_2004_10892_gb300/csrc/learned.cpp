// learned.cpp -- learned slicing proposer hook (placeholder: always falls back).
#include "graph.hpp"
namespace tnq {
int learned_propose(void*, const Graph&, const std::vector<int>&, const TreeDecomposition&) { return -1; }
}  // namespace tnq
