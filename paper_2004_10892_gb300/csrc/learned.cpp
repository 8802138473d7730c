// learned.cpp -- learned slicing proposer (host side).
//
// Candidates are the vertices of the largest bags of the current tree
// decomposition (the set the tree-trimming score of Section III.B ranks).
// Each gets a feature vector; a 3-layer MLP (ReLU, hidden width H) predicts
// the log2 of the total contraction cost after deleting it, and the proposer
// deletes the candidate with the lowest prediction. Without weights it
// returns -1 and Algorithm 2 falls back to tree-trimming.
//
// Label (dataset generation): change of the exact graph-model cost caused by
// the deletion, log2(2^(p+1) * sum_i 2^|bag_i| after) - log2(2^p * sum_i
// 2^|bag_i| before): every elimination step costs 2^|bag| products per slice
// (the cost exponents of Eq. 2, Section IV) and the deletion doubles the
// number of slices.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/tnq.h"
#include "graph.hpp"
#include "plan.hpp"
#include "program.hpp"

namespace tnq {

constexpr int LF = 12;  // features per candidate

namespace {
std::mutex g_mu;
std::vector<float> g_w;  // W1 (H x LF), b1 (H), W2 (H x H), b2 (H), W3 (H), b3 (1)
int g_hidden = 0;

double log2_cost(const Graph& g, const std::vector<int>& order, int p) {
  std::vector<int> sizes;
  treewidth_of_order(g, order, &sizes);
  double s = 0;
  for (int r : sizes) s += std::ldexp(1.0, r);
  return std::log2(std::max(s, 1.0)) + p;
}
}  // namespace

// Features of every candidate (vertices of maximum-size bags), LF floats each.
std::vector<int> candidate_features(const Graph& g, const std::vector<int>& order, const TreeDecomposition& td, int p,
                                    std::vector<float>& feats) {
  auto cands = tree_trimming_candidates(td);
  const int M = td.max_bag();
  const int nb = (int)td.bags.size();
  std::vector<int> pos(g.n, -1);
  for (size_t i = 0; i < order.size(); ++i) pos[order[i]] = (int)i;
  std::vector<int> elim_bag(g.n, 0);
  {
    std::vector<int> sizes;
    treewidth_of_order(g, order, &sizes);
    for (size_t i = 0; i < order.size(); ++i) elim_bag[order[i]] = sizes[i];
  }
  int max_len = 1, max_w = 1, max_deg = 1;
  for (auto& c : cands) {
    max_len = std::max(max_len, c.length);
    max_w = std::max(max_w, c.weight);
    max_deg = std::max(max_deg, g.degree(c.v));
  }
  std::vector<int> out;
  feats.clear();
  for (auto& c : cands) {
    if (pos[c.v] < 0) continue;
    int in_max = 0, in_near = 0;
    for (auto& b : td.bags) {
      if (!std::binary_search(b.begin(), b.end(), c.v)) continue;
      if ((int)b.size() == M) ++in_max;
      if ((int)b.size() >= M - 1) ++in_near;
    }
    int n_max = 0;
    for (auto& b : td.bags) n_max += (int)b.size() == M;
    const float f[LF] = {
        (float)c.length / max_len,
        (float)c.weight / max_w,
        (float)g.degree(c.v) / max_deg,
        order.empty() ? 0.f : (float)pos[c.v] / (float)order.size(),
        (float)in_max / std::max(n_max, 1),
        (float)in_near / std::max(nb, 1),
        (float)elim_bag[c.v] / std::max(M, 1),
        (float)c.length / std::max(nb, 1),
        (float)M / 32.f,
        (float)p / 16.f,
        (float)cands.size() / 64.f,
        1.f};
    feats.insert(feats.end(), f, f + LF);
    out.push_back(c.v);
  }
  return out;
}

float mlp_forward_host(const float* w, int H, const float* x) {
  const float* W1 = w;
  const float* b1 = W1 + H * LF;
  const float* W2 = b1 + H;
  const float* b2 = W2 + H * H;
  const float* W3 = b2 + H;
  const float* b3 = W3 + H;
  std::vector<float> h1(H), h2(H);
  for (int i = 0; i < H; ++i) {
    float a = b1[i];
    for (int j = 0; j < LF; ++j) a += W1[i * LF + j] * x[j];
    h1[i] = a > 0.f ? a : 0.f;
  }
  for (int i = 0; i < H; ++i) {
    float a = b2[i];
    for (int j = 0; j < H; ++j) a += W2[i * H + j] * h1[j];
    h2[i] = a > 0.f ? a : 0.f;
  }
  float a = b3[0];
  for (int j = 0; j < H; ++j) a += W3[j] * h2[j];
  return a;
}

int learned_propose(void*, const Graph& g, const std::vector<int>& order, const TreeDecomposition& td, int p) {
  std::vector<float> w;
  int H;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_w.empty()) return -1;
    w = g_w;
    H = g_hidden;
  }
  std::vector<float> feats;
  std::vector<int> cands = candidate_features(g, order, td, p, feats);
  int best = -1;
  float best_v = 0.f;
  for (size_t i = 0; i < cands.size(); ++i) {
    const float v = mlp_forward_host(w.data(), H, feats.data() + i * LF);
    if (best < 0 || v < best_v) {
      best = cands[i];
      best_v = v;
    }
  }
  return best;
}

}  // namespace tnq

using namespace tnq;

extern "C" {

int32_t tnq_learned_features(void) { return LF; }

size_t tnq_learned_param_count(int32_t hidden) {
  return (size_t)hidden * LF + hidden + (size_t)hidden * hidden + hidden + hidden + 1;
}

tnq_status tnq_learned_set_weights(const float* params, int32_t hidden) {
  if (hidden < 0 || hidden > 4096 || (hidden > 0 && !params)) {
    set_error("bad learned weights");
    return TNQ_EINVAL;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (hidden == 0) {
    g_w.clear();
    g_hidden = 0;
    return TNQ_OK;
  }
  g_w.assign(params, params + tnq_learned_param_count(hidden));
  g_hidden = hidden;
  return TNQ_OK;
}

tnq_status tnq_learned_dataset(int32_t n_qubits, const tnq_gate* gates, size_t n_gates, int32_t ordering,
                               int32_t max_steps, float* feats, float* labels, int32_t* step, int32_t* cand,
                               size_t cap, size_t* out_n) {
  if (!gates || !out_n || max_steps < 0) {
    set_error("NULL argument");
    return TNQ_EINVAL;
  }
  try {
    std::vector<GateIn> gi(n_gates);
    for (size_t i = 0; i < n_gates; ++i) {
      gi[i].kind = gates[i].kind;
      gi[i].q0 = gates[i].q0;
      gi[i].q1 = gates[i].q1;
      std::memcpy(gi[i].m, gates[i].m, sizeof(gi[i].m));
    }
    Network net;
    std::string err = build_network(n_qubits, gi.data(), n_gates, net);
    if (!err.empty()) {
      set_error(err);
      return TNQ_EINVAL;
    }
    Graph g = network_graph(net);
    std::vector<int> order = greedy_order(g, ordering);
    TreeDecomposition td = tree_decomposition(g, order);
    size_t n = 0;
    for (int p = 0; p < max_steps && !order.empty(); ++p) {
      std::vector<float> f;
      std::vector<int> cands = candidate_features(g, order, td, p, f);
      const double before = log2_cost(g, order, p);
      for (size_t i = 0; i < cands.size(); ++i) {
        // exact cost after deleting candidate i
        Graph g2 = g;
        delete_vertex(g2, cands[i]);
        std::vector<int> o2;
        for (int v : order)
          if (v != cands[i]) o2.push_back(v);
        if (n < cap) {
          std::copy(f.begin() + i * LF, f.begin() + (i + 1) * LF, feats + n * LF);
          labels[n] = (float)(log2_cost(g2, o2, p + 1) - before);
          step[n] = p;
          if (cand) cand[n] = cands[i];
        }
        ++n;
      }
      // continue along the tree-trimming choice (Algorithm 2, Section III.B)
      std::vector<int> pos(g.n, -1);
      for (size_t i = 0; i < order.size(); ++i) pos[order[i]] = (int)i;
      const int u = score_tree_trimming(td, pos, nullptr);
      if (u < 0) break;
      delete_vertex(g, u);
      order.erase(std::find(order.begin(), order.end(), u));
      td_remove_vertex(td, u);
    }
    *out_n = n;
    if (n > cap) {
      set_error("dataset capacity too small");
      return TNQ_EINVAL;
    }
    return TNQ_OK;
  } catch (const std::exception& e) {
    set_error(e.what());
    return TNQ_EINVAL;
  }
}

// Host forward pass of the MLP (the planner's inference), for N feature rows.
tnq_status tnq_learned_predict_host(const float* params, int32_t hidden, const float* x, size_t n, float* out) {
  if (!params || !x || !out || hidden <= 0) {
    set_error("NULL argument");
    return TNQ_EINVAL;
  }
  for (size_t i = 0; i < n; ++i) out[i] = mlp_forward_host(params, hidden, x + i * LF);
  return TNQ_OK;
}

}  // extern "C"
