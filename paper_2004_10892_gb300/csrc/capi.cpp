// capi.cpp -- host-side C-ABI entry points: errors, planning, plan queries and
// the graph-level algorithms (Algorithms 1, 2, 4 and the Section III scores).
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <exception>
#include <iterator>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "../../include/tnq.h"
#include "plan.hpp"

namespace tnq {
static thread_local std::string g_last_error;
void set_error(const std::string& msg) { g_last_error = msg; }
int learned_propose(void* ctx, const Graph& g, const std::vector<int>& order, const TreeDecomposition& td, int p);
void reset_device_state(const tnq_plan& P);

void rebuild_program(tnq_plan* P, int gemm_min_k_log2, int tile_low) {
  const tnq_plan_opts& o = P->opts;
  P->prog = compile_program(P->net, P->order, P->mu);
  P->prog.tile_low = tile_low;
  P->gemm_min_k_log2 = gemm_min_k_log2;
  if (o.precision != TNQ_PREC_C64) find_gemm_chains(P->prog, P->order, gemm_min_k_log2, 8);
  if (o.leaf_absorb) absorb_leaves(P->prog);
  fuse_chains(P->prog, P->order, o.fuse_min_rank);
  reset_device_state(*P);
}
}  // namespace tnq

using namespace tnq;

#define TNQ_TRY(...)                                         \
  try {                                                      \
    __VA_ARGS__                                              \
  } catch (const std::bad_alloc&) {                          \
    set_error("host allocation failed");                     \
    return TNQ_ENOMEM;                                       \
  } catch (const std::exception& e) {                        \
    set_error(e.what());                                     \
    return TNQ_EINVAL;                                       \
  }

extern "C" {

const char* tnq_status_string(tnq_status s) {
  switch (s) {
    case TNQ_OK: return "ok";
    case TNQ_EINVAL: return "invalid argument";
    case TNQ_ENOMEM: return "out of memory";
    case TNQ_ECUDA: return "CUDA error";
    case TNQ_ETIMEOUT: return "device wait timed out";
    case TNQ_EUNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

const char* tnq_last_error(void) { return g_last_error.c_str(); }

const char* tnq_version(void) { return "tnq 0.1 (sm_103a)"; }

void tnq_plan_opts_default(tnq_plan_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->slicer = TNQ_SLICER_TREE_TRIMMING;
  o->max_bag_log2 = 0;
  o->min_p = 0;
  o->max_p = 0;
  o->seed = 0;
  o->precision = TNQ_PREC_C64;
  o->gemm_min_k_log2 = 0;
  o->ordering = TNQ_ORDER_MIN_FILL;
  o->td_rebuild = 0;
  o->fuse_min_rank = 12;
  o->leaf_absorb = 1;
}

static bool valid_opts(const tnq_plan_opts& o) {
  return !(o.slicer < 0 || o.slicer > TNQ_SLICER_BETWEENNESS || o.min_p < 0 || o.max_p < o.min_p ||
           o.max_p > 62 || o.max_bag_log2 < 0 || o.max_bag_log2 > 40 || o.precision < 0 ||
           o.precision > TNQ_PREC_SPLIT_TF32 || o.ordering < 0 || o.ordering > TNQ_ORDER_MIN_DEGREE ||
           o.fuse_min_rank < 0 || o.fuse_min_rank > 40 || o.leaf_absorb < 0 || o.leaf_absorb > 1 ||
           o.reorder_every < 0 || o.order_trials < 0 || o.order_trials > 4096);
}

// Planning shared by circuits and general networks, once P->net is built:
// the free-variable graph, greedy orders (order_trials of them), greedy
// mu-treewidth deletion (Algorithm 2), and the compiled bucket program with
// its GEMM chains, leaf absorption and fused chains.
static void plan_network(tnq_plan* P, const tnq_plan_opts& o) {
  P->graph = network_graph(P->net);
  // order_trials > 1: also try greedy orders with seeded random ties and keep
  // the trial whose sliced plan has the lowest cost 2^p * sum over steps 2^bag
  // (bag limit met first; the earliest trial among equals); trial 0 is the
  // deterministic order. Trials are independent and run on host threads
  // (TNQ_PLAN_THREADS caps their number); the choice does not depend on it.
  const int trials = std::max(1, o.order_trials);
  struct Trial {
    std::vector<int> ord, mu, order;
    int tau = 0;
    double cost = 0;
    bool fits = false;
  };
  std::vector<Trial> tr(trials);
  auto run_trial = [&](int trial) {
    uint64_t rs = (o.seed ^ 0x9E3779B97F4A7C15ull) + (uint64_t)trial;
    Trial& T = tr[trial];
    T.ord = greedy_order(P->graph, o.ordering, trial ? &rs : nullptr);
    DeletionResult R = greedy_deletion(P->graph, T.ord, o.slicer, o.min_p, o.max_p, o.max_bag_log2, o.seed,
                                       o.td_rebuild != 0,
                                       o.slicer == TNQ_SLICER_LEARNED ? &learned_propose : nullptr, nullptr,
                                       o.reorder_every, o.ordering);
    Graph reduced = P->graph;
    for (int v : R.mu) delete_vertex(reduced, v);
    std::vector<int> bags;
    T.tau = treewidth_of_order(reduced, R.reduced_order, &bags);
    int max_bag = 0;
    for (int b : bags) {
      T.cost += std::ldexp(1.0, b);
      max_bag = std::max(max_bag, b);
    }
    T.cost = std::ldexp(T.cost, (int)R.mu.size());
    T.fits = o.max_bag_log2 <= 0 || max_bag <= o.max_bag_log2;
    T.mu = std::move(R.mu);
    T.order = std::move(R.reduced_order);
  };
  int nth = std::min(trials, std::max(1, (int)std::thread::hardware_concurrency()));
  if (const char* e = std::getenv("TNQ_PLAN_THREADS")) nth = std::max(1, std::min(nth, std::atoi(e)));
  if (nth <= 1) {
    for (int t = 0; t < trials; ++t) run_trial(t);
  } else {
    // nth - 1 helper threads and this one take trials from a shared counter
    // (if a helper cannot be started, the others still run every trial)
    std::atomic<int> next(0);
    std::vector<std::exception_ptr> err(nth);
    auto work = [&](int w) {
      try {
        for (int t; (t = next.fetch_add(1)) < trials;) run_trial(t);
      } catch (...) {
        err[w] = std::current_exception();
      }
    };
    std::vector<std::thread> pool;
    for (int w = 1; w < nth; ++w) {
      try {
        pool.emplace_back(work, w);
      } catch (const std::exception&) {
        break;
      }
    }
    work(0);
    for (auto& th : pool) th.join();
    for (auto& e : err)
      if (e) std::rethrow_exception(e);
  }
  int best = 0;
  for (int t = 1; t < trials; ++t)
    if ((tr[t].fits && !tr[best].fits) || (tr[t].fits == tr[best].fits && tr[t].cost < tr[best].cost)) best = t;
  P->order_full = std::move(tr[best].ord);
  P->mu = std::move(tr[best].mu);
  P->order = std::move(tr[best].order);
  P->tau = tr[best].tau;
  P->tau_full = treewidth_of_order(P->graph, P->order_full);
  rebuild_program(P, o.gemm_min_k_log2 > 0 ? o.gemm_min_k_log2 : 4, 64);
  P->amp_scale_log2 = -0.5 * P->net.n_sqrt2 + (double)P->net.leaf_exp;
}

tnq_status tnq_plan_from_circuit(int32_t n_qubits, const tnq_gate* gates, size_t n_gates,
                                 const tnq_plan_opts* opts, tnq_plan** out_plan) {
  if (!out_plan) { set_error("out_plan is NULL"); return TNQ_EINVAL; }
  *out_plan = nullptr;
  if (!gates && n_gates) { set_error("gates is NULL"); return TNQ_EINVAL; }
  tnq_plan_opts o;
  tnq_plan_opts_default(&o);
  if (opts) o = *opts;
  if (!valid_opts(o)) {
    set_error("invalid plan options");
    return TNQ_EINVAL;
  }
  TNQ_TRY({
    std::unique_ptr<tnq_plan> P(new tnq_plan());
    P->opts = o;
    std::vector<GateIn> gi(n_gates);
    for (size_t i = 0; i < n_gates; ++i) {
      gi[i].kind = gates[i].kind;
      gi[i].q0 = gates[i].q0;
      gi[i].q1 = gates[i].q1;
      std::memcpy(gi[i].m, gates[i].m, sizeof(gi[i].m));
    }
    std::string err = build_network(n_qubits, gi.data(), n_gates, P->net);
    if (!err.empty()) { set_error(err); return TNQ_EINVAL; }
    plan_network(P.get(), o);
    *out_plan = P.release();
    return TNQ_OK;
  })
}

tnq_status tnq_plan_from_network(int32_t n_indices, const int32_t* dims, size_t n_tensors,
                                 const int64_t* tensor_offsets, const int32_t* tensor_indices,
                                 const double* tensor_data, const tnq_plan_opts* opts, tnq_plan** out_plan) {
  if (!out_plan) { set_error("out_plan is NULL"); return TNQ_EINVAL; }
  *out_plan = nullptr;
  if ((n_indices > 0 && !dims) || (n_tensors > 0 && (!tensor_offsets || !tensor_data)) ||
      (n_tensors > 0 && tensor_offsets[n_tensors] > 0 && !tensor_indices)) {
    set_error("NULL argument");
    return TNQ_EINVAL;
  }
  if (n_tensors == 0) { set_error("a network needs at least one tensor"); return TNQ_EINVAL; }
  if (tensor_offsets[0] != 0) { set_error("tensor_offsets[0] must be 0"); return TNQ_EINVAL; }
  tnq_plan_opts o;
  tnq_plan_opts_default(&o);
  if (opts) o = *opts;
  if (!valid_opts(o)) {
    set_error("invalid plan options");
    return TNQ_EINVAL;
  }
  TNQ_TRY({
    std::unique_ptr<tnq_plan> P(new tnq_plan());
    P->opts = o;
    std::string err = build_general_network(n_indices, dims, n_tensors, tensor_offsets, tensor_indices,
                                            tensor_data, P->net);
    if (!err.empty()) { set_error(err); return TNQ_EINVAL; }
    plan_network(P.get(), o);
    *out_plan = P.release();
    return TNQ_OK;
  })
}

void tnq_plan_destroy(tnq_plan* plan) { delete plan; }

tnq_status tnq_plan_info_get(const tnq_plan* P, tnq_plan_info* out) {
  if (!P || !out) { set_error("NULL argument"); return TNQ_EINVAL; }
  std::memset(out, 0, sizeof(*out));
  out->n_qubits = P->net.n_qubits;
  out->n_free_vars = (int32_t)P->net.free_vars.size();
  out->n_leaf_tensors = (int32_t)(P->prog.leaves.size() + P->prog.scalar_leaves.size());
  out->n_buckets = (int32_t)P->order.size();
  out->p = (int32_t)P->mu.size();
  out->tau_full = P->tau_full;
  out->tau = P->tau;
  out->max_bag = P->prog.max_bag;
  out->n_slices = 1ull << P->mu.size();
  out->flops_per_slice = P->prog.flops_per_slice;
  out->bytes_per_slice = P->prog.bytes_per_slice;
  // largest live set of one slice: simulate the bucket sequence
  {
    double live = 0, peak = 0;
    for (int t : P->prog.leaves) live += std::ldexp(8.0, P->prog.tensors[t].rank());
    peak = live;
    for (const auto& b : P->prog.buckets) {
      live += std::ldexp(8.0, P->prog.tensors[b.output].rank());
      peak = std::max(peak, live);
      for (int t : b.inputs) live -= std::ldexp(8.0, P->prog.tensors[t].rank());
    }
    out->peak_bytes_per_slice = peak;
  }
  out->total_flops = std::ldexp(P->prog.flops_per_slice, (int)P->mu.size());
  out->n_gemm_buckets = 0;
  out->n_fused_groups = 0;
  for (const auto& g : P->prog.groups) {
    if (g.gemm) out->n_gemm_buckets += (int32_t)g.buckets.size();
    else out->n_fused_groups += 1;
  }
  return TNQ_OK;
}

tnq_status tnq_plan_order(const tnq_plan* P, int32_t* qubit, int32_t* segment) {
  if (!P || !qubit || !segment) { set_error("NULL argument"); return TNQ_EINVAL; }
  for (size_t i = 0; i < P->order.size(); ++i) {
    const Var& v = P->net.vars[P->net.free_vars[P->order[i]]];
    qubit[i] = v.q;
    segment[i] = v.seg;
  }
  return TNQ_OK;
}

tnq_status tnq_plan_sliced(const tnq_plan* P, int32_t* qubit, int32_t* segment) {
  if (!P || (!P->mu.empty() && (!qubit || !segment))) { set_error("NULL argument"); return TNQ_EINVAL; }
  for (size_t j = 0; j < P->mu.size(); ++j) {
    const Var& v = P->net.vars[P->net.free_vars[P->mu[j]]];
    qubit[j] = v.q;
    segment[j] = v.seg;
  }
  return TNQ_OK;
}

tnq_status tnq_plan_buckets(const tnq_plan* P, int32_t* bag, int32_t* k, int32_t* gemm) {
  if (!P) { set_error("NULL plan"); return TNQ_EINVAL; }
  // one entry per summing bucket (product-only splits fold into their bucket)
  size_t i = 0;
  int extra_k = 0;
  for (size_t bi = 0; bi < P->prog.buckets.size(); ++bi) {
    const auto& b = P->prog.buckets[bi];
    if (!b.sum) { extra_k += b.k - 1; continue; }
    const int g = P->prog.group_of.empty() ? -1 : P->prog.group_of[bi];
    if (gemm) gemm[i] = (g >= 0 && P->prog.groups[g].gemm) ? 1 : 0;
    if (bag) bag[i] = b.r;
    if (k) k[i] = b.k + extra_k;
    extra_k = 0;
    ++i;
  }
  return TNQ_OK;
}

tnq_status tnq_plan_tuning(const tnq_plan* P, int32_t* gemm_min_k_log2, int32_t* tile_low) {
  if (!P) { set_error("NULL plan"); return TNQ_EINVAL; }
  if (gemm_min_k_log2) *gemm_min_k_log2 = P->gemm_min_k_log2;
  if (tile_low) *tile_low = P->prog.tile_low;
  return TNQ_OK;
}

tnq_status tnq_plan_set_tuning(tnq_plan* P, int32_t gemm_min_k_log2, int32_t tile_low) {
  if (!P) { set_error("NULL plan"); return TNQ_EINVAL; }
  if (gemm_min_k_log2 < 1 || gemm_min_k_log2 > 16 || tile_low < 0 || tile_low > 64) {
    set_error("gemm_min_k_log2 must be in [1, 16] and tile_low in [0, 64]");
    return TNQ_EINVAL;
  }
  TNQ_TRY({
    rebuild_program(P, gemm_min_k_log2, tile_low);
    return TNQ_OK;
  })
}

// ---- graph-level API ------------------------------------------------------
static bool read_graph(int32_t n, size_t n_edges, const int32_t* edges, Graph& g) {
  if (n < 0 || n > (1 << 20) || (n_edges && !edges)) { set_error("bad graph"); return false; }
  g = Graph(n);
  for (size_t e = 0; e < n_edges; ++e) {
    int a = edges[2 * e], b = edges[2 * e + 1];
    if (a < 0 || a >= n || b < 0 || b >= n) { set_error("edge endpoint out of range"); return false; }
    g.add_edge(a, b);
  }
  return true;
}

static bool read_order(int32_t n, const int32_t* order, std::vector<int>& out) {
  if (n && !order) { set_error("order is NULL"); return false; }
  std::vector<char> seen(n, 0);
  out.assign(order, order + n);
  for (int v : out) {
    if (v < 0 || v >= n || seen[v]) { set_error("order is not a permutation"); return false; }
    seen[v] = 1;
  }
  return true;
}

tnq_status tnq_graph_treewidth(int32_t n, size_t n_edges, const int32_t* edges, const int32_t* order,
                               int32_t* out_tau, int32_t* out_bag_sizes) {
  if (!out_tau) { set_error("out_tau is NULL"); return TNQ_EINVAL; }
  TNQ_TRY({
    Graph g;
    std::vector<int> o;
    if (!read_graph(n, n_edges, edges, g) || !read_order(n, order, o)) return TNQ_EINVAL;
    std::vector<int> sizes;
    *out_tau = treewidth_of_order(g, o, &sizes);
    if (out_bag_sizes) std::copy(sizes.begin(), sizes.end(), out_bag_sizes);
    return TNQ_OK;
  })
}

tnq_status tnq_graph_order(int32_t n, size_t n_edges, const int32_t* edges, int32_t method,
                           int32_t* out_order) {
  if (!out_order || method < 0 || method > 1) { set_error("bad arguments"); return TNQ_EINVAL; }
  TNQ_TRY({
    Graph g;
    if (!read_graph(n, n_edges, edges, g)) return TNQ_EINVAL;
    auto o = greedy_order(g, method);
    std::copy(o.begin(), o.end(), out_order);
    return TNQ_OK;
  })
}

tnq_status tnq_graph_tree_decomposition(int32_t n, size_t n_edges, const int32_t* edges,
                                        const int32_t* order, int32_t bag_cap, int32_t vert_cap,
                                        int32_t* out_nb, int32_t* bag_offsets, int32_t* bag_vertices,
                                        int32_t* parent) {
  if (!out_nb || !bag_offsets || !bag_vertices || !parent) { set_error("NULL output"); return TNQ_EINVAL; }
  TNQ_TRY({
    Graph g;
    std::vector<int> o;
    if (!read_graph(n, n_edges, edges, g) || !read_order(n, order, o)) return TNQ_EINVAL;
    TreeDecomposition td = tree_decomposition(g, o);
    int nb = (int)td.bags.size(), nv = 0;
    for (auto& b : td.bags) nv += (int)b.size();
    *out_nb = nb;
    if (nb > bag_cap || nv > vert_cap) { set_error("tree decomposition capacity too small"); return TNQ_EINVAL; }
    int off = 0;
    for (int b = 0; b < nb; ++b) {
      bag_offsets[b] = off;
      for (int v : td.bags[b]) bag_vertices[off++] = v;
      parent[b] = td.parent[b];
    }
    bag_offsets[nb] = off;
    return TNQ_OK;
  })
}

tnq_status tnq_graph_greedy_deletion(int32_t n, size_t n_edges, const int32_t* edges, const int32_t* order,
                                     int32_t m, int32_t slicer, uint64_t seed, int32_t td_rebuild,
                                     int32_t reorder_every, int32_t* out_mu, int32_t* out_tau) {
  if (m < 0 || m > n || (m && (!out_mu || !out_tau)) || slicer < 0 || slicer > TNQ_SLICER_BETWEENNESS ||
      reorder_every < 0) {
    set_error("bad arguments");
    return TNQ_EINVAL;
  }
  TNQ_TRY({
    Graph g;
    std::vector<int> o;
    if (!read_graph(n, n_edges, edges, g) || !read_order(n, order, o)) return TNQ_EINVAL;
    DeletionResult R = greedy_deletion(g, o, slicer, m, m, 0, seed, td_rebuild != 0,
                                       slicer == TNQ_SLICER_LEARNED ? &learned_propose : nullptr, nullptr,
                                       reorder_every, ORDER_MIN_FILL);
    for (size_t j = 0; j < R.mu.size(); ++j) {
      out_mu[j] = R.mu[j];
      out_tau[j] = R.tau_after[j];
    }
    return TNQ_OK;
  })
}

tnq_status tnq_circuit_graph(int32_t n_qubits, const tnq_gate* gates, size_t n_gates, size_t cap,
                             int32_t* out_n, size_t* out_n_edges, int32_t* edges) {
  if ((!gates && n_gates) || !out_n || !out_n_edges) { set_error("NULL argument"); return TNQ_EINVAL; }
  TNQ_TRY({
    std::vector<GateIn> gi(n_gates);
    for (size_t i = 0; i < n_gates; ++i) {
      gi[i].kind = gates[i].kind;
      gi[i].q0 = gates[i].q0;
      gi[i].q1 = gates[i].q1;
      std::memcpy(gi[i].m, gates[i].m, sizeof(gi[i].m));
    }
    Network net;
    std::string err = build_network(n_qubits, gi.data(), n_gates, net);
    if (!err.empty()) { set_error(err); return TNQ_EINVAL; }
    const Graph g = network_graph(net);
    size_t ne = 0;
    for (int a = 0; a < g.n; ++a)
      for (int b = a + 1; b < g.n; ++b)
        if (g.has(a, b)) {
          if (ne < cap && edges) {
            edges[2 * ne] = a;
            edges[2 * ne + 1] = b;
          }
          ++ne;
        }
    *out_n = g.n;
    *out_n_edges = ne;
    if (ne > cap) { set_error("edge capacity too small"); return TNQ_EINVAL; }
    return TNQ_OK;
  })
}

tnq_status tnq_graph_betweenness(int32_t n, size_t n_edges, const int32_t* edges, double* out_scores) {
  if (!out_scores) { set_error("out_scores is NULL"); return TNQ_EINVAL; }
  TNQ_TRY({
    Graph g;
    if (!read_graph(n, n_edges, edges, g)) return TNQ_EINVAL;
    std::vector<int> all(n);
    for (int v = 0; v < n; ++v) all[v] = v;
    const std::vector<double> cb = betweenness(g, all);
    std::copy(cb.begin(), cb.end(), out_scores);
    return TNQ_OK;
  })
}

}  // extern "C"

// Internal (not in include/tnq.h): bucket structure for analysis and tests.
// Per bucket 12 ints: r, k, output rank, sum flag, then the ranks of up to
// 8 inputs (-1 past k); *n gets the bucket count. Returns 1 if cap is short.
extern "C" int tnq_internal_bucket_detail(const tnq_plan* P, int32_t* out, int cap, int32_t* n) {
  if (!P || !n) return 1;
  const auto& prog = P->prog;
  *n = (int32_t)prog.buckets.size();
  if (cap < *n * 12) return 1;
  for (size_t i = 0; i < prog.buckets.size(); ++i) {
    const auto& b = prog.buckets[i];
    int32_t* o = out + 12 * i;
    o[0] = b.r;
    o[1] = b.k;
    o[2] = prog.tensors[b.output].rank();
    o[3] = b.sum ? 1 : 0;
    for (int j = 0; j < 8; ++j) o[4 + j] = j < b.k ? prog.tensors[b.inputs[j]].rank() : -1;
  }
  return 0;
}

// Internal: per bucket, the bucket that consumes its result (-1 for a final
// scalar) and the number of variables of the union of the two bags.
extern "C" int tnq_internal_bucket_chain(const tnq_plan* P, int32_t* consumer, int32_t* union_size, int cap) {
  if (!P) return 1;
  const auto& prog = P->prog;
  if (cap < (int)prog.buckets.size()) return 1;
  std::vector<int> pos(P->net.free_vars.size(), -1);
  for (size_t i = 0; i < prog.buckets.size(); ++i) {
    const auto& b = prog.buckets[i];
    const int c = prog.tensors[b.output].consumer;
    consumer[i] = c;
    std::vector<int> u;
    for (int t : b.inputs) u.insert(u.end(), prog.tensors[t].vars.begin(), prog.tensors[t].vars.end());
    if (c >= 0)
      for (int t : prog.buckets[c].inputs) u.insert(u.end(), prog.tensors[t].vars.begin(), prog.tensors[t].vars.end());
    std::sort(u.begin(), u.end());
    u.erase(std::unique(u.begin(), u.end()), u.end());
    union_size[i] = (int)u.size();
  }
  return 0;
}

// Internal analysis: for every summing bucket with exactly two inputs of rank
// >= min_rank (the rest rank <= 2), follows the chain of consumers while each
// next bucket eliminates a variable shared by both operands and adds only
// small tensors; prints batch/M/N/K bit counts of the resulting product
// Sum_K A[S,X,K] B[S,Y,K]. Returns the number of candidates printed.
extern "C" int tnq_internal_gemm_candidates(const tnq_plan* P, int min_rank) {
  if (!P) return -1;
  const auto& prog = P->prog;
  int n = 0;
  for (size_t i = 0; i < prog.buckets.size(); ++i) {
    const auto& b = prog.buckets[i];
    if (!b.sum) continue;
    std::vector<int> big;
    bool small_rest = true;
    for (int t : b.inputs) {
      if (prog.tensors[t].rank() >= min_rank) big.push_back(t);
      else if (prog.tensors[t].rank() > 2) small_rest = false;
    }
    if (big.size() != 2 || !small_rest) continue;
    std::vector<int> A = prog.tensors[big[0]].vars, B = prog.tensors[big[1]].vars;
    std::sort(A.begin(), A.end());
    std::sort(B.begin(), B.end());
    std::vector<int> S;
    std::set_intersection(A.begin(), A.end(), B.begin(), B.end(), std::back_inserter(S));
    int k = 1;
    int cur = (int)i;
    std::vector<int> K{b.u};
    while (true) {
      const int c = prog.tensors[prog.buckets[cur].output].consumer;
      if (c < 0) break;
      const auto& cb = prog.buckets[c];
      bool ok = std::binary_search(S.begin(), S.end(), cb.u);
      for (int t : cb.inputs)
        if (t != prog.buckets[cur].output && prog.tensors[t].rank() > 2) ok = false;
      if (!ok) break;
      K.push_back(cb.u);
      ++k;
      cur = c;
    }
    const int s = (int)S.size() - k;
    std::fprintf(stderr, "bucket %zu r=%d: A rank %d, B rank %d, shared %zu -> batch 2^%d M 2^%d N 2^%d K 2^%d\n", i, b.r,
                 (int)A.size(), (int)B.size(), S.size(), s, (int)A.size() - (int)S.size(), (int)B.size() - (int)S.size(), k);
    ++n;
  }
  return n;
}
