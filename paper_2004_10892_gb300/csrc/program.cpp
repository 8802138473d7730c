// program.cpp -- circuit network (Section II.A) and bucket program (Eq. 2).
#include "program.hpp"

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <iterator>

namespace tnq {

namespace {
enum { G_H = 0, G_X12 = 1, G_Y12 = 2, G_T = 3, G_CZ = 4, G_CNOT = 5, G_U1 = 6 };
using cf = std::complex<float>;

int new_var(Network& net, int q, int seg) {
  Var v;
  v.q = q;
  v.seg = seg;
  v.kind = seg == 0 ? VAR_IN : VAR_FREE;
  net.vars.push_back(v);
  return (int)net.vars.size() - 1;
}

// Non-diagonal one-qubit gate given as sqrt2-scaled (or raw, for U1) entries
// m[row][col]: tensor over (v_new = bit 0, v_old = bit 1).
void add_nondiag(Network& net, std::vector<int>& cur, std::vector<int>& seg, int q, const cf m[2][2]) {
  GateTensor t;
  t.nv = 2;
  t.var[1] = cur[q];
  t.var[0] = new_var(net, q, ++seg[q]);
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) t.val[a + 2 * b] = m[a][b];
  cur[q] = t.var[0];
  net.tensors.push_back(t);
}

void add_cz(Network& net, const std::vector<int>& cur, int a, int b) {
  GateTensor t;
  t.nv = 2;
  t.var[0] = cur[a];
  t.var[1] = cur[b];
  t.val[0] = 1.f;
  t.val[1] = 1.f;
  t.val[2] = 1.f;
  t.val[3] = -1.f;
  net.tensors.push_back(t);
}
}  // namespace

std::string build_network(int n_qubits, const GateIn* gates, size_t n_gates, Network& net) {
  if (n_qubits < 1 || n_qubits > 4096) return "n_qubits must be in [1, 4096]";
  net = Network();
  net.n_qubits = n_qubits;
  std::vector<int> cur(n_qubits), seg(n_qubits, 0);
  for (int q = 0; q < n_qubits; ++q) cur[q] = new_var(net, q, 0);
  // sqrt2-scaled matrices: rows = output value, columns = input value
  const cf Hs[2][2] = {{1.f, 1.f}, {1.f, -1.f}};
  const cf Xs[2][2] = {{cf(1.f, 0.f), cf(0.f, -1.f)}, {cf(0.f, -1.f), cf(1.f, 0.f)}};
  const cf Ys[2][2] = {{1.f, -1.f}, {1.f, 1.f}};
  for (size_t g = 0; g < n_gates; ++g) {
    const GateIn& G = gates[g];
    const bool two = (G.kind == G_CZ || G.kind == G_CNOT);
    if (G.kind < 0 || G.kind > G_U1) return "gate " + std::to_string(g) + ": unknown kind";
    if (G.q0 < 0 || G.q0 >= n_qubits) return "gate " + std::to_string(g) + ": qubit out of range";
    if (two && (G.q1 < 0 || G.q1 >= n_qubits || G.q1 == G.q0))
      return "gate " + std::to_string(g) + ": bad second qubit";
    switch (G.kind) {
      case G_H: add_nondiag(net, cur, seg, G.q0, Hs); net.n_sqrt2 += 1; break;
      case G_X12: add_nondiag(net, cur, seg, G.q0, Xs); net.n_sqrt2 += 1; break;
      case G_Y12: add_nondiag(net, cur, seg, G.q0, Ys); net.n_sqrt2 += 1; break;
      case G_U1: {
        cf m[2][2];
        for (int a = 0; a < 2; ++a)
          for (int b = 0; b < 2; ++b) {
            double re = G.m[2 * (2 * a + b)], im = G.m[2 * (2 * a + b) + 1];
            if (!std::isfinite(re) || !std::isfinite(im)) return "gate " + std::to_string(g) + ": non-finite U1";
            m[a][b] = cf((float)re, (float)im);
          }
        add_nondiag(net, cur, seg, G.q0, m);
        break;
      }
      case G_T: {
        GateTensor t;
        t.nv = 1;
        t.var[0] = cur[G.q0];
        t.val[0] = 1.f;
        t.val[1] = cf((float)std::cos(M_PI / 4), (float)std::sin(M_PI / 4));
        net.tensors.push_back(t);
        break;
      }
      case G_CZ: add_cz(net, cur, G.q0, G.q1); break;
      case G_CNOT:
        add_nondiag(net, cur, seg, G.q1, Hs);
        add_cz(net, cur, G.q0, G.q1);
        add_nondiag(net, cur, seg, G.q1, Hs);
        net.n_sqrt2 += 2;
        break;
    }
  }
  for (int q = 0; q < n_qubits; ++q) {
    Var& v = net.vars[cur[q]];
    if (v.kind == VAR_IN) {
      v.kind = VAR_INOUT;
      net.inout_qubits.push_back(q);
    } else {
      v.kind = VAR_OUT;
    }
  }
  for (size_t i = 0; i < net.vars.size(); ++i)
    if (net.vars[i].kind == VAR_FREE) {
      net.vars[i].free_id = (int)net.free_vars.size();
      net.free_vars.push_back((int)i);
    }
  return "";
}

std::string build_general_network(int n_indices, const int32_t* dims, size_t n_tensors, const int64_t* off,
                                  const int32_t* idx, const double* data, Network& net) {
  if (n_indices < 0 || n_indices > (1 << 24)) return "n_indices must be in [0, 2^24]";
  if (n_tensors > ((size_t)1 << 24)) return "too many tensors";
  net = Network();
  net.general = true;
  net.index_dim.assign(dims, dims + n_indices);
  std::vector<int> first(n_indices + 1, 0);  // first binary variable of each index
  for (int i = 0; i < n_indices; ++i) {
    if (dims[i] < 1 || dims[i] > (1 << LEAF_VMAX)) return "index " + std::to_string(i) + ": dimension outside [1, 2^16]";
    int b = 0;
    while ((1 << b) < dims[i]) ++b;
    first[i + 1] = first[i] + b;
    for (int j = 0; j < b; ++j) {
      Var v;
      v.q = i;
      v.seg = j;
      v.kind = VAR_FREE;
      net.vars.push_back(v);
    }
  }
  std::vector<char> used(n_indices, 0);
  size_t data_pos = 0;
  for (size_t t = 0; t < n_tensors; ++t) {
    if (off[t + 1] < off[t] || off[t] < 0) return "tensor " + std::to_string(t) + ": bad index offsets";
    const int rank = (int)(off[t + 1] - off[t]);
    const int32_t* ti = idx + off[t];
    GateTensor g;
    g.var.clear();
    size_t entries = 1;
    for (int k = 0; k < rank; ++k) {
      const int i = ti[k];
      if (i < 0 || i >= n_indices) return "tensor " + std::to_string(t) + ": index id out of range";
      for (int k2 = 0; k2 < k; ++k2)
        if (ti[k2] == i) return "tensor " + std::to_string(t) + ": index " + std::to_string(i) + " listed twice";
      used[i] = 1;
      entries *= (size_t)dims[i];
      for (int v = first[i]; v < first[i + 1]; ++v) g.var.push_back(v);
    }
    g.nv = (int)g.var.size();
    if (g.nv > LEAF_VMAX) return "tensor " + std::to_string(t) + ": more than 2^16 entries after binary encoding";
    g.val.assign(std::max<size_t>(4, (size_t)1 << g.nv), std::complex<float>(0.f, 0.f));
    // largest |entry| -> exponent e with max / 2^e in [0.5, 1)
    double mx = 0;
    for (size_t e = 0; e < entries; ++e) {
      const double re = data[2 * (data_pos + e)], im = data[2 * (data_pos + e) + 1];
      if (!std::isfinite(re) || !std::isfinite(im)) return "tensor " + std::to_string(t) + ": non-finite entry";
      mx = std::max(mx, std::max(std::fabs(re), std::fabs(im)));
    }
    int ex = 0;
    if (mx > 0) std::frexp(mx, &ex);
    net.leaf_exp += ex;
    // entry of binary assignment a: the digits of each index spell its value x_k
    for (size_t a = 0; a < ((size_t)1 << g.nv); ++a) {
      size_t row = 0, bitpos = 0;
      bool pad = false;
      for (int k = 0; k < rank; ++k) {
        const int i = ti[k];
        const int nb = first[i + 1] - first[i];
        const size_t x = (a >> bitpos) & (((size_t)1 << nb) - 1);
        bitpos += nb;
        if (x >= (size_t)dims[i]) pad = true;
        row = row * (size_t)dims[i] + x;
      }
      if (pad) continue;
      const double re = std::ldexp(data[2 * (data_pos + row)], -ex), im = std::ldexp(data[2 * (data_pos + row) + 1], -ex);
      g.val[a] = std::complex<float>((float)re, (float)im);
    }
    data_pos += entries;
    net.tensors.push_back(g);
  }
  for (int i = 0; i < n_indices; ++i)
    if (!used[i]) return "index " + std::to_string(i) + " appears in no tensor";
  for (size_t i = 0; i < net.vars.size(); ++i) {
    net.vars[i].free_id = (int)net.free_vars.size();
    net.free_vars.push_back((int)i);
  }
  return "";
}

Graph network_graph(const Network& net) {
  Graph g((int)net.free_vars.size());
  for (const auto& t : net.tensors) {
    for (int x = 0; x < t.nv; ++x)
      for (int y = x + 1; y < t.nv; ++y) {
        int a = net.vars[t.var[x]].free_id, b = net.vars[t.var[y]].free_id;
        if (a >= 0 && b >= 0) g.add_edge(a, b);
      }
  }
  return g;
}

Program compile_program(const Network& net, const std::vector<int>& order, const std::vector<int>& mu) {
  Program P;
  const int nf = (int)net.free_vars.size();
  std::vector<int> pos(nf, -1);
  std::vector<char> sliced(nf, 0);
  for (size_t i = 0; i < order.size(); ++i) pos[order[i]] = (int)i;
  for (int v : mu) sliced[v] = 1;
  auto by_pos = [&](int a, int b) { return pos[a] < pos[b]; };
  std::vector<std::vector<int>> bucket_of(order.size());

  auto place = [&](int tid) {
    const PTensor& t = P.tensors[tid];
    bucket_of[pos[t.vars[0]]].push_back(tid);
  };

  for (size_t gi = 0; gi < net.tensors.size(); ++gi) {
    const GateTensor& gt = net.tensors[gi];
    PTensor t;
    t.leaf_gate = (int)gi;
    for (int a = 0; a < gt.nv; ++a) {
      const Var& v = net.vars[gt.var[a]];
      if (v.kind == VAR_OUT) t.dep_bits = true;
      if (v.kind == VAR_FREE) {
        if (sliced[v.free_id]) t.dep_slice = true;
        else t.vars.push_back(v.free_id);
      }
    }
    if (t.vars.empty()) {
      P.scalar_leaves.push_back((int)gi);
      continue;
    }
    // (a general network's tensors are stored with their largest |entry| in
    // [0.5, 1), so none is wide-range)
    if (!net.general)
      for (int e = 0; e < 4; ++e) {
        const float m = std::abs(gt.val[e]);
        if (m != 0.f && (m < 0.0625f || m > 16.f)) t.wide_range = true;
      }
    std::sort(t.vars.begin(), t.vars.end(), by_pos);
    t.vars.erase(std::unique(t.vars.begin(), t.vars.end()), t.vars.end());
    P.tensors.push_back(t);
    P.leaves.push_back((int)P.tensors.size() - 1);
    place((int)P.tensors.size() - 1);
  }

  auto add_bucket = [&](int u, bool sum, const std::vector<int>& inputs) -> int {
    PBucket b;
    b.u = u;
    b.sum = sum;
    b.inputs = inputs;
    b.k = (int)inputs.size();
    std::vector<int> uni;
    PTensor out;
    for (int tid : inputs) {
      const PTensor& t = P.tensors[tid];
      uni.insert(uni.end(), t.vars.begin(), t.vars.end());
      out.dep_slice |= t.dep_slice;
      out.dep_bits |= t.dep_bits;
    }
    std::sort(uni.begin(), uni.end(), by_pos);
    uni.erase(std::unique(uni.begin(), uni.end()), uni.end());
    b.r = (int)uni.size();
    for (int v : uni)
      if (!sum || v != u) out.vars.push_back(v);
    const int bidx = (int)P.buckets.size();
    out.producer = bidx;
    P.tensors.push_back(out);
    b.output = (int)P.tensors.size() - 1;
    for (int tid : inputs) P.tensors[tid].consumer = bidx;
    P.buckets.push_back(b);
    return b.output;
  };

  for (size_t i = 0; i < order.size(); ++i) {
    const int u = order[i];
    std::vector<int> inputs = bucket_of[i];
    if (inputs.empty()) continue;  // cannot happen for circuits: every free variable sits in its gate
    // A bucket wider than KMAX first multiplies its lowest-rank tensors
    // together (a product without summation, still containing u).
    while ((int)inputs.size() > KMAX) {
      std::stable_sort(inputs.begin(), inputs.end(),
                       [&](int a, int b) { return P.tensors[a].rank() < P.tensors[b].rank(); });
      std::vector<int> head(inputs.begin(), inputs.begin() + KMAX);
      std::vector<int> rest(inputs.begin() + KMAX, inputs.end());
      int t = add_bucket(u, false, head);
      rest.insert(rest.begin(), t);
      inputs = rest;
    }
    int out = add_bucket(u, true, inputs);
    if (P.tensors[out].vars.empty()) P.finals.push_back(out);
    else place(out);
  }
  count_costs(P);
  return P;
}

void count_costs(Program& P) {
  P.flops_per_slice = 0;
  P.bytes_per_slice = 0;
  P.max_bag = 0;
  for (const PBucket& b : P.buckets) {
    double in_elems = 0;
    for (int tid : b.inputs) in_elems += std::ldexp(1.0, P.tensors[tid].rank());
    const double full = std::ldexp(1.0, b.r);
    P.flops_per_slice += 6.0 * (b.k - 1) * full + (b.sum ? 2.0 * (full / 2) : 0.0);
    P.bytes_per_slice += 8.0 * (in_elems + std::ldexp(1.0, P.tensors[b.output].rank()));
    P.max_bag = std::max(P.max_bag, b.r);
  }
}

int absorb_leaves(Program& P) {
  const int nb = (int)P.buckets.size();
  if (P.group_of.size() != (size_t)nb) P.group_of.assign(nb, -1);
  auto in_group = [&](int b) { return P.group_of[b] >= 0; };
  int moved = 0;
  for (int b = nb - 1; b >= 0; --b) {
    if (in_group(b)) continue;
    PBucket& B = P.buckets[b];
    for (size_t li = 0; li < B.inputs.size();) {
      const int L = B.inputs[li];
      const PTensor& tl = P.tensors[L];
      int best = -1;
      if (tl.leaf_gate >= 0 && tl.rank() <= 2 && !tl.wide_range && B.inputs.size() > 1) {
        std::vector<int> lv = tl.vars;
        std::sort(lv.begin(), lv.end());
        for (int T : B.inputs) {
          const PTensor& tt = P.tensors[T];
          const int p = tt.producer;
          if (T == L || p < 0 || in_group(p) || P.buckets[p].k >= KMAX || P.buckets[p].u < 0) continue;
          if (P.buckets[p].r >= B.r) continue;
          if ((tl.dep_slice && !tt.dep_slice) || (tl.dep_bits && !tt.dep_bits)) continue;
          std::vector<int> tv = tt.vars;
          std::sort(tv.begin(), tv.end());
          if (!std::includes(tv.begin(), tv.end(), lv.begin(), lv.end())) continue;
          if (best < 0 || P.buckets[p].r < P.buckets[P.tensors[best].producer].r) best = T;
        }
      }
      if (best < 0) {
        ++li;
        continue;
      }
      const int p = P.tensors[best].producer;
      // every input of a bucket holds its eliminated variable as bit 0: give L
      // u_p as a variable it does not depend on (u_p precedes all of p's variables)
      std::vector<int>& v = P.tensors[L].vars;
      if (std::find(v.begin(), v.end(), P.buckets[p].u) == v.end()) v.insert(v.begin(), P.buckets[p].u);
      P.buckets[p].inputs.push_back(L);
      P.buckets[p].k = (int)P.buckets[p].inputs.size();
      P.tensors[L].consumer = p;
      B.inputs.erase(B.inputs.begin() + li);
      B.k = (int)B.inputs.size();
      ++moved;
    }
  }
  if (moved) {
    count_costs(P);
    P.bytes_unfused = P.bytes_per_slice;
    set_groups(P, std::vector<FusedGroup>(P.groups));
  }
  return moved;
}

}  // namespace tnq

namespace tnq {

static std::vector<int> bag_of(const Program& P, const PBucket& b) {
  std::vector<int> u;
  for (int t : b.inputs) u.insert(u.end(), P.tensors[t].vars.begin(), P.tensors[t].vars.end());
  std::sort(u.begin(), u.end());
  u.erase(std::unique(u.begin(), u.end()), u.end());
  return u;
}

// Tile shape of a fused chain: the local variables L are the chain's
// eliminated ones plus n_local - |elim| of its output variables; the others
// are tile variables. The earliest `keep_low` output variables are always
// local, so the output is written in runs of 2^keep_low consecutive entries.
// The rest are chosen greedily (ties to the earliest position) to minimise
// sum_j 2^|vars_j & L| over the chain's external inputs j: the entries of its
// operands one tile touches, i.e. what a block reads from L2 per tile (an
// input holding no local variable becomes a per-block constant). With
// keep_low >= the number of output variables this is the earliest-position
// choice. keep_low is the program's tile_low.
static void choose_tile(const Program& P, FusedGroup& g, const std::vector<int>& outv, int n_local) {
  const int keep_low = P.tile_low;
  std::vector<char> local(outv.size(), 0);
  int n = (int)g.local_vars.size();
  for (size_t i = 0; i < outv.size() && n < n_local && (int)i < keep_low; ++i, ++n) local[i] = 1;
  // per external input: which output variables it holds, and its local count so far
  std::vector<std::vector<char>> holds;
  std::vector<int> cnt;
  for (int t : g.ext_inputs) {
    const auto& tv = P.tensors[t].vars;
    std::vector<char> h(outv.size(), 0);
    int c = 0;
    for (size_t i = 0; i < outv.size(); ++i) {
      h[i] = std::find(tv.begin(), tv.end(), outv[i]) != tv.end();
      if (h[i] && local[i]) ++c;
    }
    for (int u : g.local_vars) c += std::find(tv.begin(), tv.end(), u) != tv.end();
    holds.push_back(h);
    cnt.push_back(c);
  }
  for (; n < n_local; ++n) {
    int best = -1;
    double best_cost = 0;
    for (size_t i = 0; i < outv.size(); ++i) {
      if (local[i]) continue;
      double cost = 0;
      for (size_t j = 0; j < holds.size(); ++j) cost += std::ldexp(1.0, cnt[j] + (holds[j][i] ? 1 : 0));
      if (best < 0 || cost < best_cost) {
        best = (int)i;
        best_cost = cost;
      }
    }
    if (best < 0) break;
    local[best] = 1;
    for (size_t j = 0; j < holds.size(); ++j) cnt[j] += holds[j][best];
  }
  for (size_t i = 0; i < outv.size(); ++i)
    if (local[i]) g.local_vars.push_back(outv[i]);
    else g.tile_vars.push_back(outv[i]);
}

void fuse_chains(Program& P, const std::vector<int>& order, int min_rank) {
  const int nb = (int)P.buckets.size();
  if (P.bytes_unfused == 0) P.bytes_unfused = P.bytes_per_slice;
  std::vector<FusedGroup> gemms;
  for (const auto& g : P.groups)
    if (g.gemm) gemms.push_back(g);
  P.groups = gemms;
  P.group_of.assign(nb, -1);
  for (size_t gi = 0; gi < P.groups.size(); ++gi)
    for (int b : P.groups[gi].buckets) P.group_of[b] = (int)gi;
  if (min_rank <= 0) {
    set_groups(P, gemms);
    return;
  }
  std::vector<int> pos(order.size() + 1, 0);
  {
    int maxv = 0;
    for (int v : order) maxv = std::max(maxv, v);
    pos.assign(maxv + 1, -1);
    for (size_t i = 0; i < order.size(); ++i) pos[order[i]] = (int)i;
  }
  auto by_pos = [&](int a, int b) { return pos[a] < pos[b]; };
  for (int i = 0; i < nb; ++i) {
    if (P.group_of[i] >= 0 || !P.buckets[i].sum) continue;
    std::vector<int> chain{i};
    std::vector<int> U = bag_of(P, P.buckets[i]);
    int n_ext = P.buckets[i].k;
    while ((int)chain.size() < GM_MAX) {
      const PBucket& last = P.buckets[chain.back()];
      if (P.tensors[last.output].rank() < min_rank) break;
      const int c = P.tensors[last.output].consumer;
      if (c < 0 || !P.buckets[c].sum || P.group_of[c] >= 0) break;
      std::vector<int> bc = bag_of(P, P.buckets[c]), nu;
      std::set_union(U.begin(), U.end(), bc.begin(), bc.end(), std::back_inserter(nu));
      if (nu.size() != U.size()) break;  // a new variable would enter the product space
      const int ext = n_ext + P.buckets[c].k - 1;
      if (ext > GIN_MAX) break;
      bool wide = false;
      for (int t : P.buckets[c].inputs) wide |= P.tensors[t].wide_range;
      if (chain.size() == 1)
        for (int t : P.buckets[chain[0]].inputs) wide |= P.tensors[t].wide_range;
      if (wide) break;
      if ((int)chain.size() + 1 + GL_OUT_MIN > GL_MAX) break;  // keep >= GL_OUT_MIN output variables local
      chain.push_back(c);
      n_ext = ext;
    }
    if (chain.size() < 2) continue;
    FusedGroup g;
    g.buckets = chain;
    g.output = P.buckets[chain.back()].output;
    std::vector<int> elim;
    for (int b : chain) elim.push_back(P.buckets[b].u);
    for (size_t s = 0; s < chain.size(); ++s)
      for (int t : P.buckets[chain[s]].inputs)
        if (!(s > 0 && t == P.buckets[chain[s - 1]].output)) g.ext_inputs.push_back(t);
    std::vector<int> outv = P.tensors[g.output].vars;  // already sorted by position
    std::vector<int> U2 = U;
    std::sort(U2.begin(), U2.end(), by_pos);
    const int n_local = std::min<int>(GL_MAX, (int)U2.size());
    g.local_vars = elim;
    choose_tile(P, g, outv, n_local);
    std::sort(g.local_vars.begin(), g.local_vars.end(), by_pos);
    const int gi = (int)P.groups.size();
    for (int b : chain) P.group_of[b] = gi;
    P.groups.push_back(g);
  }
  set_groups(P, std::vector<FusedGroup>(P.groups));
}

void find_gemm_chains(Program& P, const std::vector<int>& order, int min_k_log2, int min_rank) {
  const int nb = (int)P.buckets.size();
  if (P.bytes_unfused == 0) P.bytes_unfused = P.bytes_per_slice;
  if (P.group_of.size() != (size_t)nb) P.group_of.assign(nb, -1);
  int maxv = 0;
  for (int v : order) maxv = std::max(maxv, v);
  std::vector<int> pos(maxv + 1, -1);
  for (size_t i = 0; i < order.size(); ++i) pos[order[i]] = (int)i;
  auto by_pos = [&](int a, int b) { return pos[a] < pos[b]; };
  auto sorted = [&](std::vector<int> v) {
    std::sort(v.begin(), v.end());
    return v;
  };
  auto subset = [](const std::vector<int>& a, const std::vector<int>& b) {  // both sorted
    return std::includes(b.begin(), b.end(), a.begin(), a.end());
  };
  std::vector<FusedGroup> found(P.groups);
  for (int i = 0; i < nb; ++i) {
    if (P.group_of[i] >= 0 || !P.buckets[i].sum) continue;
    const PBucket& b0 = P.buckets[i];
    std::vector<int> big, small;
    for (int t : b0.inputs) (P.tensors[t].rank() >= min_rank ? big : small).push_back(t);
    if (big.size() != 2) continue;
    const std::vector<int> Av = sorted(P.tensors[big[0]].vars), Bv = sorted(P.tensors[big[1]].vars);
    std::vector<int> S;
    std::set_intersection(Av.begin(), Av.end(), Bv.begin(), Bv.end(), std::back_inserter(S));
    FusedGroup g;
    g.gemm = true;
    g.ga = big[0];
    g.gb = big[1];
    auto fold = [&](int t) {
      if (P.tensors[t].rank() > 2) return false;
      const std::vector<int> v = sorted(P.tensors[t].vars);
      if (subset(v, Av)) g.a_side.push_back(t);
      else if (subset(v, Bv)) g.b_side.push_back(t);
      else return false;
      return true;
    };
    bool ok = true;
    for (int t : small) ok = ok && fold(t);
    if (!ok || g.a_side.size() > (size_t)GEMM_SIDE_MAX || g.b_side.size() > (size_t)GEMM_SIDE_MAX) continue;
    g.buckets = {i};
    g.kvars = {b0.u};
    int cur = i;
    while (true) {
      const int c = P.tensors[P.buckets[cur].output].consumer;
      if (c < 0 || P.group_of[c] >= 0 || !P.buckets[c].sum) break;
      const PBucket& bc = P.buckets[c];
      if (!std::binary_search(S.begin(), S.end(), bc.u)) break;
      const size_t na = g.a_side.size(), nbs = g.b_side.size();
      bool fits = true;
      for (int t : bc.inputs)
        if (t != P.buckets[cur].output) fits = fits && fold(t);
      if (g.a_side.size() > (size_t)GEMM_SIDE_MAX || g.b_side.size() > (size_t)GEMM_SIDE_MAX) fits = false;
      if (!fits) {
        g.a_side.resize(na);
        g.b_side.resize(nbs);
        break;
      }
      g.buckets.push_back(c);
      g.kvars.push_back(bc.u);
      cur = c;
    }
    if ((int)g.kvars.size() < min_k_log2) continue;
    g.output = P.buckets[g.buckets.back()].output;
    const std::vector<int> K = sorted(g.kvars);
    for (int v : S)
      if (!std::binary_search(K.begin(), K.end(), v)) g.svars.push_back(v);
    for (int v : Av)
      if (!std::binary_search(S.begin(), S.end(), v)) g.xvars.push_back(v);
    for (int v : Bv)
      if (!std::binary_search(S.begin(), S.end(), v)) g.yvars.push_back(v);
    for (auto* v : {&g.kvars, &g.svars, &g.xvars, &g.yvars}) std::sort(v->begin(), v->end(), by_pos);
    // the chain's result holds exactly S' + X + Y
    if (P.tensors[g.output].rank() != (int)(g.svars.size() + g.xvars.size() + g.yvars.size())) continue;
    if (g.xvars.size() > 12 || g.yvars.size() > 12 || g.kvars.size() > 12 ||
        g.svars.size() > (size_t)GEMM_BITS_MAX)
      continue;
    {  // orientation: A rows pad to 128, B's 2^|Y| complex columns to 64; keep the smaller padded product
      auto up = [](long long v, long long a) { return (v + a - 1) / a * a; };
      const long long nx = 1ll << g.xvars.size(), ny = 1ll << g.yvars.size();
      if (up(ny, 128) * up(nx, 64) < up(nx, 128) * up(ny, 64)) {
        std::swap(g.ga, g.gb);
        std::swap(g.a_side, g.b_side);
        std::swap(g.xvars, g.yvars);
      }
    }
    g.ext_inputs = {g.ga, g.gb};
    g.ext_inputs.insert(g.ext_inputs.end(), g.a_side.begin(), g.a_side.end());
    g.ext_inputs.insert(g.ext_inputs.end(), g.b_side.begin(), g.b_side.end());
    g.local_vars = g.kvars;
    const int gi = (int)found.size();
    for (int b : g.buckets) P.group_of[b] = gi;
    found.push_back(g);
  }
  set_groups(P, found);
}

void set_groups(Program& P, const std::vector<FusedGroup>& groups) {
  if (P.bytes_unfused == 0) P.bytes_unfused = P.bytes_per_slice;
  P.groups = groups;
  P.group_of.assign(P.buckets.size(), -1);
  double saved = 0;
  for (size_t gi = 0; gi < P.groups.size(); ++gi) {
    const auto& g = P.groups[gi];
    for (int b : g.buckets) P.group_of[b] = (int)gi;
    // algorithmic bytes: intermediates inside a group are neither written nor read
    for (size_t s = 0; s + 1 < g.buckets.size(); ++s)
      saved += 2 * std::ldexp(8.0, P.tensors[P.buckets[g.buckets[s]].output].rank());
  }
  P.bytes_per_slice = P.bytes_unfused - saved;
}

Liveness tensor_liveness(const Program& P) {
  const int nb = (int)P.buckets.size();
  const int T = (int)P.tensors.size();
  Liveness L;
  L.lo.assign(T, -1);
  L.hi.assign(T, nb);
  L.internal.assign(T, 0);
  auto eff = [&](int b) {
    if (b < 0 || b >= nb || P.group_of.empty() || P.group_of[b] < 0) return b;
    return P.groups[P.group_of[b]].buckets.back();
  };
  for (int t = 0; t < T; ++t) {
    const PTensor& x = P.tensors[t];
    L.lo[t] = eff(x.producer);
    L.hi[t] = x.consumer >= 0 ? eff(x.consumer) : nb;
    if (x.producer >= 0 && !P.group_of.empty() && P.group_of[x.producer] >= 0 &&
        P.groups[P.group_of[x.producer]].output != t)
      L.internal[t] = 1;
  }
  return L;
}

}  // namespace tnq
