// program.cpp -- circuit network (Section II.A) and bucket program (Eq. 2).
#include "program.hpp"

#include <algorithm>
#include <cmath>

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

Graph network_graph(const Network& net) {
  Graph g((int)net.free_vars.size());
  for (const auto& t : net.tensors) {
    if (t.nv < 2) continue;
    int a = net.vars[t.var[0]].free_id, b = net.vars[t.var[1]].free_id;
    if (a >= 0 && b >= 0) g.add_edge(a, b);
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
    double in_elems = 0;
    for (int tid : inputs) {
      P.tensors[tid].consumer = bidx;
      in_elems += std::ldexp(1.0, P.tensors[tid].rank());
    }
    const double full = std::ldexp(1.0, b.r);
    P.flops_per_slice += 6.0 * (b.k - 1) * full + (sum ? 2.0 * (full / 2) : 0.0);
    P.bytes_per_slice += 8.0 * (in_elems + std::ldexp(1.0, P.tensors[b.output].rank()));
    P.max_bag = std::max(P.max_bag, b.r);
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
  return P;
}

}  // namespace tnq
