// program.hpp -- circuit network and compiled bucket program of a plan.
//
// Network (Section II.A): variables are wire segments (q, k); a non-diagonal
// one-qubit gate U adds U[v_new, v_old], a diagonal gate a tensor on the
// current variable (self-loop), CZ a tensor (-1)^(ab) on two current
// variables. Input segments are fixed to 0 and output segments to the
// bitstring; what is left is the free-variable graph the planner orders and
// slices.
//
// Bucket program (Eq. 2): in the reduced order pi~ every tensor joins the
// bucket of its earliest variable; bucket u multiplies its tensors and sums
// u out; the result joins the bucket of its earliest remaining variable, or
// becomes one of the slice's scalar factors when no variable is left.
#pragma once
#include <complex>
#include <cstdint>
#include <string>
#include <vector>

#include "graph.hpp"

namespace tnq {

enum VarKind { VAR_FREE = 0, VAR_IN = 1, VAR_OUT = 2, VAR_INOUT = 3 };

struct Var {
  int q = 0, seg = 0;
  int kind = VAR_FREE;
  int free_id = -1;  // index among free variables
};

// A network tensor over nv two-valued network variables: entry index
// sum_x a_x 2^x for values a_x of var[x]. Circuit gates have nv <= 2 (entry
// (a, b) at a + 2b; val always holds 4 entries); a general network's tensor
// has its indices' binary digits as variables and 2^nv entries. Non-diagonal
// gates with a 1/sqrt2 prefactor (H, X^1/2, Y^1/2) are stored multiplied by
// sqrt2; the plan keeps the count of such factors and applies 2^(-count/2) to
// the amplitude in FP64. A general tensor is stored divided by 2^e (its
// largest |entry| in [0.5, 1)); the plan applies 2^(sum of e) in FP64.
struct GateTensor {
  int nv = 0;
  std::vector<int> var;
  std::vector<std::complex<float>> val;
  GateTensor() : var(2, -1), val(4) {}
};

// Most binary variables one tensor of a general network may have (2^16 entries).
constexpr int LEAF_VMAX = 16;

struct Network {
  int n_qubits = 0;
  std::vector<Var> vars;
  std::vector<GateTensor> tensors;
  std::vector<int> free_vars;  // network var id of each free variable
  int n_sqrt2 = 0;             // number of 1/sqrt2 factors taken out of gate values
  long long leaf_exp = 0;      // general networks: sum of the exponents taken out of the tensors
  std::vector<int> inout_qubits;  // qubits whose input segment is also the output
  // General network (tnq_plan_from_network): no qubits or wires; variable
  // (q, seg) is binary digit seg of index q, whose dimension is index_dim[q].
  bool general = false;
  std::vector<int> index_dim;
};

struct GateIn {
  int kind, q0, q1;
  double m[8];
};

// Returns an empty string on success, else an error message.
std::string build_network(int n_qubits, const GateIn* gates, size_t n_gates, Network& out);

// General closed network (Section II.A for indices of any dimension L): index
// i has dims[i] values and becomes ceil(log2 dims[i]) binary variables (its
// digits); tensor t lists its indices at idx[off[t] .. off[t+1]) and its
// entries, complex128 (re, im) pairs in row-major order over that list (the
// first index varies slowest), at data[2 * data_off[t] ...], where data_off
// is the running sum of the tensors' entry counts. Entries whose digits spell
// a value >= dims[i] are zero. Returns an empty string on success.
std::string build_general_network(int n_indices, const int32_t* dims, size_t n_tensors, const int64_t* off,
                                  const int32_t* idx, const double* data, Network& out);

// Free-variable graph of the network (vertices = free ids).
Graph network_graph(const Network& net);

constexpr int KMAX = 8;  // most inputs one bucket kernel multiplies

// Tensor of the bucket program: a leaf (gate tensor restricted by the fixed
// variables) or a bucket result. `vars` are free ids sorted by position in the
// reduced order: bit i of an entry index is the value of vars[i].
struct PTensor {
  std::vector<int> vars;
  int leaf_gate = -1;   // network tensor index for leaves
  int producer = -1;    // bucket index for results
  int consumer = -1;    // bucket index that reads it (-1: a final scalar)
  bool dep_slice = false, dep_bits = false;
  bool wide_range = false;  // leaf with a nonzero entry of magnitude outside [2^-4, 2^4]
  int rank() const { return (int)vars.size(); }
};

struct PBucket {
  int u = -1;                // eliminated free id (-1: product-only step)
  bool sum = true;           // false: product of the inputs without summing (splits a wide bucket)
  std::vector<int> inputs;   // tensor ids
  int output = -1;           // tensor id
  int r = 0;                 // variables of the product (bag size)
  int k = 0;                 // tensors multiplied
};

// A chain of buckets b_1 -> b_2 -> ... -> b_m (each result consumed by the
// next) executed as one kernel: a block fixes the tile variables and runs the
// m eliminations over the local variables in shared memory, so the chain's
// intermediate results never reach HBM. Exact: Sum_{u_1..u_m} of the product
// of every tensor the chain reads (Eq. 2 applied m times, regrouped).
constexpr int GL_MAX = 13;   // local variables of a group (stage outputs have <= 12 local bits)
constexpr int GM_MAX = 8;    // buckets per group
constexpr int GL_OUT_MIN = 8;  // output variables a group keeps local (>= one entry per thread in the last stage)
constexpr int GIN_MAX = 16;  // tensors a group reads from memory
constexpr int GEMM_SIDE_MAX = 16;  // small tensors folded into one GEMM operand
constexpr int GEMM_BITS_MAX = 16;  // variables in one of a GEMM group's batch / row / column / summed sets

struct FusedGroup {
  std::vector<int> buckets;     // chain order; the group runs at the last bucket's position
  // GEMM form (tensor cores): the chain's product is Sum_K A[S,X,K] B[S,Y,K]
  // with small tensors folded into A or B
  bool gemm = false;
  int ga = -1, gb = -1;                   // the two large operands
  std::vector<int> a_side, b_side;        // small tensors multiplied into A / B
  std::vector<int> kvars, svars, xvars, yvars;  // summed, batch, row and column variables (by position)
  std::vector<int> local_vars;  // L: the eliminated variables + the earliest output variables, by position
  std::vector<int> tile_vars;   // H: the other output variables, by position
  std::vector<int> ext_inputs;  // tensors read from memory, in stage order
  int output = -1;              // result of the last bucket
};

struct Program {
  std::vector<PTensor> tensors;
  std::vector<PBucket> buckets;
  std::vector<FusedGroup> groups;
  std::vector<int> group_of;        // per bucket: group index or -1
  std::vector<int> leaves;          // tensor ids of leaves with at least one free variable
  std::vector<int> scalar_leaves;   // network tensor ids fully fixed (rank 0)
  std::vector<int> finals;          // tensor ids of rank-0 bucket results
  double flops_per_slice = 0, bytes_per_slice = 0;
  double bytes_unfused = 0;  // bytes_per_slice with no fused group
  int max_bag = 0;
  int tile_low = 64;         // output variables a fused chain always keeps local (fuse_chains' tile shape)
};

// GEMM pass: chains whose product is a batched contraction of two tensors of
// rank >= min_rank over >= min_k_log2 summed variables (every further bucket
// eliminates a variable both hold and adds only rank <= 2 tensors whose
// variables lie in one of them) become GEMM groups. Run before fuse_chains.
void find_gemm_chains(Program& prog, const std::vector<int>& order, int min_k_log2, int min_rank);

// Replaces the program's fused groups (recomputes group_of and bytes_per_slice).
void set_groups(Program& prog, const std::vector<FusedGroup>& groups);

// Compiles the bucket program for the reduced order (free ids) and sliced set.
Program compile_program(const Network& net, const std::vector<int>& order, const std::vector<int>& mu);

// Recomputes flops_per_slice, bytes_per_slice (every bucket unfused) and max_bag.
void count_costs(Program& prog);

// Leaf absorption: a gate tensor L (rank <= 2, not wide-range) of bucket b
// whose variables all lie in another input T of b, where T is the result of an
// earlier bucket p with a smaller bag (r_p < r_b), is multiplied into bucket p
// instead of b. Exact: L does not hold p's eliminated variable, so
// Sum_{u_p} L * (product of p) = L * Sum_{u_p} (product of p) (Eq. 2, by
// distributivity), and b's product is unchanged. Each move saves
// 2^r_b - 2^r_p complex multiplies per slice. Buckets in GEMM groups are left
// alone; L must not depend on the slice or the bitstring unless T does. L
// gains u_p as a variable it is constant in, so that every input of a bucket
// keeps the bucket's eliminated variable as its first (bit 0) variable. Runs
// after find_gemm_chains and before fuse_chains; returns the number of moves
// and refreshes the costs.
int absorb_leaves(Program& prog);

// Fusion pass (stages inside a group are not renormalised, so chains that
// read a wide-range leaf stay unfused): chains of summing buckets whose results are at least
// 2^min_rank entries become fused groups when no new variable enters along
// the chain (the group's product space stays the first bucket's bag) and the
// chain fits GM_MAX / GIN_MAX / GL_MAX. Updates bytes_per_slice. min_rank <= 0
// disables fusion.
void fuse_chains(Program& prog, const std::vector<int>& order, int min_rank);

// Bucket index at which a tensor is produced / consumed once groups are
// formed (a group's buckets all count as its last bucket); -1 / n_buckets for
// leaves / final scalars. `internal` tensors (inside a group) are never stored.
struct Liveness {
  std::vector<int> lo, hi;
  std::vector<char> internal;
};
Liveness tensor_liveness(const Program& prog);

}  // namespace tnq
