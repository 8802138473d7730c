// plan.hpp -- the opaque tnq_plan behind the C-ABI.
#pragma once
#include <map>
#include <memory>
#include <mutex>
#include <string>

#include "../../include/tnq.h"
#include "graph.hpp"
#include "program.hpp"

namespace tnq {
struct DeviceState;  // per-device tables and cached graphs (runtime.cu)
void destroy_device_state(DeviceState* s);
void set_error(const std::string& msg);
}  // namespace tnq

namespace tnq {
// (Re)compiles the plan's bucket program for its order and sliced set: GEMM
// chains with K >= 2^gemm_min_k_log2 (split precision only), leaf absorption,
// fused chains with tile_low forced output variables. Drops device state.
void rebuild_program(tnq_plan* P, int gemm_min_k_log2, int tile_low);
}  // namespace tnq

struct tnq_plan {
  tnq_plan_opts opts{};
  tnq::Network net;
  tnq::Graph graph;
  std::vector<int> order_full;   // greedy order before slicing (free ids)
  int tau_full = 0;
  std::vector<int> mu;           // sliced free ids, bit j of s = mu[j]
  std::vector<int> order;        // reduced order pi~
  int tau = 0;
  tnq::Program prog;
  double amp_scale_log2 = 0;     // amplitude *= 2^amp_scale_log2 (undoes the sqrt2 scaling)
  int gemm_min_k_log2 = 4;       // GEMM cut-over the program was compiled with
  mutable std::mutex layout_mu;
  mutable std::map<std::pair<int, int>, size_t> layout_bytes;  // (mode, batch) -> workspace bytes
  mutable std::mutex dev_mu;
  mutable tnq::DeviceState* dev = nullptr;
  ~tnq_plan() {
    if (dev) tnq::destroy_device_state(dev);
  }
};
