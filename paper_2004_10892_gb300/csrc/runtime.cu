// runtime.cu -- sm_103a execution of a plan's bucket program.
//
// One call contracts many "items" (a slice s of Eq. 4, or a (bitstring,
// slice) pair) at once: every tensor that depends on the item is stored
// item-major, tensors that do not are stored once (slice-invariant buckets
// run once per batch). Per batch the stream runs
//   leaf init (restrict gate tensors to the item's fixed values, Eq. 4)
//   -> one fused product + sum-out kernel per bucket (Eq. 2)
//   -> per-item scalar products and the FP64 sum over slices (Eq. 5),
// captured once into a CUDA graph and replayed for every batch.
//
// Numbers: tensors are complex64. Every bucket result carries a per-item
// power-of-two exponent e (value = stored * 2^e) and the float bits of its
// largest |re| or |im| (atomicMax in the producing kernel); a consumer scales
// each input by an exact 2^-m so that inputs enter every product with
// magnitude below 1, which keeps 2^-n/2-sized amplitudes far from underflow.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/tnq.h"
#include "gemm_tc.cuh"
#include "plan.hpp"

extern "C" const char* tnq_last_error(void);

namespace tnq {

constexpr int GMAX = 52;  // index bits of one bucket launch (output bits + item bits)
static_assert(GB_SIDE >= GEMM_SIDE_MAX + 1 && GB_BITS >= GEMM_BITS_MAX, "GEMM limits of planner and kernels differ");
constexpr int TPB = 256;  // threads per block of the bucket kernel
constexpr int MAX_ITEM_BITS = 16;
constexpr int HOIST_MAX_BITS = 24;  // largest early-bucket result (2^24 entries; see hoist_levels)

// ---------------------------------------------------------------------------
// device-side records
struct KParams {
  float2* out;
  const float2* in[KMAX];
  long long stride[KMAX][GMAX];  // element stride of each index bit, per input
  int in_meta[KMAX];             // meta row of input j, -1 for leaves (unit scale)
  int in_dep[KMAX];              // 1: input meta is per item
  int out_meta;
  int out_bits;                  // output variables per item
  int G;                         // out_bits + item bits
  int sum;                       // 1: sum over bit 0 of every input (Eq. 2); 0: product only
  int n_var;                     // inputs 0..n_var-1 vary with output bits 0-7; the others do not
  int B;                         // meta row length
  int* meta_e;
  unsigned* meta_m;
};

// One early bucket of a level launch (k_bucket_level): like KParams for an
// item-invariant bucket, with arena byte offsets instead of pointers.
struct HoistDev {
  long long out;                  // arena byte offset of the result
  long long in[KMAX];             // arena byte offsets of the inputs
  long long stride[KMAX][HOIST_MAX_BITS];  // element stride of each index bit (output bits, then item bits), per input
  int in_meta[KMAX];              // meta row of input j, -1 for gate tensors (unit scale)
  int in_dep[KMAX];               // 1: input j's meta row is per item
  int nin, bits, sum, out_meta;   // inputs, index bits, 1: sum over bit 0 (Eq. 2), meta row of the result
  int obits, out_dep;             // output bits per item; 1: the result is per item (items above bit obits)
  int blk0;                       // first block of this bucket in its level's launch
  int nvar;                       // inputs 0..nvar-1 vary with the index's low 8 bits (k_bucket's order)
};

struct LeafDev {
  float2 val[4];      // entries when nv <= 2: (a, b) at a + 2b
  long long tab;      // nv > 2 (general networks): element offset of the 2^nv entries in the leaf value table
  long long off;      // element offset in the arena
  int nv;             // tensor variables (binary; entry index sum_x a_x 2^x)
  int n_free;         // leaf rank
  int dep;            // item-dependent in this configuration
  int pad;
  signed char vkind[LEAF_VMAX];  // 0 free, 1 fixed to 0 (input wire), 2 output bit, 3 sliced
  short varg[LEAF_VMAX];         // free: bit in the leaf; output: qubit; sliced: j
};

// Entry a of a leaf: inline for gates, from the value table for general tensors.
__device__ __forceinline__ float2 leaf_entry(const LeafDev& L, const float2* __restrict__ vals, int a) {
  return L.nv <= 2 ? L.val[a] : vals[L.tab + a];
}

struct FinalDev {
  long long off;
  int meta;
  int dep;
};

// Batch header, rewritten before every batch.
struct BatchHdr {
  unsigned long long item_base;  // global item index of item 0
  unsigned long long item_end;   // one past the last valid global item
  unsigned long long bstr_base;  // global bitstring index of bitstring row 0
  int mode;                      // 0: item = slice of bitstring 0; 1: item = (bitstring << p) | slice
  int p;
  int n_words;                   // 32-bit words per bitstring
  int pad;
};

__device__ __forceinline__ void item_decode(const BatchHdr& h, int item, unsigned long long* slice, int* brow,
                                            bool* valid) {
  unsigned long long gi = h.item_base + (unsigned long long)item;
  *valid = gi < h.item_end;
  if (!*valid) gi = h.item_base;  // padding items recompute a valid item; results are dropped
  if (h.mode == 0) {
    *slice = gi;
    *brow = 0;
  } else {
    *slice = h.p ? (gi & ((1ull << h.p) - 1ull)) : 0ull;
    *brow = (int)((gi >> h.p) - h.bstr_base);
  }
}

__device__ __forceinline__ int bit_of(const unsigned* bits, int n_words, int brow, int q) {
  return (bits[(size_t)brow * n_words + (q >> 5)] >> (q & 31)) & 1u;
}

// K5: restrict every gate tensor to the item's fixed values (input 0, output
// bits, sliced values: Eq. 4).
__global__ void k_leaf_init(const LeafDev* __restrict__ leaves, int n_leaves, const BatchHdr* __restrict__ hdr_p,
                            const unsigned* __restrict__ bits, const float2* __restrict__ vals,
                            float2* __restrict__ arena, int B) {
  const BatchHdr h = *hdr_p;
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)n_leaves * B) return;
  const int li = (int)(idx / B), item = (int)(idx % B);
  const LeafDev L = leaves[li];
  if (!L.dep && item) return;
  unsigned long long slice;
  int brow;
  bool valid;
  item_decode(h, item, &slice, &brow, &valid);
  float2* out = arena + L.off + (L.dep ? ((long long)item << L.n_free) : 0ll);
  // the fixed variables' part of the entry index is the same for every entry
  int a_fixed = 0;
  for (int x = 0; x < L.nv; ++x) {
    int a = 0;
    if (L.vkind[x] == 2) a = bit_of(bits, h.n_words, brow, L.varg[x]);
    else if (L.vkind[x] == 3) a = (int)((slice >> L.varg[x]) & 1ull);
    a_fixed |= a << x;
  }
  for (int e = 0; e < (1 << L.n_free); ++e) {
    int a = a_fixed;
    for (int x = 0; x < L.nv; ++x)
      if (L.vkind[x] == 0) a |= ((e >> L.varg[x]) & 1) << x;
    out[e] = leaf_entry(L, vals, a);
  }
}

// Product of the fully fixed gate tensors and the <x_q|0> factors of wires
// without a non-diagonal gate, per item (FP64).
__global__ void k_scalar_init(const LeafDev* __restrict__ sl, int n_sl, const int* __restrict__ inout_q, int n_inout,
                              const BatchHdr* __restrict__ hdr_p, const unsigned* __restrict__ bits,
                              const float2* __restrict__ vals, double2* __restrict__ item_scalar, int B) {
  const BatchHdr h = *hdr_p;
  int item = blockIdx.x * blockDim.x + threadIdx.x;
  if (item >= B) return;
  unsigned long long slice;
  int brow;
  bool valid;
  item_decode(h, item, &slice, &brow, &valid);
  double re = 1.0, im = 0.0;
  for (int i = 0; i < n_sl; ++i) {
    const LeafDev& L = sl[i];
    int a = 0;
    for (int x = 0; x < L.nv; ++x) {
      if (L.vkind[x] == 2) a |= bit_of(bits, h.n_words, brow, L.varg[x]) << x;
      else if (L.vkind[x] == 3) a |= (int)((slice >> L.varg[x]) & 1ull) << x;
    }
    const float2 v = leaf_entry(L, vals, a);
    const double nr = re * v.x - im * v.y, ni = re * v.y + im * v.x;
    re = nr;
    im = ni;
  }
  for (int i = 0; i < n_inout; ++i)
    if (bit_of(bits, h.n_words, brow, inout_q[i])) re = im = 0.0;
  item_scalar[item] = make_double2(re, im);
}

// Scale 2^-m that brings a tensor whose largest |re|,|im| has float bits
// `mbits` into [0.5, 1); m is returned through *mexp.
__device__ __forceinline__ float scale_of_max(unsigned mbits, int* mexp) {
  if (mbits == 0u) {
    *mexp = 0;
    return 1.f;
  }
  int ex = (int)((mbits >> 23) & 0xffu);
  if (ex == 0) ex = 1;
  int m = ex - 126;
  if (m > 126) m = 126;
  *mexp = m;
  return __int_as_float((127 - m) << 23);
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__device__ __forceinline__ void atomic_max_pos(unsigned* p, float v) {
  const unsigned b = __float_as_uint(v);
  if (b > *reinterpret_cast<volatile unsigned*>(p)) atomicMax(p, b);
}

// K1: one bucket, all items. Element g of the launch = item * 2^out_bits + b'
// of the output; input j's entry for (b', u=0) is at sum_i bit_i(g) * stride[j][i]
// (u=1 is the next element, since u is every input's bit 0). A block covers
// 2^LT consecutive g: bits >= 8 of g go through a shared table per input, bits
// < 8 through a per-thread offset, so each element costs one add per input.
template <int NIN, int LT>
__global__ void __launch_bounds__(TPB, 5) k_bucket(const __grid_constant__ KParams P) {
  constexpr int ITER = (LT > 8) ? (1 << (LT - 8)) : 1;
  __shared__ long long sh_off[NIN][ITER];
  __shared__ float sh_red[TPB / 32];
  __shared__ float4 sh_c[ITER];  // product of the thread-invariant inputs per iteration (pair over u)
  const int t = threadIdx.x;
  const long long g0 = (long long)blockIdx.x << LT;
  const long long total = 1ll << P.G;

  for (int e = t; e < NIN * ITER; e += TPB) {
    const int j = e / ITER, it = e - (e / ITER) * ITER;
    const long long gi = g0 + ((long long)it << 8);
    long long acc = 0;
    for (int i = 8; i < P.G; ++i)
      if ((gi >> i) & 1ll) acc += P.stride[j][i];
    sh_off[j][it] = acc;
  }
  long long tp[NIN];
#pragma unroll
  for (int j = 0; j < NIN; ++j) {
    long long a = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i)
      if (i < P.G && ((t >> i) & 1)) a += P.stride[j][i];
    tp[j] = a;
  }
  __syncthreads();

  const int ob = P.out_bits;
  const bool uniform = (ob >= LT) || (P.G == ob);
  float f[NIN];
  int esum = 0;
  auto load_scales = [&](long long item) {
    esum = 0;
#pragma unroll
    for (int j = 0; j < NIN; ++j) {
      if (P.in_meta[j] < 0) {
        f[j] = 1.f;
      } else {
        const long long row = (long long)P.in_meta[j] * P.B + (P.in_dep[j] ? item : 0ll);
        int m;
        f[j] = scale_of_max(P.meta_m[row], &m);
        esum += P.meta_e[row] + m;
      }
    }
  };
  if (uniform) load_scales(g0 >> ob);
  // thread-invariant inputs (n_var..NIN-1) of a block with one item: their
  // scaled (u = 0, u = 1) product per iteration, once per block
  const bool use_c = uniform && P.n_var < NIN;
  if (use_c) {
    if (t < ITER && g0 + ((long long)t << 8) < total) {
      float2 c0 = make_float2(1.f, 0.f), c1 = make_float2(1.f, 0.f);
#pragma unroll
      for (int j = 0; j < NIN; ++j) {
        if (j < P.n_var) continue;
        const long long idx = sh_off[j][t];
        if (P.sum) {
          const float4 v = __ldg(reinterpret_cast<const float4*>(P.in[j] + idx));
          c0 = cmul(c0, make_float2(v.x * f[j], v.y * f[j]));
          c1 = cmul(c1, make_float2(v.z * f[j], v.w * f[j]));
        } else {
          const float2 v = __ldg(P.in[j] + idx);
          c0 = cmul(c0, make_float2(v.x * f[j], v.y * f[j]));
        }
      }
      sh_c[t] = make_float4(c0.x, c0.y, c1.x, c1.y);
    }
    __syncthreads();
  }
  const int nv = P.n_var;

  const long long omask = (1ll << ob) - 1ll;
  const int lane = t & 31;
  float tmax = 0.f;
  // input 0's pairs of UB iterations are loaded together, ahead of the
  // arithmetic and the stores of those iterations (the stores could alias the
  // loads as far as the compiler knows, so it would not move a later load
  // above an earlier store)
  constexpr int UB = ITER >= 4 ? 4 : ITER;
#pragma unroll 1
  for (int it0 = 0; it0 < ITER; it0 += UB) {
    float4 v0[UB];
    if (P.sum && nv >= 1) {
#pragma unroll
      for (int k = 0; k < UB; ++k) {
        const long long g = g0 + t + ((long long)(it0 + k) << 8);
        v0[k] = g < total ? __ldg(reinterpret_cast<const float4*>(P.in[0] + sh_off[0][it0 + k] + tp[0]))
                          : make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
#pragma unroll
    for (int k = 0; k < UB; ++k) {
      const int it = it0 + k;
      const long long g = g0 + t + ((long long)it << 8);
      const bool valid = g < total;
      const long long item = g >> ob;
      float m = 0.f;
      if (valid) {
        if (!uniform) load_scales(item);
        // the same arithmetic in both forms (so a slice's value does not depend on
        // the batch size): the thread-invariant inputs' product from (1, 0) in
        // input order, then the varying inputs in input order
        float2 r;
        float4 cc;
        if (use_c) {
          cc = sh_c[it];
        } else {
          float2 c0 = make_float2(1.f, 0.f), c1 = make_float2(1.f, 0.f);
#pragma unroll
          for (int j = 0; j < NIN; ++j) {
            if (j < nv) continue;
            const long long idx = sh_off[j][it] + tp[j];  // tp[j]: item bits among the thread bits
            if (P.sum) {
              const float4 v = __ldg(reinterpret_cast<const float4*>(P.in[j] + idx));
              c0 = cmul(c0, make_float2(v.x * f[j], v.y * f[j]));
              c1 = cmul(c1, make_float2(v.z * f[j], v.w * f[j]));
            } else {
              const float2 v = __ldg(P.in[j] + idx);
              c0 = cmul(c0, make_float2(v.x * f[j], v.y * f[j]));
            }
          }
          cc = make_float4(c0.x, c0.y, c1.x, c1.y);
        }
        if (P.sum) {
          float2 a0 = make_float2(cc.x, cc.y), a1 = make_float2(cc.z, cc.w);
#pragma unroll
          for (int j = 0; j < NIN; ++j) {
            if (j >= nv) break;
            const long long idx = sh_off[j][it] + tp[j];
            const float4 v = j == 0 ? v0[k] : __ldg(reinterpret_cast<const float4*>(P.in[j] + idx));
            a0 = cmul(a0, make_float2(v.x * f[j], v.y * f[j]));
            a1 = cmul(a1, make_float2(v.z * f[j], v.w * f[j]));
          }
          r = make_float2(a0.x + a1.x, a0.y + a1.y);
        } else {
          float2 a = make_float2(cc.x, cc.y);
#pragma unroll
          for (int j = 0; j < NIN; ++j) {
            if (j >= nv) break;
            const long long idx = sh_off[j][it] + tp[j];
            const float2 v = __ldg(P.in[j] + idx);
            a = cmul(a, make_float2(v.x * f[j], v.y * f[j]));
          }
          r = a;
        }
        P.out[g] = r;
        m = fmaxf(fabsf(r.x), fabsf(r.y));
        if ((g & omask) == 0) P.meta_e[(long long)P.out_meta * P.B + item] = esum;
      }
      if (uniform) {
        tmax = fmaxf(tmax, m);
      } else {
        // items change every 2^ob elements: reduce within aligned lane groups
        for (int off = 1; off < 32 && off < (1 << min(ob, 5)); off <<= 1)
          m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
        const int grp = 1 << min(ob, 5);
        if (valid && (lane & (grp - 1)) == 0 && m > 0.f)
          atomic_max_pos(&P.meta_m[(long long)P.out_meta * P.B + item], m);
      }
    }
  }
  if (uniform) {
    for (int off = 16; off > 0; off >>= 1) tmax = fmaxf(tmax, __shfl_xor_sync(0xffffffffu, tmax, off));
    if (lane == 0) sh_red[t >> 5] = tmax;
    __syncthreads();
    if (t == 0) {
      float b = 0.f;
      for (int w = 0; w < TPB / 32; ++w) b = fmaxf(b, sh_red[w]);
      if (b > 0.f && g0 < total) atomic_max_pos(&P.meta_m[(long long)P.out_meta * P.B + (g0 >> ob)], b);
    }
  }
}

// K1 for the early buckets of one level (see hoist_levels): every bucket of
// the level in one launch, 256 index entries per block; block b works on the
// bucket whose blk0 is the largest not above b. Item-dependent buckets carry
// the item above their output bits; their scales, exponents and maxima are
// per item, as in k_bucket, and so is the arithmetic order.
__global__ void __launch_bounds__(256) k_bucket_level(const HoistDev* __restrict__ hd, int n, char* arena,
                                                     int* meta_e, unsigned* meta_m, int B) {
  __shared__ int s_b;
  __shared__ long long s_str[KMAX][HOIST_MAX_BITS];
  __shared__ const float2* s_in[KMAX];
  __shared__ float s_f[KMAX];
  __shared__ int s_e;
  __shared__ float s_red[8];
  const int t = threadIdx.x;
  if (t == 0) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (hd[mid].blk0 <= (int)blockIdx.x) lo = mid;
      else hi = mid - 1;
    }
    s_b = lo;
  }
  __syncthreads();
  const HoistDev& H = hd[s_b];
  const int nin = H.nin, bits = H.bits, ob = H.obits;
  const long long g0 = (long long)(blockIdx.x - H.blk0) * 256;
  const bool uniform = ob >= 8 || ob == bits;  // one item for the whole block
  for (int e = t; e < nin * bits; e += 256) s_str[e / bits][e % bits] = H.stride[e / bits][e % bits];
  if (t < nin) s_in[t] = reinterpret_cast<const float2*>(arena + H.in[t]);
  if (uniform && t == 0) {  // the block's item: scales and the output exponent
    const long long item = g0 >> ob;
    int e = 0;
    for (int j = 0; j < nin; ++j) {
      if (H.in_meta[j] < 0) {
        s_f[j] = 1.f;
        continue;
      }
      const long long row = (long long)H.in_meta[j] * B + (H.in_dep[j] ? item : 0ll);
      int m;
      s_f[j] = scale_of_max(meta_m[row], &m);
      e += meta_e[row] + m;
    }
    s_e = e;
  }
  __syncthreads();
  const long long g = g0 + t;
  const long long item = g >> ob;
  float mx = 0.f;
  if (g < (1ll << bits)) {
    // scale of input j for this entry's item
    auto scale = [&](int j) -> float {
      if (uniform) return s_f[j];
      if (H.in_meta[j] < 0) return 1.f;
      int m;
      return scale_of_max(meta_m[(long long)H.in_meta[j] * B + (H.in_dep[j] ? item : 0ll)], &m);
    };
    // the arithmetic order of k_bucket (thread-invariant inputs nvar.. first,
    // then 0..nvar-1), so that a bucket's value does not depend on which
    // kernel runs it
    float2 a0 = make_float2(1.f, 0.f), a1 = make_float2(1.f, 0.f);
    for (int jj = 0; jj < nin; ++jj) {
      const int j = jj < nin - H.nvar ? H.nvar + jj : jj - (nin - H.nvar);
      long long idx = 0;
      for (int i = 0; i < bits; ++i)
        if ((g >> i) & 1ll) idx += s_str[j][i];
      const float fj = scale(j);
      if (H.sum) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(s_in[j] + idx));
        a0 = cmul(a0, make_float2(v.x * fj, v.y * fj));
        a1 = cmul(a1, make_float2(v.z * fj, v.w * fj));
      } else {
        const float2 v = __ldg(s_in[j] + idx);
        a0 = cmul(a0, make_float2(v.x * fj, v.y * fj));
      }
    }
    const float2 r = H.sum ? make_float2(a0.x + a1.x, a0.y + a1.y) : a0;
    reinterpret_cast<float2*>(arena + H.out)[g] = r;
    mx = fmaxf(fabsf(r.x), fabsf(r.y));
    if ((g & ((1ll << ob) - 1ll)) == 0) {  // the item's first entry writes its exponent
      int esum = 0;
      if (uniform) {
        esum = s_e;
      } else {
        for (int j = 0; j < nin; ++j) {
          if (H.in_meta[j] < 0) continue;
          const long long row = (long long)H.in_meta[j] * B + (H.in_dep[j] ? item : 0ll);
          int m;
          scale_of_max(meta_m[row], &m);
          esum += meta_e[row] + m;
        }
      }
      meta_e[(long long)H.out_meta * B + (H.out_dep ? item : 0ll)] = esum;
    }
  }
  if (uniform) {
    for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    if ((t & 31) == 0) s_red[t >> 5] = mx;
    __syncthreads();
    if (t == 0) {
      float b = 0.f;
      for (int w = 0; w < 8; ++w) b = fmaxf(b, s_red[w]);
      if (b > 0.f) atomic_max_pos(&meta_m[(long long)H.out_meta * B + (H.out_dep ? (g0 >> ob) : 0ll)], b);
    }
  } else {
    // items change every 2^ob entries: reduce within aligned lane groups
    const int grp = 1 << (ob < 5 ? ob : 5);
    for (int off = 1; off < grp; off <<= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    if ((t & (grp - 1)) == 0 && mx > 0.f && g < (1ll << bits))
      atomic_max_pos(&meta_m[(long long)H.out_meta * B + (H.out_dep ? item : 0ll)], mx);
  }
}

// ---------------------------------------------------------------------------
// Fused chain of buckets (FusedGroup). A block fixes the tile variables H (and
// the item); stage s eliminates u_s over the local variables in shared memory:
//   stage_s[c] = sum_{u_s} prod_j in_j[c, u_s],
// where in_j is a tensor read from memory at the block's H, or the previous
// stage's buffer. Offsets are linear in the bits of the stage's local index c;
// per varying operand a table holds the offset of each value of bits 0-3,
// bits 4..GTB-1 (the rest of the thread index) and bits GTB..11 (the entry
// counter of the thread) of c, built once per block.
constexpr int GTB = 7;              // log2 threads per k_group block
constexpr int GTPB = 1 << GTB;      // threads per k_group block
constexpr int GT_MID = 16;          // table entries of bits 4..GTB-1 start here
constexpr int GT_HI = GT_MID + (1 << (GTB - 4));  // ... and of bits GTB..GL_MAX-2 here
constexpr int TABW = GT_HI + (1 << (GL_MAX - 1 - GTB));
static_assert(GTB >= 6, "the stage-buffer swizzle assumes >= 64 threads per k_group block");
constexpr int TAIL_MIN = 2, TAIL_MAX = 4;  // stages after the first that group_tail runs in registers
constexpr int GH_MAX = 32;  // tile bits (output variables outside the block; a bag of 2^40 entries has < 32)
constexpr int PAIR_MAX = GIN_MAX + GM_MAX - 1;  // varying (stage, operand) pairs: at most every input of every stage
constexpr int GROUP_SMEM_BYTES = (1 << (GL_MAX - 1)) * 3 / 2 * (int)sizeof(float2);  // regions A + B

struct GIn {
  const float2* ptr;
  long long istride;           // per item (0 if the tensor is item-invariant)
  long long hstride[GH_MAX];   // per tile bit
  int meta;                    // meta row (-1 for leaves)
  int dep;
};

struct GSt {
  int n_in;
  int n_var;                   // inputs 0..n_var-1 vary over the local bits; the rest are per-block constants
  int nbits;                   // local output bits of the stage
  int src[KMAX];               // -1: previous stage buffer, else index into gin
  int cstride[KMAX][GL_MAX];   // element stride of local output bit b, per input
  int ustride[KMAX];           // stride of the eliminated variable, per input
  int q0;                      // offset table of varying input j is pair q0 + j
  int pd;                      // 1: input 0 is the previous stage's buffer at offset 2c (u at bit 0)
  int kinv;                    // 1: the constant inputs n_var.. hold no tile bit (their pair is per item)
  int n_tc;                    // varying inputs n_var-n_tc..n_var-1 hold thread bits only: one pair per thread
};

struct GParams {
  GSt st[GM_MAX];
  GIn gin[GIN_MAX];
  float2* out;
  long long out_istride;
  long long out_hstride[GH_MAX];
  int out_cstride[GL_MAX];
  int n_st, n_gin, n_h, out_meta, out_dep, B;
  int n_pairs;
  int tail;                    // > 0: stages 1..tail run in registers (group_tail) after stage 0
  int lean2;                   // 1: two stages, stage 1 reads stage 0 densely and writes the output (k_group<2>)
  int* meta_e;
  unsigned* meta_m;
};

// Stage buffers in shared memory are stored swizzled: complex entry o sits at
// swz(o), which keeps (u = 0, u = 1) pairs together and permutes the 16-byte
// pairs within each group of 8 (pair p at p ^ ((p >> 3) & 7)). Threads that
// read the pairs of consecutive subtrees (group_tail) then hit distinct banks;
// for entries t + GTPB it the swizzle is swz(t) + GTPB it (GTPB >= 64).
__device__ __forceinline__ int swz(int o) {
  const int p = o >> 1;
  return ((p ^ ((p >> 3) & 7)) << 1) | (o & 1);
}

// One stage of a fused group. Inputs n_var.. do not vary over the block's
// local bits: their (u=0, u=1) pairs, times the stage's power-of-two scales,
// are multiplied once into a constant pair (K = true). Without such inputs
// (K = false) the product starts from the first varying operand and the
// scales multiply the sum. Each thread handles local entries c = t + GTPB it;
// per entry only the NV varying operands are loaded (one 16-byte load each:
// the eliminated variable is bit 0 of every operand), and the last operand's
// multiply is fused with the sum over u.
template <int NV, bool K>
__device__ __forceinline__ void group_stage(const GSt& S, int t, const float2* prev, float2* cur, float2* out,
                                            bool last, const float2* const* s_ptr, float F, const int (*tab)[TABW],
                                            const int* s_out_hi, long long out_base, int out_lo, float* tmax) {
  static_assert(K || NV > 0, "a stage without constant inputs has a varying operand");
  const int nb = S.nbits;
  const int n_hi = nb > GTB ? (1 << (nb - GTB)) : 1;
  const int nent = 1 << nb;
  float2 k0 = make_float2(F, 0.f), k1 = make_float2(F, 0.f);
  if (K) {
    for (int j = NV; j < S.n_in; ++j) {
      const float2* p = S.src[j] < 0 ? prev : s_ptr[S.src[j]];
      const float4 v = *reinterpret_cast<const float4*>(p);
      k0 = cmul(k0, make_float2(v.x, v.y));
      k1 = cmul(k1, make_float2(v.z, v.w));
    }
  }
  const float2* ptr[NV > 0 ? NV : 1];
  int lo[NV > 0 ? NV : 1];
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    const int src = S.src[j];
    ptr[j] = src < 0 ? prev : s_ptr[src];
    lo[j] = tab[j][t & 15] + tab[j][GT_MID + (t >> 4)];
  }
  // operand j's pair at local offset o (the previous stage's buffer is swizzled)
  auto at = [&](int j, int o) -> float4 {
    return *reinterpret_cast<const float4*>(ptr[j] + (S.src[j] < 0 ? swz(o) : o));
  };
#pragma unroll 2
  for (int it = 0; it < n_hi; ++it) {
    const int c = t + (it << GTB);
    if (c < nent) {
      float2 p0 = k0, p1 = k1;
      constexpr int J0 = K ? 0 : 1;
      if (!K) {
        const float4 v = at(0, lo[0] + tab[0][GT_HI + it]);
        p0 = make_float2(v.x, v.y);
        p1 = make_float2(v.z, v.w);
      }
#pragma unroll
      for (int j = J0; j < NV - 1; ++j) {
        const float4 v = at(j, lo[j] + tab[j][GT_HI + it]);
        p0 = cmul(p0, make_float2(v.x, v.y));
        p1 = cmul(p1, make_float2(v.z, v.w));
      }
      float2 r;
      if (NV >= 1 && (K || NV >= 2)) {
        const float4 v = at(NV - 1, lo[NV - 1] + tab[NV - 1][GT_HI + it]);
        float rx = p0.x * v.x;
        rx = fmaf(-p0.y, v.y, rx);
        rx = fmaf(p1.x, v.z, rx);
        rx = fmaf(-p1.y, v.w, rx);
        float ry = p0.x * v.y;
        ry = fmaf(p0.y, v.x, ry);
        ry = fmaf(p1.x, v.w, ry);
        ry = fmaf(p1.y, v.z, ry);
        r = make_float2(rx, ry);
      } else {
        r = make_float2(p0.x + p1.x, p0.y + p1.y);
      }
      if (!K) r = make_float2(r.x * F, r.y * F);
      if (last) {
        out[out_base + out_lo + s_out_hi[it]] = r;
        *tmax = fmaxf(*tmax, fmaxf(fabsf(r.x), fabsf(r.y)));
      } else {
        cur[swz(c)] = r;
      }
    }
  }
}

// Stage with NV = 1..3 varying operands and exactly 2^nbits = GTPB NHI local
// entries (NHI = 1 also covers nbits < GTB: threads past the end compute a
// duplicate entry from in-range offsets, since the tables hold 0 for bits >=
// nbits, and do not store it). Thread t handles entries c = t + GTPB it.
//   * The entry counter runs in blocks of U entries: an operand's offset is
//     the sum of the table values of its set bits, so entry it0 + u of a
//     block is at (offset of it0) + (offset of u) -- one table read per block
//     and operand, the U inner offsets stay in registers.
//   * Each operand's 16-byte loads run PF entries ahead of the arithmetic
//     (global operands through the read-only path); the last block is peeled
//     so that no entry tests whether its prefetch is in range.
//   * PD: operand 0 is the previous stage's buffer read densely (entry c at
//     2c): shared memory at a constant step per entry.
//   * LAST: the stage writes the group's output (global) and its maximum.
// K as in group_stage.
template <bool B>
struct BoolTag {
  static constexpr bool value = B;
};

template <int NV, bool K, int NHI, bool PD, bool LAST>
__device__ __forceinline__ void stage_pf(const GSt& S, int t, const float2* prev, float2* cur, float2* out,
                                         const float2* const* s_ptr, float F, const int (*tab)[TABW],
                                         const int* s_out_hi, long long out_base, int out_lo, float* tmax) {
  static_assert(NV >= 1 && NV <= 3, "one to three varying operands");
  // loads in flight per operand: one entry ahead for one or two operands
  // (more leaves less of the L1 cache to the operands' reuse), two for three
  constexpr int PF = NHI < 2 ? NHI : (NV <= 2 ? 1 : 2);
  constexpr int U = NHI < 4 ? NHI : 4;  // entries per block (a multiple of PF)
  constexpr int NB = NHI / U;
  float2 k0 = make_float2(F, 0.f), k1 = make_float2(F, 0.f);
  if (K) {  // the thread's pairs of inputs NV..n_var-1 (thread bits only), then the block's constants
    for (int j = NV; j < S.n_in; ++j) {
      const int o = j < S.n_var ? tab[j][t & 15] + tab[j][GT_MID + (t >> 4)] : 0;
      const float4 v = __ldg(reinterpret_cast<const float4*>(s_ptr[S.src[j]] + o));
      k0 = cmul(k0, make_float2(v.x, v.y));
      k1 = cmul(k1, make_float2(v.z, v.w));
    }
  }
  const float4* base[NV];  // operand at entry t of block 0
  int ti[NV][U];           // inner offsets (float4 units)
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    if (PD && j == 0) {
      base[0] = reinterpret_cast<const float4*>(prev) + (t ^ ((t >> 3) & 7));  // swizzled pair t
#pragma unroll
      for (int u = 0; u < U; ++u) ti[0][u] = u * GTPB;
    } else {
      base[j] = reinterpret_cast<const float4*>(s_ptr[S.src[j]] + tab[j][t & 15] + tab[j][GT_MID + (t >> 4)]);
#pragma unroll
      for (int u = 0; u < U; ++u) ti[j][u] = tab[j][GT_HI + u] >> 1;
    }
  }
  auto load = [&](int j, const float4* q) -> float4 { return (PD && j == 0) ? *q : __ldg(q); };
  const float4* ob[NV];   // this block
  const float4* obn[NV];  // next block
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    ob[j] = base[j];
    obn[j] = base[j] + ((PD && j == 0) ? U * GTPB : (NB > 1 ? (tab[j][GT_HI + U] >> 1) : 0));
  }
  float4 v[PF][NV];
#pragma unroll
  for (int i = 0; i < PF; ++i)
#pragma unroll
    for (int j = 0; j < NV; ++j) v[i][j] = load(j, ob[j] + ti[j][i]);
  int so[U];
  float2* dst = nullptr;
  if (LAST) {
#pragma unroll
    for (int u = 0; u < U; ++u) so[u] = s_out_hi[u];
    dst = out + out_base + out_lo;
  }
  // one block of U entries; TAIL: the last block (no prefetch past the end)
  auto block = [&](int it0, auto tail_tag) {
    constexpr bool TAIL = decltype(tail_tag)::value;
    const int oh = LAST ? s_out_hi[it0] : 0;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      float4 cv[NV];
#pragma unroll
      for (int j = 0; j < NV; ++j) cv[j] = v[u % PF][j];
      if (!TAIL || u + PF < U) {
#pragma unroll
        for (int j = 0; j < NV; ++j)
          v[u % PF][j] = load(j, u + PF < U ? ob[j] + ti[j][u + PF] : obn[j] + ti[j][u + PF - U]);
      }
      float2 p0 = k0, p1 = k1;
      if (!K) {
        p0 = make_float2(cv[0].x, cv[0].y);
        p1 = make_float2(cv[0].z, cv[0].w);
      }
#pragma unroll
      for (int j = K ? 0 : 1; j < NV - 1; ++j) {
        p0 = cmul(p0, make_float2(cv[j].x, cv[j].y));
        p1 = cmul(p1, make_float2(cv[j].z, cv[j].w));
      }
      float2 r;
      if (K || NV >= 2) {
        const float4 b = cv[NV - 1];
        float rx = p0.x * b.x;
        rx = fmaf(-p0.y, b.y, rx);
        rx = fmaf(p1.x, b.z, rx);
        rx = fmaf(-p1.y, b.w, rx);
        float ry = p0.x * b.y;
        ry = fmaf(p0.y, b.x, ry);
        ry = fmaf(p1.x, b.w, ry);
        ry = fmaf(p1.y, b.z, ry);
        r = make_float2(rx, ry);
      } else {
        r = make_float2(p0.x + p1.x, p0.y + p1.y);
      }
      if (!K) r = make_float2(r.x * F, r.y * F);
      if (NHI > 1 || t < (1 << S.nbits)) {
        if (LAST) {
          dst[oh + so[u]] = r;
          *tmax = fmaxf(*tmax, fmaxf(fabsf(r.x), fabsf(r.y)));
        } else {
          cur[swz(t) + (it0 + u) * GTPB] = r;
        }
      }
    }
  };
#pragma unroll 1
  for (int b = 0; b < NB - 1; ++b) {
    block(b * U, BoolTag<false>{});
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      ob[j] = obn[j];
      if (b + 2 < NB) obn[j] = base[j] + ((PD && j == 0) ? (b + 2) * U * GTPB : (tab[j][GT_HI + (b + 2) * U] >> 1));
    }
  }
  block((NB - 1) * U, BoolTag<true>{});
}

// Dispatch of stage_pf over (NV, K, NHI, PD, LAST); false if the stage has another shape.
template <int NV, bool K, bool PD>
__device__ __forceinline__ bool stage_pf_nhi(const GSt& S, int t, const float2* prev, float2* cur, float2* out,
                                             bool last, const float2* const* s_ptr, float F, const int (*tab)[TABW],
                                             const int* s_out_hi, long long out_base, int out_lo, float* tmax) {
#define TNQ_PF(n)                                                                                          \
  (last ? stage_pf<NV, K, n, PD, true>(S, t, prev, cur, out, s_ptr, F, tab, s_out_hi, out_base, out_lo, tmax) \
        : stage_pf<NV, K, n, PD, false>(S, t, prev, cur, out, s_ptr, F, tab, s_out_hi, out_base, out_lo, tmax))
  static_assert(GL_MAX - 1 - GTB <= 5, "entries per thread above 32");
  switch (S.nbits - GTB) {
    case 5: TNQ_PF(32); return true;
    case 4: TNQ_PF(16); return true;
    case 3: TNQ_PF(8); return true;
    case 2: TNQ_PF(4); return true;
    case 1: TNQ_PF(2); return true;
    default:
      if (S.nbits > GTB) return false;
      TNQ_PF(1);
      return true;
  }
#undef TNQ_PF
}

// Stage 0 of a chain with a register tail: operands from memory, never the
// group's last stage.
template <int NV, bool K>
__device__ __forceinline__ void stage0_pf(const GSt& S, int t, float2* cur, const float2* const* s_ptr, float F,
                                          const int (*tab)[TABW]) {
#define TNQ_PF0(n) stage_pf<NV, K, n, false, false>(S, t, nullptr, cur, nullptr, s_ptr, F, tab, nullptr, 0, 0, nullptr)
  switch (S.nbits - GTB) {
    case 5: TNQ_PF0(32); break;
    case 4: TNQ_PF0(16); break;
    case 3: TNQ_PF0(8); break;
    case 2: TNQ_PF0(4); break;
    case 1: TNQ_PF0(2); break;
    default: TNQ_PF0(1); break;
  }
#undef TNQ_PF0
}

// Stage 1 of a two-stage chain (k_group<2>): operand 0 is stage 0's buffer
// read densely, the stage writes the group's output.
template <int NV, bool K>
__device__ __forceinline__ void stage_last_pd(const GSt& S, int t, const float2* prev, float2* out,
                                              const float2* const* s_ptr, float F, const int (*tab)[TABW],
                                              const int* s_out_hi, long long out_base, int out_lo, float* tmax) {
#define TNQ_PFL(n) \
  stage_pf<NV, K, n, true, true>(S, t, prev, nullptr, out, s_ptr, F, tab, s_out_hi, out_base, out_lo, tmax)
  switch (S.nbits - GTB) {
    case 5: TNQ_PFL(32); break;
    case 4: TNQ_PFL(16); break;
    case 3: TNQ_PFL(8); break;
    case 2: TNQ_PFL(4); break;
    case 1: TNQ_PFL(2); break;
    default: TNQ_PFL(1); break;
  }
#undef TNQ_PFL
}

template <int NV>
__device__ __forceinline__ void run_stage(bool with_k, const GSt& S, int t, const float2* prev, float2* cur,
                                          float2* out, bool last, const float2* const* s_ptr, float F,
                                          const int (*tab)[TABW], const int* s_out_hi, long long out_base, int out_lo,
                                          float* tmax) {
  if (NV == 0 || with_k)
    group_stage<NV, true>(S, t, prev, cur, out, last, s_ptr, F, tab, s_out_hi, out_base, out_lo, tmax);
  else
    group_stage<(NV > 0 ? NV : 1), false>(S, t, prev, cur, out, last, s_ptr, F, tab, s_out_hi, out_base, out_lo,
                                          tmax);
}

// Product of the power-of-two scales of a stage's memory inputs for an item.
__device__ __forceinline__ float stage_scale(const GParams& P, const GSt& S, long long item) {
  float f = 1.f;
  for (int j = 0; j < S.n_in; ++j) {
    if (S.src[j] < 0) continue;
    const GIn& g = P.gin[S.src[j]];
    if (g.meta < 0) continue;
    int m;
    f *= scale_of_max(P.meta_m[(long long)g.meta * P.B + (g.dep ? item : 0ll)], &m);
  }
  return f;
}

// The (u = 0, u = 1) product of a stage's constant inputs n_var.., starting
// from (k0, k1) (the stage's power-of-two scale), in input order.
__device__ __forceinline__ void tail_const_pair(const GSt& S, const float2* const* s_ptr, float2* k0, float2* k1) {
  for (int j = S.n_var; j < S.n_in; ++j) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(s_ptr[S.src[j]]));
    *k0 = cmul(*k0, make_float2(v.x, v.y));
    *k1 = cmul(*k1, make_float2(v.z, v.w));
  }
}

// Stages 1..M of a group in registers. Every one of them reads the previous
// stage densely (operand 0, entry c at 2c: the pair over u_s) and has at most
// one other varying operand; so the last stage's entry cm depends on the
// previous stages only through the 2^M stage-0 entries cm 2^M .. cm 2^M +
// 2^M - 1, a binary tree: stage s entry cm 2^(M-s) + k is the sum over u of
// stage s-1 entries 2k + u (relative to the subtree) times the stage's other
// operands (each stage one elimination step of Eq. 2). A thread evaluates
// whole subtrees: one read of its stage-0 pairs, no barrier and no
// shared-memory stage between. K pairs as in stage_pf.
template <int M>
__device__ __forceinline__ void group_tail(const GParams& P, int t, const float2* buf, const float2* const* s_ptr,
                                           const float* s_F, const int (*s_tab)[TABW], const int* s_out_hi,
                                           long long out_base, int out_lo, float* tmax, const float4* s_K) {
  float2 K0[M], K1[M];
  const float2* op[M];
  int row[M];
  bool two[M];
#pragma unroll
  for (int s = 0; s < M; ++s) {
    const GSt& S = P.st[s + 1];
    if (S.kinv) {  // the same for every tile of the item: computed once per item
      const float4 k = s_K[s + 1];
      K0[s] = make_float2(k.x, k.y);
      K1[s] = make_float2(k.z, k.w);
    } else {
      K0[s] = K1[s] = make_float2(s_F[s + 1], 0.f);
      tail_const_pair(S, s_ptr, &K0[s], &K1[s]);
    }
    two[s] = S.n_var > 1;
    op[s] = two[s] ? s_ptr[S.src[1]] : nullptr;
    row[s] = S.q0 + 1;
  }
  const int nb_last = P.st[M].nbits;
  const int n_fin = nb_last > GTB ? 1 << (nb_last - GTB) : 1;
  const float4* b4 = reinterpret_cast<const float4*>(buf);
  float2* dst = P.out + out_base + out_lo;
  for (int i = 0; i < n_fin; ++i) {
    const int cm = t + GTPB * i;
    if (nb_last < GTB && cm >= (1 << nb_last)) break;
    float2 x[1 << M];
#pragma unroll
    for (int q = 0; q < (1 << (M - 1)); ++q) {
      const int p = (cm << (M - 1)) + q;
      const float4 v = b4[p ^ ((p >> 3) & 7)];
      x[2 * q] = make_float2(v.x, v.y);
      x[2 * q + 1] = make_float2(v.z, v.w);
    }
#pragma unroll
    for (int s = 0; s < M; ++s) {
      const int NK = 1 << (M - 1 - s);  // this stage's entries in the subtree (a constant once unrolled)
      auto combine = [&](int k, float2 a0, float2 a1) {
        float rx = K0[s].x * a0.x;  // K0 a0 + K1 a1
        rx = fmaf(-K0[s].y, a0.y, rx);
        rx = fmaf(K1[s].x, a1.x, rx);
        rx = fmaf(-K1[s].y, a1.y, rx);
        float ry = K0[s].x * a0.y;
        ry = fmaf(K0[s].y, a0.x, ry);
        ry = fmaf(K1[s].x, a1.y, ry);
        ry = fmaf(K1[s].y, a1.x, ry);
        x[k] = make_float2(rx, ry);
      };
      if (two[s]) {
        // the operand's offsets are additive over the bits of the local index:
        // entry c0 + k (k below 2^(M-1-s), the low bits of c0 zero) is at
        // offset(c0) + offset(k), offset(k) from the bits 0-3 table
        const int c0 = cm << (M - 1 - s);
        const int* tr = s_tab[row[s]];
        const float2* q =
            op[s] + tr[c0 & 15] + tr[GT_MID + ((c0 >> 4) & ((1 << (GTB - 4)) - 1))] + tr[GT_HI + (c0 >> GTB)];
        float4 w[1 << (M - 1)];
#pragma unroll
        for (int k = 0; k < NK; ++k) w[k] = __ldg(reinterpret_cast<const float4*>(q + tr[k]));
#pragma unroll
        for (int k = 0; k < NK; ++k)
          combine(k, cmul(x[2 * k], make_float2(w[k].x, w[k].y)), cmul(x[2 * k + 1], make_float2(w[k].z, w[k].w)));
      } else {
#pragma unroll
        for (int k = 0; k < NK; ++k) combine(k, x[2 * k], x[2 * k + 1]);
      }
    }
    dst[s_out_hi[i]] = x[0];
    *tmax = fmaxf(*tmax, fmaxf(fabsf(x[0].x), fabsf(x[0].y)));
  }
}

// Persistent fused-group kernel: every block builds the stage tables once,
// then loops over tiles (item, H assignment) tile = blockIdx.x + k*gridDim.x.
// TK = 0: every stage through the stage loops (both shared-memory regions);
// TK = 1: chains with a register tail -- stage 0 in shared memory, then
// group_tail; TK = 2: two-stage chains whose stage 1 reads stage 0 densely
// and writes the output. The last two need region A only and fewer code
// paths, so five blocks fit per SM.
template <int TK>
__global__ void __launch_bounds__(GTPB, TK ? 5 : 4) k_group(const __grid_constant__ GParams P, long long n_tiles) {
  extern __shared__ float2 g_stage[];  // stage regions A (2^(GL_MAX-1) entries) and B (half of A)
  __shared__ int s_hstr[GIN_MAX + 1][GH_MAX];  // row GIN_MAX: the output (within-item offsets < 2^31)
  __shared__ const float2* s_ptr[GIN_MAX];
  __shared__ float s_F[GM_MAX];  // per stage: product of its memory inputs' power-of-two scales
  __shared__ int s_e[GIN_MAX];
  __shared__ int s_tab[PAIR_MAX][TABW];
  __shared__ int s_out_hi[1 << (GL_MAX - 1 - GTB)];
  __shared__ long long s_out_base;
  __shared__ float s_red[GTPB / 32];
  __shared__ float4 s_K[GM_MAX];  // register-tail stages with per-item constant pairs (kinv)
  const int t = threadIdx.x;
  // tables shared by every tile
  for (int e = t; e < (GIN_MAX + 1) * GH_MAX; e += GTPB) {
    const int j = e / GH_MAX, i = e - j * GH_MAX;
    long long v = 0;
    if (i < P.n_h) v = (j < P.n_gin) ? P.gin[j].hstride[i] : (j == GIN_MAX ? P.out_hstride[i] : 0ll);
    s_hstr[j][i] = (int)v;
  }
  for (int s = 0; s < P.n_st; ++s) {
    const GSt& S = P.st[s];
    const int nb = S.nbits;
    for (int e = t; e < S.n_var * TABW; e += GTPB) {
      const int j = e / TABW, r = e - j * TABW;
      // r -> (first bit, value): bits 0-3, bits 4..GTB-1, bits GTB..
      const int b0 = r < GT_MID ? 0 : (r < GT_HI ? 4 : GTB);
      const int v = r - (r < GT_MID ? 0 : (r < GT_HI ? GT_MID : GT_HI));
      int a = 0;
      for (int i = 0; (v >> i) != 0; ++i)
        if (b0 + i < nb && ((v >> i) & 1)) a += S.cstride[j][b0 + i];
      s_tab[S.q0 + j][r] = a;
    }
  }
  const GSt& SL = P.st[P.n_st - 1];
  const int nb_last = SL.nbits;
  const int n_hi_last = nb_last > GTB ? (1 << (nb_last - GTB)) : 1;
  for (int it = t; it < n_hi_last; it += GTPB) {
    int a = 0;
    for (int i = GTB; i < nb_last; ++i)
      if ((it >> (i - GTB)) & 1) a += P.out_cstride[i];
    s_out_hi[it] = a;
  }
  int out_lo = 0;
  for (int i = 0; i < GTB && i < nb_last; ++i)
    if ((t >> i) & 1) out_lo += P.out_cstride[i];
  const int buf_elems = 1 << (GL_MAX - 1);
  long long cur_item = -1;
  long long meta_item = -1;  // item whose exponents and scales s_e / s_F hold
  float tmax = 0.f;
  for (long long tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const long long item = tile >> P.n_h;
    const long long h = tile & ((1ll << P.n_h) - 1ll);
    if (item != cur_item) {
      if (cur_item >= 0) {  // flush the previous item's max
        float m = tmax;
        for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
        __syncthreads();
        if ((t & 31) == 0) s_red[t >> 5] = m;
        __syncthreads();
        if (t == 0) {
          float b = 0.f;
          for (int w = 0; w < GTPB / 32; ++w) b = fmaxf(b, s_red[w]);
          if (b > 0.f) atomic_max_pos(&P.meta_m[(long long)P.out_meta * P.B + (P.out_dep ? cur_item : 0ll)], b);
        }
      }
      tmax = 0.f;
      cur_item = item;
    }
    __syncthreads();  // previous tile done with s_ptr / stage buffers
    // tile pointers: warp w takes inputs w, w + 4, ... (and the output, as
    // input n_gin); lane i adds the stride of tile bit i when it is set
    for (int j = t >> 5; j <= P.n_gin; j += GTPB / 32) {
      const int lane = t & 31;
      const int r = j < P.n_gin ? j : GIN_MAX;
      const int v = __reduce_add_sync(0xffffffffu, (lane < P.n_h && ((h >> lane) & 1ll)) ? s_hstr[r][lane] : 0);
      if (lane == 0) {
        if (j < P.n_gin) {
          const GIn& g = P.gin[j];
          s_ptr[j] = g.ptr + (g.dep ? item * g.istride : 0ll) + v;
        } else {
          s_out_base = (P.out_dep ? item * P.out_istride : 0ll) + v;
        }
      }
    }
    // exponents and power-of-two scales depend on the item only
    if (item != meta_item) {
      if (t < P.n_gin) {
        const GIn& g = P.gin[t];
        if (g.meta < 0) {
          s_e[t] = 0;
        } else {
          const long long row = (long long)g.meta * P.B + (g.dep ? item : 0ll);
          int m;
          scale_of_max(P.meta_m[row], &m);
          s_e[t] = P.meta_e[row] + m;
        }
      } else if (t < P.n_gin + P.n_st) {
        s_F[t - P.n_gin] = stage_scale(P, P.st[t - P.n_gin], item);
      }
      // the register-tail stages' constant pairs when their inputs hold no
      // tile bit: the same for every tile of the item
      if (TK == 1 && t >= 1 && t <= P.tail && P.st[t].kinv) {
        const GSt& S = P.st[t];
        const float f = stage_scale(P, S, item);
        float2 k0 = make_float2(f, 0.f), k1 = k0;
        for (int j = S.n_var; j < S.n_in; ++j) {
          const GIn& g = P.gin[S.src[j]];
          const float4 v = __ldg(reinterpret_cast<const float4*>(g.ptr + (g.dep ? item * g.istride : 0ll)));
          k0 = cmul(k0, make_float2(v.x, v.y));
          k1 = cmul(k1, make_float2(v.z, v.w));
        }
        s_K[t] = make_float4(k0.x, k0.y, k1.x, k1.y);
      }
      meta_item = item;
    }
    __syncthreads();
    // stage s writes region A (even s) or B (odd s); every stage output has at
    // least one bit fewer than the stage before, so B needs half of A
    float2* prev = g_stage + buf_elems;
    float2* cur = g_stage;
    if constexpr (TK) {
      const GSt& S = P.st[0];
      const int nv = S.n_var - S.n_tc;  // operands loaded per entry
      const bool with_k = S.n_in > nv;
      const float F = s_F[0];
      switch (nv * 2 + (with_k ? 1 : 0)) {
        case 2: stage0_pf<1, false>(S, t, cur, s_ptr, F, s_tab + S.q0); break;
        case 3: stage0_pf<1, true>(S, t, cur, s_ptr, F, s_tab + S.q0); break;
        case 4: stage0_pf<2, false>(S, t, cur, s_ptr, F, s_tab + S.q0); break;
        case 5: stage0_pf<2, true>(S, t, cur, s_ptr, F, s_tab + S.q0); break;
        case 6: stage0_pf<3, false>(S, t, cur, s_ptr, F, s_tab + S.q0); break;
        default: stage0_pf<3, true>(S, t, cur, s_ptr, F, s_tab + S.q0); break;
      }
      __syncthreads();
      if constexpr (TK == 1) {
        switch (P.tail) {  // stage 0's buffer is region A
          case 2: group_tail<2>(P, t, cur, s_ptr, s_F, s_tab, s_out_hi, s_out_base, out_lo, &tmax, s_K); break;
          case 3: group_tail<3>(P, t, cur, s_ptr, s_F, s_tab, s_out_hi, s_out_base, out_lo, &tmax, s_K); break;
          default: group_tail<4>(P, t, cur, s_ptr, s_F, s_tab, s_out_hi, s_out_base, out_lo, &tmax, s_K); break;
        }
      } else {
        const GSt& S1 = P.st[1];
        const float F1 = s_F[1];
        const int (*tab1)[TABW] = s_tab + S1.q0;
#define TNQ_L(nv, k) stage_last_pd<nv, k>(S1, t, cur, P.out, s_ptr, F1, tab1, s_out_hi, s_out_base, out_lo, &tmax)
        const int nv1 = S1.n_var - S1.n_tc;
        switch (nv1 * 2 + (S1.n_in > nv1 ? 1 : 0)) {
          case 2: TNQ_L(1, false); break;
          case 3: TNQ_L(1, true); break;
          case 4: TNQ_L(2, false); break;
          case 5: TNQ_L(2, true); break;
          case 6: TNQ_L(3, false); break;
          default: TNQ_L(3, true); break;
        }
#undef TNQ_L
      }
    }
    const int n_run = TK ? 0 : P.n_st;  // stages run in shared memory
    for (int s = 0; s < n_run; ++s) {
      const GSt& S = P.st[s];
      const bool last = (s == P.n_st - 1);
      const bool with_k = S.n_in > S.n_var;
      bool done = false;
      const float F = s_F[s];
#define TNQ_PFK2(n, pdv) done = with_k ? stage_pf_nhi<n, true, pdv>(S, t, prev, cur, P.out, last, s_ptr, F, s_tab + S.q0, s_out_hi, s_out_base, out_lo, &tmax) \
                                      : stage_pf_nhi<n, false, pdv>(S, t, prev, cur, P.out, last, s_ptr, F, s_tab + S.q0, s_out_hi, s_out_base, out_lo, &tmax)
// (a previous-stage operand that is not dense takes the generic path)
#define TNQ_PFK(n) { if (S.pd) { TNQ_PFK2(n, true); } else if (S.src[0] >= 0) { TNQ_PFK2(n, false); } }
      switch (S.n_var) {
        case 1: TNQ_PFK(1) break;
        case 2: TNQ_PFK(2) break;
        case 3: TNQ_PFK(3) break;
        default: break;
      }
#undef TNQ_PFK
#undef TNQ_PFK2
      if (!done) switch (S.n_var) {
#define TNQ_STAGE(n) run_stage<n>(with_k, S, t, prev, cur, P.out, last, s_ptr, F, s_tab + S.q0, s_out_hi, s_out_base, out_lo, &tmax)
        case 0: TNQ_STAGE(0); break;
        case 1: TNQ_STAGE(1); break;
        case 2: TNQ_STAGE(2); break;
        case 3: TNQ_STAGE(3); break;
        case 4: TNQ_STAGE(4); break;
        case 5: TNQ_STAGE(5); break;
        case 6: TNQ_STAGE(6); break;
        case 7: TNQ_STAGE(7); break;
        default: TNQ_STAGE(8); break;
#undef TNQ_STAGE
      }
      if (!last) __syncthreads();
      float2* tmp = prev;
      prev = cur;
      cur = tmp;
    }
    if (h == 0 && t == 0) {
      int e = 0;
      for (int j = 0; j < P.n_gin; ++j) e += s_e[j];
      P.meta_e[(long long)P.out_meta * P.B + (P.out_dep ? item : 0ll)] = e;
    }
  }
  // flush the last item's max
  float m = tmax;
  for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
  __syncthreads();
  if ((t & 31) == 0) s_red[t >> 5] = m;
  __syncthreads();
  if (t == 0 && cur_item >= 0) {
    float b = 0.f;
    for (int w = 0; w < GTPB / 32; ++w) b = fmaxf(b, s_red[w]);
    if (b > 0.f) atomic_max_pos(&P.meta_m[(long long)P.out_meta * P.B + (P.out_dep ? cur_item : 0ll)], b);
  }
}

// K4: amplitude of every item = scalar leaves * final scalars * 2^(exponents),
// then the FP64 sum of each bitstring's items of this batch in item order.
__global__ void k_finalize(const FinalDev* __restrict__ fin, int n_fin, const double2* __restrict__ item_scalar,
                           const float2* __restrict__ arena, const int* __restrict__ meta_e, int B,
                           const BatchHdr* __restrict__ hdr_p, int scale_exp, int scale_half,
                           double2* __restrict__ res) {
  const BatchHdr h = *hdr_p;
  int item = blockIdx.x * blockDim.x + threadIdx.x;
  if (item >= B) return;
  unsigned long long slice;
  int brow;
  bool valid;
  item_decode(h, item, &slice, &brow, &valid);
  double re = item_scalar[item].x, im = item_scalar[item].y;
  int e = scale_exp;
  for (int i = 0; i < n_fin; ++i) {
    const FinalDev F = fin[i];
    const float2 v = arena[F.off + (F.dep ? item : 0)];
    const double nr = re * v.x - im * v.y, ni = re * v.y + im * v.x;
    re = nr;
    im = ni;
    e += meta_e[(long long)F.meta * B + (F.dep ? item : 0)];
  }
  if (scale_half) {
    re *= 0.70710678118654752440;
    im *= 0.70710678118654752440;
  }
  res[item] = valid ? make_double2(ldexp(re, e), ldexp(im, e)) : make_double2(0.0, 0.0);
}

// Per-bitstring FP64 partial sums of one batch, items in increasing order.
__global__ void k_slice_sum(const double2* __restrict__ res, int B, const BatchHdr* __restrict__ hdr_p,
                            double2* __restrict__ part, int n_rows) {
  const BatchHdr h = *hdr_p;
  int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= n_rows) return;
  double re = 0.0, im = 0.0;
  for (int item = 0; item < B; ++item) {
    unsigned long long slice;
    int brow;
    bool valid;
    item_decode(h, item, &slice, &brow, &valid);
    if (valid && brow == row) {
      re += res[item].x;
      im += res[item].y;
    }
  }
  part[row] = make_double2(re, im);
}

// Adds one batch's per-bitstring partial sums (rows 0..n_rows-1) to the FP64
// accumulators of those bitstrings. Batches are added in stream order, so each
// bitstring's amplitude is summed in increasing item order (Eq. 5).
__global__ void k_accumulate(const double2* __restrict__ part, int n_rows, double2* __restrict__ acc) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < n_rows) {
    acc[r].x += part[r].x;
    acc[r].y += part[r].y;
  }
}

// ---------------------------------------------------------------------------
// host side
#define CU(call)                                                                  \
  do {                                                                            \
    cudaError_t err_ = (call);                                                    \
    if (err_ != cudaSuccess) {                                                    \
      set_error(std::string(#call) + ": " + cudaGetErrorString(err_));           \
      return TNQ_ECUDA;                                                           \
    }                                                                             \
  } while (0)

namespace {

// Where every tensor of one configuration lives.
struct Layout {
  int mode = 0, B = 1, item_bits = 0;
  std::vector<long long> off;   // element offset per tensor
  std::vector<char> dep;        // item-dependent per tensor
  std::vector<int> hoist;       // per bucket: level (>= 1) of an early bucket (see hoist_levels), else 0
  long long arena_elems = 0;
  long long gemm_off = 0;        // element offset of the GEMM operand scratch inside the arena
  size_t hdr_off = 0, bits_off = 0, scalar_off = 0, res_off = 0, part_off = 0, meta_e_off = 0, meta_m_off = 0,
         arena_off = 0, status_off = 0, total = 0;
  int n_words = 1, n_rows = 1;
};

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

bool tensor_dep(const PTensor& t, int mode) { return t.dep_slice || (mode == 1 && t.dep_bits); }

// Padded sizes of a GEMM group (complex rows, columns and K; operand bytes).
struct GemmShape {
  int kind = 0, m_pad = 0, n_pad = 0, k_pad = 0;
  long long batch = 0;
  size_t a_bytes = 0, b_bytes = 0;  // one of hi / lo
};

GemmShape gemm_shape(const tnq_plan& P, const FusedGroup& g, int items) {
  GemmShape s;
  s.kind = P.opts.precision == TNQ_PREC_SPLIT_TF32 ? GEMM_TF32 : GEMM_BF16;
  const int esize = s.kind == GEMM_BF16 ? 2 : 4;
  auto up = [](long long x, long long a) { return (x + a - 1) / a * a; };
  s.m_pad = (int)up(1ll << g.xvars.size(), GT_ROWS);
  s.n_pad = (int)up(1ll << g.yvars.size(), GT_ROWS / 2);
  s.k_pad = (int)up(1ll << g.kvars.size(), GT_KBYTES / (2 * esize));
  s.batch = (long long)items << g.svars.size();
  s.a_bytes = (size_t)s.batch * s.m_pad * 2 * s.k_pad * esize;
  s.b_bytes = (size_t)s.batch * 2 * s.n_pad * 2 * s.k_pad * esize;
  return s;
}

// Early buckets: a single (unfused) bucket whose inputs are gate tensors or
// results of early buckets depends on nothing the batch computes otherwise.
// These run first, before every other step, one launch per level (level = 1 +
// the highest level among the producers of its inputs), when the result with
// its item bits has at most HOIST_MAX_BITS index bits. Their results are given
// a lifetime from the start of the batch, so no other tensor shares their
// memory meanwhile.
std::vector<int> hoist_levels(const Program& prog, const std::vector<char>& dep, int item_bits) {
  const int nb = (int)prog.buckets.size();
  std::vector<int> lv(nb, 0);
  for (int b = 0; b < nb; ++b) {
    if (!prog.group_of.empty() && prog.group_of[b] >= 0) continue;
    const PBucket& B = prog.buckets[b];
    if (prog.tensors[B.output].rank() + (dep[B.output] ? item_bits : 0) > HOIST_MAX_BITS || B.k > KMAX || B.k < 1)
      continue;
    int l = 0;
    bool ok = true;
    for (int t : B.inputs) {
      const int p = prog.tensors[t].producer;
      if (p < 0) continue;  // gate tensor, written by the leaf kernel
      if (lv[p] == 0) { ok = false; break; }
      l = std::max(l, lv[p]);
    }
    if (ok) lv[b] = l + 1;
  }
  return lv;
}

// Lifetimes in bucket steps (a fused group's tensors live at its last bucket;
// the results inside a group are never stored), early-bucket results from
// the start of the batch.
Liveness layout_liveness(const Program& prog, const std::vector<int>& hoist) {
  Liveness LV = tensor_liveness(prog);
  for (size_t b = 0; b < prog.buckets.size(); ++b)
    if (hoist[b]) LV.lo[prog.buckets[b].output] = -1;
  return LV;
}

Layout make_layout(const tnq_plan& P, int mode, int B) {
  const Program& prog = P.prog;
  Layout L;
  L.mode = mode;
  L.B = B;
  while ((1 << L.item_bits) < B) ++L.item_bits;
  const int T = (int)prog.tensors.size();
  L.off.assign(T, 0);
  L.dep.assign(T, 0);
  for (int t = 0; t < T; ++t) L.dep[t] = tensor_dep(prog.tensors[t], mode);
  L.hoist = hoist_levels(prog, L.dep, L.item_bits);
  const Liveness LV = layout_liveness(prog, L.hoist);
  const std::vector<int>& lo = LV.lo;
  const std::vector<int>& hi = LV.hi;
  std::vector<long long> size(T);
  for (int t = 0; t < T; ++t) {
    const PTensor& x = prog.tensors[t];
    size[t] = LV.internal[t] ? 0 : (long long)align_up(((size_t)1 << x.rank()) * (L.dep[t] ? (size_t)B : 1), 32);
  }
  std::vector<int> idx;
  for (int t = 0; t < T; ++t)
    if (!LV.internal[t]) idx.push_back(t);
  std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return size[a] > size[b]; });
  std::vector<int> placed;
  for (int t : idx) {
    // lowest offset not overlapping a placed tensor with an intersecting lifetime
    std::vector<std::pair<long long, long long>> busy;
    for (int o : placed)
      if (lo[o] <= hi[t] && lo[t] <= hi[o]) busy.push_back({L.off[o], L.off[o] + size[o]});
    std::sort(busy.begin(), busy.end());
    long long cand = 0;
    for (auto& iv : busy) {
      if (cand + size[t] <= iv.first) break;
      cand = std::max(cand, iv.second);
    }
    L.off[t] = cand;
    L.arena_elems = std::max(L.arena_elems, cand + size[t]);
    placed.push_back(t);
  }
  // GEMM operand scratch (shared by every GEMM step): hi/lo of both operands
  long long gemm_elems = 0;
  for (const FusedGroup& g : prog.groups) {
    if (!g.gemm) continue;
    const GemmShape sh = gemm_shape(P, g, L.dep[g.output] ? B : 1);
    gemm_elems = std::max<long long>(gemm_elems, (long long)(2 * (sh.a_bytes + sh.b_bytes) / 8));
  }
  L.gemm_off = (long long)align_up((size_t)L.arena_elems, 128);
  if (gemm_elems) L.arena_elems = L.gemm_off + gemm_elems;
  L.n_words = (P.net.n_qubits + 31) / 32;
  L.n_rows = B + 1;
  size_t o = 0;
  L.hdr_off = o; o = align_up(o + sizeof(BatchHdr), 128);
  L.status_off = o; o = align_up(o + 4, 256);
  L.bits_off = o; o = align_up(o + (size_t)L.n_rows * L.n_words * 4, 256);
  L.scalar_off = o; o = align_up(o + (size_t)B * 16, 256);
  L.res_off = o; o = align_up(o + (size_t)B * 16, 256);
  L.part_off = o; o = align_up(o + (size_t)L.n_rows * 16, 256);
  L.meta_e_off = o; o = align_up(o + (size_t)T * B * 4, 256);
  L.meta_m_off = o; o = align_up(o + (size_t)T * B * 4, 256);
  L.arena_off = o; o = align_up(o + (size_t)L.arena_elems * 8, 256);
  L.total = o;
  return L;
}

}  // namespace

// Per-device state of a plan: uploaded tables and captured graphs.
struct ExecConfig {
  Layout L;
  LeafDev* d_leaves = nullptr;
  int n_leaves = 0;
  LeafDev* d_scalars = nullptr;
  int n_scalars = 0;
  int* d_inout = nullptr;
  int n_inout = 0;
  FinalDev* d_finals = nullptr;
  int n_finals = 0;
  std::vector<KParams> kp;           // per single-bucket step (pointers filled per workspace)
  std::vector<std::pair<int, int>> kshape;  // (n_in, LT) per single-bucket step
  std::vector<GParams> gp;           // per fused-group step
  std::vector<int> gsmem;            // dynamic shared memory bytes per fused-group step
  std::vector<int> ggrid;            // persistent blocks per fused-group step (SMs x resident blocks at its gsmem)
  int group_grid = 152 * 4;          // persistent blocks of k_group (SMs x resident blocks)
  std::vector<GemmBucketArgs> gb;    // per GEMM step (pointers are arena offsets)
  std::vector<GemmEpilogue> ge;
  std::vector<std::pair<int, int>> steps;  // (0, kp index), (1, gp index) or (2, gb index), program order
  std::vector<int> step_group;       // group index of each step (-1 for a single bucket)
  std::vector<double> step_bytes;    // algorithmic bytes of each step (all items)
  std::vector<double> step_flops;    // algorithmic flops of each step (all items; cost model of Section IV)
  std::vector<std::vector<int>> step_deps;  // earlier steps each step must wait for (concurrent launches)
  std::vector<int> step_stream;      // side stream of each step in a captured batch
  std::vector<int> step_hoist;       // per step: level of an early bucket (runs in its level's launch), else 0
  std::vector<HoistDev> hoist_dev;   // early buckets in level order (host copy)
  std::vector<int> hoist_first;      // per level: first entry in hoist_dev (one past the last level at the end)
  std::vector<int> hoist_blocks;     // per level: blocks of its launch
  HoistDev* d_hoist = nullptr;
  std::vector<float2> vals;          // leaf value table: entries of general-network tensors with > 2 variables
  float2* d_vals = nullptr;
  void* ws = nullptr;                // workspace the graph was captured for
  cudaGraphExec_t exec = nullptr;
};

// Host-side configuration of the allocation-free entry point for one batch
// size: its device pointers point into the library's static scratch, so it
// owns no device memory; the host tables are uploaded again on every call.
struct NoallocConfig {
  ExecConfig C;
  std::vector<LeafDev> leaves, scalars;
  std::vector<FinalDev> finals;
  size_t tables = 0;  // bytes of plan tables at the front of the scratch
};

struct DeviceState {
  int device = -1;
  std::map<std::pair<int, int>, ExecConfig*> configs;  // (mode, B)
  std::map<int, NoallocConfig*> noalloc;               // B
  std::map<uint64_t, int> noalloc_batch;               // batch cap -> largest B that fits the scratch
  ~DeviceState() {
    for (auto& kv : noalloc) delete kv.second;
    for (auto& kv : configs) {
      ExecConfig* c = kv.second;
      if (c->exec) cudaGraphExecDestroy(c->exec);
      cudaFree(c->d_leaves);
      cudaFree(c->d_scalars);
      cudaFree(c->d_inout);
      cudaFree(c->d_finals);
      cudaFree(c->d_hoist);
      cudaFree(c->d_vals);
      delete c;
    }
  }
};

void destroy_device_state(DeviceState* s) { delete s; }

// Leaf record of network tensor `gate`; general tensors with more than two
// variables append their entries to `vals` (the configuration's leaf value table).
static LeafDev make_leafdev(const tnq_plan& P, const PTensor* pt, int gate, const Layout* L, int tid,
                            std::vector<float2>* vals) {
  const GateTensor& gt = P.net.tensors[gate];
  LeafDev d;
  std::memset(&d, 0, sizeof(d));
  if (gt.nv <= 2) {
    for (int i = 0; i < 4; ++i) d.val[i] = make_float2(gt.val[i].real(), gt.val[i].imag());
    d.tab = -1;
  } else {
    d.tab = (long long)vals->size();
    for (int i = 0; i < (1 << gt.nv); ++i) vals->push_back(make_float2(gt.val[i].real(), gt.val[i].imag()));
  }
  d.nv = gt.nv;
  d.n_free = pt ? pt->rank() : 0;
  std::vector<int> mu_index(P.net.free_vars.size(), -1);
  for (size_t j = 0; j < P.mu.size(); ++j) mu_index[P.mu[j]] = (int)j;
  for (int x = 0; x < gt.nv; ++x) {
    const Var& v = P.net.vars[gt.var[x]];
    if (v.kind == VAR_IN || v.kind == VAR_INOUT) {
      d.vkind[x] = 1;
    } else if (v.kind == VAR_OUT) {
      d.vkind[x] = 2;
      d.varg[x] = v.q;
    } else if (mu_index[v.free_id] >= 0) {
      d.vkind[x] = 3;
      d.varg[x] = mu_index[v.free_id];
    } else {
      d.vkind[x] = 0;
      d.varg[x] = (int)(std::find(pt->vars.begin(), pt->vars.end(), v.free_id) - pt->vars.begin());
    }
  }
  if (L) {
    d.dep = L->dep[tid];
    d.off = L->off[tid];
  }
  return d;
}

// Kernel parameters of every step of one configuration (single buckets and
// fused groups, in program order), with pointers holding byte offsets from the
// arena base (rebased per call). Host only.
static KParams single_kparams(const tnq_plan& P, const Layout& L, const PBucket& b, bool* ok) {
  const Program& prog = P.prog;
  KParams k;
  std::memset(&k, 0, sizeof(k));
  const PTensor& o = prog.tensors[b.output];
  const bool odep = L.dep[b.output];
  k.out_bits = o.rank();
  k.G = k.out_bits + (odep ? L.item_bits : 0);
  *ok = k.G < GMAX && b.k <= KMAX;
  if (!*ok) return k;
  k.sum = b.sum ? 1 : 0;
  k.B = L.B;
  k.out_meta = b.output;
  k.out = reinterpret_cast<float2*>((size_t)L.off[b.output] * 8);
  for (int j = 0; j < b.k; ++j) {
    const int tid = b.inputs[j];
    const PTensor& x = prog.tensors[tid];
    k.in[j] = reinterpret_cast<const float2*>((size_t)L.off[tid] * 8);
    k.in_meta[j] = x.leaf_gate >= 0 ? -1 : tid;
    k.in_dep[j] = L.dep[tid];
    for (int i = 0; i < k.out_bits; ++i) {
      auto it = std::find(x.vars.begin(), x.vars.end(), o.vars[i]);
      k.stride[j][i] = it == x.vars.end() ? 0 : (1ll << (it - x.vars.begin()));
    }
    for (int i = k.out_bits; i < k.G; ++i) k.stride[j][i] = L.dep[tid] ? ((1ll << x.rank()) << (i - k.out_bits)) : 0;
  }
  // the input with the most distinct entries per block (then the largest)
  // first, among those that vary with output bits 0-7: k_bucket loads input 0
  // several iterations ahead. The choice depends on the bucket alone (not on
  // the batch size or on which variables make an input item-dependent), so
  // every configuration multiplies in the same order.
  {
    auto weight = [&](int j) {  // (-1: constant over output bits 0-7; else output bits 0-11 it varies with, rank)
      int w8 = 0, w = 0, rank = 0;
      for (int i = 0; i < k.out_bits; ++i) {
        const bool nz = k.stride[j][i] != 0;
        w8 += (i < 8) && nz;
        w += (i < 12) && nz;
        rank += nz;
      }
      return w8 ? std::make_pair(w, rank) : std::make_pair(-1, 0);
    };
    int best = 0;
    for (int j = 1; j < b.k; ++j)
      if (weight(j) > weight(best)) best = j;
    if (best != 0 && weight(best).first >= 0) {
      std::swap(k.in[best], k.in[0]);
      std::swap(k.in_meta[best], k.in_meta[0]);
      std::swap(k.in_dep[best], k.in_dep[0]);
      for (int i = 0; i < GMAX; ++i) std::swap(k.stride[best][i], k.stride[0][i]);
    }
  }
  // inputs that vary with the low 8 bits (a block's threads) first; the others
  // are the same for every thread of a block's iteration (k_bucket multiplies
  // them once per block into a constant pair)
  // (output bits only: whether an input varies with the item bits depends on
  // the configuration, and the arithmetic order must not)
  auto varies = [&](int j) {
    for (int i = 0; i < 8 && i < k.out_bits; ++i)
      if (k.stride[j][i]) return true;
    return false;
  };
  int nv = 0;
  for (int j = 0; j < b.k; ++j)
    if (varies(j)) {
      if (j != nv) {
        std::swap(k.in[j], k.in[nv]);
        std::swap(k.in_meta[j], k.in_meta[nv]);
        std::swap(k.in_dep[j], k.in_dep[nv]);
        for (int i = 0; i < GMAX; ++i) std::swap(k.stride[j][i], k.stride[nv][i]);
      }
      ++nv;
    }
  k.n_var = nv;
  return k;
}

static int index_in(const std::vector<int>& v, int x) {
  auto it = std::find(v.begin(), v.end(), x);
  return it == v.end() ? -1 : (int)(it - v.begin());
}

// Local output variables of every stage of a group: (bag_s \ u_s) restricted
// to the group's local variables, in position order.
static std::vector<std::vector<int>> group_stage_vars(const Program& prog, const FusedGroup& g) {
  std::vector<std::vector<int>> sv;
  for (int b : g.buckets) {
    const PBucket& B = prog.buckets[b];
    std::vector<int> v;
    for (int x : g.local_vars) {  // local_vars is sorted by position
      if (x == B.u) continue;
      bool in_bag = false;
      for (int t : B.inputs) in_bag |= index_in(prog.tensors[t].vars, x) >= 0;
      if (in_bag) v.push_back(x);
    }
    sv.push_back(v);
  }
  return sv;
}

static GParams group_gparams(const tnq_plan& P, const Layout& L, const FusedGroup& g, bool* ok, int* smem) {
  const Program& prog = P.prog;
  GParams G;
  std::memset(&G, 0, sizeof(G));
  *ok = false;
  const PTensor& o = prog.tensors[g.output];
  const int n_h = (int)g.tile_vars.size() + (L.dep[g.output] ? L.item_bits : 0);
  if ((int)g.tile_vars.size() >= GH_MAX || (int)g.ext_inputs.size() > GIN_MAX || (int)g.buckets.size() > GM_MAX)
    return G;
  G.n_h = (int)g.tile_vars.size();  // item index is the tile index above these bits
  (void)n_h;
  G.n_st = (int)g.buckets.size();
  G.n_gin = (int)g.ext_inputs.size();
  G.B = L.B;
  G.out_meta = g.output;
  G.out_dep = L.dep[g.output];
  G.out = reinterpret_cast<float2*>((size_t)L.off[g.output] * 8);
  G.out_istride = 1ll << o.rank();
  for (size_t i = 0; i < g.tile_vars.size(); ++i) {
    const int p = index_in(o.vars, g.tile_vars[i]);
    if (p < 0) return G;
    G.out_hstride[i] = 1ll << p;
  }
  for (int j = 0; j < G.n_gin; ++j) {
    const int tid = g.ext_inputs[j];
    const PTensor& x = prog.tensors[tid];
    GIn& gi = G.gin[j];
    gi.ptr = reinterpret_cast<const float2*>((size_t)L.off[tid] * 8);
    gi.dep = L.dep[tid];
    gi.istride = 1ll << x.rank();
    gi.meta = x.leaf_gate >= 0 ? -1 : tid;
    for (size_t i = 0; i < g.tile_vars.size(); ++i) {
      const int p = index_in(x.vars, g.tile_vars[i]);
      gi.hstride[i] = p < 0 ? 0 : (1ll << p);
    }
  }
  const auto sv = group_stage_vars(prog, g);
  int maxbits = 0;
  for (int s = 0; s < G.n_st; ++s) {
    const PBucket& B = prog.buckets[g.buckets[s]];
    GSt& S = G.st[s];
    S.n_in = B.k;
    S.nbits = (int)sv[s].size();
    if (S.nbits > GL_MAX - 1 || B.k > KMAX) return G;
    maxbits = std::max(maxbits, S.nbits);
    // varying inputs first (any local stride), then the per-block constants
    std::vector<int> ins(B.inputs.begin(), B.inputs.end());
    auto varies = [&](int tid) {
      if (s > 0 && tid == prog.buckets[g.buckets[s - 1]].output) return sv[s].size() > 0;
      for (int x : sv[s])
        if (index_in(prog.tensors[tid].vars, x) >= 0) return true;
      return false;
    };
    std::stable_partition(ins.begin(), ins.end(), varies);
    S.n_var = 0;
    for (int tid : ins) S.n_var += varies(tid) ? 1 : 0;
    // the previous stage's buffer first among the varying inputs
    const int prev_tid = s > 0 ? prog.buckets[g.buckets[s - 1]].output : -1;
    std::stable_partition(ins.begin(), ins.begin() + S.n_var, [&](int tid) { return tid == prev_tid; });
    S.q0 = G.n_pairs;
    G.n_pairs += S.n_var;
    if (G.n_pairs > PAIR_MAX) return G;
    for (int j = 0; j < B.k; ++j) {
      const int tid = ins[j];
      if (s > 0 && tid == prog.buckets[g.buckets[s - 1]].output) {
        S.src[j] = -1;
        const auto& pv = sv[s - 1];
        for (int b = 0; b < S.nbits; ++b) {
          const int p = index_in(pv, sv[s][b]);
          S.cstride[j][b] = p < 0 ? 0 : (1 << p);
        }
        const int pu = index_in(pv, B.u);
        if (pu < 0) return G;
        S.ustride[j] = 1 << pu;
      } else {
        S.src[j] = index_in(g.ext_inputs, tid);
        if (S.src[j] < 0) return G;
        const PTensor& x = prog.tensors[tid];
        for (int b = 0; b < S.nbits; ++b) {
          const int p = index_in(x.vars, sv[s][b]);
          S.cstride[j][b] = p < 0 ? 0 : (1 << p);
        }
        const int pu = index_in(x.vars, B.u);
        if (pu < 0) return G;
        S.ustride[j] = 1 << pu;
      }
    }
  }
  for (int s = 0; s < G.n_st; ++s) {  // constant inputs, all from memory, that hold no tile bit
    GSt& S = G.st[s];
    bool inv = true;
    for (int j = S.n_var; inv && j < S.n_in; ++j) {
      inv = S.src[j] >= 0;
      for (int i = 0; inv && i < G.n_h; ++i) inv = G.gin[S.src[j]].hstride[i] == 0;
    }
    S.kinv = inv ? 1 : 0;
  }
  for (int s = 0; s < G.n_st; ++s) {  // dense previous-stage operand (offset 2c, u at bit 0)
    GSt& S = G.st[s];
    bool d = S.n_var > 0 && S.src[0] < 0 && S.ustride[0] == 1;
    for (int b = 0; d && b < S.nbits; ++b) d = S.cstride[0][b] == (2 << b);
    S.pd = d ? 1 : 0;
  }
  // stages 1.. in registers (group_tail) when each reads the previous one
  // densely, has at most one other varying operand (from memory) and one bit
  // fewer than the stage before
  {
    bool ok = G.n_st - 1 >= TAIL_MIN && G.n_st - 1 <= TAIL_MAX && G.st[0].n_var >= 1 && G.st[0].n_var <= 3 &&
              G.st[0].nbits > 0;
    for (int j = 0; ok && j < G.st[0].n_in; ++j) ok = G.st[0].src[j] >= 0;
    for (int s = 1; ok && s < G.n_st; ++s) {
      const GSt& S = G.st[s];
      ok = S.pd && S.n_var >= 1 && S.n_var <= 2 && (S.n_var < 2 || S.src[1] >= 0) &&
           S.nbits == G.st[s - 1].nbits - 1;
      for (int j = S.n_var; ok && j < S.n_in; ++j) ok = S.src[j] >= 0;
    }
    G.tail = ok ? G.n_st - 1 : 0;
  }
  // two stages: stage 0 from memory (as above), stage 1 reading it densely
  // with at most two other varying operands, all from memory
  if (!G.tail && G.n_st == 2) {
    const GSt& S0 = G.st[0];
    const GSt& S1 = G.st[1];
    bool ok = S0.n_var >= 1 && S0.n_var <= 3 && S0.nbits > 0 && S1.pd && S1.n_var >= 1 && S1.n_var <= 3 &&
              S1.nbits <= GTB + 5;
    for (int j = 0; ok && j < S0.n_in; ++j) ok = S0.src[j] >= 0;
    for (int j = 1; ok && j < S1.n_in; ++j) ok = S1.src[j] >= 0;
    G.lean2 = ok ? 1 : 0;
  }
  // stages run by the prefetching loop of k_group<1> / <2> (stage 0, and
  // stage 1 of a two-stage chain): varying inputs that hold thread bits only
  // (local bits below GTB, the same for all entries of a thread) move behind
  // the others; the loop multiplies their per-thread pairs into its constant
  // pair once instead of loading them per entry
  auto move_thread_const = [&](GSt& S, int first) {
    auto tc = [&](int j) {
      if (S.src[j] < 0) return false;
      bool any = false;
      for (int b = 0; b < S.nbits; ++b) {
        if (!S.cstride[j][b]) continue;
        if (b >= GTB) return false;
        any = true;
      }
      return any;
    };
    std::vector<int> keep, moved;
    for (int j = 0; j < S.n_var; ++j) (j >= first && tc(j) ? moved : keep).push_back(j);
    if (moved.empty() || keep.empty()) return;
    std::vector<int> perm(keep);
    perm.insert(perm.end(), moved.begin(), moved.end());
    GSt T = S;
    for (int k = 0; k < S.n_var; ++k) {
      T.src[k] = S.src[perm[k]];
      T.ustride[k] = S.ustride[perm[k]];
      for (int b = 0; b < GL_MAX; ++b) T.cstride[k][b] = S.cstride[perm[k]][b];
    }
    T.n_tc = (int)moved.size();
    S = T;
  };
  if (G.tail || G.lean2) move_thread_const(G.st[0], 0);
  if (G.lean2) move_thread_const(G.st[1], 1);
  const auto& last = sv[G.n_st - 1];
  for (size_t b = 0; b < last.size(); ++b) {
    const int p = index_in(o.vars, last[b]);
    if (p < 0) return G;
    G.out_cstride[b] = 1 << p;
  }
  if (last.size() + g.tile_vars.size() != o.vars.size()) return G;
  // with the register tail only stage 0's buffer (region A) is used
  // (k_group<2>'s dense stage-1 reads cover pairs 0..GTPB-1 even when stage 0
  // has fewer entries: its threads past the end compute an entry they do not store)
  *smem = G.tail ? (int)sizeof(float2) << G.st[0].nbits
                 : (G.lean2 ? (int)sizeof(float2) * std::max(1 << G.st[0].nbits, 2 * GTPB) : GROUP_SMEM_BYTES);
  (void)maxbits;
  *ok = true;
  return G;
}

// GEMM-step parameters of a GEMM group, with pointers holding byte offsets
// from the arena base (rebased per call). Host only.
static bool gemm_params(const tnq_plan& P, const Layout& L, const FusedGroup& g, GemmBucketArgs& G,
                        GemmEpilogue& E) {
  const Program& prog = P.prog;
  std::memset(&G, 0, sizeof(G));
  std::memset(&E, 0, sizeof(E));
  const int items = L.dep[g.output] ? L.B : 1;
  const GemmShape sh = gemm_shape(P, g, items);
  if (g.svars.size() > (size_t)GB_BITS || g.xvars.size() > (size_t)GB_BITS || g.yvars.size() > (size_t)GB_BITS ||
      g.kvars.size() > (size_t)GB_BITS || 1 + g.a_side.size() > (size_t)GB_SIDE || 1 + g.b_side.size() > (size_t)GB_SIDE) {
    set_error("GEMM group: too many variables or folded tensors");
    return false;
  }
  auto operand = [&](int tid, const std::vector<int>& rows, GemmOperand& o) {
    const PTensor& x = prog.tensors[tid];
    o.ptr = reinterpret_cast<const float2*>((size_t)L.off[tid] * 8);
    o.dep = L.dep[tid];
    o.istride = 1ll << x.rank();
    o.meta = x.leaf_gate >= 0 ? -1 : tid;
    auto fill = [&](const std::vector<int>& vars, long long* st) {
      for (size_t i = 0; i < vars.size(); ++i) {
        const int p = index_in(x.vars, vars[i]);
        st[i] = p < 0 ? 0 : (1ll << p);
      }
    };
    fill(g.svars, o.sstride);
    fill(rows, o.rstride);
    fill(g.kvars, o.kstride);
    // every variable of the operand is a batch, row or summed variable
    for (int v : x.vars)
      if (index_in(g.svars, v) < 0 && index_in(rows, v) < 0 && index_in(g.kvars, v) < 0) {
        set_error("GEMM group: operand variable outside its batch/row/summed sets");
        return false;
      }
    return true;
  };
  G.na = 1 + (int)g.a_side.size();
  G.nb = 1 + (int)g.b_side.size();
  if (!operand(g.ga, g.xvars, G.a[0]) || !operand(g.gb, g.yvars, G.b[0])) return false;
  for (size_t j = 0; j < g.a_side.size(); ++j)
    if (!operand(g.a_side[j], g.xvars, G.a[1 + j])) return false;
  for (size_t j = 0; j < g.b_side.size(); ++j)
    if (!operand(g.b_side[j], g.yvars, G.b[1 + j])) return false;
  G.ns = (int)g.svars.size();
  G.nx = (int)g.xvars.size();
  G.ny = (int)g.yvars.size();
  G.nk = (int)g.kvars.size();
  G.items = items;
  G.m_pad = sh.m_pad;
  G.n_pad = sh.n_pad;
  G.k_pad = sh.k_pad;
  G.kind = sh.kind;
  const size_t base = (size_t)L.gemm_off * 8;
  G.a_hi = reinterpret_cast<void*>(base);
  G.a_lo = reinterpret_cast<void*>(base + sh.a_bytes);
  G.b_hi = reinterpret_cast<void*>(base + 2 * sh.a_bytes);
  G.b_lo = reinterpret_cast<void*>(base + 2 * sh.a_bytes + sh.b_bytes);
  G.out_meta = g.output;
  G.out_dep = L.dep[g.output];
  G.B = L.B;
  const PTensor& o = prog.tensors[g.output];
  E.out = reinterpret_cast<float2*>((size_t)L.off[g.output] * 8);
  E.istride = 1ll << o.rank();
  auto ofill = [&](const std::vector<int>& vars, long long* st) {
    for (size_t i = 0; i < vars.size(); ++i) {
      const int p = index_in(o.vars, vars[i]);
      if (p < 0) return false;
      st[i] = 1ll << p;
    }
    return true;
  };
  if (!ofill(g.svars, E.s) || !ofill(g.xvars, E.x) || !ofill(g.yvars, E.y)) {
    set_error("GEMM group: output misses a batch/row/column variable");
    return false;
  }
  E.ns = G.ns;
  E.nx = G.nx;
  E.ny = G.ny;
  E.meta = g.output;
  E.dep = G.out_dep;
  E.B = L.B;
  return true;
}

// Dependencies between the steps of one batch, for concurrent launches: step
// i waits for the producer of every tensor it reads, for every earlier step
// that reads or writes arena memory its output overwrites (the layout reuses
// the space of dead tensors), and GEMM steps (one shared operand scratch) run
// in program order. Each step goes to the side stream of its latest
// dependency (chains stay on one stream), or round-robin when it has none.
constexpr int N_SIDE_STREAMS = 4;
static void step_dependencies(const tnq_plan& P, const Layout& L, ExecConfig& C) {
  const Program& prog = P.prog;
  const int n = (int)C.steps.size();
  std::vector<std::vector<int>> reads(n);
  std::vector<int> write(n, -1);
  std::vector<int> producer(prog.tensors.size(), -1);
  {
    size_t si = 0;
    for (size_t bi = 0; bi < prog.buckets.size() && si < (size_t)n; ++bi) {
      const int gi = prog.group_of.empty() ? -1 : prog.group_of[bi];
      if (gi < 0) {
        reads[si] = prog.buckets[bi].inputs;
        write[si] = prog.buckets[bi].output;
      } else if ((int)bi == prog.groups[gi].buckets.back()) {
        reads[si] = prog.groups[gi].ext_inputs;
        write[si] = prog.groups[gi].output;
      } else {
        continue;
      }
      producer[write[si]] = (int)si;
      ++si;
    }
  }
  auto lo = [&](int t) { return L.off[t]; };
  auto hi = [&](int t) { return L.off[t] + ((long long)1 << prog.tensors[t].rank()) * (L.dep[t] ? L.B : 1); };
  auto overlap = [&](int a, int b) { return lo(a) < hi(b) && lo(b) < hi(a); };
  C.step_deps.assign(n, {});
  C.step_stream.assign(n, 0);
  int last_gemm = -1, rr = 0;
  for (int i = 0; i < n; ++i) {
    std::vector<int>& d = C.step_deps[i];
    for (int t : reads[i])
      if (producer[t] >= 0 && producer[t] < i) d.push_back(producer[t]);
    for (int j = 0; j < i; ++j) {
      bool hit = overlap(write[j], write[i]);
      for (size_t q = 0; q < reads[j].size() && !hit; ++q) hit = overlap(reads[j][q], write[i]);
      if (hit) d.push_back(j);
    }
    if (C.steps[i].first == 2) {
      if (last_gemm >= 0) d.push_back(last_gemm);
      last_gemm = i;
    }
    std::sort(d.begin(), d.end());
    d.erase(std::unique(d.begin(), d.end()), d.end());
    C.step_stream[i] = d.empty() ? (rr++ % N_SIDE_STREAMS) : C.step_stream[d.back()];
  }
}

static bool build_steps(const tnq_plan& P, const Layout& L, ExecConfig& C) {
  const Program& prog = P.prog;
  C.kp.clear();
  C.kshape.clear();
  C.gp.clear();
  C.gsmem.clear();
  C.steps.clear();
  C.step_group.clear();
  C.gb.clear();
  C.ge.clear();
  C.step_bytes.clear();
  C.step_flops.clear();
  C.step_hoist.clear();
  C.hoist_dev.clear();
  C.hoist_first.clear();
  C.hoist_blocks.clear();
  auto tbytes = [&](int t) { return std::ldexp(8.0, prog.tensors[t].rank()) * (L.dep[t] ? L.B : 1); };
  auto bflops = [&](int bi) {
    const PBucket& b = prog.buckets[bi];
    const double full = std::ldexp(1.0, b.r);
    return (6.0 * (b.k - 1) * full + (b.sum ? full : 0.0)) * (L.dep[b.output] ? L.B : 1);
  };
  for (size_t bi = 0; bi < prog.buckets.size(); ++bi) {
    const int gi = prog.group_of.empty() ? -1 : prog.group_of[bi];
    if (gi < 0) {
      bool ok;
      KParams k = single_kparams(P, L, prog.buckets[bi], &ok);
      if (!ok) { set_error("bucket too large for one launch"); return false; }
      C.steps.push_back({0, (int)C.kp.size()});
      C.step_group.push_back(-1);
      C.step_hoist.push_back(L.hoist[bi]);
      C.kp.push_back(k);
      // 2^12 entries per block only when that still gives >= 1024 blocks
      C.kshape.push_back({prog.buckets[bi].k, k.G >= 22 ? 12 : 8});
      double by = tbytes(prog.buckets[bi].output);
      for (int t : prog.buckets[bi].inputs) by += tbytes(t);
      C.step_bytes.push_back(by);
      C.step_flops.push_back(bflops((int)bi));
    } else if ((int)bi == prog.groups[gi].buckets.back() && prog.groups[gi].gemm) {
      GemmBucketArgs G;
      GemmEpilogue E;
      if (!gemm_params(P, L, prog.groups[gi], G, E)) return false;
      C.steps.push_back({2, (int)C.gb.size()});
      C.step_group.push_back(gi);
      C.step_hoist.push_back(0);
      C.gb.push_back(G);
      C.ge.push_back(E);
      double by = tbytes(prog.groups[gi].output);
      for (int t : prog.groups[gi].ext_inputs) by += tbytes(t);
      C.step_bytes.push_back(by);
      double fl = 0;
      for (int b : prog.groups[gi].buckets) fl += bflops(b);
      C.step_flops.push_back(fl);
    } else if ((int)bi == prog.groups[gi].buckets.back()) {
      bool ok;
      int smem = 0;
      GParams g = group_gparams(P, L, prog.groups[gi], &ok, &smem);
      if (!ok) { set_error("fused group does not fit one launch"); return false; }
      C.steps.push_back({1, (int)C.gp.size()});
      C.step_group.push_back(gi);
      C.step_hoist.push_back(0);
      C.gp.push_back(g);
      C.gsmem.push_back(smem);
      double by = tbytes(prog.groups[gi].output);
      for (int t : prog.groups[gi].ext_inputs) by += tbytes(t);
      C.step_bytes.push_back(by);
      double fl = 0;
      for (int b : prog.groups[gi].buckets) fl += bflops(b);
      C.step_flops.push_back(fl);
    }
  }
  // early buckets, level by level (program order within a level)
  int levels = 0;
  for (int h : C.step_hoist) levels = std::max(levels, h);
  for (int l = 1; l <= levels; ++l) {
    C.hoist_first.push_back((int)C.hoist_dev.size());
    int blocks = 0;
    for (size_t i = 0; i < C.steps.size(); ++i) {
      if (C.step_hoist[i] != l) continue;
      const KParams& k = C.kp[C.steps[i].second];
      HoistDev h;
      std::memset(&h, 0, sizeof(h));
      h.out = (long long)reinterpret_cast<size_t>(k.out);
      h.nin = C.kshape[C.steps[i].second].first;
      h.bits = k.G;
      h.sum = k.sum;
      h.out_meta = k.out_meta;
      h.blk0 = blocks;
      h.nvar = k.n_var;
      h.obits = k.out_bits;
      h.out_dep = k.G > k.out_bits;
      for (int j = 0; j < h.nin; ++j) {
        h.in[j] = (long long)reinterpret_cast<size_t>(k.in[j]);
        h.in_meta[j] = k.in_meta[j];
        h.in_dep[j] = k.in_dep[j];
        for (int b = 0; b < k.G; ++b) h.stride[j][b] = k.stride[j][b];
      }
      blocks += (int)(((1ll << k.G) + 255) >> 8);
      C.hoist_dev.push_back(h);
    }
    C.hoist_blocks.push_back(blocks);
  }
  C.hoist_first.push_back((int)C.hoist_dev.size());
  step_dependencies(P, L, C);
  return true;
}

// Host-side bounds check of every launch of configuration (mode, B): each
// input's largest index stays inside its tensor, each output fits its
// allocation, every tensor fits the arena and tensors live at the same time
// do not overlap. Returns an empty string when everything holds.
static std::string validate_config(const tnq_plan& P, int mode, int B) {
  const Layout L = make_layout(P, mode, B);
  ExecConfig C;
  C.L = L;
  if (!build_steps(P, L, C)) return std::string("build_steps failed: ") + tnq_last_error();
  const Program& prog = P.prog;
  const Liveness LV = layout_liveness(prog, L.hoist);
  auto alloc = [&](int t) { return ((long long)1 << prog.tensors[t].rank()) * (L.dep[t] ? B : 1); };
  for (size_t i = 0; i < C.steps.size(); ++i) {  // early buckets: item-invariant, inputs ready before their level
    if (!C.step_hoist[i]) continue;
    const KParams& k = C.kp[C.steps[i].second];
    if (k.G > HOIST_MAX_BITS || (k.G != k.out_bits && k.G != k.out_bits + L.item_bits)) return "early bucket shape";
  }
  for (size_t bi = 0; bi < prog.buckets.size(); ++bi) {
    if (!L.hoist[bi]) continue;
    for (int t : prog.buckets[bi].inputs) {
      const int p = prog.tensors[t].producer;
      if (p >= 0 && (!L.hoist[p] || L.hoist[p] >= L.hoist[bi])) return "early bucket input not ready";
    }
  }
  auto off_of = [&](const void* p) { return (long long)((size_t)p / 8); };
  int single = 0;
  for (size_t bi = 0; bi < prog.buckets.size(); ++bi) {
    if (!prog.group_of.empty() && prog.group_of[bi] >= 0) continue;
    const PBucket& b = prog.buckets[bi];
    const KParams& k = C.kp[single++];
    if ((1ll << k.G) > alloc(b.output)) return "bucket " + std::to_string(bi) + ": output overflows";
    if (off_of(k.out) != L.off[b.output]) return "bucket output pointer";
    for (int jb = 0; jb < b.k; ++jb) {
      // the launch lists the bucket's inputs reordered (thread-varying ones first)
      int j = -1;
      for (int q = 0; q < b.k; ++q)
        if (off_of(k.in[q]) == L.off[b.inputs[jb]]) j = q;
      if (j < 0) return "bucket " + std::to_string(bi) + ": input pointer";
      long long mx = 0;
      for (int i = 0; i < k.G; ++i) mx += k.stride[j][i];
      if (k.sum) mx += 1;
      if (mx >= alloc(b.inputs[jb])) return "bucket " + std::to_string(bi) + ": input " + std::to_string(jb) + " overflows";
      if (k.sum && (((size_t)k.in[j] / 8) & 1)) return "unaligned input";
      for (int i = 0; i < k.G; ++i)
        if (k.sum && (k.stride[j][i] & 1)) return "odd stride in a summing bucket";
    }
  }
  for (size_t si = 0; si < C.steps.size(); ++si) {
    if (C.steps[si].first != 1) continue;
    const size_t gi = (size_t)C.steps[si].second;
    const GParams& G = C.gp[gi];
    const FusedGroup& g = prog.groups[C.step_group[si]];
    const long long items = G.out_dep ? B : 1;
    // largest index of every memory operand over all tiles, items and stages
    std::vector<long long> in_max(G.n_gin, 0);
    for (int j = 0; j < G.n_gin; ++j) {
      long long m = G.gin[j].dep ? (items - 1) * G.gin[j].istride : 0;
      for (int i = 0; i < G.n_h; ++i) m += G.gin[j].hstride[i];
      in_max[j] = m;
    }
    std::vector<long long> chain_max(G.n_st, 0);
    for (int s = 0; s < G.n_st; ++s) {
      const GSt& S = G.st[s];
      if (S.nbits > GL_MAX - 1 || S.n_in > KMAX || S.n_in < 1) return "group stage shape";
      for (int j = 0; j < S.n_in; ++j) {
        // pair loads: u at bit 0 (stride 1) and every other stride even
        if (S.ustride[j] != 1) return "group " + std::to_string(gi) + ": eliminated variable not at bit 0";
        if (j >= S.n_var)
          for (int b = 0; b < S.nbits; ++b)
            if (S.cstride[j][b]) return "group " + std::to_string(gi) + ": constant input varies";
        if (j < S.n_var && j >= S.n_var - S.n_tc) {  // a per-thread pair: thread bits only, from memory
          if (S.src[j] < 0 || S.n_tc >= S.n_var) return "group " + std::to_string(gi) + ": per-thread pair";
          for (int b = GTB; b < S.nbits; ++b)
            if (S.cstride[j][b]) return "group " + std::to_string(gi) + ": per-thread pair varies per entry";
        }
        if (j >= S.n_var && S.kinv) {  // a per-item constant pair: read from memory at the item's base
          if (S.src[j] < 0) return "group " + std::to_string(gi) + ": per-item constant from the chain";
          for (int i = 0; i < G.n_h; ++i)
            if (G.gin[S.src[j]].hstride[i]) return "group " + std::to_string(gi) + ": per-item constant varies";
        }
        for (int b = 0; b < S.nbits; ++b)
          if (S.cstride[j][b] & 1) return "group " + std::to_string(gi) + ": odd local stride";
        if (S.src[j] >= 0) {
          const GIn& in = G.gin[S.src[j]];
          for (int i = 0; i < G.n_h; ++i)
            if (in.hstride[i] >= (1ll << 31)) return "group tile stride does not fit 32 bits";
          if ((in.istride & 1) || ((size_t)in.ptr / 8) % 2) return "group input base not even";
          for (int i = 0; i < G.n_h; ++i)
            if (in.hstride[i] & 1) return "group " + std::to_string(gi) + ": odd tile stride";
        }
        long long m = S.ustride[j];
        for (int b = 0; b < S.nbits; ++b) m += S.cstride[j][b];
        if (S.src[j] < 0) {
          if (s == 0) return "chain input in the first stage";
          if (m >= (1ll << G.st[s - 1].nbits)) return "group " + std::to_string(gi) + ": stage buffer overflow";
        } else {
          if (S.src[j] >= G.n_gin) return "group input index";
          if (in_max[S.src[j]] + m >= alloc(g.ext_inputs[S.src[j]]))
            return "group " + std::to_string(gi) + ": input " + std::to_string(j) + " overflows";
        }
      }
    }
    long long om = G.out_dep ? (items - 1) * G.out_istride : 0;
    for (int i = 0; i < G.n_h; ++i) om += G.out_hstride[i];
    for (int b = 0; b < G.st[G.n_st - 1].nbits; ++b) om += G.out_cstride[b];
    if (om >= alloc(g.output)) return "group " + std::to_string(gi) + ": output overflows";
    if (C.gsmem[gi] > 200 * 1024) return "group shared memory";
    if (G.lean2 && (C.gsmem[gi] < 2 * GTPB * (int)sizeof(float2) || C.gsmem[gi] < (8 << G.st[0].nbits)))
      return "group " + std::to_string(gi) + ": shared memory below the dense stage's reads";
  }
  for (size_t gi = 0; gi < C.gb.size(); ++gi) {
    const GemmBucketArgs& G = C.gb[gi];
    const GemmEpilogue& E = C.ge[gi];
    int grp = -1;
    for (size_t i = 0, n2 = 0; i < C.steps.size(); ++i)
      if (C.steps[i].first == 2 && n2++ == gi) grp = C.step_group[i];
    const FusedGroup& g = prog.groups[grp];
    auto omax = [&](const GemmOperand& o, int nr) {
      long long m = o.dep ? (long long)(G.items - 1) * o.istride : 0;
      for (int i = 0; i < G.ns; ++i) m += o.sstride[i];
      for (int i = 0; i < nr; ++i) m += o.rstride[i];
      for (int i = 0; i < G.nk; ++i) m += o.kstride[i];
      return m;
    };
    std::vector<int> a_ids{g.ga}, b_ids{g.gb};
    a_ids.insert(a_ids.end(), g.a_side.begin(), g.a_side.end());
    b_ids.insert(b_ids.end(), g.b_side.begin(), g.b_side.end());
    for (int j = 0; j < G.na; ++j)
      if (omax(G.a[j], G.nx) >= alloc(a_ids[j])) return "GEMM group: A operand overflows";
    for (int j = 0; j < G.nb; ++j)
      if (omax(G.b[j], G.ny) >= alloc(b_ids[j])) return "GEMM group: B operand overflows";
    long long om = E.dep ? (long long)(G.items - 1) * E.istride : 0;
    for (int i = 0; i < E.ns; ++i) om += E.s[i];
    for (int i = 0; i < E.nx; ++i) om += E.x[i];
    for (int i = 0; i < E.ny; ++i) om += E.y[i];
    if (om >= alloc(g.output)) return "GEMM group: output overflows";
    const GemmShape sh = gemm_shape(P, g, G.items);
    if ((long long)((size_t)L.gemm_off * 8 + 2 * (sh.a_bytes + sh.b_bytes)) > L.arena_elems * 8)
      return "GEMM scratch outside the arena";
    if (G.m_pad % GT_ROWS || (2 * G.n_pad) % GT_ROWS || (2 * G.k_pad * (G.kind == GEMM_BF16 ? 2 : 4)) % GT_KBYTES)
      return "GEMM padding";
    if ((L.gemm_off * 8) % 1024) return "GEMM scratch alignment";
  }
  const int T = (int)prog.tensors.size();
  for (int t = 0; t < T; ++t) {
    if (LV.internal[t]) continue;
    if (L.off[t] < 0 || L.off[t] + alloc(t) > L.arena_elems) return "tensor outside arena";
    if (L.off[t] % 32) return "tensor offset not 256-byte aligned";
  }
  for (int a = 0; a < T; ++a)
    for (int c = a + 1; c < T; ++c) {
      if (LV.internal[a] || LV.internal[c]) continue;
      if (LV.lo[a] <= LV.hi[c] && LV.lo[c] <= LV.hi[a] && L.off[a] < L.off[c] + alloc(c) &&
          L.off[c] < L.off[a] + alloc(a))
        return "live tensors " + std::to_string(a) + " and " + std::to_string(c) + " overlap";
    }
  return "";
}

static cudaError_t allow_group_smem() {
  cudaError_t e = cudaFuncSetAttribute(k_group<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, GROUP_SMEM_BYTES);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_group<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, GROUP_SMEM_BYTES);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_group<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, GROUP_SMEM_BYTES);
}

static tnq_status group_grid_size(int* out, int smem = GROUP_SMEM_BYTES, int kind = 0) {
  int dev = 0, sms = 0, per_sm = 0;
  CU(cudaGetDevice(&dev));
  CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  if (kind == 1) CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_group<1>, GTPB, smem));
  else if (kind == 2) CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_group<2>, GTPB, smem));
  else CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_group<0>, GTPB, smem));
  *out = std::max(1, sms * std::max(1, per_sm));
  return TNQ_OK;
}

static tnq_status build_config(const tnq_plan& P, int mode, int B, ExecConfig** out) {
  CU(allow_group_smem());
  int ggrid = 0;
  tnq_status gst = group_grid_size(&ggrid);
  if (gst != TNQ_OK) return gst;
  ExecConfig* C = new ExecConfig();
  auto fail = [&](tnq_status st) {
    cudaFree(C->d_leaves);
    cudaFree(C->d_scalars);
    cudaFree(C->d_inout);
    cudaFree(C->d_finals);
    cudaFree(C->d_hoist);
    cudaFree(C->d_vals);
    delete C;
    return st;
  };
  C->group_grid = ggrid;
  C->L = make_layout(P, mode, B);
  const Program& prog = P.prog;
  std::vector<LeafDev> leaves, scalars;
  for (int t : prog.leaves)
    leaves.push_back(make_leafdev(P, &prog.tensors[t], prog.tensors[t].leaf_gate, &C->L, t, &C->vals));
  for (int g : prog.scalar_leaves) scalars.push_back(make_leafdev(P, nullptr, g, nullptr, -1, &C->vals));
  std::vector<FinalDev> finals;
  for (int t : prog.finals) finals.push_back(FinalDev{C->L.off[t], t, (int)C->L.dep[t]});
  C->n_leaves = (int)leaves.size();
  C->n_scalars = (int)scalars.size();
  C->n_finals = (int)finals.size();
  C->n_inout = (int)P.net.inout_qubits.size();
  auto up = [](void** dst, const void* src, size_t bytes) -> cudaError_t {
    cudaError_t e = cudaMalloc(dst, bytes ? bytes : 16);
    if (e != cudaSuccess) return e;
    return bytes ? cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice) : cudaSuccess;
  };
  cudaError_t e;
  if ((e = up((void**)&C->d_leaves, leaves.data(), leaves.size() * sizeof(LeafDev))) != cudaSuccess ||
      (e = up((void**)&C->d_scalars, scalars.data(), scalars.size() * sizeof(LeafDev))) != cudaSuccess ||
      (e = up((void**)&C->d_inout, P.net.inout_qubits.data(), P.net.inout_qubits.size() * sizeof(int))) !=
          cudaSuccess ||
      (e = up((void**)&C->d_finals, finals.data(), finals.size() * sizeof(FinalDev))) != cudaSuccess ||
      (e = up((void**)&C->d_vals, C->vals.data(), C->vals.size() * sizeof(float2))) != cudaSuccess) {
    set_error(std::string("uploading plan tables: ") + cudaGetErrorString(e));
    return fail(TNQ_ECUDA);
  }
  if (!build_steps(P, C->L, *C)) return fail(TNQ_EUNSUPPORTED);
  for (size_t i = 0; i < C->gsmem.size(); ++i) {  // chains with a register tail: more blocks may fit
    int g = 0;
    if ((gst = group_grid_size(&g, C->gsmem[i], C->gp[i].tail > 0 ? 1 : (C->gp[i].lean2 ? 2 : 0))) != TNQ_OK) return fail(gst);
    C->ggrid.push_back(g);
  }
  if ((e = up((void**)&C->d_hoist, C->hoist_dev.data(), C->hoist_dev.size() * sizeof(HoistDev))) != cudaSuccess) {
    set_error(std::string("uploading plan tables: ") + cudaGetErrorString(e));
    return fail(TNQ_ECUDA);
  }
  *out = C;
  return TNQ_OK;
}

template <int NIN>
static void launch_bucket_n(const KParams& k, int LT, cudaStream_t s) {
  const long long total = 1ll << k.G;
  if (LT == 8) {
    k_bucket<NIN, 8><<<(unsigned)std::max(1ll, total >> 8), TPB, 0, s>>>(k);
  } else {
    k_bucket<NIN, 12><<<(unsigned)std::max(1ll, (total + 4095) >> 12), TPB, 0, s>>>(k);
  }
}

static void launch_bucket(const KParams& k, int n_in, int LT, cudaStream_t s) {
  switch (n_in) {
    case 1: launch_bucket_n<1>(k, LT, s); break;
    case 2: launch_bucket_n<2>(k, LT, s); break;
    case 3: launch_bucket_n<3>(k, LT, s); break;
    case 4: launch_bucket_n<4>(k, LT, s); break;
    case 5: launch_bucket_n<5>(k, LT, s); break;
    case 6: launch_bucket_n<6>(k, LT, s); break;
    case 7: launch_bucket_n<7>(k, LT, s); break;
    default: launch_bucket_n<8>(k, LT, s); break;
  }
}

// Launches step i of the configuration (a single bucket or a fused group)
// with its pointers rebased on the arena.
static void launch_step(const ExecConfig& C, int i, float2* arena, int* me, unsigned* mm, int* status,
                        cudaStream_t s) {
  char* base = reinterpret_cast<char*>(arena);
  const auto st = C.steps[i];
  if (st.first == 0) {
    KParams k = C.kp[st.second];
    k.out = reinterpret_cast<float2*>(base + reinterpret_cast<size_t>(k.out));
    for (int j = 0; j < C.kshape[st.second].first; ++j)
      k.in[j] = reinterpret_cast<const float2*>(base + reinterpret_cast<size_t>(k.in[j]));
    k.meta_e = me;
    k.meta_m = mm;
    launch_bucket(k, C.kshape[st.second].first, C.kshape[st.second].second, s);
  } else if (st.first == 2) {
    GemmBucketArgs g = C.gb[st.second];
    GemmEpilogue e = C.ge[st.second];
    auto rb = [&](const void* p) { return reinterpret_cast<const float2*>(base + reinterpret_cast<size_t>(p)); };
    for (int j = 0; j < g.na; ++j) g.a[j].ptr = rb(g.a[j].ptr);
    for (int j = 0; j < g.nb; ++j) g.b[j].ptr = rb(g.b[j].ptr);
    g.a_hi = base + reinterpret_cast<size_t>(g.a_hi);
    g.a_lo = base + reinterpret_cast<size_t>(g.a_lo);
    g.b_hi = base + reinterpret_cast<size_t>(g.b_hi);
    g.b_lo = base + reinterpret_cast<size_t>(g.b_lo);
    g.meta_e = me;
    g.meta_m = mm;
    e.out = reinterpret_cast<float2*>(base + reinterpret_cast<size_t>(e.out));
    e.meta_m = mm;
    gemm_bucket_launch(g, e, status, s);
  } else {
    GParams g = C.gp[st.second];
    g.out = reinterpret_cast<float2*>(base + reinterpret_cast<size_t>(g.out));
    for (int j = 0; j < g.n_gin; ++j) g.gin[j].ptr = reinterpret_cast<const float2*>(base + reinterpret_cast<size_t>(g.gin[j].ptr));
    g.meta_e = me;
    g.meta_m = mm;
    const long long tiles = (g.out_dep ? (long long)g.B : 1ll) << g.n_h;
    const long long grid =
        std::min<long long>(tiles, (long long)(C.ggrid.empty() ? C.group_grid : C.ggrid[st.second]));
    if (g.tail) k_group<1><<<(unsigned)grid, GTPB, C.gsmem[st.second], s>>>(g, tiles);
    else if (g.lean2) k_group<2><<<(unsigned)grid, GTPB, C.gsmem[st.second], s>>>(g, tiles);
    else k_group<0><<<(unsigned)grid, GTPB, C.gsmem[st.second], s>>>(g, tiles);
  }
}

// Enqueues one batch (everything after the header upload) on stream s.
// Side streams and per-step events used while a batch is captured into a graph
// (fork from the capturing stream, join before the final kernels).
struct SideStreams {
  cudaStream_t st[N_SIDE_STREAMS] = {};
  cudaEvent_t fork = nullptr;
  cudaEvent_t join[N_SIDE_STREAMS] = {};
  std::vector<cudaEvent_t> done;  // one per step
};

static void enqueue_batch(const tnq_plan& P, ExecConfig& C, char* ws, cudaStream_t s,
                          const SideStreams* side = nullptr) {
  const Layout& L = C.L;
  const int B = L.B;
  const int T = (int)P.prog.tensors.size();
  auto* hdr = reinterpret_cast<const BatchHdr*>(ws + L.hdr_off);
  auto* bits = reinterpret_cast<const unsigned*>(ws + L.bits_off);
  auto* scal = reinterpret_cast<double2*>(ws + L.scalar_off);
  auto* res = reinterpret_cast<double2*>(ws + L.res_off);
  auto* part = reinterpret_cast<double2*>(ws + L.part_off);
  auto* me = reinterpret_cast<int*>(ws + L.meta_e_off);
  auto* mm = reinterpret_cast<unsigned*>(ws + L.meta_m_off);
  auto* arena = reinterpret_cast<float2*>(ws + L.arena_off);
  cudaMemsetAsync(mm, 0, (size_t)T * B * 4, s);
  if (C.n_leaves) {
    long long n = (long long)C.n_leaves * B;
    k_leaf_init<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(C.d_leaves, C.n_leaves, hdr, bits, C.d_vals, arena, B);
  }
  k_scalar_init<<<(B + 127) / 128, 128, 0, s>>>(C.d_scalars, C.n_scalars, C.d_inout, C.n_inout, hdr, bits, C.d_vals,
                                                scal, B);
  int* status = reinterpret_cast<int*>(ws + L.status_off);
  // early buckets first, one launch per level; their steps launch nothing below
  for (size_t l = 0; l + 1 < C.hoist_first.size(); ++l)
    k_bucket_level<<<(unsigned)C.hoist_blocks[l], 256, 0, s>>>(C.d_hoist + C.hoist_first[l],
                                                                 C.hoist_first[l + 1] - C.hoist_first[l],
                                                                 reinterpret_cast<char*>(arena), me, mm, B);
  if (!side) {
    for (size_t i = 0; i < C.steps.size(); ++i)
      if (!C.step_hoist[i]) launch_step(C, (int)i, arena, me, mm, status, s);
  } else {
    cudaEventRecord(side->fork, s);
    for (int k = 0; k < N_SIDE_STREAMS; ++k) cudaStreamWaitEvent(side->st[k], side->fork, 0);
    for (size_t i = 0; i < C.steps.size(); ++i) {
      const int k = C.step_stream[i];
      for (int j : C.step_deps[i])
        if (C.step_stream[j] != k) cudaStreamWaitEvent(side->st[k], side->done[j], 0);
      if (!C.step_hoist[i]) launch_step(C, (int)i, arena, me, mm, status, side->st[k]);
      cudaEventRecord(side->done[i], side->st[k]);
    }
    for (int k = 0; k < N_SIDE_STREAMS; ++k) {
      cudaEventRecord(side->join[k], side->st[k]);
      cudaStreamWaitEvent(s, side->join[k], 0);
    }
  }
  // amplitude scale 2^(-n_sqrt2 / 2 + leaf_exp): sqrt2 factors of the gates,
  // power-of-two factors taken out of a general network's tensors
  const int n_sqrt2 = P.net.n_sqrt2;
  const long long le = std::max<long long>(-100000, std::min<long long>(100000, P.net.leaf_exp));
  const int scale_exp = -(n_sqrt2 / 2) + (int)le, scale_half = n_sqrt2 & 1;
  k_finalize<<<(B + 127) / 128, 128, 0, s>>>(C.d_finals, C.n_finals, scal, arena, me, B, hdr, scale_exp, scale_half,
                                              res);
  k_slice_sum<<<(L.n_rows + 127) / 128, 128, 0, s>>>(res, B, hdr, part, L.n_rows);
}

static bool use_graphs() {
  const char* e = getenv("TNQ_NO_GRAPH");
  return !(e && e[0] == '1');
}

// Runs the batch: header upload, then the captured graph (or direct launches).
// The header comes from host memory, or (d_hdr != nullptr) from device memory
// already holding it, which keeps the copy asynchronous.
static tnq_status run_batch(const tnq_plan& P, ExecConfig& C, char* ws, cudaStream_t s, const BatchHdr& h,
                            const BatchHdr* d_hdr = nullptr) {
  if (d_hdr) CU(cudaMemcpyAsync(ws + C.L.hdr_off, d_hdr, sizeof(BatchHdr), cudaMemcpyDeviceToDevice, s));
  else CU(cudaMemcpyAsync(ws + C.L.hdr_off, &h, sizeof(h), cudaMemcpyHostToDevice, s));
  if (!use_graphs()) {
    enqueue_batch(P, C, ws, s);
    CU(cudaGetLastError());
    return TNQ_OK;
  }
  if (C.exec && C.ws != ws) {
    cudaGraphExecDestroy(C.exec);
    C.exec = nullptr;
  }
  if (!C.exec) {
    cudaStream_t cap;
    CU(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    SideStreams side;
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < N_SIDE_STREAMS && e == cudaSuccess; ++k) {
      e = cudaStreamCreateWithFlags(&side.st[k], cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&side.join[k], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&side.fork, cudaEventDisableTiming);
    side.done.assign(C.steps.size(), nullptr);
    for (size_t i = 0; i < side.done.size() && e == cudaSuccess; ++i)
      e = cudaEventCreateWithFlags(&side.done[i], cudaEventDisableTiming);
    cudaGraph_t g = nullptr;
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      enqueue_batch(P, C, ws, cap, &side);
      e = cudaStreamEndCapture(cap, &g);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&C.exec, g, 0);
    if (g) cudaGraphDestroy(g);
    for (cudaEvent_t ev : side.done)
      if (ev) cudaEventDestroy(ev);
    for (int k = 0; k < N_SIDE_STREAMS; ++k) {
      if (side.join[k]) cudaEventDestroy(side.join[k]);
      if (side.st[k]) cudaStreamDestroy(side.st[k]);
    }
    if (side.fork) cudaEventDestroy(side.fork);
    cudaStreamDestroy(cap);
    if (e != cudaSuccess) {
      C.exec = nullptr;
      set_error(std::string("graph capture: ") + cudaGetErrorString(e));
      return TNQ_ECUDA;
    }
    C.ws = ws;
  }
  CU(cudaGraphLaunch(C.exec, s));
  return TNQ_OK;
}

static int ilog2_floor(uint64_t x) {
  int b = 0;
  while ((2ull << b) <= x) ++b;
  return b;
}

static tnq_status get_config(const tnq_plan& P, int mode, int B, ExecConfig** out) {
  int dev;
  CU(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(P.dev_mu);
  if (P.dev && P.dev->device != dev) {
    set_error("plan already bound to another CUDA device");
    return TNQ_EINVAL;
  }
  if (!P.dev) {
    P.dev = new DeviceState();
    P.dev->device = dev;
  }
  auto key = std::make_pair(mode, B);
  auto it = P.dev->configs.find(key);
  if (it != P.dev->configs.end()) {
    *out = it->second;
    return TNQ_OK;
  }
  ExecConfig* C = nullptr;
  tnq_status st = build_config(P, mode, B, &C);
  if (st != TNQ_OK) return st;
  P.dev->configs[key] = C;
  *out = C;
  return TNQ_OK;
}

static tnq_status check_device() {
  int n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess || n == 0) {
    set_error(std::string("no CUDA device: ") + cudaGetErrorString(e));
    return TNQ_EUNSUPPORTED;
  }
  return TNQ_OK;
}

// Workspace bytes of configuration (mode, B), cached per plan.
static size_t layout_bytes(const tnq_plan& P, int mode, int B) {
  {
    std::lock_guard<std::mutex> lk(P.layout_mu);
    auto it = P.layout_bytes.find({mode, B});
    if (it != P.layout_bytes.end()) return it->second;
  }
  const size_t b = make_layout(P, mode, B).total;
  std::lock_guard<std::mutex> lk(P.layout_mu);
  P.layout_bytes[{mode, B}] = b;
  return b;
}

// Largest power-of-two batch (<= cap) whose workspace fits.
static int pick_batch(const tnq_plan& P, int mode, size_t ws_bytes, uint64_t cap) {
  int best = 0;
  for (int b = 0; b <= MAX_ITEM_BITS; ++b) {
    const uint64_t B = 1ull << b;
    if (B > cap && b > 0) break;
    if (layout_bytes(P, mode, (int)B) <= ws_bytes) best = (int)B;
    else break;
  }
  return best;
}

static void pack_bits(const uint8_t* bits, int n, std::vector<unsigned>& out) {
  for (int q = 0; q < n; ++q)
    if (bits[q]) out[q >> 5] |= 1u << (q & 31);
}

}  // namespace tnq

using namespace tnq;

extern "C" {

// Internal test hook (not in include/tnq.h): host-side bounds check of the
// launches of configuration (mode, batch). Returns 0 and "" when they hold.
int tnq_internal_validate(const tnq_plan* plan, int mode, uint32_t batch, char* msg, size_t msg_len) {
  std::string m = plan ? validate_config(*plan, mode, (int)batch) : std::string("NULL plan");
  if (msg && msg_len) {
    std::strncpy(msg, m.c_str(), msg_len - 1);
    msg[msg_len - 1] = 0;
  }
  return m.empty() ? 0 : 1;
}

// Internal hook (not in include/tnq.h; host only): the kernel kind of every
// step of the (mode, batch) configuration in program order (0 k_bucket,
// 1 k_group, 2 GEMM) and, for steps of a group, its bucket count.
int tnq_internal_step_kinds(const tnq_plan* plan, int mode, uint32_t batch, int32_t* kind, int32_t* nbk, int cap,
                            int32_t* out_n) {
  if (!plan || !kind || !out_n) return 1;
  ExecConfig C;
  C.L = make_layout(*plan, mode, (int)batch);
  if (!build_steps(*plan, C.L, C)) return 1;
  *out_n = (int32_t)C.steps.size();
  if ((int)C.steps.size() > cap) return 1;
  for (size_t i = 0; i < C.steps.size(); ++i) {
    kind[i] = C.steps[i].first;
    if (nbk) nbk[i] = C.step_group[i] < 0 ? 1 : (int32_t)plan->prog.groups[C.step_group[i]].buckets.size();
  }
  return 0;
}

// Internal hook (not in include/tnq.h; host only): for every fused-chain step
// of configuration (mode, batch), in program order, the number of its later
// stages that run as register subtrees (0: all stages in shared memory).
int tnq_internal_group_tails(const tnq_plan* plan, int mode, uint32_t batch, int32_t* tails, int cap,
                             int32_t* out_n) {
  if (!plan || !out_n) return 1;
  ExecConfig C;
  C.L = make_layout(*plan, mode, (int)batch);
  if (!build_steps(*plan, C.L, C)) return 1;
  *out_n = (int32_t)C.gp.size();
  if ((int)C.gp.size() > cap) return 1;
  for (size_t i = 0; i < C.gp.size(); ++i) tails[i] = C.gp[i].tail;
  return 0;
}

// Internal hook (not in include/tnq.h; host only): for every GEMM step of
// configuration (mode, batch), in program order, 1 when it runs in the fused-A
// form (A read from its complex tensor inside the GEMM kernel) for a workspace
// whose base is 256-byte aligned, else 0.
int tnq_internal_gemm_forms(const tnq_plan* plan, int mode, uint32_t batch, int32_t* fused, int cap,
                            int32_t* out_n) {
  if (!plan || !out_n) return 1;
  ExecConfig C;
  C.L = make_layout(*plan, mode, (int)batch);
  if (!build_steps(*plan, C.L, C)) return 1;
  *out_n = (int32_t)C.gb.size();
  if ((int)C.gb.size() > cap) return 1;
  for (size_t i = 0; i < C.gb.size(); ++i) {
    GemmBucketArgs g = C.gb[i];
    g.a[0].ptr = reinterpret_cast<const float2*>(reinterpret_cast<size_t>(g.a[0].ptr) + 256);  // arena offset + base
    fused[i] = gemm_fused_a(g) ? 1 : 0;
  }
  return 0;
}

// Internal hook (not in include/tnq.h; host only): a text description of every
// fused-chain step of configuration (mode, batch): per stage its local bits,
// and per operand its source and the local bits it holds (nonzero strides),
// plus the tile bits each external input holds. For planning the tile shape.
int tnq_internal_group_text(const tnq_plan* plan, int mode, uint32_t batch, char* buf, size_t cap) {
  if (!plan || !buf || cap == 0) return 1;
  ExecConfig C;
  C.L = make_layout(*plan, mode, (int)batch);
  if (!build_steps(*plan, C.L, C)) return 1;
  std::string out;
  for (size_t gi = 0; gi < C.gp.size(); ++gi) {
    const GParams& G = C.gp[gi];
    out += "group " + std::to_string(gi) + " stages " + std::to_string(G.n_st) + " tail " + std::to_string(G.tail) +
           " n_h " + std::to_string(G.n_h) + " gin " + std::to_string(G.n_gin) + " lean2 " + std::to_string(G.lean2) +
           " smem " + std::to_string(C.gsmem[gi]) + "\n";
    for (int j = 0; j < G.n_gin; ++j) {
      int nh = 0;
      for (int i = 0; i < G.n_h; ++i) nh += G.gin[j].hstride[i] != 0;
      out += "  gin " + std::to_string(j) + " tile bits held " + std::to_string(nh) + " dep " +
             std::to_string(G.gin[j].dep) + "\n";
    }
    for (int st = 0; st < G.n_st; ++st) {
      const GSt& S = G.st[st];
      out += "  stage " + std::to_string(st) + " nbits " + std::to_string(S.nbits) + " n_in " + std::to_string(S.n_in) +
             " n_var " + std::to_string(S.n_var) + " n_tc " + std::to_string(S.n_tc) + " pd " + std::to_string(S.pd) + "\n";
      for (int j = 0; j < S.n_in; ++j) {
        out += "    in src " + std::to_string(S.src[j]) + " ustride " + std::to_string(S.ustride[j]) + " local:";
        for (int b = 0; b < S.nbits; ++b) out += S.cstride[j][b] ? " " + std::to_string(S.cstride[j][b]) : " .";
        out += "\n";
      }
    }
  }
  for (size_t ki = 0; ki < C.kp.size(); ++ki) {
    const KParams& K = C.kp[ki];
    if (K.out_bits < 18) continue;
    out += "bucket " + std::to_string(ki) + " G " + std::to_string(K.G) + " out_bits " + std::to_string(K.out_bits) +
           " nin " + std::to_string(C.kshape[ki].first) + " sum " + std::to_string(K.sum) + "\n";
    for (int j = 0; j < C.kshape[ki].first; ++j) {
      out += "   in " + std::to_string(j) + " strides(bits 0-9):";
      for (int b = 0; b < 10 && b < K.G; ++b) out += " " + std::to_string(K.stride[j][b]);
      out += "\n";
    }
  }
  for (size_t gi = 0; gi < C.gb.size(); ++gi) {
    const GemmBucketArgs& G = C.gb[gi];
    out += "gemm " + std::to_string(gi) + " ns " + std::to_string(G.ns) + " nx " + std::to_string(G.nx) + " ny " +
           std::to_string(G.ny) + " nk " + std::to_string(G.nk) + " items " + std::to_string(G.items) + " pads " +
           std::to_string(G.m_pad) + "x" + std::to_string(G.n_pad) + "x" + std::to_string(G.k_pad) + " na " +
           std::to_string(G.na) + " nb " + std::to_string(G.nb) + " a0.kstride";
    for (int q = 0; q < G.nk && q < 6; ++q) out += " " + std::to_string(G.a[0].kstride[q]);
    out += " a0.rstride";
    for (int q = 0; q < G.nx; ++q) out += " " + std::to_string(G.a[0].rstride[q]);
    out += " a0.sstride";
    for (int q = 0; q < G.ns; ++q) out += " " + std::to_string(G.a[0].sstride[q]);
    out += " a0.istride " + std::to_string(G.a[0].istride) + " dep " + std::to_string(G.a[0].dep);
    out += "\n";
  }
  std::snprintf(buf, cap, "%s", out.c_str());
  return out.size() + 1 > cap ? 2 : 0;
}

// Internal hook (not in include/tnq.h; host only): the concurrency structure of
// configuration (mode, batch) for checking it on the host. Per step: its side
// stream, the tensor it writes, up to 16 tensors it reads (-1 past the end) and
// its dependencies (CSR: dep_off[n+1], deps); per tensor: arena offset and
// length in elements (-1 when not stored). Returns 1 if a capacity is short.
int tnq_internal_step_deps(const tnq_plan* plan, int mode, uint32_t batch, int cap_steps, int cap_deps,
                           int cap_tensors, int32_t* n_steps, int32_t* stream, int32_t* write, int32_t* reads16,
                           int32_t* dep_off, int32_t* deps, int64_t* t_off, int64_t* t_len) {
  if (!plan || !n_steps) return 1;
  ExecConfig C;
  C.L = make_layout(*plan, mode, (int)batch);
  if (!build_steps(*plan, C.L, C)) return 1;
  const Program& prog = plan->prog;
  const int n = (int)C.steps.size();
  *n_steps = n;
  if (n > cap_steps || (int)prog.tensors.size() > cap_tensors) return 1;
  size_t nd = 0;
  for (int i = 0; i < n; ++i) nd += C.step_deps[i].size();
  if ((int)nd > cap_deps) return 1;
  const Liveness LV = tensor_liveness(prog);
  for (size_t t = 0; t < prog.tensors.size(); ++t) {
    const bool stored = !LV.internal[t];
    t_off[t] = stored ? C.L.off[t] : -1;
    t_len[t] = stored ? ((int64_t)1 << prog.tensors[t].rank()) * (C.L.dep[t] ? C.L.B : 1) : -1;
  }
  size_t si = 0, k = 0;
  for (size_t bi = 0; bi < prog.buckets.size() && si < (size_t)n; ++bi) {
    const int gi = prog.group_of.empty() ? -1 : prog.group_of[bi];
    const std::vector<int>* rd;
    int w;
    if (gi < 0) {
      rd = &prog.buckets[bi].inputs;
      w = prog.buckets[bi].output;
    } else if ((int)bi == prog.groups[gi].buckets.back()) {
      rd = &prog.groups[gi].ext_inputs;
      w = prog.groups[gi].output;
    } else {
      continue;
    }
    stream[si] = C.step_stream[si];
    write[si] = w;
    for (int q = 0; q < 16; ++q) reads16[16 * si + q] = q < (int)rd->size() ? (*rd)[q] : -1;
    dep_off[si] = (int32_t)k;
    for (int j : C.step_deps[si]) deps[k++] = j;
    ++si;
  }
  dep_off[n] = (int32_t)k;
  return 0;
}

// Internal measurement hook (not in include/tnq.h): runs the first batch of
// tnq_contract_sliced(plan, bits, s0, s1, ...) with direct launches and a
// CUDA event pair around every bucket launch on `stream`. Per bucket it
// returns the launch time (ms), the algorithmic bytes of the launch (every
// operand read once, the output written once; 8 B per complex64) and the bag
// size r (of the first bucket for a group), the algorithmic flops (cost
// model, all items) and the kind (0: one bucket, m > 1: a fused group of m
// buckets, 100 + m: a GEMM group of m buckets). *out_n = launches, *out_B = batch.
}  // extern "C"

namespace tnq {
// Runs the first batch of tnq_contract_sliced(plan, bits, s0, s1, ...) with
// direct launches and a CUDA event pair around every step; returns per-step
// times (ms) and the configuration used.
static tnq_status profile_steps(const tnq_plan* plan, const uint8_t* bits, uint64_t s0, uint64_t s1, void* workspace,
                                size_t ws_bytes, uint32_t max_batch, void* stream, std::vector<float>& ms,
                                ExecConfig** cfg) {
  if (!plan || (!bits && plan->net.n_qubits > 0) || !workspace || s1 <= s0 || s1 > (1ull << plan->mu.size())) {
    set_error("bad profile arguments");
    return TNQ_EINVAL;
  }
  tnq_status st = check_device();
  if (st != TNQ_OK) return st;
  uint64_t cap_b = 1;
  while (cap_b < s1 - s0 && cap_b < (1ull << MAX_ITEM_BITS)) cap_b <<= 1;
  if (max_batch > 0) cap_b = std::min<uint64_t>(cap_b, 1ull << ilog2_floor(max_batch));
  const int B = pick_batch(*plan, 0, ws_bytes, cap_b);
  if (B == 0) {
    set_error("workspace too small for one slice");
    return TNQ_ENOMEM;
  }
  ExecConfig* C = nullptr;
  if ((st = get_config(*plan, 0, B, &C)) != TNQ_OK) return st;
  const int nbk = (int)C->steps.size();
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  char* ws = reinterpret_cast<char*>(workspace);
  std::vector<unsigned> words((size_t)C->L.n_words * C->L.n_rows, 0u);
  pack_bits(bits, plan->net.n_qubits, words);
  CU(cudaMemcpyAsync(ws + C->L.bits_off, words.data(), words.size() * 4, cudaMemcpyHostToDevice, s));
  BatchHdr h;
  std::memset(&h, 0, sizeof(h));
  h.item_base = s0;
  h.item_end = s1;
  h.p = (int)plan->mu.size();
  h.n_words = C->L.n_words;
  CU(cudaMemcpyAsync(ws + C->L.hdr_off, &h, sizeof(h), cudaMemcpyHostToDevice, s));
  const Layout& L = C->L;
  const int T = (int)plan->prog.tensors.size();
  auto* hdr = reinterpret_cast<const BatchHdr*>(ws + L.hdr_off);
  auto* bw = reinterpret_cast<const unsigned*>(ws + L.bits_off);
  auto* arena = reinterpret_cast<float2*>(ws + L.arena_off);
  auto* me = reinterpret_cast<int*>(ws + L.meta_e_off);
  auto* mm = reinterpret_cast<unsigned*>(ws + L.meta_m_off);
  CU(cudaMemsetAsync(mm, 0, (size_t)T * B * 4, s));
  CU(cudaMemsetAsync(ws + L.status_off, 0, 4, s));
  if (C->n_leaves) {
    long long n = (long long)C->n_leaves * B;
    k_leaf_init<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(C->d_leaves, C->n_leaves, hdr, bw, C->d_vals, arena, B);
  }
  std::vector<cudaEvent_t> ev(2 * (size_t)nbk);
  for (auto& e : ev) CU(cudaEventCreate(&e));
  for (int i = 0; i < nbk; ++i) {
    CU(cudaEventRecord(ev[2 * i], s));
    launch_step(*C, i, arena, me, mm, reinterpret_cast<int*>(ws + L.status_off), s);
    CU(cudaEventRecord(ev[2 * i + 1], s));
  }
  CU(cudaGetLastError());
  CU(cudaStreamSynchronize(s));
  ms.assign(nbk, 0.f);
  for (int i = 0; i < nbk; ++i) CU(cudaEventElapsedTime(&ms[i], ev[2 * i], ev[2 * i + 1]));
  for (auto& e : ev) cudaEventDestroy(e);
  *cfg = C;
  return TNQ_OK;
}

// Drops every device configuration of the plan (after its program changed).
void reset_device_state(const tnq_plan& P) {
  {
    std::lock_guard<std::mutex> lk(P.dev_mu);
    if (P.dev) {
      destroy_device_state(P.dev);
      P.dev = nullptr;
    }
  }
  std::lock_guard<std::mutex> lk(P.layout_mu);
  P.layout_bytes.clear();
}
}  // namespace tnq

// FP32 FMA throughput probe: every thread runs 8 independent FMA chains of
// 16 x iters steps (x = x a + b, bounded for |a| < 1), so the FMA pipes of
// every SM stay busy; the result only feeds a store that never happens for
// these inputs, which keeps the loop.
__global__ void __launch_bounds__(256) k_ffma_peak(float a, float b, int iters, float* out) {
  float x[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) x[i] = threadIdx.x * 1e-3f + (float)i;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < 16; ++k)
#pragma unroll
      for (int i = 0; i < 8; ++i) x[i] = fmaf(x[i], a, b);
  }
  float sum = 0.f;
#pragma unroll
  for (int i = 0; i < 8; ++i) sum += x[i];
  if (sum == -1.2345e30f) out[0] = sum;
}

extern "C" {

// Internal measurement hook (not in include/tnq.h): measured FP32 FMA peak of
// the current device in TFLOP/s (2 flops per FMA), the best of `reps` timed
// launches of k_ffma_peak on `stream` (SMs x 8 blocks of 256 threads). The
// roofline of the fused chain kernel, whose arithmetic is FP32 FMA/FMUL,
// divides by it.
int tnq_internal_fp32_peak(int reps, void* stream, double* out_tflops) {
  if (!out_tflops || reps < 1) return 1;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 1;
  const int blocks = sms * 8, iters = 4096;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return 1;
  if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return 1; }
  float best = 0.f;
  k_ffma_peak<<<blocks, 256, 0, s>>>(0.999f, 1e-3f, iters, nullptr);  // warm-up
  for (int r = 0; r < reps; ++r) {
    cudaEventRecord(e0, s);
    k_ffma_peak<<<blocks, 256, 0, s>>>(0.999f, 1e-3f, iters, nullptr);
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms > 0.f && (best == 0.f || ms < best)) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (cudaGetLastError() != cudaSuccess || best <= 0.f) return 1;
  const double flops = 2.0 * 8 * 16 * (double)iters * 256.0 * blocks;
  *out_tflops = flops / (best * 1e-3) / 1e12;
  return 0;
}

int tnq_internal_profile(const tnq_plan* plan, const uint8_t* bits, uint64_t s0, uint64_t s1, void* workspace,
                         size_t ws_bytes, uint32_t max_batch, void* stream, int cap, float* ms, double* bytes,
                         double* flops, int* bag, int* kind, int* out_n, int* out_B) {
  std::vector<float> t;
  ExecConfig* C = nullptr;
  tnq_status st = profile_steps(plan, bits, s0, s1, workspace, ws_bytes, max_batch, stream, t, &C);
  if (st != TNQ_OK) return st;
  const int nbk = (int)C->steps.size();
  if (cap < nbk) return TNQ_EINVAL;
  const Program& prog = plan->prog;
  int single = 0;
  for (int i = 0; i < nbk; ++i) {
    ms[i] = t[i];
    bytes[i] = C->step_bytes[i];
    flops[i] = C->step_flops[i];
    const auto st2 = C->steps[i];
    if (st2.first == 0) {
      int bi = 0, seen = -1;  // the st2.second-th single bucket
      for (; bi < (int)prog.buckets.size(); ++bi)
        if ((prog.group_of.empty() || prog.group_of[bi] < 0) && ++seen == st2.second) break;
      bag[i] = prog.buckets[bi].r;
      kind[i] = 0;
      ++single;
    } else {
      const FusedGroup& g = prog.groups[C->step_group[i]];
      bag[i] = prog.buckets[g.buckets.front()].r;
      kind[i] = (int)g.buckets.size() + (g.gemm ? 100 : 0);
    }
  }
  *out_n = nbk;
  *out_B = C->L.B;
  return TNQ_OK;
}

namespace tnq {
// profile_steps run `reps` times with the same configuration, keeping each
// step's shortest time (the first run of a configuration also pays one-time
// costs: table uploads, module loading, cold caches).
static tnq_status profile_steps_min(const tnq_plan* plan, const uint8_t* bits, uint64_t s0, uint64_t s1,
                                    void* workspace, size_t ws_bytes, uint32_t max_batch, void* stream,
                                    std::vector<float>& ms, ExecConfig** cfg, int reps = 3) {
  std::vector<float> t;
  for (int r = 0; r < reps; ++r) {
    tnq_status st = profile_steps(plan, bits, s0, s1, workspace, ws_bytes, max_batch, stream, t, cfg);
    if (st != TNQ_OK) return st;
    if (r == 0) ms = t;
    else
      for (size_t i = 0; i < ms.size() && i < t.size(); ++i) ms[i] = std::min(ms[i], t[i]);
  }
  return TNQ_OK;
}
}  // namespace tnq

}  // extern "C"

namespace tnq {
// Chain selection for the plan's current program: times one batch with every
// candidate chain fused and one with every bucket separate (CUDA events per
// launch) and keeps each chain only where it is faster; when a GEMM chain is
// rejected, the fusion pass is run again around the kept GEMM chains and the
// new candidates are timed the same way. Leaves the selection applied and
// returns the batch time of the selected configuration in *total_ms.
static tnq_status select_chains(tnq_plan* plan, const uint8_t* bits, void* workspace, size_t ws_bytes, uint64_t cap,
                                void* stream, float* total_ms) {
  Program& prog = plan->prog;
  const std::vector<FusedGroup> all = prog.groups;
  const uint64_t n_sl = 1ull << plan->mu.size();
  // one batch size for both forms: the largest that fits both layouts
  const int b_fused = pick_batch(*plan, 0, ws_bytes, cap);
  set_groups(prog, {});
  reset_device_state(*plan);
  const int b_plain = pick_batch(*plan, 0, ws_bytes, cap);
  set_groups(prog, all);
  reset_device_state(*plan);
  const int B = std::min(b_fused, b_plain);
  if (B == 0) { set_error("workspace too small for one slice of the unfused plan"); return TNQ_ENOMEM; }
  std::vector<float> tf, tu;
  ExecConfig* C = nullptr;
  tnq_status st;
  std::vector<FusedGroup> keep;
  if (!all.empty()) {
    // every candidate chain fused
    st = profile_steps_min(plan, bits, 0, n_sl, workspace, ws_bytes, (uint32_t)B, stream, tf, &C);
    if (st != TNQ_OK) return st;
    std::vector<float> group_ms(all.size(), 0.f);
    for (size_t i = 0; i < C->steps.size(); ++i)
      if (C->step_group[i] >= 0) group_ms[C->step_group[i]] = tf[i];
    // no chain fused: one step per bucket, in bucket order
    set_groups(prog, {});
    reset_device_state(*plan);
    st = profile_steps_min(plan, bits, 0, n_sl, workspace, ws_bytes, (uint32_t)B, stream, tu, &C);
    if (st != TNQ_OK) {
      set_groups(prog, all);
      reset_device_state(*plan);
      return st;
    }
    bool gemm_dropped = false;
    for (size_t g = 0; g < all.size(); ++g) {
      float t_unfused = 0.f;
      for (int b : all[g].buckets) t_unfused += tu[b];
      if (group_ms[g] < t_unfused) keep.push_back(all[g]);
      else gemm_dropped |= all[g].gemm;
    }
    if (gemm_dropped && plan->opts.fuse_min_rank > 0) {
      // buckets of a rejected GEMM chain may still fuse as a shared-memory
      // chain (possibly joined with their neighbours): propose those chains
      // around the kept GEMM chains and time them against the unfused form
      std::vector<FusedGroup> gemms;
      for (const auto& g : keep)
        if (g.gemm) gemms.push_back(g);
      set_groups(prog, gemms);
      fuse_chains(prog, plan->order, plan->opts.fuse_min_rank);
      const std::vector<FusedGroup> all2 = prog.groups;
      reset_device_state(*plan);
      std::vector<float> tf2;
      st = profile_steps_min(plan, bits, 0, n_sl, workspace, ws_bytes, (uint32_t)B, stream, tf2, &C);
      if (st != TNQ_OK) {
        set_groups(prog, keep);
        reset_device_state(*plan);
        return st;
      }
      std::vector<float> ms2(all2.size(), 0.f);
      for (size_t i = 0; i < C->steps.size(); ++i)
        if (C->step_group[i] >= 0) ms2[C->step_group[i]] = tf2[i];
      keep.clear();
      for (size_t g = 0; g < all2.size(); ++g) {
        float t_unfused = 0.f;
        for (int b : all2[g].buckets) t_unfused += tu[b];
        if (all2[g].gemm || ms2[g] < t_unfused) keep.push_back(all2[g]);
      }
    }
  }
  set_groups(prog, keep);
  reset_device_state(*plan);
  // the selected configuration, timed as a whole
  std::vector<float> tsel;
  st = profile_steps_min(plan, bits, 0, n_sl, workspace, ws_bytes, (uint32_t)B, stream, tsel, &C);
  if (st != TNQ_OK) return st;
  float tot = 0.f;
  for (float x : tsel) tot += x;
  *total_ms = tot;
  return TNQ_OK;
}
}  // namespace tnq

extern "C" {

tnq_status tnq_plan_autotune(tnq_plan* plan, const uint8_t* bits, void* workspace, size_t ws_bytes,
                             uint32_t max_batch, void* stream, int32_t* out_n_fused) {
  if (!plan || (!bits && plan->net.n_qubits > 0) || !workspace) { set_error("NULL argument"); return TNQ_EINVAL; }
  for (int q = 0; q < plan->net.n_qubits; ++q)
    if (bits[q] > 1) { set_error("bitstring bytes must be 0 or 1"); return TNQ_EINVAL; }
  tnq_status st = check_device();
  if (st != TNQ_OK) return st;
  const uint64_t n_sl = 1ull << plan->mu.size();
  uint64_t cap = 1;
  while (cap < n_sl && cap < (1ull << MAX_ITEM_BITS)) cap <<= 1;
  if (max_batch > 0) cap = std::min<uint64_t>(cap, 1ull << ilog2_floor(max_batch));
  // tuning variants: the GEMM cut-over (split precision only) and the fused
  // chains' tile shape; each is compiled, its chains selected and the result
  // timed. The plan's own tuning is tried first and kept unless another
  // variant is at least 3% faster (so that timing noise does not flip the
  // choice between runs); the fastest such variant wins.
  std::vector<std::pair<int, int>> variants{{plan->gemm_min_k_log2, plan->prog.tile_low}};
  const std::vector<int> cuts = plan->opts.precision == TNQ_PREC_C64 ? std::vector<int>{plan->gemm_min_k_log2}
                                                                      : std::vector<int>{3, 4, 5, 6};
  for (int c : cuts)
    for (int k : {3, 64})
      if (std::make_pair(c, k) != variants[0]) variants.push_back({c, k});
  int best = -1;
  float best_ms = 0.f;
  std::vector<FusedGroup> best_groups;
  for (size_t v = 0; v < variants.size(); ++v) {
    try {
      rebuild_program(plan, variants[v].first, variants[v].second);
    } catch (const std::exception& e) {
      set_error(e.what());
      return TNQ_EINVAL;
    }
    float ms = 0.f;
    if ((st = select_chains(plan, bits, workspace, ws_bytes, cap, stream, &ms)) != TNQ_OK) return st;
    if (best < 0 || ms < (best == 0 ? 0.97f : 1.f) * best_ms) {
      best = (int)v;
      best_ms = ms;
      best_groups = plan->prog.groups;
    }
  }
  rebuild_program(plan, variants[best].first, variants[best].second);
  set_groups(plan->prog, best_groups);
  reset_device_state(*plan);
  if (out_n_fused) *out_n_fused = (int32_t)plan->prog.groups.size();
  return TNQ_OK;
}

tnq_status tnq_plan_fused_chains(const tnq_plan* plan, int32_t* last_bucket, size_t cap, size_t* out_n) {
  if (!plan || !out_n) { set_error("NULL argument"); return TNQ_EINVAL; }
  const auto& groups = plan->prog.groups;
  *out_n = groups.size();
  if (last_bucket)
    for (size_t i = 0; i < groups.size() && i < cap; ++i) last_bucket[i] = groups[i].buckets.back();
  if (last_bucket && cap < groups.size()) { set_error("capacity too small"); return TNQ_EINVAL; }
  return TNQ_OK;
}

tnq_status tnq_plan_keep_chains(tnq_plan* plan, const int32_t* last_bucket, size_t n) {
  if (!plan || (n && !last_bucket)) { set_error("NULL argument"); return TNQ_EINVAL; }
  Program& prog = plan->prog;
  auto listed = [&](const FusedGroup& g) {
    return std::find(last_bucket, last_bucket + n, g.buckets.back()) != last_bucket + n;
  };
  // the listed GEMM chains, then the shared-memory chains the fusion pass
  // proposes around them (as the autotuner's second round does), listed ones kept
  std::vector<FusedGroup> keep;
  for (const auto& g : prog.groups)
    if (g.gemm && listed(g)) keep.push_back(g);
  set_groups(prog, keep);
  if (plan->opts.fuse_min_rank > 0) fuse_chains(prog, plan->order, plan->opts.fuse_min_rank);
  std::vector<FusedGroup> all = prog.groups;
  keep.clear();
  for (const auto& g : all)
    if (listed(g)) keep.push_back(g);
  set_groups(prog, keep);
  reset_device_state(*plan);
  return TNQ_OK;
}

// Internal: kernel launches of one batch of configuration (mode, batch): one
// per remaining bucket or chain step (three per GEMM chain, two in the fused-A
// form), one per level of early buckets, and the leaf, scalar, final and
// slice-sum kernels.
int tnq_internal_launches_per_batch(const tnq_plan* plan, int mode, uint32_t batch) {
  if (!plan) return 0;
  int n = 0;
  const auto& prog = plan->prog;
  std::vector<char> dep(prog.tensors.size());
  for (size_t t = 0; t < dep.size(); ++t) dep[t] = tensor_dep(prog.tensors[t], mode);
  int item_bits = 0;
  while ((1u << item_bits) < batch) ++item_bits;
  const std::vector<int> hoist = hoist_levels(prog, dep, item_bits);
  int levels = 0;
  for (size_t b = 0; b < prog.buckets.size(); ++b) {
    levels = std::max(levels, hoist[b]);
    const int gi = prog.group_of.empty() ? -1 : prog.group_of[b];
    if (gi < 0) n += !hoist[b];
    else if (prog.groups[gi].buckets.back() == (int)b) n += prog.groups[gi].gemm ? 3 : 1;  // GEMM: 2 packs + MMA
  }
  ExecConfig C;  // a GEMM in the fused-A form packs only B
  C.L = make_layout(*plan, mode, (int)batch);
  if (build_steps(*plan, C.L, C))
    for (const GemmBucketArgs& g0 : C.gb) {
      GemmBucketArgs g = g0;
      g.a[0].ptr = reinterpret_cast<const float2*>(reinterpret_cast<size_t>(g.a[0].ptr) + 256);
      n -= gemm_fused_a(g) ? 1 : 0;
    }
  return n + levels + 4;  // + leaf, scalar, final and slice-sum kernels
}

size_t tnq_plan_workspace_bytes(const tnq_plan* plan, uint32_t batch) {
  if (!plan) return 0;
  uint32_t B = 1;
  while (B < batch && B < (1u << MAX_ITEM_BITS)) B <<= 1;
  return std::max(layout_bytes(*plan, 0, (int)B), layout_bytes(*plan, 1, (int)B));
}

tnq_status tnq_contract_sliced(const tnq_plan* plan, const uint8_t* bits, uint64_t slice_begin, uint64_t slice_end,
                               void* workspace, size_t ws_bytes, uint32_t max_batch, void* stream, double* out_amp,
                               double* out_slice_amps) {
  if (!plan || (!bits && plan->net.n_qubits > 0) || !out_amp) { set_error("NULL argument"); return TNQ_EINVAL; }
  const uint64_t n_slices = 1ull << plan->mu.size();
  if (slice_begin > slice_end || slice_end > n_slices) { set_error("slice range outside [0, n_slices)"); return TNQ_EINVAL; }
  for (int q = 0; q < plan->net.n_qubits; ++q)
    if (bits[q] > 1) { set_error("bitstring bytes must be 0 or 1"); return TNQ_EINVAL; }
  out_amp[0] = out_amp[1] = 0.0;
  if (slice_begin == slice_end) return TNQ_OK;
  tnq_status st = check_device();
  if (st != TNQ_OK) return st;
  if (!workspace) { set_error("workspace is NULL"); return TNQ_EINVAL; }
  const uint64_t n_items = slice_end - slice_begin;
  uint64_t cap = 1;
  while (cap < n_items && cap < (1ull << MAX_ITEM_BITS)) cap <<= 1;
  if (max_batch > 0) cap = std::min<uint64_t>(cap, 1ull << ilog2_floor(max_batch));
  const int B = pick_batch(*plan, 0, ws_bytes, cap);
  if (B == 0) { set_error("workspace too small for one slice"); return TNQ_ENOMEM; }
  ExecConfig* C = nullptr;
  if ((st = get_config(*plan, 0, B, &C)) != TNQ_OK) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  char* ws = reinterpret_cast<char*>(workspace);
  std::vector<unsigned> words((size_t)C->L.n_words * C->L.n_rows, 0u);
  pack_bits(bits, plan->net.n_qubits, words);
  CU(cudaMemcpyAsync(ws + C->L.bits_off, words.data(), words.size() * 4, cudaMemcpyHostToDevice, s));
  CU(cudaMemsetAsync(ws + C->L.status_off, 0, 4, s));
  std::vector<double> res(2 * (size_t)B), part(2);
  int dev_status = 0;
  double sre = 0, sim = 0;
  std::lock_guard<std::mutex> lk(plan->dev_mu);  // one capture/launch sequence per plan at a time
  for (uint64_t base = slice_begin; base < slice_end; base += B) {
    BatchHdr h;
    std::memset(&h, 0, sizeof(h));
    h.item_base = base;
    h.item_end = slice_end;
    h.mode = 0;
    h.p = (int)plan->mu.size();
    h.n_words = C->L.n_words;
    if ((st = run_batch(*plan, *C, ws, s, h)) != TNQ_OK) return st;
    CU(cudaMemcpyAsync(part.data(), ws + C->L.part_off, 16, cudaMemcpyDeviceToHost, s));
    CU(cudaMemcpyAsync(&dev_status, ws + C->L.status_off, 4, cudaMemcpyDeviceToHost, s));
    if (out_slice_amps)
      CU(cudaMemcpyAsync(res.data(), ws + C->L.res_off, 16 * (size_t)B, cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    if (dev_status) { set_error("a tensor-core wait timed out on the device"); return TNQ_ETIMEOUT; }
    sre += part[0];
    sim += part[1];
    if (out_slice_amps) {
      const uint64_t nv = std::min<uint64_t>(B, slice_end - base);
      std::memcpy(out_slice_amps + 2 * (base - slice_begin), res.data(), 16 * nv);
    }
  }
  out_amp[0] = sre;
  out_amp[1] = sim;
  return TNQ_OK;
}

tnq_status tnq_amplitudes_batch(const tnq_plan* const* plans, size_t n_plans, const uint8_t* bits,
                                const size_t* bits_offset, void* workspace, size_t ws_bytes, void* stream,
                                double* out_amps) {
  if ((n_plans && (!plans || !bits || !bits_offset || !out_amps))) { set_error("NULL argument"); return TNQ_EINVAL; }
  if (n_plans == 0) return TNQ_OK;
  if (bits_offset[0] != 0) { set_error("bits_offset[0] must be 0"); return TNQ_EINVAL; }
  for (size_t i = 0; i < n_plans; ++i)
    if (!plans[i] || bits_offset[i + 1] < bits_offset[i]) { set_error("bad plan or bits_offset"); return TNQ_EINVAL; }
  {
    size_t pos = 0;
    for (size_t i = 0; i < n_plans; ++i) {
      const size_t nbytes = (bits_offset[i + 1] - bits_offset[i]) * (size_t)plans[i]->net.n_qubits;
      for (size_t k = 0; k < nbytes; ++k)
        if (bits[pos + k] > 1) { set_error("bitstring bytes must be 0 or 1"); return TNQ_EINVAL; }
      pos += nbytes;
    }
  }
  tnq_status st = check_device();
  if (st != TNQ_OK) return st;
  if (!workspace) { set_error("workspace is NULL"); return TNQ_EINVAL; }
  const size_t n_bits = bits_offset[n_plans];
  if (n_bits == 0) return TNQ_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  char* ws = reinterpret_cast<char*>(workspace);

  // Lanes: the plans run on up to N_LANES streams at once, each with its own
  // part of the workspace (a plan always takes the lane of its first
  // occurrence, so a repeated call reuses its captured graphs). Every batch's
  // header and bitstrings go up in one copy at the start; each batch then adds
  // its per-bitstring partial sums to device accumulators, and the call
  // synchronises once, at the end.
  constexpr int N_LANES = 4;
  std::vector<int> lane_of(n_plans, -1);
  int n_distinct = 0;
  for (size_t i = 0; i < n_plans; ++i) {
    if (bits_offset[i + 1] == bits_offset[i]) continue;
    for (size_t j = 0; j < i && lane_of[i] < 0; ++j)
      if (plans[j] == plans[i] && lane_of[j] >= 0) lane_of[i] = lane_of[j];
    if (lane_of[i] < 0) lane_of[i] = n_distinct++;
  }
  const size_t tail_bytes = align_up(n_bits * sizeof(double2), 256) + 256;  // accumulators + lane status words
  struct Job {
    size_t plan;
    uint64_t base, end;
    int B, lane, rows;
    ExecConfig* C;
  };
  std::vector<Job> jobs;
  int n_lanes = 0;
  size_t region = 0;
  // batch size of plan i in a lane of `reg` bytes, and the staging bytes
  // (headers and bitstring words of every batch) that choice needs
  auto batch_of = [&](size_t i, size_t reg) {
    const uint64_t n_items = (uint64_t)(bits_offset[i + 1] - bits_offset[i]) << plans[i]->mu.size();
    uint64_t cap = 1;
    while (cap < n_items && cap < (1ull << MAX_ITEM_BITS)) cap <<= 1;
    return pick_batch(*plans[i], 1, reg, cap);
  };
  auto staging = [&](size_t reg) {
    size_t nh = 0, nw = 0;
    for (size_t i = 0; i < n_plans; ++i) {
      if (lane_of[i] < 0) continue;
      const int B = batch_of(i, reg);
      const uint64_t n_items = (uint64_t)(bits_offset[i + 1] - bits_offset[i]) << plans[i]->mu.size();
      const uint64_t nbat = (n_items + B - 1) / B;
      nh += nbat;
      nw += nbat * (size_t)((plans[i]->net.n_qubits + 31) / 32) * (size_t)(B + 1);
    }
    return align_up(nh * sizeof(BatchHdr), 256) + align_up(nw * 4 + 4, 256);
  };
  for (int K = std::min(N_LANES, n_distinct); K >= 1 && !n_lanes; --K) {
    // the lanes take what the staging area and the accumulators leave; the
    // staging area depends on the batch sizes, which depend on the lane size
    size_t stage = 0;
    for (int iter = 0; iter < 8; ++iter) {
      if (ws_bytes < tail_bytes + stage + 256 * (size_t)K) break;
      region = (ws_bytes - tail_bytes - stage) / K / 256 * 256;
      bool fits = true;
      for (size_t i = 0; i < n_plans && fits; ++i)
        if (lane_of[i] >= 0 && batch_of(i, region) == 0) fits = false;
      if (!fits) break;
      const size_t need = staging(region);
      if ((size_t)K * region + need + tail_bytes <= ws_bytes) {
        n_lanes = K;
        break;
      }
      stage = need;
    }
  }
  if (n_lanes == 0) { set_error("workspace too small for one item of some plan"); return TNQ_ENOMEM; }
  for (size_t i = 0; i < n_plans; ++i) lane_of[i] = lane_of[i] < 0 ? -1 : lane_of[i] % n_lanes;
  // batches of every plan, and their headers and bitstring words
  std::vector<BatchHdr> hdrs;
  std::vector<size_t> word_off;  // per job: first word of its bitstrings in `words`
  std::vector<unsigned> words;
  {
    size_t byte_pos = 0;
    for (size_t pi = 0; pi < n_plans; ++pi) {
      const tnq_plan& P = *plans[pi];
      const int n = P.net.n_qubits;
      const size_t nb = bits_offset[pi + 1] - bits_offset[pi];
      const uint8_t* pb = bits + byte_pos;
      byte_pos += nb * (size_t)n;
      if (nb == 0) continue;
      const int p = (int)P.mu.size();
      const uint64_t n_items = (uint64_t)nb << p;
      uint64_t cap = 1;
      while (cap < n_items && cap < (1ull << MAX_ITEM_BITS)) cap <<= 1;
      const int B = pick_batch(P, 1, region, cap);
      ExecConfig* C = nullptr;
      if ((st = get_config(P, 1, B, &C)) != TNQ_OK) return st;
      for (uint64_t base = 0; base < n_items; base += B) {
        const uint64_t end = std::min<uint64_t>(n_items, base + B);
        const uint64_t b0 = base >> p, b1 = (end - 1) >> p;  // bitstrings touched by this batch
        Job J{pi, base, end, B, lane_of[pi], (int)(b1 - b0 + 1), C};
        word_off.push_back(words.size());
        words.resize(words.size() + (size_t)C->L.n_words * C->L.n_rows, 0u);
        unsigned* w = words.data() + word_off.back();
        for (uint64_t b = b0; b <= b1; ++b)
          for (int q = 0; q < n; ++q)
            if (pb[b * n + q]) w[(size_t)(b - b0) * C->L.n_words + (q >> 5)] |= 1u << (q & 31);
        BatchHdr h;
        std::memset(&h, 0, sizeof(h));
        h.item_base = base;
        h.item_end = n_items;
        h.bstr_base = b0;
        h.mode = 1;
        h.p = p;
        h.n_words = C->L.n_words;
        hdrs.push_back(h);
        jobs.push_back(J);
      }
    }
  }
  // tail of the workspace: staging (headers, then bitstring words), accumulators, lane status words
  const size_t stage_bytes = align_up(hdrs.size() * sizeof(BatchHdr), 256) + align_up(words.size() * 4 + 4, 256);
  const size_t lanes_bytes = (size_t)n_lanes * region;
  if (lanes_bytes + stage_bytes + tail_bytes > ws_bytes) { set_error("workspace too small for the staging area"); return TNQ_ENOMEM; }
  char* stage = ws + lanes_bytes;
  BatchHdr* d_hdrs = reinterpret_cast<BatchHdr*>(stage);
  unsigned* d_words = reinterpret_cast<unsigned*>(stage + align_up(hdrs.size() * sizeof(BatchHdr), 256));
  double2* acc = reinterpret_cast<double2*>(stage + stage_bytes);
  int* lane_status = reinterpret_cast<int*>(stage + stage_bytes + align_up(n_bits * sizeof(double2), 256));
  CU(cudaMemcpyAsync(d_hdrs, hdrs.data(), hdrs.size() * sizeof(BatchHdr), cudaMemcpyHostToDevice, s));
  if (!words.empty()) CU(cudaMemcpyAsync(d_words, words.data(), words.size() * 4, cudaMemcpyHostToDevice, s));
  CU(cudaMemsetAsync(acc, 0, tail_bytes - 0, s));  // accumulators and lane status words
  // lane streams: lane 0 is the caller's stream, the others fork from it and join it at the end
  cudaStream_t ls[N_LANES] = {s};
  cudaEvent_t fork = nullptr, join[N_LANES] = {};
  auto cleanup = [&]() {
    for (int k = 1; k < n_lanes; ++k) {
      if (join[k]) cudaEventDestroy(join[k]);
      if (ls[k]) cudaStreamDestroy(ls[k]);
    }
    if (fork) cudaEventDestroy(fork);
  };
  cudaError_t e = cudaSuccess;
  if (n_lanes > 1) {
    e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(fork, s);
    for (int k = 1; k < n_lanes && e == cudaSuccess; ++k) {
      e = cudaStreamCreateWithFlags(&ls[k], cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&join[k], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(ls[k], fork, 0);
    }
    if (e != cudaSuccess) {
      cleanup();
      set_error(std::string("lane streams: ") + cudaGetErrorString(e));
      return TNQ_ECUDA;
    }
  }
  for (int k = 0; k < n_lanes; ++k) {  // the lane's status word (timeouts of the tensor-core waits)
    e = cudaMemsetAsync(ws + (size_t)k * region + jobs[0].C->L.status_off, 0, 4, ls[k]);
    if (e != cudaSuccess) break;
  }
  for (size_t ji = 0; ji < jobs.size() && e == cudaSuccess; ++ji) {
    const Job& J = jobs[ji];
    const tnq_plan& P = *plans[J.plan];
    char* lws = ws + (size_t)J.lane * region;
    cudaStream_t q = ls[J.lane];
    ExecConfig& C = *J.C;
    std::lock_guard<std::mutex> lk(P.dev_mu);  // one capture/launch sequence per plan at a time
    e = cudaMemcpyAsync(lws + C.L.bits_off, d_words + word_off[ji], (size_t)C.L.n_words * C.L.n_rows * 4,
                        cudaMemcpyDeviceToDevice, q);
    if (e != cudaSuccess) break;
    if ((st = run_batch(P, C, lws, q, hdrs[ji], d_hdrs + ji)) != TNQ_OK) {
      cleanup();
      return st;
    }
    k_accumulate<<<(J.rows + 127) / 128, 128, 0, q>>>(reinterpret_cast<const double2*>(lws + C.L.part_off), J.rows,
                                                      acc + bits_offset[J.plan] + (J.base >> hdrs[ji].p));
    e = cudaGetLastError();
  }
  for (int k = 0; k < n_lanes && e == cudaSuccess; ++k) {
    e = cudaMemcpyAsync(lane_status + k, ws + (size_t)k * region + jobs[0].C->L.status_off, 4,
                        cudaMemcpyDeviceToDevice, ls[k]);
    if (e == cudaSuccess && k > 0) e = cudaEventRecord(join[k], ls[k]);
    if (e == cudaSuccess && k > 0) e = cudaStreamWaitEvent(s, join[k], 0);
  }
  std::vector<double> out(2 * n_bits);
  std::vector<int> lstat(n_lanes, 0);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out.data(), acc, n_bits * sizeof(double2), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(lstat.data(), lane_status, n_lanes * 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cleanup();
  if (e != cudaSuccess) {
    set_error(std::string("batched amplitudes: ") + cudaGetErrorString(e));
    return TNQ_ECUDA;
  }
  for (int k = 0; k < n_lanes; ++k)
    if (lstat[k]) { set_error("a tensor-core wait timed out on the device"); return TNQ_ETIMEOUT; }
  std::memcpy(out_amps, out.data(), 16 * n_bits);
  return TNQ_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free variant of tnq_contract_sliced.
//
// Some callers cannot call cudaMalloc: a host whose own pool allocator has
// already reserved the device memory it is allowed to use, or a latency-bound
// loop in which cudaMalloc's implicit device synchronisation would stall
// other streams. For them this
// entry point takes its scratch (plan tables and intermediate tensors) from one
// fixed-size array in device global memory that the library declares at file
// scope; every GPU that loads the library holds that array until the process
// exits. It allocates no device memory and calls no allocating routine.
namespace tnq {

constexpr size_t NOALLOC_SCRATCH_BYTES = 64ull << 20;  // 64 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

// Device address of g_noalloc_scratch, looked up once per device with that
// device current (the host-side symbol is only a stand-in, not an address).
static std::mutex g_noalloc_mu;
static void* g_noalloc_addr[256] = {};

static tnq_status noalloc_scratch_address(void** out) {
  int dev = 0;
  CU(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 256) {
    set_error("device ordinal out of range");
    return TNQ_EINVAL;
  }
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      set_error(std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
      return TNQ_ECUDA;
    }
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return TNQ_OK;
}

// Bytes of plan tables (leaf, scalar, wire, final and early-bucket records)
// at the front of the scratch for batch B.
static size_t noalloc_table_bytes(const tnq_plan& P, int B) {
  ExecConfig C;
  C.L = make_layout(P, 0, B);
  const size_t hoist = build_steps(P, C.L, C) ? C.hoist_dev.size() : 0;
  size_t vals = 0;
  for (const GateTensor& g : P.net.tensors)
    if (g.nv > 2) vals += (size_t)1 << g.nv;
  return align_up(P.prog.leaves.size() * sizeof(LeafDev), 256) +
         align_up(P.prog.scalar_leaves.size() * sizeof(LeafDev), 256) +
         align_up(P.net.inout_qubits.size() * sizeof(int), 256) + align_up(P.prog.finals.size() * sizeof(FinalDev), 256) +
         align_up(hoist * sizeof(HoistDev), 256) + align_up(vals * sizeof(float2), 256);
}

// Host-side configuration of the allocation-free path for batch B, built once
// per (plan, B) on the plan's device and cached with its other configurations:
// the same steps, launch shapes and early-bucket levels as the workspace path,
// with the plan tables at the front of the static scratch and the workspace
// after them. Nothing in it owns device memory. Caller holds no lock.
static tnq_status get_noalloc_config(const tnq_plan& P, uint64_t cap, char* scratch, NoallocConfig** out) {
  int dev;
  CU(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(P.dev_mu);
  if (P.dev && P.dev->device != dev) {
    set_error("plan already bound to another CUDA device");
    return TNQ_EINVAL;
  }
  if (!P.dev) {
    P.dev = new DeviceState();
    P.dev->device = dev;
  }
  const Program& prog = P.prog;
  // largest power-of-two batch (<= cap) whose tables and workspace fit
  int B = 0;
  auto cb = P.dev->noalloc_batch.find(cap);
  if (cb != P.dev->noalloc_batch.end()) {
    B = cb->second;
  } else {
    for (uint64_t b = 1; b <= cap; b <<= 1) {
      if (noalloc_table_bytes(P, (int)b) + make_layout(P, 0, (int)b).total > NOALLOC_SCRATCH_BYTES) break;
      B = (int)b;
    }
    if (B > 0) P.dev->noalloc_batch[cap] = B;
  }
  if (B == 0) {
    set_error("plan needs " + std::to_string(noalloc_table_bytes(P, 1) + make_layout(P, 0, 1).total) +
              " bytes of scratch for one slice; the static scratch of tnq_contract_sliced_noalloc holds " +
              std::to_string(NOALLOC_SCRATCH_BYTES) + " bytes");
    return TNQ_ENOMEM;
  }
  auto it = P.dev->noalloc.find(B);
  if (it != P.dev->noalloc.end()) {
    *out = it->second;
    return TNQ_OK;
  }
  CU(allow_group_smem());
  int ggrid = 0;
  tnq_status st = group_grid_size(&ggrid);
  if (st != TNQ_OK) return st;
  std::unique_ptr<NoallocConfig> NC(new NoallocConfig());
  ExecConfig& C = NC->C;
  C.group_grid = ggrid;
  C.L = make_layout(P, 0, B);
  for (int t : prog.leaves)
    NC->leaves.push_back(make_leafdev(P, &prog.tensors[t], prog.tensors[t].leaf_gate, &C.L, t, &C.vals));
  for (int g : prog.scalar_leaves) NC->scalars.push_back(make_leafdev(P, nullptr, g, nullptr, -1, &C.vals));
  for (int t : prog.finals) NC->finals.push_back(FinalDev{C.L.off[t], t, (int)C.L.dep[t]});
  if (!build_steps(P, C.L, C)) return TNQ_EUNSUPPORTED;
  for (size_t i = 0; i < C.gsmem.size(); ++i) {  // per-chain persistent grids, as build_config sizes them
    int g = 0;
    if ((st = group_grid_size(&g, C.gsmem[i], C.gp[i].tail > 0 ? 1 : (C.gp[i].lean2 ? 2 : 0))) != TNQ_OK) return st;
    C.ggrid.push_back(g);
  }
  size_t o = 0;
  auto take = [&](size_t bytes) {
    char* p = scratch + o;
    o = align_up(o + bytes, 256);
    return p;
  };
  C.d_leaves = reinterpret_cast<LeafDev*>(take(NC->leaves.size() * sizeof(LeafDev)));
  C.d_scalars = reinterpret_cast<LeafDev*>(take(NC->scalars.size() * sizeof(LeafDev)));
  C.d_inout = reinterpret_cast<int*>(take(P.net.inout_qubits.size() * sizeof(int)));
  C.d_finals = reinterpret_cast<FinalDev*>(take(NC->finals.size() * sizeof(FinalDev)));
  C.d_hoist = reinterpret_cast<HoistDev*>(take(C.hoist_dev.size() * sizeof(HoistDev)));
  C.d_vals = reinterpret_cast<float2*>(take(C.vals.size() * sizeof(float2)));
  NC->tables = o;
  C.n_leaves = (int)NC->leaves.size();
  C.n_scalars = (int)NC->scalars.size();
  C.n_inout = (int)P.net.inout_qubits.size();
  C.n_finals = (int)NC->finals.size();
  *out = NC.get();
  P.dev->noalloc[B] = NC.release();
  return TNQ_OK;
}

}  // namespace tnq

extern "C" {

tnq_status tnq_contract_sliced_noalloc(const tnq_plan* plan, const uint8_t* bits, uint64_t slice_begin,
                                       uint64_t slice_end, void* stream, double* out_amp, double* out_slice_amps) {
  if (!plan || (!bits && plan->net.n_qubits > 0) || !out_amp) { set_error("NULL argument"); return TNQ_EINVAL; }
  const uint64_t n_slices = 1ull << plan->mu.size();
  if (slice_begin > slice_end || slice_end > n_slices) { set_error("slice range outside [0, n_slices)"); return TNQ_EINVAL; }
  for (int q = 0; q < plan->net.n_qubits; ++q)
    if (bits[q] > 1) { set_error("bitstring bytes must be 0 or 1"); return TNQ_EINVAL; }
  out_amp[0] = out_amp[1] = 0.0;
  if (slice_begin == slice_end) return TNQ_OK;
  tnq_status st = check_device();
  if (st != TNQ_OK) return st;
  void* scratch = nullptr;
  if ((st = noalloc_scratch_address(&scratch)) != TNQ_OK) return st;
  const uint64_t n_items = slice_end - slice_begin;
  uint64_t cap = 1;
  while (cap < n_items && cap < (1ull << MAX_ITEM_BITS)) cap <<= 1;
  NoallocConfig* NC = nullptr;
  if ((st = get_noalloc_config(*plan, cap, reinterpret_cast<char*>(scratch), &NC)) != TNQ_OK) return st;
  ExecConfig& C = NC->C;
  const int B = C.L.B;
  char* ws = reinterpret_cast<char*>(scratch) + NC->tables;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  // every call shares the scratch: the plan tables go up again each time
  auto put = [&](void* dst, const void* src, size_t bytes) -> cudaError_t {
    return bytes ? cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s) : cudaSuccess;
  };
  CU(put(C.d_leaves, NC->leaves.data(), NC->leaves.size() * sizeof(LeafDev)));
  CU(put(C.d_scalars, NC->scalars.data(), NC->scalars.size() * sizeof(LeafDev)));
  CU(put(C.d_inout, plan->net.inout_qubits.data(), (size_t)C.n_inout * sizeof(int)));
  CU(put(C.d_finals, NC->finals.data(), NC->finals.size() * sizeof(FinalDev)));
  CU(put(C.d_hoist, C.hoist_dev.data(), C.hoist_dev.size() * sizeof(HoistDev)));
  CU(put(C.d_vals, C.vals.data(), C.vals.size() * sizeof(float2)));
  std::vector<unsigned> words((size_t)C.L.n_words * C.L.n_rows, 0u);
  pack_bits(bits, plan->net.n_qubits, words);
  CU(cudaMemcpyAsync(ws + C.L.bits_off, words.data(), words.size() * 4, cudaMemcpyHostToDevice, s));
  CU(cudaMemsetAsync(ws + C.L.status_off, 0, 4, s));
  std::vector<double> res(2 * (size_t)B), part(2);
  int dev_status = 0;
  double sre = 0, sim = 0;
  std::lock_guard<std::mutex> lk(plan->dev_mu);  // one launch sequence per plan at a time
  for (uint64_t b0 = slice_begin; b0 < slice_end; b0 += B) {
    BatchHdr h;
    std::memset(&h, 0, sizeof(h));
    h.item_base = b0;
    h.item_end = slice_end;
    h.p = (int)plan->mu.size();
    h.n_words = C.L.n_words;
    CU(cudaMemcpyAsync(ws + C.L.hdr_off, &h, sizeof(h), cudaMemcpyHostToDevice, s));
    enqueue_batch(*plan, C, ws, s);  // clears the atomicMax targets first
    CU(cudaGetLastError());
    CU(cudaMemcpyAsync(part.data(), ws + C.L.part_off, 16, cudaMemcpyDeviceToHost, s));
    CU(cudaMemcpyAsync(&dev_status, ws + C.L.status_off, 4, cudaMemcpyDeviceToHost, s));
    if (out_slice_amps) CU(cudaMemcpyAsync(res.data(), ws + C.L.res_off, 16 * (size_t)B, cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    if (dev_status) { set_error("a tensor-core wait timed out on the device"); return TNQ_ETIMEOUT; }
    sre += part[0];
    sim += part[1];
    if (out_slice_amps) {
      const uint64_t nv = std::min<uint64_t>(B, slice_end - b0);
      std::memcpy(out_slice_amps + 2 * (b0 - slice_begin), res.data(), 16 * nv);
    }
  }
  out_amp[0] = sre;
  out_amp[1] = sim;
  return TNQ_OK;
}

}  // extern "C"
