// gemm_tc.cuh -- split-precision batched GEMM on the 5th-generation tensor
// cores (tcgen05, sm_103a) used for merged buckets whose product is a
// contraction Sum_K A[S,X,K] B[S,Y,K] (several consecutive eliminations of
// variables shared by two large tensors).
//
// C[b] (rows x cols, FP32) = sum over the passes hi*hi + hi*lo + lo*hi of
// A_p[b] (rows x Kr) . B_p[b]^T (cols x Kr), where x = hi + lo splits an FP32
// value into two BF16 (or TF32) parts; FP32 accumulation in tensor memory.
//
// Operands live in global memory already in the tensor core's shared-memory
// layout ("tile-major"): a tile is 128 rows x 128 bytes of K, stored as 16
// row groups of 8 core matrices (8 rows x 16 bytes each, 128 bytes apart
// along K, 1024 bytes apart along rows), so one tile is one contiguous 16 KB
// bulk-async copy. Tile (b, rt, kt) of an operand with RT row tiles and KT
// K tiles starts at ((b * RT + rt) * KT + kt) * 16384 bytes.
#pragma once
#include <cstdint>

namespace tnq {

enum GemmKind { GEMM_BF16 = 0, GEMM_TF32 = 1 };

constexpr int GT_ROWS = 128;           // rows of an operand tile (M of one MMA)
constexpr int GT_KBYTES = 128;         // bytes of K per tile row
constexpr int GT_TILE_BYTES = GT_ROWS * GT_KBYTES;  // 16 KB

// Byte offset of element (r, k) inside its tile; esize = 2 (BF16) or 4 (TF32).
__host__ __device__ inline uint32_t gt_offset(int r, int k, int esize) {
  const int kb = (k * esize) & (GT_KBYTES - 1);
  return (uint32_t)((r >> 3) * 1024 + (kb >> 4) * 128 + (r & 7) * 16 + (kb & 15));
}

// The same layout for half tiles of 64 bytes of K per row (8 KB; the fused-A
// GEMM's operand tiles): 8-row groups 512 bytes apart.
constexpr int GT_KBYTES_H = 64;
constexpr int GT_TILE_BYTES_H = GT_ROWS * GT_KBYTES_H;  // 8 KB
__host__ __device__ inline uint32_t gt_offset_h(int r, int k, int esize) {
  const int kb = (k * esize) & (GT_KBYTES_H - 1);
  return (uint32_t)((r >> 3) * 512 + (kb >> 4) * 128 + (r & 7) * 16 + (kb & 15));
}

// ---- merged bucket as a complex GEMM --------------------------------------
// out[item, S, X, Y] = Sum_K A'[item, S, X, K] B'[item, S, Y, K], where A' (B')
// is the product of the large operand and the small tensors folded into its
// side, each scaled by its power-of-two factor. Complex through the real
// embedding: A_real = [Re A' | Im A'] (rows X), B rows interleaved
// [Re B' | -Im B'], [Im B' | Re B'], so C columns (2n, 2n+1) = (Re, Im) of out.
constexpr int GB_BITS = 16;   // most variables in one of S (with item bits), X, Y, K
constexpr int GB_SIDE = 17;   // large operand + up to 16 small tensors per side

struct GemmOperand {
  const float2* ptr;
  long long istride;           // per item (0 when item-invariant)
  long long sstride[GB_BITS];  // per batch variable
  long long rstride[GB_BITS];  // per row (X) or column (Y) variable
  long long kstride[GB_BITS];  // per summed variable
  int meta;                    // meta row (-1: leaf, unit scale)
  int dep;
};

struct GemmBucketArgs {
  GemmOperand a[GB_SIDE], b[GB_SIDE];
  int na, nb;
  int ns, nx, ny, nk;          // variable counts
  int items;                   // items of the output (1 when item-invariant)
  int m_pad, n_pad, k_pad;     // padded complex sizes (rows, columns, K)
  int kind;
  void *a_hi, *a_lo, *b_hi, *b_lo;
  int out_meta, out_dep, B;
  int* meta_e;
  unsigned* meta_m;
};

// Epilogue data of a bucket GEMM (in GemmArgs when out_c is null).
struct GemmEpilogue {
  float2* out;
  long long istride;
  long long s[GB_BITS], x[GB_BITS], y[GB_BITS];
  int ns, nx, ny;
  int meta, dep, B;
  unsigned* meta_m;
};

// Device-side status word: 0 ok, 1 a bulk-copy wait gave up, 2 an MMA wait gave up.
struct GemmArgs {
  const void* a_hi;
  const void* a_lo;
  const void* b_hi;
  const void* b_lo;
  int row_tiles_a;   // rows of A / 128
  int row_tiles_b;   // rows of B / 128 (columns of C / 128)
  int k_tiles;       // Kr bytes / 128
  int batch;
  // batch index of an operand's tiles: b & mask (all ones; or 2^ns - 1 when
  // the operand does not depend on the item, packed once for all items)
  long long a_bmask, b_bmask;
  int* status;
  // epilogue: C written as FP32 rows x cols per batch (ldc floats per row) when
  // `out_c` is set; the bucket path supplies its own epilogue data instead
  float* out_c;
  long long ldc;
  GemmEpilogue ep;  // used when out_c is null
  // Fused A (k_gemm_tc_fa, BF16): A is read directly from the complex64
  // tensor described by fa (one operand, no folded tensors; its three lowest
  // summed variables are its lowest bits), scaled, split into hi/lo and
  // written to the shared-memory tiles by producer warps. B then comes packed
  // in half tiles (64 bytes of K per row) and k_tiles counts 32-value complex
  // K steps.
  GemmOperand fa;
  int fa_ns, fa_nx, fa_nk, fa_kpad, fa_B;
  const unsigned* fa_meta_m;
};

// Launches C = sum_passes A_p B_p^T for every batch (grid = col tiles x row tiles x batch).
void gemm_tc_launch(int kind, const GemmArgs& args, void* stream);

// True when gemm_bucket_launch runs the fused-A form for g.
bool gemm_fused_a(const GemmBucketArgs& g);

// Packs both operands (in the fused-A form only B), writes the output
// exponents and runs the GEMM with the bucket epilogue on `stream`.
void gemm_bucket_launch(const GemmBucketArgs& g, const GemmEpilogue& ep, int* status, void* stream);

}  // namespace tnq
