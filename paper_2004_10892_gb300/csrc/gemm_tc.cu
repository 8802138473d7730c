// gemm_tc.cu -- tcgen05 split-precision batched GEMM (see gemm_tc.cuh).
//
// A persistent, warp-specialised kernel: per block one thread streams the
// A/B hi/lo tiles of every K step into a 3-stage shared-memory ring with
// bulk-async copies (mbarrier transaction counts), one thread issues the
// three split-precision MMA passes (hi*hi, hi*lo, lo*hi; lo*lo is below FP32
// rounding and dropped) into one of two tensor-memory accumulators, and four
// warps read the other accumulator with tcgen05.ld and write the previous
// tile. Every wait is bounded by %globaltimer: on a timeout the kernel
// records a status, waits (bounded) for the copies and MMAs it issued, frees
// its tensor memory and returns. A second form (k_gemm_tc_fa) reads the A
// operand straight from its complex64 tensor: producer warps split it into
// hi/lo in shared memory, so A needs no packed copy.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "gemm_tc.cuh"

namespace tnq {

void set_error(const std::string& msg);

namespace {

constexpr unsigned long long WAIT_NS = 2000000000ull;  // 2 s per wait

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// Waits for the phase with the given parity to complete; false after limit_ns.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, unsigned long long limit_ns = WAIT_NS) {
  const unsigned long long t0 = gtimer();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (done) return true;
    if (gtimer() - t0 > limit_ns) return false;
  }
}

// Waits on an mbarrier that nothing ever arrives on, with the same bounded
// wait the GEMM uses; records 1 in *status when the wait gives up.
__global__ void k_wait_never(int* status, unsigned long long limit_ns) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0 && !mbar_wait(&bar, 0, limit_ns)) atomicExch(status, 1);
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: no swizzle, K-major core matrices of
// 8 rows x 16 bytes, 128 bytes apart along K (leading) and `sbo` bytes apart
// along rows (stride: 1024 for tiles with 128 bytes of K per row, 512 for 64);
// descriptor version 1.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t sbo = 1024u) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((128u >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor: FP32 accumulator, A/B format fmt (1 = BF16 for
// kind::f16, 2 = TF32 for kind::tf32), both K-major, N = 128, M = 128.
__host__ __device__ constexpr uint32_t idesc(uint32_t fmt) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((128u >> 3) << 17) | ((128u >> 4) << 24);
}

template <int KIND>
__device__ __forceinline__ void mma(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t acc) {
  if (KIND == GEMM_BF16) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            tmem_d),
        "l"(a), "l"(b), "r"(idesc(1)), "r"(acc)
        : "memory");
  } else {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            tmem_d),
        "l"(a), "l"(b), "r"(idesc(2)), "r"(acc)
        : "memory");
  }
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// 32 consecutive accumulator columns of this thread's lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%"
      "19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

constexpr int STAGE_BYTES = 4 * GT_TILE_BYTES;  // A hi, A lo, B hi, B lo
constexpr int N_STAGES = 3;                      // shared-memory ring of K steps
constexpr int SMEM_BYTES = N_STAGES * STAGE_BYTES + 1024;
constexpr int GEMM_THREADS = 192;  // warp 0: copies, warp 1: MMAs, warps 2-5: epilogue
constexpr uint32_t TMEM_COLS = 256;  // two 128-column FP32 accumulators

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void epi_sync() {  // the four epilogue warps
  asm volatile("bar.sync 1, 128;" ::: "memory");
}

// Power-of-two scale bringing a tensor with largest |re|,|im| bits `mbits`
// into [0.5, 1) (same rule as the bucket kernels).
__device__ __forceinline__ float pack_scale(unsigned mbits, int* mexp) {
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

// 16 bytes of hi and lo parts of CH consecutive values (CH = 8 BF16 or 4 TF32).
template <int KIND, int CH>
__device__ __forceinline__ void split16(const float* x, uint4* hi, uint4* lo) {
  uint32_t h[4], l[4];
  if (KIND == GEMM_BF16) {
    // two values per conversion (round to nearest even); a BF16 value is
    // the upper half of its FP32 bits, so the residuals need no conversion back
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const __nv_bfloat162 hp = __floats2bfloat162_rn(x[2 * q], x[2 * q + 1]);
      const uint32_t hb = *reinterpret_cast<const uint32_t*>(&hp);
      const __nv_bfloat162 lp =
          __floats2bfloat162_rn(x[2 * q] - __uint_as_float(hb << 16), x[2 * q + 1] - __uint_as_float(hb & 0xffff0000u));
      h[q] = hb;
      l[q] = *reinterpret_cast<const uint32_t*>(&lp);
    }
  } else {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h[q]) : "f"(x[q]));
      const float rest = x[q] - __uint_as_float(h[q]);
      asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(l[q]) : "f"(rest));
    }
  }
  *hi = make_uint4(h[0], h[1], h[2], h[3]);
  *lo = make_uint4(l[0], l[1], l[2], l[3]);
}

// Epilogue warps (four, one per TMEM lane quarter): for every tile of the
// block, wait for its accumulator buffer, read it with tcgen05.ld and write
// the tile (plain FP32 rows, or complex pairs scattered into the bucket's
// output with the tile's maximum), then release the buffer.
__device__ __forceinline__ void epilogue_warps(const GemmArgs& a, uint32_t tmem_base, uint64_t* tfull_bar,
                                               uint64_t* tempty_bar, volatile int* s_fail, long long (*s_yoff)[64],
                                               int* s_epi_stop, int e, int quarter, int lane, long long n_tiles) {
  const int r_in = quarter * 32 + lane;
  long long i = 0;
  for (long long tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++i) {
    const int buf = (int)(i & 1);
    const long long j = i >> 1;
    const int ct = (int)(tile % a.row_tiles_b);
    const int rt = (int)((tile / a.row_tiles_b) % a.row_tiles_a);
    const long long b = tile / ((long long)a.row_tiles_b * a.row_tiles_a);
    const GemmEpilogue& ep = a.ep;
    if (!a.out_c && e < 64) {  // column offsets of this tile (complex column n = ct * 64 + e)
      const int n = ct * 64 + e;
      long long off = -1;
      if (n < (1 << ep.ny)) {
        off = 0;
        for (int q = 0; q < ep.ny; ++q)
          if ((n >> q) & 1) off += ep.y[q];
      }
      s_yoff[buf][e] = off;
    }
    // the four warps take the same decision: a failed wait is published in
    // this tile parity's flag before the barrier and read after it
    if (!mbar_wait(&tfull_bar[buf], (uint32_t)(j & 1)) || *s_fail) s_epi_stop[buf] = 1;
    epi_sync();
    if (s_epi_stop[buf]) {
      *s_fail = 1;
      atomicExch(a.status, 2);
      break;
    }
    tc_fence_after();
    const uint32_t taddr = tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)buf * 128u;
    if (a.out_c) {
      float* crow = a.out_c + ((long long)b * a.row_tiles_a * GT_ROWS + rt * GT_ROWS + r_in) * a.ldc +
                    (long long)ct * 128;
#pragma unroll 1
      for (int chunk = 0; chunk < 4; ++chunk) {
        float v[32];
        tmem_ld32(taddr + (uint32_t)(chunk * 32), v);
#pragma unroll
        for (int q = 0; q < 32; q += 4)
          *reinterpret_cast<float4*>(crow + chunk * 32 + q) = make_float4(v[q], v[q + 1], v[q + 2], v[q + 3]);
      }
    } else {
      // row = X assignment m, column pair (2n, 2n+1) = (Re, Im) of Y assignment n
      const int m = rt * GT_ROWS + r_in;
      const long long item = b >> ep.ns, sidx = b & ((1ll << ep.ns) - 1);
      const bool row_ok = m < (1 << ep.nx);
      long long rbase = ep.dep ? item * ep.istride : 0ll;
      for (int q = 0; q < ep.ns; ++q)
        if ((sidx >> q) & 1) rbase += ep.s[q];
      for (int q = 0; q < ep.nx; ++q)
        if ((m >> q) & 1) rbase += ep.x[q];
      float tmax = 0.f;
#pragma unroll 1
      for (int chunk = 0; chunk < 4; ++chunk) {
        float v[32];
        tmem_ld32(taddr + (uint32_t)(chunk * 32), v);  // warp-collective: every lane loads
        if (row_ok) {
#pragma unroll
          for (int q = 0; q < 32; q += 2) {
            const long long yo = s_yoff[buf][chunk * 16 + (q >> 1)];
            if (yo >= 0) {
              ep.out[rbase + yo] = make_float2(v[q], v[q + 1]);
              tmax = fmaxf(tmax, fmaxf(fabsf(v[q]), fabsf(v[q + 1])));
            }
          }
        }
      }
      for (int off = 16; off > 0; off >>= 1) tmax = fmaxf(tmax, __shfl_xor_sync(0xffffffffu, tmax, off));
      if (lane == 0 && tmax > 0.f) {
        unsigned* p = &ep.meta_m[(long long)ep.meta * ep.B + (ep.dep ? item : 0ll)];
        const unsigned bits = __float_as_uint(tmax);
        if (bits > *reinterpret_cast<volatile unsigned*>(p)) atomicMax(p, bits);
      }
    }
    tc_fence_before();
    __syncwarp();
    if (lane == 0) mbar_arrive(&tempty_bar[buf]);
  }
}

// Persistent, warp-specialised GEMM. Each block loops over output tiles
// tile = blockIdx.x + i * gridDim.x (tile -> batch b, row tile rt, column
// tile ct, ct fastest). Warp 0 (one thread) streams the four 16 KB operand
// tiles of every K step into a ring of N_STAGES shared-memory stages (bulk
// async copies completing on full[s]); warp 1 (one thread) waits for a stage,
// issues the 12 MMAs of the three split-precision passes into accumulator
// buffer i & 1 and commits them to empty[s] (stage free) and, after the last
// K step, to tfull[buf]; warps 2-5 read the accumulator lanes of their TMEM
// quarter, write the tile and arrive on tempty[buf]. The accumulators are
// double-buffered, so tile i's epilogue overlaps tile i+1's copies and MMAs.
// Every wait is bounded; on a timeout the block records a status, stops
// issuing, waits (bounded) for what it issued and frees its tensor memory.
template <int KIND>
__global__ void __launch_bounds__(GEMM_THREADS, 1) k_gemm_tc(const GemmArgs a) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint64_t full_bar[N_STAGES], empty_bar[N_STAGES], tfull_bar[2], tempty_bar[2], drain_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int s_fail;
  __shared__ long long s_yoff[2][64];
  __shared__ int s_epi_stop[2];  // per tile parity: an epilogue thread's wait failed (set once, never cleared)
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
  const long long n_tiles = (long long)a.batch * a.row_tiles_a * a.row_tiles_b;
  if (tid == 0) {
    for (int s = 0; s < N_STAGES; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull_bar[b], 1);
      mbar_init(&tempty_bar[b], 4);
    }
    mbar_init(&drain_bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    s_fail = 0;
    s_epi_stop[0] = s_epi_stop[1] = 0;
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = tmem_slot;
  const size_t tb = GT_TILE_BYTES;

  if (warp == 0 && lane == 0) {
    // ---- producer: bulk copies of every K step of every tile of this block
    int fills[N_STAGES] = {};
    long long g = 0;
    bool ok = true;
    for (long long tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
      const int ct = (int)(tile % a.row_tiles_b);
      const int rt = (int)((tile / a.row_tiles_b) % a.row_tiles_a);
      const long long b = tile / ((long long)a.row_tiles_b * a.row_tiles_a);
      const long long ba = b & a.a_bmask, bb = b & a.b_bmask;
      const char* A_hi = (const char*)a.a_hi + (size_t)(ba * a.row_tiles_a + rt) * a.k_tiles * tb;
      const char* A_lo = (const char*)a.a_lo + (size_t)(ba * a.row_tiles_a + rt) * a.k_tiles * tb;
      const char* B_hi = (const char*)a.b_hi + (size_t)(bb * a.row_tiles_b + ct) * a.k_tiles * tb;
      const char* B_lo = (const char*)a.b_lo + (size_t)(bb * a.row_tiles_b + ct) * a.k_tiles * tb;
      for (int kt = 0; kt < a.k_tiles; ++kt, ++g) {
        const int s = (int)(g % N_STAGES);
        if (fills[s] > 0 && !mbar_wait(&empty_bar[s], (fills[s] - 1) & 1)) {  // the MMAs released stage s
          ok = false;
          break;
        }
        if (s_fail) {
          ok = false;
          break;
        }
        const uint32_t st = base + (uint32_t)s * STAGE_BYTES;
        mbar_expect_tx(&full_bar[s], STAGE_BYTES);
        bulk_g2s(st + 0 * GT_TILE_BYTES, A_hi + kt * tb, GT_TILE_BYTES, &full_bar[s]);
        bulk_g2s(st + 1 * GT_TILE_BYTES, A_lo + kt * tb, GT_TILE_BYTES, &full_bar[s]);
        bulk_g2s(st + 2 * GT_TILE_BYTES, B_hi + kt * tb, GT_TILE_BYTES, &full_bar[s]);
        bulk_g2s(st + 3 * GT_TILE_BYTES, B_lo + kt * tb, GT_TILE_BYTES, &full_bar[s]);
        ++fills[s];
      }
    }
    if (!ok) {
      s_fail = 1;
      atomicExch(a.status, 1);
    }
    // every issued copy has landed before the block can exit
    for (int s = 0; s < N_STAGES; ++s)
      if (fills[s] > 0) mbar_wait(&full_bar[s], (fills[s] - 1) & 1);
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer
    long long g = 0;
    bool ok = true, issued = false;
    long long i = 0;
    for (long long tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x, ++i) {
      const int buf = (int)(i & 1);
      const long long j = i >> 1;
      if (j >= 1 && !mbar_wait(&tempty_bar[buf], (uint32_t)((j - 1) & 1))) {  // epilogue done with buffer buf
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t tmem_d = tmem_base + (uint32_t)buf * 128u;
      for (int kt = 0; kt < a.k_tiles; ++kt, ++g) {
        const int s = (int)(g % N_STAGES);
        const long long n = g / N_STAGES;
        if (!mbar_wait(&full_bar[s], (uint32_t)(n & 1)) || s_fail) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t st = base + (uint32_t)s * STAGE_BYTES;
#pragma unroll
        for (int q = 0; q < 4; ++q) {  // 4 MMAs of 32 bytes of K per 128-byte tile row
          const uint32_t off = (uint32_t)q * 256u;
          mma<KIND>(tmem_d, sdesc(st + off), sdesc(st + 2 * GT_TILE_BYTES + off), (kt > 0 || q > 0) ? 1u : 0u);
          mma<KIND>(tmem_d, sdesc(st + off), sdesc(st + 3 * GT_TILE_BYTES + off), 1u);
          mma<KIND>(tmem_d, sdesc(st + GT_TILE_BYTES + off), sdesc(st + 2 * GT_TILE_BYTES + off), 1u);
        }
        mma_commit(&empty_bar[s]);
        issued = true;
      }
      if (ok) mma_commit(&tfull_bar[buf]);
    }
    if (!ok) {
      s_fail = 1;
      atomicExch(a.status, 2);
    }
    if (issued) {  // every issued MMA has completed before the block frees tensor memory
      mma_commit(&drain_bar);
      mbar_wait(&drain_bar, 0);
    }
  } else if (warp >= 2) {
    epilogue_warps(a, tmem_base, tfull_bar, tempty_bar, &s_fail, s_yoff, s_epi_stop, tid - 64, warp & 3, lane, n_tiles);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS) : "memory");
  }
}

// Fused-A form (BF16): A is read from its complex64 tensor by the kernel
// itself. Per block: warps 0-7 (256 producer threads) write, for every K step
// of 32 complex values, the hi and lo half tiles of A's real parts and of its
// imaginary parts (one read of the complex values gives both); warp 8 (one
// thread) copies B's four packed half tiles of the step (real-part and
// imaginary-part positions of K, hi and lo); warp 9 (one thread) issues the
// 12 MMAs of the step (per part: 2 K sub-steps x 3 split-precision passes);
// warps 10-13 are the epilogue. Stage layout: A re hi, re lo, im hi, im lo,
// B re hi, re lo, im hi, im lo (8 KB each). Waits bounded as in k_gemm_tc.
constexpr int GEMM_THREADS_FA = 448;
constexpr int FA_PRODUCERS = 256;

__global__ void __launch_bounds__(GEMM_THREADS_FA, 1) k_gemm_tc_fa(const GemmArgs a) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint64_t full_bar[N_STAGES], empty_bar[N_STAGES], tfull_bar[2], tempty_bar[2], drain_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int s_fail;
  __shared__ long long s_yoff[2][64];
  __shared__ int s_epi_stop[2];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
  const long long n_tiles = (long long)a.batch * a.row_tiles_a * a.row_tiles_b;
  constexpr int HB = GT_TILE_BYTES_H;
  if (tid == 0) {
    for (int s = 0; s < N_STAGES; ++s) {
      mbar_init(&full_bar[s], 1 + FA_PRODUCERS);  // the B copy thread and every producer thread
      mbar_init(&empty_bar[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull_bar[b], 1);
      mbar_init(&tempty_bar[b], 4);
    }
    mbar_init(&drain_bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    s_fail = 0;
    s_epi_stop[0] = s_epi_stop[1] = 0;
  }
  if (warp == 9) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = tmem_slot;

  if (warp < 8) {
    // ---- producers. Thread t handles rows 8 (t >> 5) + (t & 7) and that + 64
    // and the 8-value K chunk (t >> 3) & 3 of every step: eight consecutive
    // threads fill one 128-byte core matrix with one 16-byte store per tile.
    // The loads of step g + 1 are issued before step g is converted and
    // stored, so each thread keeps 128 bytes in flight while it works.
    const GemmOperand& o = a.fa;
    const int r_lo = tid & 7, c = (tid >> 3) & 3, rg = tid >> 5;
    long long kc_off = 0;  // offset of this thread's K chunk within a 32-value step
    for (int q = 3; q < 5 && q < a.fa_nk; ++q)
      if (((8 * c) >> q) & 1) kc_off += o.kstride[q];
    // per tile: the offsets of this thread's two rows (-1 past the X range) and the operand's scale
    auto tile_setup = [&](long long tile, long long* roff, float* f) {
      const int rt = (int)((tile / a.row_tiles_b) % a.row_tiles_a);
      const long long b = tile / ((long long)a.row_tiles_b * a.row_tiles_a);
      const long long item = b >> a.fa_ns, sidx = b & ((1ll << a.fa_ns) - 1);
      *f = 1.f;
      if (o.meta >= 0) {
        int m;
        *f = pack_scale(a.fa_meta_m[(long long)o.meta * a.fa_B + (o.dep ? item : 0ll)], &m);
      }
      long long bb = o.dep ? item * o.istride : 0ll;
      for (int q = 0; q < a.fa_ns; ++q)
        if ((sidx >> q) & 1) bb += o.sstride[q];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int m = rt * GT_ROWS + 8 * rg + 64 * h + r_lo;
        long long v = -1;
        if (m < (1 << a.fa_nx)) {
          v = bb;
          for (int q = 0; q < a.fa_nx; ++q)
            if ((m >> q) & 1) v += o.rstride[q];
        }
        roff[h] = v;
      }
    };
    auto load_step = [&](const long long* roff, int q, float4* v) {
      const int k0 = 32 * q;
      long long koff = kc_off;
      for (int t = 5; t < a.fa_nk; ++t)
        if ((k0 >> t) & 1) koff += o.kstride[t];
      const bool k_ok = k0 + 8 * c < (1 << a.fa_nk);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const bool ld = roff[h] >= 0 && k_ok;
        const float4* src = reinterpret_cast<const float4*>(o.ptr + (ld ? roff[h] + koff : 0ll));
#pragma unroll
        for (int u = 0; u < 4; ++u) v[4 * h + u] = ld ? __ldg(src + u) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
    };
    const long long my_tiles = blockIdx.x < n_tiles ? (n_tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const long long n_steps = my_tiles * a.k_tiles;
    long long lt = blockIdx.x;  // load cursor: tile and K step of the next load
    int lq = -1;
    long long lroff[2] = {-1, -1};
    float lf = 1.f;
    auto load_next = [&](float4* v, float* f) {  // the next step's values and scale
      if (++lq == a.k_tiles || lq == 0) {
        if (lq == a.k_tiles) lt += gridDim.x;
        lq = 0;
        tile_setup(lt, lroff, &lf);
      }
      *f = lf;
      load_step(lroff, lq, v);
    };
    int fills[N_STAGES] = {};
    bool ok = true;
    // converts and stores step g from v; false when a wait gave up
    auto store_step = [&](long long g, const float4* v, float f) {
      const int s = (int)(g % N_STAGES);
      // every producer thread waits for the MMAs that read stage s to finish
      // before it overwrites the stage
      const bool w_ok = fills[s] == 0 || mbar_wait(&empty_bar[s], (fills[s] - 1) & 1);
      if (!__all_sync(0xffffffffu, w_ok) || s_fail) return false;
      const uint32_t st = base + (uint32_t)s * STAGE_BYTES;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int r = 8 * rg + 64 * h + r_lo;
        float re[8], im[8];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const float4 x = v[4 * h + u];
          re[2 * u] = x.x * f;
          im[2 * u] = x.y * f;
          re[2 * u + 1] = x.z * f;
          im[2 * u + 1] = x.w * f;
        }
        const uint32_t off = gt_offset_h(r, 8 * c, 2);
        uint4 hv, lv;
        split16<GEMM_BF16, 8>(re, &hv, &lv);
        asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(st + off), "r"(hv.x), "r"(hv.y), "r"(hv.z),
                     "r"(hv.w)
                     : "memory");
        asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(st + HB + off), "r"(lv.x), "r"(lv.y),
                     "r"(lv.z), "r"(lv.w)
                     : "memory");
        split16<GEMM_BF16, 8>(im, &hv, &lv);
        asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(st + 2 * HB + off), "r"(hv.x), "r"(hv.y),
                     "r"(hv.z), "r"(hv.w)
                     : "memory");
        asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(st + 3 * HB + off), "r"(lv.x), "r"(lv.y),
                     "r"(lv.z), "r"(lv.w)
                     : "memory");
      }
      // the tensor cores read shared memory through the async proxy: every
      // thread orders its own stores before its arrival
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive(&full_bar[s]);
      ++fills[s];
      return true;
    };
    // two register buffers in turn: the loads of step g + 1 are in flight
    // while step g waits for its stage and is converted
    float4 va[8], vb[8];
    float fa = 1.f, fb = 1.f;
    if (n_steps > 0) load_next(va, &fa);
    for (long long g = 0; g < n_steps && ok; g += 2) {
      if (g + 1 < n_steps) load_next(vb, &fb);
      if (!store_step(g, va, fa)) {
        ok = false;
        break;
      }
      if (g + 1 >= n_steps) break;
      if (g + 2 < n_steps) load_next(va, &fa);
      if (!store_step(g + 1, vb, fb)) ok = false;
    }
    if (!ok) {
      s_fail = 1;
      if (lane == 0) atomicExch(a.status, 1);
    }
  } else if (warp == 8 && lane == 0) {
    // ---- B copies: the real-part and imaginary-part half tiles of every step
    int fills[N_STAGES] = {};
    long long g = 0;
    bool ok = true;
    const int kth = 2 * a.fa_kpad / 32;  // B half tiles along K per (batch, column tile)
    for (long long tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
      const int ct = (int)(tile % a.row_tiles_b);
      const long long b = tile / ((long long)a.row_tiles_b * a.row_tiles_a);
      const long long bb = b & a.b_bmask;
      const char* B_hi = (const char*)a.b_hi + (size_t)(bb * a.row_tiles_b + ct) * kth * HB;
      const char* B_lo = (const char*)a.b_lo + (size_t)(bb * a.row_tiles_b + ct) * kth * HB;
      for (int q = 0; q < a.k_tiles; ++q, ++g) {
        const int s = (int)(g % N_STAGES);
        if (fills[s] > 0 && !mbar_wait(&empty_bar[s], (fills[s] - 1) & 1)) {
          ok = false;
          break;
        }
        if (s_fail) {
          ok = false;
          break;
        }
        const uint32_t st = base + (uint32_t)s * STAGE_BYTES;
        const size_t kre = (size_t)q, kim = (size_t)(a.fa_kpad / 32 + q);  // half tiles of real-K positions
        mbar_expect_tx(&full_bar[s], 4 * HB);
        bulk_g2s(st + 4 * HB, B_hi + kre * HB, HB, &full_bar[s]);
        bulk_g2s(st + 5 * HB, B_lo + kre * HB, HB, &full_bar[s]);
        bulk_g2s(st + 6 * HB, B_hi + kim * HB, HB, &full_bar[s]);
        bulk_g2s(st + 7 * HB, B_lo + kim * HB, HB, &full_bar[s]);
        ++fills[s];
      }
    }
    if (!ok) {
      s_fail = 1;
      atomicExch(a.status, 1);
    }
    for (int s = 0; s < N_STAGES; ++s)
      if (fills[s] > 0) mbar_wait(&full_bar[s], (fills[s] - 1) & 1);
  } else if (warp == 9 && lane == 0) {
    // ---- MMA issuer
    long long g = 0;
    bool ok = true, issued = false;
    long long i = 0;
    for (long long tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x, ++i) {
      const int buf = (int)(i & 1);
      const long long j = i >> 1;
      if (j >= 1 && !mbar_wait(&tempty_bar[buf], (uint32_t)((j - 1) & 1))) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t tmem_d = tmem_base + (uint32_t)buf * 128u;
      for (int q = 0; q < a.k_tiles; ++q, ++g) {
        const int s = (int)(g % N_STAGES);
        const long long n = g / N_STAGES;
        if (!mbar_wait(&full_bar[s], (uint32_t)(n & 1)) || s_fail) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t st = base + (uint32_t)s * STAGE_BYTES;
#pragma unroll
        for (int part = 0; part < 2; ++part) {
          const uint32_t ah = st + (uint32_t)(2 * part) * HB, al = ah + HB;
          const uint32_t bh = st + (uint32_t)(4 + 2 * part) * HB, bl = bh + HB;
#pragma unroll
          for (int k2 = 0; k2 < 2; ++k2) {  // 2 MMAs of 32 bytes of K per 64-byte half-tile row
            const uint32_t off = (uint32_t)k2 * 256u;
            mma<GEMM_BF16>(tmem_d, sdesc(ah + off, 512u), sdesc(bh + off, 512u), (q > 0 || part > 0 || k2 > 0) ? 1u : 0u);
            mma<GEMM_BF16>(tmem_d, sdesc(ah + off, 512u), sdesc(bl + off, 512u), 1u);
            mma<GEMM_BF16>(tmem_d, sdesc(al + off, 512u), sdesc(bh + off, 512u), 1u);
          }
        }
        mma_commit(&empty_bar[s]);
        issued = true;
      }
      if (ok) mma_commit(&tfull_bar[buf]);
    }
    if (!ok) {
      s_fail = 1;
      atomicExch(a.status, 2);
    }
    if (issued) {
      mma_commit(&drain_bar);
      mbar_wait(&drain_bar, 0);
    }
  } else if (warp >= 10) {
    epilogue_warps(a, tmem_base, tfull_bar, tempty_bar, &s_fail, s_yoff, s_epi_stop, tid - 320, warp & 3, lane,
                   n_tiles);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 9) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS) : "memory");
  }
}

// Split of real matrices (rows x K per batch, row-major FP32) into hi/lo
// operands in tile-major layout.
template <int KIND>
__global__ void k_pack_real(const float* __restrict__ X, int rows, int K, int batch, void* hi, void* lo) {
  const long long n = (long long)batch * rows * K;
  const int esize = KIND == GEMM_BF16 ? 2 : 4;
  const int kt_count = K * esize / GT_KBYTES, rt_count = rows / GT_ROWS;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(i % K);
    const int r = (int)((i / K) % rows);
    const int b = (int)(i / ((long long)K * rows));
    const float x = X[i];
    const long long tile = ((long long)(b * rt_count + r / GT_ROWS) * kt_count + (k * esize) / GT_KBYTES);
    const size_t off = (size_t)tile * GT_TILE_BYTES + gt_offset(r % GT_ROWS, k, esize);
    if (KIND == GEMM_BF16) {
      const __nv_bfloat16 h = __float2bfloat16_rn(x);
      const __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
      *reinterpret_cast<__nv_bfloat16*>((char*)hi + off) = h;
      *reinterpret_cast<__nv_bfloat16*>((char*)lo + off) = l;
    } else {
      uint32_t h, l;
      asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
      const float rest = x - __uint_as_float(h);
      asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(l) : "f"(rest));
      *reinterpret_cast<uint32_t*>((char*)hi + off) = h;
      *reinterpret_cast<uint32_t*>((char*)lo + off) = l;
    }
  }
}


// side 0: A rows = X assignments, columns [Re | Im] over K.
// side 1: B rows 2n, 2n+1 = [Re | -Im], [Im | Re] over K for Y assignment n.
// A thread forms CH consecutive K values of one row (one 16-byte chunk of a
// core-matrix row per part); consecutive threads take consecutive rows, so
// eight threads fill one 128-byte core matrix. An operand's offset is linear
// in the bits of W = batch | row << ns | (k >> log2 CH) << (ns + nr); per
// operand the block keeps only the bits with a nonzero stride (a small folded
// tensor has at most two), and an operand that does not vary with the low K
// bits is loaded once per chunk.
constexpr int PK_BITS = 3 * GB_BITS;
constexpr int PK_TABS = PK_BITS / 8;   // byte tables of operand 0's offset (W bits 8q .. 8q+7)
constexpr int PK_ITEMS = 64;           // items whose operand scales are kept in shared memory
constexpr int PK_SIDE = 512;           // entries of the folded-tensor product table (rows x K values of a chunk)
template <int KIND, bool HALF>
__global__ void k_gemm_pack(const GemmBucketArgs g, int side, int pack_items) {
  __shared__ int s_nz[GB_SIDE];
  __shared__ unsigned char s_pos[GB_SIDE][PK_BITS];
  __shared__ long long s_str[GB_SIDE][PK_BITS];
  __shared__ int s_klo[GB_SIDE][8];
  __shared__ int s_kdep[GB_SIDE];
  __shared__ int s_kvec[GB_SIDE];          // 1: the chunk's K values are consecutive entries (vector loads)
  __shared__ long long s_tab0[PK_TABS][256];  // operand 0: offset of each value of W's byte q
  __shared__ float s_f[GB_SIDE][PK_ITEMS];    // power-of-two scale of operand j for item it
  // the folded tensors' product (operands 1.., item-invariant) for every
  // value of the W bits they hold (row) and every K value of a chunk
  __shared__ float2 s_side[PK_SIDE];
  __shared__ unsigned char s_upos[16];
  __shared__ int s_nu, s_use_side;
  constexpr int ES = KIND == GEMM_BF16 ? 2 : 4;
  constexpr int CH = 16 / ES;
  constexpr int CHB = KIND == GEMM_BF16 ? 3 : 2;  // log2 CH
  const GemmOperand* ops = side == 0 ? g.a : g.b;
  const int nops = side == 0 ? g.na : g.nb;
  const int nr = side == 0 ? g.nx : g.ny;
  const long long rows = side == 0 ? g.m_pad : g.n_pad;  // complex rows
  const long long batch = (long long)pack_items << g.ns;  // 1 item when the side does not depend on it
  const int kch = g.k_pad / CH;  // chunks per row (k_pad is a multiple of 64 / ES)
  const long long n = batch * rows * kch;
  constexpr int KB = HALF ? GT_KBYTES_H : GT_KBYTES;  // bytes of K per tile row
  const int kt_count = 2 * g.k_pad * ES / KB;
  const int rt_count = (int)((side == 0 ? rows : 2 * rows) / GT_ROWS);
  char* hi = (char*)(side == 0 ? g.a_hi : g.b_hi);
  char* lo = (char*)(side == 0 ? g.a_lo : g.b_lo);
  const int wbits = g.ns + nr + (g.nk > CHB ? g.nk - CHB : 0);
  if ((int)threadIdx.x < nops) {
    const int j = threadIdx.x;
    const GemmOperand& o = ops[j];
    int n = 0;
    for (int p = 0; p < wbits; ++p) {
      const long long st = p < g.ns ? o.sstride[p] : (p < g.ns + nr ? o.rstride[p - g.ns] : o.kstride[p - g.ns - nr + CHB]);
      if (st) {
        s_pos[j][n] = (unsigned char)p;
        s_str[j][n] = st;
        ++n;
      }
    }
    s_nz[j] = n;
    int kdep = 0;
    for (int q = 0; q < CH; ++q) {
      int a = 0;
      for (int b = 0; b < CHB && b < g.nk; ++b)
        if ((q >> b) & 1) a += (int)o.kstride[b];
      s_klo[j][q] = a;
      kdep |= a != 0;
    }
    s_kdep[j] = kdep;
    int kvec = CHB <= g.nk;
    for (int q = 0; q < CH && kvec; ++q) kvec = s_klo[j][q] == q;
    s_kvec[j] = kvec;
  }
  // operand 0 (the large one): its offset as a sum of per-byte table values
  // of W, so an element costs one table read per byte instead of one test
  // per nonzero stride
  for (int e = threadIdx.x; e < PK_TABS * 256; e += blockDim.x) {
    const int q = e >> 8, v = e & 255;
    const GemmOperand& o = ops[0];
    long long a = 0;
    for (int b = 0; b < 8; ++b) {
      const int p = 8 * q + b;
      if (!((v >> b) & 1) || p >= wbits) continue;
      a += p < g.ns ? o.sstride[p] : (p < g.ns + nr ? o.rstride[p - g.ns] : o.kstride[p - g.ns - nr + CHB]);
    }
    s_tab0[q][v] = a;
  }
  const bool f_tab = g.items <= PK_ITEMS;
  if (f_tab)
    for (int e = threadIdx.x; e < nops * g.items; e += blockDim.x) {
      const int j = e / g.items, it = e - j * g.items;
      const GemmOperand& o = ops[j];
      float f = 1.f;
      if (o.meta >= 0) {
        int m;
        f = pack_scale(g.meta_m[(long long)o.meta * g.B + (o.dep ? it : 0)], &m);
      }
      s_f[j][it] = f;
    }
  __syncthreads();
  if ((side == 0 || HALF) && blockIdx.x == 0) {
    // output exponent per item (by the A pack, or by the B pack when A is
    // fused): sum over every operand of its exponent and scale shift
    for (int it = threadIdx.x; it < g.items; it += blockDim.x) {
      int e = 0;
      for (int j = 0; j < g.na + g.nb; ++j) {
        const GemmOperand& o = j < g.na ? g.a[j] : g.b[j - g.na];
        if (o.meta < 0) continue;
        const long long row = (long long)o.meta * g.B + (o.dep ? it : 0);
        int m;
        pack_scale(g.meta_m[row], &m);
        e += g.meta_e[row] + m;
      }
      g.meta_e[(long long)g.out_meta * g.B + (g.out_dep ? it : 0)] = e;
    }
  }
  // with three or more operands whose folded tensors (1..) are all
  // item-invariant and hold few W bits: their product once per block, in a
  // table indexed by those bits and the K value within the chunk, so that an
  // element multiplies operand 0 by one table entry per K value
  if (threadIdx.x == 0) {
    unsigned long long um = 0;
    bool ok = nops >= 3;
    for (int j = 1; ok && j < nops; ++j) {
      ok = !ops[j].dep;
      for (int i = 0; i < s_nz[j]; ++i) um |= 1ull << s_pos[j][i];
    }
    int nu = 0;
    for (int p = 0; p < 64 && ok; ++p)
      if ((um >> p) & 1ull) {
        if (nu == 16) ok = false;
        else s_upos[nu++] = (unsigned char)p;
      }
    ok = ok && ((CH << nu) <= PK_SIDE);
    s_nu = nu;
    s_use_side = ok ? 1 : 0;
  }
  __syncthreads();
  const bool use_side = s_use_side != 0;
  if (use_side) {
    const int nu = s_nu;
    for (int e = threadIdx.x; e < (CH << nu); e += blockDim.x) {
      const int row = e >> CHB, q = e & (CH - 1);
      unsigned long long Wp = 0;
      for (int i = 0; i < nu; ++i)
        if ((row >> i) & 1) Wp |= 1ull << s_upos[i];
      float sr = 1.f, si = 0.f;
      for (int j = 1; j < nops; ++j) {
        const GemmOperand& o = ops[j];
        float f = 1.f;
        if (o.meta >= 0) {
          int m;
          f = pack_scale(g.meta_m[(long long)o.meta * g.B], &m);
        }
        long long off = s_klo[j][q];
        for (int i = 0; i < s_nz[j]; ++i)
          if ((Wp >> s_pos[j][i]) & 1ull) off += s_str[j][i];
        const float2 v = o.ptr[off];
        const float vx = v.x * f, vy = v.y * f;
        const float nr_ = sr * vx - si * vy, ni = sr * vy + si * vx;
        sr = nr_;
        si = ni;
      }
      s_side[e] = make_float2(sr, si);
    }
    __syncthreads();
  }
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    // 8 consecutive threads: the 8 rows of one core matrix (one 128-byte
    // store each); then the next K chunks of the same rows (contiguous reads
    // when K is the operand's lowest dimension)
    const long long q = i >> 3;
    const int kc = (int)(q % kch);
    const long long r8 = rows >> 3;
    const long long r = ((q / kch) % r8) * 8 + (i & 7);
    const long long bi = q / (kch * r8);
    const long long item = bi >> g.ns, sidx = bi & ((1ll << g.ns) - 1);
    const int k0 = kc * CH;
    float re[CH], im[CH];
    const bool row_ok = r < (1ll << nr);
#pragma unroll
    for (int q = 0; q < CH; ++q) {
      re[q] = row_ok && (k0 + q) < (1 << g.nk) ? 1.f : 0.f;
      im[q] = 0.f;
    }
    if (row_ok && k0 < (1 << g.nk)) {
      const unsigned long long W = (unsigned long long)sidx | ((unsigned long long)r << g.ns) |
                                   ((unsigned long long)(k0 >> CHB) << (g.ns + nr));
      for (int j = 0; j < (use_side ? 1 : nops); ++j) {
        const GemmOperand& o = ops[j];
        float f = 1.f;
        if (f_tab) {
          f = s_f[j][item];
        } else if (o.meta >= 0) {
          int m;
          f = pack_scale(g.meta_m[(long long)o.meta * g.B + (o.dep ? item : 0ll)], &m);
        }
        long long base = o.dep ? item * o.istride : 0ll;
        if (j == 0) {
#pragma unroll
          for (int q = 0; q < PK_TABS; ++q)
            if (8 * q < wbits) base += s_tab0[q][(W >> (8 * q)) & 255ull];
        } else {
          const int nz = s_nz[j];
          for (int i = 0; i < nz; ++i)
            if ((W >> s_pos[j][i]) & 1ull) base += s_str[j][i];
        }
        if (s_kvec[j] && j == 0 && k0 + CH <= (1 << g.nk)) {
          // CH consecutive entries: vector loads; operand 0 is the first factor
          const float4* src = reinterpret_cast<const float4*>(o.ptr + base);
#pragma unroll
          for (int q = 0; q < CH / 2; ++q) {
            const float4 v = __ldg(src + q);
            re[2 * q] = v.x * f;
            im[2 * q] = v.y * f;
            re[2 * q + 1] = v.z * f;
            im[2 * q + 1] = v.w * f;
          }
        } else if (!s_kdep[j]) {  // the same value for every K of the chunk
          const float2 v = o.ptr[base];
          const float vx = v.x * f, vy = v.y * f;
#pragma unroll
          for (int q = 0; q < CH; ++q) {
            const float nre = re[q] * vx - im[q] * vy, nim = re[q] * vy + im[q] * vx;
            re[q] = nre;
            im[q] = nim;
          }
        } else {
#pragma unroll
          for (int q = 0; q < CH; ++q) {
            if (k0 + q >= (1 << g.nk)) continue;
            const float2 v = o.ptr[base + s_klo[j][q]];
            const float vx = v.x * f, vy = v.y * f;
            const float nre = re[q] * vx - im[q] * vy, nim = re[q] * vy + im[q] * vx;
            re[q] = nre;
            im[q] = nim;
          }
        }
      }
      if (use_side) {  // times the folded tensors' product (K values past the end stay 0)
        int row = 0;
        for (int i = 0; i < s_nu; ++i) row |= (int)((W >> s_upos[i]) & 1ull) << i;
        const float2* sv = s_side + (row << CHB);
#pragma unroll
        for (int q = 0; q < CH; ++q) {
          const float2 v = sv[q];
          const float nre = re[q] * v.x - im[q] * v.y, nim = re[q] * v.y + im[q] * v.x;
          re[q] = nre;
          im[q] = nim;
        }
      }
    }
    uint4 h, l;
    auto goff = [](int rr, int kk) { return HALF ? gt_offset_h(rr, kk, ES) : gt_offset(rr, kk, ES); };
    const size_t tb = HALF ? (size_t)GT_TILE_BYTES_H : (size_t)GT_TILE_BYTES;
    const int kre = k0, kim = g.k_pad + k0;
    if (side == 0) {
      const size_t t0 = (size_t)(bi * rt_count + r / GT_ROWS) * kt_count;
      split16<KIND, CH>(re, &h, &l);
      size_t off = (t0 + (size_t)(kre * ES / KB)) * tb + goff((int)(r % GT_ROWS), kre);
      *reinterpret_cast<uint4*>(hi + off) = h;
      *reinterpret_cast<uint4*>(lo + off) = l;
      split16<KIND, CH>(im, &h, &l);
      off = (t0 + (size_t)(kim * ES / KB)) * tb + goff((int)(r % GT_ROWS), kim);
      *reinterpret_cast<uint4*>(hi + off) = h;
      *reinterpret_cast<uint4*>(lo + off) = l;
    } else {
      float nim[CH];
#pragma unroll
      for (int q = 0; q < CH; ++q) nim[q] = -im[q];
      const long long r0 = 2 * r, r1 = 2 * r + 1;
      const size_t t0 = (size_t)(bi * rt_count + r0 / GT_ROWS) * kt_count;
      const size_t t1 = (size_t)(bi * rt_count + r1 / GT_ROWS) * kt_count;
      // row 2r: [Re | -Im]
      split16<KIND, CH>(re, &h, &l);
      size_t off = (t0 + (size_t)(kre * ES / KB)) * tb + goff((int)(r0 % GT_ROWS), kre);
      *reinterpret_cast<uint4*>(hi + off) = h;
      *reinterpret_cast<uint4*>(lo + off) = l;
      split16<KIND, CH>(nim, &h, &l);
      off = (t0 + (size_t)(kim * ES / KB)) * tb + goff((int)(r0 % GT_ROWS), kim);
      *reinterpret_cast<uint4*>(hi + off) = h;
      *reinterpret_cast<uint4*>(lo + off) = l;
      // row 2r + 1: [Im | Re]
      split16<KIND, CH>(im, &h, &l);
      off = (t1 + (size_t)(kre * ES / KB)) * tb + goff((int)(r1 % GT_ROWS), kre);
      *reinterpret_cast<uint4*>(hi + off) = h;
      *reinterpret_cast<uint4*>(lo + off) = l;
      split16<KIND, CH>(re, &h, &l);
      off = (t1 + (size_t)(kim * ES / KB)) * tb + goff((int)(r1 % GT_ROWS), kim);
      *reinterpret_cast<uint4*>(hi + off) = h;
      *reinterpret_cast<uint4*>(lo + off) = l;
    }
  }
}

}  // namespace

// SMs of the current device (one query per call; the attribute is cached by the runtime).
static int device_sms() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      sms <= 0)
    sms = 1;
  return sms;
}

void gemm_tc_launch(int kind, const GemmArgs& args, void* stream) {
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int sms = device_sms();
  const long long tiles = (long long)args.batch * args.row_tiles_a * args.row_tiles_b;
  const unsigned grid = (unsigned)std::max<long long>(1, std::min<long long>(tiles, sms));  // one block per SM
  if (kind == GEMM_BF16) {
    cudaFuncSetAttribute(k_gemm_tc<GEMM_BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    k_gemm_tc<GEMM_BF16><<<grid, GEMM_THREADS, SMEM_BYTES, s>>>(args);
  } else {
    cudaFuncSetAttribute(k_gemm_tc<GEMM_TF32>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    k_gemm_tc<GEMM_TF32><<<grid, GEMM_THREADS, SMEM_BYTES, s>>>(args);
  }
}

bool gemm_fused_a(const GemmBucketArgs& g) {
  const char* env = std::getenv("TNQ_GEMM_FUSED_A");  // "0": always pack A (for comparisons)
  if ((env && env[0] == '0') || g.kind != GEMM_BF16 || g.na != 1 || g.nk < 3 || g.k_pad % 32) return false;
  const GemmOperand& o = g.a[0];
  // the three lowest summed variables are the tensor's lowest bits (8
  // consecutive complex values, 64 bytes, per load), every other stride a
  // multiple of 8 entries and the tensor 64-byte aligned
  if (o.kstride[0] != 1 || o.kstride[1] != 2 || o.kstride[2] != 4) return false;
  if (reinterpret_cast<uintptr_t>(o.ptr) % 64) return false;
  auto mult8 = [](long long v) { return v % 8 == 0; };
  if (!mult8(o.istride)) return false;
  for (int q = 0; q < g.ns; ++q)
    if (!mult8(o.sstride[q])) return false;
  for (int q = 0; q < g.nx; ++q)
    if (!mult8(o.rstride[q])) return false;
  for (int q = 3; q < g.nk; ++q)
    if (!mult8(o.kstride[q])) return false;
  return true;
}

void gemm_bucket_launch(const GemmBucketArgs& g, const GemmEpilogue& ep, int* status, void* stream) {
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int esize = g.kind == GEMM_BF16 ? 2 : 4;
  // a side whose operands are all item-invariant is packed once and shared by every item
  auto invariant = [](const GemmOperand* o, int n) {
    for (int j = 0; j < n; ++j)
      if (o[j].dep) return false;
    return true;
  };
  const bool inv_a = g.items > 1 && invariant(g.a, g.na), inv_b = g.items > 1 && invariant(g.b, g.nb);
  const int items_a = inv_a ? 1 : g.items, items_b = inv_b ? 1 : g.items;
  const long long batch = (long long)g.items << g.ns;
  const int ch = 16 / esize;  // K values per thread of k_gemm_pack
  const long long na = ((long long)items_a << g.ns) * g.m_pad * (g.k_pad / ch);
  const long long nb = ((long long)items_b << g.ns) * g.n_pad * (g.k_pad / ch);
  const long long cap = 16ll * device_sms();  // grid-stride pack: 16 blocks of 256 threads per SM
  const int blocks_a = (int)std::max<long long>(1, std::min<long long>((na + 255) / 256, cap));
  const int blocks_b = (int)std::max<long long>(1, std::min<long long>((nb + 255) / 256, cap));
  GemmArgs a;
  std::memset(&a, 0, sizeof(a));
  a.row_tiles_a = g.m_pad / GT_ROWS;
  a.row_tiles_b = 2 * g.n_pad / GT_ROWS;
  a.batch = (int)batch;
  a.a_bmask = inv_a ? (1ll << g.ns) - 1 : -1ll;
  a.b_bmask = inv_b ? (1ll << g.ns) - 1 : -1ll;
  a.status = status;
  a.out_c = nullptr;
  a.ep = ep;
  if (gemm_fused_a(g)) {
    k_gemm_pack<GEMM_BF16, true><<<blocks_b, 256, 0, s>>>(g, 1, items_b);
    a.b_hi = g.b_hi;
    a.b_lo = g.b_lo;
    a.k_tiles = g.k_pad / 32;  // K steps of 32 complex values
    a.fa = g.a[0];
    a.fa_ns = g.ns;
    a.fa_nx = g.nx;
    a.fa_nk = g.nk;
    a.fa_kpad = g.k_pad;
    a.fa_B = g.B;
    a.fa_meta_m = g.meta_m;
    const long long tiles = batch * a.row_tiles_a * a.row_tiles_b;
    const unsigned grid = (unsigned)std::max<long long>(1, std::min<long long>(tiles, device_sms()));
    cudaFuncSetAttribute(k_gemm_tc_fa, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    k_gemm_tc_fa<<<grid, GEMM_THREADS_FA, SMEM_BYTES, s>>>(a);
    return;
  }
  if (g.kind == GEMM_BF16) {
    k_gemm_pack<GEMM_BF16, false><<<blocks_a, 256, 0, s>>>(g, 0, items_a);
    k_gemm_pack<GEMM_BF16, false><<<blocks_b, 256, 0, s>>>(g, 1, items_b);
  } else {
    k_gemm_pack<GEMM_TF32, false><<<blocks_a, 256, 0, s>>>(g, 0, items_a);
    k_gemm_pack<GEMM_TF32, false><<<blocks_b, 256, 0, s>>>(g, 1, items_b);
  }
  a.a_hi = g.a_hi;
  a.a_lo = g.a_lo;
  a.b_hi = g.b_hi;
  a.b_lo = g.b_lo;
  a.k_tiles = 2 * g.k_pad * esize / GT_KBYTES;
  gemm_tc_launch(g.kind, a, stream);
}

}  // namespace tnq

// Internal test hook (not in include/tnq.h): runs a kernel whose mbarrier wait
// can never complete, bounded by limit_ns; returns TNQ_ETIMEOUT when the device
// reported the timeout (the expected outcome), TNQ_OK if it did not, TNQ_ECUDA
// on a CUDA error. The context stays usable.
extern "C" int tnq_internal_wait_timeout_selftest(unsigned long long limit_ns) {
  using namespace tnq;
  int* d = nullptr;
  if (cudaMalloc(&d, 4) != cudaSuccess) return 3;
  cudaMemset(d, 0, 4);
  k_wait_never<<<1, 32>>>(d, limit_ns);
  cudaError_t e = cudaDeviceSynchronize();
  int status = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&status, d, 4, cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return 3;
  return status ? 4 : 0;
}

// Internal self-test hook (not in include/tnq.h): C[b] = A[b] B[b]^T for real
// FP32 matrices (host, row-major: A batch x M x K, B batch x N x K, C batch x M
// x N) through the split-precision tensor-core path. M, N multiples of 128;
// K a multiple of 64 (BF16) or 32 (TF32). Returns 0, or nonzero with a message.
extern "C" int tnq_internal_gemm_selftest(int kind, int batch, int M, int N, int K, const float* A, const float* B,
                                          float* C, char* msg, size_t msg_len) {
  using namespace tnq;
  auto fail = [&](const std::string& m) {
    if (msg && msg_len) {
      std::strncpy(msg, m.c_str(), msg_len - 1);
      msg[msg_len - 1] = 0;
    }
    return 1;
  };
  const int esize = kind == GEMM_BF16 ? 2 : 4;
  if (batch < 1 || M % 128 || N % 128 || (K * esize) % GT_KBYTES || K <= 0) return fail("bad shape");
  const size_t na = (size_t)batch * M * K, nb = (size_t)batch * N * K, nc = (size_t)batch * M * N;
  float *dA = nullptr, *dB = nullptr, *dC = nullptr;
  void *ah = nullptr, *al = nullptr, *bh = nullptr, *bl = nullptr;
  int* dst = nullptr;
  auto cleanup = [&]() {
    cudaFree(dA); cudaFree(dB); cudaFree(dC); cudaFree(ah); cudaFree(al); cudaFree(bh); cudaFree(bl); cudaFree(dst);
  };
  cudaError_t e = cudaSuccess;
  if ((e = cudaMalloc(&dA, na * 4)) || (e = cudaMalloc(&dB, nb * 4)) || (e = cudaMalloc(&dC, nc * 4)) ||
      (e = cudaMalloc(&ah, na * esize)) || (e = cudaMalloc(&al, na * esize)) || (e = cudaMalloc(&bh, nb * esize)) ||
      (e = cudaMalloc(&bl, nb * esize)) || (e = cudaMalloc(&dst, 4))) {
    cleanup();
    return fail(std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  cudaMemcpy(dA, A, na * 4, cudaMemcpyHostToDevice);
  cudaMemcpy(dB, B, nb * 4, cudaMemcpyHostToDevice);
  cudaMemset(dC, 0, nc * 4);
  cudaMemset(dst, 0, 4);
  if (kind == GEMM_BF16) {
    k_pack_real<GEMM_BF16><<<1024, 256>>>(dA, M, K, batch, ah, al);
    k_pack_real<GEMM_BF16><<<1024, 256>>>(dB, N, K, batch, bh, bl);
  } else {
    k_pack_real<GEMM_TF32><<<1024, 256>>>(dA, M, K, batch, ah, al);
    k_pack_real<GEMM_TF32><<<1024, 256>>>(dB, N, K, batch, bh, bl);
  }
  GemmArgs g;
  std::memset(&g, 0, sizeof(g));
  g.a_bmask = g.b_bmask = -1ll;
  g.a_hi = ah;
  g.a_lo = al;
  g.b_hi = bh;
  g.b_lo = bl;
  g.row_tiles_a = M / 128;
  g.row_tiles_b = N / 128;
  g.k_tiles = K * esize / GT_KBYTES;
  g.batch = batch;
  g.status = dst;
  g.out_c = dC;
  g.ldc = N;
  gemm_tc_launch(kind, g, nullptr);
  e = cudaDeviceSynchronize();
  int status = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&status, dst, 4, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(C, dC, nc * 4, cudaMemcpyDeviceToHost);
  cleanup();
  if (e != cudaSuccess) return fail(std::string("CUDA: ") + cudaGetErrorString(e));
  if (status) return fail("device wait timed out");
  return 0;
}
