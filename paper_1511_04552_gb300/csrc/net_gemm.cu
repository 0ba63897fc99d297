// BF16 tensor-core GEMM on the 5th-generation tensor cores (tcgen05), the contraction behind
// every convolution of the warm-start network: forward (im2col rows x weights), input gradient
// (output gradient x weights) and weight gradient (output gradient x im2col, split over K).
//
// A persistent grid (every resident CTA slot, at most one CTA per tile) of 128-thread CTAs walks
// the 128 x 128 tiles of D = A B^T (and the K splits); for each tile:
//  * all threads stage 128 x 64 slices of A and B in shared memory in a ring of kStages
//    stages, kStages - 2 slices ahead of the MMAs; the slices of all of a CTA's tiles form one
//    stream, so the next tile's loads are in flight during a tile's epilogue. Operands whose
//    extents and leading dimensions are multiples of 8 go by 16-byte asynchronous copies
//    (cp.async, zero-filled beyond K): K-major ones into the canonical K-major no-swizzle
//    layout (8-row x 16-byte core matrices, 128 B apart along K, 1024 B per 8 rows), MN-major
//    ones into the canonical MN-major layout (core matrices of 8 k x 16 bytes along M or N),
//    which the instruction descriptor marks transposed; other operands through registers into
//    the K-major layout, each thread issuing all of its 16-byte loads before storing;
//  * one thread issues four tcgen05.mma.kind::f16 (M 128, N up to 128, K 16) per slice with
//    the FP32 accumulator in tensor memory (128 columns allocated per CTA) and commits them to
//    the stage's mbarrier;
//  * the four warps read the accumulator back with tcgen05.ld (warp w owns TMEM lanes
//    32w..32w+31 = tile rows) and apply the epilogue (raw store or the convolution's bias,
//    FiLM and SiLU, written channel-major so that consecutive threads write consecutive pixels).
// Every mbarrier wait is bounded (2 s on %globaltimer); on timeout the CTA sets the error word,
// waits (bounded) for its MMAs, frees its tensor memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "net_internal.h"

namespace mcl {
namespace net {
namespace {

constexpr int kBM = 128, kBN = 128, kBK = 64;
constexpr int kStageBytes = kBM * kBK * 2;  // A and B slices are both 128 x 64 BF16 = 16 KiB
constexpr int kSwBlock = 64 * kBK * 2;      // a 64 x 64 BF16 box of an MN-major operand, 8 KiB
constexpr int kStages = 6;                  // ring of A + B slices
constexpr int kAhead = kStages - 2;         // slices staged ahead of the one the MMAs read
// A stage holds the A slice (16 KiB) and the B slice of the GEMM's instruction N (<= 128 rows
// of 128 B); stage_stride = 16 KiB + 128 B x min(128, N rounded up to 16), set per launch.
__host__ __device__ constexpr int stage_stride_for(int N) {
  return kStageBytes + (N >= kBN ? kBN : ((N + 15) & ~15)) * kBK * 2;
}
__host__ __device__ constexpr int smem_bytes_for(int N) {
  return kStages * stage_stride_for(N) + 8 * kStages + 64;
}
constexpr uint32_t kTmemCols = 128;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint64_t now_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void bar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ bool bar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Waits for the phase with the given parity; false after about 2 s.
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity) {
  if (bar_try_wait(bar, parity)) return true;
  const uint64_t t0 = now_ns();
  for (uint32_t k = 0; k < (1u << 26); ++k) {
    if (bar_try_wait(bar, parity)) return true;
    if (now_ns() - t0 > 2000000000ull) return false;
  }
  return false;
}

// ---- tcgen05 wrappers ----------------------------------------------------------------------
__device__ __forceinline__ void tmem_alloc(uint32_t slot_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot_smem),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// Shared-memory matrix descriptor: start address, leading (K-direction) and stride
// (8-row-group) byte offsets, descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, A (bit 15) and B
// (bit 16) K-major (0) or MN-major (1), N >> 3 at bit 17, M >> 4 at bit 24.
__device__ __forceinline__ uint32_t instr_desc(int m, int n, bool a_mn, bool b_mn) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((a_mn ? 1u : 0u) << 15) |
         ((b_mn ? 1u : 0u) << 16) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}
// 16 consecutive FP32 accumulator columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// Offset of element (r, k) of a staged 128 x 64 slice (canonical K-major, no swizzle).
__device__ __forceinline__ uint32_t tile_off(int r, int k) {
  return (uint32_t)((((r >> 3) * 8 + (k >> 3)) << 7) + ((r & 7) << 4) + ((k & 7) << 1));
}

// Staging of rows [r0, r0 + rows) x k [k0, k0 + 64) of an operand (rows <= 128), zero outside
// R x K, in two phases so that each thread has all of its (at most 8) 16-byte global loads in
// flight before the first shared-memory store: load_operand into registers, store_operand into
// the canonical layout. K-major: element (r, k) at p[r * ld + k]; MN-major: p[k * ld + r]. With
// vec, 16-byte loads (the contiguous extent and ld are multiples of 8 and p is 16-byte
// aligned); otherwise element loads (small layers whose extents are not multiples of 8).
// K-major items: consecutive threads take consecutive rows of one 8-wide k group, so each group
// of 8 threads stores one contiguous 128-byte core-matrix column (no bank conflicts). MN-major
// items: consecutive threads read consecutive 8-row chunks of one k (coalesced).
constexpr int kStageItems = 8;  // 16-byte items per thread: 128 x 64 BF16 / (128 x 8)

// MN-major item `it` (8 rows at one k): a warp covers 2 row chunks x 16 consecutive k, so
// pairs of threads read adjacent 16-byte pieces of one 32-byte sector and the 2-byte stores of
// a warp hit each bank at most 4 times (consecutive row chunks on one k would all hit the same
// bank: the layout puts 8-row groups 1024 bytes apart).
__device__ __forceinline__ int mn_chunk(int it) { return (it & 1) + 2 * (it >> 7); }
__device__ __forceinline__ int mn_k(int it) { return (it >> 1) & 63; }

__device__ __forceinline__ void load_operand(uint4 (&v)[kStageItems],
                                             const __nv_bfloat16* __restrict__ p, int64_t ld,
                                             int kmajor, int vec, int r0, int rows, int R,
                                             int64_t k0, int64_t K) {
  const int tid = threadIdx.x;
  const uint16_t* p16 = reinterpret_cast<const uint16_t*>(p);
  const int total = rows * 8;  // = (rows / 8) * 64 for the MN-major items as well
#pragma unroll
  for (int u = 0; u < kStageItems; ++u) {
    const int it = tid + u * 128;
    v[u] = make_uint4(0u, 0u, 0u, 0u);
    if (it >= total) continue;
    uint16_t* e = reinterpret_cast<uint16_t*>(&v[u]);
    if (kmajor) {
      const int gr = r0 + it % rows;
      const int64_t gk = k0 + (it / rows) * 8;
      if (gr < R && gk < K) {
        if (vec) {
          v[u] = __ldg(reinterpret_cast<const uint4*>(p + (int64_t)gr * ld + gk));
        } else {
#pragma unroll
          for (int j = 0; j < 8; ++j)
            if (gk + j < K) e[j] = __ldg(p16 + (int64_t)gr * ld + gk + j);
        }
      }
    } else {
      const int rc = mn_chunk(it), kk = mn_k(it);
      const int gr = r0 + rc * 8;
      const int64_t gk = k0 + kk;
      if (gr < R && gk < K) {
        if (vec) {
          v[u] = __ldg(reinterpret_cast<const uint4*>(p + gk * ld + gr));
        } else {
#pragma unroll
          for (int j = 0; j < 8; ++j)
            if (gr + j < R) e[j] = __ldg(p16 + gk * ld + gr + j);
        }
      }
    }
  }
}

// K-major, 16-byte aligned operand (vec): rows [r0, r0 + rows) x k [k0, k0 + 64) copied with
// cp.async into the canonical layout; pieces beyond K are zero-filled (source size 0, the source
// address clamped to the operand's first element), rows beyond R are not staged (they only feed
// rows or columns of D that the epilogue discards).
__device__ __forceinline__ void copy_operand_async(uint8_t* dst, const __nv_bfloat16* __restrict__ p,
                                                   int64_t ld, int r0, int rows, int R,
                                                   int64_t k0, int64_t K) {
  const int tid = threadIdx.x;
  const int total = rows * 8;
#pragma unroll
  for (int u = 0; u < kStageItems; ++u) {
    const int it = tid + u * 128;
    if (it >= total) continue;
    const int r = it % rows;
    const int kk = (it / rows) * 8;
    const int gr = r0 + r;
    if (gr >= R) continue;  // feeds only rows (A) or columns (B) of D that are discarded
    const int64_t gk = k0 + kk;
    const bool in = gk < K;
    const __nv_bfloat16* src = in ? p + (int64_t)gr * ld + gk : p;
    const uint32_t d = smem_addr(dst + tile_off(r, kk));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src),
                 "r"(in ? 16 : 0)
                 : "memory");
  }
}
// MN-major, 16-byte aligned operand (vec): element (r, k) at p[k * ld + r]. Staged in the
// canonical MN-major no-swizzle layout: a core matrix is 8 k x 8 consecutive r (8 rows of 16 B,
// 128 B), core matrices adjacent along r 128 B apart, 8-k groups rows_cap x 16 B apart; so
// each 16-byte piece of the global operand is one row of a core matrix (no transposition).
__device__ __forceinline__ uint32_t mn_off(int r, int k, int rows_cap) {
  return (uint32_t)((k >> 3) * rows_cap * 16 + (r >> 3) * 128 + (k & 7) * 16);
}
__device__ __forceinline__ void copy_operand_async_mn(uint8_t* dst,
                                                      const __nv_bfloat16* __restrict__ p,
                                                      int64_t ld, int r0, int rows, int rows_cap,
                                                      int R, int64_t k0, int64_t K) {
  const int tid = threadIdx.x;
  const int chunks = rows / 8;  // 16-byte pieces per k
  const int total = chunks * kBK;
#pragma unroll
  for (int u = 0; u < kStageItems; ++u) {
    const int it = tid + u * 128;
    if (it >= total) continue;
    const int c = it % chunks, kk = it / chunks;  // consecutive threads: consecutive pieces
    const int gr = r0 + c * 8;
    if (gr >= R) continue;  // feeds only rows (A) or columns (B) of D that are discarded
    const int64_t gk = k0 + kk;
    const bool in = gk < K;
    const __nv_bfloat16* src = in ? p + gk * ld + gr : p;
    const uint32_t d = smem_addr(dst + mn_off(c * 8, kk, rows_cap));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src),
                 "r"(in ? 16 : 0)
                 : "memory");
  }
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Rows at or beyond R are not stored: they only feed rows (A) or columns (B) of D that the
// epilogue discards, so whatever the stage buffer holds there is harmless.
__device__ __forceinline__ void store_operand(uint8_t* dst, const uint4 (&v)[kStageItems],
                                              int kmajor, int r0, int rows, int R) {
  const int tid = threadIdx.x;
  const int total = rows * 8;
#pragma unroll
  for (int u = 0; u < kStageItems; ++u) {
    const int it = tid + u * 128;
    if (it >= total) continue;
    if (kmajor) {
      const int r = it % rows;
      if (r0 + r >= R) continue;
      *reinterpret_cast<uint4*>(dst + tile_off(r, (it / rows) * 8)) = v[u];
    } else {
      const int rc = mn_chunk(it), k = mn_k(it);
      if (r0 + rc * 8 >= R) continue;
      const uint16_t* e = reinterpret_cast<const uint16_t*>(&v[u]);
#pragma unroll
      for (int j = 0; j < 8; ++j)
        *reinterpret_cast<uint16_t*>(dst + tile_off(rc * 8 + j, k)) = e[j];
    }
  }
}

// Tiles of D (128 x 128, and a K split) are numbered m fastest, then n, then the split; a
// persistent CTA takes tiles blockIdx.x, + gridDim.x, ... and the slices of all its tiles form
// one stream through the stage ring, so the next tile's loads are in flight while a tile's
// epilogue runs.
// Epilogue of 16 accumulator columns n..n+15 of one row of D (split z): a raw store
// (row-major, or column-major with d_trans: a warp's 32 rows are then 32 consecutive floats),
// or the convolution's bias, FiLM and SiLU, written channel-major.
__device__ __forceinline__ void store_cols(const GemmArgs& g, int row, int n, int z,
                                           const float (&v)[16]) {
  if (g.mode == kGemmRaw) {
    float* d = g.d + (int64_t)z * g.split_stride;
    if (g.d_trans) {
#pragma unroll
      for (int j = 0; j < 16; ++j)
        if (n + j < g.N) d[(int64_t)(n + j) * g.ldd + row] = v[j];
    } else {
      float* dst = d + (int64_t)row * g.ldd + n;
#pragma unroll
      for (int j = 0; j < 16; ++j)
        if (n + j < g.N) dst[j] = v[j];
    }
  } else {
    const ConvEpilogue& e = g.ep;
    const int b = row / e.hw;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int o = n + j;
      if (o >= g.N) break;
      const float pre = v[j] + e.bias[o];
      float zz = pre;
      if (e.film) {
        const float* f = e.film + (int64_t)b * e.film_stride + e.film_off;
        zz = (1.f + f[o]) * pre + f[g.N + o];
      }
      const int64_t idx = (int64_t)o * g.M + row;
      e.pre[idx] = pre;
      if (e.y) e.y[idx] = e.act ? zz / (1.f + expf(-zz)) : zz;
    }
  }
}

struct TileCursor {
  int tile = 0, kb = 0, nkb = 0;
  int m0 = 0, n0 = 0, z = 0;
  int64_t kbeg = 0, kend = 0;
};

__device__ __forceinline__ bool tile_at(const GemmArgs& g, int mt, int nt, int n_tiles, int t,
                                        TileCursor& c) {
  if (t >= n_tiles) return false;
  c.tile = t;
  c.kb = 0;
  c.m0 = (t % mt) * kBM;
  c.n0 = ((t / mt) % nt) * kBN;
  c.z = t / (mt * nt);
  c.kbeg = (int64_t)c.z * g.k_per_split;
  c.kend = min((int64_t)g.K, c.kbeg + g.k_per_split);
  c.nkb = c.kend > c.kbeg ? (int)((c.kend - c.kbeg + kBK - 1) / kBK) : 0;
  return true;
}

__global__ void __launch_bounds__(128) gemm_bf16_tc_kernel(const GemmArgs g) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ int s_abort;
  // stage s: A slice at smem + s stage_stride, B slice right after it
  const int stride = stage_stride_for(g.N);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kStages * stride);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + kStages);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int mt = (g.M + kBM - 1) / kBM, nt = (g.N + kBN - 1) / kBN;
  const int n_tiles = mt * nt * g.splits;
  // 16-byte asynchronous staging where the operand allows it: K-major into the K-major layout,
  // MN-major into the MN-major layout (the instruction reads it transposed)
  const bool a_mn = !g.a_kmajor && g.a_vec, b_mn = !g.b_kmajor && g.b_vec;
  const bool a_async = g.a_vec != 0, b_async = g.b_vec != 0;
  const int b_cap = stride / (kBK * 2) - kBM;  // B rows a stage holds

  if (warp == 0) tmem_alloc(smem_addr(tslot), kTmemCols);
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) bar_init(smem_addr(&bars[s]), 1);
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  // slice number gs of the stream into stage gs % kStages
  auto produce = [&](const TileCursor& c, int64_t gs) {
    const int n_inst = (min(kBN, g.N - c.n0) + 15) & ~15;
    uint8_t* sa = smem + (int)(gs % kStages) * stride;
    uint8_t* sb = sa + kStageBytes;
    const int64_t k0 = c.kbeg + (int64_t)c.kb * kBK;
    if (a_mn) {
      copy_operand_async_mn(sa, g.a, g.lda, c.m0, kBM, kBM, g.M, k0, c.kend);
    } else if (a_async) {
      copy_operand_async(sa, g.a, g.lda, c.m0, kBM, g.M, k0, c.kend);
    } else {
      uint4 va[kStageItems];
      load_operand(va, g.a, g.lda, g.a_kmajor, g.a_vec, c.m0, kBM, g.M, k0, c.kend);
      store_operand(sa, va, g.a_kmajor, c.m0, kBM, g.M);
    }
    if (b_mn) {
      copy_operand_async_mn(sb, g.b, g.ldb, c.n0, n_inst, b_cap, g.N, k0, c.kend);
    } else if (b_async) {
      copy_operand_async(sb, g.b, g.ldb, c.n0, n_inst, g.N, k0, c.kend);
    } else {
      uint4 vb[kStageItems];
      load_operand(vb, g.b, g.ldb, g.b_kmajor, g.b_vec, c.n0, n_inst, g.N, k0, c.kend);
      store_operand(sb, vb, g.b_kmajor, c.n0, n_inst, g.N);
    }
  };
  // the MMAs of slice gs arrive on bars[gs % kStages]; its use number there gives the parity
  auto mma_done = [&](int64_t gs) {
    return bar_wait(smem_addr(&bars[gs % kStages]), (uint32_t)((gs / kStages) & 1));
  };
  // the producer's cursor: the next slice to stage (tiles without slices are skipped)
  TileCursor pc;
  bool p_live = tile_at(g, mt, nt, n_tiles, blockIdx.x, pc);
  auto p_settle = [&]() {
    while (p_live && pc.kb >= pc.nkb) p_live = tile_at(g, mt, nt, n_tiles, pc.tile + gridDim.x, pc);
  };
  p_settle();
  int64_t ps = 0;  // slices staged so far
  auto produce_next = [&]() {
    if (p_live) {
      // the slice reuses the stage of slice ps - kStages: wait for its MMAs
      if (ps >= kStages && !mma_done(ps - kStages)) s_abort = 1;
      produce(pc, ps);
      ++ps;
      ++pc.kb;
      p_settle();
    }
    cp_async_commit();  // one group per call (possibly empty): the group count stays in step
  };
  for (int i = 0; i < kAhead; ++i) produce_next();

  int64_t gs = 0;       // slices consumed so far
  int64_t last = -1;    // the latest slice whose MMAs were committed
  TileCursor c;
  for (int t = blockIdx.x; t < n_tiles && !s_abort; t += gridDim.x) {
    tile_at(g, mt, nt, n_tiles, t, c);
    const int n_valid = min(kBN, g.N - c.n0);
    const int n_inst = (n_valid + 15) & ~15;  // instruction N: a multiple of 16 (M = 128)
    const uint32_t idesc = instr_desc(kBM, n_inst, a_mn, b_mn);
    for (int kb = 0; kb < c.nkb; ++kb, ++gs) {
      produce_next();
      cp_async_wait<kAhead>();  // this thread's copies of slice gs have landed
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
      if (s_abort) break;
      if (tid == 0) {
        tc_fence_after();
        const uint32_t a_base = smem_addr(smem + (int)(gs % kStages) * stride);
        const uint32_t b_base = a_base + kStageBytes;
#pragma unroll
        for (int kk = 0; kk < kBK / 16; ++kk) {
          // K = 16 spans two core matrices along K. In both no-swizzle layouts the leading
          // byte offset is the stride between core matrices along K and the stride byte offset
          // the stride along M or N: K-major LBO 128 B, SBO 1024 B (256 bytes per K step);
          // MN-major LBO rows_cap x 16 B per 8-k group, SBO 128 B (two 8-k groups per K step)
          const uint64_t ad = a_mn ? smem_desc(a_base + kk * 2 * kBM * 16, kBM * 16, 128)
                                   : smem_desc(a_base + kk * 256, 128, 1024);
          const uint64_t bd = b_mn ? smem_desc(b_base + kk * 2 * b_cap * 16, b_cap * 16, 128)
                                   : smem_desc(b_base + kk * 256, 128, 1024);
          mma_bf16(tmem, ad, bd, idesc, (kb > 0 || kk > 0) ? 1u : 0u);
        }
        mma_commit(smem_addr(&bars[gs % kStages]));
      }
      last = gs;
    }
    if (s_abort) break;
    // the commit of the tile's last slice covers all of its MMAs
    if (c.nkb > 0 && !mma_done(gs - 1)) s_abort = 1;
    __syncthreads();
    if (s_abort) break;  // uniform over the CTA: tcgen05.ld is warp-collective
    tc_fence_after();
    const int row = c.m0 + warp * 32 + lane;
    const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
    for (int c0 = 0; c0 < n_inst; c0 += 16) {
      float v[16];
      if (c.nkb > 0) {
        tmem_ld16(lane_addr + (uint32_t)c0, v);
      } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = 0.f;
      }
      if (row < g.M) store_cols(g, row, c.n0 + c0, c.z, v);
    }
    // the accumulator is read before the next tile's MMAs overwrite it
    tc_fence_before();
    __syncthreads();
  }
  cp_async_wait<0>();  // no copy may still land in shared memory after the CTA moves on
  if (s_abort) {
    if (tid == 0 && g.err) atomicOr(g.err, 1);
    if (last >= 0) mma_done(last);  // a second bounded wait before the tensor memory is freed
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}


// ---- TMA-fed, warp-specialised variant ------------------------------------------------------
// For operands whose rows are 16-byte aligned and whose extents are multiples of 8: each slice
// of A and of B comes by TMA tensor loads with the 128-byte swizzle (every request a full
// 128-byte row), zero-filled beyond the operand: K-major operands as one box of 64 k x rows;
// MN-major operands as boxes of 64 M or N indices x 64 k (two for A, one per 64 columns of B),
// which the instruction descriptor marks transposed. Six warps: warp 4 lane 0 issues
// the loads into a ring of kStages stages, warp 5 lane 0 the MMAs (two accumulators of 128
// tensor-memory columns, so a tile's epilogue overlaps the next tile's MMAs), warps 0-3 read
// the accumulators back and store. Tiles and the per-stage mbarrier protocol:
//   full[s]   TMA bytes of slice gs landed (expect_tx by the producer)
//   empty[s]  the MMAs that read stage s are done (tcgen05.commit)
//   acc_full[a]  tile's MMAs done (commit after its last slice)
//   acc_empty[a] its 128 epilogue threads have read accumulator a
// Every wait is bounded (2 s); a role that gives up sets the abort word and the error bit.
constexpr int kTmaThreads = 192;

// B bytes of a stage: K-major n_cap rows of 128 B; MN-major whole 64-column boxes
__host__ __device__ constexpr int tma_b_bytes(int N, bool b_mn) {
  return b_mn ? ((N >= kBN ? kBN : ((N + 63) & ~63)) / 64) * kSwBlock
              : (N >= kBN ? kBN : ((N + 15) & ~15)) * kBK * 2;
}
__host__ __device__ constexpr int tma_stage_stride(int N, bool b_mn) {
  return kStageBytes + tma_b_bytes(N, b_mn);
}

struct TmaGemmMaps {
  CUtensorMap a, b;
};

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int c0, int c1,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(bar)
      : "memory");
}
// Descriptor of an operand in the 128-byte swizzled layout that TMA writes with SWIZZLE_128B
// (rows of 64 BF16 = 128 B, 16-byte chunks permuted within each 8-row, 1024-byte group; layout
// type 2 at bits 61-63). K-major: a row is 64 k of one M or N index, 8-row groups 1024 B apart
// (stride byte offset), the leading byte offset unused; K steps of 16 advance the start by
// 32 B. MN-major: a row is 64 M or N indices of one k, 8-k groups 1024 B apart (stride byte
// offset), blocks of 64 M or N indices 8192 B apart (leading byte offset); K steps of 16
// advance the start by two 8-k groups, 2048 B.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t saddr, uint32_t lbo) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)(1024 >> 4) << 32) | (1ull << 46) | (2ull << 61);
}

__device__ __forceinline__ void bar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
// a bounded wait that also gives up when another role has already given up
__device__ __forceinline__ bool role_wait(uint32_t bar, uint32_t parity, volatile int* abort) {
  if (bar_try_wait(bar, parity)) return true;
  const uint64_t t0 = now_ns();
  for (uint32_t k = 0; k < (1u << 26); ++k) {
    if (bar_try_wait(bar, parity)) return true;
    if (*abort || now_ns() - t0 > 2000000000ull) return false;
  }
  return false;
}

__global__ void __launch_bounds__(kTmaThreads) gemm_bf16_tma_kernel(
    const __grid_constant__ TmaGemmMaps maps, const GemmArgs g) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ int s_abort;
  const bool a_mn = !g.a_kmajor, b_mn = !g.b_kmajor;
  const int stride = tma_stage_stride(g.N, b_mn);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kStages * stride);
  uint64_t* full = bars;
  uint64_t* empty = bars + kStages;
  uint64_t* acc_full = bars + 2 * kStages;
  uint64_t* acc_empty = acc_full + 2;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(acc_empty + 2);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int mt = (g.M + kBM - 1) / kBM, nt = (g.N + kBN - 1) / kBN;
  const int n_tiles = mt * nt * g.splits;
  const int b_bytes = tma_b_bytes(g.N, b_mn);
  const uint32_t tx_bytes = (uint32_t)(kStageBytes + b_bytes);
  volatile int* abort = &s_abort;

  if (warp == 5) tmem_alloc(smem_addr(tslot), 2 * kTmemCols);
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      bar_init(smem_addr(&full[s]), 1);
      bar_init(smem_addr(&empty[s]), 1);
    }
    for (int a = 0; a < 2; ++a) {
      bar_init(smem_addr(&acc_full[a]), 1);
      bar_init(smem_addr(&acc_empty[a]), 128);
    }
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  int64_t produced = 0, mma_last = -1;
  if (warp == 4 && lane == 0) {
    // producer: the slices of this CTA's tiles, in order, into the stage ring
    int64_t gs = 0;
    TileCursor c;
    for (int t = blockIdx.x; t < n_tiles && !*abort; t += gridDim.x) {
      tile_at(g, mt, nt, n_tiles, t, c);
      for (int kb = 0; kb < c.nkb; ++kb, ++gs) {
        const int s = (int)(gs % kStages);
        if (gs >= kStages &&
            !role_wait(smem_addr(&empty[s]), (uint32_t)(((gs / kStages) - 1) & 1), abort)) {
          *abort = 1;
          break;
        }
        const uint32_t fb = smem_addr(&full[s]);
        bar_expect_tx(fb, tx_bytes);
        const uint32_t sa = smem_addr(smem + s * stride), sb = sa + kStageBytes;
        const int ko = (int)((c.kbeg + (int64_t)kb * kBK) / 8);  // first 8-k chunk
        const int k0 = ko * 8;
        if (a_mn) {
          tma_load_2d(sa, &maps.a, c.m0, k0, fb);
          tma_load_2d(sa + kSwBlock, &maps.a, c.m0 + 64, k0, fb);
        } else {
          tma_load_2d(sa, &maps.a, k0, c.m0, fb);
        }
        if (b_mn) {
          for (int j = 0; j * kSwBlock < b_bytes; ++j)
            tma_load_2d(sb + j * kSwBlock, &maps.b, c.n0 + 64 * j, k0, fb);
        } else {
          tma_load_2d(sb, &maps.b, k0, c.n0, fb);
        }
        produced = gs + 1;
      }
    }
  } else if (warp == 5 && lane == 0) {
    // MMA issuer
    int64_t gs = 0;
    int it = 0;  // tiles of this CTA so far
    TileCursor c;
    for (int t = blockIdx.x; t < n_tiles && !*abort; t += gridDim.x, ++it) {
      tile_at(g, mt, nt, n_tiles, t, c);
      const int acc = it & 1;
      const int n_inst = (min(kBN, g.N - c.n0) + 15) & ~15;
      const uint32_t idesc = instr_desc(kBM, n_inst, a_mn, b_mn);
      const uint32_t d_tmem = tmem + (uint32_t)(acc * kTmemCols);
      if (it >= 2 &&
          !role_wait(smem_addr(&acc_empty[acc]), (uint32_t)(((it >> 1) - 1) & 1), abort)) {
        *abort = 1;
        break;
      }
      tc_fence_after();
      for (int kb = 0; kb < c.nkb; ++kb, ++gs) {
        const int s = (int)(gs % kStages);
        if (!role_wait(smem_addr(&full[s]), (uint32_t)((gs / kStages) & 1), abort)) {
          *abort = 1;
          break;
        }
        tc_fence_after();
        const uint32_t a_base = smem_addr(smem + s * stride), b_base = a_base + kStageBytes;
#pragma unroll
        for (int kk = 0; kk < kBK / 16; ++kk) {
          // 128-byte swizzle: K-major 32 B per K step; MN-major 2048 B per K step, blocks
          // of 64 M or N indices 8 KiB apart
          const uint64_t ad = a_mn ? smem_desc_sw128(a_base + kk * 2048, kSwBlock)
                                   : smem_desc_sw128(a_base + kk * 32, 16);
          const uint64_t bd = b_mn ? smem_desc_sw128(b_base + kk * 2048, kSwBlock)
                                   : smem_desc_sw128(b_base + kk * 32, 16);
          mma_bf16(d_tmem, ad, bd, idesc, (kb > 0 || kk > 0) ? 1u : 0u);
        }
        mma_commit(smem_addr(&empty[s]));
        mma_last = gs;
      }
      if (*abort) break;
      mma_commit(smem_addr(&acc_full[acc]));  // also when the tile had no slice
    }
  } else if (warp < 4) {
    // epilogue: warp w reads tensor-memory lanes 32w..32w+31 (rows of the tile)
    int it = 0;
    TileCursor c;
    for (int t = blockIdx.x; t < n_tiles; t += gridDim.x, ++it) {
      tile_at(g, mt, nt, n_tiles, t, c);
      const int acc = it & 1;
      const bool ok = role_wait(smem_addr(&acc_full[acc]), (uint32_t)((it >> 1) & 1), abort);
      // tcgen05.ld is warp-collective: the whole warp agrees on ok
      if (!__all_sync(0xffffffffu, ok)) {
        *abort = 1;
        break;
      }
      tc_fence_after();
      const int row = c.m0 + warp * 32 + lane;
      const int n_inst = (min(kBN, g.N - c.n0) + 15) & ~15;
      const uint32_t lane_addr =
          tmem + (uint32_t)(acc * kTmemCols) + ((uint32_t)(warp * 32) << 16);
      for (int c0 = 0; c0 < n_inst; c0 += 16) {
        float v[16];
        if (c.nkb > 0) {
          tmem_ld16(lane_addr + (uint32_t)c0, v);
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j) v[j] = 0.f;
        }
        if (row < g.M) store_cols(g, row, c.n0 + c0, c.z, v);
      }
      tc_fence_before();
      bar_arrive(smem_addr(&acc_empty[acc]));
    }
  }
  __syncthreads();
  if (*abort) {
    // drain what is in flight before the shared and tensor memory go away (bounded waits)
    if (warp == 4 && lane == 0) {
      for (int64_t gs = produced - kStages > 0 ? produced - kStages : 0; gs < produced; ++gs)
        bar_wait(smem_addr(&full[gs % kStages]), (uint32_t)((gs / kStages) & 1));
    }
    if (warp == 5 && lane == 0 && mma_last >= 0)
      bar_wait(smem_addr(&empty[mma_last % kStages]), (uint32_t)((mma_last / kStages) & 1));
    if (tid == 0 && g.err) atomicOr(g.err, 1);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 5) tmem_dealloc(tmem, 2 * kTmemCols);
}

}  // namespace

bool gemm_args_valid(const GemmArgs& g, int splits) {
  if (g.M <= 0 || g.N <= 0 || g.K <= 0 || splits <= 0 || splits > 65535) return false;
  if (!g.a || !g.b) return false;
  if ((reinterpret_cast<uintptr_t>(g.a) | reinterpret_cast<uintptr_t>(g.b)) & 1u) return false;
  if (g.k_per_split <= 0 || g.k_per_split % kBK) return false;
  if ((int64_t)splits * g.k_per_split < g.K) return false;
  if (g.a_kmajor ? g.lda < g.K : g.lda < g.M) return false;
  if (g.b_kmajor ? g.ldb < g.K : g.ldb < g.N) return false;
  if (g.mode == kGemmRaw) {
    if (!g.d || g.ldd < (g.d_trans ? g.M : g.N)) return false;
    if (splits > 1 && g.split_stride < (int64_t)(g.d_trans ? g.N : g.M) * g.ldd) return false;
  } else if (g.mode == kGemmConvFwd) {
    if (splits != 1 || !g.ep.bias || !g.ep.pre || g.ep.hw <= 0 || g.M % g.ep.hw) return false;
  } else {
    return false;
  }
  return true;
}

// 16-byte loads are possible when the contiguous extent and the leading dimension are multiples
// of 8 elements and the base is 16-byte aligned.
int vec_ok(const void* p, int64_t ld, int64_t extent) {
  return ((reinterpret_cast<uintptr_t>(p) & 15u) == 0 && ld % 8 == 0 && extent % 8 == 0) ? 1 : 0;
}

namespace {

// The tensor map of one operand for the TMA variant, with the 128-byte swizzle: K-major
// {K, R} in boxes of 64 k x box_rows; MN-major {R, K} in boxes of 64 x 64. R is M or N, ld the
// leading dimension in elements. False if the driver refuses the map.
bool encode_operand(CUtensorMap* map, const __nv_bfloat16* p, int64_t ld, int kmajor, int R,
                    int64_t K, int box_rows) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
      return false;
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  const cuuint64_t row_bytes = (cuuint64_t)ld * 2;
  const cuuint32_t elem[2] = {1, 1};
  CUresult r;
  if (kmajor) {  // {K, rows}, boxes of 64 k x box_rows with the 128-byte swizzle
    const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)R};
    const cuuint64_t strides[1] = {row_bytes};
    const cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)box_rows};
    r = encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16*>(p), dims,
               strides, box, elem, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
               CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  } else {  // {R, K}, boxes of 64 x 64
    const cuuint64_t dims[2] = {(cuuint64_t)R, (cuuint64_t)K};
    const cuuint64_t strides[1] = {row_bytes};
    const cuuint32_t box[2] = {64, (cuuint32_t)kBK};
    r = encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16*>(p), dims,
               strides, box, elem, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
               CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  }
  return r == CUDA_SUCCESS;
}

int device_sms() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  return sms;
}

}  // namespace

cudaError_t launch_gemm(const GemmArgs& g_in, int splits, cudaStream_t st) {
  if (!gemm_args_valid(g_in, splits)) return cudaErrorInvalidValue;
  GemmArgs g = g_in;
  g.a_vec = vec_ok(g.a, g.lda, g.a_kmajor ? g.K : g.M);
  g.b_vec = vec_ok(g.b, g.ldb, g.b_kmajor ? g.K : g.N);
  g.splits = splits;
  const int64_t tiles = (int64_t)((g.M + kBM - 1) / kBM) * ((g.N + kBN - 1) / kBN) * splits;
  if (tiles > (1ll << 30)) return cudaErrorInvalidValue;
  const int sms = device_sms();
  if (sms < 1) return cudaErrorInvalidDevice;
  // TMA-fed variant: both operands with 16-byte aligned rows and extents in multiples of 8
  if (g.a_vec && g.b_vec) {
    TmaGemmMaps maps;
    const bool b_mn = !g.b_kmajor;
    const int b_rows = std::min(kBN, (g.N + 15) & ~15);
    if (encode_operand(&maps.a, g.a, g.lda, g.a_kmajor, g.M, g.K, kBM) &&
        encode_operand(&maps.b, g.b, g.ldb, g.b_kmajor, g.N, g.K, b_rows)) {
      const int smem = kStages * tma_stage_stride(g.N, b_mn) + (2 * kStages + 4) * 8 + 16;
      cudaError_t e = cudaFuncSetAttribute(gemm_bf16_tma_kernel,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           kStages * tma_stage_stride(kBN, false) + 256);
      if (e != cudaSuccess) return e;
      int per_sm = 0;
      if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gemm_bf16_tma_kernel,
                                                             kTmaThreads, smem)) != cudaSuccess)
        return e;
      per_sm = std::min(std::max(per_sm, 1), 2);  // 2 x 256 tensor-memory columns per SM
      const int grid = (int)std::min<int64_t>(tiles, (int64_t)sms * per_sm);
      gemm_bf16_tma_kernel<<<grid, kTmaThreads, smem, st>>>(maps, g);
      return cudaGetLastError();
    }
  }
  const int smem = smem_bytes_for(g.N);
  cudaError_t e = cudaFuncSetAttribute(gemm_bf16_tc_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       smem_bytes_for(kBN));
  if (e != cudaSuccess) return e;
  // persistent grid: every resident CTA slot of the device, at most one CTA per tile
  int per_sm = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gemm_bf16_tc_kernel, 128,
                                                         smem)) != cudaSuccess)
    return e;
  const int grid = (int)std::min<int64_t>(tiles, (int64_t)sms * std::max(1, per_sm));
  gemm_bf16_tc_kernel<<<grid, 128, smem, st>>>(g);
  return cudaGetLastError();
}

}  // namespace net
}  // namespace mcl
