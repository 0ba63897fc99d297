// BF16 tensor-core GEMM on the 5th-generation tensor cores (tcgen05), the contraction behind
// every convolution of the warm-start network: forward (im2col rows x weights), input gradient
// (output gradient x weights) and weight gradient (output gradient x im2col, split over K).
//
// One CTA of 128 threads computes a 128 x 128 tile of D = A B^T:
//  * all threads stage 128 x 64 slices of A and B in shared memory in the canonical K-major
//    no-swizzle layout of the tensor cores (8-row x 16-byte core matrices: core matrices
//    adjacent along K are 128 B apart, 8-row groups 1024 B apart), from K-major or MN-major
//    global operands, each thread issuing all 16 of its 16-byte loads before storing; two
//    stages, so the next slice is staged while the MMAs read the other;
//  * one thread issues four tcgen05.mma.kind::f16 (M 128, N up to 128, K 16) per slice with
//    the FP32 accumulator in tensor memory (128 columns allocated per CTA) and commits them to
//    the stage's mbarrier;
//  * the four warps read the accumulator back with tcgen05.ld (warp w owns TMEM lanes
//    32w..32w+31 = tile rows) and apply the epilogue (raw store or the convolution's bias,
//    FiLM and SiLU, written channel-major so that consecutive threads write consecutive pixels).
// Every mbarrier wait is bounded (2 s on %globaltimer); on timeout the CTA sets the error word,
// waits (bounded) for its MMAs, frees its tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "net_internal.h"

namespace mcl {
namespace net {
namespace {

constexpr int kBM = 128, kBN = 128, kBK = 64;
constexpr int kStageBytes = kBM * kBK * 2;  // A and B slices are both 128 x 64 BF16 = 16 KiB
constexpr int kSmemBytes = 4 * kStageBytes + 64;
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
// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both K-major,
// N >> 3 at bit 17, M >> 4 at bit 24.
__device__ __forceinline__ uint32_t instr_desc(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(m >> 4) << 24);
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

__global__ void __launch_bounds__(128) gemm_bf16_tc_kernel(const GemmArgs g) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ int s_abort;
  uint8_t* sA = smem;                     // [2][16 KiB]
  uint8_t* sB = smem + 2 * kStageBytes;   // [2][16 KiB]
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + 4 * kStageBytes);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 2);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * kBN;
  const int64_t kbeg = (int64_t)blockIdx.z * g.k_per_split;
  const int64_t kend = min((int64_t)g.K, kbeg + g.k_per_split);
  const int nkb = kend > kbeg ? (int)((kend - kbeg + kBK - 1) / kBK) : 0;
  const int n_valid = min(kBN, g.N - n0);
  const int n_inst = (n_valid + 15) & ~15;  // instruction N: a multiple of 16 (M = 128)
  const uint32_t bar0 = smem_addr(&bars[0]), bar1 = smem_addr(&bars[1]);

  if (warp == 0) tmem_alloc(smem_addr(tslot), kTmemCols);
  if (tid == 0) {
    bar_init(bar0, 1);
    bar_init(bar1, 1);
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t idesc = instr_desc(kBM, n_inst);

  uint32_t phase[2] = {0u, 0u};
  int issued = 0;  // slices whose MMAs were committed
  for (int kb = 0; kb < nkb; ++kb) {
    const int s = kb & 1;
    if (kb >= 2) {
      // the MMAs of slice kb - 2 read this stage: wait for their commit
      if (!bar_wait(s ? bar1 : bar0, phase[s])) s_abort = 1;
      phase[s] ^= 1u;
    }
    const int64_t k0 = kbeg + (int64_t)kb * kBK;
    {
      uint4 va[kStageItems], vb[kStageItems];
      load_operand(va, g.a, g.lda, g.a_kmajor, g.a_vec, m0, kBM, g.M, k0, kend);
      load_operand(vb, g.b, g.ldb, g.b_kmajor, g.b_vec, n0, n_inst, g.N, k0, kend);
      store_operand(sA + s * kStageBytes, va, g.a_kmajor, m0, kBM, g.M);
      store_operand(sB + s * kStageBytes, vb, g.b_kmajor, n0, n_inst, g.N);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (s_abort) break;
    if (tid == 0) {
      tc_fence_after();
      const uint32_t a_base = smem_addr(sA + s * kStageBytes);
      const uint32_t b_base = smem_addr(sB + s * kStageBytes);
#pragma unroll
      for (int kk = 0; kk < kBK / 16; ++kk) {
        // K = 16 spans two core matrices along K: 256 bytes per step
        const uint64_t ad = smem_desc(a_base + kk * 256, 128, 1024);
        const uint64_t bd = smem_desc(b_base + kk * 256, 128, 1024);
        mma_bf16(tmem, ad, bd, idesc, (kb > 0 || kk > 0) ? 1u : 0u);
      }
      mma_commit(s ? bar1 : bar0);
    }
    issued = kb + 1;
  }
  // the commit of the last slice covers every earlier MMA of this thread
  if (issued > 0) {
    const int s = (issued - 1) & 1;
    if (!bar_wait(s ? bar1 : bar0, phase[s])) {
      s_abort = 1;
      bar_wait(s ? bar1 : bar0, phase[s]);  // second bounded wait before freeing TMEM
    }
  }
  __syncthreads();
  const bool ok = s_abort == 0;  // uniform over the CTA: tcgen05.ld is warp-collective
  if (!ok && tid == 0 && g.err) atomicOr(g.err, 1);
  tc_fence_after();

  if (ok) {
    const int row = m0 + warp * 32 + lane;
    const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
    for (int c0 = 0; c0 < n_inst; c0 += 16) {
      float v[16];
      if (issued > 0) {
        tmem_ld16(lane_addr + (uint32_t)c0, v);
      } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = 0.f;
      }
      if (row >= g.M) continue;
      if (g.mode == kGemmRaw) {
        float* d = g.d + (int64_t)blockIdx.z * g.split_stride;
        if (g.d_trans) {
          // column-major: for each column the warp's 32 rows are 32 consecutive floats
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (n0 + c0 + j < g.N) d[(int64_t)(n0 + c0 + j) * g.ldd + row] = v[j];
        } else {
          float* dst = d + (int64_t)row * g.ldd + n0 + c0;
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (n0 + c0 + j < g.N) dst[j] = v[j];
        }
      } else {
        const ConvEpilogue& e = g.ep;
        const int b = row / e.hw;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int o = n0 + c0 + j;
          if (o >= g.N) break;
          const float pre = v[j] + e.bias[o];
          float z = pre;
          if (e.film) {
            const float* f = e.film + (int64_t)b * e.film_stride + e.film_off;
            z = (1.f + f[o]) * pre + f[g.N + o];
          }
          const int64_t idx = (int64_t)o * g.M + row;
          e.pre[idx] = pre;
          if (e.y) e.y[idx] = e.act ? z / (1.f + expf(-z)) : z;
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, kTmemCols);
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

cudaError_t launch_gemm(const GemmArgs& g_in, int splits, cudaStream_t st) {
  if (!gemm_args_valid(g_in, splits)) return cudaErrorInvalidValue;
  GemmArgs g = g_in;
  g.a_vec = vec_ok(g.a, g.lda, g.a_kmajor ? g.K : g.M);
  g.b_vec = vec_ok(g.b, g.ldb, g.b_kmajor ? g.K : g.N);
  cudaError_t e = cudaFuncSetAttribute(gemm_bf16_tc_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
  if (e != cudaSuccess) return e;
  const dim3 grid((g.M + kBM - 1) / kBM, (g.N + kBN - 1) / kBN, splits);
  if (grid.y > 65535) return cudaErrorInvalidValue;
  gemm_bf16_tc_kernel<<<grid, 128, kSmemBytes, st>>>(g);
  return cudaGetLastError();
}

}  // namespace net
}  // namespace mcl
