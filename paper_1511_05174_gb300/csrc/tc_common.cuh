// Blackwell (sm_103a) building blocks shared by the tensor-core kernels:
// mbarriers with bounded waits, 2-D TMA loads, tcgen05 shared-memory and
// instruction descriptors, MMA issue/commit, TMEM loads, and the branch-free
// top-4 insertion of packed 32-bit keys.  Inline PTX; included by one
// translation unit each (internal linkage).
#pragma once
#include <cuda.h>
#include <cstdint>

namespace csp {
namespace tc {

constexpr long long kTimeoutCycles = 4000000000ll;  // about 2 s at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase of parity `parity` to complete.  Gives up (and
// records `code`) after kTimeoutCycles or when another thread recorded an error.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, unsigned long long *err, int code) {
  const long long t0 = clock64();
  int spins = 0;
  while (!mbar_try_wait(bar, parity)) {
    if (++spins == 256) {
      spins = 0;
      if (*reinterpret_cast<volatile unsigned long long *>(err) != 0ull) return false;
      if (clock64() - t0 > kTimeoutCycles) {
        atomicExch(err, (unsigned long long)code);
        return false;
      }
    }
  }
  return true;
}

// Bounded wait that ignores the error word: lets a thread wait out its own
// copies in flight before the CTA exits, even after an error elsewhere.
__device__ __forceinline__ bool mbar_drain(uint64_t *bar, uint32_t parity) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > kTimeoutCycles) return false;
  return true;
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of
// 128 bytes, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);          // start address
  d |= (uint64_t)1 << 16;                         // leading byte offset (unused for this layout)
  d |= (uint64_t)(1024 >> 4) << 32;               // stride byte offset: 8 rows x 128 B
  d |= (uint64_t)1 << 46;                         // descriptor version
  d |= (uint64_t)2 << 61;                         // 128-byte swizzle
  return d;
}

// Instruction descriptor of tcgen05.mma kind::f16: D FP32, A and B BF16, both
// K-major, shape M x N.
__host__ __device__ constexpr uint32_t instr_desc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld32_nowait(uint32_t taddr, uint32_t *r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}

__device__ __forceinline__ void tmem_ld16_nowait(uint32_t taddr, uint32_t *r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}

// Branch-free insertion of x into the sorted quadruple k0 >= k1 >= k2 >= k3.
__device__ __forceinline__ void top4_insert(uint32_t x, uint32_t &k0, uint32_t &k1, uint32_t &k2, uint32_t &k3) {
  const uint32_t l0 = min(k0, x);
  k0 = max(k0, x);
  const uint32_t l1 = min(k1, l0);
  k1 = max(k1, l0);
  const uint32_t l2 = min(k2, l1);
  k2 = max(k2, l1);
  k3 = max(k3, l2);
}

// Waits for this thread's TMEM loads; the 32 registers pass through the wait
// so that no use of them can be scheduled before it.
__device__ __forceinline__ void tmem_wait_ld32(uint32_t *r) {
  asm volatile(
      "tcgen05.wait::ld.sync.aligned;"
      : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
        "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]),
        "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]),
        "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
      :
      : "memory");
}

// Waits for this thread's TMEM loads, 16 registers passed through as above.
__device__ __forceinline__ void tmem_wait_ld16(uint32_t *r) {
  asm volatile(
      "tcgen05.wait::ld.sync.aligned;"
      : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
        "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15])
      :
      : "memory");
}

// Candidate keys of one chunk of N (16 or 32) accumulator columns (columns
// base .. base+N-1 of the dictionary, `lim` of them real atoms).  Each column's
// key is its |score| bits with the low log2(N) bits replaced by its
// complemented position in the chunk (larger score first, then the lower
// column); the chunk's two largest keys (two interleaved chains: three integer
// operations a column) are turned into global keys -- |score| bits above
// idx_bits, complemented atom index below (cb = imask - base) -- and inserted
// into the running top four.  The result holds the true top four of all
// columns seen unless three of them share a chunk; the update kernels re-score
// the candidates in FP32.  gmask must clear the low max(idx_bits, log2 N) bits.
template <int N, bool RAGGED>
__device__ __forceinline__ void chunk_top4(const uint32_t (&v)[N], int lim, uint32_t gmask, uint32_t cb,
                                           uint32_t &k0, uint32_t &k1, uint32_t &k2, uint32_t &k3) {
  static_assert(N == 16 || N == 32, "chunks of 16 or 32 columns");
  constexpr uint32_t pm = (uint32_t)N - 1u;
  const uint32_t lm = 0x7fffffffu & ~pm;
  uint32_t h0 = 0, l0 = 0, h1 = 0, l1 = 0;
#pragma unroll
  for (int i = 0; i < N; i += 2) {
    uint32_t x = (v[i] & lm) | (pm - (uint32_t)i);
    uint32_t y = (v[i + 1] & lm) | (pm - (uint32_t)(i + 1));
    if (RAGGED) {
      x = i < lim ? x : 0u;
      y = i + 1 < lim ? y : 0u;
    }
    const uint32_t t = min(h0, x);
    h0 = max(h0, x);
    l0 = max(l0, t);
    const uint32_t u = min(h1, y);
    h1 = max(h1, y);
    l1 = max(l1, u);
  }
  const uint32_t h = max(h0, h1), l = max(min(h0, h1), max(l0, l1));
  const uint32_t gh = h ? ((h & gmask) | (cb - pm + (h & pm))) : 0u;
  const uint32_t gl = l ? ((l & gmask) | (cb - pm + (l & pm))) : 0u;
  top4_insert(gh, k0, k1, k2, k3);
  top4_insert(gl, k0, k1, k2, k3);
}

}  // namespace tc

// 2-D BF16 tensor map over `rows` rows of `inner` elements, box 64 x box_rows,
// 128-byte swizzle, zero fill outside the tensor (host; false on failure).
bool tc_make_map_bf16(CUtensorMap *m, const void *base, uint64_t inner, uint64_t rows, uint32_t box_rows);

}  // namespace csp
