// Full-dictionary proxy on the 5th-generation tensor cores (sm_103a).
//
// The proxy step of OMP (Sec. II-B, Algorithm 1: k = argmax_i |<a_i, r>|)
// over a tile of 128 patches is the dense contraction C = R A^T with R the
// tile's residuals (128 x M) and A the effective dictionary (T x M), rows
// scaled to unit norm so that |C| is the angle score.  Both operands are BF16
// (zero-padded to Mp = 64 k), the accumulator FP32 in tensor memory.
//
// CTA layout (320 threads):
//   warp 0  TMA producer: the residual tile once, then the atom tiles of NT
//           rows in 64-element K chunks through a ring of NS shared-memory
//           stages (cp.async.bulk.tensor, 128-byte swizzle, mbarrier
//           transaction counts), so that M up to 512 fits;
//   warp 1  TMEM allocator and single-thread MMA issuer (tcgen05.mma
//           kind::f16, M = 128, N = NT, K = 16 per instruction) into two
//           TMEM accumulators of NT columns, released by tcgen05.commit;
//   warps 2-9  epilogue: warps w and w + 4 share TMEM lane quadrant w % 4
//           (thread <-> patch) and split each accumulator's columns in two
//           halves; every thread reduces its columns 32 at a time (the next
//           chunk's TMEM load in flight): the chunk's two best keys (|score|
//           bits, complemented position) by a min/max pair per column, then
//           these as 32-bit packed keys (|score| bits above, T-complement of
//           the atom index below, so ties go to the lowest index) into the
//           running four best with a branch-free network; the halves merge
//           through shared memory.
// The kTopP candidates per patch are re-scored in FP32 by the update kernel,
// which excludes atoms already chosen.
//
// Every mbarrier wait is bounded (kTimeoutCycles); on expiry the thread sets
// the error word, the CTA drains its own outstanding copies and MMAs (again
// with a bound), frees its tensor memory and exits.
#include <cuda.h>

#include "csp_internal.cuh"
#include "tc_common.cuh"

namespace csp {

namespace {

using namespace csp::tc;

constexpr int TC_M = 128;
constexpr int TC_EPI_WARPS = 8;                    // two per TMEM lane quadrant
constexpr int TC_THREADS = 64 + 32 * TC_EPI_WARPS;
constexpr int TC_MAX_STAGES = 8;
constexpr int TC_HCOLS_MAX = 64;                   // accumulator columns per epilogue thread and tile

struct TcLayout {
  int kb;       // 64-element K blocks
  int nt;       // atoms per tile
  int ns;       // stages of the atom ring
  int r_bytes;  // residual tile
  int a_bytes;  // one stage: one K block of an atom tile
  int bar_off;  // barriers (after the 1024-aligned tiles)
  int mrg_off;  // epilogue merge area: [TC_M][4] keys
  int total;    // dynamic shared memory requested (includes alignment slack)
};

__host__ __device__ inline TcLayout tc_layout(int Mp, int nt) {
  TcLayout L;
  L.kb = Mp / 64;
  L.nt = nt;
  L.r_bytes = L.kb * TC_M * 128;
  L.a_bytes = nt * 128;
  // two CTAs per SM while the residual tile is small, else one
  const int budget = L.r_bytes <= 48 * 1024 ? 112 * 1024 : 220 * 1024;
  int ns = (budget - L.r_bytes - 4096) / L.a_bytes;
  L.ns = ns < 2 ? 2 : (ns > TC_MAX_STAGES ? TC_MAX_STAGES : ns);
  L.bar_off = L.r_bytes + L.ns * L.a_bytes;
  L.mrg_off = L.bar_off + 256;
  L.total = L.mrg_off + TC_M * 4 * 4 + 1024;
  return L;
}

__global__ void __launch_bounds__(TC_THREADS, 2)
proxy_tc_kernel(const __grid_constant__ CUtensorMap tmR, const __grid_constant__ CUtensorMap tmA, int Mp, int T,
                int nt, int idx_bits, int64_t row0, int64_t n, const int32_t *__restrict__ ids,
                const uint8_t *__restrict__ flags, int32_t *__restrict__ cand, unsigned long long *err,
                const float *__restrict__ pinv, int tiles_per_split, uint32_t *__restrict__ part, int wait_test) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const TcLayout lay = tc_layout(Mp, nt);
  uint8_t *r_tile = smem;
  uint8_t *a_stage = smem + lay.r_bytes;
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + lay.bar_off);
  const int NS = lay.ns;
  uint64_t *full = bars;                          // [NS] TMA -> MMA
  uint64_t *empty = bars + TC_MAX_STAGES;         // [NS] MMA -> TMA
  uint64_t *tfull = bars + 2 * TC_MAX_STAGES;     // [2] MMA -> epilogue
  uint64_t *tempty = tfull + 2;                   // [2] epilogue -> MMA
  uint64_t *rfull = tfull + 4;                    // residual tile landed
  uint64_t *mdone = tfull + 5;                    // all MMAs retired
  uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(tfull + 6);
  uint32_t *merge = reinterpret_cast<uint32_t *>(smem + lay.mrg_off);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t tile0 = (int64_t)blockIdx.x * TC_M;
  // this CTA's atom tiles: [j0, j0 + n_at) of the dictionary's ceil(T / nt)
  const int j0 = blockIdx.y * tiles_per_split;
  const int n_all = (T + nt - 1) / nt;
  const int n_at = min(tiles_per_split, n_all - j0);
  const uint32_t ncols = 2u * (uint32_t)nt;

  if (threadIdx.x == 0) {
    for (int i = 0; i < NS; ++i) {
      mbar_init(full + i, 1);
      mbar_init(empty + i, 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(tfull + i, 1);
      mbar_init(tempty + i, TC_EPI_WARPS);
    }
    mbar_init(rfull, 1);
    mbar_init(mdone, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_holder)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_holder;

  if (warp == 0) {
    if (lane == 0) {
      // producer: chunk t = (atom tile j, K block kb) goes to stage t % NS
      int issued[TC_MAX_STAGES] = {};  // loads issued per stage
      bool ok = true;
      mbar_expect_tx(rfull, (uint32_t)lay.r_bytes);
      for (int kb = 0; kb < lay.kb; ++kb)
        tma_load_2d(r_tile + kb * TC_M * 128, &tmR, kb * 64, (int)(row0 + tile0), rfull);
      // wait test: no atom tiles are loaded, so the MMA thread's bounded wait expires
      const int n_chunks = wait_test ? 0 : n_at * lay.kb;
      for (int t = 0; t < n_chunks && ok; ++t) {
        const int s = t % NS, use = t / NS;
        if (use >= 1) ok = mbar_wait(empty + s, (uint32_t)((use - 1) & 1), err, 1);
        if (!ok) break;
        const int j = t / lay.kb, kb = t - j * lay.kb;
        mbar_expect_tx(full + s, (uint32_t)lay.a_bytes);
        tma_load_2d(a_stage + s * lay.a_bytes, &tmA, kb * 64, (j0 + j) * nt, full + s);
        ++issued[s];
      }
      // drain: the last load of each stage and the residual tile have landed
      mbar_wait(rfull, 0, err, 2);
      for (int s = 0; s < NS; ++s)
        if (issued[s]) mbar_wait(full + s, (uint32_t)((issued[s] - 1) & 1), err, 2);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // MMA issuer
      const uint32_t idesc = instr_desc(TC_M, nt);
      bool ok = mbar_wait(rfull, 0, err, 3);
      const uint32_t r_base = smem_u32(r_tile);
      int t = 0;  // K-block chunk index, as in the producer
      for (int j = 0; j < n_at && ok; ++j) {
        const int a = j & 1;
        if (j >= 2) ok = mbar_wait(tempty + a, (uint32_t)(((j >> 1) - 1) & 1), err, 5);
        for (int kb = 0; kb < lay.kb && ok; ++kb, ++t) {
          const int s = t % NS;
          ok = mbar_wait(full + s, (uint32_t)((t / NS) & 1), err, 4);
          if (!ok) break;
          tc_fence_after();
          const uint32_t a_base = smem_u32(a_stage + s * lay.a_bytes);
#pragma unroll
          for (int kin = 0; kin < 4; ++kin) {
            const uint64_t ad = smem_desc(r_base + kb * TC_M * 128 + kin * 32);
            const uint64_t bd = smem_desc(a_base + kin * 32);
            mma_bf16(tmem + (uint32_t)(a * nt), ad, bd, idesc, (kb | kin) ? 1u : 0u);
          }
          mma_commit(empty + s);
        }
        if (!ok) break;
        mma_commit(tfull + a);
      }
      mma_commit(mdone);
      mbar_wait(mdone, 0, err, 6);
    }
  } else {
    // epilogue: warps 2..9; quadrant warp % 4, column half (warp - 2) / 4
    const int quad = warp & 3, half = (warp - 2) >> 2;
    const int row = quad * 32 + lane;
    const uint32_t imask = (1u << idx_bits) - 1u;
    const uint32_t smask = 0x7fffffffu & ~imask;
    const int hcols = nt / 2;
    // per-patch norms (per-patch Phi): scores scaled by 1/||Phi_p U d_i|| of this thread's patch
    const int64_t wi_row = tile0 + row;
    const float *prow = (pinv && wi_row < n) ? pinv + (ids ? (int64_t)ids[wi_row] : wi_row) * (int64_t)T : nullptr;
    const uint32_t gmask = smask & ~31u;
    uint32_t a0 = 0, a1 = 0, a2 = 0, a3 = 0;
    bool ok = true;
    for (int j = 0; j < n_at && ok; ++j) {
      const int a = j & 1;
      ok = mbar_wait(tfull + a, (uint32_t)((j >> 1) & 1), err, 7);
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) break;
      tc_fence_after();
      // 32-column chunks, the next one's TMEM load in flight while this one is reduced
      const uint32_t taddr = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(a * nt + half * hcols);
      uint32_t v[2][32];
      tmem_ld32_nowait(taddr, v[0]);
      tmem_wait_ld32(v[0]);
#pragma unroll
      for (int c = 0; c < TC_HCOLS_MAX / 32; ++c) {
        if (c * 32 >= hcols) break;
        const bool more = (c + 1) * 32 < hcols;
        if (more) tmem_ld32_nowait(taddr + (uint32_t)((c + 1) * 32), v[(c + 1) & 1]);
        uint32_t(&cur)[32] = v[c & 1];
        const int base = (j0 + j) * nt + half * hcols + c * 32;
        if (pinv) {
#pragma unroll
          for (int i = 0; i < 32; ++i) {
            const float pv = (prow && base + i < T) ? __ldg(prow + base + i) : 0.f;
            cur[i] = __float_as_uint(fabsf(__uint_as_float(cur[i])) * pv);
          }
        }
        const uint32_t cb = imask - (uint32_t)base;
        if (base + 32 <= T) chunk_top4<32, false>(cur, 32, gmask, cb, a0, a1, a2, a3);
        else chunk_top4<32, true>(cur, T - base, gmask, cb, a0, a1, a2, a3);
        if (more) tmem_wait_ld32(v[(c + 1) & 1]);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(tempty + a);
    }
    if (half == 1) {
      merge[row * 4 + 0] = a0;
      merge[row * 4 + 1] = a1;
      merge[row * 4 + 2] = a2;
      merge[row * 4 + 3] = a3;
    }
    asm volatile("bar.sync 1, %0;" ::"r"(32 * TC_EPI_WARPS) : "memory");
    const int64_t wi = tile0 + row;
    if (half == 0 && ok && wi < n) {
      for (int q = 0; q < 4; ++q) top4_insert(merge[row * 4 + q], a0, a1, a2, a3);
      const int64_t b = ids ? ids[wi] : wi;
      if (part) {  // atom range split across CTAs: partial top 4, merged by proxy_merge_kernel
        uint32_t *pp = part + (wi * gridDim.y + blockIdx.y) * 4;
        pp[0] = a0;
        pp[1] = a1;
        pp[2] = a2;
        pp[3] = a3;
      } else if (!(flags[b] & 1)) {
        const uint32_t ks[4] = {a0, a1, a2, a3};
#pragma unroll
        for (int q = 0; q < kTopP; ++q)
          cand[b * kTopP + q] = (q < 4 && ks[q]) ? (int)(imask - (ks[q] & imask)) : -1;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
}

// Top 4 of the S partial top-4 lists of every patch (atom range split).
__global__ void proxy_merge_kernel(const uint32_t *__restrict__ part, int S, int idx_bits, int64_t n,
                                   const int32_t *__restrict__ ids, const uint8_t *__restrict__ flags,
                                   int32_t *__restrict__ cand) {
  const int64_t wi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (wi >= n) return;
  const int64_t b = ids ? ids[wi] : wi;
  if (flags[b] & 1) return;
  uint32_t a0 = 0, a1 = 0, a2 = 0, a3 = 0;
  const uint32_t *pp = part + wi * S * 4;
  for (int i = 0; i < 4 * S; ++i) top4_insert(pp[i], a0, a1, a2, a3);
  const uint32_t imask = (1u << idx_bits) - 1u;
  const uint32_t ks[4] = {a0, a1, a2, a3};
#pragma unroll
  for (int q = 0; q < kTopP; ++q) cand[b * kTopP + q] = (q < 4 && ks[q]) ? (int)(imask - (ks[q] & imask)) : -1;
}

using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
    else
      cudaGetLastError();
  }
  return fn;
}

// 2-D BF16 tensor map over `rows` rows of `inner` elements, box 64 x box_rows,
// 128-byte swizzle, zero fill outside the tensor.
bool make_map(CUtensorMap *m, const void *base, uint64_t inner, uint64_t rows, uint32_t box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {inner, rows};
  cuuint64_t strides[1] = {inner * 2};
  cuuint32_t box[2] = {64, box_rows};
  cuuint32_t es[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int tile_atoms(int) { return 128; }  // 2 x 128 TMEM columns: two CTAs fit one SM's 512

}  // namespace

bool tc_make_map_bf16(CUtensorMap *m, const void *base, uint64_t inner, uint64_t rows, uint32_t box_rows) {
  return make_map(m, base, inner, rows, box_rows);
}

bool proxy_bf16_supported(int M, int T) {
  const int Mp = (M + 63) / 64 * 64;
  // packed 32-bit keys keep >= 16 score bits: T <= 2^15; the residual tile
  // (128 rows x Mp BF16) stays resident in shared memory: Mp <= 512
  return M > 0 && Mp <= 512 && T > 0 && T <= (1 << 15) && encode_fn() != nullptr;
}

int proxy_bf16_splits(int64_t n, int T) {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 1;
  }
  const int64_t tiles = (n + TC_M - 1) / TC_M;
  const int n_at = (T + tile_atoms(0) - 1) / tile_atoms(0);
  if (tiles >= 2 * sms || n_at < 2) return 1;
  // about two CTAs per SM: split the atom tiles over S CTAs per patch tile
  const int S = (int)((2 * sms + tiles - 1) / tiles);
  return S < n_at ? S : n_at;
}

bool launch_proxy_bf16(const __nv_bfloat16 *Rbf, int64_t rows_total, int Mp, const __nv_bfloat16 *Abf, int T,
                       int64_t row0, const int32_t *ids, int64_t n, const uint8_t *flags, int32_t *cand,
                       unsigned long long *err, const float *pinv, uint32_t *part, bool wait_test,
                       cudaStream_t s) {
  if (n == 0) return true;
  const int nt = tile_atoms(Mp);
  CUtensorMap mR, mA;
  if (!make_map(&mR, Rbf, (uint64_t)Mp, (uint64_t)rows_total, TC_M)) return false;
  if (!make_map(&mA, Abf, (uint64_t)Mp, (uint64_t)T, (uint32_t)nt)) return false;
  const TcLayout lay = tc_layout(Mp, nt);
  // at least 80 KB per CTA keeps two CTAs (2 x 2 NT <= 512 TMEM columns) per SM at most
  const int sm = lay.total < 80 * 1024 ? 80 * 1024 : lay.total;
  // the attribute is per device and function: set it on every launch (a host-side call)
  if (cudaFuncSetAttribute(proxy_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, sm) != cudaSuccess)
    return false;

  int idx_bits = 1;
  while ((1 << idx_bits) < T) ++idx_bits;  // atom index field of the packed keys
  const int n_all = (T + nt - 1) / nt;
  const int S = part ? proxy_bf16_splits(n, T) : 1;
  const int tps = (n_all + S - 1) / S;
  const dim3 grid((unsigned)((n + TC_M - 1) / TC_M), (unsigned)((n_all + tps - 1) / tps));
  proxy_tc_kernel<<<grid, TC_THREADS, sm, s>>>(mR, mA, Mp, T, nt, idx_bits, row0, n, ids, flags, cand, err, pinv,
                                               tps, grid.y > 1 ? part : nullptr, wait_test ? 1 : 0);
  if (grid.y > 1)
    proxy_merge_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(part, (int)grid.y, idx_bits, n, ids, flags, cand);
  return true;
}

}  // namespace csp
