// Fused full-dictionary OMP for a small shared dictionary: every iteration of
// Algorithm 1 (proxy, merge, projection, residue) for tiles of 128 patches in
// one CTA, with the residuals and the per-patch state kept on chip.  This is
// the coarse step of Algorithm 2 on shared-Phi workloads (T <= 256 atoms,
// M <= 64 measurements, K <= 8), where the separate per-iteration launches
// spend most of their time reloading state.
//
// Per iteration:
//   proxy   C = R A^T on the tensor cores (tcgen05.mma kind::f16, BF16 residual
//           tile 128 x 64 and unit-norm BF16 atoms T x 64 in shared memory, FP32
//           accumulator of T columns in tensor memory); the epilogue keeps the
//           four best packed keys (|score| bits, complemented atom index) per
//           patch;
//   update  two threads per patch re-score the four candidates in FP32 against
//           the FP32 residual (atoms without the chosen ones), take the best
//           (ties to the lowest index), extend the Cholesky factor of
//           A_Omega^T A_Omega (FP64 rebuild from scratch when the pivot ratio
//           falls below kTauPivot, which also rejects dependent atoms), solve for
//           alpha, form r = y - A_Omega alpha, and write r back as the next
//           BF16 tile (128-byte swizzle, the layout the MMA reads).
// The FP32 rows of A (zero padded to 64, rows 68 words apart so that the rows
// of different patches fall on different banks) and their squared norms stay
// in shared memory, so the re-score and the residue read no global memory;
// the Gram column G[q][Omega] comes from the level's Gram matrix (L2) when
// there is one, else from the shared rows.  The two threads of a patch own
// interleaved float4 chunks (2t and 2t + 1) of every 64-vector.
//
// A CTA runs NGRP groups of 256 threads, each with its own tile of 128 patches,
// its own half of the tensor memory and its own barriers, over one copy of
// the atoms; the second group starts one epilogue late, so that one group's
// top-4 selection (integer pipe) runs beside the other's update (shared
// memory).  One launch covers every mosaic phase (each CTA's tiles belong to
// one phase, whose atoms it loads).
//
// Roles: thread 0 loads the BF16 atoms by TMA; warp 0 owns the tensor memory;
// in each group, thread 0 issues the group's MMAs once the group barrier shows
// its residual tile complete, warps 8g .. 8g+7 run the epilogue (TMEM lane
// quadrant = warp % 4, half of the columns each) and then the update (thread
// pair per patch).  Every mbarrier wait is bounded; on expiry the error word is
// set, the group's threads leave the iteration loop together, and the tensor
// memory is freed.
#include <cstring>

#include "csp_internal.cuh"
#include "grp_common.cuh"
#include "tc_common.cuh"

namespace csp {

namespace {

using namespace csp::tc;
using csp::grp::GrpSmem;
using csp::grp::key_idx;
using csp::grp::pack_key;

constexpr int FZ_M = 128;        // patches per group tile (MMA M)
constexpr int FZ_MP = 64;        // padded measurement dimension (one 128-byte K block)
constexpr int FZ_AS = 68;        // words between FP32 atom rows in shared memory
constexpr int FZ_KMAX = 8;       // largest K of the fused form
constexpr int FZ_GT = 256;       // threads of a group: a pair per patch
constexpr int FZ_NCH = 8;        // float4 chunks per thread of a pair
constexpr int FZ_MAXPH = kMaxPhases;
constexpr int FZ_HCOLS_MAX = 128;  // accumulator columns per epilogue thread (half of T <= 256)

__host__ __device__ constexpr int ftri(int i) { return i * (i + 1) / 2; }

// Shared memory: the atoms (shared by the groups), then one block per group.
struct FzLayout {
  int a_bf;   // BF16 atoms [T][64], 128-byte swizzle (offset 0, 1024-aligned)
  int a_fp;   // FP32 atoms [T][FZ_AS]
  int inv;    // [T] 1/||a_i||
  int nrm;    // [T] ||a_i||^2 (FP32, the update's own dot product)
  int grp, gstride;                 // first group block, bytes per block (1024-aligned)
  int r_bf, cand, L, Linv, z, om, V, W;  // offsets within a group block
  int ls, ks, vs;                   // per-patch strides (words, odd): L, Linv/z/om, V/W
  int bars;
  int total;
};

__host__ __device__ inline FzLayout fz_layout(int T, int Kb, int ngrp) {
  FzLayout L;
  L.ls = ftri(Kb) | 1;
  L.ks = Kb | 1;
  L.vs = (Kb + 1) | 1;
  int o = 0;
  L.a_bf = o; o += T * FZ_MP * 2;
  L.a_fp = o; o += T * FZ_AS * 4;
  L.inv = o; o += T * 4;
  L.nrm = o; o += T * 4;
  o = (o + 1023) & ~1023;
  L.grp = o;
  int g = 0;
  L.r_bf = g; g += FZ_M * FZ_MP * 2;  // BF16 residual tile [128][64], 128-byte swizzle
  L.cand = g; g += FZ_M * 16;         // [128] top-4 keys
  L.L = g; g += FZ_M * L.ls * 4;
  L.Linv = g; g += FZ_M * L.ks * 4;
  L.z = g; g += FZ_M * L.ks * 4;
  L.om = g; g += FZ_M * L.ks * 4;
  L.V = g; g += FZ_M * L.vs * 4;
  L.W = g; g += FZ_M * L.vs * 4;
  L.gstride = (g + 1023) & ~1023;
  o += ngrp * L.gstride;
  L.bars = o; o += 128;
  L.total = o + 1024;  // alignment slack
  return L;
}

// Per-phase operands of one launch.
struct FzArgs {
  CUtensorMap map[FZ_MAXPH];            // BF16 atoms of each phase
  const float *A[FZ_MAXPH];             // FP32 effective dictionary [T][M]
  const float *inv[FZ_MAXPH];           // [T] 1/||a_i||
  const float *G[FZ_MAXPH];             // [T][T] Gram matrix A A^T (null: Gram column from the rows)
  int64_t row0[FZ_MAXPH + 1];           // first position of each phase in the patch list
  int cta0[FZ_MAXPH + 1];               // first CTA of each phase
  int nph;
};

__device__ __forceinline__ float pair_sum(float v) { return v + __shfl_xor_sync(0xffffffffu, v, 1); }

// Partial dot of this thread's chunks (2t + h) of a 64-wide shared row with its
// register chunks; four independent chains, summed in a fixed order.
__device__ __forceinline__ float half_dot(const float *row, int h, const float4 (&v)[FZ_NCH]) {
  const float4 *r4 = reinterpret_cast<const float4 *>(row);
  float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
#pragma unroll
  for (int t = 0; t < FZ_NCH; ++t) {
    const float4 a = r4[2 * t + h];
    s0 = fmaf(a.x, v[t].x, s0);
    s1 = fmaf(a.y, v[t].y, s1);
    s2 = fmaf(a.z, v[t].z, s2);
    s3 = fmaf(a.w, v[t].w, s3);
  }
  return (s0 + s1) + (s2 + s3);
}

// Same for two shared rows.
__device__ __forceinline__ float half_dot2(const float *ra, const float *rb, int h) {
  const float4 *a4 = reinterpret_cast<const float4 *>(ra);
  const float4 *b4 = reinterpret_cast<const float4 *>(rb);
  float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
#pragma unroll
  for (int t = 0; t < FZ_NCH; ++t) {
    const float4 a = a4[2 * t + h], b = b4[2 * t + h];
    s0 = fmaf(a.x, b.x, s0);
    s1 = fmaf(a.y, b.y, s1);
    s2 = fmaf(a.z, b.z, s2);
    s3 = fmaf(a.w, b.w, s3);
  }
  return (s0 + s1) + (s2 + s3);
}

// BF16 copy of this thread's chunks into row `row` of the 128-byte-swizzled
// tile: 16-byte chunk j of a row (elements 8j .. 8j+7: float4 chunks 2j of
// thread 0 and 2j+1 of thread 1) sits at chunk j ^ (row % 8).
__device__ __forceinline__ void store_rbf(uint8_t *tile, int row, int h, const float4 (&r)[FZ_NCH]) {
#pragma unroll
  for (int j = 0; j < FZ_NCH; ++j) {
    __nv_bfloat162 w0 = __floats2bfloat162_rn(r[j].x, r[j].y), w1 = __floats2bfloat162_rn(r[j].z, r[j].w);
    uint2 v;
    v.x = *reinterpret_cast<uint32_t *>(&w0);
    v.y = *reinterpret_cast<uint32_t *>(&w1);
    *reinterpret_cast<uint2 *>(tile + row * 128 + ((j ^ (row & 7)) << 4) + 8 * h) = v;
  }
}

__device__ __forceinline__ void group_bar(int id) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "n"(FZ_GT) : "memory");
}

template <int NGRP>
__global__ void __launch_bounds__(NGRP * FZ_GT, 1)
omp_fused_tc_kernel(const __grid_constant__ FzArgs args, const float *__restrict__ Y, int M, int T, int idx_bits,
                    const int32_t *__restrict__ ids, const int8_t *__restrict__ Kp, int Kuni, int Kb,
                    int32_t *__restrict__ omega, float *__restrict__ alpha, int ldo, int8_t *__restrict__ k_eff,
                    int64_t *stats, unsigned long long *err) {
  extern __shared__ uint8_t fz_raw[];
  uint8_t *sm = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(fz_raw) + 1023) & ~uintptr_t(1023));
  const FzLayout lay = fz_layout(T, Kb, NGRP);
  uint8_t *a_bf = sm + lay.a_bf;
  float *a_fp = reinterpret_cast<float *>(sm + lay.a_fp);
  float *s_inv = reinterpret_cast<float *>(sm + lay.inv);
  float *s_nrm = reinterpret_cast<float *>(sm + lay.nrm);
  uint64_t *bars = reinterpret_cast<uint64_t *>(sm + lay.bars);
  uint64_t *afull = bars, *accfull = bars + 1;  // accfull[NGRP]
  uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(bars + 1 + NGRP);
  int *s_flag = reinterpret_cast<int *>(bars + 2 + NGRP);  // [NGRP]

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // this CTA's phase and tiles
  int ph = 0;
  while (ph + 1 < args.nph && (int)blockIdx.x >= args.cta0[ph + 1]) ++ph;
  const float *A = args.A[ph];
  const float *inv_norm = args.inv[ph];
  const float *Gm = args.G[ph];
  const int64_t prow0 = args.row0[ph], pn = args.row0[ph + 1] - prow0;
  const int64_t tile_first = (int64_t)(blockIdx.x - args.cta0[ph]) * NGRP;
  const int64_t ntiles = (pn + FZ_M - 1) / FZ_M;
  const int nact = (int)(ntiles - tile_first < NGRP ? ntiles - tile_first : NGRP);  // groups with a tile
  uint32_t ncols = 32;
  while ((int)ncols < T) ncols <<= 1;

  if (threadIdx.x == 0) {
    mbar_init(afull, 1);
    for (int g = 0; g < NGRP; ++g) {
      mbar_init(accfull + g, 1);
      s_flag[g] = 0;
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_holder)),
                 "r"(ncols * NGRP)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  // FP32 atoms (zero padded to 64) and inverse norms, cooperatively, four
  // 16-byte loads in flight per thread
  {
    const int nv = M >> 2, total4 = T * (FZ_MP / 4), nt = blockDim.x;
    for (int e0 = threadIdx.x; e0 < total4; e0 += 4 * nt) {
      float4 v[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int e = e0 + q * nt, i = e >> 4, c = e & 15;
        v[q] = (e < total4 && c < nv) ? __ldg(reinterpret_cast<const float4 *>(A + (int64_t)i * M) + c)
                                      : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int e = e0 + q * nt;
        if (e < total4) reinterpret_cast<float4 *>(a_fp + (e >> 4) * FZ_AS)[e & 15] = v[q];
      }
    }
    for (int i = threadIdx.x; i < T; i += nt) s_inv[i] = __ldg(inv_norm + i);
  }
  __syncthreads();
  // ||a_i||^2 with the pair arithmetic of the update (half_dot2 + pair sum)
  for (int e = threadIdx.x; e < 2 * T; e += blockDim.x) {
    const int i = e >> 1, h = e & 1;
    const float *ai = a_fp + i * FZ_AS;
    const float v = pair_sum(half_dot2(ai, ai, h));
    if (h == 0) s_nrm[i] = v;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_holder;

  if (threadIdx.x == 0) {
    mbar_expect_tx(afull, (uint32_t)(T * 128));
    tma_load_2d(a_bf, &args.map[ph], 0, 0, afull);
  }
  if (warp / 8 < nact) {
    // ---- a group: epilogue and update of one tile ----
    const int g = warp / 8;
    uint8_t *gb = sm + lay.grp + g * lay.gstride;
    uint8_t *r_bf = gb + lay.r_bf;
    uint4 *cand4 = reinterpret_cast<uint4 *>(gb + lay.cand);
    uint64_t *af = accfull + g;
    volatile int *flag = s_flag + g;
    const uint32_t tm = tmem + (uint32_t)g * ncols;
    const int bar_id = 1 + g;
    const int u = threadIdx.x - g * FZ_GT;
    const int p = u >> 1, h = u & 1;  // update: patch p, chunks 2t + h
    const int quad = warp & 3, ehalf = (warp & 7) >> 2, erow = quad * 32 + lane;  // epilogue row
    const int64_t wl = (tile_first + g) * FZ_M + p;  // position within the phase
    const bool valid = wl < pn;
    const int64_t b = valid ? (ids ? (int64_t)ids[prow0 + wl] : prow0 + wl) : 0;
    int Kpb = valid ? (Kp ? (int)Kp[b] : Kuni) : 0;
    Kpb = Kpb < Kb ? Kpb : Kb;
    float *Lp = reinterpret_cast<float *>(gb + lay.L) + p * lay.ls;
    float *Linv = reinterpret_cast<float *>(gb + lay.Linv) + p * lay.ks;
    float *zp = reinterpret_cast<float *>(gb + lay.z) + p * lay.ks;
    int *omp = reinterpret_cast<int *>(gb + lay.om) + p * lay.ks;
    float *Vp = reinterpret_cast<float *>(gb + lay.V) + p * lay.vs;
    float *Wp = reinterpret_cast<float *>(gb + lay.W) + p * lay.vs;
    auto arow = [&](int i) -> const float * { return a_fp + i * FZ_AS; };
    int fb_misc = 0;
    // r (= y at the start): this thread's chunks, zero padded.  y itself is not
    // kept: the residual is updated by the change of alpha, and z_k comes from
    // the FP32 correlation <a_q, r> of the chosen atom
    const float *yrow = Y + b * M;
    float4 rv[FZ_NCH];
#pragma unroll
    for (int t = 0; t < FZ_NCH; ++t) {
      const int m0 = 4 * (2 * t + h);
      rv[t] = (valid && m0 < M) ? __ldg(reinterpret_cast<const float4 *>(yrow + m0)) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    float ysq = 0.f;
#pragma unroll
    for (int t = 0; t < FZ_NCH; ++t)
      ysq = fmaf(rv[t].x, rv[t].x, fmaf(rv[t].y, rv[t].y, fmaf(rv[t].z, rv[t].z, fmaf(rv[t].w, rv[t].w, ysq))));
    ysq = pair_sum(ysq);
    float rsq = ysq;
    int k = 0;
    uint8_t fl = 0;  // bit 1: FP64 from here on
    bool act = valid && Kpb > 0;
    store_rbf(r_bf, p, h, rv);
    const uint32_t imask = (1u << idx_bits) - 1u;
    const uint32_t smask = 0x7fffffffu & ~imask;
    const uint32_t gmask = smask & ~15u;
    const int hcols = T / 2;
    // with two groups, group 1 starts once group 0 has finished its first
    // epilogue, so that one group's epilogue (integer-pipe bound) runs beside
    // the other's update (shared-memory bound) instead of in step with it
    const bool stagger = NGRP == 2 && nact == 2;
    bool staged = false;
    if (stagger && g == 1) asm volatile("bar.sync 3, %0;" ::"n"(2 * FZ_GT) : "memory");
    for (int it = 0; it < Kb; ++it) {
      // the residual tile is complete: C = R A^T into this group's columns
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      group_bar(bar_id);
      if (u == 0 && (it > 0 || mbar_wait(afull, 0, err, 12))) {
        tc_fence_after();
        const uint32_t idesc = instr_desc(FZ_M, T);
#pragma unroll
        for (int kin = 0; kin < 4; ++kin) {
          const uint64_t ad = smem_desc(smem_u32(r_bf) + kin * 32);
          const uint64_t bd = smem_desc(smem_u32(a_bf) + kin * 32);
          mma_bf16(tm, ad, bd, idesc, kin ? 1u : 0u);
        }
        mma_commit(af);
      }
      // ---- epilogue: top 4 keys of this row's half of the columns ----
      const bool okw = mbar_wait(af, (uint32_t)(it & 1), err, 14);
      if (!okw) *flag = 1;
      group_bar(bar_id);
      if (*flag) break;
      tc_fence_after();
      // 16-column chunks (T is a multiple of 64: every column is an atom), the
      // next chunk's TMEM load in flight while this one is reduced
      uint32_t a0 = 0, a1 = 0, a2 = 0, a3 = 0;
      {
        const uint32_t taddr = tm + ((uint32_t)(quad * 32) << 16) + (uint32_t)(ehalf * hcols);
        uint32_t v[2][16];
        tmem_ld16_nowait(taddr, v[0]);
        tmem_wait_ld16(v[0]);
#pragma unroll
        for (int c = 0; c < FZ_HCOLS_MAX / 16; ++c) {
          if (c * 16 >= hcols) break;
          const bool more = (c + 1) * 16 < hcols;
          if (more) tmem_ld16_nowait(taddr + (uint32_t)((c + 1) * 16), v[(c + 1) & 1]);
          const int base = ehalf * hcols + c * 16;
          chunk_top4<16, false>(v[c & 1], 16, gmask, imask - (uint32_t)base, a0, a1, a2, a3);
          if (more) tmem_wait_ld16(v[(c + 1) & 1]);
        }
      }
      tc_fence_before();
      if (ehalf == 1) cand4[erow] = make_uint4(a0, a1, a2, a3);
      group_bar(bar_id);
      if (ehalf == 0) {
        const uint4 o = cand4[erow];
        top4_insert(o.x, a0, a1, a2, a3);
        top4_insert(o.y, a0, a1, a2, a3);
        top4_insert(o.z, a0, a1, a2, a3);
        top4_insert(o.w, a0, a1, a2, a3);
        cand4[erow] = make_uint4(a0, a1, a2, a3);
      }
      group_bar(bar_id);
      if (stagger && g == 0 && !staged) {
        asm volatile("bar.arrive 3, %0;" ::"n"(2 * FZ_GT) : "memory");
        staged = true;
      }
      // ---- update: a thread pair per patch ----
      act = act && k < Kpb && !(rsq <= kEpsR32 * ysq);
      unsigned long long best = 0ull;
      float cq = 0.f;  // <a_q, r> of the chosen atom
      const uint4 ck = cand4[p];
      const uint32_t keys[4] = {ck.x, ck.y, ck.z, ck.w};
      int ci[4];
      float sc[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) ci[c] = keys[c] ? (int)(imask - (keys[c] & imask)) : -1;
      // A clear winner needs no re-score of the other three.  Each BF16 score
      // |<a^, r^>| (a^ the BF16 rounding of the unit atom, r^ of r, unit roundoff
      // 2^-8) lies within 2^-7 ||r|| of |<a, r>| / ||a||; a key's truncated low bits
      // put it at most a factor 1 + 2^(idx_bits - 23) below its score.  A top key
      // whose score leads the second (with twice that slack) by more than
      // 2^-5 ||r|| -- twice the 2^-6 the two errors can close -- is the strict FP32
      // argmax over every atom, the atom the full re-score would choose.  When a
      // whole warp's patches are clear (or done), only the winners' correlations
      // are formed, with the arithmetic of the full path (same results).
      bool clear = !act;
      const float inv0 = ci[0] >= 0 ? s_inv[ci[0]] : -1.f;
      if (act && ci[0] >= 0 && inv0 > 0.f) {
        const float s1 = __uint_as_float(keys[0] & smask), s2 = __uint_as_float(keys[1] & smask);
        const float slack = 1.f + __uint_as_float((uint32_t)(127 + idx_bits - 22) << 23);
        bool taken0 = false;
        for (int j = 0; j < k; ++j) taken0 |= (omp[j] == ci[0]);
        clear = !taken0 && s1 - s2 * slack > 0.03125f * sqrtf(rsq);
      }
      if (__all_sync(0xffffffffu, clear)) {
        const float s0 = pair_sum(half_dot(arow(ci[0] >= 0 ? ci[0] : 0), h, rv));
        if (act) {
          best = pack_key(fabsf(s0) * inv0, ci[0]);
          cq = s0;
        }
      } else {
#pragma unroll
        for (int c = 0; c < 4; ++c) sc[c] = half_dot(arow(ci[c] >= 0 ? ci[c] : 0), h, rv);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          sc[c] = pair_sum(sc[c]);
          bool taken = false;
          if (act && ci[c] >= 0)
            for (int j = 0; j < k; ++j) taken |= (omp[j] == ci[c]);
          const float inv = ci[c] >= 0 ? s_inv[ci[c]] : -1.f;
          if (act && ci[c] >= 0 && inv > 0.f && !taken) {
            const unsigned long long kk = pack_key(fabsf(sc[c]) * inv, ci[c]);
            if (kk > best) {
              best = kk;
              cq = sc[c];
            }
          }
        }
      }
      if (act && !best) {  // no eligible candidate
        act = false;
        if (h == 0) atomicAdd((unsigned long long *)&stats[1], 1ull);
      }
      const int q = act ? (int)key_idx(best) : 0;
      const float *aq = arow(q);
      const bool f32 = act && !(fl & 2);
      // Gram column V_j = <a_om_j, a_q> = G[q][om_j] (G symmetric), issued first
      float vr[FZ_KMAX];
      if (Gm) {
#pragma unroll
        for (int j = 0; j < FZ_KMAX; ++j) vr[j] = (f32 && h == 0 && j < k) ? __ldg(Gm + (int64_t)q * T + omp[j]) : 0.f;
      }
      const float aa = s_nrm[q];
      if (Gm) {
#pragma unroll
        for (int j = 0; j < FZ_KMAX; ++j)
          if (f32 && h == 0 && j < k) Vp[j] = vr[j];
      } else {
        const int kw = __reduce_max_sync(0xffffffffu, act ? k : 0);
        for (int j = 0; j < kw; ++j) {
          const bool o = f32 && j < k;
          const float vj = pair_sum(half_dot2(o ? arow(omp[j]) : aq, aq, h));
          if (o && h == 0) Vp[j] = vj;
        }
      }
      __syncwarp();
      // projection (scalar work on h == 0): w = L^{-1} V, pivot, z_k, alpha = L^{-T} z;
      // the substitutions run on registers (static indices, predicated on k) so
      // that their dependent chains hold no shared-memory round trip
      bool ok32 = false;
      if (f32 && h == 0) {
        float wv[FZ_KMAX];
        float ww = 0.f;
#pragma unroll
        for (int i = 0; i < FZ_KMAX; ++i) {
          wv[i] = 0.f;
          if (i < k) {
            float sacc = Vp[i];
#pragma unroll
            for (int j = 0; j < i; ++j) sacc = fmaf(-Lp[ftri(i) + j], wv[j], sacc);
            wv[i] = sacc * Linv[i];
            ww = fmaf(wv[i], wv[i], ww);
          }
        }
        const float d = aa - ww;
        ok32 = aa > 0.f && d >= kTauPivot * aa;
        if (ok32) {
          const float lkk = sqrtf(d), il = 1.f / lkk;
          // z_k = <u_k, y> = <a_q, r> / L_kk (r is orthogonal to the chosen atoms)
          const float zk = cq * il;
#pragma unroll
          for (int j = 0; j < FZ_KMAX; ++j)
            if (j < k) Lp[ftri(k) + j] = wv[j];
          Lp[ftri(k) + k] = lkk;
          Linv[k] = il;
          zp[k] = zk;
          // alpha_i = (z_i - sum_{j > i} L[j][i] alpha_j) / L_ii, i = k .. 0, with
          // row k of L = (w, lkk) and the earlier rows from shared memory
          float al[FZ_KMAX];
#pragma unroll
          for (int i = FZ_KMAX - 1; i >= 0; --i) {
            al[i] = 0.f;
            if (i <= k) {
              float sacc = i == k ? zk : zp[i];
#pragma unroll
              for (int j = i + 1; j < FZ_KMAX; ++j)
                if (j <= k) sacc = fmaf(-(j == k ? wv[i] : Lp[ftri(j) + i]), al[j], sacc);
              al[i] = sacc * (i == k ? il : Linv[i]);
            }
          }
          // the residual moves by A_Omega (alpha' - alpha): the differences go to
          // Vp (free once the Gram column is used)
#pragma unroll
          for (int i = 0; i < FZ_KMAX; ++i)
            if (i <= k) {
              Vp[i] = i < k ? al[i] - Wp[i] : al[i];
              Wp[i] = al[i];
            }
        } else {
          atomicAdd((unsigned long long *)&stats[0], 1ull);
        }
      }
      ok32 = __shfl_sync(0xffffffffu, ok32, lane & ~1);
      if (f32 && !ok32) fl |= 2;
      // FP64 from scratch (rare; one thread of the pair)
      const bool go64 = act && !ok32;
      if (go64 && h == 0) {
        const float *cp[FZ_KMAX + 1];
        for (int j = 0; j < k; ++j) cp[j] = arow(omp[j]);
        GrpSmem S{};
        S.W = Wp;
        S.colp = cp;
        fb_misc = csp::grp::fp64_projection(M, yrow, S, k, aq) ? 1 : 0;
        if (fb_misc)  // alpha from scratch: the residual is recomputed from y
          for (int j = 0; j <= k; ++j) Vp[j] = Wp[j];
      }
      const bool app64 = __shfl_sync(0xffffffffu, fb_misc, lane & ~1) != 0 && go64;
      const bool appended = ok32 || app64;
      if (act && f32 && !appended && h == 0) {
        // q depends on the chosen columns: alpha of the chosen ones from the factor
        for (int i = k - 1; i >= 0; --i) {
          float sacc = zp[i];
          for (int j = i + 1; j < k; ++j) sacc = fmaf(-Lp[ftri(j) + i], Wp[j], sacc);
          Wp[i] = sacc * Linv[i];
        }
      }
      if (act && !appended) {
        act = false;
        if (h == 0 && k < Kpb) atomicAdd((unsigned long long *)&stats[1], 1ull);
      }
      __syncwarp();
      // residue r = y - A_Omega alpha' = r - A_Omega (alpha' - alpha) with the
      // differences in Vp (after the FP64 solve: y - A_Omega alpha')
      if (appended && h == 0) omp[k] = q;
      __syncwarp();
      if (app64) {
#pragma unroll
        for (int t = 0; t < FZ_NCH; ++t) {
          const int m0 = 4 * (2 * t + h);
          rv[t] = m0 < M ? __ldg(reinterpret_cast<const float4 *>(yrow + m0)) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
      }
      const int kr = __reduce_max_sync(0xffffffffu, appended ? k + 1 : 0);
      for (int j = 0; j < kr; ++j) {
        if (appended && j <= k) {
          const float aj = Vp[j];
          const float4 *c4 = reinterpret_cast<const float4 *>(arow(omp[j]));
#pragma unroll
          for (int t = 0; t < FZ_NCH; ++t) {
            const float4 cc = c4[2 * t + h];
            rv[t].x = fmaf(-aj, cc.x, rv[t].x);
            rv[t].y = fmaf(-aj, cc.y, rv[t].y);
            rv[t].z = fmaf(-aj, cc.z, rv[t].z);
            rv[t].w = fmaf(-aj, cc.w, rv[t].w);
          }
        }
      }
      float r2x = 0.f, r2y = 0.f, r2z = 0.f, r2w = 0.f;  // four independent chains
#pragma unroll
      for (int t = 0; t < FZ_NCH; ++t) {
        r2x = fmaf(rv[t].x, rv[t].x, r2x);
        r2y = fmaf(rv[t].y, rv[t].y, r2y);
        r2z = fmaf(rv[t].z, rv[t].z, r2z);
        r2w = fmaf(rv[t].w, rv[t].w, r2w);
      }
      const float r2 = pair_sum((r2x + r2y) + (r2z + r2w));
      if (appended) {
        rsq = r2;
        ++k;
        if (k >= Kpb || rsq <= kEpsR32 * ysq) {
          if (h == 0 && k < Kpb) atomicAdd((unsigned long long *)&stats[1], 1ull);
          act = false;
        }
      }
      // next proxy input (the MMA of this iteration has retired: accfull fired)
      store_rbf(r_bf, p, h, rv);
    }
    if (stagger && g == 0 && !staged) asm volatile("bar.arrive 3, %0;" ::"n"(2 * FZ_GT) : "memory");
    if (valid) {
      if (h == 0) k_eff[b] = (int8_t)k;
      for (int j = h; j < ldo; j += 2) {
        omega[b * ldo + j] = j < k ? omp[j] : -1;
        alpha[b * ldo + j] = j < k ? Wp[j] : 0.f;
      }
    }
  }
  if (threadIdx.x == 0) mbar_drain(afull, 0);  // no TMA write outlives the CTA
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols * NGRP) : "memory");
}

int device_sms() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 1;
  }
  return sms;
}

}  // namespace

bool fused_top_supported(int M, int T, int Kb) {
  // T a multiple of 64: each epilogue half reads whole 32-column TMEM blocks
  return M > 0 && M <= FZ_MP && M % 4 == 0 && T >= 64 && T <= 256 && T % 64 == 0 && Kb >= 1 && Kb <= FZ_KMAX &&
         fz_layout(T, Kb, 1).total <= 227 * 1024;
}

int64_t fused_wave_patches(int T, int Kb) {
  const int ngrp = fz_layout(T, Kb, 2).total <= 227 * 1024 ? 2 : 1;
  return (int64_t)device_sms() * ngrp * FZ_M;
}

bool launch_omp_fused_tc(const float *Y, int M, const float *const *A, const float *const *inv_norm,
                         const __nv_bfloat16 *const *Abf, const float *const *gram, int nph, const int64_t *phase_start, int Mp, int T,
                         const int32_t *ids, int64_t n, const int8_t *Kp, int Kuni, int Kb, int32_t *omega,
                         float *alpha, int ldo, int8_t *k_eff, int64_t *stats, unsigned long long *err,
                         cudaStream_t s) {
  if (n == 0) return true;
  if (Mp != FZ_MP || nph < 1 || nph > FZ_MAXPH || !fused_top_supported(M, T, Kb)) return false;
  FzArgs args;
  memset(&args, 0, sizeof(args));
  args.nph = nph;
  int64_t tiles = 0;
  for (int ph = 0; ph <= nph; ++ph) args.row0[ph] = phase_start ? phase_start[ph] : (ph ? n : 0);
  for (int ph = 0; ph < nph; ++ph) tiles += (args.row0[ph + 1] - args.row0[ph] + FZ_M - 1) / FZ_M;
  // two tiles per CTA (sharing the atoms) once there are more tiles than SMs
  const int ngrp = (tiles > device_sms() && fz_layout(T, Kb, 2).total <= 227 * 1024) ? 2 : 1;
  int64_t ctas = 0;
  for (int ph = 0; ph < nph; ++ph) {
    if (!tc_make_map_bf16(&args.map[ph], Abf[ph], (uint64_t)Mp, (uint64_t)T, (uint32_t)T)) return false;
    args.A[ph] = A[ph];
    args.inv[ph] = inv_norm[ph];
    args.G[ph] = gram ? gram[ph] : nullptr;
    args.cta0[ph] = (int)ctas;
    const int64_t t = (args.row0[ph + 1] - args.row0[ph] + FZ_M - 1) / FZ_M;
    ctas += (t + ngrp - 1) / ngrp;
  }
  args.cta0[nph] = (int)ctas;
  if (ctas == 0) return true;
  if (ctas > INT32_MAX) return false;
  int idx_bits = 1;
  while ((1 << idx_bits) < T) ++idx_bits;
  const int sm = fz_layout(T, Kb, ngrp).total;
  auto kern = ngrp == 2 ? omp_fused_tc_kernel<2> : omp_fused_tc_kernel<1>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, sm) != cudaSuccess) return false;
  // highest stream priority: when a restricted level runs beside it (pipelined
  // solve), whole SMs go to this kernel's CTAs first
  int lo = 0, hi = 0;
  cudaDeviceGetStreamPriorityRange(&lo, &hi);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)ctas);
  cfg.blockDim = dim3(ngrp * FZ_GT);
  cfg.dynamicSmemBytes = (size_t)sm;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributePriority;
  attr[0].val.priority = hi;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, args, Y, M, T, idx_bits, ids, Kp, Kuni, Kb, omega, alpha, ldo, k_eff, stats,
                            err) == cudaSuccess;
}

}  // namespace csp
