// Fused full-dictionary OMP for a small shared dictionary: every iteration of
// Algorithm 1 (proxy, merge, projection, residue) for a tile of 128 patches in
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
// The FP32 rows of A (zero padded to 64) stay in shared memory, so the
// re-score, the Gram column and the residue read no global memory.
//
// Roles: warp 0 loads the BF16 atoms by TMA, warp 1 owns the tensor memory and
// issues the MMAs, warps 2-9 run the epilogue (TMEM lane quadrant = warp % 4,
// half of the columns each) and then the update (thread pair per patch).
// Every mbarrier wait is bounded; on expiry the error word is set, all threads
// leave the iteration loop together, and the tensor memory is freed.
#include "csp_internal.cuh"
#include "grp_common.cuh"
#include "tc_common.cuh"

namespace csp {

namespace {

using namespace csp::tc;
using csp::grp::GrpSmem;
using csp::grp::key_idx;
using csp::grp::pack_key;

constexpr int FZ_M = 128;        // patches per CTA (MMA M)
constexpr int FZ_MP = 64;        // padded measurement dimension (one 128-byte K block)
constexpr int FZ_KMAX = 8;       // largest K of the fused form
constexpr int FZ_THREADS = 320;  // warps 0-1 + eight epilogue/update warps
constexpr int FZ_HALF = FZ_MP / 2;  // elements per thread of a pair
constexpr int FZ_NCH = FZ_HALF / 4;  // float4 per thread of a pair

__host__ __device__ constexpr int ftri(int i) { return i * (i + 1) / 2; }

struct FzLayout {
  int a_bf;    // BF16 atoms [T][64], 128-byte swizzle (offset 0, 1024-aligned)
  int r_bf;    // BF16 residual tile [128][64]
  int a_fp;    // FP32 atoms [T][64]
  int inv;     // [T] 1/||a_i||
  int L, Linv, z, V, W;  // per patch, FP32
  int om, colp, cand;    // per patch
  int bars;
  int total;
};

__host__ __device__ inline FzLayout fz_layout(int T) {
  FzLayout L;
  int o = 0;
  L.a_bf = o; o += T * FZ_MP * 2;
  L.r_bf = o; o += FZ_M * FZ_MP * 2;
  L.a_fp = o; o += T * FZ_MP * 4;
  L.inv = o; o += T * 4;
  L.L = o; o += FZ_M * ftri(FZ_KMAX) * 4;
  L.Linv = o; o += FZ_M * FZ_KMAX * 4;
  L.z = o; o += FZ_M * FZ_KMAX * 4;
  L.V = o; o += FZ_M * (FZ_KMAX + 1) * 4;
  L.W = o; o += FZ_M * (FZ_KMAX + 1) * 4;
  L.om = o; o += FZ_M * FZ_KMAX * 4;
  o = (o + 15) & ~15;
  L.colp = o; o += FZ_M * (FZ_KMAX + 1) * 8;
  L.cand = o; o += FZ_M * 4 * 4;
  L.bars = o; o += 64;
  L.total = o + 1024;  // alignment slack
  return L;
}

__device__ __forceinline__ float pair_sum(float v) { return v + __shfl_xor_sync(0xffffffffu, v, 1); }

// Partial dot of this thread's half of a 64-wide row (shared or global memory)
// with its register chunks.
__device__ __forceinline__ float half_dot(const float *row, int h, const float4 (&v)[FZ_NCH]) {
  const float4 *r4 = reinterpret_cast<const float4 *>(row + h * FZ_HALF);
  float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;  // four independent chains
#pragma unroll
  for (int t = 0; t < FZ_NCH; ++t) {
    const float4 a = r4[t];
    s0 = fmaf(a.x, v[t].x, s0);
    s1 = fmaf(a.y, v[t].y, s1);
    s2 = fmaf(a.z, v[t].z, s2);
    s3 = fmaf(a.w, v[t].w, s3);
  }
  return (s0 + s1) + (s2 + s3);
}

// BF16 copy of this thread's half of the residual into row `row` of the
// 128-byte-swizzled tile (16-byte chunk c of a row sits at chunk c ^ (row % 8)).
__device__ __forceinline__ void store_rbf(uint8_t *tile, int row, int h, const float4 (&r)[FZ_NCH]) {
#pragma unroll
  for (int q = 0; q < FZ_NCH / 2; ++q) {  // 8 elements per 16-byte chunk
    const int c = h * (FZ_NCH / 2) + q;
    const float4 a = r[2 * q], b = r[2 * q + 1];
    __nv_bfloat162 w0 = __floats2bfloat162_rn(a.x, a.y), w1 = __floats2bfloat162_rn(a.z, a.w);
    __nv_bfloat162 w2 = __floats2bfloat162_rn(b.x, b.y), w3 = __floats2bfloat162_rn(b.z, b.w);
    uint4 u;
    u.x = *reinterpret_cast<uint32_t *>(&w0);
    u.y = *reinterpret_cast<uint32_t *>(&w1);
    u.z = *reinterpret_cast<uint32_t *>(&w2);
    u.w = *reinterpret_cast<uint32_t *>(&w3);
    *reinterpret_cast<uint4 *>(tile + row * 128 + ((c ^ (row & 7)) << 4)) = u;
  }
}

__global__ void __launch_bounds__(FZ_THREADS, 1)
omp_fused_tc_kernel(const __grid_constant__ CUtensorMap tmA, const float *__restrict__ Y, int M,
                    const float *__restrict__ A, const float *__restrict__ inv_norm, int T, int idx_bits,
                    const int32_t *__restrict__ ids, int64_t n, const int8_t *__restrict__ Kp, int Kuni, int Kb,
                    int32_t *__restrict__ omega, float *__restrict__ alpha, int ldo, int8_t *__restrict__ k_eff,
                    int64_t *stats, unsigned long long *err) {
  extern __shared__ uint8_t fz_raw[];
  uint8_t *sm = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(fz_raw) + 1023) & ~uintptr_t(1023));
  const FzLayout lay = fz_layout(T);
  uint8_t *a_bf = sm + lay.a_bf;
  uint8_t *r_bf = sm + lay.r_bf;
  float *a_fp = reinterpret_cast<float *>(sm + lay.a_fp);
  float *s_inv = reinterpret_cast<float *>(sm + lay.inv);
  uint64_t *bars = reinterpret_cast<uint64_t *>(sm + lay.bars);
  uint64_t *afull = bars, *rready = bars + 1, *accfull = bars + 2;
  uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(bars + 4);
  int *s_flag = reinterpret_cast<int *>(bars + 5);
  uint32_t *cand = reinterpret_cast<uint32_t *>(sm + lay.cand);  // [128][4] keys (half 1 merges in)

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t tile0 = (int64_t)blockIdx.x * FZ_M;
  uint32_t ncols = 32;
  while ((int)ncols < T) ncols <<= 1;

  if (threadIdx.x == 0) {
    mbar_init(afull, 1);
    mbar_init(rready, 1);
    mbar_init(accfull, 1);
    *s_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_holder)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  // FP32 atoms (zero padded to 64) and inverse norms, cooperatively
  for (int e = threadIdx.x; e < T * FZ_MP; e += blockDim.x) {
    const int i = e / FZ_MP, m = e - i * FZ_MP;
    a_fp[e] = m < M ? __ldg(A + (int64_t)i * M + m) : 0.f;
  }
  for (int i = threadIdx.x; i < T; i += blockDim.x) s_inv[i] = __ldg(inv_norm + i);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_holder;

  if (warp == 0) {
    if (lane == 0) {
      mbar_expect_tx(afull, (uint32_t)(T * 128));
      tma_load_2d(a_bf, &tmA, 0, 0, afull);
      mbar_wait(afull, 0, err, 11);  // drain before exit
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = instr_desc(FZ_M, T);
      bool ok = mbar_wait(afull, 0, err, 12);
      for (int it = 0; it < Kb && ok; ++it) {
        ok = mbar_wait(rready, (uint32_t)(it & 1), err, 13);
        if (!ok) break;
        tc_fence_after();
#pragma unroll
        for (int kin = 0; kin < 4; ++kin) {
          const uint64_t ad = smem_desc(smem_u32(r_bf) + kin * 32);
          const uint64_t bd = smem_desc(smem_u32(a_bf) + kin * 32);
          mma_bf16(tmem, ad, bd, idesc, kin ? 1u : 0u);
        }
        mma_commit(accfull);
      }
    }
  } else {
    // ---- epilogue / update threads (256) ----
    const int u = threadIdx.x - 64;
    const int p = u >> 1, h = u & 1;  // update: patch p, half h
    const int quad = warp & 3, ehalf = (warp - 2) >> 2, erow = quad * 32 + lane;  // epilogue row
    const int64_t wi = tile0 + p;
    const bool valid = wi < n;
    const int64_t b = valid ? (ids ? (int64_t)ids[wi] : wi) : 0;
    int Kpb = valid ? (Kp ? (int)Kp[b] : Kuni) : 0;
    Kpb = Kpb < Kb ? Kpb : Kb;
    float *Lp = reinterpret_cast<float *>(sm + lay.L) + p * ftri(FZ_KMAX);
    float *Linv = reinterpret_cast<float *>(sm + lay.Linv) + p * FZ_KMAX;
    float *zp = reinterpret_cast<float *>(sm + lay.z) + p * FZ_KMAX;
    float *Vp = reinterpret_cast<float *>(sm + lay.V) + p * (FZ_KMAX + 1);
    float *Wp = reinterpret_cast<float *>(sm + lay.W) + p * (FZ_KMAX + 1);
    int *omp = reinterpret_cast<int *>(sm + lay.om) + p * FZ_KMAX;
    const float **colp = reinterpret_cast<const float **>(sm + lay.colp) + p * (FZ_KMAX + 1);
    GrpSmem S{};  // view for the FP64 rebuild
    S.L = Lp;
    S.Linv = Linv;
    S.z = zp;
    S.V = Vp;
    S.W = Wp;
    S.om = omp;
    S.colp = colp;
    int fb_misc = 0;
    // y and r: this thread's half, zero padded
    const float *yrow = Y + b * M;
    float4 yv[FZ_NCH], rv[FZ_NCH];
#pragma unroll
    for (int t = 0; t < FZ_NCH; ++t) {
      float e4[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int m = h * FZ_HALF + 4 * t + c;
        e4[c] = (valid && m < M) ? __ldg(yrow + m) : 0.f;
      }
      yv[t] = make_float4(e4[0], e4[1], e4[2], e4[3]);
      rv[t] = yv[t];
    }
    float ysq = 0.f;
#pragma unroll
    for (int t = 0; t < FZ_NCH; ++t)
      ysq = fmaf(yv[t].x, yv[t].x, fmaf(yv[t].y, yv[t].y, fmaf(yv[t].z, yv[t].z, fmaf(yv[t].w, yv[t].w, ysq))));
    ysq = pair_sum(ysq);
    float rsq = ysq;
    int k = 0;
    uint8_t fl = 0;  // bit 1: FP64 from here on
    bool act = valid && Kpb > 0;
    store_rbf(r_bf, p, h, rv);
    const uint32_t imask = (1u << idx_bits) - 1u;
    const uint32_t smask = 0x7fffffffu & ~imask;
    const int hcols = T / 2;
    for (int it = 0; it < Kb; ++it) {
      // the residual tile is complete: hand it to the MMA
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("bar.sync 1, 256;" ::: "memory");
      if (u == 0) mbar_arrive(rready);
      // ---- epilogue: top 4 keys of this row's half of the columns ----
      bool ok = mbar_wait(accfull, (uint32_t)(it & 1), err, 14);
      if (!ok) *s_flag = 1;
      asm volatile("bar.sync 1, 256;" ::: "memory");
      if (*s_flag) break;
      tc_fence_after();
      uint32_t a0 = 0, a1 = 0, a2 = 0, a3 = 0, b0 = 0, b1 = 0, b2 = 0, b3 = 0;  // two independent chains
      for (int c0 = 0; c0 < hcols; c0 += 32) {
        uint32_t v[32];
        tmem_ld32_nowait(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(ehalf * hcols + c0), v);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        const int base = ehalf * hcols + c0;  // T is a multiple of 64: every column is an atom
        const uint32_t cb = imask - (uint32_t)base;
#pragma unroll
        for (int i = 0; i < 32; i += 2) {
          top4_insert((v[i] & smask) | (cb - (uint32_t)i), a0, a1, a2, a3);
          top4_insert((v[i + 1] & smask) | (cb - (uint32_t)(i + 1)), b0, b1, b2, b3);
        }
      }
      top4_insert(b0, a0, a1, a2, a3);
      top4_insert(b1, a0, a1, a2, a3);
      top4_insert(b2, a0, a1, a2, a3);
      top4_insert(b3, a0, a1, a2, a3);
      tc_fence_before();
      if (ehalf == 1) {
        cand[erow * 4 + 0] = a0;
        cand[erow * 4 + 1] = a1;
        cand[erow * 4 + 2] = a2;
        cand[erow * 4 + 3] = a3;
      }
      asm volatile("bar.sync 1, 256;" ::: "memory");
      if (ehalf == 0) {
        for (int q = 0; q < 4; ++q) top4_insert(cand[erow * 4 + q], a0, a1, a2, a3);
        cand[erow * 4 + 0] = a0;
        cand[erow * 4 + 1] = a1;
        cand[erow * 4 + 2] = a2;
        cand[erow * 4 + 3] = a3;
      }
      asm volatile("bar.sync 1, 256;" ::: "memory");
      // ---- update: a thread pair per patch ----
      act = act && k < Kpb && !(rsq <= kEpsR32 * ysq);
      unsigned long long best = 0ull;
      int ci[4];
      float sc[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const uint32_t key = cand[p * 4 + c];
        ci[c] = key ? (int)(imask - (key & imask)) : -1;
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) sc[c] = half_dot(a_fp + (ci[c] >= 0 ? ci[c] : 0) * FZ_MP, h, rv);
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        sc[c] = pair_sum(sc[c]);
        bool taken = false;
        if (act && ci[c] >= 0)
          for (int j = 0; j < k; ++j) taken |= (omp[j] == ci[c]);
        const float inv = ci[c] >= 0 ? s_inv[ci[c]] : -1.f;
        if (act && ci[c] >= 0 && inv > 0.f && !taken) {
          const unsigned long long kk = pack_key(fabsf(sc[c]) * inv, ci[c]);
          best = kk > best ? kk : best;
        }
      }
      if (act && !best) {  // no eligible candidate
        act = false;
        if (h == 0) atomicAdd((unsigned long long *)&stats[1], 1ull);
      }
      const int q = act ? (int)key_idx(best) : 0;
      const float *aq = a_fp + q * FZ_MP;
      float4 av[FZ_NCH];
#pragma unroll
      for (int t = 0; t < FZ_NCH; ++t) av[t] = reinterpret_cast<const float4 *>(aq + h * FZ_HALF)[t];
      const float aa = pair_sum(half_dot(aq, h, av));
      const float bq = pair_sum(half_dot(aq, h, yv));
      const bool f32 = act && !(fl & 2);
      // Gram column V_j = <a_om_j, a_q>
      const int kw = __reduce_max_sync(0xffffffffu, act ? k : 0);
      for (int j = 0; j < kw; ++j) {
        const bool o = f32 && j < k;
        const float vj = pair_sum(half_dot(o ? colp[j] : aq, h, av));
        if (o && h == 0) Vp[j] = vj;
      }
      __syncwarp();
      // projection (scalar work on h == 0): w = L^{-1} V, pivot, z_k, alpha = L^{-T} z
      bool ok32 = false;
      if (f32 && h == 0) {
        float ww = 0.f, wz = 0.f;
        for (int i = 0; i < k; ++i) {
          float s = Vp[i];
          for (int j = 0; j < i; ++j) s = fmaf(-Lp[ftri(i) + j], Wp[j], s);
          const float w = s * Linv[i];
          Wp[i] = w;
          ww = fmaf(w, w, ww);
          wz = fmaf(w, zp[i], wz);
        }
        const float d = aa - ww;
        ok32 = aa > 0.f && d >= kTauPivot * aa;
        if (ok32) {
          const float lkk = sqrtf(d), il = 1.f / lkk;
          for (int j = 0; j < k; ++j) Lp[ftri(k) + j] = Wp[j];
          Lp[ftri(k) + k] = lkk;
          Linv[k] = il;
          zp[k] = (bq - wz) * il;
          for (int i = k; i >= 0; --i) {
            float s = zp[i];
            for (int j = i + 1; j <= k; ++j) s = fmaf(-Lp[ftri(j) + i], Wp[j], s);
            Wp[i] = s * Linv[i];
          }
        } else {
          atomicAdd((unsigned long long *)&stats[0], 1ull);
        }
      }
      ok32 = __shfl_sync(0xffffffffu, ok32, lane & ~1);
      if (f32 && !ok32) fl |= 2;
      // FP64 from scratch (rare; one thread of the pair)
      const bool go64 = act && !ok32;
      if (go64 && h == 0) fb_misc = csp::grp::fp64_projection(M, yrow, S, k, aq) ? 1 : 0;
      const bool app64 = __shfl_sync(0xffffffffu, fb_misc, lane & ~1) != 0 && go64;
      const bool appended = ok32 || app64;
      if (act && f32 && !appended && h == 0) {
        // q depends on the chosen columns: alpha of the chosen ones from the factor
        for (int i = k - 1; i >= 0; --i) {
          float s = zp[i];
          for (int j = i + 1; j < k; ++j) s = fmaf(-Lp[ftri(j) + i], Wp[j], s);
          Wp[i] = s * Linv[i];
        }
      }
      if (act && !appended) {
        act = false;
        if (h == 0 && k < Kpb) atomicAdd((unsigned long long *)&stats[1], 1ull);
      }
      __syncwarp();
      // residue r = y - A_Omega alpha
      if (appended && h == 0) {
        omp[k] = q;
        colp[k] = aq;
      }
      __syncwarp();
      const int kr = __reduce_max_sync(0xffffffffu, appended ? k + 1 : 0);
      if (appended) {
#pragma unroll
        for (int t = 0; t < FZ_NCH; ++t) rv[t] = yv[t];
      }
      for (int j = 0; j < kr; ++j) {
        if (appended && j <= k) {
          const float aj = Wp[j];
          const float4 *c4 = reinterpret_cast<const float4 *>(colp[j] + h * FZ_HALF);
#pragma unroll
          for (int t = 0; t < FZ_NCH; ++t) {
            const float4 cc = c4[t];
            rv[t].x = fmaf(-aj, cc.x, rv[t].x);
            rv[t].y = fmaf(-aj, cc.y, rv[t].y);
            rv[t].z = fmaf(-aj, cc.z, rv[t].z);
            rv[t].w = fmaf(-aj, cc.w, rv[t].w);
          }
        }
      }
      float r2 = 0.f;
#pragma unroll
      for (int t = 0; t < FZ_NCH; ++t)
        r2 = fmaf(rv[t].x, rv[t].x, fmaf(rv[t].y, rv[t].y, fmaf(rv[t].z, rv[t].z, fmaf(rv[t].w, rv[t].w, r2))));
      r2 = pair_sum(r2);
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
    if (valid) {
      if (h == 0) k_eff[b] = (int8_t)k;
      for (int j = h; j < ldo; j += 2) {
        omega[b * ldo + j] = j < k ? omp[j] : -1;
        alpha[b * ldo + j] = j < k ? Wp[j] : 0.f;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
}

}  // namespace

bool fused_top_supported(int M, int T, int Kb) {
  // T a multiple of 64: each epilogue half reads whole 32-column TMEM blocks
  return M > 0 && M <= FZ_MP && M % 4 == 0 && T >= 64 && T <= 256 && T % 64 == 0 && Kb >= 1 && Kb <= FZ_KMAX &&
         fz_layout(T).total <= 227 * 1024;
}

bool launch_omp_fused_tc(const float *Y, int M, const float *A, const float *inv_norm, const __nv_bfloat16 *Abf,
                         int Mp, int T, const int32_t *ids, int64_t n, const int8_t *Kp, int Kuni, int Kb,
                         int32_t *omega, float *alpha, int ldo, int8_t *k_eff, int64_t *stats,
                         unsigned long long *err, cudaStream_t s) {
  if (n == 0) return true;
  if (Mp != FZ_MP || !fused_top_supported(M, T, Kb)) return false;
  CUtensorMap mA;
  if (!tc_make_map_bf16(&mA, Abf, (uint64_t)Mp, (uint64_t)T, (uint32_t)T)) return false;
  const int sm = fz_layout(T).total;
  if (cudaFuncSetAttribute(omp_fused_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, sm) != cudaSuccess)
    return false;
  int idx_bits = 1;
  while ((1 << idx_bits) < T) ++idx_bits;
  const unsigned grid = (unsigned)((n + FZ_M - 1) / FZ_M);
  omp_fused_tc_kernel<<<grid, FZ_THREADS, sm, s>>>(mA, Y, M, A, inv_norm, T, idx_bits, ids, n, Kp, Kuni, Kb, omega,
                                                   alpha, ldo, k_eff, stats, err);
  return true;
}

}  // namespace csp
