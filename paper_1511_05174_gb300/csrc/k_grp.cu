// Lane-group OMP kernels organised in load waves.
//
// The per-patch work of OMP (Sec. II-B, Algorithm 1: merge, projection,
// residue; the finer steps of Algorithm 2) is latency-bound: every step waits
// for rows of the effective dictionary that sit in L2.  These kernels issue all
// loads a step needs together, before any of them is used, so that a patch
// waits for a handful of memory round trips per iteration instead of one per
// row:
//   omp_update_wave_kernel   one iteration of every patch of a full-dictionary
//                            level (after the proxy kernel): re-score the
//                            proxy's candidates in FP32, project, update r;
//   omp_restricted_gram_kernel  all iterations of the restricted OMP over the
//                            children f(Omega_up): the proxy over the candidates
//                            is c_i = <a_i, y> - sum_j alpha_j G[i][omega_j]
//                            from the level's Gram matrix G = A A^T (entries
//                            cached per candidate in shared memory), its best
//                            three are re-scored exactly against the explicit
//                            residual, so the selection follows the FP32 proxy.
// Both use the incremental Cholesky projection of grp_project (FP32, rebuilt
// in FP64 when the pivot ratio falls below kTauPivot).
#include "csp_internal.cuh"
#include "grp_common.cuh"

namespace csp {

namespace {

using namespace csp::grp;

constexpr int WV_WARPS = 4;
constexpr int RB = 4;  // residual rows per load wave

// Projection step given the Gram column S.V[0..k-1] = <a_{om_j}, a_q>, the
// chunks of a_q, aa = ||a_q||^2 and bq = <a_q, y>.  S.colp[0..k-1] point at the
// chosen rows (global).  On success alpha is in S.W[0..k], r and rsq are
// updated, S.om[k] = q, S.colp[k] = aqp, and the FP32 factor gained row k.
// Returns whether q was appended.  Warp-collective.
template <int G, int NCH>
__device__ bool grp_project(bool act, int s, int M, const float *aqp, const float *__restrict__ yrow, int q, int k,
                            const float4 (&aq)[NCH], float aa, float bq, const float4 (&yv)[NCH], float4 (&rv)[NCH],
                            const GrpSmem &S, uint8_t &fl, float &rsq, int64_t *stats) {
  const int nv = M >> 2;
  const int kw = __reduce_max_sync(kFull, act ? k : 0);
  const bool f32 = act && !(fl & 2);
  // W = L^{-1} V, column-oriented: step i finalises W_i and updates V_j, j > i
  for (int i = 0; i < kw; ++i) {
    if (f32 && i < k) {
      const float wi = S.V[i] * S.Linv[i];
      if (s == 0) S.W[i] = wi;
      for (int j = i + 1 + s; j < k; j += G) S.V[j] = fmaf(-S.L[tri(j) + i], wi, S.V[j]);
    }
    __syncwarp();
  }
  float ww = 0.f, zz = 0.f;
  if (f32)
    for (int j = s; j < k; j += G) {
      ww = fmaf(S.W[j], S.W[j], ww);
      zz = fmaf(S.W[j], S.z[j], zz);
    }
  ww = gsum<G>(ww);
  zz = gsum<G>(zz);
  const float d = aa - ww;
  const bool ok32 = f32 && aa > 0.f && d >= kTauPivot * aa;
  if (f32 && !ok32) {
    fl |= 2;
    if (s == 0 && stats) atomicAdd((unsigned long long *)&stats[0], 1ull);
  }
  if (ok32) {
    const float lkk = sqrtf(d), il = 1.f / lkk;
    for (int j = s; j < k; j += G) S.L[tri(k) + j] = S.W[j];
    if (s == 0) {
      S.L[tri(k) + k] = lkk;
      S.Linv[k] = il;
      S.z[k] = (bq - zz) * il;
    }
  }
  __syncwarp();
  if (ok32)
    for (int i = s; i <= k; i += G) S.V[i] = S.z[i];
  __syncwarp();
  for (int j = kw; j >= 0; --j) {
    if (ok32 && j <= k) {
      const float aj = S.V[j] * S.Linv[j];
      if (s == 0) S.W[j] = aj;
      for (int i = s; i < j; i += G) S.V[i] = fmaf(-S.L[tri(j) + i], aj, S.V[i]);
    }
    __syncwarp();
  }
  const bool go64 = act && !ok32;
  if (go64 && s == 0) S.misc[0] = fp64_projection(M, yrow, S, k, aqp) ? 1 : 0;
  __syncwarp();
  const bool appended = ok32 || (go64 && S.misc[0] != 0);
  // residue r = y - A_Omega alpha, RB chosen rows per load wave
  if (appended) {
    const float ak = S.W[k];
#pragma unroll
    for (int t = 0; t < NCH; ++t) {
      rv[t].x = fmaf(-ak, aq[t].x, yv[t].x);
      rv[t].y = fmaf(-ak, aq[t].y, yv[t].y);
      rv[t].z = fmaf(-ak, aq[t].z, yv[t].z);
      rv[t].w = fmaf(-ak, aq[t].w, yv[t].w);
    }
  }
  for (int j0 = 0; j0 < kw; j0 += RB) {
    float4 c[RB][NCH];
#pragma unroll
    for (int u = 0; u < RB; ++u) {
      const bool o = appended && j0 + u < k;
      load_chunks<G, NCH>(c[u], o ? S.colp[j0 + u] : aqp, nv, s, o);
    }
#pragma unroll
    for (int u = 0; u < RB; ++u) {
      if (appended && j0 + u < k) {
        const float aj = S.W[j0 + u];
#pragma unroll
        for (int t = 0; t < NCH; ++t) {
          rv[t].x = fmaf(-aj, c[u][t].x, rv[t].x);
          rv[t].y = fmaf(-aj, c[u][t].y, rv[t].y);
          rv[t].z = fmaf(-aj, c[u][t].z, rv[t].z);
          rv[t].w = fmaf(-aj, c[u][t].w, rv[t].w);
        }
      }
    }
  }
  const float r2 = gsum<G>(dotc<NCH>(rv, rv));
  if (appended) {
    rsq = r2;
    if (s == 0) {
      S.om[k] = q;
      S.colp[k] = aqp;
    }
  }
  __syncwarp();
  return appended;
}

// ---------------------------------------------------------------------------
// One OMP iteration of every patch of a full-dictionary level.
// ---------------------------------------------------------------------------
template <int G, int NCH>
__global__ void __launch_bounds__(WV_WARPS * 32)
omp_update_wave_kernel(const float *__restrict__ Y, int M, const float *__restrict__ A,
                       const float *__restrict__ inv_norm, const int32_t *__restrict__ ids, int64_t n,
                       int64_t rbf_row0, int n_cand, const int8_t *__restrict__ Kp, int Kuni, OmpState st,
                       int64_t *stats, const float *__restrict__ gram, int T, int64_t a_pstride,
                       int64_t inv_pstride) {
  constexpr int NG = 32 / G;
  constexpr int KPL = (CSP_MAX_K + G - 1) / G;  // chosen-atom entries per lane
  extern __shared__ __align__(16) char smem_raw[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, s = lane & (G - 1), g = lane / G;
  const int64_t wbase = ((int64_t)blockIdx.x * WV_WARPS + wib) * NG;
  if (wbase >= n) return;  // whole warp
  const int64_t wi = wbase + g;
  const bool valid = wi < n;
  const GrpSmem S = carve(smem_raw + (size_t)(wib * NG + g) * grp_smem_bytes(st.Kb, 0), st.Kb, 0);
  const int nv = M >> 2;
  const int64_t b = valid ? (ids ? __ldg(ids + wi) : wi) : 0;
  A += b * a_pstride;            // per-patch effective dictionary (stride 0: shared)
  inv_norm += b * inv_pstride;
  // wave: per-patch state
  uint8_t fl = valid ? st.flags[b] : 1;
  const int k = valid ? st.k_eff[b] : 0;
  int Kpb = valid ? (Kp ? (int)Kp[b] : Kuni) : 0;
  Kpb = Kpb < st.Kb ? Kpb : st.Kb;
  int32_t *om_g = st.omega + b * st.ldo;
  float *L_g = st.Lpk + b * tri(st.Kb);
  float *z_g = st.z + b * st.Kb;
  const float *yrow = Y + b * M;
  float4 yv[NCH], rv[NCH];
  load_chunks<G, NCH>(yv, yrow, nv, s, valid);
  load_chunks<G, NCH>(rv, st.R + b * M, nv, s, valid);
  int candr[kTopP];
#pragma unroll
  for (int c = 0; c < kTopP; ++c) {
    // a candidate outside [0, T) (never written by an aborted proxy) is no candidate
    const int cv = (valid && c < n_cand) ? st.cand[b * kTopP + c] : -1;
    candr[c] = (cv >= 0 && cv < T) ? cv : -1;
  }
  int omr[KPL];
  float zr[KPL];
#pragma unroll
  for (int t = 0; t < KPL; ++t) {
    const int j = s + G * t;
    const bool o = valid && j < st.Kb;
    omr[t] = o ? om_g[j] : 0;
    zr[t] = o ? z_g[j] : 0.f;
  }
  bool act = !(fl & 1) && k < Kpb;
  if (valid && !(fl & 1) && k >= Kpb && s == 0) st.flags[b] = fl | 1;
  const float ysq = gsum<G>(dotc<NCH>(yv, yv));
  const float rsq0 = gsum<G>(dotc<NCH>(rv, rv));
  if (act && rsq0 <= kEpsR32 * ysq) {
    act = false;
    if (s == 0) { st.flags[b] = fl | 1; atomicAdd((unsigned long long *)&stats[1], 1ull); }
  }
#pragma unroll
  for (int t = 0; t < KPL; ++t) {
    const int j = s + G * t;
    if (act && j < k) {
      S.om[j] = omr[t];
      S.colp[j] = A + (int64_t)omr[t] * M;
      S.z[j] = zr[t];
    }
  }
  // wave: candidate rows, their norms, the factor
  float4 cr[kTopP][NCH];
  float invr[kTopP];
#pragma unroll
  for (int c = 0; c < kTopP; ++c) {
    const bool o = act && candr[c] >= 0;
    load_chunks<G, NCH>(cr[c], A + (int64_t)(o ? candr[c] : 0) * M, nv, s, o);
    invr[c] = o ? __ldg(inv_norm + candr[c]) : -1.f;
  }
  const bool f32 = act && !(fl & 2);
  const int tk = tri(k), kw = __reduce_max_sync(kFull, act ? k : 0);
  for (int e0 = s; e0 < tri(kw); e0 += 8 * G) {
    float lr[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = e0 + u * G;
      lr[u] = (f32 && e < tk) ? L_g[e] : 0.f;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = e0 + u * G;
      if (f32 && e < tk) S.L[e] = lr[u];
    }
  }
  __syncwarp();
  if (f32)
    for (int j = s; j < k; j += G) S.Linv[j] = 1.f / S.L[tri(j) + j];
  // choose q: the proxy's argmax, or the best FP32 re-score of its candidates
  int q = -1, qc = 0;
  if (n_cand <= 1) {
    q = act ? candr[0] : -1;
  } else {
    unsigned long long best = 0ull;
#pragma unroll
    for (int c = 0; c < kTopP; ++c) {
      bool dup = false;
      if (act && candr[c] >= 0)
        for (int j = s; j < k; j += G) dup |= (S.om[j] == candr[c]);
      const unsigned bal = __ballot_sync(kFull, dup);
      const bool taken = ((bal >> (g * G)) & ((G == 32) ? 0xffffffffu : ((1u << G) - 1u))) != 0u;
      const float sc = gsum<G>(dotc<NCH>(cr[c], rv));
      if (act && candr[c] >= 0 && invr[c] > 0.f && !taken) {
        const unsigned long long key = pack_key(fabsf(sc) * invr[c], candr[c]);
        if (key > best) { best = key; qc = c; }
      }
    }
    q = best ? key_idx(best) : -1;
  }
  if (act && q < 0) {
    act = false;
    if (s == 0) { st.flags[b] = fl | 1; atomicAdd((unsigned long long *)&stats[1], 1ull); }
  }
  float4 aq[NCH];
#pragma unroll
  for (int t = 0; t < NCH; ++t) {
    aq[t] = cr[0][t];
#pragma unroll
    for (int c = 1; c < kTopP; ++c)
      if (qc == c) aq[t] = cr[c][t];
  }
  const float aa = gsum<G>(dotc<NCH>(aq, aq));
  const float bq = gsum<G>(dotc<NCH>(aq, yv));
  // wave: Gram column
  const bool f32b = act && !(fl & 2);
  if (gram) {
    float vr[KPL];
#pragma unroll
    for (int t = 0; t < KPL; ++t) {
      const int j = s + G * t;
      vr[t] = (f32b && j < k) ? __ldg(gram + (int64_t)q * T + omr[t]) : 0.f;  // row q (G symmetric)
    }
#pragma unroll
    for (int t = 0; t < KPL; ++t) {
      const int j = s + G * t;
      if (f32b && j < k) S.V[j] = vr[t];
    }
  } else {
    for (int j = 0; j < kw; ++j) {
      const bool o = f32b && j < k;
      float4 c[NCH];
      load_chunks<G, NCH>(c, o ? S.colp[j] : A, nv, s, o);
      const float v = gsum<G>(dotc<NCH>(c, aq));
      if (o && s == 0) S.V[j] = v;
    }
  }
  __syncwarp();
  float rsq = rsq0;
  const bool ok = grp_project<G, NCH>(act, s, M, A + (int64_t)(act ? q : 0) * M, yrow, act ? q : 0, k, aq, aa, bq,
                                      yv, rv, S, fl, rsq, stats);
  if (act && !ok) {
    if (s == 0) { st.flags[b] = fl | 1; atomicAdd((unsigned long long *)&stats[1], 1ull); }
    return;
  }
  if (!act) return;
  if (!(fl & 2))
    for (int j = s; j <= k; j += G) L_g[tri(k) + j] = S.L[tri(k) + j];
  for (int j = s; j <= k; j += G) st.alpha[b * st.ldo + j] = S.W[j];
  float4 *R4 = reinterpret_cast<float4 *>(st.R + b * M);
#pragma unroll
  for (int t = 0; t < NCH; ++t) {
    const int j = s + G * t;
    if (j < nv) R4[j] = rv[t];
  }
  if (st.Rbf) {
    const int Mp = (M + 63) / 64 * 64;
    __nv_bfloat162 *rb = reinterpret_cast<__nv_bfloat162 *>(st.Rbf + (rbf_row0 + wi) * Mp);  // sorted position
#pragma unroll
    for (int t = 0; t < NCH; ++t) {
      const int j = s + G * t;
      if (j < nv) {
        rb[2 * j] = __floats2bfloat162_rn(rv[t].x, rv[t].y);
        rb[2 * j + 1] = __floats2bfloat162_rn(rv[t].z, rv[t].w);
      }
    }
  }
  if (s == 0) {
    if (!(fl & 2)) z_g[k] = S.z[k];
    om_g[k] = q;
    st.k_eff[b] = (int8_t)(k + 1);
    uint8_t nf = fl;
    if (k + 1 >= Kpb) nf |= 1;
    if (rsq <= kEpsR32 * ysq) nf |= 1;
    if ((nf & 1) && k + 1 < Kpb) atomicAdd((unsigned long long *)&stats[1], 1ull);
    st.flags[b] = nf;
  }
}

// ---------------------------------------------------------------------------
// Restricted OMP with the Gram-matrix proxy ("Batch-OMP" form of the same
// iteration).  With p0 = A_C^T y and G = A A^T the proxy over the candidates
// is c_i = p0_i - sum_j alpha_j G[i][omega_j] = <a_i, r> (r = y - A_Omega alpha),
// the Gram column of the projection is G[q][omega_j], <a_q, y> = p0_q, and the
// residual norm is ||r||^2 = ||y||^2 - alpha^T p0_Omega (normal equations).  In
// FP32 these carry the same eps ||y|| cancellation error as an explicitly
// formed residual; only the stopping test needs ||r||^2 below that level, so
// when the estimate falls under 1e-5 ||y||^2 the residual is formed
// explicitly from the chosen rows.  Per iteration the only global loads are
// G[c][q] for the candidates (one wave).
// Per-group shared memory: GrpSmem | p0[cap] | Gc[cap][Kb] (its first 64 words
// hold the parents' child ranges while the candidate list is built) | p0 of
// the chosen [Kb].
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ int gram_ld(int cap) { return (cap + 3) & ~3; }  // Gc column stride
__host__ __device__ __forceinline__ int gram_gc_floats(int Kb, int cap) {
  const int f = gram_ld(cap) * Kb;
  return f > 2 * CSP_MAX_K ? f : 2 * CSP_MAX_K;
}
__host__ __device__ __forceinline__ int gram_group_bytes(int Kb, int cap) {
  const int bytes = grp_smem_bytes(Kb, cap) + up16(4 * cap) + 4 * gram_gc_floats(Kb, cap) + up16(4 * Kb);
  return (bytes + 127) / 128 * 128 + 16;  // groups start on different bank offsets
}

// Candidate list f(Omega_up) of one patch into S.cs (parents in support order,
// each parent's children in link order, at most cap; overflow counted in
// stats[3]).  pstart / pbeg: 2 x CSP_MAX_K ints of scratch.  Returns |C|.
// Warp-collective.
template <int G>
__device__ int list_candidates(bool valid, int s, int64_t b, int kup, const int32_t *__restrict__ omega_up,
                               int ldo_up, const int32_t *__restrict__ child_off,
                               const int32_t *__restrict__ child_idx, int cap, const GrpSmem &S, int *pstart,
                               int *pbeg, int64_t *stats) {
  constexpr int KPL = (CSP_MAX_K + G - 1) / G;
  // parents' child ranges in one wave, then the children
  int pr[KPL], c0r[KPL], c1r[KPL];
#pragma unroll
  for (int t = 0; t < KPL; ++t) {
    const int j = s + G * t;
    pr[t] = (j < kup) ? omega_up[b * ldo_up + j] : 0;
  }
#pragma unroll
  for (int t = 0; t < KPL; ++t) {
    const int j = s + G * t;
    c0r[t] = (j < kup) ? child_off[pr[t]] : 0;
    c1r[t] = (j < kup) ? child_off[pr[t] + 1] : 0;
  }
#pragma unroll
  for (int t = 0; t < KPL; ++t) {
    const int j = s + G * t;
    if (j < kup) { pstart[j] = c1r[t] - c0r[t]; pbeg[j] = c0r[t]; }
  }
  __syncwarp();
  if (s == 0 && valid) {
    int tot = 0;
    for (int j = 0; j < kup; ++j) {
      const int cnt = pstart[j];
      pstart[j] = tot;
      tot += cnt;
    }
    S.misc[2] = tot;
  }
  __syncwarp();
  int nc = valid ? S.misc[2] : 0;
  if (nc > cap) {
    if (s == 0) atomicAdd((unsigned long long *)&stats[3], 1ull);
    nc = cap;
  }
  for (int c = s; c < nc; c += G) {
    int j = 0;
    while (j + 1 < kup && pstart[j + 1] <= c) ++j;
    S.cs[c] = child_idx[pbeg[j] + (c - pstart[j])];
  }
  __syncwarp();
  return nc;
}

// The candidate list (list_candidates), the candidates' inverse norms, and
// p0 = A_C^T y (8 rows per load wave where registers allow, else 4).  Returns
// |C|.  Warp-collective.  PP: per-patch rows, candidate c of patch b at
// A + b a_pstride + c M, its inverse norm at inv_norm[b inv_pstride + c].
template <int G, int NCH, bool PP = false>
__device__ int gram_setup(bool valid, int s, int64_t b, int kup, const int32_t *__restrict__ omega_up, int ldo_up,
                          const int32_t *__restrict__ child_off, const int32_t *__restrict__ child_idx, int cap,
                          const GrpSmem &S, int *pstart, int *pbeg, const float *__restrict__ inv_norm,
                          int64_t *stats, int M, const float *__restrict__ A, const float4 (&yv)[NCH], float *p0,
                          int64_t a_pstride = 0, int64_t inv_pstride = 0) {
  const int nv = M >> 2;
  const int nc = list_candidates<G>(valid, s, b, kup, omega_up, ldo_up, child_off, child_idx, cap, S, pstart, pbeg,
                                    stats);
  __syncwarp();  // the parents' child ranges (aliasing Gc) are no longer read
  // p0 = A_C^T y and the candidates' inverse norms, RBP rows per load wave (lane s
  // fetches the norm of row s of the wave)
  constexpr int RBP = NCH > 2 ? 2 : (G >= 8 ? 8 : 4);  // RBP <= G
  const int ncw = __reduce_max_sync(kFull, nc);
  for (int c0 = 0; c0 < ncw; c0 += RBP) {
    const int ci = c0 + s;
    const bool oi = s < RBP && ci < nc;
    const float iv = oi ? __ldg(PP ? inv_norm + b * inv_pstride + ci : inv_norm + S.cs[ci]) : -1.f;
    float4 a[RBP][NCH];
#pragma unroll
    for (int u = 0; u < RBP; ++u) {
      const bool o = c0 + u < nc;
      const float *row = PP ? A + b * a_pstride + (int64_t)(o ? c0 + u : 0) * M : A + (int64_t)(o ? S.cs[c0 + u] : 0) * M;
      load_chunks<G, NCH>(a[u], row, nv, s, o);
    }
    if (oi) S.invn[ci] = iv;
#pragma unroll
    for (int u = 0; u < RBP; ++u) {
      const float d = gsum<G>(dotc<NCH>(a[u], yv));
      if (s == 0 && c0 + u < nc) p0[c0 + u] = d;
    }
  }
  __syncwarp();
  return nc;
}

template <int G, int NCH, bool PERSIST>
__global__ void __launch_bounds__(WV_WARPS * 32, 5)
omp_restricted_gram_kernel(const float *__restrict__ Y, int M, const float *__restrict__ A,
                           const float *__restrict__ inv_norm, const int32_t *__restrict__ ids, int64_t n,
                           const int32_t *__restrict__ child_off, const int32_t *__restrict__ child_idx,
                           int cap, const int32_t *__restrict__ omega_up, int ldo_up,
                           const int8_t *__restrict__ keff_up, const int8_t *__restrict__ Kp, int Kuni,
                           int Kb, int32_t *__restrict__ omega, float *__restrict__ alpha, int ldo,
                           int8_t *__restrict__ k_eff, int64_t *stats, const float *__restrict__ gram, int T,
    unsigned long long *__restrict__ queue, const float *__restrict__ = nullptr, int64_t = 0,
    int64_t = 0) {  // the trailing per-patch arguments of omp_restricted_qr_kernel, unused
  constexpr int NG = 32 / G;
  extern __shared__ __align__(16) char smem_raw[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, s = lane & (G - 1), g = lane / G;
  // one group of NG patches starting at wbase; a static grid runs it once per
  // warp, the persistent form pulls the next group from the work queue
  auto body = [&](const int64_t wbase) {
  if (wbase >= n) return;  // whole warp
  const int64_t wi = wbase + g;
  const bool valid = wi < n;
  char *gbase = smem_raw + (size_t)(wib * NG + g) * gram_group_bytes(Kb, cap);
  const GrpSmem S = carve(gbase, Kb, cap);
  char *q_ = gbase + grp_smem_bytes(Kb, cap);
  float *p0 = reinterpret_cast<float *>(q_); q_ += up16(4 * cap);
  float *Gc = reinterpret_cast<float *>(q_); q_ += 4 * gram_gc_floats(Kb, cap);  // Gc[j * ldg + c]
  const int ldg = gram_ld(cap);
  float *p0c = reinterpret_cast<float *>(q_);
  int *pstart = reinterpret_cast<int *>(Gc);  // parents' child ranges, before Gc is used
  int *pbeg = pstart + CSP_MAX_K;
  const int nv = M >> 2;
  const int64_t b = valid ? (ids ? __ldg(ids + wi) : wi) : 0;
  int Kpb = valid ? (Kp ? (int)Kp[b] : Kuni) : 0;
  Kpb = Kpb < Kb ? Kpb : Kb;
  const int kup = valid ? keff_up[b] : 0;
  const float *yrow = Y + b * M;
  float4 yv[NCH];
  load_chunks<G, NCH>(yv, yrow, nv, s, valid);
  const int nc = gram_setup<G, NCH>(valid, s, b, kup, omega_up, ldo_up, child_off, child_idx, cap, S, pstart, pbeg,
                                   inv_norm, stats, M, A, yv, p0);
  // lane steps over the candidates (c = s + u G) any group of this warp needs, at most 8
  const int ucnt = min(8, __reduce_max_sync(kFull, (nc + G - 1) / G));
  const float ysq = gsum<G>(dotc<NCH>(yv, yv));
  float rsq = ysq;
  bool act = valid && Kpb > 0;
  uint8_t fl = 0;
  int k = 0, scored = 0;
  const int Kw = __reduce_max_sync(kFull, Kpb);
  for (int it = 0; it < Kw; ++it) {
    act = act && k < Kpb && !(rsq <= kEpsR32 * ysq);
    if (!__any_sync(kFull, act)) break;
    if (act) ++scored;
    // proxy over the candidates from p0 and the cached Gram entries
    unsigned long long best = 0ull;
    if (act)
      for (int c = s; c < nc; c += G) {
        const float inv = S.invn[c];
        if (!(inv > 0.f)) continue;
        float sc = p0[c];
        for (int j = 0; j < k; ++j) sc = fmaf(-S.W[j], Gc[j * ldg + c], sc);
        const unsigned long long key = pack_key(fabsf(sc) * inv, S.cs[c]);
        best = key > best ? key : best;
      }
    best = gmax<G>(best);
    if (act && !best) act = false;  // candidate set exhausted
    const int q = act ? key_idx(best) : 0;
    if (act)
      for (int c = s; c < nc; c += G)
        if (S.cs[c] == q) {
          S.invn[c] = -1.f;  // chosen: no longer eligible
          S.misc[1] = c;
        }
    __syncwarp();
    const int qs = act ? S.misc[1] : 0;
    // G[q][c] for the first 8G candidates (row q: G is symmetric), issued now so
    // that the L2 round trip overlaps the projection; cached as column k below
    float gpre[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      if (u >= ucnt) break;  // ucnt is uniform over the warp
      const int c = s + u * G;
      gpre[u] = (act && c < nc) ? __ldg(gram + (int64_t)q * T + S.cs[c]) : 0.f;
    }
    const float aa = act ? __ldg(gram + (int64_t)q * T + q) : 0.f;  // ||a_q||^2
    const bool f32 = act && !(fl & 2);
    if (f32)
      for (int j = s; j < k; j += G) S.V[j] = Gc[j * ldg + qs];
    const float bq = act ? p0[qs] : 0.f;
    __syncwarp();
    // projection: W = L^{-1} V, pivot, z_k, alpha = L^{-T} z (as in grp_project)
    const int kw = __reduce_max_sync(kFull, act ? k : 0);
    for (int i = 0; i < kw; ++i) {
      if (f32 && i < k) {
        const float wi2 = S.V[i] * S.Linv[i];
        if (s == 0) S.W[i] = wi2;
        for (int j = i + 1 + s; j < k; j += G) S.V[j] = fmaf(-S.L[tri(j) + i], wi2, S.V[j]);
      }
      __syncwarp();
    }
    float ww = 0.f, zz = 0.f;
    if (f32)
      for (int j = s; j < k; j += G) {
        ww = fmaf(S.W[j], S.W[j], ww);
        zz = fmaf(S.W[j], S.z[j], zz);
      }
    ww = gsum<G>(ww);
    zz = gsum<G>(zz);
    const float d = aa - ww;
    const bool ok32 = f32 && aa > 0.f && d >= kTauPivot * aa;
    if (f32 && !ok32) {
      fl |= 2;
      if (s == 0) atomicAdd((unsigned long long *)&stats[0], 1ull);
    }
    if (ok32) {
      const float lkk = sqrtf(d), il = 1.f / lkk;
      for (int j = s; j < k; j += G) S.L[tri(k) + j] = S.W[j];
      if (s == 0) {
        S.L[tri(k) + k] = lkk;
        S.Linv[k] = il;
        S.z[k] = (bq - zz) * il;
      }
    }
    __syncwarp();
    if (ok32)
      for (int i = s; i <= k; i += G) S.V[i] = S.z[i];
    __syncwarp();
    for (int j = kw; j >= 0; --j) {
      if (ok32 && j <= k) {
        const float aj = S.V[j] * S.Linv[j];
        if (s == 0) S.W[j] = aj;
        for (int i = s; i < j; i += G) S.V[i] = fmaf(-S.L[tri(j) + i], aj, S.V[i]);
      }
      __syncwarp();
    }
    const bool go64 = act && !ok32;
    if (go64 && s == 0) S.misc[0] = fp64_projection(M, yrow, S, k, A + (int64_t)q * M) ? 1 : 0;
    __syncwarp();
    const bool appended = ok32 || (go64 && S.misc[0] != 0);
    // q depends on the chosen columns: its FP32 attempt overwrote S.W; alpha of
    // the chosen ones again from the (unchanged) factor
    const bool restore = f32 && !appended;
    if (__any_sync(kFull, restore))
      grp_backsub<G>(restore, s, k - 1, __reduce_max_sync(kFull, restore ? k - 1 : 0), S);
    if (appended && s == 0) {
      S.om[k] = q;
      S.colp[k] = A + (int64_t)q * M;
      p0c[k] = bq;
    }
    __syncwarp();
    // ||r||^2 = ||y||^2 - alpha^T p0_Omega; formed explicitly when near the FP32 floor
    float e = 0.f;
    if (appended)
      for (int j = s; j <= k; j += G) e = fmaf(S.W[j], p0c[j], e);
    e = gsum<G>(e);
    const float est = ysq - e;
    const bool exact = appended && est <= 1e-5f * ysq;
    if (__any_sync(kFull, exact)) {
      float4 rv[NCH];
#pragma unroll
      for (int t = 0; t < NCH; ++t) rv[t] = yv[t];
      const int kx = __reduce_max_sync(kFull, exact ? k + 1 : 0);
      for (int j0 = 0; j0 < kx; j0 += RB) {
        float4 c[RB][NCH];
#pragma unroll
        for (int u = 0; u < RB; ++u) {
          const bool o = exact && j0 + u <= k;
          load_chunks<G, NCH>(c[u], o ? S.colp[j0 + u] : yrow, nv, s, o);
        }
#pragma unroll
        for (int u = 0; u < RB; ++u)
          if (exact && j0 + u <= k) {
            const float aj = S.W[j0 + u];
#pragma unroll
            for (int t = 0; t < NCH; ++t) {
              rv[t].x = fmaf(-aj, c[u][t].x, rv[t].x);
              rv[t].y = fmaf(-aj, c[u][t].y, rv[t].y);
              rv[t].z = fmaf(-aj, c[u][t].z, rv[t].z);
              rv[t].w = fmaf(-aj, c[u][t].w, rv[t].w);
            }
          }
      }
      const float r2 = gsum<G>(dotc<NCH>(rv, rv));
      if (exact) rsq = r2;
    }
    if (appended && !exact) rsq = est;
    if (act) {
      if (appended) {
        // cache G[c][q] for every candidate as column k (the first 8G prefetched)
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int c = s + u * G;
          if (u < ucnt && c < nc) Gc[k * ldg + c] = gpre[u];
        }
        for (int c0 = s + 8 * G; c0 < nc; c0 += 8 * G) {
          float gr[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int c = c0 + u * G;
            gr[u] = (c < nc) ? __ldg(gram + (int64_t)q * T + S.cs[c]) : 0.f;
          }
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int c = c0 + u * G;
            if (c < nc) Gc[k * ldg + c] = gr[u];
          }
        }
        ++k;
      } else {
        act = false;
      }
    }
    __syncwarp();
  }
  if (valid) {
    if (s == 0) {
      if (k < Kpb) atomicAdd((unsigned long long *)&stats[1], 1ull);
      atomicAdd((unsigned long long *)&stats[2], (unsigned long long)nc * (unsigned long long)scored);
      k_eff[b] = (int8_t)k;
    }
    for (int j = s; j < ldo; j += G) {
      omega[b * ldo + j] = (j < k) ? S.om[j] : -1;
      alpha[b * ldo + j] = (j < k) ? S.W[j] : 0.f;
    }
  }
  };
  if (!PERSIST) {
    body(((int64_t)blockIdx.x * WV_WARPS + wib) * NG);
    return;
  }
  for (;;) {  // each warp takes the next NG patches with one atomic add; nothing waits
    unsigned long long w = 0ull;
    if (lane == 0) w = atomicAdd(queue, (unsigned long long)NG);
    w = __shfl_sync(kFull, w, 0);
    if ((int64_t)w >= n) break;
    body((int64_t)w);
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// Restricted OMP in Gram-Schmidt form (same iteration, same Gram matrix).
// With u_j the orthonormal directions of the chosen atoms (A_Omega = U L^T, L
// the Cholesky factor of A_Omega^T A_Omega), the group keeps Q_C = A_C^T U
// (column j = <a_c, u_j> for every candidate c) and the correlations
// c_c = <a_c, r>.  Appending atom q needs no triangular solve: the new row of L
// is w = Q_C[q] (the row of q), L_kk = sqrt(||a_q||^2 - ||w||^2),
// z_k = <u_k, y> = (p0_q - w.z) / L_kk, the new column of Q_C is
// (G[q][C] - Q_C w) / L_kk, then c -= z_k Q_C[:, k] and ||r||^2 -= z_k^2.
// alpha = L^{-T} z is solved once at the end (and near the FP32 floor of
// ||r||^2, where the residual is formed explicitly).  A patch whose FP32 pivot
// fails continues in FP64 from scratch each iteration, with the correlations
// recomputed from the Gram rows of its chosen atoms.
// Per-group shared memory: GrpSmem | p0[cap] | c[cap] | Q_C[Kb][ldg] (its
// first 64 words hold the parents' child ranges while the candidates are
// listed) | p0 of the chosen [Kb].
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ int qr_group_bytes(int Kb, int cap) {
  const int bytes = grp_smem_bytes(Kb, cap) + 2 * up16(4 * cap) + 4 * gram_gc_floats(Kb, cap) + up16(4 * Kb);
  return (bytes + 127) / 128 * 128 + 16;  // groups start on different bank offsets
}

// PP: per-patch candidate rows (per-pixel Phi): candidate c of patch b has its
// row at A + b a_pstride + c M, its inverse norm at inv_norm[b inv_pstride + c],
// and the patch's Gram block G_C at gpp + b cap^2 (row i at i cap, in the order
// of the candidate list); chosen atoms are tracked by their slot.
template <int G, int NCH, bool PERSIST, bool PP = false>
__global__ void __launch_bounds__(WV_WARPS * 32, 5)
omp_restricted_qr_kernel(const float *__restrict__ Y, int M, const float *__restrict__ A,
                         const float *__restrict__ inv_norm, const int32_t *__restrict__ ids, int64_t n,
                         const int32_t *__restrict__ child_off, const int32_t *__restrict__ child_idx,
                         int cap, const int32_t *__restrict__ omega_up, int ldo_up,
                         const int8_t *__restrict__ keff_up, const int8_t *__restrict__ Kp, int Kuni,
                         int Kb, int32_t *__restrict__ omega, float *__restrict__ alpha, int ldo,
                         int8_t *__restrict__ k_eff, int64_t *stats, const float *__restrict__ gram, int T,
    unsigned long long *__restrict__ queue, const float *__restrict__ gpp = nullptr, int64_t a_pstride = 0,
    int64_t inv_pstride = 0) {
  constexpr int NG = 32 / G;
  extern __shared__ __align__(16) char smem_raw[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, s = lane & (G - 1), g = lane / G;
  // one group of NG patches starting at wbase; a static grid runs it once per
  // warp, the persistent form pulls the next group from the work queue
  auto body = [&](const int64_t wbase) {
  if (wbase >= n) return;  // whole warp
  const int64_t wi = wbase + g;
  const bool valid = wi < n;
  char *gbase = smem_raw + (size_t)(wib * NG + g) * qr_group_bytes(Kb, cap);
  const GrpSmem S = carve(gbase, Kb, cap);
  char *q_ = gbase + grp_smem_bytes(Kb, cap);
  float *p0 = reinterpret_cast<float *>(q_); q_ += up16(4 * cap);
  float *cc = reinterpret_cast<float *>(q_); q_ += up16(4 * cap);
  float *Qc = reinterpret_cast<float *>(q_); q_ += 4 * gram_gc_floats(Kb, cap);  // Qc[j * ldg + c]
  const int ldg = gram_ld(cap);
  float *p0c = reinterpret_cast<float *>(q_);
  int *pstart = reinterpret_cast<int *>(Qc);  // parents' child ranges, before Qc is used
  int *pbeg = pstart + CSP_MAX_K;
  const int nv = M >> 2;
  const int64_t b = valid ? (ids ? __ldg(ids + wi) : wi) : 0;
  int Kpb = valid ? (Kp ? (int)Kp[b] : Kuni) : 0;
  Kpb = Kpb < Kb ? Kpb : Kb;
  const int kup = valid ? keff_up[b] : 0;
  const float *yrow = Y + b * M;
  float4 yv[NCH];
  load_chunks<G, NCH>(yv, yrow, nv, s, valid);
  const int nc = gram_setup<G, NCH, PP>(valid, s, b, kup, omega_up, ldo_up, child_off, child_idx, cap, S, pstart,
                                       pbeg, inv_norm, stats, M, A, yv, p0, a_pstride, inv_pstride);
  const float *gb = PP ? gpp + b * (int64_t)cap * cap : nullptr;  // this patch's Gram block
  // G[q][C_c], with q in slot qs; and the row of atom q
  auto gqc = [&](int q, int qs, int c) -> float {
    return PP ? __ldg(gb + qs * cap + c) : __ldg(gram + (int64_t)q * T + S.cs[c]);
  };
  auto rowq = [&](int q, int qs) -> const float * {
    return PP ? A + b * a_pstride + (int64_t)qs * M : A + (int64_t)q * M;
  };
  // lane steps over the candidates (c = s + u G) any group of this warp needs, at most 8
  const int ucnt = min(8, __reduce_max_sync(kFull, (nc + G - 1) / G));
  for (int c = s; c < nc; c += G) cc[c] = p0[c];
  __syncwarp();
  const float ysq = gsum<G>(dotc<NCH>(yv, yv));
  float rsq = ysq;
  bool act = valid && Kpb > 0;
  uint8_t fl = 0;  // bit 1: FP64 from here on
  int k = 0, scored = 0;
  const int Kw = __reduce_max_sync(kFull, Kpb);
  for (int it = 0; it < Kw; ++it) {
    act = act && k < Kpb && !(rsq <= kEpsR32 * ysq);
    if (!__any_sync(kFull, act)) break;
    if (act) ++scored;
    // proxy from the current correlations
    unsigned long long best = 0ull;
    if (act)
      for (int c = s; c < nc; c += G) {
        const float inv = S.invn[c];
        if (!(inv > 0.f)) continue;
        const unsigned long long key = pack_key(fabsf(cc[c]) * inv, S.cs[c]);
        best = key > best ? key : best;
      }
    best = gmax<G>(best);
    if (act && !best) act = false;  // candidate set exhausted
    const int q = act ? key_idx(best) : 0;
    if (act)
      for (int c = s; c < nc; c += G)
        if (S.cs[c] == q) {
          S.invn[c] = -1.f;  // chosen: no longer eligible
          S.misc[1] = c;
        }
    __syncwarp();
    const int qs = act ? S.misc[1] : 0;
    // G[q][C] (row q: G is symmetric) and G[q][q], issued before their use
    float gpre[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      if (u >= ucnt) break;  // ucnt is uniform over the warp
      const int c = s + u * G;
      gpre[u] = (act && c < nc) ? gqc(q, qs, c) : 0.f;
    }
    const float aa = act ? (PP ? __ldg(gb + qs * cap + qs) : __ldg(gram + (int64_t)q * T + q)) : 0.f;
    const bool f32 = act && !(fl & 2);
    // new row of L: w_j = <u_j, a_q> = Q_C[q][j]
    float ww = 0.f, wz = 0.f;
    if (f32)
      for (int j = s; j < k; j += G) {
        const float w = Qc[j * ldg + qs];
        S.W[j] = w;
        ww = fmaf(w, w, ww);
        wz = fmaf(w, S.z[j], wz);
      }
    ww = gsum<G>(ww);
    wz = gsum<G>(wz);
    const float d = aa - ww;
    const bool ok32 = f32 && aa > 0.f && d >= kTauPivot * aa;
    if (f32 && !ok32) {
      fl |= 2;
      if (s == 0) atomicAdd((unsigned long long *)&stats[0], 1ull);
    }
    float il = 0.f, zk = 0.f;
    if (ok32) {
      const float lkk = sqrtf(d);
      il = 1.f / lkk;
      zk = (p0[qs] - wz) * il;
      for (int j = s; j < k; j += G) S.L[tri(k) + j] = S.W[j];
      if (s == 0) {
        S.L[tri(k) + k] = lkk;
        S.Linv[k] = il;
        S.z[k] = zk;
        S.om[k] = PP ? qs : q;
        S.colp[k] = rowq(q, qs);
        p0c[k] = p0[qs];
      }
    }
    __syncwarp();
    if (ok32) {
      // column k of Q_C and the correlations
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        if (u >= ucnt) break;
        const int c = s + u * G;
        if (c < nc) {
          float v = gpre[u];
          for (int j = 0; j < k; ++j) v = fmaf(-S.W[j], Qc[j * ldg + c], v);
          v *= il;
          Qc[k * ldg + c] = v;
          cc[c] = fmaf(-zk, v, cc[c]);
        }
      }
      for (int c = s + 8 * G; c < nc; c += G) {
        float v = gqc(q, qs, c);
        for (int j = 0; j < k; ++j) v = fmaf(-S.W[j], Qc[j * ldg + c], v);
        v *= il;
        Qc[k * ldg + c] = v;
        cc[c] = fmaf(-zk, v, cc[c]);
      }
      rsq = rsq - zk * zk;
    }
    // FP64 from scratch for the patches whose FP32 pivot failed (now or before)
    const bool go64 = act && !ok32;
    if (go64 && s == 0) S.misc[0] = fp64_projection(M, yrow, S, k, rowq(q, qs)) ? 1 : 0;
    __syncwarp();
    const bool app64 = go64 && S.misc[0] != 0;
    // q depends on the chosen columns: alpha of the chosen ones from the FP32
    // factor (S.W held w); FP64-mode patches still hold their last alpha
    const bool restore = f32 && !ok32 && !app64;
    if (__any_sync(kFull, restore))
      grp_backsub<G>(restore, s, k - 1, __reduce_max_sync(kFull, restore ? k - 1 : 0), S);
    if (app64 && s == 0) {
      S.om[k] = PP ? qs : q;
      S.colp[k] = rowq(q, qs);
    }
    __syncwarp();
    if (app64)  // correlations c = p0 - G[C][Omega] alpha from the Gram rows of the chosen atoms
      for (int c = s; c < nc; c += G) {
        float v = p0[c];
        for (int j = 0; j <= k; ++j)
          v = fmaf(-S.W[j], PP ? __ldg(gb + S.om[j] * cap + c) : __ldg(gram + (int64_t)S.om[j] * T + S.cs[c]), v);
        cc[c] = v;
      }
    // ||r||^2 formed explicitly in FP64 mode and near the FP32 floor
    const bool exact = app64 || (ok32 && rsq <= 1e-5f * ysq);
    if (__any_sync(kFull, exact)) {
      const bool need = exact && !app64;  // FP32: alpha over rows 0..k first
      grp_backsub<G>(need, s, k, __reduce_max_sync(kFull, need ? k : 0), S);
      float4 rv[NCH];
#pragma unroll
      for (int t = 0; t < NCH; ++t) rv[t] = yv[t];
      const int kx = __reduce_max_sync(kFull, exact ? k + 1 : 0);
      for (int j0 = 0; j0 < kx; j0 += RB) {
        float4 cr[RB][NCH];
#pragma unroll
        for (int u = 0; u < RB; ++u) {
          const bool o = exact && j0 + u <= k;
          load_chunks<G, NCH>(cr[u], o ? S.colp[j0 + u] : yrow, nv, s, o);
        }
#pragma unroll
        for (int u = 0; u < RB; ++u)
          if (exact && j0 + u <= k) {
            const float aj = S.W[j0 + u];
#pragma unroll
            for (int t = 0; t < NCH; ++t) {
              rv[t].x = fmaf(-aj, cr[u][t].x, rv[t].x);
              rv[t].y = fmaf(-aj, cr[u][t].y, rv[t].y);
              rv[t].z = fmaf(-aj, cr[u][t].z, rv[t].z);
              rv[t].w = fmaf(-aj, cr[u][t].w, rv[t].w);
            }
          }
      }
      const float r2 = gsum<G>(dotc<NCH>(rv, rv));
      if (exact) rsq = r2;
    }
    if (act) {
      if (ok32 || app64) ++k;
      else act = false;
    }
    __syncwarp();
  }
  // alpha = L^{-T} z for the patches that stayed in FP32 (FP64 ones hold it in S.W)
  const bool fin = valid && !(fl & 2) && k > 0;
  grp_backsub<G>(fin, s, k - 1, __reduce_max_sync(kFull, fin ? k - 1 : 0), S);
  if (valid) {
    if (s == 0) {
      if (k < Kpb) atomicAdd((unsigned long long *)&stats[1], 1ull);
      atomicAdd((unsigned long long *)&stats[2], (unsigned long long)nc * (unsigned long long)scored);
      k_eff[b] = (int8_t)k;
    }
    for (int j = s; j < ldo; j += G) {
      omega[b * ldo + j] = (j < k) ? (PP ? S.cs[S.om[j]] : S.om[j]) : -1;
      alpha[b * ldo + j] = (j < k) ? S.W[j] : 0.f;
    }
  }
  };
  if (!PERSIST) {
    body(((int64_t)blockIdx.x * WV_WARPS + wib) * NG);
    return;
  }
  for (;;) {  // each warp takes the next NG patches with one atomic add; nothing waits
    unsigned long long w = 0ull;
    if (lane == 0) w = atomicAdd(queue, (unsigned long long)NG);
    w = __shfl_sync(kFull, w, 0);
    if ((int64_t)w >= n) break;
    body((int64_t)w);
    __syncwarp();
  }
}

// x_hat = D0_Omega alpha for one patch, lanes s = 0 .. G-1 of its group each
// writing float4 chunks s, s + G, ... of the row: the chosen rows in support
// order, one FMA each from zero, as synth_kernel does (same values).  Not
// inlined, so that the solver's loop does not hold its operands.
static __device__ __noinline__ void synth_patch(const float *__restrict__ D0, int N0, float *__restrict__ xrow,
                                                const float *W, const int *om, int k, int s, int G) {
  constexpr int XS = 6;  // float4 chunks per lane per pass
  const int n4 = N0 >> 2;
  float4 *xb = reinterpret_cast<float4 *>(xrow);
  for (int c0 = s; c0 < n4; c0 += G * XS) {
    float4 acc[XS];
#pragma unroll
    for (int t = 0; t < XS; ++t) acc[t] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 2
    for (int j = 0; j < k; ++j) {
      const float aj = W[j];
      const float4 *dr = reinterpret_cast<const float4 *>(D0 + (int64_t)om[j] * N0);
      float4 d[XS];
#pragma unroll
      for (int t = 0; t < XS; ++t) {
        const int ch = c0 + G * t;
        d[t] = ch < n4 ? __ldg(dr + ch) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int t = 0; t < XS; ++t) {
        acc[t].x = fmaf(aj, d[t].x, acc[t].x);
        acc[t].y = fmaf(aj, d[t].y, acc[t].y);
        acc[t].z = fmaf(aj, d[t].z, acc[t].z);
        acc[t].w = fmaf(aj, d[t].w, acc[t].w);
      }
    }
#pragma unroll
    for (int t = 0; t < XS; ++t) {
      const int ch = c0 + G * t;
      if (ch < n4) xb[ch] = acc[t];
    }
  }
}

// ---------------------------------------------------------------------------
// The Gram-Schmidt form for Kb <= 8 with Q_C stored by candidate: row c of
// Q_C (its 8 entries <a_c, u_j>, zero beyond the chosen count) is 32 bytes,
// its two 16-byte halves swapped when bit 2 of c is set so that the 8 lanes of
// a group read 8 rows without bank conflicts.  A candidate's column update is
// then two 16-byte loads and 8 FMAs (two chains of four) against w held in
// registers; the new row of L (w = Q_C[q]) is two broadcast loads; the group
// argmax compares the score bits first and the indices only where scores tie,
// and finds the winner's lane and slot by ballot; ||w||^2 and <w, z> are formed
// by every lane (z in registers), with no group reduction.  Through
// csp_reconstruct the kernel also writes x_hat = D0_Omega alpha (synth_patch).  Same iteration, outputs and
// FP64 / explicit-residual paths as omp_restricted_qr_kernel.
// Per-group shared memory: GrpSmem | p0[cap] | c[cap] | Q_C[cap][8] (its first
// 64 words hold the parents' child ranges while the candidates are listed).
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ int qr8_q_floats(int cap) {
  return 8 * cap > 2 * CSP_MAX_K ? 8 * cap : 2 * CSP_MAX_K;
}
__host__ __device__ __forceinline__ int qr8_group_bytes(int Kb, int cap) {
  const int bytes = grp_smem_bytes(Kb, cap) + 2 * up16(4 * cap) + 4 * qr8_q_floats(cap);
  return (bytes + 127) / 128 * 128 + 16;  // groups start on different bank offsets
}

template <int G, int NCH>
__global__ void __launch_bounds__(WV_WARPS * 32, 5)
omp_restricted_qr8_kernel(const float *__restrict__ Y, int M, const float *__restrict__ A,
                          const float *__restrict__ inv_norm, const int32_t *__restrict__ ids, int64_t n,
                          const int32_t *__restrict__ child_off, const int32_t *__restrict__ child_idx,
                          int cap, const int32_t *__restrict__ omega_up, int ldo_up,
                          const int8_t *__restrict__ keff_up, const int8_t *__restrict__ Kp, int Kuni,
                          int Kb, int32_t *__restrict__ omega, float *__restrict__ alpha, int ldo,
                          int8_t *__restrict__ k_eff, int64_t *stats, const float *__restrict__ gram, int T,
                          const float *__restrict__ D0, int N0, float *__restrict__ Xh) {
  constexpr int NG = 32 / G;
  constexpr unsigned GMASK = G == 32 ? 0xffffffffu : ((1u << G) - 1u);
  extern __shared__ __align__(16) char smem_raw[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, s = lane & (G - 1), g = lane / G;
  const int64_t wbase = ((int64_t)blockIdx.x * WV_WARPS + wib) * NG;
  if (wbase >= n) return;  // whole warp
  const int64_t wi = wbase + g;
  const bool valid = wi < n;
  char *gbase = smem_raw + (size_t)(wib * NG + g) * qr8_group_bytes(Kb, cap);
  const GrpSmem S = carve(gbase, Kb, cap);
  char *q_ = gbase + grp_smem_bytes(Kb, cap);
  float *p0 = reinterpret_cast<float *>(q_); q_ += up16(4 * cap);
  float *cc = reinterpret_cast<float *>(q_); q_ += up16(4 * cap);
  float *Q = reinterpret_cast<float *>(q_);  // Q_C rows, [cap][8], halves swapped for bit 2 of c
  float4 *Q4 = reinterpret_cast<float4 *>(Q);
  int *pstart = reinterpret_cast<int *>(Q);  // parents' child ranges, before Q_C is used
  int *pbeg = pstart + CSP_MAX_K;
  const int nv = M >> 2;
  const int64_t b = valid ? (ids ? __ldg(ids + wi) : wi) : 0;
  int Kpb = valid ? (Kp ? (int)Kp[b] : Kuni) : 0;
  Kpb = Kpb < Kb ? Kpb : Kb;
  const int kup = valid ? keff_up[b] : 0;
  const float *yrow = Y + b * M;
  float4 yv[NCH];
  load_chunks<G, NCH>(yv, yrow, nv, s, valid);
  const int nc = gram_setup<G, NCH>(valid, s, b, kup, omega_up, ldo_up, child_off, child_idx, cap, S, pstart, pbeg,
                                   inv_norm, stats, M, A, yv, p0);
  const int ucnt = min(8, __reduce_max_sync(kFull, (nc + G - 1) / G));
  const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int c = s; c < nc; c += G) {
    cc[c] = p0[c];
    Q4[2 * c] = zero4;
    Q4[2 * c + 1] = zero4;
  }
  __syncwarp();
  const float ysq = gsum<G>(dotc<NCH>(yv, yv));
  float rsq = ysq;
  bool act = valid && Kpb > 0;
  uint8_t fl = 0;  // bit 1: FP64 from here on
  int k = 0, scored = 0;
  float zr[8];  // z_j of the chosen (zero beyond k)
#pragma unroll
  for (int j = 0; j < 8; ++j) zr[j] = 0.f;
  const int Kw = __reduce_max_sync(kFull, Kpb);
  for (int it = 0; it < Kw; ++it) {
    act = act && k < Kpb && !(rsq <= kEpsR32 * ysq);
    if (!__any_sync(kFull, act)) break;
    if (act) ++scored;
    // proxy from the current correlations; the lane's best key and its slot
    unsigned long long best = 0ull;
    int bslot = 0;
    if (act)
      for (int c = s; c < nc; c += G) {
        const float inv = S.invn[c];
        if (!(inv > 0.f)) continue;
        const unsigned long long key = pack_key(fabsf(cc[c]) * inv, S.cs[c]);
        if (key > best) {
          best = key;
          bslot = c;
        }
      }
    // group argmax of the packed keys: the largest score bits first, then (only
    // where two lanes tie on the score) the largest complemented index
    const unsigned bs = (unsigned)(best >> 32);
    unsigned ms = bs;
#pragma unroll
    for (int o = G / 2; o; o >>= 1) ms = max(ms, __shfl_xor_sync(kFull, ms, o));
    const bool top = best != 0ull && bs == ms;
    unsigned tb = (__ballot_sync(kFull, top) >> (g * G)) & GMASK;
    if (__any_sync(kFull, __popc(tb) > 1)) {
      const unsigned lw = top ? (unsigned)best : 0u;
      unsigned ml = lw;
#pragma unroll
      for (int o = G / 2; o; o >>= 1) ml = max(ml, __shfl_xor_sync(kFull, ml, o));
      tb = (__ballot_sync(kFull, top && lw == ml) >> (g * G)) & GMASK;
    }
    if (act && !tb) act = false;  // candidate set exhausted
    const int wl = g * G + (tb ? __ffs(tb) - 1 : 0);
    // every lane takes part in both shuffles (inactive groups read their lane 0)
    const unsigned qlw = __shfl_sync(kFull, (unsigned)best, wl);
    const int qs = __shfl_sync(kFull, bslot, wl);
    const int q = act ? (int)(0xffffffffu - qlw) : 0;
    // the winner's slot qs is no longer eligible
    const bool mine = act && lane == wl;
    if (mine) S.invn[bslot] = -1.f;
    // G[q][C] (row q: G is symmetric) and G[q][q], issued before their use
    float gpre[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      if (u >= ucnt) break;  // ucnt is uniform over the warp
      const int c = s + u * G;
      gpre[u] = (act && c < nc) ? __ldg(gram + (int64_t)q * T + S.cs[c]) : 0.f;
    }
    const float aa = act ? __ldg(gram + (int64_t)q * T + q) : 0.f;
    const bool f32 = act && !(fl & 2);
    // new row of L: w = Q_C[q] (broadcast loads of row qs)
    float w[8];
    {
      const int sq = (qs >> 2) & 1;
      const float4 h0 = f32 ? Q4[2 * qs + sq] : zero4, h1 = f32 ? Q4[2 * qs + 1 - sq] : zero4;
      w[0] = h0.x; w[1] = h0.y; w[2] = h0.z; w[3] = h0.w;
      w[4] = h1.x; w[5] = h1.y; w[6] = h1.z; w[7] = h1.w;
    }
    // two independent chains each (halves j < 4, j >= 4), then their sum
    float ww0 = 0.f, ww1 = 0.f, wz0 = 0.f, wz1 = 0.f;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      ww0 = fmaf(w[j], w[j], ww0);
      ww1 = fmaf(w[j + 4], w[j + 4], ww1);
      wz0 = fmaf(w[j], zr[j], wz0);
      wz1 = fmaf(w[j + 4], zr[j + 4], wz1);
    }
    const float ww = ww0 + ww1, wz = wz0 + wz1;
    const float d = aa - ww;
    const bool ok32 = f32 && aa > 0.f && d >= kTauPivot * aa;
    if (f32 && !ok32) {
      fl |= 2;
      if (s == 0) atomicAdd((unsigned long long *)&stats[0], 1ull);
    }
    if (ok32) {
      const float il = rsqrtf(d);  // d >= kTauPivot aa > 0
      const float lkk = d * il;
      const float zk = (p0[qs] - wz) * il;
      if (s == 0) {
#pragma unroll
        for (int j = 0; j < 8; ++j)
          if (j < k) S.L[tri(k) + j] = w[j];
        S.L[tri(k) + k] = lkk;
        S.Linv[k] = il;
        S.z[k] = zk;
        S.om[k] = q;
        S.colp[k] = A + (int64_t)q * M;
      }
#pragma unroll
      for (int j = 0; j < 8; ++j)
        if (j == k) zr[j] = zk;
      // column k of Q_C and the correlations
      const int kofs = (k & 3);
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        if (u >= ucnt) break;
        const int c = s + u * G;
        if (c < nc) {
          const int sc = (c >> 2) & 1;
          const float4 qa = Q4[2 * c + sc], qb = Q4[2 * c + 1 - sc];
          // w . Q_C[c] as two chains of four, then G[q][c] minus it
          float v0 = w[0] * qa.x, v1 = w[4] * qb.x;
          v0 = fmaf(w[1], qa.y, v0);
          v1 = fmaf(w[5], qb.y, v1);
          v0 = fmaf(w[2], qa.z, v0);
          v1 = fmaf(w[6], qb.z, v1);
          v0 = fmaf(w[3], qa.w, v0);
          v1 = fmaf(w[7], qb.w, v1);
          float v = (gpre[u] - (v0 + v1)) * il;
          Q[8 * c + ((((k >> 2) ^ sc)) << 2) + kofs] = v;
          cc[c] = fmaf(-zk, v, cc[c]);
        }
      }
      for (int c = s + 8 * G; c < nc; c += G) {
        const int sc = (c >> 2) & 1;
        const float4 qa = Q4[2 * c + sc], qb = Q4[2 * c + 1 - sc];
        float v0 = w[0] * qa.x, v1 = w[4] * qb.x;
        v0 = fmaf(w[1], qa.y, v0);
        v1 = fmaf(w[5], qb.y, v1);
        v0 = fmaf(w[2], qa.z, v0);
        v1 = fmaf(w[6], qb.z, v1);
        v0 = fmaf(w[3], qa.w, v0);
        v1 = fmaf(w[7], qb.w, v1);
        float v = (__ldg(gram + (int64_t)q * T + S.cs[c]) - (v0 + v1)) * il;
        Q[8 * c + ((((k >> 2) ^ sc)) << 2) + kofs] = v;
        cc[c] = fmaf(-zk, v, cc[c]);
      }
      rsq = rsq - zk * zk;
    }
    // FP64 from scratch for the patches whose FP32 pivot failed (now or before)
    const bool go64 = act && !ok32;
    if (go64 && s == 0) S.misc[0] = fp64_projection(M, yrow, S, k, A + (int64_t)q * M) ? 1 : 0;
    __syncwarp();
    const bool app64 = go64 && S.misc[0] != 0;
    // q depends on the chosen columns: alpha of the chosen ones from the FP32 factor
    const bool restore = f32 && !ok32 && !app64;
    if (__any_sync(kFull, restore))
      grp_backsub<G>(restore, s, k - 1, __reduce_max_sync(kFull, restore ? k - 1 : 0), S);
    if (app64 && s == 0) {
      S.om[k] = q;
      S.colp[k] = A + (int64_t)q * M;
    }
    __syncwarp();
    if (app64)  // correlations c = p0 - G[C][Omega] alpha from the Gram rows of the chosen atoms
      for (int c = s; c < nc; c += G) {
        float v = p0[c];
        for (int j = 0; j <= k; ++j) v = fmaf(-S.W[j], __ldg(gram + (int64_t)S.om[j] * T + S.cs[c]), v);
        cc[c] = v;
      }
    // ||r||^2 formed explicitly in FP64 mode and near the FP32 floor
    const bool exact = app64 || (ok32 && rsq <= 1e-5f * ysq);
    if (__any_sync(kFull, exact)) {
      const bool need = exact && !app64;  // FP32: alpha over rows 0..k first
      grp_backsub<G>(need, s, k, __reduce_max_sync(kFull, need ? k : 0), S);
      float4 rv[NCH];
#pragma unroll
      for (int t = 0; t < NCH; ++t) rv[t] = yv[t];
      const int kx = __reduce_max_sync(kFull, exact ? k + 1 : 0);
      constexpr int RBX = NCH > 2 ? 1 : RB;  // rows per load wave of this rare path
      for (int j0 = 0; j0 < kx; j0 += RBX) {
        float4 cr[RBX][NCH];
#pragma unroll
        for (int u = 0; u < RBX; ++u) {
          const bool o = exact && j0 + u <= k;
          load_chunks<G, NCH>(cr[u], o ? S.colp[j0 + u] : yrow, nv, s, o);
        }
#pragma unroll
        for (int u = 0; u < RBX; ++u)
          if (exact && j0 + u <= k) {
            const float aj = S.W[j0 + u];
#pragma unroll
            for (int t = 0; t < NCH; ++t) {
              rv[t].x = fmaf(-aj, cr[u][t].x, rv[t].x);
              rv[t].y = fmaf(-aj, cr[u][t].y, rv[t].y);
              rv[t].z = fmaf(-aj, cr[u][t].z, rv[t].z);
              rv[t].w = fmaf(-aj, cr[u][t].w, rv[t].w);
            }
          }
      }
      const float r2 = gsum<G>(dotc<NCH>(rv, rv));
      if (exact) rsq = r2;
    }
    if (act) {
      if (ok32 || app64) ++k;
      else act = false;
    }
    __syncwarp();
  }
  // alpha = L^{-T} z for the patches that stayed in FP32 (FP64 ones hold it in S.W)
  const bool fin = valid && !(fl & 2) && k > 0;
  grp_backsub<G>(fin, s, k - 1, __reduce_max_sync(kFull, fin ? k - 1 : 0), S);
  if (valid) {
    if (s == 0) {
      if (k < Kpb) atomicAdd((unsigned long long *)&stats[1], 1ull);
      atomicAdd((unsigned long long *)&stats[2], (unsigned long long)nc * (unsigned long long)scored);
      k_eff[b] = (int8_t)k;
    }
    for (int j = s; j < ldo; j += G) {
      omega[b * ldo + j] = (j < k) ? S.om[j] : -1;
      alpha[b * ldo + j] = (j < k) ? S.W[j] : 0.f;
    }
  }
  // synthesis x_hat_b = D0_Omega alpha (Sec. IV) into Xh[b] when asked for
  if (Xh && valid) synth_patch(D0, N0, Xh + b * N0, S.W, S.om, k, s, G);
}

// Restricted OMP in Gram-Schmidt form with the candidate state in registers.
// Same iteration as omp_restricted_qr_kernel, but lane s of a group owns the
// candidates c = s + G u (u < CPL) and keeps, per candidate, its atom index,
// 1/||a_c||, the correlation c_c = <a_c, r> and its row of Q_C = A_C^T U
// (8 >= Kb entries) in registers.  Per iteration: the argmax over the group,
// the owner of q publishes its row of Q_C (w, the new row of L) through shared
// memory, every lane updates its own candidates from G[q][c] (one load wave),
// so the only shared-memory traffic is the k-vector w.  A patch that is still
// active at iteration `it` has chosen exactly `it` atoms, so the iteration loop
// is unrolled: in each copy the count is a compile-time constant, the dot
// products w . Q_C[c] have exactly `it` terms and the new column of Q_C is a
// plain register write.  FP64 fallback, the explicit residual near the FP32
// floor and the outputs are those of the shared-memory form; with Xh the group
// also writes x_hat = D0_Omega alpha (synth_patch).
// M <= 4 G NCH (NCH float4 chunks of y per lane for p0 = A_C^T y).
// Per-group shared memory: GrpSmem | p0[cap] | parents' child ranges [2 x CSP_MAX_K].
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ int reg_group_bytes(int Kb, int cap, bool gs = false) {
  const int bytes = grp_smem_bytes(Kb, cap) + up16(4 * cap) + 8 * CSP_MAX_K + (gs ? up16(4 * cap * cap) : 0);
  return (bytes + 127) / 128 * 128 + 16;
}

// GS: the patch's Gram block G[C][C] is gathered into shared memory once, after
// the candidates are listed, so that no iteration waits on a load of G[q][C].
template <int G, int CPL, int NCH, bool GS = false>
__global__ void __launch_bounds__(WV_WARPS * 32, CPL >= 6 ? 3 : 4)  // 6-8 candidates a lane: up to 168 registers
omp_restricted_reg_kernel(const float *__restrict__ Y, int M, const float *__restrict__ A,
                          const float *__restrict__ inv_norm, const int32_t *__restrict__ ids, int64_t n,
                          const int32_t *__restrict__ child_off, const int32_t *__restrict__ child_idx,
                          int cap, const int32_t *__restrict__ omega_up, int ldo_up,
                          const int8_t *__restrict__ keff_up, const int8_t *__restrict__ Kp, int Kuni,
                          int Kb, int32_t *__restrict__ omega, float *__restrict__ alpha, int ldo,
                          int8_t *__restrict__ k_eff, int64_t *stats, const float *__restrict__ gram, int T,
                          const float *__restrict__ D0, int N0, float *__restrict__ Xh,
                          const float *__restrict__ p0full) {
  constexpr int KM = 8;
  constexpr int NG = 32 / G;
  extern __shared__ __align__(16) char smem_raw[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, s = lane & (G - 1), g = lane / G;
  const int64_t wbase = ((int64_t)blockIdx.x * WV_WARPS + wib) * NG;
  if (wbase >= n) return;  // whole warp
  const int64_t wi = wbase + g;
  const bool valid = wi < n;
  char *gbase = smem_raw + (size_t)(wib * NG + g) * reg_group_bytes(Kb, cap, GS);
  const GrpSmem S = carve(gbase, Kb, cap);
  float *p0 = reinterpret_cast<float *>(gbase + grp_smem_bytes(Kb, cap));
  int *pstart = reinterpret_cast<int *>(gbase + grp_smem_bytes(Kb, cap) + up16(4 * cap));
  int *pbeg = pstart + CSP_MAX_K;
  float *Gcc = reinterpret_cast<float *>(gbase + grp_smem_bytes(Kb, cap) + up16(4 * cap) + 8 * CSP_MAX_K);
  const int nv = M >> 2;
  const int64_t b = valid ? (ids ? __ldg(ids + wi) : wi) : 0;
  int Kpb = valid ? (Kp ? (int)Kp[b] : Kuni) : 0;
  Kpb = Kpb < Kb ? Kpb : Kb;
  const float *yrow = Y + b * M;
  const float4 *y4 = reinterpret_cast<const float4 *>(yrow);
  // candidates, their inverse norms and p0 = A_C^T y (group-cooperative, in shared memory)
  float4 yv[NCH];
  load_chunks<G, NCH>(yv, yrow, nv, s, valid);
  int nc;
  if (p0full) {
    // full-dictionary level (the Gram form of Algorithm 1): every atom is a
    // candidate, p0 comes from the precomputed correlations P0[b] = A y_b
    nc = valid ? (T < cap ? T : cap) : 0;
    for (int c = s; c < nc; c += G) {
      S.cs[c] = c;
      S.invn[c] = __ldg(inv_norm + c);
      p0[c] = __ldg(p0full + b * (int64_t)T + c);
    }
    __syncwarp();
  } else {
    const int kup = valid ? keff_up[b] : 0;
    nc = gram_setup<G, NCH>(valid, s, b, kup, omega_up, ldo_up, child_off, child_idx, cap, S, pstart, pbeg, inv_norm,
                            stats, M, A, yv, p0);
  }
  const float ysq = gsum<G>(dotc<NCH>(yv, yv));
  if (GS) {  // Gram block of the candidates: Gcc[i * cap + j] = G[C_i][C_j], all loads in flight first
    constexpr int GB = 8;
    const int ncw = __reduce_max_sync(kFull, nc);
    for (int e0 = 0; e0 < ncw * ncw; e0 += GB * G) {
      float v[GB];
#pragma unroll
      for (int t = 0; t < GB; ++t) {
        const int e = e0 + s + t * G, i = e / ncw, j = e - i * ncw;
        v[t] = (e < ncw * ncw && i < nc && j < nc) ? __ldg(gram + (int64_t)S.cs[i] * T + S.cs[j]) : 0.f;
      }
#pragma unroll
      for (int t = 0; t < GB; ++t) {
        const int e = e0 + s + t * G, i = e / ncw, j = e - i * ncw;
        if (e < ncw * ncw && i < nc && j < nc) Gcc[i * cap + j] = v[t];
      }
    }
    __syncwarp();
  }
  // this lane's candidates into registers (u < ucnt: a bound uniform over the warp, <= CPL)
  const int ucnt = __reduce_max_sync(kFull, (nc + G - 1) / G);
  int cs[CPL];
  float inv[CPL], cc[CPL], Q[CPL][KM];
#pragma unroll
  for (int u = 0; u < CPL; ++u) {
    const int c = s + G * u;
    const bool o = u < ucnt && c < nc;
    cs[u] = o ? S.cs[c] : -1;
    inv[u] = o ? S.invn[c] : -1.f;
    cc[u] = o ? p0[c] : 0.f;
#pragma unroll
    for (int j = 0; j < KM; ++j) Q[u][j] = 0.f;
  }
  float zr[KM];  // z_j of the chosen atoms (registers; row it of z is written at iteration it)
#pragma unroll
  for (int j = 0; j < KM; ++j) zr[j] = 0.f;
  float rsq = ysq;
  bool act = valid && Kpb > 0;
  uint8_t fl = 0;  // bit 1: FP64 from here on
  int k = 0, scored = 0;
  const int Kw = __reduce_max_sync(kFull, Kpb);
#pragma unroll
  for (int it = 0; it < KM; ++it) {
    // an active patch has chosen exactly `it` atoms here (k == it)
    if (it >= Kw) break;
    act = act && k < Kpb && !(rsq <= kEpsR32 * ysq);
    if (!__any_sync(kFull, act)) break;
    if (act) ++scored;
    // proxy from the current correlations
    unsigned long long best = 0ull;
#pragma unroll
    for (int u = 0; u < CPL; ++u)
      if (u < ucnt && act && inv[u] > 0.f) {
        const unsigned long long key = pack_key(fabsf(cc[u]) * inv[u], cs[u]);
        best = key > best ? key : best;
      }
    best = gmax<G>(best);
    if (act && !best) act = false;  // candidate set exhausted
    const int q = act ? key_idx(best) : 0;
    const bool f32 = act && !(fl & 2);
    float gpre[CPL];
    float aa = 0.f;
    if (!GS) {  // G[q][C] (row q: G is symmetric) and G[q][q], issued first
#pragma unroll
      for (int u = 0; u < CPL; ++u)
        gpre[u] = (u < ucnt && f32 && cs[u] >= 0) ? __ldg(gram + (int64_t)q * T + cs[u]) : 0.f;
      aa = f32 ? __ldg(gram + (int64_t)q * T + q) : 0.f;
    }
    // the owner of q: no longer eligible; publishes its row of Q_C, its correlation and its slot
#pragma unroll
    for (int u = 0; u < CPL; ++u)
      if (u < ucnt && act && cs[u] == q) {
        inv[u] = -1.f;
#pragma unroll
        for (int j = 0; j < it; ++j) S.V[j] = Q[u][j];
        S.V[Kb] = cc[u];  // V holds Kb + 1 entries; w uses the first it < Kb
        S.misc[1] = s + G * u;
      }
    __syncwarp();
    if (GS) {  // the row of the winner's slot in the staged Gram block
      const float *gr = Gcc + (f32 ? S.misc[1] : 0) * cap;
#pragma unroll
      for (int u = 0; u < CPL; ++u) gpre[u] = (u < ucnt && f32 && cs[u] >= 0) ? gr[s + G * u] : 0.f;
      aa = f32 ? gr[S.misc[1]] : 0.f;
    }
    // new row of L: w_j = <u_j, a_q>, j < it; z_it = c_q / L_kk (c_q = <a_q, y> - w.z)
    float w[KM];
    float ww0 = 0.f, ww1 = 0.f;
#pragma unroll
    for (int j = 0; j < it; ++j) {
      w[j] = f32 ? S.V[j] : 0.f;
      if (j & 1) ww1 = fmaf(w[j], w[j], ww1);
      else ww0 = fmaf(w[j], w[j], ww0);
    }
    const float cq = S.V[Kb];
    const float d = aa - (ww0 + ww1);
    const bool ok32 = f32 && aa > 0.f && d >= kTauPivot * aa;
    if (f32 && !ok32) {
      fl |= 2;
      if (s == 0) atomicAdd((unsigned long long *)&stats[0], 1ull);
    }
    if (ok32) {
      const float il = rsqrtf(d);  // d >= kTauPivot aa > 0
      const float lkk = d * il;
      const float zk = cq * il;
      if (s == 0) {
#pragma unroll
        for (int j = 0; j < it; ++j) S.L[tri(it) + j] = w[j];
        S.L[tri(it) + it] = lkk;
        S.Linv[it] = il;
        S.z[it] = zk;
        S.om[it] = q;
        S.colp[it] = A + (int64_t)q * M;
      }
      zr[it] = zk;
      // column `it` of Q_C and the correlations
#pragma unroll
      for (int u = 0; u < CPL; ++u)
        if (u < ucnt && cs[u] >= 0) {
          float v0 = gpre[u], v1 = 0.f;
#pragma unroll
          for (int j = 0; j < it; ++j) {
            if (j & 1) v1 = fmaf(-w[j], Q[u][j], v1);
            else v0 = fmaf(-w[j], Q[u][j], v0);
          }
          const float v = (v0 + v1) * il;
          Q[u][it] = v;
          cc[u] = fmaf(-zk, v, cc[u]);
        }
      rsq = rsq - zk * zk;
    }
    // FP64 from scratch for the patches whose FP32 pivot failed (now or before)
    const bool go64 = act && !ok32;
    if (go64 && s == 0) S.misc[0] = fp64_projection(M, yrow, S, k, A + (int64_t)q * M) ? 1 : 0;
    __syncwarp();
    const bool app64 = go64 && S.misc[0] != 0;
    // q depends on the chosen columns: alpha of the chosen ones from the FP32 factor
    const bool restore = f32 && !ok32 && !app64;
    if (__any_sync(kFull, restore))
      grp_backsub<G>(restore, s, k - 1, __reduce_max_sync(kFull, restore ? k - 1 : 0), S);
    if (app64 && s == 0) {
      S.om[k] = q;
      S.colp[k] = A + (int64_t)q * M;
    }
    __syncwarp();
    if (app64)  // correlations c = p0 - G[C][Omega] alpha from the Gram rows of the chosen atoms
#pragma unroll
      for (int u = 0; u < CPL; ++u)
        if (u < ucnt && cs[u] >= 0) {
          float v = p0[s + G * u];
          for (int j = 0; j <= k; ++j) v = fmaf(-S.W[j], __ldg(gram + (int64_t)S.om[j] * T + cs[u]), v);
          cc[u] = v;
        }
    // ||r||^2 formed explicitly in FP64 mode and near the FP32 floor
    const bool exact = app64 || (ok32 && rsq <= 1e-5f * ysq);
    if (__any_sync(kFull, exact)) {
      const bool need = exact && !app64;  // FP32: alpha over rows 0..k first
      grp_backsub<G>(need, s, k, __reduce_max_sync(kFull, need ? k : 0), S);
      float r2 = 0.f;
      if (exact)
        for (int j = s; j < nv; j += G) {
          float4 r = __ldg(y4 + j);
          for (int i = 0; i <= k; ++i) {
            const float ai = S.W[i];
            const float4 a = __ldg(reinterpret_cast<const float4 *>(S.colp[i]) + j);
            r.x = fmaf(-ai, a.x, r.x);
            r.y = fmaf(-ai, a.y, r.y);
            r.z = fmaf(-ai, a.z, r.z);
            r.w = fmaf(-ai, a.w, r.w);
          }
          r2 += dot4(r, r);
        }
      r2 = gsum<G>(r2);
      if (exact) rsq = r2;
    }
    if (act) {
      if (ok32 || app64) ++k;
      else act = false;
    }
    __syncwarp();
  }
  // alpha = L^{-T} z for the patches that stayed in FP32 (FP64 ones hold it in S.W)
  const bool fin = valid && !(fl & 2) && k > 0;
  grp_backsub<G>(fin, s, k - 1, __reduce_max_sync(kFull, fin ? k - 1 : 0), S);
  if (valid) {
    if (s == 0) {
      if (k < Kpb) atomicAdd((unsigned long long *)&stats[1], 1ull);
      atomicAdd((unsigned long long *)&stats[2], (unsigned long long)nc * (unsigned long long)scored);
      k_eff[b] = (int8_t)k;
    }
    for (int j = s; j < ldo; j += G) {
      omega[b * ldo + j] = (j < k) ? S.om[j] : -1;
      alpha[b * ldo + j] = (j < k) ? S.W[j] : 0.f;
    }
  }
  // synthesis x_hat_b = D0_Omega alpha (Sec. IV) into Xh[b] when asked for
  if (Xh && valid) synth_patch(D0, N0, Xh + b * N0, S.W, S.om, k, s, G);
}

inline unsigned blocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// (G, NCH): about eight elements per lane.
template <typename F>
bool dispatch_wave(int M, F &&f) {
  if (M % 4) return false;
  if (M <= 16) f(std::integral_constant<int, 4>{}, std::integral_constant<int, 1>{});
  else if (M <= 32) f(std::integral_constant<int, 4>{}, std::integral_constant<int, 2>{});
  else if (M <= 64) f(std::integral_constant<int, 8>{}, std::integral_constant<int, 2>{});
  else if (M <= 128) f(std::integral_constant<int, 16>{}, std::integral_constant<int, 2>{});
  else if (M <= 256) f(std::integral_constant<int, 32>{}, std::integral_constant<int, 2>{});
  else return false;
  return true;
}

int wave_group(int M) { return M <= 32 ? 4 : (M <= 64 ? 8 : (M <= 128 ? 16 : 32)); }

// (G, NCH) of the Batch-OMP restricted kernel: narrow groups by default (its
// per-iteration state is scalar; M-vectors appear only in p0 and the rare
// explicit residual); `width` doubles the lanes per patch once or twice.
int gram_group(int M, int width) {
  const int g = (M <= 64 ? 4 : (M <= 128 ? 8 : 16)) << width;
  return g > 32 ? 32 : g;
}

template <typename F>
bool dispatch_gram(int M, int width, F &&f) {
  if (M % 4 || M > 256) return false;
  const int G = gram_group(M, width);
  int nch = (M / 4 + G - 1) / G;  // chunks of four elements per lane; lanes past M hold zeros
  if (nch == 3) nch = 4;          // (instantiated for 1, 2 and 4 chunks)
  using std::integral_constant;
  switch (G * 8 + nch) {
    case 4 * 8 + 1: f(integral_constant<int, 4>{}, integral_constant<int, 1>{}); break;
    case 4 * 8 + 2: f(integral_constant<int, 4>{}, integral_constant<int, 2>{}); break;
    case 4 * 8 + 4: f(integral_constant<int, 4>{}, integral_constant<int, 4>{}); break;
    case 8 * 8 + 1: f(integral_constant<int, 8>{}, integral_constant<int, 1>{}); break;
    case 8 * 8 + 2: f(integral_constant<int, 8>{}, integral_constant<int, 2>{}); break;
    case 8 * 8 + 4: f(integral_constant<int, 8>{}, integral_constant<int, 4>{}); break;
    case 16 * 8 + 1: f(integral_constant<int, 16>{}, integral_constant<int, 1>{}); break;
    case 16 * 8 + 2: f(integral_constant<int, 16>{}, integral_constant<int, 2>{}); break;
    case 16 * 8 + 4: f(integral_constant<int, 16>{}, integral_constant<int, 4>{}); break;
    case 32 * 8 + 1: f(integral_constant<int, 32>{}, integral_constant<int, 1>{}); break;
    case 32 * 8 + 2: f(integral_constant<int, 32>{}, integral_constant<int, 2>{}); break;
    default: return false;
  }
  return true;
}

}  // namespace

void launch_omp_update_wave(const float *Y, int M, const float *A, const float *inv_norm, const int32_t *ids,
                            int64_t n, int64_t rbf_row0, int n_cand, const int8_t *Kp, int Kuni, OmpState st,
                            int64_t *stats, const float *gram, int T, int64_t a_pstride, int64_t inv_pstride,
                            cudaStream_t s) {
  if (n == 0) return;
  const int per_cta = WV_WARPS * (32 / wave_group(M));
  const size_t sm = (size_t)grp_smem_bytes(st.Kb, 0) * per_cta;
  dispatch_wave(M, [&](auto gc, auto nc) {
    constexpr int GG = decltype(gc)::value, NCH = decltype(nc)::value;
    if (sm > 48 * 1024)
      cudaFuncSetAttribute(omp_update_wave_kernel<GG, NCH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    omp_update_wave_kernel<GG, NCH><<<blocks(n, per_cta), WV_WARPS * 32, sm, s>>>(
        Y, M, A, inv_norm, ids, n, rbf_row0, n_cand, Kp, Kuni, st, stats, gram, T, a_pstride, inv_pstride);
  });
}

size_t restricted_gram_smem(int width, bool qr, int M, int Kb, int cap, bool pp) {
  const bool qr8 = qr && Kb <= 8 && !pp;
  const int per_cta = WV_WARPS * (32 / gram_group(M, width));
  return (size_t)(qr8 ? qr8_group_bytes(Kb, cap) : (qr || pp ? qr_group_bytes(Kb, cap) : gram_group_bytes(Kb, cap))) *
         per_cta;
}

bool launch_omp_restricted_gram(int width, bool qr, const float *Y, int M, const float *A, const float *inv_norm,
                                const int32_t *ids, int64_t n, const int32_t *child_off, const int32_t *child_idx,
                                int cap, const int32_t *omega_up, int ldo_up, const int8_t *keff_up,
                                const int8_t *Kp, int Kuni, int Kb, int32_t *omega, float *alpha, int ldo,
                                int8_t *k_eff, int64_t *stats, const float *gram, int T, const float *D0, int N0,
                                float *Xh, cudaStream_t s, unsigned long long *queue, const float *gpp,
                                int64_t a_pstride, int64_t inv_pstride) {
  if (gpp) qr = true;  // per-patch Gram blocks: the Gram-Schmidt form with Q_C in shared memory
  const bool qr8 = qr && Kb <= 8 && !gpp;  // Q_C stored by candidate
  const bool synth = qr8 && Xh && D0 && N0 > 0 && N0 % 4 == 0;
  if (n == 0) return synth;
  const int per_cta = WV_WARPS * (32 / gram_group(M, width));
  const size_t sm =
      (size_t)(qr8 ? qr8_group_bytes(Kb, cap) : (qr ? qr_group_bytes(Kb, cap) : gram_group_bytes(Kb, cap))) *
      per_cta;
  dispatch_gram(M, width, [&](auto gc, auto nc) {
    constexpr int GG = decltype(gc)::value, NCH = decltype(nc)::value;
    if (qr8) {
      auto kern = omp_restricted_qr8_kernel<GG, NCH>;
      if (sm > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      kern<<<blocks(n, per_cta), WV_WARPS * 32, sm, s>>>(Y, M, A, inv_norm, ids, n, child_off, child_idx, cap,
                                                        omega_up, ldo_up, keff_up, Kp, Kuni, Kb, omega, alpha, ldo,
                                                        k_eff, stats, gram, T, D0, N0, synth ? Xh : nullptr);
      return;
    }
    auto kern = gpp ? (queue ? omp_restricted_qr_kernel<GG, NCH, true, true> : omp_restricted_qr_kernel<GG, NCH, false, true>)
                : queue ? (qr ? omp_restricted_qr_kernel<GG, NCH, true> : omp_restricted_gram_kernel<GG, NCH, true>)
                        : (qr ? omp_restricted_qr_kernel<GG, NCH, false> : omp_restricted_gram_kernel<GG, NCH, false>);
    if (sm > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    unsigned grid = blocks(n, per_cta);
    if (queue) {  // persistent: as many CTAs as fit at once, fed by the work queue
      int per_sm = 0, dev = 0;
      cudaGetDevice(&dev);
      int sms = 1;
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, WV_WARPS * 32, sm) != cudaSuccess || per_sm < 1)
        per_sm = 1;
      grid = std::min<unsigned>(grid, (unsigned)(per_sm * sms));
      cudaMemsetAsync(queue, 0, sizeof(unsigned long long), s);
    }
    kern<<<grid, WV_WARPS * 32, sm, s>>>(Y, M, A, inv_norm, ids, n, child_off, child_idx, cap, omega_up, ldo_up,
                                         keff_up, Kp, Kuni, Kb, omega, alpha, ldo, k_eff, stats, gram, T, queue, gpp,
                                         a_pstride, inv_pstride);
  });
  return synth;
}

bool launch_omp_restricted_reg(int G, const float *Y, int M, const float *A, const float *inv_norm,
                               const int32_t *ids, int64_t n, const int32_t *child_off, const int32_t *child_idx,
                               int cap, const int32_t *omega_up, int ldo_up, const int8_t *keff_up,
                               const int8_t *Kp, int Kuni, int Kb, int32_t *omega, float *alpha, int ldo,
                               int8_t *k_eff, int64_t *stats, const float *gram, int T, const float *D0, int N0,
                               float *Xh, bool *synthesized, cudaStream_t s, bool stage_gram) {
  *synthesized = false;
  if (M % 4 || Kb > 8 || (G != 4 && G != 8 && G != 16)) return false;
  // float4 chunks of y per lane: 4 lanes take M <= 64 (4 chunks), 8 and 16 lanes two chunks
  const int nch = G == 4 ? 4 : 2;
  if (M > 4 * G * nch) return false;
  const int per_g = (cap + G - 1) / G;
  const int CPL = per_g <= 2 ? 2 : (per_g <= 3 ? 3 : (per_g <= 4 ? 4 : (per_g <= 6 ? 6 : (per_g <= 8 ? 8 : 0))));
  if (!CPL) return false;
  const bool synth = Xh && D0 && N0 > 0 && N0 % 4 == 0;
  // the staged Gram block needs cap^2 floats per patch: up to 32 candidates
  const bool gs = stage_gram && cap <= 32;
  if (stage_gram && !gs) return false;
  *synthesized = synth;
  if (n == 0) return true;
  const int per_cta = WV_WARPS * (32 / G);
  const size_t sm = (size_t)reg_group_bytes(Kb, cap, gs) * per_cta;
  auto go = [&](auto kern) {
    if (sm > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    kern<<<blocks(n, per_cta), WV_WARPS * 32, sm, s>>>(Y, M, A, inv_norm, ids, n, child_off, child_idx, cap, omega_up,
                                                      ldo_up, keff_up, Kp, Kuni, Kb, omega, alpha, ldo, k_eff, stats,
                                                      gram, T, D0, N0, synth ? Xh : nullptr, nullptr);
  };
  switch ((gs ? 10000 : 0) + G * 100 + CPL) {
    case 402: go(omp_restricted_reg_kernel<4, 2, 4>); break;
    case 403: go(omp_restricted_reg_kernel<4, 3, 4>); break;
    case 404: go(omp_restricted_reg_kernel<4, 4, 4>); break;
    case 406: go(omp_restricted_reg_kernel<4, 6, 4>); break;
    case 408: go(omp_restricted_reg_kernel<4, 8, 4>); break;
    case 802: go(omp_restricted_reg_kernel<8, 2, 2>); break;
    case 803: go(omp_restricted_reg_kernel<8, 3, 2>); break;
    case 804: go(omp_restricted_reg_kernel<8, 4, 2>); break;
    case 806: go(omp_restricted_reg_kernel<8, 6, 2>); break;
    case 808: go(omp_restricted_reg_kernel<8, 8, 2>); break;
    case 1602: go(omp_restricted_reg_kernel<16, 2, 2>); break;
    case 1603: go(omp_restricted_reg_kernel<16, 3, 2>); break;
    case 1604: go(omp_restricted_reg_kernel<16, 4, 2>); break;
    case 1606: go(omp_restricted_reg_kernel<16, 6, 2>); break;
    case 1608: go(omp_restricted_reg_kernel<16, 8, 2>); break;
    case 10402: go(omp_restricted_reg_kernel<4, 2, 4, true>); break;
    case 10403: go(omp_restricted_reg_kernel<4, 3, 4, true>); break;
    case 10404: go(omp_restricted_reg_kernel<4, 4, 4, true>); break;
    case 10406: go(omp_restricted_reg_kernel<4, 6, 4, true>); break;
    case 10408: go(omp_restricted_reg_kernel<4, 8, 4, true>); break;
    case 10802: go(omp_restricted_reg_kernel<8, 2, 2, true>); break;
    case 10803: go(omp_restricted_reg_kernel<8, 3, 2, true>); break;
    case 10804: go(omp_restricted_reg_kernel<8, 4, 2, true>); break;
    case 11602: go(omp_restricted_reg_kernel<16, 2, 2, true>); break;
    default: return false;
  }
  return true;
}

bool full_gram_supported(int M, int T, int Kb) { return M % 4 == 0 && M <= 256 && T >= 1 && T <= 256 && Kb <= 8; }

bool launch_omp_full_gram(const float *Y, int M, const float *A, const float *inv_norm, const int32_t *ids, int64_t n,
                          const int8_t *Kp, int Kuni, int Kb, int32_t *omega, float *alpha, int ldo, int8_t *k_eff,
                          int64_t *stats, const float *gram, int T, float *P0, cudaStream_t s) {
  if (!full_gram_supported(M, T, Kb) || !gram || !P0) return false;
  if (n == 0) return true;
  constexpr int G = 32;
  const int per_g = (T + G - 1) / G;
  const int CPL = per_g <= 2 ? 2 : (per_g <= 4 ? 4 : 8);
  const int per_cta = WV_WARPS * (32 / G);
  const size_t sm = (size_t)reg_group_bytes(Kb, T) * per_cta;
  auto go = [&](auto kern) {
    if (sm > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    kern<<<blocks(n, per_cta), WV_WARPS * 32, sm, s>>>(Y, M, A, inv_norm, ids, n, nullptr, nullptr, T, nullptr, 0,
                                                      nullptr, Kp, Kuni, Kb, omega, alpha, ldo, k_eff, stats, gram, T,
                                                      nullptr, 0, nullptr, P0);
  };
  switch ((M <= 128 ? 10 : 20) + CPL) {
    case 12: go(omp_restricted_reg_kernel<32, 2, 1>); break;
    case 14: go(omp_restricted_reg_kernel<32, 4, 1>); break;
    case 18: go(omp_restricted_reg_kernel<32, 8, 1>); break;
    case 22: go(omp_restricted_reg_kernel<32, 2, 2>); break;
    case 24: go(omp_restricted_reg_kernel<32, 4, 2>); break;
    default: go(omp_restricted_reg_kernel<32, 8, 2>); break;
  }
  return true;
}

}  // namespace csp
