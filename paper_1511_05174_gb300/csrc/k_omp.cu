// Batched OMP kernels (Algorithm 1; fine steps of Algorithm 2).
//
// Per patch and iteration OMP does (Sec. II-B):
//   proxy       k = argmax_i |<a_i, r>| / ||a_i||   (angle reading; chosen and
//               zero columns excluded; ties to the lowest index)
//   merge       Omega <- Omega u {k}
//   projection  alpha = argmin ||y - A_Omega b||, here by an incremental
//               Cholesky factor L L^T = A_Omega^T A_Omega: new row
//               w = L^{-1} A_Omega^T a_k, pivot sqrt(||a_k||^2 - ||w||^2);
//               z = L^{-1} A_Omega^T y grows by one entry; alpha = L^{-T} z
//   residue     r = y - A_Omega alpha
// When the pivot ratio (||a_k||^2 - ||w||^2) / ||a_k||^2 falls below
// kTauPivot the factor is rebuilt from scratch in FP64 for that patch, which
// also decides linear dependence (L_kk <= kEpsD64 ||a_k||) like a QR pivot.
//
// Kernels:
//   proxy_fp32_kernel      full-dictionary proxy, FP32 CUDA-core GEMM of a tile of
//                          64 residuals against all atoms, fused |.|/norm, mask and
//                          argmax (one candidate per patch)
//   omp_update_kernel      one warp per patch: (re-score candidates in FP32,) merge,
//                          projection and residue; state in global memory
//   omp_restricted_kernel  one warp per patch, all iterations of the restricted OMP
//                          over the children f(Omega_up) of the coarser support
#include "csp_internal.cuh"

namespace csp {

namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ int tri(int i) { return (i * (i + 1)) >> 1; }

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}
__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    const unsigned long long w = __shfl_xor_sync(kFull, v, o);
    v = w > v ? w : v;
  }
  return v;
}
// Packed argmax key: larger score first, then lower index.  0 = no candidate.
__device__ __forceinline__ unsigned long long pack_key(float score, int idx) {
  return ((unsigned long long)__float_as_uint(score) << 32) | (0xffffffffu - (unsigned)idx);
}
__device__ __forceinline__ int key_idx(unsigned long long k) {
  return (int)(0xffffffffu - (unsigned)(k & 0xffffffffull));
}

// ---------------------------------------------------------------------------
// Shared projection step: append column q to the support of one patch.
//
// Lanes hold y, r and a_q over m = lane + 32 t.  L (packed), z, omega and alpha
// live in global or shared memory (generic pointers).  Returns 1 when q was
// appended (alpha, r, rsq updated), 0 when q depends on the chosen columns
// (nothing changes; the patch ends).
// ---------------------------------------------------------------------------
template <int MPL>
__device__ int omp_append(int lane, int M, const float *__restrict__ A, int q,
                          const float (&aq)[MPL], const float (&yv)[MPL], float (&rv)[MPL], int k,
                          int32_t *omega, float *alpha, float *L, float *z, uint8_t &fl,
                          double *L64, float &rsq, int64_t *stats) {
  if (!(fl & 2)) {
    // Gram column v_j = <a_{omega_j}, a_q>, lane j keeps v_j.
    float vj = 0.f;
    for (int j = 0; j < k; ++j) {
      const float *aj = A + (int64_t)omega[j] * M;
      float p = 0.f;
#pragma unroll
      for (int t = 0; t < MPL; ++t) {
        const int m = lane + 32 * t;
        if (m < M) p = fmaf(__ldg(aj + m), aq[t], p);
      }
      p = warp_sum(p);
      if (lane == j) vj = p;
    }
    float aa = 0.f;
#pragma unroll
    for (int t = 0; t < MPL; ++t) aa = fmaf(aq[t], aq[t], aa);
    aa = warp_sum(aa);
    // w = L^{-1} v (column-oriented forward substitution across lanes)
    for (int i = 0; i < k; ++i) {
      const float wi = __shfl_sync(kFull, vj, i) / L[tri(i) + i];
      if (lane == i) vj = wi;
      else if (lane > i && lane < k) vj = fmaf(-L[tri(lane) + i], wi, vj);
    }
    const float ww = warp_sum(lane < k ? vj * vj : 0.f);
    const float d = aa - ww;
    if (d >= kTauPivot * aa && aa > 0.f) {
      const float lkk = sqrtf(d);
      float bq = 0.f;
#pragma unroll
      for (int t = 0; t < MPL; ++t) bq = fmaf(aq[t], yv[t], bq);
      bq = warp_sum(bq);
      const float zprev = (lane < k) ? z[lane] : 0.f;
      const float zz = warp_sum(lane < k ? vj * zprev : 0.f);
      const float zk = (bq - zz) / lkk;
      __syncwarp();
      if (lane < k) L[tri(k) + lane] = vj;
      if (lane == 0) { L[tri(k) + k] = lkk; z[k] = zk; omega[k] = q; }
      __syncwarp();
      // alpha = L^{-T} z (column-oriented back substitution; lane i ends with alpha_i)
      float acc = (lane < k) ? zprev : (lane == k ? zk : 0.f);
      for (int j = k; j >= 0; --j) {
        const float aj = __shfl_sync(kFull, acc, j) / L[tri(j) + j];
        if (lane == j) acc = aj;
        else if (lane < j) acc = fmaf(-L[tri(j) + lane], aj, acc);
      }
      if (lane <= k) alpha[lane] = acc;
      // residue r = y - A_Omega alpha
      float r2 = 0.f;
#pragma unroll
      for (int t = 0; t < MPL; ++t) rv[t] = yv[t];
      for (int j = 0; j <= k; ++j) {
        const float aj = __shfl_sync(kFull, acc, j);
        if (j == k) {
#pragma unroll
          for (int t = 0; t < MPL; ++t) rv[t] = fmaf(-aj, aq[t], rv[t]);
        } else {
          const float *col = A + (int64_t)omega[j] * M;
#pragma unroll
          for (int t = 0; t < MPL; ++t) {
            const int m = lane + 32 * t;
            if (m < M) rv[t] = fmaf(-aj, __ldg(col + m), rv[t]);
          }
        }
      }
#pragma unroll
      for (int t = 0; t < MPL; ++t) r2 = fmaf(rv[t], rv[t], r2);
      rsq = warp_sum(r2);
      __syncwarp();
      return 1;
    }
    // Low pivot ratio: switch this patch to FP64 projections for good.
    fl |= 2;
    if (lane == 0 && stats) atomicAdd((unsigned long long *)&stats[0], 1ull);
  }
  // FP64 path: rebuild the Cholesky factor of A_S^T A_S for S = omega[0..k-1] + q,
  // entry by entry (all lanes compute the same scalars; lane 0 stores).
  for (int i = 0; i <= k; ++i) {
    const float *ci = (i < k) ? A + (int64_t)omega[i] * M : nullptr;
    for (int j = 0; j <= i; ++j) {
      const float *cj = (j < k) ? A + (int64_t)omega[j] * M : nullptr;
      double g = 0.0;
#pragma unroll
      for (int t = 0; t < MPL; ++t) {
        const int m = lane + 32 * t;
        if (m < M) {
          const double u = ci ? (double)__ldg(ci + m) : (double)aq[t];
          const double v = cj ? (double)__ldg(cj + m) : (double)aq[t];
          g = fma(u, v, g);
        }
      }
      g = warp_sum_d(g);
      double s = g;
      for (int p = 0; p < j; ++p) s -= L64[tri(i) + p] * L64[tri(j) + p];
      double val;
      if (j < i) {
        val = s / L64[tri(j) + j];
      } else {
        if (i == k && !(s > kEpsD64 * kEpsD64 * g)) return 0;  // dependent column
        val = sqrt(s > 0.0 ? s : 0.0);
      }
      __syncwarp();
      if (lane == 0) L64[tri(i) + j] = val;
      __syncwarp();
    }
  }
  // z = L^{-1} A_S^T y, alpha = L^{-T} z, serially in FP64 (identical on all lanes).
  double zb[CSP_MAX_K + 1];
  for (int i = 0; i <= k; ++i) {
    const float *ci = (i < k) ? A + (int64_t)omega[i] * M : nullptr;
    double bi = 0.0;
#pragma unroll
    for (int t = 0; t < MPL; ++t) {
      const int m = lane + 32 * t;
      if (m < M) bi = fma(ci ? (double)__ldg(ci + m) : (double)aq[t], (double)yv[t], bi);
    }
    bi = warp_sum_d(bi);
    for (int p = 0; p < i; ++p) bi -= L64[tri(i) + p] * zb[p];
    zb[i] = bi / L64[tri(i) + i];
  }
  for (int i = k; i >= 0; --i) {
    double s = zb[i];
    for (int j = i + 1; j <= k; ++j) s -= L64[tri(j) + i] * zb[j];
    zb[i] = s / L64[tri(i) + i];  // zb now holds alpha_i for indices >= i
  }
  __syncwarp();
  if (lane == 0) omega[k] = q;
  if (lane <= k) {
    double a = 0.0;
    for (int i = 0; i <= k; ++i) if (i == lane) a = zb[i];
    alpha[lane] = (float)a;
  }
  __syncwarp();
  double rr[MPL];
#pragma unroll
  for (int t = 0; t < MPL; ++t) rr[t] = (double)yv[t];
  for (int j = 0; j <= k; ++j) {
    const float *col = (j < k) ? A + (int64_t)omega[j] * M : nullptr;
#pragma unroll
    for (int t = 0; t < MPL; ++t) {
      const int m = lane + 32 * t;
      if (m < M) rr[t] -= zb[j] * (col ? (double)__ldg(col + m) : (double)aq[t]);
    }
  }
  float r2 = 0.f;
#pragma unroll
  for (int t = 0; t < MPL; ++t) {
    const int m = lane + 32 * t;
    rv[t] = (m < M) ? (float)rr[t] : 0.f;
    r2 = fmaf(rv[t], rv[t], r2);
  }
  rsq = warp_sum(r2);
  return 1;
}

template <int MPL>
__device__ __forceinline__ void load_vec(float (&v)[MPL], const float *__restrict__ p, int M, int lane) {
#pragma unroll
  for (int t = 0; t < MPL; ++t) {
    const int m = lane + 32 * t;
    v[t] = (m < M) ? __ldg(p + m) : 0.f;
  }
}

template <int MPL>
__device__ __forceinline__ float dot_vec(const float (&v)[MPL], const float *__restrict__ p, int M, int lane) {
  float s = 0.f;
#pragma unroll
  for (int t = 0; t < MPL; ++t) {
    const int m = lane + 32 * t;
    if (m < M) s = fmaf(__ldg(p + m), v[t], s);
  }
  return warp_sum(s);
}

// ---------------------------------------------------------------------------
// State initialisation: r = y, empty supports.
// ---------------------------------------------------------------------------
__global__ void omp_init_kernel(const float *__restrict__ Y, int64_t B, int M, int Mp, OmpState st) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < B * M) st.R[e] = Y[e];
  if (st.Rbf && e < B * Mp) {
    const int64_t b = e / Mp;
    const int m = (int)(e - b * Mp);
    st.Rbf[e] = __float2bfloat16_rn(m < M ? Y[b * M + m] : 0.f);
  }
  if (e < B * st.ldo) { st.omega[e] = -1; st.alpha[e] = 0.f; }
  if (e < B) { st.k_eff[e] = 0; st.flags[e] = 0; }
}

// ---------------------------------------------------------------------------
// FP32 proxy: tile of 64 patches x all atoms.  256 threads as 16 x 16, each
// owning 4 patches x 4 atoms of every 64-atom tile.
// ---------------------------------------------------------------------------
constexpr int PX_TP = 64, PX_TA = 64, PX_KC = 32, PX_AS = PX_TA + 4;

__global__ void __launch_bounds__(256)
proxy_fp32_kernel(const float *__restrict__ R, int M, const float *__restrict__ A,
                  const float *__restrict__ inv_norm, int T, const int32_t *__restrict__ ids,
                  int64_t n, const int32_t *__restrict__ omega, int ldo,
                  const int8_t *__restrict__ k_eff, const uint8_t *__restrict__ flags,
                  int32_t *__restrict__ cand) {
  extern __shared__ __align__(16) float smem[];
  const int Mr = (M + PX_KC - 1) / PX_KC * PX_KC;
  float *Rs = smem;                      // [Mr][PX_TP]  residuals, measurement-major
  float *As = Rs + (size_t)Mr * PX_TP;   // [PX_KC][PX_AS] atom chunk, measurement-major
  int *Om = (int *)(As + PX_KC * PX_AS); // [PX_TP][ldo]
  int *Kc = Om + PX_TP * ldo;            // [PX_TP]
  const int tid = threadIdx.x;
  const int64_t p0 = (int64_t)blockIdx.x * PX_TP;

  for (int e = tid; e < PX_TP * Mr; e += 256) {
    const int p = e / Mr, m = e - p * Mr;
    const int64_t pi = p0 + p;
    float v = 0.f;
    if (pi < n && m < M) {
      const int64_t b = ids ? ids[pi] : pi;
      v = R[b * M + m];
    }
    Rs[m * PX_TP + p] = v;
  }
  for (int e = tid; e < PX_TP * ldo; e += 256) {
    const int p = e / ldo, j = e - p * ldo;
    const int64_t pi = p0 + p;
    Om[e] = (pi < n) ? omega[(ids ? ids[pi] : pi) * ldo + j] : -1;
  }
  for (int p = tid; p < PX_TP; p += 256) {
    const int64_t pi = p0 + p;
    Kc[p] = (pi < n) ? k_eff[ids ? ids[pi] : pi] : 0;
  }

  const int ty = tid >> 4, tx = tid & 15;
  unsigned long long best[4] = {0ull, 0ull, 0ull, 0ull};
  for (int a0 = 0; a0 < T; a0 += PX_TA) {
    float acc[4][4] = {};
    for (int m0 = 0; m0 < Mr; m0 += PX_KC) {
      __syncthreads();
      for (int e = tid; e < PX_TA * PX_KC; e += 256) {
        const int a = e / PX_KC, mm = e - a * PX_KC;
        const int ai = a0 + a, m = m0 + mm;
        As[mm * PX_AS + a] = (ai < T && m < M) ? __ldg(A + (int64_t)ai * M + m) : 0.f;
      }
      __syncthreads();
#pragma unroll 8
      for (int mm = 0; mm < PX_KC; ++mm) {
        const float4 rv = *reinterpret_cast<const float4 *>(Rs + (m0 + mm) * PX_TP + ty * 4);
        const float4 av = *reinterpret_cast<const float4 *>(As + mm * PX_AS + tx * 4);
        const float r4[4] = {rv.x, rv.y, rv.z, rv.w};
        const float a4[4] = {av.x, av.y, av.z, av.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(r4[i], a4[j], acc[i][j]);
      }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int ai = a0 + tx * 4 + j;
      if (ai >= T) continue;
      const float inv = __ldg(inv_norm + ai);
      if (!(inv > 0.f)) continue;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const unsigned long long key = pack_key(fabsf(acc[i][j]) * inv, ai);
        if (key > best[i]) {
          const int p = ty * 4 + i;
          bool chosen = false;
          for (int q = 0; q < Kc[p]; ++q) chosen |= (Om[p * ldo + q] == ai);
          if (!chosen) best[i] = key;
        }
      }
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    unsigned long long v = best[i];
#pragma unroll
    for (int o = 8; o; o >>= 1) {
      const unsigned long long w = __shfl_xor_sync(kFull, v, o);
      v = w > v ? w : v;
    }
    const int64_t pi = p0 + ty * 4 + i;
    if (tx == 0 && pi < n) {
      const int64_t b = ids ? ids[pi] : pi;
      cand[b * kTopP] = v ? key_idx(v) : -1;
#pragma unroll
      for (int c = 1; c < kTopP; ++c) cand[b * kTopP + c] = -1;
    }
  }
}

// ---------------------------------------------------------------------------
// Update: one warp per patch of the id list.
// ---------------------------------------------------------------------------
template <int MPL>
__global__ void __launch_bounds__(256)
omp_update_kernel(const float *__restrict__ Y, int M, const float *__restrict__ A,
                  const float *__restrict__ inv_norm, const int32_t *__restrict__ ids, int64_t n,
                  int n_cand, const int8_t *__restrict__ Kp, int Kuni, OmpState st, int64_t *stats) {
  extern __shared__ __align__(16) double smem64[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t wi = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
  if (wi >= n) return;
  const int64_t b = ids ? ids[wi] : wi;
  uint8_t fl = st.flags[b];
  if (fl & 1) return;
  const int k = st.k_eff[b];
  int Kb = Kp ? (int)Kp[b] : Kuni;
  Kb = Kb < st.Kb ? Kb : st.Kb;
  int32_t *om = st.omega + b * st.ldo;
  float *al = st.alpha + b * st.ldo;
  if (k >= Kb) {
    if (lane == 0) st.flags[b] = fl | 1;
    return;
  }
  float yv[MPL], rv[MPL];
  load_vec<MPL>(yv, Y + b * M, M, lane);
  load_vec<MPL>(rv, st.R + b * M, M, lane);
  const float ysq = warp_sum([&] { float s = 0.f;
#pragma unroll
    for (int t = 0; t < MPL; ++t) s = fmaf(yv[t], yv[t], s); return s; }());
  float rsq0 = 0.f;
#pragma unroll
  for (int t = 0; t < MPL; ++t) rsq0 = fmaf(rv[t], rv[t], rsq0);
  rsq0 = warp_sum(rsq0);
  if (rsq0 <= kEpsR32 * ysq) {
    if (lane == 0) { st.flags[b] = fl | 1; atomicAdd((unsigned long long *)&stats[1], 1ull); }
    return;
  }
  // Candidate choice: the FP32 proxy's argmax, or the best of the re-scored top candidates.
  const int32_t *cb = st.cand + b * kTopP;
  int q = -1;
  if (n_cand <= 1) {
    q = cb[0];
  } else {
    unsigned long long best = 0ull;
    for (int c = 0; c < n_cand; ++c) {
      const int a = cb[c];
      if (a < 0) continue;
      const float inv = __ldg(inv_norm + a);
      if (!(inv > 0.f)) continue;
      const bool chosen = __any_sync(kFull, lane < k && om[lane] == a);
      if (chosen) continue;
      const float s = fabsf(dot_vec<MPL>(rv, A + (int64_t)a * M, M, lane)) * inv;
      const unsigned long long key = pack_key(s, a);
      best = key > best ? key : best;
    }
    q = best ? key_idx(best) : -1;
  }
  if (q < 0) {
    if (lane == 0) { st.flags[b] = fl | 1; atomicAdd((unsigned long long *)&stats[1], 1ull); }
    return;
  }
  float aq[MPL];
  load_vec<MPL>(aq, A + (int64_t)q * M, M, lane);
  double *L64 = smem64 + (size_t)wib * tri(st.Kb + 1);
  float rsq = 0.f;
  const int ok = omp_append<MPL>(lane, M, A, q, aq, yv, rv, k, om, al, st.Lpk + b * tri(st.Kb),
                                 st.z + b * st.Kb, fl, L64, rsq, stats);
  if (!ok) {
    if (lane == 0) { st.flags[b] = fl | 1; atomicAdd((unsigned long long *)&stats[1], 1ull); }
    return;
  }
#pragma unroll
  for (int t = 0; t < MPL; ++t) {
    const int m = lane + 32 * t;
    if (m < M) st.R[b * M + m] = rv[t];
  }
  if (st.Rbf) {
    const int Mp = (M + 63) / 64 * 64;
    for (int t = 0; t < (Mp + 31) / 32; ++t) {
      const int m = lane + 32 * t;
      float v = 0.f;
#pragma unroll
      for (int u = 0; u < MPL; ++u) if (u == t) v = rv[u];
      if (m < Mp) st.Rbf[b * Mp + m] = __float2bfloat16_rn(m < M ? v : 0.f);
    }
  }
  if (lane == 0) {
    st.k_eff[b] = (int8_t)(k + 1);
    uint8_t nf = fl;
    if (k + 1 >= Kb) nf |= 1;
    if (rsq <= kEpsR32 * ysq) nf |= 1;
    if ((nf & 1) && k + 1 < Kb) atomicAdd((unsigned long long *)&stats[1], 1ull);
    st.flags[b] = nf;
  }
}

// ---------------------------------------------------------------------------
// Restricted OMP (fine step of Algorithm 2): one warp per patch, all iterations.
// Candidates C = children of the coarser support (disjoint lists, since every
// fine atom has one parent), proxy over C only, projection as above.
// ---------------------------------------------------------------------------
constexpr int RS_WARPS = 4;

template <int MPL>
__global__ void __launch_bounds__(RS_WARPS * 32)
omp_restricted_kernel(const float *__restrict__ Y, int M, const float *__restrict__ A,
                      const float *__restrict__ inv_norm, const int32_t *__restrict__ ids, int64_t n,
                      const int32_t *__restrict__ child_off, const int32_t *__restrict__ child_idx,
                      int cap, const int32_t *__restrict__ omega_up, int ldo_up,
                      const int8_t *__restrict__ keff_up, const int8_t *__restrict__ Kp, int Kuni,
                      int Kb, int32_t *__restrict__ omega, float *__restrict__ alpha, int ldo,
                      int8_t *__restrict__ k_eff, int64_t *stats) {
  extern __shared__ __align__(16) double smem64[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  // per-warp shared layout: L64 | L | z | alpha | r | omega | cand
  const int n64 = tri(Kb + 1);
  const int nf = tri(Kb) + 2 * Kb + M;
  const int per_warp_bytes = ((n64 * 8 + nf * 4 + (Kb + cap) * 4) + 15) / 16 * 16;
  char *base = reinterpret_cast<char *>(smem64) + (size_t)wib * per_warp_bytes;
  double *L64 = reinterpret_cast<double *>(base);
  float *Ls = reinterpret_cast<float *>(base + n64 * 8);
  float *zs = Ls + tri(Kb);
  float *as = zs + Kb;
  float *rs = as + Kb;
  int32_t *oms = reinterpret_cast<int32_t *>(rs + M);
  int32_t *cs = oms + Kb;

  const int64_t wi = (int64_t)blockIdx.x * RS_WARPS + wib;
  if (wi >= n) return;
  const int64_t b = ids ? ids[wi] : wi;
  int Kpb = Kp ? (int)Kp[b] : Kuni;
  Kpb = Kpb < Kb ? Kpb : Kb;

  // candidate set f(Omega_up)
  int nc = 0;
  const int kup = keff_up[b];
  bool overflow = false;
  for (int j = 0; j < kup; ++j) {
    const int p = omega_up[b * ldo_up + j];
    const int s = child_off[p], e = child_off[p + 1];
    for (int i = lane; i < e - s; i += 32)
      if (nc + i < cap) cs[nc + i] = child_idx[s + i];
    nc += e - s;
  }
  if (nc > cap) { overflow = true; nc = cap; }
  if (overflow && lane == 0) atomicAdd((unsigned long long *)&stats[3], 1ull);
  __syncwarp();

  float yv[MPL], rv[MPL];
  load_vec<MPL>(yv, Y + b * M, M, lane);
#pragma unroll
  for (int t = 0; t < MPL; ++t) {
    rv[t] = yv[t];
    const int m = lane + 32 * t;
    if (m < M) rs[m] = yv[t];
  }
  float ysq = 0.f;
#pragma unroll
  for (int t = 0; t < MPL; ++t) ysq = fmaf(yv[t], yv[t], ysq);
  ysq = warp_sum(ysq);
  float rsq = ysq;
  unsigned sel = 0u;  // bit t: candidate slot lane + 32 t already chosen
  uint8_t fl = 0;
  int k = 0, scored = 0;
  __syncwarp();
  while (k < Kpb) {
    if (rsq <= kEpsR32 * ysq) break;
    ++scored;
    unsigned long long best = 0ull;
    for (int c = lane, t = 0; c < nc; c += 32, ++t) {
      if ((sel >> t) & 1u) continue;
      const int a = cs[c];
      const float inv = __ldg(inv_norm + a);
      if (!(inv > 0.f)) continue;
      const float *col = A + (int64_t)a * M;
      float s = 0.f;
      for (int m = 0; m < M; ++m) s = fmaf(__ldg(col + m), rs[m], s);
      const unsigned long long key = pack_key(fabsf(s) * inv, a);
      best = key > best ? key : best;
    }
    best = warp_max_u64(best);
    if (!best) break;  // candidate set exhausted
    const int q = key_idx(best);
    for (int c = lane, t = 0; c < nc; c += 32, ++t)
      if (cs[c] == q) sel |= 1u << t;
    float aq[MPL];
    load_vec<MPL>(aq, A + (int64_t)q * M, M, lane);
    const int ok = omp_append<MPL>(lane, M, A, q, aq, yv, rv, k, oms, as, Ls, zs, fl, L64, rsq, stats);
    if (!ok) break;
    ++k;
#pragma unroll
    for (int t = 0; t < MPL; ++t) {
      const int m = lane + 32 * t;
      if (m < M) rs[m] = rv[t];
    }
    __syncwarp();
  }
  if (lane == 0) {
    if (k < Kpb) atomicAdd((unsigned long long *)&stats[1], 1ull);
    atomicAdd((unsigned long long *)&stats[2], (unsigned long long)nc * (unsigned long long)scored);
  }
  for (int j = lane; j < ldo; j += 32) {
    omega[b * ldo + j] = (j < k) ? oms[j] : -1;
    alpha[b * ldo + j] = (j < k) ? as[j] : 0.f;
  }
  if (lane == 0) k_eff[b] = (int8_t)k;
}

inline unsigned blocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

template <typename F>
void dispatch_mpl(int M, F &&f) {
  if (M <= 32) f(std::integral_constant<int, 1>{});
  else if (M <= 64) f(std::integral_constant<int, 2>{});
  else if (M <= 128) f(std::integral_constant<int, 4>{});
  else f(std::integral_constant<int, 8>{});
}

}  // namespace

void launch_omp_init(const float *Y, int64_t B, int M, int Mp, OmpState st, cudaStream_t s) {
  int64_t n = B * (int64_t)(M > Mp ? M : Mp);
  n = n > B * st.ldo ? n : B * st.ldo;
  if (n == 0) return;
  omp_init_kernel<<<blocks(n, 256), 256, 0, s>>>(Y, B, M, Mp, st);
}

void launch_proxy_fp32(const float *R, int M, const float *A, const float *inv_norm, int T,
                       const int32_t *ids, int64_t n, const int32_t *omega, int ldo,
                       const int8_t *k_eff, const uint8_t *flags, int32_t *cand, cudaStream_t s) {
  if (n == 0) return;
  const int Mr = (M + PX_KC - 1) / PX_KC * PX_KC;
  const size_t sm = sizeof(float) * ((size_t)Mr * PX_TP + PX_KC * PX_AS) + sizeof(int) * (PX_TP * ldo + PX_TP);
  static size_t configured = 0;
  if (sm > 48 * 1024 && sm > configured) {
    cudaFuncSetAttribute(proxy_fp32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    configured = sm;
  }
  proxy_fp32_kernel<<<blocks(n, PX_TP), 256, sm, s>>>(R, M, A, inv_norm, T, ids, n, omega, ldo, k_eff,
                                                      flags, cand);
}

void launch_omp_update(const float *Y, int M, const float *A, const float *inv_norm,
                       const int32_t *ids, int64_t n, int n_cand, const int8_t *Kp, int Kuni,
                       OmpState st, int64_t *stats, cudaStream_t s) {
  if (n == 0) return;
  const size_t sm = sizeof(double) * 8 * ((st.Kb + 1) * (st.Kb + 2) / 2);
  dispatch_mpl(M, [&](auto c) {
    constexpr int MPL = decltype(c)::value;
    omp_update_kernel<MPL><<<blocks(n, 8), 256, sm, s>>>(Y, M, A, inv_norm, ids, n, n_cand, Kp, Kuni,
                                                          st, stats);
  });
}

void launch_omp_restricted(const float *Y, int M, const float *A, const float *inv_norm,
                           const int32_t *ids, int64_t n, const int32_t *child_off,
                           const int32_t *child_idx, int cap, const int32_t *omega_up, int ldo_up,
                           const int8_t *keff_up, const int8_t *Kp, int Kuni, int Kb,
                           int32_t *omega, float *alpha, int ldo, int8_t *k_eff, int64_t *stats,
                           cudaStream_t s) {
  if (n == 0) return;
  const int n64 = (Kb + 1) * (Kb + 2) / 2;
  const int nf = Kb * (Kb + 1) / 2 + 2 * Kb + M;
  const size_t per_warp = ((size_t)(n64 * 8 + nf * 4 + (Kb + cap) * 4) + 15) / 16 * 16;
  const size_t sm = per_warp * RS_WARPS;
  dispatch_mpl(M, [&](auto c) {
    constexpr int MPL = decltype(c)::value;
    if (sm > 48 * 1024)
      cudaFuncSetAttribute(omp_restricted_kernel<MPL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    omp_restricted_kernel<MPL><<<blocks(n, RS_WARPS), RS_WARPS * 32, sm, s>>>(
        Y, M, A, inv_norm, ids, n, child_off, child_idx, cap, omega_up, ldo_up, keff_up, Kp, Kuni, Kb,
        omega, alpha, ldo, k_eff, stats);
  });
}

bool proxy_bf16_supported(int M, int T) { (void)M; (void)T; return false; }

void launch_proxy_bf16(const __nv_bfloat16 *, int, const __nv_bfloat16 *, int, const int32_t *,
                       int64_t, const uint8_t *, int32_t *, cudaStream_t) {}

}  // namespace csp
