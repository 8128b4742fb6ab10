// Dictionary learning kernels: the K-SVD dictionary-update sweep and the
// initialisation picks of the modified K-SVD.
//
//  * Sec. II, "Dictionary learning": K-SVD alternates sparse coding with an
//    atom-by-atom dictionary update; visiting atom k, the error matrix E_k of
//    the signals that use k (their residuals with k's term added back) is
//    replaced by its best rank-one fit d_k (E_k^T d_k)^T, d_k the leading
//    left singular vector.  Visits are sequential: atom k sees the residuals
//    left by the visits of atoms 0 .. k-1.
//  * Sec. III, "Learning cross-scale sparse models": the same sweep learns the
//    coarse dictionary (on W X) and the fine one (supports restricted to the
//    children of the coarse supports by the sparse-coding step).
//  * Sec. III, "Initialization of dictionary": heuristics 1-2 (atoms picked
//    from the training signals, for a fine atom from the signals whose coarse
//    support holds its parent) and 3-4 (an unused atom becomes the signal with
//    the largest residual, for a fine atom among those same signals).
//
// Data layout (device): D [T][M] atom-major, X and the residuals R [N][M],
// supports / coefficients [N][Kmax] as the solver writes them.
//
// Pipeline of one sweep:
//  1. ksvd_prep_kernel   r_i = x_i - sum_j alpha_ij d_omega_ij, ||r_i||^2,
//                        ||x_i||^2, support checks, per-chunk atom counts.
//  2. ksvd_scan_kernel   per-atom prefix over chunks, exclusive scan over atoms.
//  3. ksvd_fill_kernel   stable counting sort: the slots (i, j) of every atom
//                        in ascending signal order (deterministic, no atomics
//                        on global memory).
//  4. ksvd_sweep_kernel  one thread-block cluster visits the atoms in order.
//     Per atom: each CTA accumulates C_r = sum e_i e_i^T over the users it
//     owns (i mod CL == rank); the power method on C = E_k E_k^T = sum_r C_r
//     from d_old multiplies each C_r locally and adds the kCL products through
//     distributed shared memory in rank order (one cluster barrier per step,
//     identical vectors and decisions on every rank); each CTA then updates
//     the coefficients and residuals of its own users.  Ownership by signal
//     keeps every residual with one CTA: successive atoms exchange nothing else.
//  5. ksvd_sum_kernel    ||X - D S||_F^2 after the sweep (optional).

#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "csp_internal.cuh"

namespace cg = cooperative_groups;

namespace csp {

namespace {

constexpr int kChunk = 256;       // signals per counting chunk
constexpr int kCL = 8;            // CTAs of the sweep's cluster
constexpr int kMaxIt = 1000;      // power-iteration cap per atom
constexpr float kTol2 = 1.6e-11f; // converged when ||v_new - v||^2 <= (4e-6)^2

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__device__ __forceinline__ float warp_sum(float s) {
#pragma unroll
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

// 1. Residuals, norms, support checks and per-chunk atom counts.
// err bits: 1 = k_eff outside [0, Kmax], 2 = atom id outside [0, T),
// 4 = an atom repeated within one support.  R == nullptr: counts and checks only.
__global__ void ksvd_prep_kernel(const float *__restrict__ D, int M, int T, const float *__restrict__ X, int N,
                                 const int32_t *__restrict__ sup, const float *__restrict__ coef,
                                 const int8_t *__restrict__ keff, int Kmax, int split, float *__restrict__ R,
                                 float *__restrict__ rn2, float *__restrict__ xn2, int *__restrict__ hist,
                                 unsigned *err) {
  extern __shared__ int h[];
  const int nkeys = T * split;
  for (int t = threadIdx.x; t < nkeys; t += blockDim.x) h[t] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int i0 = blockIdx.x * kChunk, i1 = min(N, i0 + kChunk);
  for (int i = i0 + warp; i < i1; i += nw) {
    int k = keff[i];
    unsigned e = 0;
    if (k < 0 || k > Kmax) { e |= 1; k = 0; }
    if (lane < k) {
      const int a = sup[(size_t)i * Kmax + lane];
      if (a < 0 || a >= T) e |= 2;
      else {
        bool dup = false;
        for (int j = 0; j < lane; ++j) dup |= sup[(size_t)i * Kmax + j] == a;
        if (dup) e |= 4;
        atomicAdd(&h[a * split + i % split], 1);
      }
    }
    e = __reduce_or_sync(0xffffffffu, e);
    if (e && lane == 0) atomicOr(err, e);
    if (!R) continue;
    float rs = 0.f, xs = 0.f;
    for (int m = lane; m < M; m += 32) {
      const float x = X[(size_t)i * M + m];
      float r = x;
      for (int j = 0; j < k; ++j) {
        const int a = sup[(size_t)i * Kmax + j];
        if (a >= 0 && a < T) r = fmaf(-coef[(size_t)i * Kmax + j], D[(size_t)a * M + m], r);
      }
      R[(size_t)i * M + m] = r;
      rs = fmaf(r, r, rs);
      xs = fmaf(x, x, xs);
    }
    rs = warp_sum(rs);
    xs = warp_sum(xs);
    if (lane == 0) { rn2[i] = rs; xn2[i] = xs; }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < nkeys; t += blockDim.x) hist[(size_t)blockIdx.x * nkeys + t] = h[t];
}

// 2. hist[c][t] <- slots of key t in chunks before c; off[t] = first slot of key t
// (T here counts keys: atoms x owner ranks).
__global__ void __launch_bounds__(1024) ksvd_scan_kernel(int *__restrict__ hist, int C, int T, int *__restrict__ off) {
  __shared__ int wsum[32];
  __shared__ int carry;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int t0 = 0; t0 < T; t0 += 1024) {
    const int t = t0 + threadIdx.x;
    int tot = 0;
    if (t < T)
      for (int c = 0; c < C; ++c) {
        const int v = hist[(size_t)c * T + t];
        hist[(size_t)c * T + t] = tot;
        tot += v;
      }
    int x = tot;  // inclusive warp scan
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
      int w = wsum[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += y;
      }
      wsum[lane] = w;
    }
    __syncthreads();
    const int excl = carry + (warp ? wsum[warp - 1] : 0) + x - tot;
    if (t < T) off[t] = excl;
    __syncthreads();
    if (threadIdx.x == 1023) carry = excl + tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) off[T] = carry;
}

// 3. Stable counting sort of the slots q = i * Kmax + j by key a * split + i % split
// (atom a, owner rank i mod split; one warp per chunk).
__global__ void ksvd_fill_kernel(const int32_t *__restrict__ sup, const int8_t *__restrict__ keff, int N, int Kmax,
                                 int T, int split, const int *__restrict__ hist, const int *__restrict__ off,
                                 int32_t *__restrict__ seg) {
  extern __shared__ int base[];
  const int lane = threadIdx.x, nkeys = T * split;
  for (int t = lane; t < nkeys; t += 32) base[t] = off[t] + hist[(size_t)blockIdx.x * nkeys + t];
  __syncwarp();
  const int i0 = blockIdx.x * kChunk, i1 = min(N, i0 + kChunk);
  const int q1 = i1 * Kmax;
  for (int q0 = i0 * Kmax; q0 < q1; q0 += 32) {
    const int q = q0 + lane;
    int a = -1;
    if (q < q1) {
      const int i = q / Kmax, j = q - i * Kmax;
      const int k = keff[i];
      if (k >= 0 && k <= Kmax && j < k) {
        a = sup[q];
        a = (a < 0 || a >= T) ? -1 : a * split + i % split;
      }
    }
    const unsigned peers = __match_any_sync(0xffffffffu, a);
    int pos = 0;
    if (a >= 0) pos = base[a] + __popc(peers & lanemask_lt());
    __syncwarp();
    if (a >= 0) {
      seg[pos] = q;
      if (lane == __ffs(peers) - 1) base[a] += __popc(peers);
    }
    __syncwarp();
  }
}

// TR consecutive floats of shared memory at p (16-byte aligned for TR % 4 == 0,
// 8-byte aligned for TR % 2 == 0) with the widest loads that fit.
template <int TR>
__device__ __forceinline__ void lds_run(float (&o)[TR], const float *p) {
  if constexpr (TR % 4 == 0) {
#pragma unroll
    for (int t = 0; t < TR / 4; ++t) {
      const float4 v = reinterpret_cast<const float4 *>(p)[t];
      o[4 * t] = v.x; o[4 * t + 1] = v.y; o[4 * t + 2] = v.z; o[4 * t + 3] = v.w;
    }
  } else if constexpr (TR % 2 == 0) {
#pragma unroll
    for (int t = 0; t < TR / 2; ++t) {
      const float2 v = reinterpret_cast<const float2 *>(p)[t];
      o[2 * t] = v.x; o[2 * t + 1] = v.y;
    }
  } else {
#pragma unroll
    for (int t = 0; t < TR; ++t) o[t] = p[t];
  }
}

struct SweepArgs {
  float *D;
  int M, T;
  const float *X;
  int N;
  float *coef;
  int Kmax;
  const int *off;          // [T * kCL + 1]: slots of (atom k, owner rank r) at off[k * kCL + r] ..
  const int32_t *seg;      // slot ids q = i * Kmax + j, ascending i within each (k, r)
  float *R, *rn2;
  const float *xn2;
  uint8_t *taken;
  int replace;
  const int32_t *rparent, *rsup;
  int Kc;
  unsigned long long *stats;  // [0] power-method steps, [1] replaced atoms
};

__host__ __device__ constexpr int pad4(int n) { return (n + 3) & ~3; }

// Stage capacity (floats) of the e_i columns: kNB-free sizing by dimension.
__host__ __device__ constexpr int stage_floats(int side) { return side == 16 ? 16384 : 12288; }

// Shared-memory floats of the sweep: this rank's partial C ([M][M + 1]), the
// exchanged products C_r v (2 x M),
// share, the staged columns, the vectors and the slot lists.
__host__ __device__ inline int sweep_smem_floats(int M, int MP, int side) {
  const int CCP = pad4(M * (M + 1)), RB = 2 * pad4(M);
  const int NB = stage_floats(side) / MP;
  return CCP + RB + stage_floats(side) + 10 * pad4(M) + 128 + 6 * NB;
}

// 4. The sweep.  Threads form a SIDE x SIDE grid; thread (ty, tx) accumulates
// the TR x TR tile of C at rows ty*TR.., columns tx*TR.. (SIDE*TR >= M).
// Rank r of the cluster owns the signals i with i mod kCL == r: it reads and
// writes only their residuals and coefficients, so the visits of successive
// atoms need no exchange beyond the Gram matrix.
template <int SIDE, int TR>
__global__ void __launch_bounds__(SIDE *SIDE, 1) ksvd_sweep_kernel(const SweepArgs a) {
  constexpr int NT = SIDE * SIDE, NW = NT / 32, MP = SIDE * TR;
  constexpr int NB = stage_floats(SIDE) / MP;     // columns staged at once
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  extern __shared__ float4 smem4[];
  float *sm = reinterpret_cast<float *>(smem4);
  const int M = a.M, LDC = M + 1, CCP = pad4(M * LDC), Kmax = a.Kmax;
  float *Cb = sm;                        // [M][M + 1] this rank's partial C_r = sum e_i e_i^T
  float *yx = Cb + CCP;                  // [2][pad4(M)] C_r v of the last two steps (read by all ranks)
  float *stage = yx + 2 * pad4(M);       // [NB][MP] e_i of the staged users
  float *dold0 = stage + stage_floats(SIDE), *dold1 = dold0 + pad4(M);  // atom before the visit (2 buffers)
  float *const vb0 = dold0 + 2 * pad4(M), *const vb1 = dold0 + 3 * pad4(M);  // power-method vectors
  float *ysum = dold0 + 4 * pad4(M);     // [M] C v = sum over ranks of C_r v
  float *dd = dold0 + 5 * pad4(M);       // [M] squared change of each component
  float *yp = dold0 + 6 * pad4(M);       // [4][M] partial sums of C v
  float *scal = dold0 + 10 * pad4(M);    // [128] flags, per-warp argmax scratch
  int *ents0 = reinterpret_cast<int *>(scal + 128), *ents1 = ents0 + NB;  // staged slot ids (2 buffers)
  float *als0 = reinterpret_cast<float *>(ents1 + NB), *als1 = als0 + NB;  // their coefficients before the visit
  int *rows0 = reinterpret_cast<int *>(als1 + NB), *rows1 = rows0 + NB;     // their signals i = q / Kmax
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ty = tid / SIDE, tx = tid - ty * SIDE, r0 = ty * TR, c0 = tx * TR;
  float *slotv = scal + 8;                      // best replacement candidate of this rank
  int *sloti = reinterpret_cast<int *>(scal + 9);
  float *wv = scal + 32;                        // [32] per-warp best residual norm
  int *wi = reinterpret_cast<int *>(scal + 64); // [32] ... and its signal
  unsigned long long steps = 0, replaced = 0;
  unsigned gstep = 0;                   // power-method steps of this sweep (product buffer parity)

  for (int q = tid; q < stage_floats(SIDE); q += NT) stage[q] = 0.f;  // padding rows stay zero
  {  // slot ids, coefficients and atom of the first visit
    const int br = a.off[rank], nr = a.off[rank + 1] - br;
    for (int c = tid; c < min(nr, min(NB, NT)); c += NT) {
      ents0[c] = a.seg[br + c];
      als0[c] = a.coef[ents0[c]];
      rows0[c] = ents0[c] / Kmax;
    }
    for (int m = tid; m < M; m += NT) dold0[m] = a.D[m];
  }
  __syncthreads();
  for (int k = 0; k < a.T; ++k) {
    const int kb = a.off[k * kCL], nk = a.off[(k + 1) * kCL] - kb;
    const int br = a.off[k * kCL + rank], nr = a.off[k * kCL + rank + 1] - br;
    float *dold = (k & 1) ? dold1 : dold0;
    int *ents = (k & 1) ? ents1 : ents0;
    float *als = (k & 1) ? als1 : als0;
    int *rows = (k & 1) ? rows1 : rows0;
    // Prefetch of the next visit's slot ids, coefficients and atom: none of
    // them changes during this visit (a slot belongs to one atom, D[k + 1] is
    // written only by its own visit).  Stored after this visit.
    int pq = -1;
    float pa = 0.f, pd = 0.f;
    if (k + 1 < a.T) {
      const int br1 = a.off[(k + 1) * kCL + rank], nr1 = a.off[(k + 1) * kCL + rank + 1] - br1;
      if (tid < min(nr1, NB)) {
        pq = a.seg[br1 + tid];
        pa = a.coef[pq];
      }
      if (tid < M) pd = a.D[(size_t)(k + 1) * M + tid];
    }

    if (nk == 0) {
      // Heuristics 3 / 4: the unused atom becomes the eligible signal with the
      // largest residual norm (ties: lowest index); the signal is then taken.
      if (!a.replace) goto next;
      float bv = -1.f;
      int bi = -1;
      const int pk = a.rparent ? a.rparent[k] : -1;
      for (int i = rank + kCL * tid; i < a.N; i += kCL * NT) {
        if (a.taken[i] || !(a.xn2[i] > 0.f)) continue;
        if (a.rparent) {
          bool ok = false;
          for (int q = 0; q < a.Kc; ++q) ok |= a.rsup[(size_t)i * a.Kc + q] == pk;
          if (!ok) continue;
        }
        const float r = a.rn2[i];
        if (r > bv) { bv = r; bi = i; }
      }
#pragma unroll
      for (int o = 16; o; o >>= 1) {
        const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (oi >= 0 && (ov > bv || (ov == bv && (bi < 0 || oi < bi)))) { bv = ov; bi = oi; }
      }
      if (lane == 0) { wv[warp] = bv; wi[warp] = bi; }
      __syncthreads();
      if (tid == 0) {
        float gv = -1.f;
        int gi = -1;
        for (int w = 0; w < NW; ++w) {
          const float ov = wv[w];
          const int oi = wi[w];
          if (oi >= 0 && (ov > gv || (ov == gv && (gi < 0 || oi < gi)))) { gv = ov; gi = oi; }
        }
        *slotv = gv;
        *sloti = gi;
      }
      cl.sync();
      float gv = -1.f;
      int gi = -1;
      for (int q = 0; q < kCL; ++q) {
        const float ov = *cl.map_shared_rank(slotv, q);
        const int oi = *cl.map_shared_rank(sloti, q);
        if (oi >= 0 && (ov > gv || (ov == gv && (gi < 0 || oi < gi)))) { gv = ov; gi = oi; }
      }
      cl.sync();
      if (gi >= 0) {
        ++replaced;
        if (tid == 0 && gi % kCL == rank) a.taken[gi] = 1;
        if (rank == 0 && warp == 0) {
          float s = 0.f;
          for (int m = lane; m < M; m += 32) {
            const float x = a.X[(size_t)gi * M + m];
            s = fmaf(x, x, s);
          }
          const float nrm = sqrtf(warp_sum(s));
          for (int m = lane; m < M; m += 32) a.D[(size_t)k * M + m] = a.X[(size_t)gi * M + m] / nrm;
        }
      }
      goto next;
    }

    {  // ---- partial C = sum e_i e_i^T over this rank's users, in slot order ----
    // e_i = r_i + alpha_ik d_old for staged columns 0 .. nb-1: a warp per
    // column, SU columns' loads in flight per warp.
    auto stage_cols = [&](int nb) {
      constexpr int SU = NT >= 1024 ? 2 : 4, PL = (MP + 31) / 32;
      for (int cb = warp; cb < nb; cb += SU * NW) {
        float e[SU][PL];
#pragma unroll
        for (int u = 0; u < SU; ++u) {
          const int c = cb + u * NW;
          const float *rr = a.R + (size_t)rows[c < nb ? c : 0] * M;
          const float al = als[c < nb ? c : 0];
#pragma unroll
          for (int t = 0; t < PL; ++t) {
            const int m = lane + 32 * t;
            e[u][t] = (c < nb && m < M) ? fmaf(al, dold[m], rr[m]) : 0.f;
          }
        }
#pragma unroll
        for (int u = 0; u < SU; ++u) {
          const int c = cb + u * NW;
          if (c < nb)
#pragma unroll
            for (int t = 0; t < PL; ++t) {
              const int m = lane + 32 * t;
              if (m < M) stage[c * MP + m] = e[u][t];
            }
        }
      }
    };
    float acc[TR][TR];
#pragma unroll
    for (int i = 0; i < TR; ++i)
#pragma unroll
      for (int j = 0; j < TR; ++j) acc[i][j] = 0.f;
    for (int b0 = 0; b0 < nr; b0 += NB) {
      const int nb = min(NB, nr - b0);
      for (int c = (b0 == 0 ? NT : 0) + tid; c < nb; c += NT) {   // the first NT of batch 0 are prefetched
        const int q = a.seg[br + b0 + c];
        ents[c] = q;
        als[c] = a.coef[q];
        rows[c] = q / Kmax;
      }
      __syncthreads();
      stage_cols(nb);
      __syncthreads();
#pragma unroll 2
      for (int c = 0; c < nb; ++c) {
        const float *ec = stage + c * MP;
        float er[TR], ek[TR];
        lds_run<TR>(er, ec + r0);
        lds_run<TR>(ek, ec + c0);
#pragma unroll
        for (int i = 0; i < TR; ++i)
#pragma unroll
          for (int j = 0; j < TR; ++j) acc[i][j] = fmaf(er[i], ek[j], acc[i][j]);
      }
      if (b0 + NB < nr) __syncthreads();   // the last batch stays staged for the update
    }
#pragma unroll
    for (int i = 0; i < TR; ++i)
#pragma unroll
      for (int j = 0; j < TR; ++j)
        if (r0 + i < M && c0 + j < M) Cb[(r0 + i) * LDC + c0 + j] = acc[i][j];

    for (int m = tid; m < M; m += NT) vb0[m] = dold[m];
    __syncthreads();

    // ---- leading eigenvector of C = sum_r C_r by the power method from d_old ----
    // The ranks never form C: step t computes C_r v_t locally (thread (part,
    // r) sums column range `part` of row r, read as column r of the symmetric
    // C_r: consecutive lanes, consecutive banks), publishes it, and after one
    // cluster barrier every rank adds the kCL products in rank order, so all
    // ranks hold the same y = C v_t and take the same decisions.  v_{t+1} =
    // y / ||y||; the change ||v_{t+1} - v_t||^2 is summed one step later; stop
    // when it is <= kTol2.  The two product buffers alternate by step, so a
    // rank may overwrite one only after every rank has passed the barrier that
    // follows its reads (the alternation runs on across visits).
    int cur = 0;
    bool zero = false;
    constexpr int PARTS = NT / MP >= 4 ? 4 : (NT / MP >= 2 ? 2 : 1);
    const int CW = (M + PARTS - 1) / PARTS;
    for (int it = 0; it < kMaxIt; ++it) {
      const float *v = cur ? vb1 : vb0;
      float *vn = cur ? vb0 : vb1;
      float *yo = yx + (gstep & 1) * pad4(M);
      ++gstep;
      for (int t = tid; t < PARTS * M; t += NT) {
        const int part = t / M, r = t - part * M;
        const int ca = part * CW, cz = min(M, ca + CW);
        float s0 = 0.f, s1 = 0.f;
        int c = ca;
        for (; c + 1 < cz; c += 2) {
          s0 = fmaf(Cb[c * LDC + r], v[c], s0);
          s1 = fmaf(Cb[(c + 1) * LDC + r], v[c + 1], s1);
        }
        if (c < cz) s0 = fmaf(Cb[c * LDC + r], v[c], s0);
        yp[part * M + r] = s0 + s1;
      }
      __syncthreads();
      for (int m = tid; m < M; m += NT) {
        float ym = yp[m];
#pragma unroll
        for (int q = 1; q < PARTS; ++q) ym += yp[q * M + m];
        yo[m] = ym;
      }
      cl.sync();
      for (int m = tid; m < M; m += NT) {
        float ym = 0.f;
#pragma unroll
        for (int q = 0; q < kCL; ++q) ym += cl.map_shared_rank(yo, q)[m];
        ysum[m] = ym;
      }
      __syncthreads();
      float ss = 0.f, d2 = 0.f;
      for (int m = lane; m < M; m += 32) {
        ss = fmaf(ysum[m], ysum[m], ss);
        if (it) d2 += dd[m];
      }
      ss = warp_sum(ss);
      d2 = warp_sum(d2);
      if (it && d2 <= kTol2) { steps += it; break; }   // v_t is converged
      if (!(ss > 0.f)) { zero = true; steps += it; break; }
      const float inv = 1.f / sqrtf(ss);
      __syncthreads();                                  // every warp has read dd
      for (int m = tid; m < M; m += NT) {
        const float nv = ysum[m] * inv;
        const float d = nv - v[m];
        dd[m] = d * d;
        vn[m] = nv;
      }
      __syncthreads();
      cur ^= 1;
      if (it == kMaxIt - 1) steps += kMaxIt;
    }
    float *v = zero ? dold : (cur ? vb1 : vb0);
    {  // sign: <d_new, d_old> >= 0 (every warp computes it; all agree)
      float s = 0.f;
      for (int m = lane; m < M; m += 32) s = fmaf(v[m], dold[m], s);
      s = warp_sum(s);
      if (s < 0.f) {
        __syncthreads();
        for (int m = tid; m < M; m += NT) v[m] = -v[m];
      }
      __syncthreads();
    }
    if (rank == 0)
      for (int m = tid; m < M; m += NT) a.D[(size_t)k * M + m] = v[m];

    // ---- coefficients E_k^T d_k and residuals of this rank's users ----
    // A warp per column, four columns in flight per warp.
    auto update_cols = [&](int nbat) {
      for (int cb = warp; cb < nbat; cb += 4 * NW) {
        float dt[4] = {0.f, 0.f, 0.f, 0.f}, rs[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int c = cb + u * NW;
          if (c < nbat) {
            const float *ec = stage + c * MP;
            for (int m = lane; m < M; m += 32) dt[u] = fmaf(ec[m], v[m], dt[u]);
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) dt[u] = warp_sum(dt[u]);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int c = cb + u * NW;
          if (c < nbat) {
            const float *ec = stage + c * MP;
            float *ri = a.R + (size_t)rows[c] * M;
            for (int m = lane; m < M; m += 32) {
              const float r = fmaf(-dt[u], v[m], ec[m]);
              ri[m] = r;
              rs[u] = fmaf(r, r, rs[u]);
            }
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) rs[u] = warp_sum(rs[u]);
        if (lane == 0)
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int c = cb + u * NW;
            if (c < nbat) {
              a.coef[ents[c]] = dt[u];
              a.rn2[rows[c]] = rs[u];
            }
          }
      }
    };
    if (nr > NB) {   // restage batch by batch
      for (int b0 = 0; b0 < nr; b0 += NB) {
        const int nb = min(NB, nr - b0);
        __syncthreads();
        for (int c = tid; c < nb; c += NT) {
          const int q = a.seg[br + b0 + c];
          ents[c] = q;
          als[c] = a.coef[q];
          rows[c] = q / Kmax;
        }
        __syncthreads();
        stage_cols(nb);
        __syncthreads();
        update_cols(nb);
      }
    } else {         // all users still staged from the Gram pass
      update_cols(nr);
    }
    }  // visit
  next:
    __syncthreads();   // this visit is done with every buffer
    if (tid < NB) {
      ((k & 1) ? ents0 : ents1)[tid] = pq;
      ((k & 1) ? als0 : als1)[tid] = pa;
      ((k & 1) ? rows0 : rows1)[tid] = pq >= 0 ? pq / Kmax : 0;
    }
    if (tid < M) ((k & 1) ? dold0 : dold1)[tid] = pd;
    __syncthreads();
  }
  if (rank == 0 && tid == 0 && a.stats) {
    a.stats[0] = steps;
    a.stats[1] = replaced;
  }
  cl.sync();  // no CTA leaves while another may still read its shared memory
}

// 5. ||X - D S||_F^2 = sum of the residual norms (fixed order).
__global__ void __launch_bounds__(1024) ksvd_sum_kernel(const float *__restrict__ rn2, int N, float *out) {
  __shared__ float ws[32];
  float s = 0.f;
  for (int i = threadIdx.x; i < N; i += 1024) s += rn2[i];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = warp_sum(ws[threadIdx.x]);
    if (threadIdx.x == 0) *out = s;
  }
}

// Initialisation picks (heuristics 1 and 2): atom t = x_i / ||x_i||, with
// i = floor(u_t n) of the pool: all N signals (off == nullptr, or an empty
// pool), else the signals whose coarse support holds parent[t] (slots of the
// sorted coarse supports, Kc per signal).  A zero signal leaves the atom as is.
__global__ void ksvd_init_kernel(float *__restrict__ D, int M, int T, const float *__restrict__ X, int N,
                                 const int32_t *__restrict__ parent, const int *__restrict__ off,
                                 const int32_t *__restrict__ seg, int Kc, const double *__restrict__ u) {
  const int lane = threadIdx.x & 31;
  const int t = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (t >= T || N <= 0) return;
  int i;
  int n = 0, b = 0;
  if (off) {
    const int k = parent[t];
    b = off[k];
    n = off[k + 1] - b;
  }
  if (n > 0) {
    int q = (int)floor(u[t] * (double)n);
    if (q > n - 1) q = n - 1;
    i = seg[b + q] / Kc;
  } else {
    int q = (int)floor(u[t] * (double)N);
    if (q > N - 1) q = N - 1;
    i = q;
  }
  float s = 0.f;
  for (int m = lane; m < M; m += 32) {
    const float x = X[(size_t)i * M + m];
    s = fmaf(x, x, s);
  }
  s = warp_sum(s);
  if (!(s > 0.f)) return;
  const float nrm = sqrtf(s);
  for (int m = lane; m < M; m += 32) D[(size_t)t * M + m] = X[(size_t)i * M + m] / nrm;
}

template <int SIDE, int TR>
cudaError_t launch_sweep_t(const SweepArgs &a, cudaStream_t s) {
  constexpr int NT = SIDE * SIDE;
  const size_t smem = (size_t)sweep_smem_floats(a.M, SIDE * TR, SIDE) * 4;
  cudaError_t e = cudaFuncSetAttribute(ksvd_sweep_kernel<SIDE, TR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(kCL);
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = kCL;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, ksvd_sweep_kernel<SIDE, TR>, a);
}

}  // namespace

int ksvd_owner_split() { return kCL; }

size_t ksvd_sweep_smem_bytes(int M) {
  if (M <= 16) return (size_t)sweep_smem_floats(M, 16, 16) * 4;
  if (M <= 32) return (size_t)sweep_smem_floats(M, 32, 16) * 4;
  if (M <= 48) return (size_t)sweep_smem_floats(M, 48, 16) * 4;
  if (M <= 64) return (size_t)sweep_smem_floats(M, 64, 16) * 4;
  if (M <= 128) return (size_t)sweep_smem_floats(M, 128, 16) * 4;
  return (size_t)sweep_smem_floats(M, 192, 32) * 4;
}

int ksvd_chunks(int64_t N) { return (int)((N + kChunk - 1) / kChunk); }

void launch_ksvd_sort(const float *D, int M, int T, const float *X, int N, const int32_t *sup, const float *coef,
                      const int8_t *keff, int Kmax, int split, float *R, float *rn2, float *xn2, int *hist, int *off,
                      int32_t *seg, unsigned *err, cudaStream_t s) {
  const int C = ksvd_chunks(N), nkeys = T * split;
  if (C > 0) {
    cudaFuncSetAttribute(ksvd_prep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, nkeys * 4);
    ksvd_prep_kernel<<<C, 256, (size_t)nkeys * 4, s>>>(D, M, T, X, N, sup, coef, keff, Kmax, split, R, rn2, xn2,
                                                         hist, err);
  }
  ksvd_scan_kernel<<<1, 1024, 0, s>>>(hist, C, nkeys, off);
  if (C > 0) {
    cudaFuncSetAttribute(ksvd_fill_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, nkeys * 4);
    ksvd_fill_kernel<<<C, 32, (size_t)nkeys * 4, s>>>(sup, keff, N, Kmax, T, split, hist, off, seg);
  }
}

cudaError_t launch_ksvd_sweep(float *D, int M, int T, const float *X, int N, float *coef, int Kmax, const int *off,
                              const int32_t *seg, float *R, float *rn2, const float *xn2, uint8_t *taken, int replace,
                              const int32_t *rparent, const int32_t *rsup, int Kc, unsigned long long *stats,
                              cudaStream_t s) {
  SweepArgs a{D, M, T, X, N, coef, Kmax, off, seg, R, rn2, xn2, taken, replace, rparent, rsup, Kc, stats};
  if (M <= 16) return launch_sweep_t<16, 1>(a, s);
  if (M <= 32) return launch_sweep_t<16, 2>(a, s);
  if (M <= 48) return launch_sweep_t<16, 3>(a, s);
  if (M <= 64) return launch_sweep_t<16, 4>(a, s);
  if (M <= 128) return launch_sweep_t<16, 8>(a, s);
  return launch_sweep_t<32, 6>(a, s);
}

void launch_ksvd_sum(const float *rn2, int N, float *out, cudaStream_t s) {
  ksvd_sum_kernel<<<1, 1024, 0, s>>>(rn2, N, out);
}

void launch_ksvd_init(float *D, int M, int T, const float *X, int N, const int32_t *parent, const int *off,
                      const int32_t *seg, int Kc, const double *u, cudaStream_t s) {
  ksvd_init_kernel<<<(T + 7) / 8, 256, 0, s>>>(D, M, T, X, N, parent, off, seg, Kc, u);
}

}  // namespace csp
