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
//     from d_old multiplies each C_r locally and adds the CL products through
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
#include "ksvd.cuh"

namespace cg = cooperative_groups;

namespace csp {

namespace {

constexpr int kChunk = 256;       // signals per counting chunk
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
  const int *off;          // [T * CL + 1]: slots of (atom k, owner rank r) at off[k * CL + r] ..
  const int32_t *seg;      // slot ids q = i * Kmax + j, ascending i within each (k, r)
  float *R, *rn2;
  const float *xn2;
  uint8_t *taken;
  int replace;
  const int32_t *rparent, *rsup;
  int Kc;
  unsigned long long *stats;  // [0] power-method steps, [1] replaced atoms
  int approx;                 // 1: one alternating step from the current coefficients
};


// Stage capacity (floats) of the e_i columns: kNB-free sizing by dimension.
__host__ __device__ constexpr int stage_floats(int side) { return side == 16 ? 16384 : 12288; }

// Shared-memory floats of the sweep: the products C_q v received from every
// rank q (2 x CL x MP),
// share, the staged columns, the vectors and the slot lists.
__host__ __device__ inline int sweep_smem_floats(int MP, int side, int CL) {
  const int NB = stage_floats(side) / MP;
  return 2 * CL * MP + stage_floats(side) + 8 * MP + 128 + 6 * NB;
}

// 4. The sweep.  Threads form a SIDE x SIDE grid; thread (ty, tx) accumulates
// the TR x TR tile of C at rows ty*TR.., columns tx*TR.. (SIDE*TR >= M).
// Rank r of the cluster owns the signals i with i mod CL == r: it reads and
// writes only their residuals and coefficients, so the visits of successive
// atoms need no exchange beyond the Gram matrix.
template <int SIDE, int TR, int CL>
__global__ void __launch_bounds__(SIDE *SIDE, 1) ksvd_sweep_kernel(const SweepArgs a) {
  constexpr int NT = SIDE * SIDE, NW = NT / 32, MP = SIDE * TR;
  constexpr int NB = stage_floats(SIDE) / MP;     // columns staged at once
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  extern __shared__ float4 smem4[];
  float *sm = reinterpret_cast<float *>(smem4);
  const int M = a.M, Kmax = a.Kmax;
  float *rx = sm;                        // [2][CL][MP] C_q v pushed by every rank q (two step parities)
  float *stage = rx + 2 * CL * MP;       // [NB][MP] e_i of the staged users
  float *dold0 = stage + stage_floats(SIDE), *dold1 = dold0 + MP;  // atom before the visit (2 buffers)
  float *const vb0 = dold0 + 2 * MP, *const vb1 = dold0 + 3 * MP;  // power-method vectors (zero past M)
  float *yl = dold0 + 4 * MP;            // [MP] this rank's C_r v
  float *ysum = dold0 + 5 * MP;          // [MP] C v
  float *scal = dold0 + 8 * MP;          // [128] flags, per-warp argmax scratch
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
  for (int q = tid; q < 2 * MP; q += NT) vb0[q] = 0.f;                 // entries past M stay zero
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
    const int kb = a.off[k * CL], nk = a.off[(k + 1) * CL] - kb;
    const int br = a.off[k * CL + rank], nr = a.off[k * CL + rank + 1] - br;
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
      const int br1 = a.off[(k + 1) * CL + rank], nr1 = a.off[(k + 1) * CL + rank + 1] - br1;
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
      for (int i = rank + CL * tid; i < a.N; i += CL * NT) {
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
#pragma unroll 1
      for (int q = 0; q < CL; ++q) {
        const float ov = *cl.map_shared_rank(slotv, q);
        const int oi = *cl.map_shared_rank(sloti, q);
        if (oi >= 0 && (ov > gv || (ov == gv && (gi < 0 || oi < gi)))) { gv = ov; gi = oi; }
      }
      cl.sync();
      if (gi >= 0) {
        ++replaced;
        if (tid == 0 && gi % CL == rank) a.taken[gi] = 1;
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
    float ya = 0.f;   // approximate update: (E_r^T alpha_r)[tid], over this rank's users in slot order
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
      if (a.approx) {
        if (tid < M)
          for (int c = 0; c < nb; ++c) ya = fmaf(stage[c * MP + tid], als[c], ya);
      } else
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
    // acc now holds this thread's tile of C_r (zero past M) and stays in registers

    // y = sum over ranks of yl (rank order) into ysum: push yl into every rank's
    // receive slot of this step's parity, one cluster barrier, local sums.
    auto reduce_ranks = [&]() {
      float *rxp = rx + (gstep & 1) * CL * MP;
      ++gstep;
      for (int t = tid; t < CL * M; t += NT) {
        const int q = t / M, m = t - q * M;
        cl.map_shared_rank(rxp, q)[rank * MP + m] = yl[m];
      }
      cl.sync();
      for (int m = tid; m < M; m += NT) {
        float ym = 0.f;
#pragma unroll 4
        for (int q = 0; q < CL; ++q) ym += rxp[q * MP + m];
        ysum[m] = ym;
      }
      __syncthreads();
    };

    for (int m = tid; m < M; m += NT) vb0[m] = dold[m];
    __syncthreads();
    float *v = vb0;
    if (a.approx) {
      // ---- approximate update: d_k = E_k^T alpha_k / ||.|| (no sign rule) ----
      if (tid < M) yl[tid] = ya;
      __syncthreads();
      reduce_ranks();
      float ss = 0.f;
      for (int m = lane; m < M; m += 32) ss = fmaf(ysum[m], ysum[m], ss);
      ss = warp_sum(ss);
      if (ss > 0.f) {
        const float inv = 1.f / sqrtf(ss);
        for (int m = tid; m < M; m += NT) vb0[m] = ysum[m] * inv;
      }
      steps += 1;
      __syncthreads();
    } else {

    // ---- leading eigenvector of C = sum_r C_r by the power method from d_old ----
    // The ranks never form C.  Step t: every thread multiplies its register
    // tile of C_r with v_t, the tile rows are summed across the row's SIDE
    // threads (shuffles), each rank pushes its C_r v_t into every rank's
    // receive slot (distributed shared memory stores), and after one cluster
    // barrier every rank adds the CL products in rank order: all ranks hold
    // the same y = C v_t and take the same decisions.  v_{t+1} = y / ||y||;
    // stop when ||v_{t+1} - v_t||^2 <= kTol2.  Receive slots alternate by step
    // (the alternation runs on across visits), so a rank writes a slot only
    // after every rank has passed the barrier that follows its reads of it.
    int cur = 0;
    bool zero = false;
    for (int it = 0; it < kMaxIt; ++it) {
      const float *v = cur ? vb1 : vb0;
      float *vn = cur ? vb0 : vb1;
      {
        float vv[TR], py[TR];
        lds_run<TR>(vv, v + c0);
#pragma unroll
        for (int i = 0; i < TR; ++i) {
          float t = 0.f;
#pragma unroll
          for (int j = 0; j < TR; ++j) t = fmaf(acc[i][j], vv[j], t);
          py[i] = t;
        }
#pragma unroll
        for (int i = 0; i < TR; ++i)
#pragma unroll
          for (int o = SIDE / 2; o; o >>= 1) py[i] += __shfl_xor_sync(0xffffffffu, py[i], o);
        if (tx == 0)
#pragma unroll
          for (int i = 0; i < TR; ++i)
            if (r0 + i < M) yl[r0 + i] = py[i];
      }
      __syncthreads();
      reduce_ranks();
      if (warp == 0) {   // ||y||^2 and the change to the next vector, published to the CTA
        float s2 = 0.f, c2 = 0.f;
        for (int m = lane; m < M; m += 32) s2 = fmaf(ysum[m], ysum[m], s2);
        s2 = warp_sum(s2);
        if (s2 > 0.f) {
          const float inv = 1.f / sqrtf(s2);
          for (int m = lane; m < M; m += 32) {
            const float d = ysum[m] * inv - v[m];
            c2 = fmaf(d, d, c2);
          }
          c2 = warp_sum(c2);
        }
        if (lane == 0) { scal[0] = s2; scal[1] = c2; }
      }
      __syncthreads();
      const float ss = scal[0], d2 = scal[1];
      if (!(ss > 0.f)) { zero = true; steps += it; break; }
      const float inv = 1.f / sqrtf(ss);
      for (int m = tid; m < M; m += NT) vn[m] = ysum[m] * inv;
      __syncthreads();
      cur ^= 1;
      if (d2 <= kTol2) { steps += it + 1; break; }     // v_{t+1} is converged
      if (it == kMaxIt - 1) steps += kMaxIt;
    }
    v = zero ? dold : (cur ? vb1 : vb0);
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
    }  // exact update
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

template <int SIDE, int TR, int CL>
cudaLaunchConfig_t sweep_config(int M, cudaLaunchAttribute *at, cudaStream_t s, cudaError_t *e) {
  constexpr int NT = SIDE * SIDE;
  const size_t smem = (size_t)sweep_smem_floats(SIDE * TR, SIDE, CL) * 4;
  *e = cudaFuncSetAttribute(ksvd_sweep_kernel<SIDE, TR, CL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (*e == cudaSuccess && CL > 8)
    *e = cudaFuncSetAttribute(ksvd_sweep_kernel<SIDE, TR, CL>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(CL);
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = CL;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cfg;
}

// Whether one cluster of CL CTAs of this shape can be resident on the device.
template <int SIDE, int TR, int CL>
bool sweep_fits(int M) {
  cudaLaunchAttribute at[1];
  cudaError_t e;
  cudaLaunchConfig_t cfg = sweep_config<SIDE, TR, CL>(M, at, nullptr, &e);
  int n = 0;
  if (e != cudaSuccess || cudaOccupancyMaxActiveClusters(&n, ksvd_sweep_kernel<SIDE, TR, CL>, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return n >= 1;
}

template <int SIDE, int TR, int CL>
cudaError_t launch_sweep_t(const SweepArgs &a, cudaStream_t s) {
  cudaLaunchAttribute at[1];
  cudaError_t e;
  cudaLaunchConfig_t cfg = sweep_config<SIDE, TR, CL>(a.M, at, s, &e);
  if (e != cudaSuccess) return e;
  return cudaLaunchKernelEx(&cfg, ksvd_sweep_kernel<SIDE, TR, CL>, a);
}

template <int CL>
cudaError_t launch_sweep_cl(const SweepArgs &a, cudaStream_t s) {
  const int M = a.M;
  if (M <= 16) return launch_sweep_t<16, 1, CL>(a, s);
  if (M <= 32) return launch_sweep_t<16, 2, CL>(a, s);
  if (M <= 48) return launch_sweep_t<16, 3, CL>(a, s);
  if (M <= 64) return launch_sweep_t<16, 4, CL>(a, s);
  if (M <= 128) return launch_sweep_t<16, 8, CL>(a, s);
  // M <= 192: the exact update's Gram tiles favour 256 threads with 12 x 12
  // tiles; the approximate update (no Gram) favours 1024 threads (more warps
  // in flight for staging and the column updates)
  return a.approx ? launch_sweep_t<32, 6, CL>(a, s) : launch_sweep_t<16, 12, CL>(a, s);
}

bool sweep_fits_16(int M, bool approx) {
  if (M <= 16) return sweep_fits<16, 1, 16>(M);
  if (M <= 32) return sweep_fits<16, 2, 16>(M);
  if (M <= 48) return sweep_fits<16, 3, 16>(M);
  if (M <= 64) return sweep_fits<16, 4, 16>(M);
  if (M <= 128) return sweep_fits<16, 8, 16>(M);
  return approx ? sweep_fits<32, 6, 16>(M) : sweep_fits<16, 12, 16>(M);
}

}  // namespace

int ksvd_owner_split(int M, int T, bool approx) {
  // Sixteen ranks (a non-portable cluster) when one fits on the device and the
  // sort's shared histogram (T x 16 counters) stays within 128 KB; else eight.
  return (T * 16 <= 32768 && sweep_fits_16(M, approx)) ? 16 : 8;
}

int ksvd_owner_split(int M, int T) { return ksvd_owner_split(M, T, false); }

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

cudaError_t launch_ksvd_sweep(float *D, int M, int T, const float *X, int N, float *coef, int Kmax, int split,
                              const int *off, const int32_t *seg, float *R, float *rn2, const float *xn2,
                              uint8_t *taken, int replace, const int32_t *rparent, const int32_t *rsup, int Kc,
                              unsigned long long *stats, int approx, cudaStream_t s) {
  SweepArgs a{D, M, T, X, N, coef, Kmax, off, seg, R, rn2, xn2, taken, replace, rparent, rsup, Kc, stats, approx};
  return split == 16 ? launch_sweep_cl<16>(a, s) : launch_sweep_cl<8>(a, s);
}

void launch_ksvd_sum(const float *rn2, int N, float *out, cudaStream_t s) {
  ksvd_sum_kernel<<<1, 1024, 0, s>>>(rn2, N, out);
}

void launch_ksvd_init(float *D, int M, int T, const float *X, int N, const int32_t *parent, const int *off,
                      const int32_t *seg, int Kc, const double *u, cudaStream_t s) {
  ksvd_init_kernel<<<(T + 7) / 8, 256, 0, s>>>(D, M, T, X, N, parent, off, seg, Kc, u);
}

}  // namespace csp
