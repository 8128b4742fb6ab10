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
//     owns (i mod CL == rank), the partial Gram matrices meet through
//     distributed shared memory (reduce-scatter, then all-gather, fixed rank
//     order), every CTA runs the same power iteration on C = E_k E_k^T from
//     d_old (identical inputs, identical result), and each CTA updates the
//     coefficients and residuals of its own users.  Ownership by signal keeps
//     every residual with one CTA, so atoms need two cluster barriers each.
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
constexpr int kNB = 32;           // columns e_i staged per batch
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
                                 const int8_t *__restrict__ keff, int Kmax, float *__restrict__ R,
                                 float *__restrict__ rn2, float *__restrict__ xn2, int *__restrict__ hist,
                                 unsigned *err) {
  extern __shared__ int h[];
  for (int t = threadIdx.x; t < T; t += blockDim.x) h[t] = 0;
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
        atomicAdd(&h[a], 1);
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
  for (int t = threadIdx.x; t < T; t += blockDim.x) hist[(size_t)blockIdx.x * T + t] = h[t];
}

// 2. hist[c][t] <- users of atom t in chunks before c; off[t] = first slot of atom t.
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

// 3. Stable counting sort of the slots q = i * Kmax + j by atom (one warp per chunk).
__global__ void ksvd_fill_kernel(const int32_t *__restrict__ sup, const int8_t *__restrict__ keff, int N, int Kmax,
                                 int T, const int *__restrict__ hist, const int *__restrict__ off,
                                 int32_t *__restrict__ seg) {
  extern __shared__ int base[];
  const int lane = threadIdx.x;
  for (int t = lane; t < T; t += 32) base[t] = off[t] + hist[(size_t)blockIdx.x * T + t];
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
        if (a < 0 || a >= T) a = -1;
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

struct SweepArgs {
  float *D;
  int M, T;
  const float *X;
  int N;
  float *coef;
  int Kmax;
  const int *off;
  const int32_t *seg;
  float *R, *rn2;
  const float *xn2;
  uint8_t *taken;
  int replace;
  const int32_t *rparent, *rsup;
  int Kc;
};

__host__ __device__ constexpr int pad4(int n) { return (n + 3) & ~3; }

// Shared-memory floats of the sweep for dimension M with `nt` threads.
__host__ __device__ inline int sweep_smem_floats(int M, int MP, int nt) {
  const int MM = M * M, RB = (MM + kCL - 1) / kCL;
  return pad4(MM) + pad4(RB) + kNB * MP + 3 * pad4(M) + 128 + nt + 64;
}

// 4. The sweep.  Threads form a SIDE x SIDE grid; thread (ty, tx) accumulates
// the TR x TR tile of C at rows ty*TR.., columns tx*TR.. (SIDE*TR >= M).
template <int SIDE, int TR>
__global__ void __launch_bounds__(SIDE *SIDE, 1) ksvd_sweep_kernel(const SweepArgs a) {
  constexpr int NT = SIDE * SIDE, NW = NT / 32, MP = SIDE * TR;
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank(), CL = (int)cl.num_blocks();
  extern __shared__ float4 smem4[];
  float *sm = reinterpret_cast<float *>(smem4);
  const int M = a.M, MM = M * M, RB = (MM + CL - 1) / CL, Kmax = a.Kmax;
  float *Cb = sm;                        // [M][M] partial, then full E_k E_k^T
  float *red = Cb + pad4(MM);            // [RB] this CTA's share of the reduced matrix
  float *stage = red + pad4((MM + kCL - 1) / kCL);  // [kNB][MP] staged e_i
  float *dold = stage + kNB * MP;        // [M] atom before the visit
  float *v = dold + pad4(M);             // [M] power-iteration vector
  float *y = v + pad4(M);                // [M] C v
  float *scal = y + pad4(M);             // [128] flags, per-warp argmax scratch
  int *ents = reinterpret_cast<int *>(scal + 128);  // [NT] compacted slots
  int *wcnt = ents + NT;                 // [NW + 1]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ty = tid / SIDE, tx = tid - ty * SIDE, r0 = ty * TR, c0 = tx * TR;
  int *iflag = reinterpret_cast<int *>(scal);   // [0] converged, [1] zero matrix
  float *slotv = scal + 8;                      // best replacement candidate of this CTA
  int *sloti = reinterpret_cast<int *>(scal + 9);
  float *wv = scal + 32;                        // [32] per-warp best residual norm
  int *wi = reinterpret_cast<int *>(scal + 64); // [32] ... and its signal

  for (int k = 0; k < a.T; ++k) {
    const int base = a.off[k], n = a.off[k + 1] - base;
    for (int m = tid; m < M; m += NT) dold[m] = a.D[(size_t)k * M + m];
    for (int q = tid; q < kNB * MP; q += NT) stage[q] = 0.f;
    __syncthreads();

    if (n == 0) {
      // Heuristics 3 / 4: the unused atom becomes the eligible signal with the
      // largest residual norm (ties: lowest index); the signal is then taken.
      if (!a.replace) continue;
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
      for (int q = 0; q < CL; ++q) {
        const float ov = *cl.map_shared_rank(slotv, q);
        const int oi = *cl.map_shared_rank(sloti, q);
        if (oi >= 0 && (ov > gv || (ov == gv && (gi < 0 || oi < gi)))) { gv = ov; gi = oi; }
      }
      cl.sync();
      if (gi >= 0) {
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
      __syncthreads();
      continue;
    }

    // ---- partial C over the users this CTA owns, in slot order ----
    float acc[TR][TR];
#pragma unroll
    for (int i = 0; i < TR; ++i)
#pragma unroll
      for (int j = 0; j < TR; ++j) acc[i][j] = 0.f;
    for (int p0 = 0; p0 < n; p0 += NT) {
      const int p = p0 + tid;
      int e = -1;
      if (p < n) {
        const int q = a.seg[base + p];
        if ((q / Kmax) % CL == rank) e = q;
      }
      const unsigned bal = __ballot_sync(0xffffffffu, e >= 0);
      if (lane == 0) wcnt[warp] = __popc(bal);
      __syncthreads();
      if (tid == 0) {
        int s = 0;
        for (int w = 0; w < NW; ++w) { const int c = wcnt[w]; wcnt[w] = s; s += c; }
        wcnt[NW] = s;
      }
      __syncthreads();
      if (e >= 0) ents[wcnt[warp] + __popc(bal & lanemask_lt())] = e;
      __syncthreads();
      const int cnt = wcnt[NW];
      for (int b0 = 0; b0 < cnt; b0 += kNB) {
        const int nb = min(kNB, cnt - b0);
        for (int q = tid; q < nb * M; q += NT) {
          const int c = q / M, m = q - c * M;
          const int s = ents[b0 + c];
          const int i = s / Kmax;
          stage[c * MP + m] = fmaf(a.coef[s], dold[m], a.R[(size_t)i * M + m]);
        }
        __syncthreads();
        for (int c = 0; c < nb; ++c) {
          const float *ec = stage + c * MP;
          float er[TR], ek[TR];
#pragma unroll
          for (int t = 0; t < TR; ++t) { er[t] = ec[r0 + t]; ek[t] = ec[c0 + t]; }
#pragma unroll
          for (int i = 0; i < TR; ++i)
#pragma unroll
            for (int j = 0; j < TR; ++j) acc[i][j] = fmaf(er[i], ek[j], acc[i][j]);
        }
        __syncthreads();
      }
    }
#pragma unroll
    for (int i = 0; i < TR; ++i)
#pragma unroll
      for (int j = 0; j < TR; ++j)
        if (r0 + i < M && c0 + j < M) Cb[(r0 + i) * M + c0 + j] = acc[i][j];

    // ---- C = sum over ranks (reduce-scatter, all-gather) ----
    cl.sync();
    {
      const int e0 = rank * RB, e1 = min(MM, e0 + RB);
      for (int el = e0 + tid; el < e1; el += NT) {
        float s = 0.f;
        for (int q = 0; q < CL; ++q) s += cl.map_shared_rank(Cb, q)[el];
        red[el - e0] = s;
      }
    }
    cl.sync();
    for (int el = tid; el < MM; el += NT) {
      const int q = el / RB;
      Cb[el] = cl.map_shared_rank(red, q)[el - q * RB];
    }
    for (int m = tid; m < M; m += NT) v[m] = dold[m];
    __syncthreads();

    // ---- leading eigenvector of C by the power method from d_old ----
    for (int it = 0; it < kMaxIt; ++it) {
      for (int r = warp; r < M; r += NW) {
        float s = 0.f;
        for (int c = lane; c < M; c += 32) s = fmaf(Cb[r * M + c], v[c], s);
        s = warp_sum(s);
        if (lane == 0) y[r] = s;
      }
      __syncthreads();
      if (warp == 0) {
        float s = 0.f;
        for (int m = lane; m < M; m += 32) s = fmaf(y[m], y[m], s);
        s = warp_sum(s);
        int conv = 0, zero = 0;
        if (!(s > 0.f)) {
          zero = 1;
        } else {
          const float inv = 1.f / sqrtf(s);
          float d2 = 0.f;
          for (int m = lane; m < M; m += 32) {
            const float nv = y[m] * inv;
            const float d = nv - v[m];
            d2 = fmaf(d, d, d2);
            v[m] = nv;
          }
          d2 = warp_sum(d2);
          conv = d2 <= kTol2;
        }
        if (lane == 0) { iflag[0] = conv; iflag[1] = zero; }
      }
      __syncthreads();
      const bool stop = iflag[0] | iflag[1];
      __syncthreads();
      if (stop) break;
    }
    if (warp == 0) {  // sign: <d_new, d_old> >= 0
      float s = 0.f;
      for (int m = lane; m < M; m += 32) s = fmaf(v[m], dold[m], s);
      s = warp_sum(s);
      if (s < 0.f)
        for (int m = lane; m < M; m += 32) v[m] = -v[m];
    }
    __syncthreads();
    if (rank == 0)
      for (int m = tid; m < M; m += NT) a.D[(size_t)k * M + m] = v[m];

    // ---- coefficients E_k^T d_k and residuals of the users this CTA owns ----
    for (int p = warp; p < n; p += NW) {
      const int q = a.seg[base + p];
      const int i = q / Kmax;
      if (i % CL != rank) continue;
      const float al = a.coef[q];
      float ev[(MP + 31) / 32];
      float s = 0.f;
#pragma unroll
      for (int t = 0; t < (MP + 31) / 32; ++t) {
        const int m = lane + 32 * t;
        ev[t] = 0.f;
        if (m < M) {
          ev[t] = fmaf(al, dold[m], a.R[(size_t)i * M + m]);
          s = fmaf(ev[t], v[m], s);
        }
      }
      const float an = warp_sum(s);
      float rs = 0.f;
#pragma unroll
      for (int t = 0; t < (MP + 31) / 32; ++t) {
        const int m = lane + 32 * t;
        if (m < M) {
          const float r = fmaf(-an, v[m], ev[t]);
          a.R[(size_t)i * M + m] = r;
          rs = fmaf(r, r, rs);
        }
      }
      rs = warp_sum(rs);
      if (lane == 0) { a.coef[q] = an; a.rn2[i] = rs; }
    }
    __syncthreads();
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
  const size_t smem = (size_t)sweep_smem_floats(a.M, SIDE * TR, NT) * 4;
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

size_t ksvd_sweep_smem_bytes(int M) {
  if (M <= 16) return (size_t)sweep_smem_floats(M, 16, 256) * 4;
  if (M <= 32) return (size_t)sweep_smem_floats(M, 32, 256) * 4;
  if (M <= 48) return (size_t)sweep_smem_floats(M, 48, 256) * 4;
  if (M <= 64) return (size_t)sweep_smem_floats(M, 64, 256) * 4;
  if (M <= 128) return (size_t)sweep_smem_floats(M, 128, 256) * 4;
  return (size_t)sweep_smem_floats(M, 192, 1024) * 4;
}

int ksvd_chunks(int64_t N) { return (int)((N + kChunk - 1) / kChunk); }

void launch_ksvd_sort(const float *D, int M, int T, const float *X, int N, const int32_t *sup, const float *coef,
                      const int8_t *keff, int Kmax, float *R, float *rn2, float *xn2, int *hist, int *off,
                      int32_t *seg, unsigned *err, cudaStream_t s) {
  const int C = ksvd_chunks(N);
  if (C > 0) {
    cudaFuncSetAttribute(ksvd_prep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, T * 4);
    ksvd_prep_kernel<<<C, 256, (size_t)T * 4, s>>>(D, M, T, X, N, sup, coef, keff, Kmax, R, rn2, xn2, hist, err);
  }
  ksvd_scan_kernel<<<1, 1024, 0, s>>>(hist, C, T, off);
  if (C > 0) {
    cudaFuncSetAttribute(ksvd_fill_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, T * 4);
    ksvd_fill_kernel<<<C, 32, (size_t)T * 4, s>>>(sup, keff, N, Kmax, T, hist, off, seg);
  }
}

cudaError_t launch_ksvd_sweep(float *D, int M, int T, const float *X, int N, float *coef, int Kmax, const int *off,
                              const int32_t *seg, float *R, float *rn2, const float *xn2, uint8_t *taken, int replace,
                              const int32_t *rparent, const int32_t *rsup, int Kc, cudaStream_t s) {
  SweepArgs a{D, M, T, X, N, coef, Kmax, off, seg, R, rn2, xn2, taken, replace, rparent, rsup, Kc};
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
