// Device helpers shared by the lane-group OMP kernels (k_omp.cu, k_grp.cu).
//
// A GROUP of G lanes solves one patch; lane s of a group owns the float4
// chunks j = s, s + G, s + 2G, ... of every M-vector.  Group reductions must
// be called by every lane of the warp together (converged control flow).
#pragma once

#include "csp_internal.cuh"

namespace csp {
namespace grp {

constexpr unsigned kFull = 0xffffffffu;

__host__ __device__ __forceinline__ int tri(int i) { return (i * (i + 1)) >> 1; }
__host__ __device__ __forceinline__ int up16(int bytes) { return (bytes + 15) & ~15; }

// Packed argmax key: larger score first, then lower index.  0 = no candidate.
__device__ __forceinline__ unsigned long long pack_key(float score, int idx) {
  return ((unsigned long long)__float_as_uint(score) << 32) | (0xffffffffu - (unsigned)idx);
}
__device__ __forceinline__ int key_idx(unsigned long long k) {
  return (int)(0xffffffffu - (unsigned)(k & 0xffffffffull));
}

// ---- group reductions (every lane of the warp must call them together) ----
template <int G>
__device__ __forceinline__ float gsum(float v) {
#pragma unroll
  for (int o = G / 2; o; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}
template <int G>
__device__ __forceinline__ unsigned long long gmax(unsigned long long v) {
#pragma unroll
  for (int o = G / 2; o; o >>= 1) {
    const unsigned long long w = __shfl_xor_sync(kFull, v, o);
    v = w > v ? w : v;
  }
  return v;
}

__device__ __forceinline__ float dot4(const float4 &a, const float4 &b) {
  return fmaf(a.x, b.x, fmaf(a.y, b.y, fmaf(a.z, b.z, a.w * b.w)));
}

// Chunks j = s + G t (t < NCH) of a 16-byte aligned row of nv float4; zeros past nv.
template <int G, int NCH>
__device__ __forceinline__ void load_chunks(float4 (&v)[NCH], const float *__restrict__ row, int nv, int s,
                                            bool on) {
  const float4 *r4 = reinterpret_cast<const float4 *>(row);
#pragma unroll
  for (int t = 0; t < NCH; ++t) {
    const int j = s + G * t;
    v[t] = (on && j < nv) ? __ldg(r4 + j) : make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

// Same with plain (generic) loads: `row` may be in shared or global memory.
template <int G, int NCH>
__device__ __forceinline__ void load_chunks_gen(float4 (&v)[NCH], const float *row, int nv, int s, bool on) {
  const float4 *r4 = reinterpret_cast<const float4 *>(row);
#pragma unroll
  for (int t = 0; t < NCH; ++t) {
    const int j = s + G * t;
    v[t] = (on && j < nv) ? r4[j] : make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

// Full dot product of two 16-byte aligned rows of nv float4 (generic loads),
// four independent accumulators.
__device__ __forceinline__ float row_dot(const float *a, const float *b, int nv) {
  const float4 *a4 = reinterpret_cast<const float4 *>(a);
  const float4 *b4 = reinterpret_cast<const float4 *>(b);
  float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
  for (int j = 0; j < nv; ++j) {
    const float4 x = a4[j], y = b4[j];
    s0 = fmaf(x.x, y.x, s0);
    s1 = fmaf(x.y, y.y, s1);
    s2 = fmaf(x.z, y.z, s2);
    s3 = fmaf(x.w, y.w, s3);
  }
  return (s0 + s1) + (s2 + s3);
}

template <int NCH>
__device__ __forceinline__ float dotc(const float4 (&a)[NCH], const float4 (&b)[NCH]) {
  float s0 = 0.f, s1 = 0.f;
#pragma unroll
  for (int t = 0; t < NCH; ++t) {
    if (t & 1) s1 += dot4(a[t], b[t]);
    else s0 += dot4(a[t], b[t]);
  }
  return s0 + s1;
}

// ---------------------------------------------------------------------------
// Per-group shared-memory block.
// ---------------------------------------------------------------------------
struct GrpSmem {
  float *L;      // [tri(Kb)]   packed lower factor
  float *Linv;   // [Kb]        1 / L_jj
  float *z;      // [Kb]
  float *V;      // [Kb+1]      Gram column / back-substitution accumulator
  float *W;      // [Kb+1]      w = L^{-1} v, then alpha
  int *om;       // [Kb]        chosen atoms
  const float **colp;  // [Kb+1] row of each chosen column (shared or global memory)
  int *cs;       // [cap]       candidate atoms (restricted kernel)
  float *invn;   // [cap]       their 1/||a|| (-1 once chosen or ineligible)
  int *misc;     // [4]
};

__host__ __device__ __forceinline__ int grp_smem_bytes(int Kb, int cap) {
  return up16(4 * tri(Kb)) + 2 * up16(4 * Kb) + 2 * up16(4 * (Kb + 1)) +
         up16(4 * Kb) + up16(8 * (Kb + 1)) + 2 * up16(4 * cap) + 16;
}

__device__ __forceinline__ GrpSmem carve(char *p, int Kb, int cap) {
  GrpSmem S;
  S.L = reinterpret_cast<float *>(p); p += up16(4 * tri(Kb));
  S.Linv = reinterpret_cast<float *>(p); p += up16(4 * Kb);
  S.z = reinterpret_cast<float *>(p); p += up16(4 * Kb);
  S.V = reinterpret_cast<float *>(p); p += up16(4 * (Kb + 1));
  S.W = reinterpret_cast<float *>(p); p += up16(4 * (Kb + 1));
  S.om = reinterpret_cast<int *>(p); p += up16(4 * Kb);
  S.colp = reinterpret_cast<const float **>(p); p += up16(8 * (Kb + 1));
  S.cs = reinterpret_cast<int *>(p); p += up16(4 * cap);
  S.invn = reinterpret_cast<float *>(p); p += up16(4 * cap);
  S.misc = reinterpret_cast<int *>(p);
  return S;
}

// alpha = L^{-T} z over rows 0 .. kl of the packed factor (into S.W), for the
// groups with `on`; kw >= kl for every group of the warp.  Warp-collective.
template <int G>
__device__ __forceinline__ void grp_backsub(bool on, int s, int kl, int kw, const GrpSmem &S) {
  if (on)
    for (int i = s; i <= kl; i += G) S.V[i] = S.z[i];
  __syncwarp();
  for (int j = kw; j >= 0; --j) {
    if (on && j <= kl) {
      const float aj = S.V[j] * S.Linv[j];
      if (s == 0) S.W[j] = aj;
      for (int i = s; i < j; i += G) S.V[i] = fmaf(-S.L[tri(j) + i], aj, S.V[i]);
    }
    __syncwarp();
  }
}

// FP64 projection from scratch, run by one lane: Cholesky of A_S^T A_S for
// S = chosen + q (rows S.colp[0..k-1] and aq) with entries accumulated in FP64
// from the FP32 columns, then z = L^{-1} A_S^T y and alpha = L^{-T} z (into
// S.W).  Returns false when q depends on the chosen columns.  The factor is a
// temporary of this (rare) path and lives in the thread's local memory.
static __device__ __noinline__ bool fp64_projection(int M, const float *__restrict__ y, const GrpSmem &S, int k,
                                                    const float *aq) {
  double L64[(CSP_MAX_K + 1) * (CSP_MAX_K + 2) / 2];
  for (int i = 0; i <= k; ++i) {
    const float *ci = i < k ? S.colp[i] : aq;
    for (int j = 0; j <= i; ++j) {
      const float *cj = j < k ? S.colp[j] : aq;
      double g = 0.0;
      for (int m = 0; m < M; ++m) g = fma((double)ci[m], (double)cj[m], g);
      double r = g;
      for (int p = 0; p < j; ++p) r -= L64[tri(i) + p] * L64[tri(j) + p];
      if (j < i) {
        L64[tri(i) + j] = r / L64[tri(j) + j];
      } else {
        if (i == k && !(r > kEpsD64 * kEpsD64 * g)) return false;
        L64[tri(i) + i] = sqrt(r > 0.0 ? r : 0.0);
      }
    }
  }
  double zb[CSP_MAX_K + 1];
  for (int i = 0; i <= k; ++i) {
    const float *ci = i < k ? S.colp[i] : aq;
    double bi = 0.0;
    for (int m = 0; m < M; ++m) bi = fma((double)ci[m], (double)y[m], bi);
    for (int p = 0; p < i; ++p) bi -= L64[tri(i) + p] * zb[p];
    zb[i] = bi / L64[tri(i) + i];
  }
  for (int i = k; i >= 0; --i) {
    double r = zb[i];
    for (int j = i + 1; j <= k; ++j) r -= L64[tri(j) + i] * zb[j];
    zb[i] = r / L64[tri(i) + i];
  }
  for (int i = 0; i <= k; ++i) S.W[i] = (float)zb[i];
  return true;
}


}  // namespace grp
}  // namespace csp
