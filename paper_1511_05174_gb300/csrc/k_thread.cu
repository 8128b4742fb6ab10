// Restricted OMP (the finer-scale step of Algorithm 2, problem (P_high)) with
// ONE THREAD PER PATCH, for sparsity budgets Kb <= 8 and candidate sets
// |f(Omega)| <= CPL.
//
// The iteration is the Gram-Schmidt form of the restricted kernels in
// k_grp.cu: with U the orthonormal directions of the chosen atoms, the thread
// keeps Q_C = A_C^T U (one row of <= 8 entries per candidate) and the
// correlations c = A_C^T r.  Choosing atom q (argmax |c_i| / ||a_i|| over the
// candidates not chosen yet) needs no triangular solve:
//   w = Q_C[q] (the new row of the Cholesky factor L of A_Omega^T A_Omega),
//   L_kk = sqrt(||a_q||^2 - ||w||^2),   z_k = c_q / L_kk   (c_q = <a_q, y> - w.z),
//   new column Q_C[:, k] = (G[C][q] - Q_C w) / L_kk,   c -= z_k Q_C[:, k],
//   ||r||^2 -= z_k^2,
// with G = A A^T the level's Gram matrix; alpha = L^{-T} z is solved once at
// the end.  The row of Q_C of the k-th chosen atom holds (L[k][0..k-1], L_kk),
// so L is read back from Q_C for that solve.
//
// Why one thread per patch: with lane groups (k_grp.cu) every per-patch scalar
// step (argmax, pivot, w.w, the L row) is replicated over the group's lanes and
// joined by shuffles, so most instructions are overhead.  Here each thread owns
// its patch: the candidates' correlations, inverse norms and atom indices sit in
// registers (CPL of each), the argmax is a register scan with no shuffle, and
// only Q_C lives in shared memory, stored by column with the thread index
// fastest (entry (c, j) of thread t at ((c * 8 + j) * 32 + t) floats), so every
// access of a warp is one conflict-free wavefront whatever the candidate each
// thread touches.
//
// FP32 with the same safeguards as the other restricted kernels: when the
// pivot ratio L_kk^2 / ||a_q||^2 falls below kTauPivot the projection is redone
// in FP64 from scratch and the patch stays in FP64 (correlations and ||r||^2
// then formed from an explicit residual); an atom that FP64 finds dependent
// ends the patch; near the FP32 floor (||r||^2 <= 1e-5 ||y||^2) the residual is
// formed explicitly.  Through csp_reconstruct the warp also writes
// x_hat_p = D0_Omega alpha_p for its 32 patches (the synthesis of Sec. IV), in
// the FMA order of synth_kernel.
#include "csp_internal.cuh"

namespace csp {

namespace {

constexpr int TP_WARPS = 2;  // warps per CTA (shared memory: TP_WARPS * CPL KB)

__host__ __device__ __forceinline__ size_t tp_smem_bytes(int cpl) { return (size_t)TP_WARPS * cpl * 8 * 32 * 4; }

__device__ __forceinline__ int tri_(int i) { return (i * (i + 1)) >> 1; }

// FP64 least squares over the columns om[0..k-1] and q of A (rows of M floats)
// from scratch: Cholesky of the Gram matrix accumulated in FP64, z = L^{-1}
// A_S^T y, alpha = L^{-T} z.  Returns false when q depends on the others
// (pivot L_kk <= kEpsD64 ||a_q||).
__device__ __noinline__ bool tp_fp64_solve(int M, const float *__restrict__ y, const float *__restrict__ A,
                                           const int *om, int k, int q, double *alpha) {
  double L64[(8 + 1) * (8 + 2) / 2];
  for (int i = 0; i <= k; ++i) {
    const float *ci = A + (int64_t)(i < k ? om[i] : q) * M;
    for (int j = 0; j <= i; ++j) {
      const float *cj = A + (int64_t)(j < k ? om[j] : q) * M;
      double g = 0.0;
      for (int m = 0; m < M; ++m) g = fma((double)ci[m], (double)cj[m], g);
      double r = g;
      for (int p = 0; p < j; ++p) r -= L64[tri_(i) + p] * L64[tri_(j) + p];
      if (j < i) {
        L64[tri_(i) + j] = r / L64[tri_(j) + j];
      } else {
        if (i == k && !(r > kEpsD64 * kEpsD64 * g)) return false;
        L64[tri_(i) + i] = sqrt(r > 0.0 ? r : 0.0);
      }
    }
  }
  double zb[9];
  for (int i = 0; i <= k; ++i) {
    const float *ci = A + (int64_t)(i < k ? om[i] : q) * M;
    double bi = 0.0;
    for (int m = 0; m < M; ++m) bi = fma((double)ci[m], (double)y[m], bi);
    for (int p = 0; p < i; ++p) bi -= L64[tri_(i) + p] * zb[p];
    zb[i] = bi / L64[tri_(i) + i];
  }
  for (int i = k; i >= 0; --i) {
    double r = zb[i];
    for (int j = i + 1; j <= k; ++j) r -= L64[tri_(j) + i] * zb[j];
    zb[i] = r / L64[tri_(i) + i];
  }
  for (int i = 0; i <= k; ++i) alpha[i] = zb[i];
  return true;
}

// Explicit residual r = y - A_Omega alpha (FP32, over the kk chosen columns),
// returns ||r||^2; with cs != nullptr also the correlations cc[u] = <a_cs[u], r>
// of the nc candidates.
__device__ __noinline__ float tp_explicit(int M, const float *__restrict__ y, const float *__restrict__ A,
                                          const int *om, const float *al, int kk, const int *cs, int nc,
                                          float *cc) {
  float r[256];
  float r2 = 0.f;
  for (int m = 0; m < M; ++m) {
    float v = y[m];
    for (int i = 0; i < kk; ++i) v = fmaf(-al[i], A[(int64_t)om[i] * M + m], v);
    r[m] = v;
    r2 = fmaf(v, v, r2);
  }
  if (cs)
    for (int u = 0; u < nc; ++u) {
      const float *a = A + (int64_t)cs[u] * M;
      float s = 0.f;
      for (int m = 0; m < M; ++m) s = fmaf(a[m], r[m], s);
      cc[u] = s;
    }
  return r2;
}

template <int CPL>
__global__ void __launch_bounds__(TP_WARPS * 32)
omp_restricted_thread_kernel(const float *__restrict__ Y, int M, const float *__restrict__ A,
                             const float *__restrict__ inv_norm, const int32_t *__restrict__ ids, int64_t n,
                             const int32_t *__restrict__ child_off, const int32_t *__restrict__ child_idx, int cap,
                             const int32_t *__restrict__ omega_up, int ldo_up, const int8_t *__restrict__ keff_up,
                             const int8_t *__restrict__ Kp, int Kuni, int Kb, int32_t *__restrict__ omega,
                             float *__restrict__ alpha, int ldo, int8_t *__restrict__ k_eff, int64_t *stats,
                             const float *__restrict__ gram, int T, const float *__restrict__ D0, int N0,
                             float *__restrict__ Xh) {
  extern __shared__ __align__(16) float tp_sm[];
  const unsigned kFull = 0xffffffffu;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t wbase = ((int64_t)blockIdx.x * TP_WARPS + wib) * 32;
  if (wbase >= n) return;  // whole warp
  float *Qw = tp_sm + (size_t)wib * CPL * 8 * 32;  // this warp's Q_C
  float *Qt = Qw + lane;                           // entry (c, j) of this thread: Qt[(c * 8 + j) * 32]
  const int64_t wi = wbase + lane;
  const bool valid = wi < n;
  const int64_t b = valid ? (ids ? __ldg(ids + wi) : wi) : 0;
  int Kpb = valid ? (Kp ? (int)Kp[b] : Kuni) : 0;
  Kpb = Kpb < Kb ? Kpb : Kb;
  const float *yrow = Y + b * M;

  // ---- candidates f(Omega_up): parents in support order, children in link order
  int nc = 0;
  {
    const int kup = valid ? (int)keff_up[b] : 0;
    int tot = 0;
    for (int j = 0; j < kup; ++j) {
      const int p = omega_up[b * ldo_up + j];
      const int c0 = child_off[p], c1 = child_off[p + 1];
      for (int c = c0; c < c1; ++c, ++tot)
        if (tot < cap) reinterpret_cast<int *>(Qt)[(tot * 8) * 32] = child_idx[c];
    }
    if (tot > cap) {
      atomicAdd((unsigned long long *)&stats[3], 1ull);
      tot = cap;
    }
    nc = tot;
  }
  const int ncw = __reduce_max_sync(kFull, nc);
  // registers: ncs = complemented atom index (0: not eligible), inverse norm, correlation
  unsigned ncs[CPL];
  float inv[CPL], cc[CPL];
#pragma unroll
  for (int u = 0; u < CPL; ++u) {
    const int a = u < nc ? reinterpret_cast<const int *>(Qt)[(u * 8) * 32] : -1;
    const float iv = a >= 0 ? __ldg(inv_norm + a) : -1.f;
    const bool el = a >= 0 && iv > 0.f;
    ncs[u] = el ? 0xffffffffu - (unsigned)a : 0u;
    inv[u] = el ? iv : 0.f;
    cc[u] = 0.f;
  }
  // p0 = A_C^T y (the starting correlations) and ||y||^2, one float4 of y at a time
  float ysq = 0.f;
  {
    const float4 *y4 = reinterpret_cast<const float4 *>(yrow);
    const int nv = M >> 2;
    for (int j = 0; j < nv; ++j) {
      const float4 yv = valid ? __ldg(y4 + j) : make_float4(0.f, 0.f, 0.f, 0.f);
      ysq = fmaf(yv.x, yv.x, fmaf(yv.y, yv.y, fmaf(yv.z, yv.z, fmaf(yv.w, yv.w, ysq))));
#pragma unroll
      for (int u = 0; u < CPL; ++u)
        if (u < ncw && ncs[u]) {
          const float4 a = __ldg(reinterpret_cast<const float4 *>(A + (int64_t)(0xffffffffu - ncs[u]) * M) + j);
          cc[u] = fmaf(a.x, yv.x, fmaf(a.y, yv.y, fmaf(a.z, yv.z, fmaf(a.w, yv.w, cc[u]))));
        }
    }
  }

  // per-thread arrays indexed by the (per-patch) iteration count: local memory
  int om[8], slot[8];
  float zl[8], linv[8];
  double a64[9];
  float rsq = ysq;
  bool act = valid && Kpb > 0;
  bool mode64 = false;  // FP32 pivot failed: FP64 projections from here on, alpha in a64
  int k = 0, scored = 0;
  const int Kw = __reduce_max_sync(kFull, Kpb);
  for (int it = 0; it < Kw; ++it) {
    act = act && k < Kpb && !(rsq <= kEpsR32 * ysq);
    if (!__any_sync(kFull, act)) break;
    if (act) ++scored;
    // proxy: packed key (score bits, complemented index) -> largest score, ties to the lowest index
    unsigned long long best = 0ull;
    int bslot = 0;
    float cq = 0.f;
#pragma unroll
    for (int u = 0; u < CPL; ++u)
      if (u < ncw) {
        const unsigned long long key =
            ((unsigned long long)__float_as_uint(fabsf(cc[u]) * inv[u]) << 32) | (unsigned long long)ncs[u];
        const bool gt = ncs[u] != 0u && key > best;
        best = gt ? key : best;
        bslot = gt ? u : bslot;
        cq = gt ? cc[u] : cq;
      }
    if (act && best == 0ull) act = false;  // candidate set exhausted
    const unsigned qlo = act ? (unsigned)best : 0u;
    const int q = act ? (int)(0xffffffffu - qlo) : 0;
    const bool f32 = act && !mode64;
    // G[q][c] for the eligible candidates and G[q][q], issued first
    const float *grow = gram + (int64_t)q * T;
    float gq[CPL];
#pragma unroll
    for (int u = 0; u < CPL; ++u)
      gq[u] = (u < ncw && f32 && ncs[u] && ncs[u] != qlo) ? __ldg(grow + (0xffffffffu - ncs[u])) : 0.f;
    const float aa = f32 ? __ldg(grow + q) : 0.f;
    // w = Q_C[q][0..k-1] (the new row of L)
    float w[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) w[j] = (f32 && j < k) ? Qt[(bslot * 8 + j) * 32] : 0.f;
    float ww0 = 0.f, ww1 = 0.f;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      ww0 = fmaf(w[j], w[j], ww0);
      ww1 = fmaf(w[j + 4], w[j + 4], ww1);
    }
    const float d = aa - (ww0 + ww1);
    const bool ok32 = f32 && aa > 0.f && d >= kTauPivot * aa;
    if (f32 && !ok32) atomicAdd((unsigned long long *)&stats[0], 1ull);
    if (ok32) {
      const float il = rsqrtf(d);  // d >= kTauPivot aa > 0
      const float lkk = d * il;
      const float zk = cq * il;
      om[k] = q;
      slot[k] = bslot;
      zl[k] = zk;
      linv[k] = il;
      Qt[(bslot * 8 + k) * 32] = lkk;  // the chosen row now holds (L[k][0..k-1], L_kk)
      // column k of Q_C and the correlations of the candidates still eligible
#pragma unroll
      for (int u = 0; u < CPL; ++u)
        if (u < ncw) {
          const bool upd = ncs[u] != 0u && ncs[u] != qlo;
          float v0 = 0.f, v1 = 0.f;
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            if (upd && j < k) v0 = fmaf(w[j], Qt[(u * 8 + j) * 32], v0);
            if (upd && j + 4 < k) v1 = fmaf(w[j + 4], Qt[(u * 8 + j + 4) * 32], v1);
          }
          const float v = (gq[u] - (v0 + v1)) * il;
          if (upd) {
            Qt[(u * 8 + k) * 32] = v;
            cc[u] = fmaf(-zk, v, cc[u]);
          }
        }
      rsq = rsq - zk * zk;
    }
    // the chosen candidate is no longer eligible
#pragma unroll
    for (int u = 0; u < CPL; ++u)
      if (act && ncs[u] == qlo) {
        ncs[u] = 0u;
        inv[u] = 0.f;
      }
    // FP64 from scratch once the FP32 pivot has failed (now or before)
    if (act && !ok32) {
      bool app = tp_fp64_solve(M, yrow, A, om, k, q, a64);
      if (app) {
        om[k] = q;
        slot[k] = bslot;
        mode64 = true;
        float al[8];
        for (int i = 0; i <= k; ++i) al[i] = (float)a64[i];
        int csl[CPL];
        float ccl[CPL];
#pragma unroll
        for (int u = 0; u < CPL; ++u) csl[u] = ncs[u] ? (int)(0xffffffffu - ncs[u]) : (int)(0xffffffffu - qlo);
        rsq = tp_explicit(M, yrow, A, om, al, k + 1, csl, ncw, ccl);
#pragma unroll
        for (int u = 0; u < CPL; ++u) cc[u] = ccl[u];
        ++k;
      } else {
        act = false;  // q depends on the chosen atoms: the patch ends with k atoms
      }
    } else if (ok32) {
      ++k;
      if (rsq <= 1e-5f * ysq) {  // near the FP32 floor: ||r||^2 from an explicit residual
        float al[8];
        for (int j = k - 1; j >= 0; --j) {
          float v = zl[j];
          for (int i = j + 1; i < k; ++i) v = fmaf(-Qt[(slot[i] * 8 + j) * 32], al[i], v);
          al[j] = v * linv[j];
        }
        rsq = tp_explicit(M, yrow, A, om, al, k, nullptr, 0, nullptr);
      }
    }
  }
  // alpha = L^{-T} z (FP32 patches; FP64 ones hold it in a64)
  float al[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) al[j] = 0.f;
  if (valid) {
    if (mode64) {
      for (int j = 0; j < k; ++j) al[j] = (float)a64[j];
    } else {
      for (int j = k - 1; j >= 0; --j) {
        float v = zl[j];
        for (int i = j + 1; i < k; ++i) v = fmaf(-Qt[(slot[i] * 8 + j) * 32], al[i], v);
        al[j] = v * linv[j];
      }
    }
  }
  {  // statistics: one atomic per warp
    const unsigned es = __reduce_add_sync(kFull, (valid && k < Kpb) ? 1u : 0u);
    const unsigned sc = __reduce_add_sync(kFull, valid ? (unsigned)(nc * scored) : 0u);
    if (lane == 0) {
      if (es) atomicAdd((unsigned long long *)&stats[1], (unsigned long long)es);
      atomicAdd((unsigned long long *)&stats[2], (unsigned long long)sc);
    }
  }
  if (valid) {
    k_eff[b] = (int8_t)k;
    for (int j = 0; j < ldo; ++j) {
      omega[b * ldo + j] = (j < k) ? om[j] : -1;
      alpha[b * ldo + j] = (j < k) ? al[j] : 0.f;
    }
  }
  // synthesis x_hat_p = D0_Omega alpha_p of the warp's patches, one patch at a
  // time over the warp's lanes (coalesced rows of D0 and of Xh)
  if (!Xh) return;
  __syncwarp();
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    Qt[j * 32] = al[j];
    reinterpret_cast<int *>(Qt)[(8 + j) * 32] = (j < k) ? om[j] : 0;
  }
  __syncwarp();
  const int n4 = N0 >> 2;
  for (int p = 0; p < 32; ++p) {
    const int kp = __shfl_sync(kFull, k, p);
    const int64_t bp = __shfl_sync(kFull, b, p);
    if (!__shfl_sync(kFull, valid ? 1 : 0, p)) continue;
    float4 *xb = reinterpret_cast<float4 *>(Xh + bp * N0);
    for (int c = lane; c < n4; c += 32) {
      float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
      for (int j = 0; j < kp; ++j) {
        const float aj = Qw[j * 32 + p];
        const int oj = reinterpret_cast<const int *>(Qw)[(8 + j) * 32 + p];
        const float4 dv = __ldg(reinterpret_cast<const float4 *>(D0 + (int64_t)oj * N0) + c);
        acc.x = fmaf(aj, dv.x, acc.x);
        acc.y = fmaf(aj, dv.y, acc.y);
        acc.z = fmaf(aj, dv.z, acc.z);
        acc.w = fmaf(aj, dv.w, acc.w);
      }
      xb[c] = acc;
    }
  }
}

}  // namespace

int restricted_thread_cpl(int cap) { return cap <= 8 ? 8 : (cap <= 16 ? 16 : (cap <= 24 ? 24 : (cap <= 32 ? 32 : 0))); }

bool launch_omp_restricted_thread(const float *Y, int M, const float *A, const float *inv_norm, const int32_t *ids,
                                  int64_t n, const int32_t *child_off, const int32_t *child_idx, int cap,
                                  const int32_t *omega_up, int ldo_up, const int8_t *keff_up, const int8_t *Kp,
                                  int Kuni, int Kb, int32_t *omega, float *alpha, int ldo, int8_t *k_eff,
                                  int64_t *stats, const float *gram, int T, const float *D0, int N0, float *Xh,
                                  bool *synthesized, cudaStream_t s) {
  *synthesized = false;
  const int cpl = restricted_thread_cpl(cap);
  if (!cpl || Kb > 8 || M % 4 || M > 256 || !gram) return false;
  const bool synth = Xh && D0 && N0 > 0 && N0 % 4 == 0;
  *synthesized = synth;
  if (n == 0) return true;
  const size_t sm = tp_smem_bytes(cpl);
  const unsigned grid = (unsigned)((n + TP_WARPS * 32 - 1) / (TP_WARPS * 32));
  auto go = [&](auto kern) {
    if (sm > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    kern<<<grid, TP_WARPS * 32, sm, s>>>(Y, M, A, inv_norm, ids, n, child_off, child_idx, cap, omega_up, ldo_up,
                                         keff_up, Kp, Kuni, Kb, omega, alpha, ldo, k_eff, stats, gram, T, D0, N0,
                                         synth ? Xh : nullptr);
  };
  switch (cpl) {
    case 8: go(omp_restricted_thread_kernel<8>); break;
    case 16: go(omp_restricted_thread_kernel<16>); break;
    case 24: go(omp_restricted_thread_kernel<24>); break;
    default: go(omp_restricted_thread_kernel<32>); break;
  }
  return true;
}

}  // namespace csp
