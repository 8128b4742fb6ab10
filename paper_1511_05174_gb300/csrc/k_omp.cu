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
// also decides linear dependence (L_kk <= kEpsD64 ||a_k||, the FP64 analogue of
// a QR pivot test above the rounding floor of the normal equations).
//
// Work decomposition: a GROUP of G lanes (G = 4, 8 or 16) solves one patch;
// a warp holds 32 / G patches.  Lane s of a group owns the float4 chunks
// j = s, s + G, s + 2G, ... of every M-vector (y, r, columns), so the group
// reads each column row as contiguous 16 G-byte segments and reduces a dot
// product with log2(G) shuffles.  Loops whose trip counts differ between the
// patches of a warp run to the warp maximum with per-group predicates, so all
// shuffles execute in converged control flow.  The triangular factor, z, the
// Gram column and alpha live in per-group shared memory.
//
// Kernels:
//   proxy_fp32_kernel      full-dictionary proxy, FP32 CUDA-core GEMM of a tile of
//                          64 residuals against all atoms, fused |.|/norm, mask and
//                          argmax (one candidate per patch)
//   omp_update_kernel      one iteration for every patch: (re-score the proxy's
//                          candidates in FP32,) merge, projection, residue; state
//                          kept in global memory between launches
//   omp_restricted_kernel  all iterations of the restricted OMP over the children
//                          f(Omega_up) of the coarser support (Algorithm 2 fine step)
#include "csp_internal.cuh"
#include "grp_common.cuh"

namespace csp {

namespace {

using namespace csp::grp;

// ---------------------------------------------------------------------------
// Group projection step.  `act`: this group appends atom q (row aqp, shared or
// global memory) as its k-th column (S.om / S.colp [0..k-1] chosen; S.L/Linv/z
// valid unless fl has bit 1).  Lanes hold their chunks of y and r.  On success
// alpha is in S.W[0..k], r and rsq are updated, S.om[k] = q, S.colp[k] = aqp,
// and the FP32 factor gained row k.  Returns whether q was appended (false: q
// depends on the chosen columns).  Warp-collective.
// ---------------------------------------------------------------------------
template <int G, int NCH, bool COOP>
__device__ bool grp_append(bool act, int s, int M, const float *aqp, const float *__restrict__ yrow, int q, int k,
                           const float4 (&yv)[NCH], float4 (&rv)[NCH], const GrpSmem &S, uint8_t &fl, float &rsq,
                           int64_t *stats, const float *__restrict__ gram, int T) {
  const int nv = M >> 2;
  float4 aq[NCH];
  load_chunks_gen<G, NCH>(aq, aqp, nv, s, act);
  const float aa_dot = gsum<G>(dotc<NCH>(aq, aq));
  const float bq = gsum<G>(dotc<NCH>(aq, yv));
  const int kw = __reduce_max_sync(kFull, act ? k : 0);
  const bool f32 = act && !(fl & 2);
  // Gram column V[j] = <a_{om_j}, a_q>: looked up in the precomputed Gram matrix
  // of the effective dictionary when there is one; else COOP: the group reads
  // each chosen row as contiguous chunks and reduces with shuffles (columns in
  // global memory); otherwise one full-row dot product per lane (shared memory).
  const float aa = gram ? (act ? __ldg(gram + (int64_t)q * T + q) : 0.f) : aa_dot;
  if (gram) {
    if (f32)
      for (int j = s; j < k; j += G) S.V[j] = __ldg(gram + (int64_t)q * T + S.om[j]);  // row q (G symmetric)
  } else if (COOP) {
    for (int j = 0; j < kw; ++j) {
      const bool o = f32 && j < k;
      float4 c[NCH];
      load_chunks_gen<G, NCH>(c, o ? S.colp[j] : aqp, nv, s, o);
      const float v = gsum<G>(dotc<NCH>(c, aq));
      if (o && s == 0) S.V[j] = v;
    }
  } else if (f32) {
    for (int j = s; j < k; j += G) S.V[j] = row_dot(S.colp[j], aqp, nv);
  }
  __syncwarp();
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
  // back substitution alpha = L^{-T} z (accumulator V; alpha into W)
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
  // FP64 rebuild for the groups that need it (rare; one lane per group)
  const bool go64 = act && !ok32;
  if (go64 && s == 0) S.misc[0] = fp64_projection(M, yrow, S, k, aqp) ? 1 : 0;
  __syncwarp();
  const bool appended = ok32 || (go64 && S.misc[0] != 0);
  // q depends on the chosen columns: its FP32 attempt overwrote S.W; alpha of
  // the chosen ones again from the (unchanged) factor
  const bool restore = f32 && !appended;
  if (__any_sync(kFull, restore))
    grp_backsub<G>(restore, s, k - 1, __reduce_max_sync(kFull, restore ? k - 1 : 0), S);
  // residue r = y - A_Omega alpha
  if (appended) {
#pragma unroll
    for (int t = 0; t < NCH; ++t) rv[t] = yv[t];
  }
  if (appended) {
#pragma unroll
    for (int t = 0; t < NCH; ++t) {
      const float aj = S.W[k];
      rv[t].x = fmaf(-aj, aq[t].x, rv[t].x);
      rv[t].y = fmaf(-aj, aq[t].y, rv[t].y);
      rv[t].z = fmaf(-aj, aq[t].z, rv[t].z);
      rv[t].w = fmaf(-aj, aq[t].w, rv[t].w);
    }
    // chosen columns two at a time, both rows' loads issued before use
    for (int j = 0; j < k; j += 2) {
      const bool two = j + 1 < k;
      float4 c0[NCH], c1[NCH];
      load_chunks_gen<G, NCH>(c0, S.colp[j], nv, s, true);
      load_chunks_gen<G, NCH>(c1, two ? S.colp[j + 1] : S.colp[j], nv, s, two);
      const float a0 = S.W[j], a1 = two ? S.W[j + 1] : 0.f;
#pragma unroll
      for (int t = 0; t < NCH; ++t) {
        rv[t].x = fmaf(-a1, c1[t].x, fmaf(-a0, c0[t].x, rv[t].x));
        rv[t].y = fmaf(-a1, c1[t].y, fmaf(-a0, c0[t].y, rv[t].y));
        rv[t].z = fmaf(-a1, c1[t].z, fmaf(-a0, c0[t].z, rv[t].z));
        rv[t].w = fmaf(-a1, c1[t].w, fmaf(-a0, c0[t].w, rv[t].w));
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
// State initialisation: r = y, empty supports.
// ---------------------------------------------------------------------------
__global__ void omp_init_kernel(const float *__restrict__ Y, int64_t B, int M, int Mp,
                                const int32_t *__restrict__ perm, OmpState st) {
  // four consecutive elements per thread (M and Mp are multiples of 4)
  const int64_t e4 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e4 < B * M / 4) reinterpret_cast<float4 *>(st.R)[e4] = __ldg(reinterpret_cast<const float4 *>(Y) + e4);
  if (st.Rbf && e4 < B * Mp / 4) {
    const int64_t p = e4 / (Mp / 4);
    const int m = 4 * (int)(e4 - p * (Mp / 4));
    const int64_t b = perm ? perm[p] : p;
    const float4 v = m < M ? __ldg(reinterpret_cast<const float4 *>(Y + b * M + m)) : make_float4(0.f, 0.f, 0.f, 0.f);
    __nv_bfloat162 *o = reinterpret_cast<__nv_bfloat162 *>(st.Rbf + 4 * e4);
    o[0] = __floats2bfloat162_rn(v.x, v.y);
    o[1] = __floats2bfloat162_rn(v.z, v.w);
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int64_t e = 4 * e4 + u;
    if (e < B * st.ldo) { st.omega[e] = -1; st.alpha[e] = 0.f; }
    if (e < B) { st.k_eff[e] = 0; st.flags[e] = 0; }
  }
}

// ---------------------------------------------------------------------------
// FP32 proxy (FP32 CUDA cores): a tile of 128 patches x 128 atoms per step,
// 256 threads as 16 x 16, each owning 8 patches x 8 atoms; the contraction
// over M runs in chunks of 16 through double-buffered shared memory (the next
// chunk is loaded into registers while the current one is used).  Fused
// epilogue: |score| / ||a_i|| (shared or per-patch norms), chosen atoms masked
// through a per-tile bit set, running argmax as packed keys (ties to the lowest
// index).  With few patch tiles the atoms are split over grid.y CTAs whose
// best keys meet in `keys` by atomicMax; proxy_keys_kernel then writes cand.
// ---------------------------------------------------------------------------
constexpr int PF_TP = 128, PF_TA = 128, PF_KC = 16, PF_LD = PF_TP + 4;

__host__ __device__ inline size_t proxy_fp32_smem(int ldo) {
  return sizeof(float) * 4 * PF_KC * PF_LD + sizeof(uint32_t) * PF_TP * 4 + sizeof(int) * (PF_TP * ldo + PF_TP) +
         sizeof(int64_t) * PF_TP + 16;
}

__global__ void __launch_bounds__(256, 1)
proxy_fp32_kernel(const float *__restrict__ R, int M, const float *__restrict__ A,
                  const float *__restrict__ inv_norm, int T, const int32_t *__restrict__ ids,
                  int64_t n, const int32_t *__restrict__ omega, int ldo,
                  const int8_t *__restrict__ k_eff, const uint8_t *__restrict__ flags,
                  int32_t *__restrict__ cand, const float *__restrict__ pinv, int tiles_per_split,
                  unsigned long long *__restrict__ keys) {
  extern __shared__ __align__(16) float smem[];
  float *Rs = smem;                             // [2][PF_KC][PF_LD]  residual chunk, k-major
  float *As = Rs + 2 * PF_KC * PF_LD;           // [2][PF_KC][PF_LD]  atom chunk, k-major
  uint32_t *msk = reinterpret_cast<uint32_t *>(As + 2 * PF_KC * PF_LD);  // [PF_TP][4] chosen atoms of the tile
  int *Om = reinterpret_cast<int *>(msk + PF_TP * 4);                    // [PF_TP][ldo]
  int *Kc = Om + PF_TP * ldo;                                            // [PF_TP]
  int64_t *Pb = reinterpret_cast<int64_t *>(reinterpret_cast<uintptr_t>(Kc + PF_TP + 3) & ~uintptr_t(7));
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  const int64_t p0 = (int64_t)blockIdx.x * PF_TP;
  for (int p = tid; p < PF_TP; p += 256) {
    const int64_t pi = p0 + p;
    const int64_t bb = pi < n ? (ids ? ids[pi] : pi) : 0;
    Kc[p] = pi < n ? k_eff[bb] : 0;
    Pb[p] = bb;
  }
  __syncthreads();
  for (int e = tid; e < PF_TP * ldo; e += 256) {
    const int p = e / ldo;
    Om[e] = (p0 + p < n) ? omega[Pb[p] * ldo + (e - p * ldo)] : -1;
  }
  // global -> register chunk loader: thread t covers row t / 2, k offsets (t & 1) * 8 .. + 7
  const int lrow = tid >> 1, lk = (tid & 1) * 8;
  const bool rrow_ok = p0 + lrow < n;
  const float *rrow = R + (rrow_ok ? Pb[lrow] : 0) * (int64_t)M;
  const int a_lo = blockIdx.y * tiles_per_split * PF_TA;
  const int a_hi = min(T, a_lo + tiles_per_split * PF_TA);
  unsigned long long best[8] = {0ull, 0ull, 0ull, 0ull, 0ull, 0ull, 0ull, 0ull};
  for (int a0 = a_lo; a0 < a_hi; a0 += PF_TA) {
    const bool arow_ok = a0 + lrow < T;
    const float *arow = A + (arow_ok ? a0 + lrow : 0) * (int64_t)M;
    __syncthreads();  // the previous tile's epilogue no longer reads msk
    for (int e = tid; e < PF_TP * 4; e += 256) msk[e] = 0u;
    __syncthreads();
    for (int e = tid; e < PF_TP * ldo; e += 256) {
      const int p = e / ldo, j = e - p * ldo, a = Om[e] - a0;
      if (j < Kc[p] && a >= 0 && a < PF_TA) atomicOr(&msk[p * 4 + (a >> 5)], 1u << (a & 31));
    }
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
    float4 gr[2], ga[2];
    auto load = [&](int k0) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int k = k0 + lk + 4 * h;
        gr[h] = (rrow_ok && k < M) ? __ldg(reinterpret_cast<const float4 *>(rrow + k)) : make_float4(0.f, 0.f, 0.f, 0.f);
        ga[h] = (arow_ok && k < M) ? __ldg(reinterpret_cast<const float4 *>(arow + k)) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
    };
    auto stash = [&](int buf) {
      float *rs = Rs + buf * PF_KC * PF_LD, *as = As + buf * PF_KC * PF_LD;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int k = lk + 4 * h;
        rs[(k + 0) * PF_LD + lrow] = gr[h].x;
        rs[(k + 1) * PF_LD + lrow] = gr[h].y;
        rs[(k + 2) * PF_LD + lrow] = gr[h].z;
        rs[(k + 3) * PF_LD + lrow] = gr[h].w;
        as[(k + 0) * PF_LD + lrow] = ga[h].x;
        as[(k + 1) * PF_LD + lrow] = ga[h].y;
        as[(k + 2) * PF_LD + lrow] = ga[h].z;
        as[(k + 3) * PF_LD + lrow] = ga[h].w;
      }
    };
    load(0);
    stash(0);
    __syncthreads();
    int buf = 0;
    for (int k0 = 0; k0 < M; k0 += PF_KC) {
      const bool more = k0 + PF_KC < M;
      if (more) load(k0 + PF_KC);
      const float *rs = Rs + buf * PF_KC * PF_LD, *as = As + buf * PF_KC * PF_LD;
#pragma unroll 4
      for (int kk = 0; kk < PF_KC; ++kk) {
        const float4 r0 = *reinterpret_cast<const float4 *>(rs + kk * PF_LD + ty * 8);
        const float4 r1 = *reinterpret_cast<const float4 *>(rs + kk * PF_LD + ty * 8 + 4);
        const float4 x0 = *reinterpret_cast<const float4 *>(as + kk * PF_LD + tx * 8);
        const float4 x1 = *reinterpret_cast<const float4 *>(as + kk * PF_LD + tx * 8 + 4);
        const float rv[8] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w};
        const float av[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
          for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(rv[i], av[j], acc[i][j]);
      }
      if (more) stash(buf ^ 1);
      __syncthreads();
      buf ^= 1;
    }
    // epilogue: masked angle scores, running argmax per patch
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int p = ty * 8 + i;
      const uint32_t m32 = msk[p * 4 + (tx >> 2)];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int ai = a0 + tx * 8 + j;
        if (ai >= a_hi) continue;
        const float inv = pinv ? __ldg(pinv + Pb[p] * (int64_t)T + ai) : __ldg(inv_norm + ai);
        if (!(inv > 0.f) || ((m32 >> ((tx & 3) * 8 + j)) & 1u)) continue;
        const unsigned long long key = pack_key(fabsf(acc[i][j]) * inv, ai);
        best[i] = key > best[i] ? key : best[i];
      }
    }
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    unsigned long long v = best[i];
#pragma unroll
    for (int o = 8; o; o >>= 1) {
      const unsigned long long w = __shfl_xor_sync(kFull, v, o);
      v = w > v ? w : v;
    }
    const int64_t pi = p0 + ty * 8 + i;
    if (tx == 0 && pi < n) {
      const int64_t b = Pb[ty * 8 + i];
      if (keys) {
        if (v) atomicMax(keys + b, v);
      } else {
        cand[b * kTopP] = v ? key_idx(v) : -1;
#pragma unroll
        for (int c = 1; c < kTopP; ++c) cand[b * kTopP + c] = -1;
      }
    }
  }
}

// Split atom range: cand from the merged best keys (and the keys reset for the
// next iteration).
__global__ void proxy_keys_kernel(unsigned long long *__restrict__ keys, const int32_t *__restrict__ ids, int64_t n,
                                  int32_t *__restrict__ cand) {
  const int64_t wi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (wi >= n) return;
  const int64_t b = ids ? ids[wi] : wi;
  const unsigned long long v = keys[b];
  keys[b] = 0ull;
  cand[b * kTopP] = v ? key_idx(v) : -1;
#pragma unroll
  for (int c = 1; c < kTopP; ++c) cand[b * kTopP + c] = -1;
}

constexpr int GRP_WARPS = 4;

// ---------------------------------------------------------------------------
// Restricted OMP (fine step of Algorithm 2), all iterations, one group per
// patch.  Candidates C = children of the coarser support (disjoint lists:
// every finer atom has one parent).  The first capS candidate rows are copied
// once into per-group shared memory (cp.async, rows padded to M + 4 floats so
// that lanes reading different rows hit different banks); further candidates
// are read from the L2-resident effective dictionary.  The proxy gives each
// lane whole candidates (full-row dot products against r in shared memory,
// no shuffles), then one group max; the projection uses the staged rows.
// ---------------------------------------------------------------------------
__host__ __device__ inline int rs_group_bytes(int M, int Kb, int cap, int capS) {
  const int b = grp_smem_bytes(Kb, cap) + up16(4 * M) + 4 * capS * (M + 4);
  return (b + 127) / 128 * 128 + 16;  // odd multiple of 16 bytes mod 128: group blocks start on different banks
}

__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}

template <int G, int NCH>
__global__ void __launch_bounds__(GRP_WARPS * 32)
omp_restricted_staged_kernel(const float *__restrict__ Y, int M, const float *__restrict__ A,
                      const float *__restrict__ inv_norm, const int32_t *__restrict__ ids, int64_t n,
                      const int32_t *__restrict__ child_off, const int32_t *__restrict__ child_idx,
                      int cap, int capS, const int32_t *__restrict__ omega_up, int ldo_up,
                      const int8_t *__restrict__ keff_up, const int8_t *__restrict__ Kp, int Kuni,
                      int Kb, int32_t *__restrict__ omega, float *__restrict__ alpha, int ldo,
                      int8_t *__restrict__ k_eff, int64_t *stats, const float *__restrict__ gram, int T,
                      int64_t a_pstride, int64_t inv_pstride, bool cpos) {
  constexpr int NG = 32 / G;
  extern __shared__ __align__(16) char smem_raw[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, s = lane & (G - 1), g = lane / G;
  const int64_t wbase = ((int64_t)blockIdx.x * GRP_WARPS + wib) * NG;
  if (wbase >= n) return;  // whole warp
  const int64_t wi = wbase + g;
  const bool valid = wi < n;
  const int64_t b = valid ? (ids ? ids[wi] : wi) : 0;
  A += b * a_pstride;            // per-patch effective dictionary (stride 0: shared)
  inv_norm += b * inv_pstride;
  char *gbase = smem_raw + (size_t)(wib * NG + g) * rs_group_bytes(M, Kb, cap, capS);
  const GrpSmem S = carve(gbase, Kb, cap);
  float *rs = reinterpret_cast<float *>(gbase + grp_smem_bytes(Kb, cap));
  float *rows = rs + ((M + 3) & ~3);
  const int ldr = M + 4;
  const int nv = M >> 2;
  int Kpb = valid ? (Kp ? (int)Kp[b] : Kuni) : 0;
  Kpb = Kpb < Kb ? Kpb : Kb;

  // candidate set f(Omega_up)
  int nc = 0;
  if (valid) {
    const int kup = keff_up[b];
    for (int j = 0; j < kup; ++j) {
      const int p = omega_up[b * ldo_up + j];
      const int c0 = child_off[p], c1 = child_off[p + 1];
      for (int i = s; i < c1 - c0; i += G)
        if (nc + i < cap) {
          const int a = child_idx[c0 + i];
          S.cs[nc + i] = a;
          S.invn[nc + i] = __ldg(inv_norm + (cpos ? nc + i : a));
        }
      nc += c1 - c0;
    }
    if (nc > cap) {
      if (s == 0) atomicAdd((unsigned long long *)&stats[3], 1ull);
      nc = cap;
    }
  }
  __syncwarp();
  // stage the first capS candidate rows
  const int nst = nc < capS ? nc : capS;
  for (int c = 0; c < nst; ++c) {
    const float *src = A + (int64_t)(cpos ? c : S.cs[c]) * M;
    float *dst = rows + c * ldr;
    for (int j = s; j < nv; j += G) cp_async16(dst + 4 * j, src + 4 * j);
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
  const float *yrow = Y + b * M;
  float4 yv[NCH], rv[NCH];
  load_chunks<G, NCH>(yv, yrow, nv, s, valid);
#pragma unroll
  for (int t = 0; t < NCH; ++t) {
    rv[t] = yv[t];
    const int j = s + G * t;
    if (j < nv) reinterpret_cast<float4 *>(rs)[j] = yv[t];
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  __syncwarp();
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
    // proxy: each lane scores whole candidates
    unsigned long long best = 0ull;
    if (act)
      for (int c = s; c < nc; c += G) {
        const float inv = S.invn[c];
        if (!(inv > 0.f)) continue;
        const float *row = c < capS ? rows + c * ldr : A + (int64_t)(cpos ? c : S.cs[c]) * M;
        const unsigned long long key = pack_key(fabsf(row_dot(row, rs, nv)) * inv, S.cs[c]);
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
    const float *aqp = (act && qs < capS) ? rows + qs * ldr : A + (int64_t)(cpos ? qs : q) * M;
    const bool ok = grp_append<G, NCH, false>(act, s, M, aqp, yrow, q, k, yv, rv, S, fl, rsq, stats, gram, T);
    if (act) {
      if (ok) {
        ++k;
#pragma unroll
        for (int t = 0; t < NCH; ++t) {
          const int j = s + G * t;
          if (j < nv) reinterpret_cast<float4 *>(rs)[j] = rv[t];
        }
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
}

// Variant without staging: candidate rows are read from the L2-resident effective
// dictionary on every pass, G = 4..16 lanes cooperate on each row (two rows per
// pass), and the projection reads its columns from global memory.
template <int G, int NCH>
__global__ void __launch_bounds__(GRP_WARPS * 32)
omp_restricted_coop_kernel(const float *__restrict__ Y, int M, const float *__restrict__ A,
                      const float *__restrict__ inv_norm, const int32_t *__restrict__ ids, int64_t n,
                      const int32_t *__restrict__ child_off, const int32_t *__restrict__ child_idx,
                      int cap, const int32_t *__restrict__ omega_up, int ldo_up,
                      const int8_t *__restrict__ keff_up, const int8_t *__restrict__ Kp, int Kuni,
                      int Kb, int32_t *__restrict__ omega, float *__restrict__ alpha, int ldo,
                      int8_t *__restrict__ k_eff, int64_t *stats, const float *__restrict__ gram, int T,
                      int64_t a_pstride, int64_t inv_pstride, bool cpos) {
  constexpr int NG = 32 / G;
  extern __shared__ __align__(16) char smem_raw[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, s = lane & (G - 1), g = lane / G;
  const int64_t wbase = ((int64_t)blockIdx.x * GRP_WARPS + wib) * NG;
  if (wbase >= n) return;  // whole warp
  const int64_t wi = wbase + g;
  const bool valid = wi < n;
  const int64_t b = valid ? (ids ? ids[wi] : wi) : 0;
  A += b * a_pstride;            // per-patch effective dictionary (stride 0: shared)
  inv_norm += b * inv_pstride;
  const GrpSmem S = carve(smem_raw + (size_t)(wib * NG + g) * grp_smem_bytes(Kb, cap), Kb, cap);
  const int nv = M >> 2;
  int Kpb = valid ? (Kp ? (int)Kp[b] : Kuni) : 0;
  Kpb = Kpb < Kb ? Kpb : Kb;

  // candidate set f(Omega_up)
  int nc = 0;
  if (valid) {
    const int kup = keff_up[b];
    for (int j = 0; j < kup; ++j) {
      const int p = omega_up[b * ldo_up + j];
      const int c0 = child_off[p], c1 = child_off[p + 1];
      for (int i = s; i < c1 - c0; i += G)
        if (nc + i < cap) {
          const int a = child_idx[c0 + i];
          S.cs[nc + i] = a;
          S.invn[nc + i] = __ldg(inv_norm + (cpos ? nc + i : a));
        }
      nc += c1 - c0;
    }
    if (nc > cap) {
      if (s == 0) atomicAdd((unsigned long long *)&stats[3], 1ull);
      nc = cap;
    }
  }
  __syncwarp();
  const float *yrow = Y + b * M;
  float4 yv[NCH], rv[NCH];
  load_chunks<G, NCH>(yv, yrow, nv, s, valid);
#pragma unroll
  for (int t = 0; t < NCH; ++t) rv[t] = yv[t];
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
    // proxy over the candidates, two per pass
    unsigned long long best = 0ull;
    const int ncw = __reduce_max_sync(kFull, act ? nc : 0);
    for (int c = 0; c < ncw; c += 2) {
      const bool ok0 = act && c < nc && S.invn[c] > 0.f;
      const bool ok1 = act && c + 1 < nc && S.invn[c + 1] > 0.f;
      float4 a0[NCH], a1[NCH];
      load_chunks<G, NCH>(a0, A + (int64_t)(ok0 ? (cpos ? c : S.cs[c]) : 0) * M, nv, s, ok0);
      load_chunks<G, NCH>(a1, A + (int64_t)(ok1 ? (cpos ? c + 1 : S.cs[c + 1]) : 0) * M, nv, s, ok1);
      const float p0 = gsum<G>(dotc<NCH>(a0, rv));
      const float p1 = gsum<G>(dotc<NCH>(a1, rv));
      if (ok0) {
        const unsigned long long key = pack_key(fabsf(p0) * S.invn[c], S.cs[c]);
        best = key > best ? key : best;
      }
      if (ok1) {
        const unsigned long long key = pack_key(fabsf(p1) * S.invn[c + 1], S.cs[c + 1]);
        best = key > best ? key : best;
      }
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
    const bool ok = grp_append<G, NCH, true>(act, s, M, A + (int64_t)(cpos ? qs : q) * M, yrow, q, k, yv, rv, S, fl,
                                             rsq, stats, gram, T);
    if (act) {
      if (ok) ++k;
      else act = false;
    }
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
}

inline unsigned blocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// Gram matrix G = A A^T of an effective dictionary (rows a_i): 64 x 64 output
// tiles, FP32, 4 x 4 outputs per thread.
__global__ void __launch_bounds__(256) gram_kernel(const float *__restrict__ A, int T, int M, float *__restrict__ Gm) {
  __shared__ float As[32][64 + 4], Bs[32][64 + 4];
  const int i0 = blockIdx.y * 64, j0 = blockIdx.x * 64;
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  float acc[4][4] = {};
  for (int m0 = 0; m0 < M; m0 += 32) {
    for (int e = tid; e < 64 * 32; e += 256) {
      const int r = e >> 5, mm = e & 31;
      As[mm][r] = (i0 + r < T && m0 + mm < M) ? A[(int64_t)(i0 + r) * M + m0 + mm] : 0.f;
      Bs[mm][r] = (j0 + r < T && m0 + mm < M) ? A[(int64_t)(j0 + r) * M + m0 + mm] : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int mm = 0; mm < 32; ++mm)
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[a][c] = fmaf(As[mm][ty * 4 + a], Bs[mm][tx * 4 + c], acc[a][c]);
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int i = i0 + ty * 4 + a, j = j0 + tx * 4 + c;
      if (i < T && j < T) Gm[(int64_t)i * T + j] = acc[a][c];
    }
}

// (G, NCH) by problem dimension: M <= 16 G NCH, NCH <= 4.
template <typename F>
bool dispatch_group(int M, F &&f) {
  if (M % 4) return false;
  if (M <= 16) f(std::integral_constant<int, 4>{}, std::integral_constant<int, 1>{});
  else if (M <= 32) f(std::integral_constant<int, 4>{}, std::integral_constant<int, 2>{});
  else if (M <= 64) f(std::integral_constant<int, 4>{}, std::integral_constant<int, 4>{});
  else if (M <= 128) f(std::integral_constant<int, 8>{}, std::integral_constant<int, 4>{});
  else if (M <= 256) f(std::integral_constant<int, 16>{}, std::integral_constant<int, 4>{});
  else return false;
  return true;
}

int group_size(int M) { return M <= 64 ? 4 : (M <= 128 ? 8 : 16); }

}  // namespace

bool omp_dims_supported(int M) { return M > 0 && M % 4 == 0 && M <= 256; }

void launch_gram(const float *A, int T, int M, float *Gm, cudaStream_t s) {
  if (T == 0) return;
  const dim3 grid((unsigned)((T + 63) / 64), (unsigned)((T + 63) / 64));
  gram_kernel<<<grid, 256, 0, s>>>(A, T, M, Gm);
}

void launch_omp_init(const float *Y, int64_t B, int M, int Mp, const int32_t *perm, OmpState st, cudaStream_t s) {
  int64_t n = B * (int64_t)(M > Mp ? M : Mp);
  n = n > B * st.ldo ? n : B * st.ldo;
  if (n == 0) return;
  omp_init_kernel<<<blocks((n + 3) / 4, 256), 256, 0, s>>>(Y, B, M, Mp, perm, st);
}

int proxy_fp32_splits(int64_t n, int T) {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 1;
  }
  const int64_t tiles = (n + PF_TP - 1) / PF_TP;
  const int n_at = (T + PF_TA - 1) / PF_TA;
  if (tiles >= 2 * sms || n_at < 2) return 1;
  const int S = (int)((2 * sms + tiles - 1) / tiles);  // about two CTAs per SM
  return S < n_at ? S : n_at;
}

void launch_proxy_fp32(const float *R, int M, const float *A, const float *inv_norm, int T,
                       const int32_t *ids, int64_t n, const int32_t *omega, int ldo,
                       const int8_t *k_eff, const uint8_t *flags, int32_t *cand, const float *pinv,
                       unsigned long long *keys, cudaStream_t s) {
  if (n == 0) return;
  const size_t sm = proxy_fp32_smem(ldo);
  // the attribute is per device and function: set it on every launch (a host-side call)
  if (sm > 48 * 1024) cudaFuncSetAttribute(proxy_fp32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  const int n_all = (T + PF_TA - 1) / PF_TA;
  const int S = keys ? proxy_fp32_splits(n, T) : 1;
  const int tps = (n_all + S - 1) / S;
  const dim3 grid((unsigned)((n + PF_TP - 1) / PF_TP), (unsigned)((n_all + tps - 1) / tps));
  unsigned long long *kk = grid.y > 1 ? keys : nullptr;
  proxy_fp32_kernel<<<grid, 256, sm, s>>>(R, M, A, inv_norm, T, ids, n, omega, ldo, k_eff, flags, cand, pinv, tps,
                                          kk);
  if (kk) proxy_keys_kernel<<<blocks(n, 256), 256, 0, s>>>(kk, ids, n, cand);
}

// P0 = Y A^T for the patches ids[0..n) (all correlations <a_i, y_b> of a
// shared dictionary: the starting point of the Gram form of the full-dictionary
// level).  The GEMM of proxy_fp32_kernel (128 patches x 128 atoms per CTA, 8 x 8
// per thread, contraction in double-buffered chunks of 16) with an epilogue that
// stores the FP32 products row by row: P0[b][a], b the patch id.
__global__ void __launch_bounds__(256)
p0_gemm_kernel(const float *__restrict__ Y, int M, const float *__restrict__ A, int T,
               const int32_t *__restrict__ ids, int64_t n, float *__restrict__ P0) {
  __shared__ __align__(16) float Rs[2 * PF_KC * PF_LD];
  __shared__ __align__(16) float As[2 * PF_KC * PF_LD];
  __shared__ int64_t Pb[PF_TP];
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  const int64_t p0 = (int64_t)blockIdx.x * PF_TP;
  const int a0 = blockIdx.y * PF_TA;
  for (int p = tid; p < PF_TP; p += 256) {
    const int64_t pi = p0 + p;
    Pb[p] = pi < n ? (ids ? ids[pi] : pi) : -1;
  }
  __syncthreads();
  const int lrow = tid >> 1, lk = (tid & 1) * 8;
  const bool rrow_ok = Pb[lrow] >= 0;
  const float *rrow = Y + (rrow_ok ? Pb[lrow] : 0) * (int64_t)M;
  const bool arow_ok = a0 + lrow < T;
  const float *arow = A + (arow_ok ? a0 + lrow : 0) * (int64_t)M;
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
  float4 gr[2], ga[2];
  auto load = [&](int k0) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int k = k0 + lk + 4 * h;
      gr[h] = (rrow_ok && k < M) ? __ldg(reinterpret_cast<const float4 *>(rrow + k)) : make_float4(0.f, 0.f, 0.f, 0.f);
      ga[h] = (arow_ok && k < M) ? __ldg(reinterpret_cast<const float4 *>(arow + k)) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
  };
  auto stash = [&](int buf) {
    float *rs = Rs + buf * PF_KC * PF_LD, *as = As + buf * PF_KC * PF_LD;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int k = lk + 4 * h;
      rs[(k + 0) * PF_LD + lrow] = gr[h].x;
      rs[(k + 1) * PF_LD + lrow] = gr[h].y;
      rs[(k + 2) * PF_LD + lrow] = gr[h].z;
      rs[(k + 3) * PF_LD + lrow] = gr[h].w;
      as[(k + 0) * PF_LD + lrow] = ga[h].x;
      as[(k + 1) * PF_LD + lrow] = ga[h].y;
      as[(k + 2) * PF_LD + lrow] = ga[h].z;
      as[(k + 3) * PF_LD + lrow] = ga[h].w;
    }
  };
  load(0);
  stash(0);
  __syncthreads();
  int buf = 0;
  for (int k0 = 0; k0 < M; k0 += PF_KC) {
    const bool more = k0 + PF_KC < M;
    if (more) load(k0 + PF_KC);
    const float *rs = Rs + buf * PF_KC * PF_LD, *as = As + buf * PF_KC * PF_LD;
#pragma unroll 4
    for (int kk = 0; kk < PF_KC; ++kk) {
      const float4 r0 = *reinterpret_cast<const float4 *>(rs + kk * PF_LD + ty * 8);
      const float4 r1 = *reinterpret_cast<const float4 *>(rs + kk * PF_LD + ty * 8 + 4);
      const float4 x0 = *reinterpret_cast<const float4 *>(as + kk * PF_LD + tx * 8);
      const float4 x1 = *reinterpret_cast<const float4 *>(as + kk * PF_LD + tx * 8 + 4);
      const float rv[8] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w};
      const float av[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(rv[i], av[j], acc[i][j]);
    }
    if (more) stash(buf ^ 1);
    __syncthreads();
    buf ^= 1;
  }
  // rows of 8 consecutive atoms per thread: two float4 stores when the row is whole
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int64_t b = Pb[ty * 8 + i];
    if (b < 0) continue;
    const int a = a0 + tx * 8;
    float *dst = P0 + b * (int64_t)T + a;
    if (a + 8 <= T && (T & 3) == 0) {
      reinterpret_cast<float4 *>(dst)[0] = make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
      reinterpret_cast<float4 *>(dst)[1] = make_float4(acc[i][4], acc[i][5], acc[i][6], acc[i][7]);
    } else {
#pragma unroll
      for (int j = 0; j < 8; ++j)
        if (a + j < T) dst[j] = acc[i][j];
    }
  }
}

// (G, NCH) of the restricted kernel: wide groups (one candidate per lane).
template <typename F>
bool dispatch_group_wide(int M, F &&f) {
  if (M % 4) return false;
  if (M <= 64) f(std::integral_constant<int, 16>{}, std::integral_constant<int, 1>{});
  else if (M <= 128) f(std::integral_constant<int, 32>{}, std::integral_constant<int, 1>{});
  else if (M <= 256) f(std::integral_constant<int, 32>{}, std::integral_constant<int, 2>{});
  else return false;
  return true;
}

// ---- work order: counting sort of the patches by budget, largest first ----
__global__ void budget_hist_kernel(const int8_t *__restrict__ K, int64_t n, int *__restrict__ hist) {
  __shared__ int h[CSP_MAX_K + 1];
  for (int i = threadIdx.x; i <= CSP_MAX_K; i += blockDim.x) h[i] = 0;
  __syncthreads();
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < n; b += (int64_t)gridDim.x * blockDim.x) {
    int k = K[b];
    k = k < 0 ? 0 : (k > CSP_MAX_K ? CSP_MAX_K : k);
    atomicAdd(&h[k], 1);
  }
  __syncthreads();
  for (int i = threadIdx.x; i <= CSP_MAX_K; i += blockDim.x)
    if (h[i]) atomicAdd(&hist[i], h[i]);
}

// cursor[k] = number of patches with a larger budget (the start of bucket k)
__global__ void budget_scan_kernel(int *__restrict__ hist, int *__restrict__ cursor) {
  if (threadIdx.x != 0) return;
  int acc = 0;
  for (int k = CSP_MAX_K; k >= 0; --k) {
    cursor[k] = acc;
    acc += hist[k];
  }
}

__global__ void budget_scatter_kernel(const int8_t *__restrict__ K, int64_t n, int *__restrict__ cursor,
                                      int32_t *__restrict__ ids) {
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < n; b += (int64_t)gridDim.x * blockDim.x) {
    int k = K[b];
    k = k < 0 ? 0 : (k > CSP_MAX_K ? CSP_MAX_K : k);
    ids[atomicAdd(&cursor[k], 1)] = (int32_t)b;
  }
}

void launch_sort_by_budget(const int8_t *K, int64_t n, int32_t *ids, int *counts, cudaStream_t s) {
  if (n == 0) return;
  cudaMemsetAsync(counts, 0, sizeof(int) * 2 * (CSP_MAX_K + 1), s);
  const unsigned g = (unsigned)std::min<int64_t>((n + 255) / 256, 1024);
  budget_hist_kernel<<<g, 256, 0, s>>>(K, n, counts);
  budget_scan_kernel<<<1, 32, 0, s>>>(counts, counts + CSP_MAX_K + 1);
  budget_scatter_kernel<<<g, 256, 0, s>>>(K, n, counts + CSP_MAX_K + 1, ids);
}

void launch_p0_gemm(const float *Y, int M, const float *A, int T, const int32_t *ids, int64_t n, float *P0,
                    cudaStream_t s) {
  if (n == 0) return;
  const dim3 grid((unsigned)((n + PF_TP - 1) / PF_TP), (unsigned)((T + PF_TA - 1) / PF_TA));
  p0_gemm_kernel<<<grid, 256, 0, s>>>(Y, M, A, T, ids, n, P0);
}

constexpr size_t kMaxSmemPerCta = 227 * 1024;  // dynamic shared memory of one CTA at most (opt-in)

bool launch_omp_restricted(int variant, const float *Y, int M, const float *A, const float *inv_norm,
                           const int32_t *ids, int64_t n, const int32_t *child_off,
                           const int32_t *child_idx, int cap, const int32_t *omega_up, int ldo_up,
                           const int8_t *keff_up, const int8_t *Kp, int Kuni, int Kb,
                           int32_t *omega, float *alpha, int ldo, int8_t *k_eff, int64_t *stats,
                           const float *gram, int T, int64_t a_pstride, int64_t inv_pstride, bool cpos,
                           cudaStream_t s, const float *D0, int N0, float *Xh, unsigned long long *queue,
                           const float *gpp) {
  if (n == 0) return false;
  if (gpp && cpos && variant >= 2) {
    // per-patch rows with their Gram blocks: the Gram-Schmidt form, the variant's
    // lane width or the narrowest wider one whose shared memory fits
    for (int width = variant >= 8 ? 1 : (variant - 2) % 3; width <= 2; ++width)
      if (restricted_gram_smem(width, true, M, Kb, cap, true) <= kMaxSmemPerCta)
        return launch_omp_restricted_gram(width, true, Y, M, A, inv_norm, ids, n, child_off, child_idx, cap,
                                          omega_up, ldo_up, keff_up, Kp, Kuni, Kb, omega, alpha, ldo, k_eff, stats,
                                          nullptr, T, D0, N0, Xh, s, queue, gpp, a_pstride, inv_pstride);
  }
  if (variant >= 2 && (!gram || a_pstride || cpos)) variant = 0;  // the Gram variants need the level's shared Gram matrix
  if (variant >= 2 && variant < 8 && restricted_gram_smem((variant - 2) % 3, variant >= 5, M, Kb, cap, false) >
                                         kMaxSmemPerCta)
    variant = 0;  // candidate sets too large for the Gram forms' shared memory
  if (variant >= 8) {  // 8-10 (11-13 with the Gram block staged): register-resident candidates, 8 / 16 / 4 lanes
    bool sy = false;
    const int vv = variant >= 11 ? variant - 3 : variant;
    if (launch_omp_restricted_reg(vv == 8 ? 8 : (vv == 9 ? 16 : 4), Y, M, A, inv_norm, ids, n, child_off,
                                  child_idx, cap,
                                  omega_up, ldo_up, keff_up, Kp, Kuni, Kb, omega, alpha, ldo, k_eff, stats, gram, T,
                                  D0, N0, Xh, &sy, s, variant >= 11))
      return sy;
    variant = 6;  // shape outside the register form: the shared-memory Gram-Schmidt form
  }
  if (variant >= 2)  // 2-4: Gram proxy p0 - G alpha; 5-7: Gram-Schmidt form; narrow to wide lane groups
    return launch_omp_restricted_gram((variant - 2) % 3, variant >= 5, Y, M, A, inv_norm, ids, n, child_off,
                                      child_idx, cap, omega_up, ldo_up, keff_up, Kp, Kuni, Kb, omega, alpha, ldo,
                                      k_eff, stats, gram, T, D0, N0, Xh, s, queue);
  if (variant == 0) {
    const int G = group_size(M);
    const int per_cta = GRP_WARPS * (32 / G);
    const size_t sm = (size_t)grp_smem_bytes(Kb, cap) * per_cta;
    dispatch_group(M, [&](auto gc, auto nc) {
      constexpr int GG = decltype(gc)::value, NCH = decltype(nc)::value;
      if (sm > 48 * 1024)
        cudaFuncSetAttribute(omp_restricted_coop_kernel<GG, NCH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      omp_restricted_coop_kernel<GG, NCH><<<blocks(n, per_cta), GRP_WARPS * 32, sm, s>>>(
          Y, M, A, inv_norm, ids, n, child_off, child_idx, cap, omega_up, ldo_up, keff_up, Kp, Kuni, Kb, omega,
          alpha, ldo, k_eff, stats, gram, T, a_pstride, inv_pstride, cpos);
    });
    return false;
  }
  const int G = M <= 64 ? 16 : 32;
  const int per_cta = GRP_WARPS * (32 / G);
  // staged rows per patch: about 6 KB of rows (at least 4, at most the capacity)
  int capS = 6144 / (4 * (M + 4));
  capS = capS < 4 ? 4 : (capS > cap ? cap : capS);
  const size_t sm = (size_t)rs_group_bytes(M, Kb, cap, capS) * per_cta;
  dispatch_group_wide(M, [&](auto gc, auto nc) {
    constexpr int GG = decltype(gc)::value, NCH = decltype(nc)::value;
    if (sm > 48 * 1024)
      cudaFuncSetAttribute(omp_restricted_staged_kernel<GG, NCH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    omp_restricted_staged_kernel<GG, NCH><<<blocks(n, per_cta), GRP_WARPS * 32, sm, s>>>(
        Y, M, A, inv_norm, ids, n, child_off, child_idx, cap, capS, omega_up, ldo_up, keff_up, Kp, Kuni, Kb,
        omega, alpha, ldo, k_eff, stats, gram, T, a_pstride, inv_pstride, cpos);
  });
  return false;
}

}  // namespace csp
