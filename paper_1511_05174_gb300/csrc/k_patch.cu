// Patch extraction, scale operators W/U, effective dictionaries and
// overlap-add aggregation.
//
//  * extraction: y_p = the measurement pixels under patch p (Sec. III-C,
//    y = Phi x + e; patches overlap, Sec. IV);
//  * W: uniform (box) downsampler of a patch vector to a coarser scale, U:
//    nearest-neighbour upsampler, W U = I (Sec. III-C, problem (P_low));
//  * effective dictionary of a scale: a_i = Phi U_l d_i (the operator of
//    (P_low) and, restricted, of (P_high)); for Phi = I the scale's own
//    dictionary D^(l) against W_l x (Algorithm 2);
//  * aggregation: x_hat_p = D_|Omega alpha, overlap-add averaged over the
//    covering patches (Sec. IV: overlapping patches).
#include <algorithm>

#include "csp_internal.cuh"

namespace csp {

namespace {

__device__ __forceinline__ int origin(int i, int stride, int extent, int P) {
  int o = i * stride;
  return o < extent - P ? o : extent - P;
}

// Index into a level-l patch vector of the level-0 position (ly, lx, py, px).
__device__ __forceinline__ int level_index(const GeomDev &g, int l, int ly, int lx, int py, int px) {
  const int fy = g.f[l][0], fx = g.f[l][1], sy = g.f[l][2], sx = g.f[l][3];
  const int Lxl = g.Lx / fx, Pyl = g.P / sy, Pxl = g.P / sx;
  return (((ly / fy) * Lxl + lx / fx) * Pyl + py / sy) * Pxl + px / sx;
}

// One thread per output element (b, m).  For every sensing kind the measurement
// of row m of patch b is meas[q][oy + py][ox + px] with q = m / (P*P) (plane for
// Phi = I, shot for coded aperture, 0 otherwise).
__global__ void extract_kernel(GeomDev g, const float *__restrict__ meas, float *__restrict__ Y,
                               int64_t B, int M) {
  // thread (x, y) of a block: four consecutive rows m = 4x of patch
  // blockIdx.x * blockDim.y + y (blockDim.x = M / 4; M and P are multiples of
  // 4, so the four lie in one row of the patch); no 64-bit divisions
  const int b = (int)(blockIdx.x * blockDim.y + threadIdx.y);  // B < 2^31 (launcher)
  if (b >= B) return;
  const int m = 4 * (int)threadIdx.x;
  const int iy = b / g.nx, ix = b - iy * g.nx;
  const int oy = origin(iy, g.stride, g.H, g.P), ox = origin(ix, g.stride, g.W, g.P);
  const int PP = g.P * g.P;
  const int q = m / PP, r = m - q * PP, py = r / g.P, px = r - py * g.P;
  const float *src = meas + ((int64_t)q * g.H + oy + py) * g.W + ox + px;
  reinterpret_cast<float4 *>(Y + (int64_t)b * M)[threadIdx.x] =
      make_float4(__ldg(src), __ldg(src + 1), __ldg(src + 2), __ldg(src + 3));
}

// Scalar variant for patch sides that are not a multiple of 4.
__global__ void extract1_kernel(GeomDev g, const float *__restrict__ meas, float *__restrict__ Y,
                                int64_t B, int M) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= B * M) return;
  const int64_t b = e / M;
  const int m = (int)(e - b * M);
  const int iy = (int)(b / g.nx), ix = (int)(b - (int64_t)iy * g.nx);
  const int oy = origin(iy, g.stride, g.H, g.P), ox = origin(ix, g.stride, g.W, g.P);
  const int PP = g.P * g.P;
  const int q = m / PP, r = m - q * PP, py = r / g.P, px = r - py * g.P;
  Y[e] = __ldg(meas + ((int64_t)q * g.H + oy + py) * g.W + ox + px);
}

// y_l = W_l y_0 for Phi = I: box average over the level's factor block.
__global__ void downsample_kernel(GeomDev g, int l, const float *__restrict__ Y0,
                                  float *__restrict__ Yl, int64_t B) {
  const int fy = g.f[l][0], fx = g.f[l][1], sy = g.f[l][2], sx = g.f[l][3];
  const int Lyl = g.Ly / fy, Lxl = g.Lx / fx, Pyl = g.P / sy, Pxl = g.P / sx;
  const int Nl = Lyl * Lxl * Pyl * Pxl, N0 = g.Ly * g.Lx * g.P * g.P;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= B * Nl) return;
  const int64_t b = e / Nl;
  int n = (int)(e - b * Nl);
  const int pxl = n % Pxl; n /= Pxl;
  const int pyl = n % Pyl; n /= Pyl;
  const int lxl = n % Lxl; const int lyl = n / Lxl;
  const float *y = Y0 + b * N0;
  float acc = 0.f;
  for (int a = 0; a < fy; ++a)
    for (int c = 0; c < fx; ++c)
      for (int d = 0; d < sy; ++d)
        for (int e2 = 0; e2 < sx; ++e2) {
          const int ly = lyl * fy + a, lx = lxl * fx + c, py = pyl * sy + d, px = pxl * sx + e2;
          acc += y[((ly * g.Lx + lx) * g.P + py) * g.P + px];
        }
  Yl[e] = acc / (float)(fy * fx * sy * sx);
}

// a_i[m] = (Phi U_l d_i)[m] for a Phi shared by all patches of one phase.
__global__ void effective_dict_kernel(GeomDev g, int kind, int shots, const uint8_t *__restrict__ codes,
                                      int l, int phase, const float *__restrict__ D, int T, int N,
                                      float *__restrict__ A, int M) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)T * M) return;
  const int i = (int)(e / M), m = (int)(e - (int64_t)i * M);
  const float *d = D + (int64_t)i * N;
  const int PP = g.P * g.P;
  float v = 0.f;
  if (kind == CSP_SENSE_BAYER_RGGB) {
    const int py = m / g.P, px = m - py * g.P;
    const int ry = ((phase >> 1) + py) & 1, rx = ((phase & 1) + px) & 1;
    const int ch = (ry == 0 && rx == 0) ? 0 : ((ry == 1 && rx == 1) ? 2 : 1);
    v = d[level_index(g, l, 0, ch, py, px)];
  } else if (kind == CSP_SENSE_CODED_APERTURE) {
    const int s = m / PP, r = m - s * PP, py = r / g.P, px = r - py * g.P;
    const int V = g.Ly * g.Lx;
    for (int vv = 0; vv < V; ++vv)
      if (codes[s * V + vv]) v += d[level_index(g, l, vv / g.Lx, vv % g.Lx, py, px)];
  } else {  // identity: the scale's own atoms
    v = d[m];
  }
  A[e] = v;
}

// Per-patch code blocks of per-pixel coded exposure: pc[b][(t * P + py) * P + px]
// = code[t][oy + py][ox + px] for the patch at (oy, ox) (plane grid 1 x F).
__global__ void patch_codes_kernel(GeomDev g, const uint8_t *__restrict__ codes, int64_t B,
                                   uint8_t *__restrict__ pc) {
  const int F = g.Lx, PP = g.P * g.P;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= B * F * PP) return;
  const int64_t b = e / (F * PP);
  const int r = (int)(e - b * F * PP);
  const int t = r / PP, m = r - t * PP, py = m / g.P, px = m - py * g.P;
  const int iy = (int)(b / g.nx), ix = (int)(b - (int64_t)iy * g.nx);
  const int oy = origin(iy, g.stride, g.H, g.P), ox = origin(ix, g.stride, g.W, g.P);
  pc[e] = codes[((int64_t)t * g.H + oy + py) * g.W + ox + px];
}


// Per-pixel coded exposure: the full per-patch effective dictionary of level l,
// a_i = Phi_p U_l d_i, and its row norms, one CTA per patch: the patch's code block is
// turned once into a table of level-element offsets (off[t][m] = the element of
// frame t, pixel m at level l, -1 where the code is 0) in shared memory; then a
// warp per atom row writes a_i[m] = sum_t d_i[off[t][m]] (frames in order) for
// m = lane, lane + 32, ... and the row's norm in the order
// of row_norms_kernel (per-lane FMA chain over its elements, then the xor tree),
// with the running maximum of the norms in *mx.  The index arithmetic is done
// once per patch instead of once per element and frame.
__global__ void __launch_bounds__(256)
effective_dict_pp_rows_kernel(GeomDev g, const uint8_t *__restrict__ pc, int l, const float *__restrict__ D, int T,
                              int N, float *__restrict__ A, float *__restrict__ nrm, unsigned int *mx, int64_t B) {
  extern __shared__ int pp_off[];  // [F][M]
  const int64_t b = blockIdx.x;
  if (b >= B) return;
  const int M = g.P * g.P, F = g.Lx;
  const uint8_t *cb = pc + b * (int64_t)F * M;
  for (int e = threadIdx.x; e < F * M; e += blockDim.x) {
    const int t = e / M, m = e - t * M, py = m / g.P, px = m - py * g.P;
    pp_off[e] = cb[e] ? level_index(g, l, 0, t, py, px) : -1;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  unsigned int wmax = 0u;
  for (int i = warp; i < T; i += nw) {
    const float *d = D + (int64_t)i * N;
    float *row = A + (b * T + i) * (int64_t)M;
    float sq = 0.f;
    for (int m = lane; m < M; m += 32) {
      float v = 0.f;
      for (int t = 0; t < F; ++t) {
        const int o = pp_off[t * M + m];
        if (o >= 0) v += __ldg(d + o);
      }
      row[m] = v;
      sq = fmaf(v, v, sq);
    }
    for (int o = 16; o; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
    if (lane == 0) {
      const float r = sqrtf(sq);
      nrm[b * T + i] = r;
      wmax = max(wmax, __float_as_uint(r));
    }
  }
  if (lane == 0 && wmax) atomicMax(mx, wmax);
}

// The candidate atoms f(Omega_up) of patch b in the order of the restricted
// kernels (parents in support order, each parent's children in link order, at
// most cap), listed by one warp: lane j takes parent j of each group of 32, and an
// inclusive scan of the children counts gives each parent its first slot.
// Returns the number listed (all lanes).
__device__ __forceinline__ int list_candidates_warp(int64_t b, const int32_t *__restrict__ omega_up, int ldo_up,
                                                    const int8_t *__restrict__ keff_up,
                                                    const int32_t *__restrict__ child_off,
                                                    const int32_t *__restrict__ child_idx, int cap, int *cs,
                                                    int lane) {
  const int kup = keff_up[b];
  int base = 0;
  for (int j0 = 0; j0 < kup && base < cap; j0 += 32) {
    const int j = j0 + lane;
    int lo = 0, cnt = 0;
    if (j < kup) {
      const int p = omega_up[b * ldo_up + j];
      lo = child_off[p];
      cnt = child_off[p + 1] - lo;
    }
    int inc = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += v;
    }
    const int first = base + inc - cnt;
    for (int i = 0; i < cnt && first + i < cap; ++i) cs[first + i] = child_idx[lo + i];
    base += __shfl_sync(0xffffffffu, inc, 31);
  }
  return base < cap ? base : cap;
}

// Candidate rows of per-pixel coded exposure at a restricted level: one CTA
// per patch.  The CTA lists f(Omega_up) in the order of the restricted kernels
// (parents in support order, each parent's children in link order, at most
// cap) and tabulates, per (frame t, pixel m), the offset of the level element
// d[level index of (t, m)] when the patch's code there is 1 (-1 otherwise);
// then a warp per candidate c writes a_c[m] = sum_t pc_p[t][m] d_c[...] -- the
// arithmetic and order of effective_dict_pp_rows_kernel -- and 1/||a_c|| (-1 for a
// zero row), the norm reduced as in row_norms_kernel.
__global__ void __launch_bounds__(256)
pp_candidates_kernel(GeomDev g, const uint8_t *__restrict__ pc, int l, const float *__restrict__ D, int N, int M,
                     const int32_t *__restrict__ omega_up, int ldo_up, const int8_t *__restrict__ keff_up,
                     const int32_t *__restrict__ child_off, const int32_t *__restrict__ child_idx, int cap,
                     int64_t B, float *__restrict__ Ac, float *__restrict__ invc) {
  extern __shared__ int sm_pp[];  // [F * M] element offsets (-1: code 0) | [cap] candidate atoms
  const int64_t b = blockIdx.x;
  if (b >= B) return;
  const int F = g.Lx;
  int *off = sm_pp;
  int *cs = sm_pp + F * M;
  __shared__ int s_nc;
  const uint8_t *cb = pc + b * (int64_t)F * M;
  for (int e = threadIdx.x; e < F * M; e += blockDim.x) {
    const int t = e / M, m = e - t * M, py = m / g.P, px = m - py * g.P;
    off[e] = cb[e] ? level_index(g, l, 0, t, py, px) : -1;
  }
  if (threadIdx.x < 32) {
    const int nc = list_candidates_warp(b, omega_up, ldo_up, keff_up, child_off, child_idx, cap, cs, threadIdx.x);
    if (threadIdx.x == 0) s_nc = nc;
  }
  __syncthreads();
  const int nc = s_nc;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int c = warp; c < nc; c += nw) {
    const float *d = D + (int64_t)cs[c] * N;
    float *row = Ac + (b * cap + c) * (int64_t)M;
    float sq = 0.f;
    for (int m = lane; m < M; m += 32) {
      float dv[8];
      float v = 0.f;
      for (int t0 = 0; t0 < F; t0 += 8) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int o = t0 + u < F ? off[(t0 + u) * M + m] : -1;
          dv[u] = o >= 0 ? __ldg(d + o) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (t0 + u < F && off[(t0 + u) * M + m] >= 0) v += dv[u];
      }
      row[m] = v;
      sq = fmaf(v, v, sq);
    }
    for (int o = 16; o; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
    if (lane == 0) {
      const float nrm = sqrtf(sq);
      invc[b * cap + c] = nrm > 0.f ? 1.f / nrm : -1.f;
    }
  }
}

// Per-pixel coded exposure in time-bin form.  At level l the frames t of one
// time bin k (t / fx = k, fx the level's frame factor) all send pixel m to the
// same level element k S + s(m) (S = the level's pixels per frame, s(m) the
// element of m's pixel), so a row of the effective dictionary is
//   a_i[m] = sum_k c_k(m) d_i[k S + s(m)],   k = 0 .. F / fx - 1 in order,
// with c_k(m) the number of frames of bin k whose code at m is 1: the operator
// Phi_p U_l of the patch applied to d_i, the frame sums of one bin taken as
// one multiply-add.  A lane keeps the element offsets and counts of its pixels
// m = lane + 32 j in registers for the whole patch, so a row costs one load and
// one FMA per (pixel, bin) and no index arithmetic.  Bins past the level's
// count (the template rounds it up) and pixels past M get count 0 and a valid
// offset (s(m), or 0), so the loads need no guard.
template <int NB, int MPL>
struct PpBins {
  int off[MPL][NB];
  float c[MPL][NB];
};

template <int NB, int MPL>
__device__ __forceinline__ void pp_bins_setup(const GeomDev &g, int l, const uint8_t *__restrict__ cb, int M, int S,
                                              int nb, int lane, PpBins<NB, MPL> &t) {
  const int fx = g.f[l][1], sy = g.f[l][2], sx = g.f[l][3], Pxl = g.P / sx;
#pragma unroll
  for (int j = 0; j < MPL; ++j) {
    const int m = lane + 32 * j;
    const bool ok = m < M;
    const int py = ok ? m / g.P : 0, px = ok ? m - py * g.P : 0;
    const int sm = (py / sy) * Pxl + px / sx;
#pragma unroll
    for (int k = 0; k < NB; ++k) {
      int n = 0;
      if (ok && k < nb)
        for (int u = 0; u < fx; ++u) n += cb[(k * fx + u) * M + m] ? 1 : 0;
      t.off[j][k] = (k < nb ? k * S : 0) + sm;
      t.c[j][k] = (float)n;
    }
  }
}

// The lane's pixels of one row: v[j] = a[lane + 32 j].
template <int NB, int MPL>
__device__ __forceinline__ void pp_bins_eval(const float *__restrict__ d, const PpBins<NB, MPL> &t,
                                             float (&v)[MPL]) {
  float x[MPL][NB];
#pragma unroll
  for (int j = 0; j < MPL; ++j)
#pragma unroll
    for (int k = 0; k < NB; ++k) x[j][k] = __ldg(d + t.off[j][k]);
#pragma unroll
  for (int j = 0; j < MPL; ++j) {
    v[j] = 0.f;
#pragma unroll
    for (int k = 0; k < NB; ++k) v[j] = fmaf(t.c[j][k], x[j][k], v[j]);
  }
}

// Warp sums of eight values at once: lane l ends with the sum over all lanes of
// q[r], r = 4 (l >> 4 & 1) + 2 (l >> 3 & 1) + (l >> 2 & 1) -- three halving
// exchanges and two plain ones, nine shuffles for eight sums.
__device__ __forceinline__ float warp_sum8(const float (&q)[8], int lane) {
  const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
  float h4[4], h2[2];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const float send = b4 ? q[u] : q[u + 4], keep = b4 ? q[u + 4] : q[u];
    h4[u] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const float send = b3 ? h4[u] : h4[u + 2], keep = b3 ? h4[u + 2] : h4[u];
    h2[u] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  float h = (b2 ? h2[1] : h2[0]) + __shfl_xor_sync(0xffffffffu, b2 ? h2[0] : h2[1], 4);
  h += __shfl_xor_sync(0xffffffffu, h, 2);
  h += __shfl_xor_sync(0xffffffffu, h, 1);
  return h;
}

__device__ __forceinline__ int sum8_row(int lane) { return ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1); }

// The full per-patch effective dictionary of level l and its row norms in
// time-bin form: one warp per patch (eight patches per CTA), rows taken in
// groups of eight (r0 + u, u < 8), written, and their eight squared norms
// reduced together.  A warp per patch, not a CTA: the per-patch set-up (the
// bins of the lane's pixels) is done once and no barrier is needed.
template <int NB, int MPL>
__global__ void __launch_bounds__(256, 2)
pp_bins_rows_kernel(GeomDev g, const uint8_t *__restrict__ pc, int l, const float *__restrict__ D, int T, int N,
                    int S, int nb, float *__restrict__ A, float *__restrict__ nrm, unsigned int *mx, int64_t B) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t b = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
  if (b >= B) return;
  const int M = g.P * g.P;
  PpBins<NB, MPL> t;
  pp_bins_setup<NB, MPL>(g, l, pc + b * (int64_t)g.Lx * M, M, S, nb, lane, t);
  unsigned int wmax = 0u;
  float *Ab = A + b * (int64_t)T * M;
  for (int r0 = 0; r0 < T; r0 += 8) {
    float q[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int i = r0 + u;
      q[u] = 0.f;
      if (i < T) {
        float v[MPL];
        pp_bins_eval<NB, MPL>(D + (int64_t)i * N, t, v);
        float *row = Ab + (int64_t)i * M;
#pragma unroll
        for (int j = 0; j < MPL; ++j) {
          if (lane + 32 * j < M) row[lane + 32 * j] = v[j];
          q[u] = fmaf(v[j], v[j], q[u]);
        }
      }
    }
    const float tot = warp_sum8(q, lane);
    const int i = r0 + sum8_row(lane);
    if ((lane & 3) == 0 && i < T) {
      const float r = sqrtf(tot);
      nrm[b * T + i] = r;
      wmax = max(wmax, __float_as_uint(r));
    }
  }
  // the largest norm: one global atomic per patch
  wmax = __reduce_max_sync(0xffffffffu, wmax);
  if (lane == 0 && wmax) atomicMax(mx, wmax);
}

// Candidate rows of a restricted level in time-bin form (the candidate list
// and the outputs of pp_candidates_kernel, the row arithmetic and grouping of
// pp_bins_rows_kernel): one warp per patch, its candidate list in its own
// slice of shared memory.  GRAM: the rows also go to shared memory ([cap][M + 1]
// per warp) and the warp writes the patch's Gram block G[i][j] = <a_i, a_j>
// (i, j < |C|, FMA chain over m in order) to Gpp + b cap^2, each lane a 4 x 4
// tile of the upper triangle at a time, mirrored.
template <int NB, int MPL, bool GRAM>
__global__ void __launch_bounds__(256, 2)
pp_bins_candidates_kernel(GeomDev g, const uint8_t *__restrict__ pc, int l, const float *__restrict__ D, int N,
                          int M, int S, int nb, const int32_t *__restrict__ omega_up, int ldo_up,
                          const int8_t *__restrict__ keff_up, const int32_t *__restrict__ child_off,
                          const int32_t *__restrict__ child_idx, int cap, int64_t B, float *__restrict__ Ac,
                          float *__restrict__ invc, float *__restrict__ Gpp) {
  extern __shared__ int cs_all[];  // [warps][cap] candidate atoms | GRAM: [warps][cap][M + 1] rows
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwc = blockDim.x >> 5;
  const int64_t b = (int64_t)blockIdx.x * nwc + warp;
  if (b >= B) return;
  int *cs = cs_all + warp * cap;
  const int ldr = M + 1;
  float *Rs = reinterpret_cast<float *>(cs_all + nwc * cap) + (size_t)warp * cap * ldr;
  const int nc = list_candidates_warp(b, omega_up, ldo_up, keff_up, child_off, child_idx, cap, cs, lane);
  PpBins<NB, MPL> t;
  pp_bins_setup<NB, MPL>(g, l, pc + b * (int64_t)g.Lx * M, M, S, nb, lane, t);
  __syncwarp();
  float *Ab = Ac + b * (int64_t)cap * M;
  for (int r0 = 0; r0 < nc; r0 += 8) {
    float q[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int c = r0 + u;
      q[u] = 0.f;
      if (c < nc) {
        float v[MPL];
        pp_bins_eval<NB, MPL>(D + (int64_t)cs[c] * N, t, v);
        float *row = Ab + (int64_t)c * M;
#pragma unroll
        for (int j = 0; j < MPL; ++j) {
          if (lane + 32 * j < M) {
            row[lane + 32 * j] = v[j];
            if (GRAM) Rs[c * ldr + lane + 32 * j] = v[j];
          }
          q[u] = fmaf(v[j], v[j], q[u]);
        }
      }
    }
    const float tot = warp_sum8(q, lane);
    const int c = r0 + sum8_row(lane);
    if ((lane & 3) == 0 && c < nc) {
      const float r = sqrtf(tot);
      invc[b * cap + c] = r > 0.f ? 1.f / r : -1.f;
    }
  }
  if (GRAM) {
    __syncwarp();
    float *Gb = Gpp + b * (int64_t)cap * cap;
    const int nt = (nc + 3) >> 2, ntile = nt * (nt + 1) / 2;
    for (int tix = lane; tix < ntile; tix += 32) {
      int ti = 0, rem = tix;  // tile (ti, tj), ti <= tj, row-major over the upper triangle
      while (rem >= nt - ti) {
        rem -= nt - ti;
        ++ti;
      }
      const int tj = ti + rem;
      float acc[4][4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = 0.f;
      int ri[4], rj[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        ri[u] = min(4 * ti + u, nc - 1) * ldr;  // rows past |C| repeat the last one (not written)
        rj[u] = min(4 * tj + u, nc - 1) * ldr;
      }
      for (int m = 0; m < M; ++m) {
        float x[4], y[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          x[u] = Rs[ri[u] + m];
          y[u] = Rs[rj[u] + m];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(x[u], y[v], acc[u][v]);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const int i = 4 * ti + u, j = 4 * tj + v;
          if (i < nc && j < nc && i <= j) {
            Gb[i * cap + j] = acc[u][v];
            Gb[j * cap + i] = acc[u][v];
          }
        }
    }
  }
}

// Dense Phi (the same for every patch): a_i = Phi U_l d_i, one thread per
// (atom i, measurement m), the level-0 patch index n = (plane, py, px) mapped
// to its level-l element by U_l (nearest replication).
__global__ void effective_dict_dense_kernel(GeomDev g, const float *__restrict__ phi, int l,
                                            const float *__restrict__ D, int T, int N, float *__restrict__ A,
                                            int M) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)T * M) return;
  const int i = (int)(e / M), m = (int)(e - (int64_t)i * M);
  const int PP = g.P * g.P, N0 = g.Ly * g.Lx * PP;
  const float *d = D + (int64_t)i * N;
  const float *row = phi + (int64_t)m * N0;
  float v = 0.f;
  for (int n = 0; n < N0; ++n) {
    const int pl = n / PP, r = n - pl * PP, py = r / g.P, px = r - py * g.P;
    v = fmaf(__ldg(row + n), __ldg(d + level_index(g, l, pl / g.Lx, pl % g.Lx, py, px)), v);
  }
  A[e] = v;
}

// Row norms of a [rows][M] matrix: out = ||row|| (first pass), running max
// of the norms in *mx (float bits, non-negative, compared as integers).
__global__ void row_norms_kernel(const float *__restrict__ A, int64_t rows, int M, float *__restrict__ out,
                                 unsigned int *mx) {
  const int lane = threadIdx.x & 31;
  const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (r >= rows) return;
  float s = 0.f;
  for (int m = lane; m < M; m += 32) { const float a = A[r * M + m]; s = fmaf(a, a, s); }
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) {
    const float nrm = sqrtf(s);
    out[r] = nrm;
    atomicMax(mx, __float_as_uint(nrm));
  }
}

// Second pass: 1/norm, or -1 for rows with norm <= 1e-12 of the largest.
__global__ void inv_norms_kernel(float *__restrict__ v, int64_t rows, const unsigned int *mx) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= rows) return;
  const float thr = 1e-12f * __uint_as_float(*mx);
  const float nrm = v[r];
  v[r] = (nrm > thr && nrm > 0.f) ? 1.f / nrm : -1.f;
}

// BF16 copy of dictionary rows (not normalised), zero padded to Np.
__global__ void bf16_rows_kernel(const float *__restrict__ D, int T, int N, int Np, __nv_bfloat16 *__restrict__ out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)T * Np) return;
  const int i = (int)(e / Np), n = (int)(e - (int64_t)i * Np);
  out[e] = __float2bfloat16_rn(n < N ? D[(int64_t)i * N + n] : 0.f);
}

// Lifted residual of per-pixel coded exposure at level l: z = U_l^T Phi_p^T r,
// z[(t_l, py_l, px_l)] = sum over the factor block of pc_p[t][py][px] r[py][px].
// One thread per (patch, level element); FP32 (optional) and a BF16 copy
// (optional) padded to Np.
__global__ void lift_kernel(GeomDev g, const uint8_t *__restrict__ pc, int l, const float *__restrict__ R,
                            int64_t B, float *__restrict__ Z, __nv_bfloat16 *__restrict__ Zbf, int Np) {
  const int fx = g.f[l][1], sy = g.f[l][2], sx = g.f[l][3];
  const int Lxl = g.Lx / fx, Pyl = g.P / sy, Pxl = g.P / sx;
  const int Nl = Lxl * Pyl * Pxl, PP = g.P * g.P;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= B * Np) return;
  const int64_t b = e / Np;
  const int n = (int)(e - b * Np);
  float acc = 0.f;
  if (n < Nl) {
    const int pxl = n % Pxl, pyl = (n / Pxl) % Pyl, tl = n / (Pxl * Pyl);
    const float *r = R + b * PP;
    const uint8_t *c = pc + b * (int64_t)g.Lx * PP;
    for (int dt = 0; dt < fx; ++dt)
      for (int dy = 0; dy < sy; ++dy)
        for (int dx = 0; dx < sx; ++dx) {
          const int t = tl * fx + dt, py = pyl * sy + dy, px = pxl * sx + dx;
          if (c[t * PP + py * g.P + px]) acc += r[py * g.P + px];
        }
    if (Z) Z[b * Nl + n] = acc;
  }
  if (Zbf) Zbf[e] = __float2bfloat16_rn(acc);
}

// Column norms of A; 1/||a_i|| (or -1 for columns with ||a_i|| <= 1e-12 max_j ||a_j||,
// which are never chosen) and the BF16 copy of a_i/||a_i|| padded to Mp.
// One CTA, run once per dictionary.
__global__ void norms_kernel(const float *__restrict__ A, int T, int M, int Mp, float *inv_norm,
                             __nv_bfloat16 *Abf) {
  __shared__ float red[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  float mx = 0.f;
  for (int i = warp; i < T; i += nw) {
    float s = 0.f;
    for (int m = lane; m < M; m += 32) { const float a = A[(int64_t)i * M + m]; s = fmaf(a, a, s); }
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    const float nrm = sqrtf(s);
    if (lane == 0) inv_norm[i] = nrm;
    mx = fmaxf(mx, nrm);
  }
  if (lane == 0) red[warp] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    float v = 0.f;
    for (int w = 0; w < nw; ++w) v = fmaxf(v, red[w]);
    red[0] = v;
  }
  __syncthreads();
  const float thr = 1e-12f * red[0];
  for (int i = warp; i < T; i += nw) {
    const float nrm = inv_norm[i];
    __syncwarp();
    const bool ok = nrm > thr && nrm > 0.f;
    const float inv = ok ? 1.f / nrm : 0.f;
    if (Abf)
      for (int m = lane; m < Mp; m += 32)
        Abf[(int64_t)i * Mp + m] = __float2bfloat16_rn(m < M ? A[(int64_t)i * M + m] * inv : 0.f);
    if (lane == 0) inv_norm[i] = ok ? inv : -1.f;
  }
}

// Synthesis x_hat_p = D0 alpha_p (Sec. IV), patch-major Xh[b][n]: a warp per
// patch, lanes over the elements n (coalesced rows of D0 and of Xh), the
// patch's atoms eight at a time with their row pointers and coefficients in
// registers; v = fma(alpha_j, D0[a_j][n], v) in j order.
__global__ void synth_kernel(const float *__restrict__ D0, int N0, const int32_t *__restrict__ support,
                             const float *__restrict__ coef, const int8_t *__restrict__ k_eff, int Kmax,
                             int64_t B, float *__restrict__ Xh) {
  const int lane = threadIdx.x & 31;
  const int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (b >= B) return;
  int ke = k_eff[b];
  ke = ke < Kmax ? ke : Kmax;
  float *xb = Xh + b * N0;
  for (int j0 = 0; j0 == 0 || j0 < ke; j0 += 8) {
    const int cnt = ke - j0 < 8 ? ke - j0 : 8;
    const float *rp[8];
    float cj[8];
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) {
      rp[jj] = D0 + (int64_t)(jj < cnt ? __ldg(support + b * Kmax + j0 + jj) : 0) * N0;
      cj[jj] = jj < cnt ? __ldg(coef + b * Kmax + j0 + jj) : 0.f;
    }
    // two elements per pass: 16 loads in flight per lane
    for (int n = lane; n < N0; n += 64) {
      const bool two = n + 32 < N0;
      float dv[8], dw[8];
#pragma unroll
      for (int jj = 0; jj < 8; ++jj) {
        dv[jj] = jj < cnt ? __ldg(rp[jj] + n) : 0.f;
        dw[jj] = (two && jj < cnt) ? __ldg(rp[jj] + n + 32) : 0.f;
      }
      float v = j0 ? xb[n] : 0.f, u = (two && j0) ? xb[n + 32] : 0.f;
#pragma unroll
      for (int jj = 0; jj < 8; ++jj)
        if (jj < cnt) {
          v = fmaf(cj[jj], dv[jj], v);
          u = fmaf(cj[jj], dw[jj], u);
        }
      xb[n] = v;
      if (two) xb[n + 32] = u;
    }
  }
}

// Overlap-add: one thread per image pixel (plane, y, x), mean over the covering
// patches of x_hat_p at that pixel, summed in patch raster order (deterministic).
__global__ void gather_kernel(GeomDev g, const float *__restrict__ Xh, int N0,
                              const int32_t *__restrict__ cover_y, const int32_t *__restrict__ cover_x,
                              float *__restrict__ img) {
  const int planes = g.Ly * g.Lx;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)planes * g.H * g.W) return;
  const int x = (int)(e % g.W);
  const int y = (int)((e / g.W) % g.H);
  const int pl = (int)(e / ((int64_t)g.W * g.H));
  const int y0 = cover_y[2 * y], y1 = cover_y[2 * y + 1];
  const int x0 = cover_x[2 * x], x1 = cover_x[2 * x + 1];
  const int np = (y1 - y0 + 1) * (x1 - x0 + 1);
  // covering patches in raster order, eight loads in flight, summed in order
  float acc = 0.f;
  int iy = y0, ix = x0;
  for (int p0 = 0; p0 < np; p0 += 8) {
    float v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      v[u] = 0.f;
      if (p0 + u < np) {
        const int py = y - origin(iy, g.stride, g.H, g.P), px = x - origin(ix, g.stride, g.W, g.P);
        v[u] = __ldg(Xh + ((int64_t)iy * g.nx + ix) * N0 + (pl * g.P + py) * g.P + px);
        if (++ix > x1) { ix = x0; ++iy; }
      }
    }
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (p0 + u < np) acc += v[u];
  }
  img[e] = np ? acc / (float)np : 0.f;
}

// Fused synthesis + overlap-add over an output tile of TY x TX pixels (all
// planes).  Phase 0 stages the codes (support, coefficients) of every patch q
// covering the tile and the (py, px) of every patch element n; phase 1 (a warp
// per covering patch) synthesizes x_hat_q = D0 alpha_q into shared memory
// (rows of ldp floats, ldp = stride mod 32 so that neighbouring pixels, which
// read neighbouring patches, hit distinct banks), only at the elements inside
// the tile; phase 2 averages, per pixel, over its covering patches in patch
// raster order.  The arithmetic and its order are those of synth_kernel +
// gather_kernel, so both paths give identical images.
__global__ void __launch_bounds__(512, 2)
agg_tile_kernel(GeomDev g, const float *__restrict__ D0, int N0, const int32_t *__restrict__ support,
                const float *__restrict__ coef, const int8_t *__restrict__ k_eff, int Kmax,
                const int32_t *__restrict__ cover_y, const int32_t *__restrict__ cover_x, int TY, int TX, int ldp,
                int nq_max, float *__restrict__ img) {
  extern __shared__ float xs[];  // [nq_max][ldp] patches | [nq_max][Kmax] atoms | [nq_max][Kmax] coefs |
                                 // [nq_max] k_eff | [N0] (py, px)
  int *s_sup = reinterpret_cast<int *>(xs + (size_t)nq_max * ldp);
  float *s_coef = reinterpret_cast<float *>(s_sup + nq_max * Kmax);
  int *s_keff = reinterpret_cast<int *>(s_coef + nq_max * Kmax);
  int *s_yx = s_keff + nq_max;
  const int ty0 = blockIdx.y * TY, tx0 = blockIdx.x * TX;
  const int ty1 = min(ty0 + TY, g.H), tx1 = min(tx0 + TX, g.W);
  const int iy0 = cover_y[2 * ty0], iy1 = cover_y[2 * (ty1 - 1) + 1];
  const int ix0 = cover_x[2 * tx0], ix1 = cover_x[2 * (tx1 - 1) + 1];
  const int nxc = ix1 - ix0 + 1, nq = (iy1 - iy0 + 1) * nxc;
  const int PP = g.P * g.P;
  for (int e = threadIdx.x; e < nq * Kmax; e += blockDim.x) {
    const int q = e / Kmax, j = e - q * Kmax;
    const int64_t b = (int64_t)(iy0 + q / nxc) * g.nx + (ix0 + q % nxc);
    const int ke = k_eff[b];
    if (j == 0) s_keff[q] = ke < Kmax ? ke : Kmax;
    s_sup[e] = j < ke ? support[b * Kmax + j] : -1;
    s_coef[e] = j < ke ? coef[b * Kmax + j] : 0.f;
  }
  for (int n = threadIdx.x; n < N0; n += blockDim.x) {
    const int r = n % PP;
    s_yx[n] = ((r / g.P) << 16) | (r % g.P);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  for (int q = warp; q < nq; q += nwarps) {
    // the part of patch q inside the tile, in patch coordinates
    const int oy = origin(iy0 + q / nxc, g.stride, g.H, g.P), ox = origin(ix0 + q % nxc, g.stride, g.W, g.P);
    const int py0 = ty0 - oy, py1 = ty1 - oy, px0 = tx0 - ox, px1 = tx1 - ox;
    const int ke = s_keff[q];
    float *xq = xs + q * ldp;
    // atoms j0 .. j0 + 7 at a time: their rows and coefficients in registers,
    // x_hat accumulated in place in j order (the order of synth_kernel)
    for (int j0 = 0; j0 == 0 || j0 < ke; j0 += 8) {
      const int cnt = ke - j0 < 8 ? ke - j0 : 8;
      const float *rp[8];
      float cj[8];
#pragma unroll
      for (int jj = 0; jj < 8; ++jj) {
        const int j = jj < cnt ? j0 + jj : j0;
        rp[jj] = D0 + (int64_t)(jj < cnt ? s_sup[q * Kmax + j] : 0) * N0;
        cj[jj] = jj < cnt ? s_coef[q * Kmax + j] : 0.f;
      }
      for (int n = lane; n < N0; n += 32) {
        const int yx = s_yx[n], py = yx >> 16, px = yx & 0xffff;
        if (py < py0 || py >= py1 || px < px0 || px >= px1) continue;  // outside the tile: never read
        float dv[8];
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) dv[jj] = jj < cnt ? __ldg(rp[jj] + n) : 0.f;
        float v = j0 ? xq[n] : 0.f;
#pragma unroll
        for (int jj = 0; jj < 8; ++jj)
          if (jj < cnt) v = fmaf(cj[jj], dv[jj], v);
        xq[n] = v;
      }
    }
  }
  __syncthreads();
  const int planes = g.Ly * g.Lx, th = ty1 - ty0, tw = tx1 - tx0;
  for (int e = threadIdx.x; e < planes * th * tw; e += blockDim.x) {
    const int x = tx0 + e % tw, r = e / tw;
    const int y = ty0 + r % th, pl = r / th;
    const int y0 = cover_y[2 * y], y1 = cover_y[2 * y + 1];
    const int x0 = cover_x[2 * x], x1 = cover_x[2 * x + 1];
    float acc = 0.f;
    int cnt = 0;
    for (int iy = y0; iy <= y1; ++iy) {
      const int py = y - origin(iy, g.stride, g.H, g.P);
      const float *row = xs + (iy - iy0) * nxc * ldp;
      for (int ix = x0; ix <= x1; ++ix) {
        const int px = x - origin(ix, g.stride, g.W, g.P);
        acc += row[(ix - ix0) * ldp + (pl * g.P + py) * g.P + px];
        ++cnt;
      }
    }
    img[((int64_t)pl * g.H + y) * g.W + x] = cnt ? acc / (float)cnt : 0.f;
  }
}

inline unsigned blocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

void launch_extract(const GeomDev &g, int sense_kind, int shots, const float *meas, float *Y,
                    int64_t B, int M, cudaStream_t s) {
  (void)sense_kind; (void)shots;
  if (B * M == 0) return;
  if (g.P % 4 == 0 && M % 4 == 0 && M <= 1024 && B < ((int64_t)1 << 31) - 256) {
    const int M4 = M / 4, per = M4 >= 256 ? 1 : 256 / M4;
    extract_kernel<<<(unsigned)((B + per - 1) / per), dim3(M4, per), 0, s>>>(g, meas, Y, B, M);
  }
  else
    extract1_kernel<<<blocks(B * M, 256), 256, 0, s>>>(g, meas, Y, B, M);
}

void launch_downsample(const GeomDev &g, int level, const float *Y0, float *Yl, int64_t B,
                       cudaStream_t s) {
  const int Nl = (g.Ly / g.f[level][0]) * (g.Lx / g.f[level][1]) * (g.P / g.f[level][2]) *
                 (g.P / g.f[level][3]);
  if (B * Nl == 0) return;
  downsample_kernel<<<blocks(B * Nl, 256), 256, 0, s>>>(g, level, Y0, Yl, B);
}

void launch_effective_dict(const GeomDev &g, int sense_kind, int shots, const uint8_t *codes,
                           int level, int phase, const float *D, int T, int N, float *A, int M,
                           cudaStream_t s) {
  if ((int64_t)T * M == 0) return;
  effective_dict_kernel<<<blocks((int64_t)T * M, 256), 256, 0, s>>>(g, sense_kind, shots, codes, level,
                                                                     phase, D, T, N, A, M);
}

void launch_norms(const float *A, int T, int M, int Mp, float *inv_norm, __nv_bfloat16 *Abf,
                  cudaStream_t s) {
  if (T == 0) return;
  norms_kernel<<<1, 1024, 0, s>>>(A, T, M, Mp, inv_norm, Abf);
}

// Copy of n floats (16-byte aligned source and destination), e.g. from a
// page-locked host buffer through its device mapping: coalesced 16-byte loads,
// many in flight, one pass over the source.
__global__ void copy4_kernel(const float4 *__restrict__ src, float4 *__restrict__ dst, int64_t n4) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

void launch_copy_floats(const float *src, float *dst, int64_t n, cudaStream_t s) {
  const int64_t n4 = n / 4;
  if (n4 > 0) {
    const int64_t want = (n4 + 255) / 256;
    copy4_kernel<<<(unsigned)(want < 1216 ? want : 1216), 256, 0, s>>>(reinterpret_cast<const float4 *>(src),
                                                                      reinterpret_cast<float4 *>(dst), n4);
  }
  if (n % 4) cudaMemcpyAsync(dst + 4 * n4, src + 4 * n4, (n % 4) * sizeof(float), cudaMemcpyDefault, s);
}

void launch_synth(const GeomDev &g, const float *D0, int N0, const int32_t *support, const float *coef,
                  const int8_t *k_eff, int Kmax, float *Xh, cudaStream_t s) {
  const int64_t B = (int64_t)g.nx * g.ny;
  if (B * N0) synth_kernel<<<blocks(B * 32, 256), 256, 0, s>>>(D0, N0, support, coef, k_eff, Kmax, B, Xh);
}

void launch_gather(const GeomDev &g, const float *Xh, int N0, const int32_t *cover_y, const int32_t *cover_x,
                   float *img, cudaStream_t s) {
  const int64_t n = (int64_t)g.Ly * g.Lx * g.H * g.W;
  if (n) gather_kernel<<<blocks(n, 256), 256, 0, s>>>(g, Xh, N0, cover_y, cover_x, img);
}

void launch_aggregate(const GeomDev &g, const float *D0, int N0, const int32_t *support, const float *coef,
                      const int8_t *k_eff, int Kmax, const int32_t *cover_y, const int32_t *cover_x, float *Xh,
                      float *img, cudaStream_t s) {
  if ((int64_t)g.Ly * g.Lx * g.H * g.W == 0) return;
  launch_synth(g, D0, N0, support, coef, k_eff, Kmax, Xh, s);
  launch_gather(g, Xh, N0, cover_y, cover_x, img, s);
}

// Largest number of patches covering one tile of T pixels along an axis of
// extent E (patch origins min(i * stride, E - P)), over all tiles.
static int max_cover(int E, int P, int stride, int n, int T) {
  // first / last patch covering pixel y (origins are nondecreasing)
  auto org = [&](int i) { return std::min(i * stride, E - P); };
  int best = 0;
  int lo = 0;
  for (int t0 = 0; t0 < E; t0 += T) {
    const int t1 = std::min(t0 + T, E) - 1;
    while (lo < n && org(lo) + P <= t0) ++lo;
    int hi = lo;
    while (hi + 1 < n && org(hi + 1) <= t1) ++hi;
    best = std::max(best, hi - lo + 1);
  }
  return best;
}

struct AggTile {
  int TY = 0, TX = 0, ldp = 0, nq = 0;
  size_t smem = 0;
};

static bool agg_tile_plan(const GeomDev &g, int N0, int Kmax, AggTile &p) {
  constexpr size_t kSmemCap = 113 * 1024;  // two CTAs per SM
  static const int tiles[][2] = {{16, 32}, {8, 32}, {4, 32}, {8, 16}, {4, 16}, {4, 8}, {2, 8}};
  p.ldp = N0 + (((g.stride - N0) % 32) + 32) % 32;
  if (g.stride > g.P) return false;  // rows between patches are uncovered: no contiguous covering range
  for (const auto &t : tiles) {
    p.TY = t[0];
    p.TX = t[1];
    p.nq = max_cover(g.H, g.P, g.stride, g.ny, p.TY) * max_cover(g.W, g.P, g.stride, g.nx, p.TX);
    p.smem = sizeof(float) * ((size_t)p.nq * (p.ldp + 2 * Kmax + 1) + N0);
    if (p.smem <= kSmemCap) return true;
  }
  return false;
}

bool aggregate_tiled_fits(const GeomDev &g, int N0, int Kmax) {
  AggTile p;
  return agg_tile_plan(g, N0, Kmax, p);
}

bool launch_aggregate_tiled(const GeomDev &g, const float *D0, int N0, const int32_t *support, const float *coef,
                            const int8_t *k_eff, int Kmax, const int32_t *cover_y, const int32_t *cover_x, float *img,
                            cudaStream_t s) {
  if ((int64_t)g.Ly * g.Lx * g.H * g.W == 0) return true;
  AggTile p;
  if (!agg_tile_plan(g, N0, Kmax, p)) return false;
  if (p.smem > 48 * 1024)
    cudaFuncSetAttribute(agg_tile_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem);
  const dim3 grid((unsigned)((g.W + p.TX - 1) / p.TX), (unsigned)((g.H + p.TY - 1) / p.TY));
  agg_tile_kernel<<<grid, 512, p.smem, s>>>(g, D0, N0, support, coef, k_eff, Kmax, cover_y, cover_x, p.TY, p.TX,
                                             p.ldp, p.nq, img);
  return true;
}

void launch_effective_dict_dense(const GeomDev &g, const float *phi, int level, const float *D, int T, int N,
                                 float *A, int M, cudaStream_t s) {
  if ((int64_t)T * M == 0) return;
  effective_dict_dense_kernel<<<blocks((int64_t)T * M, 256), 256, 0, s>>>(g, phi, level, D, T, N, A, M);
}

void launch_patch_codes(const GeomDev &g, const uint8_t *codes, int64_t B, uint8_t *pc, cudaStream_t s) {
  const int64_t n = B * g.Lx * (int64_t)(g.P * g.P);
  if (n == 0) return;
  patch_codes_kernel<<<blocks(n, 256), 256, 0, s>>>(g, codes, B, pc);
}

// Time-bin form of a per-pixel level: bins per pixel, level pixels per frame,
// and the template instance (bins rounded up to 1, 2, 4, 8 or 16; pixels per
// lane 1, 2 or 4), or false when the shape needs the general kernels.
struct PpShape {
  int nb, S, NB, MPL;
};

bool pp_shape(const GeomDev &g, int level, int M, PpShape &p) {
  p.nb = g.Lx / g.f[level][1];
  p.S = (g.P / g.f[level][2]) * (g.P / g.f[level][3]);
  p.NB = p.nb <= 1 ? 1 : p.nb <= 2 ? 2 : p.nb <= 4 ? 4 : p.nb <= 8 ? 8 : p.nb <= 16 ? 16 : 0;
  p.MPL = M <= 32 ? 1 : M <= 64 ? 2 : M <= 128 ? 4 : 0;
  return p.NB && p.MPL && g.Ly == 1;
}

template <int NB, int MPL>
void launch_pp_bins_rows(const GeomDev &g, const uint8_t *pc, int level, const float *D, int T, int N,
                         const PpShape &p, float *A, float *nrm, unsigned int *mx, int64_t B, cudaStream_t s) {
  pp_bins_rows_kernel<NB, MPL><<<(unsigned)((B + 7) / 8), 256, 0, s>>>(g, pc, level, D, T, N, p.S, p.nb, A, nrm,
                                                                        mx, B);
}

template <int NB>
void launch_pp_bins_rows_m(const GeomDev &g, const uint8_t *pc, int level, const float *D, int T, int N,
                           const PpShape &p, float *A, float *nrm, unsigned int *mx, int64_t B, cudaStream_t s) {
  if (p.MPL == 1) launch_pp_bins_rows<NB, 1>(g, pc, level, D, T, N, p, A, nrm, mx, B, s);
  else if (p.MPL == 2) launch_pp_bins_rows<NB, 2>(g, pc, level, D, T, N, p, A, nrm, mx, B, s);
  else launch_pp_bins_rows<NB, 4>(g, pc, level, D, T, N, p, A, nrm, mx, B, s);
}

void launch_effective_dict_pp_norms(const GeomDev &g, const uint8_t *pc, int level, const float *D, int T, int N,
                                    float *A, float *inv, unsigned int *scratch, int64_t B, cudaStream_t s) {
  if (B * T == 0) return;
  cudaMemsetAsync(scratch, 0, sizeof(unsigned int), s);
  PpShape p;
  if (pp_shape(g, level, g.P * g.P, p)) {
    switch (p.NB) {
      case 1: launch_pp_bins_rows_m<1>(g, pc, level, D, T, N, p, A, inv, scratch, B, s); break;
      case 2: launch_pp_bins_rows_m<2>(g, pc, level, D, T, N, p, A, inv, scratch, B, s); break;
      case 4: launch_pp_bins_rows_m<4>(g, pc, level, D, T, N, p, A, inv, scratch, B, s); break;
      case 8: launch_pp_bins_rows_m<8>(g, pc, level, D, T, N, p, A, inv, scratch, B, s); break;
      default: launch_pp_bins_rows_m<16>(g, pc, level, D, T, N, p, A, inv, scratch, B, s); break;
    }
  } else {
    const size_t sm = sizeof(int) * (size_t)g.Lx * g.P * g.P;
    if (sm > 48 * 1024)
      cudaFuncSetAttribute(effective_dict_pp_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    effective_dict_pp_rows_kernel<<<(unsigned)B, 256, sm, s>>>(g, pc, level, D, T, N, A, inv, scratch, B);
  }
  inv_norms_kernel<<<blocks(B * T, 256), 256, 0, s>>>(inv, B * T, scratch);
}

// Shared memory of one warp of pp_bins_candidates_kernel: its candidate list
// and, with the Gram block, its rows.
size_t pp_cand_warp_bytes(int cap, int M, bool gram) {
  return sizeof(int) * (size_t)cap + (gram ? sizeof(float) * (size_t)cap * (M + 1) : 0);
}
constexpr size_t kPpCandSmem = 200 * 1024;  // shared memory of one CTA at most

template <int NB, int MPL>
void launch_pp_bins_cand(const GeomDev &g, const uint8_t *pc, int level, const float *D, int N, int M,
                         const PpShape &p, const int32_t *omega_up, int ldo_up, const int8_t *keff_up,
                         const int32_t *child_off, const int32_t *child_idx, int cap, int64_t B, float *Ac,
                         float *invc, cudaStream_t s, float *Gpp) {
  const size_t per = pp_cand_warp_bytes(cap, M, Gpp != nullptr);
  const int nw = (int)std::max<size_t>(1, std::min<size_t>(8, kPpCandSmem / per));  // warps (patches) per CTA
  const size_t sm = per * nw;
  auto kern = Gpp ? pp_bins_candidates_kernel<NB, MPL, true> : pp_bins_candidates_kernel<NB, MPL, false>;
  if (sm > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  kern<<<(unsigned)((B + nw - 1) / nw), 32 * nw, sm, s>>>(g, pc, level, D, N, M, p.S, p.nb, omega_up, ldo_up,
                                                          keff_up, child_off, child_idx, cap, B, Ac, invc, Gpp);
}

template <int NB>
void launch_pp_bins_cand_m(const GeomDev &g, const uint8_t *pc, int level, const float *D, int N, int M,
                           const PpShape &p, const int32_t *omega_up, int ldo_up, const int8_t *keff_up,
                           const int32_t *child_off, const int32_t *child_idx, int cap, int64_t B, float *Ac,
                           float *invc, cudaStream_t s, float *Gpp) {
  if (p.MPL == 1)
    launch_pp_bins_cand<NB, 1>(g, pc, level, D, N, M, p, omega_up, ldo_up, keff_up, child_off, child_idx, cap, B, Ac,
                               invc, s, Gpp);
  else if (p.MPL == 2)
    launch_pp_bins_cand<NB, 2>(g, pc, level, D, N, M, p, omega_up, ldo_up, keff_up, child_off, child_idx, cap, B, Ac,
                               invc, s, Gpp);
  else
    launch_pp_bins_cand<NB, 4>(g, pc, level, D, N, M, p, omega_up, ldo_up, keff_up, child_off, child_idx, cap, B, Ac,
                               invc, s, Gpp);
}

bool launch_pp_candidates(const GeomDev &g, const uint8_t *pc, int level, const float *D, int N, int M,
                          const int32_t *omega_up, int ldo_up, const int8_t *keff_up, const int32_t *child_off,
                          const int32_t *child_idx, int cap, int64_t B, float *Ac, float *invc, cudaStream_t s,
                          float *Gpp) {
  PpShape p;
  const bool bins = pp_shape(g, level, M, p) && pp_cand_warp_bytes(cap, M, false) <= kPpCandSmem;
  if (Gpp && !(bins && pp_cand_warp_bytes(cap, M, true) <= kPpCandSmem)) Gpp = nullptr;  // no Gram form here
  if (B == 0) return Gpp != nullptr;
  if (bins) {
#define CSP_PP_CAND(nb_)                                                                                         \
  launch_pp_bins_cand_m<nb_>(g, pc, level, D, N, M, p, omega_up, ldo_up, keff_up, child_off, child_idx, cap, B, Ac, \
                             invc, s, Gpp)
    switch (p.NB) {
      case 1: CSP_PP_CAND(1); break;
      case 2: CSP_PP_CAND(2); break;
      case 4: CSP_PP_CAND(4); break;
      case 8: CSP_PP_CAND(8); break;
      default: CSP_PP_CAND(16); break;
    }
#undef CSP_PP_CAND
    return Gpp != nullptr;
  }
  const size_t sm = sizeof(int) * ((size_t)g.Lx * M + cap);
  if (sm > 48 * 1024) cudaFuncSetAttribute(pp_candidates_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  pp_candidates_kernel<<<(unsigned)B, 256, sm, s>>>(g, pc, level, D, N, M, omega_up, ldo_up, keff_up, child_off,
                                                    child_idx, cap, B, Ac, invc);
  return false;
}

void launch_inv_row_norms(const float *A, int64_t rows, int M, float *inv, unsigned int *scratch, cudaStream_t s) {
  if (rows == 0) return;
  cudaMemsetAsync(scratch, 0, sizeof(unsigned int), s);
  row_norms_kernel<<<blocks(rows * 32, 256), 256, 0, s>>>(A, rows, M, inv, scratch);
  inv_norms_kernel<<<blocks(rows, 256), 256, 0, s>>>(inv, rows, scratch);
}

void launch_bf16_rows(const float *D, int T, int N, int Np, __nv_bfloat16 *out, cudaStream_t s) {
  if ((int64_t)T * Np == 0) return;
  bf16_rows_kernel<<<blocks((int64_t)T * Np, 256), 256, 0, s>>>(D, T, N, Np, out);
}

void launch_lift(const GeomDev &g, const uint8_t *pc, int level, const float *R, int64_t B, float *Z,
                 __nv_bfloat16 *Zbf, int Np, cudaStream_t s) {
  if (B * Np == 0) return;
  lift_kernel<<<blocks(B * Np, 256), 256, 0, s>>>(g, pc, level, R, B, Z, Zbf, Np);
}

}  // namespace csp
