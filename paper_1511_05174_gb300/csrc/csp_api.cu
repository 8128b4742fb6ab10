// C ABI of the cross-scale OMP library: context, loaders, validation,
// workspace and the launch sequence of each entry point (declared in csp.h).
#include <algorithm>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "csp_internal.cuh"
#include "ksvd.cuh"

using namespace csp;

namespace {

thread_local std::string g_create_error;

csp_status fail(csp_ctx *ctx, csp_status st, const std::string &msg) {
  if (ctx) ctx->err = msg;
  else g_create_error = msg;
  return st;
}

#define CSP_CUDA(ctx, call)                                                              \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return fail(ctx, CSP_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

#define CSP_TRY(expr)             \
  do {                            \
    csp_status s_ = (expr);       \
    if (s_ != CSP_OK) return s_;  \
  } while (0)

// Makes the context's device current for the duration of a call.
struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

csp_status dev_alloc(csp_ctx *ctx, void **p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) return CSP_OK;
  if (ctx->budget && ctx->held + bytes > ctx->budget)
    return fail(ctx, CSP_ERR_OOM, "device memory budget exceeded (" + std::to_string(ctx->held + bytes) +
                                      " > " + std::to_string(ctx->budget) + " bytes)");
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(ctx, CSP_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  ctx->held += bytes;
  ctx->allocs.push_back({*p, bytes});
  return CSP_OK;
}

void dev_free(csp_ctx *ctx, void *p) {
  if (!p) return;
  for (size_t i = 0; i < ctx->allocs.size(); ++i)
    if (ctx->allocs[i].first == p) {
      cudaFree(p);
      ctx->held -= ctx->allocs[i].second;
      ctx->allocs.erase(ctx->allocs.begin() + (long)i);
      return;
    }
}

template <typename T>
csp_status dev_alloc_t(csp_ctx *ctx, T **p, size_t count) {
  void *v = nullptr;
  csp_status s = dev_alloc(ctx, &v, count * sizeof(T));
  *p = static_cast<T *>(v);
  return s;
}

// Grow-only workspace slot (allocations count against ctx's budget).
csp_status ws_get(csp_ctx *ctx, Workspace &W, int slot, size_t bytes, void **out) {
  if (W.owner) ctx = W.owner;
  if ((int)W.ws.size() <= slot) W.ws.resize(slot + 1);
  Buf &b = W.ws[slot];
  if (b.bytes < bytes) {
    dev_free(ctx, b.p);
    b.p = nullptr;
    b.bytes = 0;
    CSP_TRY(dev_alloc(ctx, &b.p, bytes));
    b.bytes = bytes;
    ++ctx->state_version;  // recorded graphs hold the old buffer
  }
  *out = b.p;
  return CSP_OK;
}
template <typename T>
csp_status ws_get_t(csp_ctx *ctx, Workspace &W, int slot, size_t count, T **out) {
  void *v = nullptr;
  csp_status s = ws_get(ctx, W, slot, count * sizeof(T) + 16, &v);
  *out = static_cast<T *>(v);
  return s;
}

const char *const kKernelNames[KK_COUNT] = {"extract", "downsample", "prepare", "omp_init", "proxy_fp32",
                                            "proxy_bf16", "omp_update", "restricted", "aggregate", "lift",
                                            "omp_fused", "ksvd_sort", "ksvd_sweep", "full_gram"};

cudaEvent_t pool_event(csp_ctx *ctx) {
  if (!ctx->ev_pool.empty()) {
    cudaEvent_t e = ctx->ev_pool.back();
    ctx->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); return nullptr; }
  return e;
}

// Counts one launch of `kind` and, while profiling, brackets it with events.
template <typename F>
void run(csp_ctx *ctx, int kind, cudaStream_t s, int64_t n, F &&launch) {
  if (n <= 0) return;
  cudaEvent_t a = nullptr, b = nullptr;
  if (ctx->prof) {
    a = pool_event(ctx);
    b = pool_event(ctx);
    if (a) cudaEventRecord(a, s);
  }
  launch();
  if (ctx->prof && a && b) {
    cudaEventRecord(b, s);
    ctx->pending.push_back({kind, a, b});
  }
  ctx->launches[kind] += 1;
}

csp_status drain_profile(csp_ctx *ctx) {
  for (auto &r : ctx->pending) {
    CSP_CUDA(ctx, cudaEventSynchronize(r.b));
    float ms = 0.f;
    CSP_CUDA(ctx, cudaEventElapsedTime(&ms, r.a, r.b));
    ctx->prof_ms[r.kind] += ms;
    ctx->ev_pool.push_back(r.a);
    ctx->ev_pool.push_back(r.b);
  }
  ctx->pending.clear();
  return CSP_OK;
}


enum Slot {
  WS_R, WS_RBF, WS_L, WS_Z, WS_FLAGS, WS_CAND,
  WS_LV_OMEGA, WS_LV_ALPHA = WS_LV_OMEGA + CSP_MAX_LEVELS, WS_LV_KEFF = WS_LV_ALPHA + CSP_MAX_LEVELS,
  WS_LV_Y = WS_LV_KEFF + CSP_MAX_LEVELS,
  WS_XH = WS_LV_Y + CSP_MAX_LEVELS,
  WS_SCRATCH, WS_LIFT, WS_LIFTBF, WS_PPC_A, WS_PPC_INV, WS_PPC_G, WS_PART, WS_KEYS, WS_P0, WS_ORDER, WS_ORDER_CNT, WS_QUEUE,
  WS_KS_R, WS_KS_RN2, WS_KS_XN2, WS_KS_TAKEN, WS_KS_HIST, WS_KS_OFF, WS_KS_SEG, WS_KS_ERR, WS_KS_STATS,
  WS_COUNT
};

int level_dim(const csp_geometry &g, int l) {
  return (g.plane_rows / g.factors[l][0]) * (g.plane_cols / g.factors[l][1]) * (g.P / g.factors[l][2]) *
         (g.P / g.factors[l][3]);
}

int count_1d(int E, int P, int s) {
  if (E < P) return 0;
  int n = (E - P) / s + 1;
  if ((E - P) % s) ++n;
  return n;
}

void free_level_derived(csp_ctx *ctx, LevelData &L) {
  dev_free(ctx, L.Dbf);
  L.Dbf = nullptr;
  L.per_patch = false;
  for (int p = 0; p < kMaxPhases; ++p) {
    if (L.A[p] && L.A[p] != L.D) dev_free(ctx, L.A[p]);
    dev_free(ctx, L.inv_norm[p]);
    dev_free(ctx, L.Abf[p]);
    dev_free(ctx, L.G[p]);
    L.A[p] = nullptr;
    L.inv_norm[p] = nullptr;
    L.Abf[p] = nullptr;
    L.G[p] = nullptr;
  }
  L.n_phase = 0;
}

// Per-patch data of the context's own grid (coded exposure).
void free_own_patches(csp_ctx *ctx) {
  for (int l = 0; l < CSP_MAX_LEVELS; ++l) {
    dev_free(ctx, ctx->pp_A[l]);
    dev_free(ctx, ctx->pp_inv[l]);
    ctx->pp_A[l] = ctx->pp_inv[l] = nullptr;
  }
}

void free_links(csp_ctx *ctx, LevelData &L) {
  dev_free(ctx, L.child_off);
  dev_free(ctx, L.child_idx);
  L.child_off = L.child_idx = nullptr;
  L.max_children = 0;
  L.links = false;
}

csp_status prepare(csp_ctx *ctx, cudaStream_t s) {
  if (ctx->prepared) return CSP_OK;
  if (!ctx->has_geom) return fail(ctx, CSP_ERR_NOT_READY, "geometry not set");
  if (!ctx->has_sensing) return fail(ctx, CSP_ERR_NOT_READY, "sensing operator not set");
  const int nl = ctx->geom.n_levels;
  for (int l = 0; l < nl; ++l) {
    LevelData &L = ctx->lv[l];
    if (!L.D) return fail(ctx, CSP_ERR_NOT_READY, "dictionary of level " + std::to_string(l) + " not loaded");
    free_level_derived(ctx, L);
    if (ctx->sense_kind == CSP_SENSE_CODED_EXPOSURE) {
      // per-patch Phi: one effective dictionary per patch, per-patch column norms,
      // and BF16 rows of D for the lifted tensor-core proxy
      L.M = ctx->M;
      L.Mp = (L.M + 63) / 64 * 64;
      L.Np = (L.N + 63) / 64 * 64;
      if (!omp_dims_supported(L.M))
        return fail(ctx, CSP_ERR_UNSUPPORTED, "problem dimension must be a multiple of 4, <= 256");
      CSP_TRY(dev_alloc_t(ctx, &L.Dbf, (size_t)L.T * L.Np));
      run(ctx, KK_PREP, s, L.T, [&] { launch_bf16_rows(L.D, L.T, L.N, L.Np, L.Dbf, s); });
      L.per_patch = true;
      L.n_phase = 1;
      continue;
    }
    const bool ident = ctx->sense_kind == CSP_SENSE_IDENTITY;
    L.M = ident ? L.N : ctx->M;
    L.Mp = (L.M + 63) / 64 * 64;
    if (!omp_dims_supported(L.M))
      return fail(ctx, CSP_ERR_UNSUPPORTED, "problem dimension " + std::to_string(L.M) +
                                                " of level " + std::to_string(l) + " must be a multiple of 4, <= 256");
    const int nph = ctx->sense_kind == CSP_SENSE_BAYER_RGGB ? 4 : 1;
    for (int p = 0; p < nph; ++p) {
      if (ident) {
        L.A[p] = L.D;
      } else {
        CSP_TRY(dev_alloc_t(ctx, &L.A[p], (size_t)L.T * L.M));
        run(ctx, KK_PREP, s, (int64_t)L.T * L.M, [&] {
          if (ctx->sense_kind == CSP_SENSE_DENSE)
            launch_effective_dict_dense(ctx->gd, ctx->phi, l, L.D, L.T, L.N, L.A[p], L.M, s);
          else
            launch_effective_dict(ctx->gd, ctx->sense_kind, ctx->shots, ctx->codes, l, p, L.D, L.T, L.N, L.A[p],
                                  L.M, s);
        });
      }
      CSP_TRY(dev_alloc_t(ctx, &L.inv_norm[p], (size_t)L.T));
      CSP_TRY(dev_alloc_t(ctx, &L.Abf[p], (size_t)L.T * L.Mp));
      run(ctx, KK_PREP, s, L.T, [&] { launch_norms(L.A[p], L.T, L.M, L.Mp, L.inv_norm[p], L.Abf[p], s); });
      // Gram matrix of the effective dictionary (projection step's Gram column),
      // kept when it is at most 256 MiB and fits the memory budget
      const size_t gbytes = (size_t)L.T * L.T * sizeof(float);
      if (gbytes <= (size_t(256) << 20) && (!ctx->budget || ctx->held + gbytes <= ctx->budget)) {
        CSP_TRY(dev_alloc_t(ctx, &L.G[p], (size_t)L.T * L.T));
        run(ctx, KK_PREP, s, L.T, [&] { launch_gram(L.A[p], L.T, L.M, L.G[p], s); });
      }
    }
    L.n_phase = nph;
  }
  for (int l = 0; l + 1 < nl; ++l)
    if (ctx->lv[l].links && ctx->lv[l].T == 0)
      return fail(ctx, CSP_ERR_INVALID, "links of level " + std::to_string(l) + " inconsistent");
  CSP_CUDA(ctx, cudaGetLastError());
  ctx->prepared = true;
  return CSP_OK;
}

bool valid_ptr_or_empty(const void *p, int64_t n) { return p != nullptr || n == 0; }

// Shape limits of a solve on this context (after prepare).
csp_status check_solve_shape(csp_ctx *ctx, const csp_solve_params *prm) {
  const int nl = prm->mode == CSP_MODE_PLAIN ? 1 : ctx->geom.n_levels;
  const int top = nl - 1;
  const LevelData &LT = ctx->lv[top];
  if (prm->precision == CSP_PREC_BF16 && !proxy_bf16_supported(LT.per_patch ? LT.N : LT.M, LT.T))
    return fail(ctx, CSP_ERR_UNSUPPORTED, "BF16 tensor-core proxy not available for this shape (proxy dimension <= 512, T <= 32768)");
  for (int l = 1; l < nl; ++l) {
    const int Kl = prm->K_patch[l] ? prm->Kmax : prm->K[l];
    const int cap = ctx->lv[l - 1].max_children * Kl;
    if (cap > 1024) return fail(ctx, CSP_ERR_UNSUPPORTED, "candidate capacity above 1024 (max children x K)");
  }
  return CSP_OK;
}

// Per-patch effective dictionaries and norms for B patches with code blocks
// pc, into A_pp/inv_pp (allocated by the caller, [B][T_l][M] and [B][T_l]).
csp_status build_patch_dicts(csp_ctx *ctx, int l, const uint8_t *pc, int64_t B, float *A_pp, float *inv_pp,
                             unsigned int *scratch, cudaStream_t s) {
  LevelData &L = ctx->lv[l];
  const int64_t rows = B * L.T;
  run(ctx, KK_PREP, s, rows,
      [&] { launch_effective_dict_pp_norms(ctx->gd, pc, l, L.D, L.T, L.N, A_pp, inv_pp, scratch, B, s); });
  CSP_CUDA(ctx, cudaGetLastError());
  return CSP_OK;
}

// Coded exposure: this context's own patch grid gets the full per-patch
// effective dictionary of level l (the full-dictionary level of a solve) once.
csp_status prepare_own_patches(csp_ctx *ctx, int l, cudaStream_t s) {
  if (ctx->sense_kind != CSP_SENSE_CODED_EXPOSURE || ctx->pp_A[l]) return CSP_OK;
  const LevelData &L = ctx->lv[l];
  CSP_TRY(dev_alloc_t(ctx, &ctx->pp_A[l], (size_t)ctx->B * L.T * L.M));
  CSP_TRY(dev_alloc_t(ctx, &ctx->pp_inv[l], (size_t)ctx->B * L.T));
  unsigned int *scratch = nullptr;
  CSP_TRY(ws_get_t(ctx, ctx->wsp, WS_SCRATCH, 4, &scratch));
  return build_patch_dicts(ctx, l, ctx->pcodes, ctx->B, ctx->pp_A[l], ctx->pp_inv[l], scratch, s);
}

// The second stream and the fork/join events of the pipelined solve.
csp_status ensure_aux(csp_ctx *ctx) {
  if (!ctx->aux) CSP_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->aux, cudaStreamNonBlocking));
  if (!ctx->ev_fork) CSP_CUDA(ctx, cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming));
  if (!ctx->ev_join) CSP_CUDA(ctx, cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming));
  return CSP_OK;
}

// Solve the patch set `ps` with the context's dictionaries (prepared), using
// workspace W.  With Xh (B x N0 floats), the finest restricted level may also
// synthesize x_hat_b = D0 alpha_b into Xh (*synthesized tells whether it did).  Arguments validated by the caller.
csp_status solve_core(csp_ctx *ctx, const PatchSet &ps, Workspace &W, const csp_solve_params *prm, const float *Y,
                      int32_t *support_out, float *coef_out, int8_t *k_eff_out, cudaStream_t s, float *Xh = nullptr,
                      bool *synthesized = nullptr) {
  const int64_t B = ps.B;
  const int nl = prm->mode == CSP_MODE_PLAIN ? 1 : ctx->geom.n_levels;
  if (synthesized) *synthesized = false;
  bool synth_all = Xh != nullptr && nl > 1;  // the finest level is restricted only in cross-scale mode
  int Kb[CSP_MAX_LEVELS];
  for (int l = 0; l < nl; ++l) Kb[l] = prm->K_patch[l] ? prm->Kmax : prm->K[l];
  const bool bf16 = prm->precision == CSP_PREC_BF16;
  const int top = nl - 1;
  CSP_CUDA(ctx, cudaMemsetAsync(W.stats_dev, 0, 8 * sizeof(int64_t), s));
  if (B == 0) return CSP_OK;

  // phase groups
  const bool phased = ps.phase_ids != nullptr;
  const int nph = phased ? 4 : 1;
  // work order (csp_set_work_order): with per-patch budgets and one operator
  // group, every level takes the patches sorted by the finest budget, largest
  // first, and the restricted levels pull them from a work queue
  const int32_t *order = nullptr;
  unsigned long long *queue = nullptr;
  if (ctx->work_order == 1 && !phased && prm->K_patch[0]) {
    int32_t *ord = nullptr;
    int *cnt = nullptr;
    CSP_TRY(ws_get_t(ctx, W, WS_ORDER, (size_t)B, &ord));
    CSP_TRY(ws_get_t(ctx, W, WS_ORDER_CNT, (size_t)2 * (CSP_MAX_K + 1), &cnt));
    CSP_TRY(ws_get_t(ctx, W, WS_QUEUE, (size_t)1, &queue));
    run(ctx, KK_PREP, s, B, [&] { launch_sort_by_budget(prm->K_patch[0], B, ord, cnt, s); });
    order = ord;
  }
  auto ids_of = [&](int ph) -> const int32_t * { return phased ? ps.phase_ids + ps.phase_start[ph] : order; };
  auto n_of = [&](int ph) -> int64_t { return phased ? ps.phase_start[ph + 1] - ps.phase_start[ph] : B; };

  // per-level measurement vectors (Phi = I: y_l = W_l y)
  const float *Yl[CSP_MAX_LEVELS];
  for (int l = 0; l < nl; ++l) {
    if (l > 0 && ctx->sense_kind == CSP_SENSE_IDENTITY) {
      float *buf = nullptr;
      CSP_TRY(ws_get_t(ctx, W, WS_LV_Y + l, (size_t)B * ctx->lv[l].M, &buf));
      run(ctx, KK_DOWNSAMPLE, s, B, [&] { launch_downsample(ctx->gd, l, Y, buf, B, s); });
      Yl[l] = buf;
    } else {
      Yl[l] = Y;
    }
  }

  // per-level outputs (level 0 writes straight into the caller's buffers)
  int32_t *lv_om[CSP_MAX_LEVELS];
  float *lv_al[CSP_MAX_LEVELS];
  int8_t *lv_ke[CSP_MAX_LEVELS];
  int ldo[CSP_MAX_LEVELS];
  for (int l = 0; l < nl; ++l) {
    if (l == 0) {
      lv_om[0] = support_out; lv_al[0] = coef_out; lv_ke[0] = k_eff_out; ldo[0] = prm->Kmax;
    } else {
      ldo[l] = Kb[l];
      CSP_TRY(ws_get_t(ctx, W, WS_LV_OMEGA + l, (size_t)B * Kb[l], &lv_om[l]));
      CSP_TRY(ws_get_t(ctx, W, WS_LV_ALPHA + l, (size_t)B * Kb[l], &lv_al[l]));
      CSP_TRY(ws_get_t(ctx, W, WS_LV_KEFF + l, (size_t)B, &lv_ke[l]));
    }
  }

  // full-dictionary OMP at the top level (the only level in plain mode), form 3:
  // the Gram form -- correlations P0 = Y A^T once (FP32 GEMM), then every
  // iteration from the level's Gram matrix with all atoms as candidates
  bool fused_done = false;
  if (ctx->top_form == 3) {
    const LevelData &L = ctx->lv[top];
    bool ok = !L.per_patch && full_gram_supported(L.M, L.T, Kb[top]);
    for (int ph = 0; ph < nph; ++ph) ok = ok && L.G[ph] != nullptr;
    if (ok) {
      float *P0 = nullptr;
      CSP_TRY(ws_get_t(ctx, W, WS_P0, (size_t)B * L.T, &P0));
      for (int ph = 0; ph < nph; ++ph) {
        // the correlation GEMM, then the iteration (timed apart while profiling)
        run(ctx, KK_PROXY_FP32, s, n_of(ph), [&] { launch_p0_gemm(Yl[top], L.M, L.A[ph], L.T, ids_of(ph), n_of(ph), P0, s); });
        run(ctx, KK_FULL_GRAM, s, n_of(ph), [&] {
          launch_omp_full_gram(Yl[top], L.M, L.A[ph], L.inv_norm[ph], ids_of(ph), n_of(ph), prm->K_patch[top],
                               prm->K[top], Kb[top], lv_om[top], lv_al[top], ldo[top], lv_ke[top], W.stats_dev,
                               L.G[ph], L.T, P0, s);
        });
      }
      fused_done = true;
    }
  }
  // otherwise all iterations in one fused kernel when the dictionary is small and shared
  if (!fused_done) {
    const LevelData &L = ctx->lv[top];
    const bool want = ctx->top_form == 0 || ctx->top_form == 2;  // automatic and 2: fused wherever it applies
    if (want && bf16 && !L.per_patch && L.Mp == 64 && fused_top_supported(L.M, L.T, Kb[top])) {
      const float *Aph[kMaxPhases] = {}, *Iph[kMaxPhases] = {};
      const __nv_bfloat16 *Bph[kMaxPhases] = {};
      const float *Gph[kMaxPhases] = {};
      for (int ph = 0; ph < nph; ++ph) {
        Aph[ph] = L.A[ph];
        Iph[ph] = L.inv_norm[ph];
        Bph[ph] = L.Abf[ph];
        Gph[ph] = L.G[ph];
      }
      // pipelined cross-scale solve: the first chunk (one full wave of the fused
      // kernel) goes down the scales on a second stream while the fused kernel
      // runs the rest, so the restricted solver fills the SMs the fused
      // kernel's last wave leaves idle.  Patches are independent: same results.
      // Applies to one non-empty phase group (positions map to patch ids
      // through its ids when there are ids, else they are the patch ids).
      bool finer_shared = top > 0;
      for (int l = 0; l < top; ++l) finer_shared = finer_shared && !ctx->lv[l].per_patch;
      int ph0 = 0, nonempty = 0;
      for (int ph = 0; ph < nph; ++ph)
        if (n_of(ph) > 0) { ph0 = ph; ++nonempty; }
      const int64_t wave = fused_wave_patches(L.T, Kb[top]);
      if (ctx->pipeline && nonempty == 1 && finer_shared && B > wave) {
        CSP_TRY(ensure_aux(ctx));
        const int32_t *ids0 = ids_of(ph0);
        auto fused_range = [&](int64_t off, int64_t n, cudaStream_t st) {
          const int64_t d = ids0 ? 0 : off;  // data offset
          bool ok = false;
          run(ctx, KK_FUSED, st, n, [&] {
            ok = launch_omp_fused_tc(Yl[top] + d * L.M, L.M, Aph + ph0, Iph + ph0, Bph + ph0, Gph + ph0, 1, nullptr,
                                     L.Mp, L.T, ids0 ? ids0 + off : nullptr, n,
                                     prm->K_patch[top] ? prm->K_patch[top] + d : nullptr, prm->K[top], Kb[top],
                                     lv_om[top] + d * ldo[top], lv_al[top] + d * ldo[top], ldo[top], lv_ke[top] + d,
                                     W.stats_dev, (unsigned long long *)(W.stats_dev + 4), st);
          });
          return ok;
        };
        auto restrict_range = [&](int64_t off, int64_t n, cudaStream_t st) {
          const int64_t d = ids0 ? 0 : off;
          for (int l = top - 1; l >= 0; --l) {
            const LevelData &Lr = ctx->lv[l];
            const int cap = std::max(1, Lr.max_children * Kb[l + 1]);
            run(ctx, KK_RESTRICTED, st, n, [&] {
              const bool sy = launch_omp_restricted(
                  ctx->restricted_variant, Yl[l] + d * Lr.M, Lr.M, Lr.A[ph0], Lr.inv_norm[ph0],
                  ids0 ? ids0 + off : nullptr, n, Lr.child_off, Lr.child_idx, cap, lv_om[l + 1] + d * ldo[l + 1],
                  ldo[l + 1], lv_ke[l + 1] + d, prm->K_patch[l] ? prm->K_patch[l] + d : nullptr, prm->K[l], Kb[l],
                  lv_om[l] + d * ldo[l], lv_al[l] + d * ldo[l], ldo[l], lv_ke[l] + d, W.stats_dev, Lr.G[ph0], Lr.T, 0,
                  0, false, st, l == 0 ? ctx->lv[0].D : nullptr, ctx->lv[0].N,
                  (l == 0 && Xh) ? Xh + d * ctx->lv[0].N : nullptr);
              if (l == 0) synth_all = synth_all && sy;
            });
          }
        };
        if (!fused_range(0, wave, s)) return fail(ctx, CSP_ERR_CUDA, "fused full-dictionary kernel could not be launched");
        CSP_CUDA(ctx, cudaEventRecord(ctx->ev_fork, s));
        if (!fused_range(wave, B - wave, s))
          return fail(ctx, CSP_ERR_CUDA, "fused full-dictionary kernel could not be launched");
        CSP_CUDA(ctx, cudaStreamWaitEvent(ctx->aux, ctx->ev_fork, 0));
        restrict_range(0, wave, ctx->aux);
        restrict_range(wave, B - wave, s);
        CSP_CUDA(ctx, cudaEventRecord(ctx->ev_join, ctx->aux));
        CSP_CUDA(ctx, cudaStreamWaitEvent(s, ctx->ev_join, 0));
        CSP_CUDA(ctx, cudaGetLastError());
        if (synthesized) *synthesized = synth_all;
        return CSP_OK;
      }
      run(ctx, KK_FUSED, s, B, [&] {
        fused_done = launch_omp_fused_tc(Yl[top], L.M, Aph, Iph, Bph, Gph, nph, phased ? ps.phase_start : nullptr, L.Mp,
                                         L.T, phased ? ps.phase_ids : order, B, prm->K_patch[top], prm->K[top],
                                         Kb[top], lv_om[top], lv_al[top], ldo[top], lv_ke[top], W.stats_dev,
                                         (unsigned long long *)(W.stats_dev + 4), s);
      });
      if (!fused_done) return fail(ctx, CSP_ERR_CUDA, "fused full-dictionary kernel could not be launched");
    }
  }
  if (!fused_done) {
    const LevelData &L = ctx->lv[top];
    const bool pp = L.per_patch;
    OmpState st{};
    CSP_TRY(ws_get_t(ctx, W, WS_R, (size_t)B * L.M, &st.R));
    st.Rbf = nullptr;
    if (bf16 && !pp) CSP_TRY(ws_get_t(ctx, W, WS_RBF, (size_t)B * L.Mp, &st.Rbf));
    // per-patch Phi: the proxy runs on the lifted residual z = U^T Phi_p^T r against D
    float *Zl = nullptr;
    __nv_bfloat16 *Zbf = nullptr;
    if (pp) {
      if (!bf16) CSP_TRY(ws_get_t(ctx, W, WS_LIFT, (size_t)B * L.N, &Zl));
      else CSP_TRY(ws_get_t(ctx, W, WS_LIFTBF, (size_t)B * L.Np, &Zbf));
    }
    // partial top-4 keys when the tensor-core proxy splits the atoms over CTAs;
    // best keys of the split FP32 proxy (zeroed here, left zeroed by each use)
    uint32_t *part = nullptr;
    unsigned long long *keys = nullptr;
    if (bf16) {
      int S = 1;
      for (int ph = 0; ph < nph; ++ph) S = std::max(S, proxy_bf16_splits(n_of(ph), L.T));
      if (S > 1) CSP_TRY(ws_get_t(ctx, W, WS_PART, (size_t)B * S * 4, &part));
    } else {
      int S = 1;
      for (int ph = 0; ph < nph; ++ph) S = std::max(S, proxy_fp32_splits(n_of(ph), L.T));
      if (S > 1) {
        CSP_TRY(ws_get_t(ctx, W, WS_KEYS, (size_t)B, &keys));
        CSP_CUDA(ctx, cudaMemsetAsync(keys, 0, (size_t)B * sizeof(unsigned long long), s));
      }
    }
    st.Kb = Kb[top];
    st.ldo = ldo[top];
    CSP_TRY(ws_get_t(ctx, W, WS_L, (size_t)B * (Kb[top] * (Kb[top] + 1) / 2), &st.Lpk));
    CSP_TRY(ws_get_t(ctx, W, WS_Z, (size_t)B * Kb[top], &st.z));
    CSP_TRY(ws_get_t(ctx, W, WS_FLAGS, (size_t)B, &st.flags));
    CSP_TRY(ws_get_t(ctx, W, WS_CAND, (size_t)B * kTopP, &st.cand));
    st.omega = lv_om[top];
    st.alpha = lv_al[top];
    st.k_eff = lv_ke[top];
    const int64_t a_ps = pp ? (int64_t)L.T * L.M : 0, inv_ps = pp ? (int64_t)L.T : 0;
    run(ctx, KK_INIT, s, B, [&] {
      launch_omp_init(Yl[top], B, L.M, (bf16 && !pp) ? L.Mp : 0, phased ? ps.phase_ids : order, st, s);
    });
    bool maps_ok = true;
    for (int it = 0; it < Kb[top]; ++it) {
      if (pp)
        run(ctx, KK_LIFT, s, B, [&] { launch_lift(ctx->gd, ps.pcodes, top, st.R, B, Zl, Zbf, bf16 ? L.Np : L.N, s); });
      for (int ph = 0; ph < nph; ++ph) {
        if (bf16)
          run(ctx, KK_PROXY_BF16, s, n_of(ph), [&] {
            maps_ok &= pp ? launch_proxy_bf16(Zbf, B, L.Np, L.Dbf, L.T, 0, ids_of(ph), n_of(ph), st.flags, st.cand,
                                              (unsigned long long *)(W.stats_dev + 4), ps.inv_pp[top], part, ctx->wait_test, s)
                          : launch_proxy_bf16(st.Rbf, B, L.Mp, L.Abf[ph], L.T, phased ? ps.phase_start[ph] : 0,
                                              ids_of(ph), n_of(ph), st.flags, st.cand,
                                              (unsigned long long *)(W.stats_dev + 4), nullptr, part, ctx->wait_test, s);
          });
        else
          run(ctx, KK_PROXY_FP32, s, n_of(ph), [&] {
            if (pp)
              launch_proxy_fp32(Zl, L.N, L.D, nullptr, L.T, ids_of(ph), n_of(ph), st.omega, st.ldo, st.k_eff, st.flags,
                                st.cand, ps.inv_pp[top], keys, s);
            else
              launch_proxy_fp32(st.R, L.M, L.A[ph], L.inv_norm[ph], L.T, ids_of(ph), n_of(ph), st.omega, st.ldo,
                                st.k_eff, st.flags, st.cand, nullptr, keys, s);
          });
      }
      for (int ph = 0; ph < nph; ++ph)
        run(ctx, KK_UPDATE, s, n_of(ph), [&] {
          launch_omp_update_wave(Yl[top], L.M, pp ? ps.A_pp[top] : L.A[ph], pp ? ps.inv_pp[top] : L.inv_norm[ph],
                                 ids_of(ph), n_of(ph),
                                 phased ? ps.phase_start[ph] : 0, bf16 ? kTopP : 1, prm->K_patch[top], prm->K[top],
                                 st, W.stats_dev, L.G[ph], L.T, a_ps, inv_ps, s);
        });
      if (!maps_ok) return fail(ctx, CSP_ERR_CUDA, "tensor map encoding for the BF16 proxy failed");
    }
  }
  // restricted OMP down the scales (Algorithm 2 fine steps)
  for (int l = top - 1; l >= 0; --l) {
    const LevelData &L = ctx->lv[l];
    const int cap = std::max(1, L.max_children * Kb[l + 1]);
    float *Ac = nullptr, *invc = nullptr, *Gpp = nullptr;
    if (L.per_patch) {
      // per-patch Phi: rows of this level's effective dictionary for each patch's
      // candidates only, with their Gram block for the Gram-Schmidt variants
      CSP_TRY(ws_get_t(ctx, W, WS_PPC_A, (size_t)B * cap * L.M, &Ac));
      CSP_TRY(ws_get_t(ctx, W, WS_PPC_INV, (size_t)B * cap, &invc));
      if (ctx->restricted_variant >= 2) CSP_TRY(ws_get_t(ctx, W, WS_PPC_G, (size_t)B * cap * cap, &Gpp));
      run(ctx, KK_PREP, s, B, [&] {
        if (!launch_pp_candidates(ctx->gd, ps.pcodes, l, L.D, L.N, L.M, lv_om[l + 1], ldo[l + 1], lv_ke[l + 1],
                                  L.child_off, L.child_idx, cap, B, Ac, invc, s, Gpp))
          Gpp = nullptr;
      });
    }
    for (int ph = 0; ph < nph; ++ph)
      run(ctx, KK_RESTRICTED, s, n_of(ph), [&] {
        const bool sy = launch_omp_restricted(
            ctx->restricted_variant, Yl[l], L.M, L.per_patch ? Ac : L.A[ph], L.per_patch ? invc : L.inv_norm[ph],
            ids_of(ph), n_of(ph), L.child_off, L.child_idx, cap, lv_om[l + 1], ldo[l + 1], lv_ke[l + 1],
            prm->K_patch[l], prm->K[l], Kb[l], lv_om[l], lv_al[l], ldo[l], lv_ke[l], W.stats_dev, L.G[ph], L.T,
            L.per_patch ? (int64_t)cap * L.M : 0, L.per_patch ? (int64_t)cap : 0, L.per_patch, s,
            l == 0 ? ctx->lv[0].D : nullptr, ctx->lv[0].N, l == 0 ? Xh : nullptr, queue, Gpp);
        if (l == 0) synth_all = synth_all && sy;
      });
  }
  CSP_CUDA(ctx, cudaGetLastError());
  if (synthesized) *synthesized = synth_all;
  return CSP_OK;
}

}  // namespace

namespace csp {

csp_status prepare_model(csp_ctx *ctx, cudaStream_t s) { return prepare(ctx, s); }

csp_status check_solve_params(csp_ctx *ctx, const csp_solve_params *prm) {
  if (!prm) return fail(ctx, CSP_ERR_INVALID, "params is NULL");
  if (prm->mode != CSP_MODE_PLAIN && prm->mode != CSP_MODE_CROSS_SCALE) return fail(ctx, CSP_ERR_INVALID, "unknown mode");
  if (prm->precision != CSP_PREC_FP32 && prm->precision != CSP_PREC_BF16)
    return fail(ctx, CSP_ERR_INVALID, "unknown precision");
  if (prm->Kmax < 1 || prm->Kmax > CSP_MAX_K) return fail(ctx, CSP_ERR_INVALID, "Kmax must be in 1..CSP_MAX_K");
  const int nl = prm->mode == CSP_MODE_PLAIN ? 1 : ctx->geom.n_levels;
  for (int l = 0; l < nl; ++l)
    if (!prm->K_patch[l] && (prm->K[l] < 1 || prm->K[l] > CSP_MAX_K))
      return fail(ctx, CSP_ERR_INVALID, "K[l] must be in 1..CSP_MAX_K");
  if (!prm->K_patch[0] && prm->K[0] > prm->Kmax) return fail(ctx, CSP_ERR_INVALID, "K[0] exceeds Kmax");
  for (int l = 0; l + 1 < nl; ++l)
    if (!ctx->lv[l].links) return fail(ctx, CSP_ERR_NOT_READY, "scale links of level " + std::to_string(l) + " not loaded");
  return check_solve_shape(ctx, prm);
}

csp_status solve_patchset(csp_ctx *ctx, const PatchSet &ps, Workspace &W, const csp_solve_params *prm,
                          const float *Y, int32_t *support_out, float *coef_out, int8_t *k_eff_out, cudaStream_t s) {
  return solve_core(ctx, ps, W, prm, Y, support_out, coef_out, k_eff_out, s);
}

csp_status build_patch_dicts_for(csp_ctx *ctx, int level, const uint8_t *pc, int64_t B, float *A_pp, float *inv_pp,
                                 unsigned int *scratch, cudaStream_t s) {
  return build_patch_dicts(ctx, level, pc, B, A_pp, inv_pp, scratch, s);
}

int64_t patch_count_1d(int E, int P, int stride) { return count_1d(E, P, stride); }

void cover_ranges(int E, int P, int stride, int n, std::vector<int32_t> &c) {
  // origins are nondecreasing, so the patches covering row y are the contiguous
  // range [lo, hi] with origin(hi) <= y < origin(lo) + P: one sweep over y
  // ((0, -2) where no patch covers y)
  c.assign(2 * (size_t)E, 0);
  auto org = [&](int i) { return std::min(i * stride, E - P); };
  int lo = 0, hi = -1;
  for (int y = 0; y < E; ++y) {
    while (hi + 1 < n && org(hi + 1) <= y) ++hi;
    while (lo < n && org(lo) + P <= y) ++lo;
    c[2 * y] = lo <= hi ? lo : 0;
    c[2 * y + 1] = lo <= hi ? hi : -2;
  }
}

GeomDev make_geom_dev(const csp_geometry &g, int H, int W) {
  GeomDev d{};
  d.H = H; d.W = W; d.Ly = g.plane_rows; d.Lx = g.plane_cols; d.P = g.P; d.stride = g.stride;
  d.nx = (int)count_1d(W, g.P, g.stride);
  d.ny = (int)count_1d(H, g.P, g.stride);
  d.n_levels = g.n_levels;
  for (int l = 0; l < CSP_MAX_LEVELS; ++l)
    for (int c = 0; c < 4; ++c) d.f[l][c] = l < g.n_levels ? g.factors[l][c] : 1;
  return d;
}

}  // namespace csp

namespace csp {

// Checks of csp_solve's arguments (buffers checked by the caller).
csp_status check_solve_args(csp_ctx *ctx, const csp_solve_params *prm, int64_t B) {
  if (!prm) return fail(ctx, CSP_ERR_INVALID, "params is NULL");
  if (B < 0) return fail(ctx, CSP_ERR_INVALID, "B < 0");
  if (prm->mode != CSP_MODE_PLAIN && prm->mode != CSP_MODE_CROSS_SCALE) return fail(ctx, CSP_ERR_INVALID, "unknown mode");
  if (prm->precision != CSP_PREC_FP32 && prm->precision != CSP_PREC_BF16)
    return fail(ctx, CSP_ERR_INVALID, "unknown precision");
  if (prm->Kmax < 1 || prm->Kmax > CSP_MAX_K) return fail(ctx, CSP_ERR_INVALID, "Kmax must be in 1..CSP_MAX_K");
  if (!ctx->has_geom || !ctx->has_sensing) return fail(ctx, CSP_ERR_NOT_READY, "geometry and sensing must be set");
  const int nl = prm->mode == CSP_MODE_PLAIN ? 1 : ctx->geom.n_levels;
  for (int l = 0; l < nl; ++l)
    if (!prm->K_patch[l] && (prm->K[l] < 1 || prm->K[l] > CSP_MAX_K))
      return fail(ctx, CSP_ERR_INVALID, "K[l] must be in 1..CSP_MAX_K");
  if (!prm->K_patch[0] && prm->K[0] > prm->Kmax) return fail(ctx, CSP_ERR_INVALID, "K[0] exceeds Kmax");
  for (int l = 0; l + 1 < nl; ++l)
    if (!ctx->lv[l].links) return fail(ctx, CSP_ERR_NOT_READY, "scale links of level " + std::to_string(l) + " not loaded");
  if ((ctx->sense_kind == CSP_SENSE_BAYER_RGGB || ctx->sense_kind == CSP_SENSE_CODED_EXPOSURE) && B != ctx->B)
    return fail(ctx, CSP_ERR_INVALID, "Bayer / coded-exposure sensing solves the geometry's patch grid: B must equal the patch count");
  return CSP_OK;
}

// Prepared dictionaries and the patch set of a solve of B patches.
csp_status solve_setup(csp_ctx *ctx, const csp_solve_params *prm, int64_t B, cudaStream_t s, PatchSet &ps) {
  const int nl = prm->mode == CSP_MODE_PLAIN ? 1 : ctx->geom.n_levels;
  CSP_TRY(prepare(ctx, s));
  CSP_TRY(check_solve_shape(ctx, prm));
  CSP_TRY(prepare_own_patches(ctx, nl - 1, s));  // the full-dictionary level of this solve
  ps.B = B;
  if (ctx->sense_kind == CSP_SENSE_BAYER_RGGB) {
    ps.phase_ids = ctx->phase_ids;
    for (int p = 0; p <= kMaxPhases; ++p) ps.phase_start[p] = ctx->phase_start[p];
  }
  ps.pcodes = ctx->pcodes;
  for (int l = 0; l < CSP_MAX_LEVELS; ++l) { ps.A_pp[l] = ctx->pp_A[l]; ps.inv_pp[l] = ctx->pp_inv[l]; }
  ctx->last_B = B;
  ctx->last_stream = s;
  return CSP_OK;
}

// Graph mode: replay the graph in `slot` when `key` matches the call it was
// recorded from; otherwise run `body` on s (which allocates whatever it
// needs and gives the result), then record the same launches on a private
// stream into the slot for the next calls.
template <typename F>
csp_status run_graphed(csp_ctx *ctx, csp_ctx::GraphSlot &slot, const csp_ctx::GraphKey &key, cudaStream_t s,
                       F &&body) {
  if (slot.exec && std::memcmp(&key, &slot.key, sizeof(key)) == 0) {
    CSP_CUDA(ctx, cudaGraphLaunch(slot.exec, s));
    return CSP_OK;
  }
  if (slot.exec) {
    cudaGraphExecDestroy(slot.exec);
    slot.exec = nullptr;
  }
  CSP_TRY(body(s));
  if (!ctx->gstream) CSP_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->gstream, cudaStreamNonBlocking));
  CSP_CUDA(ctx, cudaStreamBeginCapture(ctx->gstream, cudaStreamCaptureModeRelaxed));
  const csp_status st = body(ctx->gstream);
  cudaGraph_t graph = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(ctx->gstream, &graph);
  if (st != CSP_OK || ec != cudaSuccess || !graph) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return st != CSP_OK ? st : fail(ctx, CSP_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ec));
  }
  const cudaError_t ei = cudaGraphInstantiate(&slot.exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ei != cudaSuccess) {
    slot.exec = nullptr;
    cudaGetLastError();
    return fail(ctx, CSP_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ei));
  }
  std::memcpy(&slot.key, &key, sizeof(key));
  return CSP_OK;
}

// The context state and call arguments a recorded graph depends on.
csp_ctx::GraphKey graph_key(const csp_ctx *ctx, const csp_solve_params *prm) {
  csp_ctx::GraphKey key;
  std::memset(&key, 0, sizeof(key));  // padding included: compared byte by byte
  key.prm.mode = prm->mode;
  key.prm.precision = prm->precision;
  for (int l = 0; l < CSP_MAX_LEVELS; ++l) {
    key.prm.K[l] = prm->K[l];
    key.prm.K_patch[l] = prm->K_patch[l];
  }
  key.prm.Kmax = prm->Kmax;
  key.version = ctx->state_version;
  key.restricted_variant = ctx->restricted_variant;
  key.top_form = ctx->top_form;
  key.wait_test = ctx->wait_test;
  key.pipeline = ctx->pipeline;
  key.aggregate_path = ctx->aggregate_path;
  key.work_order = ctx->work_order;
  return key;
}

// Extraction, solve and aggregation of the context's patch grid from the
// device measurement image `meas` into the device image `img`, with the
// context's own buffers for the patches and codes.
csp_status reconstruct_core(csp_ctx *ctx, const csp_solve_params *prm, const float *meas, float *img, cudaStream_t s) {
  const int64_t B = ctx->B;
  const int N0 = ctx->lv[0].N;
  float *Y = (float *)ctx->h_Y.p;
  int32_t *sup = (int32_t *)ctx->h_sup.p;
  float *coef = (float *)ctx->h_coef.p;
  int8_t *keff = (int8_t *)ctx->h_keff.p;
  CSP_TRY(csp_extract_patches(ctx, meas, Y, nullptr, s));
  PatchSet ps;
  CSP_TRY(solve_setup(ctx, prm, B, s, ps));
  bool tiled = aggregate_use_tiled(ctx->aggregate_path, ctx->gd, N0, prm->Kmax);
  float *Xh = nullptr;
  if (!tiled) CSP_TRY(ws_get_t(ctx, ctx->wsp, WS_XH, (size_t)B * N0, &Xh));
  bool synthesized = false;
  CSP_TRY(solve_core(ctx, ps, ctx->wsp, prm, Y, sup, coef, keff, s, Xh, &synthesized));
  ctx->recon_synth = synthesized;
  if (tiled)
    run(ctx, KK_AGGREGATE, s, B, [&] {
      tiled = launch_aggregate_tiled(ctx->gd, ctx->lv[0].D, N0, sup, coef, keff, prm->Kmax, ctx->cover_y,
                                     ctx->cover_x, img, s);
    });
  if (!tiled) {
    if (!Xh) CSP_TRY(ws_get_t(ctx, ctx->wsp, WS_XH, (size_t)B * N0, &Xh));
    run(ctx, KK_AGGREGATE, s, B, [&] {
      if (!synthesized) launch_synth(ctx->gd, ctx->lv[0].D, N0, sup, coef, keff, prm->Kmax, Xh, s);
      launch_gather(ctx->gd, Xh, N0, ctx->cover_y, ctx->cover_x, img, s);
    });
  }
  CSP_CUDA(ctx, cudaGetLastError());
  return CSP_OK;
}

// Device buffers of the context's own patch grid for a reconstruction.
csp_status reconstruct_buffers(csp_ctx *ctx, const csp_solve_params *prm) {
  auto grow = [&](Buf &b, size_t bytes) -> csp_status {
    if (b.bytes >= bytes) return CSP_OK;
    dev_free(ctx, b.p);
    b.p = nullptr;
    b.bytes = 0;
    CSP_TRY(dev_alloc(ctx, &b.p, bytes));
    b.bytes = bytes;
    ++ctx->state_version;  // recorded graphs hold the old buffers
    return CSP_OK;
  };
  const int64_t B = ctx->B;
  CSP_TRY(grow(ctx->h_Y, (size_t)B * ctx->M * 4 + 16));
  CSP_TRY(grow(ctx->h_sup, (size_t)B * prm->Kmax * 4 + 16));
  CSP_TRY(grow(ctx->h_coef, (size_t)B * prm->Kmax * 4 + 16));
  CSP_TRY(grow(ctx->h_keff, (size_t)B + 16));
  return CSP_OK;
}

}  // namespace csp

using csp::check_solve_args;
using csp::solve_setup;
using csp::run_graphed;
using csp::graph_key;
using csp::reconstruct_core;
using csp::reconstruct_buffers;

namespace csp {
// Support checks and the by-atom sort of a [N][K] support array (K-SVD sweep
// and initialisation); synchronises `s` to read the device checks.
csp_status ksvd_sort(csp_ctx *ctx, const float *D, int M, int T, const float *X, int N, const int32_t *sup,
                     const float *coef, const int8_t *keff, int K, int split, bool resid, int **off, int32_t **seg,
                     float **R, float **rn2, float **xn2, cudaStream_t s) {
  const int C = ksvd_chunks(N);
  int *hist = nullptr;
  unsigned *err = nullptr;
  CSP_TRY(ws_get_t(ctx, ctx->wsp, WS_KS_HIST, (size_t)std::max(C, 1) * T * split, &hist));
  CSP_TRY(ws_get_t(ctx, ctx->wsp, WS_KS_OFF, (size_t)T * split + 1, off));
  CSP_TRY(ws_get_t(ctx, ctx->wsp, WS_KS_SEG, (size_t)std::max<int64_t>((int64_t)N * K, 1), seg));
  CSP_TRY(ws_get_t(ctx, ctx->wsp, WS_KS_ERR, 1, &err));
  if (resid) {
    CSP_TRY(ws_get_t(ctx, ctx->wsp, WS_KS_R, (size_t)std::max(N, 1) * M, R));
    CSP_TRY(ws_get_t(ctx, ctx->wsp, WS_KS_RN2, (size_t)std::max(N, 1), rn2));
    CSP_TRY(ws_get_t(ctx, ctx->wsp, WS_KS_XN2, (size_t)std::max(N, 1), xn2));
  }
  CSP_CUDA(ctx, cudaMemsetAsync(err, 0, sizeof(unsigned), s));
  run(ctx, KK_KSVD_SORT, s, 1, [&] {
    launch_ksvd_sort(D, M, T, X, N, sup, coef, keff, K, split, resid ? *R : nullptr, resid ? *rn2 : nullptr,
                     resid ? *xn2 : nullptr, hist, *off, *seg, err, s);
  });
  CSP_CUDA(ctx, cudaGetLastError());
  unsigned herr = 0;
  CSP_CUDA(ctx, cudaMemcpyAsync(&herr, err, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  CSP_CUDA(ctx, cudaStreamSynchronize(s));
  if (herr & 1) return fail(ctx, CSP_ERR_INVALID, "k_eff outside [0, K]");
  if (herr & 2) return fail(ctx, CSP_ERR_INVALID, "support entry outside [0, T)");
  if (herr & 4) return fail(ctx, CSP_ERR_INVALID, "an atom appears twice in one support");
  return CSP_OK;
}
}  // namespace csp

extern "C" {

csp_status csp_create(csp_ctx **out, int device, size_t mem_budget_bytes) {
  if (!out) return fail(nullptr, CSP_ERR_INVALID, "out is NULL");
  *out = nullptr;
  int n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(nullptr, CSP_ERR_CUDA, std::string("cudaGetDeviceCount: ") + cudaGetErrorString(e));
  }
  if (device < 0 || device >= n) return fail(nullptr, CSP_ERR_INVALID, "device index out of range");
  csp_ctx *ctx = new (std::nothrow) csp_ctx();
  if (!ctx) return fail(nullptr, CSP_ERR_OOM, "host allocation failed");
  ctx->device = device;
  ctx->budget = mem_budget_bytes;
  DeviceGuard g(device);
  if (!g.ok) { delete ctx; return fail(nullptr, CSP_ERR_CUDA, "cudaSetDevice failed"); }
  if (dev_alloc_t(ctx, &ctx->wsp.stats_dev, 8) != CSP_OK) {
    std::string m = ctx->err;
    delete ctx;
    return fail(nullptr, CSP_ERR_OOM, m);
  }
  cudaMemset(ctx->wsp.stats_dev, 0, 8 * sizeof(int64_t));
  csp::noalloc_setup(device);  // the no-alloc aggregation's scratch address, once per device
  *out = ctx;
  return CSP_OK;
}

void csp_destroy(csp_ctx *ctx) {
  if (!ctx) return;
  DeviceGuard g(ctx->device);
  cudaDeviceSynchronize();
  for (auto &a : ctx->allocs) cudaFree(a.first);
  for (auto &r : ctx->pending) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
  for (auto e : ctx->ev_pool) cudaEventDestroy(e);
  if (ctx->g_solve.exec) cudaGraphExecDestroy(ctx->g_solve.exec);
  if (ctx->g_recon.exec) cudaGraphExecDestroy(ctx->g_recon.exec);
  if (ctx->g_host.exec) cudaGraphExecDestroy(ctx->g_host.exec);
  if (ctx->gstream) cudaStreamDestroy(ctx->gstream);
  if (ctx->aux) cudaStreamDestroy(ctx->aux);
  if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
  if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
  delete ctx;
}

const char *csp_last_error(const csp_ctx *ctx) { return ctx ? ctx->err.c_str() : g_create_error.c_str(); }

csp_status csp_set_geometry(csp_ctx *ctx, const csp_geometry *geom) {
  if (!ctx) return fail(nullptr, CSP_ERR_INVALID, "ctx is NULL");
  if (!geom) return fail(ctx, CSP_ERR_INVALID, "geometry is NULL");
  const csp_geometry &g = *geom;
  if (g.P < 1 || g.stride < 1 || g.H < g.P || g.W < g.P || g.plane_rows < 1 || g.plane_cols < 1)
    return fail(ctx, CSP_ERR_INVALID, "invalid extents: need 1 <= P <= H, W; stride >= 1; plane grid >= 1");
  if (g.n_levels < 1 || g.n_levels > CSP_MAX_LEVELS)
    return fail(ctx, CSP_ERR_INVALID, "n_levels must be in 1..CSP_MAX_LEVELS");
  const int dims[4] = {g.plane_rows, g.plane_cols, g.P, g.P};
  for (int l = 0; l < g.n_levels; ++l)
    for (int c = 0; c < 4; ++c) {
      const int f = g.factors[l][c];
      if (f < 1 || dims[c] % f) return fail(ctx, CSP_ERR_INVALID, "scale factor does not divide the extent");
      if (l == 0 && f != 1) return fail(ctx, CSP_ERR_INVALID, "level 0 factors must be 1");
      if (l > 0 && f % g.factors[l - 1][c]) return fail(ctx, CSP_ERR_INVALID, "scale factors must nest");
    }
  DeviceGuard dg(ctx->device);
  const int64_t ny = count_1d(g.H, g.P, g.stride), nx = count_1d(g.W, g.P, g.stride);
  if (ny * nx > (int64_t)INT32_MAX) return fail(ctx, CSP_ERR_INVALID, "too many patches");
  // cover ranges: patches iy with origin(iy) <= y < origin(iy) + P
  auto cover = [&](int E, int n) {
    std::vector<int32_t> c;
    cover_ranges(E, g.P, g.stride, n, c);
    return c;
  };
  std::vector<int32_t> cy = cover(g.H, (int)ny), cx = cover(g.W, (int)nx);
  dev_free(ctx, ctx->cover_y);
  dev_free(ctx, ctx->cover_x);
  ctx->cover_y = ctx->cover_x = nullptr;
  CSP_TRY(dev_alloc_t(ctx, &ctx->cover_y, cy.size()));
  CSP_TRY(dev_alloc_t(ctx, &ctx->cover_x, cx.size()));
  CSP_CUDA(ctx, cudaMemcpy(ctx->cover_y, cy.data(), cy.size() * 4, cudaMemcpyHostToDevice));
  CSP_CUDA(ctx, cudaMemcpy(ctx->cover_x, cx.data(), cx.size() * 4, cudaMemcpyHostToDevice));
  // a new geometry invalidates everything shaped by it
  for (int l = 0; l < CSP_MAX_LEVELS; ++l) {
    free_level_derived(ctx, ctx->lv[l]);
    free_links(ctx, ctx->lv[l]);
    dev_free(ctx, ctx->lv[l].D);
    ctx->lv[l] = LevelData();
  }
  dev_free(ctx, ctx->codes);
  ctx->codes = nullptr;
  dev_free(ctx, ctx->pcodes);
  ctx->pcodes = nullptr;
  dev_free(ctx, ctx->phi);
  ctx->phi = nullptr;
  dev_free(ctx, ctx->phase_ids);
  ctx->phase_ids = nullptr;
  ctx->has_sensing = false;
  ctx->geom = g;
  GeomDev &d = ctx->gd;
  d.H = g.H; d.W = g.W; d.Ly = g.plane_rows; d.Lx = g.plane_cols; d.P = g.P; d.stride = g.stride;
  d.nx = (int)nx; d.ny = (int)ny; d.n_levels = g.n_levels;
  for (int l = 0; l < CSP_MAX_LEVELS; ++l)
    for (int c = 0; c < 4; ++c) d.f[l][c] = l < g.n_levels ? g.factors[l][c] : 1;
  ctx->B = nx * ny;
  ctx->has_geom = true;
  ctx->prepared = false;
  ++ctx->state_version;
  free_own_patches(ctx);
  return CSP_OK;
}

csp_status csp_set_sensing(csp_ctx *ctx, const csp_sensing *sensing) {
  if (!ctx) return fail(nullptr, CSP_ERR_INVALID, "ctx is NULL");
  if (!sensing) return fail(ctx, CSP_ERR_INVALID, "sensing is NULL");
  if (!ctx->has_geom) return fail(ctx, CSP_ERR_NOT_READY, "set the geometry first");
  const csp_geometry &g = ctx->geom;
  const int planes = g.plane_rows * g.plane_cols;
  const int PP = g.P * g.P;
  size_t code_bytes = 0;
  int M = 0;
  switch (sensing->kind) {
    case CSP_SENSE_IDENTITY: M = planes * PP; break;
    case CSP_SENSE_BAYER_RGGB:
      if (g.plane_rows != 1 || g.plane_cols != 3) return fail(ctx, CSP_ERR_INVALID, "Bayer sensing needs a 1x3 (RGB) plane grid");
      M = PP;
      break;
    case CSP_SENSE_CODED_EXPOSURE:
      if (!sensing->codes) return fail(ctx, CSP_ERR_INVALID, "coded exposure needs codes");
      if (g.plane_rows != 1) return fail(ctx, CSP_ERR_INVALID, "coded exposure needs a 1 x F (frames) plane grid");
      M = PP;
      code_bytes = (size_t)planes * g.H * g.W;
      break;
    case CSP_SENSE_CODED_APERTURE:
      if (!sensing->codes || sensing->shots < 1) return fail(ctx, CSP_ERR_INVALID, "coded aperture needs shots >= 1 and codes");
      M = sensing->shots * PP;
      code_bytes = (size_t)sensing->shots * planes;
      break;
    case CSP_SENSE_DENSE:
      if (!sensing->phi || sensing->shots < 4 || sensing->shots % 4)
        return fail(ctx, CSP_ERR_INVALID, "dense sensing needs phi and M = shots, a positive multiple of 4");
      M = sensing->shots;
      break;
    default: return fail(ctx, CSP_ERR_INVALID, "unknown sensing kind");
  }
  if (M > 256) return fail(ctx, CSP_ERR_UNSUPPORTED, "measurement dimension above 256 is not supported");
  DeviceGuard dg(ctx->device);
  dev_free(ctx, ctx->codes);
  ctx->codes = nullptr;
  if (code_bytes) {
    CSP_TRY(dev_alloc_t(ctx, &ctx->codes, code_bytes));
    CSP_CUDA(ctx, cudaMemcpy(ctx->codes, sensing->codes, code_bytes, cudaMemcpyHostToDevice));
  }
  dev_free(ctx, ctx->phi);
  ctx->phi = nullptr;
  if (sensing->kind == CSP_SENSE_DENSE) {
    const size_t n = (size_t)M * planes * PP;
    CSP_TRY(dev_alloc_t(ctx, &ctx->phi, n));
    CSP_CUDA(ctx, cudaMemcpy(ctx->phi, sensing->phi, n * sizeof(float), cudaMemcpyHostToDevice));
  }
  // patches grouped by Bayer phase (a single group for every other operator)
  dev_free(ctx, ctx->phase_ids);
  ctx->phase_ids = nullptr;
  std::fill(std::begin(ctx->phase_start), std::end(ctx->phase_start), 0);
  if (sensing->kind == CSP_SENSE_BAYER_RGGB) {
    std::vector<int32_t> ids;
    ids.reserve((size_t)ctx->B);
    for (int ph = 0; ph < 4; ++ph) {
      ctx->phase_start[ph] = (int64_t)ids.size();
      for (int64_t b = 0; b < ctx->B; ++b) {
        const int iy = (int)(b / ctx->gd.nx), ix = (int)(b % ctx->gd.nx);
        const int oy = std::min(iy * g.stride, g.H - g.P), ox = std::min(ix * g.stride, g.W - g.P);
        if (2 * (oy & 1) + (ox & 1) == ph) ids.push_back((int32_t)b);
      }
    }
    ctx->phase_start[4] = (int64_t)ids.size();
    CSP_TRY(dev_alloc_t(ctx, &ctx->phase_ids, ids.size()));
    CSP_CUDA(ctx, cudaMemcpy(ctx->phase_ids, ids.data(), ids.size() * 4, cudaMemcpyHostToDevice));
  }
  dev_free(ctx, ctx->pcodes);
  ctx->pcodes = nullptr;
  if (sensing->kind == CSP_SENSE_CODED_EXPOSURE) {
    // per-patch code blocks of this grid: the per-patch operators read only these
    CSP_TRY(dev_alloc_t(ctx, &ctx->pcodes, (size_t)ctx->B * planes * PP));
    launch_patch_codes(ctx->gd, ctx->codes, ctx->B, ctx->pcodes, nullptr);
    CSP_CUDA(ctx, cudaDeviceSynchronize());
  }
  ctx->sense_kind = sensing->kind;
  ctx->shots = sensing->kind == CSP_SENSE_CODED_APERTURE ? sensing->shots : 0;
  ctx->M = M;
  ctx->has_sensing = true;
  ctx->prepared = false;
  ++ctx->state_version;
  free_own_patches(ctx);
  return CSP_OK;
}

csp_status csp_load_dictionary(csp_ctx *ctx, int level, const float *D, int N_l, int T_l, int is_device_ptr) {
  if (!ctx) return fail(nullptr, CSP_ERR_INVALID, "ctx is NULL");
  if (!ctx->has_geom) return fail(ctx, CSP_ERR_NOT_READY, "set the geometry first");
  if (level < 0 || level >= ctx->geom.n_levels) return fail(ctx, CSP_ERR_INVALID, "level out of range");
  if (N_l != level_dim(ctx->geom, level))
    return fail(ctx, CSP_ERR_INVALID, "N_l = " + std::to_string(N_l) + " does not match the level's patch dimension " +
                                          std::to_string(level_dim(ctx->geom, level)));
  if (T_l < 1 || !D) return fail(ctx, CSP_ERR_INVALID, "empty dictionary");
  DeviceGuard dg(ctx->device);
  LevelData &L = ctx->lv[level];
  free_level_derived(ctx, L);
  free_links(ctx, L);
  if (level > 0) free_links(ctx, ctx->lv[level - 1]);
  dev_free(ctx, L.D);
  L.D = nullptr;
  CSP_TRY(dev_alloc_t(ctx, &L.D, (size_t)N_l * T_l));
  CSP_CUDA(ctx, cudaMemcpy(L.D, D, sizeof(float) * (size_t)N_l * T_l,
                           is_device_ptr ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice));
  L.N = N_l;
  L.T = T_l;
  ctx->prepared = false;
  ++ctx->state_version;
  free_own_patches(ctx);
  return CSP_OK;
}

csp_status csp_load_scale_links(csp_ctx *ctx, int level, const int32_t *parent, int T_l, int Q) {
  if (!ctx) return fail(nullptr, CSP_ERR_INVALID, "ctx is NULL");
  if (!ctx->has_geom) return fail(ctx, CSP_ERR_NOT_READY, "set the geometry first");
  if (level < 0 || level + 1 >= ctx->geom.n_levels) return fail(ctx, CSP_ERR_INVALID, "level out of range for links");
  LevelData &F = ctx->lv[level], &C = ctx->lv[level + 1];
  if (!F.D || !C.D) return fail(ctx, CSP_ERR_NOT_READY, "load both dictionaries before their links");
  if (T_l != F.T) return fail(ctx, CSP_ERR_INVALID, "T_l does not match the loaded dictionary");
  std::vector<int32_t> par((size_t)T_l);
  if (!parent) {
    if (Q < 1 || (int64_t)Q * C.T != T_l) return fail(ctx, CSP_ERR_INVALID, "block map needs T_l = Q * T_{l+1}");
    for (int i = 0; i < T_l; ++i) par[i] = i / Q;
  } else {
    std::memcpy(par.data(), parent, sizeof(int32_t) * (size_t)T_l);
    for (int i = 0; i < T_l; ++i)
      if (par[i] < 0 || par[i] >= C.T)
        return fail(ctx, CSP_ERR_INVALID, "parent[" + std::to_string(i) + "] out of range");
  }
  std::vector<int32_t> off((size_t)C.T + 1, 0), idx((size_t)T_l);
  for (int i = 0; i < T_l; ++i) ++off[par[i] + 1];
  int mx = 0;
  for (int p = 0; p < C.T; ++p) { mx = std::max(mx, off[p + 1]); off[p + 1] += off[p]; }
  std::vector<int32_t> fillp(off.begin(), off.end() - 1);
  for (int i = 0; i < T_l; ++i) idx[fillp[par[i]]++] = i;  // ascending within each parent
  DeviceGuard dg(ctx->device);
  free_links(ctx, F);
  CSP_TRY(dev_alloc_t(ctx, &F.child_off, off.size()));
  CSP_TRY(dev_alloc_t(ctx, &F.child_idx, idx.size()));
  CSP_CUDA(ctx, cudaMemcpy(F.child_off, off.data(), off.size() * 4, cudaMemcpyHostToDevice));
  CSP_CUDA(ctx, cudaMemcpy(F.child_idx, idx.data(), idx.size() * 4, cudaMemcpyHostToDevice));
  F.max_children = mx;
  F.links = true;
  ++ctx->state_version;
  return CSP_OK;
}

csp_status csp_problem_size(const csp_ctx *ctx, int64_t *B_out, int *M_out) {
  if (!ctx) return fail(nullptr, CSP_ERR_INVALID, "ctx is NULL");
  if (!ctx->has_geom || !ctx->has_sensing) return CSP_ERR_NOT_READY;
  if (B_out) *B_out = ctx->B;
  if (M_out) *M_out = ctx->M;
  return CSP_OK;
}

csp_status csp_extract_patches(csp_ctx *ctx, const float *meas, float *Y_out, int64_t *B_out, void *stream) {
  if (!ctx) return fail(nullptr, CSP_ERR_INVALID, "ctx is NULL");
  if (!ctx->has_geom || !ctx->has_sensing) return fail(ctx, CSP_ERR_NOT_READY, "geometry and sensing must be set");
  if (!meas || !Y_out) return fail(ctx, CSP_ERR_INVALID, "NULL buffer");
  if (ctx->sense_kind == CSP_SENSE_DENSE)
    return fail(ctx, CSP_ERR_UNSUPPORTED, "dense sensing measures each patch: pass the measurements to csp_solve");
  DeviceGuard dg(ctx->device);
  run(ctx, KK_EXTRACT, (cudaStream_t)stream, ctx->B * ctx->M, [&] {
    launch_extract(ctx->gd, ctx->sense_kind, ctx->shots, meas, Y_out, ctx->B, ctx->M, (cudaStream_t)stream);
  });
  CSP_CUDA(ctx, cudaGetLastError());
  if (B_out) *B_out = ctx->B;
  return CSP_OK;
}


csp_status csp_solve(csp_ctx *ctx, const csp_solve_params *prm, const float *Y, int64_t B,
                     int32_t *support_out, float *coef_out, int8_t *k_eff_out, void *stream) {
  if (!ctx) return fail(nullptr, CSP_ERR_INVALID, "ctx is NULL");
  CSP_TRY(check_solve_args(ctx, prm, B));
  if (!valid_ptr_or_empty(Y, B) || !valid_ptr_or_empty(support_out, B) || !valid_ptr_or_empty(coef_out, B) ||
      !valid_ptr_or_empty(k_eff_out, B))
    return fail(ctx, CSP_ERR_INVALID, "NULL buffer");
  cudaStream_t s = (cudaStream_t)stream;
  DeviceGuard dg(ctx->device);
  PatchSet ps;
  CSP_TRY(solve_setup(ctx, prm, B, s, ps));
  ctx->last_synth = false;
  auto body = [&](cudaStream_t st) {
    return solve_core(ctx, ps, ctx->wsp, prm, Y, support_out, coef_out, k_eff_out, st);
  };
  if (!ctx->graph_mode || ctx->prof) return body(s);
  csp_ctx::GraphKey key = graph_key(ctx, prm);
  key.Y = Y;
  key.B = B;
  key.sup = support_out;
  key.coef = coef_out;
  key.keff = k_eff_out;
  return run_graphed(ctx, ctx->g_solve, key, s, body);
}

csp_status csp_reconstruct(csp_ctx *ctx, const csp_solve_params *prm, const float *meas, float *image_out,
                           void *stream) {
  if (!ctx) return fail(nullptr, CSP_ERR_INVALID, "ctx is NULL");
  if (!prm || !meas || !image_out) return fail(ctx, CSP_ERR_INVALID, "NULL argument");
  for (int l = 0; l < CSP_MAX_LEVELS; ++l)
    if (prm->K_patch[l]) return fail(ctx, CSP_ERR_INVALID, "per-patch budgets are not accepted by csp_reconstruct");
  if (ctx->sense_kind == CSP_SENSE_DENSE)
    return fail(ctx, CSP_ERR_UNSUPPORTED, "dense sensing has no measurement image to extract patches from");
  CSP_TRY(check_solve_args(ctx, prm, ctx->B));
  if (!ctx->lv[0].D) return fail(ctx, CSP_ERR_NOT_READY, "fine dictionary not loaded");
  cudaStream_t s = (cudaStream_t)stream;
  DeviceGuard dg(ctx->device);
  CSP_TRY(reconstruct_buffers(ctx, prm));
  auto body = [&](cudaStream_t st) { return reconstruct_core(ctx, prm, meas, image_out, st); };
  csp_status st = CSP_OK;
  if (!ctx->graph_mode || ctx->prof) {
    st = body(s);
  } else {
    csp_ctx::GraphKey key = graph_key(ctx, prm);
    key.Y = meas;
    key.B = ctx->B;
    key.coef = image_out;
    st = run_graphed(ctx, ctx->g_recon, key, s, body);
  }
  ctx->last_synth = st == CSP_OK && ctx->recon_synth;
  return st;
}

csp_status csp_set_graph_mode(csp_ctx *ctx, int on) {
  if (!ctx) return fail(nullptr, CSP_ERR_INVALID, "ctx is NULL");
  ctx->graph_mode = on != 0;
  if (!ctx->graph_mode)
    for (csp_ctx::GraphSlot *g : {&ctx->g_solve, &ctx->g_recon, &ctx->g_host})
      if (g->exec) {
        cudaGraphExecDestroy(g->exec);
        g->exec = nullptr;
      }
  return CSP_OK;
}

csp_status csp_set_pipeline(csp_ctx *ctx, int on) {
  if (!ctx) return fail(nullptr, CSP_ERR_INVALID, "ctx is NULL");
  ctx->pipeline = on != 0;
  return CSP_OK;
}

csp_status csp_solve_stats_get(csp_ctx *ctx, csp_solve_stats *out) {
  if (!ctx || !out) return fail(ctx, CSP_ERR_INVALID, "NULL argument");
  DeviceGuard dg(ctx->device);
  int64_t h[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  CSP_CUDA(ctx, cudaStreamSynchronize(ctx->last_stream));
  CSP_CUDA(ctx, cudaMemcpy(h, ctx->wsp.stats_dev, sizeof(h), cudaMemcpyDeviceToHost));
  out->patches = ctx->last_B;
  out->fp64_fallbacks = h[0];
  out->early_stops = h[1];
  out->overflow = h[3];
  out->restricted_scores = h[2];
  out->timeouts = h[4] != 0 ? 1 : 0;
  out->synthesized = ctx->last_synth ? 1 : 0;
  if (h[4] != 0)
    return fail(ctx, CSP_ERR_TIMEOUT, "a bounded device wait expired (code " + std::to_string(h[4]) + ")");
  return CSP_OK;
}

csp_status csp_aggregate(csp_ctx *ctx, const int32_t *support, const float *coef, const int8_t *k_eff, int64_t B,
                         int Kmax, float *image_out, void *stream) {
  if (!ctx) return fail(nullptr, CSP_ERR_INVALID, "ctx is NULL");
  if (!ctx->has_geom) return fail(ctx, CSP_ERR_NOT_READY, "geometry not set");
  if (!ctx->lv[0].D) return fail(ctx, CSP_ERR_NOT_READY, "fine dictionary not loaded");
  if (B != ctx->B) return fail(ctx, CSP_ERR_INVALID, "B must equal the geometry's patch count");
  if (Kmax < 1 || Kmax > CSP_MAX_K) return fail(ctx, CSP_ERR_INVALID, "Kmax must be in 1..CSP_MAX_K");
  if (!support || !coef || !k_eff || !image_out) return fail(ctx, CSP_ERR_INVALID, "NULL buffer");
  DeviceGuard dg(ctx->device);
  bool tiled = aggregate_use_tiled(ctx->aggregate_path, ctx->gd, ctx->lv[0].N, Kmax);
  if (tiled)
    run(ctx, KK_AGGREGATE, (cudaStream_t)stream, B, [&] {
      tiled = launch_aggregate_tiled(ctx->gd, ctx->lv[0].D, ctx->lv[0].N, support, coef, k_eff, Kmax, ctx->cover_y,
                                     ctx->cover_x, image_out, (cudaStream_t)stream);
    });
  if (!tiled) {  // two-pass: synthesis scratch in HBM (L2-resident at these sizes)
    float *Xh = nullptr;
    CSP_TRY(ws_get_t(ctx, ctx->wsp, WS_XH, (size_t)B * ctx->lv[0].N, &Xh));
    run(ctx, KK_AGGREGATE, (cudaStream_t)stream, B, [&] {
      launch_aggregate(ctx->gd, ctx->lv[0].D, ctx->lv[0].N, support, coef, k_eff, Kmax, ctx->cover_y, ctx->cover_x,
                       Xh, image_out, (cudaStream_t)stream);
    });
  }
  CSP_CUDA(ctx, cudaGetLastError());
  return CSP_OK;
}

csp_status csp_reconstruct_host(csp_ctx *ctx, const csp_solve_params *prm, const float *meas_host,
                                float *image_host, void *stream) {
  if (!ctx) return fail(nullptr, CSP_ERR_INVALID, "ctx is NULL");
  if (!prm || !meas_host || !image_host) return fail(ctx, CSP_ERR_INVALID, "NULL argument");
  for (int l = 0; l < CSP_MAX_LEVELS; ++l)
    if (prm->K_patch[l]) return fail(ctx, CSP_ERR_INVALID, "per-patch budgets are not accepted by csp_reconstruct_host");
  if (!ctx->has_geom || !ctx->has_sensing) return fail(ctx, CSP_ERR_NOT_READY, "geometry and sensing must be set");
  const csp_geometry &g = ctx->geom;
  const int planes = g.plane_rows * g.plane_cols;
  size_t meas_n = 0;
  switch (ctx->sense_kind) {
    case CSP_SENSE_IDENTITY: meas_n = (size_t)planes * g.H * g.W; break;
    case CSP_SENSE_CODED_APERTURE: meas_n = (size_t)ctx->shots * g.H * g.W; break;
    default: meas_n = (size_t)g.H * g.W;
  }
  const size_t img_n = (size_t)planes * g.H * g.W;
  cudaStream_t s = (cudaStream_t)stream;
  DeviceGuard dg(ctx->device);
  auto grow = [&](Buf &b, size_t bytes) -> csp_status {
    if (b.bytes >= bytes) return CSP_OK;
    dev_free(ctx, b.p);
    b.p = nullptr;
    b.bytes = 0;
    CSP_TRY(dev_alloc(ctx, &b.p, bytes));
    b.bytes = bytes;
    ++ctx->state_version;  // recorded graphs hold the old buffers
    return CSP_OK;
  };
  CSP_TRY(grow(ctx->h_meas, meas_n * 4));
  CSP_TRY(grow(ctx->h_img, img_n * 4));
  // page-locked host buffers: the overlap-add writes the image straight into
  // the host buffer through its device mapping (over the host link, no staging
  // copy), and in graph mode the input copy joins the recorded graph
  auto pinned = [](const void *p) {
    cudaPointerAttributes a;
    const bool ok = cudaPointerGetAttributes(&a, p) == cudaSuccess && a.type == cudaMemoryTypeHost;
    cudaGetLastError();
    return ok;
  };
  float *img_view = nullptr;
  if (pinned(image_host) && cudaHostGetDevicePointer((void **)&img_view, image_host, 0) != cudaSuccess) {
    cudaGetLastError();
    img_view = nullptr;
  }
  float *img_out = img_view ? img_view : (float *)ctx->h_img.p;
  // a page-locked, 16-byte aligned meas_host is read once by a copy kernel
  // through its device mapping (faster than a copy-engine transfer of this size)
  const float *meas_view = nullptr;
  if (pinned(meas_host) && (reinterpret_cast<uintptr_t>(meas_host) & 15) == 0 &&
      cudaHostGetDevicePointer((void **)&meas_view, (void *)meas_host, 0) != cudaSuccess) {
    cudaGetLastError();
    meas_view = nullptr;
  }
  auto copy_in = [&](cudaStream_t st) -> csp_status {
    if (meas_view) run(ctx, KK_EXTRACT, st, (int64_t)meas_n, [&] {
      launch_copy_floats(meas_view, (float *)ctx->h_meas.p, (int64_t)meas_n, st);
    });
    else CSP_CUDA(ctx, cudaMemcpyAsync(ctx->h_meas.p, meas_host, meas_n * 4, cudaMemcpyHostToDevice, st));
    return CSP_OK;
  };
  if (ctx->graph_mode && !ctx->prof && pinned(meas_host)) {
    if (ctx->sense_kind == CSP_SENSE_DENSE)
      return fail(ctx, CSP_ERR_UNSUPPORTED, "dense sensing has no measurement image to extract patches from");
    CSP_TRY(check_solve_args(ctx, prm, ctx->B));
    if (!ctx->lv[0].D) return fail(ctx, CSP_ERR_NOT_READY, "fine dictionary not loaded");
    CSP_TRY(reconstruct_buffers(ctx, prm));
    auto body = [&](cudaStream_t st) -> csp_status {
      CSP_TRY(copy_in(st));
      CSP_TRY(reconstruct_core(ctx, prm, (const float *)ctx->h_meas.p, img_out, st));
      if (!img_view) CSP_CUDA(ctx, cudaMemcpyAsync(image_host, ctx->h_img.p, img_n * 4, cudaMemcpyDeviceToHost, st));
      return CSP_OK;
    };
    csp_ctx::GraphKey key = graph_key(ctx, prm);
    key.Y = meas_host;
    key.B = ctx->B;
    key.coef = image_host;
    const csp_status st = run_graphed(ctx, ctx->g_host, key, s, body);
    ctx->last_synth = st == CSP_OK && ctx->recon_synth;
    CSP_TRY(st);
    CSP_CUDA(ctx, cudaStreamSynchronize(s));
    return CSP_OK;
  }
  CSP_TRY(copy_in(s));
  CSP_TRY(csp_reconstruct(ctx, prm, (const float *)ctx->h_meas.p, img_out, stream));
  if (!img_view) CSP_CUDA(ctx, cudaMemcpyAsync(image_host, ctx->h_img.p, img_n * 4, cudaMemcpyDeviceToHost, s));
  CSP_CUDA(ctx, cudaStreamSynchronize(s));
  return CSP_OK;
}

csp_status csp_autotune(csp_ctx *ctx, const csp_solve_params *params, const float *Y, int64_t B,
                        int32_t *support_out, float *coef_out, int8_t *k_eff_out, void *stream,
                        csp_tune_result *out) {
  if (!ctx) return fail(nullptr, CSP_ERR_INVALID, "ctx is NULL");
  if (!out) return fail(ctx, CSP_ERR_INVALID, "out is NULL");
  DeviceGuard dg(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CSP_CUDA(ctx, cudaEventCreate(&e0));
  CSP_CUDA(ctx, cudaEventCreate(&e1));
  const int saved = ctx->restricted_variant;
  int best = saved;
  double best_ms = 1e300;
  csp_status st = CSP_OK;
  // A cross-scale batch of the context's own patch grid is timed with the
  // synthesis x_hat_p = D0 alpha_p of every patch, as csp_reconstruct runs it
  // (inside the finest restricted kernel where the variant writes it, else the
  // synthesis kernel): the variants differ in that part too.
  const bool with_synth = params && params->mode == CSP_MODE_CROSS_SCALE && ctx->geom.n_levels > 1 &&
                          B == ctx->B && B > 0 && ctx->lv[0].D && Y && support_out && coef_out && k_eff_out;
  float *Xh = nullptr;
  if (with_synth && (st = ws_get_t(ctx, ctx->wsp, WS_XH, (size_t)B * ctx->lv[0].N, &Xh)) != CSP_OK) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
  }
  auto once = [&]() -> csp_status {
    if (!with_synth) return csp_solve(ctx, params, Y, B, support_out, coef_out, k_eff_out, stream);
    PatchSet ps;
    CSP_TRY(solve_setup(ctx, params, B, s, ps));
    bool synthesized = false;
    CSP_TRY(solve_core(ctx, ps, ctx->wsp, params, Y, support_out, coef_out, k_eff_out, s, Xh, &synthesized));
    if (!synthesized)
      launch_synth(ctx->gd, ctx->lv[0].D, ctx->lv[0].N, support_out, coef_out, k_eff_out, params->Kmax, Xh, s);
    CSP_CUDA(ctx, cudaGetLastError());
    return CSP_OK;
  };
  // one untimed run (workspace, caches), then the best of three timed ones
  auto time_solve = [&](float *best_of) -> csp_status {
    csp_status r = csp_solve(ctx, params, Y, B, support_out, coef_out, k_eff_out, stream);
    if (r == CSP_OK) r = once();
    *best_of = 3.4e38f;
    for (int rep = 0; rep < 3 && r == CSP_OK; ++rep) {
      cudaEventRecord(e0, s);
      r = once();
      cudaEventRecord(e1, s);
      if (r != CSP_OK) break;
      if (cudaEventSynchronize(e1) != cudaSuccess) return fail(ctx, CSP_ERR_CUDA, "event synchronize failed");
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      *best_of = ms < *best_of ? ms : *best_of;
    }
    return r;
  };
  for (int v = 0; v < CSP_TUNE_VARIANTS && st == CSP_OK; ++v) {
    ctx->restricted_variant = v;
    float ms = 0.f;
    st = time_solve(&ms);
    if (st != CSP_OK) break;
    out->ms[v] = ms;
    if (ms < best_ms) { best_ms = ms; best = v; }
  }
  ctx->restricted_variant = st == CSP_OK ? best : saved;
  out->restricted_variant = ctx->restricted_variant;
  // full-dictionary form: per-iteration kernels (1) against the fused kernel (2)
  const int saved_form = ctx->top_form;
  out->top_level_form = 1;
  out->ms_top[0] = out->ms_top[1] = 0.0;
  const int nl = params->mode == CSP_MODE_PLAIN ? 1 : ctx->geom.n_levels;
  const LevelData &LT = ctx->lv[nl - 1];
  const int Ktop = params->K_patch[nl - 1] ? params->Kmax : params->K[nl - 1];
  const bool fusable = params->precision == CSP_PREC_BF16 && !LT.per_patch && LT.Mp == 64 &&
                       fused_top_supported(LT.M, LT.T, Ktop);
  bool gramable = !LT.per_patch && full_gram_supported(LT.M, LT.T, Ktop);
  for (int ph = 0; ph < kMaxPhases; ++ph) gramable = gramable && (!LT.A[ph] || LT.G[ph]);
  out->ms_top[2] = 0.0;
  for (int form = 1; form <= 3 && st == CSP_OK; ++form) {
    if ((form == 2 && !fusable) || (form == 3 && !gramable)) continue;
    ctx->top_form = form;
    float ms = 0.f;
    st = time_solve(&ms);
    if (st != CSP_OK) break;
    out->ms_top[form - 1] = ms;
    if (ms < out->ms_top[out->top_level_form - 1]) out->top_level_form = form;
  }
  ctx->top_form = st == CSP_OK ? out->top_level_form : saved_form;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return st;
}

csp_status csp_set_work_order(csp_ctx *ctx, int order) {
  if (!ctx) return fail(nullptr, CSP_ERR_INVALID, "ctx is NULL");
  if (order < 0 || order > 1) return fail(ctx, CSP_ERR_INVALID, "unknown work order");
  ctx->work_order = order;
  return CSP_OK;
}

csp_status csp_set_wait_test(csp_ctx *ctx, int on) {
  if (!ctx) return fail(nullptr, CSP_ERR_INVALID, "ctx is NULL");
  ctx->wait_test = on != 0;
  return CSP_OK;
}

csp_status csp_set_top_level_form(csp_ctx *ctx, int form) {
  if (!ctx) return fail(nullptr, CSP_ERR_INVALID, "ctx is NULL");
  if (form < 0 || form > 3) return fail(ctx, CSP_ERR_INVALID, "unknown full-dictionary form");
  ctx->top_form = form;
  return CSP_OK;
}

csp_status csp_set_aggregate_path(csp_ctx *ctx, int path) {
  if (!ctx) return fail(nullptr, CSP_ERR_INVALID, "ctx is NULL");
  if (path < 0 || path > 2) return fail(ctx, CSP_ERR_INVALID, "unknown aggregation path");
  ctx->aggregate_path = path;
  return CSP_OK;
}

csp_status csp_set_kernel_variant(csp_ctx *ctx, int restricted_variant) {
  if (!ctx) return fail(nullptr, CSP_ERR_INVALID, "ctx is NULL");
  if (restricted_variant < 0 || restricted_variant >= CSP_TUNE_VARIANTS)
    return fail(ctx, CSP_ERR_INVALID, "unknown kernel variant");
  ctx->restricted_variant = restricted_variant;
  return CSP_OK;
}

csp_status csp_profile_enable(csp_ctx *ctx, int on) {
  if (!ctx) return fail(nullptr, CSP_ERR_INVALID, "ctx is NULL");
  ctx->prof = on != 0;
  return CSP_OK;
}

csp_status csp_profile_read(csp_ctx *ctx, csp_kernel_time *out, int cap, int *n_out, int reset) {
  if (!ctx) return fail(nullptr, CSP_ERR_INVALID, "ctx is NULL");
  if (cap < 0 || (cap > 0 && !out)) return fail(ctx, CSP_ERR_INVALID, "bad output array");
  DeviceGuard dg(ctx->device);
  CSP_TRY(drain_profile(ctx));
  int n = 0;
  for (int k = 0; k < KK_COUNT; ++k) {
    if (!ctx->launches[k]) continue;
    if (n < cap) {
      std::memset(out[n].name, 0, sizeof(out[n].name));
      std::strncpy(out[n].name, kKernelNames[k], sizeof(out[n].name) - 1);
      out[n].launches = ctx->launches[k];
      out[n].total_ms = ctx->prof_ms[k];
    }
    ++n;
  }
  if (n_out) *n_out = n;
  if (reset)
    for (int k = 0; k < KK_COUNT; ++k) { ctx->launches[k] = 0; ctx->prof_ms[k] = 0.0; }
  return CSP_OK;
}

// ---- Dictionary learning ----

csp_status csp_downsample(csp_ctx *ctx, int level, const float *X, int64_t N, float *X_low, void *stream) {
  if (!ctx) return fail(nullptr, CSP_ERR_INVALID, "ctx is NULL");
  if (!ctx->has_geom) return fail(ctx, CSP_ERR_NOT_READY, "geometry not set");
  if (level < 1 || level >= ctx->geom.n_levels) return fail(ctx, CSP_ERR_INVALID, "level must be in 1 .. n_levels - 1");
  if (N < 0 || N > INT32_MAX) return fail(ctx, CSP_ERR_INVALID, "N out of range");
  if (N > 0 && (!X || !X_low)) return fail(ctx, CSP_ERR_INVALID, "NULL buffer");
  DeviceGuard dg(ctx->device);
  run(ctx, KK_DOWNSAMPLE, (cudaStream_t)stream, N, [&] {
    launch_downsample(ctx->gd, level, X, X_low, N, (cudaStream_t)stream);
  });
  CSP_CUDA(ctx, cudaGetLastError());
  return CSP_OK;
}


csp_status csp_ksvd_update(csp_ctx *ctx, float *D, int M, int T, const float *X, int64_t N, const int32_t *support,
                           float *coef, const int8_t *k_eff, int Kmax, int replace_unused, int approximate,
                           const int32_t *repl_parent, const int32_t *repl_support, int Kc, float *err_out,
                           void *stream) {
  if (!ctx) return fail(nullptr, CSP_ERR_INVALID, "ctx is NULL");
  if (M < 1 || M > 192) return fail(ctx, M < 1 ? CSP_ERR_INVALID : CSP_ERR_UNSUPPORTED, "M must be in 1 .. 192");
  if (T < 1) return fail(ctx, CSP_ERR_INVALID, "T must be positive");
  if (T > 4096) return fail(ctx, CSP_ERR_UNSUPPORTED, "T must be at most 4096");
  if (Kmax < 1 || Kmax > CSP_MAX_K) return fail(ctx, CSP_ERR_INVALID, "Kmax must be in 1 .. CSP_MAX_K");
  if (N < 0 || N * Kmax > INT32_MAX) return fail(ctx, CSP_ERR_INVALID, "N * Kmax must be below 2^31");
  if (replace_unused != 0 && replace_unused != 1) return fail(ctx, CSP_ERR_INVALID, "replace_unused must be 0 or 1");
  if (approximate != 0 && approximate != 1) return fail(ctx, CSP_ERR_INVALID, "approximate must be 0 or 1");
  if ((repl_parent == nullptr) != (repl_support == nullptr))
    return fail(ctx, CSP_ERR_INVALID, "repl_parent and repl_support go together");
  if (repl_support && (Kc < 1 || N * Kc > INT32_MAX)) return fail(ctx, CSP_ERR_INVALID, "Kc out of range");
  if (!D || (N > 0 && (!X || !support || !coef || !k_eff))) return fail(ctx, CSP_ERR_INVALID, "NULL buffer");
  DeviceGuard dg(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  const int n = (int)N;
  int *off = nullptr;
  int32_t *seg = nullptr;
  float *R = nullptr, *rn2 = nullptr, *xn2 = nullptr;
  uint8_t *taken = nullptr;
  const int split = ksvd_owner_split(M, T, approximate != 0);
  CSP_TRY(ksvd_sort(ctx, D, M, T, X, n, support, coef, k_eff, Kmax, split, true, &off, &seg, &R, &rn2, &xn2, s));
  unsigned long long *st = nullptr;
  CSP_TRY(ws_get_t(ctx, ctx->wsp, WS_KS_TAKEN, (size_t)std::max(n, 1), &taken));
  CSP_TRY(ws_get_t(ctx, ctx->wsp, WS_KS_STATS, 2, &st));
  CSP_CUDA(ctx, cudaMemsetAsync(taken, 0, (size_t)std::max(n, 1), s));
  cudaError_t le = cudaSuccess;
  run(ctx, KK_KSVD_SWEEP, s, 1, [&] {
    le = launch_ksvd_sweep(D, M, T, X, n, coef, Kmax, split, off, seg, R, rn2, xn2, taken, replace_unused,
                           repl_parent, repl_support, Kc, st, approximate, s);
  });
  if (le != cudaSuccess) return fail(ctx, CSP_ERR_CUDA, std::string("K-SVD sweep launch: ") + cudaGetErrorString(le));
  if (err_out) {
    if (n > 0) launch_ksvd_sum(rn2, n, err_out, s);
    else CSP_CUDA(ctx, cudaMemsetAsync(err_out, 0, sizeof(float), s));
  }
  unsigned long long hst[2] = {0, 0};
  CSP_CUDA(ctx, cudaMemcpyAsync(hst, st, sizeof(hst), cudaMemcpyDeviceToHost, s));
  CSP_CUDA(ctx, cudaGetLastError());
  CSP_CUDA(ctx, cudaStreamSynchronize(s));
  ctx->ksvd_steps = (int64_t)hst[0];
  ctx->ksvd_replaced = (int64_t)hst[1];
  ctx->ksvd_ranks = split;
  return CSP_OK;
}

csp_status csp_ksvd_stats_get(csp_ctx *ctx, int64_t *power_steps, int64_t *replaced, int64_t *ranks) {
  if (!ctx) return fail(nullptr, CSP_ERR_INVALID, "ctx is NULL");
  if (power_steps) *power_steps = ctx->ksvd_steps;
  if (replaced) *replaced = ctx->ksvd_replaced;
  if (ranks) *ranks = ctx->ksvd_ranks;
  return CSP_OK;
}

csp_status csp_ksvd_init_atoms(csp_ctx *ctx, float *D, int M, int T, const float *X, int64_t N,
                               const int32_t *parent, const int32_t *support_low, const int8_t *keff_low, int Kc,
                               int T_low, const double *u, void *stream) {
  if (!ctx) return fail(nullptr, CSP_ERR_INVALID, "ctx is NULL");
  if (M < 1 || T < 1) return fail(ctx, CSP_ERR_INVALID, "M and T must be positive");
  if (N < 1 || N > INT32_MAX) return fail(ctx, CSP_ERR_INVALID, "N must be in 1 .. 2^31 - 1");
  if (!D || !X || !u) return fail(ctx, CSP_ERR_INVALID, "NULL buffer");
  if (parent && (!support_low || !keff_low || Kc < 1 || Kc > CSP_MAX_K || T_low < 1 || T_low > 32768 ||
                 N * Kc > INT32_MAX))
    return fail(ctx, CSP_ERR_INVALID, "parent needs support_low, keff_low, Kc in 1 .. CSP_MAX_K and T_low");
  DeviceGuard dg(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  int *off = nullptr;
  int32_t *seg = nullptr;
  if (parent) {
    // parent[t] must name a coarse atom: checked on the host copy
    std::vector<int32_t> hp(T);
    CSP_CUDA(ctx, cudaMemcpyAsync(hp.data(), parent, (size_t)T * 4, cudaMemcpyDeviceToHost, s));
    CSP_CUDA(ctx, cudaStreamSynchronize(s));
    for (int t = 0; t < T; ++t)
      if (hp[t] < 0 || hp[t] >= T_low) return fail(ctx, CSP_ERR_INVALID, "parent entry outside [0, T_low)");
    CSP_TRY(ksvd_sort(ctx, nullptr, M, T_low, nullptr, (int)N, support_low, nullptr, keff_low, Kc, 1, false, &off,
                      &seg, nullptr, nullptr, nullptr, s));
  }
  run(ctx, KK_KSVD_SORT, s, 1, [&] { launch_ksvd_init(D, M, T, X, (int)N, parent, off, seg, Kc, u, s); });
  CSP_CUDA(ctx, cudaGetLastError());
  CSP_CUDA(ctx, cudaStreamSynchronize(s));
  return CSP_OK;
}

}  // extern "C"
