// Internal declarations of the cross-scale OMP library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <algorithm>
#include <cuda_bf16.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "csp.h"

namespace csp {

// Numerical thresholds of the GPU path.
//  - kTauPivot: the FP32 Cholesky pivot d = ||a||^2 - ||w||^2 is trusted when
//    d / ||a||^2 >= kTauPivot; below it the projection is redone in FP64.
//  - kEpsD64: in FP64, an atom with L_kk <= kEpsD64 * ||a_k|| depends on the
//    chosen atoms and ends the patch.  The FP64 factor comes from the normal
//    equations A_S^T A_S, whose rounding leaves L_kk of an exactly dependent
//    atom near sqrt(eps_64) ||a_k|| (about 1e-8), not near eps ||a_k|| as a QR
//    pivot would; the threshold sits above that floor.  It classifies atoms
//    like the oracle's QR test (|R_kk| <= 1e-10 ||a_k||) except those whose
//    distance from the chosen atoms' span lies between 1e-10 and 3e-7 of
//    their norm.
//  - kEpsR32: the patch ends when ||r||^2 <= kEpsR32 * ||y||^2 (FP32 noise floor).
constexpr float kTauPivot = 1e-3f;
constexpr double kEpsD64 = 3e-7;
constexpr float kEpsR32 = 1e-12f;

constexpr int kMaxPhases = 4;      // Bayer: 4 mosaic phases; other operators: 1
constexpr int kTopP = 4;           // BF16 proxy: candidates re-scored in FP32 per patch

// Device-side description of geometry, shared by the extraction, precompute
// and aggregation kernels.
struct GeomDev {
  int H, W, Ly, Lx, P, stride, nx, ny, n_levels;
  int f[CSP_MAX_LEVELS][4];
};

struct LevelData {
  int N = 0, T = 0;            // patch dimension and atom count of this scale
  float *D = nullptr;          // [T][N] atom-major
  int M = 0;                   // dimension of this level's problem (rows of A)
  int n_phase = 0;             // effective dictionaries held (0 = not prepared)
  float *A[kMaxPhases] = {};   // [T][M]  a_i = Phi U_l d_i  (or d_i for Phi = I)
  float *inv_norm[kMaxPhases] = {};   // [T] 1/||a_i||, or -1 for an ineligible zero column
  __nv_bfloat16 *Abf[kMaxPhases] = {};  // [T][Mp] a_i / ||a_i|| in BF16 (tensor-core proxy)
  int Mp = 0;                  // BF16 row length (M rounded up to 64)
  float *G[kMaxPhases] = {};   // [T][T] Gram matrix A A^T (null when T is too large)
  bool per_patch = false;      // A[0] holds one effective dictionary per patch ([B][T][M])
  __nv_bfloat16 *Dbf = nullptr;  // per-patch mode: BF16 rows of D (unnormalised, padded to Np)
  int Np = 0;                  // per-patch mode: lifted dimension N rounded up to 64
  // Cross-scale map f to the next coarser level (valid when this level < n_levels - 1).
  int32_t *child_off = nullptr;   // [T_{l+1} + 1]
  int32_t *child_idx = nullptr;   // [T] children of each coarse atom, ascending
  int max_children = 0;
  bool links = false;
};

// Grow-only device buffer owned by a context.
struct Buf {
  void *p = nullptr;
  size_t bytes = 0;
};

}  // namespace csp

struct csp_ctx;
namespace csp {
// The patches of one solve.  A context solves its own patch grid; the serving
// engine solves batches that concatenate the patches of several images.
struct PatchSet {
  int64_t B = 0;
  const int32_t *phase_ids = nullptr;       // Bayer: patch ids sorted by mosaic phase (null: one group)
  int64_t phase_start[kMaxPhases + 1] = {};
  const uint8_t *pcodes = nullptr;          // coded exposure: [B][F*P*P] per-patch code blocks
  float *A_pp[CSP_MAX_LEVELS] = {};         // coded exposure: per-patch effective dictionaries [B][T_l][M]
  float *inv_pp[CSP_MAX_LEVELS] = {};       // ... and their inverse column norms [B][T_l]
                                            // (needed for the full-dictionary level only; the
                                            // restricted levels build their candidates' rows)
};

// Grow-only workspace slots and solve counters of one solver instance.
struct Workspace {
  std::vector<Buf> ws;
  int64_t *stats_dev = nullptr;  // 8 counters (see csp_solve_stats)
  csp_ctx *owner = nullptr;      // context whose allocator owns the slots (null: the solving context)
};

enum KernelKind {
  KK_EXTRACT, KK_DOWNSAMPLE, KK_PREP, KK_INIT, KK_PROXY_FP32, KK_PROXY_BF16, KK_UPDATE, KK_RESTRICTED,
  KK_AGGREGATE, KK_LIFT, KK_FUSED, KK_KSVD_SORT, KK_KSVD_SWEEP, KK_FULL_GRAM, KK_COUNT
};
struct ProfRec {
  int kind;
  cudaEvent_t a, b;
};
}  // namespace csp

struct csp_ctx {
  int device = 0;
  size_t budget = 0;  // 0 = unlimited
  size_t held = 0;
  std::string err;
  bool has_geom = false, has_sensing = false, prepared = false;
  csp_geometry geom{};
  csp::GeomDev gd{};
  int sense_kind = -1, shots = 0;
  uint8_t *codes = nullptr;     // device copy of the codes
  float *phi = nullptr;         // dense sensing: device copy of Phi [M][planes * P * P]
  size_t codes_bytes = 0;
  int64_t B = 0;
  int M = 0;
  csp::LevelData lv[CSP_MAX_LEVELS];
  // Patches grouped by Bayer phase (phase = 2 * (oy % 2) + ox % 2).
  int32_t *phase_ids = nullptr;          // [B] patch ids sorted by phase
  int64_t phase_start[csp::kMaxPhases + 1] = {};
  // Aggregation: covering patch-index range of every row / column.
  int32_t *cover_y = nullptr, *cover_x = nullptr;
  // Workspace (grown on demand) and counters of csp_solve.
  csp::Workspace wsp;
  // Coded exposure: per-patch code blocks and per-patch effective dictionaries of this grid.
  uint8_t *pcodes = nullptr;
  float *pp_A[CSP_MAX_LEVELS] = {};
  float *pp_inv[CSP_MAX_LEVELS] = {};
  int64_t last_B = 0;
  cudaStream_t last_stream = nullptr;
  // Host-path buffers of csp_reconstruct_host.
  csp::Buf h_meas, h_Y, h_sup, h_coef, h_keff, h_img;
  // Instrumentation: launches per kernel kind, optional event timing.
  int64_t launches[csp::KK_COUNT] = {};
  double prof_ms[csp::KK_COUNT] = {};
  bool prof = false;
  int restricted_variant = 8;  // restricted-OMP kernel variant (see launch_omp_restricted)
  int aggregate_path = 0;      // 0 automatic, 1 two-pass (synthesis scratch), 2 fused shared-memory tiles
  int work_order = 0;          // 0 patch order on static grids; 1 sorted by budget, restricted levels on a work queue
  int top_form = 0;            // full-dictionary level: 0 automatic, 1 per-iteration kernels, 2 fused kernel,
                               // 3 Gram form (P0 GEMM + Gram-Schmidt iteration over every atom)
  bool wait_test = false;      // test hook: the tensor-core proxy loads no atom tiles (its waits expire)
  // CUDA graphs of the last csp_solve and csp_reconstruct (csp_set_graph_mode):
  // replayed while the call and the context's buffers are unchanged
  // (state_version counts the changes)
  bool graph_mode = false;
  uint64_t state_version = 0;
  struct GraphKey {
    csp_solve_params prm;
    const float *Y;  // csp_solve: the patch vectors; csp_reconstruct: the measurement image
    int64_t B;
    int32_t *sup;
    float *coef;     // csp_reconstruct: the output image
    int8_t *keff;
    uint64_t version;
    int restricted_variant, top_form, wait_test, pipeline, aggregate_path, work_order;
  };
  struct GraphSlot {
    GraphKey key{};
    cudaGraphExec_t exec = nullptr;
  };
  GraphSlot g_solve, g_recon, g_host;  // csp_solve, csp_reconstruct, csp_reconstruct_host (copies included)
  cudaStream_t gstream = nullptr;
  // second stream of the pipelined cross-scale solve (restricted level of the
  // first chunk beside the fused full-dictionary level of the second)
  cudaStream_t aux = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  bool pipeline = true;        // csp_set_pipeline
  bool recon_synth = false;    // the recorded / last csp_reconstruct fused the synthesis
  bool last_synth = false;     // reported by csp_solve_stats_get
  int64_t ksvd_steps = 0, ksvd_replaced = 0, ksvd_ranks = 0;  // last csp_ksvd_update (csp_ksvd_stats_get)
  std::vector<csp::ProfRec> pending;
  std::vector<cudaEvent_t> ev_pool;
  // All device allocations (for the memory budget and destroy).
  std::vector<std::pair<void *, size_t>> allocs;
};

namespace csp {

// ---- kernels (launch wrappers; all enqueue on `s`) ----
void launch_extract(const GeomDev &g, int sense_kind, int shots, const float *meas, float *Y,
                    int64_t B, int M, cudaStream_t s);
void launch_downsample(const GeomDev &g, int level, const float *Y0, float *Yl, int64_t B,
                       cudaStream_t s);
void launch_effective_dict(const GeomDev &g, int sense_kind, int shots, const uint8_t *codes,
                           int level, int phase, const float *D, int T, int N, float *A, int M,
                           cudaStream_t s);
void launch_norms(const float *A, int T, int M, int Mp, float *inv_norm, __nv_bfloat16 *Abf,
                  cudaStream_t s);
// Per-patch sensing (per-pixel coded exposure): A_p = Phi_p U_l D for every patch
// ([B][T][P*P]), inverse row norms over `rows` rows (scratch: one device uint),
// BF16 rows of D (unnormalised, padded to Np), lifted residual z = U_l^T Phi_p^T r.
// Dense Phi: A[i][m] = sum_n Phi[m][n] (U_l d_i)[n] (level-0 patch index n).
void launch_effective_dict_dense(const GeomDev &g, const float *phi, int level, const float *D, int T, int N,
                                 float *A, int M, cudaStream_t s);
void launch_patch_codes(const GeomDev &g, const uint8_t *codes, int64_t B, uint8_t *pc, cudaStream_t s);
// Per-patch effective dictionaries of level l and their inverse row norms in
// one pass per patch (-1 for rows at or below 1e-12 of the largest norm); the
// norms of launch_inv_row_norms.  scratch: 4 bytes.
void launch_effective_dict_pp_norms(const GeomDev &g, const uint8_t *pc, int level, const float *D, int T, int N,
                                    float *A, float *inv, unsigned int *scratch, int64_t B, cudaStream_t s);
void launch_inv_row_norms(const float *A, int64_t rows, int M, float *inv, unsigned int *scratch, cudaStream_t s);
void launch_bf16_rows(const float *D, int T, int N, int Np, __nv_bfloat16 *out, cudaStream_t s);
void launch_lift(const GeomDev &g, const uint8_t *pc, int level, const float *R, int64_t B, float *Z,
                 __nv_bfloat16 *Zbf, int Np, cudaStream_t s);
// Synthesis into Xh ([B][N0] scratch) then per-pixel overlap-add average (2 launches).
// Fused synthesis + overlap-add without scratch; false when no tile shape fits
// shared memory (then use launch_aggregate, which needs B * N0 floats of scratch).
bool aggregate_tiled_fits(const GeomDev &g, int N0, int Kmax);
// Automatic choice: the two-pass path unless its B * N0 scratch exceeds 1 GiB.
inline bool aggregate_use_tiled(int path, const GeomDev &g, int N0, int Kmax) {
  if (path == 1) return false;
  if (path == 2) return aggregate_tiled_fits(g, N0, Kmax);
  return (int64_t)g.nx * g.ny * N0 * 4 > (int64_t(1) << 30) && aggregate_tiled_fits(g, N0, Kmax);
}
bool launch_aggregate_tiled(const GeomDev &g, const float *D0, int N0, const int32_t *support, const float *coef,
                            const int8_t *k_eff, int Kmax, const int32_t *cover_y, const int32_t *cover_x, float *img,
                            cudaStream_t s);
// Set-up of csp_aggregate_noalloc on `dev` (current): looks up its scratch
// array's device address once per device.
void noalloc_setup(int dev);

void launch_aggregate(const GeomDev &g, const float *D0, int N0, const int32_t *support,
                      const float *coef, const int8_t *k_eff, int Kmax, const int32_t *cover_y,
                      const int32_t *cover_x, float *Xh, float *img, cudaStream_t s);
// Copy of n floats with a kernel (16-byte aligned pointers; the source may be a
// page-locked host buffer's device mapping).
void launch_copy_floats(const float *src, float *dst, int64_t n, cudaStream_t s);
// The two passes of launch_aggregate: x_hat_p = D0 alpha_p into Xh [B][N0], then
// the overlap-add of Xh into the image.
void launch_synth(const GeomDev &g, const float *D0, int N0, const int32_t *support, const float *coef,
                  const int8_t *k_eff, int Kmax, float *Xh, cudaStream_t s);
void launch_gather(const GeomDev &g, const float *Xh, int N0, const int32_t *cover_y, const int32_t *cover_x,
                   float *img, cudaStream_t s);

// OMP state of a full-dictionary level, in device memory.
struct OmpState {
  float *R;          // [B][M] residuals
  __nv_bfloat16 *Rbf;// [B][Mp] residuals in BF16 for the tensor-core proxy (may be null)
  float *Lpk;        // [B][Kb*(Kb+1)/2] packed Cholesky factor of A_Omega^T A_Omega
  float *z;          // [B][Kb]  L^{-1} A_Omega^T y
  int32_t *omega;    // [B][ldo] chosen columns
  float *alpha;      // [B][ldo]
  int8_t *k_eff;     // [B]
  uint8_t *flags;    // [B] bit0 done, bit1 FP64 mode
  int32_t *cand;     // [B][kTopP] proxy candidates
  int Kb;            // Cholesky capacity (max budget)
  int ldo;           // row length of omega/alpha
};

// r = y, empty supports; the BF16 residual copy is written in sorted-position
// order (row p holds patch perm[p]; perm == nullptr: identity).
void launch_omp_init(const float *Y, int64_t B, int M, int Mp, const int32_t *perm, OmpState st, cudaStream_t s);
// pinv: optional per-patch inverse norms [B][T] (per-patch Phi), else inv_norm[T].
// keys: optional [B] zeroed scratch; with few patch tiles the atoms are then
// split over several CTAs per tile whose best keys meet there (keys are left zeroed).
int proxy_fp32_splits(int64_t n, int T);
void launch_proxy_fp32(const float *R, int M, const float *A, const float *inv_norm, int T,
                       const int32_t *ids, int64_t n, const int32_t *omega, int ldo,
                       const int8_t *k_eff, const uint8_t *flags, int32_t *cand, const float *pinv,
                       unsigned long long *keys, cudaStream_t s);
bool proxy_bf16_supported(int M, int T);
bool omp_dims_supported(int M);  // M % 4 == 0 and M <= 256
// Tensor-core proxy over the patches at sorted positions row0 .. row0 + n - 1
// (list ids, may be null).  Returns false when a tensor map cannot be built.
// With few patch tiles the atom tiles are split over proxy_bf16_splits(n, T)
// CTAs per patch tile; `part` ([n][splits][4] uint32 scratch) then holds their
// partial top-4 keys until a merge kernel writes cand.  part == null: no split.
int proxy_bf16_splits(int64_t n, int T);
bool launch_proxy_bf16(const __nv_bfloat16 *Rbf, int64_t rows_total, int Mp, const __nv_bfloat16 *Abf, int T,
                       int64_t row0, const int32_t *ids, int64_t n, const uint8_t *flags, int32_t *cand,
                       unsigned long long *err, const float *pinv, uint32_t *part, bool wait_test,
                       cudaStream_t s);
// Fused full-dictionary OMP (k_fused.cu): all Kb iterations of a shared
// dictionary with T <= 256 (multiple of 64) atoms, M <= 64, Kb <= 8, BF16
// tensor-core proxy with FP32 re-score; writes omega/alpha/k_eff directly.
// One launch covers the nph phase groups (host phase_start[nph + 1] gives the
// positions of each group in `ids`; null: one group of n patches, ids may be
// null); A / inv_norm / Abf / gram hold one pointer per phase (a null Gram
// matrix: the Gram columns from the rows).  Returns false when the shape is
// not supported or a tensor map fails.
bool fused_top_supported(int M, int T, int Kb);
// Patches one wave of the fused kernel holds (every SM busy), for this shape.
int64_t fused_wave_patches(int T, int Kb);
bool launch_omp_fused_tc(const float *Y, int M, const float *const *A, const float *const *inv_norm,
                         const __nv_bfloat16 *const *Abf, const float *const *gram, int nph,
                         const int64_t *phase_start, int Mp, int T,
                         const int32_t *ids, int64_t n, const int8_t *Kp, int Kuni, int Kb, int32_t *omega,
                         float *alpha, int ldo, int8_t *k_eff, int64_t *stats, unsigned long long *err,
                         cudaStream_t s);
// Load-wave variants (k_grp.cu): one update iteration; restricted OMP with the Gram-matrix proxy.
// a_pstride / inv_pstride: per-patch strides of A and inv_norm (0: shared by all patches).
void launch_omp_update_wave(const float *Y, int M, const float *A, const float *inv_norm, const int32_t *ids,
                            int64_t n, int64_t rbf_row0, int n_cand, const int8_t *Kp, int Kuni, OmpState st,
                            int64_t *stats, const float *gram, int T, int64_t a_pstride, int64_t inv_pstride,
                            cudaStream_t s);
// width 0, 1, 2: 4, 8, 16 lanes per patch for M <= 64 (doubled per doubling of M, at most 32);
// qr: Gram-Schmidt form (correlations updated per appended atom) instead of p0 - G alpha.
// gpp: per-patch candidate rows (A, inv_norm with strides a_pstride, inv_pstride)
// and Gram blocks ([B][cap][cap], candidate order) instead of the level's shared
// Gram matrix; the Gram-Schmidt form with Q_C in shared memory runs then.
// Shared memory of one CTA of launch_omp_restricted_gram for these arguments
// (pp: per-patch Gram blocks).
size_t restricted_gram_smem(int width, bool qr, int M, int Kb, int cap, bool pp);
bool launch_omp_restricted_gram(int width, bool qr, const float *Y, int M, const float *A, const float *inv_norm,
                                const int32_t *ids, int64_t n, const int32_t *child_off, const int32_t *child_idx,
                                int cap, const int32_t *omega_up, int ldo_up, const int8_t *keff_up,
                                const int8_t *Kp, int Kuni, int Kb, int32_t *omega, float *alpha, int ldo,
                                int8_t *k_eff, int64_t *stats, const float *gram, int T, const float *D0, int N0,
                                float *Xh, cudaStream_t s, unsigned long long *queue = nullptr,
                                const float *gpp = nullptr, int64_t a_pstride = 0, int64_t inv_pstride = 0);
// Gram-Schmidt form with the candidates' state in registers (G = 4, 8 or 16
// lanes per patch); false (nothing launched) when M > 16 G (G = 4) or 8 G,
// Kb > 8 or cap > 8 G.
// With Xh (and D0, N0) it also writes x_hat_p = D0_Omega alpha_p; *synthesized
// tells whether it did.  stage_gram: each patch's Gram block G[C][C] is gathered
// into shared memory at set-up (cap <= 32; false when it does not fit).
bool launch_omp_restricted_reg(int G, const float *Y, int M, const float *A, const float *inv_norm,
                               const int32_t *ids, int64_t n, const int32_t *child_off, const int32_t *child_idx,
                               int cap, const int32_t *omega_up, int ldo_up, const int8_t *keff_up,
                               const int8_t *Kp, int Kuni, int Kb, int32_t *omega, float *alpha, int ldo,
                               int8_t *k_eff, int64_t *stats, const float *gram, int T, const float *D0, int N0,
                               float *Xh, bool *synthesized, cudaStream_t s, bool stage_gram = false);
// Gram matrix A A^T ([T][T] FP32) of an effective dictionary.
void launch_gram(const float *A, int T, int M, float *Gm, cudaStream_t s);
// variant 0: rows from L2 every pass (cooperative groups); 1: rows staged in shared memory;
// 2: proxy from the Gram matrix + exact re-score of the best three (falls back to 0 without gram).
// P0 = Y A^T (FP32) for the patches ids[0..n): P0[b][a] = <a_a, y_b>.
void launch_p0_gemm(const float *Y, int M, const float *A, int T, const int32_t *ids, int64_t n, float *P0,
                    cudaStream_t s);
// Full-dictionary level in the Gram form (form 3), after launch_p0_gemm has
// written P0 = Y A^T: the register-resident Gram-Schmidt iteration with every
// atom a candidate (32 lanes per patch; T <= 256, Kb <= 8, M <= 256); needs the
// level's Gram matrix; P0 holds T floats per patch id.  False when the shape
// does not fit.
bool full_gram_supported(int M, int T, int Kb);
bool launch_omp_full_gram(const float *Y, int M, const float *A, const float *inv_norm, const int32_t *ids, int64_t n,
                          const int8_t *Kp, int Kuni, int Kb, int32_t *omega, float *alpha, int ldo, int8_t *k_eff,
                          int64_t *stats, const float *gram, int T, float *P0, cudaStream_t s);
bool launch_omp_restricted(int variant, const float *Y, int M, const float *A, const float *inv_norm,
                           const int32_t *ids, int64_t n, const int32_t *child_off,
                           const int32_t *child_idx, int cap, const int32_t *omega_up, int ldo_up,
                           const int8_t *keff_up, const int8_t *Kp, int Kuni, int Kb,
                           int32_t *omega, float *alpha, int ldo, int8_t *k_eff, int64_t *stats,
                           const float *gram, int T, int64_t a_pstride, int64_t inv_pstride, bool cpos,
                           cudaStream_t s, const float *D0 = nullptr, int N0 = 0, float *Xh = nullptr,
                           unsigned long long *queue = nullptr, const float *gpp = nullptr);
// Work order: ids[0..n) = the patches 0..n-1 sorted by budget K[b] (int8,
// 0..CSP_MAX_K), largest first; `counts` is scratch of 2 x (CSP_MAX_K + 1) ints.
// Patches of equal budget keep no particular order.
void launch_sort_by_budget(const int8_t *K, int64_t n, int32_t *ids, int *counts, cudaStream_t s);
// Per-pixel coded exposure, restricted level l: rows of the effective
// dictionary for the candidates f(Omega_up) of every patch only, in candidate
// order ([B][cap][M], row c of patch b = a_{cs_c} for that patch's codes) and
// their inverse norms ([B][cap]); read by launch_omp_restricted(cpos = true).
// With Gpp it also writes each patch's Gram block of those rows ([B][cap][cap],
// G[i][j] = <a_i, a_j> for i, j < |C|) and returns true; false when the shape
// has no such form (Gpp then untouched).
bool launch_pp_candidates(const GeomDev &g, const uint8_t *pc, int level, const float *D, int N, int M,
                          const int32_t *omega_up, int ldo_up, const int8_t *keff_up, const int32_t *child_off,
                          const int32_t *child_idx, int cap, int64_t B, float *Ac, float *invc, cudaStream_t s,
                          float *Gpp = nullptr);

// ---- K-SVD dictionary update and initialisation (k_ksvd.cu) ----
// Ranks of the sweep's cluster (16 when such a cluster fits, else 8): the sort
// for the sweep splits every atom's slots by owner rank i mod this count.
int ksvd_owner_split(int M, int T);
// Counting chunks of N signals (rows of the [chunks][T * split] histogram).
int ksvd_chunks(int64_t N);
// Residuals R = X - D S, their squared norms rn2 and those of X (xn2), support
// checks (err bits 1: k_eff range, 2: atom range, 4: repeated atom) and the
// stable counting sort of the support slots by key atom * split + i % split:
// off[T * split + 1], seg[slots] (ascending i within a key).
// R == nullptr: checks and sort only (D, X, coef, rn2, xn2 unused).
void launch_ksvd_sort(const float *D, int M, int T, const float *X, int N, const int32_t *sup, const float *coef,
                      const int8_t *keff, int Kmax, int split, float *R, float *rn2, float *xn2, int *hist, int *off,
                      int32_t *seg, unsigned *err, cudaStream_t s);
// The sequential atom sweep (one thread-block cluster); stats[0] = power-method
// steps, stats[1] = replaced atoms; approx = 1: one alternating step per atom.
cudaError_t launch_ksvd_sweep(float *D, int M, int T, const float *X, int N, float *coef, int Kmax, int split,
                              const int *off, const int32_t *seg, float *R, float *rn2, const float *xn2,
                              uint8_t *taken, int replace, const int32_t *rparent, const int32_t *rsup, int Kc,
                              unsigned long long *stats, int approx, cudaStream_t s);
void launch_ksvd_sum(const float *rn2, int N, float *out, cudaStream_t s);
// Initialisation picks; off == nullptr: from all N signals.
void launch_ksvd_init(float *D, int M, int T, const float *X, int N, const int32_t *parent, const int *off,
                      const int32_t *seg, int Kc, const double *u, cudaStream_t s);

// ---- solve entry points shared by csp_solve and the serving engine (csp_api.cu) ----
csp_status prepare_model(csp_ctx *ctx, cudaStream_t s);                       // effective dictionaries etc.
csp_status check_solve_params(csp_ctx *ctx, const csp_solve_params *prm);   // argument and shape checks
csp_status solve_patchset(csp_ctx *ctx, const PatchSet &ps, Workspace &W, const csp_solve_params *prm,
                          const float *Y, int32_t *support_out, float *coef_out, int8_t *k_eff_out, cudaStream_t s);
csp_status build_patch_dicts_for(csp_ctx *ctx, int level, const uint8_t *pc, int64_t B, float *A_pp, float *inv_pp,
                                 unsigned int *scratch, cudaStream_t s);
// Patch origins helper (host): covering-patch ranges of every row/column for aggregation.
void cover_ranges(int E, int P, int stride, int n, std::vector<int32_t> &out);
int64_t patch_count_1d(int E, int P, int stride);
GeomDev make_geom_dev(const csp_geometry &g, int H, int W);

}  // namespace csp
