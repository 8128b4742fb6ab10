// Serving engine: continuous batching of reconstruction jobs (declared in csp.h).
//
// One scheduler thread per server.  Each loop: (1) retire batches whose CUDA
// event has completed (copy images out, release memory); (2) while a batch
// slot is free, admit queued jobs in arrival order as long as their device
// memory fits the budget, coalescing queued jobs of the same model into one
// batch of at most max_batch_patches patches, and enqueue the batch on the
// slot's stream: per job copy-in and patch extraction into the batch's rows,
// one solve over all patches of the batch (shared launches), per job
// overlap-add and copy-out.  Slots run on separate streams, so batches
// overlap on the device.  Device memory of a batch comes from the
// stream-ordered allocator and is released after the batch completes.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "csp_internal.cuh"

using namespace csp;

namespace {

struct Model {
  csp_ctx *ctx = nullptr;  // resident dictionaries, links, effective dictionaries
  csp_geometry geom{};
  int sense_kind = 0;
  csp_solve_params params{};
  int M = 0, N0 = 0, planes = 0, PP = 0;
  size_t bytes_per_patch = 0;
  size_t pp_bytes = 0;       // coded exposure: per-patch effective dictionaries and norms, all levels
  int64_t pp_slice = 0;      // ... built for at most this many patches at a time
};

struct Job {
  uint64_t id = 0;
  int model = 0, H = 0, W = 0;
  int64_t B = 0, off = 0;
  const float *meas_host = nullptr;
  float *image_host = nullptr;
  std::vector<uint8_t> codes;
  size_t meas_floats = 0, img_floats = 0, bytes = 0;
  double t_submit = 0, t_admit = 0, t_done = 0, t_gpu_done = 0;
  double enqueue_ms = 0, stage_ms[4] = {0, 0, 0, 0}, host_out_ms = 0;  // stages: copy-in, solve, aggregate, copy-out
  double build_ms = 0;  // per-patch operator builds within the solve (coded exposure)
  int batch_jobs = 0;
  int64_t batch_patches = 0;
  csp_status status = CSP_ERR_NOT_READY;
  bool done = false;
  GeomDev gd{};
  float *h_img = nullptr;  // output image in the slot's pinned staging area
};

struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t ev = nullptr;
  cudaEvent_t tev[5] = {};  // timing events at the batch's stage boundaries
  std::vector<cudaEvent_t> bev;  // around each operator-slice build (pairs), created on demand
  int nbev = 0;                  // pairs recorded for the current batch
  Workspace W;              // solver workspace, kept at its high-water mark
  bool busy = false;
  std::vector<Job *> jobs;
  void *dev = nullptr;      // the batch's device memory (stream-ordered allocation)
  uint8_t *host = nullptr;  // pinned staging of the batch's codes, cover ranges, ids and images
  size_t host_cap = 0;
  size_t reserved = 0;
};

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

int tri(int i) { return i * (i + 1) / 2; }

// Bump allocator over one block; offsets are 256-byte aligned.
struct Carve {
  size_t off = 0;
  template <typename T>
  size_t take(size_t count) {
    const size_t o = off;
    off += (count * sizeof(T) + 255) / 256 * 256;
    return o;
  }
};

}  // namespace

struct csp_server {
  int device = 0;
  size_t budget = 0;
  int64_t max_batch = 0;
  csp_ctx *alloc_ctx = nullptr;  // allocator of the slots' workspaces
  std::vector<Model> models;
  std::vector<Slot> slots;
  std::mutex mu;
  std::condition_variable cv, cv_done;
  std::deque<Job *> queue;
  std::map<uint64_t, Job *> jobs;
  size_t in_use = 0;
  uint64_t next_id = 1;
  bool stop = false;
  bool paused = false;
  std::thread th;
  std::string err;
};

namespace {

csp_status sfail(csp_server *srv, csp_status st, const std::string &m) {
  if (srv) srv->err = m;
  return st;
}

// Device bytes one patch of a model needs while its batch is in flight: the
// batch rows, outputs and per-patch operators (the batch allocation) and the
// solver workspace.  Jobs are admitted against this estimate.
size_t model_patch_bytes(const Model &m) {
  const csp_ctx *c = m.ctx;
  const csp_solve_params &p = m.params;
  const int nl = p.mode == CSP_MODE_PLAIN ? 1 : m.geom.n_levels;
  size_t b = 0;
  b += (size_t)m.M * 4 * 2;                 // Y, R
  b += (size_t)((m.M + 63) / 64 * 64) * 2;  // BF16 residual
  b += (size_t)p.Kmax * 8 + 1 + 4 + 16;     // outputs, phase id, candidates
  b += (size_t)m.N0 * 4;                    // synthesized patch
  for (int l = 0; l < nl; ++l) {
    const int K = p.K[l] > 0 ? p.K[l] : p.Kmax;
    b += (size_t)(tri(K) + K) * 4 + (size_t)K * 9 + 1;
    b += (size_t)c->lv[l].N * 4;            // downsampled y (Phi = I) or lifted residual
  }
  if (m.sense_kind == CSP_SENSE_CODED_EXPOSURE) b += (size_t)m.planes * m.PP;  // code block
  return b;
}

// Coded exposure: bytes of one patch's effective dictionary (and norms) of the
// full-dictionary level, plus the candidate rows (and their Gram blocks) of the
// restricted levels.
size_t model_pp_bytes(const Model &m) {
  if (m.sense_kind != CSP_SENSE_CODED_EXPOSURE) return 0;
  const csp_solve_params &p = m.params;
  const int nl = p.mode == CSP_MODE_PLAIN ? 1 : m.geom.n_levels;
  const LevelData &LT = m.ctx->lv[nl - 1];
  size_t b = ((size_t)LT.T * m.M + LT.T) * 4 + 512;
  for (int l = 0; l + 1 < nl; ++l) {
    const int cap = std::max(1, m.ctx->lv[l].max_children * (p.K[l + 1] > 0 ? p.K[l + 1] : p.Kmax));
    b += ((size_t)cap * m.M + cap) * 4 + 32;
    if (m.ctx->restricted_variant >= 2) b += (size_t)cap * cap * 4;  // the candidates' Gram block
  }
  return b;
}

// Enqueue one batch on its slot (called without the server lock).  Returns a
// CUDA error; the jobs of the batch then fail.
cudaError_t launch_batch(csp_server *srv, Slot &sl) {
  Model &m = srv->models[sl.jobs[0]->model];
  cudaStream_t s = sl.stream;
  const bool ce = m.sense_kind == CSP_SENSE_CODED_EXPOSURE;
  const bool bayer = m.sense_kind == CSP_SENSE_BAYER_RGGB;
  const int Kmax = m.params.Kmax;
  const size_t codes_pp = (size_t)m.planes * m.PP;
  int64_t Bt = 0, Bmax = 0;
  for (Job *j : sl.jobs) {
    j->off = Bt;
    Bt += j->B;
    Bmax = std::max(Bmax, j->B);
  }
  // layout of the batch's device block and pinned staging area
  Carve dv, hs;
  const size_t o_Y = dv.take<float>((size_t)Bt * m.M);
  const size_t o_sup = dv.take<int32_t>((size_t)Bt * Kmax);
  const size_t o_coef = dv.take<float>((size_t)Bt * Kmax);
  const size_t o_keff = dv.take<int8_t>((size_t)Bt);
  bool tiled = true;  // fused synthesis + overlap-add (no scratch) for very large jobs only
  for (Job *j : sl.jobs) tiled &= aggregate_use_tiled(0, j->gd, m.N0, Kmax);
  const size_t o_xh = dv.take<float>(tiled ? 0 : (size_t)Bmax * m.N0);
  const size_t o_pc = ce ? dv.take<uint8_t>((size_t)Bt * codes_pp) : 0;
  // coded exposure: the per-patch effective dictionaries of the full-dictionary
  // level exist for one slice of at most m.pp_slice patches at a time
  const int top = m.params.mode == CSP_MODE_PLAIN ? 0 : m.geom.n_levels - 1;
  const int64_t slice = ce ? std::min<int64_t>(Bt, m.pp_slice) : 0;
  const size_t o_A = ce ? dv.take<float>((size_t)slice * m.ctx->lv[top].T * m.ctx->lv[top].M) : 0;
  const size_t o_inv = ce ? dv.take<float>((size_t)slice * m.ctx->lv[top].T) : 0;
  const size_t o_scr = dv.take<unsigned int>(4);
  const size_t o_ids = dv.take<int32_t>((size_t)Bt), h_ids = hs.take<int32_t>((size_t)Bt);
  struct JobLayout { size_t d_meas, d_codes, d_img, d_cov, h_codes, h_img, h_cov; };
  std::vector<JobLayout> jl(sl.jobs.size());
  for (size_t k = 0; k < sl.jobs.size(); ++k) {
    const Job *j = sl.jobs[k];
    const size_t cov = 2 * (size_t)(j->H + j->W);
    jl[k] = {dv.take<float>(j->meas_floats), dv.take<uint8_t>(j->codes.size()), dv.take<float>(j->img_floats),
             dv.take<int32_t>(cov), hs.take<uint8_t>(j->codes.size()), hs.take<float>(j->img_floats),
             hs.take<int32_t>(cov)};
  }
  cudaError_t e;
  if (sl.host_cap < hs.off) {
    if (sl.host) cudaFreeHost(sl.host);
    sl.host = nullptr;
    sl.host_cap = 0;
    if ((e = cudaMallocHost((void **)&sl.host, hs.off)) != cudaSuccess) return e;
    sl.host_cap = hs.off;
  }
  if ((e = cudaMallocAsync(&sl.dev, dv.off, s)) != cudaSuccess) {
    sl.dev = nullptr;
    return e;
  }
  cudaEventRecord(sl.tev[0], s);
  uint8_t *D = static_cast<uint8_t *>(sl.dev), *Hs = sl.host;
  auto dp = [&](size_t o) { return D + o; };
  auto hp = [&](size_t o) { return Hs + o; };
  float *Y = (float *)dp(o_Y), *coef = (float *)dp(o_coef), *xh = (float *)dp(o_xh);
  int32_t *sup = (int32_t *)dp(o_sup);
  int8_t *keff = (int8_t *)dp(o_keff);
  // inputs: staged, copied and extracted job by job
  std::vector<std::vector<int32_t>> per_phase(kMaxPhases);
  std::vector<int32_t> cy, cx;
  for (size_t k = 0; k < sl.jobs.size(); ++k) {
    Job *j = sl.jobs[k];
    const JobLayout &L = jl[k];
    // the measurements straight from the caller's buffer (it stays alive until
    // the job is done): one driver-staged copy instead of a host copy into the
    // pinned area followed by a device copy
    if ((e = cudaMemcpyAsync(dp(L.d_meas), j->meas_host, j->meas_floats * 4, cudaMemcpyHostToDevice, s)) != cudaSuccess)
      return e;
    launch_extract(j->gd, m.sense_kind, 0, (const float *)dp(L.d_meas), Y + j->off * m.M, j->B, m.M, s);
    if (ce) {
      std::memcpy(hp(L.h_codes), j->codes.data(), j->codes.size());
      if ((e = cudaMemcpyAsync(dp(L.d_codes), hp(L.h_codes), j->codes.size(), cudaMemcpyHostToDevice, s)) !=
          cudaSuccess)
        return e;
      launch_patch_codes(j->gd, dp(L.d_codes), j->B, dp(o_pc) + j->off * codes_pp, s);
    }
    if (bayer)
      for (int64_t b = 0; b < j->B; ++b) {
        const int iy = (int)(b / j->gd.nx), ix = (int)(b % j->gd.nx);
        const int oy = std::min(iy * m.geom.stride, j->H - m.geom.P);
        const int ox = std::min(ix * m.geom.stride, j->W - m.geom.P);
        per_phase[2 * (oy & 1) + (ox & 1)].push_back((int32_t)(j->off + b));
      }
    cover_ranges(j->H, m.geom.P, m.geom.stride, j->gd.ny, cy);
    cover_ranges(j->W, m.geom.P, m.geom.stride, j->gd.nx, cx);
    int32_t *hc = (int32_t *)hp(L.h_cov);
    std::memcpy(hc, cy.data(), cy.size() * 4);
    std::memcpy(hc + cy.size(), cx.data(), cx.size() * 4);
    if ((e = cudaMemcpyAsync(dp(L.d_cov), hc, (cy.size() + cx.size()) * 4, cudaMemcpyHostToDevice, s)) != cudaSuccess)
      return e;
    j->h_img = (float *)hp(L.h_img);
  }
  PatchSet ps;
  ps.B = Bt;
  cudaEventRecord(sl.tev[1], s);
  if (bayer) {
    int32_t *ids = (int32_t *)hp(h_ids);
    int64_t n = 0;
    for (int p = 0; p < kMaxPhases; ++p) {
      ps.phase_start[p] = n;
      std::memcpy(ids + n, per_phase[p].data(), per_phase[p].size() * 4);
      n += (int64_t)per_phase[p].size();
    }
    ps.phase_start[kMaxPhases] = n;
    if ((e = cudaMemcpyAsync(dp(o_ids), ids, (size_t)n * 4, cudaMemcpyHostToDevice, s)) != cudaSuccess) return e;
    ps.phase_ids = (const int32_t *)dp(o_ids);
  }
  sl.nbev = 0;
  if (ce) {
    // slice by slice: per-patch operators, then the solve of those patches
    for (int64_t off = 0; off < Bt; off += slice) {
      const int pe = 2 * sl.nbev;  // timing pair of this slice's build
      while ((int)sl.bev.size() < pe + 2) {
        cudaEvent_t ev = nullptr;
        if ((e = cudaEventCreate(&ev)) != cudaSuccess) return e;
        sl.bev.push_back(ev);
      }
      cudaEventRecord(sl.bev[pe], s);
      PatchSet pss;
      pss.B = std::min(slice, Bt - off);
      pss.pcodes = dp(o_pc) + off * codes_pp;
      pss.A_pp[top] = (float *)dp(o_A);
      pss.inv_pp[top] = (float *)dp(o_inv);
      if (build_patch_dicts_for(m.ctx, top, pss.pcodes, pss.B, pss.A_pp[top], pss.inv_pp[top],
                                (unsigned int *)dp(o_scr), s) != CSP_OK)
        return cudaErrorUnknown;
      cudaEventRecord(sl.bev[pe + 1], s);
      ++sl.nbev;
      if (solve_patchset(m.ctx, pss, sl.W, &m.params, Y + off * m.M, sup + off * Kmax, coef + off * Kmax,
                         keff + off, s) != CSP_OK)
        return cudaErrorUnknown;
    }
  } else if (solve_patchset(m.ctx, ps, sl.W, &m.params, Y, sup, coef, keff, s) != CSP_OK) {
    // one solve over every patch of the batch
    return cudaErrorUnknown;
  }
  cudaEventRecord(sl.tev[2], s);
  // outputs: overlap-add job by job, then the copies out
  for (size_t k = 0; k < sl.jobs.size(); ++k) {
    Job *j = sl.jobs[k];
    const JobLayout &L = jl[k];
    const int32_t *dcy = (const int32_t *)dp(L.d_cov), *dcx = dcy + 2 * (size_t)j->H;
    float *img = (float *)dp(L.d_img);
    if (!tiled || !launch_aggregate_tiled(j->gd, m.ctx->lv[0].D, m.N0, sup + j->off * Kmax, coef + j->off * Kmax,
                                          keff + j->off, Kmax, dcy, dcx, img, s))
      launch_aggregate(j->gd, m.ctx->lv[0].D, m.N0, sup + j->off * Kmax, coef + j->off * Kmax, keff + j->off, Kmax,
                       dcy, dcx, xh, img, s);
  }
  cudaEventRecord(sl.tev[3], s);
  for (size_t k = 0; k < sl.jobs.size(); ++k) {
    Job *j = sl.jobs[k];
    if ((e = cudaMemcpyAsync(j->h_img, dp(jl[k].d_img), j->img_floats * 4, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
      return e;
  }
  cudaEventRecord(sl.tev[4], s);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return cudaEventRecord(sl.ev, s);
}

// Host copy of a finished image into the caller's buffer.  One thread copies at
// about 20 GB/s on the host of a GB300, so images above 4 MB are copied by up to
// four threads (chunks of at least 2 MB; the last one by the calling thread).
void host_copy(void *dst, const void *src, size_t bytes) {
  constexpr size_t kMin = size_t(4) << 20, kChunk = size_t(2) << 20;
  const int nt = bytes < kMin ? 1 : (int)std::min<size_t>(4, bytes / kChunk);
  if (nt <= 1) {
    std::memcpy(dst, src, bytes);
    return;
  }
  const size_t part = (bytes / nt + 63) & ~size_t(63);
  std::vector<std::thread> th;
  th.reserve(nt - 1);
  for (int t = 0; t + 1 < nt; ++t) {
    auto copy = [=] {
      std::memcpy(static_cast<char *>(dst) + t * part, static_cast<const char *>(src) + t * part, part);
    };
    try {
      th.emplace_back(copy);
    } catch (...) {  // no thread to be had: this chunk inline
      copy();
    }
  }
  const size_t last = (size_t)(nt - 1) * part;
  std::memcpy(static_cast<char *>(dst) + last, static_cast<const char *>(src) + last, bytes - last);
  for (std::thread &x : th) x.join();
}

// Stage times of a completed batch into its jobs (device events; host times
// were recorded by the scheduler).
void batch_stage_times(Slot &sl) {
  float ms[4] = {0, 0, 0, 0};
  for (int i = 0; i < 4; ++i)
    if (cudaEventElapsedTime(&ms[i], sl.tev[i], sl.tev[i + 1]) != cudaSuccess) {
      cudaGetLastError();
      ms[i] = 0.f;
    }
  float build = 0.f;
  for (int p = 0; p < sl.nbev; ++p) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, sl.bev[2 * p], sl.bev[2 * p + 1]) != cudaSuccess) {
      cudaGetLastError();
      t = 0.f;
    }
    build += t;
  }
  for (Job *j : sl.jobs) {
    for (int i = 0; i < 4; ++i) j->stage_ms[i] = ms[i];
    j->build_ms = build;
  }
}

// Called with the server lock held, after the batch's work has completed
// (or failed and its stream was synchronized) and its images were copied out.
void release_batch(csp_server *srv, Slot &sl, csp_status st) {
  if (sl.dev) cudaFreeAsync(sl.dev, sl.stream);
  sl.dev = nullptr;
  const double t = now_s();
  for (Job *j : sl.jobs) {
    j->h_img = nullptr;
    j->codes.clear();
    j->codes.shrink_to_fit();
    j->t_done = t;
    j->status = st;
    j->done = true;
  }
  sl.jobs.clear();
  srv->in_use -= sl.reserved;
  sl.reserved = 0;
  sl.busy = false;
}

void scheduler(csp_server *srv) {
  cudaSetDevice(srv->device);
  std::unique_lock<std::mutex> lk(srv->mu);
  for (;;) {
    bool progressed = false;
    // (1) retire completed batches
    for (Slot &sl : srv->slots) {
      if (!sl.busy) continue;
      const cudaError_t q = cudaEventQuery(sl.ev);
      if (q == cudaErrorNotReady) continue;
      if (q == cudaSuccess) {
        // images from the pinned staging area to the callers' buffers, without
        // the lock (the slot stays busy and its jobs not done meanwhile).  A
        // device-to-host copy straight into the caller's pageable buffer here
        // was slower for small jobs in the mix: the scheduler thread waited in
        // it while other batches ran.
        const double tg = now_s();
        batch_stage_times(sl);
        lk.unlock();
        for (Job *j : sl.jobs) {
          const double t0 = now_s();
          if (j->image_host && j->h_img) host_copy(j->image_host, j->h_img, j->img_floats * 4);
          j->t_gpu_done = tg;
          j->host_out_ms = 1e3 * (now_s() - t0);
        }
        lk.lock();
      }
      release_batch(srv, sl, q == cudaSuccess ? CSP_OK : CSP_ERR_CUDA);
      if (q != cudaSuccess) srv->err = std::string("batch failed: ") + cudaGetErrorString(q);
      progressed = true;
      srv->cv_done.notify_all();
    }
    // (2) admit and launch
    for (Slot &sl : srv->slots) {
      if (sl.busy || srv->queue.empty() || srv->paused) continue;
      Job *head = srv->queue.front();
      if (srv->in_use + head->bytes > srv->budget) break;  // wait for memory (arrival order)
      sl.jobs.clear();
      sl.jobs.push_back(head);
      srv->queue.pop_front();
      int64_t Bt = head->B;
      size_t res = head->bytes;
      for (auto it = srv->queue.begin(); it != srv->queue.end();) {
        Job *j = *it;
        if (j->model == head->model && Bt + j->B <= srv->max_batch && srv->in_use + res + j->bytes <= srv->budget) {
          sl.jobs.push_back(j);
          Bt += j->B;
          res += j->bytes;
          it = srv->queue.erase(it);
        } else {
          ++it;
        }
      }
      srv->in_use += res;
      sl.reserved = res;
      sl.busy = true;
      const double t = now_s();
      for (Job *j : sl.jobs) {
        j->t_admit = t;
        j->batch_jobs = (int)sl.jobs.size();
        j->batch_patches = Bt;
      }
      lk.unlock();  // submitters may queue while the batch is being enqueued
      const cudaError_t e = launch_batch(srv, sl);
      const double te = 1e3 * (now_s() - t);
      for (Job *j : sl.jobs) j->enqueue_ms = te;
      lk.lock();
      if (e != cudaSuccess) {
        cudaGetLastError();
        cudaStreamSynchronize(sl.stream);
        srv->err = e == cudaErrorUnknown ? std::string("solve failed: ") + srv->models[sl.jobs[0]->model].ctx->err
                                         : std::string("launch failed: ") + cudaGetErrorString(e);
        release_batch(srv, sl, CSP_ERR_CUDA);
        srv->cv_done.notify_all();
      }
      progressed = true;
    }
    bool busy = false;
    for (const Slot &sl : srv->slots) busy |= sl.busy;
    if (srv->stop && srv->queue.empty() && !busy) break;
    if (!progressed) srv->cv.wait_for(lk, std::chrono::microseconds(busy ? 50 : 2000));
  }
}

}  // namespace

extern "C" {

csp_status csp_server_create(csp_server **out, const csp_server_config *cfg) {
  if (!out || !cfg) return CSP_ERR_INVALID;
  *out = nullptr;
  csp_server *srv = new csp_server();
  srv->device = cfg->device;
  srv->budget = cfg->mem_budget_bytes ? cfg->mem_budget_bytes : (size_t(16) << 30);
  srv->max_batch = cfg->max_batch_patches > 0 ? cfg->max_batch_patches : 262144;
  const int ns = cfg->n_streams > 0 ? std::min(cfg->n_streams, 8) : 2;
  if (csp_create(&srv->alloc_ctx, cfg->device, 0) != CSP_OK) {
    delete srv;
    return CSP_ERR_CUDA;
  }
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(cfg->device);
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, cfg->device) == cudaSuccess) {
    uint64_t thr = UINT64_MAX;  // keep freed batch memory cached in the pool
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  srv->slots.resize(ns);
  for (Slot &sl : srv->slots) {
    cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
    cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming);
    for (cudaEvent_t &e : sl.tev) cudaEventCreate(&e);
    sl.W.owner = srv->alloc_ctx;
    void *st = nullptr;
    cudaMalloc(&st, 8 * sizeof(int64_t));
    sl.W.stats_dev = static_cast<int64_t *>(st);
  }
  if (prev >= 0) cudaSetDevice(prev);
  srv->th = std::thread(scheduler, srv);
  *out = srv;
  return CSP_OK;
}

void csp_server_destroy(csp_server *srv) {
  if (!srv) return;
  {
    std::lock_guard<std::mutex> g(srv->mu);
    srv->stop = true;
    srv->paused = false;  // queued jobs run before the server goes away
  }
  srv->cv.notify_all();
  if (srv->th.joinable()) srv->th.join();
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(srv->device);
  for (Slot &sl : srv->slots) {
    cudaStreamSynchronize(sl.stream);
    cudaStreamDestroy(sl.stream);
    cudaEventDestroy(sl.ev);
    for (cudaEvent_t e : sl.tev) cudaEventDestroy(e);
    for (cudaEvent_t e : sl.bev) cudaEventDestroy(e);
    cudaFree(sl.W.stats_dev);
    if (sl.host) cudaFreeHost(sl.host);
    sl.W.ws.clear();  // buffers are owned (and freed) by alloc_ctx
  }
  for (auto &kv : srv->jobs) delete kv.second;
  for (Model &m : srv->models) csp_destroy(m.ctx);
  csp_destroy(srv->alloc_ctx);
  if (prev >= 0) cudaSetDevice(prev);
  delete srv;
}

const char *csp_server_last_error(const csp_server *srv) { return srv ? srv->err.c_str() : ""; }

csp_status csp_server_add_model(csp_server *srv, const csp_model_desc *d, int *model_id) {
  if (!srv) return CSP_ERR_INVALID;
  if (!d || !model_id) return sfail(srv, CSP_ERR_INVALID, "NULL argument");
  if (d->sense_kind != CSP_SENSE_IDENTITY && d->sense_kind != CSP_SENSE_BAYER_RGGB &&
      d->sense_kind != CSP_SENSE_CODED_EXPOSURE)
    return sfail(srv, CSP_ERR_UNSUPPORTED, "serving supports identity, Bayer and coded-exposure models");
  for (int l = 0; l < CSP_MAX_LEVELS; ++l)
    if (d->params.K_patch[l]) return sfail(srv, CSP_ERR_INVALID, "per-patch budgets are not accepted by the server");
  Model m;
  if (csp_create(&m.ctx, srv->device, 0) != CSP_OK) return sfail(srv, CSP_ERR_CUDA, csp_last_error(nullptr));
  auto bad = [&](csp_status st) {
    srv->err = csp_last_error(m.ctx);
    csp_destroy(m.ctx);
    return st;
  };
  // no two-stream pipeline inside a batch: the slots' streams overlap batches,
  // and the model context's second stream would be shared by every slot
  m.ctx->pipeline = false;
  csp_geometry g = d->geom;
  g.H = g.W = g.P;  // a one-patch template: the image extent is per job
  csp_status st = csp_set_geometry(m.ctx, &g);
  if (st != CSP_OK) return bad(st);
  const int planes = g.plane_rows * g.plane_cols;
  std::vector<uint8_t> zero((size_t)planes * g.P * g.P, 0);
  csp_sensing sens{d->sense_kind, 0, d->sense_kind == CSP_SENSE_CODED_EXPOSURE ? zero.data() : nullptr};
  if ((st = csp_set_sensing(m.ctx, &sens)) != CSP_OK) return bad(st);
  for (int l = 0; l < g.n_levels; ++l) {
    const int N = (g.plane_rows / g.factors[l][0]) * (g.plane_cols / g.factors[l][1]) * (g.P / g.factors[l][2]) *
                  (g.P / g.factors[l][3]);
    if ((st = csp_load_dictionary(m.ctx, l, d->D[l], N, d->T[l], 0)) != CSP_OK) return bad(st);
  }
  for (int l = 0; l + 1 < g.n_levels; ++l)  // links are needed by cross-scale models only
    if (d->parent[l] && (st = csp_load_scale_links(m.ctx, l, d->parent[l], d->T[l], 0)) != CSP_OK) return bad(st);
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(srv->device);
  st = prepare_model(m.ctx, nullptr);
  if (st == CSP_OK) st = check_solve_params(m.ctx, &d->params);
  cudaDeviceSynchronize();
  if (prev >= 0) cudaSetDevice(prev);
  if (st != CSP_OK) return bad(st);
  m.geom = d->geom;
  m.sense_kind = d->sense_kind;
  m.params = d->params;
  m.M = m.ctx->M;
  m.N0 = m.ctx->lv[0].N;
  m.planes = planes;
  m.PP = g.P * g.P;
  m.bytes_per_patch = model_patch_bytes(m);
  m.pp_bytes = model_pp_bytes(m);
  if (m.pp_bytes) {
    const size_t slice_bytes = std::max<size_t>(size_t(512) << 20, srv->budget / 4);
    m.pp_slice = std::max<int64_t>(1, (int64_t)(slice_bytes / m.pp_bytes));
  }
  std::lock_guard<std::mutex> lk(srv->mu);
  srv->models.push_back(m);
  *model_id = (int)srv->models.size() - 1;
  return CSP_OK;
}

csp_status csp_server_pause(csp_server *srv, int paused) {
  if (!srv) return CSP_ERR_INVALID;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->paused = paused != 0;
  }
  srv->cv.notify_all();
  return CSP_OK;
}

csp_status csp_submit(csp_server *srv, const csp_job_desc *jd, uint64_t *job_id) {
  if (!srv) return CSP_ERR_INVALID;
  if (!jd || !job_id || !jd->meas_host || !jd->image_host) return sfail(srv, CSP_ERR_INVALID, "NULL argument");
  std::unique_lock<std::mutex> lk(srv->mu);
  if (jd->model_id < 0 || jd->model_id >= (int)srv->models.size()) return sfail(srv, CSP_ERR_INVALID, "unknown model");
  const Model &m = srv->models[jd->model_id];
  if (jd->H < m.geom.P || jd->W < m.geom.P) return sfail(srv, CSP_ERR_INVALID, "image smaller than a patch");
  if (m.sense_kind == CSP_SENSE_CODED_EXPOSURE && !jd->codes_host)
    return sfail(srv, CSP_ERR_INVALID, "coded exposure jobs need codes");
  Job *j = new Job();
  j->model = jd->model_id;
  j->H = jd->H;
  j->W = jd->W;
  j->gd = make_geom_dev(m.geom, jd->H, jd->W);
  j->B = (int64_t)j->gd.nx * j->gd.ny;
  j->meas_host = jd->meas_host;
  j->image_host = jd->image_host;
  const size_t HW = (size_t)jd->H * jd->W;
  j->meas_floats = m.sense_kind == CSP_SENSE_IDENTITY ? (size_t)m.planes * HW : HW;
  j->img_floats = (size_t)m.planes * HW;
  if (m.sense_kind == CSP_SENSE_CODED_EXPOSURE) j->codes.assign(jd->codes_host, jd->codes_host + (size_t)m.planes * HW);
  j->bytes = (size_t)j->B * m.bytes_per_patch + (size_t)std::min<int64_t>(j->B, m.pp_slice) * m.pp_bytes +
             (j->meas_floats + j->img_floats) * 4 + j->codes.size() +
             (size_t)(jd->H + jd->W) * 8 + 4096;
  if (j->bytes > srv->budget) {
    delete j;
    return sfail(srv, CSP_ERR_OOM, "job needs more device memory than the server's budget");
  }
  j->id = srv->next_id++;
  j->t_submit = now_s();
  srv->jobs[j->id] = j;
  srv->queue.push_back(j);
  *job_id = j->id;
  lk.unlock();
  srv->cv.notify_all();
  return CSP_OK;
}

csp_status csp_poll(csp_server *srv, uint64_t job_id, int *done) {
  if (!srv || !done) return CSP_ERR_INVALID;
  std::lock_guard<std::mutex> lk(srv->mu);
  auto it = srv->jobs.find(job_id);
  if (it == srv->jobs.end()) return sfail(srv, CSP_ERR_INVALID, "unknown job");
  *done = it->second->done ? 1 : 0;
  return CSP_OK;
}

csp_status csp_wait(csp_server *srv, uint64_t job_id, int64_t timeout_us) {
  if (!srv) return CSP_ERR_INVALID;
  std::unique_lock<std::mutex> lk(srv->mu);
  auto it = srv->jobs.find(job_id);
  if (it == srv->jobs.end()) return sfail(srv, CSP_ERR_INVALID, "unknown job");
  Job *j = it->second;
  auto pred = [&] { return j->done; };
  if (timeout_us < 0) srv->cv_done.wait(lk, pred);
  else if (!srv->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), pred))
    return sfail(srv, CSP_ERR_TIMEOUT, "job not done within the timeout");
  return j->status;
}

csp_status csp_job_release(csp_server *srv, uint64_t job_id) {
  if (!srv) return CSP_ERR_INVALID;
  std::lock_guard<std::mutex> lk(srv->mu);
  auto it = srv->jobs.find(job_id);
  if (it == srv->jobs.end()) return sfail(srv, CSP_ERR_INVALID, "unknown job");
  if (!it->second->done) return sfail(srv, CSP_ERR_NOT_READY, "job not done");
  delete it->second;
  srv->jobs.erase(it);
  return CSP_OK;
}

csp_status csp_job_info_get(csp_server *srv, uint64_t job_id, csp_job_info *out) {
  if (!srv || !out) return CSP_ERR_INVALID;
  std::lock_guard<std::mutex> lk(srv->mu);
  auto it = srv->jobs.find(job_id);
  if (it == srv->jobs.end()) return sfail(srv, CSP_ERR_INVALID, "unknown job");
  const Job *j = it->second;
  out->patches = j->B;
  out->t_submit = j->t_submit;
  out->t_admit = j->t_admit;
  out->t_done = j->t_done;
  out->batch_jobs = j->batch_jobs;
  out->batch_patches = j->batch_patches;
  out->status = j->status;
  out->enqueue_ms = j->enqueue_ms;
  out->copy_in_ms = j->stage_ms[0];
  out->solve_ms = j->stage_ms[1];
  out->aggregate_ms = j->stage_ms[2];
  out->copy_out_ms = j->stage_ms[3];
  out->t_gpu_done = j->t_gpu_done;
  out->host_out_ms = j->host_out_ms;
  out->build_ms = j->build_ms;
  return CSP_OK;
}

}  // extern "C"
