#!/usr/bin/env python
"""Throughput of cross-scale (zero-tree) OMP vs plain OMP on one GB300.

Workload: Bayer RGGB demosaicing of a 512x512 RGB synthetic image, 8x8x3
patches at stride 2 (253 x 253 = 64,009 patches), fine dictionary 192 x 1024,
64 measurements per patch, K = 8.  Default link reading "model": the coarse
dictionary (48 x 256) is the box-downsampled fine atoms (each coarse atom the
renormalised 2x2 downsample of its Q = 4 children), so the signal model of
Sec. III-A holds exactly and the two forms reach matched PSNR; the coarse
budget is K_low = 6 (truth codes use 4 coarse atoms per tile; patches that
straddle tiles mix their coarse codes).  One step = the whole hot path on that
image: patch extraction -> solve (cross-scale for the headline value; plain OMP
reported beside it) -> overlap-add aggregation.  After the timing, both forms'
codes of every patch are compared with the FP64 oracle (support-set match,
per-patch relative L2, image PSNR against the oracle's image).

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
on a bounded sample of the same workload instead.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "patches/s cross-scale vs full OMP on one GB300 at matched PSNR; p50/p99 job latency"
UNIT = "patches/s"
L2_FLUSH_BYTES = 512 << 20
FP32_LANES_PER_SM = 128
MAX_SM_GHZ = 2.070


def fp32_peak_tflops(sms: int) -> float:
    """FP32 CUDA-core peak: SMs x FP32 lanes x 2 (FMA) x maximum SM clock."""
    return sms * FP32_LANES_PER_SM * 2 * MAX_SM_GHZ * 1e9 / 1e12


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="bayer")
    ap.add_argument("--links", default="model", choices=["model", "paper", "literal"],
                    help="scale-link reading of the synthetic model (model: Sec. III-A holds exactly; "
                         "paper: coarse atoms = downsampled subset, nearest-parent links; literal: identity links)")
    ap.add_argument("--accuracy-sample", type=int, default=70000,
                    help="largest number of patches compared with the oracle per form (a seeded sample above it)")
    ap.add_argument("--precision", default="bf16", choices=["fp32", "bf16"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--serving-only", action="store_true", help="run the serving measurement alone (no headline)")
    ap.add_argument("--variant", type=int, default=None,
                    help="pin the restricted-solver variant (0-9) instead of autotuning (profiling runs)")
    ap.add_argument("--sweep-q", default=None,
                    help="comma-separated children-per-coarse-atom counts Q (e.g. 2,4,8,16): instead of the "
                         "headline, time cross-scale and plain OMP and report PSNR for each Q (the link-size "
                         "trade-off of Sec. III-E / Fig. 4 on synthetic data)")
    ap.add_argument("--ksvd", action="store_true",
                    help="instead of the headline, time the modified K-SVD (Sec. III, learning cross-scale "
                         "models) on a synthetic training set shaped like --workload: one Step-2 iteration "
                         "(zero-tree coding + dictionary-update sweep) against one plain K-SVD iteration")
    ap.add_argument("--ksvd-signals", type=int, default=65536, help="training signals of --ksvd")
    ap.add_argument("--uneven", action="store_true",
                    help="instead of the headline, time the light-field workload with per-patch budgets K in [8, 20] "
                         "with the work order off and on (sorted by budget, persistent warps on a work queue)")
    ap.add_argument("--no-pipeline", action="store_true",
                    help="one stream throughout (csp_set_pipeline off; profiling runs)")
    ap.add_argument("--top-form", type=int, default=None, choices=[1, 2, 3],
                    help="pin the full-dictionary form (1 per-iteration, 2 fused, 3 Gram) with --variant (profiling runs)")
    return ap.parse_args()


def workload_config(w, args):
    g = w.geometry
    return {
        "workload": f"{w.name}_{w.sensing.kind}_{g.H}x{g.W}x{g.planes}_patch{g.P}_stride{g.stride}",
        "patches": int(w.n_patches),
        "dictionaries": [f"{d.shape[1]}x{d.shape[0]}" for d in w.dicts],
        "K": [int(k[0]) for k in w.K_levels],
        "links": args.links,
        "reading": {"model": "coarse atoms = downsampled children (Sec. III-A exact), block links, "
                             "sign-coherent codes; coarse budgets 1.5x the truth's",
                    "paper": "coarse atoms = downsampled subset of T/4 fine atoms, nearest-parent links",
                    "literal": "coarse atoms = every downsampled fine atom, identity links"}[args.links],
        "seed": int(w.seed),
        "l2": "flushed between steps (512 MiB write)",
        "parallelism": "replicas (one image per GPU)",
    }


# ----------------------------------------------------------------------------
# clocks sampled during the timed region
# ----------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.lines = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.idx)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------
# multi-rank bookkeeping (one replica per GPU; no collective on the data path)
# ----------------------------------------------------------------------------
def dist_env():
    """(world, rank, local_rank) from the torchrun environment (1, 0, 0 without it)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(value: float, world: int, device=None) -> float:
    """The slowest rank's time: an all-reduce MAX (any backend; CPU tensors with gloo)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, patches_per_rank: int, steps: int, total_seconds: float) -> float:
    """Whole-job patches/s: every rank processes its own image per step (weak scaling),
    timed by the slowest rank."""
    return world * patches_per_rank * steps / total_seconds


# ----------------------------------------------------------------------------
# roofline bookkeeping
# ----------------------------------------------------------------------------
# Sources that define, instantiate or launch each kernel kind whose DRAM traffic
# may be quoted (a capture stays valid while these files are unchanged).
KERNEL_SOURCES = {
    "restricted": ("k_grp.cu", "k_omp.cu", "grp_common.cuh", "csp_internal.cuh"),
    "omp_fused": ("k_fused.cu", "tc_common.cuh", "csp_internal.cuh"),
    "proxy_bf16": ("k_proxy_tc.cu", "tc_common.cuh", "csp_internal.cuh"),
}


def kernel_source_sha(kernel: str = ""):
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1511_05174_gb300", "csrc")
    files = KERNEL_SOURCES.get(kernel) or sorted(f for f in os.listdir(csrc) if f.endswith((".cu", ".cuh")))
    for f in files:
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def read_traffic(kernel: str, workload: str):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on the
    current kernel sources (profiles/traffic_<kernel>_<workload>.txt: key: value)."""
    path = os.path.join(ROOT, "profiles", f"traffic_{kernel}_{workload}.txt")
    if not os.path.exists(path):
        return None
    kv = {}
    for line in open(path):
        if ":" in line and not line.startswith("#"):
            k, v = line.split(":", 1)
            kv[k.strip()] = v.strip()
    if kv.get("source_sha") != kernel_source_sha(kernel):
        return None
    try:
        return float(kv["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def algorithmic(kind, w, prof_launches, stats, B, steps, M):
    """Algorithmic work of one launch of `kind` on this workload: (amount, unit, bound).
    `stats` are the solve statistics of one step; M the measurements per patch."""
    g = w.geometry
    top = w.dicts[-1].shape[0]
    per_patch_phi = w.sensing.kind == "coded_exposure"
    if kind in ("proxy_fp32", "proxy_bf16"):
        cross = bool(prof_launches.get("restricted"))
        D = w.dicts[-1] if cross else w.dicts[0]
        T = D.shape[0]
        dim = D.shape[1] if per_patch_phi else M  # per-pixel Phi: the lifted proxy runs at the atom dimension
        if kind == "proxy_bf16":
            dim = (dim + 63) // 64 * 64
        # one launch per iteration and Bayer phase group: the step's proxy work
        # (every patch, every iteration) over the step's launches
        iters = int(np.max(w.K_levels[-1 if cross else 0]))
        launches = max(prof_launches[kind][0] / steps, 1.0)
        return 2.0 * dim * T * B * iters / launches, "TFLOP/s", ("tensor" if kind == "proxy_bf16" else "alu")
    if kind == "omp_fused":
        # the tensor-core proxy of every iteration of the full-dictionary level (coarsest level
        # in cross-scale mode): 2 Mp T flops per patch per iteration, Mp = M padded to 64
        cross = bool(prof_launches.get("restricted"))
        lvl = -1 if cross else 0
        T = w.dicts[lvl].shape[0]
        dim = (M + 63) // 64 * 64
        iters = int(np.max(w.K_levels[lvl]))
        launches = max(prof_launches[kind][0] / steps, 1.0)
        return 2.0 * dim * T * B * iters / launches, "TFLOP/s", "tensor"
    if kind == "restricted":
        per_step = max(prof_launches.get("restricted", (1,))[0] / steps, 1.0)
        flops = 2.0 * M * stats.get("restricted_scores", 0)
        if stats.get("synthesized"):  # x_hat_p = D0 alpha_p written by the finest level: 2 N0 K per patch
            flops += 2.0 * w.dicts[0].shape[1] * float(np.sum(w.K_levels[0]))
        return flops / per_step, "TFLOP/s", "alu"
    if kind == "omp_update":
        # y, r read and r written, 4 B each, per patch
        return 3.0 * 4 * M * B, "GB/s", "hbm"
    if kind == "aggregate":
        K = int(np.max(w.K_levels[0]))
        return 4.0 * g.planes * g.H * g.W + B * (K * 8 + 1), "GB/s", "hbm"
    if kind == "extract":
        return 4.0 * B * M + 4.0 * w.meas.size, "GB/s", "hbm"
    if kind == "full_gram":
        # the Gram form of the full-dictionary level: per patch and appended atom k
        # (k = 0 .. K-1) a new column of Q over all T atoms (T k FMAs) and the
        # correlation update (T FMAs): T K (K + 1) flops per patch
        cross = bool(prof_launches.get("restricted"))
        lvl = -1 if cross else 0
        T = w.dicts[lvl].shape[0]
        K = int(np.max(w.K_levels[lvl]))
        launches = max(prof_launches[kind][0] / steps, 1.0)
        return float(T) * K * (K + 1) * B / launches, "TFLOP/s", "alu"
    return None, None, None


# ----------------------------------------------------------------------------
# reference arm: the FP64 CPU oracle on a bounded sample
# ----------------------------------------------------------------------------
def run_reference(args):
    import oracle
    import synthetic

    world, rank, _ = dist_env()
    if rank != 0:
        return  # the CPU oracle runs once, on rank 0
    w = synthetic.make_workload(args.workload, links=args.links)
    Y = oracle.extract_patches(w)
    cores = oracle.num_threads()
    sample = int(os.environ.get("CSP_REF_SAMPLE", "2048"))
    rng = np.random.default_rng(1)
    times = []
    for i in range(args.warmup + args.steps):
        sel = np.sort(rng.choice(w.n_patches, min(sample, w.n_patches), replace=False))
        t0 = time.perf_counter()
        oracle.cross_scale_omp(w, Y=Y, patches=sel, nthreads=cores)
        t1 = time.perf_counter()
        if i >= args.warmup:
            times.append(t1 - t0)
    total = sum(times)
    value = sample * len(times) / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {**workload_config(w, args), "form": "cross_scale"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{sample} random patches of the {w.n_patches}-patch image per step, "
                                   "extraction excluded, cross-scale solve"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def cpu_baseline(w, gpu_codes=None, sample_cap=70000, seconds=6.0):
    """The oracle as it stands on the host cores: both forms on all threads over
    the whole image (a seeded sample of `sample_cap` patches when the image has
    more), cross-scale on one thread over a sample sized to about `seconds`.
    The oracle's codes of the all-thread runs are then compared with the GPU's
    (`gpu_codes`, see `accuracy`).  Returns (cpu_baseline dict, accuracy dict)."""
    import oracle

    cores = oracle.num_threads()
    Y = oracle.extract_patches(w)
    B = w.n_patches
    sample = None if B <= sample_cap else np.sort(np.random.default_rng(3).choice(B, sample_cap, replace=False))
    n_all = B if sample is None else len(sample)
    runs = {}
    for mode, fn in (("cross_scale", oracle.cross_scale_omp), ("plain", oracle.plain_omp)):
        t0 = time.perf_counter()
        res = fn(w, Y=Y, patches=sample, nthreads=cores)
        runs[mode] = (n_all / (time.perf_counter() - t0), res)
    rng = np.random.default_rng(2)
    sel = np.sort(rng.choice(B, min(64, B), replace=False))
    t0 = time.perf_counter()
    oracle.cross_scale_omp(w, Y=Y, patches=sel, nthreads=1)
    dt = time.perf_counter() - t0
    n1 = int(min(B, max(len(sel), len(sel) * seconds / max(dt, 1e-6))))
    sel = np.sort(rng.choice(B, n1, replace=False))
    t0 = time.perf_counter()
    oracle.cross_scale_omp(w, Y=Y, patches=sel, nthreads=1)
    one = n1 / (time.perf_counter() - t0)
    what = "every patch of the image" if sample is None else f"{n_all} seeded random patches"
    cpu = {"value": runs["cross_scale"][0], "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"{what} (cross-scale solve; extraction and aggregation excluded); plain OMP on the same "
                     f"patches: {runs['plain'][0]:.1f} patches/s",
           "plain": {"value": runs["plain"][0], "unit": UNIT, "cores": cores},
           "one_core": {"value": one, "unit": UNIT, "cores": 1, "sample": f"{n1} random patches, cross-scale solve"}}
    acc = None
    if gpu_codes:
        acc = accuracy(w, gpu_codes, {m: runs[m][1] for m in runs}, sample)
    return cpu, acc


def _synth(D0, sup, coef, keff):
    """x_hat_p = D0_|Omega alpha_p for every patch (FP64), [B, N0]."""
    D = D0.astype(np.float64)
    B, Km = sup.shape
    out = np.zeros((B, D.shape[1]))
    valid = np.arange(Km)[None, :] < np.asarray(keff).reshape(-1, 1)
    for b0 in range(0, B, 4096):
        v = valid[b0:b0 + 4096]
        idx = np.where(v, sup[b0:b0 + 4096], 0)
        a = np.where(v, coef[b0:b0 + 4096].astype(np.float64), 0.0)
        out[b0:b0 + 4096] = np.einsum("bk,bkn->bn", a, D[idx])
    return out


def accuracy(w, results, oracle_codes, sample):
    """Error of each form's GPU result against the FP64 oracle on the same
    patches: support-set match rate (and in selection order), the relative L2
    of x_hat_p = D_|Omega alpha_p per patch (over matching patches and over all),
    and the GPU image's PSNR beside the oracle image's.  `results[mode]` =
    (sup, coef, keff, image) of the GPU, `oracle_codes[mode]` = the oracle's
    (omega, alpha, k_eff, rsq) on the patches `sample` (None: all)."""
    import oracle

    B = w.n_patches
    sel = np.arange(B) if sample is None else sample
    out = {}
    for mode in ("cross_scale", "plain"):
        sup, coef, keff, img = results[mode]
        o, a, k, _ = oracle_codes[mode]
        sup, coef, keff = sup[sel], coef[sel], keff[sel].astype(np.int64)
        km = max(o.shape[1], sup.shape[1])
        same_k = keff == k
        set_match = np.array([same_k[i] and set(sup[i, :keff[i]].tolist()) == set(o[i, :k[i]].tolist())
                              for i in range(len(sel))])
        ord_match = np.array([same_k[i] and list(sup[i, :keff[i]]) == list(o[i, :k[i]]) for i in range(len(sel))])
        xg = _synth(w.dicts[0], sup, coef, keff)
        xo = _synth(w.dicts[0], np.pad(o, ((0, 0), (0, km - o.shape[1])), constant_values=0)[:, :km],
                    np.pad(a, ((0, 0), (0, km - a.shape[1]))), k)
        rel = np.linalg.norm(xg - xo, axis=1) / np.maximum(np.linalg.norm(xo, axis=1), 1e-30)
        row = {"patches_compared": int(len(sel)), "support_match": float(set_match.mean()),
               "support_match_ordered": float(ord_match.mean()),
               "rel_l2_max_on_match": float(rel[set_match].max()) if set_match.any() else None,
               "rel_l2_median_all": float(np.median(rel)), "rel_l2_max_all": float(rel.max()),
               "psnr_db": oracle.psnr(w.truth, img)}
        if sample is None:
            row["oracle_psnr_db"] = oracle.psnr(w.truth, oracle.aggregate(w, o, a, k))
            row["psnr_minus_oracle_db"] = row["psnr_db"] - row["oracle_psnr_db"]
        out[mode] = row
    if sample is None:
        out["oracle_psnr_gap_plain_minus_cross_db"] = out["plain"]["oracle_psnr_db"] - out["cross_scale"]["oracle_psnr_db"]
    out["gpu_psnr_gap_plain_minus_cross_db"] = out["plain"]["psnr_db"] - out["cross_scale"]["psnr_db"]
    out["bar"] = "support sets identical on >= 99.9 % of patches, rel L2 <= 1e-4 on those; PSNR within 0.05 dB"
    return out


# ----------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------
SERVING_RATES = {"cross_scale": (5, 10, 20, 30, 50, 100, 200), "plain": (1, 2, 5, 10)}  # offered jobs/s
SERVING_JOBS = {"cross_scale": 48, "plain": 12}  # jobs per offered rate


def serving_pool(kinds=("denoise", "bayer", "video"), per_kind=4, seed=0, lo=128, hi=2048, links="model"):
    """Distinct jobs of each kind (own seed, own coded-exposure mask), sides
    uniform in [lo, hi] (multiples of 8); one model (dictionaries and links)
    per kind.  Returns [(kind, workload)]."""
    import synthetic
    rng = np.random.default_rng(seed)
    pool = []
    for kind in kinds:
        for i in range(per_kind):
            side = int(rng.integers(lo // 8, hi // 8 + 1)) * 8
            pool.append((kind, synthetic.make_workload(kind, seed=1000 + 10 * i + len(pool), H=side, W=side,
                                                       dict_seed=0, links=links)))
    return pool


def standalone_job_ms(device, pool, mode, precision, reps=3, rebuild=False):
    """Device time of each pool job alone through csp_reconstruct (device
    buffers, default kernel choices as the server's models use them): the
    extraction, the solve and the overlap-add, best of `reps`, CUDA events.
    With `rebuild`, a per-pixel-Phi job (coded exposure) has its sensing codes
    set again before every repetition, so that its per-patch operator of the
    full-dictionary level is rebuilt inside the timed region, as it is for a
    served job that brings its own codes.  Returns [ms] in pool order."""
    import torch
    from paper_1511_05174_gb300.context import Context

    from paper_1511_05174_gb300 import _binding as binding

    dev = torch.device("cuda", device)
    out = []
    for kind, w in pool:
        ctx = Context(device, mem_budget_bytes=48 << 30)  # whole-image per-patch operators beyond it: skipped
        ctx.load_workload(w)
        K = [int(k[0]) for k in w.K_levels]
        Km = K if mode == "cross_scale" else K[:1]
        meas = torch.from_numpy(np.ascontiguousarray(w.meas)).to(dev)
        img = torch.empty((w.geometry.planes, w.geometry.H, w.geometry.W), dtype=torch.float32, device=dev)
        try:
            ctx.reconstruct(meas, img, mode, precision, K=Km, Kmax=K[0])
        except binding.CspError as e:
            if e.status != binding.CSP_ERR_OOM:
                raise
            out.append(None)
            ctx.close()
            continue
        best = float("inf")
        for _ in range(reps):
            if rebuild and w.sensing.kind == "coded_exposure":
                ctx.set_sensing(w.sensing.kind, w.sensing.codes)
                torch.cuda.synchronize()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record()
            ctx.reconstruct(meas, img, mode, precision, K=Km, Kmax=K[0])
            ev1.record()
            torch.cuda.synchronize()
            best = min(best, ev0.elapsed_time(ev1))
        out.append(best)
        ctx.close()
        del meas, img
        torch.cuda.empty_cache()
    return out


def standalone_summary(device, pool, mode, precision):
    """Each pool job alone, with the per-patch operators cached in the context
    and rebuilt per job; jobs/s = jobs that fit / their summed device time."""
    out = {}
    for key, rebuild in (("standalone", False), ("standalone_with_build", True)):
        alone = standalone_job_ms(device, pool, mode, precision, rebuild=rebuild)
        fit = [t for t in alone if t is not None]
        out[key + "_device_ms"] = [None if t is None else round(t, 3) for t in alone]
        out[key + "_jobs_per_s"] = len(fit) / (sum(fit) / 1e3) if fit else None
    return out


def serving_bench(args, device, pool, mode, jobs_per_rate):
    """Serving engine on this GPU: continuous batching of a Poisson stream of
    jobs drawn uniformly from `pool`, at each offered rate in SERVING_RATES.
    Host buffers in and out; per job the latency is done - submitted.
    Returns a dict for the JSON line."""
    from paper_1511_05174_gb300.server import Server

    srv = Server(device, mem_budget_bytes=64 << 30, n_streams=2)
    try:
        models = {}
        for kind, w in pool:
            if kind not in models:
                models[kind] = srv.add_workload_model(w, mode, args.precision)
        outs = [np.empty((w.geometry.planes, w.geometry.H, w.geometry.W), np.float32) for _, w in pool]
        meas = [np.ascontiguousarray(w.meas, dtype=np.float32) for _, w in pool]

        def run(order, gaps=None):
            ids = []
            t_next = time.perf_counter()
            for n, i in enumerate(order):
                if gaps is not None:
                    t_next += gaps[n]
                    while time.perf_counter() < t_next:
                        pass
                kind, w = pool[i]
                codes = w.sensing.codes if w.sensing.kind == "coded_exposure" else None
                ids.append(srv.submit(models[kind], meas[i], w.geometry.H, w.geometry.W, codes=codes, out=outs[i]))
            infos = []
            for j in ids:
                st = srv.wait(j, 600)
                if st != 0:
                    raise RuntimeError(f"serving job failed with status {st}")
                infos.append(srv.info(j))
                srv.release(j)
            return infos

        run(range(len(pool)))  # warm-up: every job once (workspaces, pools, staging)
        rng = np.random.default_rng(1)
        rates = []
        for rate in SERVING_RATES[mode]:
            order = rng.integers(0, len(pool), size=jobs_per_rate)
            infos = run(order, rng.exponential(1.0 / rate, size=jobs_per_rate))
            lat = np.array([i["t_done"] - i["t_submit"] for i in infos]) * 1e3
            span = max(i["t_done"] for i in infos) - min(i["t_submit"] for i in infos)
            patches = sum(i["patches"] for i in infos)

            def med(f):
                return float(np.median([f(i) for i in infos]))
            stages = {  # medians over the jobs (device stages are per batch)
                "wait_ms": med(lambda i: 1e3 * (i["t_admit"] - i["t_submit"])),
                "enqueue_ms": med(lambda i: i["enqueue_ms"]),
                "copy_in_ms": med(lambda i: i["copy_in_ms"]), "solve_ms": med(lambda i: i["solve_ms"]),
                "operator_build_ms": med(lambda i: i["build_ms"]),
                "aggregate_ms": med(lambda i: i["aggregate_ms"]), "copy_out_ms": med(lambda i: i["copy_out_ms"]),
                "admit_to_gpu_done_ms": med(lambda i: 1e3 * (i["t_gpu_done"] - i["t_admit"])),
                "host_out_ms": med(lambda i: i["host_out_ms"]),
                "device_ms_per_job": float(np.sum([(i["copy_in_ms"] + i["solve_ms"] + i["aggregate_ms"]
                                                    + i["copy_out_ms"]) / max(i["batch_jobs"], 1) for i in infos])
                                           / len(infos)),
            }
            by_kind = {}
            for kind in sorted({k for k, _ in pool}):
                sel = [inf for inf, i in zip(infos, order) if pool[i][0] == kind]
                if not sel:
                    continue
                by_kind[kind] = {
                    "jobs": len(sel),
                    "latency_ms_median": float(np.median([1e3 * (i["t_done"] - i["t_submit"]) for i in sel])),
                    "solve_ms_median": float(np.median([i["solve_ms"] for i in sel])),
                    "operator_build_ms_median": float(np.median([i["build_ms"] for i in sel])),
                    "copy_in_ms_median": float(np.median([i["copy_in_ms"] for i in sel])),
                    "aggregate_ms_median": float(np.median([i["aggregate_ms"] for i in sel])),
                    "copy_out_ms_median": float(np.median([i["copy_out_ms"] for i in sel])),
                    "admit_to_gpu_done_ms_median": float(np.median([1e3 * (i["t_gpu_done"] - i["t_admit"])
                                                                    for i in sel])),
                    "mean_batch_jobs": float(np.mean([i["batch_jobs"] for i in sel]))}
            rates.append({"offered_jobs_per_s": rate, "jobs": len(infos), "value": patches / span, "unit": UNIT,
                          "jobs_per_s": len(infos) / span, "latency_ms_p50": float(np.percentile(lat, 50)),
                          "latency_ms_p99": float(np.percentile(lat, 99)),
                          "mean_batch_jobs": float(np.mean([i["batch_jobs"] for i in infos])),
                          "stages_median": stages, "by_kind": by_kind})
        return rates
    finally:
        srv.close()


def q_sweep(args):
    """Cross-scale vs plain OMP for several children-per-coarse-atom counts Q on
    the synthetic workload (the coarse dictionary has T/Q atoms): patches/s of
    csp_reconstruct (graph-replayed, L2 flushed between steps) and PSNR against
    the synthetic ground truth.  One JSON line."""
    import torch
    import synthetic
    from paper_1511_05174_gb300.context import Context

    dev = torch.device("cuda", 0)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    rows = []
    for Q in [int(q) for q in args.sweep_q.split(",")]:
        w = synthetic.make_workload(args.workload, links=args.links, Q=Q)
        ctx = Context(0)
        ctx.load_workload(w)
        K = [int(k[0]) for k in w.K_levels]
        meas_d = torch.from_numpy(w.meas).to(dev)
        img = torch.empty((w.geometry.planes, w.geometry.H, w.geometry.W), dtype=torch.float32, device=dev)
        Y = ctx.extract(meas_d)
        ctx.autotune(Y, "cross_scale", args.precision, K=K, Kmax=K[0])
        ctx.set_graph_mode(True)
        row = {"Q": Q, "coarse_atoms": int(w.dicts[-1].shape[0]), "patches": int(w.n_patches)}
        for mode in ("cross_scale", "plain"):
            Km = K if mode == "cross_scale" else K[:1]
            for _ in range(max(args.warmup, 3)):
                ctx.reconstruct(meas_d, img, mode, args.precision, K=Km, Kmax=K[0])
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(args.steps)]
            torch.cuda.synchronize()
            for a, b in ev:
                flush.zero_()
                a.record()
                ctx.reconstruct(meas_d, img, mode, args.precision, K=Km, Kmax=K[0])
                b.record()
            torch.cuda.synchronize()
            ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
            est = img.double().cpu().numpy()
            mse = float(np.mean((w.truth - est) ** 2))
            peak = float(w.truth.max() - w.truth.min())
            row[mode] = {"patches_per_s": w.n_patches / (ms / 1e3), "ms_per_image": ms,
                         "psnr_db": 10 * np.log10(peak * peak / mse)}
        row["speedup"] = row["cross_scale"]["patches_per_s"] / row["plain"]["patches_per_s"]
        rows.append(row)
        ctx.close()
    print(json.dumps({"sweep": "children per coarse atom (Q)", "workload": w.name, "precision": args.precision,
                      "data": "synthetic (seeded)", "l2": "flushed between steps", "rows": rows}))


def ksvd_bench(args):
    """Modified K-SVD on a seeded training set with the patch shape, atom counts
    and sparsities of the workload: time of one Step-2 iteration (zero-tree
    coding of every signal, csp_solve cross-scale, then one dictionary-update
    sweep, csp_ksvd_update) and of one plain K-SVD iteration (plain OMP over all
    fine atoms, then the same sweep) on the same dictionaries, CUDA events,
    FP32 coding.  The sweep visits the atoms in order inside one thread-block
    cluster; its roofline is FP32 FMA work (Gram matrices, power steps,
    residual updates) against the peak of the cluster's SMs.  The oracle's
    sweep (FP64 CPU, the same inputs) is timed once beside it.  One JSON line."""
    import torch
    import synthetic
    import oracle  # noqa: F401  (the CPU baseline below)
    from oracle import ksvd as oksvd
    from paper_1511_05174_gb300.context import Context
    from paper_1511_05174_gb300.ksvd import ModifiedKSVD

    dev = torch.device("cuda", 0)
    ts = synthetic.make_training_set(args.workload, args.ksvd_signals, seed=0)
    g = ts.geometry
    mk = ModifiedKSVD(g.P, g.plane_grid, g.level_factors, ts.parents[0], ts.K_high, ts.K_low)
    X = torch.from_numpy(ts.X).to(dev)
    t0 = time.perf_counter()
    D_low, D_high, sup_low, keff_low, el, eh = mk.fit(X, ts.u_low, ts.u_high, 2, 2)
    torch.cuda.synchronize()
    fit_s = time.perf_counter() - t0
    plain = Context(0)
    plain.set_geometry(g.P, g.P, g.plane_grid, g.P, g.P, [(1, 1, 1, 1)])
    plain.set_sensing("identity")
    n, N0 = X.shape
    T = D_high.shape[0]
    err = torch.zeros(1, dtype=torch.float32, device=dev)

    def one(kind, approximate=False):
        Dw = D_high.clone()
        a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        a.record()
        if kind == "cross_scale":
            sup, coef, keff = mk.code_high(Dw, D_low, X)
        else:
            plain.load_dictionary(0, Dw)
            sup, coef, keff = plain.solve(X, mode="plain", precision="fp32", K=(ts.K_high,))
        b.record()
        ctx = mk.fine if kind == "cross_scale" else plain
        ctx.profile(True)
        ctx.profile_read(reset=True)
        if kind == "cross_scale":
            ctx.ksvd_update(Dw, X, sup, coef, keff, True, mk.parent_dev, sup_low, err, approximate=approximate)
        else:
            ctx.ksvd_update(Dw, X, sup, coef, keff, True, err_out=err, approximate=approximate)
        c.record()
        torch.cuda.synchronize()
        prof = ctx.profile_read(reset=True)
        ctx.profile(False)
        return a.elapsed_time(b), b.elapsed_time(c), prof, ctx.ksvd_stats(), (sup, coef, keff)

    res, approx = {}, {}
    for kind in ("cross_scale", "plain"):
        for _ in range(max(args.warmup, 1)):
            one(kind, True)
        runs = [one(kind, True) for _ in range(max(args.steps, 1))]
        approx[kind] = {"coding_ms": sorted(r[0] for r in runs)[len(runs) // 2],
                        "update_ms": sorted(r[1] for r in runs)[len(runs) // 2],
                        "sweep_kernel_ms": sorted(r[2]["ksvd_sweep"][1] for r in runs)[len(runs) // 2]}
        approx[kind]["iteration_ms"] = approx[kind]["coding_ms"] + approx[kind]["update_ms"]
        for _ in range(max(args.warmup, 1)):
            one(kind)
        runs = [one(kind) for _ in range(max(args.steps, 1))]
        code = sorted(r[0] for r in runs)[len(runs) // 2]
        upd = sorted(r[1] for r in runs)[len(runs) // 2]
        sweep_ms = sorted(r[2]["ksvd_sweep"][1] for r in runs)[len(runs) // 2]
        steps, replaced, ranks = runs[-1][3]
        res[kind] = {"coding_ms": code, "update_ms": upd, "iteration_ms": code + upd, "sweep_kernel_ms": sweep_ms,
                     "power_steps": steps, "replaced_atoms": replaced, "cluster_ranks": ranks, "last": runs[-1][4]}
    # algorithmic FP32 work of the Step-2 sweep: Gram matrices n_k M^2, power steps M^2 each, residual
    # and coefficient updates 4 M per slot (2 FLOP per FMA)
    sup, coef, keff = res["cross_scale"].pop("last")
    res["plain"].pop("last")
    slots = int(keff.to(torch.int64).sum())
    flops = 2.0 * (slots * N0 * N0 + res["cross_scale"]["power_steps"] * N0 * N0 + 2 * slots * N0)
    achieved = flops / (res["cross_scale"]["sweep_kernel_ms"] / 1e3) / 1e12
    ranks = res["cross_scale"]["cluster_ranks"]
    cluster_peak = ranks * 128 * 2 * 2.070e9 / 1e12
    # CPU oracle of the same sweep (FP64), once
    cpu_s = None
    if not args.no_cpu_baseline:
        s_np, c_np, k_np = sup.cpu().numpy(), coef.cpu().numpy(), keff.cpu().numpy()
        t1 = time.perf_counter()
        oksvd.ksvd_update(D_high.cpu().numpy(), ts.X, s_np, c_np, k_np, True, ts.parents[0], sup_low.cpu().numpy())
        cpu_s = time.perf_counter() - t1
    out = {
        "metric": "modified K-SVD iteration time (Step 2: zero-tree coding + dictionary update)",
        "value": res["cross_scale"]["iteration_ms"], "unit": "ms", "higher_is_better": False,
        "workload": f"training set shaped like {args.workload}: {n} signals of dimension {N0}, "
                    f"T {T}/{D_low.shape[0]}, K {ts.K_high}/{ts.K_low}",
        "data": "synthetic (seeded two-scale model)",
        "step2": res["cross_scale"], "plain_ksvd": res["plain"],
        "training_speedup": res["plain"]["iteration_ms"] / res["cross_scale"]["iteration_ms"],
        "approximate_update": {"step2": approx["cross_scale"], "plain_ksvd": approx["plain"],
                               "training_speedup": approx["plain"]["iteration_ms"]
                               / approx["cross_scale"]["iteration_ms"]},
        "fit_2x2_s": fit_s, "err_low": el, "err_high": eh,
        "roofline": {"kernel": "ksvd_sweep", "bound": "alu", "achieved": achieved, "peak": cluster_peak,
                     "peak_source": f"derived: {ranks} SMs (one cluster) x 128 FP32 lanes x 2 x 2.07 GHz",
                     "unit": "TFLOP/s", "frac": achieved / cluster_peak, "traffic": None},
        "cpu_baseline": None if cpu_s is None else {
            "value": cpu_s * 1e3, "unit": "ms per sweep", "cores": 1, "kind": "oracle",
            "sample": "the same sweep (all signals and atoms), FP64 numpy"},
    }
    print(json.dumps(out))


def uneven_bench(args):
    """Uneven per-patch work: the light-field workload (4 coded-aperture shots
    of 4 x 4 views, 3,969 patches, D 1024 x 8192, K drawn per patch in [8, 20],
    three scales) solved with per-patch budgets, cross-scale and plain, with the
    work order off (static grids in patch order) and on (patches sorted by
    budget, largest first; restricted levels on persistent warps fed by a work
    queue).  CUDA graph replay, L2 flushed between steps; per-kernel times from
    a one-stream pass with graph replay off.  One JSON line."""
    import torch
    import synthetic
    from paper_1511_05174_gb300.context import Context

    dev = torch.device("cuda", 0)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    w = synthetic.make_workload("lightfield", links=args.links)
    ctx = Context(0)
    ctx.load_workload(w)
    Y = ctx.extract(torch.from_numpy(np.ascontiguousarray(w.meas)).to(dev))
    B = w.n_patches
    out = {"workload": f"lightfield_coded_aperture_{w.geometry.H}x{w.geometry.W}x{w.geometry.planes}_patch8_stride4",
           "patches": int(B), "K_range": [int(w.K_levels[0].min()), int(w.K_levels[0].max())],
           "links": args.links, "precision": args.precision, "data": "synthetic (seeded)", "l2": "flushed between steps"}
    for mode in ("cross_scale", "plain"):
        levels = w.K_levels if mode == "cross_scale" else w.K_levels[:1]
        Kmax = int(max(int(k.max()) for k in levels))
        K_patch = [torch.from_numpy(k.astype(np.int8)).to(dev) for k in levels]
        K = [Kmax] * len(levels)
        tune = ctx.autotune(Y, mode, args.precision, K=K, K_patch=K_patch, Kmax=Kmax)
        row = {"restricted_variant": tune["restricted_variant"], "top_level_form": tune["top_level_form"]}
        outs = {}
        for order in (0, 1):
            ctx.set_work_order(order)
            ctx.set_graph_mode(True)
            for _ in range(max(args.warmup, 3)):
                res = ctx.solve(Y, mode, args.precision, K=K, K_patch=K_patch, Kmax=Kmax)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(args.steps)]
            torch.cuda.synchronize()
            for a, b in ev:
                flush.zero_()
                a.record()
                res = ctx.solve(Y, mode, args.precision, K=K, K_patch=K_patch, Kmax=Kmax)
                b.record()
            torch.cuda.synchronize()
            ms = sorted(a.elapsed_time(b) for a, b in ev)
            outs[order] = [t.cpu().numpy() for t in res]
            ctx.set_graph_mode(False)
            ctx.profile_read(reset=True)
            ctx.profile(True)
            for _ in range(args.steps):
                flush.zero_()
                ctx.solve(Y, mode, args.precision, K=K, K_patch=K_patch, Kmax=Kmax)
            torch.cuda.synchronize()
            prof = ctx.profile_read(reset=True)
            ctx.profile(False)
            row["sorted_queue" if order else "static"] = {
                "ms_median": ms[len(ms) // 2], "ms_min": ms[0], "patches_per_s": B / (ms[len(ms) // 2] / 1e3),
                "kernels_ms_per_step": {k: v[1] / args.steps for k, v in prof.items()}}
        ctx.set_work_order(0)
        row["identical_results"] = all(np.array_equal(a, b) for a, b in zip(outs[0], outs[1]))
        row["speedup_sorted_queue"] = row["static"]["ms_median"] / row["sorted_queue"]["ms_median"]
        out[mode] = row
    print(json.dumps(out))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.sweep_q:
        q_sweep(args)
        return
    if args.ksvd:
        ksvd_bench(args)
        return
    if args.uneven:
        uneven_bench(args)
        return
    if args.serving_only:
        import torch
        pool = serving_pool(links=args.links)
        out = {"pool": [{"kind": k, "side": int(w.geometry.H), "patches": int(w.n_patches)} for k, w in pool]}
        for mode in ("cross_scale", "plain"):
            alone = standalone_summary(0, pool, mode, args.precision)
            out[mode] = {"rates": serving_bench(args, 0, pool, mode, SERVING_JOBS[mode]), **alone}
        print(json.dumps(out))
        return

    import torch
    import torch.distributed as dist

    import synthetic
    from paper_1511_05174_gb300.context import Context

    world, rank, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    w = synthetic.make_workload(args.workload, links=args.links, seed=rank)
    ctx = Context(local)
    ctx.load_workload(w)
    B, M = ctx.B, ctx.M
    K = [int(k[0]) for k in w.K_levels]
    Kmax = K[0]
    meas_d = torch.from_numpy(w.meas).to(dev)
    Y = torch.empty((B, M), dtype=torch.float32, device=dev)
    sup = torch.empty((B, Kmax), dtype=torch.int32, device=dev)
    coef = torch.empty((B, Kmax), dtype=torch.float32, device=dev)
    keff = torch.empty((B,), dtype=torch.int8, device=dev)
    img = torch.empty((w.geometry.planes, w.geometry.H, w.geometry.W), dtype=torch.float32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(mode):
        # the whole path in one library call: extraction, solve, synthesis + overlap-add
        ctx.reconstruct(meas_d, img, mode, args.precision, K=K if mode == "cross_scale" else K[:1], Kmax=Kmax)

    def barrier():
        if world > 1:
            dist.barrier()

    if args.variant is not None:
        ctx.set_kernel_variant(args.variant)
    if args.top_form is not None:
        ctx.set_top_level_form(args.top_form)
    if args.no_pipeline:
        ctx.set_pipeline(False)
    for _ in range(max(args.warmup, 3)):
        step("cross_scale")
        step("plain")
    # the library's autotuner picks the restricted-solver variant for this shape (untimed)
    if args.variant is None:
        ctx.extract(meas_d, Y)
        tune = ctx.autotune(Y, "cross_scale", args.precision, K=K, Kmax=Kmax)
        step("cross_scale")
    else:
        tune = {"restricted_variant": args.variant, "ms": [], "top_level_form": args.top_form or 0, "ms_top": []}
    torch.cuda.synchronize()

    def timed(mode, sampler=None):
        """Headline timing (CUDA events around each step, solves replayed from
        the library's CUDA graph, pipelined on two streams where it applies),
        then a second pass with per-kernel profiling (launch-by-launch events
        on one stream: graph replay and the pipeline off) for the breakdown."""
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        step(mode)  # records the graph of this mode's solve
        barrier()
        torch.cuda.synchronize()
        if sampler:
            sampler.start()
        for i in range(args.steps):
            flush.zero_()
            ev[i][0].record(stream)
            step(mode)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        clocks = sampler.stop() if sampler else None
        barrier()
        ms = sum(a.elapsed_time(b) for a, b in ev)
        st = ctx.stats()
        # the library's launches of one headline step (same configuration,
        # launched one by one instead of from the graph, to count them)
        ctx.profile_read(reset=True)
        ctx.profile(True)
        step(mode)
        torch.cuda.synchronize()
        per_step = int(sum(v[0] for v in ctx.profile_read(reset=True).values()))
        ctx.set_pipeline(False)
        for i in range(args.steps):
            flush.zero_()
            step(mode)
        torch.cuda.synchronize()
        prof = ctx.profile_read(reset=True)
        ctx.profile(False)
        ctx.set_pipeline(not args.no_pipeline)
        return max_over_ranks(ms, world, dev), prof, st, clocks, per_step

    ctx.set_graph_mode(True)
    cs_ms, cs_prof, cs_stats, clocks, cs_launches_per_step = timed("cross_scale", ClockSampler(local))
    cs_img = img.double().cpu().numpy()
    pl_ms, pl_prof, pl_stats, _, _ = timed("plain")
    pl_img = img.double().cpu().numpy()

    value = job_throughput(world, B, args.steps, cs_ms / 1e3)
    plain_value = job_throughput(world, B, args.steps, pl_ms / 1e3)

    # dominant kernel of the headline (cross-scale) step
    launches = {k: v for k, v in cs_prof.items()}
    dom = max(cs_prof.items(), key=lambda kv: kv[1][1])[0]
    n_launch, tot_ms = cs_prof[dom]
    amount, unit, bound = algorithmic(dom, w, launches, cs_stats, B, args.steps, M)
    roofline = None
    if amount is not None and n_launch:
        per_s = amount / (tot_ms / n_launch / 1e3)
        peaks = {}
        try:
            peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        except (OSError, ValueError):
            pass
        if bound == "hbm":
            peak, src = (peaks.get("hbm_gbs"), "measured") if peaks.get("hbm_gbs") else (6800.0, "fallback")
            achieved = per_s / 1e9
        elif bound == "tensor":
            peak, src = ((peaks.get("bf16_tflops"), "measured (BF16 dense, burst)") if peaks.get("bf16_tflops")
                         else (1900.0, "fallback"))
            achieved = per_s / 1e12
        else:
            sms = torch.cuda.get_device_properties(dev).multi_processor_count
            peak = fp32_peak_tflops(sms)
            src = f"derived: {sms} SM x {FP32_LANES_PER_SM} FP32 lanes x 2 x {MAX_SM_GHZ} GHz"
            achieved = per_s / 1e12
        roofline = {"kernel": dom, "bound": bound, "achieved": achieved, "peak": peak, "peak_source": src,
                    "unit": unit, "frac": achieved / peak if peak else None,
                    "traffic": read_traffic(dom, workload_config(w, args)["workload"]),
                    "avg_launch_us": 1e3 * tot_ms / n_launch, "launches_per_step": n_launch / args.steps}

    gpu_launches = cs_launches_per_step * args.steps  # the library's kernels in the timed region
    kernels = {k: {"launches_per_step": v[0] / args.steps, "ms_per_step": v[1] / args.steps}
               for k, v in cs_prof.items()}
    kernels_plain = {k: {"launches_per_step": v[0] / args.steps, "ms_per_step": v[1] / args.steps}
                     for k, v in pl_prof.items()}

    # end to end through the C ABI from pinned host memory
    e2e = None
    if not args.no_e2e:
        meas_h = torch.from_numpy(w.meas.copy()).pin_memory()
        img_h = torch.empty(img.shape, dtype=torch.float32).pin_memory()
        for _ in range(2):
            ctx.reconstruct_host(meas_h, img_h, "cross_scale", args.precision, K=K, Kmax=Kmax)
        barrier()
        tot = 0.0
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ctx.reconstruct_host(meas_h, img_h, "cross_scale", args.precision, K=K, Kmax=Kmax)
            tot += time.perf_counter() - t0
        e2e = {"value": job_throughput(world, B, args.steps, max_over_ranks(tot, world, dev)), "unit": UNIT,
               "h2d_bytes_per_step": int(w.meas.nbytes), "d2h_bytes_per_step": int(img.numel() * 4)}

    def psnr(est):
        mse = float(np.mean((w.truth - est) ** 2))
        peak = float(w.truth.max() - w.truth.min())
        return 10 * np.log10(peak * peak / mse)

    # the codes of both forms (the same context and settings solve the image once
    # more, from the solve's own CUDA graph) for the comparison with the oracle
    gpu_codes = {}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        ctx.extract(meas_d, Y)
        for mode, im in (("cross_scale", cs_img), ("plain", pl_img)):
            ctx.solve(Y, mode, args.precision, K=K if mode == "cross_scale" else K[:1], Kmax=Kmax,
                      out=(sup, coef, keff))
            torch.cuda.synchronize()
            gpu_codes[mode] = (sup.cpu().numpy(), coef.cpu().numpy(), keff.cpu().numpy().astype(np.int64), im)

    serving = None
    if not args.no_serving:
        pool = serving_pool(links=args.links)
        serving = {"pool": [{"kind": k, "side": int(w.geometry.H), "patches": int(w.n_patches)} for k, w in pool],
                   "precision": args.precision, "n_streams": 2, "per_gpu": True,
                   "note": "Poisson arrivals; each job drawn uniformly from the pool; host buffers in and out"}
        for mode in ("cross_scale", "plain"):
            alone = standalone_summary(local, pool, mode, args.precision)
            serving[mode] = {"rates": serving_bench(args, local, pool, mode, SERVING_JOBS[mode]), **alone,
                             "standalone_note": "each pool job alone through csp_reconstruct on device buffers "
                                                "(extraction, solve, overlap-add), default kernel choices, 48 GiB "
                                                "budget (null: the whole image's per-patch operators exceed it; the "
                                                "server builds them slice by slice); 'with_build': a coded-exposure "
                                                "job's per-patch operator rebuilt in the timed region, as for a "
                                                "served job with its own codes; jobs/s = jobs that fit / their "
                                                "summed device time"}

    cpu, acc = None, None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu, acc = cpu_baseline(w, gpu_codes, args.accuracy_sample)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": cs_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.precision == "fp32" else "bf16+f32",
            "data": "synthetic (seeded; Gaussian unit-norm atoms, K-sparse N(0,1) codes)",
            "config": {**workload_config(w, args), "form": "cross_scale", "precision": args.precision,
                       "cuda_graph": "extraction, solve and aggregation of a step replayed from one CUDA graph "
                                     "(csp_reconstruct in graph mode)",
                       "synthesis": ("written by the finest restricted level" if cs_stats.get("synthesized")
                                     else "separate pass"),
                       "pipeline": ("off (one stream)" if args.no_pipeline else
                                    "fused coarse level of the second chunk beside the restricted level of the "
                                    "first on a second stream (csp_set_pipeline); per-kernel times from a "
                                    "one-stream pass"),
                       "restricted_variant": tune["restricted_variant"],
                       "autotune_ms": [round(t, 4) for t in tune["ms"]],
                       "top_level_form": tune.get("top_level_form"),
                       "top_level_ms": [round(t, 4) for t in tune.get("ms_top", [])]},
            "plain_omp": {"value": plain_value, "unit": UNIT, "ms_per_step": pl_ms / args.steps,
                          "kernels": kernels_plain},
            "speedup_cross_scale_vs_plain": value / plain_value,
            "psnr_db": {"cross_scale": psnr(cs_img), "plain": psnr(pl_img)},
            "accuracy_vs_oracle": acc,
            "solve_stats": {"cross_scale": cs_stats, "plain": pl_stats},
            "kernels": kernels,
            "roofline": roofline,
            "gpu_launches": gpu_launches,
            "clocks": clocks,
            "e2e": e2e,
            "serving": serving,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
