"""ctypes binding of libcsp.so: the C ABI declared in include/csp.h, same names.

Argument marshalling only -- every step of the computation runs in the CUDA
library.  Loading fails loudly when the library has not been built; there is
no CPU fallback.
"""

from __future__ import annotations

import ctypes
import os

MAX_LEVELS = 4
MAX_K = 32

CSP_OK = 0
CSP_ERR_INVALID = -1
CSP_ERR_OOM = -2
CSP_ERR_NOT_READY = -3
CSP_ERR_CUDA = -4
CSP_ERR_TIMEOUT = -5
CSP_ERR_UNSUPPORTED = -6

SENSE = {"identity": 0, "bayer_rggb": 1, "coded_exposure": 2, "coded_aperture": 3, "dense": 4}
MODE = {"plain": 0, "cross_scale": 1}
PREC = {"fp32": 0, "bf16": 1}

TUNE_VARIANTS = 14  # CSP_TUNE_VARIANTS
STATUS_NAMES = {0: "CSP_OK", -1: "CSP_ERR_INVALID", -2: "CSP_ERR_OOM", -3: "CSP_ERR_NOT_READY",
                -4: "CSP_ERR_CUDA", -5: "CSP_ERR_TIMEOUT", -6: "CSP_ERR_UNSUPPORTED"}

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libcsp.so")

# Every entry point declared in include/csp.h.
EXPORTS = ("csp_create", "csp_destroy", "csp_last_error", "csp_set_geometry", "csp_set_sensing",
           "csp_load_dictionary", "csp_load_scale_links", "csp_problem_size", "csp_extract_patches",
           "csp_solve", "csp_solve_stats_get", "csp_aggregate", "csp_aggregate_noalloc", "csp_reconstruct_host",
           "csp_autotune", "csp_set_kernel_variant", "csp_profile_enable", "csp_profile_read",
           "csp_server_create", "csp_server_destroy", "csp_server_last_error", "csp_server_add_model",
           "csp_submit", "csp_poll", "csp_wait", "csp_job_info_get", "csp_job_release",
           "csp_server_pause", "csp_set_aggregate_path", "csp_set_top_level_form",
           "csp_set_wait_test", "csp_set_graph_mode", "csp_set_pipeline", "csp_set_work_order", "csp_reconstruct",
           "csp_downsample", "csp_ksvd_update", "csp_ksvd_init_atoms", "csp_ksvd_stats_get")


class csp_geometry(ctypes.Structure):
    _fields_ = [("H", ctypes.c_int), ("W", ctypes.c_int), ("plane_rows", ctypes.c_int),
                ("plane_cols", ctypes.c_int), ("P", ctypes.c_int), ("stride", ctypes.c_int),
                ("n_levels", ctypes.c_int), ("factors", (ctypes.c_int * 4) * MAX_LEVELS)]


class csp_sensing(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("shots", ctypes.c_int), ("codes", ctypes.c_void_p), ("phi", ctypes.c_void_p)]


class csp_solve_params(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int), ("precision", ctypes.c_int), ("K", ctypes.c_int * MAX_LEVELS),
                ("K_patch", ctypes.c_void_p * MAX_LEVELS), ("Kmax", ctypes.c_int)]


class csp_solve_stats(ctypes.Structure):
    _fields_ = [("patches", ctypes.c_int64), ("fp64_fallbacks", ctypes.c_int64),
                ("early_stops", ctypes.c_int64), ("overflow", ctypes.c_int64),
                ("restricted_scores", ctypes.c_int64), ("timeouts", ctypes.c_int64),
                ("synthesized", ctypes.c_int64)]


class csp_kernel_time(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double)]


class csp_tune_result(ctypes.Structure):
    _fields_ = [("restricted_variant", ctypes.c_int), ("ms", ctypes.c_double * TUNE_VARIANTS),
                ("top_level_form", ctypes.c_int), ("ms_top", ctypes.c_double * 3)]


class csp_server_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("mem_budget_bytes", ctypes.c_size_t),
                ("max_batch_patches", ctypes.c_int64), ("n_streams", ctypes.c_int)]


class csp_model_desc(ctypes.Structure):
    _fields_ = [("geom", csp_geometry), ("sense_kind", ctypes.c_int), ("D", ctypes.c_void_p * MAX_LEVELS),
                ("T", ctypes.c_int * MAX_LEVELS), ("parent", ctypes.c_void_p * MAX_LEVELS),
                ("params", csp_solve_params)]


class csp_job_desc(ctypes.Structure):
    _fields_ = [("model_id", ctypes.c_int), ("H", ctypes.c_int), ("W", ctypes.c_int),
                ("meas_host", ctypes.c_void_p), ("codes_host", ctypes.c_void_p), ("image_host", ctypes.c_void_p)]


class csp_job_info(ctypes.Structure):
    _fields_ = [("patches", ctypes.c_int64), ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double),
                ("t_done", ctypes.c_double), ("batch_jobs", ctypes.c_int), ("batch_patches", ctypes.c_int64),
                ("status", ctypes.c_int), ("enqueue_ms", ctypes.c_double), ("copy_in_ms", ctypes.c_double),
                ("solve_ms", ctypes.c_double), ("aggregate_ms", ctypes.c_double), ("copy_out_ms", ctypes.c_double),
                ("t_gpu_done", ctypes.c_double), ("host_out_ms", ctypes.c_double), ("build_ms", ctypes.c_double)]


class CspError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_LIB = None


def load_library(path: str = LIB_PATH):
    """Load libcsp.so (built in-tree by paper_1511_05174_gb300.build)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build the CUDA library first "
                           "(python -m paper_1511_05174_gb300.build or __graft_entry__.build())")
    lib = ctypes.CDLL(path)
    vp, i, i64p = ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int64)
    sig = {
        "csp_create": (i, [ctypes.POINTER(vp), i, ctypes.c_size_t]),
        "csp_destroy": (None, [vp]),
        "csp_last_error": (ctypes.c_char_p, [vp]),
        "csp_set_geometry": (i, [vp, ctypes.POINTER(csp_geometry)]),
        "csp_set_sensing": (i, [vp, ctypes.POINTER(csp_sensing)]),
        "csp_load_dictionary": (i, [vp, i, vp, i, i, i]),
        "csp_load_scale_links": (i, [vp, i, vp, i, i]),
        "csp_problem_size": (i, [vp, i64p, ctypes.POINTER(ctypes.c_int)]),
        "csp_extract_patches": (i, [vp, vp, vp, i64p, vp]),
        "csp_solve": (i, [vp, ctypes.POINTER(csp_solve_params), vp, ctypes.c_int64, vp, vp, vp, vp]),
        "csp_solve_stats_get": (i, [vp, ctypes.POINTER(csp_solve_stats)]),
        "csp_aggregate": (i, [vp, vp, vp, vp, ctypes.c_int64, i, vp, vp]),
        "csp_aggregate_noalloc": (i, [vp, vp, vp, vp, ctypes.c_int64, i, vp, vp]),
        "csp_reconstruct_host": (i, [vp, ctypes.POINTER(csp_solve_params), vp, vp, vp]),
        "csp_reconstruct": (i, [vp, ctypes.POINTER(csp_solve_params), vp, vp, vp]),
        "csp_autotune": (i, [vp, ctypes.POINTER(csp_solve_params), vp, ctypes.c_int64, vp, vp, vp, vp,
                             ctypes.POINTER(csp_tune_result)]),
        "csp_set_kernel_variant": (i, [vp, i]),
        "csp_set_aggregate_path": (i, [vp, i]),
        "csp_set_top_level_form": (i, [vp, i]),
        "csp_set_wait_test": (i, [vp, i]),
        "csp_set_graph_mode": (i, [vp, i]),
        "csp_set_pipeline": (i, [vp, i]),
        "csp_set_work_order": (i, [vp, i]),
        "csp_profile_enable": (i, [vp, i]),
        "csp_profile_read": (i, [vp, ctypes.POINTER(csp_kernel_time), i, ctypes.POINTER(ctypes.c_int), i]),
        "csp_server_create": (i, [ctypes.POINTER(vp), ctypes.POINTER(csp_server_config)]),
        "csp_server_destroy": (None, [vp]),
        "csp_server_last_error": (ctypes.c_char_p, [vp]),
        "csp_server_add_model": (i, [vp, ctypes.POINTER(csp_model_desc), ctypes.POINTER(ctypes.c_int)]),
        "csp_submit": (i, [vp, ctypes.POINTER(csp_job_desc), ctypes.POINTER(ctypes.c_uint64)]),
        "csp_poll": (i, [vp, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int)]),
        "csp_wait": (i, [vp, ctypes.c_uint64, ctypes.c_int64]),
        "csp_job_info_get": (i, [vp, ctypes.c_uint64, ctypes.POINTER(csp_job_info)]),
        "csp_job_release": (i, [vp, ctypes.c_uint64]),
        "csp_server_pause": (i, [vp, i]),
        "csp_downsample": (i, [vp, i, vp, ctypes.c_int64, vp, vp]),
        "csp_ksvd_update": (i, [vp, vp, i, i, vp, ctypes.c_int64, vp, vp, vp, i, i, i, vp, vp, i, vp, vp]),
        "csp_ksvd_init_atoms": (i, [vp, vp, i, i, vp, ctypes.c_int64, vp, vp, vp, i, i, vp, vp]),
        "csp_ksvd_stats_get": (i, [vp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                                   ctypes.POINTER(ctypes.c_int64)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _LIB = lib
    return lib


def check(status: int, ctx) -> None:
    if status != CSP_OK:
        lib = load_library()
        raise CspError(status, lib.csp_last_error(ctx).decode(errors="replace"))


# Thin wrappers with the C names: status is checked and raised as CspError.

def csp_create(device: int = 0, mem_budget_bytes: int = 0):
    lib = load_library()
    ctx = ctypes.c_void_p()
    check(lib.csp_create(ctypes.byref(ctx), device, mem_budget_bytes), None)
    return ctx


def csp_destroy(ctx) -> None:
    load_library().csp_destroy(ctx)


def csp_last_error(ctx) -> str:
    return load_library().csp_last_error(ctx).decode(errors="replace")


def csp_set_geometry(ctx, geom: csp_geometry) -> None:
    check(load_library().csp_set_geometry(ctx, ctypes.byref(geom)), ctx)


def csp_set_sensing(ctx, sensing: csp_sensing) -> None:
    check(load_library().csp_set_sensing(ctx, ctypes.byref(sensing)), ctx)


def csp_load_dictionary(ctx, level: int, D_ptr: int, N_l: int, T_l: int, is_device_ptr: int) -> None:
    check(load_library().csp_load_dictionary(ctx, level, D_ptr, N_l, T_l, is_device_ptr), ctx)


def csp_load_scale_links(ctx, level: int, parent_ptr, T_l: int, Q: int) -> None:
    check(load_library().csp_load_scale_links(ctx, level, parent_ptr, T_l, Q), ctx)


def csp_problem_size(ctx):
    B = ctypes.c_int64()
    M = ctypes.c_int()
    check(load_library().csp_problem_size(ctx, ctypes.byref(B), ctypes.byref(M)), ctx)
    return B.value, M.value


def csp_extract_patches(ctx, meas_ptr: int, Y_ptr: int, stream: int) -> int:
    B = ctypes.c_int64()
    check(load_library().csp_extract_patches(ctx, meas_ptr, Y_ptr, ctypes.byref(B), stream), ctx)
    return B.value


def csp_solve(ctx, params: csp_solve_params, Y_ptr: int, B: int, sup_ptr: int, coef_ptr: int,
              keff_ptr: int, stream: int) -> None:
    check(load_library().csp_solve(ctx, ctypes.byref(params), Y_ptr, B, sup_ptr, coef_ptr, keff_ptr, stream), ctx)


def csp_solve_stats_get(ctx) -> csp_solve_stats:
    st = csp_solve_stats()
    check(load_library().csp_solve_stats_get(ctx, ctypes.byref(st)), ctx)
    return st


def csp_aggregate(ctx, sup_ptr: int, coef_ptr: int, keff_ptr: int, B: int, Kmax: int, img_ptr: int,
                  stream: int) -> None:
    check(load_library().csp_aggregate(ctx, sup_ptr, coef_ptr, keff_ptr, B, Kmax, img_ptr, stream), ctx)


def csp_aggregate_noalloc(ctx, sup_ptr: int, coef_ptr: int, keff_ptr: int, B: int, Kmax: int, img_ptr: int,
                          stream: int) -> None:
    """csp_aggregate without any device allocation (fixed 16 MiB scratch; B * N0 <= 4 Mi)."""
    check(load_library().csp_aggregate_noalloc(ctx, sup_ptr, coef_ptr, keff_ptr, B, Kmax, img_ptr, stream), ctx)


def csp_reconstruct(ctx, params: csp_solve_params, meas_ptr: int, image_ptr: int, stream: int) -> None:
    check(load_library().csp_reconstruct(ctx, ctypes.byref(params), meas_ptr, image_ptr, stream), ctx)


def csp_reconstruct_host(ctx, params: csp_solve_params, meas_ptr: int, img_ptr: int, stream: int) -> None:
    check(load_library().csp_reconstruct_host(ctx, ctypes.byref(params), meas_ptr, img_ptr, stream), ctx)


def csp_profile_enable(ctx, on: bool) -> None:
    check(load_library().csp_profile_enable(ctx, int(bool(on))), ctx)


def csp_profile_read(ctx, reset: bool = False):
    """{kernel kind: (launches, total_ms)}."""
    cap = 32
    arr = (csp_kernel_time * cap)()
    n = ctypes.c_int()
    check(load_library().csp_profile_read(ctx, arr, cap, ctypes.byref(n), int(bool(reset))), ctx)
    return {arr[i].name.decode(): (int(arr[i].launches), float(arr[i].total_ms)) for i in range(min(n.value, cap))}


def csp_autotune(ctx, params: csp_solve_params, Y_ptr: int, B: int, sup_ptr: int, coef_ptr: int, keff_ptr: int,
                 stream: int) -> csp_tune_result:
    res = csp_tune_result()
    check(load_library().csp_autotune(ctx, ctypes.byref(params), Y_ptr, B, sup_ptr, coef_ptr, keff_ptr, stream,
                                      ctypes.byref(res)), ctx)
    return res


def csp_set_graph_mode(ctx, on: bool) -> None:
    check(load_library().csp_set_graph_mode(ctx, int(bool(on))), ctx)


def csp_set_pipeline(ctx, on: bool) -> None:
    check(load_library().csp_set_pipeline(ctx, int(bool(on))), ctx)


def csp_set_work_order(ctx, order: int) -> None:
    check(load_library().csp_set_work_order(ctx, int(order)), ctx)


def csp_set_wait_test(ctx, on: bool) -> None:
    check(load_library().csp_set_wait_test(ctx, int(bool(on))), ctx)


def csp_set_top_level_form(ctx, form: int) -> None:
    check(load_library().csp_set_top_level_form(ctx, int(form)), ctx)


def csp_set_aggregate_path(ctx, path: int) -> None:
    check(load_library().csp_set_aggregate_path(ctx, int(path)), ctx)


def csp_set_kernel_variant(ctx, restricted_variant: int) -> None:
    check(load_library().csp_set_kernel_variant(ctx, int(restricted_variant)), ctx)


# Serving (continuous batching of reconstruction jobs).

def check_server(status: int, srv) -> None:
    if status != CSP_OK:
        raise CspError(status, load_library().csp_server_last_error(srv).decode(errors="replace"))


def csp_server_create(device: int = 0, mem_budget_bytes: int = 0, max_batch_patches: int = 0, n_streams: int = 0):
    lib = load_library()
    srv = ctypes.c_void_p()
    cfg = csp_server_config(device, mem_budget_bytes, max_batch_patches, n_streams)
    st = lib.csp_server_create(ctypes.byref(srv), ctypes.byref(cfg))
    if st != CSP_OK:
        raise CspError(st, lib.csp_last_error(None).decode(errors="replace"))
    return srv


def csp_server_destroy(srv) -> None:
    load_library().csp_server_destroy(srv)


def csp_server_last_error(srv) -> str:
    return load_library().csp_server_last_error(srv).decode(errors="replace")


def csp_server_add_model(srv, desc: csp_model_desc) -> int:
    mid = ctypes.c_int()
    check_server(load_library().csp_server_add_model(srv, ctypes.byref(desc), ctypes.byref(mid)), srv)
    return mid.value


def csp_submit(srv, job: csp_job_desc) -> int:
    jid = ctypes.c_uint64()
    check_server(load_library().csp_submit(srv, ctypes.byref(job), ctypes.byref(jid)), srv)
    return jid.value


def csp_poll(srv, job_id: int) -> bool:
    done = ctypes.c_int()
    check_server(load_library().csp_poll(srv, job_id, ctypes.byref(done)), srv)
    return bool(done.value)


def csp_wait(srv, job_id: int, timeout_us: int = -1) -> int:
    """Status of the job (raises CspError only for an unknown job; a timeout
    returns CSP_ERR_TIMEOUT)."""
    return int(load_library().csp_wait(srv, job_id, timeout_us))


def csp_job_info_get(srv, job_id: int) -> csp_job_info:
    info = csp_job_info()
    check_server(load_library().csp_job_info_get(srv, job_id, ctypes.byref(info)), srv)
    return info


def csp_job_release(srv, job_id: int) -> None:
    check_server(load_library().csp_job_release(srv, job_id), srv)


def csp_server_pause(srv, paused: bool) -> None:
    check_server(load_library().csp_server_pause(srv, int(bool(paused))), srv)


def csp_downsample(ctx, level: int, X_ptr: int, N: int, X_low_ptr: int, stream: int = 0) -> None:
    check(load_library().csp_downsample(ctx, level, X_ptr, N, X_low_ptr, stream), ctx)


def csp_ksvd_update(ctx, D_ptr: int, M: int, T: int, X_ptr: int, N: int, sup_ptr: int, coef_ptr: int,
                    keff_ptr: int, Kmax: int, replace_unused: int, approximate: int, parent_ptr, rsup_ptr, Kc: int,
                    err_ptr, stream: int = 0) -> None:
    check(load_library().csp_ksvd_update(ctx, D_ptr, M, T, X_ptr, N, sup_ptr, coef_ptr, keff_ptr, Kmax,
                                         replace_unused, approximate, parent_ptr, rsup_ptr, Kc, err_ptr, stream),
          ctx)


def csp_ksvd_init_atoms(ctx, D_ptr: int, M: int, T: int, X_ptr: int, N: int, parent_ptr, sup_low_ptr,
                        keff_low_ptr, Kc: int, T_low: int, u_ptr: int, stream: int = 0) -> None:
    check(load_library().csp_ksvd_init_atoms(ctx, D_ptr, M, T, X_ptr, N, parent_ptr, sup_low_ptr, keff_low_ptr,
                                             Kc, T_low, u_ptr, stream), ctx)


def csp_ksvd_stats_get(ctx):
    steps, rep, ranks = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    check(load_library().csp_ksvd_stats_get(ctx, ctypes.byref(steps), ctypes.byref(rep), ctypes.byref(ranks)), ctx)
    return int(steps.value), int(rep.value), int(ranks.value)
