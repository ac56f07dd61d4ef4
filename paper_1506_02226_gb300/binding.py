"""ctypes binding of include/dbscan.h (argument marshalling only).

Every function here has the name of the C function it calls and only converts
arguments; all clustering work runs in libdbscan_gb300.so's CUDA kernels.
There is no CPU fallback: if the library is missing, ``lib()`` raises.
Device buffers are passed as integer addresses (``tensor.data_ptr()``) and
streams as ``torch.cuda.Stream.cuda_stream``.
"""
from __future__ import annotations

import ctypes
import os
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libdbscan_gb300.so")

# status codes
DBSCAN_OK = 0
DBSCAN_ERR_ARG = 1
DBSCAN_ERR_NOT_QUANTISED = 2
DBSCAN_ERR_OOM = 3
DBSCAN_ERR_CUDA = 4
DBSCAN_ERR_TIMEOUT = 5
DBSCAN_ERR_BUSY = 6
DBSCAN_ERR_UNSUPPORTED = 7
DBSCAN_ERR_NOT_FOUND = 8
# options
DBSCAN_PREC_AUTO, DBSCAN_PREC_EXACT_SIMT, DBSCAN_PREC_FP16_GRAM, DBSCAN_PREC_BF16_GRAM = 0, 1, 2, 3
DBSCAN_GRID_AUTO, DBSCAN_GRID_ON, DBSCAN_GRID_OFF = 0, 1, 2
DBSCAN_LABEL_ROOT_INDEX, DBSCAN_LABEL_COMPACT = 0, 1
DBSCAN_PATH_NONE, DBSCAN_PATH_GRID, DBSCAN_PATH_ALLPAIRS_SIMT, DBSCAN_PATH_ALLPAIRS_TC = 0, 1, 2, 3
DBSCAN_PATH_GRID_PROJECTED, DBSCAN_PATH_PAPER = 4, 5
DBSCAN_PAPER_MAX_N = 65536
DBSCAN_HOOK_NONE, DBSCAN_HOOK_TC_STALL = 0, 1

c_i32, c_i64, c_f32, c_p = ctypes.c_int32, ctypes.c_int64, ctypes.c_float, ctypes.c_void_p


class dbscan_opts(ctypes.Structure):
    _fields_ = [("device", c_i32), ("synchronous", c_i32), ("stream", c_p), ("max_n", c_i64),
                ("max_d", c_i32), ("precision", c_i32), ("grid", c_i32), ("label_mode", c_i32),
                ("profile", c_i32), ("reserved", c_i32 * 7)]


class dbscan_stats(ctypes.Structure):
    _fields_ = [("n_clusters", c_i64), ("n_core", c_i64), ("n_border", c_i64), ("n_noise", c_i64),
                ("candidate_pairs", c_i64), ("band_pairs", c_i64), ("path", c_i32), ("cells", c_i32),
                ("threshold", c_i64), ("ms_total", c_f32), ("kernels", c_i32), ("pair_tests", c_i64),
                ("reserved_f", c_f32 * 4)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if not k.startswith("reserved")}


class dbscan_instance(ctypes.Structure):
    _fields_ = [("points", c_p), ("n", c_i64), ("d", c_i32), ("eps", c_f32), ("min_pts", c_i32),
                ("labels_out", c_p)]


class dbscan_tc_report(ctypes.Structure):
    _fields_ = [("pairs", c_i64), ("band_pairs", c_i64), ("wrong_outside_band", c_i64),
                ("max_abs_error_2g", c_i64), ("band_halfwidth_2g", c_i64), ("threshold", c_i64)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class dbscan_serve_opts(ctypes.Structure):
    _fields_ = [("device", c_i32), ("slots", c_i32), ("hbm_budget_bytes", c_i64), ("label_mode", c_i32),
                ("precision", c_i32), ("max_n", c_i64), ("max_d", c_i32), ("max_queue", c_i32),
                ("reserved", c_i32 * 4)]


class dbscan_serve_stats(ctypes.Structure):
    _fields_ = [("jobs_done", c_i64), ("jobs_queued", c_i64), ("jobs_running", c_i32), ("max_jobs_running", c_i32),
                ("hbm_budget_bytes", c_i64), ("bytes_in_flight", c_i64), ("peak_bytes_in_flight", c_i64),
                ("pool_reserved_bytes", c_i64), ("pool_peak_reserved_bytes", c_i64), ("reserved", c_i64 * 4)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


_SIGS = {
    "dbscan_opts_default": (None, [c_p]),
    "dbscan_plan_create": (ctypes.c_int, [c_p, c_p]),
    "dbscan_plan_destroy": (ctypes.c_int, [c_p]),
    "dbscan_run": (ctypes.c_int, [c_p, c_p, c_i64, c_i32, c_f32, c_i32, c_p, c_p]),
    "dbscan_run_detail": (ctypes.c_int, [c_p, c_p, c_i64, c_i32, c_f32, c_i32, c_p, c_p, c_p, c_p]),
    "dbscan_run_host": (ctypes.c_int, [c_p, c_p, c_i64, c_i32, c_f32, c_i32, c_p, c_p]),
    "dbscan_run_paper": (ctypes.c_int, [c_p, c_p, c_i64, c_i32, c_f32, c_i32, c_p, c_p]),
    "dbscan_plan_sync": (ctypes.c_int, [c_p]),
    "dbscan_plan_workspace_bytes": (c_i64, [c_p]),
    "dbscan_plan_test_hook": (ctypes.c_int, [c_p, c_i32]),
    "dbscan_tc_verify": (ctypes.c_int, [c_p, c_p, c_i64, c_i32, c_f32, c_i32, c_p]),
    "dbscan_plan_counters": (ctypes.c_int, [c_p, c_p, c_i32]),
    "dbscan_plan_phase_times": (ctypes.c_int, [c_p, c_i32, c_p, c_p, c_p]),
    "dbscan_batch": (ctypes.c_int, [c_p, c_p, c_i32, c_p]),
    "dbscan_batch_config": (ctypes.c_int, [c_p, c_p, c_p]),
    "dbscan_batch_tile": (ctypes.c_int, [c_p, c_p, c_p]),
    "dbscan_serve_opts_default": (None, [c_p]),
    "dbscan_serve_create": (ctypes.c_int, [c_p, c_p]),
    "dbscan_serve_submit": (ctypes.c_int, [c_p, c_p, c_p]),
    "dbscan_serve_poll": (ctypes.c_int, [c_p, ctypes.c_uint64, c_p]),
    "dbscan_serve_wait": (ctypes.c_int, [c_p, ctypes.c_uint64, c_i64, c_p]),
    "dbscan_serve_destroy": (ctypes.c_int, [c_p]),
    "dbscan_serve_info": (ctypes.c_int, [c_p, c_p]),
    "dbscan_serve_job_bytes": (c_i64, [c_p, c_i64, c_i32]),
    "dbscan_run_noalloc": (ctypes.c_int, [c_p, c_i64, c_i32, c_f32, c_i32, c_i32, c_p, c_p]),
    "dbscan_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "dbscan_abi_version": (c_i32, []),
}

_lock = threading.Lock()
_lib = None


def lib() -> ctypes.CDLL:
    """The loaded libdbscan_gb300.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1506_02226_gb300.build.build() "
                                   "(there is no CPU fallback)")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in _SIGS.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def exported_symbols() -> list[str]:
    return list(_SIGS)


class DbscanError(RuntimeError):
    def __init__(self, status: int, where: str = ""):
        self.status = status
        msg = lib().dbscan_strerror(status).decode()
        super().__init__(f"{where}: {msg} (status {status})" if where else f"{msg} (status {status})")


def _check(st: int, where: str):
    if st != DBSCAN_OK:
        raise DbscanError(st, where)


def dbscan_strerror(status: int) -> str:
    return lib().dbscan_strerror(status).decode()


def dbscan_abi_version() -> int:
    return int(lib().dbscan_abi_version())


def dbscan_opts_default() -> dbscan_opts:
    o = dbscan_opts()
    lib().dbscan_opts_default(ctypes.byref(o))
    return o


def dbscan_plan_create(opts: dbscan_opts | None = None) -> int:
    """Returns the plan handle (an address)."""
    h = c_p()
    _check(lib().dbscan_plan_create(ctypes.byref(h), ctypes.byref(opts) if opts is not None else None),
           "dbscan_plan_create")
    return h.value


def dbscan_plan_destroy(plan: int) -> None:
    _check(lib().dbscan_plan_destroy(plan), "dbscan_plan_destroy")


def dbscan_run(plan: int, points: int, n: int, d: int, eps: float, min_pts: int, labels_out: int,
               stats: dbscan_stats | None = None) -> int:
    """Status code of the call (0 = OK); raises nothing, so callers can test error paths."""
    return lib().dbscan_run(plan, points, n, d, eps, min_pts, labels_out,
                            ctypes.byref(stats) if stats is not None else None)


def dbscan_run_detail(plan: int, points: int, n: int, d: int, eps: float, min_pts: int, labels_out: int,
                      counts_out: int | None, core_out: int | None, stats: dbscan_stats | None = None) -> int:
    return lib().dbscan_run_detail(plan, points, n, d, eps, min_pts, labels_out, counts_out, core_out,
                                   ctypes.byref(stats) if stats is not None else None)


def dbscan_run_paper(plan: int, points: int, n: int, d: int, eps: float, min_pts: int, labels_out: int,
                     stats: dbscan_stats | None = None) -> int:
    return lib().dbscan_run_paper(plan, points, n, d, eps, min_pts, labels_out,
                                  ctypes.byref(stats) if stats is not None else None)


def dbscan_run_host(plan: int, host_points: int, n: int, d: int, eps: float, min_pts: int, host_labels: int,
                    stats: dbscan_stats | None = None) -> int:
    return lib().dbscan_run_host(plan, host_points, n, d, eps, min_pts, host_labels,
                                 ctypes.byref(stats) if stats is not None else None)


def dbscan_plan_sync(plan: int) -> int:
    return lib().dbscan_plan_sync(plan)


def dbscan_plan_phase_times(plan: int, max_phases: int = 32) -> list[tuple[str, float]]:
    """(kernel name, ms) of every kernel of the plan's last run (plan made with profile=1)."""
    ms = (ctypes.c_float * max_phases)()
    names = (ctypes.c_char_p * max_phases)()
    cnt = c_i32()
    _check(lib().dbscan_plan_phase_times(plan, max_phases, ms, names, ctypes.byref(cnt)), "dbscan_plan_phase_times")
    k = min(cnt.value, max_phases)
    return [(names[i].decode(), float(ms[i])) for i in range(k)]


def dbscan_tc_verify(plan: int, points: int, n: int, d: int, eps: float, bf16: int) -> dict:
    rep = dbscan_tc_report()
    _check(lib().dbscan_tc_verify(plan, points, n, d, eps, bf16, ctypes.byref(rep)), "dbscan_tc_verify")
    return rep.as_dict()


DBSCAN_NCTR = 32  # device counters per plan; 16..19 = pair tests of the count, merge, border, outer-ring passes


def dbscan_plan_counters(plan: int) -> list[int]:
    out = (ctypes.c_uint64 * DBSCAN_NCTR)()
    _check(lib().dbscan_plan_counters(plan, out, DBSCAN_NCTR), "dbscan_plan_counters")
    return list(out)


def dbscan_plan_workspace_bytes(plan: int) -> int:
    return int(lib().dbscan_plan_workspace_bytes(plan))


def dbscan_plan_test_hook(plan: int, hook: int) -> None:
    _check(lib().dbscan_plan_test_hook(plan, hook), "dbscan_plan_test_hook")


def dbscan_batch(plan: int, instances, per_inst=None) -> int:
    """instances: a ctypes array of dbscan_instance; per_inst: ctypes array of dbscan_stats or None."""
    return lib().dbscan_batch(plan, ctypes.cast(instances, c_p), len(instances),
                              ctypes.cast(per_inst, c_p) if per_inst is not None else None)


DBSCAN_NOALLOC_MAX_N = 16384
DBSCAN_NOALLOC_MAX_D = 16


def dbscan_run_noalloc(points: int, n: int, d: int, eps: float, min_pts: int, label_mode: int, labels_out: int,
                       stream: int | None = None) -> int:
    """Status code of the call; clusters without any device allocation (see include/dbscan.h)."""
    return lib().dbscan_run_noalloc(points, n, d, eps, min_pts, label_mode, labels_out, stream)


def dbscan_batch_config(plan: int) -> tuple[int, int]:
    ch, bps = c_i32(), c_i32()
    _check(lib().dbscan_batch_config(plan, ctypes.byref(ch), ctypes.byref(bps)), "dbscan_batch_config")
    return ch.value, bps.value


def dbscan_batch_tile(plan: int) -> tuple[int, int]:
    rows, cols = c_i32(), c_i32()
    _check(lib().dbscan_batch_tile(plan, ctypes.byref(rows), ctypes.byref(cols)), "dbscan_batch_tile")
    return rows.value, cols.value


def dbscan_serve_opts_default() -> dbscan_serve_opts:
    o = dbscan_serve_opts()
    lib().dbscan_serve_opts_default(ctypes.byref(o))
    return o


def dbscan_serve_create(opts: dbscan_serve_opts | None = None) -> int:
    h = c_p()
    _check(lib().dbscan_serve_create(ctypes.byref(h), ctypes.byref(opts) if opts is not None else None),
           "dbscan_serve_create")
    return h.value


def dbscan_serve_submit(server: int, inst: dbscan_instance) -> int:
    jid = ctypes.c_uint64()
    _check(lib().dbscan_serve_submit(server, ctypes.byref(inst), ctypes.byref(jid)), "dbscan_serve_submit")
    return jid.value


def dbscan_serve_poll(server: int, job_id: int) -> tuple[int, bool]:
    done = c_i32()
    st = lib().dbscan_serve_poll(server, job_id, ctypes.byref(done))
    return st, bool(done.value)


def dbscan_serve_wait(server: int, job_id: int, timeout_us: int = -1) -> tuple[int, float]:
    lat = ctypes.c_double()
    st = lib().dbscan_serve_wait(server, job_id, timeout_us, ctypes.byref(lat))
    return st, lat.value


def dbscan_serve_destroy(server: int) -> None:
    _check(lib().dbscan_serve_destroy(server), "dbscan_serve_destroy")


def dbscan_serve_info(server: int) -> dict:
    out = dbscan_serve_stats()
    _check(lib().dbscan_serve_info(server, ctypes.byref(out)), "dbscan_serve_info")
    return out.as_dict()


def dbscan_serve_job_bytes(server: int, n: int, d: int) -> int:
    return int(lib().dbscan_serve_job_bytes(server, n, d))
