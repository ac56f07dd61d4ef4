"""Torch-tensor front end over the C ABI (device memory and streams only).

    with Plan(max_n=500_000, max_d=3) as plan:
        labels = plan.run(points_cuda_f32, eps=0.005, min_pts=10)

All arithmetic runs in libdbscan_gb300.so; this module allocates output
tensors and passes their addresses.
"""
from __future__ import annotations

import ctypes

import torch

from . import binding as B


class Plan:
    def __init__(self, max_n: int, max_d: int = 64, device: int = 0, precision: int = B.DBSCAN_PREC_AUTO,
                 grid: int = B.DBSCAN_GRID_AUTO, label_mode: int = B.DBSCAN_LABEL_ROOT_INDEX,
                 synchronous: bool = True, stream: torch.cuda.Stream | None = None, profile: bool = False):
        o = B.dbscan_opts_default()
        o.device = device
        o.max_n = max_n
        o.max_d = max_d
        o.precision = precision
        o.grid = grid
        o.label_mode = label_mode
        o.synchronous = 1 if synchronous else 0
        o.profile = 1 if profile else 0
        o.stream = stream.cuda_stream if stream is not None else None
        self.device = torch.device("cuda", device)
        self.stream = stream
        self.handle = B.dbscan_plan_create(o)

    def close(self):
        if self.handle:
            B.dbscan_plan_destroy(self.handle)
            self.handle = 0

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _check_points(points: torch.Tensor):
        if not (points.is_cuda and points.dtype == torch.float32 and points.dim() == 2 and points.is_contiguous()):
            raise ValueError("points must be a contiguous CUDA float32 tensor of shape [n, d]")

    def run(self, points: torch.Tensor, eps: float, min_pts: int, labels: torch.Tensor | None = None,
            stats: bool = False):
        """Labels (int32 [n], on the device); with stats=True also a dict of dbscan_stats."""
        self._check_points(points)
        n, d = points.shape
        if labels is None:
            labels = torch.empty(n, dtype=torch.int32, device=points.device)
        st = B.dbscan_stats() if stats else None
        rc = B.dbscan_run(self.handle, points.data_ptr(), n, d, eps, min_pts, labels.data_ptr(), st)
        if rc:
            raise B.DbscanError(rc, "dbscan_run")
        return (labels, st.as_dict()) if stats else labels

    def run_detail(self, points: torch.Tensor, eps: float, min_pts: int):
        """(labels, exact neighbour counts, core flags, stats dict), all on the device."""
        self._check_points(points)
        n, d = points.shape
        labels = torch.empty(n, dtype=torch.int32, device=points.device)
        counts = torch.empty(n, dtype=torch.int32, device=points.device)
        core = torch.empty(n, dtype=torch.uint8, device=points.device)
        st = B.dbscan_stats()
        rc = B.dbscan_run_detail(self.handle, points.data_ptr(), n, d, eps, min_pts, labels.data_ptr(),
                                 counts.data_ptr(), core.data_ptr(), st)
        if rc:
            raise B.DbscanError(rc, "dbscan_run_detail")
        return labels, counts, core, st.as_dict()

    def run_paper(self, points: torch.Tensor, eps: float, min_pts: int, labels: torch.Tensor | None = None,
                  stats: bool = False):
        """The paper's materialised pipeline (comparison variant); same labels as run()."""
        self._check_points(points)
        n, d = points.shape
        if labels is None:
            labels = torch.empty(n, dtype=torch.int32, device=points.device)
        st = B.dbscan_stats() if stats else None
        rc = B.dbscan_run_paper(self.handle, points.data_ptr(), n, d, eps, min_pts, labels.data_ptr(), st)
        if rc:
            raise B.DbscanError(rc, "dbscan_run_paper")
        return (labels, st.as_dict()) if stats else labels

    def run_host(self, points: torch.Tensor, eps: float, min_pts: int, labels: torch.Tensor | None = None):
        """End-to-end call on host tensors (pinned for speed): copies in, clusters, copies out."""
        if points.is_cuda or points.dtype != torch.float32 or not points.is_contiguous():
            raise ValueError("points must be a contiguous host float32 tensor")
        n, d = points.shape
        if labels is None:
            labels = torch.empty(n, dtype=torch.int32, pin_memory=True)
        rc = B.dbscan_run_host(self.handle, points.data_ptr(), n, d, eps, min_pts, labels.data_ptr(), None)
        if rc:
            raise B.DbscanError(rc, "dbscan_run_host")
        return labels

    def phase_times(self):
        return B.dbscan_plan_phase_times(self.handle)

    def counters(self) -> list[int]:
        """The plan's device counters after its last run (waits for the plan's stream)."""
        return B.dbscan_plan_counters(self.handle)

    def pair_tests(self) -> list[int]:
        """Pair predicates the last run evaluated: [count, merge, border, outer-ring merge] passes."""
        return self.counters()[16:20]

    def sync(self) -> int:
        return B.dbscan_plan_sync(self.handle)


def cluster(points: torch.Tensor, eps: float, min_pts: int, **plan_kw) -> torch.Tensor:
    """One-shot convenience: plan sized for this input, run, destroy."""
    n, d = points.shape
    with Plan(max_n=max(n, 1), max_d=d, device=points.device.index or 0, **plan_kw) as p:
        return p.run(points, eps, min_pts)


def make_instances(items):
    """ctypes array of dbscan_instance from (points_cuda, eps, min_pts, labels_cuda) tuples."""
    arr = (B.dbscan_instance * len(items))()
    for k, (pts, eps, mp, lab) in enumerate(items):
        arr[k].points = pts.data_ptr()
        arr[k].n = pts.shape[0]
        arr[k].d = pts.shape[1]
        arr[k].eps = eps
        arr[k].min_pts = mp
        arr[k].labels_out = lab.data_ptr()
    return arr


__all__ = ["Plan", "cluster", "make_instances", "ctypes"]
