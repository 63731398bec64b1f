"""Serving form: continuous batching of lattice solves on one GPU.

Requests (a lattice, a workload, a collision model, a storage precision, a side length
and a step count) arrive over time.  The scheduler admits them first-in first-out as soon
as free device memory allows, keeps every admitted lattice resident, and advances all of
them in ticks: active requests are grouped by (lattice, collision, precision), each group
is one batch (one kernel launch per time step for all its members, on the group's own
stream, so groups overlap on the device), and a tick advances every group by
min(tick_steps, fewest remaining steps in the group).  Finished requests are harvested
(conserved sums and the centre-line velocity profile read back), their memory freed, and
waiting requests admitted in the freed space at the next tick.

The scheduler is host logic only; the GPU work sits behind ``GpuBackend`` (the C ABI
through ``lbm``), so the scheduling rules can be tested with a fake backend.
"""
from __future__ import annotations

import dataclasses
import time
from collections import deque

import numpy as np

from . import inputs as I


@dataclasses.dataclass
class Request:
    id: int
    arrival_s: float
    lattice: int
    workload: str       # "cavity" or "taylor_green"
    collision: str      # model name, e.g. "BGK_W2" or "K"
    precision: str      # "f32" or "f64"
    side: int
    steps: int
    reynolds: float = 100.0


@dataclasses.dataclass
class Result:
    id: int
    arrival_s: float
    admitted_s: float
    finished_s: float
    steps: int
    cells: int
    mass: float = float("nan")
    energy: float = float("nan")
    profile: np.ndarray | None = None
    error: str | None = None

    @property
    def latency_s(self):
        return self.finished_s - self.arrival_s


class _Active:
    __slots__ = ("req", "handle", "remaining", "admitted_s")

    def __init__(self, req, handle, admitted_s):
        self.req, self.handle, self.remaining, self.admitted_s = req, handle, req.steps, admitted_s


class Scheduler:
    """FIFO admission by free device memory, ticks of grouped batched steps, harvesting."""

    def __init__(self, backend, tick_steps: int = 64, reserve_bytes: int = 0, clock=time.perf_counter,
                 max_active: int | None = None, max_active_cells: int | None = None):
        self.backend = backend
        self.limit = max_active  # None: bounded by memory only; 1: a plain FIFO queue, one solve at a time
        # slot budget in lattice cells: enough active work to saturate the GPU without letting
        # every waiting request share it (which delays all completions); None: memory only
        self.cell_budget = max_active_cells
        self.tick_steps = int(tick_steps)
        self.reserve = int(reserve_bytes)
        self.clock = clock
        self.pending: deque[Request] = deque()
        self.active: list[_Active] = []
        self.results: list[Result] = []
        self.t0 = None
        self.ticks = 0
        self.max_active = 0

    def now(self):
        return self.clock() - self.t0

    def offer(self, req: Request):
        self.pending.append(req)

    def admit(self):
        """Admit waiting requests in arrival order while they fit in free memory."""
        admitted = []
        while self.pending and (self.limit is None or len(self.active) < self.limit):
            req = self.pending[0]
            need = self.backend.bytes_needed(req)
            if need + self.reserve > self.backend.total_bytes():
                self.pending.popleft()
                t = self.now()
                self.results.append(Result(req.id, req.arrival_s, t, t, 0, req.side ** 3,
                                           error="request larger than the device"))
                continue
            if need + self.reserve > self.backend.free_bytes():
                break  # head of line waits for memory to free up
            if self.cell_budget is not None and self.active:
                if sum(a.req.side ** 3 for a in self.active) + req.side ** 3 > self.cell_budget:
                    break  # head of line waits for a slot
            self.pending.popleft()
            h = self.backend.start(req)
            self.active.append(_Active(req, h, self.now()))
            admitted.append(req.id)
        self.max_active = max(self.max_active, len(self.active))
        return admitted

    def tick(self):
        """Advance every active group once; harvest the finished requests."""
        if not self.active:
            return []
        groups: dict[tuple, list[_Active]] = {}
        for a in self.active:
            groups.setdefault(self.backend.group_key(a.req), []).append(a)
        for key, members in groups.items():
            n = min(self.tick_steps, min(a.remaining for a in members))
            self.backend.step(key, [a.handle for a in members], n)
            for a in members:
                a.remaining -= n
        self.backend.sync()
        self.ticks += 1
        done = [a for a in self.active if a.remaining == 0]
        self.active = [a for a in self.active if a.remaining > 0]
        out = []
        for a in done:
            payload = self.backend.finish(a.handle)
            r = Result(a.req.id, a.req.arrival_s, a.admitted_s, self.now(), a.req.steps, a.req.side ** 3, **payload)
            self.results.append(r)
            out.append(r.id)
        return out

    def run(self, trace, time_scale: float = 1.0, idle_sleep: float = 0.0005):
        """Replay a trace in real time (arrival_s * time_scale); returns the results."""
        queue = deque(sorted(trace, key=lambda r: r.arrival_s))
        self.t0 = self.clock()
        total = len(queue)
        while len(self.results) < total:
            t = self.now()
            while queue and queue[0].arrival_s * time_scale <= t:
                self.offer(queue.popleft())
            self.admit()
            if self.active:
                self.tick()
            elif queue:
                time.sleep(max(0.0, min(idle_sleep, queue[0].arrival_s * time_scale - t)))
            elif self.pending:
                raise RuntimeError("pending requests but nothing active: memory never frees up")
        return sorted(self.results, key=lambda r: r.id)


def summarize(results, wall_s):
    ok = [r for r in results if r.error is None]
    lat = np.array([r.latency_s for r in ok]) if ok else np.array([np.nan])
    cells_steps = sum(r.cells * r.steps for r in ok)
    return {"requests": len(results), "completed": len(ok), "failed": len(results) - len(ok),
            "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
            "mean_latency_s": float(lat.mean()), "makespan_s": wall_s,
            "mlups": cells_steps / wall_s / 1e6 if wall_s > 0 else float("nan")}


def trace_requests(raw, reynolds=100.0):
    return [Request(r["id"], r["arrival_s"], r["lattice"], r["workload"], r["collision"], r["precision"], r["side"],
                    r["steps"], reynolds) for r in raw]


class GpuBackend:
    """Serving backend on the CUDA library: one AA/SoA lattice per request, one batch per group."""

    U_LID = 0.02
    U0_TG = 0.02

    def __init__(self, device_total_bytes=None):
        import torch

        from . import lbm as L

        self.L, self.torch = L, torch
        self.batches = {}
        self._total = device_total_bytes

    def total_bytes(self):
        if self._total is None:
            self._total = self.torch.cuda.mem_get_info()[1]
        return self._total

    def free_bytes(self):
        return self.torch.cuda.mem_get_info()[0]

    def bytes_needed(self, req):
        n = req.side ** 3
        s = 8 if req.precision == "f64" else 4
        # populations (AA: one array) + flags + staging of the read-back fields (4 doubles per cell)
        return req.lattice * n * s + n + 32 * n + (1 << 20)

    def group_key(self, req):
        return (req.lattice, req.collision, req.precision)

    def make_lattice(self, req):
        """The request's lattice, initialised (cavity at rest, Taylor-Green from its analytic field)."""
        L = self.L
        n = req.side
        if req.workload == "cavity":
            nu = I.cavity_nu(self.U_LID, n, req.reynolds)
            flags = I.cavity_flags(n, n, n)
            walls = {I.LID: (self.U_LID, 0.0, 0.0)}
        else:
            nu = self.U0_TG * n / req.reynolds
            flags = I.periodic_flags(n, n, n)
            walls = {}
        omega = 1.0 / (3.0 * nu + 0.5)
        g = L.Lattice(req.lattice, n, n, n, "aa", req.collision, omega, flags,
                      precision=L.PRECISIONS[req.precision], wall_velocities=walls)
        if req.workload == "cavity":
            g.init_equilibrium()
        else:
            rho, u = I.taylor_green_fields_torch(n, n, n, self.U0_TG)
            g.init_equilibrium(rho, u)
        return g

    def start(self, req):
        g = self.make_lattice(req)
        key = self.group_key(req)
        if key not in self.batches:
            self.batches[key] = self.L.Batch()
        self.batches[key].add(g)
        return g

    def step(self, key, handles, n):
        self.batches[key].step(n, use_graph=False)

    def sync(self):
        for b in self.batches.values():
            b.sync()

    def read_result(self, g):
        """Conserved sums and the centre-line x-velocity profile along z at x = y = n/2."""
        torch = self.torch
        payload = {}
        try:
            m, e = g.reduce()
            payload["mass"], payload["energy"] = m, e
            n = g.nx
            u = torch.empty(3 * g.N, dtype=torch.float64, device="cuda")
            g.macroscopic(None, u)
            payload["profile"] = u[: g.N].view(n, n, n)[n // 2, n // 2, :].cpu().numpy()
        except self.L.LBMError as exc:
            payload["error"] = str(exc)
        return payload

    def finish(self, g):
        for b in self.batches.values():
            if g in b.members:
                b.remove(g)
                break
        payload = self.read_result(g)
        g.close()
        return payload

    def close(self):
        for b in self.batches.values():
            b.close()
        self.batches.clear()
