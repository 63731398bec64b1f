"""Serving form: continuous batching of lattice solves on one GPU.

Requests (a lattice, a workload, a collision model, a storage precision, a side length
and a step count) arrive over time.  The scheduler admits them as soon as free device memory
and the active-cell budget allow, keeps every admitted lattice resident, and advances all of
them in ticks: active requests are grouped by (lattice, collision, precision), each group
is one batch (one kernel launch per time step for all its members, on the group's own
stream, so groups overlap on the device), and a tick advances every group by a number of
steps that never overshoots its member with the fewest remaining steps.  Finished requests
are harvested (conserved sums and the centre-line velocity profile read back), their memory
freed, and waiting requests admitted in the freed space at the next tick.

Two admission orders: "fifo" (arrival order; the head of the line waits for memory) and
"shortest" (least work first -- cell updates weighted by the group's measured time per
cell-step -- so that a small request arriving behind large ones is admitted and finishes early; a request that has waited longer than ``max_wait_s`` goes
first, and while it does not fit nothing behind it is admitted, so large requests cannot
starve).  With ``tick_seconds`` set, each group's steps per tick come from its measured time
per cell-step (the backend's estimate), so that a tick of a slow group (an FP64 cumulant
solve) and of a fast one take about the same time and a finished request is harvested
without waiting for a long tick of another group.  Under "shortest" the group holding the
request with the least remaining work runs on a high-priority CUDA stream for the tick.

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
    """Admission by free device memory and a cell budget, ticks of grouped batched steps, harvesting."""

    def __init__(self, backend, tick_steps: int = 64, reserve_bytes: int = 0, clock=time.perf_counter,
                 max_active: int | None = None, max_active_cells: int | None = None, policy: str = "fifo",
                 max_wait_s: float = 10.0, tick_seconds: float | None = None):
        if policy not in ("fifo", "shortest"):
            raise ValueError(f"unknown admission policy {policy!r}")
        self.backend = backend
        self.limit = max_active  # None: bounded by memory only; 1: a plain FIFO queue, one solve at a time
        # slot budget in lattice cells: enough active work to saturate the GPU without letting
        # every waiting request share it (which delays all completions); None: memory only
        self.cell_budget = max_active_cells
        self.tick_steps = int(tick_steps)
        self.tick_seconds = tick_seconds
        self.policy = policy
        self.max_wait_s = float(max_wait_s)
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

    def _order(self):
        """Pending requests in admission order."""
        if self.policy == "fifo":
            return list(self.pending)
        t = self.now()
        aged = [r for r in self.pending if t - r.arrival_s > self.max_wait_s]
        rest = sorted((r for r in self.pending if t - r.arrival_s <= self.max_wait_s),
                      key=lambda r: (self._work(r), r.arrival_s))
        return aged + rest

    def _work(self, req):
        """Work of a request: its cell updates, weighted by its group's measured time per
        cell-step when the backend has one (an FP64 cumulant update costs several FP32 BGK ones)."""
        est = getattr(self.backend, "step_seconds", None)
        w = est(self.backend.group_key(req), 1) if est is not None else None
        return req.side ** 3 * req.steps * (w if w else 1.0)

    def admit(self):
        """Admit waiting requests, in the policy's order, while they fit in free memory and in
        the cell budget.  Under "fifo" the first request that does not fit stops admission; under
        "shortest" it is passed over, unless it has waited longer than max_wait_s."""
        admitted = []
        for req in self._order():
            if self.limit is not None and len(self.active) >= self.limit:
                break
            need = self.backend.bytes_needed(req)
            if need + self.reserve > self.backend.total_bytes():
                self.pending.remove(req)
                t = self.now()
                self.results.append(Result(req.id, req.arrival_s, t, t, 0, req.side ** 3,
                                           error="request larger than the device"))
                continue
            fits = need + self.reserve <= self.backend.free_bytes()
            if fits and self.cell_budget is not None and self.active:
                fits = sum(a.req.side ** 3 for a in self.active) + req.side ** 3 <= self.cell_budget
            if not fits:
                if self.policy == "fifo" or self.now() - req.arrival_s > self.max_wait_s:
                    break  # head of line (or an aged request) waits for memory or a slot
                continue
            self.pending.remove(req)
            h = self.backend.start(req)
            self.active.append(_Active(req, h, self.now()))
            admitted.append(req.id)
        self.max_active = max(self.max_active, len(self.active))
        return admitted

    def _group_steps(self, key, members):
        most = min(a.remaining for a in members)
        if self.tick_seconds is not None:
            est = self.backend.step_seconds(key, sum(a.req.side ** 3 for a in members))
            if est is not None and est > 0.0:
                return max(1, min(most, int(self.tick_seconds / est)))
        return min(self.tick_steps, most)

    def tick(self):
        """Advance every active group once; harvest the finished requests."""
        if not self.active:
            return []
        groups: dict[tuple, list[_Active]] = {}
        for a in self.active:
            groups.setdefault(self.backend.group_key(a.req), []).append(a)
        # the group holding the request with the least remaining work runs at high priority
        # (with a backend that supports it), so that a short request keeps near its alone speed
        prioritize = getattr(self.backend, "prioritize", None)
        if prioritize is not None and self.policy == "shortest":
            first = min(self.active, key=lambda a: (a.req.side ** 3 * a.remaining, a.req.arrival_s))
            prioritize(self.backend.group_key(first.req))
        for key, members in groups.items():
            n = self._group_steps(key, members)
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
        self.streams = {}
        self._timed = {}  # group key -> (start event, end event, cell-steps) of its last step call
        self._rate = {}   # group key -> seconds per cell-step (moving average)
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
            # priority 0 (the default) and the highest (torch maps large negative values to it)
            self.streams[key] = (self.torch.cuda.Stream(priority=0), self.torch.cuda.Stream(priority=-64))
            self.batches[key].set_stream(self.streams[key][0].cuda_stream)
        self.batches[key].add(g)
        return g

    def prioritize(self, key):
        """Run group `key` on its high-priority stream from the next step on, the others on their
        low-priority ones (the scheduler calls this between ticks, after a sync, so that no
        group's work is in flight on the stream it leaves)."""
        self._urgent = key

    def step(self, key, handles, n):
        torch = self.torch
        st = self.streams[key][1 if key == getattr(self, "_urgent", None) else 0]
        self.batches[key].set_stream(st.cuda_stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        self.batches[key].step(n, use_graph=False)
        e1.record(st)
        self._timed[key] = (e0, e1, n * sum(h.N for h in handles))

    def step_seconds(self, key, cells):
        """Estimated seconds per time step of a group of `cells` cells (None until measured).
        Groups run concurrently on their own streams, so a measured time is the group's time
        under the load of that tick."""
        rate = self._rate.get(key)
        return None if rate is None else rate * cells

    def sync(self):
        for b in self.batches.values():
            b.sync()
        for key, (e0, e1, cell_steps) in self._timed.items():
            sec = e0.elapsed_time(e1) * 1e-3 / max(cell_steps, 1)
            old = self._rate.get(key)
            self._rate[key] = sec if old is None else 0.5 * (old + sec)
        self._timed.clear()

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
        self.streams.clear()
