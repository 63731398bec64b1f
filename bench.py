"""Benchmark of the fused stream-and-collide step on B300 (one JSON line on stdout).

Workload (default): D3Q19 lid-driven cavity 256^3 in FP64, Re 1000, lid u = 0.02 along x on
the whole plane z = 255, bounce-back walls on the other faces, nu = u N / Re,
omega = 1 / (3 nu + 1/2), AA pattern, SoA layout, BGK-W2 collision.  A step is one time
iteration over the whole lattice.  The 2.5 GB population array is far larger than the
126 MB L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]
                  [--lattice 19|27] [--n 256] [--scheme aa] [--collision BGK_W2]
                  [--precision f64|f32|f16] [--matrix]

MLUPS counts every lattice node (walls included), the paper's convention.  Under torchrun
(N > 1) each rank runs an independent replica of the workload (replicas only: the method
needs no data exchange between independent lattices); the value is the sum of all ranks'
updates over the slowest rank's time.  --impl reference times the FP64 CPU oracle on the
host cores instead (rank 0 only).
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2010_11751_b300 import inputs as I  # noqa: E402

MEASURED = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6400.0
# FP64 pipe operations (DADD, DMUL, DFMA thread instructions) per fluid-cell update of the AA step
# kernels, D3Q19/D3Q27 cavity 128^3, from one ncu capture per model (the even and odd kernels execute
# the same counts).  The plain FP64 operators (K, ...) are bound by the FP64 pipe, which issues
# one of them per slot, so their roofline counts operations (flops are reported beside).  BGK-W2,
# TRT and RR run their collision on the FP32 and integer pipes (exact integer moments,
# double-float arithmetic; BGK-W2 and TRT keep one FP64 FMA per population, RR none): their
# roofline is memory's (RR is bound by instruction issue short of it).
FP64_OPS_PER_FLUID_CELL = {
    # (lattice, collision): (dadd, dmul, dfma) per fluid cell
    (19, "BGK_W2"): (0.24, 0.00, 19.00),
    (19, "TRT"): (0.24, 0.00, 19.00),
    (19, "RR"): (0.24, 0.00, 0.00),
    (19, "K"): (81.24, 31.00, 111.00),
    (27, "BGK_W2"): (0.43, 0.00, 27.00),
    (27, "RR"): (0.43, 0.00, 0.00),
    (27, "K"): (161.43, 67.00, 187.00),
}
# models whose FP64 collision runs off the FP64 pipe (memory-bound roofline)
FP64_OFF_PIPE = {"BGK_W2", "TRT", "RR"}
# B300 FP64 pipe: 2 DFMA (or DADD / DMUL) per SM per clock (ncu peak_sustained)
FP64_OPS_PER_SM_CLK = 2
# time budget of the reference arm (the FP64 CPU oracle timed on the host cores)
REFERENCE_SECONDS = 120.0
# DRAM bytes (read + write) of the AA-odd step of the headline configuration, from one ncu capture
# of the D3Q19 128^3 cavity (the small case the capture rules allow) per cell each kernel updates:
# the staged kernel's bulk cells and the listed-cell kernel's cells (next to a wall or on a domain
# face); a full step's traffic is scaled from those by the cell counts of the lattice.  Reported
# only while the kernel sources hash to the value recorded with the capture; any later kernel
# change turns the figure back to null.
KERNEL_SOURCES = ["lattice.cuh", "collision.cuh", "kernels.cuh", "fx64.cuh", "fx_rr.cuh", "dfloat.cuh", "staged.cuh"]
TRAFFIC = {
    # (precision, lattice, collision, scheme): (bytes per bulk cell, bytes per listed cell, source hash)
    ("f64", 19, "BGK_W2", "aa"): ((319938304 + 241436160) / 124 ** 3, (67292928 + 6498560) / (126 ** 3 - 124 ** 3),
                                  "28fe1f13e8f68c65"),
}


def bulk_and_listed(flags, n, Q):
    """Fluid cells with every lattice neighbour fluid and off the domain faces (the staged kernel's
    bulk cells), and the other fluid cells (the listed-cell kernel's)."""
    fl = flags.reshape(n, n, n) != 0
    fluid = ~fl
    near = np.zeros_like(fl)
    for c in np.ndindex(3, 3, 3):
        c = np.array(c) - 1
        n2 = int((c * c).sum())
        if n2 == 0 or (Q == 19 and n2 == 3):
            continue
        near |= np.roll(fl, shift=tuple(-c), axis=(0, 1, 2))
    face = np.zeros_like(fl)
    face[0], face[-1], face[:, 0], face[:, -1], face[:, :, 0], face[:, :, -1] = (True,) * 6
    bulk = fluid & ~near & ~face
    return int(bulk.sum()), int((fluid & ~bulk).sum())


def kernel_source_hash():
    import hashlib
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2010_11751_b300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    # 1000 steps: the step count of the 256^3 cavity configuration
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--lattice", type=int, default=19)
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--scheme", default="aa")
    ap.add_argument("--collision", default="BGK_W2")
    ap.add_argument("--precision", default="f64")
    ap.add_argument("--reynolds", type=float, default=1000.0)
    ap.add_argument("--matrix", action="store_true", help="also time every scheme x collision x lattice")
    ap.add_argument("--matrix-steps", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--clocks-dir", default=None, help="where to keep the raw nvidia-smi samples (default: temp dir)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the forms (D3Q27, precision, batching, serving) measured after the headline")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--forms", default="",
                    help="precision | batching | serving | sweep | unrolling: the forms and studies besides "
                         "the headline")
    ap.add_argument("--form-steps", type=int, default=2000)
    ap.add_argument("--trace", type=int, default=500, help="serving: number of requests")
    ap.add_argument("--rate", type=float, default=50.0, help="serving: mean arrival rate (1/s)")
    ap.add_argument("--tick", type=int, default=64, help="serving: steps per tick")
    ap.add_argument("--slot-cells", type=int, default=1 << 24, help="serving: active-cell budget")
    ap.add_argument("--tick-seconds", type=float, default=0.05, help="serving: time per group and tick")
    return ap.parse_args()


def peaks():
    try:
        with open(MEASURED) as fh:
            m = json.load(fh)
        return float(m["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def workload(args):
    n = args.n
    nu = I.cavity_nu(0.02, n, args.reynolds)
    omega = 1.0 / (3.0 * nu + 0.5)
    return n, omega, I.cavity_flags(n, n, n), {I.LID: (0.02, 0.0, 0.0)}


def config_dict(args, world):
    return {"workload": workload_name(args), "lattice": f"D3Q{args.lattice}", "n": args.n,
            "scheme": args.scheme, "layout": "soa", "collision": args.collision, "reynolds": args.reynolds,
            "parallelism": f"replicas x{world}",
            "l2": "no flush: population state larger than L2 (inputs larger than L2)"}


def workload_name(args):
    return (f"D3Q{args.lattice} lid-driven cavity {args.n}^3 {args.precision.upper()}, Re {args.reynolds:g}, "
            f"{args.scheme} scheme, SoA, {args.collision}")


class Clocks:
    """nvidia-smi sampler running during the timed region."""

    def __init__(self, index, directory=None):
        self.index = index
        self.proc = None
        # raw samples; only their summary goes into the JSON line
        self.path = os.path.join(directory or tempfile.gettempdir(), f"clocks_rank{index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
                 "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                 "clocks_event_reasons.sw_power_cap", "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                p = [x.strip() for x in line.split(",")]
                if len(p) < 7:
                    continue
                try:
                    sm.append(float(p[0]))
                    smax = float(p[1])
                except ValueError:
                    continue
                for name, v in zip(names, p[3:7]):
                    if v.lower() == "active":
                        reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(value, device):
    """Slowest rank's value (the timing rule: the job is as fast as its slowest replica)."""
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_mlups(world, cells_per_rank, steps, max_ms):
    """Whole-job throughput: all ranks' cell updates over the slowest rank's time."""
    return world * cells_per_rank * steps / (max_ms * 1e-3) / 1e6


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "native" else "gloo"
        dist.init_process_group(backend=backend)
        pg = dist
    return world, rank, local, pg


def time_native(args, rank, local, pg):
    import torch

    from paper_2010_11751_b300 import lbm as L

    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    n, omega, flags, walls = workload(args)
    N = n ** 3
    g = L.Lattice(args.lattice, n, n, n, args.scheme, args.collision, omega, flags,
                  precision=L.PRECISIONS[args.precision], wall_velocities=walls, stream=stream.cuda_stream)
    g.init_equilibrium()
    g.step(args.warmup)
    torch.cuda.synchronize()
    if pg is not None:
        pg.barrier()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    with Clocks(local, args.clocks_dir) as clk:
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            evs[0].record(stream)
            for s in range(args.steps):
                g.step(1)
                evs[s + 1].record(stream)
        torch.cuda.synchronize()
    per = [evs[s].elapsed_time(evs[s + 1]) for s in range(args.steps)]
    total_ms = evs[0].elapsed_time(evs[-1])
    if pg is not None:
        total_ms = max_over_ranks(total_ms, "cuda")
    m, e = g.reduce()
    bpc = g.bytes_per_cell_update
    # step kinds alternate for AA (even: local, odd: neighbour pull/push); the first timed
    # step has the parity of the warm-up count
    first = args.warmup % 2
    odd = [t for s, t in enumerate(per) if (first + s) % 2 == 1]
    even = [t for s, t in enumerate(per) if (first + s) % 2 == 0]
    launches_per_step = L.lbm_kernels_per_step(g.h)
    res = dict(N=N, fluid=int((flags == 0).sum()), total_ms=total_ms, per=per, odd=odd, even=even, bpc=bpc,
               mass=m, energy=e,
               clocks=clk.summary(), launches=args.steps * launches_per_step, kernels_per_step=launches_per_step)
    g.close()
    if not args.no_e2e:
        res["e2e"] = e2e_native(args, L, torch)
    return res


def e2e_native(args, L, torch):
    """Same metric through the public C ABI with host buffers: host (rho, u) -> init, K x
    lbm_step_sums_async(1) (one step and the FP64 conserved sums of the state it read, copied to
    pinned host memory; the host reads and checks each step's sums while the next step runs),
    host (rho, u) read back at the end."""
    n, omega, flags, walls = workload(args)
    N = n ** 3
    rho = torch.ones(N, dtype=torch.float64).pin_memory()
    u = torch.zeros(3 * N, dtype=torch.float64).pin_memory()
    rho_out = torch.empty(N, dtype=torch.float64).pin_memory()
    u_out = torch.empty(3 * N, dtype=torch.float64).pin_memory()
    g = L.Lattice(args.lattice, n, n, n, args.scheme, args.collision, omega, flags,
                  precision=L.PRECISIONS[args.precision], wall_velocities=walls)
    g.init_equilibrium(rho, u)  # first call allocates; not timed
    g.step(args.warmup)
    g.reduce()
    torch.cuda.synchronize()
    sums = torch.empty((2, 2), dtype=torch.float64).pin_memory()
    done = [torch.cuda.Event(), torch.cuda.Event()]
    t0 = time.perf_counter()
    g.init_equilibrium(rho, u)
    for i in range(args.steps):
        # step i, and the FP64 mass and energy of the state it read, into pinned host memory
        g.step_sums_async(sums[i % 2])
        done[i % 2].record()
        if i > 0:
            # the previous step's sums, read on the host while step i runs
            done[(i - 1) % 2].synchronize()
            m, e = sums[(i - 1) % 2].tolist()
            if not (math.isfinite(m) and math.isfinite(e)):
                raise RuntimeError(f"diverged at step {i - 1}")
    done[(args.steps - 1) % 2].synchronize()
    m, e = sums[(args.steps - 1) % 2].tolist()
    if not (math.isfinite(m) and math.isfinite(e)):
        raise RuntimeError("diverged at the last step")
    g.macroscopic(rho_out, u_out)
    t1 = time.perf_counter()
    g.close()
    mlups = N * args.steps / (t1 - t0) / 1e6
    return {"value": round(mlups, 2), "unit": "MLUPS", "h2d_bytes_per_step": int(32 * N / args.steps),
            "d2h_bytes_per_step": int(16 + 32 * N / args.steps),
            "note": "host rho/u upload, K x lbm_step_sums_async(1) (step + FP64 mass/energy of the state it "
                    "read, copied to pinned host memory and checked on the host while the next step runs), "
                    "host rho/u download"}


def oracle_baseline(args, seconds, max_steps=None, warmup=0):
    """The FP64 CPU oracle, as it stands, on the host cores: same workload, full lattice."""
    import ctypes

    from oracle import oracle as O

    n, omega, flags, walls = workload(args)
    N = n ** 3
    threads = os.cpu_count() or 1
    lat = O.Lattice(args.lattice, n, n, n, flags, args.collision, O.params(omega), walls)
    lat.init_equilibrium()
    out = np.zeros_like(lat.f)
    lib = O.lib()
    fl = lat.flags.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
    steps, t_total = 0, 0.0
    cur, nxt = lat.f, out
    for _ in range(warmup):
        lib.orc_step(args.lattice, n, n, n, fl, O._dp(lat.wall_u), O.MODELS[args.collision], O._dp(lat.prm),
                     None, None, threads, O._dp(cur), O._dp(nxt))
        cur, nxt = nxt, cur
    while t_total < seconds and (max_steps is None or steps < max_steps):
        t0 = time.perf_counter()
        rc = lib.orc_step(args.lattice, n, n, n, fl, O._dp(lat.wall_u), O.MODELS[args.collision], O._dp(lat.prm),
                          None, None, threads, O._dp(cur), O._dp(nxt))
        t_total += time.perf_counter() - t0
        if rc != 0:
            raise RuntimeError("oracle step failed")
        cur, nxt = nxt, cur
        steps += 1
    return {"value": round(N * steps / t_total / 1e6, 3), "unit": "MLUPS", "cores": threads, "kind": "oracle",
            "sample": f"{steps} full {n}^3 time steps of the same workload ({N * steps} cell updates, "
                      f"{t_total:.1f} s)"}, steps, t_total


def matrix(args):
    """Every scheme x collision x lattice of the 256^3 cavity (FP64), a few steps each."""
    import torch

    from paper_2010_11751_b300 import lbm as L

    n, omega, flags, walls = workload(args)
    hbm, _ = peaks()
    rows = []
    for Q in (19, 27):
        for scheme in ("twopop", "swap", "aa", "esotwist"):
            for coll in ("BGK_W2", "TRT", "RR", "K"):
                stream = torch.cuda.Stream()
                g = L.Lattice(Q, n, n, n, scheme, coll, omega, flags, wall_velocities=walls,
                              stream=stream.cuda_stream)
                g.init_equilibrium()
                g.step(2)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                e0.record(stream)
                g.step(args.matrix_steps)
                e1.record(stream)
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / args.matrix_steps
                mlups = n ** 3 / (ms * 1e-3) / 1e6
                gbs = g.bytes_per_cell_update * n ** 3 / (ms * 1e-3) / 1e9
                rows.append({"lattice": f"D3Q{Q}", "scheme": scheme, "collision": coll, "mlups": round(mlups, 1),
                             "ms_per_step": round(ms, 3), "hbm_gbs": round(gbs, 1), "hbm_frac": round(gbs / hbm, 3)})
                g.close()
                del stream
    return rows


def precision_form(args):
    """D3Q19 AA 512^3, periodic Taylor-Green (u0 0.05, Re 1000) and cavity (Re 1000): populations
    stored shifted in FP32 and FP16 with FP32 arithmetic, against the FP64 mode (itself checked
    against the FP64 oracle), relative L2 velocity error after form_steps steps."""
    import torch

    from paper_2010_11751_b300 import lbm as L

    n = args.n
    N = n ** 3
    hbm, _ = peaks()
    out = []
    for wl in ("taylor_green", "cavity"):
        if wl == "taylor_green":
            u0 = 0.05
            nu = u0 * n / 1000.0
            flags = I.periodic_flags(n, n, n)
            walls = {}
            rho_t, u_t = I.taylor_green_fields_torch(n, n, n, u0)
        else:
            nu = I.cavity_nu(0.02, n, 1000.0)
            flags = I.cavity_flags(n, n, n)
            walls = {I.LID: (0.02, 0.0, 0.0)}
            rho_t = u_t = None
        omega = 1.0 / (3.0 * nu + 0.5)
        coll = "BGK_W2" if wl == "taylor_green" else "TRT"
        fluid = torch.from_numpy(flags == 0).cuda()
        res = {}
        for prec in ("f64", "f32", "f16"):
            g = L.Lattice(19, n, n, n, "aa", coll, omega, flags, precision=L.PRECISIONS[prec], wall_velocities=walls)
            g.init_equilibrium(rho_t, u_t)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            g.step(args.form_steps)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / args.form_steps
            uu = torch.empty(3 * N, dtype=torch.float64, device="cuda")
            g.macroscopic(None, uu)
            res[prec] = (uu.view(3, N), ms, g.bytes_per_cell_update)
            g.close()
        uref = res["f64"][0][:, fluid]
        for prec in ("f64", "f32", "f16"):
            uu, ms, bpc = res[prec]
            d = uu[:, fluid] - uref
            err = float(torch.sqrt((d * d).sum() / (uref * uref).sum()))
            gbs = bpc * N / (ms * 1e-3) / 1e9
            out.append({"workload": wl, "collision": coll, "precision": prec, "steps": args.form_steps,
                        "mlups": round(N / (ms * 1e-3) / 1e6, 1), "ms_per_step": round(ms, 4),
                        "hbm_gbs": round(gbs, 1), "hbm_frac": round(gbs / hbm, 4),
                        "l2_rel_velocity_error_vs_f64": err})
        del res, uref
        torch.cuda.empty_cache()
    return out


def batching_form(args):
    """256 independent D3Q19 cavities, sides uniform in [16, 96] (non-cubic), Re uniform in
    [100, 1000] (nu = u nx / Re), TRT, FP32 shifted storage, AA: the plain per-lattice launch
    loop against one launch per step for the whole batch (autotuned, CUDA graph)."""
    import torch

    from paper_2010_11751_b300 import lbm as L

    steps = args.form_steps
    specs = I.batch_cavities(256, 16, 96, 100.0, 1000.0)
    lid = {I.LID: (0.02, 0.0, 0.0)}

    def make():
        lats = []
        for nx, ny, nz, re in specs:
            omega = 1.0 / (3.0 * I.cavity_nu(0.02, nx, re) + 0.5)
            g = L.Lattice(19, nx, ny, nz, "aa", "TRT", omega, I.cavity_flags(nx, ny, nz), precision=L.F32,
                          wall_velocities=lid)
            g.init_equilibrium()
            lats.append(g)
        return lats

    cells = sum(a * b * c for a, b, c, _ in specs)
    res = {"members": len(specs), "cells": cells, "steps": steps}
    # plain per-lattice launch loop: each lattice advanced by its own launches, one after the other
    lats = make()
    for g in lats:
        g.step(2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for g in lats:
        g.step(steps)
    torch.cuda.synchronize()
    t_loop = time.perf_counter() - t0
    loop_pops = [g.get_populations() for g in lats[:4]]
    for g in lats:
        g.close()
    res["per_lattice_loop_mlups"] = round(cells * steps / t_loop / 1e6, 1)
    # batched: one launch per step for all 256 lattices, captured in a CUDA graph
    lats = make()
    with L.Batch(lats) as b:
        b.step(2, use_graph=False)
        tb0 = time.perf_counter()
        thr, cpt = b.autotune()
        t_tune = time.perf_counter() - tb0
        tuned_steps = lats[0].steps_done - 2
        b.step(steps, use_graph=True)  # capture + first replay (not timed)
        b.sync()
        t0 = time.perf_counter()
        b.step(steps, use_graph=True)
        b.sync()
        t_batch = time.perf_counter() - t0
        same = None
        if tuned_steps == 0:
            same = all(np.array_equal(g.get_populations(), ref) for g, ref in zip(lats[:4], loop_pops))
    for g in lats:
        g.close()
    res.update({"batched_graph_mlups": round(cells * steps / t_batch / 1e6, 1), "autotuned_threads": thr,
                "autotuned_cells_per_thread": cpt, "autotune_seconds": round(t_tune, 2),
                "speedup_vs_loop": round(t_loop / t_batch, 3),
                "note": "bit-identity of batched and per-lattice results is checked in tests/test_gpu_batch.py"})
    hbm, _ = peaks()
    res["batched_hbm_frac"] = round(2 * 19 * 4 * cells * steps / t_batch / 1e9 / hbm, 4)
    return res


def size_sweep(args):
    """Performance against domain size (the paper's N-dependence study, Section 3.3.3): D3Q19
    cavity N^3 for N = 16..320, AA and two-population, BGK-W2 and RR, at the given precision."""
    import torch

    from paper_2010_11751_b300 import lbm as L

    rows = []
    for n in (16, 24, 32, 48, 64, 96, 128, 160, 192, 224, 256, 320):
        args.n = n
        _, omega, flags, walls = workload(args)
        for scheme in ("aa", "twopop"):
            for coll in ("BGK_W2", "RR"):
                stream = torch.cuda.Stream()
                g = L.Lattice(19, n, n, n, scheme, coll, omega, flags, precision=L.PRECISIONS[args.precision],
                              wall_velocities=walls, stream=stream.cuda_stream)
                g.init_equilibrium()
                steps = max(4, min(200, int(2e9 // n ** 3)))
                g.step(4)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                e0.record(stream)
                g.step(steps)
                e1.record(stream)
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / steps
                rows.append({"n": n, "scheme": scheme, "collision": coll, "steps": steps,
                             "mlups": round(n ** 3 / (ms * 1e-3) / 1e6, 1)})
                g.close()
    return rows


def unrolling_form(args):
    """The loop-unrolling study of Section 4 (BGK-W2, AA-SoA, N = 128, and here 256 too): the
    unrolled BGK-W2 kernels against BGK-W2 in the educational form (loops over the directions,
    tabulated c_k and t_k), compiled as the compiler chooses, and with the loops kept rolled."""
    import torch

    from paper_2010_11751_b300 import lbm as L

    rows = []
    for prec in ("f64", "f32"):
        for n in (128, 256):
            args.n = n
            _, omega, flags, walls = workload(args)
            for coll in ("BGK_W2", "BGK_W2_EDU", "BGK_W2_LOOP"):
                stream = torch.cuda.Stream()
                g = L.Lattice(19, n, n, n, "aa", coll, omega, flags, precision=L.PRECISIONS[prec],
                              wall_velocities=walls, stream=stream.cuda_stream)
                g.init_equilibrium()
                steps = 200 if prec == "f32" else 50
                g.step(6)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                e0.record(stream)
                g.step(steps)
                e1.record(stream)
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / steps
                rows.append({"precision": prec, "n": n, "collision": coll, "steps": steps,
                             "mlups": round(n ** 3 / (ms * 1e-3) / 1e6, 1)})
                g.close()
    for r in rows:
        base = next(b for b in rows if b["precision"] == r["precision"] and b["n"] == r["n"]
                    and b["collision"] == "BGK_W2")
        r["unrolled_speedup"] = round(base["mlups"] / r["mlups"], 3)
    return rows


def time_config(Q, n, scheme, coll, prec, steps, warmup=4, reynolds=1000.0):
    """ms per step of one lattice-driven cavity configuration (CUDA events on its stream)."""
    import torch

    from paper_2010_11751_b300 import lbm as L

    omega = 1.0 / (3.0 * I.cavity_nu(0.02, n, reynolds) + 0.5)
    stream = torch.cuda.Stream()
    g = L.Lattice(Q, n, n, n, scheme, coll, omega, I.cavity_flags(n, n, n), precision=L.PRECISIONS[prec],
                  wall_velocities={I.LID: (0.02, 0.0, 0.0)}, stream=stream.cuda_stream)
    g.init_equilibrium()
    g.step(warmup)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    g.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    bpc = g.bytes_per_cell_update
    g.close()
    del stream
    torch.cuda.empty_cache()
    return ms, bpc


def forms(args):
    """The forms beside the headline, measured after its timed region: the D3Q27 FP64 cavity, the
    precision form at 512^3 (FP32/FP16 shifted storage against the FP64 mode), the batching form
    (256 uneven cavities: per-lattice loop against one launch per step) and the serving form (a short
    trace, continuous batching against a FIFO queue, over and below capacity)."""
    import copy

    hbm, _ = peaks()
    out = {}
    t0 = time.perf_counter()
    ms, bpc = time_config(27, 256, "aa", "BGK_W2", "f64", 20)
    n3 = 256 ** 3
    out["d3q27_cavity256_f64_aa_bgk_w2"] = {"mlups": round(n3 / (ms * 1e-3) / 1e6, 1), "ms_per_step": round(ms, 4),
                                           "hbm_frac": round(bpc * n3 / (ms * 1e-3) / 1e9 / hbm, 4)}
    a = copy.copy(args)
    a.n, a.form_steps = 512, 200
    out["precision_512"] = {"steps": a.form_steps, "rows": precision_form(a)}
    a = copy.copy(args)
    a.form_steps = 100
    out["batching"] = batching_form(a)
    out["serving"] = serving_compact(args)
    out["seconds"] = round(time.perf_counter() - t0, 1)
    return out


def serving_compact(args, count=40):
    """A short serving trace (count requests, the configured mix), replayed over capacity (Poisson
    args.rate/s) and below it (60 % of the request rate the over-capacity replay sustained), each by
    continuous batching (least remaining work first, an active-cell budget of args.slot_cells, ticks of
    args.tick_seconds per group) and by a plain FIFO
    queue (one solve at a time).  A sample of the FP32 requests is re-run alone in FP64 (the mode
    the parity tests tie to the oracle) for the served results' error."""
    import torch

    from paper_2010_11751_b300.serve import GpuBackend, Scheduler, summarize, trace_requests

    modes = (("continuous_batching", dict(policy="shortest", tick_seconds=args.tick_seconds,
                                          max_active_cells=args.slot_cells)),
             ("fifo_queue_one_at_a_time", dict(policy="fifo", max_active=1)))
    out = {"requests": count, "rows": []}
    rate = args.rate
    served = None
    for label in ("over_capacity", "below_capacity"):
        trace = trace_requests(I.serving_trace(count, rate), reynolds=100.0)
        for mode, kw in modes:
            be = GpuBackend()
            sched = Scheduler(be, tick_steps=args.tick, reserve_bytes=8 << 30, **kw)
            t0 = time.perf_counter()
            res = sched.run(trace)
            wall = time.perf_counter() - t0
            be.close()
            torch.cuda.empty_cache()
            summ = summarize(res, wall)
            summ.update({"trace": label, "mode": mode, "rate_hz": round(rate, 4), "ticks": sched.ticks,
                         "max_active": sched.max_active})
            if summ["failed"]:
                summ["errors"] = sorted({r.error for r in res if r.error is not None})
            out["rows"].append(summ)
            if mode == "continuous_batching" and label == "over_capacity":
                served = (trace, res)
                cap = summ["completed"] / wall
        rate = 0.6 * cap
    # each request of the over-capacity trace alone on the GPU: its service time without any
    # queueing or sharing (the floor of any scheduler's latency)
    trace, res = served
    be = GpuBackend()
    alone = []
    for q in trace:
        g = be.make_lattice(q)
        torch.cuda.synchronize()
        ta = time.perf_counter()
        g.step(q.steps)
        torch.cuda.synchronize()
        alone.append(time.perf_counter() - ta)
        g.close()
    be.close()
    out["alone_service_s"] = {"p50": float(np.percentile(alone, 50)), "p99": float(np.percentile(alone, 99)),
                              "mean": float(np.mean(alone))}
    # error of served FP32 results against the same request alone in FP64
    f32 = sorted((q for q in trace if q.precision == "f32"), key=lambda q: q.side ** 3 * q.steps)[:4]
    be = GpuBackend()
    errs = []
    for q in f32:
        r = next(x for x in res if x.id == q.id)
        ref = dataclasses_replace(q, precision="f64")
        g = be.make_lattice(ref)
        g.step(ref.steps)
        prof = be.read_result(g)["profile"]
        g.close()
        errs.append({"id": q.id, "lattice": q.lattice, "workload": q.workload, "collision": q.collision,
                     "side": q.side, "steps": q.steps,
                     "l2_rel_profile_error_vs_f64": float(np.linalg.norm(r.profile - prof) / np.linalg.norm(prof))})
    be.close()
    out["f32_error_vs_f64_mode"] = errs
    return out


def dataclasses_replace(obj, **kw):
    import dataclasses

    return dataclasses.replace(obj, **kw)


def sm_count():
    import torch

    return torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count


def roofline(args, r, dom_ms, hbm, src):
    """Roofline of the dominant step kernel: HBM bytes per cell update, or FP64 pipe operations for
    the FP64 operators bound by that pipe (with the HBM fraction beside)."""
    N = r["N"]
    achieved = r["bpc"] * N / (dom_ms * 1e-3) / 1e9
    ops = FP64_OPS_PER_FLUID_CELL.get((args.lattice, args.collision)) if args.precision == "f64" else None
    fluid = (args.n - 2) ** 3
    clk = (r["clocks"].get("sm_max_mhz") or 2032.0) * 1e6
    sms = sm_count()
    fp64_peak = FP64_OPS_PER_SM_CLK * sms * clk / 1e9
    if ops is not None and args.collision not in FP64_OFF_PIPE:
        nops = sum(ops)
        rate = nops * fluid / (dom_ms * 1e-3) / 1e9
        flops = ops[0] + ops[1] + 2 * ops[2]
        roof = {"bound": "alu", "achieved": round(rate, 1), "peak": round(fp64_peak, 1), "unit": "G FP64 op/s",
                "frac": round(rate / fp64_peak, 4), "traffic": None,
                "peak_source": f"derived: {FP64_OPS_PER_SM_CLK} FP64 operations (DADD, DMUL or DFMA) per SM per "
                               f"clock x {sms} SMs x max SM clock",
                "fp64_ops_per_fluid_cell": round(nops, 2), "flops_per_fluid_cell": round(flops, 2),
                "hbm_achieved_gbs": round(achieved, 1), "hbm_frac": round(achieved / hbm, 4)}
    else:
        roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                "frac": round(achieved / hbm, 4), "traffic": None, "peak_source": f"{src} hbm_gbs"}
        if ops is not None:
            nops = sum(ops)
            rate = nops * fluid / (dom_ms * 1e-3) / 1e9
            roof["fp64_pipe"] = {"ops_per_fluid_cell": round(nops, 2), "achieved": round(rate, 1),
                                 "peak": round(fp64_peak, 1), "unit": "G FP64 op/s",
                                 "frac": round(rate / fp64_peak, 4)}
    tr = TRAFFIC.get((args.precision, args.lattice, args.collision, args.scheme))
    if tr is not None and tr[2] == kernel_source_hash():
        _, _, flags, _ = workload(args)
        bulk, listed = bulk_and_listed(flags, args.n, args.lattice)
        roof["traffic"] = int(round(tr[0] * bulk + tr[1] * listed))
        roof["traffic_source"] = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of the AA-odd staged and "
                                  "listed-cell launches at 128^3, per cell each updates, scaled by this lattice's "
                                  f"{bulk} bulk and {listed} listed cells")
    roof["kernel"] = f"{args.scheme} step" + (" (odd: neighbour pull/push)" if args.scheme == "aa" else "")
    if r.get("kernels_per_step", 1) == 2:
        roof["kernel"] += ("; staged bulk-cell kernel with the listed-cell kernel beside it on a second stream, "
                           "timed together per step")
    roof["bytes_per_cell_update"] = r["bpc"]
    return roof


def main():
    args = parse()
    if args.forms == "unrolling":
        print(json.dumps({"form": "unrolling", "config": "D3Q19 cavity, AA, SoA, BGK-W2 unrolled vs educational",
                          "rows": unrolling_form(args)}))
        return
    if args.forms == "sweep":
        print(json.dumps({"form": "size_sweep", "precision": args.precision, "rows": size_sweep(args)}))
        return
    if args.forms == "serving":
        print(json.dumps({"form": "serving", "config": f"{args.trace} requests, Poisson {args.rate:g}/s and below "
                          "capacity, side U[32,192], 100-2000 steps, D3Q19/D3Q27, cavity/TG, BGK/K, FP32/FP64, Re 100",
                          "result": serving_compact(args, count=args.trace)}))
        return
    if args.forms == "batching":
        if args.form_steps == 2000:
            args.form_steps = 500
        print(json.dumps({"form": "batching", "config": "256 D3Q19 cavities, sides U[16,96], Re U[100,1000], TRT, "
                          "FP32, AA", "result": batching_form(args)}))
        return
    if args.forms == "precision":
        print(json.dumps({"form": "precision", "config": f"D3Q19 AA {args.n}^3, FP32/FP16 shifted vs FP64",
                          "rows": precision_form(args)}))
        return
    world, rank, local, pg = dist_setup(args)
    if args.impl == "reference":
        if rank != 0:
            return
        # the oracle takes ~0.9 s per 256^3 step on 16 cores: at most K full steps, and no
        # more than REFERENCE_SECONDS of them, so that the run ends within a few minutes
        W = min(args.warmup, 3)
        base, steps, t = oracle_baseline(args, REFERENCE_SECONDS, max_steps=args.steps, warmup=W)
        line = {"impl": "reference", "metric": f"MLUPS ({workload_name(args)})", "value": base["value"],
                "unit": "MLUPS", "n_gpus": world, "steps": steps, "warmup": W,
                "ms_per_step": round(1e3 * t / steps, 3), "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": args.precision, "data": "synthetic", "config": config_dict(args, world),
                "cpu_baseline": {"value": base["value"], "unit": "MLUPS", "cores": base["cores"], "kind": "oracle",
                                 "sample": base["sample"]},
                "e2e": {"value": base["value"], "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    r = time_native(args, rank, local, pg)
    if rank != 0:
        return
    hbm, src = peaks()
    N, K = r["N"], args.steps
    value = aggregate_mlups(world, N, K, r["total_ms"])
    dominant = r["odd"] if (args.scheme == "aa" and r["odd"]) else r["per"]
    dom_ms = sum(dominant) / len(dominant)
    roof = roofline(args, r, dom_ms, hbm, src)
    line = {
        "metric": f"MLUPS ({workload_name(args)})",
        "value": round(value, 2),
        "unit": "MLUPS",
        "n_gpus": world,
        "steps": K,
        "warmup": args.warmup,
        "ms_per_step": round(r["total_ms"] / K, 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": args.precision,
        "data": "synthetic",
        "config": config_dict(args, world),
        "roofline": roof,
        "hbm_frac_step": round(r["bpc"] * N * K / (r["total_ms"] * 1e-3) / 1e9 / hbm, 4),
        "gpu_launches": r["launches"],
        "clocks": r["clocks"],
        "conserved": {"mass": r["mass"], "energy": r["energy"]},
        # the same throughput counting fluid cells only (walls excluded)
        "fluid_mlups": round(value * r["fluid"] / N, 2),
    }
    if args.scheme == "aa" and r["odd"] and r["even"]:
        line["per_launch_ms"] = {"even": round(sum(r["even"]) / len(r["even"]), 4),
                                 "odd": round(sum(r["odd"]) / len(r["odd"]), 4)}
    if "e2e" in r:
        line["e2e"] = r["e2e"]
    if not args.no_cpu_baseline:
        base, _, _ = oracle_baseline(args, args.cpu_seconds, max_steps=20)
        line["cpu_baseline"] = base
    if args.matrix:
        line["matrix"] = matrix(args)
    if not args.no_forms and world == 1:
        line["forms"] = forms(args)
    print(json.dumps(line))
    if pg is not None:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
