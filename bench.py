#!/usr/bin/env python
"""Benchmark: matrix-free H.v for the J1-J2 Heisenberg model on the periodic
4x8 square lattice (N=32, J1=1, J2=0.5), Sz=0, dim 601,080,390.

One step is one y = H x through the CUDA library on inputs resident in HBM
(x and y are 4.8 GB in FP64, 2.4 GB in FP32: larger than L2, so no flush is
needed between steps).  Reported: Hamiltonian elements applied per second
(value), compulsory-byte HBM GB/s and its roofline fraction for the apply
kernel, Lanczos seconds per iteration, an end-to-end number through the
public API with host buffers, and the CPU oracle timed on a bounded sample.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--form f64|f32]
    python bench.py --impl reference      # the CPU oracle on the host cores
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

LX, LY, J1, J2 = 4, 8, 1.0, 0.5
N, NUP = LX * LY, LX * LY // 2
SEED = 2
METRIC = "Hamiltonian elements applied/s for H.v at N=32 Sz=0 (4x8 J1-J2)"
WORKLOAD = "4x8 periodic J1-J2 Heisenberg (J1=1, J2=0.5), N=32, Sz=0, dim 601080390, y = H x"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def elements_per_matvec(bonds) -> int:
    """dim (diagonal) + sum over bonds of the states whose two spins differ:
    2 C(N-2, nup-1) per bond."""
    return math.comb(N, NUP) + len(bonds) * 2 * math.comb(N - 2, NUP - 1)


class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index, self.samples, self.proc = index, [], None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            p = [v.strip() for v in line.split(",")]
            if len(p) >= 6:
                self.samples.append(p)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=2)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for s in self.samples for k in range(4) if s[2 + k] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(self.samples)}


def cpu_baseline(seconds: float = 12.0):
    """The oracle's sampled-row product (counting index, no stored list) on
    the host cores, on a bounded random sample of rows of this workload."""
    import numpy as np

    import oracle
    from paper_2505_02901_gb300 import workloads as W
    bonds, J = W.square_j1j2(LX, LY, J1, J2)
    dim = math.comb(N, NUP)
    rng = np.random.default_rng(0)
    cores = os.cpu_count() or 1
    n, t_used, total_rows = 64 * cores, 0.0, 0
    while t_used < seconds:
        rows = rng.integers(0, dim, n)
        t0 = time.perf_counter()
        oracle.apply_rows_rng(N, NUP, bonds, J, SEED, rows)
        dt = time.perf_counter() - t0
        t_used += dt
        total_rows += n
        if dt < seconds / 4:
            n *= 2
    rows_per_s = total_rows / t_used
    el_per_row = elements_per_matvec(bonds) / dim
    return {"value": rows_per_s * el_per_row, "unit": "elements/s", "cores": cores, "kind": "oracle",
            "sample": f"{total_rows} random rows of the N=32 block, x from the seeded generator, "
                      f"{t_used:.1f} s (OpenMP over rows)"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    cb = cpu_baseline(seconds=max(5.0, 20.0 / max(1, args.steps + args.warmup)))
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": "elements/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": "bounded row sample"},
            "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": "elements/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--form", default="f32", choices=["f64", "f32"])
    ap.add_argument("--lanczos-steps", type=int, default=10)
    ap.add_argument("--no-cpu", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch

    from paper_2505_02901_gb300 import api, build, workloads as W
    build.build()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    bonds, J = W.square_j1j2(LX, LY, J1, J2)
    basis = api.Basis(N, NUP, bonds)
    ham = api.Hamiltonian(basis, J)
    dim = basis.dim
    dtype = torch.float64 if args.form == "f64" else torch.float32
    esize = 8 if args.form == "f64" else 4
    x = api.random_vector(dim, SEED, dtype)
    y = torch.empty_like(x)
    elements = elements_per_matvec(bonds)
    compulsory = 2 * esize * dim
    stream = torch.cuda.current_stream()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(max(3, args.warmup)):
        ham.apply(x, out=y)
    barrier()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * args.steps)]
    with Clocks(local) as clk:
        barrier()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for k in range(args.steps):
            ev[2 * k].record(stream)
            ham.apply(x, out=y)
            ev[2 * k + 1].record(stream)
        t1.record(stream)
        barrier()
    total_ms = t0.elapsed_time(t1)
    per = [ev[2 * k].elapsed_time(ev[2 * k + 1]) for k in range(args.steps)]
    kern_ms = statistics.mean(per)
    if dist is not None:
        t = torch.tensor([total_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step = total_ms / args.steps
    value = world * elements / (ms_per_step / 1e3)
    hbm, peak_kind = peaks()
    achieved = compulsory / (kern_ms / 1e3) / 1e9

    # Lanczos seconds per iteration (same workload and storage form)
    lz = ham.lanczos(max_iter=args.lanczos_steps, seed=SEED, storage=dtype)
    t_l = time.perf_counter()
    lz = ham.lanczos(max_iter=args.lanczos_steps, seed=SEED, storage=dtype)
    lz_s = (time.perf_counter() - t_l) / max(1, lz["n_iter"])

    # end to end through the public API with pinned host buffers
    xh = x.cpu().pin_memory()
    yh = torch.empty_like(xh).pin_memory()
    xd = torch.empty_like(x)
    e2e_steps = max(2, min(args.steps, 5))
    ham.apply(xd.copy_(xh, non_blocking=True), out=y)
    yh.copy_(y, non_blocking=True)
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(e2e_steps):
        xd.copy_(xh, non_blocking=True)
        ham.apply(xd, out=y)
        yh.copy_(y, non_blocking=True)
    e1.record(stream)
    barrier()
    e2e_ms = e0.elapsed_time(e1) / e2e_steps
    del xh, yh, xd

    line = {
        "metric": METRIC, "value": value, "unit": "elements/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.form == "f64" else "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "form": args.form, "dim": dim, "bonds": len(bonds),
                   "elements_per_matvec": elements, "seed": SEED,
                   "l2": "inputs larger than L2 (x, y %.1f GB each)" % (esize * dim / 1e9),
                   "parallelism": f"replicas{world}"},
        "hbm_gbs_compulsory": achieved,
        "lanczos_s_per_iter": lz_s,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "traffic": None,
                     "note": f"compulsory bytes 2*{esize}*dim per matvec; peak {peak_kind}"},
        "clocks": clk.summary(),
        "e2e": {"value": world * elements / (e2e_ms / 1e3), "unit": "elements/s",
                "h2d_bytes_per_step": esize * dim, "d2h_bytes_per_step": esize * dim},
        "gpu_launches": args.steps,
    }
    if rank == 0 and world == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline()
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
