#!/usr/bin/env python
"""Benchmark: matrix-free H.v for the J1-J2 Heisenberg model on the periodic
4x8 square lattice (N=32, J1=1, J2=0.5), Sz=0, dim 601,080,390.

One step is one y = H x through the CUDA library on inputs resident in HBM
(x and y are 4.8 GB in FP64, 2.4 GB in FP32: larger than L2, so no flush is
needed between steps).  The headline is the FP64 form (the paper's
precision); the FP32-storage form is reported beside it.  Reported:
Hamiltonian elements applied per second (value), compulsory-byte HBM GB/s
and its roofline fraction for the product, Lanczos seconds per iteration,
ground energies with their stated errors for every Lanczos result, an
end-to-end number through the public API with host buffers, and the CPU
oracle timed on a bounded sample.

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
FORM_NOTE = {
    "f32": "FP32 vector storage and FP32 products (Lanczos dots, alpha, beta in FP64-class arithmetic)",
    "f64": ("FP64 vectors in and out (the paper's precision, FP64 tolerance 1e-12 on every parity test); "
            "the product without FP64 arithmetic per element: these couplings are integer multiples of "
            "q = 1/2, so the device takes exact 64-bit fixed-point sums (x rounded to 52 bits of its "
            "largest entry, double-float when a vector's dynamic range asks for it), one FP64 "
            "conversion per row"),
}
# dram__bytes_read.sum + dram__bytes_write.sum of one product launch at this
# workload (ncu, profiles/apply_4x8_*.md); None until measured for the
# kernel as it stands
# FP64: the sum over the product's kernels, captured at 4x7 (the 4x8 workload
# holds too much device memory for a multi-pass capture) and scaled to 4x8
# by rows (profiles/apply64_4x7_passes_full.md)
TRAFFIC = {"f32": 71.64e9, "f64": 3.4073e9 * 601080390 / 40116600}
# the kernels each form's product runs at this workload
KERNEL = {"f32": "k_spmm<12>",
          "f64": "k_x64_stats, k_x64_convert, 2 x k_tpass<PolFX>, k_main<PolFX, 4> (dominant, 56%)"}
# kernels of this library launched per product (FP64: statistics, conversion,
# the fixed-point passes and main kernel, and their double-float instances,
# which return at once)
LAUNCHES = {"f32": 1, "f64": 8}
# GB300 HBM3e nominal bandwidth (the measured copy bandwidth is the peak used)
HBM_NOMINAL_GBS = 7900.0


# ground energies of the Lanczos results, each with its stated error
ENERGIES = {}


class _Null:
    def __enter__(self):
        return self

    def __exit__(self, *a):
        return False


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


def cpu_baseline(seconds: float = 12.0, extras: bool = True):
    """The oracle's sampled-row product (counting index, no stored list) on
    the host cores, on a bounded random sample of rows of this workload;
    with extras, also its one-thread rate and its Lanczos iteration on the
    N=16 chain."""
    import numpy as np

    import oracle
    from paper_2505_02901_gb300 import workloads as W
    bonds, J = W.square_j1j2(LX, LY, J1, J2)
    dim = math.comb(N, NUP)
    rng = np.random.default_rng(0)
    el_per_row = elements_per_matvec(bonds) / dim

    def rate(budget, n):
        t_used, total = 0.0, 0
        while t_used < budget:
            rows = rng.integers(0, dim, n)
            t0 = time.perf_counter()
            oracle.apply_rows_rng(N, NUP, bonds, J, SEED, rows)
            dt = time.perf_counter() - t0
            t_used += dt
            total += n
            if dt < budget / 4:
                n *= 2
        return total, t_used

    cores = oracle.threads()
    total_rows, t_used = rate(seconds, 64 * cores)
    out = {"value": total_rows / t_used * el_per_row, "unit": "elements/s", "cores": cores, "kind": "oracle",
           "seconds": t_used,
           "host": _host_cpu(),
           "sample": f"{total_rows} random rows of the N=32 block, x from the seeded generator, "
                     f"{t_used:.1f} s (OpenMP over rows)"}
    if not extras:
        return out
    # the oracle's Lanczos (FP64, full reorthogonalisation) on the N=16 chain,
    # Sz=0 (dim 12,870), 100 steps, as context for the device's iteration time
    st16 = oracle.enumerate_states(16, 8)
    b16 = W.chain(16)
    t0 = time.perf_counter()
    a16, _ = oracle.lanczos(lambda v: oracle.apply_u1(16, st16, b16, [1.0] * 16, v), st16.size,
                            oracle.rng_normal(1, 0, st16.size), 100)
    lz16 = (time.perf_counter() - t0) / len(a16)
    e16 = float(oracle.tridiag_eigvals(a16, _)[0])
    # one thread on a smaller sample of the same rows, for the per-core rate
    oracle.threads(1)
    try:
        rows1, t1 = rate(max(1.0, seconds / 6), 256)
    finally:
        oracle.threads(cores)
    out.update({"single_core_value": rows1 / t1 * el_per_row, "lanczos_chain16_s_per_iter": lz16,
                "lanczos_chain16_e0": e16})
    out["sample"] += f"; one thread: {rows1} rows, {t1:.1f} s"
    return out


def _host_cpu() -> str:
    """Machine and CPU model of the host, as far as /proc/cpuinfo tells."""
    import platform
    model = ""
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                key = ln.split(":")[0].strip().lower()
                if key in ("model name", "cpu part", "cpu implementer") and ":" in ln:
                    model = (model + " " if model else "") + key + "=" + ln.split(":", 1)[1].strip()
                    if key == "model name" or model.count("=") >= 2:
                        break
    except OSError:
        pass
    return f"{platform.machine()} {os.cpu_count()} cpus {model}".strip()


def _event_time(fn, reps=3):
    """Mean CUDA-event time (ms) of fn() on the current stream after one warm-up."""
    import torch
    fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def max_over_ranks(ms: float, dist=None, device: str = "cuda") -> float:
    """The slowest rank's time (every rank runs the same replica workload)."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, units_per_rank: float, ms: float) -> float:
    """Units all ranks processed per second over the slowest rank's time."""
    return world * units_per_rank / (ms / 1e3)


def _lanczos_steady(ham, dtype, iters, short=2):
    """Seconds per Lanczos iteration in steady state: the wall time of a run
    of short + iters steps minus that of a run of `short` steps (both pay the
    same vector allocation, seeded start vector and normalisation)."""
    import torch
    ham.lanczos(max_iter=short, seed=SEED, storage=dtype)
    ts = []
    for n in (short, short + iters):
        torch.cuda.synchronize()
        t = time.perf_counter()
        info = ham.lanczos(max_iter=n, seed=SEED, storage=dtype)
        ts.append((time.perf_counter() - t, info["n_iter"]))
    return (ts[1][0] - ts[0][0]) / max(1, ts[1][1] - ts[0][1])


def extra_rows(hbm, c5=True):
    """One measurement per remaining hot-path row, each on its own workload:
    batched product (64 uneven instances, 8 FP32 right-hand sides), per-bond
    bilinear forms (14-rung ladder, FP64), symmetric products (6x6 J1-J2,
    k=(0,0) FP64 and k=(pi/3,0) complex128; the square and triangular space
    groups, 288 and 432 elements), the 6x6 U(1) product in FP32
    (dim 9,075,135,300), the paper's N=36 chain U(1) benchmark (product and
    steady-state Lanczos iteration, FP64 and FP32 storage), its N=36 and
    N=40 chain U(1) + lattice benchmarks (translations and reflections) and
    the N=16 chain Lanczos.  Fractions are
    compulsory bytes (vectors read and written once) over time, of the
    measured HBM bandwidth."""
    import numpy as np
    import torch

    from paper_2505_02901_gb300 import api, workloads as W
    out = {}

    def row(name, ms, bytes_, elements=None, **kw):
        d = {"ms": ms, "compulsory_gb": bytes_ / 1e9, "hbm_gbs_compulsory": bytes_ / (ms / 1e3) / 1e9,
             "roofline_frac": bytes_ / (ms / 1e3) / 1e9 / hbm}
        if elements:
            d["elements_per_s"] = elements / (ms / 1e3)
        d.update(kw)
        out[name] = d

    def elems(N, nup, nb):
        return math.comb(N, nup) + nb * 2 * math.comb(N - 2, nup - 1)

    # a9: batched persistent form
    insts = W.batched_instances(64, seed=4)
    hams, xs, ys, el = [], [], [], 0
    for k, d in enumerate(insts):
        h = api.Hamiltonian(api.Basis(d["N"], d["nup"], d["bonds"]), d["J"])
        hams.append(h)
        xs.append(torch.randn(h.dim, 8, dtype=torch.float32, device="cuda"))
        ys.append(torch.empty_like(xs[-1]))
        el += 8 * elems(d["N"], d["nup"], len(d["bonds"]))
    rows_total = sum(h.dim for h in hams)
    ms = _event_time(lambda: api.batch_apply(hams, xs, ys))
    row("a9_batched_64x8_f32", ms, 2 * 4 * 8 * rows_total, el, rows=rows_total, instances=64, nvec=8)
    del hams, xs, ys
    torch.cuda.empty_cache()
    # a8: bilinear forms on the 56-bond ladder
    bl = W.ladder(14, 2)
    h = api.Hamiltonian(api.Basis(28, 14, bl), W.uniform_couplings(56, 3))
    g = api.random_vector(h.dim, 1, torch.float64)
    x = api.random_vector(h.dim, 2, torch.float64)
    ms = _event_time(lambda: h.bilinear(g, x))
    row("a8_bilinear_ladder28_f64", ms, 2 * 8 * h.dim, h.dim * 56, bonds=56)
    ms = _event_time(lambda: h.apply(x))
    row("a5_apply_ladder28_f64", ms, 2 * 8 * h.dim, elems(28, 14, 56))
    del g, x
    torch.cuda.empty_cache()
    # C3 energies: ground state by two FP64 Lanczos passes (200 steps), the
    # backward kernel's dE0/dJ checked by Euler's identity sum_b J_b dE/dJ_b
    # = E0 and by equal derivatives of the two copies of each rung; the
    # FP32-storage ground energy against the FP64 one
    Jl = W.uniform_couplings(56, 3)
    t0 = time.perf_counter()
    e0, psi, info = h.ground_state(max_iter=200, seed=3)
    gs_s = time.perf_counter() - t0
    grad = h.energy_grad(psi)
    e32 = float(h.lanczos(max_iter=200, seed=3, storage=torch.float32)["evals"][0])
    ENERGIES["c3_ladder28"] = {
        "e0_f64": e0, "lanczos_steps": info["n_iter"], "resid_f64": float(info["resid"][0]),
        "ground_state_s": gs_s, "euler_identity_rel_err": abs(float(Jl @ grad) - e0) / abs(e0),
        "rung_copies_max_grad_diff": float(np.abs(grad[28:42] - grad[42:56]).max()),
        "e0_f32_storage": e32, "f32_vs_f64_rel_err": abs(e32 - e0) / abs(e0)}
    del h, psi
    torch.cuda.empty_cache()
    # next row 1: eigenvector and observables -- ground state of the N=28
    # chain (two Lanczos passes, FP64) and its <S0.Sj>, <Sz0 Szj> for all j
    hc = api.Hamiltonian(api.Basis(28, 14, W.chain(28)), [1.0] * 28)
    t0 = time.perf_counter()
    e0, psi, info = hc.ground_state(max_iter=150, seed=SEED)
    gs_s = time.perf_counter() - t0
    pairs = [(0, j) for j in range(28)]
    t0 = time.perf_counter()
    ss = hc.basis.correlations(psi, pairs, "ss")
    ss_ms = (time.perf_counter() - t0) * 1e3
    t0 = time.perf_counter()
    zz = hc.basis.correlations(psi, pairs, "zz")
    zz_ms = (time.perf_counter() - t0) * 1e3
    out["next1_correlations_chain28_f64"] = {
        "ground_state_s": gs_s, "lanczos_steps": info["n_iter"], "e0": e0,
        "ss_ms_28_pairs": ss_ms, "zz_ms_28_pairs": zz_ms, "s0s1_minus_e0_over_n": float(ss[1] - e0 / 28),
        "su2_max_dev": float(np.abs(ss - 3 * zz).max()), "sum_rule": float(ss.sum())}
    del hc, psi
    torch.cuda.empty_cache()
    # next row 2: time evolution (Sec. 3.6.2) -- a domain wall |up..up down..down>
    # in the open ferromagnetic Heisenberg chain, N=28 (dim 40,116,600),
    # evolved to t = 4 by the two-pass Lanczos method
    N28 = 28
    hd = api.Hamiltonian(api.Basis(N28, 14, np.array([(i, i + 1) for i in range(N28 - 1)], dtype=np.int32)),
                         [-1.0] * (N28 - 1))
    psi0 = torch.zeros(hd.dim, dtype=torch.complex128, device="cuda")
    psi0[hd.basis.index((1 << 14) - 1)] = 1.0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    psit, info = hd.evolve(psi0, t=4.0, tol=1e-10, max_iter=300)
    ev_s = time.perf_counter() - t0
    out["next2_evolve_domain_wall_chain28"] = {
        "s": ev_s, "krylov_steps": info["n_iter"], "err_estimate": info["err"],
        "s_per_step_two_passes": ev_s / max(1, info["n_iter"]),
        "norm_deviation": abs(float(psit.norm()) - 1.0), "dim": hd.dim}
    del hd, psi0, psit
    torch.cuda.empty_cache()
    # next row 3: thermodynamics by finite-temperature Lanczos (R random
    # starts through the eight-vector product) on the 4x6 J1-J2 square lattice
    b46, J46 = W.square_j1j2(4, 6)
    hf = api.Hamiltonian(api.Basis(24, 12, b46), J46)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    fa, fb, fn = hf.ftlm(32, 80, SEED)
    ftlm_s = time.perf_counter() - t0
    temps = [0.1, 0.3, 1.0, 3.0]
    Zt, Et, Ct = api.ftlm_thermo(fa, fb, fn, hf.dim, temps)
    out["next3_ftlm_square4x6"] = {
        "s": ftlm_s, "starts": 32, "steps": 80, "dim": hf.dim,
        "s_per_step_of_8_vectors": ftlm_s / (4 * 80),
        "T": temps, "E_per_site": [float(e) / 24 for e in Et], "C_per_site": [float(c) / 24 for c in Ct]}
    del hf
    torch.cuda.empty_cache()
    # a4': symmetric 6x6 blocks
    b6, J6 = W.square_j1j2(6, 6)
    for mx in (0, 1):
        t0 = time.perf_counter()
        basis = api.Basis(36, 18, b6, symmetry=(W.torus_translations(6, 6), W.torus_characters(6, 6, mx, 0)))
        build_s = time.perf_counter() - t0
        h = api.Hamiltonian(basis, J6)
        dt = torch.complex128 if basis.is_complex else torch.float64
        es = 16 if basis.is_complex else 8
        x = torch.randn(basis.dim, dtype=dt, device="cuda")
        y = torch.empty_like(x)
        ms = _event_time(lambda: h.apply(x, out=y), reps=2)
        tag = f"k{mx}0_{'c128' if basis.is_complex else 'f64'}"
        row(f"a4p_sym6x6_{tag}", ms, (2 * es + 10) * basis.dim, dim=basis.dim, basis_build_s=build_s)
        del x, y
        torch.cuda.empty_cache()
        if c5:
            # config 5: 100 Lanczos steps on the momentum block
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            info = h.lanczos(max_iter=100, seed=SEED, storage=dt)
            lz = time.perf_counter() - t0
            ENERGIES[f"c5_sym6x6_{tag}"] = {"e0": float(info["evals"][0]), "lanczos_steps": info["n_iter"],
                                            "resid": float(info["resid"][0]), "s_per_iter": lz / info["n_iter"],
                                            "dim": basis.dim}
        del basis, h
        torch.cuda.empty_cache()
    # next row 4: full space groups of the 36-site tori, fully symmetric irrep
    # (translations times C4v, 288 elements; times C6v, 432 elements)
    for lat in ("square", "triangular"):
        bl, Jl = (b6, J6) if lat == "square" else W.triangular(6)
        perms = W.space_group(6, 6, lat)
        t0 = time.perf_counter()
        basis = api.Basis(36, 18, bl, symmetry=(perms, W.space_group_characters(6, 6, lat)))
        build_s = time.perf_counter() - t0
        h = api.Hamiltonian(basis, Jl)
        x = torch.randn(basis.dim, dtype=torch.float64, device="cuda")
        y = torch.empty_like(x)
        ms = _event_time(lambda: h.apply(x, out=y), reps=2)
        row(f"next4_space_group_{lat}6x6_f64", ms, (2 * 8 + 10) * basis.dim, dim=basis.dim,
            group=len(perms), bonds=len(bl), basis_build_s=build_s, ns_per_row=ms * 1e6 / basis.dim)
        del basis, h, x, y
        torch.cuda.empty_cache()
    # 6x6 U(1) product, FP32 storage
    h = api.Hamiltonian(api.Basis(36, 18, b6), J6)
    x = api.random_vector(h.dim, 5, torch.float32)
    y = torch.empty_like(x)
    ms = _event_time(lambda: h.apply(x, out=y), reps=2)
    row("a5_apply_6x6_u1_f32", ms, 2 * 4 * h.dim, elems(36, 18, 144), dim=h.dim)
    del x, y
    torch.cuda.empty_cache()
    if c5:
        # config 5: the no-symmetry sector (dim 9,075,135,300) in FP32 vector
        # storage (three 36 GB vectors), 100 Lanczos steps; its ground energy
        # against the lowest of the momentum blocks'
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        info = h.lanczos(max_iter=100, seed=SEED, storage=torch.float32)
        lz = time.perf_counter() - t0
        e_u1 = float(info["evals"][0])
        e_k = min(v["e0"] for k, v in ENERGIES.items() if k.startswith("c5_sym6x6_"))
        ENERGIES["c5_u1_6x6_f32"] = {"e0": e_u1, "lanczos_steps": info["n_iter"], "resid": float(info["resid"][0]),
                                     "s_per_iter": lz / info["n_iter"], "dim": h.dim,
                                     "lowest_momentum_block_e0": e_k,
                                     "rel_diff_to_momentum_blocks": abs(e_u1 - e_k) / abs(e_k)}
    del h
    torch.cuda.empty_cache()
    # The paper's largest U(1) Lanczos benchmark: the N=36 Heisenberg chain,
    # Sz=0 (dim 9,075,135,300), one iteration 3.1 s in FP64 on 2304 cores.
    # FP64 Lanczos keeps three 72.6 GB vectors resident.
    h = api.Hamiltonian(api.Basis(36, 18, W.chain(36)), [1.0] * 36)
    for dt, es, tag in ((torch.float64, 8, "f64"), (torch.float32, 4, "f32")):
        x = api.random_vector(h.dim, 5, dt)
        y = torch.empty_like(x)
        ms = _event_time(lambda: h.apply(x, out=y), reps=2)
        del x, y
        torch.cuda.empty_cache()
        s_it = _lanczos_steady(h, dt, 4)
        torch.cuda.empty_cache()
        row(f"paper_chain36_u1_{tag}", ms, 2 * es * h.dim, elems(36, 18, 36), dim=h.dim,
            lanczos_s_per_iter=s_it, paper_fp64_s_per_iter=3.1,
            paper_hardware="2304 MPI processes (32 x 72-core Xeon Platinum 8360Y)")
    del h
    torch.cuda.empty_cache()
    # The paper's U(1) + lattice Lanczos benchmark at N=36: the chain with its
    # translations and reflections (D_36), fully symmetric irrep (dim
    # 126,068,558, quoted as 1.3e8), one iteration 7.60 s in FP64 on 64 threads.
    # The same at N=40 (dim 1,723,176,308, quoted as 1.7e9): 131 s per iteration.
    for Nc, paper_s in ((36, 7.60), (40, 131.0)):
        t0 = time.perf_counter()
        basis = api.Basis(Nc, Nc // 2, W.chain(Nc),
                          symmetry=(W.chain_dihedral(Nc), W.chain_dihedral_characters(Nc, 0, 1)))
        build_s = time.perf_counter() - t0
        h = api.Hamiltonian(basis, [1.0] * Nc)
        x = torch.randn(basis.dim, dtype=torch.float64, device="cuda")
        y = torch.empty_like(x)
        ms = _event_time(lambda: h.apply(x, out=y), reps=2)
        del x, y
        torch.cuda.empty_cache()
        row(f"paper_chain{Nc}_lattice_f64", ms, (2 * 8 + 10) * basis.dim, dim=basis.dim, group=2 * Nc,
            basis_build_s=build_s, lanczos_s_per_iter=_lanczos_steady(h, torch.float64, 3),
            paper_fp64_s_per_iter=paper_s, paper_hardware="64 OpenMP threads, Xeon Platinum 8360Y")
        del basis, h
        torch.cuda.empty_cache()
    # a6/a7: chain N=16 Lanczos, 100 steps
    h = api.Hamiltonian(api.Basis(16, 8, W.chain(16)), [1.0] * 16)
    h.lanczos(max_iter=100, seed=1)
    t0 = time.perf_counter()
    info = h.lanczos(max_iter=100, seed=1)
    out["a6_a7_lanczos_chain16_f64"] = {"s_per_iter": (time.perf_counter() - t0) / info["n_iter"],
                                        "n_iter": info["n_iter"], "e0": float(info["evals"][0])}
    return out


def run_reference(args):
    """The reference arm: the oracle as it stands on the host cores, W untimed
    and K timed steps, each a bounded random-row sample of the product (the
    sample per step shrinks with K + W so that the run stays near a minute)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from paper_2505_02901_gb300 import workloads as W
    bonds, _ = W.square_j1j2(LX, LY, J1, J2)
    per_step = min(10.0, max(1.0, 60.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        cpu_baseline(seconds=per_step, extras=False)
    rates = [cpu_baseline(seconds=per_step, extras=k == args.steps - 1) for k in range(max(1, args.steps))]
    value = statistics.mean(r["value"] for r in rates)
    step_ms = statistics.mean(r["seconds"] for r in rates) * 1e3
    elements = elements_per_matvec(bonds)
    cb = dict(rates[-1])
    cb["value"] = value
    cb["sample"] = f"{len(rates)} steps of about {per_step:.1f} s each; last: " + rates[-1]["sample"]
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "elements/s",
            "n_gpus": args.gpus, "steps": len(rates), "warmup": args.warmup,
            "ms_per_step": step_ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "ms_per_full_product_extrapolated": elements / value * 1e3,
            "config": {"workload": WORKLOAD, "dim": math.comb(N, NUP), "bonds": len(bonds),
                       "elements_per_matvec": elements, "seed": SEED,
                       "form": ("CPU oracle, FP64; each step is a bounded random sample of rows of the "
                                "product (ms_per_step is that sample's measured time; the full product's "
                                "time, extrapolated, is ms_per_full_product_extrapolated)"),
                       "parallelism": "host cores"},
            "cpu_baseline": cb,
            "e2e": {"value": value, "unit": "elements/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_sym_chain(n: int):
    """The symmetric product on the n-site chain block with D_n, four times."""
    import torch

    from paper_2505_02901_gb300 import api, build, workloads as W
    build.build()
    basis = api.Basis(n, n // 2, W.chain(n),
                      symmetry=(W.chain_dihedral(n), W.chain_dihedral_characters(n, 0, 1)))
    h = api.Hamiltonian(basis, [1.0] * n)
    x = api.random_vector(basis.dim, SEED, torch.float64)
    y = torch.empty_like(x)
    ms = _event_time(lambda: h.apply(x, out=y), reps=3)
    print(json.dumps({"case": "sym-chain", "N": n, "group": 2 * n, "dim": basis.dim, "ms": ms}))
    return 0


def run_space_group(lattice: str, nup: int):
    """The symmetric product on the 36-site torus with its full space group
    (square: translations x C4v, 288 elements, J1-J2; triangular:
    translations x C6v, 432 elements) or its 36 translations alone (J1-J2,
    momentum (0, 0)), fully symmetric irrep, four times."""
    import torch

    from paper_2505_02901_gb300 import api, build, workloads as W
    build.build()
    if lattice == "translations":
        bonds, J = W.square_j1j2(6, 6)
        perms = W.torus_translations(6, 6)
        chi = W.torus_characters(6, 6, 0, 0)
    else:
        bonds, J = W.square_j1j2(6, 6) if lattice == "square" else W.triangular(6)
        perms = W.space_group(6, 6, lattice)
        chi = W.space_group_characters(6, 6, lattice)
    basis = api.Basis(36, nup, bonds, symmetry=(perms, chi))
    h = api.Hamiltonian(basis, J)
    x = api.random_vector(basis.dim, SEED, torch.float64)
    y = torch.empty_like(x)
    ms = _event_time(lambda: h.apply(x, out=y), reps=3)
    print(json.dumps({"case": "space-group", "lattice": lattice, "nup": nup, "group": len(perms),
                      "dim": basis.dim, "ms": ms}))
    return 0


def run_profile_case(case: str):
    """apply8: Y = H X with eight FP32 columns on the benchmark lattice;
    bilinear: per-bond forms <g|S_i.S_j|x> of the 56-bond ladder in FP64;
    batch: the batched product of 64 uneven instances (one fused launch)."""
    import torch

    from paper_2505_02901_gb300 import api, build, workloads as W
    build.build()
    if case == "batch":
        insts = W.batched_instances(64, seed=4)
        hams = [api.Hamiltonian(api.Basis(d["N"], d["nup"], d["bonds"]), d["J"]) for d in insts]
        xs = [torch.stack([api.random_vector(h.dim, 1000 * k + v, torch.float64) for v in range(8)], 1)
              .float().contiguous() for k, h in enumerate(hams)]
        ys = [torch.empty_like(x) for x in xs]
        ms = _event_time(lambda: api.batch_apply(hams, xs, ys), reps=3)
        print(json.dumps({"case": case, "workload": "64 chains and ladders, N 18-28, 8 FP32 vectors each",
                          "rows": sum(h.dim for h in hams), "ms": ms}))
        return 0
    if case == "apply8":
        bonds, J = W.square_j1j2(LX, LY, J1, J2)
        h = api.Hamiltonian(api.Basis(N, NUP, bonds), J)
        x = torch.stack([api.random_vector(h.dim, SEED + c, torch.float32) for c in range(8)], 1).contiguous()
        y = torch.empty_like(x)
        ms = _event_time(lambda: h.apply(x, out=y), reps=3)
        print(json.dumps({"case": case, "workload": WORKLOAD, "nvec": 8, "ms": ms}))
    else:
        h = api.Hamiltonian(api.Basis(28, 14, W.ladder(14, 2)), W.uniform_couplings(56, 3))
        g = api.random_vector(h.dim, 1, torch.float64)
        x = api.random_vector(h.dim, 2, torch.float64)
        ms = _event_time(lambda: h.bilinear(g, x), reps=3)
        print(json.dumps({"case": case, "workload": "14-rung ladder, 56 bonds, N=28", "ms": ms}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--form", default="f64", choices=["f64", "f32"])
    ap.add_argument("--no-c5", action="store_true",
                    help="skip the 100-step Lanczos runs of the 6x6 blocks (about four minutes)")
    ap.add_argument("--lanczos-steps", type=int, default=10)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--only", action="store_true", help="time the headline form only")
    ap.add_argument("--no-extras", action="store_true", help="skip the per-row measurements")
    ap.add_argument("--case", default="bench",
                    choices=["bench", "sym-chain", "space-group", "apply8", "bilinear", "batch"],
                    help="single products for profiling captures, four launches each: sym-chain, "
                         "the symmetric product of the N-site chain with its translations and "
                         "reflections (fully symmetric irrep, N from --chain-n); space-group, the "
                         "symmetric product of the 36-site torus with its full space group "
                         "(--group square or triangular) or its translations (--group translations), "
                         "--nup; apply8, the "
                         "eight-vector FP32 product on the --lattice block; bilinear, the per-bond "
                         "forms of the 56-bond ladder (FP64); batch, the batched product of 64 "
                         "chains and ladders with eight FP32 vectors each")
    ap.add_argument("--chain-n", type=int, default=32)
    ap.add_argument("--group", default="square", choices=["square", "triangular", "translations"])
    ap.add_argument("--nup", type=int, default=18)
    ap.add_argument("--lattice", default="4x8",
                    help="LxxLy of the periodic J1-J2 lattice (4x8 is the benchmark; smaller "
                         "ones serve ncu captures, e.g. 4x7)")
    args = ap.parse_args()
    global LX, LY, N, NUP, WORKLOAD
    LX, LY = (int(v) for v in args.lattice.lower().split("x"))
    N, NUP = LX * LY, LX * LY // 2
    if args.lattice != "4x8":
        WORKLOAD = (f"{LX}x{LY} periodic J1-J2 Heisenberg (J1=1, J2=0.5), N={N}, Sz=0, "
                    f"dim {math.comb(N, NUP)}, y = H x")
    if args.impl == "reference":
        return run_reference(args)
    if args.case == "sym-chain":
        return run_sym_chain(args.chain_n)
    if args.case == "space-group":
        return run_space_group(args.group, args.nup)
    if args.case in ("apply8", "bilinear", "batch"):
        return run_profile_case(args.case)

    import numpy as np
    import torch

    from paper_2505_02901_gb300 import api, build, workloads as W
    build.build()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    torch.cuda.synchronize()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    bonds, J = W.square_j1j2(LX, LY, J1, J2)
    basis = api.Basis(N, NUP, bonds)
    ham = api.Hamiltonian(basis, J)
    dim = basis.dim
    elements = elements_per_matvec(bonds)
    stream = torch.cuda.current_stream()
    hbm, peak_kind = peaks()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def time_form(form, steps, warmup, clocks=None):
        """K timed applies on resident inputs; per-launch CUDA events on the
        launching stream; returns (ms per step over the whole region, mean
        kernel ms)."""
        dtype = torch.float64 if form == "f64" else torch.float32
        x = api.random_vector(dim, SEED, dtype)
        y = torch.empty_like(x)
        for _ in range(max(3, warmup)):
            ham.apply(x, out=y)
        barrier()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * steps)]
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        ctx = clocks if clocks is not None else _Null()
        with ctx:
            barrier()
            t0.record(stream)
            for k in range(steps):
                ev[2 * k].record(stream)
                ham.apply(x, out=y)
                ev[2 * k + 1].record(stream)
            t1.record(stream)
            barrier()
        total = max_over_ranks(t0.elapsed_time(t1), dist)
        kern = statistics.mean(ev[2 * k].elapsed_time(ev[2 * k + 1]) for k in range(steps))
        del x, y
        torch.cuda.empty_cache()
        return total / steps, kern

    def lanczos_s_per_iter(form, iters):
        dtype = torch.float64 if form == "f64" else torch.float32
        return _lanczos_steady(ham, dtype, iters)

    forms = {}
    head = args.form
    clk = Clocks(local)
    for form in (["f64", "f32"] if head == "f32" else ["f32", "f64"]) if not args.only else [head]:
        steps = args.steps if form == head else max(3, args.steps // 4)
        ms_step, kern_ms = time_form(form, steps, args.warmup, clk if form == head else None)
        esize = 8 if form == "f64" else 4
        compulsory = 2 * esize * dim
        achieved = compulsory / (kern_ms / 1e3) / 1e9
        forms[form] = {
            "value": whole_job_rate(world, elements, ms_step), "unit": "elements/s", "ms_per_step": ms_step,
            "steps": steps, "kernel_ms": kern_ms, "hbm_gbs_compulsory": achieved,
            "roofline_frac": achieved / hbm,
            "lanczos_s_per_iter": lanczos_s_per_iter(form, args.lanczos_steps),
        }
    fh = forms[head]
    esize = 8 if head == "f64" else 4
    if rank == 0 and world == 1 and args.lattice == "4x8" and not args.only:
        # C2 energies: 200 Lanczos steps from the seeded start in FP64 vectors
        # and in FP32 vector storage (FP64-class dots); their relative
        # difference is the FP32 form's stated error
        c2 = {}
        for form in ("f64", "f32"):
            dtype = torch.float64 if form == "f64" else torch.float32
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            info = ham.lanczos(max_iter=200, seed=SEED, storage=dtype, nev=2)
            c2[form] = (info, time.perf_counter() - t0)
            torch.cuda.empty_cache()
        e64, e32 = float(c2["f64"][0]["evals"][0]), float(c2["f32"][0]["evals"][0])
        ENERGIES["c2_square4x8"] = {
            "e0_f64": e64, "e0_f32_storage": e32, "f32_vs_f64_rel_err": abs(e32 - e64) / abs(e64),
            "e1_f64": float(c2["f64"][0]["evals"][1]), "lanczos_steps": c2["f64"][0]["n_iter"],
            "resid_f64": float(c2["f64"][0]["resid"][0]), "s_f64": c2["f64"][1], "s_f32": c2["f32"][1],
            "e0_per_site": e64 / N}
    # end to end through the public API with pinned host buffers (headline
    # form): every step copies its x up and its y down.  Double-buffered:
    # step k's upload runs on a copy stream while step k-1 computes, and its
    # download on another while step k+1 computes; events order the buffers.
    dtype = torch.float64 if head == "f64" else torch.float32
    xh = api.random_vector(dim, SEED, dtype).cpu().pin_memory()
    yh = [torch.empty_like(xh).pin_memory() for _ in range(2)]
    xd = [torch.empty(dim, dtype=dtype, device="cuda") for _ in range(2)]
    yd = [torch.empty(dim, dtype=dtype, device="cuda") for _ in range(2)]
    s_up, s_comp, s_down = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    x_ready, x_free, y_ready, y_free = ([torch.cuda.Event(), torch.cuda.Event()] for _ in range(4))

    def e2e_run(steps):
        for k in range(steps):
            b = k & 1
            with torch.cuda.stream(s_up):
                if k >= 2:
                    s_up.wait_event(x_free[b])
                xd[b].copy_(xh, non_blocking=True)
                x_ready[b].record(s_up)
            with torch.cuda.stream(s_comp):
                s_comp.wait_event(x_ready[b])
                if k >= 2:
                    s_comp.wait_event(y_free[b])
                ham.apply(xd[b], out=yd[b])
                x_free[b].record(s_comp)
                y_ready[b].record(s_comp)
            with torch.cuda.stream(s_down):
                s_down.wait_event(y_ready[b])
                yh[b].copy_(yd[b], non_blocking=True)
                y_free[b].record(s_down)

    e2e_steps = max(4, min(args.steps, 8))
    e2e_run(2)
    torch.cuda.synchronize()
    barrier()
    t_e2e = time.perf_counter()
    e2e_run(e2e_steps)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks((time.perf_counter() - t_e2e) * 1e3 / e2e_steps, dist)
    del xh, yh, xd, yd

    line = {
        "metric": METRIC, "value": fh["value"], "unit": "elements/s", "n_gpus": world,
        "steps": fh["steps"], "warmup": args.warmup, "ms_per_step": fh["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": head, "data": "synthetic",
        "config": {"workload": WORKLOAD, "form": FORM_NOTE[head], "dim": dim, "bonds": len(bonds),
                   "elements_per_matvec": elements, "seed": SEED,
                   "l2": "inputs larger than L2 (x, y %.1f GB each), no flush" % (esize * dim / 1e9),
                   "parallelism": f"replicas{world}"},
        "hbm_gbs_compulsory": fh["hbm_gbs_compulsory"],
        "lanczos_s_per_iter": fh["lanczos_s_per_iter"],
        "roofline": {"bound": "hbm", "achieved": fh["hbm_gbs_compulsory"], "peak": hbm, "unit": "GB/s",
                     "frac": fh["roofline_frac"], "traffic": TRAFFIC.get(head),
                     "kernel": KERNEL[head], "peak_kind": peak_kind,
                     "frac_of_nominal": fh["hbm_gbs_compulsory"] / HBM_NOMINAL_GBS,
                     "nominal_peak": HBM_NOMINAL_GBS,
                     "note": (f"achieved = compulsory 2*{esize}*dim bytes per H.v / mean CUDA-event time of the "
                              "whole product call (all its kernels); traffic = DRAM bytes of one product "
                              + ("(sum over its kernels, 4x7 capture scaled by rows)" if head == "f64" else
                                 "(one k_spmm launch, full-size capture)"))},
        "forms": forms,
        "clocks": clk.summary(),
        "e2e": {"value": whole_job_rate(world, elements, e2e_ms), "unit": "elements/s",
                "h2d_bytes_per_step": esize * dim, "d2h_bytes_per_step": esize * dim,
                "how": ("public API: torch copy_ of x from pinned host memory to the device, Hamiltonian.apply "
                        "(xd_apply), torch copy_ of y to pinned host memory; double-buffered on two copy "
                        "streams, wall clock over the steps")},
        "gpu_launches": fh["steps"] * LAUNCHES[head],
    }
    if rank == 0 and world == 1 and not args.no_extras and args.lattice == "4x8":
        line["rows"] = extra_rows(hbm, c5=not args.no_c5)
        gpu16 = line["rows"].get("a6_a7_lanczos_chain16_f64", {}).get("e0")
        if gpu16 is not None:
            ENERGIES["c1_chain16"] = {"e0_f64": gpu16, "lanczos_steps": line["rows"]["a6_a7_lanczos_chain16_f64"]["n_iter"]}
    if rank == 0 and world == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline()
        e16 = line["cpu_baseline"].get("lanczos_chain16_e0")
        if e16 is not None and "c1_chain16" in ENERGIES:
            ENERGIES["c1_chain16"].update({"e0_oracle": e16,
                                           "rel_err_vs_oracle": abs(ENERGIES["c1_chain16"]["e0_f64"] - e16) / abs(e16)})
    if ENERGIES:
        line["energies"] = ENERGIES
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
