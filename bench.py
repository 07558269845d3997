#!/usr/bin/env python3
"""k-point solves per second of the mixed-variational band structure.

One step = the whole hot path over one cell: bs_assemble (material fields,
form factors, Gram Cholesky factors, k-monomials) and bs_solve_k over the
workload's wavevectors (per-k builder, reduction to tridiagonal form,
bisection).  Inputs are resident in HBM when the timed region starts; L2
is flushed (a 256 MiB write) between timed steps, outside the timed
events.  Each step is timed with CUDA events on the launching stream.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--config c1|c0]
                  [--impl ours|reference] [--no-cpu-baseline]

For N > 1 (torchrun, one process per GPU) every rank runs an independent
replica of the workload (the method needs no exchange between GPUs);
value = all ranks' k-solves / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "k-point solves/sec at <=1e-6 rel omega err vs FP64 oracle"


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--config", default="c1", choices=["c0", "c1", "c2", "c3", "c4", "modes",
                                                          "mesh", "aniso", "3d"])
    ap.add_argument("--cells", type=int, default=None,
                    help="cells of the config-3 batch (4096) or config-4 evaluation set (1024)")
    ap.add_argument("--weights", default=os.path.join(ROOT, "paper_1310_6380_gb300", "data",
                                                       "warmstart.npz"),
                    help="trained warm-start network (config 4)")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-sub", action="store_true",
                    help="config 1: skip the reduced config-3 and config-4 measurements")
    ap.add_argument("--no-graph", action="store_true",
                    help="config 3: time the plain solve only (no CUDA graph record/replay)")
    ap.add_argument("--cpu-sample-k", type=int, default=6)
    ap.add_argument("--kpoints", type=int, default=None,
                    help="single-cell configs and mode shapes: use the first K wavevectors only "
                         "(small profiling runs)")
    return ap.parse_args()


def workload(name):
    """(cell config, JSON config, precision) of a named workload."""
    from paper_1310_6380_gb300 import cells
    if name == "mesh":
        cell = cells.steel_epoxy_hex_mesh(22)
        cfg = dict(cell=cell, M=5, Q=cells.ibz_path("hex", 70, cell.h1, cell.h2), nbands=18)
        config = {
            "workload": "mesh: the paper's steel/epoxy hexagonal cell (steel cylinder d = 4 mm, "
                        "a = 6.023 mm, SI units) on a seeded jittered triangle mesh of 968 "
                        "elements (2 x 22^2; the paper's meshes have 964-1180), centroid rule, "
                        "M=5 (121 plane waves, n=242), 70 k on the hexagonal IBZ boundary, "
                        "lowest 18 branches, FP64 path",
            "cells": 1, "elements": cell.nel, "k_points": 70, "plane_waves": 121, "n": 242,
            "nbands": 18, "precision": "fp64",
            "l2": "flushed between timed steps (256 MiB write, untimed)",
        }
        return cfg, config, 0
    if name == "aniso":
        cfg = cells.config1()
        cfg["cell"] = cells.anisotropic_cell(cfg["cell"], seed=6380)
        config = {
            "workload": "aniso: the c1 cell (256x256 periodic Voronoi, 1132 phases, seed 1310) "
                        "with every phase a rotated orthotropic material (c11, c22 ~ U[20, 200], "
                        "c66 ~ U[5, 60], c12 ~ U[0, 0.4 sqrt(c11 c22)], orientation ~ U[0, pi), "
                        "seed 6380), full 3N x 3N compliance Gram matrix, M=10 (441 plane "
                        "waves, n=882), 90 k on G-X-M-G, lowest 18 branches, FP64 path",
            "cells": 1, "k_points": 90, "plane_waves": 441, "n": 882, "nbands": 18,
            "precision": "fp64", "l2": "flushed between timed steps (256 MiB write, untimed)",
        }
        return cfg, config, 0
    cfg = cells.config0() if name == "c0" else cells.config1()
    N = (2 * cfg["M"] + 1) ** 2
    desc = {
        "c1": "256x256 periodic Voronoi, 1132 phases (seed 1310), square a=1",
        "c2": "256x256 periodic Voronoi, 1132 phases (seed 1310), square a=1",
        "c0": "32x32 circle r=0.3a, two phases, square a=1",
    }[name]
    path = ("mixed path (FP32 reduction + FP64 Rayleigh-Ritz, tolerance 1e-6)" if name == "c2"
            else "FP64 path")
    config = {
        "workload": f"{name}: {desc}, M={cfg['M']} ({N} plane waves, n={2 * N}), "
                    f"{len(cfg['Q'])} k on G-X-M-G, lowest {cfg['nbands']} branches, {path}",
        "cells": 1, "k_points": len(cfg["Q"]), "plane_waves": N, "n": 2 * N,
        "nbands": cfg["nbands"], "precision": "mixed" if name == "c2" else "fp64",
        "l2": "flushed between timed steps (256 MiB write, untimed)",
    }
    return cfg, config, (1 if name == "c2" else 0)


# ---------------------------------------------------------------- replicas
class Replicas:
    """One independent replica of the workload per rank (the method has no
    exchange between GPUs): rank/world from the launcher's environment, a
    barrier, and the max over ranks of a step time.  backend "nccl" on GPUs;
    "gloo" serves the CPU tests of this logic."""

    def __init__(self, backend="nccl", device=None):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.dist = None
        self.cuda = backend == "nccl"
        if self.world > 1:
            import torch.distributed as dist
            kw = {"device_id": device} if device is not None else {}
            dist.init_process_group(backend, **kw)
            self.dist = dist

    def barrier(self):
        import torch
        if self.cuda:
            torch.cuda.synchronize()
        if self.dist:
            self.dist.barrier()
        if self.cuda:
            torch.cuda.synchronize()

    def max(self, x: float) -> float:
        """max over ranks of a per-rank number (a step time)."""
        if not self.dist:
            return float(x)
        import torch
        t = torch.tensor([float(x)], dtype=torch.float64,
                         device="cuda" if self.cuda else "cpu")
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def value(self, units_per_rank: float, ms: float) -> float:
        """whole-job throughput: every rank's units over the slowest rank's time."""
        return self.world * units_per_rank / (ms / 1e3)

    def close(self):
        if self.dist:
            self.dist.destroy_process_group()
            self.dist = None


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,pci.bus_id,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id=None):
        self.bus_id = bus_id
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 10:
                continue
            if self.bus_id and self.bus_id.lower() not in f[1].lower():
                continue
            rows.append(f)
        os.unlink(self.path)
        if not rows:
            return None
        if not self.bus_id:                    # keep the first GPU listed
            idx0 = rows[0][0]
            rows = [r for r in rows if r[0] == idx0]
        sm = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[6 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": float(rows[0][3]) if rows[0][3].replace(".", "").isdigit() else None,
                "power_w_max": max(float(r[4]) for r in rows if r[4].replace(".", "").isdigit())
                if any(r[4].replace(".", "").isdigit() for r in rows) else None,
                "samples": len(rows), "reasons": reasons}


def device_bus_id(torch):
    try:
        p = torch.cuda.get_device_properties(torch.cuda.current_device())
        return f"{p.pci_domain_id:08X}:{p.pci_bus_id:02X}:{p.pci_device_id:02X}"
    except Exception:
        return None


# ---------------------------------------------------------------- helpers
def measured_peaks():
    """(HBM copy GB/s, bf16 burst TFLOP/s, note) measured on this GPU model;
    the earlier single measurement (6.8 TB/s, 1.9 PFLOP/s) when the file of
    measured peaks is absent."""
    try:
        p = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(p["hbm_gbs"]), float(p["bf16_tflops"]), "measured (MEASURED_PEAKS.json)"
    except Exception:
        return 6800.0, 1900.0, "fallback (no MEASURED_PEAKS.json)"


def device_peaks(torch, bs=None):
    """SM count and maximum SM clock of this device (queried, not assumed),
    the nominal FP64 and FP32 CUDA-core peaks from them (GB300: 2 FP64 FMA
    and 128 FP32 FMA per SM per clock), and, with the library, the FP64
    peak measured by its FMA-chain probe."""
    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    sms = int(p.multi_processor_count)
    mhz = None
    try:
        mhz = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["sm_max_mhz"])
    except Exception:
        try:
            q = subprocess.run(["nvidia-smi", "-i", str(torch.cuda.current_device()),
                                "--query-gpu=clocks.max.sm", "--format=csv,noheader,nounits"],
                               capture_output=True, text=True, timeout=10)
            mhz = float(q.stdout.strip().splitlines()[0])
        except Exception:
            mhz = 2070.0
    out = {"sms": sms, "sm_max_mhz": mhz,
           "fp64_nominal_tflops": sms * 2 * 2 * mhz * 1e6 / 1e12,
           "fp32_nominal_tflops": sms * 128 * 2 * mhz * 1e6 / 1e12}
    if bs is not None:
        out["fp64_probe_tflops"] = bs.bs_probe_fp64(4, 20000)
    return out


def traffic_record(kernel, key="dram_bytes_per_step"):
    """DRAM bytes (`key`) of `kernel` from the committed ncu summary, if the
    kernel's source is unchanged since the counters were taken."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(path))[kernel]
        src = os.path.join(ROOT, "paper_1310_6380_gb300", "csrc", rec["source"])
        if hashlib.sha256(open(src, "rb").read()).hexdigest()[:16] != rec["sha256_16"]:
            return None
        return rec[key]
    except Exception:
        return None


def cpu_oracle_sample(cfg, nk_sample):
    """The FP64 oracle as it stands on this host: cell set-up plus a sample
    of wavevectors; returns (solves/s extrapolated to the full k list,
    sampled indices, sampled omegas, description)."""
    from oracle import mixed_variational as mv
    Q = cfg["Q"]
    idx = np.linspace(0, len(Q) - 1, nk_sample).round().astype(int)
    t0 = time.perf_counter()
    oc = mv.OracleCell(cfg["cell"], cfg["M"])
    t1 = time.perf_counter()
    ws = [oc.omega(Q[i], cfg["nbands"]) for i in idx]
    t2 = time.perf_counter()
    per_k = (t2 - t1) / len(idx)
    total = (t1 - t0) + len(Q) * per_k
    desc = (f"oracle cell set-up ({t1 - t0:.1f} s) + {len(idx)} of {len(Q)} wavevectors "
            f"({per_k:.2f} s each); value extrapolated to all {len(Q)}")
    return len(Q) / total, idx, np.array(ws), desc, t2 - t0


def rel_err(w, ref, cell):
    A = np.array([cell.h1, cell.h2])
    qm = 2 * np.pi * np.linalg.inv(A)
    if getattr(cell, "stiffness", None) is not None:
        c2 = min(np.linalg.eigvalsh(C)[0] / r for C, r in zip(cell.stiffness, cell.rho))
    else:
        c2 = np.min(cell.mu / cell.rho)
    floor = np.sqrt(c2) * min(np.linalg.norm(qm[:, 0]), np.linalg.norm(qm[:, 1])) / 2
    return np.abs(w ** 2 - ref ** 2) / (2 * np.maximum(ref ** 2, floor ** 2))


# ---------------------------------------------------------------- arms
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    if args.config in ("c3", "c4"):
        return run_reference_batch(args)
    cfg, config, _ = workload(args.config)
    cores = len(os.sched_getaffinity(0))
    times, vals = [], []
    for i in range(args.warmup + args.steps):
        v, _, _, desc, secs = cpu_oracle_sample(cfg, 2)
        if i >= args.warmup:
            times.append(secs)
            vals.append(v)
    value = statistics.mean(vals)
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "k-solves/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * statistics.mean(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config,
        "cpu_baseline": {"value": value, "unit": "k-solves/s", "cores": cores, "kind": "oracle",
                         "sample": "each step: " + desc},
        "e2e": {"value": value, "unit": "k-solves/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))


def measure_mixed(bs, torch, args, cell, M, nb, nk, Qd, stream, flush, barrier, dev, ms_fp64,
                  omega_fp64, world):
    """Config 2: the config-1 cell on the mixed path, timed like the main line."""
    hm = bs.bs_create_cell(cell.h1, cell.h2, dev(cell.phase.astype(np.uint16)), dev(cell.lam),
                           dev(cell.mu), dev(cell.rho), M, bs.BS_PREC_MIXED)
    bs.bs_set_profiling(hm, True)
    wm = torch.empty((nk, nb), dtype=torch.float64, device="cuda")
    stm = torch.empty(nk, dtype=torch.int32, device="cuda")
    for _ in range(args.warmup):
        bs.bs_assemble(hm, stream)
        bs.bs_solve_k(hm, Qd, nb, wm, stm, stream)
    barrier()
    times, phs = [], []
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        bs.bs_assemble(hm, stream)
        bs.bs_solve_k(hm, Qd, nb, wm, stm, stream)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        phs.append(bs.bs_phase_times(hm))
    bs.bs_destroy_cell(hm)
    mms = statistics.mean(times)
    om = wm.cpu().numpy()
    return {"config": "c2: the c1 cell, FP32 Householder reduction + FP64 Rayleigh-Ritz "
                      "(tensor-core exact-slice products), tolerance 1e-6",
            "value": world * nk / (mms / 1e3), "unit": "k-solves/s", "ms_per_step": mms,
            "speedup_vs_fp64_path": ms_fp64 / mms,
            "status_nonzero": int(np.count_nonzero(stm.cpu().numpy())),
            "phases_ms": {k: round(statistics.mean(p[k] for p in phs), 3)
                          for k in phs[0]},
            "max_rel_err_vs_fp64_path": float(rel_err(om, omega_fp64, cell).max()),
            "_omega": om}


def slice_slabs(S, Kp, slab_k=4032):
    """Lengths of the slabs of an exact-slice product with S digit planes of
    width Kp: digit order u spans (u + 1) Kp terms, cut at slab_k."""
    out = []
    for u in range(S):
        n = (u + 1) * Kp
        out += [min(slab_k, n - k0) for k0 in range(0, n, slab_k)]
    return out


def measure_tensor(bs, torch, stream, nk, n, b=28, S=7):
    """Tensor-core utilisation of the exact-slice contraction on the shape of the
    mixed path's Rayleigh-Ritz products: per wavevector, the slabs of the
    digit orders of [n x 2b] over K = 2n (their mean length)."""
    gen = torch.Generator(device="cuda").manual_seed(0)
    slabs = slice_slabs(S, (2 * n + 63) // 64 * 64)
    zb, Mg, Ng, Kg = nk * len(slabs), n, 2 * b, sum(slabs) // len(slabs) // 64 * 64
    digits = lambda shape: torch.randint(-64, 65, shape, generator=gen, device="cuda",
                                         dtype=torch.int8).to(torch.bfloat16).view(torch.uint16)
    Ag = digits((zb, Mg, Kg))
    Bg = digits((zb, Ng, Kg))
    Dg = torch.empty((zb, Ng, Mg), dtype=torch.float32, device="cuda")
    for _ in range(2):
        bs.bs_gemm_bf16(Ag, Bg, Dg, stream)
    tcs = []
    for _ in range(3):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        bs.bs_gemm_bf16(Ag, Bg, Dg, stream)
        e1.record(stream)
        e1.synchronize()
        tcs.append(e0.elapsed_time(e1))
    tc_ms = min(tcs)
    _, bf16_peak, note = measured_peaks()
    tflops = 2.0 * zb * Mg * Ng * Kg / (tc_ms / 1e3) / 1e12
    return {"kernel": "slice_gemm_kernel (tcgen05.mma kind::f16, TMA, TMEM)",
            "shape": f"{zb} x [{Mg} x {Ng} x {Kg}] BF16 -> FP32 ({nk} wavevectors x "
                     f"{len(slabs)} digit-order slabs of mean length {Kg})", "ms": tc_ms,
            "achieved_tflops": tflops, "peak_tflops": bf16_peak,
            "peak_source": "bf16 burst, " + note, "frac": tflops / bf16_peak}


def measure_c3(bs, torch, rep, args, ncell, steps, warmup, graph=True, oracle_cells=8,
               cpu_baseline=True):
    """Config 3: a ragged batch of `ncell` cells on the dense mixed path
    (bs_batch_*); returns the JSON dict of its measurement."""
    from paper_1310_6380_gb300 import cells
    world, rank = rep.world, rep.rank
    nk, nb = 30, 10
    cfgs = [cells.config3_cell(i) for i in range(ncell)]
    cargs = [(c["cell"].h1, c["cell"].h2, np.ascontiguousarray(c["cell"].phase, np.uint16),
              c["cell"].lam, c["cell"].mu, c["cell"].rho, c["M"], bs.BS_PREC_MIXED) for c in cfgs]
    Ms = [c["M"] for c in cfgs]
    ns = np.array([2 * (2 * m + 1) ** 2 for m in Ms])
    Qd = torch.tensor(np.stack([c["Q"] for c in cfgs]), device="cuda")
    b = bs.bs_batch_create(cargs, nk, nb)
    w = torch.empty((ncell, nk, nb), dtype=torch.float64, device="cuda")
    st = torch.empty((ncell, nk), dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    barrier = rep.barrier

    def timed(graph):
        bs.bs_batch_set_graph(b, graph)
        bs.bs_batch_set_profiling(b, not graph)
        for _ in range(warmup):
            bs.bs_batch_solve(b, Qd, w, st, stream)
        barrier()
        times, phs = [], []
        for _ in range(steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            bs.bs_batch_solve(b, Qd, w, st, stream)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            if not graph:
                phs.append(bs.bs_batch_phase_times(b))
        barrier()
        return statistics.mean(times), phs

    launches0 = bs.bs_launch_count()
    sampler = ClockSampler(device_bus_id(torch))
    sampler.start()
    ms_plain, phs = timed(False)
    clocks = sampler.stop()
    launches = (bs.bs_launch_count() - launches0) // max(1, steps + warmup)
    ms_graph = timed(True)[0] if graph else None
    ms = ms_plain if ms_graph is None else min(ms_plain, ms_graph)
    ms = rep.max(ms)
    omega = w.cpu().numpy()
    status = st.cpu().numpy()
    ph = {k: statistics.mean(p[k] for p in phs) for k in phs[0]}
    tiles_chosen = bs.bs_batch_tiles(b)
    _, fb_flags = bs.bs_batch_stats(b, ncell * nk)
    bs.bs_batch_destroy(b)

    # end to end through the public API with pinned host buffers: create the
    # batch from host arrays (includes the copies to the device), solve with
    # host wavevectors and outputs (includes the first call's tile tuning), destroy
    hQ = torch.from_numpy(np.stack([c["Q"] for c in cfgs])).pin_memory()
    hw = torch.empty((ncell, nk, nb), dtype=torch.float64).pin_memory()
    hs = torch.empty((ncell, nk), dtype=torch.int32).pin_memory()
    barrier()
    t0 = time.perf_counter()
    for _ in range(steps):
        b2 = bs.bs_batch_create(cargs, nk, nb)
        bs.bs_batch_solve(b2, hQ, hw, hs, stream)
        bs.bs_batch_destroy(b2)
    torch.cuda.synchronize()
    e2e_s = rep.max((time.perf_counter() - t0) / steps)
    h2d = sum(a[2].nbytes + 3 * a[3].nbytes for a in cargs) + hQ.numel() * 8
    e2e = {"value": world * ncell * nk / e2e_s, "unit": "k-solves/s", "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": hw.numel() * 8 + hs.numel() * 4,
           "api": "bs_batch_create (host arrays) + bs_batch_solve (host Q, outputs; first call "
                  "includes tile autotuning) + bs_batch_destroy"}
    # dominant kernel: the FP32 Householder reduction, bound by HBM on the
    # read + write of every trailing triangle
    hbm_peak, _, note = measured_peaks()
    tri_bytes = sum(nk * sum(m * (m + 1) // 2 for m in range(1, int(n))) * 16.0 for n in ns)
    achieved = tri_bytes / (ph["reduction"] / 1e3) / 1e9
    roofline = {"bound": "hbm", "kernel": "tridiag_step_kernel<float> (all launches of one step)",
                "achieved": achieved, "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
                "traffic": None, "peak_source": "copy bandwidth, " + note,
                "algorithmic": "read + write (8 B each) of every trailing lower triangle of "
                               f"{ncell * nk} matrices (n = 242..578)"}
    value = world * ncell * nk / (ms / 1e3)
    out = {
        "metric": METRIC, "value": value, "unit": "k-solves/s", "n_gpus": world,
        "steps": steps, "warmup": warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 reduction, bf16 exact-slice tensor products, f64 refinement",
        "data": "synthetic",
        "config": {"workload": f"c3: {ncell} cells (seeds 6380+i), 64x64 pixels, square/hex, "
                               "ellipse/Voronoi maps with 2-16 phases, M = 5..8 (n = 242..578), "
                               "30 k per cell on its IBZ path, lowest 10 branches, mixed path",
                   "cells": ncell, "k_points": ncell * nk,
                   "cells_per_M": {int(m): Ms.count(m) for m in sorted(set(Ms))},
                   "l2": "flushed between timed steps (256 MiB write, untimed)"},
        "ms_per_step_plain": ms_plain, "ms_per_step_graph": ms_graph,
        "tiles": tiles_chosen, "phases_ms": {k: round(v, 1) for k, v in ph.items()},
        "status_nonzero": int(np.count_nonzero(status)),
        "fp64_fallbacks": int((fb_flags == 1).sum()), "gpu_launches_per_step": launches,
        "gpu_launches": launches * steps, "e2e": e2e, "roofline": roofline, "clocks": clocks,
    }
    if rank == 0 and world == 1 and cpu_baseline and oracle_cells > 0:
        from oracle import mixed_variational as mv
        samp = list(range(0, ncell, max(1, ncell // oracle_cells)))[:oracle_cells]
        t0 = time.perf_counter()
        errs = []
        for i in samp:
            c = cfgs[i]
            oc = mv.OracleCell(c["cell"], c["M"])
            ref = np.array([oc.omega(q, nb) for q in c["Q"]])
            errs.append(rel_err(omega[i], ref, c["cell"]).max())
        secs = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": len(samp) * nk / secs, "unit": "k-solves/s",
                               "cores": len(os.sched_getaffinity(0)), "kind": "oracle",
                               "sample": f"{len(samp)} of the {ncell} cells, all 30 k each "
                                         f"({secs:.1f} s); value = their k-solves / time"}
        out["max_rel_err_vs_oracle"] = float(max(errs))
        out["oracle_sampled_cells"] = samp
    return out


def measure_assembly(bs, torch, stream, cell, M, ph_c1):
    """The form-factor assembly's tensor-core launch (the first separable
    stage, exact-slice digit planes on tcgen05) alone: on the c1 cell (its
    time from the c1 steps' profiling) and on c3-shaped cells (64 x 64
    pixels, M = 8 and M = 5, assembled alone, L2 flushed before each)."""
    from paper_1310_6380_gb300 import cells
    _, bf16_peak, note = measured_peaks()
    S = 7   # digit planes per operand in the assembly

    def figures(P, Mt, ms):
        D = 4 * Mt + 1
        slabs = slice_slabs(S, (P + 63) // 64 * 64)
        issued = 2.0 * (3 * P) * (2 * D) * sum(slabs)
        algo = 3.0 * (4.0 * D * P * P + 8.0 * D * D * P)
        return {"P": P, "M": Mt, "gemm": f"{len(slabs)} digit-order slabs of [{3 * P} x {2 * D}], "
                                         f"{sum(slabs)} BF16 terms in all",
                "ms_per_launch": ms, "issued_bf16_flops": issued,
                "algorithmic_flops_per_cell": algo,
                "issued_tflops": issued / (ms / 1e3) / 1e12,
                "frac_of_bf16_peak": issued / (ms / 1e3) / 1e12 / bf16_peak,
                "algorithmic_tflops": algo / (ms / 1e3) / 1e12}

    out = {"kernel": "slice_gemm_kernel (tcgen05.mma kind::f16, TMA, TMEM), first stage of the "
                     "form factors", "peak_tflops": bf16_peak,
           "peak_source": "bf16 burst, " + note,
           "algorithmic": "3 [4 D P^2 + 8 D^2 P] real flops per cell (both separable stages; the "
                          "second runs in FP64 on CUDA cores); issued = 2 x digit-plane GEMM "
                          "flops of the tensor-core launch",
           "c1": figures(cell.P, M, ph_c1["assembly_tc"])}
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for Mt in (8, 5):
        i = next(i for i in range(200) if cells.config3_cell(i)["M"] == Mt)
        c = cells.config3_cell(i)["cell"]
        h = bs.bs_create_cell(c.h1, c.h2, np.ascontiguousarray(c.phase, np.uint16), c.lam.copy(),
                              c.mu.copy(), c.rho.copy(), Mt, bs.BS_PREC_MIXED)
        try:
            bs.bs_set_profiling(h, True)
            ts = []
            for r in range(8):
                flush.zero_()
                bs.bs_assemble(h, stream)
                t = bs.bs_phase_times(h)["assembly_tc"]
                if r >= 3:
                    ts.append(t)
        finally:
            bs.bs_destroy_cell(h)
        out[f"c3_M{Mt}"] = figures(c.P, Mt, statistics.mean(ts))
    return out


def run_batch(args):
    """Config 3 on its own line (bench.py --config c3)."""
    import torch
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    rep = Replicas("nccl", torch.device("cuda", local))
    from paper_1310_6380_gb300 import binding as bs
    out = measure_c3(bs, torch, rep, args, args.cells, args.steps, args.warmup,
                     graph=not args.no_graph, oracle_cells=8,
                     cpu_baseline=not args.no_cpu_baseline)
    if rep.rank == 0:
        print(json.dumps(out))
    rep.close()


def run_reference_batch(args):
    """The oracle on the host cores for configs 3 and 4: each step solves 2 of
    the batch's cells (all 30 k), value = k-solves / time."""
    from oracle import mixed_variational as mv
    from paper_1310_6380_gb300 import cells
    gen = cells.config3_cell if args.config == "c3" else cells.config4_eval_cell
    ncell = args.cells or (4096 if args.config == "c3" else 1024)
    times, vals = [], []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        nsolve = 0
        for ci in (2 * i, 2 * i + 1):
            c = gen(ci)
            oc = mv.OracleCell(c["cell"], c["M"])
            for q in c["Q"]:
                oc.omega(q, 10)
                nsolve += 1
        secs = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(secs)
            vals.append(nsolve / secs)
    value = statistics.mean(vals)
    cores = len(os.sched_getaffinity(0))
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "k-solves/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * statistics.mean(times), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{args.config}: {ncell} cells, 64x64, M = 5..8, 30 k, 10 branches"},
        "cpu_baseline": {"value": value, "unit": "k-solves/s", "cores": cores, "kind": "oracle",
                         "sample": "each step: 2 cells of the batch, all 30 k each"},
        "e2e": {"value": value, "unit": "k-solves/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0}}))


BAND_NB = 8


def band_roofline(red, n, nk_all, ph, peaks):
    """Roofline of the dominant kernel group of the two-stage reduction (live
    event times per group, summed over the panel steps of one solve; the
    reduction runs the batch in parts on concurrent streams and the events
    bracket the first part's launches, so the work counted is that part's)
    and the reduction's rate on the one-stage flop count (16/3) n^3 per k."""
    hbm_peak, _, note = measured_peaks()
    red = dict(red)
    nk = int(red.pop("matrices"))
    fp64_peak = peaks["fp64_nominal_tflops"]
    nb = BAND_NB
    ms = [n - j - nb for j in range(0, n, nb) if n - j - nb > 1]   # trailing sizes per step
    # algorithmic work of each group for the nk matrices of one solve
    rank2_bytes = nk * sum(32.0 * m * (m + 1) / 2 + 16.0 * m * (m - 1) / 2 for m in ms)
    av_bytes = nk * sum(16.0 * m * m for m in ms)
    tasks = sum((n - 1 - s + nb - 1) // nb for s in range(n - 1))
    chase_flops = nk * tasks * 6.0 * nb * nb * 8.0
    qr_flops = nk * sum(8.0 * 4.0 * m * nb * nb for m in ms)
    w_flops = nk * sum(8.0 * 2.0 * m * nb * nb for m in ms)
    groups = {
        "rank2_update": {"bound": "hbm", "kernel": "pack_rank2_kernel + rank2_update_kernel "
                         "(tcgen05, eight digit orders in TMEM, FP64 epilogue)",
                         "work": rank2_bytes, "unit": "GB/s", "peak": hbm_peak,
                         "peak_source": "copy bandwidth, " + note,
                         "algorithmic": "read + write (16 B each) of the trailing lower "
                                        "triangle and write of its mirror, per panel step"},
        "a22_v": {"bound": "hbm", "kernel": "pack_trail_kernel + slice_gemm_kernel (A22 V) + "
                  "recombine", "work": av_bytes, "unit": "GB/s", "peak": hbm_peak,
                  "peak_source": "copy bandwidth, " + note,
                  "algorithmic": "one read (16 B) of the trailing block per panel step"},
        "bulge_chase": {"bound": "alu", "kernel": "bulge_kernel (band 8 -> tridiagonal, FP64)",
                        "work": chase_flops, "unit": "TFLOP/s", "peak": fp64_peak,
                        "peak_source": "nominal FP64", "algorithmic":
                        "6 nb^2 complex multiply-adds per chase task (one-sided products of "
                        "the off-diagonal block on both sides, two-sided diagonal block)"},
        "panel_qr": {"bound": "alu", "kernel": "panel_qr_kernel (FP64)", "work": qr_flops,
                     "unit": "TFLOP/s", "peak": fp64_peak, "peak_source": "nominal FP64",
                     "algorithmic": "Householder QR of an m x 8 complex panel, 4 m nb^2 "
                                    "complex multiply-adds"},
        "w_form": {"bound": "alu", "kernel": "wz_kernel + wrow_kernel (FP64)", "work": w_flops,
                   "unit": "TFLOP/s", "peak": fp64_peak, "peak_source": "nominal FP64",
                   "algorithmic": "2 m nb^2 complex multiply-adds per panel"},
    }
    # The dominant kernel is the bulge chase: the largest share of the
    # reduction's launch list (serialised, one step of config 1) and the tail
    # every part ends with.  Its events time it alone on its SMs; the other
    # groups' events also count time queued behind the concurrent parts (the
    # bulk of the rank-2 update runs on low-priority streams), so their rates
    # below are lower bounds.
    top = "bulge_chase"
    g = groups[top]
    t = red[top] / 1e3
    scale = 1e9 if g["unit"] == "GB/s" else 1e12
    achieved = g["work"] / t / scale
    sms = peaks.get("sms") or 152
    occ_peak = g["peak"] * min(nk, sms) / sms
    # DRAM traffic of one bulge_kernel launch: the committed ncu capture's
    # bytes per matrix (the band is read once into shared memory) times this
    # launch's matrices, while band.cu is the file the counters were taken on
    rec = traffic_record("bulge_kernel", "dram_bytes_per_matrix")
    traffic = rec * nk if rec is not None and n == 882 else None
    roofline = {"bound": g["bound"], "kernel": g["kernel"], "achieved": achieved,
                "peak": g["peak"], "unit": g["unit"], "frac": achieved / g["peak"],
                "traffic": traffic, "peak_source": g["peak_source"],
                "algorithmic": g["algorithmic"] + f"; {nk} matrices, n={n}",
                "group_ms_per_step": red[top],
                "occupied_sms": min(nk, sms),
                "frac_of_occupied_sms": achieved / occ_peak,
                "occupied_note": "one CTA per matrix (the band lives in its shared memory): a "
                                 "launch can use at most as many SMs as it has matrices; "
                                 "frac_of_occupied_sms compares with the FP64 peak of those SMs",
                "group_rates": {k: groups[k]["work"] / (red[k] / 1e3) /
                                (1e9 if groups[k]["unit"] == "GB/s" else 1e12)
                                for k in groups if red.get(k)},
                "group_rates_note": "work / event time per group (GB/s for rank2_update and "
                                    "a22_v, TFLOP/s for the rest); the events of every group but "
                                    "the bulge chase include time queued behind the other parts"}
    eff = nk_all * 16.0 / 3.0 * n ** 3 / (ph["tridiag"] / 1e3) / 1e12
    reduction = {"method": "two-stage: dense -> band 8 (Householder panels, trailing updates as "
                           "8-digit exact-slice products on tcgen05), band -> tridiagonal "
                           "(bulge chase, FP64)",
                 "groups_ms_per_step": red, "timed_part_matrices": nk,
                 "tridiag_phase_ms": ph["tridiag"],
                 "tridiag_phase_includes": "the bisection (each part's runs right behind its "
                                           "bulge chase, beside the other parts')",
                 "one_stage_equivalent_tflops": eff,
                 "one_stage_equivalent_frac_of_fp64_peak": eff / fp64_peak,
                 "note": "(16/3) n^3 per k is the one-stage reduction's flop count; a value "
                         "above the FP64 peak means the reduction no longer runs on the FP64 "
                         "pipe, not that the FP64 pipe does more"}
    return roofline, reduction


def run_ours(args):
    import torch
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    rep = Replicas("nccl", torch.device("cuda", local))
    world, rank = rep.world, rep.rank

    from paper_1310_6380_gb300 import binding as bs

    cfg, config, prec = workload(args.config)
    if args.kpoints:   # a reduced case for profiling: the first K wavevectors only
        cfg["Q"] = cfg["Q"][:args.kpoints]
        config = dict(config, k_points=len(cfg["Q"]),
                      workload=config["workload"] + f" (first {len(cfg['Q'])} wavevectors only)")
    cell, M, nb = cfg["cell"], cfg["M"], cfg["nbands"]
    Q = np.ascontiguousarray(cfg["Q"])
    nk = len(Q)
    n = 2 * (2 * M + 1) ** 2
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    is_mesh = hasattr(cell, "centroid")

    C6 = None
    if getattr(cell, "stiffness", None) is not None:
        Cs = cell.stiffness
        C6 = np.ascontiguousarray(np.stack([Cs[:, 0, 0], Cs[:, 1, 1], Cs[:, 0, 1], Cs[:, 0, 2],
                                            Cs[:, 1, 2], Cs[:, 2, 2]], axis=1))

    def create(conv):
        if is_mesh:
            c = bs.bs_create_cell_mesh(cell.h1, cell.h2, conv(cell.centroid), conv(cell.area),
                                       conv(cell.phase.astype(np.uint16)), conv(cell.lam),
                                       conv(cell.mu), conv(cell.rho), M, prec)
        else:
            c = bs.bs_create_cell(cell.h1, cell.h2, conv(cell.phase.astype(np.uint16)),
                                  conv(cell.lam), conv(cell.mu), conv(cell.rho), M, prec)
        if C6 is not None:
            bs.bs_set_stiffness(c, conv(C6))
        return c

    h = create(dev)
    bs.bs_set_profiling(h, True)
    stream = torch.cuda.current_stream()
    Qd = dev(Q)
    w = torch.empty((nk, nb), dtype=torch.float64, device="cuda")
    st = torch.empty(nk, dtype=torch.int32, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def step():
        bs.bs_assemble(h, stream)
        bs.bs_solve_k(h, Qd, nb, w, st, stream)

    for _ in range(args.warmup):
        step()
    bs.bs_sync(h, stream)

    barrier = rep.barrier

    sampler = ClockSampler(device_bus_id(torch))
    step_ms, phases, reds = [], [], []
    barrier()
    launches0 = bs.bs_launch_count()
    sampler.start()
    t_wall = time.perf_counter()
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        phases.append(bs.bs_phase_times(h))
        reds.append(bs.bs_reduction_times(h))
    t_wall = time.perf_counter() - t_wall
    barrier()
    clocks = sampler.stop()
    launches = bs.bs_launch_count() - launches0 - 0
    bs.bs_sync(h, stream)
    assert not st.cpu().numpy().any(), "a wavevector did not converge"
    ms = statistics.mean(step_ms)
    ms = rep.max(ms)
    value = world * nk / (ms / 1e3)
    omega = w.cpu().numpy()

    # dominant kernel: the reduction to tridiagonal form (its largest kernel
    # group when the reduction is two-stage)
    ph = {k: statistics.mean(p[k] for p in phases) for k in phases[0]}
    peaks = device_peaks(torch, bs)
    red = {k: statistics.mean(r[k] for r in reds) for k in reds[0]}
    if prec == 0 and red["matrices"] > 0:
        roofline, reduction = band_roofline(red, n, nk, ph, peaks)
    elif prec == 0:
        reduction = None
        trid_flops = nk * 16.0 / 3.0 * n ** 3
        achieved = trid_flops / (ph["tridiag"] / 1e3) / 1e12
        fp64_peak = peaks["fp64_nominal_tflops"]
        roofline = {"bound": "alu", "kernel": "tridiag_step_kernel<double> (all launches of one step)",
                    "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
                    "frac": achieved / fp64_peak,
                    "traffic": traffic_record("tridiag_step_kernel") if args.config == "c1" else None,
                    "peak_source": f"nominal FP64: {peaks['sms']} SMs (queried) x 2 FMA/clk x 2 "
                                   f"flop x {peaks['sm_max_mhz']:.0f} MHz",
                    "peak_measured_fma_probe": peaks["fp64_probe_tflops"],
                    "frac_of_probe": achieved / peaks["fp64_probe_tflops"],
                    "algorithmic": f"(16/3) n^3 real flops per k x {nk} k, n={n}"}
    else:
        reduction = None
        hbm_peak, _, note = measured_peaks()
        tri_bytes = nk * sum(m * (m + 1) // 2 for m in range(1, n)) * 16.0
        achieved = tri_bytes / (ph["tridiag"] / 1e3) / 1e9
        roofline = {"bound": "hbm", "kernel": "tridiag_step_kernel<float> (all launches of one step)",
                    "achieved": achieved, "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
                    "traffic": None, "peak_source": "copy bandwidth, " + note,
                    "algorithmic": "read + write (8 B each) of every trailing lower triangle, "
                                   f"{nk} matrices, n={n}"}

    # end to end through the public API with host (pinned) buffers
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    hQ = pin(Q)
    hw = torch.empty((nk, nb), dtype=torch.float64).pin_memory()
    hs = torch.empty(nk, dtype=torch.int32).pin_memory()
    host_bufs = {}
    for name, arr in (("phase", cell.phase.astype(np.uint16)), ("lam", cell.lam), ("mu", cell.mu),
                      ("rho", cell.rho)) + ((("centroid", cell.centroid), ("area", cell.area))
                                            if is_mesh else ()):
        host_bufs[name] = pin(arr)

    if C6 is not None:
        host_bufs["stiffness"] = pin(C6)

    def e2e_create():
        b = host_bufs
        if is_mesh:
            c = bs.bs_create_cell_mesh(cell.h1, cell.h2, b["centroid"], b["area"], b["phase"],
                                       b["lam"], b["mu"], b["rho"], M, prec)
        else:
            c = bs.bs_create_cell(cell.h1, cell.h2, b["phase"], b["lam"], b["mu"], b["rho"], M,
                                  prec)
        if C6 is not None:
            bs.bs_set_stiffness(c, b["stiffness"])
        return c

    def e2e_step():
        c = e2e_create()
        try:
            bs.bs_assemble(c, stream)
            bs.bs_solve_k(c, hQ, nb, hw, hs, stream)
        finally:
            bs.bs_destroy_cell(c)

    for _ in range(max(1, args.warmup)):
        e2e_step()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / args.steps
    e2e_s = rep.max(e2e_s)
    h2d = sum(t.numel() * t.element_size() for t in host_bufs.values()) + hQ.numel() * 8
    d2h = hw.numel() * 8 + hs.numel() * 4
    e2e = {"value": world * nk / e2e_s, "unit": "k-solves/s", "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": d2h,
           "api": "bs_create_cell + bs_assemble + bs_solve_k + bs_destroy_cell, pinned host buffers"}

    # on config 1, also measure config 2 (the same cell on the mixed path), the
    # tensor-core utilisation of the exact-slice contraction, the assembly's
    # tensor-core launch, and (reduced cell counts) configs 3 and 4
    mixed = tensor = assembly = sub3 = sub4 = None
    if args.config == "c1":
        mixed = measure_mixed(bs, torch, args, cell, M, nb, nk, Qd, stream, flush, barrier, dev,
                              ms, omega, world)
        tensor = measure_tensor(bs, torch, stream, nk, n)
        assembly = measure_assembly(bs, torch, stream, cell, M, ph)
        if not args.no_sub:
            sub_steps, sub_warm = min(args.steps, 3), 3
            sub3 = measure_c3(bs, torch, rep, args, 512, sub_steps, sub_warm, graph=True,
                              oracle_cells=3, cpu_baseline=not args.no_cpu_baseline)
            sub4 = measure_c4(bs, torch, rep, args, 256, sub_steps, sub_warm, oracle_cells=2,
                              fp64_cells=64, cpu_baseline=not args.no_cpu_baseline)

    out = {
        "metric": METRIC, "value": value, "unit": "k-solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if prec == 0 else "f32 reduction, bf16 exact-slice tensor products, f64 refinement",
        "data": "synthetic", "config": config, "e2e": e2e, "gpu_launches": launches,
        "gpu_launches_per_step": launches // max(1, args.steps), "roofline": roofline,
        "phases_ms": {k: round(v, 3) for k, v in ph.items() if v > 0},
        "wall_s_timed_region": t_wall, "clocks": clocks,
    }
    if reduction is not None:
        out["reduction"] = reduction
    if args.config == "mesh":
        out["paper_context"] = ("the paper's run of this workload (1000-element steel/epoxy mesh, "
                                "M=5, 70 k, 18 branches) took 90 s on a Quadro K2000 desktop GPU, "
                                "about 0.78 k-solves/s; other hardware and mesh, context only")
    out["device"] = peaks
    omega_mixed = None
    if mixed is not None:
        omega_mixed = mixed.pop("_omega")
        out["mixed_path"] = mixed
        out["tensor_core"] = tensor
        out["assembly"] = assembly
    for key, sub in (("c3", sub3), ("c4", sub4)):
        if sub is not None:
            for drop in ("metric", "n_gpus", "higher_is_better", "scaling", "vs_baseline", "data",
                         "clocks"):
                sub.pop(drop, None)
            out[key] = sub
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, idx, ws, desc, _ = cpu_oracle_sample(cfg, args.cpu_sample_k)
        out["cpu_baseline"] = {"value": v, "unit": "k-solves/s",
                               "cores": len(os.sched_getaffinity(0)), "kind": "oracle",
                               "sample": desc}
        out["max_rel_err_vs_oracle"] = float(rel_err(omega[idx], ws, cell).max())
        if omega_mixed is not None:
            out["mixed_path"]["max_rel_err_vs_oracle"] = float(
                rel_err(omega_mixed[idx], ws, cell).max())
        out["oracle_sampled_k"] = idx.tolist()
    bs.bs_destroy_cell(h)
    if rank == 0:
        print(json.dumps(out))
    rep.close()


def measure_c4(bs, torch, rep, args, ncell, steps, warmup, oracle_cells=6, fp64_cells=128,
               cpu_baseline=True):
    """Config 4: the learned warm start.  Held-out cells (seeds 2e6 + i), 30 k
    each, 10 branches, batch LOBPCG from (a) the cold start and (b) the trained
    network's 12-vector starting subspaces; one step = network inference for
    every (cell, k) + the batch solve (assembly, LOBPCG, FP64 Rayleigh-Ritz,
    certificate, count check, dense rescues).  The plain FP64 dense GPU path
    is timed on a sample of the same cells for comparison.  Returns the JSON
    dict of the measurement."""
    world, rank = rep.world, rep.rank
    from paper_1310_6380_gb300 import cells
    from paper_1310_6380_gb300 import warmstart as ws

    if not os.path.exists(args.weights):
        raise SystemExit(f"no trained network at {args.weights}: run "
                         "python -m paper_1310_6380_gb300.train_warmstart --out <file>")
    saved = np.load(args.weights)
    meta = json.loads(str(saved["meta"]))
    nk, nb, Mp, nvec = 30, 10, meta["Mp"], meta["nvec"]
    cfgs = [cells.config4_eval_cell(i) for i in range(ncell)]
    cl = [c["cell"] for c in cfgs]
    Ms = [c["M"] for c in cfgs]
    Qh = np.ascontiguousarray(np.stack([c["Q"] for c in cfgs]))
    cargs = [(c.h1, c.h2, np.ascontiguousarray(c.phase, np.uint16), c.lam, c.mu, c.rho, M,
              bs.BS_PREC_MIXED) for c, M in zip(cl, Ms)]
    net = ws.WarmStartNet(nvec, Mp, max_cells=256, max_samples=256 * nk)
    net.set_params(saved["params"])
    pack = ws.CellPack(cl)
    b = bs.bs_batch_create(cargs, nk, nb)
    bs.bs_batch_set_solver(b, bs.BS_SOLVER_LOBPCG)
    Qd = torch.tensor(Qh, device="cuda")
    w = torch.empty((ncell, nk, nb), dtype=torch.float64, device="cuda")
    st = torch.empty((ncell, nk), dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    barrier = rep.barrier

    def step(warm):
        if warm:
            U = net.predict(pack, Qh)
            bs.bs_batch_set_start(b, U, Mp)
        else:
            bs.bs_batch_set_start(b, None)
        bs.bs_batch_solve(b, Qd, w, st, stream)

    def timed(warm):
        for _ in range(warmup):
            step(warm)
        barrier()
        times = []
        for _ in range(steps):
            flush.zero_()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step(warm)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        barrier()
        it, fb = bs.bs_batch_stats(b, ncell * nk)
        return statistics.mean(times), it, fb, w.cpu().numpy(), st.cpu().numpy()

    ms_cold, it_cold, fb_cold, om_cold, st_cold = timed(False)
    launches0 = bs.bs_launch_count()
    sampler = ClockSampler(device_bus_id(torch))
    sampler.start()
    ms_warm, it_warm, fb_warm, om_warm, st_warm = timed(True)
    clocks = sampler.stop()
    launches = (bs.bs_launch_count() - launches0) // max(1, steps + warmup)
    bs.bs_batch_set_profiling(b, True)
    step(True)
    torch.cuda.synchronize()
    ph = bs.bs_batch_phase_times(b)
    bs.bs_batch_set_profiling(b, False)
    ms = ms_warm
    ms = rep.max(ms)
    value = world * ncell * nk / (ms / 1e3)

    # the plain FP64 dense GPU path (FP64 C(k), reduction to tridiagonal form,
    # Sturm multisection), batched over the cells like the other solvers, on a
    # sample of the cells
    samp = list(range(0, ncell, max(1, ncell // fp64_cells)))[:fp64_cells]
    bf = bs.bs_batch_create([cargs[i] for i in samp], nk, nb)
    bs.bs_batch_set_solver(bf, bs.BS_SOLVER_FP64)
    Qf = torch.tensor(Qh[samp], device="cuda")
    wf = torch.empty((len(samp), nk, nb), dtype=torch.float64, device="cuda")
    bs.bs_batch_solve(bf, Qf, wf, None, stream)
    torch.cuda.synchronize()
    flush.zero_()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    bs.bs_batch_solve(bf, Qf, wf, None, stream)
    e1.record(stream)
    e1.synchronize()
    fp64_ms = e0.elapsed_time(e1)
    bs.bs_batch_destroy(bf)
    fp64_rate = len(samp) * nk / (fp64_ms / 1e3)

    # end to end through the public API, host buffers: network inference on
    # host inputs, batch creation from host arrays, solve with host Q/outputs
    hw = torch.empty((ncell, nk, nb), dtype=torch.float64).pin_memory()
    hs = torch.empty((ncell, nk), dtype=torch.int32).pin_memory()
    hQ = torch.from_numpy(Qh).pin_memory()
    barrier()
    t0 = time.perf_counter()
    for _ in range(steps):
        b2 = bs.bs_batch_create(cargs, nk, nb)
        bs.bs_batch_set_solver(b2, bs.BS_SOLVER_LOBPCG)
        bs.bs_batch_set_start(b2, net.predict(pack, Qh), Mp)
        bs.bs_batch_solve(b2, hQ, hw, hs, stream)
        bs.bs_batch_destroy(b2)
    torch.cuda.synchronize()
    e2e_s = rep.max((time.perf_counter() - t0) / steps)
    h2d = (sum(a[2].nbytes + 3 * a[3].nbytes for a in cargs) + Qh.nbytes + pack.phase.nbytes
           + pack.table.nbytes + ncell * nk * nvec * 2 * (2 * Mp + 1) ** 2 * 8)
    e2e = {"value": world * ncell * nk / e2e_s, "unit": "k-solves/s", "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": hw.numel() * 8 + hs.numel() * 4
           + ncell * nk * nvec * 2 * (2 * Mp + 1) ** 2 * 8,
           "api": "bs_cnn_forward (host inputs, starting vectors to host) + bs_batch_create + "
                  "bs_batch_set_solver/set_start + bs_batch_solve (host Q, outputs) + "
                  "bs_batch_destroy"}
    ns = np.array([2 * (2 * m + 1) ** 2 for m in Ms], float)
    # dominant phase: the LOBPCG iterations; algorithmic FP32 flops of the
    # C W products at the full block width (an upper bound on the active width)
    b_lob = 16
    cw_flops = float(np.sum(it_warm.reshape(ncell, nk) * (8.0 * ns[:, None] ** 2 * b_lob)))
    achieved = cw_flops / (ph["reduction"] / 1e3) / 1e12
    fp32_peak = device_peaks(torch)["fp32_nominal_tflops"]
    roofline = {"bound": "alu", "kernel": "LOBPCG iterations (lob_cw_kernel + lob_eig_kernel + "
                                          "lob_update_kernel, one step)",
                "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": achieved / fp32_peak, "traffic": None,
                "peak_source": "nominal FP32 CUDA-core rate: SMs x 128 FMA/clk x 2 x max SM clock "
                               "(queried)",
                "algorithmic": "8 n^2 b flops (C W, b = 16) per LOBPCG iteration per (cell, k)"}
    out = {
        "metric": METRIC, "value": value, "unit": "k-solves/s", "n_gpus": world,
        "steps": steps, "warmup": warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 network and LOBPCG, bf16 exact-slice tensor products, f64 Rayleigh-Ritz",
        "data": "synthetic",
        "config": {"workload": f"c4: learned warm start, {ncell} held-out cells (seeds 2e6+i, "
                               "64x64, square/hex, ellipse/Voronoi, 2-16 phases, M = 5..8), 30 k "
                               "each, lowest 10 branches, batch LOBPCG from the network's "
                               f"{nvec}-vector subspaces (|alpha|,|beta| <= {Mp})",
                   "cells": ncell, "k_points": ncell * nk,
                   "network": {k: meta[k] for k in ("cells", "kper", "epochs", "M_train", "Mp",
                                                   "nvec", "seeds")},
                   "l2": "flushed between timed steps (256 MiB write, untimed)"},
        "cold_start": {"value": world * ncell * nk / (ms_cold / 1e3), "ms_per_step": ms_cold,
                       "iterations_mean": float(it_cold.mean()),
                       "dense_mixed_rescues": int((fb_cold == 2).sum()),
                       "fp64_fallbacks": int((fb_cold == 1).sum())},
        "warm_start": {"iterations_mean": float(it_warm.mean()),
                       "dense_mixed_rescues": int((fb_warm == 2).sum()),
                       "fp64_fallbacks": int((fb_warm == 1).sum()),
                       "iteration_ratio_vs_cold": float(it_warm.mean() / it_cold.mean()),
                       "speedup_vs_cold": ms_cold / ms_warm},
        "fp64_dense_gpu": {"value": fp64_rate, "unit": "k-solves/s",
                           "sample": f"{len(samp)} of the cells x {nk} k, one ragged batch "
                                     "on BS_SOLVER_FP64 (assembly, FP64 C(k), FP64 reduction "
                                     "to tridiagonal form, two-stage for n >= 400, Sturm "
                                     "multisection)",
                           "speedup_of_value": value / fp64_rate},
        "speedup_vs_fp64_batched": value / fp64_rate,
        "speedup_target": 10.0,
        "status_nonzero": int(np.count_nonzero(st_warm)),
        "phases_ms": {k: round(v, 1) for k, v in ph.items()},
        "gpu_launches_per_step": launches, "gpu_launches": launches * steps,
        "e2e": e2e, "roofline": roofline, "clocks": clocks,
    }
    if rank == 0 and world == 1 and cpu_baseline and oracle_cells > 0:
        from oracle import mixed_variational as mv
        osamp = list(range(0, ncell, max(1, ncell // oracle_cells)))[:oracle_cells]
        t0 = time.perf_counter()
        errs = []
        for i in osamp:
            oc = mv.OracleCell(cl[i], Ms[i])
            ref = np.array([oc.omega(q, nb) for q in Qh[i]])
            errs.append(max(rel_err(om_warm[i], ref, cl[i]).max(),
                            rel_err(om_cold[i], ref, cl[i]).max()))
        secs = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": len(osamp) * nk / secs, "unit": "k-solves/s",
                               "cores": len(os.sched_getaffinity(0)), "kind": "oracle",
                               "sample": f"{len(osamp)} of the {ncell} cells, all 30 k each "
                                         f"({secs:.1f} s); value = their k-solves / time"}
        out["max_rel_err_vs_oracle"] = float(max(errs))
        out["oracle_sampled_cells"] = osamp
    bs.bs_batch_destroy(b)
    net.close()
    return out


def run_c4(args):
    """Config 4 on its own line (bench.py --config c4)."""
    import torch
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    rep = Replicas("nccl", torch.device("cuda", local))
    from paper_1310_6380_gb300 import binding as bs
    out = measure_c4(bs, torch, rep, args, args.cells or 1024, args.steps, args.warmup,
                     cpu_baseline=not args.no_cpu_baseline)
    if rep.rank == 0:
        print(json.dumps(out))
    rep.close()


# ---------------------------------------------------------------- mode shapes
MODES_METRIC = "Bloch mode shapes/sec (stress coefficients + u, sigma on the cell's pixel grid)"


def modes_workload():
    from paper_1310_6380_gb300 import cells
    cfg = cells.config1()
    nvec, G = 12, cfg["cell"].P
    N = (2 * cfg["M"] + 1) ** 2
    config = {
        "workload": f"modes: the 256x256 periodic Voronoi cell (1132 phases, seed 1310), "
                    f"M={cfg['M']} ({N} plane waves), {len(cfg['Q'])} k on G-X-M-G, the lowest "
                    f"{nvec} modes of each from bs_solve_k_lobpcg; one step = stress "
                    f"coefficients S = -Phi^-1 H^* U (FP64) and the 5 fields u1, u2, S11, S22, "
                    f"S12 of every mode on the {G}x{G} pixel-centre grid (complex64)",
        "cells": 1, "k_points": len(cfg["Q"]), "modes_per_k": nvec, "grid": G,
        "plane_waves": N, "l2": "outputs (2.8 GB) larger than L2; L2 flushed between steps",
    }
    return cfg, config, nvec, G


def modes_oracle_sample(cfg, nvec, G, idx):
    """The oracle on the sampled wavevectors idx: its own lowest nvec modes U
    (eigh of the pencil, untimed), then the timed stress coefficients and the
    five fields of every mode on the G x G grid.  Returns (U, S, F, seconds)."""
    import scipy.linalg as sla
    from oracle import mixed_variational as mv
    from oracle import mode_shapes as ms
    oc = mv.OracleCell(cfg["cell"], cfg["M"])
    Us = []
    for i in idx:
        A, Om = oc.pencil(cfg["Q"][i])
        Us.append(np.ascontiguousarray(sla.eigh(A, Om, subset_by_index=[0, nvec - 1])[1].T))
    t0 = time.perf_counter()
    oc = mv.OracleCell(cfg["cell"], cfg["M"])
    S, F = [], []
    N = oc.N
    for j, i in enumerate(idx):
        q = cfg["Q"][i]
        Si = ms.stress_coefficients(oc, q, Us[j])
        coef = np.concatenate([Us[j].reshape(2 * nvec, N), Si.reshape(3 * nvec, N)])
        S.append(Si)
        F.append(ms.field_on_grid(cfg["cell"], cfg["M"], q, coef, G))
    return Us, S, F, time.perf_counter() - t0


def run_modes(args):
    import torch
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    rep = Replicas("nccl", torch.device("cuda", local))
    world, rank = rep.world, rep.rank
    from paper_1310_6380_gb300 import binding as bs

    cfg, config, nvec, G = modes_workload()
    if args.kpoints:
        cfg["Q"] = cfg["Q"][:args.kpoints]
        config["k_points"] = len(cfg["Q"])
        config["workload"] += f" (first {len(cfg['Q'])} wavevectors only)"
    cell, M = cfg["cell"], cfg["M"]
    Q = np.ascontiguousarray(cfg["Q"])
    nk, N = len(Q), (2 * M + 1) ** 2
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    stream = torch.cuda.current_stream()
    h = bs.bs_create_cell(cell.h1, cell.h2, dev(cell.phase.astype(np.uint16)), dev(cell.lam),
                          dev(cell.mu), dev(cell.rho), M, bs.BS_PREC_MIXED)
    bs.bs_assemble(h, stream)
    Qd = dev(Q)
    # the modes (input of the step, computed once): LOBPCG vectors
    w = torch.empty((nk, nvec), dtype=torch.float64, device="cuda")
    vec = torch.empty((nk, nvec, 2 * N), dtype=torch.complex64, device="cuda")
    bs.bs_solve_k_lobpcg(h, Qd, nvec, w, vec_out=vec, stream=stream)
    Ud = vec.to(torch.complex128).contiguous()
    Sd = torch.empty((nk, nvec, 3 * N), dtype=torch.complex128, device="cuda")
    Fu = torch.empty((nk, 2 * nvec, G, G), dtype=torch.complex64, device="cuda")
    Fs = torch.empty((nk, 3 * nvec, G, G), dtype=torch.complex64, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    Uv, Sv = Ud.view(nk, 2 * nvec, N), Sd.view(nk, 3 * nvec, N)

    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]

    def step():
        ev[0].record(stream)
        bs.bs_stress_coefficients(h, Qd, Ud, Sd, stream)
        ev[1].record(stream)
        bs.bs_mode_field(h, Qd, Uv, G, Fu, stream)
        ev[2].record(stream)
        bs.bs_mode_field(h, Qd, Sv, G, Fs, stream)
        ev[3].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    sampler = ClockSampler(device_bus_id(torch))
    parts = {"stress": [], "field_u": [], "field_sigma": []}
    step_ms = []
    rep.barrier()
    launches0 = bs.bs_launch_count()
    sampler.start()
    for _ in range(args.steps):
        flush.zero_()
        step()
        ev[3].synchronize()
        step_ms.append(ev[0].elapsed_time(ev[3]))
        parts["stress"].append(ev[0].elapsed_time(ev[1]))
        parts["field_u"].append(ev[1].elapsed_time(ev[2]))
        parts["field_sigma"].append(ev[2].elapsed_time(ev[3]))
    rep.barrier()
    clocks = sampler.stop()
    launches = bs.bs_launch_count() - launches0
    ms = rep.max(statistics.mean(step_ms))
    pm = {k: statistics.mean(v) for k, v in parts.items()}
    units = nk * nvec
    value = rep.value(units, ms)

    # rooflines of the two kinds of work; the JSON roofline is the dominant one
    W = 2 * M + 1
    stress_flops = units * 3 * 8.0 * N * N          # three Gram solves, two triangular products
    fld = nk * 5 * nvec
    field_flops = fld * (8.0 * W * G * G + 8.0 * W * W * G)
    field_bytes = fld * G * G * 8.0 + fld * N * 16.0
    dpk = device_peaks(torch)
    fp32_peak = dpk["fp32_nominal_tflops"]
    hbm_peak, _, note = measured_peaks()
    t_field = (pm["field_u"] + pm["field_sigma"]) / 1e3
    rl_stress = {"bound": "alu", "kernel": "bs_stress_coefficients (stress_rhs_kernel, "
                                           "zgemm_kernel x4, stress_combine_kernel)",
                 "achieved": stress_flops / (pm["stress"] / 1e3) / 1e12,
                 "peak": dpk["fp64_nominal_tflops"], "unit": "TFLOP/s", "traffic": None,
                 "peak_source": "nominal FP64: SMs (queried) x 2 FMA/clk x 2 flop x max SM clock",
                 "algorithmic": "3 Gram solves per mode, each two triangular products: 24 N^2 "
                                "real flops per mode"}
    rl_stress["frac"] = rl_stress["achieved"] / rl_stress["peak"]
    rl_field = {"bound": "alu", "kernel": "field_kernel<24> (+ field_table_kernel)",
                "achieved": field_flops / t_field / 1e12, "peak": fp32_peak, "unit": "TFLOP/s",
                "traffic": None,
                "peak_source": "nominal FP32 CUDA-core rate: SMs (queried) x 128 FMA/clk x 2 x max "
                               "SM clock",
                "algorithmic": "8 W G^2 + 8 W^2 G real flops per field (W = 2M+1 = 21, G = 256); "
                               f"stores {field_bytes / 1e9:.2f} GB per step",
                "hbm_gbs": field_bytes / t_field / 1e9, "hbm_frac": field_bytes / t_field / 1e9
                / hbm_peak, "hbm_peak_source": "copy bandwidth, " + note}
    rl_field["frac"] = rl_field["achieved"] / rl_field["peak"]
    roofline = rl_stress if pm["stress"] >= pm["field_u"] + pm["field_sigma"] else rl_field

    # end to end: host modes in, host stress and fields out (pinned)
    hQ = torch.from_numpy(Q).pin_memory()
    hU = Ud.cpu().pin_memory()
    hS = torch.empty_like(Sd, device="cpu").pin_memory()
    hFu = torch.empty(tuple(Fu.shape), dtype=torch.complex64).pin_memory()
    hFs = torch.empty(tuple(Fs.shape), dtype=torch.complex64).pin_memory()

    def e2e_step():
        bs.bs_stress_coefficients(h, hQ, hU, hS, stream)
        bs.bs_mode_field(h, hQ, hU.view(nk, 2 * nvec, N), G, hFu, stream)
        bs.bs_mode_field(h, hQ, hS.view(nk, 3 * nvec, N), G, hFs, stream)

    e2e_step()
    rep.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    torch.cuda.synchronize()
    e2e_s = rep.max((time.perf_counter() - t0) / args.steps)
    e2e = {"value": world * units / e2e_s, "unit": "modes/s",
           "h2d_bytes_per_step": hQ.numel() * 8 + hU.numel() * 16 + hS.numel() * 16,
           "d2h_bytes_per_step": hS.numel() * 16 + (hFu.numel() + hFs.numel()) * 8,
           "api": "bs_stress_coefficients (host U in, host S out) + bs_mode_field x2 (host "
                  "coefficients in, host fields out)"}

    out = {
        "metric": MODES_METRIC, "value": value, "unit": "modes/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64 stress solves, f32 field contractions (complex64 fields)",
        "data": "synthetic", "config": config, "e2e": e2e, "gpu_launches": launches,
        "gpu_launches_per_step": launches // max(1, args.steps), "roofline": roofline,
        "rooflines": {"stress": rl_stress, "fields": rl_field},
        "parts_ms": {k: round(v, 3) for k, v in pm.items()}, "clocks": clocks,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the oracle on two wavevectors with its own modes; the library run on
        # the same modes for the parity figures
        idx = [nk // 9, nk // 3]
        Us, S_ref, F_ref, secs = modes_oracle_sample(cfg, nvec, G, idx)
        U2 = np.ascontiguousarray(np.stack(Us))
        S2 = np.empty((len(idx), nvec, 3 * N), np.complex128)
        bs.bs_stress_coefficients(h, Q[idx], U2, S2)
        coef2 = np.ascontiguousarray(np.concatenate(
            [U2.reshape(len(idx), 2 * nvec, N), S2.reshape(len(idx), 3 * nvec, N)], axis=1))
        F2 = np.empty((len(idx), 5 * nvec, G, G), np.complex64)
        bs.bs_mode_field(h, Q[idx], coef2, G, F2)
        err_s = max(float(np.abs(S2[j] - S_ref[j]).max() / np.abs(S_ref[j]).max())
                    for j in range(len(idx)))
        err_f = 0.0
        for j in range(len(idx)):
            coef = np.concatenate([Us[j].reshape(2 * nvec, N), S_ref[j].reshape(3 * nvec, N)])
            bound = (2 * W + 4) * 2.0 ** -24 * np.abs(coef).sum(axis=1)
            err_f = max(err_f, float((np.abs(F2[j] - F_ref[j]).max(axis=(1, 2)) / bound).max()))
        out["cpu_baseline"] = {"value": len(idx) * nvec / secs, "unit": "modes/s",
                               "cores": len(os.sched_getaffinity(0)), "kind": "oracle",
                               "sample": f"k {idx} of {nk}, the oracle's own lowest {nvec} modes "
                                         f"each: oracle cell set-up, stress and the 5 fields on "
                                         f"the grid ({secs:.1f} s)"}
        out["max_rel_err_stress_vs_oracle"] = err_s
        out["max_field_err_over_bound"] = err_f
    bs.bs_destroy_cell(h)
    if rank == 0:
        print(json.dumps(out))
    rep.close()


def run_reference_modes(args):
    if int(os.environ.get("RANK", "0")) != 0:
        return
    cfg, config, nvec, G = modes_workload()
    nk = len(cfg["Q"])
    times = []
    for i in range(args.warmup + args.steps):
        secs = modes_oracle_sample(cfg, nvec, G, [(i * 7) % nk])[3]
        if i >= args.warmup:
            times.append(secs)
    value = nvec / statistics.mean(times)
    desc = (f"each step: oracle cell set-up, stress and the 5 fields of the oracle's own lowest "
            f"{nvec} modes at one k")
    print(json.dumps({
        "impl": "reference", "metric": MODES_METRIC, "value": value, "unit": "modes/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * statistics.mean(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config,
        "cpu_baseline": {"value": value, "unit": "modes/s", "cores": len(os.sched_getaffinity(0)),
                         "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": "modes/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0}}))


# ---------------------------------------------------------------- 3-D cells
def workload3d():
    from paper_1310_6380_gb300 import cells
    cell = cells.sphere_cell3(32, 0.3)
    M, nb, nk = 3, 12, 30
    Q = cells.ibz_path_cubic(nk)
    config = {
        "workload": "3d: simple cubic cell a=1, 32^3 voxels, one spherical inclusion r=0.3a "
                    "(matrix lam=4, mu=1.5, rho=1.2; inclusion 110, 80, 7.8), M=3 (343 plane "
                    "waves, n=1029), 30 k on G-X-M-R-G, lowest 12 branches, FP64 path",
        "cells": 1, "k_points": nk, "plane_waves": 343, "n": 1029, "nbands": nb,
        "precision": "fp64", "l2": "flushed between timed steps (256 MiB write, untimed)",
    }
    return dict(cell=cell, M=M, Q=Q, nbands=nb), config


def oracle3d_sample(cfg, idx):
    from oracle import mixed_variational_3d as mv3
    t0 = time.perf_counter()
    oc = mv3.OracleCell3(cfg["cell"], cfg["M"])
    ws = [oc.omega(cfg["Q"][i], cfg["nbands"]) for i in idx]
    return np.array(ws), time.perf_counter() - t0


def run_3d(args):
    import torch
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    rep = Replicas("nccl", torch.device("cuda", local))
    world, rank = rep.world, rep.rank
    from paper_1310_6380_gb300 import binding as bs

    cfg, config = workload3d()
    cell, M, nb = cfg["cell"], cfg["M"], cfg["nbands"]
    Q = np.ascontiguousarray(cfg["Q"])
    nk = len(Q)
    n = 3 * (2 * M + 1) ** 3
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    stream = torch.cuda.current_stream()
    h = bs.bs_create_cell3(cell.h1, cell.h2, cell.h3, dev(cell.phase.astype(np.uint16)),
                           dev(cell.lam), dev(cell.mu), dev(cell.rho), M)
    Qd = dev(Q)
    w = torch.empty((nk, nb), dtype=torch.float64, device="cuda")
    st = torch.empty(nk, dtype=torch.int32, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]

    def step():
        ev[0].record(stream)
        bs.bs_assemble3(h, stream)
        ev[1].record(stream)
        bs.bs_solve_k3(h, Qd, nb, w, st, stream)
        ev[2].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    sampler = ClockSampler(device_bus_id(torch))
    step_ms, asm_ms, sol_ms = [], [], []
    rep.barrier()
    launches0 = bs.bs_launch_count()
    sampler.start()
    for _ in range(args.steps):
        flush.zero_()
        step()
        ev[2].synchronize()
        step_ms.append(ev[0].elapsed_time(ev[2]))
        asm_ms.append(ev[0].elapsed_time(ev[1]))
        sol_ms.append(ev[1].elapsed_time(ev[2]))
    rep.barrier()
    clocks = sampler.stop()
    launches = bs.bs_launch_count() - launches0
    assert not st.cpu().numpy().any(), "a wavevector did not converge"
    ms = rep.max(statistics.mean(step_ms))
    value = rep.value(nk, ms)
    omega = w.cpu().numpy()
    t_sol = statistics.mean(sol_ms)
    flops = nk * 16.0 / 3.0 * n ** 3
    achieved = flops / (t_sol / 1e3) / 1e12
    two_stage = n >= 400   # BS_REDUCE_AUTO: the two-stage reduction from n = 400 on
    kern = ("bs_solve_k3 of one step: two-stage reduction (tcgen05 dense -> band, FP64 bulge "
            "chase), per-k builder, bisection" if two_stage else
            "tridiag_step_kernel<double> (with the per-k builder and bisection: bs_solve_k3 of "
            "one step)")
    roofline = {"bound": "alu", "kernel": kern,
                "achieved": achieved, "peak": device_peaks(torch)["fp64_nominal_tflops"],
                "unit": "TFLOP/s", "traffic": None,
                "peak_source": "nominal FP64: SMs (queried) x 2 FMA/clk x 2 flop x max SM clock",
                "algorithmic": f"(16/3) n^3 real flops per k x {nk} k, n={n}" +
                               ("; the one-stage reduction's flop count, so above 1.0 of the "
                                "FP64 peak means the work left the FP64 pipe" if two_stage else "")}
    roofline["frac"] = roofline["achieved"] / roofline["peak"]
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    hp, hl, hm, hr, hQ = (pin(cell.phase.astype(np.uint16)), pin(cell.lam), pin(cell.mu),
                          pin(cell.rho), pin(Q))
    hw = torch.empty((nk, nb), dtype=torch.float64).pin_memory()

    def e2e_step():
        c = bs.bs_create_cell3(cell.h1, cell.h2, cell.h3, hp, hl, hm, hr, M)
        try:
            bs.bs_assemble3(c, stream)
            bs.bs_solve_k3(c, hQ, nb, hw, None, stream)
        finally:
            bs.bs_destroy_cell3(c)

    e2e_step()
    rep.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    torch.cuda.synchronize()
    e2e_s = rep.max((time.perf_counter() - t0) / args.steps)
    e2e = {"value": world * nk / e2e_s, "unit": "k-solves/s",
           "h2d_bytes_per_step": hp.numel() * 2 + 3 * hl.numel() * 8 + hQ.numel() * 8,
           "d2h_bytes_per_step": hw.numel() * 8,
           "api": "bs_create_cell3 + bs_assemble3 + bs_solve_k3 + bs_destroy_cell3, pinned host "
                  "buffers"}
    out = {
        "metric": METRIC, "value": value, "unit": "k-solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config, "e2e": e2e, "gpu_launches": launches,
        "gpu_launches_per_step": launches // max(1, args.steps), "roofline": roofline,
        "phases_ms": {"assemble3": round(statistics.mean(asm_ms), 3),
                      "solve_k3": round(t_sol, 3)},
        "clocks": clocks,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        idx = [4, 17]
        ws, secs = oracle3d_sample(cfg, idx)
        A = np.array([cell.h1, cell.h2, cell.h3])
        qm = 2 * np.pi * np.linalg.inv(A)
        fl = np.sqrt(np.min(cell.mu / cell.rho)) * min(np.linalg.norm(qm[:, i]) for i in range(3)) / 2
        err = np.abs(omega[idx] ** 2 - ws ** 2) / (2 * np.maximum(ws ** 2, fl ** 2))
        out["cpu_baseline"] = {"value": len(idx) / secs, "unit": "k-solves/s",
                               "cores": len(os.sched_getaffinity(0)), "kind": "oracle",
                               "sample": f"oracle cell set-up + wavevectors {idx} of {nk} "
                                         f"({secs:.1f} s); value = their k-solves / time"}
        out["max_rel_err_vs_oracle"] = float(err.max())
    bs.bs_destroy_cell3(h)
    if rank == 0:
        print(json.dumps(out))
    rep.close()


def run_reference_3d(args):
    if int(os.environ.get("RANK", "0")) != 0:
        return
    cfg, config = workload3d()
    nk = len(cfg["Q"])
    times = []
    for i in range(args.warmup + args.steps):
        _, secs = oracle3d_sample(cfg, [(i * 7) % nk])
        if i >= args.warmup:
            times.append(secs)
    value = 1.0 / statistics.mean(times)
    desc = "each step: oracle cell set-up and one wavevector"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "k-solves/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * statistics.mean(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config,
        "cpu_baseline": {"value": value, "unit": "k-solves/s", "cores": len(os.sched_getaffinity(0)),
                         "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": "k-solves/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0}}))


def main():
    args = parse_args()
    if args.impl == "reference":
        if args.config == "modes":
            run_reference_modes(args)
        elif args.config == "3d":
            run_reference_3d(args)
        else:
            run_reference(args)
    elif args.config == "3d":
        run_3d(args)
    elif args.config == "modes":
        run_modes(args)
    elif args.config == "c3":
        args.cells = args.cells or 4096
        run_batch(args)
    elif args.config == "c4":
        run_c4(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
