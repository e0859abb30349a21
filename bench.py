#!/usr/bin/env python
"""Throughput of the Kubo-formula anomalous Hall sum on GB300: k-points/s.

Workload (synthetic stand-in for the paper's Wannier models, seeded): W = 64 orbitals,
R in {-5..5}^3 (N_R = 1331), hoppings N(0,1) exp(-|R|/1.5) with random phases, 128^3
Gamma-centred mesh, 64 Fermi levels in [-1, 1], eta = 1e-3.

One step = one ``kubo_ahc`` call (the whole hot path: Fourier sum, eigensolver, rotations,
curvature, k-sum) over a slab of ``--planes`` k_1-planes of the mesh (planes x 128 x 128
k-points).  The headline is the mixed-precision form (tensor-core Fourier sum, FP64
eigensolver, FP32 rotations); the plain FP64 path and the double-float-eigensolver variant
are timed beside it on the same slabs, with their errors against the FP64 path.  Ranks (torchrun, one GPU each) take disjoint slabs: weak scaling, no data-path
collective.  Timed: exactly K steps after W warm-up steps, CUDA events on the library's
stream (torch's current stream), barrier + synchronize on both sides, max over ranks.

``--impl reference`` times the FP64 CPU oracle (tests' reference) on the host cores instead.

Other workloads (``--workload``, one JSON line each, not the headline):
  batched  64 uneven models (W 8..96, R boxes 7^3..11^3, meshes 32^3..64^3), one
           kubo_ahc_batched call over every model's whole mesh
  grad     W = 32, N_R = 729, 48^3 mesh, kT = 25 meV, eta = 5e-3: kubo_ahc_grad (FP64)
  sweep    W = 128, N_R = 1331, 96^3 mesh, 512 Fermi levels x 4 etas (slabs of the mesh)
  pad      the W = 64 workload with padded (W + 1) and unpadded (W) shared-memory matrices in
           the eigenvector and rotation kernels: the padding ablation
  separable the W = 64 workload with the separable Fourier sum (FP64, and with FP32 rotations)
           next to the dense contraction
"""
from __future__ import annotations

import argparse
import json
import os
import resource
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import tbgen  # noqa: E402

METRIC = "k-points/sec for σ_xy (W=64, N_R=1331), mixed vs FP64 GPU at rel err ≤1e-5; % roofline"
WORKLOAD = "w64_r1331_k128"
FP64_PEAK_TFLOPS = 152 * 4 * 2.07e9 / 1e12   # 152 SMs x 4 FP64 flop/clk/SM x 2.07 GHz (derived)
FP32_PEAK_TOPS = 152 * 128 * 2.07e9 / 1e12   # FP32 pipe: 152 SMs x 128 lanes x 2.07 GHz (derived)
# padded K of the tensor-core Fourier contraction (N_R = 1331 -> multiple of 64)
TC_KPAD = (1331 + 63) // 64 * 64
# minimal FP32 operations of one double-float multiply-accumulate (TwoProd by FMA with the two
# cross terms, Knuth's TwoSum into the accumulator, the low-part update)
DF_OPS_PER_MAC = 12
# DRAM bytes (read + write) per k-point of the kernels that can dominate a step, by (path,
# stage), from one ncu capture of the current kernel (profiles/, W = 64); a kernel that
# changes after its capture leaves this table.
DRAM_BYTES_PER_K = {("mixed", "tridiag"): 87.0e3, ("mixed_df", "tridiag"): 97.3e3}
# algorithmic flops per k-point by stage (useful work of each step of the method)
def stage_flops(W, N_R, prec="fp64"):
    """Algorithmic flops per k-point of each stage (useful work, not issued slice products).

    Eigenvector stage ("backtransform"): inverse iteration for the eigenvectors Z of the
    tridiagonal, then U = Q D Z (8 W^3) -- in FP64 on the FP64 path, in FP32 on the reduced
    ones: by a kernel of its own before the 3xTF32 rotation (W > 40, the default there), inside
    the SIMT rotation kernel otherwise (counted in "berry").
    """
    mixed = prec != "fp64"
    asm_in_rotation = mixed and W <= 40
    return {
        "fourier": 6.0 * N_R * W * W,     # real contraction [3 x N_R] . [N_R x W^2]
        "tridiag": 16.0 / 3.0 * W ** 3,   # complex Householder reduction
        "ql": 25.0 * 1.2 * W * W,         # ~1.2 W^2 Givens steps of ~25 flops
        "backtransform": 42.0 * W * W + (0.0 if asm_in_rotation else 8.0 * W ** 3),
        # two Hermitian rotations U^H dH U (+ the FP32 assembly of U when it runs inside)
        "berry": 24.0 * W ** 3 + (8.0 * W ** 3 if asm_in_rotation else 0.0),
        "ksum": 2.0 * W * 64,
        "prep": 0.0,
        "fixup": 0.0,
        "adjoint": 0.0,
    }


def measured_peaks():
    """bf16 burst / sustained TFLOP/s and HBM GB/s from MEASURED_PEAKS.json (else the fallback)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return {"bf16": float(d["bf16_tflops"]), "bf16_sustained": float(d["bf16_tflops_sustained"]),
                "hbm_gbs": float(d["hbm_gbs"]), "how": "measured"}
    except (OSError, KeyError, ValueError):
        return {"bf16": 1900.0, "bf16_sustained": 1700.0, "hbm_gbs": 6800.0, "how": "fallback"}


def issued_tc_flops_per_k(W, prec):
    """BF16 slice-pair products the tensor-core Fourier sum issues per k-point: 10 pairs (4
    slices per operand) on the W^2 columns of H, 6 pairs (3 slices) on the 2 W^2 velocity
    columns when the rotation that consumes them is FP32 (else 10 there too); x 2 flops x the
    padded K."""
    vel_pairs = 6 if prec in ("mixed", "mixed_df", "mixed_rotation") else 10
    return 2.0 * TC_KPAD * (10 * W * W + vel_pairs * 2 * W * W)


def roofline_of(dom, head, W, N_R, k_per_launch, ms_per_launch):
    """Roofline of the dominant kernel: algorithmic work per launch / its average duration,
    against the peak of the pipe that kernel runs on."""
    t = ms_per_launch / 1e3
    if head == "mixed_df" and dom == "tridiag":
        ops = DF_OPS_PER_MAC * (8.0 / 3.0) * W ** 3 * k_per_launch
        return {"bound": "alu", "achieved": ops / t / 1e12, "peak": FP32_PEAK_TOPS,
                "unit": "T FP32-op/s",
                "peak_note": "FP32 pipe: 152 SMs x 128 lanes x 2.07 GHz (derived).  Work: the "
                             "double-float reduction's 8/3 W^3 real multiply-adds at the minimal "
                             f"{DF_OPS_PER_MAC} FP32 operations each"}
    if head != "fp64" and dom == "berry":
        fl = stage_flops(W, N_R, head)["berry"] * k_per_launch
        return {"bound": "alu", "achieved": fl / t / 1e12, "peak": 2 * FP32_PEAK_TOPS,
                "unit": "TFLOP/s", "peak_note": "FP32 FMA: 152 SMs x 128 lanes x 2 flop x 2.07 GHz "
                                                "(derived); the rotations' 24 W^3 (+ the U assembly's 8 W^3 at W <= 40)"}
    if head != "fp64" and dom == "fourier":
        fl = issued_tc_flops_per_k(W, head) * k_per_launch   # issued BF16 slice products
        pk = measured_peaks()
        return {"bound": "tensor", "achieved": fl / t / 1e12, "peak": pk["bf16_sustained"],
                "unit": "TFLOP/s",
                "peak_note": f"bf16 dense sustained, {pk['how']}; work: issued BF16 slice-pair products"}
    fl = stage_flops(W, N_R, head)[dom] * k_per_launch
    return {"bound": "alu", "achieved": fl / t / 1e12, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "peak_note": "FP64 pipe: 152 SMs x 4 flop/clk/SM (one DFMA warp instruction per 16 "
                         "cycles, measured) x 2.07 GHz (derived; measured DFMA loop 1.199 TFLOP/s)"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="kubo", choices=["kubo", "reference"])
    ap.add_argument("--precision", default="both", choices=["both", "mixed", "fp64", "mixed_df"],
                    help="both = the mixed headline, the FP64 path and the double-float variant")
    ap.add_argument("--planes", type=int, default=4, help="k_1-planes of the 128^3 mesh per step")
    ap.add_argument("--cpu-sample", type=int, default=768, help="k-points for the CPU oracle baseline")
    ap.add_argument("--chunk", type=int, default=0, help="k-points per internal batch (0 = auto)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--rotation", default=None, choices=["simt", "exact", "tf32"],
                    help="step (3) kernel of the reduced modes (default: the library's)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the compact batched / grad / sweep results of the default line")
    ap.add_argument("--workload", default="w64", choices=["w64", "batched", "grad", "sweep", "pad", "separable"])
    return ap.parse_args()


# ------------------------------------------------------------------ sharding (N > 1 ranks)
def slab_of(rank, world, step, n_slabs):
    """k1-slab a rank evaluates at a step: within a step the ranks take consecutive slabs, so
    ranks never share work while world <= n_slabs (the k-points are independent: weak scaling,
    no data-path collective)."""
    return (step * world + rank) % n_slabs


def max_over_ranks(x, dist, device):
    """The step time of the slowest rank (every rank gets it)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def workload():
    model, kmesh, E_F, etas, kT = tbgen.config(WORKLOAD)
    return model, kmesh, E_F, float(etas[0]), kT


# ------------------------------------------------------------------ clocks
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.gpu = gpu_index
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.QUERY,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = [l.strip().split(",") for l in open(self.f.name) if l.strip()]
        os.unlink(self.f.name)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                smax = float(r[2])
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ reference arm
def run_reference(args, rank, world):
    if rank != 0:
        return
    from oracle import kubo_oracle as O
    model, kmesh, E_F, eta, kT = workload()
    plane = kmesh[1] * kmesh[2]
    n_per_step = 64
    rng = np.random.default_rng(0)
    times, cpus = [], []
    for s in range(args.warmup + args.steps):
        base = (s * args.planes) % kmesh[0] * plane
        kidx = np.sort(rng.choice(args.planes * plane, n_per_step, replace=False)) + base
        r0 = resource.getrusage(resource.RUSAGE_SELF)
        t0 = time.perf_counter()
        O.ahc(model.H_R, model.R, kmesh, E_F, etas=[eta], kT=kT, kidx=kidx)
        dt = time.perf_counter() - t0
        r1 = resource.getrusage(resource.RUSAGE_SELF)
        if s >= args.warmup:
            times.append(dt)
            cpus.append((r1.ru_utime - r0.ru_utime) + (r1.ru_stime - r0.ru_stime))
    tot = sum(times)
    value = n_per_step * args.steps / tot
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    sample = (f"{n_per_step} random k-points of each step's slab, numpy/LAPACK FP64 oracle "
              f"({sum(cpus) / tot:.1f} cores busy on average)")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "k-points/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded tbgen model)",
        "config": {"workload": WORKLOAD, "W": 64, "N_R": 1331, "kmesh": list(kmesh), "n_EF": 64,
                   "eta": eta, "k_per_step": n_per_step},
        "cpu_baseline": {"value": value, "unit": "k-points/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "k-points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# ------------------------------------------------------------------ library arm
def cpu_baseline(model, kmesh, E_F, eta, kT, n):
    from oracle import kubo_oracle as O
    kidx = tbgen.k_sample(kmesh, n, seed=123)
    r0 = resource.getrusage(resource.RUSAGE_SELF)
    t0 = time.perf_counter()
    O.ahc(model.H_R, model.R, kmesh, E_F, etas=[eta], kT=kT, kidx=kidx)
    dt = time.perf_counter() - t0
    r1 = resource.getrusage(resource.RUSAGE_SELF)
    cpu = (r1.ru_utime - r0.ru_utime) + (r1.ru_stime - r0.ru_stime)
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    return {"value": n / dt, "unit": "k-points/s", "cores": cores, "kind": "oracle",
            "sample": f"{n} seeded random k-points of the 128^3 mesh ({dt:.1f} s wall, "
                      f"{cpu:.1f} s CPU: {cpu / dt:.1f} cores busy on average), numpy/LAPACK FP64"}


def stage_table(st, fl, k_total):
    tot = max(1e-9, sum(x["ms"] for x in st.values()))
    return {s: {"launches": v["launches"], "ms": round(v["ms"], 3), "share": round(v["ms"] / tot, 4),
                "tflops": round(fl[s] * k_total / (v["ms"] / 1e3) / 1e12, 4)
                if v["ms"] > 0 and fl[s] > 0 else None}
            for s, v in st.items()}


# ------------------------------------------------------------------ other workloads
def _timed(fn, steps, warmup, local):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(steps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / steps, clocks.stop()


def workload_batched(kubo, torch, dev, steps, warmup, local, prec, every=1):
    """64 uneven models (tbgen.batch_recipe), one kubo_ahc_batched call per step over every
    model's whole mesh; every > 1 keeps each every-th model (a bounded slab of the batch)."""
    rec = tbgen.batch_recipe()[::every]
    P, nk = [], 0
    for r in rec:
        m = tbgen.random_tb(r["W"], r["half_width"], r["decay"], r["seed"])
        H = torch.from_numpy(m.H_R).to(dev)
        # Fermi level: midpoint of the two middle levels of H(k=0), from the library itself
        Hp, _, _ = kubo.bloch(H, m.R, (1, 1, 1), torch.zeros(1, dtype=torch.int64, device=dev))
        E, _ = kubo.eigh_batched(Hp, m.W, vectors=False)
        E = E[0].cpu().numpy()
        h = (m.W + 1) // 2
        ef = 0.5 * (E[h - 1] + E[h])
        P.append((H, m.R, (r["mesh"],) * 3, torch.tensor([ef], dtype=torch.float64, device=dev)))
        nk += r["mesh"] ** 3
    sched = {}

    def step():
        _, sc, _ = kubo.ahc_batched(P, precision=prec, tune=True)
        sched.update(sc)
    ms, clk = _timed(step, steps, warmup, local)
    return {"value": nk / (ms / 1e3), "unit": "k-points/s", "ms_per_step": ms,
            "models": len(P), "k_points": nk, "precision": prec, "schedule": sched, "clocks": clk,
            "workload": "batch64_w8-96_r343-1331_k32-64" + (f"[::{every}]" if every > 1 else "")}


def workload_grad(kubo, torch, dev, steps, warmup, local, k_limit=0):
    """W = 32, N_R = 729, 48^3 mesh, kT = 25 meV, eta = 5e-3: value + gradient (FP64);
    k_limit > 0 evaluates the first k_limit k-points of the mesh (a bounded slab)."""
    model, kmesh, E_F, etas, kT = tbgen.config("w32_r729_k48_fd")
    H = torch.from_numpy(model.H_R).to(dev)
    EF = torch.from_numpy(E_F).to(dev)
    g = torch.ones((1, E_F.size), dtype=torch.float64, device=dev)
    nk = int(np.prod(kmesh)) if k_limit <= 0 else int(k_limit)
    rng = None if k_limit <= 0 else (0, nk)
    prof = kubo.Profile()

    def step():
        kubo.ahc_grad(H, model.R, kmesh, EF, g, eta=float(etas[0]), kT=kT, with_value=True,
                      profile=prof, k_range=rng)
    ms, clk = _timed(step, steps, warmup, local)
    ms_f, _ = _timed(lambda: kubo.ahc(H, model.R, kmesh, EF, eta=float(etas[0]), kT=kT, k_range=rng),
                     steps, 1, local)
    return {"value": nk / (ms / 1e3), "unit": "k-points/s", "ms_per_step": ms, "k_per_step": nk,
            "forward_only": {"value": nk / (ms_f / 1e3), "ms_per_step": ms_f}, "dtype": "f64",
            "stages": {k: v for k, v in prof.as_dict().items() if v["launches"]}, "clocks": clk,
            "workload": "w32_r729_k48_fd", "W": model.W, "N_R": model.N_R, "kmesh": list(kmesh),
            "kT": kT, "eta": float(etas[0])}


def workload_sweep(kubo, torch, dev, steps, warmup, local, prec, planes):
    """W = 128, N_R = 1331, 96^3 mesh, 512 Fermi levels x 4 broadenings, slabs of k1-planes."""
    model, kmesh, E_F, etas, kT = tbgen.config("w128_r1331_k96")
    H = torch.from_numpy(model.H_R).to(dev)
    EF = torch.from_numpy(E_F).to(dev)
    k_step = planes * kmesh[1] * kmesh[2]
    state = {"s": 0}

    def step():
        s = state["s"] % (kmesh[0] // planes)
        state["s"] += 1
        kubo.ahc(H, model.R, kmesh, EF, etas=list(etas), kT=kT, precision=prec,
                 k_range=(s * k_step, (s + 1) * k_step))
    ms, clk = _timed(step, steps, warmup, local)
    return {"value": k_step / (ms / 1e3), "unit": "k-points/s", "ms_per_step": ms,
            "k_per_step": k_step, "precision": prec, "clocks": clk, "workload": "w128_r1331_k96"}


def run_extra(args, local):
    """Informational lines for the other workloads (see the module docstring)."""
    import torch
    import paper_2309_06675_gb300 as kubo
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    line = {"n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "data": "synthetic (tbgen)", "unit": "k-points/s"}
    prec = "mixed" if args.precision == "both" else args.precision
    if args.workload == "batched":
        r = workload_batched(kubo, torch, dev, args.steps, args.warmup, local, prec)
        line.update(metric="k-points/sec over a batch of 64 uneven models (one kubo_ahc_batched call)",
                    value=r["value"], ms_per_step=r["ms_per_step"], dtype=prec,
                    config={k: r[k] for k in ("workload", "models", "k_points", "precision", "schedule")},
                    clocks=r["clocks"])
    elif args.workload == "grad":
        r = workload_grad(kubo, torch, dev, args.steps, args.warmup, local)
        line.update(metric="k-points/sec for dσ_xy/dH(R) (value and gradient, FP64)",
                    value=r["value"], ms_per_step=r["ms_per_step"], dtype="f64",
                    config={k: r[k] for k in ("workload", "W", "N_R", "kmesh", "kT", "eta")},
                    forward_only=r["forward_only"], stages=r["stages"], clocks=r["clocks"])
    elif args.workload == "pad":
        model, kmesh, E_F, etas, kT = tbgen.config(WORKLOAD)
        H = torch.from_numpy(model.H_R).to(dev)
        EF = torch.from_numpy(E_F).to(dev)
        plane = kmesh[1] * kmesh[2]
        k_step = args.planes * plane
        res = {}
        for p in ("fp64", "mixed"):
            for unp in (False, True):
                prof = kubo.Profile()
                # the ablation's subject is the SIMT rotation kernel's shared-memory layout
                ms, _ = _timed(lambda: kubo.ahc(H, model.R, kmesh, EF, eta=float(etas[0]), precision=p,
                                                k_range=(0, k_step), profile=prof, unpadded=unp,
                                                rotation="simt"),
                               args.steps, args.warmup, local)
                st = prof.as_dict()
                n = args.steps + args.warmup
                res[f"{p}_{'unpadded' if unp else 'padded'}"] = {
                    "k_per_s": k_step / (ms / 1e3),
                    "backtransform_ms": st["backtransform"]["ms"] / n, "berry_ms": st["berry"]["ms"] / n}
        line.update(metric="padding ablation: k-points/s with padded vs unpadded shared-memory matrices",
                    value=res["fp64_padded"]["k_per_s"], ms_per_step=None, dtype="f64",
                    config={"workload": WORKLOAD, "k_per_step": k_step}, ablation=res)
    elif args.workload == "separable":
        model, kmesh, E_F, etas, kT = tbgen.config(WORKLOAD)
        H = torch.from_numpy(model.H_R).to(dev)
        EF = torch.from_numpy(E_F).to(dev)
        k_step = args.planes * kmesh[1] * kmesh[2]
        res, outs = {}, {}
        for name, kw in (("fp64_dense", {}), ("fp64_separable", {"separable": True}),
                         ("mixed_rotation_separable", {"separable": True, "precision": "mixed_rotation"})):
            prof = kubo.Profile()
            ms, _ = _timed(lambda: outs.__setitem__(name, kubo.ahc(H, model.R, kmesh, EF, eta=float(etas[0]),
                                                                   k_range=(0, k_step), profile=prof, **kw)),
                           args.steps, args.warmup, local)
            n = args.steps + args.warmup
            res[name] = {"k_per_s": k_step / (ms / 1e3),
                         "stages_ms": {k: v["ms"] / n for k, v in prof.as_dict().items() if v["launches"]}}
        ref = outs["fp64_dense"].cpu().numpy()
        for name in ("fp64_separable", "mixed_rotation_separable"):
            o = outs[name].cpu().numpy()
            res[name]["rel_err_vs_dense"] = float(np.max(np.abs(o - ref)) / np.max(np.abs(ref)))
        line.update(metric="k-points/sec with the separable Fourier sum vs the dense contraction (W=64)",
                    value=res["fp64_separable"]["k_per_s"], ms_per_step=None, dtype="f64",
                    config={"workload": WORKLOAD, "k_per_step": k_step}, separable=res)
    else:  # sweep
        r = workload_sweep(kubo, torch, dev, args.steps, args.warmup, local, prec, args.planes)
        line.update(metric="k-points/sec for σ_xy (W=128, N_R=1331, 512 E_F x 4 eta)",
                    value=r["value"], ms_per_step=r["ms_per_step"], dtype=prec,
                    config={"workload": r["workload"], "k_per_step": r["k_per_step"], "precision": prec},
                    clocks=r["clocks"])
    print(json.dumps(line))


DTYPE = {"mixed": "bf16-slices(Ozaki) Fourier + f64 eigh (f64 Householder, inverse iteration and "
                  "Rayleigh-quotient eigenvalues; QL shifts in f32 pairs) + 3xtf32 rotation + "
                  "f64 denominators/k-sum",
         "mixed_df": "bf16-slices(Ozaki) Fourier + double-float(f32 pairs) eigh + 3xtf32 rotation",
         "fp64": "f64"}


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.workload != "w64":
        return run_extra(args, local)

    import torch
    import paper_2309_06675_gb300 as kubo
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    model, kmesh, E_F, eta, kT = workload()
    plane = kmesh[1] * kmesh[2]
    n_slabs = kmesh[0] // args.planes
    k_per_step = args.planes * plane
    H = torch.from_numpy(model.H_R).to(dev)
    EF = torch.from_numpy(E_F).to(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    precisions = ["mixed", "fp64", "mixed_df"] if args.precision == "both" else [args.precision]

    def slab(step):
        s = slab_of(rank, world, step, n_slabs)
        return (s * k_per_step, (s + 1) * k_per_step)

    def timed(prec, rotation=None, ql_fp64=False):
        outs = []
        def one_step(step, prof=None):
            flush.fill_(step & 0xFF)   # evict L2 (256 MiB > 135 MB) before every step
            o = torch.empty((1, E_F.size), dtype=torch.float64, device=dev)
            kubo.ahc(H, model.R, kmesh, EF, eta=eta, kT=kT, precision=prec, k_range=slab(step),
                     out=o, profile=prof, chunk_k=args.chunk, rotation=rotation, ql_fp64=ql_fp64)
            return o
        for s in range(args.warmup):
            one_step(s)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        prof = kubo.Profile()
        clocks = ClockSampler(local)
        clocks.start()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record()
        for s in range(args.steps):
            outs.append(one_step(args.warmup + s, prof))
        ev1.record()
        torch.cuda.synchronize()
        clk = clocks.stop()
        ms = max_over_ranks(ev0.elapsed_time(ev1), dist, dev)
        if dist:
            dist.barrier()
        d = prof.as_dict()
        d["_fixup_k"] = int(prof.fixup_k)
        return ms, d, clk, torch.cat(outs).cpu().numpy()

    res = {p: timed(p, rotation=args.rotation) for p in precisions}
    # the mixed form with the other step (3) kernels (labelled variants, same slabs)
    rot_res = {}
    if args.precision == "both" and not args.no_extras and args.rotation is None:
        rot_res = {r: timed("mixed", rotation=r) for r in ("simt", "exact")}
    # the mixed form with its QL iteration in FP64 as well (every eigensolver operation FP64)
    ql64 = timed("mixed", rotation=args.rotation, ql_fp64=True) if args.precision == "both" else None

    # ---- end to end through the host-buffer entry point (pinned host memory), headline path
    head = precisions[0]
    e2e = None
    if not args.no_e2e:
        H_pin = torch.from_numpy(model.H_R).pin_memory()
        EF_pin = torch.from_numpy(E_F).pin_memory()
        h2d = H_pin.numel() * 16 + EF_pin.numel() * 8
        d2h = E_F.size * 8
        kubo.ahc_host(H_pin.numpy(), model.R, kmesh, EF_pin.numpy(), eta=eta, kT=kT,
                      precision=head, k_range=slab(0))
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for s in range(args.steps):
            flush.fill_(s & 0xFF)
            kubo.ahc_host(H_pin.numpy(), model.R, kmesh, EF_pin.numpy(), eta=eta, kT=kT,
                          precision=head, k_range=slab(args.warmup + s))
        torch.cuda.synchronize()
        dt = max_over_ranks(time.perf_counter() - t0, dist, dev)
        e2e = {"value": world * args.steps * k_per_step / dt, "unit": "k-points/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h), "precision": head}

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    k_total = args.steps * k_per_step
    paths = {}
    fixup_k = {p: r[1].pop("_fixup_k") for p, r in res.items()}
    for p, (ms, st, clk, outs) in res.items():
        paths[p] = {"value": world * k_total / (ms / 1e3), "ms_per_step": ms / args.steps,
                    "stages": stage_table(st, stage_flops(model.W, model.N_R, p), k_total),
                    "gpu_launches": int(sum(v["launches"] for v in st.values())), "clocks": clk}

    def roofline_for(p):
        st = res[p][1]
        dom = max((s for s in st if st[s]["launches"] > 0), key=lambda s: st[s]["ms"])
        launches = st[dom]["launches"]
        k_per_launch = k_total / launches
        rl = roofline_of(dom, p, model.W, model.N_R, k_per_launch, st[dom]["ms"] / launches)
        key = (p, dom)
        traffic = (DRAM_BYTES_PER_K[key] * k_per_launch
                   if key in DRAM_BYTES_PER_K and model.W == 64 else None)
        return {"bound": rl["bound"], "kernel": dom, "achieved": rl["achieved"], "peak": rl["peak"],
                "unit": rl["unit"], "frac": rl["achieved"] / rl["peak"], "traffic": traffic,
                "traffic_unit": "bytes per launch (ncu dram__bytes_read.sum + write.sum, scaled "
                                "by k-points per launch)",
                "peak_note": rl["peak_note"]}

    ms, st, clk, outs = res[head]
    line = {
        "metric": METRIC, "value": paths[head]["value"], "unit": "k-points/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPE.get(head, head),
        "data": "synthetic (seeded random TB model, tbgen.random_tb)",
        "config": {"workload": WORKLOAD, "W": model.W, "N_R": model.N_R, "kmesh": list(kmesh),
                   "n_EF": int(E_F.size), "eta": eta, "precision": head,
                   "eigensolver": {"fp64": "f64",
                                   "mixed": "f64 (Householder, inverse iteration, Rayleigh-quotient "
                                            "eigenvalues; QL shifts in f32 pairs)"}.get(
                                       head, "double-float (f32 pairs)"),
                   "k_per_step": k_per_step, "chunk_k": args.chunk or "auto",
                   "parallelism": f"k-slabs x{world}",
                   "l2": "flushed (256 MiB write) before every step; per-step working set >> L2"},
        "roofline": roofline_for(head),
        "stages": paths[head]["stages"],
        "gpu_launches": paths[head]["gpu_launches"],
        "clocks": clk,
        "e2e": e2e,
    }
    if "fp64" in res:
        of = res["fp64"][3]
        den = np.maximum(np.max(np.abs(of), axis=1, keepdims=True), 1e-300)

        def rel_vs_fp64(p):
            return float(np.max(np.abs(res[p][3] - of) / den))
        if "mixed" in res:
            tc = res["mixed"][1]["fourier"]
            fl = stage_flops(model.W, model.N_R, "mixed")
            pk = measured_peaks()
            line["mixed_vs_fp64"] = {
                "speedup": paths["mixed"]["value"] / paths["fp64"]["value"],
                "fixup_fraction": fixup_k["mixed"] / k_total,
                "rel_err_max_over_steps": rel_vs_fp64("mixed"),
                "fp64": {k: paths["fp64"][k] for k in ("value", "ms_per_step", "stages", "gpu_launches")},
                "fp64_roofline": roofline_for("fp64"),
                "tensor_core_fourier": {
                    "useful_tflops": fl["fourier"] * k_total / (tc["ms"] / 1e3) / 1e12,
                    "issued_bf16_tflops": issued_tc_flops_per_k(model.W, "mixed") * k_total
                                          / (tc["ms"] / 1e3) / 1e12,
                    "bf16_peak_tflops": pk["bf16"], "bf16_peak_sustained_tflops": pk["bf16_sustained"],
                    "peak_source": pk["how"] + " (MEASURED_PEAKS.json)",
                    "note": "stage = coef_slice + fourier_tc (tcgen05, fixed-point BF16 slices: 10 "
                            "slice-pair products on the H columns, 6 on the velocity columns; exact "
                            "FP32 block sums)"},
            }
        if rot_res:
            line["mixed_rotation_kernels"] = {
                "what": "the mixed form with step (3) in FP32 on the FMA pipe (simt) or on the "
                        "tensor cores with exact fixed-point BF16 slices (exact), instead of the "
                        "default 3xTF32 tensor-core kernel (tcgen05 kind::tf32)",
                **{r: {"value": world * k_total / (v[0] / 1e3),
                       "berry_ms_per_step": v[1]["berry"]["ms"] / args.steps,
                       "rel_err_max_over_steps": float(np.max(np.abs(v[3] - of) / den))}
                   for r, v in rot_res.items()},
                "tf32_berry_ms_per_step": res["mixed"][1]["berry"]["ms"] / args.steps}
        if ql64 is not None:
            line["mixed_ql_fp64_variant"] = {
                "what": "the headline form with kubo_options.ql_fp64 = 1: the QL iteration in FP64 "
                        "too and its eigenvalues reported (the default runs QL in FP32 pairs for "
                        "the inverse iteration's shifts and reports FP64 Rayleigh quotients)",
                "value": world * k_total / (ql64[0] / 1e3), "ms_per_step": ql64[0] / args.steps,
                "ql_ms_per_step": ql64[1]["ql"]["ms"] / args.steps,
                "speedup_vs_fp64": world * k_total / (ql64[0] / 1e3) / paths["fp64"]["value"],
                "rel_err_max_over_steps": float(np.max(np.abs(ql64[3] - of) / den))}
        if "mixed_df" in res:
            line["mixed_df_variant"] = {
                "what": "the mixed form with its eigensolver in double-float (FP32 pairs, ~2^-46 "
                        "per operation) instead of FP64: a labelled variant, not the headline",
                "value": paths["mixed_df"]["value"], "ms_per_step": paths["mixed_df"]["ms_per_step"],
                "speedup_vs_fp64": paths["mixed_df"]["value"] / paths["fp64"]["value"],
                "rel_err_max_over_steps": rel_vs_fp64("mixed_df"),
                "stages": paths["mixed_df"]["stages"], "roofline": roofline_for("mixed_df"),
                "gpu_launches": paths["mixed_df"]["gpu_launches"]}
    if not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(model, kmesh, E_F, eta, kT, args.cpu_sample)
    if not args.no_extras and world == 1:
        # compact results of the other workloads, one bounded slab each
        line["workloads"] = {
            "batched": workload_batched(kubo, torch, dev, 1, 1, local, "mixed", every=4),
            "grad": workload_grad(kubo, torch, dev, 2, 1, local, k_limit=8 * 48 * 48),
            "sweep": workload_sweep(kubo, torch, dev, 3, 1, local, "mixed", 2),
        }
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
