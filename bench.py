#!/usr/bin/env python3
"""Benchmark: PCG time to relative residual 1e-8, mixed precision vs FP64, on one GB300.

One step = one pass of the whole hot path on the 1024x512 MBB workload (1,051,650 DOFs,
periodic Bernoulli(0.4) 32x32 cell, filter radius 3, beta 8, coarse cells H = 32 with 6
eigenvectors): density filter + projection + SIMP, preconditioner build (agglomerate
de-duplication, local eigen-solves, coarse matrix, patch factors), MIXED flexible CG to a
true FP64 relative residual of 1e-8, compliance and design sensitivity.  Inputs are
resident in HBM; L2 is flushed (256 MiB write) before every timed step.

value        = mean device time of the MIXED solve (PCG to 1e-8), ms
fp64         = the same solve with the FP64 method on the same inputs
matvec       = FP32 matrix-free matvec on the 3200x4096 mesh (26.2M DOFs, inputs > L2)
roofline     = the dominant kernel of the step (event-timed inside this run)
cpu_baseline = the FP64 CPU oracle's PCG on the same workload (one full solve, one thread)
e2e          = the MIXED solve through mstopo_solve_host (pinned host f and u, copies timed)

--impl reference times the CPU oracle (the reference arm of this build) on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "PCG time to 1e-8 rel. residual & matvec GB/s, mixed vs FP64, up to 26M DOFs"
WORKLOAD = "mbb_c2"
WORKLOAD_DESC = ("MBB beam 1024x512 Q4 (1,051,650 DOFs), periodic 32x32 Bernoulli(0.4) void cell, "
                 "rmin 3, beta 8, eta 0.5, E0/Emin 1e9, p 3, H 32, 6 eigenvectors, tol 1e-8")
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}
# FP32 CUDA-core peak: 152 SMs x 128 FP32 lanes x 2 flop/FMA x 2.07 GHz (max SM clock)
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
# FP64 peak: 152 SMs x 2 FP64 FMA/clk (measured 1.19 TFLOP/s at ~1.95 GHz) x 2 x 2.07 GHz
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# DRAM bytes (read + write) of one FP32 patch-solve launch on the 1024x512 workload, from an
# ncu capture of `bench.py --only patch --reps 3` (dram__bytes_read.sum 106.02 MB +
# dram__bytes_write.sum 13.42 MB of k_patch_tri<float, 4, 1, 3, 1>, profiles/k_patch_tri_f32_mbb_c2.md);
# set to None whenever the kernel changes until it is captured again
PATCH_TRAFFIC_BYTES = 119_618_304


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return {"hbm_gbs": float(p["hbm_gbs"]), "bf16_tflops": float(p["bf16_tflops"]),
                "source": "measured"}
    except Exception:
        return {**PEAKS_FALLBACK, "source": "fallback"}


# ------------------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi clock / throttle-reason samples while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_id: str):
        self.device_id = device_id
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.device_id, f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            parts = [x.strip() for x in l.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "samples": len(sm),
                "reasons": sorted(reasons)}


# ------------------------------------------------------------------------ CPU oracle
_ORACLE_SETUP = """
import os, sys, time, json
sys.path.insert(0, {root!r})
import numpy as np
import workloads
from oracle import pipeline, msfem
wl = workloads.make({name!r})
grid, K0, prob, chain = pipeline.build(wl)
t0 = time.perf_counter()
fw = chain.forward(wl.rho)
tl = msfem.TwoLevel(prob, fw["E"][0], wl.H, wl.n_eig)
t1 = time.perf_counter()
Kf = prob.free_matrix(fw["E"][0])
f = grid.nodal_from_neutral(wl.force)[prob.free]
"""


def _oracle_env():
    return dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
                CUDA_VISIBLE_DEVICES="")


def _run_oracle(code: str, timeout: int = 1800) -> dict:
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True,
                       env=_oracle_env(), timeout=timeout)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def oracle_full_solve() -> dict:
    """The FP64 oracle's two-level PCG on the whole benchmark workload (not a reduced copy),
    to the same tolerance, in a fresh process limited to one BLAS thread: build time and
    solve time measured separately."""
    code = _ORACLE_SETUP.format(root=ROOT, name=WORKLOAD) + """
t2 = time.perf_counter()
x, it, rr = msfem.pcg(Kf, f, tl.apply, tol=wl.tol)
t3 = time.perf_counter()
print(json.dumps({"build_s": t1 - t0, "solve_s": t3 - t2, "iterations": it, "rel_residual": rr,
                  "dofs": grid.n_dof, "nelx": wl.nelx, "nely": wl.nely}))
"""
    return _run_oracle(code)


def oracle_iteration_samples(n_iter: int, steps: int, warmup: int) -> dict:
    """Bounded samples of the same oracle PCG on the whole workload: the preconditioner is
    built once (timed separately); then every step runs n_iter PCG iterations from zero
    (the same iterations the full solve starts with) and is timed on its own."""
    code = _ORACLE_SETUP.format(root=ROOT, name=WORKLOAD) + f"""
steps = []
for s in range({warmup} + {steps}):
    t2 = time.perf_counter()
    msfem.pcg(Kf, f, tl.apply, tol=1e-300, maxit={n_iter})
    t3 = time.perf_counter()
    if s >= {warmup}:
        steps.append(t3 - t2)
print(json.dumps({{"build_s": t1 - t0, "step_s": steps, "dofs": grid.n_dof}}))
"""
    return _run_oracle(code)


def cpu_baseline() -> dict:
    s = oracle_full_solve()
    return {"value": s["solve_s"] * 1e3, "unit": "ms", "cores": 1, "kind": "oracle",
            "iterations": s["iterations"], "rel_residual": s["rel_residual"],
            "build_s": s["build_s"], "host_cpus": os.cpu_count(),
            "sample": (f"the whole {s['nelx']}x{s['nely']} workload ({s['dofs']} DOFs): the "
                       f"oracle's two-level PCG to 1e-8, {s['iterations']} iterations, one run; "
                       f"preconditioner build {s['build_s']:.1f} s reported separately, not "
                       f"included; SuperLU and NumPy on one thread")}


# ------------------------------------------------------------------------------ our arm
def max_over_ranks(values, world: int, device="cpu"):
    """Each timing's maximum over the ranks: the replicas run concurrently, so the slowest
    one sets the job's time.  One all-reduce over the default process group (NCCL on the
    GPUs; any backend works)."""
    import torch
    t = torch.tensor(list(values), dtype=torch.float64, device=device)
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return t.tolist()


def run_ours(args, rank: int, world: int):
    import numpy as np
    import torch

    import paper_1411_3923_gb300 as m
    import workloads

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    peaks = load_peaks()
    wl = workloads.make(WORKLOAD)
    rho = torch.from_numpy(wl.rho).to(dev)
    f = torch.from_numpy(wl.force).to(dev)

    # the FP32 patch-solve configuration is autotuned: the first (warm-up) build times each
    # candidate, the timed steps keep the choice
    def problem(prec, preconditioner="additive", krylov="fcg"):
        return m.Problem(wl.nelx, wl.nely, wl.fixed, nu=wl.nu, E0=wl.E0, Emin=wl.Emin,
                         penal=wl.penal, H=wl.H, n_eig=wl.n_eig, precision=prec, tol=wl.tol,
                         max_iter=5000, preconditioner=preconditioner, krylov=krylov,
                         autotune=not args.no_autotune)

    mixed, fp64 = problem("mixed"), problem("fp64")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step(prob, ev):
        ev[0].record()
        prob.set_design(rho, wl.rmin, wl.beta, wl.etas, wl.cell)
        ev[1].record()
        binfo = prob.build_preconditioner(-1)
        ev[2].record()
        _, infos = prob.solve(f, -1)
        ev[3].record()
        c, fr, g = prob.compliance_and_sensitivity(1.0)
        ev[4].record()
        return binfo, infos, c

    def new_events():
        return [torch.cuda.Event(enable_timing=True) for _ in range(5)]

    for _ in range(args.warmup):
        step(mixed, new_events())
        step(fp64, new_events())
    torch.cuda.synchronize()

    # ---- timed region: K steps of the MIXED path (no per-kernel events: CUDA graphs on) ----
    launches0 = mixed.stats()["launches"]
    dev_id = str(torch.cuda.get_device_properties(dev).uuid) if hasattr(
        torch.cuda.get_device_properties(dev), "uuid") else str(dev.index)
    if dev_id and not dev_id.startswith("GPU-") and len(dev_id) > 8:
        dev_id = "GPU-" + dev_id
    sampler = ClockSampler(dev_id)
    sampler.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    per = []
    t_wall0 = time.perf_counter()
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        ev = new_events()
        binfo, infos, c = step(mixed, ev)
        torch.cuda.synchronize()
        per.append({"design": ev[0].elapsed_time(ev[1]), "build": ev[1].elapsed_time(ev[2]),
                    "solve": ev[2].elapsed_time(ev[3]), "sens": ev[3].elapsed_time(ev[4]),
                    "step": ev[0].elapsed_time(ev[4]), "iters": [i["iterations"] for i in infos],
                    "res": [i["rel_residual"] for i in infos]})
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall0
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    launches = mixed.stats()["launches"] - launches0
    # ---- profiled pass: the same step with per-kernel events (graphs off) ----
    mixed.set_profiling(True)
    for _ in range(max(1, min(2, args.steps))):
        flush.zero_()
        torch.cuda.synchronize()
        step(mixed, new_events())
    torch.cuda.synchronize()
    st = mixed.stats()
    mixed.set_profiling(False)
    nprof = max(1, min(2, args.steps))

    solve_ms = statistics.mean(p["solve"] for p in per)
    step_ms = statistics.mean(p["step"] for p in per)

    # ---- FP64 method on the same inputs (same step, FP64 solve) ----
    per64 = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        ev = new_events()
        _, infos64, c64 = step(fp64, ev)
        torch.cuda.synchronize()
        per64.append({"solve": ev[2].elapsed_time(ev[3]), "iters": [i["iterations"] for i in infos64]})
    fp64_ms = statistics.mean(p["solve"] for p in per64)

    # ---- the paper's own preconditioner (Sec. 2.4.2: symmetric Gauss-Seidel, coarse
    #      correction, symmetric Gauss-Seidel, multiplicative) on the same inputs, MIXED ----
    sgs = problem("mixed", "sgs")
    for _ in range(args.warmup):
        step(sgs, new_events())
    persgs = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        ev = new_events()
        _, infos_s, c_s = step(sgs, ev)
        torch.cuda.synchronize()
        persgs.append({"solve": ev[2].elapsed_time(ev[3]), "build": ev[1].elapsed_time(ev[2]),
                       "iters": [i["iterations"] for i in infos_s],
                       "res": [i["rel_residual"] for i in infos_s]})
    sgs_ms = statistics.mean(p["solve"] for p in persgs)
    c_add = [i["compliance"] for i in infos]
    c_sgs = [i["compliance"] for i in infos_s]
    sgs.close()
    # the same preconditioner under the paper's outer method, GMRES(50)
    gm = problem("mixed", "sgs", "gmres")
    for _ in range(args.warmup):
        step(gm, new_events())
    pergm = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        ev = new_events()
        _, infos_g, c_g = step(gm, ev)
        torch.cuda.synchronize()
        pergm.append({"solve": ev[2].elapsed_time(ev[3]), "iters": [i["iterations"] for i in infos_g],
                      "res": [i["rel_residual"] for i in infos_g]})
    gm_ms = statistics.mean(p["solve"] for p in pergm)
    c_gm = [i["compliance"] for i in infos_g]
    gm.close()

    # ---- roofline of the dominant profiled kernel in the mixed step ----
    kern = {k: v for k, v in st.items() if isinstance(v, dict)}
    nsteps = nprof
    wl_N = 2 * wl.H + 1
    nb = 2 * wl_N
    n_agg = (wl.nelx // wl.H + 1) * (wl.nely // wl.H + 1)
    n_iter_total = sum(sum(p["iters"]) for p in per)
    # algorithmic work per launch
    nodes = (wl.nelx + 1) * (wl.nely + 1)
    # banded triangular-solve pair per patch: 4 n b flops, n = NL nb box DOFs, b = nb
    patch_flops = 4.0 * (wl_N * nb) * nb * n_agg * len(wl.etas)
    mv_bytes = nodes * 8 * 2 + wl.nelx * wl.nely * 4 + nodes          # u, y (float2), E, mask
    cand = []
    if kern["patch_solve"]["launches"]:
        t = kern["patch_solve"]["ms"] / kern["patch_solve"]["launches"]
        ach = patch_flops / (t * 1e-3) / 1e12
        cand.append((kern["patch_solve"]["ms"], {
            "kernel": "k_patch_tri<float>", "bound": "alu", "achieved": ach,
            "work": "4 n b flops per patch (n = 65 x 130 box DOFs, b = 130), 561 patches",
            "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": ach / FP32_PEAK_TFLOPS,
            "traffic": PATCH_TRAFFIC_BYTES, "traffic_unit": "B per launch (ncu)", "avg_launch_ms": t,
            "peak_source": "derived: 152 SMs x 128 FP32 FMA/clk x 2 x 2070 MHz"}))
    if kern["matvec_f32"]["launches"]:
        t = kern["matvec_f32"]["ms"] / kern["matvec_f32"]["launches"]
        ach = mv_bytes / (t * 1e-3) / 1e9
        cand.append((kern["matvec_f32"]["ms"], {
            "kernel": "k_matvec<float>", "bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"],
            "unit": "GB/s", "frac": ach / peaks["hbm_gbs"], "traffic": None, "avg_launch_ms": t}))
    cand.sort(key=lambda x: -x[0])
    roofline = cand[0][1] if cand else None
    shares = {k: {"launches": v["launches"], "ms_per_step": v["ms"] / nsteps} for k, v in kern.items()}

    # ---- FP32 matvec on the 26.2M-DOF mesh (inputs larger than L2) ----
    # headline: the flexible CG's own launch (all three realisations in one launch, inputs zero
    # at the Dirichlet DOFs); beside it the single-vector ABI call that reads the input mask
    mv = None
    pt5 = None
    if not args.skip_big_matvec:
        import numpy as np
        big = workloads.make("mbb_c5")
        pb = m.Problem(big.nelx, big.nely, big.fixed, nu=big.nu, E0=big.E0, Emin=big.Emin,
                       penal=big.penal, H=big.H, n_eig=big.n_eig, precision="mixed",
                       autotune=not args.no_autotune)
        pb.set_design(torch.from_numpy(big.rho).to(dev), big.rmin, big.beta, big.etas, big.cell)
        ns = len(big.etas)
        nb_nodes = (big.nelx + 1) * (big.nely + 1)
        free = torch.from_numpy(~np.asarray(big.fixed, dtype=bool).reshape(-1)).to(dev)
        u32 = torch.randn(ns, 2 * nb_nodes, device=dev, dtype=torch.float32) * free
        y32 = torch.empty_like(u32)
        # per system u 8 + y 8 B per node (float2) and E 4 B per element; the output mask
        # (1 B per node) is shared by the systems of one launch and counted once
        byts = nb_nodes * 8 * 2 + big.nelx * big.nely * 4                # one system
        mask_b = nb_nodes

        def timed(realisation, masked, reps=20):
            for _ in range(5):
                pb.apply_K_f32(u32, realisation, y32, input_masked=masked)
            pb.set_profiling(True)
            for _ in range(reps):
                flush.zero_()
                pb.apply_K_f32(u32, realisation, y32, input_masked=masked)
            sb = pb.stats()
            pb.set_profiling(False)
            return sb["matvec_f32"]["ms"] / max(sb["matvec_f32"]["launches"], 1)

        t_all = timed(-1, True)
        t_one = timed(0, False)
        gbs = (ns * byts + mask_b) / (t_all * 1e-3) / 1e9
        gbs1 = (byts + 2 * mask_b) / (t_one * 1e-3) / 1e9   # reads the input and output masks
        mv = {"mesh": f"{big.nelx}x{big.nely}", "dofs": 2 * nb_nodes, "systems_per_launch": ns,
              "launch": "flexible-CG configuration (3 realisations, inputs zero at Dirichlet DOFs)",
              "avg_launch_ms": t_all, "algorithmic_bytes": ns * byts + mask_b, "gbs": gbs,
              "peak_gbs": peaks["hbm_gbs"], "frac": gbs / peaks["hbm_gbs"],
              "bytes_per_node": "u 8 + y 8 (float2) + E 4/element per system, output mask 1 once per launch",
              "single_vector_masked_input": {"avg_launch_ms": t_one, "algorithmic_bytes": byts + 2 * mask_b,
                                             "gbs": gbs1, "frac": gbs1 / peaks["hbm_gbs"]}}
        del u32, y32

        # ---- FP32 patch solves on the same workload (realisation 0, one launch) with the
        #      kernel the automatic choice builds (the tensor cores here: 128 patches of a
        #      type per MMA, profiles/k_patch_twtc_mbb_c5_800x1024.md) ----
        bi5 = pb.build_preconditioner(-1)
        r5 = torch.randn((big.nely + 1, big.nelx + 1, 2), dtype=torch.float64, device=dev)
        for _ in range(3):
            pb.apply_precond(r5, m.MIXED, 2)
        pb.set_profiling(True)
        for _ in range(10):
            flush.zero_()
            pb.apply_precond(r5, m.MIXED, 2)
        sp = pb.stats()
        pb.set_profiling(False)
        t_p5 = sp["patch_solve"]["ms"] / max(sp["patch_solve"]["launches"], 1)
        nl5 = 2 * big.H + 1
        nb5 = 2 * nl5
        alg5 = 4.0 * nl5 * nb5 * nb5 * bi5["n_agglomerates"]       # 4 n b flops per patch solve
        tc5 = bi5["patch_kernel"] == 2
        groups5 = bi5["patch_groups"] // ns                          # realisation 0's groups
        ks5, npad5 = (nb5 + 7) // 8, (nb5 + 15) // 16 * 16
        # executed on the tensor cores: per group two CTAs x NL line steps x 3 KS MMAs of
        # 128 x npad x 8
        mma5 = 2.0 * groups5 * nl5 * 3 * ks5 * 2 * 128 * npad5 * 8
        tf32_peak = peaks["bf16_tflops"] / 2.0   # TF32 at half the BF16 rate (nominal ratio)
        pt5 = {
            "kernel": "k_patch_twtc<130> (tensor cores)" if tc5 else "k_patch_tri<float> (CUDA cores)",
            "choice": {0: "cost model", 1: "autotuned", 2: "autotuned earlier"}[bi5["patch_tuned"]],
            "cols": bi5["patch_cols"], "realisation": 0, "patches": bi5["n_agglomerates"],
            "types": bi5["n_types"], "groups": groups5, "avg_launch_ms": t_p5,
            "algorithmic_gflop": alg5 / 1e9,
            "fp32_equivalent_tflops": alg5 / (t_p5 * 1e-3) / 1e12,
            "frac_of_fp32_peak": alg5 / (t_p5 * 1e-3) / 1e12 / FP32_PEAK_TFLOPS,
            "tf32_mma_tflops": (mma5 / (t_p5 * 1e-3) / 1e12) if tc5 else None,
            "tf32_peak_tflops": tf32_peak if tc5 else None,
            "frac_of_tf32_peak": (mma5 / (t_p5 * 1e-3) / 1e12 / tf32_peak) if tc5 else None,
            "peak_source": "FP32: derived (152 SMs x 128 FMA/clk x 2 x 2070 MHz); TF32: measured "
                           "BF16 peak x the nominal TF32/BF16 ratio 1/2"}
        pb.close()

    # ---- e2e through the host-pointer entry point (pinned buffers, copies timed) ----
    fh = torch.from_numpy(wl.force).pin_memory()
    uh = torch.empty((len(wl.etas), wl.nely + 1, wl.nelx + 1, 2), dtype=torch.float64).pin_memory()
    mixed.set_design(rho, wl.rmin, wl.beta, wl.etas, wl.cell)
    mixed.build_preconditioner(-1)
    e2e_ms = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        mixed.solve_host(fh.numpy(), -1, u=uh.numpy())
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e = {"value": statistics.mean(e2e_ms), "unit": "ms", "h2d_bytes_per_step": fh.numel() * 8,
           "d2h_bytes_per_step": uh.numel() * 8,
           "api": "mstopo_solve_host (pinned host f in, u out)"}

    # ---- max over ranks ----
    solve_ms, step_ms, fp64_ms, e2e_v = max_over_ranks([solve_ms, step_ms, fp64_ms, e2e["value"]],
                                                       world, dev)
    e2e["value"] = e2e_v
    if rank != 0:
        return None
    out = {
        "metric": METRIC, "value": solve_ms, "unit": "ms", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
        "config": {"workload": WORKLOAD_DESC, "dofs": 2 * nodes, "realisations": len(wl.etas),
                   "l2": "flushed before every timed step (256 MiB write)",
                   "parallelism": f"replicas x{world}"},
        "paper_preconditioner": {
            "preconditioner": "multiplicative: SGS (4-colour node blocks), spectral coarse "
                              "correction, SGS (Sec. 2.4.2); same flexible CG, MIXED",
            "value": sgs_ms, "unit": "ms", "iterations": persgs[-1]["iters"],
            "rel_residual": persgs[-1]["res"],
            "build_ms": statistics.mean(p["build"] for p in persgs),
            "compliance_rel_diff_vs_additive": max(abs(a - b) / abs(a) for a, b in zip(c_add, c_sgs)),
            "gmres": {"method": "GMRES(50), right preconditioned, the paper's outer method "
                                "(Sec. 2.4.2), same preconditioner, MIXED",
                      "value": gm_ms, "unit": "ms", "iterations": pergm[-1]["iters"],
                      "rel_residual": pergm[-1]["res"],
                      "compliance_rel_diff_vs_additive": max(abs(a - b) / abs(a) for a, b in zip(c_add, c_gm))}},
        "fp64": {"value": fp64_ms, "unit": "ms", "iterations": per64[-1]["iters"],
                 "speedup_mixed_vs_fp64": fp64_ms / solve_ms},
        "mixed": {"iterations": per[-1]["iters"], "rel_residual": per[-1]["res"],
                  "phases_ms": {k: statistics.mean(p[k] for p in per)
                                for k in ("design", "build", "solve", "sens")},
                  "build": binfo},
        "matvec": mv, "patch_solve_26m": pt5, "roofline": roofline, "kernels": shares, "gpu_launches": launches,
        "clocks": clocks, "e2e": e2e, "wall_s_timed": t_wall, "peaks": peaks,
    }
    if not args.skip_cpu:
        out["cpu_baseline"] = cpu_baseline()
    return out


def run_reference(args, rank: int, world: int):
    """The reference arm: the FP64 CPU oracle, timed as it stands on the host cores (one BLAS
    thread) on the whole benchmark workload.  Its full PCG to 1e-8 runs once (that measures
    its iteration count N and its solve time); each timed step is then a bounded sample of
    the same solve, the first --ref-iterations PCG iterations from zero, and reports
    step time x (N + 1) / (--ref-iterations + 1) in the metric's unit (a PCG run of n
    iterations applies the preconditioner n + 1 times)."""
    if rank != 0:
        return None
    import workloads
    wl = workloads.make(WORKLOAD)
    t0 = time.perf_counter()
    full = oracle_full_solve()
    n_it = max(1, args.ref_iterations)
    smp = oracle_iteration_samples(n_it, args.steps, args.warmup)
    # a PCG run of n iterations applies the preconditioner n + 1 times (once before the loop)
    vals = [t * (full["iterations"] + 1) / (n_it + 1) * 1e3 for t in smp["step_s"]]
    v = statistics.mean(vals)
    sample = (f"the whole {wl.nelx}x{wl.nely} workload ({full['dofs']} DOFs): each step runs the "
              f"oracle's first {n_it} PCG iterations from zero ({statistics.mean(smp['step_s']):.2f} s) "
              f"and is scaled by (N + 1) / ({n_it} + 1) preconditioner applications, N the "
              f"oracle's own iteration count to 1e-8 on this workload "
              f"({full['iterations']}, measured in one full solve of {full['solve_s']:.1f} s); "
              f"build {smp['build_s']:.1f} s not included; one thread")
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": "ms", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": statistics.mean(smp["step_s"]) * 1e3,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD_DESC, "dofs": full["dofs"], "parallelism": "cpu oracle"},
            "full_solve": {"ms": full["solve_s"] * 1e3, "iterations": full["iterations"],
                           "rel_residual": full["rel_residual"], "build_s": full["build_s"]},
            "cpu_baseline": {"value": v, "unit": "ms", "cores": 1, "kind": "oracle",
                             "host_cpus": os.cpu_count(), "sample": sample},
            "e2e": {"value": v, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": time.perf_counter() - t0}


def run_gradcheck(args):
    """Adjoint design gradient of the robust objective (mean + std of the three realisations'
    compliances) against central differences on `args.gradcheck` seeded design variables of
    the 3200x4096 periodic workload.  Solves: MIXED to 1e-8 with the preconditioner of the
    unperturbed design re-used (Sec. 5.1).  The difference quotients use the variational
    compliance 2 f.u - u.K u (FP64 matvec), whose error is quadratic in the solve error."""
    import numpy as np
    import torch
    import workloads
    import paper_1411_3923_gb300 as m

    wl = workloads.make(args.gradcheck_workload)
    prob = m.Problem(wl.nelx, wl.nely, wl.fixed, nu=wl.nu, E0=wl.E0, Emin=wl.Emin,
                     penal=wl.penal, H=wl.H, n_eig=wl.n_eig, precision="mixed", tol=1e-8,
                     reuse_preconditioner=True)
    f = torch.from_numpy(np.ascontiguousarray(wl.force)).cuda()
    kappa, h = 1.0, 1e-3

    def robust(rho, build=False):
        prob.set_design(torch.from_numpy(np.ascontiguousarray(rho)).cuda(), wl.rmin, wl.beta,
                        wl.etas, wl.cell)
        if build:
            prob.build_preconditioner()
        u, infos = prob.solve(f, -1)
        cs = []
        for k in range(len(wl.etas)):
            uk = u[k].reshape(-1)
            Ku = prob.apply_K(u[k], k, m.FP64).reshape(-1)
            cs.append(float(2.0 * torch.dot(f.reshape(-1), uk) - torch.dot(uk, Ku)))
        cs = np.array(cs)
        return cs.mean() + kappa * cs.std(), [i["iterations"] for i in infos]

    t0 = time.time()
    f0, it0 = robust(wl.rho, build=True)
    c, fr, g = prob.compliance_and_sensitivity(kappa)
    g = g.cpu().numpy().reshape(-1)
    idx = np.random.default_rng(20).choice(g.size, args.gradcheck, replace=False)
    rows, worst = [], 0.0
    for j in idx:
        rp = wl.rho.reshape(-1).copy(); rp[j] += h
        rm = wl.rho.reshape(-1).copy(); rm[j] -= h
        fp, _ = robust(rp.reshape(wl.rho.shape))
        fm, _ = robust(rm.reshape(wl.rho.shape))
        fd = (fp - fm) / (2 * h)
        err = abs(fd - g[j]) / max(abs(g[j]), 1e-3 * np.abs(g).max())
        worst = max(worst, err)
        rows.append({"index": int(j), "adjoint": float(g[j]), "central_difference": float(fd),
                     "rel_err": float(err)})
    print(json.dumps({"gradcheck": args.gradcheck_workload, "dofs": prob.n_dof,
                      "objective": f0, "objective_library": fr, "iterations": it0,
                      "h": h, "variables": len(idx), "max_rel_err": worst, "tolerance": 1e-5,
                      "pass": bool(worst <= 1e-5), "seconds": round(time.time() - t0, 1),
                      "entries": rows}))


def run_workload(args):
    """The whole path on one named workload (no L2 flush, wall and event times): design chain,
    preconditioner build, MIXED solve of all realisations (and FP64 unless --workload-mixed-only),
    robust compliance and design gradient.  'cantilever_batch' runs the 64-instance uneven
    batch through the batch entry points (and, beside it, the instances one after another)."""
    import numpy as np
    import torch
    import workloads
    import paper_1411_3923_gb300 as m

    name = args.workload_run
    out = {"workload_run": name}
    if name == "cantilever_batch":
        wls = workloads.cantilever_batch()
        probs = []
        for wl in wls:
            p = m.Problem(wl.nelx, wl.nely, wl.fixed, nu=wl.nu, E0=wl.E0, Emin=wl.Emin,
                          penal=wl.penal, H=wl.H, n_eig=wl.n_eig, precision="mixed", tol=1e-8)
            p.set_design(torch.from_numpy(np.ascontiguousarray(wl.rho)).cuda(), wl.rmin, wl.beta,
                         wl.etas, wl.cell)
            probs.append(p)
        dofs = sum(p.n_dof for p in probs)
        torch.cuda.synchronize()
        t = time.time()
        binfo = m.batch_build_preconditioner(probs)
        torch.cuda.synchronize()
        tb = time.time() - t
        fs = [torch.from_numpy(np.ascontiguousarray(wl.force)).cuda() for wl in wls]
        m.batch_solve(probs, fs)   # warm-up (graph capture)
        torch.cuda.synchronize()
        t = time.time()
        us, infos = m.batch_solve(probs, fs)
        torch.cuda.synchronize()
        ts = time.time() - t
        t = time.time()
        for p, f in zip(probs, fs):
            p.solve(f, -1)
        torch.cuda.synchronize()
        tq = time.time() - t
        its = [i[0]["iterations"] for i in infos]
        one_graph = all(p.stats()["batch_graph_solves"] >= 2 for p in probs)
        out.update({"instances": len(probs), "dofs": dofs, "build_s": tb,
                    "batch_one_graph_launch": one_graph,
                    "coarse_solvers": sorted(set(b["coarse_solver"] for b in binfo)),
                    "batch_solve_s": ts, "batch_mdof_per_s": dofs / ts / 1e6,
                    "sequential_solve_s": tq, "iterations_min_mean_max": [min(its), float(np.mean(its)), max(its)],
                    "max_rel_residual": max(i[0]["rel_residual"] for i in infos),
                    "all_converged": all(i[0]["status"] == 0 for i in infos)})
        print(json.dumps(out))
        return
    wl = workloads.make(name)
    f = torch.from_numpy(np.ascontiguousarray(wl.force)).cuda()
    rho = torch.from_numpy(np.ascontiguousarray(wl.rho)).cuda()
    out.update({"mesh": [wl.nelx, wl.nely], "dofs": 2 * (wl.nelx + 1) * (wl.nely + 1),
                "realisations": len(wl.etas), "preconditioner": args.preconditioner,
                "krylov": args.krylov,
                "patch_kernel": args.patch_kernel})
    precisions = ["mixed"] if args.workload_mixed_only else ["mixed", "fp64"]
    for prec in precisions:
        prob = m.Problem(wl.nelx, wl.nely, wl.fixed, nu=wl.nu, E0=wl.E0, Emin=wl.Emin,
                         penal=wl.penal, H=wl.H, n_eig=wl.n_eig, precision=prec, tol=1e-8,
                         preconditioner=args.preconditioner, max_iter=args.max_iter,
                         patch_kernel=args.patch_kernel, krylov=args.krylov)
        torch.cuda.synchronize()
        t0 = time.time()
        prob.set_design(rho, wl.rmin, wl.beta, wl.etas, wl.cell)
        info = prob.build_preconditioner()
        torch.cuda.synchronize()
        t1 = time.time()
        prob.solve(f, -1, check=False)            # warm-up (graph capture)
        torch.cuda.synchronize()
        t2 = time.time()
        u, infos = prob.solve(f, -1, check=False)
        torch.cuda.synchronize()
        t3 = time.time()
        try:
            c, fr, g = prob.compliance_and_sensitivity(1.0)
        except m.MstopoError:   # a system did not converge: no compliance to report
            fr = None
        torch.cuda.synchronize()
        t4 = time.time()
        # one more solve with per-kernel events (graphs off): where the solve's time goes
        prob.set_profiling(True)
        _, infos_p = prob.solve(f, -1, check=False)
        st = prob.stats()
        prob.set_profiling(False)
        out[prec] = {"build_s": t1 - t0, "build": {k: info[k] for k in ("n_agglomerates", "n_types", "n_coarse",
                                                                        "coarse_solver", "ms_eigen", "ms_patch_factor",
                                                                        "ms_coarse", "ms_total")},
                     "solve_s": t3 - t2, "solve_event_ms": infos[0]["ms"],
                     "iterations": [i["iterations"] for i in infos],
                     "status": [i["status"] for i in infos],
                     "rel_residual": [i["rel_residual"] for i in infos],
                     "compliance": [i["compliance"] for i in infos], "f_robust": fr,
                     "sensitivity_s": t4 - t3,
                     "profiled_solve": {"event_ms": infos_p[0]["ms"],
                                        "kernels_ms": {k: v["ms"] for k, v in st.items()
                                                       if isinstance(v, dict) and "ms" in v},
                                        "launches": {k: v["launches"] for k, v in st.items()
                                                     if isinstance(v, dict) and "launches" in v}}}
        prob.close()
        del prob
        torch.cuda.empty_cache()
    if "fp64" in out:
        out["speedup_mixed_vs_fp64"] = out["fp64"]["solve_s"] / out["mixed"]["solve_s"]
    print(json.dumps(out))


def run_only(args):
    """One kernel in a short loop: 'patch' = FP32 patch solves of a workload's preconditioner
    (apply_precond, MIXED, patches only, realisation 0; default the 1024x512 workload);
    'solve' = whole MIXED solves of a workload (default the 1024x512 workload);
    'matvec' = FP32 matvec as the flexible CG launches it (all realisations, default the
    3200x4096 mesh, 26.2M DOFs x 3).  --only-workload and
    --only-scale pick another workload or a reduced copy of it."""
    import torch
    import paper_1411_3923_gb300 as m
    import workloads
    dev = torch.device("cuda", 0)
    name = args.only_workload or (WORKLOAD if args.only in ("patch", "solve") else "mbb_c5")
    wl = workloads.make(name, args.only_scale)
    prob = m.Problem(wl.nelx, wl.nely, wl.fixed, nu=wl.nu, E0=wl.E0, Emin=wl.Emin,
                     penal=wl.penal, H=wl.H, n_eig=wl.n_eig, precision="mixed",
                     patch_kernel=args.patch_kernel)
    prob.set_design(torch.from_numpy(wl.rho).to(dev), wl.rmin, wl.beta, wl.etas, wl.cell)
    if args.only == "patch":
        prob.build_preconditioner(-1)
        r = torch.randn((wl.nely + 1, wl.nelx + 1, 2), dtype=torch.float64, device=dev)
        for _ in range(args.reps):
            prob.apply_precond(r, m.MIXED, 2)
    elif args.only == "solve":   # whole MIXED solves of the workload (after one build)
        prob.build_preconditioner(-1)
        f = torch.from_numpy(wl.force).to(dev)
        for _ in range(args.reps):
            prob.solve(f, -1)
    else:   # the flexible CG's launch: every realisation, inputs zero at Dirichlet DOFs
        import numpy as np
        free = torch.from_numpy(~np.asarray(wl.fixed, dtype=bool).reshape(-1)).to(dev)
        u = torch.randn(len(wl.etas), prob.n_dof, device=dev, dtype=torch.float32) * free
        y = torch.empty_like(u)
        for _ in range(args.reps):
            prob.apply_K_f32(u, -1, y, input_masked=True)
    torch.cuda.synchronize()
    print(json.dumps({"only": args.only, "workload": name, "scale": args.only_scale,
                      "mesh": [wl.nelx, wl.nely], "reps": args.reps, "ok": True}))


def run_design_loop(args):
    """The design loop on the device (robust compliance, expected-volume constraint, MMA,
    continuation: Sec. 4.4, 4.5) on a workload's mesh and realisations, from a uniform start
    design at the volume fraction: two stages (penal 3; beta 1 then the workload's beta) of
    --design-iters iterations each; then the robust verification of the result over 9
    thresholds in [0.3, 0.7].  Reports the time per design iteration (set_design, build,
    solve of every realisation, objective, gradient, volume, MMA step) and the history."""
    import numpy as np
    import torch
    import paper_1411_3923_gb300 as m
    import workloads
    wl = workloads.make(args.design_loop)
    shape = (wl.cell[1], wl.cell[0]) if wl.cell else (wl.nely, wl.nelx)
    vf = 0.5
    rho0 = torch.full(shape, vf, dtype=torch.float64, device="cuda")
    f = torch.from_numpy(np.ascontiguousarray(wl.force)).cuda()
    prob = m.Problem(wl.nelx, wl.nely, wl.fixed, nu=wl.nu, E0=wl.E0, Emin=wl.Emin,
                     penal=wl.penal, H=wl.H, n_eig=wl.n_eig, precision="mixed", tol=1e-8,
                     max_iter=5000)
    prob.set_design(rho0, wl.rmin, wl.beta, wl.etas, wl.cell)
    stages = [(3.0, 1.0, args.design_iters), (3.0, float(wl.beta), args.design_iters)]
    torch.cuda.synchronize()
    t0 = time.time()
    rho, hist = prob.optimise(rho0, f, stages, vf, kappa=1.0, rel_change=1e-4)
    torch.cuda.synchronize()
    t1 = time.time()
    etas = np.linspace(0.3, 0.7, 9)
    prob.set_design(rho, wl.rmin, wl.beta, wl.etas, wl.cell)
    c = prob.robust_verification(rho, f, etas)
    torch.cuda.synchronize()
    t2 = time.time()
    print(json.dumps({"design_loop": args.design_loop, "mesh": [wl.nelx, wl.nely],
                      "design_vars": int(rho.numel()), "realisations": len(wl.etas),
                      "iterations": len(hist), "s_per_iteration": (t1 - t0) / max(1, len(hist)),
                      "total_s": t1 - t0, "verification_s": t2 - t1,
                      "f_first_last": [hist[0]["f"], hist[-1]["f"]],
                      "g_last": hist[-1]["g"], "solve_iterations": [h["solve_iterations"] for h in hist],
                      "verification_etas": etas.tolist(), "verification_c": c.tolist()}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--ref-iterations", type=int, default=4,
                    help="PCG iterations per timed step of the reference arm")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-big-matvec", action="store_true")
    ap.add_argument("--only", choices=["patch", "matvec", "solve"], default=None,
                    help="run one kernel in a short loop (for ncu captures) and exit")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--only-workload", default=None)
    ap.add_argument("--only-scale", type=int, default=1)
    ap.add_argument("--gradcheck", type=int, default=0,
                    help="check the adjoint gradient against central differences on this many "
                         "seeded design variables (no benchmark)")
    ap.add_argument("--gradcheck-workload", default="mbb_c5")
    ap.add_argument("--workload-run", default=None,
                    help="run the whole path on a named workload (mbb_c1, mbb_c2, mbb_c3, mbb_c5, "
                         "cantilever_batch) and print one JSON line (no benchmark)")
    ap.add_argument("--workload-mixed-only", action="store_true")
    ap.add_argument("--max-iter", type=int, default=5000, help="--workload-run: iteration cap")
    ap.add_argument("--no-autotune", action="store_true",
                    help="choose the FP32 patch-solve configuration by the cost model instead of timing")
    ap.add_argument("--patch-kernel", default="auto", choices=["auto", "cuda_cores", "tensor_cores"],
                    help="with --workload-run: the FP32 patch-solve kernel")
    ap.add_argument("--design-loop", default=None,
                    help="run the device design loop (MMA, continuation) on this workload")
    ap.add_argument("--design-iters", type=int, default=10)
    ap.add_argument("--krylov", default="fcg", choices=["fcg", "gmres"],
                    help="with --workload-run: the outer Krylov method")
    ap.add_argument("--preconditioner", default="additive", choices=["additive", "sgs"],
                    help="with --workload-run: the additive two-level Schwarz preconditioner, or "
                         "the paper's multiplicative one (SGS, coarse correction, SGS)")
    args = ap.parse_args()
    if args.only:
        run_only(args)
        return
    if args.gradcheck:
        run_gradcheck(args)
        return
    if args.workload_run:
        run_workload(args)
        return
    if args.design_loop:
        run_design_loop(args)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    else:
        if world > 1:
            import torch
            torch.distributed.init_process_group("nccl")
        out = run_ours(args, rank, world)
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()
    if out is not None:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
