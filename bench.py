#!/usr/bin/env python3
"""Time-step benchmark of the repartitioning hot path on GB300.

One step = one simulated time step of the paper's pressure solve (Sec. 3-4):
a new coefficient draw is pushed through ``rp_update_values_packed`` (the
permutation update of the continuous buffer) and the merged system is solved
with ``rp_solve`` to relative residual 1e-9 from x = 0. The default workload
is 256^3 cells decomposed into k = 128 CPU ranks (8x4x4) merged into one CSR
matrix, lognormal(0, 1) face coefficients, rhs U[-1, 1] seed 0.

Both precisions are timed (FP64 Jacobi-PCG and FP32-inner / FP64-outer
refinement); ``--precision`` picks the headline ``value``. Inputs are
resident in HBM when the timed region starts and are larger than L2
(0.94 GB coefficient buffer, 1.4 GB matrix), so no L2 flush is needed.

``--impl reference`` times the CPU oracle instead (its C / OpenMP
restatement on every host core, full time steps of the same workload, each
timed end to end): the paper ships no code, so the oracle is the reference
arm. ``cpu_baseline`` in the GPU line reports the same oracle on all cores
and on one, and on the 32^3 and 128^3 configurations.

Multi-GPU (torchrun): the path does not shard; every rank runs an
independent replica of the workload (weak scaling): ``value`` is the slowest
replica's ms per time step, the whole job's time steps per second are
reported beside it.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "update+PCG ms/time-step at 256^3 cells, FP64 vs mixed; SpMV HBM GB/s vs peak"
# DRAM bytes per launch from ncu captures of the same kernels on the 192^3 case, scaled to
# a 256^3 launch by the ratio of algorithmic bytes (one pass per array): sliced FP32 SpMV
# (uniform-slice instance, evict-first copies) 261.5 MB of 285.2 MB algorithmic -- the
# q writes now stay in L2 --, sliced FP64 507.1 MB of 539.4 MB, CSR FP32 477.4 MB of
# 479.5 MB. Remove an entry when its kernel changes, until it is captured again.
PROFILED_TRAFFIC = {("mixed_256", "k_it_spmv_sl<float, true>"): 620.1e6,
                    ("mixed_256", "k_it_spmv_sl<double, true>"): 1202.6e6,
                    ("mixed_256", "k_it_spmv<float>"): 1132.7e6}
# FP64 FMA issue rate of a GB300 SM (2 per clock; 152 SMs x 2 x 2 flop x 2.07 GHz =
# 1.26 TFLOP/s, the nominal 1.25): the FP64 path is bound by it, not by HBM.
FP64_FMA_PER_SM_CLK = 2
MAX_SM_MHZ = 2070.0  # GB300 maximum SM clock (the sampled clocks.max.sm where available)


def fp64_peak_tflops(dev, sm_mhz):
    """Derived FP64 peak: SMs x FP64 FMA per SM clock x 2 flop x SM clock."""
    import torch
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    return sms * FP64_FMA_PER_SM_CLK * 2 * sm_mhz * 1e6 / 1e12
WORKLOAD_TEXT = {
    "mixed_256": "256^3 cells (16,777,216), k=128 CPU ranks (8x4x4) merged into 1 CSR, lognormal(0,1.0) face "
                 "coefficients redrawn every step, rhs U[-1,1] seed 0, rel. residual 1e-9 from x=0, inner tol 1e-5",
    "update_128": "128^3 cells (2,097,152), k=64 CPU ranks (4x4x4) merged into 1 CSR, lognormal(0,0.5) face "
                  "coefficients redrawn every step, rhs U[-1,1] seed 0, rel. residual 1e-9 from x=0",
    "plain_fp64_32": "32^3 cells, k=8 ranks (2x2x2), uniform a_f=1, rhs U[-1,1] seed 0, rel. residual 1e-9",
    "adjoint_128": "128^3 cells, k=64 ranks (4x4x4), lognormal(0,0.5) faces, rhs U[-1,1] seed 0, rel. residual 1e-9",
    "profile_192": "192^3 cells, k=27 ranks (3x3x3), lognormal(0,1.0) faces (profiling size, larger than L2)",
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="mixed_256", choices=sorted(WORKLOAD_TEXT))
    ap.add_argument("--precision", default="mixed_ru", choices=["mixed_ru", "mixed", "fp64"])
    ap.add_argument("--draws", type=int, default=4, help="distinct coefficient draws, cycled over the steps")
    ap.add_argument("--only", default=None, choices=["mixed_ru", "mixed", "fp64"],
                    help="time one precision only (profiling runs)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-form measurement")
    ap.add_argument("--no-small", action="store_true", help="skip the 32^3 and 128^3 configurations")
    ap.add_argument("--only-bicgstab", action="store_true",
                    help="run only the momentum (BiCGStab) measurement, FP64 and mixed: profiling runs")
    ap.add_argument("--only-batch", action="store_true",
                    help="run only the batched form (default launch shape, no loop baseline): profiling runs")
    ap.add_argument("--batch-systems", type=int, default=256)
    ap.add_argument("--batch-shape", default=None,
                    help="CLUSTERxTHREADS launch shape of the batched kernel instead of the autotuner's choice")
    ap.add_argument("--no-bicgstab", action="store_true",
                    help="skip the non-symmetric (momentum) solve and the adjoint measurement")
    ap.add_argument("--no-line", action="store_true", help="skip the line-preconditioner measurement")
    ap.add_argument("--alpha-sweep", action="store_true",
                    help="repartitioning-ratio study at 128^3: GPU parts and CPU ranks merged")
    ap.add_argument("--host-loop", action="store_true",
                    help="launch the solve kernels from the host (for profilers; not a timing mode)")
    ap.add_argument("--oracle-leg", default=None, help=argparse.SUPPRESS)
    return ap.parse_args()


# ---------------------------------------------------------------- helpers


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.proc = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(gpu_id), "-lms", "200"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def make_inputs(workload, draws, symmetric=False):
    import numpy as np

    from paper_2510_08536_gb300 import synth
    w = synth.WORKLOADS[workload]
    mesh = synth.workload_mesh(workload)
    asm = synth.Assembler(mesh, symmetric)
    stg = [asm.staging(synth.face_coeffs(mesh, w["sigma"], 100 + t)) for t in range(draws)]
    b = synth.uniform_vector(mesh, 0)
    return mesh, asm, stg, np.ascontiguousarray(b)


# ---------------------------------------------------------------- oracle leg


def oracle_leg(spec):
    """Time the CPU oracle (runs in a child process, no GPU): its C / OpenMP
    restatement of the value update and FP64 Jacobi-PCG (pinned against the
    Python oracle), on the merged map of the Python oracle.

    spec = {"workload", "seeds", "threads", "mode", "iters", "warmup"}. Per
    seed, one time step: value update vals = buf[src_of], Jacobi diagonal and
    PCG to relative residual 1e-9 from x = 0, timed end to end ("full"); or
    the update plus ``iters`` PCG iterations, scaled to the oracle's iteration
    count for that system ("sample", labelled extrapolated). The coefficient
    buffers are drawn before the timing; ``warmup`` untimed update-only steps
    come first."""
    import numpy as np

    from oracle import pcg_omp as C
    from oracle import repart_oracle as O
    from paper_2510_08536_gb300 import synth
    t0 = time.perf_counter()
    w = synth.WORKLOADS[spec["workload"]]
    mesh = synth.workload_mesh(spec["workload"])
    asm = synth.Assembler(mesh)
    (m,) = O.repartition_map(mesh.ranks, 1)
    b = synth.uniform_vector(mesh, 0)
    seeds = spec["seeds"]
    bufs = {s: asm.staging(synth.face_coeffs(mesh, w["sigma"], s)) for s in sorted(set(seeds))}
    th = int(spec.get("threads", 0))
    setup_s = time.perf_counter() - t0
    for k in range(int(spec.get("warmup", 0))):
        C.update_values(m.src_of, bufs[seeds[k % len(seeds)]], threads=th)
    steps = []
    for s in seeds:
        ta = time.perf_counter()
        vals = C.update_values(m.src_of, bufs[s], threads=th)
        dinv = C.jacobi_inverse(m.diag_pos, vals, threads=th)
        tb = time.perf_counter()
        if spec["mode"] == "full":
            r = C.pcg(m.row_ptr, m.col_idx, vals, dinv, b, tol=1e-9, threads=th)
            tc = time.perf_counter()
            steps.append({"ms": 1e3 * (tc - ta), "update_ms": 1e3 * (tb - ta), "pcg_ms": 1e3 * (tc - tb),
                          "iterations": r.iterations, "status": r.status, "true_rel_residual": r.true_rel_residual})
        else:
            iters, count = int(spec["iters"]), int(spec["count"])
            C.pcg(m.row_ptr, m.col_idx, vals, dinv, b, tol=0.0, max_iter=iters, threads=th)
            tc = time.perf_counter()
            it_ms = 1e3 * (tc - tb) / iters
            steps.append({"ms": 1e3 * (tb - ta) + count * it_ms, "update_ms": 1e3 * (tb - ta), "iter_ms": it_ms,
                          "iterations_timed": iters, "iterations_scaled_to": count})
        del vals, dinv
    return {"workload": spec["workload"], "threads": C.threads(th), "mode": spec["mode"],
            "setup_s": round(setup_s, 1), "steps": steps}


def run_oracle_subprocess(spec, timeout=1800):
    """oracle_leg in a child process without a GPU, on the cores this process may use."""
    env = dict(os.environ)
    env["CUDA_VISIBLE_DEVICES"] = ""
    env["OMP_NUM_THREADS"] = str(len(os.sched_getaffinity(0)))
    env.pop("OMP_PROC_BIND", None)
    p = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-leg", json.dumps(spec)], env=env,
                       capture_output=True, text=True, timeout=timeout)
    if p.returncode:
        raise RuntimeError("oracle leg failed: " + p.stderr[-2000:])
    return json.loads(p.stdout.strip().splitlines()[-1])


def cpu_baseline(args, fp64_iterations):
    """The oracle on the host cores, same workload and tolerance as the GPU line:
    one full 256^3 time step on every core (measured), the 1-core figure from a
    bounded sample (extrapolated, labelled), and full time steps of the 32^3 and
    128^3 configurations on every core and on one."""
    cores = len(os.sched_getaffinity(0))
    legs = []
    full = run_oracle_subprocess({"workload": args.workload, "seeds": [100], "threads": cores, "mode": "full",
                                  "warmup": 1})
    st = full["steps"][0]
    legs.append({"workload": args.workload, "cores": full["threads"], "kind": "oracle", "measured": True,
                 "ms": round(st["ms"], 1), "update_ms": round(st["update_ms"], 1), "pcg_ms": round(st["pcg_ms"], 1),
                 "iterations": st["iterations"], "true_rel_residual": st["true_rel_residual"]})
    one = run_oracle_subprocess({"workload": args.workload, "seeds": [100], "threads": 1, "mode": "sample",
                                 "iters": 20, "count": st["iterations"]})
    s1 = one["steps"][0]
    legs.append({"workload": args.workload, "cores": 1, "kind": "oracle, extrapolated", "measured": False,
                 "ms": round(s1["ms"], 1), "update_ms": round(s1["update_ms"], 1), "iter_ms": round(s1["iter_ms"], 2),
                 "sample": f"value update + 20 PCG iterations on one core, per-iteration time scaled to the "
                           f"{st['iterations']} iterations of the measured all-core step"})
    for wl in ("plain_fp64_32", "update_128"):
        for th in (cores, 1):
            r = run_oracle_subprocess({"workload": wl, "seeds": [100], "threads": th, "mode": "full", "warmup": 1})
            q = r["steps"][0]
            legs.append({"workload": wl, "cores": r["threads"], "kind": "oracle", "measured": True,
                         "ms": round(q["ms"], 2), "iterations": q["iterations"]})
    return {"value": legs[0]["ms"], "unit": "ms/time-step", "cores": legs[0]["cores"], "kind": "oracle",
            "sample": f"one full time step of the workload (draw seed 100): value update, Jacobi diagonal and FP64 "
                      f"Jacobi-PCG to 1e-9 from x = 0, by the oracle's C / OpenMP restatement on all {cores} host "
                      f"cores, timed end to end (measured, not scaled)",
            "legs": legs, "gpu_fp64_iterations": fp64_iterations}


# ---------------------------------------------------------------- adjoint (gradients)


def run_adjoint(dev, reps=3):
    """128^3, k = 64: forward FP64 solve, adjoint solve A^T lambda = x - x_t, entry and
    face gradients (all faces), each timed with CUDA events (mean of reps)."""
    import torch

    from paper_2510_08536_gb300 import repart, synth
    mesh = synth.workload_mesh("adjoint_128")
    stg = torch.from_numpy(synth.Assembler(mesh).staging(synth.face_coeffs(mesh, 0.5, 100))).to(dev)
    b = torch.from_numpy(synth.uniform_vector(mesh, 0)).to(dev)
    xt = torch.from_numpy(synth.uniform_vector(mesh, 1)).to(dev)
    t0 = time.perf_counter()
    h = repart.build_repartition(mesh.ranks, want_transpose=True, want_fp32=False)
    build_ms = 1e3 * (time.perf_counter() - t0)
    n, nf = mesh.n_cells, sum(r.n_faces + r.n_iface for r in mesh.ranks)
    x = torch.zeros(n, dtype=torch.float64, device=dev)
    lam = torch.zeros_like(x)
    gbuf = torch.zeros(h.n_slots, dtype=torch.float64, device=dev)
    gface = torch.zeros(nf, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    out = {}

    def timed(name, fn):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = [fn() for _ in range(reps)]
        e1.record(stream)
        torch.cuda.synchronize()
        out[name + "_ms"] = round(e0.elapsed_time(e1) / reps, 3)
        return res[-1]

    timed("update", lambda: repart.update_values_packed(h, stg))
    info = timed("forward_solve", lambda: repart.solve(h, b, x, tol=1e-9))
    g = x - xt
    ainfo = timed("adjoint_solve", lambda: repart.solve_adjoint(h, g, lam, tol=1e-9))
    timed("entry_grad", lambda: repart.entry_grad(h, lam, x, gbuf))
    timed("face_grad", lambda: repart.face_grad(h, lam, x, gface))
    h.close()
    out.update({"workload": "adjoint_128: 128^3 cells, k=64 (4x4x4), lognormal(0,0.5) faces, rhs U[-1,1] seed 0, "
                            "x_target U[-1,1] seed 1, FP64, rel. residual 1e-9",
                "map_build_with_transpose_ms": round(build_ms, 1), "faces": nf,
                "forward_iterations": info["iterations"], "adjoint_iterations": ainfo["iterations"],
                "statuses": [info["status"], ainfo["status"]]})
    return out


# ---------------------------------------------------------------- momentum (BiCGStab)


def run_bicgstab(dev, steps, warmup, draws=2, host_loop=False, precs=("fp64", "mixed")):
    """Non-symmetric momentum system on the headline mesh (256^3, k = 128): per step a
    value update (new coefficient draw) + a BiCGStab solve to 1e-9 from x = 0, in FP64
    (rp_solve_bicgstab) and as FP32-inner / FP64-outer refinement (rp_solve_bicgstab_mixed)."""
    import torch

    from paper_2510_08536_gb300 import repart, synth
    t0 = time.time()
    mesh = synth.workload_mesh("momentum_256")
    stg = [torch.from_numpy(synth.momentum_staging(mesh, 0.5, 100 + t)).to(dev) for t in range(draws)]
    b = torch.from_numpy(synth.uniform_vector(mesh, 0)).to(dev)
    x = torch.zeros(mesh.n_cells, dtype=torch.float64, device=dev)
    setup_s = time.time() - t0
    h = repart.build_repartition(mesh.ranks, host_loop=int(host_loop))
    n, sliced = mesh.n_cells, repart.sliced_sizes(h)
    entries = sliced[1] if sliced else h.nnz
    stream = torch.cuda.current_stream()
    runs = {}
    for prec in precs:
        for t in range(warmup):
            repart.update_values_packed(h, stg[t % draws])
            repart.solve_bicgstab(h, b, x, tol=1e-9, precision=prec)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        infos = []
        e0.record(stream)
        for t in range(steps):
            repart.update_values_packed(h, stg[(warmup + t) % draws])
            infos.append(repart.solve_bicgstab(h, b, x, tol=1e-9, precision=prec))
        e1.record(stream)
        torch.cuda.synchronize()
        runs[prec] = (e0.elapsed_time(e1) / steps, infos)
    h.close()
    if "fp64" not in runs:  # a profiling run of the mixed form alone
        mms, minfos = runs["mixed"]
        return {"mixed": {"ms_per_step": round(mms, 3),
                          "inner_iterations_mean": statistics.mean(i["iterations"] for i in minfos),
                          "statuses": sorted({i["status"] for i in minfos})}}
    ms, infos = runs["fp64"]
    it = statistics.mean(i["iterations"] for i in infos)
    # per iteration: two products (one FMA per stored entry + the fused dots) and
    # ~14 FP64 instructions per row in the three vector kernels
    ops = it * (2 * entries + 14 * n)
    peak = fp64_peak_tflops(dev, MAX_SM_MHZ)
    ach = 2 * ops / (ms * 1e-3) / 1e12
    mms, minfos = runs.get("mixed", (float("nan"), [{"iterations": 0, "outer_iterations": 0, "status": -1,
                                                     "rel_residual": float("nan")}]))
    return {"workload": "momentum_256: 256^3 cells, k=128 (8x4x4) merged, upwind convection-diffusion "
                        "(lognormal(0,0.5) diffusion, cavity-vortex flux, ct=0.1), rhs U[-1,1] seed 0, "
                        "rel. residual 1e-9 from x=0, FP64",
            "ms_per_step": round(ms, 3), "iterations_mean": it, "steps": steps,
            "statuses": sorted({i["status"] for i in infos}),
            "max_rel_residual": max(i["rel_residual"] for i in infos), "input_setup_s": round(setup_s, 1),
            "fp64_alu": {"bound": "alu", "unit": "TFLOP/s", "achieved": round(ach, 4), "peak": round(peak, 4),
                         "frac": round(ach / peak, 4)},
            "mixed": {"ms_per_step": round(mms, 3),
                      "inner_iterations_mean": statistics.mean(i["iterations"] for i in minfos),
                      "refinements_mean": statistics.mean(i["outer_iterations"] for i in minfos),
                      "statuses": sorted({i["status"] for i in minfos}),
                      "max_rel_residual": max(i["rel_residual"] for i in minfos)}}


# ---------------------------------------------------------------- batched form


def run_batch(args, dev, steps, warmup, loop_steps=1):
    """256 uneven independent systems (8k-300k cells, aspect 1-4, lognormal(0, 0.5)):
    update + solve of all of them in one persistent launch per step, FP64 and mixed,
    launch shape autotuned; compared with a loop of single-system rp_solve calls."""
    import numpy as np
    import torch

    from paper_2510_08536_gb300 import repart, synth
    t0 = time.time()
    B = synth.Batch(args.batch_systems, 8000, 300000, seed=0)
    draws = 2
    stg = [torch.from_numpy(B.staging(0.5, 100 + t)).to(dev) for t in range(draws)]
    b = torch.from_numpy(B.rhs(0)).to(dev)
    x = torch.zeros(B.n_rows, dtype=torch.float64, device=dev)
    setup_s = time.time() - t0
    h = repart.batch_build(B.systems)
    out = {"workload": f"{len(B.systems)} independent box systems, cells log-uniform in [8k, 300k], aspect "
                       "ratios U[1,4], lognormal(0,0.5) faces, Dirichlet at x=0, rhs U[-1,1], rel. residual 1e-9 "
                       "from x=0",
           "systems": len(B.systems), "rows": B.n_rows, "nnz": h.nnz, "input_setup_s": round(setup_s, 1)}
    sizes = [(m.n_cells, m.nnz()) for m in B.meshes]
    # per system (padded entries E, index words I, slices S) of the sliced layout, when built
    view = repart.get_sliced_view(h)
    sl_sizes = None
    if view is not None:
        d = view["desc"].cpu().numpy().view(np.uint32).reshape(-1, 2).astype(np.int64)
        so = np.cumsum([0] + [(m.n_cells + 31) // 32 for m in B.meshes])
        sl_sizes = [(int(d[so[i + 1], 0] - d[so[i], 0]), int(d[so[i + 1], 1] - d[so[i], 1]), int(so[i + 1] - so[i]))
                    for i in range(len(B.meshes))]
        del view
    out["layout"] = "sliced" if sl_sizes else "csr"
    hbm_peak, _ = load_peaks()
    if args.batch_shape:
        c, t = (int(v) for v in args.batch_shape.lower().split("x"))
        repart.batch_set_config(h, c, t)
        out["shape"] = {"cluster": c, "threads": t}
    elif not args.only_batch:
        c, t, ms = repart.batch_autotune(h, stg[0], b, x, tol=1e-9, precision="fp64")
        out["autotuned"] = {"cluster": c, "threads": t, "tuning_ms": round(ms, 2)}
    stream = torch.cuda.current_stream()
    for prec in ([args.only] if args.only else ("fp64", "mixed", "mixed_ru")):
        for i in range(warmup):
            repart.batch_update_solve(h, stg[i % draws], b, x, 1e-9, prec)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        infos_all = []
        e0.record(stream)
        for i in range(steps):
            infos_all.append(repart.batch_update_solve(h, stg[(warmup + i) % draws], b, x, 1e-9, prec))
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        bad = sum(1 for infos in infos_all for i in infos if i["status"] != 0)
        iters = [sum(i["iterations"] for i in infos) for infos in infos_all]
        # algorithmic bytes of one step: update (24 B/entry + 20 B/row, plus the sliced
        # values: position, source index, buffer value, FP64 (and FP32) value per padded
        # entry), every iteration (FP64: SpMV + 80 B/row; FP32: SpMV + 40 B/row, 32 on the
        # scaled system S A S that the mixed forms run on the sliced layout: no diagonal
        # reads; its FP32 values add a column and s_j per padded entry and s per row to the
        # update), every FP64 residual pass; SpMV on CSR: values, columns, row pointers, x,
        # y; sliced: padded values, index words, descriptors and table references, x, y
        w = 8 if prec == "fp64" else 4
        scaled_b = prec != "fp64" and sl_sizes is not None
        moved = 0.0
        for infos in infos_all:
            for s, inf in enumerate(infos):
                nn, nz = sizes[s]
                if sl_sizes:
                    E, I, S = sl_sizes[s]
                    spmv = w * E + 4 * I + 12 * S + 2 * w * nn
                    res = 8 * E + 4 * I + 12 * S + 40 * nn
                    upd = 24 * nz + 20 * nn + (24 + (w == 4) * 4) * E + (12 * E + 8 * nn if scaled_b else 0)
                else:
                    spmv = (w + 4) * nz + 4 * (nn + 1) + 2 * w * nn
                    res = 12 * nz + 4 * (nn + 1) + 40 * nn
                    upd = 24 * nz + 20 * nn
                moved += upd + inf["iterations"] * (spmv + (8 if scaled_b else 10) * w * nn) + inf["passes"] * res
        gbps = moved / len(infos_all) / (ms * 1e-3) / 1e9
        out[prec] = {"ms_per_step": round(ms, 3), "not_converged_systems": bad,
                     "iterations_sum_mean": statistics.mean(iters),
                     "algorithmic_GBps": round(gbps, 1), "frac_of_hbm": round(gbps / hbm_peak, 4),
                     "max_rel_residual": max(i["rel_residual"] for infos in infos_all for i in infos)}
        if prec == "fp64":
            # FP64 instructions of one step: per iteration one FMA per entry + ~8 per row
            # (p.q, r update, r.z, r.r, z, x and p updates), per residual pass nz + 8 n
            ops = sum(inf["iterations"] * (nz + 8 * nn) + inf["passes"] * (nz + 8 * nn)
                      for infos in infos_all for inf, (nn, nz) in zip(infos, sizes)) / len(infos_all)
            peak = fp64_peak_tflops(dev, MAX_SM_MHZ)
            ach = 2 * ops / (ms * 1e-3) / 1e12
            out[prec]["fp64_alu"] = {"bound": "alu", "unit": "TFLOP/s", "achieved": round(ach, 4),
                                     "peak": round(peak, 4), "frac": round(ach / peak, 4),
                                     "fp64_instructions_per_step": int(ops)}
    h.close()
    if args.only_batch:
        return out
    # baseline: one handle per system, rp_update_values_packed + rp_solve in a loop
    handles = [repart.build_repartition([s]) for s in B.systems]
    offs, so = [], 0
    for m in B.meshes:
        offs.append((so, so + m.staging_size()))
        so += m.staging_size()
    roffs, ro = [], 0
    for m in B.meshes:
        roffs.append((ro, ro + m.n_cells))
        ro += m.n_cells

    def loop_step(src):
        for hh, (a0, a1), (r0, r1) in zip(handles, offs, roffs):
            repart.update_values_packed(hh, src[a0:a1])
            repart.solve(hh, b[r0:r1], x[r0:r1], tol=1e-9, wait=False)

    loop_step(stg[0])
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(loop_steps):
        loop_step(stg[(1 + i) % draws])
    e1.record(stream)
    torch.cuda.synchronize()
    out["loop_of_single_solves_fp64_ms_per_step"] = round(e0.elapsed_time(e1) / loop_steps, 3)
    for hh in handles:
        hh.close()
    del stg
    torch.cuda.empty_cache()
    return out


# ---------------------------------------------------------------- configurations C0, C1


def reference_errors(workload, x):
    """Distance of a solution (device tensor, draw seed 100) to the oracle's, on the rows
    sampled in tests/golden/reference_solutions.json (written by a script that calls only
    the oracle): against its FP64 PCG at 1e-9 (the same recurrence) and at 1e-13."""
    import numpy as np
    p = os.path.join(ROOT, "tests", "golden", "reference_solutions.json")
    if not os.path.exists(p):
        return None
    g = json.load(open(p)).get(workload)
    if g is None or g["n"] != x.numel():
        return None
    import torch
    xs = x[torch.tensor(g["idx"], device=x.device)].cpu().numpy()
    xr, xe = np.asarray(g["x_ref"]), np.asarray(g["x_exact"])
    return {"vs_oracle_1e-9": float(np.linalg.norm(xs - xr) / np.linalg.norm(xr)),
            "vs_oracle_1e-13": float(np.linalg.norm(xs - xe) / np.linalg.norm(xe)),
            "oracle_1e-9_vs_1e-13": g["ref_vs_exact"], "rows_sampled": len(g["idx"])}


def run_small_configs(dev, steps=20):
    """C0: 32^3 / k = 8, uniform coefficients, FP64 PCG to 1e-9 (latency-bound, L2
    resident): us per time step. C1: 128^3 / k = 64, 20 time steps each with a new
    lognormal(0, 0.5) draw, update + FP64 PCG to 1e-9: map build, update, solve, SpMV
    GB/s; the mean over steps excludes the first (the paper's protocol). Errors
    against the oracle's solutions for draw seed 100."""
    import torch

    from paper_2510_08536_gb300 import repart, synth
    stream = torch.cuda.current_stream()
    hbm_peak, _ = load_peaks()
    out = {}
    for name, wl in (("C0", "plain_fp64_32"), ("C1", "update_128")):
        w = synth.WORKLOADS[wl]
        mesh = synth.workload_mesh(wl)
        asm = synth.Assembler(mesh)
        k = steps if w["sigma"] is not None else 1
        stg = [torch.from_numpy(asm.staging(synth.face_coeffs(mesh, w["sigma"], 100 + t))).to(dev) for t in range(k)]
        b = torch.from_numpy(synth.uniform_vector(mesh, 0)).to(dev)
        x = torch.zeros(mesh.n_cells, dtype=torch.float64, device=dev)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h = repart.build_repartition(mesh.ranks)
        build_ms = 1e3 * (time.perf_counter() - t0)
        n, nnz, sl = h.n, h.nnz, repart.sliced_sizes(h)
        for t in range(3):  # warm-up: graphs instantiated, clocks up
            repart.update_values_packed(h, stg[t % k])
            repart.solve(h, b, x, tol=1e-9)
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3 * steps)]
        infos = []
        for t in range(steps):
            ev[3 * t].record(stream)
            repart.update_values_packed(h, stg[t % k])
            ev[3 * t + 1].record(stream)
            infos.append(repart.solve(h, b, x, tol=1e-9))
            ev[3 * t + 2].record(stream)
            if t == 0:
                err = reference_errors(wl, x)
        torch.cuda.synchronize()
        upd = [ev[3 * t].elapsed_time(ev[3 * t + 1]) for t in range(1, steps)]
        sol = [ev[3 * t + 1].elapsed_time(ev[3 * t + 2]) for t in range(1, steps)]
        spmv_ms = repart.profile_iteration(h, b, "fp64", iters=20)["spmv"]
        if sl:
            spmv_bytes = 8 * sl[1] + 4 * sl[2] + 4 * sl[0] + 4 * sl[3] + 8 * (sl[0] + 1) + 16 * n
        else:
            spmv_bytes = 12 * nnz + 4 * (n + 1) + 16 * n
        r = {"workload": f"{wl}: {WORKLOAD_TEXT[wl]}", "steps": steps, "steps_averaged": steps - 1,
             "map_build_ms": round(build_ms, 2), "update_ms": round(statistics.mean(upd), 4),
             "solve_ms": round(statistics.mean(sol), 4),
             "ms_per_step": round(statistics.mean(u + v for u, v in zip(upd, sol)), 4),
             "iterations_mean": statistics.mean(i["iterations"] for i in infos[1:]),
             "statuses": sorted({i["status"] for i in infos}),
             "max_rel_residual": max(i["rel_residual"] for i in infos),
             "spmv_fp64_ms": round(spmv_ms, 5), "spmv_fp64_GBps": round(spmv_bytes / (spmv_ms * 1e-3) / 1e9, 1),
             "spmv_frac_of_hbm": round(spmv_bytes / (spmv_ms * 1e-3) / 1e9 / hbm_peak, 4),
             "error_vs_oracle_draw100": err}
        if name == "C0":
            r["us_per_step"] = round(1e3 * r["ms_per_step"], 1)
            r["note"] = "L2 resident (1.3 MB of vectors, 2.7 MB of matrix): latency-bound, GB/s not meaningful"
        out[name] = r
        h.close()
        del stg
    torch.cuda.empty_cache()
    return out


# ---------------------------------------------------------------- alpha sweep


def run_alpha_sweep(args, dev):
    """Single-GPU analogue of the paper's repartitioning-ratio study (Sec. 4): the
    128^3 mesh decomposed into k = 64 CPU ranks, solved as n_parts = 64 / alpha GPU
    parts (local + non-local matrices, halo gathered on the device), and, at one part,
    with k = 1 .. 512 CPU ranks merged."""
    import torch

    from paper_2510_08536_gb300 import repart, synth
    stream = torch.cuda.current_stream()

    def measure(mesh, n_parts, stg, b):
        t0 = time.perf_counter()
        h = repart.build_repartition(mesh.ranks, n_parts=n_parts)
        build_ms = 1e3 * (time.perf_counter() - t0)
        nl = sum(repart.get_part_map(h, p)["nl_nnz"] for p in range(n_parts))
        repart.update_values_packed(h, stg)
        out = {"n_parts": n_parts, "k": mesh.k, "map_build_ms": round(build_ms, 1), "nonlocal_entries": nl,
               "spmv_fp64_ms": round(repart.profile_iteration(h, b, "fp64", iters=10)["spmv"], 4),
               "spmv_fp32_ms": round(repart.profile_iteration(h, b, "mixed", iters=10)["spmv"], 4)}
        x = torch.zeros(mesh.n_cells, dtype=torch.float64, device=dev)
        for prec in ("fp64", "mixed_ru"):
            repart.solve(h, b, x, tol=1e-9, precision=prec)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            info = repart.solve(h, b, x, tol=1e-9, precision=prec)
            e1.record(stream)
            torch.cuda.synchronize()
            out[prec] = {"ms": round(e0.elapsed_time(e1), 2), "iterations": info["iterations"],
                         "status": info["status"]}
        h.close()
        return out

    res = {"workload": "128^3 cells, lognormal(0,0.5) faces seed 100, rhs U[-1,1] seed 0, rel. residual 1e-9",
           "alpha_sweep": [], "k_sweep": []}
    mesh = synth.box_mesh(128, 128, 128, 4, 4, 4)
    a = synth.face_coeffs(mesh, 0.5, 100)
    stg = torch.from_numpy(synth.Assembler(mesh).staging(a)).to(dev)
    b = torch.from_numpy(synth.uniform_vector(mesh, 0)).to(dev)
    for n_parts in (1, 2, 4, 8, 16, 32, 64):
        r = measure(mesh, n_parts, stg, b)
        r["alpha"] = mesh.k // n_parts
        res["alpha_sweep"].append(r)
    for p in ((1, 1, 1), (2, 2, 2), (4, 4, 4), (8, 8, 8)):
        mesh = synth.box_mesh(128, 128, 128, *p)
        stg = torch.from_numpy(synth.Assembler(mesh).staging(a)).to(dev)
        b = torch.from_numpy(synth.uniform_vector(mesh, 0)).to(dev)
        res["k_sweep"].append(measure(mesh, 1, stg, b))
    return res


# ---------------------------------------------------------------- ours


def replica_ms_per_step(ms_local, steps, device=None):
    """Timing of N independent replicas (weak scaling: every rank solves a whole
    time step of the workload per step). Each rank timed `steps` steps in
    ms_local; the job took the slowest rank's time (max over ranks). Returns
    (ms per time step of the slowest replica, that rank's ms, time steps per
    second of the whole job = N * steps / slowest time). Works over any
    initialised process group (NCCL on the GPUs, gloo in the CPU tests)."""
    import torch
    import torch.distributed as dist
    world = 1
    ms_max = float(ms_local)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        world = dist.get_world_size()
        t = torch.tensor([ms_max], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_max = float(t.item())
    return ms_max / steps, ms_max, world * steps / (ms_max * 1e-3)


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def run_ours(args):
    import numpy as np
    import torch

    from paper_2510_08536_gb300 import repart
    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    repart.load()
    hbm_peak, peak_kind = load_peaks()
    props = torch.cuda.get_device_properties(dev)
    gpu_id = f"GPU-{props.uuid}" if getattr(props, "uuid", None) else str(local)

    t0 = time.time()
    draws = max(1, min(args.draws, args.steps + args.warmup))
    mesh, asm, stg_host, b_np = make_inputs(args.workload, draws)
    setup_s = time.time() - t0
    n = mesh.n_cells
    stg_dev = [torch.from_numpy(s).to(dev) for s in stg_host]
    b = torch.from_numpy(b_np).to(dev)
    x = torch.zeros(n, dtype=torch.float64, device=dev)
    torch.cuda.synchronize()

    tb = time.perf_counter()
    h = repart.build_repartition(mesh.ranks, host_loop=int(args.host_loop))
    build_ms = 1e3 * (time.perf_counter() - tb)
    nnz, n_slots = h.nnz, h.n_slots
    sliced = repart.sliced_sizes(h)  # (slices, padded entries, table + index words) or None
    uniform4 = repart.sliced_uniform4(h)
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    def step(t, prec, src, bb, xx):
        repart.update_values_packed(h, src[t % draws])
        return repart.solve(h, bb, xx, tol=1e-9, precision=prec)

    def launches(prec, info):
        per_pass = {"fp64": 1, "mixed": 2, "mixed_ru": 3}[prec]  # residual (+ correction, + p continuation)
        solve = 1 + 3 * info["iterations"] + per_pass * info["passes"]
        return 2 + (1 if sliced else 0) + solve  # permutation + Jacobi diagonal (+ sliced values)

    results = {}
    clocks = {}
    precs = [args.only] if args.only else ["fp64", "mixed", "mixed_ru"]
    head = args.only or args.precision
    for prec in precs:
        for t in range(args.warmup):
            info = step(t, prec, stg_dev, b, x)
            assert info["status"] == 0, info
        barrier()
        sampler = Clocks(gpu_id)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        infos = []
        e0.record(stream)
        for t in range(args.steps):
            infos.append(step(args.warmup + t, prec, stg_dev, b, x))
        e1.record(stream)
        barrier()
        clocks[prec] = sampler.stop()
        ms_step, ms, job_rate = replica_ms_per_step(e0.elapsed_time(e1), args.steps, dev)
        bad = [i for i in infos if i["status"] != 0]
        results[prec] = {
            "ms_per_step": ms_step,
            "job_time_steps_per_s": job_rate,
            "iterations_mean": statistics.mean(i["iterations"] for i in infos),
            "outer_mean": statistics.mean(i["outer_iterations"] for i in infos),
            "max_rel_residual": max(i["rel_residual"] for i in infos),
            "not_converged_steps": len(bad),
            "gpu_launches": sum(launches(prec, i) for i in infos),
        }

    # error of each result (draw seed 100) against the oracle's solutions of the same
    # system (sampled rows, tests/golden/reference_solutions.json) and, whole vector,
    # against the FP64 result of this path
    repart.update_values_packed(h, stg_dev[0])
    sols = {}
    for prec in precs:
        xx = torch.zeros(n, dtype=torch.float64, device=dev)
        repart.solve(h, b, xx, tol=1e-9, precision=prec)
        sols[prec] = xx
        results[prec]["error_vs_oracle_draw100"] = reference_errors(args.workload, xx)
    if "fp64" in sols:
        ref_norm = float(torch.linalg.norm(sols["fp64"]))
        for prec in precs:
            results[prec]["rel_error_vs_fp64"] = float(torch.linalg.norm(sols[prec] - sols["fp64"])) / ref_norm
    del sols

    # the same steps with the line (block-tridiagonal, 32-row blocks) preconditioner
    line = None
    if not args.no_line and world == 1:
        repart.set_solver_options(h, precond=repart.RP_PRECOND_LINE)
        line = {"precond": "block-Jacobi over 32-row blocks (tridiagonal part): x-lines of the 256^3 ranks"}
        ln_steps = max(1, min(args.steps, 5))
        for prec in precs:
            for t in range(2):
                assert step(t, prec, stg_dev, b, x)["status"] == 0
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            infos = []
            e0.record(stream)
            for t in range(ln_steps):
                infos.append(step(t, prec, stg_dev, b, x))
            e1.record(stream)
            torch.cuda.synchronize()
            line[prec] = {"ms_per_step": round(e0.elapsed_time(e1) / ln_steps, 3),
                          "iterations_mean": statistics.mean(i["iterations"] for i in infos),
                          "max_rel_residual": max(i["rel_residual"] for i in infos),
                          "statuses": sorted({i["status"] for i in infos})}
        for prec in ("fp64", "mixed"):
            if prec in precs:
                kk = [repart.profile_iteration(h, b, prec, iters=20) for _ in range(2)]
                line[prec]["kernel_ms"] = {k2: round(v, 5) for k2, v in kk[-1].items()}
        repart.set_solver_options(h, precond=repart.RP_PRECOND_JACOBI)
        repart.update_values_packed(h, stg_dev[0])

    # kernel durations (CUDA events on the launching stream, same kernels as the graph runs)
    kern = {}
    for prec in precs:
        if prec == "mixed_ru" and "mixed" in kern:  # the same FP32 iteration kernels
            kern[prec] = kern["mixed"]
            continue
        kk = [repart.profile_iteration(h, b, prec, iters=20) for _ in range(2)]
        kern[prec] = kk[-1]
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record(stream)
    reps = 10
    for t in range(reps):
        repart.update_values_packed(h, stg_dev[t % draws])
    ev[1].record(stream)
    torch.cuda.synchronize()
    upd_ms = ev[0].elapsed_time(ev[1]) / reps

    def spmv_bytes(prec):
        w = 8 if prec == "fp64" else 4
        if sliced:  # values + index words + table references + tables + slice descriptors + p read + q write
            slices, entries, ibuf_len, tabs_len = sliced
            return w * entries + 4 * ibuf_len + 4 * slices + 4 * tabs_len + 8 * (slices + 1) + 2 * w * n
        return (w + 4) * nnz + 4 * (n + 1) + 2 * w * n

    def gbs(bytes_, ms):
        return bytes_ / (ms * 1e-3) / 1e9

    upd_bytes = 20 * nnz + 4 * nnz + 20 * n  # idx + gather + FP64 write + FP32 write; diag read + 2 writes
    if sliced:  # sliced values: position + CSR value read, FP64 + FP32 write per padded entry
        upd_bytes += 24 * sliced[1]
    if sliced and repart.inner_scaled(h):
        # S A S values: FP64 sliced value read, s (FP64) at the column, FP32 write per
        # padded entry, index words; s itself: diagonal position + value read, FP64 write per row
        upd_bytes += (8 + 8 + 4) * sliced[1] + 4 * sliced[2] + 20 * n
    k1_name = "k_it_spmv_sl" if sliced else "k_it_spmv"
    u4 = ", true" if sliced and uniform4 else ""  # the uniform-slice instance
    roof = {"bound": "hbm", "kernel": f"{k1_name}<{'double' if head == 'fp64' else 'float'}{u4}>",
            "achieved": round(gbs(spmv_bytes(head), kern[head]["spmv"]), 1), "peak": hbm_peak, "unit": "GB/s",
            "peak_kind": peak_kind}
    roof["frac"] = round(roof["achieved"] / hbm_peak, 4)
    roof["traffic"] = PROFILED_TRAFFIC.get((args.workload, roof["kernel"]))
    roof["algorithmic_bytes"] = spmv_bytes(head)
    roof["ms_per_launch"] = kern[head]["spmv"]
    other = [p for p in precs if p != head]
    # FP64 SpMV against the FP64 FMA rate: one FMA per stored (padded) entry and one for p.q
    fp64_alu = None
    if "fp64" in kern:
        fma = (sliced[1] if sliced else nnz) + n
        sm_mhz = clocks.get("fp64", {}).get("sm_max_mhz") or MAX_SM_MHZ
        peak_tf = fp64_peak_tflops(dev, sm_mhz)
        ach_tf = 2 * fma / (kern["fp64"]["spmv"] * 1e-3) / 1e12
        fp64_alu = {"bound": "alu", "kernel": f"{k1_name}<double{u4}>", "achieved": round(ach_tf, 4), "unit": "TFLOP/s",
                    "peak": round(peak_tf, 4), "peak_kind": "derived: SMs x 2 FP64 FMA/clk x 2 flop x max SM clock",
                    "frac": round(ach_tf / peak_tf, 4), "fma_per_launch": fma}
    kernels = {}
    scaled = repart.inner_scaled(h)  # mixed: FP32 iteration on S A S (no diagonal reads in K2, K3)
    for prec in precs:
        w = 8 if prec == "fp64" else 4
        if prec != "fp64" and scaled:
            kb = {"spmv": spmv_bytes(prec), "resid": 3 * w * n, "xp": 5 * w * n}
        else:
            kb = {"spmv": spmv_bytes(prec), "resid": 4 * w * n, "xp": 6 * w * n}
        kernels[prec] = {k: {"ms": round(kern[prec][k], 5), "GB/s": round(gbs(kb[k], kern[prec][k]), 1),
                             "frac": round(gbs(kb[k], kern[prec][k]) / hbm_peak, 4)} for k in kb}
    kernels["update"] = {"ms": round(upd_ms, 4), "GB/s": round(gbs(upd_bytes, upd_ms), 1),
                         "frac": round(gbs(upd_bytes, upd_ms) / hbm_peak, 4)}

    # value update from a host buffer: H2D copy + permutation vs the permutation kernel
    # gathering from host memory in place over the CPU-GPU link
    update_paths = None
    stg_pin = None
    if not args.no_e2e:
        stg_pin = [torch.from_numpy(s).pin_memory() for s in stg_host]
        update_paths = {"device_buffer_ms": round(upd_ms, 3)}
        for name, direct in (("host_copy_then_permute_ms", False), ("host_direct_gather_ms", True)):
            repart.update_values_packed(h, stg_pin[0], direct=direct)
            torch.cuda.synchronize()
            ev[0].record(stream)
            for t in range(reps):
                repart.update_values_packed(h, stg_pin[t % draws], direct=direct)
            ev[1].record(stream)
            torch.cuda.synchronize()
            update_paths[name] = round(ev[0].elapsed_time(ev[1]) / reps, 3)
        update_paths["host_bytes_per_update"] = 8 * n_slots

    # end to end through the C ABI with host buffers: every step uploads its coefficient
    # buffer and b from pinned host memory and reads x back. Pipelined (the headline
    # e2e): step t+1's buffer goes up on the handle's copy stream (RP_MEM_HOST_ASYNC)
    # while step t solves, and rp_get_solve_info reads step t's outcome after that
    # upload is queued. Serial: each step's upload waits for the previous solve.
    e2e = None
    if not args.no_e2e:
        b_pin = torch.from_numpy(b_np).pin_memory()
        x_pin = torch.zeros(n, dtype=torch.float64).pin_memory()

        def alone(fn, reps=3):
            fn()
            torch.cuda.synchronize()
            ev[0].record(stream)
            for _ in range(reps):
                fn()
            ev[1].record(stream)
            torch.cuda.synchronize()
            return ev[0].elapsed_time(ev[1]) / reps

        stg_dev0, x_dev = stg_dev[0], torch.empty(n, dtype=torch.float64, device=dev)
        phases = {"h2d_buffer_ms": alone(lambda: stg_dev0.copy_(stg_pin[0], non_blocking=True)),
                  "h2d_b_ms": alone(lambda: x_dev.copy_(b_pin, non_blocking=True)),
                  "d2h_x_ms": alone(lambda: x_pin.copy_(x_dev, non_blocking=True)),
                  "permute_ms": upd_ms, "solve_ms": results[head]["ms_per_step"] - upd_ms}
        phases = {k: round(v, 3) for k, v in phases.items()}
        phases["h2d_buffer_GBps"] = round(8 * n_slots / (phases["h2d_buffer_ms"] * 1e-3) / 1e9, 1)
        del x_dev

        def pipelined(t0, steps, evs=None):
            repart.update_values_packed(h, stg_pin[t0 % draws], asynchronous=True)
            for t in range(steps):
                repart.solve(h, b_pin, x_pin, tol=1e-9, precision=head, wait=False)
                if t + 1 < steps:
                    repart.update_values_packed(h, stg_pin[(t0 + t + 1) % draws], asynchronous=True)
                info = repart.solve_info(h)
                assert info["status"] == 0, info
                if evs is not None:
                    evs[t + 1].record(stream)

        pipelined(0, max(1, args.warmup))
        barrier()
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
        evs[0].record(stream)
        pipelined(args.warmup, args.steps, evs)
        barrier()
        ems_step, _, _ = replica_ms_per_step(evs[0].elapsed_time(evs[-1]), args.steps, dev)
        per_step = [evs[t].elapsed_time(evs[t + 1]) for t in range(args.steps)]
        # the same steps without the overlap (each call waits for the previous one)
        s_steps = max(1, min(args.steps, 5))
        step(0, head, stg_pin, b_pin, x_pin)
        barrier()
        ev[0].record(stream)
        for t in range(s_steps):
            assert step(args.warmup + t, head, stg_pin, b_pin, x_pin)["status"] == 0
        ev[1].record(stream)
        barrier()
        e2e = {"value": round(ems_step, 3), "unit": "ms/time-step",
               "h2d_bytes_per_step": 8 * n_slots + 8 * n, "d2h_bytes_per_step": 8 * n,
               "path": "per step: rp_update_values_packed(RP_MEM_HOST_ASYNC) of the next step's pinned buffer "
                       "queued behind rp_solve (pinned b, x) + rp_get_solve_info",
               "step_ms_median": round(statistics.median(per_step), 3), "step_ms_max": round(max(per_step), 3),
               "serial_ms_per_step": round(ev[0].elapsed_time(ev[1]) / s_steps, 3),
               "serial_path": "rp_update_values_packed(RP_MEM_HOST) + rp_solve with info, one after the other",
               "phases_alone": phases}
        del stg_pin

    h.close()
    del stg_dev
    torch.cuda.empty_cache()

    # the other forms are measured on one GPU only: a replica run times the headline step
    small = None
    if world == 1 and not args.no_small:
        small = run_small_configs(dev)
    batched = None
    if not args.no_batch and world == 1:
        batched = run_batch(args, dev, steps=max(1, min(args.steps, 5)), warmup=max(1, min(args.warmup, 2)))
    adj = None
    if not args.no_bicgstab and args.workload == "mixed_256" and world == 1:
        adj = run_adjoint(dev)
    bicg = None
    if not args.no_bicgstab and args.workload == "mixed_256" and world == 1:
        bicg = run_bicgstab(dev, steps=max(1, min(args.steps, 3)), warmup=max(1, min(args.warmup, 2)))

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            cpu = cpu_baseline(args, results.get("fp64", {}).get("iterations_mean"))
        except Exception as exc:  # report, do not hide
            cpu = {"value": None, "error": str(exc)[-300:]}

    if rank != 0:
        return None
    headr = results[head]
    line = {
        "metric": METRIC, "value": round(headr["ms_per_step"], 3), "unit": "ms/time-step", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(headr["ms_per_step"], 3),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if head == "fp64" else "f32-in-f64", "data": "synthetic",
        "config": {"workload": f"{args.workload}: {WORKLOAD_TEXT[args.workload]}", "headline": head,
                   "n_rows": n, "nnz": nnz, "draws_cycled": draws, "l2": "inputs larger than L2, no flush",
                   "layout": ({"kind": "sliced", "slices": sliced[0], "padded_entries": sliced[1],
                               "index_words": sliced[2], "table_words": sliced[3], "uniform4": uniform4}
                              if sliced else {"kind": "csr"}),
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "fp64_ms_per_step": round(results["fp64"]["ms_per_step"], 3) if "fp64" in results else None,
        "mixed_ms_per_step": round(results["mixed"]["ms_per_step"], 3) if "mixed" in results else None,
        "mixed_ru_ms_per_step": round(results["mixed_ru"]["ms_per_step"], 3) if "mixed_ru" in results else None,
        "mixed_ru_delta": 0.1,
        "per_precision": results, "kernels": kernels, "roofline": roof,
        "mixed_inner_system": "S A S (Jacobi made explicit)" if scaled else "A, Jacobi-preconditioned",
        "roofline_other_spmv": {o: {"achieved": round(gbs(spmv_bytes(o), kern[o]["spmv"]), 1),
                                    "frac": round(gbs(spmv_bytes(o), kern[o]["spmv"]) / hbm_peak, 4)} for o in other},
        "roofline_fp64_spmv": fp64_alu,
        "map_build_ms": round(build_ms, 1), "input_setup_s": round(setup_s, 1), "update_paths": update_paths,
        "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": results[head]["gpu_launches"], "batched": batched,
        "bicgstab": bicg, "line_precond": line, "adjoint": adj, "configs_small": small,
        "clocks": clocks[head], "clocks_other": {o: clocks[o] for o in other},
    }
    return line


def run_reference(args):
    """The reference arm: the oracle (its C / OpenMP restatement) on every host core.
    Each timed step is one full time step of the workload -- value update, Jacobi
    diagonal, FP64 Jacobi-PCG to 1e-9 from x = 0 -- timed end to end, nothing
    scaled; the coefficient draws cycle like the GPU arm's. Warm-up steps are
    value updates only (untimed)."""
    world, rank, _ = dist_env()
    if rank != 0:
        return None
    draws = max(1, min(args.draws, args.steps + args.warmup))
    seeds = [100 + ((args.warmup + t) % draws) for t in range(args.steps)]
    t0 = time.time()
    leg = run_oracle_subprocess({"workload": args.workload, "seeds": seeds, "threads": 0, "mode": "full",
                                 "warmup": args.warmup}, timeout=3600)
    ms = statistics.mean(st["ms"] for st in leg["steps"])
    return {
        "impl": "reference", "metric": METRIC, "value": round(ms, 1), "unit": "ms/time-step", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 1), "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{args.workload}: {WORKLOAD_TEXT[args.workload]}", "headline": "fp64 oracle"},
        "cpu_baseline": {"value": round(ms, 1), "unit": "ms/time-step", "cores": leg["threads"], "kind": "oracle",
                         "sample": f"{args.steps} full time steps (value update, Jacobi diagonal, FP64 Jacobi-PCG "
                                   f"to 1e-9 from x = 0) of the workload by the oracle's C / OpenMP restatement on "
                                   f"{leg['threads']} host cores, each timed end to end; {args.warmup} untimed "
                                   f"update-only warm-up steps"},
        "e2e": {"value": round(ms, 1), "unit": "ms/time-step", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "iterations_mean": statistics.mean(st["iterations"] for st in leg["steps"]),
        "max_true_rel_residual": max(st["true_rel_residual"] for st in leg["steps"]),
        "setup_s": leg["setup_s"], "wall_s": round(time.time() - t0, 1),
    }


def main():
    args = parse()
    if args.oracle_leg:
        print(json.dumps(oracle_leg(json.loads(args.oracle_leg))))
        return
    if args.alpha_sweep and args.impl == "ours":
        import torch
        from paper_2510_08536_gb300 import repart
        torch.cuda.set_device(0)
        repart.load()
        print(json.dumps(run_alpha_sweep(args, torch.device("cuda", 0))))
        return
    if args.only_bicgstab and args.impl == "ours":
        import torch
        from paper_2510_08536_gb300 import repart
        torch.cuda.set_device(0)
        repart.load()
        precs = ("mixed",) if args.only == "mixed" else ("fp64",) if args.only == "fp64" else ("fp64", "mixed")
        print(json.dumps({"bicgstab": run_bicgstab(torch.device("cuda", 0), steps=args.steps, warmup=args.warmup,
                                                   host_loop=args.host_loop, precs=precs)}))
        return
    if args.only_batch and args.impl == "ours":
        import torch
        from paper_2510_08536_gb300 import repart
        torch.cuda.set_device(0)
        repart.load()
        print(json.dumps({"batched": run_batch(args, torch.device("cuda", 0), steps=args.steps, warmup=args.warmup)}))
        return
    line = run_reference(args) if args.impl == "reference" else run_ours(args)
    if line is not None:
        print(json.dumps(line))
    if int(os.environ.get("WORLD_SIZE", "1")) > 1 and args.impl == "ours":
        import torch.distributed as dist
        if dist.is_initialized():
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
