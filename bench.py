"""Benchmark: V-cycle throughput of the GB300 multigrid solve (DOFs per second per V-cycle).

Workload (default): the largest single-GPU workload, 3D diffusion -div(k grad u) = 1 on
the unit cube, conforming Q1 on a 256^3 hex mesh (16,581,375 interior DOFs), k piecewise
constant on 16^3 blocks with log10 k ~ U[-2, 2] (SplitMix64 seed 20260101), 7 levels
(coarsest 4^3 cells, dense LU; Galerkin levels where the cells straddle the blocks),
V(2,2) with one degree-2 Chebyshev polynomial per smoothing phase, in the precision the
workload specifies: FP32 V-cycle inside FP64 defect correction. A step is one
defect-correction iteration: FP64 outer residual and its norm, one FP32 V-cycle, x += c.

Prints one JSON line (rank 0). Besides the throughput it reports
  * roofline: the dominant kernel of the step (events around each of its launches inside
    the timed region), against the roofline that binds it, with the HBM fraction beside
    it; roofline_kernels: the finest level's other dominant class the same way, timed in
    an instrumented pass (events around every launch) that precedes the timed region;
  * ms_per_step_no_events: the same number of steps without any events;
  * whole_cycle: algorithmic bytes of every launch of one step over the step time;
  * e2e: full solves to 1e-10 through mg_solve_host from pinned host memory;
  * time_to_solution: mixed vs plain FP64 to 1e-10 on the same inputs (and CG);
  * configs: the 128^3 constant-coefficient Q1 workload in both precisions;
  * cpu_baseline: the FP64 CPU oracle on a bounded sample of the same workload, on all
    host cores and on one.
--impl reference times the oracle alone (the reference arm) on the host cores.
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "V-cycle DOFs/s"
UNIT = "DOF/s"
DEFAULT_CONFIG = "q1_3d_256_vark"
WORKLOADS = {
    "q1_3d_256_vark": "3D diffusion, Q1, 256^3 cells (16,581,375 DOFs), k on 16^3 blocks (log10 k ~ U[-2,2]), "
                      "7 levels, V(2,2) Chebyshev deg 2, FP32 V-cycle in FP64 defect correction",
    "q1_3d_128_cheb": "3D Poisson, Q1, 128^3 cells (2,048,383 DOFs), 6 levels, V(2,2) Chebyshev deg 2, FP64",
    "q1_2d_64": "2D Poisson, Q1, 64^2 cells (3,969 DOFs), 5 levels, V(2,2) Jacobi 0.8, FP64",
    "rq1_3d_96": "3D Poisson, rotated Q1, 96^3 cells (2,626,560 DOFs), 6 levels, V(2,2) Jacobi 0.7, FP64",
    "p1_3d_128_cheb": "3D Poisson, P1 on Kuhn tetrahedra, 128^3 cells (2,048,383 DOFs), 6 levels, Chebyshev deg 2, FP64",
    "p2_3d_64_cheb": "3D Poisson, P2 on Kuhn tetrahedra, 64^3 cells (2,048,383 DOFs), 5 levels, Chebyshev deg 2, FP64",
}


def _env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def _max_sm_mhz():
    """Maximum SM clock: nvidia-smi, else MEASURED_PEAKS.json, else the nominal 2070 MHz."""
    try:
        out = subprocess.run(["nvidia-smi", "-i", "0", "--query-gpu=clocks.max.sm", "--format=csv,noheader,nounits"],
                             capture_output=True, text=True, timeout=20).stdout.strip().splitlines()
        return float(out[0]), "nvidia-smi clocks.max.sm"
    except (OSError, ValueError, IndexError, subprocess.SubprocessError):
        pass
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return float(json.load(open(p)).get("sm_max_mhz", 2070.0)), "MEASURED_PEAKS.json sm_max_mhz"
    return 2070.0, "nominal"


def fp64_peak():
    """FP64 pipe peak of this device: SMs x maximum SM clock x 2 FP64 FMA per clock per SM
    x 2 flop (GB300's unit count; the nominal 1.25 TFLOP/s at 152 SMs and 2.07 GHz)."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    mhz, src = _max_sm_mhz()
    return sms * mhz * 1e6 * 2 * 2 / 1e12, "FP64 pipe: %d SMs x %.0f MHz (%s) x 2 DFMA/clk/SM x 2 flop" % (sms, mhz, src)

class ClockSampler:
    """nvidia-smi clock / throttle samples every 25 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "25"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.lines:
            return None
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


CSRC = os.path.join(ROOT, "paper_1609_04809_gb300", "csrc")
# the source a kernel's code consists of: (file, function or struct) in order
KERNEL_PARTS = {
    "k_dia_sweep": [("sweep.cuh", "pdl_enter"), ("sweep.cuh", "struct Ar<double>"), ("sweep.cuh", "struct Ar<float>"),
                    ("sweep.cuh", "sweep_out"), ("sweep.cuh", "k_dia_sweep")],
    "k_coef_sweep": [("sweep.cuh", "pdl_enter"), ("sweep.cuh", "struct Ar<float>"), ("sweep.cuh", "sweep_out"),
                     ("sweep.cuh", "sweep_out_v"), ("sweep.cuh", "fused_update"), ("sweep.cuh", "struct CoefView"),
                     ("sweep.cuh", "k_coef_sweep")],
    "k_outer_resid": [("sweep.cuh", "pdl_enter"), ("sweep.cuh", "struct Ar<float>"), ("sweep.cuh", "sweep_out_v"),
                      ("kernels.cuh", "block_sum"), ("kernels.cuh", "finish_norm"), ("kernels.cuh", "fp64_row"),
                      ("kernels.cuh", "fp64_dof"), ("kernels.cuh", "struct ZStep"), ("kernels.cuh", "zstep_dinv"),
                      ("kernels.cuh", "fp64_rows_blocks_per_sm"), ("kernels.cuh", "k_outer_resid")],
}
SWEEP_KERNELS = {"dia": "k_dia_sweep", "ell": "k_ell_sweep", "csr": "k_csr_sweep", "sell": "k_sell_sweep",
                 "stencil": "k_stencil_sweep", "coef": "k_coef_sweep"}


def _source_part(src, name):
    """The text of one function (its template line included) or struct of a source file."""
    if name.startswith("struct "):
        start = src.index(name + " {")
        return src[start:src.index("\n};\n", start) + 4]
    import re
    m = re.search(r"(^template <[^\n]*\n)?^\S[^\n]*?\b" + re.escape(name) + r"\(", src, re.M)
    if m is None:
        raise KeyError(name)
    line_end = src.index("\n", m.end())
    if src[m.end():line_end].rstrip().endswith("}"):  # a one-line function
        return src[m.start():line_end + 1]
    return src[m.start():src.index("\n}\n", m.start()) + 3]


def _kernel_sha(kernel, sources=None):
    """sha256[:16] of the code a kernel consists of (KERNEL_PARTS), comments and blank lines
    dropped. sources: {file: text} (default: the files in csrc/)."""
    text = []
    for f, name in KERNEL_PARTS[kernel]:
        src = sources[f] if sources else open(os.path.join(CSRC, f)).read()
        text.append(_source_part(src, name))
    lines = [ln.split("//")[0].rstrip() for ln in "\n".join(text).splitlines()]
    return hashlib.sha256("\n".join(ln for ln in lines if ln.strip()).encode()).hexdigest()[:16]


def _traffic(tag, kernel, n_dofs):
    """DRAM bytes per launch of `kernel` from the committed ncu record `tag`, if the record
    was taken on the kernel's code as it is now; records taken on a smaller case of the
    workload are scaled to n_dofs rows (the traffic of these passes grows with the rows)."""
    if kernel not in KERNEL_PARTS:
        return None
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    sha = _kernel_sha(kernel)
    for line in open(path):
        parts = line.split()
        if len(parts) >= 4 and parts[0] == tag and parts[1] == sha:
            return float(parts[2]) * n_dofs / float(parts[3])
    return None


def kernel_roofline(kclass, precision, storage, workload, n_dofs, ms, cnt, nbytes, flops, peak_gbs, peak_kind,
                    fp64_tf, fp64_kind):
    """One kernel class of the finest level against the roofline that binds it: the FP64
    pipe for FP64 passes (GB300 issues about 2 DFMA per clock per SM, below HBM speed for
    these passes), HBM bandwidth for the FP32 ones; the HBM fraction is reported beside
    the FP64 one. ms, cnt: event-timed total and launches; nbytes, flops: algorithmic per
    launch (mg_profile_read)."""
    if not cnt:
        return None
    sec = ms / cnt * 1e-3
    gbs = nbytes / sec / 1e9
    kernel = {"outer": "k_outer_resid", "smooth": SWEEP_KERNELS.get(storage)}.get(kclass)
    tag = "%s_%s_%s_%s" % (kclass, precision, workload, "dia" if kclass == "outer" else storage)
    hbm = {"achieved": gbs, "peak": peak_gbs, "unit": "GB/s", "frac": gbs / peak_gbs,
           "peak_kind": "%s HBM copy bandwidth (MEASURED_PEAKS.json hbm_gbs)" % peak_kind}
    what = {"outer": "FP64 outer residual r = b - A x and ||r||^2 (defect correction)",
            "smooth": "finest-level smoother sweep (%s storage, %s)" % (storage, precision)}[kclass]
    common = {"kernel": what, "bytes_per_launch": nbytes, "flops_per_launch": flops, "launches": cnt,
              "us_per_launch": 1e6 * sec, "traffic": _traffic(tag, kernel, n_dofs) if kernel else None,
              "traffic_record": tag}
    if precision == "fp64" or kclass == "outer":
        tf = flops / sec / 1e12
        out = {"bound": "alu", "achieved": tf, "peak": fp64_tf, "unit": "TFLOP/s", "frac": tf / fp64_tf,
               "peak_kind": fp64_kind, "hbm": hbm}
    else:
        out = dict(hbm)
        out["bound"] = "hbm"
    out.update(common)
    return out


def replica_throughput(ms_local, n_dofs, steps, world, dist=None, device="cpu"):
    """Whole-job V-cycle DOFs/s of `world` independent replicas: every rank ran `steps`
    iterations on its own n_dofs problem; the job time is the slowest rank's."""
    import torch
    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    if dist is not None and world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    return world * n_dofs * steps / (ms_max * 1e-3), ms_max


SMOOTHERS = {"jacobi": 0, "chebyshev": 1, "gauss-seidel": 2}
STORAGES = {"auto": 0, "csr": 1, "ell": 2, "dia": 3, "sell": 4, "stencil": 5, "coef": 6}
STORAGE_NAMES = {v: k for k, v in STORAGES.items()}
SWEEP_TEXT = {0: "fused residual + damped Jacobi update", 1: "fused residual + Chebyshev update",
              2: "one colour of a multicolour Gauss-Seidel sweep, in place"}


def _tail_mode(args):
    if args.no_tail or args.tail == "off":
        return 0
    return 1 if args.tail == "on" else 2


def _config_args(name, smoother="workload", cells=None):
    """The workload's parameters; `smoother` other than "workload" replaces its smoother;
    `cells` runs the same workload on another grid (levels adjusted so that the coarsest
    grid keeps its size; used for profiling a smaller case)."""
    from paper_1609_04809_gb300 import workloads as W
    c = dict({**W.CONFIGS, **W.TET_CONFIGS}[name])
    if smoother != "workload":
        c["smoother"] = SMOOTHERS[smoother]
    if cells and cells != c["n_cells"]:
        coarse = c["n_cells"] >> (c["n_levels"] - 1)
        c["n_levels"] = int(round(np.log2(cells / coarse))) + 1
        c["n_cells"] = cells
    return c


def _k_field(c):
    from paper_1609_04809_gb300 import workloads as W
    if c.get("k") == "blocks16":
        return W.k_blocks(c["n_cells"], dim=3, blocks_per_axis=16, seed=20260101)
    return None


def _modes(c):
    from paper_1609_04809_gb300 import workloads as W
    return W.manufactured_modes(c["dim"]) if c["rhs"] == "manufactured" else None


def _problem_rhs(c):
    from paper_1609_04809_gb300 import mg
    return mg.mg_load_vector(c["dim"], c["element"], c["n_cells"], modes=_modes(c), f_const=1.0)


def _hierarchy(c, precision, args=None):
    from paper_1609_04809_gb300 import mg
    kw = {}
    if args is not None:
        kw = dict(use_pdl=0 if args.no_pdl else 1, coarse_tail=_tail_mode(args), storage=STORAGES[args.storage])
    return mg.Hierarchy(c["dim"], c["element"], c["n_cells"], c["n_levels"], k_cell=_k_field(c),
                        smoother=c["smoother"], omega=c["omega"], cheb_degree=c["cheb_degree"], nu_pre=c["nu_pre"],
                        nu_post=c["nu_post"], precision=mg.MG_MIXED if precision == "mixed" else mg.MG_FP64, **kw)


def _oracle_workload(name, smoother="workload", cells=None):
    import oracle
    c = _config_args(name, smoother, cells)
    O = oracle.Hierarchy(c["dim"], c["element"], c["n_cells"], c["n_levels"], k_cell=_k_field(c),
                         opts=oracle.Options(smoother=c["smoother"], omega=c["omega"], cheb_degree=c["cheb_degree"],
                                             nu_pre=c["nu_pre"], nu_post=c["nu_post"]))
    b = oracle.load_vector(c["dim"], c["element"], c["n_cells"], modes=_modes(c))
    return O, O.A(c["n_levels"] - 1), b


def _oracle_step(O, A, b, x):
    """One defect-correction iteration of the oracle: r = b - A x, c = V(r), x + c."""
    import oracle
    r = b - oracle.spmv(A, x)
    return x + O.vcycle(r)


def _host_cpu():
    model = None
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith(("model name", "cpu model")):
                model = ln.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    if model is None:
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for ln in out.splitlines():
                if ln.startswith("Model name"):
                    model = ln.split(":", 1)[1].strip()
                    break
        except (OSError, subprocess.SubprocessError):
            pass
    return {"nproc": os.cpu_count(), "model": model}


def _workload_config(name, c, n, nnz_finest):
    """The bench line's `config`: the workload alone, the same for both arms."""
    return {"workload": name, "description": WORKLOADS.get(name, name), "n_dofs": int(n), "n_cells": c["n_cells"],
            "l2": "inputs larger than L2 (finest FP64 matrix %.0f MB > 129 MB L2)" % (int(nnz_finest) * 8 / 1e6)}


def cpu_baseline(name, cycles_all=3, cycles_one=1, smoother="workload"):
    """The oracle (plain FP64 C; row loops on OpenMP threads) on the same workload: setup
    (not timed), then `cycles_all` defect-correction iterations on all host cores and
    `cycles_one` on one core."""
    import oracle
    t0 = time.perf_counter()
    O, A, b = _oracle_workload(name, smoother)
    setup = time.perf_counter() - t0
    cores = os.cpu_count() or 1
    out = {}
    for tag, th, cyc in (("all", cores, cycles_all), ("one", 1, cycles_one)):
        oracle.set_threads(th)
        x = np.zeros(O.n)
        t0 = time.perf_counter()
        for _ in range(cyc):
            x = _oracle_step(O, A, b, x)
        dt = time.perf_counter() - t0
        out[tag] = (O.n * cyc / dt, dt, th, cyc)
    oracle.set_threads(cores)
    return out, setup


def serve_bench(args):
    """Serving workload: seeded trace of Q1 Poisson solves, Poisson arrivals at 70% of capacity.

    1. operator cache warm-up (one solve per problem shape) and tile-shape autotuning;
    2. capacity: the first requests of the trace submitted at once (closed loop);
    3. the whole trace with Poisson arrivals at 0.7 x capacity; latency = completion -
       arrival (submission happens at the arrival time), right-hand sides assembled by
       the server from the four sine modes, tolerance 1e-8, FP32 V-cycle in FP64.
    """
    import threading as th

    from paper_1609_04809_gb300 import mg, workloads as W
    tol = 1e-8
    levels = lambda N: int(round(np.log2(N))) - 1  # coarsest 4 cells per axis
    trace = W.serving_trace(n_requests=args.serve_requests, seed=4096)
    shapes = sorted(set((r["dim"], r["n_cells"]) for r in trace))
    S = mg.Server(int(args.serve_budget_gb * (1 << 30)), max_active=args.serve_slots)
    try:
        t0 = time.perf_counter()
        tuned = S.tune([(d, n, levels(n)) for d, n in shapes], repeats=2, rel_tol=tol)
        t_tune = time.perf_counter() - t0
        nmax = max(mg.mg_ndofs(d, 0, n) for d, n in shapes)
        xbuf = np.zeros(nmax)

        def run(reqs, rate):
            S.reset_stats()
            tickets = [None] * len(reqs)
            start = time.perf_counter()

            def submitter():
                for k, r in enumerate(reqs):
                    if rate:
                        delay = start + r["arrival"] - time.perf_counter()
                        if delay > 0:
                            time.sleep(delay)
                    tickets[k] = S.submit_rhs(r["dim"], r["n_cells"], levels(r["n_cells"]), r["modes"], tol)

            th_sub = th.Thread(target=submitter)
            th_sub.start()
            iters = []
            for k, r in enumerate(reqs):
                while tickets[k] is None:
                    time.sleep(0.0005)
                n = mg.mg_ndofs(r["dim"], 0, r["n_cells"])
                st, x, it, _ = S.wait(tickets[k], n, timeout_s=1200.0)
                if st != mg.MG_OK:
                    raise RuntimeError("request %d ended with status %d" % (k, st))
                iters.append(it)
            th_sub.join()
            return time.perf_counter() - start, S.stats(), iters

        cap_n = min(args.serve_capacity_requests, len(trace))
        cap_wall, cap_stats, cap_iters = run(trace[:cap_n], None)
        capacity = cap_n / cap_wall
        cap_work = sum(mg.mg_ndofs(r["dim"], 0, r["n_cells"]) * it for r, it in zip(trace[:cap_n], cap_iters))
        rate = 0.7 * capacity
        trace = W.serving_trace(n_requests=args.serve_requests, seed=4096, rate=rate)
        wall, st, iters = run(trace, rate)
        dofs = sum(mg.mg_ndofs(r["dim"], 0, r["n_cells"]) for r in trace)
        return {"requests": len(trace), "tol": tol, "precision": "FP32 V-cycle in FP64 defect correction",
                "arrival_rate_per_s": rate, "capacity_solves_per_s": capacity,
                "capacity_sample": cap_n,
                "capacity_dof_vcycles_per_s": cap_work / cap_wall,
                "capacity_gpu_busy_frac": cap_stats["gpu_ms"] / max(cap_stats["span_ms"], 1e-9),
                "capacity_mean_batch": cap_stats["mean_batch"],
                "solves_per_s": st["solves_per_s"], "p50_ms": st["p50_ms"],
                "p99_ms": st["p99_ms"], "max_ms": st["max_ms"], "mean_batch": st["mean_batch"],
                "gpu_busy_frac": st["gpu_ms"] / max(st["span_ms"], 1e-9),
                "setup_busy_frac": st["setup_ms"] / max(st["span_ms"], 1e-9),
                "iterations_mean": float(np.mean(iters)), "iterations_max": int(np.max(iters)),
                "dofs_total": int(dofs), "wall_s": wall, "budget_gb": args.serve_budget_gb,
                "device_bytes_peak": int(st["device_bytes_peak"]), "operator_sets": st["operator_sets"],
                "tile": {"rows_per_thread": tuned[0], "blocks_per_sm": tuned[1], "tune_s": t_tune}}
    finally:
        S.close()


def heat_report(n_cells=128, n_levels=6, dt=0.01, t_end=5.0, smoother=1, nu=1, tol=1e-10, methods=("dc", "pcg"),
                precisions=("fp64", "mixed"), element=0):
    """The heat-equation workload (Crank-Nicolson, the paper's model problem; element 0:
    Q1 hexahedra, 2: P1 on the Kuhn tetrahedra): the whole time loop with u resident on
    the device (mg_heat), per method and precision, and once through the host API
    (mg_heat_host, host arrays in and out)."""
    import torch

    from paper_1609_04809_gb300 import mg, workloads as W
    wl = W.heat_workload(dim=3, n_cells=n_cells, n_levels=n_levels, dt=dt, t_end=t_end)
    bF = mg.mg_load_vector(3, element, n_cells, modes=wl["source_modes"])
    bFd = torch.from_numpy(bF).cuda()
    exact = W.q1_nodal_sine(3, n_cells, amp=wl["exact_amp"])  # Q1 and P1 share the vertex DOFs
    n = bF.size
    out = {"workload": "heat_%s_3d_%d" % ("p1" if element == 2 else "q1", n_cells), "n_dofs": int(n), "dt": dt,
           "t_end": t_end,
           "n_steps": wl["n_steps"], "tol_per_step": tol,
           "smoother": [k for k, v in SMOOTHERS.items() if v == smoother][0], "nu": nu}
    meth = {"dc": mg.MG_METHOD_DC, "pcg": mg.MG_METHOD_PCG}
    for prec in precisions:
        H = mg.Hierarchy(3, element, n_cells, n_levels, mass=wl["sigma"], smoother=smoother, nu_pre=nu, nu_post=nu,
                         precision=mg.MG_MIXED if prec == "mixed" else mg.MG_FP64)
        for m in methods:
            u = torch.from_numpy(wl["u0"].copy()).cuda()
            H.heat(bFd, wl["g"][:4], u, tol, meth[m])  # warm-up: graphs, clocks
            u.copy_(torch.from_numpy(wl["u0"]))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st, its = H.heat(bFd, wl["g"], u, tol, meth[m])
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
            err = float(np.max(np.abs(u.cpu().numpy() - exact)) / np.max(np.abs(exact)))
            out["%s_%s" % (m, prec)] = {"status": int(st), "wall_s": wall, "ms_per_step": 1e3 * wall / wl["n_steps"],
                                        "dof_steps_per_s": n * wl["n_steps"] / wall,
                                        "vcycles_per_step_mean": float(np.mean(its)),
                                        "vcycles_per_step_max": int(np.max(its)),
                                        "rel_max_error_vs_exact": err}
        if prec == "fp64":  # end to end through the host API
            uh = torch.from_numpy(wl["u0"].copy()).pin_memory()
            bh = torch.from_numpy(bF).pin_memory()
            t0 = time.perf_counter()
            st, its = H.heat_host(bh.numpy(), wl["g"], uh.numpy(), tol, mg.MG_METHOD_DC)
            wall = time.perf_counter() - t0
            out["dc_fp64_host_api"] = {"wall_s": wall, "ms_per_step": 1e3 * wall / wl["n_steps"],
                                       "h2d_bytes": 16 * n, "d2h_bytes": 8 * n}
        H.close()
        del H
        torch.cuda.empty_cache()
    return out


_ORACLE_SOLUTIONS = {}


def oracle_solution_error(name, x_gpu, tol):
    """||x - x_oracle|| / ||x_oracle|| for a GPU solution of workload `name`, the oracle
    solving the same problem (its own matrix and right-hand side) to `tol` in FP64 (once
    per workload)."""
    if (name, tol) not in _ORACLE_SOLUTIONS:
        O, A, b = _oracle_workload(name)
        xo, ho, ito, conv = O.solve(b, tol)
        _ORACLE_SOLUTIONS[(name, tol)] = (xo, int(ito))
        del O, A
    xo, ito = _ORACLE_SOLUTIONS[(name, tol)]
    return float(np.linalg.norm(x_gpu - xo) / np.linalg.norm(xo)), ito


def config_report(name, steps=20, warmup=5, smoother="workload", oracle_error=False):
    """One workload in both precisions: V-cycle throughput, the finest sweep against its
    roofline, and time to 1e-10 (median of 3 solves); with oracle_error, the distance of
    each precision's solution to the oracle's."""
    import torch

    from paper_1609_04809_gb300 import mg
    c = _config_args(name, smoother)
    b = _problem_rhs(c)
    bd = torch.from_numpy(b).cuda()
    out = {"workload": name, "smoother": [k for k, v in SMOOTHERS.items() if v == c["smoother"]][0],
           "n_dofs": int(b.size)}
    peak, _ = _peaks()
    for prec, tag in ((mg.MG_FP64, "fp64"), (mg.MG_MIXED, "mixed")):
        t0 = time.perf_counter()
        H = _hierarchy(c, tag)
        setup_s = time.perf_counter() - t0
        info = H.info()
        Lf = c["n_levels"] - 1
        x = torch.zeros_like(bd)
        H.cycle(bd, x, warmup)
        mg.mg_profile_enable(H.h, True, classes=[mg.MG_K_SMOOTH], levels=[Lf])
        x.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        H.cycle(bd, x, steps)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        k_ms, k_cnt, k_bytes, k_flops = mg.mg_profile_read(H.h, mg.MG_K_SMOOTH, Lf)
        mg.mg_profile_enable(H.h, False)
        ts, its, rel = [], 0, None
        for _ in range(4):
            x.zero_()
            torch.cuda.synchronize()
            s0 = time.perf_counter()
            st, it, hist = H.solve(bd, x, c["tol"])
            ts.append(time.perf_counter() - s0)
            its, rel = it, hist[-1]
        rd = torch.empty_like(bd)
        true_rel = mg.mg_residual_norm_noalloc(H.h, bd, x, rd) / float(np.linalg.norm(b))
        err = oracle_solution_error(name, x.cpu().numpy(), c["tol"]) if oracle_error else None
        pcg = None
        if c["nu_pre"] == c["nu_post"]:
            pts, pits = [], 0
            for rep_i in range(4):
                x.zero_()
                if rep_i == 3:
                    mg.mg_profile_enable(H.h, True, classes=[mg.MG_K_KRYLOV], levels=[Lf])
                torch.cuda.synchronize()
                s0 = time.perf_counter()
                st, pits, ph = H.pcg(bd, x, c["tol"])
                pts.append(time.perf_counter() - s0)
            kk_ms, kk_cnt, kk_bytes, _ = mg.mg_profile_read(H.h, mg.MG_K_KRYLOV, Lf)
            mg.mg_profile_enable(H.h, False)
            ptrue = mg.mg_residual_norm_noalloc(H.h, bd, x, rd) / float(np.linalg.norm(b))
            pcg = {"time_to_tol_ms": 1e3 * float(np.median(pts[1:3])), "iterations": pits,
                   "true_fp64_rel_residual": ptrue,
                   "krylov_kernels_gbs": kk_bytes * kk_cnt / (kk_ms * 1e-3) / 1e9 if kk_cnt else None,
                   "krylov_kernels_us_per_iteration": 1e3 * kk_ms / max(pits, 1) if kk_cnt else None}
        ks = k_ms / k_cnt * 1e-3 if k_cnt else None
        out[tag] = {"dofs_per_s_per_vcycle": b.size / (ms * 1e-3), "ms_per_iteration": ms,
                    "finest_sweep_us": 1e6 * ks if ks else None,
                    "finest_sweep_gbs": k_bytes / ks / 1e9 if ks else None,
                    "finest_sweep_hbm_frac": k_bytes / ks / 1e9 / peak if ks else None,
                    "finest_sweep_fp64_tflops": k_flops / ks / 1e12 if (ks and tag == "fp64") else None,
                    "time_to_tol_ms": 1e3 * float(np.median(ts[1:])), "iterations": its,
                    "final_rel_residual": rel, "true_fp64_rel_residual": true_rel,
                    "storage": [STORAGE_NAMES[v] for v in info["storage"]], "setup_s": setup_s,
                    "device_gb": info["device_bytes"] / 1e9, "tail_levels": info["tail_levels"], "pcg": pcg}
        if err is not None:
            out[tag]["rel_error_vs_oracle"] = err[0]
            out[tag]["oracle_iterations"] = err[1]
        H.close()
        del H
        torch.cuda.empty_cache()
    out["speedup_mixed_vs_fp64"] = out["fp64"]["time_to_tol_ms"] / out["mixed"]["time_to_tol_ms"]
    return out


def run_reference(args):
    """The reference arm: the oracle, as it stands, on all host cores, on the bench's
    workload: setup (not timed), W warm-up and K timed defect-correction iterations."""
    rank = _env_int("RANK", 0)
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    name = args.config
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    O, A, b = _oracle_workload(name, args.smoother, args.cells)
    x = np.zeros(O.n)
    steps, warm = args.steps, min(args.warmup, 3)
    for _ in range(warm):
        x = _oracle_step(O, A, b, x)
    t0 = time.perf_counter()
    for _ in range(steps):
        x = _oracle_step(O, A, b, x)
    dt = time.perf_counter() - t0
    val = O.n * steps / dt
    cpu = _host_cpu()
    sample = ("%d defect-correction iterations (FP64 residual + V-cycle + update) of the %s workload after %d "
              "warm-up iterations, oracle setup excluded; plain FP64 C with its row loops on %d OpenMP threads (%s)"
              % (steps, name, warm, cores, cpu["model"]))
    c = _config_args(name, args.smoother, args.cells)
    out = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": _workload_config(name, c, int(O.n), A.nnz if hasattr(A, "nnz")
                                                            else len(A.val)),
           "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                            "host": cpu},
           "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


def _class_totals(h, kclasses, levels):
    """(ms, launches, bytes per launch, flops per launch) summed over the given levels."""
    from paper_1609_04809_gb300 import mg
    out = {}
    for kc in kclasses:
        tot = [0.0, 0, 0.0, 0.0]
        for l in levels:
            ms, cnt, by, fl = mg.mg_profile_read(h, kc, l)
            tot[0] += ms
            tot[1] += cnt
            if cnt:
                tot[2], tot[3] = by, fl
        out[kc] = tot
    return out


def run_ours(args):
    import torch

    from paper_1609_04809_gb300 import mg
    import __graft_entry__

    world = _env_int("WORLD_SIZE", 1)
    rank = _env_int("RANK", 0)
    local = _env_int("LOCAL_RANK", 0)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    if rank == 0 or world == 1:
        __graft_entry__.build_library()
    if dist:
        dist.barrier()

    name = args.config
    c = _config_args(name, args.smoother, args.cells)
    precision = c["precision"] if args.precision == "workload" else args.precision
    b_host = _problem_rhs(c)
    n = b_host.size
    t0 = time.perf_counter()
    H = _hierarchy(c, precision, args)
    setup_s = time.perf_counter() - t0
    info = H.info()
    Lf = c["n_levels"] - 1
    storage = STORAGE_NAMES[info["storage"][Lf]]
    bd = torch.from_numpy(b_host).cuda()
    xd = torch.zeros_like(bd)
    stream = torch.cuda.current_stream()

    # warm-up steps
    H.cycle(bd, xd, args.warmup)
    torch.cuda.synchronize()
    # the same number of steps without the per-launch events of the timed region below
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    H.cycle(bd, xd, args.steps)
    f1.record(stream)
    torch.cuda.synchronize()
    ms_no_events = f0.elapsed_time(f1) / args.steps
    # an instrumented pass over every launch of 5 steps: per-class device time and the
    # algorithmic bytes of every launch (events around each launch serialise the graph, so
    # these times add up to more than the step; they are reported as shares too). It also
    # names the dominant kernel class of the finest level, the one the timed region below
    # brackets with events.
    mg.mg_profile_enable(H.h, True)
    xk = torch.zeros_like(bd)
    H.cycle(bd, xk, 5)
    inst = _class_totals(H.h, range(mg.MG_K_COUNT), range(c["n_levels"]))
    inst_fin = _class_totals(H.h, [mg.MG_K_OUTER, mg.MG_K_SMOOTH], [Lf])
    step_bytes = 0.0
    for kc in range(mg.MG_K_COUNT):
        for l in range(c["n_levels"]):
            ms_l, cnt_l, by_l, _ = mg.mg_profile_read(H.h, kc, l)
            step_bytes += by_l * cnt_l / 5.0
    mg.mg_profile_enable(H.h, False)
    inst_ms = {mg.KCLASS_NAMES[kc]: inst[kc][0] / 5.0 for kc in inst}
    inst_total = sum(inst_ms.values())
    dom_class = max((mg.MG_K_OUTER, mg.MG_K_SMOOTH), key=lambda kc: inst_fin[kc][0])

    # the timed region: events around each launch of the dominant class only (event nodes
    # break the overlap of the launches they bracket; the step without any is reported too)
    timed_classes = [dom_class]
    mg.mg_profile_enable(H.h, True, classes=timed_classes, levels=[Lf])
    xd.zero_()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        e0.record(stream)
        H.cycle(bd, xd, args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    value, ms_max = replica_throughput(ms, n, args.steps, world, dist, device="cuda")
    ms_step = ms_max / args.steps
    timed = _class_totals(H.h, timed_classes, [Lf])
    mg.mg_profile_enable(H.h, False)
    kernel_ms = {"instrumented": {k: round(v, 4) for k, v in inst_ms.items()},
                 "share": {k: round(v / inst_total, 4) for k, v in inst_ms.items()} if inst_total else None,
                 "scaled_to_step": {k: round(v / inst_total * ms_step, 4) for k, v in inst_ms.items()}
                 if inst_total else None,
                 "note": "instrumented: events around every launch of 5 steps (serialised, so the sum exceeds "
                         "ms_per_step); scaled_to_step: the shares applied to ms_per_step"}
    peak, peak_kind = _peaks()
    fp64_tf, fp64_kind = fp64_peak()
    roofs = {}
    for kc, key in ((mg.MG_K_OUTER, "outer"), (mg.MG_K_SMOOTH, "smooth")):
        live = kc == dom_class
        t_ms, cnt, by, fl = timed[kc] if live else inst_fin[kc]
        r = kernel_roofline(key, precision, storage, name if not args.cells else "%s_cells%d" % (name, c["n_cells"]),
                            n, t_ms, cnt, by, fl, peak, peak_kind, fp64_tf, fp64_kind)
        if r:
            r["ms_per_step"] = t_ms / (args.steps if live else 5)
            r["timing"] = ("events around each launch in the timed region" if live else
                           "events around each launch of the instrumented pass (5 steps)")
            roofs[key] = r
    dominant = "outer" if dom_class == mg.MG_K_OUTER else "smooth"
    if dominant not in roofs:
        dominant = None
    whole = {"bytes_per_step": step_bytes, "achieved": step_bytes / (ms_step * 1e-3) / 1e9, "peak": peak,
             "unit": "GB/s", "frac": step_bytes / (ms_step * 1e-3) / 1e9 / peak,
             "note": "algorithmic bytes of every launch of one step (all levels, the FP64 outer residual and "
                     "the update included) over the timed ms_per_step"}

    out = None
    if rank == 0:
        tol = c["tol"]
        # end to end through the public host API: full solves from pinned host memory
        bh = torch.from_numpy(b_host).pin_memory()
        xh = torch.zeros(n, dtype=torch.float64).pin_memory()
        e2e = None
        if args.e2e_solves > 0:
            mg.mg_solve_host(H.h, bh.numpy(), xh.numpy(), tol)  # warm
            e2e_runs, e2e_iters = [], 0
            for _ in range(args.e2e_solves):
                xh.zero_()
                t0 = time.perf_counter()
                st, it, hist = mg.mg_solve_host(H.h, bh.numpy(), xh.numpy(), tol)
                e2e_runs.append(time.perf_counter() - t0)
                e2e_iters = it
            e2e_t = float(np.median(e2e_runs))
            e2e = {"value": n * e2e_iters / e2e_t, "unit": UNIT, "h2d_bytes_per_step": 16 * n,
                   "d2h_bytes_per_step": 8 * n,
                   "step": "one mg_solve_host call to rel. residual %g (%d V-cycles, %.3f ms)"
                           % (tol, e2e_iters, 1e3 * e2e_t)}

        # time to solution on the same inputs: this precision and the other one, defect
        # correction and CG
        tts = None
        if not args.no_tts:
            def solve_time(h, fn=mg.mg_solve):
                x = torch.zeros_like(bd)
                fn(h.h, bd, x, tol, 200)
                ts = []
                for _ in range(3):
                    x.zero_()
                    torch.cuda.synchronize()
                    s0 = time.perf_counter()
                    st, it, hist = fn(h.h, bd, x, tol, 200)
                    ts.append(time.perf_counter() - s0)
                rd = torch.empty_like(bd)
                true_rel = mg.mg_residual_norm_noalloc(h.h, bd, x, rd) / float(np.linalg.norm(b_host))
                return float(np.median(ts)), it, true_rel
            other = "fp64" if precision == "mixed" else "mixed"
            Ho = _hierarchy(c, other, args)
            res = {}
            for tag, h in ((precision, H), (other, Ho)):
                t_dc, it_dc, r_dc = solve_time(h)
                t_cg, it_cg, r_cg = solve_time(h, mg.mg_pcg) if c["nu_pre"] == c["nu_post"] else (None, None, None)
                res[tag] = {"ms": 1e3 * t_dc, "iters": it_dc, "true_fp64_rel_residual": r_dc,
                            "pcg_ms": 1e3 * t_cg if t_cg else None, "pcg_iters": it_cg,
                            "pcg_true_fp64_rel_residual": r_cg}
            Ho.close()
            del Ho
            torch.cuda.empty_cache()
            tts = {"tol": tol, "fp64": res["fp64"], "mixed": res["mixed"],
                   "speedup_mixed_vs_fp64": res["fp64"]["ms"] / res["mixed"]["ms"],
                   "speedup_mixed_vs_fp64_pcg": (res["fp64"]["pcg_ms"] / res["mixed"]["pcg_ms"]
                                                 if res["mixed"]["pcg_ms"] else None),
                   "method": "defect correction with V-cycles (mg_solve); pcg: CG preconditioned by one V-cycle "
                             "(mg_pcg); true_fp64_rel_residual recomputed in FP64 after the solve"}

        H.close()
        torch.cuda.empty_cache()
        configs = None
        if world == 1 and not args.no_configs:
            configs = {}
            for other_name in ("q1_3d_128_cheb",):
                if other_name != name:
                    configs[other_name] = config_report(other_name)
                    torch.cuda.empty_cache()

        heat = None
        if world == 1 and not args.no_heat:
            heat = heat_report(methods=("dc", "pcg"), precisions=("fp64", "mixed"))

        serving = None
        if world == 1 and args.serve_requests > 0:
            serving = serve_bench(args)

        cpu = None
        if world == 1 and not args.no_cpu:
            res, osetup = cpu_baseline(name, args.cpu_cycles, 1, args.smoother)
            host = _host_cpu()
            va, dta, tha, cya = res["all"]
            v1, dt1, _, cy1 = res["one"]
            cpu = {"value": va, "unit": UNIT, "cores": tha, "kind": "oracle",
                   "sample": "%d defect-correction iterations of the %s workload by the FP64 C oracle with its row "
                             "loops on %d OpenMP threads (%.1f s; oracle setup %.1f s, not timed)"
                             % (cya, name, tha, dta, osetup),
                   "single_core": {"value": v1, "unit": UNIT, "cores": 1,
                                   "sample": "%d iteration on one thread (%.1f s)" % (cy1, dt1)},
                   "host": host}

        clocks = clk.summary()
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None,
               "ms_per_step_no_events": ms_no_events,
               "dtype": "f64" if precision == "fp64" else "f32 V-cycle / f64 outer", "data": "synthetic",
               "config": _workload_config(name, c, n, info["nnz"][Lf]),
               "run": {"precision": precision, "parallelism": "replicas" if world > 1 else "single-gpu",
                       "storage": [STORAGE_NAMES[v] for v in info["storage"]],
                       "smoother": [k for k, v in SMOOTHERS.items() if v == c["smoother"]][0],
                       "setup_s": setup_s,
                       "headline": "the largest single-GPU workload, in the precision it specifies"
                                   if name == DEFAULT_CONFIG else "chosen by --config"},
               "roofline": roofs.get(dominant),
               "roofline_kernels": roofs,
               "whole_cycle": whole,
               "kernel_ms_per_step": kernel_ms,
               "e2e": e2e, "time_to_solution": tts, "cpu_baseline": cpu,
               "gpu_launches": info["kernels_per_cycle"] * args.steps + 1,
               "configs": configs,
               "heat": heat,
               "serving": serving,
               "clocks": clocks}
        print(json.dumps(out))
    else:
        H.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default=DEFAULT_CONFIG, choices=sorted(WORKLOADS))
    ap.add_argument("--cells", type=int, default=None,
                    help="run the workload on another grid (profiling a smaller case; not a bench line)")
    ap.add_argument("--e2e-solves", type=int, default=3)
    ap.add_argument("--cpu-cycles", type=int, default=3)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-tts", action="store_true", help="skip the time-to-solution comparison")
    ap.add_argument("--no-configs", action="store_true", help="skip the nested 128^3 workload")
    ap.add_argument("--no-heat", action="store_true", help="skip the Crank-Nicolson heat workload")
    ap.add_argument("--serve-requests", type=int, default=4096)
    ap.add_argument("--serve-capacity-requests", type=int, default=1024)
    ap.add_argument("--serve-budget-gb", type=float, default=150.0)
    ap.add_argument("--serve-slots", type=int, default=256)
    ap.add_argument("--no-pdl", action="store_true", help="launch without programmatic dependent launch")
    ap.add_argument("--no-tail", action="store_true", help="run the small levels as separate kernels")
    ap.add_argument("--tail", default="auto", choices=["auto", "on", "off"],
                    help="coarse-level tail launch: auto times the V-cycle with and without it at setup "
                         "(pin it under a profiler); --no-tail is --tail off")
    ap.add_argument("--storage", default="auto", choices=sorted(STORAGES),
                    help="level-matrix storage; auto times the candidates at setup (pin it under a profiler, "
                         "whose serialisation would skew that timing)")
    ap.add_argument("--smoother", default="workload", choices=["workload"] + sorted(SMOOTHERS),
                    help="replace the workload's smoother (the headline uses the workload's own)")
    ap.add_argument("--all-configs", action="store_true",
                    help="report every solve workload (FP64 and mixed, with the distance to the oracle's "
                         "solution) instead of the bench line")
    ap.add_argument("--precision", default="workload", choices=["workload", "fp64", "mixed"],
                    help="workload: the precision the workload specifies (headline); fp64 / mixed for analysis")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.all_configs:
        import torch

        import __graft_entry__
        __graft_entry__.build_library()
        torch.cuda.set_device(0)
        from paper_1609_04809_gb300 import workloads as W
        for name in list(W.CONFIGS) + list(W.TET_CONFIGS):
            print(json.dumps(config_report(name, smoother=args.smoother, oracle_error=not args.no_cpu)), flush=True)
            _ORACLE_SOLUTIONS.clear()
        if not args.no_heat:
            print(json.dumps(heat_report()), flush=True)
            # the paper's own configuration: P1 tetrahedra, Gauss-Seidel with three sweeps
            # before and after the coarse correction, six levels, dt = 0.01 to t = 5
            print(json.dumps(heat_report(element=2, smoother=2, nu=3, methods=("dc", "pcg"))), flush=True)
        return 0
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
