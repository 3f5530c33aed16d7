"""Benchmark: implicit cell-updates/s of the radiation / ionization / gas-energy step on GB300.

One bench step = one rhi_implicit_step (g^n, Newton iterations with the fused residual /
Jacobian / Schur kernel, multigrid-preconditioned CG on the Schur system, recovery and
positivity-limited update) over the 256^3 hydrogen + helium lognormal workload (64 lognormal
point sources, T_B = 1e5 K blackbody, 5e12 s steps, Newton tol 1e-8, PCG tol 1e-10).  The
headline form runs the FP32 multigrid preconditioner inside FP64 CG; the plain FP64 form is
timed beside it on the same workload.  Inputs (about 8 GB of fields per form) exceed the
129 MB L2, so no flush is needed between steps.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--n 256]
Under torchrun each rank runs its own replica (independent problem, different seed).
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "implicit cell-updates/s at 256^3 (learned+FP32-MG vs plain FP64), HBM GB/s frac"
UNIT = "cell-updates/s"


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            pk = json.load(fh)
        return pk.get("hbm_gbs", 6800.0), "measured"
    except OSError:
        return 6800.0, "fallback"


# FP64 peak of the CUDA cores derived from the unit counts: 152 SMs x 2070 MHz x 2 DFMA/clk/SM
# x 2 flop = 1.259 TFLOP/s (a register-resident DFMA loop measures 1.20 TFLOP/s)
FP64_PEAK_TFLOPS = 152 * 2.070e9 * 4 / 1e12

# algorithmic DRAM bytes per cell of each kernel (H + He; FP64 fields 8 B): the fields each
# launch must read and write once; stencil neighbours come from cache
ALG_BYTES = {
    "cell_residual_schur": 8 * (5 + 5 + 3 + 3 + 1) + 8 * (1 + 1 + 4 + 4),
    "cell_prep_residual_schur": 8 * (4 + 1 + 3 + 3) + 8 * (5 + 1 + 1 + 4 + 4),
    "faces_limiter": 8 * 2 + 8 * 3,
    "update_recover_limit": 8 * (5 + 1 + 1 + 1 + 4 + 4) + 8 * (5 + 1),
    "cg_matvec_dot": 8 * (1 + 3 + 1) + 8,
    "cg_update_xr": 8 * 4 + 8 * 2,
    "cg_update_p": 8 * 2 + 8,
    "kappa": 8 * 3 + 8,
}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.samples = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None
        sm = [num(s[1]) for s in self.samples if len(s) > 2 and num(s[1]) is not None]
        mx = [num(s[2]) for s in self.samples if len(s) > 2 and num(s[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for s in self.samples:
            for nm, v in zip(names, s[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(self.samples)}


def _oracle_subbox(n, nsrc):
    """A sub-box of the 256^3 recipe (same generator, same cell size) as an oracle problem."""
    from paper_0901_1110_gb300 import inputs
    from oracle import closure as cl, model as md
    w = inputs.config_lognormal(n, nsrc=nsrc, seed=0, box=1.0 * inputs.MPC * n / 256)
    grey = cl.grey_constants(*w.spectrum, w.ns)
    p = md.Problem(nx=n, ny=n, nz=n, dx=w.dx, ns=w.ns, nH=w.nH, grey=grey, y_he=w.y_he,
                   src=cl.deposit_sources(w.nH.shape, w.dx, w.src_ijk, w.src_rate, grey["eps"]),
                   theta=w.theta, u_e=w.u_e, u_n=w.u_n, u_E=w.u_E)
    return w, p


def reference_arm(args, rank, world):
    """The FP64 CPU oracle on a bounded sample of the same workload (implicit steps of a
    sub-box drawn by the same generator), timed on this host's cores."""
    if rank != 0:
        return
    from oracle import solve as sv
    n = int(os.environ.get("RHI_REF_SAMPLE_N", "48"))
    w, p = _oracle_subbox(n, 1)
    st = w.state()
    times = []
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        st, _ = sv.implicit_step(p, st, w.dt, 1.0, 0.0, w.newton_tol, linear="schur_cg")
        if k >= args.warmup:
            times.append(time.perf_counter() - t0)
    tot = sum(times)
    val = w.N * len(times) / tot
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"lognormal_hhe {n}^3 sub-box of the 256^3 recipe",
                       "form": "oracle (numpy/scipy FP64, Schur + plain CG)"},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": host_cores(), "kind": "oracle",
                             "sample": f"{args.steps} implicit steps of a {n}^3 sub-box "
                                       "(same generator, 1 Mpc/256 cells)"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count()


def cpu_baseline_sample():
    """Oracle on a bounded sample: 3 implicit steps of a 48^3 sub-box (same recipe)."""
    from oracle import solve as sv
    n, steps = 48, 3
    w, p = _oracle_subbox(n, 1)
    st = w.state()
    t0 = time.perf_counter()
    for _ in range(steps):
        st, _ = sv.implicit_step(p, st, w.dt, 1.0, 0.0, w.newton_tol, linear="schur_cg")
    dt = time.perf_counter() - t0
    return {"value": w.N * steps / dt, "unit": UNIT, "cores": host_cores(), "kind": "oracle",
            "sample": f"{steps} implicit steps of a {n}^3 sub-box of the 256^3 recipe "
                      "(numpy/scipy; BLAS threads over the host cores)"}


def run_form(rhi, w, torch, steps, warmup, precond, profile, limiter_jacobian=0,
             max_newton=200):
    """Times `steps` implicit steps after `warmup` with CUDA events on the library's stream."""
    stream = torch.cuda.Stream()
    s = rhi.solver_for_workload(w, stream=stream.cuda_stream, precond=precond, mg_levels=6,
                                theta=1.0, limiter_jacobian=limiter_jacobian,
                                max_newton=max_newton)
    for _ in range(warmup):
        rc = s.step(w.dt, 1.0, 0.0, w.newton_tol, w.lin_tol, check=False)
        if rc:
            st = s.stats()
            raise RuntimeError(f"warm-up step failed ({rc}): newton_its={st['newton_its']} "
                               f"residuals={st['res_history']}")
    s.set_profiling(profile)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    agg = dict(newton_its=0, pcg_its=0, vcycles=0, launches=0, backtracks=0)
    e0.record(stream)
    hist = []
    for _ in range(steps):
        s.step(w.dt, 1.0, 0.0, w.newton_tol, w.lin_tol)
        st = s.stats()
        for k in agg:
            agg[k] += st[k]
        hist.append(st["res_history"])
    agg["res_history_last"] = hist[-1]
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    kt = s.kernel_times() if profile else {}
    s.set_profiling(False)
    return s, ms, agg, kt


def e2e_form(rhi, w, torch, steps, warmup, precond, limiter_jacobian=0, max_newton=200):
    """Same metric through the public API with host buffers: each timed step copies the
    step's inputs (E, e, n, n_H and the point-source list) from pinned host memory, runs the
    step and reads the state (E, e, n) back into pinned host memory."""
    s = rhi.solver_for_workload(w, precond=precond, mg_levels=6, theta=1.0,
                                limiter_jacobian=limiter_jacobian, max_newton=max_newton)
    N = w.N
    pin = lambda m: torch.empty(m, dtype=torch.float64, pin_memory=True).numpy()
    st = w.state()
    E, e, n, nH = pin(N), pin(N), pin(w.ns * N), pin(N)
    E[:] = st["E"]; e[:] = st["e"]; n[:] = st["n"].ravel(); nH[:] = w.nH.ravel()
    oE, oe, on = pin(N), pin(N), pin(w.ns * N)
    # the same step indices as the device-timed region: warm-up steps first, untimed
    for _ in range(warmup):
        s.step(w.dt, 1.0, 0.0, w.newton_tol, w.lin_tol)
    s.get_state(E, e, n)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        s.set_state(E, e, n, nH, None)
        s.set_sources(w.src_ijk, w.src_rate)
        s.step(w.dt, 1.0, 0.0, w.newton_tol, w.lin_tol)
        s.get_state(oE, oe, on)
        E, oE = oE, E
        e, oe = oe, e
        n, on = on, n
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    s.close()
    h2d = 8 * N * (3 + w.ns) + 20 * len(w.src_rate)
    d2h = 8 * N * (2 + w.ns)
    return N * steps / dt, h2d, d2h


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="rhi")
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--forms", default="plain_fp64,mixed_fp32mg",
                    help="comma list of forms to time (the last one is the headline)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--max-newton", type=int, default=200)
    ap.add_argument("--limiter-jacobian", type=int, default=0,
                    help="1: keep dD/dE in the Newton matrix (BiCGStab)")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", str(args.gpus)))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return reference_arm(args, rank, world)

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    from paper_0901_1110_gb300 import _build
    if rank == 0:
        _build.build()
    if dist:
        dist.barrier()
    import paper_0901_1110_gb300 as rhi
    from paper_0901_1110_gb300 import inputs

    n = args.n
    nsrc = max(1, round(64 * (n / 256) ** 3))
    w = inputs.config_lognormal(n, nsrc=nsrc, seed=rank)
    hbm_peak, peak_src = load_peaks()

    # plain FP64 form (FP64 multigrid), then the mixed form (FP32 multigrid) as headline
    forms = {}
    codes = {"plain_fp64": rhi.RHI_PRECOND_MG_FP64, "mixed_fp32mg": rhi.RHI_PRECOND_MG_FP32}
    ljac = {"plain_fp64": args.limiter_jacobian, "mixed_fp32mg": args.limiter_jacobian}
    order = [f for f in args.forms.split(",") if f]
    for name in order:
        pc = codes[name]
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        clk = ClockSampler(local)
        clk.start()
        s, ms, agg, kt = run_form(rhi, w, torch, args.steps, args.warmup, pc, profile=True,
                                  limiter_jacobian=ljac[name], max_newton=args.max_newton)
        clocks = clk.stop()
        t = torch.tensor([ms], device="cuda", dtype=torch.float64)
        if dist:
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
        forms[name] = dict(ms=float(t.item()), agg=agg, kt=kt, clocks=clocks)
        s.close()
        del s
        torch.cuda.empty_cache()

    head = forms[order[-1]]
    ms_step = head["ms"] / args.steps
    value = world * w.N * args.steps / (head["ms"] * 1e-3)

    # dominant kernel and its roofline
    kt = head["kt"]
    tot = sum(v[0] for v in kt.values())
    tname, (tms, tcnt) = max(kt.items(), key=lambda kv: kv[1][0])
    avg_s = tms / tcnt * 1e-3
    roof = {"kernel": tname, "share": tms / tot if tot else None, "avg_launch_ms": avg_s * 1e3}
    if tname in ALG_BYTES:
        ach = ALG_BYTES[tname] * w.N / avg_s / 1e9
        roof.update(bound="hbm", achieved=ach, peak=hbm_peak, unit="GB/s", frac=ach / hbm_peak,
                    traffic=None, peak_source=peak_src)
    # HBM fraction of the FP64 CG stencil / vector kernels (one full-grid launch each)
    lin = {}
    for k in ("cg_matvec_dot", "cg_update_xr", "cg_update_p"):
        if k in kt:
            ms_k, c_k = kt[k]
            lin[k] = ALG_BYTES[k] * w.N / (ms_k / c_k * 1e-3) / 1e9 / hbm_peak

    plain = forms.get("plain_fp64", head)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"lognormal_hhe {n}^3 H+He, sigma_ln=1, P(k)~k^-2, {nsrc} sources "
                               "(median 1e49/s), T_B=1e5 K, dt=5e12 s, theta=1, Newton tol "
                               "1e-8 (u_E = 1e-16), PCG tol 1e-10",
                   "form": "FP64 Newton/Schur/CG + FP32 multigrid V-cycle (6 levels, 2+2 "
                           "Jacobi, 16 coarse sweeps)",
                   "parallelism": "replicas" if world > 1 else "1 GPU",
                   "l2": "inputs larger than L2 (~8 GB of fields per form)"},
        "roofline": roof,
        "plain_fp64": {"value": world * w.N * args.steps / (plain["ms"] * 1e-3),
                       "ms_per_step": plain["ms"] / args.steps,
                       **{k: v / args.steps for k, v in plain["agg"].items()
                          if k != "res_history_last"}},
        "iterations_per_step": {k: v / args.steps for k, v in head["agg"].items()
                                if k != "res_history_last"},
        "newton_residuals_last_step": head["agg"]["res_history_last"],
        "gpu_launches": head["agg"]["launches"],
        "clocks": head["clocks"],
        "kernel_ms_per_step": {k: v[0] / args.steps
                               for k, v in sorted(kt.items(), key=lambda kv: -kv[1][0])},
        "plain_kernel_ms_per_step": {k: v[0] / args.steps
                                     for k, v in sorted(plain["kt"].items(),
                                                        key=lambda kv: -kv[1][0])},
        "hbm_frac_linear_kernels": lin,
    }
    if rank == 0:
        if not args.no_e2e:
            e2e_val, h2d, d2h = e2e_form(rhi, w, torch, args.steps, args.warmup,
                                         codes[order[-1]], ljac[order[-1]], args.max_newton)
            line["e2e"] = {"value": world * e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d,
                           "d2h_bytes_per_step": d2h}
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline_sample()
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
