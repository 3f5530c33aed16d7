"""Benchmark: implicit cell-updates/s of the radiation / ionization / gas-energy step on GB300.

One bench step = one rhi_implicit_step: g^n, Newton iterations with the fused residual /
Jacobian / Schur kernel, the Schur system solved by BiCGStab (exact Newton matrix, the default;
CG with D lagged) preconditioned by a multigrid V-cycle of that matrix, recovery and the
positivity-limited update, over the 256^3 hydrogen + helium lognormal workload (64 lognormal
point sources, T_B = 1e5 K blackbody, 5e12 s steps, Newton tol 1e-8, Krylov tol 1e-10).  Three
forms run on the same workload: plain FP64 (FP64 multigrid), mixed (FP32 multigrid inside the
FP64 Krylov solve) and, as the headline, learned + mixed (the mixed form started from the
learned Newton guess, trained on the GPU beforehand from a 128^3 run at the same cell size;
training time is reported, not timed).  The fields (about 12 GB per form) exceed the 129 MB
L2, so no flush is needed between steps.

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


def workload_sources(n):
    """Point sources of the n^3 lognormal workload: 64 at 256^3, the same density otherwise."""
    return max(1, round(64 * (n / 256) ** 3))


def workload_text(n):
    """The timed workload as the JSON line names it (both arms)."""
    return (f"lognormal_hhe {n}^3 H+He, sigma_ln=1, P(k)~k^-2, {workload_sources(n)} sources "
            "(median 1e49/s), T_B=1e5 K, dt=5e12 s, theta=1, Newton tol 1e-8 (u_E = 1e-16), "
            "Krylov tol 1e-10 relative to ||f||")


def max_over_ranks(x, dist, device):
    """The largest x over the ranks of the process group (x itself without one)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(world, cells, steps, ms):
    """Whole-job cell-updates/s of world replicas of `cells` cells each, every rank having
    taken `steps` steps within the slowest rank's `ms` milliseconds."""
    return world * cells * steps / (ms * 1e-3)


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

# FP64 flops per cell of the fused cell kernels (bound by the FP64 pipe, about 1.2 TFLOP/s here),
# counted by ncu as 2 DFMA + DMUL + DADD thread instructions per cell (175, 106, 76 on the
# H + He lognormal 128^3 case)
ALU_FLOPS = {
    "cell_residual_schur": 532,
}
# DRAM bytes per launch (read + write) from ncu, per cell of a capture times the cells of the
# timed grid (each of these kernels streams its fields once, so traffic grows with the cells);
# an entry is removed when its kernel changes.  k_cell<3,1> at 128^3: 368.94 MB read +
# 151.53 MB written per launch (ncu --set full, the current kernel).
TRAFFIC_PER_CELL = {"cell_residual_schur": (368.936192e6 + 151.531520e6) / 128 ** 3}

FORM_TEXT = {
    "plain_fp64": "FP64 Newton/Schur/BiCGStab + FP64 multigrid V-cycle of the Newton matrix "
                  "(6 levels, 2+2 Jacobi, 16 coarse sweeps), BiCGStab restarted only on "
                  "stagnation, Newton from U^n",
    "mixed_fp32mg": "FP64 Newton/Schur/BiCGStab + FP32 multigrid V-cycle of the Newton matrix "
                    "(6 levels, 2+2 Jacobi, 16 coarse sweeps), BiCGStab restarted at each 100x "
                    "residual reduction, Newton from U^n",
    "learned_mixed": "mixed form + learned Newton guess (BF16 tensor-core MLP, falls back to U^n "
                     "when its ||f|| is larger)",
}
NEWTON_TEXT = {0: "Newton matrix with D lagged (symmetric Schur matrix, CG)",
               1: "Newton matrix with dD/dE kept (BiCGStab)",
               2: "exact Newton matrix: dD/dE and D's opacity dependence kept (BiCGStab)"}


def alg_bytes(nonsym):
    """Algorithmic DRAM bytes per cell of each kernel (H + He; FP64 fields 8 B, FP32 4 B): the
    fields each launch must read and write once; stencil neighbours come from cache.  nonsym:
    the multigrid levels carry both couplings of each face (the Newton matrix that keeps
    dD/dE), 6 face arrays instead of 3."""
    f = 6 if nonsym else 3
    return {
        "cell_residual_schur": 8 * (5 + 5 + 3 + 3 + 1) + 8 * (1 + 1 + 4 + 4),
        "cell_prep_residual_schur": 8 * (4 + 1 + 3 + 3) + 8 * (5 + 1 + 1 + 4 + 4),
        "faces_limiter": 8 * 2 + 8 * 3,
        # a trial iterate the Newton loop expects to converge: W alone, then f alone
        "faces_w": 8 * 2 + 8 * 3,
        "cell_residual": 8 * (5 + 5 + 3 + 3 + 1),
        "update_recover_limit": 8 * (5 + 1 + 1 + 1 + 4 + 4) + 8 * (5 + 1),
        "cg_matvec_dot": 8 * (1 + 3 + 1) + 8,
        "cg_update_xr": 8 * 4 + 8 * 2,
        "cg_update_p": 8 * 2 + 8,
        # BiCGStab (exact Newton matrix): y = A x reads x, diag, P and Q of 3 faces, the dot's
        # vector; writes y
        "bicg_matvec": 8 * (1 + 1 + 3 + 3 + 1) + 8,
        "bicg_update_xr": 8 * 6 + 8 * 2,
        "bicg_update_p": 8 * 3 + 8,
        "bicg_update_s": 8 * 2 + 8,
        "kappa": 8 * 3 + 8,
        # weighted-Jacobi sweep on the finest level: x, b, omega / diag and the face arrays
        # read, x written; the first sweep of a cycle starts from x = 0: b, omega / diag read
        "mg_smooth_f32_fine": 4 * (3 + f) + 4,
        "mg_smooth_f32_fine_first": 4 * 2 + 4,
        "mg_smooth_f64_fine": 8 * (3 + f) + 8,
        "mg_smooth_f64_fine_first": 8 * 2 + 8,
        # residual restriction from the finest level: b, x, diag and the face arrays of each
        # fine cell read, one coarse value per 8 fine cells written
        "mg_restrict_f32_fine": 4 * (3 + f) + 4 / 8,
        "mg_restrict_f64_fine": 8 * (3 + f) + 8 / 8,
        # prolongation to the finest level: the parent's correction (one per 8 cells) read, x
        # read and written
        "mg_prolong_f32_fine": 4 / 8 + 4 + 4,
        "mg_prolong_f64_fine": 8 / 8 + 8 + 8,
        # FP64 Krylov vector to the FP32 right-hand side, and the FP32 result back to FP64
        "mg_to_f32": 8 + 4,
        "mg_from_f32": 4 + 8,
        "mg_from_f32_dot": 4 + 8 + 8,
    }


# the stencil / vector kernels of the Krylov solver and the multigrid preconditioner whose HBM
# fraction is reported per form
LINEAR_KERNELS = ("cg_matvec_dot", "cg_update_xr", "cg_update_p", "bicg_matvec",
                  "bicg_update_xr", "bicg_update_p", "bicg_update_s", "mg_smooth_f32_fine",
                  "mg_smooth_f32_fine_first", "mg_smooth_f64_fine", "mg_smooth_f64_fine_first",
                  "mg_restrict_f32_fine", "mg_restrict_f64_fine", "mg_prolong_f32_fine",
                  "mg_prolong_f64_fine", "mg_to_f32", "mg_from_f32", "mg_from_f32_dot")


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


def _oracle_subbox(n, nsrc, **overrides):
    """A sub-box of the 256^3 recipe (same generator, same cell size) as an oracle problem."""
    from paper_0901_1110_gb300 import inputs
    from oracle import closure as cl, model as md
    w = inputs.config_lognormal(n, nsrc=nsrc, seed=0, box=1.0 * inputs.MPC * n / 256)
    grey = cl.grey_constants(*w.spectrum, w.ns)
    p = md.Problem(nx=n, ny=n, nz=n, dx=w.dx, ns=w.ns, nH=w.nH, grey=grey, y_he=w.y_he,
                   src=cl.deposit_sources(w.nH.shape, w.dx, w.src_ijk, w.src_rate, grey["eps"]),
                   theta=w.theta, u_e=w.u_e, u_n=w.u_n, u_E=w.u_E, **overrides)
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
            "config": {"workload": workload_text(args.n),
                       "form": "oracle (numpy/scipy FP64, Schur + plain CG), each step on a "
                               f"{n}^3 sub-box of that workload"},
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


def cpu_baseline_sample(n=48, steps=3):
    """Oracle on a bounded sample: 3 implicit steps of a 48^3 sub-box (same recipe), timed.
    Untimed afterwards, the oracle's states of the same steps converged to 1e-14 (exact
    Newton matrix, Schur complement and BiCGStab to 1e-14), against which the GPU forms'
    per-element errors are reported."""
    from oracle import solve as sv
    w, p = _oracle_subbox(n, 1)
    st = w.state()
    t0 = time.perf_counter()
    for _ in range(steps):
        st, _ = sv.implicit_step(p, st, w.dt, 1.0, 0.0, w.newton_tol, linear="schur_cg")
    dt = time.perf_counter() - t0
    base = {"value": w.N * steps / dt, "unit": UNIT, "cores": host_cores(), "kind": "oracle",
            "sample": f"{steps} implicit steps of a {n}^3 sub-box of the 256^3 recipe "
                      "(numpy/scipy; BLAS threads over the host cores)"}
    _, pe = _oracle_subbox(n, 1, limiter_jacobian="exact")
    ref, refs = w.state(), []
    for _ in range(steps):
        ref, _ = sv.implicit_step(pe, ref, w.dt, 1.0, 0.0, 1e-14, linear="schur_cg")
        refs.append(ref)
    return base, (w, refs)


def _per_element(got, ref, nH, y_he):
    """max over cells of |got - ref| / (|ref| + 1e-12 max|ref|) for E, e and the species
    fractions x_HI, x_HII, x_HeI, x_HeII, x_HeIII."""
    def rel(a, b, ulps=0.0):
        a, b = np.asarray(a).ravel(), np.asarray(b).ravel()
        d = np.maximum(np.abs(a - b) - ulps * 2.0 ** -52, 0.0)
        return float((d / (np.abs(b) + 1e-12 * np.abs(b).max())).max())

    def fr(n):
        n = np.asarray(n).reshape(3, -1)
        nHe = y_he * nH
        return {"x_HI": n[0] / nH, "x_HII": (nH - n[0]) / nH, "x_HeI": n[1] / nHe,
                "x_HeII": n[2] / nHe, "x_HeIII": (nHe - n[1] - n[2]) / nHe}

    out = {"E": rel(got["E"], ref["E"]), "e": rel(got["e"], ref["e"])}
    fg, fo = fr(got["n"]), fr(ref["n"])
    # derived fractions (formed by subtraction from the element total) net of 4 units of 2^-52
    out.update({k: rel(fg[k], fo[k], 4.0 if k in ("x_HII", "x_HeIII") else 0.0) for k in fo})
    return out


def error_vs_oracle(rhi, forms, w, refs, limiter_jacobian, weights):
    """Per-element error of each GPU form after each of the oracle's steps of the sub-box, run
    with the timed run's settings (tolerances, Newton matrix, 6 multigrid levels); the worst
    over the steps per field."""
    out = {}
    nH = w.nH.ravel()
    for name, (pc, guess) in forms.items():
        s = rhi.solver_for_workload(w, precond=pc, mg_levels=6, theta=1.0,
                                    limiter_jacobian=limiter_jacobian, max_newton=200,
                                    guess=guess)
        if guess == rhi.RHI_GUESS_LEARNED:
            s.mlp_set_weights(weights)
        worst, scaled = {}, {}
        for ref in refs:
            s.step(w.dt, 1.0, 0.0, w.newton_tol, w.lin_tol)
            got = s.get_state()
            for k, v in _per_element(got, ref, nH, w.y_he).items():
                worst[k] = max(worst.get(k, 0.0), v)
            # distance in the scaled unknowns whose RMS residual Newton stops on
            for k, u in (("E", w.u_E), ("e", w.u_e)):
                v = float(np.abs(np.asarray(got[k]).ravel() - np.asarray(ref[k]).ravel()).max() / u)
                scaled[k] = max(scaled.get(k, 0.0), v)
            dn = (np.asarray(got["n"]).reshape(3, -1) - np.asarray(ref["n"]).reshape(3, -1)) / w.u_n
            scaled["n"] = max(scaled.get("n", 0.0), float(np.abs(dn).max()))
            # the RMS of the scaled distance over all N (N_s + 2) unknowns, which the Newton
            # tolerance bounds (the largest element may reach sqrt(N (N_s + 2)) times that)
            parts = [(np.asarray(got["E"]).ravel() - np.asarray(ref["E"]).ravel()) / w.u_E,
                     (np.asarray(got["e"]).ravel() - np.asarray(ref["e"]).ravel()) / w.u_e, dn.ravel()]
            rms = float(np.sqrt(np.mean(np.concatenate(parts) ** 2)))
            scaled["rms"] = max(scaled.get("rms", 0.0), rms)
        s.close()
        out[name] = {"per_element": worst, "scaled": scaled}
    return out


def dominant_kernel(kt, ab):
    """The kernel with the largest share of the profiled step among those with a byte or flop
    model (graph wrappers excluded)."""
    cands = {k: v for k, v in kt.items() if k in ab or k in ALU_FLOPS}
    return max(cands.items(), key=lambda kv: kv[1][0])[0] if cands else None


def run_form(rhi, w, torch, steps, warmup, precond, ab, limiter_jacobian=0, max_newton=200,
             guess=0, weights=None):
    """Times `steps` implicit steps after `warmup` with CUDA events on the library's stream.
    The last warm-up step brackets every launch with events (the per-kernel breakdown; the
    Krylov solve then runs as direct launches); it names the dominant kernel, and inside the
    timed region only that kernel's launches are bracketed (their mean device time gives the
    roofline).  The Krylov solve runs as a CUDA graph unless that kernel is one of its own."""
    stream = torch.cuda.Stream()
    s = rhi.solver_for_workload(w, stream=stream.cuda_stream, precond=precond, mg_levels=6,
                                theta=1.0, limiter_jacobian=limiter_jacobian,
                                max_newton=max_newton, guess=guess)
    if weights is not None:
        s.mlp_set_weights(weights)
    for k in range(warmup):
        if k == warmup - 1:
            s.set_profiling(True)
        rc = s.step(w.dt, 1.0, 0.0, w.newton_tol, w.lin_tol, check=False)
        if rc:
            st = s.stats()
            raise RuntimeError(f"warm-up step failed ({rc}): newton_its={st['newton_its']} "
                               f"residuals={st['res_history']}")
    kt_all = s.kernel_times()
    tname = dominant_kernel(kt_all, ab)
    s.set_profiling(True, names=[tname] if tname else None)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    agg = dict(newton_its=0, pcg_its=0, vcycles=0, launches=0, backtracks=0, learned_used=0,
               guess_restarts=0, host_syncs=0, krylov_fallbacks=0, krylov_stalls=0,
               final_predicted=0, final_missed=0)
    e0.record(stream)
    hist, res0, prev0 = [], [], []
    agg["newton_per_step"], agg["krylov_per_step"] = [], []
    for _ in range(steps):
        s.step(w.dt, 1.0, 0.0, w.newton_tol, w.lin_tol)
        st = s.stats()
        agg["newton_per_step"].append(st["newton_its"])
        agg["krylov_per_step"].append(st["pcg_its"])
        for k in agg:
            if k in st:
                agg[k] += st[k]
        agg["learned_used"] += int(st["guess_used"] == rhi.RHI_GUESS_LEARNED)
        hist.append(st["res_history"])
        res0.append(st["res_initial"])
        prev0.append(st["res_guess_prev"])
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    kt_timed = s.kernel_times()
    s.set_profiling(False)
    agg["res_history_last"] = hist[-1]
    agg["res_initial"] = res0
    agg["res_prev_guess"] = prev0
    return s, ms, agg, kt_timed, kt_all, tname


def config_128_plain(rhi, torch, limiter_jacobian, max_newton):
    """The 128^3 plain FP64 configuration as specified: H + He lognormal medium, 16 sources,
    20 steps of 5e12 s from the initial state, FP64 multigrid; device time of the 20 steps and
    the Newton and Krylov counts per step."""
    from paper_0901_1110_gb300 import inputs
    w = inputs.config_lognormal(128, nsrc=16, seed=0)
    stream = torch.cuda.Stream()
    s = rhi.solver_for_workload(w, stream=stream.cuda_stream, precond=rhi.RHI_PRECOND_MG_FP64,
                                mg_levels=6, theta=1.0, limiter_jacobian=limiter_jacobian,
                                max_newton=max_newton)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    its = []
    for _ in range(w.nsteps):
        s.step(w.dt, 1.0, 0.0, w.newton_tol, w.lin_tol)
        st = s.stats()
        its.append((st["newton_its"], st["pcg_its"], st["vcycles"]))
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    s.close()
    a = np.asarray(its, dtype=np.float64)
    return {"workload": "lognormal_hhe 128^3 H+He, 16 sources, 20 steps of 5e12 s from the "
                        "initial state, plain FP64 (FP64 multigrid)",
            "value": w.N * w.nsteps / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / w.nsteps,
            "newton_its_per_step": float(a[:, 0].mean()),
            "krylov_its_per_step": float(a[:, 1].mean()),
            "vcycles_per_step": float(a[:, 2].mean()),
            "newton_its": a[:, 0].astype(int).tolist(), "krylov_its": a[:, 1].astype(int).tolist()}


def config_cosmo_run(rhi, torch, n, intervals, max_newton, budget_s=600.0):
    """The cosmological configuration (H + He, sigma_ln = 1.5, 256 clustered sources at 512^3,
    flat Lambda-CDM from z = 10 in 100 equal intervals of cosmic time) over its first
    `intervals` intervals, each with (a, adot) at its middle.  The plain FP64 form takes
    adaptive implicit steps inside each interval (eqs. time_error_estimator and
    time_step_selection with p = 2, tau_tol = 0.05; a failed step is retried at half its
    length), Newton tol 1e-8; the mixed form then takes the same steps, so that the two final
    states differ only by the forms' arithmetic, and is compared with the plain form per
    element and in the scaled unknowns.  The plain form stops after the interval in which its
    wall time passes budget_s; each finished interval is reported on stderr."""
    from paper_0901_1110_gb300 import inputs
    w = inputs.config_cosmo(n, nsrc=max(1, round(256 * (n / 512) ** 3)))
    out, states, seq = {}, {}, []
    for name, pc in (("plain_fp64", rhi.RHI_PRECOND_MG_FP64), ("mixed_fp32mg", rhi.RHI_PRECOND_MG_FP32)):
        stream = torch.cuda.Stream()
        s = rhi.solver_for_workload(w, stream=stream.cuda_stream, precond=pc, mg_levels=6,
                                    theta=1.0, limiter_jacobian=2, max_newton=max_newton,
                                    dt_norm=2, dt_tau_tol=0.05)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        stats, failed = [], 0
        if name == "plain_fp64":
            dt = 1e11
            t_wall = time.perf_counter()
            done = 0
            for k in range(intervals):
                if time.perf_counter() - t_wall > budget_s:
                    break
                span, a, adot = w.schedule[k]
                t = 0.0
                while t < span * (1.0 - 1e-12) and time.perf_counter() - t_wall <= 2.0 * budget_s:
                    d = min(dt, span - t)
                    rc = s.step(d, a, adot, w.newton_tol, w.lin_tol, check=False)
                    while rc in (rhi.RHI_ERR_NONCONVERGED, rhi.RHI_ERR_NONPHYSICAL) and d > 1e6:
                        st = s.stats()
                        print(f"  step of {d:.3e} s failed ({rc}) after {st['newton_its']} Newton "
                              f"iterations, ||f|| {st['res_final']:.2e}, {st['ms']:.0f} ms",
                              file=sys.stderr, flush=True)
                        failed += 1
                        d *= 0.5
                        rc = s.step(d, a, adot, w.newton_tol, w.lin_tol, check=False)
                    if rc:
                        raise RuntimeError(f"cosmological step failed at dt = {d:.3e} ({rc})")
                    st = s.stats()
                    stats.append(st)
                    seq.append((d, a, adot))
                    print(f"  step {len(stats)}: dt {d:.3e} s, {st['newton_its']} Newton, "
                          f"{st['pcg_its']} BiCGStab, {st['ms']:.0f} ms", file=sys.stderr, flush=True)
                    t += d
                    dt = max(st["dt_next"], 1e6)
                if t < span * (1.0 - 1e-12):
                    break                       # the time budget ended inside this interval
                done = k + 1
                print(f"cosmological interval {done}: {len(stats)} steps, "
                      f"{time.perf_counter() - t_wall:.1f} s", file=sys.stderr, flush=True)
            intervals = done
        else:
            for d, a, adot in seq:
                rc = s.step(d, a, adot, w.newton_tol, w.lin_tol, check=False)
                if rc:
                    raise RuntimeError(f"mixed form failed the plain form's step dt = {d:.3e} ({rc})")
                stats.append(s.stats())
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        states[name] = s.get_state()
        s.close()
        del s
        torch.cuda.empty_cache()
        steps = len(stats)
        out[name] = {"implicit_steps": steps, "failed_steps_retried": failed, "ms": ms,
                     "value": w.N * steps / (ms * 1e-3), "unit": UNIT,
                     "dt_per_step": [round(x[0], -6) for x in seq],
                     "newton_per_step": [st["newton_its"] for st in stats],
                     "krylov_per_step": [st["pcg_its"] for st in stats],
                     "krylov_stalls": sum(st["krylov_stalls"] for st in stats),
                     "krylov_fallbacks": sum(st["krylov_fallbacks"] for st in stats),
                     "step_ms": [round(st["ms"], 1) for st in stats]}
    a_end = float(inputs.flat_lcdm_a(inputs.flat_lcdm_t(1.0 / 11.0) + intervals * w.dt))
    nH = w.nH.ravel()
    out["mixed_vs_plain"] = {
        "per_element": _per_element(states["mixed_fp32mg"], states["plain_fp64"], nH, w.y_he),
        "scaled": {k: float(np.abs(np.asarray(states["mixed_fp32mg"][k]).ravel()
                                   - np.asarray(states["plain_fp64"][k]).ravel()).max() / u)
                   for k, u in (("E", w.u_E), ("e", w.u_e))}}
    out["workload"] = (f"cosmological configuration {n}^3, {len(w.src_rate)} clustered sources, "
                       f"sigma_ln 1.5, first {intervals} of 100 intervals from z = 10 "
                       f"(to z = {1.0 / a_end - 1.0:.3f}), adaptive steps (p = 2, tau_tol 0.05) "
                       "of the plain form, replayed by the mixed form; Newton tol 1e-8")
    return out


def train_guess(rhi, torch, rank, train_steps, epochs):
    """Trains the learned guess on the GPU from Newton solutions of a 128^3 lognormal run at
    the timed workload's cell size and source density (a 0.5 Mpc box with 8 sources, a seed
    distinct from the timed workload's), mixed form, exact Newton matrix."""
    from paper_0901_1110_gb300 import inputs
    t0 = time.perf_counter()
    w = inputs.config_lognormal(128, nsrc=workload_sources(128), seed=1000 + rank,
                                box=inputs.MPC * 128 / 256)
    s = rhi.solver_for_workload(w, precond=rhi.RHI_PRECOND_MG_FP32, mg_levels=6, theta=1.0,
                                max_newton=200, limiter_jacobian=2)
    N = w.N
    X = torch.empty((train_steps * N, rhi.RHI_MLP_IN), dtype=torch.float32, device="cuda")
    Y = torch.empty((train_steps * N, rhi.RHI_MLP_OUT), dtype=torch.float32, device="cuda")
    old = {k: torch.empty(m * N, dtype=torch.float64, device="cuda")
           for k, m in (("E", 1), ("e", 1), ("n", w.ns))}
    for k in range(train_steps):
        s.get_state(old["E"], old["e"], old["n"])
        s.mlp_features(w.dt, out=X[k * N:(k + 1) * N])
        s.step(w.dt, 1.0, 0.0, w.newton_tol, w.lin_tol)
        s.mlp_targets(old, out=Y[k * N:(k + 1) * N])
    t_data = time.perf_counter() - t0
    g = torch.Generator(device="cuda")
    g.manual_seed(0)
    perm = torch.randperm(X.shape[0], device="cuda", generator=g)
    X = X[perm].contiguous()
    Y = Y[perm].contiguous()
    mean = X.mean(dim=0)
    sd = X.std(dim=0)
    sd = torch.where(sd > 1e-3, sd, torch.ones_like(sd))
    w0 = init_weights(rhi, mean.cpu().numpy(), sd.cpu().numpy())
    s.mlp_set_weights(w0)
    losses = []
    for ep in range(epochs):
        lr = 2e-3 if ep < epochs - 1 else 5e-4
        losses.append(s.mlp_train(X, Y, epochs=1, batch=4096, lr=lr))
    torch.cuda.synchronize()
    wts = s.mlp_get_weights()
    s.close()
    info = {"samples": int(X.shape[0]), "epochs": epochs, "loss_per_epoch": losses,
            "data_s": t_data, "total_s": time.perf_counter() - t0,
            "source": f"{train_steps} steps of lognormal_hhe 128^3, {workload_sources(128)} "
                      f"sources, 0.5 Mpc (the timed run's cell size), seed {1000 + rank}"}
    return wts, info


def init_weights(rhi, mean, scale, seed=0):
    """He-initialised weights in the library's layout with the given input normalisation."""
    rng = np.random.default_rng(seed)
    I, H, O = rhi.RHI_MLP_IN, rhi.RHI_MLP_HID, rhi.RHI_MLP_OUT
    parts = []
    for rows, cols in ((H, I), (H, H), (H, H), (O, H)):
        parts.append(rng.standard_normal(rows * cols) * np.sqrt(2.0 / cols))
        parts.append(np.zeros(rows))
    parts += [np.asarray(mean, dtype=np.float64), np.asarray(scale, dtype=np.float64)]
    return np.concatenate(parts).astype(np.float32)


def e2e_form(rhi, w, torch, steps, warmup, precond, limiter_jacobian=0, max_newton=200,
             guess=0, weights=None):
    """Same metric through the public API with host buffers: each timed step copies the
    step's inputs (E, e, n, n_H and the point-source list) from pinned host memory, runs the
    step and reads the state (E, e, n) back into pinned host memory."""
    s = rhi.solver_for_workload(w, precond=precond, mg_levels=6, theta=1.0,
                                limiter_jacobian=limiter_jacobian, max_newton=max_newton,
                                guess=guess)
    if weights is not None:
        s.mlp_set_weights(weights)
    N = w.N
    pinned = []

    def pin(m):
        t = torch.empty(m, dtype=torch.float64, pin_memory=True)
        pinned.append(t)
        return t.numpy()
    st = w.state()
    E, e, n, nH = pin(N), pin(N), pin(w.ns * N), pin(N)
    E[:] = st["E"]; e[:] = st["e"]; n[:] = st["n"].ravel(); nH[:] = w.nH.ravel()
    oE, oe, on = pin(N), pin(N), pin(w.ns * N)
    # the host link's rate into and out of these pinned buffers, by torch's own copies of the
    # state's bytes (best of three), beside which the library's copies are read
    outs = pinned[4:7]                                   # oE, oe, on
    devs = [torch.empty_like(t, device="cuda") for t in outs]
    rates = {}
    for name in ("d2h", "h2d"):
        best = float("inf")
        for _ in range(3):
            torch.cuda.synchronize()
            t = time.perf_counter()
            for hb, db in zip(outs, devs):
                (hb.copy_(db, non_blocking=True) if name == "d2h" else db.copy_(hb, non_blocking=True))
            torch.cuda.synchronize()
            best = min(best, time.perf_counter() - t)
        rates[name] = sum(d.numel() for d in devs) * 8 / best / 1e9
    del devs
    # the same step indices as the device-timed region: warm-up steps first, untimed
    for _ in range(warmup):
        s.step(w.dt, 1.0, 0.0, w.newton_tol, w.lin_tol)
    s.get_state(E, e, n)
    torch.cuda.synchronize()
    # each call returns after its stream work is done, so the wall clock between calls splits
    # the step into copies in, the solve and copies out
    split = dict(set_state=0.0, set_sources=0.0, step=0.0, get_state=0.0)
    t0 = time.perf_counter()
    for _ in range(steps):
        ta = time.perf_counter()
        s.set_state(E, e, n, nH, None)
        tb = time.perf_counter()
        s.set_sources(w.src_ijk, w.src_rate)
        tc = time.perf_counter()
        s.step(w.dt, 1.0, 0.0, w.newton_tol, w.lin_tol)
        td = time.perf_counter()
        s.get_state(oE, oe, on)
        te = time.perf_counter()
        split["set_state"] += tb - ta
        split["set_sources"] += tc - tb
        split["step"] += td - tc
        split["get_state"] += te - td
        E, oE = oE, E
        e, oe = oe, e
        n, on = on, n
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    # after the timed loop: the device time of get_state's copies right after a step, beside
    # torch's own copy of the same bytes from device buffers into pinned buffers just after it
    # (both on the legacy stream); a slow host link slows both, a slow library copy only one
    def dev_ms(f):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        f()
        b.record()
        b.synchronize()
        return a.elapsed_time(b)

    def torch_copy():
        for hb, db in zip(outs, devs):
            hb.copy_(db, non_blocking=True)
    devs = [torch.empty_like(t, device="cuda") for t in outs]
    after = []
    for _ in range(4):
        s.step(w.dt, 1.0, 0.0, w.newton_tol, w.lin_tol)
        after.append((dev_ms(lambda: s.get_state(oE, oe, on)), dev_ms(torch_copy)))
    del devs
    rates["after_step_ms"] = {"get_state": [round(a, 2) for a, _ in after],
                              "torch_copy": [round(b, 2) for _, b in after]}
    try:                                  # the CUDA runtime(s) this process has mapped
        with open("/proc/self/maps") as f:
            rates["cudart_mapped"] = sorted({ln.split()[-1] for ln in f if "libcudart" in ln})
    except OSError:
        pass
    s.close()
    h2d = 8 * N * (3 + w.ns) + 20 * len(w.src_rate)
    d2h = 8 * N * (2 + w.ns)
    return N * steps / dt, h2d, d2h, {k: 1e3 * v / steps for k, v in split.items()}, rates


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="rhi")
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--forms", default="plain_fp64,mixed_fp32mg,learned_mixed",
                    help="comma list of forms to time (the last one is the headline)")
    ap.add_argument("--train-steps", type=int, default=20,
                    help="steps of the 128^3 training run for the learned guess")
    ap.add_argument("--train-epochs", type=int, default=4)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-config2", action="store_true",
                    help="skip the 128^3 plain FP64 configuration (20 steps)")
    ap.add_argument("--cosmo-intervals", type=int, default=0,
                    help="also run the first K intervals of the cosmological configuration")
    ap.add_argument("--cosmo-n", type=int, default=512)
    ap.add_argument("--max-newton", type=int, default=200)
    ap.add_argument("--limiter-jacobian", type=int, default=2,
                    help="0: D lagged (CG); 1: dD/dE kept; 2: exact Newton matrix (BiCGStab)")
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
    nsrc = workload_sources(n)
    w = inputs.config_lognormal(n, nsrc=nsrc, seed=rank)
    hbm_peak, peak_src = load_peaks()
    AB = alg_bytes(args.limiter_jacobian != 0)

    # forms: plain FP64 (FP64 multigrid), mixed (FP32 multigrid), learned + mixed (headline)
    FORMS = {"plain_fp64": (rhi.RHI_PRECOND_MG_FP64, rhi.RHI_GUESS_PREVIOUS),
             "mixed_fp32mg": (rhi.RHI_PRECOND_MG_FP32, rhi.RHI_GUESS_PREVIOUS),
             "learned_mixed": (rhi.RHI_PRECOND_MG_FP32, rhi.RHI_GUESS_LEARNED)}
    order = [f for f in args.forms.split(",") if f]
    weights, train_info = None, None
    if any(FORMS[f][1] == rhi.RHI_GUESS_LEARNED for f in order):
        weights, train_info = train_guess(rhi, torch, rank, args.train_steps, args.train_epochs)
        torch.cuda.empty_cache()
    forms = {}
    for name in order:
        pc, guess = FORMS[name]
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        clk = ClockSampler(local)
        clk.start()
        s, ms, agg, kt_timed, kt_all, tname = run_form(
            rhi, w, torch, args.steps, args.warmup, pc, AB,
            limiter_jacobian=args.limiter_jacobian, max_newton=args.max_newton, guess=guess,
            weights=weights if guess == rhi.RHI_GUESS_LEARNED else None)
        clocks = clk.stop()
        forms[name] = dict(ms=max_over_ranks(ms, dist, "cuda"), agg=agg, kt=kt_all,
                           kt_timed=kt_timed, clocks=clocks, tname=tname)
        s.close()
        del s
        torch.cuda.empty_cache()

    head = forms[order[-1]]
    ms_step = head["ms"] / args.steps
    value = replica_throughput(world, w.N, args.steps, head["ms"])

    # the dominant kernel (largest share of the breakdown step, among the kernels with a byte
    # or flop model) and its roofline from the per-launch device times inside the timed region
    kt = head["kt"]
    tot = sum(v[0] for v in kt.values())
    tname = head["tname"]
    roof = {"kernel": tname, "share": kt[tname][0] / tot if tot else None,
            "launches_breakdown_step": kt[tname][1]}
    if tname in head["kt_timed"]:
        tms, tcnt = head["kt_timed"][tname]
        avg_s = tms / tcnt * 1e-3
        roof["avg_launch_ms"] = avg_s * 1e3
        roof["launches_timed"] = tcnt
        roof["units_per_launch"] = w.N
        if tname in ALU_FLOPS:
            ach = ALU_FLOPS[tname] * w.N / avg_s / 1e12
            roof.update(bound="alu", achieved=ach, peak=FP64_PEAK_TFLOPS, unit="TFLOP/s",
                        frac=ach / FP64_PEAK_TFLOPS,
                        traffic=TRAFFIC_PER_CELL[tname] * w.N if tname in TRAFFIC_PER_CELL else None,
                        flops_per_cell=ALU_FLOPS[tname],
                        peak_source="derived: 152 SMs x 2070 MHz x 2 DFMA/clk/SM x 2 flop")
        elif tname in AB:
            ach = AB[tname] * w.N / avg_s / 1e9
            roof.update(bound="hbm", achieved=ach, peak=hbm_peak, unit="GB/s",
                        frac=ach / hbm_peak, bytes_per_cell=AB[tname],
                        traffic=TRAFFIC_PER_CELL[tname] * w.N if tname in TRAFFIC_PER_CELL else None,
                        peak_source=peak_src + " copy bandwidth (MEASURED_PEAKS hbm_gbs)"
                        if peak_src == "measured" else peak_src)
    # HBM fraction of the Krylov / multigrid stencil and vector kernels (full-grid launches):
    # algorithmic bytes over the mean launch time of the profiled step, against the measured
    # copy bandwidth
    def hbm_fracs(kt_f):
        out = {}
        for k in LINEAR_KERNELS:
            if k in kt_f and kt_f[k][1] > 0 and kt_f[k][0] > 0:
                ms_k, c_k = kt_f[k]
                out[k] = AB[k] * w.N / (ms_k / c_k * 1e-3) / 1e9 / hbm_peak
        return out

    lin = hbm_fracs(kt)

    def summary(f):
        return {"value": replica_throughput(world, w.N, args.steps, f["ms"]),
                "ms_per_step": f["ms"] / args.steps,
                **{k: v / args.steps for k, v in f["agg"].items()
                   if isinstance(v, (int, float))},
                "kernel_ms_breakdown_step": {k: v[0] for k, v in
                                             sorted(f["kt"].items(), key=lambda kv: -kv[1][0])},
                "kernel_launches_breakdown_step": {k: v[1] for k, v in
                                                   sorted(f["kt"].items(), key=lambda kv: -kv[1][0])},
                "roofline_kernel": f["tname"],
                "newton_per_step": f["agg"]["newton_per_step"],
                "krylov_per_step": f["agg"]["krylov_per_step"],
                "hbm_frac": hbm_fracs(f["kt"])}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_text(n),
                   "form": FORM_TEXT[order[-1]],
                   "newton_matrix": NEWTON_TEXT[args.limiter_jacobian],
                   "parallelism": "replicas" if world > 1 else "1 GPU",
                   "l2": "inputs larger than L2 (about 12 GB of fields per form)"},
        "roofline": roof,
        "forms": {k: summary(f) for k, f in forms.items()},
        "iterations_per_step": {k: v / args.steps for k, v in head["agg"].items()
                                if isinstance(v, (int, float))},
        "newton_residuals_last_step": head["agg"]["res_history_last"],
        "gpu_launches": head["agg"]["launches"],
        "clocks": head["clocks"],
        "hbm_frac_linear_kernels": lin,
    }
    if "plain_fp64" in forms and order[-1] != "plain_fp64":
        line["speedup_vs_plain_fp64"] = forms["plain_fp64"]["ms"] / head["ms"]
    if train_info:
        line["learned_guess_training"] = train_info
    if not args.no_config2:
        line["config_128_plain_fp64"] = config_128_plain(rhi, torch, args.limiter_jacobian,
                                                         args.max_newton)
    if args.cosmo_intervals > 0:
        line["config_cosmo"] = config_cosmo_run(rhi, torch, args.cosmo_n, args.cosmo_intervals,
                                                min(args.max_newton, 40))
    if rank == 0:
        if not args.no_e2e:
            pc, guess = FORMS[order[-1]]
            e2e_val, h2d, d2h, split, rates = e2e_form(
                rhi, w, torch, args.steps, args.warmup, pc, args.limiter_jacobian,
                args.max_newton, guess, weights if guess == rhi.RHI_GUESS_LEARNED else None)
            line["e2e"] = {"value": world * e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d,
                           "d2h_bytes_per_step": d2h, "wall_ms_per_step": split,
                           "host_link_gbs": rates,
                           "get_state_gbs": d2h / (split["get_state"] * 1e-3) / 1e9,
                           "set_state_gbs": (h2d - 20 * len(w.src_rate)) / (split["set_state"] * 1e-3) / 1e9}
        if not args.no_cpu_baseline:
            line["cpu_baseline"], (wsub, refs) = cpu_baseline_sample()
            line["error_vs_oracle"] = {
                "sample": f"{len(refs)} steps of the {wsub.nx}^3 sub-box of the cpu_baseline "
                          "sample at the timed run's settings, against the oracle converged to "
                          "1e-14; per field the worst over the steps of max |gpu - oracle| / "
                          "(|oracle| + 1e-12 max|oracle|), species as fractions of their element "
                          "(per_element), and of max |gpu - oracle| / u in the scaled unknowns "
                          "the Newton tolerance applies to, with their RMS over all unknowns "
                          "(scaled)",
                **error_vs_oracle(rhi, {k: FORMS[k] for k in order}, wsub, refs,
                                  args.limiter_jacobian, weights)}
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
