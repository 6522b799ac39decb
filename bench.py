#!/usr/bin/env python
"""Throughput benchmark of the DG shallow-water / regularized-Bingham hot path.

Workload (default): the large 2D Bingham slump on a 2048 x 2048 structured
triangulation of [-1, 1]^2 (8,388,608 triangles), order p = 2, Gaussian
mound of depth 1 (sigma 0.15) on a plane of slope 0.05 with a 16-mode seeded
bed of amplitude 0.05, bi-viscosity regularization (yield stress 0.05,
gamma = 1e3, eta = 0.01), in FP64.  One benchmark step advances the state by
``--inner`` CFL-limited SSP-RK3 steps (each step = 3 x (E-step, face flux,
volume/lift/mass-solve/update) + FP64 step-size reduction).  The same
workload then runs in FP32 (FP64 step-size and mass reductions) and is
reported under "mixed", with its relative L2 distance from the FP64 run at
full size and from the FP64 oracle on a sample.  The L2 cache is flushed
(256 MiB write) before every timed step, outside the timed events.

Metric: DOF-updates/s = elements x nodes x fields x RK3 steps / time (the
auxiliary E is not counted), summed over all instances and all ranks.

Other workloads (--workload): the 9-instance radial dam-break sweep, the 1D
dam break, the bump dam break, the 256-instance ensemble, the paper's 1D
implicit dam break and a 2D backward-Euler Newton-Krylov run.
``--impl reference`` times the FP64 CPU oracle instead (see ``oracle/``).
"""
import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DOF-updates/sec at stated L2 error vs FP64 oracle; % HBM roofline; FP64 vs mixed/batched"
UNIT = "DOF-updates/s"
SIGMAS = (0.0, 0.02, 0.1)
REGS = (1, 2, 3)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="slump",
                    choices=["radial", "dam1d", "bump", "ensemble", "slump", "implicit_dam", "newton2d", "drybed"],
                    help="radial: 9-instance radial dam-break sweep (64x64x2, p=2); dam1d: 1D dam break "
                         "(200 el, p=1); bump: dam break over a bump (512x512x2 jittered, p=3); ensemble: "
                         "256 heterogeneous instances; slump: 2048x2048x2 Bingham slump (p=2); implicit_dam: "
                         "the paper's 1D dam break with backward Euler + Newton (100 el, p=1, m3=0, dt=1e-6); "
                         "newton2d: 2D radial dam break (64x64x2, p=2) with backward Euler + Newton-Krylov; "
                         "drybed: 2D dam break onto a dry bed in wet/dry mode (1024x1024x2, p=1)")
    ap.add_argument("--solver", default="mixed", choices=["fp64", "mixed"],
                    help="implicit_dam: FP64 block Thomas, or FP32 factorization + FP64 refinement")
    ap.add_argument("--precision", default=None, choices=["fp64", "fp32", "fp32tc"],
                    help="fp32tc: FP32 with the p >= 2 triangle volume contractions on the tensor cores")
    ap.add_argument("--mode", default="batch", choices=["batch", "solo"],
                    help="batch: all instances in one dg_batch (one launch per phase); solo: one context each")
    ap.add_argument("--inner", type=int, default=None, help="RK3 steps per instance per bench step")
    ap.add_argument("--n", type=int, default=None,
                    help="squares per side of the 2D mesh (radial 64, bump 512, slump 2048); "
                         "smaller values give profiling cases of the same kernels")
    ap.add_argument("--order", type=int, default=2)
    ap.add_argument("--persistent", action="store_true",
                    help="batch mode: one persistent launch per group and step (dg_batch_set_persistent)")
    ap.add_argument("--tiles", default=None,
                    help="JSON list of [estep, face, volume] block sizes per group (encoded as in "
                         "dg_batch_set_tiles) instead of the autotuner's choice; for profiling")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-mixed", action="store_true",
                    help="slump in FP64: skip the FP32 companion run reported under 'mixed'")
    ap.add_argument("--compare-steps", type=int, default=10,
                    help="slump in FP64: steps of the full-size FP64-vs-FP32 comparison")
    ap.add_argument("--oracle-worker", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--oracle-seconds", type=float, default=15.0)
    a = ap.parse_args()
    d = WORKLOAD_DEFAULTS[a.workload]
    if a.precision is None:
        a.precision = d["precision"]
    if a.inner is None:
        a.inner = d["inner"]
    if a.n is None:
        a.n = {"bump": 512, "slump": 2048, "drybed": 1024}.get(a.workload, 64)
    return a


WORKLOAD_DEFAULTS = {
    "radial": dict(precision="fp64", inner=100),
    "dam1d": dict(precision="fp64", inner=100),
    "bump": dict(precision="fp32", inner=10),
    "ensemble": dict(precision="fp32", inner=10),
    "slump": dict(precision="fp64", inner=1),
    "implicit_dam": dict(precision="fp64", inner=200),
    "newton2d": dict(precision="fp64", inner=2),
    "drybed": dict(precision="fp64", inner=10),
}

# backward-Euler step of the newton2d workload, in multiples of the explicit
# SSP-RK3 step bound at the initial state
NEWTON2D_DT_FACTOR = 10.0


def newton2d_case(n, order):
    import synth
    return synth.radial_dam_2d(n=n, order=order, reg=3, sigma0=0.02, gamma=50.0, eta=0.01)


def sweep_cases(n, order):
    import synth
    out = []
    for s0 in SIGMAS:
        for reg in REGS:
            out.append(synth.radial_dam_2d(n=n, order=order, reg=reg, sigma0=s0, eta=0.01,
                                           gamma=1e3, beta=1e3))
    return out


def workload_cases(args):
    import synth
    if args.workload == "radial":
        return sweep_cases(args.n, args.order)
    if args.workload == "dam1d":
        return [synth.dam_break_1d()]
    if args.workload == "bump":
        return [synth.bump_dam_2d(n=args.n)]
    if args.workload == "ensemble":
        return synth.ensemble_cases()
    if args.workload == "implicit_dam":
        return [synth.paper_dam_break_1d(n_el=100, order=1, m3=0, reg=1, gamma=1e2, beta=1e2)]
    if args.workload == "newton2d":
        return [newton2d_case(args.n, args.order)]
    if args.workload == "drybed":
        return [synth.dry_dam_2d(n=args.n)]
    return [synth.slump_2d(n=args.n)]


def sample_case(workload, n, order):
    """The bounded sample the CPU oracle times (and the accuracy check runs):
    the workload itself when it is small, else the same physics on a smaller
    mesh (stated in the JSON line)."""
    import synth
    if workload == "radial":
        return sweep_cases(n, order)[0], f"instance 0 (sigma0=0, reg 1) of the sweep, {n}x{n}x2, full size"
    if workload == "dam1d":
        return synth.dam_break_1d(), "the full 1D dam break (200 elements, p=1)"
    if workload == "bump":
        return synth.bump_dam_2d(n=32), "bump dam break on a 32x32x2 jittered mesh (p=3), same physics"
    if workload == "implicit_dam":
        return (synth.paper_dam_break_1d(n_el=100, order=1, m3=0, reg=1, gamma=1e2, beta=1e2),
                "the paper's implicit dam break (100 elements, p=1, m3=0, dt=1e-6)")
    if workload == "newton2d":
        return (newton2d_case(6, order),
                f"the same physics on a 6x6x2 mesh (p={order}), dt = {NEWTON2D_DT_FACTOR:g} x its explicit bound")
    if workload == "drybed":
        return synth.dry_dam_2d(n=32), "dry-bed dam break on a 32x32x2 mesh (p=1, wet/dry mode), same physics"
    if workload == "ensemble":
        c = synth.ensemble_cases(n_inst=8, size_scale=0.1)[1]
        return c, f"one ensemble-style instance ({c.dim}D, p={c.order}, {c.etov.shape[0]} elements)"
    return synth.slump_2d(n=32), "Bingham slump on a 32x32x2 mesh (p=2), same physics"


def workload_name(args):
    if args.workload == "radial":
        return (f"radial_dam_2d {args.n}x{args.n}x2 triangles on [-1,1]^2, p={args.order}, "
                f"sigma0 in {list(SIGMAS)} x regularization in {list(REGS)} (gamma=beta=1e3, eta=0.01)")
    return {"dam1d": "dam_break_1d 200 elements on [0,1], p=1, exponential regularization m=1e3, sigma0=0.05",
            "bump": f"bump_dam_2d {args.n}x{args.n}x2 jittered triangles (seed 3), p=3, tanh regularization gamma=1e3",
            "ensemble": "ensemble of 256 instances (seed 4): 1D/2D, p in {1,2,3}, 1e3..5e4 elements",
            "slump": f"slump_2d {args.n}x{args.n}x2 triangles, p=2, slope 0.05, 16-mode bed (seed 5), bi-viscosity",
            "implicit_dam": "paper_dam_break_1d 100 elements, p=1, m3=0, backward Euler + Newton, dt=1e-6, "
                            "regularization 1 gamma=beta=1e2",
            "drybed": f"dry_dam_2d {args.n}x{args.n}x2 triangles on [-1,1]^2, p=1, depth 1 | 0 (dry) at x_1 = 0, "
                      "Newtonian limit, reflecting walls, wet/dry mode (conservative-moment stages, depth limiter)",
            "newton2d": f"radial_dam_2d {args.n}x{args.n}x2 triangles, p={args.order}, tanh regularization "
                        f"sigma0=0.02 gamma=50 eta=0.01, backward Euler + Newton-Krylov, dt = "
                        f"{NEWTON2D_DT_FACTOR:g} x the explicit bound"}[
        args.workload]



# ---------------------------------------------------------------- multi-rank aggregation

def max_over_ranks(x, device="cpu"):
    """Largest value of x over all ranks (the slowest rank's time); x itself
    without an initialised multi-rank process group."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_throughput(units_per_rank_step, steps, world, max_ms):
    """Units processed by all ranks divided by the slowest rank's time (weak
    scaling: every rank runs its own replica of the workload)."""
    return units_per_rank_step * steps * world / (max_ms / 1e3)

# ---------------------------------------------------------------- analytic counts

def shape(dim, p):
    nq1 = (3 * p + 1) // 2
    return dict(NP=p + 1 if dim == 1 else (p + 1) * (p + 2) // 2, NQ=nq1 if dim == 1 else nq1 * nq1,
                NF=dim + 1, NFP=1 if dim == 1 else p + 1, NFQ=1 if dim == 1 else (3 * p + 2) // 2,
                NV=dim + 1, NE=dim * dim)


def volume_flops(dim, p, bed=False):
    """Floating-point operations of one volume-kernel element (FMA = 2):
    interpolation to the volume points, pointwise flux/stress/source,
    weighted-derivative contraction, face lift, the h-weighted mass matrix,
    its Cholesky factorization and the two triangular solves per velocity
    component, and the stage update.  Divisions, square roots and
    transcendental calls count as 1."""
    s = shape(dim, p)
    NP, NQ, NV, NE, NF, NFP, NFQ = s["NP"], s["NQ"], s["NV"], s["NE"], s["NF"], s["NFP"], s["NFQ"]
    f = 0
    per_q = 2 * NP * (NV + NE) + (4 * NP * dim if bed else 0)
    per_q += 25 if dim == 2 else 8          # stress (norm, sqrt, regularization, products)
    per_q += 6 * dim * NV                   # F and Q components, reference rotation
    per_q += 2 * NP * NV * (dim + 1)        # contraction with Wr, Ws, Wm
    f += NQ * per_q + NV * NP               # + J scaling
    f += NF * NFP * NV * 2 * NFQ            # lift of face fluxes
    f += 2 * NP * NP + NP                   # dh/dt = -Minv r_h / J
    per_q2 = 2 * NP + NP * (NP + 1) + 2 * NP * dim + 3
    f += NQ * per_q2                        # dh/dt at the points, M_h and M_u dh/dt (h and u
                                            # at the points are the ones interpolated above)
    f += NP ** 3 // 3 + NP * NP             # Cholesky
    f += dim * 2 * NP * NP                  # two triangular solves per component
    f += NV * NP * 5                        # stage update
    return f


def estep_flops(dim, p):
    s = shape(dim, p)
    NP, NF, NFP = s["NP"], s["NF"], s["NFP"]
    return dim * NP * NP * 2 * dim + NP * dim * dim * 2 * dim + NF * NFP * dim * 2 + NP * NF * NFP * dim * dim * 3


def face_flops_per_point(dim, p):
    s = shape(dim, p)
    return 2 * 2 * s["NFP"] * (s["NV"] + s["NE"]) + 60 + 2 * (30 if dim == 2 else 10)


def volume_bytes(dim, p, rs):
    """Compulsory bytes of one volume-kernel element: read Vin (NV x NP),
    V0 (NV x NP), E (NE x NP), geometry (5), face ids (NF x 4 B) and the face
    fluxes it lifts (NF x NV x NFQ, each face read by both neighbours), write
    Vout (NV x NP)."""
    s = shape(dim, p)
    NP, NV, NE, NF, NFQ = s["NP"], s["NV"], s["NE"], s["NF"], s["NFQ"]
    return rs * (3 * NV * NP + NE * NP + 5 + NF * NV * NFQ) + 4 * NF


# ---------------------------------------------------------------- helpers

def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# FP64 and FP32 pipe peaks are derived from unit counts and the maximum SM
# clock (SMs x 2070 MHz x 2 flop/FMA x FMA lanes/SM/clk: FP32 128, FP64 2 on
# GB300, whose nominal FP64 rate is 1.25 TFLOP/s) and measured beside that by
# the library's FMA probe (include/dg_probe.h).
SM_MAX_MHZ = 2070.0


def traffic_record(kernel, workload):
    """Per-launch DRAM bytes of a kernel from the committed ncu summary, or
    None when the summary is missing or the kernel source changed since."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
            rec = json.load(f)
    except Exception:
        return None
    src = os.path.join(ROOT, "paper_2301_11238_gb300", "csrc", "dg_kernels.cuh")
    h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    r = rec.get(f"{kernel}|{workload}")
    if not r or r.get("source_sha") != h:
        return None
    return r.get("bytes_per_launch")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.tmp = None

    def __enter__(self):
        try:
            self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.tmp, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if self.proc is None or self.tmp is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.tmp.flush()
        rows = []
        with open(self.tmp.name) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.tmp.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = sorted(float(r[1]) for r in rows if r[1].replace(".", "").isdigit())
        mx = max(float(r[2]) for r in rows if r[2].replace(".", "").isdigit())
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows
                                                         if r[3].replace(".", "").isdigit())}


# ---------------------------------------------------------------- oracle legs

def oracle_worker(spec_path):
    """Runs in a subprocess with one BLAS/OpenMP thread: times the oracle on
    instance 0 of the workload for about ``seconds`` and writes JSON."""
    import numpy as np
    with open(spec_path) as f:
        spec = json.load(f)
    from oracle.run import build as oracle_build
    case, _ = sample_case(spec["workload"], spec["n"], spec["order"])
    d, V0, _ = oracle_build(case)
    Vh = d.to_modal(V0)
    units = d.K * d.Np * d.nV
    steps, times = 0, []
    implicit = spec["workload"] == "implicit_dam"
    newton = spec["workload"] == "newton2d"
    if implicit:
        from oracle.implicit import Implicit1D
        im = Implicit1D(d, case.dt)
        X = im.pack(Vh, im.initial_E(Vh))
    if newton:
        from oracle.implicit_reduced import ImplicitReduced
        nr = ImplicitReduced(d, NEWTON2D_DT_FACTOR * d.stable_dt(Vh))
    t_all = time.perf_counter()
    while True:
        t0 = time.perf_counter()
        if implicit:
            X, _, _ = im.step(X)
            Vh, _ = im.unpack(X)
        elif newton:
            Vh, _, _ = nr.step(Vh, rtol=1e-14, atol=1e-11)
        else:
            Vh, _ = d.ssp_rk3_step(Vh)
        times.append(time.perf_counter() - t0)
        steps += 1
        if steps >= spec.get("max_steps", 10 ** 9):
            break
        if time.perf_counter() - t_all > spec["seconds"] and steps >= spec.get("min_steps", 1):
            break
    out = dict(steps=steps, seconds=sum(times), units_per_step=units, step_times=times,
               final=d.to_nodal(Vh).tolist() if spec.get("return_state") else None)
    with open(spec["out"], "w") as f:
        json.dump(out, f)


def run_oracle_subprocess(workload, n, order, seconds, min_steps=1, max_steps=10 ** 9, return_state=False):
    with tempfile.TemporaryDirectory() as td:
        spec = dict(workload=workload, n=n, order=order, seconds=seconds, min_steps=min_steps,
                    max_steps=max_steps,
                    out=os.path.join(td, "out.json"), return_state=return_state)
        sp = os.path.join(td, "spec.json")
        with open(sp, "w") as f:
            json.dump(spec, f)
        env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
        subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-worker", sp], check=True,
                       env=env, cwd=ROOT)
        with open(spec["out"]) as f:
            return json.load(f)


def reference_main(args):
    """The oracle as it stands, on one host core, same workload, metric and unit.
    Each step is one SSP-RK3 step of one sweep instance (the oracle needs about
    half a second for it); warm-up steps are untimed."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    res = run_oracle_subprocess(args.workload, args.n, args.order, seconds=0.0,
                                min_steps=args.warmup + args.steps, max_steps=args.warmup + args.steps)
    _, sample_desc = sample_case(args.workload, args.n, args.order)
    times = res["step_times"][args.warmup:]
    secs = sum(times)
    value = res["units_per_step"] * len(times) / secs
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": workload_name(args), "sample": f"one SSP-RK3 step per step of {sample_desc}"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{len(times)} SSP-RK3 steps of {sample_desc}"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)



def implicit_main(args):
    """Backward Euler + Newton on the paper's dam break: each bench step is
    ``--inner`` implicit time steps in one persistent launch."""
    import numpy as np
    import torch
    import paper_2301_11238_gb300 as G
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    case = workload_cases(args)[0]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        s, V0 = G.implicit_from_case(case, dt=case.dt, mixed=(args.solver == "mixed"), stream=stream)
        units_per_inner = s.K * s.Np * 2
        for _ in range(args.warmup):
            s.run(args.inner)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        torch.cuda.synchronize()
        its0 = s.run(0)
        with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
            for k in range(args.steps):
                evs[k][0].record(stream)
                s.L.dg_implicit_run(s.ctx, int(args.inner), None)
                evs[k][1].record(stream)
            stream.synchronize()
        st = s.run(0)
    total_ms = sum(a.elapsed_time(b) for a, b in evs)
    steps_timed = args.steps * args.inner
    its = (st["newton_its"] - its0["newton_its"]) / max(1, st["steps"] - its0["steps"])
    value = units_per_inner * steps_timed * world / (total_ms / 1e3)
    cpu = acc = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        res = run_oracle_subprocess(args.workload, args.n, args.order, seconds=args.oracle_seconds, min_steps=2,
                                    return_state=True)
        cpu = {"value": res["units_per_step"] * res["steps"] / res["seconds"], "unit": UNIT, "cores": 1,
               "kind": "oracle", "sample": f"{res['steps']} backward-Euler Newton steps of the same problem, "
                                           f"{res['seconds']:.1f} s on one host core"}
        with torch.cuda.stream(stream):
            s2, _ = G.implicit_from_case(case, dt=case.dt, mixed=(args.solver == "mixed"), stream=stream)
            s2.run(res["steps"])
            Vg, _ = s2.get_state()
            s2.close()
        Vo = np.asarray(res["final"])
        acc = {"rel_l2_vs_fp64_oracle": float(np.linalg.norm(Vg - Vo) / np.linalg.norm(Vo)),
               "after_steps": res["steps"], "case": "same problem", "precision": "fp64 residual"}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(args), "inner_implicit_steps_per_step": args.inner,
                       "linear_solver": args.solver, "newton_its_per_step": its,
                       "l2": "working set (a few hundred KB) is cache-resident by nature; not flushed",
                       "parallelism": f"replicas x{world}"},
            "roofline": {"bound": "latency", "kernel": "implicit_kernel<1,0> (one thread block)",
                         "achieved": None, "peak": None, "unit": None, "frac": None, "traffic": None,
                         "note": "one 100-element problem in one block: the Newton loop is a dependent "
                                 "chain on one SM (the block-Thomas sweep is one warp)",
                         "ms_per_time_step": total_ms / steps_timed},
            "cpu_baseline": cpu, "e2e": None, "gpu_launches": args.steps,
            "clocks": clk.summary(), "accuracy": acc,
            "paper": {"cpu_time_s_for_150000_steps": 1.4e4, "hardware": "unstated", "cite": "Table damBreakFuns"}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    s.close()

def newton_main(args):
    """Backward Euler + Newton-Krylov (dg_newton.h) on a 2D radial dam break:
    each bench step is ``--inner`` implicit time steps; dt is a fixed
    multiple of the explicit step bound at the initial state."""
    import numpy as np
    import torch
    import paper_2301_11238_gb300 as G
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    case = workload_cases(args)[0]
    stream = torch.cuda.Stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    with torch.cuda.stream(stream):
        probe, V0, _ = G.solver_from_case(case, stream=stream)
        dt = NEWTON2D_DT_FACTOR * probe.step(0.0)  # explicit bound at the initial state
        probe.close()
        s, V0, _ = G.solver_from_case(case, stream=stream)
        kw = dict(rtol=1e-10, atol=1e-11, krylov_dim=30, krylov_rtol=1e-4)
        nk = G.Newton(s, dt, **kw)
        for _ in range(args.warmup):
            nk.run(args.inner)
        st0 = nk.run(0)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        torch.cuda.synchronize()
        with ClockSampler(local) as clk:
            for k in range(args.steps):
                flush.zero_()
                evs[k][0].record(stream)
                nk.run(args.inner)
                evs[k][1].record(stream)
            stream.synchronize()
        st = nk.run(0)
    total_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in evs))
    # the same instance with the explicit SSP-RK3 integrator (CFL-limited step),
    # for simulated time per wall second at the same physics
    with torch.cuda.stream(stream):
        sx, _, _ = G.solver_from_case(case, stream=stream)
        sx.run(5)
        t0 = sx.sync()["t"]
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sx.advance(200)
        e1.record(stream)
        stream.synchronize()
        explicit_sim_rate = (sx.sync()["t"] - t0) / (e0.elapsed_time(e1) / 1e3)
        sx.close()
    steps_timed = args.steps * args.inner
    units_per_step = s.K * s.Np * s.nV
    value = whole_job_throughput(units_per_step * args.inner, args.steps, world, total_ms)
    dn = st["newton_its"] - st0["newton_its"]
    dk = st["krylov_its"] - st0["krylov_its"]
    cpu = acc = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        res = run_oracle_subprocess(args.workload, args.n, args.order, seconds=args.oracle_seconds, min_steps=2,
                                    return_state=True)
        sc, sdesc = sample_case(args.workload, args.n, args.order)
        cpu = {"value": res["units_per_step"] * res["steps"] / res["seconds"], "unit": UNIT, "cores": 1,
               "kind": "oracle", "sample": f"{res['steps']} backward-Euler steps of {sdesc}, "
                                           f"{res['seconds']:.1f} s on one host core"}
        from oracle.run import build as oracle_build
        d, V0s, _ = oracle_build(sc)
        with torch.cuda.stream(stream):
            s2, _, _ = G.solver_from_case(sc, stream=stream)
            nk2 = G.Newton(s2, NEWTON2D_DT_FACTOR * d.stable_dt(d.to_modal(V0s)), rtol=1e-13, atol=1e-11,
                           krylov_dim=64, krylov_rtol=1e-11)
            nk2.run(res["steps"])
            Vg = s2.get_state(with_E=False)
            nk2.close()
            s2.close()
        Vo = np.asarray(res["final"])
        acc = {"rel_l2_vs_fp64_oracle": float(np.linalg.norm(Vg - Vo) / np.linalg.norm(Vo)),
               "after_steps": res["steps"], "case": sdesc, "precision": "fp64",
               "oracle": "reduced Newton with a coloured finite-difference Jacobian and a sparse direct solve"}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(args), "implicit_steps_per_step": args.inner, "dt": dt,
                       "newton_its_per_step": dn / max(1, steps_timed),
                       "krylov_its_per_newton_it": dk / max(1, dn), "newton": kw,
                       "simulated_time_per_second": dt * steps_timed / (total_ms / 1e3),
                       "explicit_rk3_simulated_time_per_second": explicit_sim_rate,
                       "l2": "flushed (256 MiB write) before each step", "parallelism": f"replicas x{world}"},
            "roofline": {"bound": "alu", "kernel": "residual evaluations (estep, face, volume mode 2, time term)",
                         "achieved": None, "peak": None, "unit": None, "frac": None, "traffic": None,
                         "note": "each Krylov iteration is one residual evaluation plus the preconditioner and "
                                 "Gram-Schmidt reductions with one host synchronization; the residual kernels "
                                 "are the explicit path's (FP64 pipe bound, see the default line)",
                         "ms_per_time_step": total_ms / steps_timed},
            "cpu_baseline": cpu, "e2e": None, "gpu_launches": None,
            "clocks": clk.summary(), "accuracy": acc}
    if rank == 0:
        print(json.dumps(line), flush=True)
    nk.close()
    s.close()

# ---------------------------------------------------------------- GPU leg

def pipe_peaks(G, stream):
    """FP64 and FP32 pipe peaks (TFLOP/s): derived from the unit counts and
    the maximum SM clock, and measured live by the library's FMA probe."""
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    derived = {"fp64": sms * SM_MAX_MHZ * 1e6 * 2 * 2 / 1e12, "fp32": sms * SM_MAX_MHZ * 1e6 * 2 * 128 / 1e12}
    probe = {"fp64": G.fma_rate(G.PREC_FP64, stream=stream) / 1e12,
             "fp32": G.fma_rate(G.PREC_FP32, stream=stream) / 1e12}
    return derived, probe, sms


def measure(args, G, cases, prec, stream, flush, world, local, clocks=True, e2e_on=True, compare_steps=0):
    """Builds the workload at one precision, times ``args.steps`` bench steps
    (after ``args.warmup``), times the dominant kernel on its own launching
    stream and (optionally) the end-to-end path with host buffers.  With
    compare_steps > 0 it finally resets every instance to its initial state,
    runs that many steps and returns instance 0's state (a CUDA tensor)."""
    import numpy as np
    import torch
    import torch.distributed as dist
    batch, solvers, V0s, tiles = None, [], [], None
    with torch.cuda.stream(stream):
        if args.mode == "batch":
            batch, V0s = G.batch_from_cases(cases, precision=prec, stream=stream)
            if args.tiles:
                batch.set_tiles(json.loads(args.tiles))
                tiles = batch.tiles()
            else:
                tiles = batch.autotune(5)
            if args.persistent:
                batch.set_persistent(True)
            units_per_inner = batch.info()["dofs"]
            launches_per_step = batch.launches_per_step() * args.inner
        else:
            for c in cases:
                s, V0, _ = G.solver_from_case(c, precision=prec, stream=stream)
                solvers.append(s)
                V0s.append(V0)
            units_per_inner = sum(s.K * s.Np * s.nV for s in solvers)
            launches_per_step = sum(s.launches_per_step() for s in solvers) * args.inner
    units_per_step = units_per_inner * args.inner

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def one_step():
        if batch is not None:
            batch.advance(args.inner)
        else:
            for s in solvers:
                s.advance(args.inner)

    class _NoClock:
        def __enter__(self):
            return self

        def __exit__(self, *a):
            pass

        def summary(self):
            return None

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            one_step()
        stream.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        barrier()
        with (ClockSampler(local) if clocks else _NoClock()) as clk:
            for k in range(args.steps):
                flush.zero_()
                evs[k][0].record(stream)
                one_step()
                evs[k][1].record(stream)
            stream.synchronize()
        barrier()
    ms = [a.elapsed_time(b) for a, b in evs]
    total_ms = max_over_ranks(sum(ms), device="cuda")
    value = whole_job_throughput(units_per_step, args.steps, world, total_ms)
    stats = batch.stats() if batch is not None else [s.sync() for s in solvers]

    # ---- dominant kernel: live per-launch timing on the launching stream
    with torch.cuda.stream(stream):
        if batch is not None:
            groups = []
            for c in cases:
                key = (c.dim, c.order)
                if key not in [g[0] for g in groups]:
                    groups.append([key, 0])
                for g in groups:
                    if g[0] == key:
                        g[1] += c.etov.shape[0]
            kts = batch.time_kernels(10)
            gi = max(range(len(kts)), key=lambda i: kts[i]["volume"])
            kt = kts[gi]
            (dim, p), K = groups[gi]
        else:
            kt = solvers[min(3, len(solvers) - 1)].time_kernels(20)
            dim, p, K = cases[0].dim, cases[0].order, solvers[min(3, len(solvers) - 1)].K

    # ---- end to end through the public API with host buffers.  Every step
    # copies its input from pinned host memory and its result back; the copies
    # run on their own streams and overlap the compute of the neighbouring
    # steps (double-buffered device staging: the input of step k + 1 arrives
    # while step k computes, the result of step k leaves while step k + 1
    # computes).  Timed from the first input copy to the last result copy.
    e2e = None
    if e2e_on:
        pinned = [torch.from_numpy(np.ascontiguousarray(v)).pin_memory() for v in V0s]
        out_host = [torch.empty_like(x).pin_memory() for x in pinned]
        dev_in = [[torch.empty_like(x, device="cuda") for x in pinned] for _ in range(2)]
        dev_out = [[torch.empty_like(x, device="cuda") for x in pinned] for _ in range(2)]
        h2d = sum(x.numel() * 8 for x in pinned)
        ch, cd = torch.cuda.Stream(), torch.cuda.Stream()
        K_ = args.steps
        ev = lambda: torch.cuda.Event()
        in_done, used, res, out_done = ([ev() for _ in range(K_)] for _ in range(4))
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

        def h2d_copy(k):
            with torch.cuda.stream(ch):
                if k >= 2:
                    ch.wait_event(used[k - 2])
                for i in range(len(V0s)):
                    dev_in[k % 2][i].copy_(pinned[i], non_blocking=True)
                in_done[k].record(ch)

        barrier()
        with torch.cuda.stream(stream):
            t0.record(stream)
            ch.wait_event(t0)
            cd.wait_event(t0)
            h2d_copy(0)
            for k in range(K_):
                if k + 1 < K_:
                    h2d_copy(k + 1)
                stream.wait_event(in_done[k])
                for i in range(len(V0s)):
                    if batch is not None:
                        batch.set_state(i, dev_in[k % 2][i])
                    else:
                        solvers[i].set_state(dev_in[k % 2][i])
                used[k].record(stream)
                one_step()
                if k >= 2:
                    stream.wait_event(out_done[k - 2])
                for i in range(len(V0s)):
                    if batch is not None:
                        batch.get_state_device(i, dev_out[k % 2][i])
                    else:
                        solvers[i].get_state_device(dev_out[k % 2][i])
                res[k].record(stream)
                with torch.cuda.stream(cd):
                    cd.wait_event(res[k])
                    for i in range(len(V0s)):
                        out_host[i].copy_(dev_out[k % 2][i], non_blocking=True)
                    out_done[k].record(cd)
            stream.wait_event(out_done[K_ - 1])
            t1.record(stream)
            stream.synchronize()
        barrier()
        e_ms = max_over_ranks(t0.elapsed_time(t1), device="cuda")
        e2e = {"value": units_per_step * args.steps * world / (e_ms / 1e3), "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": h2d,
               "note": "per step: pinned host->device copy of every instance's state, set_state, advance, "
                       "get_state, device->host copy; the copies run on two copy streams, overlapping the "
                       "neighbouring steps' compute (double-buffered device staging)"}
        del pinned, out_host, dev_in, dev_out
    final = None
    if compare_steps > 0:
        with torch.cuda.stream(stream):
            for i, v in enumerate(V0s):
                if batch is not None:
                    batch.set_state(i, v)
                else:
                    solvers[i].set_state(v)
            if batch is not None:
                batch.run(compare_steps)
                final = torch.empty(batch.shapes[0], dtype=torch.float64, device="cuda")
                batch.get_state_device(0, final)
            else:
                solvers[0].run(compare_steps)
                final = torch.empty((solvers[0].nV, solvers[0].K, solvers[0].Np), dtype=torch.float64,
                                    device="cuda")
                solvers[0].get_state_device(final)
            stream.synchronize()
    for s in solvers:
        s.close()
    if batch is not None:
        batch.close()
    return dict(value=value, total_ms=total_ms, stats=stats, kt=kt, dim=dim, p=p, K=K, tiles=tiles,
                e2e=e2e, clk=clk.summary(), launches=launches_per_step * args.steps, n_inst=len(V0s),
                final=final)


def roofline(r, prec, G, args, peaks_derived, peaks_probe, batch_mode):
    """Roofline object of the dominant (volume) kernel: the FP64 or FP32
    pipe at algorithmic flops, with HBM at algorithmic bytes beside it."""
    dim, p, K, kt = r["dim"], r["p"], r["K"], r["kt"]
    vol_ms = kt["volume"]
    rs = 8 if prec == G.PREC_FP64 else 4
    key = "fp64" if rs == 8 else "fp32"
    flops = volume_flops(dim, p) * K
    achieved_tf = flops / (vol_ms * 1e-3) / 1e12
    pk, pk_kind = peaks()
    vbytes = volume_bytes(dim, p, rs) * K
    peak = peaks_derived[key]
    tcf = prec == G.PREC_FP32_TC and dim == 2 and p >= 2
    wl_key = f"{args.workload}_{args.mode}_{'fp64' if rs == 8 else ('fp32tc' if tcf else 'fp32')}"
    kname = (f"volume_tc_kernel<{p},{'true' if batch_mode else 'false'}>" if tcf else
             f"volume_kernel<{dim},{p},{'double' if rs == 8 else 'float'},{'true' if batch_mode else 'false'}>")
    if args.workload == "drybed":
        # wet/dry mode: the volume pass is the residual (volume kernel, mode 2)
        # plus the FP64 conservative stage kernel; kernel_ms covers both
        kname = f"{kname} (residual) + wetdry_stage_kernel<{dim},{p},{'double' if rs == 8 else 'float'}>"
    return {"bound": "alu", "kernel": kname,
            "achieved": achieved_tf, "peak": peak, "unit": "TFLOP/s", "frac": achieved_tf / peak,
            "peak_source": (f"{'FP64' if rs == 8 else 'FP32'} pipe from unit counts: SMs x "
                            f"{2 if rs == 8 else 128} FMA lanes/SM/clk x 2 flop x {SM_MAX_MHZ:g} MHz"),
            "peak_probe": peaks_probe[key], "frac_of_probe": achieved_tf / peaks_probe[key],
            "traffic": traffic_record("volume_kernel", wl_key),
            "elements_per_launch": K,
            "algorithmic_flops_per_launch": flops, "algorithmic_bytes_per_launch": vbytes,
            "hbm_gbs_at_algorithmic_bytes": vbytes / (vol_ms * 1e-3) / 1e9,
            "hbm_frac": vbytes / (vol_ms * 1e-3) / 1e9 / pk["hbm_gbs"], "hbm_peak_source": pk_kind,
            "kernel_ms": kt}


def accuracy_vs_oracle(args, G, prec, stream, res, sdesc, sc):
    import numpy as np
    import torch
    with torch.cuda.stream(stream):
        s_acc, _, _ = G.solver_from_case(sc, precision=prec, stream=stream)
        s_acc.run(res["steps"])
        Vg = s_acc.get_state(with_E=False)
        s_acc.close()
    Vo = np.asarray(res["final"])
    return {"rel_l2_vs_fp64_oracle": float(np.linalg.norm(Vg - Vo) / np.linalg.norm(Vo)),
            "after_steps": res["steps"], "case": sdesc,
            "precision": {G.PREC_FP64: "fp64", G.PREC_FP32: "fp32", G.PREC_FP32_TC: "fp32tc"}[prec],
            "sigma0": sc.params["sigma0"], "regularization": sc.params["reg"]}


def main():
    args = parse()
    if args.oracle_worker:
        oracle_worker(args.oracle_worker)
        return
    if args.impl == "reference":
        reference_main(args)
        return
    import torch
    import torch.distributed as dist
    import paper_2301_11238_gb300 as G
    if args.workload == "implicit_dam":
        implicit_main(args)
        return
    if args.workload == "newton2d":
        newton_main(args)
        return

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    prec = {"fp64": G.PREC_FP64, "fp32": G.PREC_FP32, "fp32tc": G.PREC_FP32_TC}[args.precision]
    stream = torch.cuda.Stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    cases = workload_cases(args)
    # the mixed-precision companion run of the FP64 headline (same mesh and
    # physics in FP32) and the full-size FP64-vs-FP32 comparison
    mixed_on = args.precision == "fp64" and args.workload == "slump" and not args.no_mixed
    cmp_steps = args.compare_steps if mixed_on else 0
    r = measure(args, G, cases, prec, stream, flush, world, local, e2e_on=not args.no_e2e,
                compare_steps=cmp_steps)
    # pipe peaks measured right after the timed work, with the GPU's clocks up
    peaks_derived, peaks_probe, sms = pipe_peaks(G, stream)
    roof = roofline(r, prec, G, args, peaks_derived, peaks_probe, args.mode == "batch")
    final64 = r.pop("final")

    mixed = None
    if mixed_on:
        r32 = measure(args, G, cases, G.PREC_FP32, stream, flush, world, local, clocks=True,
                      e2e_on=not args.no_e2e, compare_steps=cmp_steps)
        final32 = r32.pop("final")
        diff = float(torch.linalg.vector_norm(final32 - final64) / torch.linalg.vector_norm(final64))
        del final32
        mixed = {"precision": "fp32 state and arithmetic; FP64 step-size and mass reductions",
                 "value": r32["value"], "unit": UNIT, "ms_per_step": r32["total_ms"] / args.steps,
                 "speedup_vs_fp64": r32["value"] / r["value"],
                 "roofline": roofline(r32, G.PREC_FP32, G, args, peaks_derived, peaks_probe, args.mode == "batch"),
                 "e2e": r32["e2e"], "gpu_launches": r32["launches"], "clocks": r32["clk"], "tiles": r32["tiles"],
                 "rel_l2_vs_gpu_fp64_full_size": diff, "compare_steps": cmp_steps}
    del final64

    # ---- accuracy and CPU baseline (rank 0, N=1 only)
    cpu = None
    acc = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        res = run_oracle_subprocess(args.workload, args.n, args.order, seconds=args.oracle_seconds, min_steps=2,
                                    return_state=True)
        sc, sdesc = sample_case(args.workload, args.n, args.order)
        cpu = {"value": res["units_per_step"] * res["steps"] / res["seconds"], "unit": UNIT, "cores": 1,
               "kind": "oracle",
               "sample": f"{res['steps']} SSP-RK3 steps of {sdesc}, {res['seconds']:.1f} s on one host core"}
        acc = accuracy_vs_oracle(args, G, prec, stream, res, sdesc, sc)
        if mixed is not None:
            mixed["accuracy"] = accuracy_vs_oracle(args, G, G.PREC_FP32, stream, res, sdesc, sc)

    stats = r["stats"]
    dt_info = ({f"sigma0={c.params['sigma0']},reg={c.params['reg']}": st["dt_last"]
                for c, st in zip(cases, stats)} if len(cases) <= 16 else
               {"min": min(st["dt_last"] for st in stats), "max": max(st["dt_last"] for st in stats)})
    line = {"metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": r["total_ms"] / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if prec == G.PREC_FP64 else "f32",
            "data": "synthetic",
            "config": {"workload": workload_name(args), "instances": r["n_inst"],
                       "elements_total": int(sum(c.etov.shape[0] for c in cases)), "mode": args.mode,
                       "tiles": r["tiles"],
                       "inner_rk3_steps_per_step": args.inner, "l2": "flushed (256 MiB write) before each step",
                       "launch": "persistent (one launch per group and step)" if args.persistent else
                                 "graph of 11 launches per group and step",
                       "parallelism": f"replicas x{world}", "dt_last": dt_info,
                       "simulated_time_per_step": {k: v * args.inner for k, v in dt_info.items()},
                       "sms": sms},
            "roofline": roof, "cpu_baseline": cpu, "e2e": r["e2e"], "gpu_launches": r["launches"],
            "clocks": r["clk"], "accuracy": acc, "mixed": mixed}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
