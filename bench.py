"""Benchmark: solid Newton steps per second on the two-layer artery tube.

Workload (per GPU): artery tube, inner radius 1.0, media 0.13 (4 element
layers), adventitia 0.10 (4 layers), length 8, 64 x 8 x 128 hexahedra x 6
tetrahedra = 393,216 elements, 74,304 nodes, 297,216 unknowns; c10 = 3.0 /
0.3, k1 = 2.3 / 0.56, k2 = 0.84 / 0.71, fibres at +-29 / +-62 degrees,
kappa = 1e3 c10 (media); ends fixed axially; internal pressure ramped
0 -> 1.6 in 10 load steps (synthetic, seeded geometry: no dataset).

One bench step = one call of fsi_solid_newton_step: FP64 residual, tangent
assembly, numeric AMG set-up, FGMRES + AMG V-cycle to a relative residual of
1e-8, update.  The load advances when a step starts from a converged state;
after the last load step the ramp restarts from the reference state.  The
matrix, hierarchy and Krylov basis (~1 GB) are far larger than the 129 MB L2,
so no explicit flush is done between steps.

--impl reference times the FP64 CPU oracle (the only reference this method
has) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "solid Newton steps/s (assemble+AMG-Krylov to 1e-8)"
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}
FP64_PEAK_TFLOPS = 1.196      # project-measured dependent-FMA rate on this GB300 (FP64 pipe)
N_LOADS = 10
P_MAX = 1.6


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return PEAKS_FALLBACK, "fallback"


def workload_mesh(nz=128, config="tube", nseg=256):
    from fixtures import artery_layers, artery_tube, batched_tubes
    if config == "batched":
        return batched_tubes(n_seg=nseg, seed=4)
    if config == "refined":
        return artery_tube(n_theta=128, n_media=8, n_adv=8, n_z=2 * nz, length=8.0 * nz / 128,
                           materials=artery_layers(1.0e5))
    return artery_tube(n_theta=64, n_media=4, n_adv=4, n_z=nz, length=8.0 * nz / 128,
                       materials=artery_layers(1.0e3))


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""

    def __init__(self, index=0):
        self.index = index
        self.samples = []
        self._stop = threading.Event()
        self._thr = None

    def start(self):
        def run():
            q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
            while not self._stop.is_set():
                try:
                    out = subprocess.run(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits"], capture_output=True, text=True,
                                         timeout=5).stdout.strip()
                    if out:
                        self.samples.append([x.strip() for x in out.split(",")])
                except Exception:
                    pass
                self._stop.wait(0.2)
        self._thr = threading.Thread(target=run, daemon=True)
        self._thr.start()

    def stop(self):
        self._stop.set()
        if self._thr:
            self._thr.join(timeout=10)
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for s in self.samples for k in range(4) if "Active" in s[2 + k]
                          and "Not" not in s[2 + k]})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def max_over_ranks(x, world, device="cuda"):
    """The largest value of x over all ranks (the step time every rank waits for)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(steps_per_s_max_time, world):
    """Whole-job throughput of N independent replicas: N x the per-replica rate
    measured with the slowest rank's time."""
    return steps_per_s_max_time * world


# ------------------------------------------------------------------ GPU arm
# DRAM bytes (read + write) per launch of the finest-level block-Jacobi sweep,
# from the ncu full capture summarised in profiles/jacobi0_tube393k_full.md
# (393k-tet tube, FP32 values).  Reset to None whenever that kernel changes.
JACOBI0_TRAFFIC = {("tube", 128, "fp32"): 79_937_664}


def jacobi0_bytes(n, nb, fp32):
    """Algorithmic bytes of one finest-level damped block-Jacobi sweep:
    4x4 values + column index per block, row pointer, x / b / y vectors and
    the 4x4 inverse per block row."""
    vb = 4 if fp32 else 8
    return nb * (16 * vb + 4) + (n + 1) * 4 + n * (3 * 4 * vb + 16 * vb)


class RampDriver:
    """Advances the pressure ramp between Newton steps."""

    def __init__(self, solver, n, torch, face_pressure=None):
        from paper_1312_5561_gb300.binding import Load
        self.Load = Load
        self.fp = None if face_pressure is None else torch.tensor(face_pressure, device="cuda", dtype=torch.float64)
        self.solver = solver
        self.torch = torch
        self.state = torch.zeros((n, 4), device="cuda", dtype=torch.float64)
        self.k = 1
        self.r0 = None
        self.newton_in_load = 0
        self.krylov_cap_hits = 0       # Newton steps whose linear solve ended at max_krylov above tolerance

    def step(self, state=None):
        st = self.state if state is None else state
        scale = (P_MAX if self.fp is None else 1.0) * self.k / N_LOADS
        info = self.solver.newton_step(st, self.Load(pressure=scale, face_pressure=self.fp), check=False)
        if info.status not in (0, -5):
            raise RuntimeError(f"newton_step failed with status {info.status}")
        self.krylov_cap_hits += info.status == -5
        if self.r0 is None:
            self.r0 = info.res0
        self.newton_in_load += 1
        if info.res0 <= 1e-8 * self.r0 or self.newton_in_load > 12:
            self.k += 1
            self.r0 = None
            self.newton_in_load = 0
            if self.k > N_LOADS:
                self.k = 1
                st.zero_()
        return info


def run_gpu(args, rank, world):
    import torch
    from paper_1312_5561_gb300.binding import SolidSolver, launch_count
    torch.cuda.set_device(args.local_rank)
    mesh = workload_mesh(args.nz, args.config, args.nseg)
    prec = 1 if args.precision == "fp32" else 0
    t_create = time.perf_counter()
    # fgmres-amg: FGMRES(100) + one AMG V-cycle on the whole u-p tangent;
    # bicgstab-pl: the paper's solid solver, BiCGStab + block-triangular P_L (Sec. 5.4.2)
    kry = dict(krylov=1, precond=1, max_krylov=3000) if args.solver == "bicgstab-pl" else dict(max_krylov=600)
    if args.coarse_bf16:
        kry.update(coarse_bf16=1)
    agg = args.aggregation or ("grow" if args.config == "refined" else "ring")
    kry.update(aggregation=1 if agg == "grow" else 0)
    if args.smoother == "vanka":       # the paper's Vanka smoother on the finest level (Sec. 5.5.2)
        kry.update(smoother=1, vanka_omega=0.86, nu_pre=args.nu, nu_post=args.nu)
    solver = SolidSolver(mesh, precision=prec, newton_rtol=1e-8, krylov_rtol=1e-8, use_graphs=int(args.graphs),
                         amg_lag=int(args.amg_lag), **kry)
    t_create = time.perf_counter() - t_create
    levels = solver.levels()
    drv = RampDriver(solver, mesh.n_nodes, torch, getattr(mesh, "face_pressure", None))
    for _ in range(args.warmup):
        drv.step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    l0 = launch_count()
    clocks = ClockSampler(args.local_rank)
    clocks.start()
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    krylov = 0
    caps0 = drv.krylov_cap_hits
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(args.steps):
        info = drv.step()
        krylov += info.krylov_its_last
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    launches = launch_count() - l0
    cap_hits = drv.krylov_cap_hits - caps0
    ms_total = ev0.elapsed_time(ev1)
    # kernel-timing pass: the same Newton steps continued, with CUDA events recorded
    # on the launching stream around every launch (the V-cycle is then launched
    # kernel by kernel instead of from its graph)
    solver.kernel_timing(True)
    for _ in range(args.prof_steps):
        drv.step()
    torch.cuda.synchronize()
    prof = solver.kernel_timing(False)
    ms_total = max_over_ranks(ms_total, world)
    steps_per_s = args.steps / (ms_total * 1e-3)

    # element tangents / s (residual + tangent assembly, device resident)
    st = drv.state
    for _ in range(2):
        solver.residual_tangent(st)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 5
    e0.record(stream)
    for _ in range(reps):
        solver.residual_tangent(st)
    e1.record(stream)
    torch.cuda.synchronize()
    tangents_per_s = mesh.n_elems * reps / (e0.elapsed_time(e1) * 1e-3)

    # end to end through the C ABI with host buffers (pinned), copies timed
    host = torch.zeros((mesh.n_nodes, 4), dtype=torch.float64).pin_memory()
    host.copy_(drv.state.cpu())
    dev = torch.empty_like(drv.state)
    e_steps = max(3, args.steps // 2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e_steps):
        dev.copy_(host, non_blocking=True)
        drv.step(dev)
        host.copy_(dev, non_blocking=True)
        torch.cuda.current_stream().synchronize()
    e2e = e_steps / (time.perf_counter() - t0)
    nbytes = mesh.n_nodes * 4 * 8

    L0n, L0nb = levels[0]
    dominant = max(prof, key=lambda k: prof[k][0])
    peaks, src = _peaks()
    roof = None
    jt, jc = prof["jacobi0"]
    if jc > 0 and args.smoother != "vanka":   # with Vanka this class holds the patch sweeps
        per_launch_s = jt * 1e-3 / jc
        byt = jacobi0_bytes(L0n, L0nb, prec == 1)
        ach = byt / per_launch_s / 1e9
        roof = {"kernel": "bsr_kernel<...,4,4,MODE=2> (finest-level block-Jacobi sweep)", "bound": "hbm",
                "achieved": round(ach, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": round(ach / peaks["hbm_gbs"], 3),
                "traffic": JACOBI0_TRAFFIC.get((args.config, args.nz, args.precision)), "peak_source": src,
                "bytes_per_launch": int(byt), "avg_launch_us": round(per_launch_s * 1e6, 2),
                "timing": f"CUDA events around each launch over a {args.prof_steps}-step kernel-timing pass "
                          f"following the timed region (same workload, V-cycle launched eagerly)"}
    return {
        "steps_per_s": steps_per_s, "ms_per_step": ms_total / args.steps, "tangents_per_s": tangents_per_s,
        "e2e_steps_per_s": e2e, "bytes": nbytes, "launches": launches, "clocks": clk,
        "prof": {k: [round(v[0], 3), v[1]] for k, v in prof.items()}, "dominant": dominant, "roofline": roof,
        "krylov_per_step": krylov / args.steps, "krylov_cap_hits": cap_hits, "levels": levels, "n_elems": mesh.n_elems,
        "n_nodes": mesh.n_nodes, "create_s": t_create,
    }


# ------------------------------------------------------------------ oracle (CPU) arm
_ORACLE_SNIPPET = r"""
import json, sys, time
sys.path.insert(0, {root!r})
import numpy as np
import scipy.sparse.linalg as spla
from fixtures import artery_layers, artery_tube
from oracle import solid as O
nz, steps, warm = {nz}, {steps}, {warm}
mesh = artery_tube(n_theta=64, n_z=nz, length=8.0 * nz / 128, materials=artery_layers(1.0e3))
P = O.Problem(mesh)
state = np.zeros((mesh.n_nodes, 4))
fext = P.external_force(0.16)
times = []
for k in range(warm + steps):
    t0 = time.perf_counter()
    R = P.residual(state, fext)
    K = P.tangent(state)
    dv = spla.spsolve(K.tocsc(), -R.ravel())
    state = state + dv.reshape(-1, 4)
    times.append(time.perf_counter() - t0)
idx = np.arange(min(mesh.n_elems, 4096))
t0 = time.perf_counter(); P.element_tangents(state, idx); tt = time.perf_counter() - t0
print(json.dumps({{"n_elems": mesh.n_elems, "step_s": float(np.mean(times[warm:])), "tangent_s": tt / len(idx)}}))
"""


def run_oracle(nz_sample, steps, warm):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = _ORACLE_SNIPPET.format(root=ROOT, nz=nz_sample, steps=steps, warm=warm)
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=1800)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


def oracle_line(args, full_elems, nz_sample, steps, warm):
    r = run_oracle(nz_sample, steps, warm)
    scale = full_elems / r["n_elems"]
    value = 1.0 / (r["step_s"] * scale)
    return {
        "value": value, "unit": "steps/s", "cores": 1, "kind": "oracle",
        "sample": (f"FP64 oracle Newton step (complex-step tangent, scipy sparse direct solve) on the first "
                   f"{r['n_elems']} elements (64x8x{nz_sample} slab) of the workload tube, time scaled by "
                   f"{scale:.0f} to the full mesh"),
        "tangents_per_s": 1.0 / r["tangent_s"],
    }


# ------------------------------------------------------------------ main
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--nz", type=int, default=128)
    ap.add_argument("--config", default="tube", choices=["tube", "batched", "refined"])
    ap.add_argument("--amg-lag", type=int, default=0, help="refresh the coarse AMG levels every (lag+1) steps")
    ap.add_argument("--nseg", type=int, default=256)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--single", action="store_true", help="skip the plain-FP64 comparison run")
    ap.add_argument("--graphs", type=int, default=1, help="replay the V-cycle from a captured CUDA graph")
    ap.add_argument("--prof-steps", type=int, default=6, help="Newton steps of the kernel-timing pass")
    ap.add_argument("--solver", default="fgmres-amg", choices=["fgmres-amg", "bicgstab-pl"])
    ap.add_argument("--smoother", default="jacobi", choices=["jacobi", "vanka"])
    ap.add_argument("--nu", type=int, default=1, help="Vanka sweeps before / after the coarse correction")
    ap.add_argument("--coarse-bf16", type=int, default=0, help="BF16 coarse-level operators in the V-cycle")
    ap.add_argument("--aggregation", default=None, choices=["ring", "grow"],
                    help="AMG aggregation (default: grow for the 16-layer refined tube, ring otherwise)")
    ap.add_argument("--compare-paper-solver", action="store_true",
                    help="also time BiCGStab + P_L (the paper's solid solver) on the same workload")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    args.local_rank = int(os.environ.get("LOCAL_RANK", 0))
    full_elems = 64 * 8 * args.nz * 6
    wl = (f"two-layer artery tube 64x8x{args.nz} hex x6 tets ({full_elems} tets), kappa=1e3*c10, "
          f"pressure ramp 0->1.6 in 10 load steps")
    if args.config == "refined":
        full_elems = 128 * 16 * 2 * args.nz * 6
        wl = (f"two-layer artery tube 128x16x{2 * args.nz} hex x6 tets ({full_elems} tets), kappa=1e5*c10, "
              f"pressure ramp 0->1.6 in 10 load steps")
    if args.config == "batched":
        wl = (f"{args.nseg} independent artery segments in one handle (seed 4): n_e logU[5e3,2e5], angles U[20,70], "
              f"kappa/c10 logU[1e2,1e5], pressure U[0.5,2.0] ramped in 10 load steps")
    config = {"workload": wl, "mesh_elems": full_elems,
              "l2": "inputs larger than L2 (matrix + AMG hierarchy + Krylov basis ~1 GB)", "parallelism": "replicas"}

    if args.impl == "reference":
        if rank != 0:
            return
        nz_s = 4
        line = oracle_line(args, full_elems, nz_s, args.steps, args.warmup)
        ms = 1e3 / line["value"]
        out = {"impl": "reference", "metric": METRIC, "value": line["value"], "unit": "steps/s",
               "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
               "data": "synthetic", "config": config,
               "cpu_baseline": {k: line[k] for k in ("value", "unit", "cores", "kind", "sample")},
               "e2e": {"value": line["value"], "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(out))
        return

    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    res = run_gpu(args, rank, world)
    other = None
    if args.precision == "fp32" and not args.single:
        a2 = argparse.Namespace(**vars(args))
        a2.precision = "fp64"
        a2.steps = max(5, args.steps // 2)
        other = run_gpu(a2, rank, world)
    paper = None
    if args.compare_paper_solver and args.solver != "bicgstab-pl":
        a3 = argparse.Namespace(**vars(args))
        a3.solver = "bicgstab-pl"
        a3.steps = max(5, args.steps // 2)
        paper = run_gpu(a3, rank, world)
    if rank != 0:
        return
    value = job_value(res["steps_per_s"], world)
    out = {
        "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": res["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64" if args.precision == "fp32" else "f64", "data": "synthetic",
        "config": dict(config, precision=("FP32 tangent + FP32 V-cycle under FP64 residual / outer FGMRES"
                                          if args.precision == "fp32" else "FP64 throughout"),
                       solver=("BiCGStab + block-triangular P_L (AMG V-cycle on A)" if args.solver == "bicgstab-pl"
                               else "FGMRES(100) + AMG V-cycle on K"),
                       finest_smoother=(f"Vanka, {args.nu}+{args.nu} sweeps, omega 0.86" if args.smoother == "vanka"
                                        else "damped block Jacobi, 4+4 sweeps, omega 0.7"),
                       coarse_operators="BF16 (V-cycle reads)" if args.coarse_bf16 else "FP32",
                       aggregation=(args.aggregation or ("grow" if args.config == "refined" else "ring")),
                       krylov_its_per_step=round(res["krylov_per_step"], 1),
                       krylov_cap_hits_in_timed_steps=res["krylov_cap_hits"], amg_levels=res["levels"]),
        "element_tangents_per_s": res["tangents_per_s"] * world,
        "e2e": {"value": res["e2e_steps_per_s"] * world, "unit": "steps/s",
                "h2d_bytes_per_step": res["bytes"], "d2h_bytes_per_step": res["bytes"]},
        "gpu_launches": res["launches"], "clocks": res["clocks"], "roofline": res["roofline"],
        "kernel_ms": res["prof"], "dominant_kernel_class": res["dominant"],
        "create_s": round(res["create_s"], 2),
    }
    if args.config == "batched":
        out["config"]["mesh_elems"] = res["n_elems"]
        out["segment_newton_steps_per_s"] = value * args.nseg
    if other is not None:
        out["plain_fp64"] = {"value": other["steps_per_s"] * world, "ms_per_step": other["ms_per_step"],
                             "element_tangents_per_s": other["tangents_per_s"] * world,
                             "krylov_its_per_step": round(other["krylov_per_step"], 1),
                             "speedup_vs_plain_fp64": res["steps_per_s"] / other["steps_per_s"],
                             "roofline": other["roofline"], "dominant_kernel_class": other["dominant"]}
    if paper is not None:
        out["paper_solver"] = {"solver": "BiCGStab + block-triangular P_L (Sec. 5.4.2), same precision",
                               "value": paper["steps_per_s"] * world, "ms_per_step": paper["ms_per_step"],
                               "krylov_its_per_step": round(paper["krylov_per_step"], 1),
                               "krylov_cap_hits_in_timed_steps": paper["krylov_cap_hits"],
                               "speedup_of_ours": res["steps_per_s"] / paper["steps_per_s"]}
    if not args.no_cpu_baseline and world == 1:
        try:
            out["cpu_baseline"] = oracle_line(args, full_elems, 4, 2, 1)
        except Exception as e:  # the GPU number stands without it
            out["cpu_baseline"] = {"error": str(e)[-300:]}
    print(json.dumps(out))


if __name__ == "__main__":
    main()
