"""Benchmark: solid Newton steps per second on the refined two-layer artery tube.

Workload (per GPU, default ``--config refined``): two-layer artery tube,
inner radius 1.0, media 0.13 (8 element layers), adventitia 0.10 (8 layers),
length 8, 128 x 16 x 256 hexahedra x 6 tetrahedra = 3,145,728 elements,
559,232 nodes, 2,236,928 unknowns; c10 = 3.0 / 0.3, k1 = 2.3 / 0.56,
k2 = 0.84 / 0.71, fibres at +-29 / +-62 degrees, kappa = 1e5 c10 (media);
ends fixed axially; internal pressure ramped 0 -> 1.6 in 10 load steps
(synthetic, seeded geometry: no dataset).  FP32 tangent and V-cycle under
the FP64 residual and FP64 outer FGMRES (iterative refinement); a plain-FP64
run of the same workload is timed beside it.  ``--config tube`` is the
64 x 8 x 128 tube (393,216 elements) at kappa = 1e3 c10; ``--config batched``
the 256 independent segments.

One bench step = one call of fsi_solid_newton_step: FP64 residual, tangent
assembly, numeric AMG set-up, FGMRES + AMG V-cycle to a relative residual of
1e-8, update.  The load advances when a step starts from a converged state
(relative residual 1e-8) or after 12 Newton steps (counted as a Newton cap
hit); after the last load step the ramp restarts from the reference state.
The matrix, hierarchy and Krylov basis (several GB) are far larger than the
129 MB L2, so no explicit flush is done between steps.

Accuracy is reported beside the throughput: the error of the same solver
against stored FP64 oracle solutions of a 98k-element section of the tube
(first load step, kappa 1e3 and 1e5 c10), and on the timed workload itself
the oracle's own residual at the GPU's converged first load step (the
oracle's Newton solve does not finish in hours at 3.1M elements).

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
N_LOADS = 10
P_MAX = 1.6
NEWTON_CAP = 12
GOLDEN_DIR = os.path.join(ROOT, "tests", "golden")


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return PEAKS_FALLBACK, "fallback"


def workload_mesh(nz=128, config="refined", nseg=256):
    from fixtures import artery_layers, artery_tube, batched_tubes
    if config == "batched":
        return batched_tubes(n_seg=nseg, seed=4)
    if config == "refined":
        return artery_tube(n_theta=128, n_media=8, n_adv=8, n_z=2 * nz, length=8.0 * nz / 128,
                           materials=artery_layers(1.0e5))
    return artery_tube(n_theta=64, n_media=4, n_adv=4, n_z=nz, length=8.0 * nz / 128,
                       materials=artery_layers(1.0e3))


def solver_options(args):
    """Solver options of the timed workload (everything else is the library default:
    FGMRES(100), block Jacobi 4+4 on the finest level, minimal-residual block
    Jacobi 2+2 on the coarser levels, V-cycle replayed from a CUDA graph)."""
    prec = 1 if args.precision == "fp32" else 0
    kry = dict(krylov=1, precond=1, max_krylov=3000) if args.solver == "bicgstab-pl" else dict(max_krylov=600)
    if args.coarse_bf16:
        kry.update(coarse_bf16=1)
    kry.update(aggregation=1 if aggregation_of(args) == "grow" else 0)
    if args.smoother == "vanka":       # the paper's Vanka smoother on the finest level (Sec. 5.5.2)
        kry.update(smoother=1, vanka_omega=0.86, nu_pre=args.nu, nu_post=args.nu)
    if args.coarse_jacobi:
        kry.update(coarse_smoother=0, nu_coarse=1)
    kry.update(segment_krylov=int(args.segment_krylov))
    if args.exact_candidates:
        kry.update(exact_candidates=1)
    if args.power_steps != 20:
        kry.update(power_steps=args.power_steps)
    if args.nu_finest > 0 and args.smoother != "vanka":
        kry.update(nu_pre=args.nu_finest, nu_post=args.nu_finest)
    return dict(precision=prec, newton_rtol=1e-8, krylov_rtol=1e-8, use_graphs=int(args.graphs),
                amg_lag=int(args.amg_lag), **kry)


def aggregation_of(args):
    return args.aggregation or ("grow" if args.config == "refined" else "ring")


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
# DRAM bytes (read + write) per launch of the finest-level block-Jacobi sweep
# from ncu captures of that kernel (FP32 values); the entry is removed whenever
# the kernel changes.  393k tube: captured on the workload itself.  3.1M tube:
# captured on the same tube shortened to 64 axial cells (2,038,144 blocks,
# 156.77 MB per launch = 1.011 x its algorithmic bytes) and scaled by the block
# count to 8,108,416 blocks (traffic grows in proportion to the blocks).
JACOBI0_TRAFFIC = {("tube", 128, "fp32"): 79_937_664, ("refined", 128, "fp32"): 623_688_583}


def level1_spmv_bytes(n, nb, fp32, bf16=False):
    """Algorithmic bytes of one w = A z product on AMG level 1 (7x7 blocks):
    values + column index per block, row pointer, z read and w written once."""
    vb = 2 if bf16 else (4 if fp32 else 8)
    xb = 4 if fp32 else 8
    return nb * (49 * vb + 4) + (n + 1) * 4 + 2 * n * 7 * xb


def jacobi0_bytes(n, nb, fp32):
    """Algorithmic bytes of one finest-level damped block-Jacobi sweep:
    4x4 values + column index per block, row pointer, x / b / y vectors and
    the 4x4 inverse per block row."""
    vb = 4 if fp32 else 8
    return nb * (16 * vb + 4) + (n + 1) * 4 + n * (3 * 4 * vb + 16 * vb)


class RampDriver:
    """Advances the pressure ramp between Newton steps."""

    def __init__(self, solver, n, torch, face_pressure=None, max_krylov=600, krylov_rtol=1e-8):
        from paper_1312_5561_gb300.binding import Load
        self.Load = Load
        self.fp = None if face_pressure is None else torch.tensor(face_pressure, device="cuda", dtype=torch.float64)
        self.solver = solver
        self.torch = torch
        self.state = torch.zeros((n, 4), device="cuda", dtype=torch.float64)
        self.k = 1
        self.r0 = None
        self.newton_in_load = 0
        self.max_krylov = max_krylov
        self.krylov_rtol = krylov_rtol
        self.krylov_cap_hits = 0       # linear solves that stopped at max_krylov above krylov_rtol
        self.newton_cap_hits = 0       # load steps left after NEWTON_CAP steps without reaching 1e-8

    def load(self, k):
        return self.Load(pressure=(P_MAX if self.fp is None else 1.0) * k / N_LOADS, face_pressure=self.fp)

    def step(self, state=None):
        st = self.state if state is None else state
        info = self.solver.newton_step(st, self.load(self.k), check=False)
        if info.status not in (0, -5):
            raise RuntimeError(f"newton_step failed with status {info.status}")
        if info.status == -5 or (info.krylov_its_last >= self.max_krylov and info.lin_res > self.krylov_rtol):
            self.krylov_cap_hits += 1
        if self.r0 is None:
            self.r0 = info.res0
        self.newton_in_load += 1
        converged = info.res0 <= 1e-8 * self.r0
        if converged or self.newton_in_load > NEWTON_CAP:
            self.newton_cap_hits += 0 if converged else 1
            self.k += 1
            self.r0 = None
            self.newton_in_load = 0
            if self.k > N_LOADS:
                self.k = 1
                st.zero_()
        return info


def golden_errors(args):
    """Error of the bench's solver settings against the stored FP64 oracle
    solutions of a quarter-length section of the 393k-element tube (64 x 8 x 32
    hexahedra, first load step P = 0.16): max |v - v_ref| / max |v_ref| per kappa
    ratio; None where a golden file is absent."""
    import torch
    from fixtures import artery_layers, artery_tube
    from paper_1312_5561_gb300.binding import Load, SolidSolver
    out = {}
    for ratio, name in ((1.0e3, "tube98k_k1e3_p016"), (1.0e5, "tube98k_k1e5_p016")):
        path = os.path.join(GOLDEN_DIR, name + ".npz")
        if not os.path.exists(path):
            out[name] = None
            continue
        ref = np.load(path)["state"]
        mesh = artery_tube(n_theta=64, n_media=4, n_adv=4, n_z=32, length=2.0, materials=artery_layers(ratio))
        a2 = argparse.Namespace(**vars(args))
        a2.config, a2.aggregation = "tube", None
        solver = SolidSolver(mesh, **solver_options(a2))
        state = torch.zeros((mesh.n_nodes, 4), device="cuda", dtype=torch.float64)
        info = solver.solve(state, Load(pressure=0.16), check=False)
        got = state.cpu().numpy()
        out[name] = {"rel_err": float(np.abs(got - ref).max() / np.abs(ref).max()), "status": int(info.status),
                     "newton_its": int(info.newton_its)}
        solver.close()
    return out


def run_gpu(args, rank, world, verify_path=None):
    import torch
    from paper_1312_5561_gb300.binding import SolidSolver, launch_count
    torch.cuda.set_device(args.local_rank)
    mesh = workload_mesh(args.nz, args.config, args.nseg)
    opts = solver_options(args)
    prec = opts["precision"]
    t_create = time.perf_counter()
    solver = SolidSolver(mesh, **opts)
    t_create = time.perf_counter() - t_create
    levels = solver.levels()
    tuning = solver.tuning()
    drv = RampDriver(solver, mesh.n_nodes, torch, getattr(mesh, "face_pressure", None), opts["max_krylov"],
                     opts["krylov_rtol"])
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
    caps0, ncaps0 = drv.krylov_cap_hits, drv.newton_cap_hits
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(args.steps):
        info = drv.step()
        krylov += info.krylov_its_last
    ev1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    launches = launch_count() - l0
    cap_hits = drv.krylov_cap_hits - caps0
    newton_caps = drv.newton_cap_hits - ncaps0
    ms_total = ev0.elapsed_time(ev1)
    # kernel-timing pass: the same Newton steps continued, with CUDA events recorded
    # on the launching stream around every launch (the V-cycle is then launched
    # kernel by kernel instead of from its graph)
    prof = {}
    if args.prof_steps > 0:
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
    e_steps = max(3, args.steps // 2) if args.e2e_steps < 0 else args.e2e_steps
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e_steps):
        dev.copy_(host, non_blocking=True)
        drv.step(dev)
        host.copy_(dev, non_blocking=True)
        torch.cuda.current_stream().synchronize()
    e2e = e_steps / (time.perf_counter() - t0) if e_steps > 0 else None
    nbytes = mesh.n_nodes * 4 * 8

    # the converged first load step, for the oracle's residual check (cpu_baseline leg)
    verify = None
    if verify_path is not None:
        vstate = torch.zeros((mesh.n_nodes, 4), device="cuda", dtype=torch.float64)
        vinfo = solver.solve(vstate, drv.load(1), check=False)
        v = vstate.cpu().numpy()
        verify = {"status": int(vinfo.status), "newton_its": int(vinfo.newton_its),
                  "gpu_rel_res": float(vinfo.res / vinfo.res0) if vinfo.res0 > 0 else 0.0,
                  "pressure": P_MAX / N_LOADS}
        if args.config == "batched":
            # the two smallest segments, whose oracle solves take seconds
            sizes = [sg["n_elems"] for sg in mesh.meta["segments"]]
            pick = [int(i) for i in np.argsort(sizes)[:2]]
            np.savez(verify_path + ".npz", **{f"seg{i}": v[mesh.seg_node == i] for i in pick})
            verify.update(segments=pick, pressure=1.0 / N_LOADS)
        else:
            np.save(verify_path, v)

    L0n, L0nb = levels[0]
    dominant = max(prof, key=lambda k: prof[k][0]) if prof else None
    peaks, src = _peaks()
    timing = (f"CUDA events around each launch over a {args.prof_steps}-step kernel-timing pass following the "
              f"timed region (same workload, V-cycle launched eagerly)")
    roofs = {}
    jt, jc = prof.get("jacobi0", (0.0, 0))
    if jc > 0 and args.smoother != "vanka":   # with Vanka this class holds the patch sweeps
        per_launch_s = jt * 1e-3 / jc
        byt = jacobi0_bytes(L0n, L0nb, prec == 1)
        ach = byt / per_launch_s / 1e9
        roofs["jacobi0"] = (jt, {
            "kernel": "bsr_kernel<...,4,4,MODE=2> (finest-level block-Jacobi sweep)", "bound": "hbm",
            "achieved": round(ach, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": round(ach / peaks["hbm_gbs"], 3),
            "traffic": JACOBI0_TRAFFIC.get((args.config, args.nz, args.precision)), "peak_source": src,
            "bytes_per_launch": int(byt), "avg_launch_us": round(per_launch_s * 1e6, 2),
            "class_ms_per_step": round(jt / args.prof_steps, 2), "timing": timing})
    lt, lc = prof.get("level1_spmv", (0.0, 0))
    if lc > 0 and len(levels) > 1:
        per_launch_s = lt * 1e-3 / lc
        L1n, L1nb = levels[1]
        byt = level1_spmv_bytes(L1n, L1nb, prec == 1, bool(args.coarse_bf16))
        ach = byt / per_launch_s / 1e9
        roofs["level1_spmv"] = (lt, {
            "kernel": "bsr7_kernel<...,7,MODE=0> (w = A z on AMG level 1 in the minimal-residual sweeps)",
            "bound": "hbm", "achieved": round(ach, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": round(ach / peaks["hbm_gbs"], 3), "traffic": None, "peak_source": src,
            "bytes_per_launch": int(byt), "avg_launch_us": round(per_launch_s * 1e6, 2),
            "class_ms_per_step": round(lt / args.prof_steps, 2), "timing": timing})
    # the line's roofline is the kernel with the larger share of the step; the other is reported beside it
    order = sorted(roofs.values(), key=lambda v: -v[0])
    roof = order[0][1] if order else None
    roof_other = order[1][1] if len(order) > 1 else None
    solver.close()
    return {
        "steps_per_s": steps_per_s, "ms_per_step": ms_total / args.steps, "tangents_per_s": tangents_per_s,
        "e2e_steps_per_s": e2e, "bytes": nbytes, "launches": launches, "clocks": clk,
        "prof": {k: [round(v[0], 3), v[1]] for k, v in prof.items()}, "dominant": dominant, "roofline": roof,
        "roofline_other": roof_other,
        "krylov_per_step": krylov / args.steps, "krylov_cap_hits": cap_hits, "newton_cap_hits": newton_caps,
        "levels": levels, "n_elems": mesh.n_elems, "n_nodes": mesh.n_nodes, "create_s": t_create,
        "verify": verify, "tuning": tuning,
    }


# ------------------------------------------------------------------ oracle (CPU) arm
# Sample of the oracle: full Newton steps (element residual, complex-step
# tangent, assembly, sparse direct solve) on an axial slab of the workload's
# cross-section (two axial cells), scaled to the full workload linearly in the
# element count.  The element work scales exactly so; the direct solve grows
# faster than linearly, so the scaled rate is an upper bound on the oracle's
# full-workload rate.
_ORACLE_SNIPPET = r"""
import json, sys, time
sys.path.insert(0, {root!r})
import numpy as np
import scipy.sparse.linalg as spla
from fixtures import artery_layers, artery_tube
from oracle import solid as O
nt, nr, ratio, slabs, steps, warm, full, nz_full = {nt}, {nr}, {ratio}, {slabs}, {steps}, {warm}, {full}, {nz_full}
out = {{"slabs": []}}
for nz in slabs:
    mesh = artery_tube(n_theta=nt, n_media=nr // 2, n_adv=nr // 2, n_z=nz, length=8.0 * nz / nz_full,
                       materials=artery_layers(ratio))
    P = O.Problem(mesh)
    state = np.zeros((mesh.n_nodes, 4))
    fext = P.external_force(0.16)
    te, ts, tt = [], [], []
    for k in range(warm + steps):
        t0 = time.perf_counter()
        R = P.residual(state, fext)
        K = P.tangent(state)
        t1 = time.perf_counter()
        dv = spla.spsolve(K.tocsc(), -R.ravel())
        state = state + dv.reshape(-1, 4)
        t2 = time.perf_counter()
        if k >= warm:
            te.append(t1 - t0); ts.append(t2 - t1); tt.append(t2 - t0)
    out["slabs"].append({{"nz": nz, "n_elems": mesh.n_elems, "elem_s": float(np.mean(te)), "solve_s": float(np.mean(ts)),
                         "step_s": float(np.mean(tt)), "steps_s": tt}})
a, b = out["slabs"][0], out["slabs"][-1]
if len(slabs) > 1:
    out["solve_exponent"] = float(np.log(b["solve_s"] / a["solve_s"]) / np.log(b["n_elems"] / a["n_elems"]))
out["elem_s_per_elem"] = b["elem_s"] / b["n_elems"]
out["full_step_s"] = b["step_s"] * full / b["n_elems"]
print(json.dumps(out))
"""

_RESIDUAL_SNIPPET = r"""
import json, sys, time
sys.path.insert(0, {root!r})
import numpy as np
from fixtures import artery_layers, artery_tube
from oracle import solid as O
v = np.load({path!r})
mesh = artery_tube(n_theta={nt}, n_media={nr} // 2, n_adv={nr} // 2, n_z={nz}, length=8.0, materials=artery_layers({ratio}))
P = O.Problem(mesh)
fext = P.external_force({pressure})
t0 = time.perf_counter()
r0 = float(np.linalg.norm(P.residual(np.zeros((mesh.n_nodes, 4)), fext)))
r = float(np.linalg.norm(P.residual(v, fext)))
print(json.dumps({{"oracle_rel_res": r / r0, "r0": r0, "r": r, "s": time.perf_counter() - t0}}))
"""


_SEGMENT_SNIPPET = r"""
import json, sys, time
sys.path.insert(0, {root!r})
import numpy as np
from fixtures import batched_segment
from oracle import solid as O
d = np.load({path!r} + ".npz")
out = {{}}
for i in {segments}:
    mesh, off = batched_segment(i, n_seg={nseg}, seed=4)
    P = O.Problem(mesh)
    fext = P.external_force({scale}, face_pressure=mesh.face_pressure)
    t0 = time.perf_counter()
    ref, its = P.newton(np.zeros((mesh.n_nodes, 4)), fext=fext, rtol=1e-12)
    got = d["seg%d" % i]
    out[str(i)] = {{"n_elems": int(mesh.n_elems), "kappa_ratio": float(mesh.meta["kappa_ratio"]),
                   "rel_err": float(np.abs(got - ref).max() / np.abs(ref).max()), "oracle_newton_its": int(its),
                   "oracle_s": time.perf_counter() - t0}}
print(json.dumps(out))
"""


def _workload_geometry(args):
    if args.config == "refined":
        return 128, 16, 2 * args.nz, 1.0e5
    return 64, 8, args.nz, 1.0e3


def _run_py(code, timeout=1800):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=timeout)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


def run_oracle(args, steps, warm, slabs=(2,)):
    nt, nr, nz, ratio = _workload_geometry(args)
    full = nt * nr * nz * 6
    code = _ORACLE_SNIPPET.format(root=ROOT, nt=nt, nr=nr, ratio=ratio, slabs=list(slabs), steps=steps, warm=warm,
                                  full=full, nz_full=nz)
    return _run_py(code), full


def oracle_line(args, steps, warm):
    r, full = run_oracle(args, steps, warm)
    b = r["slabs"][-1]
    return {
        "value": 1.0 / r["full_step_s"], "unit": "steps/s", "cores": 1, "kind": "oracle",
        "sample": (f"FP64 oracle Newton steps (element residual, complex-step tangent, sparse direct solve) on an "
                   f"axial slab of the workload tube ({b['n_elems']} elements: its full cross-section, two axial "
                   f"cells; load P = 0.16 from the reference state), one core; the step time is scaled to "
                   f"{full} elements linearly, an upper bound on the oracle's rate (its direct solve grows "
                   f"faster than linearly)"),
        "tangents_per_s": 1.0 / r["elem_s_per_elem"],
        "sample_ms_per_step": 1e3 * b["step_s"], "sample_step_times_s": b["steps_s"],
    }


def oracle_residual_check(args, verify_path, pressure):
    nt, nr, nz, ratio = _workload_geometry(args)
    code = _RESIDUAL_SNIPPET.format(root=ROOT, path=verify_path, nt=nt, nr=nr, nz=nz, ratio=ratio, pressure=pressure)
    return _run_py(code)


# ------------------------------------------------------------------ main
def make_parser():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--nz", type=int, default=128)
    ap.add_argument("--config", default="refined", choices=["refined", "tube", "batched"])
    ap.add_argument("--amg-lag", type=int, default=0, help="refresh the coarse AMG levels every (lag+1) steps")
    ap.add_argument("--nseg", type=int, default=256)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-golden", action="store_true", help="skip the error against the stored oracle solutions")
    ap.add_argument("--single", action="store_true", help="skip the plain-FP64 comparison run")
    ap.add_argument("--graphs", type=int, default=1, help="replay the V-cycle from a captured CUDA graph")
    ap.add_argument("--prof-steps", type=int, default=6, help="Newton steps of the kernel-timing pass (0: none)")
    ap.add_argument("--e2e-steps", type=int, default=-1,
                    help="Newton steps of the end-to-end pass (default max(3, steps // 2); 0: none)")
    ap.add_argument("--solver", default="fgmres-amg", choices=["fgmres-amg", "bicgstab-pl"])
    ap.add_argument("--smoother", default="jacobi", choices=["jacobi", "vanka"])
    ap.add_argument("--nu", type=int, default=1, help="Vanka sweeps before / after the coarse correction")
    ap.add_argument("--coarse-bf16", type=int, default=0, help="BF16 coarse-level operators in the V-cycle")
    ap.add_argument("--segment-krylov", type=int, default=1,
                    help="batched meshes: 1 = one Arnoldi process per segment, 0 = one over the union")
    ap.add_argument("--nu-finest", type=int, default=0,
                    help="block-Jacobi sweeps before / after on the finest level (0: the library default, 4)")
    ap.add_argument("--coarse-jacobi", action="store_true",
                    help="damped block Jacobi (1+1) on the coarse levels instead of minimal-residual block Jacobi")
    ap.add_argument("--aggregation", default=None, choices=["ring", "grow"],
                    help="AMG aggregation (default: grow for the 16-layer refined tube, ring otherwise)")
    ap.add_argument("--exact-candidates", action="store_true",
                    help="coarse near-null space from the whole QR factor of each aggregate (opts.exact_candidates)")
    ap.add_argument("--power-steps", type=int, default=20,
                    help="power-iteration steps for lambda_max(D^-1 A) of each AMG level (opts.power_steps)")
    ap.add_argument("--compare-paper-solver", action="store_true",
                    help="also time BiCGStab + P_L (the paper's solid solver) on the same workload")
    return ap


def main():
    args = make_parser().parse_args()
    args.warmup = max(args.warmup, 3)
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    args.local_rank = int(os.environ.get("LOCAL_RANK", 0))
    nt, nr, nz, ratio = _workload_geometry(args)
    full_elems = nt * nr * nz * 6
    wl = (f"two-layer artery tube {nt}x{nr}x{nz} hex x6 tets ({full_elems} tets), kappa={ratio:.0e}*c10, "
          f"pressure ramp 0->1.6 in 10 load steps")
    if args.config == "batched":
        wl = (f"{args.nseg} independent artery segments in one handle (seed 4): n_e logU[5e3,2e5], angles U[20,70], "
              f"kappa/c10 logU[1e2,1e5], pressure U[0.5,2.0] ramped in 10 load steps")
    config = {"workload": wl, "mesh_elems": full_elems,
              "l2": "inputs larger than L2 (matrix + AMG hierarchy + Krylov basis, several GB)",
              "parallelism": "replicas"}

    if args.impl == "reference":
        if rank != 0:
            return
        t0 = time.perf_counter()
        line = oracle_line(args, args.steps, args.warmup)
        out = {"impl": "reference", "metric": METRIC, "value": line["value"], "unit": "steps/s",
               "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
               "ms_per_step": line["sample_ms_per_step"], "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "f64", "data": "synthetic",
               "config": dict(config, reference_step=("one oracle Newton step on the sample slab; value = "
                                                       "the full-workload rate scaled from it")),
               "cpu_baseline": {k: line[k] for k in ("value", "unit", "cores", "kind", "sample")},
               "e2e": {"value": line["value"], "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
               "wall_s": round(time.perf_counter() - t0, 1)}
        print(json.dumps(out))
        return

    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    verify_path = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import tempfile
        verify_path = os.path.join(tempfile.mkdtemp(prefix="fsi_bench_"), "verify_state.npy")
    res = run_gpu(args, rank, world, verify_path)
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
    gold = None
    if rank == 0 and not args.no_golden:
        gold = golden_errors(args)
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
                                        else f"damped block Jacobi, {args.nu_finest or 4}+{args.nu_finest or 4} "
                                             f"sweeps, omega 0.7"),
                       coarse_smoother=("damped block Jacobi 1+1" if args.coarse_jacobi or args.solver == "bicgstab-pl"
                                        else "minimal-residual block Jacobi 2+2"),
                       coarse_operators="BF16 (V-cycle reads)" if args.coarse_bf16 else "FP32",
                       aggregation=aggregation_of(args),
                       coarse_candidates=("whole QR factor" if args.exact_candidates else
                                          "QR factor without dependent columns"),
                       power_steps=args.power_steps,
                       krylov=("per-segment FGMRES (one Arnoldi process per segment)"
                               if args.config == "batched" and args.segment_krylov and args.solver != "bicgstab-pl"
                               else None),
                       krylov_its_per_step=round(res["krylov_per_step"], 1),
                       krylov_cap_hits_in_timed_steps=res["krylov_cap_hits"],
                       newton_cap_hits_in_timed_steps=res["newton_cap_hits"], amg_levels=res["levels"]),
        "element_tangents_per_s": res["tangents_per_s"] * world,
        "e2e": ({"value": res["e2e_steps_per_s"] * world, "unit": "steps/s",
                 "h2d_bytes_per_step": res["bytes"], "d2h_bytes_per_step": res["bytes"]}
                if res["e2e_steps_per_s"] is not None else None),
        "gpu_launches": res["launches"], "clocks": res["clocks"], "roofline": res["roofline"],
        "roofline_second_kernel": res["roofline_other"],
        "kernel_ms": res["prof"], "dominant_kernel_class": res["dominant"],
        "create_s": round(res["create_s"], 2),
        "autotuned_launch_shapes": {"element_cta": res["tuning"][0], "levels": res["tuning"][1:],
                                    "meaning": "level 0: CTA size; coarser levels: 1 = CTA per block row, "
                                               "2 = warp per block row"},
    }
    if res["krylov_cap_hits"] or res["newton_cap_hits"]:
        out["warning"] = "some timed steps hit the Krylov or Newton cap: not a to-1e-8 number"
    if args.config == "batched":
        out["config"]["mesh_elems"] = res["n_elems"]
        out["segment_newton_steps_per_s"] = value * args.nseg
    if other is not None:
        out["plain_fp64"] = {"value": other["steps_per_s"] * world, "ms_per_step": other["ms_per_step"],
                             "element_tangents_per_s": other["tangents_per_s"] * world,
                             "krylov_its_per_step": round(other["krylov_per_step"], 1),
                             "krylov_cap_hits_in_timed_steps": other["krylov_cap_hits"],
                             "newton_cap_hits_in_timed_steps": other["newton_cap_hits"],
                             "speedup_vs_plain_fp64": res["steps_per_s"] / other["steps_per_s"],
                             "roofline": other["roofline"], "dominant_kernel_class": other["dominant"]}
    if paper is not None:
        out["paper_solver"] = {"solver": "BiCGStab + block-triangular P_L (Sec. 5.4.2), same precision",
                               "value": paper["steps_per_s"] * world, "ms_per_step": paper["ms_per_step"],
                               "krylov_its_per_step": round(paper["krylov_per_step"], 1),
                               "krylov_cap_hits_in_timed_steps": paper["krylov_cap_hits"],
                               "speedup_of_ours": res["steps_per_s"] / paper["steps_per_s"]}
    if gold is not None:
        out["rel_err_vs_oracle"] = {
            "what": ("max|v - v_oracle| / max|v_oracle| of this solver's settings on a 98k-element section of the "
                     "tube (64x8x32 hexes, length 2), first load step P = 0.16, against stored FP64 oracle "
                     "solutions (tests/golden)"),
            **gold}
    if not args.no_cpu_baseline and world == 1:
        if args.config != "batched":
            try:
                out["cpu_baseline"] = oracle_line(args, 2, 1)
            except Exception as e:  # the GPU number stands without it
                out["cpu_baseline"] = {"error": str(e)[-300:]}
        if verify_path is not None and res["verify"] is not None and args.config == "batched":
            try:
                code = _SEGMENT_SNIPPET.format(root=ROOT, path=verify_path, segments=res["verify"]["segments"],
                                               nseg=args.nseg, scale=res["verify"]["pressure"])
                segs = _run_py(code)
                out["oracle_check"] = dict(res["verify"], segment_errors=segs, what=(
                    "the GPU's converged first load step of the union mesh against the oracle's Newton solution "
                    "of each sampled segment alone (max |v - v_oracle| / max |v_oracle|)"))
                per_elem = sum(v["oracle_s"] / v["oracle_newton_its"] for v in segs.values()) / \
                    sum(v["n_elems"] for v in segs.values())
                out["cpu_baseline"] = {
                    "value": 1.0 / (per_elem * res["n_elems"]), "unit": "steps/s", "cores": 1, "kind": "oracle",
                    "sample": (f"FP64 oracle Newton steps on the two smallest segments "
                               f"({', '.join(str(v['n_elems']) for v in segs.values())} elements), time per element "
                               f"scaled linearly to the {res['n_elems']} elements of the union mesh (an upper bound "
                               f"on the oracle's rate: its direct solve grows faster than linearly)")}
            except Exception as e:
                out["oracle_check"] = {"error": str(e)[-300:]}
        elif verify_path is not None and res["verify"] is not None:
            try:
                chk = oracle_residual_check(args, verify_path, res["verify"]["pressure"])
                out["oracle_check"] = dict(res["verify"], **chk, what=(
                    "the GPU's converged first load step of the timed workload, checked with the oracle's own "
                    "residual: ||R_oracle(v_gpu)|| / ||R_oracle(v_0)||"))
            except Exception as e:
                out["oracle_check"] = {"error": str(e)[-300:]}
    print(json.dumps(out))


if __name__ == "__main__":
    main()
