"""Learned Newton initial guess for a time-stepped solid under a pulsatile
interface traction.

A per-node MLP (32 features -> 256 -> 256 -> 256 -> 4, tanh, FP32 weights)
maps the node's reference position, layer, surface flag, the interface
pressure now and one and two steps ago, the node's own (noisy) traction now
and one step ago and the node's last two converged increments to the next
increment
(d_x, d_y, d_z, p).  It predicts the correction to the linear extrapolation
(the previous increment), so the proposal starts from that extrapolation.
It is trained on the GPU by the library's own forward / backward / Adam
kernels on increments produced by the plain solver, and proposes the initial
increment of Newton's method; fsi_solid_solve keeps the proposal only if its
FP64 residual is no larger than that of the zero increment, and Newton then
runs to the same tolerance, so the network can change the work but not the
answer.

The time discretisation is the Newmark-beta scheme of Sec. 4.1.2 (beta =
0.625, gamma = 1).  Feature assembly is tensor bookkeeping on the device;
the arithmetic of the method stays in the CUDA library.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

from . import binding as B

N_FEATURES = 32
SIZES = (N_FEATURES, 256, 256, 256, 4)


def pulsatile_pressure(t, period):
    """p(t) = 1 + 0.6 sin(2 pi t / T) + 0.2 sin(4 pi t / T)."""
    return 1.0 + 0.6 * math.sin(2 * math.pi * t / period) + 0.2 * math.sin(4 * math.pi * t / period)


def static_features(mesh):
    """[n, 6]: x/R, y/R, z/L, normalised radius, inner-surface flag, outer-layer flag."""
    X = mesh.X
    r = np.hypot(X[:, 0], X[:, 1])
    R = r.max()
    L = max(float(np.ptp(X[:, 2])), 1e-12)
    rn = (r - r.min()) / max(np.ptp(r), 1e-12)
    surf = np.zeros(mesh.n_nodes)
    surf[np.unique(mesh.neu_faces)] = 1.0
    outer = (rn > 0.5).astype(np.float64)
    return np.stack([X[:, 0] / R, X[:, 1] / R, (X[:, 2] - X[:, 2].min()) / L, rn, surf, outer], axis=1)


@dataclasses.dataclass
class StepRecord:
    p_now: float
    p_prev: float
    p_prev2: float
    node_p: object         # device FP64 [n]
    node_p_prev: object    # device FP64 [n], the previous step's nodal traction
    prev_inc: object       # device FP64 [n, 4]
    prev_inc2: object      # device FP64 [n, 4]
    inc: object            # device FP64 [n, 4]
    newton_its: int


class TimeLoop:
    """Newmark time stepping of the solid under p(t) plus Gaussian noise (one draw per
    step, or one per node and step)."""

    def __init__(self, mesh, solver, dt=0.01, period=1.0, noise=0.02, ramp_steps=20, beta=0.625, gamma=1.0,
                 seed=5, noise_mode="uniform"):
        import torch
        self.torch = torch
        self.mesh = mesh
        self.solver = solver
        self.dt, self.period, self.noise, self.ramp = dt, period, noise, ramp_steps
        self.noise_mode = noise_mode   # "uniform": one N(0, noise^2) draw per step; "per_node": one per node
        self.beta, self.gamma = beta, gamma
        self.rng = np.random.default_rng(seed)
        n = mesh.n_nodes
        z = lambda *s: torch.zeros(s, device="cuda", dtype=torch.float64)
        self.state = z(n, 4)
        self.disp, self.vel, self.acc, self.hist = z(n, 3), z(n, 3), z(n, 3), z(n, 3)
        self.prev_inc = z(n, 4)
        self.prev_inc2 = z(n, 4)
        self.step_index = 0
        self.p_prev = 0.0
        self.p_prev2 = 0.0
        self.node_p_prev = z(n)
        self.surface = np.zeros(n, bool)
        self.surface[np.unique(mesh.neu_faces)] = True

    def residual_norm(self, increment, load):
        """||R(v + increment)||_2 at the current state v, by the library's FP64
        residual and its allocation-free dot product (inf if an element inverts)."""
        import ctypes
        torch = self.torch
        trial = (self.state + increment).contiguous()
        try:
            r = self.solver.residual_tangent(trial, load, want_tangent=False)
        except B.FsiError:
            return float("inf")
        out = torch.zeros(1, device="cuda", dtype=torch.float64)
        st = B.lib.fsi_dots_static(r.data_ptr(), r.numel(), 1, r.data_ptr(), r.numel(), out.data_ptr(),
                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        if st != 0:
            raise B.FsiError(st, "fsi_dots_static failed")
        return float(out.item()) ** 0.5

    def pressure(self, k):
        t = k * self.dt
        ramp = min(1.0, k / self.ramp) if self.ramp else 1.0
        return ramp * pulsatile_pressure(t, self.period)

    def snapshot(self):
        keys = ("state", "disp", "vel", "acc", "hist", "prev_inc", "prev_inc2", "node_p_prev")
        return {k: getattr(self, k).clone() for k in keys} | {"step_index": self.step_index, "p_prev": self.p_prev,
                                                             "p_prev2": self.p_prev2,
                                                             "rng": self.rng.bit_generator.state}

    def restore(self, snap):
        for k in ("state", "disp", "vel", "acc", "hist", "prev_inc", "prev_inc2", "node_p_prev"):
            getattr(self, k).copy_(snap[k])
        self.step_index = snap["step_index"]
        self.p_prev = snap["p_prev"]
        self.p_prev2 = snap["p_prev2"]
        self.rng.bit_generator.state = snap["rng"]

    def step(self, guess_fn=None):
        torch = self.torch
        k = self.step_index + 1
        p = self.pressure(k)
        if self.noise_mode == "per_node":
            node_p = np.full(self.mesh.n_nodes, p) + self.noise * self.rng.standard_normal(self.mesh.n_nodes)
        else:
            node_p = np.full(self.mesh.n_nodes, p + self.noise * self.rng.standard_normal())
        node_p[~self.surface] = 0.0
        node_p_t = torch.tensor(node_p, device="cuda", dtype=torch.float64)
        load = B.Load(pressure=1.0, node_pressure=node_p_t, hist=self.hist)
        guess = None
        if guess_fn is not None:
            guess = guess_fn(p, self.p_prev, self.p_prev2, node_p_t, self.node_p_prev, self.prev_inc, self.prev_inc2)
            if callable(guess):      # a family of candidates: keep the one with the smallest residual
                guess = guess(lambda g: self.residual_norm(g, load))
        before = self.state.clone()
        info = self.solver.solve(self.state, load, guess=guess)
        inc = self.state - before
        rec = StepRecord(p, self.p_prev, self.p_prev2, node_p_t, self.node_p_prev.clone(), self.prev_inc.clone(),
                         self.prev_inc2.clone(), inc, info.newton_its)
        self.solver.newmark_advance(self.state, self.disp, self.vel, self.acc, self.hist, self.beta, self.gamma,
                                    self.dt)
        self.prev_inc2 = self.prev_inc
        self.prev_inc = inc
        self.p_prev2 = self.p_prev
        self.p_prev = p
        self.node_p_prev = node_p_t
        self.step_index = k
        rec.guess_accepted = info.guess_accepted
        return rec


class GuessModel:
    """Feature scaling + the library MLP."""

    def __init__(self, mesh, seed=0):
        import torch
        self.torch = torch
        self.static = torch.tensor(static_features(mesh), device="cuda", dtype=torch.float32)
        self.net = B.Mlp(SIZES, seed=seed)
        self.inc_scale = torch.ones(4, device="cuda", dtype=torch.float32)
        self.corr_scale = torch.ones(4, device="cuda", dtype=torch.float32)
        self.p_scale = 1.0
        self.dp_scale = 1.0

    def features(self, p_now, p_prev, p_prev2, node_p, node_p_prev, prev_inc, prev_inc2):
        torch = self.torch
        n = self.static.shape[0]
        f = torch.zeros((n, N_FEATURES), device="cuda", dtype=torch.float32)
        f[:, 0:6] = self.static
        f[:, 6] = p_now / self.p_scale
        f[:, 7] = p_prev / self.p_scale
        f[:, 8] = (p_now - p_prev) / self.dp_scale
        f[:, 9] = (p_prev - p_prev2) / self.dp_scale
        f[:, 10] = node_p.float() / self.p_scale
        f[:, 11:15] = prev_inc.float() / self.inc_scale
        f[:, 15:19] = prev_inc2.float() / self.inc_scale
        f[:, 19] = node_p_prev.float() / self.p_scale
        f[:, 20] = (node_p - node_p_prev).float() / self.dp_scale
        return f

    def fit_scales(self, records):
        incs = self.torch.cat([r.inc.float() for r in records])
        self.inc_scale = incs.std(dim=0).clamp_min(1e-12)
        corr = self.torch.cat([(r.inc - r.prev_inc).float() for r in records])
        self.corr_scale = corr.std(dim=0).clamp_min(1e-12)
        self.p_scale = max(abs(r.p_now) for r in records) or 1.0
        self.dp_scale = max(abs(r.p_now - r.p_prev) for r in records) or 1.0

    def dataset(self, records, nodes_per_step, seed=0):
        torch = self.torch
        g = torch.Generator(device="cuda").manual_seed(seed)
        X, T = [], []
        for r in records:
            idx = torch.randint(0, self.static.shape[0], (nodes_per_step,), device="cuda", generator=g)
            f = self.features(r.p_now, r.p_prev, r.p_prev2, r.node_p, r.node_p_prev, r.prev_inc, r.prev_inc2)
            X.append(f[idx])
            T.append(((r.inc - r.prev_inc).float() / self.corr_scale)[idx])
        return torch.cat(X).contiguous(), torch.cat(T).contiguous()

    def train(self, X, T, steps=2000, batch=16384, lr=1e-3, seed=0):
        torch = self.torch
        g = torch.Generator(device="cuda").manual_seed(seed)
        losses = []
        for it in range(steps):
            idx = torch.randint(0, X.shape[0], (batch,), device="cuda", generator=g)
            lr_t = lr * (0.1 ** (it / max(steps, 1)))
            losses.append(self.net.train_step(X[idx].contiguous(), T[idx].contiguous(), lr=lr_t))
        return losses

    def guess(self, p_now, p_prev, p_prev2, node_p, node_p_prev, prev_inc, prev_inc2, bf16=True):
        """The network's correction of the linear extrapolation, as a family of
        candidates prev + s * correction, s in (1, 1/2, 0): the time loop keeps the
        one with the smallest FP64 residual.  Per-node errors of the network break
        the displacement-pressure consistency of the extrapolated increment, so a
        shorter step along its correction can leave a smaller residual; s = 0 is
        the extrapolation itself, so the proposal is never worse than it in
        residual."""
        f = self.features(p_now, p_prev, p_prev2, node_p, node_p_prev, prev_inc, prev_inc2)
        corr = (self.net.forward(f, bf16=bf16) * self.corr_scale).double()

        def pick(rnorm):
            best, best_r = None, float("inf")
            for s_ in (1.0, 0.5, 0.0):
                g = (prev_inc + s_ * corr).contiguous()
                r = rnorm(g)
                if r < best_r:
                    best, best_r = g, r
            return best
        return pick


def run_study(mesh, n_steps, n_train, dt=0.01, period=1.0, train_steps=2000, nodes_per_step=4096, seed=5,
              solver_opts: Optional[dict] = None, log=None, noise_mode="uniform"):
    """Plain solver for n_steps time steps (records the first n_train), train the
    MLP, then replay steps n_train+1..n_steps from the same state three times:
    zero increment, previous increment (linear extrapolation), MLP guess.
    Returns mean Newton iterations of each and the training losses."""
    opts = dict(precision=1, newton_rtol=1e-8, krylov_rtol=1e-8, max_krylov=800, max_newton=30,
                inertia_coef=1.0 / (0.625 * dt * dt))
    opts.update(solver_opts or {})
    solver = B.SolidSolver(mesh, **opts)
    loop = TimeLoop(mesh, solver, dt=dt, period=period, seed=seed, noise_mode=noise_mode)
    records = []
    for k in range(n_train):
        rec = loop.step()
        records.append(rec)
        if log and k % 50 == 0:
            log(f"train data step {k} newton {rec.newton_its}")
    snap = loop.snapshot()
    model = GuessModel(mesh, seed=seed)
    model.fit_scales(records[loop.ramp:])
    X, T = model.dataset(records[loop.ramp:], nodes_per_step, seed=seed)
    losses = model.train(X, T, steps=train_steps)
    results = {}
    strategies = {
        "zero": None,
        "linear_extrapolation": lambda p, pp, pp2, npr, npp, prev, prev2: prev.contiguous(),
        "mlp": model.guess,
    }
    for name, fn in strategies.items():
        loop.restore(snap)
        its, acc = [], []
        for j in range(n_steps - n_train):
            try:
                rec = loop.step(fn)
            except B.FsiError:
                if log:
                    log(f"{name}: solve failed at step {loop.step_index + 1}")
                raise
            its.append(rec.newton_its)
            acc.append(getattr(rec, "guess_accepted", 0))
            if log and j % 50 == 0:
                log(f"{name} step {loop.step_index} newton {rec.newton_its}")
        results[name] = {"mean_newton_its": float(np.mean(its)), "accepted": float(np.mean(acc))}
        if log:
            log(f"{name}: mean Newton its {np.mean(its):.3f} accepted {np.mean(acc):.2f}")
    solver.close()
    return {"results": results, "loss_first": losses[0], "loss_last": float(np.mean(losses[-50:])),
            "train_records": len(records)}


def main():
    import argparse
    import json
    import os
    import sys
    import time
    ap = argparse.ArgumentParser(description="learned Newton initial guess on the two-layer artery")
    ap.add_argument("--nz", type=int, default=128, help="axial hexahedra (128: the 393k-element tube)")
    ap.add_argument("--steps", type=int, default=2000, help="time steps (replayed: steps - train)")
    ap.add_argument("--train", type=int, default=1500, help="time steps whose increments train the MLP")
    ap.add_argument("--train-steps", type=int, default=3000)
    # The noise is one draw per time step on the interface traction p(t) (uniform
    # over the interface).  Drawn independently per node instead, its net lateral
    # force pumps the slow bending modes of the 8-long tube, whose ends are fixed
    # axially only: the lateral displacement reaches 0.7 of the radius and Newton
    # breaks down near step 1690.
    ap.add_argument("--noise", default="uniform", choices=["uniform", "per_node"])
    ap.add_argument("--ends", default="axial", choices=["axial", "clamped"])
    args = ap.parse_args()
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    from fixtures import artery_layers, artery_tube
    from fixtures.meshes import tube_end_bc
    mesh = artery_tube(n_theta=64, n_z=args.nz, length=8.0 * args.nz / 128, materials=artery_layers(1.0e3, rho=1.2))
    if args.ends == "clamped":
        mesh = tube_end_bc(mesh, clamped=True)
    t0 = time.time()
    out = run_study(mesh, args.steps, args.train, train_steps=args.train_steps, noise_mode=args.noise,
                    log=lambda m: print(m, file=sys.stderr, flush=True))
    out["wall_s"] = time.time() - t0
    out["workload"] = f"artery tube 64x8x{args.nz} ({mesh.n_elems} tets, ends {args.ends}), Newmark beta 0.625 " \
                      f"gamma 1 dt 0.01, p(t)=1+0.6sin(2pi t)+0.2sin(4pi t)+N(0,0.02^2) ({args.noise}), {args.steps} steps, " \
                      f"train {args.train}"
    print(json.dumps(out))


if __name__ == "__main__":
    main()
