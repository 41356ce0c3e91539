"""Parity at the workload sizes.

* Stored FP64 oracle solutions (tests/golden, written by
  make_tube_goldens.py, which calls only the oracle) of a 98k-element
  section of the workload tube at kappa 1e3 and 1e5 c10: the GPU Newton
  solution in FP64 and in FP32 + refinement, entry by entry, within 1e-8 of
  the largest entry.
* The 393k-element tube and the 3.1M-element refined tube at the bench's
  settings: the oracle's own residual at the GPU's converged first load step
  (a property that holds at any size: the GPU state solves the oracle's
  discrete equations to the Newton tolerance), and the assembled FP32
  tangent on a sample of block rows against the oracle's element tangents
  assembled for those rows.
"""
import os

import numpy as np
import pytest

from fixtures import artery_layers, artery_tube
from oracle import solid as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _solver(mesh, **kw):
    from paper_1312_5561_gb300.binding import SolidSolver
    return SolidSolver(mesh, **kw)


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp32_ir"])
@pytest.mark.parametrize("ratio", [1.0e3, 1.0e5], ids=["k1e3", "k1e5"])
def test_tube_section_matches_the_stored_oracle_solution(ratio, precision):
    from paper_1312_5561_gb300.binding import Load
    path = os.path.join(GOLDEN, f"tube98k_k{ratio:.0e}_p016.npz".replace("+0", ""))
    ref = np.load(path)["state"]
    mesh = artery_tube(n_theta=64, n_media=4, n_adv=4, n_z=32, length=2.0, materials=artery_layers(ratio))
    solver = _solver(mesh, precision=precision, newton_rtol=1e-10, krylov_rtol=1e-10, max_krylov=600)
    state = torch.zeros((mesh.n_nodes, 4), device="cuda", dtype=torch.float64)
    info = solver.solve(state, Load(pressure=0.16))
    assert info.status == 0
    got = state.cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-8 * np.abs(ref).max()


def _block_rows_from_oracle(P, mesh, state, nodes):
    """Block rows of the assembled tangent (Dirichlet rows -> identity, columns
    -> zero) for the given nodes, from the oracle's element tangents."""
    near = np.flatnonzero(np.isin(mesh.tets, nodes).any(axis=1))
    inc = [near[(mesh.tets[near] == i).any(axis=1)] for i in nodes]
    idx = np.unique(np.concatenate(inc))
    Ke = P.element_tangents(state, idx)
    pos = {e: q for q, e in enumerate(idx)}
    free = mesh.dir_mask == 0
    rows = []
    for i, els in zip(nodes, inc):
        row = {}
        for e in els:
            t = mesh.tets[e]
            a = int(np.flatnonzero(t == i)[0])
            for b in range(4):
                blk = Ke[pos[e]][4 * a:4 * a + 4, 4 * b:4 * b + 4]
                row[int(t[b])] = row.get(int(t[b]), 0.0) + blk
        for j in row:
            row[j] = row[j] * free[i][:, None] * free[j][None, :]
        for c in range(4):
            if not free[i][c]:
                row[i][c, c] = 1.0
        rows.append(row)
    return rows


def _check_at_scale(mesh, aggregation):
    from paper_1312_5561_gb300.binding import Load
    solver = _solver(mesh, precision=1, aggregation=aggregation, newton_rtol=1e-8, krylov_rtol=1e-8, max_krylov=600)
    state = torch.zeros((mesh.n_nodes, 4), device="cuda", dtype=torch.float64)
    info = solver.solve(state, Load(pressure=0.16))
    assert info.status == 0
    v = state.cpu().numpy()
    P = O.Problem(mesh)
    fext = P.external_force(0.16)
    r0 = np.linalg.norm(P.residual(np.zeros_like(v), fext))
    r = np.linalg.norm(P.residual(v, fext))
    assert r <= 1.0001e-8 * r0        # the GPU stopped at 1e-8 of its own residual norm
    # tangent at the converged state on sampled block rows
    solver.residual_tangent(state, Load(pressure=0.16))
    rp, ci, vals = solver.bsr()
    rng = np.random.default_rng(11)
    nodes = rng.choice(mesh.n_nodes, size=48, replace=False)
    for i, row in zip(nodes, _block_rows_from_oracle(P, mesh, v, nodes)):
        got = {int(ci[k]): vals[k].astype(np.float64) for k in range(rp[i], rp[i + 1])}
        assert set(got) == set(row)
        scale = max(np.abs(b).max() for b in row.values())
        err = max(np.abs(got[j] - row[j]).max() for j in row)
        assert err <= 1e-5 * scale
    solver.close()


def test_workload_tube_393k_solves_the_oracle_equations():
    mesh = artery_tube(n_theta=64, n_media=4, n_adv=4, n_z=128, length=8.0, materials=artery_layers(1.0e3))
    _check_at_scale(mesh, aggregation=0)


def test_refined_tube_3m_solves_the_oracle_equations():
    mesh = artery_tube(n_theta=128, n_media=8, n_adv=8, n_z=256, length=8.0, materials=artery_layers(1.0e5))
    _check_at_scale(mesh, aggregation=1)
