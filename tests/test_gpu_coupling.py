"""The Dirichlet-Neumann coupling loop with Aitken relaxation (Sec. 5.1, 5.2)
through the C ABI, against the oracle's loop on the same surrogate fluid."""
import numpy as np
import pytest

from fixtures import artery_layers, artery_tube
from oracle import coupling as Cp
from oracle import solid as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _mesh():
    return artery_tube(n_theta=16, n_z=2, length=0.125, materials=artery_layers(1.0e3))


@pytest.mark.parametrize("precision", [0, 1])
def test_dn_aitken_two_time_levels_match_the_oracle(precision):
    """Two time levels: p0 = 0.08 from the reference configuration, then
    p0 = 0.16 with the first level's wall as d_ref; added mass 3, omega0 0.3."""
    from paper_1312_5561_gb300.binding import SolidSolver
    mesh = _mesh()
    P = O.Problem(mesh)
    solver = SolidSolver(mesh, precision=precision, newton_rtol=1e-10, krylov_rtol=1e-12, max_krylov=1000)
    state = torch.zeros((mesh.n_nodes, 4), device="cuda", dtype=torch.float64)
    ref = np.zeros((mesh.n_nodes, 4))
    d_ref_gpu, d_ref_cpu = None, None
    nodes, _ = Cp.interface(mesh)
    for p0 in (0.08, 0.16):
        info = solver.dn_solve(state, p0, 3.0, d_ref=d_ref_gpu, omega0=0.3, tol=1e-10, max_cycles=40)
        ref, k = Cp.dn_solve(P, ref, p0, 3.0, d_ref=d_ref_cpu, omega0=0.3, tol=1e-10, max_iter=40)
        assert info.converged == 1 and info.n_interface == len(nodes)
        # the Aitken sequence near the 1e-10 stop reacts to rounding in the solid
        # solves (FP32 V-cycle, nonlinear coarse smoothing): cycle counts agree
        # within a few cycles, the fixed point to 1e-7
        assert abs(info.cycles - k) <= 5
        got = state.cpu().numpy()
        assert np.abs(got - ref).max() <= 1e-7 * np.abs(ref).max()
        d_ref_gpu, d_ref_cpu = state.clone(), ref.copy()


def test_plain_dn_diverges_and_reports_it():
    """omega = 1 without Aitken at added mass 2: the interface residual grows and
    the call returns FSI_ERR_NOT_CONVERGED with its info filled."""
    from paper_1312_5561_gb300.binding import SolidSolver
    mesh = _mesh()
    solver = SolidSolver(mesh, newton_rtol=1e-10, krylov_rtol=1e-12, max_krylov=1000)
    state = torch.zeros((mesh.n_nodes, 4), device="cuda", dtype=torch.float64)
    info = solver.dn_solve(state, 0.16, 2.0, omega0=1.0, aitken=0, tol=1e-10, max_cycles=3, check=False)
    assert info.converged == 0 and info.cycles == 3
    assert info.res_last > info.res_first
    state.zero_()
    info = solver.dn_solve(state, 0.16, 2.0, omega0=1.0, tol=1e-9, max_cycles=40)
    assert info.converged == 1 and info.cycles < 20


def test_dn_rejects_bad_options():
    from paper_1312_5561_gb300.binding import FsiError, SolidSolver
    mesh = _mesh()
    solver = SolidSolver(mesh)
    state = torch.zeros((mesh.n_nodes, 4), device="cuda", dtype=torch.float64)
    with pytest.raises(FsiError):
        solver.dn_solve(state, 0.16, 2.0, omega0=0.0)
    with pytest.raises(FsiError):
        solver.dn_solve(state, 0.16, -1.0)
