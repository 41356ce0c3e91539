"""Failure handling on the GPU path, with every failure made on the host: a
non-finite input, an iteration cap set too low, and a garbage initial guess.
No test here faults, traps or hangs the GPU; each checks the status the
library returns and that the handle stays usable."""
import numpy as np
import pytest

from fixtures import cube_uniaxial_bc, kuhn_cube
from oracle import solid as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _t(a):
    return torch.tensor(np.ascontiguousarray(a), device="cuda", dtype=torch.float64)


def _solver(mesh, **kw):
    from paper_1312_5561_gb300.binding import SolidSolver
    return SolidSolver(mesh, **kw)


@pytest.mark.parametrize("where", ["displacement", "pressure"])
def test_non_finite_state_is_reported(where):
    """A NaN in the state gives FSI_ERR_INVERTED from the residual/tangent
    (displacement: J is not finite) or from Newton (pressure: the residual
    norm is not finite), and the next call on the handle works."""
    from paper_1312_5561_gb300.binding import FsiError, Load
    mesh = cube_uniaxial_bc(kuhn_cube(3), stretch=0.1)
    solver = _solver(mesh)
    s = np.zeros((mesh.n_nodes, 4))
    s[21, 0 if where == "displacement" else 3] = np.nan     # an interior node: no component constrained
    state = _t(s)
    info = solver.solve(state, Load(dir_values=_t(mesh.dir_values(0.5))), check=False)
    assert info.status == -4
    with pytest.raises(FsiError):
        solver.newton_step(_t(s), Load())
    state = torch.zeros((mesh.n_nodes, 4), device="cuda", dtype=torch.float64)
    info = solver.solve(state, Load(dir_values=_t(mesh.dir_values(0.5))))
    assert info.status == 0 and info.newton_its >= 1


def test_iteration_caps_are_reported():
    """Newton capped at one iteration and Krylov capped at two iterations end
    with FSI_ERR_NOT_CONVERGED and filled statistics; the handle stays usable."""
    from paper_1312_5561_gb300.binding import Load
    mesh = cube_uniaxial_bc(kuhn_cube(4), stretch=0.2)
    solver = _solver(mesh, max_newton=1)
    state = torch.zeros((mesh.n_nodes, 4), device="cuda", dtype=torch.float64)
    info = solver.solve(state, Load(dir_values=_t(mesh.dir_values(1.0))), check=False)
    assert info.status == -5 and info.newton_its == 1 and info.res < info.res0
    solver = _solver(mesh, max_krylov=2, krylov_rtol=1e-12)
    P = O.Problem(mesh)
    s = P.apply_dirichlet(np.zeros((mesh.n_nodes, 4)), mesh.dir_values(0.5))
    solver.residual_tangent(_t(s))
    b = np.random.default_rng(1).standard_normal((mesh.n_nodes, 4)) * (mesh.dir_mask == 0)
    x, info = solver.linear_solve(_t(b), check=False)
    assert info.status == -5 and info.krylov_its_last == 2 and info.lin_res > 1e-12


@pytest.mark.parametrize("kind", ["huge", "nan"])
def test_garbage_guess_falls_back_to_the_zero_increment(kind):
    """An initial increment that raises the residual (or is not finite) is
    dropped: Newton starts from the zero increment and reaches the same
    solution as without a guess."""
    from paper_1312_5561_gb300.binding import Load
    mesh = cube_uniaxial_bc(kuhn_cube(4), stretch=0.2)
    rng = np.random.default_rng(3)
    g = 1.0e3 * rng.standard_normal((mesh.n_nodes, 4)) if kind == "huge" else np.full((mesh.n_nodes, 4), np.nan)
    sols = []
    for guess in (None, _t(g)):
        solver = _solver(mesh, newton_rtol=1e-10, krylov_rtol=1e-12, max_krylov=1000)
        state = torch.zeros((mesh.n_nodes, 4), device="cuda", dtype=torch.float64)
        info = solver.solve(state, Load(dir_values=_t(mesh.dir_values(0.2))), guess=guess)
        assert info.status == 0 and info.guess_accepted == 0
        sols.append(state.cpu().numpy())
    assert np.array_equal(sols[0], sols[1])
