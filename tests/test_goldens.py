"""The stored oracle solutions under tests/golden/ are what their script says:
converged oracle Newton solutions of the 98k-element tube section under the
internal dead pressure of the first load step (Sec. 4.2.3 weak form with the
pressure load on the lumen wall), checked against the current oracle's
residual without re-running the 17-minute direct solves."""
import os
import sys

import numpy as np
import pytest

from oracle import solid as O

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))

from make_tube_goldens import golden_mesh, golden_path  # noqa: E402


@pytest.mark.parametrize("ratio", [1.0e3, 1.0e5])
def test_stored_solution_is_an_oracle_equilibrium(ratio):
    z = np.load(golden_path(ratio))
    assert float(z["pressure"]) == 0.16 and float(z["kappa_ratio"]) == ratio
    mesh = golden_mesh(ratio)
    state = z["state"]
    assert state.shape == (mesh.n_nodes, 4) and np.isfinite(state).all()
    P = O.Problem(mesh)
    fext = P.external_force(0.16)
    r0 = np.linalg.norm(P.residual(np.zeros_like(state), fext=fext))
    assert np.linalg.norm(P.residual(state, fext=fext)) <= 1e-12 * r0
    # Dirichlet values (zero) kept, and the lumen wall moves outwards under the internal pressure
    assert (state[mesh.dir_mask != 0] == 0.0).all()
    X = mesh.X
    r = np.hypot(X[:, 0], X[:, 1])
    inner = np.isclose(r, r.min()) & (X[:, 2] > 0.25) & (X[:, 2] < X[:, 2].max() - 0.25)
    ur = (state[inner, 0] * X[inner, 0] + state[inner, 1] * X[inner, 1]) / r[inner]
    assert ur.min() > 0.0
