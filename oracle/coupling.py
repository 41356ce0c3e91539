"""FP64 oracle of the Dirichlet-Neumann coupling loop with Aitken relaxation
(test infrastructure).

TEST INFRASTRUCTURE ONLY: imported by ``tests/`` and never by the product path.

What it computes (Sec. 5.1 and 5.2 of the paper):

* one DN cycle maps the interface displacement d_{Gamma,k-1} to the fluid force
  on Gamma^0 and the structure displacement under that force,
  d~_{Gamma,k} = S^-1(F(d_{Gamma,k-1}));
* the interface residual r_k = d~_{Gamma,k} - d_{Gamma,k-1}, the stop
  |r_k| / sqrt(n_Gamma) < eps;
* the relaxation d_{Gamma,k} = omega_{k-1} d~_{Gamma,k} + (1 - omega_{k-1}) d_{Gamma,k-1}
  (Eq. acceit) with the Aitken recursion
  omega_k = -omega_{k-1} r_k^T (r_{k+1} - r_k) / |r_{k+1} - r_k|^2 (Eq. dnomega).

The fluid sub-problem (Navier-Stokes on a moving domain) is not part of the
solid step, so F is a surrogate Dirichlet-to-Neumann map: an added-mass model
of the blood column, p_i = p0 - c_am w_i . (d_i - d_i^ref) on every interface
node, where w_i is the unit direction in which a positive pressure pushes the
wall at node i and d^ref the wall at rest (the previous time level).  With
c_am large against the wall stiffness the plain DN iteration (omega = 1)
diverges, the added-mass instability the paper's Aitken step is there for.
"""
from __future__ import annotations

import numpy as np


def interface(mesh):
    """Interface nodes (the vertices of the loaded faces) and, per node, the unit
    direction w_i of the pressure force: the P1 load of a unit pressure,
    f_i = -sum_faces |face| n_face / 3, normalised (Sec. 4.2.3 dead load)."""
    faces = np.asarray(mesh.neu_faces)
    nodes = np.unique(faces)
    X = mesh.X
    nrm2 = np.cross(X[faces[:, 1]] - X[faces[:, 0]], X[faces[:, 2]] - X[faces[:, 0]])
    f = np.zeros((mesh.n_nodes, 3))
    for a in range(3):
        np.add.at(f, faces[:, a], -nrm2)
    w = f[nodes]
    w /= np.linalg.norm(w, axis=1)[:, None]
    return nodes, w


def surrogate_fluid(d, p0, c_am, w, d_ref=None):
    """Added-mass Dirichlet-to-Neumann map: interface pressures [n_Gamma]."""
    dd = d if d_ref is None else d - d_ref
    return p0 - c_am * np.einsum("ij,ij->i", w, dd)


def aitken_fixed_point(G, d0, omega0=1.0, tol=1e-8, max_iter=100, aitken=True, record=None):
    """Relaxed fixed-point iteration d = G(d) (Eq. acceit, dnomega).

    G maps an interface displacement [n_Gamma, 3] to the next one; the stop is
    |r_k| / sqrt(n_Gamma) < tol.  Returns (d~ of the last cycle, cycles, omegas).
    """
    d = np.array(d0, dtype=float)
    n_gamma = d.shape[0]
    omega = omega0
    r_prev = None
    omegas = []
    for k in range(1, max_iter + 1):
        d_tilde = G(d)
        r = d_tilde - d
        res = np.linalg.norm(r) / np.sqrt(n_gamma)
        if record is not None:
            record.append(res)
        if res < tol:
            return d_tilde, k, omegas
        if aitken and r_prev is not None:
            dr = r - r_prev
            omega = -omega * float(np.vdot(r_prev, dr)) / float(np.vdot(dr, dr))
        omegas.append(omega)
        d = omega * d_tilde + (1.0 - omega) * d
        r_prev = r
    raise RuntimeError(f"DN iteration did not converge in {max_iter} cycles: {record}")


def dn_solve(problem, state, p0, c_am, d_ref=None, omega0=1.0, tol=1e-8, max_iter=100, aitken=True,
             newton_rtol=1e-10, hist=None, record=None):
    """The DN loop around the oracle's Newton solve of the solid.

    state [n, 4] is the start (its interface displacement is d_{Gamma,0}); each
    cycle solves the solid from the previous cycle's solid state.  Newton stops
    relative to the first cycle's initial residual norm in every cycle (near
    the fixed point a cycle starts almost converged, and a stop relative to its
    own initial residual would ask for accuracy below rounding).  Returns the
    solid state of the last cycle and the cycle count."""
    nodes, w = interface(problem.mesh)
    ref = None if d_ref is None else d_ref[nodes, :3]
    cur = {"v": np.array(state, dtype=float), "r_ref": None}

    def cycle(d):
        node_p = np.zeros(problem.n)
        node_p[nodes] = surrogate_fluid(d, p0, c_am, w, ref)
        fext = problem.external_force(1.0, node_pressure=node_p)
        if cur["r_ref"] is None:
            cur["r_ref"] = float(np.linalg.norm(problem.residual(cur["v"], fext, hist)))
        cur["v"], _ = problem.newton(cur["v"], fext=fext, hist=hist, rtol=newton_rtol, r_ref=cur["r_ref"])
        return cur["v"][nodes, :3].copy()

    _, k, _ = aitken_fixed_point(cycle, cur["v"][nodes, :3], omega0, tol, max_iter, aitken, record)
    return cur["v"], k
