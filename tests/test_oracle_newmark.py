"""Pins of the Newmark-beta oracle and of the oracle's inertia term (Sec. 4.1.2)
against closed forms."""
import dataclasses

import numpy as np

from fixtures import artery_layers, artery_tube
from oracle import newmark as N
from oracle import solid as O


def test_average_acceleration_conserves_the_oscillator_energy():
    """beta = 1/4, gamma = 1/2 on m u'' + k u = 0: 1/2 m v^2 + 1/2 k u^2 is
    invariant, even at omega dt = 2."""
    m, k = 2.0, 8.0                       # omega = 2
    _, _, e = N.sdof(m, k, 0.3, -0.7, 1.0, 1000, 0.25, 0.5)
    assert np.abs(e - e[0]).max() <= 1e-12 * e[0]


def test_average_acceleration_is_second_order():
    """Error of u(T) against u0 cos(w T) + v0 / w sin(w T) falls by ~4 when dt halves."""
    m, k, u0, v0, T = 1.0, 4.0, 1.0, 0.5, 3.0
    w = np.sqrt(k / m)
    exact = u0 * np.cos(w * T) + v0 / w * np.sin(w * T)
    errs = []
    for n in (200, 400, 800):
        u, _, _ = N.sdof(m, k, u0, v0, T / n, n, 0.25, 0.5)
        errs.append(abs(u[-1] - exact))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.8 < r1 < 4.2 and 3.8 < r2 < 4.2


def _amplification(beta, gamma, w_dt):
    """One-step map (u, v) -> (u', v') of the oscillator (m = 1, k = w^2, dt = 1);
    the acceleration is fixed by equilibrium at every step."""
    cols = []
    for u0, v0 in ((1.0, 0.0), (0.0, 1.0)):
        u, v, _ = N.sdof(1.0, w_dt * w_dt, u0, v0, 1.0, 1, beta, gamma)
        cols.append([u[1], v[1]])
    return np.array(cols).T


def test_spectral_radius_of_the_step():
    """Unconditional stability and dissipation: rho(A) = 1 for beta = 1/4,
    gamma = 1/2; rho(A) < 1 for the paper's beta = 0.625, gamma = 1
    (gamma > 1/2, beta >= (gamma + 1/2)^2 / 4) at every omega dt."""
    for w_dt in (0.1, 1.0, 10.0, 100.0):
        r_avg = np.abs(np.linalg.eigvals(_amplification(0.25, 0.5, w_dt))).max()
        r_pap = np.abs(np.linalg.eigvals(_amplification(0.625, 1.0, w_dt))).max()
        assert abs(r_avg - 1.0) <= 1e-12
        assert r_pap < 1.0
    # and the criterion has teeth: beta = 0.05 < (gamma + 1/2)^2 / 4 with
    # gamma = 1/2 is only conditionally stable and blows up at omega dt = 10
    assert np.abs(np.linalg.eigvals(_amplification(0.05, 0.5, 10.0))).max() > 1.0


def test_the_papers_parameters_damp_the_oscillator():
    """beta = 0.625, gamma = 1: after 400 steps the energy has dropped (the
    kinetic + potential energy need not fall at every step at large omega dt)."""
    for dt in (0.05, 5.0):
        _, _, e = N.sdof(1.0, 4.0, 1.0, 0.0, dt, 400, 0.625, 1.0)
        assert e[-1] < 0.5 * e[0]


def test_update_reproduces_the_displacement_recurrence():
    """The a_n and v_n returned satisfy the Newmark displacement recurrence
    d_n = d_(n-1) + dt v_(n-1) + dt^2/2 ((1 - 2 beta) a_(n-1) + 2 beta a_n)."""
    rng = np.random.default_rng(0)
    d0, v0, a0, d1 = (rng.standard_normal(50) for _ in range(4))
    beta, gamma, dt = 0.625, 1.0, 0.01
    a1, v1, h1 = N.newmark_update(d1, d0, v0, a0, beta, gamma, dt)
    assert np.allclose(d0 + dt * v0 + 0.5 * dt * dt * ((1 - 2 * beta) * a0 + 2 * beta * a1), d1, rtol=0, atol=1e-13)
    assert np.allclose(v1, v0 + dt * ((1 - gamma) * a0 + gamma * a1), rtol=0, atol=1e-12)
    # the next step's inertia: c d_2 - h_1 is the acceleration a_2 of the recurrence
    d2 = rng.standard_normal(50)
    a2, _, _ = N.newmark_update(d2, d1, v1, a1, beta, gamma, dt)
    assert np.allclose(d2 / (beta * dt * dt) - h1, a2, rtol=1e-12, atol=1e-9)


def _translation(mesh, t):
    s = np.zeros((mesh.n_nodes, 4))
    s[:, :3] = t
    return s


def test_inertia_of_a_rigid_translation():
    """F = I and p = 0: only the inertia term acts.  With history h = c d the
    acceleration vanishes and so does the whole residual; with h = 0 the nodal
    inertial forces add up to rho c V_total t (the consistent mass matrix has
    total mass rho V)."""
    mesh = artery_tube(n_theta=16, n_z=2, length=0.125, materials=artery_layers(1.0e3, rho=1.2))
    c = 1.0 / (0.625 * 0.01 ** 2)
    P = O.Problem(mesh, O.Options(inertia_coef=c))
    t = np.array([0.01, -0.02, 0.005])
    s = _translation(mesh, t)
    R0 = P.residual(s, hist=np.tile(c * t, (mesh.n_nodes, 1)))
    assert np.abs(R0).max() <= 1e-9 * c * np.abs(t).max()
    # without Dirichlet rows every nodal force counts
    Pfree = O.Problem(dataclasses.replace(mesh, dir_mask=np.zeros_like(mesh.dir_mask)), O.Options(inertia_coef=c))
    tot = Pfree.residual(s, hist=np.zeros((mesh.n_nodes, 3)))[:, :3].sum(axis=0)
    assert np.allclose(tot, 1.2 * c * Pfree.V.sum() * t, rtol=1e-12, atol=0)


def _deformed_state(mesh, seed):
    """A smooth deformation with a pressure field (no inverted element)."""
    rng = np.random.default_rng(seed)
    X = mesh.X
    s = np.zeros((mesh.n_nodes, 4))
    s[:, :3] = 0.01 * np.sin(X @ rng.standard_normal((3, 3)))
    s[:, 3] = 0.05 * np.cos(X @ rng.standard_normal(3))
    return s * (mesh.dir_mask == 0)


def test_zero_density_is_the_quasi_static_problem():
    """rho -> 0: with rho = 0 the inertia coefficient and any history change
    neither the residual nor the tangent (also not through the PSPG term)."""
    mesh = artery_tube(n_theta=16, n_z=2, length=0.125, materials=artery_layers(1.0e3, rho=0.0))
    s = _deformed_state(mesh, 1)
    hist = np.random.default_rng(2).standard_normal((mesh.n_nodes, 3))
    c = 1.0 / (0.625 * 0.01 ** 2)
    Pq = O.Problem(mesh)
    Pd = O.Problem(mesh, O.Options(inertia_coef=c))
    assert np.array_equal(Pd.residual(s, hist=hist), Pq.residual(s))
    Kd, Kq = Pd.tangent(s, hist=hist), Pq.tangent(s)
    assert abs(Kd - Kq).max() <= 1e-14 * abs(Kq).max()


def test_history_of_a_motion_without_acceleration_leaves_the_static_residual():
    """With h = c d (c = 1/(beta dt^2)) the Newmark acceleration vanishes at every
    node, so for any deformation d and pressure p the dynamic residual equals the
    quasi-static one; the inertia term alone is of size rho c V |d|."""
    mesh = artery_tube(n_theta=16, n_z=2, length=0.125, materials=artery_layers(1.0e3, rho=1.2))
    s = _deformed_state(mesh, 3)
    c = 1.0 / (0.625 * 0.01 ** 2)
    Pq = O.Problem(mesh)
    Pd = O.Problem(mesh, O.Options(inertia_coef=c))
    Rq = Pq.residual(s)
    Rd = Pd.residual(s, hist=c * s[:, :3])
    scale = 1.2 * c * Pd.V.max() * np.abs(s[:, :3]).max()
    assert np.abs(Rd - Rq).max() <= 1e-12 * scale
    # and a history off by a uniform acceleration a gives the consistent inertial force rho V a in total
    a = np.array([0.3, -0.1, 0.2])
    Pfree = O.Problem(dataclasses.replace(mesh, dir_mask=np.zeros_like(mesh.dir_mask)), O.Options(inertia_coef=c))
    Pfq = O.Problem(dataclasses.replace(mesh, dir_mask=np.zeros_like(mesh.dir_mask)))
    s_free = _deformed_state(dataclasses.replace(mesh, dir_mask=np.zeros_like(mesh.dir_mask)), 3)
    tot = (Pfree.residual(s_free, hist=c * s_free[:, :3] - a) - Pfq.residual(s_free))[:, :3].sum(axis=0)
    assert np.allclose(tot, 1.2 * Pfree.V.sum() * a, rtol=1e-10, atol=0)


def test_inertia_of_one_accelerated_vertex_on_a_single_tetrahedron():
    """One unit right tetrahedron at rest (F = I, p = 0), acceleration a at
    vertex 0 only (history h_0 = -a, h = 0 elsewhere, d = 0): the consistent P1
    mass gives the forces rho V a (1 + delta_a0)/20, i.e. rho V a/10 at vertex 0
    and rho V a/20 at the others (a lumped mass would give rho V a/4 and 0), and
    the PSPG term gives tau V (rho hbar) . g_a = -tau V rho (a . g_a)/4 on the
    pressure rows, with tau = h_T^2/(4 mu_l), h_T = sqrt 2, mu_l = 2 (c10 + c01)."""
    from fixtures import mooney_rivlin
    from fixtures.meshes import Mesh
    c10, c01, rho = 0.5, 0.1, 1.2
    mesh = Mesh(X=np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], np.float64),
                tets=np.array([[0, 1, 2, 3]], np.int32), mat_id=np.zeros(1, np.int32),
                fibre=np.zeros((1, 2, 3)), dir_mask=np.zeros((4, 4), np.uint8),
                neu_faces=np.zeros((0, 3), np.int32), materials=mooney_rivlin(c10, c01, 1.0e3, rho))
    c = 1.0 / (0.625 * 0.01 ** 2)
    P = O.Problem(mesh, O.Options(inertia_coef=c))
    a = np.array([0.3, -0.7, 0.2])
    hist = np.zeros((4, 3))
    hist[0] = -a
    R = P.residual(np.zeros((4, 4)), hist=hist)
    V = 1.0 / 6.0
    want = np.outer([2.0, 1.0, 1.0, 1.0], rho * V * a / 20.0)
    assert np.allclose(R[:, :3], want, rtol=1e-13, atol=0)
    g = np.array([[-1.0, -1.0, -1.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0]])
    tau = 2.0 / (4.0 * 2.0 * (c10 + c01))
    assert np.allclose(R[:, 3], -tau * V * rho * (g @ a) / 4.0, rtol=1e-13, atol=1e-300)
