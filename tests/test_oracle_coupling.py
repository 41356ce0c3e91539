"""Pins of the coupling-loop oracle (Sec. 5.1, 5.2: DN iteration, Aitken
relaxation) against closed forms and the definition of a fixed point."""
import numpy as np
import pytest

from fixtures import artery_layers, artery_tube
from oracle import coupling as Cp
from oracle import solid as O


def test_aitken_solves_a_scalar_linear_map_in_two_relaxations():
    """For G(d) = a d + b the recursion gives omega_1 = 1 / (1 - a), which lands
    on d* = b / (1 - a) exactly; the third cycle sees a zero residual."""
    a = -3.0                                    # |a| > 1: the plain iteration diverges
    rng = np.random.default_rng(0)
    b = rng.standard_normal((7, 3))
    G = lambda d: a * d + b
    d, k, omegas = Cp.aitken_fixed_point(G, np.zeros((7, 3)), omega0=0.5, tol=1e-13)
    assert k == 3
    assert omegas[0] == 0.5 and abs(omegas[1] - 1.0 / (1.0 - a)) <= 1e-14
    assert np.abs(d - b / (1.0 - a)).max() <= 1e-13
    with pytest.raises(RuntimeError):
        Cp.aitken_fixed_point(G, np.zeros((7, 3)), omega0=1.0, tol=1e-13, max_iter=30, aitken=False)


def test_aitken_reaches_the_fixed_point_of_a_linear_map():
    """G(d) = A d + b with A symmetric, eigenvalues in [-3, -0.5]: the limit is
    (I - A)^-1 b (closed form); omega = 1 alone diverges."""
    rng = np.random.default_rng(1)
    Q, _ = np.linalg.qr(rng.standard_normal((12, 12)))
    A = Q @ np.diag(np.linspace(-3.0, -0.5, 12)) @ Q.T
    b = rng.standard_normal(12)
    G = lambda d: (A @ d.ravel() + b).reshape(4, 3)
    d, k, _ = Cp.aitken_fixed_point(G, np.zeros((4, 3)), omega0=0.3, tol=1e-12, max_iter=200)
    x = np.linalg.solve(np.eye(12) - A, b)
    assert np.abs(d.ravel() - x).max() <= 1e-10 * np.abs(x).max()
    rec = []
    with pytest.raises(RuntimeError):
        Cp.aitken_fixed_point(G, np.zeros((4, 3)), omega0=1.0, tol=1e-12, max_iter=20, aitken=False, record=rec)
    assert rec[-1] > 100 * rec[0]


def test_interface_is_the_inner_wall_with_outward_radial_load():
    """On the tube the loaded faces are the lumen wall (r = 1): every interface
    node lies there, the unit load direction has no axial part and points
    outwards within the half-angle pi / n_theta of one facet."""
    nt = 16
    mesh = artery_tube(n_theta=nt, n_z=2, length=0.125, materials=artery_layers(1.0e3))
    nodes, w = Cp.interface(mesh)
    X = mesh.X[nodes]
    r = np.hypot(X[:, 0], X[:, 1])
    assert np.abs(r - 1.0).max() <= 1e-12
    assert len(nodes) == nt * 3
    er = np.stack([X[:, 0] / r, X[:, 1] / r], axis=1)
    assert np.abs(w[:, 2]).max() <= 1e-12
    assert (np.einsum("ij,ij->i", w[:, :2], er) >= np.cos(np.pi / nt) - 1e-12).all()


@pytest.fixture(scope="module")
def tiny_tube():
    mesh = artery_tube(n_theta=16, n_z=2, length=0.125, materials=artery_layers(1.0e3))
    return mesh, O.Problem(mesh)


def test_dn_limit_is_a_fixed_point_of_the_coupled_problem(tiny_tube):
    """At the DN limit the solid is in equilibrium with the fluid pressure of its
    own interface displacement: R(v*) - f(p0 - c w.d*(v*)) is at Newton level."""
    mesh, P = tiny_tube
    p0, c = 0.16, 4.0
    v, k = Cp.dn_solve(P, np.zeros((mesh.n_nodes, 4)), p0, c, omega0=0.3, tol=1e-10, max_iter=40)
    nodes, w = Cp.interface(mesh)
    node_p = np.zeros(mesh.n_nodes)
    node_p[nodes] = Cp.surrogate_fluid(v[nodes, :3], p0, c, w)
    f_self = P.external_force(1.0, node_pressure=node_p)
    f_rest = P.external_force(p0)
    R = P.residual(v, f_self)
    assert np.linalg.norm(R) <= 1e-7 * np.linalg.norm(f_rest)
    # the wall moved outwards, so the fluid pressure fell below p0
    assert (node_p[nodes] < p0).all()


def test_plain_dn_diverges_where_aitken_converges(tiny_tube):
    """Added-mass instability: with omega = 1 the interface residual grows; the
    Aitken-relaxed loop from the same start converges."""
    mesh, P = tiny_tube
    rec = []
    with pytest.raises(RuntimeError):
        Cp.dn_solve(P, np.zeros((mesh.n_nodes, 4)), 0.16, 2.0, omega0=1.0, tol=1e-10, max_iter=3, aitken=False,
                    record=rec)
    assert rec[2] > rec[1] > rec[0]
    v, k = Cp.dn_solve(P, np.zeros((mesh.n_nodes, 4)), 0.16, 2.0, omega0=1.0, tol=1e-9, max_iter=40)
    assert k < 20


def test_wall_at_rest_under_p0_is_the_dn_limit_for_any_added_mass(tiny_tube):
    """The surrogate fluid acts on the displacement from the wall at rest d_ref:
    if d_ref is the solid's equilibrium under the uniform pressure p0, that
    state sees exactly p0, so it is the DN limit whatever the added mass (the
    loop starts from the undeformed state; its first cycle loads the solid with
    p0 + c w.d_ref, which the oracle's undamped Newton takes in one step for
    c up to 1 on this tube)."""
    mesh, P = tiny_tube
    p0 = 0.16
    v0, _ = P.newton(np.zeros((mesh.n_nodes, 4)), fext=P.external_force(p0), rtol=1e-12)
    for c in (0.5, 1.0):
        v, k = Cp.dn_solve(P, np.zeros((mesh.n_nodes, 4)), p0, c, d_ref=v0, omega0=0.3, tol=1e-11, max_iter=60)
        assert np.abs(v - v0).max() <= 1e-8 * np.abs(v0).max()


def test_stop_measure_is_the_root_mean_square_over_interface_nodes():
    """|r_k| / sqrt(n_Gamma) (Sec. 5.1) is the RMS interface residual: the same
    one-node problem copied onto 1, 4 and 25 nodes gives the same residual
    history and the same number of cycles."""
    rng = np.random.default_rng(4)
    a = -2.0
    b = rng.standard_normal(3)
    runs = []
    for n in (1, 4, 25):
        rec = []
        d, k, _ = Cp.aitken_fixed_point(lambda d: a * d + b, np.zeros((n, 3)), omega0=0.4, tol=1e-12,
                                        record=rec)
        runs.append((k, rec))
    for k, rec in runs[1:]:
        assert k == runs[0][0]
        big = np.asarray(runs[0][1]) > 1e-10 * runs[0][1][0]      # above the rounding floor of the last cycle
        assert np.allclose(np.asarray(rec)[big], np.asarray(runs[0][1])[big], rtol=1e-12, atol=0)
    assert abs(runs[0][1][0] - np.linalg.norm(b)) <= 1e-14 * np.linalg.norm(b)
