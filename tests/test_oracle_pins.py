"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than its own formulas:
closed forms, invariances, textbook special cases, numerical derivatives and
energies differentiated by sympy.  A plausible slip anywhere in the oracle
(a dropped term, a sign, a transposed operand) breaks at least one of them.
"""
import dataclasses

import numpy as np
import pytest
import scipy.optimize as so
from scipy.linalg import expm

from fixtures import (Material, artery_tube, cube_uniaxial_bc, kuhn_cube, mooney_rivlin)
from fixtures.meshes import MODEL_ARTERY
from oracle import solid as O


def _rot(seed):
    rng = np.random.default_rng(seed)
    w = rng.standard_normal(3)
    Kx = np.array([[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0.0]])
    return expm(Kx)


def _smooth_state(mesh, seed, amp=0.08, pamp=0.3, noise=0.002):
    rng = np.random.default_rng(seed)
    s = np.zeros((mesh.n_nodes, 4))
    s[:, :3] = mesh.X @ (amp * rng.standard_normal((3, 3))).T + noise * rng.standard_normal((mesh.n_nodes, 3))
    s[:, 3] = pamp * rng.standard_normal(mesh.n_nodes)
    return s


@pytest.fixture(scope="module")
def small_tube():
    return artery_tube(n_theta=16, n_z=4)


# ---------------------------------------------------------------- geometry
def test_p1_gradients_reproduce_linear_fields():
    m = kuhn_cube(3)
    g, V, h = O.p1_geometry(m.X, m.tets)
    x = m.X[m.tets]
    # sum_a x_a (x) grad N_a = I for the identity field; sum_a grad N_a = 0
    assert np.allclose(np.einsum("eai,eaj->eij", x, g), np.eye(3), atol=1e-13)
    assert np.allclose(g.sum(axis=1), 0.0, atol=1e-12)
    assert np.isclose(V.sum(), 1.0, rtol=1e-14)
    assert np.all(V > 0)
    # Kuhn cells of edge 1/3: the longest edge of every tet is the cell diagonal
    assert np.allclose(h, np.sqrt(3.0) / 3.0)


# ---------------------------------------------------------------- stress-free states
def test_zero_residual_at_reference_state(small_tube):
    P = O.Problem(small_tube)
    R = P.element_residuals(np.zeros((small_tube.n_nodes, 4)))
    assert np.abs(R).max() == 0.0


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_zero_residual_under_rigid_motion(small_tube, seed):
    P = O.Problem(small_tube)
    Q = _rot(seed)
    s = np.zeros((small_tube.n_nodes, 4))
    s[:, :3] = small_tube.X @ Q.T - small_tube.X + np.array([0.3, -0.1, 0.2])
    R = P.element_residuals(s)
    scale = np.abs(P.element_residuals(_smooth_state(small_tube, 0))).max()
    assert np.abs(R).max() < 1e-12 * max(scale, 1.0)


def test_frame_invariance(small_tube):
    """S depends on C only; R^1 rotates with Q, R^2 is unchanged (Sec. 2.3)."""
    P = O.Problem(small_tube)
    s = _smooth_state(small_tube, 4)
    Q = _rot(5)
    x = small_tube.X + s[:, :3]
    s2 = s.copy()
    s2[:, :3] = x @ Q.T - small_tube.X
    R = P.element_residuals(s)
    R2 = P.element_residuals(s2)
    sc = np.abs(R).max()
    assert np.abs(R2[:, :, :3] - R[:, :, :3] @ Q.T).max() < 1e-12 * sc
    assert np.abs(R2[:, :, 3] - R[:, :, 3]).max() < 1e-12 * sc
    # stress itself: S(QF) = S(F)
    g, V, h, mp, fib = P._sub(np.arange(small_tube.n_elems))
    H = np.einsum("eai,eaj->eij", s[small_tube.tets][:, :, :3], g)
    F = np.eye(3) + H
    S1 = O.isochoric_stress(O.kinematics(H), mp["c10"], mp["c01"], mp["k1"], mp["k2"], mp["model"], fib)
    S2 = O.isochoric_stress(O.kinematics(Q @ F - np.eye(3)), mp["c10"], mp["c01"], mp["k1"], mp["k2"], mp["model"], fib)
    assert np.abs(S1 - S2).max() < 1e-12 * np.abs(S1).max()


# ---------------------------------------------------------------- tangent
@pytest.mark.parametrize("pspg", [True, False])
def test_tangent_matches_central_differences(small_tube, pspg):
    P = O.Problem(small_tube, O.Options(use_pspg=pspg))
    s = _smooth_state(small_tube, 7)
    idx = np.arange(0, small_tube.n_elems, 7)
    Kc = P.element_tangents(s, idx)
    g, V, h, mp, fib = P._sub(idx)
    Kf = O.element_tangent_fd(s[small_tube.tets[idx]], g, V, h, mp, fib, P.opts)
    err = np.abs(Kc - Kf).max(axis=(1, 2)) / np.abs(Kc).max(axis=(1, 2))
    assert err.max() < 1e-6


def test_tangent_block_structure(small_tube):
    """A = A^T and C = C^T always; B2 = B1 when the PSPG term is off (Sec. 4.4)."""
    s = _smooth_state(small_tube, 8)
    for pspg in (True, False):
        P = O.Problem(small_tube, O.Options(use_pspg=pspg))
        K = P.element_tangents(s).reshape(-1, 4, 4, 4, 4)     # e, a, i, b, j
        A = K[:, :, :3, :, :3].reshape(-1, 12, 12)
        Cb = K[:, :, 3, :, 3]
        B1T = K[:, :, :3, :, 3].reshape(-1, 12, 4)
        B2 = K[:, :, 3, :, :3].reshape(-1, 4, 12)
        assert np.abs(A - A.transpose(0, 2, 1)).max() < 1e-13 * np.abs(A).max()
        assert np.abs(Cb - Cb.transpose(0, 2, 1)).max() < 1e-13 * np.abs(Cb).max()
        d = np.abs(B2 - B1T.transpose(0, 2, 1)).max() / np.abs(B1T).max()
        if pspg:
            assert d > 1e-6          # B1 != B2 with stabilisation
        else:
            assert d < 1e-13


def _textbook_p1(g, V, mu, lam):
    """Small-strain P1 stiffness V B^T D B in Voigt notation."""
    ne = len(V)
    B = np.zeros((ne, 6, 12))
    for a in range(4):
        gx, gy, gz = g[:, a, 0], g[:, a, 1], g[:, a, 2]
        c = 3 * a
        B[:, 0, c + 0] = gx
        B[:, 1, c + 1] = gy
        B[:, 2, c + 2] = gz
        B[:, 3, c + 1] = gz
        B[:, 3, c + 2] = gy
        B[:, 4, c + 0] = gz
        B[:, 4, c + 2] = gx
        B[:, 5, c + 0] = gy
        B[:, 5, c + 1] = gx
    D = np.zeros((6, 6))
    D[:3, :3] = lam
    D += mu * np.diag([2, 2, 2, 1, 1, 1.0])
    return V[:, None, None] * np.einsum("eki,kl,elj->eij", B, D, B)


@pytest.mark.parametrize("model", ["mr", "artery"])
def test_small_strain_limit_is_textbook(model):
    """At F = I, p = 0 the tangent is the P1 deviatoric stiffness with
    mu = c10 + c01 and Lame lambda = -2 mu / 3; B1 = B2 = -(V/4) g_a;
    C = M / kappa + tau V g_a . g_b."""
    if model == "mr":
        m = kuhn_cube(2, materials=mooney_rivlin(0.7, 0.2, 1.0e3))
        mu = 0.9
    else:
        m = artery_tube(n_theta=8, n_z=2)
        m.mat_id[:] = 0
        mu = m.materials[0].c10
    P = O.Problem(m)
    K = P.element_tangents(np.zeros((m.n_nodes, 4))).reshape(-1, 4, 4, 4, 4)
    A = K[:, :, :3, :, :3].reshape(-1, 12, 12)
    Kt = _textbook_p1(P.g, P.V, mu, -2.0 * mu / 3.0)
    assert np.abs(A - Kt).max() < 1e-12 * np.abs(Kt).max()
    B1T = K[:, :, :3, :, 3]                                # [e, a, i, b]
    exp_B1T = -(P.V / 4.0)[:, None, None, None] * P.g[:, :, :, None] * np.ones(4)[None, None, None, :]
    assert np.abs(B1T - exp_B1T).max() < 1e-13 * np.abs(exp_B1T).max()
    B2 = K[:, :, 3, :, :3]                                 # [e, a, b, j]
    exp_B2 = -(P.V / 4.0)[:, None, None, None] * np.broadcast_to(P.g[:, None, :, :], B2.shape)
    assert np.abs(B2 - exp_B2).max() < 1e-13 * np.abs(exp_B2).max()
    kappa = m.materials[0].kappa
    M = (P.V / 20.0)[:, None, None] * (np.ones((4, 4)) + np.eye(4))
    mul = 2.0 * (m.materials[0].c10 + (m.materials[0].c01 if model == "mr"
                                       else m.materials[0].k1 / (2 * m.materials[0].k2)))
    tau = P.h ** 2 / (4.0 * mul)
    exp_C = -M / kappa - (tau * P.V)[:, None, None] * np.einsum("eai,ebi->eab", P.g, P.g)
    assert np.abs(K[:, :, 3, :, 3] - exp_C).max() < 1e-13 * np.abs(exp_C).max()


# ---------------------------------------------------------------- patch test
@pytest.mark.parametrize("seed", [11, 12])
def test_patch_test_affine_field(seed):
    """Any affine displacement with p = -kappa (J - 1) has zero residual at
    interior nodes (the PSPG term vanishes because grad p = 0)."""
    m = artery_tube(n_theta=16, n_z=6)
    m.mat_id[:] = 0                       # one material: p = -kappa (J-1) is one constant
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((2, 3))
    m.fibre[:] = a / np.linalg.norm(a, axis=1, keepdims=True)   # one fibre field: S uniform
    Gd = 0.1 * rng.standard_normal((3, 3))
    P = O.Problem(m)
    F = np.eye(3) + Gd
    kappa = m.materials[0].kappa
    s = np.zeros((m.n_nodes, 4))
    s[:, :3] = m.X @ Gd.T + rng.standard_normal(3)
    s[:, 3] = -kappa * (np.linalg.det(F) - 1.0)
    Re = P.element_residuals(s)
    R = np.zeros((m.n_nodes, 4))
    np.add.at(R, m.tets, Re)
    r = np.hypot(m.X[:, 0], m.X[:, 1])
    interior = (r > r.min() + 1e-9) & (r < r.max() - 1e-9) & (m.X[:, 2] > 1e-9) & (m.X[:, 2] < 8 - 1e-9)
    scale = np.abs(Re).max()
    assert np.abs(R[interior]).max() < 1e-11 * scale
    assert np.abs(R[~interior, :3]).max() > 1e-3 * scale   # boundary nodes carry the traction


# ---------------------------------------------------------------- uniaxial closed forms
def _energy_mr(c10, c01, kappa):
    import sympy as sy
    a, b, l = sy.symbols("a b l", positive=True)
    J = a * b * l
    I1 = a ** 2 + b ** 2 + l ** 2
    I2 = a ** 2 * b ** 2 + a ** 2 * l ** 2 + b ** 2 * l ** 2
    psi = c10 / 2 * (I1 * J ** sy.Rational(-2, 3) - 3) + c01 / 2 * (I2 * J ** sy.Rational(-4, 3) - 3) \
        + kappa / 2 * (J - 1) ** 2
    return sy, (a, b, l), psi


def _energy_artery(c10, k1, k2, kappa, alpha):
    import sympy as sy
    a, b, l = sy.symbols("a b l", positive=True)
    J = a * b * l
    I1 = a ** 2 + b ** 2 + l ** 2
    # fibre (0, cos, +-sin): a.C.a = b^2 cos^2 + l^2 sin^2 for both families
    I4 = b ** 2 * np.cos(alpha) ** 2 + l ** 2 * np.sin(alpha) ** 2
    J4 = I4 * J ** sy.Rational(-2, 3)
    psi = c10 / 2 * (I1 * J ** sy.Rational(-2, 3) - 3) \
        + 2 * k1 / (2 * k2) * (sy.exp(k2 * (J4 - 1) ** 2) - 1) + kappa / 2 * (J - 1) ** 2
    return sy, (a, b, l), psi


def _solve_lateral(sy, syms, psi, lam):
    a, b, l = syms
    fa = sy.lambdify((a, b), sy.diff(psi, a).subs(l, lam))
    fb = sy.lambdify((a, b), sy.diff(psi, b).subs(l, lam))
    sol = so.fsolve(lambda x: [fa(x[0], x[1]), fb(x[0], x[1])], [1.0 / np.sqrt(lam)] * 2, xtol=1e-15)
    Pzz = float(sy.diff(psi, l).subs({a: sol[0], b: sol[1], l: lam}))
    return sol, Pzz


def _run_uniaxial(mesh, lam, steps):
    P = O.Problem(mesh)
    s = np.zeros((mesh.n_nodes, 4))
    for k in range(1, steps + 1):
        s = P.apply_dirichlet(s, mesh.dir_values(k / steps))
        s, _ = P.newton(s, rtol=1e-13, max_it=40)
    return P, s


def test_uniaxial_mooney_rivlin_closed_form():
    """Roller cube, top moved to stretch lam: the FE solution is homogeneous
    with the lateral stretch solving dPsi/da = 0 and the summed top reaction
    equal to the nominal stress dPsi/dlam times the area (energy by sympy)."""
    c10, c01, kappa, lam = 0.5, 0.1, 1.0e3, 1.2
    m = cube_uniaxial_bc(kuhn_cube(2, materials=mooney_rivlin(c10, c01, kappa)), stretch=lam - 1,
                         variant="roller")
    P, s = _run_uniaxial(m, lam, 2)
    sy, syms, psi = _energy_mr(c10, c01, kappa)
    (a, b), Pzz = _solve_lateral(sy, syms, psi, lam)
    X = m.X
    assert np.abs(s[:, 0] - (a - 1) * X[:, 0]).max() < 1e-10
    assert np.abs(s[:, 1] - (b - 1) * X[:, 1]).max() < 1e-10
    assert np.abs(s[:, 2] - (lam - 1) * X[:, 2]).max() < 1e-12
    assert np.abs(s[:, 3] - (-kappa * (a * b * lam - 1))).max() < 1e-8 * max(1.0, abs(s[:, 3]).max())
    Re = P.element_residuals(s)
    R = np.zeros((m.n_nodes, 4))
    np.add.at(R, m.tets, Re)
    top = np.abs(X[:, 2] - 1.0) < 1e-12
    assert abs(R[top, 2].sum() - Pzz) < 1e-9 * abs(Pzz)


def test_uniaxial_mr_incompressible_limit():
    """As kappa grows, P -> c10 (lam - lam^-2) + c01 (1 - lam^-3) for Psi as printed."""
    c10, c01, lam = 0.5, 0.1, 1.2
    m = cube_uniaxial_bc(kuhn_cube(1, materials=mooney_rivlin(c10, c01, 1.0e7)), stretch=lam - 1,
                         variant="roller")
    P, s = _run_uniaxial(m, lam, 2)
    Re = P.element_residuals(s)
    R = np.zeros((m.n_nodes, 4))
    np.add.at(R, m.tets, Re)
    top = np.abs(m.X[:, 2] - 1.0) < 1e-12
    limit = c10 * (lam - lam ** -2) + c01 * (1 - lam ** -3)
    assert abs(R[top, 2].sum() - limit) < 1e-5 * limit


def test_uniaxial_artery_closed_form():
    """Fibres (0, cos a, +-sin a) in every element; homogeneous F = diag(a, b, lam)
    with dPsi/da = dPsi/db = 0.  Pins S_aniso = 2 dPsi/dC (factor 2 k1)."""
    c10, k1, k2, kappa, alpha, lam = 3.0, 2.3, 0.84, 3.0e3, np.deg2rad(50.0), 1.15
    mat = Material(MODEL_ARTERY, c10, 0.0, k1, k2, kappa, 0.0)
    m = cube_uniaxial_bc(kuhn_cube(2, materials=[mat]), stretch=lam - 1, variant="roller")
    m.fibre[:, 0] = [0.0, np.cos(alpha), np.sin(alpha)]
    m.fibre[:, 1] = [0.0, np.cos(alpha), -np.sin(alpha)]
    P, s = _run_uniaxial(m, lam, 3)
    sy, syms, psi = _energy_artery(c10, k1, k2, kappa, alpha)
    (a, b), Pzz = _solve_lateral(sy, syms, psi, lam)
    X = m.X
    assert np.abs(s[:, 0] - (a - 1) * X[:, 0]).max() < 1e-10
    assert np.abs(s[:, 1] - (b - 1) * X[:, 1]).max() < 1e-10
    Re = P.element_residuals(s)
    R = np.zeros((m.n_nodes, 4))
    np.add.at(R, m.tets, Re)
    top = np.abs(X[:, 2] - 1.0) < 1e-12
    assert abs(R[top, 2].sum() - Pzz) < 1e-9 * abs(Pzz)
    # the fibres are in extension here, so the anisotropic term was active
    J4 = (b ** 2 * np.cos(alpha) ** 2 + lam ** 2 * np.sin(alpha) ** 2) * (a * b * lam) ** (-2 / 3)
    assert J4 > 1.0


def test_fibres_inactive_in_compression():
    """A fibre family only acts while J_i > 1: under axial compression the
    artery response equals the neo-Hookean one (k1 = 0)."""
    m = cube_uniaxial_bc(kuhn_cube(1), stretch=-0.1, variant="roller")
    m.fibre[:, 0] = [0.0, 0.0, 1.0]
    m.fibre[:, 1] = [0.0, 0.0, 1.0]
    with_f = [Material(MODEL_ARTERY, 3.0, 0.0, 2.3, 0.84, 3e3, 0.0)]
    no_f = [Material(MODEL_ARTERY, 3.0, 0.0, 0.0, 0.84, 3e3, 0.0)]
    s = np.zeros((m.n_nodes, 4))
    s[:, 2] = -0.1 * m.X[:, 2]
    s[:, 0] = 0.03 * m.X[:, 0]
    s[:, 1] = 0.03 * m.X[:, 1]
    m.materials = with_f
    R1 = O.Problem(m).element_residuals(s)
    m.materials = no_f
    R0 = O.Problem(m).element_residuals(s)
    assert np.abs(R1[:, :, :3] - R0[:, :, :3]).max() == 0.0


# ---------------------------------------------------------------- loads, PSPG, Newton
def test_pressure_load_resultants():
    """Dead pressure on the closed inner surface of a periodic tube: zero net
    force; radial resultant density equals P times the surface area."""
    m = artery_tube(n_theta=32, n_z=4)
    P = O.Problem(m)
    f = P.external_force(pressure=1.3)
    assert np.abs(f.sum(axis=0)[:2]).max() < 1e-12
    nodes = np.unique(m.neu_faces)
    r = m.X[nodes, :2] / np.hypot(m.X[nodes, 0], m.X[nodes, 1])[:, None]
    radial = np.einsum("ij,ij->", f[nodes, :2], r)
    # polygonal inner surface: perimeter of the inscribed 32-gon times length
    area = 32 * 2 * np.sin(np.pi / 32) * m.meta["r_in"] * m.meta["length"]
    assert abs(radial - 1.3 * area * np.cos(np.pi / 32)) < 1e-3 * 1.3 * area
    # pointing outward (away from the axis) and no axial component
    assert radial > 0 and abs(f[:, 2]).max() < 1e-14


def test_linear_nodal_pressure_load_is_the_consistent_p1_load():
    """A P1-interpolated (linear) pressure on one tilted triangle: each nodal
    load must equal -n times the integral of N_a P over the face (Sec. 4.2.3,
    the <g_n, v> term).  The integral is evaluated here independently, by the
    edge-midpoint rule, which is exact for the quadratic N_a P.  The moment of
    the load about the face centroid separates this from a lumped load
    (A/3 P_a per vertex), which has the right resultant but the wrong moment."""
    from fixtures.meshes import Mesh
    X = np.array([[0.1, 0.0, 0.2], [1.3, 0.4, 0.0], [0.2, 1.1, 0.5], [0.3, 0.2, -1.0]])
    tets = np.array([[0, 2, 1, 3]], dtype=np.int32)
    face = np.array([[0, 1, 2]], dtype=np.int32)      # right-hand normal away from vertex 3
    m = Mesh(X=X, tets=tets, mat_id=np.zeros(1, np.int32), fibre=np.zeros((1, 2, 3)),
             dir_mask=np.zeros((4, 4), np.uint8), neu_faces=face, materials=mooney_rivlin())
    assert O.p1_geometry(X, tets)[1][0] > 0
    Pn = np.array([0.7, -0.2, 2.5, 9.9])              # value at vertex 3 is off the face
    f = O.Problem(m).external_force(pressure=1.5, node_pressure=Pn)
    v = face[0]
    x = X[v]
    nvec = np.cross(x[1] - x[0], x[2] - x[0])
    area = 0.5 * np.linalg.norm(nvec)
    n_out = nvec / np.linalg.norm(nvec)
    assert np.dot(n_out, X[3] - x[0]) < 0
    # midpoint rule: weights area/3 at the three edge midpoints; there N_a is 1/2
    # on the two vertices of the edge and 0 on the third
    mids = [(0, 1), (1, 2), (0, 2)]
    expect = np.zeros((4, 3))
    for a in range(3):
        integ = 0.0
        for (i, j) in mids:
            Na = 0.5 if a in (i, j) else 0.0
            Pm = 1.5 * 0.5 * (Pn[v[i]] + Pn[v[j]])
            integ += area / 3.0 * Na * Pm
        expect[v[a]] = -n_out * integ
    assert np.abs(f - expect).max() < 1e-14
    assert np.abs(f[3]).max() == 0.0
    # moment about the centroid: -n x-products of int (x - c) P dA, midpoint rule again
    c = x.mean(axis=0)
    mom_expect = np.zeros(3)
    for (i, j) in mids:
        xm = 0.5 * (x[i] + x[j])
        Pm = 1.5 * 0.5 * (Pn[v[i]] + Pn[v[j]])
        mom_expect += area / 3.0 * Pm * np.cross(xm - c, -n_out)
    mom = sum(np.cross(X[k] - c, f[k]) for k in v)
    assert np.abs(mom - mom_expect).max() < 1e-13
    lumped = [-n_out * area / 3.0 * 1.5 * Pn[k] for k in v]
    mom_lumped = sum(np.cross(X[k] - c, lk) for k, lk in zip(v, lumped))
    assert np.abs(mom_lumped - mom_expect).max() > 1e-2


def test_mass_norm_integrates_fields_exactly():
    """||v||_M of Sec. 4.4 is the L2 norm of the P1 field: for a constant
    field it is |c| sqrt(vol), and for a linear field on the unit cube the P1
    interpolant is exact, so int x^2 dV = 1/3 and int (x + 2y)^2 dV =
    1/3 + 4/4 + 4/3 = 8/3 (int x y = 1/4)."""
    m = kuhn_cube(3)
    P = O.Problem(m)
    c = np.array([0.3, -1.2, 0.5, 2.0])
    v = np.tile(c, (m.n_nodes, 1))
    assert abs(P.mass_norm(v) - np.linalg.norm(c)) < 1e-13
    v = np.zeros((m.n_nodes, 4))
    v[:, 0] = m.X[:, 0]
    assert abs(P.mass_norm(v) ** 2 - 1.0 / 3.0) < 1e-13
    v[:, 0] = 0.0
    v[:, 3] = m.X[:, 0] + 2.0 * m.X[:, 1]
    assert abs(P.mass_norm(v) ** 2 - 8.0 / 3.0) < 1e-13


def test_pspg_under_uniform_dilation():
    """With F = lam I and a linear pressure field the PSPG term reduces to
    -tau V lam grad p . g_a (J F^-T grad p . F^-T g_a = lam grad p . g_a)."""
    m = kuhn_cube(2)
    P = O.Problem(m)
    lam = 1.1
    s = np.zeros((m.n_nodes, 4))
    s[:, :3] = (lam - 1) * m.X
    gp = np.array([0.3, -0.2, 0.5])
    s[:, 3] = m.X @ gp
    R_on = P.element_residuals(s)
    R_off = O.Problem(m, O.Options(use_pspg=False)).element_residuals(s)
    tau = P.h ** 2 / (4 * 2 * (0.5 + 0.1))
    expect = -(tau * P.V * lam)[:, None] * np.einsum("eai,i->ea", P.g, gp)
    assert np.abs((R_on - R_off)[:, :, 3] - expect).max() < 1e-14


def test_newton_converges_quadratically():
    """Quadratic rate of Newton's method (Sec. 6: observed for both models)."""
    m = cube_uniaxial_bc(kuhn_cube(3), stretch=0.15)
    P = O.Problem(m)
    s = P.apply_dirichlet(np.zeros((m.n_nodes, 4)), m.dir_values(1.0))
    rec = []
    P.newton(s, rtol=1e-12, record=rec)
    r = np.asarray(rec) / rec[0]
    assert len(r) >= 4
    # in the final phase the ratio r_{k+1} / r_k^2 stays bounded while r_k -> 0
    k = np.argmax(r < 1e-3)
    assert k > 0 and r[k + 1] < 50 * r[k] ** 2 + 1e-13


def test_dirichlet_rows_and_columns():
    m = cube_uniaxial_bc(kuhn_cube(2), stretch=0.1)
    P = O.Problem(m)
    s = _smooth_state(m, 3, amp=0.05)
    K = P.tangent(s).toarray()
    c = np.flatnonzero(m.dir_mask.ravel())
    f = np.flatnonzero(m.dir_mask.ravel() == 0)
    assert np.array_equal(K[np.ix_(c, c)], np.eye(len(c)))
    assert np.abs(K[np.ix_(c, f)]).max() == 0 and np.abs(K[np.ix_(f, c)]).max() == 0
    assert np.abs(P.residual(s)[m.dir_mask.astype(bool)]).max() == 0


def test_greedy_colouring_spec():
    m = kuhn_cube(3)
    col = O.greedy_colouring(m.tets, m.n_nodes)
    for c in range(col.max() + 1):
        t = m.tets[col == c].ravel()
        assert len(np.unique(t)) == len(t)            # no shared node within a colour
    # first fit: an element of colour c has an earlier neighbour of each colour < c
    node_elems = [[] for _ in range(m.n_nodes)]
    for e, t in enumerate(m.tets):
        for a in t:
            node_elems[a].append(e)
    for e, t in enumerate(m.tets):
        earlier = {col[f] for a in t for f in node_elems[a] if f < e}
        assert set(range(col[e])) <= earlier


# ---------------------------------------------------------------- further pins (mutation check)
def test_characteristic_length_is_the_longest_edge():
    """h_T (reading r7) is the largest vertex-to-vertex distance, whichever
    edge it is: random tetrahedra and one whose longest edge is (2, 3)."""
    from scipy.spatial.distance import pdist
    rng = np.random.default_rng(12)
    X = rng.standard_normal((40, 3))
    tets = np.array([rng.choice(40, 4, replace=False) for _ in range(200)], np.int32)
    D = X[tets[:, 1:]] - X[tets[:, :1]]
    flip = np.linalg.det(D) < 0
    tets[flip] = tets[flip][:, [0, 2, 1, 3]]          # positive orientation
    X = np.vstack([X, [[0, 0, 0], [0, 1, 0], [-2, 0, 0], [2, 0, 1]]])   # |x3 - x2| = sqrt 17, the others <= sqrt 6
    tets = np.vstack([tets, [[40, 41, 42, 43]]]).astype(np.int32)
    _, _, h = O.p1_geometry(X, tets)
    want = np.array([pdist(X[t]).max() for t in tets])
    assert np.allclose(h, want, rtol=1e-15, atol=0)
    assert abs(h[-1] - np.hypot(4.0, 1.0)) <= 1e-15


def test_face_pressures_add_up_face_by_face(small_tube):
    """Per-face dead pressures (the batched segments' loads): the load equals
    the sum over faces of each face's pressure times the load of that face
    alone under a unit uniform pressure."""
    mesh = small_tube
    P = O.Problem(mesh)
    faces = mesh.neu_faces
    fp = np.random.default_rng(13).uniform(0.5, 2.0, len(faces))
    got = P.external_force(0.3, face_pressure=fp)
    want = np.zeros_like(got)
    for f in range(len(faces)):
        P.mesh = dataclasses.replace(mesh, neu_faces=faces[f:f + 1])
        want += 0.3 * fp[f] * P.external_force(1.0)
    P.mesh = mesh
    assert np.allclose(got, want, rtol=1e-13, atol=1e-16)


def test_mooney_rivlin_ignores_fibre_parameters(small_tube):
    """The fibre terms belong to the artery model only: a Mooney-Rivlin
    material with nonzero k1, k2 and fibre directions gives the residual of
    the same material with k1 = 0."""
    base = Material(0, 0.5, 0.1, 0.0, 1.0, 1.0e3, 0.0)
    with_fibres = Material(0, 0.5, 0.1, 5.0, 2.0, 1.0e3, 0.0)
    s = _smooth_state(small_tube, 14)
    R = [O.Problem(dataclasses.replace(small_tube, materials=[m, m])).residual(s) for m in (base, with_fibres)]
    assert np.array_equal(R[0], R[1])


@pytest.mark.parametrize("pressure", [1.0e-4, 0.16])
def test_newton_stops_at_the_first_relative_residual_below_rtol(pressure):
    """Sec. 4.4 stop, relative reading r11: Newton returns the first iterate
    with ||R|| <= rtol ||R_0|| (for both a tiny and a moderate load, so the
    scale of R_0 does not matter)."""
    mesh = artery_tube(n_theta=16, n_z=2, length=0.125)
    P = O.Problem(mesh)
    rec = []
    v, k = P.newton(np.zeros((mesh.n_nodes, 4)), fext=P.external_force(pressure), rtol=1e-6, record=rec)
    assert len(rec) == k + 1
    assert rec[-1] <= 1e-6 * rec[0]
    assert all(r > 1e-6 * rec[0] for r in rec[:-1])
