"""GPU path (through the C ABI) against the FP64 oracle, element by element.

Tolerances (FP64 mode): residual and tangent entries within 1e-12 of the
largest reference entry of the same block row; linear solves within 1e-10;
Newton solutions within 1e-8 (relative to the largest entry).  Colouring and
assembly are compared bit for bit.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from fixtures import artery_layers, artery_tube, cube_uniaxial_bc, kuhn_cube, mooney_rivlin
from oracle import solid as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _solver(mesh, **kw):
    from paper_1312_5561_gb300.binding import SolidSolver
    return SolidSolver(mesh, **kw)


def _t(a):
    return torch.tensor(np.ascontiguousarray(a), device="cuda", dtype=torch.float64)


def _smooth_state(mesh, seed, amp=0.06, pamp=0.3, noise=0.001):
    rng = np.random.default_rng(seed)
    s = np.zeros((mesh.n_nodes, 4))
    s[:, :3] = mesh.X @ (amp * rng.standard_normal((3, 3))).T + noise * rng.standard_normal((mesh.n_nodes, 3))
    s[:, 3] = pamp * rng.standard_normal(mesh.n_nodes)
    return s


def _bsr_to_csr(row_ptr, col_idx, vals, n):
    return sp.bsr_matrix((vals.astype(np.float64), col_idx, row_ptr), shape=(4 * n, 4 * n)).tocsr()


def _blockrow_rel_err(Kg, Kr, n):
    """max over block rows of max|Kg - Kr| / max|Kr| within that block row."""
    D = (Kg - Kr).tocsr()
    worst = 0.0
    Ar = abs(Kr).tocsr()
    Ad = abs(D).tocsr()
    for i in range(n):
        sl = slice(4 * i, 4 * i + 4)
        ref = Ar[sl].max()
        d = Ad[sl].max()
        if ref > 0:
            worst = max(worst, d / ref)
    return worst


MESHES = {
    "cube_mr": lambda: cube_uniaxial_bc(kuhn_cube(4), stretch=0.1),
    "tube_artery": lambda: artery_tube(n_theta=16, n_z=6, materials=artery_layers(1.0e3)),
}


@pytest.mark.parametrize("assembly", [0, 1], ids=["gather", "colour"])
@pytest.mark.parametrize("name", list(MESHES))
def test_residual_and_tangent_parity(name, assembly):
    """Both assembly paths: element buffers + fixed-order gather (0) and the
    colour-ordered scatter (1)."""
    mesh = MESHES[name]()
    P = O.Problem(mesh)
    s = _smooth_state(mesh, 3)
    pressure = 1.3 if len(mesh.neu_faces) else 0.0
    from paper_1312_5561_gb300.binding import Load
    solver = _solver(mesh, assembly=assembly)
    R = solver.residual_tangent(_t(s), Load(pressure=pressure)).cpu().numpy()
    R_ref = P.residual(s, P.external_force(pressure))
    scale = np.abs(R_ref).max(axis=1, keepdims=True)
    assert np.all(np.abs(R - R_ref) <= 1e-12 * np.maximum(scale, np.abs(R_ref).max() * 1e-3))
    rp, ci, vals = solver.bsr()
    Kg = _bsr_to_csr(rp, ci, vals, mesh.n_nodes)
    Kr = P.tangent(s)
    assert _blockrow_rel_err(Kg, Kr, mesh.n_nodes) <= 1e-12
    if name == "tube_artery":
        # both fibre families were active in part of the mesh
        g, V, h, mp, fib = P._sub(np.arange(mesh.n_elems))
        act = O.fibre_activity(s[mesh.tets], g, fib)
        assert act.any(axis=1).all() and not act.all()


@pytest.mark.parametrize("assembly", [0, 1], ids=["gather", "colour"])
def test_assembly_is_bitwise_deterministic_and_colouring_matches(assembly):
    mesh = MESHES["tube_artery"]()
    s = _t(_smooth_state(mesh, 5))
    solver = _solver(mesh, assembly=assembly)
    R1 = solver.residual_tangent(s).clone()
    _, _, v1 = solver.bsr()
    R2 = solver.residual_tangent(s).clone()
    _, _, v2 = solver.bsr()
    assert torch.equal(R1, R2)
    assert np.array_equal(v1.view(np.uint64), v2.view(np.uint64))
    col, nc = solver.colouring()
    ref = O.greedy_colouring(mesh.tets, mesh.n_nodes)
    assert np.array_equal(col, ref) and nc == ref.max() + 1


def test_spmv_parity():
    mesh = MESHES["cube_mr"]()
    P = O.Problem(mesh)
    s = _smooth_state(mesh, 9)
    solver = _solver(mesh)
    solver.residual_tangent(_t(s))
    x = np.random.default_rng(1).standard_normal((mesh.n_nodes, 4))
    y = solver.spmv(_t(x)).cpu().numpy().ravel()
    y_ref = P.tangent(s) @ x.ravel()
    assert np.abs(y - y_ref).max() <= 1e-12 * np.abs(y_ref).max()


@pytest.mark.parametrize("n,krylov,precond,smoother", [(2, 0, 0, 0), (8, 0, 0, 0), (8, 1, 0, 0), (2, 1, 1, 0),
                                                      (8, 1, 1, 0), (8, 0, 1, 0), (2, 0, 0, 1), (8, 0, 0, 1),
                                                      (8, 1, 1, 1)])
def test_linear_solve_against_direct(n, krylov, precond, smoother):
    """Krylov (FGMRES or BiCGStab) preconditioned by one AMG V-cycle on K
    (precond 0) or by the block-triangular P_L of Eq. lpre (precond 1), with
    block-Jacobi (smoother 0) or Vanka (smoother 1) on the finest level,
    against a direct solve (dense LU for the 2x2x2 cube)."""
    mesh = cube_uniaxial_bc(kuhn_cube(n), stretch=0.1)
    P = O.Problem(mesh)
    s = P.apply_dirichlet(_smooth_state(mesh, 4, amp=0.05), mesh.dir_values(1.0))
    # BiCGStab's recursively updated residual stalls near 1e-13: ask it for 1e-12
    solver = _solver(mesh, krylov_rtol=1e-13 if krylov == 0 else 1e-12, max_krylov=2000, krylov=krylov,
                     precond=precond, smoother=smoother, vanka_omega=0.78)
    solver.residual_tangent(_t(s))
    rng = np.random.default_rng(2)
    b = rng.standard_normal((mesh.n_nodes, 4)) * (mesh.dir_mask == 0)
    x, info = solver.linear_solve(_t(b))
    K = P.tangent(s)
    if n == 2:
        x_ref = np.linalg.solve(K.toarray(), b.ravel())
    else:
        x_ref = spla.spsolve(K.tocsc(), b.ravel())
    x = x.cpu().numpy().ravel()
    assert np.abs(x - x_ref).max() <= 1e-10 * np.abs(x_ref).max()


def _oracle_ramp(mesh, steps, pressure=0.0, rtol=1e-12):
    P = O.Problem(mesh)
    s = np.zeros((mesh.n_nodes, 4))
    for k in range(1, steps + 1):
        s = P.apply_dirichlet(s, mesh.dir_values(k / steps))
        fext = P.external_force(pressure * k / steps) if pressure else None
        s, _ = P.newton(s, fext=fext, rtol=rtol)
    return s


def test_newton_cube_mooney_rivlin_config():
    """Unit cube 8^3 x 6 tets, MR c10=0.5 c01=0.1 kappa=1e3, bottom clamped, top
    stretched 20% in 5 load steps; Newton rtol 1e-10, Krylov rtol 1e-12."""
    from paper_1312_5561_gb300.binding import Load
    mesh = cube_uniaxial_bc(kuhn_cube(8, materials=mooney_rivlin(0.5, 0.1, 1.0e3)), stretch=0.2)
    solver = _solver(mesh, newton_rtol=1e-10, krylov_rtol=1e-12, max_krylov=1000)
    state = torch.zeros((mesh.n_nodes, 4), device="cuda", dtype=torch.float64)
    for k in range(1, 6):
        info = solver.solve(state, Load(dir_values=_t(mesh.dir_values(k / 5))))
        assert info.newton_its <= 10
    ref = _oracle_ramp(mesh, 5)
    got = state.cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-8 * np.abs(ref).max()


@pytest.fixture(scope="module")
def small_artery():
    mesh = artery_tube(n_theta=64, n_z=8, length=0.5, materials=artery_layers(1.0e3))
    return mesh, _oracle_ramp(mesh, 4, pressure=0.64)


@pytest.mark.parametrize("solver_kw", [
    dict(krylov_rtol=1e-12, max_krylov=1000),
    # the paper's solid solver: BiCGStab with P_L (Sec. 5.4.2), FP32 tangent and V-cycle
    dict(krylov=1, precond=1, precision=1, krylov_rtol=1e-10, max_krylov=3000),
    # the paper's Vanka smoother (Sec. 5.5.2) on the finest level, FP32
    dict(smoother=1, precision=1, krylov_rtol=1e-12, max_krylov=1000),
    # FP32 + refinement with BF16 coarse-level operators in the V-cycle
    dict(precision=1, coarse_bf16=1, krylov_rtol=1e-12, max_krylov=1000),
], ids=["fgmres_amg", "bicgstab_pl_fp32", "vanka_fp32", "coarse_bf16"])
def test_newton_small_artery_pressure_ramp(small_artery, solver_kw):
    """Two-layer artery, 64 x 8 x 8 hexes (length 0.5), internal pressure
    ramped to 0.64 in 4 steps (the same increments as 0 -> 1.6 in 10)."""
    from paper_1312_5561_gb300.binding import Load
    mesh, ref = small_artery
    solver = _solver(mesh, newton_rtol=1e-10, **solver_kw)
    state = torch.zeros((mesh.n_nodes, 4), device="cuda", dtype=torch.float64)
    steps = 4
    for k in range(1, steps + 1):
        info = solver.solve(state, Load(pressure=0.16 * k))
        assert info.newton_its <= 8
    got = state.cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-8 * np.abs(ref).max()


def test_inverted_element_is_reported():
    from paper_1312_5561_gb300.binding import FsiError
    mesh = kuhn_cube(2)
    solver = _solver(mesh)
    s = np.zeros((mesh.n_nodes, 4))
    s[:, 2] = -2.0 * mesh.X[:, 2]            # J < 0 everywhere
    with pytest.raises(FsiError) as e:
        solver.residual_tangent(_t(s))
    assert e.value.status == -4
    # the handle stays usable
    R = solver.residual_tangent(_t(np.zeros((mesh.n_nodes, 4))))
    assert float(R.abs().max()) == 0.0


def test_single_element_mesh():
    from fixtures.meshes import Mesh
    X = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1.0]])
    mesh = Mesh(X=X, tets=np.array([[0, 1, 2, 3]], np.int32), mat_id=np.zeros(1, np.int32),
                fibre=np.zeros((1, 2, 3)), dir_mask=np.zeros((4, 4), np.uint8),
                neu_faces=np.zeros((0, 3), np.int32), materials=mooney_rivlin())
    P = O.Problem(mesh)
    s = _smooth_state(mesh, 1, amp=0.1)
    solver = _solver(mesh)
    R = solver.residual_tangent(_t(s)).cpu().numpy()
    assert np.abs(R - P.residual(s)).max() <= 1e-12 * np.abs(P.residual(s)).max()


# ---------------------------------------------------------------- FP32 tangent + FP32 V-cycle, FP64 residual
@pytest.mark.parametrize("name", list(MESHES))
def test_fp32_tangent_parity(name):
    """FP32 tangent entries within 1e-5 of the largest reference entry of their block row."""
    mesh = MESHES[name]()
    P = O.Problem(mesh)
    s = _smooth_state(mesh, 3)
    solver = _solver(mesh, precision=1)
    R = solver.residual_tangent(_t(s)).cpu().numpy()
    R_ref = P.residual(s)
    assert np.abs(R - R_ref).max() <= 1e-12 * np.abs(R_ref).max()      # the residual stays FP64
    rp, ci, vals = solver.bsr()
    assert vals.dtype == np.float32
    assert _blockrow_rel_err(_bsr_to_csr(rp, ci, vals, mesh.n_nodes), P.tangent(s), mesh.n_nodes) <= 1e-5


def test_fp32_refinement_reaches_fp64_solution():
    """Newton with the FP32 tangent and V-cycle (iterative refinement by the FP64
    residual) converges to the FP64 oracle solution within 1e-8."""
    from paper_1312_5561_gb300.binding import Load
    mesh = artery_tube(n_theta=64, n_z=8, length=0.5, materials=artery_layers(1.0e5))
    solver = _solver(mesh, precision=1, newton_rtol=1e-11, krylov_rtol=1e-8, max_krylov=1000)
    state = torch.zeros((mesh.n_nodes, 4), device="cuda", dtype=torch.float64)
    for k in range(1, 3):
        solver.solve(state, Load(pressure=0.16 * k))
    ref = _oracle_ramp(mesh, 2, pressure=0.32)
    got = state.cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-8 * np.abs(ref).max()


# ---------------------------------------------------------------- batched independent segments
def test_batched_segments_match_oracle():
    """Four uneven artery segments in one handle (seed 35: 6,144 to 29,184
    elements, kappa/c10 from 101 to 63,829, own fibre angles and pressures):
    after two load steps each segment matches the oracle solution of that
    segment alone."""
    from fixtures import batched_tubes
    from paper_1312_5561_gb300.binding import Load
    mesh = batched_tubes(n_seg=4, seed=35, ne_range=(5.0e3, 3.0e4))
    kr = [sg["kappa_ratio"] for sg in mesh.meta["segments"]]
    assert min(kr) < 2e2 and max(kr) > 5e4
    solver = _solver(mesh, precision=1, newton_rtol=1e-10, krylov_rtol=1e-8, max_krylov=600)
    assert solver.levels()[-1][0] >= 4            # the coarsest level keeps one block per segment at least
    fp = _t(mesh.face_pressure)
    state = torch.zeros((mesh.n_nodes, 4), device="cuda", dtype=torch.float64)
    for k in (1, 2):
        info = solver.solve(state, Load(pressure=0.1 * k, face_pressure=fp))
        assert info.status == 0
    got = state.cpu().numpy()
    for sg in range(4):
        sub = _segment(mesh, sg)
        P = O.Problem(sub)
        ref = np.zeros((sub.n_nodes, 4))
        for k in (1, 2):
            ref, _ = P.newton(ref, fext=P.external_force(0.1 * k, face_pressure=sub.face_pressure), rtol=1e-12)
        m = mesh.seg_node == sg
        assert np.abs(got[m] - ref).max() <= 1e-8 * np.abs(ref).max()


def _segment(mesh, sg):
    """Segment sg of a batched mesh as a mesh of its own (nodes keep their order)."""
    from fixtures.meshes import Mesh
    nodes = np.flatnonzero(mesh.seg_node == sg)
    off = nodes[0]
    em = mesh.seg_elem == sg
    fm = mesh.seg_face == sg
    mats = mesh.materials[2 * sg:2 * sg + 2]
    return Mesh(X=mesh.X[nodes], tets=(mesh.tets[em] - off).astype(np.int32), mat_id=mesh.mat_id[em] - 2 * sg,
                fibre=mesh.fibre[em], dir_mask=mesh.dir_mask[nodes], neu_faces=(mesh.neu_faces[fm] - off).astype(np.int32),
                materials=mats, face_pressure=mesh.face_pressure[fm])


def test_adaptive_inner_tolerance_keeps_the_solution():
    """eps_1,k = eps_2,k-1^2 (Sec. 4.4): fewer Krylov iterations, same Newton solution."""
    from paper_1312_5561_gb300.binding import Load
    mesh = artery_tube(n_theta=64, n_z=8, length=0.5, materials=artery_layers(1.0e3))
    its = {}
    sols = {}
    for adaptive in (0, 1):
        solver = _solver(mesh, newton_rtol=1e-10, krylov_rtol=1e-10, adaptive_tol=adaptive, max_krylov=600)
        state = torch.zeros((mesh.n_nodes, 4), device="cuda", dtype=torch.float64)
        info = solver.solve(state, Load(pressure=0.16))
        its[adaptive] = info.krylov_its_total
        sols[adaptive] = state.cpu().numpy()
    assert its[1] < its[0]
    assert np.abs(sols[1] - sols[0]).max() <= 1e-8 * np.abs(sols[0]).max()


@pytest.mark.parametrize("precision", [0, 1])
def test_vanka_solve_is_bitwise_reproducible(precision):
    """Patches of one colour share no unknown, so the smoother has no race: two
    solves of the same system agree bit for bit."""
    mesh = cube_uniaxial_bc(kuhn_cube(6), stretch=0.1)
    s = _smooth_state(mesh, 4, amp=0.05)
    solver = _solver(mesh, smoother=1, precision=precision, krylov_rtol=1e-10, max_krylov=500)
    solver.residual_tangent(_t(s))
    b = np.random.default_rng(5).standard_normal((mesh.n_nodes, 4)) * (mesh.dir_mask == 0)
    x1, i1 = solver.linear_solve(_t(b))
    x2, i2 = solver.linear_solve(_t(b))
    assert i1.krylov_its_last == i2.krylov_its_last
    assert torch.equal(x1, x2)


def test_grown_aggregates_on_a_wall_of_sixteen_thin_layers():
    """Tube wall meshed with 16 element layers (the refined tube's radial
    resolution), pressure ramp to 0.32 in 2 steps: with aggregates grown along
    the strongest connections the solve converges to the oracle's solution."""
    from paper_1312_5561_gb300.binding import Load
    mesh = artery_tube(n_theta=32, n_media=8, n_adv=8, n_z=4, length=0.25, materials=artery_layers(1.0e3))
    solver = _solver(mesh, aggregation=1, precision=1, newton_rtol=1e-10, krylov_rtol=1e-12, max_krylov=1000)
    state = torch.zeros((mesh.n_nodes, 4), device="cuda", dtype=torch.float64)
    for k in (1, 2):
        info = solver.solve(state, Load(pressure=0.16 * k))
        assert info.newton_its <= 8
    ref = _oracle_ramp(mesh, 2, pressure=0.32)
    got = state.cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-8 * np.abs(ref).max()


def test_newmark_advance_matches_the_oracle():
    """fsi_solid_newmark_advance against the oracle's Newmark-beta bookkeeping
    (Sec. 4.1.2): new acceleration, velocity and history, and d_(n) stored."""
    from oracle import newmark as N
    mesh = MESHES["cube_mr"]()
    solver = _solver(mesh)
    rng = np.random.default_rng(7)
    n = mesh.n_nodes
    state = rng.standard_normal((n, 4))
    disp, vel, acc = (rng.standard_normal((n, 3)) for _ in range(3))
    beta, gamma, dt = 0.625, 1.0, 0.01
    a_ref, v_ref, h_ref = N.newmark_update(state[:, :3], disp, vel, acc, beta, gamma, dt)
    D, Vv, A = _t(disp), _t(vel), _t(acc)
    H = torch.zeros((n, 3), device="cuda", dtype=torch.float64)
    solver.newmark_advance(_t(state), D, Vv, A, H, beta, gamma, dt)
    assert np.array_equal(D.cpu().numpy(), state[:, :3])
    for got, ref in ((A, a_ref), (Vv, v_ref), (H, h_ref)):
        assert np.abs(got.cpu().numpy() - ref).max() <= 1e-13 * np.abs(ref).max()


def test_inertia_residual_and_tangent_parity():
    """Residual and tangent with the Newmark inertia terms (inertia coefficient
    1 / (beta dt^2), rho = 1.2, a nodal history) against the oracle."""
    from paper_1312_5561_gb300.binding import Load
    mesh = artery_tube(n_theta=16, n_z=6, materials=artery_layers(1.0e3, rho=1.2))
    c = 1.0 / (0.625 * 0.01 ** 2)
    P = O.Problem(mesh, O.Options(inertia_coef=c))
    s = _smooth_state(mesh, 4)
    hist = c * s[:, :3] + np.random.default_rng(9).standard_normal((mesh.n_nodes, 3))
    solver = _solver(mesh, inertia_coef=c)
    R = solver.residual_tangent(_t(s), Load(pressure=1.3, hist=_t(hist))).cpu().numpy()
    R_ref = P.residual(s, P.external_force(1.3), hist)
    scale = np.abs(R_ref).max(axis=1, keepdims=True)
    assert np.all(np.abs(R - R_ref) <= 1e-12 * np.maximum(scale, np.abs(R_ref).max() * 1e-3))
    rp, ci, vals = solver.bsr()
    Kg = _bsr_to_csr(rp, ci, vals, mesh.n_nodes)
    assert _blockrow_rel_err(Kg, P.tangent(s, hist), mesh.n_nodes) <= 1e-12


@pytest.mark.parametrize("precision", [0, 1])
def test_newton_step_reports_the_mass_norm_increment(precision):
    """info.inc_mnorm is ||dv||_M (Sec. 4.4, Eq. newstop) of the update the
    step applied, and info.inc_norm its Euclidean norm."""
    from paper_1312_5561_gb300.binding import Load
    mesh = MESHES["cube_mr"]()
    P = O.Problem(mesh)
    s0 = P.apply_dirichlet(np.zeros((mesh.n_nodes, 4)), mesh.dir_values(0.5))
    solver = _solver(mesh, precision=precision)
    state = _t(s0)
    info = solver.newton_step(state, Load())
    dv = state.cpu().numpy() - s0
    assert abs(info.inc_mnorm - P.mass_norm(dv)) <= 1e-12 * P.mass_norm(dv)
    assert abs(info.inc_norm - np.linalg.norm(dv)) <= 1e-12 * np.linalg.norm(dv)
    assert info.inc_mnorm > 0


def test_autotuner_choices_are_valid_and_keep_the_solution():
    """The launch shapes the autotuner picks lie in their candidate sets, and
    the tuned and the default launch shapes give the same Newton solution."""
    from paper_1312_5561_gb300.binding import Load
    mesh = artery_tube(n_theta=64, n_z=8, length=0.5, materials=artery_layers(1.0e3))
    sols = []
    for tune in (1, 0):
        solver = _solver(mesh, precision=1, autotune=tune, newton_rtol=1e-10, krylov_rtol=1e-10, max_krylov=600)
        t = solver.tuning()
        assert len(t) == len(solver.levels())          # element CTA + every smoothed level
        if tune:
            assert t[0] in (64, 128) and t[1] in (64, 128, 256) and all(v in (1, 2) for v in t[2:])
        else:
            assert t[0] == 128 and all(v == 0 for v in t[1:])
        state = torch.zeros((mesh.n_nodes, 4), device="cuda", dtype=torch.float64)
        info = solver.solve(state, Load(pressure=0.16))
        assert info.status == 0
        sols.append(state.cpu().numpy())
    assert np.abs(sols[0] - sols[1]).max() <= 1e-8 * np.abs(sols[1]).max()
