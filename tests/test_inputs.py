"""The seeded input recipes and the benchmark's byte model (host logic, no GPU)."""
import math
import os
import sys

import numpy as np

from fixtures import artery_layers, artery_tube, batched_tubes

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _volumes(mesh):
    X, T = mesh.X, mesh.tets
    d = X[T[:, 1:]] - X[T[:, :1]]
    return np.linalg.det(d) / 6.0


def test_tube_sizes_and_orientation():
    """64 x 8 x 128 hexahedra x 6 tets: 393,216 tets, 74,304 nodes (theta
    periodic), all positively oriented, wall volume equal to the annulus."""
    mesh = artery_tube(materials=artery_layers(1.0e3))
    assert mesh.n_elems == 393216 and mesh.n_nodes == 64 * 9 * 129
    v = _volumes(mesh)
    assert (v > 0).all()
    # polygonal annulus of 64 sides between r = 1 and r = 1.23, length 8
    poly = 0.5 * 64 * math.sin(2 * math.pi / 64)
    assert abs(v.sum() - poly * (1.23 ** 2 - 1.0) * 8.0) <= 1e-9 * v.sum()


def test_batched_segments_recipe():
    """Segments of the seed-4 recipe (the first 32 of the 256: the draws are
    sequential per segment): contiguous node and element ranges, sizes drawn
    in [5e3, 2e5] up to the rounding of n_z, pressure in [0.5, 2.0]."""
    mesh = batched_tubes(32, seed=4)
    seg = mesh.seg_node
    assert (np.diff(seg) >= 0).all() and seg[0] == 0 and seg[-1] == 31
    sege = mesh.seg_elem
    assert (np.diff(sege) >= 0).all()
    counts = np.bincount(sege, minlength=32)
    # n_z = max(2, round(n_e / (6 n_r n_theta))) moves a segment by at most half a ring of hexahedra
    assert counts.min() >= 5.0e3 - 3 * 8 * 64 and counts.max() <= 2.0e5 + 3 * 8 * 64
    assert (mesh.face_pressure >= 0.5).all() and (mesh.face_pressure <= 2.0).all()
    assert (_volumes(mesh) > 0).all()
    # every tet lies in one segment
    assert (seg[mesh.tets] == sege[:, None]).all()


def test_bench_byte_model_of_the_block_jacobi_sweep():
    """The roofline numerator: n_b (64 + 4) + 4 (n + 1) + n (48 + 64) bytes per
    FP32 sweep, 79,622,148 at the 393k-tet tube (1,044,160 blocks)."""
    sys.path.insert(0, ROOT)
    import bench
    assert bench.jacobi0_bytes(74304, 1044160, True) == 1044160 * 68 + 4 * 74305 + 74304 * 112 == 79622148
    assert bench.jacobi0_bytes(74304, 1044160, False) == 1044160 * 132 + 4 * 74305 + 74304 * 224


def test_bench_byte_model_of_the_level1_product():
    """The second roofline numerator: n_b (49 v + 4) + 4 (n + 1) + 2 * 7 n x
    bytes per w = A z on level 1 (v, x: bytes per value and per vector entry),
    988,479,044 for the 3.1M tube's level 1 (69,904 rows, 4,921,424 blocks)."""
    sys.path.insert(0, ROOT)
    import bench
    assert bench.level1_spmv_bytes(69904, 4921424, True) == 4921424 * 200 + 4 * 69905 + 14 * 69904 * 4 == 988479044
    assert bench.level1_spmv_bytes(69904, 4921424, False) == 4921424 * 396 + 4 * 69905 + 14 * 69904 * 8
    assert bench.level1_spmv_bytes(69904, 4921424, True, bf16=True) == 4921424 * 102 + 4 * 69905 + 14 * 69904 * 4


def test_bench_reference_arm_prints_the_contract_line():
    """`bench.py --impl reference` times the oracle on the host and prints one
    JSON line with the contract's keys (no GPU involved)."""
    import json
    import subprocess
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line
    assert line["impl"] == "reference" and line["warmup"] >= 3 and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert "workload" in line["config"]
    # the reported steps at the reported time per step fit in what the arm ran
    assert line["steps"] * line["ms_per_step"] <= 1e3 * line["wall_s"]


def test_batched_segment_reproduces_the_union_mesh_segment():
    """batched_segment(i) rebuilds segment i of batched_tubes alone: same
    connectivity (shifted by the node offset), fibres, masks, face pressures and
    coordinates up to the x shift that keeps the segments apart."""
    from fixtures import batched_segment, batched_tubes
    m = batched_tubes(n_seg=5, seed=4)
    for i in range(5):
        t, off = batched_segment(i, n_seg=5, seed=4)
        nodes = np.flatnonzero(m.seg_node == i)
        assert nodes[0] == off and len(nodes) == t.n_nodes
        em = m.seg_elem == i
        assert np.array_equal(m.tets[em] - off, t.tets)
        assert np.array_equal(m.dir_mask[nodes], t.dir_mask)
        assert np.allclose(m.fibre[em], t.fibre)
        assert np.allclose(m.face_pressure[m.seg_face == i], t.face_pressure)
        assert np.allclose(m.X[nodes, 1:], t.X[:, 1:]) and np.allclose(np.ptp(m.X[nodes, 0] - t.X[:, 0]), 0.0)


def test_bench_ramp_driver_counts_newton_and_krylov_cap_hits():
    """The bench's load ramp advances on a converged start residual or after 12
    Newton steps (a Newton-cap hit), and counts linear solves that stopped at
    the Krylov cap above their tolerance (host logic, scripted solver)."""
    import types
    sys.path.insert(0, ROOT)
    import bench

    class FakeTorch:
        @staticmethod
        def zeros(shape, device=None, dtype=None):
            return types.SimpleNamespace(zero_=lambda: None)

    class FakeSolver:
        def __init__(self, script):
            self.script = list(script)

        def newton_step(self, state, load, check=False):
            res0, kits, lin_res = self.script.pop(0)
            return types.SimpleNamespace(status=0, res0=res0, krylov_its_last=kits, lin_res=lin_res)

    # load 1: converges at the 3rd step; load 2: never converges -> 13 steps then advance
    script = [(1.0, 10, 1e-9), (1e-3, 10, 1e-9), (1e-9, 600, 1e-6)]
    script += [(1.0, 10, 1e-9)] + [(0.5, 10, 1e-9)] * 12
    drv = bench.RampDriver.__new__(bench.RampDriver)
    drv.Load = lambda **kw: kw
    drv.fp = None
    drv.solver = FakeSolver(script)
    drv.torch = FakeTorch
    drv.state = FakeTorch.zeros(())
    drv.k, drv.r0, drv.newton_in_load = 1, None, 0
    drv.max_krylov, drv.krylov_rtol = 600, 1e-8
    drv.krylov_cap_hits = drv.newton_cap_hits = 0
    for _ in range(3):
        drv.step()
    assert drv.k == 2 and drv.krylov_cap_hits == 1 and drv.newton_cap_hits == 0
    for _ in range(13):
        drv.step()
    assert drv.k == 3 and drv.newton_cap_hits == 1


def test_tube_fibres_and_boundary_conditions():
    """Fibre directions (readings r1, r2): per element two unit vectors with
    no radial part at the element centroid, at +alpha and -alpha from e_theta
    towards e_z, alpha = 29 deg in the media (inner four layers) and 62 deg in
    the adventitia.  Ends (reading r13): u_z fixed on both end planes, u_x
    where x = 0 and u_y where y = 0 on them, nothing else, pressure free."""
    mesh = artery_tube(n_theta=16, n_z=4, length=1.0, materials=artery_layers(1.0e3))
    xc = mesh.X[mesh.tets].mean(axis=1)
    th = np.arctan2(xc[:, 1], xc[:, 0])
    e_r = np.stack([np.cos(th), np.sin(th), 0 * th], axis=1)
    e_t = np.stack([-np.sin(th), np.cos(th), 0 * th], axis=1)
    alpha = np.deg2rad(np.where(mesh.mat_id == 0, 29.0, 62.0))
    layer_r = np.hypot(xc[:, 0], xc[:, 1])
    assert (mesh.mat_id[layer_r < 1.13 * np.cos(np.pi / 16)] == 0).all() and (mesh.mat_id[layer_r > 1.13] == 1).all()
    for i, sgn in ((0, 1.0), (1, -1.0)):
        a = mesh.fibre[:, i, :]
        assert np.allclose(np.linalg.norm(a, axis=1), 1.0, atol=1e-14)
        assert np.abs(np.einsum("ei,ei->e", a, e_r)).max() <= 1e-14
        assert np.allclose(np.einsum("ei,ei->e", a, e_t), np.cos(alpha), atol=1e-14)
        assert np.allclose(a[:, 2], sgn * np.sin(alpha), atol=1e-14)
    X, m = mesh.X, mesh.dir_mask
    end = np.isclose(X[:, 2], 0.0) | np.isclose(X[:, 2], 1.0)
    assert (m[:, 2] == end).all()
    assert (m[:, 0] == (end & np.isclose(X[:, 0], 0.0, atol=1e-12))).all()
    assert (m[:, 1] == (end & np.isclose(X[:, 1], 0.0, atol=1e-12))).all()
    assert (m[:, 3] == 0).all()


def test_bench_default_is_the_documented_headline_configuration():
    """`python bench.py` with no flags times the refined tube (128 x 16 x 256
    hexahedra, kappa = 1e5 c10) in FP32 + refinement with grown aggregates,
    FGMRES to 1e-8 (Krylov cap 600) and the library's default smoothers; the
    plain-FP64 arm differs only in precision; `--config tube` switches to ring
    aggregates on the 393k tube at kappa = 1e3 c10."""
    sys.path.insert(0, ROOT)
    import bench
    args = bench.make_parser().parse_args([])
    assert (args.config, args.precision, args.gpus, args.steps >= 10, args.warmup >= 3) == \
        ("refined", "fp32", 1, True, True)
    assert bench._workload_geometry(args) == (128, 16, 256, 1.0e5)
    o = bench.solver_options(args)
    assert o == dict(precision=1, newton_rtol=1e-8, krylov_rtol=1e-8, use_graphs=1, amg_lag=0, max_krylov=600,
                     aggregation=1, segment_krylov=1)
    args.precision = "fp64"
    assert bench.solver_options(args) == dict(o, precision=0)
    tube = bench.make_parser().parse_args(["--config", "tube"])
    assert bench._workload_geometry(tube) == (64, 8, 128, 1.0e3)
    assert bench.solver_options(tube)["aggregation"] == 0


def test_batched_segment_parameters_follow_the_recipe():
    """Per segment of the seed-4 recipe: n_theta = 32 below 5e4 tets, else 64;
    n_z = max(2, round(n_e / (6 * 8 * n_theta))); one fibre angle in
    [20, 70] deg used at +/- alpha in both layers; kappa = ratio * c10 of the
    media for both layers with ratio in [1e2, 1e5]; the segment's pressure on
    its own faces."""
    mesh = batched_tubes(32, seed=4)
    segs = mesh.meta["segments"]
    for s, sg in enumerate(segs):
        em = mesh.seg_elem == s
        n_e = int(em.sum())
        assert sg["n_elems"] == n_e and sg["n_theta"] == (32 if n_e < 5.0e4 else 64)
        assert n_e == 6 * 8 * sg["n_theta"] * sg["n_z"] and sg["n_z"] >= 2
        assert 20.0 <= sg["alpha_deg"] <= 70.0 and 1.0e2 <= sg["kappa_ratio"] <= 1.0e5
        a = mesh.fibre[em]
        assert np.allclose(np.abs(a[:, :, 2]), np.sin(np.deg2rad(sg["alpha_deg"])), atol=1e-12)
        mats = [mesh.materials[m] for m in np.unique(mesh.mat_id[em])]
        assert len(mats) == 2 and all(m.kappa == mats[0].kappa for m in mats)
        assert np.isclose(mats[0].kappa, sg["kappa_ratio"] * max(m.c10 for m in mats), rtol=1e-12)
        assert np.allclose(mesh.face_pressure[mesh.seg_face == s], sg["pressure"])
    # the draws spread over their ranges (32 segments)
    alphas = np.array([sg["alpha_deg"] for sg in segs])
    ratios = np.log10([sg["kappa_ratio"] for sg in segs])
    assert alphas.max() - alphas.min() > 30.0 and ratios.max() - ratios.min() > 2.0
