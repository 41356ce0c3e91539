"""The allocation-free entry point fsi_dots_static against the solver's own
reduction.

Some callers cannot allocate device memory (a host application that owns all
device allocations, or code that must not call cudaMalloc after start-up
because it synchronises the device).  fsi_dots_static serves them with a
fixed device array instead of handle memory.  Here its result is compared,
through the C ABI, with the residual norm that fsi_solid_newton_step reports
(the same deterministic reduction run from handle memory), on two calls in a
row.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _state(mesh, seed=3):
    rng = np.random.default_rng(seed)
    s = np.zeros((mesh.n_nodes, 4))
    s[:, :3] = mesh.X @ (0.05 * rng.standard_normal((3, 3))).T
    s[:, 3] = 0.2 * rng.standard_normal(mesh.n_nodes)
    return torch.tensor(s, device="cuda", dtype=torch.float64)


def test_dots_static_matches_the_newton_step_residual_norm():
    from fixtures import cube_uniaxial_bc, kuhn_cube
    from paper_1312_5561_gb300 import binding as B

    mesh = cube_uniaxial_bc(kuhn_cube(4), stretch=0.1)
    solver = B.SolidSolver(mesh)
    state = _state(mesh)
    R = solver.residual_tangent(state).contiguous()
    info = solver.newton_step(state.clone())           # existing entry point: reports ||R(state)||_2
    ref = info.res0
    assert ref > 0
    n = R.numel()
    stream = torch.cuda.current_stream().cuda_stream
    out = torch.full((4,), float("nan"), device="cuda", dtype=torch.float64)
    for _ in range(2):                                  # two calls in a row share the static scratch
        st = B.lib.fsi_dots_static(R.data_ptr(), n, 1, R.data_ptr(), n, out.data_ptr(), ctypes.c_void_p(stream))
        assert st == 0
        got = float(out[0].sqrt().item())
        assert got == ref                               # same 304-partial reduction as the solver

    # several vectors at once: V = [R, 2R, state]
    V = torch.stack([R.reshape(-1), 2.0 * R.reshape(-1), state.reshape(-1)]).contiguous()
    st = B.lib.fsi_dots_static(V.data_ptr(), n, 3, R.data_ptr(), n, out.data_ptr(), ctypes.c_void_p(stream))
    assert st == 0
    got = out[:3].cpu().numpy()
    assert abs(got[0] - ref * ref) <= 1e-12 * ref * ref
    assert abs(got[1] - 2.0 * ref * ref) <= 1e-12 * ref * ref
    exp2 = float(torch.dot(state.reshape(-1), R.reshape(-1)).item())
    assert abs(got[2] - exp2) <= 1e-12 * max(abs(exp2), ref * float(state.norm().item()))


def test_dots_static_rejects_sizes_beyond_its_array():
    from paper_1312_5561_gb300 import binding as B

    x = torch.ones(16, device="cuda", dtype=torch.float64)
    out = torch.empty(64, device="cuda", dtype=torch.float64)
    too_many = 33                                       # FSI_DOTS_STATIC_MAX_VECTORS + 1
    V = torch.ones((too_many, 16), device="cuda", dtype=torch.float64)
    assert B.lib.fsi_dots_static(V.data_ptr(), 16, too_many, x.data_ptr(), 16, out.data_ptr(), None) == -1
    assert B.lib.fsi_dots_static(V.data_ptr(), 16, 0, x.data_ptr(), 16, out.data_ptr(), None) == -1
    assert B.lib.fsi_dots_static(V.data_ptr(), 16, 32, x.data_ptr(), 16, out.data_ptr(), None) == 0
    assert float(out[31].item()) == 16.0
