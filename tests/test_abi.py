"""The C-ABI library loads and exports every symbol include/fsi_solid.h declares
(no compute calls: these run without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "fsi_solid.h")).read()
    return sorted(set(re.findall(r"\b(fsi_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1312_5561_gb300 import build
    if not os.path.exists(build.lib_path()):
        build.build()
    return ctypes.CDLL(build.lib_path())


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n


def test_binding_lists_every_symbol():
    from paper_1312_5561_gb300 import binding
    assert sorted(binding.EXPORTS) == _declared()


def test_struct_layouts_match_header():
    """Sizes of the ctypes mirrors equal the C sizes (checked with the host compiler)."""
    import subprocess
    import tempfile
    from paper_1312_5561_gb300 import binding as b
    code = ('#include "fsi_solid.h"\n#include <stdio.h>\n#include <stddef.h>\nint main(){printf("%zu %zu %zu %zu %zu %zu '
            '%zu %zu %zu %zu\\n",'
            'sizeof(fsi_mesh_desc),sizeof(fsi_material),sizeof(fsi_solver_opts),sizeof(fsi_load),sizeof(fsi_info),'
            'offsetof(fsi_solver_opts, omega),offsetof(fsi_solver_opts, schur_theta),sizeof(fsi_dn_opts),'
            'sizeof(fsi_dn_info),offsetof(fsi_dn_opts, max_cycles));}')
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "s.c")
        open(src, "w").write(code)
        exe = os.path.join(d, "s")
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), src, "-o", exe])
        sizes = list(map(int, subprocess.check_output([exe]).split()))
    got = [ctypes.sizeof(b.MeshDesc), ctypes.sizeof(b.MaterialDesc), ctypes.sizeof(b.SolverOpts),
           ctypes.sizeof(b.LoadDesc), ctypes.sizeof(b.Info), b.SolverOpts.omega.offset,
           b.SolverOpts.schur_theta.offset, ctypes.sizeof(b.DnOpts), ctypes.sizeof(b.DnInfo),
           b.DnOpts.max_cycles.offset]
    assert got == sizes


def test_create_error_is_reported_without_gpu_work(lib):
    """A NULL mesh is rejected before any CUDA call."""
    from paper_1312_5561_gb300 import binding as b
    h = ctypes.c_void_p()
    st = b.lib.fsi_solid_create(None, 0, None, None, ctypes.byref(h))
    assert st == -1 and not h.value
    assert b"required" in b.lib.fsi_solid_last_error(None)


def _one_tet_desc(seg, n_segments):
    """A single positively oriented tetrahedron with the given segment ids."""
    import numpy as np
    from paper_1312_5561_gb300 import binding as b
    keep = dict(X=np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], np.float64),
                tets=np.array([[0, 1, 2, 3]], np.int32), mat=np.zeros(1, np.int32),
                mask=np.zeros((4, 4), np.uint8), seg=np.asarray(seg, np.int32))
    d = b.MeshDesc()
    d.n_nodes, d.n_elems = 4, 1
    d.X, d.tets, d.mat_id = keep["X"].ctypes.data, keep["tets"].ctypes.data, keep["mat"].ctypes.data
    d.dir_mask = keep["mask"].ctypes.data
    d.n_segments = n_segments
    d.seg_node = keep["seg"].ctypes.data
    mats = (b.MaterialDesc * 1)(b.MaterialDesc(0, 0.5, 0.1, 0.0, 1.0, 500.0, 0.0))
    return d, mats, keep


@pytest.mark.parametrize("seg, n_segments, msg", [
    ([0, 0, 1, 1], 2, b"joins two segments"),
    ([-1, 0, 0, 0], 1, b"seg_node out of range"),
    ([0, 0, 0, 2], 2, b"seg_node out of range"),
    ([1, 1, 0, 0], 2, b"non-decreasing"),
    ([0, 0, 0, 0], 0, b"n_segments < 1"),
])
def test_bad_segment_tables_are_rejected_before_gpu_work(lib, seg, n_segments, msg):
    """Segment ids outside [0, n_segments), a decreasing table or an element
    spanning two segments is an argument error found on the host."""
    from paper_1312_5561_gb300 import binding as b
    d, mats, keep = _one_tet_desc(seg, n_segments)
    h = ctypes.c_void_p()
    st = b.lib.fsi_solid_create(ctypes.byref(d), 1, mats, None, ctypes.byref(h))
    assert st == -1 and not h.value
    assert msg in b.lib.fsi_solid_last_error(None)


def test_binding_fails_loudly_without_the_library(tmp_path):
    """No CPU fallback: importing the binding from a package copy whose
    library was never built raises ImportError naming the missing file."""
    import shutil
    import subprocess
    import sys
    pkg = os.path.join(ROOT, "paper_1312_5561_gb300")
    dst = tmp_path / "paper_1312_5561_gb300"
    shutil.copytree(pkg, dst, ignore=shutil.ignore_patterns("_lib", "__pycache__", "csrc"))
    code = ("import sys; sys.path.insert(0, %r)\n"
            "try:\n    import paper_1312_5561_gb300.binding\nexcept ImportError as e:\n    print('IMPORT-ERROR', e)\n"
            "else:\n    print('LOADED')\n") % str(tmp_path)
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300, cwd=str(tmp_path))
    assert "IMPORT-ERROR" in out.stdout and "libfsi_solid.so is missing" in out.stdout, out.stdout + out.stderr


def test_bad_power_steps_is_rejected_before_gpu_work(lib):
    """opts.power_steps outside [1, 10000] is an argument error found on the host."""
    from paper_1312_5561_gb300 import binding as b
    d, mats, keep = _one_tet_desc([0, 0, 0, 0], 1)
    for steps in (0, 20000):
        o = b.default_opts(power_steps=steps)
        h = ctypes.c_void_p()
        st = b.lib.fsi_solid_create(ctypes.byref(d), 1, mats, ctypes.byref(o), ctypes.byref(h))
        assert st == -1 and not h.value
        assert b"power_steps" in b.lib.fsi_solid_last_error(None)
    assert b.default_opts().power_steps == 20 and b.default_opts().exact_candidates == 0
