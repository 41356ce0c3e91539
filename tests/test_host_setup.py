"""The host mesh set-up of the library (element colouring, node-block pattern,
block lookup), run on the CPU through a small C++ driver: the colouring is the
oracle's greedy first-fit colouring element for element and is a proper
colouring; the pattern is the node adjacency of the mesh plus the diagonal."""
import os
import subprocess

import numpy as np
import pytest
import scipy.sparse as sp

import oracle.solid as O
from fixtures import artery_layers, artery_tube, kuhn_cube
from host_cxx import compile_driver


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    return compile_driver("host_setup_main.cpp", ["setup.cpp"], tmp_path_factory.mktemp("setup") / "host_setup_main")


def _star(n_spokes):
    """n_spokes tetrahedra that all share node 0 (so the colouring needs
    n_spokes colours, more than one 64-bit word of the colour sets)."""
    tets = np.array([[0, 1 + 3 * k, 2 + 3 * k, 3 + 3 * k] for k in range(n_spokes)], np.int32)
    return 1 + 3 * n_spokes, tets


def _run(exe, d, n_nodes, tets, queries):
    os.makedirs(d, exist_ok=True)
    np.array([n_nodes, len(tets), len(queries)], np.int64).tofile(os.path.join(d, "dims.bin"))
    np.ascontiguousarray(tets, np.int32).tofile(os.path.join(d, "tets.bin"))
    np.ascontiguousarray(queries, np.int32).reshape(-1, 2).tofile(os.path.join(d, "queries.bin"))
    out = subprocess.run([exe, d], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    rd = lambda name: np.fromfile(os.path.join(d, name), np.int32)  # noqa: E731
    return int(out.stdout), rd("colour.bin"), rd("rp.bin"), rd("ci.bin"), rd("found.bin")


def _adjacency(n_nodes, tets):
    r = np.repeat(tets, 4, axis=1).ravel()
    c = np.tile(tets, (1, 4)).ravel()
    A = sp.csr_matrix((np.ones(r.size), (r, c)), shape=(n_nodes, n_nodes)) + sp.identity(n_nodes, format="csr")
    A.sort_indices()
    return A


@pytest.mark.parametrize("case", ["cube", "tube", "star", "shuffled"])
def test_colouring_and_pattern(exe, tmp_path, case):
    rng = np.random.default_rng(3)
    if case == "cube":
        m = kuhn_cube(5)
        n, tets = m.n_nodes, m.tets
    elif case == "tube":
        m = artery_tube(n_theta=16, n_z=6, length=0.5, materials=artery_layers(1.0e3))
        n, tets = m.n_nodes, m.tets
    elif case == "star":
        n, tets = _star(150)
    else:   # the tube's elements in a random order with renumbered nodes
        m = artery_tube(n_theta=16, n_z=6, length=0.5, materials=artery_layers(1.0e3))
        perm = rng.permutation(m.n_nodes)
        n, tets = m.n_nodes, perm[m.tets][rng.permutation(m.n_elems)]
    tets = np.asarray(tets, np.int32)
    A = _adjacency(n, tets)
    # lookups: every stored block, and as many node pairs that share no element
    present = np.stack([np.repeat(np.arange(n), np.diff(A.indptr)), A.indices], axis=1)
    cand = rng.integers(0, n, size=(4 * len(present), 2))
    absent = cand[np.asarray(A[cand[:, 0], cand[:, 1]]).ravel() == 0][:len(present)]
    queries = np.concatenate([present, absent]).astype(np.int32)
    nc, colour, rp, ci, found = _run(exe, str(tmp_path / case), n, tets, queries)
    ref = O.greedy_colouring(tets, n)
    assert np.array_equal(colour, ref)
    assert nc == ref.max() + 1
    if case == "star":
        assert nc == 150
    # proper colouring: no two elements of one colour share a node
    for c in range(nc):
        nodes = tets[colour == c].ravel()
        assert np.unique(nodes).size == nodes.size
    assert np.array_equal(rp, A.indptr) and np.array_equal(ci, A.indices)
    assert np.array_equal(found[:len(present)], np.arange(len(present)))
    assert (found[len(present):] == -1).all()
