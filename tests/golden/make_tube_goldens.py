"""Writes the stored oracle solutions used by the full-size parity tests.

Calls only ``oracle/`` (and the seeded mesh generators of ``fixtures/``):
a quarter-length section of the 393k-element workload tube -- the same
cross-section and element shape, 64 x 8 x 32 hexahedra x 6 tetrahedra
(98,304 elements, 18,720 nodes, length 2), ends fixed axially -- under the
internal dead pressure P = 0.16 (the first of the ten load steps 0 -> 1.6),
bulk modulus kappa = ratio x c10 of the media for ratio 1e3 and 1e5; Newton
from the reference state with the oracle's sparse direct solve, to
||R|| <= 1e-12 ||R_0||.  (The oracle's direct solve grows roughly with the
square of the length of the tube: the full 8-long tube does not finish in
hours.)  Output: ``tube98k_k<ratio>_p016.npz`` with the converged state
[n, 4] (float64) and the Newton residual history.

Run from the repository root:  python tests/golden/make_tube_goldens.py
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from fixtures import artery_layers, artery_tube  # noqa: E402
from oracle import solid as O  # noqa: E402


def golden_path(ratio):
    return os.path.join(HERE, f"tube98k_k{ratio:.0e}_p016.npz".replace("+0", ""))


def golden_mesh(ratio):
    return artery_tube(n_theta=64, n_media=4, n_adv=4, n_z=32, length=2.0, materials=artery_layers(ratio))


def make(ratio, pressure=0.16):
    mesh = golden_mesh(ratio)
    P = O.Problem(mesh)
    hist = []
    t0 = time.time()
    state, its = P.newton(np.zeros((mesh.n_nodes, 4)), fext=P.external_force(pressure), rtol=1e-12, record=hist)
    np.savez_compressed(golden_path(ratio), state=state, residual_history=np.asarray(hist), pressure=pressure,
                        kappa_ratio=ratio, newton_its=its)
    print(f"ratio {ratio:g}: {its} Newton its, {time.time() - t0:.0f} s, history {hist}", flush=True)


if __name__ == "__main__":
    ratios = [float(a) for a in sys.argv[1:]] or [1.0e3, 1.0e5]
    for r in ratios:
        make(r)
