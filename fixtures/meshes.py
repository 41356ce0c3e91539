"""Structured tetrahedral meshes, boundary data and material tables.

The paper's Netgen meshes of a rabbit carotid (Sec. 6.1-6.2) are not
available, so seeded structured meshes stand in for them:

* ``kuhn_cube``: the unit cube cut into n^3 hexahedra, each split into six
  tetrahedra around its main diagonal (Kuhn / Freudenthal split).  The split
  is invariant under integer translations of the index lattice, so it is
  conforming and also conforming across a periodic wrap.
* ``artery_tube``: a thick-walled two-layer tube (media inside, adventitia
  outside) in (theta, r, z) index space with theta periodic, mapped to
  (r cos theta, r sin theta, z); the same Kuhn split.

Everything here is bookkeeping: coordinates, connectivity, orientation,
boundary masks, face lists, fibre direction fields and material tables.
None of the finite element arithmetic lives here.
"""
from __future__ import annotations

import dataclasses
import itertools
import math
from typing import List, Optional, Sequence

import numpy as np

# material model ids (shared meaning with the C-ABI header)
MODEL_MOONEY_RIVLIN = 0
MODEL_ARTERY = 1


@dataclasses.dataclass
class Material:
    """Parameters of one material (Sec. 2.3.1 / 2.3.2 of the paper)."""

    model: int
    c10: float
    c01: float = 0.0
    k1: float = 0.0
    k2: float = 1.0
    kappa: float = 1.0e3
    rho: float = 0.0

    def as_tuple(self):
        return (self.model, self.c10, self.c01, self.k1, self.k2, self.kappa, self.rho)


def mooney_rivlin(c10=0.5, c01=0.1, kappa=1.0e3, rho=0.0) -> List[Material]:
    return [Material(MODEL_MOONEY_RIVLIN, c10, c01, 0.0, 1.0, kappa, rho)]


def artery_layers(kappa_ratio=1.0e3, rho=0.0, c10=(3.0, 0.3), k1=(2.3, 0.56),
                  k2=(0.84, 0.71)) -> List[Material]:
    """Media (id 0) and adventitia (id 1).  One bulk modulus for both layers,
    kappa = kappa_ratio * c10 of the media."""
    kappa = kappa_ratio * c10[0]
    return [Material(MODEL_ARTERY, c10[i], 0.0, k1[i], k2[i], kappa, rho) for i in range(2)]


@dataclasses.dataclass
class Mesh:
    X: np.ndarray            # float64 [n, 3] reference coordinates
    tets: np.ndarray         # int32 [e, 4], positively oriented
    mat_id: np.ndarray       # int32 [e]
    fibre: np.ndarray        # float64 [e, 2, 3] unit fibre directions a01, a02
    dir_mask: np.ndarray     # uint8 [n, 4] 1 = constrained component (ux, uy, uz, p)
    neu_faces: np.ndarray    # int32 [f, 3], ordered so the right-hand normal points out of the body
    materials: List[Material]
    name: str = ""
    # optional per-node prescribed displacement direction for ramped Dirichlet loads
    dir_target: Optional[np.ndarray] = None   # float64 [n, 4]: value at load factor 1
    # batching: segment id per node / element / face (None for a single mesh)
    seg_node: Optional[np.ndarray] = None
    seg_elem: Optional[np.ndarray] = None
    seg_face: Optional[np.ndarray] = None
    face_pressure: Optional[np.ndarray] = None   # per-face dead pressure at load factor 1
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def n_nodes(self) -> int:
        return int(self.X.shape[0])

    @property
    def n_elems(self) -> int:
        return int(self.tets.shape[0])

    def dir_values(self, load_factor: float) -> np.ndarray:
        """Prescribed values [n, 4] at a load factor (zero where unconstrained)."""
        if self.dir_target is None:
            return np.zeros((self.n_nodes, 4))
        return self.dir_target * float(load_factor)


_PERMS = list(itertools.permutations(range(3)))


def _kuhn_hex_tets(corner):
    """The six tetrahedra of one lattice cell as lists of 3-D lattice offsets."""
    out = []
    for perm in _PERMS:
        v = [0, 0, 0]
        verts = [tuple(v)]
        for ax in perm:
            v[ax] += 1
            verts.append(tuple(v))
        out.append([tuple(corner[d] + o[d] for d in range(3)) for o in verts])
    return out


def _orient(X, tets):
    """Swap the last two vertices of tetrahedra with negative signed volume."""
    x0 = X[tets[:, 0]]
    d = np.einsum("ij,ij->i", np.cross(X[tets[:, 1]] - x0, X[tets[:, 2]] - x0), X[tets[:, 3]] - x0)
    neg = d < 0
    t = tets.copy()
    t[neg, 2], t[neg, 3] = tets[neg, 3], tets[neg, 2]
    return t


def _boundary_faces(X, tets):
    """Faces used by exactly one tetrahedron, oriented with outward normal."""
    loc = [(1, 2, 3, 0), (0, 3, 2, 1), (0, 1, 3, 2), (0, 2, 1, 3)]
    faces = []
    for a, b, c, d in loc:
        faces.append(np.stack([tets[:, a], tets[:, b], tets[:, c], tets[:, d]], axis=1))
    F = np.concatenate(faces, axis=0)
    key = np.sort(F[:, :3], axis=1)
    _, inv, cnt = np.unique(key, axis=0, return_inverse=True, return_counts=True)
    bnd = F[cnt[inv.ravel()] == 1]
    xa = X[bnd[:, 0]]
    n = np.cross(X[bnd[:, 1]] - xa, X[bnd[:, 2]] - xa)
    inward = np.einsum("ij,ij->i", n, X[bnd[:, 3]] - xa) > 0
    out = bnd[:, :3].copy()
    out[inward, 1], out[inward, 2] = bnd[inward, 2], bnd[inward, 1]
    return out.astype(np.int32)


def kuhn_cube(n: int = 8, materials: Optional[Sequence[Material]] = None, size: float = 1.0) -> Mesh:
    """Unit cube, n^3 hexahedra x 6 tetrahedra; node id = i + (n+1)(j + (n+1)k)."""
    m = n + 1
    g = np.arange(m) * (size / n)
    k, j, i = np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij")
    X = np.stack([g[i.ravel()], g[j.ravel()], g[k.ravel()]], axis=1).astype(np.float64)

    def nid(p):
        return p[0] + m * (p[1] + m * p[2])

    tets = []
    for kk in range(n):
        for jj in range(n):
            for ii in range(n):
                for t in _kuhn_hex_tets((ii, jj, kk)):
                    tets.append([nid(p) for p in t])
    tets = _orient(X, np.asarray(tets, dtype=np.int64)).astype(np.int32)
    mats = list(materials) if materials is not None else mooney_rivlin()
    return Mesh(X=X, tets=tets, mat_id=np.zeros(len(tets), np.int32),
                fibre=np.zeros((len(tets), 2, 3)), dir_mask=np.zeros((m ** 3, 4), np.uint8),
                neu_faces=np.zeros((0, 3), np.int32), materials=mats, name=f"cube{n}",
                meta={"n": n, "size": size})


def cube_uniaxial_bc(mesh: Mesh, stretch: float = 0.2, variant: str = "clamped") -> Mesh:
    """Bottom face clamped (or on rollers), top face moved by ``stretch`` in z.

    ``clamped``: u = 0 on z = 0, u_z = stretch on z = size.
    ``roller``:  u_x = 0 on x = 0, u_y = 0 on y = 0, u_z = 0 on z = 0,
                 u_z = stretch on z = size (homogeneous uniaxial state).
    """
    X = mesh.X
    size = mesh.meta.get("size", 1.0)
    tol = 1e-12 * size
    mask = np.zeros((mesh.n_nodes, 4), np.uint8)
    target = np.zeros((mesh.n_nodes, 4))
    bot = np.abs(X[:, 2]) < tol
    top = np.abs(X[:, 2] - size) < tol
    if variant == "clamped":
        mask[bot, 0:3] = 1
    elif variant == "roller":
        mask[np.abs(X[:, 0]) < tol, 0] = 1
        mask[np.abs(X[:, 1]) < tol, 1] = 1
        mask[bot, 2] = 1
    else:
        raise ValueError(variant)
    mask[top, 2] = 1
    target[top, 2] = stretch * size
    out = dataclasses.replace(mesh, dir_mask=mask, dir_target=target)
    out.meta = dict(mesh.meta, bc=variant, stretch=stretch)
    return out


def _tube_radii(r_in, t_media, t_adv, n_media, n_adv):
    rm = r_in + np.linspace(0.0, t_media, n_media + 1)
    ra = r_in + t_media + np.linspace(0.0, t_adv, n_adv + 1)[1:]
    return np.concatenate([rm, ra])


def artery_tube(n_theta=64, n_media=4, n_adv=4, n_z=128, r_in=1.0, t_media=0.13, t_adv=0.10,
                length=8.0, alpha_deg=(29.0, 62.0), materials=None) -> Mesh:
    """Two-layer thick-walled tube; theta periodic.

    node id = j + n_theta * (i + (n_r + 1) * k) for theta index j, radial index
    i, axial index k.  Element material id: 0 = media (inner n_media radial
    layers), 1 = adventitia.  Fibre directions per element use the local
    cylindrical frame at the element centroid: a01 = cos(a) e_theta + sin(a) e_z,
    a02 = cos(a) e_theta - sin(a) e_z with the layer's angle a.
    """
    n_r = n_media + n_adv
    radii = _tube_radii(r_in, t_media, t_adv, n_media, n_adv)
    theta = 2.0 * math.pi * np.arange(n_theta) / n_theta
    z = np.linspace(0.0, length, n_z + 1)
    K, I, Jt = np.meshgrid(np.arange(n_z + 1), np.arange(n_r + 1), np.arange(n_theta), indexing="ij")
    r = radii[I.ravel()]
    th = theta[Jt.ravel()]
    X = np.stack([r * np.cos(th), r * np.sin(th), z[K.ravel()]], axis=1)

    cells = []
    for perm in _PERMS:
        v = [0, 0, 0]
        verts = [tuple(v)]
        for ax in perm:
            v[ax] += 1
            verts.append(tuple(v))
        cells.append(verts)
    cells = np.asarray(cells)  # [6, 4, 3] offsets in (j, i, k)

    kk, ii, jj = np.meshgrid(np.arange(n_z), np.arange(n_r), np.arange(n_theta), indexing="ij")
    base = np.stack([jj.ravel(), ii.ravel(), kk.ravel()], axis=1)  # hex-major order [h, 3]
    P = base[:, None, None, :] + cells[None, :, :, :]               # [h, 6, 4, 3]
    jn = P[..., 0] % n_theta
    tets = (jn + n_theta * (P[..., 1] + (n_r + 1) * P[..., 2])).reshape(-1, 4)
    tets = _orient(X, tets.astype(np.int64)).astype(np.int32)
    layer = np.repeat(ii.ravel(), 6)
    mat_id = (layer >= n_media).astype(np.int32)

    xc = X[tets].mean(axis=1)
    thc = np.arctan2(xc[:, 1], xc[:, 0])
    e_t = np.stack([-np.sin(thc), np.cos(thc), np.zeros_like(thc)], axis=1)
    e_z = np.tile(np.array([0.0, 0.0, 1.0]), (len(tets), 1))
    alpha = np.deg2rad(np.asarray(alpha_deg, dtype=np.float64))[mat_id]
    ca, sa = np.cos(alpha)[:, None], np.sin(alpha)[:, None]
    fibre = np.stack([ca * e_t + sa * e_z, ca * e_t - sa * e_z], axis=1)

    faces = _boundary_faces(X, tets)
    rn = np.hypot(X[:, 0], X[:, 1])
    inner = np.all(np.abs(rn[faces] - r_in) < 1e-9, axis=1)
    mats = list(materials) if materials is not None else artery_layers()
    mesh = Mesh(X=X, tets=tets, mat_id=mat_id, fibre=fibre,
                dir_mask=np.zeros((X.shape[0], 4), np.uint8), neu_faces=faces[inner],
                materials=mats, name=f"tube{n_theta}x{n_r}x{n_z}",
                meta={"n_theta": n_theta, "n_r": n_r, "n_z": n_z, "length": length,
                      "r_in": r_in, "alpha_deg": tuple(alpha_deg)})
    return tube_end_bc(mesh)


def tube_end_bc(mesh: Mesh, clamped: bool = False) -> Mesh:
    """Ends fixed axially: u_z = 0 on z = 0 and z = L; at the end nodes,
    u_x = 0 where x = 0 and u_y = 0 where y = 0 (removes rigid modes).
    ``clamped`` fixes all three displacement components on both ends."""
    X = mesh.X
    L = mesh.meta["length"]
    zmin = float(X[:, 2].min())
    ends = (np.abs(X[:, 2] - zmin) < 1e-12) | (np.abs(X[:, 2] - (zmin + L)) < 1e-12)
    scale = max(1.0, float(np.abs(X).max()))
    mask = np.zeros((mesh.n_nodes, 4), np.uint8)
    mask[ends, 2] = 1
    if clamped:
        mask[ends, 0:3] = 1
    else:
        if mesh.seg_node is None:
            ctr = np.zeros((mesh.n_nodes, 2))
        else:
            ctr = mesh.meta["seg_center"][mesh.seg_node]
        mask[ends & (np.abs(X[:, 0] - ctr[:, 0]) < 1e-12 * scale), 0] = 1
        mask[ends & (np.abs(X[:, 1] - ctr[:, 1]) < 1e-12 * scale), 1] = 1
    out = dataclasses.replace(mesh, dir_mask=mask, dir_target=np.zeros((mesh.n_nodes, 4)))
    return out


def batched_tubes(n_seg=256, seed=4, ne_range=(5.0e3, 2.0e5), n_r=8, dz=8.0 / 128,
                  spacing=4.0) -> Mesh:
    """Many independent artery segments of uneven size in one union mesh.

    Per segment (seeded ``numpy.random.default_rng``): n_e ~ logU[ne_range];
    n_theta = 32 if n_e < 5e4 else 64; n_z = max(2, round(n_e / (6 n_r n_theta)));
    fibre angle a ~ U[20, 70] deg in both layers (+-a); kappa/c10_media ~
    logU[1e2, 1e5]; internal pressure P ~ U[0.5, 2.0] (stored per face).
    Segments are placed side by side in x so that they never touch.
    """
    rng = np.random.default_rng(seed)
    X_all, T_all, M_all, F_all, D_all, N_all = [], [], [], [], [], []
    segn, sege, segf, fp = [], [], [], []
    mats: List[Material] = []
    centers = []
    seg_info = []
    off_n = 0
    for s in range(n_seg):
        ne = math.exp(rng.uniform(math.log(ne_range[0]), math.log(ne_range[1])))
        n_theta = 32 if ne < 5.0e4 else 64
        n_z = max(2, int(round(ne / (6 * n_r * n_theta))))
        alpha = rng.uniform(20.0, 70.0)
        kratio = math.exp(rng.uniform(math.log(1.0e2), math.log(1.0e5)))
        pres = rng.uniform(0.5, 2.0)
        t = artery_tube(n_theta=n_theta, n_media=n_r // 2, n_adv=n_r - n_r // 2, n_z=n_z,
                        length=n_z * dz, alpha_deg=(alpha, alpha),
                        materials=artery_layers(kratio))
        cx = spacing * s
        X = t.X.copy()
        X[:, 0] += cx
        centers.append((cx, 0.0))
        X_all.append(X)
        T_all.append(t.tets + off_n)
        M_all.append(t.mat_id + 2 * s)
        F_all.append(t.fibre)
        D_all.append(t.dir_mask)
        N_all.append(t.neu_faces + off_n)
        segn.append(np.full(t.n_nodes, s, np.int32))
        sege.append(np.full(t.n_elems, s, np.int32))
        segf.append(np.full(len(t.neu_faces), s, np.int32))
        fp.append(np.full(len(t.neu_faces), pres))
        mats.extend(t.materials)
        seg_info.append({"n_elems": t.n_elems, "n_nodes": t.n_nodes, "n_theta": n_theta,
                         "n_z": n_z, "alpha_deg": alpha, "kappa_ratio": kratio, "pressure": pres})
        off_n += t.n_nodes
    mesh = Mesh(X=np.concatenate(X_all), tets=np.concatenate(T_all).astype(np.int32),
                mat_id=np.concatenate(M_all).astype(np.int32), fibre=np.concatenate(F_all),
                dir_mask=np.concatenate(D_all), neu_faces=np.concatenate(N_all).astype(np.int32),
                materials=mats, name=f"batch{n_seg}", seg_node=np.concatenate(segn),
                seg_elem=np.concatenate(sege), seg_face=np.concatenate(segf),
                face_pressure=np.concatenate(fp), dir_target=None,
                meta={"segments": seg_info, "seg_center": np.asarray(centers)})
    return mesh


def batched_segment(index, n_seg=256, seed=4, ne_range=(5.0e3, 2.0e5), n_r=8, dz=8.0 / 128):
    """Segment ``index`` of ``batched_tubes`` (same arguments) as a mesh of its
    own, in its own frame, with its per-face pressure; also returns the offset
    of its first node in the union mesh.  Replays the generator's seeded draws
    up to that segment without building the others."""
    rng = np.random.default_rng(seed)
    off_n = 0
    for s in range(index + 1):
        ne = math.exp(rng.uniform(math.log(ne_range[0]), math.log(ne_range[1])))
        n_theta = 32 if ne < 5.0e4 else 64
        n_z = max(2, int(round(ne / (6 * n_r * n_theta))))
        alpha = rng.uniform(20.0, 70.0)
        kratio = math.exp(rng.uniform(math.log(1.0e2), math.log(1.0e5)))
        pres = rng.uniform(0.5, 2.0)
        if s < index:
            off_n += n_theta * (n_r + 1) * (n_z + 1)
    t = artery_tube(n_theta=n_theta, n_media=n_r // 2, n_adv=n_r - n_r // 2, n_z=n_z, length=n_z * dz,
                    alpha_deg=(alpha, alpha), materials=artery_layers(kratio))
    t = dataclasses.replace(t, face_pressure=np.full(len(t.neu_faces), pres))
    t.meta = dict(t.meta, kappa_ratio=kratio, pressure=pres)
    return t, off_n


def tube_subset(mesh: Mesh, n_elems: int) -> Mesh:
    """The first ``n_elems`` elements of a mesh (axial slab order) re-indexed as
    a mesh of its own; used to bound CPU baselines on large meshes."""
    tets = mesh.tets[:n_elems]
    used = np.unique(tets)
    remap = -np.ones(mesh.n_nodes, np.int64)
    remap[used] = np.arange(len(used))
    return Mesh(X=mesh.X[used], tets=remap[tets].astype(np.int32), mat_id=mesh.mat_id[:n_elems],
                fibre=mesh.fibre[:n_elems], dir_mask=mesh.dir_mask[used],
                neu_faces=np.zeros((0, 3), np.int32), materials=mesh.materials,
                name=mesh.name + f"[:{n_elems}]", meta=dict(mesh.meta))
