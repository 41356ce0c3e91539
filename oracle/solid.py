"""FP64 oracle of the residual-stabilised P1/P1 u-p solid (test infrastructure).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline / reference leg of ``bench.py``; never by the product path.

What it computes, in the paper's order and notation:

* kinematics F = I + grad d, J = det F, C = F^T F, I1, I2, I3 (Sec. 2.3);
* the isochoric stress S' of the modified Mooney-Rivlin model (Eq. mmreng,
  mmrpkt, mmrpktmix) and of the two-layer artery (Eq. areng, arinv46, arpkt,
  arpktmix), with p = -kappa (J - 1) carried as an unknown;
* the element residuals R_s^1, R_s^2 of the time semi-discrete weak form
  (Sec. 4.2.3) plus the PSPG term W_s of Eq. stelas with
  tau = h_T^2 / (4 mu^l) (Sec. 4.3.2), on P1 tetrahedra;
* the consistent Newton tangent K = [A B1^T; B2 -C] (Eq. linsys, globsys) as
  the complex-step derivative of the element residual: exact to rounding,
  so it is the plain definition of dR/dv;
* assembly, Dirichlet rows/columns, a direct sparse solve and Newton's method
  (Sec. 4.4).

Readings where the paper is silent or garbled (each one is also listed in the
design notes): a02 = (0, cos a, -sin a) in the local (e_r, e_theta, e_z) frame;
S_aniso derived from Psi gives the factor 2 k1 (``fibre_factor`` = 2; the
printed Eq. arpkt has k1, ``fibre_factor`` = 1); a fibre family contributes
only while J_i - 1 > 0; mu^l as printed enters tau only; h_T is the longest
edge; centroid quadrature (exact for P1 except the mass products, which use
the exact P1 mass matrix); dead pressure load on the reference surface.

Every array here is float64 (or complex128 inside the complex step).
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

MODEL_MOONEY_RIVLIN = 0
MODEL_ARTERY = 1


@dataclasses.dataclass
class Options:
    use_pspg: bool = True
    fibre_factor: float = 2.0     # 2: S = 2 dPsi/dC;  1: as printed in Eq. arpkt
    inertia_coef: float = 0.0     # 1 / (beta dt^2) for Newmark-beta; 0 = quasi-static


# ----------------------------------------------------------------- geometry
def p1_geometry(X, tets):
    """Gradients of the P1 hat functions (Sec. 4.3.2), volume and h_T.

    Returns g [e, 4, 3] with g[:, a] = grad N_a, V [e], h [e] (longest edge).
    The gradients satisfy grad N_a . (x_b - x_0) = delta_ab for a, b = 1..3
    and sum_a grad N_a = 0.
    """
    x = X[tets]
    D = x[:, 1:, :] - x[:, :1, :]           # rows d_b = x_b - x_0
    G = np.linalg.inv(np.transpose(D, (0, 2, 1)))   # G D^T = I  ->  G = (D^T)^-1
    g = np.concatenate([-G.sum(axis=1, keepdims=True), G], axis=1)
    V = np.linalg.det(D) / 6.0
    edges = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]
    h = np.max(np.stack([np.linalg.norm(x[:, a] - x[:, b], axis=1) for a, b in edges]), axis=0)
    return g, V, h


# ----------------------------------------------------------------- tensors
def _det3(A):
    return (A[..., 0, 0] * (A[..., 1, 1] * A[..., 2, 2] - A[..., 1, 2] * A[..., 2, 1])
            - A[..., 0, 1] * (A[..., 1, 0] * A[..., 2, 2] - A[..., 1, 2] * A[..., 2, 0])
            + A[..., 0, 2] * (A[..., 1, 0] * A[..., 2, 1] - A[..., 1, 1] * A[..., 2, 0]))


def _adj3(A):
    """Adjugate (transpose of the cofactor matrix): A adj(A) = det(A) I."""
    c = np.empty_like(A)
    c[..., 0, 0] = A[..., 1, 1] * A[..., 2, 2] - A[..., 1, 2] * A[..., 2, 1]
    c[..., 0, 1] = A[..., 0, 2] * A[..., 2, 1] - A[..., 0, 1] * A[..., 2, 2]
    c[..., 0, 2] = A[..., 0, 1] * A[..., 1, 2] - A[..., 0, 2] * A[..., 1, 1]
    c[..., 1, 0] = A[..., 1, 2] * A[..., 2, 0] - A[..., 1, 0] * A[..., 2, 2]
    c[..., 1, 1] = A[..., 0, 0] * A[..., 2, 2] - A[..., 0, 2] * A[..., 2, 0]
    c[..., 1, 2] = A[..., 0, 2] * A[..., 1, 0] - A[..., 0, 0] * A[..., 1, 2]
    c[..., 2, 0] = A[..., 1, 0] * A[..., 2, 1] - A[..., 1, 1] * A[..., 2, 0]
    c[..., 2, 1] = A[..., 0, 1] * A[..., 2, 0] - A[..., 0, 0] * A[..., 2, 1]
    c[..., 2, 2] = A[..., 0, 0] * A[..., 1, 1] - A[..., 0, 1] * A[..., 1, 0]
    return c


def _tr(A):
    return A[..., 0, 0] + A[..., 1, 1] + A[..., 2, 2]


def _mm(A, B):
    return np.einsum("...ij,...jk->...ik", A, B)


def _T(A):
    return np.swapaxes(A, -1, -2)


def kinematics(H):
    """F = I + H, J - 1 (expanded so that it keeps its digits when J is near 1),
    C = F^T F, the invariants I1, I2, I3 = J^2, C^-1 and F^-1 (Sec. 2.3)."""
    eye = np.eye(3)
    F = eye + H
    trH = _tr(H)
    Jm1 = trH + 0.5 * (trH * trH - _tr(_mm(H, H))) + _det3(H)   # det(I + H) - 1
    J = 1.0 + Jm1
    E = 0.5 * (H + _T(H) + _mm(_T(H), H))                       # C = I + 2E
    C = eye + 2.0 * E
    I1 = _tr(C)
    I2 = 0.5 * (I1 * I1 - np.einsum("...ij,...ij->...", C, C))
    I3 = J * J
    Finv = _adj3(F) / J[..., None, None]
    Cinv = _mm(Finv, _T(Finv))
    return dict(F=F, J=J, Jm1=Jm1, E=E, C=C, I1=I1, I2=I2, I3=I3, Finv=Finv, Cinv=Cinv)


def isochoric_stress(kin, c10, c01, k1, k2, model, fibre, fibre_factor=2.0, active=None):
    """S' of Eq. mmrpkt / arpkt (the pressure part is carried separately).

    dJ1/dC = I3^{-1/3} (I - I1/3 C^-1), dJ2/dC = I3^{-2/3} (I1 I - C - 2/3 I2 C^-1),
    dJi/dC = I3^{-1/3} (A_i - 1/3 (A_i : C) C^-1), A_i = a0i (x) a0i (Eq. arinv46).
    I3^{-1/3} = J^{-2/3} is formed as exp(-2/3 log1p(J - 1)).
    ``active`` [2, e] (optional) fixes the fibre switch J_i - 1 > 0 from outside
    (the complex step decides it on the unperturbed real state).
    """
    eye = np.eye(3)
    J23 = np.exp(-(2.0 / 3.0) * np.log1p(kin["Jm1"]))            # I3^{-1/3}
    J23m1 = np.expm1(-(2.0 / 3.0) * np.log1p(kin["Jm1"]))         # I3^{-1/3} - 1
    I1, I2, C, Cinv = kin["I1"], kin["I2"], kin["C"], kin["Cinv"]
    dJ1 = J23[..., None, None] * (eye - (I1 / 3.0)[..., None, None] * Cinv)
    dJ2 = (J23 * J23)[..., None, None] * (I1[..., None, None] * eye - C
                                          - (2.0 / 3.0) * I2[..., None, None] * Cinv)
    S = c10[..., None, None] * dJ1 + c01[..., None, None] * dJ2
    is_artery = model == MODEL_ARTERY
    E = kin["E"]
    for i in range(2):
        a = fibre[:, i, :]
        A = np.einsum("ei,ej->eij", a, a)
        I4 = np.einsum("eij,eij->e", A, C)                         # A_i : C
        Jim1 = J23m1 + J23 * 2.0 * np.einsum("ei,eij,ej->e", a, E, a)   # J_i - 1
        dJi = J23[..., None, None] * (A - (I4 / 3.0)[..., None, None] * Cinv)
        act = (np.real(Jim1) > 0.0) if active is None else active[i]
        act = is_artery & act                                      # fibres act in extension
        coef = fibre_factor * k1 * np.exp(k2 * Jim1 * Jim1) * Jim1
        S = S + np.where(act, coef, 0.0)[..., None, None] * dJi
    return S


def shear_modulus_l(model, c10, c01, k1, k2):
    """mu^l of Sec. 4.3.2: 2 (c10 + c01) (Mooney-Rivlin), 2 (c10 + k1 / (2 k2)) (artery)."""
    return np.where(model == MODEL_ARTERY, 2.0 * (c10 + k1 / (2.0 * k2)), 2.0 * (c10 + c01))


# ----------------------------------------------------------------- element residual
def fibre_activity(ve, g, fibre):
    """[2, e] booleans J_i - 1 > 0 of the two fibre families (real state)."""
    H = np.einsum("eai,eaj->eij", ve[:, :, 0:3], g)
    kin = kinematics(H)
    J23 = np.exp(-(2.0 / 3.0) * np.log1p(kin["Jm1"]))
    J23m1 = np.expm1(-(2.0 / 3.0) * np.log1p(kin["Jm1"]))
    out = []
    for i in range(2):
        a = fibre[:, i, :]
        out.append(J23m1 + J23 * 2.0 * np.einsum("ei,eij,ej->e", a, kin["E"], a) > 0.0)
    return np.stack(out)


def element_residual(ve, g, V, h, mp, fibre, opts: Options, hist_e=None, active=None):
    """Element residuals of Sec. 4.2.3 + Eq. stelas for P1/P1 tetrahedra.

    ve    : [e, 4, 4] nodal (d_x, d_y, d_z, p) of each element
    g, V, h : P1 geometry from ``p1_geometry``
    mp    : dict of per-element material arrays (model, c10, c01, k1, k2, kappa, rho)
    fibre : [e, 2, 3] fibre directions a01, a02
    hist_e: [e, 4, 3] nodal Newmark history h_s (r_s = rho h_s), or None
    Returns [e, 4, 4]: (R^1_a in rows 0..2, R^2_a in row 3) for each node a.

    R^1_a = V [F S' g_a - pbar J F^-T g_a] + rho c0 sum_b M_ab d_b - rho sum_b M_ab h_b
    R^2_a = -V (J - 1)/4 - (1/kappa) sum_b M_ab p_b
            + tau V (rho hbar - rho c0 dbar - J F^-T grad p) . (F^-T g_a)
    with M_ab = V (1 + delta_ab)/20, c0 = 1/(beta dt^2), grad p = sum_b p_b g_b.
    """
    d = ve[:, :, 0:3]
    p = ve[:, :, 3]
    H = np.einsum("eai,eaj->eij", d, g)                   # grad d = sum_a d_a (x) g_a
    kin = kinematics(H)
    F, J, Finv = kin["F"], kin["J"], kin["Finv"]
    S = isochoric_stress(kin, mp["c10"], mp["c01"], mp["k1"], mp["k2"], mp["model"], fibre,
                         opts.fibre_factor, active)
    pbar = p.mean(axis=1)
    gsp = np.einsum("eji,eaj->eai", Finv, g)               # F^-T g_a
    FS = _mm(F, S)
    R1 = V[:, None, None] * (np.einsum("eij,eaj->eai", FS, g)
                             - (pbar * J)[:, None, None] * gsp)
    rho = mp["rho"]
    c0 = opts.inertia_coef
    if hist_e is None:
        hist_e = np.zeros_like(d, dtype=np.float64)
    dsum = d.sum(axis=1, keepdims=True)
    hsum = hist_e.sum(axis=1, keepdims=True)
    Md = (V / 20.0)[:, None, None] * (d + dsum)           # sum_b M_ab d_b
    Mh = (V / 20.0)[:, None, None] * (hist_e + hsum)
    R1 = R1 + (rho * c0)[:, None, None] * Md - rho[:, None, None] * Mh

    Mp = (V / 20.0)[:, None] * (p + p.sum(axis=1, keepdims=True))
    R2 = -(V * kin["Jm1"] / 4.0)[:, None] - Mp / mp["kappa"][:, None]
    if opts.use_pspg:
        tau = h * h / (4.0 * shear_modulus_l(mp["model"], mp["c10"], mp["c01"], mp["k1"], mp["k2"]))
        gradp = np.einsum("eb,ebj->ej", p, g)
        w = (rho[:, None] * hist_e.mean(axis=1) - (rho * c0)[:, None] * d.mean(axis=1)
             - J[:, None] * np.einsum("eji,ej->ei", Finv, gradp))
        R2 = R2 + (tau * V)[:, None] * np.einsum("ei,eai->ea", w, gsp)
    return np.concatenate([R1, R2[:, :, None]], axis=2)


def element_tangent(ve, g, V, h, mp, fibre, opts: Options, hist_e=None, step=1e-30):
    """16 x 16 element Jacobian dR_e/dv_e by the complex step (Eq. linsys):
    column (b, c) = Im R_e(v_e + i s e_(b,c)) / s.  No subtraction occurs, so
    the result is the derivative to rounding.  Row/column index = 4 a + comp."""
    ne = ve.shape[0]
    K = np.empty((ne, 16, 16))
    active = fibre_activity(ve, g, fibre)
    for col in range(16):
        b, c = divmod(col, 4)
        z = ve.astype(np.complex128)
        z[:, b, c] += 1j * step
        R = element_residual(z, g, V, h, mp, fibre, opts, hist_e, active)
        K[:, :, col] = R.imag.reshape(ne, 16) / step
    return K


def element_tangent_fd(ve, g, V, h, mp, fibre, opts: Options, hist_e=None, rel=1e-6):
    """Central finite-difference Jacobian (real arithmetic only)."""
    ne = ve.shape[0]
    K = np.empty((ne, 16, 16))
    scale = np.maximum(np.abs(ve).max(axis=(1, 2)), 1e-3)
    for col in range(16):
        b, c = divmod(col, 4)
        s = rel * scale
        vp = ve.copy(); vp[:, b, c] += s
        vm = ve.copy(); vm[:, b, c] -= s
        Rp = element_residual(vp, g, V, h, mp, fibre, opts, hist_e)
        Rm = element_residual(vm, g, V, h, mp, fibre, opts, hist_e)
        K[:, :, col] = ((Rp - Rm).reshape(ne, 16)) / (2.0 * s)[:, None]
    return K


# ----------------------------------------------------------------- problem
class Problem:
    """Mesh + materials + options; global residual, tangent and Newton."""

    def __init__(self, mesh, opts: Optional[Options] = None):
        self.mesh = mesh
        self.opts = opts or Options()
        self.g, self.V, self.h = p1_geometry(mesh.X, mesh.tets)
        mats = mesh.materials
        mid = mesh.mat_id
        tab = np.array([m.as_tuple() for m in mats], dtype=np.float64)
        self.mp = {
            "model": tab[mid, 0].astype(np.int64),
            "c10": tab[mid, 1], "c01": tab[mid, 2], "k1": tab[mid, 3], "k2": tab[mid, 4],
            "kappa": tab[mid, 5], "rho": tab[mid, 6],
        }
        self.n = mesh.n_nodes
        self.free = (mesh.dir_mask == 0).astype(np.float64)      # [n, 4]

    # -- per element subsets (for sampled parity at large sizes)
    def _sub(self, idx):
        mp = {k: v[idx] for k, v in self.mp.items()}
        return self.g[idx], self.V[idx], self.h[idx], mp, self.mesh.fibre[idx]

    def element_residuals(self, state, idx=None, hist=None):
        idx = np.arange(self.mesh.n_elems) if idx is None else np.asarray(idx)
        g, V, h, mp, fib = self._sub(idx)
        tets = self.mesh.tets[idx]
        he = None if hist is None else hist[tets]
        return element_residual(state[tets], g, V, h, mp, fib, self.opts, he)

    def element_tangents(self, state, idx=None, hist=None):
        idx = np.arange(self.mesh.n_elems) if idx is None else np.asarray(idx)
        g, V, h, mp, fib = self._sub(idx)
        tets = self.mesh.tets[idx]
        he = None if hist is None else hist[tets]
        return element_tangent(state[tets], g, V, h, mp, fib, self.opts, he)

    def external_force(self, pressure=1.0, node_pressure=None, face_pressure=None):
        """Dead pressure load on the reference surface (<g_n, v> of Sec. 4.2.3):
        traction t = -P n on each triangle, integrated exactly against the P1
        hat functions: f_a = -(x1-x0) x (x2-x0) * sum_b P_b (1 + delta_ab) / 24."""
        f = np.zeros((self.n, 3))
        faces = self.mesh.neu_faces
        if len(faces) == 0:
            return f
        X = self.mesh.X
        nrm2 = np.cross(X[faces[:, 1]] - X[faces[:, 0]], X[faces[:, 2]] - X[faces[:, 0]])
        if node_pressure is not None:
            Pn = node_pressure[faces] * pressure
        elif face_pressure is not None:
            Pn = np.repeat((face_pressure * pressure)[:, None], 3, axis=1)
        else:
            Pn = np.full(faces.shape, float(pressure))
        for a in range(3):
            wa = (Pn.sum(axis=1) + Pn[:, a]) / 24.0
            np.add.at(f, faces[:, a], -nrm2 * wa[:, None])
        return f

    def residual(self, state, fext=None, hist=None):
        """Global residual [n, 4] with zero rows on constrained components."""
        Re = self.element_residuals(state, hist=hist)
        R = np.zeros((self.n, 4))
        np.add.at(R, self.mesh.tets, Re)
        if fext is not None:
            R[:, 0:3] -= fext
        return R * self.free

    def tangent(self, state, hist=None, dirichlet=True):
        """Global Jacobian (CSR, dof = 4 node + comp); constrained rows become
        identity rows and constrained columns are zeroed."""
        Ke = self.element_tangents(state, hist=hist)
        tets = self.mesh.tets
        dofs = (4 * tets[:, :, None] + np.arange(4)[None, None, :]).reshape(-1, 16)
        rows = np.repeat(dofs, 16, axis=1).ravel()
        cols = np.tile(dofs, (1, 16)).ravel()
        K = sp.coo_matrix((Ke.ravel(), (rows, cols)), shape=(4 * self.n, 4 * self.n)).tocsr()
        K.sum_duplicates()
        if dirichlet:
            fr = self.free.ravel()
            Df = sp.diags(fr)
            K = (Df @ K @ Df + sp.diags(1.0 - fr)).tocsr()
        return K

    def mass_matrix(self):
        """Consistent P1 mass matrix of one scalar field (CSR, n x n):
        M_ab = int N_a N_b dV = V (1 + delta_ab) / 20 on each tetrahedron."""
        tets = self.mesh.tets
        Me = (self.V / 20.0)[:, None, None] * (np.ones((4, 4)) + np.eye(4))[None]
        rows = np.repeat(tets, 4, axis=1).ravel()
        cols = np.tile(tets, (1, 4)).ravel()
        return sp.coo_matrix((Me.ravel(), (rows, cols)), shape=(self.n, self.n)).tocsr()

    def mass_norm(self, dv):
        """||dv||_M = sqrt(dv^T M dv), M = diag[M_1, M_2]: the L2 norm of the
        displacement and pressure increment of Sec. 4.4 (Eq. newstop); M_1 is
        the scalar mass matrix on each displacement component, M_2 on p."""
        M = self.mass_matrix()
        return float(np.sqrt(sum(dv[:, c] @ (M @ dv[:, c]) for c in range(4))))

    def apply_dirichlet(self, state, values):
        """Prescribed values go into the state at the start of a load step."""
        s = state.copy()
        m = self.mesh.dir_mask.astype(bool)
        s[m] = values[m]
        return s

    def newton(self, state, fext=None, hist=None, rtol=1e-10, max_it=30, record=None, r_ref=None):
        """Newton's method (Sec. 4.4) with an exact sparse direct linear solve.
        Stops when ||R(v_k)||_2 <= rtol ||R(v_0)||_2, or rtol * r_ref when a
        reference norm is given."""
        v = state.copy()
        r0 = r_ref
        for k in range(max_it + 1):
            R = self.residual(v, fext, hist)
            rn = float(np.linalg.norm(R))
            if record is not None:
                record.append(rn)
            if r0 is None:
                r0 = rn
            if rn <= rtol * r0 or rn == 0.0:
                return v, k
            if k == max_it:
                break
            K = self.tangent(v, hist)
            dv = spla.spsolve(K.tocsc(), -R.ravel())
            v = v + dv.reshape(self.n, 4)
        raise RuntimeError(f"oracle Newton did not converge: {record}")


def greedy_colouring(tets, n_nodes):
    """Greedy first-fit colouring of elements in element order: an element
    takes the smallest colour not used by an earlier element sharing a node."""
    used = [set() for _ in range(n_nodes)]
    col = np.empty(len(tets), np.int32)
    for e, t in enumerate(tets):
        taken = used[t[0]] | used[t[1]] | used[t[2]] | used[t[3]]
        c = 0
        while c in taken:
            c += 1
        col[e] = c
        for a in t:
            used[a].add(c)
    return col
