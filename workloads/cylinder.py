"""Unstructured P1 finite-element Helmholtz matrix on a jittered cylinder.

Stand-in for the paper's "Cylinder3D" matrices (Section 3.1), which come from
an FE discretisation of -lap(u) - k^2 u = g (Section 2) and are not
distributed with it.  The mesh is a structured cylindrical grid (nr rings,
ntheta sectors, nz layers; one axis node per z-level) whose hexahedra are
split into 6 tetrahedra by the Kuhn (Freudenthal) rule in index space, with
the innermost ring of wedges split into the 3 non-degenerate Kuhn tetrahedra.
Interior nodes are jittered uniformly by +-0.2 of the local spacing per
direction (dr, r*dtheta, dz).  The assembled operator is

    A = K - k^2 (1 + i*damping) M - i k B,

with K the P1 stiffness matrix, M the P1 mass matrix and B the boundary mass
matrix of the two end faces z = 0 and z = L (first-order impedance condition
du/dn - i k u = 0 there); the lateral surface is natural (Neumann).  A is
complex symmetric.  Rows are reordered by reverse Cuthill-McKee.
"""

import numpy as np
import scipy.sparse as sp
from scipy.sparse.csgraph import reverse_cuthill_mckee

from .csr import CSR

# Kuhn paths: each permutation of the three index directions (0=r, 1=theta,
# 2=z) gives one tetrahedron (0,0,0) -> +e_a -> +e_b -> +e_c = (1,1,1).
_PERMS = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]


def _node_ids(nr, nth, nz):
    per = 1 + nr * nth

    def vid(i, j, k):
        j = np.mod(j, nth)
        return np.where(i == 0, k * per, k * per + 1 + (i - 1) * nth + j)
    return per, vid


def cylinder_mesh(nr, ntheta, nz, radius=1.0, length=4.0, jitter=0.2, seed=None):
    """Nodes (N,3) Cartesian, tetrahedra (T,4) int64, end-face triangles (F,3)."""
    per, vid = _node_ids(nr, ntheta, nz)
    nnode = per * (nz + 1)
    dr, dth, dz = radius / nr, 2.0 * np.pi / ntheta, length / nz

    # cylindrical coordinates of every node
    rr = np.zeros(nnode)
    tt = np.zeros(nnode)
    zz = np.zeros(nnode)
    k_of = np.arange(nnode) // per
    loc = np.arange(nnode) % per
    ring = np.where(loc == 0, 0, (loc - 1) // ntheta + 1)
    sect = np.where(loc == 0, 0, (loc - 1) % ntheta)
    rr[:] = ring * dr
    tt[:] = sect * dth
    zz[:] = k_of * dz
    if jitter and seed is not None:
        rng = np.random.default_rng(seed)
        u = rng.uniform(-jitter, jitter, size=(nnode, 3))
        interior = (ring > 0) & (ring < nr) & (k_of > 0) & (k_of < nz)
        rr = np.where(interior, rr + u[:, 0] * dr, rr)
        tt = np.where(interior, tt + u[:, 1] * dth, tt)
        zz = np.where(interior, zz + u[:, 2] * dz, zz)
    xyz = np.stack([rr * np.cos(tt), rr * np.sin(tt), zz], axis=1)

    # cells
    I, J, K = np.meshgrid(np.arange(nr), np.arange(ntheta), np.arange(nz), indexing="ij")
    I, J, K = I.ravel(), J.ravel(), K.ravel()
    tets = []
    for perm in _PERMS:
        c = [np.zeros_like(I), np.zeros_like(I), np.zeros_like(I)]
        verts = [vid(I, J, K)]
        for d in perm:
            c[d] = c[d] + 1
            verts.append(vid(I + c[0], J + c[1], K + c[2]))
        tets.append(np.stack(verts, axis=1))
    tets = np.concatenate(tets, axis=0)
    # wedge cells collapse some Kuhn paths onto the axis: drop degenerate ones
    srt = np.sort(tets, axis=1)
    ok = np.all(srt[:, 1:] != srt[:, :-1], axis=1)
    tets = tets[ok]

    # end-face triangles: traces of the tetrahedra on z = 0 and z = L
    I2, J2 = np.meshgrid(np.arange(nr), np.arange(ntheta), indexing="ij")
    I2, J2 = I2.ravel(), J2.ravel()
    tris = []
    for kk in (0, nz):
        Kc = np.full_like(I2, kk)
        a = vid(I2, J2, Kc)
        b = vid(I2 + 1, J2, Kc)
        c = vid(I2 + 1, J2 + 1, Kc)
        d = vid(I2, J2 + 1, Kc)
        tris.append(np.stack([a, b, c], axis=1))
        quad = I2 > 0
        tris.append(np.stack([a[quad], d[quad], c[quad]], axis=1))
    tris = np.concatenate(tris, axis=0)
    return xyz, tets.astype(np.int64), tris.astype(np.int64)


def p1_matrices(xyz, tets, tris):
    """Assemble P1 stiffness K, mass M and end-face boundary mass B (real, CSR)."""
    nnode = xyz.shape[0]
    P = xyz[tets]                                   # (T,4,3)
    Jm = np.stack([P[:, 1] - P[:, 0], P[:, 2] - P[:, 0], P[:, 3] - P[:, 0]], axis=2)
    det = np.linalg.det(Jm)
    vol = np.abs(det) / 6.0
    Jinv = np.linalg.inv(Jm)                        # rows = gradients of xi_1..3
    G = np.concatenate([-Jinv.sum(axis=1, keepdims=True), Jinv], axis=1)   # (T,4,3)
    Ke = vol[:, None, None] * np.einsum("tad,tbd->tab", G, G)
    Me = (vol / 20.0)[:, None, None] * (np.ones((4, 4)) + np.eye(4))[None]
    rows = np.repeat(tets, 4, axis=1).ravel()
    cols = np.tile(tets, (1, 4)).ravel()
    K = sp.coo_matrix((Ke.ravel(), (rows, cols)), shape=(nnode, nnode)).tocsr()
    M = sp.coo_matrix((Me.ravel(), (rows, cols)), shape=(nnode, nnode)).tocsr()

    Q = xyz[tris]                                   # (F,3,3)
    area = 0.5 * np.linalg.norm(np.cross(Q[:, 1] - Q[:, 0], Q[:, 2] - Q[:, 0]), axis=1)
    Be = (area / 12.0)[:, None, None] * (np.ones((3, 3)) + np.eye(3))[None]
    br = np.repeat(tris, 3, axis=1).ravel()
    bc = np.tile(tris, (1, 3)).ravel()
    B = sp.coo_matrix((Be.ravel(), (br, bc)), shape=(nnode, nnode)).tocsr()
    return K, M, B, vol


def cylinder_helmholtz(nr, ntheta, nz, k=None, kh=None, damping=0.0, radius=1.0, length=4.0,
                       jitter=0.2, seed=None, source=(0.3, 0.0, 1.0), rcm=True,
                       return_parts=False):
    """Build the cylinder Helmholtz system.

    Exactly one of ``k`` (wavenumber) or ``kh`` (k times the axial spacing) is
    given.  Returns (CSR A, rhs b); b = M g with g a Gaussian of width
    2*dz centred at ``source`` times (1+i)/sqrt(2).
    """
    dz = length / nz
    if k is None:
        k = kh / dz
    xyz, tets, tris = cylinder_mesh(nr, ntheta, nz, radius, length, jitter, seed)
    K, M, B, _ = p1_matrices(xyz, tets, tris)
    A = K.astype(np.complex128) - (k * k * (1.0 + 1j * damping)) * M - (1j * k) * B
    sigma = 2.0 * dz
    d2 = np.sum((xyz - np.asarray(source)[None, :]) ** 2, axis=1)
    g = np.exp(-d2 / (2.0 * sigma * sigma)) * (1.0 + 1.0j) / np.sqrt(2.0)
    b = M @ g
    perm = np.arange(A.shape[0])
    if rcm:
        pat = sp.csr_matrix((np.ones(A.nnz), A.indices, A.indptr), shape=A.shape)
        perm = np.asarray(reverse_cuthill_mckee(pat, symmetric_mode=True), dtype=np.int64)
        A = A[perm][:, perm]
        b = b[perm]
    meta = {"kind": "cylinder_p1", "nr": nr, "ntheta": ntheta, "nz": nz, "k": float(k),
            "kh": float(k * dz), "damping": damping, "jitter": jitter, "seed": seed}
    csr = CSR.from_scipy(A, meta=meta)
    b = np.ascontiguousarray(b, dtype=np.complex128)
    if return_parts:
        return csr, b, {"K": K, "M": M, "B": B, "perm": perm, "xyz": xyz}
    return csr, b
