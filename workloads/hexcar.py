"""Trilinear (Q1) hexahedral finite-element Helmholtz matrix on a car-cabin
shaped cavity.

Stand-in for the paper's "Audi3D" and "Twingo3D" matrices (Section 3.1):
acoustic cavities of car interiors meshed with hexahedra, whose statistics
table gives at most 27 nonzeros per row (a node and its 26 neighbours in a
hexahedral mesh).  Those meshes are not distributed with the paper.  Here the
cabin is a voxel body on a uniform grid of cubes with side h: a box of
length L, width W and height H from which the engine bay and dashboard
(front, below a sloping windscreen), the boot (rear, below a sloping rear
window) and the two seat rows (blocks with backrests) are cut out.  Every
kept cube is a Q1 element.  The assembled operator is

    A = K - k^2 (1 + i*damping) M - i k B,

with K, M the Q1 stiffness and mass matrices (tensor products of the 1D
linear element matrices) and B the Q1 boundary mass of the faces that touch
a seat (first-order impedance: absorbing upholstery); the other walls are
rigid (natural condition).  A is complex symmetric; rows are reordered by
reverse Cuthill-McKee like the cylinder.
"""

import numpy as np
import scipy.sparse as sp
from scipy.sparse.csgraph import reverse_cuthill_mckee

from .csr import CSR

# 1D linear element on [0, 1]: mass and stiffness
_M1 = np.array([[1.0 / 3.0, 1.0 / 6.0], [1.0 / 6.0, 1.0 / 3.0]])
_K1 = np.array([[1.0, -1.0], [-1.0, 1.0]])


def q1_reference():
    """8x8 Q1 stiffness and mass on the unit cube, local node (a, b, c) -> 4a + 2b + c."""
    M = np.kron(np.kron(_M1, _M1), _M1)
    K = np.kron(np.kron(_K1, _M1), _M1) + np.kron(np.kron(_M1, _K1), _M1) + np.kron(np.kron(_M1, _M1), _K1)
    return K, M


def _centres(nx, ny, nz, length, width, height):
    x = (np.arange(nx) + 0.5) * (length / nx)
    y = (np.arange(ny) + 0.5) * (width / ny)
    z = (np.arange(nz) + 0.5) * (height / nz)
    return np.meshgrid(x, y, z, indexing="ij")


def body_mask(nx, ny, nz, length=4.0, width=1.8, height=1.3):
    """Cubes of the car body around the cabin: the engine bay and dashboard
    (front 0.9 m up to 0.55 H, then below a windscreen rising to the roof at
    1.5 m) and the boot (below a rear window from the roof at 3.3 m down to
    0.5 H at the back)."""
    X, _, Z = _centres(nx, ny, nz, length, width, height)
    body = (X < 0.9) & (Z < 0.55 * height)
    body |= (X < 1.5) & (X < 0.9 + (Z - 0.55 * height) * (0.6 / (0.45 * height)))
    body |= X > 3.3 + (height - Z) * (0.7 / (0.5 * height))
    return body


def seat_mask(nx, ny, nz, length=4.0, width=1.8, height=1.3):
    """Cubes of the two seat rows: cushions 0.5 m deep and 0.25 m high with
    backrests 0.12 m thick and 0.75 m high, split by a 0.2 m aisle."""
    X, Y, Z = _centres(nx, ny, nz, length, width, height)
    side = np.abs(Y - 0.5 * width) > 0.1
    seats = np.zeros((nx, ny, nz), dtype=bool)
    for x0 in (1.75, 2.75):
        seats |= (X > x0) & (X < x0 + 0.5) & (Z < 0.25) & side
        seats |= (X > x0 + 0.5) & (X < x0 + 0.62) & (Z < 0.75) & side
    return seats


def cabin_mask(nx, ny, nz, length=4.0, width=1.8, height=1.3):
    """Boolean (nx, ny, nz) array: cube (i, j, k) belongs to the cabin air."""
    return ~(body_mask(nx, ny, nz, length, width, height) | seat_mask(nx, ny, nz, length, width, height))


def hexcar_helmholtz(nx=120, kh=0.5, damping=0.05, length=4.0, width=1.8, height=1.3,
                     source=(1.9, 0.45, 1.0), rcm=True, return_parts=False):
    """Build the cabin Helmholtz system on a grid of cubes with side
    h = length / nx (ny = round(width / h), nz = round(height / h) cubes
    across and up, so the cabin is nx h x ny h x nz h), k = kh / h.
    Returns (CSR A, rhs b); b = M g with g a Gaussian of width 2h at
    ``source`` (a head position above the front-left seat) times (1+i)/sqrt(2).
    """
    h = length / nx
    ny, nz = int(round(width / h)), int(round(height / h))
    width, height = ny * h, nz * h
    k = kh / h
    keep = cabin_mask(nx, ny, nz, length, width, height)
    ci, cj, ck = np.nonzero(keep)
    # global node number of grid point (i, j, k) before compaction
    nid = lambda i, j, kk: (i * (ny + 1) + j) * (nz + 1) + kk
    corners = np.stack([nid(ci + a, cj + b, ck + c) for a in (0, 1) for b in (0, 1) for c in (0, 1)], axis=1)
    used, inv = np.unique(corners, return_inverse=True)
    elems = inv.reshape(corners.shape)                 # (E, 8) compact node ids
    nnode = used.size
    Kr, Mr = q1_reference()
    rows = np.repeat(elems, 8, axis=1).ravel()
    cols = np.tile(elems, (1, 8)).ravel()
    ne = elems.shape[0]
    K = sp.coo_matrix((np.tile((h * Kr).ravel(), ne), (rows, cols)), shape=(nnode, nnode)).tocsr()
    M = sp.coo_matrix((np.tile((h ** 3 * Mr).ravel(), ne), (rows, cols)), shape=(nnode, nnode)).tocsr()
    # impedance faces: faces shared by a kept cube and a removed seat cube
    seat = seat_mask(nx, ny, nz, length, width, height)
    faces = []
    for axis in range(3):
        for side in (0, 1):
            sh = [0, 0, 0]
            sh[axis] = 1 if side else -1
            nb = np.array([ci + sh[0], cj + sh[1], ck + sh[2]])
            inside = (nb[0] >= 0) & (nb[0] < nx) & (nb[1] >= 0) & (nb[1] < ny) & (nb[2] >= 0) & (nb[2] < nz)
            hit = np.zeros(ci.size, dtype=bool)
            hit[inside] = seat[nb[0][inside], nb[1][inside], nb[2][inside]]
            if not hit.any():
                continue
            loc = [(a, b, c) for a in (0, 1) for b in (0, 1) for c in (0, 1) if (a, b, c)[axis] == side]
            idx = [4 * a + 2 * b + c for a, b, c in loc]
            faces.append(elems[hit][:, idx])
    B = sp.csr_matrix((nnode, nnode))
    if faces:
        F = np.concatenate(faces, axis=0)                # (nf, 4) in tensor order of the face
        Bf = np.kron(_M1, _M1) * h * h
        br = np.repeat(F, 4, axis=1).ravel()
        bc = np.tile(F, (1, 4)).ravel()
        B = sp.coo_matrix((np.tile(Bf.ravel(), F.shape[0]), (br, bc)), shape=(nnode, nnode)).tocsr()
    A = K.astype(np.complex128) - (k * k * (1.0 + 1j * damping)) * M - (1j * k) * B
    # node coordinates and the source
    gi = used // ((ny + 1) * (nz + 1))
    gj = (used // (nz + 1)) % (ny + 1)
    gk = used % (nz + 1)
    xyz = np.stack([gi * h, gj * h, gk * h], axis=1)
    sigma = 2.0 * h
    d2 = np.sum((xyz - np.asarray(source)[None, :]) ** 2, axis=1)
    g = np.exp(-d2 / (2.0 * sigma * sigma)) * (1.0 + 1.0j) / np.sqrt(2.0)
    b = M @ g
    perm = np.arange(nnode)
    if rcm:
        pat = sp.csr_matrix((np.ones(A.nnz), A.indices, A.indptr), shape=A.shape)
        perm = np.asarray(reverse_cuthill_mckee(pat, symmetric_mode=True), dtype=np.int64)
        A = A[perm][:, perm]
        b = b[perm]
    A.sort_indices()
    meta = {"kind": "hexcar_q1", "nx": nx, "ny": ny, "nz": nz, "h": h, "k": float(k), "kh": kh,
            "damping": damping, "elements": int(ne)}
    csr = CSR.from_scipy(A, meta=meta)
    b = np.ascontiguousarray(b, dtype=np.complex128)
    if return_parts:
        return csr, b, {"K": K, "M": M, "B": B, "perm": perm, "xyz": xyz, "volume": ne * h ** 3}
    return csr, b
