"""Seeded test inputs shared by the oracle tests and the GPU parity tests.

Input construction only (matrices, vectors, fixtures); no SpMV, dot product
or solver arithmetic lives here.
"""

import os

import numpy as np
import scipy.sparse as sp

from workloads import CSR, complex_normal

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def worked_example():
    """(dense 5x5 matrix, 1-based (row, col) pattern) from tests/golden."""
    rows, pattern = [], []
    with open(os.path.join(GOLDEN, "csr_worked_example.txt")) as f:
        for line in f:
            if line.startswith("row "):
                rows.append([float(v) for v in line.split()[1:]])
            elif line.startswith("pattern "):
                pattern = [tuple(int(q) for q in p.split("/")) for p in line.split()[1:]]
    return np.array(rows), pattern


def worked_example_csr(scale=1.0 + 0.0j) -> CSR:
    dense, _ = worked_example()
    return CSR.from_scipy(sp.csr_matrix(dense.astype(np.complex128) * scale))


def random_csr(n, seed, max_row=40, empty_frac=0.05, long_rows=(), diag=True) -> CSR:
    """Ragged random CSR: row lengths uniform in [0, max_row], a fraction of
    empty rows, a few long rows of given lengths, sorted columns."""
    rng = np.random.default_rng(seed)
    lens = rng.integers(0, max_row + 1, size=n)
    lens[rng.random(n) < empty_frac] = 0
    for i, L in enumerate(long_rows):
        lens[(7 * i + 3) % n] = min(L, n)
    rows, cols = [], []
    for i in range(n):
        L = int(min(lens[i], n))
        c = rng.choice(n, size=L, replace=False) if L else np.zeros(0, dtype=np.int64)
        if diag and L and i not in c:
            c[0] = i
        rows.append(np.full(L, i))
        cols.append(np.sort(c))
    r = np.concatenate(rows) if rows else np.zeros(0, np.int64)
    c = np.concatenate(cols) if cols else np.zeros(0, np.int64)
    v = complex_normal(rng, r.size)
    m = sp.csr_matrix((v, (r, c)), shape=(n, n))
    m.sort_indices()
    return CSR(n, m.indptr.astype(np.int32), m.indices.astype(np.int32),
               m.data.astype(np.complex128))


def small_cylinder(seed=7, kh=0.5, damping=0.05):
    from workloads import cylinder_helmholtz
    return cylinder_helmholtz(6, 16, 20, kh=kh, damping=damping, jitter=0.2, seed=seed)


def row_abs_scale(A: CSR, x: np.ndarray) -> np.ndarray:
    """sum_j |a_ij| |x_j| per row: the magnitude an entry of A x is rounded against."""
    m = sp.csr_matrix((np.abs(A.val), A.col, A.rowptr), shape=(A.n, A.n))
    return m @ np.abs(x)


def vectors(n, seed, count=2):
    rng = np.random.default_rng(seed)
    return [complex_normal(rng, n) for _ in range(count)]


def breakdown_2x2() -> CSR:
    """A = [[0, 1], [-1, 0]]: with b = e_1, <r0, A r0> = 0 in the first step."""
    return CSR.from_scipy(sp.csr_matrix(np.array([[0.0, 1.0], [-1.0, 0.0]], dtype=np.complex128)))
