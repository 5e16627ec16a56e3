"""CSR container and seeded random vectors.

The storage follows Section 3.2 of the paper (three arrays: values AA, column
indices JA, row pointers IA), written 0-based with int32 indices and
complex128 values (two contiguous doubles per entry, Section 4).
"""

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp


@dataclass
class CSR:
    n: int
    rowptr: np.ndarray          # int32[n+1], rowptr[0] == 0, rowptr[n] == nnz
    col: np.ndarray             # int32[nnz], sorted within each row
    val: np.ndarray             # complex128[nnz]
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    @staticmethod
    def from_scipy(m, meta=None) -> "CSR":
        m = sp.csr_matrix(m)
        m.sum_duplicates()
        m.sort_indices()
        return CSR(
            n=m.shape[0],
            rowptr=np.ascontiguousarray(m.indptr, dtype=np.int32),
            col=np.ascontiguousarray(m.indices, dtype=np.int32),
            val=np.ascontiguousarray(m.data, dtype=np.complex128),
            meta=dict(meta or {}),
        )

    def to_scipy(self):
        return sp.csr_matrix((self.val, self.col, self.rowptr), shape=(self.n, self.n))

    def row_lengths(self) -> np.ndarray:
        return np.diff(self.rowptr.astype(np.int64))

    def stats(self) -> dict:
        """Row statistics in the layout of the paper's matrix table (Section 3.1):
        size, nonzeros, density %, bandwidth, max row, mean row, row stddev."""
        rl = self.row_lengths()
        rows = np.repeat(np.arange(self.n, dtype=np.int64), rl)
        bw = int(np.max(np.abs(self.col.astype(np.int64) - rows))) if self.nnz else 0
        return {
            "h": self.n,
            "nz": self.nnz,
            "density_pct": 100.0 * self.nnz / float(self.n) ** 2 if self.n else 0.0,
            "bandwidth": bw,
            "max_row": int(rl.max()) if self.n else 0,
            "nz_per_h": float(rl.mean()) if self.n else 0.0,
            "stddev": float(rl.std()) if self.n else 0.0,
        }


def complex_normal(rng: np.random.Generator, n: int) -> np.ndarray:
    """Complex normal vector: real and imaginary parts i.i.d. N(0, 1/2)."""
    s = np.sqrt(0.5)
    re = rng.standard_normal(n) * s
    im = rng.standard_normal(n) * s
    return (re + 1j * im).astype(np.complex128)
