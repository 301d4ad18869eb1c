"""Seeded synthetic workloads shaped like the paper's two examples.

This module builds matrices and nothing else: it holds none of the sampler's
arithmetic, so both the CUDA library's tests/benchmark and the FP64 oracle can
be fed from it.  Every generator is deterministic given its seed (numpy PCG64).

Workloads
---------
* ``random_dominant``  -- real non-symmetric sparse C: diagonal plus a fixed
  number of off-diagonals at distinct random columns, values U(-1, 1), diagonal
  set to ``dominance`` x the row's off-diagonal absolute sum.
* ``pedigree``         -- stands in for Wu and Schaeffer's animal-breeding
  coefficient matrix (Sec. 3.1, Table 1).  Row i couples to two parents drawn
  from earlier rows and to the parents' mate entries, following the pattern of
  the four rules listed for the non-symmetric relationship inverse
  (Sec. 3.1): (i,s), (i,d) lower, (s,i), (d,i) upper, (s,d), (d,s) between
  mates.  Each insertion carries its own -0.5*U(0.5, 1.5) value so C is
  non-symmetric; duplicates are summed; c_ii = dominance x row abs-sum.
* ``u1_lattice``       -- stands in for the free Wilson-Dirac operator of
  Sec. 3.2 (Eq. 16, Table 3) as a scalar complex non-Hermitian lattice
  operator C = I - kf sum_mu U_mu(x) d_{x+mu} - kb sum_mu conj(U_mu(x-mu))
  d_{x-mu} with U(1) link phases.  Site index i = x0 + L0*(x1 + L1*(...)),
  x0 fastest.  ``pure_gauge=True`` makes the links a gauge transform of the
  free field, so diag(C^-1) has a closed form (used as a truth value).
* ``batch_sizes``      -- n log-uniform in [lo, hi] for the batched form.

All CSR outputs: ``row_ptr`` int64[n+1], ``col`` int32[nnz] strictly
increasing per row, ``val`` float64[nnz] or complex128[nnz].
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class CSR:
    n: int
    row_ptr: np.ndarray  # int64 [n+1]
    col: np.ndarray      # int32 [nnz]
    val: np.ndarray      # float64 or complex128 [nnz]

    @property
    def nnz(self) -> int:
        return int(self.col.shape[0])

    @property
    def is_complex(self) -> bool:
        return np.iscomplexobj(self.val)

    def to_dense(self) -> np.ndarray:
        a = np.zeros((self.n, self.n), dtype=self.val.dtype)
        rows = np.repeat(np.arange(self.n), np.diff(self.row_ptr))
        a[rows, self.col] = self.val
        return a

    def to_scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.val, self.col.astype(np.int64), self.row_ptr),
                             shape=(self.n, self.n))


def csr_from_coo(n: int, rows, cols, vals) -> CSR:
    """Sum duplicate (row, col) entries and sort columns within each row."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    vals = np.asarray(vals)
    key = rows * n + cols
    order = np.argsort(key, kind="stable")
    key = key[order]
    vals = vals[order]
    uniq, start = np.unique(key, return_index=True)
    summed = np.add.reduceat(vals, start) if len(vals) else vals
    r = uniq // n
    c = uniq % n
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(row_ptr, r + 1, 1)
    row_ptr = np.cumsum(row_ptr)
    return CSR(n, row_ptr, c.astype(np.int32), summed)


def _with_dominant_diagonal(n, rows, cols, vals, dominance):
    """Append c_ii = dominance * sum_j |c_ij| (1.0 for a row with no off-diagonals)."""
    rows = np.asarray(rows, dtype=np.int64)
    absum = np.zeros(n)
    np.add.at(absum, rows, np.abs(vals))
    diag = dominance * absum
    diag[absum == 0] = 1.0
    allr = np.concatenate([rows, np.arange(n)])
    allc = np.concatenate([np.asarray(cols, dtype=np.int64), np.arange(n)])
    allv = np.concatenate([np.asarray(vals), diag.astype(np.asarray(vals).dtype)])
    return csr_from_coo(n, allr, allc, allv)


def random_dominant(n: int = 256, off_per_row: int = 4, dominance: float = 1.5,
                    seed: int = 0) -> CSR:
    """Real non-symmetric, strictly diagonally dominant sparse matrix."""
    rng = np.random.default_rng(seed)
    k = min(off_per_row, n - 1)
    rows, cols = [], []
    for i in range(n):
        c = rng.choice(n - 1, size=k, replace=False)
        c[c >= i] += 1  # distinct columns, never the diagonal
        rows.append(np.full(k, i))
        cols.append(c)
    rows = np.concatenate(rows) if rows else np.zeros(0, np.int64)
    cols = np.concatenate(cols) if cols else np.zeros(0, np.int64)
    vals = rng.uniform(-1.0, 1.0, size=rows.shape[0])
    # coalesce duplicates before taking absolute sums (there are none here by construction)
    return _with_dominant_diagonal(n, rows, cols, vals, dominance)


def pedigree(n: int = 50_000, dominance: float = 1.2, seed: int = 0) -> CSR:
    """Pedigree-shaped real non-symmetric matrix (about 7 nnz per row).

    Rows 0 and 1 are founders; every later row i draws two distinct parents
    s, d uniformly from [0, i).
    """
    rng = np.random.default_rng(seed)
    i = np.arange(2, n, dtype=np.int64)
    s = np.floor(rng.random(i.shape[0]) * i).astype(np.int64)
    d = np.floor(rng.random(i.shape[0]) * (i - 1)).astype(np.int64)
    d = np.where(d >= s, d + 1, d)
    rows = np.concatenate([i, i, s, d, s, d])
    cols = np.concatenate([s, d, i, i, d, s])
    vals = -0.5 * rng.uniform(0.5, 1.5, size=rows.shape[0])
    off = csr_from_coo(n, rows, cols, vals)  # sums duplicate mate entries
    r = np.repeat(np.arange(n), np.diff(off.row_ptr))
    return _with_dominant_diagonal(n, r, off.col, off.val, dominance)


def u1_lattice(dims=(128, 128), kappa_f: float = 0.12, kappa_b: float = 0.08,
               seed: int = 0, pure_gauge: bool = False) -> CSR:
    """Complex non-Hermitian periodic lattice operator with U(1) links."""
    dims = tuple(int(L) for L in dims)
    rng = np.random.default_rng(seed)
    n = int(np.prod(dims))
    coords = np.indices(dims[::-1]).reshape(len(dims), -1)[::-1]  # coords[mu][site], x0 fastest
    strides = np.cumprod((1,) + dims[:-1])

    def site(c):
        return (c * strides[:, None]).sum(axis=0)

    if pure_gauge:
        g = np.exp(1j * rng.uniform(0.0, 2 * math.pi, size=n))
    else:
        theta = rng.uniform(0.0, 2 * math.pi, size=(len(dims), n))
    x = site(coords)
    rows, cols, vals = [np.arange(n)], [np.arange(n)], [np.ones(n, dtype=np.complex128)]
    for mu, L in enumerate(dims):
        fwd = coords.copy()
        fwd[mu] = (fwd[mu] + 1) % L
        xf = site(fwd)
        if pure_gauge:
            link = g[x] * np.conj(g[xf])
        else:
            link = np.exp(1j * theta[mu])
        # C[x, x+mu] = -kf U_mu(x) ; C[x+mu, x] = -kb conj(U_mu(x))
        rows += [x, xf]
        cols += [xf, x]
        vals += [-kappa_f * link, -kappa_b * np.conj(link)]
    return csr_from_coo(n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))


def batch_sizes(count: int = 512, lo: int = 64, hi: int = 4096, seed: int = 0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return np.floor(np.exp(rng.uniform(math.log(lo), math.log(hi), size=count))).astype(np.int64)


def q_diag(n: int, seed: int = 0) -> np.ndarray:
    """Diagonal of Q for the trace estimate, entries U(0, 1)."""
    return np.random.default_rng(seed + 7919).uniform(0.0, 1.0, size=n)


def free_lattice_diag(dims, kappa_f, kappa_b) -> complex:
    """diag(C^-1) of the free (or pure-gauge) lattice operator, exactly.

    C is circulant on the periodic lattice; a plane wave e^{ip.x} has
    eigenvalue 1 - kf sum_mu e^{i p_mu} - kb sum_mu e^{-i p_mu}; every
    diagonal entry of C^-1 is the mean of the reciprocal eigenvalues.
    """
    grids = np.meshgrid(*[2 * math.pi * np.arange(L) / L for L in dims], indexing="ij")
    lam = np.ones_like(grids[0], dtype=np.complex128)
    for p in grids:
        lam -= kappa_f * np.exp(1j * p) + kappa_b * np.exp(-1j * p)
    return complex(np.mean(1.0 / lam))


# -- the five workloads the library is measured on ---------------------------------

@dataclasses.dataclass
class Workload:
    name: str
    K: int
    burnin: int
    samples: int
    estimates: tuple
    build: callable


WORKLOADS = {
    "random256": Workload("random256: real non-symmetric n=256, 4 off-diagonals/row, K=128",
                          128, 200, 2000, ("block_full",),
                          lambda: random_dominant(256, 4, 1.5, 0)),
    "pedigree50k": Workload("pedigree50k: real non-symmetric pedigree n=50000, ~7 nnz/row, K=1024",
                            1024, 500, 5000, ("diag", "block_cols512"),
                            lambda: pedigree(50_000, 1.2, 0)),
    "lattice2d128": Workload("lattice2d128: complex U(1) 2D periodic L=128, n=16384, K=4096",
                             4096, 300, 4000, ("diag", "trace"),
                             lambda: u1_lattice((128, 128), 0.12, 0.08, 0)),
    "lattice4d16": Workload("lattice4d16: complex U(1) 4D periodic 16^4, n=65536, K=8192",
                            8192, 50, 0, ("block4096",),
                            lambda: u1_lattice((16, 16, 16, 16), 0.06, 0.04, 0)),
}
