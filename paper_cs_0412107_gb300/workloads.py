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
* ``wilson_dirac``     -- the paper's own Example 2 matrix (Sec. 3.2, Eqs.
  disDirac and explicit): the free 4-spinor Wilson-Dirac operator on a periodic
  N1 x N2 x N3 x N0 lattice, 14 nonzeros per row (Table 3).
  ``wilson_dirac_propagator`` / ``wilson_dirac_inverse_trace`` give its exact
  inverse from the momentum-space closed form (truth values, not the sampler).
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


# Euclidean gamma matrices in the Dirac representation: gamma^k = [[0, -i s_k], [i s_k, 0]]
# (k = 1, 2, 3, Pauli s_k) and gamma^4 = diag(1, 1, -1, -1).  Hermitian, square to 1 and
# anticommute.  The paper prints gamma^k without the -i / i factors and with s_2 = [[0,-i],[-i,0]];
# only this Hermitian set reproduces its exact traces (Tables 4, 5), and only the Dirac form of
# gamma^4 gives its 14 nonzeros per row (Table 3).
_PAULI = (np.array([[0, 1], [1, 0]], dtype=np.complex128),
          np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
          np.array([[1, 0], [0, -1]], dtype=np.complex128))
_Z2 = np.zeros((2, 2), dtype=np.complex128)
DIRAC_GAMMA = tuple([np.block([[_Z2, -1j * s], [1j * s, _Z2]]) for s in _PAULI]
                    + [np.diag([1.0, 1.0, -1.0, -1.0]).astype(np.complex128)])


def wilson_dirac(dims=(18, 18, 18, 18), kappa: float = 0.1, spin_fastest: bool = False) -> CSR:
    """The free Wilson-Dirac matrix of Sec. 3.2 (Eqs. disDirac and explicit).

    L = I + kappa sum_mu [(1 + gamma^mu) d_{y, x+mu} + (1 - gamma^mu) d_{y, x-mu}] on a
    periodic lattice ``dims = (N1, N2, N3, N0)``; direction mu = 1, 2, 3, 4 moves
    coordinate N1, N2, N3, N0 (time last).  Row index, 0-based, follows the paper's
    mapping with the spinor index slowest: i = a + N1 (b + N2 (c + N3 (d + N0 s))).
    ``spin_fastest`` numbers the same operator with the spinor index fastest,
    i = s + 4 (a + N1 (...)): a relabelling (P L P^T) that keeps a site's four spinor
    rows together.  Zero entries of (1 +- gamma^4) are not stored: 14 nonzeros per row.
    """
    dims = tuple(int(L) for L in dims)
    V = int(np.prod(dims))
    coords = np.indices(dims[::-1]).reshape(4, -1)[::-1]  # coords[mu][site], N1 fastest
    strides = np.cumprod((1,) + dims[:-1])
    x = (coords * strides[:, None]).sum(axis=0)
    rows, cols, vals = [np.arange(4 * V)], [np.arange(4 * V)], [np.ones(4 * V, dtype=np.complex128)]
    eye = np.eye(4, dtype=np.complex128)
    for mu in range(4):
        for sign in (1, -1):
            nb = coords.copy()
            nb[mu] = (nb[mu] + sign) % dims[mu]
            y = (nb * strides[:, None]).sum(axis=0)
            blk = kappa * (eye + sign * DIRAC_GAMMA[mu])
            for s in range(4):
                for t in range(4):
                    if blk[s, t] != 0:
                        if spin_fastest:
                            rows.append(4 * x + s)
                            cols.append(4 * y + t)
                        else:
                            rows.append(x + V * s)
                            cols.append(y + V * t)
                        vals.append(np.full(V, blk[s, t]))
    return csr_from_coo(4 * V, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))


def wilson_dirac_propagator(dims, kappa: float, r=(0, 0, 0, 0)) -> np.ndarray:
    """The 4x4 spinor block L^-1(x, x + r) of ``wilson_dirac``, exactly (any site x).

    L is block-circulant on the periodic lattice: a plane wave e^{ip.y} u is mapped to
    e^{ip.x} M(p) u with M(p) = I + kappa sum_mu [2 cos p_mu + 2i sin p_mu gamma^mu], so
    L^-1(x, x + r) = (1/V) sum_p e^{-ip.r} M(p)^-1, p_mu = 2 pi k / N_mu.
    """
    grids = np.meshgrid(*[2 * math.pi * np.arange(L) / L for L in dims], indexing="ij")
    P = np.stack([g.ravel() for g in grids], axis=-1)
    M = np.broadcast_to(np.eye(4, dtype=np.complex128), (len(P), 4, 4)).copy()
    for mu in range(4):
        M += kappa * (2 * np.cos(P[:, mu])[:, None, None] * np.eye(4)
                      + 2j * np.sin(P[:, mu])[:, None, None] * DIRAC_GAMMA[mu])
    phase = np.exp(-1j * (P @ np.asarray(r, dtype=np.float64)))
    return np.einsum("p,pij->ij", phase, np.linalg.inv(M)) / len(P)


def wilson_dirac_inverse_trace(dims, kappa: float) -> complex:
    """tr(L^-1) of ``wilson_dirac``: the lattice volume times the trace of the r = 0 block."""
    return complex(np.prod(dims) * np.trace(wilson_dirac_propagator(dims, kappa)))


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
