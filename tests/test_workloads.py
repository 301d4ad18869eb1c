"""The synthetic inputs follow the stated recipes: sizes, nonzeros per row, value
ranges, dominance, structure and determinism of the seeded generators."""
import numpy as np
import pytest

from paper_cs_0412107_gb300 import workloads as wl


def _rows(c):
    return np.repeat(np.arange(c.n), np.diff(c.row_ptr))


def _check_csr(c):
    assert c.row_ptr[0] == 0 and c.row_ptr[-1] == c.nnz and np.all(np.diff(c.row_ptr) >= 1)
    r = _rows(c)
    for i in (0, c.n // 2, c.n - 1):
        cols = c.col[c.row_ptr[i]:c.row_ptr[i + 1]]
        assert np.all(np.diff(cols) > 0), "columns strictly increasing per row"
        assert i in cols, "the diagonal is stored"
    assert np.all((c.col >= 0) & (c.col < c.n)) and r.shape[0] == c.nnz


def test_random256_recipe():
    c = wl.WORKLOADS["random256"].build()
    _check_csr(c)
    assert c.n == 256 and c.nnz == 256 * 5 and not c.is_complex
    r = _rows(c)
    off = r != c.col
    assert np.all(np.abs(c.val[off]) < 1.0)
    diag = c.val[~off]
    absoff = np.bincount(r[off], weights=np.abs(c.val[off]), minlength=c.n)
    assert np.allclose(diag, 1.5 * absoff)
    assert not np.allclose(c.to_dense(), c.to_dense().T)  # non-symmetric


def test_pedigree50k_recipe():
    c = wl.WORKLOADS["pedigree50k"].build()
    _check_csr(c)
    assert c.n == 50_000 and not c.is_complex
    assert 6.5 <= c.nnz / c.n <= 7.5  # about 7 nonzeros a row
    r = _rows(c)
    off = r != c.col
    # single couplings are -0.5 x U(0.5, 1.5); summed duplicate mate entries stay negative
    assert np.all(c.val[off] < 0) and np.all(c.val[off] <= -0.25)
    single = c.val[off][c.val[off] >= -0.75]
    assert single.size > 0.9 * off.sum()
    absoff = np.bincount(r[off], weights=np.abs(c.val[off]), minlength=c.n)
    assert np.allclose(c.val[~off], 1.2 * absoff)
    # structurally symmetric (parents <-> children, mates), values not
    pairs = set(zip(r[off].tolist(), c.col[off].tolist()))
    assert all((j, i) in pairs for (i, j) in list(pairs)[:5000])
    d = {(i, j): v for i, j, v in zip(r[off][:20000].tolist(), c.col[off][:20000].tolist(), c.val[off][:20000])}
    assert any(abs(v - d.get((j, i), v)) > 1e-3 for (i, j), v in d.items() if (j, i) in d)


@pytest.mark.parametrize("name,dims,kf,kb,deg", [("lattice2d128", (128, 128), 0.12, 0.08, 5),
                                                  ("lattice4d16", (16, 16, 16, 16), 0.06, 0.04, 9)])
def test_lattice_recipes(name, dims, kf, kb, deg):
    c = wl.WORKLOADS[name].build()
    _check_csr(c)
    n = int(np.prod(dims))
    assert c.n == n and c.nnz == deg * n and c.is_complex
    r = _rows(c)
    off = r != c.col
    assert np.allclose(c.val[~off], 1.0)
    mags = np.abs(c.val[off])
    assert np.all(np.isclose(mags, kf) | np.isclose(mags, kb))
    assert np.isclose(mags, kf).sum() == np.isclose(mags, kb).sum() == (deg - 1) // 2 * n
    # random U(1) phases: the hop values are not all real
    assert np.abs(np.angle(c.val[off])).std() > 0.5
    # site i = x0 + L x1 + ...: the x0 neighbours of site 0 are 1 and L0 - 1
    cols0 = set(c.col[c.row_ptr[0]:c.row_ptr[1]].tolist())
    assert {0, 1, dims[0] - 1, dims[0]} <= cols0


def test_batch_sizes_are_log_uniform_in_range():
    s = wl.batch_sizes(512, 64, 4096, 0)
    assert s.shape == (512,) and s.min() >= 64 and s.max() <= 4096
    # log-uniform: the median near the geometric mean 512; P(n < 128) = ln 2 / ln 64 = 1/6
    assert 350 < np.median(s) < 750
    assert 0.10 < np.mean(s < 128) < 0.23


def test_generators_are_deterministic():
    for make in (lambda: wl.pedigree(3000, 1.2, 5), lambda: wl.u1_lattice((12, 10), 0.12, 0.08, 3),
                 lambda: wl.random_dominant(300, 4, 1.5, 9)):
        a, b = make(), make()
        assert np.array_equal(a.row_ptr, b.row_ptr) and np.array_equal(a.col, b.col)
        assert np.array_equal(a.val, b.val)
    q = wl.q_diag(1000, 4)
    assert np.array_equal(q, wl.q_diag(1000, 4)) and q.min() >= 0 and q.max() < 1
