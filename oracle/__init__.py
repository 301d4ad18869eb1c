"""FP64 CPU oracle for the correlated-chains (CC) Monte Carlo inverse.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package.  It shares no code with
the CUDA library (``paper_cs_0412107_gb300``) and never imports it.

Contents
--------
* ``mcinv_oracle.c`` (built here into ``_build/liboracle.so``): Philox4x32-10,
  the Z2 noise draw, the in-place CC sweep of Eqs. 4/5 chain by chain, the
  accumulation of Eq. 1/C, and the coupling burn-in of Algorithm 1.
* This module: ctypes wrappers, plus plain numpy statements of what the sweep
  must satisfy (dense truths used as pins): the matrix form of the update
  (Eqs. mform1/mform2, zk/wk), the exact expected covariance recursion behind
  Eqs. series/recursive, group standard errors.

Parity pinned: Philox (published known-answer vectors), the sweep (matrix
form, closed forms, dense-LU statistics), the accumulation (brute force).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mcinv_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (portable flags only: no -march)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp", "-fno-fast-math",
               "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            P = ctypes.POINTER
            u32p = P(ctypes.c_uint32)
            L.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
            L.orc_philox4x32_10.restype = None
            L.orc_phi.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                  ctypes.c_uint32, ctypes.c_uint32]
            L.orc_phi.restype = ctypes.c_int
            vp = ctypes.c_void_p
            L.orc_row_constants.argtypes = [ctypes.c_int64, vp, vp, vp, ctypes.c_int, vp, vp, vp]
            L.orc_row_constants.restype = ctypes.c_int64
            L.orc_cc_run.argtypes = [ctypes.c_int64, vp, vp, vp, ctypes.c_int, ctypes.c_int64,
                                     ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32,
                                     ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                     vp, vp, ctypes.c_int64, vp, vp, ctypes.c_int64, vp,
                                     ctypes.c_int64, vp, vp, vp, ctypes.c_int]
            L.orc_cc_run.restype = ctypes.c_int64
            L.orc_coupling_burnin.argtypes = [ctypes.c_int64, vp, vp, vp, ctypes.c_int,
                                              ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                              ctypes.c_double, ctypes.c_int64, vp, vp]
            L.orc_coupling_burnin.restype = ctypes.c_int64
            L.orc_noise_plane.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32,
                                          ctypes.c_uint32, ctypes.c_uint32, vp]
            L.orc_noise_plane.restype = None
            _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _csr_arrays(csr):
    rp = np.ascontiguousarray(csr.row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(csr.col, dtype=np.int32)
    if np.iscomplexobj(csr.val):
        val = np.ascontiguousarray(csr.val, dtype=np.complex128).view(np.float64)
        return rp, col, val, 1
    return rp, col, np.ascontiguousarray(csr.val, dtype=np.float64), 0


# -- noise --------------------------------------------------------------------------

def philox4x32_10(ctr, key):
    c = (ctypes.c_uint32 * 4)(*[int(x) & 0xffffffff for x in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(x) & 0xffffffff for x in key])
    o = (ctypes.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return tuple(int(x) for x in o)


def phi(seed, matrix, chain, cycle, row) -> int:
    return int(lib().orc_phi(seed, matrix, chain, cycle, row))


def noise_plane(n, K, seed, matrix, chain0, cycle) -> np.ndarray:
    """phi^(cycle) of every row and of chains chain0 .. chain0+K-1: float64 [n][K]."""
    out = np.empty((n, K), dtype=np.int8)
    lib().orc_noise_plane(ctypes.c_int64(n), ctypes.c_int64(K), ctypes.c_uint64(seed), ctypes.c_uint32(matrix),
                          ctypes.c_uint32(chain0), ctypes.c_uint32(cycle), _ptr(out))
    return out.astype(np.float64)


def noise_matrix(n, seed, matrix, chain, cycle) -> np.ndarray:
    """phi^(cycle) for one chain as a length-n float vector (row loop; small n)."""
    L = lib()
    return np.array([L.orc_phi(seed, matrix, chain, cycle, i) for i in range(n)], dtype=np.float64)


# -- per-row constants --------------------------------------------------------------

def row_constants(csr):
    rp, col, val, cx = _csr_arrays(csr)
    n = csr.n
    a = np.zeros(2 * n); b = np.zeros(2 * n); d = np.zeros(2 * n)
    bad = lib().orc_row_constants(n, _ptr(rp), _ptr(col), _ptr(val), cx, _ptr(a), _ptr(b), _ptr(d))
    if bad:
        raise ValueError(f"singular diagonal at row {-bad - 1}")
    v = lambda x: x.view(np.complex128)
    return v(a), v(b), v(d)


# -- the sampler --------------------------------------------------------------------

class State:
    """Chain state [n][K] complex128 for z and w (Algorithm 1 step 1: zeros)."""

    def __init__(self, n, K):
        self.z = np.zeros((n, K), dtype=np.complex128)
        self.w = np.zeros((n, K), dtype=np.complex128)


def run(csr, K, seed=0, matrix=0, chain0=0, cycle0=0, ncycles=1, acc_from=None,
        state=None, cpg=None, R=None, S=None, diag=True, threads=1, q=None, series_out=None):
    """Advance K chains ``ncycles`` cycles from ``state`` (zeros if None).

    Cycles with global index >= ``acc_from`` are accumulated (default: none).
    Returns (state, diag_acc [G][n] or None, blk_acc [G][|R|][|S|] or None).
    With ``q`` and a list ``series_out``, the realised per-cycle trace values
    (1/K) sum_chains sum_i q_i Re(z_i conj(w_i)) of the accumulated cycles are
    appended to ``series_out``.
    """
    n = csr.n
    if state is None:
        state = State(n, K)
    if acc_from is None:
        acc_from = cycle0 + ncycles  # accumulate nothing
    cpg = K if cpg is None else int(cpg)
    G = (K + cpg - 1) // cpg
    rp, col, val, cx = _csr_arrays(csr)
    dacc = np.zeros((G, n), dtype=np.complex128) if diag else None
    if R is not None:
        R = np.ascontiguousarray(R, dtype=np.int64)
        S = np.ascontiguousarray(S, dtype=np.int64)
        bacc = np.zeros((G, len(R), len(S)), dtype=np.complex128)
    else:
        bacc = None
    zv = state.z.view(np.float64)
    wv = state.w.view(np.float64)
    nacc = max(0, cycle0 + ncycles - max(acc_from, cycle0))
    qv = None if q is None else np.ascontiguousarray(q, dtype=np.float64)
    tser = np.zeros((G, max(nacc, 1))) if qv is not None else None
    assert state.z.flags.c_contiguous and state.w.flags.c_contiguous
    rc = lib().orc_cc_run(n, _ptr(rp), _ptr(col), _ptr(val), cx, K, chain0, seed, matrix,
                          cycle0, ncycles, acc_from, _ptr(zv), _ptr(wv), cpg,
                          _ptr(None if dacc is None else dacc.view(np.float64)),
                          _ptr(R), 0 if R is None else len(R), _ptr(S), 0 if S is None else len(S),
                          _ptr(None if bacc is None else bacc.view(np.float64)), _ptr(qv), _ptr(tser), threads)
    if rc:
        raise ValueError(f"singular diagonal at row {-rc - 1}")
    if tser is not None and series_out is not None:
        series_out.extend((tser.sum(axis=0)[:nacc] / K).tolist())
    return state, dacc, bacc


def coupling_burnin(csr, seed=0, matrix=0, chain=0, tol=5e-5, max_cycles=10000):
    """Algorithm 1 steps 1-5 for one chain; returns (p, z, w)."""
    rp, col, val, cx = _csr_arrays(csr)
    z = np.zeros(csr.n, dtype=np.complex128)
    w = np.zeros(csr.n, dtype=np.complex128)
    p = lib().orc_coupling_burnin(csr.n, _ptr(rp), _ptr(col), _ptr(val), cx, seed, matrix, chain,
                                  tol, max_cycles, _ptr(z.view(np.float64)), _ptr(w.view(np.float64)))
    return int(p), z, w


# -- estimates and standard errors ---------------------------------------------------

def group_estimate(acc, counts, samples):
    """Mean and standard error from independent chain groups.

    acc: [G, ...] sums over each group's chains and samples; counts: [G] chains
    per group.  Mean = sum / (chains * samples); SE^2 = sum_g n_g (m_g - m)^2 /
    ((G - 1) N) (for equal groups: the variance of the group means over G).
    Real and imaginary parts get separate SEs.
    """
    acc = np.asarray(acc)
    counts = np.asarray(counts, dtype=np.float64)
    N = counts.sum()
    shape = (-1,) + (1,) * (acc.ndim - 1)
    mg = acc / (counts.reshape(shape) * samples)
    m = acc.sum(axis=0) / (N * samples)
    G = acc.shape[0]

    def se(x, mx):
        return np.sqrt((counts.reshape(shape) * (x - mx) ** 2).sum(axis=0) / ((G - 1) * N))

    if np.iscomplexobj(acc):
        return m, se(mg.real, m.real) + 1j * se(mg.imag, m.imag)
    return m, se(mg, m)


def geyer_ims(x):
    """Geyer's (1992) initial monotone sequence estimator for a stationary series
    (the effective length Sec. 2.3 and Sec. 3.1 take from Geyer).

    gamma(k): lag-k autocovariance (divided by M); the pair sums
    Gamma_j = gamma(2j) + gamma(2j+1) are taken while positive (the initial
    positive sequence), and each is then capped by the one before it, so the
    summed sequence is non-increasing (the monotone refinement);
    asymptotic variance sigma^2 = -gamma(0) + 2 sum Gamma_j; effective length
    M gamma(0) / sigma^2; standard error of the mean
    sqrt(sigma^2 / M) = sqrt(gamma(0) / ess).  Returns dict(mean, var, ess, se).
    """
    x = np.asarray(x, dtype=np.float64)
    M = len(x)
    d = x - x.mean()
    # autocovariances through an FFT of the zero-padded series
    f = np.fft.rfft(d, 2 * M)
    acov = np.fft.irfft(f * np.conj(f))[:M] / M
    total, prev = 0.0, np.inf
    for j in range(M // 2):
        G = acov[2 * j] + acov[2 * j + 1]
        if G <= 0:
            break
        G = min(G, prev)
        prev = G
        total += G
    sigma2 = -acov[0] + 2 * total
    ess = M * acov[0] / sigma2
    return {"mean": float(x.mean()), "var": float(acov[0]), "ess": float(ess), "se": float(np.sqrt(sigma2 / M))}


# -- dense statements used as pins (small n) -------------------------------------------

def split_ldu(a):
    """C = L + D + U (Sec. 2.1): strictly lower, diagonal, strictly upper."""
    return np.tril(a, -1), np.diag(np.diag(a)), np.triu(a, 1)


def matrix_form_step(a, alpha, beta, phi_vec, z_prev, w_prev):
    """One cycle in the matrix form of Eqs. mform1/mform2 (solved as Eqs. zk/wk).

    (D+L) z^(k) = D diag(alpha) phi - U z^(k-1)
    (D+U)^H w^(k) = D^H diag(beta) phi - L^H w^(k-1)
    """
    import scipy.linalg as sl
    L, D, U = split_ldu(a)
    rhs_z = D @ (alpha * phi_vec) - U @ z_prev
    z = sl.solve_triangular(D + L, rhs_z, lower=True)
    rhs_w = D.conj().T @ (beta * phi_vec) - L.conj().T @ w_prev
    w = sl.solve_triangular((D + U).conj().T, rhs_w, lower=True)
    return z, w


def expected_covariance(a, k):
    """E[z^(k) w^(k)H] from zero start: X_k = G + T X_{k-1} S, X_0 = 0.

    T = (D+L)^-1 U, S = L (D+U)^-1, G = (D+L)^-1 D (D+U)^-1 (Eqs. T, S, series);
    the fixed point is C^-1 (Eq. recursive).
    """
    L, D, U = split_ldu(a)
    DL = np.linalg.inv(D + L)
    DU = np.linalg.inv(D + U)
    T = DL @ U
    S = L @ DU
    Gm = DL @ D @ DU
    X = np.zeros_like(a, dtype=np.complex128)
    for _ in range(k):
        X = Gm + T @ X @ S
    return X


# -- the block partition of Sec. 4 ---------------------------------------------------
#
# C is cut into contiguous diagonal blocks D_b (block_ptr[b] .. block_ptr[b+1]-1); the
# sweep visits the blocks in ascending order and updates each block as a whole:
#   z_b <- A_b phi_b - D_b^-1 sum_{c != b} C_bc z_c       (new z_c for c < b, old for c > b)
#   w_b <- B_b phi_b - D_b^-H sum_{c != b} (C^H)_bc w_c
# with A_b B_b^H = D_b^-1, the condition that makes E[z w^H] converge to C^-1 (the block
# form of the demonstration of Sec. 2.2).  The factors are read from the scalar case
# (alpha = 1/sqrt(c_ii), beta = 1/conj(sqrt(c_ii))): A_b = S_b^-1 and B_b = (S_b^-1)^H with
# S_b the principal square root of D_b, which exists when no eigenvalue of D_b lies on the
# closed negative real axis (a block without one is rejected).  Blocks of one row keep the
# scalar constants.

def block_factors(csr, block_ptr):
    """Per block: (rows, D_b^-1, A_b, B_b).  One-row blocks take the scalar constants
    (row_constants: alpha, beta, 1/c_ii, including the real reading for c_ii < 0)."""
    import scipy.linalg as sl
    a = csr.to_dense().astype(np.complex128)
    out = []
    for b in range(len(block_ptr) - 1):
        r = np.arange(block_ptr[b], block_ptr[b + 1])
        if len(r) == 1:
            c = a[r[0], r[0]]
            if c == 0:
                raise ValueError(f"one-row block {b} has a zero diagonal")
            if not csr.is_complex and c.real < 0:  # the real reading: alpha = 1/sqrt|c|, beta = -alpha
                al = 1.0 / np.sqrt(-c.real); be = -al
            else:
                sq = np.sqrt(c)
                al = 1.0 / sq; be = 1.0 / np.conj(sq)
            out.append((r, np.array([[1.0 / c]]), np.array([[al]]), np.array([[be]])))
        else:
            D = a[np.ix_(r, r)]
            ev = np.linalg.eigvals(D)
            if np.any((np.abs(ev.imag) <= 1e-12 * np.abs(ev)) & (ev.real <= 0)):
                raise ValueError(f"block {b} has no principal square root (an eigenvalue on the closed negative real axis)")
            A = np.linalg.inv(sl.sqrtm(D))
            out.append((r, np.linalg.inv(D), A, A.conj().T))
    return out


def block_cycle(a, fac, st, ph):
    """One cycle of the block sweep on the dense matrix a with noise ph [n][K], in place."""
    ah = a.conj().T
    for r, Dinv, A, B in fac:
        sz = a[r, :] @ st.z - a[np.ix_(r, r)] @ st.z[r, :]  # sum over the other blocks
        st.z[r, :] = A @ ph[r, :] - Dinv @ sz
    for r, Dinv, A, B in fac:
        sw = ah[r, :] @ st.w - ah[np.ix_(r, r)] @ st.w[r, :]
        st.w[r, :] = B @ ph[r, :] - Dinv.conj().T @ sw
    return st


def run_block(csr, block_ptr, K, seed=0, matrix=0, chain0=0, cycle0=0, ncycles=1, state=None):
    """The block-partition sweep above, FP64 complex, dense (small n); returns the state."""
    a = csr.to_dense().astype(np.complex128)
    st = state if state is not None else State(csr.n, K)
    fac = block_factors(csr, block_ptr)
    for cyc in range(cycle0, cycle0 + ncycles):
        block_cycle(a, fac, st, noise_plane(csr.n, K, seed, matrix, chain0, cyc))
    return st


def block_expected_covariance(a, block_ptr, k):
    """E[z^(k) w^(k)H] of the block sweep from zero: the recursion of expected_covariance
    with D block-diagonal and L, U the blocks below and above it (A_b B_b^H = D_b^-1)."""
    a = np.asarray(a, dtype=np.complex128)
    n = a.shape[0]
    D = np.zeros_like(a)
    for b in range(len(block_ptr) - 1):
        r = np.arange(block_ptr[b], block_ptr[b + 1])
        D[np.ix_(r, r)] = a[np.ix_(r, r)]
    blk = np.zeros(n, dtype=np.int64)
    for b in range(len(block_ptr) - 1):
        blk[block_ptr[b]:block_ptr[b + 1]] = b
    lower = blk[:, None] > blk[None, :]
    L = np.where(lower, a, 0)
    U = np.where(blk[:, None] < blk[None, :], a, 0)
    DL = np.linalg.inv(D + L)
    DU = np.linalg.inv(D + U)
    T = DL @ U
    S = L @ DU
    Gm = DL @ D @ DU
    X = np.zeros_like(a)
    for _ in range(k):
        X = Gm + T @ X @ S
    return X

