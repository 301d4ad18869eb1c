"""The BF16 tensor-core block contraction (tcgen05 + TMA + TMEM).

1. The contraction itself, D = A B^T on BF16 inputs with FP32 accumulation,
   against float64 numpy on the same BF16 values: ragged M, N and several K
   tiles; bound = FP32 accumulation error, inner * 2^-23 * sum_k |a_k b_k|.
2. The block estimate through the BF16 path against the FP32 path on the same
   draws: each product z_r conj(w_s) is formed from BF16-rounded operands, so
   |dz w| <= (2u + u^2) |z| |w| with u = 2^-8 per entry and sample.
3. Statistics: the BF16 estimate of the random256 inverse covers the dense LU
   inverse within its Monte Carlo error.
"""
import numpy as np
import pytest

from paper_cs_0412107_gb300 import build as libbuild
from paper_cs_0412107_gb300 import mcinv
from paper_cs_0412107_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
U_BF16 = 2.0 ** -8


@pytest.fixture(scope="module", autouse=True)
def _lib():
    libbuild.build()
    mcinv.lib()


def to_bf16_bits(x):
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = (u + 0x7FFF + ((u >> 16) & 1)) >> 16
    return r.astype(np.uint16)


def from_bf16_bits(b):
    return (b.astype(np.uint32) << 16).view(np.float32)


@pytest.mark.parametrize("M,N,inner", [(128, 256, 64), (300, 200, 192), (1000, 600, 1024), (129, 513, 64 * 37),
                                       # more tiles than SMs (152 on GB300) with short tiles: a last wave of
                                       # 8, 3 or 100 tiles run whole
                                       (10240, 512, 2048), (19500, 300, 64 * 40), (16100, 512, 256)])
def test_tc_contraction_matches_fp64(M, N, inner):
    rng = np.random.default_rng(M + N + inner)
    A = to_bf16_bits(rng.normal(size=(M, inner)))
    B = to_bf16_bits(rng.normal(size=(N, inner)))
    D = mcinv.mcinv_selftest_tc_gemm(A, B)
    a = from_bf16_bits(A).astype(np.float64)
    b = from_bf16_bits(B).astype(np.float64)
    want = a @ b.T
    bound = inner * 2.0 ** -23 * (np.abs(a) @ np.abs(b).T) + 1e-30
    assert np.all(np.abs(D - want) <= bound), np.abs(D - want).max()


def test_tc_split_last_wave_is_exact():
    """170 tiles of 128 x 256 on 152 SMs with 515 k-slices of 64 a tile: the last
    wave's 18 tiles are split along the contraction into 8 uneven parts each, written
    to a workspace and summed in part order by the warp completing each 32-row
    quarter.  Operands are small integers (exact in BF16) and every partial sum stays
    below 2^24, so FP32 accumulation is exact in any order: D must equal the integer
    product bit for bit, the ragged N = 40 columns included."""
    rng = np.random.default_rng(5)
    M, N, inner = 128 * 170, 40, 64 * 515
    Ai = rng.integers(-4, 5, size=(M, inner), dtype=np.int8)
    Bi = rng.integers(-4, 5, size=(N, inner), dtype=np.int8)
    bits = (np.arange(-4, 5, dtype=np.float32).view(np.uint32) >> 16).astype(np.uint16)  # BF16 of -4..4
    A = bits[Ai.astype(np.int16) + 4]
    B = bits[Bi.astype(np.int16) + 4]
    D = mcinv.mcinv_selftest_tc_gemm(A, B)
    del A
    Bf = Bi.astype(np.float32)
    for r0 in range(0, M, 2048):  # float32 products of integers < 2^24: exact
        want = Ai[r0:r0 + 2048].astype(np.float32) @ Bf.T
        assert np.array_equal(D[r0:r0 + 2048], want), r0


@pytest.mark.parametrize("complex_", [False, True])
def test_tc_block_matches_fp32_path(complex_):
    if complex_:
        csr = wl.u1_lattice((12, 11), 0.12, 0.08, seed=4)
    else:
        csr = wl.random_dominant(300, 4, 1.5, 6)
    n, K, B = csr.n, 96, 4
    R = np.arange(0, n, 2)
    S = np.arange(n // 3, n)
    hs = []
    for acc in (mcinv.MCINV_ACC_FP32_SIMT, mcinv.MCINV_ACC_BF16_TC):
        h = mcinv.create_from_csr(csr, K=K, seed=12, acc=acc, batch_cycles=B, block_rows=R, block_cols=S)
        mcinv.mcinv_burnin(h, 10)
        mcinv.mcinv_sample(h, 3 * B + 2)  # a ragged final batch too
        hs.append(h)
    m32, se32 = mcinv.mcinv_estimate(hs[0], mcinv.MCINV_EST_BLOCK)
    m16, se16 = mcinv.mcinv_estimate(hs[1], mcinv.MCINV_EST_BLOCK)
    z, w, _ = mcinv.mcinv_get_state(hs[1])
    zmax = np.abs(z).max()
    wmax = np.abs(w).max()
    bound = 2 * (2 * U_BF16 + U_BF16 ** 2) * zmax * wmax * (2 if complex_ else 1)
    assert np.abs(m16 - m32).max() <= bound
    # and the error is what BF16 rounding makes of it, far below the Monte Carlo error
    assert np.abs(m16 - m32).max() < 0.2 * np.median(np.abs(se32))


def test_tc_random256_within_3se_of_lu():
    csr = wl.random_dominant(256, 4, 1.5, 0)
    R = np.arange(256)
    h = mcinv.create_from_csr(csr, K=128, seed=0, acc=mcinv.MCINV_ACC_BF16_TC, block_rows=R, block_cols=R,
                              batch_cycles=50)
    mcinv.mcinv_burnin(h, 200)
    mcinv.mcinv_sample(h, 2000)
    m, se = mcinv.mcinv_estimate(h, mcinv.MCINV_EST_BLOCK)
    truth = np.linalg.inv(csr.to_dense())
    zs = (m - truth) / se
    assert np.mean(np.abs(zs) > 3) < 0.01
    assert 0.8 < np.sqrt(np.mean(zs ** 2)) < 1.25
