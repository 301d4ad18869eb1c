"""Host-only checks of the C-ABI library: it builds, loads, exports every
symbol include/mcinv.h declares, and rejects malformed input on the host
before touching a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_cs_0412107_gb300 import build as libbuild
from paper_cs_0412107_gb300 import mcinv

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    libbuild.build()
    return mcinv.lib()


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "mcinv.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mcinv_[a-z_]+)\s*\(", text)))


def test_exports_every_declared_symbol(L):
    names = declared_symbols()
    assert len(names) >= 12
    for name in names:
        assert hasattr(L, name), name
    assert set(names) == set(mcinv.EXPORTS)


def test_options_layout_matches_header(L):
    opt = mcinv.mcinv_default_options()
    assert opt.K == 1024 and opt.acc == mcinv.MCINV_ACC_BF16_TC
    # C layout: 3 x 8-byte fields, 7 x 4-byte fields, 4 bytes of padding, 5 x 8-byte
    # fields, 2 x 4-byte fields
    assert ctypes.sizeof(mcinv.mcinv_options) == 104
    assert mcinv.mcinv_options.stream.offset == 56
    # mcinv_info_t: 3 x 8, 10 x 4, 5 x 8, then sweep_kernel and grid_ctas (2 x 4)
    assert ctypes.sizeof(mcinv.mcinv_info_t) == 112
    assert mcinv.mcinv_info_t.sweep_kernel.offset == 104


def _create(n, rp, col, val, **kw):
    return mcinv.mcinv_create(n, rp, col, val, stream=None, **kw)


def test_rejects_missing_diagonal(L):
    with pytest.raises(mcinv.McinvError) as e:
        _create(2, [0, 1, 2], [1, 1], [1.0, 2.0])
    assert e.value.status == 2 and "row 0" in str(e.value)


def test_rejects_zero_diagonal(L):
    with pytest.raises(mcinv.McinvError) as e:
        _create(2, [0, 1, 2], [0, 1], [1.0, 0.0])
    assert e.value.status == 2 and "row 1" in str(e.value)
    with pytest.raises(mcinv.McinvError) as e:
        _create(1, [0, 1], [0], np.array([0j]))
    assert e.value.status == 2


@pytest.mark.parametrize("rp,col,val,msg", [
    ([0, 2, 3], [1, 0, 1], [1.0, 1.0, 1.0], "strictly increasing"),
    ([0, 1, 2], [0, 2], [1.0, 1.0], "out of range"),
    ([1, 1, 2], [0, 1], [1.0, 1.0], "row_ptr"),
    ([0, 1, 2], [0, 1], [1.0, np.nan], "non-finite"),
])
def test_rejects_malformed_csr(L, rp, col, val, msg):
    with pytest.raises(mcinv.McinvError) as e:
        _create(2, rp, col, val)
    assert e.value.status == 1 and msg in str(e.value)


def test_rejects_bad_options(L):
    with pytest.raises(mcinv.McinvError) as e:
        _create(1, [0, 1], [0], [1.0], K=0)
    assert e.value.status == 1


def test_rejects_empty_and_oversized_problems(L):
    with pytest.raises(mcinv.McinvError) as e:
        _create(0, [0], [], np.zeros(0))
    assert e.value.status == 1
    n = 1 << 20  # n * K beyond the state the library addresses (4e9 elements)
    rp = np.arange(n + 1, dtype=np.int64)
    with pytest.raises(mcinv.McinvError) as e:
        _create(n, rp, np.arange(n, dtype=np.int32), np.ones(n), K=1 << 13)
    assert e.value.status == 1 and "n*K" in str(e.value)


@pytest.mark.parametrize("bp,status", [
    ([0, 2, 5], 1),         # does not end at n = 4
    ([0, 3, 2, 4], 1),      # decreasing
    ([0, 4], 2),            # D_b = [[0,1,..]]: the 4x4 block below is singular
])
def test_partition_rejections_before_any_device_work(L, bp, status):
    # rows 0-1 and 2-3: [[0, 2], [2, 0]] blocks (eigenvalues +-2: no principal root) would be
    # rejected too; here the 4x4 diagonal block is singular (rows 0 and 1 are equal)
    rp = [0, 2, 4, 5, 6]
    col = [0, 1, 0, 1, 2, 3]
    val = [1.0, 1.0, 1.0, 1.0, 1.0, 1.0]
    with pytest.raises(mcinv.McinvError) as e:
        mcinv.mcinv_create(4, rp, col, val, stream=None, partition=np.array(bp))
    assert e.value.status == status


def test_partition_block_size_limit_and_square_roots(L):
    rp, col, val = [0, 1, 2], [1, 0], [2.0, 2.0]  # [[0, 2], [2, 0]]: eigenvalues +-2
    with pytest.raises(mcinv.McinvError) as e:
        mcinv.mcinv_create(2, rp, col, val, stream=None, partition=np.array([0, 2]))
    assert e.value.status == 2 and "square root" in str(e.value)
    with pytest.raises(mcinv.McinvError) as e:  # one-row blocks need their own diagonal
        mcinv.mcinv_create(2, rp, col, val, stream=None, partition=np.array([0, 1, 2]))
    assert e.value.status == 2
    n = 9
    with pytest.raises(mcinv.McinvError) as e:  # a 9-row block exceeds the limit
        mcinv.mcinv_create(n, np.arange(n + 1), np.arange(n, dtype=np.int32), np.ones(n), stream=None,
                           partition=np.array([0, n]))
    assert e.value.status == 1


def test_colour_order_rejects_malformed_input(L):
    with pytest.raises(mcinv.McinvError) as e:
        mcinv.mcinv_create(2, [0, 1, 2], [0, 3], [1.0, 1.0], stream=None, flags=mcinv.MCINV_F_COLOR_ORDER)
    assert e.value.status == 1
