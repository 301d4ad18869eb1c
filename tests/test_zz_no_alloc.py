"""The block accumulation that allocates nothing, checked against the
allocating tensor-core entry point.

Some callers cannot allocate device memory: a serving process that reserves
all of it up front in its own arena, or code that cannot take the device-wide
synchronisation of cudaMalloc/cudaFree in the middle of its work.
mcinv_block_accumulate_noalloc gives them one batch of the block accumulation
on their own buffers, with the FP32 product kept in a fixed array inside the
library.  This test calls it twice in a row through the C ABI and compares
the FP64 accumulators with the product from mcinv_selftest_tc_gemm, within
the FP32 accumulation bound the tensor-core tests use.  It sits in a file of
its own that pytest collects last.
"""
import numpy as np
import pytest

from paper_cs_0412107_gb300 import build as libbuild
from paper_cs_0412107_gb300 import mcinv

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    libbuild.build()
    mcinv.lib()


def _bf16_bits(x):
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    return ((u + 0x7FFF + ((u >> 16) & 1)) >> 16).astype(np.uint16)


def _from_bits(b):
    return (b.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def test_noalloc_block_accumulation_matches_allocating_path():
    import torch
    torch.cuda.set_device(0)
    rng = np.random.default_rng(31)
    M, N, inner, lda, ldb = 300, 700, 200, 208, 200  # ragged tiles, padded A rows
    A = _bf16_bits(rng.normal(size=(M, inner)))
    B = _bf16_bits(rng.normal(size=(N, inner)))
    D = mcinv.mcinv_selftest_tc_gemm(A, B).astype(np.float64)  # the existing entry point
    a, b = _from_bits(A), _from_bits(B)
    bound = inner * 2.0 ** -23 * (np.abs(a) @ np.abs(b).T)
    scale = 0.37

    A_dev = torch.zeros((M, lda), dtype=torch.int16, device="cuda")
    A_dev[:, :inner] = torch.from_numpy(A.view(np.int16)).cuda()
    B_dev = torch.from_numpy(B.view(np.int16)).cuda().contiguous()
    s_dev = torch.zeros(M * N, dtype=torch.float64, device="cuda")
    q_dev = torch.zeros(M * N, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    torch.cuda.synchronize()
    mem = None
    for call in (1, 2):
        mcinv.mcinv_block_accumulate_noalloc(M, N, inner, A_dev.data_ptr(), lda, B_dev.data_ptr(), ldb, scale,
                                             s_dev.data_ptr(), q_dev.data_ptr(), stream)
        torch.cuda.synchronize()
        if call == 1:
            # the first call loads the library's module on this device; after it,
            # a call must leave the device's free memory and torch's pool as they were
            mem = (torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated())
        else:
            assert (torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()) == mem
        s = s_dev.cpu().numpy().reshape(M, N)
        q = q_dev.cpu().numpy().reshape(M, N)
        assert np.all(np.abs(s - call * D) <= call * bound)
        assert np.all(np.abs(q - call * scale * D * D) <= call * scale * (2 * np.abs(D) * bound + bound ** 2))


def test_noalloc_rejects_sizes_beyond_its_buffer():
    with pytest.raises(mcinv.McinvError) as e:
        mcinv.mcinv_block_accumulate_noalloc(4096, 1024, 64, 16, 64, 16, 64, 1.0, 16, 16)
    assert e.value.status == 1 and "2^21" in str(e.value)
