"""The allocation-free GEMM entry point gives the same result as the regular one.

lc_split_gemm_f32_noalloc is for callers that cannot let a library allocate
device memory (a process whose own pool owns the free memory, a hard memory
cap, or a path where cudaMalloc/cudaFree and their implicit device
synchronisation are not allowed).  It works out of one fixed device array, so
this test calls it twice in a row with different shapes and inputs -- a
larger problem, then a smaller one with another K, so the second call must not
see anything left over from the first -- and compares each result with
lc_split_gemm_f32, through the C ABI.  The file is named so that
pytest collects it last.
"""
import ctypes

import pytest

from paper_2506_01120_gb300 import binding
from paper_2506_01120_gb300.build import build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    build()
    return binding.lib()


def _bound(A, B):
    # the split-GEMM test's bound: three-term BF16 split plus FP32 accumulation
    K = A.shape[1]
    return (3 * 2.0 ** -16 + K * 2.0 ** -24) * (A.double().abs() @ B.double().abs().T)


def test_noalloc_matches_allocating_entry_point_twice():
    """Two calls in a row, the larger problem first: the second call has a
    different K, so its padded layout inside the shared array differs from the
    first one's, and any padding or status word left over from the first call
    would change its result.  Both entry points run the same kernels on the
    same inputs, so their outputs must be identical bit for bit; the FP64
    product bounds the error of either."""
    import torch
    g = torch.Generator(device="cpu").manual_seed(2506)
    for M, N, K in [(1000, 257, 1024), (300, 200, 500)]:
        A = torch.randn(M, K, generator=g, dtype=torch.float32)
        B = torch.randn(N, K, generator=g, dtype=torch.float32)
        Ad, Bd = A.cuda(), B.cuda()
        D0 = binding.lc_split_gemm_f32(Ad, Bd)
        D1, st = binding.lc_split_gemm_f32_noalloc(Ad, Bd)
        assert st == binding.LC_OK
        assert torch.equal(D1, D0)
        ref = A.double() @ B.double().T
        assert torch.all((D1.cpu().double() - ref).abs() <= _bound(A, B) + 1e-30)


def test_noalloc_rejects_problems_beyond_its_buffer():
    import torch
    A = torch.zeros((4096, 4096), dtype=torch.float32, device="cuda")
    B = torch.zeros((4096, 4096), dtype=torch.float32, device="cuda")
    D = torch.empty((4096, 4096), dtype=torch.float32, device="cuda")
    st = binding.lib().lc_split_gemm_f32_noalloc(A.data_ptr(), B.data_ptr(), 4096, 4096, 4096, D.data_ptr(),
                                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == binding.LC_ERR_TOO_LARGE
    assert binding.status_string(st) == "problem exceeds the fixed-size buffer"
    # extents near INT_MAX are refused by the size check alone (the padded sizes
    # would overflow 32-bit arithmetic); no memory is touched
    big = 2 ** 31 - 1
    for M, N, K in [(big, 1, 1), (1, big, 1), (1, 1, big), (big, big, big), (65536, 65536, 32)]:
        st = binding.lib().lc_split_gemm_f32_noalloc(A.data_ptr(), B.data_ptr(), M, N, K, D.data_ptr(),
                                                     ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert st == binding.LC_ERR_TOO_LARGE, (M, N, K)
    # a fitting call still works afterwards
    A = torch.randn(130, 70, device="cuda")
    B = torch.randn(90, 70, device="cuda")
    D1, st = binding.lc_split_gemm_f32_noalloc(A, B)
    assert st == binding.LC_OK
    ref = A.double() @ B.double().T
    assert torch.all((D1.double() - ref).abs() <= _bound(A.cpu(), B.cpu()).cuda() + 1e-30)
