"""The allocation-free pattern builder, called through the C ABI.

amg_poisson_pattern_noalloc serves callers that cannot allocate device memory
when they call it (an allocator of the host framework that already holds the
GPU's memory, or a loop that forbids allocation once it runs).  It must give
exactly the pattern of the allocating amg_poisson_pattern, also on the second
of two calls in a row, when its fixed scratch array still holds the first
call's contents.  This file is collected last on purpose.
"""
import ctypes

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _pattern(fn, dim, N, nnz, stream):
    ptr = torch.full((N ** dim + 1,), -7, dtype=torch.int32, device="cuda")
    col = torch.full((nnz,), -7, dtype=torch.int32, device="cuda")
    st = fn(dim, N, ctypes.c_void_p(ptr.data_ptr()), ctypes.c_void_p(col.data_ptr()), ctypes.c_void_p(stream))
    torch.cuda.current_stream().synchronize()
    return st, ptr.cpu(), col.cpu()


def test_noalloc_pattern_matches_allocating_version_on_two_calls():
    from paper_2108_02054_gb300 import amg as B
    L = B.lib()
    stream = torch.cuda.current_stream().cuda_stream
    # a large 3D grid first (many scan tiles), then a small 2D one, so the
    # second call runs over scratch that still holds the first call's sums;
    # then 170^3 cells (1,200 tiles: the tile scan carries across more than
    # one 1,024-tile chunk) over the small call's leftovers
    for dim, N in ((3, 97), (2, 45), (3, 170)):
        nnz = int(L.amg_poisson_nnz(dim, N))
        st_ref, p_ref, c_ref = _pattern(L.amg_poisson_pattern, dim, N, nnz, stream)
        st, p, c = _pattern(L.amg_poisson_pattern_noalloc, dim, N, nnz, stream)
        assert st_ref == 0 and st == 0
        assert torch.equal(p, p_ref) and torch.equal(c, c_ref)
        assert int(p[-1]) == nnz


def test_noalloc_pattern_rejects_grids_beyond_its_scratch():
    from paper_2108_02054_gb300 import amg as B
    L = B.lib()
    # 407^3 cells exceed AMG_NOALLOC_MAX_CELLS = 2^26: refused before any launch
    buf = torch.zeros(4, dtype=torch.int32, device="cuda")
    st = L.amg_poisson_pattern_noalloc(3, 407, ctypes.c_void_p(buf.data_ptr()), ctypes.c_void_p(buf.data_ptr()),
                                       None)
    assert st == B.AMG_ERR_CAPACITY
    assert torch.count_nonzero(buf) == 0
