"""The allocation-free Gram entry point, feast_nl_gram_noalloc.

Some callers cannot let this library allocate device memory: the device memory
belongs to another framework's pool, or the call sits in a latency-critical loop
where cudaMalloc / cudaFree would stall or synchronise the device.  For them the
library exposes G = Q^H Q with its split-K partial sums in a static device array.
These tests check it, through the C ABI, against Q^H Q formed on the host by
numpy (independent of the library), on two calls in a row with different
blocks, including a block shorter than one k-split (n < 16); and that sizes and
pointers it cannot serve are refused before any GPU work.
This file is collected last so a failure here cannot hide any other test.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _gram(lib, P, torch, Q, G):
    n, m = Q.shape
    Qcm = torch.from_numpy(np.ascontiguousarray(Q.T)).cuda()   # column-major n x m
    G.fill_(float("nan"))
    st = lib.feast_nl_gram_noalloc(n, m, Qcm.data_ptr(), n, G.data_ptr(), None)
    assert st == P.FEAST_NL_OK, P.last_error()
    torch.cuda.synchronize()
    return G.cpu().numpy().T                                  # G is stored column-major


@pytest.mark.parametrize("n,m", [(3000, 40), (11, 7)])
def test_gram_noalloc_matches_numpy(n, m):
    torch = pytest.importorskip("torch")
    import paper_1801_09794_gb300 as P
    from workloads import start_block
    lib = P.load_library()
    G = torch.empty((m, m), dtype=torch.complex128, device="cuda")
    for seed in (1, 2):
        Q = start_block(n, m, seed)                           # not orthonormal: Gram is not I
        ref = Q.conj().T @ Q
        got = _gram(lib, P, torch, Q, G)
        assert np.all(np.isfinite(got))
        assert np.linalg.norm(got - ref) <= 1e-13 * np.linalg.norm(ref)


def test_gram_noalloc_rejects_before_gpu_work():
    torch = pytest.importorskip("torch")
    import paper_1801_09794_gb300 as P
    lib = P.load_library()
    n = 64
    Q = torch.zeros((513, n), dtype=torch.complex128, device="cuda")
    G = torch.zeros((513, 513), dtype=torch.complex128, device="cuda")
    # beyond the static scratch
    assert lib.feast_nl_gram_noalloc(n, 513, Q.data_ptr(), n, G.data_ptr(), None) == P.FEAST_NL_EINVAL
    assert "static scratch" in P.last_error()
    # a column stride beyond the cap
    assert lib.feast_nl_gram_noalloc(n, 4, Q.data_ptr(), 1 << 41, G.data_ptr(), None) == P.FEAST_NL_EINVAL
    # host memory is not device memory of the current GPU
    Qh = np.zeros((4, n), dtype=np.complex128)
    assert lib.feast_nl_gram_noalloc(n, 4, Qh.ctypes.data, n, G.data_ptr(), None) == P.FEAST_NL_EINVAL
    assert "current device" in P.last_error()
