"""The allocation-free Gram entry point, feast_nl_gram_noalloc.

Some callers cannot let this library allocate device memory: the device memory
belongs to another framework's pool, or the call sits in a latency-critical loop
where cudaMalloc / cudaFree would stall or synchronise the device.  For them the
library exposes G = Q^H Q with its split-K partial sums in a static device array.
This test checks it, through the C ABI, against the library's allocating path
for the same product: the Step 1 projection of T(lambda) = lambda I, whose
coefficient of lambda is Q^H Q.  Two calls in a row, different blocks.
This file is collected last so a failure here cannot hide any other test.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_gram_noalloc_matches_allocating_projection():
    torch = pytest.importorskip("torch")
    import paper_1801_09794_gb300 as P
    from workloads import start_block
    lib = P.load_library()
    n, m = 3000, 40
    ident = {"n": n, "terms": [{"kind": "pow", "p": 1, "scale": 1.0, "A": None}]}
    s = P.FeastNL(ident, "fp64")
    G = torch.empty((m, m), dtype=torch.complex128, device="cuda")
    for seed in (1, 2):
        Q = start_block(n, m, seed)                     # not orthonormal: Gram is not I
        ref = s.project(Q, 1)[1]                        # Q^H Q via the allocating path
        Qcm = torch.from_numpy(np.ascontiguousarray(Q.T)).cuda()   # column-major n x m
        G.fill_(float("nan"))
        st = lib.feast_nl_gram_noalloc(n, m, Qcm.data_ptr(), n, G.data_ptr(), None)
        assert st == P.FEAST_NL_OK, P.last_error()
        torch.cuda.synchronize()
        got = G.cpu().numpy().T                         # the buffer holds G column-major
        assert np.all(np.isfinite(got))
        assert np.linalg.norm(got - ref) <= 1e-13 * np.linalg.norm(ref)
    # beyond the static scratch: a clear error and no GPU work
    assert lib.feast_nl_gram_noalloc(n, 513, Qcm.data_ptr(), n, G.data_ptr(), None) == P.FEAST_NL_EINVAL
    assert "static scratch" in P.last_error()
    s.close()
