"""Failure path of the tensor-core kernels, exercised without a fault: a
bounded mbarrier wait that nothing satisfies must run out, report through the
status bits, and leave the CUDA context usable."""
import ctypes

import numpy as np
import pytest

from workloads import random_pep, start_block

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_1801_09794_gb300 as P
    P.load_library()
    return P


def test_bounded_wait_runs_out_and_reports(P):
    lib = P.load_library()
    flags = ctypes.c_int32(-1)
    # about a millisecond at GB300 clocks
    assert lib.feast_nl_selftest_bounded_wait(2_000_000, ctypes.byref(flags)) == P.FEAST_NL_OK
    assert flags.value == 16
    # the context is still usable: a small solve on the tensor-core path
    n, m0 = 64, 12
    p = random_pep(n, 2, seed=5)
    s = P.FeastNL(p, "fp32")
    s.set_contour(0.2, 0.3, 0.3, 8)
    st, info = s.solve(m0, tol=1e-10, maxit=40, X0=start_block(n, m0, 0),
                       allow=(P.FEAST_NL_ENOT_CONVERGED, P.FEAST_NL_ETOO_MANY))
    lam, X, rr = s.get_eigpairs()
    assert np.all(np.isfinite(lam))
    s.close()


def test_bounded_wait_rejects_bad_limits(P):
    lib = P.load_library()
    flags = ctypes.c_int32(0)
    assert lib.feast_nl_selftest_bounded_wait(0, ctypes.byref(flags)) == P.FEAST_NL_EINVAL
    assert lib.feast_nl_selftest_bounded_wait(1 << 40, ctypes.byref(flags)) == P.FEAST_NL_EINVAL
    assert lib.feast_nl_selftest_bounded_wait(100, None) == P.FEAST_NL_EINVAL
