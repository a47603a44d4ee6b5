"""Host-side checks of the serving loop (no GPU needed): footprint model,
lifecycle, argument validation."""
import ctypes

import numpy as np
import pytest

from workloads import closed_form_family, config2_qep


@pytest.fixture(scope="module")
def P():
    import paper_1801_09794_gb300 as P
    P.load_library()
    return P


def test_footprint_grows_with_size_and_nodes(P):
    small = P.request_footprint(config2_qep(64, 0), 8, 16, "fp32")
    big_n = P.request_footprint(config2_qep(128, 0), 8, 16, "fp32")
    more_nodes = P.request_footprint(config2_qep(64, 0), 16, 16, "fp32")
    fp64 = P.request_footprint(config2_qep(64, 0), 8, 16, "fp64")
    slices = P.request_footprint(config2_qep(64, 0), 8, 16, "fp32_i8")
    assert 0 < small < big_n and small < more_nodes and small < fp64 and small < slices
    # dominant terms: 3 dense complex128 coefficients + 16 complex64 node factors
    n = 4096
    est = 3 * 16 * n * n + 16 * 8 * n * n
    fp = P.request_footprint({"n": n, "terms": config2_qep(8, 0)["terms"]}, 16, 96, "fp32")
    assert est < fp < 1.2 * est


def test_server_lifecycle_without_requests(P):
    s = P.Server(max_active=3, hbm_budget=1 << 30)
    assert s.stats() == {"max_concurrent": 0, "completed": 0, "max_group": 0}
    s.close()


def test_server_rejects_invalid(P):
    lib = P.load_library()
    s = ctypes.c_void_p()
    assert lib.feast_nl_server_create(ctypes.byref(s), 0, 1 << 20) == P.FEAST_NL_EINVAL
    srv = P.Server(max_active=1, hbm_budget=1 << 30)
    p = closed_form_family(10, [0.1, 0.0, 1.0], [1.0, 0.1, 0.0], 2.0)
    with pytest.raises(P.FeastError):
        srv.submit(p, 0.0, 1.0, 1.0, 8, 0)          # m0 = 0
    with pytest.raises(P.FeastError):
        srv.poll(12345)                             # unknown ticket
    srv.close()
