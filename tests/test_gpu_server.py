"""The serving loop on the GPU: requests run concurrently on their own handles
give exactly the results they give alone; admission by device footprint;
results against the closed form."""
import numpy as np
import pytest

from tests.closed_forms import delay_family_eigs, family_eigs, inside_mask, match_sets
from workloads import closed_form_family, delay_family

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_1801_09794_gb300 as P
    P.load_library()
    return P


def _requests():
    out = []
    for n, target in ((300, -0.3 + 0.9j), (520, 0.2 + 1.1j), (800, -0.1 + 1.0j)):
        c, d, a = [0.4, 0.02, 1.0], [0.9, 0.01, 0.0], 2.0
        p = closed_form_family(n, c, d, a)
        lam = family_eigs(n, c, d, a)
        ctr = lam[np.argmin(np.abs(lam - target))]
        dist = np.sort(np.abs(lam - ctr))
        k = max(range(10, 15), key=lambda q: (dist[q] - dist[q - 1]) / dist[q])   # widest gap
        r = 0.5 * (dist[k - 1] + dist[k])
        out.append((p, complex(ctr), float(r), 16, 20, lam[inside_mask(lam, ctr, r, r)]))
    fam = dict(n=30, c=[-1.0, 0.3], d=[0.5, 0.1], a=2.0, tau=1.0)
    lam = delay_family_eigs(fam["n"], fam["c"], fam["d"], fam["a"], fam["tau"])
    real0 = np.sort(lam[np.abs(lam.imag) < 1e-12].real)
    ctr = complex(0.5 * (real0[10] + real0[3]))
    r = float(0.5 * (real0[10] - real0[3]) + 1e-3)
    out.append((delay_family(**fam), ctr, r, 16, 12, lam[inside_mask(lam, ctr, r, r)]))
    return out


def _run(P, reqs, max_active):
    srv = P.Server(max_active=max_active, hbm_budget=64 << 30)
    tickets = [srv.submit(p, c, r, r, nc, m0, "fp32", tol=1e-11, maxit=40, seed=7)
               for p, c, r, nc, m0, _ in reqs]
    res = []
    for t in tickets:
        st, info, lat = srv.wait(t)
        res.append((st, srv.fetch(t)))
    stats = srv.stats()
    srv.close()
    return res, stats


def test_alone_and_mixed_give_identical_results(P):
    reqs = _requests()
    alone, st1 = _run(P, reqs, 1)
    mixed, st4 = _run(P, reqs, 4)
    assert st1["max_concurrent"] == 1 and st4["max_concurrent"] >= 2
    # submitted together, the four are admitted together and factored as one group
    assert st1["max_group"] == 1 and st4["max_group"] >= 2
    for (sa, (la, Xa, ra)), (sm, (lm, Xm, rm)), req in zip(alone, mixed, reqs):
        assert sa == sm == P.FEAST_NL_OK
        assert np.array_equal(la, lm) and np.array_equal(ra, rm) and np.array_equal(Xa, Xm)
        ref = req[5]
        ins = inside_mask(la, req[1], req[2], req[2])
        assert ins.sum() == len(ref) and match_sets(la[ins], ref) < 1e-10
        assert np.all(ra[ins] <= 1e-11)


def test_admission_by_footprint(P):
    reqs = _requests()[:3]
    fp = max(P.request_footprint(p, nc, m0, "fp32") for p, _, _, nc, m0, _ in reqs)
    srv = P.Server(max_active=3, hbm_budget=int(1.2 * fp))   # room for one large request
    big = [(p, c, r, nc, m0) for p, c, r, nc, m0, _ in reqs[2:]] * 3
    tickets = [srv.submit(p, c, r, r, nc, m0, "fp32", tol=1e-11, maxit=40, seed=1)
               for p, c, r, nc, m0 in big]
    for t in tickets:
        srv.wait(t)
        srv.fetch(t, vectors=False)
    assert srv.stats() == {"max_concurrent": 1, "completed": 3, "max_group": 1}
    srv.close()
