"""ctypes binding of libfeast_nl.so: argument marshalling only.

Every function of include/feast_nl.h is exposed under its C name; ``FeastNL``
wraps a handle for numpy (host) or torch (device) arrays.  Nothing here
computes: every step of the method runs in the CUDA library, and importing
fails loudly when the library has not been built.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfeast_nl.so")

FEAST_NL_OK = 0
FEAST_NL_EINVAL = 1
FEAST_NL_ESINGULAR_NODE = 2
FEAST_NL_ENOT_CONVERGED = 3
FEAST_NL_ETOO_MANY = 4
FEAST_NL_ENOMEM = 5
FEAST_NL_EDEVICE = 6
FEAST_NL_EUNSUPPORTED = 7
FEAST_NL_POW, FEAST_NL_EXP = 0, 1
FEAST_NL_FP64, FEAST_NL_FP32, FEAST_NL_FP32_I8 = 0, 1, 2
FEAST_NL_GL, FEAST_NL_TRAPEZOID, FEAST_NL_GL_HALVES = 0, 1, 2
RULES = {"gl": FEAST_NL_GL, "trapezoid": FEAST_NL_TRAPEZOID, "gl_halves": FEAST_NL_GL_HALVES}
PRECISIONS = {"fp64": FEAST_NL_FP64, "fp32": FEAST_NL_FP32, "fp32_i8": FEAST_NL_FP32_I8}

# every exported symbol of include/feast_nl.h
EXPORTS = ["feast_nl_create", "feast_nl_set_contour", "feast_nl_solve", "feast_nl_get_eigpairs",
           "feast_nl_get_nodes", "feast_nl_node_solve", "feast_nl_filter_apply",
           "feast_nl_project", "feast_nl_destroy", "feast_nl_strerror", "feast_nl_last_error",
           "feast_nl_set_profiling", "feast_nl_get_profile", "feast_nl_set_iteration_graph", "feast_nl_launch_count",
           "feast_nl_gram_noalloc", "feast_nl_request_footprint", "feast_nl_server_create",
           "feast_nl_server_submit", "feast_nl_server_poll", "feast_nl_server_wait",
           "feast_nl_server_fetch", "feast_nl_server_stats", "feast_nl_server_destroy",
           "feast_nl_slices_create", "feast_nl_slices_solve", "feast_nl_slices_get_eigpairs",
           "feast_nl_slices_graph_launches", "feast_nl_slices_destroy",
           "feast_nl_set_contour_group", "feast_nl_server_set_group_limit",
           "feast_nl_selftest_bounded_wait"]
FEAST_NL_SLICES_NO_GRAPH = 1
PHASES = ["assemble", "lu", "apply", "project", "reduced", "ritz", "solve", "accum", "orth", "io"]


class feast_nl_term(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("p", ctypes.c_int32), ("tau", ctypes.c_double),
                ("scale_re", ctypes.c_double), ("scale_im", ctypes.c_double),
                ("A", ctypes.c_void_p), ("lda", ctypes.c_int64), ("on_device", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class feast_nl_info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("n_inside", ctypes.c_int32),
                ("n_converged", ctypes.c_int32), ("status", ctypes.c_int32),
                ("max_relres", ctypes.c_double), ("ms_factor", ctypes.c_double),
                ("ms_iterate", ctypes.c_double)]


class feast_nl_request(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nterms", ctypes.c_int32),
                ("terms", ctypes.POINTER(feast_nl_term)), ("precision", ctypes.c_int32),
                ("c_re", ctypes.c_double), ("c_im", ctypes.c_double), ("ra", ctypes.c_double),
                ("rb", ctypes.c_double), ("nc", ctypes.c_int32), ("rule", ctypes.c_int32),
                ("m0", ctypes.c_int32), ("tol", ctypes.c_double), ("maxit", ctypes.c_int32),
                ("seed", ctypes.c_uint64)]


class FeastError(RuntimeError):
    def __init__(self, status, where, detail):
        super().__init__(f"{where}: status {status} ({strerror(status)}): {detail}")
        self.status = status


_lib = None


def load_library(path=LIB_PATH):
    """Load the CUDA library (raises if it is missing: there is no CPU fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build() "
                           "(the library has no CPU fallback)")
    lib = ctypes.CDLL(path)
    P, I32, I64, D, U64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_uint64
    lib.feast_nl_create.argtypes = [ctypes.POINTER(P), I64, I32, ctypes.POINTER(feast_nl_term), I32, P]
    lib.feast_nl_set_contour.argtypes = [P, D, D, D, D, I32, I32]
    lib.feast_nl_solve.argtypes = [P, I32, D, I32, U64, P, ctypes.POINTER(feast_nl_info)]
    lib.feast_nl_get_eigpairs.argtypes = [P, I32, ctypes.POINTER(I32), P, P, P, I32]
    lib.feast_nl_get_nodes.argtypes = [P, P, P]
    lib.feast_nl_node_solve.argtypes = [P, I32, I32, P, P]
    lib.feast_nl_filter_apply.argtypes = [P, I32, P, P, P]
    lib.feast_nl_project.argtypes = [P, I32, P, P, ctypes.POINTER(I32)]
    lib.feast_nl_destroy.argtypes = [P]
    lib.feast_nl_destroy.restype = None
    lib.feast_nl_strerror.argtypes = [ctypes.c_int]
    lib.feast_nl_strerror.restype = ctypes.c_char_p
    lib.feast_nl_last_error.argtypes = []
    lib.feast_nl_last_error.restype = ctypes.c_char_p
    lib.feast_nl_set_profiling.argtypes = [P, I32]
    lib.feast_nl_set_iteration_graph.argtypes = [P, I32]
    lib.feast_nl_get_profile.argtypes = [P, I32, P, P]
    lib.feast_nl_launch_count.argtypes = []
    lib.feast_nl_launch_count.restype = ctypes.c_int64
    lib.feast_nl_gram_noalloc.argtypes = [I64, I32, P, I64, P, P]
    lib.feast_nl_request_footprint.argtypes = [ctypes.POINTER(feast_nl_request)]
    lib.feast_nl_request_footprint.restype = I64
    lib.feast_nl_server_create.argtypes = [ctypes.POINTER(P), I32, I64]
    lib.feast_nl_server_submit.argtypes = [P, ctypes.POINTER(feast_nl_request), ctypes.POINTER(U64)]
    lib.feast_nl_server_poll.argtypes = [P, U64, ctypes.POINTER(I32)]
    lib.feast_nl_server_wait.argtypes = [P, U64, ctypes.POINTER(feast_nl_info), ctypes.POINTER(D)]
    lib.feast_nl_server_fetch.argtypes = [P, U64, I32, ctypes.POINTER(I32), P, P, P, I32]
    lib.feast_nl_server_stats.argtypes = [P, ctypes.POINTER(I32), ctypes.POINTER(I64),
                                          ctypes.POINTER(I32)]
    lib.feast_nl_server_destroy.argtypes = [P]
    lib.feast_nl_server_set_group_limit.argtypes = [P, I32]
    lib.feast_nl_server_destroy.restype = None
    lib.feast_nl_slices_create.argtypes = [ctypes.POINTER(P), P, I32, P, P, P, P, I32, I32, P]
    lib.feast_nl_slices_solve.argtypes = [P, I32, D, I32, U64, I32, P]
    lib.feast_nl_slices_get_eigpairs.argtypes = [P, I32, I32, ctypes.POINTER(I32), P, P, P, I32]
    lib.feast_nl_slices_graph_launches.argtypes = [P]
    lib.feast_nl_slices_graph_launches.restype = I64
    lib.feast_nl_set_contour_group.argtypes = [I32, P, P, P, P, P, P, I32, P]
    lib.feast_nl_selftest_bounded_wait.argtypes = [I64, ctypes.POINTER(I32)]
    lib.feast_nl_slices_destroy.argtypes = [P]
    lib.feast_nl_slices_destroy.restype = None
    for name in EXPORTS:
        if name not in ("feast_nl_destroy", "feast_nl_strerror", "feast_nl_last_error",
                        "feast_nl_launch_count", "feast_nl_request_footprint",
                        "feast_nl_server_destroy", "feast_nl_slices_graph_launches",
                        "feast_nl_slices_destroy"):
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def strerror(status):
    return load_library().feast_nl_strerror(int(status)).decode()


def last_error():
    return load_library().feast_nl_last_error().decode()


def launch_count():
    """Kernels launched by the library in this process so far."""
    return int(load_library().feast_nl_launch_count())


def _ptr(a):
    """(address, on_device) of a numpy array or torch tensor (C-contiguous)."""
    if a is None:
        return None, False
    if hasattr(a, "data_ptr"):                      # torch tensor
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr(), a.device.type == "cuda"
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    return a.ctypes.data, False


def _c128(a):
    if a is None or hasattr(a, "data_ptr"):
        return a
    return np.ascontiguousarray(a, dtype=np.complex128)


def _check(status, where, ok=(FEAST_NL_OK,)):
    if status not in ok:
        raise FeastError(status, where, last_error())
    return status


class FeastNL:
    """One solver handle.  ``problem`` is the dict of ``workloads`` (terms with
    kind "pow"/"exp", scale, A as numpy complex128 or a CUDA torch tensor)."""

    def __init__(self, problem, precision="fp32", stream=None):
        self.lib = load_library()
        self.n = int(problem["n"])
        self._keep = []
        terms = (feast_nl_term * len(problem["terms"]))()
        for t, src in zip(terms, problem["terms"]):
            t.kind = FEAST_NL_POW if src["kind"] == "pow" else FEAST_NL_EXP
            t.p = int(src.get("p", 0))
            t.tau = float(src.get("tau", 0.0))
            sc = complex(src.get("scale", 1.0))
            t.scale_re, t.scale_im = sc.real, sc.imag
            A = _c128(src["A"])
            if A is not None:
                self._keep.append(A)
                addr, dev = _ptr(A)
                t.A = addr
                t.lda = self.n
                t.on_device = int(dev)
            else:
                t.A = None
                t.lda = self.n
                t.on_device = 0
        h = ctypes.c_void_p()
        st = None if stream is None else ctypes.c_void_p(int(stream))
        _check(self.lib.feast_nl_create(ctypes.byref(h), self.n, len(problem["terms"]), terms,
                                        PRECISIONS[precision], st), "feast_nl_create")
        self._keep = []
        self.h = h
        self.m0 = 0
        self.nc = 0

    def close(self):
        if getattr(self, "h", None):
            self.lib.feast_nl_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_contour(self, center, ra, rb, nc, rule="gl"):
        c = complex(center)
        _check(self.lib.feast_nl_set_contour(self.h, c.real, c.imag, float(ra), float(rb), int(nc),
                                             RULES[rule]), "feast_nl_set_contour")
        self.nc = int(nc)

    def solve(self, m0, tol=1e-10, maxit=50, seed=0, X0=None, allow=()):
        X0 = _c128(X0)
        addr, _ = _ptr(X0)
        info = feast_nl_info()
        st = self.lib.feast_nl_solve(self.h, int(m0), float(tol), int(maxit), int(seed),
                                     addr, ctypes.byref(info))
        _check(st, "feast_nl_solve", ok=(FEAST_NL_OK,) + tuple(allow))
        self.m0 = int(m0)
        return st, info

    def get_eigpairs(self, inside_only=False, vectors=True):
        cap = self.m0
        lam = np.zeros(2 * cap)
        rr = np.zeros(cap)
        X = np.zeros((self.n, cap), dtype=np.complex128) if vectors else None
        mo = ctypes.c_int32()
        _check(self.lib.feast_nl_get_eigpairs(self.h, cap, ctypes.byref(mo), lam.ctypes.data,
                                              X.ctypes.data if vectors else None, rr.ctypes.data,
                                              int(inside_only)), "feast_nl_get_eigpairs")
        m = mo.value
        lamc = lam[0:2 * m:2] + 1j * lam[1:2 * m:2]
        return lamc, (X[:, :m] if vectors else None), rr[:m]

    def set_profiling(self, on=True):
        _check(self.lib.feast_nl_set_profiling(self.h, int(bool(on))), "feast_nl_set_profiling")

    def set_iteration_graph(self, on=True):
        """Replay Steps 4, 5, 1-3 as one captured CUDA graph from the second iteration on."""
        _check(self.lib.feast_nl_set_iteration_graph(self.h, int(bool(on))),
               "feast_nl_set_iteration_graph")

    def get_profile(self):
        """{phase: (device ms, launches)} accumulated since set_profiling."""
        ms = np.zeros(len(PHASES))
        ln = np.zeros(len(PHASES), dtype=np.int64)
        _check(self.lib.feast_nl_get_profile(self.h, len(PHASES), ms.ctypes.data, ln.ctypes.data),
               "feast_nl_get_profile")
        return {p: (float(ms[i]), int(ln[i])) for i, p in enumerate(PHASES)}

    def get_nodes(self):
        z = np.zeros(2 * self.nc)
        w = np.zeros(2 * self.nc)
        _check(self.lib.feast_nl_get_nodes(self.h, z.ctypes.data, w.ctypes.data), "feast_nl_get_nodes")
        return z[0::2] + 1j * z[1::2], w[0::2] + 1j * w[1::2]

    def node_solve(self, j, R):
        R = _c128(R)
        Y = np.zeros_like(R)
        _check(self.lib.feast_nl_node_solve(self.h, int(j), R.shape[1], R.ctypes.data,
                                            Y.ctypes.data), "feast_nl_node_solve")
        return Y

    def filter_apply(self, X, lam):
        X = _c128(X)
        lam = np.asarray(lam, dtype=np.complex128)
        lam2 = np.ascontiguousarray(np.stack([lam.real, lam.imag], axis=1).reshape(-1))
        Q = np.zeros_like(X)
        _check(self.lib.feast_nl_filter_apply(self.h, X.shape[1], X.ctypes.data, lam2.ctypes.data,
                                              Q.ctypes.data), "feast_nl_filter_apply")
        return Q

    def project(self, Q, kmax):
        Q = _c128(Q)
        m = Q.shape[1]
        out = np.zeros((kmax + 1, m, m), dtype=np.complex128)
        k = ctypes.c_int32()
        _check(self.lib.feast_nl_project(self.h, m, Q.ctypes.data, out.ctypes.data, ctypes.byref(k)),
               "feast_nl_project")
        return out[: k.value + 1]


def _host_terms(problem, keep):
    """feast_nl_term array for host-resident coefficients (references kept in `keep`)."""
    n = int(problem["n"])
    terms = (feast_nl_term * len(problem["terms"]))()
    for t, src in zip(terms, problem["terms"]):
        t.kind = FEAST_NL_POW if src["kind"] == "pow" else FEAST_NL_EXP
        t.p = int(src.get("p", 0))
        t.tau = float(src.get("tau", 0.0))
        sc = complex(src.get("scale", 1.0))
        t.scale_re, t.scale_im = sc.real, sc.imag
        t.lda = n
        t.on_device = 0
        if src["A"] is None:
            t.A = None
        else:
            A = np.ascontiguousarray(src["A"], dtype=np.complex128)
            keep.append(A)
            t.A = A.ctypes.data
    keep.append(terms)
    return terms


def make_request(problem, center, ra, rb, nc, m0, precision="fp32", rule="gl", tol=1e-10,
                 maxit=50, seed=0, keep=None):
    keep = [] if keep is None else keep
    terms = _host_terms(problem, keep)
    r = feast_nl_request(n=int(problem["n"]), nterms=len(problem["terms"]), terms=terms,
                         precision=PRECISIONS[precision], c_re=complex(center).real,
                         c_im=complex(center).imag, ra=float(ra), rb=float(rb), nc=int(nc),
                         rule=RULES[rule], m0=int(m0), tol=float(tol), maxit=int(maxit),
                         seed=int(seed))
    keep.append(r)
    return r, keep


def request_footprint(problem, nc, m0, precision="fp32"):
    r, _ = make_request(problem, 0.0, 1.0, 1.0, nc, m0, precision)
    return int(load_library().feast_nl_request_footprint(ctypes.byref(r)))


class Server:
    """Serving loop of the library: requests run concurrently on their own handles."""

    def __init__(self, max_active=4, hbm_budget=64 << 30, group_limit=None):
        self.lib = load_library()
        s = ctypes.c_void_p()
        _check(self.lib.feast_nl_server_create(ctypes.byref(s), int(max_active), int(hbm_budget)),
               "feast_nl_server_create")
        self.s = s
        if group_limit is not None:
            _check(self.lib.feast_nl_server_set_group_limit(s, int(group_limit)),
                   "feast_nl_server_set_group_limit")
        self._keep = {}
        self._meta = {}

    def submit(self, problem, center, ra, rb, nc, m0, precision="fp32", rule="gl", tol=1e-10,
               maxit=50, seed=0):
        r, keep = make_request(problem, center, ra, rb, nc, m0, precision, rule, tol, maxit, seed)
        t = ctypes.c_uint64()
        _check(self.lib.feast_nl_server_submit(self.s, ctypes.byref(r), ctypes.byref(t)),
               "feast_nl_server_submit")
        self._keep[t.value] = keep
        self._meta[t.value] = (int(problem["n"]), int(m0))
        return t.value

    def poll(self, ticket):
        st = ctypes.c_int32()
        _check(self.lib.feast_nl_server_poll(self.s, ticket, ctypes.byref(st)), "feast_nl_server_poll")
        return st.value

    def wait(self, ticket, allow=(FEAST_NL_OK, FEAST_NL_ENOT_CONVERGED, FEAST_NL_ETOO_MANY)):
        info = feast_nl_info()
        lat = ctypes.c_double()
        st = self.lib.feast_nl_server_wait(self.s, ticket, ctypes.byref(info), ctypes.byref(lat))
        self._keep.pop(ticket, None)          # the request has run: its inputs may go
        _check(st, "feast_nl_server_wait", ok=allow)
        return st, info, lat.value

    def fetch(self, ticket, inside_only=False, vectors=True):
        n, cap = self._meta.pop(ticket)
        lam = np.zeros(2 * cap)
        rr = np.zeros(cap)
        X = np.zeros((n, cap), dtype=np.complex128) if vectors else None
        mo = ctypes.c_int32()
        self.lib.feast_nl_server_fetch(self.s, ticket, cap, ctypes.byref(mo), lam.ctypes.data,
                                       X.ctypes.data if vectors else None, rr.ctypes.data,
                                       int(inside_only))
        m = mo.value
        return lam[0:2 * m:2] + 1j * lam[1:2 * m:2], (X[:, :m] if vectors else None), rr[:m]

    def stats(self):
        mc = ctypes.c_int32()
        done = ctypes.c_int64()
        mg = ctypes.c_int32()
        _check(self.lib.feast_nl_server_stats(self.s, ctypes.byref(mc), ctypes.byref(done),
                                              ctypes.byref(mg)), "feast_nl_server_stats")
        return {"max_concurrent": mc.value, "completed": done.value, "max_group": mg.value}

    def close(self):
        if getattr(self, "s", None):
            self.lib.feast_nl_server_destroy(self.s)
            self.s = None
            self._keep.clear()

    def __del__(self):
        self.close()


class Slices:
    """Spectrum slicing: many contours of the problem of ``solver`` (a FeastNL)
    factored in one batch and iterated together."""

    def __init__(self, solver, centers, ra, rb, nc, rule="gl", stream=None):
        self.lib = load_library()
        self.solver = solver                  # keeps the handle alive
        centers = np.asarray(centers, dtype=np.complex128).reshape(-1)
        self.nd = centers.size
        cre = np.ascontiguousarray(centers.real)
        cim = np.ascontiguousarray(centers.imag)
        ra = np.ascontiguousarray(np.broadcast_to(np.asarray(ra, dtype=np.float64), (self.nd,)))
        rb = np.ascontiguousarray(np.broadcast_to(np.asarray(rb, dtype=np.float64), (self.nd,)))
        self.n = solver.n
        s = ctypes.c_void_p()
        _check(self.lib.feast_nl_slices_create(ctypes.byref(s), solver.h, self.nd, cre.ctypes.data,
                                               cim.ctypes.data, ra.ctypes.data, rb.ctypes.data,
                                               int(nc), RULES[rule],
                                               None if stream is None else ctypes.c_void_p(int(stream))),
               "feast_nl_slices_create")
        self.s = s
        self.m0 = 0

    def solve(self, m0, tol=1e-10, maxit=50, seed=0, graph=True, allow=()):
        infos = (feast_nl_info * self.nd)()
        flags = 0 if graph else FEAST_NL_SLICES_NO_GRAPH
        st = self.lib.feast_nl_slices_solve(self.s, int(m0), float(tol), int(maxit), int(seed),
                                            flags, infos)
        _check(st, "feast_nl_slices_solve", ok=(FEAST_NL_OK,) + tuple(allow))
        self.m0 = int(m0)
        return st, list(infos)

    def get_eigpairs(self, disc, inside_only=False, vectors=True):
        cap = self.m0
        lam = np.zeros(2 * cap)
        rr = np.zeros(cap)
        X = np.zeros((self.n, cap), dtype=np.complex128) if vectors else None
        mo = ctypes.c_int32()
        _check(self.lib.feast_nl_slices_get_eigpairs(self.s, int(disc), cap, ctypes.byref(mo),
                                                     lam.ctypes.data,
                                                     X.ctypes.data if vectors else None,
                                                     rr.ctypes.data, int(inside_only)),
               "feast_nl_slices_get_eigpairs")
        m = mo.value
        return lam[0:2 * m:2] + 1j * lam[1:2 * m:2], (X[:, :m] if vectors else None), rr[:m]

    def graph_launches(self):
        return int(self.lib.feast_nl_slices_graph_launches(self.s))

    def close(self):
        if getattr(self, "s", None):
            self.lib.feast_nl_slices_destroy(self.s)
            self.s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def set_contour_group(solvers, centers, ra, rb, nc, rule="gl", stream=None):
    """Sets one contour per FeastNL handle (their orders may differ) and factors
    the node matrices of all of them together (feast_nl_set_contour_group)."""
    lib = load_library()
    k = len(solvers)
    centers = np.asarray(centers, dtype=np.complex128).reshape(-1)
    cre = np.ascontiguousarray(centers.real)
    cim = np.ascontiguousarray(centers.imag)
    ra = np.ascontiguousarray(np.broadcast_to(np.asarray(ra, dtype=np.float64), (k,)))
    rb = np.ascontiguousarray(np.broadcast_to(np.asarray(rb, dtype=np.float64), (k,)))
    ncs = np.ascontiguousarray(np.broadcast_to(np.asarray(nc, dtype=np.int32), (k,)))
    hs = (ctypes.c_void_p * k)(*[s.h.value for s in solvers])
    _check(lib.feast_nl_set_contour_group(k, hs, cre.ctypes.data, cim.ctypes.data, ra.ctypes.data,
                                          rb.ctypes.data, ncs.ctypes.data, RULES[rule],
                                          None if stream is None else ctypes.c_void_p(int(stream))),
           "feast_nl_set_contour_group")
    for s_, n_ in zip(solvers, ncs):
        s_.nc = int(n_)

