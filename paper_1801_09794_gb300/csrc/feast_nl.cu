// C ABI of the nonlinear FEAST filter library (declared in include/feast_nl.h).
// Host-side orchestration of Algorithm 1; every numerical step runs in the
// kernels of k_dense.cu, k_lu.cu and k_reduced.cu on the handle's stream.
#include "../../include/feast_nl.h"
#include "internal.h"

#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <new>
#include <string>
#include <vector>

using namespace fnl;
typedef std::complex<double> zd;

static thread_local std::string g_last_error;
void fnl::set_last_error(const char* msg) { g_last_error = msg ? msg : ""; }

namespace {

int fail(int code, const std::string& msg) {
    g_last_error = msg;
    return code;
}
int fail_cuda(cudaError_t e, const char* what, int line) {
    g_last_error = std::string("CUDA error ") + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) +
                   ") in " + what + " at feast_nl.cu:" + std::to_string(line);
    return e == cudaErrorMemoryAllocation ? FEAST_NL_ENOMEM : FEAST_NL_EDEVICE;
}
#define CK(x)                                                                   \
    do {                                                                        \
        cudaError_t _e = (x);                                                   \
        if (_e != cudaSuccess) return fail_cuda(_e, #x, __LINE__);              \
    } while (0)
#define CKS(x)                                                                  \
    do {                                                                        \
        int _s = (x);                                                           \
        if (_s != FEAST_NL_OK) return _s;                                       \
    } while (0)

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Device memory is stream-ordered (cudaMallocAsync / cudaFreeAsync on the
// handle's stream, from the device's default pool): no allocation or release
// synchronises the device, so handles on different streams (the serving loop)
// never stall one another.  Every entry point that allocates sets the stream.
thread_local cudaStream_t g_alloc_stream = nullptr;
struct AllocScope {
    cudaStream_t prev;
    explicit AllocScope(cudaStream_t s) : prev(g_alloc_stream) { g_alloc_stream = s; }
    ~AllocScope() { g_alloc_stream = prev; }
};
void keep_pool_memory() {
    // freed blocks stay in the pool for the next handle instead of going back
    // to the driver at every synchronisation
    static std::atomic<bool> done{false};
    if (done.exchange(true)) return;
    int dev = 0;
    cudaMemPool_t pool;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t keep = (uint64_t)32 << 30;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    cudaGetLastError();
}
template <typename T>
cudaError_t dalloc(T** p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    return cudaMallocAsync((void**)p, count * sizeof(T), g_alloc_stream);
}
template <typename T>
void dfree(T*& p) {
    if (p) cudaFreeAsync(p, g_alloc_stream);
    p = nullptr;
}

// Gauss-Legendre nodes/weights on [-1, 1], ascending (Newton on P_n).
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
        double dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            if (n == 1) { p1 = z; p0 = 1.0; }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            if (n == 1) { p1 = z; p0 = 1.0; }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
        }
        double wi = 2.0 / ((1.0 - z * z) * dp * dp);
        x[i] = -z;
        x[n - 1 - i] = z;
        w[i] = wi;
        w[n - 1 - i] = wi;
    }
    if (n % 2 == 1) x[n / 2] = 0.0;
}

zd term_f_host(int kind, int p, double tau, zd scale, zd z) {
    zd v = 1.0;
    if (kind == FEAST_NL_POW) {
        for (int q = 0; q < p; ++q) v *= z;
    } else {
        v = std::exp(-tau * z);
    }
    return scale * v;
}

struct HostTerm {
    int kind, p;
    double tau;
    zd scale;
    int aidx;
    double norm;
};

}  // namespace

namespace {
// seed of the probe block of the reduced solver for non-polynomial T (the
// result does not depend on it once the probe spans the wanted eigenvectors)
constexpr uint64_t kBeynProbeSeed = 0x6265796e2d70726full;
}  // namespace


namespace {

// Quadrature nodes of nd contours (nd * nc nodes, contour-major) and the LU
// factors of T at every node.  A handle holds one contour; a spectrum-slicing
// set holds many, factored in one batch.
struct NodeSet {
    int nd = 0, nc = 0, rule = 0;
    std::vector<double> c_re, c_im, ra, rb;   // per contour
    std::vector<zd> z, w;                      // nd * nc
    double2* dz = nullptr;
    double2* dw = nullptr;
    void* dF = nullptr;             // nd * nc factors of n x n, LU precision
    int* dpiv = nullptr;
    int* dinfo = nullptr;
    int2* dGather = nullptr;        // per node and panel: row interchanges as a gather list
    int* dGcount = nullptr;
    double ms_factor = 0.0;
    bool ready = false;
};

// Subspace workspace of nd contours with m columns each; every per-contour
// block is contiguous, contour d at offset d * (block size).
struct Work {
    int nd = 0, mcap = 0, nc = 0;
    double2 *Q = nullptr, *Qt = nullptr, *X = nullptr, *R = nullptr;
    double2* W = nullptr;           // per contour: [A_0 Q | .. | A_{T-1} Q], n x T m
    void* Y = nullptr;              // per contour: nc node right-hand sides, LU precision
    double2 *G = nullptr, *Split = nullptr, *Ahat = nullptr, *Yred = nullptr, *Ycat = nullptr;
    double2 *G2 = nullptr, *Rinv = nullptr, *Lam = nullptr, *Coef = nullptr, *Fsum = nullptr;
    double *Nu = nullptr, *Rnorm = nullptr, *Relres = nullptr;
    unsigned char* Red = nullptr;   // reduced-problem workspace (bytes)
    size_t red_bytes = 0;
    unsigned char* Beyn = nullptr;  // reduced solver for non-polynomial T (bytes)
    size_t beyn_bytes = 0;
    double2* Stage = nullptr;       // n x (nd mcap) staging for layout changes
    IterStatus* Status = nullptr;   // one per contour
    int splits = 1;
    unsigned char* Qsl = nullptr;   // digit slices of Q' (all contours at once)
    double* Tau = nullptr;          // their column scales
    unsigned char* Oz = nullptr;    // digit-split workspace of the tall, thin FP64 products
};

// One contour's view of a NodeSet and a Work, with the stream its per-contour
// steps run on.
struct Disc {
    int d = 0, m = 0, nc = 0;
    cudaStream_t st = nullptr;
    bool prof = false;
    double c_re = 0, c_im = 0, ra = 1, rb = 1;
    const double2 *z = nullptr, *w = nullptr;
    double2 *Q, *Qt, *X, *R, *W, *G, *Split, *Ahat, *Yred, *Ycat, *G2, *Rinv, *Lam, *Coef, *Fsum;
    double *Nu, *Rnorm, *Relres;
    unsigned char *Red, *Beyn;
    unsigned char* Oz;              // non-null: tall, thin FP64 products on the tensor cores
    void* Y;
    IterStatus* status;
    int splits;
};

}  // namespace

struct feast_nl_handle {
    int64_t n = 0;
    int nterms = 0, nA = 0, kmax = 0, precision = 0;
    bool has_exp = false;
    cudaStream_t st = nullptr;
    bool own_stream = false;
    std::vector<HostTerm> terms;
    double2* dA = nullptr;          // nA x n x n, column-major
    TermDev* dTerms = nullptr;
    NodeSet ns;                     // the handle's contour
    Work wk;                        // its subspace workspace
    IterStatus* dStatus = nullptr;  // status of create / set_contour / stage calls
    // pageable: freeing pinned memory would synchronise the whole device
    std::unique_ptr<IterStatus> hStatus{new IterStatus()};
    // digit-split products on the tensor cores (precision FEAST_NL_FP32_I8)
    int oz_s = 0;
    unsigned char* dAsl = nullptr;  // nA x s slices of A'
    double* dSigma = nullptr;       // nA x Mpad row scales
    int* dSlot = nullptr;           // sliced index -> term index
    int nsl = 0;                    // dense terms with digit slices
    // dense terms that are diagonal (exact zeros off the diagonal): their
    // products A_t Q are diagonal scalings (term index, diagonal on the device)
    std::vector<std::pair<int, double2*>> diag_terms;
    // results of the last solve
    bool have_result = false;
    int m_last = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // optional per-phase device timing
    struct Mark { int phase; cudaEvent_t a, b; uint64_t l0, l1; };
    bool prof = false;
    bool iter_graph = true;         // feast_nl_set_iteration_graph
    std::vector<Mark> marks;
    std::vector<cudaEvent_t> pool;
    size_t pool_used = 0;
    double prof_ms[FEAST_NL_NPHASES] = {0};
    int64_t prof_launches[FEAST_NL_NPHASES] = {0};

    size_t lu_elem() const { return precision == FEAST_NL_FP64 ? sizeof(double2) : sizeof(float2); }
};

// Spectrum slicing: nd contours of one problem solved together.  All nd * nc
// node matrices are assembled and factored in one batch; every iteration runs
// the wide steps (A_t Q for all contours, the node solves of all nodes) as
// single launches and the per-contour steps on parallel streams, captured
// once per solve as a CUDA graph and replayed.
struct feast_nl_slices {
    feast_nl_handle* h = nullptr;   // the problem (not owned)
    cudaStream_t st = nullptr;
    bool own_stream = false;
    NodeSet ns;
    Work wk;
    IterStatus* dStatus = nullptr;  // factorisation status
    std::vector<cudaStream_t> side; // one per contour (at most kMaxSide)
    std::vector<cudaEvent_t> join;
    cudaEvent_t fork = nullptr, ev0 = nullptr, ev1 = nullptr;
    // results: each contour's pairs at its convergence (or at maxit)
    int m_last = 0;
    double2* dLamRes = nullptr;
    double* dRelresRes = nullptr;
    double2* dXRes = nullptr;
    int* dActive = nullptr;         // per contour: 1 while it still iterates
    std::vector<int> live;          // contours whose per-contour steps are launched
    std::vector<feast_nl_info> info;
    bool have_result = false;
    int64_t graph_launches = 0;     // kernels per replay of the iteration graph
};

namespace {

constexpr int kMaxSide = 128;
// subspaces at least this wide take the digit-split path for their tall, thin
// FP64 products (narrower ones are latency-bound either way)
constexpr int kOzMinCols = 32;

cudaEvent_t prof_event(feast_nl_handle* h) {
    if (h->pool_used == h->pool.size()) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        h->pool.push_back(e);
    }
    return h->pool[h->pool_used++];
}
// NVTX range names of the phases (host ranges around each phase's launches,
// for a timeline tool; no cost without one attached)
const char* const kPhaseNames[FEAST_NL_NPHASES] = {"assemble", "lu", "apply", "project", "reduced",
                                                  "ritz", "solve", "accum", "orth", "io"};
// Scoped device-time measurement of one phase on the handle's stream (no-op
// unless profiling is on and the caller asks for it), inside an NVTX range.
struct Phase {
    feast_nl_handle* h;
    int idx = -1;
    Phase(feast_nl_handle* hh, int phase, bool on = true) : h(hh) {
        nvtxRangePushA(kPhaseNames[phase]);
        if (!on || !h->prof) return;
        cudaEvent_t a = prof_event(h), b = prof_event(h);
        if (!a || !b) return;
        cudaEventRecord(a, h->st);
        h->marks.push_back({phase, a, b, launch_count(), 0});
        idx = (int)h->marks.size() - 1;
    }
    ~Phase() {
        nvtxRangePop();
        if (idx < 0) return;
        cudaEventRecord(h->marks[idx].b, h->st);
        h->marks[idx].l1 = launch_count();
    }
};
void prof_flush(feast_nl_handle* h) {
    if (!h->prof || h->marks.empty()) return;
    cudaStreamSynchronize(h->st);
    for (auto& mk : h->marks) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, mk.a, mk.b) == cudaSuccess) h->prof_ms[mk.phase] += ms;
        h->prof_launches[mk.phase] += (int64_t)(mk.l1 - mk.l0);
    }
    h->marks.clear();
    h->pool_used = 0;
}

size_t round_up(size_t b, size_t a) { return (b + a - 1) / a * a; }

void free_nodes(NodeSet& ns) {
    dfree(ns.dF);
    dfree(ns.dpiv); dfree(ns.dinfo); dfree(ns.dz); dfree(ns.dw);
    dfree(ns.dGather); dfree(ns.dGcount);
    ns.ready = false;
}

void free_work(Work& wk) {
    dfree(wk.Q); dfree(wk.Qt); dfree(wk.X); dfree(wk.R); dfree(wk.W); dfree(wk.Y);
    dfree(wk.G); dfree(wk.Split); dfree(wk.Ahat); dfree(wk.Yred); dfree(wk.Ycat);
    dfree(wk.G2); dfree(wk.Rinv); dfree(wk.Lam); dfree(wk.Coef); dfree(wk.Fsum);
    dfree(wk.Nu); dfree(wk.Rnorm); dfree(wk.Relres); dfree(wk.Red); dfree(wk.Beyn); dfree(wk.Stage);
    dfree(wk.Status); dfree(wk.Qsl); dfree(wk.Tau); dfree(wk.Oz);
    wk.nd = 0;
    wk.mcap = 0;
}

// Workspace for nd contours of m columns and nc nodes each.
int alloc_work(const feast_nl_handle* h, Work& wk, int nd, int nc, int m) {
    free_work(wk);
    const int64_t n = h->n;
    const int T = h->nterms;
    nc = std::max(nc, 1);
    const int64_t M = (int64_t)nd * m;
    CK(dalloc(&wk.Q, (size_t)(n * M)));
    CK(dalloc(&wk.Qt, (size_t)(n * M)));
    CK(dalloc(&wk.X, (size_t)(n * M)));
    CK(dalloc(&wk.R, (size_t)(n * M)));
    CK(dalloc(&wk.W, (size_t)(n * M * T)));
    CK(dalloc(&wk.Stage, (size_t)(n * M)));
    {
        unsigned char* y = nullptr;
        CK(dalloc(&y, (size_t)nc * n * M * h->lu_elem()));
        wk.Y = y;
    }
    // split-K so that the m x (T m) products fill the GPU
    const int tiles = ((m + 63) / 64) * ((T * m + 63) / 64);
    wk.splits = (int)std::max<int64_t>(1, std::min<int64_t>(64, std::min<int64_t>(n / 64, 304 / tiles)));
    const size_t mm = (size_t)m * m;
    CK(dalloc(&wk.G, nd * mm * T));
    CK(dalloc(&wk.Split, nd * (wk.splits * mm * T + 16)));
    CK(dalloc(&wk.Ahat, nd * (h->kmax + 1) * mm));
    CK(dalloc(&wk.Yred, nd * mm));
    CK(dalloc(&wk.Ycat, nd * mm * T));
    CK(dalloc(&wk.G2, nd * mm));
    CK(dalloc(&wk.Rinv, nd * mm));
    CK(dalloc(&wk.Lam, (size_t)M));
    CK(dalloc(&wk.Coef, (size_t)M * nc));
    CK(dalloc(&wk.Fsum, (size_t)M));
    CK(dalloc(&wk.Nu, (size_t)M));
    CK(dalloc(&wk.Rnorm, (size_t)M));
    CK(dalloc(&wk.Relres, (size_t)M));
    wk.red_bytes = round_up(reduced_work_bytes(m, std::max(h->kmax, 1)), 256);
    CK(dalloc(&wk.Red, nd * wk.red_bytes));
    wk.beyn_bytes = 0;
    if (h->has_exp && m <= beyn_max_m()) {
        wk.beyn_bytes = round_up(beyn_work_bytes(m), 256);
        CK(dalloc(&wk.Beyn, nd * wk.beyn_bytes));
    }
    CK(dalloc(&wk.Status, (size_t)nd));
    if (h->oz_s > 0) {
        const OzakiLayout L = ozaki_layout(n, (int)M, h->oz_s);
        const size_t qb = (size_t)(L.b_slice * h->oz_s) * ozaki_elem_bytes();
        CK(dalloc(&wk.Qsl, qb));
        CK(cudaMemsetAsync(wk.Qsl, 0, qb, g_alloc_stream));
        CK(dalloc(&wk.Tau, (size_t)M));
        // one contour with a subspace wide enough for the tensor cores to pay:
        // X = Q Y, T(X, Lambda) = W Ycat and Q R^{-1} as digit-split products
        // (and the projections Q^H W, split over K)
        if (nd == 1 && m >= kOzMinCols && ozaki_supported((int64_t)T * m, h->oz_s))
            CK(dalloc(&wk.Oz, std::max(ozaki_general_work_bytes(n, T * m, m, h->oz_s),
                                       ozaki_project_work_bytes(n, T * m, m))));
    }
    wk.nd = nd;
    wk.mcap = m;
    wk.nc = nc;
    return FEAST_NL_OK;
}

// Contour d's blocks when every contour has m columns.
Disc disc_view(const feast_nl_handle* h, const NodeSet& ns, const Work& wk, int d, int m,
               cudaStream_t st, bool prof) {
    const int64_t n = h->n;
    const int T = h->nterms;
    const size_t mm = (size_t)m * m;
    Disc D;
    D.d = d;
    D.m = m;
    D.nc = ns.nc;
    D.st = st;
    D.prof = prof;
    if (d < ns.nd) {
        D.c_re = ns.c_re[d]; D.c_im = ns.c_im[d]; D.ra = ns.ra[d]; D.rb = ns.rb[d];
        D.z = ns.dz + (int64_t)d * ns.nc;
        D.w = ns.dw + (int64_t)d * ns.nc;
    }
    const int64_t nm = n * m;
    D.Q = wk.Q + d * nm;
    D.Qt = wk.Qt + d * nm;
    D.X = wk.X + d * nm;
    D.R = wk.R + d * nm;
    D.W = wk.W + d * nm * T;
    D.Y = static_cast<unsigned char*>(wk.Y) + (size_t)d * wk.nc * nm * h->lu_elem();
    D.G = wk.G + d * mm * T;
    D.Split = wk.Split + d * (wk.splits * mm * T + 16);
    D.Ahat = wk.Ahat + d * (h->kmax + 1) * mm;
    D.Yred = wk.Yred + d * mm;
    D.Ycat = wk.Ycat + d * mm * T;
    D.G2 = wk.G2 + d * mm;
    D.Rinv = wk.Rinv + d * mm;
    D.Lam = wk.Lam + (int64_t)d * m;
    D.Coef = wk.Coef + (int64_t)d * m * wk.nc;
    D.Fsum = wk.Fsum + (int64_t)d * m;
    D.Nu = wk.Nu + (int64_t)d * m;
    D.Rnorm = wk.Rnorm + (int64_t)d * m;
    D.Relres = wk.Relres + (int64_t)d * m;
    D.Red = wk.Red + d * wk.red_bytes;
    D.Beyn = wk.Beyn ? wk.Beyn + d * wk.beyn_bytes : nullptr;
    D.Oz = (wk.Oz && wk.nd == 1) ? wk.Oz : nullptr;
    D.status = wk.Status + d;
    D.splits = wk.splits;
    return D;
}

int ensure_workspace(feast_nl_handle* h, int m) {
    if (m <= h->wk.mcap && h->wk.nd == 1 && h->wk.nc == std::max(h->ns.nc, 1)) return FEAST_NL_OK;
    h->have_result = false;
    return alloc_work(h, h->wk, 1, h->ns.nc, m);
}

// Copy an n x m complex128 row-major block (host or device) into column-major dst.
int load_block(const feast_nl_handle* h, cudaStream_t st, double2* stage, const void* src, int m,
               double2* dst) {
    const size_t bytes = (size_t)h->n * m * sizeof(double2);
    const double2* s = static_cast<const double2*>(src);
    if (!is_device_ptr(src)) {
        CK(cudaMemcpyAsync(stage, src, bytes, cudaMemcpyHostToDevice, st));
        s = stage;
    }
    CK(transpose_rowmajor_to_colmajor(st, h->n, m, s, m, dst, h->n));
    return FEAST_NL_OK;
}
// Copy column-major src (n x m, ld n) out as row-major with row stride ldd (host or device).
int store_block(const feast_nl_handle* h, cudaStream_t st, double2* stage, const double2* src,
                int m, void* dst, int64_t ldd) {
    if (is_device_ptr(dst)) {
        CK(transpose_colmajor_to_rowmajor(st, h->n, m, src, h->n, static_cast<double2*>(dst), ldd));
        CK(cudaStreamSynchronize(st));
        return FEAST_NL_OK;
    }
    CK(transpose_colmajor_to_rowmajor(st, h->n, m, src, h->n, stage, m));
    CK(cudaMemcpy2DAsync(dst, ldd * sizeof(double2), stage, m * sizeof(double2),
                         m * sizeof(double2), h->n, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return FEAST_NL_OK;
}

// W = [A_0 Q_d, .., A_{T-1} Q_d] for the nd contours' blocks Q_d (n x m each,
// contiguous) at once: one product over all nd m columns (identity terms copy Q).
int apply_terms(const feast_nl_handle* h, const Work& wk, int nd, int m, const double2* Q,
                double2* W, cudaStream_t st, int* err, const int* active = nullptr) {
    const int64_t n = h->n;
    const int T = h->nterms;
    const int M = nd * m;
    const double2 one = make_double2(1.0, 0.0), zero = make_double2(0.0, 0.0);
    if (h->oz_s > 0 && h->nA > 0) {
        // all sliced dense terms and all contours at once on the BF16 tensor
        // cores; diagonal terms as diagonal scalings (FP64 products)
        if (h->nsl > 0) {
            const OzakiLayout L = ozaki_layout(n, M, h->oz_s);
            CK(ozaki_split_Q(st, n, M, h->oz_s, Q, wk.Tau, wk.Qsl, L));
            CK(ozaki_gemm(st, n, M, m, T, L, h->nsl, h->dAsl, h->dSigma, wk.Qsl, wk.Tau, W, h->dSlot,
                          err, active));
        }
        for (const auto& dt : h->diag_terms) CK(diag_times(st, n, m, nd, T, dt.first, dt.second, Q, W));
        CK(copy_identity_terms(st, n, m, nd, T, h->dTerms, Q, W));
        return FEAST_NL_OK;
    }
    for (int t = 0; t < T; ++t) {
        const HostTerm& ht = h->terms[t];
        if (ht.aidx < 0) continue;
        CK(gemm<double2>(st, 0, (int)n, m, (int)n, one, h->dA + (int64_t)ht.aidx * n * n, n, 0, Q, n,
                         n * m, zero, W + (int64_t)t * n * m, n, (int64_t)T * n * m, nd));
    }
    CK(copy_identity_terms(st, n, m, nd, T, h->dTerms, Q, W));
    return FEAST_NL_OK;
}

// Q <- Q R^{-1} twice (CholQR with a small diagonal shift), columns pre-equilibrated.
// Only the product Q R^{-1} has to be exact to FP64 rounding (it must keep the
// span); the Gram matrix feeds an FP32 Cholesky, so it is formed from an FP32
// copy of Q (held in the contour's node right-hand-side buffer, free at this
// point).  D is a copy: its Q / Qt swaps stay local, and after the two passes
// the result is back in the caller's Q.
int orthonormalize(feast_nl_handle* h, Disc D) {
    Phase ph(h, FEAST_NL_PH_ORTH, D.prof);
    const int64_t n = h->n;
    const int m = D.m;
    const double2 one = make_double2(1.0, 0.0), zero = make_double2(0.0, 0.0);
    float2* Q32 = static_cast<float2*>(D.Y);
    CK(column_norms(D.st, n, m, D.Q, n, D.Nu));
    CK(ritz_scale(D.st, n, m, 0, h->dTerms, D.Lam, D.Nu, D.Q, D.Yred, D.Ycat));
    for (int pass = 0; pass < 2; ++pass) {
        CK(to_float(D.st, n * m, D.Q, Q32));
        CK(gram_f32(D.st, m, (int)n, Q32, n, D.G2, m, reinterpret_cast<float2*>(D.Split), D.splits));
        CK(chol_inverse(D.st, m, D.G2, 1e-6, D.Rinv, D.status));
        if (D.Oz)
            CK(ozaki_gemm_general(D.st, n, m, m, D.Q, n, D.Rinv, m, D.Qt, n, h->oz_s, D.Oz,
                                  &D.status->flags));
        else
            CK(gemm<double2>(D.st, 0, (int)n, m, m, one, D.Q, n, 0, D.Rinv, m, 0, zero, D.Qt, n, 0, 1));
        std::swap(D.Q, D.Qt);
    }
    return FEAST_NL_OK;
}

// Step 1's projections G = Q^H W (m x T m), W = [A_t Q]: on the BF16 tensor
// cores (digit-split product, split over K) when the contour has the
// digit-split workspace, else the FP64 split-K product.
int project_block(feast_nl_handle* h, const Disc& D) {
    const int64_t n = h->n;
    const int T = h->nterms;
    const int m = D.m;
    if (D.Oz) {
        CK(ozaki_project(D.st, n, T * m, m, D.W, n, D.Q, n, D.G, D.Oz, &D.status->flags));
        return FEAST_NL_OK;
    }
    const double2 one = make_double2(1.0, 0.0), zero = make_double2(0.0, 0.0);
    CK(gemm_splitk_d(D.st, 1, m, T * m, (int)n, one, D.Q, n, D.W, n, zero, D.G, m, D.Split,
                     D.splits));
    return FEAST_NL_OK;
}

// Rayleigh-Ritz (Steps 1-2) and the block residual (Step 3) for contour D, with
// W = [A_t Q] already formed.
int ritz_and_residual(feast_nl_handle* h, const Disc& D, double tol) {
    const int64_t n = h->n;
    const int T = h->nterms;
    const int m = D.m;
    const double2 one = make_double2(1.0, 0.0), zero = make_double2(0.0, 0.0);
    {
        Phase ph(h, FEAST_NL_PH_PROJECT, D.prof);
        CKS(project_block(h, D));
        if (!h->has_exp) CK(form_reduced(D.st, m, T, h->kmax, h->dTerms, D.G, D.Ahat));
    }
    {
        Phase ph(h, FEAST_NL_PH_REDUCED, D.prof);
        if (h->has_exp)
            CK(reduced_solve_general(D.st, m, T, h->dTerms, D.G, D.c_re, D.c_im, D.ra, D.rb,
                                     kBeynProbeSeed, D.Beyn, D.Lam, D.Yred, D.status));
        else
            CK(reduced_solve(D.st, m, h->kmax, D.Ahat, m, D.c_re, D.c_im, D.ra, D.rb, D.Red, D.Lam,
                             D.Yred, D.status));
    }
    Phase ph(h, FEAST_NL_PH_RITZ, D.prof);
    if (D.Oz)
        CK(ozaki_gemm_general(D.st, n, m, m, D.Q, n, D.Yred, m, D.X, n, h->oz_s, D.Oz,
                              &D.status->flags));
    else
        CK(gemm<double2>(D.st, 0, (int)n, m, m, one, D.Q, n, 0, D.Yred, m, 0, zero, D.X, n, 0, 1));
    CK(column_norms(D.st, n, m, D.X, n, D.Nu));
    CK(ritz_scale(D.st, n, m, T, h->dTerms, D.Lam, D.Nu, D.X, D.Yred, D.Ycat));
    if (D.Oz)
        CK(ozaki_gemm_general(D.st, n, T * m, m, D.W, n, D.Ycat, (int64_t)T * m, D.R, n, h->oz_s,
                              D.Oz, &D.status->flags));
    else
        CK(gemm<double2>(D.st, 0, (int)n, m, T * m, one, D.W, n, 0, D.Ycat, (int64_t)T * m, 0, zero,
                         D.R, n, 0, 1));
    CK(column_norms(D.st, n, m, D.R, n, D.Rnorm));
    CK(residual_summary(D.st, m, T, h->dTerms, D.Lam, D.Rnorm, D.c_re, D.c_im, D.ra, D.rb, tol,
                        D.Relres, D.status));
    return FEAST_NL_OK;
}

// Step 4, first half, for every contour at once: each contour's T(X, Lambda)
// is copied to its nodes and all nd * nc systems are solved as one batch.
int filter_solve(feast_nl_handle* h, const NodeSet& ns, const Work& wk, int nd, int m,
                 cudaStream_t st, int* err, bool prof, const int* active = nullptr) {
    Phase ph(h, FEAST_NL_PH_SOLVE, prof);
    const int64_t n = h->n;
    const int nb = nd * ns.nc;
    if (h->precision == FEAST_NL_FP64) {
        double2* Y = static_cast<double2*>(wk.Y);
        CK(broadcast_rhs<double2>(st, n, m, wk.R, nd, ns.nc, Y, n * m));
        CK(lu_solve_batched<double2>(st, n, lu_block_size<double2>(),
                                     static_cast<const double2*>(ns.dF), n * n, ns.dGather,
                                     ns.dGcount, nb, Y, n * m, m, err, 0, active, ns.nc));
    } else {
        float2* Y = static_cast<float2*>(wk.Y);
        const float2* F = static_cast<const float2*>(ns.dF);
        // tile width from the autotuner (times the candidates on Y before it is filled)
        const int bn = lu_solve_pick_bn(st, n, lu_block_size<float2>(), F, n * n, ns.dGather,
                                        ns.dGcount, nb, Y, n * m, m, err);
        CK(broadcast_rhs<float2>(st, n, m, wk.R, nd, ns.nc, Y, n * m));
        CK(lu_solve_batched<float2>(st, n, lu_block_size<float2>(), F, n * n, ns.dGather,
                                    ns.dGcount, nb, Y, n * m, m, err, bn, active, ns.nc));
    }
    return FEAST_NL_OK;
}

// Step 4, second half, for contour D: quadrature weights and accumulation into Q.
int filter_accumulate(feast_nl_handle* h, const Disc& D) {
    Phase ph(h, FEAST_NL_PH_ACCUM, D.prof);
    const int64_t n = h->n;
    const int m = D.m;
    CK(filter_coefficients(D.st, D.nc, m, D.z, D.w, D.Lam, D.Coef, D.Fsum, D.status));
    if (h->precision == FEAST_NL_FP64)
        CK(accumulate_filter<double2>(D.st, n, m, D.nc, D.X, static_cast<const double2*>(D.Y), n * m,
                                      D.Coef, D.Fsum, D.Q));
    else
        CK(accumulate_filter<float2>(D.st, n, m, D.nc, D.X, static_cast<const float2*>(D.Y), n * m,
                                     D.Coef, D.Fsum, D.Q));
    return FEAST_NL_OK;
}

// Quadrature nodes of nd contours, assembly of T at all of them and the batched
// LU factorisation.  Fails with ESINGULAR_NODE on an exact zero pivot.
int build_nodes(feast_nl_handle* h, NodeSet& ns, int nd, const double* c_re, const double* c_im,
                const double* ra, const double* rb, int nc, int rule, cudaStream_t st,
                IterStatus* dstat, bool prof, bool factor = true) {
    for (int d = 0; d < nd; ++d)
        if (!(ra[d] > 0.0) || !(rb[d] > 0.0) || !std::isfinite(c_re[d]) || !std::isfinite(c_im[d]))
            return fail(FEAST_NL_EINVAL, "contour needs finite center and ra, rb > 0");
    if (nc < 1 || nc > 1024) return fail(FEAST_NL_EINVAL, "nc must be in [1, 1024]");
    if ((int64_t)nd * nc > 65535) return fail(FEAST_NL_EINVAL, "ndisc * nc must be <= 65535");
    if (rule < FEAST_NL_GL || rule > FEAST_NL_GL_HALVES) return fail(FEAST_NL_EINVAL, "unknown rule");
    if (rule == FEAST_NL_GL_HALVES && (nc % 2)) return fail(FEAST_NL_EINVAL, "GL_HALVES needs even nc");
    const int64_t n = h->n;
    const int nb = nd * nc;
    // nodes and weights: z(theta) = c + ra cos + i rb sin, omega = w z'(theta)/(2 pi i)
    std::vector<double> th(nc), wt(nc);
    if (rule == FEAST_NL_GL) {
        std::vector<double> x, w;
        gauss_legendre(nc, x, w);
        for (int j = 0; j < nc; ++j) { th[j] = M_PI * (x[j] + 1.0); wt[j] = M_PI * w[j]; }
    } else if (rule == FEAST_NL_TRAPEZOID) {
        for (int j = 0; j < nc; ++j) { th[j] = 2.0 * M_PI * (j + 0.5) / nc; wt[j] = 2.0 * M_PI / nc; }
    } else {
        std::vector<double> x, w;
        gauss_legendre(nc / 2, x, w);
        for (int j = 0; j < nc / 2; ++j) {
            th[j] = 0.5 * M_PI * (x[j] + 1.0);
            wt[j] = 0.5 * M_PI * w[j];
            th[j + nc / 2] = th[j] + M_PI;
            wt[j + nc / 2] = wt[j];
        }
    }
    free_nodes(ns);
    ns.z.assign(nb, 0.0);
    ns.w.assign(nb, 0.0);
    ns.c_re.assign(c_re, c_re + nd);
    ns.c_im.assign(c_im, c_im + nd);
    ns.ra.assign(ra, ra + nd);
    ns.rb.assign(rb, rb + nd);
    for (int d = 0; d < nd; ++d) {
        const zd c(c_re[d], c_im[d]);
        for (int j = 0; j < nc; ++j) {
            ns.z[d * nc + j] = c + ra[d] * std::cos(th[j]) + zd(0.0, 1.0) * rb[d] * std::sin(th[j]);
            zd dz(-ra[d] * std::sin(th[j]), rb[d] * std::cos(th[j]));
            ns.w[d * nc + j] = wt[j] * dz / zd(0.0, 2.0 * M_PI);
        }
    }
    // node-matrix coefficients
    std::vector<double2> coef((size_t)std::max(h->nA, 1) * nb), diagc(nb);
    for (int j = 0; j < nb; ++j) {
        zd dsum = 0.0;
        for (int t = 0; t < h->nterms; ++t) {
            const HostTerm& ht = h->terms[t];
            zd f = term_f_host(ht.kind, ht.p, ht.tau, ht.scale, ns.z[j]);
            if (ht.aidx < 0) dsum += f;
            else coef[(size_t)ht.aidx * nb + j] = make_double2(f.real(), f.imag());
        }
        diagc[j] = make_double2(dsum.real(), dsum.imag());
    }
    double2 *dcoef = nullptr, *ddiag = nullptr;
    auto free_tmp = [&]() { dfree(dcoef); dfree(ddiag); };
    int rc = [&]() -> int {
        {
            unsigned char* f = nullptr;
            CK(dalloc(&f, (size_t)nb * n * n * h->lu_elem()));
            ns.dF = f;
        }
        CK(dalloc(&ns.dpiv, (size_t)nb * n));
        {
            const int blk = h->precision == FEAST_NL_FP64 ? lu_block_size<double2>() : lu_block_size<float2>();
            const int gs = lu_gather_stride(n, blk);
            CK(dalloc(&ns.dGather, (size_t)nb * gs));
            CK(dalloc(&ns.dGcount, (size_t)nb * (gs / 128)));
        }
        CK(dalloc(&ns.dinfo, (size_t)nb));
        CK(dalloc(&ns.dz, (size_t)nb));
        CK(dalloc(&ns.dw, (size_t)nb));
        CK(dalloc(&dcoef, coef.size()));
        CK(dalloc(&ddiag, (size_t)nb));
        ns.nd = nd;
        ns.nc = nc;
        ns.rule = rule;
        std::vector<double2> zz(nb), ww(nb);
        for (int j = 0; j < nb; ++j) {
            zz[j] = make_double2(ns.z[j].real(), ns.z[j].imag());
            ww[j] = make_double2(ns.w[j].real(), ns.w[j].imag());
        }
        CK(cudaMemcpyAsync(ns.dz, zz.data(), sizeof(double2) * nb, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(ns.dw, ww.data(), sizeof(double2) * nb, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(dcoef, coef.data(), sizeof(double2) * coef.size(), cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(ddiag, diagc.data(), sizeof(double2) * nb, cudaMemcpyHostToDevice, st));
        CK(cudaMemsetAsync(ns.dinfo, 0, sizeof(int) * nb, st));
        CK(cudaMemsetAsync(dstat, 0, sizeof(IterStatus), st));
        cudaEvent_t e0, e1;
        CK(cudaEventCreate(&e0));
        CK(cudaEventCreate(&e1));
        CK(cudaEventRecord(e0, st));
        if (h->precision == FEAST_NL_FP64) {
            double2* F = static_cast<double2*>(ns.dF);
            {
                Phase ph(h, FEAST_NL_PH_ASSEMBLE, prof);
                CK(assemble_nodes<double2>(st, n, h->nA, h->dA, dcoef, ddiag, nb, F, n * n));
            }
            Phase ph(h, FEAST_NL_PH_LU, prof);
            CK(lu_factor_batched<double2>(st, n, lu_block_size<double2>(), F, n * n, ns.dpiv, nb,
                                          ns.dinfo, ns.dGather, ns.dGcount, &dstat->flags));
        } else {
            float2* F = static_cast<float2*>(ns.dF);
            {
                Phase ph(h, FEAST_NL_PH_ASSEMBLE, prof);
                CK(assemble_nodes<float2>(st, n, h->nA, h->dA, dcoef, ddiag, nb, F, n * n));
            }
            if (factor) {
                Phase ph(h, FEAST_NL_PH_LU, prof);
                CK(lu_factor_batched<float2>(st, n, lu_block_size<float2>(), F, n * n, ns.dpiv, nb,
                                             ns.dinfo, ns.dGather, ns.dGcount, &dstat->flags));
            }
        }
        if (!factor) {                       // assembled only: a grouped factorisation follows
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return FEAST_NL_OK;
        }
        CK(cudaEventRecord(e1, st));
        std::vector<int> info(nb);
        IterStatus hs{};
        CK(cudaMemcpyAsync(info.data(), ns.dinfo, sizeof(int) * nb, cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(&hs, dstat, sizeof(IterStatus), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        float ms = 0.0f;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        ns.ms_factor = ms;
        if (prof) prof_flush(h);
        if (hs.flags & 16) return fail(FEAST_NL_EDEVICE, "tensor-core wait timed out in the node LU");
        for (int j = 0; j < nb; ++j)
            if (info[j] != 0)
                return fail(FEAST_NL_ESINGULAR_NODE,
                            "zero pivot in T(z_" + std::to_string(j) + ") at column " + std::to_string(info[j] - 1));
        return FEAST_NL_OK;
    }();
    free_tmp();
    if (rc != FEAST_NL_OK) {
        free_nodes(ns);
        ns.nd = 0;
        return rc;
    }
    ns.ready = factor;
    return FEAST_NL_OK;
}

// Copies the pairs (lam, relres, X: m columns) of one contour out to the
// caller, in Step 2's order, optionally only those strictly inside.
int copy_pairs(const feast_nl_handle* h, cudaStream_t st, double2* gather, double2* stage, int m,
               const double2* dlam, const double* drr, const double2* dX, double c_re, double c_im,
               double ra, double rb, int capacity, int32_t* m_out, double* lambda, void* X,
               double* relres, int inside_only) {
    std::vector<double2> lam(m);
    std::vector<double> rr(m);
    CK(cudaMemcpyAsync(lam.data(), dlam, sizeof(double2) * m, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(rr.data(), drr, sizeof(double) * m, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    std::vector<int> idx;
    for (int i = 0; i < m; ++i) {
        double dx = (lam[i].x - c_re) / ra, dy = (lam[i].y - c_im) / rb;
        bool ins = std::sqrt(dx * dx + dy * dy) < 1.0;
        if (!inside_only || ins) idx.push_back(i);
    }
    const int cnt = std::min<int>((int)idx.size(), capacity);
    *m_out = cnt;
    if (cnt == 0) return FEAST_NL_OK;
    std::vector<double2> lo(cnt);
    std::vector<double> ro(cnt);
    for (int q = 0; q < cnt; ++q) { lo[q] = lam[idx[q]]; ro[q] = rr[idx[q]]; }
    if (lambda) {
        if (is_device_ptr(lambda)) CK(cudaMemcpyAsync(lambda, lo.data(), sizeof(double2) * cnt, cudaMemcpyHostToDevice, st));
        else std::memcpy(lambda, lo.data(), sizeof(double2) * cnt);
    }
    if (relres) {
        if (is_device_ptr(relres)) CK(cudaMemcpyAsync(relres, ro.data(), sizeof(double) * cnt, cudaMemcpyHostToDevice, st));
        else std::memcpy(relres, ro.data(), sizeof(double) * cnt);
    }
    if (X) {
        // gather the chosen columns (column-major), then store
        for (int q = 0; q < cnt; ++q)
            CK(cudaMemcpyAsync(gather + (int64_t)q * h->n, dX + (int64_t)idx[q] * h->n,
                               sizeof(double2) * h->n, cudaMemcpyDeviceToDevice, st));
        CKS(store_block(h, st, stage, gather, cnt, X, capacity));
    }
    CK(cudaStreamSynchronize(st));
    return FEAST_NL_OK;
}

// FEAST_NL_TRACE=1 prints every iteration's kept Ritz values to stderr.
bool trace_enabled() {
    static int v = -1;
    if (v < 0) {
        const char* e = getenv("FEAST_NL_TRACE");
        v = (e && e[0] && e[0] != '0') ? 1 : 0;
    }
    return v == 1;
}

int validate_handle(feast_nl_handle* h) {
    if (!h) return fail(FEAST_NL_EINVAL, "null handle");
    return FEAST_NL_OK;
}

int check_solve_args(const feast_nl_handle* h, int m0, double tol, int maxit) {
    if (m0 < 1 || m0 > kMaxM0 || m0 > h->n) return fail(FEAST_NL_EINVAL, "m0 must be in [1, min(n, 112)]");
    if (h->has_exp && m0 > beyn_max_m())
        return fail(FEAST_NL_EINVAL, "non-polynomial T: m0 must be <= " + std::to_string(beyn_max_m()));
    if (h->kmax * m0 > 1024) return fail(FEAST_NL_EINVAL, "degree * m0 must be <= 1024");
    if (maxit < 1) return fail(FEAST_NL_EINVAL, "maxit must be >= 1");
    if (!(tol > 0.0)) return fail(FEAST_NL_EINVAL, "tol must be > 0");
    return FEAST_NL_OK;
}

// Final status of one contour from its last iteration's summary.
int contour_status(const IterStatus& s, bool converged, int m) {
    int status = converged ? FEAST_NL_OK : FEAST_NL_ENOT_CONVERGED;
    if (s.n_inside >= m) status = FEAST_NL_ETOO_MANY;
    if (s.flags & 2) status = FEAST_NL_ESINGULAR_NODE;
    if (s.flags & 16) status = FEAST_NL_EDEVICE;
    return status;
}

}  // namespace

// ============================================================================
// entry points
// ============================================================================
extern "C" {

const char* feast_nl_strerror(int status) {
    switch (status) {
        case FEAST_NL_OK: return "success";
        case FEAST_NL_EINVAL: return "invalid argument";
        case FEAST_NL_ESINGULAR_NODE: return "singular node matrix or Ritz value on a node";
        case FEAST_NL_ENOT_CONVERGED: return "not converged within maxit";
        case FEAST_NL_ETOO_MANY: return "all kept Ritz values inside the contour: increase m0";
        case FEAST_NL_ENOMEM: return "out of memory";
        case FEAST_NL_EDEVICE: return "CUDA device error";
        case FEAST_NL_EUNSUPPORTED: return "unsupported request";
        default: return "unknown status";
    }
}

const char* feast_nl_last_error(void) { return g_last_error.c_str(); }

int64_t feast_nl_launch_count(void) { return (int64_t)launch_count(); }

int feast_nl_selftest_bounded_wait(int64_t cycles, int32_t* flags_out) {
    g_last_error.clear();
    if (!flags_out || cycles < 1 || cycles > ((int64_t)1 << 32))
        return fail(FEAST_NL_EINVAL, "need flags_out and 1 <= cycles <= 2^32");
    cudaStream_t st = nullptr;
    CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    int rc = [&]() -> int {
        AllocScope as(st);
        int* d = nullptr;
        CK(dalloc(&d, 1));
        CK(cudaMemsetAsync(d, 0, sizeof(int), st));
        CK(bounded_wait_probe(st, (long long)cycles, d));
        int h = 0;
        CK(cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        dfree(d);
        *flags_out = h;
        return FEAST_NL_OK;
    }();
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
    return rc;
}

int feast_nl_set_iteration_graph(feast_nl_handle* h, int32_t on) {
    CKS(validate_handle(h));
    h->iter_graph = on != 0;
    return FEAST_NL_OK;
}

int feast_nl_set_profiling(feast_nl_handle* h, int32_t on) {
    CKS(validate_handle(h));
    h->prof = on != 0;
    h->marks.clear();
    h->pool_used = 0;
    for (int i = 0; i < FEAST_NL_NPHASES; ++i) { h->prof_ms[i] = 0.0; h->prof_launches[i] = 0; }
    return FEAST_NL_OK;
}

int feast_nl_get_profile(feast_nl_handle* h, int32_t nphases, double* ms, int64_t* launches) {
    CKS(validate_handle(h));
    if (nphases < 0) return fail(FEAST_NL_EINVAL, "nphases < 0");
    prof_flush(h);
    for (int i = 0; i < nphases && i < FEAST_NL_NPHASES; ++i) {
        if (ms) ms[i] = h->prof_ms[i];
        if (launches) launches[i] = h->prof_launches[i];
    }
    return FEAST_NL_OK;
}

void feast_nl_destroy(feast_nl_handle* h) {
    if (!h) return;
    AllocScope as(h->st);
    if (h->st) cudaStreamSynchronize(h->st);
    free_work(h->wk);
    free_nodes(h->ns);
    dfree(h->dA);
    dfree(h->dAsl);
    dfree(h->dSigma);
    dfree(h->dSlot);
    for (auto& dt : h->diag_terms) dfree(dt.second);
    h->diag_terms.clear();
    dfree(h->dTerms);
    dfree(h->dStatus);
    for (cudaEvent_t e : h->pool) cudaEventDestroy(e);
    if (h->ev0) cudaEventDestroy(h->ev0);
    if (h->ev1) cudaEventDestroy(h->ev1);
    if (h->own_stream && h->st) {
        cudaStreamSynchronize(h->st);
        cudaStreamDestroy(h->st);
    }
    delete h;
}

int feast_nl_create(feast_nl_handle** out, int64_t n, int32_t nterms, const feast_nl_term* terms,
                    int32_t precision, void* stream) {
    g_last_error.clear();
    if (!out) return fail(FEAST_NL_EINVAL, "out handle pointer is NULL");
    *out = nullptr;
    if (n < 1 || n > 65536) return fail(FEAST_NL_EINVAL, "n must be in [1, 65536]");
    if (nterms < 1 || nterms > kMaxTerms) return fail(FEAST_NL_EINVAL, "nterms must be in [1, 16]");
    if (!terms) return fail(FEAST_NL_EINVAL, "terms is NULL");
    if (precision != FEAST_NL_FP64 && precision != FEAST_NL_FP32 && precision != FEAST_NL_FP32_I8)
        return fail(FEAST_NL_EINVAL, "unknown precision");
    feast_nl_handle* h = new (std::nothrow) feast_nl_handle();
    if (!h) return fail(FEAST_NL_ENOMEM, "host allocation failed");
    h->n = n;
    h->nterms = nterms;
    h->precision = precision;
    for (int t = 0; t < nterms; ++t) {
        const feast_nl_term& tt = terms[t];
        if (tt.kind != FEAST_NL_POW && tt.kind != FEAST_NL_EXP) {
            delete h;
            return fail(FEAST_NL_EINVAL, "term kind must be POW or EXP");
        }
        if (tt.kind == FEAST_NL_POW && (tt.p < 0 || tt.p > kMaxPow)) {
            delete h;
            return fail(FEAST_NL_EINVAL, "power must be in [0, 8]");
        }
        if (tt.A && tt.lda < n) {
            delete h;
            return fail(FEAST_NL_EINVAL, "lda < n");
        }
        HostTerm ht;
        ht.kind = tt.kind;
        ht.p = tt.kind == FEAST_NL_POW ? tt.p : 0;
        ht.tau = tt.tau;
        ht.scale = zd(tt.scale_re, tt.scale_im);
        ht.aidx = tt.A ? h->nA++ : -1;
        ht.norm = 1.0;
        if (tt.kind == FEAST_NL_EXP) h->has_exp = true;
        else h->kmax = std::max(h->kmax, ht.p);
        h->terms.push_back(ht);
    }
    if (h->kmax < 1 && !h->has_exp) {
        delete h;
        return fail(FEAST_NL_EINVAL, "T(lambda) must depend on lambda");
    }
    auto cleanup = [&](int s) { feast_nl_destroy(h); return s; };
    cudaError_t e;
    if (stream) {
        h->st = static_cast<cudaStream_t>(stream);
    } else {
        e = cudaStreamCreateWithFlags(&h->st, cudaStreamNonBlocking);
        if (e != cudaSuccess) return cleanup(fail_cuda(e, "cudaStreamCreate", __LINE__));
        h->own_stream = true;
    }
    keep_pool_memory();
    AllocScope as(h->st);
    if ((e = cudaEventCreate(&h->ev0)) != cudaSuccess || (e = cudaEventCreate(&h->ev1)) != cudaSuccess)
        return cleanup(fail_cuda(e, "cudaEventCreate", __LINE__));
    if ((e = dalloc(&h->dA, (size_t)h->nA * n * n)) != cudaSuccess ||
        (e = dalloc(&h->dTerms, (size_t)nterms)) != cudaSuccess ||
        (e = dalloc(&h->dStatus, 1)) != cudaSuccess)
        return cleanup(fail_cuda(e, "allocation", __LINE__));
    if (precision == FEAST_NL_FP32_I8 && h->nA > 0 && ozaki_supported(n, kOzakiSlices)) {
        h->oz_s = kOzakiSlices;
        const OzakiLayout L = ozaki_layout(n, 1, h->oz_s);
        if ((e = dalloc(&h->dAsl, (size_t)(L.a_term * h->nA) * ozaki_elem_bytes())) != cudaSuccess ||
            (e = dalloc(&h->dSigma, (size_t)(L.Mpad * h->nA))) != cudaSuccess ||
            (e = dalloc(&h->dSlot, (size_t)h->nA)) != cudaSuccess)
            return cleanup(fail_cuda(e, "allocation of digit slices", __LINE__));
    }
    // copy the coefficients in, transposed to column-major
    double2* stage = nullptr;
    double2 *v = nullptr, *u = nullptr, *gw = nullptr;
    double* nrm = nullptr;
    int* dflag = nullptr;
    std::vector<int> slot;                    // sliced index -> term index
    auto free_tmp = [&]() { dfree(stage); dfree(v); dfree(u); dfree(gw); dfree(nrm); dfree(dflag); };
    bool need_stage = false;
    for (int t = 0; t < nterms; ++t)
        if (terms[t].A && !terms[t].on_device) need_stage = true;
    if (need_stage && (e = dalloc(&stage, (size_t)n * n)) != cudaSuccess) {
        free_tmp();
        return cleanup(fail_cuda(e, "staging allocation", __LINE__));
    }
    if ((e = dalloc(&v, (size_t)n)) != cudaSuccess || (e = dalloc(&u, (size_t)n)) != cudaSuccess ||
        (e = dalloc(&gw, (size_t)n * 32)) != cudaSuccess || (e = dalloc(&nrm, 2)) != cudaSuccess ||
        (e = dalloc(&dflag, 1)) != cudaSuccess) {
        free_tmp();
        return cleanup(fail_cuda(e, "allocation", __LINE__));
    }
    for (int t = 0; t < nterms; ++t) {
        const feast_nl_term& tt = terms[t];
        if (!tt.A) continue;
        double2* dst = h->dA + (int64_t)h->terms[t].aidx * n * n;
        const double2* src = static_cast<const double2*>(tt.A);
        if (!tt.on_device) {
            e = cudaMemcpy2DAsync(stage, n * sizeof(double2), tt.A, tt.lda * sizeof(double2),
                                  n * sizeof(double2), n, cudaMemcpyHostToDevice, h->st);
            if (e != cudaSuccess) { free_tmp(); return cleanup(fail_cuda(e, "copy of A", __LINE__)); }
            e = transpose_rowmajor_to_colmajor(h->st, n, n, stage, n, dst, n);
        } else {
            e = transpose_rowmajor_to_colmajor(h->st, n, n, src, tt.lda, dst, n);
        }
        if (e != cudaSuccess) { free_tmp(); return cleanup(fail_cuda(e, "transpose of A", __LINE__)); }
        if (h->oz_s > 0) {
            // a diagonal term's product A_t Q is a diagonal scaling: no slices
            int hflag = 0;
            e = cudaMemsetAsync(dflag, 0, sizeof(int), h->st);
            if (e == cudaSuccess) e = offdiag_nonzero(h->st, n, dst, n, dflag);
            if (e == cudaSuccess) e = cudaMemcpyAsync(&hflag, dflag, sizeof(int), cudaMemcpyDeviceToHost, h->st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
            if (e != cudaSuccess) { free_tmp(); return cleanup(fail_cuda(e, "diagonal test", __LINE__)); }
            if (!hflag) {
                double2* dg = nullptr;
                if ((e = dalloc(&dg, (size_t)n)) == cudaSuccess) {
                    h->diag_terms.push_back({t, dg});
                    e = extract_diagonal(h->st, n, dst, n, dg);
                }
                if (e != cudaSuccess) { free_tmp(); return cleanup(fail_cuda(e, "diagonal of A", __LINE__)); }
            } else {
                const OzakiLayout L = ozaki_layout(n, 1, h->oz_s);
                const int a = h->nsl++;
                slot.push_back(t);
                e = ozaki_split_A(h->st, n, h->oz_s, dst, h->dSigma + (int64_t)a * L.Mpad,
                                  h->dAsl + (int64_t)a * L.a_term * ozaki_elem_bytes(), L);
                if (e != cudaSuccess) { free_tmp(); return cleanup(fail_cuda(e, "digit split of A", __LINE__)); }
            }
        }
        if (!tt.on_device) {
            // the staging buffer is reused by the next term
            e = cudaStreamSynchronize(h->st);
            if (e != cudaSuccess) { free_tmp(); return cleanup(fail_cuda(e, "sync", __LINE__)); }
        }
        // ||A||_2 by 30 power steps on A^H A from ones/sqrt(n)
        e = fill_ones(h->st, n, v);
        if (e == cudaSuccess) e = normalize_vec(h->st, n, v, nrm);
        for (int it = 0; it < 30 && e == cudaSuccess; ++it) {
            e = gemv_n(h->st, n, dst, v, u, gw);
            if (e == cudaSuccess) e = gemv_c(h->st, n, dst, u, v);
            if (e == cudaSuccess) e = normalize_vec(h->st, n, v, nrm);
        }
        double s = 0.0;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&s, nrm, sizeof(double), cudaMemcpyDeviceToHost, h->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
        if (e != cudaSuccess) { free_tmp(); return cleanup(fail_cuda(e, "norm estimate", __LINE__)); }
        h->terms[t].norm = std::sqrt(s);
    }
    free_tmp();
    if (h->oz_s > 0 && !slot.empty()) {
        e = cudaMemcpyAsync(h->dSlot, slot.data(), sizeof(int) * slot.size(), cudaMemcpyHostToDevice,
                            h->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
        if (e != cudaSuccess) return cleanup(fail_cuda(e, "copy of the slice slots", __LINE__));
    }
    std::vector<TermDev> td(nterms);
    for (int t = 0; t < nterms; ++t) {
        const HostTerm& ht = h->terms[t];
        td[t].kind = ht.kind;
        td[t].p = ht.p;
        td[t].tau = ht.tau;
        td[t].scale = make_double2(ht.scale.real(), ht.scale.imag());
        td[t].norm = ht.norm;
        td[t].aidx = ht.aidx;
        td[t].pad = 0;
    }
    e = cudaMemcpyAsync(h->dTerms, td.data(), sizeof(TermDev) * nterms, cudaMemcpyHostToDevice, h->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
    if (e != cudaSuccess) return cleanup(fail_cuda(e, "term upload", __LINE__));
    *out = h;
    return FEAST_NL_OK;
}

int feast_nl_set_contour(feast_nl_handle* h, double c_re, double c_im, double ra, double rb,
                         int32_t nc, int32_t rule) {
    g_last_error.clear();
    CKS(validate_handle(h));
    AllocScope as(h->st);
    h->have_result = false;
    free_work(h->wk);
    return build_nodes(h, h->ns, 1, &c_re, &c_im, &ra, &rb, nc, rule, h->st, h->dStatus, true);
}

int feast_nl_set_contour_group(int32_t count, feast_nl_handle* const* hs, const double* c_re,
                               const double* c_im, const double* ra, const double* rb,
                               const int32_t* nc, int32_t rule, void* stream) {
    g_last_error.clear();
    if (count < 1 || count > 4096 || !hs || !c_re || !c_im || !ra || !rb || !nc)
        return fail(FEAST_NL_EINVAL, "count in [1, 4096] and non-NULL arrays required");
    int64_t nodes_total = 0;
    for (int i = 0; i < count; ++i) {
        feast_nl_handle* h = hs[i];
        if (!h) return fail(FEAST_NL_EINVAL, "NULL handle in the group");
        for (int j = 0; j < i; ++j)
            if (hs[j] == h) return fail(FEAST_NL_EINVAL, "a handle appears twice in the group");
        if (h->precision == FEAST_NL_FP64)
            return fail(FEAST_NL_EINVAL, "grouped factorisation needs complex64 factors (FP32 precisions)");
        if (h->n > 4096) return fail(FEAST_NL_EINVAL, "grouped factorisation needs n <= 4096");
        if (nc[i] < 1 || nc[i] > 1024) return fail(FEAST_NL_EINVAL, "nc must be in [1, 1024]");
        nodes_total += nc[i];
    }
    if (nodes_total > 65535) return fail(FEAST_NL_EINVAL, "more than 65535 nodes in the group");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    bool own = false;
    if (!st) {
        CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        own = true;
    }
    int rc = [&]() -> int {
        AllocScope as(st);
        LuNode* dnodes = nullptr;
        IterStatus* dstat = nullptr;
        std::vector<LuNode> nodes;
        std::vector<int64_t> ns_n;
        // every handle's earlier work is finished before its buffers are replaced
        for (int i = 0; i < count; ++i) CK(cudaStreamSynchronize(hs[i]->st));
        CK(dalloc(&dstat, 1));
        CK(cudaMemsetAsync(dstat, 0, sizeof(IterStatus), st));
        for (int i = 0; i < count; ++i) {
            feast_nl_handle* h = hs[i];
            h->have_result = false;
            free_work(h->wk);
            int r = build_nodes(h, h->ns, 1, &c_re[i], &c_im[i], &ra[i], &rb[i], nc[i], rule, st,
                                dstat, false, false);
            if (r != FEAST_NL_OK) { dfree(dstat); return r; }
            const int gs = lu_gather_stride(h->n, lu_block_size<float2>());
            for (int j = 0; j < nc[i]; ++j) {
                LuNode d;
                d.F = static_cast<float2*>(h->ns.dF) + (int64_t)j * h->n * h->n;
                d.piv = h->ns.dpiv + (int64_t)j * h->n;
                d.info = h->ns.dinfo + j;
                d.gather = h->ns.dGather + (int64_t)j * gs;
                d.gcount = h->ns.dGcount + (int64_t)j * (gs / 128);
                d.n = h->n;
                nodes.push_back(d);
                ns_n.push_back(h->n);
            }
        }
        const int nb_nodes = (int)nodes.size();
        CK(dalloc(&dnodes, (size_t)nb_nodes));
        CK(cudaMemcpyAsync(dnodes, nodes.data(), sizeof(LuNode) * nb_nodes, cudaMemcpyHostToDevice, st));
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        CK(cudaEventCreate(&e0));
        CK(cudaEventCreate(&e1));
        CK(cudaEventRecord(e0, st));
        CK(lu_factor_grouped(st, dnodes, ns_n.data(), nb_nodes, lu_block_size<float2>(), &dstat->flags));
        CK(cudaEventRecord(e1, st));
        IterStatus hst{};
        CK(cudaMemcpyAsync(&hst, dstat, sizeof(IterStatus), cudaMemcpyDeviceToHost, st));
        std::vector<std::vector<int>> infos(count);
        for (int i = 0; i < count; ++i) {
            infos[i].resize(nc[i]);
            CK(cudaMemcpyAsync(infos[i].data(), hs[i]->ns.dinfo, sizeof(int) * nc[i],
                               cudaMemcpyDeviceToHost, st));
        }
        CK(cudaStreamSynchronize(st));
        float ms = 0.0f;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        dfree(dnodes);
        dfree(dstat);
        if (hst.flags & 16) return fail(FEAST_NL_EDEVICE, "tensor-core wait timed out in the node LU");
        for (int i = 0; i < count; ++i)
            for (int j = 0; j < nc[i]; ++j)
                if (infos[i][j] != 0)
                    return fail(FEAST_NL_ESINGULAR_NODE, "zero pivot in node " + std::to_string(j) +
                                                             " of group member " + std::to_string(i));
        for (int i = 0; i < count; ++i) {
            hs[i]->ns.ms_factor = ms;
            hs[i]->ns.ready = true;
        }
        return FEAST_NL_OK;
    }();
    if (own) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    return rc;
}

int feast_nl_solve(feast_nl_handle* h, int32_t m0, double tol, int32_t maxit, uint64_t seed,
                   const void* X0, feast_nl_info* info) {
    g_last_error.clear();
    CKS(validate_handle(h));
    AllocScope as(h->st);
    if (info) std::memset(info, 0, sizeof(*info));
    if (!h->ns.ready) return fail(FEAST_NL_EINVAL, "set_contour must succeed before solve");
    CKS(check_solve_args(h, m0, tol, maxit));
    CKS(ensure_workspace(h, m0));
    h->have_result = false;
    const int m = m0;
    const Disc D = disc_view(h, h->ns, h->wk, 0, m, h->st, true);
    CK(cudaMemsetAsync(D.status, 0, sizeof(IterStatus), h->st));
    CK(cudaEventRecord(h->ev0, h->st));
    {
        Phase ph(h, FEAST_NL_PH_IO);
        if (X0) CKS(load_block(h, h->st, h->wk.Stage, X0, m, D.Q));
        else CK(random_block(h->st, h->n, m, seed, D.Q));
    }
    CKS(orthonormalize(h, D));                                  // Step 0
    int it = 0;
    bool converged = false;
    IterStatus stt{};
    // Steps 4, 5 and 1-3 of the next iteration, as launched eagerly
    auto filter_then_ritz = [&]() -> int {
        CKS(filter_solve(h, h->ns, h->wk, 1, m, h->st, &D.status->flags, true));   // Step 4
        CKS(filter_accumulate(h, D));
        CKS(orthonormalize(h, D));                              // Step 5
        {
            Phase ph(h, FEAST_NL_PH_APPLY);
            CKS(apply_terms(h, h->wk, 1, m, D.Q, D.W, h->st, &D.status->flags));
        }
        return ritz_and_residual(h, D, tol);                    // Steps 1-3
    };
    // ... or as one captured graph, replayed (not with per-phase events or the trace)
    const bool use_graph = h->iter_graph && !h->prof && !trace_enabled();
    cudaGraphExec_t exec = nullptr;
    int64_t per_iter = 0;
    struct ExecGuard {
        cudaGraphExec_t* e;
        ~ExecGuard() { if (*e) cudaGraphExecDestroy(*e); }
    } exec_guard{&exec};
    auto capture = [&]() -> int {
        if (h->precision != FEAST_NL_FP64)      // tune the node solves before the capture
            lu_solve_pick_bn(h->st, h->n, lu_block_size<float2>(), static_cast<const float2*>(h->ns.dF),
                             h->n * h->n, h->ns.dGather, h->ns.dGcount, h->ns.nc,
                             static_cast<float2*>(h->wk.Y), h->n * m, m, &D.status->flags);
        cudaGraph_t graph = nullptr;
        const uint64_t l0 = launch_count();
        CK(cudaStreamBeginCapture(h->st, cudaStreamCaptureModeThreadLocal));
        const int rc2 = filter_then_ritz();
        const cudaError_t ec = cudaStreamEndCapture(h->st, &graph);
        if (rc2 != FEAST_NL_OK) { if (graph) cudaGraphDestroy(graph); return rc2; }
        CK(ec);
        per_iter = (int64_t)(launch_count() - l0);
        note_launch(-(int)per_iter);          // captured, not launched: counted at each replay
        const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        CK(ei);
        return FEAST_NL_OK;
    };
    for (it = 1; it <= maxit; ++it) {
        if (it == 1) {
            {
                Phase ph(h, FEAST_NL_PH_APPLY);
                CKS(apply_terms(h, h->wk, 1, m, D.Q, D.W, h->st, &D.status->flags));
            }
            CKS(ritz_and_residual(h, D, tol));                  // Steps 1-3
        } else if (use_graph) {
            if (!exec) CKS(capture());
            CK(cudaGraphLaunch(exec, h->st));
            note_launch((int)per_iter);       // the graph's kernels count as this library's launches
        } else {
            CKS(filter_then_ritz());
        }
        CK(cudaMemcpyAsync(h->hStatus.get(), D.status, sizeof(IterStatus), cudaMemcpyDeviceToHost, h->st));
        CK(cudaStreamSynchronize(h->st));
        stt = *h->hStatus;
        if (trace_enabled()) {
            std::vector<double2> lam(m);
            std::vector<double> rr(m);
            cudaMemcpyAsync(lam.data(), D.Lam, sizeof(double2) * m, cudaMemcpyDeviceToHost, h->st);
            cudaMemcpyAsync(rr.data(), D.Relres, sizeof(double) * m, cudaMemcpyDeviceToHost, h->st);
            cudaStreamSynchronize(h->st);
            fprintf(stderr, "[feast_nl] it %d inside %d conv %d max_relres %.3e flags %d qr_sweeps %d\n",
                    it, stt.n_inside, stt.n_conv, stt.max_relres, stt.flags, stt.qr_sweeps);
            for (int i = 0; i < m; ++i)
                fprintf(stderr, "    %2d  % .12e % .12e  relres %.3e\n", i, lam[i].x, lam[i].y, rr[i]);
        }
        // a timed-out tensor-core wait (bit 4) or a Ritz value on a node (bit 1)
        // leaves the iterate invalid: stop now rather than at maxit
        if (stt.flags & (16 | 2)) break;
        if (it > 1 && stt.n_conv == stt.n_inside) { converged = true; break; }
        if (it == maxit) break;
    }
    CK(cudaEventRecord(h->ev1, h->st));
    CK(cudaEventSynchronize(h->ev1));
    float ms = 0.0f;
    CK(cudaEventElapsedTime(&ms, h->ev0, h->ev1));
    prof_flush(h);
    h->have_result = true;
    h->m_last = m;
    const int status = contour_status(stt, converged, m);
    if (info) {
        info->iters = std::min(it, maxit);
        info->n_inside = stt.n_inside;
        info->n_converged = stt.n_conv;
        info->status = status;
        info->max_relres = stt.max_relres;
        info->ms_factor = h->ns.ms_factor;
        info->ms_iterate = ms;
    }
    if (status == FEAST_NL_ENOT_CONVERGED) g_last_error = "maxit reached";
    if (status == FEAST_NL_ETOO_MANY) g_last_error = "all kept Ritz values are inside the contour";
    if (status == FEAST_NL_ESINGULAR_NODE) g_last_error = "a Ritz value coincides with a node";
    return status;
}

int feast_nl_get_eigpairs(feast_nl_handle* h, int32_t capacity, int32_t* m_out, double* lambda,
                          void* X, double* relres, int32_t inside_only) {
    g_last_error.clear();
    CKS(validate_handle(h));
    AllocScope as(h->st);
    if (!h->have_result) return fail(FEAST_NL_EINVAL, "no solve result");
    if (capacity < 0 || !m_out) return fail(FEAST_NL_EINVAL, "bad capacity or m_out");
    const Disc D = disc_view(h, h->ns, h->wk, 0, h->m_last, h->st, false);
    return copy_pairs(h, h->st, h->wk.Qt, h->wk.Stage, h->m_last, D.Lam, D.Relres, D.X, D.c_re,
                      D.c_im, D.ra, D.rb, capacity, m_out, lambda, X, relres, inside_only);
}

int feast_nl_get_nodes(feast_nl_handle* h, double* z, double* omega) {
    g_last_error.clear();
    CKS(validate_handle(h));
    if (!h->ns.ready) return fail(FEAST_NL_EINVAL, "no contour");
    for (int j = 0; j < h->ns.nc; ++j) {
        if (z) { z[2 * j] = h->ns.z[j].real(); z[2 * j + 1] = h->ns.z[j].imag(); }
        if (omega) { omega[2 * j] = h->ns.w[j].real(); omega[2 * j + 1] = h->ns.w[j].imag(); }
    }
    return FEAST_NL_OK;
}

int feast_nl_node_solve(feast_nl_handle* h, int32_t j, int32_t m, const void* R, void* Y) {
    g_last_error.clear();
    CKS(validate_handle(h));
    AllocScope as(h->st);
    if (!h->ns.ready) return fail(FEAST_NL_EINVAL, "no contour");
    if (j < 0 || j >= h->ns.nc || m < 1 || m > kMaxM0 || !R || !Y) return fail(FEAST_NL_EINVAL, "bad node, m or pointer");
    CKS(ensure_workspace(h, std::max(m, h->wk.mcap)));
    h->have_result = false;
    const int64_t n = h->n;
    const Work& wk = h->wk;
    CKS(load_block(h, h->st, wk.Stage, R, m, wk.R));
    CK(cudaMemsetAsync(h->dStatus, 0, sizeof(IterStatus), h->st));
    const NodeSet& ns = h->ns;
    if (h->precision == FEAST_NL_FP64) {
        double2* Yb = static_cast<double2*>(wk.Y);
        CK(broadcast_rhs<double2>(h->st, n, m, wk.R, 1, 1, Yb, n * m));
        const int gs = lu_gather_stride(n, lu_block_size<double2>());
        CK(lu_solve_batched<double2>(h->st, n, lu_block_size<double2>(),
                                     static_cast<const double2*>(ns.dF) + (int64_t)j * n * n, n * n,
                                     ns.dGather + (int64_t)j * gs, ns.dGcount + (int64_t)j * (gs / 128),
                                     1, Yb, n * m, m, &h->dStatus->flags));
        CK(to_double<double2>(h->st, n * m, Yb, wk.X));
    } else {
        float2* Yb = static_cast<float2*>(wk.Y);
        CK(broadcast_rhs<float2>(h->st, n, m, wk.R, 1, 1, Yb, n * m));
        const int gs = lu_gather_stride(n, lu_block_size<float2>());
        CK(lu_solve_batched<float2>(h->st, n, lu_block_size<float2>(),
                                    static_cast<const float2*>(ns.dF) + (int64_t)j * n * n, n * n,
                                    ns.dGather + (int64_t)j * gs, ns.dGcount + (int64_t)j * (gs / 128),
                                    1, Yb, n * m, m, &h->dStatus->flags));
        CK(to_double<float2>(h->st, n * m, Yb, wk.X));
    }
    CK(cudaMemcpyAsync(h->hStatus.get(), h->dStatus, sizeof(IterStatus), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    if (h->hStatus->flags & 16) return fail(FEAST_NL_EDEVICE, "tensor-core wait timed out in the node solve");
    return store_block(h, h->st, wk.Stage, wk.X, m, Y, m);
}

int feast_nl_filter_apply(feast_nl_handle* h, int32_t m, const void* X, const double* lambda,
                          void* Q) {
    g_last_error.clear();
    CKS(validate_handle(h));
    AllocScope as(h->st);
    if (!h->ns.ready) return fail(FEAST_NL_EINVAL, "no contour");
    if (m < 1 || m > kMaxM0 || m > h->n || !X || !lambda || !Q) return fail(FEAST_NL_EINVAL, "bad m or pointer");
    CKS(ensure_workspace(h, std::max(m, h->wk.mcap)));
    const int64_t n = h->n;
    const int T = h->nterms;
    const double2 one = make_double2(1.0, 0.0), zero = make_double2(0.0, 0.0);
    h->have_result = false;
    const Disc D = disc_view(h, h->ns, h->wk, 0, m, h->st, false);
    CKS(load_block(h, h->st, h->wk.Stage, X, m, D.X));
    if (is_device_ptr(lambda))
        CK(cudaMemcpyAsync(D.Lam, lambda, sizeof(double2) * m, cudaMemcpyDeviceToDevice, h->st));
    else
        CK(cudaMemcpyAsync(D.Lam, lambda, sizeof(double2) * m, cudaMemcpyHostToDevice, h->st));
    CK(cudaMemsetAsync(D.status, 0, sizeof(IterStatus), h->st));
    // R = sum_t A_t X diag(scale_t f_t(lambda))
    CKS(apply_terms(h, h->wk, 1, m, D.X, D.W, h->st, &D.status->flags));
    CK(set_identity(h->st, m, D.Yred, D.Nu));
    CK(ritz_scale(h->st, n, m, T, h->dTerms, D.Lam, D.Nu, D.X, D.Yred, D.Ycat));
    CK(gemm<double2>(h->st, 0, (int)n, m, T * m, one, D.W, n, 0, D.Ycat, (int64_t)T * m, 0, zero,
                     D.R, n, 0, 1));
    CKS(filter_solve(h, h->ns, h->wk, 1, m, h->st, &D.status->flags, false));
    CKS(filter_accumulate(h, D));
    CK(cudaMemcpyAsync(h->hStatus.get(), D.status, sizeof(IterStatus), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    if (h->hStatus->flags & 16) return fail(FEAST_NL_EDEVICE, "tensor-core wait timed out in the node solve");
    if (h->hStatus->flags & 2) return fail(FEAST_NL_ESINGULAR_NODE, "a lambda equals a node");
    return store_block(h, h->st, h->wk.Stage, D.Q, m, Q, m);
}

int feast_nl_project(feast_nl_handle* h, int32_t m, const void* Q, void* Ahat, int32_t* kmax_out) {
    g_last_error.clear();
    CKS(validate_handle(h));
    AllocScope as(h->st);
    if (h->has_exp) return fail(FEAST_NL_EUNSUPPORTED, "projection by powers needs polynomial T");
    if (m < 1 || m > kMaxM0 || m > h->n || !Q || !Ahat) return fail(FEAST_NL_EINVAL, "bad m or pointer");
    CKS(ensure_workspace(h, std::max(m, h->wk.mcap)));
    h->have_result = false;
    const Disc D = disc_view(h, h->ns, h->wk, 0, m, h->st, false);
    CKS(load_block(h, h->st, h->wk.Stage, Q, m, D.Q));
    CKS(apply_terms(h, h->wk, 1, m, D.Q, D.W, h->st, &h->dStatus->flags));
    CKS(project_block(h, D));
    CK(form_reduced(h->st, m, h->nterms, h->kmax, h->dTerms, D.G, D.Ahat));
    const bool dev = is_device_ptr(Ahat);
    for (int p = 0; p <= h->kmax; ++p) {
        double2* dst = static_cast<double2*>(Ahat) + (int64_t)p * m * m;
        if (dev) {
            CK(transpose_colmajor_to_rowmajor(h->st, m, m, D.Ahat + (int64_t)p * m * m, m, dst, m));
        } else {
            CK(transpose_colmajor_to_rowmajor(h->st, m, m, D.Ahat + (int64_t)p * m * m, m, h->wk.Stage, m));
            CK(cudaMemcpyAsync(dst, h->wk.Stage, sizeof(double2) * m * m, cudaMemcpyDeviceToHost, h->st));
            CK(cudaStreamSynchronize(h->st));
        }
    }
    CK(cudaStreamSynchronize(h->st));
    if (kmax_out) *kmax_out = h->kmax;
    return FEAST_NL_OK;
}

// ---------------------------------------------------------------- spectrum slicing

void feast_nl_slices_destroy(feast_nl_slices* s) {
    if (!s) return;
    AllocScope as(s->st);
    if (s->st) cudaStreamSynchronize(s->st);
    free_work(s->wk);
    free_nodes(s->ns);
    dfree(s->dStatus);
    dfree(s->dLamRes);
    dfree(s->dRelresRes);
    dfree(s->dXRes);
    dfree(s->dActive);
    for (cudaEvent_t e : s->join) cudaEventDestroy(e);
    for (cudaStream_t t : s->side) cudaStreamDestroy(t);
    if (s->fork) cudaEventDestroy(s->fork);
    if (s->ev0) cudaEventDestroy(s->ev0);
    if (s->ev1) cudaEventDestroy(s->ev1);
    if (s->st) cudaStreamSynchronize(s->st);
    if (s->own_stream && s->st) cudaStreamDestroy(s->st);
    delete s;
}

int feast_nl_slices_create(feast_nl_slices** out, feast_nl_handle* h, int32_t ndisc,
                           const double* c_re, const double* c_im, const double* ra,
                           const double* rb, int32_t nc, int32_t rule, void* stream) {
    g_last_error.clear();
    if (!out) return fail(FEAST_NL_EINVAL, "out pointer is NULL");
    *out = nullptr;
    CKS(validate_handle(h));
    if (ndisc < 1 || ndisc > 4096) return fail(FEAST_NL_EINVAL, "ndisc must be in [1, 4096]");
    if (!c_re || !c_im || !ra || !rb) return fail(FEAST_NL_EINVAL, "contour arrays are NULL");
    feast_nl_slices* s = new (std::nothrow) feast_nl_slices();
    if (!s) return fail(FEAST_NL_ENOMEM, "host allocation failed");
    s->h = h;
    auto cleanup = [&](int st) { feast_nl_slices_destroy(s); return st; };
    cudaError_t e;
    if (stream) {
        s->st = static_cast<cudaStream_t>(stream);
    } else {
        if ((e = cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking)) != cudaSuccess)
            return cleanup(fail_cuda(e, "cudaStreamCreate", __LINE__));
        s->own_stream = true;
    }
    AllocScope as(s->st);
    // the problem's device data may still be in flight on the handle's stream
    if ((e = cudaStreamSynchronize(h->st)) != cudaSuccess) return cleanup(fail_cuda(e, "sync", __LINE__));
    const int nside = std::min<int>(ndisc, kMaxSide);
    for (int i = 0; i < nside; ++i) {
        cudaStream_t t = nullptr;
        cudaEvent_t ev = nullptr;
        if ((e = cudaStreamCreateWithFlags(&t, cudaStreamNonBlocking)) != cudaSuccess)
            return cleanup(fail_cuda(e, "cudaStreamCreate", __LINE__));
        s->side.push_back(t);
        if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess)
            return cleanup(fail_cuda(e, "cudaEventCreate", __LINE__));
        s->join.push_back(ev);
    }
    if ((e = cudaEventCreateWithFlags(&s->fork, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreate(&s->ev0)) != cudaSuccess || (e = cudaEventCreate(&s->ev1)) != cudaSuccess)
        return cleanup(fail_cuda(e, "cudaEventCreate", __LINE__));
    if ((e = dalloc(&s->dStatus, 1)) != cudaSuccess) return cleanup(fail_cuda(e, "allocation", __LINE__));
    const int rc = build_nodes(h, s->ns, ndisc, c_re, c_im, ra, rb, nc, rule, s->st, s->dStatus, false);
    if (rc != FEAST_NL_OK) return cleanup(rc);
    *out = s;
    return FEAST_NL_OK;
}

}  // extern "C"

namespace {

// Runs f(Disc) for every contour of s->live, each on its own side stream,
// between a fork from and a join back into the set's stream (a fan-out in a
// captured graph).
template <class F>
int per_disc(feast_nl_slices* s, int m, F&& f) {
    const int nside = (int)s->side.size();
    CK(cudaEventRecord(s->fork, s->st));
    for (int i = 0; i < nside; ++i) CK(cudaStreamWaitEvent(s->side[i], s->fork, 0));
    for (int d : s->live)
        CKS(f(disc_view(s->h, s->ns, s->wk, d, m, s->side[d % nside], false)));
    for (int i = 0; i < nside; ++i) {
        CK(cudaEventRecord(s->join[i], s->side[i]));
        CK(cudaStreamWaitEvent(s->st, s->join[i], 0));
    }
    return FEAST_NL_OK;
}

// Steps 1-3 for every contour: one product A_t Q over all contours, then each
// contour's Rayleigh-Ritz and residual test in parallel.
int slices_ritz(feast_nl_slices* s, int m, double tol) {
    feast_nl_handle* h = s->h;
    CKS(apply_terms(h, s->wk, s->ns.nd, m, s->wk.Q, s->wk.W, s->st, &s->dStatus->flags,
                    s->dActive));
    return per_disc(s, m, [&](const Disc& D) { return ritz_and_residual(h, D, tol); });
}

// Steps 4-5 for every contour: all node solves in one batch, then each
// contour's accumulation and orthonormalisation in parallel.
int slices_filter(feast_nl_slices* s, int m) {
    feast_nl_handle* h = s->h;
    CKS(filter_solve(h, s->ns, s->wk, s->ns.nd, m, s->st, &s->dStatus->flags, false, s->dActive));
    return per_disc(s, m, [&](const Disc& D) {
        CKS(filter_accumulate(h, D));
        return orthonormalize(h, D);
    });
}

// Keeps contour d's current pairs as its result.
int slices_keep(feast_nl_slices* s, int d, int m) {
    const int64_t n = s->h->n;
    const Disc D = disc_view(s->h, s->ns, s->wk, d, m, s->st, false);
    CK(cudaMemcpyAsync(s->dLamRes + (int64_t)d * m, D.Lam, sizeof(double2) * m, cudaMemcpyDeviceToDevice, s->st));
    CK(cudaMemcpyAsync(s->dRelresRes + (int64_t)d * m, D.Relres, sizeof(double) * m, cudaMemcpyDeviceToDevice, s->st));
    CK(cudaMemcpyAsync(s->dXRes + (int64_t)d * n * m, D.X, sizeof(double2) * n * m, cudaMemcpyDeviceToDevice, s->st));
    return FEAST_NL_OK;
}

}  // namespace

extern "C" {

int feast_nl_slices_solve(feast_nl_slices* s, int32_t m0, double tol, int32_t maxit,
                          uint64_t seed, int32_t flags, feast_nl_info* infos) {
    g_last_error.clear();
    if (!s) return fail(FEAST_NL_EINVAL, "null slices");
    feast_nl_handle* h = s->h;
    AllocScope as(s->st);
    const int nd = s->ns.nd;
    if (infos) std::memset(infos, 0, sizeof(feast_nl_info) * nd);
    CKS(check_solve_args(h, m0, tol, maxit));
    const int m = m0;
    const int64_t n = h->n;
    s->have_result = false;
    if (s->wk.mcap != m || s->wk.nd != nd) {
        CKS(alloc_work(h, s->wk, nd, s->ns.nc, m));
        dfree(s->dLamRes);
        dfree(s->dRelresRes);
        dfree(s->dXRes);
        CK(dalloc(&s->dLamRes, (size_t)nd * m));
        CK(dalloc(&s->dRelresRes, (size_t)nd * m));
        CK(dalloc(&s->dXRes, (size_t)nd * n * m));
    }
    if (!s->dActive) CK(dalloc(&s->dActive, (size_t)nd));
    // every contour iterates until it passes Step 3; then the batched steps (A_t Q
    // and the node solves) skip it, its pairs being kept from that iteration
    std::vector<int> active(nd, 1);
    CK(cudaMemcpyAsync(s->dActive, active.data(), sizeof(int) * nd, cudaMemcpyHostToDevice, s->st));
    s->live.resize(nd);
    for (int d = 0; d < nd; ++d) s->live[d] = d;
    const bool use_graph = (flags & FEAST_NL_SLICES_NO_GRAPH) == 0;
    CK(cudaMemsetAsync(s->wk.Status, 0, sizeof(IterStatus) * nd, s->st));
    CK(cudaMemsetAsync(s->dStatus, 0, sizeof(IterStatus), s->st));   // the batched steps' flags
    CK(cudaEventRecord(s->ev0, s->st));
    CK(random_block(s->st, n, nd * m, seed, s->wk.Q));
    CKS(per_disc(s, m, [&](const Disc& D) { return orthonormalize(h, D); }));   // Step 0
    CKS(slices_ritz(s, m, tol));                                                 // Steps 1-3
    if (h->precision != FEAST_NL_FP64)           // tune the node solves before any capture
        lu_solve_pick_bn(s->st, n, lu_block_size<float2>(), static_cast<const float2*>(s->ns.dF),
                         n * n, s->ns.dGather, s->ns.dGcount, nd * s->ns.nc,
                         static_cast<float2*>(s->wk.Y), n * m, m, &s->dStatus->flags);
    // the rest of every iteration (Steps 4, 5, 1-3) as one graph over the
    // contours of s->live, captured again whenever that set has halved
    cudaGraphExec_t exec = nullptr;
    int64_t per_iter = 0, first_graph = 0;
    auto capture = [&]() -> int {
        if (exec) {
            cudaGraphExecDestroy(exec);
            exec = nullptr;
        }
        cudaGraph_t graph = nullptr;
        const uint64_t l0 = launch_count();
        CK(cudaStreamBeginCapture(s->st, cudaStreamCaptureModeThreadLocal));
        int rc2 = slices_filter(s, m);
        if (rc2 == FEAST_NL_OK) rc2 = slices_ritz(s, m, tol);
        const cudaError_t ec = cudaStreamEndCapture(s->st, &graph);
        if (rc2 != FEAST_NL_OK) { if (graph) cudaGraphDestroy(graph); return rc2; }
        CK(ec);
        per_iter = (int64_t)(launch_count() - l0);
        note_launch(-(int)per_iter);          // captured, not launched: counted at each replay
        if (!first_graph) first_graph = per_iter;
        const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        CK(ei);
        return FEAST_NL_OK;
    };
    if (use_graph) CKS(capture());
    auto run_iteration = [&]() -> int {
        if (exec) {
            CK(cudaGraphLaunch(exec, s->st));
            // the graph's kernels count as launches of this library
            note_launch((int)per_iter);
            return FEAST_NL_OK;
        }
        CKS(slices_filter(s, m));
        return slices_ritz(s, m, tol);
    };
    std::vector<IterStatus> stt(nd), kept(nd);
    std::vector<char> done(nd, 0), conv_at(nd, 0);
    IterStatus wide{};
    int remaining = nd, it = 1;
    int rc = FEAST_NL_OK;
    for (it = 1; it <= maxit; ++it) {
        if (it > 1) {
            rc = run_iteration();
            if (rc != FEAST_NL_OK) break;
        }
        cudaError_t e = cudaMemcpyAsync(stt.data(), s->wk.Status, sizeof(IterStatus) * nd,
                                        cudaMemcpyDeviceToHost, s->st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(&wide, s->dStatus, sizeof(IterStatus), cudaMemcpyDeviceToHost, s->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
        if (e != cudaSuccess) {
            rc = fail_cuda(e, "status read", __LINE__);
            break;
        }
        if (wide.flags & 16) {
            rc = fail(FEAST_NL_EDEVICE, "tensor-core wait timed out in a batched step");
            break;
        }
        for (int d = 0; d < nd; ++d) {
            if (done[d]) continue;
            const bool conv = it > 1 && stt[d].n_conv == stt[d].n_inside;
            const bool fatal = (stt[d].flags & (2 | 16)) != 0;
            if (conv || fatal || it == maxit) {
                rc = slices_keep(s, d, m);
                if (rc != FEAST_NL_OK) break;
                done[d] = 1;
                conv_at[d] = conv;
                kept[d] = stt[d];
                active[d] = 0;
                --remaining;
                if (infos) {
                    infos[d].iters = it;
                    infos[d].n_inside = stt[d].n_inside;
                    infos[d].n_converged = stt[d].n_conv;
                    infos[d].status = contour_status(stt[d], conv, m);
                    infos[d].max_relres = stt[d].max_relres;
                }
            }
        }
        if (rc != FEAST_NL_OK || remaining == 0) break;
        if (2 * remaining <= (int)s->live.size()) {
            // drop the finished contours' per-contour steps (graph and eager alike)
            s->live.clear();
            for (int d = 0; d < nd; ++d)
                if (!done[d]) s->live.push_back(d);
            if (use_graph && (rc = capture()) != FEAST_NL_OK) break;
        }
        // read by the next replay (stream order); the host copy outlives it
        if (cudaMemcpyAsync(s->dActive, active.data(), sizeof(int) * nd, cudaMemcpyHostToDevice,
                            s->st) != cudaSuccess) {
            rc = fail_cuda(cudaGetLastError(), "contour mask", __LINE__);
            break;
        }
    }
    if (exec) cudaGraphExecDestroy(exec);
    CKS(rc);
    CK(cudaEventRecord(s->ev1, s->st));
    CK(cudaEventSynchronize(s->ev1));
    float ms = 0.0f;
    CK(cudaEventElapsedTime(&ms, s->ev0, s->ev1));
    int worst = FEAST_NL_OK;
    for (int d = 0; d < nd; ++d) {
        if (infos) {
            infos[d].ms_factor = s->ns.ms_factor;
            infos[d].ms_iterate = ms;
        }
        const int sd = contour_status(kept[d], conv_at[d] != 0, m);
        if (sd == FEAST_NL_EDEVICE) worst = sd;
        else if (worst == FEAST_NL_OK && sd != FEAST_NL_OK) worst = sd;
    }
    s->m_last = m;
    s->have_result = true;
    s->graph_launches = first_graph;
    if (worst != FEAST_NL_OK) g_last_error = "some contours did not converge (see their infos)";
    return worst;
}

int feast_nl_slices_get_eigpairs(feast_nl_slices* s, int32_t disc, int32_t capacity,
                                 int32_t* m_out, double* lambda, void* X, double* relres,
                                 int32_t inside_only) {
    g_last_error.clear();
    if (!s) return fail(FEAST_NL_EINVAL, "null slices");
    AllocScope as(s->st);
    if (!s->have_result) return fail(FEAST_NL_EINVAL, "no solve result");
    if (disc < 0 || disc >= s->ns.nd) return fail(FEAST_NL_EINVAL, "disc out of range");
    if (capacity < 0 || !m_out) return fail(FEAST_NL_EINVAL, "bad capacity or m_out");
    const int m = s->m_last;
    const int64_t n = s->h->n;
    return copy_pairs(s->h, s->st, s->wk.Qt, s->wk.Stage, m, s->dLamRes + (int64_t)disc * m,
                      s->dRelresRes + (int64_t)disc * m, s->dXRes + (int64_t)disc * n * m,
                      s->ns.c_re[disc], s->ns.c_im[disc], s->ns.ra[disc], s->ns.rb[disc], capacity,
                      m_out, lambda, X, relres, inside_only);
}

int64_t feast_nl_slices_graph_launches(feast_nl_slices* s) { return s ? s->graph_launches : -1; }

}  // extern "C"
