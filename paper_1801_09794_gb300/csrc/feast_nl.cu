// C ABI of the nonlinear FEAST filter library (declared in include/feast_nl.h).
// Host-side orchestration of Algorithm 1; every numerical step runs in the
// kernels of k_dense.cu, k_lu.cu and k_reduced.cu on the handle's stream.
#include "../../include/feast_nl.h"
#include "internal.h"

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

struct feast_nl_handle {
    int64_t n = 0;
    int nterms = 0, nA = 0, kmax = 0, precision = 0;
    bool has_exp = false;
    cudaStream_t st = nullptr;
    bool own_stream = false;
    std::vector<HostTerm> terms;
    double2* dA = nullptr;          // nA x n x n, column-major
    TermDev* dTerms = nullptr;
    // contour
    bool have_contour = false;
    double c_re = 0, c_im = 0, ra = 1, rb = 1;
    int nc = 0, rule = 0;
    std::vector<zd> z, w;
    double2* dz = nullptr;
    double2* dw = nullptr;
    void* dF = nullptr;             // nc x n x n in LU precision
    int* dpiv = nullptr;
    int* dinfo = nullptr;
    int2* dGather = nullptr;        // per node and panel: row interchanges as a gather list
    int* dGcount = nullptr;
    double ms_factor = 0.0;
    // subspace workspace (sized for mcap columns)
    int mcap = 0;
    double2 *dQ = nullptr, *dQt = nullptr, *dX = nullptr, *dR = nullptr, *dW = nullptr;
    void* dY = nullptr;
    double2 *dG = nullptr, *dSplit = nullptr, *dAhat = nullptr, *dYred = nullptr, *dYcat = nullptr;
    double2 *dG2 = nullptr, *dRinv = nullptr, *dLam = nullptr, *dCoef = nullptr, *dFsum = nullptr;
    double *dNu = nullptr, *dRnorm = nullptr, *dRelres = nullptr;
    unsigned char* dRed = nullptr;  // reduced-problem workspace (bytes)
    unsigned char* dBeyn = nullptr; // reduced solver for non-polynomial T (bytes)
    double2* dStage = nullptr;      // n x mcap staging for layout changes
    IterStatus* dStatus = nullptr;
    // pageable: freeing pinned memory would synchronise the whole device
    std::unique_ptr<IterStatus> hStatus{new IterStatus()};
    int splits = 1;
    // digit-split products on the tensor cores (precision FEAST_NL_FP32_I8)
    int oz_s = 0;
    OzakiLayout oz;                 // layout for mcap columns
    unsigned char* dAsl = nullptr;  // nA x s slices of A'
    double* dSigma = nullptr;       // nA x Mpad row scales
    unsigned char* dQsl = nullptr;  // s slices of Q'
    double* dTau = nullptr;         // column scales
    int* dSlot = nullptr;           // dense index -> term index
    // results of the last solve
    bool have_result = false;
    int m_last = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // optional per-phase device timing
    struct Mark { int phase; cudaEvent_t a, b; uint64_t l0, l1; };
    bool prof = false;
    std::vector<Mark> marks;
    std::vector<cudaEvent_t> pool;
    size_t pool_used = 0;
    double prof_ms[FEAST_NL_NPHASES] = {0};
    int64_t prof_launches[FEAST_NL_NPHASES] = {0};

    size_t lu_elem() const { return precision == FEAST_NL_FP64 ? sizeof(double2) : sizeof(float2); }
};

namespace {

cudaEvent_t prof_event(feast_nl_handle* h) {
    if (h->pool_used == h->pool.size()) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        h->pool.push_back(e);
    }
    return h->pool[h->pool_used++];
}
// Scoped device-time measurement of one phase (no-op unless profiling is on).
struct Phase {
    feast_nl_handle* h;
    int idx = -1;
    Phase(feast_nl_handle* hh, int phase) : h(hh) {
        if (!h->prof) return;
        cudaEvent_t a = prof_event(h), b = prof_event(h);
        if (!a || !b) return;
        cudaEventRecord(a, h->st);
        h->marks.push_back({phase, a, b, launch_count(), 0});
        idx = (int)h->marks.size() - 1;
    }
    ~Phase() {
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

void release_workspace(feast_nl_handle* h) {
    dfree(h->dQ); dfree(h->dQt); dfree(h->dX); dfree(h->dR); dfree(h->dW);
    dfree(h->dY);
    dfree(h->dG); dfree(h->dSplit); dfree(h->dAhat); dfree(h->dYred); dfree(h->dYcat);
    dfree(h->dG2); dfree(h->dRinv); dfree(h->dLam); dfree(h->dCoef); dfree(h->dFsum);
    dfree(h->dNu); dfree(h->dRnorm); dfree(h->dRelres); dfree(h->dRed); dfree(h->dBeyn); dfree(h->dStage);
    dfree(h->dQsl); dfree(h->dTau);
    h->mcap = 0;
    h->have_result = false;
}

int ensure_workspace(feast_nl_handle* h, int m) {
    if (m <= h->mcap && (h->dY || h->nc == 0)) return FEAST_NL_OK;
    release_workspace(h);
    const int64_t n = h->n;
    const int T = h->nterms;
    const int nc = std::max(h->nc, 1);
    CK(dalloc(&h->dQ, (size_t)n * m));
    CK(dalloc(&h->dQt, (size_t)n * m));
    CK(dalloc(&h->dX, (size_t)n * m));
    CK(dalloc(&h->dR, (size_t)n * m));
    CK(dalloc(&h->dW, (size_t)n * m * T));
    {
        unsigned char* y = nullptr;
        CK(dalloc(&y, (size_t)nc * n * m * h->lu_elem()));
        h->dY = y;
    }
    // split-K so that the m x (T m) products fill the GPU
    int tiles = ((m + 63) / 64) * ((T * m + 63) / 64);
    h->splits = (int)std::max<int64_t>(1, std::min<int64_t>(64, std::min<int64_t>(n / 64, 304 / tiles)));
    CK(dalloc(&h->dG, (size_t)m * m * T));
    CK(dalloc(&h->dSplit, (size_t)h->splits * m * m * T + 16));
    CK(dalloc(&h->dAhat, (size_t)(h->kmax + 1) * m * m));
    CK(dalloc(&h->dYred, (size_t)m * m));
    CK(dalloc(&h->dYcat, (size_t)T * m * m));
    CK(dalloc(&h->dG2, (size_t)m * m));
    CK(dalloc(&h->dRinv, (size_t)m * m));
    CK(dalloc(&h->dLam, (size_t)m));
    CK(dalloc(&h->dCoef, (size_t)nc * m));
    CK(dalloc(&h->dFsum, (size_t)m));
    CK(dalloc(&h->dNu, (size_t)m));
    CK(dalloc(&h->dRnorm, (size_t)m));
    CK(dalloc(&h->dRelres, (size_t)m));
    CK(dalloc(&h->dRed, reduced_work_bytes(m, std::max(h->kmax, 1))));
    if (h->has_exp && m <= beyn_max_m()) CK(dalloc(&h->dBeyn, beyn_work_bytes(m)));
    CK(dalloc(&h->dStage, (size_t)n * m));
    if (h->oz_s > 0) {
        h->oz = ozaki_layout(n, m, h->oz_s);
        const size_t qb = (size_t)(h->oz.b_slice * h->oz_s) * ozaki_elem_bytes();
        CK(dalloc(&h->dQsl, qb));
        CK(cudaMemsetAsync(h->dQsl, 0, qb, h->st));
        CK(dalloc(&h->dTau, (size_t)m));
    }
    h->mcap = m;
    return FEAST_NL_OK;
}

// Copy an n x m complex128 row-major block (host or device) into column-major dst.
int load_block(feast_nl_handle* h, const void* src, int m, double2* dst) {
    const size_t bytes = (size_t)h->n * m * sizeof(double2);
    const double2* s = static_cast<const double2*>(src);
    if (!is_device_ptr(src)) {
        CK(cudaMemcpyAsync(h->dStage, src, bytes, cudaMemcpyHostToDevice, h->st));
        s = h->dStage;
    }
    CK(transpose_rowmajor_to_colmajor(h->st, h->n, m, s, m, dst, h->n));
    return FEAST_NL_OK;
}
// Copy column-major src (n x m, ld n) out as row-major with row stride ldd (host or device).
int store_block(feast_nl_handle* h, const double2* src, int m, void* dst, int64_t ldd) {
    if (is_device_ptr(dst)) {
        CK(transpose_colmajor_to_rowmajor(h->st, h->n, m, src, h->n,
                                          static_cast<double2*>(dst), ldd));
        CK(cudaStreamSynchronize(h->st));
        return FEAST_NL_OK;
    }
    CK(transpose_colmajor_to_rowmajor(h->st, h->n, m, src, h->n, h->dStage, m));
    CK(cudaMemcpy2DAsync(dst, ldd * sizeof(double2), h->dStage, m * sizeof(double2),
                         m * sizeof(double2), h->n, cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    return FEAST_NL_OK;
}

// Columns of the stacked product W = [A_0 Q, ..., A_{T-1} Q] (identity terms copy Q).
int apply_terms(feast_nl_handle* h, const double2* Q, int m, double2* W) {
    const int64_t n = h->n;
    const double2 one = make_double2(1.0, 0.0), zero = make_double2(0.0, 0.0);
    if (h->oz_s > 0 && h->nA > 0) {
        // all dense terms at once on the INT8 tensor cores
        const OzakiLayout L = ozaki_layout(n, m, h->oz_s);
        CK(ozaki_split_Q(h->st, n, m, h->oz_s, Q, h->dTau, h->dQsl, L));
        CK(ozaki_gemm(h->st, n, m, L, h->nA, h->dAsl, h->dSigma, h->dQsl, h->dTau, W, h->dSlot,
                      &h->dStatus->flags));
        CK(copy_identity_terms(h->st, n, m, h->nterms, h->dTerms, Q, W));
        return FEAST_NL_OK;
    }
    for (int t = 0; t < h->nterms; ++t) {
        const HostTerm& ht = h->terms[t];
        if (ht.aidx < 0) continue;
        CK(gemm<double2>(h->st, 0, (int)n, m, (int)n, one, h->dA + (int64_t)ht.aidx * n * n, n, 0,
                         Q, n, 0, zero, W + (int64_t)t * n * m, n, 0, 1));
    }
    CK(copy_identity_terms(h->st, n, m, h->nterms, h->dTerms, Q, W));
    return FEAST_NL_OK;
}

// Q <- Q R^{-1} twice (CholQR with a small diagonal shift), columns pre-equilibrated.
// Only the product Q R^{-1} has to be exact to FP64 rounding (it must keep the
// span); the Gram matrix feeds an FP32 Cholesky, so it is formed from an FP32
// copy of Q (held in the node right-hand-side buffer, free at this point).
int orthonormalize(feast_nl_handle* h, int m) {
    Phase ph(h, FEAST_NL_PH_ORTH);
    const int64_t n = h->n;
    const double2 one = make_double2(1.0, 0.0), zero = make_double2(0.0, 0.0);
    float2* Q32 = static_cast<float2*>(h->dY);
    if (!Q32) return fail(FEAST_NL_EINVAL, "no contour: node buffers not allocated");
    CK(column_norms(h->st, n, m, h->dQ, n, h->dNu));
    CK(ritz_scale(h->st, n, m, 0, h->dTerms, h->dLam, h->dNu, h->dQ, h->dYred, h->dYcat));
    for (int pass = 0; pass < 2; ++pass) {
        CK(to_float(h->st, n * m, h->dQ, Q32));
        CK(gram_f32(h->st, m, (int)n, Q32, n, h->dG2, m, reinterpret_cast<float2*>(h->dSplit),
                    h->splits));
        CK(chol_inverse(h->st, m, h->dG2, 1e-6, h->dRinv, h->dStatus));
        CK(gemm<double2>(h->st, 0, (int)n, m, m, one, h->dQ, n, 0, h->dRinv, m, 0, zero, h->dQt, n,
                         0, 1));
        std::swap(h->dQ, h->dQt);
    }
    return FEAST_NL_OK;
}

// Rayleigh-Ritz (Steps 1-2) and the block residual (Step 3) for the current Q.
int ritz_and_residual(feast_nl_handle* h, int m, double tol) {
    const int64_t n = h->n;
    const int T = h->nterms;
    const double2 one = make_double2(1.0, 0.0), zero = make_double2(0.0, 0.0);
    {
        Phase ph(h, FEAST_NL_PH_APPLY);
        CKS(apply_terms(h, h->dQ, m, h->dW));
    }
    {
        Phase ph(h, FEAST_NL_PH_PROJECT);
        CK(gemm_splitk_d(h->st, 1, m, T * m, (int)n, one, h->dQ, n, h->dW, n, zero, h->dG, m,
                         h->dSplit, h->splits));
        if (!h->has_exp) CK(form_reduced(h->st, m, T, h->kmax, h->dTerms, h->dG, h->dAhat));
    }
    {
        Phase ph(h, FEAST_NL_PH_REDUCED);
        if (h->has_exp)
            CK(reduced_solve_general(h->st, m, T, h->dTerms, h->dG, h->c_re, h->c_im, h->ra, h->rb,
                                     kBeynProbeSeed, h->dBeyn, h->dLam, h->dYred, h->dStatus));
        else
            CK(reduced_solve(h->st, m, h->kmax, h->dAhat, m, h->c_re, h->c_im, h->ra, h->rb,
                             h->dRed, h->dLam, h->dYred, h->dStatus));
    }
    Phase ph(h, FEAST_NL_PH_RITZ);
    CK(gemm<double2>(h->st, 0, (int)n, m, m, one, h->dQ, n, 0, h->dYred, m, 0, zero, h->dX, n, 0,
                     1));
    CK(column_norms(h->st, n, m, h->dX, n, h->dNu));
    CK(ritz_scale(h->st, n, m, T, h->dTerms, h->dLam, h->dNu, h->dX, h->dYred, h->dYcat));
    CK(gemm<double2>(h->st, 0, (int)n, m, T * m, one, h->dW, n, 0, h->dYcat, (int64_t)T * m, 0,
                     zero, h->dR, n, 0, 1));
    CK(column_norms(h->st, n, m, h->dR, n, h->dRnorm));
    CK(residual_summary(h->st, m, T, h->dTerms, h->dLam, h->dRnorm, h->c_re, h->c_im, h->ra,
                        h->rb, tol, h->dRelres, h->dStatus));
    return FEAST_NL_OK;
}

// Step 4 for the current (X, Lambda, R): node solves and weighted accumulation into Q.
int filter_step(feast_nl_handle* h, int m) {
    const int64_t n = h->n;
    if (h->precision == FEAST_NL_FP64) {
        double2* Y = static_cast<double2*>(h->dY);
        {
            Phase ph(h, FEAST_NL_PH_SOLVE);
            CK(broadcast_rhs<double2>(h->st, n, m, h->dR, h->nc, Y, n * m));
            CK(lu_solve_batched<double2>(h->st, n, lu_block_size<double2>(),
                                         static_cast<const double2*>(h->dF), n * n, h->dGather,
                                         h->dGcount, h->nc, Y, n * m, m, &h->dStatus->flags));
        }
        Phase ph(h, FEAST_NL_PH_ACCUM);
        CK(filter_coefficients(h->st, h->nc, m, h->dz, h->dw, h->dLam, h->dCoef, h->dFsum,
                               h->dStatus));
        CK(accumulate_filter<double2>(h->st, n, m, h->nc, h->dX, Y, n * m, h->dCoef, h->dFsum,
                                      h->dQ));
    } else {
        float2* Y = static_cast<float2*>(h->dY);
        {
            Phase ph(h, FEAST_NL_PH_SOLVE);
            CK(broadcast_rhs<float2>(h->st, n, m, h->dR, h->nc, Y, n * m));
            CK(lu_solve_batched<float2>(h->st, n, lu_block_size<float2>(),
                                        static_cast<const float2*>(h->dF), n * n, h->dGather,
                                        h->dGcount, h->nc, Y, n * m, m, &h->dStatus->flags));
        }
        Phase ph(h, FEAST_NL_PH_ACCUM);
        CK(filter_coefficients(h->st, h->nc, m, h->dz, h->dw, h->dLam, h->dCoef, h->dFsum,
                               h->dStatus));
        CK(accumulate_filter<float2>(h->st, n, m, h->nc, h->dX, Y, n * m, h->dCoef, h->dFsum,
                                     h->dQ));
    }
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
    release_workspace(h);
    dfree(h->dA);
    dfree(h->dAsl);
    dfree(h->dSigma);
    dfree(h->dSlot);
    dfree(h->dTerms);
    dfree(h->dz);
    dfree(h->dw);
    dfree(h->dF);
    dfree(h->dpiv);
    dfree(h->dinfo);
    dfree(h->dGather);
    dfree(h->dGcount);
    dfree(h->dStatus);
    for (cudaEvent_t e : h->pool) cudaEventDestroy(e);
    if (h->ev0) cudaEventDestroy(h->ev0);
    if (h->ev1) cudaEventDestroy(h->ev1);
    if (h->own_stream && h->st) cudaStreamDestroy(h->st);
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
        std::vector<int> slot;
        for (int t = 0; t < nterms; ++t)
            if (h->terms[t].aidx >= 0) slot.push_back(t);
        if ((e = dalloc(&h->dAsl, (size_t)(L.a_term * h->nA) * ozaki_elem_bytes())) != cudaSuccess ||
            (e = dalloc(&h->dSigma, (size_t)(L.Mpad * h->nA))) != cudaSuccess ||
            (e = dalloc(&h->dSlot, slot.size())) != cudaSuccess ||
            (e = cudaMemcpyAsync(h->dSlot, slot.data(), sizeof(int) * slot.size(),
                                 cudaMemcpyHostToDevice, h->st)) != cudaSuccess ||
            (e = cudaStreamSynchronize(h->st)) != cudaSuccess)
            return cleanup(fail_cuda(e, "allocation of digit slices", __LINE__));
    }
    // copy the coefficients in, transposed to column-major
    double2* stage = nullptr;
    double2 *v = nullptr, *u = nullptr, *gw = nullptr;
    double* nrm = nullptr;
    auto free_tmp = [&]() { dfree(stage); dfree(v); dfree(u); dfree(gw); dfree(nrm); };
    bool need_stage = false;
    for (int t = 0; t < nterms; ++t)
        if (terms[t].A && !terms[t].on_device) need_stage = true;
    if (need_stage && (e = dalloc(&stage, (size_t)n * n)) != cudaSuccess) {
        free_tmp();
        return cleanup(fail_cuda(e, "staging allocation", __LINE__));
    }
    if ((e = dalloc(&v, (size_t)n)) != cudaSuccess || (e = dalloc(&u, (size_t)n)) != cudaSuccess ||
        (e = dalloc(&gw, (size_t)n * 32)) != cudaSuccess || (e = dalloc(&nrm, 2)) != cudaSuccess) {
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
            const OzakiLayout L = ozaki_layout(n, 1, h->oz_s);
            const int a = h->terms[t].aidx;
            e = ozaki_split_A(h->st, n, h->oz_s, dst, h->dSigma + (int64_t)a * L.Mpad,
                              h->dAsl + (int64_t)a * L.a_term * ozaki_elem_bytes(), L);
            if (e != cudaSuccess) { free_tmp(); return cleanup(fail_cuda(e, "digit split of A", __LINE__)); }
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
    if (!(ra > 0.0) || !(rb > 0.0) || !std::isfinite(c_re) || !std::isfinite(c_im))
        return fail(FEAST_NL_EINVAL, "contour needs finite center and ra, rb > 0");
    if (nc < 1 || nc > 1024) return fail(FEAST_NL_EINVAL, "nc must be in [1, 1024]");
    if (rule < FEAST_NL_GL || rule > FEAST_NL_GL_HALVES) return fail(FEAST_NL_EINVAL, "unknown rule");
    if (rule == FEAST_NL_GL_HALVES && (nc % 2)) return fail(FEAST_NL_EINVAL, "GL_HALVES needs even nc");
    const int64_t n = h->n;
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
    h->z.assign(nc, 0.0);
    h->w.assign(nc, 0.0);
    const zd c(c_re, c_im);
    for (int j = 0; j < nc; ++j) {
        h->z[j] = c + ra * std::cos(th[j]) + zd(0.0, 1.0) * rb * std::sin(th[j]);
        zd dz(-ra * std::sin(th[j]), rb * std::cos(th[j]));
        h->w[j] = wt[j] * dz / zd(0.0, 2.0 * M_PI);
    }
    // node-matrix coefficients
    std::vector<double2> coef((size_t)std::max(h->nA, 1) * nc), diagc(nc);
    for (int j = 0; j < nc; ++j) {
        zd dsum = 0.0;
        for (int t = 0; t < h->nterms; ++t) {
            const HostTerm& ht = h->terms[t];
            zd f = term_f_host(ht.kind, ht.p, ht.tau, ht.scale, h->z[j]);
            if (ht.aidx < 0) dsum += f;
            else coef[(size_t)ht.aidx * nc + j] = make_double2(f.real(), f.imag());
        }
        diagc[j] = make_double2(dsum.real(), dsum.imag());
    }
    // (re)allocate node storage
    dfree(h->dF);
    dfree(h->dpiv); dfree(h->dinfo); dfree(h->dz); dfree(h->dw);
    dfree(h->dGather); dfree(h->dGcount);
    h->have_contour = false;
    h->have_result = false;
    release_workspace(h);
    double2 *dcoef = nullptr, *ddiag = nullptr;
    {
        unsigned char* f = nullptr;
        CK(dalloc(&f, (size_t)nc * n * n * h->lu_elem()));
        h->dF = f;
    }
    CK(dalloc(&h->dpiv, (size_t)nc * n));
    {
        const int nb = h->precision == FEAST_NL_FP64 ? lu_block_size<double2>() : lu_block_size<float2>();
        const int gs = lu_gather_stride(n, nb);
        CK(dalloc(&h->dGather, (size_t)nc * gs));
        CK(dalloc(&h->dGcount, (size_t)nc * (gs / 128)));
    }
    CK(dalloc(&h->dinfo, (size_t)nc));
    CK(dalloc(&h->dz, (size_t)nc));
    CK(dalloc(&h->dw, (size_t)nc));
    CK(dalloc(&dcoef, coef.size()));
    CK(dalloc(&ddiag, (size_t)nc));
    h->nc = nc;
    h->rule = rule;
    h->c_re = c_re; h->c_im = c_im; h->ra = ra; h->rb = rb;
    std::vector<double2> zz(nc), ww(nc);
    for (int j = 0; j < nc; ++j) {
        zz[j] = make_double2(h->z[j].real(), h->z[j].imag());
        ww[j] = make_double2(h->w[j].real(), h->w[j].imag());
    }
    CK(cudaMemcpyAsync(h->dz, zz.data(), sizeof(double2) * nc, cudaMemcpyHostToDevice, h->st));
    CK(cudaMemcpyAsync(h->dw, ww.data(), sizeof(double2) * nc, cudaMemcpyHostToDevice, h->st));
    CK(cudaMemcpyAsync(dcoef, coef.data(), sizeof(double2) * coef.size(), cudaMemcpyHostToDevice, h->st));
    CK(cudaMemcpyAsync(ddiag, diagc.data(), sizeof(double2) * nc, cudaMemcpyHostToDevice, h->st));
    CK(cudaMemsetAsync(h->dinfo, 0, sizeof(int) * nc, h->st));
    CK(cudaMemsetAsync(h->dStatus, 0, sizeof(IterStatus), h->st));
    CK(cudaEventRecord(h->ev0, h->st));
    if (h->precision == FEAST_NL_FP64) {
        double2* F = static_cast<double2*>(h->dF);
        {
            Phase ph(h, FEAST_NL_PH_ASSEMBLE);
            CK(assemble_nodes<double2>(h->st, n, h->nA, h->dA, dcoef, ddiag, nc, F, n * n));
        }
        Phase ph(h, FEAST_NL_PH_LU);
        CK(lu_factor_batched<double2>(h->st, n, lu_block_size<double2>(), F, n * n, h->dpiv, nc,
                                      h->dinfo, h->dGather, h->dGcount, &h->dStatus->flags));
    } else {
        float2* F = static_cast<float2*>(h->dF);
        {
            Phase ph(h, FEAST_NL_PH_ASSEMBLE);
            CK(assemble_nodes<float2>(h->st, n, h->nA, h->dA, dcoef, ddiag, nc, F, n * n));
        }
        Phase ph(h, FEAST_NL_PH_LU);
        CK(lu_factor_batched<float2>(h->st, n, lu_block_size<float2>(), F, n * n, h->dpiv, nc,
                                     h->dinfo, h->dGather, h->dGcount, &h->dStatus->flags));
    }
    CK(cudaEventRecord(h->ev1, h->st));
    std::vector<int> info(nc);
    CK(cudaMemcpyAsync(info.data(), h->dinfo, sizeof(int) * nc, cudaMemcpyDeviceToHost, h->st));
    CK(cudaMemcpyAsync(h->hStatus.get(), h->dStatus, sizeof(IterStatus), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    float ms = 0.0f;
    CK(cudaEventElapsedTime(&ms, h->ev0, h->ev1));
    h->ms_factor = ms;
    prof_flush(h);
    dfree(dcoef);
    dfree(ddiag);
    if (h->hStatus->flags & 16) return fail(FEAST_NL_EDEVICE, "tensor-core wait timed out in the node LU");
    for (int j = 0; j < nc; ++j)
        if (info[j] != 0)
            return fail(FEAST_NL_ESINGULAR_NODE,
                        "zero pivot in T(z_" + std::to_string(j) + ") at column " + std::to_string(info[j] - 1));
    h->have_contour = true;
    return FEAST_NL_OK;
}

int feast_nl_solve(feast_nl_handle* h, int32_t m0, double tol, int32_t maxit, uint64_t seed,
                   const void* X0, feast_nl_info* info) {
    g_last_error.clear();
    CKS(validate_handle(h));
    AllocScope as(h->st);
    if (info) std::memset(info, 0, sizeof(*info));
    if (!h->have_contour) return fail(FEAST_NL_EINVAL, "set_contour must succeed before solve");
    if (m0 < 1 || m0 > kMaxM0 || m0 > h->n) return fail(FEAST_NL_EINVAL, "m0 must be in [1, min(n, 112)]");
    if (h->has_exp && m0 > beyn_max_m())
        return fail(FEAST_NL_EINVAL, "non-polynomial T: m0 must be <= " + std::to_string(beyn_max_m()));
    if (h->kmax * m0 > 1024) return fail(FEAST_NL_EINVAL, "degree * m0 must be <= 1024");
    if (maxit < 1) return fail(FEAST_NL_EINVAL, "maxit must be >= 1");
    if (!(tol > 0.0)) return fail(FEAST_NL_EINVAL, "tol must be > 0");
    CKS(ensure_workspace(h, m0));
    h->have_result = false;
    const int m = m0;
    CK(cudaMemsetAsync(h->dStatus, 0, sizeof(IterStatus), h->st));
    CK(cudaEventRecord(h->ev0, h->st));
    {
        Phase ph(h, FEAST_NL_PH_IO);
        if (X0) CKS(load_block(h, X0, m, h->dQ));
        else CK(random_block(h->st, h->n, m, seed, h->dQ));
    }
    CKS(orthonormalize(h, m));                                  // Step 0
    int it = 0;
    bool converged = false;
    IterStatus stt{};
    for (it = 1; it <= maxit; ++it) {
        CKS(ritz_and_residual(h, m, tol));                      // Steps 1-3
        CK(cudaMemcpyAsync(h->hStatus.get(), h->dStatus, sizeof(IterStatus), cudaMemcpyDeviceToHost, h->st));
        CK(cudaStreamSynchronize(h->st));
        stt = *h->hStatus;
        if (trace_enabled()) {
            std::vector<double2> lam(m);
            std::vector<double> rr(m);
            cudaMemcpyAsync(lam.data(), h->dLam, sizeof(double2) * m, cudaMemcpyDeviceToHost, h->st);
            cudaMemcpyAsync(rr.data(), h->dRelres, sizeof(double) * m, cudaMemcpyDeviceToHost, h->st);
            cudaStreamSynchronize(h->st);
            fprintf(stderr, "[feast_nl] it %d inside %d conv %d max_relres %.3e flags %d qr_sweeps %d\n",
                    it, stt.n_inside, stt.n_conv, stt.max_relres, stt.flags, stt.qr_sweeps);
            for (int i = 0; i < m; ++i)
                fprintf(stderr, "    %2d  % .12e % .12e  relres %.3e\n", i, lam[i].x, lam[i].y, rr[i]);
        }
        if (it > 1 && stt.n_conv == stt.n_inside) { converged = true; break; }
        if (it == maxit) break;
        CKS(filter_step(h, m));                                 // Step 4
        CKS(orthonormalize(h, m));                              // Step 5
    }
    CK(cudaEventRecord(h->ev1, h->st));
    CK(cudaEventSynchronize(h->ev1));
    float ms = 0.0f;
    CK(cudaEventElapsedTime(&ms, h->ev0, h->ev1));
    prof_flush(h);
    h->have_result = true;
    h->m_last = m;
    int status = converged ? FEAST_NL_OK : FEAST_NL_ENOT_CONVERGED;
    if (stt.n_inside >= m) status = FEAST_NL_ETOO_MANY;
    if (stt.flags & 2) status = FEAST_NL_ESINGULAR_NODE;
    if (stt.flags & 16) status = FEAST_NL_EDEVICE;
    if (info) {
        info->iters = std::min(it, maxit);
        info->n_inside = stt.n_inside;
        info->n_converged = stt.n_conv;
        info->status = status;
        info->max_relres = stt.max_relres;
        info->ms_factor = h->ms_factor;
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
    const int m = h->m_last;
    std::vector<double2> lam(m);
    std::vector<double> rr(m);
    CK(cudaMemcpyAsync(lam.data(), h->dLam, sizeof(double2) * m, cudaMemcpyDeviceToHost, h->st));
    CK(cudaMemcpyAsync(rr.data(), h->dRelres, sizeof(double) * m, cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    std::vector<int> idx;
    for (int i = 0; i < m; ++i) {
        double dx = (lam[i].x - h->c_re) / h->ra, dy = (lam[i].y - h->c_im) / h->rb;
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
        if (is_device_ptr(lambda)) CK(cudaMemcpyAsync(lambda, lo.data(), sizeof(double2) * cnt, cudaMemcpyHostToDevice, h->st));
        else std::memcpy(lambda, lo.data(), sizeof(double2) * cnt);
    }
    if (relres) {
        if (is_device_ptr(relres)) CK(cudaMemcpyAsync(relres, ro.data(), sizeof(double) * cnt, cudaMemcpyHostToDevice, h->st));
        else std::memcpy(relres, ro.data(), sizeof(double) * cnt);
    }
    if (X) {
        // gather the chosen columns into the staging buffer (column-major), then store
        for (int q = 0; q < cnt; ++q)
            CK(cudaMemcpyAsync(h->dQt + (int64_t)q * h->n, h->dX + (int64_t)idx[q] * h->n,
                               sizeof(double2) * h->n, cudaMemcpyDeviceToDevice, h->st));
        CKS(store_block(h, h->dQt, cnt, X, capacity));
    }
    CK(cudaStreamSynchronize(h->st));
    return FEAST_NL_OK;
}

int feast_nl_get_nodes(feast_nl_handle* h, double* z, double* omega) {
    g_last_error.clear();
    CKS(validate_handle(h));
    if (!h->have_contour) return fail(FEAST_NL_EINVAL, "no contour");
    for (int j = 0; j < h->nc; ++j) {
        if (z) { z[2 * j] = h->z[j].real(); z[2 * j + 1] = h->z[j].imag(); }
        if (omega) { omega[2 * j] = h->w[j].real(); omega[2 * j + 1] = h->w[j].imag(); }
    }
    return FEAST_NL_OK;
}

int feast_nl_node_solve(feast_nl_handle* h, int32_t j, int32_t m, const void* R, void* Y) {
    g_last_error.clear();
    CKS(validate_handle(h));
    AllocScope as(h->st);
    if (!h->have_contour) return fail(FEAST_NL_EINVAL, "no contour");
    if (j < 0 || j >= h->nc || m < 1 || m > kMaxM0 || !R || !Y) return fail(FEAST_NL_EINVAL, "bad node, m or pointer");
    CKS(ensure_workspace(h, std::max(m, h->mcap)));
    const int64_t n = h->n;
    CKS(load_block(h, R, m, h->dR));
    CK(cudaMemsetAsync(h->dStatus, 0, sizeof(IterStatus), h->st));
    if (h->precision == FEAST_NL_FP64) {
        double2* Yb = static_cast<double2*>(h->dY);
        CK(broadcast_rhs<double2>(h->st, n, m, h->dR, 1, Yb, n * m));
        const int gs = lu_gather_stride(n, lu_block_size<double2>());
        CK(lu_solve_batched<double2>(h->st, n, lu_block_size<double2>(),
                                     static_cast<const double2*>(h->dF) + (int64_t)j * n * n, n * n,
                                     h->dGather + (int64_t)j * gs, h->dGcount + (int64_t)j * (gs / 128),
                                     1, Yb, n * m, m, &h->dStatus->flags));
        CK(to_double<double2>(h->st, n * m, Yb, h->dX));
    } else {
        float2* Yb = static_cast<float2*>(h->dY);
        CK(broadcast_rhs<float2>(h->st, n, m, h->dR, 1, Yb, n * m));
        const int gs = lu_gather_stride(n, lu_block_size<float2>());
        CK(lu_solve_batched<float2>(h->st, n, lu_block_size<float2>(),
                                    static_cast<const float2*>(h->dF) + (int64_t)j * n * n, n * n,
                                    h->dGather + (int64_t)j * gs, h->dGcount + (int64_t)j * (gs / 128),
                                    1, Yb, n * m, m, &h->dStatus->flags));
        CK(to_double<float2>(h->st, n * m, Yb, h->dX));
    }
    h->have_result = false;
    CK(cudaMemcpyAsync(h->hStatus.get(), h->dStatus, sizeof(IterStatus), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    if (h->hStatus->flags & 16) return fail(FEAST_NL_EDEVICE, "tensor-core wait timed out in the node solve");
    return store_block(h, h->dX, m, Y, m);
}

int feast_nl_filter_apply(feast_nl_handle* h, int32_t m, const void* X, const double* lambda,
                          void* Q) {
    g_last_error.clear();
    CKS(validate_handle(h));
    AllocScope as(h->st);
    if (!h->have_contour) return fail(FEAST_NL_EINVAL, "no contour");
    if (m < 1 || m > kMaxM0 || m > h->n || !X || !lambda || !Q) return fail(FEAST_NL_EINVAL, "bad m or pointer");
    CKS(ensure_workspace(h, std::max(m, h->mcap)));
    const int64_t n = h->n;
    const int T = h->nterms;
    const double2 one = make_double2(1.0, 0.0), zero = make_double2(0.0, 0.0);
    h->have_result = false;
    CKS(load_block(h, X, m, h->dX));
    if (is_device_ptr(lambda))
        CK(cudaMemcpyAsync(h->dLam, lambda, sizeof(double2) * m, cudaMemcpyDeviceToDevice, h->st));
    else
        CK(cudaMemcpyAsync(h->dLam, lambda, sizeof(double2) * m, cudaMemcpyHostToDevice, h->st));
    CK(cudaMemsetAsync(h->dStatus, 0, sizeof(IterStatus), h->st));
    // R = sum_t A_t X diag(scale_t f_t(lambda))
    CKS(apply_terms(h, h->dX, m, h->dW));
    CK(set_identity(h->st, m, h->dYred, h->dNu));
    CK(ritz_scale(h->st, n, m, T, h->dTerms, h->dLam, h->dNu, h->dX, h->dYred, h->dYcat));
    CK(gemm<double2>(h->st, 0, (int)n, m, T * m, one, h->dW, n, 0, h->dYcat, (int64_t)T * m, 0,
                     zero, h->dR, n, 0, 1));
    CKS(filter_step(h, m));
    CK(cudaMemcpyAsync(h->hStatus.get(), h->dStatus, sizeof(IterStatus), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    if (h->hStatus->flags & 16) return fail(FEAST_NL_EDEVICE, "tensor-core wait timed out in the node solve");
    if (h->hStatus->flags & 2) return fail(FEAST_NL_ESINGULAR_NODE, "a lambda equals a node");
    return store_block(h, h->dQ, m, Q, m);
}

int feast_nl_project(feast_nl_handle* h, int32_t m, const void* Q, void* Ahat, int32_t* kmax_out) {
    g_last_error.clear();
    CKS(validate_handle(h));
    AllocScope as(h->st);
    if (h->has_exp) return fail(FEAST_NL_EUNSUPPORTED, "projection by powers needs polynomial T");
    if (m < 1 || m > kMaxM0 || m > h->n || !Q || !Ahat) return fail(FEAST_NL_EINVAL, "bad m or pointer");
    CKS(ensure_workspace(h, std::max(m, h->mcap)));
    const int64_t n = h->n;
    const int T = h->nterms;
    const double2 one = make_double2(1.0, 0.0), zero = make_double2(0.0, 0.0);
    h->have_result = false;
    CKS(load_block(h, Q, m, h->dQ));
    CKS(apply_terms(h, h->dQ, m, h->dW));
    CK(gemm_splitk_d(h->st, 1, m, T * m, (int)n, one, h->dQ, n, h->dW, n, zero, h->dG, m,
                     h->dSplit, h->splits));
    CK(form_reduced(h->st, m, T, h->kmax, h->dTerms, h->dG, h->dAhat));
    const bool dev = is_device_ptr(Ahat);
    for (int p = 0; p <= h->kmax; ++p) {
        double2* dst = static_cast<double2*>(Ahat) + (int64_t)p * m * m;
        if (dev) {
            CK(transpose_colmajor_to_rowmajor(h->st, m, m, h->dAhat + (int64_t)p * m * m, m, dst, m));
        } else {
            CK(transpose_colmajor_to_rowmajor(h->st, m, m, h->dAhat + (int64_t)p * m * m, m, h->dStage, m));
            CK(cudaMemcpyAsync(dst, h->dStage, sizeof(double2) * m * m, cudaMemcpyDeviceToHost, h->st));
            CK(cudaStreamSynchronize(h->st));
        }
    }
    CK(cudaStreamSynchronize(h->st));
    if (kmax_out) *kmax_out = h->kmax;
    return FEAST_NL_OK;
}

}  // extern "C"
