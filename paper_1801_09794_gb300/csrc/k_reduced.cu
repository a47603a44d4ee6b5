// Reduced problem of Steps 1-2 (Algorithm 1) on the GPU, and the small
// Cholesky factorisation used by the orthonormalisation of Step 5.
//
// Step 1 asks for the eigenpairs of the projected polynomial
//     Ahat(lambda) = sum_p lambda^p Ahat_p   (m x m, Ahat_p = Q^H A_p Q)
// "by a simple linearization" (Sec. 4.2).  GB300 runs FP64 at ~1/64 of its
// FP32 rate, and the eigenvalues of the linearisation come from a chain of
// dependent plane rotations (one SM), so the work is staged:
//   stage 1: eigenvalues of the block companion matrix
//            C = [[-Ahat_k^{-1} Ahat_{k-1} ... -Ahat_k^{-1} Ahat_0], [I 0 ..], ...]
//            (the first companion pencil of Sec. 2 with its leading block
//            inverted) by Householder reduction to Hessenberg form and the
//            implicit complex QR algorithm (multishift sweeps), in FP32;
//            Step 2 keeps the m Ritz values of smallest normalised radius; each
//            is refined in FP64 by Newton's method on Ahat(lambda) y = 0 with the
//            normalisation x^H y = 1 (nonlinear inverse iteration) with an FP32
//            factor, one CTA per pair, which also yields the Ritz vector y;
//   retry:   a pair whose Newton run was rejected (not converged, or moved
//            beyond 0.3 of the distance to its nearest neighbour without
//            landing clearly inside the kept region) runs again from the same
//            start with an FP64 factor -- except a pair clearly outside C, which
//            keeps its FP32 value and inverse-iteration vector;
//   stage 2: only if the retry failed too, or two kept values coincide --
//            clustered, ill-conditioned Ritz values that FP32 cannot separate --
//            the companion / Hessenberg / QR / selection runs in FP64 and
//            Newton polishes from those values.
// Every retry and stage-2 kernel reads the failure flags on the device and
// returns at once when they are clear, so the stream never waits on the host.
// Newton's fixed point is an exact eigenpair of the FP64 projected problem, so
// the kept pairs carry FP64 accuracy either way.
#include "internal.h"
#include <cfloat>

#include <cooperative_groups.h>

namespace fnl {
namespace {

template <typename R> struct cx;
template <> struct cx<float> { typedef float2 type; static __device__ float eps() { return FLT_EPSILON; }
                               static __device__ float tiny() { return FLT_MIN / FLT_EPSILON; } };
template <> struct cx<double> { typedef double2 type; static __device__ double eps() { return DBL_EPSILON; }
                                static __device__ double tiny() { return DBL_MIN / DBL_EPSILON; } };

__device__ __forceinline__ float2 cscale(float s, float2 a) { return make_float2(s * a.x, s * a.y); }
__device__ __forceinline__ double2 cscale(double s, double2 a) { return make_double2(s * a.x, s * a.y); }
template <typename C> __device__ __forceinline__ C czero();
template <> __device__ __forceinline__ float2 czero<float2>() { return make_float2(0.f, 0.f); }
template <> __device__ __forceinline__ double2 czero<double2>() { return make_double2(0.0, 0.0); }
template <typename C> __device__ __forceinline__ C cone();
template <> __device__ __forceinline__ float2 cone<float2>() { return make_float2(1.f, 0.f); }
template <> __device__ __forceinline__ double2 cone<double2>() { return make_double2(1.0, 0.0); }
__device__ __forceinline__ float2 cfrom(double2 a, float2*) { return make_float2((float)a.x, (float)a.y); }
__device__ __forceinline__ double2 cfrom(double2 a, double2*) { return a; }

template <typename R>
__device__ typename cx<R>::type csqrt_(typename cx<R>::type z) {
    typedef typename cx<R>::type C;
    R r = hypot(z.x, z.y);
    C out;
    if (r == (R)0) { out.x = 0; out.y = 0; return out; }
    R t = sqrt((R)0.5 * (fabs(z.x) + r));
    if (z.x >= (R)0) { out.x = t; out.y = z.y / ((R)2 * t); }
    else { out.x = fabs(z.y) / ((R)2 * t); out.y = copysign(t, z.y); }
    return out;
}

// Two eigenvalues of [[a, b], [c, d]].
template <typename R>
__device__ void eig2x2(typename cx<R>::type a, typename cx<R>::type b, typename cx<R>::type c,
                       typename cx<R>::type d, typename cx<R>::type* e1,
                       typename cx<R>::type* e2) {
    typedef typename cx<R>::type C;
    C h = cscale((R)0.5, a + d);
    C q = cscale((R)0.5, a - d);
    C disc = csqrt_<R>(q * q + b * c);
    *e1 = h + disc;
    *e2 = h - disc;
}

constexpr int kRedThreads = 1024;
constexpr size_t kRedSmemCap = 216 * 1024;   // dynamic shared memory cap of the single-CTA kernels
constexpr int kQrChunk = 16;        // rotations per window in the QR sweep (<= 29)
static_assert(kQrChunk >= 1 && kQrChunk <= 29, "lane t owns column k-1+t: a window spans kb+3 <= 32 columns");
// flags word shared by the stages (device memory)
constexpr int kNeed64 = 1;      // the FP64 companion / Hessenberg / QR stage runs
constexpr int kRetry64 = 2;     // some pairs retry Newton with an FP64 factor
// The FP64 stage runs for a pair that neither FP32- nor FP64-factor Newton could
// refine only once the previous iteration's largest relative residual inside C
// is at most this (Step 3's test then needs FP64-exact Ritz pairs).
constexpr double kExactStageRelres = 1e-6;

// The reduced problem seen by the refinement: the projected matrix polynomial
// (kmax >= 0: Ahat holds the kmax + 1 coefficients, stacked m x m), or general
// terms (kmax < 0): That(l) = sum_t f_t(l) G_t, G_t = Q^H A_t Q stacked m x m,
// f_t with the term's scale.
struct RedProblem {
    int kmax;
    const double2* Ahat;
    int nterms;
    const TermDev* terms;
    const double2* G;
    double c_re, c_im, ra, rb;      // the contour (Step 2's normalised radius)
};

// ---------------------------------------------------------------------------
// companion matrix: LU of Ahat_k, solve for the top block row (precision R).
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(kRedThreads) companion_kernel(
    int m, int kmax, const double2* __restrict__ Ahat, typename cx<R>::type* __restrict__ C,
    typename cx<R>::type* __restrict__ Lk, int* __restrict__ piv, int* redflag, int stage) {
    typedef typename cx<R>::type CT;
    if (stage == 2 && !(*redflag & kNeed64)) return;
    const int N = kmax * m;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int64_t mm = (int64_t)m * m;
    __shared__ int s_p;
    if (stage == 1) {
        __syncthreads();
        if (tid == 0) *redflag = 0;
    }
    for (int64_t e = tid; e < (int64_t)N * N; e += nt) {
        int r = (int)(e % N), c = (int)(e / N);
        CT v = czero<CT>();
        if (r < m) {
            int b = c / m, cc = c - b * m;
            v = cfrom(Ahat[(int64_t)(kmax - 1 - b) * mm + r + (int64_t)cc * m], (CT*)nullptr);
        } else if (c == r - m) {
            v = cone<CT>();
        }
        C[e] = v;
    }
    for (int64_t e = tid; e < mm; e += nt) Lk[e] = cfrom(Ahat[(int64_t)kmax * mm + e], (CT*)nullptr);
    __syncthreads();
    for (int c = 0; c < m; ++c) {
        if (tid < 32) {
            R best = (R)-1;
            int bi = c;
            for (int r = c + tid; r < m; r += 32) {
                R v = cabs1(Lk[r + c * m]);
                if (v > best) { best = v; bi = r; }
            }
            for (int o = 16; o > 0; o >>= 1) {
                R ov = __shfl_down_sync(0xffffffffu, best, o);
                int oi = __shfl_down_sync(0xffffffffu, bi, o);
                if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
            }
            if (tid == 0) { s_p = bi; piv[c] = bi; }
        }
        __syncthreads();
        int p = s_p;
        if (p != c)
            for (int cc = tid; cc < m; cc += nt) {
                CT a = Lk[c + cc * m];
                Lk[c + cc * m] = Lk[p + cc * m];
                Lk[p + cc * m] = a;
            }
        __syncthreads();
        CT inv = crcp(Lk[c + c * m]);
        int rem = m - c - 1;
        for (int r = c + 1 + tid; r < m; r += nt) Lk[r + c * m] = Lk[r + c * m] * inv;
        __syncthreads();
        for (int e = tid; e < rem * rem; e += nt) {
            int r = c + 1 + e % rem, cc = c + 1 + e / rem;
            Lk[r + cc * m] = cfms(Lk[r + c * m], Lk[c + cc * m], Lk[r + cc * m]);
        }
        __syncthreads();
    }
    // top block row <- -Ahat_k^{-1} (top block row): rows 0..m-1 of every column.
    // Interchanges per column, then substitution steps parallel over (row, column).
    for (int col = tid; col < N; col += nt) {
        CT* x = C + (int64_t)col * N;
        for (int c = 0; c < m; ++c) {
            int p = piv[c];
            if (p != c) { CT t = x[c]; x[c] = x[p]; x[p] = t; }
        }
    }
    __syncthreads();
    for (int i = 0; i < m - 1; ++i) {
        const int rows = m - 1 - i;
        for (int e = tid; e < rows * N; e += nt) {
            int r = i + 1 + e % rows, col = e / rows;
            CT* x = C + (int64_t)col * N;
            x[r] = cfms(Lk[r + i * m], x[i], x[r]);
        }
        __syncthreads();
    }
    for (int i = m - 1; i >= 0; --i) {
        const CT di = crcp(Lk[i + i * m]);
        for (int col = tid; col < N; col += nt) {
            CT* x = C + (int64_t)col * N;
            x[i] = x[i] * di;
        }
        __syncthreads();
        for (int e = tid; e < i * N; e += nt) {
            int r = e % i, col = e / i;
            CT* x = C + (int64_t)col * N;
            x[r] = cfms(Lk[r + i * m], x[i], x[r]);
        }
        __syncthreads();
    }
    for (int e = tid; e < m * N; e += nt) {
        int r = e % m, col = e / m;
        C[r + (int64_t)col * N] = -C[r + (int64_t)col * N];
    }
}

// ---------------------------------------------------------------------------
// Householder reduction of C (N x N, in place) to upper Hessenberg form.
// ---------------------------------------------------------------------------
// Columns c0..N-1 (those that fit) are held in shared memory for the whole
// reduction: at step j only columns > j are touched, so from j = c0 on every
// access is on chip.
template <typename R>
__global__ void __launch_bounds__(kRedThreads) hessenberg_kernel(int N, typename cx<R>::type* __restrict__ C,
                                                                 int c0, const int* redflag, int stage) {
    typedef typename cx<R>::type CT;
    if (stage == 2 && !(*redflag & kNeed64)) return;
    extern __shared__ unsigned char smem_raw[];
    CT* sv = reinterpret_cast<CT*>(smem_raw);   // N
    CT* wp = sv + N;                              // G x N partial products
    CT* S = wp + max(N, (int)blockDim.x);         // columns c0..N-1, N each
    auto colp = [&](int c) -> CT* { return c >= c0 ? S + (int64_t)(c - c0) * N : C + (int64_t)c * N; };
    {
        const int64_t ns = (int64_t)(N - c0) * N;
        for (int64_t e = threadIdx.x; e < ns; e += blockDim.x) S[e] = C[(int64_t)c0 * N + e];
        __syncthreads();
    }
    __shared__ R red[32];
    __shared__ CT s_alpha;
    __shared__ R s_beta;
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;
    const int nwarps = nt >> 5;
    const int G = (N <= nt) ? nt / N : 1;         // column groups of the right update
    const int g = (N <= nt) ? tid / N : 0;
    const int r0 = (N <= nt) ? tid % N : tid, rstep = (N <= nt) ? N : nt;
    for (int j = 0; j + 2 < N; ++j) {
        const int len = N - j - 1;
        CT* xcol = colp(j) + (j + 1);
        R s = 0;
        for (int r = tid; r < len; r += nt) s += cnorm2(xcol[r]);
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) red[warp] = s;
        __syncthreads();
        if (tid == 0) {
            R t = 0;
            for (int w = 0; w < nwarps; ++w) t += red[w];
            CT x0 = xcol[0];
            R ax0 = cabs(x0);
            R nx = sqrt(t);
            R tail = t - ax0 * ax0;
            if (nx == (R)0 || !(tail > (R)1e-30 * t)) {
                s_beta = 0;
            } else {
                CT ph;
                if (ax0 > (R)0) { ph.x = x0.x / ax0; ph.y = x0.y / ax0; }
                else { ph.x = 1; ph.y = 0; }
                CT alpha;
                alpha.x = -ph.x * nx;
                alpha.y = -ph.y * nx;
                CT v0 = x0 - alpha;
                s_alpha = alpha;
                s_beta = (R)2 / (tail + cnorm2(v0));
                sv[0] = v0;
            }
        }
        __syncthreads();
        const R beta = s_beta;
        if (beta == (R)0) continue;
        for (int r = 1 + tid; r < len; r += nt) sv[r] = xcol[r];
        __syncthreads();
        for (int cc = j + 1 + warp; cc < N; cc += nwarps) {
            CT* col = colp(cc) + (j + 1);
            CT w = czero<CT>();
            for (int r = lane; r < len; r += 32) w = cfma(cconj(sv[r]), col[r], w);
            for (int o = 16; o > 0; o >>= 1) {
                w.x += __shfl_xor_sync(0xffffffffu, w.x, o);
                w.y += __shfl_xor_sync(0xffffffffu, w.y, o);
            }
            w = cscale(beta, w);
            for (int r = lane; r < len; r += 32) col[r] = cfms(sv[r], w, col[r]);
        }
        if (tid == 0) xcol[0] = s_alpha;
        for (int r = 1 + tid; r < len; r += nt) xcol[r] = czero<CT>();
        __syncthreads();
        // right update C[:, j+1:] -= beta (C[:, j+1:] v) v^H: the columns are
        // dealt round G thread groups (every warp busy even when N is small),
        // the partial products meet in shared memory
        for (int r = r0; r < N; r += rstep) {
            CT w = czero<CT>();
            if (g < G)
                for (int c = g; c < len; c += G) w = cfma(colp(j + 1 + c)[r], sv[c], w);
            if (g < G) wp[g * N + r] = w;
        }
        __syncthreads();
        for (int r = r0; r < N; r += rstep) {
            if (g >= G) break;
            CT w = czero<CT>();
            for (int q = 0; q < G; ++q) w = w + wp[q * N + r];
            w = cscale(beta, w);
            for (int c = g; c < len; c += G) {
                CT* p = colp(j + 1 + c) + r;
                *p = cfms(w, cconj(sv[c]), *p);
            }
        }
        __syncthreads();
    }
    __syncthreads();
    const int64_t ns = (int64_t)(N - c0) * N;
    for (int64_t e = threadIdx.x; e < ns; e += blockDim.x) C[(int64_t)c0 * N + e] = S[e];
}

// First column the Hessenberg kernel holds in shared memory, and its launch
// size: as many trailing columns as fit beside the vector and the partial
// products under the kernels' shared-memory cap.
template <typename R>
void hessenberg_launch_shape(int N, int* c0, size_t* smem) {
    const size_t base = sizeof(typename cx<R>::type) * ((size_t)N + (size_t)max(N, kRedThreads));
    const size_t cap = kRedSmemCap;
    const size_t col = sizeof(typename cx<R>::type) * (size_t)N;
    const size_t fit = base < cap ? (cap - base) / col : 0;
    const int ncs = (int)min((size_t)N, fit);
    *c0 = N - ncs;
    *smem = base + (size_t)ncs * col;
}

// ---------------------------------------------------------------------------
// FP32 stage: the companion matrix by several CTAs, its Householder reduction
// to Hessenberg form by a thread-block cluster.
// ---------------------------------------------------------------------------
constexpr int kCompCols = 32;        // companion columns per CTA (one warp each)
constexpr int kCompThreads = 32 * kCompCols;

// CTA b forms columns [b kCompCols, ...) of C: every CTA factors Ahat_k in
// shared memory (the same arithmetic, so the same factors, in each), then each
// warp solves one column of the top block row and writes the whole column of C.
// The per-element operation order is that of companion_kernel: LU with partial
// pivoting on cabs1 (lowest row on ties), forward substitution with the unit L,
// back substitution multiplying by the reciprocal pivot, then negation.
__global__ void __launch_bounds__(kCompThreads) companion_cols_kernel(
    int m, int kmax, const double2* __restrict__ Ahat, float2* __restrict__ C, int* redflag) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int ld = m + 1;                                       // see chol_inverse_kernel
    float2* Lk = reinterpret_cast<float2*>(smem_raw);          // m x m, col-major, ld m + 1
    float2* X = Lk + (size_t)ld * m;                            // m x kCompCols
    int* piv = reinterpret_cast<int*>(X + (size_t)m * kCompCols);
    __shared__ int s_p;
    const int N = kmax * m;
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;
    const int64_t mm = (int64_t)m * m;
    if (blockIdx.x == 0 && tid == 0) *redflag = 0;
    for (int c = warp; c < m; c += kCompCols)
        for (int r = lane; r < m; r += 32) {
            const double2 a = Ahat[(int64_t)kmax * mm + r + (int64_t)c * m];
            Lk[r + c * ld] = make_float2((float)a.x, (float)a.y);
        }
    const int col = blockIdx.x * kCompCols + warp;              // this warp's column of C
    const bool has = col < N;
    if (has) {
        const int b = col / m, cc = col - b * m;
        const double2* src = Ahat + (int64_t)(kmax - 1 - b) * mm + (int64_t)cc * m;
        for (int r = lane; r < m; r += 32) X[r + (size_t)warp * m] = make_float2((float)src[r].x, (float)src[r].y);
    }
    __syncthreads();
    for (int c = 0; c < m; ++c) {
        if (warp == 0) {
            float best = -1.0f;
            int bi = c;
            for (int r = c + lane; r < m; r += 32) {
                const float v = cabs1(Lk[r + c * ld]);
                if (v > best) { best = v; bi = r; }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const float ov = __shfl_down_sync(0xffffffffu, best, o);
                const int oi = __shfl_down_sync(0xffffffffu, bi, o);
                if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
            }
            if (lane == 0) { s_p = bi; piv[c] = bi; }
        }
        __syncthreads();
        const int p = s_p;
        if (p != c)
            for (int cc = tid; cc < m; cc += nt) {
                const float2 a = Lk[c + cc * ld];
                Lk[c + cc * ld] = Lk[p + cc * ld];
                Lk[p + cc * ld] = a;
            }
        __syncthreads();
        const float2 inv = crcp(Lk[c + c * ld]);
        for (int r = c + 1 + tid; r < m; r += nt) Lk[r + c * ld] = Lk[r + c * ld] * inv;
        __syncthreads();
        for (int cc = c + 1 + warp; cc < m; cc += kCompCols) {     // warp per column
            const float2 u = Lk[c + cc * ld];
            for (int r = c + 1 + lane; r < m; r += 32)
                Lk[r + cc * ld] = cfms(Lk[r + c * ld], u, Lk[r + cc * ld]);
        }
        __syncthreads();
    }
    if (!has) return;
    float2* x = X + (size_t)warp * m;
    if (lane == 0)
        for (int c = 0; c < m; ++c) {
            const int p = piv[c];
            if (p != c) { const float2 t = x[c]; x[c] = x[p]; x[p] = t; }
        }
    __syncwarp();
    for (int i = 0; i < m - 1; ++i) {
        const float2 xi = x[i];
        for (int r = i + 1 + lane; r < m; r += 32) x[r] = cfms(Lk[r + i * ld], xi, x[r]);
        __syncwarp();
    }
    for (int i = m - 1; i >= 0; --i) {
        if (lane == 0) x[i] = x[i] * crcp(Lk[i + i * ld]);
        __syncwarp();
        const float2 xi = x[i];
        for (int r = lane; r < i; r += 32) x[r] = cfms(Lk[r + i * ld], xi, x[r]);
        __syncwarp();
    }
    float2* out = C + (int64_t)col * N;
    for (int r = lane; r < N; r += 32)
        out[r] = r < m ? -x[r] : make_float2(r == col + m ? 1.0f : 0.0f, 0.0f);
}

size_t companion_cols_smem(int m) {
    return sizeof(float2) * ((size_t)(m + 1) * m + (size_t)m * kCompCols) + sizeof(int) * (size_t)m;
}

// Householder reduction of C (N x N, FP32, in place) to upper Hessenberg form
// by a cluster of CS CTAs that hold the matrix in distributed shared memory:
// CTA q owns the columns j = q (mod CS).  Step j (owner o = j mod CS):
//   1. the owner forms the reflector P = I - beta v v^H from column j (v zero
//      in rows <= j) and writes v and beta into every CTA's shared memory;
//   2. every CTA forms w_c = v^H H(:, c) for its columns c > j and its share
//      of y = H v (the sum over its columns), and writes the share into every
//      CTA;
//   3. every CTA sums the shares in rank order, gamma = v^H y, and updates its
//      columns by the two-sided reflection
//         H(r, c) <- H(r, c) - beta v_r w_c - beta (y_r - beta gamma v_r) conj(v_c).
// Two cluster barriers per column; v is double-buffered because the owner of
// column j + 1 may write it while other CTAs still read column j's.
constexpr int kHcThreads = 1024;
constexpr int kHcMaxN = 320;         // largest order the cluster reduction takes (registers per lane)

template <int CS>
__global__ void __cluster_dims__(CS, 1, 1) __launch_bounds__(kHcThreads)
hess_cluster_kernel(int N, float2* __restrict__ C) {
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    const int q = (int)cluster.block_rank();
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;
    const int nw = nt >> 5;
    const int ncl = (N - q + CS - 1) / CS;             // own columns j = q + CS lc
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* S = reinterpret_cast<float2*>(smem_raw);   // ncl x N, column-major
    float2* vbuf = S + (size_t)ncl * N;                // 2 x N
    float2* ypart = vbuf + 2 * (size_t)N;              // CS x N: the CTAs' shares of y
    float2* wv = ypart + (size_t)CS * N;               // ncl
    float2* yv = wv + ncl;                             // N
    float2* ywarp = yv + N;                            // nw x N: the warps' shares
    __shared__ float s_beta[2];
    __shared__ float2 s_gamma;
    for (int lc = warp; lc < ncl; lc += nw)
        for (int r = lane; r < N; r += 32) S[(size_t)lc * N + r] = C[(int64_t)(q + CS * lc) * N + r];
    __syncthreads();
    cluster.sync();
    for (int j = 0; j + 2 < N; ++j) {
        const int o = j % CS, buf = j & 1, len = N - j - 1;
        float2* v = vbuf + (size_t)buf * N;             // v[i] <-> row j + 1 + i
        if (q == o && warp == 0) {
            float2* col = S + (size_t)(j / CS) * N + (j + 1);
            float sq = 0.0f;
            for (int r = lane; r < len; r += 32) sq += cnorm2(col[r]);
            for (int off = 16; off > 0; off >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, off);
            const float2 x0 = col[0];
            const float ax0 = cabs(x0), nx = sqrtf(sq), tail = sq - ax0 * ax0;
            float beta = 0.0f;
            float2 alpha = make_float2(0.0f, 0.0f), v0 = make_float2(0.0f, 0.0f);
            if (nx > 0.0f && tail > 1e-30f * sq) {
                const float2 ph = ax0 > 0.0f ? make_float2(x0.x / ax0, x0.y / ax0) : make_float2(1.0f, 0.0f);
                alpha = make_float2(-ph.x * nx, -ph.y * nx);
                v0 = x0 - alpha;
                beta = 2.0f / (tail + cnorm2(v0));
            }
#pragma unroll
            for (int d = 0; d < CS; ++d) {
                float2* vd = cluster.map_shared_rank(v, d);
                for (int r = lane; r < len; r += 32) vd[r] = r == 0 ? v0 : col[r];
                if (lane == 0) *cluster.map_shared_rank(&s_beta[buf], d) = beta;
            }
            __syncwarp();
            if (beta != 0.0f)
                for (int r = lane; r < len; r += 32) col[r] = r == 0 ? alpha : make_float2(0.0f, 0.0f);
        }
        cluster.sync();                                 // v, beta of column j everywhere
        const float beta = s_beta[buf];
        const int lc0 = (j + CS - q) / CS;              // first own column > j
        if (beta != 0.0f) {
            // one pass per own column c > j (a warp each): w_c = v^H H(:, c) and
            // the column's share of y = H v, kept per warp in registers
            float2 yl[(kHcMaxN + 31) / 32];
#pragma unroll
            for (int q2 = 0; q2 < (kHcMaxN + 31) / 32; ++q2) yl[q2] = make_float2(0.0f, 0.0f);
            for (int lc = lc0 + warp; lc < ncl; lc += nw) {
                const float2* hc = S + (size_t)lc * N;
                const float2 vc = v[q + CS * lc - j - 1];
                float2 w = make_float2(0.0f, 0.0f);
#pragma unroll
                for (int q2 = 0; q2 < (kHcMaxN + 31) / 32; ++q2) {
                    const int r = lane + 32 * q2;
                    if (r < N) {
                        const float2 h = hc[r];
                        yl[q2] = cfma(h, vc, yl[q2]);
                        if (r > j) w = cfma(cconj(v[r - j - 1]), h, w);
                    }
                }
                for (int off = 16; off > 0; off >>= 1) {
                    w.x += __shfl_xor_sync(0xffffffffu, w.x, off);
                    w.y += __shfl_xor_sync(0xffffffffu, w.y, off);
                }
                if (lane == 0) wv[lc] = w;
            }
#pragma unroll
            for (int q2 = 0; q2 < (kHcMaxN + 31) / 32; ++q2) {
                const int r = lane + 32 * q2;
                if (r < N) ywarp[(size_t)warp * N + r] = yl[q2];
            }
            __syncthreads();
            // the CTA's share of y (warps summed in order) into every CTA
            for (int r = tid; r < N; r += nt) {
                float2 y = ywarp[r];
                for (int w2 = 1; w2 < nw; ++w2) y = y + ywarp[(size_t)w2 * N + r];
#pragma unroll
                for (int d = 0; d < CS; ++d) cluster.map_shared_rank(ypart + (size_t)q * N, d)[r] = y;
            }
        }
        cluster.sync();                                 // every share of y everywhere
        if (beta != 0.0f) {
            for (int r = tid; r < N; r += nt) {
                float2 y = ypart[r];
                for (int d = 1; d < CS; ++d) y = y + ypart[(size_t)d * N + r];
                yv[r] = y;
            }
            __syncthreads();
            if (warp == 0) {
                float2 g = make_float2(0.0f, 0.0f);
                for (int i = lane; i < len; i += 32) g = cfma(cconj(v[i]), yv[j + 1 + i], g);
                for (int off = 16; off > 0; off >>= 1) {
                    g.x += __shfl_xor_sync(0xffffffffu, g.x, off);
                    g.y += __shfl_xor_sync(0xffffffffu, g.y, off);
                }
                if (lane == 0) s_gamma = g;
            }
            __syncthreads();
            const float2 bg = beta * s_gamma;
            for (int lc = lc0 + warp; lc < ncl; lc += nw) {   // warp per own column
                const int c = q + CS * lc;
                const float2 bvc = beta * cconj(v[c - j - 1]);
                const float2 bw = beta * wv[lc];
                float2* hc = S + (size_t)lc * N;
                for (int r = lane; r < N; r += 32) {
                    const float2 vr = r > j ? v[r - j - 1] : make_float2(0.0f, 0.0f);
                    const float2 yt = cfms(bg, vr, yv[r]);             // y_r - beta gamma v_r
                    float2 h = hc[r];
                    h = cfms(vr, bw, h);
                    h = cfms(yt, bvc, h);
                    hc[r] = h;
                }
            }
        }
        __syncthreads();
    }
    cluster.sync();
    for (int lc = warp; lc < ncl; lc += nw)
        for (int r = lane; r < N; r += 32) C[(int64_t)(q + CS * lc) * N + r] = S[(size_t)lc * N + r];
}

size_t hess_cluster_smem(int N, int CS) {
    const size_t ncl = (size_t)(N + CS - 1) / CS;
    return sizeof(float2) * (ncl * N + 2 * (size_t)N + (size_t)CS * N + ncl + (size_t)N +
                             (size_t)(kHcThreads / 32) * N);
}

constexpr size_t kHcSmemCap = 200 * 1024;
// Cluster size for the FP32 Hessenberg reduction of order N (0: the matrix does
// not fit eight CTAs, or N is too small to pay; the single-CTA kernel runs).
int hess_cluster_size(int N) {
    if (N < 64 || N > kHcMaxN) return 0;
    if (hess_cluster_smem(N, 4) <= kHcSmemCap) return 4;
    if (hess_cluster_smem(N, 8) <= kHcSmemCap) return 8;
    return 0;
}

// Packed Hessenberg storage with one bulge row: column j holds rows 0..j+2.
#define PK(i, j) ((((j) * ((j) + 5)) >> 1) + (i))

constexpr int kQrThreads = 256;
constexpr int kMsShifts = 8;                  // bulges of a multishift sweep
constexpr int kMsWarps = kQrThreads / 32 / kMsShifts;   // warps per bulge
static_assert(kMsWarps >= 1 && kMsShifts * kMsWarps * 32 == kQrThreads, "whole warps per bulge");
// Multishift sweeps without a deflation at the bottom of the active block after
// which the block continues with single-shift sweeps until the next deflation
// (a safety net: the chain has no deflation checks inside the sweep; a healthy
// block deflates within a few sweeps).
constexpr int kMsMaxStall = 10;
constexpr int kSmallMax = 32;      // active blocks up to this order go to one warp
constexpr int kSmallLd = 33;       // leading dimension of that dense copy (bank spread)

template <typename R> struct givens_range;
template <> struct givens_range<float> { static __device__ float lo() { return 1e-30f; }
                                         static __device__ float hi() { return 1e30f; } };
template <> struct givens_range<double> { static __device__ double lo() { return 1e-280; }
                                          static __device__ double hi() { return 1e280; } };

// The rotation of givens() when |x|^2 + |y|^2 is tiny or huge: both are divided
// by their largest component first, so no square underflows or overflows (a
// collapsed bulge of a multishift sweep reaches |x|, |y| ~ 1e-21, where
// 1 / (|x| rho) overflows FP32).  Any common factor cancels in c and s.
template <typename R>
__device__ __noinline__ void givens_scaled(typename cx<R>::type x, typename cx<R>::type y, R& c,
                                           typename cx<R>::type& s) {
    typedef typename cx<R>::type CT;
    const R mx = fmax(fmax(fabs(x.x), fabs(x.y)), fmax(fabs(y.x), fabs(y.y)));
    if (!(mx > (R)0) || !isfinite(mx)) { c = 1; s = czero<CT>(); return; }
    CT xs, ys;
    xs.x = x.x / mx; xs.y = x.y / mx;
    ys.x = y.x / mx; ys.y = y.y / mx;
    const R irho = (R)1 / sqrt(cnorm2(xs) + cnorm2(ys));   // the sum lies in [1, 2]
    const R ax = sqrt(cnorm2(xs));
    CT ph;
    if (ax > (R)0) { ph.x = xs.x / ax; ph.y = xs.y / ax; }
    else { ph.x = 1; ph.y = 0; }
    c = ax * irho;
    s = cscale(irho, ph * cconj(ys));
}

// G = [[c, s], [-conj(s), c]] with c real maps (x, y) to (rho, 0).  Written
// with selects (no branches) so that a sweep step stays one basic block; the
// rare tiny or huge (x, y) go to givens_scaled (the branch is uniform: every
// lane of a warp computes the same rotation).
template <typename R>
__device__ __forceinline__ void givens(typename cx<R>::type x, typename cx<R>::type y, R& c,
                                       typename cx<R>::type& s) {
    const R nx = cnorm2(x), ny = cnorm2(y);
    if (!(nx + ny >= givens_range<R>::lo() && nx + ny <= givens_range<R>::hi())) {
        if (nx + ny == (R)0) { c = 1; s = czero<typename cx<R>::type>(); return; }
        givens_scaled<R>(x, y, c, s);
        return;
    }
    const R irho = rsqrt(nx + ny), ix = rsqrt(nx), iy = rsqrt(ny);
    const R f = ix * irho;
    const typename cx<R>::type xy = x * cconj(y);
    const bool yz = ny == (R)0, xz = nx == (R)0;
    c = yz ? (R)1 : (xz ? (R)0 : nx * ix * irho);  // |x| / rho
    s.x = yz ? (R)0 : (xz ? y.x * iy : f * xy.x);  // (x/|x|) conj(y) / rho
    s.y = yz ? (R)0 : (xz ? -y.y * iy : f * xy.y);
    // rsqrt is approximate (a few ulp), so c^2 + |s|^2 = 1 + d with d of that
    // size, and tens of thousands of such rotations per QR random-walk into the
    // eigenvalues (3x coarser in FP32).  One Newton step on the normalisation
    // leaves d = O(ulp^2).
    const R g = (R)1.5 - (R)0.5 * (c * c + cnorm2(s));
    c *= g;
    s.x *= g;
    s.y *= g;
}

// Eigenvalues of the ns x ns (ns <= 32) Hessenberg matrix S (column-major, ld
// kSmallLd, overwritten) by single-shift complex QR, one warp: lane j owns
// column j in the row rotations and row j in the column rotations.  Returns the
// number of sweeps, negated when the iteration cap was reached.
template <typename R>
__device__ int small_hess_eig(typename cx<R>::type* S, int ns, typename cx<R>::type* ev) {
    typedef typename cx<R>::type CT;
    const int lane = threadIdx.x & 31;
    const R eps = cx<R>::eps(), tiny = cx<R>::tiny();
#define SS(i, j) S[(i) + (j) * kSmallLd]
    int hi = ns - 1, its = 0, total = 0;
    while (hi >= 0) {
        if (hi == 0) { if (lane == 0) ev[0] = SS(0, 0); __syncwarp(); break; }
        bool neg = false;
        if (lane >= 1 && lane <= hi) {
            const R h = cabs1(SS(lane, lane - 1));
            const R sd = cabs1(SS(lane - 1, lane - 1)) + cabs1(SS(lane, lane));
            neg = (h <= eps * sd) || (h <= tiny);
        }
        const unsigned bal = __ballot_sync(0xffffffffu, neg);
        const int l = bal ? 31 - __clz(bal) : 0;
        __syncwarp();
        if (l > 0 && lane == 0) SS(l, l - 1) = czero<CT>();
        __syncwarp();
        if (l == hi) { if (lane == 0) ev[hi] = SS(hi, hi); __syncwarp(); --hi; its = 0; continue; }
        if (l == hi - 1) {
            CT e1, e2;
            eig2x2<R>(SS(hi - 1, hi - 1), SS(hi - 1, hi), SS(hi, hi - 1), SS(hi, hi), &e1, &e2);
            if (lane == 0) { ev[hi - 1] = e1; ev[hi] = e2; }
            __syncwarp();
            hi -= 2; its = 0;
            continue;
        }
        ++its;
        if (++total > 30 * ns) {       // iteration cap: report, keep the diagonal
            for (int i = lane; i <= hi; i += 32) ev[i] = SS(i, i);
            __syncwarp();
            return -total;
        }
        CT mu;
        const CT d = SS(hi, hi);
        if (its % 11 == 10) { mu = d; mu.x += (R)0.75 * cabs(SS(hi, hi - 1)); }
        else {
            CT e1, e2;
            eig2x2<R>(SS(hi - 1, hi - 1), SS(hi - 1, hi), SS(hi, hi - 1), d, &e1, &e2);
            mu = (cabs1(e1 - d) <= cabs1(e2 - d)) ? e1 : e2;
        }
        for (int k = l; k < hi; ++k) {
            CT x, y;
            if (k == l) { x = SS(l, l) - mu; y = SS(l + 1, l); }
            else        { x = SS(k, k - 1); y = SS(k + 1, k - 1); }
            R c;
            CT s;
            givens<R>(x, y, c, s);
            __syncwarp();
            if (lane >= max(l, k - 1) && lane <= hi) {
                const CT h1 = SS(k, lane), h2 = SS(k + 1, lane);
                SS(k, lane) = cscale(c, h1) + s * h2;
                SS(k + 1, lane) = (lane == k - 1) ? czero<CT>() : cscale(c, h2) - cconj(s) * h1;
            }
            __syncwarp();
            if (lane >= l && lane <= min(k + 2, hi)) {
                const CT h1 = SS(lane, k), h2 = SS(lane, k + 1);
                SS(lane, k) = cscale(c, h1) + cconj(s) * h2;
                SS(lane, k + 1) = cscale(c, h2) - s * h1;
            }
            __syncwarp();
        }
    }
#undef SS
    return total;
}

// An integer that orders like the double v (v not NaN; -0 taken as +0).
__device__ __forceinline__ unsigned long long order_key(double v) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v + 0.0);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

// One window of a single-shift sweep over the active block l..hi: rotations
// G_kk, kk = k..k+kb-1 (kb <= 29), one warp.  The matrix must hold the state
// after rotation k-1 in full; on return it holds the state after rotation
// k+kb-1 except for what the CTA applies afterwards (the row rotations on the
// columns right of the window, the column rotations on rows <= kk).
//
// Every lane carries the bulge neighbourhood of the current rotation in
// registers (x = H(kk,kk-1), y = H(kk+1,kk-1) [x = H(l,l) - mu, y = H(l+1,l)
// for kk = l], P = H(kk,kk), Qv = H(kk+1,kk), U = H(kk,kk+1), D = H(kk+1,kk+1),
// E = H(kk+2,kk+1)) and computes the rotation itself, so a step's only serial
// dependence is rotation -> next bulge.  Lane t owns column k-1+t.  At step kk
// it writes that column's row kk: the final row-rotation value while the
// column is right of the frontier (it keeps the carry H(kk+1, .) meanwhile),
// then H(kk,kk+1), H(kk,kk) and the new subdiagonal H(kk,kk-1) as the frontier
// passes; it hands H(kk+1,kk+2), H(kk+2,kk+2), H(kk+3,kk+2) to all lanes when
// its column enters the frontier.  A column rotation only has to reach rows
// kk+1, kk+2 before the next row rotation; on rows <= kk it is deferred.  The
// bulge slot H(kk+1,kk-1) is not cleared: it is read only as the opening y of
// the next window, which the closing writes below provide.  Each matrix
// location (shared or global memory) is read and written by its column's lane
// only after the opening broadcast reads, so the steps need no warp barrier.
template <typename R, int KB>
__device__ __forceinline__ void qr_window(typename cx<R>::type* H, int l, int hi, int k, int kb,
                                          int w1, typename cx<R>::type mu, R* s_c,
                                          typename cx<R>::type* s_s) {
    typedef typename cx<R>::type CT;
    const unsigned full = 0xffffffffu;
    const int t = threadIdx.x & 31;
    const CT zero = czero<CT>();
    CT P = H[PK(k, k)], Qv = H[PK(k + 1, k)];
    CT x, y;
    if (k == l) { x = P - mu; y = Qv; }
    else        { x = H[PK(k, k - 1)]; y = H[PK(k + 1, k - 1)]; }
    CT U = H[PK(k, k + 1)], D = H[PK(k + 1, k + 1)];
    CT E = (k + 2 <= hi) ? H[PK(k + 2, k + 1)] : zero;
    const int col = k - 1 + t;
    const bool own = col >= l && col <= w1;
    CT* pc = H + (own ? PK(0, col) : 0);          // pc[i] = H(i, col)
    CT a = zero, Dl = zero, El = zero;
    if (own && t >= 3) {
        a = pc[k];
        Dl = pc[col];
        if (col + 1 <= hi) El = pc[col + 1];
    }
    __syncwarp();                      // the broadcast reads above come first
    const int nsteps = KB ? KB : kb;
#pragma unroll 4
    for (int r = 0; r < nsteps; ++r) {
        const int kk = k + r;
        const bool carry = own && t >= r + 3;
        const CT h = carry ? pc[kk + 1] : zero;
        R c;
        CT s;
        givens<R>(x, y, c, s);
        if (t == 0) { s_c[r] = c; s_s[r] = s; }
        const CT R00 = cscale(c, P) + s * Qv, R10 = cscale(c, Qv) - cconj(s) * P;
        const CT R01 = cscale(c, U) + s * D, R11 = cscale(c, D) - cconj(s) * U;
        const CT rho = cscale(c, x) + s * y;
        const CT out = cscale(c, a) + s * h;
        const CT val = carry ? out : (t == r + 2 ? R01 : (t == r + 1 ? R00 : rho));
        if (own && t >= r) pc[kk] = val;
        if (carry) a = cscale(c, h) - cconj(s) * a;
        // column rotation kk on rows kk+1, kk+2 (H(kk+2, kk) was zero)
        x = cscale(c, R10) + cconj(s) * R11;
        P = cscale(c, R11) - s * R10;
        y = cconj(s) * E;
        Qv = cscale(c, E);
        // column kk+2 (lane r+3) enters the frontier
        U.x = __shfl_sync(full, a.x, r + 3);  U.y = __shfl_sync(full, a.y, r + 3);
        D.x = __shfl_sync(full, Dl.x, r + 3); D.y = __shfl_sync(full, Dl.y, r + 3);
        E.x = __shfl_sync(full, El.x, r + 3); E.y = __shfl_sync(full, El.y, r + 3);
    }
    const int kl = k + nsteps - 1;
    const bool more = kl + 2 <= hi;
    if (t == nsteps)     { pc[kl + 1] = x; if (more) pc[kl + 2] = y; }
    if (t == nsteps + 1) { pc[kl + 1] = P; if (more) pc[kl + 2] = Qv; }
    if (t == nsteps + 2 && more) pc[kl + 1] = a;
}

// ---------------------------------------------------------------------------
// Eigenvalues of the Hessenberg matrix by the implicit QR algorithm, then Step
// 2's selection.  Blocks of order <= kSmallMax: one warp on a dense copy,
// single shifts.  Larger active blocks:
//  * MS (the FP32 stage): small-bulge multishift sweeps.  The kMsShifts
//    eigenvalues of the trailing kMsShifts x kMsShifts block are the shifts;
//    each opens a single-shift bulge at the top of the block, three rows
//    behind the previous one, and the chain is chased down in lockstep, one
//    warp per bulge.  Bulges three rows apart act on disjoint row pairs and
//    disjoint column pairs, so at each step every bulge applies its row
//    rotation (across the whole active block), the CTA synchronises, every
//    bulge applies its column rotation, and the CTA synchronises again; left
//    and right rotations commute, so this equals the one-by-one chase in exact
//    arithmetic.  (A single-shift chase is one dependent rotation after
//    another on one warp, ~470 cycles per rotation on GB300; the chain keeps
//    eight warps busy at the cost of ~1.4x the rotations: ~6,000 chain steps
//    instead of ~27,000 rotations for the 192 x 192 companion matrices of the
//    n = 4096 QEP, with the same FP32 eigenvalue accuracy.)
//    After kMsMaxStall multishift sweeps without a deflation the block goes on
//    with single-shift sweeps until the next one.
//  * otherwise (the FP64 fallback stage): single-shift sweeps; one warp chases
//    the bulge through windows of kQrChunk rotations, the CTA applies each
//    window's rotations to the rest of the block.
// ---------------------------------------------------------------------------
template <typename R, bool SMEM, bool MS = false>
__global__ void __launch_bounds__(kQrThreads) qr_select_kernel(
    int N, int m0, const typename cx<R>::type* __restrict__ C, typename cx<R>::type* Hglobal,
    double c_re, double c_im, double ra, double rb, double2* __restrict__ lam0,
    double* __restrict__ gap, const int* redflag, int stage, IterStatus* status) {
    typedef typename cx<R>::type CT;
    if (stage == 2 && !(*redflag & kNeed64)) return;
    extern __shared__ unsigned char smem_raw[];
    CT* ev = reinterpret_cast<CT*>(smem_raw);   // N
    CT* Ssm = ev + N;                            // kSmallLd x kSmallMax
    // the packed matrix in shared memory when it fits (fixed at compile time, so
    // the accesses are shared-memory ones), else in the global workspace
    CT* H = SMEM ? Ssm + kSmallLd * kSmallMax : Hglobal;
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31;
#define HH(i, j) H[PK(i, j)]
    for (int j = tid; j < N; j += nt)
        for (int i = 0; i <= j + 2; ++i)
            HH(i, j) = (i < N && i <= j + 1) ? C[i + (int64_t)j * N] : czero<CT>();
    __syncthreads();
    __shared__ R s_c[kQrChunk];
    __shared__ CT s_s[kQrChunk];
    __shared__ R s_red[32];
    const int warp = tid >> 5;
    const R eps = cx<R>::eps();
    // deflation: a subdiagonal is negligible below eps times its diagonal
    // neighbours or below eps^2 ||H||_F (the kept values are polished in FP64)
    R hn = 0;
    for (int j = tid; j < N; j += nt)
        for (int i = 0; i <= j + 1 && i < N; ++i) hn += cnorm2(HH(i, j));
    for (int o = 16; o > 0; o >>= 1) hn += __shfl_down_sync(0xffffffffu, hn, o);
    if (lane == 0) s_red[warp] = hn;
    __syncthreads();
    hn = 0;
    for (int w = 0; w < (nt >> 5); ++w) hn += s_red[w];
    const R tiny = fmax(cx<R>::tiny(), eps * eps * sqrt(hn));
    int hi = N - 1, its = 0, total = 0;
    bool failed = false;
    while (hi >= 0) {
        if (hi == 0) {
            if (tid == 0) ev[0] = HH(0, 0);
            break;
        }
        int l = 0;
        for (int base = hi; base >= 1; base -= 32) {
            int i = base - lane;
            bool neg = false;
            if (i >= 1) {
                R h = cabs1(HH(i, i - 1));
                R sd = cabs1(HH(i - 1, i - 1)) + cabs1(HH(i, i));
                neg = (h <= eps * sd) || (h <= tiny);
            }
            unsigned b = __ballot_sync(0xffffffffu, neg);
            if (b) { l = base - (__ffs(b) - 1); break; }
        }
        __syncthreads();
        if (l > 0 && tid == 0) HH(l, l - 1) = czero<CT>();
        if (l == hi) {
            if (tid == 0) ev[hi] = HH(hi, hi);
            __syncthreads();
            hi -= 1; its = 0;
            continue;
        }
        if (l == hi - 1) {
            CT e1, e2;
            eig2x2<R>(HH(hi - 1, hi - 1), HH(hi - 1, hi), HH(hi, hi - 1),
                      HH(hi, hi), &e1, &e2);
            if (tid == 0) { ev[hi - 1] = e1; ev[hi] = e2; }
            __syncthreads();
            hi -= 2; its = 0;
            continue;
        }
        ++its; ++total;
        if (total > 40 * N) { failed = true; break; }
        if (hi - l < kSmallMax) {
            // ---- the whole active block (order <= kSmallMax) by one warp in a
            // dense copy: same single-shift QR, no CTA-wide barriers
            const int ns = hi - l + 1;
            if (warp == 0) {
                for (int j = lane; j < ns; j += 32)
                    for (int i = 0; i < ns; ++i)
                        Ssm[i + j * kSmallLd] = (i <= j + 1) ? HH(l + i, l + j) : czero<CT>();
                __syncwarp();
                const int sw = small_hess_eig<R>(Ssm, ns, ev + l);
                if (lane == 0) {
                    if (sw < 0) atomicOr(&status->flags, 1);
                    s_red[0] = (R)(sw < 0 ? -sw : sw);
                }
            }
            __syncthreads();
            total += (int)s_red[0];
            hi = l - 1;
            its = 0;
            __syncthreads();
            continue;
        }
        if (MS && its <= kMsMaxStall) {
            // ---- small-bulge multishift sweep
            __shared__ CT s_sig[kMsShifts];
            const int ns = kMsShifts;
            if (warp == 0) {
                const int s0 = hi - ns + 1;
                for (int j = lane; j < ns; j += 32)
                    for (int i = 0; i < ns; ++i)
                        Ssm[i + j * kSmallLd] = (i <= j + 1) ? HH(s0 + i, s0 + j) : czero<CT>();
                __syncwarp();
                small_hess_eig<R>(Ssm, ns, s_sig);
                if (lane == 0) {
                    const CT d = HH(hi, hi);
                    if (its % 6 == 5) {            // exceptional shifts around the corner entry
                        const R rad = (R)0.75 * cabs(HH(hi, hi - 1));
                        for (int q = 0; q < ns; ++q) {
                            double sn_, cs_;
                            sincos(2.0 * M_PI * q / ns, &sn_, &cs_);
                            s_sig[q] = d + cmake<CT>(rad * cs_, rad * sn_);
                        }
                    }
                    // the shift nearest the corner entry goes last (its bulge leaves last)
                    for (int a = 1; a < ns; ++a) {
                        const CT v = s_sig[a];
                        const R kv = cabs1(v - d);
                        int b = a - 1;
                        while (b >= 0 && cabs1(s_sig[b] - d) < kv) { s_sig[b + 1] = s_sig[b]; --b; }
                        s_sig[b + 1] = v;
                    }
                }
            }
            __syncthreads();
            // bulge b is carried by warps b kMsWarps .. (b + 1) kMsWarps - 1; g indexes
            // its threads.  The bulge column k-1 (its new subdiagonal entry and the
            // cleared bulge) is written in the second phase, after every thread of
            // the bulge has read x and y in the first.
            const int bb = warp / kMsWarps;
            const int g = (warp - bb * kMsWarps) * 32 + lane, gs = kMsWarps * 32;
            const int T = (hi - l) + 3 * (ns - 1);
            for (int t = 0; t < T; ++t) {
                const int k = l + t - 3 * bb;            // this bulge's position
                const bool act = k >= l && k <= hi - 1;
                R c = 1;
                CT sn = czero<CT>(), rho = czero<CT>();
                if (act) {
                    CT x, y;
                    if (k == l) { x = HH(l, l) - s_sig[bb]; y = HH(l + 1, l); }
                    else        { x = HH(k, k - 1); y = HH(k + 1, k - 1); }
                    givens<R>(x, y, c, sn);
                    rho = cscale(c, x) + sn * y;
                    // row rotation: rows k, k+1 of columns k .. hi, three columns per
                    // thread and pass so that their loads are in flight together
                    for (int j = k + g; j <= hi; j += 3 * gs) {
                        const bool p1 = j + gs <= hi, p2 = j + 2 * gs <= hi;
                        // (indices of absent columns clamped: every address stays in range)
                        const int o0 = PK(k, j), o1 = PK(k, p1 ? j + gs : j), o2 = PK(k, p2 ? j + 2 * gs : j);
                        const CT a0 = H[o0], b0 = H[o0 + 1];
                        const CT a1 = p1 ? H[o1] : czero<CT>(), b1 = p1 ? H[o1 + 1] : czero<CT>();
                        const CT a2 = p2 ? H[o2] : czero<CT>(), b2 = p2 ? H[o2 + 1] : czero<CT>();
                        H[o0] = cscale(c, a0) + sn * b0;
                        H[o0 + 1] = cscale(c, b0) - cconj(sn) * a0;
                        if (p1) { H[o1] = cscale(c, a1) + sn * b1; H[o1 + 1] = cscale(c, b1) - cconj(sn) * a1; }
                        if (p2) { H[o2] = cscale(c, a2) + sn * b2; H[o2 + 1] = cscale(c, b2) - cconj(sn) * a2; }
                    }
                }
                __syncthreads();
                if (act) {
                    if (k > l && g == 0) { HH(k, k - 1) = rho; HH(k + 1, k - 1) = czero<CT>(); }
                    // column rotation: columns k, k+1 of rows l .. min(k+2, hi)
                    const int i1 = min(k + 2, hi);
                    const int ck = PK(0, k), ck1 = PK(0, k + 1);
                    for (int i = l + g; i <= i1; i += 3 * gs) {
                        const bool p1 = i + gs <= i1, p2 = i + 2 * gs <= i1;
                        const int r1 = p1 ? i + gs : i, r2 = p2 ? i + 2 * gs : i;   // clamped rows
                        const CT a0 = H[ck + i], b0 = H[ck1 + i];
                        const CT a1 = p1 ? H[ck + r1] : czero<CT>(), b1 = p1 ? H[ck1 + r1] : czero<CT>();
                        const CT a2 = p2 ? H[ck + r2] : czero<CT>(), b2 = p2 ? H[ck1 + r2] : czero<CT>();
                        H[ck + i] = cscale(c, a0) + cconj(sn) * b0;
                        H[ck1 + i] = cscale(c, b0) - sn * a0;
                        if (p1) { H[ck + r1] = cscale(c, a1) + cconj(sn) * b1; H[ck1 + r1] = cscale(c, b1) - sn * a1; }
                        if (p2) { H[ck + r2] = cscale(c, a2) + cconj(sn) * b2; H[ck1 + r2] = cscale(c, b2) - sn * a2; }
                    }
                }
                __syncthreads();
            }
            continue;
        }
        // ---- single-shift sweep
        CT mu;
        {
            CT d = HH(hi, hi);
            if (its % 11 == 10) {
                mu = d;
                mu.x += (R)0.75 * cabs(HH(hi, hi - 1));
            } else {
                CT e1, e2;
                eig2x2<R>(HH(hi - 1, hi - 1), HH(hi - 1, hi), HH(hi, hi - 1), d, &e1, &e2);
                mu = (cabs1(e1 - d) <= cabs1(e2 - d)) ? e1 : e2;
            }
        }
        __syncthreads();
        for (int k = l; k < hi; k += kQrChunk) {
            const int kb = min(kQrChunk, hi - k);
            const int w1 = min(k + kb + 1, hi);
            if (warp == 0) {
                if (kb == kQrChunk) qr_window<R, kQrChunk>(H, l, hi, k, kb, w1, mu, s_c, s_s);
                else                qr_window<R, 0>(H, l, hi, k, kb, w1, mu, s_c, s_s);
            }
            __syncthreads();
            // deferred: the window's row rotations on the columns right of it
            // (rows k..k+kb), its column rotations on the rows above the
            // frontier (row i takes rotations max(i, k)..k+kb-1)
            const int nfc = hi - w1, nfr = k + kb - l;
            for (int t = tid; t < nfc + nfr; t += nt) {
                if (t < nfc) {
                    CT* col = H + PK(k, w1 + 1 + t);
                    CT a = col[0];
                    for (int r = 0; r < kb; ++r) {
                        const R c = s_c[r];
                        const CT s = s_s[r];
                        const CT b = col[r + 1];
                        col[r] = cscale(c, a) + s * b;
                        a = cscale(c, b) - cconj(s) * a;
                    }
                    col[kb] = a;
                } else {
                    const int i = l + (t - nfc);
                    const int r0 = max(i, k) - k;
                    int cj = k + r0;                  // column of the carry
                    int off = PK(i, cj);
                    CT a = H[off];
                    for (int r = r0; r < kb; ++r) {
                        const R c = s_c[r];
                        const CT s = s_s[r];
                        const int off1 = off + cj + 3;   // PK(i, cj + 1)
                        const CT b = H[off1];
                        H[off] = cscale(c, a) + cconj(s) * b;
                        a = cscale(c, b) - s * a;
                        off = off1;
                        ++cj;
                    }
                    H[off] = a;
                }
            }
            __syncthreads();
        }
    }
    __syncthreads();
    if (failed) {
        for (int i = tid; i <= hi; i += nt) ev[i] = HH(i, i);
        if (tid == 0) atomicOr(&status->flags, 1);
    }
    if (tid == 0) status->qr_sweeps = total;
    __syncthreads();
    #undef HH
    // Step 2: rank by (rho, Re, Im, index); keep the first m0.  Each value's
    // keys are formed once (rho in FP64 as the ranking defines it) into the
    // matrix storage, dead now, as integers that order like the doubles; gap[]
    // is the distance to the nearest other value (found in R, taken in FP64).
    unsigned long long* key = reinterpret_cast<unsigned long long*>(H);   // 3 per value
    for (int i = tid; i < N; i += nt) {
        const CT e = ev[i];
        const double ex = e.x, ey = e.y;
        const bool fin = isfinite(ex) && isfinite(ey);
        const double rx = (ex - c_re) / ra, ry = (ey - c_im) / rb;
        key[3 * i] = order_key(fin ? sqrt(rx * rx + ry * ry) : INFINITY);
        key[3 * i + 1] = order_key(fin ? ex : INFINITY);
        key[3 * i + 2] = order_key(fin ? ey : INFINITY);
    }
    if (tid == 0) gap[m0] = INFINITY;   // normalised radius of the first value left out
    __syncthreads();
    for (int i = tid; i < N; i += nt) {
        const unsigned long long k0 = key[3 * i], k1 = key[3 * i + 1], k2 = key[3 * i + 2];
        const CT e = ev[i];
        const bool fin = isfinite(e.x) && isfinite(e.y);
        int rank = 0, jn = -1;
        R dn = (R)INFINITY;
        for (int j = 0; j < N; ++j) {
            if (j == i) continue;
            const unsigned long long j0 = key[3 * j], j1 = key[3 * j + 1], j2 = key[3 * j + 2];
            const bool less = j0 < k0 || (j0 == k0 && (j1 < k1 || (j1 == k1 && (j2 < k2 || (j2 == k2 && j < i)))));
            rank += less ? 1 : 0;
            const CT f = ev[j];
            if (fin && isfinite(f.x) && isfinite(f.y)) {
                const R dx = f.x - e.x, dy = f.y - e.y;
                const R d2 = dx * dx + dy * dy;
                if (jn < 0 || d2 < dn) { dn = d2; jn = j; }
            }
        }
        if (rank < m0) {
            lam0[rank] = make_double2((double)e.x, (double)e.y);
            gap[rank] = jn < 0 ? INFINITY
                               : hypot((double)ev[jn].x - (double)e.x, (double)ev[jn].y - (double)e.y);
        } else if (rank == m0 && fin) {
            const double rx = ((double)e.x - c_re) / ra, ry = ((double)e.y - c_im) / rb;
            gap[m0] = sqrt(rx * rx + ry * ry);
        }
    }
}

// ---------------------------------------------------------------------------
// Newton refinement of one kept Ritz pair per CTA: FP64 residuals T(l) x and
// T'(l) x, corrections through an FP32 LU of T(lf) (mixed-precision chord
// iteration: its fixed point is T(l) x = 0 to FP64 accuracy, the FP32 factor
// only sets the contraction rate).
// smem: T (m x m FP32 complex, col-major, LU in place), x, u, xf, a (m FP64
// complex each), fa, fu (m FP32 complex each), piv (m)
// ---------------------------------------------------------------------------
constexpr int kNewtonThreads = 256;
static_assert(2 * kMaxM0 <= kNewtonThreads, "each row of the FP64 residual takes two threads");
constexpr int kNewtonMax = 8;

// f_t(l) (scale included) or its derivative, for the general reduced problem
__device__ __forceinline__ double2 rp_term(const TermDev& t, double2 l, bool deriv) {
    double2 v;
    if (t.kind == 0) {
        const int p = deriv ? t.p - 1 : t.p;
        if (p < 0) return make_double2(0.0, 0.0);
        v = make_double2(1.0, 0.0);
        for (int q = 0; q < p; ++q) v = v * l;
        if (deriv) v = (double)t.p * v;
    } else {
        const double er = exp(-t.tau * l.x);
        double sn, cs;
        sincos(-t.tau * l.y, &sn, &cs);
        v = make_double2(er * cs, er * sn);
        if (deriv) v = (-t.tau) * v;
    }
    return t.scale * v;
}

// Leading dimension of the m x m factorisations held in shared memory: m + 1,
// so that the rows of a column-major array (m a multiple of 16 for the usual
// subspace sizes) do not all fall into one shared-memory bank.
__host__ __device__ __forceinline__ int nld(int m) { return m + 1; }

// T = That(lam) in the factorisation's precision, column-major, leading
// dimension nld(m); a warp per column, lanes over rows.
template <typename LT>
__device__ void newton_build(int m, const RedProblem& P, double2 lam, LT* T) {
    const int64_t mm = (int64_t)m * m;
    const int ld = nld(m), lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (P.kmax >= 0) {
        const LT lf = cmake<LT>(lam.x, lam.y);
        for (int c = warp; c < m; c += nw)
            for (int r = lane; r < m; r += 32) {
                const int64_t e = r + (int64_t)c * m;
                double2 a = P.Ahat[(int64_t)P.kmax * mm + e];      // Horner in lambda
                LT v = cmake<LT>(a.x, a.y);
                for (int p = P.kmax - 1; p >= 0; --p) {
                    a = P.Ahat[(int64_t)p * mm + e];
                    v = cfma(v, lf, cmake<LT>(a.x, a.y));
                }
                T[r + c * ld] = v;
            }
    } else {
        for (int c = warp; c < m; c += nw)
            for (int r = lane; r < m; r += 32) {
                const int64_t e = r + (int64_t)c * m;
                double2 v = make_double2(0.0, 0.0);
                for (int t = 0; t < P.nterms; ++t)
                    v = cfma(rp_term(P.terms[t], lam, false), P.G[(int64_t)t * mm + e], v);
                T[r + c * ld] = cmake<LT>(v.x, v.y);
            }
    }
}

// Rows r of T(l) x and T'(l) x over the columns [c0, c1), in FP64 (the sum over
// two column ranges is the whole product: both are linear in the row sums).
__device__ void newton_apply(int m, const RedProblem& P, double2 l, const double2* x, int r, int c0,
                             int c1, double2* v_out, double2* dv_out) {
    const int64_t mm = (int64_t)m * m;
    double2 v = make_double2(0.0, 0.0), dv = make_double2(0.0, 0.0);
    if (P.kmax >= 0) {
        for (int p = P.kmax; p >= 0; --p) {                 // Horner for T(l)x and T'(l)x
            double2 row = make_double2(0.0, 0.0);
            const double2* Ap = P.Ahat + (int64_t)p * mm;
            for (int c = c0; c < c1; ++c) row = cfma(Ap[r + (int64_t)c * m], x[c], row);
            dv = cfma(dv, l, v);
            v = cfma(v, l, row);
        }
    } else {
        for (int t = 0; t < P.nterms; ++t) {
            double2 row = make_double2(0.0, 0.0);
            const double2* Gt = P.G + (int64_t)t * mm;
            for (int c = c0; c < c1; ++c) row = cfma(Gt[r + (int64_t)c * m], x[c], row);
            v = cfma(rp_term(P.terms[t], l, false), row, v);
            dv = cfma(rp_term(P.terms[t], l, true), row, dv);
        }
    }
    *v_out = v;
    *dv_out = dv;
}

// LU with partial pivoting (cabs1, lowest row on ties) in place, leading
// dimension nld(m).  Per column: warp 0 finds the pivot, swaps it into the
// column and scales the multipliers (keeping the reciprocal pivot in rd[c]);
// one thread per column swaps the two rows in the others; then each warp
// updates whole columns right of c (lanes over rows).
template <typename LT>
__device__ void newton_lu(int m, LT* T, int* piv, LT* rd, int* s_p) {
    typedef typename cplx_real<LT>::type LR;
    const int ld = nld(m);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int c = 0; c < m; ++c) {
        if (warp == 0) {
            LR best = -1;
            int bi = c;
            for (int r = c + lane; r < m; r += 32) {
                LR v = cabs1(T[r + c * ld]);
                if (v > best) { best = v; bi = r; }
            }
            for (int o = 16; o > 0; o >>= 1) {
                LR ov = __shfl_down_sync(0xffffffffu, best, o);
                int oi = __shfl_down_sync(0xffffffffu, bi, o);
                if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
            }
            bi = __shfl_sync(0xffffffffu, bi, 0);
            if (lane == 0) {
                *s_p = bi;
                piv[c] = bi;
                if (bi != c) { const LT t = T[c + c * ld]; T[c + c * ld] = T[bi + c * ld]; T[bi + c * ld] = t; }
            }
            __syncwarp();
            LT d = T[c + c * ld];
            if (d.x == (LR)0 && d.y == (LR)0) d = cmake<LT>(1e-30, 0.0);
            const LT inv = crcp(d);
            for (int r = c + 1 + lane; r < m; r += 32) T[r + c * ld] = T[r + c * ld] * inv;
            if (lane == 0) { T[c + c * ld] = d; rd[c] = inv; }
        }
        __syncthreads();
        const int p = *s_p;
        if (p != c) {
            for (int cc = threadIdx.x; cc < m; cc += blockDim.x)
                if (cc != c) { const LT t = T[c + cc * ld]; T[c + cc * ld] = T[p + cc * ld]; T[p + cc * ld] = t; }
            __syncthreads();
        }
        for (int cc = c + 1 + warp; cc < m; cc += nw) {
            const LT u = T[c + cc * ld];
            for (int r = c + 1 + lane; r < m; r += 32) T[r + cc * ld] = cfms(T[r + c * ld], u, T[r + cc * ld]);
        }
        __syncthreads();
    }
}

// One warp solves L U y = P b in place (factors of newton_lu, reciprocal pivots
// rd): the row interchanges in shared memory, then both substitutions with b in
// registers (lane j holds rows j, j + 32, ..; m <= 128), each step's pivot
// value broadcast by a shuffle.
template <typename LT>
__device__ __forceinline__ LT pick4(const LT* br, int q) {
    return q == 0 ? br[0] : (q == 1 ? br[1] : (q == 2 ? br[2] : br[3]));
}
template <typename LT>
__device__ void warp_lu_solve(int m, const LT* T, const int* piv, const LT* rd, LT* b) {
    const int lane = threadIdx.x & 31, ld = nld(m);
    if (lane == 0)
        for (int c = 0; c < m; ++c) {
            const int p = piv[c];
            if (p != c) { const LT t = b[c]; b[c] = b[p]; b[p] = t; }
        }
    __syncwarp();
    LT br[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int r = lane + 32 * q;
        br[q] = r < m ? b[r] : cmake<LT>(0.0, 0.0);
    }
    for (int i = 0; i + 1 < m; ++i) {                    // unit lower triangle
        const LT own = pick4(br, i >> 5);
        LT bi;
        bi.x = __shfl_sync(0xffffffffu, own.x, i & 31);
        bi.y = __shfl_sync(0xffffffffu, own.y, i & 31);
        const LT* Ti = T + (size_t)i * ld;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int r = lane + 32 * q;
            if (r > i && r < m) br[q] = cfms(Ti[r], bi, br[q]);
        }
    }
    for (int i = m - 1; i >= 0; --i) {                   // upper triangle
        const int qi = i >> 5;
        const LT own = pick4(br, qi);
        LT bi;
        bi.x = __shfl_sync(0xffffffffu, own.x, i & 31);
        bi.y = __shfl_sync(0xffffffffu, own.y, i & 31);
        bi = bi * rd[i];
        const LT* Ti = T + (size_t)i * ld;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int r = lane + 32 * q;
            if (r == i) br[q] = bi;
            else if (r < i) br[q] = cfms(Ti[r], bi, br[q]);
        }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int r = lane + 32 * q;
        if (r < m) b[r] = br[q];
    }
    __syncwarp();
}

// Solves T y = b in place with the LU held in T; warp 0 takes b0 and warp 1
// takes b1 (when given), so the two right-hand sides of a Newton step proceed
// side by side.
template <typename LT>
__device__ void newton_solve(int m, const LT* T, const int* piv, const LT* rd, LT* b0, LT* b1) {
    const int w = threadIdx.x >> 5;
    LT* b = (w == 0) ? b0 : b1;
    if (w < 2 && b != nullptr) warp_lu_solve(m, T, piv, rd, b);
    __syncthreads();
}

__device__ double block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        red[32] = t;
    }
    __syncthreads();
    double r = red[32];
    __syncthreads();
    return r;
}

// four block sums in one pass; red holds at least 4 * 33 doubles
struct Sum4 { double x, y, z, w; };
__device__ Sum4 block_sum4(Sum4 v, double* red) {
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_down_sync(0xffffffffu, v.x, o);
        v.y += __shfl_down_sync(0xffffffffu, v.y, o);
        v.z += __shfl_down_sync(0xffffffffu, v.z, o);
        v.w += __shfl_down_sync(0xffffffffu, v.w, o);
    }
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if ((threadIdx.x & 31) == 0) { red[w] = v.x; red[33 + w] = v.y; red[66 + w] = v.z; red[99 + w] = v.w; }
    __syncthreads();
    Sum4 t = {0.0, 0.0, 0.0, 0.0};
    for (int q = 0; q < nw; ++q) { t.x += red[q]; t.y += red[33 + q]; t.z += red[66 + q]; t.w += red[99 + q]; }
    __syncthreads();
    return t;
}

__device__ __forceinline__ double2 to_d2f(float2 v) { return make_double2(v.x, v.y); }
__device__ __forceinline__ double2 to_d2f(double2 v) { return v; }

// Dynamic shared memory of newton_kernel<LT> for subspace size m.
template <typename LT>
size_t newton_smem(int m) {
    return sizeof(double2) * 6 * (size_t)m + sizeof(LT) * ((size_t)m * nld(m) + 3 * (size_t)m) +
           sizeof(int) * (size_t)m;
}

// LT: arithmetic of the factorisation (float2 in stage 1, double2 in the FP64
// fallback stage, where clustered reduced eigenvalues need the FP64 factor).
template <typename LT>
__global__ void __launch_bounds__(kNewtonThreads) newton_kernel(
    int m, RedProblem P, const double2* __restrict__ lam0,
    const double* __restrict__ gap, double2* __restrict__ lam, double2* __restrict__ Y,
    int* redflag, int stage, IterStatus* status, const int* __restrict__ nkeep,
    double2 filler, int* __restrict__ need) {
    if (stage == 2 && !(*redflag & kNeed64)) return;
    if (stage == 3 && (!(*redflag & kRetry64) || !need[blockIdx.x])) return;
    if (stage == 1 && need != nullptr && threadIdx.x == 0) need[blockIdx.x] = 0;
    if (nkeep != nullptr && (int)blockIdx.x >= *nkeep) {
        // a slot the reduced solver left empty: lambda outside C, unit vector
        if (threadIdx.x == 0) lam[blockIdx.x] = filler;
        for (int r = threadIdx.x; r < m; r += blockDim.x)
            Y[r + (int64_t)blockIdx.x * m] = make_double2(r == (int)(blockIdx.x % m) ? 1.0 : 0.0, 0.0);
        return;
    }
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2* x = reinterpret_cast<double2*>(smem_raw);
    double2* u = x + m;
    double2* xf = u + m;
    double2* a = xf + m;
    double2* pv = a + m;                       // the second column half's partial rows
    double2* pdv = pv + m;
    LT* T = reinterpret_cast<LT*>(pdv + m);    // m x m, leading dimension nld(m)
    LT* fa = T + (int64_t)m * nld(m);
    LT* fu = fa + m;
    LT* rd = fu + m;                           // reciprocal pivots
    int* piv = reinterpret_cast<int*>(rd + m);
    __shared__ double red[4 * 33];
    __shared__ int s_p;
    const int i = blockIdx.x;
    const double2 l0 = lam0[i];
    double2 l = l0;
    newton_build(m, P, l, T);
    __syncthreads();
    newton_lu(m, T, piv, rd, &s_p);
    for (int r = threadIdx.x; r < m; r += blockDim.x) fa[r] = cmake<LT>(1.0, 0.0);
    __syncthreads();
    newton_solve<LT>(m, T, piv, rd, fa, nullptr);
    {
        double s = 0.0;
        for (int r = threadIdx.x; r < m; r += blockDim.x) s += cnorm2(to_d2f(fa[r]));
        s = sqrt(block_sum(s, red));
        double inv = (s > 0.0 && isfinite(s)) ? 1.0 / s : 0.0;
        for (int r = threadIdx.x; r < m; r += blockDim.x) { x[r] = inv * to_d2f(fa[r]); xf[r] = x[r]; }
        __syncthreads();
    }
    // Newton on [T(l) y = 0, x^H y = 1] with the Jacobian's T block frozen at the
    // factorised point (chord iteration).  Each step:
    //   a = T(lf)^{-1} T(l) x,  u = T(lf)^{-1} T'(l) x,
    //   dl = -(x^H a)/(x^H u),  x <- x - a - dl u,  l <- l + dl.
    // With lf = l this is exactly Newton; the factorisation is refreshed while
    // the steps are still large.
    bool ok = true, conv = false;
    int refreshes = 0;
    double prev = INFINITY;
    for (int it = 0; it < kNewtonMax; ++it) {
        {   // FP64 rows of T(l) x and T'(l) x, each row's columns split over two threads
            const int half = (m + 1) / 2;
            double2 v = make_double2(0.0, 0.0), dv = v;
            const int t = threadIdx.x;
            if (t < 2 * m) {
                const int r = t < m ? t : t - m;
                newton_apply(m, P, l, x, r, t < m ? 0 : half, t < m ? half : m, &v, &dv);
                if (t >= m) { pv[r] = v; pdv[r] = dv; }
            }
            __syncthreads();
            if (t < m) {
                v = v + pv[t];
                dv = dv + pdv[t];
                fa[t] = cmake<LT>(v.x, v.y);
                fu[t] = cmake<LT>(dv.x, dv.y);
            }
            __syncthreads();
        }
        newton_solve(m, T, piv, rd, fa, fu);
        double are = 0.0, aim = 0.0, ure = 0.0, uim = 0.0;
        for (int r = threadIdx.x; r < m; r += blockDim.x) {
            a[r] = to_d2f(fa[r]);
            u[r] = to_d2f(fu[r]);
            double2 ta = cconj(x[r]) * a[r], tu = cconj(x[r]) * u[r];
            are += ta.x; aim += ta.y; ure += tu.x; uim += tu.y;
        }
        const Sum4 sums = block_sum4(Sum4{are, aim, ure, uim}, red);
        are = sums.x; aim = sums.y; ure = sums.z; uim = sums.w;
        double2 xu = make_double2(ure, uim);
        if (!(cabs(xu) > 0.0) || !isfinite(xu.x) || !isfinite(xu.y)) { ok = false; break; }
        double2 dl = -(make_double2(are, aim) * crcp(xu));
        if (!isfinite(dl.x) || !isfinite(dl.y)) { ok = false; break; }
        double s = 0.0;
        for (int r = threadIdx.x; r < m; r += blockDim.x) {
            double2 nx = x[r] - a[r] - dl * u[r];
            u[r] = nx;
            s += cnorm2(nx);
        }
        s = sqrt(block_sum(s, red));
        double inv = (s > 0.0 && isfinite(s)) ? 1.0 / s : 0.0;
        for (int r = threadIdx.x; r < m; r += blockDim.x) x[r] = inv * u[r];
        __syncthreads();
        l = l + dl;
        const double rel = cabs(dl) / fmax(cabs(l), 1e-300);
        // converged, or stalled at the FP64 rounding level of the residual
        if (rel <= 64.0 * DBL_EPSILON || (rel < 1e-12 && rel > 0.25 * prev)) { conv = true; break; }
        prev = rel;
        if (rel > 1e-9 && refreshes < 2 && (it == 1 || it == 4)) {
            newton_build(m, P, l, T);
            __syncthreads();
            newton_lu(m, T, piv, rd, &s_p);
            ++refreshes;
        }
    }
    // Accept a move of at most 0.3 of the distance to the nearest other start,
    // or any converged move that lands clearly inside the kept region: below the
    // normalised radius of the first value Step 2 left out (gap[m0]) by twice
    // the move in normalised units.  Two pairs landing on one eigenvalue are
    // caught by the duplicate check.
    const double moved = cabs(l - l0);
    const double lim = 0.3 * gap[i];
    const double rmin = fmin(P.ra, P.rb);
    const double rx = (l.x - P.c_re) / P.ra, ry = (l.y - P.c_im) / P.rb;
    const bool kept = conv && sqrt(rx * rx + ry * ry) + 2.0 * moved / rmin < gap[gridDim.x];
    const double sx = (l0.x - P.c_re) / P.ra, sy = (l0.y - P.c_im) / P.rb;
    const bool outside = sqrt(sx * sx + sy * sy) > 1.0 + 4.0 * moved / rmin;
    if (!conv && stage != 2) ok = false;     // a later stage takes over
    if (!ok || !isfinite(l.x) || !isfinite(l.y) || !(moved <= lim || kept)) {
        l = l0;
        for (int r = threadIdx.x; r < m; r += blockDim.x) x[r] = xf[r];
        if (threadIdx.x == 0) {
            // A pair clearly outside C whose polish stalls -- typically a
            // near-multiple Ritz value, where Newton converges only linearly --
            // keeps its FP32 value and inverse-iteration vector: Step 3 never
            // tests it, and were it inside C its true residual would show.
            if (stage != 2 && outside) {
            } else if (stage != 2 && !(status->n_inside > 0 && status->max_relres <= kExactStageRelres)) {
                // Far from convergence (the previous iteration's residuals inside
                // C above kExactStageRelres, or no previous test) the pair keeps
                // its FP32 value and inverse-iteration vector: the Ritz pairs of
                // such an iterate are approximations at the filter's level of
                // progress anyway, and neither an FP64-factor retry nor the FP64
                // re-run of the whole stage (about as much as eight iterations of
                // the n = 4096 QEP) would change that.
            } else if (stage == 1 && need != nullptr) {
                // retry this pair alone with an FP64 factor from the same start
                need[i] = 1;
                atomicOr(redflag, kRetry64);
            } else {
                atomicOr(&status->flags, 8);
                atomicOr(redflag, kNeed64);
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) lam[i] = l;
    for (int r = threadIdx.x; r < m; r += blockDim.x) Y[r + (int64_t)i * m] = x[r];
}

// Two kept Ritz values that coincide after Newton mean stage 1 lost one.
// Every pair (i, j) is one thread's test, on squared distances.
constexpr int kDupThreads = 1024;
__global__ void __launch_bounds__(kDupThreads) duplicate_check_kernel(int m0, const double2* __restrict__ lam,
                                                                      int* redflag) {
    __shared__ double2 s_l[kMaxM0];
    __shared__ int s_dup;
    if (threadIdx.x == 0) s_dup = 0;
    for (int i = threadIdx.x; i < m0; i += blockDim.x) s_l[i] = lam[i];
    __syncthreads();
    const int np = m0 * m0;
    bool dup = false;
    for (int e = threadIdx.x; e < np; e += blockDim.x) {
        const int i = e / m0, j = e - i * m0;
        if (j <= i) continue;
        const double2 a = s_l[i], b = s_l[j];
        const double dx = a.x - b.x, dy = a.y - b.y;
        dup = dup || (dx * dx + dy * dy <= 1e-18 * fmax(a.x * a.x + a.y * a.y, 1e-300));
    }
    if (dup) s_dup = 1;
    __syncthreads();
    if (threadIdx.x == 0 && s_dup) atomicOr(redflag, kNeed64);
}

// ---------------------------------------------------------------------------
// Cholesky G + shift*trace(G)*I = R^H R and R^{-1}, one CTA, FP32 arithmetic:
// the orthonormalisation only needs a well-conditioned basis of the same span,
// and Q R^{-1} is applied in FP64 by the caller.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(512) chol_inverse_kernel(int m, const double2* __restrict__ G,
                                                           double shift_rel,
                                                           double2* __restrict__ Rinv,
                                                           IterStatus* status) {
    extern __shared__ unsigned char smem_raw[];
    // leading dimension m + 1: the rows of a column-major m x m array with m a
    // multiple of 16 would otherwise sit in one shared-memory bank
    const int ld = m + 1;
    float2* R = reinterpret_cast<float2*>(smem_raw);   // m x m col-major (upper used)
    float2* X = R + ld * m;                             // m x m col-major: R^{-1}
    __shared__ float s_tr;
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    {   // trace (real parts of the diagonal), one warp
        if (warp == 0) {
            double tr = 0.0;
            for (int i = lane; i < m; i += 32) tr += G[i + (int64_t)i * m].x;
            for (int o = 16; o > 0; o >>= 1) tr += __shfl_xor_sync(0xffffffffu, tr, o);
            if (lane == 0) s_tr = (float)(shift_rel * tr);
        }
        __syncthreads();
    }
    for (int c = warp; c < m; c += nw)
        for (int r = lane; r < m; r += 32) {
            const double2 g = G[r + (int64_t)c * m];
            float2 v = make_float2((float)g.x, (float)g.y);
            if (r == c) v = make_float2(v.x + s_tr, 0.0f);
            R[r + c * ld] = v;
            X[r + c * ld] = make_float2(r == c ? 1.0f : 0.0f, 0.0f);
        }
    __syncthreads();
    // right-looking Cholesky: row j of R, then the trailing upper triangle; the
    // trailing update gives each warp whole columns and each lane rows
    for (int j = 0; j < m; ++j) {
        float d = R[j + j * ld].x;
        const bool bad = !(d > 0.0f);
        if (bad) d = 1e-30f;
        const float rjj = sqrtf(d), inv = 1.0f / rjj;
        __syncthreads();                               // every thread has read the pivot
        if (tid == 0) {
            if (bad) atomicOr(&status->flags, 4);
            R[j + j * ld] = make_float2(rjj, 0.0f);
        }
        for (int c = j + 1 + tid; c < m; c += nt) R[j + c * ld] = inv * R[j + c * ld];
        __syncthreads();
        for (int c = j + 1 + warp; c < m; c += nw) {
            const float2 uc = R[j + c * ld];
            for (int r = j + 1 + lane; r <= c; r += 32)
                R[r + c * ld] = cfms(cconj(R[j + r * ld]), uc, R[r + c * ld]);
        }
        __syncthreads();
    }
    // column c of R^{-1} by back substitution, one warp per column, with the
    // reciprocal pivots formed once
    __shared__ float2 s_rdiag[kMaxM0];
    for (int i = tid; i < m; i += nt) s_rdiag[i] = crcp(R[i + i * ld]);
    __syncthreads();
    for (int c = warp; c < m; c += nw) {
        float2* x = X + c * ld;
        for (int i = c; i >= 0; --i) {
            if (lane == 0) x[i] = x[i] * s_rdiag[i];
            __syncwarp();
            const float2 xi = x[i];
            for (int r = lane; r < i; r += 32) x[r] = cfms(R[r + i * ld], xi, x[r]);
            __syncwarp();
        }
    }
    __syncthreads();
    for (int c = warp; c < m; c += nw)
        for (int r = lane; r < m; r += 32) {
            const float2 v = X[r + c * ld];
            Rinv[r + (int64_t)c * m] = make_double2(v.x, v.y);
        }
}

size_t packed_elems(int N) { return (size_t)N * (N + 5) / 2 + 4; }
constexpr int kMaxSmemPacked = 200 * 1024;

cudaError_t qr_select_attributes() {
    const int cap = kMaxSmemPacked + 16 * 1024;
    cudaError_t e0;
    if ((e0 = cudaFuncSetAttribute(companion_cols_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)companion_cols_smem(kMaxM0))) != cudaSuccess) return e0;
    if ((e0 = cudaFuncSetAttribute(hess_cluster_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)kHcSmemCap)) != cudaSuccess) return e0;
    if ((e0 = cudaFuncSetAttribute(hess_cluster_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)kHcSmemCap)) != cudaSuccess) return e0;
    static_assert(kRedSmemCap <= (size_t)kMaxSmemPacked + 16 * 1024, "one cap for the single-CTA kernels");
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(hessenberg_kernel<float>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, cap)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(hessenberg_kernel<double>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, cap)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(qr_select_kernel<float, true, true>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, cap)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(qr_select_kernel<float, false, true>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, cap)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(qr_select_kernel<double, true>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, cap)) != cudaSuccess) return e;
    return cudaFuncSetAttribute(qr_select_kernel<double, false>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
}

// Workspace layout, every region 256-byte aligned.
struct RedLayout {
    size_t c32, lk32, c64, lk64, piv, h32, h64, lam0, gap, flag, need, total;
};
RedLayout red_layout(int m, int kmax) {
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t N = (size_t)kmax * m;
    RedLayout L;
    size_t o = 0;
    L.c32 = o;  o = al(o + N * N * sizeof(float2));
    L.lk32 = o; o = al(o + (size_t)m * m * sizeof(float2));
    L.c64 = o;  o = al(o + N * N * sizeof(double2));
    L.lk64 = o; o = al(o + (size_t)m * m * sizeof(double2));
    L.piv = o;  o = al(o + (size_t)m * sizeof(int));
    L.h32 = o;  o = al(o + packed_elems((int)N) * sizeof(float2));
    L.h64 = o;  o = al(o + packed_elems((int)N) * sizeof(double2));
    L.lam0 = o; o = al(o + (size_t)m * sizeof(double2));
    L.gap = o;  o = al(o + (size_t)(m + 1) * sizeof(double));
    L.flag = o; o = al(o + 16);
    L.need = o; o = al(o + (size_t)m * sizeof(int));
    L.total = o;
    return L;
}

template <typename R>
cudaError_t run_stage(cudaStream_t st, int stage, int m, int kmax, const double2* Ahat, int m0,
                      double c_re, double c_im, double ra, double rb, unsigned char* base,
                      const RedLayout& L, IterStatus* status) {
    typedef typename cx<R>::type CT;
    const int N = kmax * m;
    CT* C = reinterpret_cast<CT*>(base + (sizeof(R) == 4 ? L.c32 : L.c64));
    CT* Lk = reinterpret_cast<CT*>(base + (sizeof(R) == 4 ? L.lk32 : L.lk64));
    CT* Hg = reinterpret_cast<CT*>(base + (sizeof(R) == 4 ? L.h32 : L.h64));
    int* piv = reinterpret_cast<int*>(base + L.piv);
    int* flag = reinterpret_cast<int*>(base + L.flag);
    double2* lam0 = reinterpret_cast<double2*>(base + L.lam0);
    double* gap = reinterpret_cast<double*>(base + L.gap);
    cudaError_t e;
    const int cs = sizeof(R) == 4 ? hess_cluster_size(N) : 0;
    if (cs > 0) {
        // FP32 stage: companion by column slices on several CTAs, Hessenberg
        // reduction by a cluster holding the matrix in distributed shared memory
        note_launch();
        companion_cols_kernel<<<(N + kCompCols - 1) / kCompCols, kCompThreads, companion_cols_smem(m), st>>>(
            m, kmax, Ahat, reinterpret_cast<float2*>(C), flag);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        note_launch();
        if (cs == 4)
            hess_cluster_kernel<4><<<4, kHcThreads, hess_cluster_smem(N, 4), st>>>(N, reinterpret_cast<float2*>(C));
        else
            hess_cluster_kernel<8><<<8, kHcThreads, hess_cluster_smem(N, 8), st>>>(N, reinterpret_cast<float2*>(C));
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    } else {
        note_launch();
        companion_kernel<R><<<1, kRedThreads, 0, st>>>(m, kmax, Ahat, C, Lk, piv, flag, stage);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        note_launch();
        int c0;
        size_t hsm;
        hessenberg_launch_shape<R>(N, &c0, &hsm);
        hessenberg_kernel<R><<<1, kRedThreads, hsm, st>>>(N, C, c0, flag, stage);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    size_t hbytes = packed_elems(N) * sizeof(CT);
    const size_t fixed = sizeof(CT) * ((size_t)N + kSmallLd * kSmallMax);   // ev, dense block
    int use_smem = (hbytes + fixed) <= (size_t)kMaxSmemPacked;
    size_t smem = fixed + (use_smem ? hbytes : 0);
    note_launch();
    // FP32 stage: multishift sweeps; FP64 fallback stage: single-shift sweeps
    constexpr bool kMs = sizeof(R) == 4;
    if (use_smem)
        qr_select_kernel<R, true, kMs><<<1, kQrThreads, smem, st>>>(N, m0, C, Hg, c_re, c_im, ra, rb,
                                                                    lam0, gap, flag, stage, status);
    else
        qr_select_kernel<R, false, kMs><<<1, kQrThreads, smem, st>>>(N, m0, C, Hg, c_re, c_im, ra, rb,
                                                                     lam0, gap, flag, stage, status);
    return cudaGetLastError();
}

}  // namespace

size_t reduced_work_bytes(int m, int kmax) { return red_layout(m, kmax).total; }

cudaError_t reduced_solve(cudaStream_t st, int m, int kmax, const double2* Ahat, int m0,
                          double c_re, double c_im, double ra, double rb, void* work,
                          double2* lam, double2* Yred, IterStatus* status) {
    static std::atomic<bool> attr_done{false};   // idempotent setup; atomic for concurrent handles
    cudaError_t e;
    if (!attr_done) {
        if ((e = qr_select_attributes()) != cudaSuccess) return e;
        if ((e = cudaFuncSetAttribute(newton_kernel<float2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      220 * 1024)) != cudaSuccess) return e;
        if ((e = cudaFuncSetAttribute(newton_kernel<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      220 * 1024)) != cudaSuccess) return e;
        attr_done = true;
    }
    const RedLayout L = red_layout(m, kmax);
    unsigned char* base = static_cast<unsigned char*>(work);
    int* flag = reinterpret_cast<int*>(base + L.flag);
    double2* lam0 = reinterpret_cast<double2*>(base + L.lam0);
    double* gap = reinterpret_cast<double*>(base + L.gap);
    const size_t nsm32 = newton_smem<float2>(m);
    const size_t nsm64 = newton_smem<double2>(m);
    int* need = reinterpret_cast<int*>(base + L.need);
    // stage 1: FP32 eigenvalues, Newton with an FP32 factor and FP64 residuals
    if ((e = run_stage<float>(st, 1, m, kmax, Ahat, m0, c_re, c_im, ra, rb, base, L, status)) != cudaSuccess) return e;
    note_launch();
    const RedProblem P{kmax, Ahat, 0, nullptr, nullptr, c_re, c_im, ra, rb};
    newton_kernel<float2><<<m0, kNewtonThreads, nsm32, st>>>(m, P, lam0, gap, lam, Yred, flag, 1,
                                                             status, nullptr, make_double2(0.0, 0.0), need);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // the pairs stage 1 rejected, again from the same starts with FP64 factors
    // (device-side no-op for the others); failing that, the FP64 stage below
    note_launch();
    newton_kernel<double2><<<m0, kNewtonThreads, nsm64, st>>>(m, P, lam0, gap, lam, Yred, flag, 3,
                                                              status, nullptr, make_double2(0.0, 0.0), need);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    note_launch();
    duplicate_check_kernel<<<1, kDupThreads, 0, st>>>(m0, lam, flag);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // stage 2 (device-side no-op unless the retry failed or two values coincide):
    // FP64 eigenvalues of the companion matrix, Newton with FP64 factors
    if ((e = run_stage<double>(st, 2, m, kmax, Ahat, m0, c_re, c_im, ra, rb, base, L, status)) != cudaSuccess) return e;
    note_launch();
    newton_kernel<double2><<<m0, kNewtonThreads, nsm64, st>>>(m, P, lam0, gap, lam, Yred, flag,
                                                              2, status, nullptr, make_double2(0.0, 0.0), nullptr);
    return cudaGetLastError();
}

// ===========================================================================
// Reduced solver for general T: the first two contour moments of That^{-1}
// (Beyn's method) on the contour scaled by 1.5, 256 trapezoid nodes, an m x m
// probe; the moments' pipeline runs in FP32 (node solves, SVD, the small
// eigenproblem) with the rank cut at the FP32 noise level, and every kept
// value is then refined by the Newton kernel (FP64 residuals).  Empty slots:
// lambda = c + 1.5 ra and unit vectors.
// ===========================================================================
namespace {
constexpr int kBeynNodes = 256;
constexpr double kBeynScale = 1.5;
constexpr float kBeynRankTol = 1e-5f;   // FP32 moments: noise near 1e-7 sigma_1
constexpr int kBeynThreads = 256;
constexpr int kSvdThreads = 512;
constexpr int kSvdMaxSweeps = 40;

__device__ __forceinline__ void beyn_node(int k, double c_re, double c_im, double ra, double rb,
                                          double2* z, double2* w) {
    const double th = 2.0 * M_PI * (k + 0.5) / kBeynNodes;
    double sn, cs;
    sincos(th, &sn, &cs);
    const double a = kBeynScale * ra, b = kBeynScale * rb;
    *z = make_double2(c_re + a * cs, c_im + b * sn);
    const double2 dz = make_double2(-a * sn, b * cs);
    // w = dz * (2 pi / nodes) / (2 pi i) = dz * (-i) / nodes
    *w = make_double2(dz.y / kBeynNodes, -dz.x / kBeynNodes);
}

// CTA k: Y = That(z_k)^{-1} V (FP32 LU: the nodes lie away from the
// eigenvalues), written as w_k Y and w_k z_k Y.
__global__ void __launch_bounds__(kBeynThreads) beyn_solve_kernel(
    int m, RedProblem P, double c_re, double c_im, double ra, double rb,
    const double2* __restrict__ V, float2* __restrict__ P0, float2* __restrict__ P1) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* T = reinterpret_cast<float2*>(smem_raw);          // leading dimension nld(m)
    float2* Y = T + (int64_t)m * nld(m);
    float2* rd = Y + (int64_t)m * m;
    int* piv = reinterpret_cast<int*>(rd + m);
    __shared__ int s_p;
    const int k = blockIdx.x;
    double2 z, w;
    beyn_node(k, c_re, c_im, ra, rb, &z, &w);
    newton_build(m, P, z, T);
    const int64_t mm = (int64_t)m * m;
    for (int64_t e = threadIdx.x; e < mm; e += blockDim.x)
        Y[e] = make_float2((float)V[e].x, (float)V[e].y);
    __syncthreads();
    newton_lu(m, T, piv, rd, &s_p);
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int col = warp; col < m; col += nw) warp_lu_solve(m, T, piv, rd, Y + (int64_t)col * m);
    __syncthreads();
    const float2 wf = make_float2((float)w.x, (float)w.y);
    const double2 wz = w * z;
    const float2 wzf = make_float2((float)wz.x, (float)wz.y);
    for (int64_t e = threadIdx.x; e < mm; e += blockDim.x) {
        P0[(int64_t)k * mm + e] = wf * Y[e];
        P1[(int64_t)k * mm + e] = wzf * Y[e];
    }
}

// A0 = sum_k P0[k], A1 = sum_k P1[k] in node order (deterministic), summed in FP64
__global__ void beyn_reduce_kernel(int64_t mm, const float2* __restrict__ P0,
                                   const float2* __restrict__ P1, float2* __restrict__ A0,
                                   float2* __restrict__ A1) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= mm) return;
    double2 s0 = make_double2(0.0, 0.0), s1 = make_double2(0.0, 0.0);
    for (int k = 0; k < kBeynNodes; ++k) {
        const float2 a = P0[(int64_t)k * mm + e], b = P1[(int64_t)k * mm + e];
        s0 = s0 + make_double2(a.x, a.y);
        s1 = s1 + make_double2(b.x, b.y);
    }
    A0[e] = make_float2((float)s0.x, (float)s0.y);
    A1[e] = make_float2((float)s1.x, (float)s1.y);
}

// One CTA, FP32: one-sided Jacobi SVD A0 = U diag(sigma) W^H (round-robin pair
// ordering, one warp per pair); rank r (sigma > kBeynRankTol sigma_max); the
// small matrix B = U_K^H A1 W_K diag(1/sigma_K) of the kept columns K in the
// top-left r x r of Bfull (m x m); the rest of Bfull is a diagonal far outside
// the contour, which Step 2's ranking puts last.
__global__ void __launch_bounds__(kSvdThreads) beyn_svd_kernel(
    int m, const float2* __restrict__ A0, const float2* __restrict__ A1, double c_re,
    double c_im, double ra, float2* __restrict__ Bfull, int* __restrict__ rank,
    IterStatus* status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* M = reinterpret_cast<float2*>(smem_raw);             // m x m, becomes U diag(sigma)
    float2* W = M + (int64_t)m * m;                               // m x m
    float2* T1 = W + (int64_t)m * m;                              // m x r
    float* sig = reinterpret_cast<float*>(T1 + (int64_t)m * m);  // m
    int* keep = reinterpret_cast<int*>(sig + m);                  // m
    __shared__ float s_off, s_nmax;
    __shared__ int s_r;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const int64_t mm = (int64_t)m * m;
    for (int64_t e = tid; e < mm; e += blockDim.x) {
        M[e] = A0[e];
        W[e] = make_float2((e % m) == (e / m) ? 1.0f : 0.0f, 0.0f);
    }
    __syncthreads();
    const int me = (m + 1) & ~1;          // players (a phantom column when m is odd)
    for (int sweep = 0; sweep < kSvdMaxSweeps; ++sweep) {
        // largest squared column norm: a column far below it (under the rank
        // cut) only carries the rounding of the others' updates, so pairs with
        // such a column are left alone (they would never settle)
        if (tid == 0) { s_off = 0.0f; s_nmax = 0.0f; }
        __syncthreads();
        for (int j = warp; j < m; j += nw) {
            float sj = 0.0f;
            for (int r = lane; r < m; r += 32) sj += cnorm2(M[r + (int64_t)j * m]);
            for (int o = 16; o > 0; o >>= 1) sj += __shfl_xor_sync(0xffffffffu, sj, o);
            if (lane == 0) atomicMax(reinterpret_cast<unsigned int*>(&s_nmax), __float_as_uint(sj));
        }
        __syncthreads();
        const float negl = 1e-12f * s_nmax;
        float off = 0.0f;
        for (int round = 0; round < me - 1; ++round) {
            for (int pr = warp; pr < me / 2; pr += nw) {
                auto idx = [&](int j) { return j == 0 ? 0 : 1 + (j - 1 + round) % (me - 1); };
                int p = idx(pr), q = idx(me - 1 - pr);
                if (p > q) { int t = p; p = q; q = t; }
                if (q >= m) continue;                                  // phantom
                float2* ap = M + (int64_t)p * m;
                float2* aq = M + (int64_t)q * m;
                float al = 0.0f, be = 0.0f;
                float2 ga = make_float2(0.0f, 0.0f);
                for (int r = lane; r < m; r += 32) {
                    al += cnorm2(ap[r]);
                    be += cnorm2(aq[r]);
                    ga = cfma(cconj(ap[r]), aq[r], ga);
                }
                for (int o = 16; o > 0; o >>= 1) {
                    al += __shfl_xor_sync(0xffffffffu, al, o);
                    be += __shfl_xor_sync(0xffffffffu, be, o);
                    ga.x += __shfl_xor_sync(0xffffffffu, ga.x, o);
                    ga.y += __shfl_xor_sync(0xffffffffu, ga.y, o);
                }
                const float g = cabs(ga);
                const float nrm = sqrtf(al * be);
                if (!(g > 1e-7f * nrm) || !(nrm > 0.0f) || fminf(al, be) <= negl) continue;
                off = fmaxf(off, g / nrm);
                const float2 e = make_float2(ga.x / g, ga.y / g);       // phase of gamma
                const float zeta = (be - al) / (2.0f * g);
                const float t = (zeta >= 0.0f ? 1.0f : -1.0f) / (fabsf(zeta) + sqrtf(1.0f + zeta * zeta));
                const float c = 1.0f / sqrtf(1.0f + t * t), s = c * t;
                // [a_p, a_q] <- [a_p, a_q] diag(1, conj(e)) [[c, s], [-s, c]]
                float2* wp = W + (int64_t)p * m;
                float2* wq = W + (int64_t)q * m;
                for (int r = lane; r < m; r += 32) {
                    const float2 x = ap[r], y = cconj(e) * aq[r];
                    ap[r] = make_float2(c * x.x - s * y.x, c * x.y - s * y.y);
                    aq[r] = make_float2(s * x.x + c * y.x, s * x.y + c * y.y);
                    const float2 u = wp[r], v = cconj(e) * wq[r];
                    wp[r] = make_float2(c * u.x - s * v.x, c * u.y - s * v.y);
                    wq[r] = make_float2(s * u.x + c * v.x, s * u.y + c * v.y);
                }
            }
            __syncthreads();
        }
        if (lane == 0 && off > 0.0f) atomicMax(reinterpret_cast<unsigned int*>(&s_off), __float_as_uint(off));
        __syncthreads();
        if (s_off < 2e-7f) break;
        if (sweep == kSvdMaxSweeps - 1 && tid == 0) atomicOr(&status->flags, 1);
        __syncthreads();
    }
    // singular values, rank
    for (int j = warp; j < m; j += nw) {
        float sj = 0.0f;
        for (int r = lane; r < m; r += 32) sj += cnorm2(M[r + (int64_t)j * m]);
        for (int o = 16; o > 0; o >>= 1) sj += __shfl_xor_sync(0xffffffffu, sj, o);
        if (lane == 0) sig[j] = sqrtf(sj);
    }
    __syncthreads();
    if (tid == 0) {
        float smax = 0.0f;
        for (int j = 0; j < m; ++j) smax = fmaxf(smax, sig[j]);
        int r = 0;
        for (int j = 0; j < m; ++j)
            if (smax > 0.0f && sig[j] > kBeynRankTol * smax) keep[r++] = j;
        s_r = r;
        *rank = r;
    }
    __syncthreads();
    const int r = s_r;
    // T1 = A1 W_K (m x r), then B(i, j) = U_K_i^H T1_j / sigma_K_j with U = M / sigma
    for (int e = tid; e < m * r; e += blockDim.x) {
        const int a = e % m, j = e / m;
        const float2* wj = W + (int64_t)keep[j] * m;
        float2 t = make_float2(0.0f, 0.0f);
        for (int b = 0; b < m; ++b) t = cfma(A1[a + (int64_t)b * m], wj[b], t);
        T1[e] = t;
    }
    __syncthreads();
    for (int e = tid; e < m * m; e += blockDim.x) {
        const int i = e % m, j = e / m;
        float2 v = make_float2(0.0f, 0.0f);
        if (i < r && j < r) {
            const int ki = keep[i], kj = keep[j];
            const float2* ui = M + (int64_t)ki * m;
            const float2* tj = T1 + (int64_t)j * m;
            for (int a = 0; a < m; ++a) v = cfma(cconj(ui[a]), tj[a], v);
            v = (1.0f / (sig[ki] * sig[kj])) * v;
        } else if (i == j) {
            v = make_float2((float)(c_re + 10.0 * ra * (1.0 + i)), (float)c_im);
        }
        Bfull[e] = v;
    }
}

struct BeynLayout { size_t V, P0, P1, A0, A1, B, Hg, lam0, gap, flag, rank, total; };
BeynLayout beyn_layout(int m) {
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t mm = (size_t)m * m;
    BeynLayout L;
    size_t o = 0;
    L.V = o;    o = al(o + mm * sizeof(double2));
    L.P0 = o;   o = al(o + mm * sizeof(float2) * kBeynNodes);
    L.P1 = o;   o = al(o + mm * sizeof(float2) * kBeynNodes);
    L.A0 = o;   o = al(o + mm * sizeof(float2));
    L.A1 = o;   o = al(o + mm * sizeof(float2));
    L.B = o;    o = al(o + mm * sizeof(float2));
    L.Hg = o;   o = al(o + packed_elems(m) * sizeof(float2));
    L.lam0 = o; o = al(o + (size_t)m * sizeof(double2));
    L.gap = o;  o = al(o + (size_t)(m + 1) * sizeof(double));
    L.flag = o; o = al(o + 16);
    L.rank = o; o = al(o + 16);
    L.total = o;
    return L;
}
}  // namespace

size_t beyn_work_bytes(int m) { return beyn_layout(m).total; }
int beyn_max_m() { return 64; }

cudaError_t reduced_solve_general(cudaStream_t st, int m, int nterms, const TermDev* terms,
                                  const double2* G, double c_re, double c_im, double ra,
                                  double rb, uint64_t probe_seed, void* work, double2* lam,
                                  double2* Yred, IterStatus* status) {
    if (m < 1 || m > beyn_max_m()) return cudaErrorInvalidValue;
    cudaError_t e;
    static std::atomic<bool> attr_done{false};   // idempotent setup; atomic for concurrent handles
    const size_t solve_smem = sizeof(float2) * ((size_t)m * nld(m) + (size_t)m * m + m) + sizeof(int) * m;
    const size_t svd_smem = 3 * sizeof(float2) * (size_t)m * m + (sizeof(float) + sizeof(int)) * m;
    if (!attr_done) {
        const int cap = 3 * 8 * 64 * 64 + 8 * 64 + 64;
        if ((e = cudaFuncSetAttribute(beyn_solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      cap)) != cudaSuccess) return e;
        if ((e = cudaFuncSetAttribute(beyn_svd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      cap)) != cudaSuccess) return e;
        if ((e = qr_select_attributes()) != cudaSuccess) return e;
        if ((e = cudaFuncSetAttribute(newton_kernel<float2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      220 * 1024)) != cudaSuccess) return e;
        if ((e = cudaFuncSetAttribute(newton_kernel<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      220 * 1024)) != cudaSuccess) return e;
        attr_done = true;
    }
    const BeynLayout L = beyn_layout(m);
    unsigned char* base = static_cast<unsigned char*>(work);
    double2* V = reinterpret_cast<double2*>(base + L.V);
    float2* P0 = reinterpret_cast<float2*>(base + L.P0);
    float2* P1 = reinterpret_cast<float2*>(base + L.P1);
    float2* A0 = reinterpret_cast<float2*>(base + L.A0);
    float2* A1 = reinterpret_cast<float2*>(base + L.A1);
    float2* B = reinterpret_cast<float2*>(base + L.B);
    float2* Hg = reinterpret_cast<float2*>(base + L.Hg);
    double2* lam0 = reinterpret_cast<double2*>(base + L.lam0);
    double* gap = reinterpret_cast<double*>(base + L.gap);
    int* flag = reinterpret_cast<int*>(base + L.flag);
    int* rank = reinterpret_cast<int*>(base + L.rank);
    const RedProblem P{-1, nullptr, nterms, terms, G, c_re, c_im, ra, rb};
    if ((e = random_block(st, m, m, probe_seed, V)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(flag, 0, sizeof(int), st)) != cudaSuccess) return e;
    note_launch();
    beyn_solve_kernel<<<kBeynNodes, kBeynThreads, solve_smem, st>>>(m, P, c_re, c_im, ra, rb, V, P0, P1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int64_t mm = (int64_t)m * m;
    note_launch();
    beyn_reduce_kernel<<<(unsigned)((mm + 255) / 256), 256, 0, st>>>(mm, P0, P1, A0, A1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    note_launch();
    beyn_svd_kernel<<<1, kSvdThreads, svd_smem, st>>>(m, A0, A1, c_re, c_im, ra, B, rank, status);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // eigenvalues of B (FP32 Hessenberg + QR), ranked by Step 2's rule
    int c0;
    size_t hsm;
    hessenberg_launch_shape<float>(m, &c0, &hsm);
    note_launch();
    hessenberg_kernel<float><<<1, kRedThreads, hsm, st>>>(m, B, c0, flag, 1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const size_t hbytes = packed_elems(m) * sizeof(float2);
    const size_t fixed = sizeof(float2) * ((size_t)m + kSmallLd * kSmallMax);
    const int use_smem = (hbytes + fixed) <= (size_t)kMaxSmemPacked;
    const size_t qsm = fixed + (use_smem ? hbytes : 0);
    note_launch();
    if (use_smem)
        qr_select_kernel<float, true, true><<<1, kQrThreads, qsm, st>>>(m, m, B, Hg, c_re, c_im, ra, rb,
                                                                        lam0, gap, flag, 1, status);
    else
        qr_select_kernel<float, false, true><<<1, kQrThreads, qsm, st>>>(m, m, B, Hg, c_re, c_im, ra,
                                                                         rb, lam0, gap, flag, 1, status);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // Newton per kept value (FP32 factor, FP64 residuals), fillers beyond the rank
    const size_t nsm32 = newton_smem<float2>(m);
    note_launch();
    newton_kernel<float2><<<m, kNewtonThreads, nsm32, st>>>(
        m, P, lam0, gap, lam, Yred, flag, 1, status, rank, make_double2(c_re + kBeynScale * ra, c_im),
        nullptr);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // a pair the FP32-factor Newton did not converge or moved too far: all kept
    // values refined again from the same starts with FP64 factors (device-side
    // no-op otherwise), so no Ritz value is left at its FP32 moment estimate
    const size_t nsm64 = newton_smem<double2>(m);
    note_launch();
    newton_kernel<double2><<<m, kNewtonThreads, nsm64, st>>>(
        m, P, lam0, gap, lam, Yred, flag, 2, status, rank, make_double2(c_re + kBeynScale * ra, c_im),
        nullptr);
    return cudaGetLastError();
}

cudaError_t chol_inverse(cudaStream_t st, int m, const double2* G, double shift_rel,
                         double2* Rinv, IterStatus* status) {
    static std::atomic<bool> attr_done{false};   // idempotent setup; atomic for concurrent handles
    if (!attr_done) {
        cudaError_t e = cudaFuncSetAttribute(chol_inverse_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             200 * 1024);
        if (e != cudaSuccess) return e;
        attr_done = true;
    }
    size_t smem = sizeof(float2) * 2 * (size_t)(m + 1) * m;
    note_launch();
    chol_inverse_kernel<<<1, 512, smem, st>>>(m, G, shift_rel, Rinv, status);
    return cudaGetLastError();
}

}  // namespace fnl
