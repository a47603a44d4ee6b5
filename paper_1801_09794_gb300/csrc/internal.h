// Internal declarations shared by the library's translation units.
// Storage convention inside the library: column-major, leading dimension given
// explicitly, complex numbers interleaved (double2 = complex128, float2 = complex64).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

// ---------------------------------------------------------------------------
// complex arithmetic on double2 / float2
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ double2 operator+(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ double2 operator-(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ double2 operator-(double2 a) { return make_double2(-a.x, -a.y); }
__host__ __device__ __forceinline__ double2 operator*(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__host__ __device__ __forceinline__ double2 operator*(double s, double2 a) { return make_double2(s * a.x, s * a.y); }
__host__ __device__ __forceinline__ float2 operator+(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 operator-(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ float2 operator-(float2 a) { return make_float2(-a.x, -a.y); }
__host__ __device__ __forceinline__ float2 operator*(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__host__ __device__ __forceinline__ float2 operator*(float s, float2 a) { return make_float2(s * a.x, s * a.y); }

// c + a*b
__host__ __device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 c) {
    return make_double2(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}
__host__ __device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 c) {
    return make_float2(fmaf(a.x, b.x, fmaf(-a.y, b.y, c.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, c.y)));
}
// c - a*b
__host__ __device__ __forceinline__ double2 cfms(double2 a, double2 b, double2 c) {
    return make_double2(fma(-a.x, b.x, fma(a.y, b.y, c.x)), fma(-a.x, b.y, fma(-a.y, b.x, c.y)));
}
__host__ __device__ __forceinline__ float2 cfms(float2 a, float2 b, float2 c) {
    return make_float2(fmaf(-a.x, b.x, fmaf(a.y, b.y, c.x)), fmaf(-a.x, b.y, fmaf(-a.y, b.x, c.y)));
}
__host__ __device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__host__ __device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__host__ __device__ __forceinline__ double cabs1(double2 a) { return fabs(a.x) + fabs(a.y); }
__host__ __device__ __forceinline__ float cabs1(float2 a) { return fabsf(a.x) + fabsf(a.y); }
__host__ __device__ __forceinline__ double cabs(double2 a) { return hypot(a.x, a.y); }
__host__ __device__ __forceinline__ float cabs(float2 a) { return hypotf(a.x, a.y); }
__host__ __device__ __forceinline__ double cnorm2(double2 a) { return a.x * a.x + a.y * a.y; }
__host__ __device__ __forceinline__ float cnorm2(float2 a) { return a.x * a.x + a.y * a.y; }
// 1/a with scaling against overflow
__host__ __device__ __forceinline__ double2 crcp(double2 a) {
    double s = fmax(fabs(a.x), fabs(a.y));
    if (s == 0.0) return make_double2(0.0, 0.0);
    double ar = a.x / s, ai = a.y / s, d = (ar * ar + ai * ai) * s;
    return make_double2(ar / d, -ai / d);
}
__host__ __device__ __forceinline__ float2 crcp(float2 a) {
    float s = fmaxf(fabsf(a.x), fabsf(a.y));
    if (s == 0.0f) return make_float2(0.0f, 0.0f);
    float ar = a.x / s, ai = a.y / s, d = (ar * ar + ai * ai) * s;
    return make_float2(ar / d, -ai / d);
}
__host__ __device__ __forceinline__ double2 cdiv(double2 a, double2 b) { return a * crcp(b); }

template <typename T> struct cplx_real;
template <> struct cplx_real<double2> { typedef double type; };
template <> struct cplx_real<float2> { typedef float type; };

template <typename T> __host__ __device__ __forceinline__ T cmake(double re, double im);
template <> __host__ __device__ __forceinline__ double2 cmake<double2>(double re, double im) { return make_double2(re, im); }
template <> __host__ __device__ __forceinline__ float2 cmake<float2>(double re, double im) { return make_float2((float)re, (float)im); }
__host__ __device__ __forceinline__ double2 to_d2(double2 a) { return a; }
__host__ __device__ __forceinline__ double2 to_d2(float2 a) { return make_double2(a.x, a.y); }
template <typename T> __host__ __device__ __forceinline__ T from_d2(double2 a);
template <> __host__ __device__ __forceinline__ double2 from_d2<double2>(double2 a) { return a; }
template <> __host__ __device__ __forceinline__ float2 from_d2<float2>(double2 a) { return make_float2((float)a.x, (float)a.y); }

namespace fnl {

constexpr int kMaxM0 = 112;       // largest subspace the single-CTA reduced kernels hold
constexpr int kMaxTerms = 16;
constexpr int kMaxPow = 8;

// Device-side description of one term of T(lambda).
struct TermDev {
    int kind;      // 0 pow, 1 exp
    int p;
    double tau;
    double2 scale;
    double norm;   // ||A_t||_2 estimate (1 for identity)
    int aidx;      // index into the stacked dense matrices, -1 = identity
    int pad;
};

// Per-iteration scalar results written by the device, read by the host.
struct IterStatus {
    int n_inside;
    int n_conv;
    int flags;         // bit 0: reduced QR hit its limit; bit 1: Ritz value on a node;
                       // bit 2: Cholesky breakdown; bit 3: Newton fallback used;
                       // bit 4: a tensor-core pipeline wait timed out
    int qr_sweeps;     // QR sweeps of the last reduced eigenvalue computation
    double max_relres;
};

// Sets the text returned by feast_nl_last_error() on the calling thread.
void set_last_error(const char* msg);

// Process-wide count of kernel launches issued by this library.
void note_launch(int k = 1);
uint64_t launch_count();

// ------------------------------------------------------------------ dense kernels (k_dense.cu)
// C = alpha * op(A) * B + beta * C, column-major, batched over `batch` with element
// strides sA, sB, sC.  opA: 0 = A (m x k), 1 = A^H (A stored k x m).
template <typename T>
cudaError_t gemm(cudaStream_t st, int opA, int m, int n, int k, T alpha, const T* A, int64_t lda,
                 int64_t sA, const T* B, int64_t ldb, int64_t sB, T beta, T* C, int64_t ldc,
                 int64_t sC, int batch);
// Same product with the k dimension split into `splits` chunks summed in a fixed
// order through `work` (splits * m * n elements); batch = 1.
cudaError_t gemm_splitk_d(cudaStream_t st, int opA, int m, int n, int k, double2 alpha,
                          const double2* A, int64_t lda, const double2* B, int64_t ldb,
                          double2 beta, double2* C, int64_t ldc, double2* work, int splits);

// G = Q^H Q (m x m, FP64 storage) from a complex64 Q (k x m): k split into
// `splits` chunks accumulated in FP32, the chunk sums added in FP64 (work holds
// splits * m * m complex64).
cudaError_t gram_f32(cudaStream_t st, int m, int k, const float2* Q, int64_t ldq, double2* G,
                     int64_t ldg, float2* work, int splits);
cudaError_t to_float(cudaStream_t st, int64_t cnt, const double2* src, float2* dst);

cudaError_t transpose_rowmajor_to_colmajor(cudaStream_t st, int64_t rows, int64_t cols,
                                           const double2* src, int64_t lds, double2* dst,
                                           int64_t ldd);
cudaError_t transpose_colmajor_to_rowmajor(cudaStream_t st, int64_t rows, int64_t cols,
                                           const double2* src, int64_t lds, double2* dst,
                                           int64_t ldd);
// y = A x (A n x n col-major) and y = A^H x
cudaError_t gemv_n(cudaStream_t st, int64_t n, const double2* A, const double2* x, double2* y,
                   double2* work);
cudaError_t gemv_c(cudaStream_t st, int64_t n, const double2* A, const double2* x, double2* y);
// out[0] = ||x||_2, x /= out[0] (if nonzero)
cudaError_t normalize_vec(cudaStream_t st, int64_t n, double2* x, double* out);
cudaError_t fill_ones(cudaStream_t st, int64_t n, double2* x);

// T(z_j) = sum_t coef[t*nc + j] * A_t + diagc[j] * I for every node j (FP64 arithmetic,
// result rounded once to T).
template <typename T>
cudaError_t assemble_nodes(cudaStream_t st, int64_t n, int nA, const double2* A,
                           const double2* coef, const double2* diagc, int nc, T* F,
                           int64_t strideF);

// complex normal start block (counter-based: splitmix64 + Box-Muller), n x m col-major
cudaError_t random_block(cudaStream_t st, int64_t n, int m, uint64_t seed, double2* X);
// Y_b <- convert(R_{b / nc}) for the nd * nc nodes b (R: nd blocks of n x m)
template <typename T>
cudaError_t broadcast_rhs(cudaStream_t st, int64_t n, int m, const double2* R, int nd, int nc,
                          T* Y, int64_t strideY);
cudaError_t filter_coefficients(cudaStream_t st, int nc, int m, const double2* z,
                                const double2* w, const double2* lam, double2* coef,
                                double2* fsum, IterStatus* status);
template <typename T>
cudaError_t accumulate_filter(cudaStream_t st, int64_t n, int m, int nc, const double2* X,
                              const T* Y, int64_t strideY, const double2* coef,
                              const double2* fsum, double2* Q);
// nrm[i] = ||col_i(X)||_2
cudaError_t column_norms(cudaStream_t st, int64_t n, int m, const double2* X, int64_t ldx,
                         double* nrm);
// X[:, i] /= nrm[i]; Ycat[t*m + a, i] = Y[a, i] * scale_t f_t(lam_i) / nrm[i]
cudaError_t ritz_scale(cudaStream_t st, int64_t n, int m, int nterms, const TermDev* terms,
                       const double2* lam, const double* nrm, double2* X, const double2* Y,
                       double2* Ycat);
// relres_i and the convergence summary
cudaError_t residual_summary(cudaStream_t st, int m, int nterms, const TermDev* terms,
                             const double2* lam, const double* rnorm, double c_re, double c_im,
                             double ra, double rb, double tol, double* relres,
                             IterStatus* status);
// Ahat_p = sum_{t: pow p} scale_t G_t  (G = Q^H [W_0 .. W_{T-1}], m x (T m))
cudaError_t form_reduced(cudaStream_t st, int m, int nterms, int kmax, const TermDev* terms,
                         const double2* G, double2* Ahat);
template <typename T>
cudaError_t to_double(cudaStream_t st, int64_t cnt, const T* src, double2* dst);
// Y = I (m x m), ones[0..m) = 1
cudaError_t set_identity(cudaStream_t st, int m, double2* Y, double* ones);
// identity terms of W (layout of ozaki_gemm, nd blocks of m columns): slot t of
// block b <- Q_b
// Diagonal coefficient terms: *flag <- 1 when A (n x n, column-major) has a
// nonzero off-diagonal entry; d <- diag(A); W block t of each of the nd
// contours <- diag(d) Q_d (Q: nd blocks of n x m, W: nd blocks of nterms).
cudaError_t offdiag_nonzero(cudaStream_t st, int64_t n, const double2* A, int64_t lda, int* flag);
cudaError_t extract_diagonal(cudaStream_t st, int64_t n, const double2* A, int64_t lda, double2* d);
cudaError_t diag_times(cudaStream_t st, int64_t n, int m, int nd, int nterms, int t, const double2* d,
                       const double2* Q, double2* W);
cudaError_t copy_identity_terms(cudaStream_t st, int64_t n, int m, int nd, int nterms,
                                const TermDev* terms, const double2* Q, double2* W);

// ------------------------------------------------------------------ digit-split products (k_ozaki.cu)
struct OzakiLayout {
    int s = 0;           // digit slices per operand
    int64_t Mpad = 0;    // rows of A' padded to the 128-row tile
    int64_t Kp = 0;      // 2n padded to the 64-byte K stage
    int64_t Npad = 0;    // 2m padded to the 64-column tile
    int64_t a_slice = 0, a_term = 0, b_slice = 0;   // elements (BF16)
};
// Digit slices per operand: the truncation remainder is below 2^{-7s} of the row /
// column scale, so s = 7 keeps the products at ~1e-14 relative accuracy.
constexpr int kOzakiSlices = 7;
OzakiLayout ozaki_layout(int64_t n, int m, int s);
bool ozaki_supported(int64_t n, int s);
// sigma (Mpad doubles) and the s digit slices of A' = [Re A | Im A] (A n x n col-major)
size_t ozaki_elem_bytes();
cudaError_t ozaki_split_A(cudaStream_t st, int64_t n, int s, const double2* A, double* sigma,
                          void* slices, const OzakiLayout& L);
// tau (m doubles) and the s digit slices of the real embedding of Q (n x m col-major)
cudaError_t ozaki_split_Q(cudaStream_t st, int64_t n, int m, int s, const double2* Q, double* tau,
                          void* slices, const OzakiLayout& L);
// A_t Q for the dense terms t < nterms, Q = n x m (complex128, col-major, ld n)
// made of m / mb blocks of mb columns (one block per contour); W holds per block
// `wterms` n x mb slots and A_t Q_b goes to slot term_slot[t] of block b:
// W + (b * wterms + term_slot[t]) * n * mb.  A failed internal wait sets bit 4 of *err.
// active (device, optional): column tiles whose blocks all have active[b] == 0
// are skipped (their W blocks are left as they were).
cudaError_t ozaki_gemm(cudaStream_t st, int64_t n, int m, int mb, int wterms, const OzakiLayout& L,
                       int nterms, const void* Aslices, const double* sigma, const void* Qslices,
                       const double* tau, double2* W, const int* term_slot, int* err,
                       const int* active = nullptr);

// C (M x N) = A (M x K) B (K x N), complex128 column-major (leading dimensions
// lda, ldb, ldc), FP64-accurate on the BF16 tensor cores (s digit slices of the
// row-scaled A and column-scaled B); work holds ozaki_general_work_bytes.  For
// the tall, thin products of the subspace steps (M = n, K and N a few m0).
size_t ozaki_general_work_bytes(int64_t M, int K, int N, int s);
cudaError_t ozaki_gemm_general(cudaStream_t st, int64_t M, int K, int N, const double2* A,
                               int64_t lda, const double2* B, int64_t ldb, double2* C, int64_t ldc,
                               int s, void* work, int* err);

// G (m x NT, col-major, ld m) = Q^H W for W (n x NT, col-major, ld ldw) and Q
// (n x m, col-major, ld ldq); FP64-accurate on the BF16 tensor cores (eight
// digit slices per operand), split over K.  work holds
// ozaki_project_work_bytes.  A failed internal wait sets bit 4 of *err.
size_t ozaki_project_work_bytes(int64_t n, int NT, int m);
cudaError_t ozaki_project(cudaStream_t st, int64_t n, int NT, int m, const double2* W, int64_t ldw,
                          const double2* Q, int64_t ldq, double2* G, void* work, int* err);

// ------------------------------------------------------------------ LU (k_lu.cu)
// One node matrix of a grouped factorisation (orders may differ): F is n x n
// column-major (leading dimension n) in the LU precision; piv (n), info (1),
// gather / gcount are this node's own slots (lu_gather_stride(n, nb) entries).
struct LuNode {
    void* F;
    int* piv;
    int* info;
    int2* gather;
    int* gcount;
    int64_t n;
};
// Column range of the look-ahead split for a node of order n at panel k0:
// the panel is jb wide; mode 0 = the next panel's columns, mode 1 = the rest.
// False when the range is empty (or the node has no panel k0).
__host__ __device__ __forceinline__ bool lookahead_cols(int64_t n, int k0, int nb, int mode, int* jb,
                                                        int* c0, int* ncols) {
    if (k0 >= n) return false;
    *jb = (int)(n - k0 < nb ? n - k0 : nb);
    const int64_t rest = n - k0 - *jb;
    const int64_t jn = rest < nb ? rest : nb;
    *c0 = (int)(k0 + *jb + (mode == 0 ? 0 : jn));
    *ncols = (int)(mode == 0 ? jn : rest - jn);
    return *ncols > 0;
}
// Factors nodes of different orders in one launch sequence per panel (grid
// dimension = node; a node whose order is exhausted skips the rest), complex64
// only, every order <= 4096; nodes: device array of count descriptors; n_host:
// their orders.  Same look-ahead as lu_factor_batched.
cudaError_t lu_factor_grouped(cudaStream_t st, const LuNode* nodes, const int64_t* n_host,
                              int count, int nb, int* err);

// The factorisation also writes, per node and panel, the panel's row interchanges
// as a gather list (gather: nc x lu_gather_stride int2, gcount: nc x panels ints),
// which the solves apply to the right-hand sides.
int lu_gather_stride(int64_t n, int nb);
// complex64 factors use the tensor-core update below; a failed internal wait
// sets bit 4 of *err.
template <typename T>
cudaError_t lu_factor_batched(cudaStream_t st, int64_t n, int nb, T* F, int64_t strideF,
                              int* piv, int nc, int* info, int2* gather, int* gcount, int* err);
// bn: tile width of the complex64 tensor-core updates (0 = cgemm_default_bn).
// active (device, optional): the systems of group g = node / group are skipped
// when active[g] == 0 (a finished contour's nodes; their Y is left as it was).
template <typename T>
cudaError_t lu_solve_batched(cudaStream_t st, int64_t n, int nb, const T* F, int64_t strideF,
                             const int2* gather, const int* gcount, int nc, T* Y,
                             int64_t strideY, int m, int* err, int bn = 0,
                             const int* active = nullptr, int group = 1);
// Autotuner of the complex64 solves: the tile width for nc systems of order n
// with m right-hand sides, chosen once per (n, m, nc) in the process by timing
// lu_solve_batched with every width on the given factors and on Y (which it
// overwrites: pass a scratch or not-yet-filled block), then cached.  During a
// stream capture, or when timing fails, the cached or default width is returned.
int lu_solve_pick_bn(cudaStream_t st, int64_t n, int nb, const float2* F, int64_t strideF,
                     const int2* gather, const int* gcount, int nc, float2* Y, int64_t strideY,
                     int m, int* err);

// ------------------------------------------------------------------ k_cgemm_tc.cu
// C -= A B (complex64, column-major, batch z advances A, B, C by sA, sB, sC) on
// the TF32 tensor cores with FP32-level accuracy (three TF32 products of the
// split operands); a failed internal wait sets bit 4 of *err.  bn: complex
// columns per CTA tile (16, 32, 48 or 64; 0 = the widest with the least waste).
// active (device, optional): batch entry z is skipped when active[z / group] == 0.
cudaError_t cgemm_sub_tf32x3(cudaStream_t st, int m, int n, int k, const float2* A, int64_t lda,
                             int64_t sA, const float2* B, int64_t ldb, int64_t sB, float2* C,
                             int64_t ldc, int64_t sC, int batch, int* err, int bn = 0,
                             const int* active = nullptr, int group = 1);
int cgemm_default_bn(int n);
// One CTA waits `cycles` on an mbarrier nothing signals, then sets bit 4 of *flags.
cudaError_t bounded_wait_probe(cudaStream_t st, long long cycles, int* flags);
// tile width of every LU trailing update (uniform and grouped alike, so that a
// node's factors do not depend on the path)
constexpr int kLuUpdateBn = 64;
// The LU's trailing update for grouped nodes (lu_factor_grouped): node z of
// `nodes`, panel at k0 of width min(nb, n - k0), columns of the look-ahead
// split `mode`; the grid covers the largest node (max_rows x max_cols).
cudaError_t cgemm_sub_grouped(cudaStream_t st, const LuNode* nodes, int count, int k0, int nb,
                              int mode, int64_t max_rows, int64_t max_cols, int* err);
template <typename T> int lu_block_size();

// ------------------------------------------------------------------ reduced problem (k_reduced.cu)
// From Ahat (kmax+1 stacked m x m FP64), compute all k*m eigenvalues of the
// companion pencil (FP32 Hessenberg QR), keep the m0 with the smallest normalised
// radius, refine each by Newton's method on the m x m polynomial in FP64, and
// return lam (m0) and unit vectors Yred (m x m0).
cudaError_t reduced_solve(cudaStream_t st, int m, int kmax, const double2* Ahat, int m0,
                          double c_re, double c_im, double ra, double rb, void* work,
                          double2* lam, double2* Yred, IterStatus* status);
size_t reduced_work_bytes(int m, int kmax);
// Steps 1-2 for general T (any term kinds): G = [G_0 | .. | G_{T-1}] (m x T m,
// G_t = Q^H A_t Q, scales applied through `terms`).  Eigenvalues of
// That(z) = sum_t f_t(z) G_t inside the contour scaled by 1.5 from the first two
// contour moments (FP32, 256 trapezoid nodes, probe drawn from probe_seed), ranked
// by Step 2's rule, refined by Newton; slots beyond the moments' rank get
// lambda = c + 1.5 ra and unit vectors.  m <= beyn_max_m().
size_t beyn_work_bytes(int m);
int beyn_max_m();
cudaError_t reduced_solve_general(cudaStream_t st, int m, int nterms, const TermDev* terms,
                                  const double2* G, double c_re, double c_im, double ra,
                                  double rb, uint64_t probe_seed, void* work, double2* lam,
                                  double2* Yred, IterStatus* status);
// Cholesky G = R^H R (with diagonal shift), returns R^{-1} (upper) in Rinv.
cudaError_t chol_inverse(cudaStream_t st, int m, const double2* G, double shift_rel,
                         double2* Rinv, IterStatus* status);

}  // namespace fnl
