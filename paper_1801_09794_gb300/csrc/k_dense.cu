// Dense building blocks of the filter step: complex GEMM, node assembly,
// filter accumulation and the bookkeeping of Steps 2-4 (Algorithm 1).
#include "internal.h"
#include <atomic>

namespace fnl {

static std::atomic<uint64_t> g_launches{0};
void note_launch(int k) { g_launches.fetch_add((uint64_t)k, std::memory_order_relaxed); }
uint64_t launch_count() { return g_launches.load(std::memory_order_relaxed); }

// ============================================================================
// Complex GEMM, SIMT, 64x64 output tile per 256-thread CTA, 4x4 per thread.
//   C = alpha * op(A) * B + beta * C      (column-major)
// blockIdx.z enumerates (batch, k-split) pairs: z = b * splits + s, and the CTA
// sums k over [s*kchunk, min(k, (s+1)*kchunk)).  C advances by sC per z.
// ============================================================================
namespace {
constexpr int BM = 64, BN = 64, BK = 16;

template <typename T, int OPA>
__global__ void __launch_bounds__(256) gemm_kernel(int m, int n, int k, int kchunk, int splits,
                                                   T alpha, const T* __restrict__ A,
                                                   int64_t lda, int64_t sA,
                                                   const T* __restrict__ B, int64_t ldb,
                                                   int64_t sB, T beta, T* __restrict__ C,
                                                   int64_t ldc, int64_t sC) {
    __shared__ T As[BK][BM + 1];
    __shared__ T Bs[BK][BN + 1];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int z = blockIdx.z;
    const int b = z / splits, s = z - b * splits;
    const int row0 = blockIdx.x * BM, col0 = blockIdx.y * BN;
    const int kbeg = s * kchunk;
    const int kend = min(k, kbeg + kchunk);
    A += b * sA;
    B += b * sB;
    C += (int64_t)z * sC;
    typedef typename cplx_real<T>::type R;
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = cmake<T>(0.0, 0.0);

    for (int k0 = kbeg; k0 < kend; k0 += BK) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int idx = tid + 256 * q;
            int r, kk;
            if (OPA == 0) { r = idx & 63; kk = idx >> 6; }
            else          { kk = idx & 15; r = idx >> 4; }
            int gr = row0 + r, gk = k0 + kk;
            T v = cmake<T>(0.0, 0.0);
            if (gr < m && gk < kend) {
                if (OPA == 0) v = A[gr + (int64_t)gk * lda];
                else          v = cconj(A[gk + (int64_t)gr * lda]);
            }
            As[kk][r] = v;
            int kb = idx & 15, c = idx >> 4;
            int gc = col0 + c, gkb = k0 + kb;
            T w = cmake<T>(0.0, 0.0);
            if (gc < n && gkb < kend) w = B[gkb + (int64_t)gc * ldb];
            Bs[kb][c] = w;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            T a[4], bb[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][tx + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bb[j] = Bs[kk][ty + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = cfma(a[i], bb[j], acc[i][j]);
        }
        __syncthreads();
    }
    const bool zero_beta = (beta.x == (R)0 && beta.y == (R)0);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        int gc = col0 + ty + 16 * j;
        if (gc >= n) continue;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            int gr = row0 + tx + 16 * i;
            if (gr >= m) continue;
            T* p = C + gr + (int64_t)gc * ldc;
            T v = alpha * acc[i][j];
            if (!zero_beta) v = cfma(beta, *p, v);
            *p = v;
        }
    }
}

__global__ void reduce_splits_kernel(int m, int n, int splits, double2 alpha,
                                     const double2* __restrict__ work, double2 beta,
                                     double2* __restrict__ C, int64_t ldc) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t mn = (int64_t)m * n;
    if (e >= mn) return;
    double2 s = make_double2(0.0, 0.0);
    for (int q = 0; q < splits; ++q) s = s + work[q * mn + e];
    int i = (int)(e % m), j = (int)(e / m);
    double2* p = C + i + (int64_t)j * ldc;
    double2 v = alpha * s;
    if (beta.x != 0.0 || beta.y != 0.0) v = cfma(beta, *p, v);
    *p = v;
}
}  // namespace

template <typename T>
cudaError_t gemm(cudaStream_t st, int opA, int m, int n, int k, T alpha, const T* A, int64_t lda,
                 int64_t sA, const T* B, int64_t ldb, int64_t sB, T beta, T* C, int64_t ldc,
                 int64_t sC, int batch) {
    if (m <= 0 || n <= 0 || batch <= 0) return cudaSuccess;
    dim3 grid((m + BM - 1) / BM, (n + BN - 1) / BN, batch);
    int kc = k > 0 ? k : 1;
    note_launch();
    if (opA == 0)
        gemm_kernel<T, 0><<<grid, 256, 0, st>>>(m, n, k, kc, 1, alpha, A, lda, sA, B, ldb, sB,
                                                beta, C, ldc, sC);
    else
        gemm_kernel<T, 1><<<grid, 256, 0, st>>>(m, n, k, kc, 1, alpha, A, lda, sA, B, ldb, sB,
                                                beta, C, ldc, sC);
    return cudaGetLastError();
}
template cudaError_t gemm<double2>(cudaStream_t, int, int, int, int, double2, const double2*,
                                   int64_t, int64_t, const double2*, int64_t, int64_t, double2,
                                   double2*, int64_t, int64_t, int);
template cudaError_t gemm<float2>(cudaStream_t, int, int, int, int, float2, const float2*,
                                  int64_t, int64_t, const float2*, int64_t, int64_t, float2,
                                  float2*, int64_t, int64_t, int);

cudaError_t gemm_splitk_d(cudaStream_t st, int opA, int m, int n, int k, double2 alpha,
                          const double2* A, int64_t lda, const double2* B, int64_t ldb,
                          double2 beta, double2* C, int64_t ldc, double2* work, int splits) {
    if (m <= 0 || n <= 0) return cudaSuccess;
    if (splits < 1) splits = 1;
    int kchunk = (k + splits - 1) / splits;
    kchunk = ((kchunk + BK - 1) / BK) * BK;
    if (kchunk < BK) kchunk = BK;
    splits = (k + kchunk - 1) / kchunk;
    if (splits < 1) splits = 1;
    dim3 grid((m + BM - 1) / BM, (n + BN - 1) / BN, splits);
    const double2 one = make_double2(1.0, 0.0), zero = make_double2(0.0, 0.0);
    int64_t mn = (int64_t)m * n;
    note_launch();
    if (opA == 0)
        gemm_kernel<double2, 0><<<grid, 256, 0, st>>>(m, n, k, kchunk, splits, one, A, lda, 0, B,
                                                      ldb, 0, zero, work, m, mn);
    else
        gemm_kernel<double2, 1><<<grid, 256, 0, st>>>(m, n, k, kchunk, splits, one, A, lda, 0, B,
                                                      ldb, 0, zero, work, m, mn);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    note_launch();
    reduce_splits_kernel<<<(unsigned)((mn + 255) / 256), 256, 0, st>>>(m, n, splits, alpha, work,
                                                                       beta, C, ldc);
    return cudaGetLastError();
}

namespace {
__global__ void reduce_splits_f_kernel(int m, int splits, const float2* __restrict__ work,
                                       double2* __restrict__ G, int64_t ldg) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t mm = (int64_t)m * m;
    if (e >= mm) return;
    double2 s = make_double2(0.0, 0.0);
    for (int q = 0; q < splits; ++q) {
        const float2 v = work[q * mm + e];
        s = s + make_double2(v.x, v.y);
    }
    G[(e % m) + (e / m) * ldg] = s;
}
__global__ void to_float_kernel(int64_t cnt, const double2* __restrict__ src, float2* __restrict__ dst) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < cnt) dst[i] = make_float2((float)src[i].x, (float)src[i].y);
}
}  // namespace

cudaError_t gram_f32(cudaStream_t st, int m, int k, const float2* Q, int64_t ldq, double2* G,
                     int64_t ldg, float2* work, int splits) {
    if (m <= 0) return cudaSuccess;
    if (splits < 1) splits = 1;
    int kchunk = (k + splits - 1) / splits;
    kchunk = ((kchunk + BK - 1) / BK) * BK;
    if (kchunk < BK) kchunk = BK;
    splits = (k + kchunk - 1) / kchunk;
    if (splits < 1) splits = 1;
    dim3 grid((m + BM - 1) / BM, (m + BN - 1) / BN, splits);
    const int64_t mm = (int64_t)m * m;
    note_launch();
    gemm_kernel<float2, 1><<<grid, 256, 0, st>>>(m, m, k, kchunk, splits, make_float2(1.f, 0.f), Q,
                                                 ldq, 0, Q, ldq, 0, make_float2(0.f, 0.f), work, m,
                                                 mm);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    note_launch();
    reduce_splits_f_kernel<<<(unsigned)((mm + 255) / 256), 256, 0, st>>>(m, splits, work, G, ldg);
    return cudaGetLastError();
}

cudaError_t to_float(cudaStream_t st, int64_t cnt, const double2* src, float2* dst) {
    if (cnt <= 0) return cudaSuccess;
    note_launch();
    to_float_kernel<<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(cnt, src, dst);
    return cudaGetLastError();
}

// ============================================================================
// Layout changes at the ABI boundary (row-major <-> column-major)
// ============================================================================
namespace {
__global__ void transpose_kernel(int64_t rows, int64_t cols, const double2* __restrict__ src,
                                 int64_t lds, double2* __restrict__ dst, int64_t ldd,
                                 int src_rowmajor) {
    // Reads a 32x32 block of the source in its storage order and writes it in the
    // other order; src_rowmajor selects which side is row-major.
    __shared__ double2 tile[32][33];
    int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
    int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
    if (src_rowmajor) {
        for (int q = ty; q < 32; q += 8) {
            int64_t r = r0 + q, c = c0 + tx;
            if (r < rows && c < cols) tile[q][tx] = src[r * lds + c];
        }
        __syncthreads();
        for (int q = ty; q < 32; q += 8) {
            int64_t c = c0 + q, r = r0 + tx;
            if (r < rows && c < cols) dst[r + c * ldd] = tile[tx][q];
        }
    } else {
        for (int q = ty; q < 32; q += 8) {
            int64_t c = c0 + q, r = r0 + tx;
            if (r < rows && c < cols) tile[tx][q] = src[r + c * lds];
        }
        __syncthreads();
        for (int q = ty; q < 32; q += 8) {
            int64_t r = r0 + q, c = c0 + tx;
            if (r < rows && c < cols) dst[r * ldd + c] = tile[q][tx];
        }
    }
}
}  // namespace

cudaError_t transpose_rowmajor_to_colmajor(cudaStream_t st, int64_t rows, int64_t cols,
                                           const double2* src, int64_t lds, double2* dst,
                                           int64_t ldd) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    dim3 grid((unsigned)((cols + 31) / 32), (unsigned)((rows + 31) / 32));
    note_launch();
    transpose_kernel<<<grid, dim3(32, 8), 0, st>>>(rows, cols, src, lds, dst, ldd, 1);
    return cudaGetLastError();
}
cudaError_t transpose_colmajor_to_rowmajor(cudaStream_t st, int64_t rows, int64_t cols,
                                           const double2* src, int64_t lds, double2* dst,
                                           int64_t ldd) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    dim3 grid((unsigned)((cols + 31) / 32), (unsigned)((rows + 31) / 32));
    note_launch();
    transpose_kernel<<<grid, dim3(32, 8), 0, st>>>(rows, cols, src, lds, dst, ldd, 0);
    return cudaGetLastError();
}

// ============================================================================
// Matrix-vector products for the ||A||_2 power estimate
// ============================================================================
namespace {
constexpr int kGemvSplit = 32;
__global__ void gemv_n_kernel(int64_t n, const double2* __restrict__ A,
                              const double2* __restrict__ x, double2* __restrict__ work) {
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int s = blockIdx.y;
    int64_t chunk = (n + kGemvSplit - 1) / kGemvSplit;
    int64_t c0 = s * chunk, c1 = min(n, c0 + chunk);
    if (r >= n) return;
    // four independent accumulators keep four column loads in flight
    double2 acc[4] = {make_double2(0.0, 0.0), make_double2(0.0, 0.0), make_double2(0.0, 0.0),
                      make_double2(0.0, 0.0)};
    int64_t c = c0;
    for (; c + 3 < c1; c += 4) {
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[q] = cfma(A[r + (c + q) * n], x[c + q], acc[q]);
    }
    for (; c < c1; ++c) acc[0] = cfma(A[r + c * n], x[c], acc[0]);
    work[s * n + r] = (acc[0] + acc[1]) + (acc[2] + acc[3]);
}
__global__ void gemv_n_reduce(int64_t n, const double2* __restrict__ work, double2* __restrict__ y) {
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n) return;
    double2 acc = make_double2(0.0, 0.0);
    for (int s = 0; s < kGemvSplit; ++s) acc = acc + work[s * n + r];
    y[r] = acc;
}
__global__ void gemv_c_kernel(int64_t n, const double2* __restrict__ A,
                              const double2* __restrict__ x, double2* __restrict__ y) {
    int64_t col = blockIdx.x * (int64_t)(blockDim.x / 32) + threadIdx.x / 32;
    int lane = threadIdx.x & 31;
    if (col >= n) return;
    const double2* a = A + col * n;
    double2 acc4[4] = {make_double2(0.0, 0.0), make_double2(0.0, 0.0), make_double2(0.0, 0.0),
                       make_double2(0.0, 0.0)};
    int64_t r = lane;
    for (; r + 96 < n; r += 128) {
#pragma unroll
        for (int q = 0; q < 4; ++q) acc4[q] = cfma(cconj(a[r + 32 * q]), x[r + 32 * q], acc4[q]);
    }
    for (; r < n; r += 32) acc4[0] = cfma(cconj(a[r]), x[r], acc4[0]);
    double2 acc = (acc4[0] + acc4[1]) + (acc4[2] + acc4[3]);
    for (int o = 16; o > 0; o >>= 1) {
        acc.x += __shfl_down_sync(0xffffffffu, acc.x, o);
        acc.y += __shfl_down_sync(0xffffffffu, acc.y, o);
    }
    if (lane == 0) y[col] = acc;
}
__global__ void normalize_kernel(int64_t n, double2* x, double* out) {
    __shared__ double red[32];
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += cnorm2(x[i]);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) red[0] = sqrt(s);
    }
    __syncthreads();
    double nrm = red[0];
    if (threadIdx.x == 0) out[0] = nrm;
    if (nrm > 0.0) {
        double inv = 1.0 / nrm;
        for (int64_t i = threadIdx.x; i < n; i += blockDim.x) x[i] = inv * x[i];
    }
}
__global__ void fill_ones_kernel(int64_t n, double2* x) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) x[i] = make_double2(1.0, 0.0);
}
}  // namespace

cudaError_t gemv_n(cudaStream_t st, int64_t n, const double2* A, const double2* x, double2* y,
                   double2* work) {
    dim3 grid((unsigned)((n + 127) / 128), kGemvSplit);
    note_launch();
    gemv_n_kernel<<<grid, 128, 0, st>>>(n, A, x, work);
    note_launch();
    gemv_n_reduce<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, work, y);
    return cudaGetLastError();
}
cudaError_t gemv_c(cudaStream_t st, int64_t n, const double2* A, const double2* x, double2* y) {
    note_launch();
    gemv_c_kernel<<<(unsigned)((n + 7) / 8), 256, 0, st>>>(n, A, x, y);
    return cudaGetLastError();
}
cudaError_t normalize_vec(cudaStream_t st, int64_t n, double2* x, double* out) {
    note_launch();
    normalize_kernel<<<1, 1024, 0, st>>>(n, x, out);
    return cudaGetLastError();
}
cudaError_t fill_ones(cudaStream_t st, int64_t n, double2* x) {
    note_launch();
    fill_ones_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, x);
    return cudaGetLastError();
}

// ============================================================================
// Node assembly T(z_j) = sum_t f_t(z_j) scale_t A_t (+ identity terms)
// One pass over the A_t: every element is read once and written for all nodes.
// ============================================================================
namespace {
template <typename T, int NA>
__global__ void assemble_kernel(int64_t n, int nA, const double2* __restrict__ A,
                                const double2* __restrict__ coef,
                                const double2* __restrict__ diagc, int nc, T* __restrict__ F,
                                int64_t strideF) {
    const int64_t nn = n * n;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nn;
         e += (int64_t)gridDim.x * blockDim.x) {
        const bool diag = (e % (n + 1)) == 0;
        double2 a[NA > 0 ? NA : 1];
        if (NA > 0) {
#pragma unroll
            for (int t = 0; t < NA; ++t) a[t] = A[t * nn + e];
        }
        for (int j = 0; j < nc; ++j) {
            double2 v = diag ? diagc[j] : make_double2(0.0, 0.0);
            if (NA > 0) {
#pragma unroll
                for (int t = 0; t < NA; ++t) v = cfma(coef[t * nc + j], a[t], v);
            } else {
                for (int t = 0; t < nA; ++t) v = cfma(coef[t * nc + j], A[t * nn + e], v);
            }
            F[j * strideF + e] = from_d2<T>(v);
        }
    }
}
// Complex64 node matrices are formed without FP64 arithmetic: the FP64 version
// above is bound by the FP64 rate (4 DFMA per term, node and element), this one
// by the HBM writes of the factors.  To keep the result as accurate as the
// FP64 sum rounded once (the node matrices of the delay problem are
// ill-conditioned enough for a few extra FP32 roundings to slow the iteration
// down), every A_t entry and coefficient is split into two FP32 parts (hi + lo,
// the lo part from the exact FP64 difference, once per element or per block),
// each real product is formed as hi*hi with its exact FMA error plus the two
// cross terms, and the terms are summed as an unevaluated FP32 pair (TwoSum);
// the pair is rounded once to complex64.
struct FF { float hi, lo; };
__device__ __forceinline__ FF ff_split(double x) {
    const float h = (float)x;
    return {h, (float)(x - (double)h)};
}
// s += x * y (x, y, s as FP32 pairs; the lo*lo term is below the FP32 ulp of the sum)
// (explicitly rounded operations: a contraction into an FMA would break TwoSum)
__device__ __forceinline__ void ff_madd(FF& s, FF x, FF y, float sign) {
    const float xh = sign * x.hi, xl = sign * x.lo;
    const float ph = __fmul_rn(xh, y.hi);
    const float pe = fmaf(xh, y.hi, -ph);
    const float pl = fmaf(xh, y.lo, fmaf(xl, y.hi, pe));
    const float t = __fadd_rn(s.hi, ph);
    const float bv = __fsub_rn(t, s.hi);
    const float err = __fadd_rn(__fsub_rn(s.hi, __fsub_rn(t, bv)), __fsub_rn(ph, bv));
    s.hi = t;
    s.lo += err + pl;
}
template <int NA>
__global__ void assemble_f32_kernel(int64_t n, int nA, const double2* __restrict__ A,
                                    const double2* __restrict__ coef,
                                    const double2* __restrict__ diagc, int nc,
                                    float2* __restrict__ F, int64_t strideF) {
    extern __shared__ FF s_coef[];              // (re, im) pairs: nA * nc coefficients, then nc diagonal ones
    const int ncoef = nA * nc;
    for (int e = threadIdx.x; e < ncoef + nc; e += blockDim.x) {
        const double2 c = e < ncoef ? coef[e] : diagc[e - ncoef];
        s_coef[2 * e] = ff_split(c.x);
        s_coef[2 * e + 1] = ff_split(c.y);
    }
    __syncthreads();
    const FF* s_diag = s_coef + 2 * ncoef;
    const int64_t nn = n * n;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nn;
         e += (int64_t)gridDim.x * blockDim.x) {
        const bool diag = (e % (n + 1)) == 0;
        FF ar[NA], ai[NA];
#pragma unroll
        for (int t = 0; t < NA; ++t) {
            const double2 v = A[t * nn + e];
            ar[t] = ff_split(v.x);
            ai[t] = ff_split(v.y);
        }
        for (int j = 0; j < nc; ++j) {
            FF re = diag ? s_diag[2 * j] : FF{0.f, 0.f};
            FF im = diag ? s_diag[2 * j + 1] : FF{0.f, 0.f};
#pragma unroll
            for (int t = 0; t < NA; ++t) {
                const FF cr = s_coef[2 * (t * nc + j)], ci = s_coef[2 * (t * nc + j) + 1];
                ff_madd(re, cr, ar[t], 1.f);
                ff_madd(re, ci, ai[t], -1.f);
                ff_madd(im, cr, ai[t], 1.f);
                ff_madd(im, ci, ar[t], 1.f);
            }
            F[j * strideF + e] = make_float2(re.hi + re.lo, im.hi + im.lo);
        }
    }
}
}  // namespace

template <typename T>
cudaError_t assemble_nodes(cudaStream_t st, int64_t n, int nA, const double2* A,
                           const double2* coef, const double2* diagc, int nc, T* F,
                           int64_t strideF) {
    int64_t nn = n * n;
    int64_t want = (nn + 255) / 256;
    int blocks = (int)(want < 152 * 16 ? want : 152 * 16);
    if constexpr (sizeof(T) == 8) {
        const size_t smem = 2 * sizeof(float2) * (size_t)nc * (nA + 1);
        if (nA >= 1 && nA <= 4 && smem <= 48 * 1024) {
            note_launch();
            switch (nA) {
                case 1: assemble_f32_kernel<1><<<blocks, 256, smem, st>>>(n, nA, A, coef, diagc, nc, F, strideF); break;
                case 2: assemble_f32_kernel<2><<<blocks, 256, smem, st>>>(n, nA, A, coef, diagc, nc, F, strideF); break;
                case 3: assemble_f32_kernel<3><<<blocks, 256, smem, st>>>(n, nA, A, coef, diagc, nc, F, strideF); break;
                default: assemble_f32_kernel<4><<<blocks, 256, smem, st>>>(n, nA, A, coef, diagc, nc, F, strideF); break;
            }
            return cudaGetLastError();
        }
    }
    switch (nA) {
        case 1: note_launch(); assemble_kernel<T, 1><<<blocks, 256, 0, st>>>(n, nA, A, coef, diagc, nc, F, strideF); break;
        case 2: note_launch(); assemble_kernel<T, 2><<<blocks, 256, 0, st>>>(n, nA, A, coef, diagc, nc, F, strideF); break;
        case 3: note_launch(); assemble_kernel<T, 3><<<blocks, 256, 0, st>>>(n, nA, A, coef, diagc, nc, F, strideF); break;
        case 4: note_launch(); assemble_kernel<T, 4><<<blocks, 256, 0, st>>>(n, nA, A, coef, diagc, nc, F, strideF); break;
        default: note_launch(); assemble_kernel<T, 0><<<blocks, 256, 0, st>>>(n, nA, A, coef, diagc, nc, F, strideF); break;
    }
    return cudaGetLastError();
}
template cudaError_t assemble_nodes<double2>(cudaStream_t, int64_t, int, const double2*,
                                             const double2*, const double2*, int, double2*,
                                             int64_t);
template cudaError_t assemble_nodes<float2>(cudaStream_t, int64_t, int, const double2*,
                                            const double2*, const double2*, int, float2*,
                                            int64_t);

// ============================================================================
// Start block, node right-hand sides, filter coefficients and accumulation
// ============================================================================
namespace {
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}
__global__ void random_block_kernel(int64_t total, uint64_t seed, double2* X) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= total) return;
    uint64_t h1 = splitmix64(seed * 0x100000001B3ull + 2 * (uint64_t)e);
    uint64_t h2 = splitmix64(seed * 0x100000001B3ull + 2 * (uint64_t)e + 1);
    double u1 = ((h1 >> 11) + 1.0) * (1.0 / 9007199254740993.0);   // (0, 1]
    double u2 = (h2 >> 11) * (1.0 / 9007199254740992.0);           // [0, 1)
    double rad = sqrt(-2.0 * log(u1));
    double s, c;
    sincospi(2.0 * u2, &s, &c);
    X[e] = make_double2(rad * c * 0.7071067811865476, rad * s * 0.7071067811865476);
}
template <typename T>
__global__ void broadcast_rhs_kernel(int64_t nm, const double2* __restrict__ R, int nc,
                                     T* __restrict__ Y, int64_t strideY) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= nm) return;
    const int d = blockIdx.y;                      // contour: nodes d*nc .. d*nc+nc-1
    T v = from_d2<T>(R[d * nm + e]);
    T* Yd = Y + (int64_t)d * nc * strideY;
    for (int j = 0; j < nc; ++j) Yd[j * strideY + e] = v;
}
__global__ void filter_coef_kernel(int nc, int m, const double2* __restrict__ z,
                                   const double2* __restrict__ w,
                                   const double2* __restrict__ lam, double2* __restrict__ coef,
                                   double2* __restrict__ fsum, IterStatus* status) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    double2 f = make_double2(0.0, 0.0);
    double2 li = lam[i];
    for (int j = 0; j < nc; ++j) {
        double2 d = z[j] - li;
        if (d.x == 0.0 && d.y == 0.0) {
            atomicOr(&status->flags, 2);
            coef[j * m + i] = make_double2(0.0, 0.0);
            continue;
        }
        double2 c = cdiv(w[j], d);
        coef[j * m + i] = c;
        f = f + c;
    }
    fsum[i] = f;
}
template <typename T>
__global__ void accumulate_kernel(int64_t n, int m, int nc, const double2* __restrict__ X,
                                  const T* __restrict__ Y, int64_t strideY,
                                  const double2* __restrict__ coef,
                                  const double2* __restrict__ fsum, double2* __restrict__ Q) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n * m) return;
    int i = (int)(e / n);
    double2 q = fsum[i] * X[e];
    for (int j = 0; j < nc; ++j) q = cfms(coef[j * m + i], to_d2(Y[j * strideY + e]), q);
    Q[e] = q;
}
}  // namespace

cudaError_t random_block(cudaStream_t st, int64_t n, int m, uint64_t seed, double2* X) {
    int64_t tot = n * m;
    note_launch();
    random_block_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(tot, seed, X);
    return cudaGetLastError();
}
template <typename T>
cudaError_t broadcast_rhs(cudaStream_t st, int64_t n, int m, const double2* R, int nd, int nc,
                          T* Y, int64_t strideY) {
    int64_t nm = n * m;
    note_launch();
    dim3 g((unsigned)((nm + 255) / 256), (unsigned)nd);
    broadcast_rhs_kernel<T><<<g, 256, 0, st>>>(nm, R, nc, Y, strideY);
    return cudaGetLastError();
}
template cudaError_t broadcast_rhs<double2>(cudaStream_t, int64_t, int, const double2*, int, int,
                                            double2*, int64_t);
template cudaError_t broadcast_rhs<float2>(cudaStream_t, int64_t, int, const double2*, int, int,
                                           float2*, int64_t);
cudaError_t filter_coefficients(cudaStream_t st, int nc, int m, const double2* z,
                                const double2* w, const double2* lam, double2* coef,
                                double2* fsum, IterStatus* status) {
    note_launch();
    filter_coef_kernel<<<(m + 127) / 128, 128, 0, st>>>(nc, m, z, w, lam, coef, fsum, status);
    return cudaGetLastError();
}
template <typename T>
cudaError_t accumulate_filter(cudaStream_t st, int64_t n, int m, int nc, const double2* X,
                              const T* Y, int64_t strideY, const double2* coef,
                              const double2* fsum, double2* Q) {
    int64_t nm = n * m;
    note_launch();
    accumulate_kernel<T><<<(unsigned)((nm + 255) / 256), 256, 0, st>>>(n, m, nc, X, Y, strideY,
                                                                      coef, fsum, Q);
    return cudaGetLastError();
}
template cudaError_t accumulate_filter<double2>(cudaStream_t, int64_t, int, int, const double2*,
                                                const double2*, int64_t, const double2*,
                                                const double2*, double2*);
template cudaError_t accumulate_filter<float2>(cudaStream_t, int64_t, int, int, const double2*,
                                               const float2*, int64_t, const double2*,
                                               const double2*, double2*);

// ============================================================================
// Ritz vectors, block residual bookkeeping, Step 3 test
// ============================================================================
namespace {
__device__ double2 term_f(const TermDev& t, double2 lam) {
    double2 v;
    if (t.kind == 0) {
        v = make_double2(1.0, 0.0);
        for (int q = 0; q < t.p; ++q) v = v * lam;
    } else {
        // exp(-tau * lam)
        double er = exp(-t.tau * lam.x);
        double s, c;
        sincos(-t.tau * lam.y, &s, &c);
        v = make_double2(er * c, er * s);
    }
    return t.scale * v;
}
__global__ void column_norms_kernel(int64_t n, const double2* __restrict__ X, int64_t ldx,
                                    double* __restrict__ nrm) {
    __shared__ double red[32];
    const double2* x = X + blockIdx.x * ldx;
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += cnorm2(x[i]);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) nrm[blockIdx.x] = sqrt(s);
    }
}
__global__ void scale_columns_kernel(int64_t n, int m, const double* __restrict__ nrm,
                                     double2* __restrict__ X) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n * m) return;
    int i = (int)(e / n);
    double s = nrm[i] > 0.0 ? 1.0 / nrm[i] : 0.0;
    X[e] = s * X[e];
}
__global__ void ycat_kernel(int m, int nterms, const TermDev* __restrict__ terms,
                            const double2* __restrict__ lam, const double* __restrict__ nrm,
                            const double2* __restrict__ Y, double2* __restrict__ Ycat) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t Tm = (int64_t)nterms * m;
    if (e >= Tm * m) return;
    int i = (int)(e / Tm);
    int r = (int)(e - (int64_t)i * Tm);
    int t = r / m, a = r - t * m;
    double s = nrm[i] > 0.0 ? 1.0 / nrm[i] : 0.0;
    Ycat[e] = s * (Y[a + (int64_t)i * m] * term_f(terms[t], lam[i]));
}
__global__ void residual_summary_kernel(int m, int nterms, const TermDev* __restrict__ terms,
                                        const double2* __restrict__ lam,
                                        const double* __restrict__ rnorm, double c_re,
                                        double c_im, double ra, double rb, double tol,
                                        double* __restrict__ relres, IterStatus* status) {
    __shared__ int s_in, s_conv;
    __shared__ double s_max;
    if (threadIdx.x == 0) { s_in = 0; s_conv = 0; s_max = 0.0; }
    __syncthreads();
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        double den = 0.0;
        for (int t = 0; t < nterms; ++t) den += cabs(term_f(terms[t], lam[i])) * terms[t].norm;
        double rr = den > 0.0 ? rnorm[i] / den : rnorm[i];
        relres[i] = rr;
        double dx = (lam[i].x - c_re) / ra, dy = (lam[i].y - c_im) / rb;
        double rho = sqrt(dx * dx + dy * dy);
        if (rho < 1.0) {
            atomicAdd(&s_in, 1);
            if (rr <= tol) atomicAdd(&s_conv, 1);
            // max of non-negative doubles through their bit patterns
            atomicMax((unsigned long long*)&s_max, (unsigned long long)__double_as_longlong(rr));
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        status->n_inside = s_in;
        status->n_conv = s_conv;
        status->max_relres = s_max;
    }
}
__global__ void form_reduced_kernel(int m, int nterms, int kmax, const TermDev* __restrict__ terms,
                                    const double2* __restrict__ G, double2* __restrict__ Ahat) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t mm = (int64_t)m * m;
    if (e >= (kmax + 1) * mm) return;
    int p = (int)(e / mm);
    int64_t ab = e - p * mm;
    int a = (int)(ab % m), b = (int)(ab / m);
    double2 v = make_double2(0.0, 0.0);
    for (int t = 0; t < nterms; ++t) {
        if (terms[t].kind != 0 || terms[t].p != p) continue;
        v = cfma(terms[t].scale, G[a + (int64_t)(t * m + b) * m], v);
    }
    Ahat[e] = v;
}
// flag <- 1 when some off-diagonal entry of the n x n column-major A is
// nonzero (exact test)
__global__ void offdiag_nonzero_kernel(int64_t n, const double2* __restrict__ A, int64_t lda,
                                       int* flag) {
    bool nz = false;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e % n, j = e / n;
        const double2 a = A[i + j * lda];
        nz = nz || (i != j && (a.x != 0.0 || a.y != 0.0));
    }
    if (__syncthreads_or(nz) && threadIdx.x == 0) *flag = 1;
}
__global__ void diagonal_kernel(int64_t n, const double2* __restrict__ A, int64_t lda,
                                double2* __restrict__ d) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) d[i] = A[i + i * lda];
}
// W block t of every contour d <- diag(dg) Q_d (FP64 products, rounded once)
__global__ void diag_times_kernel(int64_t n, int64_t nm, int nterms, int t,
                                  const double2* __restrict__ dg, const double2* __restrict__ Q,
                                  double2* __restrict__ W) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= nm) return;
    const int d = blockIdx.y;
    W[(int64_t)d * nterms * nm + (int64_t)t * nm + e] = dg[e % n] * Q[d * nm + e];
}
__global__ void copy_identity_kernel(int64_t nm, int nterms, const TermDev* __restrict__ terms,
                                     const double2* __restrict__ Q, double2* __restrict__ W) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= nm) return;
    const int d = blockIdx.y;                      // contour block
    double2 q = Q[d * nm + e];
    double2* Wd = W + (int64_t)d * nterms * nm;
    for (int t = 0; t < nterms; ++t)
        if (terms[t].aidx < 0) Wd[t * nm + e] = q;
}
}  // namespace

cudaError_t column_norms(cudaStream_t st, int64_t n, int m, const double2* X, int64_t ldx,
                         double* nrm) {
    note_launch();
    column_norms_kernel<<<m, 256, 0, st>>>(n, X, ldx, nrm);
    return cudaGetLastError();
}
cudaError_t ritz_scale(cudaStream_t st, int64_t n, int m, int nterms, const TermDev* terms,
                       const double2* lam, const double* nrm, double2* X, const double2* Y,
                       double2* Ycat) {
    int64_t nm = n * m;
    if (nm > 0) {
        note_launch();
        scale_columns_kernel<<<(unsigned)((nm + 255) / 256), 256, 0, st>>>(n, m, nrm, X);
    }
    int64_t tot = (int64_t)nterms * m * m;
    if (tot > 0) {
        note_launch();
        ycat_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(m, nterms, terms, lam, nrm, Y,
                                                                   Ycat);
    }
    return cudaGetLastError();
}
cudaError_t residual_summary(cudaStream_t st, int m, int nterms, const TermDev* terms,
                             const double2* lam, const double* rnorm, double c_re, double c_im,
                             double ra, double rb, double tol, double* relres,
                             IterStatus* status) {
    note_launch();
    residual_summary_kernel<<<1, 128, 0, st>>>(m, nterms, terms, lam, rnorm, c_re, c_im, ra, rb,
                                               tol, relres, status);
    return cudaGetLastError();
}
cudaError_t form_reduced(cudaStream_t st, int m, int nterms, int kmax, const TermDev* terms,
                         const double2* G, double2* Ahat) {
    int64_t tot = (int64_t)(kmax + 1) * m * m;
    note_launch();
    form_reduced_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(m, nterms, kmax, terms, G,
                                                                      Ahat);
    return cudaGetLastError();
}
cudaError_t offdiag_nonzero(cudaStream_t st, int64_t n, const double2* A, int64_t lda, int* flag) {
    note_launch();
    offdiag_nonzero_kernel<<<1216, 256, 0, st>>>(n, A, lda, flag);
    return cudaGetLastError();
}
cudaError_t extract_diagonal(cudaStream_t st, int64_t n, const double2* A, int64_t lda, double2* d) {
    note_launch();
    diagonal_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, A, lda, d);
    return cudaGetLastError();
}
cudaError_t diag_times(cudaStream_t st, int64_t n, int m, int nd, int nterms, int t, const double2* dg,
                       const double2* Q, double2* W) {
    const int64_t nm = n * m;
    note_launch();
    dim3 g((unsigned)((nm + 255) / 256), (unsigned)nd);
    diag_times_kernel<<<g, 256, 0, st>>>(n, nm, nterms, t, dg, Q, W);
    return cudaGetLastError();
}
cudaError_t copy_identity_terms(cudaStream_t st, int64_t n, int m, int nd, int nterms,
                                const TermDev* terms, const double2* Q, double2* W) {
    int64_t nm = n * m;
    note_launch();
    dim3 g((unsigned)((nm + 255) / 256), (unsigned)nd);
    copy_identity_kernel<<<g, 256, 0, st>>>(nm, nterms, terms, Q, W);
    return cudaGetLastError();
}

}  // namespace fnl

namespace fnl {
namespace {
template <typename T>
__global__ void to_double_kernel(int64_t cnt, const T* __restrict__ src, double2* __restrict__ dst) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < cnt) dst[e] = to_d2(src[e]);
}
__global__ void identity_kernel(int m, double2* __restrict__ Y, double* __restrict__ ones) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < m * m) Y[e] = make_double2((e % m) == (e / m) ? 1.0 : 0.0, 0.0);
    if (e < m) ones[e] = 1.0;
}
}  // namespace
template <typename T>
cudaError_t to_double(cudaStream_t st, int64_t cnt, const T* src, double2* dst) {
    note_launch();
    to_double_kernel<T><<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(cnt, src, dst);
    return cudaGetLastError();
}
template cudaError_t to_double<double2>(cudaStream_t, int64_t, const double2*, double2*);
template cudaError_t to_double<float2>(cudaStream_t, int64_t, const float2*, double2*);
cudaError_t set_identity(cudaStream_t st, int m, double2* Y, double* ones) {
    note_launch();
    identity_kernel<<<(m * m + 255) / 256, 256, 0, st>>>(m, Y, ones);
    return cudaGetLastError();
}
}  // namespace fnl
