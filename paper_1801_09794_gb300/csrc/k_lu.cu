// Batched blocked LU with partial pivoting of the node matrices T(z_j), and the
// multi-right-hand-side solves T(z_j)^{-1} R of Step 4 (Algorithm 1).
//
// Right-looking blocked LU, one panel of nb columns at a time, all nodes of the
// contour in one launch (grid dimension = node):
//   1. panel:  factor F[k0:n, k0:k0+jb] column by column; pivot = first row of
//              maximal |Re|+|Im| (LAPACK's cabs1); swap, scale, rank-1 update;
//   2. swap + trsm: apply the panel's interchanges to the columns right of the
//              panel, then U12 = L11^{-1} A12;
//   3. update: A22 -= L21 U12 (complex GEMM).
// Interchanges are never applied to the columns LEFT of a panel: every L block
// stays in the row order it had when it was formed, and the forward solve
// applies each panel's interchanges to the right-hand side just before that
// panel's elimination (the order Gaussian elimination itself uses), which is
// equivalent to P T = L U and saves the strided row traffic on L.
#include "internal.h"
#include <climits>

namespace fnl {
namespace {

constexpr int kTrsmCols = 64;   // right-hand-side columns per CTA in the triangular kernels

template <typename T>
__global__ void __launch_bounds__(1024) lu_panel_kernel(int64_t n, int k0, int jb, T* F,
                                                        int64_t ld, int64_t strideF, int* piv,
                                                        int* info) {
    typedef typename cplx_real<T>::type R;
    T* A = F + blockIdx.x * strideF;
    int* ip = piv + (int64_t)blockIdx.x * n;
    __shared__ R s_v[32];
    __shared__ int s_i[32];
    __shared__ int s_p;
    __shared__ T s_u[128];
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;
    const int nwarps = (nt + 31) >> 5;
    for (int c = k0; c < k0 + jb; ++c) {
        // --- pivot search in column c, rows c..n-1 (first index among equal maxima)
        R best = (R)-1;
        int bi = INT_MAX;
        for (int64_t r = c + tid; r < n; r += nt) {
            R v = cabs1(A[r + c * ld]);
            if (v > best) { best = v; bi = (int)r; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            R ov = __shfl_down_sync(0xffffffffu, best, o);
            int oi = __shfl_down_sync(0xffffffffu, bi, o);
            if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
        }
        if (lane == 0) { s_v[warp] = best; s_i[warp] = bi; }
        __syncthreads();
        if (warp == 0) {
            best = lane < nwarps ? s_v[lane] : (R)-1;
            bi = lane < nwarps ? s_i[lane] : INT_MAX;
            for (int o = 16; o > 0; o >>= 1) {
                R ov = __shfl_down_sync(0xffffffffu, best, o);
                int oi = __shfl_down_sync(0xffffffffu, bi, o);
                if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
            }
            if (lane == 0) {
                if (bi == INT_MAX || bi < c || bi >= n) bi = c;
                if (!(best > (R)0) && info[blockIdx.x] == 0) info[blockIdx.x] = c + 1;
                s_p = bi;
                ip[c] = bi;
            }
        }
        __syncthreads();
        const int p = s_p;
        // --- interchange rows c and p inside the panel
        if (p != c) {
            for (int cc = k0 + tid; cc < k0 + jb; cc += nt) {
                T a = A[c + cc * ld], b = A[p + cc * ld];
                A[c + cc * ld] = b;
                A[p + cc * ld] = a;
            }
        }
        __syncthreads();
        for (int cc = c + tid; cc < k0 + jb; cc += nt) s_u[cc - k0] = A[c + cc * ld];
        __syncthreads();
        // --- scale the column below the pivot and update the rest of the panel
        const T inv = crcp(s_u[c - k0]);
        for (int64_t r = c + 1 + tid; r < n; r += nt) {
            T l = A[r + c * ld] * inv;
            A[r + c * ld] = l;
            for (int cc = c + 1; cc < k0 + jb; ++cc)
                A[r + cc * ld] = cfms(l, s_u[cc - k0], A[r + cc * ld]);
        }
        __syncthreads();
    }
}

// Columns [col_begin, col_begin+ncols) of B: interchanges of rows k0..k0+jb-1,
// then B[k0:k0+jb, col] <- L11^{-1} B[k0:k0+jb, col] (L11 unit lower, from F).
template <typename T>
__global__ void __launch_bounds__(kTrsmCols) swap_trsm_lower_kernel(
    int64_t n, int k0, int jb, const T* __restrict__ F, int64_t ld, int64_t strideF,
    const int* __restrict__ piv, T* B, int64_t ldb, int64_t strideB, int col_begin, int ncols) {
    extern __shared__ unsigned char smem_raw[];
    T* sL = reinterpret_cast<T*>(smem_raw);          // jb x (jb+1), row-major sL[r*(jb+1)+c]
    T* sX = sL + jb * (jb + 1);                       // jb x kTrsmCols
    const int node = blockIdx.y;
    F += node * strideF;
    B += node * strideB;
    const int* ip = piv + (int64_t)node * n;
    const int tid = threadIdx.x;
    for (int e = tid; e < jb * jb; e += blockDim.x) {
        int r = e % jb, c = e / jb;
        sL[r * (jb + 1) + c] = F[(k0 + r) + (int64_t)(k0 + c) * ld];
    }
    const int cl = blockIdx.x * kTrsmCols + tid;
    const bool active = cl < ncols;
    T* col = B + (int64_t)(col_begin + (active ? cl : 0)) * ldb;
    if (active) {
        for (int c = k0; c < k0 + jb; ++c) {
            int p = ip[c];
            if (p != c) {
                T a = col[c], b = col[p];
                col[c] = b;
                col[p] = a;
            }
        }
        for (int i = 0; i < jb; ++i) sX[i * kTrsmCols + tid] = col[k0 + i];
    }
    __syncthreads();
    if (!active) return;
    for (int i = 0; i < jb; ++i) {
        T xi = sX[i * kTrsmCols + tid];
        for (int r = i + 1; r < jb; ++r)
            sX[r * kTrsmCols + tid] = cfms(sL[r * (jb + 1) + i], xi, sX[r * kTrsmCols + tid]);
    }
    for (int i = 0; i < jb; ++i) col[k0 + i] = sX[i * kTrsmCols + tid];
}

// B[k0:k0+jb, col] <- U11^{-1} B[k0:k0+jb, col] (U11 upper with its diagonal, from F).
template <typename T>
__global__ void __launch_bounds__(kTrsmCols) trsm_upper_kernel(
    int64_t n, int k0, int jb, const T* __restrict__ F, int64_t ld, int64_t strideF, T* B,
    int64_t ldb, int64_t strideB, int ncols) {
    extern __shared__ unsigned char smem_raw[];
    T* sU = reinterpret_cast<T*>(smem_raw);
    T* sX = sU + jb * (jb + 1);
    const int node = blockIdx.y;
    F += node * strideF;
    B += node * strideB;
    const int tid = threadIdx.x;
    for (int e = tid; e < jb * jb; e += blockDim.x) {
        int r = e % jb, c = e / jb;
        T v = F[(k0 + r) + (int64_t)(k0 + c) * ld];
        sU[r * (jb + 1) + c] = (r == c) ? crcp(v) : v;   // diagonal stored inverted
    }
    const int cl = blockIdx.x * kTrsmCols + tid;
    const bool active = cl < ncols;
    T* col = B + (int64_t)(active ? cl : 0) * ldb;
    if (active)
        for (int i = 0; i < jb; ++i) sX[i * kTrsmCols + tid] = col[k0 + i];
    __syncthreads();
    if (!active) return;
    for (int i = jb - 1; i >= 0; --i) {
        T xi = sX[i * kTrsmCols + tid] * sU[i * (jb + 1) + i];
        sX[i * kTrsmCols + tid] = xi;
        for (int r = 0; r < i; ++r)
            sX[r * kTrsmCols + tid] = cfms(sU[r * (jb + 1) + i], xi, sX[r * kTrsmCols + tid]);
    }
    for (int i = 0; i < jb; ++i) col[k0 + i] = sX[i * kTrsmCols + tid];
}

template <typename T>
size_t tri_smem(int jb) {
    return sizeof(T) * ((size_t)jb * (jb + 1) + (size_t)jb * kTrsmCols);
}

template <typename T>
cudaError_t ensure_attrs() {
    static bool done = false;   // per process; the attribute is per function
    if (done) return cudaSuccess;
    int nb = lu_block_size<T>();
    int bytes = (int)tri_smem<T>(nb);
    cudaError_t e = cudaFuncSetAttribute(swap_trsm_lower_kernel<T>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(trsm_upper_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             bytes);
    if (e != cudaSuccess) return e;
    done = true;
    return cudaSuccess;
}

}  // namespace

template <> int lu_block_size<double2>() { return 32; }
template <> int lu_block_size<float2>() { return 64; }

template <typename T>
cudaError_t lu_factor_batched(cudaStream_t st, int64_t n, int nb, T* F, int64_t strideF,
                              int* piv, int nc, int* info) {
    cudaError_t e = ensure_attrs<T>();
    if (e != cudaSuccess) return e;
    const T minus1 = cmake<T>(-1.0, 0.0), one = cmake<T>(1.0, 0.0);
    for (int64_t k0 = 0; k0 < n; k0 += nb) {
        int jb = (int)((n - k0) < nb ? (n - k0) : nb);
        note_launch();
        lu_panel_kernel<T><<<nc, 1024, 0, st>>>(n, (int)k0, jb, F, n, strideF, piv, info);
        int64_t rest = n - k0 - jb;
        if (rest > 0) {
            dim3 g((unsigned)((rest + kTrsmCols - 1) / kTrsmCols), nc);
            note_launch();
            swap_trsm_lower_kernel<T><<<g, kTrsmCols, tri_smem<T>(jb), st>>>(
                n, (int)k0, jb, F, n, strideF, piv, F, n, strideF, (int)(k0 + jb), (int)rest);
            e = gemm<T>(st, 0, (int)rest, (int)rest, jb, minus1, F + (k0 + jb) + k0 * n, n,
                        strideF, F + k0 + (k0 + jb) * n, n, strideF, one,
                        F + (k0 + jb) + (k0 + jb) * n, n, strideF, nc);
            if (e != cudaSuccess) return e;
        }
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t lu_solve_batched(cudaStream_t st, int64_t n, int nb, const T* F, int64_t strideF,
                             const int* piv, int nc, T* Y, int64_t strideY, int m) {
    cudaError_t e = ensure_attrs<T>();
    if (e != cudaSuccess) return e;
    const T minus1 = cmake<T>(-1.0, 0.0), one = cmake<T>(1.0, 0.0);
    dim3 g((unsigned)((m + kTrsmCols - 1) / kTrsmCols), nc);
    for (int64_t k0 = 0; k0 < n; k0 += nb) {
        int jb = (int)((n - k0) < nb ? (n - k0) : nb);
        note_launch();
        swap_trsm_lower_kernel<T><<<g, kTrsmCols, tri_smem<T>(jb), st>>>(
            n, (int)k0, jb, F, n, strideF, piv, Y, n, strideY, 0, m);
        int64_t rest = n - k0 - jb;
        if (rest > 0) {
            e = gemm<T>(st, 0, (int)rest, m, jb, minus1, F + (k0 + jb) + k0 * n, n, strideF,
                        Y + k0, n, strideY, one, Y + k0 + jb, n, strideY, nc);
            if (e != cudaSuccess) return e;
        }
    }
    int64_t last = ((n - 1) / nb) * nb;
    for (int64_t k0 = last; k0 >= 0; k0 -= nb) {
        int jb = (int)((n - k0) < nb ? (n - k0) : nb);
        note_launch();
        trsm_upper_kernel<T><<<g, kTrsmCols, tri_smem<T>(jb), st>>>(n, (int)k0, jb, F, n, strideF,
                                                                    Y, n, strideY, m);
        if (k0 > 0) {
            e = gemm<T>(st, 0, (int)k0, m, jb, minus1, F + k0 * n, n, strideF, Y + k0, n, strideY,
                        one, Y, n, strideY, nc);
            if (e != cudaSuccess) return e;
        }
    }
    return cudaGetLastError();
}

template cudaError_t lu_factor_batched<double2>(cudaStream_t, int64_t, int, double2*, int64_t,
                                                int*, int, int*);
template cudaError_t lu_factor_batched<float2>(cudaStream_t, int64_t, int, float2*, int64_t, int*,
                                               int, int*);
template cudaError_t lu_solve_batched<double2>(cudaStream_t, int64_t, int, const double2*,
                                               int64_t, const int*, int, double2*, int64_t, int);
template cudaError_t lu_solve_batched<float2>(cudaStream_t, int64_t, int, const float2*, int64_t,
                                              const int*, int, float2*, int64_t, int);

}  // namespace fnl
