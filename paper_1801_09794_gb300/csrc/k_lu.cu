// Batched blocked LU with partial pivoting of the node matrices T(z_j), and the
// multi-right-hand-side solves T(z_j)^{-1} R of Step 4 (Algorithm 1).
//
// Right-looking blocked LU, one panel of nb columns at a time, all nodes of the
// contour in one launch (grid dimension = node):
//   1. panel:  factor F[k0:n, k0:k0+jb]; pivot = first row of maximal |Re|+|Im|
//              (LAPACK's cabs1).  The panel is processed in mini-panels of 4
//              columns held in registers (each of the 1024 threads owns up to 4
//              rows), so the in-panel rank-1 updates never touch memory; after a
//              mini-panel its interchanges, triangular solve and rank-4 update are
//              applied to the rest of the panel in one pass.  The panel's
//              interchanges are also emitted as a gather list (dst <- src rows).
//   2. swap + trsm: the gather list applied to the columns right of the panel,
//              then U12 = L11^{-1} A12 (one warp per column);
//   3. update: A22 -= L21 U12 (complex64: TF32 tensor cores on split operands,
//              FP32-accurate; complex128: FP64 SIMT GEMM).
//   4. pair swap: for an odd panel k, its gather list applied to the L columns
//              of panel k - 1 as well, on a third, low-priority stream (nothing
//              on the critical path reads them), so that panels k - 1 and k form
//              one block of 2 nb columns whose L carries the row order after
//              both panels' interchanges -- the factors of a blocked LU with
//              block size 2 nb.
// Interchanges are otherwise not applied to the columns left of a block: the
// forward solve applies each block's two gather lists to the right-hand side
// just before that block's substitution (the order Gaussian elimination itself
// uses), equivalent to P T = L U without the strided row traffic on all of L.
// The solves step through blocks of 2 nb rows (128 for complex64, 64 for
// complex128): half the dependent steps of per-panel substitution and twice
// the depth of each tensor-core update.
#include "internal.h"
#include "tc_common.cuh"
#include "cgemm_tile.cuh"

#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <tuple>
#include <utility>
#include <vector>
#include <climits>
#include <cstdlib>

#include <cooperative_groups.h>

namespace fnl {
namespace {

constexpr int kPanelThreads = 1024;
constexpr int kMini = 4;           // columns per register-resident mini-panel
// diagonal-block tile of the triangular kernels (jb <= nb: 64 complex64 / 32 complex128)
template <typename T> struct TriMax;
template <> struct TriMax<float2> { static constexpr int value = 64; };
template <> struct TriMax<double2> { static constexpr int value = 32; };
constexpr int kWarpsPerCta = 8;    // triangular kernels: one warp per column


// ---------------------------------------------------------------------------
// block-wide argmax of (value, row): larger value wins, lower row on ties
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ void argmax_warp(R& v, int& i) {
    for (int o = 16; o > 0; o >>= 1) {
        R ov = __shfl_down_sync(0xffffffffu, v, o);
        int oi = __shfl_down_sync(0xffffffffu, i, o);
        if (ov > v || (ov == v && oi < i)) { v = ov; i = oi; }
    }
}

// Gather list of a panel's interchanges: the sequential swaps (c, piv[c]),
// c = k0..k0+jb-1, permute the rows of the set {k0..k0+jb-1} U {piv[c]}; after
// them row dst[e] holds what row src[e] held before.  One thread, <= 2 jb <= MAXR
// rows; ip[c] is the pivot row of column k0 + c.
template <int MAXR>
__device__ void gather_list(int k0, int jb, const int* ip, int2* list, int* count) {
    int rows[MAXR], src[MAXR];
    int cnt = 0;
    for (int c = 0; c < jb; ++c) { rows[cnt] = k0 + c; src[cnt] = k0 + c; ++cnt; }
    for (int c = 0; c < jb; ++c) {
        const int a = k0 + c, b = ip[c];
        if (a == b) continue;
        int ia = a - k0, ib = -1;
        if (b < k0 + jb) ib = b - k0;
        else {
            for (int e = jb; e < cnt; ++e)
                if (rows[e] == b) { ib = e; break; }
            if (ib < 0) { rows[cnt] = b; src[cnt] = b; ib = cnt++; }
        }
        int t = src[ia]; src[ia] = src[ib]; src[ib] = t;
    }
    int out = 0;
    for (int e = 0; e < cnt; ++e)
        if (rows[e] != src[e]) list[out++] = make_int2(rows[e], src[e]);
    *count = out;
}

// ---------------------------------------------------------------------------
// Panel factorisation, register-resident mini-panels.  ROWS = rows per thread.
// ---------------------------------------------------------------------------
// One node's panel: A (n x n, leading dimension ld), its pivot array ip, its
// info word, and this panel's gather-list slot (gl, gc; gl may be null).
template <typename T, int ROWS>
__device__ __forceinline__ void panel_reg_body(int64_t n, int k0, int jb, T* A, int64_t ld,
                                               int* ip, int* info1, int2* gl, int* gc) {
    typedef typename cplx_real<T>::type R;
    __shared__ R s_v[32];
    __shared__ int s_i[32];
    __shared__ int s_p;
    __shared__ T s_prow[kMini];     // pivot row of the mini-panel
    __shared__ T s_crow[kMini];     // row being replaced by the pivot row
    __shared__ T s_L11[kMini][kMini];
    __shared__ T s_U[kMini][64];    // U12 rows of the mini-panel (rest of the panel)
    __shared__ int s_piv[kMini];    // the mini-panel's pivot rows
    __shared__ int2 s_gl[2 * kMini];
    __shared__ int s_gc;
    static_assert(kPanelThreads / 16 >= 64, "a 16-thread group per panel column");
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int pend = k0 + jb;
    // panel columns per batch in the in-panel update: ROWS x kUpd loads in
    // flight per thread, as many as the registers left next to the mini-panel
    // allow at 1024 threads
    constexpr int kUpd = (sizeof(T) == 8) ? 8 / ROWS : (ROWS == 1 ? 4 : 2);
    T v[ROWS][kMini];

    for (int mb0 = k0; mb0 < pend; mb0 += kMini) {
        const int w = min(kMini, pend - mb0);
        // load the mini-panel rows owned by this thread: row k0 + tid + i * 1024
#pragma unroll
        for (int i = 0; i < ROWS; ++i) {
            const int64_t r = k0 + tid + (int64_t)i * kPanelThreads;
#pragma unroll
            for (int c = 0; c < kMini; ++c)
                v[i][c] = (r < n && c < w) ? A[r + (int64_t)(mb0 + c) * ld] : cmake<T>(0.0, 0.0);
        }
        for (int c = 0; c < w; ++c) {
            const int col = mb0 + c;
            // pivot search among rows >= col
            R best = (R)-1;
            int bi = INT_MAX;
#pragma unroll
            for (int i = 0; i < ROWS; ++i) {
                const int64_t r = k0 + tid + (int64_t)i * kPanelThreads;
                T x = v[i][0];
#pragma unroll
                for (int cc = 1; cc < kMini; ++cc) if (cc == c) x = v[i][cc];
                if (r >= col && r < n) {
                    R a = cabs1(x);
                    if (a > best) { best = a; bi = (int)r; }
                }
            }
            argmax_warp(best, bi);
            if (lane == 0) { s_v[warp] = best; s_i[warp] = bi; }
            __syncthreads();
            if (warp == 0) {
                best = s_v[lane];
                bi = s_i[lane];
                argmax_warp(best, bi);
                if (lane == 0) {
                    if (bi == INT_MAX || bi < col || bi >= n) bi = col;
                    if (!(best > (R)0) && *info1 == 0) *info1 = col + 1;
                    s_p = bi;
                    s_piv[c] = bi;
                    ip[col] = bi;
                }
            }
            __syncthreads();
            const int p = s_p;
            const int owner_p = (p - k0) % kPanelThreads, slot_p = (p - k0) / kPanelThreads;
            const int owner_c = (col - k0) % kPanelThreads, slot_c = (col - k0) / kPanelThreads;
            if (tid == owner_p) {
#pragma unroll
                for (int i = 0; i < ROWS; ++i)
                    if (i == slot_p)
#pragma unroll
                        for (int cc = 0; cc < kMini; ++cc) s_prow[cc] = v[i][cc];
            }
            if (tid == owner_c && p != col) {
#pragma unroll
                for (int i = 0; i < ROWS; ++i)
                    if (i == slot_c)
#pragma unroll
                        for (int cc = 0; cc < kMini; ++cc) s_crow[cc] = v[i][cc];
            }
            __syncthreads();
            if (p != col) {
                if (tid == owner_c) {
#pragma unroll
                    for (int i = 0; i < ROWS; ++i)
                        if (i == slot_c)
#pragma unroll
                            for (int cc = 0; cc < kMini; ++cc) v[i][cc] = s_prow[cc];
                }
                if (tid == owner_p) {
#pragma unroll
                    for (int i = 0; i < ROWS; ++i)
                        if (i == slot_p)
#pragma unroll
                            for (int cc = 0; cc < kMini; ++cc) v[i][cc] = s_crow[cc];
                }
            }
            // scale and rank-1 update inside the mini-panel (rows > col)
            T piv_v = s_prow[0];
#pragma unroll
            for (int cc = 1; cc < kMini; ++cc) if (cc == c) piv_v = s_prow[cc];
            const T inv = crcp(piv_v);
#pragma unroll
            for (int i = 0; i < ROWS; ++i) {
                const int64_t r = k0 + tid + (int64_t)i * kPanelThreads;
                if (r > col && r < n) {
                    T l = cmake<T>(0.0, 0.0);
#pragma unroll
                    for (int cc = 0; cc < kMini; ++cc) if (cc == c) { l = v[i][cc] * inv; v[i][cc] = l; }
#pragma unroll
                    for (int cc = 0; cc < kMini; ++cc)
                        if (cc > c && cc < w) v[i][cc] = cfms(l, s_prow[cc], v[i][cc]);
                }
            }
            __syncthreads();   // s_prow / s_crow reuse
        }
        // write the factored mini-panel back; keep its L11 block in smem
#pragma unroll
        for (int i = 0; i < ROWS; ++i) {
            const int64_t r = k0 + tid + (int64_t)i * kPanelThreads;
            if (r < n)
#pragma unroll
                for (int c = 0; c < kMini; ++c)
                    if (c < w) A[r + (int64_t)(mb0 + c) * ld] = v[i][c];
            if (r >= mb0 && r < mb0 + w)
#pragma unroll
                for (int c = 0; c < kMini; ++c) s_L11[r - mb0][c] = v[i][c];
        }
        const int rest0 = mb0 + w, nrest = pend - rest0;   // remaining panel columns
        if (tid == 0) gather_list<2 * kMini>(mb0, w, s_piv, s_gl, &s_gc);
        __syncthreads();
        const int gcnt = s_gc;
        // this mini-panel's interchanges on the other panel columns -- factored
        // ones, so that the whole panel ends in the row order of all its
        // interchanges, and remaining ones, whose mini-panel rows (the U12 rows
        // to solve for) go to s_U.  Thread (column jj = tid / 16, slot e =
        // tid % 16): slots 0..7 read a gather source, slots 8..11 a mini-panel
        // row; every read lands before any write (one round trip per column).
        {
            const int jj = tid >> 4, e = tid & 15;
            const int cidx = k0 + jj;
            const bool left = cidx < mb0, rest = cidx >= rest0 && cidx < pend;
            T* colp = A + (int64_t)cidx * ld;
            T val = cmake<T>(0.0, 0.0);
            int dst = -1;
            if ((left || rest) && e < gcnt) { val = colp[s_gl[e].y]; dst = s_gl[e].x; }
            if (rest && e >= 2 * kMini && e - 2 * kMini < w)
                s_U[e - 2 * kMini][cidx - rest0] = colp[mb0 + e - 2 * kMini];
            __syncthreads();
            if (dst >= 0) {
                if (rest && dst < mb0 + w) s_U[dst - mb0][cidx - rest0] = val;
                else colp[dst] = val;
            }
            __syncthreads();
        }
        if (nrest > 0) {
            // U12 = L11^{-1} A12 on the remaining panel columns, one thread each
            if (tid < nrest) {
                T* colp = A + (int64_t)(rest0 + tid) * ld;
                T u[kMini];
#pragma unroll
                for (int c = 0; c < kMini; ++c) u[c] = (c < w) ? s_U[c][tid] : cmake<T>(0.0, 0.0);
#pragma unroll
                for (int c = 0; c < kMini; ++c)
#pragma unroll
                    for (int r2 = c + 1; r2 < kMini; ++r2)
                        if (r2 < w) u[r2] = cfms(s_L11[r2][c], u[c], u[r2]);
#pragma unroll
                for (int c = 0; c < kMini; ++c) {
                    if (c < w) colp[mb0 + c] = u[c];
                    s_U[c][tid] = u[c];
                }
            }
            __syncthreads();
            // rank-w update of rows below the mini-panel, remaining panel columns;
            // per batch of kUpd columns every owned row's loads are issued first
            for (int j0 = 0; j0 < nrest; j0 += kUpd) {
                T a[ROWS][kUpd];
#pragma unroll
                for (int i = 0; i < ROWS; ++i) {
                    const int64_t r = k0 + tid + (int64_t)i * kPanelThreads;
                    const T* ar = A + r + (int64_t)(rest0 + j0) * ld;
#pragma unroll
                    for (int q = 0; q < kUpd; ++q)
                        a[i][q] = (r >= rest0 && r < n && j0 + q < nrest) ? ar[(int64_t)q * ld]
                                                                           : cmake<T>(0.0, 0.0);
                }
#pragma unroll
                for (int i = 0; i < ROWS; ++i) {
                    const int64_t r = k0 + tid + (int64_t)i * kPanelThreads;
                    if (r >= rest0 && r < n) {
                        T* ar = A + r + (int64_t)(rest0 + j0) * ld;
#pragma unroll
                        for (int q = 0; q < kUpd; ++q) {
                            if (j0 + q < nrest) {
#pragma unroll
                                for (int c = 0; c < kMini; ++c)
                                    if (c < w) a[i][q] = cfms(v[i][c], s_U[c][j0 + q], a[i][q]);
                                ar[(int64_t)q * ld] = a[i][q];
                            }
                        }
                    }
                }
            }
            __syncthreads();
        }
    }
    if (tid == 0 && gl != nullptr) gather_list<128>(k0, jb, ip + k0, gl, gc);
}

template <typename T, int ROWS>
__global__ void __launch_bounds__(kPanelThreads) lu_panel_reg_kernel(
    int64_t n, int k0, int jb, T* F, int64_t ld, int64_t strideF, int* piv, int* info,
    int2* gather, int* gcount, int panel_index, int gstride) {
    panel_reg_body<T, ROWS>(n, k0, jb, F + blockIdx.x * strideF, ld, piv + (int64_t)blockIdx.x * n,
                            info + blockIdx.x,
                            gather ? gather + (int64_t)blockIdx.x * gstride + panel_index * 2 * 64 : nullptr,
                            gcount + (int64_t)blockIdx.x * (gstride / 128) + panel_index);
}

// Nodes of different orders in one launch: node blockIdx.x from its
// descriptor; nodes whose order ends before this panel do nothing.
// Each node runs the rows-per-thread variant it would get in a factorisation
// of its own (chosen per CTA from its remaining rows, so nodes of every class
// share the launch).
template <typename T>
__global__ void __launch_bounds__(kPanelThreads) lu_panel_reg_grouped_kernel(
    const LuNode* __restrict__ nodes, int k0, int nb, int panel_index) {
    const LuNode d = nodes[blockIdx.x];
    if (k0 >= d.n) return;
    const int64_t rows = d.n - k0;
    const int jb = (int)min((int64_t)nb, d.n - k0);
    T* F = static_cast<T*>(d.F);
    if (rows <= kPanelThreads)
        panel_reg_body<T, 1>(d.n, k0, jb, F, d.n, d.piv, d.info, d.gather + panel_index * 2 * 64,
                             d.gcount + panel_index);
    else if (rows <= 2 * kPanelThreads)
        panel_reg_body<T, 2>(d.n, k0, jb, F, d.n, d.piv, d.info, d.gather + panel_index * 2 * 64,
                             d.gcount + panel_index);
    else
        panel_reg_body<T, 4>(d.n, k0, jb, F, d.n, d.piv, d.info, d.gather + panel_index * 2 * 64,
                             d.gcount + panel_index);
}

// ---------------------------------------------------------------------------
// Panel factorisation spread over a thread-block cluster (complex64).
// ---------------------------------------------------------------------------
// The CL CTAs of one cluster share one node's panel: thread g = rank * NT + tid
// of the cluster owns rows k0 + g + i * CL * NT (i < ROWS), so every row has
// one owner thread and one owner CTA.  Per column, each CTA reduces its own
// rows to one pivot candidate and stores it -- value, row and the row's four
// mini-panel entries -- into a slot of every CTA's shared memory
// (distributed shared memory), the owner of the diagonal row stores that row
// too, and one cluster barrier later every CTA picks the same pivot and holds
// both rows it needs for the interchange and the rank-1 update.  The slots
// alternate between two buffers by column parity, so a CTA that runs ahead
// into the next column cannot overwrite a slot another CTA is still reading
// (it has to pass that CTA at the barrier first).  The pivot row as chosen at
// column c is the final row c of the mini-panel (later steps only touch rows
// below it), so the L11 block needs no exchange of its own.
// A mini-panel's interchanges on the other panel columns take one more
// cluster barrier (every read before any write, as in the one-CTA panel);
// each moved row is written by its owner CTA, so every later access to a row
// in global memory is made by the CTA that wrote it or after a barrier.
// Per element the operations and their order are those of the one-CTA panel
// (same pivot rule: first row of maximal cabs1; same scaling and rank-1 and
// rank-w updates), so the factors are the same bits whatever CL and ROWS are.
namespace cg = cooperative_groups;
constexpr int kClusterMax = 8;       // portable cluster size
constexpr int kClusterThreads = 512;
// mini-panel width of the cluster panels: 8 columns halve the passes over the
// rest of the panel (the per-element operations and their order are those of
// 4-column mini-panels, so the factors are unchanged)
constexpr int kClusterMini = 8;

template <typename T, int MINI>
struct PanelCand {
    typename cplx_real<T>::type v;   // cabs1 of the candidate (-1: none)
    int i;                           // its row (INT_MAX: none)
    T row[MINI];                     // its mini-panel entries
};

template <typename T, int ROWS, int MINI = kMini>
__device__ __forceinline__ void panel_cluster_body(int64_t n, int k0, int jb, T* A, int64_t ld,
                                                   int* ip, int* info1, int2* gl, int* gc) {
    typedef typename cplx_real<T>::type R;
    constexpr int NT = kClusterThreads, NW = NT / 32;
    cg::cluster_group cl = cg::this_cluster();
    const int CL = (int)cl.num_blocks();
    const int rank = (int)cl.block_rank();
    const int G = CL * NT;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = rank * NT + tid;
    __shared__ PanelCand<T, MINI> s_cand[2][kClusterMax];
    __shared__ T s_crow[2][MINI];
    __shared__ PanelCand<T, MINI> s_wc[NW];
    __shared__ T s_L11[MINI][MINI];
    __shared__ T s_U[MINI][64];
    __shared__ T s_gval[2 * MINI][64];
    __shared__ int s_piv[MINI];
    __shared__ int2 s_gl[2 * MINI];
    __shared__ int s_gc;
    const int pend = k0 + jb;
    constexpr int kUpd = ROWS == 1 ? 8 : 4;
    T v[ROWS][MINI];

    for (int mb0 = k0; mb0 < pend; mb0 += MINI) {
        const int w = min(MINI, pend - mb0);
#pragma unroll
        for (int i = 0; i < ROWS; ++i) {
            const int64_t r = k0 + g + (int64_t)i * G;
#pragma unroll
            for (int c = 0; c < MINI; ++c)
                v[i][c] = (r < n && c < w) ? A[r + (int64_t)(mb0 + c) * ld] : cmake<T>(0.0, 0.0);
        }
        for (int c = 0; c < w; ++c) {
            const int col = mb0 + c, par = col & 1;
            // this thread's candidate among its rows >= col
            R best = (R)-1;
            int bi = INT_MAX, bslot = 0;
#pragma unroll
            for (int i = 0; i < ROWS; ++i) {
                const int64_t r = k0 + g + (int64_t)i * G;
                T x = v[i][0];
#pragma unroll
                for (int cc = 1; cc < MINI; ++cc) if (cc == c) x = v[i][cc];
                if (r >= col && r < n) {
                    R a = cabs1(x);
                    if (a > best) { best = a; bi = (int)r; bslot = i; }
                }
            }
            R wb = best;
            int wi = bi;
            argmax_warp(wb, wi);
            wi = __shfl_sync(0xffffffffu, wi, 0);
            wb = __shfl_sync(0xffffffffu, wb, 0);
            if (wi != INT_MAX && bi == wi) {          // this lane holds the warp's candidate row
                PanelCand<T, MINI>& e = s_wc[warp];
                e.v = wb;
                e.i = wi;
#pragma unroll
                for (int i = 0; i < ROWS; ++i)
                    if (i == bslot)
#pragma unroll
                        for (int cc = 0; cc < MINI; ++cc) e.row[cc] = v[i][cc];
            }
            if (lane == 0 && wi == INT_MAX) { s_wc[warp].v = (R)-1; s_wc[warp].i = INT_MAX; }
            // the diagonal row, for the interchange
#pragma unroll
            for (int i = 0; i < ROWS; ++i) {
                if (k0 + g + (int64_t)i * G == col) {
                    for (int d = 0; d < CL; ++d) {
                        T* dst = cl.map_shared_rank(&s_crow[par][0], d);
#pragma unroll
                        for (int cc = 0; cc < MINI; ++cc) dst[cc] = v[i][cc];
                    }
                }
            }
            __syncthreads();
            if (warp == 0) {
                const R cv = lane < NW ? s_wc[lane].v : (R)-1;
                const int ci = lane < NW ? s_wc[lane].i : INT_MAX;
                R rv = cv;
                int ri = ci;
                argmax_warp(rv, ri);
                ri = __shfl_sync(0xffffffffu, ri, 0);
                const unsigned m = __ballot_sync(0xffffffffu, lane < NW && ci == ri);
                const int src = m ? __ffs(m) - 1 : 0;
                if (lane < CL) {
                    PanelCand<T, MINI>* dst = cl.map_shared_rank(&s_cand[par][rank], lane);
                    *dst = s_wc[src];
                }
            }
            cl.sync();
            // every thread combines the CL candidates the same way
            R pb = (R)-1;
            int p = INT_MAX, wd = -1;
            for (int d = 0; d < CL; ++d) {
                const R vd = s_cand[par][d].v;
                const int id = s_cand[par][d].i;
                if (vd > pb || (vd == pb && id < p)) { pb = vd; p = id; wd = d; }
            }
            const bool found = !(p == INT_MAX || p < col || p >= n);
            if (!found) p = col;
            T prow[MINI];
#pragma unroll
            for (int cc = 0; cc < MINI; ++cc)
                prow[cc] = found ? s_cand[par][wd].row[cc] : s_crow[par][cc];
            if (tid == 0) {
                s_piv[c] = p;
#pragma unroll
                for (int cc = 0; cc < MINI; ++cc) s_L11[c][cc] = prow[cc];
                if (rank == 0) {
                    if (!(pb > (R)0) && *info1 == 0) *info1 = col + 1;
                    ip[col] = p;
                }
            }
            if (p != col) {
#pragma unroll
                for (int i = 0; i < ROWS; ++i) {
                    const int64_t r = k0 + g + (int64_t)i * G;
                    if (r == col) {
#pragma unroll
                        for (int cc = 0; cc < MINI; ++cc) v[i][cc] = prow[cc];
                    } else if (r == p) {
#pragma unroll
                        for (int cc = 0; cc < MINI; ++cc) v[i][cc] = s_crow[par][cc];
                    }
                }
            }
            T piv_v = prow[0];
#pragma unroll
            for (int cc = 1; cc < MINI; ++cc) if (cc == c) piv_v = prow[cc];
            const T inv = crcp(piv_v);
#pragma unroll
            for (int i = 0; i < ROWS; ++i) {
                const int64_t r = k0 + g + (int64_t)i * G;
                if (r > col && r < n) {
                    T l = cmake<T>(0.0, 0.0);
#pragma unroll
                    for (int cc = 0; cc < MINI; ++cc) if (cc == c) { l = v[i][cc] * inv; v[i][cc] = l; }
#pragma unroll
                    for (int cc = 0; cc < MINI; ++cc)
                        if (cc > c && cc < w) v[i][cc] = cfms(l, prow[cc], v[i][cc]);
                }
            }
        }
        // the factored mini-panel back to memory (own rows)
#pragma unroll
        for (int i = 0; i < ROWS; ++i) {
            const int64_t r = k0 + g + (int64_t)i * G;
            if (r < n)
#pragma unroll
                for (int c = 0; c < MINI; ++c)
                    if (c < w) A[r + (int64_t)(mb0 + c) * ld] = v[i][c];
        }
        const int rest0 = mb0 + w, nrest = pend - rest0;
        if (tid == 0) gather_list<2 * MINI>(mb0, w, s_piv, s_gl, &s_gc);
        __syncthreads();
        const int gcnt = s_gc;
        // reads: (a) the mini-panel rows of the remaining columns after the
        // interchanges (every CTA, for its own copy of U12); (b) the moved
        // entries of the other panel columns whose destination row this CTA owns
        for (int it = tid; it < w * nrest; it += NT) {
            const int j = it / nrest, cr = it - j * nrest;
            int src = mb0 + j;
            for (int e = 0; e < gcnt; ++e)
                if (s_gl[e].x == mb0 + j) src = s_gl[e].y;
            s_U[j][cr] = __ldcg(A + src + (int64_t)(rest0 + cr) * ld);
        }
        for (int it = tid; it < gcnt * jb; it += NT) {
            const int e = it / jb, cj = it - e * jb, cidx = k0 + cj;
            const int dst = s_gl[e].x;
            const bool left = cidx < mb0, rest = cidx >= rest0;
            if ((left || (rest && dst >= mb0 + w)) &&
                (int)(((int64_t)(dst - k0) % G) / NT) == rank)
                s_gval[e][cj] = __ldcg(A + s_gl[e].y + (int64_t)cidx * ld);
        }
        cl.sync();                                  // every read before any write
        for (int it = tid; it < gcnt * jb; it += NT) {
            const int e = it / jb, cj = it - e * jb, cidx = k0 + cj;
            const int dst = s_gl[e].x;
            const bool left = cidx < mb0, rest = cidx >= rest0;
            if ((left || (rest && dst >= mb0 + w)) &&
                (int)(((int64_t)(dst - k0) % G) / NT) == rank)
                A[dst + (int64_t)cidx * ld] = s_gval[e][cj];
        }
        __syncthreads();
        if (nrest > 0) {
            // U12 = L11^{-1} A12 on the remaining panel columns (every CTA)
            if (tid < nrest) {
                T u[MINI];
#pragma unroll
                for (int c = 0; c < MINI; ++c) u[c] = (c < w) ? s_U[c][tid] : cmake<T>(0.0, 0.0);
#pragma unroll
                for (int c = 0; c < MINI; ++c)
#pragma unroll
                    for (int r2 = c + 1; r2 < MINI; ++r2)
                        if (r2 < w) u[r2] = cfms(s_L11[r2][c], u[c], u[r2]);
#pragma unroll
                for (int c = 0; c < MINI; ++c) s_U[c][tid] = u[c];
            }
            __syncthreads();
            // the U12 rows go to memory from the CTA that owns them
            for (int it = tid; it < w * nrest; it += NT) {
                const int j = it / nrest, cr = it - j * nrest;
                if ((int)(((int64_t)(mb0 + j - k0) % G) / NT) == rank)
                    A[mb0 + j + (int64_t)(rest0 + cr) * ld] = s_U[j][cr];
            }
            // rank-w update of the own rows below the mini-panel
            for (int j0 = 0; j0 < nrest; j0 += kUpd) {
                T a[ROWS][kUpd];
#pragma unroll
                for (int i = 0; i < ROWS; ++i) {
                    const int64_t r = k0 + g + (int64_t)i * G;
                    const T* ar = A + r + (int64_t)(rest0 + j0) * ld;
#pragma unroll
                    for (int q = 0; q < kUpd; ++q)
                        a[i][q] = (r >= rest0 && r < n && j0 + q < nrest) ? ar[(int64_t)q * ld]
                                                                           : cmake<T>(0.0, 0.0);
                }
#pragma unroll
                for (int i = 0; i < ROWS; ++i) {
                    const int64_t r = k0 + g + (int64_t)i * G;
                    if (r >= rest0 && r < n) {
                        T* ar = A + r + (int64_t)(rest0 + j0) * ld;
#pragma unroll
                        for (int q = 0; q < kUpd; ++q) {
                            if (j0 + q < nrest) {
#pragma unroll
                                for (int c = 0; c < MINI; ++c)
                                    if (c < w) a[i][q] = cfms(v[i][c], s_U[c][j0 + q], a[i][q]);
                                ar[(int64_t)q * ld] = a[i][q];
                            }
                        }
                    }
                }
            }
        }
        __syncthreads();
    }
    if (rank == 0 && tid == 0 && gl != nullptr) gather_list<128>(k0, jb, ip + k0, gl, gc);
}

template <int ROWS>
__global__ void __launch_bounds__(kClusterThreads, 1) lu_panel_cluster_kernel(
    int64_t n, int k0, int jb, float2* F, int64_t ld, int64_t strideF, int* piv, int* info,
    int2* gather, int* gcount, int panel_index, int gstride) {
    const int node = blockIdx.y;
    panel_cluster_body<float2, ROWS, kClusterMini>(
        n, k0, jb, F + node * strideF, ld, piv + (int64_t)node * n, info + node,
        gather ? gather + (int64_t)node * gstride + panel_index * 2 * 64 : nullptr,
        gcount + (int64_t)node * (gstride / 128) + panel_index);
}

// Nodes of different orders: cluster blockIdx.y is node blockIdx.y; a node
// whose order ends before this panel returns (the whole cluster at once).
template <int ROWS>
__global__ void __launch_bounds__(kClusterThreads, 1) lu_panel_cluster_grouped_kernel(
    const LuNode* __restrict__ nodes, int k0, int nb, int panel_index) {
    const LuNode d = nodes[blockIdx.y];
    if (k0 >= d.n) return;
    const int jb = (int)min((int64_t)nb, d.n - k0);
    panel_cluster_body<float2, ROWS, kClusterMini>(d.n, k0, jb, static_cast<float2*>(d.F), d.n, d.piv, d.info,
                                     d.gather + panel_index * 2 * 64, d.gcount + panel_index);
}

// Column-at-a-time panel in global memory (any n; used above 8192 rows).
template <typename T>
__global__ void __launch_bounds__(kPanelThreads) lu_panel_kernel(
    int64_t n, int k0, int jb, T* F, int64_t ld, int64_t strideF, int* piv, int* info,
    int2* gather, int* gcount, int panel_index, int gstride) {
    typedef typename cplx_real<T>::type R;
    T* A = F + blockIdx.x * strideF;
    int* ip = piv + (int64_t)blockIdx.x * n;
    __shared__ R s_v[32];
    __shared__ int s_i[32];
    __shared__ int s_p;
    __shared__ T s_u[128];
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;
    for (int c = k0; c < k0 + jb; ++c) {
        R best = (R)-1;
        int bi = INT_MAX;
        for (int64_t r = c + tid; r < n; r += nt) {
            R v = cabs1(A[r + c * ld]);
            if (v > best) { best = v; bi = (int)r; }
        }
        argmax_warp(best, bi);
        if (lane == 0) { s_v[warp] = best; s_i[warp] = bi; }
        __syncthreads();
        if (warp == 0) {
            best = s_v[lane];
            bi = s_i[lane];
            argmax_warp(best, bi);
            if (lane == 0) {
                if (bi == INT_MAX || bi < c || bi >= n) bi = c;
                if (!(best > (R)0) && info[blockIdx.x] == 0) info[blockIdx.x] = c + 1;
                s_p = bi;
                ip[c] = bi;
            }
        }
        __syncthreads();
        const int p = s_p;
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
        const T inv = crcp(s_u[c - k0]);
        for (int64_t r = c + 1 + tid; r < n; r += nt) {
            T l = A[r + c * ld] * inv;
            A[r + c * ld] = l;
            for (int cc = c + 1; cc < k0 + jb; ++cc)
                A[r + cc * ld] = cfms(l, s_u[cc - k0], A[r + cc * ld]);
        }
        __syncthreads();
    }
    if (tid == 0 && gather != nullptr)
        gather_list<128>(k0, jb, ip + k0, gather + (int64_t)blockIdx.x * gstride + panel_index * 2 * 64,
                         gcount + (int64_t)blockIdx.x * (gstride / 128) + panel_index);
}

// ---------------------------------------------------------------------------
// Triangular kernels, one warp per right-hand-side column; the jb rows of the
// diagonal block are spread over the lanes (lane l holds rows l and l + 32).
// ---------------------------------------------------------------------------
// One element global -> shared without a register round trip (cp.async; the
// copies of a whole triangle are in flight together).
__device__ __forceinline__ void cp_async_elem(float2* dst, const float2* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(tc::smem_u32(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_elem(double2* dst, const double2* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(tc::smem_u32(dst)), "l"(src)
                 : "memory");
}
// Starts the copy of one triangle of the jb x jb diagonal block of F at k0
// into sD[r * lds + c]: the strictly lower part (upper == 0) or the upper part
// with the diagonal.  Columns over the CTA's warps, rows over the lanes
// (coalesced).  Completion: cp.async.wait_all, then a barrier.
template <typename T>
__device__ __forceinline__ void stage_triangle(const T* __restrict__ F, int64_t ld, int k0, int jb,
                                               T* sD, int lds, int upper) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int c = warp; c < jb; c += nw) {
        const T* fc = F + k0 + (int64_t)(k0 + c) * ld;
        for (int r = upper ? lane : c + 1 + lane; r < (upper ? c + 1 : jb); r += 32)
            cp_async_elem(sD + r * lds + c, fc + r);
    }
}

// Columns [col_begin, col_begin+ncols) of B: the panel's gather list, then
// B[k0:k0+jb, col] <- L11^{-1} B[k0:k0+jb, col] (L11 unit lower, from F,
// staged in sL with row stride TriMax + 1).  Warp w takes the columns
// first + w, first + w + stride, ...
template <typename T>
__device__ __forceinline__ void swap_trsm_cols(int k0, int jb, const T* __restrict__ F, int64_t ld,
                                               const int2* __restrict__ gl, int cnt, T* B,
                                               int64_t ldb, int col_begin, int ncols, T* sL,
                                               int first, int stride) {
    constexpr int LDS = TriMax<T>::value + 1;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    stage_triangle(F, ld, k0, jb, sL, LDS, 0);
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    for (int cl = first + warp; cl < ncols; cl += stride) {
        T* col = B + (int64_t)(col_begin + cl) * ldb;
        // interchanges: every src read before any dst written
        T g[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = lane + 32 * q;
            if (e < cnt) g[q] = col[gl[e].y];
        }
        __syncwarp();
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = lane + 32 * q;
            if (e < cnt) col[gl[e].x] = g[q];
        }
        __syncwarp();
        T x0 = (lane < jb) ? col[k0 + lane] : cmake<T>(0.0, 0.0);
        T x1 = (lane + 32 < jb) ? col[k0 + lane + 32] : cmake<T>(0.0, 0.0);
        for (int i = 0; i < jb; ++i) {
            T src = (i < 32) ? x0 : x1;
            T xi;
            xi.x = __shfl_sync(0xffffffffu, src.x, i & 31);
            xi.y = __shfl_sync(0xffffffffu, src.y, i & 31);
            if (lane > i) x0 = cfms(sL[lane * LDS + i], xi, x0);
            if (lane + 32 > i && lane + 32 < jb) x1 = cfms(sL[(lane + 32) * LDS + i], xi, x1);
        }
        if (lane < jb) col[k0 + lane] = x0;
        if (lane + 32 < jb) col[k0 + lane + 32] = x1;
    }
}

// One column per warp: column blockIdx.x * kWarpsPerCta + warp.
template <typename T>
__device__ __forceinline__ void swap_trsm_body(int k0, int jb, const T* __restrict__ F, int64_t ld,
                                               const int2* __restrict__ gl, int cnt, T* B,
                                               int64_t ldb, int col_begin, int ncols) {
    __shared__ __align__(16) T sL[TriMax<T>::value * (TriMax<T>::value + 1)];
    swap_trsm_cols<T>(k0, jb, F, ld, gl, cnt, B, ldb, col_begin, ncols, sL,
                      blockIdx.x * kWarpsPerCta, ncols > 0 ? ncols : 1);
}

template <typename T>
__global__ void __launch_bounds__(32 * kWarpsPerCta) swap_trsm_lower_kernel(
    int64_t n, int k0, int jb, const T* __restrict__ F, int64_t ld, int64_t strideF,
    const int2* __restrict__ gather, const int* __restrict__ gcount, int gstride, int panel_index,
    T* B, int64_t ldb, int64_t strideB, int col_begin, int ncols, const int* __restrict__ active,
    int group) {
    const int node = blockIdx.y;
    if (active && !active[node / group]) return;     // a finished contour's nodes
    swap_trsm_body<T>(k0, jb, F + node * strideF, ld,
                      gather + (int64_t)node * gstride + panel_index * 2 * 64,
                      gcount[(int64_t)node * (gstride / 128) + panel_index], B + node * strideB, ldb,
                      col_begin, ncols);
}

// Columns of nodes of different orders, from their descriptors: mode 0 the
// next panel's columns, mode 1 the columns right of it (the look-ahead split).
template <typename T>
__global__ void __launch_bounds__(32 * kWarpsPerCta) swap_trsm_grouped_kernel(
    const LuNode* __restrict__ nodes, int k0, int nb, int panel_index, int mode) {
    const LuNode d = nodes[blockIdx.y];
    int jb, c0, ncols;
    if (!lookahead_cols(d.n, k0, nb, mode, &jb, &c0, &ncols)) return;
    T* F = static_cast<T*>(d.F);
    swap_trsm_body<T>(k0, jb, F, d.n, d.gather + panel_index * 2 * 64, d.gcount[panel_index], F,
                      d.n, c0, ncols);
}

// ---------------------------------------------------------------------------
// Interchanges of panel k on the L columns of panel k - 1 (k odd), so that the
// solves can treat panels k - 1 and k as one block of 2 nb rows.
// ---------------------------------------------------------------------------
// One warp applies a gather list (dst <- src rows, at most 128 entries) to one
// column: every src read before any dst written.
template <typename T>
__device__ __forceinline__ void gather_rows_warp(const int2* __restrict__ gl, int cnt, T* col) {
    const int lane = threadIdx.x & 31;
    T g[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int e = lane + 32 * q;
        if (e < cnt) g[q] = col[gl[e].y];
    }
    __syncwarp();
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int e = lane + 32 * q;
        if (e < cnt) col[gl[e].x] = g[q];
    }
    __syncwarp();
}

template <typename T>
__global__ void __launch_bounds__(32 * kWarpsPerCta) swap_cols_kernel(
    int c0, int ncols, T* F, int64_t ld, int64_t strideF, const int2* __restrict__ gather,
    const int* __restrict__ gcount, int gstride, int panel_index) {
    const int node = blockIdx.y;
    const int c = blockIdx.x * kWarpsPerCta + (threadIdx.x >> 5);
    if (c >= ncols) return;
    gather_rows_warp(gather + (int64_t)node * gstride + panel_index * 2 * 64,
                     gcount[(int64_t)node * (gstride / 128) + panel_index],
                     F + node * strideF + (int64_t)(c0 + c) * ld);
}

// The same for nodes of different orders: panel k's list on the nb columns of
// panel k - 1, in every node that has a panel k.
template <typename T>
__global__ void __launch_bounds__(32 * kWarpsPerCta) swap_cols_grouped_kernel(
    const LuNode* __restrict__ nodes, int k0, int nb, int panel_index) {
    const LuNode d = nodes[blockIdx.y];
    if (k0 >= d.n) return;
    const int c = blockIdx.x * kWarpsPerCta + (threadIdx.x >> 5);
    if (c >= nb) return;
    gather_rows_warp(d.gather + panel_index * 2 * 64, d.gcount[panel_index],
                     static_cast<T*>(d.F) + (int64_t)(k0 - nb + c) * d.n);
}

// ---------------------------------------------------------------------------
// Block substitution step of the solves, one warp per right-hand-side column,
// on a diagonal block of jb <= SB rows (two panels):
//   lower (forward): the interchanges of the block's panels, then
//          B[k0:k0+jb, col] <- L_bb^{-1} B[k0:k0+jb, col] (unit lower);
//   upper (backward): B[k0:k0+jb, col] <- U_bb^{-1} B[k0:k0+jb, col].
// The triangle in use is staged in shared memory row-major with row stride
// SB + 1 (conflict-free for the lanes' rows; the diagonal of U stored
// inverted); lane l holds rows l, l + 32, l + 64, l + 96 in registers.
// ---------------------------------------------------------------------------
constexpr int kBlockWarps = 16;

template <typename T>
__device__ __forceinline__ T pick_slot(const T* x, int q) {
    T v = x[0];
#pragma unroll
    for (int u = 1; u < 4; ++u)
        if (u == q) v = x[u];
    return v;
}

// One CTA's share of a block substitution: stage the triangle, then its warps
// take the column groups first + warp, first + warp + stride, ... (group g =
// columns g NC .. g NC + NC - 1 below ncols of B; column cl at B + cl * ldb;
// the block's rows are k0 .. k0 + jb - 1 of every column).  A warp solves the
// NC columns of a group together, so each triangle entry it reads from shared
// memory serves NC columns; per column the operations and their order are
// those of a one-column solve.  gl / gc: the block's first panel's gather list
// and count (the second panel's follow at gl + 128, gc + 1).
template <typename T, int SB, int NC>
__device__ __forceinline__ void trsm_block_body(int k0, int jb, int nb, const T* __restrict__ F,
                                                int64_t ld, const int2* __restrict__ gl,
                                                const int* __restrict__ gc, T* B, int64_t ldb,
                                                int ncols, int upper, int first, int stride) {
    static_assert(SB % 32 == 0 && SB <= 128, "at most four rows per lane");
    constexpr int Q = SB / 32, LDS = SB + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sD = reinterpret_cast<T*>(smem_raw);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    stage_triangle(F, ld, k0, jb, sD, LDS, upper);
    int grp = first + warp;
    auto gather_group = [&](int g) {
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const int cl = g * NC + c;
            if (cl < ncols) {
                T* col = B + (int64_t)cl * ldb;
                gather_rows_warp(gl, gc[0], col);
                if (jb > nb) gather_rows_warp(gl + 2 * 64, gc[1], col);
            }
        }
    };
    if (!upper && grp * NC < ncols) gather_group(grp);    // while the triangle is in flight
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    if (upper) {                                  // the diagonal, inverted
        for (int r = threadIdx.x; r < jb; r += blockDim.x) sD[r * LDS + r] = crcp(sD[r * LDS + r]);
        __syncthreads();
    }
    for (; grp * NC < ncols; grp += stride) {
        if (!upper && grp != first + warp) gather_group(grp);
        T x[NC][4];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const int cl = grp * NC + c;
            const T* col = B + (int64_t)min(cl, ncols - 1) * ldb + k0;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int r = lane + 32 * q;
                x[c][q] = (cl < ncols && q < Q && r < jb) ? col[r] : cmake<T>(0.0, 0.0);
            }
        }
        if (!upper) {
#pragma unroll 2
            for (int i = 0; i + 1 < jb; ++i) {
                T xi[NC];
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    const T own = pick_slot(x[c], i >> 5);
                    xi[c].x = __shfl_sync(0xffffffffu, own.x, i & 31);
                    xi[c].y = __shfl_sync(0xffffffffu, own.y, i & 31);
                }
#pragma unroll
                for (int q = 0; q < Q; ++q) {
                    const int r = lane + 32 * q;
                    if (r > i && r < jb) {
                        const T l = sD[r * LDS + i];
#pragma unroll
                        for (int c = 0; c < NC; ++c) x[c][q] = cfms(l, xi[c], x[c][q]);
                    }
                }
            }
        } else {
#pragma unroll 2
            for (int i = jb - 1; i >= 0; --i) {
                const T dinv = sD[i * LDS + i];
                T xi[NC];
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    const T own = pick_slot(x[c], i >> 5);
                    xi[c].x = __shfl_sync(0xffffffffu, own.x, i & 31);
                    xi[c].y = __shfl_sync(0xffffffffu, own.y, i & 31);
                    xi[c] = xi[c] * dinv;
                }
#pragma unroll
                for (int q = 0; q < Q; ++q) {
                    const int r = lane + 32 * q;
                    if (r == i) {
#pragma unroll
                        for (int c = 0; c < NC; ++c) x[c][q] = xi[c];
                    } else if (r < i) {
                        const T u = sD[r * LDS + i];
#pragma unroll
                        for (int c = 0; c < NC; ++c) x[c][q] = cfms(u, xi[c], x[c][q]);
                    }
                }
            }
        }
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const int cl = grp * NC + c;
            if (cl < ncols) {
                T* col = B + (int64_t)cl * ldb + k0;
#pragma unroll
                for (int q = 0; q < Q; ++q) {
                    const int r = lane + 32 * q;
                    if (r < jb) col[r] = x[c][q];
                }
            }
        }
    }
}

// NC: columns per warp (1 for the solves' right-hand sides, where the chain
// of a column is the latency to hide; kLuTrsmCols for the factorisation's
// trailing columns, where the triangle's shared-memory reads bound)
constexpr int kLuTrsmCols = 4;
template <typename T, int SB, int NC>
__global__ void __launch_bounds__(32 * kBlockWarps) trsm_block_kernel(
    int k0, int jb, int nb, const T* __restrict__ F, int64_t ld, int64_t strideF,
    const int2* __restrict__ gather, const int* __restrict__ gcount, int gstride, int panel_index,
    T* B, int64_t ldb, int64_t strideB, int ncols, int upper, const int* __restrict__ active,
    int group) {
    const int node = blockIdx.y;
    if (active && !active[node / group]) return;     // a finished contour's nodes
    trsm_block_body<T, SB, NC>(k0, jb, nb, F + node * strideF, ld,
                           gather + (int64_t)node * gstride + panel_index * 2 * 64,
                           gcount + (int64_t)node * (gstride / 128) + panel_index,
                           B + node * strideB, ldb, ncols, upper, blockIdx.x * kBlockWarps,
                           gridDim.x * kBlockWarps);
}

// A pair's block substitution on the columns of nodes of different orders:
// mode 0 the next pair's columns, mode 1 the columns right of them.
template <int SB, int NC>
__global__ void __launch_bounds__(32 * kBlockWarps) trsm_block_grouped_kernel(
    const LuNode* __restrict__ nodes, int k0, int nb, int panel_index, int mode) {
    const LuNode d = nodes[blockIdx.y];
    int jb, c0, ncols;
    if (!lookahead_cols(d.n, k0, 2 * nb, mode, &jb, &c0, &ncols)) return;
    float2* F = static_cast<float2*>(d.F);
    trsm_block_body<float2, SB, NC>(k0, jb, nb, F, d.n, d.gather + panel_index * 2 * 64,
                                d.gcount + panel_index, F + (int64_t)c0 * d.n, d.n, ncols, 0,
                                blockIdx.x * kBlockWarps, gridDim.x * kBlockWarps);
}

// ---------------------------------------------------------------------------
// The batched factorisation as one persistent launch
// ---------------------------------------------------------------------------
// The pair scheme of lu_factor_batched (see above) as a device work queue:
// per node d and pair p (k0 = 2 nb p) the tasks
//   P0  panel 2p                     needs: column block 2p updated by pair p-1
//   B1  panel 2p on block 2p+1       needs: P0, block 2p+1 updated by pair p-1
//       (swap + nb-row triangle, update with K = nb)
//   P1  panel 2p+1                   needs: B1
//   SW  pair swap (2p+1's list on 2p's L)   needs: P1
//   COL(cb) pair p on column block cb (both lists, 2 nb-row triangle, update
//       with K = 2 nb)               needs: SW, block cb updated by pair p-1
// are listed in an order in which every task comes after the tasks it needs
// (P0..SW of pair p+1 before the wide blocks of pair p, so the next panels
// overlap them).  Each CTA (512 threads: the panels, triangles and swaps on
// all of them; the updates on three 160-thread tensor-core units with 128
// TMEM columns each) takes the next task from a counter, waits for the flags
// of what it needs and raises its own when done.  A task only waits on tasks
// taken before it, each held by a running CTA, so the queue always moves; the
// waits are still bounded (on expiry: error bit 16, every CTA stops).  Every
// task does the arithmetic of the launch-per-step path with the same device
// functions and tiles, so the factors are the same bits.
constexpr int kPersistThreads = 512;
constexpr int kPersistUnits = 3;                 // tensor-core units per CTA
constexpr long long kPersistSpin = 1ll << 24;    // x ~128 ns sleep: ~2 s
constexpr int kPersistSmem = kPersistUnits * tcu::stage_smem<kLuUpdateBn>();
static_assert(kPersistUnits * tcu::kTcThreads <= kPersistThreads, "units fit the CTA");
static_assert((int)(128 * 129 * sizeof(float2)) <= kPersistSmem, "the triangle fits the rings' space");

enum : int { kTaskP0 = 0, kTaskB1 = 1, kTaskP1 = 2, kTaskSW = 3, kTaskCol = 4 };
struct PersistTask { int kind, node, pair, cb; };

struct PersistPlan {
    const LuNode* nodes;
    const PersistTask* tasks;
    int ntasks;
    int nb;
    int* next;            // the queue's counter
    int* flags;           // per node and pair: P0, B1, P1, SW, then one per column block
    int pair_stride;      // 4 + column blocks
    int node_stride;      // pairs * pair_stride
    int* err;
};

__device__ __forceinline__ int ld_acquire_gpu(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_gpu(int* p, int v) {
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// one thread: bounded wait for a raised flag
__device__ __forceinline__ bool wait_flag(const int* f) {
    for (long long i = 0; i < kPersistSpin; ++i) {
        if (ld_acquire_gpu(f)) return true;
        __nanosleep(128);
    }
    return false;
}

// The panel of column k0p on this CTA alone (a cluster of one), rows per thread
// chosen from the remaining rows.
__device__ __forceinline__ void persist_panel(const LuNode& d, int k0p, int nb, int panel) {
    const int64_t rows = d.n - k0p;
    const int jb = (int)min((int64_t)nb, rows);
    float2* F = static_cast<float2*>(d.F);
    int2* gl = d.gather + panel * 2 * 64;
    int* gc = d.gcount + panel;
    if (rows <= 2 * kClusterThreads)
        panel_cluster_body<float2, 2>(d.n, k0p, jb, F, d.n, d.piv, d.info, gl, gc);
    else if (rows <= 4 * kClusterThreads)
        panel_cluster_body<float2, 4>(d.n, k0p, jb, F, d.n, d.piv, d.info, gl, gc);
    else
        panel_cluster_body<float2, 8>(d.n, k0p, jb, F, d.n, d.piv, d.info, gl, gc);
}

// The update rows [0, rows) x columns [0, ncols) of C -= A B (K = k) on the
// CTA's tensor-core units, 128-row tiles dealt round-robin; false on a timeout.
__device__ __forceinline__ bool persist_update(tcu::TcUnit& u, int unit, int rows, int ncols, int k,
                                               const float2* A, const float2* B, float2* C,
                                               int64_t ld) {
    bool ok = true;
    if (unit < kPersistUnits) {
        const int utid = threadIdx.x - unit * tcu::kTcThreads;
        const int tiles = (rows + tcu::kTcM - 1) / tcu::kTcM;
        for (int i = unit; i < tiles; i += kPersistUnits)
            if (!tcu::cgemm_tile<kLuUpdateBn, false>(u, utid, rows, ncols, k, A, ld, B, ld, C, ld,
                                              i * tcu::kTcM, 0)) {
                ok = false;                       // unit-uniform: stop this unit's tiles
                break;
            }
    }
    return ok;
}

__global__ void __launch_bounds__(kPersistThreads, 1) lu_persistent_kernel(PersistPlan P) {
    extern __shared__ __align__(1024) unsigned char dsm[];     // the units' rings, or a triangle
    __shared__ __align__(8) uint64_t ufull[kPersistUnits][tcu::kTcStages];
    __shared__ __align__(8) uint64_t uempty[kPersistUnits][tcu::kTcStages];
    __shared__ __align__(8) uint64_t udone[kPersistUnits];
    __shared__ uint32_t s_tmem;
    __shared__ PersistTask s_task;
    __shared__ int s_stop;
    const int tid = threadIdx.x, warp = tid >> 5;
    if (tid == 0) {
        for (int q = 0; q < kPersistUnits; ++q) tcu::unit_init_barriers(ufull[q], uempty[q], &udone[q]);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         tc::smem_u32(&s_tmem)),
                     "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int unit = tid / tcu::kTcThreads;         // 3: the spare warp
    const int uq = unit < kPersistUnits ? unit : 0;
    tcu::TcUnit u{dsm + uq * tcu::stage_smem<kLuUpdateBn>(), ufull[uq], uempty[uq], &udone[uq],
                  s_tmem + (uint32_t)(uq * 128), 1 + uq, 0u, 0u};
    const int nb = P.nb;
    for (;;) {
        if (tid == 0) {
            int stop = 0;
            const int t = atomicAdd(P.next, 1);
            if (t >= P.ntasks || (ld_acquire_gpu(P.err) & 16)) {
                stop = 1;
            } else {
                const PersistTask tk = P.tasks[t];
                s_task = tk;
                const int* f = P.flags + (int64_t)tk.node * P.node_stride;
                const int* fp = f + tk.pair * P.pair_stride;            // this pair
                const int* fq = fp - P.pair_stride;                      // the previous pair
                bool ok = true;
                switch (tk.kind) {
                    case kTaskP0: if (tk.pair > 0) ok = wait_flag(fq + 4 + 2 * tk.pair); break;
                    case kTaskB1:
                        ok = wait_flag(fp + 0) && (tk.pair == 0 || wait_flag(fq + 4 + 2 * tk.pair + 1));
                        break;
                    case kTaskP1: ok = wait_flag(fp + 1); break;
                    case kTaskSW: ok = wait_flag(fp + 2); break;
                    default: ok = wait_flag(fp + 3) && (tk.pair == 0 || wait_flag(fq + 4 + tk.cb)); break;
                }
                if (!ok) {
                    atomicOr(P.err, 16);
                    stop = 1;
                }
            }
            s_stop = stop;
        }
        __syncthreads();
        if (s_stop) break;
        const PersistTask tk = s_task;
        const LuNode d = P.nodes[tk.node];
        float2* F = static_cast<float2*>(d.F);
        const int64_t n = d.n;
        const int k0 = 2 * nb * tk.pair;
        bool ok = true;
        switch (tk.kind) {
            case kTaskP0: persist_panel(d, k0, nb, 2 * tk.pair); break;
            case kTaskP1: persist_panel(d, k0 + nb, nb, 2 * tk.pair + 1); break;
            case kTaskB1: {
                const int jb1 = (int)min((int64_t)nb, n - k0 - nb);
                swap_trsm_cols<float2>(k0, nb, F, n, d.gather + 2 * tk.pair * 2 * 64,
                                       d.gcount[2 * tk.pair], F, n, k0 + nb, jb1,
                                       reinterpret_cast<float2*>(dsm), 0, kPersistThreads / 32);
                __syncthreads();                      // the triangle's space goes to the rings
                ok = persist_update(u, unit, (int)(n - k0 - nb), jb1, nb,
                                    F + (k0 + nb) + (int64_t)k0 * n, F + k0 + (int64_t)(k0 + nb) * n,
                                    F + (k0 + nb) + (int64_t)(k0 + nb) * n, n);
                break;
            }
            case kTaskSW:
                for (int c = warp; c < nb; c += kPersistThreads / 32)
                    gather_rows_warp(d.gather + (2 * tk.pair + 1) * 2 * 64, d.gcount[2 * tk.pair + 1],
                                     F + (int64_t)(k0 + c) * n);
                break;
            default: {
                const int jb = 2 * nb;
                const int c0 = tk.cb * nb;
                const int ncols = (int)min((int64_t)nb, n - c0);
                trsm_block_body<float2, 128, kLuTrsmCols>(k0, jb, nb, F, n, d.gather + 2 * tk.pair * 2 * 64,
                                             d.gcount + 2 * tk.pair, F + (int64_t)c0 * n, n, ncols, 0,
                                             0, kPersistThreads / 32);
                __syncthreads();
                ok = persist_update(u, unit, (int)(n - k0 - jb), ncols, jb,
                                    F + (k0 + jb) + (int64_t)k0 * n, F + k0 + (int64_t)c0 * n,
                                    F + (k0 + jb) + (int64_t)c0 * n, n);
                break;
            }
        }
        if (!ok && (threadIdx.x % tcu::kTcThreads) == 0) atomicOr(P.err, 16);
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            const int slot = tk.kind == kTaskCol ? 4 + tk.cb : tk.kind;
            st_release_gpu(P.flags + (int64_t)tk.node * P.node_stride + tk.pair * P.pair_stride + slot, 1);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(s_tmem), "r"(512));
}

// rows of a solve block: two panels
template <typename T> struct SolveBlock;
template <> struct SolveBlock<float2> { static constexpr int value = 128; };
template <> struct SolveBlock<double2> { static constexpr int value = 64; };

template <typename T>
constexpr size_t solve_block_smem() {
    return (size_t)SolveBlock<T>::value * (SolveBlock<T>::value + 1) * sizeof(T);
}

// the dynamic shared memory of the block substitution kernels, once per device
template <typename T>
cudaError_t trsm_block_attr() {
    constexpr int SB = SolveBlock<T>::value;
    constexpr int smem = (int)solve_block_smem<T>();
    static std::atomic<bool> attr_set[64] = {};   // idempotent setup; atomic for concurrent handles
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64 || !attr_set[dev]) {
        if ((e = cudaFuncSetAttribute(trsm_block_kernel<T, SB, 1>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess ||
            (e = cudaFuncSetAttribute(trsm_block_kernel<T, SB, kLuTrsmCols>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess)
            return e;
        if constexpr (sizeof(T) == 8)
            if ((e = cudaFuncSetAttribute(trsm_block_grouped_kernel<SB, kLuTrsmCols>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess)
                return e;
        if (dev >= 0 && dev < 64) attr_set[dev] = true;
    }
    return cudaSuccess;
}

// CTAs per node of a block substitution over `groups` column groups (one per
// warp at a time): enough for about four waves of one CTA per SM over all
// nodes; the warps loop over the rest
inline unsigned trsm_block_ctas(int64_t groups, int nodes) {
    const int64_t need = (groups + kBlockWarps - 1) / kBlockWarps;
    const int64_t cap = std::max<int64_t>(1, (4 * 152 + nodes - 1) / nodes);
    return (unsigned)std::max<int64_t>(1, std::min(need, cap));
}

// Cluster shape of a complex64 panel of `rows` rows: CL CTAs of 512 threads,
// ROWS rows per thread.  Taller panels spread over more CTAs, one per
// FEAST_NL_PANEL_ROWS_PER_CTA rows (default 1024, measured best of 300, 512
// and 1024 on the n = 4096 QEP: node LU 50.2, 47.0 and 46.3 ms against 54.3
// with every panel on one CTA; 0 keeps every panel on one CTA); false when
// one CTA takes the panel.  The factors do not depend on it.
constexpr int64_t kPanelRowsPerCta = 1024;
bool panel_cluster_shape(int64_t rows, int* cl, int* rows_per_thread) {
    const char* e = getenv("FEAST_NL_PANEL_ROWS_PER_CTA");
    const int64_t rpc = e ? atoll(e) : kPanelRowsPerCta;
    if (rpc <= 0 || rows <= rpc || rows > 2 * kClusterMax * kClusterThreads) return false;
    int c = (int)std::min<int64_t>(kClusterMax, (rows + rpc - 1) / rpc);
    int r = (int)((rows + (int64_t)c * kClusterThreads - 1) / ((int64_t)c * kClusterThreads));
    if (r > 2) { c = kClusterMax; r = 2; }
    *cl = c;
    *rows_per_thread = r;
    return true;
}

// launch with a cluster of cl CTAs along x (one cluster per node row of the grid)
template <typename... KArgs, typename... Args>
cudaError_t launch_clustered(void (*kernel)(KArgs...), int cl, int ny, cudaStream_t st,
                             Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)cl, (unsigned)ny, 1);
    cfg.blockDim = dim3(kClusterThreads, 1, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)cl;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

template <typename T>
cudaError_t launch_panel(cudaStream_t st, int64_t n, int k0, int jb, T* F, int64_t strideF,
                         int* piv, int nc, int* info, int2* gather, int* gcount, int panel,
                         int gstride) {
    const int64_t rows = n - k0;
    note_launch();
    if constexpr (sizeof(T) == 8) {
        int cl = 0, rt = 0;
        if (panel_cluster_shape(rows, &cl, &rt)) {
            float2* F32 = reinterpret_cast<float2*>(F);
            const int64_t ld = n;
            if (rt == 1)
                return launch_clustered(lu_panel_cluster_kernel<1>, cl, nc, st, n, k0, jb, F32, ld,
                                        strideF, piv, info, gather, gcount, panel, gstride);
            return launch_clustered(lu_panel_cluster_kernel<2>, cl, nc, st, n, k0, jb, F32, ld,
                                    strideF, piv, info, gather, gcount, panel, gstride);
        }
    }
    if (rows <= kPanelThreads)
        lu_panel_reg_kernel<T, 1><<<nc, kPanelThreads, 0, st>>>(n, k0, jb, F, n, strideF, piv, info,
                                                                gather, gcount, panel, gstride);
    else if (rows <= kPanelThreads * 2)
        lu_panel_reg_kernel<T, 2><<<nc, kPanelThreads, 0, st>>>(n, k0, jb, F, n, strideF, piv, info,
                                                                gather, gcount, panel, gstride);
    else if constexpr (sizeof(T) == 8) {                     // complex128 would spill at 4 rows
        if (rows <= kPanelThreads * 4)
            lu_panel_reg_kernel<T, 4><<<nc, kPanelThreads, 0, st>>>(n, k0, jb, F, n, strideF, piv,
                                                                    info, gather, gcount, panel,
                                                                    gstride);
        else
            lu_panel_kernel<T><<<nc, kPanelThreads, 0, st>>>(n, k0, jb, F, n, strideF, piv, info,
                                                             gather, gcount, panel, gstride);
    } else
        lu_panel_kernel<T><<<nc, kPanelThreads, 0, st>>>(n, k0, jb, F, n, strideF, piv, info,
                                                         gather, gcount, panel, gstride);
    return cudaGetLastError();
}

// C -= A B: FP64 SIMT for complex128, tensor cores for complex64.
cudaError_t update(cudaStream_t st, int m, int n, int k, const double2* A, int64_t lda, int64_t sA,
                   const double2* B, int64_t ldb, int64_t sB, double2* C, int64_t ldc, int64_t sC,
                   int batch, int*, int, const int* = nullptr, int = 1) {
    return gemm<double2>(st, 0, m, n, k, make_double2(-1.0, 0.0), A, lda, sA, B, ldb, sB,
                         make_double2(1.0, 0.0), C, ldc, sC, batch);
}
cudaError_t update(cudaStream_t st, int m, int n, int k, const float2* A, int64_t lda, int64_t sA,
                   const float2* B, int64_t ldb, int64_t sB, float2* C, int64_t ldc, int64_t sC,
                   int batch, int* err, int bn, const int* active = nullptr, int group = 1) {
    return cgemm_sub_tf32x3(st, m, n, k, A, lda, sA, B, ldb, sB, C, ldc, sC, batch, err, bn, active,
                            group);
}

}  // namespace

template <> int lu_block_size<double2>() { return 32; }
template <> int lu_block_size<float2>() { return 64; }

int lu_gather_stride(int64_t n, int nb) {
    // per node: one 128-entry slot (2 * 64 rows max) per panel
    return (int)(((n + nb - 1) / nb) * 128);
}

// swap + trsm of panel k0 on the columns [c0, c0 + nc_cols), then their update
// with the panel's L21 (all rows below the panel)
template <typename T>
cudaError_t panel_apply(cudaStream_t st, int64_t n, int k0, int jb, T* F, int64_t strideF,
                        int nc, const int2* gather, const int* gcount, int gstride, int panel,
                        int64_t c0, int64_t ncols, int* err) {
    if (ncols <= 0) return cudaSuccess;
    dim3 g((unsigned)((ncols + kWarpsPerCta - 1) / kWarpsPerCta), nc);
    note_launch();
    swap_trsm_lower_kernel<T><<<g, 32 * kWarpsPerCta, 0, st>>>(
        n, k0, jb, F, n, strideF, gather, gcount, gstride, panel, F, n, strideF, (int)c0,
        (int)ncols, nullptr, 1);
    const int64_t rows = n - k0 - jb;
    if (rows <= 0) return cudaGetLastError();
    // the same tile width as the grouped factorisation, so that a node's
    // factors do not depend on which path formed them
    return update(st, (int)rows, (int)ncols, jb, F + (k0 + jb) + (int64_t)k0 * n, n, strideF,
                  F + k0 + c0 * n, n, strideF, F + (k0 + jb) + c0 * n, n, strideF, nc, err,
                  kLuUpdateBn);
}

// A pair of panels (rows and columns k0 .. k0 + jb - 1, jb = 2 nb, the pair
// swap done) on the columns [c0, c0 + ncols): both gather lists and the
// 2 nb x 2 nb unit lower triangle, then the update of every row below the pair
// with K = 2 nb.
template <typename T>
cudaError_t block_apply(cudaStream_t st, int64_t n, int k0, int jb, int nb, T* F, int64_t strideF,
                        int nc, const int2* gather, const int* gcount, int gstride, int panel,
                        int64_t c0, int64_t ncols, int* err) {
    if (ncols <= 0) return cudaSuccess;
    constexpr int SB = SolveBlock<T>::value;
    constexpr int smem = (int)solve_block_smem<T>();
    cudaError_t e = trsm_block_attr<T>();
    if (e != cudaSuccess) return e;
    dim3 g(trsm_block_ctas((ncols + kLuTrsmCols - 1) / kLuTrsmCols, nc), nc);
    note_launch();
    trsm_block_kernel<T, SB, kLuTrsmCols><<<g, 32 * kBlockWarps, smem, st>>>(
        k0, jb, nb, F, n, strideF, gather, gcount, gstride, panel, F + c0 * n, n, strideF,
        (int)ncols, 0, nullptr, 1);
    const int64_t rows = n - k0 - jb;
    if (rows <= 0) return cudaGetLastError();
    return update(st, (int)rows, (int)ncols, jb, F + (k0 + jb) + (int64_t)k0 * n, n, strideF,
                  F + k0 + c0 * n, n, strideF, F + (k0 + jb) + c0 * n, n, strideF, nc, err,
                  kLuUpdateBn);
}

// Right-looking blocked LU by pairs of panels with a look-ahead.  Pair p
// covers the columns B0 = [k0, k0 + nb) and B1 = [k0 + nb, k0 + 2 nb),
// k0 = 2 nb p; N = the next pair's 2 nb columns, R = the columns right of N.
//   high:  panel(B0) -> apply panel B0 to B1 (swap, nb-row triangle, update
//          with K = nb) -> panel(B1) -> pair swap (B1's list on B0's L) -> [P]
//          -> wait R(p-1) -> pair p on N (both lists, 2 nb-row triangle,
//          update with K = 2 nb)
//   low:   wait P -> pair p on R -> [R(p)]
// so the wide trailing updates of R take K = 2 nb: each entry of the trailing
// matrix is read and written once per pair instead of once per panel, which
// halves the factorisation's dominant DRAM traffic.  The panels and the
// updates feeding the next panel stay on the high-priority stream, so each
// pair's panels overlap the previous pair's update of R (the low stream's
// update of pair p-1 covers N, hence the wait).
namespace {
struct FactorStreams {
    cudaStream_t hi = nullptr, side = nullptr;
    cudaEvent_t evP = nullptr, evR[2] = {nullptr, nullptr}, evH = nullptr;
    ~FactorStreams() {
        for (cudaEvent_t ev : {evP, evR[0], evR[1], evH})
            if (ev) cudaEventDestroy(ev);
        for (cudaStream_t s : {hi, side})         // released once their work completes
            if (s) cudaStreamDestroy(s);
    }
    // both streams start after everything already queued on st (the assembly)
    cudaError_t create(cudaStream_t st) {
        int prio_lo = 0, prio_hi = 0;
        cudaError_t e;
        if ((e = cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi)) != cudaSuccess ||
            (e = cudaStreamCreateWithPriority(&hi, cudaStreamNonBlocking, prio_hi)) != cudaSuccess ||
            (e = cudaStreamCreateWithPriority(&side, cudaStreamNonBlocking, prio_lo)) != cudaSuccess)
            return e;
        for (cudaEvent_t* ev : {&evP, &evR[0], &evR[1], &evH})
            if ((e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming)) != cudaSuccess) return e;
        if ((e = cudaEventRecord(evP, st)) != cudaSuccess) return e;
        for (cudaStream_t s : {hi, side})
            if ((e = cudaStreamWaitEvent(s, evP, 0)) != cudaSuccess) return e;
        return cudaSuccess;
    }
    // everything the streams did is ordered before what follows on st
    cudaError_t join(cudaStream_t st, int last_r) {
        cudaError_t e;
        if ((e = cudaEventRecord(evH, hi)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(st, evH, 0)) != cudaSuccess)
            return e;
        if (last_r >= 0) return cudaStreamWaitEvent(st, evR[last_r & 1], 0);
        return cudaSuccess;
    }
};
}  // namespace

// The persistent factorisation: FEAST_NL_LU_PERSISTENT=1 uses it whenever it
// applies (complex64, nb = 64, every order <= 4096); otherwise the launches per
// panel step, which measured faster (64 discs of n = 2048: 217 against 574 ms;
// the mixed-order batch: 41 against 196 ms).
static bool lu_persistent_wanted(int count, int64_t nmax, int nb) {
    if (nmax > 4096 || nb != 64 || count <= 0) return false;
    const char* e = getenv("FEAST_NL_LU_PERSISTENT");
    return e && e[0] == '1';
}

// The task list of lu_persistent_kernel for nodes of orders n_host[0..count).
static std::vector<PersistTask> persist_tasks(const int64_t* n_host, int count, int nb, int* npair_out,
                                       int* ncb_out) {
    int64_t nmax = 0;
    for (int i = 0; i < count; ++i) nmax = std::max(nmax, n_host[i]);
    const int npair = (int)((nmax + 2 * nb - 1) / (2 * nb));
    const int ncb = (int)((nmax + nb - 1) / nb);
    std::vector<PersistTask> t;
    auto head = [&](int p) {                      // P0, B1, P1, SW of pair p, kind by kind
        const int64_t k0 = 2ll * nb * p;
        for (int i = 0; i < count; ++i)
            if (k0 < n_host[i]) t.push_back({kTaskP0, i, p, 0});
        for (int kind : {kTaskB1, kTaskP1, kTaskSW})
            for (int i = 0; i < count; ++i)
                if (n_host[i] - k0 > nb) t.push_back({kind, i, p, 0});
    };
    // the next pair's blocks, or those right of them, node by node: the tasks
    // running together then share one node's L21 block in L2 (ordered block
    // by block over the nodes, each task re-read its own node's L21 from DRAM)
    auto cols = [&](int p, bool next) {
        const int64_t k0 = 2ll * nb * p;
        const int lo = next ? 2 * p + 2 : 2 * p + 4, hi = next ? 2 * p + 4 : ncb;
        for (int i = 0; i < count; ++i)
            for (int cb = lo; cb < hi; ++cb)
                if (n_host[i] - k0 > 2 * nb && (int64_t)cb * nb < n_host[i]) t.push_back({kTaskCol, i, p, cb});
    };
    head(0);
    for (int p = 0; p < npair; ++p) {
        cols(p, true);
        if (p + 1 < npair) head(p + 1);
        cols(p, false);
    }
    *npair_out = npair;
    *ncb_out = ncb;
    return t;
}

// nodes: the descriptors in device memory, or null with nodes_host in host memory
static cudaError_t lu_factor_persistent(cudaStream_t st, const LuNode* nodes, const LuNode* nodes_host,
                                 const int64_t* n_host, int count, int nb, int* err) {
    int npair = 0, ncb = 0;
    const std::vector<PersistTask> tasks = persist_tasks(n_host, count, nb, &npair, &ncb);
    if (tasks.empty()) return cudaSuccess;
    static std::atomic<bool> attr_set[64] = {};
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if (dev < 0 || dev >= 64 || !attr_set[dev]) {
        if ((e = cudaFuncSetAttribute(lu_persistent_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      kPersistSmem)) != cudaSuccess)
            return e;
        if (dev >= 0 && dev < 64) attr_set[dev] = true;
    }
    // one device block: the counter, the flags, the node descriptors, the tasks
    const int pair_stride = 4 + ncb, node_stride = npair * pair_stride;
    const size_t head = 256, fbytes = (size_t)count * node_stride * sizeof(int);
    const size_t nbytes = nodes ? 0 : (size_t)count * sizeof(LuNode);
    const size_t tbytes = tasks.size() * sizeof(PersistTask);
    const size_t off_nodes = (head + fbytes + 255) / 256 * 256, off_tasks = (off_nodes + nbytes + 255) / 256 * 256;
    unsigned char* buf = nullptr;
    if ((e = cudaMallocAsync(&buf, off_tasks + tbytes, st)) != cudaSuccess) return e;
    e = cudaMemsetAsync(buf, 0, head + fbytes, st);
    if (e == cudaSuccess && !nodes)
        e = cudaMemcpyAsync(buf + off_nodes, nodes_host, nbytes, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(buf + off_tasks, tasks.data(), tbytes, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        PersistPlan P{nodes ? nodes : reinterpret_cast<const LuNode*>(buf + off_nodes),
                      reinterpret_cast<const PersistTask*>(buf + off_tasks), (int)tasks.size(), nb,
                      reinterpret_cast<int*>(buf), reinterpret_cast<int*>(buf + head), pair_stride,
                      node_stride, err};
        const int grid = (int)std::min<size_t>((size_t)sms, tasks.size());
        note_launch();
        lu_persistent_kernel<<<grid, kPersistThreads, kPersistSmem, st>>>(P);
        e = cudaGetLastError();
    }
    const cudaError_t ef = cudaFreeAsync(buf, st);
    return e != cudaSuccess ? e : ef;
}

template <typename T>
cudaError_t lu_factor_batched(cudaStream_t st, int64_t n, int nb, T* F, int64_t strideF,
                              int* piv, int nc, int* info, int2* gather, int* gcount, int* err) {
    const int gstride = lu_gather_stride(n, nb);
    const int npanel = (int)((n + nb - 1) / nb);
    if (nb % kWarpsPerCta != 0 || 2 * nb != SolveBlock<T>::value) return cudaErrorInvalidValue;
    if constexpr (sizeof(T) == 8) {
        if (lu_persistent_wanted(nc, n, nb)) {
            std::vector<LuNode> nodes(nc);
            std::vector<int64_t> ns(nc, n);
            for (int i = 0; i < nc; ++i)
                nodes[i] = LuNode{F + i * strideF, piv + (int64_t)i * n, info + i,
                                  gather + (int64_t)i * gstride, gcount + (int64_t)i * (gstride / 128), n};
            return lu_factor_persistent(st, nullptr, nodes.data(), ns.data(), nc, nb, err);
        }
    }
    FactorStreams S;
    cudaError_t e;
    if ((e = S.create(st)) != cudaSuccess) return e;
    cudaStream_t hi = S.hi, side = S.side;
    cudaEvent_t evP = S.evP, *evR = S.evR;
    int last_r = -1;                              // pair whose low-stream update was recorded last
    for (int p = 0; 2 * p < npanel; ++p) {
        const int k0 = 2 * nb * p;
        const int jb0 = (int)std::min<int64_t>(nb, n - k0);
        if ((e = launch_panel<T>(hi, n, k0, jb0, F, strideF, piv, nc, info, gather, gcount, 2 * p,
                                 gstride)) != cudaSuccess)
            return e;
        const int64_t r1 = n - k0 - jb0;
        if (r1 <= 0) break;
        const int jb1 = (int)std::min<int64_t>(nb, r1);
        if ((e = panel_apply<T>(hi, n, k0, jb0, F, strideF, nc, gather, gcount, gstride, 2 * p,
                                k0 + jb0, jb1, err)) != cudaSuccess)
            return e;
        if ((e = launch_panel<T>(hi, n, k0 + jb0, jb1, F, strideF, piv, nc, info, gather, gcount,
                                 2 * p + 1, gstride)) != cudaSuccess)
            return e;
        note_launch();                            // pair swap: B1's list on B0's L columns
        swap_cols_kernel<T><<<dim3((unsigned)(nb / kWarpsPerCta), nc), 32 * kWarpsPerCta, 0, hi>>>(
            k0, nb, F, n, strideF, gather, gcount, gstride, 2 * p + 1);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        const int jb = jb0 + jb1;
        const int64_t rest = n - k0 - jb;
        if (rest <= 0) break;
        const int64_t jn = std::min<int64_t>(2 * nb, rest);  // the next pair's columns
        const int64_t rr = rest - jn;                         // columns beyond them
        if (rr > 0) {
            if ((e = cudaEventRecord(evP, hi)) != cudaSuccess ||
                (e = cudaStreamWaitEvent(side, evP, 0)) != cudaSuccess)
                return e;
            if ((e = block_apply<T>(side, n, k0, jb, nb, F, strideF, nc, gather, gcount, gstride,
                                    2 * p, k0 + jb + jn, rr, err)) != cudaSuccess)
                return e;
        }
        if (last_r >= 0 && (e = cudaStreamWaitEvent(hi, evR[last_r & 1], 0)) != cudaSuccess)
            return e;
        if (rr > 0) {
            if ((e = cudaEventRecord(evR[p & 1], side)) != cudaSuccess) return e;
            last_r = p;
        }
        if ((e = block_apply<T>(hi, n, k0, jb, nb, F, strideF, nc, gather, gcount, gstride, 2 * p,
                                k0 + jb, jn, err)) != cudaSuccess)
            return e;
    }
    if ((e = S.join(st, last_r)) != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t lu_factor_grouped(cudaStream_t st, const LuNode* nodes, const int64_t* n_host,
                              int count, int nb, int* err) {
    int64_t nmax = 0;
    for (int i = 0; i < count; ++i) nmax = std::max(nmax, n_host[i]);
    if (count <= 0 || nmax <= 0) return cudaSuccess;
    if (nmax > 4 * kPanelThreads || count > 65535) return cudaErrorInvalidValue;
    const int npanel = (int)((nmax + nb - 1) / nb);
    if (nb % kWarpsPerCta != 0 || 2 * nb != SolveBlock<float2>::value) return cudaErrorInvalidValue;
    constexpr int SB = SolveBlock<float2>::value;
    constexpr int smem = (int)solve_block_smem<float2>();
    if (lu_persistent_wanted(count, nmax, nb))
        return lu_factor_persistent(st, nodes, nullptr, n_host, count, nb, err);
    FactorStreams S;
    cudaError_t e;
    if ((e = trsm_block_attr<float2>()) != cudaSuccess) return e;
    if ((e = S.create(st)) != cudaSuccess) return e;
    cudaStream_t hi = S.hi, side = S.side;
    cudaEvent_t evP = S.evP, *evR = S.evR;
    // one panel launch over the nodes that have panel k (rows: their largest
    // remaining order)
    auto panel = [&](int k0, int k, int64_t rows) -> cudaError_t {
        note_launch();
        int pcl = 0, prt = 0;
        cudaError_t pe = cudaSuccess;
        if (panel_cluster_shape(rows, &pcl, &prt))
            pe = prt == 1 ? launch_clustered(lu_panel_cluster_grouped_kernel<1>, pcl, count, hi, nodes, k0, nb, k)
                          : launch_clustered(lu_panel_cluster_grouped_kernel<2>, pcl, count, hi, nodes, k0, nb, k);
        else
            lu_panel_reg_grouped_kernel<float2><<<count, kPanelThreads, 0, hi>>>(nodes, k0, nb, k);
        return pe != cudaSuccess ? pe : cudaGetLastError();
    };
    // a pair's substitution and update on the nodes' columns of `mode`
    auto pair_apply = [&](cudaStream_t s, int k0, int p, int mode, int64_t rows_below,
                          int64_t cols) -> cudaError_t {
        dim3 g(trsm_block_ctas((cols + kLuTrsmCols - 1) / kLuTrsmCols, count), count);
        note_launch();
        trsm_block_grouped_kernel<SB, kLuTrsmCols><<<g, 32 * kBlockWarps, smem, s>>>(nodes, k0, nb,
                                                                                     2 * p, mode);
        cudaError_t pe = cudaGetLastError();
        if (pe != cudaSuccess) return pe;
        return cgemm_sub_grouped(s, nodes, count, k0, 2 * nb, mode, rows_below, cols, err);
    };
    int last_r = -1;
    for (int p = 0; 2 * p < npanel; ++p) {
        const int k0 = 2 * nb * p;
        // the largest extents over the nodes that have these panels
        int64_t rows0 = 0, rows1 = 0, b1_below = 0, b1_cols = 0, pr_below = 0, n_cols = 0, r_cols = 0;
        for (int i = 0; i < count; ++i) {
            const int64_t ni = n_host[i];
            int jb, c0, nn;
            if (k0 >= ni) continue;
            rows0 = std::max(rows0, ni - k0);
            if (ni - k0 > nb) rows1 = std::max(rows1, ni - k0 - nb);
            if (lookahead_cols(ni, k0, nb, 0, &jb, &c0, &nn)) {
                b1_cols = std::max<int64_t>(b1_cols, nn);
                b1_below = std::max(b1_below, ni - k0 - jb);
            }
            if (lookahead_cols(ni, k0, 2 * nb, 0, &jb, &c0, &nn)) {
                n_cols = std::max<int64_t>(n_cols, nn);
                pr_below = std::max(pr_below, ni - k0 - jb);
            }
            if (lookahead_cols(ni, k0, 2 * nb, 1, &jb, &c0, &nn)) r_cols = std::max<int64_t>(r_cols, nn);
        }
        if (rows0 <= 0) break;
        if ((e = panel(k0, 2 * p, rows0)) != cudaSuccess) return e;
        if (rows1 <= 0) continue;
        if (b1_cols > 0) {                        // panel B0 on B1
            dim3 g((unsigned)((b1_cols + kWarpsPerCta - 1) / kWarpsPerCta), count);
            note_launch();
            swap_trsm_grouped_kernel<float2><<<g, 32 * kWarpsPerCta, 0, hi>>>(nodes, k0, nb, 2 * p, 0);
            if ((e = cgemm_sub_grouped(hi, nodes, count, k0, nb, 0, b1_below, b1_cols, err)) !=
                cudaSuccess)
                return e;
        }
        if ((e = panel(k0 + nb, 2 * p + 1, rows1)) != cudaSuccess) return e;
        note_launch();                            // pair swap: B1's list on B0's L columns
        swap_cols_grouped_kernel<float2><<<dim3((unsigned)(nb / kWarpsPerCta), count),
                                           32 * kWarpsPerCta, 0, hi>>>(nodes, k0 + nb, nb, 2 * p + 1);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if (n_cols <= 0) continue;
        if (r_cols > 0) {
            if ((e = cudaEventRecord(evP, hi)) != cudaSuccess ||
                (e = cudaStreamWaitEvent(side, evP, 0)) != cudaSuccess)
                return e;
            if ((e = pair_apply(side, k0, p, 1, pr_below, r_cols)) != cudaSuccess) return e;
        }
        if (last_r >= 0 && (e = cudaStreamWaitEvent(hi, evR[last_r & 1], 0)) != cudaSuccess)
            return e;
        if (r_cols > 0) {
            if ((e = cudaEventRecord(evR[p & 1], side)) != cudaSuccess) return e;
            last_r = p;
        }
        if ((e = pair_apply(hi, k0, p, 0, pr_below, n_cols)) != cudaSuccess) return e;
    }
    if ((e = S.join(st, last_r)) != cudaSuccess) return e;
    return cudaGetLastError();
}

template <typename T>
cudaError_t lu_solve_batched(cudaStream_t st, int64_t n, int nb, const T* F, int64_t strideF,
                             const int2* gather, const int* gcount, int nc, T* Y, int64_t strideY,
                             int m, int* err, int bn, const int* active, int group) {
    constexpr int SB = SolveBlock<T>::value;
    constexpr int smem = (int)solve_block_smem<T>();
    const int sb = 2 * nb;                        // a block: two panels
    if (sb > SB) return cudaErrorInvalidValue;
    cudaError_t e = trsm_block_attr<T>();
    if (e != cudaSuccess) return e;
    const int gstride = lu_gather_stride(n, nb);
    dim3 g((unsigned)((m + kBlockWarps - 1) / kBlockWarps), nc);
    for (int64_t k0 = 0, panel = 0; k0 < n; k0 += sb, panel += 2) {
        const int jb = (int)std::min<int64_t>(sb, n - k0);
        note_launch();
        trsm_block_kernel<T, SB, 1><<<g, 32 * kBlockWarps, smem, st>>>(
            (int)k0, jb, nb, F, n, strideF, gather, gcount, gstride, (int)panel, Y, n, strideY, m, 0,
            active, group);
        const int64_t rest = n - k0 - jb;
        if (rest > 0) {
            e = update(st, (int)rest, m, jb, F + (k0 + jb) + k0 * n, n, strideF, Y + k0, n,
                       strideY, Y + k0 + jb, n, strideY, nc, err, bn, active, group);
            if (e != cudaSuccess) return e;
        }
    }
    const int64_t last = ((n - 1) / sb) * sb;
    for (int64_t k0 = last; k0 >= 0; k0 -= sb) {
        const int jb = (int)std::min<int64_t>(sb, n - k0);
        note_launch();
        trsm_block_kernel<T, SB, 1><<<g, 32 * kBlockWarps, smem, st>>>(
            (int)k0, jb, nb, F, n, strideF, gather, gcount, gstride, 0, Y, n, strideY, m, 1, active,
            group);
        if (k0 > 0) {
            e = update(st, (int)k0, m, jb, F + k0 * n, n, strideF, Y + k0, n, strideY, Y, n,
                       strideY, nc, err, bn, active, group);
            if (e != cudaSuccess) return e;
        }
    }
    return cudaGetLastError();
}

template cudaError_t lu_factor_batched<double2>(cudaStream_t, int64_t, int, double2*, int64_t,
                                                int*, int, int*, int2*, int*, int*);
template cudaError_t lu_factor_batched<float2>(cudaStream_t, int64_t, int, float2*, int64_t, int*,
                                               int, int*, int2*, int*, int*);
template cudaError_t lu_solve_batched<double2>(cudaStream_t, int64_t, int, const double2*,
                                               int64_t, const int2*, const int*, int, double2*,
                                               int64_t, int, int*, int, const int*, int);
template cudaError_t lu_solve_batched<float2>(cudaStream_t, int64_t, int, const float2*, int64_t,
                                              const int2*, const int*, int, float2*, int64_t, int,
                                              int*, int, const int*, int);

namespace {
std::mutex g_tune_mu;
std::map<std::tuple<int64_t, int, int>, int> g_tuned_bn;   // (n, m, nc) -> tile width
}  // namespace

int lu_solve_pick_bn(cudaStream_t st, int64_t n, int nb, const float2* F, int64_t strideF,
                     const int2* gather, const int* gcount, int nc, float2* Y, int64_t strideY,
                     int m, int* err) {
    const auto key = std::make_tuple(n, m, nc);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tuned_bn.find(key);
        if (it != g_tuned_bn.end()) return it->second;
    }
    const int fallback = cgemm_default_bn(m);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone)
        return fallback;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        cudaGetLastError();
        return fallback;
    }
    int best = fallback;
    float best_ms = 0.0f;
    bool ok = true;
    for (int bn : {16, 32, 48, 64}) {
        if (bn >= 2 * m + 16 && bn != fallback) continue;   // mostly empty tiles
        float ms_min = 0.0f;
        for (int rep = 0; rep < 3 && ok; ++rep) {           // first run warms the kernel
            ok = cudaEventRecord(e0, st) == cudaSuccess &&
                 lu_solve_batched<float2>(st, n, nb, F, strideF, gather, gcount, nc, Y, strideY, m,
                                          err, bn) == cudaSuccess &&
                 cudaEventRecord(e1, st) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess;
            float ms = 0.0f;
            if (ok) ok = cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
            if (rep == 1 || (rep > 1 && ms < ms_min)) ms_min = ms;
        }
        if (!ok) break;
        if (best_ms == 0.0f || ms_min < best_ms) { best_ms = ms_min; best = bn; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!ok) {
        cudaGetLastError();
        return fallback;
    }
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned_bn[key] = best;
    return best;
}

}  // namespace fnl
