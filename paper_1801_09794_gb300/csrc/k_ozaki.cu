// FP64-accurate complex products W = A Q on the BF16 tensor cores (tcgen05).
//
// GB300 executes FP64 at ~1.1 TFLOP/s and dense BF16 MMA at ~2 PFLOP/s.  The
// block residual T(X, Lambda) and the projections Q^H A Q of Algorithm 1 need
// FP64-level accuracy, and their cost is dominated by the products A_t Q
// (8 n^2 m0 flops per term and iteration).  They are computed here by an
// error-free splitting into small-integer digit slices (the idea of Ozaki,
// Ogita, Oishi and Rump for accurate matrix products, written from its
// definition):
//
//   A' = [Re A | Im A]  (n x 2n, real) and Q' (2n x 2m, real; column 2j is
//   [Re q_j; -Im q_j], column 2j+1 is [Im q_j; Re q_j]), so A' Q' holds Re W and
//   Im W column-interleaved;
//   A'_ik = sigma_i (sum_{p=1..s} a^(p)_ik 2^{-7p} + r_ik),  |r_ik| < 2^{-7s},
//   Q'_kj = tau_j   (sum_{q=1..s} b^(q)_kj 2^{-7q} + r'_kj), |r'_kj| < 2^{-7s},
//   a, b integers in [-127, 127] (truncated base-128 digits after scaling by a
//   power of two strictly above the row / column maximum), stored as BF16,
//   which holds them exactly;
//   W'_ij ~= sigma_i tau_j sum_{L=2..s+1} 2^{-7L} S_L(i,j),  S_L = sum_{p+q=L} a^(p) b^(q).
//
// Each product of digits is exact in FP32 and an FP32 sum of integers is exact
// while it stays below 2^24.  The three leading levels L = 2, 3, 4 (at most
// three slice pairs each) are therefore accumulated in TMEM over 256-element
// K chunks (3 * 256 * 127^2 < 2^24) and drained into int32 registers after
// every chunk, which keeps them exact; levels L >= 5 carry weights <= 2^-35 and
// are accumulated in FP32 over the whole K, i.e. K/16 sequential additions
// into TMEM.  Their rounding error: each level sum has at most 4 digit pairs,
// so |S_L| <= 4 * 127^2 * K, and K/16 additions at unit roundoff 2^-24 give
// at most (K/16) 2^-24 |S_L| -- after the level weight, <= 2^-47 K relative to
// sigma_i tau_j K (the row maximum times the column maximum times K): 5.8e-11
// at the largest K here (2n = 8192) in the worst case, where every rounding
// error has the same sign.  With rounding errors of random sign (the usual
// model) the sum's error grows like sqrt(K/16) instead, ~2^-45 relative to
// sigma_i tau_j K at any K.  The dropped pairs (p + q > s + 1) and the
// truncation remainders are below 2^{-7s} of sigma_i (resp. tau_j) per operand
// entry.  With s = 7 the measured error of the projections at n = 4096,
// m0 = 96 is ~1e-15 relative (a GPU parity test checks it against FP64).
//
// Kernel: one CTA (256 threads) per 128 x 48 tile of W'.  K advances in
// 16-element stages through a 5-slot cp.async ring (loads three stages ahead,
// the MMAs of two stages queued behind them; one block barrier per stage,
// after which the stage's copies have all landed and the slot to refill is
// free);
// thread 0 issues tcgen05.mma.kind::f16 (M = 128, K = 16) once per A slice p
// against the B slices q = 0 .. s-1-p side by side (N = 48 per slice, at most
// five per instruction), with D placed so that slice q's columns fall on
// level p + q's TMEM region (nine MMAs per K step instead of 28, which cuts
// the shared-memory reads of A that bound the small-N products), and commits
// each stage to the slot's mbarrier, which releases the slot for the stage
// five ahead.  Warps w
// and w + 4 read TMEM lanes 32 (w mod 4) .. and split the 48 columns.  Operand
// tiles use the canonical K-major layout without swizzle: 8-row x 16-byte core
// matrices (128 bytes), the two K chunks of a row group side by side
// (LBO = 128 B along K, SBO = 256 B between row groups).
#include "internal.h"
#include "tc_common.cuh"

#include <cuda_bf16.h>

#include <algorithm>

namespace fnl {
namespace {
using namespace tc;

constexpr int kOzM = 128;          // rows of W' per CTA (TMEM lanes)
constexpr int kOzN = 48;           // columns of W' per CTA
constexpr int kOzBK = 16;          // K elements (32 bytes) per stage
constexpr int kOzStages = 5;       // shared-memory ring depth
// Stages loaded ahead of the one being multiplied, and stages of MMAs left
// queued while a slot is refilled: kOzLead + kOzMmaAhead = kOzStages, so the
// refilled slot is the one the MMAs of stage t - kOzMmaAhead have released.
constexpr int kOzLead = 3;
constexpr int kOzMmaAhead = kOzStages - kOzLead;
constexpr int kOzGroup = 5;        // B slices per MMA (N = 5 x 48 <= 256)
constexpr int kOzThreads = 256;
constexpr int kOzMaxSlices = 8;
constexpr int kOzExact = 3;        // levels drained exactly (L = 2..4)
constexpr int kOzChunkStages = 16; // 16 x 16 = 256 K elements between drains
constexpr uint32_t kTmemCols = 512;
// cp.async items (16 bytes) of a stage per thread, at most
constexpr int kOzLoadIters = (kOzMaxSlices * (kOzM + kOzN) * 2 + kOzThreads - 1) / kOzThreads;

// Instruction descriptor: kind::f16, D = F32, A = B = BF16, both K-major.
__host__ __device__ constexpr uint32_t bf16_idesc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

__global__ void __launch_bounds__(kOzThreads, 1) ozaki_bf16_gemm_kernel(
    int s, int Mrows, int Kp, const __nv_bfloat16* __restrict__ Aslices, int64_t a_slice_stride,
    int64_t a_term_stride, const double* __restrict__ sigma, int64_t sigma_term_stride,
    const __nv_bfloat16* __restrict__ Bslices, int64_t b_slice_stride, const double* __restrict__ tau,
    double2* __restrict__ W, int64_t ldw, int64_t w_term_stride, int mb, int64_t w_block_stride,
    const int* __restrict__ term_slot, int ncols_complex, int* __restrict__ err,
    const int* __restrict__ active, int split_stages, int64_t split_stride) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t mbar[kOzStages];
    __shared__ uint32_t s_tmem;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int quarter = warp & 3, colhalf = warp >> 2;     // TMEM lanes / column half
    // column tiles vary fastest, so the CTAs that share a row block of the A'
    // slices run together and read them from HBM once (the rest hit in L2)
    const int row0 = blockIdx.y * kOzM;
    const int col0 = blockIdx.x * kOzN;                    // real column of W'
    // split-K mode (split_stages > 0, one term): blockIdx.z takes K stages
    // [z * split_stages, ...) and writes its partial product to W + z * split_stride
    const int term = split_stages > 0 ? 0 : blockIdx.z;
    const int kst0 = split_stages > 0 ? blockIdx.z * split_stages : 0;
    if (active) {
        // complex columns [c_lo, c_hi] of this tile belong to blocks c / mb
        const int c_lo = col0 / 2, c_hi = min(ncols_complex, (col0 + kOzN) / 2) - 1;
        bool any = false;
        for (int b = c_lo / mb; b <= c_hi / mb; ++b) any = any || active[b] != 0;
        if (!any) return;
    }
    const __nv_bfloat16* A = Aslices + term * a_term_stride;
    const double* sg = sigma + term * sigma_term_stride;
    double2* Wt = W + (int64_t)term_slot[term] * w_term_stride +
                  (split_stages > 0 ? (int64_t)blockIdx.z * split_stride : 0);
    const int a_tile = kOzM * kOzBK * 2;                   // bytes per A slice tile (4 KB)
    const int b_tile = kOzN * kOzBK * 2;                   // 1.5 KB
    const int stage_bytes = s * (a_tile + b_tile);

    if (tid == 0) {
        for (int q = 0; q < kOzStages; ++q) mbar_init(smem_u32(&mbar[q]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&s_tmem)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s_tmem;
    const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);

    const int nk = split_stages > 0 ? min(Kp / kOzBK - kst0, split_stages) : Kp / kOzBK;
    int exact[kOzExact][kOzN / 2];                         // running sums of levels 2..4
#pragma unroll
    for (int L = 0; L < kOzExact; ++L)
#pragma unroll
        for (int c = 0; c < kOzN / 2; ++c) exact[L][c] = 0;
    // stage t (16 K elements of every slice) into ring slot t % kOzStages; each
    // row's 32 bytes are two 16-byte core-matrix rows (LBO 128 B, SBO 256 B).
    // A thread's copies are the same (slice, row, chunk) items at every stage,
    // so their source rows and shared-memory offsets are formed once here and
    // a stage only adds its K offset.
    const int nitems = s * (kOzM + kOzN) * 2;
    const __nv_bfloat16* lsrc[kOzLoadIters];
    uint32_t ldst[kOzLoadIters];
#pragma unroll
    for (int j = 0; j < kOzLoadIters; ++j) {
        const int idx = tid + j * kOzThreads;
        const int chunk = idx & 1;                         // 16-byte K chunk (8 elements)
        const int r = idx >> 1;
        int p = 0, rr = 0;
        uint32_t base = 0;
        const __nv_bfloat16* src = A;
        if (idx < nitems) {
            if (r < s * kOzM) {
                p = r / kOzM;
                rr = r - p * kOzM;
                src = A + p * a_slice_stride + (int64_t)(row0 + rr) * Kp + chunk * 8;
                base = (uint32_t)(p * a_tile);
            } else {
                const int r2 = r - s * kOzM;
                p = r2 / kOzN;
                rr = r2 - p * kOzN;
                src = Bslices + p * b_slice_stride + (int64_t)(col0 + rr) * Kp + chunk * 8;
                base = (uint32_t)(s * a_tile + p * b_tile);
            }
        }
        lsrc[j] = src;
        ldst[j] = base + (uint32_t)(((rr >> 3) * 2 + chunk) * 128 + (rr & 7) * 16);
    }
    auto load = [&](int t) {
        const int64_t k0 = (int64_t)(kst0 + t) * kOzBK;
        const uint32_t sbase = smem_u32(smem + (t % kOzStages) * stage_bytes);
#pragma unroll
        for (int j = 0; j < kOzLoadIters; ++j)
            if (tid + j * kOzThreads < nitems) cp_async16(sbase + ldst[j], lsrc[j] + k0);
    };
    bool ok = true;
    int issued = 0;                                        // stages committed to MMA
    // prologue: kOzLead stages in flight (one commit group each)
    for (int t = 0; t < kOzLead; ++t) {
        if (t < nk) load(t);
        asm volatile("cp.async.commit_group;" ::: "memory");
    }
    for (int t = 0; t < nk && ok; ++t) {
        const int slot = t % kOzStages;
        asm volatile("cp.async.wait_group %0;" ::"n"(kOzLead - 1) : "memory");   // stage t landed
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        // the slot refilled below with stage t + kOzLead is the one the MMAs of
        // stage t - kOzMmaAhead read: wait for them here, so that one barrier
        // per stage covers both (every copy of stage t landed, the slot free)
        if (t >= kOzMmaAhead && t + kOzLead < nk)
            ok = mbar_wait(smem_u32(&mbar[(t - kOzMmaAhead) % kOzStages]),
                           ((t - kOzMmaAhead) / kOzStages) & 1);
        ok = __syncthreads_and(ok);                          // uniform exit on a timeout
        if (!ok) break;
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t sa = smem_u32(smem + slot * stage_bytes);
            const uint32_t sb = sa + s * a_tile;
            // one MMA per A slice p against B slices q0.. side by side (N up to
            // 5 x 48): column block q of D lands on level p + q's TMEM region,
            // so each A slice is read once per K step.  The first step
            // initialises every level (p = 0 covers them all); the exact levels
            // are cleared again after each drain.
            for (int p = 0; p < s; ++p) {
                for (int q0 = 0; q0 < s - p; q0 += kOzGroup) {
                    const int cnt = min(kOzGroup, s - p - q0);
                    const uint32_t dcol = tmem + (uint32_t)((p + q0) * kOzN);
                    const uint64_t ad = smem_desc(sa + p * a_tile, 128, 256);
                    const uint64_t bd = smem_desc(sb + q0 * b_tile, 128, 256);
                    const uint32_t acc = (t == 0 && p == 0) ? 0u : 1u;
                    asm volatile(
                        "{\n\t.reg .pred pa;\n\tsetp.ne.b32 pa, %4, 0;\n\t"
                        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, pa;\n\t}" ::"r"(dcol),
                        "l"(ad), "l"(bd), "r"(bf16_idesc(kOzM, cnt * kOzN)), "r"(acc));
                }
            }
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    smem_u32(&mbar[slot]))
                : "memory");
        }
        ++issued;
        if (t + kOzLead < nk) load(t + kOzLead);
        asm volatile("cp.async.commit_group;" ::: "memory");
        // ---- end of a 256-element chunk (or of K): drain the exact levels
        if ((t % kOzChunkStages) == kOzChunkStages - 1 || t == nk - 1) {
            ok = mbar_wait(smem_u32(&mbar[slot]), (t / kOzStages) & 1);
            ok = __syncthreads_and(ok);
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (ok) {
#pragma unroll
                for (int L = 0; L < kOzExact; ++L) {
                    if (L >= s) break;
#pragma unroll
                    for (int g = 0; g < kOzN / 2 / 8; ++g) {
                        uint32_t v[8];
                        tmem_ld8(lane_base + (uint32_t)(L * kOzN + colhalf * (kOzN / 2) + g * 8), v);
                        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                        for (int c = 0; c < 8; ++c)
                            exact[L][g * 8 + c] += __float2int_rn(__uint_as_float(v[c]));
                        const uint32_t z = 0u;
                        asm volatile(
                            "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %1, %1, %1, %1, %1, %1, %1};" ::"r"(
                                lane_base + (uint32_t)(L * kOzN + colhalf * (kOzN / 2) + g * 8)),
                            "r"(z)
                            : "memory");
                    }
                }
                asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncthreads();
        }
    }
    // copies still in flight (a timeout exit) land before the CTA ends
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    if (!ok && issued > 0) {
        // let the queued MMAs finish (bounded) before TMEM is released
        const int last = issued - 1;
        (void)mbar_wait(smem_u32(&mbar[last % kOzStages]), (last / kOzStages) & 1);
    }
    if (!ok && tid == 0) atomicOr(err, 16);
    __syncthreads();
    if (ok) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int row = row0 + quarter * 32 + lane;
        const double sgm = (row < Mrows) ? sg[row] : 0.0;
        double acc[kOzN / 2];
#pragma unroll
        for (int c = 0; c < kOzN / 2; ++c) acc[c] = 0.0;
        for (int L = s - 1; L >= kOzExact; --L) {          // small levels, FP32 in TMEM
            const double scale = ldexp(1.0, -7 * (L + 2));
#pragma unroll
            for (int g = 0; g < kOzN / 2 / 8; ++g) {
                uint32_t v[8];
                tmem_ld8(lane_base + (uint32_t)(L * kOzN + colhalf * (kOzN / 2) + g * 8), v);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int c = 0; c < 8; ++c) acc[g * 8 + c] = fma((double)__uint_as_float(v[c]), scale, acc[g * 8 + c]);
            }
        }
#pragma unroll
        for (int L = kOzExact - 1; L >= 0; --L) {
            if (L >= s) continue;
            const double scale = ldexp(1.0, -7 * (L + 2));
#pragma unroll
            for (int c = 0; c < kOzN / 2; ++c) acc[c] = fma((double)exact[L][c], scale, acc[c]);
        }
        if (row < Mrows) {
#pragma unroll
            for (int c = 0; c < kOzN / 2; ++c) {
                const int cc = col0 + colhalf * (kOzN / 2) + c;    // real column of W'
                const int j = cc >> 1;
                if (j < ncols_complex) {
                    // column j belongs to block j / mb (one subspace block per contour)
                    const int blk = j / mb, jj = j - blk * mb;
                    double* dst = reinterpret_cast<double*>(Wt + blk * w_block_stride + row +
                                                            (int64_t)jj * ldw) + (cc & 1);
                    *dst = sgm * tau[j] * acc[c];
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kTmemCols));
    }
}

// ---------------------------------------------------------------------------
// digit slices
// ---------------------------------------------------------------------------
// sigma_i = 2^e with max_k |A'_ik| < 2^e (1 for a zero row).  A CTA of 32 x 8
// threads takes 32 rows; its 8 thread rows stride over K (coalesced along the
// rows), then reduce through shared memory.
__global__ void row_scale_kernel(int64_t M, int64_t K, const double2* __restrict__ A, int64_t lda,
                                 double* __restrict__ sigma, int64_t Mrows_pad) {
    __shared__ double red[8][33];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int64_t i = blockIdx.x * (int64_t)32 + tx;
    double mx = 0.0;
    if (i < M)
        for (int64_t k = ty; k < K; k += 8) {
            const double2 a = A[i + k * lda];
            mx = fmax(mx, fmax(fabs(a.x), fabs(a.y)));
        }
    red[ty][tx] = mx;
    __syncthreads();
    if (ty == 0 && i < Mrows_pad) {
        for (int q = 1; q < 8; ++q) mx = fmax(mx, red[q][tx]);
        int e = 0;
        if (mx > 0.0) frexp(mx, &e);   // mx = f 2^e, f in [0.5, 1)
        sigma[i] = (mx > 0.0) ? ldexp(1.0, e) : 1.0;
    }
}

// The s base-128 digits of r (|r| < 1), truncated toward zero, given
// r2 = r * 2^(7 s) (exact: a power-of-two scaling): |r2| < 2^(7 s) <= 2^56 is
// converted to an integer once (truncation toward zero), and digit p is bits
// 7 (s-1-p) .. 7 (s-p) - 1 of its magnitude, with r's sign.  The same digits as
// s steps of r <- 128 r, t = trunc(r), r <- r - t (all exact), without FP64
// arithmetic beyond the scaling.
__device__ __forceinline__ void digits_scaled(double r2, int s, float* d) {
    const long long q = (long long)r2;
    const unsigned long long u = (unsigned long long)(q < 0 ? -q : q);
    const float sg = q < 0 ? -1.0f : 1.0f;
    for (int p = 0; p < s; ++p) d[p] = sg * (float)(int)((u >> (7 * (s - 1 - p))) & 127ull);
}

// A' slices [slice][Mpad][Kp] (bf16) of an M x K block A (leading dimension
// lda): K index k -> Re A[i,k], K + k -> Im A[i,k].
// Block 32 x 8 handles 32 rows x 32 complex columns through shared memory.
__global__ void split_rows_kernel(int64_t M, int64_t K, int s, const double2* __restrict__ A,
                                  int64_t lda, const double* __restrict__ sigma,
                                  __nv_bfloat16* __restrict__ out, int64_t slice_stride, int64_t Kp) {
    __shared__ float tile[kOzMaxSlices][2][32][33];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int64_t i0 = (int64_t)blockIdx.x * 32, k0 = (int64_t)blockIdx.y * 32;
    const int64_t i = i0 + tx;
    const double inv = (i < M) ? 1.0 / sigma[i] : 0.0;     // exact: sigma is a power of 2
    const double sc = ldexp(inv, 7 * s);
    for (int kk = ty; kk < 32; kk += 8) {
        const int64_t k = k0 + kk;
        double2 a = make_double2(0.0, 0.0);
        if (i < M && k < K) a = A[i + k * lda];
        float dr[kOzMaxSlices], di[kOzMaxSlices];
        digits_scaled(a.x * sc, s, dr);
        digits_scaled(a.y * sc, s, di);
        for (int p = 0; p < s; ++p) { tile[p][0][tx][kk] = dr[p]; tile[p][1][tx][kk] = di[p]; }
    }
    __syncthreads();
    for (int rr = ty; rr < 32; rr += 8) {
        const int64_t row = i0 + rr;
        const int64_t k = k0 + tx;
        if (k >= K) continue;
        for (int p = 0; p < s; ++p) {
            __nv_bfloat16* o = out + p * slice_stride + row * Kp;
            o[k] = __float2bfloat16_rn(tile[p][0][rr][tx]);
            o[K + k] = __float2bfloat16_rn(tile[p][1][rr][tx]);
        }
    }
}

// Q' slices for complex column j of a K x N block Q (leading dimension ldq):
// rows 2j, 2j+1 of [slice][Npad][Kp], and tau_j.
__global__ void split_cols_kernel(int64_t K, int s, const double2* __restrict__ Q, int64_t ldq,
                                  double* __restrict__ tau, __nv_bfloat16* __restrict__ out,
                                  int64_t slice_stride, int64_t Kp) {
    __shared__ double red[32];
    const int j = blockIdx.x;
    const double2* q = Q + (int64_t)j * ldq;
    double mx = 0.0;
    for (int64_t k = threadIdx.x; k < K; k += blockDim.x)
        mx = fmax(mx, fmax(fabs(q[k].x), fabs(q[k].y)));
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = fmax(t, red[w]);
        int e = 0;
        if (t > 0.0) frexp(t, &e);
        red[0] = (t > 0.0) ? ldexp(1.0, e) : 1.0;
        tau[j] = red[0];
    }
    __syncthreads();
    const double sc = ldexp(1.0 / red[0], 7 * s);
    for (int64_t k = threadIdx.x; k < K; k += blockDim.x) {
        float dr[kOzMaxSlices], di[kOzMaxSlices];
        digits_scaled(q[k].x * sc, s, dr);
        digits_scaled(q[k].y * sc, s, di);
        for (int p = 0; p < s; ++p) {
            __nv_bfloat16* r0 = out + p * slice_stride + (int64_t)(2 * j) * Kp;
            __nv_bfloat16* r1 = r0 + Kp;
            r0[k] = __float2bfloat16_rn(dr[p]);
            r0[K + k] = __float2bfloat16_rn(-di[p]);
            r1[k] = __float2bfloat16_rn(di[p]);
            r1[K + k] = __float2bfloat16_rn(dr[p]);
        }
    }
}

}  // namespace

OzakiLayout ozaki_layout(int64_t n, int m, int s) {
    OzakiLayout L;
    L.s = s;
    L.Mpad = (n + kOzM - 1) / kOzM * kOzM;
    L.Kp = (2 * n + kOzBK - 1) / kOzBK * kOzBK;
    L.Npad = (2 * (int64_t)m + kOzN - 1) / kOzN * kOzN;
    L.a_slice = L.Mpad * L.Kp;             // elements
    L.a_term = L.a_slice * s;
    L.b_slice = L.Npad * L.Kp;
    return L;
}

bool ozaki_supported(int64_t n, int s) {
    // int32 running sums of the exact levels: 3 pairs * 2n * 127^2 < 2^31
    return s >= 1 && s <= kOzMaxSlices && 3.0 * 2.0 * n * 127.0 * 127.0 < 2147483647.0;
}

size_t ozaki_elem_bytes() { return sizeof(__nv_bfloat16); }

cudaError_t ozaki_split_A(cudaStream_t st, int64_t n, int s, const double2* A, double* sigma,
                          void* slices, const OzakiLayout& L) {
    cudaError_t e = cudaMemsetAsync(slices, 0, (size_t)L.a_term * sizeof(__nv_bfloat16), st);
    if (e != cudaSuccess) return e;
    note_launch();
    row_scale_kernel<<<(unsigned)((L.Mpad + 31) / 32), dim3(32, 8), 0, st>>>(n, n, A, n, sigma, L.Mpad);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    dim3 g((unsigned)((n + 31) / 32), (unsigned)((n + 31) / 32));
    note_launch();
    split_rows_kernel<<<g, dim3(32, 8), 0, st>>>(n, n, s, A, n, sigma,
                                                  static_cast<__nv_bfloat16*>(slices), L.a_slice,
                                                  L.Kp);
    return cudaGetLastError();
}

cudaError_t ozaki_split_Q(cudaStream_t st, int64_t n, int m, int s, const double2* Q, double* tau,
                          void* slices, const OzakiLayout& L) {
    note_launch();
    split_cols_kernel<<<m, 256, 0, st>>>(n, s, Q, n, tau, static_cast<__nv_bfloat16*>(slices),
                                         L.b_slice, L.Kp);
    return cudaGetLastError();
}

cudaError_t ozaki_gemm(cudaStream_t st, int64_t n, int m, int mb, int wterms, const OzakiLayout& L,
                       int nterms, const void* Aslices, const double* sigma, const void* Qslices,
                       const double* tau, double2* W, const int* term_slot, int* err,
                       const int* active) {
    static std::atomic<bool> attr_done{false};   // idempotent setup; atomic for concurrent handles
    const int s = L.s;
    const int smem = kOzStages * s * (kOzM + kOzN) * kOzBK * 2;
    if (!attr_done) {
        cudaError_t e = cudaFuncSetAttribute(ozaki_bf16_gemm_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             kOzStages * kOzMaxSlices * (kOzM + kOzN) * kOzBK * 2);
        if (e != cudaSuccess) return e;
        attr_done = true;
    }
    dim3 grid((unsigned)(L.Npad / kOzN), (unsigned)(L.Mpad / kOzM), (unsigned)nterms);
    note_launch();
    ozaki_bf16_gemm_kernel<<<grid, kOzThreads, smem, st>>>(
        s, (int)n, (int)L.Kp, static_cast<const __nv_bfloat16*>(Aslices), L.a_slice, L.a_term,
        sigma, L.Mpad, static_cast<const __nv_bfloat16*>(Qslices), L.b_slice, tau, W, n, n * mb, mb,
        (int64_t)wterms * n * mb, term_slot, m, err, active, 0, 0);
    return cudaGetLastError();
}

// General product on the same kernel: one "term" A (M x K), B (K x N).
namespace {
struct OzGeneralLayout {
    OzakiLayout L;
    size_t a_bytes, sigma_off, b_off, b_bytes, tau_off, slot_off, total;
};
OzGeneralLayout oz_general_layout(int64_t M, int K, int N, int s) {
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    OzGeneralLayout G;
    G.L.s = s;
    G.L.Mpad = (M + kOzM - 1) / kOzM * kOzM;
    G.L.Kp = (2 * (int64_t)K + kOzBK - 1) / kOzBK * kOzBK;
    G.L.Npad = (2 * (int64_t)N + kOzN - 1) / kOzN * kOzN;
    G.L.a_slice = G.L.Mpad * G.L.Kp;
    G.L.a_term = G.L.a_slice * s;
    G.L.b_slice = G.L.Npad * G.L.Kp;
    size_t o = 0;
    G.a_bytes = (size_t)G.L.a_term * sizeof(__nv_bfloat16);
    o = al(G.a_bytes);
    G.sigma_off = o; o = al(o + (size_t)G.L.Mpad * sizeof(double));
    G.b_off = o;
    G.b_bytes = (size_t)G.L.b_slice * s * sizeof(__nv_bfloat16);
    o = al(o + G.b_bytes);
    G.tau_off = o; o = al(o + (size_t)N * sizeof(double));
    G.slot_off = o; o = al(o + sizeof(int));
    G.total = o;
    return G;
}
}  // namespace

size_t ozaki_general_work_bytes(int64_t M, int K, int N, int s) {
    return oz_general_layout(M, K, N, s).total;
}

cudaError_t ozaki_gemm_general(cudaStream_t st, int64_t M, int K, int N, const double2* A,
                               int64_t lda, const double2* B, int64_t ldb, double2* C, int64_t ldc,
                               int s, void* work, int* err) {
    if (M <= 0 || K <= 0 || N <= 0) return cudaSuccess;
    if (!ozaki_supported(K, s)) return cudaErrorInvalidValue;
    const OzGeneralLayout G = oz_general_layout(M, K, N, s);
    unsigned char* w = static_cast<unsigned char*>(work);
    __nv_bfloat16* Asl = reinterpret_cast<__nv_bfloat16*>(w);
    double* sigma = reinterpret_cast<double*>(w + G.sigma_off);
    __nv_bfloat16* Bsl = reinterpret_cast<__nv_bfloat16*>(w + G.b_off);
    double* tau = reinterpret_cast<double*>(w + G.tau_off);
    int* slot = reinterpret_cast<int*>(w + G.slot_off);
    // the K padding of both operands must read as zero
    cudaError_t e;
    if ((e = cudaMemsetAsync(Asl, 0, G.a_bytes, st)) != cudaSuccess ||
        (e = cudaMemsetAsync(Bsl, 0, G.b_bytes, st)) != cudaSuccess ||
        (e = cudaMemsetAsync(slot, 0, sizeof(int), st)) != cudaSuccess)
        return e;
    note_launch();
    row_scale_kernel<<<(unsigned)((G.L.Mpad + 31) / 32), dim3(32, 8), 0, st>>>(M, K, A, lda, sigma, G.L.Mpad);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    note_launch();
    dim3 g((unsigned)((M + 31) / 32), (unsigned)((K + 31) / 32));
    split_rows_kernel<<<g, dim3(32, 8), 0, st>>>(M, K, s, A, lda, sigma, Asl, G.L.a_slice, G.L.Kp);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    note_launch();
    split_cols_kernel<<<N, 256, 0, st>>>(K, s, B, ldb, tau, Bsl, G.L.b_slice, G.L.Kp);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    static std::atomic<bool> attr_done{false};
    const int smem = kOzStages * s * (kOzM + kOzN) * kOzBK * 2;
    if (!attr_done) {
        e = cudaFuncSetAttribute(ozaki_bf16_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kOzStages * kOzMaxSlices * (kOzM + kOzN) * kOzBK * 2);
        if (e != cudaSuccess) return e;
        attr_done = true;
    }
    dim3 grid((unsigned)(G.L.Npad / kOzN), (unsigned)(G.L.Mpad / kOzM), 1u);
    note_launch();
    ozaki_bf16_gemm_kernel<<<grid, kOzThreads, smem, st>>>(
        s, (int)M, (int)G.L.Kp, Asl, G.L.a_slice, G.L.a_term, sigma, G.L.Mpad, Bsl, G.L.b_slice,
        tau, C, ldc, 0, N, 0, slot, N, err, nullptr, 0, 0);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Projections G = Q^H W (Step 1) as C = W^H Q on the same kernel, split over K.
// The product is short and wide in K (m x n times n x T m), so its tiles alone
// would give a dozen CTAs: K is split across blockIdx.z and the FP64 partial
// products are summed in a fixed order.
// ---------------------------------------------------------------------------
namespace {

// Row i of A' = W^H (i < NT; column i of W, K x NT col-major, ld ldw): its
// scale sigma_i (power of two above the largest |Re|, |Im|) and its s digit
// slices, Re conj(w) at k, Im conj(w) at K + k, zeros in the K padding; rows
// NT .. Mpad-1 are written as zeros.  One CTA per row.
__global__ void split_rows_conjT_kernel(int64_t K, int NT, int s, const double2* __restrict__ Wm,
                                        int64_t ldw, double* __restrict__ sigma,
                                        __nv_bfloat16* __restrict__ out, int64_t slice_stride,
                                        int64_t Kp) {
    __shared__ double red[32];
    const int i = blockIdx.x;
    const bool live = i < NT;
    const double2* w = Wm + (int64_t)(live ? i : 0) * ldw;
    double mx = 0.0;
    if (live)
        for (int64_t k = threadIdx.x; k < K; k += blockDim.x)
            mx = fmax(mx, fmax(fabs(w[k].x), fabs(w[k].y)));
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t = fmax(t, red[q]);
        int e = 0;
        if (t > 0.0) frexp(t, &e);
        red[0] = (t > 0.0) ? ldexp(1.0, e) : 1.0;
        sigma[i] = red[0];
    }
    __syncthreads();
    const double sc = ldexp(1.0 / red[0], 7 * s);
    for (int64_t k = threadIdx.x; k < Kp; k += blockDim.x) {
        float d[kOzMaxSlices];
        const bool re = k < K, im = k >= K && k < 2 * K;
        double v = 0.0;
        if (live && re) v = w[k].x * sc;
        if (live && im) v = -w[k - K].y * sc;
        digits_scaled(v, s, d);
        for (int p = 0; p < s; ++p) out[p * slice_stride + (int64_t)i * Kp + k] = __float2bfloat16_rn(d[p]);
    }
}

// G (m x NT, col-major, ld m) = conj of the sum over the splits of the partial
// products P_z = (W^H Q)_z (NT x m, col-major, ld NT), in split order.
__global__ void splitk_reduce_conjT_kernel(int NT, int m, int S, const double2* __restrict__ P,
                                           double2* __restrict__ G) {
    const int64_t total = (int64_t)NT * m;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        double2 acc = make_double2(0.0, 0.0);
        for (int z = 0; z < S; ++z) {
            const double2 v = P[(int64_t)z * total + e];
            acc.x += v.x;
            acc.y += v.y;
        }
        const int64_t i = e % NT, j = e / NT;
        G[j + i * m] = make_double2(acc.x, -acc.y);
    }
}

// Digit slices of both operands of the projections.  Eight slices, one more
// than the A_t Q product uses: G = Q^H W is a product of unit columns with
// cancellation in its off-diagonal entries, and with seven slices its error
// (~1.5e-13 relative to ||G||_F at n = 4096, m0 = 96) is two orders above an
// FP64 product's; the eighth slice puts it back at the FP64 level.
constexpr int kOzProjSlices = kOzMaxSlices;

struct OzProjLayout {
    int64_t Mpad, a_slice;
    int S, stages;                 // K splits and K stages per split
    size_t sigma_off, slot_off, qsl_off, tau_off, part_off, total;
};
OzProjLayout oz_proj_layout(int64_t n, int NT, int m, int s) {
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const OzakiLayout LQ = ozaki_layout(n, m, s);
    OzProjLayout P;
    P.Mpad = ((int64_t)NT + kOzM - 1) / kOzM * kOzM;
    P.a_slice = P.Mpad * LQ.Kp;
    const int nk = (int)(LQ.Kp / kOzBK);
    const int tiles = (int)((LQ.Npad / kOzN) * (P.Mpad / kOzM));
    // about one CTA per SM (152), each at least one 256-element drain chunk of K
    int S = std::max(1, 152 / std::max(tiles, 1));
    S = std::min(S, std::max(1, nk / kOzChunkStages));
    P.stages = (nk + S - 1) / S;
    P.S = (nk + P.stages - 1) / P.stages;
    size_t o = al((size_t)P.a_slice * s * sizeof(__nv_bfloat16));
    P.sigma_off = o; o = al(o + (size_t)P.Mpad * sizeof(double));
    P.slot_off = o;  o = al(o + sizeof(int));
    P.qsl_off = o;   o = al(o + (size_t)LQ.b_slice * s * sizeof(__nv_bfloat16));
    P.tau_off = o;   o = al(o + (size_t)m * sizeof(double));
    P.part_off = o;  o = al(o + (size_t)P.S * NT * m * sizeof(double2));
    P.total = o;
    return P;
}

}  // namespace

size_t ozaki_project_work_bytes(int64_t n, int NT, int m) {
    return oz_proj_layout(n, NT, m, kOzProjSlices).total;
}

cudaError_t ozaki_project(cudaStream_t st, int64_t n, int NT, int m, const double2* Wm, int64_t ldw,
                          const double2* Q, int64_t ldq, double2* G, void* work, int* err) {
    const int s = kOzProjSlices;
    if (n <= 0 || NT <= 0 || m <= 0) return cudaSuccess;
    if (!ozaki_supported(n, s)) return cudaErrorInvalidValue;
    const OzakiLayout LQ = ozaki_layout(n, m, s);
    const OzProjLayout P = oz_proj_layout(n, NT, m, s);
    unsigned char* w = static_cast<unsigned char*>(work);
    __nv_bfloat16* Asl = reinterpret_cast<__nv_bfloat16*>(w);
    double* sigma = reinterpret_cast<double*>(w + P.sigma_off);
    int* slot = reinterpret_cast<int*>(w + P.slot_off);
    __nv_bfloat16* Qsl = reinterpret_cast<__nv_bfloat16*>(w + P.qsl_off);
    double* tau = reinterpret_cast<double*>(w + P.tau_off);
    double2* part = reinterpret_cast<double2*>(w + P.part_off);
    cudaError_t e;
    if ((e = cudaMemsetAsync(slot, 0, sizeof(int), st)) != cudaSuccess) return e;
    // B' = digit slices of Q (the K padding and the padded columns read as zero)
    if ((e = cudaMemsetAsync(Qsl, 0, (size_t)LQ.b_slice * s * sizeof(__nv_bfloat16), st)) != cudaSuccess)
        return e;
    note_launch();
    split_cols_kernel<<<m, 256, 0, st>>>(n, s, Q, ldq, tau, Qsl, LQ.b_slice, LQ.Kp);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    note_launch();
    split_rows_conjT_kernel<<<(unsigned)P.Mpad, 256, 0, st>>>(n, NT, s, Wm, ldw, sigma, Asl,
                                                              P.a_slice, LQ.Kp);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    static std::atomic<bool> attr_done{false};
    const int smem = kOzStages * s * (kOzM + kOzN) * kOzBK * 2;
    if (!attr_done) {
        e = cudaFuncSetAttribute(ozaki_bf16_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kOzStages * kOzMaxSlices * (kOzM + kOzN) * kOzBK * 2);
        if (e != cudaSuccess) return e;
        attr_done = true;
    }
    dim3 grid((unsigned)(LQ.Npad / kOzN), (unsigned)(P.Mpad / kOzM), (unsigned)P.S);
    note_launch();
    ozaki_bf16_gemm_kernel<<<grid, kOzThreads, smem, st>>>(
        s, NT, (int)LQ.Kp, Asl, P.a_slice, 0, sigma, 0, Qsl, LQ.b_slice, tau, part, NT, 0, m, 0, slot,
        m, err, nullptr, P.stages, (int64_t)NT * m);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    note_launch();
    splitk_reduce_conjT_kernel<<<(unsigned)std::min<int64_t>(((int64_t)NT * m + 255) / 256, 1024), 256, 0,
                                 st>>>(NT, m, P.S, part, G);
    return cudaGetLastError();
}

}  // namespace fnl
