// Complex64 update C -= A B on the TF32 tensor cores (tcgen05.mma.kind::tf32)
// with FP32-level accuracy: the trailing updates of the node LU factorisations
// and the block forward / back substitutions of the node solves (Step 4 of
// Algorithm 1 in its mixed-precision form, Sec. 4).
//
// Each FP32 operand entry is split into two TF32 parts, x = x_hi + x_lo with
// x_hi = rn_tf32(x) and x_lo = rn_tf32(x - x_hi) (the difference is exact in
// FP32).  The product keeps a_hi b_hi + a_hi b_lo + a_lo b_hi; the dropped
// a_lo b_lo and the rounding of the low parts are each below 2^-24 |a| |b|, the
// size of one FP32 rounding, so three TF32 products give an FP32-accurate
// product with FP32 accumulation in TMEM.
//
// Complex arithmetic by a real embedding: row i of A' is
// (Re a_i0, Im a_i0, Re a_i1, Im a_i1, ...) (length 2k), column 2j of B' is
// (Re b_0j, -Im b_0j, Re b_1j, -Im b_1j, ...) and column 2j+1 is
// (Im b_0j, Re b_0j, ...), so (A' B')[i, 2j] = Re (AB)_ij and [i, 2j+1] = Im.
// A complex64 entry of a column-major A is exactly one (Re, Im) pair of a row
// of A', and one entry of B fills one pair in each of two rows of B'.
//
// CTA: 128 threads and one 128 x BN complex tile of C, held in TMEM as 128
// lanes x 2 BN FP32 columns.  K advances 8 complex (16 real) entries per stage
// through a 2-stage shared-memory ring: the threads load a stage, split it and
// store the four parts (A_hi, A_lo, B_hi, B_lo) in the canonical K-major
// SWIZZLE_NONE layout (8-row x 16-byte core matrices, the four K core matrices
// of a row group side by side: LBO 128 B, SBO 512 B); thread 0 issues six
// MMAs (M = 128, N = 2 BN, K = 8) per stage and commits the stage to its
// mbarrier, which frees the slot two stages later (two stages rather than
// three: the kernel is latency-bound, and the smaller ring fits three CTAs per
// SM instead of two).  The epilogue reads TMEM
// with lane = row of C and updates C column by column (coalesced along rows).
#include "internal.h"
#include "tc_common.cuh"

namespace fnl {
namespace {
using namespace tc;

constexpr int kTcM = 128;                      // rows of C per CTA (TMEM lanes)
constexpr int kTcBK = 8;                       // complex K entries per stage
constexpr int kTcStages = 2;
constexpr int kTcThreads = 128;
constexpr uint32_t kTcTmemCols = 128;
constexpr int kTcAtile = kTcM * 2 * kTcBK * 4;  // bytes of one A part (8 KB)

// Instruction descriptor: kind::tf32, D = F32, A = B = TF32, both K-major.
__host__ __device__ constexpr uint32_t tf32_idesc(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

// x rounded to TF32 (11 significant bits), low 13 bits cleared
__device__ __forceinline__ float tf32_rn(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r & 0xFFFFE000u);
}

// byte offset of the real pair (2 kc, 2 kc + 1) of row r in a 16-real-K tile
__device__ __forceinline__ uint32_t pair_off(int r, int kc) {
    return (uint32_t)((r >> 3) * 512 + (kc >> 1) * 128 + (r & 7) * 16 + (kc & 1) * 8);
}

__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred pa;\n\tsetp.ne.b32 pa, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, pa;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

// One CTA's 128 x BN tile (blockIdx.x, blockIdx.y) of C -= A B for one matrix.
template <int BN>
__device__ __forceinline__ void cgemm_body(int m, int n, int k, const float2* __restrict__ A,
                                           int64_t lda, const float2* __restrict__ B, int64_t ldb,
                                           float2* __restrict__ C, int64_t ldc,
                                           int* __restrict__ err) {
    constexpr int NR = 2 * BN;                   // real columns of the tile
    constexpr int kBtile = NR * 2 * kTcBK * 4;   // bytes of one B part
    constexpr int kStage = 2 * kTcAtile + 2 * kBtile;
    constexpr int kAIt = (kTcM / 16) * (kTcBK / 2) / 4;   // A loads per thread and stage
    constexpr int kBIt = 2 * (BN / 8) / 4;                 // B loads per thread and stage
    static_assert(BN % 16 == 0 && NR <= 256, "tile width");

    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t mbar[kTcStages];
    __shared__ uint32_t s_tmem;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int row0 = blockIdx.x * kTcM, col0 = blockIdx.y * BN;

    if (tid == 0) {
        for (int q = 0; q < kTcStages; ++q) mbar_init(smem_u32(&mbar[q]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&s_tmem)),
                     "r"(kTcTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s_tmem;

    // the C tile into L2 while the K loop runs, so that the epilogue's
    // read-modify-write hits in L2 (up to 9 lines of 128 bytes per column)
    if (row0 < m) {
        const int rows = min(kTcM, m - row0);
        for (int idx = tid; idx < BN * 9; idx += kTcThreads) {
            const int j = idx / 9, t = idx - j * 9;
            if (col0 + j >= n) continue;
            const char* p0 = reinterpret_cast<const char*>(C + row0 + (int64_t)(col0 + j) * ldc);
            const uintptr_t l0 = reinterpret_cast<uintptr_t>(p0) >> 7;
            const uintptr_t l1 = (reinterpret_cast<uintptr_t>(p0) + (uintptr_t)rows * 8 - 1) >> 7;
            if (l0 + t <= l1)
                asm volatile("prefetch.global.L2 [%0];" ::"l"((l0 + t) << 7));
        }
    }

    // A: a warp step covers 16 rows x 2 complex k; lanes 0-7 / 8-15 take the
    // even / odd k of rows 0-7, lanes 16-31 the same for rows 8-15, so each
    // 16-lane half stores 128 distinct bytes (no bank conflict).
    const int a_r = (lane & 7) + 8 * (lane >> 4), a_k = (lane >> 3) & 1;
    // B: a warp step covers 4 complex k x 8 columns (32 contiguous bytes of a
    // column per 4 lanes); lanes 16-31 store their odd row first, so every
    // store instruction covers the 8 row slots of a core matrix.
    const int b_k = lane & 3, b_j = lane >> 2;
    const bool b_sw = (lane >> 4) & 1;
    float2 ra[kAIt], rb[kBIt];

    auto load = [&](int t) {
        const int k0 = t * kTcBK;
#pragma unroll
        for (int q = 0; q < kAIt; ++q) {
            const int it = warp + 4 * q;
            const int r = (it & 7) * 16 + a_r, kc = (it >> 3) * 2 + a_k;
            const int gr = row0 + r, gk = k0 + kc;
            ra[q] = (gr < m && gk < k) ? __ldg(A + gr + (int64_t)gk * lda) : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int q = 0; q < kBIt; ++q) {
            const int it = warp + 4 * q;
            const int kc = (it & 1) * 4 + b_k, j = (it >> 1) * 8 + b_j;
            const int gk = k0 + kc, gc = col0 + j;
            rb[q] = (gk < k && gc < n) ? __ldg(B + gk + (int64_t)gc * ldb) : make_float2(0.f, 0.f);
        }
    };
    auto store = [&](int slot) {
        unsigned char* ahi = smem + slot * kStage;
        unsigned char* alo = ahi + kTcAtile;
        unsigned char* bhi = ahi + 2 * kTcAtile;
        unsigned char* blo = bhi + kBtile;
#pragma unroll
        for (int q = 0; q < kAIt; ++q) {
            const int it = warp + 4 * q;
            const uint32_t off = pair_off((it & 7) * 16 + a_r, (it >> 3) * 2 + a_k);
            const float2 v = ra[q];
            const float hr = tf32_rn(v.x), hm = tf32_rn(v.y);
            *reinterpret_cast<float2*>(ahi + off) = make_float2(hr, hm);
            *reinterpret_cast<float2*>(alo + off) = make_float2(tf32_rn(v.x - hr), tf32_rn(v.y - hm));
        }
#pragma unroll
        for (int q = 0; q < kBIt; ++q) {
            const int it = warp + 4 * q;
            const int kc = (it & 1) * 4 + b_k, j = (it >> 1) * 8 + b_j;
            const float2 v = rb[q];
            const float hr = tf32_rn(v.x), hm = tf32_rn(v.y);
            const float lr = tf32_rn(v.x - hr), lm = tf32_rn(v.y - hm);
            // row 2j: (Re, -Im); row 2j + 1: (Im, Re)
            const float2 h0 = make_float2(hr, -hm), h1 = make_float2(hm, hr);
            const float2 l0 = make_float2(lr, -lm), l1 = make_float2(lm, lr);
            const uint32_t o0 = pair_off(2 * j, kc), o1 = pair_off(2 * j + 1, kc);
            const uint32_t oA = b_sw ? o1 : o0, oB = b_sw ? o0 : o1;
            *reinterpret_cast<float2*>(bhi + oA) = b_sw ? h1 : h0;
            *reinterpret_cast<float2*>(bhi + oB) = b_sw ? h0 : h1;
            *reinterpret_cast<float2*>(blo + oA) = b_sw ? l1 : l0;
            *reinterpret_cast<float2*>(blo + oB) = b_sw ? l0 : l1;
        }
    };

    const uint32_t idesc = tf32_idesc(kTcM, NR);
    const int nk = (k + kTcBK - 1) / kTcBK;
    bool ok = true;
    int issued = 0;
    load(0);
    for (int t = 0; t < nk; ++t) {
        const int slot = t % kTcStages;
        if (t >= kTcStages) ok = mbar_wait(smem_u32(&mbar[slot]), ((t / kTcStages) - 1) & 1);
        ok = __syncthreads_and(ok);                // uniform exit on a timeout
        if (!ok) break;
        store(slot);
        if (t + 1 < nk) load(t + 1);              // in flight while the MMAs run
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t base = smem_u32(smem + slot * kStage);
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) {       // two K = 8 (32-byte) steps
                const uint64_t ah = smem_desc(base + ks * 256, 128, 512);
                const uint64_t al = smem_desc(base + kTcAtile + ks * 256, 128, 512);
                const uint64_t bh = smem_desc(base + 2 * kTcAtile + ks * 256, 128, 512);
                const uint64_t bl = smem_desc(base + 2 * kTcAtile + kBtile + ks * 256, 128, 512);
                mma_tf32(tmem, al, bh, idesc, (t > 0 || ks > 0) ? 1u : 0u);
                mma_tf32(tmem, ah, bl, idesc, 1u);
                mma_tf32(tmem, ah, bh, idesc, 1u);
            }
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    smem_u32(&mbar[slot]))
                : "memory");
        }
        ++issued;
    }
    // all MMAs complete once the last committed stage has arrived (also on the
    // timeout path, so that TMEM is released only after its writers finished)
    bool done = true;
    if (issued > 0)
        done = mbar_wait(smem_u32(&mbar[(issued - 1) % kTcStages]), ((issued - 1) / kTcStages) & 1);
    ok = __syncthreads_and(ok && done);
    if (!ok && tid == 0) atomicOr(err, 16);
    if (ok && issued > 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int row = row0 + warp * 32 + lane;
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
        for (int g = 0; g < NR / 32; ++g) {        // 16 complex columns per group
            uint32_t v[32];
#pragma unroll
            for (int c = 0; c < 4; ++c) tmem_ld8(taddr + (uint32_t)(g * 32 + c * 8), v + c * 8);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (row < m) {
                float2 cv[16];
#pragma unroll
                for (int jj = 0; jj < 16; ++jj) {
                    const int j = col0 + g * 16 + jj;
                    if (j < n) cv[jj] = C[row + (int64_t)j * ldc];
                }
#pragma unroll
                for (int jj = 0; jj < 16; ++jj) {
                    const int j = col0 + g * 16 + jj;
                    if (j < n)
                        C[row + (int64_t)j * ldc] =
                            make_float2(cv[jj].x - __uint_as_float(v[2 * jj]),
                                        cv[jj].y - __uint_as_float(v[2 * jj + 1]));
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kTcTmemCols));
    }
}

template <int BN>
__global__ void __launch_bounds__(kTcThreads, 3) cgemm_tf32x3_kernel(
    int m, int n, int k, const float2* __restrict__ A, int64_t lda, int64_t sA,
    const float2* __restrict__ B, int64_t ldb, int64_t sB, float2* __restrict__ C, int64_t ldc,
    int64_t sC, int* __restrict__ err, const int* __restrict__ active, int group) {
    // batch entries of a finished contour (active[z / group] == 0) do nothing
    if (active && !active[blockIdx.z / group]) return;
    cgemm_body<BN>(m, n, k, A + blockIdx.z * sA, lda, B + blockIdx.z * sB, ldb, C + blockIdx.z * sC,
                   ldc, err);
}

// Trailing update of grouped LU nodes (orders may differ): node blockIdx.z;
// tiles outside that node's update do nothing.
template <int BN>
__global__ void __launch_bounds__(kTcThreads, 3) cgemm_grouped_kernel(
    const LuNode* __restrict__ nodes, int k0, int nb, int mode, int* __restrict__ err) {
    const LuNode d = nodes[blockIdx.z];
    int jb, c0, ncols;
    if (!lookahead_cols(d.n, k0, nb, mode, &jb, &c0, &ncols)) return;
    const int rows = (int)(d.n - k0 - jb);
    if ((int)blockIdx.x * kTcM >= rows || (int)blockIdx.y * BN >= ncols) return;
    float2* F = static_cast<float2*>(d.F);
    const int64_t n = d.n;
    cgemm_body<BN>(rows, ncols, jb, F + (k0 + jb) + (int64_t)k0 * n, n, F + k0 + (int64_t)c0 * n, n,
                   F + (k0 + jb) + (int64_t)c0 * n, n, err);
}

template <int BN>
constexpr int stage_smem() {
    return kTcStages * (2 * kTcAtile + 2 * (2 * BN) * 2 * kTcBK * 4);
}

template <int BN>
cudaError_t launch(cudaStream_t st, int m, int n, int k, const float2* A, int64_t lda, int64_t sA,
                   const float2* B, int64_t ldb, int64_t sB, float2* C, int64_t ldc, int64_t sC,
                   int batch, int* err, const int* active, int group) {
    constexpr int smem = stage_smem<BN>();
    static std::atomic<bool> attr_set[64] = {};   // idempotent setup; atomic for concurrent handles
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64 || !attr_set[dev]) {
        e = cudaFuncSetAttribute(cgemm_tf32x3_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 smem);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) attr_set[dev] = true;
    }
    dim3 grid((unsigned)((m + kTcM - 1) / kTcM), (unsigned)((n + BN - 1) / BN), (unsigned)batch);
    note_launch();
    cgemm_tf32x3_kernel<BN><<<grid, kTcThreads, smem, st>>>(m, n, k, A, lda, sA, B, ldb, sB, C, ldc,
                                                           sC, err, active, group);
    return cudaGetLastError();
}
}  // namespace

cudaError_t cgemm_sub_grouped(cudaStream_t st, const LuNode* nodes, int count, int k0, int nb,
                              int mode, int64_t max_rows, int64_t max_cols, int* err) {
    constexpr int BN = kLuUpdateBn;
    if (count <= 0 || max_rows <= 0 || max_cols <= 0) return cudaSuccess;
    if (count > 65535) return cudaErrorInvalidValue;
    constexpr int smem = stage_smem<BN>();
    static std::atomic<bool> attr_set[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64 || !attr_set[dev]) {
        e = cudaFuncSetAttribute(cgemm_grouped_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 smem);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) attr_set[dev] = true;
    }
    dim3 grid((unsigned)((max_rows + kTcM - 1) / kTcM), (unsigned)((max_cols + BN - 1) / BN),
              (unsigned)count);
    note_launch();
    cgemm_grouped_kernel<BN><<<grid, kTcThreads, smem, st>>>(nodes, k0, nb, mode, err);
    return cudaGetLastError();
}

namespace {
// Waits on an mbarrier that nothing arrives at, with the kernels' bounded wait
// and a caller-chosen limit: the wait must run out, set the error bit and
// return (the failure path every tensor-core kernel takes on a lost arrival).
__global__ void bounded_wait_probe_kernel(long long limit, int* __restrict__ flags) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&bar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const bool ok = mbar_wait_for(smem_u32(&bar), 0, limit);
    if (!ok && threadIdx.x == 0) atomicOr(flags, 16);
}
}  // namespace

cudaError_t bounded_wait_probe(cudaStream_t st, long long cycles, int* flags) {
    note_launch();
    bounded_wait_probe_kernel<<<1, 32, 0, st>>>(cycles, flags);
    return cudaGetLastError();
}

int cgemm_default_bn(int n) {
    // the widest tile that wastes the fewest columns (e.g. 48 for 96 right-hand sides)
    int best = 64, waste = ((n + 63) / 64) * 64 - n;
    for (int bn : {48, 32, 16}) {
        const int w = ((n + bn - 1) / bn) * bn - n;
        if (w < waste) { best = bn; waste = w; }
    }
    return best;
}

cudaError_t cgemm_sub_tf32x3(cudaStream_t st, int m, int n, int k, const float2* A, int64_t lda,
                             int64_t sA, const float2* B, int64_t ldb, int64_t sB, float2* C,
                             int64_t ldc, int64_t sC, int batch, int* err, int bn,
                             const int* active, int group) {
    if (m <= 0 || n <= 0 || k <= 0 || batch <= 0) return cudaSuccess;
    if (batch > 65535) return cudaErrorInvalidValue;
    if (bn == 0) bn = cgemm_default_bn(n);
    switch (bn) {
        case 16: return launch<16>(st, m, n, k, A, lda, sA, B, ldb, sB, C, ldc, sC, batch, err, active, group);
        case 32: return launch<32>(st, m, n, k, A, lda, sA, B, ldb, sB, C, ldc, sC, batch, err, active, group);
        case 48: return launch<48>(st, m, n, k, A, lda, sA, B, ldb, sB, C, ldc, sC, batch, err, active, group);
        case 64: return launch<64>(st, m, n, k, A, lda, sA, B, ldb, sB, C, ldc, sC, batch, err, active, group);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace fnl
