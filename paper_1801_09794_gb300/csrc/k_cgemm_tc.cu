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
// CTA: one 128 x BN complex tile of C, held in TMEM as 128 lanes x 2 BN FP32
// columns; 160 threads.  K advances 8 complex (16 real) entries per stage
// through a 2-slot shared-memory ring.  Warps 0-3 load a stage into registers
// two stages ahead, split it and store the four parts (A_hi, A_lo, B_hi, B_lo)
// in the canonical K-major SWIZZLE_NONE layout (8-row x 16-byte core
// matrices, the four K core matrices of a row group side by side: LBO 128 B,
// SBO 512 B) with 16-byte stores, and count themselves on the slot's full
// barrier; warp 4's lane 0 issues six MMAs (M = 128, N = 2 BN, K = 8) per full
// slot and commits them to the slot's empty barrier (its other lanes prefetch
// the C tile into L2).  No block-wide barrier inside the K loop.  The epilogue
// reads TMEM with lane = row of C and updates C in groups of 8 columns
// (coalesced along rows), the next group's loads in flight during the current
// group's stores.
#include "internal.h"
#include "tc_common.cuh"
#include "cgemm_tile.cuh"


namespace fnl {
namespace {
using namespace tc;
using namespace tcu;

// One CTA = one unit and one 128 x BN tile (blockIdx.x, blockIdx.y) of C -= A B.
template <int BN>
__device__ __forceinline__ void cgemm_body(int m, int n, int k, const float2* __restrict__ A,
                                           int64_t lda, const float2* __restrict__ B, int64_t ldb,
                                           float2* __restrict__ C, int64_t ldc,
                                           int* __restrict__ err) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t full[kTcStages], empty[kTcStages], done;
    __shared__ uint32_t s_tmem;
    const int tid = threadIdx.x, warp = tid >> 5;
    if (tid == 0) {
        unit_init_barriers(full, empty, &done);
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
    TcUnit u{smem, full, empty, &done, s_tmem, 1, 0u, 0u};
    const bool ok = cgemm_tile<BN>(u, tid, m, n, k, A, lda, B, ldb, C, ldc, blockIdx.x * kTcM,
                                   blockIdx.y * BN);
    if (!ok && tid == 0) atomicOr(err, 16);
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(u.tmem),
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
