// The complex64 tensor-core update tile C -= A B (tcgen05.mma.kind::tf32 on
// split operands), as a unit of 160 threads that the update kernels and the
// persistent factorisation run.  Included by the .cu files that launch it.
#pragma once
#include "internal.h"
#include "tc_common.cuh"

namespace fnl {
namespace tcu {
using namespace tc;

constexpr int kTcM = 128;                      // rows of C per CTA (TMEM lanes)
constexpr int kTcBK = 8;                       // complex K entries per stage
constexpr int kTcStages = 2;
constexpr int kTcLoaders = 128;                // loader / epilogue threads (warps 0-3)
constexpr int kTcThreads = kTcLoaders + 32;     // + the MMA-issuing warp
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

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// One update unit: 160 threads (warps 0-3 load, split and store the operand
// stages and later run the epilogue; warp 4 issues the MMAs), its ring of
// kTcStages stages in shared memory, its mbarriers and 128 TMEM columns.  A
// unit can run many tiles in turn (the persistent factorisation runs three
// per CTA): the mbarrier phases carry over from tile to tile through `stages`
// (ring stages used so far) and `tiles` (tiles finished).
struct TcUnit {
    unsigned char* ring;
    uint64_t* full;       // [kTcStages]
    uint64_t* empty;      // [kTcStages]
    uint64_t* done;
    uint32_t tmem;
    int bar;              // named barrier of the unit's 160 threads
    uint32_t stages;
    uint32_t tiles;
};

__device__ __forceinline__ void unit_sync(int bar) {
    asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(kTcThreads) : "memory");
}
// every thread of the unit gets the AND of v over the unit
__device__ __forceinline__ bool unit_and(int bar, bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\t"
        "bar.red.and.pred q, %2, %3, p;\n\tselp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(bar), "r"(kTcThreads)
        : "memory");
    return r != 0;
}

// Mbarriers of a unit (one thread, before any use; then a fence and a barrier).
__device__ __forceinline__ void unit_init_barriers(uint64_t* full, uint64_t* empty, uint64_t* done) {
    for (int q = 0; q < kTcStages; ++q) {
        mbar_init(smem_u32(&full[q]), kTcLoaders);
        mbar_init(smem_u32(&empty[q]), 1);
    }
    mbar_init(smem_u32(done), 1);
}

// The unit's 128 x BN tile at (row0, col0) of C -= A B (utid: thread index
// within the unit).  The loaders and the MMA warp meet only at mbarriers:
// full[slot] counts the 128 loader threads' stores of a stage, empty[slot] is
// the MMAs' commit of that slot, done the commit after the tile's last stage
// -- no unit-wide barrier inside the K loop.  Each loader keeps two stages in
// registers, so a stage's global loads are issued two stages ahead of its
// split.  Returns false (on every thread of the unit) when a wait timed out;
// the tile is then not written.
// Operand loads: through the read-only path when A and B stay unchanged for
// the whole launch (NC), else as ordinary cached loads (ld.global.ca), which a
// persistent kernel that changes the matrix between its tasks may use after
// its acquire of the producing task's flag.
template <bool NC, typename V>
__device__ __forceinline__ V ld_operand(const V* p) {
    if constexpr (NC) return __ldg(p);
    else return __ldca(p);
}

template <int BN, bool NC = true>
__device__ __forceinline__ bool cgemm_tile(TcUnit& u, int utid, int m, int n, int k,
                                           const float2* __restrict__ A, int64_t lda,
                                           const float2* __restrict__ B, int64_t ldb,
                                           float2* __restrict__ C, int64_t ldc, int row0,
                                           int col0) {
    constexpr int NR = 2 * BN;                   // real columns of the tile
    constexpr int kBtile = NR * 2 * kTcBK * 4;   // bytes of one B part
    constexpr int kStage = 2 * kTcAtile + 2 * kBtile;
    constexpr int kAP = kTcBK / 2;                         // k pairs of a stage (A items per thread)
    constexpr int kBIt = (BN / 8 + 3) / 4;                 // B warp steps per warp and stage
    static_assert(BN % 16 == 0 && NR <= 256, "tile width");
    unsigned char* smem = u.ring;
    uint64_t* full = u.full;
    uint64_t* empty = u.empty;
    const int tid = utid, warp = tid >> 5, lane = tid & 31;
    const int nk = (k + kTcBK - 1) / kTcBK;
    const uint32_t T0 = u.stages;                // global index of this tile's first stage
    const uint32_t tmem = u.tmem;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    bool ok = true;

    if (warp == kTcLoaders / 32) {
        if (lane == 0) {                             // MMA issuer
            const uint32_t idesc = tf32_idesc(kTcM, NR);
            int t = 0;
            for (; t < nk; ++t) {
                const uint32_t g = T0 + (uint32_t)t;
                const int slot = (int)(g % kTcStages);
                if (!mbar_wait(smem_u32(&full[slot]), (g / kTcStages) & 1)) { ok = false; break; }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t base = smem_u32(smem + slot * kStage);
#pragma unroll
                for (int ks = 0; ks < 2; ++ks) {     // two K = 8 (32-byte) steps
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
                        smem_u32(&empty[slot]))
                    : "memory");
            }
            // all MMAs issued have completed once `done` arrives (also on the
            // timeout path, so that TMEM is read or released only after them)
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    smem_u32(u.done))
                : "memory");
            if (!mbar_wait(smem_u32(u.done), u.tiles & 1) || t < nk) ok = false;
        } else if (row0 < m) {
            // the other lanes: the C tile into L2 while the K loop runs (up to 9
            // lines of 128 bytes per column)
            const int rows = min(kTcM, m - row0);
            for (int idx = lane - 1; idx < BN * 9; idx += 31) {
                const int j = idx / 9, t9 = idx - j * 9;
                if (col0 + j >= n) continue;
                const char* p0 = reinterpret_cast<const char*>(C + row0 + (int64_t)(col0 + j) * ldc);
                const uintptr_t l0 = reinterpret_cast<uintptr_t>(p0) >> 7;
                const uintptr_t l1 = (reinterpret_cast<uintptr_t>(p0) + (uintptr_t)rows * 8 - 1) >> 7;
                if (l0 + t9 <= l1) asm volatile("prefetch.global.L2 [%0];" ::"l"((l0 + t9) << 7));
            }
        }
    } else {
        // Every smem store writes one 16-byte row chunk of a core matrix: two
        // complex k (a k pair) of one row of A' or B'.
        // A: warp w takes rows 32 w + lane and, per item, the k pair p; the 8
        // lanes of a store phase hold 8 consecutive rows of one core matrix
        // (distinct 16-byte bank groups), and each load reads 32 consecutive rows.
        // B: a warp step covers 16 columns x 2 k pairs: lane = 8 jg + 4 psel + jo
        // takes column 4 jg + jo of its 16 and pair psel; it writes rows 2j and
        // 2j + 1 of B', the psel = 1 lanes the odd row first, so that each store
        // phase covers the 8 row slots of a core matrix.
        const int b_jo = lane & 3, b_ps = (lane >> 2) & 1, b_jg = lane >> 3;
        const int gr = row0 + warp * 32 + lane;
        // a k pair of B is 16-byte aligned when B is and its columns are an even number of entries apart
        const bool b_pair = ((reinterpret_cast<uintptr_t>(B) & 15) == 0) && ((ldb & 1) == 0);
        float2 ra0[2 * kAP], rb0[2 * kBIt], ra1[2 * kAP], rb1[2 * kBIt];

        auto load = [&](int t, float2* ra, float2* rb) {
            const int k0 = t * kTcBK;
#pragma unroll
            for (int p = 0; p < kAP; ++p) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int gk = k0 + 2 * p + h;
                    ra[2 * p + h] = (gr < m && gk < k) ? ld_operand<NC>(A + gr + (int64_t)gk * lda)
                                                       : make_float2(0.f, 0.f);
                }
            }
#pragma unroll
            for (int q = 0; q < kBIt; ++q) {
                const int it = warp + 4 * q;           // warp step: column chunk it >> 1, pairs 2 (it & 1)
                const int j = (it >> 1) * 16 + 4 * b_jg + b_jo, pp = (it & 1) * 2 + b_ps;
                const int gc = col0 + j, gk = k0 + 2 * pp;
                const float2* bp = B + gk + (int64_t)gc * ldb;
                if (b_pair && it < BN / 8 && gk + 1 < k && gc < n) {   // the k pair in one 16-byte load
                    const float4 w = ld_operand<NC>(reinterpret_cast<const float4*>(bp));
                    rb[2 * q] = make_float2(w.x, w.y);
                    rb[2 * q + 1] = make_float2(w.z, w.w);
                } else {
#pragma unroll
                    for (int h = 0; h < 2; ++h)
                        rb[2 * q + h] = (it < BN / 8 && gk + h < k && gc < n) ? ld_operand<NC>(bp + h)
                                                                              : make_float2(0.f, 0.f);
                }
            }
        };
        auto store = [&](int slot, const float2* ra, const float2* rb) {
            unsigned char* ahi = smem + slot * kStage;
            unsigned char* alo = ahi + kTcAtile;
            unsigned char* bhi = ahi + 2 * kTcAtile;
            unsigned char* blo = bhi + kBtile;
            const int r = warp * 32 + lane;
#pragma unroll
            for (int p = 0; p < kAP; ++p) {
                const uint32_t off = pair_off(r, 2 * p);
                const float2 v0 = ra[2 * p], v1 = ra[2 * p + 1];
                const float h0 = tf32_rn(v0.x), h1 = tf32_rn(v0.y), h2 = tf32_rn(v1.x), h3 = tf32_rn(v1.y);
                *reinterpret_cast<float4*>(ahi + off) = make_float4(h0, h1, h2, h3);
                *reinterpret_cast<float4*>(alo + off) =
                    make_float4(tf32_rn(v0.x - h0), tf32_rn(v0.y - h1), tf32_rn(v1.x - h2), tf32_rn(v1.y - h3));
            }
#pragma unroll
            for (int q = 0; q < kBIt; ++q) {
                const int it = warp + 4 * q;
                if (it >= BN / 8) break;
                const int j = (it >> 1) * 16 + 4 * b_jg + b_jo, pp = (it & 1) * 2 + b_ps;
                const float2 v0 = rb[2 * q], v1 = rb[2 * q + 1];
                const float r0 = tf32_rn(v0.x), i0 = tf32_rn(v0.y), r1 = tf32_rn(v1.x), i1 = tf32_rn(v1.y);
                const float lr0 = tf32_rn(v0.x - r0), li0 = tf32_rn(v0.y - i0);
                const float lr1 = tf32_rn(v1.x - r1), li1 = tf32_rn(v1.y - i1);
                // row 2j: (Re, -Im) per k; row 2j + 1: (Im, Re)
                const float4 he = make_float4(r0, -i0, r1, -i1), ho = make_float4(i0, r0, i1, r1);
                const float4 le = make_float4(lr0, -li0, lr1, -li1), lo = make_float4(li0, lr0, li1, lr1);
                const uint32_t oe = pair_off(2 * j, 2 * pp), oo = pair_off(2 * j + 1, 2 * pp);
                const uint32_t o1 = b_ps ? oo : oe, o2 = b_ps ? oe : oo;
                *reinterpret_cast<float4*>(bhi + o1) = b_ps ? ho : he;
                *reinterpret_cast<float4*>(bhi + o2) = b_ps ? he : ho;
                *reinterpret_cast<float4*>(blo + o1) = b_ps ? lo : le;
                *reinterpret_cast<float4*>(blo + o2) = b_ps ? le : lo;
            }
        };
        // stage t: wait until its slot's previous MMAs are done, split the
        // registers into it, count this thread on full[slot], then load stage t + 2
        auto step = [&](int t, float2* ra, float2* rb) {
            const uint32_t g = T0 + (uint32_t)t;
            const int slot = (int)(g % kTcStages);
            bool w = true;
            if (g >= kTcStages) w = mbar_wait(smem_u32(&empty[slot]), ((g / kTcStages) - 1) & 1);
            if (!__all_sync(0xffffffffu, w)) return false;   // warp-uniform exit on a timeout
            store(slot, ra, rb);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(smem_u32(&full[slot]));
            if (t + 2 < nk) load(t + 2, ra, rb);
            return true;
        };
        load(0, ra0, rb0);
        if (nk > 1) load(1, ra1, rb1);
        for (int t = 0; t < nk; t += 2) {            // two register sets, used in turn
            if (!step(t, ra0, rb0)) { ok = false; break; }
            if (t + 1 < nk && !step(t + 1, ra1, rb1)) { ok = false; break; }
        }
        // the accumulator is complete once `done` has arrived
        if (!__all_sync(0xffffffffu, mbar_wait(smem_u32(u.done), u.tiles & 1))) ok = false;
    }
    ok = unit_and(u.bar, ok);
    if (ok && warp < kTcLoaders / 32) {
        // epilogue: C -= accumulator, 8 complex columns per group; the next
        // group's C loads are issued before this group's stores
        // a warp may read only the TMEM lane quarter (CTA warp index mod 4): the
        // unit's four loader warps cover the four quarters in some order
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int quarter = (int)((threadIdx.x >> 5) & 3);
        const int row = row0 + quarter * 32 + lane;
        const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16);
        const bool live = row < m;
        constexpr int kGroups = NR / 16;
        float2 cv[8], cn[8];
        auto cload = [&](int g, float2* dst) {
#pragma unroll
            for (int jj = 0; jj < 8; ++jj) {
                const int j = col0 + g * 8 + jj;
                if (live && j < n) dst[jj] = C[row + (int64_t)j * ldc];
            }
        };
        cload(0, cv);
#pragma unroll 1
        for (int g = 0; g < kGroups; g += 2) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {            // groups g (cv) and g + 1 (cn)
                const int gg = g + h;
                if (gg >= kGroups) break;
                float2* cur = h ? cn : cv;
                float2* nxt = h ? cv : cn;
                if (gg + 1 < kGroups) cload(gg + 1, nxt);
                uint32_t v[16];
                tmem_ld8(taddr + (uint32_t)(gg * 16), v);
                tmem_ld8(taddr + (uint32_t)(gg * 16 + 8), v + 8);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int jj = 0; jj < 8; ++jj) {
                    const int j = col0 + gg * 8 + jj;
                    if (live && j < n)
                        C[row + (int64_t)j * ldc] = make_float2(cur[jj].x - __uint_as_float(v[2 * jj]),
                                                                cur[jj].y - __uint_as_float(v[2 * jj + 1]));
                }
            }
        }
    }
    // the next tile's MMAs overwrite TMEM only after this epilogue's reads
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    unit_sync(u.bar);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    u.stages += (uint32_t)nk;
    u.tiles += 1;
    return ok;
}

template <int BN>
constexpr int stage_smem() {
    return kTcStages * (2 * kTcAtile + 2 * (2 * BN) * 2 * kTcBK * 4);
}

}  // namespace tcu
}  // namespace fnl
