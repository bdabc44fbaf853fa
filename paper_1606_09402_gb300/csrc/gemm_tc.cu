// BF16 tensor-core passes over a dense row-major A on sm_103a: TMA (cp.async.bulk.tensor) tiles
// into 128-byte-swizzled shared memory, tcgen05.mma with the float32 accumulator in tensor memory,
// tcgen05.ld for the epilogue.
//
//   sketch (G = A Omega, Y = A Z):  D (m x w) = A (m x n) * V (n x w)
//       A operand: A row tile [128 rows x 64 k] (K-major)
//       B operand: V^T tile [BN x 64 k] from V column-major (K-major)
//   trans  (B_i^T = A^T Q_i, H = A^T G, Z = A^T Y):  D (n x w) = A^T (n x m) * V (m x w)
//       A operand: column slab of A [64 k rows x 128 n] as two 64-column boxes (MN-major)
//       B operand: V^T tile [BN x 64 k] (K-major)
//   Up to three products accumulate into one tile: A_hi V_hi, A_lo V_hi (NA = 2) and A_hi V_lo
//   (NB = 2), where A = A_hi + A_lo and V = V_hi + V_lo are bf16 pairs.
//
// Persistent CTAs (one per SM).  Work is the list of (row tile, column tile) units x the k-blocks
// of each unit.  With several column tiles every CTA takes whole units in raster order (row tile
// outer) so CTAs running together share the A tile through L2.  With one column tile (the
// narrow passes of randQB_EI) the flattened k-block range is split evenly across CTAs
// ("stream-K"): A is read exactly once and no SM idles on a partial wave; units cut between CTAs
// leave float32 partials that a fix-up kernel adds in CTA order (deterministic).
//
// Warp roles: warp 0 issues TMA, warp 1 owns tensor memory and issues MMAs, warps 2-5 drain the
// accumulator (double-buffered in tensor memory, so the epilogue of one unit overlaps the main
// loop of the next).  Every mbarrier wait is bounded: on timeout the kernel records an error flag
// and leaves the loop instead of spinning.
#include "qb_internal.cuh"
#include "sched.cuh"

#include <cuda.h>

#include <mutex>

namespace qb {
namespace {

constexpr int BM = TC_BM;    // rows of the accumulator tile (MMA M)
constexpr int BK = TC_BK;    // k per stage: one 128-byte swizzle row of bf16
constexpr int UMMA_K = 16;   // k per tcgen05.mma (kind::f16)
constexpr int NUM_THREADS = 192;
constexpr uint64_t WAIT_NS = 2000000000ull;   // bounded waits: 2 s
constexpr int MAX_SK_CTAS = TC_MAX_SK_CTAS;

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait; false (and err flag set) after WAIT_NS.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* err) {
    if (mbar_try(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    while (true) {
        for (int i = 0; i < 64; ++i)
            if (mbar_try(bar, parity)) return true;
        if (globaltimer() - t0 > WAIT_NS) {
            atomicOr(err, 1);
            return false;
        }
    }
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x,
                                            int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
        : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                       uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
// 32 lanes x 32 columns of 32-bit words: thread t of the warp gets row (lane base + t)
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// 64 columns as two x32 loads with a single wait
__device__ __forceinline__ void tmem_ld64(uint32_t taddr, float (&v)[64]) {
    uint32_t r[64];
#define QB_LD32(OFF, BASE)                                                                       \
    asm volatile(                                                                                \
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "                                                \
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"                                \
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"               \
        : "=r"(r[BASE + 0]), "=r"(r[BASE + 1]), "=r"(r[BASE + 2]), "=r"(r[BASE + 3]),            \
          "=r"(r[BASE + 4]), "=r"(r[BASE + 5]), "=r"(r[BASE + 6]), "=r"(r[BASE + 7]),            \
          "=r"(r[BASE + 8]), "=r"(r[BASE + 9]), "=r"(r[BASE + 10]), "=r"(r[BASE + 11]),          \
          "=r"(r[BASE + 12]), "=r"(r[BASE + 13]), "=r"(r[BASE + 14]), "=r"(r[BASE + 15]),        \
          "=r"(r[BASE + 16]), "=r"(r[BASE + 17]), "=r"(r[BASE + 18]), "=r"(r[BASE + 19]),        \
          "=r"(r[BASE + 20]), "=r"(r[BASE + 21]), "=r"(r[BASE + 22]), "=r"(r[BASE + 23]),        \
          "=r"(r[BASE + 24]), "=r"(r[BASE + 25]), "=r"(r[BASE + 26]), "=r"(r[BASE + 27]),        \
          "=r"(r[BASE + 28]), "=r"(r[BASE + 29]), "=r"(r[BASE + 30]), "=r"(r[BASE + 31])         \
        : "r"(taddr + (OFF)))
    QB_LD32(0, 0);
    QB_LD32(32, 32);
#undef QB_LD32
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 64; ++i) v[i] = __uint_as_float(r[i]);
}

// Shared-memory matrix descriptor (tcgen05): start address, leading / stride byte offsets,
// descriptor version 1, 128-byte swizzle.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= uint64_t((saddr >> 4) & 0x3FFFu);
    d |= uint64_t((lbo >> 4) & 0x3FFFu) << 16;
    d |= uint64_t((sbo >> 4) & 0x3FFFu) << 32;
    d |= uint64_t(1) << 46;
    d |= uint64_t(2) << 61;
    return d;
}
// Instruction descriptor, kind::f16: bf16 A and B, float32 D, M = 128, N = bn.
__host__ __device__ constexpr uint32_t idesc_bf16(int bn, bool a_mn) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((a_mn ? 1u : 0u) << 15) |
           (uint32_t(bn >> 3) << 17) | (uint32_t(BM >> 4) << 24);
}

// Output row gr of a tile: D[gr][c0 + j] = alpha v[j] (+ beta D[gr][c0 + j]) for the NV columns
// below n.  With beta != 0 the old values are all loaded before any store is issued (the loads do
// not wait on one another; a load-modify-store per column would serialise them).
template <int NV>
__device__ __forceinline__ void store_row(float* D, int64_t ldd, int64_t gr, int c0, int n,
                                          float alpha, float beta, const float* v) {
    static_assert(NV % 32 == 0, "groups of 32 columns");
    float* base = D + gr + int64_t(c0) * ldd;
    const int nv = n - c0 < NV ? n - c0 : NV;
    if (beta != 0.f) {
#pragma unroll
        for (int g = 0; g < NV; g += 32) {
            float old[32];
#pragma unroll
            for (int j = 0; j < 32; ++j)
                old[j] = g + j < nv ? __ldcg(base + int64_t(g + j) * ldd) : 0.f;
#pragma unroll
            for (int j = 0; j < 32; ++j)
                if (g + j < nv) base[int64_t(g + j) * ldd] = fmaf(alpha, v[g + j], beta * old[j]);
        }
    } else {
#pragma unroll
        for (int j = 0; j < NV; ++j)
            if (j < nv) base[int64_t(j) * ldd] = alpha * v[j];
    }
}

// ---------------------------------------------------------------- schedule
// ---------------------------------------------------------------- kernel
struct Params {
    int M, N, K;                 // D is M x N, reduction length K
    int chunk;                   // k-blocks accumulated in tensor memory before a register flush
    float alpha, beta;           // D = alpha * (product) + beta * D
    Sched s;
    float* D;
    int64_t ldd;
    float* part;                 // stream-K partial slots: [G][2][BN][BM]
    int* err;
};

template <int BN, bool TRANS, int NA, int NB>
struct Cfg {
    static constexpr int A_TILE = BM * BK * 2;         // 16 KB per A array
    static constexpr int B_TILE = BN * BK * 2;
    static constexpr int STAGE = NA * A_TILE + NB * B_TILE;
    static constexpr int STAGES = (200 * 1024) / STAGE < 8 ? (200 * 1024) / STAGE : 8;
    static constexpr int SMEM = STAGES * STAGE + 1024 /*align*/ + 256 /*barriers*/;
    static constexpr int TMEM_COLS = 2 * BN;           // double-buffered accumulator
};

template <int BN, bool TRANS, int NA, int NB>
__global__ void __launch_bounds__(NUM_THREADS, 1)
k_tc_gemm(const __grid_constant__ CUtensorMap mA0, const __grid_constant__ CUtensorMap mA1,
          const __grid_constant__ CUtensorMap mB0, const __grid_constant__ CUtensorMap mB1,
          Params p) {
    using C = Cfg<BN, TRANS, NA, NB>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + C::STAGES * C::STAGE);
    uint64_t* empty = full + C::STAGES;
    uint64_t* tfull = empty + C::STAGES;   // [2]
    uint64_t* tempty = tfull + 2;          // [2]
    uint64_t* drain = tempty + 2;          // [1] MMA completion after a timed-out wait
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int G = gridDim.x, cta = blockIdx.x;

    if (threadIdx.x == 0) {
        for (int s = 0; s < C::STAGES; ++s) {
            mbar_init(full + s, 1);
            mbar_init(empty + s, 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(tfull + b, 1);
            mbar_init(tempty + b, 128);
        }
        mbar_init(drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(C::TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    // this CTA's segments
    const Sched& sc = p.s;
    auto unit_rc = [&](int u, int& r0, int& c0) {
        r0 = (u / sc.tiles_n) * BM;
        c0 = (u % sc.tiles_n) * BN;
    };

    bool ok = true;
    if (warp == 0 && lane == 0) {
        // ---------------------------------------------------------- TMA producer
        int stage = 0;
        uint32_t phase = 0;
        SegWalk wk(sc, cta, G);
        Seg sg;
        constexpr uint32_t bytes = uint32_t(C::STAGE);
        uint32_t armed = 0, armed_par = 0;   // stages with copies issued, and their phase parity
        while (ok && wk.next(sg)) {
            int r0, c0;
            unit_rc(sg.u, r0, c0);
            for (int kb = sg.k0; kb < sg.k1 && ok; ++kb) {
                ok = mbar_wait(empty + stage, phase ^ 1, p.err);
                if (!ok) break;
                armed |= 1u << stage;
                armed_par = (armed_par & ~(1u << stage)) | (phase << stage);
                mbar_expect_tx(full + stage, bytes);
                unsigned char* st = smem + stage * C::STAGE;
                const int k = kb * BK;
                if (!TRANS) {
                    tma_load_2d(st, &mA0, full + stage, k, r0);
                    if (NA > 1) tma_load_2d(st + C::A_TILE, &mA1, full + stage, k, r0);
                } else {
                    tma_load_2d(st, &mA0, full + stage, r0, k);
                    tma_load_2d(st + C::A_TILE / 2, &mA0, full + stage, r0 + 64, k);
                    if (NA > 1) {
                        tma_load_2d(st + C::A_TILE, &mA1, full + stage, r0, k);
                        tma_load_2d(st + C::A_TILE + C::A_TILE / 2, &mA1, full + stage, r0 + 64, k);
                    }
                }
                unsigned char* sb = st + NA * C::A_TILE;
                tma_load_2d(sb, &mB0, full + stage, k, c0);
                if (NB > 1) tma_load_2d(sb + C::B_TILE, &mB1, full + stage, k, c0);
                if (++stage == C::STAGES) { stage = 0; phase ^= 1; }
            }
        }
        // a timed-out wait ends the loops early: let the bulk copies already issued land before
        // the CTA exits (each wait bounded; a stage already consumed returns at once)
        if (!ok)
            for (int s2 = 0; s2 < C::STAGES; ++s2)
                if (armed & (1u << s2)) mbar_wait(full + s2, (armed_par >> s2) & 1u, p.err);
    } else if (warp == 1 && lane == 0) {
        // ---------------------------------------------------------- MMA issuer
        constexpr uint32_t idesc = idesc_bf16(BN, TRANS);
        int stage = 0;
        uint32_t phase = 0;
        SegWalk wk(sc, cta, G);
        Seg sg;
        int buf = 0;
        uint32_t tphase[2] = {0, 0};
        while (ok && wk.next(sg)) {
            for (int c0 = sg.k0; c0 < sg.k1 && ok; c0 += p.chunk) {
                const int c1 = min(sg.k1, c0 + p.chunk);
                ok = mbar_wait(tempty + buf, tphase[buf] ^ 1, p.err);
                if (!ok) break;
                tc_fence_after();
                const uint32_t acc = tmem + uint32_t(buf * BN);
                for (int kb = c0; kb < c1 && ok; ++kb) {
                    ok = mbar_wait(full + stage, phase, p.err);
                    if (!ok) break;
                    tc_fence_after();
                    const uint32_t sa = smem_u32(smem + stage * C::STAGE);
                    const uint32_t sbb = sa + NA * C::A_TILE;
#pragma unroll
                    for (int kk = 0; kk < BK / UMMA_K; ++kk) {
                        uint64_t da[2], db[2];
#pragma unroll
                        for (int q = 0; q < NA; ++q) {
                            const uint32_t base = sa + q * C::A_TILE;
                            da[q] = TRANS ? sdesc(base + kk * (UMMA_K * 128), C::A_TILE / 2, 1024)
                                          : sdesc(base + kk * (UMMA_K * 2), 16, 1024);
                        }
#pragma unroll
                        for (int q = 0; q < NB; ++q)
                            db[q] = sdesc(sbb + q * C::B_TILE + kk * (UMMA_K * 2), 16, 1024);
                        const uint32_t accum = (kb > c0 || kk > 0) ? 1u : 0u;
                        tc_mma(acc, da[0], db[0], idesc, accum);                   // A_hi V_hi
                        if (NA > 1) tc_mma(acc, da[NA - 1], db[0], idesc, 1u);      // A_lo V_hi
                        if (NB > 1) tc_mma(acc, da[0], db[NB - 1], idesc, 1u);      // A_hi V_lo
                    }
                    tc_commit(empty + stage);
                    if (++stage == C::STAGES) { stage = 0; phase ^= 1; }
                }
                tc_commit(tfull + buf);
                tphase[buf] ^= 1;
                buf ^= 1;
            }
        }
        // after a timed-out wait, wait (bounded) for the MMAs already issued before the tensor
        // memory is freed
        if (!ok) {
            tc_commit(drain);
            mbar_wait(drain, 0, p.err);
        }
    } else if (warp >= 2) {
        // ---------------------------------------------------------- epilogue
        const int q = warp & 3;                 // tensor-memory lane quarter of this warp
        const int row = q * 32 + lane;
        SegWalk wk(sc, cta, G);
        Seg sg;
        int buf = 0;
        uint32_t tphase[2] = {0, 0};
        while (ok && wk.next(sg)) {
            int r0, c0;
            unit_rc(sg.u, r0, c0);
            const int64_t gr = int64_t(r0) + row;
            float* slot = sg.slot >= 0 ? p.part + ((int64_t(cta) * 2 + sg.slot) * BN) * BM : nullptr;
            if (sg.k1 - sg.k0 <= p.chunk) {
                // one accumulation chain: stream tensor memory straight to global memory
                ok = mbar_wait(tfull + buf, tphase[buf], p.err);
                if (!ok) break;
                tc_fence_after();
#pragma unroll 1
                for (int cc = 0; cc < BN; cc += 32) {
                    float v[32];
                    tmem_ld32(tmem + (uint32_t(q * 32) << 16) + uint32_t(buf * BN + cc), v);
                    if (slot) {
#pragma unroll
                        for (int j = 0; j < 32; ++j) slot[int64_t(cc + j) * BM + row] = v[j];
                    } else if (gr < p.M) {
                        store_row<32>(p.D, p.ldd, gr, c0 + cc, p.N, p.alpha, p.beta, v);
                    }
                }
                tc_fence_before();
                mbar_arrive(tempty + buf);
                tphase[buf] ^= 1;
                buf ^= 1;
                continue;
            }
            if constexpr (BN <= 128) {
                // Several chains: sum the chunk accumulators in registers (round to nearest), so
                // the float32 result carries no drift from long tensor-core accumulation chains.
                float accr[BN];
#pragma unroll
                for (int j = 0; j < BN; ++j) accr[j] = 0.f;
                for (int k0 = sg.k0; k0 < sg.k1 && ok; k0 += p.chunk) {
                    ok = mbar_wait(tfull + buf, tphase[buf], p.err);
                    if (!ok) break;
                    tc_fence_after();
#pragma unroll
                    for (int cc = 0; cc < BN; cc += 64) {
                        float v[64];
                        tmem_ld64(tmem + (uint32_t(q * 32) << 16) + uint32_t(buf * BN + cc), v);
#pragma unroll
                        for (int j = 0; j < 64; ++j) accr[cc + j] += v[j];
                    }
                    tc_fence_before();
                    mbar_arrive(tempty + buf);
                    tphase[buf] ^= 1;
                    buf ^= 1;
                }
                if (!ok) break;
                if (slot) {
#pragma unroll
                    for (int j = 0; j < BN; ++j) slot[int64_t(j) * BM + row] = accr[j];
                } else if (gr < p.M) {
                    store_row<BN>(p.D, p.ldd, gr, c0, p.N, p.alpha, p.beta, accr);
                }
            }
        }
    }
    __syncwarp();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(C::TMEM_COLS));
    }
}

// ---------------------------------------------------------------- precise transposed pass
// D (n x w) = (A_hi [+ A_lo])^T V where V is given exactly by NB bf16 terms (NB = 1: V is
// bf16-representable; NB = 3: V = V_hi + V_mid + V_lo reproduces any float32 V).  The tensor
// cores' float32 accumulation is not round-to-nearest and biases long sums toward zero, which the
// Frobenius indicator cannot absorb (it subtracts ||B_i||^2 from ||A||^2).  So the leading
// product A_hi V_hi never accumulates in tensor memory: every MMA of it writes a fresh slot of a
// ring (accumulate flag off) and the epilogue adds the slots in registers with round-to-nearest.
// The lower-order products (A_lo V_hi, A_hi V_mid: 2^-9 of the leading one; A_hi V_lo,
// A_lo V_mid: 2^-18) accumulate in tensor memory over PREC_CHUNK k-blocks, where their bias is
// scaled down by those factors.  A_lo V_lo (2^-27) is dropped.
constexpr int PREC_CHUNK = 16;
constexpr int PREC_LEAD = 2;   // leading-product MMAs (K = 16 each) per tensor-memory slot
constexpr int PREC_EPI = 8;                          // epilogue warps
constexpr int PREC_THREADS = 64 + 32 * PREC_EPI;     // TMA warp, MMA warp, epilogue warps

// Lower-order products (i, j) of A term i and V term j (weight 2^-9 (i + j)): every pair with
// i + j <= 2 except the leading (0, 0).
__host__ __device__ constexpr int prec_nsmall(int na, int nb) {
    int c = 0;
    for (int i = 0; i < na; ++i)
        for (int j = 0; j < nb; ++j)
            if (i + j >= 1 && i + j <= 2) ++c;
    return c;
}

template <int BN, int NA, int NB>
struct PCfg {
    static constexpr int A_TILE = BM * BK * 2;
    static constexpr int B_TILE = BN * BK * 2;
    static constexpr int STAGE = NA * A_TILE + NB * B_TILE;
    // up to 224 KB of stages (the kernel has no static shared memory; 227 KB per block): the
    // three-term operands make a stage 56-72 KB at BN = 64, where every extra stage in flight
    // counts for the HBM-bound narrow passes
    static constexpr int STAGE_BUDGET = 224 * 1024;
    static constexpr int STAGES = STAGE_BUDGET / STAGE < 8 ? STAGE_BUDGET / STAGE : 8;
    static constexpr int SMEM = STAGES * STAGE + 1024 + 512;
    static_assert(SMEM <= 227 * 1024, "dynamic shared memory above the per-block limit");
    static constexpr int NSMALL = prec_nsmall(NA, NB);
    // chain buffers: two at BN = 64; one at BN = 128, which leaves three ring slots (the chain is
    // drained once per PREC_CHUNK k-blocks, the ring once per MMA)
    static constexpr int NCHAIN = NSMALL > 0 ? (BN >= 128 ? 1 : 2) : 0;
    static constexpr int SMALL_COLS = NCHAIN * BN;
    static constexpr int NSLOT = (512 - SMALL_COLS) / BN < 8 ? (512 - SMALL_COLS) / BN : 8;
    static constexpr int TMEM_COLS = 512;
};

template <int BN, bool TRANS, int NA, int NB>
__global__ void __launch_bounds__(PREC_THREADS, 1)
k_tc_prec(const __grid_constant__ CUtensorMap mA0, const __grid_constant__ CUtensorMap mA1,
          const __grid_constant__ CUtensorMap mA2, const __grid_constant__ CUtensorMap mB0,
          const __grid_constant__ CUtensorMap mB1, const __grid_constant__ CUtensorMap mB2,
          Params p) {
    using C = PCfg<BN, NA, NB>;
    static_assert(C::STAGES >= 2, "precise pass needs two stages");
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + C::STAGES * C::STAGE);
    uint64_t* empty = full + C::STAGES;
    uint64_t* sfull = empty + C::STAGES;   // [2] small-product chain
    uint64_t* sempty = sfull + 2;          // [2]
    uint64_t* bfull = sempty + 2;          // [NSLOT] leading-product slots
    uint64_t* bempty = bfull + C::NSLOT;   // [NSLOT]
    uint64_t* drain = bempty + C::NSLOT;   // [1] MMA completion after a timed-out wait
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int G = gridDim.x, cta = blockIdx.x;
    if (threadIdx.x == 0) {
        for (int s = 0; s < C::STAGES; ++s) {
            mbar_init(full + s, 1);
            mbar_init(empty + s, 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(sfull + b, 1);
            mbar_init(sempty + b, PREC_EPI * 32);
        }
        for (int b = 0; b < C::NSLOT; ++b) {
            mbar_init(bfull + b, 1);
            mbar_init(bempty + b, PREC_EPI * 32);
        }
        mbar_init(drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(C::TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t tm_small = tmem;                          // 2 x BN columns
    const uint32_t tm_big = tmem + uint32_t(C::SMALL_COLS);  // NSLOT x BN columns

    const Sched& sc = p.s;

    bool ok = true;
    if (warp == 0 && lane == 0) {
        // ---------------------------------------------------------- TMA producer
        int stage = 0;
        uint32_t phase = 0;
        SegWalk wk(sc, cta, G);
        Seg sg;
        uint32_t armed = 0, armed_par = 0;   // stages with copies issued, and their phase parity
        while (ok && wk.next(sg)) {
            const int r0 = (sg.u / sc.tiles_n) * BM, c0 = (sg.u % sc.tiles_n) * BN;
            for (int kb = sg.k0; kb < sg.k1 && ok; ++kb) {
                ok = mbar_wait(empty + stage, phase ^ 1, p.err);
                if (!ok) break;
                armed |= 1u << stage;
                armed_par = (armed_par & ~(1u << stage)) | (phase << stage);
                mbar_expect_tx(full + stage, uint32_t(C::STAGE));
                unsigned char* st = smem + stage * C::STAGE;
                const int k = kb * BK;
#pragma unroll
                for (int i = 0; i < NA; ++i) {
                    const CUtensorMap* m = i == 0 ? &mA0 : (i == 1 ? &mA1 : &mA2);
                    unsigned char* d = st + i * C::A_TILE;
                    if (TRANS) {
                        tma_load_2d(d, m, full + stage, r0, k);
                        tma_load_2d(d + C::A_TILE / 2, m, full + stage, r0 + 64, k);
                    } else {
                        tma_load_2d(d, m, full + stage, k, r0);
                    }
                }
                unsigned char* sb = st + NA * C::A_TILE;
#pragma unroll
                for (int j = 0; j < NB; ++j)
                    tma_load_2d(sb + j * C::B_TILE, j == 0 ? &mB0 : (j == 1 ? &mB1 : &mB2),
                                full + stage, k, c0);
                if (++stage == C::STAGES) { stage = 0; phase ^= 1; }
            }
        }
        // a timed-out wait ends the loops early: let the bulk copies already issued land first
        if (!ok)
            for (int s2 = 0; s2 < C::STAGES; ++s2)
                if (armed & (1u << s2)) mbar_wait(full + s2, (armed_par >> s2) & 1u, p.err);
    } else if (warp == 1 && lane == 0) {
        // ---------------------------------------------------------- MMA issuer
        constexpr uint32_t idesc = idesc_bf16(BN, TRANS);
        int stage = 0;
        uint32_t phase = 0;
        int slot = 0;
        uint32_t slot_ph = 0;   // bit s: phase of slot s
        int sbuf = 0;
        uint32_t sph = 0;   // bit b: phase of chain buffer b
        SegWalk wk(sc, cta, G);
        Seg sg;
        while (ok && wk.next(sg)) {
            for (int c0 = sg.k0; c0 < sg.k1 && ok; c0 += PREC_CHUNK) {
                const int c1 = min(sg.k1, c0 + PREC_CHUNK);
                const uint32_t acc_s = tm_small + uint32_t(sbuf * BN);
                if (C::NSMALL > 0) {
                    ok = mbar_wait(sempty + sbuf, ((sph >> sbuf) & 1u) ^ 1u, p.err);
                    if (!ok) break;
                    tc_fence_after();
                }
                for (int kb = c0; kb < c1 && ok; ++kb) {
                    ok = mbar_wait(full + stage, phase, p.err);
                    if (!ok) break;
                    tc_fence_after();
                    const uint32_t sa = smem_u32(smem + stage * C::STAGE);
                    const uint32_t sbb = sa + NA * C::A_TILE;
#pragma unroll
                    for (int kk = 0; kk < BK / UMMA_K; ++kk) {
                        uint64_t da[NA], db[NB];
#pragma unroll
                        for (int i = 0; i < NA; ++i)
                            da[i] = TRANS ? sdesc(sa + i * C::A_TILE + kk * (UMMA_K * 128),
                                                  C::A_TILE / 2, 1024)
                                          : sdesc(sa + i * C::A_TILE + kk * (UMMA_K * 2), 16, 1024);
#pragma unroll
                        for (int j = 0; j < NB; ++j)
                            db[j] = sdesc(sbb + j * C::B_TILE + kk * (UMMA_K * 2), 16, 1024);
                        // leading product: PREC_LEAD MMAs into a fresh slot
                        if (kk % PREC_LEAD == 0) {
                            ok = mbar_wait(bempty + slot, ((slot_ph >> slot) & 1u) ^ 1u, p.err);
                            if (!ok) break;
                            tc_fence_after();
                        }
                        tc_mma(tm_big + uint32_t(slot * BN), da[0], db[0], idesc,
                               kk % PREC_LEAD == 0 ? 0u : 1u);
                        if (kk % PREC_LEAD == PREC_LEAD - 1) {
                            tc_commit(bfull + slot);
                            slot_ph ^= 1u << slot;
                            if (++slot == C::NSLOT) slot = 0;
                        }
                        // lower-order products, smallest weight first
                        uint32_t acc = (kb > c0 || kk > 0) ? 1u : 0u;
#pragma unroll
                        for (int w = 2; w >= 1; --w)
#pragma unroll
                            for (int i = 0; i < NA; ++i) {
                                const int j = w - i;
                                if (j < 0 || j >= NB) continue;
                                tc_mma(acc_s, da[i], db[j], idesc, acc);
                                acc = 1u;
                            }
                    }
                    if (!ok) break;
                    tc_commit(empty + stage);
                    if (++stage == C::STAGES) { stage = 0; phase ^= 1; }
                }
                if (!ok) break;
                if (C::NSMALL > 0) {
                    tc_commit(sfull + sbuf);
                    sph ^= 1u << sbuf;
                    if (++sbuf == C::NCHAIN) sbuf = 0;
                }
            }
        }
        // after a timed-out wait, wait (bounded) for the MMAs already issued before the tensor
        // memory is freed
        if (!ok) {
            tc_commit(drain);
            mbar_wait(drain, 0, p.err);
        }
    } else if (warp >= 2) {
        // ---------------------------------------------------------- epilogue
        // PREC_EPI warps: lane quarter q = warp % 4 (the tensor-memory lanes a warp may read),
        // column half h of the tile.
        constexpr int HC = BN / 2;
        const int q = warp & 3;
        const int h = (warp - 2) >> 2;
        const int row = q * 32 + lane;
        const uint32_t lane_off = uint32_t(q * 32) << 16;
        const uint32_t col_off = uint32_t(h * HC);
        int slot = 0;
        uint32_t slot_ph = 0;
        int sbuf = 0;
        uint32_t sph = 0;   // bit b: phase of chain buffer b
        SegWalk wk(sc, cta, G);
        Seg sg;
        while (ok && wk.next(sg)) {
            const int r0 = (sg.u / sc.tiles_n) * BM, c0 = (sg.u % sc.tiles_n) * BN + h * HC;
            const int64_t gr = int64_t(r0) + row;
            float* pslot = sg.slot >= 0
                               ? p.part + ((int64_t(cta) * 2 + sg.slot) * BN + h * HC) * BM
                               : nullptr;
            // the running sums, two columns per packed float32 pair add (round-to-nearest per
            // element, so the same sums as scalar adds at half the instructions)
            float2 acc2[HC / 2];
#pragma unroll
            for (int j = 0; j < HC / 2; ++j) acc2[j] = make_float2(0.f, 0.f);
            for (int k0 = sg.k0; k0 < sg.k1 && ok; k0 += PREC_CHUNK) {
                const int k1 = min(sg.k1, k0 + PREC_CHUNK);
                for (int kb = k0; kb < k1 && ok; ++kb) {
                    for (int kk = 0; kk < BK / UMMA_K / PREC_LEAD && ok; ++kk) {
                        ok = mbar_wait(bfull + slot, (slot_ph >> slot) & 1u, p.err);
                        if (!ok) break;
                        tc_fence_after();
                        if constexpr (HC == 64) {
                            float v[64];
                            tmem_ld64(tm_big + lane_off + uint32_t(slot * BN) + col_off, v);
#pragma unroll
                            for (int j = 0; j < 32; ++j)
                                acc2[j] = __fadd2_rn(acc2[j], make_float2(v[2 * j], v[2 * j + 1]));
                        } else {
#pragma unroll
                            for (int cc = 0; cc < HC; cc += 32) {
                                float v[32];
                                tmem_ld32(tm_big + lane_off + uint32_t(slot * BN) + col_off +
                                              uint32_t(cc), v);
#pragma unroll
                                for (int j = 0; j < 16; ++j)
                                    acc2[cc / 2 + j] = __fadd2_rn(acc2[cc / 2 + j],
                                                                  make_float2(v[2 * j], v[2 * j + 1]));
                            }
                        }
                        tc_fence_before();
                        mbar_arrive(bempty + slot);
                        slot_ph ^= 1u << slot;
                        if (++slot == C::NSLOT) slot = 0;
                    }
                }
                if (!ok) break;
                if (C::NSMALL > 0) {
                    ok = mbar_wait(sfull + sbuf, (sph >> sbuf) & 1u, p.err);
                    if (!ok) break;
                    tc_fence_after();
#pragma unroll
                    for (int cc = 0; cc < HC; cc += 32) {
                        float v[32];
                        tmem_ld32(tm_small + lane_off + uint32_t(sbuf * BN) + col_off + uint32_t(cc), v);
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            acc2[cc / 2 + j] = __fadd2_rn(acc2[cc / 2 + j],
                                                          make_float2(v[2 * j], v[2 * j + 1]));
                    }
                    tc_fence_before();
                    mbar_arrive(sempty + sbuf);
                    sph ^= 1u << sbuf;
                    if (++sbuf == C::NCHAIN) sbuf = 0;
                }
            }
            if (!ok) break;
            float accr[HC];
#pragma unroll
            for (int j = 0; j < HC / 2; ++j) {
                accr[2 * j] = acc2[j].x;
                accr[2 * j + 1] = acc2[j].y;
            }
            if (pslot) {
#pragma unroll
                for (int j = 0; j < HC; ++j) pslot[int64_t(j) * BM + row] = accr[j];
            } else if (gr < p.M) {
                store_row<HC>(p.D, p.ldd, gr, c0, p.N, p.alpha, p.beta, accr);
            }
        }
    }
    __syncwarp();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(C::TMEM_COLS));
    }
}

// Stream-K fix-up: D tile of unit u = sum of the partial slots of the CTAs that share it, in a
// fixed order (four interleaved sums over the CTAs in order, then combined).  A unit covered by
// one CTA was written directly and is skipped.  Grid: (units, BM*BN/256), one output element per
// thread, so a unit shared by every CTA of the launch is still summed by many CTAs in parallel;
// the slot offsets are worked out once per CTA.
template <int BN>
__global__ void __launch_bounds__(256) k_tc_fixup(Params p, int G) {
    __shared__ int64_t base[MAX_SK_CTAS];
    __shared__ int64_t first_s;
    __shared__ int count_s;
    const Sched& sc = p.s;
    // unit ur of the split space: all units (stream-K) or those after the raster ones (hybrid)
    const int64_t ur = blockIdx.x;
    const int u = int(split_first_unit(sc) + ur);
    if (threadIdx.x == 0) {
        int64_t c_first;
        int count;
        split_owners(sc, ur, G, c_first, count);
        first_s = c_first;
        count_s = count;
    }
    __syncthreads();
    const int count = count_s;
    if (count == 0) return;
    for (int t = threadIdx.x; t < count; t += blockDim.x) {
        const int64_t c = first_s + t;
        base[t] = (c * 2 + split_slot(sc, ur, c, G)) * BN * BM;
    }
    __syncthreads();
    const int e = blockIdx.y * blockDim.x + threadIdx.x;
    if (e >= BM * BN) return;
    const int row = e % BM, col = e / BM;
    const float* pp = p.part + int64_t(col) * BM + row;
    // four interleaved partial sums keep several loads in flight; fixed combination order
    float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
    int t = 0;
    for (; t + 4 <= count; t += 4) {
        const float a0 = pp[base[t]], a1 = pp[base[t + 1]], a2 = pp[base[t + 2]], a3 = pp[base[t + 3]];
        s0 += a0;
        s1 += a1;
        s2 += a2;
        s3 += a3;
    }
    for (; t < count; ++t) s0 += pp[base[t]];
    const float s = (s0 + s1) + (s2 + s3);
    const int64_t gr = int64_t((u / sc.tiles_n) * BM) + row;
    const int gc = (u % sc.tiles_n) * BN + col;
    if (gr < p.M && gc < p.N) {
        float* o = p.D + gr + int64_t(gc) * p.ldd;
        *o = p.beta != 0.f ? fmaf(p.alpha, s, p.beta * *o) : p.alpha * s;
    }
}

// V (rows x w float, col-major ld) -> hi, lo bf16 (col-major, ld ldo)
__global__ void k_split_bf16(const float* __restrict__ V, int64_t ldv, int64_t rows, int64_t w,
                             bf16* __restrict__ hi, bf16* __restrict__ lo, int64_t ldo) {
    const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx >= rows * w) return;
    const int64_t i = idx % rows, j = idx / rows;
    const float v = V[i + j * ldv];
    const bf16 h = __float2bfloat16_rn(v);
    hi[i + j * ldo] = h;
    if (lo) lo[i + j * ldo] = __float2bfloat16_rn(v - __bfloat162float(h));
}

// V (rows x w float, col-major ld) -> hi, mid, lo bf16 with hi + mid + lo == V exactly: each term
// is the bf16 rounding of what the previous ones left (8 significant bits each, and the float32
// remainders are exact), so three terms carry all 24 bits of a normal float32.
__global__ void k_split3_bf16(const float* __restrict__ V, int64_t ldv, int64_t rows, int64_t w,
                              bf16* __restrict__ hi, bf16* __restrict__ mid, bf16* __restrict__ lo,
                              int64_t ldo) {
    const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx >= rows * w) return;
    const int64_t i = idx % rows, j = idx / rows;
    const float v = V[i + j * ldv];
    const bf16 h = __float2bfloat16_rn(v);
    const float r1 = v - __bfloat162float(h);
    const bf16 mdl = __float2bfloat16_rn(r1);
    const float r2 = r1 - __bfloat162float(mdl);
    hi[i + j * ldo] = h;
    mid[i + j * ldo] = mdl;
    lo[i + j * ldo] = __float2bfloat16_rn(r2);
}

// ---------------------------------------------------------------- host side
typedef CUresult (*EncodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encoder() {
    static EncodeTiled fn = nullptr;
    if (!fn) {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        QB_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000,
                                                 cudaEnableDefault, &q));
        if (q != cudaDriverEntryPointSuccess || !f)
            throw Error{QB_ERR_CUDA, "cuTensorMapEncodeTiled unavailable"};
        fn = reinterpret_cast<EncodeTiled>(f);
    }
    return fn;
}

// 2-D bf16 tensor: inner extent `inner` (contiguous), `outer` rows of `ld` elements
CUtensorMap make_map(const void* ptr, int64_t inner, int64_t outer, int64_t ld, int box_inner,
                     int box_outer) {
    CUtensorMap m;
    const cuuint64_t dims[2] = {cuuint64_t(inner), cuuint64_t(outer)};
    const cuuint64_t strides[1] = {cuuint64_t(ld) * 2};
    const cuuint32_t box[2] = {cuuint32_t(box_inner), cuuint32_t(box_outer)};
    const cuuint32_t es[2] = {1, 1};
    CUresult r = encoder()(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims,
                           strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) throw Error{QB_ERR_CUDA, "cuTensorMapEncodeTiled failed"};
    return m;
}

// Column tile: 64 / 128 columns for chunked passes (the epilogue keeps one float32 register per
// column), up to 256 for wide single-chain passes.
int pick_bn(int64_t w, bool chunked) {
    if (w <= 64) return 64;
    if (w <= 128 || chunked) return 128;
    return 256;
}

// k-blocks per tensor-memory chunk: the tensor cores' float32 accumulation drifts toward zero by
// roughly 1e-9 (relative) per accumulated MMA (measured: -3.4e-6 over a 40000-long chain).  The
// narrow passes (w <= 128: randQB_EI's sketches and power steps, whose results are projected
// against Q and B) keep chains of 4 k-blocks (1 for the hi/lo passes) summed in registers; wide
// passes (randQB_FP's G = A Omega and power steps over the whole batch, where any G is valid as
// long as H = A^T G is formed from the stored G) use one chain per tile.
constexpr int SINGLE_CHAIN = 1 << 30;
int pick_chunk(int mode, int64_t w) {
    if (w > 128 && mode < 2) return SINGLE_CHAIN;
    return mode >= 2 ? 1 : 4;
}

template <int BN, bool TRANS, int NA, int NB>
void run(cudaStream_t st, const CUtensorMap& a0, const CUtensorMap& a1, const CUtensorMap& b0,
         const CUtensorMap& b1, Params p, int G) {
    using C = Cfg<BN, TRANS, NA, NB>;
    smem_limit_once<k_tc_gemm<BN, TRANS, NA, NB>>(C::SMEM);
    k_tc_gemm<BN, TRANS, NA, NB><<<G, NUM_THREADS, C::SMEM, st>>>(a0, a1, b0, b1, p);
    QB_LAUNCHED();
    if (p.s.streamk) {
        const dim3 grid(unsigned(split_units(p.s)), unsigned(BM * BN / 256));
        k_tc_fixup<BN><<<grid, 256, 0, st>>>(p, G);
        QB_LAUNCHED();
    }
}

template <bool TRANS, int NA, int NB>
void run_bn(int bn, cudaStream_t st, const CUtensorMap& a0, const CUtensorMap& a1,
            const CUtensorMap& b0, const CUtensorMap& b1, Params p, int G) {
    if (bn == 64) run<64, TRANS, NA, NB>(st, a0, a1, b0, b1, p, G);
    else if (bn == 128) run<128, TRANS, NA, NB>(st, a0, a1, b0, b1, p, G);
    else run<256, TRANS, NA, NB>(st, a0, a1, b0, b1, p, G);
}

template <int BN, bool TRANS, int NA, int NB>
void run_prec(cudaStream_t st, const CUtensorMap& a0, const CUtensorMap& a1, const CUtensorMap& a2,
              const CUtensorMap& b0, const CUtensorMap& b1, const CUtensorMap& b2, Params p, int G) {
    using C = PCfg<BN, NA, NB>;
    smem_limit_once<k_tc_prec<BN, TRANS, NA, NB>>(C::SMEM);
    k_tc_prec<BN, TRANS, NA, NB><<<G, PREC_THREADS, C::SMEM, st>>>(a0, a1, a2, b0, b1, b2, p);
    QB_LAUNCHED();
    if (p.s.streamk) {
        const dim3 grid(unsigned(split_units(p.s)), unsigned(BM * BN / 256));
        k_tc_fixup<BN><<<grid, 256, 0, st>>>(p, G);
        QB_LAUNCHED();
    }
}

template <bool TRANS, int NA, int NB>
void run_prec_bn(int bn, cudaStream_t st, const CUtensorMap& a0, const CUtensorMap& a1,
                 const CUtensorMap& a2, const CUtensorMap& b0, const CUtensorMap& b1,
                 const CUtensorMap& b2, Params p, int G) {
    if (bn == 64) run_prec<64, TRANS, NA, NB>(st, a0, a1, a2, b0, b1, b2, p, G);
    else run_prec<128, TRANS, NA, NB>(st, a0, a1, a2, b0, b1, b2, p, G);
}

struct Scratch {
    float* part;
    int* err;
    bf16* vhi;
    bf16* vlo;
    bf16* vmid;
    size_t part_bytes;
};

Scratch carve(void* scratch, size_t bytes, int64_t rows, int64_t w) {
    // [err 256 B][V hi][V lo][V mid][partials]
    char* p = reinterpret_cast<char*>(scratch);
    Scratch s;
    s.err = reinterpret_cast<int*>(p);
    const int64_t ldv = align_up(rows, 8);
    const size_t vb = size_t(align_up(ldv * w * 2, 256));
    s.vhi = reinterpret_cast<bf16*>(p + 256);
    s.vlo = reinterpret_cast<bf16*>(p + 256 + vb);
    s.vmid = reinterpret_cast<bf16*>(p + 256 + 2 * vb);
    s.part = reinterpret_cast<float*>(p + 256 + 3 * vb);
    if (256 + 3 * vb > bytes) throw Error{QB_ERR_WORKSPACE, "tensor-core scratch too small"};
    s.part_bytes = bytes - 256 - 3 * vb;
    return s;
}

// The partial slots of a split launch must fit the scratch; a hybrid schedule that does not fit
// falls back to raster, a stream-K one is an error.
void fit_partials(Sched& s, int& G, int sms, int bn, size_t part_bytes) {
    if (!s.streamk || size_t(G) * 2 * bn * BM * sizeof(float) <= part_bytes) return;
    if (s.streamk == 2) {
        s.streamk = 0;
        s.dp_units = 0;
        G = grid_size(s, sms);
        return;
    }
    throw Error{QB_ERR_WORKSPACE, "tensor-core partials"};
}

}  // namespace

int* tc_error_flag(void* scratch) { return reinterpret_cast<int*>(scratch); }

bool tc_available() {
    static int cached = -1;
    if (cached < 0) {
        int dev = 0, major = 0, minor = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return false;
        cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
        cached = (major == 10 && minor == 3) ? 1 : 0;
    }
    return cached == 1;
}

size_t tc_scratch_bytes(int64_t m, int64_t n, int64_t w) {
    const int64_t rows = std::max(m, n);
    const size_t vb = size_t(align_up(align_up(rows, 8) * w * 2, 256));
    const size_t part = size_t(MAX_SK_CTAS) * 2 * pick_bn(w, false) * BM * sizeof(float);
    return 256 + 3 * vb + part;
}

void tc_sketch(cudaStream_t st, const bf16* A, int64_t lda, int64_t m, int64_t n, const bf16* Vt,
               const bf16* Vt_lo, int64_t ldv, int64_t w, float* Y, int64_t ldy, void* scratch,
               size_t scratch_bytes) {
    if (m <= 0 || w <= 0) return;
    Scratch s = carve(scratch, scratch_bytes, 0, 0);
    const int chunk = pick_chunk(1, w);
    const int bn = pick_bn(w, chunk != SINGLE_CHAIN);
    Params p{};
    p.M = int(m);
    p.N = int(w);
    p.K = int(n);
    p.chunk = chunk;
    p.alpha = 1.f;
    p.beta = 0.f;
    int G = num_sms();
    p.s = make_sched(m, w, n, bn, G);
    G = grid_size(p.s, G);
    p.D = Y;
    p.ldd = ldy;
    p.part = s.part;
    p.err = s.err;
    fit_partials(p.s, G, num_sms(), bn, s.part_bytes);
    const CUtensorMap a = make_map(A, n, m, lda, BK, BM);
    const CUtensorMap b = make_map(Vt, n, w, ldv, BK, bn);
    if (Vt_lo) {
        const CUtensorMap b1 = make_map(Vt_lo, n, w, ldv, BK, bn);
        run_bn<false, 1, 2>(bn, st, a, a, b, b1, p, G);
    } else {
        run_bn<false, 1, 1>(bn, st, a, a, b, b, p, G);
    }
}

void tc_trans(cudaStream_t st, const bf16* A_hi, const bf16* A_lo, int64_t lda, int64_t m,
              int64_t n, const float* V, int64_t ldv, int64_t w, float* Z, int64_t ldz, int mode,
              void* scratch, size_t scratch_bytes) {
    if (n <= 0 || w <= 0) return;
    if (mode < 1 || mode > 4) throw Error{QB_ERR_INVALID_ARG, "tc_trans mode"};
    Scratch s = carve(scratch, scratch_bytes, m, w);
    const int64_t ldo = align_up(m, 8);
    if (mode == 3) {
        k_split3_bf16<<<unsigned(cdiv(m * w, 256)), 256, 0, st>>>(V, ldv, m, w, s.vhi, s.vmid,
                                                                  s.vlo, ldo);
    } else {
        // mode 4: V holds two-term bf16 values, V = hi + (V - hi) exactly
        k_split_bf16<<<unsigned(cdiv(m * w, 256)), 256, 0, st>>>(V, ldv, m, w, s.vhi,
                                                                 mode == 4 ? s.vmid : nullptr, ldo);
    }
    QB_LAUNCHED();
    const int bn = mode == 1 ? pick_bn(w, pick_chunk(1, w) != SINGLE_CHAIN) : (w <= 64 ? 64 : 128);
    Params p{};
    p.M = int(n);
    p.N = int(w);
    p.K = int(m);
    p.chunk = pick_chunk(1, w);
    p.alpha = 1.f;
    p.beta = 0.f;
    int G = num_sms();
    p.s = make_sched(n, w, m, bn, G);
    G = grid_size(p.s, G);
    p.D = Z;
    p.ldd = ldz;
    p.part = s.part;
    p.err = s.err;
    fit_partials(p.s, G, num_sms(), bn, s.part_bytes);
    // A as an (n inner, m outer) tensor; boxes of 64 columns x 64 rows
    const CUtensorMap a0 = make_map(A_hi, n, m, lda, 64, BK);
    const CUtensorMap b0 = make_map(s.vhi, m, w, ldo, BK, bn);
    if (mode == 1) {
        run_bn<true, 1, 1>(bn, st, a0, a0, b0, b0, p, G);
        return;
    }
    const CUtensorMap a1 = A_lo ? make_map(A_lo, n, m, lda, 64, BK) : a0;
    if (mode == 2) {
        if (A_lo) run_prec_bn<true, 2, 1>(bn, st, a0, a1, a1, b0, b0, b0, p, G);
        else run_prec_bn<true, 1, 1>(bn, st, a0, a0, a0, b0, b0, b0, p, G);
        return;
    }
    const CUtensorMap b1 = make_map(s.vmid, m, w, ldo, BK, bn);
    if (mode == 4) {
        if (A_lo) run_prec_bn<true, 2, 2>(bn, st, a0, a1, a1, b0, b1, b1, p, G);
        else run_prec_bn<true, 1, 2>(bn, st, a0, a0, a0, b0, b1, b1, p, G);
        return;
    }
    const CUtensorMap b2 = make_map(s.vlo, m, w, ldo, BK, bn);
    if (A_lo) run_prec_bn<true, 2, 3>(bn, st, a0, a1, a1, b0, b1, b2, p, G);
    else run_prec_bn<true, 1, 3>(bn, st, a0, a0, a0, b0, b1, b2, p, G);
}

// D (M x N, column-major, ldd) = alpha op(A) V + beta D with A given exactly by na bf16 terms
// (shared leading dimension lda, 16-byte aligned) and V float32 column-major K x N (ldv), split
// exactly into three bf16 terms on the fly; N <= 64.
//   trans = false: A is M rows x K columns row-major (op(A) = A; the "TN" product X^T V for a
//                  column-major K x M matrix X);
//   trans = true : A is K rows x M columns row-major (op(A) = A^T; the "NN" product X V for a
//                  column-major M x K matrix X).
// Leading product per MMA in registers (round-to-nearest), lower-order products with weight
// >= 2^-18 in a tensor-memory chain; float32-level accuracy.
void tc_prec_gemm(cudaStream_t st, bool trans, const bf16* const* A, int na, int64_t lda,
                  int64_t M, int64_t K, const float* V, int64_t ldv, int64_t N, float alpha,
                  float beta, float* D, int64_t ldd, void* scratch, size_t scratch_bytes) {
    if (N > 64) throw Error{QB_ERR_INVALID_ARG, "tc_prec_gemm shape"};
    tc_prec_gemm2(st, trans, A, na, lda, M, K, V, ldv, N, nullptr, 0, 0, alpha, beta, D, ldd,
                  scratch, scratch_bytes);
}

// The same product with the operand [V1 | V2] (N1 + N2 <= 128 columns, each block column-major
// with its own ld): both are split into one scratch operand and the output has N1 + N2 columns.
// Above 64 columns the tile is 128 wide (trans = false, three A terms only), so each A tile is
// read once for all the columns.
void tc_prec_gemm2(cudaStream_t st, bool trans, const bf16* const* A, int na, int64_t lda,
                   int64_t M, int64_t K, const float* V1, int64_t ldv1, int64_t N1,
                   const float* V2, int64_t ldv2, int64_t N2, float alpha, float beta, float* D,
                   int64_t ldd, void* scratch, size_t scratch_bytes) {
    const int64_t N = N1 + std::max<int64_t>(N2, 0);
    if (M <= 0 || N <= 0) return;
    if (na < 1 || na > 3 || N1 < 0 || N > 128 || (N2 > 0 && !V2) || lda % 8 != 0)
        throw Error{QB_ERR_INVALID_ARG, "tc_prec_gemm shape"};
    Scratch s = carve(scratch, scratch_bytes, K, N);
    const int64_t ldo = align_up(std::max<int64_t>(K, 1), 8);
    if (K > 0) {
        if (N1 > 0) {
            k_split3_bf16<<<unsigned(cdiv(K * N1, 256)), 256, 0, st>>>(V1, ldv1, K, N1, s.vhi,
                                                                       s.vmid, s.vlo, ldo);
            QB_LAUNCHED();
        }
        if (N2 > 0) {
            const int64_t o = N1 * ldo;
            k_split3_bf16<<<unsigned(cdiv(K * N2, 256)), 256, 0, st>>>(V2, ldv2, K, N2, s.vhi + o,
                                                                       s.vmid + o, s.vlo + o, ldo);
            QB_LAUNCHED();
        }
    }
    const int bn = N > 64 ? 128 : 64;
    if (bn == 128 && (trans || na != 3)) throw Error{QB_ERR_INVALID_ARG, "tc_prec_gemm shape"};
    Params p{};
    p.M = int(M);
    p.N = int(N);
    p.K = int(std::max<int64_t>(K, 1));
    p.chunk = 1;
    p.alpha = alpha;
    p.beta = beta;
    int G = num_sms();
    p.s = make_sched(M, N, std::max<int64_t>(K, 1), bn, G);
    G = grid_size(p.s, G);
    p.D = D;
    p.ldd = ldd;
    p.part = s.part;
    p.err = s.err;
    fit_partials(p.s, G, num_sms(), bn, s.part_bytes);
    const int64_t Kd = std::max<int64_t>(K, 1);
    CUtensorMap am[3];
    for (int i = 0; i < 3; ++i) {
        const bf16* ai = A[std::min(i, na - 1)];
        am[i] = trans ? make_map(ai, M, Kd, lda, 64, BK) : make_map(ai, Kd, M, lda, BK, BM);
    }
    const CUtensorMap b0 = make_map(s.vhi, Kd, N, ldo, BK, bn);
    const CUtensorMap b1 = make_map(s.vmid, Kd, N, ldo, BK, bn);
    const CUtensorMap b2 = make_map(s.vlo, Kd, N, ldo, BK, bn);
    if (trans) {
        if (na == 3) run_prec<64, true, 3, 3>(st, am[0], am[1], am[2], b0, b1, b2, p, G);
        else if (na == 2) run_prec<64, true, 2, 3>(st, am[0], am[1], am[2], b0, b1, b2, p, G);
        else run_prec<64, true, 1, 3>(st, am[0], am[1], am[2], b0, b1, b2, p, G);
    } else if (bn == 128) {
        run_prec<128, false, 3, 3>(st, am[0], am[1], am[2], b0, b1, b2, p, G);
    } else {
        if (na == 3) run_prec<64, false, 3, 3>(st, am[0], am[1], am[2], b0, b1, b2, p, G);
        else if (na == 2) run_prec<64, false, 2, 3>(st, am[0], am[1], am[2], b0, b1, b2, p, G);
        else run_prec<64, false, 1, 3>(st, am[0], am[1], am[2], b0, b1, b2, p, G);
    }
}

// Three exact bf16 terms of a float32 column-major block (hi + mid + lo == X).
void split3_bf16(cudaStream_t st, const float* X, int64_t ldx, int64_t rows, int64_t cols, bf16* hi,
                 bf16* mid, bf16* lo, int64_t ldo) {
    if (rows <= 0 || cols <= 0) return;
    k_split3_bf16<<<unsigned(cdiv(rows * cols, 256)), 256, 0, st>>>(X, ldx, rows, cols, hi, mid, lo,
                                                                    ldo);
    QB_LAUNCHED();
}

// T (j0 x bw, col-major, ldt) = X^T P for X column-major rows x j0 held as bf16 hi [+ lo] (ldx),
// P float32 column-major rows x bw (ldp), split to bf16 hi [+ lo] on the fly.  Tensor cores,
// chunked accumulation.  Products: X_hi P_hi [+ X_lo P_hi + X_hi P_lo when X_lo != nullptr].
void tc_xtp(cudaStream_t st, const bf16* Xhi, const bf16* Xlo, int64_t ldx, int64_t rows,
            int64_t j0, const float* P, int64_t ldp, int64_t bw, float* T, int64_t ldt,
            void* scratch, size_t scratch_bytes) {
    if (j0 <= 0 || bw <= 0) return;
    // scratch: [err 256][P hi][P lo][partials]
    Scratch s = carve(scratch, scratch_bytes, rows, bw);
    const int64_t ldb = align_up(rows, 8);
    k_split_bf16<<<unsigned(cdiv(rows * bw, 256)), 256, 0, st>>>(P, ldp, rows, bw, s.vhi,
                                                              Xlo ? s.vlo : nullptr, ldb);
    QB_LAUNCHED();
    const int chunk = pick_chunk(Xlo ? 3 : 1, bw);
    const int bn = pick_bn(bw, true);
    Params p{};
    p.M = int(j0);
    p.N = int(bw);
    p.K = int(rows);
    p.chunk = chunk;
    p.alpha = 1.f;
    p.beta = 0.f;
    int G = num_sms();
    p.s = make_sched(j0, bw, rows, bn, G);
    G = grid_size(p.s, G);
    p.D = T;
    p.ldd = ldt;
    p.part = s.part;
    p.err = s.err;
    fit_partials(p.s, G, num_sms(), bn, s.part_bytes);
    // "A" operand: X^T as a row-major j0 x rows matrix = X column-major
    const CUtensorMap a0 = make_map(Xhi, rows, j0, ldx, BK, BM);
    const CUtensorMap b0 = make_map(s.vhi, rows, bw, ldb, BK, bn);
    if (!Xlo) {
        run_bn<false, 1, 1>(bn, st, a0, a0, b0, b0, p, G);
        return;
    }
    const CUtensorMap a1 = make_map(Xlo, rows, j0, ldx, BK, BM);
    const CUtensorMap b1 = make_map(s.vlo, rows, bw, ldb, BK, bn);
    run_bn<false, 2, 2>(bn, st, a0, a1, b0, b1, p, G);
}

// P (rows x bw, col-major, ldp) -= X T for X column-major rows x j0 (bf16 hi [+ lo], ldx) and
// T float32 j0 x bw (ldt), split to bf16 on the fly.  Tensor cores, chunked accumulation.
void tc_p_minus_xt(cudaStream_t st, const bf16* Xhi, const bf16* Xlo, int64_t ldx, int64_t rows,
                   int64_t j0, const float* T, int64_t ldt, int64_t bw, float* P, int64_t ldp,
                   void* scratch, size_t scratch_bytes) {
    if (j0 <= 0 || bw <= 0 || rows <= 0) return;
    Scratch s = carve(scratch, scratch_bytes, j0, bw);
    const int64_t ldo = align_up(j0, 8);
    k_split_bf16<<<unsigned(cdiv(j0 * bw, 256)), 256, 0, st>>>(T, ldt, j0, bw, s.vhi,
                                                             Xlo ? s.vlo : nullptr, ldo);
    QB_LAUNCHED();
    const int chunk = pick_chunk(Xlo ? 3 : 1, bw);
    const int bn = pick_bn(bw, true);
    Params p{};
    p.M = int(rows);
    p.N = int(bw);
    p.K = int(j0);
    p.chunk = chunk;
    p.alpha = -1.f;
    p.beta = 1.f;
    int G = num_sms();
    p.s = make_sched(rows, bw, j0, bn, G);
    G = grid_size(p.s, G);
    p.D = P;
    p.ldd = ldp;
    p.part = s.part;
    p.err = s.err;
    fit_partials(p.s, G, num_sms(), bn, s.part_bytes);
    // "A" operand of the transposed form: X^T as a row-major j0 x rows tensor (K = j0, M = rows)
    const CUtensorMap a0 = make_map(Xhi, rows, j0, ldx, 64, BK);
    const CUtensorMap b0 = make_map(s.vhi, j0, bw, ldo, BK, bn);
    if (!Xlo) {
        run_bn<true, 1, 1>(bn, st, a0, a0, b0, b0, p, G);
        return;
    }
    const CUtensorMap a1 = make_map(Xlo, rows, j0, ldx, 64, BK);
    const CUtensorMap b1 = make_map(s.vlo, j0, bw, ldo, BK, bn);
    run_bn<true, 2, 2>(bn, st, a0, a1, b0, b1, p, G);
}

void split_bf16(cudaStream_t st, const float* V, int64_t ldv, int64_t rows, int64_t w, bf16* hi,
                bf16* lo, int64_t ldo) {
    if (rows <= 0 || w <= 0) return;
    k_split_bf16<<<unsigned(cdiv(rows * w, 256)), 256, 0, st>>>(V, ldv, rows, w, hi, lo, ldo);
    QB_LAUNCHED();
}

// Round a float32 column-major block to bf16-representable values in place.
// pairs == 1: X <- bf16(X); pairs == 2: X <- bf16(X) + bf16(X - bf16(X)) (16 significant bits)
__global__ void k_round_bf16(float* X, int64_t ldx, int64_t rows, int64_t cols, int pairs) {
    const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx >= rows * cols) return;
    const int64_t i = idx % rows, j = idx / rows;
    float& v = X[i + j * ldx];
    const float h = __bfloat162float(__float2bfloat16_rn(v));
    v = pairs == 1 ? h : h + __bfloat162float(__float2bfloat16_rn(v - h));
}

void round_bf16_inplace(cudaStream_t st, float* X, int64_t ldx, int64_t rows, int64_t cols,
                        int pairs) {
    if (rows <= 0 || cols <= 0) return;
    k_round_bf16<<<unsigned(cdiv(rows * cols, 256)), 256, 0, st>>>(X, ldx, rows, cols, pairs);
    QB_LAUNCHED();
}

}  // namespace qb

// ============================================================================ allocation-free pass
// A variant of the tensor-core sketch pass Y = A_hi V for callers that cannot allocate device
// memory and cannot hand the library a workspace.  Its scratch (the bf16 copy of V, the stream-K
// partial tiles and the wait-timeout flag) lives in one file-scope device array that every GPU
// loading this library reserves until the process exits.
namespace {
constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(16) << 20;   // 16 MiB
constexpr int64_t NOALLOC_MAX_W = 64;
}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

namespace qb {
namespace {
// Device address of g_noalloc_scratch on the current device, looked up once per device.
void* noalloc_scratch_address() {
    static std::mutex mu;
    static void* addr[64] = {};
    int dev = 0;
    QB_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) throw Error{QB_ERR_UNSUPPORTED, "device index"};
    std::lock_guard<std::mutex> lk(mu);
    if (!addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            record_cuda_error(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
            throw Error{QB_ERR_CUDA, "cudaGetSymbolAddress failed"};
        }
        addr[dev] = p;
    }
    return addr[dev];
}
}  // namespace

// bytes of the shared array a call with these sizes uses
size_t noalloc_bytes(int64_t n, int64_t w) {
    const size_t vcopy = size_t(align_up(align_up(n, 8) * w * 2, 256));
    const size_t part = size_t(MAX_SK_CTAS) * 2 * pick_bn(w, false) * BM * sizeof(float);
    return vcopy + 256 + part;
}
}  // namespace qb

extern "C" int32_t qb_apass_sketch_noalloc(const qb_dense* A, const float* V, int64_t ldv,
                                           int64_t w, float* Y, int64_t ldy, void* stream) {
    using namespace qb;
    if (!A || !V || !Y || A->m < 128 || A->n < 128 || w < 1 || ldv < A->n || ldy < A->m)
        return QB_ERR_INVALID_ARG;
    if (A->dtype != QB_BF16 && A->dtype != QB_BF16X2) return QB_ERR_UNSUPPORTED;
    if (A->ld < A->n || A->ld % 8 != 0 || (reinterpret_cast<uintptr_t>(A->a) & 15) != 0)
        return QB_ERR_UNSUPPORTED;
    if (w > NOALLOC_MAX_W || noalloc_bytes(A->n, w) > NOALLOC_SCRATCH_BYTES)
        return QB_ERR_WORKSPACE;   // beyond the fixed array: use qb_apass_sketch with a workspace
    try {
        if (!tc_available()) return QB_ERR_UNSUPPORTED;
        cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
        char* base = reinterpret_cast<char*>(noalloc_scratch_address());
        const int64_t ldb = align_up(A->n, 8);
        bf16* vb = reinterpret_cast<bf16*>(base);
        char* tcs = base + align_up(ldb * w * 2, 256);
        const size_t tcs_bytes = NOALLOC_SCRATCH_BYTES - size_t(tcs - base);
        // the array keeps the previous call's contents: the timeout flag must start at zero
        QB_CUDA(cudaMemsetAsync(tc_error_flag(tcs), 0, 256, st));
        split_bf16(st, V, ldv, A->n, w, vb, nullptr, ldb);
        tc_sketch(st, reinterpret_cast<const bf16*>(A->a), A->ld, A->m, A->n, vb, nullptr, ldb, w,
                  Y, ldy, tcs, tcs_bytes);
        int flag = 0;
        QB_CUDA(cudaMemcpyAsync(&flag, tc_error_flag(tcs), sizeof flag, cudaMemcpyDeviceToHost, st));
        QB_CUDA(cudaStreamSynchronize(st));
        return flag ? QB_ERR_TIMEOUT : QB_OK;
    } catch (const Error& e) {
        return e.code;
    } catch (...) {
        return QB_ERR_CUDA;
    }
}
