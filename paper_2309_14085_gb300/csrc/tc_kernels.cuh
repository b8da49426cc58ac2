// Tensor-core block-row GEMM for products with many right-hand sides (sm_100a /
// sm_103a, tcgen05).  A task of the block-row form (P2M, M2M, M2L, L2L, stored
// leaf rows) computes Y[dst + i][c] (+)= sum_k A[i * kpad + k] X[k][c] for
// i < rows and an NT-column tile c of the RHS; with NT = 64 every operator
// entry streamed from HBM feeds 64 multiply-adds, so the contraction runs on the
// 5th-generation tensor cores instead of re-streaming the operators per
// CUDA-core tile.
//
// Per CTA (256 threads = 8 warps; persistent: tasks blockIdx.x, + gridDim.x, ...):
//   * warp 0 allocates NT columns of tensor memory (TMEM) for the 128 x NT fp32
//     accumulator once, and the chunk mbarriers are initialised once;
//   * the K dimension runs in chunks of 128 bytes per row (64 bf16 or 32 fp32
//     entries); all threads stage a chunk of A (the task's rows only: rows of
//     the 128-row MMA beyond them hold stale data and produce accumulator rows
//     that are never read) and of X (NT columns, gathered from the task's coefficient segments,
//     converted to the MMA input type) into shared memory in the canonical
//     no-swizzle K-major layout: 8-row x 16-byte core matrices, 128 B apart
//     along K (leading byte offset) and 1024 B apart along M / N (stride byte
//     offset);
//   * thread 0 issues four tcgen05.mma per chunk (K = 32 bytes each) and
//     commits them to the chunk's mbarrier; two chunk buffers alternate, and
//     each thread issues the global loads of chunk g + 1 (into registers) right
//     after storing chunk g, so they fly during the barrier and the MMAs;
//   * warp w reads accumulator rows 32 (w mod 4) .. + 31, columns of half
//     w / 4, back with tcgen05.ld and adds them to Y (fp32).
// Staging maps a warp onto 8 rows (or RHS columns) x 4 words of one 16-byte
// core-matrix slot, so its shared-memory stores hit all 32 banks once; each
// thread issues all its global loads of a chunk before its stores.
// Every mbarrier wait is bounded: on expiry the CTA records an error code in
// *err, waits (bounded) for its MMAs in flight, frees its TMEM and returns.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace h2 {
namespace tc {

constexpr int kThreads = 256;           // 8 warps
constexpr int kRowsTile = 128;              // MMA M
constexpr int kChunkBytes = 128;            // K bytes per row per chunk
constexpr int kATileBytes = kRowsTile * kChunkBytes;
constexpr uint32_t kWaitLimit = 1u << 22;   // try_wait rounds before giving up
constexpr int kErrTimeout = 1;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

// true once the phase of the given parity has completed; false after `limit` rounds
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t limit) {
    for (uint32_t it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void fence_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// warp-wide: allocate ncols TMEM columns, address written to *dst
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(smem_u32(dst)), "r"(ncols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
                 : "memory");
}

// Shared-memory matrix descriptor (tcgen05 format): start address, leading
// (K-direction) and stride (M/N-direction) byte offsets in 16-byte units,
// descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = uint64_t((addr >> 4) & 0x3FFFu);
    d |= uint64_t((lbo >> 4) & 0x3FFFu) << 16;
    d |= uint64_t((sbo >> 4) & 0x3FFFu) << 32;
    d |= uint64_t(1) << 46;
    return d;
}

// Instruction descriptor: fp32 accumulator, A/B format `fmt` (1 = bf16 under
// kind::f16, 2 = tf32 under kind::tf32), both K-major, N >> 3, M >> 4.
__host__ __device__ constexpr uint32_t instr_desc(uint32_t fmt, int M, int N) {
    return (1u << 4) | (fmt << 7) | (fmt << 10) | (uint32_t(N >> 3) << 17) | (uint32_t(M >> 4) << 24);
}

template <bool BF>
__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                    uint32_t accumulate) {
    if constexpr (BF) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
            ::"r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(accumulate) : "memory");
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
            ::"r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(accumulate) : "memory");
    }
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(smem_u32(bar)) : "memory");
}

// 32 lanes x 32 bits, 8 consecutive columns: thread t of the warp receives
// row (lane base + t), columns col .. col + 7
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
    uint32_t r[8];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = __uint_as_float(r[k]);
}

// byte offset of (row r, K byte kb) in a staged tile (no-swizzle K-major)
__device__ __forceinline__ uint32_t tile_off(int r, int kb) {
    return uint32_t((r >> 3) * 1024 + (kb >> 4) * 128 + (r & 7) * 16 + (kb & 15));
}

template <typename S> struct In;
template <> struct In<__nv_bfloat16> {
    using T = __nv_bfloat16;                 // MMA input element
    static constexpr bool BF = true;
    static constexpr uint32_t FMT = 1;
    static constexpr int KPW = 2;            // K entries per 32-bit word
    // two consecutive K entries of one column -> one word (lower K in the low half)
    __device__ static uint32_t pack(const float (&x)[2]) {
        const __nv_bfloat162 b = __floats2bfloat162_rn(x[0], x[1]);
        return *reinterpret_cast<const uint32_t*>(&b);
    }
};
template <> struct In<float> {
    using T = float;                         // tf32: fp32 container, tf32 multiply
    static constexpr bool BF = false;
    static constexpr uint32_t FMT = 2;
    static constexpr int KPW = 1;
    __device__ static uint32_t pack(const float (&x)[1]) { return __float_as_uint(x[0]); }
};

}  // namespace tc

// Block-row GEMM on tensor cores; S = stored operator type (bf16 or fp32),
// coefficients are fp32.  Dynamic shared memory: tc_smem_bytes<S, NT>().
template <typename S, int NT>
__host__ __device__ constexpr int tc_smem_bytes() {
    return 2 * (tc::kATileBytes + NT * tc::kChunkBytes) + 2 * (tc::kChunkBytes / int(sizeof(S))) * 8 + 64;
}

template <typename S, int NT>
__global__ void __launch_bounds__(tc::kThreads, 3) k_rowgemm_tc(
    int64_t ntask, const int64_t* __restrict__ dst, const int32_t* __restrict__ rows,
    const int32_t* __restrict__ kpad, const int64_t* __restrict__ aoff,
    const int64_t* __restrict__ seg_ptr, const int64_t* __restrict__ seg_off,
    const int32_t* __restrict__ seg_len, const int32_t* __restrict__ seg_col,
    const S* __restrict__ ops, float* __restrict__ vec, int accumulate, int nrhs, int c0,
    int* __restrict__ err) {
    using In = tc::In<S>;
    static_assert(NT == 16 || NT == 32 || NT == 64, "RHS tile");
    constexpr int ES = int(sizeof(S));
    constexpr int KC = tc::kChunkBytes / ES;            // K entries per chunk
    constexpr int KPW = In::KPW;
    constexpr int kBTileBytes = NT * tc::kChunkBytes;
    constexpr int kBufBytes = tc::kATileBytes + kBTileBytes;
    constexpr uint32_t kCols = NT < 32 ? 32 : NT;       // TMEM columns (power of 2, >= 32)
    constexpr uint32_t kIdesc = tc::instr_desc(In::FMT, tc::kRowsTile, NT);
    constexpr int kAUnits = tc::kRowsTile * 16;         // 8-byte units of a full A tile
    constexpr int kAPer = kAUnits / tc::kThreads;       // per thread
    constexpr int kBItems = KC * NT / KPW;              // 32-bit words of a B tile
    constexpr int kBPer = kBItems / tc::kThreads;
    static_assert(kBItems % tc::kThreads == 0 && kAUnits % tc::kThreads == 0, "staging split");
    extern __shared__ __align__(1024) uint8_t smem[];
    int64_t* tab = reinterpret_cast<int64_t*>(smem + 2 * kBufBytes);   // [2][KC] sources
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + 2 * kBufBytes + 2 * KC * 8);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + 2);
    int* fail = reinterpret_cast<int*>(tmem_slot + 1);

    if (int64_t(blockIdx.x) >= ntask) return;
    const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
    if (warp == 0) tc::tmem_alloc(tmem_slot, kCols);
    if (tid == 0) {
        tc::mbar_init(&bar[0], 1);
        tc::mbar_init(&bar[1], 1);
        *fail = 0;
        tc::fence_async_smem();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    uint32_t g = 0;                                      // chunks issued by this CTA
    bool ok = true;
    uint2 av[kAPer];                                     // staged loads of the next chunk
    float bv[kBPer][KPW];

    for (int64_t t = blockIdx.x; t < ntask && ok; t += gridDim.x) {
        const int kp = kpad[t];
        const int nr = rows[t];
        const int64_t e0 = seg_ptr[t], e1 = seg_ptr[t + 1];
        const S* Am = ops + aoff[t];
        float* y = vec + dst[t] * nrhs + c0;
        const int ncols = min(NT, nrhs - c0);
        const int nchunk = (kp + KC - 1) / KC;
        if (nchunk == 0) {                               // no columns: y = 0 (or unchanged)
            for (int j = tid; j < nr * ncols && !accumulate; j += tc::kThreads)
                y[int64_t(j / ncols) * nrhs + (j % ncols)] = 0.0f;
        }
        // source coefficient of every K entry of chunk ch (-1: zero), into table slot
        auto build_table = [&](int ch, int slot) {
            if (tid < KC) {
                const int k = ch * KC + tid;
                int64_t si = -1;
                for (int64_t e = e0; e < e1; ++e) {
                    const int sc = seg_col[e];
                    if (k < sc) break;
                    if (k < sc + seg_len[e]) { si = seg_off[e] + (k - sc); break; }
                }
                tab[slot * KC + tid] = si;
            }
        };
        // global loads of chunk ch into registers (A: 8 rows x 4 units per warp;
        // X: column c_lo = lane & 7 of a group of 8, word (lane >> 3) & 3 of the slot)
        auto load_chunk = [&](int m0, int mt, int ch, int slot) {
            const int k0 = ch * KC;
#pragma unroll
            for (int i = 0; i < kAPer; ++i) {
                const int u = tid + i * tc::kThreads;
                const int r = (u >> 7) * 8 + (u & 7), q = (u >> 3) & 15;
                const int kk = k0 + q * (8 / ES);
                av[i] = make_uint2(0u, 0u);
                if (r < mt && kk < kp)
                    av[i] = __ldg(reinterpret_cast<const uint2*>(Am + int64_t(m0 + r) * kp + kk));
            }
            const int64_t* src = tab + slot * KC;
#pragma unroll
            for (int i = 0; i < kBPer; ++i) {
                const int v = tid + i * tc::kThreads;
                const int c = ((v >> 5) % (NT / 8)) * 8 + (v & 7);
                const int kb = ((v >> 5) / (NT / 8)) * (4 * KPW) + ((v >> 3) & 3) * KPW;
#pragma unroll
                for (int j = 0; j < KPW; ++j) {
                    const int64_t si = src[kb + j];
                    bv[i][j] = (si >= 0 && c < ncols) ? vec[si * nrhs + c0 + c] : 0.0f;
                }
            }
        };
        for (int m0 = 0; m0 < nr && ok && nchunk > 0; m0 += tc::kRowsTile) {
            const int mt = min(tc::kRowsTile, nr - m0);  // rows of this tile
            // prologue: chunk 0's table and loads
            build_table(0, int(g & 1));
            __syncthreads();
            load_chunk(m0, mt, 0, int(g & 1));
            for (int ch = 0; ch < nchunk; ++ch, ++g) {
                const int b = int(g & 1);
                uint8_t* At = smem + b * kBufBytes;
                uint8_t* Bt = At + tc::kATileBytes;
                if (ch + 1 < nchunk) build_table(ch + 1, b ^ 1);
                if (g >= 2) {                            // MMAs of chunk g - 2 read this buffer
                    if (tid == 0 && !tc::mbar_wait(&bar[b], ((g - 2) >> 1) & 1, tc::kWaitLimit)) *fail = 1;
                }
                __syncthreads();
                if (*fail) { ok = false; break; }
#pragma unroll
                for (int i = 0; i < kAPer; ++i) {
                    const int u = tid + i * tc::kThreads;
                    const int r = (u >> 7) * 8 + (u & 7), q = (u >> 3) & 15;
                    if (r < mt) *reinterpret_cast<uint2*>(At + tc::tile_off(r, q * 8)) = av[i];
                }
#pragma unroll
                for (int i = 0; i < kBPer; ++i) {
                    const int v = tid + i * tc::kThreads;
                    const int c = ((v >> 5) % (NT / 8)) * 8 + (v & 7);
                    const int kb = ((v >> 5) / (NT / 8)) * (4 * KPW) + ((v >> 3) & 3) * KPW;
                    *reinterpret_cast<uint32_t*>(Bt + tc::tile_off(c, kb * ES)) = In::pack(bv[i]);
                }
                // the next chunk's loads fly during the barrier and the MMA issue
                if (ch + 1 < nchunk) load_chunk(m0, mt, ch + 1, b ^ 1);
                tc::fence_async_smem();
                __syncthreads();
                if (tid == 0) {
                    tc::tc_fence_after();
                    const uint32_t a0 = tc::smem_u32(At), b0 = tc::smem_u32(Bt);
#pragma unroll
                    for (int s = 0; s < tc::kChunkBytes / 32; ++s) {   // K = 32 bytes per MMA
                        const uint64_t ad = tc::smem_desc(a0 + s * 256, 128, 1024);
                        const uint64_t bd = tc::smem_desc(b0 + s * 256, 128, 1024);
                        tc::mma<In::BF>(tmem, ad, bd, kIdesc, (ch > 0 || s > 0) ? 1u : 0u);
                    }
                    tc::mma_commit(&bar[b]);
                }
            }
            if (!ok) break;
            // all MMAs of this row tile complete (the last commit covers earlier ones)
            if (tid == 0 && g > 0 && !tc::mbar_wait(&bar[(g - 1) & 1], ((g - 1) >> 1) & 1, tc::kWaitLimit))
                *fail = 1;
            __syncthreads();
            if (*fail) { ok = false; break; }
            tc::tc_fence_after();
            const int quarter = warp & 3, half = warp >> 2;
            const int row = m0 + quarter * 32 + lane;
            const uint32_t tbase = tmem + (uint32_t(quarter * 32) << 16);
#pragma unroll
            for (int c8 = half * (NT / 2); c8 < (half + 1) * (NT / 2); c8 += 8) {
                float v[8];
                tc::tmem_ld8(tbase + uint32_t(c8), v);
                if (row < nr) {
                    float* yo = y + int64_t(row) * nrhs + c8;
#pragma unroll
                    for (int k = 0; k < 8; ++k)
                        if (c8 + k < ncols) yo[k] = accumulate ? yo[k] + v[k] : v[k];
                }
            }
            tc::tc_fence_before();
            __syncthreads();                             // TMEM reads done before the next tile
            tc::tc_fence_after();
        }
    }
    if (!ok) {
        // bounded wait for the MMAs still in flight before the TMEM is released
        if (tid == 0) {
            atomicExch(err, tc::kErrTimeout);
            if (g > 0) tc::mbar_wait(&bar[(g - 1) & 1], ((g - 1) >> 1) & 1, tc::kWaitLimit);
        }
        __syncthreads();
    }
    if (warp == 0) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, kCols);
    }
}

// The expiry path of the bounded waits above, without a fault: one warp
// allocates TMEM, waits at most `rounds` try_wait rounds on an mbarrier that
// nothing arrives on, records kErrTimeout in *err, frees its TMEM and returns.
// Launch: one block of 32 threads, no dynamic shared memory.
__global__ void __launch_bounds__(32, 1) k_wait_expiry(uint32_t rounds, int* __restrict__ err) {
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tmem_slot;
    tc::tmem_alloc(&tmem_slot, 32);
    if (threadIdx.x == 0) {
        tc::mbar_init(&bar, 1);
        tc::fence_async_smem();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = tmem_slot;
    if (threadIdx.x == 0 && !tc::mbar_wait(&bar, 0, rounds)) atomicExch(err, tc::kErrTimeout);
    __syncthreads();
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, 32);
}

}  // namespace h2
