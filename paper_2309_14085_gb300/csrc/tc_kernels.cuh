// Tensor-core block-row GEMM for products with many right-hand sides (sm_100a /
// sm_103a, tcgen05).  A task of the block-row form (P2M, M2M, M2L, L2L, stored
// leaf rows) computes Y[dst + i][c] (+)= sum_k A[i * kpad + k] X[k][c] for
// i < rows and an NT-column tile c of the RHS; with NT = 64 every operator
// entry streamed from HBM feeds 64 multiply-adds, so the contraction runs on the
// 5th-generation tensor cores instead of re-streaming the operators per
// CUDA-core tile.  The kernel (k_rowgemm_tc, below) is warp-specialised:
// producer warps fill a ring of shared-memory stages with cp.async copies of
// the operator rows and gathered coefficients, one thread issues tcgen05.mma
// into one of two TMEM accumulators, epilogue warps drain the other.  fp32
// operators run as a 3-term tf32 product (hi / lo split of both operands), so
// the result carries ~2^-21 relative rounding per product instead of tf32's
// 2^-11; bf16 operators run as one bf16 product.
//
// Shared-memory tiles use the canonical no-swizzle K-major layout: 8-row x
// 16-byte core matrices, 128 B apart along K (leading byte offset) and 8 kCB
// bytes apart along M / N (stride byte offset).  Every mbarrier wait is bounded: on
// expiry the CTA records an error code in *err, waits (bounded) for its MMAs in
// flight, frees its TMEM and returns.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace h2 {
namespace tc {

constexpr int kRowsTile = 128;              // MMA M
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


// asynchronous global -> shared copies (cp.async) of 16 bytes (L2 only), 8 or 4
// bytes; bytes past src_bytes (0 .. size) are zero-filled and not read
__device__ __forceinline__ void cp_async16(void* dst, const void* src, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src),
                 "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src, int src_bytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(smem_u32(dst)), "l"(src),
                 "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src, int src_bytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(smem_u32(dst)), "l"(src),
                 "r"(src_bytes) : "memory");
}
// one arrival on `bar` once every cp.async this thread issued so far has
// landed (the barrier's count includes these arrivals)
__device__ __forceinline__ void cp_async_arrive(uint64_t* bar) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar))
                 : "memory");
}
// barrier `id` (1..15) among `n` threads of the CTA (a multiple of 32)
__device__ __forceinline__ void named_sync(int id, int n) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}

// x = hi + lo with hi on the tf32 grid (10 fraction bits, rounded to nearest)
// and lo = x - hi exact in fp32 (|lo| <= 2^-11 |x|): the terms of the 3-term
// tf32 product a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi (the dropped a_lo b_lo
// and the tf32 rounding of the lo terms leave ~2^-21 of |a b|)
__device__ __forceinline__ void split_tf32(float x, float& hi, float& lo) {
    hi = __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
    lo = x - hi;
}

// Warp roles of the block-row GEMM: 4 producer warps, 4 epilogue warps (warp
// 4 + q reads TMEM lanes 32 q .. 32 q + 31), 1 MMA warp (TMEM owner).
constexpr int kProducerWarps = 4;
constexpr int kProducerThreads = 32 * kProducerWarps;
constexpr int kEpiThreads = 128;
constexpr int kMmaWarp = 8;
constexpr int kThreadsWs = 32 * 9;
constexpr int kCB = 64;                         // K bytes per row per pipeline chunk

// byte offset of (row r, K byte kb < kCB) in a chunk tile (no-swizzle K-major:
// 8-row x 16-byte core matrices, 128 B apart along K, 8 kCB apart along M / N)
__device__ __forceinline__ uint32_t ctile_off(int r, int kb) {
    return uint32_t((r >> 3) * (8 * kCB) + (kb >> 4) * 128 + (r & 7) * 16 + (kb & 15));
}

// Shared-memory plan of k_rowgemm_tc<S, NT>.  A stage holds one K chunk:
// fp32 storage (3-term tf32 product) A_hi, A_lo, B_hi, B_lo and the raw
// gathered coefficients; bf16 storage A, B and the raw coefficients.
template <typename S, int NT>
struct Plan {
    static constexpr bool kSplit = sizeof(S) == 4;
    static constexpr int kES = int(sizeof(S));
    static constexpr int kKC = kCB / kES;                     // K entries per chunk
    static constexpr int kATile = kRowsTile * kCB;
    static constexpr int kBTile = NT * kCB;
    // raw coefficients [k][n], rows of NT + 8 floats: the 4 K rows a warp
    // reads at once fall on disjoint banks
    static constexpr int kRawLd = NT + 8;
    static constexpr int kBRaw = kKC * kRawLd * 4;
    static constexpr int kStage = (kSplit ? 2 : 1) * (kATile + kBTile) + kBRaw;
    static constexpr int kStages = kSplit ? 3 : 4;
    static constexpr int kLag = kStages - 2;                  // chunks in flight past the published one
    // per producer warp: the source of every K entry of its current chunk, and
    // the segments (column, length, offset) of its current task, up to kSegCap
    // (a task with more searches global memory)
    static constexpr int kSegCap = 96;
    static constexpr int kTabOff = kStages * kStage;
    static constexpr int kSegOff = kTabOff + kProducerWarps * kKC * 8;
    // the tile ring: producer warp 0 posts every tile (and zero-filled task) in
    // order, the MMA thread and the epilogue read it: {y offset, chunks, rows}
    static constexpr int kRing = 8;
    static constexpr int kRingOff = kSegOff + kProducerWarps * kSegCap * 16;
    static constexpr int kBarOff = kRingOff + kRing * 16;
    // landed[kStages], full[kStages], empty[kStages], acc_full[2], acc_empty[2],
    // info[kRing], info_free[kRing]; then the TMEM address and the failure flag
    static constexpr int kNBar = 3 * kStages + 4 + 2 * kRing;
    static constexpr int kBytes = kBarOff + kNBar * 8 + 16;
    static constexpr uint32_t kCols = 2 * NT < 32 ? 32 : 2 * NT;   // two accumulators
    static_assert(kStage % 128 == 0 && kTabOff % 16 == 0, "stage alignment");
};

}  // namespace tc

// Block-row GEMM on tensor cores, warp-specialised: Y[dst + i][c0 + c] (+)=
// sum_k A[i * kpad + k] X[k][c0 + c] for every task of the list, an NT-column
// RHS tile, S = stored operator type (fp32: 3-term tf32 product; bf16), fp32
// coefficients.  Persistent CTAs (two per SM) take tasks blockIdx.x,
// + gridDim.x, ...; a task's rows run in tiles of 128 (the MMA's M) and its K
// in chunks of kCB = 64 bytes per row, through a ring of tc::Plan::kStages
// shared-memory stages:
//   producers  (warps 0-3, each on its own over its quarter of every chunk):
//              the source table of the chunk's K entries (from the task's
//              segments, copied to shared memory once per task); cp.async of
//              the operator rows into the stage's canonical no-swizzle K-major
//              tile (bytes past kpad zero-filled, rows past the task's left
//              stale: their accumulator rows are never read) and of the
//              coefficient rows (a task's own column count, if its record
//              gives one, bounds the columns read: the others are zero),
//              16 bytes of the RHS tile at a time, into a raw
//              [k][n] tile, each thread then arriving on landed[s] when its
//              copies land; kLag chunks later (landed[s] complete) the fp32
//              tiles are split into tf32 hi / lo terms, the coefficients
//              transposed into the K-major B tile (bf16 pairs, or hi / lo), and
//              the stage published on full[s].  A stage is refilled after the
//              MMAs that read it committed to empty[s].
//   MMA thread (warp 8, lane 0): per chunk 2 K-steps of 32 bytes, each one
//              tcgen05.mma (bf16) or three (a_hi b_hi + a_hi b_lo + a_lo b_hi),
//              committed to empty[s]; the tile's last commit goes to acc_full[a]
//              of one of two TMEM accumulators, so the next tile's MMAs overlap
//              the epilogue of this one.
//   epilogue   (warps 4-7): tcgen05.ld of accumulator rows 32 (w - 4) .. + 31,
//              added to / stored in Y; then acc_empty[a].
// Every mbarrier wait is bounded; an expired wait records kErrTimeout in *err
// and the CTA winds down (each producer warp at its next chunk, the others at
// their next expired wait), waits (bounded) for its MMAs in flight and frees
// its TMEM.  Dynamic shared memory: tc::Plan<S, NT>::kBytes.
template <typename S, int NT>
__host__ __device__ constexpr int tc_smem_bytes() {
    return tc::Plan<S, NT>::kBytes;
}

template <typename S, int NT>
__global__ void __launch_bounds__(tc::kThreadsWs, 2) k_rowgemm_tc(
    int64_t ntask, const int64_t* __restrict__ meta, const int64_t* __restrict__ seg_off,
    const int32_t* __restrict__ seg_len, const int32_t* __restrict__ seg_col,
    const S* __restrict__ ops, float* __restrict__ vec, int accumulate, int nrhs, int c0,
    int* __restrict__ err) {
    using P = tc::Plan<S, NT>;
    static_assert(NT == 16 || NT == 32 || NT == 64, "RHS tile");
    constexpr bool SPLIT = P::kSplit;
    constexpr int KC = P::kKC, NS = P::kStages, CB = tc::kCB, RING = P::kRing;
    constexpr int UPR = CB / (SPLIT ? 16 : 8);                         // A copy units per row
    constexpr int SPG = UPR / 4;                                       // warp steps per row group
    constexpr int AUNITS = tc::kRowsTile * UPR / tc::kProducerThreads;  // per thread
    constexpr int RTOTAL = KC * (NT / 4);                              // raw 16-byte units per chunk
    constexpr int RUNITS = (RTOTAL + tc::kProducerThreads - 1) / tc::kProducerThreads;
    constexpr int BWORDS = NT * (CB / 4) / tc::kProducerThreads;      // B tile words per thread
    static_assert(BWORDS >= 1 && BWORDS * tc::kProducerThreads == NT * (CB / 4), "producer split");
    constexpr uint32_t kIdesc = tc::instr_desc(SPLIT ? 2u : 1u, tc::kRowsTile, NT);
    extern __shared__ __align__(1024) uint8_t smem[];
    int64_t* tab = reinterpret_cast<int64_t*>(smem + P::kTabOff);
    int64_t* ring = reinterpret_cast<int64_t*>(smem + P::kRingOff);   // [RING][2]
    uint64_t* landed = reinterpret_cast<uint64_t*>(smem + P::kBarOff);
    uint64_t* full = landed + NS;
    uint64_t* empty = full + NS;
    uint64_t* acc_full = empty + NS;
    uint64_t* acc_empty = acc_full + 2;
    uint64_t* info = acc_empty + 2;
    uint64_t* info_free = info + RING;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(info_free + RING);
    volatile int* fail = reinterpret_cast<volatile int*>(tmem_slot + 1);

    if (int64_t(blockIdx.x) >= ntask) return;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ncols = min(NT, nrhs - c0);
    if (warp == tc::kMmaWarp) tc::tmem_alloc(tmem_slot, P::kCols);
    if (tid == 0) {
        for (int i = 0; i < NS; ++i) {
            tc::mbar_init(&landed[i], tc::kProducerThreads);
            tc::mbar_init(&full[i], tc::kProducerThreads);
            tc::mbar_init(&empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            tc::mbar_init(&acc_full[i], 1);
            tc::mbar_init(&acc_empty[i], tc::kEpiThreads);
        }
        for (int i = 0; i < RING; ++i) {
            tc::mbar_init(&info[i], 1);
            tc::mbar_init(&info_free[i], tc::kEpiThreads + 1);
        }
        *fail = 0;
        tc::fence_async_smem();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    auto on_fail = [&]() {
        *fail = 1;
        atomicExch(err, tc::kErrTimeout);
    };

    if (warp < tc::kProducerWarps) {
        // ------------------------------------------------------------ producers
        // Each producer warp runs the chunk sequence on its own (its quarter of
        // the units of every chunk): lane 0 waits for the stage, the warp builds
        // its table, issues its copies, and publishes its chunk kLag back; the
        // 128 producer threads arrive on full[s].  The task records are loaded
        // two tasks ahead and the segments of the next task are copied while
        // the current one runs; warp 0 posts every tile to the ring.
        const int pw = warp, ptid = tid;
        int64_t* wtab = tab + pw * KC;
        const bool raw16 = (nrhs % 4 == 0) && (c0 % 4 == 0);   // 16-byte aligned coefficient rows
        struct Task {
            int64_t aoff, dst, e0, nseg, rows, kpad, ncols;
        };
        auto load_task = [&](int64_t t) -> Task {
            Task k{0, 0, 0, 0, 0, 0, -1};
            if (t < ntask) {
                const longlong2* m = reinterpret_cast<const longlong2*>(meta + t * 8);
                const longlong2 a = __ldg(m), b = __ldg(m + 1), c = __ldg(m + 2), e = __ldg(m + 3);
                k = Task{a.x, a.y, b.x, b.y, c.x, c.y, e.x};
            }
            return k;
        };
        // the warp's segment copy in shared memory
        int32_t* const wcol = reinterpret_cast<int32_t*>(smem + P::kSegOff) + pw * P::kSegCap * 4;
        int32_t* const wlen = wcol + P::kSegCap;
        int64_t* const woff = reinterpret_cast<int64_t*>(wlen + P::kSegCap);
        constexpr int SPL = P::kSegCap / 32;               // segments per lane
        struct Segs {
            int32_t col[SPL], len[SPL];
            int64_t off[SPL];
        };
        // global loads of task k's segments into registers (issued a task ahead)
        auto load_segs = [&](const Task& k, Segs& r) {
#pragma unroll
            for (int j = 0; j < SPL; ++j) {
                const int e = lane + 32 * j;
                if (k.rows > 0 && k.kpad > 0 && k.nseg <= P::kSegCap && e < k.nseg) {
                    r.col[j] = __ldg(seg_col + k.e0 + e);
                    r.len[j] = __ldg(seg_len + k.e0 + e);
                    r.off[j] = __ldg(seg_off + k.e0 + e);
                }
            }
        };
        auto store_segs = [&](const Task& k, const Segs& r) {
            __syncwarp();                                  // the previous task's searches done
#pragma unroll
            for (int j = 0; j < SPL; ++j) {
                const int e = lane + 32 * j;
                if (k.nseg <= P::kSegCap && e < k.nseg) {
                    wcol[e] = r.col[j];
                    wlen[e] = r.len[j];
                    woff[e] = r.off[j];
                }
            }
            __syncwarp();
        };
        const int64_t G = gridDim.x;
        int64_t t = blockIdx.x;
        Task cur = load_task(t), nx1 = load_task(t + G), nx2 = load_task(t + 2 * G);
        Segs pre;
        load_segs(cur, pre);
        int nseg = 0, kp = 0, nr = 0, nchunk = 0, m0 = 0, ch = -1;
        int tcols = ncols;                  // coefficient columns of the current task
        const S* Am = ops;
        uint32_t posted = 0;                               // ring entries (warp 0)
        bool ok = true;
        // warp 0, lane 0: post a ring entry {y offset, chunks (0: zero-fill, -1: end), rows}
        // (called by every lane of every producer warp: `ok` stays warp-uniform)
        auto post = [&](int64_t yoff, int nch, int rows) {
            if (pw != 0) return;
            if (lane == 0 && ok) {
                const uint32_t e = posted++;
                const int slot = int(e % RING);
                if (e >= RING && !tc::mbar_wait(&info_free[slot], ((e / RING) - 1) & 1, tc::kWaitLimit)) {
                    on_fail();
                    ok = false;
                } else {
                    ring[slot * 2] = yoff;
                    ring[slot * 2 + 1] = (int64_t(nch) << 32) | uint32_t(rows);
                    tc::mbar_arrive(&info[slot]);
                }
            }
            ok = __shfl_sync(0xffffffffu, ok, 0);
        };
        // move on to the task after `cur`: its segments landed; prefetch the one after
        auto next_task = [&]() {
            cur = nx1;
            nx1 = nx2;
            t += G;
            nx2 = load_task(t + 2 * G);
        };
        // the next chunk of this CTA's sequence (false when none is left)
        bool entered = false;
        auto advance = [&]() -> bool {
            if (nchunk > 0 && ++ch < nchunk) return true;
            ch = 0;
            if (nchunk > 0 && (m0 += tc::kRowsTile) < nr) {
                post((cur.dst + m0) * nrhs + c0, nchunk, min(tc::kRowsTile, nr - m0));
                return true;
            }
            nchunk = 0;
            while (ok) {
                if (entered) next_task();
                entered = true;
                if (t >= ntask) return false;
                // the segments of `cur` (loaded a task ago) to shared memory; the
                // next task's loads go out now
                store_segs(cur, pre);
                load_segs(nx1, pre);
                kp = int(cur.kpad);
                nr = int(cur.rows);
                if (nr <= 0) continue;
                if (kp <= 0) {
                    if (!accumulate) post(cur.dst * nrhs + c0, 0, nr);
                    continue;
                }
                nchunk = (kp + KC - 1) / KC;
                Am = ops + cur.aoff;
                tcols = cur.ncols >= 0 ? min(ncols, int(cur.ncols)) : ncols;
                nseg = cur.nseg <= P::kSegCap ? int(cur.nseg) : -1;
                m0 = 0;
                post(cur.dst * nrhs + c0, nchunk, min(tc::kRowsTile, nr));
                return true;
            }
            return false;
        };
        // coefficient row of K entry k (-1: none): the segment with col <= k < col + len
        // (k grows along a row tile, so the segment index `h` of a lane only moves forward)
        int hint[(KC + 31) / 32];
        auto source = [&](int k, int& h) -> int64_t {
            if (k >= kp) return -1;
            if (nseg >= 0) {
                while (h < nseg && wcol[h] + wlen[h] <= k) ++h;
                return (h < nseg && wcol[h] <= k) ? woff[h] + (k - wcol[h]) : -1;
            }
            int64_t lo = cur.e0, hi = cur.e0 + cur.nseg;
            while (lo < hi) {
                const int64_t mid = (lo + hi) >> 1;
                if (seg_col[mid] <= k) lo = mid + 1; else hi = mid;
            }
            return (lo > cur.e0 && k < seg_col[lo - 1] + seg_len[lo - 1])
                       ? seg_off[lo - 1] + (k - seg_col[lo - 1]) : -1;
        };
        uint32_t g = 0;             // chunks issued
        // issue chunk g into stage g % NS: table, cp.async of its A units and
        // coefficient rows (zero-filled where there is no source)
        auto issue = [&]() -> bool {
            const int st = int(g % NS);
            int go_on = 1;
            if (lane == 0) {
                if (g >= NS && !tc::mbar_wait(&empty[st], ((g / NS) - 1) & 1, tc::kWaitLimit)) on_fail();
                go_on = !*fail;
            }
            if (!__shfl_sync(0xffffffffu, go_on, 0)) return false;
            if (lane != 0 && g >= NS) tc::mbar_wait(&empty[st], ((g / NS) - 1) & 1, tc::kWaitLimit);
#pragma unroll
            for (int j = 0; j < (KC + 31) / 32; ++j) {
                const int e = lane + 32 * j;
                if (e < KC) {
                    if (ch == 0) hint[j] = 0;
                    wtab[e] = source(ch * KC + e, hint[j]);
                }
            }
            __syncwarp();
            uint8_t* At = smem + st * P::kStage;
            float* raw = reinterpret_cast<float*>(At + (SPLIT ? 2 : 1) * (P::kATile + P::kBTile));
            const int mt = min(tc::kRowsTile, nr - m0);
            const int k0 = ch * KC;
#pragma unroll
            for (int i = 0; i < AUNITS; ++i) {
                // a warp step covers 8 rows x 4 units (16 bytes fp32, 8 bytes
                // bf16); SPG steps cover a row group
                const int r = (pw * AUNITS + i) / SPG * 8 + (lane & 7);
                const int q = ((pw * AUNITS + i) % SPG) * 4 + (lane >> 3);
                if (r < mt) {
                    const int kk = k0 + q * 4;              // 4 entries per unit
                    const S* rowp = Am + int64_t(m0 + r) * kp;
                    if constexpr (SPLIT) {
                        const int bytes = max(0, min(16, (kp - kk) * 4));
                        tc::cp_async16(At + tc::ctile_off(r, q * 16), rowp + (bytes > 0 ? kk : 0), bytes);
                    } else {
                        const int bytes = max(0, min(8, (kp - kk) * 2));
                        tc::cp_async8(At + tc::ctile_off(r, q * 8), rowp + (bytes > 0 ? kk : 0), bytes);
                    }
                }
            }
#pragma unroll
            for (int i = 0; i < RUNITS; ++i) {
                const int u = ptid + tc::kProducerThreads * i;
                if (RTOTAL % tc::kProducerThreads != 0 && u >= RTOTAL) break;
                const int k = u / (NT / 4), n = 4 * (u % (NT / 4));
                const int64_t si = wtab[k];
                float* d = raw + k * P::kRawLd + n;
                const float* src = vec + (si >= 0 ? si : 0) * nrhs + c0 + n;
                if (raw16) {
                    const int bytes = si >= 0 ? max(0, min(16, (tcols - n) * 4)) : 0;
                    tc::cp_async16(d, bytes > 0 ? src : vec, bytes);
                } else {
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const bool has = si >= 0 && n + j < tcols;
                        tc::cp_async4(d + j, has ? src + j : vec, has ? 4 : 0);
                    }
                }
            }
            tc::cp_async_arrive(&landed[st]);
            __syncwarp();                                  // table read before the next chunk's
            return true;
        };
        // publish chunk c (its copies landed): split the fp32 A units into tf32
        // hi / lo terms, transpose the raw coefficients into the K-major B tile
        // (hi / lo, or bf16 pairs), then arrive on full[s]
        auto publish = [&](uint32_t c) -> bool {
            const int st = int(c % NS);
            // every producer's copies of this chunk landed (the transpose reads
            // coefficients other threads copied)
            if (!tc::mbar_wait(&landed[st], (c / NS) & 1, tc::kWaitLimit)) {
                on_fail();
                return false;
            }
            uint8_t* At = smem + st * P::kStage;
            uint8_t* Bt = At + (SPLIT ? 2 : 1) * P::kATile;
            const float* raw = reinterpret_cast<const float*>(At + (SPLIT ? 2 : 1) * (P::kATile + P::kBTile));
            if constexpr (SPLIT) {
                uint8_t* Alo = At + P::kATile;
#pragma unroll
                for (int i = 0; i < AUNITS; ++i) {
                    const int r = (pw * AUNITS + i) / SPG * 8 + (lane & 7);
                    const int q = ((pw * AUNITS + i) % SPG) * 4 + (lane >> 3);
                    const uint32_t off = tc::ctile_off(r, q * 16);
                    float4 x = *reinterpret_cast<const float4*>(At + off), h, l;
                    tc::split_tf32(x.x, h.x, l.x);
                    tc::split_tf32(x.y, h.y, l.y);
                    tc::split_tf32(x.z, h.z, l.z);
                    tc::split_tf32(x.w, h.w, l.w);
                    *reinterpret_cast<float4*>(At + off) = h;
                    *reinterpret_cast<float4*>(Alo + off) = l;
                }
            }
#pragma unroll
            for (int i = 0; i < BWORDS; ++i) {
                const int combo = pw + 4 * i;
                const int n = (combo % (NT / 8)) * 8 + (lane & 7);
                const int kw = (combo / (NT / 8)) * 4 + (lane >> 3);
                const uint32_t off = tc::ctile_off(n, kw * 4);
                if constexpr (SPLIT) {
                    float h, l;
                    tc::split_tf32(raw[kw * P::kRawLd + n], h, l);
                    *reinterpret_cast<float*>(Bt + off) = h;
                    *reinterpret_cast<float*>(Bt + P::kBTile + off) = l;
                } else {
                    const __nv_bfloat162 v =
                        __floats2bfloat162_rn(raw[(2 * kw) * P::kRawLd + n], raw[(2 * kw + 1) * P::kRawLd + n]);
                    *reinterpret_cast<uint32_t*>(Bt + off) = *reinterpret_cast<const uint32_t*>(&v);
                }
            }
            tc::fence_async_smem();
            tc::mbar_arrive(&full[st]);
            return true;
        };
        // chunks g - kLag + 1 .. g stay in flight while chunk g - kLag is published
        uint32_t pub = 0;
        bool go = advance();
        while (go) {
            if (!issue()) break;
            ++g;
            if (g - pub > uint32_t(P::kLag) && !publish(pub++)) break;
            go = advance();
        }
        if (!go && ok) {
            while (pub < g && publish(pub)) ++pub;
            post(0, -1, 0);                                // end of the sequence
        }
        tc::cp_async_wait_all();
    } else if (warp == tc::kMmaWarp) {
        // ------------------------------------------------------------ MMA issue
        if (lane == 0) {
            uint32_t e = 0, g = 0, ti = 0;
            for (;;) {
                const int slot = int(e % RING);
                if (!tc::mbar_wait(&info[slot], (e / RING) & 1, tc::kWaitLimit)) {
                    on_fail();
                    break;
                }
                const int nchunk = int(ring[slot * 2 + 1] >> 32);
                tc::mbar_arrive(&info_free[slot]);
                ++e;
                if (nchunk < 0) break;
                if (nchunk == 0) continue;                 // zero-filled by the epilogue
                const uint32_t a = ti & 1;
                if (ti >= 2 && !tc::mbar_wait(&acc_empty[a], ((ti >> 1) - 1) & 1, tc::kWaitLimit)) {
                    on_fail();
                    break;
                }
                tc::tc_fence_after();
                const uint32_t d = tmem + a * NT;
                bool ok = true;
                for (int ch = 0; ch < nchunk; ++ch, ++g) {
                    const int st = int(g % NS);
                    if (!tc::mbar_wait(&full[st], (g / NS) & 1, tc::kWaitLimit)) {
                        on_fail();
                        ok = false;
                        break;
                    }
                    tc::tc_fence_after();
                    const uint32_t a0 = tc::smem_u32(smem + st * P::kStage);
                    const uint32_t b0 = a0 + (SPLIT ? 2 : 1) * P::kATile;
#pragma unroll
                    for (int s = 0; s < CB / 32; ++s) {            // K = 32 bytes per MMA
                        const uint64_t ad = tc::smem_desc(a0 + s * 256, 128, 8 * CB);
                        const uint64_t bd = tc::smem_desc(b0 + s * 256, 128, 8 * CB);
                        tc::mma<!SPLIT>(d, ad, bd, kIdesc, (ch > 0 || s > 0) ? 1u : 0u);
                        if constexpr (SPLIT) {
                            const uint64_t adl = tc::smem_desc(a0 + P::kATile + s * 256, 128, 8 * CB);
                            const uint64_t bdl = tc::smem_desc(b0 + P::kBTile + s * 256, 128, 8 * CB);
                            tc::mma<false>(d, ad, bdl, kIdesc, 1u);
                            tc::mma<false>(d, adl, bd, kIdesc, 1u);
                        }
                    }
                    tc::mma_commit(&empty[st]);
                }
                if (!ok) break;
                tc::mma_commit(&acc_full[a]);
                ++ti;
            }
            // every MMA of this CTA complete before the TMEM is released
            if (g > 0) {
                const uint32_t last = g - 1;
                tc::mbar_wait(&empty[last % NS], (last / NS) & 1, tc::kWaitLimit);
            }
        }
    } else {
        // ------------------------------------------------------------ epilogue
        const int quarter = warp & 3, etid = tid - 32 * tc::kProducerWarps;
        const bool vec4 = (nrhs % 4 == 0) && (c0 % 4 == 0) && ncols == NT;
        uint32_t e = 0, ti = 0;
        for (;;) {
            const int slot = int(e % RING);
            if (!tc::mbar_wait(&info[slot], (e / RING) & 1, tc::kWaitLimit)) {
                on_fail();
                break;
            }
            const int64_t yoff = ring[slot * 2];
            const int64_t w = ring[slot * 2 + 1];
            tc::mbar_arrive(&info_free[slot]);
            ++e;
            const int nchunk = int(w >> 32), nrow = int(uint32_t(w));
            if (nchunk < 0) break;
            float* y = vec + yoff;
            if (nchunk == 0) {                             // a task without columns: y = 0
                for (int j = etid; j < nrow * ncols; j += tc::kEpiThreads)
                    y[int64_t(j / ncols) * nrhs + (j % ncols)] = 0.0f;
                continue;
            }
            const uint32_t a = ti & 1;
            if (!tc::mbar_wait(&acc_full[a], (ti >> 1) & 1, tc::kWaitLimit)) {
                on_fail();
                break;
            }
            ++ti;
            tc::tc_fence_after();
            const int row = quarter * 32 + lane;
            const uint32_t tb = tmem + (uint32_t(quarter * 32) << 16) + a * NT;
            uint32_t v[NT];
#pragma unroll
            for (int c8 = 0; c8 < NT; c8 += 8)
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                    : "=r"(v[c8]), "=r"(v[c8 + 1]), "=r"(v[c8 + 2]), "=r"(v[c8 + 3]), "=r"(v[c8 + 4]),
                      "=r"(v[c8 + 5]), "=r"(v[c8 + 6]), "=r"(v[c8 + 7])
                    : "r"(tb + uint32_t(c8)));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            tc::tc_fence_before();
            tc::mbar_arrive(&acc_empty[a]);                // accumulator free for tile ti + 2
            if (row < nrow) {
                float* yo = y + int64_t(row) * nrhs;
                if (vec4) {
#pragma unroll
                    for (int c = 0; c < NT; c += 4) {
                        float4 o = make_float4(__uint_as_float(v[c]), __uint_as_float(v[c + 1]),
                                               __uint_as_float(v[c + 2]), __uint_as_float(v[c + 3]));
                        if (accumulate) {
                            const float4 p = *reinterpret_cast<const float4*>(yo + c);
                            o.x += p.x; o.y += p.y; o.z += p.z; o.w += p.w;
                        }
                        *reinterpret_cast<float4*>(yo + c) = o;
                    }
                } else {
#pragma unroll
                    for (int c = 0; c < NT; ++c)
                        if (c < ncols) yo[c] = accumulate ? yo[c] + __uint_as_float(v[c]) : __uint_as_float(v[c]);
                }
            }
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == tc::kMmaWarp) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, P::kCols);
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
