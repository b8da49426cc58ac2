// CUDA kernels of the H2* matrix-vector product (§5.1.2, §5.2.2, App. A.2).
//
// Every kernel is templated on an arithmetic policy:
//   F64  -- operators, coefficients and sums in IEEE double (FP64 pipe);
//   F32  -- everything in float (FP32 pipe);
//   BF16 -- operators stored in bfloat16 (8-bit significand), coefficients and
//           sums in float; products with 16 or more right-hand sides run on
//           the tensor cores (tc_kernels.cuh);
//   DF   -- "double-float": every operator entry and coefficient is a pair
//           (hi, lo) of floats with hi + lo equal to the fp64 value to 48
//           significant bits, and every multiply-add runs as error-free
//           transformations on the FP32 pipe (Dekker's product via FMA,
//           Knuth's two-sum).  On GB300 the FP64 pipe delivers ~0.5 TFMA/s,
//           1/73 of FP32, so fp64-grade GEMV is ALU-bound at ~4 TB/s in F64
//           but HBM-bound in DF (about 12 FP32 operations per multiply-add).
//
// Data layout (HBM, built once per geometry):
//   ops   every operator entry: leaf bases U_X, L2L matrices U~_{X_c X}
//         (r_c x r_X row-major), block rows for M2L and the stored near field,
//         (H2+H)* factors (column-major).
//   vec   one coefficient buffer [ q (N) | v (vlen) | u (vlen) | phi (N) ]:
//         charges and potentials in tree order (leaf-contiguous) and the
//         multipole / local coefficients of every (basis, level, box) slot.
//   xs    coordinates in tree order, structure of arrays (xs[k * N + i]).
//
// A "block row" task computes y[dst + i] (+)= sum_k A[i * kpad + k] x[k] for
// i < rows, where x is the concatenation of segments of `vec` (gathered into
// shared memory) and A is stored row-major, zero padded to kpad (a multiple of
// 4 entries, so rows start 16-byte aligned).  Every step of the MVP except the
// on-the-fly near field is a list of such tasks:
//   P2M  one task per (basis, leaf): A = U_X^T, x = q_X, y = v_X;
//   M2M  one per parent: A = [U~_{X_1 X}^T | ...], x = the children's v, y = v_X;
//   M2L  one per target: A = [T_{X,Y_1} | ...], x = the sources' v, y = u_X;
//   L2L  one per child: A = U~_{X_c X}, x = u_X, y = u_{X_c} (accumulate);
//   leaf one per leaf: A = [K_{t^X, s^X'} ... | U_X^far | U_X^ver],
//        x = the neighbours' q then the leaf's u, y = phi_X (L2P fused).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace h2 {

constexpr int kWarp = 32;

// ---------------------------------------------------------------------------
// arithmetic policies
struct F64 {
    using S = double;       // stored operator entry
    using V = double;       // coefficient / accumulator
    using L = double2;      // one 16-byte load of stored entries
    static constexpr int W = 2;
    __device__ static V zero() { return 0.0; }
    __device__ static V mac(V acc, S a, V x) { return fma(a, x, acc); }
    __device__ static V add(V a, V b) { return a + b; }
    __device__ static V from_double(double a) { return a; }
    __device__ static double to_double(V a) { return a; }
    __device__ static V shfl_xor(V a, int o) { return __shfl_xor_sync(0xffffffffu, a, o); }
    __device__ static S lget(const L& l, int k) { return k == 0 ? l.x : l.y; }
};

struct F32 {
    using S = float;
    using V = float;
    using L = float4;
    static constexpr int W = 4;
    __device__ static V zero() { return 0.0f; }
    __device__ static V mac(V acc, S a, V x) { return fmaf(a, x, acc); }
    __device__ static V add(V a, V b) { return a + b; }
    __device__ static V from_double(double a) { return float(a); }
    __device__ static double to_double(V a) { return double(a); }
    __device__ static V shfl_xor(V a, int o) { return __shfl_xor_sync(0xffffffffu, a, o); }
    __device__ static S lget(const L& l, int k) {
        return k == 0 ? l.x : (k == 1 ? l.y : (k == 2 ? l.z : l.w));
    }
};

struct BF16 {
    using S = __nv_bfloat16;
    using V = float;
    using L = uint2;        // four entries (rows start on 4-entry boundaries)
    static constexpr int W = 4;
    __device__ static V zero() { return 0.0f; }
    __device__ static V mac(V acc, float a, V x) { return fmaf(a, x, acc); }
    __device__ static V add(V a, V b) { return a + b; }
    __device__ static V from_double(double a) { return float(a); }
    __device__ static double to_double(V a) { return double(a); }
    __device__ static V shfl_xor(V a, int o) { return __shfl_xor_sync(0xffffffffu, a, o); }
    // entry k of the load as float: a bfloat16 is the upper half of a float
    __device__ static float lget(const L& l, int k) {
        const uint32_t w = k < 2 ? l.x : l.y;
        return __uint_as_float((k & 1) ? (w & 0xFFFF0000u) : (w << 16));
    }
};

struct DF {
    using S = float2;       // (hi, lo)
    using V = float2;
    using L = float4;       // two entries
    static constexpr int W = 2;
    __device__ static V zero() { return make_float2(0.0f, 0.0f); }
    // Knuth's two-sum of a and b, exact: s + e = a + b.
    __device__ static void two_sum(float a, float b, float& s, float& e) {
        s = a + b;
        const float bb = s - a;
        e = (a - (s - bb)) + (b - bb);
    }
    // acc + a * x: the product a.hi x.hi is split exactly with an FMA (Dekker),
    // the cross terms are added in float, the sum with acc.hi is exact (two-sum).
    __device__ static V mac(V acc, S a, V x) {
        const float p = a.x * x.x;
        float e = fmaf(a.x, x.x, -p);
        e = fmaf(a.x, x.y, e);
        e = fmaf(a.y, x.x, e);
        float s, t;
        two_sum(acc.x, p, s, t);
        return make_float2(s, acc.y + (t + e));
    }
    __device__ static V add(V a, V b) {
        float s, t;
        two_sum(a.x, b.x, s, t);
        const float lo = t + a.y + b.y;
        const float hi = s + lo;                 // renormalise (fast two-sum)
        return make_float2(hi, lo - (hi - s));
    }
    __device__ static V from_double(double a) {
        const float hi = __double2float_rn(a);
        return make_float2(hi, __double2float_rn(a - double(hi)));
    }
    __device__ static double to_double(V a) { return double(a.x) + double(a.y); }
    __device__ static V shfl_xor(V a, int o) {
        return make_float2(__shfl_xor_sync(0xffffffffu, a.x, o), __shfl_xor_sync(0xffffffffu, a.y, o));
    }
    __device__ static S lget(const L& l, int k) {
        return k == 0 ? make_float2(l.x, l.y) : make_float2(l.z, l.w);
    }
};

template <class A>
__device__ __forceinline__ typename A::V warp_sum(typename A::V v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = A::add(v, A::shfl_xor(v, o));
    return v;
}

// G(r) from r^2 for the on-the-fly near field; the diagonal (coincident
// points) takes `diag`.
template <typename T, int KIND>
__device__ __forceinline__ T kernel_r2(T r2, T param, T diag);

template <>
__device__ __forceinline__ double kernel_r2<double, 0>(double r2, double, double diag) {
    return r2 == 0.0 ? diag : log(sqrt(r2));
}
template <>
__device__ __forceinline__ double kernel_r2<double, 1>(double r2, double, double diag) {
    return r2 == 0.0 ? diag : 1.0 / sqrt(r2);
}
template <>
__device__ __forceinline__ double kernel_r2<double, 2>(double r2, double c, double diag) {
    if (r2 == 0.0) return diag;
    const double s = sqrt(r2) / c;
    return 1.0 / sqrt(1.0 + s * s);
}
template <>
__device__ __forceinline__ double kernel_r2<double, 3>(double r2, double, double diag) {
    return r2 == 0.0 ? diag : exp(-sqrt(r2));
}
template <>
__device__ __forceinline__ float kernel_r2<float, 0>(float r2, float, float diag) {
    return r2 == 0.0f ? diag : 0.5f * __logf(r2);
}
template <>
__device__ __forceinline__ float kernel_r2<float, 1>(float r2, float, float diag) {
    return r2 == 0.0f ? diag : rsqrtf(r2);
}
template <>
__device__ __forceinline__ float kernel_r2<float, 2>(float r2, float c, float diag) {
    return r2 == 0.0f ? diag : rsqrtf(1.0f + r2 / (c * c));
}
template <>
__device__ __forceinline__ float kernel_r2<float, 3>(float r2, float, float diag) {
    return r2 == 0.0f ? diag : __expf(-sqrtf(r2));
}

// ---- gather / scatter between user order and tree order --------------------
// Coefficients of nrhs right-hand sides are stored point-major, RHS fastest:
// entry (i, c) of a region at region[i * nrhs + c].
template <class A>
__global__ void k_gather(const double* __restrict__ X, int64_t ldx, int nrhs,
                         const int64_t* __restrict__ perm, typename A::V* __restrict__ q, int64_t N) {
    const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t >= N * nrhs) return;
    const int64_t i = t / nrhs;
    const int c = int(t - i * nrhs);
    q[t] = A::from_double(X[int64_t(c) * ldx + perm[i]]);
}

template <class A>
__global__ void k_scatter(const typename A::V* __restrict__ phi, int nrhs,
                          const int64_t* __restrict__ perm, double* __restrict__ Y, int64_t ldy,
                          int64_t N) {
    const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t >= N * nrhs) return;
    const int64_t i = t / nrhs;
    const int c = int(t - i * nrhs);
    Y[int64_t(c) * ldy + perm[i]] = A::to_double(phi[t]);
}

// 2 to 64 right-hand sides: a CTA takes 32 consecutive user indices j and all
// columns, reads each column's 32 entries (coalesced), transposes through
// shared memory and writes each point's row of nrhs coefficients at its tree
// position iperm[j] (contiguous), or the reverse for the scatter.
constexpr int kTransRows = 32;

template <class A>
__global__ void __launch_bounds__(256) k_gather_t(const double* __restrict__ X, int64_t ldx, int nrhs,
                                                 const int64_t* __restrict__ iperm,
                                                 typename A::V* __restrict__ q, int64_t N) {
    using V = typename A::V;
    __shared__ V tile[kTransRows][65];
    const int64_t j0 = int64_t(blockIdx.x) * kTransRows;
    const int n = (N - j0 < kTransRows) ? int(N - j0) : kTransRows;
    for (int idx = threadIdx.x; idx < kTransRows * nrhs; idx += blockDim.x) {
        const int c = idx / kTransRows, jj = idx - c * kTransRows;
        if (jj < n) tile[jj][c] = A::from_double(X[int64_t(c) * ldx + j0 + jj]);
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < kTransRows * nrhs; idx += blockDim.x) {
        const int jj = idx / nrhs, c = idx - jj * nrhs;
        if (jj < n) q[iperm[j0 + jj] * nrhs + c] = tile[jj][c];
    }
}

template <class A>
__global__ void __launch_bounds__(256) k_scatter_t(const typename A::V* __restrict__ phi, int nrhs,
                                                  const int64_t* __restrict__ iperm,
                                                  double* __restrict__ Y, int64_t ldy, int64_t N) {
    using V = typename A::V;
    __shared__ V tile[kTransRows][65];
    const int64_t j0 = int64_t(blockIdx.x) * kTransRows;
    const int n = (N - j0 < kTransRows) ? int(N - j0) : kTransRows;
    for (int idx = threadIdx.x; idx < kTransRows * nrhs; idx += blockDim.x) {
        const int jj = idx / nrhs, c = idx - jj * nrhs;
        if (jj < n) tile[jj][c] = phi[iperm[j0 + jj] * nrhs + c];
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < kTransRows * nrhs; idx += blockDim.x) {
        const int c = idx / kTransRows, jj = idx - c * kTransRows;
        if (jj < n) Y[int64_t(c) * ldy + j0 + jj] = A::to_double(tile[jj][c]);
    }
}

// ---- block-row GEMV: M2L, L2L and the stored near field (+ fused L2P) ---------
// One CTA (8 warps) per task.  The gathered coefficients of an NR-column tile
// (columns c0 .. c0 + NR - 1 of nrhs) are staged through a 32 KB shared-memory
// chunk; each warp owns RW rows (rows warp, warp + 8, ...) and streams them
// with 16-byte loads, two k-steps per iteration, so one loaded operator entry
// feeds NR multiply-adds and one staged coefficient RW of them, and each lane
// keeps 2 RW independent loads in flight.  Segments are sorted by column
// (seg_col = first column of each).
template <class A, int RW, int NR>
__global__ void __launch_bounds__(256) k_rowgemv(
    int64_t ntask, const int64_t* __restrict__ dst, const int32_t* __restrict__ rows,
    const int32_t* __restrict__ kpad, const int64_t* __restrict__ aoff,
    const int64_t* __restrict__ seg_ptr, const int64_t* __restrict__ seg_off,
    const int32_t* __restrict__ seg_len, const int32_t* __restrict__ seg_col,
    const typename A::S* __restrict__ ops, typename A::V* __restrict__ vec, int accumulate,
    int nrhs, int c0, int row_chunk) {
    using V = typename A::V;
    using L = typename A::L;
    constexpr int W = A::W;
    constexpr int C = 4096 * 8 / int(sizeof(V)) / NR;   // staged columns per chunk
    constexpr int NW = 8;
    static_assert(C % (2 * kWarp * W) == 0, "chunk must hold whole warp steps");
    __shared__ __align__(16) V xs[C * NR];
    const int64_t t = blockIdx.x;
    if (t >= ntask) return;
    const int kp = kpad[t];
    const int nr = rows[t];
    const int64_t e0 = seg_ptr[t], e1 = seg_ptr[t + 1];
    const int ktot = (e1 > e0) ? seg_col[e1 - 1] + seg_len[e1 - 1] : 0;
    const typename A::S* Am = ops + aoff[t];
    V* y = vec + dst[t] * nrhs + c0;
    const int warp = threadIdx.x / kWarp, lane = threadIdx.x % kWarp;
    const int rb0 = int(blockIdx.y) * row_chunk, rb1 = min(nr, rb0 + row_chunk);
    for (int r0 = rb0; r0 < rb1; r0 += NW * RW) {
        V acc[RW][NR];
        bool ok[RW];
        const L* arow[RW];
#pragma unroll
        for (int w = 0; w < RW; ++w) {
#pragma unroll
            for (int c = 0; c < NR; ++c) acc[w][c] = A::zero();
            const int row = r0 + warp + NW * w;
            ok[w] = row < nr;
            arow[w] = reinterpret_cast<const L*>(Am + int64_t(ok[w] ? row : 0) * kp);
        }
        int64_t ef = e0;                      // first segment not yet fully consumed
        for (int ch = 0; ch < kp; ch += C) {
            const int cw = min(C, kp - ch);
            __syncthreads();
            while (ef < e1 && seg_col[ef] + seg_len[ef] <= ch) ++ef;
            for (int64_t e = ef; e < e1; ++e) {
                const int sc = seg_col[e];
                if (sc >= ch + cw) break;
                const int lo = max(sc, ch), hi = min(sc + seg_len[e], ch + cw);
                const V* src = vec + (seg_off[e] + (lo - sc)) * nrhs + c0;
                const int n = (hi - lo) * NR;
                for (int j = threadIdx.x; j < n; j += blockDim.x) {
                    const int rr = j / NR, cc = j - rr * NR;
                    xs[(lo - ch + rr) * NR + cc] = src[int64_t(rr) * nrhs + cc];
                }
            }
            for (int j = max(ktot - ch, 0) * NR + threadIdx.x; j < cw * NR; j += blockDim.x)
                xs[j] = A::zero();
            __syncthreads();
            const int nv = cw / W, k0 = ch / W;
            for (int k = lane; k < nv; k += 2 * kWarp) {
                const bool two = k + kWarp < nv;
                L a0[RW], a1[RW];
#pragma unroll
                for (int w = 0; w < RW; ++w) {
                    if (ok[w]) a0[w] = __ldg(arow[w] + k0 + k);
                    if (ok[w] && two) a1[w] = __ldg(arow[w] + k0 + k + kWarp);
                }
                // first k-step for every z, then the second: the summation
                // order of k_rowgemv1, so each column matches it bit for bit
#pragma unroll
                for (int z = 0; z < W; ++z) {
                    V x0[NR];
#pragma unroll
                    for (int c = 0; c < NR; ++c) x0[c] = xs[(k * W + z) * NR + c];
#pragma unroll
                    for (int w = 0; w < RW; ++w)
                        if (ok[w]) {
                            const auto s0 = A::lget(a0[w], z);
#pragma unroll
                            for (int c = 0; c < NR; ++c) acc[w][c] = A::mac(acc[w][c], s0, x0[c]);
                        }
                }
                if (two) {
#pragma unroll
                    for (int z = 0; z < W; ++z) {
                        V x1[NR];
#pragma unroll
                        for (int c = 0; c < NR; ++c) x1[c] = xs[((k + kWarp) * W + z) * NR + c];
#pragma unroll
                        for (int w = 0; w < RW; ++w)
                            if (ok[w]) {
                                const auto s1 = A::lget(a1[w], z);
#pragma unroll
                                for (int c = 0; c < NR; ++c) acc[w][c] = A::mac(acc[w][c], s1, x1[c]);
                            }
                    }
                }
            }
        }
#pragma unroll
        for (int w = 0; w < RW; ++w) {
            if (!ok[w]) continue;
            const int row = r0 + warp + NW * w;
#pragma unroll
            for (int c = 0; c < NR; ++c) {
                const V sum = warp_sum<A>(acc[w][c]);
                if (lane == 0) {
                    V* yo = y + int64_t(row) * nrhs + c;
                    *yo = accumulate ? A::add(*yo, sum) : sum;
                }
            }
        }
    }
}

// The same block-row GEMV for a single right-hand side (nrhs = 1): the staged
// chunk is contiguous, so each lane reads its W coefficients of both k-steps
// with two 16-byte shared loads before the row loop, and each row's W
// multiply-adds of a k-step run back to back on one accumulator.
template <class A, int RW>
__global__ void __launch_bounds__(256) k_rowgemv1(
    int64_t ntask, const int64_t* __restrict__ dst, const int32_t* __restrict__ rows,
    const int32_t* __restrict__ kpad, const int64_t* __restrict__ aoff,
    const int64_t* __restrict__ seg_ptr, const int64_t* __restrict__ seg_off,
    const int32_t* __restrict__ seg_len, const int32_t* __restrict__ seg_col,
    const typename A::S* __restrict__ ops, typename A::V* __restrict__ vec, int accumulate,
    int row_chunk) {
    using V = typename A::V;
    using L = typename A::L;
    constexpr int W = A::W;
    constexpr int C = 4096 * 8 / int(sizeof(V));   // 32 KB of staged coefficients
    constexpr int NW = 8;
    static_assert(C % (2 * kWarp * W) == 0, "chunk must hold whole warp steps");
    __shared__ __align__(16) V xs[C];
    const int64_t t = blockIdx.x;
    if (t >= ntask) return;
    const int kp = kpad[t];
    const int nr = rows[t];
    const int64_t e0 = seg_ptr[t], e1 = seg_ptr[t + 1];
    const int ktot = (e1 > e0) ? seg_col[e1 - 1] + seg_len[e1 - 1] : 0;
    const typename A::S* Am = ops + aoff[t];
    V* y = vec + dst[t];
    const int warp = threadIdx.x / kWarp, lane = threadIdx.x % kWarp;
    const int rb0 = int(blockIdx.y) * row_chunk, rb1 = min(nr, rb0 + row_chunk);
    for (int r0 = rb0; r0 < rb1; r0 += NW * RW) {
        V acc[RW];
        bool ok[RW];
        const L* arow[RW];
#pragma unroll
        for (int w = 0; w < RW; ++w) {
            acc[w] = A::zero();
            const int row = r0 + warp + NW * w;
            ok[w] = row < nr;
            arow[w] = reinterpret_cast<const L*>(Am + int64_t(ok[w] ? row : 0) * kp);
        }
        int64_t ef = e0;
        for (int ch = 0; ch < kp; ch += C) {
            const int cw = min(C, kp - ch);
            __syncthreads();
            while (ef < e1 && seg_col[ef] + seg_len[ef] <= ch) ++ef;
            for (int64_t e = ef; e < e1; ++e) {
                const int sc = seg_col[e];
                if (sc >= ch + cw) break;
                const int lo = max(sc, ch), hi = min(sc + seg_len[e], ch + cw);
                const V* src = vec + seg_off[e] + (lo - sc);
                for (int j = threadIdx.x; j < hi - lo; j += blockDim.x) xs[lo - ch + j] = src[j];
            }
            for (int j = max(ktot - ch, 0) + threadIdx.x; j < cw; j += blockDim.x) xs[j] = A::zero();
            __syncthreads();
            const int nv = cw / W, k0 = ch / W;
            for (int k = lane; k < nv; k += 2 * kWarp) {
                const bool two = k + kWarp < nv;
                L a0[RW], a1[RW];
#pragma unroll
                for (int w = 0; w < RW; ++w) {
                    if (ok[w]) a0[w] = __ldg(arow[w] + k0 + k);
                    if (ok[w] && two) a1[w] = __ldg(arow[w] + k0 + k + kWarp);
                }
                V x0[W], x1[W];
#pragma unroll
                for (int z = 0; z < W; ++z) {
                    x0[z] = xs[k * W + z];
                    x1[z] = two ? xs[(k + kWarp) * W + z] : A::zero();
                }
#pragma unroll
                for (int w = 0; w < RW; ++w)
                    if (ok[w]) {
#pragma unroll
                        for (int z = 0; z < W; ++z) acc[w] = A::mac(acc[w], A::lget(a0[w], z), x0[z]);
                        if (two) {
#pragma unroll
                            for (int z = 0; z < W; ++z) acc[w] = A::mac(acc[w], A::lget(a1[w], z), x1[z]);
                        }
                    }
            }
        }
#pragma unroll
        for (int w = 0; w < RW; ++w) {
            if (!ok[w]) continue;
            const V sum = warp_sum<A>(acc[w]);
            const int row = r0 + warp + NW * w;
            if (lane == 0) y[row] = accumulate ? A::add(y[row], sum) : sum;
        }
    }
}

// ---- leaves, near field on the fly (F64 / F32) --------------------------------
// phi_X = sum_b U_X^b u_X^b + sum_{X' in N(X)} K_{t^X, s^X'} q_X' for an NR-column
// tile; one CTA per leaf, one target per thread; the kernel value of each pair
// is evaluated once and applied to all NR columns; source points staged
// through shared memory.
template <typename T, int D, int KIND, int NR, bool NEAR = true>
__global__ void k_leaf_fly(int64_t nleaf, int nb, int64_t box_total, int64_t leaf_base,
                           const int64_t* __restrict__ leaf_ptr, const int64_t* __restrict__ near_ptr,
                           const int64_t* __restrict__ near_idx, const int32_t* __restrict__ rank,
                           const int64_t* __restrict__ voff, const int64_t* __restrict__ uoff,
                           const int32_t* __restrict__ ustride, const T* __restrict__ ops,
                           const T* __restrict__ u, const T* __restrict__ xs, int64_t N,
                           const T* __restrict__ q, T* __restrict__ phi, T param, T diag,
                           int nrhs, int c0) {
    constexpr int TILE = 128;
    __shared__ T sx[D][TILE];
    __shared__ T sq[TILE * NR];
    const int64_t L = blockIdx.x;
    if (L >= nleaf) return;
    const int64_t p0 = leaf_ptr[L];
    const int m = int(leaf_ptr[L + 1] - p0);
    for (int i0 = 0; i0 < m; i0 += blockDim.x) {
        const int i = i0 + threadIdx.x;
        const bool active = i < m;
        T acc[NR];
#pragma unroll
        for (int c = 0; c < NR; ++c) acc[c] = T(0);
        T xi[D];
        if (active) {
#pragma unroll
            for (int k = 0; k < D; ++k) xi[k] = xs[k * N + p0 + i];
            for (int b = 0; b < nb; ++b) {
                const int64_t s = b * box_total + leaf_base + L;
                const int r = rank[s];
                if (r == 0) continue;
                const T* U = ops + uoff[s] + int64_t(i) * ustride[s];
                const T* ub = u + voff[s] * nrhs + c0;
                for (int j = 0; j < r; ++j) {
                    const T a = U[j];
#pragma unroll
                    for (int c = 0; c < NR; ++c) acc[c] += a * ub[int64_t(j) * nrhs + c];
                }
            }
        }
        for (int64_t e = near_ptr[L]; NEAR && e < near_ptr[L + 1]; ++e) {
            const int64_t Y = near_idx[e];
            const int64_t s0 = leaf_ptr[Y];
            const int ms = int(leaf_ptr[Y + 1] - s0);
            for (int j0 = 0; j0 < ms; j0 += TILE) {
                const int nt = min(TILE, ms - j0);
                __syncthreads();
                for (int j = threadIdx.x; j < nt; j += blockDim.x) {
#pragma unroll
                    for (int k = 0; k < D; ++k) sx[k][j] = xs[k * N + s0 + j0 + j];
#pragma unroll
                    for (int c = 0; c < NR; ++c) sq[j * NR + c] = q[(s0 + j0 + j) * nrhs + c0 + c];
                }
                __syncthreads();
                if (active) {
                    for (int j = 0; j < nt; ++j) {
                        T r2 = T(0);
#pragma unroll
                        for (int k = 0; k < D; ++k) {
                            const T t = xi[k] - sx[k][j];
                            r2 = r2 + t * t;
                        }
                        const T g = kernel_r2<T, KIND>(r2, param, diag);
#pragma unroll
                        for (int c = 0; c < NR; ++c) acc[c] += g * sq[j * NR + c];
                    }
                }
            }
        }
        if (active) {
#pragma unroll
            for (int c = 0; c < NR; ++c) {
                T* o = phi + (p0 + i) * nrhs + c0 + c;
                *o = NEAR ? acc[c] : *o + acc[c];      // without NEAR: added to the near field
            }
        }
    }
}

// ---- near field on the fly in double-float arithmetic (fp64 storage) -------------
// phi_X = sum_{X' in N(X)} K_{t^X, s^X'} q_X' for 1/r and the inverse
// multiquadric without the FP64 pipe: coordinates and charges are split into
// float pairs (hi + lo, 48-bit significand) once per staged point, and every
// pair's kernel value is formed in double-float arithmetic on the FP32 pipe --
// the differences and squares with Knuth's two-sum and the FMA product
// (Dekker), 1/sqrt(t) as one Newton step y0 + y0 (1 - t y0^2) / 2 from the
// fp32 rsqrtf seed (whose relative error ~2^-22 the step squares) -- and
// accumulated with the charges in double-float.  Per kernel value ~2^-44 of
// relative error, where the fp64 path (sqrt and division on the FP64 pipe,
// 1/64 of the FP32 rate on this GPU) rounds to 2^-53.  One CTA per leaf, one
// target per thread, sources staged through shared memory; writes phi (=).
namespace dd {
struct F2 {
    float hi, lo;
};
__device__ __forceinline__ F2 fast_two_sum(float a, float b) {   // |a| >= |b|
    const float s = a + b;
    return F2{s, b - (s - a)};
}
__device__ __forceinline__ F2 two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    return F2{s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ F2 split(double x) {
    const float hi = __double2float_rn(x);
    return F2{hi, __double2float_rn(x - double(hi))};
}
__device__ __forceinline__ F2 sub(F2 a, F2 b) {
    F2 s = two_sum(a.hi, -b.hi);
    return fast_two_sum(s.hi, s.lo + (a.lo - b.lo));
}
__device__ __forceinline__ F2 add(F2 a, F2 b) {
    F2 s = two_sum(a.hi, b.hi);
    return fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}
__device__ __forceinline__ F2 sqr(F2 a) {
    const float p = a.hi * a.hi;
    float e = fmaf(a.hi, a.hi, -p);
    e = fmaf(2.0f * a.hi, a.lo, e);
    return fast_two_sum(p, e);
}
__device__ __forceinline__ F2 mul(F2 a, F2 b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return fast_two_sum(p, e);
}
// 1 / sqrt(t), t > 0: y1 = y0 + y0 h with h = (1 - t y0^2) / 2 and y0 = rsqrtf(t.hi)
__device__ __forceinline__ F2 rsqrt(F2 t) {
    const float y0 = rsqrtf(t.hi);
    const float p = y0 * y0;
    const F2 y2 = F2{p, fmaf(y0, y0, -p)};                      // y0^2 exactly
    const F2 r = sub(F2{1.0f, 0.0f}, mul(t, y2));               // 1 - t y0^2, tiny
    const float h = 0.5f * (r.hi + r.lo);
    return fast_two_sum(y0, y0 * h);
}
}  // namespace dd

template <int D, int KIND, int NR>
__global__ void k_near_df(int64_t nleaf, const int64_t* __restrict__ leaf_ptr,
                          const int64_t* __restrict__ near_ptr, const int64_t* __restrict__ near_idx,
                          const double* __restrict__ xs, int64_t N, const double* __restrict__ q,
                          double* __restrict__ phi, double param2, double diag, int nrhs, int c0) {
    static_assert(KIND == 1 || KIND == 2, "1/r or the inverse multiquadric");
    constexpr int TILE = 128;
    __shared__ dd::F2 sx[D][TILE];
    __shared__ dd::F2 sq[TILE * NR];
    const int64_t L = blockIdx.x;
    if (L >= nleaf) return;
    const int64_t p0 = leaf_ptr[L];
    const int m = int(leaf_ptr[L + 1] - p0);
    const dd::F2 p2 = dd::split(param2);
    const float dg = float(diag);
    for (int i0 = 0; i0 < m; i0 += blockDim.x) {
        const int i = i0 + threadIdx.x;
        const bool active = i < m;
        dd::F2 acc[NR];
#pragma unroll
        for (int c = 0; c < NR; ++c) acc[c] = dd::F2{0.0f, 0.0f};
        dd::F2 xi[D];
#pragma unroll
        for (int k = 0; k < D; ++k) xi[k] = dd::split(active ? xs[k * N + p0 + i] : 0.0);
        for (int64_t e = near_ptr[L]; e < near_ptr[L + 1]; ++e) {
            const int64_t Y = near_idx[e];
            const int64_t s0 = leaf_ptr[Y];
            const int ms = int(leaf_ptr[Y + 1] - s0);
            for (int j0 = 0; j0 < ms; j0 += TILE) {
                const int nt = min(TILE, ms - j0);
                __syncthreads();
                for (int j = threadIdx.x; j < nt; j += blockDim.x) {
#pragma unroll
                    for (int k = 0; k < D; ++k) sx[k][j] = dd::split(xs[k * N + s0 + j0 + j]);
#pragma unroll
                    for (int c = 0; c < NR; ++c) sq[j * NR + c] = dd::split(q[(s0 + j0 + j) * nrhs + c0 + c]);
                }
                __syncthreads();
                if (active) {
                    for (int j = 0; j < nt; ++j) {
                        dd::F2 r2 = dd::sqr(dd::sub(xi[0], sx[0][j]));
#pragma unroll
                        for (int k = 1; k < D; ++k) r2 = dd::add(r2, dd::sqr(dd::sub(xi[k], sx[k][j])));
                        dd::F2 g;
                        if (r2.hi == 0.0f) {
                            g = dd::F2{dg, 0.0f};               // coincident points: the diagonal value
                        } else if constexpr (KIND == 1) {
                            g = dd::rsqrt(r2);
                        } else {
                            g = dd::rsqrt(dd::add(dd::F2{1.0f, 0.0f}, dd::mul(r2, p2)));
                        }
#pragma unroll
                        for (int c = 0; c < NR; ++c) {
                            const dd::F2 gq = dd::mul(g, sq[j * NR + c]);
                            const dd::F2 s = dd::two_sum(acc[c].hi, gq.hi);
                            acc[c] = dd::F2{s.hi, acc[c].lo + (s.lo + gq.lo)};
                        }
                    }
                }
            }
        }
        if (active) {
#pragma unroll
            for (int c = 0; c < NR; ++c)
                phi[(p0 + i) * nrhs + c0 + c] = double(acc[c].hi) + double(acc[c].lo);
        }
    }
}

// ---- M2L evaluated on the fly (fp32) ----------------------------------------
// In H2* the coupling block T_{X,Y} is the kernel matrix between the incoming
// pivots of X and those of Y (§3.6.4), so u_X = sum_{Y in IL(X)} G(t^{X,i},
// t^{Y,i}) v_Y can be evaluated from pivot coordinates instead of streaming
// the stored blocks: px holds the coordinate k of the pivot whose v / u
// coefficient sits at offset o of the v (or u) region at px[k * vlen + o].
// log r uses the accurate logf (the nested bases amplify entry errors);
// param2 = 1 / c^2 for the IMQ.
template <int KIND>
__device__ __forceinline__ float m2l_kernel(float r2, float param2, float diag) {
    if (r2 == 0.0f) return diag;
    if constexpr (KIND == 0) return 0.5f * logf(r2);
    else if constexpr (KIND == 1) return rsqrtf(r2);
    else if constexpr (KIND == 2) return rsqrtf(fmaf(r2, param2, 1.0f));
    else return __expf(-sqrtf(r2));
}

// One CTA per target (the M2L task list); the sources -- the task's segments,
// concatenated -- are staged in tiles of 256 as float4 (coordinates, then the
// coefficient for one RHS; coordinates only for NR > 1, coefficients apart),
// so a pair costs one shared load; each thread evaluates four sources at a
// time into four partial sums; the 256 threads cover the target rows in 64- or
// 128-row groups, the groups taking alternate sets of four sources (4 or 2
// parts), and the parts' sums are added at the end.
template <typename T, int D, int KIND, int NR>
__global__ void __launch_bounds__(256) k_m2l_fly(
    int64_t ntask, const int64_t* __restrict__ dst, const int32_t* __restrict__ rows,
    const int64_t* __restrict__ seg_ptr, const int64_t* __restrict__ seg_off,
    const int32_t* __restrict__ seg_len, const int32_t* __restrict__ seg_col,
    const T* __restrict__ px, int64_t vlen, int64_t v_base, int64_t u_base,
    T* __restrict__ vec, T param2, T diag, int nrhs, int c0) {
    static_assert(D <= 3, "float4 staging holds up to 3 coordinates");
    constexpr int TILE = 256;
    constexpr bool PACKED = NR == 1;                  // (x, y, z, v); 2D: (x, y, v, -)
    constexpr int VSLOT = D == 3 ? 3 : 2;
    __shared__ float4 s4[TILE];
    __shared__ T sv[PACKED || NR == 1 ? 1 : TILE * NR];
    __shared__ T red[3 * 64 * NR];
    const int64_t t = blockIdx.x;
    if (t >= ntask) return;
    // stale entries past a partial tile stay finite: zero the tiles once
    for (int j = threadIdx.x; j < TILE; j += blockDim.x) {
        s4[j] = make_float4(0.f, 0.f, 0.f, 0.f);
        if constexpr (NR > 1) {
#pragma unroll
            for (int c = 0; c < NR; ++c) sv[j * NR + c] = T(0);
        }
    }
    const int nr = rows[t];
    const int64_t e0 = seg_ptr[t], e1 = seg_ptr[t + 1];
    const int ktot = (e1 > e0) ? seg_col[e1 - 1] + seg_len[e1 - 1] : 0;
    const int64_t d0 = dst[t] - u_base;                 // pivot index of the first target row
    const int R = nr <= 64 ? 64 : 128;                   // rows per group
    const int nparts = int(blockDim.x) / R;              // 4 or 2
    const int part = int(threadIdx.x) / R;
    const int step = 4 * nparts;
    const int li = int(threadIdx.x) % R;
    for (int i0 = 0; i0 < nr; i0 += R) {
        const int i = i0 + li;
        const bool active = i < nr;
        float xi[3] = {0.f, 0.f, 0.f};
        T acc[4][NR];
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int c = 0; c < NR; ++c) acc[q][c] = T(0);
#pragma unroll
        for (int k = 0; k < D; ++k) xi[k] = active ? px[k * vlen + d0 + i] : T(0);
        int64_t ef = e0;
        for (int ch = 0; ch < ktot; ch += TILE) {
            const int cw = min(TILE, ktot - ch);
            __syncthreads();
            while (ef < e1 && seg_col[ef] + seg_len[ef] <= ch) ++ef;
            for (int64_t e = ef; e < e1; ++e) {
                const int sc = seg_col[e];
                if (sc >= ch + cw) break;
                const int lo = max(sc, ch), hi = min(sc + seg_len[e], ch + cw);
                const int64_t so = seg_off[e] + (lo - sc);       // vec offset of the first source
                for (int j = threadIdx.x; j < hi - lo; j += blockDim.x) {
                    const int64_t o = so + j;
                    float w[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                    for (int k = 0; k < D; ++k) w[k] = px[k * vlen + (o - v_base)];
                    if constexpr (NR == 1) {
                        w[VSLOT] = vec[o * nrhs + c0];
                    } else {
#pragma unroll
                        for (int c = 0; c < NR; ++c) sv[(lo - ch + j) * NR + c] = vec[o * nrhs + c0 + c];
                    }
                    s4[lo - ch + j] = make_float4(w[0], w[1], w[2], w[3]);
                }
            }
            __syncthreads();
            if (active) {
                // jb is a multiple of 4 below cw <= TILE, so jb + 3 < TILE
                for (int jb = part * 4; jb < cw; jb += step) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int j = jb + q;
                        const float4 s = s4[j];
                        const float dx = xi[0] - s.x, dy = xi[1] - s.y;
                        float r2 = fmaf(dy, dy, dx * dx);
                        if constexpr (D == 3) {
                            const float dz = xi[2] - s.z;
                            r2 = fmaf(dz, dz, r2);
                        }
                        const T gk = j < cw ? m2l_kernel<KIND>(r2, param2, diag) : T(0);
                        if constexpr (NR == 1) {
                            acc[q][0] = fmaf(gk, D == 3 ? s.w : s.z, acc[q][0]);
                        } else {
#pragma unroll
                            for (int c = 0; c < NR; ++c) acc[q][c] = fmaf(gk, sv[j * NR + c], acc[q][c]);
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int c = 0; c < NR; ++c) acc[0][c] = (acc[0][c] + acc[1][c]) + (acc[2][c] + acc[3][c]);
        __syncthreads();
        if (part > 0 && active) {
#pragma unroll
            for (int c = 0; c < NR; ++c) red[((part - 1) * R + li) * NR + c] = acc[0][c];
        }
        __syncthreads();
        if (part == 0 && active) {
            for (int p2 = 1; p2 < nparts; ++p2)
#pragma unroll
                for (int c = 0; c < NR; ++c) acc[0][c] += red[((p2 - 1) * R + li) * NR + c];
        }
        if (part == 0 && active) {
#pragma unroll
            for (int c = 0; c < NR; ++c) vec[(dst[t] + i) * nrhs + c0 + c] = acc[0][c];
        }
    }
}

// ---- (H2+H)*: t = V^T q_Y per block (partial sums over point chunks) ----------
template <typename T>
__global__ void k_lr_vtq(int64_t b0, int64_t nblk, const int64_t* __restrict__ y0,
                         const int64_t* __restrict__ my, const int32_t* __restrict__ kk,
                         const int64_t* __restrict__ voffs, const int64_t* __restrict__ toffs,
                         const T* __restrict__ ops, const T* __restrict__ q, T* __restrict__ t,
                         int chunk, int nrhs, int col) {
    const int64_t blk = b0 + blockIdx.y;
    if (blockIdx.y >= nblk) return;
    const int64_t m = my[blk];
    const int64_t i0 = int64_t(blockIdx.x) * chunk;
    if (i0 >= m) return;
    const int64_t i1 = min(m, i0 + chunk);
    const int k = kk[blk];
    const T* V = ops + voffs[blk];
    const T* qy = q + y0[blk] * nrhs;
    __shared__ T red[32];
    for (int c = 0; c < k; ++c) {
        T part = T(0);
        for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x)
            part += V[c * m + i] * qy[i * nrhs + col];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        if (threadIdx.x % kWarp == 0) red[threadIdx.x / kWarp] = part;
        __syncthreads();
        if (threadIdx.x < kWarp) {
            T s = threadIdx.x < blockDim.x / kWarp ? red[threadIdx.x] : T(0);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (threadIdx.x == 0) atomicAdd(t + (toffs[blk] + c) * nrhs + col, s);
        }
        __syncthreads();
    }
}

// phi(X) += sum_{blocks of X} U t, one thread per target point
template <typename T>
__global__ void k_lr_ut(int64_t g0, int64_t ngroup, const int64_t* __restrict__ gptr,
                        const int64_t* __restrict__ x0, const int64_t* __restrict__ mx,
                        const int32_t* __restrict__ kk, const int64_t* __restrict__ uoffs,
                        const int64_t* __restrict__ toffs, const T* __restrict__ ops,
                        const T* __restrict__ t, T* __restrict__ phi, int nrhs, int col) {
    const int64_t g = g0 + blockIdx.y;
    if (blockIdx.y >= ngroup) return;
    const int64_t bfirst = gptr[g], blast = gptr[g + 1];
    const int64_t m = mx[bfirst];
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= m) return;
    T acc = T(0);
    for (int64_t blk = bfirst; blk < blast; ++blk) {
        const int k = kk[blk];
        const T* U = ops + uoffs[blk];
        const T* tb = t + toffs[blk] * nrhs + col;
        for (int c = 0; c < k; ++c) acc += U[c * m + i] * tb[int64_t(c) * nrhs];
    }
    phi[(x0[bfirst] + i) * nrhs + col] += acc;
}

// ---- M2L blocks formed on the device ------------------------------------
// G(r) from r^2 in fp64 with every operation rounded on its own (no fused
// multiply-add), the same operations as the host construction: r = sqrt(r^2);
// log r, 1 / r, 1 / sqrt(1 + (r / c)^2), exp(-r).
template <int KIND>
__device__ __forceinline__ double fill_kernel(double r2, double c, double diag) {
    if (r2 == 0.0) return diag;
    const double r = __dsqrt_rn(r2);
    if constexpr (KIND == 0) return log(r);
    else if constexpr (KIND == 1) return __ddiv_rn(1.0, r);
    else if constexpr (KIND == 2) {
        const double s = __ddiv_rn(r, c);
        return __ddiv_rn(1.0, __dsqrt_rn(__dadd_rn(1.0, __dmul_rn(s, s))));
    } else return exp(-r);
}

// fp64 -> stored entry, rounded once (bf16: round-to-nearest-even of the
// float's upper 16 bits; double-float: hi = fl32(a), lo = fl32(a - hi))
template <class A> struct StoreAs;
template <> struct StoreAs<F64> {
    __device__ static double of(double a) { return a; }
};
template <> struct StoreAs<F32> {
    __device__ static float of(double a) { return __double2float_rn(a); }
};
template <> struct StoreAs<BF16> {
    __device__ static __nv_bfloat16 of(double a) {
        const uint32_t u = __float_as_uint(__double2float_rn(a));
        const uint16_t b = ((u & 0x7F800000u) == 0x7F800000u && (u & 0x007FFFFFu))
                               ? uint16_t(0x7FC0)
                               : uint16_t((u + 0x7FFFu + ((u >> 16) & 1u)) >> 16);
        return __ushort_as_bfloat16(b);
    }
};
template <> struct StoreAs<DF> {
    __device__ static float2 of(double a) {
        const float hi = __double2float_rn(a);
        return make_float2(hi, __double2float_rn(__dsub_rn(a, double(hi))));
    }
};

// Stored coupling blocks T_{X,Y} = G(t^{X,i}, t^{Y,i}) (§3.6.4) written by the
// device from the pivot coordinates: one CTA per M2L task (target X) fills its
// block row, rows x kpad row-major at ops + aoff; column k of segment e is the
// source pivot whose coefficient sits at seg_off[e] + (k - seg_col[e]), row r
// the target pivot of coefficient dst + r.  px[k * vlen + o] is coordinate k
// of the pivot of v / u offset o.  Threads run along the columns of one row
// segment, so the writes are contiguous; padding columns are not written (the
// caller clears the region first).
template <class A, int D, int KIND>
__global__ void __launch_bounds__(256) k_m2l_fill(
    int64_t ntask, const int64_t* __restrict__ dst, const int32_t* __restrict__ rows,
    const int32_t* __restrict__ kpad, const int64_t* __restrict__ aoff,
    const int64_t* __restrict__ seg_ptr, const int64_t* __restrict__ seg_off,
    const int32_t* __restrict__ seg_len, const int32_t* __restrict__ seg_col,
    const double* __restrict__ px, int64_t vlen, int64_t v_base, int64_t u_base, double param,
    double diag, typename A::S* __restrict__ ops) {
    const int64_t t = blockIdx.x;
    if (t >= ntask) return;
    const int nr = rows[t];
    const int64_t kp = kpad[t];
    const int64_t d0 = dst[t] - u_base;
    typename A::S* Am = ops + aoff[t];
    for (int64_t e = seg_ptr[t]; e < seg_ptr[t + 1]; ++e) {
        const int len = seg_len[e];
        const int64_t col = seg_col[e];
        const int64_t s0 = seg_off[e] - v_base;
        const int64_t n = int64_t(nr) * len;
        for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
            const int r = int(j / len), c = int(j - int64_t(r) * len);
            double r2 = 0.0;
#pragma unroll
            for (int k = 0; k < D; ++k) {
                const double dx = __dsub_rn(px[k * vlen + d0 + r], px[k * vlen + s0 + c]);
                r2 = __dadd_rn(r2, __dmul_rn(dx, dx));
            }
            Am[int64_t(r) * kp + col + c] = StoreAs<A>::of(fill_kernel<KIND>(r2, param, diag));
        }
    }
}

}  // namespace h2
