// CUDA kernels of the H2* matrix-vector product (§5.1.2, §5.2.2, App. A.2),
// templated on the storage / arithmetic type T (double or float).
//
// Data layout (all in HBM, built once per geometry):
//   ops      every operator entry: leaf bases U_X (m x r, row-major), L2L
//            matrices U~_{X_c X} (r_c x r_X, row-major), M2L blocks per target
//            [T_{X,Y1} | T_{X,Y2} | ...] (r_X x kpad, row-major, zero padded
//            to a multiple of 4 columns), (H2+H)* factors (column-major).
//   v, u     multipole / local coefficients of every (basis, level, box) slot.
//   q, phi   charges / potentials in tree order (leaf-contiguous).
//   xs       coordinates in tree order, structure of arrays (xs[k * N + i]).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace h2 {

constexpr int kWarp = 32;

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// G(r) from r^2; the diagonal (coincident points) takes `diag`.
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
template <typename T>
__global__ void k_gather(const double* __restrict__ X, const int64_t* __restrict__ perm,
                         T* __restrict__ q, int64_t N) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < N) q[i] = T(X[perm[i]]);
}

template <typename T>
__global__ void k_scatter(const T* __restrict__ phi, const int64_t* __restrict__ perm,
                          double* __restrict__ Y, int64_t N) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < N) Y[perm[i]] = double(phi[i]);
}

// ---- P2M: v_X = U_X^T q_X at the leaves, one warp per (basis, leaf) ----------
template <typename T>
__global__ void k_p2m(int64_t ntask, int64_t nleaf, int64_t box_total, int64_t leaf_base,
                      const int64_t* __restrict__ leaf_ptr, const int32_t* __restrict__ rank,
                      const int64_t* __restrict__ voff, const int64_t* __restrict__ uoff,
                      const T* __restrict__ ops, const T* __restrict__ q, T* __restrict__ v) {
    const int64_t task = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) / kWarp;
    const int lane = threadIdx.x % kWarp;
    if (task >= ntask) return;
    const int64_t b = task / nleaf, L = task - b * nleaf;
    const int64_t s = b * box_total + leaf_base + L;
    const int r = rank[s];
    if (r == 0) return;
    const int64_t p0 = leaf_ptr[L];
    const int m = int(leaf_ptr[L + 1] - p0);
    const T* U = ops + uoff[s];
    for (int j = lane; j < r; j += kWarp) {
        T acc = T(0);
        for (int i = 0; i < m; ++i) acc += U[int64_t(i) * r + j] * q[p0 + i];
        v[voff[s] + j] = acc;
    }
}

// ---- M2M: v_X = sum_c U~_{X_c X}^T v_{X_c}, one warp per parent -------------
template <typename T>
__global__ void k_m2m(const int64_t* __restrict__ tasks, int64_t ntask, int64_t box_total,
                      int64_t base_l, int64_t base_child, int nchild,
                      const int32_t* __restrict__ rank, const int64_t* __restrict__ voff,
                      const int64_t* __restrict__ utoff, const T* __restrict__ ops,
                      T* __restrict__ v) {
    const int64_t w = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) / kWarp;
    const int lane = threadIdx.x % kWarp;
    if (w >= ntask) return;
    const int64_t s = tasks[w];
    const int64_t b = s / box_total, X = s - b * box_total - base_l;
    const int r = rank[s];
    for (int j = lane; j < r; j += kWarp) {
        T acc = T(0);
        for (int c = 0; c < nchild; ++c) {
            const int64_t sc = b * box_total + base_child + X * nchild + c;
            const int rc = rank[sc];
            if (rc == 0) continue;
            const T* Ut = ops + utoff[sc];
            const T* vc = v + voff[sc];
            for (int i = 0; i < rc; ++i) acc += Ut[int64_t(i) * r + j] * vc[i];
        }
        v[voff[s] + j] = acc;
    }
}

// ---- M2L: u_X = sum_{Y in IL(X)} T_{X,Y} v_Y, one CTA per target -----------
// The sources' coefficients are gathered into shared memory (kpad values);
// each warp takes rows of the concatenated coupling block and streams them
// with coalesced vector loads.
template <typename T>
__global__ void k_m2l(int64_t ntask, const int64_t* __restrict__ slot,
                      const int64_t* __restrict__ toff, const int32_t* __restrict__ kpad,
                      const int64_t* __restrict__ src_ptr, const int64_t* __restrict__ src,
                      const int32_t* __restrict__ rank, const int64_t* __restrict__ voff,
                      const T* __restrict__ ops, const T* __restrict__ v, T* __restrict__ u) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* vg = reinterpret_cast<T*>(smem_raw);
    const int64_t task = blockIdx.x;
    if (task >= ntask) return;
    const int64_t s = slot[task];
    const int r = rank[s];
    const int kp = kpad[task];
    int col = 0;
    for (int64_t e = src_ptr[task]; e < src_ptr[task + 1]; ++e) {
        const int64_t sy = src[e];
        const int ry = rank[sy];
        const T* vy = v + voff[sy];
        for (int j = threadIdx.x; j < ry; j += blockDim.x) vg[col + j] = vy[j];
        col += ry;
    }
    for (int j = col + threadIdx.x; j < kp; j += blockDim.x) vg[j] = T(0);
    __syncthreads();
    const int warp = threadIdx.x / kWarp, lane = threadIdx.x % kWarp;
    const int nwarp = blockDim.x / kWarp;
    const T* Tm = ops + toff[task];
    using V2 = typename std::conditional<sizeof(T) == 8, double2, float4>::type;
    constexpr int W = sizeof(V2) / sizeof(T);   // elements per vector load (2 or 4)
    for (int row = warp; row < r; row += nwarp) {
        const V2* trow = reinterpret_cast<const V2*>(Tm + int64_t(row) * kp);
        const V2* vrow = reinterpret_cast<const V2*>(vg);
        T acc = T(0);
        const int nv = kp / W;
#pragma unroll 4
        for (int k = lane; k < nv; k += kWarp) {
            const V2 a = __ldg(trow + k);
            const V2 x = vrow[k];
            if constexpr (W == 2) {
                acc += a.x * x.x + a.y * x.y;
            } else {
                acc += a.x * x.x + a.y * x.y + a.z * x.z + a.w * x.w;
            }
        }
        acc = warp_sum(acc);
        if (lane == 0) u[voff[s] + row] = acc;
    }
}

// ---- L2L: u_{X_c} += U~_{X_c X} u_X, one warp per child ---------------------
template <typename T>
__global__ void k_l2l(const int64_t* __restrict__ tasks, int64_t ntask, int64_t box_total,
                      int64_t base_l, int64_t base_parent, int dshift,
                      const int32_t* __restrict__ rank, const int64_t* __restrict__ voff,
                      const int64_t* __restrict__ utoff, const T* __restrict__ ops,
                      T* __restrict__ u) {
    const int64_t w = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) / kWarp;
    const int lane = threadIdx.x % kWarp;
    if (w >= ntask) return;
    const int64_t s = tasks[w];
    const int64_t b = s / box_total, X = s - b * box_total - base_l;
    const int64_t sp = b * box_total + base_parent + (X >> dshift);
    const int rc = rank[s], rp = rank[sp];
    const T* Ut = ops + utoff[s];
    const T* up = u + voff[sp];
    T* uc = u + voff[s];
    for (int i = 0; i < rc; ++i) {
        T part = T(0);
        for (int j = lane; j < rp; j += kWarp) part += Ut[int64_t(i) * rp + j] * up[j];
        part = warp_sum(part);
        if (lane == 0) uc[i] += part;
    }
}

// ---- leaves: phi_X = sum_b U_X^b u_X^b + sum_{X' in N(X)} K_{t^X, s^X'} q_X' ----
// One CTA per leaf; each thread owns targets; source points of the neighbour
// leaves are staged through shared memory in tiles of blockDim.
template <typename T, int D, int KIND>
__global__ void k_leaf(int64_t nleaf, int nb, int64_t box_total, int64_t leaf_base,
                       const int64_t* __restrict__ leaf_ptr, const int64_t* __restrict__ near_ptr,
                       const int64_t* __restrict__ near_idx, const int32_t* __restrict__ rank,
                       const int64_t* __restrict__ voff, const int64_t* __restrict__ uoff,
                       const T* __restrict__ ops, const T* __restrict__ u,
                       const T* __restrict__ xs, int64_t N, const T* __restrict__ q,
                       T* __restrict__ phi, T param, T diag) {
    constexpr int TILE = 128;
    __shared__ T sx[D][TILE];
    __shared__ T sq[TILE];
    const int64_t L = blockIdx.x;
    if (L >= nleaf) return;
    const int64_t p0 = leaf_ptr[L];
    const int m = int(leaf_ptr[L + 1] - p0);
    for (int i0 = 0; i0 < m; i0 += blockDim.x) {
        const int i = i0 + threadIdx.x;
        const bool active = i < m;
        T acc = T(0);
        T xi[D];
        if (active) {
#pragma unroll
            for (int k = 0; k < D; ++k) xi[k] = xs[k * N + p0 + i];
            for (int b = 0; b < nb; ++b) {
                const int64_t s = b * box_total + leaf_base + L;
                const int r = rank[s];
                if (r == 0) continue;
                const T* U = ops + uoff[s] + int64_t(i) * r;
                const T* ub = u + voff[s];
                for (int j = 0; j < r; ++j) acc += U[j] * ub[j];
            }
        }
        for (int64_t e = near_ptr[L]; e < near_ptr[L + 1]; ++e) {
            const int64_t Y = near_idx[e];
            const int64_t s0 = leaf_ptr[Y];
            const int ms = int(leaf_ptr[Y + 1] - s0);
            for (int j0 = 0; j0 < ms; j0 += TILE) {
                const int nt = min(TILE, ms - j0);
                __syncthreads();
                for (int j = threadIdx.x; j < nt; j += blockDim.x) {
#pragma unroll
                    for (int k = 0; k < D; ++k) sx[k][j] = xs[k * N + s0 + j0 + j];
                    sq[j] = q[s0 + j0 + j];
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
                        acc += kernel_r2<T, KIND>(r2, param, diag) * sq[j];
                    }
                }
            }
        }
        if (active) phi[p0 + i] = acc;
    }
}

// ---- (H2+H)*: t = V^T q_Y per block (atomic partial sums over point chunks) --
template <typename T>
__global__ void k_lr_vtq(int64_t b0, int64_t nblk, const int64_t* __restrict__ y0,
                         const int64_t* __restrict__ my, const int32_t* __restrict__ kk,
                         const int64_t* __restrict__ voffs, const int64_t* __restrict__ toffs,
                         const T* __restrict__ ops, const T* __restrict__ q, T* __restrict__ t,
                         int chunk) {
    // grid.x over (block, column, chunk) flattened by the host into work items
    // passed as blockIdx.y = block index relative to b0, blockIdx.x = chunk id,
    // loop over columns inside.
    const int64_t blk = b0 + blockIdx.y;
    if (blockIdx.y >= nblk) return;
    const int64_t m = my[blk];
    const int64_t i0 = int64_t(blockIdx.x) * chunk;
    if (i0 >= m) return;
    const int64_t i1 = min(m, i0 + chunk);
    const int k = kk[blk];
    const T* V = ops + voffs[blk];
    const T* qy = q + y0[blk];
    __shared__ T red[32];
    for (int c = 0; c < k; ++c) {
        T part = T(0);
        for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) part += V[c * m + i] * qy[i];
        part = warp_sum(part);
        if (threadIdx.x % kWarp == 0) red[threadIdx.x / kWarp] = part;
        __syncthreads();
        if (threadIdx.x < kWarp) {
            T s = threadIdx.x < blockDim.x / kWarp ? red[threadIdx.x] : T(0);
            s = warp_sum(s);
            if (threadIdx.x == 0) atomicAdd(t + toffs[blk] + c, s);
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
                        const T* __restrict__ t, T* __restrict__ phi) {
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
        const T* tb = t + toffs[blk];
        for (int c = 0; c < k; ++c) acc += U[c * m + i] * tb[c];
    }
    phi[x0[bfirst] + i] += acc;
}

}  // namespace h2
