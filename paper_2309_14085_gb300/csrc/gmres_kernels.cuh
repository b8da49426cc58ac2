// FP64 vector kernels of the GMRES solver (§6 solves the systems K sigma = f
// with GMRES; here on the device).  The Krylov basis V is column-major,
// N x nvec; every reduction is two-pass with a fixed order (deterministic).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace h2 {

constexpr int kDotBlocks = 304;      // 2 x 152 SMs: row slices
constexpr int kDotThreads = 256;     // 8 warps, one vector each
constexpr int kDotWarps = kDotThreads / 32;

inline dim3 dot_grid(int nvec) { return dim3(kDotBlocks, unsigned((nvec + kDotWarps - 1) / kDotWarps)); }

// partial[b * nvec + v] = sum over row slice b of V[:, v] . w.  Grid
// dot_grid(nvec): block (b, y) covers slice b for vectors 8 y .. 8 y + 7, one
// warp per vector (lanes stride the slice, then a shuffle reduction), so long
// Krylov bases need no block-wide barrier per vector.
__global__ void k_multidot(const double* __restrict__ V, int64_t ldv, int nvec,
                           const double* __restrict__ w, int64_t N,
                           double* __restrict__ partial) {
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int v = int(blockIdx.y) * kDotWarps + warp;
    if (v >= nvec) return;
    const int64_t per = (N + gridDim.x - 1) / gridDim.x;
    const int64_t i0 = int64_t(blockIdx.x) * per, i1 = min(N, i0 + per);
    const double* col = V + int64_t(v) * ldv;
    double s = 0.0;
    for (int64_t k = i0 + lane; k < i1; k += 32) s = fma(col[k], w[k], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) partial[int64_t(blockIdx.x) * nvec + v] = s;
}

// out[i] = sum_b partial[b * nvec + i], b in order
__global__ void k_reduce_partials(const double* __restrict__ partial, int nblk, int nvec,
                                  double* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nvec) return;
    double t = 0.0;
    for (int b = 0; b < nblk; ++b) t += partial[int64_t(b) * nvec + i];
    out[i] = t;
}

// w += alpha * V[:, 0:nvec] c    (c on the device)
__global__ void k_gemv_cols(const double* __restrict__ V, int64_t ldv, int nvec,
                            const double* __restrict__ c, double alpha, double* __restrict__ w,
                            int64_t N) {
    const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (k >= N) return;
    double s = 0.0;
    for (int v = 0; v < nvec; ++v) s = fma(V[int64_t(v) * ldv + k], c[v], s);
    w[k] = fma(alpha, s, w[k]);
}

// y = a * x + b * y
__global__ void k_axpby(double a, const double* __restrict__ x, double b, double* __restrict__ y,
                        int64_t N) {
    const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (k < N) y[k] = a * x[k] + b * y[k];
}

// z = a * x + b * y
__global__ void k_axpbyz(double a, const double* __restrict__ x, double b,
                         const double* __restrict__ y, double* __restrict__ z, int64_t N) {
    const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (k < N) z[k] = a * x[k] + b * y[k];
}

}  // namespace h2
