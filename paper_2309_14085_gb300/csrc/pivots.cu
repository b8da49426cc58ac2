// Pivot search on the device: the partially pivoted ACA of the B2T and T2B
// NCA sweeps (§3.6, Algorithm 1, §5.1.1 item 2) for all ACA problems of a
// level at once.
//
// The device runs the host's ACA (build.cpp, `aca`) step by step: the same
// first-row start, the same first-index argmax rules, the same noise floor,
// the same look-ahead stopping rule, and the same IEEE operations on every
// value -- kernel entries (1/r and the IMQ through correctly rounded square
// roots and divisions), residual rows and columns (a rounded product and a
// rounded subtraction per cross, in cross order) and the four sums of the
// stopping estimate in the host's fixed order (fused multiply-adds over
// segments of 4096 terms on 256 lanes, a pairwise tree per segment, segment
// totals in order).  Its pivots are therefore the host's, index for
// index, for 1/r and the IMQ; log r and exp(-r) go through the device's
// log / exp, which may differ from the host library's in the last bit, so
// their pivots can differ where a comparison is that close.
//
// One ACA step is six short launches over every live problem of the level,
// with no waiting inside a kernel: a search set J (and a row set I) is cut
// into segments of 4096 entries with one CTA each, so a level with a few large
// problems (the top T2B levels: a handful of boxes, each searching 10^5
// points) spreads over the whole GPU like a level of thousands of small ones.
//   A  [J segments]  fresh residual row when one is due; segment argmax of |r|
//   B  [problem]     column pivot jb (or the row is spent: next free row)
//   C  [J, I segs]   v = r / r[jb]; residual column u; |v|^2, |u|^2 segments;
//                    segment argmax of |u| over unused rows
//   D  [problem]     |u|^2, |v|^2; next row ib
//   E  [J, I segs]   one sweep over the previous crosses: the next residual
//                    row and v_l . v, and u_l . u, per segment
//   F  [problem]     Frobenius estimate, stopping test, next row
// The crosses live in HBM (U: k x |I|, V: k x |J|, cross-major); step E
// streams them once, the work the host spends most of its construction time
// on.  The host loop only launches; it reads one counter every eight steps to
// see whether every problem has finished.  A problem that needs more crosses
// than its workspace holds stops with a status and is run again with more
// room; beyond 1024 crosses, or when the device has no memory for its batch,
// the host solves it.

#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <mutex>
#include <cstdio>
#include <string>
#include <vector>

#include "h2_internal.hpp"

namespace h2 {
namespace {

constexpr int kNT = 256;             // threads per CTA = lanes of the stopping sums
constexpr int kSeg = 4096;           // terms per segment
constexpr int kPer = kSeg / kNT;     // terms per thread and segment
constexpr int kLC = 8;               // previous crosses per sweep chunk (one tree per warp)
constexpr int kKMax = 1024;          // crosses a device problem may hold
constexpr int kLook = 2;             // the host's look-ahead (kAcaLookahead)
constexpr double kNoise = 0x1p-46;   // the host's noise floor (kAcaNoise)

struct Prob {
    int64_t i0, j0;     // first entry in Iidx / Jidx
    int64_t ws;         // workspace offset (doubles)
    int64_t out;        // output offset (rows / cols entries)
    int32_t nI, nJ, kc, nsI, nsJ, pad;
};

// state of one problem between launches
struct St {
    int i, k, first, done, status, fresh, ok, fuse, jb, ib, par, pad;
    double S2, pmax, piv, uu, vv;
};

struct Lv {
    const double* x;            // N x d tree-order coordinates
    int d, kind;
    double c, diag, eps;
    const int32_t* Iidx;
    const int32_t* Jidx;
    const Prob* prob;
    St* st;
    double* ws;
    int32_t* rows;
    int32_t* cols;
    const int32_t* mapJ;        // J-segment CTA -> problem
    const int32_t* mapI;        // I-segment CTA -> problem
    const int64_t* segJ0;       // first J-segment CTA of each problem
    const int64_t* segI0;
    int64_t totJ;
    int32_t* ndone;             // problems finished
};

// a problem's workspace (doubles), in this order
struct WS {
    double *xI, *xJ, *U, *V, *r0, *r1, *col, *svv, *suu, *spv, *spu, *arv, *ari, *auv, *aui;
    unsigned char *ur, *uc;
};

__host__ __device__ inline int64_t ws_doubles(int64_t d, int64_t nI, int64_t nJ, int64_t kc, int64_t nsI,
                                             int64_t nsJ) {
    const int64_t w = d * (nI + nJ) + kc * (nI + nJ) + 2 * nJ + kc + nsJ + nsI + kc * (nsJ + nsI) +
                      2 * nsJ + 2 * nsI + (nI + nJ + 7) / 8;
    return (w + 31) / 32 * 32;
}

__device__ inline WS ws_of(const Lv& L, const Prob& P) {
    WS w;
    const int64_t d = L.d, nI = P.nI, nJ = P.nJ, kc = P.kc, nsI = P.nsI, nsJ = P.nsJ;
    double* p = L.ws + P.ws;
    w.xI = p; p += d * nI;
    w.xJ = p; p += d * nJ;
    w.U = p; p += kc * nI;
    w.V = p; p += kc * nJ;
    w.r0 = p; p += nJ;
    w.r1 = p; p += nJ;
    w.col = p; p += kc;
    w.svv = p; p += nsJ;
    w.suu = p; p += nsI;
    w.spv = p; p += kc * nsJ;
    w.spu = p; p += kc * nsI;
    w.arv = p; p += nsJ;
    w.ari = p; p += nsJ;
    w.auv = p; p += nsI;
    w.aui = p; p += nsI;
    w.ur = reinterpret_cast<unsigned char*>(p);
    w.uc = w.ur + nI;
    return w;
}

__device__ __forceinline__ double kernel_value(double s, int kind, double c, double diag) {
    if (s == 0.0) return diag;
    const double r = __dsqrt_rn(s);
    switch (kind) {
        case 0: return log(r);
        case 1: return __ddiv_rn(1.0, r);
        case 2: {
            const double t = __ddiv_rn(r, c);
            return __ddiv_rn(1.0, __dsqrt_rn(__dadd_rn(1.0, __dmul_rn(t, t))));
        }
        default: return exp(-r);
    }
}

// G(|x_a - y_j|) with the squares summed in coordinate order (coordinate-major
// copies of the problem's points)
__device__ __forceinline__ double entry(const Lv& L, const WS& w, int nI, int a, int nJ, int j) {
    double s = 0.0;
    for (int k = 0; k < L.d; ++k) {
        const double q = __dsub_rn(w.xI[int64_t(k) * nI + a], w.xJ[int64_t(k) * nJ + j]);
        s = __dadd_rn(s, __dmul_rn(q, q));
    }
    return kernel_value(s, L.kind, L.c, L.diag);
}

// One warp sums 256 lane partials in the host's pairwise order (p + w into p
// for w = 128, ..., 1); the result is returned in lane 0.
__device__ __forceinline__ double lane_tree(double* s, int lane) {
#pragma unroll
    for (int m = 0; m < 4; ++m) s[lane + 32 * m] = __dadd_rn(s[lane + 32 * m], s[lane + 32 * m + 128]);
    __syncwarp();
#pragma unroll
    for (int m = 0; m < 2; ++m) s[lane + 32 * m] = __dadd_rn(s[lane + 32 * m], s[lane + 32 * m + 64]);
    __syncwarp();
    double v = __dadd_rn(s[lane], s[lane + 32]);
#pragma unroll
    for (int w = 16; w >= 1; w >>= 1) v = __dadd_rn(v, __shfl_down_sync(0xffffffffu, v, w));
    __syncwarp();
    return v;
}

// Block-wide first argmax: the largest value, and among equal values the
// smallest index (INT_MAX when no thread saw a value above its start).  All
// threads return the result.
__device__ __forceinline__ void block_argmax(double& v, int& idx) {
    __shared__ double sv[kNT / 32];
    __shared__ int si[kNT / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        const double v2 = __shfl_xor_sync(0xffffffffu, v, o);
        const int i2 = __shfl_xor_sync(0xffffffffu, idx, o);
        if (v2 > v || (v2 == v && i2 < idx)) { v = v2; idx = i2; }
    }
    __syncthreads();
    if (lane == 0) { sv[warp] = v; si[warp] = idx; }
    __syncthreads();
    v = sv[0];
    idx = si[0];
    for (int w = 1; w < kNT / 32; ++w)
        if (sv[w] > v || (sv[w] == v && si[w] < idx)) { v = sv[w]; idx = si[w]; }
}

// first a < n with flag[a] == 0, INT_MAX if none (all threads)
__device__ __forceinline__ int block_first_free(const unsigned char* flag, int n) {
    __shared__ int si[kNT / 32];
    int v = INT_MAX;
    for (int a = threadIdx.x; a < n; a += kNT)
        if (!flag[a]) { v = a; break; }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if (lane == 0) si[warp] = v;
    __syncthreads();
    v = si[0];
    for (int w = 1; w < kNT / 32; ++w) v = min(v, si[w]);
    return v;
}

// segment sum of one term per thread-slot, tree in lane order, to *out (lane 0 of warp 0)
__device__ __forceinline__ void segment_total(double part, double* out) {
    __shared__ double red[kNT];
    red[threadIdx.x] = part;
    __syncthreads();
    if (threadIdx.x < 32) {
        const double t = lane_tree(red, threadIdx.x);
        if (threadIdx.x == 0) *out = t;
    }
    __syncthreads();
}

// coordinates and flags
__global__ void __launch_bounds__(kNT) k_init(Lv L) {
    const bool jrole = blockIdx.x < L.totJ;
    const int X = jrole ? L.mapJ[blockIdx.x] : L.mapI[blockIdx.x - L.totJ];
    const Prob P = L.prob[X];
    const WS w = ws_of(L, P);
    const int d = L.d;
    if (jrole) {
        const int g = int(blockIdx.x - L.segJ0[X]);
        for (int m = 0; m < kPer; ++m) {
            const int j = g * kSeg + threadIdx.x + kNT * m;
            if (j >= P.nJ) break;
            const int64_t p = L.Jidx[P.j0 + j];
            for (int k = 0; k < d; ++k) w.xJ[int64_t(k) * P.nJ + j] = L.x[p * d + k];
            w.uc[j] = 0;
        }
    } else {
        const int g = int(blockIdx.x - L.totJ - L.segI0[X]);
        for (int m = 0; m < kPer; ++m) {
            const int a = g * kSeg + threadIdx.x + kNT * m;
            if (a >= P.nI) break;
            const int64_t p = L.Iidx[P.i0 + a];
            for (int k = 0; k < d; ++k) w.xI[int64_t(k) * P.nI + a] = L.x[p * d + k];
            w.ur[a] = 0;
        }
    }
}

// A: a fresh residual row when due; segment argmax of |r| over unused columns
__global__ void __launch_bounds__(kNT) k_stepA(Lv L) {
    __shared__ double col[kKMax];
    const int X = L.mapJ[blockIdx.x];
    const St s = L.st[X];
    if (s.done) return;
    const Prob P = L.prob[X];
    const WS w = ws_of(L, P);
    const int g = int(blockIdx.x - L.segJ0[X]);
    const int nI = P.nI, nJ = P.nJ, k = s.k;
    double* r = s.par ? w.r1 : w.r0;
    if (s.fresh) {
        for (int l = threadIdx.x; l < k; l += kNT) col[l] = w.U[int64_t(l) * nI + s.i];
        __syncthreads();
        for (int m = 0; m < kPer; ++m) {
            const int j = g * kSeg + threadIdx.x + kNT * m;
            if (j >= nJ) break;
            double val = entry(L, w, nI, s.i, nJ, j);
            for (int l = 0; l < k; ++l) val = __dsub_rn(val, __dmul_rn(col[l], w.V[int64_t(l) * nJ + j]));
            r[j] = val;
        }
    }
    double best = -1.0;
    int jb = INT_MAX;
    for (int m = 0; m < kPer; ++m) {
        const int j = g * kSeg + threadIdx.x + kNT * m;
        if (j >= nJ) break;
        const double a = w.uc[j] ? -1.0 : fabs(r[j]);
        if (a > best) { best = a; jb = j; }
    }
    block_argmax(best, jb);
    if (threadIdx.x == 0) {
        w.arv[g] = best;
        w.ari[g] = double(jb);
    }
}

// B: the column pivot, or the row is spent
__global__ void __launch_bounds__(kNT) k_stepB(Lv L) {
    const int X = blockIdx.x;
    St s = L.st[X];
    if (s.done) return;
    const Prob P = L.prob[X];
    const WS w = ws_of(L, P);
    double best = -1.0;
    int jb = INT_MAX;
    for (int g = threadIdx.x; g < P.nsJ; g += kNT) {
        const double v = w.arv[g];
        const int i = int(w.ari[g]);
        if (v > best || (v == best && i < jb)) { best = v; jb = i; }
    }
    block_argmax(best, jb);
    if (threadIdx.x == 0) w.ur[s.i] = 1;
    __syncthreads();
    if (best <= __dmul_rn(kNoise, s.pmax) || best <= 0.0) {
        const int ni = block_first_free(w.ur, P.nI);
        if (threadIdx.x == 0) {
            s.ok = 0;
            if (ni == INT_MAX) {
                s.done = 1;
                atomicAdd(L.ndone, 1);
            } else {
                s.i = ni;
                s.fresh = 1;
            }
            L.st[X] = s;
        }
        return;
    }
    for (int l = threadIdx.x; l < s.k; l += kNT) w.col[l] = w.V[int64_t(l) * P.nJ + jb];
    if (threadIdx.x == 0) {
        s.pmax = (s.pmax < best) ? best : s.pmax;
        s.jb = jb;
        s.piv = (s.par ? w.r1 : w.r0)[jb];
        s.ok = 1;
        s.fresh = 0;
        w.uc[jb] = 1;
        L.st[X] = s;
    }
}

// C: v = r / r[jb] and |v|^2 (J segments); residual column u, |u|^2 and the
// segment argmax of |u| over unused rows (I segments)
__global__ void __launch_bounds__(kNT) k_stepC(Lv L) {
    __shared__ double col[kKMax];
    const bool jrole = blockIdx.x < L.totJ;
    const int X = jrole ? L.mapJ[blockIdx.x] : L.mapI[blockIdx.x - L.totJ];
    const St s = L.st[X];
    if (s.done || !s.ok) return;
    const Prob P = L.prob[X];
    const WS w = ws_of(L, P);
    const int nI = P.nI, nJ = P.nJ, k = s.k;
    if (jrole) {
        const int g = int(blockIdx.x - L.segJ0[X]);
        const double* r = s.par ? w.r1 : w.r0;
        double* v = w.V + int64_t(k) * nJ;
        double part = 0.0;
        for (int m = 0; m < kPer; ++m) {
            const int j = g * kSeg + threadIdx.x + kNT * m;
            if (j >= nJ) break;
            const double vj = __ddiv_rn(r[j], s.piv);
            v[j] = vj;
            part = __fma_rn(vj, vj, part);
        }
        segment_total(part, w.svv + g);
    } else {
        const int g = int(blockIdx.x - L.totJ - L.segI0[X]);
        for (int l = threadIdx.x; l < k; l += kNT) col[l] = w.col[l];
        __syncthreads();
        double* u = w.U + int64_t(k) * nI;
        double part = 0.0, best = -1.0;
        int ib = INT_MAX;
        for (int m = 0; m < kPer; ++m) {
            const int a = g * kSeg + threadIdx.x + kNT * m;
            if (a >= nI) break;
            double val = entry(L, w, nI, a, nJ, s.jb);
            for (int l = 0; l < k; ++l) val = __dsub_rn(val, __dmul_rn(col[l], w.U[int64_t(l) * nI + a]));
            u[a] = val;
            part = __fma_rn(val, val, part);
            const double q = w.ur[a] ? -1.0 : fabs(val);
            if (q > best) { best = q; ib = a; }
        }
        segment_total(part, w.suu + g);
        block_argmax(best, ib);
        if (threadIdx.x == 0) {
            w.auv[g] = best;
            w.aui[g] = double(ib);
        }
    }
}

// D: |u|^2, |v|^2 and the next row
__global__ void __launch_bounds__(kNT) k_stepD(Lv L) {
    const int X = blockIdx.x;
    St s = L.st[X];
    if (s.done || !s.ok) return;
    const Prob P = L.prob[X];
    const WS w = ws_of(L, P);
    double bi = -1.0;
    int ib = INT_MAX;
    for (int g = threadIdx.x; g < P.nsI; g += kNT) {
        const double v = w.auv[g];
        const int i = int(w.aui[g]);
        if (v > bi || (v == bi && i < ib)) { bi = v; ib = i; }
    }
    block_argmax(bi, ib);
    const bool fuse = bi > 0.0;
    if (fuse)
        for (int l = threadIdx.x; l < s.k; l += kNT) w.col[l] = w.U[int64_t(l) * P.nI + ib];
    if (threadIdx.x == 0) {
        double uu = 0.0, vv = 0.0;
        for (int g = 0; g < P.nsI; ++g) uu = __dadd_rn(uu, w.suu[g]);
        for (int g = 0; g < P.nsJ; ++g) vv = __dadd_rn(vv, w.svv[g]);
        s.uu = uu;
        s.vv = vv;
        s.fuse = fuse ? 1 : 0;
        s.ib = fuse ? ib : -1;
        L.st[X] = s;
    }
}

// E: the sweep over the previous crosses -- the next residual row and the
// segment sums of v_l . v (J segments), the segment sums of u_l . u (I)
__global__ void __launch_bounds__(kNT) k_stepE(Lv L) {
    __shared__ double col[kKMax];
    __shared__ double red[kLC][kNT];
    const bool jrole = blockIdx.x < L.totJ;
    const int X = jrole ? L.mapJ[blockIdx.x] : L.mapI[blockIdx.x - L.totJ];
    const St s = L.st[X];
    if (s.done || !s.ok) return;
    const Prob P = L.prob[X];
    const WS w = ws_of(L, P);
    const int nI = P.nI, nJ = P.nJ, k = s.k, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (jrole) {
        const int g = int(blockIdx.x - L.segJ0[X]);
        const bool fuse = s.fuse != 0;
        if (fuse)
            for (int l = tid; l < k; l += kNT) col[l] = w.col[l];
        __syncthreads();
        const double* v = w.V + int64_t(k) * nJ;
        const int j0 = g * kSeg + tid;
        double xr[kPer], vj[kPer];
#pragma unroll
        for (int m = 0; m < kPer; ++m) {
            const int j = j0 + kNT * m;
            const bool in = j < nJ;
            vj[m] = in ? v[j] : 0.0;
            xr[m] = (fuse && in) ? entry(L, w, nI, s.ib, nJ, j) : 0.0;
        }
        for (int c0 = 0; c0 < k; c0 += kLC) {
            const int nl = min(kLC, k - c0);
            double part[kLC];
#pragma unroll
            for (int q = 0; q < kLC; ++q) part[q] = 0.0;
#pragma unroll
            for (int m = 0; m < kPer; ++m) {
                const int j = j0 + kNT * m;
                if (j < nJ) {
#pragma unroll
                    for (int q = 0; q < kLC; ++q)
                        if (q < nl) {
                            const double wv = w.V[int64_t(c0 + q) * nJ + j];
                            if (fuse) xr[m] = __dsub_rn(xr[m], __dmul_rn(col[c0 + q], wv));
                            part[q] = __fma_rn(wv, vj[m], part[q]);
                        }
                }
            }
#pragma unroll
            for (int q = 0; q < kLC; ++q) red[q][tid] = part[q];
            __syncthreads();
            if (warp < nl) {
                const double t = lane_tree(red[warp], lane);
                if (lane == 0) w.spv[int64_t(c0 + warp) * P.nsJ + g] = t;
            }
            __syncthreads();
        }
        if (fuse) {
            const double uib = w.U[int64_t(k) * nI + s.ib];
            double* rn = s.par ? w.r0 : w.r1;
#pragma unroll
            for (int m = 0; m < kPer; ++m) {
                const int j = j0 + kNT * m;
                if (j < nJ) rn[j] = __dsub_rn(xr[m], __dmul_rn(uib, vj[m]));
            }
        }
    } else {
        const int g = int(blockIdx.x - L.totJ - L.segI0[X]);
        const double* u = w.U + int64_t(k) * nI;
        const int a0 = g * kSeg + tid;
        double ua[kPer];
#pragma unroll
        for (int m = 0; m < kPer; ++m) {
            const int a = a0 + kNT * m;
            ua[m] = a < nI ? u[a] : 0.0;
        }
        for (int c0 = 0; c0 < k; c0 += kLC) {
            const int nl = min(kLC, k - c0);
            double part[kLC];
#pragma unroll
            for (int q = 0; q < kLC; ++q) part[q] = 0.0;
#pragma unroll
            for (int m = 0; m < kPer; ++m) {
                const int a = a0 + kNT * m;
                if (a < nI) {
#pragma unroll
                    for (int q = 0; q < kLC; ++q)
                        if (q < nl) part[q] = __fma_rn(w.U[int64_t(c0 + q) * nI + a], ua[m], part[q]);
                }
            }
#pragma unroll
            for (int q = 0; q < kLC; ++q) red[q][tid] = part[q];
            __syncthreads();
            if (warp < nl) {
                const double t = lane_tree(red[warp], lane);
                if (lane == 0) w.spu[int64_t(c0 + warp) * P.nsI + g] = t;
            }
            __syncthreads();
        }
    }
}

// F: the Frobenius estimate, the stopping test and the next row
__global__ void __launch_bounds__(kNT) k_stepF(Lv L) {
    __shared__ double pv[kKMax], pu[kKMax];
    __shared__ int need_row;
    const int X = blockIdx.x;
    St s = L.st[X];
    if (s.done || !s.ok) return;
    const Prob P = L.prob[X];
    const WS w = ws_of(L, P);
    const int k = s.k;
    for (int l = threadIdx.x; l < k; l += kNT) {
        double a = 0.0, b = 0.0;
        for (int g = 0; g < P.nsJ; ++g) a = __dadd_rn(a, w.spv[int64_t(l) * P.nsJ + g]);
        for (int g = 0; g < P.nsI; ++g) b = __dadd_rn(b, w.spu[int64_t(l) * P.nsI + g]);
        pv[l] = a;
        pu[l] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double cross = 0.0;
        for (int l = 0; l < k; ++l) cross = __fma_rn(pu[l], pv[l], cross);
        s.S2 = __dadd_rn(__dadd_rn(s.S2, __dmul_rn(2.0, cross)), __dmul_rn(s.uu, s.vv));
        L.rows[P.out + k] = s.i;
        L.cols[P.out + k] = s.jb;
        s.k = k + 1;
        const double lhs = __dmul_rn(__dsqrt_rn(s.uu), __dsqrt_rn(s.vv));
        const double rhs = __dmul_rn(L.eps, __dsqrt_rn(s.S2 < 0.0 ? 0.0 : s.S2));
        bool stop = false;
        if (lhs <= rhs) {
            if (s.first < 0) s.first = s.k;
            if (s.k - s.first >= kLook) stop = true;
        } else {
            s.first = -1;
        }
        need_row = 0;
        if (stop) {
            s.done = 1;
        } else if (s.fuse) {
            s.i = s.ib;
            s.par ^= 1;
        } else {
            need_row = 1;
        }
    }
    __syncthreads();
    if (need_row) {
        const int ni = block_first_free(w.ur, P.nI);
        if (threadIdx.x == 0) {
            if (ni == INT_MAX) {
                s.done = 1;
            } else {
                s.i = ni;
                s.fresh = 1;
            }
        }
    }
    if (threadIdx.x == 0) {
        const int kmax = min(P.nI, P.nJ);
        if (!s.done && s.k >= kmax) s.done = 1;
        if (!s.done && s.k >= P.kc) {
            s.done = 1;
            s.status = 1;
        }
        s.ok = 0;
        if (s.done) atomicAdd(L.ndone, 1);
        L.st[X] = s;
    }
}

// the kept crosses of finished problems, packed: problem b's U (rank x |I|)
// then V (rank x |J|), cross-major (the (H2+H)* factors, point index fastest)
__global__ void __launch_bounds__(kNT) k_pack_factors(const double* __restrict__ ws,
                                                      const Prob* __restrict__ prob,
                                                      const int32_t* __restrict__ rk,
                                                      const int64_t* __restrict__ foff,
                                                      double* __restrict__ out, int d) {
    const Prob P = prob[blockIdx.x];
    const int r = rk[blockIdx.x];
    if (r <= 0) return;
    const double* U = ws + P.ws + int64_t(d) * (P.nI + P.nJ);
    const double* V = U + int64_t(P.kc) * P.nI;
    double* o = out + foff[blockIdx.x];
    const int64_t nu = int64_t(r) * P.nI, nv = int64_t(r) * P.nJ;
    for (int64_t i = threadIdx.x; i < nu; i += kNT) o[i] = U[i];
    for (int64_t i = threadIdx.x; i < nv; i += kNT) o[nu + i] = V[i];
}

#define PIV_CUDA(call)                                                              \
    do {                                                                            \
        const cudaError_t e_ = (call);                                              \
        if (e_ != cudaSuccess) return std::string("CUDA: ") + cudaGetErrorString(e_); \
    } while (0)

}  // namespace

struct PivotDevice {
    double* x = nullptr;
    int d = 0;
    int64_t N = 0;
    cudaStream_t stream = nullptr;
};

PivotDevice* pivot_device_open(const Tree& t, std::string& err) {
    PivotDevice* p = new PivotDevice();
    p->d = t.d;
    p->N = t.N;
    cudaError_t e = cudaStreamCreateWithFlags(&p->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&p->x, sizeof(double) * size_t(t.N) * t.d);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(p->x, t.x.data(), sizeof(double) * size_t(t.N) * t.d,
                            cudaMemcpyHostToDevice, p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) {
        err = std::string("CUDA: ") + cudaGetErrorString(e);
        pivot_device_close(p);
        return nullptr;
    }
    return p;
}

void pivot_device_close(PivotDevice* p) {
    if (!p) return;
    if (p->x) cudaFree(p->x);
    if (p->stream) cudaStreamDestroy(p->stream);
    delete p;
}

namespace {

// Runs the problems `ids` (all with capacity kc_of[X]) to completion on the
// device; fills rank / rows / cols of the finished ones and status 1 for those
// that ran out of crosses (2: no device memory for the batch).
std::string run_batch(PivotDevice* dev, const KernelSpec& G, double eps, const AcaSets& S,
                      const std::vector<int64_t>& ids, const std::vector<int32_t>& kc_of,
                      std::vector<int32_t>& rank, std::vector<int32_t>& status,
                      std::vector<std::vector<int32_t>>& prow, std::vector<std::vector<int32_t>>& pcol,
                      bool keep, std::vector<std::vector<double>>& fac) {
    const int d = dev->d;
    const int64_t np = int64_t(ids.size());
    std::vector<Prob> probs(np);
    std::vector<int32_t> iidx, jidx, mapJ, mapI;
    std::vector<int64_t> segJ0(np), segI0(np);
    int64_t ws = 0, outn = 0, bound = 0;
    for (int64_t b = 0; b < np; ++b) {
        const int64_t X = ids[b];
        const int64_t nI = S.Iptr[X + 1] - S.Iptr[X], nJ = S.Jptr[X + 1] - S.Jptr[X];
        Prob& p = probs[b];
        p.i0 = int64_t(iidx.size());
        p.j0 = int64_t(jidx.size());
        p.nI = int32_t(nI);
        p.nJ = int32_t(nJ);
        p.kc = kc_of[X];
        p.nsI = int32_t((nI + kSeg - 1) / kSeg);
        p.nsJ = int32_t((nJ + kSeg - 1) / kSeg);
        p.pad = 0;
        p.ws = ws;
        p.out = outn;
        ws += ws_doubles(d, nI, nJ, p.kc, p.nsI, p.nsJ);
        outn += p.kc;
        iidx.insert(iidx.end(), S.Iidx.begin() + S.Iptr[X], S.Iidx.begin() + S.Iptr[X + 1]);
        jidx.insert(jidx.end(), S.Jidx.begin() + S.Jptr[X], S.Jidx.begin() + S.Jptr[X + 1]);
        segJ0[b] = int64_t(mapJ.size());
        for (int g = 0; g < p.nsJ; ++g) mapJ.push_back(int32_t(b));
        segI0[b] = int64_t(mapI.size());
        for (int g = 0; g < p.nsI; ++g) mapI.push_back(int32_t(b));
        bound = std::max(bound, nI + std::min(nI, nJ) + 2);
    }
    const int64_t totJ = int64_t(mapJ.size()), totI = int64_t(mapI.size());
    std::vector<St> st(np);
    for (auto& s : st) {
        s = St();
        s.first = -1;
        s.fresh = 1;
    }
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t b_prob = sizeof(Prob) * np, b_st = sizeof(St) * np, b_i = 4 * iidx.size(),
                 b_j = 4 * jidx.size(), b_out = 4 * size_t(outn), b_mj = 4 * mapJ.size(),
                 b_mi = 4 * mapI.size(), b_s0 = 8 * size_t(np), b_ws = 8 * size_t(ws);
    const size_t total = al(b_prob) + al(b_st) + al(b_i) + al(b_j) + 2 * al(b_out) + al(b_mj) +
                         al(b_mi) + 2 * al(b_s0) + al(4) + b_ws;
    char* buf = nullptr;
    if (cudaMalloc(&buf, total) != cudaSuccess) {
        // no room for this batch now (other work holds the memory): the host
        // solves its problems
        cudaGetLastError();
        for (int64_t X : ids) status[X] = 2;
        return "";
    }
    std::string err;
    auto run = [&]() -> std::string {
        char* q = buf;
        Prob* d_prob = reinterpret_cast<Prob*>(q); q += al(b_prob);
        St* d_st = reinterpret_cast<St*>(q); q += al(b_st);
        int32_t* d_i = reinterpret_cast<int32_t*>(q); q += al(b_i);
        int32_t* d_j = reinterpret_cast<int32_t*>(q); q += al(b_j);
        int32_t* d_rows = reinterpret_cast<int32_t*>(q); q += al(b_out);
        int32_t* d_cols = reinterpret_cast<int32_t*>(q); q += al(b_out);
        int32_t* d_mj = reinterpret_cast<int32_t*>(q); q += al(b_mj);
        int32_t* d_mi = reinterpret_cast<int32_t*>(q); q += al(b_mi);
        int64_t* d_sj = reinterpret_cast<int64_t*>(q); q += al(b_s0);
        int64_t* d_si = reinterpret_cast<int64_t*>(q); q += al(b_s0);
        int32_t* d_nd = reinterpret_cast<int32_t*>(q); q += al(4);
        double* d_ws = reinterpret_cast<double*>(q);
        cudaStream_t sm = dev->stream;
        PIV_CUDA(cudaMemcpyAsync(d_prob, probs.data(), b_prob, cudaMemcpyHostToDevice, sm));
        PIV_CUDA(cudaMemcpyAsync(d_st, st.data(), b_st, cudaMemcpyHostToDevice, sm));
        if (b_i) PIV_CUDA(cudaMemcpyAsync(d_i, iidx.data(), b_i, cudaMemcpyHostToDevice, sm));
        if (b_j) PIV_CUDA(cudaMemcpyAsync(d_j, jidx.data(), b_j, cudaMemcpyHostToDevice, sm));
        PIV_CUDA(cudaMemcpyAsync(d_mj, mapJ.data(), b_mj, cudaMemcpyHostToDevice, sm));
        PIV_CUDA(cudaMemcpyAsync(d_mi, mapI.data(), b_mi, cudaMemcpyHostToDevice, sm));
        PIV_CUDA(cudaMemcpyAsync(d_sj, segJ0.data(), b_s0, cudaMemcpyHostToDevice, sm));
        PIV_CUDA(cudaMemcpyAsync(d_si, segI0.data(), b_s0, cudaMemcpyHostToDevice, sm));
        PIV_CUDA(cudaMemsetAsync(d_nd, 0, 4, sm));
        Lv L;
        L.x = dev->x;
        L.d = d;
        L.kind = G.kind;
        L.c = G.param;
        L.diag = G.diag();
        L.eps = eps;
        L.Iidx = d_i;
        L.Jidx = d_j;
        L.prob = d_prob;
        L.st = d_st;
        L.ws = d_ws;
        L.rows = d_rows;
        L.cols = d_cols;
        L.mapJ = d_mj;
        L.mapI = d_mi;
        L.segJ0 = d_sj;
        L.segI0 = d_si;
        L.totJ = totJ;
        L.ndone = d_nd;
        const unsigned gJ = unsigned(totJ), gJI = unsigned(totJ + totI), gP = unsigned(np);
        k_init<<<gJI, kNT, 0, sm>>>(L);
        PIV_CUDA(cudaGetLastError());
        int32_t nd = 0;
        int64_t step = 0;
        for (; step < bound; ++step) {
            k_stepA<<<gJ, kNT, 0, sm>>>(L);
            k_stepB<<<gP, kNT, 0, sm>>>(L);
            k_stepC<<<gJI, kNT, 0, sm>>>(L);
            k_stepD<<<gP, kNT, 0, sm>>>(L);
            k_stepE<<<gJI, kNT, 0, sm>>>(L);
            k_stepF<<<gP, kNT, 0, sm>>>(L);
            PIV_CUDA(cudaGetLastError());
            if ((step & 7) == 7) {
                PIV_CUDA(cudaMemcpyAsync(&nd, d_nd, 4, cudaMemcpyDeviceToHost, sm));
                PIV_CUDA(cudaStreamSynchronize(sm));
                if (nd >= np) break;
            }
        }
        std::vector<int32_t> hr(outn), hc(outn);
        PIV_CUDA(cudaMemcpyAsync(st.data(), d_st, b_st, cudaMemcpyDeviceToHost, sm));
        PIV_CUDA(cudaMemcpyAsync(hr.data(), d_rows, b_out, cudaMemcpyDeviceToHost, sm));
        PIV_CUDA(cudaMemcpyAsync(hc.data(), d_cols, b_out, cudaMemcpyDeviceToHost, sm));
        PIV_CUDA(cudaStreamSynchronize(sm));
        for (int64_t b = 0; b < np; ++b) {
            const int64_t X = ids[b];
            const St& s = st[b];
            if (!s.done) return "device pivot search did not finish";
            status[X] = s.status;
            if (s.status) continue;
            const int32_t rk = s.first >= 0 ? s.first : s.k;
            if (rk < 0 || rk > probs[b].kc) return "device pivot search returned a bad rank";
            prow[X].assign(hr.begin() + probs[b].out, hr.begin() + probs[b].out + rk);
            pcol[X].assign(hc.begin() + probs[b].out, hc.begin() + probs[b].out + rk);
            for (int32_t a : prow[X])
                if (a < 0 || a >= probs[b].nI) return "device pivot search returned a bad row";
            for (int32_t a : pcol[X])
                if (a < 0 || a >= probs[b].nJ) return "device pivot search returned a bad column";
            rank[X] = rk;
        }
        if (keep) {
            std::vector<int64_t> foff(np + 1, 0);
            std::vector<int32_t> rks(np, 0);
            for (int64_t b = 0; b < np; ++b) {
                rks[b] = status[ids[b]] ? 0 : rank[ids[b]];
                foff[b + 1] = foff[b] + int64_t(rks[b]) * (probs[b].nI + probs[b].nJ);
            }
            if (foff[np] > 0) {
                char* fb = nullptr;
                const size_t b_f = 8 * size_t(foff[np]);
                PIV_CUDA(cudaMalloc(&fb, al(b_f) + al(8 * size_t(np + 1)) + al(4 * size_t(np))));
                double* d_f = reinterpret_cast<double*>(fb);
                int64_t* d_fo = reinterpret_cast<int64_t*>(fb + al(b_f));
                int32_t* d_rk = reinterpret_cast<int32_t*>(fb + al(b_f) + al(8 * size_t(np + 1)));
                std::vector<double> hf(foff[np]);
                auto pack = [&]() -> std::string {
                    PIV_CUDA(cudaMemcpyAsync(d_fo, foff.data(), 8 * size_t(np + 1), cudaMemcpyHostToDevice, sm));
                    PIV_CUDA(cudaMemcpyAsync(d_rk, rks.data(), 4 * size_t(np), cudaMemcpyHostToDevice, sm));
                    k_pack_factors<<<unsigned(np), kNT, 0, sm>>>(d_ws, d_prob, d_rk, d_fo, d_f, d);
                    PIV_CUDA(cudaGetLastError());
                    PIV_CUDA(cudaMemcpyAsync(hf.data(), d_f, b_f, cudaMemcpyDeviceToHost, sm));
                    PIV_CUDA(cudaStreamSynchronize(sm));
                    return "";
                };
                const std::string e = pack();
                cudaFree(fb);
                if (!e.empty()) return e;
                for (int64_t b = 0; b < np; ++b)
                    if (rks[b] > 0) fac[ids[b]].assign(hf.begin() + foff[b], hf.begin() + foff[b + 1]);
            }
        }
        return "";
    };
    err = run();
    cudaFree(buf);
    return err;
}

}  // namespace

std::string pivot_device_level(PivotDevice* dev, const KernelSpec& G, double eps, const AcaSets& S,
                               AcaPivots& out, bool keep) {
    const int64_t n = int64_t(S.Iptr.size()) - 1;
    out.ptr.assign(n + 1, 0);
    out.rows.clear();
    out.cols.clear();
    out.redo.assign(n, 0);
    out.factors.assign(keep ? n : 0, {});
    if (n <= 0) return "";
    // one search at a time per process: each sizes its workspace from the
    // free device memory
    static std::mutex one_at_a_time;
    std::lock_guard<std::mutex> lock(one_at_a_time);
    const int d = dev->d;
    std::vector<int32_t> rank(n, 0), status(n, 0), kc_of(n, 0);
    std::vector<std::vector<int32_t>> prow(n), pcol(n);
    auto nI_of = [&](int64_t X) { return S.Iptr[X + 1] - S.Iptr[X]; };
    auto nJ_of = [&](int64_t X) { return S.Jptr[X + 1] - S.Jptr[X]; };
    auto bytes = [&](int64_t X, int64_t kc) {
        const int64_t nI = nI_of(X), nJ = nJ_of(X);
        return 8 * ws_doubles(d, nI, nJ, kc, (nI + kSeg - 1) / kSeg, (nJ + kSeg - 1) / kSeg);
    };
    size_t free_b = 0, total_b = 0;
    PIV_CUDA(cudaMemGetInfo(&free_b, &total_b));
    const int64_t budget = std::max<int64_t>(int64_t(1) << 28, int64_t(free_b) / 10 * 7);
    std::vector<int64_t> todo;
    for (int64_t X = 0; X < n; ++X)
        if (nI_of(X) > 0 && nJ_of(X) > 0) todo.push_back(X);
    // the capacity: the largest of these whose workspaces for the whole level
    // fit the budget (problems that need more run again with 1024)
    static const int64_t kCaps[] = {1024, 768, 512, 384, 256, 192};
    int64_t cap = 192;
    for (int64_t c : kCaps) {
        int64_t sum = 0;
        for (int64_t X : todo) sum += bytes(X, std::min(c, std::min(nI_of(X), nJ_of(X))));
        if (sum <= budget) { cap = c; break; }
    }
    for (int pass = 0; pass < 2 && !todo.empty(); ++pass) {
        const int64_t c = pass == 0 ? cap : kKMax;
        std::vector<int64_t> again;
        size_t at = 0;
        while (at < todo.size()) {
            // one batch: problems in order while their workspaces fit the budget
            std::vector<int64_t> ids;
            int64_t sum = 0;
            while (at < todo.size()) {
                const int64_t X = todo[at];
                const int64_t kc = std::min(c, std::min(nI_of(X), nJ_of(X)));
                const int64_t b = bytes(X, kc);
                if (b > budget) {   // too large for the device workspace: the host solves it
                    out.redo[X] = 1;
                    ++at;
                    continue;
                }
                if (!ids.empty() && sum + b > budget) break;
                kc_of[X] = int32_t(kc);
                ids.push_back(X);
                sum += b;
                ++at;
            }
            if (ids.empty()) continue;
            const std::string err = run_batch(dev, G, eps, S, ids, kc_of, rank, status, prow, pcol,
                                              keep, out.factors);
            if (!err.empty()) return err;
            for (int64_t X : ids)
                if (status[X] == 2) {
                    out.redo[X] = 1;
                } else if (status[X]) {
                    // ran out of crosses: again with the largest capacity, unless
                    // it had that already (the host then solves it)
                    if (pass == 0 && kc_of[X] < std::min<int64_t>(kKMax, std::min(nI_of(X), nJ_of(X))))
                        again.push_back(X);
                    else
                        out.redo[X] = 1;
                }
        }
        todo.swap(again);
    }
    for (int64_t X : todo) out.redo[X] = 1;
    for (int64_t X = 0; X < n; ++X) {
        const bool ok = !out.redo[X] && nI_of(X) > 0 && nJ_of(X) > 0;
        out.ptr[X + 1] = out.ptr[X] + (ok ? rank[X] : 0);
        if (ok) {
            out.rows.insert(out.rows.end(), prow[X].begin(), prow[X].end());
            out.cols.insert(out.cols.end(), pcol[X].begin(), pcol[X].end());
        }
    }
    return "";
}

}  // namespace h2
