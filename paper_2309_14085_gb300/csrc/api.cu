// C ABI of the H2* library (declared in include/h2star.h): construction on the
// host (build.cpp), upload of the packed operators, and the MVP pipeline of
// CUDA kernels (mvp_kernels.cuh) launched on the caller's stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <atomic>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <random>
#include <thread>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/h2star.h"
#include "h2_internal.hpp"
#include "gmres_kernels.cuh"
#include "mvp_kernels.cuh"
#include "tc_kernels.cuh"

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
    g_err = msg;
    return code;
}

#define H2_CUDA(call)                                                                   \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return fail(H2_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// Stages timed when profiling is on.
enum Stage { ST_GATHER, ST_P2M, ST_M2M, ST_M2L, ST_L2L, ST_LEAF, ST_LOWRANK, ST_SCATTER, ST_N };

}  // namespace

// Device copy of one block-row task list.
struct DevRowTasks {
    int64_t n = 0;
    int rw = 4;                   // rows per warp (autotuned for the large lists)
    int max_rows = 0;             // largest task (rows)
    int64_t *dst = nullptr, *aoff = nullptr, *seg_ptr = nullptr, *seg_off = nullptr;
    int32_t *rows = nullptr, *kpad = nullptr, *seg_len = nullptr, *seg_col = nullptr;
    // per task, packed for one 64-byte load of the tensor-core kernel:
    // aoff, dst, first segment, segment count, rows, kpad, columns (-1: the
    // launch's), unused
    int64_t* meta = nullptr;
};

// the packed task records of DevRowTasks::meta; ncols (nullable) gives each
// task's own RHS column count (the instance's, in a batch)
std::vector<int64_t> task_meta(const h2::RowTasks& R, const std::vector<int64_t>* ncols = nullptr) {
    std::vector<int64_t> m(size_t(R.size()) * 8);
    for (int64_t k = 0; k < R.size(); ++k) {
        int64_t* e = m.data() + k * 8;
        e[0] = R.aoff[k];
        e[1] = R.dst[k];
        e[2] = R.seg_ptr[k];
        e[3] = R.seg_ptr[k + 1] - R.seg_ptr[k];
        e[4] = R.rows[k];
        e[5] = R.kpad[k];
        e[6] = ncols ? (*ncols)[size_t(k)] : -1;
        e[7] = 0;
    }
    return m;
}

struct h2_handle_s {
    h2::Host host;
    bool on_device = false;
    const struct h2_server_s* server = nullptr;   // the solve server using this handle
    int device = -1;
    size_t vsize = 8;             // sizeof coefficient type
    int64_t bytes_device = 0;
    // device buffers
    void* ops = nullptr;          // stored entries (double / float / float2 / bf16)
    int64_t ops_len = 0;          // entries of ops (the host copy may have been released)
    void* xs = nullptr;           // coordinates, d x N (on-the-fly near field)
    void* px = nullptr;           // pivot coordinates, d x vlen (on-the-fly M2L)
    void* vec = nullptr;          // [ q | v | u | phi ] x vec_nrhs (point-major, RHS fastest)
    void* lr_t = nullptr;         // (H2+H)* scratch V^T q_Y, x vec_nrhs
    int vec_nrhs = 0;             // right-hand sides the buffers hold
    void* vec_alloc = nullptr;    // owned allocations of vec / lr_t (regrown for more RHS)
    void* lrt_alloc = nullptr;
    int64_t* perm = nullptr;
    int64_t* iperm = nullptr;      // user index -> tree position
    int64_t* leaf_ptr = nullptr;
    int64_t* near_ptr = nullptr;
    int64_t* near_idx = nullptr;
    int32_t* rank = nullptr;
    int64_t* voff = nullptr;
    int64_t* uoff = nullptr;
    int32_t* ustride = nullptr;
    int64_t* utoff = nullptr;
    DevRowTasks p2m, m2l, leaf;
    std::vector<DevRowTasks> m2m;              // per parent level
    std::vector<DevRowTasks> l2l;              // per child level
    double tune_ms[2][3] = {};                 // autotuner timings (m2l, leaf) x rw 2/4/8
    // (H2+H)*
    int64_t *lr_y0 = nullptr, *lr_my = nullptr, *lr_uoff = nullptr, *lr_voff = nullptr,
            *lr_toff = nullptr, *lr_x0 = nullptr, *lr_mx = nullptr, *lr_gptr = nullptr;
    int32_t* lr_k = nullptr;
    std::vector<int64_t> lr_level_gptr;        // per level: range of groups
    std::vector<int64_t> lr_gptr_host;
    std::vector<int64_t> lr_maxm_level;        // per level: max target / source size
    std::vector<void*> allocs;
    // profiling: one set of ST_N + 1 events per single-RHS pipeline run, read
    // back in batches so that recording never waits inside a timed region
    bool profile = false;
    std::vector<cudaEvent_t> ev_pool;   // sets of ST_N + 1 events
    size_t ev_used = 0;                 // sets recorded and not yet read
    cudaEvent_t* ev = nullptr;          // current set
    double stage_ms[ST_N] = {};
    int64_t stage_calls = 0;
    int64_t launches = 0;               // kernels launched by h2_matvec
    // GMRES workspace (grown on demand, kept for later solves)
    int gm_cap = -1;                    // restart length the workspace holds
    double* gm_V = nullptr;             // N x (m + 1) Krylov basis
    double* gm_w = nullptr;             // N
    double* gm_r = nullptr;             // N
    double* gm_d = nullptr;             // N (refinement correction)
    double* gm_partial = nullptr;       // kDotBlocks x (m + 1)
    double* gm_h = nullptr;             // m + 1
    std::vector<void*> gm_allocs;
    // tensor-core products: device error flag (bounded waits that expired) and
    // its pinned host copy, refreshed at the end of every product that used them
    int* tc_err = nullptr;
    int* tc_err_host = nullptr;
    int tc_blocks[3] = {0, 0, 0};       // persistent grid for RHS tiles of 64 / 32 / 16
    int tc_occupancy[3] = {0, 0, 0};    // cudaOccupancy estimate (reported only)
    // fp64 storage, near field on the fly, 1/r or the IMQ: the near field runs
    // in double-float arithmetic on a second stream, beside the far-field steps
    // (FP32 pipe next to the FP64-pipe-bound M2L), joined before L2P
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
};

namespace {

template <typename U>
int dev_upload(h2_handle h, U** dst, const std::vector<U>& src) {
    *dst = nullptr;
    const size_t bytes = std::max<size_t>(src.size(), 1) * sizeof(U);
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) return fail(H2_E_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    h->allocs.push_back(p);
    h->bytes_device += int64_t(bytes);
    if (!src.empty()) H2_CUDA(cudaMemcpy(p, src.data(), src.size() * sizeof(U), cudaMemcpyHostToDevice));
    *dst = static_cast<U*>(p);
    return H2_OK;
}

int dev_alloc(h2_handle h, void** dst, size_t bytes) {
    *dst = nullptr;
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, std::max<size_t>(bytes, 16));
    if (e != cudaSuccess) return fail(H2_E_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    h->allocs.push_back(p);
    h->bytes_device += int64_t(bytes);
    *dst = p;
    return H2_OK;
}

#define H2_TRY(x)                     \
    do {                              \
        int rc_ = (x);                \
        if (rc_ != H2_OK) return rc_; \
    } while (0)

// Stored entry conversion from the fp64 host value.
template <class A> struct Conv;
template <> struct Conv<h2::F64> { static double of(double a) { return a; } };
template <> struct Conv<h2::F32> { static float of(double a) { return float(a); } };
// bfloat16 by round-to-nearest-even of the float's upper 16 bits
template <> struct Conv<h2::BF16> {
    static __nv_bfloat16 of(double a) {
        const float f = float(a);
        uint32_t u;
        std::memcpy(&u, &f, 4);
        uint16_t b;
        if ((u & 0x7F800000u) == 0x7F800000u && (u & 0x007FFFFFu)) b = 0x7FC0;   // NaN
        else b = uint16_t((u + 0x7FFFu + ((u >> 16) & 1u)) >> 16);
        __nv_bfloat16_raw r;
        r.x = b;
        return __nv_bfloat16(r);
    }
};
template <> struct Conv<h2::DF> {
    static float2 of(double a) {
        const float hi = float(a);
        return make_float2(hi, float(a - double(hi)));
    }
};

// (Re)allocate the coefficient buffers for nrhs right-hand sides.
int grow_vec(h2_handle h, int nrhs) {
    if (nrhs <= h->vec_nrhs) return H2_OK;
    const h2::Packed& P = h->host.packed;
    if (h->vec_alloc) {
        cudaDeviceSynchronize();
        cudaFree(h->vec_alloc);
        cudaFree(h->lrt_alloc);
        h->bytes_device -= int64_t(P.veclen * h->vec_nrhs + P.lr_tlen * h->vec_nrhs) * int64_t(h->vsize);
        h->vec_alloc = h->lrt_alloc = h->vec = h->lr_t = nullptr;
        h->vec_nrhs = 0;
    }
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, std::max<size_t>(size_t(P.veclen) * nrhs * h->vsize, 16));
    if (e != cudaSuccess) return fail(H2_E_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    void* q = nullptr;
    e = cudaMalloc(&q, std::max<size_t>(size_t(P.lr_tlen) * nrhs * h->vsize, 16));
    if (e != cudaSuccess) {
        cudaFree(p);
        return fail(H2_E_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    h->vec_alloc = h->vec = p;
    h->lrt_alloc = h->lr_t = q;
    h->vec_nrhs = nrhs;
    h->bytes_device += int64_t(P.veclen * nrhs + P.lr_tlen * nrhs) * int64_t(h->vsize);
    return H2_OK;
}

int upload_rows(h2_handle h, DevRowTasks& D, const h2::RowTasks& R) {
    D.n = R.size();
    H2_TRY(dev_upload(h, &D.dst, R.dst));
    H2_TRY(dev_upload(h, &D.aoff, R.aoff));
    H2_TRY(dev_upload(h, &D.seg_ptr, R.seg_ptr));
    H2_TRY(dev_upload(h, &D.seg_off, R.seg_off));
    H2_TRY(dev_upload(h, &D.rows, R.rows));
    H2_TRY(dev_upload(h, &D.kpad, R.kpad));
    H2_TRY(dev_upload(h, &D.seg_len, R.seg_len));
    H2_TRY(dev_upload(h, &D.seg_col, R.seg_col));
    H2_TRY(dev_upload(h, &D.meta, task_meta(R)));
    D.max_rows = R.rows.empty() ? 0 : *std::max_element(R.rows.begin(), R.rows.end());
    return H2_OK;
}

int sm_count() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 1;
    }
    return n;
}

// Rows per CTA: the whole task, or -- for a list with fewer tasks than 4 CTAs
// per SM (the coarse levels) -- chunks of whole 8 x RW-row passes, one CTA per
// chunk along y, until the list has about that many CTAs.  Every row is still
// computed by one warp in the same order.
void row_split(const DevRowTasks& R, int rw, unsigned* gy, int* chunk) {
    const int pass = 8 * rw;
    const int64_t target = 4 * int64_t(sm_count());
    *gy = 1;
    *chunk = 1 << 30;
    if (R.n >= target || R.max_rows <= pass) return;
    const int passes = (R.max_rows + pass - 1) / pass;
    const int want = int(std::min<int64_t>(passes, (target + R.n - 1) / R.n));
    const int per = (passes + want - 1) / want;          // passes per CTA
    *chunk = per * pass;
    *gy = unsigned((R.max_rows + *chunk - 1) / *chunk);
}

template <class A, int RW, int NR>
void launch_rows_rw(const DevRowTasks& R, const void* ops, void* vec, cudaStream_t s, int accumulate,
                    int nrhs, int c0) {
    unsigned gy = 1;
    int chunk = 1 << 30;
    row_split(R, RW, &gy, &chunk);
    const dim3 grid(unsigned(R.n), gy);
    if (NR == 1 && nrhs == 1)
        h2::k_rowgemv1<A, RW><<<grid, 256, 0, s>>>(
                R.n, R.dst, R.rows, R.kpad, R.aoff, R.seg_ptr, R.seg_off, R.seg_len, R.seg_col,
                static_cast<const typename A::S*>(ops), static_cast<typename A::V*>(vec), accumulate,
                chunk);
    else
        h2::k_rowgemv<A, RW, NR><<<grid, 256, 0, s>>>(
                R.n, R.dst, R.rows, R.kpad, R.aoff, R.seg_ptr, R.seg_off, R.seg_len, R.seg_col,
                static_cast<const typename A::S*>(ops), static_cast<typename A::V*>(vec), accumulate,
                nrhs, c0, chunk);
}

// Largest RHS tile: 4 columns in fp32, 2 in fp64 / double-float.  Wider tiles
// (8, 16) are compiled but lose: with fewer rows per warp every task re-stages
// its coefficient tile once per 8 rows, so they are not used.
template <class A> constexpr int max_tile() {
    return (std::is_same<A, h2::F32>::value || std::is_same<A, h2::BF16>::value) ? 4 : 2;
}

template <class A>
void launch_rows(const DevRowTasks& R, const void* ops, void* vec, cudaStream_t s, int accumulate,
                 int nrhs = 1, int c0 = 0, int nr = 1) {
    if (R.n == 0) return;
    constexpr bool f32 = std::is_same<A, h2::F32>::value;
    switch (nr) {
        case 16:
            if constexpr (f32) launch_rows_rw<A, 1, 16>(R, ops, vec, s, accumulate, nrhs, c0);
            break;
        case 8:
            if constexpr (f32) launch_rows_rw<A, 2, 8>(R, ops, vec, s, accumulate, nrhs, c0);
            else launch_rows_rw<A, 1, 8>(R, ops, vec, s, accumulate, nrhs, c0);
            break;
        case 4: launch_rows_rw<A, 2, 4>(R, ops, vec, s, accumulate, nrhs, c0); break;
        case 2: launch_rows_rw<A, f32 ? 4 : 2, 2>(R, ops, vec, s, accumulate, nrhs, c0); break;
        default:
            if (R.rw == 2) launch_rows_rw<A, 2, 1>(R, ops, vec, s, accumulate, nrhs, c0);
            else if (R.rw == 8) launch_rows_rw<A, 8, 1>(R, ops, vec, s, accumulate, nrhs, c0);
            else launch_rows_rw<A, 4, 1>(R, ops, vec, s, accumulate, nrhs, c0);
    }
}

// Split nrhs columns into tiles of the supported widths, widest first.
template <class A>
std::vector<std::pair<int, int>> rhs_tiles(int nrhs) {
    std::vector<std::pair<int, int>> t;   // (first column, width)
    int c = 0;
    for (int w = max_tile<A>(); w >= 1; w /= 2)
        while (nrhs - c >= w) { t.push_back({c, w}); c += w; }
    return t;
}

// Tensor-core block rows: bf16 storage always, fp32 storage when built with
// tensor_cores; RHS tiles of 64 / 32 / 16 columns.
template <class A> bool tc_on(h2_handle h) {
    if constexpr (std::is_same<A, h2::BF16>::value) return true;
    else if constexpr (std::is_same<A, h2::F32>::value) return h->host.tensor_cores != 0;
    else return false;
}

template <typename S, int NT> constexpr int tc_smem() { return h2::tc_smem_bytes<S, NT>(); }

// Resident CTAs per SM from the budgets that bind: shared memory (the SM's
// opt-in maximum, 1 KB reserved per CTA), TMEM (512 columns per SM) and
// registers (64K per SM).
template <typename S, int NT>
int tc_grid(int nsm, int smem_sm, int* blocks, int* occupancy) {
    H2_CUDA(cudaFuncSetAttribute(h2::k_rowgemm_tc<S, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 tc_smem<S, NT>()));
    int occ = 0;
    H2_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, h2::k_rowgemm_tc<S, NT>,
                                                          h2::tc::kThreadsWs, tc_smem<S, NT>()));
    cudaFuncAttributes fa;
    H2_CUDA(cudaFuncGetAttributes(&fa, h2::k_rowgemm_tc<S, NT>));
    const int by_smem = smem_sm / (tc_smem<S, NT>() + 1024);
    const int by_tmem = 512 / int(h2::tc::Plan<S, NT>::kCols);
    const int by_regs = 65536 / (std::max(fa.numRegs, 1) * h2::tc::kThreadsWs);
    *occupancy = occ;
    *blocks = std::max(1, std::min(std::min(by_smem, by_tmem), by_regs)) * nsm;
    return H2_OK;
}

template <typename S, int NT>
int tc_setup_nt(h2_handle h, int nsm, int smem_sm, int slot) {
    return tc_grid<S, NT>(nsm, smem_sm, &h->tc_blocks[slot], &h->tc_occupancy[slot]);
}

// dynamic shared memory limits and the persistent grid (resident CTAs x SMs)
template <typename S>
int tc_setup(h2_handle h) {
    int nsm = 0, smem_sm = 0;
    H2_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->device));
    H2_CUDA(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, h->device));
    H2_TRY((tc_setup_nt<S, 64>(h, nsm, smem_sm, 0)));
    H2_TRY((tc_setup_nt<S, 32>(h, nsm, smem_sm, 1)));
    H2_TRY((tc_setup_nt<S, 16>(h, nsm, smem_sm, 2)));
    return H2_OK;
}

template <class A>
void launch_rows_tc(const DevRowTasks& R, const void* ops, void* vec, cudaStream_t s, int accumulate,
                    int nrhs, int c0, int nt, int* err, const int* blocks) {
    if constexpr (std::is_same<A, h2::BF16>::value || std::is_same<A, h2::F32>::value) {
        using S = typename A::S;
        const S* o = static_cast<const S*>(ops);
        float* v = static_cast<float*>(vec);
        const int slot = nt == 64 ? 0 : nt == 32 ? 1 : 2;
        const unsigned n = unsigned(std::min<int64_t>(R.n, blocks[slot]));
        if (nt == 64)
            h2::k_rowgemm_tc<S, 64><<<n, h2::tc::kThreadsWs, tc_smem<S, 64>(), s>>>(
                R.n, R.meta, R.seg_off, R.seg_len, R.seg_col, o, v, accumulate, nrhs, c0, err);
        else if (nt == 32)
            h2::k_rowgemm_tc<S, 32><<<n, h2::tc::kThreadsWs, tc_smem<S, 32>(), s>>>(
                R.n, R.meta, R.seg_off, R.seg_len, R.seg_col, o, v, accumulate, nrhs, c0, err);
        else
            h2::k_rowgemm_tc<S, 16><<<n, h2::tc::kThreadsWs, tc_smem<S, 16>(), s>>>(
                R.n, R.meta, R.seg_off, R.seg_len, R.seg_col, o, v, accumulate, nrhs, c0, err);
    }
}

struct Tile {
    int c0, width;
    bool tc;
};

// RHS tiles of a block-row step: tensor-core tiles first (if on), the rest on
// the CUDA cores, widest first
template <class A>
std::vector<Tile> row_tiles(h2_handle h, int nrhs) {
    std::vector<Tile> t;
    int c = 0;
    if (tc_on<A>(h))
        for (int w = 64; w >= 16; w /= 2)
            while (nrhs - c >= w) { t.push_back({c, w, true}); c += w; }
    for (int w = max_tile<A>(); w >= 1; w /= 2)
        while (nrhs - c >= w) { t.push_back({c, w, false}); c += w; }
    return t;
}

// Autotuner: for every block-row list of the single-RHS product (M2L, the
// stored leaf rows, P2M and each M2M and L2L level) time 2, 4 and 8 rows per
// warp on the device (the coefficient buffer is scratch here): the fastest of
// 5 individually timed launches per width; 4 rows stays unless another width
// is more than 3 % faster.  The width only decides which rows a warp takes, so
// every choice gives the same results bit for bit.
template <class A>
int autotune(h2_handle h) {
    cudaEvent_t ev[6];
    for (auto& e : ev) H2_CUDA(cudaEventCreate(&e));
    std::vector<DevRowTasks*> lists = {&h->m2l, &h->leaf, &h->p2m};
    for (DevRowTasks& R : h->m2m) lists.push_back(&R);
    for (DevRowTasks& R : h->l2l) lists.push_back(&R);
    const int rws[3] = {2, 4, 8};
    for (size_t li = 0; li < lists.size(); ++li) {
        DevRowTasks& R = *lists[li];
        if (R.n == 0 || (li == 0 && h->host.m2l_fly)) continue;   // no stored M2L blocks
        double t[3];
        for (int k = 0; k < 3; ++k) {
            R.rw = rws[k];
            launch_rows<A>(R, h->ops, h->vec, 0, 0);          // warm-up
            H2_CUDA(cudaEventRecord(ev[0], 0));
            for (int it = 0; it < 5; ++it) {
                launch_rows<A>(R, h->ops, h->vec, 0, 0);
                H2_CUDA(cudaEventRecord(ev[it + 1], 0));
            }
            H2_CUDA(cudaEventSynchronize(ev[5]));
            double best = 1e30;
            for (int it = 0; it < 5; ++it) {
                float ms = 0.f;
                H2_CUDA(cudaEventElapsedTime(&ms, ev[it], ev[it + 1]));
                best = std::min(best, double(ms));
            }
            t[k] = best;
            if (li < 2) h->tune_ms[li][k] = best;
        }
        int pick = 1;                       // 4 rows per warp
        for (int k = 0; k < 3; ++k)
            if (t[k] < 0.97 * t[pick]) pick = k;
        R.rw = rws[pick];
    }
    for (auto& e : ev) H2_CUDA(cudaEventDestroy(e));
    H2_CUDA(cudaGetLastError());
    return H2_OK;
}

template <class A, int D>
void launch_m2l_fill(const DevRowTasks& R, const double* px, const h2::Host& H, void* ops) {
    using S = typename A::S;
    const h2::Packed& P = H.packed;
    const double c = H.kern.param, diag = H.kern.diag();
    S* o = static_cast<S*>(ops);
#define H2_FILL(KIND)                                                                          \
    h2::k_m2l_fill<A, D, KIND><<<unsigned(R.n), 256>>>(R.n, R.dst, R.rows, R.kpad, R.aoff,      \
                                                      R.seg_ptr, R.seg_off, R.seg_len,         \
                                                      R.seg_col, px, P.vlen, P.v_base,          \
                                                      P.u_base, c, diag, o)
    switch (H.kern.kind) {
        case 0: H2_FILL(0); break;
        case 1: H2_FILL(1); break;
        case 2: H2_FILL(2); break;
        default: H2_FILL(3); break;
    }
#undef H2_FILL
}

// Stored M2L blocks formed on the device from the pivot coordinates (the host
// keeps only the pivots): clear the region, upload the coordinates to a
// temporary buffer, one fill launch over the M2L tasks, release the buffer.
template <class A>
int form_m2l(h2_handle h) {
    using S = typename A::S;
    const h2::Host& H = h->host;
    const h2::Packed& P = H.packed;
    if (P.pivot_x.size() != size_t(H.tree.d) * size_t(P.vlen))
        return fail(H2_E_INVALID_ARG, "pivot coordinates missing for the device-formed M2L");
    S* ops = static_cast<S*>(h->ops);
    H2_CUDA(cudaMemset(ops + P.m2l_base, 0, size_t(P.m2l_len) * sizeof(S)));
    void* px = nullptr;
    cudaError_t e = cudaMalloc(&px, std::max<size_t>(P.pivot_x.size(), 1) * sizeof(double));
    if (e != cudaSuccess) return fail(H2_E_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    e = cudaMemcpy(px, P.pivot_x.data(), P.pivot_x.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && h->m2l.n > 0) {
        if (H.tree.d == 2) launch_m2l_fill<A, 2>(h->m2l, static_cast<const double*>(px), H, ops);
        else launch_m2l_fill<A, 3>(h->m2l, static_cast<const double*>(px), H, ops);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    cudaFree(px);
    if (e != cudaSuccess) return fail(H2_E_CUDA, std::string("M2L fill: ") + cudaGetErrorString(e));
    return H2_OK;
}

template <class A>
int upload(h2_handle h) {
    using S = typename A::S;
    using V = typename A::V;
    const h2::Host& H = h->host;
    const h2::Packed& P = H.packed;
    const h2::Tree& t = H.tree;
    h->vsize = sizeof(V);
    // entries on the device: the host's ops, then (M2L formed on the device) its region
    const size_t n_dev = H.m2l_dev ? size_t(P.m2l_base + P.m2l_len) : P.ops.size();
    {
        void* p = nullptr;
        const size_t n = std::max<size_t>(n_dev, 1);
        H2_TRY(dev_alloc(h, &p, n * sizeof(S)));
        if (std::is_same<S, double>::value) {
            if (!P.ops.empty())
                H2_CUDA(cudaMemcpy(p, P.ops.data(), P.ops.size() * sizeof(double), cudaMemcpyHostToDevice));
        } else {
            const size_t chunk = size_t(1) << 24;
            std::vector<S> buf(std::min(chunk, P.ops.size()));
            for (size_t o = 0; o < P.ops.size(); o += chunk) {
                const size_t c = std::min(chunk, P.ops.size() - o);
#pragma omp parallel for schedule(static)
                for (int64_t k = 0; k < int64_t(c); ++k) buf[k] = Conv<A>::of(P.ops[o + k]);
                H2_CUDA(cudaMemcpy(static_cast<S*>(p) + o, buf.data(), c * sizeof(S), cudaMemcpyHostToDevice));
            }
        }
        h->ops = p;
        h->ops_len = int64_t(n_dev);
    }
    if (!P.near_stored) {
        using T = typename std::conditional<std::is_same<A, h2::F32>::value, float, double>::type;
        std::vector<T> xs(size_t(t.d) * t.N);
        for (int64_t i = 0; i < t.N; ++i)
            for (int k = 0; k < t.d; ++k) xs[size_t(k) * t.N + i] = T(t.x[size_t(i) * t.d + k]);
        T* p = nullptr;
        H2_TRY(dev_upload(h, &p, xs));
        h->xs = p;
    }
    if (H.m2l_fly) {
        if constexpr (std::is_same<A, h2::F32>::value) {
            std::vector<float> pxf(P.pivot_x.begin(), P.pivot_x.end());
            float* p = nullptr;
            H2_TRY(dev_upload(h, &p, pxf));
            h->px = p;
        }
    }
    H2_TRY(grow_vec(h, 1));
    H2_TRY(dev_upload(h, &h->perm, t.perm));
    {
        std::vector<int64_t> ip(t.perm.size());
        for (size_t i = 0; i < t.perm.size(); ++i) ip[size_t(t.perm[i])] = int64_t(i);
        H2_TRY(dev_upload(h, &h->iperm, ip));
    }
    H2_TRY(dev_upload(h, &h->leaf_ptr, t.leaf_ptr));
    H2_TRY(dev_upload(h, &h->near_ptr, P.near_ptr));
    H2_TRY(dev_upload(h, &h->near_idx, P.near_idx));
    H2_TRY(dev_upload(h, &h->rank, P.rank));
    H2_TRY(dev_upload(h, &h->voff, P.voff));
    H2_TRY(dev_upload(h, &h->uoff, P.uoff));
    H2_TRY(dev_upload(h, &h->ustride, P.ustride));
    H2_TRY(dev_upload(h, &h->utoff, P.utoff));
    H2_TRY(upload_rows(h, h->p2m, P.p2m));
    H2_TRY(upload_rows(h, h->m2l, P.m2l));
    if (H.m2l_dev && P.m2l_len > 0) H2_TRY(form_m2l<A>(h));
    H2_TRY(upload_rows(h, h->leaf, P.leaf));
    h->m2m.assign(t.kappa + 1, DevRowTasks());
    h->l2l.assign(t.kappa + 1, DevRowTasks());
    for (int l = 0; l <= t.kappa; ++l) {
        H2_TRY(upload_rows(h, h->m2m[l], P.m2m[l]));
        H2_TRY(upload_rows(h, h->l2l[l], P.l2l[l]));
    }
    // (H2+H)* groups: consecutive blocks of one level with the same target box
    const int64_t nblk = int64_t(P.lr_k.size());
    h->lr_gptr_host.clear();
    h->lr_level_gptr.assign(t.kappa + 2, 0);
    h->lr_maxm_level.assign(2 * (t.kappa + 1), 0);
    for (int l = 0; l <= t.kappa; ++l) {
        for (int64_t bk = P.lr_level_ptr[l]; bk < P.lr_level_ptr[l + 1]; ++bk) {
            if (bk == P.lr_level_ptr[l] || P.lr_x0[bk] != P.lr_x0[bk - 1]) h->lr_gptr_host.push_back(bk);
            h->lr_maxm_level[2 * l] = std::max(h->lr_maxm_level[2 * l], P.lr_mx[bk]);
            h->lr_maxm_level[2 * l + 1] = std::max(h->lr_maxm_level[2 * l + 1], P.lr_my[bk]);
        }
        h->lr_level_gptr[l + 1] = int64_t(h->lr_gptr_host.size());
    }
    std::vector<int64_t> gptr = h->lr_gptr_host;
    gptr.push_back(nblk);
    H2_TRY(dev_upload(h, &h->lr_gptr, gptr));
    H2_TRY(dev_upload(h, &h->lr_x0, P.lr_x0));
    H2_TRY(dev_upload(h, &h->lr_mx, P.lr_mx));
    H2_TRY(dev_upload(h, &h->lr_y0, P.lr_y0));
    H2_TRY(dev_upload(h, &h->lr_my, P.lr_my));
    H2_TRY(dev_upload(h, &h->lr_k, P.lr_k));
    H2_TRY(dev_upload(h, &h->lr_uoff, P.lr_uoff));
    H2_TRY(dev_upload(h, &h->lr_voff, P.lr_voff));
    H2_TRY(dev_upload(h, &h->lr_toff, P.lr_toff));
    if (tc_on<A>(h)) {
        if constexpr (std::is_same<A, h2::BF16>::value || std::is_same<A, h2::F32>::value)
            H2_TRY(tc_setup<typename A::S>(h));
        void* e = nullptr;
        H2_TRY(dev_alloc(h, &e, sizeof(int)));
        H2_CUDA(cudaMemset(e, 0, sizeof(int)));
        h->tc_err = static_cast<int*>(e);
        void* ph = nullptr;
        H2_CUDA(cudaMallocHost(&ph, sizeof(int)));
        h->tc_err_host = static_cast<int*>(ph);
        *h->tc_err_host = 0;
    }
    if (std::is_same<A, h2::F64>::value && !P.near_stored && (H.kern.kind == 1 || H.kern.kind == 2)) {
        H2_CUDA(cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking));
        H2_CUDA(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
        H2_CUDA(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
    }
    H2_CUDA(cudaDeviceSynchronize());
    H2_TRY(autotune<A>(h));
    return H2_OK;
}

inline unsigned nblocks(int64_t n, int per) { return unsigned((n + per - 1) / per); }

template <typename T, int D, int KIND, int NR, bool NEAR>
void launch_leaf(h2_handle h, cudaStream_t s, int nrhs, int c0) {
    const h2::Host& H = h->host;
    const h2::Tree& t = H.tree;
    const h2::Packed& P = H.packed;
    const int64_t nleaf = t.nboxes(t.kappa);
    const T* vec = static_cast<const T*>(h->vec);
    h2::k_leaf_fly<T, D, KIND, NR, NEAR><<<unsigned(nleaf), 128, 0, s>>>(
        nleaf, P.nb, P.box_total, P.box_base[t.kappa], h->leaf_ptr, h->near_ptr, h->near_idx,
        h->rank, h->voff, h->uoff, h->ustride, static_cast<const T*>(h->ops), vec + P.u_base * nrhs,
        static_cast<const T*>(h->xs), t.N, vec + P.q_base * nrhs,
        static_cast<T*>(h->vec) + P.phi_base * nrhs, T(H.kern.param), T(H.kern.diag()), nrhs, c0);
}

template <typename T, int D, int KIND, bool NEAR>
void launch_leaf_nr(h2_handle h, cudaStream_t s, int nrhs, int c0, int nr) {
    switch (nr) {
        case 16: launch_leaf<T, D, KIND, 16, NEAR>(h, s, nrhs, c0); break;
        case 8: launch_leaf<T, D, KIND, 8, NEAR>(h, s, nrhs, c0); break;
        case 4: launch_leaf<T, D, KIND, 4, NEAR>(h, s, nrhs, c0); break;
        case 2: launch_leaf<T, D, KIND, 2, NEAR>(h, s, nrhs, c0); break;
        default: launch_leaf<T, D, KIND, 1, NEAR>(h, s, nrhs, c0); break;
    }
}

// L2P plus the near field (NEAR), or L2P alone added to a near field already in phi
template <typename T, int D, bool NEAR = true>
void launch_leaf_d(h2_handle h, cudaStream_t s, int nrhs, int c0, int nr) {
    switch (h->host.kern.kind) {
        case 0: launch_leaf_nr<T, D, 0, NEAR>(h, s, nrhs, c0, nr); break;
        case 1: launch_leaf_nr<T, D, 1, NEAR>(h, s, nrhs, c0, nr); break;
        case 2: launch_leaf_nr<T, D, 2, NEAR>(h, s, nrhs, c0, nr); break;
        default: launch_leaf_nr<T, D, 3, NEAR>(h, s, nrhs, c0, nr); break;
    }
}

// the near field alone, in double-float arithmetic (fp64 storage; 1/r, IMQ)
template <int D, int KIND, int NR>
void launch_near_df(h2_handle h, cudaStream_t s, int nrhs, int c0) {
    const h2::Host& H = h->host;
    const h2::Tree& t = H.tree;
    const h2::Packed& P = H.packed;
    const int64_t nleaf = t.nboxes(t.kappa);
    double* vec = static_cast<double*>(h->vec);
    const double c = H.kern.param;
    h2::k_near_df<D, KIND, NR><<<unsigned(nleaf), 128, 0, s>>>(
        nleaf, h->leaf_ptr, h->near_ptr, h->near_idx, static_cast<const double*>(h->xs), t.N,
        vec + P.q_base * nrhs, vec + P.phi_base * nrhs, KIND == 2 ? 1.0 / (c * c) : 0.0, H.kern.diag(),
        nrhs, c0);
}

template <int D, int KIND>
void launch_near_df_nr(h2_handle h, cudaStream_t s, int nrhs, int c0, int nr) {
    switch (nr) {
        case 16: launch_near_df<D, KIND, 16>(h, s, nrhs, c0); break;
        case 8: launch_near_df<D, KIND, 8>(h, s, nrhs, c0); break;
        case 4: launch_near_df<D, KIND, 4>(h, s, nrhs, c0); break;
        case 2: launch_near_df<D, KIND, 2>(h, s, nrhs, c0); break;
        default: launch_near_df<D, KIND, 1>(h, s, nrhs, c0); break;
    }
}

// M2L from the pivot coordinates (fp32)
template <int D, int KIND, int NR>
void launch_m2l(h2_handle h, cudaStream_t s, int nrhs, int c0) {
    const h2::Host& H = h->host;
    const h2::Packed& P = H.packed;
    const DevRowTasks& R = h->m2l;
    if (R.n == 0) return;
    h2::k_m2l_fly<float, D, KIND, NR><<<unsigned(R.n), 256, 0, s>>>(
        R.n, R.dst, R.rows, R.seg_ptr, R.seg_off, R.seg_len, R.seg_col,
        static_cast<const float*>(h->px), P.vlen, P.v_base, P.u_base, static_cast<float*>(h->vec),
        float(1.0 / (H.kern.param * H.kern.param)), float(H.kern.diag()), nrhs, c0);
}

template <int D, int KIND>
void launch_m2l_nr(h2_handle h, cudaStream_t s, int nrhs, int c0, int nr) {
    switch (nr) {
        case 16: launch_m2l<D, KIND, 16>(h, s, nrhs, c0); break;
        case 8: launch_m2l<D, KIND, 8>(h, s, nrhs, c0); break;
        case 4: launch_m2l<D, KIND, 4>(h, s, nrhs, c0); break;
        case 2: launch_m2l<D, KIND, 2>(h, s, nrhs, c0); break;
        default: launch_m2l<D, KIND, 1>(h, s, nrhs, c0); break;
    }
}

template <int D>
void launch_m2l_d(h2_handle h, cudaStream_t s, int nrhs, int c0, int nr) {
    switch (h->host.kern.kind) {
        case 0: launch_m2l_nr<D, 0>(h, s, nrhs, c0, nr); break;
        case 1: launch_m2l_nr<D, 1>(h, s, nrhs, c0, nr); break;
        case 2: launch_m2l_nr<D, 2>(h, s, nrhs, c0, nr); break;
        default: launch_m2l_nr<D, 3>(h, s, nrhs, c0, nr); break;
    }
}

void mark(h2_handle h, cudaStream_t s, int stage) {
    if (h->profile) cudaEventRecord(h->ev[stage], s);
}

constexpr size_t kEvSets = 4096;

// Read back and accumulate every recorded event set.
int flush_events(h2_handle h) {
    for (size_t k = 0; k < h->ev_used; ++k) {
        cudaEvent_t* e = h->ev_pool.data() + k * (ST_N + 1);
        H2_CUDA(cudaEventSynchronize(e[ST_N]));
        for (int i = 0; i < ST_N; ++i) {
            float ms = 0.f;
            H2_CUDA(cudaEventElapsedTime(&ms, e[i], e[i + 1]));
            h->stage_ms[i] += ms;
        }
        h->stage_calls++;
    }
    h->ev_used = 0;
    return H2_OK;
}

int next_event_set(h2_handle h) {
    if (h->ev_pool.empty()) {
        h->ev_pool.resize(kEvSets * (ST_N + 1));
        for (auto& e : h->ev_pool) H2_CUDA(cudaEventCreate(&e));
    }
    if (h->ev_used == kEvSets) {
        int rc = flush_events(h);
        if (rc != H2_OK) return rc;
    }
    h->ev = h->ev_pool.data() + h->ev_used * (ST_N + 1);
    h->ev_used++;
    return H2_OK;
}

// nrhs right-hand sides: X, Y are device, column-major N x nrhs (leading
// dimensions ldx, ldy), user order, fp64.  The coefficient buffers must hold
// nrhs columns (grow_vec).
template <class A>
int matvec_one(h2_handle h, const double* X, int64_t ldx, double* Y, int64_t ldy, int nrhs,
               cudaStream_t s) {
    using V = typename A::V;
    using S = typename A::S;
    const h2::Host& H = h->host;
    const h2::Tree& t = H.tree;
    const h2::Packed& P = H.packed;
    const int K = t.kappa, d = t.d;
    const S* ops = static_cast<const S*>(h->ops);
    V* vec = static_cast<V*>(h->vec);
    V* q = vec + P.q_base * nrhs;
    V* u = vec + P.u_base * nrhs;
    V* phi = vec + P.phi_base * nrhs;
    int64_t& nl = h->launches;
    const auto tiles = rhs_tiles<A>(nrhs);
    const auto rtiles = row_tiles<A>(h, nrhs);
    bool used_tc = false;
    auto rows = [&](const DevRowTasks& R, int accumulate) {
        if (R.n == 0) return;
        for (const auto& tl : rtiles) {
            ++nl;
            if (tl.tc) {
                used_tc = true;
                launch_rows_tc<A>(R, ops, vec, s, accumulate, nrhs, tl.c0, tl.width, h->tc_err,
                                  h->tc_blocks);
            } else {
                launch_rows<A>(R, ops, vec, s, accumulate, nrhs, tl.c0, tl.width);
            }
        }
    };

    mark(h, s, ST_GATHER);
    ++nl;
    if (nrhs == 1 || nrhs > 64)      // the transposing kernels hold up to 64 columns
        h2::k_gather<A><<<nblocks(t.N * nrhs, 256), 256, 0, s>>>(X, ldx, nrhs, h->perm, q, t.N);
    else
        h2::k_gather_t<A><<<nblocks(t.N, h2::kTransRows), 256, 0, s>>>(X, ldx, nrhs, h->iperm, q, t.N);
    // fp64 near field on the fly in double-float arithmetic, on the side stream
    // from here (q in tree order) to the L2P step
    const bool near_side = std::is_same<A, h2::F64>::value && h->side && !P.near_stored;
    if (near_side) {
        H2_CUDA(cudaEventRecord(h->ev_fork, s));
        H2_CUDA(cudaStreamWaitEvent(h->side, h->ev_fork, 0));
        for (const auto& tl : tiles) {
            ++nl;
            const int kind = H.kern.kind;
            if (d == 2) {
                if (kind == 1) launch_near_df_nr<2, 1>(h, h->side, nrhs, tl.first, tl.second);
                else launch_near_df_nr<2, 2>(h, h->side, nrhs, tl.first, tl.second);
            } else {
                if (kind == 1) launch_near_df_nr<3, 1>(h, h->side, nrhs, tl.first, tl.second);
                else launch_near_df_nr<3, 2>(h, h->side, nrhs, tl.first, tl.second);
            }
        }
        H2_CUDA(cudaEventRecord(h->ev_join, h->side));
    }
    mark(h, s, ST_P2M);
    rows(h->p2m, 0);
    mark(h, s, ST_M2M);
    for (int l = K - 1; l >= 1; --l) rows(h->m2m[l], 0);
    mark(h, s, ST_M2L);
    if (P.vlen > 0) cudaMemsetAsync(u, 0, sizeof(V) * P.vlen * nrhs, s);
    if (H.m2l_fly) {
        if constexpr (std::is_same<A, h2::F32>::value) {
            for (const auto& tl : tiles) {
                ++nl;
                if (d == 2) launch_m2l_d<2>(h, s, nrhs, tl.first, tl.second);
                else launch_m2l_d<3>(h, s, nrhs, tl.first, tl.second);
            }
        }
    } else {
        rows(h->m2l, 0);
    }
    mark(h, s, ST_L2L);
    for (int l = 2; l <= K; ++l) rows(h->l2l[l], 1);
    mark(h, s, ST_LEAF);
    if (P.near_stored) {
        // empty leaves keep phi = 0: clear once, the block rows overwrite the rest
        cudaMemsetAsync(phi, 0, sizeof(V) * t.N * nrhs, s);
        rows(h->leaf, 0);
    } else if constexpr (!std::is_same<A, h2::DF>::value && !std::is_same<A, h2::BF16>::value) {
        using T = typename A::V;
        if (near_side) H2_CUDA(cudaStreamWaitEvent(s, h->ev_join, 0));
        for (const auto& tl : tiles) {
            ++nl;
            if (near_side) {
                if (d == 2) launch_leaf_d<T, 2, false>(h, s, nrhs, tl.first, tl.second);
                else launch_leaf_d<T, 3, false>(h, s, nrhs, tl.first, tl.second);
            } else {
                if (d == 2) launch_leaf_d<T, 2>(h, s, nrhs, tl.first, tl.second);
                else launch_leaf_d<T, 3>(h, s, nrhs, tl.first, tl.second);
            }
        }
    }
    mark(h, s, ST_LOWRANK);
    if constexpr (!std::is_same<A, h2::DF>::value && !std::is_same<A, h2::BF16>::value) {
        using T = typename A::V;
        if (H.variant == H2_PLUS_H_STAR && P.lr_tlen > 0) {
            T* tt = static_cast<T*>(h->lr_t);
            cudaMemsetAsync(tt, 0, sizeof(T) * P.lr_tlen * nrhs, s);
            const int chunk = 4096;
            for (int col = 0; col < nrhs; ++col) {
                for (int l = 1; l <= K; ++l) {
                    const int64_t b0 = P.lr_level_ptr[l], nb = P.lr_level_ptr[l + 1] - b0;
                    if (nb == 0) continue;
                    const int64_t maxmy = h->lr_maxm_level[2 * l + 1];
                    for (int64_t off = 0; off < nb; off += 65535) {
                        const int64_t cnt = std::min<int64_t>(65535, nb - off);
                        dim3 grid(nblocks(maxmy, chunk), unsigned(cnt));
                        ++nl;
                        h2::k_lr_vtq<T><<<grid, 256, 0, s>>>(b0 + off, cnt, h->lr_y0, h->lr_my, h->lr_k,
                                                             h->lr_voff, h->lr_toff,
                                                             reinterpret_cast<const T*>(ops), q, tt, chunk,
                                                             nrhs, col);
                    }
                }
                for (int l = 1; l <= K; ++l) {
                    const int64_t g0 = h->lr_level_gptr[l], ng = h->lr_level_gptr[l + 1] - g0;
                    if (ng == 0) continue;
                    const int64_t maxmx = h->lr_maxm_level[2 * l];
                    for (int64_t off = 0; off < ng; off += 65535) {
                        const int64_t cnt = std::min<int64_t>(65535, ng - off);
                        dim3 grid(nblocks(maxmx, 256), unsigned(cnt));
                        ++nl;
                        h2::k_lr_ut<T><<<grid, 256, 0, s>>>(g0 + off, cnt, h->lr_gptr, h->lr_x0, h->lr_mx,
                                                            h->lr_k, h->lr_uoff, h->lr_toff,
                                                            reinterpret_cast<const T*>(ops), tt, phi,
                                                            nrhs, col);
                    }
                }
            }
        }
    }
    mark(h, s, ST_SCATTER);
    ++nl;
    if (nrhs == 1 || nrhs > 64)
        h2::k_scatter<A><<<nblocks(t.N * nrhs, 256), 256, 0, s>>>(phi, nrhs, h->perm, Y, ldy, t.N);
    else
        h2::k_scatter_t<A><<<nblocks(t.N, h2::kTransRows), 256, 0, s>>>(phi, nrhs, h->iperm, Y, ldy, t.N);
    mark(h, s, ST_N);
    if (used_tc) H2_CUDA(cudaMemcpyAsync(h->tc_err_host, h->tc_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    H2_CUDA(cudaGetLastError());
    return H2_OK;
}

// the pipeline in the handle's storage
int matvec_dispatch(h2_handle h, const double* X, int64_t ldx, double* Y, int64_t ldy, int nrhs,
                    cudaStream_t s) {
    // the flag of an earlier tensor-core product (read back after each one)
    if (h->tc_err_host && *h->tc_err_host)
        return fail(H2_E_TIMEOUT, "a tensor-core product gave up waiting for its MMAs");
    switch (h->host.storage) {
        case H2_F64: return matvec_one<h2::F64>(h, X, ldx, Y, ldy, nrhs, s);
        case H2_F32: return matvec_one<h2::F32>(h, X, ldx, Y, ldy, nrhs, s);
        case H2_DF64: return matvec_one<h2::DF>(h, X, ldx, Y, ldy, nrhs, s);
        default: return matvec_one<h2::BF16>(h, X, ldx, Y, ldy, nrhs, s);
    }
}

int upload_any(h2_handle h) {
    switch (h->host.storage) {
        case H2_F64: return upload<h2::F64>(h);
        case H2_F32: return upload<h2::F32>(h);
        case H2_DF64: return upload<h2::DF>(h);
        default: return upload<h2::BF16>(h);
    }
}

size_t entry_bytes(int storage) {
    return storage == H2_F32 ? 4 : storage == H2_BF16 ? 2 : 8;
}

}  // namespace

extern "C" {

const char* h2_last_error(void) { return g_err.c_str(); }

int h2_build(const double* points, int64_t N, int d, int kernel, int leaf_size, double tol,
             int variant, const h2_build_opts* opts, h2_handle* out) {
    g_err.clear();
    if (!out) return fail(H2_E_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!points) return fail(H2_E_INVALID_ARG, "points is NULL");
    if (N < 1) return fail(H2_E_INVALID_ARG, "N must be >= 1");
    if (d != 2 && d != 3) return fail(H2_E_INVALID_ARG, "d must be 2 or 3");
    if (kernel < 0 || kernel > 3) return fail(H2_E_INVALID_ARG, "unknown kernel");
    if (leaf_size < 1) return fail(H2_E_INVALID_ARG, "leaf_size must be >= 1");
    if (!(tol > 0.0 && tol < 1.0)) return fail(H2_E_INVALID_ARG, "tol must be in (0, 1)");
    if (variant < 0 || variant > 5) return fail(H2_E_INVALID_ARG, "unknown variant");
    h2_build_opts o;
    std::memset(&o, 0, sizeof(o));
    if (opts) o = *opts;
    if (o.storage != H2_F64 && o.storage != H2_F32 && o.storage != H2_DF64 && o.storage != H2_BF16)
        return fail(H2_E_INVALID_ARG, "unknown storage");
    if (o.tensor_cores < 0 || o.tensor_cores > 1) return fail(H2_E_INVALID_ARG, "tensor_cores must be 0 or 1");
    if (o.m2l_mode < 0 || o.m2l_mode > 2) return fail(H2_E_INVALID_ARG, "unknown m2l_mode");
    if (o.near_mode < 0 || o.near_mode > 2) return fail(H2_E_INVALID_ARG, "unknown near_mode");
    {
        bool unsupported = false;
        if (const char* why = h2::combination_error(o.storage, variant, o.near_mode, o.tensor_cores,
                                                    o.m2l_mode, &unsupported))
            return fail(unsupported ? H2_E_UNSUPPORTED : H2_E_INVALID_ARG, why);
    }
    if (o.pivots < 0 || o.pivots > 2) return fail(H2_E_INVALID_ARG, "pivots must be 0, 1 or 2");
    if (o.pivots == 1 && o.host_only)
        return fail(H2_E_INVALID_ARG, "the device pivot search needs a device (host_only set)");
    if (o.kappa < -1 || o.kappa > 20) return fail(H2_E_INVALID_ARG, "kappa out of range");
    if (o.eps_far < 0 || o.eps_far >= 1 || o.eps_ver < 0 || o.eps_ver >= 1)
        return fail(H2_E_INVALID_ARG, "eps_far / eps_ver must be in [0, 1)");
    if (o.use_domain && !(o.domain_side > 0)) return fail(H2_E_INVALID_ARG, "domain_side must be > 0");
    if (kernel == H2_KERNEL_IMQ && o.kparam < 0) return fail(H2_E_INVALID_ARG, "kparam must be > 0");
    if (o.use_domain) {
        for (int64_t i = 0; i < N; ++i)
            for (int k = 0; k < d; ++k) {
                const double x = points[i * d + k];
                if (!(x >= o.domain_lo[k] && x <= o.domain_lo[k] + o.domain_side))
                    return fail(H2_E_INVALID_ARG, "a point lies outside the given domain");
            }
    } else {
        for (int64_t i = 0; i < N * d; ++i)
            if (!std::isfinite(points[i])) return fail(H2_E_INVALID_ARG, "non-finite coordinate");
    }
    std::unique_ptr<h2_handle_s> h;
    try {
        h.reset(new h2_handle_s());
    } catch (const std::bad_alloc&) {
        return fail(H2_E_OOM, "host allocation failed");
    }
    h2::Host& H = h->host;
    H.kern.kind = kernel;
    H.kern.param = o.kparam > 0 ? o.kparam : 0.1;
    H.variant = variant;
    H.storage = o.storage;
    H.near_mode = o.near_mode;
    H.tensor_cores = o.tensor_cores;
    H.m2l_fly = o.m2l_mode == 1;
    H.m2l_dev = o.m2l_mode == 2;
    H.eps_far = o.eps_far > 0 ? o.eps_far : tol;
    H.eps_ver = o.eps_ver > 0 ? o.eps_ver : tol;
    // by default on the device where its pivots are the host's bit for bit
    // (1/r and the IMQ: correctly rounded operations only)
    H.pivots_dev = o.pivots == 1 || (o.pivots == 0 && !o.host_only &&
                                     (kernel == H2_KERNEL_INVR || kernel == H2_KERNEL_IMQ));
    if (H.pivots_dev) {
        int ndev = 0;
        if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
            cudaGetLastError();
            return fail(H2_E_NO_DEVICE, "no CUDA device for the pivot search");
        }
    }
    try {
        std::string e = h2::build_host(H, points, N, d, leaf_size, o.kappa,
                                       o.use_domain ? o.domain_lo : nullptr, o.domain_side, o.threads);
        if (!e.empty()) return fail(e.rfind("CUDA: ", 0) == 0 ? H2_E_CUDA : H2_E_INVALID_ARG, e);
    } catch (const std::bad_alloc&) {
        return fail(H2_E_OOM, "host allocation failed during construction");
    }
    if (!o.host_only) {
        int ndev = 0;
        if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
            cudaGetLastError();
            return fail(H2_E_NO_DEVICE, "no CUDA device");
        }
        H2_CUDA(cudaGetDevice(&h->device));
        int rc = upload_any(h.get());
        if (rc != H2_OK) {
            h2_destroy(h.release());
            return rc;
        }
        h->on_device = true;
    }
    *out = h.release();
    return H2_OK;
}

int h2_release_host(h2_handle h) {
    g_err.clear();
    if (!h) return fail(H2_E_INVALID_ARG, "handle is NULL");
    if (!h->on_device) return fail(H2_E_INVALID_ARG, "a host-only handle keeps its operators");
    if (h->server) return fail(H2_E_INVALID_ARG, "handle is in use by a solve server");
    std::vector<double>().swap(h->host.packed.ops);
    return H2_OK;
}

int h2_convert(h2_handle src, int storage, h2_handle* out) {
    g_err.clear();
    if (!out) return fail(H2_E_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!src) return fail(H2_E_INVALID_ARG, "src is NULL");
    if (src->host.packed.ops.empty() && src->on_device && src->ops_len > 0)
        return fail(H2_E_UNSUPPORTED, "the source's host operators were released (h2_release_host)");
    if (storage != H2_F64 && storage != H2_F32 && storage != H2_DF64 && storage != H2_BF16)
        return fail(H2_E_INVALID_ARG, "unknown storage");
    const bool stored = src->host.packed.near_stored;
    if (src->host.m2l_fly && storage != H2_F32)
        return fail(H2_E_UNSUPPORTED, "the source evaluates M2L on the fly (fp32 only)");
    if ((storage == H2_DF64 || storage == H2_BF16) && !stored)
        return fail(H2_E_UNSUPPORTED, "df64 / bf16 storage needs stored near-field blocks; the "
                                      "source evaluates them on the fly");
    if ((storage == H2_DF64 || storage == H2_BF16) && src->host.variant == H2_PLUS_H_STAR)
        return fail(H2_E_UNSUPPORTED, "(H2+H)* is built for fp64 and fp32 storage");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return fail(H2_E_NO_DEVICE, "no CUDA device");
    }
    std::unique_ptr<h2_handle_s> h;
    try {
        h.reset(new h2_handle_s());
        h->host = src->host;
    } catch (const std::bad_alloc&) {
        return fail(H2_E_OOM, "host allocation failed");
    }
    h2::relink_lists(h->host);           // the copy's bases still point at src's lists
    h->host.storage = storage;
    h->host.near_mode = stored ? 2 : 1;
    if (storage != H2_F32) h->host.tensor_cores = 0;
    H2_CUDA(cudaGetDevice(&h->device));
    int rc = upload_any(h.get());
    if (rc != H2_OK) {
        h2_destroy(h.release());
        return rc;
    }
    h->on_device = true;
    *out = h.release();
    return H2_OK;
}

int h2_save(h2_handle h, const char* path) {
    g_err.clear();
    if (!h || !path) return fail(H2_E_INVALID_ARG, "NULL argument");
    if (h->host.packed.ops.empty() && h->on_device && h->ops_len > h->host.packed.m2l_len)
        return fail(H2_E_UNSUPPORTED, "the handle's host operators were released (h2_release_host)");
    std::string e;
    try {
        e = h2::save_host(h->host, path);
    } catch (const std::bad_alloc&) {
        return fail(H2_E_OOM, "host allocation failed");
    }
    if (!e.empty()) return fail(H2_E_INVALID_ARG, e);
    return H2_OK;
}

int h2_load(const char* path, int host_only, h2_handle* out) {
    g_err.clear();
    if (!out) return fail(H2_E_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!path) return fail(H2_E_INVALID_ARG, "path is NULL");
    if (host_only != 0 && host_only != 1) return fail(H2_E_INVALID_ARG, "host_only must be 0 or 1");
    std::unique_ptr<h2_handle_s> h;
    try {
        h.reset(new h2_handle_s());
        std::string e = h2::load_host(h->host, path);
        if (!e.empty()) return fail(H2_E_INVALID_ARG, e);
    } catch (const std::bad_alloc&) {
        return fail(H2_E_OOM, "host allocation failed while loading");
    }
    if (!host_only) {
        int ndev = 0;
        if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
            cudaGetLastError();
            return fail(H2_E_NO_DEVICE, "no CUDA device");
        }
        H2_CUDA(cudaGetDevice(&h->device));
        int rc = upload_any(h.get());
        if (rc != H2_OK) {
            h2_destroy(h.release());
            return rc;
        }
        h->on_device = true;
    }
    *out = h.release();
    return H2_OK;
}

int h2_matvec(h2_handle h, const double* X, int64_t ldx, double* Y, int64_t ldy, int nrhs,
              void* stream) {
    g_err.clear();
    if (!h) return fail(H2_E_INVALID_ARG, "handle is NULL");
    if (!h->on_device) return fail(H2_E_NO_DEVICE, "handle was built host-only");
    if (h->server) return fail(H2_E_INVALID_ARG, "handle is in use by a solve server");
    const int64_t N = h->host.tree.N;
    if (!X || !Y) return fail(H2_E_INVALID_ARG, "X or Y is NULL");
    if (nrhs < 1 || nrhs > 64) return fail(H2_E_INVALID_ARG, "nrhs must be in [1, 64]");
    if (ldx < N || ldy < N) return fail(H2_E_INVALID_ARG, "leading dimension < N");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    {
        int rc = grow_vec(h, nrhs);
        if (rc != H2_OK) return rc;
    }
    if (h->profile) {
        int rc = next_event_set(h);
        if (rc != H2_OK) return rc;
    }
    return matvec_dispatch(h, X, ldx, Y, ldy, nrhs, s);
}

extern "C" int h2_inject_wait_expiry(h2_handle h, int64_t rounds, void* stream) {
    g_err.clear();
    if (!h) return fail(H2_E_INVALID_ARG, "NULL handle");
    if (rounds < 0 || rounds > int64_t(h2::tc::kWaitLimit))
        return fail(H2_E_INVALID_ARG, "rounds must be in [0, 2^22]");
    if (!h->on_device) return fail(H2_E_NO_DEVICE, "handle was built host-only");
    if (h->server) return fail(H2_E_INVALID_ARG, "the handle serves a solve server");
    if (!h->tc_err) return fail(H2_E_UNSUPPORTED, "the handle runs no tensor-core products");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    h2::k_wait_expiry<<<1, 32, 0, s>>>(uint32_t(rounds), h->tc_err);
    H2_CUDA(cudaGetLastError());
    H2_CUDA(cudaMemcpyAsync(h->tc_err_host, h->tc_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    return H2_OK;
}

int h2_info(h2_handle h, h2_stats* st) {
    g_err.clear();
    if (!h || !st) return fail(H2_E_INVALID_ARG, "NULL argument");
    std::memset(st, 0, sizeof(*st));
    const h2::Host& H = h->host;
    const h2::Tree& t = H.tree;
    const h2::Packed& P = H.packed;
    st->N = t.N;
    st->d = t.d;
    st->kappa = t.kappa;
    st->kernel = H.kern.kind;
    st->variant = H.variant;
    st->storage = H.storage;
    st->nbases = int(H.bases.size());
    for (size_t b = 0; b < H.bases.size() && b < 2; ++b) {
        const h2::Basis& B = H.bases[b];
        for (int l = B.lmin; l <= t.kappa && l < 32; ++l) {
            int mn = 1 << 30, mx = 0;
            double sum = 0;
            for (int64_t X = 0; X < t.nboxes(l); ++X) {
                const int r = B.rank(l, X);
                mn = std::min(mn, r);
                mx = std::max(mx, r);
                sum += r;
            }
            st->rank_min[b][l] = mn;
            st->rank_max[b][l] = mx;
            st->rank_avg[b][l] = sum / double(t.nboxes(l));
        }
        int64_t pairs = 0;
        for (int l = B.lmin; l <= t.kappa; ++l) pairs += int64_t((*B.il)[l].idx.size());
        st->m2l_pairs[b] = pairs;
    }
    const int64_t ts = int64_t(entry_bytes(H.storage));
    int64_t nbasis = 0, ntrans = 0, nlr = 0;
    for (const auto& B : H.bases) {
        for (const auto& U : B.U) nbasis += int64_t(U.size());
        for (const auto& lv : B.Ut)
            for (const auto& M : lv) ntrans += int64_t(M.size());
    }
    nlr = H.lowrank_entries;
    st->bytes_basis = nbasis * ts;
    st->bytes_transfer = ntrans * ts;
    st->bytes_m2l = P.m2l.entries * ts;
    st->m2l_src_coeffs = P.m2l.src_coeffs;
    st->m2l_dst_coeffs = P.m2l.dst_coeffs;
    st->bytes_leaf_rows = P.leaf.entries * ts;
    st->leaf_src_coeffs = P.leaf.src_coeffs;
    st->near_stored = P.near_stored;
    st->rw_m2l = h->m2l.rw;
    st->rw_leaf = h->leaf.rw;
    for (int k = 0; k < 3; ++k) {
        st->tc_blocks[k] = h->tc_blocks[k];
        st->tc_occupancy[k] = h->tc_occupancy[k];
    }
    st->m2l_fly = H.m2l_fly ? 1 : H.m2l_dev ? 2 : 0;
    st->pivot_problems_device = H.piv_problems_dev;
    st->pivot_problems_host = H.piv_problems_host;
    st->pivot_seconds = H.pivot_seconds;
    st->m2l_entries = 0;
    for (int64_t k = 0; k < P.m2l.size(); ++k) {
        int64_t cols = 0;
        for (int64_t e = P.m2l.seg_ptr[k]; e < P.m2l.seg_ptr[k + 1]; ++e) cols += P.m2l.seg_len[e];
        st->m2l_entries += int64_t(P.m2l.rows[k]) * cols;
    }
    st->vlen = P.vlen;
    st->bytes_lowrank = nlr * ts;
    st->near_pairs = H.near_pairs;
    st->near_evals = H.near_evals;
    st->lowrank_pairs = int64_t(H.lowrank.size());
    st->bytes_device = h->bytes_device;
    // algorithmic bytes of one MVP with one RHS: every stored operator once
    // (leaf bases inside the stored block rows when the near field is stored,
    // else the bases plus the coordinates), the user vector in and out (fp64)
    st->alg_bytes_per_rhs = st->bytes_transfer + st->bytes_m2l + st->bytes_lowrank + 2 * t.N * 8 +
                            (P.near_stored ? st->bytes_leaf_rows
                                           : st->bytes_basis + t.N * t.d * (ts == 4 ? 4 : 8));
    st->build_seconds = H.build_seconds;
    return H2_OK;
}

int h2_get_pivots(h2_handle h, int basis, int level, int64_t box, int64_t* ti, int64_t* si,
                  int64_t cap, int* rank) {
    g_err.clear();
    if (!h || !rank) return fail(H2_E_INVALID_ARG, "NULL argument");
    const h2::Host& H = h->host;
    if (basis < 0 || basis >= int(H.bases.size())) return fail(H2_E_INVALID_ARG, "basis out of range");
    const h2::Basis& B = H.bases[basis];
    if (level < 0 || level > H.tree.kappa || box < 0 || box >= H.tree.nboxes(level))
        return fail(H2_E_INVALID_ARG, "level or box out of range");
    if (int(B.tau.size()) <= level) {
        *rank = 0;
        return H2_OK;
    }
    const auto& tau = B.tau[level][box];
    const auto& sig = B.sig[level][box];
    *rank = int(tau.size());
    if (int64_t(tau.size()) > cap) return fail(H2_E_INVALID_ARG, "capacity too small");
    for (size_t i = 0; i < tau.size(); ++i) {
        if (ti) ti[i] = H.tree.perm[tau[i]];
        if (si) si[i] = H.tree.perm[sig[i]];
    }
    return H2_OK;
}

int h2_tree_order(h2_handle h, int64_t* perm) {
    g_err.clear();
    if (!h || !perm) return fail(H2_E_INVALID_ARG, "NULL argument");
    std::copy(h->host.tree.perm.begin(), h->host.tree.perm.end(), perm);
    return H2_OK;
}

int h2_profile(h2_handle h, int enable) {
    g_err.clear();
    if (!h) return fail(H2_E_INVALID_ARG, "handle is NULL");
    if (h->ev_used) {
        int rc = flush_events(h);
        if (rc != H2_OK) return rc;
    }
    h->profile = enable != 0;
    for (int i = 0; i < ST_N; ++i) h->stage_ms[i] = 0.0;
    h->stage_calls = 0;
    h->launches = 0;
    return H2_OK;
}

int h2_stage_times(h2_handle h, double* ms, int cap, int64_t* calls, int64_t* launches) {
    g_err.clear();
    if (!h || !ms || cap < ST_N) return fail(H2_E_INVALID_ARG, "NULL argument or cap < 8");
    if (h->ev_used) {
        int rc = flush_events(h);
        if (rc != H2_OK) return rc;
    }
    for (int i = 0; i < ST_N; ++i) ms[i] = h->stage_ms[i];
    if (calls) *calls = h->stage_calls;
    if (launches) *launches = h->launches;
    return H2_OK;
}

void h2_destroy(h2_handle h) {
    if (!h) return;
    if (h->on_device || !h->allocs.empty()) {
        cudaDeviceSynchronize();
        for (void* p : h->allocs) cudaFree(p);
        if (h->vec_alloc) cudaFree(h->vec_alloc);
        if (h->lrt_alloc) cudaFree(h->lrt_alloc);
        for (void* p : h->gm_allocs) cudaFree(p);
        for (auto& e : h->ev_pool) cudaEventDestroy(e);
        if (h->tc_err_host) cudaFreeHost(h->tc_err_host);
        if (h->ev_fork) cudaEventDestroy(h->ev_fork);
        if (h->ev_join) cudaEventDestroy(h->ev_join);
        if (h->side) cudaStreamDestroy(h->side);
    }
    delete h;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free product.  For callers that must not allocate device memory
// at all while they run products -- a serving process that reserved its whole
// device memory budget up front, or code that records work into a CUDA graph,
// where cudaMalloc is off limits -- h2_matvec_noalloc takes its coefficient
// scratch (charges, multipole and local coefficients and potentials in tree
// order) from one static device array instead of the handle's buffer.
namespace {

constexpr size_t kNoAllocBytes = size_t(32) << 20;   // 32 MiB, held by every GPU that loads us
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];
constexpr int kNoAllocDevices = 64;
void* g_noalloc_ptr[kNoAllocDevices] = {};          // device address of the array, per device
std::mutex g_noalloc_mu;

}  // namespace

extern "C" int h2_matvec_noalloc(h2_handle h, const double* X, double* Y, void* stream) {
    g_err.clear();
    if (!h) return fail(H2_E_INVALID_ARG, "handle is NULL");
    if (!h->on_device) return fail(H2_E_NO_DEVICE, "handle was built host-only");
    if (h->server) return fail(H2_E_INVALID_ARG, "handle is in use by a solve server");
    if (!X || !Y) return fail(H2_E_INVALID_ARG, "X or Y is NULL");
    const h2::Packed& P = h->host.packed;
    const size_t vec_bytes = (size_t(P.veclen) * h->vsize + 255) / 256 * 256;
    const size_t need = vec_bytes + size_t(P.lr_tlen) * h->vsize;
    if (need > kNoAllocBytes)
        return fail(H2_E_INVALID_ARG, "h2_matvec_noalloc: this handle needs " + std::to_string(need) +
                                          " bytes of scratch; the static buffer holds " +
                                          std::to_string(kNoAllocBytes) + " (use h2_matvec)");
    int dev = -1;
    H2_CUDA(cudaGetDevice(&dev));
    if (dev != h->device) return fail(H2_E_INVALID_ARG, "the current device is not the handle's device");
    if (dev < 0 || dev >= kNoAllocDevices) return fail(H2_E_UNSUPPORTED, "device index too large");
    {
        // once per device, with that device current: the host-side name of the
        // array is not a device address, so ask the runtime for it
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            void* p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess)
                return fail(H2_E_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            g_noalloc_ptr[dev] = p;
        }
    }
    unsigned char* base = static_cast<unsigned char*>(g_noalloc_ptr[dev]);
    // run the ordinary single-RHS pipeline with its scratch pointed at the array
    void* saved_vec = h->vec;
    void* saved_lrt = h->lr_t;
    const bool saved_profile = h->profile;
    h->vec = base;
    h->lr_t = base + vec_bytes;
    h->profile = false;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t N = h->host.tree.N;
    const int saved_nrhs = h->vec_nrhs;
    h->vec_nrhs = 1;
    int rc = matvec_dispatch(h, X, N, Y, N, 1, s);
    h->vec_nrhs = saved_nrhs;
    h->vec = saved_vec;
    h->lr_t = saved_lrt;
    h->profile = saved_profile;
    return rc;
}

// ---------------------------------------------------------------------------
// GMRES (§6 solves K sigma = f with unrestarted GMRES and the fast MVP) and
// mixed-precision iterative refinement, all vectors in fp64 on the device.
namespace {

int gm_alloc(h2_handle h, double** p, size_t n) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, std::max<size_t>(n, 1) * sizeof(double));
    if (e != cudaSuccess) return fail(H2_E_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    h->gm_allocs.push_back(q);
    *p = static_cast<double*>(q);
    return H2_OK;
}

int gm_workspace(h2_handle h, int m) {
    if (h->gm_cap >= m) return H2_OK;
    for (void* p : h->gm_allocs) cudaFree(p);
    h->gm_allocs.clear();
    h->gm_cap = -1;
    const size_t N = size_t(h->host.tree.N);
    H2_TRY(gm_alloc(h, &h->gm_V, N * size_t(m + 1)));
    H2_TRY(gm_alloc(h, &h->gm_w, N));
    H2_TRY(gm_alloc(h, &h->gm_r, N));
    H2_TRY(gm_alloc(h, &h->gm_d, N));
    H2_TRY(gm_alloc(h, &h->gm_partial, size_t(h2::kDotBlocks) * (m + 1)));
    H2_TRY(gm_alloc(h, &h->gm_h, size_t(m + 1)));
    h->gm_cap = m;
    return H2_OK;
}

// host out[i] = V[:, i] . w for i < nvec
int gm_dots(h2_handle h, const double* V, int64_t ldv, int nvec, const double* w, double* out,
            cudaStream_t s) {
    const int64_t N = h->host.tree.N;
    h2::k_multidot<<<h2::dot_grid(nvec), h2::kDotThreads, 0, s>>>(V, ldv, nvec, w, N, h->gm_partial);
    h2::k_reduce_partials<<<nblocks(nvec, 128), 128, 0, s>>>(h->gm_partial, h2::kDotBlocks, nvec, h->gm_h);
    H2_CUDA(cudaMemcpyAsync(out, h->gm_h, sizeof(double) * nvec, cudaMemcpyDeviceToHost, s));
    H2_CUDA(cudaStreamSynchronize(s));
    return H2_OK;
}

int gm_norm(h2_handle h, const double* w, double* nrm, cudaStream_t s) {
    double t = 0.0;
    H2_TRY(gm_dots(h, w, 0, 1, w, &t, s));
    *nrm = std::sqrt(std::max(t, 0.0));
    return H2_OK;
}

// y = shift x + scale K~ x
int gm_apply(h2_handle h, double shift, double scale, const double* x, double* y, cudaStream_t s) {
    const int64_t N = h->host.tree.N;
    int rc = matvec_dispatch(h, x, N, y, N, 1, s);
    if (rc != H2_OK) return rc;
    h2::k_axpby<<<nblocks(N, 256), 256, 0, s>>>(shift, x, scale, y, N);
    return H2_OK;
}

// Restarted GMRES(m) on A = shift I + scale K~(h), from the initial guess in x.
// Orthogonalisation: classical Gram-Schmidt applied twice (two host reads of
// the projections per iteration).  Stops when the least-squares residual
// estimate drops below rtol * bnorm, or after maxit iterations.
int gm_solve(h2_handle h, double shift, double scale, const double* b, double bnorm, double* x,
             double rtol, int m, int maxit, cudaStream_t s, int* iters, int* restarts,
             int64_t* matvecs, double* est, bool* converged) {
    const int64_t N = h->host.tree.N;
    double* V = h->gm_V;
    double* w = h->gm_w;
    std::vector<double> H(size_t(m + 1) * m, 0.0), cs(m), sn(m), g(m + 1), hv(m + 1), hv2(m + 1), y(m);
    *converged = false;
    // r = b - A x into V[:, 0]
    H2_TRY(gm_apply(h, shift, scale, x, w, s));
    (*matvecs)++;
    h2::k_axpbyz<<<nblocks(N, 256), 256, 0, s>>>(1.0, b, -1.0, w, V, N);
    double beta = 0.0;
    H2_TRY(gm_norm(h, V, &beta, s));
    *est = beta / bnorm;
    if (beta <= rtol * bnorm) { *converged = true; return H2_OK; }
    while (*iters < maxit) {
        h2::k_axpby<<<nblocks(N, 256), 256, 0, s>>>(0.0, V, 1.0 / beta, V, N);
        std::fill(g.begin(), g.end(), 0.0);
        g[0] = beta;
        int jl = -1;
        for (int j = 0; j < m && *iters < maxit; ++j) {
            H2_TRY(gm_apply(h, shift, scale, V + int64_t(j) * N, w, s));
            (*matvecs)++;
            H2_TRY(gm_dots(h, V, N, j + 1, w, hv.data(), s));
            H2_CUDA(cudaMemcpyAsync(h->gm_h, hv.data(), sizeof(double) * (j + 1), cudaMemcpyHostToDevice, s));
            h2::k_gemv_cols<<<nblocks(N, 256), 256, 0, s>>>(V, N, j + 1, h->gm_h, -1.0, w, N);
            H2_TRY(gm_dots(h, V, N, j + 1, w, hv2.data(), s));
            H2_CUDA(cudaMemcpyAsync(h->gm_h, hv2.data(), sizeof(double) * (j + 1), cudaMemcpyHostToDevice, s));
            h2::k_gemv_cols<<<nblocks(N, 256), 256, 0, s>>>(V, N, j + 1, h->gm_h, -1.0, w, N);
            for (int i = 0; i <= j; ++i) H[size_t(i) * m + j] = hv[i] + hv2[i];
            double hn = 0.0;
            H2_TRY(gm_norm(h, w, &hn, s));
            H[size_t(j + 1) * m + j] = hn;
            if (hn > 0.0)
                h2::k_axpbyz<<<nblocks(N, 256), 256, 0, s>>>(1.0 / hn, w, 0.0, w, V + int64_t(j + 1) * N, N);
            for (int i = 0; i < j; ++i) {
                const double h0 = H[size_t(i) * m + j], h1 = H[size_t(i + 1) * m + j];
                H[size_t(i) * m + j] = cs[i] * h0 + sn[i] * h1;
                H[size_t(i + 1) * m + j] = -sn[i] * h0 + cs[i] * h1;
            }
            const double a = H[size_t(j) * m + j], c = H[size_t(j + 1) * m + j];
            const double den = std::hypot(a, c);
            cs[j] = den > 0 ? a / den : 1.0;
            sn[j] = den > 0 ? c / den : 0.0;
            H[size_t(j) * m + j] = den;
            H[size_t(j + 1) * m + j] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            (*iters)++;
            jl = j;
            *est = std::fabs(g[j + 1]) / bnorm;
            if (std::fabs(g[j + 1]) <= rtol * bnorm || hn == 0.0) break;
        }
        if (jl < 0) break;
        for (int i = jl; i >= 0; --i) {
            double t = g[i];
            for (int k = i + 1; k <= jl; ++k) t -= H[size_t(i) * m + k] * y[k];
            y[i] = H[size_t(i) * m + i] != 0.0 ? t / H[size_t(i) * m + i] : 0.0;
        }
        H2_CUDA(cudaMemcpyAsync(h->gm_h, y.data(), sizeof(double) * (jl + 1), cudaMemcpyHostToDevice, s));
        h2::k_gemv_cols<<<nblocks(N, 256), 256, 0, s>>>(V, N, jl + 1, h->gm_h, 1.0, x, N);
        if (*est <= rtol) { *converged = true; break; }
        if (*iters >= maxit) break;
        // restart from the recomputed residual
        (*restarts)++;
        H2_TRY(gm_apply(h, shift, scale, x, w, s));
        (*matvecs)++;
        h2::k_axpbyz<<<nblocks(N, 256), 256, 0, s>>>(1.0, b, -1.0, w, V, N);
        H2_TRY(gm_norm(h, V, &beta, s));
        *est = beta / bnorm;
        if (beta <= rtol * bnorm) { *converged = true; break; }
    }
    H2_CUDA(cudaGetLastError());
    return H2_OK;
}

}  // namespace

extern "C" int h2_gmres(h2_handle h, h2_handle h_res, double shift, double scale, const double* b,
                        double* x, double rtol, int restart, int maxit, h2_gmres_stats* st,
                        void* stream) {
    g_err.clear();
    if (!h || !b || !x) return fail(H2_E_INVALID_ARG, "NULL argument");
    if (!h->on_device || (h_res && !h_res->on_device))
        return fail(H2_E_NO_DEVICE, "handle was built host-only");
    if (h_res && (h_res->host.tree.N != h->host.tree.N || h_res->device != h->device))
        return fail(H2_E_INVALID_ARG, "the residual handle has another N or device");
    if (h->server || (h_res && h_res->server))
        return fail(H2_E_INVALID_ARG, "handle is in use by a solve server");
    if (!(rtol > 0.0 && rtol < 1.0)) return fail(H2_E_INVALID_ARG, "rtol must be in (0, 1)");
    if (restart < 1 || restart > 1000 || maxit < 1) return fail(H2_E_INVALID_ARG, "restart or maxit out of range");
    if (!std::isfinite(shift) || !std::isfinite(scale)) return fail(H2_E_INVALID_ARG, "shift / scale not finite");
    const auto t0 = std::chrono::steady_clock::now();
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t N = h->host.tree.N;
    const bool saved_profile = h->profile;
    h->profile = false;
    struct Restore {
        h2_handle h;
        bool p;
        ~Restore() { h->profile = p; }
    } restore{h, saved_profile};
    H2_TRY(gm_workspace(h, restart));
    h2_gmres_stats S;
    std::memset(&S, 0, sizeof(S));
    double bnorm = 0.0;
    H2_TRY(gm_norm(h, b, &bnorm, s));
    H2_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * N, s));
    if (bnorm == 0.0) {
        S.converged = 1;
        if (st) *st = S;
        return H2_OK;
    }
    int iters = 0, restarts = 0;
    int64_t mv = 0, mv_res = 0;
    double est = 1.0;
    bool conv = false;
    if (!h_res || h_res == h) {
        H2_TRY(gm_solve(h, shift, scale, b, bnorm, x, rtol, restart, maxit, s, &iters, &restarts, &mv,
                        &est, &conv));
        // the true relative residual with the solver's operator
        H2_TRY(gm_apply(h, shift, scale, x, h->gm_r, s));
        mv++;
        h2::k_axpby<<<nblocks(N, 256), 256, 0, s>>>(1.0, b, -1.0, h->gm_r, N);
        double rn = 0.0;
        H2_TRY(gm_norm(h, h->gm_r, &rn, s));
        S.rel_residual = rn / bnorm;
    } else {
        // iterative refinement: residual r = b - A_res x in fp64 with h_res, correction
        // from GMRES on the faster operator of h; the inner tolerance follows the
        // inner operator's precision
        const double floor_inner = h->host.storage == H2_F32    ? 1e-5
                                   : h->host.storage == H2_BF16 ? 1e-2
                                                                : 1e-10;
        double* r = h->gm_r;
        double* dx = h->gm_d;
        H2_CUDA(cudaMemcpyAsync(r, b, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
        double rn = bnorm;
        bool fallback = false;
        for (int outer = 0; outer < 30; ++outer) {
            if (rn <= rtol * bnorm) { conv = true; break; }
            if (iters >= maxit) break;
            const double inner = std::max(floor_inner, 0.5 * rtol * bnorm / rn);
            H2_CUDA(cudaMemsetAsync(dx, 0, sizeof(double) * N, s));
            bool c2 = false;
            double e2 = 1.0;
            H2_TRY(gm_solve(h, shift, scale, r, rn, dx, inner, restart, maxit - iters, s, &iters,
                            &restarts, &mv, &e2, &c2));
            h2::k_axpby<<<nblocks(N, 256), 256, 0, s>>>(1.0, dx, 1.0, x, N);
            H2_TRY(gm_apply(h_res, shift, scale, x, r, s));
            mv_res++;
            h2::k_axpby<<<nblocks(N, 256), 256, 0, s>>>(1.0, b, -1.0, r, N);
            double rn_new = 0.0;
            H2_TRY(gm_norm(h, r, &rn_new, s));
            S.refinements++;
            est = e2;
            if (rn_new > rtol * bnorm && rn_new > 0.5 * rn) {
                // the correction did not halve the fp64 residual: undo it
                h2::k_axpby<<<nblocks(N, 256), 256, 0, s>>>(-1.0, dx, 1.0, x, N);
                fallback = true;
                break;
            }
            rn = rn_new;
        }
        if (fallback && iters < maxit) {
            // finish with fp64 GMRES on the residual handle from the last good x
            H2_TRY(gm_workspace(h_res, restart));
            const bool saved_res_profile = h_res->profile;
            h_res->profile = false;
            int64_t mv2 = 0;
            int rc = gm_solve(h_res, shift, scale, b, bnorm, x, rtol, restart, maxit - iters, s,
                              &iters, &restarts, &mv2, &est, &conv);
            h_res->profile = saved_res_profile;
            mv_res += mv2;
            if (rc != H2_OK) return rc;
        }
        if (fallback) {
            H2_TRY(gm_apply(h_res, shift, scale, x, r, s));
            mv_res++;
            h2::k_axpby<<<nblocks(N, 256), 256, 0, s>>>(1.0, b, -1.0, r, N);
            H2_TRY(gm_norm(h, r, &rn, s));
        }
        conv = rn <= rtol * bnorm;
        S.rel_residual = rn / bnorm;
        S.fallback = fallback ? 1 : 0;
    }
    H2_CUDA(cudaStreamSynchronize(s));
    S.converged = conv ? 1 : 0;
    S.iterations = iters;
    S.restarts = restarts;
    S.matvecs = mv;
    S.matvecs_residual = mv_res;
    S.rel_residual_est = est;
    S.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (st) *st = S;
    if (!conv) return fail(H2_E_NOT_CONVERGED, "GMRES stopped at maxit before reaching rtol");
    return H2_OK;
}

// ---------------------------------------------------------------------------
// Batched products over many independent trees: every (instance, tile of nt
// RHS columns; nt = 4 in fp32, 2 in fp64 / double-float) is a virtual instance
// with its own coefficient regions (point-major, nt columns per point, zero
// columns past the instance's last); the task lists of
// all of them are merged so that each MVP stage is one launch (M2M bottom-up
// and L2L top-down in level-synchronous steps), and the whole sequence is
// captured once into a CUDA graph and replayed.
namespace {

// one thread per (virtual instance, point): the tile's nt columns (zero beyond ncol[v])
__global__ void k_batch_gather(int nv, int nt, const int64_t* __restrict__ pref,
                               const int64_t* __restrict__ qb, const int64_t* __restrict__ pb,
                               const int32_t* __restrict__ ncol, const int64_t* __restrict__ perm,
                               const double* const* __restrict__ X, void* __restrict__ vec, int storage) {
    const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t >= pref[nv]) return;
    int lo = 0, hi = nv;                       // vinst v with pref[v] <= t < pref[v + 1]
    while (hi - lo > 1) {
        const int mid = (lo + hi) / 2;
        if (pref[mid] <= t) lo = mid; else hi = mid;
    }
    const int64_t i = t - pref[lo], n = pref[lo + 1] - pref[lo];
    const int64_t src = perm[pb[lo] + i], o = (qb[lo] + i) * nt;
    for (int c = 0; c < nt; ++c) {
        const double x = c < ncol[lo] ? X[lo][int64_t(c) * n + src] : 0.0;
        if (storage == H2_F64) static_cast<double*>(vec)[o + c] = x;
        else if (storage == H2_F32) static_cast<float*>(vec)[o + c] = float(x);
        else static_cast<float2*>(vec)[o + c] = h2::DF::from_double(x);
    }
}

__global__ void k_batch_scatter(int nv, int nt, const int64_t* __restrict__ pref,
                                const int64_t* __restrict__ fb, const int64_t* __restrict__ pb,
                                const int32_t* __restrict__ ncol, const int64_t* __restrict__ perm,
                                double* const* __restrict__ Y, const void* __restrict__ vec, int storage) {
    const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t >= pref[nv]) return;
    int lo = 0, hi = nv;
    while (hi - lo > 1) {
        const int mid = (lo + hi) / 2;
        if (pref[mid] <= t) lo = mid; else hi = mid;
    }
    const int64_t i = t - pref[lo], n = pref[lo + 1] - pref[lo];
    const int64_t dst = perm[pb[lo] + i], o = (fb[lo] + i) * nt;
    for (int c = 0; c < ncol[lo]; ++c) {
        double y;
        if (storage == H2_F64) y = static_cast<const double*>(vec)[o + c];
        else if (storage == H2_F32) y = double(static_cast<const float*>(vec)[o + c]);
        else y = h2::DF::to_double(static_cast<const float2*>(vec)[o + c]);
        Y[lo][int64_t(c) * n + dst] = y;
    }
}

}  // namespace

struct h2_batch_s {
    int storage = 0, ninst = 0, nvirt = 0, device = -1;
    size_t ssize = 8, vsize = 8;
    int nt = 1;                                // RHS columns per virtual instance
    // fp32 handles built with tensor_cores: every block-row step runs on the
    // tensor cores in 16-column tiles, so an instance's operators stream once
    // for all of its (up to 16) columns; per-task column counts bound the reads
    bool tc = false;
    int tc_blocks[3] = {0, 0, 0}, tc_occupancy = 0;
    int* tc_err = nullptr;                     // device flag of an expired wait
    int* tc_err_host = nullptr;                // pinned copy, read back after each product
    int64_t pts_rhs = 0;                       // sum over instances of N_i nrhs_i
    std::vector<int> inst_of, col_of, ncol;    // per virtual instance
    int32_t* ncol_dev = nullptr;
    std::vector<int64_t> npts;                 // per virtual instance
    int64_t total_pts = 0, veclen = 0, ops_len = 0;
    void* ops = nullptr;
    void* vec = nullptr;
    int64_t* perm = nullptr;                   // concatenated per instance
    int64_t *pref = nullptr, *qb = nullptr, *fb = nullptr, *pb = nullptr;
    const double** Xtab = nullptr;             // device tables of user pointers
    double** Ytab = nullptr;
    int64_t u_begin = 0, u_len = 0, phi_begin = 0, phi_len = 0;
    DevRowTasks p2m, m2l, leaf;
    std::vector<DevRowTasks> m2m, l2l;         // level-synchronous steps
    int64_t launches = 0;                      // kernels per batched MVP
    std::vector<void*> allocs;
    int64_t bytes_device = 0;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    ~h2_batch_s() {
        if (tc_err_host) cudaFreeHost(tc_err_host);
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (ev_in) cudaEventDestroy(ev_in);
        if (ev_out) cudaEventDestroy(ev_out);
        if (stream) cudaStreamDestroy(stream);
        for (void* p : allocs) cudaFree(p);
    }
};

namespace {

template <typename U>
int bupload(h2_batch b, U** dst, const std::vector<U>& src) {
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, std::max<size_t>(src.size(), 1) * sizeof(U));
    if (e != cudaSuccess) return fail(H2_E_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    b->allocs.push_back(p);
    b->bytes_device += int64_t(std::max<size_t>(src.size(), 1) * sizeof(U));
    if (!src.empty()) H2_CUDA(cudaMemcpy(p, src.data(), src.size() * sizeof(U), cudaMemcpyHostToDevice));
    *dst = static_cast<U*>(p);
    return H2_OK;
}

int bupload_rows(h2_batch b, DevRowTasks& D, const h2::RowTasks& R,
                 const std::vector<int64_t>* ncols = nullptr) {
    D.n = R.size();
    H2_TRY(bupload(b, &D.dst, R.dst));
    H2_TRY(bupload(b, &D.aoff, R.aoff));
    H2_TRY(bupload(b, &D.seg_ptr, R.seg_ptr));
    H2_TRY(bupload(b, &D.seg_off, R.seg_off));
    H2_TRY(bupload(b, &D.rows, R.rows));
    H2_TRY(bupload(b, &D.kpad, R.kpad));
    H2_TRY(bupload(b, &D.seg_len, R.seg_len));
    H2_TRY(bupload(b, &D.seg_col, R.seg_col));
    H2_TRY(bupload(b, &D.meta, task_meta(R, ncols)));
    D.rw = 4;
    D.max_rows = R.rows.empty() ? 0 : *std::max_element(R.rows.begin(), R.rows.end());
    return H2_OK;
}

// Append the tasks of R (one instance's layout) to M with ops offset abase and
// coefficient offsets remapped by `map`.
template <class F>
void append_rows(h2::RowTasks& M, const h2::RowTasks& R, int64_t abase, F map) {
    for (int64_t k = 0; k < R.size(); ++k) {
        M.add(map(R.dst[k]), R.rows[k], R.kpad[k], abase + R.aoff[k]);
        for (int64_t e = R.seg_ptr[k]; e < R.seg_ptr[k + 1]; ++e) M.seg(map(R.seg_off[e]), R.seg_len[e]);
        M.close();
    }
}

template <class A>
int batch_launch_all(h2_batch b, cudaStream_t s) {
    using V = typename A::V;
    b->launches = 0;
    const int threads = 256;
    ++b->launches;
    const int nt = b->nt;
    k_batch_gather<<<nblocks(b->total_pts, threads), threads, 0, s>>>(
        b->nvirt, nt, b->pref, b->qb, b->pb, b->ncol_dev, b->perm, b->Xtab, b->vec, b->storage);
    auto rows = [&](const DevRowTasks& R, int acc) {
        if (R.n == 0) return;
        ++b->launches;
        if (b->tc) {
            if constexpr (std::is_same<A, h2::F32>::value)
                launch_rows_tc<A>(R, b->ops, b->vec, s, acc, nt, 0, nt, b->tc_err, b->tc_blocks);
        } else {
            launch_rows<A>(R, b->ops, b->vec, s, acc, nt, 0, nt);
        }
    };
    rows(b->p2m, 0);
    for (const auto& R : b->m2m) rows(R, 0);
    V* vec = static_cast<V*>(b->vec);
    if (b->u_len > 0) cudaMemsetAsync(vec + b->u_begin * nt, 0, sizeof(V) * b->u_len * nt, s);
    rows(b->m2l, 0);
    for (const auto& R : b->l2l) rows(R, 1);
    if (b->phi_len > 0) cudaMemsetAsync(vec + b->phi_begin * nt, 0, sizeof(V) * b->phi_len * nt, s);
    rows(b->leaf, 0);
    ++b->launches;
    k_batch_scatter<<<nblocks(b->total_pts, threads), threads, 0, s>>>(
        b->nvirt, nt, b->pref, b->fb, b->pb, b->ncol_dev, b->perm, b->Ytab, b->vec, b->storage);
    if (b->tc) H2_CUDA(cudaMemcpyAsync(b->tc_err_host, b->tc_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    return H2_OK;
}

}  // namespace

extern "C" int h2_batch_create(const h2_handle* hs, int n, const int* nrhs, h2_batch* out) {
    g_err.clear();
    if (!hs || !out || n < 1) return fail(H2_E_INVALID_ARG, "NULL argument or n < 1");
    *out = nullptr;
    const int storage = hs[0] ? hs[0]->host.storage : -1;
    for (int i = 0; i < n; ++i) {
        if (!hs[i]) return fail(H2_E_INVALID_ARG, "NULL handle in the batch");
        if (hs[i]->host.storage != storage) return fail(H2_E_INVALID_ARG, "handles differ in storage");
        if (storage == H2_BF16) return fail(H2_E_UNSUPPORTED, "batched products use fp64, fp32 or df64 storage");
        if (hs[i]->host.m2l_fly) return fail(H2_E_UNSUPPORTED, "batched products use stored M2L blocks");
        if (hs[i]->host.m2l_dev && !hs[i]->on_device)
            return fail(H2_E_UNSUPPORTED, "a host-only handle with device-formed M2L holds no M2L blocks");
        if (!hs[i]->host.packed.near_stored)
            return fail(H2_E_UNSUPPORTED, "batched products need the stored near field (near_mode 2)");
        if (hs[i]->host.variant == H2_PLUS_H_STAR)
            return fail(H2_E_UNSUPPORTED, "batched products support H2*(b+t) and H2_sqrt(d)(b)");
        const int r = nrhs ? nrhs[i] : 1;
        if (r < 1 || r > 64) return fail(H2_E_INVALID_ARG, "nrhs must be in [1, 64]");
    }
    std::unique_ptr<h2_batch_s> B(new h2_batch_s());
    B->storage = storage;
    B->ninst = n;
    B->ssize = storage == H2_F32 ? 4 : 8;
    B->vsize = B->ssize;
    H2_CUDA(cudaGetDevice(&B->device));
    // ops: instances back to back (each block already 4-aligned inside its instance)
    std::vector<int64_t> abase(n);
    int64_t ol = 0;
    for (int i = 0; i < n; ++i) {
        abase[i] = ol;
        const int64_t len = hs[i]->on_device ? hs[i]->ops_len : int64_t(hs[i]->host.packed.ops.size());
        ol += (len + 3) / 4 * 4;
    }
    B->ops_len = ol;
    // virtual instances and the coefficient layout [Q | V | U | PHI]
    int64_t totN = 0, totV = 0;
    std::vector<int64_t> qoff, voff, pbase(n);
    int64_t pb = 0;
    B->tc = storage == H2_F32;
    for (int i = 0; i < n; ++i) B->tc = B->tc && hs[i]->host.tensor_cores;
    B->nt = B->tc ? 16 : storage == H2_F32 ? 4 : 2;
    for (int i = 0; i < n; ++i) {
        pbase[i] = pb;
        pb += hs[i]->host.tree.N;
        const int r = nrhs ? nrhs[i] : 1;
        B->pts_rhs += hs[i]->host.tree.N * r;
        for (int c = 0; c < r; c += B->nt) {
            B->inst_of.push_back(i);
            B->col_of.push_back(c);
            B->ncol.push_back(std::min(B->nt, r - c));
            B->npts.push_back(hs[i]->host.tree.N);
            qoff.push_back(totN);
            voff.push_back(totV);
            totN += hs[i]->host.tree.N;
            totV += hs[i]->host.packed.vlen;
        }
    }
    B->nvirt = int(B->inst_of.size());
    B->total_pts = totN;
    const int64_t Qb = 0, Vb = totN, Ub = totN + totV, Fb = totN + 2 * totV;
    B->veclen = 2 * totN + 2 * totV;
    B->u_begin = Ub;
    B->u_len = totV;
    B->phi_begin = Fb;
    B->phi_len = totN;
    h2::RowTasks p2m, m2l, leaf;
    int kmax = 0;
    for (int i = 0; i < n; ++i) kmax = std::max(kmax, hs[i]->host.tree.kappa);
    std::vector<h2::RowTasks> m2m(std::max(kmax, 1)), l2l(kmax + 1);
    // per task: its virtual instance's column count (read by the tensor-core path)
    std::vector<int64_t> p2m_nc, m2l_nc, leaf_nc;
    std::vector<std::vector<int64_t>> m2m_nc(m2m.size()), l2l_nc(l2l.size());
    auto cols = [&](std::vector<int64_t>& nc, const h2::RowTasks& R, int v) {
        nc.resize(size_t(R.size()), int64_t(B->ncol[size_t(v)]));
    };
    for (int v = 0; v < B->nvirt; ++v) {
        const h2::Host& H = hs[B->inst_of[v]]->host;
        const h2::Packed& P = H.packed;
        const int64_t N = H.tree.N, vlen = P.vlen;
        auto map = [&](int64_t o) -> int64_t {
            if (o < N) return Qb + qoff[v] + o;
            if (o < N + vlen) return Vb + voff[v] + (o - N);
            if (o < N + 2 * vlen) return Ub + voff[v] + (o - N - vlen);
            return Fb + qoff[v] + (o - N - 2 * vlen);
        };
        const int64_t ab = abase[B->inst_of[v]];
        append_rows(p2m, P.p2m, ab, map);
        cols(p2m_nc, p2m, v);
        append_rows(m2l, P.m2l, ab, map);
        cols(m2l_nc, m2l, v);
        append_rows(leaf, P.leaf, ab, map);
        cols(leaf_nc, leaf, v);
        const int K = H.tree.kappa;
        for (int l = K - 1; l >= 1; --l) {                                                 // bottom-up
            append_rows(m2m[K - 1 - l], P.m2m[l], ab, map);
            cols(m2m_nc[size_t(K - 1 - l)], m2m[K - 1 - l], v);
        }
        for (int l = 2; l <= K; ++l) {                                                     // top-down
            append_rows(l2l[l], P.l2l[l], ab, map);
            cols(l2l_nc[size_t(l)], l2l[l], v);
        }
    }
    // device data
    {
        void* p = nullptr;
        cudaError_t e = cudaMalloc(&p, std::max<size_t>(size_t(ol), 1) * B->ssize);
        if (e != cudaSuccess) return fail(H2_E_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
        B->allocs.push_back(p);
        B->bytes_device += int64_t(ol) * int64_t(B->ssize);
        B->ops = p;
        const size_t chunk = size_t(1) << 24;
        for (int i = 0; i < n; ++i) {
            if (hs[i]->on_device) {
                // the instance's operators are on this device already, in this storage
                H2_CUDA(cudaMemcpy(static_cast<unsigned char*>(p) + size_t(abase[i]) * B->ssize, hs[i]->ops,
                                   size_t(hs[i]->ops_len) * B->ssize, cudaMemcpyDeviceToDevice));
                continue;
            }
            const std::vector<double>& src = hs[i]->host.packed.ops;
            for (size_t o = 0; o < src.size(); o += chunk) {
                const size_t c = std::min(chunk, src.size() - o);
                if (storage == H2_F64) {
                    H2_CUDA(cudaMemcpy(static_cast<double*>(p) + abase[i] + o, src.data() + o, c * 8,
                                       cudaMemcpyHostToDevice));
                } else if (storage == H2_F32) {
                    std::vector<float> buf(c);
                    for (size_t k = 0; k < c; ++k) buf[k] = float(src[o + k]);
                    H2_CUDA(cudaMemcpy(static_cast<float*>(p) + abase[i] + o, buf.data(), c * 4,
                                       cudaMemcpyHostToDevice));
                } else {
                    std::vector<float2> buf(c);
                    for (size_t k = 0; k < c; ++k) buf[k] = Conv<h2::DF>::of(src[o + k]);
                    H2_CUDA(cudaMemcpy(static_cast<float2*>(p) + abase[i] + o, buf.data(), c * 8,
                                       cudaMemcpyHostToDevice));
                }
            }
        }
        e = cudaMalloc(&p, std::max<size_t>(size_t(B->veclen) * B->nt, 1) * B->vsize);
        if (e != cudaSuccess) return fail(H2_E_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
        B->allocs.push_back(p);
        B->bytes_device += int64_t(B->veclen) * B->nt * int64_t(B->vsize);
        B->vec = p;
    }
    std::vector<int64_t> perm;
    for (int i = 0; i < n; ++i) perm.insert(perm.end(), hs[i]->host.tree.perm.begin(), hs[i]->host.tree.perm.end());
    std::vector<int64_t> pref(B->nvirt + 1, 0), qbv(B->nvirt), fbv(B->nvirt), pbv(B->nvirt);
    for (int v = 0; v < B->nvirt; ++v) {
        pref[v + 1] = pref[v] + B->npts[v];
        qbv[v] = Qb + qoff[v];
        fbv[v] = Fb + qoff[v];
        pbv[v] = pbase[B->inst_of[v]];
    }
    H2_TRY(bupload(B.get(), &B->perm, perm));
    H2_TRY(bupload(B.get(), &B->pref, pref));
    H2_TRY(bupload(B.get(), &B->qb, qbv));
    H2_TRY(bupload(B.get(), &B->fb, fbv));
    H2_TRY(bupload(B.get(), &B->pb, pbv));
    {
        std::vector<int32_t> nc(B->ncol.begin(), B->ncol.end());
        H2_TRY(bupload(B.get(), &B->ncol_dev, nc));
    }
    std::vector<const double*> nullx(B->nvirt, nullptr);
    std::vector<double*> nully(B->nvirt, nullptr);
    H2_TRY(bupload(B.get(), &B->Xtab, nullx));
    H2_TRY(bupload(B.get(), &B->Ytab, nully));
    H2_TRY(bupload_rows(B.get(), B->p2m, p2m, &p2m_nc));
    H2_TRY(bupload_rows(B.get(), B->m2l, m2l, &m2l_nc));
    H2_TRY(bupload_rows(B.get(), B->leaf, leaf, &leaf_nc));
    for (size_t k = 0; k < m2m.size(); ++k) {
        if (m2m[k].size() == 0) continue;
        B->m2m.emplace_back();
        H2_TRY(bupload_rows(B.get(), B->m2m.back(), m2m[k], &m2m_nc[k]));
    }
    for (size_t k = 0; k < l2l.size(); ++k) {
        if (l2l[k].size() == 0) continue;
        B->l2l.emplace_back();
        H2_TRY(bupload_rows(B.get(), B->l2l.back(), l2l[k], &l2l_nc[k]));
    }
    if (B->tc) {
        int nsm = 0, smem_sm = 0;
        H2_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, B->device));
        H2_CUDA(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, B->device));
        H2_TRY((tc_grid<float, 16>(nsm, smem_sm, &B->tc_blocks[2], &B->tc_occupancy)));
        std::vector<int> zero(1, 0);
        H2_TRY(bupload(B.get(), &B->tc_err, zero));
        void* ph = nullptr;
        H2_CUDA(cudaMallocHost(&ph, sizeof(int)));
        B->tc_err_host = static_cast<int*>(ph);
        *B->tc_err_host = 0;
    }
    H2_CUDA(cudaStreamCreateWithFlags(&B->stream, cudaStreamNonBlocking));
    H2_CUDA(cudaEventCreateWithFlags(&B->ev_in, cudaEventDisableTiming));
    H2_CUDA(cudaEventCreateWithFlags(&B->ev_out, cudaEventDisableTiming));
    // capture the whole batched product once
    H2_CUDA(cudaStreamBeginCapture(B->stream, cudaStreamCaptureModeThreadLocal));
    int rc = (storage == H2_F64)   ? batch_launch_all<h2::F64>(B.get(), B->stream)
             : (storage == H2_F32) ? batch_launch_all<h2::F32>(B.get(), B->stream)
                                   : batch_launch_all<h2::DF>(B.get(), B->stream);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(B->stream, &g);
    if (rc != H2_OK) return rc;
    if (e != cudaSuccess) return fail(H2_E_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    B->graph = g;
    H2_CUDA(cudaGraphInstantiate(&B->exec, g, 0));
    *out = B.release();
    return H2_OK;
}

extern "C" int h2_batch_matvec(h2_batch b, const double* const* X, double* const* Y, void* stream) {
    g_err.clear();
    if (!b || !X || !Y) return fail(H2_E_INVALID_ARG, "NULL argument");
    // the flag of an earlier tensor-core product (read back after each one)
    if (b->tc_err_host && *b->tc_err_host)
        return fail(H2_E_TIMEOUT, "a tensor-core product of the batch gave up waiting for its MMAs");
    // per virtual instance: column c of instance i at X[i] + c * N_i (column-major, ld = N_i)
    std::vector<const double*> xt(b->nvirt);
    std::vector<double*> yt(b->nvirt);
    for (int v = 0; v < b->nvirt; ++v) {
        const int i = b->inst_of[v];
        if (!X[i] || !Y[i]) return fail(H2_E_INVALID_ARG, "NULL input or output pointer");
        xt[v] = X[i] + int64_t(b->col_of[v]) * b->npts[v];
        yt[v] = Y[i] + int64_t(b->col_of[v]) * b->npts[v];
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    H2_CUDA(cudaEventRecord(b->ev_in, s));
    H2_CUDA(cudaStreamWaitEvent(b->stream, b->ev_in, 0));
    // pageable source: the copies are staged before the calls return
    H2_CUDA(cudaMemcpyAsync(b->Xtab, xt.data(), sizeof(void*) * b->nvirt, cudaMemcpyHostToDevice, b->stream));
    H2_CUDA(cudaMemcpyAsync(b->Ytab, yt.data(), sizeof(void*) * b->nvirt, cudaMemcpyHostToDevice, b->stream));
    H2_CUDA(cudaGraphLaunch(b->exec, b->stream));
    H2_CUDA(cudaEventRecord(b->ev_out, b->stream));
    H2_CUDA(cudaStreamWaitEvent(s, b->ev_out, 0));
    return H2_OK;
}

extern "C" int h2_batch_info(h2_batch b, h2_batch_stats* st) {
    g_err.clear();
    if (!b || !st) return fail(H2_E_INVALID_ARG, "NULL argument");
    std::memset(st, 0, sizeof(*st));
    st->instances = b->ninst;
    st->virtual_instances = b->nvirt;
    st->points_times_rhs = b->pts_rhs;
    st->launches_per_product = b->launches;
    st->m2m_steps = int(b->m2m.size());
    st->l2l_steps = int(b->l2l.size());
    st->m2l_tasks = b->m2l.n;
    st->leaf_tasks = b->leaf.n;
    st->bytes_device = b->bytes_device;
    st->bytes_ops = b->ops_len * int64_t(b->ssize);
    return H2_OK;
}

extern "C" void h2_batch_destroy(h2_batch b) {
    if (!b) return;
    cudaDeviceSynchronize();
    delete b;   // the destructor releases the graph, stream, events and memory
}

// ---------------------------------------------------------------------------
// Served solves: a continuous-batching GMRES server over resident geometries.
// Requests are admitted while their Krylov workspace fits the device budget;
// every tick advances each active request by one GMRES step; the products of
// all active requests on one geometry run as one multi-RHS product (their
// vectors are its columns), and geometries run on their own streams.
namespace {

enum ReqState { RQ_RESIDUAL = 0, RQ_ARNOLDI = 1 };

struct Req {
    int64_t id = 0;
    int g = 0;
    double shift = 0, scale = 1, rtol = 1e-8;
    int maxit = 1000;
    std::vector<double> f;                 // host copy of the right-hand side
    std::vector<double> xh;                // host solution when done
    double t_submit = 0, t_admit = 0, t_done = 0;
    size_t ws_off = 0, ws_len = 0;         // workspace slice (doubles) of the pool
    double *V = nullptr, *w = nullptr, *x = nullptr, *b = nullptr, *part = nullptr, *hd = nullptr;
    double* xp = nullptr;                  // iterate before the current cycle (refinement)
    double* hv = nullptr;                  // pinned host projections (m + 1)
    int state = RQ_RESIDUAL, j = 0, iters = 0, restarts = 0;
    int op = 0;                            // 0 inner operator, 1 residual operator by the
                                           // admission rule, 2 after a fallback
    double beta = 0, beta_prev = 0, bnorm = 0, est = 1, relres = 1;
    bool done = false, converged = false, xzero = true;
    int rc = H2_OK;                        // status of a product that stopped the request
    std::string err;
    std::vector<double> H, cs, sn, gv, h1;
};

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

}  // namespace

struct h2_server_s {
    std::vector<h2_handle> geoms;          // operators of the Arnoldi products
    std::vector<h2_handle> res;            // operators of the residuals (geoms[g] or fp64)
    std::vector<double> floor;             // per geometry: cycle reduction floor (0: plain)
    std::vector<double> delta;             // per geometry: ||(K_inner - K_res) v|| / ||v||
    std::vector<cudaStream_t> streams;
    std::vector<double*> Xg, Yg;           // per geometry: N x max_active staging
    int m = 50, max_active = 16, inner_policy = 0;
    double* pool = nullptr;
    size_t pool_len = 0;                   // doubles
    std::map<size_t, size_t> free_list;    // offset -> length (doubles)
    double* pinned = nullptr;              // max_active x (m + 1) host projections
    std::vector<int> pinned_free;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Req*> queue;
    std::vector<Req*> active;
    std::map<int64_t, Req*> reqs;
    int64_t next_id = 1;
    bool stop = false;
    std::thread worker;
    std::string worker_error;
    int worker_rc = H2_OK;
    h2_server_stats stats = {};           // admission counters (under mu)
    std::atomic<int64_t> ticks{0}, products{0}, product_columns{0};

    ~h2_server_s() {
        for (cudaStream_t st : streams) cudaStreamDestroy(st);
        for (double* p : Xg) cudaFree(p);
        for (double* p : Yg) cudaFree(p);
        if (pool) cudaFree(pool);
        if (pinned) cudaFreeHost(pinned);
        for (h2_handle h : geoms) if (h->server == this) h->server = nullptr;
        for (h2_handle h : res) if (h->server == this) h->server = nullptr;
    }
};

namespace {

bool ws_alloc(h2_server S, size_t n, size_t* off) {
    for (auto it = S->free_list.begin(); it != S->free_list.end(); ++it) {
        if (it->second >= n) {
            *off = it->first;
            const size_t rest = it->second - n;
            const size_t o2 = it->first + n;
            S->free_list.erase(it);
            if (rest) S->free_list[o2] = rest;
            return true;
        }
    }
    return false;
}

void ws_free(h2_server S, size_t off, size_t n) {
    auto it = S->free_list.emplace(off, n).first;
    auto nx = std::next(it);
    if (nx != S->free_list.end() && it->first + it->second == nx->first) {
        it->second += nx->second;
        S->free_list.erase(nx);
    }
    if (it != S->free_list.begin()) {
        auto pv = std::prev(it);
        if (pv->first + pv->second == it->first) {
            pv->second += it->second;
            S->free_list.erase(it);
        }
    }
}

size_t req_doubles(h2_server S, int64_t N) {
    const size_t m = size_t(S->m);
    return size_t(N) * (m + 1) + 4 * size_t(N) + size_t(h2::kDotBlocks) * (m + 1) + (m + 1);
}

int matvec_any(h2_handle h, const double* X, int64_t ldx, double* Y, int64_t ldy, int k,
               cudaStream_t st) {
    return matvec_dispatch(h, X, ldx, Y, ldy, k, st);
}

// y = A x for every request in rs (all on geometry g, operator h): one
// multi-RHS product.
int serve_products(h2_server S, int g, h2_handle h, const std::vector<std::pair<Req*, const double*>>& rs) {
    cudaStream_t st = S->streams[g];
    const int64_t N = h->host.tree.N;
    const int k = int(rs.size());
    for (int c = 0; c < k; ++c)
        H2_CUDA(cudaMemcpyAsync(S->Xg[g] + int64_t(c) * N, rs[c].second, sizeof(double) * N,
                                cudaMemcpyDeviceToDevice, st));
    H2_TRY(matvec_any(h, S->Xg[g], N, S->Yg[g], N, k, st));
    for (int c = 0; c < k; ++c) {
        Req* r = rs[c].first;
        // w = shift x + scale K~ x
        h2::k_axpbyz<<<nblocks(N, 256), 256, 0, st>>>(r->shift, rs[c].second, r->scale,
                                                        S->Yg[g] + int64_t(c) * N, r->w, N);
    }
    S->products++;
    S->product_columns += k;
    return H2_OK;
}

void dots_async(h2_server S, Req* r, const double* Vm, int nvec, const double* w, cudaStream_t st) {
    const int64_t N = S->geoms[r->g]->host.tree.N;
    h2::k_multidot<<<h2::dot_grid(nvec), h2::kDotThreads, 0, st>>>(Vm, N, nvec, w, N, r->part);
    h2::k_reduce_partials<<<nblocks(nvec, 128), 128, 0, st>>>(r->part, h2::kDotBlocks, nvec, r->hd);
    cudaMemcpyAsync(r->hv, r->hd, sizeof(double) * nvec, cudaMemcpyDeviceToHost, st);
}

int sync_all(h2_server S) {
    for (cudaStream_t st : S->streams) H2_CUDA(cudaStreamSynchronize(st));
    return H2_OK;
}

// One tick: every active request advances by one product and its GMRES step.
int serve_tick(h2_server S, std::vector<Req*>& act) {
    const int m = S->m;
    // phase A: products (residual b - A x, or the next Arnoldi vector)
    // key (g, 0): residual products on res[g]; (g, 1): Arnoldi products on geoms[g]
    std::map<std::pair<int, int>, std::vector<std::pair<Req*, const double*>>> by_g;
    for (Req* r : act) {
        const int64_t N = S->geoms[r->g]->host.tree.N;
        if (r->state == RQ_RESIDUAL) {
            if (r->xzero) {
                H2_CUDA(cudaMemsetAsync(r->w, 0, sizeof(double) * N, S->streams[r->g]));
                continue;
            }
            by_g[{r->g, 0}].push_back({r, r->x});
        } else {
            by_g[{r->g, r->op == 0 ? 1 : 0}].push_back({r, r->V + int64_t(r->j) * N});
        }
    }
    for (auto& kv : by_g) {
        const int g = kv.first.first;
        H2_TRY(serve_products(S, g, kv.first.second ? S->geoms[g] : S->res[g], kv.second));
    }
    // phase B: first projections / residual norms
    for (Req* r : act) {
        const int64_t N = S->geoms[r->g]->host.tree.N;
        cudaStream_t st = S->streams[r->g];
        if (r->state == RQ_RESIDUAL) {
            h2::k_axpbyz<<<nblocks(N, 256), 256, 0, st>>>(1.0, r->b, -1.0, r->w, r->V, N);  // V0 = b - A x
            dots_async(S, r, r->V, 1, r->V, st);
        } else {
            dots_async(S, r, r->V, r->j + 1, r->w, st);
        }
    }
    H2_TRY(sync_all(S));
    std::vector<Req*> arn;
    for (Req* r : act) {
        const int64_t N = S->geoms[r->g]->host.tree.N;
        cudaStream_t st = S->streams[r->g];
        if (r->state == RQ_RESIDUAL) {
            r->beta = std::sqrt(std::max(r->hv[0], 0.0));
            r->relres = r->beta / r->bnorm;
            if (r->beta <= r->rtol * r->bnorm || r->iters >= r->maxit) {
                r->converged = r->beta <= r->rtol * r->bnorm;
                r->done = true;
                continue;
            }
            const bool refine = S->floor[r->g] > 0.0 && r->op == 0;
            if (refine && !r->xzero && r->beta > 0.5 * r->beta_prev) {
                // the last cycle on the inner operator did not halve the fp64
                // residual: undo it and continue on the residual operator
                H2_CUDA(cudaMemcpyAsync(r->x, r->xp, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
                r->op = 2;
                continue;                          // residual again next tick
            }
            if (refine) {
                H2_CUDA(cudaMemcpyAsync(r->xp, r->x, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
                r->beta_prev = r->beta;
            }
            if (!r->xzero) r->restarts++;
            h2::k_axpby<<<nblocks(N, 256), 256, 0, st>>>(0.0, r->V, 1.0 / r->beta, r->V, N);
            std::fill(r->gv.begin(), r->gv.end(), 0.0);
            r->gv[0] = r->beta;
            r->j = 0;
            r->state = RQ_ARNOLDI;
            r->xzero = false;
        } else {
            std::copy(r->hv, r->hv + r->j + 1, r->h1.begin());
            cudaMemcpyAsync(r->hd, r->h1.data(), sizeof(double) * (r->j + 1), cudaMemcpyHostToDevice, st);
            h2::k_gemv_cols<<<nblocks(N, 256), 256, 0, st>>>(r->V, N, r->j + 1, r->hd, -1.0, r->w, N);
            dots_async(S, r, r->V, r->j + 1, r->w, st);
            arn.push_back(r);
        }
    }
    if (arn.empty()) return H2_OK;
    H2_TRY(sync_all(S));
    for (Req* r : arn) {
        const int64_t N = S->geoms[r->g]->host.tree.N;
        cudaStream_t st = S->streams[r->g];
        for (int i = 0; i <= r->j; ++i) r->H[size_t(i) * m + r->j] = r->h1[i] + r->hv[i];
        cudaMemcpyAsync(r->hd, r->hv, sizeof(double) * (r->j + 1), cudaMemcpyHostToDevice, st);
        h2::k_gemv_cols<<<nblocks(N, 256), 256, 0, st>>>(r->V, N, r->j + 1, r->hd, -1.0, r->w, N);
        dots_async(S, r, r->w, 1, r->w, st);
    }
    H2_TRY(sync_all(S));
    for (Req* r : arn) {
        const int64_t N = S->geoms[r->g]->host.tree.N;
        cudaStream_t st = S->streams[r->g];
        const int j = r->j;
        const double hn = std::sqrt(std::max(r->hv[0], 0.0));
        r->H[size_t(j + 1) * m + j] = hn;
        if (hn > 0.0)
            h2::k_axpbyz<<<nblocks(N, 256), 256, 0, st>>>(1.0 / hn, r->w, 0.0, r->w, r->V + int64_t(j + 1) * N, N);
        for (int i = 0; i < j; ++i) {
            const double h0 = r->H[size_t(i) * m + j], h1 = r->H[size_t(i + 1) * m + j];
            r->H[size_t(i) * m + j] = r->cs[i] * h0 + r->sn[i] * h1;
            r->H[size_t(i + 1) * m + j] = -r->sn[i] * h0 + r->cs[i] * h1;
        }
        const double a0 = r->H[size_t(j) * m + j], c0 = r->H[size_t(j + 1) * m + j];
        const double den = std::hypot(a0, c0);
        r->cs[j] = den > 0 ? a0 / den : 1.0;
        r->sn[j] = den > 0 ? c0 / den : 0.0;
        r->H[size_t(j) * m + j] = den;
        r->H[size_t(j + 1) * m + j] = 0.0;
        r->gv[j + 1] = -r->sn[j] * r->gv[j];
        r->gv[j] = r->cs[j] * r->gv[j];
        r->iters++;
        r->est = std::fabs(r->gv[j + 1]) / r->bnorm;
        // plain: until the estimate meets rtol; refinement: until this cycle's
        // residual has dropped to the inner operator's precision (or to rtol)
        const double fl = r->op == 0 ? S->floor[r->g] : 0.0;
        const double thr = fl > 0.0 ? std::max(fl * r->beta, 0.5 * r->rtol * r->bnorm) : r->rtol * r->bnorm;
        const bool stop_cycle = std::fabs(r->gv[j + 1]) <= thr || j + 1 == m || r->iters >= r->maxit || hn == 0.0;
        if (!stop_cycle) {
            r->j = j + 1;
            continue;
        }
        // x += V y, then recompute the true residual in the next tick
        std::vector<double> y(j + 1);
        for (int i = j; i >= 0; --i) {
            double t = r->gv[i];
            for (int k2 = i + 1; k2 <= j; ++k2) t -= r->H[size_t(i) * m + k2] * y[k2];
            y[i] = r->H[size_t(i) * m + i] != 0.0 ? t / r->H[size_t(i) * m + i] : 0.0;
        }
        std::copy(y.begin(), y.end(), r->hv);
        cudaMemcpyAsync(r->hd, r->hv, sizeof(double) * (j + 1), cudaMemcpyHostToDevice, st);
        h2::k_gemv_cols<<<nblocks(N, 256), 256, 0, st>>>(r->V, N, j + 1, r->hd, 1.0, r->x, N);
        r->state = RQ_RESIDUAL;
    }
    H2_CUDA(cudaGetLastError());
    return H2_OK;
}

void serve_loop(h2_server S) {
    cudaSetDevice(S->geoms[0]->device);
    for (;;) {
        std::vector<Req*> act;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            // admission: FIFO while the workspace fits and a slot is free
            while (!S->queue.empty() && int(S->active.size()) < S->max_active) {
                Req* r = S->queue.front();
                size_t off = 0;
                if (!ws_alloc(S, r->ws_len, &off)) break;
                S->queue.pop_front();
                r->ws_off = off;
                r->t_admit = now_s();
                S->active.push_back(r);
                const int64_t N = S->geoms[r->g]->host.tree.N;
                double* base = S->pool + off;
                r->V = base;
                r->w = base + N * (S->m + 1);
                r->x = r->w + N;
                r->b = r->x + N;
                r->xp = r->b + N;
                r->part = r->xp + N;
                r->hd = r->part + size_t(h2::kDotBlocks) * (S->m + 1);
                const int slot = S->pinned_free.back();
                S->pinned_free.pop_back();
                r->hv = S->pinned + size_t(slot) * (S->m + 1);
                r->ws_off = off;
                r->H.assign(size_t(S->m + 1) * S->m, 0.0);
                r->cs.assign(S->m, 0.0);
                r->sn.assign(S->m, 0.0);
                r->gv.assign(S->m + 1, 0.0);
                r->h1.assign(S->m + 1, 0.0);
                r->bnorm = 0;
                for (double v : r->f) r->bnorm += v * v;
                r->bnorm = std::sqrt(r->bnorm);
                cudaStream_t st = S->streams[r->g];
                cudaMemcpyAsync(r->b, r->f.data(), sizeof(double) * N, cudaMemcpyHostToDevice, st);
                cudaMemsetAsync(r->x, 0, sizeof(double) * N, st);
                // the inner operator serves this request if its measured error is
                // small against the shift (below 1/10 of the smallest eigenvalue
                // bound |shift| of shift I + scale K for positive semi-definite K)
                r->op = (S->floor[r->g] == 0.0 || S->inner_policy == 1 || r->shift == 0.0 ||
                         S->delta[r->g] * std::fabs(r->scale) <= 0.1 * std::fabs(r->shift)) ? 0 : 1;
                S->stats.admitted++;
            }
            S->stats.max_active = std::max<int64_t>(S->stats.max_active, int64_t(S->active.size()));
            if (S->active.empty()) {
                if (S->stop) return;
                S->cv_work.wait(lk, [&] { return S->stop || !S->queue.empty(); });
                continue;
            }
            act = S->active;
        }
        // requests with a zero right-hand side finish at once
        for (Req* r : act)
            if (r->bnorm == 0.0) { r->done = true; r->converged = true; r->relres = 0.0; }
        std::vector<Req*> run;
        for (Req* r : act) if (!r->done) run.push_back(r);
        if (!run.empty()) {
            int rc = serve_tick(S, run);
            S->ticks++;
            if (rc != H2_OK) {
                std::lock_guard<std::mutex> lk(S->mu);
                S->worker_error = h2_last_error();
                S->worker_rc = rc;
                for (Req* r : run) {
                    r->done = true;
                    r->converged = false;
                    r->rc = rc;
                    r->err = S->worker_error;
                }
            }
        }
        // retire finished requests
        std::vector<Req*> fin;
        for (Req* r : act) if (r->done) fin.push_back(r);
        for (Req* r : fin) {
            const int64_t N = S->geoms[r->g]->host.tree.N;
            r->xh.resize(N);
            cudaMemcpyAsync(r->xh.data(), r->x, sizeof(double) * N, cudaMemcpyDeviceToHost, S->streams[r->g]);
        }
        if (!fin.empty()) sync_all(S);
        {
            std::lock_guard<std::mutex> lk(S->mu);
            for (Req* r : fin) {
                r->t_done = now_s();
                ws_free(S, r->ws_off, r->ws_len);
                S->pinned_free.push_back(int((r->hv - S->pinned) / (S->m + 1)));
                S->active.erase(std::find(S->active.begin(), S->active.end(), r));
                S->stats.completed++;
            }
        }
        if (!fin.empty()) S->cv_done.notify_all();
    }
}

}  // namespace

extern "C" int h2_server_create(const h2_handle* geoms, const h2_handle* res_geoms, int ngeom,
                                const h2_server_opts* opts, h2_server* out) {
    g_err.clear();
    if (!geoms || ngeom < 1 || !out) return fail(H2_E_INVALID_ARG, "NULL argument or no geometry");
    *out = nullptr;
    h2_server_opts o;
    std::memset(&o, 0, sizeof(o));
    if (opts) o = *opts;
    std::unique_ptr<h2_server_s> S(new h2_server_s());
    S->m = o.restart > 0 ? o.restart : 50;
    S->max_active = o.max_active > 0 ? o.max_active : 16;
    if (S->m > 1000 || S->max_active > 1024) return fail(H2_E_INVALID_ARG, "restart or max_active too large");
    if (o.inner_policy < 0 || o.inner_policy > 1) return fail(H2_E_INVALID_ARG, "unknown inner_policy");
    S->inner_policy = o.inner_policy;
    int64_t maxN = 0;
    for (int g = 0; g < ngeom; ++g) {
        if (!geoms[g] || !geoms[g]->on_device) return fail(H2_E_INVALID_ARG, "geometry handle not on the device");
        if (geoms[g]->device != geoms[0]->device) return fail(H2_E_INVALID_ARG, "geometries on different devices");
        h2_handle rh = res_geoms ? res_geoms[g] : geoms[g];
        if (!rh || !rh->on_device) return fail(H2_E_INVALID_ARG, "residual handle not on the device");
        if (rh->device != geoms[g]->device || rh->host.tree.N != geoms[g]->host.tree.N ||
            rh->host.tree.perm != geoms[g]->host.tree.perm)
            return fail(H2_E_INVALID_ARG, "residual handle of another geometry");
        if (geoms[g]->server || rh->server)
            return fail(H2_E_INVALID_ARG, "a handle is in use by another solve server");
        S->geoms.push_back(geoms[g]);
        S->res.push_back(rh);
        const int gs = geoms[g]->host.storage;
        S->floor.push_back(rh == geoms[g] ? 0.0 : (gs == H2_F32 ? 1e-5 : gs == H2_BF16 ? 1e-2 : 1e-10));
        maxN = std::max(maxN, geoms[g]->host.tree.N);
    }
    const size_t budget = o.workspace_bytes > 0 ? size_t(o.workspace_bytes)
                                                : req_doubles(S.get(), maxN) * S->max_active * sizeof(double);
    S->pool_len = budget / sizeof(double);
    if (S->pool_len < req_doubles(S.get(), 1)) return fail(H2_E_INVALID_ARG, "workspace budget too small");
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, S->pool_len * sizeof(double));
    if (e != cudaSuccess) return fail(H2_E_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    S->pool = static_cast<double*>(p);
    S->free_list[0] = S->pool_len;
    e = cudaMallocHost(&p, sizeof(double) * size_t(S->max_active) * (S->m + 1));
    if (e != cudaSuccess) return fail(H2_E_OOM, std::string("cudaMallocHost: ") + cudaGetErrorString(e));
    S->pinned = static_cast<double*>(p);
    for (int k = S->max_active - 1; k >= 0; --k) S->pinned_free.push_back(k);
    for (int g = 0; g < ngeom; ++g) {
        cudaStream_t st;
        H2_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        S->streams.push_back(st);
        const int64_t N = geoms[g]->host.tree.N;
        double *x = nullptr, *y = nullptr;
        H2_CUDA(cudaMalloc(&x, sizeof(double) * N * S->max_active));
        H2_CUDA(cudaMalloc(&y, sizeof(double) * N * S->max_active));
        S->Xg.push_back(x);
        S->Yg.push_back(y);
        int rc = grow_vec(geoms[g], S->max_active);
        if (rc != H2_OK) return rc;
        geoms[g]->profile = false;
        double delta = 0.0;
        if (S->res[g] != geoms[g]) {
            rc = grow_vec(S->res[g], S->max_active);
            if (rc != H2_OK) return rc;
            S->res[g]->profile = false;
            // error of the inner operator on one seeded N(0, 1) vector
            std::vector<double> v(static_cast<size_t>(N)), ya(static_cast<size_t>(N)), yb(static_cast<size_t>(N));
            std::mt19937_64 gen(0x5eed + uint64_t(g));
            std::normal_distribution<double> nd(0.0, 1.0);
            for (auto& a : v) a = nd(gen);
            H2_CUDA(cudaMemcpyAsync(x, v.data(), sizeof(double) * N, cudaMemcpyHostToDevice, st));
            H2_TRY(matvec_any(geoms[g], x, N, y, N, 1, st));
            H2_CUDA(cudaMemcpyAsync(ya.data(), y, sizeof(double) * N, cudaMemcpyDeviceToHost, st));
            H2_TRY(matvec_any(S->res[g], x, N, y, N, 1, st));
            H2_CUDA(cudaMemcpyAsync(yb.data(), y, sizeof(double) * N, cudaMemcpyDeviceToHost, st));
            H2_CUDA(cudaStreamSynchronize(st));
            double dn = 0.0, vn = 0.0;
            for (int64_t i = 0; i < N; ++i) {
                dn += (ya[i] - yb[i]) * (ya[i] - yb[i]);
                vn += v[i] * v[i];
            }
            delta = std::sqrt(dn / vn);
        }
        S->delta.push_back(delta);
    }
    S->stats.workspace_bytes = int64_t(S->pool_len * sizeof(double));
    {
        // every handle serves one geometry slot: products of different slots run
        // concurrently and each handle has one coefficient buffer
        std::map<h2_handle, int> slot;
        for (int g = 0; g < ngeom; ++g)
            for (h2_handle hh : {S->geoms[g], S->res[g]}) {
                auto it = slot.find(hh);
                if (it != slot.end() && it->second != g)
                    return fail(H2_E_INVALID_ARG, "one handle appears in two geometry slots");
                slot[hh] = g;
            }
    }
    for (int g = 0; g < ngeom; ++g) {
        S->geoms[g]->server = S.get();
        S->res[g]->server = S.get();
    }
    h2_server_s* raw = S.get();
    S->worker = std::thread([raw] { serve_loop(raw); });
    *out = S.release();
    return H2_OK;
}

extern "C" int h2_server_submit(h2_server S, int geom, double shift, double scale, const double* f,
                                double rtol, int maxit, int64_t* ticket) {
    g_err.clear();
    if (!S || !f || !ticket) return fail(H2_E_INVALID_ARG, "NULL argument");
    if (geom < 0 || geom >= int(S->geoms.size())) return fail(H2_E_INVALID_ARG, "unknown geometry");
    if (!(rtol > 0.0 && rtol < 1.0) || maxit < 1) return fail(H2_E_INVALID_ARG, "rtol or maxit out of range");
    const int64_t N = S->geoms[geom]->host.tree.N;
    std::unique_ptr<Req> r(new Req());
    r->g = geom;
    r->shift = shift;
    r->scale = scale;
    r->rtol = rtol;
    r->maxit = maxit;
    r->f.assign(f, f + N);
    r->ws_len = req_doubles(S, N);
    if (r->ws_len > S->pool_len) return fail(H2_E_OOM, "request workspace exceeds the server's budget");
    r->t_submit = now_s();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (!S->worker_error.empty()) return fail(S->worker_rc, "server stopped: " + S->worker_error);
        Req* raw = r.release();
        raw->id = S->next_id++;
        *ticket = raw->id;
        S->queue.push_back(raw);
        S->reqs[raw->id] = raw;
        S->stats.submitted++;
    }
    S->cv_work.notify_one();
    return H2_OK;
}

extern "C" int h2_server_wait(h2_server S, int64_t ticket, double* x, h2_request_stats* st) {
    g_err.clear();
    if (!S) return fail(H2_E_INVALID_ARG, "NULL server");
    Req* r = nullptr;
    {
        std::unique_lock<std::mutex> lk(S->mu);
        auto it = S->reqs.find(ticket);
        if (it == S->reqs.end()) return fail(H2_E_INVALID_ARG, "unknown ticket");
        r = it->second;
        S->cv_done.wait(lk, [&] { return r->t_done > 0.0; });
        S->reqs.erase(it);
    }
    std::unique_ptr<Req> own(r);
    if (x) std::copy(r->xh.begin(), r->xh.end(), x);
    if (st) {
        std::memset(st, 0, sizeof(*st));
        st->converged = r->converged ? 1 : 0;
        st->iterations = r->iters;
        st->restarts = r->restarts;
        st->op = r->op;
        st->rel_residual = r->relres;
        st->queue_seconds = r->t_admit - r->t_submit;
        st->latency_seconds = r->t_done - r->t_submit;
    }
    if (r->rc != H2_OK) return fail(r->rc, "request stopped by a device error: " + r->err);
    if (!r->converged) return fail(H2_E_NOT_CONVERGED, "request stopped before reaching rtol");
    return H2_OK;
}

extern "C" int h2_server_stats_get(h2_server S, h2_server_stats* st) {
    g_err.clear();
    if (!S || !st) return fail(H2_E_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    *st = S->stats;
    st->ticks = S->ticks.load();
    st->products = S->products.load();
    st->product_columns = S->product_columns.load();
    st->queued = int64_t(S->queue.size());
    st->active = int64_t(S->active.size());
    return H2_OK;
}

extern "C" void h2_server_destroy(h2_server S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        S->queue.clear();
    }
    S->cv_work.notify_all();
    if (S->worker.joinable()) S->worker.join();
    cudaDeviceSynchronize();
    for (auto& kv : S->reqs) delete kv.second;
    delete S;   // the destructor frees streams and buffers and releases the handles
}

