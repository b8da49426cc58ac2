// C ABI of the H2* library (declared in include/h2star.h): construction on the
// host (build.cpp), upload of the packed operators, and the MVP pipeline of
// CUDA kernels (mvp_kernels.cuh) launched on the caller's stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <memory>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/h2star.h"
#include "h2_internal.hpp"
#include "mvp_kernels.cuh"

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

struct h2_handle_s {
    h2::Host host;
    bool on_device = false;
    int device = -1;
    size_t tsize = 8;             // sizeof storage type
    int64_t bytes_device = 0;
    // device buffers
    void* ops = nullptr;          // T
    void* xs = nullptr;           // T, d x N
    void* q = nullptr;            // T, N
    void* phi = nullptr;          // T, N
    void* v = nullptr;            // T, vlen
    void* u = nullptr;            // T, vlen
    void* lr_t = nullptr;         // T, lr_tlen
    int64_t* perm = nullptr;
    int64_t* leaf_ptr = nullptr;
    int64_t* near_ptr = nullptr;
    int64_t* near_idx = nullptr;
    int32_t* rank = nullptr;
    int64_t* voff = nullptr;
    int64_t* uoff = nullptr;
    int64_t* utoff = nullptr;
    int64_t* m2m_tasks = nullptr;  // all levels concatenated
    int64_t* l2l_tasks = nullptr;
    std::vector<int64_t> m2m_lptr, l2l_lptr;   // host offsets per level
    int64_t* m2l_slot = nullptr;
    int64_t* m2l_toff = nullptr;
    int32_t* m2l_kpad = nullptr;
    int64_t* m2l_src_ptr = nullptr;
    int64_t* m2l_src = nullptr;
    int64_t m2l_ntask = 0;
    size_t m2l_smem = 0;
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
    int64_t launches = 0;               // kernels launched by h2_matvec (all calls)
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

template <typename T>
std::vector<T> convert(const std::vector<double>& a) {
    return std::vector<T>(a.begin(), a.end());
}

#define H2_TRY(x)                \
    do {                         \
        int rc_ = (x);           \
        if (rc_ != H2_OK) return rc_; \
    } while (0)

template <typename T>
int upload(h2_handle h) {
    const h2::Host& H = h->host;
    const h2::Packed& P = H.packed;
    const h2::Tree& t = H.tree;
    h->tsize = sizeof(T);
    {
        // operators: fp64 uploads the packed array directly, fp32 converts in chunks
        void* p = nullptr;
        const size_t n = std::max<size_t>(P.ops.size(), 1);
        H2_TRY(dev_alloc(h, &p, n * sizeof(T)));
        if (std::is_same<T, double>::value) {
            if (!P.ops.empty())
                H2_CUDA(cudaMemcpy(p, P.ops.data(), P.ops.size() * sizeof(double), cudaMemcpyHostToDevice));
        } else {
            const size_t chunk = size_t(1) << 24;
            std::vector<T> buf(std::min(chunk, P.ops.size()));
            for (size_t o = 0; o < P.ops.size(); o += chunk) {
                const size_t c = std::min(chunk, P.ops.size() - o);
                for (size_t k = 0; k < c; ++k) buf[k] = T(P.ops[o + k]);
                H2_CUDA(cudaMemcpy(static_cast<T*>(p) + o, buf.data(), c * sizeof(T), cudaMemcpyHostToDevice));
            }
        }
        h->ops = p;
    }
    {
        std::vector<T> xs(size_t(t.d) * t.N);
        for (int64_t i = 0; i < t.N; ++i)
            for (int k = 0; k < t.d; ++k) xs[size_t(k) * t.N + i] = T(t.x[size_t(i) * t.d + k]);
        T* p = nullptr;
        H2_TRY(dev_upload(h, &p, xs));
        h->xs = p;
    }
    H2_TRY(dev_alloc(h, &h->q, sizeof(T) * t.N));
    H2_TRY(dev_alloc(h, &h->phi, sizeof(T) * t.N));
    H2_TRY(dev_alloc(h, &h->v, sizeof(T) * std::max<int64_t>(P.vlen, 1)));
    H2_TRY(dev_alloc(h, &h->u, sizeof(T) * std::max<int64_t>(P.vlen, 1)));
    H2_TRY(dev_alloc(h, &h->lr_t, sizeof(T) * std::max<int64_t>(P.lr_tlen, 1)));
    H2_TRY(dev_upload(h, &h->perm, t.perm));
    H2_TRY(dev_upload(h, &h->leaf_ptr, t.leaf_ptr));
    H2_TRY(dev_upload(h, &h->near_ptr, P.near_ptr));
    H2_TRY(dev_upload(h, &h->near_idx, P.near_idx));
    H2_TRY(dev_upload(h, &h->rank, P.rank));
    H2_TRY(dev_upload(h, &h->voff, P.voff));
    H2_TRY(dev_upload(h, &h->uoff, P.uoff));
    H2_TRY(dev_upload(h, &h->utoff, P.utoff));
    std::vector<int64_t> m2m, l2l;
    h->m2m_lptr.assign(t.kappa + 2, 0);
    h->l2l_lptr.assign(t.kappa + 2, 0);
    for (int l = 0; l <= t.kappa; ++l) {
        m2m.insert(m2m.end(), P.m2m_tasks[l].begin(), P.m2m_tasks[l].end());
        l2l.insert(l2l.end(), P.l2l_tasks[l].begin(), P.l2l_tasks[l].end());
        h->m2m_lptr[l + 1] = int64_t(m2m.size());
        h->l2l_lptr[l + 1] = int64_t(l2l.size());
    }
    H2_TRY(dev_upload(h, &h->m2m_tasks, m2m));
    H2_TRY(dev_upload(h, &h->l2l_tasks, l2l));
    H2_TRY(dev_upload(h, &h->m2l_slot, P.m2l_slot));
    H2_TRY(dev_upload(h, &h->m2l_toff, P.m2l_toff));
    H2_TRY(dev_upload(h, &h->m2l_kpad, P.m2l_kpad));
    H2_TRY(dev_upload(h, &h->m2l_src_ptr, P.m2l_src_ptr));
    H2_TRY(dev_upload(h, &h->m2l_src, P.m2l_src));
    h->m2l_ntask = int64_t(P.m2l_slot.size());
    h->m2l_smem = size_t(P.m2l_kpad_max) * sizeof(T);
    if (h->m2l_smem > 48 * 1024) {
        if (h->m2l_smem > 227 * 1024)
            return fail(H2_E_UNSUPPORTED, "M2L source coefficients exceed shared memory (ranks too high)");
        H2_CUDA(cudaFuncSetAttribute(h2::k_m2l<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     int(h->m2l_smem)));
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
    H2_CUDA(cudaDeviceSynchronize());
    return H2_OK;
}

inline unsigned nblocks(int64_t n, int per) { return unsigned((n + per - 1) / per); }

template <typename T, int D, int KIND>
void launch_leaf(h2_handle h, cudaStream_t s) {
    const h2::Host& H = h->host;
    const h2::Tree& t = H.tree;
    const h2::Packed& P = H.packed;
    const int64_t nleaf = t.nboxes(t.kappa);
    h2::k_leaf<T, D, KIND><<<unsigned(nleaf), 128, 0, s>>>(
        nleaf, P.nb, P.box_total, P.box_base[t.kappa], h->leaf_ptr, h->near_ptr, h->near_idx,
        h->rank, h->voff, h->uoff, static_cast<const T*>(h->ops), static_cast<const T*>(h->u),
        static_cast<const T*>(h->xs), t.N, static_cast<const T*>(h->q), static_cast<T*>(h->phi),
        T(H.kern.param), T(H.kern.diag()));
}

template <typename T, int D>
void launch_leaf_d(h2_handle h, cudaStream_t s) {
    switch (h->host.kern.kind) {
        case 0: launch_leaf<T, D, 0>(h, s); break;
        case 1: launch_leaf<T, D, 1>(h, s); break;
        case 2: launch_leaf<T, D, 2>(h, s); break;
        default: launch_leaf<T, D, 3>(h, s); break;
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

// One right-hand side: X, Y are single device columns (user order, fp64).
template <typename T>
int matvec_one(h2_handle h, const double* X, double* Y, cudaStream_t s) {
    const h2::Host& H = h->host;
    const h2::Tree& t = H.tree;
    const h2::Packed& P = H.packed;
    const int K = t.kappa, d = t.d;
    const T* ops = static_cast<const T*>(h->ops);
    T* q = static_cast<T*>(h->q);
    T* phi = static_cast<T*>(h->phi);
    T* v = static_cast<T*>(h->v);
    T* u = static_cast<T*>(h->u);
    const int64_t nleaf = t.nboxes(K);

    int64_t& nl = h->launches;
    mark(h, s, ST_GATHER);
    ++nl;
    h2::k_gather<T><<<nblocks(t.N, 256), 256, 0, s>>>(X, h->perm, q, t.N);
    mark(h, s, ST_P2M);
    if (P.nb > 0 && P.vlen > 0) {
        const int64_t ntask = P.nb * nleaf;
        ++nl;
        h2::k_p2m<T><<<nblocks(ntask * 32, 256), 256, 0, s>>>(
            ntask, nleaf, P.box_total, P.box_base[K], h->leaf_ptr, h->rank, h->voff, h->uoff, ops, q, v);
    }
    mark(h, s, ST_M2M);
    for (int l = K - 1; l >= 1; --l) {
        const int64_t n = h->m2m_lptr[l + 1] - h->m2m_lptr[l];
        if (n == 0) continue;
        ++nl;
        h2::k_m2m<T><<<nblocks(n * 32, 256), 256, 0, s>>>(
            h->m2m_tasks + h->m2m_lptr[l], n, P.box_total, P.box_base[l], P.box_base[l + 1], 1 << d,
            h->rank, h->voff, h->utoff, ops, v);
    }
    mark(h, s, ST_M2L);
    if (P.vlen > 0) cudaMemsetAsync(u, 0, sizeof(T) * P.vlen, s);
    if (h->m2l_ntask > 0) {
        ++nl;
        h2::k_m2l<T><<<unsigned(h->m2l_ntask), 256, h->m2l_smem, s>>>(
            h->m2l_ntask, h->m2l_slot, h->m2l_toff, h->m2l_kpad, h->m2l_src_ptr, h->m2l_src, h->rank,
            h->voff, ops, v, u);
    }
    mark(h, s, ST_L2L);
    for (int l = 2; l <= K; ++l) {
        const int64_t n = h->l2l_lptr[l + 1] - h->l2l_lptr[l];
        if (n == 0) continue;
        ++nl;
        h2::k_l2l<T><<<nblocks(n * 32, 256), 256, 0, s>>>(
            h->l2l_tasks + h->l2l_lptr[l], n, P.box_total, P.box_base[l], P.box_base[l - 1], d,
            h->rank, h->voff, h->utoff, ops, u);
    }
    mark(h, s, ST_LEAF);
    ++nl;
    if (d == 2) launch_leaf_d<T, 2>(h, s);
    else launch_leaf_d<T, 3>(h, s);
    mark(h, s, ST_LOWRANK);
    if (H.variant == H2_PLUS_H_STAR && P.lr_tlen > 0) {
        T* tt = static_cast<T*>(h->lr_t);
        cudaMemsetAsync(tt, 0, sizeof(T) * P.lr_tlen, s);
        const int chunk = 4096;
        for (int l = 1; l <= K; ++l) {
            const int64_t b0 = P.lr_level_ptr[l], nb = P.lr_level_ptr[l + 1] - b0;
            if (nb == 0) continue;
            const int64_t maxmy = h->lr_maxm_level[2 * l + 1];
            for (int64_t off = 0; off < nb; off += 65535) {
                const int64_t cnt = std::min<int64_t>(65535, nb - off);
                dim3 grid(nblocks(maxmy, chunk), unsigned(cnt));
                ++nl;
                h2::k_lr_vtq<T><<<grid, 256, 0, s>>>(b0 + off, cnt, h->lr_y0, h->lr_my, h->lr_k, h->lr_voff,
                                                     h->lr_toff, ops, q, tt, chunk);
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
                h2::k_lr_ut<T><<<grid, 256, 0, s>>>(g0 + off, cnt, h->lr_gptr, h->lr_x0, h->lr_mx, h->lr_k,
                                                    h->lr_uoff, h->lr_toff, ops, tt, phi);
            }
        }
    }
    mark(h, s, ST_SCATTER);
    ++nl;
    h2::k_scatter<T><<<nblocks(t.N, 256), 256, 0, s>>>(phi, h->perm, Y, t.N);
    mark(h, s, ST_N);
    H2_CUDA(cudaGetLastError());
    return H2_OK;
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
    if (variant < 0 || variant > 2) return fail(H2_E_INVALID_ARG, "unknown variant");
    h2_build_opts o;
    std::memset(&o, 0, sizeof(o));
    if (opts) o = *opts;
    if (o.storage != H2_F64 && o.storage != H2_F32) return fail(H2_E_INVALID_ARG, "unknown storage");
    if (o.kappa < 0 || o.kappa > 20) return fail(H2_E_INVALID_ARG, "kappa out of range");
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
    H.eps_far = o.eps_far > 0 ? o.eps_far : tol;
    H.eps_ver = o.eps_ver > 0 ? o.eps_ver : tol;
    try {
        std::string e = h2::build_host(H, points, N, d, leaf_size, o.kappa,
                                       o.use_domain ? o.domain_lo : nullptr, o.domain_side, o.threads);
        if (!e.empty()) return fail(H2_E_INVALID_ARG, e);
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
        int rc = (o.storage == H2_F64) ? upload<double>(h.get()) : upload<float>(h.get());
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
    const int64_t N = h->host.tree.N;
    if (!X || !Y) return fail(H2_E_INVALID_ARG, "X or Y is NULL");
    if (nrhs < 1 || nrhs > 64) return fail(H2_E_INVALID_ARG, "nrhs must be in [1, 64]");
    if (ldx < N || ldy < N) return fail(H2_E_INVALID_ARG, "leading dimension < N");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    for (int c = 0; c < nrhs; ++c) {
        const double* x = X + int64_t(c) * ldx;
        double* y = Y + int64_t(c) * ldy;
        if (h->profile) {
            int rc = next_event_set(h);
            if (rc != H2_OK) return rc;
        }
        int rc = (h->tsize == 8) ? matvec_one<double>(h, x, y, s) : matvec_one<float>(h, x, y, s);
        if (rc != H2_OK) return rc;
    }
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
    const int64_t ts = H.storage == H2_F64 ? 8 : 4;
    int64_t nbasis = 0, ntrans = 0, nlr = 0;
    for (const auto& B : H.bases) {
        for (const auto& U : B.U) nbasis += int64_t(U.size());
        for (const auto& lv : B.Ut)
            for (const auto& M : lv) ntrans += int64_t(M.size());
    }
    nlr = H.lowrank_entries;
    st->bytes_basis = nbasis * ts;
    st->bytes_transfer = ntrans * ts;
    st->bytes_m2l = P.m2l_entries * ts;
    for (size_t k = 0; k < P.m2l_slot.size(); ++k) {
        st->m2l_src_coeffs += P.m2l_kpad[k];
        st->m2l_dst_coeffs += P.rank[P.m2l_slot[k]];
    }
    st->vlen = P.vlen;
    st->bytes_lowrank = nlr * ts;
    st->near_pairs = H.near_pairs;
    st->near_evals = H.near_evals;
    st->lowrank_pairs = int64_t(H.lowrank.size());
    st->bytes_device = h->bytes_device;
    // algorithmic bytes of one MVP with one RHS: every stored operator once,
    // coordinates for the near field, user vector in and out (fp64)
    st->alg_bytes_per_rhs = st->bytes_basis + st->bytes_transfer + st->bytes_m2l + st->bytes_lowrank +
                            t.N * t.d * ts + 2 * t.N * 8;
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
        for (auto& e : h->ev_pool) cudaEventDestroy(e);
    }
    delete h;
}

}  // extern "C"
