// Checkpoint of a constructed representation: the whole host state (tree,
// lists, pivots, operators and the packed device layout) written to one file
// and read back, so a geometry is constructed once and reloaded instead of
// rebuilt.  The paper has no counterpart; construction is its dominant cost
// (the initialization times of §6's tables).
//
// Format: the 8 bytes "H2STAR\0" + version, then every field in a fixed
// order, native little-endian, 64-bit sizes (a vector is its length, int64,
// followed by its elements), then an 8-byte checksum of everything before it.
// A file is read with every length bounded by the bytes left, its checksum is
// compared, and the loaded state is checked index by index against the
// buffers the device kernels address (offsets, lengths, alignment), so a
// truncated or corrupted file gives an error and never an out-of-range access.

#include <cstdio>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "h2_internal.hpp"

namespace h2 {
namespace {

// the last byte is the format version: raise it whenever fields() changes
constexpr char kMagic[8] = {'H', '2', 'S', 'T', 'A', 'R', '\0', '\3'};

// Checksum of the byte stream: the bytes as little-endian 64-bit words w_k,
// h <- (h xor w_k) * P (the 64-bit FNV prime, odd, so every step is a
// bijection of h and a change in any one word always changes the result),
// then the length mixed in the same way.  Streamed, so chunk boundaries do
// not matter.
struct Checksum {
    static constexpr uint64_t kPrime = 0x100000001b3ull;
    uint64_t h = 0xcbf29ce484222325ull;
    uint64_t total = 0;
    unsigned char buf[8] = {};
    int nbuf = 0;
    void word(uint64_t w) { h = (h ^ w) * kPrime; }
    void feed(const void* p, size_t n) {
        const unsigned char* b = static_cast<const unsigned char*>(p);
        total += n;
        if (nbuf > 0) {                       // complete the pending word first
            const size_t take = std::min(n, size_t(8 - nbuf));
            std::memcpy(buf + nbuf, b, take);
            nbuf += int(take);
            b += take;
            n -= take;
            if (nbuf < 8) return;
            uint64_t w;
            std::memcpy(&w, buf, 8);
            word(w);
            nbuf = 0;
        }
        for (; n >= 8; n -= 8, b += 8) { uint64_t w; std::memcpy(&w, b, 8); word(w); }
        std::memcpy(buf, b, n);               // n < 8
        nbuf = int(n);
    }
    uint64_t value() const {
        Checksum c = *this;
        if (c.nbuf > 0) {
            std::memset(c.buf + c.nbuf, 0, size_t(8 - c.nbuf));
            uint64_t w;
            std::memcpy(&w, c.buf, 8);
            c.word(w);
        }
        c.word(total);
        return c.h;
    }
};

struct Writer {
    std::FILE* f;
    bool ok = true;
    Checksum sum;
    void raw(const void* p, size_t n) {
        if (ok && n > 0 && std::fwrite(p, 1, n, f) != n) ok = false;
        sum.feed(p, n);
    }
    template <class T> void pod(const T& v) {
        static_assert(std::is_trivially_copyable<T>::value, "plain data only");
        raw(&v, sizeof(T));
    }
    template <class T> void vec(const std::vector<T>& v) {
        pod(int64_t(v.size()));
        raw(v.data(), v.size() * sizeof(T));
    }
    template <class T> void vec2(const std::vector<std::vector<T>>& v) {
        pod(int64_t(v.size()));
        for (const auto& a : v) vec(a);
    }
    template <class T> void vec3(const std::vector<std::vector<std::vector<T>>>& v) {
        pod(int64_t(v.size()));
        for (const auto& a : v) vec2(a);
    }
};

struct Reader {
    std::FILE* f;
    int64_t left;                     // bytes of fields left (the checksum excluded)
    bool ok = true;
    Checksum sum;
    void raw(void* p, size_t n) {
        if (!ok) return;
        if (int64_t(n) > left || (n > 0 && std::fread(p, 1, n, f) != n)) { ok = false; return; }
        left -= int64_t(n);
        sum.feed(p, n);
    }
    template <class T> void pod(T& v) { raw(&v, sizeof(T)); }
    int64_t count(size_t min_bytes_each) {
        int64_t n = -1;
        pod(n);
        if (!ok || n < 0 || (min_bytes_each > 0 && n > left / int64_t(min_bytes_each))) {
            ok = false;
            return 0;
        }
        return n;
    }
    template <class T> void vec(std::vector<T>& v) {
        const int64_t n = count(sizeof(T));
        if (!ok) return;
        v.resize(size_t(n));
        raw(v.data(), size_t(n) * sizeof(T));
    }
    template <class T> void vec2(std::vector<std::vector<T>>& v) {
        const int64_t n = count(8);
        if (!ok) return;
        v.resize(size_t(n));
        for (auto& a : v) vec(a);
    }
    template <class T> void vec3(std::vector<std::vector<std::vector<T>>>& v) {
        const int64_t n = count(8);
        if (!ok) return;
        v.resize(size_t(n));
        for (auto& a : v) vec2(a);
    }
};

// One set of routines lists the fields for both directions (IO = Writer on a
// const state, Reader on a mutable one), so writer and reader cannot disagree
// on the order.
template <class IO, class C> void csr(IO& io, C& c) {
    io.vec(c.ptr);
    io.vec(c.idx);
}

template <class IO, class C> void csr_list(IO& io, C& v) {
    int64_t n = int64_t(v.size());
    if constexpr (std::is_same<IO, Writer>::value) {
        io.pod(n);
    } else {
        n = io.count(16);
        if (!io.ok) return;
        v.resize(size_t(n));
    }
    for (auto& c : v) csr(io, c);
}

template <class IO, class R> void rows(IO& io, R& r) {
    io.vec(r.dst);
    io.vec(r.aoff);
    io.vec(r.seg_ptr);
    io.vec(r.seg_off);
    io.vec(r.rows);
    io.vec(r.kpad);
    io.vec(r.seg_len);
    io.vec(r.seg_col);
    io.pod(r.cur_col);
    io.pod(r.kpad_max);
    io.pod(r.entries);
    io.pod(r.src_coeffs);
    io.pod(r.dst_coeffs);
}

template <class IO, class V> void rows_list(IO& io, V& v) {
    int64_t n = int64_t(v.size());
    if constexpr (std::is_same<IO, Writer>::value) {
        io.pod(n);
    } else {
        n = io.count(64);
        if (!io.ok) return;
        v.resize(size_t(n));
    }
    for (auto& r : v) rows(io, r);
}

template <class IO, class H> void fields(IO& io, H& h) {
    io.pod(h.kern.kind);
    io.pod(h.kern.param);
    io.pod(h.variant);
    io.pod(h.storage);
    io.pod(h.near_mode);
    io.pod(h.tensor_cores);
    io.pod(h.m2l_fly);
    io.pod(h.m2l_dev);
    io.pod(h.eps_far);
    io.pod(h.eps_ver);
    io.pod(h.build_seconds);
    io.pod(h.pivot_seconds);
    io.pod(h.piv_problems_dev);
    io.pod(h.piv_problems_host);
    io.pod(h.near_pairs);
    io.pod(h.near_evals);
    io.pod(h.lowrank_entries);
    // tree
    auto& t = h.tree;
    io.pod(t.d);
    io.pod(t.kappa);
    io.pod(t.N);
    for (int k = 0; k < 3; ++k) io.pod(t.lo[k]);
    io.pod(t.side);
    io.vec(t.perm);
    io.vec(t.leaf_ptr);
    io.vec(t.x);
    // lists
    csr_list(io, h.lists.far);
    csr_list(io, h.lists.ver);
    csr_list(io, h.lists.sqrtd);
    csr_list(io, h.lists.star);
    csr(io, h.lists.near_star);
    csr(io, h.lists.near_sqrt);
    // bases
    int64_t nb = int64_t(h.bases.size());
    if constexpr (std::is_same<IO, Writer>::value) io.pod(nb);
    else { nb = io.count(64); if (!io.ok) return; h.bases.resize(size_t(nb)); }
    for (auto& B : h.bases) {
        io.pod(B.lmin);
        io.pod(B.il_kind);
        io.vec3(B.tau);
        io.vec3(B.sig);
        io.vec2(B.U);
        io.vec3(B.Ut);
        io.vec3(B.T);
    }
    // (H2+H)* blocks
    int64_t nl = int64_t(h.lowrank.size());
    if constexpr (std::is_same<IO, Writer>::value) io.pod(nl);
    else { nl = io.count(40); if (!io.ok) return; h.lowrank.resize(size_t(nl)); }
    for (auto& L : h.lowrank) {
        io.pod(L.level);
        io.pod(L.X);
        io.pod(L.Y);
        io.pod(L.k);
        io.vec(L.U);
        io.vec(L.V);
    }
    // packed device layout
    auto& P = h.packed;
    io.pod(P.nb);
    io.vec(P.pivot_x);
    io.pod(P.m2l_base);
    io.pod(P.m2l_len);
    io.pod(P.near_stored);
    io.pod(P.box_total);
    io.vec(P.box_base);
    io.vec(P.rank);
    io.vec(P.voff);
    io.pod(P.vlen);
    io.pod(P.q_base);
    io.pod(P.v_base);
    io.pod(P.u_base);
    io.pod(P.phi_base);
    io.pod(P.veclen);
    io.vec(P.ops);
    io.vec(P.uoff);
    io.vec(P.ustride);
    io.vec(P.utoff);
    rows(io, P.p2m);
    rows_list(io, P.m2m);
    rows_list(io, P.l2l);
    rows(io, P.m2l);
    rows(io, P.leaf);
    io.pod(P.rank_max);
    io.pod(P.near_entries);
    io.vec(P.near_ptr);
    io.vec(P.near_idx);
    io.vec(P.lr_level_ptr);
    io.vec(P.lr_x0);
    io.vec(P.lr_mx);
    io.vec(P.lr_y0);
    io.vec(P.lr_my);
    io.vec(P.lr_uoff);
    io.vec(P.lr_voff);
    io.vec(P.lr_toff);
    io.vec(P.lr_k);
    io.pod(P.lr_tlen);
}

// ---- consistency of a loaded state ------------------------------------------

bool monotone_from0(const std::vector<int64_t>& p, int64_t last) {
    if (p.empty() || p[0] != 0 || p.back() != last) return false;
    for (size_t i = 1; i < p.size(); ++i)
        if (p[i] < p[i - 1]) return false;
    return true;
}

bool csr_ok(const Csr& c, int64_t nrow, int64_t ncol) {
    if (int64_t(c.ptr.size()) != nrow + 1 || !monotone_from0(c.ptr, int64_t(c.idx.size()))) return false;
    for (int64_t v : c.idx)
        if (v < 0 || v >= ncol) return false;
    return true;
}

// every access of a block-row task list stays inside ops (n_ops entries),
// targets inside [d_lo, d_hi) and sources inside [s_lo, s_hi) of the
// coefficient buffer; rows start 16-byte aligned; segments tile [0, kpad)
std::string rows_ok(const RowTasks& R, int64_t n_ops, int64_t d_lo, int64_t d_hi, int64_t s_lo,
                    int64_t s_hi, bool check_ops, const char* what) {
    const size_t n = R.dst.size();
    const std::string w = std::string(what) + ": ";
    if (R.rows.size() != n || R.kpad.size() != n || R.aoff.size() != n || R.seg_ptr.size() != n + 1)
        return w + "task arrays differ in length";
    const size_t ns = R.seg_off.size();
    if (R.seg_len.size() != ns || R.seg_col.size() != ns) return w + "segment arrays differ in length";
    if (!monotone_from0(R.seg_ptr, int64_t(ns))) return w + "segment pointers";
    int32_t kmax = 0;
    int64_t entries = 0, src = 0, dstc = 0;
    for (size_t t = 0; t < n; ++t) {
        const int64_t r = R.rows[t], kp = R.kpad[t], a = R.aoff[t], d = R.dst[t];
        if (r < 0 || kp < 0 || kp % 4 != 0 || a < 0 || a % 4 != 0) return w + "task shape or alignment";
        if (check_ops && a + r * kp > n_ops) return w + "operator block outside the operator array";
        if (d < d_lo || d + r > d_hi) return w + "target outside its coefficient region";
        int64_t col = 0;
        for (int64_t e = R.seg_ptr[t]; e < R.seg_ptr[t + 1]; ++e) {
            const int64_t o = R.seg_off[size_t(e)], len = R.seg_len[size_t(e)];
            if (len < 0 || o < s_lo || o + len > s_hi) return w + "segment outside its coefficient region";
            if (R.seg_col[size_t(e)] != col) return w + "segment columns";
            col += len;
        }
        if (col > kp) return w + "segments wider than the padded row";
        kmax = std::max(kmax, int32_t(kp));
        entries += r * kp;
        src += kp;
        dstc += r;
    }
    if (R.kpad_max != kmax || (check_ops && R.entries != entries) || R.src_coeffs != src ||
        R.dst_coeffs != dstc)
        return w + "task totals";
    return "";
}

std::string validate(const Host& H) {
    const Tree& t = H.tree;
    const Packed& P = H.packed;
    if (H.kern.kind < 0 || H.kern.kind > 3 || H.variant < 0 || H.variant > 5 || H.storage < 0 ||
        H.storage > 3 || H.near_mode < 0 || H.near_mode > 2 || (H.tensor_cores & ~1) ||
        (H.m2l_fly & ~1) || (H.m2l_dev & ~1) || (H.m2l_fly && H.m2l_dev))
        return "options out of range";
    {
        bool unsupported = false;
        if (const char* why = combination_error(H.storage, H.variant, H.near_mode, H.tensor_cores,
                                                H.m2l_fly ? 1 : H.m2l_dev ? 2 : 0, &unsupported))
            return std::string("option combination: ") + why;
        // the packed near field is the one the options select (h2_build and
        // h2_convert keep them in step)
        const bool stored = H.near_mode == 2 || (H.near_mode == 0 && H.storage != 1);
        if (bool(H.packed.near_stored) != stored) return "near-field mode disagrees with the packed near field";
    }
    if ((t.d != 2 && t.d != 3) || t.kappa < 0 || t.d * t.kappa > 24 || t.N < 1) return "tree shape";
    const int K = t.kappa;
    const int64_t N = t.N, nleaf = t.nboxes(K);
    if (int64_t(t.perm.size()) != N || int64_t(t.x.size()) != N * t.d) return "tree arrays";
    {
        std::vector<char> seen(size_t(N), 0);
        for (int64_t p : t.perm) {
            if (p < 0 || p >= N || seen[size_t(p)]) return "the tree permutation is not one";
            seen[size_t(p)] = 1;
        }
    }
    if (int64_t(t.leaf_ptr.size()) != nleaf + 1 || !monotone_from0(t.leaf_ptr, N)) return "leaf pointers";
    // lists (level-indexed ones: kappa + 1 levels, or empty)
    for (const std::vector<Csr>* L : {&H.lists.far, &H.lists.ver, &H.lists.sqrtd, &H.lists.star}) {
        if (L->empty()) continue;
        if (int64_t(L->size()) != K + 1) return "interaction lists";
        for (int l = 0; l <= K; ++l)
            if (!csr_ok((*L)[size_t(l)], t.nboxes(l), t.nboxes(l))) return "interaction lists";
    }
    for (const Csr* c : {&H.lists.near_star, &H.lists.near_sqrt})
        if (!c->ptr.empty() && !csr_ok(*c, nleaf, nleaf)) return "near-field lists";
    // bases
    if (H.bases.empty() || H.bases.size() > 2) return "number of bases";
    for (const Basis& B : H.bases) {
        if (B.lmin < 0 || B.lmin > std::max(K, 2) || B.il_kind < 0 || B.il_kind > 3) return "basis header";
        const std::vector<Csr>& L = B.il_kind == 0 ? H.lists.far : B.il_kind == 1 ? H.lists.ver
                                  : B.il_kind == 2 ? H.lists.sqrtd : H.lists.star;
        if (int64_t(L.size()) != K + 1) return "a basis refers to a missing list";
        if (int64_t(B.tau.size()) != K + 1 || int64_t(B.sig.size()) != K + 1) return "pivot levels";
        for (int l = 0; l <= K; ++l) {
            if (int64_t(B.tau[size_t(l)].size()) != t.nboxes(l) ||
                int64_t(B.sig[size_t(l)].size()) != t.nboxes(l))
                return "pivot boxes";
            for (const auto* pv : {&B.tau[size_t(l)], &B.sig[size_t(l)]})
                for (const auto& v : *pv)
                    for (int64_t p : v)
                        if (p < 0 || p >= N) return "pivot index";
        }
    }
    // packed layout
    if (P.nb != int(H.bases.size()) || int64_t(P.box_base.size()) != K + 2) return "packed header";
    for (int l = 0; l <= K; ++l)
        if (P.box_base[size_t(l) + 1] - P.box_base[size_t(l)] != t.nboxes(l) || P.box_base[0] != 0)
            return "box numbering";
    if (P.box_total != P.box_base[size_t(K) + 1]) return "box numbering";
    const int64_t ns = int64_t(P.nb) * P.box_total;
    if (int64_t(P.rank.size()) != ns || int64_t(P.voff.size()) != ns || int64_t(P.uoff.size()) != ns ||
        int64_t(P.ustride.size()) != ns || int64_t(P.utoff.size()) != ns)
        return "slot arrays";
    if (P.vlen < 0 || P.q_base != 0 || P.v_base != N || P.u_base != N + P.vlen ||
        P.phi_base != N + 2 * P.vlen || P.veclen != 2 * N + 2 * P.vlen)
        return "coefficient layout";
    if (P.m2l_base < 0 || P.m2l_len < 0 || (!H.m2l_dev && P.m2l_len != 0) ||
        (H.m2l_dev && int64_t(P.ops.size()) != P.m2l_base))
        return "operator array extent";
    const int64_t n_ops = H.m2l_dev ? P.m2l_base + P.m2l_len : int64_t(P.ops.size());
    for (int64_t s = 0; s < ns; ++s) {
        const int64_t r = P.rank[size_t(s)], o = P.voff[size_t(s)];
        if (r < 0 || o < 0 || o + r > P.vlen) return "coefficient slots";
        const int64_t ut = P.utoff[size_t(s)];
        if (ut < -1 || ut > n_ops) return "transfer offsets";   // an empty block may sit at the end
    }
    // leaf bases addressed by the on-the-fly leaf kernel: rows of U_X
    for (int b = 0; b < P.nb; ++b)
        for (int64_t X = 0; X < nleaf; ++X) {
            const int64_t s = b * P.box_total + P.box_base[size_t(K)] + X;
            const int64_t r = P.rank[size_t(s)], m = t.leaf_ptr[size_t(X) + 1] - t.leaf_ptr[size_t(X)];
            if (r == 0 || m == 0) continue;
            const int64_t uo = P.uoff[size_t(s)], st = P.ustride[size_t(s)];
            if (uo < 0 || st < r || uo + (m - 1) * st + r > n_ops) return "leaf basis offsets";
        }
    const int64_t V = P.veclen, v0 = P.v_base, u0 = P.u_base, vl = P.vlen;
    std::string e = rows_ok(P.p2m, n_ops, 0, V, 0, V, true, "P2M");
    if (!e.empty()) return e;
    if (int64_t(P.m2m.size()) != K + 1 || int64_t(P.l2l.size()) != K + 1) return "transfer task levels";
    for (int l = 0; l <= K; ++l) {
        if (!(e = rows_ok(P.m2m[size_t(l)], n_ops, 0, V, 0, V, true, "M2M")).empty()) return e;
        if (!(e = rows_ok(P.l2l[size_t(l)], n_ops, 0, V, 0, V, true, "L2L")).empty()) return e;
    }
    // M2L: targets in u and sources in v (the pivot coordinates are indexed
    // by the offset inside those regions)
    if (!(e = rows_ok(P.m2l, n_ops, u0, u0 + vl, v0, v0 + vl, !H.m2l_fly, "M2L")).empty()) return e;
    if (!(e = rows_ok(P.leaf, n_ops, 0, V, 0, V, true, "leaf")).empty()) return e;
    if ((H.m2l_fly || H.m2l_dev) && int64_t(P.pivot_x.size()) != t.d * P.vlen) return "pivot coordinates";
    if (H.m2l_dev) {
        for (size_t k = 0; k < P.m2l.aoff.size(); ++k)
            if (P.m2l.aoff[k] < P.m2l_base) return "device-formed M2L block inside the host array";
    }
    if (P.near_stored & ~1) return "near-field mode";
    if (!csr_ok(Csr{P.near_ptr, P.near_idx}, nleaf, nleaf)) return "near-field lists";
    // (H2+H)* blocks
    const size_t nbk = P.lr_k.size();
    for (const auto* a : {&P.lr_x0, &P.lr_mx, &P.lr_y0, &P.lr_my, &P.lr_uoff, &P.lr_voff, &P.lr_toff})
        if (a->size() != nbk) return "low-rank arrays differ in length";
    // the product reads lr_level_ptr[0 .. kappa + 1] whether or not there are blocks
    if (int64_t(P.lr_level_ptr.size()) != K + 2 || !monotone_from0(P.lr_level_ptr, int64_t(nbk)))
        return "low-rank level pointers";
    if (P.lr_tlen < 0) return "low-rank scratch length";
    for (size_t k = 0; k < nbk; ++k) {
        const int64_t x0 = P.lr_x0[k], mx = P.lr_mx[k], y0 = P.lr_y0[k], my = P.lr_my[k], kk = P.lr_k[k];
        if (x0 < 0 || mx < 0 || x0 + mx > N || y0 < 0 || my < 0 || y0 + my > N || kk < 0)
            return "low-rank block shape";
        if (P.lr_uoff[k] < 0 || P.lr_uoff[k] + mx * kk > n_ops || P.lr_voff[k] < 0 ||
            P.lr_voff[k] + my * kk > n_ops || P.lr_toff[k] < 0 || P.lr_toff[k] + kk > P.lr_tlen)
            return "low-rank block offsets";
    }
    return "";
}

}  // namespace

void relink_lists(Host& H) {
    for (Basis& B : H.bases)
        B.il = B.il_kind == 0 ? &H.lists.far : B.il_kind == 1 ? &H.lists.ver
             : B.il_kind == 2 ? &H.lists.sqrtd : &H.lists.star;
}

std::string save_host(const Host& H, const char* path) {
    std::FILE* f = std::fopen(path, "wb");
    if (!f) return std::string("cannot open ") + path + " for writing";
    Writer w{f};
    w.raw(kMagic, sizeof(kMagic));
    fields(w, H);
    const uint64_t check = w.sum.value();
    if (w.ok && std::fwrite(&check, 1, sizeof(check), f) != sizeof(check)) w.ok = false;
    const bool closed = std::fclose(f) == 0;
    if (!w.ok || !closed) {
        std::remove(path);
        return std::string("write to ") + path + " failed";
    }
    return "";
}

std::string load_host(Host& H, const char* path) {
    std::FILE* f = std::fopen(path, "rb");
    if (!f) return std::string("cannot open ") + path;
    int64_t size = -1;
    if (std::fseek(f, 0, SEEK_END) == 0) size = int64_t(std::ftell(f));
    std::rewind(f);
    if (size < int64_t(sizeof(kMagic) + 8)) {
        std::fclose(f);
        return "not an H2* checkpoint (too short)";
    }
    Reader r{f, size - 8};
    char magic[8] = {};
    r.raw(magic, sizeof(magic));
    if (!r.ok || std::memcmp(magic, kMagic, sizeof(kMagic) - 1) != 0) {
        std::fclose(f);
        return "not an H2* checkpoint (magic)";
    }
    if (magic[7] != kMagic[7]) {
        std::fclose(f);
        return "checkpoint format version " + std::to_string(int(magic[7])) + ", this library reads " +
               std::to_string(int(kMagic[7]));
    }
    fields(r, H);
    const int64_t left = r.left;
    uint64_t check = 0;
    const bool got = r.ok && left == 0 && std::fread(&check, 1, sizeof(check), f) == sizeof(check);
    std::fclose(f);
    if (!r.ok) return "truncated or corrupted checkpoint";
    if (left != 0) return "trailing bytes after the checkpoint";
    if (!got || check != r.sum.value()) return "checkpoint checksum mismatch (corrupted file)";
    relink_lists(H);
    std::string e = validate(H);
    if (!e.empty()) return "inconsistent checkpoint: " + e;
    return "";
}

}  // namespace h2
