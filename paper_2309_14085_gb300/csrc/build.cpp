// Host construction of H2*(b+t), (H2+H)* and H2_sqrt(d)(b):
//   tree (§3.1), lists (§3.5 / §3.3), partially pivoted ACA (§3.6),
//   B2T NCA (Algorithm 1), T2B NCA (§5.1.1 item 2), pure ACA of the
//   vertex-sharing blocks (Algorithm 3), operators (§3.6.4) and the packed
//   level-batched layout the CUDA kernels read.
//
// Compiled with -ffp-contract=off so that the arithmetic is the same on x86
// and Arm hosts (no fused multiply-add contraction).
#include <omp.h>

#include <algorithm>
#include <chrono>
#include <memory>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <numeric>

#include "h2_internal.hpp"

namespace h2 {
namespace {

int64_t morton(const int* c, int level, int d) {
    int64_t key = 0;
    for (int b = 0; b < level; ++b)
        for (int k = 0; k < d; ++k) key |= int64_t((c[k] >> b) & 1) << (b * d + k);
    return key;
}

void demorton(int64_t key, int level, int d, int* c) {
    for (int k = 0; k < d; ++k) c[k] = 0;
    for (int b = 0; b < level; ++b)
        for (int k = 0; k < d; ++k) c[k] |= int((key >> (b * d + k)) & 1) << b;
}

// 'self' 0, far 1, vertex-sharing 2, other neighbour (shares a d'-surface, d' >= 1) 3
int classify(const int* a, const int* b, int d) {
    int m = 0, neq = 0;
    for (int k = 0; k < d; ++k) {
        const int t = std::abs(a[k] - b[k]);
        m = std::max(m, t);
        neq += (t == 0);
    }
    if (m == 0) return 0;
    if (m >= 2) return 1;
    return neq == 0 ? 2 : 3;
}

// ---------------------------------------------------------------------------
// Tree (§3.1)
// deepest tree the strict depth rule may reach
constexpr int kKappaCap = 20;

// Returns "" or an error message (the strict depth rule found no separating depth).
std::string build_tree(Tree& t, const double* P, int64_t N, int d, int leaf_size, int kappa_forced,
                       const double* dom_lo, double dom_side) {
    t.N = N;
    t.d = d;
    if (kappa_forced > 0) {
        t.kappa = kappa_forced;
    } else {
        int k = 0;
        while (double(leaf_size) * double(int64_t(1) << (d * k)) < double(N)) ++k;
        t.kappa = k;
    }
    if (dom_lo) {
        for (int k = 0; k < d; ++k) t.lo[k] = dom_lo[k];
        t.side = dom_side;
    } else {
        double hi[3];
        for (int k = 0; k < d; ++k) { t.lo[k] = P[k]; hi[k] = P[k]; }
        for (int64_t i = 1; i < N; ++i)
            for (int k = 0; k < d; ++k) {
                t.lo[k] = std::min(t.lo[k], P[i * d + k]);
                hi[k] = std::max(hi[k], P[i * d + k]);
            }
        double s = 0.0;
        for (int k = 0; k < d; ++k) s = std::max(s, hi[k] - t.lo[k]);
        t.side = s > 0.0 ? s : 1.0;
    }
    if (kappa_forced < 0) {
        // the strict reading of §3.1: from the formula's depth, deepen until
        // every leaf box holds at most leaf_size points
        for (;; ++t.kappa) {
            if (t.kappa > kKappaCap || int64_t(1) << (d * t.kappa) > (int64_t(1) << 24))
                return "no tree depth up to 2^24 leaves separates the points into leaves of leaf_size";
            const double sc = double(int64_t(1) << t.kappa);
            const int cm = (1 << t.kappa) - 1;
            std::vector<int64_t> keys(N);
#pragma omp parallel for schedule(static)
            for (int64_t i = 0; i < N; ++i) {
                int c[3];
                for (int k = 0; k < d; ++k) {
                    const double f = std::floor((P[i * d + k] - t.lo[k]) / t.side * sc);
                    c[k] = f < 0.0 ? 0 : (f > double(cm) ? cm : int(f));
                }
                keys[i] = morton(c, t.kappa, d);
            }
            std::sort(keys.begin(), keys.end());
            int64_t run = 0, worst = 0;
            for (int64_t i = 0; i < N; ++i) {
                run = (i > 0 && keys[i] == keys[i - 1]) ? run + 1 : 1;
                worst = std::max(worst, run);
            }
            if (worst <= leaf_size) break;
        }
    }
    const double scale = double(int64_t(1) << t.kappa);
    const int cmax = (1 << t.kappa) - 1;
    std::vector<int64_t> key(N);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        int c[3];
        for (int k = 0; k < d; ++k) {
            const double f = std::floor((P[i * d + k] - t.lo[k]) / t.side * scale);
            int ci = f < 0.0 ? 0 : (f > double(cmax) ? cmax : int(f));
            c[k] = ci;
        }
        key[i] = morton(c, t.kappa, d);
    }
    t.perm.resize(N);
    std::iota(t.perm.begin(), t.perm.end(), int64_t(0));
    std::stable_sort(t.perm.begin(), t.perm.end(),
                     [&](int64_t a, int64_t b) { return key[a] < key[b]; });
    const int64_t nleaf = t.nboxes(t.kappa);
    t.leaf_ptr.assign(nleaf + 1, 0);
    for (int64_t i = 0; i < N; ++i) t.leaf_ptr[key[i] + 1]++;
    for (int64_t L = 0; L < nleaf; ++L) t.leaf_ptr[L + 1] += t.leaf_ptr[L];
    t.x.resize(size_t(N) * d);
    for (int64_t i = 0; i < N; ++i)
        for (int k = 0; k < d; ++k) t.x[i * d + k] = P[t.perm[i] * d + k];
    return "";
}

// ---------------------------------------------------------------------------
// Lists (§3.5 weak admissibility with IL_far / IL_ver, §3.3 strong with eta = sqrt d)
void build_lists(const Tree& t, Lists& L) {
    const int d = t.d, K = t.kappa;
    L.far.assign(K + 1, Csr());
    L.ver.assign(K + 1, Csr());
    L.sqrtd.assign(K + 1, Csr());
    for (int l = 0; l <= K; ++l) {
        const int64_t n = t.nboxes(l);
        const int side = 1 << l;
        std::vector<std::vector<int64_t>> F(n), V(n), S(n);
        if (l >= 1) {
#pragma omp parallel for schedule(static)
            for (int64_t X = 0; X < n; ++X) {
                int c[3], p[3];
                demorton(X, l, d, c);
                for (int k = 0; k < d; ++k) p[k] = c[k] >> 1;
                const int nofs = (d == 2) ? 9 : 27;
                for (int o = 0; o < nofs; ++o) {
                    int q[3], nzero = 0;
                    bool ok = true;
                    int oo = o;
                    for (int k = 0; k < d; ++k) {
                        const int off = oo % 3 - 1;
                        oo /= 3;
                        q[k] = p[k] + off;
                        nzero += (off == 0);
                        if (q[k] < 0 || q[k] >= (side >> 1)) ok = false;
                    }
                    if (!ok) continue;
                    // parent neighbour in N_* (self or sharing a d'-surface, d' >= 1)
                    const bool in_near_star = nzero >= 1;
                    for (int ch = 0; ch < (1 << d); ++ch) {
                        int cc[3];
                        for (int k = 0; k < d; ++k) cc[k] = 2 * q[k] + ((ch >> k) & 1);
                        const int cls = classify(c, cc, d);
                        const int64_t key = morton(cc, l, d);
                        if (cls == 1) S[X].push_back(key);       // IL_sqrt: far, parent in N_sqrt
                        if (!in_near_star || cls == 0) continue;
                        if (cls == 1) F[X].push_back(key);
                        else if (cls == 2) V[X].push_back(key);
                    }
                }
                std::sort(F[X].begin(), F[X].end());
                std::sort(V[X].begin(), V[X].end());
                std::sort(S[X].begin(), S[X].end());
            }
        }
        auto pack = [n](std::vector<std::vector<int64_t>>& src, Csr& dst) {
            dst.ptr.assign(n + 1, 0);
            for (int64_t X = 0; X < n; ++X) dst.ptr[X + 1] = dst.ptr[X] + int64_t(src[X].size());
            dst.idx.resize(dst.ptr[n]);
            for (int64_t X = 0; X < n; ++X)
                std::copy(src[X].begin(), src[X].end(), dst.idx.begin() + dst.ptr[X]);
        };
        pack(F, L.far[l]);
        pack(V, L.ver[l]);
        pack(S, L.sqrtd[l]);
    }
    // leaf near fields
    const int64_t n = t.nboxes(K);
    const int side = 1 << K;
    std::vector<std::vector<int64_t>> NS(n), NQ(n);
#pragma omp parallel for schedule(static)
    for (int64_t X = 0; X < n; ++X) {
        int c[3];
        demorton(X, K, d, c);
        const int nofs = (d == 2) ? 9 : 27;
        for (int o = 0; o < nofs; ++o) {
            int q[3];
            bool ok = true;
            int oo = o;
            for (int k = 0; k < d; ++k) {
                q[k] = c[k] + oo % 3 - 1;
                oo /= 3;
                if (q[k] < 0 || q[k] >= side) ok = false;
            }
            if (!ok) continue;
            const int cls = classify(c, q, d);
            const int64_t key = morton(q, K, d);
            NQ[X].push_back(key);
            if (cls == 0 || cls == 3) NS[X].push_back(key);
        }
        std::sort(NS[X].begin(), NS[X].end());
        std::sort(NQ[X].begin(), NQ[X].end());
    }
    auto pack = [n](std::vector<std::vector<int64_t>>& src, Csr& dst) {
        dst.ptr.assign(n + 1, 0);
        for (int64_t X = 0; X < n; ++X) dst.ptr[X + 1] = dst.ptr[X] + int64_t(src[X].size());
        dst.idx.resize(dst.ptr[n]);
        for (int64_t X = 0; X < n; ++X)
            std::copy(src[X].begin(), src[X].end(), dst.idx.begin() + dst.ptr[X]);
    };
    pack(NS, L.near_star);
    pack(NQ, L.near_sqrt);
}

// ---------------------------------------------------------------------------
// Partially pivoted ACA (§3.6), in the reading documented with the oracle:
// first row first; residual row; column pivot = first argmax over unused
// columns; a row whose largest residual is at most kAcaNoise times the largest
// pivot so far (rounding: coincident points, a block captured to full rank)
// is spent -> next unused row; residual column; incremental Frobenius norm;
// next row = first argmax of |u| over unused rows.  Stopping: the first cross
// k with |u||v| <= eps ||S||_F whose next kAcaLookahead crosses pass the test
// too; crosses 1..k are kept and the look-ahead ones dropped (one cross
// under-estimates the remaining error of the large, nearly singular search
// blocks -- stopping at the first pass left H2*(b+t) an order of magnitude
// less accurate than the paper's tables -- while keeping the look-ahead
// crosses, which lie below the tolerance, makes the interpolation operators
// ill-conditioned).
constexpr int kAcaLookahead = 2;
constexpr double kAcaNoise = 0x1p-46;

// The sums of the stopping estimate (|u|^2, |v|^2, u_l . u, v_l . v) in one
// fixed order: the terms in segments of kSumSeg, each segment over 256 lanes
// (lane p summing the segment's terms p, p + 256, p + 512, ... in turn) and
// then over the lanes pairwise (p + w into p for w = 128, 64, ..., 1), and the
// segment totals in segment order, the products fused into the additions
// (std::fma rounds once on every host).  The residual entries themselves take
// a rounded product and a rounded subtraction per cross, in cross order, as
// the oracle does: their exact values decide the argmax ties (symmetric point
// sets have many).  The device pivot search sums in the same
// order with the same operations (one CTA per segment), so both take the same
// stopping decisions bit for bit.
constexpr int kSumLanes = 256;
constexpr int64_t kSumSeg = 4096;

double lane_tree(double* s) {
    for (int w = kSumLanes / 2; w >= 1; w >>= 1)
        for (int p = 0; p < w; ++p) s[p] = s[p] + s[p + w];
    return s[0];
}

// sum_j a[j] * b[j] in the order above
double lane_dot(const double* a, const double* b, int64_t n) {
    double S = 0.0;
    for (int64_t g0 = 0; g0 < n; g0 += kSumSeg) {
        double s[kSumLanes] = {};
        const int64_t e = std::min(n, g0 + kSumSeg);
        for (int64_t j0 = g0; j0 < e; j0 += kSumLanes) {
            const int m = int(std::min<int64_t>(kSumLanes, e - j0));
            for (int p = 0; p < m; ++p) s[p] = std::fma(a[j0 + p], b[j0 + p], s[p]);
        }
        S = S + lane_tree(s);
    }
    return S;
}

struct AcaResult {
    std::vector<int> rows, cols;
    std::vector<std::vector<double>> us, vs;   // kept only when requested
};

void aca(const Tree& t, const KernelSpec& G, const std::vector<int64_t>& I,
         const std::vector<int64_t>& J, double eps, bool keep, AcaResult& out) {
    out.rows.clear();
    out.cols.clear();
    out.us.clear();
    out.vs.clear();
    const int64_t nI = int64_t(I.size()), nJ = int64_t(J.size());
    if (nI == 0 || nJ == 0) return;
    const int d = t.d;
    std::vector<double> xI(nI * d), xJ(nJ * d);
    for (int64_t i = 0; i < nI; ++i)
        for (int k = 0; k < d; ++k) xI[i * d + k] = t.x[I[i] * d + k];
    for (int64_t j = 0; j < nJ; ++j)
        for (int k = 0; k < d; ++k) xJ[j * d + k] = t.x[J[j] * d + k];
    auto entry = [&](int64_t i, int64_t j) {
        double s = 0.0;
        for (int k = 0; k < d; ++k) { const double q = xI[i * d + k] - xJ[j * d + k]; s = s + q * q; }
        return G(s);
    };
    // a whole row K(x_i, x_J): for 1/r and the IMQ the same operations as
    // entry() in a loop without calls or branches, which the compiler turns
    // into vector square roots and divisions (IEEE, so the values are equal)
    auto entry_row = [&](int64_t i, double* out) {
        const double* xi = xI.data() + i * d;
        if (G.kind == 1 || G.kind == 2) {
            const double diag = G.diag(), c = G.param;
            const bool imq = G.kind == 2;
            for (int64_t j = 0; j < nJ; ++j) {
                double s = 0.0;
                for (int k = 0; k < d; ++k) { const double q = xi[k] - xJ[j * d + k]; s = s + q * q; }
                const double r = std::sqrt(s);
                double g;
                if (imq) { const double t = r / c; g = 1.0 / std::sqrt(1.0 + t * t); }
                else g = 1.0 / r;
                out[j] = s == 0.0 ? diag : g;
            }
        } else {
            for (int64_t j = 0; j < nJ; ++j) out[j] = entry(i, j);
        }
    };
    std::vector<std::vector<double>>& us = out.us;
    std::vector<std::vector<double>>& vs = out.vs;
    std::vector<char> row_used(nI, 0), col_used(nJ, 0);
    std::vector<double> r(nJ), rn(nJ), u(nI), pv;
    double S2 = 0.0;
    int64_t i = 0;
    double pmax = 0.0;
    int64_t first = -1;     // crosses kept if the running look-ahead confirms the stop
    const int64_t kmax = std::min(nI, nJ);
    auto next_free_row = [&]() -> int64_t {
        for (int64_t a = 0; a < nI; ++a)
            if (!row_used[a]) return a;
        return -1;
    };
    // residual row of row position `ir` against every accepted cross, l in order
    auto fresh_row = [&](int64_t ir, std::vector<double>& out_r) {
        entry_row(ir, out_r.data());
        for (size_t l = 0; l < us.size(); ++l) {
            const double a = us[l][ir];
            const double* vl = vs[l].data();
            for (int64_t j = 0; j < nJ; ++j) out_r[j] = out_r[j] - a * vl[j];
        }
    };
    fresh_row(i, r);
    while (int64_t(out.rows.size()) < kmax) {
        row_used[i] = 1;
        int64_t jb = -1;
        double best = -1.0;
        for (int64_t j = 0; j < nJ; ++j) {
            const double a = col_used[j] ? -1.0 : std::fabs(r[j]);
            if (a > best) { best = a; jb = j; }
        }
        if (best <= kAcaNoise * pmax || best <= 0.0) {
            i = next_free_row();
            if (i < 0) break;
            fresh_row(i, r);
            continue;
        }
        pmax = std::max(pmax, best);
        const double piv = r[jb];
        std::vector<double> v(nJ);
        for (int64_t j = 0; j < nJ; ++j) v[j] = r[j] / piv;
        for (int64_t a = 0; a < nI; ++a) u[a] = entry(a, jb);
        for (size_t l = 0; l < us.size(); ++l) {
            const double bb = vs[l][jb];
            const double* ul = us[l].data();
            for (int64_t a = 0; a < nI; ++a) u[a] = u[a] - bb * ul[a];
        }
        col_used[jb] = 1;
        const double uu = lane_dot(u.data(), u.data(), nI);
        const double vv = lane_dot(v.data(), v.data(), nJ);
        // next row: first argmax of |u| over unused rows (the same choice the
        // step after the stopping test makes)
        int64_t ib = -1;
        double bi = -1.0;
        for (int64_t a = 0; a < nI; ++a) {
            const double q = row_used[a] ? -1.0 : std::fabs(u[a]);
            if (q > bi) { bi = q; ib = a; }
        }
        const bool fuse = bi > 0.0;
        // one pass over the previous crosses: v_l . v for the norm update and,
        // when the next row is known, its residual.  Four crosses share a sweep
        // over j: each rn[j] takes its subtractions in l order and each v_l . v
        // its terms in the order of lane_dot, so the results are those of one
        // cross at a time.
        pv.assign(us.size(), 0.0);
        if (fuse)
            entry_row(ib, rn.data());
        const size_t np = us.size();
        size_t l = 0;
        double s0[kSumLanes], s1[kSumLanes], s2[kSumLanes], s3[kSumLanes];
        for (; l + 4 <= np; l += 4) {
            const double *v0 = vs[l].data(), *v1 = vs[l + 1].data(), *v2 = vs[l + 2].data(),
                         *v3 = vs[l + 3].data();
            const double a0 = fuse ? us[l][ib] : 0.0, a1 = fuse ? us[l + 1][ib] : 0.0,
                         a2 = fuse ? us[l + 2][ib] : 0.0, a3 = fuse ? us[l + 3][ib] : 0.0;
            for (int64_t g0 = 0; g0 < nJ; g0 += kSumSeg) {
                std::fill(s0, s0 + kSumLanes, 0.0);
                std::fill(s1, s1 + kSumLanes, 0.0);
                std::fill(s2, s2 + kSumLanes, 0.0);
                std::fill(s3, s3 + kSumLanes, 0.0);
                const int64_t e = std::min(nJ, g0 + kSumSeg);
                for (int64_t j0 = g0; j0 < e; j0 += kSumLanes) {
                    const int m = int(std::min<int64_t>(kSumLanes, e - j0));
                    const double *w0 = v0 + j0, *w1 = v1 + j0, *w2 = v2 + j0, *w3 = v3 + j0;
                    const double* vj = v.data() + j0;
                    if (fuse) {
                        double* x = rn.data() + j0;
                        for (int p = 0; p < m; ++p) {
                            double y = x[p];
                            y = y - a0 * w0[p];
                            y = y - a1 * w1[p];
                            y = y - a2 * w2[p];
                            y = y - a3 * w3[p];
                            x[p] = y;
                        }
                    }
                    for (int p = 0; p < m; ++p) {
                        s0[p] = std::fma(w0[p], vj[p], s0[p]);
                        s1[p] = std::fma(w1[p], vj[p], s1[p]);
                        s2[p] = std::fma(w2[p], vj[p], s2[p]);
                        s3[p] = std::fma(w3[p], vj[p], s3[p]);
                    }
                }
                pv[l] = pv[l] + lane_tree(s0);
                pv[l + 1] = pv[l + 1] + lane_tree(s1);
                pv[l + 2] = pv[l + 2] + lane_tree(s2);
                pv[l + 3] = pv[l + 3] + lane_tree(s3);
            }
        }
        for (; l < np; ++l) {
            const double* vl = vs[l].data();
            if (fuse) {
                const double a = us[l][ib];
                for (int64_t j = 0; j < nJ; ++j) rn[j] = rn[j] - a * vl[j];
            }
            pv[l] = lane_dot(vl, v.data(), nJ);
        }
        double cross = 0.0;
        for (size_t l = 0; l < us.size(); ++l) {
            const double pu = lane_dot(us[l].data(), u.data(), nI);
            cross = std::fma(pu, pv[l], cross);
        }
        S2 = S2 + 2.0 * cross + uu * vv;
        if (fuse) {
            const double a = u[ib];
            for (int64_t j = 0; j < nJ; ++j) rn[j] = rn[j] - a * v[j];
        }
        us.emplace_back(u);
        vs.emplace_back(std::move(v));
        out.rows.push_back(int(i));
        out.cols.push_back(int(jb));
        if (std::sqrt(uu) * std::sqrt(vv) <= eps * std::sqrt(std::max(S2, 0.0))) {
            if (first < 0) first = int64_t(out.rows.size());
            if (int64_t(out.rows.size()) - first >= kAcaLookahead) break;
        } else {
            first = -1;
        }
        if (fuse) {
            i = ib;
            std::swap(r, rn);
        } else {
            i = next_free_row();
            if (i < 0) break;
            fresh_row(i, r);
        }
    }
    if (first >= 0) {
        out.rows.resize(size_t(first));
        out.cols.resize(size_t(first));
        if (us.size() > size_t(first)) {
            us.resize(size_t(first));
            vs.resize(size_t(first));
        }
    }
    if (!keep) {
        us.clear();
        vs.clear();
    }
}

// ---------------------------------------------------------------------------
// Dense LU with partial pivoting (row-major n x n, in place) and solves.
bool lu_factor(std::vector<double>& A, int n, std::vector<int>& piv) {
    piv.resize(n);
    for (int k = 0; k < n; ++k) {
        int p = k;
        double best = std::fabs(A[size_t(k) * n + k]);
        for (int i = k + 1; i < n; ++i) {
            const double a = std::fabs(A[size_t(i) * n + k]);
            if (a > best) { best = a; p = i; }
        }
        piv[k] = p;
        if (best == 0.0) return false;
        if (p != k)
            for (int j = 0; j < n; ++j) std::swap(A[size_t(k) * n + j], A[size_t(p) * n + j]);
        const double inv = A[size_t(k) * n + k];
        for (int i = k + 1; i < n; ++i) {
            const double f = A[size_t(i) * n + k] / inv;
            A[size_t(i) * n + k] = f;
            if (f != 0.0)
                for (int j = k + 1; j < n; ++j)
                    A[size_t(i) * n + j] = A[size_t(i) * n + j] - f * A[size_t(k) * n + j];
        }
    }
    return true;
}

void lu_solve(const std::vector<double>& A, int n, const std::vector<int>& piv, double* b) {
    for (int k = 0; k < n; ++k) std::swap(b[k], b[piv[k]]);
    for (int i = 1; i < n; ++i) {
        double s = b[i];
        for (int j = 0; j < i; ++j) s = s - A[size_t(i) * n + j] * b[j];
        b[i] = s;
    }
    for (int i = n - 1; i >= 0; --i) {
        double s = b[i];
        for (int j = i + 1; j < n; ++j) s = s - A[size_t(i) * n + j] * b[j];
        b[i] = s / A[size_t(i) * n + i];
    }
}

// ---------------------------------------------------------------------------
// Pivot selection

// with H2_VERBOSE set: the time of one level of a pivot sweep, on stderr
void level_time(const char* what, int l, std::chrono::steady_clock::time_point t0) {
    static const bool verbose = std::getenv("H2_VERBOSE") != nullptr;
    if (!verbose) return;
    std::fprintf(stderr, "[h2 build]   %s level %2d %8.3f s\n", what, l,
                 std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count());
}

// The ACA problems of one level: sets(X, I, J) fills box X's row set and search
// set; its pivots go to tau[X] (rows) and sig[X] (columns), as tree positions.
// With a device the problems run there (the same pivots) and the host solves
// only those the device hands back; otherwise each runs on the host.
template <class Sets>
std::string level_pivots(Host& H, PivotDevice* dev, int64_t n, double eps, Sets sets,
                         std::vector<std::vector<int64_t>>& tau,
                         std::vector<std::vector<int64_t>>& sig) {
    const Tree& t = H.tree;
    if (!dev) {
#pragma omp parallel for schedule(dynamic, 1)
        for (int64_t X = 0; X < n; ++X) {
            std::vector<int64_t> I, J;
            sets(X, I, J);
            AcaResult R;
            aca(t, H.kern, I, J, eps, false, R);
            for (int a : R.rows) tau[X].push_back(I[a]);
            for (int a : R.cols) sig[X].push_back(J[a]);
        }
        H.piv_problems_host += n;
        return "";
    }
    std::vector<std::vector<int64_t>> Is(n), Js(n);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t X = 0; X < n; ++X) sets(X, Is[X], Js[X]);
    AcaSets S;
    S.Iptr.assign(n + 1, 0);
    S.Jptr.assign(n + 1, 0);
    for (int64_t X = 0; X < n; ++X) {
        S.Iptr[X + 1] = S.Iptr[X] + int64_t(Is[X].size());
        S.Jptr[X + 1] = S.Jptr[X] + int64_t(Js[X].size());
    }
    S.Iidx.resize(size_t(S.Iptr[n]));
    S.Jidx.resize(size_t(S.Jptr[n]));
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t X = 0; X < n; ++X) {
        std::copy(Is[X].begin(), Is[X].end(), S.Iidx.begin() + S.Iptr[X]);
        std::copy(Js[X].begin(), Js[X].end(), S.Jidx.begin() + S.Jptr[X]);
    }
    AcaPivots P;
    const std::string err = pivot_device_level(dev, H.kern, eps, S, P);
    if (!err.empty()) return err;
    int64_t redo = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : redo)
    for (int64_t X = 0; X < n; ++X) {
        if (P.redo[X]) {
            AcaResult R;
            aca(t, H.kern, Is[X], Js[X], eps, false, R);
            for (int a : R.rows) tau[X].push_back(Is[X][a]);
            for (int a : R.cols) sig[X].push_back(Js[X][a]);
            ++redo;
        } else {
            for (int64_t e = P.ptr[X]; e < P.ptr[X + 1]; ++e) {
                tau[X].push_back(Is[X][P.rows[e]]);
                sig[X].push_back(Js[X][P.cols[e]]);
            }
        }
    }
    H.piv_problems_host += redo;
    H.piv_problems_dev += n - redo;
    return "";
}

std::string b2t(Host& H, PivotDevice* dev, Basis& B, const std::vector<Csr>& il, double eps,
                int lmin = 2) {
    const Tree& t = H.tree;
    const int K = t.kappa, d = t.d;
    B.lmin = lmin;
    B.il = &il;
    B.tau.assign(K + 1, {});
    B.sig.assign(K + 1, {});
    for (int l = 0; l <= K; ++l) { B.tau[l].resize(t.nboxes(l)); B.sig[l].resize(t.nboxes(l)); }
    for (int l = K; l >= lmin; --l) {
        const auto tl = std::chrono::steady_clock::now();
        const Csr& L = il[l];
        auto sets = [&](int64_t X, std::vector<int64_t>& I, std::vector<int64_t>& J) {
            if (l == K) {
                for (int64_t p = t.begin(l, X); p < t.end(l, X); ++p) I.push_back(p);
                for (int64_t e = L.ptr[X]; e < L.ptr[X + 1]; ++e) {
                    const int64_t Y = L.idx[e];
                    for (int64_t p = t.begin(l, Y); p < t.end(l, Y); ++p) J.push_back(p);
                }
            } else {
                for (int c = 0; c < (1 << d); ++c) {
                    const auto& tc = B.tau[l + 1][X * (int64_t(1) << d) + c];
                    I.insert(I.end(), tc.begin(), tc.end());
                }
                for (int64_t e = L.ptr[X]; e < L.ptr[X + 1]; ++e) {
                    const int64_t Y = L.idx[e];
                    for (int c = 0; c < (1 << d); ++c) {   // s^{Y_c,o} = t^{Y_c,i}
                        const auto& tc = B.tau[l + 1][Y * (int64_t(1) << d) + c];
                        J.insert(J.end(), tc.begin(), tc.end());
                    }
                }
            }
        };
        const std::string err = level_pivots(H, dev, t.nboxes(l), eps, sets, B.tau[l], B.sig[l]);
        if (!err.empty()) return err;
        level_time("b2t", l, tl);
    }
    return "";
}

std::string t2b(Host& H, PivotDevice* dev, Basis& B, const std::vector<Csr>& il, double eps) {
    const Tree& t = H.tree;
    const int K = t.kappa, d = t.d;
    B.lmin = 1;
    B.il = &il;
    B.tau.assign(K + 1, {});
    B.sig.assign(K + 1, {});
    for (int l = 0; l <= K; ++l) { B.tau[l].resize(t.nboxes(l)); B.sig[l].resize(t.nboxes(l)); }
    for (int l = 1; l <= K; ++l) {
        const auto tl = std::chrono::steady_clock::now();
        const Csr& L = il[l];
        auto sets = [&](int64_t X, std::vector<int64_t>& I, std::vector<int64_t>& J) {
            for (int64_t p = t.begin(l, X); p < t.end(l, X); ++p) I.push_back(p);
            for (int64_t e = L.ptr[X]; e < L.ptr[X + 1]; ++e) {
                const int64_t Y = L.idx[e];
                for (int64_t p = t.begin(l, Y); p < t.end(l, Y); ++p) J.push_back(p);
            }
            if (l > 1) {
                const auto& sp = B.sig[l - 1][X >> d];
                J.insert(J.end(), sp.begin(), sp.end());
            }
        };
        const std::string err = level_pivots(H, dev, t.nboxes(l), eps, sets, B.tau[l], B.sig[l]);
        if (!err.empty()) return err;
        level_time("t2b", l, tl);
    }
    return "";
}

// ---------------------------------------------------------------------------
// Operators (§3.6.4), symmetric reading: U_X = K_{t^X,s^{X,i}} (K_{t^{X,i},s^{X,i}})^{-1},
// L2L U~_{X_c X} = K_{t^{X_c,i}, s^{X,i}} (K_{t^{X,i},s^{X,i}})^{-1}, P2M / M2M their
// transposes, M2L T_{X,Y} = K_{t^{X,i}, t^{Y,i}}.
std::string operators(const Host& H, Basis& B) {
    const Tree& t = H.tree;
    const int K = t.kappa, d = t.d;
    B.U.assign(t.nboxes(K), {});
    B.Ut.assign(K + 1, {});
    B.T.assign(K + 1, {});
    if (K < B.lmin) return "";
    for (int l = 0; l <= K; ++l) { B.Ut[l].resize(t.nboxes(l)); B.T[l].resize(t.nboxes(l)); }
    std::string err;
    for (int l = B.lmin; l <= K; ++l) {
        const int64_t n = t.nboxes(l);
#pragma omp parallel for schedule(dynamic, 4)
        for (int64_t X = 0; X < n; ++X) {
            const auto& tau = B.tau[l][X];
            const auto& sig = B.sig[l][X];
            const int r = int(tau.size());
            // Pt = (K_{tau, sig})^T, factorised once; rows of B A^{-1} solve Pt x = b
            std::vector<double> Pt(size_t(r) * r);
            std::vector<int> piv;
            for (int a = 0; a < r; ++a)
                for (int b = 0; b < r; ++b) Pt[size_t(a) * r + b] = H.kern(t.r2(tau[b], sig[a]));
            if (r > 0 && !lu_factor(Pt, r, piv)) {
#pragma omp critical
                err = "singular pivot matrix";
                continue;
            }
            auto solve_rows = [&](const std::vector<int64_t>& rows, std::vector<double>& out) {
                out.resize(rows.size() * size_t(r));
                for (size_t i = 0; i < rows.size(); ++i) {
                    double* b = out.data() + i * r;
                    for (int a = 0; a < r; ++a) b[a] = H.kern(t.r2(rows[i], sig[a]));
                    lu_solve(Pt, r, piv, b);
                }
            };
            if (l == K) {
                std::vector<int64_t> pts;
                for (int64_t p = t.begin(l, X); p < t.end(l, X); ++p) pts.push_back(p);
                solve_rows(pts, B.U[X]);
            }
            if (l < K)
                for (int c = 0; c < (1 << d); ++c) {
                    const int64_t Xc = X * (int64_t(1) << d) + c;
                    solve_rows(B.tau[l + 1][Xc], B.Ut[l + 1][Xc]);
                }
            // M2L: concatenated T_{X,Y} over Y in the list, r_X x sum r_Y (not
            // formed here when the product evaluates it from the pivots or the
            // device forms it)
            if (H.m2l_fly || H.m2l_dev) continue;
            const Csr& L = (*B.il)[l];
            int64_t kx = 0;
            for (int64_t e = L.ptr[X]; e < L.ptr[X + 1]; ++e) kx += B.rank(l, L.idx[e]);
            auto& T = B.T[l][X];
            T.assign(size_t(r) * kx, 0.0);
            int64_t col = 0;
            for (int64_t e = L.ptr[X]; e < L.ptr[X + 1]; ++e) {
                const auto& ty = B.tau[l][L.idx[e]];
                for (int a = 0; a < r; ++a)
                    for (size_t b = 0; b < ty.size(); ++b)
                        T[size_t(a) * kx + col + b] = H.kern(t.r2(tau[a], ty[b]));
                col += int64_t(ty.size());
            }
        }
    }
    return err;
}

// (H2+H)*: one ACA per vertex-sharing pair with its crosses kept (Algorithm 3);
// all pairs are independent, so with a device they run there as one set of
// problems (the same crosses, bit for bit, as the host's for 1/r and the IMQ)
std::string pure_aca(Host& H, PivotDevice* dev) {
    const Tree& t = H.tree;
    const int K = t.kappa;
    std::vector<std::pair<int, std::pair<int64_t, int64_t>>> pairs;
    for (int l = 1; l <= K; ++l)
        for (int64_t X = 0; X < t.nboxes(l); ++X)
            for (int64_t e = H.lists.ver[l].ptr[X]; e < H.lists.ver[l].ptr[X + 1]; ++e)
                pairs.push_back({l, {X, H.lists.ver[l].idx[e]}});
    const int64_t np = int64_t(pairs.size());
    H.lowrank.assign(np, LowRankBlock());
    auto sets = [&](int64_t p, std::vector<int64_t>& I, std::vector<int64_t>& J) {
        const int l = pairs[p].first;
        const int64_t X = pairs[p].second.first, Y = pairs[p].second.second;
        for (int64_t a = t.begin(l, X); a < t.end(l, X); ++a) I.push_back(a);
        for (int64_t a = t.begin(l, Y); a < t.end(l, Y); ++a) J.push_back(a);
    };
    auto on_host = [&](int64_t p) {
        std::vector<int64_t> I, J;
        sets(p, I, J);
        AcaResult R;
        aca(t, H.kern, I, J, H.eps_ver, true, R);
        LowRankBlock& B = H.lowrank[p];
        B.k = int(R.rows.size());
        B.U.resize(I.size() * size_t(B.k));
        B.V.resize(J.size() * size_t(B.k));
        for (int k = 0; k < B.k; ++k) {
            std::copy(R.us[k].begin(), R.us[k].end(), B.U.begin() + size_t(k) * I.size());
            std::copy(R.vs[k].begin(), R.vs[k].end(), B.V.begin() + size_t(k) * J.size());
        }
    };
    for (int64_t p = 0; p < np; ++p) {
        LowRankBlock& B = H.lowrank[p];
        B.level = pairs[p].first;
        B.X = pairs[p].second.first;
        B.Y = pairs[p].second.second;
    }
    if (!dev) {
#pragma omp parallel for schedule(dynamic, 1)
        for (int64_t p = 0; p < np; ++p) on_host(p);
        H.piv_problems_host += np;
        return "";
    }
    AcaSets S;
    S.Iptr.assign(np + 1, 0);
    S.Jptr.assign(np + 1, 0);
    for (int64_t p = 0; p < np; ++p) {
        const int l = pairs[p].first;
        const int64_t X = pairs[p].second.first, Y = pairs[p].second.second;
        S.Iptr[p + 1] = S.Iptr[p] + (t.end(l, X) - t.begin(l, X));
        S.Jptr[p + 1] = S.Jptr[p] + (t.end(l, Y) - t.begin(l, Y));
    }
    S.Iidx.resize(size_t(S.Iptr[np]));
    S.Jidx.resize(size_t(S.Jptr[np]));
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t p = 0; p < np; ++p) {
        const int l = pairs[p].first;
        const int64_t X = pairs[p].second.first, Y = pairs[p].second.second;
        for (int64_t a = t.begin(l, X); a < t.end(l, X); ++a) S.Iidx[S.Iptr[p] + a - t.begin(l, X)] = int32_t(a);
        for (int64_t a = t.begin(l, Y); a < t.end(l, Y); ++a) S.Jidx[S.Jptr[p] + a - t.begin(l, Y)] = int32_t(a);
    }
    AcaPivots P;
    const std::string err = pivot_device_level(dev, H.kern, H.eps_ver, S, P, true);
    if (!err.empty()) return err;
    int64_t redo = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : redo)
    for (int64_t p = 0; p < np; ++p) {
        if (P.redo[p]) {
            on_host(p);
            ++redo;
            continue;
        }
        LowRankBlock& B = H.lowrank[p];
        const int64_t nI = S.Iptr[p + 1] - S.Iptr[p], nJ = S.Jptr[p + 1] - S.Jptr[p];
        B.k = int(P.ptr[p + 1] - P.ptr[p]);
        const std::vector<double>& f = P.factors[p];
        B.U.assign(f.begin(), f.begin() + size_t(B.k) * size_t(nI));
        B.V.assign(f.begin() + size_t(B.k) * size_t(nI), f.begin() + size_t(B.k) * size_t(nI + nJ));
    }
    H.piv_problems_host += redo;
    H.piv_problems_dev += np - redo;
    return "";
}

// ---------------------------------------------------------------------------
// Packing into the flat level-batched layout read by the kernels.
void pack(Host& H) {
    const Tree& t = H.tree;
    const int K = t.kappa, d = t.d;
    Packed& P = H.packed;
    P.nb = int(H.bases.size());
    // near field stored as leaf block rows unless fp32 (on the fly) or asked otherwise
    P.near_stored = H.near_mode == 2 || (H.near_mode == 0 && H.storage != 1);
    P.box_base.assign(K + 2, 0);
    for (int l = 0; l <= K; ++l) P.box_base[l + 1] = P.box_base[l] + t.nboxes(l);
    P.box_total = P.box_base[K + 1];
    const int64_t ns = P.nb * P.box_total;
    P.rank.assign(ns, 0);
    P.voff.assign(ns, 0);
    P.uoff.assign(ns, -1);
    P.ustride.assign(ns, 0);
    P.utoff.assign(ns, -1);
    P.rank_max = 0;
    auto slot = [&](int b, int l, int64_t X) { return b * P.box_total + P.box_base[l] + X; };
    int64_t vo = 0;
    for (int b = 0; b < P.nb; ++b)
        for (int l = 0; l <= K; ++l)
            for (int64_t X = 0; X < t.nboxes(l); ++X) {
                const int64_t s = slot(b, l, X);
                const int r = (l >= H.bases[b].lmin && l <= K) ? H.bases[b].rank(l, X) : 0;
                P.rank[s] = r;
                P.voff[s] = vo;
                P.rank_max = std::max(P.rank_max, r);
                vo += r;
            }
    P.vlen = vo;
    P.q_base = 0;
    P.v_base = t.N;
    P.u_base = t.N + P.vlen;
    P.phi_base = t.N + 2 * P.vlen;
    P.veclen = 2 * t.N + 2 * P.vlen;
    // ---- first pass: the offset of every block (each block starts on a
    //      multiple of 4 elements), then one allocation and a parallel fill
    int64_t total = 0;
    auto place = [&](int64_t n) {
        const int64_t o = (total + 3) / 4 * 4;
        total = o + n;
        return o;
    };
    auto pad4 = [](int64_t n) { return (n + 3) / 4 * 4; };
    struct Copy { const std::vector<double>* src; int64_t dst; int64_t rows, cols, pad; };
    std::vector<Copy> copies;
    const int64_t nleaf = t.nboxes(K);
    const Csr& NL = (H.variant == 2 || H.variant == 4) ? H.lists.near_sqrt : H.lists.near_star;
    P.near_ptr = NL.ptr;
    P.near_idx = NL.idx;
    // leaf block rows: [ K(t^X, t^X') for X' in N(X) | U_X^b for each basis ]
    P.leaf = RowTasks();
    P.near_entries = 0;
    std::vector<int64_t> leaf_aoff(nleaf, -1), leaf_ncols(nleaf, 0), leaf_kp(nleaf, 0);
    if (P.near_stored) {
        for (int64_t X = 0; X < nleaf; ++X) {
            const int64_t m = t.leaf_ptr[X + 1] - t.leaf_ptr[X];
            int64_t nc = 0;
            for (int64_t e = NL.ptr[X]; e < NL.ptr[X + 1]; ++e)
                nc += t.leaf_ptr[NL.idx[e] + 1] - t.leaf_ptr[NL.idx[e]];
            int64_t cols = nc;
            for (int b = 0; b < P.nb; ++b) cols += P.rank[slot(b, K, X)];
            const int64_t kp = pad4(cols);
            leaf_ncols[X] = nc;
            leaf_kp[X] = kp;
            if (m == 0) continue;
            const int64_t o = place(m * kp);
            leaf_aoff[X] = o;
            P.near_entries += m * nc;
            P.leaf.add(P.phi_base + t.leaf_ptr[X], int32_t(m), int32_t(kp), o);
            for (int64_t e = NL.ptr[X]; e < NL.ptr[X + 1]; ++e) {
                const int64_t Y = NL.idx[e];
                const int64_t my = t.leaf_ptr[Y + 1] - t.leaf_ptr[Y];
                if (my > 0) P.leaf.seg(P.q_base + t.leaf_ptr[Y], int32_t(my));
            }
            int64_t col = nc;
            for (int b = 0; b < P.nb; ++b) {
                const int64_t s = slot(b, K, X);
                if (P.rank[s] > 0) {
                    P.leaf.seg(P.u_base + P.voff[s], P.rank[s]);
                    P.uoff[s] = o + col;
                    P.ustride[s] = int32_t(kp);
                }
                col += P.rank[s];
            }
            P.leaf.close();
        }
    } else {
        for (int b = 0; b < P.nb; ++b) {
            const Basis& B = H.bases[b];
            if (K < B.lmin) continue;
            for (int64_t X = 0; X < nleaf; ++X) {
                const int64_t o = place(int64_t(B.U[X].size()));
                P.uoff[slot(b, K, X)] = o;
                P.ustride[slot(b, K, X)] = B.rank(K, X);
                copies.push_back({&B.U[X], o, 1, int64_t(B.U[X].size()), int64_t(B.U[X].size())});
            }
        }
    }
    // L2L matrices U~_{X_c X}: r_c x pad4(r_X) row-major, one L2L task per child
    // with both ranks > 0
    P.l2l.assign(K + 1, RowTasks());
    for (int b = 0; b < P.nb; ++b) {
        const Basis& B = H.bases[b];
        for (int l = B.lmin + 1; l <= K; ++l)
            for (int64_t X = 0; X < t.nboxes(l); ++X) {
                const int rc = B.rank(l, X), rp = B.rank(l - 1, X >> d);
                const int64_t kp = pad4(rp);
                const int64_t o = place(int64_t(rc) * kp);
                P.utoff[slot(b, l, X)] = o;
                copies.push_back({&B.Ut[l][X], o, rc, rp, kp});
                if (rc > 0 && rp > 0) {
                    const int64_t sp = slot(b, l - 1, X >> d);
                    P.l2l[l].add(P.u_base + P.voff[slot(b, l, X)], rc, int32_t(kp), o);
                    P.l2l[l].seg(P.u_base + P.voff[sp], rp);
                    P.l2l[l].close();
                }
            }
    }
    // P2M and M2M as block rows over transposed copies: v_X = U_X^T q_X at the
    // leaves (r x pad4(m)), v_X = [U~_{X_1 X}^T | ... | U~_{X_2^d X}^T] [v_1; ...]
    // above (r_X x pad4(sum_c r_c)); filled after the allocation.
    struct TBlock { int b, l; int64_t X, o, kp; };
    std::vector<TBlock> tblocks;
    P.p2m = RowTasks();
    P.m2m.assign(K + 1, RowTasks());
    for (int b = 0; b < P.nb; ++b) {
        const Basis& B = H.bases[b];
        if (K < B.lmin) continue;
        for (int64_t X = 0; X < nleaf; ++X) {
            const int r = B.rank(K, X);
            const int64_t m = t.leaf_ptr[X + 1] - t.leaf_ptr[X];
            if (r == 0 || m == 0) continue;
            const int64_t kp = pad4(m);
            const int64_t o = place(int64_t(r) * kp);
            tblocks.push_back({b, K, X, o, kp});
            P.p2m.add(P.v_base + P.voff[slot(b, K, X)], r, int32_t(kp), o);
            P.p2m.seg(P.q_base + t.leaf_ptr[X], int32_t(m));
            P.p2m.close();
        }
        for (int l = B.lmin; l < K; ++l)
            for (int64_t X = 0; X < t.nboxes(l); ++X) {
                const int r = B.rank(l, X);
                int64_t kc = 0;
                for (int c = 0; c < (1 << d); ++c) kc += B.rank(l + 1, X * (int64_t(1) << d) + c);
                if (r == 0 || kc == 0) continue;
                const int64_t kp = pad4(kc);
                const int64_t o = place(int64_t(r) * kp);
                tblocks.push_back({b, l, X, o, kp});
                P.m2m[l].add(P.v_base + P.voff[slot(b, l, X)], r, int32_t(kp), o);
                for (int c = 0; c < (1 << d); ++c) {
                    const int64_t sc = slot(b, l + 1, X * (int64_t(1) << d) + c);
                    if (P.rank[sc] > 0) P.m2m[l].seg(P.v_base + P.voff[sc], P.rank[sc]);
                }
                P.m2m[l].close();
            }
    }
    // M2L: one block row per target, rows padded with zeros to a multiple of 4;
    // blocks formed on the device get offsets in a region of their own, moved
    // past the end of ops once every other block is placed
    P.m2l = RowTasks();
    int64_t m2l_total = 0;
    for (int b = 0; b < P.nb; ++b) {
        const Basis& B = H.bases[b];
        for (int l = B.lmin; l <= K; ++l) {
            const Csr& L = (*B.il)[l];
            for (int64_t X = 0; X < t.nboxes(l); ++X) {
                const int r = B.rank(l, X);
                int64_t kx = 0;
                for (int64_t e = L.ptr[X]; e < L.ptr[X + 1]; ++e) kx += B.rank(l, L.idx[e]);
                if (r == 0 || kx == 0) continue;
                const int64_t kp = pad4(kx);
                if (H.m2l_fly) {
                    P.m2l.add(P.u_base + P.voff[slot(b, l, X)], r, int32_t(kp), 0);
                } else if (H.m2l_dev) {
                    P.m2l.add(P.u_base + P.voff[slot(b, l, X)], r, int32_t(kp), m2l_total);
                    m2l_total += int64_t(r) * kp;          // r * kp is a multiple of 4
                } else {
                    const int64_t o = place(int64_t(r) * kp);
                    P.m2l.add(P.u_base + P.voff[slot(b, l, X)], r, int32_t(kp), o);
                    copies.push_back({&B.T[l][X], o, r, kx, kp});
                }
                for (int64_t e = L.ptr[X]; e < L.ptr[X + 1]; ++e) {
                    const int64_t sy = slot(b, l, L.idx[e]);
                    if (P.rank[sy] > 0) P.m2l.seg(P.v_base + P.voff[sy], P.rank[sy]);
                }
                P.m2l.close();
            }
        }
    }
    if (H.m2l_fly || H.m2l_dev) {
        if (H.m2l_fly) P.m2l.entries = 0;               // nothing stored
        // pivot coordinates in the coefficient layout: slot (b, l, X) holds the
        // incoming pivots t^{X,i} of that cluster, in pivot order
        P.pivot_x.assign(size_t(d) * size_t(P.vlen), 0.0);
        for (int b = 0; b < P.nb; ++b) {
            const Basis& B = H.bases[b];
            for (int l = 0; l <= K; ++l) {
                if (l < B.lmin) continue;
                for (int64_t X = 0; X < t.nboxes(l); ++X) {
                    const auto& tau = B.tau[l][X];
                    const int64_t o = P.voff[slot(b, l, X)];
                    for (size_t a = 0; a < tau.size(); ++a)
                        for (int k = 0; k < d; ++k)
                            P.pivot_x[size_t(k) * P.vlen + o + a] = t.x[size_t(tau[a]) * d + k];
                }
            }
        }
    }
    // (H2+H)* factors grouped by level (blocks of one target stay consecutive)
    P.lr_level_ptr.assign(K + 2, 0);
    P.lr_x0.clear(); P.lr_mx.clear(); P.lr_y0.clear(); P.lr_my.clear();
    P.lr_uoff.clear(); P.lr_voff.clear(); P.lr_toff.clear(); P.lr_k.clear();
    P.lr_tlen = 0;
    {
        std::vector<size_t> order(H.lowrank.size());
        std::iota(order.begin(), order.end(), size_t(0));
        std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) {
            return H.lowrank[a].level < H.lowrank[b].level;
        });
        for (size_t o : order) {
            const LowRankBlock& B = H.lowrank[o];
            P.lr_level_ptr[B.level + 1]++;
            P.lr_x0.push_back(t.begin(B.level, B.X));
            P.lr_mx.push_back(t.end(B.level, B.X) - t.begin(B.level, B.X));
            P.lr_y0.push_back(t.begin(B.level, B.Y));
            P.lr_my.push_back(t.end(B.level, B.Y) - t.begin(B.level, B.Y));
            P.lr_k.push_back(B.k);
            const int64_t ou = place(int64_t(B.U.size()));
            copies.push_back({&B.U, ou, 1, int64_t(B.U.size()), int64_t(B.U.size())});
            P.lr_uoff.push_back(ou);
            const int64_t ov = place(int64_t(B.V.size()));
            copies.push_back({&B.V, ov, 1, int64_t(B.V.size()), int64_t(B.V.size())});
            P.lr_voff.push_back(ov);
            P.lr_toff.push_back(P.lr_tlen);
            P.lr_tlen += B.k;
        }
        for (int l = 0; l <= K; ++l) P.lr_level_ptr[l + 1] += P.lr_level_ptr[l];
    }
    total = (total + 3) / 4 * 4;
    P.m2l_base = total;
    P.m2l_len = H.m2l_dev ? m2l_total : 0;
    if (H.m2l_dev)
        for (int64_t& a : P.m2l.aoff) a += total;
    std::vector<double>().swap(P.ops);
    P.ops.assign(size_t(total), 0.0);     // zero: padding and alignment gaps
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t c = 0; c < int64_t(copies.size()); ++c) {
        const Copy& C = copies[c];
        const double* src = C.src->data();
        double* dst = P.ops.data() + C.dst;
        for (int64_t r = 0; r < C.rows; ++r)
            std::memcpy(dst + r * C.pad, src + r * C.cols, size_t(C.cols) * sizeof(double));
    }
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t k = 0; k < int64_t(tblocks.size()); ++k) {
        const TBlock& T = tblocks[k];
        const Basis& B = H.bases[T.b];
        double* A = P.ops.data() + T.o;
        const int r = B.rank(T.l, T.X);
        if (T.l == K) {                      // U_X^T: A[j][i] = U_X[i][j]
            const int64_t m = t.leaf_ptr[T.X + 1] - t.leaf_ptr[T.X];
            for (int64_t i = 0; i < m; ++i)
                for (int j = 0; j < r; ++j) A[j * T.kp + i] = B.U[T.X][i * r + j];
        } else {                             // U~_c^T blocks side by side
            int64_t col = 0;
            for (int c = 0; c < (1 << d); ++c) {
                const int64_t Xc = T.X * (int64_t(1) << d) + c;
                const int rc = B.rank(T.l + 1, Xc);
                const std::vector<double>& Ut = B.Ut[T.l + 1][Xc];   // rc x r
                for (int i = 0; i < rc; ++i)
                    for (int j = 0; j < r; ++j) A[j * T.kp + col + i] = Ut[size_t(i) * r + j];
                col += rc;
            }
        }
    }
    if (P.near_stored) {
#pragma omp parallel for schedule(dynamic, 8)
        for (int64_t X = 0; X < nleaf; ++X) {
            if (leaf_aoff[X] < 0) continue;
            const int64_t p0 = t.leaf_ptr[X], m = t.leaf_ptr[X + 1] - p0, kp = leaf_kp[X];
            double* A = P.ops.data() + leaf_aoff[X];
            for (int64_t i = 0; i < m; ++i) {
                double* row = A + i * kp;
                int64_t col = 0;
                for (int64_t e = NL.ptr[X]; e < NL.ptr[X + 1]; ++e) {
                    const int64_t Y = NL.idx[e];
                    for (int64_t j = t.leaf_ptr[Y]; j < t.leaf_ptr[Y + 1]; ++j)
                        row[col++] = H.kern(t.r2(p0 + i, j));
                }
                for (int b = 0; b < P.nb; ++b) {
                    const int r = P.rank[slot(b, K, X)];
                    if (r > 0) std::memcpy(row + col, H.bases[b].U[X].data() + i * r, size_t(r) * sizeof(double));
                    col += r;
                }
            }
        }
    }
}

}  // namespace

std::string build_host(Host& H, const double* points, int64_t N, int d, int leaf_size,
                       int kappa_forced, const double* domain_lo, double domain_side,
                       int threads) {
    const auto t0 = std::chrono::steady_clock::now();
    auto tp = t0;
    const bool verbose = std::getenv("H2_VERBOSE") != nullptr;
    auto tick = [&](const char* what) {
        const auto now = std::chrono::steady_clock::now();
        if (verbose)
            std::fprintf(stderr, "[h2 build] %-10s %8.3f s\n", what,
                         std::chrono::duration<double>(now - tp).count());
        tp = now;
    };
    // the thread count applies to this construction only: restored on return
    struct ThreadCount {
        int prev;
        explicit ThreadCount(int n) : prev(omp_get_max_threads()) { if (n > 0) omp_set_num_threads(n); }
        ~ThreadCount() { omp_set_num_threads(prev); }
    } thread_count(threads);
    {
        const std::string e = build_tree(H.tree, points, N, d, leaf_size, kappa_forced, domain_lo,
                                         domain_side);
        if (!e.empty()) return e;
    }
    if (H.tree.kappa > 20 / (d == 2 ? 1 : 1) || H.tree.nboxes(H.tree.kappa) > (int64_t(1) << 24))
        return "tree too deep (more than 2^24 leaves)";
    tick("tree");
    build_lists(H.tree, H.lists);
    tick("lists");
    const auto tpiv = std::chrono::steady_clock::now();
    H.piv_problems_dev = H.piv_problems_host = 0;
    // the pivot search on the device when asked; the handle is closed on every
    // return below
    std::unique_ptr<PivotDevice, void (*)(PivotDevice*)> dev(nullptr, pivot_device_close);
    if (H.pivots_dev) {
        std::string e;
        dev.reset(pivot_device_open(H.tree, e));
        if (!dev) return e;
    }
    std::string perr;
    H.bases.clear();
    if (H.variant == 0 || H.variant == 1) {
        H.bases.emplace_back();
        perr = b2t(H, dev.get(), H.bases.back(), H.lists.far, H.eps_far);
        if (!perr.empty()) return perr;
        H.bases.back().il_kind = 0;
    }
    if (H.variant == 0) {
        H.bases.emplace_back();
        perr = t2b(H, dev.get(), H.bases.back(), H.lists.ver, H.eps_ver);
        if (!perr.empty()) return perr;
        H.bases.back().il_kind = 1;
    }
    if (H.variant == 2) {
        H.bases.emplace_back();
        perr = b2t(H, dev.get(), H.bases.back(), H.lists.sqrtd, H.eps_far);
        if (!perr.empty()) return perr;
        H.bases.back().il_kind = 2;
    }
    if (H.variant == 3 || H.variant == 5) {
        // IL_* = IL_far u IL_ver per box
        H.lists.star.assign(H.tree.kappa + 1, Csr());
        for (int l = 0; l <= H.tree.kappa; ++l) {
            const Csr &F = H.lists.far[l], &V = H.lists.ver[l];
            Csr& S = H.lists.star[l];
            const int64_t n = H.tree.nboxes(l);
            S.ptr.assign(n + 1, 0);
            for (int64_t X = 0; X < n; ++X) {
                // both lists are in ascending key order: merge them
                int64_t a = F.ptr[X], b = V.ptr[X];
                while (a < F.ptr[X + 1] || b < V.ptr[X + 1]) {
                    if (b >= V.ptr[X + 1] || (a < F.ptr[X + 1] && F.idx[a] < V.idx[b])) S.idx.push_back(F.idx[a++]);
                    else S.idx.push_back(V.idx[b++]);
                }
                S.ptr[X + 1] = int64_t(S.idx.size());
            }
        }
        H.bases.emplace_back();
        if (H.variant == 3)   // H2*(t) (App. C): one basis, T2B NCA over the whole IL_*
            perr = t2b(H, dev.get(), H.bases.back(), H.lists.star, H.eps_far);
        else                  // §4.1: B2T NCA over the whole IL_*, levels kappa .. 1
            perr = b2t(H, dev.get(), H.bases.back(), H.lists.star, H.eps_far, 1);
        if (!perr.empty()) return perr;
        H.bases.back().il_kind = 3;
    }
    if (H.variant == 4) {
        // H2_sqrt(d)(t) (App. B): one basis, T2B NCA over the strong-admissibility lists
        H.bases.emplace_back();
        perr = t2b(H, dev.get(), H.bases.back(), H.lists.sqrtd, H.eps_far);
        if (!perr.empty()) return perr;
        H.bases.back().il_kind = 2;
    }
    H.pivot_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - tpiv).count();
    tick("pivots");
    for (Basis& B : H.bases) {
        std::string e = operators(H, B);
        if (!e.empty()) return e;
    }
    if (H.variant == 1) {
        perr = pure_aca(H, dev.get());
        if (!perr.empty()) return perr;
    }
    dev.reset();
    tick("operators");
    pack(H);
    // the packed array now holds every operator: keep only pivots and sizes
    for (Basis& B : H.bases) {
        for (auto& lv : B.T) for (auto& M : lv) { std::vector<double>().swap(M); }
    }
    H.lowrank_entries = 0;
    for (LowRankBlock& B : H.lowrank) {
        H.lowrank_entries += int64_t(B.U.size() + B.V.size());
        std::vector<double>().swap(B.U);
        std::vector<double>().swap(B.V);
    }
    tick("pack");
    // near-field work
    const Tree& t = H.tree;
    const Csr& NL = (H.variant == 2 || H.variant == 4) ? H.lists.near_sqrt : H.lists.near_star;
    H.near_pairs = 0;
    H.near_evals = 0;
    for (int64_t X = 0; X < t.nboxes(t.kappa); ++X)
        for (int64_t e = NL.ptr[X]; e < NL.ptr[X + 1]; ++e) {
            const int64_t Y = NL.idx[e];
            H.near_pairs++;
            H.near_evals += (t.end(t.kappa, X) - t.begin(t.kappa, X)) *
                            (t.end(t.kappa, Y) - t.begin(t.kappa, Y));
        }
    H.build_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return "";
}

}  // namespace h2
