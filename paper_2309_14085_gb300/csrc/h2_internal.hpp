// Internal host-side structures of the H2* library (not part of the C ABI).
#pragma once

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <string>
#include <vector>

namespace h2 {

// G(r) evaluated from r^2 on the host, fp64.  Diagonal / coincident points
// take G's diagonal value: 0 for log r and 1/r (§6.1.1, §6.2.1), 1 for exp(-r)
// and the inverse multiquadric.
struct KernelSpec {
    int kind = 0;
    double param = 0.1;
    double diag() const { return (kind == 0 || kind == 1) ? 0.0 : 1.0; }
    double operator()(double r2) const {
        if (r2 == 0.0) return diag();
        const double r = std::sqrt(r2);
        switch (kind) {
            case 0: return std::log(r);
            case 1: return 1.0 / r;
            case 2: { const double s = r / param; return 1.0 / std::sqrt(1.0 + s * s); }
            default: return std::exp(-r);
        }
    }
};

// 2^d uniform tree (§3.1), points stored in tree order (by leaf key, then by
// user index).  Box keys are bit-interleaved, x fastest.
struct Tree {
    int d = 0, kappa = 0;
    int64_t N = 0;
    double lo[3] = {0, 0, 0};
    double side = 1.0;
    std::vector<int64_t> perm;      // tree position -> user index
    std::vector<int64_t> leaf_ptr;  // 2^(d kappa) + 1 prefix offsets
    std::vector<double> x;          // N x d coordinates in tree order

    int64_t nboxes(int l) const { return int64_t(1) << (d * l); }
    int64_t begin(int l, int64_t key) const { return leaf_ptr[size_t(key << (d * (kappa - l)))]; }
    int64_t end(int l, int64_t key) const { return leaf_ptr[size_t((key + 1) << (d * (kappa - l)))]; }
    double r2(int64_t a, int64_t b) const {   // |x_a - x_b|^2, squares summed in coordinate order
        double s = 0.0;
        for (int k = 0; k < d; ++k) { const double t = x[a * d + k] - x[b * d + k]; s = s + t * t; }
        return s;
    }
};

// Compressed sparse rows: lists of box keys per box of one level.
struct Csr {
    std::vector<int64_t> ptr, idx;
    int64_t size(int64_t X) const { return ptr[X + 1] - ptr[X]; }
};

// Interaction and near-field lists, per level (§3.5 weak, §3.3 strong).
struct Lists {
    std::vector<Csr> far, ver, sqrtd;   // [level]
    std::vector<Csr> star;              // [level] IL_* = IL_far u IL_ver, ascending keys
    Csr near_star, near_sqrt;           // leaf level
};

// One nested basis (far field / vertex-sharing / sqrt(d)).  Pivots are tree
// positions; for symmetric kernels with equal sources and targets the outgoing
// pivots are t^{X,o} = s^{X,i}, s^{X,o} = t^{X,i} and V = U.
struct Basis {
    int lmin = 0;
    int il_kind = 0;                                          // il: 0 far, 1 ver, 2 sqrtd, 3 star
    const std::vector<Csr>* il = nullptr;                    // interaction lists used
    std::vector<std::vector<std::vector<int64_t>>> tau, sig;  // [l][X] t^{X,i}, s^{X,i}
    std::vector<std::vector<double>> U;                       // [leaf] m x r row-major (L2P)
    std::vector<std::vector<std::vector<double>>> Ut;         // [l][X] r_X x r_parent (L2L), l > lmin
    std::vector<std::vector<std::vector<double>>> T;          // [l][X] r_X x sum_Y r_Y (M2L)
    int rank(int l, int64_t X) const { return int(tau[l][X].size()); }
};

// (H2+H)*: one ACA per vertex-sharing pair (Algorithm 3).
struct LowRankBlock {
    int level;
    int64_t X, Y;
    int k;
    std::vector<double> U;   // |t^X| x k, column-major (point index fastest)
    std::vector<double> V;   // |t^Y| x k, column-major
};

// Block-row GEMV tasks: y[dst + i] = sum_k A[aoff + i * kpad + k] x[k], i < rows,
// with x the concatenation of the segments (off, len) of the coefficient buffer.
struct RowTasks {
    std::vector<int64_t> dst, aoff, seg_ptr{0}, seg_off;
    std::vector<int32_t> rows, kpad, seg_len, seg_col;
    int32_t cur_col = 0;
    int32_t kpad_max = 0;
    int64_t entries = 0;       // sum of rows * kpad
    int64_t src_coeffs = 0;    // sum of kpad (coefficients gathered)
    int64_t dst_coeffs = 0;    // sum of rows
    void add(int64_t d, int32_t r, int32_t kp, int64_t a) {
        dst.push_back(d); rows.push_back(r); kpad.push_back(kp); aoff.push_back(a);
        cur_col = 0;
        kpad_max = std::max(kpad_max, kp);
        entries += int64_t(r) * kp;
        src_coeffs += kp;
        dst_coeffs += r;
    }
    void seg(int64_t off, int32_t len) {
        seg_off.push_back(off); seg_len.push_back(len); seg_col.push_back(cur_col);
        cur_col += len;
    }
    void close() { seg_ptr.push_back(int64_t(seg_off.size())); }
    int64_t size() const { return int64_t(dst.size()); }
};

// Device-ready flat layout (all offsets in elements).  The coefficient buffer
// is [ q (N) | v (vlen) | u (vlen) | phi (N) ].
struct Packed {
    int nb = 0;                       // nested bases (1 or 2)
    std::vector<double> pivot_x;      // M2L on the fly or formed on the device: d x vlen
                                      // pivot coordinates, in the v / u coefficient layout
                                      // (coordinate-major)
    int64_t m2l_base = 0;             // M2L formed on the device: its blocks occupy entries
    int64_t m2l_len = 0;              // [m2l_base, m2l_base + m2l_len) of the device array,
                                      // past the end of ops (not held on the host)
    int near_stored = 0;              // 1: near field stored as leaf block rows
    int64_t box_total = 0;            // boxes over levels 0..kappa
    std::vector<int64_t> box_base;    // first box id of each level
    std::vector<int32_t> rank;        // [slot] slot = b * box_total + box_base[l] + X
    std::vector<int64_t> voff;        // [slot] offset of its v / u coefficients
    int64_t vlen = 0;
    int64_t q_base = 0, v_base = 0, u_base = 0, phi_base = 0, veclen = 0;
    std::vector<double> ops;          // every operator entry
    std::vector<int64_t> uoff;        // [slot] leaf basis U row 0 (leaf slots)
    std::vector<int32_t> ustride;     // [slot] distance between rows of U
    std::vector<int64_t> utoff;       // [slot] L2L matrix (child slot), -1 if none
    RowTasks p2m;                     // v_X = U_X^T q_X (transposed copies of the leaf bases)
    std::vector<RowTasks> m2m;        // [parent level] v_X = [U~_c1^T | U~_c2^T | ...] v
    std::vector<RowTasks> l2l;        // [child level] u_c += U~_c u_parent
    RowTasks m2l, leaf;               // M2L targets; stored near field + L2P
    int32_t rank_max = 0;
    int64_t near_entries = 0;         // stored near-field kernel values
    std::vector<int64_t> near_ptr, near_idx;   // per leaf, neighbour leaf keys
    // (H2+H)* vertex-sharing factors: per level, blocks grouped by target X
    std::vector<int64_t> lr_level_ptr;         // [kappa + 2] into the lr_* arrays
    std::vector<int64_t> lr_x0, lr_mx, lr_y0, lr_my, lr_uoff, lr_voff, lr_toff;
    std::vector<int32_t> lr_k;
    int64_t lr_tlen = 0;                       // scratch length for V^T q_Y
};

struct Host {
    KernelSpec kern;
    int pivots_dev = 0;              // 1: B2T / T2B pivot search on the device
    int64_t piv_problems_dev = 0;    // ACA problems the device solved
    int64_t piv_problems_host = 0;   // ACA problems solved on the host
    double pivot_seconds = 0;        // wall time of the pivot phase
    int variant = 0;
    int storage = 0;
    int near_mode = 0;               // 0 default, 1 on the fly, 2 stored
    int tensor_cores = 0;            // fp32 storage: multi-RHS tiles on tcgen05 (tf32)
    int m2l_fly = 0;                 // 1: M2L from pivot coordinates, T not stored
    int m2l_dev = 0;                 // 1: T stored, formed on the device from the pivots
    double eps_far = 0, eps_ver = 0;
    Tree tree;
    Lists lists;
    std::vector<Basis> bases;
    std::vector<LowRankBlock> lowrank;
    Packed packed;
    double build_seconds = 0;
    int64_t near_pairs = 0, near_evals = 0;
    int64_t lowrank_entries = 0;     // stored (H2+H)* factor entries
};

// The option combinations the library builds (storage 0 fp64, 1 fp32, 2
// double-float, 3 bf16; variant 1 = (H2+H)*; near_mode 0 default, 1 on the
// fly, 2 stored; m2l_mode 0 stored, 1 on the fly, 2 formed on the device).
// Returns nullptr when supported, else the reason, with *unsupported = true for
// a combination that is well formed but not built (false: an invalid value).
// h2_build refuses the same combinations that a loaded checkpoint may not hold.
inline const char* combination_error(int storage, int variant, int near_mode, int tensor_cores,
                                     int m2l_mode, bool* unsupported) {
    *unsupported = false;
    if (tensor_cores && storage != 1)
        return "tensor_cores applies to H2_F32 storage (H2_BF16 always uses them)";
    *unsupported = true;
    if (m2l_mode == 1 && storage != 1) return "M2L on the fly is built for fp32 storage";
    if (storage == 3 && near_mode == 1) return "bf16 storage evaluates the near field from stored blocks only";
    if (storage == 2 && near_mode == 1)
        return "df64 storage evaluates the near field from stored blocks only";
    if ((storage == 2 || storage == 3) && variant == 1) return "(H2+H)* is built for fp64 and fp32 storage";
    return nullptr;
}

// The ACA problems of one level of a pivot sweep: problem X has row set
// Iidx[Iptr[X] .. Iptr[X+1]) and search set Jidx[Jptr[X] .. Jptr[X+1]), both
// as tree positions.
struct AcaSets {
    std::vector<int64_t> Iptr{0}, Jptr{0};
    std::vector<int32_t> Iidx, Jidx;
};

// Their pivots: rows[ptr[X] .. ptr[X+1]) are positions into problem X's row
// set, cols the matching positions into its search set; redo[X] = 1 marks a
// problem the device did not finish (more crosses than its workspace holds),
// which the host then solves.  With keep, factors[X] holds the kept crosses:
// U (rank x |I|) then V (rank x |J|), cross-major.
struct AcaPivots {
    std::vector<int64_t> ptr;
    std::vector<int32_t> rows, cols;
    std::vector<char> redo;
    std::vector<std::vector<double>> factors;
};

// Pivot search on the current CUDA device (pivots.cu): the host's ACA, one
// CTA per problem, the same pivots.  open() copies the tree-order
// coordinates; every call blocks until its results are on the host.
struct PivotDevice;
PivotDevice* pivot_device_open(const Tree& t, std::string& err);
void pivot_device_close(PivotDevice* p);
std::string pivot_device_level(PivotDevice* p, const KernelSpec& G, double eps, const AcaSets& S,
                               AcaPivots& out, bool keep = false);

// Construction (build.cpp).  Return "" on success or an error message.
std::string build_host(Host& H, const double* points, int64_t N, int d, int leaf_size,
                       int kappa_forced, const double* domain_lo, double domain_side,
                       int threads);

// Point every basis's list pointer into H's own lists (after a copy or a load).
void relink_lists(Host& H);

// Checkpoint of the whole host state (serialize.cpp).  Return "" on success or
// an error message; load_host checks every offset the device kernels use.
std::string save_host(const Host& H, const char* path);
std::string load_host(Host& H, const char* path);

}  // namespace h2
