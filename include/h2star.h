/*
 * h2star.h -- C ABI of the GB300 (sm_103a) library for the algebraic H2* fast
 * matrix-vector product of Khan & Ambikasaran, "New algebraic fast algorithms
 * for N-body problems in two and three dimensions" (arXiv 2309.14085).
 *
 * The library compresses a kernel matrix K(i,j) = G(|x_i - x_j|) over N points
 * in d = 2 or 3 dimensions (same sources and targets) into
 *   - H2*(b+t)      (§5.1): far-field clusters compressed by B2T NCA (Algorithm 1)
 *                           and vertex-sharing clusters by T2B NCA (Algorithm 2),
 *                           two independent nested bases;
 *   - (H2+H)*       (§5.2): the same far field plus one ACA per vertex-sharing
 *                           pair (Algorithms 3 and 4);
 *   - H2_sqrt(d)(b) (App. A): standard far-field H2, one basis from B2T NCA;
 *   - H2*(t), H2_sqrt(d)(t) (App. C, App. B): one basis from T2B NCA over the
 *                           whole weak / strong admissibility lists;
 * and applies it on the GPU (upward pass, coupling products, downward pass and
 * the near field, §5.1.2).  Solves (GMRES with mixed-precision refinement),
 * batched products over many trees and a continuous-batching solve server sit
 * on top of the same products.
 *
 * Conventions for every entry point:
 *   - the return value is H2_OK (0) or a negative H2_E_* code; the message of
 *     the last failure on the calling thread is h2_last_error();
 *   - no entry point aborts the process or traps on the device;
 *   - "host" pointers are read or written before the call returns; "device"
 *     pointers are accessed asynchronously on the stream passed in, so the
 *     caller keeps them alive until that stream has synchronised;
 *   - a handle is used by one host thread / one stream at a time.
 */
#ifndef H2STAR_H
#define H2STAR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes --------------------------------------------------------- */
#define H2_OK                 0
#define H2_E_INVALID_ARG     -1   /* a size, pointer, enum or option is out of range  */
#define H2_E_OOM             -2   /* host or device allocation failed                 */
#define H2_E_CUDA            -3   /* a CUDA runtime call failed                       */
#define H2_E_NOT_CONVERGED   -4   /* iterative solve stopped at maxit                 */
#define H2_E_UNSUPPORTED     -5   /* valid request this build does not implement      */
#define H2_E_NO_DEVICE       -6   /* no CUDA device, or the handle was built host-only */
#define H2_E_TIMEOUT         -7   /* a bounded device wait expired (the kernel recorded it,
                                     released its resources and returned)              */

/* ---- kernel functions G(r) (diagonal value in brackets) -------------------- */
#define H2_KERNEL_LOG2D       0   /* log r      [0]  single-layer Laplace 2D, §6.1.1   */
#define H2_KERNEL_INVR        1   /* 1 / r      [0]  single-layer Laplace 3D, §6.2.1   */
#define H2_KERNEL_IMQ         2   /* 1/sqrt(1+(r/c)^2) [1], c = kparam (default 0.1)   */
#define H2_KERNEL_MATERN12    3   /* exp(-r)    [1]  Matérn nu = 1/2, App. D           */

/* ---- hierarchical representations ------------------------------------------ */
#define H2_STAR_BT            0   /* H2*(b+t),      §5.1   */
#define H2_PLUS_H_STAR        1   /* (H2+H)*,       §5.2   */
#define H2_SQRTD_B            2   /* H2_sqrt(d)(b), App. A */
#define H2_STAR_T             3   /* H2*(t),        App. C: one basis, T2B NCA over IL_*   */
#define H2_SQRTD_T            4   /* H2_sqrt(d)(t), App. B: one basis, T2B NCA over IL_sqrt */
#define H2_STAR_B             5   /* B2T NCA over the whole IL_* (§4.1): the construction the
                                     paper shows to lose accuracy on vertex-sharing clusters;
                                     built for comparison                                     */

/* ---- operator storage precision ------------------------------------------- */
#define H2_F64                0   /* operators, coefficients and accumulation in fp64 (FP64 pipe) */
#define H2_F32                1   /* operators and near field in fp32, fp32 accumulate          */
#define H2_DF64               2   /* double-float: every fp64 operator entry and coefficient is
                                     kept as a pair of floats (hi + lo, 48-bit significand) and
                                     multiplied / accumulated with error-free transformations
                                     on the FP32 pipe (near field from stored blocks)           */
#define H2_BF16               3   /* operators and near-field blocks stored in bfloat16, fp32
                                     coefficients; RHS tiles of 16-64 columns run on the tensor
                                     cores (tcgen05, bf16 x bf16 -> fp32 accumulate: the
                                     coefficients are rounded to bf16 as MMA inputs), narrower
                                     tiles on the CUDA cores (fp32 multiply-add)             */

/* Optional build settings; pass NULL for all defaults.  Zero-initialise and
 * set the fields you need: every zero field means "default". */
typedef struct {
    double eps_far;        /* NCA tolerance for the far field (default: tol)           */
    double eps_ver;        /* tolerance for vertex-sharing clusters (default: tol)     */
    int    storage;        /* H2_F64 (default), H2_F32, H2_DF64 or H2_BF16             */
    int    kappa;          /* leaf level; 0 = smallest kappa with leaf_size 2^(d kappa) >= N
                              (§3.1); a positive value forces that depth; -1 = the
                              strict reading of §3.1: from that depth on, the first
                              at which every leaf holds at most leaf_size points
                              (H2_E_INVALID_ARG if none up to 2^24 leaves does,
                              e.g. more than leaf_size coincident points)         */
    int    use_domain;     /* 1: use domain_lo / domain_side as the root hyper-cube C  */
    double domain_lo[3];   /*    lower corner of C                                    */
    double domain_side;    /*    edge length of C; default C = tight bounding cube    */
    int    threads;        /* host threads for the construction (default: all)        */
    int    host_only;      /* 1: build the host representation only (no device use);
                              h2_info / h2_get_pivots work, h2_matvec returns
                              H2_E_NO_DEVICE                                        */
    double kparam;         /* kernel parameter (IMQ c; default 0.1)                    */
    int    near_mode;      /* near field: 0 default (stored blocks for H2_F64 / H2_DF64,
                              on the fly from the coordinates for H2_F32), 1 on the fly,
                              2 stored kernel blocks (with L2P fused into them)       */
    int    tensor_cores;   /* H2_F32 only: 1 = RHS tiles of 16-64 columns run on the
                              tensor cores in tf32 (10-bit significand multiplies,
                              fp32 accumulate); 0 (default) = fp32 CUDA-core FMA     */
    int    m2l_mode;       /* the coupling blocks T_{X,Y} = G(t^{X,i}, t^{Y,i}) (§3.6.4):
                              0 (default) = stored, formed on the host and uploaded;
                              1 (H2_F32 only) = evaluated in each product from the
                              pivot coordinates, not stored; 2 = stored, formed on
                              the device from the pivot coordinates (fp64 entries,
                              each rounded once to the storage; the host never holds
                              them, so host_only handles of this mode have no M2L
                              values and batches refuse them)                        */
    int    pivots;         /* where the B2T / T2B pivot search runs (ACA of §3.6 inside
                              Algorithm 1 and §5.1.1): 0 (default) = the current CUDA
                              device for 1/r and the IMQ unless host_only is set,
                              else host threads; 1 = the device; 2 = host threads.  The device runs every
                              ACA problem of a level together (one CTA per 4096-entry
                              segment of a search set) with the host's operations in
                              the host's order: the same pivots for 1/r and the IMQ
                              (log r and exp(-r) use the device's log / exp and may
                              differ in the last bit); a problem needing more than
                              1024 crosses is solved on the host.  The (H2+H)* ACA
                              blocks (Algorithm 3) go the same way.  1 with
                              host_only is an error.                                */
} h2_build_opts;

typedef struct h2_handle_s* h2_handle;

/*
 * h2_build -- construct the hierarchical representation (once per geometry).
 *
 *   points     host, N x d row-major fp64 coordinates; copied, not retained.
 *   N, d       N >= 1 points, d = 2 or 3.
 *   kernel     H2_KERNEL_*.
 *   leaf_size  n_max of §3.1 (>= 1): the tree depth kappa is the smallest with
 *              leaf_size * 2^(d kappa) >= N unless opts->kappa forces it.
 *   tol        ACA / NCA tolerance eps of §3.6 (> 0, < 1), used for eps_far
 *              and eps_ver unless opts sets them (§6 uses eps = eps_far = eps_ver).
 *   variant    H2_STAR_BT, H2_PLUS_H_STAR, H2_SQRTD_B, H2_STAR_T, H2_SQRTD_T or
 *              H2_STAR_B.
 *   opts       NULL or build options (above).
 *   out        receives the handle (owns all host and device memory).
 *
 * The tree (§3.1), the interaction lists (§3.5 / §3.3), the pivots (B2T NCA
 * Algorithm 1, T2B NCA §5.1.1, ACA §3.6) and the operators (§3.6.4) are built
 * on the host with OpenMP (the pivot search on the device with opts->pivots); the operators are then packed per level and copied
 * to the current CUDA device (synchronously, on the legacy default stream),
 * where m2l_mode 2 forms the coupling blocks instead of copying them.
 * Errors: H2_E_INVALID_ARG, H2_E_UNSUPPORTED (an option this storage or
 * variant does not implement, e.g. m2l_mode 1 without H2_F32, on-the-fly near
 * field in H2_DF64 / H2_BF16, (H2+H)* in H2_DF64 / H2_BF16), H2_E_OOM,
 * H2_E_CUDA, H2_E_NO_DEVICE.
 */
int h2_build(const double* points, int64_t N, int d, int kernel, int leaf_size,
             double tol, int variant, const h2_build_opts* opts, h2_handle* out);

/*
 * h2_release_host -- free the host copy of the packed operators of a handle
 * that is on the device (the largest host allocation: every stored operator
 * entry in fp64).  Products, solves, servers and batches keep working from the
 * device copy; h2_convert from this handle then returns H2_E_UNSUPPORTED.
 * Errors: H2_E_INVALID_ARG (NULL, host-only or served handle).
 */
int h2_release_host(h2_handle h);

/*
 * h2_convert -- a second device copy of the same compressed operator in another
 * storage precision, without repeating the construction: the tree, lists,
 * pivots and packed operators of `src` are copied on the host and uploaded in
 * `storage` (H2_F64, H2_F32 or H2_DF64) to the current CUDA device.  The result
 * is an independent handle (h2_destroy it separately); its products equal those
 * of a handle built by h2_build with the same arguments, this storage and
 * near_mode 2 (src stores its near-field blocks) or 1 (src evaluates them on
 * the fly).  Mixed-precision solves pair the two: h2_gmres(converted fp32,
 * fp64 src, ...), or a server with residual handles.
 * Errors: H2_E_INVALID_ARG, H2_E_UNSUPPORTED (H2_DF64 from a source without
 * stored near-field blocks, or from (H2+H)*), H2_E_OOM, H2_E_CUDA,
 * H2_E_NO_DEVICE.
 */
int h2_convert(h2_handle src, int storage, h2_handle* out);

/*
 * h2_save / h2_load -- checkpoint of a constructed representation (the paper
 * has no counterpart; construction dominates its run times).  h2_save writes
 * the handle's whole host state -- tree, interaction lists, pivots, operators
 * and the packed device layout, with its kernel, variant, storage and modes --
 * to the file `path` (host; native little-endian, 64-bit sizes).  h2_load reads
 * it into a new handle: host-only if host_only = 1, else uploaded to the
 * current CUDA device in the saved storage, with the same products as the
 * saved handle's; M2L blocks formed on the device (m2l_mode 2) are formed again
 * there.  A loaded file is bounds-checked field by field (every length against
 * the bytes left), its trailing 64-bit checksum is compared, and the state is
 * checked index by index against the buffers the device kernels address, so a
 * truncated or corrupted file is an error, never an out-of-range access.
 * Errors: H2_E_INVALID_ARG (NULL argument, file not readable or writable, not
 * a checkpoint, truncated or inconsistent), H2_E_UNSUPPORTED (h2_save of a
 * handle whose host operators were released), H2_E_OOM, H2_E_NO_DEVICE,
 * H2_E_CUDA.
 */
int h2_save(h2_handle h, const char* path);
int h2_load(const char* path, int host_only, h2_handle* out);

/*
 * h2_matvec -- Y = K~ X for nrhs right-hand sides (§5.1.2 / §5.2.2 / App. A.2,
 * App. B.2 and App. C.2 for the T2B-only variants).
 *
 *   X      device, fp64, column-major N x nrhs with leading dimension ldx >= N,
 *          rows in the user's point order (the order of `points`).
 *   Y      device, fp64, column-major N x nrhs, leading dimension ldy >= N;
 *          overwritten.  X and Y must not overlap.
 *   nrhs   1 <= nrhs <= 64.
 *   stream cudaStream_t (NULL = legacy default stream); the call is asynchronous.
 *
 * Every step runs in this library's CUDA kernels: gather into tree order,
 * P2M, M2M, M2L (far and vertex-sharing), L2L, L2P fused with the near field
 * (evaluated on the fly from the coordinates, or from stored kernel blocks,
 * per h2_build_opts.near_mode), scatter back; with h2_build_opts.m2l_mode = 1
 * the M2L blocks are evaluated from the pivot coordinates.  Precision follows
 * the build's storage (H2_F64, H2_F32, H2_DF64 or H2_BF16); RHS tiles of 16-64
 * columns run on the tensor cores for H2_BF16 and for H2_F32 built with
 * tensor_cores = 1.  Each column of a multi-RHS product equals the single-RHS
 * product of that column bit for bit, except columns run on the tensor cores.
 * Errors: H2_E_INVALID_ARG (also: the handle serves a solve server),
 * H2_E_NO_DEVICE (host-only handle), H2_E_CUDA, H2_E_TIMEOUT (a tensor-core
 * product of an earlier call gave up waiting for its MMAs: every later call on
 * the handle returns it).
 */
int h2_matvec(h2_handle h, const double* X, int64_t ldx, double* Y, int64_t ldy,
              int nrhs, void* stream);

/* Construction statistics and the per-MVP work, filled by h2_info. */
typedef struct {
    int64_t N;
    int     d, kappa, kernel, variant, storage, nbases;
    int     rank_min[2][32], rank_max[2][32];   /* [basis][level]; basis 0 far, 1 ver   */
    double  rank_avg[2][32];
    int64_t m2l_pairs[2];          /* stored M2L blocks per basis                          */
    int64_t near_pairs;            /* (leaf, neighbour leaf) near-field blocks            */
    int64_t near_evals;            /* kernel evaluations per RHS in the near field         */
    int64_t lowrank_pairs;         /* (H2+H)*: vertex-sharing ACA blocks                   */
    int64_t bytes_basis;           /* stored leaf bases U_X (read by P2M and L2P)          */
    int64_t bytes_transfer;        /* stored L2L / M2M transfer matrices                   */
    int64_t bytes_m2l;             /* stored M2L coupling matrices (rows padded to 4)      */
    int64_t m2l_src_coeffs;        /* M2L: source coefficients gathered, summed over targets */
    int64_t m2l_dst_coeffs;        /* M2L: target coefficients written                     */
    int64_t vlen;                  /* multipole (= local) coefficients over all clusters   */
    int64_t bytes_leaf_rows;       /* stored near-field blocks + fused leaf bases (0 when
                                      the near field is evaluated on the fly)               */
    int64_t leaf_src_coeffs;       /* leaf block rows: coefficients gathered, summed        */
    int     near_stored;           /* 1: near field from stored blocks, 0: on the fly      */
    int     rw_m2l, rw_leaf;       /* rows per warp the build-time autotuner chose          */
    int64_t bytes_lowrank;         /* stored (H2+H)* U, V factors                          */
    int64_t bytes_device;          /* total device bytes held by the handle                */
    int64_t alg_bytes_per_rhs;     /* algorithmic HBM bytes of one MVP with one RHS      */
    double  build_seconds;         /* host construction wall time                          */
    int     tc_blocks[3];          /* tensor-core products: persistent CTAs per launch for
                                      RHS tiles of 64 / 32 / 16 (0: no tensor cores)     */
    int     tc_occupancy[3];       /* the runtime's resident-CTA estimate per SM (report) */
    int     m2l_fly;               /* the build's m2l_mode: 0 stored (host-formed), 1 M2L
                                      evaluated from pivot coordinates, 2 stored
                                      (device-formed)                                    */
    int64_t m2l_entries;           /* entries of all T_{X,Y} (sum of rows x columns)     */
    int64_t pivot_problems_device; /* ACA problems solved on the device: the B2T / T2B pivot
                                      search and the (H2+H)* blocks of Algorithm 3       */
    int64_t pivot_problems_host;   /* ... and on the host                                  */
    double  pivot_seconds;         /* wall time of the pivot search (part of build_seconds) */
} h2_stats;

/* h2_info -- fill *st (host).  Errors: H2_E_INVALID_ARG. */
int h2_info(h2_handle h, h2_stats* st);

/*
 * h2_get_pivots -- the incoming pivots t^{X,i} (rows) and s^{X,i} (columns) of
 * cluster `box` (bit-interleaved key) at `level` in basis `basis` (0 far /
 * sqrt(d), 1 vertex-sharing), as user point indices in selection order.
 * ti and si are host arrays of capacity `cap`; *rank receives the count.
 * The outgoing pivots are t^{X,o} = s^{X,i}, s^{X,o} = t^{X,i} (symmetric
 * kernels, same sources and targets).  Errors: H2_E_INVALID_ARG (also when
 * cap < rank; *rank is still set).
 */
int h2_get_pivots(h2_handle h, int basis, int level, int64_t box, int64_t* ti,
                  int64_t* si, int64_t cap, int* rank);

/* h2_tree_order -- the permutation from tree order to user order: perm[i] is
 * the user index of the i-th point in tree order (host array of N).  */
int h2_tree_order(h2_handle h, int64_t* perm);

/*
 * h2_profile -- turn per-stage timing of h2_matvec on (1) or off (0) and reset
 * the accumulated times and the launch counter.  While on, h2_matvec records
 * CUDA events between its stages on the caller's stream (no host wait, except
 * one read-back of the recorded events every 4096 pipeline runs).
 * Errors: H2_E_INVALID_ARG.
 *
 * h2_stage_times -- accumulated milliseconds per stage since the last
 * h2_profile call (waits for the recorded events): ms[0..7] = gather, P2M,
 * M2M, M2L, L2L, leaf (L2P + near field), (H2+H)* low-rank, scatter;
 * *calls = single-RHS pipeline runs timed; *launches = CUDA kernels launched
 * by h2_matvec since the last h2_profile call (calls and launches nullable).
 * ms is a host array with cap >= 8.  Errors: H2_E_INVALID_ARG, H2_E_CUDA.
 */
int h2_profile(h2_handle h, int enable);
int h2_stage_times(h2_handle h, double* ms, int cap, int64_t* calls, int64_t* launches);

/* Result of a solve, filled by h2_gmres. */
typedef struct {
    int     converged;         /* 1 if the relative residual reached rtol              */
    int     iterations;        /* GMRES iterations (Arnoldi steps), all cycles         */
    int     restarts;          /* restarts of GMRES(restart)                           */
    int     refinements;       /* outer iterative-refinement steps (0 without h_res)   */
    int64_t matvecs;           /* products with the solver's handle                    */
    int64_t matvecs_residual;  /* products with the residual handle                    */
    double  rel_residual;      /* ||b - A x||_2 / ||b||_2, recomputed in fp64 at exit  */
    double  rel_residual_est;  /* the last GMRES least-squares estimate                */
    double  seconds;           /* wall time of the call (it synchronises the stream)   */
    int     fallback;          /* 1 if refinement stopped contracting and the solve was
                                  finished by fp64 GMRES on h_res                        */
    int     pad_;
} h2_gmres_stats;

/*
 * h2_gmres -- solve (shift I + scale K~) x = b in fp64 on the device.
 *
 * §6 solves the discretised integral equations and RBF systems with GMRES,
 * the matrix-vector product accelerated by the hierarchical representation,
 * stopped when the relative residual ||b - A x|| / ||b|| drops below
 * eps_GMRES.  Here: restarted GMRES(restart) (restart >= maxit gives the
 * unrestarted method), x0 = 0, classical Gram-Schmidt applied twice, Givens
 * rotations; the Krylov basis (N x (restart + 1) doubles) is kept in the
 * handle for later solves.
 *
 *   h      handle whose product the GMRES iterations use (any storage).
 *   h_res  NULL, or a second handle on the same points and device (e.g.
 *          fp64 storage when h is fp32): then the solve is an iterative
 *          refinement -- residuals r = b - A x are recomputed in fp64 with
 *          h_res, each correction comes from GMRES on h -- so it reaches an
 *          fp64 tolerance while the iterations use the faster product.  A
 *          correction that does not halve the fp64 residual (h too coarse for
 *          this system: its error exceeds the smallest singular value) is
 *          undone, and GMRES on h_res finishes the solve (st->fallback = 1).
 *   b, x   device, fp64, N entries in user order (x overwritten).
 *   rtol   relative residual target in (0, 1); restart in [1, 1000]; maxit >= 1
 *          bounds the GMRES iterations over all cycles and refinements.
 *   st     nullable; filled also on H2_E_NOT_CONVERGED (x then holds the last
 *          iterate).  The call synchronises `stream`.
 * Errors: H2_E_INVALID_ARG, H2_E_NO_DEVICE, H2_E_OOM, H2_E_CUDA, H2_E_NOT_CONVERGED,
 * H2_E_TIMEOUT (as for h2_matvec, for h or h_res).
 */
int h2_gmres(h2_handle h, h2_handle h_res, double shift, double scale, const double* b,
             double* x, double rtol, int restart, int maxit, h2_gmres_stats* st, void* stream);

/*
 * h2_matvec_noalloc -- y = K~ x for one right-hand side, without any device
 * allocation (the paper has no counterpart; this is a deployment entry point).
 *
 * For callers that cannot call cudaMalloc while products run -- a serving
 * process that reserved its whole device memory budget up front, or code
 * recording work into a CUDA graph -- the product's scratch (charges,
 * multipole / local coefficients and potentials in tree order) comes from one
 * static device array of 32 MiB that every GPU loading this library holds
 * until exit, instead of the handle's own buffer.  The handle (built by
 * h2_build on the current device) still supplies the operators.
 *
 *   x, y   device, fp64, N entries in user point order (y overwritten).
 *   stream cudaStream_t (NULL = legacy default stream); asynchronous.
 *
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  Every call shares the one array and the call
 * clears what must start at zero, so calls that overlap on the GPU (other
 * streams, other handles, other host threads) race: serialise them.  While
 * the call runs on the host it points the handle's own scratch at the array,
 * so no other call may use the same handle from another host thread meanwhile.
 * Errors: H2_E_INVALID_ARG (NULL pointers, wrong current device, or a handle
 * whose scratch exceeds 32 MiB -- the message states both sizes),
 * H2_E_NO_DEVICE, H2_E_CUDA.
 */
int h2_matvec_noalloc(h2_handle h, const double* x, double* y, void* stream);

/*
 * h2_inject_wait_expiry -- failure injection without a GPU fault (the paper
 * has no counterpart).  Every mbarrier wait of the tensor-core products is
 * bounded: on expiry the kernel records it in the handle's device error flag,
 * lets its MMAs in flight finish, frees its TMEM and returns, and the host
 * reports H2_E_TIMEOUT.  This call runs that path on demand: one warp
 * allocates TMEM, waits at most `rounds` try_wait rounds (0 <= rounds <= 2^22)
 * on an mbarrier that nothing arrives on, sets the flag, frees its TMEM and
 * returns; the flag is then read back on `stream` (asynchronous).  Once the
 * stream has reached that point, every product on h (h2_matvec,
 * h2_matvec_noalloc, h2_gmres, a solve server's products) returns
 * H2_E_TIMEOUT; the device context and other handles stay usable.
 * Errors: H2_E_INVALID_ARG (NULL handle, rounds out of range, a handle that
 * serves a solve server), H2_E_NO_DEVICE, H2_E_UNSUPPORTED (the handle runs no
 * tensor-core products: storage other than H2_BF16 and H2_F32 with
 * tensor_cores), H2_E_CUDA.
 */
int h2_inject_wait_expiry(h2_handle h, int64_t rounds, void* stream);

/* ---- batched products over many independent trees ------------------------ */
typedef struct h2_batch_s* h2_batch;

typedef struct {
    int     instances, virtual_instances;   /* handles; (handle, RHS column) pairs      */
    int64_t points_times_rhs;               /* sum over instances of N * nrhs          */
    int64_t launches_per_product;           /* kernels in the captured product graph   */
    int     m2m_steps, l2l_steps;           /* level-synchronous launch steps          */
    int64_t m2l_tasks, leaf_tasks;          /* merged block-row tasks                  */
    int64_t bytes_device, bytes_ops;        /* device memory; of it, operator entries  */
} h2_batch_stats;

/*
 * h2_batch_create -- merge n handles (any mix of N, d, kernel and depth; one
 * storage; stored near field, h2_build_opts.near_mode = 2; H2*(b+t) or
 * H2_sqrt(d)(b)) into one device layout for batched products.  Operators are
 * copied from the device copy of handles on the device (their host copy may be
 * released) and from the host copy of host-only handles, into one operator
 * array.  nrhs[i] in [1, 64] (NULL = all 1) is instance i's column count.
 * Every (instance, tile of up to 4 columns in fp32 / 2 in fp64 and df64) pair
 * becomes a virtual instance with its own coefficients (the tile's operators
 * are streamed once for all its columns); the tasks of all of them are merged
 * so one product is ~2 kappa_max
 * + 4 launches (P2M, M2M bottom-up and L2L top-down in level-synchronous steps,
 * one M2L launch, one leaf launch, gather and scatter), captured once into a
 * CUDA graph.  The handles may be destroyed afterwards.
 * Errors: H2_E_INVALID_ARG, H2_E_UNSUPPORTED, H2_E_OOM, H2_E_CUDA.
 */
int h2_batch_create(const h2_handle* hs, int n, const int* nrhs, h2_batch* out);

/*
 * h2_batch_matvec -- Y[i] = K~_i X[i] for every instance i, replaying the graph.
 * X[i], Y[i]: device, fp64, column-major N_i x nrhs[i] (leading dimension N_i),
 * user point order; the host arrays X, Y of n pointers are read before the call
 * returns.  Ordered after prior work on `stream`; later work on `stream` waits
 * for it.  One product at a time per batch.  Errors: H2_E_INVALID_ARG, H2_E_CUDA.
 */
int h2_batch_matvec(h2_batch b, const double* const* X, double* const* Y, void* stream);

/* h2_batch_info -- fill *st (host).  Errors: H2_E_INVALID_ARG. */
int h2_batch_info(h2_batch b, h2_batch_stats* st);

/* h2_batch_destroy -- release the batch (NULL is ignored); synchronises the device. */
void h2_batch_destroy(h2_batch b);

/* ---- served solves: a continuous-batching GMRES server --------------------- */
typedef struct h2_server_s* h2_server;

typedef struct {
    int64_t workspace_bytes;   /* device budget for request workspaces (admission by HBM
                                  footprint); 0 = max_active requests of the largest N  */
    int     restart;           /* GMRES(restart) per request (default 50)               */
    int     max_active;        /* requests iterated together at most (default 16)       */
    int     inner_policy;      /* with res_geoms: 0 = the measured admission rule below,
                                  1 = every request starts on geoms[g] (guard only)     */
    int     pad_;
} h2_server_opts;

typedef struct {
    int64_t submitted, admitted, completed, queued, active, max_active;
    int64_t ticks;             /* GMRES steps of the whole active set                  */
    int64_t products;          /* multi-RHS products (one per geometry per tick)       */
    int64_t product_columns;   /* request vectors those products carried               */
    int64_t workspace_bytes;
} h2_server_stats;

typedef struct {
    int    converged, iterations, restarts;
    int    op;                 /* Arnoldi operator: 0 geoms[g] throughout; 1 res_geoms[g]
                                  (geoms[g] error > |shift| / 10 for this request);
                                  2 res_geoms[g] after a geoms[g] cycle that did not halve
                                  the fp64 residual (that cycle is undone)              */
    double rel_residual;       /* ||f - A x|| / ||f||, recomputed at the end            */
    double queue_seconds;      /* submit -> admission                                   */
    double latency_seconds;    /* submit -> solution ready                              */
} h2_request_stats;

/*
 * h2_server_create -- start a solve server over resident geometries (handles
 * built by h2_build or h2_convert on the current device; they stay owned by
 * the caller and must outlive the server).  The server takes the handles for
 * its lifetime: h2_matvec, h2_matvec_noalloc, h2_gmres and another server
 * refuse them (H2_E_INVALID_ARG) until h2_server_destroy, and one handle may
 * not serve two geometry slots (each has one coefficient buffer).  One worker
 * thread iterates all admitted requests together: each tick performs one
 * GMRES step (fp64 vectors, classical Gram-Schmidt twice) for every active
 * request, the products of the requests on one geometry running as a single
 * multi-RHS h2 product and different geometries on their own CUDA streams, so
 * their work overlaps on the device.  Requests that arrive while others run
 * join at the next tick once their Krylov workspace ((restart + 1 + 4) N
 * doubles) fits the budget and a slot is free (first come, first served).
 *
 *   geoms      host array of ngeom handles: the operators of the Arnoldi
 *              products.
 *   res_geoms  NULL, or host array of ngeom handles of the same geometries
 *              (same N and point order, e.g. the fp64 source of an fp32
 *              h2_convert copy; an entry may equal geoms[g]).  The residual
 *              f - A x that starts every GMRES cycle and the final residual
 *              then use res_geoms[g], so a request on an fp32 geometry reaches
 *              an fp64 tolerance by iterative refinement: each cycle solves
 *              for the correction until its own residual has dropped by 1e-5
 *              (fp32; 1e-10 for other storage) or to rtol ||f||.  Two guards
 *              keep every request convergent: at creation the server measures
 *              delta_g = ||(K_geoms - K_res) v|| / ||v|| on one seeded random
 *              vector, and (inner_policy 0) a request with shift != 0 and
 *              delta_g |scale| > |shift| / 10 iterates on res_geoms[g] from the
 *              start; a cycle on geoms[g] that does not halve the fp64 residual
 *              is undone and the request continues on res_geoms[g]
 *              (h2_request_stats.op tells which happened).
 * Errors: H2_E_INVALID_ARG, H2_E_OOM, H2_E_CUDA.
 */
int h2_server_create(const h2_handle* geoms, const h2_handle* res_geoms, int ngeom,
                     const h2_server_opts* opts, h2_server* out);

/*
 * h2_server_submit -- queue a solve of (shift I + scale K~_geom) x = f to relative
 * residual rtol within maxit iterations.  f: host, N fp64 in user order, copied
 * before the call returns.  *ticket identifies the request.  Non-blocking.
 * Errors: H2_E_INVALID_ARG, H2_E_OOM (workspace larger than the whole budget),
 * H2_E_CUDA or H2_E_TIMEOUT (the server stopped after that device error).
 */
int h2_server_submit(h2_server s, int geom, double shift, double scale, const double* f,
                     double rtol, int maxit, int64_t* ticket);

/*
 * h2_server_wait -- block until the request is done; x (host, N, nullable)
 * receives the solution and st (nullable) its statistics.  Each ticket is
 * waited for once.  Returns H2_E_NOT_CONVERGED (x and st still filled) when
 * maxit ran out, and the error of a product that stopped the request
 * (H2_E_CUDA, H2_E_TIMEOUT; st->converged = 0).  Errors: H2_E_INVALID_ARG
 * (unknown ticket).
 */
int h2_server_wait(h2_server s, int64_t ticket, double* x, h2_request_stats* st);

/* h2_server_stats_get -- counters of the server (host).  Errors: H2_E_INVALID_ARG. */
int h2_server_stats_get(h2_server s, h2_server_stats* st);

/* h2_server_destroy -- drop queued requests, finish the active ones, stop the worker. */
void h2_server_destroy(h2_server s);

/* h2_last_error -- message of the last failure on this thread ("" if none). */
const char* h2_last_error(void);

/* h2_destroy -- release the handle and all its memory (NULL is ignored).
 * Synchronises the device first so no MVP on the handle is still running. */
void h2_destroy(h2_handle h);

#ifdef __cplusplus
}
#endif
#endif /* H2STAR_H */
