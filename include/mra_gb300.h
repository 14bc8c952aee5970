/*
 * mra_gb300.h -- C ABI of the GB300 (sm_103a) adaptive non-standard-form apply.
 *
 * The library applies a radial-kernel operator T with kernel
 * K_{mu,alpha}(r) (the kernel of (-Laplacian + mu^2)^{-alpha}) to a function f
 * on B = [0,1]^3 stored as an adaptive tree of Legendre-multiwavelet scaling
 * blocks, following Beylkin, Cheruvu and Perez, "Fast Adaptive Algorithms in the
 * Non-Standard Form for Multidimensional Problems":
 *   - the kernel is a weighted sum of Gaussians (Sec. 3, eqs. IntegralRepr and
 *     KernelApproxByGaussians);
 *   - the operator is applied in the modified non-standard form scale by scale
 *     (Sec. 2.3, eq. apply_algo; Algorithm 3), with the separated 1-D blocks
 *     F^{j;m,l} (eq. KernelFactor) and norm-based screening (Sec. 4);
 *   - the per-scale outputs are assembled by eq. g_assemble and truncated.
 *
 * Conventions shared by every entry point
 *   - Every call returns an int status: MRA_OK (0) or one of the codes below.
 *     mra_last_error() returns a static, NUL-terminated message for the last
 *     failure on the calling thread.
 *   - Pointers named *_host point to host memory; all other array pointers are
 *     device memory.  `stream` is a cudaStream_t passed as void* (NULL = the
 *     legacy default stream).  Work is queued on that stream; calls return when
 *     queued unless stated otherwise ("synchronous").
 *   - Handles (mra_tree*, mra_op*, mra_plan*, mra_mlp*) are owned by the
 *     library, opaque, and freed exactly once with mra_free() (or the typed
 *     free of their kind).  Output handles are set to NULL on failure, and a
 *     failing call releases every device block it took before it returns.
 *   - Device memory comes from the optional allocator hook (mra_alloc); when the
 *     hook is NULL the library uses cudaMallocAsync / cudaFreeAsync on `stream`.
 *     Blocks the library frees are kept (up to 4 GiB) for reuse by later calls
 *     with the same hook, stream and size, and go back to the hook only through
 *     mra_release_cached(): a hook must stay valid until then.  A handle takes
 *     and returns its blocks in the order of the stream it was created on: a
 *     call that queues work on another stream must be ordered with that stream
 *     by the caller (an event), since a freed block can be handed out again at once.
 *   - There is no CPU fallback: every arithmetic step runs in the library's
 *     CUDA kernels on the current device.
 *
 * Blocks are k x k x k arrays s[i1][i2][i3] (i3 fastest) of coefficients in the
 * tensor basis phi^j_{i1,a1}(x1) phi^j_{i2,a2}(x2) phi^j_{i3,a3}(x3), where
 * phi^j_{i,a}(x) = 2^{j/2} sqrt(2i+1) P_i(2^{j+1} x - 2a - 1) on box a of level j
 * (Appendix, eq. scalingFNC).  Trees are complete 2^3-trees: every internal node
 * has its 8 children (Algorithm 1 refines the 8 children together).
 */
#ifndef MRA_GB300_H
#define MRA_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define MRA_OK        0
#define MRA_EINVAL    1   /* invalid argument (k, eps, alpha, sizes, NULL, ...) */
#define MRA_ENOMEM    2   /* the allocator returned NULL                        */
#define MRA_ECUDA     3   /* a CUDA runtime call or kernel launch failed        */
#define MRA_ETIMEOUT  4   /* a bounded device-side wait gave up                 */
#define MRA_EDEPTH    5   /* warning: max_level reached with the l-inf test     */
                          /* still failing; the tree is valid (Algorithm 1)     */
#define MRA_ESTATE    6   /* the handle is not in the state the call needs      */

#define MRA_MAX_K      12  /* largest basis order k (polynomials per direction) */
#define MRA_MAX_LEVEL  12  /* deepest level j of a tree / operator table        */
#define MRA_MAX_TERMS 512  /* largest number M of Gaussian terms                */

typedef struct mra_tree mra_tree;
typedef struct mra_op mra_op;
typedef struct mra_mlp mra_mlp;
typedef struct mra_tree2 mra_tree2;

/* Device allocator hook: alloc returns device memory of `bytes` usable on
 * `stream` (NULL on failure); free releases it.  ctx is passed through.  The
 * library keeps the blocks it frees in a stream-ordered cache keyed by
 * (hook, stream, size) and reuses them for requests with the same key, so a
 * repeated call reaches the hook only for sizes it has not seen. */
typedef struct {
    void* (*alloc)(size_t bytes, void* stream, void* ctx);
    void  (*free)(void* ptr, void* stream, void* ctx);
    void* ctx;
} mra_alloc;

/* A density f(x) = sum_g (coef_g + r2coef_g |x - c_g|^2) exp(-expo_g |x - c_g|^2)
 * (host arrays, copied by the call).  r2coef may be NULL (all zero).  This
 * covers unit-mass Gaussians and the paper's Poisson test density
 * rho = -Laplacian sum exp(-a r^2) (Sec. 6.1). */
typedef struct {
    int n;
    const double* coef_host;     /* n      */
    const double* r2coef_host;   /* n or NULL */
    const double* expo_host;     /* n, > 0 */
    const double* center_host;   /* 3n, (x, y, z) per term */
} mra_density;

/* Tree states */
#define MRA_TREE_LEAVES     0  /* data on leaves only (adaptive tree, Sec. 2.2.1)  */
#define MRA_TREE_REDUNDANT  1  /* s on all nodes, d norms on internal nodes        */
#define MRA_TREE_NSFORM     2  /* per-scale outputs ghat^j on all nodes            */

typedef struct {
    int k;                     /* basis order                                     */
    int n_nodes;               /* nodes, sorted by level then Morton key          */
    int n_levels;              /* deepest level + 1                               */
    int state;                 /* MRA_TREE_*                                      */
    int depth_hit;             /* 1 when Algorithm 1 stopped at max_level         */
    int level_offset[MRA_MAX_LEVEL + 2];  /* nodes of level j: [off[j], off[j+1]) */
} mra_tree_info;

/* ------------------------------------------------------------------------ */
/* Algorithm 1 (Sec. 2.2): adaptive function decomposition in d = 3.
 * Level by level, each box's k^3 Gauss-Legendre values are projected
 * (eq. fvals2coefs, tensor form), interpolated to the GL nodes of its 8
 * children and compared with direct evaluation; if any child differs by more
 * than eps * max_g |f(c_g)| (l-infinity) the 8 children are processed, else the
 * box is a leaf holding its own coefficients.  init_level: refine uniformly up
 * to this level before testing.  uniform_level >= 0: build the uniform tree of
 * that depth instead (no test).  Leaves deeper than max_level are never made;
 * a failing test there returns MRA_EDEPTH with a valid tree.
 * Output: *out in state MRA_TREE_LEAVES.  Synchronous (level sizes are read
 * back to size the next level).
 * Errors: MRA_EINVAL for k outside [1, MRA_MAX_K], eps <= 0, max_level outside
 * [0, MRA_MAX_LEVEL], an empty density or non-positive exponents. */
int mra_build_tree(const mra_density* f, int k, double eps, int max_level,
                   int uniform_level, int init_level,
                   const mra_alloc* alloc, void* stream, mra_tree** out);

/* Create a tree from host arrays (e.g. an externally built tree).
 * n nodes; coords_host: 4n int32 rows (j, a1, a2, a3) sorted by level then by
 * box; leaf_host: n int32 flags; blocks_host: n * k^3 doubles (values of
 * internal nodes are ignored).  The node set must be a complete 2^3-tree
 * rooted at (0,0,0,0).  Output state MRA_TREE_LEAVES.  Synchronous.
 * Errors: MRA_EINVAL for an unsorted, incomplete or out-of-range node set. */
int mra_tree_import(int k, int n, const int32_t* coords_host, const int32_t* leaf_host,
                    const double* blocks_host, const mra_alloc* alloc, void* stream,
                    mra_tree** out);

/* Copy a tree to host arrays (sizes from mra_tree_info).  Any pointer may be
 * NULL to skip it.  coords_host: 4n int32; leaf_host: n int32; blocks_host:
 * n k^3 doubles; dnorm_host: n doubles (wavelet norms, 0 on leaves).
 * Synchronous on `stream`. */
int mra_tree_export(const mra_tree* t, int32_t* coords_host, int32_t* leaf_host,
                    double* blocks_host, double* dnorm_host, void* stream);

int mra_tree_get_info(const mra_tree* t, mra_tree_info* info);

/* Device views of a tree's arrays (valid until the tree is freed or changed
 * by reconstruct/truncate): blocks (n k^3 doubles) and leaf flags (n int32). */
int mra_tree_device_arrays(const mra_tree* t, double** blocks, int32_t** leaf);

/* Overwrite the blocks of a tree from device memory on `stream` (n k^3 doubles,
 * same node order).  The state is unchanged: the caller keeps the blocks
 * consistent with it. */
int mra_tree_set_blocks(mra_tree* t, const double* blocks, void* stream);

/* Output skeleton refinement.  The paper takes the output tree as a copy of
 * the input's redundant tree and says the assumption will be removed later
 * (Algorithm 2/3, Initialization); this entry removes it.  A potential is
 * broader than its density, so the input tree, coarse wherever the density is
 * negligible, is too coarse for the output near the sources.  One pass gives
 * every leaf at level j < max_level whose 26-neighbourhood at level j holds an
 * internal node its 8 children, filled with the exact two-scale refinement of
 * the leaf's block (the d = 0 half of eqs. recon_even / recon_odd); `passes`
 * passes are made (fewer if one splits nothing).  The function represented is
 * unchanged: applying the operator to the refined tree gives the output on the
 * graded skeleton, and the final truncation (mra_reconstruct) removes output
 * blocks that are insignificant.
 *   - f: a tree with leaf data (MRA_TREE_LEAVES or MRA_TREE_REDUNDANT); the
 *     new tree has f's state (a split leaf keeps its block, which is the
 *     projection its children refine, and a zero wavelet norm).
 *   - n_split_host (optional): leaves split over all passes.
 * Synchronous (the structure is built on the host).
 * Errors: MRA_EINVAL for passes outside [0, 8] or max_level outside
 * [0, MRA_MAX_LEVEL]; MRA_ESTATE for an ns-form tree. */
int mra_tree_refine(const mra_tree* f, int passes, int max_level, void* stream, mra_tree** out,
                    int* n_split_host);

/* ------------------------------------------------------------------------ */
/* Redundant tree (Sec. 2.2.1): bottom-up, each internal node receives
 * s^j = sum_p (H^(p1) x H^(p2) x H^(p3)) s^{j+1}_{child p} (eq. decomp_scaling)
 * and its seven wavelet blocks (eq. decomp_wavelet), i.e. the orthogonal
 * 2k x 2k filter [[H0 H1],[G0 G1]] applied in each direction to the (2k)^3
 * cube of its children.  G is the orthonormal completion of [H0 H1] by
 * Gram-Schmidt of (e_i, -e_i)/sqrt(2) (the paper defers G to Alpert et al.;
 * wavelet norms do not depend on the completion).  In place; state becomes
 * MRA_TREE_REDUNDANT.  mode:
 *   MRA_COMPRESS_NORMS    the scaling blocks of every internal node and its
 *                         wavelet norm ||d|| (what the final truncation reads);
 *   MRA_COMPRESS_STORE_D  also keeps the wavelet cubes, so that
 *                         mra_reconstruct(MRA_RECON_INVERSE) can undo the transform;
 *   MRA_COMPRESS_SCALING  the scaling blocks only -- all that Algorithm 3 reads of
 *                         its input (s^j at every level) -- with the wavelet norms
 *                         left at zero; half of the arithmetic of MRA_COMPRESS_NORMS.
 * Errors: MRA_EINVAL for another mode, MRA_ESTATE for an ns-form tree. */
#define MRA_COMPRESS_NORMS   0
#define MRA_COMPRESS_STORE_D 1
#define MRA_COMPRESS_SCALING 2
int mra_compress(mra_tree* t, int mode, void* stream);

/* ------------------------------------------------------------------------ */
/* make_operator: the Gaussian sum of K_{mu,alpha} (Sec. 3) and the operator
 * tables on levels 0..max_level:
 *   - tau_m = e^{2 s_m}, w_m = h C_alpha exp(-mu^2 e^{-2 s_m}/4 + (3-2alpha)s_m),
 *     s_m = A + m h (m = 1..M), C_alpha = 2 2^{-2alpha} pi^{-3/2} / Gamma(alpha);
 *     A, B, h by the rule: h0 = pi^2/(2 ln(1/eps)); lower tail below
 *     0.1 eps K_{0,alpha}(R); B = ln((ln(1/eps)+5)/delta^2)/2; h shrunk by 3 %
 *     until the sup of |K - sum| / K_{0,alpha} on 4000 log-spaced r in
 *     [delta, R] is <= eps (eq. KernelApproxByGaussians), delta = eps/10,
 *     R = sqrt(3);
 *   - F^{j;m,l}, l = -3..3 (eq. KernelFactor), from the cross-correlations
 *     Phi_ii' (eq. CrossCor) by quadrature;
 *   - block norms N_F, N_upF, N_dif (eq. BlockNorms, Frobenius) and the maximum
 *     over the coarse core of the 18-term estimate (eq. NormEstimateUsing1DBlocks).
 * FP64 throughout.  Synchronous (M is read back).
 * Errors: MRA_EINVAL for mu < 0, alpha outside (0, 3/2), eps outside (0, 0.5],
 * k outside [1, MRA_MAX_K], max_level outside [0, MRA_MAX_LEVEL]; MRA_ECUDA if
 * more than MRA_MAX_TERMS terms would be needed. */
int mra_make_operator(double mu, double alpha, double eps, int k, int max_level,
                      const mra_alloc* alloc, void* stream, mra_op** out);

typedef struct {
    int M;                 /* number of Gaussian terms             */
    int k, max_level;
    double mu, alpha, eps;
} mra_op_info;
int mra_op_get_info(const mra_op* op, mra_op_info* info);

/* Re-weight op for another mu on its own term grid: tau_m = e^{2 s_m} and
 * every table that depends only on tau (F, the block norms, the estimate)
 * are kept, and w_m = h C_alpha exp(-mu^2 e^{-2 s_m}/4 + (3-2alpha) s_m) is
 * recomputed (Sec. 3).  The new sum must pass the same sup-norm test as
 * make_operator (|K_{mu,alpha} - sum| <= eps K_{0,alpha} on 4000 radii in
 * [delta, R]); the grid was chosen for the construction's mu, so a new mu
 * above it passes (its weights drop the broad terms faster) and one well
 * below it may not.  Not concurrent with another call on op.  Synchronous.
 * Errors: MRA_EINVAL (op unchanged) for mu < 0 or a grid that fails the test. */
int mra_op_retune(mra_op* op, double mu, void* stream);

/* Copy operator tables to host (any pointer may be NULL):
 * w_host, tau_host: M doubles; F_host: (max_level+1) * M * 7 * k * k doubles,
 * index [j][m][l+3][i][i']; nF_host: (max_level+1) * M * 7; est_host:
 * (max_level+1) * M (max over the coarse core of the 18-term estimate, without
 * w_m; 0 at j = 0).  Synchronous. */
int mra_op_export(const mra_op* op, double* w_host, double* tau_host, double* F_host,
                  double* nF_host, double* est_host, void* stream);

/* ------------------------------------------------------------------------ */
/* Algorithm 3 (Sec. 5): the modified ns-form apply in d = 3.
 * For every node a of the input's redundant tree (the output skeleton) at
 * level j, every translation t in the parity band (t_d in [-3,2] for even a_d,
 * [-2,3] for odd a_d; eq. fine_scale_band with b_j = 3) whose input box
 * b = a - t lies in [0, 2^j)^3, and every kept term m:
 *     ghat^j_a += w_m (F^{j;m,t1} x F^{j;m,t2} x F^{j;m,t3}) f^j_b.
 * Kept terms: eta = eps ||T_0 f_0|| / ||f||; J_m = finest j >= 1 with
 * w_m Est(j,m) > eta/M (else 0); terms with j <= J_m; at internal nodes with
 * j < J_m the core |t|_inf <= 1 is left to the finer scale (outer band,
 * eq. apply_algo); per scale and Core/Boundary-1/2/3 subset, a term range
 * [m1, m2] trimmed at both ends while the cumulative w_m prod max N_F stays
 * below eta/432 (Sec. 4).  Missing input boxes are refined from their
 * ancestor leaf (Step 2).
 * The input tree must be MRA_TREE_REDUNDANT (mra_compress) and no deeper than
 * the operator's max_level.  Output: a new tree in state MRA_TREE_NSFORM.
 * Returns after the work is queued (the call synchronises once to size the
 * worklist).  When stats (host) is not NULL the call also waits for the apply,
 * fills stats and reads back the errors found on the device: MRA_ETIMEOUT
 * when a tensor-core completion wait gave up, MRA_EINVAL when a tensor-core
 * output scale w_m / (s_V s_F) or an input value falls outside FP32's range
 * (use MRA_PREC_FP64), MRA_ECUDA for a failed Step-2 lookup; with stats NULL
 * these are not checked. */

#define MRA_PREC_FP64     0   /* FP64 SIMT contractions                        */
#define MRA_PREC_FP32     1   /* FP32 SIMT contractions, FP64 accumulation     */
#define MRA_PREC_TC_SPLIT 2   /* FP16 hi+lo split products on tcgen05 tensor   */
                              /* cores with FP32 accumulation (TMEM), each    */
                              /* chunk of terms added to the output block in  */
                              /* FP64; Step-2 blocks refined in FP64          */
#define MRA_PREC_TC_LADDER 3  /* precision ladder on the tensor cores: per     */
                              /* output node and term, single FP16 products    */
                              /* (one MMA instead of three) when the term's    */
                              /* bound w_m sum_items prod N_F ||f_b|| times    */
                              /* 2^-8 fits the node's share of the budget      */
                              /* eps ||T_0 f_0|| / (4 sqrt(N)), else FP16 hi+lo */
                              /* (FP64 output accumulation and Step 2)         */
#define MRA_PREC_TC_FAST   4  /* MRA_PREC_TC_SPLIT with the Step-2 blocks,     */
                              /* which only become FP16 hi/lo operands,        */
                              /* refined in FP32 under the static screen: a    */
                              /* variant outside the FP64 contract, kept to    */
                              /* measure what that contract costs              */

/* Screens of the (output box, translation) pairs' term ranges.  The test of
 * an item is w_m N_F(t1) N_F(t2) N_F(t3) ||f_b|| > eta_blk with
 * eta_blk = eps ||T_0 f_0|| / sqrt(N 216 M) (Sec. 4's bound with the input
 * block's own norm; Step-2 blocks after refinement). */
#define MRA_SCREEN_STATIC  0  /* Sec. 4's ranges per scale and class only       */
#define MRA_SCREEN_PAIR    1  /* exact: per pair, first..last passing term      */
#define MRA_SCREEN_LEARNED 2  /* the network's per-box, per-class cut-offs,     */
                              /* widened by `margin` terms, and every passing   */
                              /* term outside them restored (a miss, counted)   */

typedef struct {
    int precision;          /* MRA_PREC_*                                     */
    int block_screen;       /* 1: also drop items whose w prod N_F ||f_b|| is  */
                            /* below eps ||T_0 f_0|| / sqrt(N 216 M)           */
    int unscreened;         /* 1: every term at every scale (band only; tests) */
    int itemwise;           /* 1: SIMT paths apply each item's three mode     */
                            /* products separately instead of the nested sums */
                            /* of Algorithm 3 (same items; for comparison)    */
    int screen_mode;        /* MRA_SCREEN_*                                   */
    int margin;             /* learned screen: terms added on each side        */
    int wait_limit;         /* tensor-core apply: polls of one MMA completion  */
                            /* wait before it gives up (MRA_ETIMEOUT); 0 means */
                            /* the default 2^26                                */
    int test_flags;         /* 0 in normal use; MRA_TEST_WITHHOLD_MMA for the  */
                            /* test of the bounded wait                        */
    const mra_mlp* schedule;  /* learned screen: a 16 -> 12 network (mra_mlp_*) */
} mra_apply_opts;

/* Test hook of the bounded device waits: the tensor-core apply's issuing
 * threads send neither the first group of MMAs of a node nor its commit, so
 * the first completion wait of every CTA can only end by reaching
 * wait_limit.  Nothing is in flight when it gives up: the kernel records
 * MRA_ETIMEOUT, frees its tensor memory and returns, and the output is not
 * valid. */
#define MRA_TEST_WITHHOLD_MMA 1

typedef struct {
    int64_t n_pairs;        /* (output node, translation) pairs                */
    int64_t n_items;        /* (output node, translation, term) items          */
    int64_t n_ghosts;       /* input blocks refined by Step 2                  */
    int64_t n_out_nodes;
    double eta;             /* operator-block threshold used                   */
    double sigma;           /* ||T_0 f_0||                                     */
    double fnorm;           /* ||f||_2                                         */
    float ms_screen, ms_ghost, ms_apply; /* device times (CUDA events)         */
    int64_t n_items_lowp;   /* items done with single FP16 products (ladder)   */
    int64_t n_misses;       /* learned screen: passing items outside the      */
                            /* prediction, restored by the exact test          */
    int64_t n_pairs_empty;  /* pair / learned screens: pairs left with no term */
} mra_apply_stats;

int mra_apply_ns(const mra_op* op, const mra_tree* f, const mra_apply_opts* opts,
                 void* stream, mra_tree** g_ns, mra_apply_stats* stats);

/* The same apply for callers that cannot allocate device memory.  The paper
 * has no counterpart: this is a deployment variant of mra_apply_ns.
 *
 * Some callers cannot call cudaMalloc or cudaFree during the apply: code that
 * runs where another component owns the device allocator, or work that must
 * not change the device's memory map while it runs.  This entry point
 * allocates nothing: its scratch (worklist, Step-2 hash set and refined input
 * blocks) is one fixed 21 MiB array in device memory that every GPU loading the
 * library holds until the process exits.
 *   - f: an MRA_TREE_REDUNDANT tree with at most 1024 nodes and k <= 8, whose
 *     Step-2 refinement needs at most 4096 input blocks; op as for
 *     mra_apply_ns (static screening only, no per-block screen).
 *   - precision: MRA_PREC_FP64 or MRA_PREC_FP32.
 *   - ghat_out: caller-owned device memory of f's n_nodes * k^3 doubles; on
 *     return it holds ghat^j for every node in f's node order (the data of the
 *     MRA_TREE_NSFORM tree mra_apply_ns would return).
 *   - n_items_host (optional): the number of (node, translation, term) items.
 * Sizes beyond these limits return MRA_EINVAL with a message, before any work
 * is queued (nodes, k) or right after the screen (refined blocks: then only
 * the screen has run, and nothing past it is queued).
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress).  Every call shares the one array and leaves its
 * contents behind; the call clears what must start at zero.  Calls that
 * overlap on the GPU (other streams or threads) race on the array: serialise
 * them.  The call synchronises `stream` twice -- after the screen, to read the
 * worklist sizes, and at the end, to read the device's error words (a failed
 * Step-2 lookup returns MRA_ECUDA) -- so it cannot be called while `stream` is
 * being captured into a CUDA graph. */
int mra_apply_ns_noalloc(const mra_op* op, const mra_tree* f, int precision, double* ghat_out,
                         void* stream, int64_t* n_items_host);

/* ------------------------------------------------------------------------ */
/* Learned schedule.  The paper has no learned part; this group trains and
 * runs a small network that predicts, per output box, the term cut-offs of
 * the exact per-pair screen (MRA_SCREEN_PAIR), so the apply can use them
 * (MRA_SCREEN_LEARNED) with the exact test as the judge of every miss.
 *
 * Network: 3 hidden layers of 128 ReLU units, FP16 weights and activations,
 * FP32 accumulation; FP32 master weights trained by Adam (beta 0.9 / 0.999,
 * eps 1e-8).  Parameters, one FP32 vector: W1 [128][n_in], b1 [128],
 * W2 [128][128], b2, W3 [128][128], b3, W4 [n_out][128], b4 [n_out],
 * row-major.  Arrays x, y, target are device FP32, row-major [n][width].
 *
 * mra_mlp_create: params_host (n_params floats) or, when NULL, He-uniform
 * weights from a splitmix64 stream seeded with `seed` and zero biases.
 * Synchronous.
 * mra_mlp_forward: y = network(x) for n rows (queued on `stream`).
 * mra_mlp_loss_grad: the schedule loss (n_out must be 12; per class S
 * [e_S, lo_S, hi_S] against [E_S, LO_S, HI_S]:
 *   sum_S softplus(e_S) - E_S e_S + (1 - E_S)((lo_S - LO_S)^2 + (hi_S - HI_S)^2),
 * averaged over the rows) and its gradient with respect to every parameter
 * (grad_host: n_params floats, may be NULL).  Synchronous.
 * mra_mlp_train_step: one Adam step on the batch's mean loss (queued; when
 * loss_host is not NULL the call synchronises and returns the batch loss
 * before the step).
 * mra_screen_data: for a compressed tree, the network's 16 inputs per node
 * and the exact screen's 12 targets per node (either pointer may be NULL),
 * device FP32 [n_nodes][16] and [n_nodes][12] in node order:
 *   inputs   j / max_level; leaf flag; log10(||s_a|| / eta_blk) / 10; per
 *            class S = 0..3 the log10(.)/10 of the maximum and of the sum of
 *            ||f_b|| / eta_blk over the box's pairs of that class (0 when
 *            none); the number of such pairs / 64 per class; mu / 2;
 *   targets  per class: [1, 0, 0] when no term of the class passes the exact
 *            test, else [0, first / (M - 1), last / (M - 1)].
 * Synchronous.  Errors as for mra_apply_ns. */
#define MRA_SCHED_INPUTS  16
#define MRA_SCHED_OUTPUTS 12
int mra_mlp_create(int n_in, int n_out, const float* params_host, unsigned long long seed,
                   const mra_alloc* alloc, void* stream, mra_mlp** out);
int mra_mlp_num_params(const mra_mlp* net, int64_t* n_params);
int mra_mlp_get_params(const mra_mlp* net, float* params_host, void* stream);
int mra_mlp_set_params(mra_mlp* net, const float* params_host, void* stream);
int mra_mlp_forward(const mra_mlp* net, const float* x, int64_t n, float* y, void* stream);
int mra_mlp_loss_grad(mra_mlp* net, const float* x, const float* target, int64_t n, float* grad_host,
                      double* loss_host, void* stream);
int mra_mlp_train_step(mra_mlp* net, const float* x, const float* target, int64_t n, float lr,
                       void* stream, double* loss_host);
int mra_mlp_free(mra_mlp* net);
int mra_screen_data(const mra_op* op, const mra_tree* f, float* inputs, float* targets, void* stream);

/* ------------------------------------------------------------------------ */
/* Batched apply: one operator, many independent inputs.  The paper applies
 * the operator to one function at a time (Algorithm 3); this group is its
 * deployment form for many right-hand sides at once, with the same items
 * per input as mra_apply_ns.
 *
 * mra_plan_create screens all trees together (synchronous: one host
 * synchronisation sizes the joint worklist).  Each tree keeps its own norms,
 * eta, J_m and term ranges; Step-2 blocks are found per tree.  The trees are
 * borrowed, not copied: they must stay alive, compressed and unchanged in
 * structure while the plan exists (their blocks may be rewritten, e.g. with
 * mra_tree_set_blocks + mra_compress; the plan keeps the screen it made at
 * creation).  op must outlive the plan.
 *   - trees: ntrees (>= 1) handles in MRA_TREE_REDUNDANT state, order k of op,
 *     depth <= op's max_level.
 *   - opts (may be NULL): precision (default MRA_PREC_TC_SPLIT for k <= 8,
 *     else MRA_PREC_FP64; the tensor-core paths MRA_PREC_TC_SPLIT and
 *     MRA_PREC_TC_LADDER need k <= 8; the ladder's budget is per tree) and use_graph
 *     (default 1 when opts is NULL).
 * mra_plan_execute queues, on `stream`: the gather of every tree's current
 * blocks, the Step-2 refinement and one Step-3 launch over the nodes of all
 * trees (a persistent kernel taking nodes from an atomic counter).  With
 * use_graph the first execute captures these launches into a CUDA graph (on
 * a stream the plan owns) and every execute launches that graph; `stream`
 * must not be capturing.  Executes on one plan must not overlap.
 * mra_plan_autotune (synchronous) times the tensor-core kernel variants on
 * the plan's worklist, reps launches each: (terms per chunk, CTAs per SM) in
 * (8,3) (8,2) (4,3) (4,2) (4,4), node order as screened or heaviest first
 * (most pairs).  The fastest becomes the plan's variant (ms_variant[v],
 * v = pair index + 5 heavy_first); other precisions have one variant.
 * mra_plan_set_variant chooses one by hand.  Both drop a captured graph.
 * mra_plan_output copies the output of tree b (as of the last execute
 * queued before it on `stream`) into a new MRA_TREE_NSFORM tree.
 * mra_plan_get_info and mra_plan_tree_stats are synchronous; get_info also
 * reports a device error of past executes (MRA_ETIMEOUT, MRA_ECUDA). */
typedef struct mra_plan mra_plan;
#define MRA_PLAN_VARIANTS 10

typedef struct {
    int precision;          /* MRA_PREC_*                                     */
    int use_graph;          /* 1: executes replay one captured CUDA graph      */
    int screen_mode;        /* MRA_SCREEN_STATIC, MRA_SCREEN_PAIR or           */
                            /* MRA_SCREEN_LEARNED (per-pair ranges narrowed at */
                            /* creation with the blocks then; the learned      */
                            /* screen's misses are found and restored by the   */
                            /* exact test, per tree, as in mra_apply_ns)       */
    int margin;             /* learned screen: terms added on each side        */
    int reserved[4];
    const mra_mlp* schedule;  /* learned screen: a 16 -> 12 network; it must   */
                              /* outlive mra_plan_create only                 */
} mra_plan_opts;

typedef struct {
    int n_trees;
    int64_t n_nodes;        /* output nodes of all trees                       */
    int64_t n_pairs;
    int64_t n_ghosts;       /* Step-2 blocks of all trees                      */
    int64_t n_items;        /* items applied by the last execute               */
    int precision;
    int terms_per_chunk;    /* tensor-core variant in use                      */
    int ctas_per_sm;
    int heavy_first;
    int tuned;              /* 1 after mra_plan_autotune                       */
    float ms_variant[MRA_PLAN_VARIANTS]; /* autotune: mean apply time per variant */
    int graph;              /* 1 when a captured graph exists                  */
    int graph_kernels;      /* kernels in one execute's graph                  */
    float ms_screen;        /* device time of the screen at creation           */
    int64_t n_items_lowp;   /* items of the last execute done with single FP16 */
    int screen_mode;        /* MRA_SCREEN_* of the plan                        */
    int64_t n_misses;       /* learned screen: passing items outside the       */
                            /* network's ranges, restored at creation          */
    int64_t n_pairs_empty;  /* pair / learned screens: pairs left with no term */
} mra_plan_info;

int mra_plan_create(const mra_op* op, mra_tree* const* trees, int ntrees, const mra_plan_opts* opts,
                    void* stream, mra_plan** out);
int mra_plan_execute(mra_plan* p, void* stream);
int mra_plan_autotune(mra_plan* p, int reps, void* stream);
int mra_plan_set_variant(mra_plan* p, int terms_per_chunk, int ctas_per_sm, int heavy_first);
int mra_plan_output(const mra_plan* p, int b, void* stream, mra_tree** g_ns);
int mra_plan_get_info(const mra_plan* p, mra_plan_info* info, void* stream);
/* Per-tree screen results: fnorm, sigma, eta, n_pairs, n_out_nodes, and the
 * items of the last execute; n_ghosts is -1 (counted per batch). */
int mra_plan_tree_stats(const mra_plan* p, int b, void* stream, mra_apply_stats* stats);
int mra_free_plan(mra_plan* p);

/* ------------------------------------------------------------------------ */
/* Reconstruct.
 * MRA_RECON_ASSEMBLE: for an MRA_TREE_NSFORM tree, eq. g_assemble top-down
 * (each child adds the d = 0 upsampling of its parent, eqs. recon_even /
 * recon_odd), then mra_compress (MRA_COMPRESS_NORMS); if truncate != 0, leaf siblings whose
 * parent has ||d|| < eps ||g|| / sqrt(N) are merged bottom-up (Algorithm 3,
 * Step 4, "discard unnecessary blocks").  State becomes MRA_TREE_REDUNDANT
 * (the tree may shrink).
 * MRA_RECON_INVERSE: for an MRA_TREE_REDUNDANT tree compressed with
 * MRA_COMPRESS_STORE_D, the inverse two-scale transform from the root down (the
 * filter matrix is orthogonal; its transpose inverts it); state becomes
 * MRA_TREE_LEAVES with the leaves rebuilt. */
#define MRA_RECON_ASSEMBLE 0
#define MRA_RECON_INVERSE  1
int mra_reconstruct(mra_tree* t, int mode, int truncate, double eps, void* stream,
                    double* truncation_l2_host);

/* ------------------------------------------------------------------------ */
/* Products and inner products of trees, for the hydrogen ground-state
 * iteration phi = -2 G_mu V phi of Sec. 6.2 (Steps 2 and 4).  The paper
 * computes these by the method of its reference [A-B-G-V:2002], which it does
 * not describe; the definitions below are this library's.
 *
 * A potential V(x) = sum_g (coef_g + r2coef_g |x - c_g|^2) exp(-expo_g |x - c_g|^2)
 *                  + sum_n charge_n / |x - R_n|
 * (host arrays, copied by the call; r2coef may be NULL).  expo_g >= 0, so a
 * term with expo 0 is a polynomial; a nucleus of charge Z at R is the term
 * charge -Z.  A quadrature point that coincides with some R_n takes 0 from
 * that term. */
typedef struct {
    int n_gauss;
    const double* coef_host;     /* n_gauss            */
    const double* r2coef_host;   /* n_gauss or NULL     */
    const double* expo_host;     /* n_gauss, >= 0       */
    const double* center_host;   /* 3 n_gauss           */
    int n_charge;
    const double* charge_host;   /* n_charge            */
    const double* position_host; /* 3 n_charge          */
} mra_potential;

/* out = scale * P(V f): a new tree on f's skeleton (state MRA_TREE_LEAVES,
 * internal blocks zero) whose leaf (j, a) holds the coefficients of V f
 * projected by the box's k-point Gauss-Legendre rule per direction,
 *   s'_i = 2^{-3j/2} sum_q w_q phi_i(u_q) V(x_q) f(x_q),
 * with f(x_q) from the leaf's block (eq. fvals2coefs and its inverse in
 * tensor form).  Exact when V f restricted to the box is a polynomial of
 * degree < 2k - 1 - (k - 1) = k per direction; otherwise the discrete
 * projection of the product.  f: MRA_TREE_LEAVES or MRA_TREE_REDUNDANT.
 * Synchronous.  Errors: MRA_EINVAL for an empty potential, a negative
 * exponent, a NULL array or a non-finite value; MRA_ESTATE for an ns-form f. */
int mra_tree_multiply(const mra_tree* f, const mra_potential* v, double scale, void* stream,
                      mra_tree** out);

/* <a, b> = sum over the leaves of sum_i a_i b_i: the L2 inner product over the
 * unit cube of the two functions (the leaf blocks are coefficients in an
 * orthonormal basis).  a and b must have the same skeleton (same k, node list
 * and leaf flags) and leaf data (MRA_TREE_LEAVES or MRA_TREE_REDUNDANT).  FP64;
 * the order of the partial sums is not fixed.  Synchronous (*out_host is
 * written).  Errors: MRA_EINVAL for different skeletons; MRA_ESTATE for an
 * ns-form tree. */
int mra_tree_dot(const mra_tree* a, const mra_tree* b, void* stream, double* out_host);

/* t *= alpha on every block (leaf and internal; stored wavelet cubes are
 * dropped).  Stream-ordered; no synchronisation. */
int mra_tree_scale(mra_tree* t, double alpha, void* stream);

/* One pass of the ground-state iteration phi = -2 G_mu V phi (Sec. 6.2,
 * eq. Kalos; Steps 2-5) on a cube of side `length` (physical units) mapped to
 * the unit cube by x = length * u.  V is given in cube coordinates with
 * physical values, V~(u) = V(length u): a nucleus of charge Z at the cube
 * point u0 is the point charge -Z / length at u0.
 *   2. P = V phi (mra_tree_multiply);
 *   3. phi_new = -2 length^2 G~_{mu length} P: compress, mra_apply_ns with
 *      the operator K_{mu length, 1} built for this call (eps, max_level,
 *      opts as given; NULL opts = FP64 defaults), then eq. g_assemble
 *      without truncation, so phi_new keeps phi's skeleton;
 *   4. E_new = (-<P, phi_new> - mu^2/2 <phi_new, phi_new>
 *               + <V phi_new, phi_new>) / <phi_new, phi_new>,
 *      the paper's energy with (1/2)<grad phi_new, grad phi_new> replaced by
 *      -<V phi, phi_new> - mu^2/2 ||phi_new||^2, which the equation
 *      (-Laplacian + mu^2) phi_new = -2 V phi gives by integration by parts;
 *   5. *phi_next = phi_new / ||phi_new|| (physical L2 norm; state
 *      MRA_TREE_LEAVES), and the next mu.
 * phi: leaf data (MRA_TREE_LEAVES or MRA_TREE_REDUNDANT); it is not changed.
 * op_cache: NULL, or the address of an operator handle kept between steps.
 * With NULL the step builds its operator and frees it.  Otherwise an
 * operator in *op_cache with this k, eps and max_level (alpha 1) is
 * re-weighted for mu * length (mra_op_retune); when its grid fails the
 * sup-norm test for that mu, or *op_cache is NULL or does not match, a new
 * operator is built, the old one freed and the new one stored in *op_cache
 * (other errors of the re-weighting are returned).  The caller frees it
 * (mra_free).
 * Synchronous.  Errors: those of the calls above; MRA_EINVAL for length or
 * mu not positive and finite. */
typedef struct {
    double energy;     /* E_new                                                   */
    double mu_next;    /* sqrt(-2 E_new), or mu when E_new >= 0                   */
    double norm_new;   /* ||phi_new|| (physical units) before normalisation       */
    int n_terms;       /* Gaussian terms M of the operator                        */
    int op_rebuilt;    /* 1 when the step built its operator, 0 when it re-weighted */
    int64_t n_items;   /* items applied by Step 3                                 */
    float ms_apply;    /* device time of Step 3's apply kernels (CUDA events)     */
} mra_kalos_info;

int mra_kalos_step(const mra_tree* phi, const mra_potential* v, double length, double mu, double eps,
                   int max_level, const mra_apply_opts* opts, mra_op** op_cache, void* stream,
                   mra_tree** phi_next, mra_kalos_info* info);

/* ------------------------------------------------------------------------ */
/* The d = 2 variant.  The paper implemented the apply for d = 2 and d = 3
 * (Sec. 6) and illustrates Algorithm 3 for d = 2; in d = 2 the band
 * translations fall into three subsets, Core / Boundary-1 / Boundary-2 (Sec. 4).
 * Functions on the unit square: a mra_tree2 holds k x k blocks in the basis
 * phi^j_{i1,a1}(x1) phi^j_{i2,a2}(x2), nodes sorted by level then 2-D Morton key
 * (bit 2b+1 from a1, bit 2b from a2), the 4 children of an internal node
 * contiguous in quadrant order (p1 p2) = 00, 01, 10, 11.  Handles are released
 * with mra_free (or mra_free_tree2); the conventions of the d = 3 calls hold. */

/* Algorithm 1 in d = 2.  f->center_host holds 2 numbers per term (x, y); the
 * other fields as in mra_build_tree.  Errors as mra_build_tree. */
int mra_build_tree2(const mra_density* f, int k, double eps, int max_level, int uniform_level,
                    int init_level, const mra_alloc* alloc, void* stream, mra_tree2** out);

/* A d = 2 tree from host arrays: coords_host 3n int32 rows (j, a1, a2) sorted
 * by level then key, leaf_host n flags, blocks_host n k^2 doubles.  The node set
 * must be a complete quadtree rooted at (0, 0, 0).  Synchronous. */
int mra_tree2_import(int k, int n, const int32_t* coords_host, const int32_t* leaf_host,
                     const double* blocks_host, const mra_alloc* alloc, void* stream, mra_tree2** out);

/* Copy coords (3n), leaf flags (n), blocks (n k^2) and wavelet norms (n) to host
 * (any pointer may be NULL).  Synchronous. */
int mra_tree2_export(const mra_tree2* t, int32_t* coords_host, int32_t* leaf_host, double* blocks_host,
                     double* dnorm_host, void* stream);
int mra_tree2_get_info(const mra_tree2* t, mra_tree_info* info);

/* Redundant tree in d = 2: every internal node receives s^j and the norm of its
 * three wavelet blocks from the (2k)^2 square of its 4 children, W sq W^T
 * (eqs. decomp_scaling / decomp_wavelet).  In place; state MRA_TREE_REDUNDANT. */
int mra_compress2(mra_tree2* t, void* stream);

/* The operator K_{mu,alpha} in R^2: the Gaussian sum of the integral
 * representation (eq. IntegralRepr with pi^{-1} in C_alpha and exponent
 * (2 - 2 alpha) s; sup test relative to K_{0,alpha}(r) = C_alpha Gamma(1 - alpha)
 * / (2 r^{2 - 2 alpha}) on [delta, sqrt 2]); the 1-D blocks F^{j;m,l} and norms
 * as in d = 3; the estimate of eq. NormEstimateUsing1DBlocks for two factors
 * (the mean of N_dif N_F + N_upF N_dif over both orderings).  alpha = 1/2,
 * mu = 0 gives 1/(2 pi r).  Errors: MRA_EINVAL for alpha outside (0, 1) and as
 * mra_make_operator.  The operator is usable only with mra_apply_ns2. */
int mra_make_operator2(double mu, double alpha, double eps, int k, int max_level, const mra_alloc* alloc,
                       void* stream, mra_op** out);

/* Algorithm 3 in d = 2 (FP64): for every node a of the compressed input (the
 * output skeleton), every translation t of the parity band whose input box
 * lies in [0, 2^j)^2 and every kept term m,
 *     ghat^j_a += w_m F^{j;m,t1} f^j_{a-t} (F^{j;m,t2})^T,
 * with J_m, the subsets S = number of |t_d| <= 1 (0, 1, 2) and their ranges
 * trimmed while the cumulative w_m prod_d max N_F stays <= eta / 72; a missing
 * input block is refined from its ancestor leaf (Step 2, d = 0).  f must be
 * MRA_TREE_REDUNDANT; the result is a new MRA_TREE_NSFORM tree on f's
 * skeleton.  stats (optional): n_pairs, n_items, n_ghosts (Step-2 refinements
 * made), eta, sigma, fnorm, ms_apply.  Synchronous.  Errors: MRA_EINVAL for a
 * d = 3 operator, k mismatch or a tree deeper than the operator. */
int mra_apply_ns2(const mra_op* op, const mra_tree2* f, void* stream, mra_tree2** g_ns,
                  mra_apply_stats* stats);

/* eq. g_assemble, compress and (truncate != 0) the merge of leaf siblings whose
 * parent has ||d|| < eps ||g|| / sqrt(N) (Algorithm 3, Step 4), as
 * mra_reconstruct(MRA_RECON_ASSEMBLE) in d = 3.  t must be MRA_TREE_NSFORM. */
int mra_reconstruct2(mra_tree2* t, int truncate, double eps, void* stream, double* truncation_l2_host);

int mra_free_tree2(mra_tree2* t);

/* Free any handle of this library -- a tree, operator, plan or network --
 * exactly once (NULL is ignored).  The kind is read from the tag every handle
 * starts with; a pointer that is not a live handle returns MRA_EINVAL.  The
 * typed frees below do the same for one kind each. */
int mra_free(void* handle);
int mra_free_tree(mra_tree* t);
int mra_free_op(mra_op* op);

/* Static message for the last error on this thread. */
const char* mra_last_error(void);

/* Library version string. */
const char* mra_version(void);

/* Number of kernels this library has launched in this process (all
 * devices, all threads); differences bracket a region of interest. */
unsigned long long mra_kernel_launches(void);

/* Return every device block in the library's reuse cache to the hook (or
 * cudaFreeAsync) it came from, on the stream it was used on; the number of
 * bytes released.  Call it before an allocator hook goes away, or to give the
 * memory back.  Thread-safe; blocks held by live handles are not affected. */
size_t mra_release_cached(void);

#ifdef __cplusplus
}
#endif
#endif /* MRA_GB300_H */
