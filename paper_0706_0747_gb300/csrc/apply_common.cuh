// Worklist records shared by the apply kernels (apply.cu, apply_fact.cu).
#pragma once
#include <cuda_fp16.h>

#include "mra_internal.cuh"

namespace mra {

struct Pair {
    int32_t out;    // output node
    int32_t in;     // input node (>= 0) or -1 - ghost id
    int16_t m_lo, m_hi;
    int8_t t1, t2, t3;
    uint8_t flags;  // bit 0: core translation at an internal node
};
static_assert(sizeof(Pair) == 16, "Pair is 16 bytes");

struct ApplyArgs {
    int k, M, n;
    const Pair* pairs;
    const int32_t* pair_off;
    const int32_t* coord;
    const double* s;
    const double* gblk;
    const double* w;
    const void* F;         // double or float table [j][m][l+3][k][k]
    const double* nF;
    const int32_t* Jm;     // per-tree term schedules: J_m of tree b at Jm[b * jm_stride + m]
    const int32_t* node_tree = nullptr;  // tree of each node (NULL: one tree)
    int jm_stride = 0;
    double eta_blk;        // < 0: no per-block screen
    double* out;
    unsigned long long* n_items;  // items applied, per tree
};

// tensor-core apply (apply_tc.cu)
struct TcArgs {
    ApplyArgs A;           // A.n: number of node blocks (Step-2 blocks follow them)
    const __half* xh;      // FP16 hi/lo input blocks in the stage-I layout
    const __half* xl;
    const float* sx;       // per-block power-of-two scale
    const float* xmax;     // per-block max |x|
    const float* xnrm;     // per-block ||x||_2
    const __half* Fh;      // FP16 hi/lo operator blocks, 8 x 8, per (j, m, t)
    const __half* Fl;
    const float* sF;       // per-(j, m) scale
    const float* maxF;
    const double* lpb;     // per-tree error budget of one node for single-FP16 terms (NULL: all hi+lo)
    unsigned long long* n_lowp;  // items done with single FP16 operands (may be NULL)
    int* err;              // set to 4 when a completion wait reaches its limit
    unsigned wait_limit;   // polls of one completion wait
    int withhold;          // test hook: the first MMA group and its commit are not sent
    int* counter;          // work counter (zeroed by tc_launch)
    const int* order;      // node order (NULL: 0..nwork-1)
    int nwork;
    int kr;                // basis order (<= 8; padded to 8 inside)
};

struct TcBuffers {
    __half *xh = nullptr, *xl = nullptr, *Fh = nullptr, *Fl = nullptr;
    float *sx = nullptr, *xmax = nullptr, *xnrm = nullptr, *sF = nullptr, *maxF = nullptr;
    int* counter = nullptr;
};

// The screen works on a forest: one tree, or many trees whose node arrays are
// concatenated (tree b owns a contiguous node range, level-major and Morton
// sorted within a level, its root first).  Per tree: level offsets as
// absolute node indices (lm + 1 entries), its number of levels, and in the
// outputs its norms and schedule.
struct Forest {
    int k, ntrees, n, lm;        // order; trees; nodes in all; levels of the per-tree layouts
    const int32_t* coord;        // [n][4]: (j, a1, a2, a3)
    const int32_t* leaf;         // [n]
    const uint64_t* key;         // [n]
    const int32_t* off;          // [ntrees][lm + 1]
    const int32_t* node_tree;    // [n] (NULL: one tree)
    const int32_t* nlev;         // [ntrees] (NULL: lm)
    const double* s;             // [n][k^3]
    const double* filt;          // H0, H1 (k x k each)
};

// device results of the screen over a forest (screen_forest in apply.cu)
struct ScreenOut {
    double* dv = nullptr;         // [ntrees][4]: ||f_b||^2, sigma_b, eta_b, unused
    int32_t* sched = nullptr;     // [ntrees][sl]: Jm | m1 | m2 | cnt
    int sl = 0;
    int32_t* count = nullptr;     // [n + 1] pairs per output node
    int32_t* pair_off = nullptr;  // [n + 1]
    int32_t* total = nullptr;     // [2]: pairs, Step-2 blocks
    int32_t* err = nullptr;       // [0] screen, [1] Step 2 / apply
    uint64_t* gtab = nullptr;     // Step-2 set: parent keys of the missing boxes
    int32_t* gid = nullptr;       // slot -> id of its first needed child
    uint32_t* gmask = nullptr;    // slot -> octants needed
    uint64_t* gkeys = nullptr;    // [nghost] level | tree | Morton key of each child, by id
    uint32_t gcap = 0;
    Pair* pairs = nullptr;        // [npairs], out and in are forest node indices
    int npairs = 0, nghost = 0;
};

int screen_forest(const mra_op* op, const Forest& F, int unscreened, const Alloc& A, cudaStream_t st, ScreenOut* S);
void screen_release(const Alloc& A, ScreenOut* S);
// Step 2 for every missing input block of a forest; fp32: refine in FP32 (for blocks that
// only feed FP16 hi/lo tensor-core operands), else FP64
int ghost_refine_forest(const Forest& F, const ScreenOut& S, double* gblk, cudaStream_t st, bool fp32 = false);
Forest forest_of_tree(const mra_tree* f);

int tc_alloc(const mra_op* op, int nb, TcBuffers* B);            // nb: node + Step-2 blocks
int tc_prep_F(const mra_op* op, const TcBuffers& B, cudaStream_t st);
int tc_prep_blocks(int nb, int kr, int n, const double* s, const double* gblk, const TcBuffers& B, cudaStream_t st);
void tc_release(const mra_op* op, TcBuffers* B);
int tc_configure();
TcArgs tc_args(const ApplyArgs& A, const TcBuffers& B, int* err);
int tc_launch(const TcArgs& T, int mc, int ctas_per_sm, cudaStream_t st);
int tc3_configure();                               // apply_tc3.cu
int tc3_launch(const TcArgs& T, cudaStream_t st);  // counter zeroed by the caller

int launch_apply_fact(const ApplyArgs& A, int precision, cudaStream_t st);
int launch_apply_tc(const ApplyArgs& A, int nghost, const mra_op* op, int* err, const double* lpb,
                    unsigned long long* n_lowp, unsigned wait_limit, int withhold, cudaStream_t st);
int lp_budget(const Forest& F, const ScreenOut& S, double eps, double* lpb, cudaStream_t st);
int schedule_narrow(const mra_op* op, const Forest& F, const ScreenOut& S, const double* gblk, int mode,
                    const void* model, int margin, float* X_out, float* T_out, unsigned long long* counts,
                    const Alloc& A, cudaStream_t st);
int screen_data_impl(const mra_op* op, const mra_tree* f, float* X, float* T, cudaStream_t st);

}  // namespace mra
