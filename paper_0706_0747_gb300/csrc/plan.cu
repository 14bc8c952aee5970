// Batched apply of one operator to many independent inputs: Algorithm 3 over
// a forest.
//
// mra_plan_create concatenates the trees' node arrays (each tree keeps its
// level-major Morton order inside its own node range) and screens them all in
// one pass of the forest kernels of apply.cu: per tree its own ||f||,
// ||T_0 f_0||, eta, J_m and term ranges (Sec. 4), one warp per output node,
// Step-2 keys carrying the tree index.  Pair records hold forest node indices,
// so Step 3 is one launch over all nodes of all trees: the persistent
// tensor-core kernel takes nodes from an atomic counter, optionally in
// heaviest-first order.  mra_plan_execute gathers the trees' current blocks,
// refines the Step-2 blocks and applies; the first execute captures these
// launches in a CUDA graph that later executes replay.  The autotuner times
// the apply kernel's variants (terms per chunk, CTAs per SM, node order) on
// the plan's own worklist and keeps the fastest.
#include <algorithm>
#include <vector>

#include "apply_common.cuh"


namespace mra {

void count_launch_add(long long n);

struct TreeRef {
    const int32_t* coord;
    const int32_t* leaf;
    const uint64_t* key;
    const double* s;
};

// forest node i: tree b with base[b] <= i < base[b+1]
__device__ inline int tree_of(const int32_t* base, int ntrees, int i) {
    int lo = 0, hi = ntrees - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (base[mid] <= i) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__global__ void k_forest_struct(int n, int ntrees, const int32_t* base, const TreeRef* tr, int32_t* coord,
                                int32_t* leaf, uint64_t* key, int32_t* node_tree) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int b = tree_of(base, ntrees, i), l = i - base[b];
        for (int q = 0; q < 4; ++q) coord[4 * i + q] = tr[b].coord[4 * l + q];
        leaf[i] = tr[b].leaf[l];
        key[i] = tr[b].key[l];
        node_tree[i] = b;
    }
}

// s[i] <- block of node i in its own tree (the trees' current coefficients)
__global__ void k_forest_blocks(int n, int k3, const int32_t* base, const int32_t* node_tree, const TreeRef* tr,
                                double* s) {
    const size_t total = (size_t)n * k3;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / k3), r = (int)(e % k3);
        const int b = node_tree[i];
        s[e] = tr[b].s[(size_t)(i - base[b]) * k3 + r];
    }
}

}  // namespace mra

struct mra_plan {
    uint32_t magic = 0;
    const mra_op* op = nullptr;
    int k = 0, ntrees = 0, n = 0, lm = 0, precision = 0;
    std::vector<const mra_tree*> trees;
    std::vector<int32_t> base;        // ntrees + 1
    std::vector<int32_t> off_host;    // ntrees * (lm + 1)
    std::vector<int32_t> nlev_host;   // ntrees
    mra::Alloc A;
    // forest arrays (device)
    mra::TreeRef* tref = nullptr;
    int32_t *dbase = nullptr, *coord = nullptr, *leaf = nullptr, *off = nullptr, *node_tree = nullptr,
            *nlev = nullptr;
    uint64_t* key = nullptr;
    double* s = nullptr;
    mra::Forest F;
    mra::ScreenOut S;
    double* gblk = nullptr;
    double* out = nullptr;
    unsigned long long* nitems = nullptr;  // per tree, then the single-FP16 items of all trees
    double* lpb = nullptr;                 // precision-ladder budgets per tree
    bool tc = false;
    mra::TcBuffers tcb;
    int32_t* order_heavy = nullptr;
    // apply variant
    int mc = 8, ctas = 3, use_order = 0;
    float ms_variant[MRA_PLAN_VARIANTS] = {0};
    int tuned = 0;
    float ms_screen = 0.0f;
    // graph
    int use_graph = 1;
    int screen_mode = MRA_SCREEN_STATIC;
    const mra_mlp* schedule = nullptr;  // learned screen (used at creation only)
    int margin = 0;
    long long n_misses = 0, n_pairs_empty = 0;
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    long long graph_kernels = 0;
    long long executes = 0;
};

namespace mra {

static int plan_apply_args(const mra_plan* p, ApplyArgs* aa) {
    const mra_op* op = p->op;
    aa->k = p->k; aa->M = op->M; aa->n = p->n;
    aa->pairs = p->S.pairs; aa->pair_off = p->S.pair_off; aa->coord = p->coord;
    aa->s = p->s; aa->gblk = p->gblk; aa->w = op->w; aa->nF = op->nF;
    aa->Jm = p->S.sched; aa->node_tree = p->node_tree; aa->jm_stride = p->S.sl;
    aa->eta_blk = -1.0; aa->out = p->out; aa->n_items = p->nitems;
    aa->F = p->precision == MRA_PREC_FP64 ? (const void*)op->F : (const void*)op->F32;
    return MRA_OK;
}

static int plan_tc_launch(const mra_plan* p, int mc, int ctas, int ordered, cudaStream_t st) {
    ApplyArgs aa;
    plan_apply_args(p, &aa);
    TcArgs T = tc_args(aa, p->tcb, p->S.err + 1);
    T.order = ordered ? p->order_heavy : nullptr;
    T.lpb = p->lpb;
    T.n_lowp = p->nitems + p->ntrees;
    return tc_launch(T, mc, ctas, st);
}

// the launches of one execute (captured once when graphs are on)
static int plan_enqueue(const mra_plan* p, cudaStream_t st) {
    const int k3 = p->k * p->k * p->k;
    const size_t total = (size_t)p->n * k3;
    const int nb = (int)std::max<size_t>(1, std::min<size_t>(num_sms() * 8, (total + 255) / 256));
    k_forest_blocks<<<nb, 256, 0, st>>>(p->n, k3, p->dbase, p->node_tree, p->tref, p->s);
    MRA_CK_LAUNCH();
    MRA_TRY(ghost_refine_forest(p->F, p->S, p->gblk, st,
                                p->precision == MRA_PREC_TC_FAST && p->screen_mode == MRA_SCREEN_STATIC));
    MRA_CK(cudaMemsetAsync(p->nitems, 0, ((size_t)p->ntrees + 1) * sizeof(unsigned long long), st));
    if (p->tc) {
        MRA_TRY(tc_prep_blocks(p->n + p->S.nghost, p->k, p->n, p->s, p->gblk, p->tcb, st));
        MRA_TRY(plan_tc_launch(p, p->mc, p->ctas, p->use_order, st));
    } else {
        ApplyArgs aa;
        plan_apply_args(p, &aa);
        MRA_TRY(launch_apply_fact(aa, p->precision, st));
    }
    return MRA_OK;
}

static void plan_drop_graph(mra_plan* p) {
    if (p->gexec) cudaGraphExecDestroy(p->gexec);
    if (p->graph) cudaGraphDestroy(p->graph);
    p->gexec = nullptr;
    p->graph = nullptr;
    p->graph_kernels = 0;
}

static void plan_release(mra_plan* p) {
    plan_drop_graph(p);
    if (p->cap) cudaStreamDestroy(p->cap);
    const Alloc& A = p->A;
    screen_release(A, &p->S);
    if (p->op) tc_release(p->op, &p->tcb);
    A.put(p->tref); A.put(p->dbase); A.put(p->coord); A.put(p->leaf); A.put(p->off); A.put(p->node_tree);
    A.put(p->nlev); A.put(p->key); A.put(p->s); A.put(p->gblk); A.put(p->out); A.put(p->nitems);
    A.put(p->order_heavy); A.put(p->lpb);
    p->magic = 0;
    delete p;
}

static int plan_build(mra_plan* p, cudaStream_t st) {
    const mra_op* op = p->op;
    const int k3 = p->k * p->k * p->k, nt = p->ntrees, lm = p->lm;
    const Alloc& A = p->A;
    std::vector<TreeRef> tr(nt);
    for (int b = 0; b < nt; ++b) {
        const mra_tree* t = p->trees[b];
        tr[b] = TreeRef{t->a.coord, t->a.leaf, t->a.key, t->s};
        for (int j = 0; j <= lm; ++j) p->off_host[b * (lm + 1) + j] = p->base[b] + t->off[std::min(j, t->nlev)];
        p->nlev_host[b] = t->nlev;
    }
    const int n = p->n;
    MRA_TRY(dalloc(A, &p->tref, nt));
    MRA_TRY(dalloc(A, &p->dbase, nt + 1));
    MRA_TRY(dalloc(A, &p->off, (size_t)nt * (lm + 1)));
    MRA_TRY(dalloc(A, &p->nlev, nt));
    MRA_TRY(dalloc(A, &p->coord, 4 * (size_t)n));
    MRA_TRY(dalloc(A, &p->leaf, n));
    MRA_TRY(dalloc(A, &p->key, n));
    MRA_TRY(dalloc(A, &p->node_tree, n));
    MRA_TRY(dalloc(A, &p->s, (size_t)n * k3));
    MRA_CK(cudaMemcpyAsync(p->tref, tr.data(), nt * sizeof(TreeRef), cudaMemcpyHostToDevice, st));
    MRA_CK(cudaMemcpyAsync(p->dbase, p->base.data(), (nt + 1) * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    MRA_CK(cudaMemcpyAsync(p->off, p->off_host.data(), p->off_host.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    MRA_CK(cudaMemcpyAsync(p->nlev, p->nlev_host.data(), nt * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    const int nb = std::max(1, std::min(num_sms() * 8, (n + 255) / 256));
    k_forest_struct<<<nb, 256, 0, st>>>(n, nt, p->dbase, p->tref, p->coord, p->leaf, p->key, p->node_tree);
    MRA_CK_LAUNCH();
    const size_t total = (size_t)n * k3;
    const int nbs = (int)std::max<size_t>(1, std::min<size_t>(num_sms() * 8, (total + 255) / 256));
    k_forest_blocks<<<nbs, 256, 0, st>>>(n, k3, p->dbase, p->node_tree, p->tref, p->s);
    MRA_CK_LAUNCH();

    Forest& F = p->F;
    F.k = p->k; F.ntrees = nt; F.n = n; F.lm = lm;
    F.coord = p->coord; F.leaf = p->leaf; F.key = p->key; F.off = p->off;
    F.node_tree = p->node_tree; F.nlev = p->nlev; F.s = p->s; F.filt = p->trees[0]->filt;

    struct Events {
        cudaEvent_t e[2] = {nullptr, nullptr};
        ~Events() {
            for (cudaEvent_t x : e)
                if (x) cudaEventDestroy(x);
        }
    } ev;
    MRA_CK(cudaEventCreate(&ev.e[0]));
    MRA_CK(cudaEventCreate(&ev.e[1]));
    MRA_CK(cudaEventRecord(ev.e[0], st));
    MRA_TRY(screen_forest(op, F, 0, A, st, &p->S));
    MRA_CK(cudaEventRecord(ev.e[1], st));
    MRA_CK(cudaEventSynchronize(ev.e[1]));
    cudaEventElapsedTime(&p->ms_screen, ev.e[0], ev.e[1]);

    MRA_TRY(dalloc(A, &p->gblk, (size_t)(p->S.nghost + 1) * k3));
    if (p->screen_mode != MRA_SCREEN_STATIC) {
        // per-pair term ranges from the blocks at creation (Step 2 first): the exact
        // screen, or the network's per-box ranges with every miss restored
        Scratch tmp(A);
        unsigned long long* counts;
        MRA_TRY(tmp.get(&counts, 2));
        MRA_CK(cudaMemsetAsync(counts, 0, 2 * sizeof(unsigned long long), st));
        MRA_TRY(ghost_refine_forest(F, p->S, p->gblk, st));
        MRA_TRY(schedule_narrow(op, F, p->S, p->gblk, p->screen_mode == MRA_SCREEN_PAIR ? 1 : 2, p->schedule,
                                p->margin, nullptr, nullptr, counts, A, st));
        unsigned long long hc[2] = {0, 0};
        MRA_CK(cudaMemcpyAsync(hc, counts, sizeof(hc), cudaMemcpyDeviceToHost, st));
        MRA_CK(cudaStreamSynchronize(st));
        p->n_misses = (long long)hc[0];
        p->n_pairs_empty = (long long)hc[1];
    }
    MRA_TRY(dalloc(A, &p->out, (size_t)n * k3));
    MRA_TRY(dalloc(A, &p->nitems, (size_t)nt + 1));
    MRA_CK(cudaMemsetAsync(p->nitems, 0, ((size_t)nt + 1) * sizeof(unsigned long long), st));
    if (p->precision == MRA_PREC_TC_LADDER) {
        MRA_TRY(dalloc(A, &p->lpb, nt));
        MRA_TRY(lp_budget(F, p->S, op->eps, p->lpb, st));
    }

    // heaviest-first node order: counting sort of the per-node pair counts
    std::vector<int32_t> cnt(n), order(n);
    MRA_CK(cudaMemcpyAsync(cnt.data(), p->S.count, n * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    MRA_CK(cudaStreamSynchronize(st));
    std::vector<int32_t> start(218, 0);
    for (int i = 0; i < n; ++i) start[216 - std::min(216, std::max(0, cnt[i])) + 1]++;
    for (int c = 1; c < 218; ++c) start[c] += start[c - 1];
    for (int i = 0; i < n; ++i) order[start[216 - std::min(216, std::max(0, cnt[i]))]++] = i;
    MRA_TRY(dalloc(A, &p->order_heavy, n));
    MRA_CK(cudaMemcpyAsync(p->order_heavy, order.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice, st));

    if (p->tc) {
        MRA_TRY(tc_alloc(op, n + p->S.nghost, &p->tcb));
        MRA_TRY(tc_prep_F(op, p->tcb, st));
        MRA_TRY(tc_configure());
    }
    MRA_CK(cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking));
    MRA_CK(cudaStreamSynchronize(st));  // host vectors above are read by the copies
    return MRA_OK;
}

}  // namespace mra

using namespace mra;

static bool plan_ok(const mra_plan* p) { return p && p->magic == MRA_PLAN_MAGIC; }

extern "C" {

int mra_plan_create(const mra_op* op, mra_tree* const* trees, int ntrees, const mra_plan_opts* opts, void* stream,
                    mra_plan** out) {
    if (!out) { set_error("out is NULL"); return MRA_EINVAL; }
    *out = nullptr;
    if (!op || op->magic != MRA_OP_MAGIC) { set_error("invalid operator handle"); return MRA_EINVAL; }
    if (op->d != 3) { set_error("the operator is for d = 2"); return MRA_EINVAL; }
    if (!trees || ntrees < 1 || ntrees >= (1 << 22)) { set_error("ntrees must lie in [1, 2^22)"); return MRA_EINVAL; }
    const int prec = opts ? opts->precision : (op->k <= 8 ? MRA_PREC_TC_SPLIT : MRA_PREC_FP64);
    if (prec != MRA_PREC_FP64 && prec != MRA_PREC_FP32 && prec != MRA_PREC_TC_SPLIT && prec != MRA_PREC_TC_LADDER &&
        prec != MRA_PREC_TC_FAST) {
        set_error("precision %d is not available", prec);
        return MRA_EINVAL;
    }
    const bool tc = prec == MRA_PREC_TC_SPLIT || prec == MRA_PREC_TC_LADDER || prec == MRA_PREC_TC_FAST;
    if (tc && op->k > 8) { set_error("the tensor-core apply needs k <= 8"); return MRA_EINVAL; }
    long long total = 0;
    int lm = 0;
    for (int b = 0; b < ntrees; ++b) {
        const mra_tree* t = trees[b];
        if (!t || t->magic != MRA_TREE_MAGIC) { set_error("tree %d: invalid handle", b); return MRA_EINVAL; }
        if (t->k != op->k) { set_error("tree %d: order k=%d differs from operator k=%d", b, t->k, op->k); return MRA_EINVAL; }
        if (t->state != MRA_TREE_REDUNDANT) { set_error("tree %d: needs a compressed (redundant) tree", b); return MRA_ESTATE; }
        if (t->nlev - 1 > op->J) { set_error("tree %d: depth %d exceeds operator max_level %d", b, t->nlev - 1, op->J); return MRA_EINVAL; }
        total += t->n;
        lm = std::max(lm, t->nlev);
    }
    if (total >= (1ll << 31) / 216) { set_error("too many nodes in the batch (%lld)", total); return MRA_EINVAL; }
    cudaStream_t st = (cudaStream_t)stream;
    mra_plan* p = new mra_plan();
    p->magic = MRA_PLAN_MAGIC;
    p->op = op;
    p->k = op->k;
    p->ntrees = ntrees;
    p->n = (int)total;
    p->lm = lm;
    p->precision = prec;
    p->tc = tc;
    p->use_graph = opts ? (opts->use_graph != 0) : 1;
    p->screen_mode = opts ? opts->screen_mode : MRA_SCREEN_STATIC;
    p->schedule = opts ? opts->schedule : nullptr;
    p->margin = opts ? std::max(0, opts->margin) : 0;
    if (p->screen_mode != MRA_SCREEN_STATIC && p->screen_mode != MRA_SCREEN_PAIR &&
        p->screen_mode != MRA_SCREEN_LEARNED) {
        set_error("screen mode %d is not available", p->screen_mode);
        delete p;
        return MRA_EINVAL;
    }
    if (p->screen_mode == MRA_SCREEN_LEARNED && !p->schedule) {
        set_error("the learned screen needs a network handle (mra_plan_opts.schedule)");
        delete p;
        return MRA_EINVAL;
    }
    p->A = trees[0]->A;
    p->A.stream = st;
    p->trees.assign(trees, trees + ntrees);
    p->base.assign(ntrees + 1, 0);
    for (int b = 0; b < ntrees; ++b) p->base[b + 1] = p->base[b] + trees[b]->n;
    p->off_host.assign((size_t)ntrees * (lm + 1), 0);
    p->nlev_host.assign(ntrees, 0);
    int rc = plan_build(p, st);
    if (rc != MRA_OK) {
        cudaStreamSynchronize(st);
        plan_release(p);
        return rc;
    }
    *out = p;
    return MRA_OK;
}

int mra_plan_execute(mra_plan* p, void* stream) {
    if (!plan_ok(p)) { set_error("invalid plan handle"); return MRA_EINVAL; }
    cudaStream_t st = (cudaStream_t)stream;
    p->executes++;
    if (!p->use_graph) return plan_enqueue(p, st);
    if (!p->gexec) {
        const unsigned long long before = mra_kernel_launches();
        MRA_CK(cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal));
        const int rc = plan_enqueue(p, p->cap);
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(p->cap, &g);
        if (rc != MRA_OK) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (e != cudaSuccess) { set_error("graph capture: %s", cudaGetErrorString(e)); return MRA_ECUDA; }
        p->graph = g;
        MRA_CK(cudaGraphInstantiate(&p->gexec, p->graph, 0));
        // the captured launches run when the graph does
        p->graph_kernels = (long long)(mra_kernel_launches() - before);
        count_launch_add(-p->graph_kernels);
    }
    MRA_CK(cudaGraphLaunch(p->gexec, st));
    count_launch_add(p->graph_kernels);
    return MRA_OK;
}

int mra_plan_autotune(mra_plan* p, int reps, void* stream) {
    if (!plan_ok(p)) { set_error("invalid plan handle"); return MRA_EINVAL; }
    if (reps < 1) { set_error("reps must be >= 1"); return MRA_EINVAL; }
    if (!p->tc) return MRA_OK;  // one variant only
    cudaStream_t st = (cudaStream_t)stream;
    plan_drop_graph(p);
    // operands of the current blocks, then each variant timed on its own
    const int k3 = p->k * p->k * p->k;
    const size_t total = (size_t)p->n * k3;
    const int nb = (int)std::max<size_t>(1, std::min<size_t>(num_sms() * 8, (total + 255) / 256));
    k_forest_blocks<<<nb, 256, 0, st>>>(p->n, k3, p->dbase, p->node_tree, p->tref, p->s);
    MRA_CK_LAUNCH();
    MRA_TRY(ghost_refine_forest(p->F, p->S, p->gblk, st,
                                p->precision == MRA_PREC_TC_FAST && p->screen_mode == MRA_SCREEN_STATIC));
    MRA_TRY(tc_prep_blocks(p->n + p->S.nghost, p->k, p->n, p->s, p->gblk, p->tcb, st));
    cudaEvent_t e0, e1;
    MRA_CK(cudaEventCreate(&e0));
    MRA_CK(cudaEventCreate(&e1));
    float best = 1e30f;
    // (terms per chunk, CTAs per SM)
    static const int kMC[5] = {8, 8, 4, 4, 4}, kCTA[5] = {3, 2, 3, 2, 4};
    for (int v = 0; v < MRA_PLAN_VARIANTS; ++v) {
        const int mc = kMC[v % 5], ctas = kCTA[v % 5], ord = v / 5;
        MRA_TRY(plan_tc_launch(p, mc, ctas, ord, st));  // warm-up
        MRA_CK(cudaEventRecord(e0, st));
        for (int r = 0; r < reps; ++r) MRA_TRY(plan_tc_launch(p, mc, ctas, ord, st));
        MRA_CK(cudaEventRecord(e1, st));
        MRA_CK(cudaEventSynchronize(e1));
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= reps;
        p->ms_variant[v] = ms;
        if (ms < best) {
            best = ms;
            p->mc = mc;
            p->ctas = ctas;
            p->use_order = ord;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    p->tuned = 1;
    return MRA_OK;
}

int mra_plan_set_variant(mra_plan* p, int mc, int ctas_per_sm, int heavy_first) {
    if (!plan_ok(p)) { set_error("invalid plan handle"); return MRA_EINVAL; }
    if ((mc != 4 && mc != 8) || ctas_per_sm < 1 || ctas_per_sm > (mc == 4 ? 4 : 3)) {
        set_error("variant: terms per chunk 8 with 1 to 3 CTAs per SM, or 4 with 1 to 4");
        return MRA_EINVAL;
    }
    plan_drop_graph(p);
    p->mc = mc;
    p->ctas = ctas_per_sm;
    p->use_order = heavy_first ? 1 : 0;
    return MRA_OK;
}

int mra_plan_output(const mra_plan* p, int b, void* stream, mra_tree** g_ns) {
    if (!g_ns) { set_error("g_ns is NULL"); return MRA_EINVAL; }
    *g_ns = nullptr;
    if (!plan_ok(p)) { set_error("invalid plan handle"); return MRA_EINVAL; }
    if (b < 0 || b >= p->ntrees) { set_error("tree index %d outside [0, %d)", b, p->ntrees); return MRA_EINVAL; }
    const mra_tree* f = p->trees[b];
    mra_tree* g = nullptr;
    MRA_TRY(tree_clone_skeleton(f, &g));
    g->state = MRA_TREE_NSFORM;
    const size_t k3 = (size_t)p->k * p->k * p->k;
    cudaError_t e = cudaMemcpyAsync(g->s, p->out + (size_t)p->base[b] * k3, (size_t)f->n * k3 * sizeof(double),
                                    cudaMemcpyDeviceToDevice, (cudaStream_t)stream);
    if (e != cudaSuccess) {
        set_error("plan output copy: %s", cudaGetErrorString(e));
        mra_free_tree(g);
        return MRA_ECUDA;
    }
    *g_ns = g;
    return MRA_OK;
}

int mra_plan_get_info(const mra_plan* p, mra_plan_info* info, void* stream) {
    if (!plan_ok(p) || !info) { set_error("invalid plan handle"); return MRA_EINVAL; }
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<unsigned long long> ni(p->ntrees + 1);
    int32_t herr[2] = {0, 0};
    MRA_CK(cudaMemcpyAsync(ni.data(), p->nitems, (p->ntrees + 1) * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                           st));
    MRA_CK(cudaMemcpyAsync(herr, p->S.err, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    MRA_CK(cudaStreamSynchronize(st));
    memset(info, 0, sizeof(*info));
    info->n_trees = p->ntrees;
    info->n_nodes = p->n;
    info->n_pairs = p->S.npairs;
    info->n_ghosts = p->S.nghost;
    for (int b = 0; b < p->ntrees; ++b) info->n_items += (int64_t)ni[b];
    info->n_items_lowp = (int64_t)ni[p->ntrees];
    info->precision = p->precision;
    info->terms_per_chunk = p->mc;
    info->ctas_per_sm = p->ctas;
    info->heavy_first = p->use_order;
    info->tuned = p->tuned;
    for (int v = 0; v < MRA_PLAN_VARIANTS; ++v) info->ms_variant[v] = p->ms_variant[v];
    info->graph = p->gexec != nullptr;
    info->graph_kernels = (int)p->graph_kernels;
    info->ms_screen = p->ms_screen;
    info->screen_mode = p->screen_mode;
    info->n_misses = p->n_misses;
    info->n_pairs_empty = p->n_pairs_empty;
    if (herr[1] == 4) { set_error("tensor-core apply: an MMA completion wait reached its limit"); return MRA_ETIMEOUT; }
    if (herr[1] == 5) { set_error("tensor-core apply: an output scale is outside the FP32 range (use fp64)"); return MRA_EINVAL; }
    if (herr[0] || herr[1]) { set_error("screen/Step-2 error code %d/%d", herr[0], herr[1]); return MRA_ECUDA; }
    return MRA_OK;
}

int mra_plan_tree_stats(const mra_plan* p, int b, void* stream, mra_apply_stats* st) {
    if (!plan_ok(p) || !st) { set_error("invalid plan handle"); return MRA_EINVAL; }
    if (b < 0 || b >= p->ntrees) { set_error("tree index %d outside [0, %d)", b, p->ntrees); return MRA_EINVAL; }
    cudaStream_t s = (cudaStream_t)stream;
    double dv[3];
    unsigned long long ni = 0;
    int32_t po[2];
    MRA_CK(cudaMemcpyAsync(dv, p->S.dv + 4 * (size_t)b, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
    MRA_CK(cudaMemcpyAsync(&ni, p->nitems + b, sizeof(ni), cudaMemcpyDeviceToHost, s));
    MRA_CK(cudaMemcpyAsync(&po[0], p->S.pair_off + p->base[b], sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    MRA_CK(cudaMemcpyAsync(&po[1], p->S.pair_off + p->base[b + 1], sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    MRA_CK(cudaStreamSynchronize(s));
    memset(st, 0, sizeof(*st));
    st->n_pairs = po[1] - po[0];
    st->n_items = (int64_t)ni;
    st->n_ghosts = -1;  // Step-2 blocks are counted for the whole batch (mra_plan_get_info)
    st->n_out_nodes = p->base[b + 1] - p->base[b];
    st->fnorm = sqrt(dv[0]);
    st->sigma = dv[1];
    st->eta = dv[2];
    return MRA_OK;
}

int mra_free_plan(mra_plan* p) {
    if (!p) return MRA_OK;
    if (!plan_ok(p)) { set_error("invalid plan handle"); return MRA_EINVAL; }
    cudaStreamSynchronize(p->A.stream);
    plan_release(p);
    return MRA_OK;
}

}  // extern "C"
