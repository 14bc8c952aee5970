// C ABI entry points (declared in include/mra_gb300.h): argument checks,
// handle ownership, allocator hook and per-thread error messages.  All
// arithmetic is done by the kernels in operator.cu, tree.cu, apply*.cu and product.cu.
#include <stdarg.h>

#include <atomic>
#include <cmath>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "mra_internal.cuh"

namespace mra {

static thread_local char g_err[512] = "";
static std::atomic<unsigned long long> g_launches(0);

int num_sms() {
    static std::atomic<int> cache[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) {
        cudaGetLastError();
        dev = 0;
    }
    std::atomic<int>& c = cache[dev & 63];
    int v = c.load(std::memory_order_relaxed);
    if (v <= 0) {
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) {
            cudaGetLastError();
            v = 1;
        }
        c.store(v, std::memory_order_relaxed);
    }
    return v;
}

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void count_launch_add(long long n) { g_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed); }

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

// ---------------------------------------------------------------- block cache
// Stream-ordered cache in front of the allocator hook (or cudaMallocAsync): a
// block the library frees is kept under (hook, stream, size) and handed out
// again to the next request with the same hook, stream and size.  Every use of
// a block is ordered on its stream, so reuse on that stream needs no event, and
// nothing is reused across streams or hooks.  A step of the method allocates the
// same sizes every time, so after the first step no call reaches the hook (each
// hook call can be a round trip into an interpreter).  At most kCacheLimit bytes
// are kept; mra_release_cached() returns every cached block to its hook.
namespace {
struct CacheKey {
    void* alloc_fn;
    void* free_fn;
    void* ctx;
    void* stream;
    size_t bytes;
    bool operator==(const CacheKey& o) const {
        return alloc_fn == o.alloc_fn && free_fn == o.free_fn && ctx == o.ctx && stream == o.stream &&
               bytes == o.bytes;
    }
};
struct CacheKeyHash {
    size_t operator()(const CacheKey& k) const {
        size_t h = std::hash<void*>()(k.alloc_fn);
        for (const void* q : {k.free_fn, k.ctx, k.stream}) h = h * 1000003u ^ std::hash<const void*>()(q);
        return h * 1000003u ^ std::hash<size_t>()(k.bytes);
    }
};
struct BlockCache {
    std::mutex mu;
    std::unordered_map<CacheKey, std::vector<void*>, CacheKeyHash> free_blocks;
    std::unordered_map<void*, CacheKey> live;  // blocks handed out: their key
    size_t cached_bytes = 0;
};
constexpr size_t kCacheLimit = (size_t)4 << 30;
BlockCache& block_cache() {
    static BlockCache* c = new BlockCache();  // never destroyed: frees may run at exit
    return *c;
}
void raw_free(const CacheKey& k, void* p) {
    if (k.free_fn) {
        auto fn = (void (*)(void*, void*, void*))k.free_fn;
        fn(p, k.stream, k.ctx);
    } else {
        cudaFreeAsync(p, (cudaStream_t)k.stream);
    }
}
}  // namespace

void* Alloc::get(size_t bytes) const {
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) / 256 * 256;
    const CacheKey key{has ? (void*)hook.alloc : nullptr, has ? (void*)hook.free : nullptr, has ? hook.ctx : nullptr,
                       (void*)stream, bytes};
    BlockCache& C = block_cache();
    {
        std::lock_guard<std::mutex> lk(C.mu);
        auto it = C.free_blocks.find(key);
        if (it != C.free_blocks.end() && !it->second.empty()) {
            void* p = it->second.back();
            it->second.pop_back();
            C.cached_bytes -= bytes;
            C.live.emplace(p, key);
            return p;
        }
    }
    void* p = nullptr;
    if (has) {
        p = hook.alloc(bytes, (void*)stream, hook.ctx);
    } else if (cudaMallocAsync(&p, bytes, stream) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) {
        std::lock_guard<std::mutex> lk(C.mu);
        C.live.emplace(p, key);
    }
    return p;
}

void Alloc::put(void* p) const {
    if (!p) return;
    BlockCache& C = block_cache();
    CacheKey key{};
    {
        std::lock_guard<std::mutex> lk(C.mu);
        auto it = C.live.find(p);
        if (it != C.live.end()) {
            key = it->second;
            C.live.erase(it);
            if (C.cached_bytes + key.bytes <= kCacheLimit) {
                C.free_blocks[key].push_back(p);
                C.cached_bytes += key.bytes;
                return;
            }
        } else {  // not from Alloc::get: straight back to the hook
            key = CacheKey{has ? (void*)hook.alloc : nullptr, has ? (void*)hook.free : nullptr,
                           has ? hook.ctx : nullptr, (void*)stream, 0};
        }
    }
    raw_free(key, p);
}

size_t release_cached() {
    BlockCache& C = block_cache();
    std::vector<std::pair<CacheKey, void*>> out;
    {
        std::lock_guard<std::mutex> lk(C.mu);
        for (auto& kv : C.free_blocks)
            for (void* p : kv.second) out.emplace_back(kv.first, p);
        C.free_blocks.clear();
        C.cached_bytes = 0;
    }
    size_t bytes = 0;
    for (auto& e : out) {
        raw_free(e.first, e.second);
        bytes += e.first.bytes;
    }
    return bytes;
}

Alloc make_alloc(const mra_alloc* a, void* stream) {
    Alloc A;
    A.stream = (cudaStream_t)stream;
    if (a && a->alloc && a->free) {
        A.hook = *a;
        A.has = true;
    }
    return A;
}

static bool tree_ok(const mra_tree* t) { return t && t->magic == MRA_TREE_MAGIC; }
static bool op_ok(const mra_op* o) { return o && o->magic == MRA_OP_MAGIC; }

}  // namespace mra

using namespace mra;

extern "C" {

const char* mra_last_error(void) { return g_err; }
const char* mra_version(void) { return "mra_gb300 0.1 (sm_103a)"; }
unsigned long long mra_kernel_launches(void) { return g_launches.load(); }
size_t mra_release_cached(void) { return release_cached(); }

int mra_build_tree(const mra_density* f, int k, double eps, int max_level, int uniform_level, int init_level,
                   const mra_alloc* alloc, void* stream, mra_tree** out) {
    if (!out) { set_error("out is NULL"); return MRA_EINVAL; }
    *out = nullptr;
    if (!f || f->n <= 0 || !f->coef_host || !f->expo_host || !f->center_host) {
        set_error("empty or NULL density");
        return MRA_EINVAL;
    }
    if (k < 1 || k > MRA_MAX_K) { set_error("k=%d outside [1, %d]", k, MRA_MAX_K); return MRA_EINVAL; }
    if (!(eps > 0.0)) { set_error("eps must be > 0"); return MRA_EINVAL; }
    if (max_level < 0 || max_level > MRA_MAX_LEVEL) { set_error("max_level outside [0, %d]", MRA_MAX_LEVEL); return MRA_EINVAL; }
    for (int g = 0; g < f->n; ++g)
        if (!(f->expo_host[g] > 0.0)) { set_error("density exponent %d is not positive", g); return MRA_EINVAL; }
    Alloc A = make_alloc(alloc, stream);
    return build_tree_impl(f, k, eps, max_level, uniform_level, init_level, A, out);
}

int mra_tree_import(int k, int n, const int32_t* coords_host, const int32_t* leaf_host, const double* blocks_host,
                    const mra_alloc* alloc, void* stream, mra_tree** out) {
    if (!out) { set_error("out is NULL"); return MRA_EINVAL; }
    *out = nullptr;
    if (k < 1 || k > MRA_MAX_K || n < 1 || !coords_host || !leaf_host || !blocks_host) {
        set_error("invalid import arguments");
        return MRA_EINVAL;
    }
    mra_tree* t = new mra_tree();
    t->magic = MRA_TREE_MAGIC;
    t->k = k;
    t->A = make_alloc(alloc, stream);
    t->state = MRA_TREE_LEAVES;
    t->depth_hit = 0;
    int rc = tree_alloc_arrays(t, n, true);
    if (rc == MRA_OK) {
        // the blocks first: from pinned memory the copy runs while the host links the
        // node list below (which ends with a synchronisation of the stream)
        const size_t bytes = (size_t)n * k * k * k * sizeof(double);
        cudaError_t e = cudaMemcpyAsync(t->s, blocks_host, bytes, cudaMemcpyHostToDevice, t->A.stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(t->dnorm, 0, n * sizeof(double), t->A.stream);
        if (e != cudaSuccess) { set_error("import copy: %s", cudaGetErrorString(e)); rc = MRA_ECUDA; }
    }
    if (rc == MRA_OK) rc = tree_link_and_upload(t, coords_host, leaf_host);
    if (rc != MRA_OK) {
        cudaStreamSynchronize(t->A.stream);  // no copy still reads the caller's buffers
        cudaGetLastError();
        tree_free_arrays(t);
        t->A.put(t->filt);
        t->magic = 0;
        delete t;
        return rc;
    }
    *out = t;
    return MRA_OK;
}

int mra_tree_export(const mra_tree* t, int32_t* coords_host, int32_t* leaf_host, double* blocks_host,
                    double* dnorm_host, void* stream) {
    if (!tree_ok(t)) { set_error("invalid tree handle"); return MRA_EINVAL; }
    cudaStream_t st = (cudaStream_t)stream;
    const int n = t->n;
    if (coords_host) MRA_CK(cudaMemcpyAsync(coords_host, t->a.coord, 4 * (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    if (leaf_host) MRA_CK(cudaMemcpyAsync(leaf_host, t->a.leaf, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    if (blocks_host) MRA_CK(cudaMemcpyAsync(blocks_host, t->s, (size_t)n * t->k * t->k * t->k * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (dnorm_host) MRA_CK(cudaMemcpyAsync(dnorm_host, t->dnorm, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, st));
    MRA_CK(cudaStreamSynchronize(st));
    return MRA_OK;
}

int mra_tree_get_info(const mra_tree* t, mra_tree_info* info) {
    if (!tree_ok(t) || !info) { set_error("invalid tree handle"); return MRA_EINVAL; }
    info->k = t->k;
    info->n_nodes = t->n;
    info->n_levels = t->nlev;
    info->state = t->state;
    info->depth_hit = t->depth_hit;
    memcpy(info->level_offset, t->off, sizeof(t->off));
    return MRA_OK;
}

int mra_tree_device_arrays(const mra_tree* t, double** blocks, int32_t** leaf) {
    if (!tree_ok(t)) { set_error("invalid tree handle"); return MRA_EINVAL; }
    if (blocks) *blocks = t->s;
    if (leaf) *leaf = t->a.leaf;
    return MRA_OK;
}

int mra_tree_set_blocks(mra_tree* t, const double* blocks, void* stream) {
    if (!tree_ok(t) || !blocks) { set_error("invalid tree handle or blocks"); return MRA_EINVAL; }
    MRA_CK(cudaMemcpyAsync(t->s, blocks, (size_t)t->n * t->k * t->k * t->k * sizeof(double),
                           cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    return MRA_OK;
}

int mra_tree_refine(const mra_tree* f, int passes, int max_level, void* stream, mra_tree** out,
                    int* n_split_host) {
    if (!out) { set_error("out is NULL"); return MRA_EINVAL; }
    *out = nullptr;
    if (!tree_ok(f)) { set_error("invalid tree handle"); return MRA_EINVAL; }
    if (passes < 0 || passes > 8) { set_error("passes must lie in [0, 8]"); return MRA_EINVAL; }
    if (max_level < 0 || max_level > MRA_MAX_LEVEL) { set_error("max_level outside [0, %d]", MRA_MAX_LEVEL); return MRA_EINVAL; }
    if (f->state == MRA_TREE_NSFORM) { set_error("refine needs leaf data, not an ns-form tree"); return MRA_ESTATE; }
    return refine_impl(f, passes, max_level, (cudaStream_t)stream, out, n_split_host);
}

static bool all_finite(const double* p, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(p[i])) return false;
    return true;
}

int mra_tree_multiply(const mra_tree* f, const mra_potential* v, double scale, void* stream, mra_tree** out) {
    if (!out) { set_error("out is NULL"); return MRA_EINVAL; }
    *out = nullptr;
    if (!tree_ok(f)) { set_error("invalid tree handle"); return MRA_EINVAL; }
    if (!v || v->n_gauss < 0 || v->n_charge < 0 || v->n_gauss + v->n_charge == 0) {
        set_error("the potential has no terms");
        return MRA_EINVAL;
    }
    if (v->n_gauss > 0 && (!v->coef_host || !v->expo_host || !v->center_host)) {
        set_error("a Gaussian array of the potential is NULL");
        return MRA_EINVAL;
    }
    if (v->n_charge > 0 && (!v->charge_host || !v->position_host)) {
        set_error("a charge array of the potential is NULL");
        return MRA_EINVAL;
    }
    const size_t ng = v->n_gauss, nc = v->n_charge;
    if (!std::isfinite(scale) || (ng && !(all_finite(v->coef_host, ng) && all_finite(v->expo_host, ng) &&
                                          all_finite(v->center_host, 3 * ng) &&
                                          (!v->r2coef_host || all_finite(v->r2coef_host, ng)))) ||
        (nc && !(all_finite(v->charge_host, nc) && all_finite(v->position_host, 3 * nc)))) {
        set_error("non-finite potential parameter or scale");
        return MRA_EINVAL;
    }
    for (size_t g = 0; g < ng; ++g)
        if (v->expo_host[g] < 0.0) { set_error("exponent %zu is negative", g); return MRA_EINVAL; }
    if (f->state == MRA_TREE_NSFORM) { set_error("multiply needs leaf data, not an ns-form tree"); return MRA_ESTATE; }
    return tree_multiply_impl(f, v, scale, (cudaStream_t)stream, out);
}

int mra_tree_dot(const mra_tree* a, const mra_tree* b, void* stream, double* out_host) {
    if (!out_host) { set_error("out_host is NULL"); return MRA_EINVAL; }
    if (!tree_ok(a) || !tree_ok(b)) { set_error("invalid tree handle"); return MRA_EINVAL; }
    if (a->k != b->k || a->n != b->n || memcmp(a->off, b->off, sizeof(a->off)) != 0) {
        set_error("the two trees have different skeletons");
        return MRA_EINVAL;
    }
    if (a->state == MRA_TREE_NSFORM || b->state == MRA_TREE_NSFORM) {
        set_error("dot needs leaf data, not an ns-form tree");
        return MRA_ESTATE;
    }
    return tree_dot_impl(a, b, out_host, (cudaStream_t)stream);
}

int mra_tree_scale(mra_tree* t, double alpha, void* stream) {
    if (!tree_ok(t)) { set_error("invalid tree handle"); return MRA_EINVAL; }
    if (!std::isfinite(alpha)) { set_error("alpha is not finite"); return MRA_EINVAL; }
    return tree_scale_impl(t, alpha, (cudaStream_t)stream);
}

int mra_op_retune(mra_op* op, double mu, void* stream) {
    if (!op_ok(op)) { set_error("invalid operator handle"); return MRA_EINVAL; }
    if (!(mu >= 0.0) || !std::isfinite(mu)) { set_error("mu must be finite and >= 0"); return MRA_EINVAL; }
    return retune_operator(op, mu, (cudaStream_t)stream);
}

int mra_kalos_step(const mra_tree* phi, const mra_potential* v, double length, double mu, double eps, int max_level,
                   const mra_apply_opts* opts, mra_op** op_cache, void* stream, mra_tree** phi_next,
                   mra_kalos_info* info) {
    if (!phi_next) { set_error("phi_next is NULL"); return MRA_EINVAL; }
    *phi_next = nullptr;
    if (!tree_ok(phi)) { set_error("invalid tree handle"); return MRA_EINVAL; }
    if (!(length > 0.0 && std::isfinite(length)) || !(mu > 0.0 && std::isfinite(mu))) {
        set_error("length and mu must be positive and finite");
        return MRA_EINVAL;
    }
    // every handle made here is freed on every return
    struct Owned {
        mra_tree *P = nullptr, *g = nullptr, *Q = nullptr;
        mra_op* op = nullptr;
        ~Owned() {
            mra_free_tree(P);
            mra_free_tree(g);
            mra_free_tree(Q);
            mra_free_op(op);
        }
    } o;
    if (op_cache && *op_cache && !op_ok(*op_cache)) { set_error("op_cache holds no operator"); return MRA_EINVAL; }
    MRA_TRY(mra_tree_multiply(phi, v, 1.0, stream, &o.P));                          // Step 2
    mra_op* op = op_cache ? *op_cache : nullptr;
    int rebuilt = 0, reuse = 0;
    if (op && op->d == 3 && op->k == phi->k && op->eps == eps && op->J == max_level && op->alpha == 1.0) {
        // a grid that fails the sup-norm test for this mu is rebuilt; any other error is returned
        const int rc = retune_operator(op, mu * length, (cudaStream_t)stream);
        if (rc != MRA_OK && rc != MRA_EINVAL) return rc;
        reuse = rc == MRA_OK;
    }
    if (!reuse) {
        MRA_TRY(mra_make_operator(mu * length, 1.0, eps, phi->k, max_level, phi->A.has ? &phi->A.hook : nullptr,
                                  stream, &o.op));
        rebuilt = 1;
        if (op_cache) {  // the cache takes the new operator
            mra_free_op(*op_cache);
            *op_cache = o.op;
            o.op = nullptr;
        }
    }
    if (!rebuilt) op = *op_cache;
    else op = op_cache ? *op_cache : o.op;
    MRA_TRY(mra_compress(o.P, MRA_COMPRESS_SCALING, stream));                       // Step 3
    mra_apply_stats st{};
    MRA_TRY(mra_apply_ns(op, o.P, opts, stream, &o.g, &st));
    MRA_TRY(assemble_impl(o.g, (cudaStream_t)stream));  // eq. g_assemble; leaf data only
    MRA_TRY(mra_tree_scale(o.g, -2.0 * length * length, stream));
    MRA_TRY(mra_tree_multiply(o.g, v, 1.0, stream, &o.Q));                          // Step 4
    // <phi_new, phi_new>, <P, phi_new>, <V phi_new, phi_new>: one pass (the four trees share
    // phi's skeleton by construction)
    double d3[3] = {0.0, 0.0, 0.0};
    {
        const mra_tree* da[3] = {o.g, o.P, o.Q};
        const mra_tree* db[3] = {o.g, o.g, o.g};
        MRA_TRY(tree_dot3_impl(da, db, d3, (cudaStream_t)stream));
    }
    const double nn = d3[0], pg = d3[1], qg = d3[2];
    if (!(nn > 0.0)) { set_error("phi_new vanishes"); return MRA_EINVAL; }
    const double E = (-pg - 0.5 * mu * mu * nn + qg) / nn;
    const double norm = std::sqrt(nn * length * length * length);
    MRA_TRY(mra_tree_scale(o.g, 1.0 / norm, stream));                               // Step 5
    MRA_CK(cudaStreamSynchronize((cudaStream_t)stream));
    if (info) {
        info->energy = E;
        info->mu_next = E < 0.0 ? std::sqrt(-2.0 * E) : mu;
        info->norm_new = norm;
        info->n_terms = op->M;
        info->op_rebuilt = rebuilt;
        info->n_items = st.n_items;
        info->ms_apply = st.ms_screen + st.ms_ghost + st.ms_apply;
    }
    *phi_next = o.g;
    o.g = nullptr;
    return MRA_OK;
}

int mra_compress(mra_tree* t, int mode, void* stream) {
    if (!tree_ok(t)) { set_error("invalid tree handle"); return MRA_EINVAL; }
    if (t->state == MRA_TREE_NSFORM) { set_error("compress needs leaf data; assemble an ns-form tree first"); return MRA_ESTATE; }
    if (mode != MRA_COMPRESS_NORMS && mode != MRA_COMPRESS_STORE_D && mode != MRA_COMPRESS_SCALING) {
        set_error("compress mode %d is not one of MRA_COMPRESS_NORMS, _STORE_D, _SCALING", mode);
        return MRA_EINVAL;
    }
    return compress_impl(t, mode, (cudaStream_t)stream);
}

// the operator in R^d (d = 3; d = 2 for the two-dimensional variant)
static int make_operator_d(int d, double mu, double alpha, double eps, int k, int max_level, const mra_alloc* alloc,
                           void* stream, mra_op** out) {
    if (!out) { set_error("out is NULL"); return MRA_EINVAL; }
    *out = nullptr;
    if (!(mu >= 0.0)) { set_error("mu must be >= 0"); return MRA_EINVAL; }
    if (!(alpha > 0.0 && alpha < 0.5 * d)) { set_error("alpha must lie in (0, %d/2)", d); return MRA_EINVAL; }
    if (!(eps > 0.0 && eps <= 0.5)) { set_error("eps must lie in (0, 0.5]"); return MRA_EINVAL; }
    if (k < 1 || k > MRA_MAX_K) { set_error("k=%d outside [1, %d]", k, MRA_MAX_K); return MRA_EINVAL; }
    if (max_level < 0 || max_level > MRA_MAX_LEVEL) { set_error("max_level outside [0, %d]", MRA_MAX_LEVEL); return MRA_EINVAL; }
    mra_op* op = new mra_op();
    op->magic = MRA_OP_MAGIC;
    op->k = k;
    op->J = max_level;
    op->mu = mu;
    op->alpha = alpha;
    op->eps = eps;
    op->d = d;
    op->A = make_alloc(alloc, stream);
    int rc = build_operator(op, (cudaStream_t)stream);
    if (rc == MRA_OK) {
        cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
        if (e != cudaSuccess) { set_error("make_operator: %s", cudaGetErrorString(e)); rc = MRA_ECUDA; }
    }
    if (rc != MRA_OK) {
        mra_free_op(op);
        return rc;
    }
    *out = op;
    return MRA_OK;
}

int mra_make_operator(double mu, double alpha, double eps, int k, int max_level, const mra_alloc* alloc, void* stream,
                      mra_op** out) {
    return make_operator_d(3, mu, alpha, eps, k, max_level, alloc, stream, out);
}

int mra_make_operator2(double mu, double alpha, double eps, int k, int max_level, const mra_alloc* alloc,
                       void* stream, mra_op** out) {
    if (!(alpha < 1.0)) {
        if (out) *out = nullptr;
        set_error("the d = 2 operator needs alpha in (0, 1)");
        return MRA_EINVAL;
    }
    return make_operator_d(2, mu, alpha, eps, k, max_level, alloc, stream, out);
}

int mra_op_get_info(const mra_op* op, mra_op_info* info) {
    if (!op_ok(op) || !info) { set_error("invalid operator handle"); return MRA_EINVAL; }
    info->M = op->M;
    info->k = op->k;
    info->max_level = op->J;
    info->mu = op->mu;
    info->alpha = op->alpha;
    info->eps = op->eps;
    return MRA_OK;
}

int mra_op_export(const mra_op* op, double* w_host, double* tau_host, double* F_host, double* nF_host,
                  double* est_host, void* stream) {
    if (!op_ok(op)) { set_error("invalid operator handle"); return MRA_EINVAL; }
    cudaStream_t st = (cudaStream_t)stream;
    const size_t JM = (size_t)(op->J + 1) * op->M;
    if (w_host) MRA_CK(cudaMemcpyAsync(w_host, op->w, op->M * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (tau_host) MRA_CK(cudaMemcpyAsync(tau_host, op->tau, op->M * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (F_host) MRA_CK(cudaMemcpyAsync(F_host, op->F, JM * 7 * op->k * op->k * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (nF_host) MRA_CK(cudaMemcpyAsync(nF_host, op->nF, JM * 7 * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (est_host) MRA_CK(cudaMemcpyAsync(est_host, op->est, JM * sizeof(double), cudaMemcpyDeviceToHost, st));
    MRA_CK(cudaStreamSynchronize(st));
    return MRA_OK;
}

int mra_apply_ns(const mra_op* op, const mra_tree* f, const mra_apply_opts* opts, void* stream, mra_tree** g_ns,
                 mra_apply_stats* stats) {
    if (!g_ns) { set_error("g_ns is NULL"); return MRA_EINVAL; }
    *g_ns = nullptr;
    if (!op_ok(op) || !tree_ok(f)) { set_error("invalid operator or tree handle"); return MRA_EINVAL; }
    if (op->d != 3) { set_error("the operator is for d = 2 (use the d = 2 entry points)"); return MRA_EINVAL; }
    return apply_impl(op, f, opts, (cudaStream_t)stream, g_ns, stats);
}

int mra_apply_ns_noalloc(const mra_op* op, const mra_tree* f, int precision, double* ghat_out, void* stream,
                         int64_t* n_items_host) {
    if (!op_ok(op) || !tree_ok(f)) { set_error("invalid operator or tree handle"); return MRA_EINVAL; }
    if (op->d != 3) { set_error("the operator is for d = 2 (use the d = 2 entry points)"); return MRA_EINVAL; }
    return apply_noalloc_impl(op, f, precision, ghat_out, (cudaStream_t)stream, n_items_host);
}

int mra_screen_data(const mra_op* op, const mra_tree* f, float* inputs, float* targets, void* stream) {
    if (!op_ok(op) || !tree_ok(f)) { set_error("invalid operator or tree handle"); return MRA_EINVAL; }
    if (op->d != 3) { set_error("the operator is for d = 2 (use the d = 2 entry points)"); return MRA_EINVAL; }
    return screen_data_impl(op, f, inputs, targets, (cudaStream_t)stream);
}

int mra_reconstruct(mra_tree* t, int mode, int truncate, double eps, void* stream, double* truncation_l2_host) {
    if (!tree_ok(t)) { set_error("invalid tree handle"); return MRA_EINVAL; }
    cudaStream_t st = (cudaStream_t)stream;
    if (truncation_l2_host) *truncation_l2_host = 0.0;
    if (mode == MRA_RECON_ASSEMBLE) {
        if (t->state != MRA_TREE_NSFORM) { set_error("assemble needs an ns-form tree"); return MRA_ESTATE; }
        MRA_TRY(assemble_impl(t, st));
        MRA_TRY(compress_impl(t, MRA_COMPRESS_NORMS, st));
        if (truncate) {
            if (!(eps > 0.0)) { set_error("truncation eps must be > 0"); return MRA_EINVAL; }
            MRA_TRY(truncate_impl(t, eps, st, truncation_l2_host));
        }
        return MRA_OK;
    }
    if (mode == MRA_RECON_INVERSE) {
        if (t->state != MRA_TREE_REDUNDANT) { set_error("inverse needs a compressed tree"); return MRA_ESTATE; }
        return inverse_impl(t, st);
    }
    set_error("unknown reconstruct mode %d", mode);
    return MRA_EINVAL;
}

int mra_free_tree(mra_tree* t) {
    if (!t) return MRA_OK;
    if (!tree_ok(t)) { set_error("invalid tree handle"); return MRA_EINVAL; }
    tree_free_arrays(t);
    t->A.put(t->filt);
    t->magic = 0;
    delete t;
    return MRA_OK;
}

int mra_free(void* handle) {
    if (!handle) return MRA_OK;
    uint32_t tag;
    memcpy(&tag, handle, sizeof(tag));  // every handle type starts with its tag
    switch (tag) {
        case MRA_TREE_MAGIC: return mra_free_tree((mra_tree*)handle);
        case MRA_TREE2_MAGIC: return mra_free_tree2((mra_tree2*)handle);
        case MRA_OP_MAGIC: return mra_free_op((mra_op*)handle);
        case MRA_PLAN_MAGIC: return mra_free_plan((mra_plan*)handle);
        case MRA_MLP_MAGIC: return mra_mlp_free((mra_mlp*)handle);
        default: set_error("mra_free: not a live handle of this library"); return MRA_EINVAL;
    }
}

int mra_free_op(mra_op* op) {
    if (!op) return MRA_OK;
    if (op->magic != MRA_OP_MAGIC) { set_error("invalid operator handle"); return MRA_EINVAL; }
    const Alloc& A = op->A;
    A.put(op->w); A.put(op->tau); A.put(op->F); A.put(op->F32); A.put(op->nF); A.put(op->est);
    A.put(op->filt); A.put(op->scratch_i); A.put(op->rmq);
    op->magic = 0;
    delete op;
    return MRA_OK;
}

}  // extern "C"
