// The d = 2 variant of the method (Sec. 6: the apply was implemented for
// d = 2 and d = 3; Algorithm 3 as the paper illustrates it for d = 2; Sec. 4:
// three subsets Core / Boundary-1 / Boundary-2 in d = 2): quadtrees,
// Algorithm 1, the redundant tree, Algorithm 3 with Step 2, eq. g_assemble and
// the truncation in two dimensions, all FP64.  The operator tables come from
// operator.cu (built with d = 2); the 1-D blocks are the same as in d = 3.
#include <algorithm>
#include <cmath>

#include "mra_internal.cuh"

namespace mra {

// ------------------------------------------------------------ keys and reductions
__host__ __device__ inline uint64_t spread2(uint32_t v) {
    uint64_t x = v;
    x = (x | (x << 16)) & 0x0000FFFF0000FFFFull;
    x = (x | (x << 8)) & 0x00FF00FF00FF00FFull;
    x = (x | (x << 4)) & 0x0F0F0F0F0F0F0F0Full;
    x = (x | (x << 2)) & 0x3333333333333333ull;
    x = (x | (x << 1)) & 0x5555555555555555ull;
    return x;
}
// bit 2b+1 <- a1 bit b, bit 2b <- a2 bit b: child quadrant (p1 p2) appends two bits
__host__ __device__ inline uint64_t morton2(uint32_t a1, uint32_t a2) { return (spread2(a1) << 1) | spread2(a2); }

__device__ double blk2_max(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    for (int i = 0; i < nw; ++i) s = fmax(s, red[i]);
    __syncthreads();
    return s;
}

__device__ double blk2_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    for (int i = 0; i < nw; ++i) s += red[i];
    __syncthreads();
    return s;
}

struct Offs2 {
    int v[MRA_MAX_LEVEL + 2];
};

// ------------------------------------------------------------ tree arrays
static int tree2_alloc(mra_tree2* t, int n) {
    const Alloc& A = t->A;
    const size_t kk = (size_t)t->k * t->k;
    MRA_TRY(dalloc(A, &t->key, n));
    MRA_TRY(dalloc(A, &t->coord, 3 * (size_t)n));
    MRA_TRY(dalloc(A, &t->leaf, n));
    MRA_TRY(dalloc(A, &t->child, n));
    MRA_TRY(dalloc(A, &t->parent, n));
    MRA_TRY(dalloc(A, &t->s, (size_t)n * kk));
    MRA_TRY(dalloc(A, &t->dnorm, n));
    if (!t->filt) {
        MRA_TRY(dalloc(A, &t->filt, 6 * t->k * t->k));
        MRA_TRY(launch_filters(t->k, t->filt, A.stream));
    }
    t->n = n;
    return MRA_OK;
}

static void tree2_free_arrays(mra_tree2* t) {
    const Alloc& A = t->A;
    A.put(t->key); A.put(t->coord); A.put(t->leaf); A.put(t->child); A.put(t->parent);
    A.put(t->s); A.put(t->dnorm);
    t->key = nullptr; t->coord = nullptr; t->leaf = nullptr; t->child = nullptr; t->parent = nullptr;
    t->s = nullptr; t->dnorm = nullptr;
}

static mra_tree2* tree2_new(int k, const Alloc& A) {
    mra_tree2* t = new mra_tree2();
    t->magic = MRA_TREE2_MAGIC;
    t->k = k;
    t->A = A;
    t->state = MRA_TREE_LEAVES;
    t->depth_hit = 0;
    t->n = 0;
    t->nlev = 0;
    for (int j = 0; j < MRA_MAX_LEVEL + 2; ++j) t->off[j] = 0;
    return t;
}

static void tree2_delete(mra_tree2* t) {
    if (!t) return;
    tree2_free_arrays(t);
    t->A.put(t->filt);
    t->magic = 0;
    delete t;
}

// the tree is freed on every error return of the function holding the guard
struct Tree2Guard {
    mra_tree2* t;
    ~Tree2Guard() { tree2_delete(t); }
};

// host-side validation and linking of an imported node list (coords: 3n)
static int tree2_link_upload(mra_tree2* t, const int32_t* coords, const int32_t* leaf) {
    const int n = t->n;
    std::vector<uint64_t> key(n);
    std::vector<int32_t> child(n, -1), parent(n, -1), lf(n);
    int off[MRA_MAX_LEVEL + 2];
    for (int j = 0; j < MRA_MAX_LEVEL + 2; ++j) off[j] = n;
    int nlev = 0;
    for (int i = 0; i < n; ++i) {
        const int j = coords[3 * i];
        if (j < 0 || j > MRA_MAX_LEVEL) { set_error("node %d: level %d out of range", i, j); return MRA_EINVAL; }
        for (int d = 1; d < 3; ++d)
            if (coords[3 * i + d] < 0 || coords[3 * i + d] >= (1 << j)) {
                set_error("node %d: box index out of range", i);
                return MRA_EINVAL;
            }
        key[i] = morton2(coords[3 * i + 1], coords[3 * i + 2]);
        if (i > 0) {
            const int jp = coords[3 * (i - 1)];
            if (jp > j || (jp == j && key[i - 1] >= key[i])) {
                set_error("nodes not sorted by (level, Morton key) at %d", i);
                return MRA_EINVAL;
            }
        }
        if (off[j] == n) off[j] = i;
        nlev = std::max(nlev, j + 1);
        lf[i] = leaf[i] ? 1 : 0;
    }
    if (n == 0 || coords[0] != 0) { set_error("tree must start with the root (0,0,0)"); return MRA_EINVAL; }
    for (int j = nlev; j >= 0; --j)
        if (off[j] == n && j < nlev) off[j] = off[j + 1];
    for (int j = nlev; j < MRA_MAX_LEVEL + 2; ++j) off[j] = n;
    for (int i = 0; i < n; ++i) {
        const int j = coords[3 * i];
        if (lf[i]) continue;
        if (j + 1 >= nlev) { set_error("internal node %d lacks children", i); return MRA_EINVAL; }
        const uint64_t ck = key[i] << 2;
        const int lo = off[j + 1], hi = off[j + 2];
        const int pos = (int)(std::lower_bound(key.begin() + lo, key.begin() + hi, ck) - key.begin());
        if (pos + 4 > hi) { set_error("internal node %d lacks children", i); return MRA_EINVAL; }
        for (int o = 0; o < 4; ++o)
            if (key[pos + o] != ck + o) { set_error("internal node %d lacks child %d", i, o); return MRA_EINVAL; }
        child[i] = pos;
        for (int o = 0; o < 4; ++o) parent[pos + o] = i;
    }
    for (int i = 1; i < n; ++i)
        if (parent[i] < 0) { set_error("node %d has no parent", i); return MRA_EINVAL; }
    t->nlev = nlev;
    memcpy(t->off, off, sizeof(off));
    cudaStream_t st = t->A.stream;
    MRA_CK(cudaMemcpyAsync(t->key, key.data(), n * sizeof(uint64_t), cudaMemcpyHostToDevice, st));
    MRA_CK(cudaMemcpyAsync(t->coord, coords, 3 * (size_t)n * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    MRA_CK(cudaMemcpyAsync(t->leaf, lf.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    MRA_CK(cudaMemcpyAsync(t->child, child.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    MRA_CK(cudaMemcpyAsync(t->parent, parent.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    MRA_CK(cudaStreamSynchronize(st));  // host vectors go out of scope
    return MRA_OK;
}

static int tree2_clone_skeleton(const mra_tree2* src, mra_tree2** out) {
    *out = nullptr;
    mra_tree2* t = tree2_new(src->k, src->A);
    Tree2Guard g{t};
    t->nlev = src->nlev;
    t->state = src->state;
    t->depth_hit = src->depth_hit;
    memcpy(t->off, src->off, sizeof(t->off));
    cudaStream_t st = t->A.stream;
    MRA_TRY(dalloc(t->A, &t->filt, 6 * t->k * t->k));
    MRA_CK(cudaMemcpyAsync(t->filt, src->filt, 6 * t->k * t->k * sizeof(double), cudaMemcpyDeviceToDevice, st));
    MRA_TRY(tree2_alloc(t, src->n));
    const int n = src->n;
    MRA_CK(cudaMemcpyAsync(t->key, src->key, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, st));
    MRA_CK(cudaMemcpyAsync(t->coord, src->coord, 3 * (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
    MRA_CK(cudaMemcpyAsync(t->leaf, src->leaf, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
    MRA_CK(cudaMemcpyAsync(t->child, src->child, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
    MRA_CK(cudaMemcpyAsync(t->parent, src->parent, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
    g.t = nullptr;
    *out = t;
    return MRA_OK;
}

// ------------------------------------------------------------ Algorithm 1 in d = 2
struct Dens2 {
    int n;
    const double *coef, *r2, *expo, *cen;  // cen: 2 per term
};

__device__ double dens2_eval(const Dens2& D, double x, double y) {
    double f = 0.0;
    for (int g = 0; g < D.n; ++g) {
        const double dx = x - D.cen[2 * g], dy = y - D.cen[2 * g + 1];
        const double r2 = dx * dx + dy * dy;
        f += (D.coef[g] + D.r2[g] * r2) * exp(-D.expo[g] * r2);
    }
    return f;
}

__global__ void k_dens_scale2(Dens2 D, double eps, double* tol) {
    __shared__ double red[32];
    double m = 0.0;
    for (int g = threadIdx.x; g < D.n; g += blockDim.x)
        m = fmax(m, fabs(dens2_eval(D, D.cen[2 * g], D.cen[2 * g + 1])));
    m = blk2_max(m, red);
    if (threadIdx.x == 0) tol[0] = eps * m;
}

// One block per box of level j.  mode: 0 adaptive test, 1 refine, 2 leaf.
// Projection s = 2^{-j} P v P^T from the values v at the box's k x k GL nodes
// (eq. fvals2coefs); the test compares the density with the block's values at
// the 4 children's GL nodes.
__global__ void k_build_level2(int k, int j, Dens2 D, const int32_t* boxes, const double* tolp, int mode, int at_max,
                               double* s_out, int32_t* refine, int32_t* depth_hit) {
    extern __shared__ double sm[];
    const int kk = k * k;
    double* g = sm;
    double* gw = g + k;
    double* P = gw + k;   // [i][q] phi_i(g_q) w_q
    double* Q = P + kk;   // [p][q][i] phi_i((g_q + p)/2)
    double* v = Q + 2 * kk;
    double* t1 = v + kk;
    double* s = t1 + kk;
    __shared__ double red[32];
    const int b = blockIdx.x, tid = threadIdx.x;
    const int a1 = boxes[2 * b], a2 = boxes[2 * b + 1];
    if (tid < k) gauss_legendre01_root(k, tid, g, gw);
    __syncthreads();
    if (tid < k) {
        double tmp[MRA_MAX_K];
        phi_all(k, g[tid], tmp);
        for (int i = 0; i < k; ++i) P[i * k + tid] = tmp[i] * gw[tid];
        for (int p = 0; p < 2; ++p) {
            phi_all(k, 0.5 * (g[tid] + p), tmp);
            for (int i = 0; i < k; ++i) Q[p * kk + tid * k + i] = tmp[i];
        }
    }
    const double h = exp2(-(double)j);
    for (int e = tid; e < kk; e += blockDim.x) v[e] = dens2_eval(D, (g[e / k] + a1) * h, (g[e % k] + a2) * h);
    __syncthreads();
    for (int e = tid; e < kk; e += blockDim.x) {
        const int i1 = e / k, q2 = e % k;
        double acc = 0.0;
        for (int q1 = 0; q1 < k; ++q1) acc += P[i1 * k + q1] * v[q1 * k + q2];
        t1[e] = acc;
    }
    __syncthreads();
    const double sc = exp2(-(double)j);
    for (int e = tid; e < kk; e += blockDim.x) {
        const int i1 = e / k, i2 = e % k;
        double acc = 0.0;
        for (int q2 = 0; q2 < k; ++q2) acc += t1[i1 * k + q2] * P[i2 * k + q2];
        s[e] = acc * sc;
    }
    __syncthreads();
    int ref = (mode == 1);
    if (mode == 0) {
        double err = 0.0;
        const double hc = 0.5 * h, up = exp2((double)j);
        for (int o = 0; o < 4; ++o) {
            const int p1 = o >> 1, p2 = o & 1;
            for (int e = tid; e < kk; e += blockDim.x) {
                const int a = e / k, i2 = e % k;
                double acc = 0.0;
                for (int i1 = 0; i1 < k; ++i1) acc += Q[p1 * kk + a * k + i1] * s[i1 * k + i2];
                t1[e] = acc;
            }
            __syncthreads();
            for (int e = tid; e < kk; e += blockDim.x) {
                const int a = e / k, c = e % k;
                double acc = 0.0;
                for (int i2 = 0; i2 < k; ++i2) acc += t1[a * k + i2] * Q[p2 * kk + c * k + i2];
                const double f = dens2_eval(D, (g[a] + 2 * a1 + p1) * hc, (g[c] + 2 * a2 + p2) * hc);
                err = fmax(err, fabs(f - up * acc));
            }
            __syncthreads();
        }
        err = blk2_max(err, red);
        ref = err > tolp[0];
        if (ref && at_max) {
            ref = 0;
            if (tid == 0) atomicExch(depth_hit, 1);
        }
    }
    for (int e = tid; e < kk; e += blockDim.x) s_out[(size_t)b * kk + e] = s[e];
    if (tid == 0) refine[b] = ref;
}

__global__ void k_make_children2(int nb, const int32_t* boxes, const int32_t* refine, const int32_t* pos,
                                 int32_t* next, int32_t* parent_local) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb || !refine[b]) return;
    const int p = pos[b];
    parent_local[p] = b;
    for (int o = 0; o < 4; ++o) {
        const int c = 4 * p + o;
        next[2 * c] = 2 * boxes[2 * b] + (o >> 1);
        next[2 * c + 1] = 2 * boxes[2 * b + 1] + (o & 1);
    }
}

struct Tree2Dev {
    uint64_t* key;
    int32_t *coord, *leaf, *child, *parent;
    double* s;
};

__global__ void k_place_level2(int nb, int j, int base, int next_base, const int32_t* boxes, const int32_t* refine,
                               const int32_t* pos, const int32_t* parent_local, int prev_base, int kk,
                               const double* s_lvl, Tree2Dev T) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    const int i = base + b;
    T.key[i] = morton2(boxes[2 * b], boxes[2 * b + 1]);
    T.coord[3 * i] = j;
    T.coord[3 * i + 1] = boxes[2 * b];
    T.coord[3 * i + 2] = boxes[2 * b + 1];
    T.leaf[i] = refine[b] ? 0 : 1;
    T.child[i] = refine[b] ? next_base + 4 * pos[b] : -1;
    T.parent[i] = (j == 0) ? -1 : prev_base + parent_local[b / 4];
    // (the level's blocks are copied as one contiguous range by the caller)
}

static int build_tree2_impl(const mra_density* f, int k, double eps, int max_level, int uniform_level, int init_level,
                            const Alloc& A, mra_tree2** out) {
    cudaStream_t st = A.stream;
    const int kk = k * k, ng = f->n;
    Scratch tmp(A);
    double* dd;
    MRA_TRY(tmp.get(&dd, 5 * (size_t)ng + 1));
    std::vector<double> h(5 * (size_t)ng + 1, 0.0);
    for (int g = 0; g < ng; ++g) {
        h[g] = f->coef_host[g];
        h[ng + g] = f->r2coef_host ? f->r2coef_host[g] : 0.0;
        h[2 * ng + g] = f->expo_host[g];
        h[3 * ng + 2 * g] = f->center_host[2 * g];
        h[3 * ng + 2 * g + 1] = f->center_host[2 * g + 1];
    }
    MRA_CK(cudaMemcpyAsync(dd, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    Dens2 D{ng, dd, dd + ng, dd + 2 * ng, dd + 3 * ng};
    double* tol;
    int32_t* flags;  // [0] depth_hit, [1] refined count
    MRA_TRY(tmp.get(&tol, 2));
    MRA_TRY(tmp.get(&flags, 4));
    MRA_CK(cudaMemsetAsync(flags, 0, 4 * sizeof(int32_t), st));
    k_dens_scale2<<<1, 256, 0, st>>>(D, eps, tol);
    MRA_CK_LAUNCH();
    struct Level {
        int n;
        int32_t *boxes, *refine, *pos, *parent_local;
        double* s;
    };
    std::vector<Level> L;
    int32_t* boxes0;
    MRA_TRY(tmp.get(&boxes0, 2));
    MRA_CK(cudaMemsetAsync(boxes0, 0, 2 * sizeof(int32_t), st));
    int nb = 1;
    int32_t* cur = boxes0;
    int32_t* plocal_prev = nullptr;
    const size_t smem = (2 * (size_t)k + 6 * (size_t)kk) * sizeof(double);
    for (int j = 0; j <= max_level; ++j) {
        Level lv{nb, cur, nullptr, nullptr, plocal_prev, nullptr};
        MRA_TRY(tmp.get(&lv.refine, nb));
        MRA_TRY(tmp.get(&lv.pos, nb));
        MRA_TRY(tmp.get(&lv.s, (size_t)nb * kk));
        int mode;
        if (uniform_level >= 0) mode = (j < uniform_level) ? 1 : 2;
        else mode = (j < init_level) ? 1 : 0;
        if (j == max_level && mode == 1) mode = 2;
        k_build_level2<<<nb, 64, smem, st>>>(k, j, D, cur, tol, mode, j >= max_level, lv.s, lv.refine, flags);
        MRA_CK_LAUNCH();
        MRA_TRY(scan_exclusive(lv.refine, lv.pos, nb, flags + 1, st));
        int32_t nref = 0;
        MRA_CK(cudaMemcpyAsync(&nref, flags + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        MRA_CK(cudaStreamSynchronize(st));
        L.push_back(lv);
        if (nref == 0) break;
        int32_t *next, *plocal;
        MRA_TRY(tmp.get(&next, 2 * 4 * (size_t)nref));
        MRA_TRY(tmp.get(&plocal, nref));
        k_make_children2<<<(nb + 255) / 256, 256, 0, st>>>(nb, cur, lv.refine, lv.pos, next, plocal);
        MRA_CK_LAUNCH();
        cur = next;
        nb = 4 * nref;
        plocal_prev = plocal;
    }
    mra_tree2* t = tree2_new(k, A);
    Tree2Guard tg{t};
    int n = 0;
    for (auto& lv : L) n += lv.n;
    MRA_TRY(tree2_alloc(t, n));
    t->nlev = (int)L.size();
    for (int j = 0; j < MRA_MAX_LEVEL + 2; ++j) t->off[j] = n;
    int base = 0;
    for (int j = 0; j < t->nlev; ++j) {
        t->off[j] = base;
        base += L[j].n;
    }
    base = 0;
    const Tree2Dev T{t->key, t->coord, t->leaf, t->child, t->parent, t->s};
    for (int j = 0; j < t->nlev; ++j) {
        const int nbj = L[j].n, next_base = base + nbj, prev_base = j ? t->off[j - 1] : 0;
        k_place_level2<<<(nbj + 127) / 128, 128, 0, st>>>(nbj, j, base, next_base, L[j].boxes, L[j].refine, L[j].pos,
                                                           L[j].parent_local, prev_base, kk, L[j].s, T);
        MRA_CK_LAUNCH();
        MRA_CK(cudaMemcpyAsync(t->s + (size_t)base * kk, L[j].s, (size_t)nbj * kk * sizeof(double),
                               cudaMemcpyDeviceToDevice, st));
        base = next_base;
    }
    MRA_CK(cudaMemsetAsync(t->dnorm, 0, n * sizeof(double), st));
    int32_t hit = 0;
    MRA_CK(cudaMemcpyAsync(&hit, flags, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    MRA_CK(cudaStreamSynchronize(st));
    t->depth_hit = hit;
    tg.t = nullptr;
    *out = t;
    return hit ? MRA_EDEPTH : MRA_OK;
}

// ------------------------------------------------------------ two-scale transforms in d = 2
// compress: block per node of a level; an internal node gathers the (2k)^2
// square of its 4 children, forms W sq W^T, keeps the k x k corner as its s
// and the norm of the rest (its three wavelet blocks) as dnorm.
__global__ void k_compress2_level(int k, int lo, int hi, const int32_t* child, double* s, double* dnorm,
                                  const double* filt) {
    extern __shared__ double sm[];
    __shared__ double red[32];
    const int i = lo + blockIdx.x;
    if (i >= hi || child[i] < 0) return;
    const int n2 = 2 * k, kk = k * k, c0 = child[i];
    const double* W = filt + 2 * kk;
    double* sq = sm;
    double* t = sq + 4 * kk;
    for (int e = threadIdx.x; e < 4 * kk; e += blockDim.x) {
        const int r = e / n2, c = e % n2;
        const int o = 2 * (r / k) + c / k;
        sq[e] = s[(size_t)(c0 + o) * kk + (r % k) * k + (c % k)];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 4 * kk; e += blockDim.x) {
        const int a = e / n2, c = e % n2;
        double acc = 0.0;
        for (int r = 0; r < n2; ++r) acc += W[a * n2 + r] * sq[r * n2 + c];
        t[e] = acc;
    }
    __syncthreads();
    double nrm = 0.0;
    for (int e = threadIdx.x; e < 4 * kk; e += blockDim.x) {
        const int a = e / n2, b = e % n2;
        double acc = 0.0;
        for (int c = 0; c < n2; ++c) acc += t[a * n2 + c] * W[b * n2 + c];
        if (a < k && b < k) s[(size_t)i * kk + a * k + b] = acc;
        else nrm += acc * acc;
    }
    nrm = blk2_sum(nrm, red);
    if (threadIdx.x == 0) dnorm[i] = sqrt(nrm);
}

static int compress2_impl(mra_tree2* t, cudaStream_t st) {
    const int kk = t->k * t->k;
    for (int j = t->nlev - 2; j >= 0; --j) {
        const int lo = t->off[j], hi = t->off[j + 1];
        if (hi <= lo) continue;
        k_compress2_level<<<hi - lo, 128, 8 * (size_t)kk * sizeof(double), st>>>(t->k, lo, hi, t->child, t->s,
                                                                                t->dnorm, t->filt);
        MRA_CK_LAUNCH();
    }
    t->state = MRA_TREE_REDUNDANT;
    return MRA_OK;
}

// eq. g_assemble: each child of an internal node adds H^(p1)T s H^(p2)
__global__ void k_up2_level(int k, int lo, int hi, const int32_t* child, double* s, const double* filt) {
    extern __shared__ double sm[];
    const int i = lo + blockIdx.x;
    if (i >= hi || child[i] < 0) return;
    const int kk = k * k, c0 = child[i];
    double* x = sm;
    double* t = x + kk;
    for (int e = threadIdx.x; e < kk; e += blockDim.x) x[e] = s[(size_t)i * kk + e];
    __syncthreads();
    for (int o = 0; o < 4; ++o) {
        const double* H1 = filt + (o >> 1) * kk;
        const double* H2 = filt + (o & 1) * kk;
        for (int e = threadIdx.x; e < kk; e += blockDim.x) {
            const int a = e / k, i2 = e % k;
            double acc = 0.0;
            for (int i1 = 0; i1 < k; ++i1) acc += H1[i1 * k + a] * x[i1 * k + i2];
            t[e] = acc;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < kk; e += blockDim.x) {
            const int a = e / k, b = e % k;
            double acc = 0.0;
            for (int i2 = 0; i2 < k; ++i2) acc += t[a * k + i2] * H2[i2 * k + b];
            s[(size_t)(c0 + o) * kk + e] += acc;
        }
        __syncthreads();
    }
}

static int assemble2_impl(mra_tree2* t, cudaStream_t st) {
    const int kk = t->k * t->k;
    for (int j = 0; j + 1 < t->nlev; ++j) {
        const int lo = t->off[j], hi = t->off[j + 1];
        if (hi <= lo) continue;
        k_up2_level<<<hi - lo, 64, 2 * (size_t)kk * sizeof(double), st>>>(t->k, lo, hi, t->child, t->s, t->filt);
        MRA_CK_LAUNCH();
    }
    t->state = MRA_TREE_LEAVES;
    return MRA_OK;
}

// sum of the squares of the leaf blocks: fixed 256 partial sums, then one
// thread adds them in order (the result does not depend on scheduling)
#define NORM_PARTS 256
__global__ void k_leaf_sq_partial2(int n, int kk, const int32_t* leaf, const double* s, double* part) {
    __shared__ double red[32];
    double acc = 0.0;
    for (int i = blockIdx.x; i < n; i += gridDim.x) {
        if (!leaf[i]) continue;
        for (int e = threadIdx.x; e < kk; e += blockDim.x) acc += s[(size_t)i * kk + e] * s[(size_t)i * kk + e];
    }
    acc = blk2_sum(acc, red);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

__global__ void k_sum_parts2(int np, const double* part, double* out) {
    if (threadIdx.x != 0) return;
    double s = 0.0;
    for (int i = 0; i < np; ++i) s += part[i];
    *out = s;
}

static int leaf_norm2(const mra_tree2* t, double* part, double* out, cudaStream_t st) {
    k_leaf_sq_partial2<<<NORM_PARTS, 128, 0, st>>>(t->n, t->k * t->k, t->leaf, t->s, part);
    MRA_CK_LAUNCH();
    k_sum_parts2<<<1, 32, 0, st>>>(NORM_PARTS, part, out);
    MRA_CK_LAUNCH();
    return MRA_OK;
}

// ------------------------------------------------------------ truncation in d = 2
__global__ void k_trunc_thr2(double eps, int n, const double* norm2, double* thr) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *thr = eps * sqrt(*norm2) / sqrt((double)n);
}

// an internal node of the level whose 4 children are leaves and whose wavelet
// norm is below the threshold becomes a leaf; its children are dropped
__global__ void k_merge2_level(int lo, int hi, const int32_t* child, int32_t* leaf, const double* dnorm,
                               const double* thr, int32_t* alive, double* removed2) {
    const int i = lo + blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= hi || leaf[i]) return;
    const int c = child[i];
    if (!(leaf[c] && leaf[c + 1] && leaf[c + 2] && leaf[c + 3])) return;
    if (!(dnorm[i] < *thr)) return;
    leaf[i] = 1;
    for (int o = 0; o < 4; ++o) alive[c + o] = 0;
    atomicAdd(removed2, dnorm[i] * dnorm[i]);
}

__global__ void k_compact2(int n, int kk, const int32_t* alive, const int32_t* newidx, Tree2Dev src,
                           const double* dnorm_src, Tree2Dev dst, double* dnorm_dst) {
    for (int i = blockIdx.x; i < n; i += gridDim.x) {
        if (!alive[i]) continue;
        const int ni = newidx[i];
        if (threadIdx.x == 0) {
            dst.key[ni] = src.key[i];
            for (int d = 0; d < 3; ++d) dst.coord[3 * ni + d] = src.coord[3 * i + d];
            dst.leaf[ni] = src.leaf[i];
            dst.child[ni] = src.leaf[i] ? -1 : newidx[src.child[i]];
            dst.parent[ni] = src.parent[i] < 0 ? -1 : newidx[src.parent[i]];
            dnorm_dst[ni] = src.leaf[i] ? 0.0 : dnorm_src[i];
        }
        for (int e = threadIdx.x; e < kk; e += blockDim.x) dst.s[(size_t)ni * kk + e] = src.s[(size_t)i * kk + e];
    }
}

__global__ void k_new_offsets2(Offs2 off, int nlev, int n, const int32_t* newidx, const int32_t* total, int32_t* out) {
    const int j = threadIdx.x;
    if (j >= MRA_MAX_LEVEL + 2) return;
    out[j] = (j < nlev && off.v[j] < n) ? newidx[off.v[j]] : *total;
}

static int truncate2_impl(mra_tree2* t, double eps, cudaStream_t st, double* removed_host) {
    const int n = t->n, kk = t->k * t->k;
    Scratch tmp(t->A);
    double *part, *sc;  // sc: [0] norm^2, [1] threshold, [2] removed^2
    int32_t *alive, *newidx, *total, *offs;
    MRA_TRY(tmp.get(&part, NORM_PARTS));
    MRA_TRY(tmp.get(&sc, 4));
    MRA_TRY(tmp.get(&alive, n));
    MRA_TRY(tmp.get(&newidx, n));
    MRA_TRY(tmp.get(&total, 1));
    MRA_TRY(tmp.get(&offs, MRA_MAX_LEVEL + 2));
    MRA_TRY(leaf_norm2(t, part, sc, st));
    k_trunc_thr2<<<1, 32, 0, st>>>(eps, n, sc, sc + 1);
    MRA_CK_LAUNCH();
    MRA_CK(cudaMemsetAsync(sc + 2, 0, sizeof(double), st));
    std::vector<int32_t> ones(n, 1);
    MRA_CK(cudaMemcpyAsync(alive, ones.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    for (int j = t->nlev - 2; j >= 0; --j) {
        const int lo = t->off[j], hi = t->off[j + 1];
        if (hi <= lo) continue;
        k_merge2_level<<<(hi - lo + 127) / 128, 128, 0, st>>>(lo, hi, t->child, t->leaf, t->dnorm, sc + 1, alive,
                                                               sc + 2);
        MRA_CK_LAUNCH();
    }
    MRA_TRY(scan_exclusive(alive, newidx, n, total, st));
    Offs2 off;
    memcpy(off.v, t->off, sizeof(off.v));
    k_new_offsets2<<<1, 32, 0, st>>>(off, t->nlev, n, newidx, total, offs);
    MRA_CK_LAUNCH();
    int32_t hoffs[MRA_MAX_LEVEL + 2];
    double removed2 = 0.0;
    MRA_CK(cudaMemcpyAsync(hoffs, offs, sizeof(hoffs), cudaMemcpyDeviceToHost, st));
    MRA_CK(cudaMemcpyAsync(&removed2, sc + 2, sizeof(double), cudaMemcpyDeviceToHost, st));
    MRA_CK(cudaStreamSynchronize(st));  // also keeps `ones` alive until its copy is done
    if (removed_host) *removed_host = sqrt(removed2);
    const int nn = hoffs[MRA_MAX_LEVEL + 1];
    if (nn == n) return MRA_OK;
    // the compacted arrays, swapped into t
    mra_tree2 fresh = {};
    fresh.k = t->k;
    fresh.A = t->A;
    fresh.filt = t->filt;  // kept, not reallocated
    const int rc = tree2_alloc(&fresh, nn);
    if (rc != MRA_OK) {
        tree2_free_arrays(&fresh);
        return rc;
    }
    const Tree2Dev src{t->key, t->coord, t->leaf, t->child, t->parent, t->s};
    const Tree2Dev dst{fresh.key, fresh.coord, fresh.leaf, fresh.child, fresh.parent, fresh.s};
    k_compact2<<<std::max(1, std::min(n, num_sms() * 8)), 64, 0, st>>>(n, kk, alive, newidx, src, t->dnorm, dst,
                                                                        fresh.dnorm);
    cudaError_t e = cudaGetLastError();
    count_launch();
    if (e != cudaSuccess) {
        fresh.filt = nullptr;
        tree2_free_arrays(&fresh);
        set_error("compaction launch: %s", cudaGetErrorString(e));
        return MRA_ECUDA;
    }
    tree2_free_arrays(t);
    t->key = fresh.key; t->coord = fresh.coord; t->leaf = fresh.leaf; t->child = fresh.child;
    t->parent = fresh.parent; t->s = fresh.s; t->dnorm = fresh.dnorm;
    t->n = nn;
    int nlev = 0;
    for (int j = 0; j < MRA_MAX_LEVEL + 1; ++j)
        if (hoffs[j] < hoffs[j + 1]) nlev = j + 1;
    t->nlev = nlev;
    for (int j = 0; j < MRA_MAX_LEVEL + 2; ++j) t->off[j] = (j <= nlev) ? hoffs[j] : nn;
    return MRA_OK;
}

// ------------------------------------------------------------ Algorithm 3 in d = 2
// ||T_0 f_0||: y = sum_m w_m F_m X F_m^T on the root block (j = 0, t = 0); dv[1]
__global__ void k_pilot2(int k, int M, const double* w, const double* F, const double* s_root, double* dv) {
    extern __shared__ double sm[];
    __shared__ double red[32];
    const int kk = k * k, tid = threadIdx.x;
    double* X = sm;
    double* Z = X + kk;
    for (int e = tid; e < kk; e += blockDim.x) X[e] = s_root[e];
    __syncthreads();
    double y0 = 0.0, y1 = 0.0;
    for (int m = 0; m < M; ++m) {
        const double* Fm = F + ((size_t)m * 7 + 3) * kk;
        for (int e = tid; e < kk; e += blockDim.x) {
            const int a = e / k, c = e % k;
            double acc = 0.0;
            for (int i = 0; i < k; ++i) acc += Fm[a * k + i] * X[i * k + c];
            Z[e] = acc;
        }
        __syncthreads();
        if (tid < kk) {
            double acc = 0.0;
            for (int c = 0; c < k; ++c) acc += Z[(tid / k) * k + c] * Fm[(tid % k) * k + c];
            y0 += w[m] * acc;
        }
        if (tid + (int)blockDim.x < kk) {
            const int e = tid + blockDim.x;
            double acc = 0.0;
            for (int c = 0; c < k; ++c) acc += Z[(e / k) * k + c] * Fm[(e % k) * k + c];
            y1 += w[m] * acc;
        }
        __syncthreads();
    }
    const double nrm = blk2_sum(y0 * y0 + y1 * y1, red);
    if (tid == 0) dv[1] = sqrt(nrm);
}

// eta = eps sigma / ||f||; J_m; per scale j and subset S = 0, 1, 2 the range
// [m1, m2] trimmed from both ends while the cumulative w_m c^S b^(2-S) stays
// <= eta / 72 (c, b: the largest N_F over |l| <= 1 and over 2 <= |l| <= 3).
// Layout: Jm[M] | m1[nlev*3] | m2[nlev*3].
__global__ void k_schedule2(int M, int nlev, double eps, const double* w, const double* nF, const double* est,
                            double* dv, int32_t* sched) {
    int32_t* Jm = sched;
    int32_t* m1 = Jm + M;
    int32_t* m2 = m1 + nlev * 3;
    const double fn = sqrt(dv[0]);
    const double eta = fn > 0.0 ? eps * dv[1] / fn : 0.0;
    if (threadIdx.x == 0) dv[2] = eta;
    for (int m = threadIdx.x; m < M; m += blockDim.x) {
        int jm = 0;
        for (int j = 1; j < nlev; ++j)
            if (w[m] * est[(size_t)j * M + m] > eta / M) jm = j;
        Jm[m] = jm;
    }
    __syncthreads();
    const double budget = eta / (2.0 * 36.0);
    for (int js = threadIdx.x; js < nlev * 3; js += blockDim.x) {
        const int j = js / 3, S = js % 3;
        int lo_m = 0, hi_m = -1, first = -1, last = -1;
        for (int m = 0; m < M; ++m)
            if (Jm[m] >= j) {
                if (first < 0) first = m;
                last = m;
            }
        if (first >= 0) {
            auto e_of = [&](int m) {
                const double* r = nF + ((size_t)j * M + m) * 7;
                const double c = fmax(fmax(r[2], r[3]), r[4]);
                const double bb = fmax(fmax(r[0], r[1]), fmax(r[5], r[6]));
                double v = w[m];
                for (int q = 0; q < S; ++q) v *= c;
                for (int q = S; q < 2; ++q) v *= bb;
                return v;
            };
            double acc = 0.0;
            int lo = first;
            for (; lo <= last; ++lo) {
                if (Jm[lo] < j) continue;
                const double e = e_of(lo);
                if (acc + e <= budget) acc += e;
                else break;
            }
            acc = 0.0;
            int hi = last;
            for (; hi >= lo; --hi) {
                if (Jm[hi] < j) continue;
                const double e = e_of(hi);
                if (acc + e <= budget) acc += e;
                else break;
            }
            if (hi >= lo && lo <= last) {
                lo_m = lo;
                hi_m = hi;
            }
        }
        m1[js] = lo_m;
        m2[js] = hi_m;
    }
}

// One block per output node.  For every band translation whose input box lies
// in the square and that keeps a term: the input block (the node at level j,
// or the ancestor leaf refined down with H^(p1)T X H^(p2) per level: Step 2),
// then ghat += w_m F^{t1}_m X (F^{t2}_m)^T over the kept terms.
// counters: [0] items, [1] pairs, [2] Step-2 refinements, [3] lookups that
// found no ancestor (0 for a valid tree).
__global__ void __launch_bounds__(128) k_apply2(int k, int M, int nlev, Offs2 off, const uint64_t* key,
                                                const int32_t* coord, const int32_t* leaf, const double* s,
                                                const double* F, const double* w, const int32_t* sched,
                                                const double* filt, double* gout, unsigned long long* counters) {
    extern __shared__ double sm[];
    const int kk = k * k, tid = threadIdx.x;
    double* X = sm;
    double* Z = X + kk;
    double* T = Z + kk;
    double* Hs = T + kk;
    int* Js = (int*)(Hs + 2 * kk);
    __shared__ int s_src, s_lev;
    const int node = blockIdx.x;
    for (int e = tid; e < 2 * kk; e += blockDim.x) Hs[e] = filt[e];
    for (int m = tid; m < M; m += blockDim.x) Js[m] = sched[m];
    const int32_t* m1 = sched + M;
    const int32_t* m2 = m1 + nlev * 3;
    const int j = coord[3 * node], a1 = coord[3 * node + 1], a2 = coord[3 * node + 2];
    const bool isleaf = leaf[node] != 0;
    const int N = 1 << j;
    double y0 = 0.0, y1 = 0.0;
    unsigned long long items = 0, pairs = 0, ghosts = 0, lost = 0;
    __syncthreads();
    for (int q1 = 0; q1 < 6; ++q1) {
        const int t1 = band_t(a1, q1), b1 = a1 - t1;
        if (b1 < 0 || b1 >= N) continue;
        for (int q2 = 0; q2 < 6; ++q2) {
            const int t2 = band_t(a2, q2), b2 = a2 - t2;
            if (b2 < 0 || b2 >= N) continue;
            const int S = (abs(t1) <= 1) + (abs(t2) <= 1);
            const int lo = m1[j * 3 + S], hi = m2[j * 3 + S];
            if (lo > hi) continue;
            const bool core = S == 2;
            int cnt = 0;
            for (int m = lo; m <= hi; ++m) {
                if (Js[m] < j || (core && !isleaf && Js[m] > j)) continue;
                ++cnt;
            }
            if (cnt == 0) continue;
            if (tid == 0) {
                int jj = j, idx = -1;
                for (; jj >= 0; --jj) {
                    idx = find_key_exact(key, off.v[jj], off.v[jj + 1], morton2(b1 >> (j - jj), b2 >> (j - jj)));
                    if (idx >= 0) break;
                }
                s_src = idx;
                s_lev = jj;
            }
            __syncthreads();
            const int src = s_src, jj = s_lev;
            if (src < 0) {  // impossible for a complete tree; counted, skipped
                ++lost;
                __syncthreads();
                continue;
            }
            for (int e = tid; e < kk; e += blockDim.x) X[e] = s[(size_t)src * kk + e];
            __syncthreads();
            for (int lev = jj; lev < j; ++lev) {
                const int sh = j - lev - 1, p1 = (b1 >> sh) & 1, p2 = (b2 >> sh) & 1;
                for (int e = tid; e < kk; e += blockDim.x) {
                    const int a = e / k, c = e % k;
                    double acc = 0.0;
                    for (int i = 0; i < k; ++i) acc += Hs[p1 * kk + i * k + a] * X[i * k + c];
                    T[e] = acc;
                }
                __syncthreads();
                for (int e = tid; e < kk; e += blockDim.x) {
                    const int a = e / k, b = e % k;
                    double acc = 0.0;
                    for (int c = 0; c < k; ++c) acc += T[a * k + c] * Hs[p2 * kk + c * k + b];
                    X[e] = acc;
                }
                __syncthreads();
            }
            if (jj < j) ++ghosts;
            ++pairs;
            items += cnt;
            for (int m = lo; m <= hi; ++m) {
                if (Js[m] < j || (core && !isleaf && Js[m] > j)) continue;
                const double* F1 = F + (((size_t)j * M + m) * 7 + t1 + 3) * kk;
                const double* F2 = F + (((size_t)j * M + m) * 7 + t2 + 3) * kk;
                for (int e = tid; e < kk; e += blockDim.x) {
                    const int a = e / k, c = e % k;
                    double acc = 0.0;
                    for (int i = 0; i < k; ++i) acc += F1[a * k + i] * X[i * k + c];
                    Z[e] = acc;
                }
                __syncthreads();
                const double wm = w[m];
                if (tid < kk) {
                    double acc = 0.0;
                    for (int c = 0; c < k; ++c) acc += Z[(tid / k) * k + c] * F2[(tid % k) * k + c];
                    y0 += wm * acc;
                }
                if (tid + (int)blockDim.x < kk) {
                    const int e = tid + blockDim.x;
                    double acc = 0.0;
                    for (int c = 0; c < k; ++c) acc += Z[(e / k) * k + c] * F2[(e % k) * k + c];
                    y1 += wm * acc;
                }
                __syncthreads();
            }
        }
    }
    if (tid < kk) gout[(size_t)node * kk + tid] = y0;
    if (tid + (int)blockDim.x < kk) gout[(size_t)node * kk + tid + blockDim.x] = y1;
    if (tid == 0) {
        atomicAdd(&counters[0], items);
        atomicAdd(&counters[1], pairs);
        atomicAdd(&counters[2], ghosts);
        if (lost) atomicAdd(&counters[3], lost);
    }
}

static int apply2_impl(const mra_op* op, const mra_tree2* f, cudaStream_t st, mra_tree2** gout,
                       mra_apply_stats* stats) {
    *gout = nullptr;
    const int k = op->k, kk = k * k, M = op->M, n = f->n, nlev = f->nlev;
    if (f->k != k) { set_error("tree order k=%d differs from operator k=%d", f->k, k); return MRA_EINVAL; }
    if (nlev - 1 > op->J) { set_error("tree depth %d exceeds operator max_level %d", nlev - 1, op->J); return MRA_EINVAL; }
    if (f->state != MRA_TREE_REDUNDANT) { set_error("apply_ns2 needs a compressed (redundant) tree"); return MRA_ESTATE; }
    Scratch tmp(f->A);
    double *part, *dv;
    int32_t* sched;
    unsigned long long* counters;
    MRA_TRY(tmp.get(&part, NORM_PARTS));
    MRA_TRY(tmp.get(&dv, 4));
    MRA_TRY(tmp.get(&sched, (size_t)M + 6 * nlev));
    MRA_TRY(tmp.get(&counters, 4));
    MRA_CK(cudaMemsetAsync(counters, 0, 4 * sizeof(unsigned long long), st));
    MRA_TRY(leaf_norm2(f, part, dv, st));
    k_pilot2<<<1, 128, 2 * (size_t)kk * sizeof(double), st>>>(k, M, op->w, op->F, f->s, dv);
    MRA_CK_LAUNCH();
    k_schedule2<<<1, 256, 0, st>>>(M, nlev, op->eps, op->w, op->nF, op->est, dv, sched);
    MRA_CK_LAUNCH();
    mra_tree2* g = nullptr;
    MRA_TRY(tree2_clone_skeleton(f, &g));
    Tree2Guard tg{g};
    g->state = MRA_TREE_NSFORM;
    Offs2 off;
    memcpy(off.v, f->off, sizeof(off.v));
    const size_t smem = 5 * (size_t)kk * sizeof(double) + (size_t)M * sizeof(int);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    MRA_CK(cudaEventCreate(&e0));
    struct Ev {
        cudaEvent_t& a;
        cudaEvent_t& b;
        ~Ev() {
            if (a) cudaEventDestroy(a);
            if (b) cudaEventDestroy(b);
        }
    } ev{e0, e1};
    MRA_CK(cudaEventCreate(&e1));
    MRA_CK(cudaEventRecord(e0, st));
    k_apply2<<<n, 128, smem, st>>>(k, M, nlev, off, f->key, f->coord, f->leaf, f->s, op->F, op->w, sched, f->filt,
                                   g->s, counters);
    MRA_CK_LAUNCH();
    MRA_CK(cudaEventRecord(e1, st));
    MRA_CK(cudaMemsetAsync(g->dnorm, 0, n * sizeof(double), st));
    unsigned long long hc[4];
    double hdv[4];
    MRA_CK(cudaMemcpyAsync(hc, counters, sizeof(hc), cudaMemcpyDeviceToHost, st));
    MRA_CK(cudaMemcpyAsync(hdv, dv, sizeof(hdv), cudaMemcpyDeviceToHost, st));
    MRA_CK(cudaStreamSynchronize(st));
    if (hc[3]) { set_error("%llu input boxes without an ancestor (tree not complete)", hc[3]); return MRA_ECUDA; }
    if (stats) {
        memset(stats, 0, sizeof(*stats));
        stats->n_items = (int64_t)hc[0];
        stats->n_pairs = (int64_t)hc[1];
        stats->n_ghosts = (int64_t)hc[2];
        stats->n_out_nodes = n;
        stats->fnorm = sqrt(hdv[0]);
        stats->sigma = hdv[1];
        stats->eta = hdv[2];
        float ms = 0.0f;
        MRA_CK(cudaEventElapsedTime(&ms, e0, e1));
        stats->ms_apply = ms;
    }
    tg.t = nullptr;
    *gout = g;
    return MRA_OK;
}

}  // namespace mra

using namespace mra;

static bool tree2_ok(const mra_tree2* t) { return t && t->magic == MRA_TREE2_MAGIC; }
static bool op2_ok(const mra_op* o) { return o && o->magic == MRA_OP_MAGIC && o->d == 2; }

int mra_build_tree2(const mra_density* f, int k, double eps, int max_level, int uniform_level, int init_level,
                    const mra_alloc* alloc, void* stream, mra_tree2** out) {
    if (!out) { set_error("out is NULL"); return MRA_EINVAL; }
    *out = nullptr;
    if (!f || f->n <= 0 || !f->coef_host || !f->expo_host || !f->center_host) {
        set_error("empty or invalid density");
        return MRA_EINVAL;
    }
    if (k < 1 || k > MRA_MAX_K) { set_error("k=%d outside [1, %d]", k, MRA_MAX_K); return MRA_EINVAL; }
    if (!(eps > 0.0)) { set_error("eps must be > 0"); return MRA_EINVAL; }
    if (max_level < 0 || max_level > MRA_MAX_LEVEL) { set_error("max_level outside [0, %d]", MRA_MAX_LEVEL); return MRA_EINVAL; }
    for (int g = 0; g < f->n; ++g)
        if (!(f->expo_host[g] > 0.0)) { set_error("exponent %d is not positive", g); return MRA_EINVAL; }
    return build_tree2_impl(f, k, eps, max_level, uniform_level, init_level, make_alloc(alloc, stream), out);
}

int mra_tree2_import(int k, int n, const int32_t* coords_host, const int32_t* leaf_host, const double* blocks_host,
                     const mra_alloc* alloc, void* stream, mra_tree2** out) {
    if (!out) { set_error("out is NULL"); return MRA_EINVAL; }
    *out = nullptr;
    if (k < 1 || k > MRA_MAX_K || n < 1 || !coords_host || !leaf_host || !blocks_host) {
        set_error("invalid import arguments");
        return MRA_EINVAL;
    }
    mra_tree2* t = tree2_new(k, make_alloc(alloc, stream));
    Tree2Guard g{t};
    MRA_TRY(tree2_alloc(t, n));
    MRA_TRY(tree2_link_upload(t, coords_host, leaf_host));
    cudaStream_t st = t->A.stream;
    MRA_CK(cudaMemcpyAsync(t->s, blocks_host, (size_t)n * k * k * sizeof(double), cudaMemcpyHostToDevice, st));
    MRA_CK(cudaMemsetAsync(t->dnorm, 0, n * sizeof(double), st));
    MRA_CK(cudaStreamSynchronize(st));
    g.t = nullptr;
    *out = t;
    return MRA_OK;
}

int mra_tree2_export(const mra_tree2* t, int32_t* coords_host, int32_t* leaf_host, double* blocks_host,
                     double* dnorm_host, void* stream) {
    if (!tree2_ok(t)) { set_error("invalid d = 2 tree handle"); return MRA_EINVAL; }
    cudaStream_t st = (cudaStream_t)stream;
    const int n = t->n;
    if (coords_host) MRA_CK(cudaMemcpyAsync(coords_host, t->coord, 3 * (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    if (leaf_host) MRA_CK(cudaMemcpyAsync(leaf_host, t->leaf, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    if (blocks_host) MRA_CK(cudaMemcpyAsync(blocks_host, t->s, (size_t)n * t->k * t->k * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (dnorm_host) MRA_CK(cudaMemcpyAsync(dnorm_host, t->dnorm, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, st));
    MRA_CK(cudaStreamSynchronize(st));
    return MRA_OK;
}

int mra_tree2_get_info(const mra_tree2* t, mra_tree_info* info) {
    if (!tree2_ok(t) || !info) { set_error("invalid d = 2 tree handle"); return MRA_EINVAL; }
    info->k = t->k;
    info->n_nodes = t->n;
    info->n_levels = t->nlev;
    info->state = t->state;
    info->depth_hit = t->depth_hit;
    memcpy(info->level_offset, t->off, sizeof(t->off));
    return MRA_OK;
}

int mra_compress2(mra_tree2* t, void* stream) {
    if (!tree2_ok(t)) { set_error("invalid d = 2 tree handle"); return MRA_EINVAL; }
    if (t->state == MRA_TREE_NSFORM) { set_error("compress needs leaf data; assemble an ns-form tree first"); return MRA_ESTATE; }
    return compress2_impl(t, (cudaStream_t)stream);
}

int mra_apply_ns2(const mra_op* op, const mra_tree2* f, void* stream, mra_tree2** g_ns, mra_apply_stats* stats) {
    if (!g_ns) { set_error("g_ns is NULL"); return MRA_EINVAL; }
    *g_ns = nullptr;
    if (!op2_ok(op)) { set_error("invalid operator handle or not a d = 2 operator"); return MRA_EINVAL; }
    if (!tree2_ok(f)) { set_error("invalid d = 2 tree handle"); return MRA_EINVAL; }
    return apply2_impl(op, f, (cudaStream_t)stream, g_ns, stats);
}

int mra_reconstruct2(mra_tree2* t, int truncate, double eps, void* stream, double* truncation_l2_host) {
    if (!tree2_ok(t)) { set_error("invalid d = 2 tree handle"); return MRA_EINVAL; }
    if (truncation_l2_host) *truncation_l2_host = 0.0;
    if (t->state != MRA_TREE_NSFORM) { set_error("reconstruct2 needs an ns-form tree"); return MRA_ESTATE; }
    if (truncate && !(eps > 0.0)) { set_error("truncation eps must be > 0"); return MRA_EINVAL; }
    cudaStream_t st = (cudaStream_t)stream;
    MRA_TRY(assemble2_impl(t, st));
    MRA_TRY(compress2_impl(t, st));
    if (truncate) MRA_TRY(truncate2_impl(t, eps, st, truncation_l2_host));
    return MRA_OK;
}

int mra_free_tree2(mra_tree2* t) {
    if (!t) return MRA_OK;
    if (!tree2_ok(t)) { set_error("invalid d = 2 tree handle"); return MRA_EINVAL; }
    tree2_delete(t);
    return MRA_OK;
}
