// Trees on the device: Algorithm 1 (adaptive decomposition), the redundant
// tree (two-scale decomposition, eqs. decomp_scaling / decomp_wavelet), its
// inverse (eqs. recon_even / recon_odd), the adaptive projection of
// eq. g_assemble, and the final truncation (Algorithm 3, Step 4).
//
// Layout in HBM: nodes sorted by level, then by Morton key within a level, so
// the 8 children of a node are contiguous in octant order (p1 p2 p3) and each
// level is a sorted key range for binary search.  Blocks are k^3 FP64 arrays
// s[i1][i2][i3] (i3 fastest), one per node, contiguous in node order.
#include <math.h>

#include <algorithm>
#include <vector>

#include "mra_internal.cuh"

namespace mra {

// ------------------------------------------------------------ small utilities
// Single-block exclusive scan of n int32 values (n up to a few million); the
// total is written to *total.
__global__ void k_scan_exclusive(const int32_t* in, int32_t* out, int n, int32_t* total) {
    __shared__ int32_t part[1024];
    const int tid = threadIdx.x, nt = blockDim.x;
    const int per = (n + nt - 1) / nt;
    const int lo = min(n, tid * per), hi = min(n, lo + per);
    int32_t s = 0;
    for (int i = lo; i < hi; ++i) s += in[i];
    part[tid] = s;
    __syncthreads();
    for (int d = 1; d < nt; d <<= 1) {
        int32_t v = (tid >= d) ? part[tid - d] : 0;
        __syncthreads();
        part[tid] += v;
        __syncthreads();
    }
    int32_t run = part[tid] - s;
    for (int i = lo; i < hi; ++i) {
        int32_t v = in[i];
        out[i] = run;
        run += v;
    }
    if (tid == nt - 1 && total) *total = part[nt - 1];
}

int scan_exclusive(const int32_t* in, int32_t* out, int n, int32_t* total, cudaStream_t st) {
    if (n <= 0) {
        MRA_CK(cudaMemsetAsync(total, 0, sizeof(int32_t), st));
        return MRA_OK;
    }
    k_scan_exclusive<<<1, 1024, 0, st>>>(in, out, n, total);
    MRA_CK_LAUNCH();
    return MRA_OK;
}

// out[along dim] = Mat * in[along dim] for a k^3 array in shared memory;
// Mat is k x k row-major (out index, in index).  All threads of the block.
__device__ void mode_product(const double* in, double* out, const double* Mat, int dim, int k) {
    const int n = k * k * k;
    for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
        int i3 = idx % k, i2 = (idx / k) % k, i1 = idx / (k * k);
        int r = dim == 0 ? i1 : (dim == 1 ? i2 : i3);
        int stride = dim == 0 ? k * k : (dim == 1 ? k : 1);
        const double* src = in + idx - r * stride;
        double acc = 0.0;
        for (int c = 0; c < k; ++c) acc += Mat[r * k + c] * src[c * stride];
        out[idx] = acc;
    }
    __syncthreads();
}

// In-place 2k-point transform along one direction of a (2k)^3 cube:
// line <- M line (transpose = 0) or M^T line (transpose = 1), M = 2k x 2k.
__device__ void cube_transform(double* cube, int n2, const double* Mt, int transpose, int dim) {
    const int lines = n2 * n2;
    const int stride = dim == 0 ? n2 * n2 : (dim == 1 ? n2 : 1);
    for (int ln = threadIdx.x; ln < lines; ln += blockDim.x) {
        int u = ln / n2, v = ln % n2;
        int base = dim == 0 ? (u * n2 + v) : (dim == 1 ? (u * n2 * n2 + v) : (u * n2 * n2 + v * n2));
        double x[2 * MRA_MAX_K];
        for (int c = 0; c < n2; ++c) x[c] = cube[base + c * stride];
        for (int r = 0; r < n2; ++r) {
            double acc = 0.0;
            for (int c = 0; c < n2; ++c) acc += (transpose ? Mt[c * n2 + r] : Mt[r * n2 + c]) * x[c];
            cube[base + r * stride] = acc;
        }
    }
    __syncthreads();
}

__device__ double block_sum(double v, double* red) {
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

__device__ double block_max(double v, double* red) {
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

// ------------------------------------------------------------ arrays
// A tree's node arrays, wavelet norms and blocks share one allocation (one call
// into the allocator), each array on a 256-byte boundary; the node arrays come
// first, in the order below, so that a skeleton is one contiguous copy.
struct SlabLayout {
    size_t key, coord, leaf, child, parent, off, nodes_end, dnorm, s, total;
    SlabLayout(size_t n, size_t k3, bool with_s) {
        size_t at = 0;
        auto take = [&](size_t bytes) {
            const size_t o = at;
            at += (bytes + 255) / 256 * 256;
            return o;
        };
        key = take(n * sizeof(uint64_t));
        coord = take(4 * n * sizeof(int32_t));
        leaf = take(n * sizeof(int32_t));
        child = take(n * sizeof(int32_t));
        parent = take(n * sizeof(int32_t));
        off = take((MRA_MAX_LEVEL + 2) * sizeof(int32_t));
        nodes_end = at;
        dnorm = take(n * sizeof(double));
        s = take(with_s ? n * k3 * sizeof(double) : 0);
        total = at;
    }
};

int tree_alloc_arrays(mra_tree* t, int n, bool with_s) {
    const Alloc& A = t->A;
    const SlabLayout L((size_t)n, (size_t)t->k * t->k * t->k, with_s);
    unsigned char* base;
    MRA_TRY(dalloc(A, &base, L.total));
    t->slab = base;
    t->a.key = (uint64_t*)(base + L.key);
    t->a.coord = (int32_t*)(base + L.coord);
    t->a.leaf = (int32_t*)(base + L.leaf);
    t->a.child = (int32_t*)(base + L.child);
    t->a.parent = (int32_t*)(base + L.parent);
    t->a.off = (int32_t*)(base + L.off);
    t->dnorm = (double*)(base + L.dnorm);
    t->s = with_s ? (double*)(base + L.s) : nullptr;
    if (!t->filt) {
        MRA_TRY(dalloc(A, &t->filt, 6 * t->k * t->k));
        MRA_TRY(launch_filters(t->k, t->filt, A.stream));
    }
    t->n = n;
    return MRA_OK;
}

void tree_free_arrays(mra_tree* t) {
    const Alloc& A = t->A;
    A.put(t->slab);
    A.put(t->dcube);
    t->a = TreeArrays();
    t->dnorm = nullptr; t->s = nullptr; t->dcube = nullptr; t->slab = nullptr;
}

// Host-side validation and linking of an imported node list; uploads key,
// coord, leaf, child, parent and offsets.
int tree_link_and_upload(mra_tree* t, const int32_t* coords, const int32_t* leaf) {
    const int n = t->n;
    std::vector<uint64_t> key(n);
    std::vector<int32_t> child(n, -1), parent(n, -1), lf(n);
    int off[MRA_MAX_LEVEL + 2];
    for (int j = 0; j < MRA_MAX_LEVEL + 2; ++j) off[j] = n;
    int nlev = 0;
    for (int i = 0; i < n; ++i) {
        int j = coords[4 * i];
        if (j < 0 || j > MRA_MAX_LEVEL) { set_error("node %d: level %d out of range", i, j); return MRA_EINVAL; }
        for (int d = 1; d < 4; ++d)
            if (coords[4 * i + d] < 0 || coords[4 * i + d] >= (1 << j)) {
                set_error("node %d: box index out of range", i);
                return MRA_EINVAL;
            }
        key[i] = morton3(coords[4 * i + 1], coords[4 * i + 2], coords[4 * i + 3]);
        if (i > 0) {
            int jp = coords[4 * (i - 1)];
            if (jp > j || (jp == j && key[i - 1] >= key[i])) { set_error("nodes not sorted by (level, Morton key) at %d", i); return MRA_EINVAL; }
        }
        if (off[j] == n) off[j] = i;
        nlev = std::max(nlev, j + 1);
        lf[i] = leaf[i] ? 1 : 0;
    }
    if (n == 0 || coords[0] != 0) { set_error("tree must start with the root (0,0,0,0)"); return MRA_EINVAL; }
    for (int j = nlev; j >= 0; --j) if (off[j] == n && j < nlev) off[j] = off[j + 1];
    for (int j = nlev; j < MRA_MAX_LEVEL + 2; ++j) off[j] = n;
    // link children: every internal node must have its 8 children at level j+1
    for (int i = 0; i < n; ++i) {
        int j = coords[4 * i];
        if (lf[i]) continue;
        if (j >= MRA_MAX_LEVEL) { set_error("internal node %d lacks children (deepest level)", i); return MRA_EINVAL; }
        uint64_t ck = key[i] << 3;
        int lo = off[j + 1], hi = off[j + 2];
        int pos = (int)(std::lower_bound(key.begin() + lo, key.begin() + hi, ck) - key.begin());
        if (pos + 8 > hi) { set_error("internal node %d lacks children", i); return MRA_EINVAL; }
        for (int o = 0; o < 8; ++o)
            if (key[pos + o] != ck + o) { set_error("internal node %d lacks child %d", i, o); return MRA_EINVAL; }
        child[i] = pos;
        for (int o = 0; o < 8; ++o) parent[pos + o] = i;
    }
    for (int i = 1; i < n; ++i)
        if (parent[i] < 0) { set_error("node %d has no parent", i); return MRA_EINVAL; }
    t->nlev = nlev;
    memcpy(t->off, off, sizeof(off));
    // the node arrays in the slab's layout on the host, then one copy
    const SlabLayout L((size_t)n, (size_t)t->k * t->k * t->k, true);
    std::vector<unsigned char> stage(L.nodes_end);
    memcpy(stage.data() + L.key, key.data(), n * sizeof(uint64_t));
    memcpy(stage.data() + L.coord, coords, 4 * (size_t)n * sizeof(int32_t));
    memcpy(stage.data() + L.leaf, lf.data(), n * sizeof(int32_t));
    memcpy(stage.data() + L.child, child.data(), n * sizeof(int32_t));
    memcpy(stage.data() + L.parent, parent.data(), n * sizeof(int32_t));
    memcpy(stage.data() + L.off, off, sizeof(off));
    cudaStream_t st = t->A.stream;
    MRA_CK(cudaMemcpyAsync(t->slab, stage.data(), L.nodes_end, cudaMemcpyHostToDevice, st));
    MRA_CK(cudaStreamSynchronize(st));  // the staging vector goes out of scope
    return MRA_OK;
}

int tree_clone_skeleton(const mra_tree* src, mra_tree** out) {
    mra_tree* t = new mra_tree();
    t->magic = MRA_TREE_MAGIC;
    t->k = src->k;
    t->A = src->A;
    t->nlev = src->nlev;
    t->state = src->state;
    t->depth_hit = src->depth_hit;
    memcpy(t->off, src->off, sizeof(t->off));
    // the filters depend on k only: copy them instead of recomputing
    int rc = dalloc(t->A, &t->filt, 6 * t->k * t->k);
    if (rc == MRA_OK &&
        cudaMemcpyAsync(t->filt, src->filt, 6 * t->k * t->k * sizeof(double), cudaMemcpyDeviceToDevice,
                        t->A.stream) != cudaSuccess) {
        set_error("filter copy failed");
        rc = MRA_ECUDA;
    }
    if (rc == MRA_OK) rc = tree_alloc_arrays(t, src->n, true);
    if (rc != MRA_OK) { tree_free_arrays(t); t->A.put(t->filt); delete t; return rc; }
    // both slabs are laid out for the same node count: the skeleton is one copy
    const SlabLayout L((size_t)src->n, (size_t)src->k * src->k * src->k, true);
    MRA_CK(cudaMemcpyAsync(t->slab, src->slab, L.nodes_end, cudaMemcpyDeviceToDevice, t->A.stream));
    *out = t;
    return MRA_OK;
}

// ------------------------------------------------------------ Algorithm 1
struct DensDev {
    int n;
    const double *coef, *r2, *expo, *cen;
};

__device__ double dens_eval(const DensDev& D, double x, double y, double z) {
    double f = 0.0;
    for (int g = 0; g < D.n; ++g) {
        double dx = x - D.cen[3 * g], dy = y - D.cen[3 * g + 1], dz = z - D.cen[3 * g + 2];
        double r2 = dx * dx + dy * dy + dz * dz;
        f += (D.coef[g] + D.r2[g] * r2) * exp(-D.expo[g] * r2);
    }
    return f;
}

__global__ void k_dens_scale(DensDev D, double eps, double* tol) {
    __shared__ double red[32];
    double m = 0.0;
    for (int g = threadIdx.x; g < D.n; g += blockDim.x)
        m = fmax(m, fabs(dens_eval(D, D.cen[3 * g], D.cen[3 * g + 1], D.cen[3 * g + 2])));
    m = block_max(m, red);
    if (threadIdx.x == 0) {
        tol[0] = eps * m;
        tol[1] = 1e-18 * m;  // terms below this on a box are skipped (rounding level)
    }
}

// Values of the density on the tensor grid X[0][q1] x X[1][q2] x X[2][q3]
// (k increasing points per direction) added into v[(q1 k + q2) k + q3],
// block-cooperatively.  Each term factors by direction,
// exp(-a|x - c|^2) = prod_d exp(-a (x_d - c_d)^2) and |x - c|^2 = sum_d (x_d - c_d)^2,
// so per term the block forms 3k one-dimensional factors (in shared memory,
// DG_CHUNK terms at a time) and each grid point costs a few products instead
// of an exponential.  A term whose bound on the grid's box,
// (|c| + |b| dmax^2) exp(-a dmin^2), is below `cut` is skipped.
#define DG_CHUNK 32
__device__ void dens_grid(const DensDev& D, int k, const double* X, double* v, double* E, double* R,
                          double* cb, int* act, double cut) {
    const int k3 = k * k * k, kk = k * k, k3d = 3 * k;
    __shared__ int nact;
    for (int g0 = 0; g0 < D.n; g0 += DG_CHUNK) {
        const int ng = min(DG_CHUNK, D.n - g0);
        if (threadIdx.x < 32) {  // warp 0: which terms of the chunk reach the box
            const int g = g0 + threadIdx.x;
            bool on = false;
            if ((int)threadIdx.x < ng) {
                double dmin2 = 0.0, dmax2 = 0.0;
                for (int d = 0; d < 3; ++d) {
                    const double lo = X[d * k] - D.cen[3 * g + d], hi = X[d * k + k - 1] - D.cen[3 * g + d];
                    const double dn = lo > 0.0 ? lo : (hi < 0.0 ? -hi : 0.0);
                    const double dx = fmax(fabs(lo), fabs(hi));
                    dmin2 += dn * dn;
                    dmax2 += dx * dx;
                }
                on = (fabs(D.coef[g]) + fabs(D.r2[g]) * dmax2) * exp(-D.expo[g] * dmin2) >= cut;
            }
            const unsigned mask = __ballot_sync(0xffffffffu, on);
            if (on) {
                const int slot = __popc(mask & ((1u << threadIdx.x) - 1u));
                act[slot] = g;
                cb[2 * slot] = D.coef[g];
                cb[2 * slot + 1] = D.r2[g];
            }
            if (threadIdx.x == 0) nact = __popc(mask);
        }
        __syncthreads();
        const int na = nact;
        for (int e = threadIdx.x; e < na * k3d; e += blockDim.x) {
            const int a = e / k3d, d = (e / k) % 3, q = e % k, g = act[a];
            const double dx = X[d * k + q] - D.cen[3 * g + d];
            R[e] = dx * dx;
            E[e] = exp(-D.expo[g] * dx * dx);
        }
        __syncthreads();
        for (int idx = threadIdx.x; idx < k3; idx += blockDim.x) {
            const int q1 = idx / kk, q2 = (idx / k) % k, q3 = idx % k;
            double acc = v[idx];
            for (int g = 0; g < na; ++g) {
                const double* Eg = E + g * k3d;
                const double* Rg = R + g * k3d;
                const double prod = Eg[q1] * Eg[k + q2] * Eg[2 * k + q3];
                acc += (cb[2 * g] + cb[2 * g + 1] * (Rg[q1] + Rg[k + q2] + Rg[2 * k + q3])) * prod;
            }
            v[idx] = acc;
        }
        __syncthreads();
    }
}

// One block per box of level j.  mode: 0 adaptive test, 1 refine, 2 leaf.
__global__ void k_build_level(int k, int j, DensDev D, const int32_t* boxes, const double* tolp, int mode,
                              int at_max, double* s_out, int32_t* refine, int32_t* depth_hit) {
    extern __shared__ double sm[];
    const int k3 = k * k * k, kk = k * k;
    double* g = sm;             // k nodes
    double* gw = g + k;         // k weights
    double* P = gw + k;         // [i][q] phi_i(g_q) w_q
    double* Q = P + kk;         // [p][q][i] phi_i((g_q + p)/2): (q, i) as a k x k matrix per p
    double* v = Q + 2 * kk;     // k^3 values
    double* t1 = v + k3;
    double* t2 = t1 + k3;
    double* s = t2 + k3;
    double* X = s + k3;          // 3k grid coordinates
    double* E = X + 3 * k;       // DG_CHUNK * 3k factors
    double* R = E + DG_CHUNK * 3 * k;
    double* cb = R + DG_CHUNK * 3 * k;  // (coef, r2coef) per term of a chunk
    __shared__ double red[32];
    __shared__ int act[DG_CHUNK];
    const double cut = tolp[1];
    const int b = blockIdx.x, tid = threadIdx.x;
    const int a1 = boxes[3 * b], a2 = boxes[3 * b + 1], a3 = boxes[3 * b + 2];
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
    for (int e = tid; e < 3 * k; e += blockDim.x) {
        const int d = e / k, q = e % k;
        X[e] = (g[q] + (d == 0 ? a1 : (d == 1 ? a2 : a3))) * h;
    }
    for (int idx = tid; idx < k3; idx += blockDim.x) v[idx] = 0.0;
    __syncthreads();
    dens_grid(D, k, X, v, E, R, cb, act, cut);
    // s = 2^{-3j/2} (P x P x P) v  (eq. fvals2coefs in tensor form)
    mode_product(v, t1, P, 2, k);
    mode_product(t1, t2, P, 1, k);
    mode_product(t2, s, P, 0, k);
    const double sc = exp2(-1.5 * j);
    for (int idx = tid; idx < k3; idx += blockDim.x) s[idx] *= sc;
    __syncthreads();
    int ref = (mode == 1);
    if (mode == 0) {
        double err = 0.0;
        const double hc = 0.5 * h, up = exp2(1.5 * j);
        for (int o = 0; o < 8; ++o) {
            int p1 = (o >> 2) & 1, p2 = (o >> 1) & 1, p3 = o & 1;
            // interpolate: f~ = 2^{3j/2} sum_i s_i prod_d phi_{i_d}((g_q + p_d)/2)
            mode_product(s, t1, Q + p3 * kk, 2, k);
            mode_product(t1, t2, Q + p2 * kk, 1, k);
            mode_product(t2, t1, Q + p1 * kk, 0, k);
            // the child's GL grid, its density values into v
            for (int e = tid; e < 3 * k; e += blockDim.x) {
                const int d = e / k, q = e % k;
                X[e] = (g[q] + (d == 0 ? 2 * a1 + p1 : (d == 1 ? 2 * a2 + p2 : 2 * a3 + p3))) * hc;
            }
            for (int idx = tid; idx < k3; idx += blockDim.x) v[idx] = 0.0;
            __syncthreads();
            dens_grid(D, k, X, v, E, R, cb, act, cut);
            for (int idx = tid; idx < k3; idx += blockDim.x) err = fmax(err, fabs(v[idx] - up * t1[idx]));
            __syncthreads();
        }
        err = block_max(err, red);
        ref = err > *tolp;
        if (ref && at_max) {
            ref = 0;
            if (tid == 0) atomicExch(depth_hit, 1);
        }
    }
    for (int idx = tid; idx < k3; idx += blockDim.x) s_out[(size_t)b * k3 + idx] = s[idx];
    if (tid == 0) refine[b] = ref;
}

// children of refined boxes (octant order) and the refined-parent list
__global__ void k_make_children(int nb, const int32_t* boxes, const int32_t* refine, const int32_t* pos,
                                int32_t* next, int32_t* parent_local) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb || !refine[b]) return;
    int p = pos[b];
    parent_local[p] = b;
    for (int o = 0; o < 8; ++o) {
        int c = 8 * p + o;
        next[3 * c] = 2 * boxes[3 * b] + ((o >> 2) & 1);
        next[3 * c + 1] = 2 * boxes[3 * b + 1] + ((o >> 1) & 1);
        next[3 * c + 2] = 2 * boxes[3 * b + 2] + (o & 1);
    }
}

// scatter one level into the final node arrays
__global__ void k_place_level(int nb, int j, int base, int next_base, const int32_t* boxes, const int32_t* refine,
                              const int32_t* pos, const int32_t* parent_local, int prev_base, int k3,
                              const double* s_lvl, mra::TreeArrays a, double* s) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    int i = base + b;
    a.key[i] = morton3(boxes[3 * b], boxes[3 * b + 1], boxes[3 * b + 2]);
    a.coord[4 * i] = j;
    a.coord[4 * i + 1] = boxes[3 * b];
    a.coord[4 * i + 2] = boxes[3 * b + 1];
    a.coord[4 * i + 3] = boxes[3 * b + 2];
    a.leaf[i] = refine[b] ? 0 : 1;
    a.child[i] = refine[b] ? next_base + 8 * pos[b] : -1;
    a.parent[i] = (j == 0) ? -1 : prev_base + parent_local[b / 8];
    // (the level's blocks are copied as one contiguous range by the caller)
}

int build_tree_impl(const mra_density* f, int k, double eps, int max_level, int uniform_level, int init_level,
                    const Alloc& A, mra_tree** out) {
    cudaStream_t st = A.stream;
    const int k3 = k * k * k;
    const int ng = f->n;
    Scratch tmp(A);  // everything but the tree itself
    double* dd;
    MRA_TRY(tmp.get(&dd, 6 * (size_t)ng + 1));
    {
        std::vector<double> h(6 * (size_t)ng + 1, 0.0);
        for (int g = 0; g < ng; ++g) {
            h[g] = f->coef_host[g];
            h[ng + g] = f->r2coef_host ? f->r2coef_host[g] : 0.0;
            h[2 * ng + g] = f->expo_host[g];
            for (int d = 0; d < 3; ++d) h[3 * ng + 3 * g + d] = f->center_host[3 * g + d];
        }
        MRA_CK(cudaMemcpyAsync(dd, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice, st));
        MRA_CK(cudaStreamSynchronize(st));
    }
    DensDev D{ng, dd, dd + ng, dd + 2 * ng, dd + 3 * ng};
    double* tol;
    int32_t *flags;  // [0] depth_hit, [1] total
    MRA_TRY(tmp.get(&tol, 2));
    MRA_TRY(tmp.get(&flags, 4));
    MRA_CK(cudaMemsetAsync(flags, 0, 4 * sizeof(int32_t), st));
    k_dens_scale<<<1, 256, 0, st>>>(D, eps, tol);
    MRA_CK_LAUNCH();

    struct Level {
        int n;
        int32_t *boxes, *refine, *pos, *parent_local;
        double* s;
    };
    std::vector<Level> L;
    int32_t* boxes0;
    MRA_TRY(tmp.get(&boxes0, 3));
    MRA_CK(cudaMemsetAsync(boxes0, 0, 3 * sizeof(int32_t), st));
    int nb = 1;
    int32_t* cur = boxes0;
    int32_t* plocal_prev = nullptr;
    const size_t smem =
        (2 * k + 3 * k * k + 4 * (size_t)k3 + 3 * k + 2 * DG_CHUNK * 3 * (size_t)k + 2 * DG_CHUNK) * sizeof(double);
    MRA_CK(cudaFuncSetAttribute(k_build_level, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    for (int j = 0; j <= max_level; ++j) {
        Level lv{nb, cur, nullptr, nullptr, plocal_prev, nullptr};
        MRA_TRY(tmp.get(&lv.refine, nb));
        MRA_TRY(tmp.get(&lv.pos, nb));
        MRA_TRY(tmp.get(&lv.s, (size_t)nb * k3));
        int mode;
        if (uniform_level >= 0) mode = (j < uniform_level) ? 1 : 2;
        else mode = (j < init_level) ? 1 : 0;
        if (j == max_level && mode == 1) mode = 2;
        k_build_level<<<nb, 128, smem, st>>>(k, j, D, cur, tol, mode, j >= max_level, lv.s, lv.refine, flags);
        MRA_CK_LAUNCH();
        MRA_TRY(scan_exclusive(lv.refine, lv.pos, nb, flags + 1, st));
        int32_t nref = 0;
        MRA_CK(cudaMemcpyAsync(&nref, flags + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        MRA_CK(cudaStreamSynchronize(st));
        L.push_back(lv);
        if (nref == 0) break;
        int32_t *next, *plocal;
        MRA_TRY(tmp.get(&next, 3 * 8 * (size_t)nref));
        MRA_TRY(tmp.get(&plocal, nref));
        k_make_children<<<(nb + 255) / 256, 256, 0, st>>>(nb, cur, lv.refine, lv.pos, next, plocal);
        MRA_CK_LAUNCH();
        cur = next;
        nb = 8 * nref;
        plocal_prev = plocal;
    }
    mra_tree* t = new mra_tree();
    t->magic = MRA_TREE_MAGIC;
    t->k = k;
    t->A = A;
    t->state = MRA_TREE_LEAVES;
    // the new tree is freed on every error return below
    struct TreeGuard {
        mra_tree* t;
        ~TreeGuard() {
            if (t) mra_free_tree(t);
        }
    } tg{t};
    int n = 0;
    for (auto& lv : L) n += lv.n;
    MRA_TRY(tree_alloc_arrays(t, n, true));
    t->nlev = (int)L.size();
    int base = 0;
    for (int j = 0; j < MRA_MAX_LEVEL + 2; ++j) t->off[j] = n;
    for (int j = 0; j < t->nlev; ++j) {
        t->off[j] = base;
        base += L[j].n;
    }
    base = 0;
    for (int j = 0; j < t->nlev; ++j) {
        int nbj = L[j].n;
        int next_base = base + nbj;
        int prev_base = j ? t->off[j - 1] : 0;
        k_place_level<<<(nbj + 127) / 128, 128, 0, st>>>(nbj, j, base, next_base, L[j].boxes, L[j].refine, L[j].pos,
                                                          L[j].parent_local, prev_base, k3, L[j].s, t->a, t->s);
        MRA_CK_LAUNCH();
        MRA_CK(cudaMemcpyAsync(t->s + (size_t)base * k3, L[j].s, (size_t)nbj * k3 * sizeof(double),
                               cudaMemcpyDeviceToDevice, st));
        base = next_base;
    }
    MRA_CK(cudaMemcpyAsync(t->a.off, t->off, sizeof(t->off), cudaMemcpyHostToDevice, st));
    MRA_CK(cudaMemsetAsync(t->dnorm, 0, n * sizeof(double), st));
    int32_t hit = 0;
    MRA_CK(cudaMemcpyAsync(&hit, flags, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    MRA_CK(cudaStreamSynchronize(st));
    t->depth_hit = hit;
    tg.t = nullptr;
    *out = t;
    return hit ? MRA_EDEPTH : MRA_OK;
}

// ------------------------------------------------------------ two-scale transforms
// Block per node of level j (internal nodes only do work).
// compress: the 8 children's blocks form a (2k)^3 cube, W is applied along each
// direction, the k^3 corner is the parent's s and the rest its wavelet cube.
__global__ void k_compress_level(int k, int lo, int hi, const int32_t* child, double* s, double* dnorm,
                                 double* dcube, const double* filt) {
    extern __shared__ double cube[];
    __shared__ double red[32];
    const int i = lo + blockIdx.x;
    if (i >= hi || child[i] < 0) return;
    const int n2 = 2 * k, k3 = k * k * k, c0 = child[i];
    const double* W = filt + 2 * k * k;
    for (int e = threadIdx.x; e < 8 * k3; e += blockDim.x) {
        int o = e / k3, r = e % k3;
        int i3 = r % k, i2 = (r / k) % k, i1 = r / (k * k);
        int x1 = ((o >> 2) & 1) * k + i1, x2 = ((o >> 1) & 1) * k + i2, x3 = (o & 1) * k + i3;
        cube[(x1 * n2 + x2) * n2 + x3] = s[(size_t)(c0 + o) * k3 + r];
    }
    __syncthreads();
    for (int d = 0; d < 3; ++d) cube_transform(cube, n2, W, 0, d);
    double acc = 0.0;
    const int n3 = n2 * n2 * n2;
    for (int e = threadIdx.x; e < n3; e += blockDim.x) {
        int x3 = e % n2, x2 = (e / n2) % n2, x1 = e / (n2 * n2);
        bool corner = x1 < k && x2 < k && x3 < k;
        double v = cube[e];
        if (corner) s[(size_t)i * k3 + (x1 * k + x2) * k + x3] = v;
        else acc += v * v;
        if (dcube) dcube[(size_t)i * n3 + e] = corner ? 0.0 : v;
    }
    acc = block_sum(acc, red);
    if (threadIdx.x == 0) dnorm[i] = sqrt(acc);
}

// inverse (dcube != NULL: full s+d) or assemble (dcube == NULL: d = 0, the
// children accumulate the upsampled parent block, eq. g_assemble).
__global__ void k_expand_level(int k, int lo, int hi, const int32_t* child, double* s, const double* dcube,
                               const double* filt) {
    extern __shared__ double cube[];
    const int i = lo + blockIdx.x;
    if (i >= hi || child[i] < 0) return;
    const int n2 = 2 * k, k3 = k * k * k, c0 = child[i], n3 = n2 * n2 * n2;
    const double* W = filt + 2 * k * k;
    for (int e = threadIdx.x; e < n3; e += blockDim.x) {
        int x3 = e % n2, x2 = (e / n2) % n2, x1 = e / (n2 * n2);
        bool corner = x1 < k && x2 < k && x3 < k;
        double v = corner ? s[(size_t)i * k3 + (x1 * k + x2) * k + x3] : 0.0;
        if (dcube && !corner) v = dcube[(size_t)i * n3 + e];
        cube[e] = v;
    }
    __syncthreads();
    for (int d = 0; d < 3; ++d) cube_transform(cube, n2, W, 1, d);
    for (int e = threadIdx.x; e < 8 * k3; e += blockDim.x) {
        int o = e / k3, r = e % k3;
        int i3 = r % k, i2 = (r / k) % k, i1 = r / (k * k);
        int x1 = ((o >> 2) & 1) * k + i1, x2 = ((o >> 1) & 1) * k + i2, x3 = (o & 1) * k + i3;
        double v = cube[(x1 * n2 + x2) * n2 + x3];
        size_t dst = (size_t)(c0 + o) * k3 + r;
        if (dcube) s[dst] = v;
        else s[dst] += v;
    }
}

// One stage of a separable transform in shared memory: `in` has extents
// (n[0], n[1], n[2]) with n[dim] = nin; `out` has the same extents except
// nout along dim; out = Mat (nout x nin, row-major) applied along dim.
__device__ void stage_mul(const double* in, double* out, const int* n, int dim, const double* Mat, int nout) {
    const int nin = n[dim];
    int e[3] = {n[0], n[1], n[2]};
    e[dim] = nout;
    const int total = e[0] * e[1] * e[2];
    const int sin[3] = {n[1] * n[2], n[2], 1};
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        int x[3] = {idx / (e[1] * e[2]), (idx / e[2]) % e[1], idx % e[2]};
        const int r = x[dim];
        x[dim] = 0;
        const double* src = in + x[0] * sin[0] + x[1] * sin[1] + x[2] * sin[2];
        const int st = sin[dim];
        double acc = 0.0;
        for (int c = 0; c < nin; ++c) acc += Mat[r * nin + c] * src[c * st];
        out[idx] = acc;
    }
    __syncthreads();
}

// U = [H0^T; H1^T] (2k x k): child block p from its parent, U[(p k + a)][i] = H^(p)[i][a];
// D = U^T (k x 2k): parent block from its two children (the top rows of W).
__device__ void load_UD(int k, const double* filt, double* U, double* D) {
    const int kk = k * k;
    for (int e = threadIdx.x; e < 2 * kk; e += blockDim.x) {
        const int p = e / kk, i = (e / k) % k, a = e % k;  // H^(p)[i][a]
        const double h = filt[p * kk + i * k + a];
        U[(p * k + a) * k + i] = h;
        D[i * 2 * k + p * k + a] = h;
    }
    __syncthreads();
}

// Assembly (eq. g_assemble) with d = 0: children += (U x U x U) s_parent, in
// three stages (2k^4 + 4k^4 + 8k^4 multiply-adds).  Block per node of level j.
__global__ void k_up_level(int k, int lo, int hi, const int32_t* child, double* s, const double* filt) {
    extern __shared__ double sm[];
    const int i = lo + blockIdx.x;
    if (i >= hi || child[i] < 0) return;
    const int k2 = 2 * k, k3 = k * k * k, c0 = child[i];
    double* U = sm;
    double* D = U + 2 * k * k;
    double* x = D + 2 * k * k;     // k^3
    double* t1 = x + k3;           // 2k^3
    double* t2 = t1 + 2 * k3;      // 4k^3
    load_UD(k, filt, U, D);
    for (int e = threadIdx.x; e < k3; e += blockDim.x) x[e] = s[(size_t)i * k3 + e];
    __syncthreads();
    int n0[3] = {k, k, k};
    stage_mul(x, t1, n0, 0, U, k2);
    int n1[3] = {k2, k, k};
    stage_mul(t1, t2, n1, 1, U, k2);
    // last stage on the fly, added into the children (octant (p1 p2 p3))
    for (int idx = threadIdx.x; idx < 8 * k3; idx += blockDim.x) {
        const int x1 = idx / (k2 * k2), x2 = (idx / k2) % k2, x3 = idx % k2;
        const double* src = t2 + (x1 * k2 + x2) * k;
        double acc = 0.0;
        for (int c = 0; c < k; ++c) acc += U[x3 * k + c] * src[c];
        const int o = ((x1 / k) << 2) | ((x2 / k) << 1) | (x3 / k);
        s[(size_t)(c0 + o) * k3 + ((x1 % k) * k + (x2 % k)) * k + (x3 % k)] += acc;
    }
}

// Redundant tree without stored wavelet cubes: s_parent = (D x D x D) cube of
// the children (eq. decomp_scaling, 8k^4 + 4k^4 + 2k^4), and the wavelet norm
// as ||cube - (U x U x U) s_parent||, which equals ||d|| because the filter
// matrix is orthogonal (cube = W^T [s; d]).  Block per node of level j.
__global__ void k_compress_fast_level(int k, int lo, int hi, const int32_t* child, double* s, double* dnorm,
                                      const double* filt, int norms) {
    extern __shared__ double sm[];
    __shared__ double red[32];
    const int i = lo + blockIdx.x;
    if (i >= hi || child[i] < 0) return;
    const int k2 = 2 * k, k3 = k * k * k, c0 = child[i];
    double* U = sm;
    double* D = U + 2 * k * k;
    double* cube = D + 2 * k * k;  // 8k^3
    double* r1 = cube + 8 * k3;    // 4k^3  (k, 2k, 2k), later (2k, 2k, k)
    double* r2 = r1 + 4 * k3;      // 2k^3  (k, k, 2k),  later (2k, k, k)
    double* sp = r2 + 2 * k3;      // k^3
    load_UD(k, filt, U, D);
    for (int e = threadIdx.x; e < 8 * k3; e += blockDim.x) {
        const int o = e / k3, r = e % k3;
        const int i1 = r / (k * k), i2 = (r / k) % k, i3 = r % k;
        const int x1 = ((o >> 2) & 1) * k + i1, x2 = ((o >> 1) & 1) * k + i2, x3 = (o & 1) * k + i3;
        cube[(x1 * k2 + x2) * k2 + x3] = s[(size_t)(c0 + o) * k3 + r];
    }
    __syncthreads();
    int n0[3] = {k2, k2, k2};
    stage_mul(cube, r1, n0, 0, D, k);
    int n1[3] = {k, k2, k2};
    stage_mul(r1, r2, n1, 1, D, k);
    int n2[3] = {k, k, k2};
    stage_mul(r2, sp, n2, 2, D, k);
    for (int e = threadIdx.x; e < k3; e += blockDim.x) s[(size_t)i * k3 + e] = sp[e];
    if (!norms) return;
    int m0[3] = {k, k, k};
    stage_mul(sp, r2, m0, 0, U, k2);
    int m1[3] = {k2, k, k};
    stage_mul(r2, r1, m1, 1, U, k2);
    double acc = 0.0;
    for (int idx = threadIdx.x; idx < 8 * k3; idx += blockDim.x) {
        const int x1 = idx / (k2 * k2), x2 = (idx / k2) % k2, x3 = idx % k2;
        const double* src = r1 + (x1 * k2 + x2) * k;
        double up = 0.0;
        for (int c = 0; c < k; ++c) up += U[x3 * k + c] * src[c];
        const double dv = cube[idx] - up;
        acc += dv * dv;
    }
    acc = block_sum(acc, red);
    if (threadIdx.x == 0) dnorm[i] = sqrt(acc);
}

// ---- triangular two-scale filters, one fiber per thread
// H^(p)_{ia} = (1/sqrt 2) int_0^1 phi_i((u + p)/2) phi_a(u) du vanishes for a > i:
// phi_i((u + p)/2) is a polynomial of degree i in u, and phi_a is orthogonal to
// every polynomial of lower degree.  So D = [H0 | H1] (k x 2k, parent from
// children) has in row i the columns a <= i of each half, and U = D^T (2k x k,
// child from parent) has in row p k + a the columns i >= a: the mode products
// below skip the structural zeros (k(k+1) multiply-adds per fiber instead of
// 2k^2).  Each thread takes whole fibers along the contracted direction: it
// loads the fiber's inputs into registers and writes all its outputs, so the
// triangular loop bounds are compile-time constants and no warp diverges.
// Shared-memory arrays keep their innermost extent padded to an odd number of
// doubles, so that fibers along it (one per thread) hit distinct banks.
enum { TRI_DENSE = 0, TRI_D = 1, TRI_U = 2 };

// in: extents (N0, N1, N2), strides (IS0, IS1, 1); out: the same with NOUT along DIM,
// strides (OS0, OS1, 1); Mat: NOUT x NIN row-major with structure TRI (KT = k)
template <int N0, int N1, int N2, int IS0, int IS1, int DIM, int NOUT, int OS0, int OS1, int TRI, int KT>
__device__ __forceinline__ void fiber_stage(const double* in, double* out, const double* Mat) {
    constexpr int NIN = DIM == 0 ? N0 : (DIM == 1 ? N1 : N2);
    constexpr int IST = DIM == 0 ? IS0 : (DIM == 1 ? IS1 : 1);
    constexpr int OST = DIM == 0 ? OS0 : (DIM == 1 ? OS1 : 1);
    constexpr int FA = DIM == 0 ? N1 : N0, FB = DIM == 2 ? N1 : N2;  // the fiber's two other coordinates
    constexpr int IA = DIM == 0 ? IS1 : IS0, IB = DIM == 2 ? IS1 : 1;
    constexpr int OA = DIM == 0 ? OS1 : OS0, OB = DIM == 2 ? OS1 : 1;
    for (int f = threadIdx.x; f < FA * FB; f += blockDim.x) {
        const int a = f / FB, b = f - a * FB;
        const double* src = in + a * IA + b * IB;
        double v[NIN];
#pragma unroll
        for (int c = 0; c < NIN; ++c) v[c] = src[c * IST];
        double* dst = out + a * OA + b * OB;
#pragma unroll
        for (int r = 0; r < NOUT; ++r) {
            double acc = 0.0;
#pragma unroll
            for (int c = 0; c < NIN; ++c) {
                const bool nz = TRI == TRI_DENSE || (TRI == TRI_D && (c % KT) <= r) || (TRI == TRI_U && c >= r % KT);
                if (nz) acc += Mat[r * NIN + c] * v[c];
            }
            dst[r * OST] = acc;
        }
    }
    __syncthreads();
}

template <int K>
struct TriSmem {
    static constexpr int K2 = 2 * K, P2 = K2 + 1, P1 = K + 1;  // padded innermost extents
    static constexpr int MATS = 4 * K * K;                   // U (2k x k) and D (k x 2k)
    static constexpr int CUBE = K2 * K2 * P2;                // (2k, 2k, 2k)
    static constexpr int RA = K * K2 * P2 > K2 * K * P1 ? K * K2 * P2 : K2 * K * P1;  // (k,2k,2k) | (2k,k,k)
    static constexpr int RB = K * K * P2 > K2 * K2 * P1 ? K * K * P2 : K2 * K2 * P1;  // (k,k,2k) | (2k,2k,k)
    static constexpr int SP = K * K * P1;                                            // (k, k, k)
};

// Redundant tree, scaling part: s_parent = (D x D x D) cube of the children (eq.
// decomp_scaling).  Block per internal node of level j: the children of level j's
// internal nodes are the level-(j+1) nodes in groups of eight, in the order of their
// parents, so block b takes the group at cbase + 8 b (cbase: level j+1's first node)
// and its parent.  The wavelet norms follow for all levels at once (k_wnorm_all).
template <int K>
__global__ void k_compress_fast_level_t(int cbase, const int32_t* parent, double* s, const double* filt) {
    using L = TriSmem<K>;
    constexpr int K2 = 2 * K, K3 = K * K * K, P1 = L::P1, P2 = L::P2;
    extern __shared__ double sm[];
    const int c0 = cbase + 8 * blockIdx.x;
    const int i = parent[c0];
    double* U = sm;
    double* D = U + 2 * K * K;
    double* cube = D + 2 * K * K;  // (2k, 2k, 2k), stride P2
    double* ra = cube + L::CUBE;
    double* rb = ra + L::RA;
    double* sp = rb + L::RB;       // (k, k, k), stride P1
    load_UD(K, filt, U, D);
    for (int e = threadIdx.x; e < 8 * K3; e += blockDim.x) {
        const int o = e / K3, r = e % K3;
        const int i1 = r / (K * K), i2 = (r / K) % K, i3 = r % K;
        const int x1 = ((o >> 2) & 1) * K + i1, x2 = ((o >> 1) & 1) * K + i2, x3 = (o & 1) * K + i3;
        cube[(x1 * K2 + x2) * P2 + x3] = s[(size_t)(c0 + o) * K3 + r];
    }
    __syncthreads();
    fiber_stage<K2, K2, K2, K2 * P2, P2, 0, K, K2 * P2, P2, TRI_D, K>(cube, ra, D);  // (k, 2k, 2k)
    fiber_stage<K, K2, K2, K2 * P2, P2, 1, K, K * P2, P2, TRI_D, K>(ra, rb, D);      // (k, k, 2k)
    fiber_stage<K, K, K2, K * P2, P2, 2, K, K * P1, P1, TRI_D, K>(rb, sp, D);        // (k, k, k)
    for (int e = threadIdx.x; e < K3; e += blockDim.x) {
        const int i1 = e / (K * K), i2 = (e / K) % K, i3 = e % K;
        s[(size_t)i * K3 + e] = sp[(i1 * K + i2) * P1 + i3];
    }
}

// ---- the scaling blocks of a small level: one parent over k/2 blocks
// Block (b, q) computes rows i1 in {q, K-1-q} of the parent's block (the contractions
// along directions 2 and 3 never mix rows of direction 1), one output element per
// thread and step.  It pays where a level has fewer parents than SMs: each parent then
// runs on k/2 SMs; on the large levels the per-parent kernel below is faster.
template <int K>
__global__ void __launch_bounds__(128) k_down_slice(int cbase, const int32_t* parent, double* s,
                                                    const double* filt) {
    constexpr int K2 = 2 * K, K3 = K * K * K, P2 = K2 + 1, R = 2;
    __shared__ double D[K * K2];
    __shared__ double cube[K2 * K2 * P2];  // (x1, x2, x3), x3 padded
    __shared__ double o1[R * K2 * P2];     // (r, x2, x3)
    __shared__ double o2[R * K * P2];      // (r, i2, x3)
    const int c0 = cbase + 8 * blockIdx.x, i = parent[c0], q = blockIdx.y, tid = threadIdx.x;
    for (int e = tid; e < 2 * K * K; e += blockDim.x) {
        const int p = e / (K * K), ii = (e / K) % K, a = e % K;  // H^(p)[ii][a]
        D[ii * K2 + p * K + a] = filt[p * K * K + ii * K + a];
    }
    for (int e = tid; e < 8 * K3; e += blockDim.x) {
        const int o = e / K3, r = e % K3;
        const int i1 = r / (K * K), i2 = (r / K) % K, i3 = r % K;
        const int x1 = ((o >> 2) & 1) * K + i1, x2 = ((o >> 1) & 1) * K + i2, x3 = (o & 1) * K + i3;
        cube[(x1 * K2 + x2) * P2 + x3] = s[(size_t)(c0 + o) * K3 + r];
    }
    __syncthreads();
    // direction 1: D = [H0 | H1] has in row i the columns a <= i of each half
    for (int e = tid; e < R * K2 * K2; e += blockDim.x) {
        const int r = e / (K2 * K2), x2 = (e / K2) % K2, x3 = e % K2, i1 = r ? K - 1 - q : q;
        const double* Dr = D + i1 * K2;
        double acc = 0.0;
        for (int a = 0; a <= i1; ++a)
            acc += Dr[a] * cube[(a * K2 + x2) * P2 + x3] + Dr[K + a] * cube[((K + a) * K2 + x2) * P2 + x3];
        o1[(r * K2 + x2) * P2 + x3] = acc;
    }
    __syncthreads();
    // direction 2 (i2 slowest: a warp shares its loop bound)
    for (int e = tid; e < R * K * K2; e += blockDim.x) {
        const int i2 = e / (R * K2), r = (e / K2) % R, x3 = e % K2;
        const double* Dr = D + i2 * K2;
        double acc = 0.0;
        for (int a = 0; a <= i2; ++a)
            acc += Dr[a] * o1[(r * K2 + a) * P2 + x3] + Dr[K + a] * o1[(r * K2 + K + a) * P2 + x3];
        o2[(r * K + i2) * P2 + x3] = acc;
    }
    __syncthreads();
    // direction 3, into rows i1 of the parent's block
    for (int e = tid; e < R * K * K; e += blockDim.x) {
        const int i3 = e / (R * K), r = (e / K) % R, i2 = e % K, i1 = r ? K - 1 - q : q;
        const double* Dr = D + i3 * K2;
        const double* src = o2 + (r * K + i2) * P2;
        double acc = 0.0;
        for (int a = 0; a <= i3; ++a) acc += Dr[a] * src[a] + Dr[K + a] * src[K + a];
        s[(size_t)i * K3 + (i1 * K + i2) * K + i3] = acc;
    }
}

// ---- the assembly sliced: one parent over k/2 blocks
// Each block takes four rows x1 of the children's cube, r, k-1-r, k+r and 2k-1-r (their
// triangular loops then have equal length), and runs the three contractions for those
// rows alone: the contractions along directions 2 and 3 never mix rows of direction 1.
// A level's work thus spreads over k/2 times as many blocks, which balances the large
// levels over the SMs and runs a small level's few parents on several SMs each.

// Assembly (eq. g_assemble, d = 0): children += (U x U x U) s_parent, U = D^T (row
// p K + r has the columns c >= r), rows x1 in {q, K-1-q, K+q, 2K-1-q} of the cube.
template <int K>
__global__ void __launch_bounds__(128) k_up_slice(int cbase, const int32_t* parent, double* s, const double* filt) {
    constexpr int K2 = 2 * K, K3 = K * K * K, P1 = K + 1, RX = 4;
    __shared__ double U[K2 * K];
    __shared__ double sp[K * K * P1];    // (i1, i2, i3), i3 padded
    __shared__ double t1[RX * K * P1];   // (rx, i2, i3)
    __shared__ double t2[RX * K2 * P1];  // (rx, x2, i3)
    const int c0 = cbase + 8 * blockIdx.x, i = parent[c0], q = blockIdx.y, tid = threadIdx.x;
    for (int e = tid; e < 2 * K * K; e += blockDim.x) {
        const int p = e / (K * K), ii = (e / K) % K, a = e % K;  // H^(p)[ii][a]
        U[(p * K + a) * K + ii] = filt[p * K * K + ii * K + a];
    }
    for (int e = tid; e < K3; e += blockDim.x) {
        const int i1 = e / (K * K), i2 = (e / K) % K, i3 = e % K;
        sp[(i1 * K + i2) * P1 + i3] = s[(size_t)i * K3 + e];
    }
    __syncthreads();
    auto row_x1 = [&](int rx) { return (rx & 2 ? K : 0) + (rx & 1 ? K - 1 - q : q); };
    // direction 1
    for (int e = tid; e < RX * K * K; e += blockDim.x) {
        const int rx = e / (K * K), i2 = (e / K) % K, i3 = e % K, x1 = row_x1(rx);
        const double* Ur = U + x1 * K;
        double acc = 0.0;
        for (int c = x1 % K; c < K; ++c) acc += Ur[c] * sp[(c * K + i2) * P1 + i3];
        t1[(rx * K + i2) * P1 + i3] = acc;
    }
    __syncthreads();
    // direction 2 (x2 slowest: a warp shares its loop bound)
    for (int e = tid; e < RX * K2 * K; e += blockDim.x) {
        const int x2 = e / (RX * K), rx = (e / K) % RX, i3 = e % K;
        const double* Ur = U + x2 * K;
        double acc = 0.0;
        for (int c = x2 % K; c < K; ++c) acc += Ur[c] * t1[(rx * K + c) * P1 + i3];
        t2[(rx * K2 + x2) * P1 + i3] = acc;
    }
    __syncthreads();
    // direction 3, added into the children's blocks
    for (int e = tid; e < RX * K2 * K2; e += blockDim.x) {
        const int rx = e / (K2 * K2), x2 = (e / K2) % K2, x3 = e % K2, x1 = row_x1(rx);
        const double* Ur = U + x3 * K;
        const double* src = t2 + (rx * K2 + x2) * P1;
        double acc = 0.0;
        for (int c = x3 % K; c < K; ++c) acc += Ur[c] * src[c];
        const int o = ((x1 / K) << 2) | ((x2 / K) << 1) | (x3 / K);
        s[(size_t)(c0 + o) * K3 + ((x1 % K) * K + x2 % K) * K + x3 % K] += acc;
    }
}

// Wavelet norms of every internal node at once (after the scaling blocks of all
// levels are in place): ||cube - (U x U x U) s_parent|| = ||d|| (the filter matrix is
// orthogonal).  Block g takes the sibling group at 1 + 8 g -- the groups of all
// levels in turn -- and its parent.
template <int K>
__global__ void k_wnorm_all(const int32_t* parent, const double* s, double* dnorm, const double* filt) {
    using L = TriSmem<K>;
    constexpr int K2 = 2 * K, K3 = K * K * K, P1 = L::P1, P2 = L::P2;
    extern __shared__ double sm[];
    __shared__ double red[32];
    const int c0 = 1 + 8 * blockIdx.x;
    const int i = parent[c0];
    double* U = sm;
    double* D = U + 2 * K * K;
    double* cube = D + 2 * K * K;  // (2k, 2k, 2k), stride P2
    double* ra = cube + L::CUBE;
    double* rb = ra + L::RA;
    double* sp = rb + L::RB;       // (k, k, k), stride P1
    load_UD(K, filt, U, D);
    for (int e = threadIdx.x; e < 8 * K3; e += blockDim.x) {
        const int o = e / K3, r = e % K3;
        const int i1 = r / (K * K), i2 = (r / K) % K, i3 = r % K;
        const int x1 = ((o >> 2) & 1) * K + i1, x2 = ((o >> 1) & 1) * K + i2, x3 = (o & 1) * K + i3;
        cube[(x1 * K2 + x2) * P2 + x3] = s[(size_t)(c0 + o) * K3 + r];
    }
    for (int e = threadIdx.x; e < K3; e += blockDim.x) {
        const int i1 = e / (K * K), i2 = (e / K) % K, i3 = e % K;
        sp[(i1 * K + i2) * P1 + i3] = s[(size_t)i * K3 + e];
    }
    __syncthreads();
    fiber_stage<K, K, K, K * P1, P1, 0, K2, K * P1, P1, TRI_U, K>(sp, ra, U);       // (2k, k, k)
    fiber_stage<K2, K, K, K * P1, P1, 1, K2, K2 * P1, P1, TRI_U, K>(ra, rb, U);     // (2k, 2k, k)
    double acc = 0.0;
    for (int f = threadIdx.x; f < K2 * K2; f += blockDim.x) {
        const int x1 = f / K2, x2 = f % K2;
        const double* src = rb + (x1 * K2 + x2) * P1;
        const double* cb = cube + (x1 * K2 + x2) * P2;
        double v[K];
#pragma unroll
        for (int c = 0; c < K; ++c) v[c] = src[c];
#pragma unroll
        for (int r = 0; r < K2; ++r) {
            double up = 0.0;
#pragma unroll
            for (int c = 0; c < K; ++c)
                if (c >= r % K) up += U[r * K + c] * v[c];
            const double dv = cb[r] - up;
            acc += dv * dv;
        }
    }
    acc = block_sum(acc, red);
    if (threadIdx.x == 0) dnorm[i] = sqrt(acc);
}

template <int K>
static int compress_fast_t(mra_tree* t, bool norms, cudaStream_t st) {
    // the scaling blocks level by level, then the wavelet norms of all internal nodes in
    // one launch
    using L = TriSmem<K>;
    const size_t smem = (size_t)(L::MATS + L::CUBE + L::RA + L::RB + L::SP) * sizeof(double);
    MRA_CK(cudaFuncSetAttribute(k_compress_fast_level_t<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    for (int j = t->nlev - 2; j >= 0; --j) {
        const int nparents = (t->off[j + 2] - t->off[j + 1]) / 8;
        if (nparents <= 0) continue;
        if (2 * nparents < num_sms())  // a small level: each parent over k/2 blocks
            k_down_slice<K><<<dim3(nparents, K / 2), 128, 0, st>>>(t->off[j + 1], t->a.parent, t->s, t->filt);
        else
            k_compress_fast_level_t<K><<<nparents, 256, smem, st>>>(t->off[j + 1], t->a.parent, t->s, t->filt);
        MRA_CK_LAUNCH();
    }
    if (norms && t->n > 1) {
        MRA_CK(cudaFuncSetAttribute(k_wnorm_all<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_wnorm_all<K><<<(t->n - 1) / 8, 256, smem, st>>>(t->a.parent, t->s, t->dnorm, t->filt);
        MRA_CK_LAUNCH();
    }
    return MRA_OK;
}

template <int K>
static int assemble_t(mra_tree* t, cudaStream_t st) {
    for (int j = 0; j + 1 < t->nlev; ++j) {
        const int nparents = (t->off[j + 2] - t->off[j + 1]) / 8;
        if (nparents <= 0) continue;
        k_up_slice<K><<<dim3(nparents, K / 2), 128, 0, st>>>(t->off[j + 1], t->a.parent, t->s, t->filt);
        MRA_CK_LAUNCH();
    }
    return MRA_OK;
}

static int cube_smem(int k, size_t* bytes, const void* fn) {
    *bytes = (size_t)8 * k * k * k * sizeof(double);
    MRA_CK(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)*bytes));
    return MRA_OK;
}

int compress_impl(mra_tree* t, int mode, cudaStream_t st) {
    if (mode != MRA_COMPRESS_STORE_D) {
        const int k = t->k;
        const bool norms = mode == MRA_COMPRESS_NORMS;
        if (t->dcube) {  // wavelet cubes of an earlier compress no longer match the blocks
            t->A.put(t->dcube);
            t->dcube = nullptr;
        }
        MRA_CK(cudaMemsetAsync(t->dnorm, 0, t->n * sizeof(double), st));
        if (k == 4 || k == 6 || k == 8) {
            MRA_TRY(k == 4 ? compress_fast_t<4>(t, norms, st)
                           : (k == 6 ? compress_fast_t<6>(t, norms, st) : compress_fast_t<8>(t, norms, st)));
            t->state = MRA_TREE_REDUNDANT;
            return MRA_OK;
        }
        const size_t smem = (4 * (size_t)k * k + 15 * (size_t)k * k * k) * sizeof(double);
        MRA_CK(cudaFuncSetAttribute(k_compress_fast_level, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        for (int j = t->nlev - 2; j >= 0; --j) {
            int lo = t->off[j], hi = t->off[j + 1];
            if (hi <= lo) continue;
            k_compress_fast_level<<<hi - lo, 256, smem, st>>>(k, lo, hi, t->a.child, t->s, t->dnorm, t->filt,
                                                              norms ? 1 : 0);
            MRA_CK_LAUNCH();
        }
        t->state = MRA_TREE_REDUNDANT;
        return MRA_OK;
    }
    size_t smem;
    MRA_TRY(cube_smem(t->k, &smem, (const void*)k_compress_level));
    if (!t->dcube) MRA_TRY(dalloc(t->A, &t->dcube, (size_t)t->n * 8 * t->k * t->k * t->k));
    MRA_CK(cudaMemsetAsync(t->dnorm, 0, t->n * sizeof(double), st));
    for (int j = t->nlev - 2; j >= 0; --j) {
        int lo = t->off[j], hi = t->off[j + 1];
        if (hi <= lo) continue;
        k_compress_level<<<hi - lo, 256, smem, st>>>(t->k, lo, hi, t->a.child, t->s, t->dnorm,
                                                     t->dcube, t->filt);
        MRA_CK_LAUNCH();
    }
    t->state = MRA_TREE_REDUNDANT;
    return MRA_OK;
}

int inverse_impl(mra_tree* t, cudaStream_t st) {
    if (!t->dcube) {
        set_error("inverse transform needs a tree compressed with MRA_COMPRESS_STORE_D");
        return MRA_ESTATE;
    }
    size_t smem;
    MRA_TRY(cube_smem(t->k, &smem, (const void*)k_expand_level));
    for (int j = 0; j + 1 < t->nlev; ++j) {
        int lo = t->off[j], hi = t->off[j + 1];
        k_expand_level<<<hi - lo, 256, smem, st>>>(t->k, lo, hi, t->a.child, t->s, t->dcube, t->filt);
        MRA_CK_LAUNCH();
    }
    t->state = MRA_TREE_LEAVES;
    return MRA_OK;
}

int assemble_impl(mra_tree* t, cudaStream_t st) {
    const int k = t->k;
    if (k == 4 || k == 6 || k == 8) {
        MRA_TRY(k == 4 ? assemble_t<4>(t, st) : (k == 6 ? assemble_t<6>(t, st) : assemble_t<8>(t, st)));
        t->state = MRA_TREE_LEAVES;
        return MRA_OK;
    }
    const size_t smem = (4 * (size_t)k * k + 7 * (size_t)k * k * k) * sizeof(double);
    MRA_CK(cudaFuncSetAttribute(k_up_level, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    for (int j = 0; j + 1 < t->nlev; ++j) {
        int lo = t->off[j], hi = t->off[j + 1];
        if (hi <= lo) continue;
        k_up_level<<<hi - lo, 256, smem, st>>>(k, lo, hi, t->a.child, t->s, t->filt);
        MRA_CK_LAUNCH();
    }
    t->state = MRA_TREE_LEAVES;
    return MRA_OK;
}

// ------------------------------------------------------------ truncation
// sum over the leaves of ||s||^2; a block takes whole nodes (no per-element division)
__global__ void k_leaf_norm2(int n, int k3, const int32_t* leaf, const double* s, double* out) {
    __shared__ double red[32];
    double acc = 0.0;
    for (int i = blockIdx.x; i < n; i += gridDim.x) {
        if (!leaf[i]) continue;
        const double* x = s + (size_t)i * k3;
        for (int e = threadIdx.x; e < k3; e += blockDim.x) acc += x[e] * x[e];
    }
    acc = block_sum(acc, red);
    if (threadIdx.x == 0) atomicAdd(out, acc);
}

static int leaf_norm2_grid(int n) { return std::max(1, std::min(n, num_sms() * 4)); }

int leaf_norm2(const mra_tree* t, double* out, cudaStream_t st) {
    k_leaf_norm2<<<leaf_norm2_grid(t->n), 256, 0, st>>>(t->n, t->k * t->k * t->k, t->a.leaf, t->s, out);
    MRA_CK_LAUNCH();
    return MRA_OK;
}

// merge node i when its 8 children are leaves and ||d_i||^2 < thr2
__global__ void k_merge_level(int lo, int hi, int n, const double* thr2, int32_t* leaf, const int32_t* child,
                              const double* dnorm, int32_t* alive, double* removed2) {
    int i = lo + blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= hi || leaf[i]) return;
    double t = *thr2;
    int c0 = child[i];
    for (int o = 0; o < 8; ++o)
        if (!leaf[c0 + o]) return;
    if (dnorm[i] * dnorm[i] < t) {
        leaf[i] = 1;
        for (int o = 0; o < 8; ++o) alive[c0 + o] = 0;
        atomicAdd(removed2, dnorm[i] * dnorm[i]);
    }
}

__global__ void k_thr2(const double* norm2, int n, double eps, double* thr2) {
    // (eps ||g|| / sqrt(N))^2
    *thr2 = eps * eps * (*norm2) / (double)n;
}

__global__ void k_fill_i32(int32_t* p, int n, int32_t v) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

// lev[j] = newidx[off[j]] (n2 for a level that starts at or past the end), lev[MAX+2] = n2
__global__ void k_level_starts(int n, const int32_t* off, const int32_t* newidx, const int32_t* total, int32_t* lev) {
    const int j = threadIdx.x;
    const int32_t n2 = *total;
    if (j < MRA_MAX_LEVEL + 2) lev[j] = off[j] < n ? newidx[off[j]] : n2;
    if (j == 0) lev[MRA_MAX_LEVEL + 2] = n2;
}

__global__ void k_compact(int n, int k3, const int32_t* alive, const int32_t* newidx, mra::TreeArrays a,
                          const double* s, const double* dnorm, mra::TreeArrays b, double* s2, double* dn2) {
    int i = blockIdx.x;
    if (i >= n || !alive[i]) return;
    int d = newidx[i];
    if (threadIdx.x == 0) {
        b.key[d] = a.key[i];
        for (int q = 0; q < 4; ++q) b.coord[4 * d + q] = a.coord[4 * i + q];
        b.leaf[d] = a.leaf[i];
        b.child[d] = a.leaf[i] ? -1 : newidx[a.child[i]];
        b.parent[d] = a.parent[i] < 0 ? -1 : newidx[a.parent[i]];
        dn2[d] = a.leaf[i] ? 0.0 : dnorm[i];
    }
    for (int e = threadIdx.x; e < k3; e += blockDim.x) s2[(size_t)d * k3 + e] = s[(size_t)i * k3 + e];
}

int truncate_impl(mra_tree* t, double eps, cudaStream_t st, double* removed_host) {
    const int n = t->n, k3 = t->k * t->k * t->k;
    Scratch tmpmem(t->A);
    double* dv;  // [0] ||g||^2, [1] thr^2, [2] removed^2
    int32_t *alive, *newidx, *total, *lev;
    MRA_TRY(tmpmem.get(&dv, 4));
    MRA_TRY(tmpmem.get(&alive, n));
    MRA_TRY(tmpmem.get(&newidx, n));
    MRA_TRY(tmpmem.get(&total, 1));
    MRA_TRY(tmpmem.get(&lev, MRA_MAX_LEVEL + 3));
    MRA_CK(cudaMemsetAsync(dv, 0, 4 * sizeof(double), st));
    k_leaf_norm2<<<leaf_norm2_grid(n), 256, 0, st>>>(n, k3, t->a.leaf, t->s, dv);
    MRA_CK_LAUNCH();
    k_thr2<<<1, 1, 0, st>>>(dv, n, eps, dv + 1);
    MRA_CK_LAUNCH();
    k_fill_i32<<<(n + 255) / 256, 256, 0, st>>>(alive, n, 1);
    MRA_CK_LAUNCH();
    for (int j = t->nlev - 2; j >= 0; --j) {
        int lo = t->off[j], hi = t->off[j + 1];
        if (hi <= lo) continue;
        k_merge_level<<<(hi - lo + 127) / 128, 128, 0, st>>>(lo, hi, n, dv + 1, t->a.leaf, t->a.child, t->dnorm, alive,
                                                             dv + 2);
        MRA_CK_LAUNCH();
    }
    MRA_TRY(scan_exclusive(alive, newidx, n, total, st));
    // the new first index of every level (the exclusive scan at the level's old first
    // index) and the new node count, gathered on the device: one small read-back
    k_level_starts<<<1, 32, 0, st>>>(n, t->a.off, newidx, total, lev);
    MRA_CK_LAUNCH();
    int32_t hlev[MRA_MAX_LEVEL + 3];
    double rem2 = 0.0;
    MRA_CK(cudaMemcpyAsync(hlev, lev, sizeof(hlev), cudaMemcpyDeviceToHost, st));
    MRA_CK(cudaMemcpyAsync(&rem2, dv + 2, sizeof(double), cudaMemcpyDeviceToHost, st));
    MRA_CK(cudaStreamSynchronize(st));
    const int32_t n2 = hlev[MRA_MAX_LEVEL + 2];
    if (removed_host) *removed_host = sqrt(rem2);
    if (n2 != n) {
        mra_tree tmp;
        tmp.k = t->k;
        tmp.A = t->A;
        tmp.filt = t->filt;
        const int rc = tree_alloc_arrays(&tmp, n2, true);
        if (rc != MRA_OK) {
            tree_free_arrays(&tmp);
            return rc;
        }
        k_compact<<<n, 128, 0, st>>>(n, k3, alive, newidx, t->a, t->s, t->dnorm, tmp.a, tmp.s, tmp.dnorm);
        MRA_CK_LAUNCH();
        int off2[MRA_MAX_LEVEL + 2];
        int nlev2 = 0;
        // exclusive scan at a level's old first index = its new first index
        for (int j = 0; j < MRA_MAX_LEVEL + 2; ++j) off2[j] = hlev[j];
        for (int j = 0; j < t->nlev; ++j)
            if (off2[j] < n2) nlev2 = j + 1;
        for (int j = nlev2; j < MRA_MAX_LEVEL + 2; ++j) off2[j] = n2;
        tree_free_arrays(t);
        t->a = tmp.a;
        t->s = tmp.s;
        t->dnorm = tmp.dnorm;
        t->slab = tmp.slab;
        t->n = n2;
        t->nlev = nlev2;
        memcpy(t->off, off2, sizeof(off2));
        MRA_CK(cudaMemcpyAsync(t->a.off, t->off, sizeof(t->off), cudaMemcpyHostToDevice, st));
        tmp.filt = nullptr;
    }
    return MRA_OK;
}

}  // namespace mra

namespace mra {

// ------------------------------------------------------------ output skeleton refinement
// The paper takes the output tree as a copy of the input's redundant tree and
// leaves the removal of that assumption for later (Algorithm 2/3,
// Initialization).  A potential is broader than its density: Algorithm 1 keeps
// the input tree coarse wherever the density is negligible, but there the
// output still varies on the scale of its distance to the sources.  Refinement
// pass (reading): every leaf at level j < max_level whose 26-neighbourhood at
// level j holds an internal node gets its 8 children, with the exact
// two-scale refinement of its block (the d = 0 half of eqs. recon_even /
// recon_odd), so the function represented is unchanged and the split leaf
// keeps its own block (its wavelet part is zero).  Applying the operator on
// the refined tree gives the output on the graded skeleton; the final
// truncation removes the output blocks that turn out to be insignificant.

// block per node of the refined tree: copy of an old node's block, or the
// refinement to octant (p1 p2 p3) of its parent's old block
__global__ void k_refine_blocks(int k, int n, const int32_t* src, const int32_t* oct, const double* s_old,
                                double* s_new, const double* filt) {
    extern __shared__ double sm[];
    const int k3 = k * k * k, kk = k * k;
    double* HT = sm;          // 2 k x k: HT[p][a][i] = H^(p)[i][a]
    double* x = HT + 2 * kk;  // k^3
    double* y = x + k3;
    for (int e = threadIdx.x; e < 2 * kk; e += blockDim.x) {
        const int p = e / kk, r = e % kk, a = r / k, i = r % k;
        HT[e] = filt[p * kk + i * k + a];
    }
    for (int i = blockIdx.x; i < n; i += gridDim.x) {
        const double* in = s_old + (size_t)src[i] * k3;
        double* out = s_new + (size_t)i * k3;
        const int o = oct[i];
        if (o < 0) {
            for (int e = threadIdx.x; e < k3; e += blockDim.x) out[e] = in[e];
            continue;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < k3; e += blockDim.x) x[e] = in[e];
        __syncthreads();
        // x <- (H^(p1)T x H^(p2)T x H^(p3)T) x, one direction at a time
        for (int d = 2; d >= 0; --d) {
            const int p = (o >> (2 - d)) & 1, st = d == 0 ? kk : (d == 1 ? k : 1);
            const double* H = HT + p * kk;
            for (int e = threadIdx.x; e < k3; e += blockDim.x) {
                const int c = (e / st) % k;
                const double* col = x + e - c * st;
                double acc = 0.0;
                for (int q = 0; q < k; ++q) acc += H[c * k + q] * col[q * st];
                y[e] = acc;
            }
            __syncthreads();
            for (int e = threadIdx.x; e < k3; e += blockDim.x) x[e] = y[e];
            __syncthreads();
        }
        for (int e = threadIdx.x; e < k3; e += blockDim.x) out[e] = x[e];
    }
}

// one refinement pass of t into a new tree (*out); *nsplit: leaves split
static int refine_pass(const mra_tree* t, int max_level, cudaStream_t st, mra_tree** out, int* nsplit) {
    *out = nullptr;
    const int n = t->n, k = t->k, k3 = k * k * k;
    std::vector<int32_t> coords(4 * (size_t)n), leaf(n);
    MRA_CK(cudaMemcpyAsync(coords.data(), t->a.coord, coords.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    MRA_CK(cudaMemcpyAsync(leaf.data(), t->a.leaf, n * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    MRA_CK(cudaStreamSynchronize(st));
    // internal boxes per level (keys sorted within a level, as the node order is)
    std::vector<uint64_t> key(n);
    for (int i = 0; i < n; ++i) key[i] = morton3(coords[4 * i + 1], coords[4 * i + 2], coords[4 * i + 3]);
    auto internal_at = [&](int j, int b1, int b2, int b3) {
        const int N = 1 << j;
        if (b1 < 0 || b2 < 0 || b3 < 0 || b1 >= N || b2 >= N || b3 >= N) return false;
        const uint64_t kk = morton3(b1, b2, b3);
        const int lo = t->off[j], hi = t->off[j + 1];
        const auto it = std::lower_bound(key.begin() + lo, key.begin() + hi, kk);
        return it != key.begin() + hi && *it == kk && !leaf[it - key.begin()];
    };
    std::vector<char> split(n, 0);
    int ns = 0;
    for (int i = 0; i < n; ++i) {
        const int j = coords[4 * i];
        if (!leaf[i] || j >= max_level) continue;
        bool found = false;
        for (int d = 0; d < 27 && !found; ++d) {
            if (d == 13) continue;
            found = internal_at(j, coords[4 * i + 1] + d / 9 - 1, coords[4 * i + 2] + (d / 3) % 3 - 1,
                                coords[4 * i + 3] + d % 3 - 1);
        }
        if (found) {
            split[i] = 1;
            ++ns;
        }
    }
    *nsplit = ns;
    // the new node list: every old node, and 8 children per split leaf; sorted by
    // (level, Morton key) -- a child's key is its parent's key times 8 plus its octant
    struct Rec {
        int j;
        uint64_t key;
        int32_t src, oct, leaf;
    };
    std::vector<Rec> rec;
    rec.reserve(n + 8 * (size_t)ns);
    for (int i = 0; i < n; ++i) {
        rec.push_back({coords[4 * i], key[i], i, -1, split[i] ? 0 : leaf[i]});
        if (split[i])
            for (int o = 0; o < 8; ++o) rec.push_back({coords[4 * i] + 1, (key[i] << 3) | (uint64_t)o, i, o, 1});
    }
    std::sort(rec.begin(), rec.end(), [](const Rec& a, const Rec& b) {
        return a.j != b.j ? a.j < b.j : a.key < b.key;
    });
    const int n2 = (int)rec.size();
    if (n2 >= (1 << 30) / 216) { set_error("refined tree too large (%d nodes)", n2); return MRA_EINVAL; }
    std::vector<int32_t> c2(4 * (size_t)n2), l2(n2), src(n2), oct(n2);
    for (int i = 0; i < n2; ++i) {
        const Rec& r = rec[i];
        c2[4 * i] = r.j;
        if (r.oct < 0) {
            for (int d = 1; d < 4; ++d) c2[4 * i + d] = coords[4 * r.src + d];
        } else {
            for (int d = 1; d < 4; ++d) c2[4 * i + d] = 2 * coords[4 * r.src + d] + ((r.oct >> (3 - d)) & 1);
        }
        l2[i] = r.leaf;
        src[i] = r.src;
        oct[i] = r.oct;
    }
    mra_tree* g = new mra_tree();
    g->magic = MRA_TREE_MAGIC;
    g->k = k;
    g->A = t->A;
    g->A.stream = st;
    g->state = t->state;
    g->depth_hit = t->depth_hit;
    struct TreeGuard {
        mra_tree* t;
        ~TreeGuard() {
            if (t) mra_free_tree(t);
        }
    } tg{g};
    MRA_TRY(tree_alloc_arrays(g, n2, true));
    MRA_TRY(tree_link_and_upload(g, c2.data(), l2.data()));
    Scratch tmp(g->A);
    int32_t *dsrc, *doct;
    MRA_TRY(tmp.get(&dsrc, n2));
    MRA_TRY(tmp.get(&doct, n2));
    MRA_CK(cudaMemcpyAsync(dsrc, src.data(), n2 * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    MRA_CK(cudaMemcpyAsync(doct, oct.data(), n2 * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    const size_t smem = (2 * (size_t)k * k + 2 * (size_t)k3) * sizeof(double);
    k_refine_blocks<<<std::max(1, std::min(n2, num_sms() * 8)), 128, smem, st>>>(k, n2, dsrc, doct, t->s, g->s,
                                                                                t->filt);
    MRA_CK_LAUNCH();
    // wavelet norms: old nodes keep theirs, split leaves have none (exact refinement)
    std::vector<double> dn(n), dn2(n2, 0.0);
    MRA_CK(cudaMemcpyAsync(dn.data(), t->dnorm, n * sizeof(double), cudaMemcpyDeviceToHost, st));
    MRA_CK(cudaStreamSynchronize(st));
    for (int i = 0; i < n2; ++i)
        if (oct[i] < 0 && !split[src[i]]) dn2[i] = dn[src[i]];
    MRA_CK(cudaMemcpyAsync(g->dnorm, dn2.data(), n2 * sizeof(double), cudaMemcpyHostToDevice, st));
    MRA_CK(cudaStreamSynchronize(st));  // host vectors go out of scope
    tg.t = nullptr;
    *out = g;
    return MRA_OK;
}

int refine_impl(const mra_tree* f, int passes, int max_level, cudaStream_t st, mra_tree** out, int* nsplit_total) {
    *out = nullptr;
    mra_tree* cur = nullptr;
    int total = 0;
    for (int p = 0; p < passes; ++p) {
        mra_tree* next = nullptr;
        int ns = 0;
        const int rc = refine_pass(cur ? cur : f, max_level, st, &next, &ns);
        if (cur) mra_free_tree(cur);
        if (rc != MRA_OK) return rc;
        cur = next;
        total += ns;
        if (ns == 0) break;
    }
    if (!cur) {  // no pass: a copy
        int ns = 0;
        MRA_TRY(refine_pass(f, -1, st, &cur, &ns));
    }
    if (nsplit_total) *nsplit_total = total;
    *out = cur;
    return MRA_OK;
}

}  // namespace mra
