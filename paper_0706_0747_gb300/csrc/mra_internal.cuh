// Internal declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <vector>

#include "../../include/mra_gb300.h"

// every handle starts with one of these 32-bit tags (mra_free dispatches on it)
#define MRA_TREE_MAGIC 0x54524545u  // "TREE"
#define MRA_OP_MAGIC 0x4f504552u    // "OPER"
#define MRA_PLAN_MAGIC 0x504c414eu  // "PLAN"
#define MRA_MLP_MAGIC 0x4d4c5030u   // "MLP0"
#define MRA_TREE2_MAGIC 0x54524532u // "TRE2"

namespace mra {

// ---------------------------------------------------------------- errors
void set_error(const char* fmt, ...);

#define MRA_CK(call)                                                              \
    do {                                                                          \
        cudaError_t e_ = (call);                                                  \
        if (e_ != cudaSuccess) {                                                  \
            ::mra::set_error("%s:%d %s: %s", __FILE__, __LINE__, #call,           \
                             cudaGetErrorString(e_));                             \
            return MRA_ECUDA;                                                     \
        }                                                                         \
    } while (0)

// streaming multiprocessors of the current device (queried once per device;
// grids of persistent and grid-stride kernels are sized in multiples of it)
int num_sms();

// every kernel launch is followed by MRA_CK_LAUNCH(), which also counts it
void count_launch();
#define MRA_CK_LAUNCH()            \
    do {                           \
        ::mra::count_launch();     \
        MRA_CK(cudaGetLastError()); \
    } while (0)

#define MRA_TRY(expr)                \
    do {                             \
        int rc_ = (expr);            \
        if (rc_ != MRA_OK) return rc_; \
    } while (0)

// ---------------------------------------------------------------- memory
struct Alloc {
    mra_alloc hook;
    bool has = false;
    cudaStream_t stream = nullptr;
    void* get(size_t bytes) const;
    void put(void* p) const;
};
Alloc make_alloc(const mra_alloc* a, void* stream);

template <class T>
inline int dalloc(const Alloc& A, T** p, size_t count) {
    *p = (T*)A.get(count * sizeof(T) + 16);
    if (!*p) {
        set_error("device allocation of %zu bytes failed", count * sizeof(T));
        return MRA_ENOMEM;
    }
    return MRA_OK;
}

// Temporary device memory of one call: every block taken through it is
// released (stream-ordered) when the Scratch goes out of scope, on success
// and on every error return.
struct Scratch {
    const Alloc& A;
    std::vector<void*> p;
    explicit Scratch(const Alloc& a) : A(a) {}
    Scratch(const Scratch&) = delete;
    Scratch& operator=(const Scratch&) = delete;
    template <class T>
    int get(T** out, size_t count) {
        const int rc = dalloc(A, out, count);
        if (rc == MRA_OK) p.push_back((void*)*out);
        return rc;
    }
    ~Scratch() {
        for (size_t i = p.size(); i-- > 0;) A.put(p[i]);
    }
};

// ---------------------------------------------------------------- handles
struct TreeArrays {
    uint64_t* key = nullptr;    // Morton key of the box at its level
    int32_t* coord = nullptr;   // (j, a1, a2, a3) per node
    int32_t* leaf = nullptr;    // 1 = leaf
    int32_t* child = nullptr;   // index of first child (octants contiguous) or -1
    int32_t* parent = nullptr;  // -1 for the root
    int32_t* off = nullptr;     // level offsets (device copy), MRA_MAX_LEVEL + 2
};

}  // namespace mra

struct mra_tree {
    uint32_t magic;
    int k, n, nlev, state, depth_hit;
    int off[MRA_MAX_LEVEL + 2];
    mra::TreeArrays a;
    double* s = nullptr;      // n * k^3 blocks
    double* dnorm = nullptr;  // n
    void* slab = nullptr;     // one allocation holding a's arrays, s and dnorm
    double* dcube = nullptr;  // n * (2k)^3 wavelet cubes (optional)
    double* filt = nullptr;   // H0, H1 (2 k^2) then W (4 k^2), row-major
    mra::Alloc A;
};

// A tree of the d = 2 variant: nodes sorted by (level, 2-D Morton key), the 4
// children of an internal node contiguous in quadrant order, blocks k x k.
struct mra_tree2 {
    uint32_t magic;
    int k, n, nlev, state, depth_hit;
    int off[MRA_MAX_LEVEL + 2];
    uint64_t* key = nullptr;
    int32_t* coord = nullptr;   // (j, a1, a2) per node
    int32_t* leaf = nullptr;
    int32_t* child = nullptr;   // first of the 4 children, or -1
    int32_t* parent = nullptr;  // -1 for the root
    double* s = nullptr;        // n * k^2
    double* dnorm = nullptr;    // n
    double* filt = nullptr;     // H0, H1, W
    mra::Alloc A;
};

struct mra_op {
    uint32_t magic;
    int k, J, M;  // J = max_level
    int d = 3;    // dimension of the kernel: 3, or 2 for the two-dimensional variant
    double mu, alpha, eps;
    double* w = nullptr;      // M
    double* tau = nullptr;    // M
    double* F = nullptr;      // (J+1) M 7 k k
    float* F32 = nullptr;     // same, FP32
    double* nF = nullptr;     // (J+1) M 7
    double* est = nullptr;    // (J+1) M
    double* filt = nullptr;   // H0, H1, W
    int* scratch_i = nullptr; // device ints (status, M)
    // per-pair screen tables (built on first use by a pair or learned screen):
    // sparse-table range maxima over m of w_m N_F(t1) N_F(t2) N_F(t3) per (j, t)
    double* rmq = nullptr;
    int rmq_L = 0;
    double gs_A = 0.0, gs_h = 0.0;  // the term grid: s_m = gs_A + (m + 1) gs_h
    mra::Alloc A;
};

namespace mra {

// ---------------------------------------------------------------- launchers
// operator.cu
int launch_filters(int k, double* filt, cudaStream_t st);
int build_operator(mra_op* op, cudaStream_t st);
int retune_operator(mra_op* op, double mu, cudaStream_t st);

// tree.cu
int tree_alloc_arrays(mra_tree* t, int n, bool with_s);
void tree_free_arrays(mra_tree* t);
int tree_link_and_upload(mra_tree* t, const int32_t* coords_host, const int32_t* leaf_host);
int build_tree_impl(const mra_density* f, int k, double eps, int max_level, int uniform_level,
                    int init_level, const Alloc& A, mra_tree** out);
int compress_impl(mra_tree* t, int mode, cudaStream_t st);  // mode: MRA_COMPRESS_*
int scan_exclusive(const int32_t* in, int32_t* out, int n, int32_t* total, cudaStream_t st);
int inverse_impl(mra_tree* t, cudaStream_t st);
int assemble_impl(mra_tree* t, cudaStream_t st);
int truncate_impl(mra_tree* t, double eps, cudaStream_t st, double* removed_host);
int tree_clone_skeleton(const mra_tree* src, mra_tree** out);
int refine_impl(const mra_tree* f, int passes, int max_level, cudaStream_t st, mra_tree** out, int* nsplit_total);
// product.cu
int tree_multiply_impl(const mra_tree* f, const mra_potential* v, double scale, cudaStream_t st, mra_tree** out);
int tree_dot_impl(const mra_tree* a, const mra_tree* b, double* out_host, cudaStream_t st);
// <a[p], b[p]> for p = 0, 1, 2 in one pass; all six trees share a's skeleton (not checked)
int tree_dot3_impl(const mra_tree* const* a, const mra_tree* const* b, double* out_host, cudaStream_t st);
int tree_scale_impl(mra_tree* t, double alpha, cudaStream_t st);

// apply.cu
int apply_impl(const mra_op* op, const mra_tree* f, const mra_apply_opts* o, cudaStream_t st,
               mra_tree** g, mra_apply_stats* stats);
int apply_noalloc_impl(const mra_op* op, const mra_tree* f, int precision, double* ghat, cudaStream_t st,
                       int64_t* n_items_host);

// schedule.cu
int screen_data_impl(const mra_op* op, const mra_tree* f, float* X, float* T, cudaStream_t st);

// ---------------------------------------------------------------- device helpers
__host__ __device__ inline uint64_t spread3(uint32_t v) {
    uint64_t x = v & 0x1fffffu;
    x = (x | (x << 32)) & 0x1f00000000ffffull;
    x = (x | (x << 16)) & 0x1f0000ff0000ffull;
    x = (x | (x << 8)) & 0x100f00f00f00f00full;
    x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
    x = (x | (x << 2)) & 0x1249249249249249ull;
    return x;
}
// key bit 3b+2 <- a1 bit b, 3b+1 <- a2 bit b, 3b <- a3 bit b: child octant
// (p1 p2 p3) appends three bits, so a level's keys sort children contiguously.
__host__ __device__ inline uint64_t morton3(uint32_t a1, uint32_t a2, uint32_t a3) {
    return (spread3(a1) << 2) | (spread3(a2) << 1) | spread3(a3);
}

// index of key k in the sorted range [lo, hi), or -1 if absent
__device__ inline int find_key_exact(const uint64_t* keys, int lo, int hi, uint64_t k) {
    int l = lo, h = hi;
    while (l < h) {
        int mid = (l + h) >> 1;
        if (keys[mid] < k) l = mid + 1;
        else h = mid;
    }
    return (l < hi && keys[l] == k) ? l : -1;
}

// phi_i(u) = sqrt(2i+1) P_i(2u-1), i < n, written to out[0..n)
__host__ __device__ inline void phi_all(int n, double u, double* out) {
    double v = 2.0 * u - 1.0;
    double p0 = 1.0, p1 = v;
    for (int i = 0; i < n; ++i) {
        double p;
        if (i == 0) p = 1.0;
        else if (i == 1) p = v;
        else {
            p = ((2.0 * i - 1.0) * v * p1 - (i - 1.0) * p0) / i;
            p0 = p1;
            p1 = p;
        }
        out[i] = sqrt(2.0 * i + 1.0) * p;
    }
}

// Root i of the n-point Gauss-Legendre rule on [0, 1] (n <= 32) by Newton on
// P_n from the asymptotic start cos(pi (i + 3/4) / (n + 1/2)): stops once the
// step is below 1e-15 (quadratic convergence leaves the root at rounding
// level), then refreshes the derivative for the weight.  Node index
// n - 1 - i (nodes increase with the index).
__host__ __device__ inline void gauss_legendre01_root(int n, int i, double* x, double* w) {
    double z = cos(3.14159265358979323846 * (i + 0.75) / (n + 0.5));
    double pn = 0.0, pm = 0.0;
    for (int it = 0; it < 100; ++it) {
        double p0 = 1.0, p1 = z;
        for (int q = 2; q <= n; ++q) {
            double p2 = ((2.0 * q - 1.0) * z * p1 - (q - 1.0) * p0) / q;
            p0 = p1;
            p1 = p2;
        }
        pn = (n == 1) ? z : p1;
        pm = (n == 1) ? 1.0 : p0;
        const double dz = pn / (n * (z * pn - pm) / (z * z - 1.0));
        z -= dz;
        if (fabs(dz) < 1e-15) break;
    }
    double p0 = 1.0, p1 = z;
    for (int q = 2; q <= n; ++q) {
        double p2 = ((2.0 * q - 1.0) * z * p1 - (q - 1.0) * p0) / q;
        p0 = p1;
        p1 = p2;
    }
    pn = (n == 1) ? z : p1;
    pm = (n == 1) ? 1.0 : p0;
    const double dp = n * (z * pn - pm) / (z * z - 1.0);
    const int idx = n - 1 - i;  // cos(.) decreases with i
    x[idx] = 0.5 * (z + 1.0);
    w[idx] = 1.0 / ((1.0 - z * z) * dp * dp);
}

// all n nodes and weights, by one thread
__host__ __device__ inline void gauss_legendre01(int n, double* x, double* w) {
    for (int i = 0; i < n; ++i) gauss_legendre01_root(n, i, x, w);
}

// parity band of the modified ns-form: t_d in [-3, 2] (even a_d) or [-2, 3] (odd)
__host__ __device__ inline int band_t(int a_d, int q) { return (a_d & 1) ? q - 2 : q - 3; }

}  // namespace mra
