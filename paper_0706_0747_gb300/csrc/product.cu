// Products, inner products and scaling of trees: the pointwise work of the
// hydrogen ground-state iteration phi = -2 G_mu V phi (Sec. 6.2, Steps 2 and 4).
#include <algorithm>

#include "mra_internal.cuh"

namespace mra {

struct PotDev {
    int ng, nc;
    const double *coef, *r2coef, *expo, *center;  // Gaussian terms
    const double *charge, *pos;                   // point charges
};

__device__ double pot_eval(const PotDev& V, double x1, double x2, double x3) {
    double v = 0.0;
    for (int g = 0; g < V.ng; ++g) {
        const double d1 = x1 - V.center[3 * g], d2 = x2 - V.center[3 * g + 1], d3 = x3 - V.center[3 * g + 2];
        const double r2 = d1 * d1 + d2 * d2 + d3 * d3;
        v += (V.coef[g] + V.r2coef[g] * r2) * exp(-V.expo[g] * r2);
    }
    for (int c = 0; c < V.nc; ++c) {
        const double d1 = x1 - V.pos[3 * c], d2 = x2 - V.pos[3 * c + 1], d3 = x3 - V.pos[3 * c + 2];
        const double r2 = d1 * d1 + d2 * d2 + d3 * d3;
        if (r2 > 0.0) v += V.charge[c] / sqrt(r2);
    }
    return v;
}

// One block per leaf (grid-stride over nodes).  In shared memory: the GL
// nodes and weights of [0, 1], Phi[q][i] = phi_i(u_q), and two k^3 buffers
// used in turn.  Coefficients -> values at the box's GL points are three mode
// products with Phi (the 2^{3j/2} of the values and the 2^{-3j/2} of the
// projection cancel); the values are multiplied by w_q1 w_q2 w_q3 V(x_q) scale;
// three mode products with Phi^T give the projected coefficients.  KT > 0
// fixes k at compile time (the inner loops unroll); KT = 0 takes k at run time.
template <int KT>
__global__ void k_tree_multiply(int k_rt, int n, const int32_t* coord, const int32_t* leaf, const double* s,
                                PotDev V, double scale, double* out) {
    extern __shared__ double sm[];
    const int k = KT > 0 ? KT : k_rt;
    const int k3 = k * k * k, kk = k * k;
    double* xq = sm;
    double* wq = xq + MRA_MAX_K;
    double* Phi = wq + MRA_MAX_K;
    double* a = Phi + MRA_MAX_K * MRA_MAX_K;
    double* b = a + k3;
    if (threadIdx.x < k) gauss_legendre01_root(k, threadIdx.x, xq, wq);
    __syncthreads();
    if (threadIdx.x < k) {
        double ph[MRA_MAX_K];
        phi_all(k, xq[threadIdx.x], ph);
        for (int i = 0; i < k; ++i) Phi[threadIdx.x * k + i] = ph[i];
    }
    __syncthreads();
    for (int node = blockIdx.x; node < n; node += gridDim.x) {
        double* dst = out + (size_t)node * k3;
        if (!leaf[node]) {
            for (int e = threadIdx.x; e < k3; e += blockDim.x) dst[e] = 0.0;
            continue;
        }
        const int j = coord[4 * node];
        const double h = ldexp(1.0, -j);
        const double o1 = coord[4 * node + 1] * h, o2 = coord[4 * node + 2] * h, o3 = coord[4 * node + 3] * h;
        double* x = a;
        double* y = b;
        for (int e = threadIdx.x; e < k3; e += blockDim.x) x[e] = s[(size_t)node * k3 + e];
        __syncthreads();
        // direction d has stride kk, k, 1 for d = 0, 1, 2 (block index i1 i2 i3, C order)
        for (int d = 0; d < 3; ++d) {
            const int st = d == 0 ? kk : (d == 1 ? k : 1);
            for (int e = threadIdx.x; e < k3; e += blockDim.x) {
                const int q = (e / st) % k;
                const double* col = x + e - q * st;
                double acc = 0.0;
#pragma unroll
                for (int i = 0; i < (KT > 0 ? KT : MRA_MAX_K); ++i)
                    if (KT > 0 || i < k) acc += Phi[q * k + i] * col[i * st];
                y[e] = acc;
            }
            __syncthreads();
            double* t = x;
            x = y;
            y = t;
        }
        for (int e = threadIdx.x; e < k3; e += blockDim.x) {
            const int q1 = e / kk, q2 = (e / k) % k, q3 = e % k;
            const double v = pot_eval(V, o1 + h * xq[q1], o2 + h * xq[q2], o3 + h * xq[q3]);
            x[e] *= wq[q1] * wq[q2] * wq[q3] * v * scale;
        }
        __syncthreads();
        for (int d = 0; d < 3; ++d) {
            const int st = d == 0 ? kk : (d == 1 ? k : 1);
            for (int e = threadIdx.x; e < k3; e += blockDim.x) {
                const int i = (e / st) % k;
                const double* col = x + e - i * st;
                double acc = 0.0;
#pragma unroll
                for (int q = 0; q < (KT > 0 ? KT : MRA_MAX_K); ++q)
                    if (KT > 0 || q < k) acc += Phi[q * k + i] * col[q * st];
                y[e] = acc;
            }
            __syncthreads();
            double* t = x;
            x = y;
            y = t;
        }
        for (int e = threadIdx.x; e < k3; e += blockDim.x) dst[e] = x[e];
        __syncthreads();
    }
}

// sum over the leaves of <sa_i, sb_i>; a warp per node, partial sums added to
// *out with FP64 atomics (order not fixed)
__global__ void k_tree_dot(int n, int k3, const int32_t* leaf, const double* sa, const double* sb, double* out) {
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nwarps = (gridDim.x * blockDim.x) >> 5;
    double acc = 0.0;
    for (int i = warp; i < n; i += nwarps) {
        if (!leaf[i]) continue;
        for (int e = lane; e < k3; e += 32) acc += sa[(size_t)i * k3 + e] * sb[(size_t)i * k3 + e];
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0 && acc != 0.0) atomicAdd(out, acc);
}

// three inner products on one skeleton in one pass: out[p] = <sa[p], sb[p]>
struct Dot3 {
    const double* a[3];
    const double* b[3];
};
__global__ void k_tree_dot3(int n, int k3, const int32_t* leaf, Dot3 D, double* out) {
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nwarps = (gridDim.x * blockDim.x) >> 5;
    double acc[3] = {0.0, 0.0, 0.0};
    for (int i = warp; i < n; i += nwarps) {
        if (!leaf[i]) continue;
        for (int e = lane; e < k3; e += 32) {
            const size_t o = (size_t)i * k3 + e;
#pragma unroll
            for (int p = 0; p < 3; ++p) acc[p] += D.a[p][o] * D.b[p][o];
        }
    }
#pragma unroll
    for (int p = 0; p < 3; ++p) {
        double v = acc[p];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0 && v != 0.0) atomicAdd(out + p, v);
    }
}

// 1 in *diff when the two node lists or leaf flags differ anywhere
__global__ void k_same_skeleton(int n, const int32_t* ca, const int32_t* cb, const int32_t* la, const int32_t* lb,
                                int* diff) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const bool same = ca[4 * i] == cb[4 * i] && ca[4 * i + 1] == cb[4 * i + 1] && ca[4 * i + 2] == cb[4 * i + 2] &&
                          ca[4 * i + 3] == cb[4 * i + 3] && la[i] == lb[i];
        if (!same) *diff = 1;
    }
}

__global__ void k_scale(size_t total, double alpha, double* s) {
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x)
        s[e] *= alpha;
}

static int grid_for(size_t work, int per_block) {
    return (int)std::max<size_t>(1, std::min<size_t>((size_t)num_sms() * 8, (work + per_block - 1) / per_block));
}

int tree_multiply_impl(const mra_tree* f, const mra_potential* v, double scale, cudaStream_t st, mra_tree** out) {
    *out = nullptr;
    const int k = f->k, k3 = k * k * k, ng = v->n_gauss, nc = v->n_charge;
    mra_tree* g = nullptr;
    MRA_TRY(tree_clone_skeleton(f, &g));
    struct TreeGuard {
        mra_tree* t;
        ~TreeGuard() {
            if (t) mra_free_tree(t);
        }
    } tg{g};
    g->state = MRA_TREE_LEAVES;
    // potential parameters: [coef | r2coef | expo | centres (3) | charges | positions (3)]
    const size_t nv = 6 * (size_t)ng + 4 * (size_t)nc + 1;
    std::vector<double> hv(nv, 0.0);
    for (int i = 0; i < ng; ++i) {
        hv[i] = v->coef_host[i];
        hv[ng + i] = v->r2coef_host ? v->r2coef_host[i] : 0.0;
        hv[2 * ng + i] = v->expo_host[i];
        for (int d = 0; d < 3; ++d) hv[3 * ng + 3 * i + d] = v->center_host[3 * i + d];
    }
    for (int c = 0; c < nc; ++c) {
        hv[6 * ng + c] = v->charge_host[c];
        for (int d = 0; d < 3; ++d) hv[6 * ng + nc + 3 * c + d] = v->position_host[3 * c + d];
    }
    Scratch tmp(g->A);
    double* dv;
    MRA_TRY(tmp.get(&dv, nv));
    MRA_CK(cudaMemcpyAsync(dv, hv.data(), nv * sizeof(double), cudaMemcpyHostToDevice, st));
    PotDev P{ng, nc, dv, dv + ng, dv + 2 * ng, dv + 3 * ng, dv + 6 * ng, dv + 6 * ng + nc};
    const size_t smem = (2 * MRA_MAX_K + MRA_MAX_K * MRA_MAX_K + 2 * (size_t)k3) * sizeof(double);
    auto kern = k == 8 ? k_tree_multiply<8> : (k == 6 ? k_tree_multiply<6> : (k == 4 ? k_tree_multiply<4>
                                                                                     : k_tree_multiply<0>));
    MRA_CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<grid_for(f->n, 1), 128, smem, st>>>(k, f->n, f->a.coord, f->a.leaf, f->s, P, scale, g->s);
    MRA_CK_LAUNCH();
    MRA_CK(cudaMemsetAsync(g->dnorm, 0, f->n * sizeof(double), st));
    MRA_CK(cudaStreamSynchronize(st));  // hv goes out of scope
    tg.t = nullptr;
    *out = g;
    return MRA_OK;
}

int tree_dot_impl(const mra_tree* a, const mra_tree* b, double* out_host, cudaStream_t st) {
    const int k3 = a->k * a->k * a->k;
    Scratch tmp(a->A);
    double* acc;
    int* diff;
    MRA_TRY(tmp.get(&acc, 1));
    MRA_TRY(tmp.get(&diff, 1));
    MRA_CK(cudaMemsetAsync(acc, 0, sizeof(double), st));
    MRA_CK(cudaMemsetAsync(diff, 0, sizeof(int), st));
    k_same_skeleton<<<grid_for(a->n, 256), 256, 0, st>>>(a->n, a->a.coord, b->a.coord, a->a.leaf, b->a.leaf, diff);
    MRA_CK_LAUNCH();
    k_tree_dot<<<grid_for((size_t)a->n * 32, 256), 256, 0, st>>>(a->n, k3, a->a.leaf, a->s, b->s, acc);
    MRA_CK_LAUNCH();
    int hdiff = 0;
    MRA_CK(cudaMemcpyAsync(out_host, acc, sizeof(double), cudaMemcpyDeviceToHost, st));
    MRA_CK(cudaMemcpyAsync(&hdiff, diff, sizeof(int), cudaMemcpyDeviceToHost, st));
    MRA_CK(cudaStreamSynchronize(st));
    if (hdiff) {
        set_error("the two trees have different skeletons");
        return MRA_EINVAL;
    }
    return MRA_OK;
}

int tree_dot3_impl(const mra_tree* const* a, const mra_tree* const* b, double* out_host, cudaStream_t st) {
    const mra_tree* t = a[0];
    const int k3 = t->k * t->k * t->k;
    Scratch tmp(t->A);
    double* acc;
    MRA_TRY(tmp.get(&acc, 3));
    MRA_CK(cudaMemsetAsync(acc, 0, 3 * sizeof(double), st));
    Dot3 D;
    for (int p = 0; p < 3; ++p) {
        D.a[p] = a[p]->s;
        D.b[p] = b[p]->s;
    }
    k_tree_dot3<<<grid_for((size_t)t->n * 32, 256), 256, 0, st>>>(t->n, k3, t->a.leaf, D, acc);
    MRA_CK_LAUNCH();
    MRA_CK(cudaMemcpyAsync(out_host, acc, 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
    MRA_CK(cudaStreamSynchronize(st));
    return MRA_OK;
}

int tree_scale_impl(mra_tree* t, double alpha, cudaStream_t st) {
    const size_t total = (size_t)t->n * t->k * t->k * t->k;
    k_scale<<<grid_for(total, 256), 256, 0, st>>>(total, alpha, t->s);
    MRA_CK_LAUNCH();
    if (t->dcube) {
        k_scale<<<grid_for(8 * total, 256), 256, 0, st>>>(8 * total, alpha, t->dcube);
        MRA_CK_LAUNCH();
    }
    return MRA_OK;
}

}  // namespace mra
