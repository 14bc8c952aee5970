// The learned schedule's network: a 3 x 128 ReLU MLP with FP16 weights and
// activations, FP32 accumulation, FP32 master weights and Adam, trained and
// run by the kernels below.  The paper has no learned part; the network
// predicts, per output box, the term cut-offs of the exact per-pair screen
// (Sec. 4's term ranges narrowed per box), which the apply then checks.
//
// Parameter order (one FP32 vector): W1 [H][n_in], b1 [H], W2 [H][H], b2,
// W3 [H][H], b3, W4 [n_out][H], b4 [n_out], row-major.  Per layer l the
// FP16 copies hold W_l both row-major ([out][in], for the backward data pass)
// and transposed ([in][out], for the forward pass), so a thread per output
// unit reads a coalesced row either way.
//
// Loss per box (n_out = 12, per class S: [e_S, lo_S, hi_S], targets
// [E_S, LO_S, HI_S]):
//   sum_S softplus(e_S) - E_S e_S + (1 - E_S) ((lo_S - LO_S)^2 + (hi_S - HI_S)^2)
// averaged over the batch.
#include <cuda_fp16.h>
#include <math.h>

#include <algorithm>
#include <vector>

#include "mra_internal.cuh"

#define MLP_H 128
#define MLP_RB 32  // rows per block

struct mra_mlp {
    uint32_t magic = 0;
    int n_in = 0, n_out = 0;
    int64_t np = 0;                 // parameters
    int64_t off_w[4], off_b[4];     // offsets of W_l, b_l in the flat vector
    int din[4], dout[4];
    float* master = nullptr;        // FP32 parameters
    float* grad = nullptr;
    float* m = nullptr;             // Adam moments
    float* v = nullptr;
    __half* w16 = nullptr;          // per layer [out][in] then [in][out], at off_w * 2
    int step = 0;
    // activations of the last training batch (capacity rows)
    int64_t cap = 0;
    __half *h1 = nullptr, *h2 = nullptr, *h3 = nullptr;
    float *y = nullptr, *d3 = nullptr, *d2 = nullptr, *d1 = nullptr, *dy = nullptr;
    double* loss = nullptr;
    mra::Alloc A;
};

namespace mra {

// out[r][o] for a block of MLP_RB rows; in: float or half [n][din];
// Wio: half [din][dout] (element (i, o) at i * dout + o).
//   mode 0: relu(in W + b) -> half     (hidden layer, forward)
//   mode 1: in W + b       -> float    (output layer, forward)
//   mode 2: (in W) * [mask > 0] -> float  (backward data pass; mask half [n][dout])
template <class TI, int MODE>
__global__ void k_dense(int64_t n, int din, int dout, const TI* in, const __half* Wio, const float* b,
                        const __half* mask, void* out) {
    extern __shared__ float xs[];  // [MLP_RB][din]
    const int64_t r0 = (int64_t)blockIdx.x * MLP_RB;
    const int rows = (int)min((int64_t)MLP_RB, n - r0);
    for (int e = threadIdx.x; e < rows * din; e += blockDim.x)
        xs[e] = (float)in[r0 * din + e];
    __syncthreads();
    for (int o = threadIdx.x; o < dout; o += blockDim.x) {
        float acc[MLP_RB];
        const float bo = b ? b[o] : 0.0f;
#pragma unroll
        for (int r = 0; r < MLP_RB; ++r) acc[r] = bo;
        for (int i = 0; i < din; ++i) {
            const float w = __half2float(Wio[(size_t)i * dout + o]);
#pragma unroll
            for (int r = 0; r < MLP_RB; ++r) acc[r] += w * xs[r * din + i];
        }
#pragma unroll
        for (int r = 0; r < MLP_RB; ++r) {
            if (r >= rows) break;
            const size_t idx = (size_t)(r0 + r) * dout + o;
            if (MODE == 0) ((__half*)out)[idx] = __float2half_rn(fmaxf(acc[r], 0.0f));
            else if (MODE == 1) ((float*)out)[idx] = acc[r];
            else ((float*)out)[idx] = __half2float(mask[idx]) > 0.0f ? acc[r] : 0.0f;
        }
    }
}

// loss and dL/dy (divided by n); loss accumulated in FP64
__global__ void k_mlp_loss(int64_t n, const float* y, const float* t, float* dy, double* loss) {
    __shared__ double red[32];
    double acc = 0.0;
    const double inv = 1.0 / (double)n;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        for (int S = 0; S < 4; ++S) {
            const float e = y[r * 12 + 3 * S], lo = y[r * 12 + 3 * S + 1], hi = y[r * 12 + 3 * S + 2];
            const float E = t[r * 12 + 3 * S], LO = t[r * 12 + 3 * S + 1], HI = t[r * 12 + 3 * S + 2];
            const double sp = e > 0.0f ? (double)e + log1p(exp(-(double)e)) : log1p(exp((double)e));
            acc += sp - (double)E * e + (1.0 - E) * ((double)(lo - LO) * (lo - LO) + (double)(hi - HI) * (hi - HI));
            const double sg = 1.0 / (1.0 + exp(-(double)e));
            dy[r * 12 + 3 * S] = (float)((sg - E) * inv);
            dy[r * 12 + 3 * S + 1] = (float)(2.0 * (1.0 - E) * (lo - LO) * inv);
            dy[r * 12 + 3 * S + 2] = (float)(2.0 * (1.0 - E) * (hi - HI) * inv);
        }
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        atomicAdd(loss, s * inv);
    }
}

// gW[o][i] = sum_r d[r][o] h[r][i], gb[o] = sum_r d[r][o]; thread per (o, i)
// (i == din: the bias)
template <class TI>
__global__ void k_wgrad(int64_t n, int din, int dout, const float* d, const TI* h, float* gW, float* gb) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)dout * (din + 1)) return;
    const int o = (int)(e / (din + 1)), i = (int)(e % (din + 1));
    float acc = 0.0f;
    if (i < din) {
        for (int64_t r = 0; r < n; ++r) acc += d[r * dout + o] * (float)h[r * din + i];
        gW[(size_t)o * din + i] = acc;
    } else {
        for (int64_t r = 0; r < n; ++r) acc += d[r * dout + o];
        gb[o] = acc;
    }
}

__global__ void k_adam(int64_t np, float* p, const float* g, float* m, float* v, float lr, float c1, float c2) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < np; e += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[e];
        const float mi = 0.9f * m[e] + 0.1f * gi;
        const float vi = 0.999f * v[e] + 0.001f * gi * gi;
        m[e] = mi;
        v[e] = vi;
        p[e] -= lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
    }
}

// FP16 copies of the weight matrices: [out][in] at 2 off_w, [in][out] right after
struct W16Layout {
    int64_t off_w[4];
    int din[4], dout[4];
};

__global__ void k_refresh16(W16Layout L, const float* p, __half* w16) {
    for (int l = 0; l < 4; ++l) {
        const int64_t sz = (int64_t)L.din[l] * L.dout[l];
        __half* rm = w16 + 2 * L.off_w[l];
        __half* tr = rm + sz;
        for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < sz; e += (int64_t)gridDim.x * blockDim.x) {
            const int o = (int)(e / L.din[l]), i = (int)(e % L.din[l]);
            const __half h = __float2half_rn(p[L.off_w[l] + e]);
            rm[e] = h;
            tr[(size_t)i * L.dout[l] + o] = h;
        }
    }
}

static W16Layout w16_layout(const mra_mlp* M) {
    W16Layout L;
    for (int l = 0; l < 4; ++l) {
        L.off_w[l] = M->off_w[l];
        L.din[l] = M->din[l];
        L.dout[l] = M->dout[l];
    }
    return L;
}

static const __half* w_rowmajor(const mra_mlp* M, int l) { return M->w16 + 2 * M->off_w[l]; }
static const __half* w_trans(const mra_mlp* M, int l) {
    return M->w16 + 2 * M->off_w[l] + (int64_t)M->din[l] * M->dout[l];
}

static int refresh16(const mra_mlp* M, cudaStream_t st) {
    k_refresh16<<<num_sms(), 256, 0, st>>>(w16_layout(M), M->master, M->w16);
    MRA_CK_LAUNCH();
    return MRA_OK;
}

static int ensure_cap(mra_mlp* M, int64_t n) {
    if (n <= M->cap) return MRA_OK;
    const Alloc& A = M->A;
    A.put(M->h1); A.put(M->h2); A.put(M->h3); A.put(M->y); A.put(M->d3); A.put(M->d2); A.put(M->d1); A.put(M->dy);
    // a failure below leaves no stale buffer behind (capacity 0, the rest NULL)
    M->h1 = M->h2 = M->h3 = nullptr;
    M->y = M->d3 = M->d2 = M->d1 = M->dy = nullptr;
    M->cap = 0;
    int64_t c = std::max<int64_t>(n, 4096);
    MRA_TRY(dalloc(A, &M->h1, c * MLP_H));
    MRA_TRY(dalloc(A, &M->h2, c * MLP_H));
    MRA_TRY(dalloc(A, &M->h3, c * MLP_H));
    MRA_TRY(dalloc(A, &M->y, c * M->n_out));
    MRA_TRY(dalloc(A, &M->dy, c * M->n_out));
    MRA_TRY(dalloc(A, &M->d3, c * MLP_H));
    MRA_TRY(dalloc(A, &M->d2, c * MLP_H));
    MRA_TRY(dalloc(A, &M->d1, c * MLP_H));
    M->cap = c;
    return MRA_OK;
}

template <class TI, int MODE>
static int dense(int64_t n, int din, int dout, const TI* in, const __half* Wio, const float* b, const __half* mask,
                 void* out, cudaStream_t st) {
    if (n <= 0) return MRA_OK;
    const int64_t blocks = (n + MLP_RB - 1) / MLP_RB;
    k_dense<TI, MODE><<<(unsigned)blocks, 128, (size_t)MLP_RB * din * sizeof(float), st>>>(n, din, dout, in, Wio, b,
                                                                                          mask, out);
    MRA_CK_LAUNCH();
    return MRA_OK;
}

// forward with the activations kept (h1, h2, h3 in M's buffers), output y
int mlp_forward_impl(const mra_mlp* M, const float* x, int64_t n, float* y, __half* h1, __half* h2, __half* h3,
                     cudaStream_t st) {
    const float* p = M->master;
    MRA_TRY((dense<float, 0>(n, M->n_in, MLP_H, x, w_trans(M, 0), p + M->off_b[0], nullptr, h1, st)));
    MRA_TRY((dense<__half, 0>(n, MLP_H, MLP_H, h1, w_trans(M, 1), p + M->off_b[1], nullptr, h2, st)));
    MRA_TRY((dense<__half, 0>(n, MLP_H, MLP_H, h2, w_trans(M, 2), p + M->off_b[2], nullptr, h3, st)));
    MRA_TRY((dense<__half, 1>(n, MLP_H, M->n_out, h3, w_trans(M, 3), p + M->off_b[3], nullptr, y, st)));
    return MRA_OK;
}

template <class TI>
static int wgrad(int64_t n, int din, int dout, const float* d, const TI* h, float* gW, float* gb, cudaStream_t st) {
    const int64_t tot = (int64_t)dout * (din + 1);
    k_wgrad<TI><<<(unsigned)((tot + 127) / 128), 128, 0, st>>>(n, din, dout, d, h, gW, gb);
    MRA_CK_LAUNCH();
    return MRA_OK;
}

// forward, loss and gradients of the batch into M->grad (loss into M->loss)
static int mlp_loss_grad_impl(mra_mlp* M, const float* x, const float* t, int64_t n, cudaStream_t st) {
    MRA_TRY(ensure_cap(M, n));
    MRA_TRY(mlp_forward_impl(M, x, n, M->y, M->h1, M->h2, M->h3, st));
    MRA_CK(cudaMemsetAsync(M->loss, 0, sizeof(double), st));
    k_mlp_loss<<<(unsigned)std::min<int64_t>(1024, (n + 255) / 256), 256, 0, st>>>(n, M->y, t, M->dy, M->loss);
    MRA_CK_LAUNCH();
    float* g = M->grad;
    // layer 4 (linear), then back through the ReLU layers
    MRA_TRY(wgrad<__half>(n, MLP_H, M->n_out, M->dy, M->h3, g + M->off_w[3], g + M->off_b[3], st));
    MRA_TRY((dense<float, 2>(n, M->n_out, MLP_H, M->dy, w_rowmajor(M, 3), nullptr, M->h3, M->d3, st)));
    MRA_TRY(wgrad<__half>(n, MLP_H, MLP_H, M->d3, M->h2, g + M->off_w[2], g + M->off_b[2], st));
    MRA_TRY((dense<float, 2>(n, MLP_H, MLP_H, M->d3, w_rowmajor(M, 2), nullptr, M->h2, M->d2, st)));
    MRA_TRY(wgrad<__half>(n, MLP_H, MLP_H, M->d2, M->h1, g + M->off_w[1], g + M->off_b[1], st));
    MRA_TRY((dense<float, 2>(n, MLP_H, MLP_H, M->d2, w_rowmajor(M, 1), nullptr, M->h1, M->d1, st)));
    MRA_TRY(wgrad<float>(n, M->n_in, MLP_H, M->d1, x, g + M->off_w[0], g + M->off_b[0], st));
    return MRA_OK;
}

}  // namespace mra

using namespace mra;

static bool mlp_ok(const mra_mlp* M) { return M && M->magic == MRA_MLP_MAGIC; }

namespace mra {
const mra_mlp* mlp_checked(const void* h) {
    const mra_mlp* M = (const mra_mlp*)h;
    return mlp_ok(M) ? M : nullptr;
}
int mlp_forward(const mra_mlp* M, const float* x, int64_t n, float* y, const Alloc& A, cudaStream_t st) {
    Scratch tmp(A);
    __half *h1, *h2, *h3;
    MRA_TRY(tmp.get(&h1, (size_t)std::max<int64_t>(n, 1) * MLP_H));
    MRA_TRY(tmp.get(&h2, (size_t)std::max<int64_t>(n, 1) * MLP_H));
    MRA_TRY(tmp.get(&h3, (size_t)std::max<int64_t>(n, 1) * MLP_H));
    return mlp_forward_impl(M, x, n, y, h1, h2, h3, st);
}
int mlp_n_in(const mra_mlp* M) { return M->n_in; }
int mlp_n_out(const mra_mlp* M) { return M->n_out; }
}  // namespace mra

// splitmix64: seeded parameter initialisation on the host
static uint64_t splitmix(uint64_t& s) {
    uint64_t z = (s += 0x9e3779b97f4a7c15ull);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

extern "C" {

int mra_mlp_create(int n_in, int n_out, const float* params_host, unsigned long long seed, const mra_alloc* alloc,
                   void* stream, mra_mlp** out) {
    if (!out) { set_error("out is NULL"); return MRA_EINVAL; }
    *out = nullptr;
    if (n_in < 1 || n_in > 1024 || n_out < 1 || n_out > 1024) { set_error("n_in, n_out must lie in [1, 1024]"); return MRA_EINVAL; }
    cudaStream_t st = (cudaStream_t)stream;
    mra_mlp* M = new mra_mlp();
    M->magic = MRA_MLP_MAGIC;
    M->n_in = n_in;
    M->n_out = n_out;
    M->A = make_alloc(alloc, stream);
    const int din[4] = {n_in, MLP_H, MLP_H, MLP_H}, dout[4] = {MLP_H, MLP_H, MLP_H, n_out};
    int64_t o = 0;
    for (int l = 0; l < 4; ++l) {
        M->din[l] = din[l];
        M->dout[l] = dout[l];
        M->off_w[l] = o;
        o += (int64_t)din[l] * dout[l];
        M->off_b[l] = o;
        o += dout[l];
    }
    M->np = o;
    std::vector<float> h(o, 0.0f);
    if (params_host) {
        memcpy(h.data(), params_host, o * sizeof(float));
    } else {
        // He-uniform weights, zero biases
        uint64_t s = seed;
        for (int l = 0; l < 4; ++l) {
            const double a = sqrt(6.0 / din[l]);
            for (int64_t e = 0; e < (int64_t)din[l] * dout[l]; ++e) {
                const double u = (double)(splitmix(s) >> 11) * (1.0 / 9007199254740992.0);
                h[M->off_w[l] + e] = (float)((2.0 * u - 1.0) * a);
            }
        }
    }
    int rc = MRA_OK;
    const Alloc& A = M->A;
    if (rc == MRA_OK) rc = dalloc(A, &M->master, o);
    if (rc == MRA_OK) rc = dalloc(A, &M->grad, o);
    if (rc == MRA_OK) rc = dalloc(A, &M->m, o);
    if (rc == MRA_OK) rc = dalloc(A, &M->v, o);
    if (rc == MRA_OK) rc = dalloc(A, &M->w16, 2 * o);
    if (rc == MRA_OK) rc = dalloc(A, &M->loss, 1);
    if (rc == MRA_OK) {
        cudaError_t e = cudaMemcpyAsync(M->master, h.data(), o * sizeof(float), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(M->m, 0, o * sizeof(float), st);
        if (e == cudaSuccess) e = cudaMemsetAsync(M->v, 0, o * sizeof(float), st);
        if (e == cudaSuccess) e = cudaMemsetAsync(M->w16, 0, 2 * o * sizeof(__half), st);
        if (e != cudaSuccess) { set_error("mlp upload: %s", cudaGetErrorString(e)); rc = MRA_ECUDA; }
    }
    if (rc == MRA_OK) rc = refresh16(M, st);
    if (rc == MRA_OK) {
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) { set_error("mlp create: %s", cudaGetErrorString(e)); rc = MRA_ECUDA; }
    }
    if (rc != MRA_OK) {
        mra_mlp_free(M);
        return rc;
    }
    *out = M;
    return MRA_OK;
}

int mra_mlp_num_params(const mra_mlp* M, int64_t* n) {
    if (!mlp_ok(M) || !n) { set_error("invalid network handle"); return MRA_EINVAL; }
    *n = M->np;
    return MRA_OK;
}

int mra_mlp_get_params(const mra_mlp* M, float* params_host, void* stream) {
    if (!mlp_ok(M) || !params_host) { set_error("invalid network handle"); return MRA_EINVAL; }
    MRA_CK(cudaMemcpyAsync(params_host, M->master, M->np * sizeof(float), cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    MRA_CK(cudaStreamSynchronize((cudaStream_t)stream));
    return MRA_OK;
}

int mra_mlp_set_params(mra_mlp* M, const float* params_host, void* stream) {
    if (!mlp_ok(M) || !params_host) { set_error("invalid network handle"); return MRA_EINVAL; }
    cudaStream_t st = (cudaStream_t)stream;
    MRA_CK(cudaMemcpyAsync(M->master, params_host, M->np * sizeof(float), cudaMemcpyHostToDevice, st));
    MRA_CK(cudaMemsetAsync(M->m, 0, M->np * sizeof(float), st));
    MRA_CK(cudaMemsetAsync(M->v, 0, M->np * sizeof(float), st));
    M->step = 0;
    MRA_TRY(refresh16(M, st));
    MRA_CK(cudaStreamSynchronize(st));
    return MRA_OK;
}

int mra_mlp_forward(const mra_mlp* M, const float* x, int64_t n, float* y, void* stream) {
    if (!mlp_ok(M) || (!x && n > 0) || (!y && n > 0) || n < 0) { set_error("invalid network forward arguments"); return MRA_EINVAL; }
    return mlp_forward(M, x, n, y, M->A, (cudaStream_t)stream);
}

int mra_mlp_loss_grad(mra_mlp* M, const float* x, const float* target, int64_t n, float* grad_host, double* loss_host,
                      void* stream) {
    if (!mlp_ok(M) || !x || !target || n < 1) { set_error("invalid network arguments"); return MRA_EINVAL; }
    if (M->n_out != 12) { set_error("the schedule loss needs 12 outputs"); return MRA_EINVAL; }
    cudaStream_t st = (cudaStream_t)stream;
    MRA_TRY(mlp_loss_grad_impl(M, x, target, n, st));
    if (grad_host) MRA_CK(cudaMemcpyAsync(grad_host, M->grad, M->np * sizeof(float), cudaMemcpyDeviceToHost, st));
    if (loss_host) MRA_CK(cudaMemcpyAsync(loss_host, M->loss, sizeof(double), cudaMemcpyDeviceToHost, st));
    MRA_CK(cudaStreamSynchronize(st));
    return MRA_OK;
}

int mra_mlp_train_step(mra_mlp* M, const float* x, const float* target, int64_t n, float lr, void* stream,
                       double* loss_host) {
    if (!mlp_ok(M) || !x || !target || n < 1 || !(lr > 0.0f)) { set_error("invalid training arguments"); return MRA_EINVAL; }
    if (M->n_out != 12) { set_error("the schedule loss needs 12 outputs"); return MRA_EINVAL; }
    cudaStream_t st = (cudaStream_t)stream;
    MRA_TRY(mlp_loss_grad_impl(M, x, target, n, st));
    M->step++;
    const float c1 = (float)(1.0 - pow(0.9, M->step)), c2 = (float)(1.0 - pow(0.999, M->step));
    k_adam<<<num_sms(), 256, 0, st>>>(M->np, M->master, M->grad, M->m, M->v, lr, c1, c2);
    MRA_CK_LAUNCH();
    MRA_TRY(refresh16(M, st));
    if (loss_host) {
        MRA_CK(cudaMemcpyAsync(loss_host, M->loss, sizeof(double), cudaMemcpyDeviceToHost, st));
        MRA_CK(cudaStreamSynchronize(st));
    }
    return MRA_OK;
}

int mra_mlp_free(mra_mlp* M) {
    if (!M) return MRA_OK;
    if (!mlp_ok(M)) { set_error("invalid network handle"); return MRA_EINVAL; }
    const Alloc& A = M->A;
    A.put(M->master); A.put(M->grad); A.put(M->m); A.put(M->v); A.put(M->w16); A.put(M->loss);
    A.put(M->h1); A.put(M->h2); A.put(M->h3); A.put(M->y); A.put(M->d3); A.put(M->d2); A.put(M->d1); A.put(M->dy);
    M->magic = 0;
    delete M;
    return MRA_OK;
}

}  // extern "C"
