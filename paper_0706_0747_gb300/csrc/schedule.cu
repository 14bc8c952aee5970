// Per-pair term cut-offs: the exact per-pair screen, the learned schedule's
// inputs and targets, and the learned cut-offs with the exact screen as the
// judge of every miss.
//
// Exact test of an item (a, t, m) (the norm bound of Sec. 4 with the input
// block's own norm): w_m N_F(j,m,t1) N_F(j,m,t2) N_F(j,m,t3) ||f_{a-t}|| >
// eta_blk, eta_blk = eps ||T_0 f_0|| / sqrt(N 216 M).  Per (output box,
// translation) pair the static schedule's term range (Sec. 4, per scale and
// Core/Boundary class) becomes:
//   exact screen    the first .. last term that passes (empty if none);
//   learned screen  the network's predicted range for the box and class,
//                   widened by a margin, clipped to the static range, and
//                   extended to every term that passes the exact test (a
//                   passing term outside the prediction is a miss: counted
//                   and restored).
// Every term of the static schedule inside the final range is applied.
#include <math.h>

#include <mutex>

#include "apply_common.cuh"

namespace mra {

const mra_mlp* mlp_checked(const void* h);
int mlp_forward(const mra_mlp* M, const float* x, int64_t n, float* y, const Alloc& A, cudaStream_t st);
int mlp_n_in(const mra_mlp* M);
int mlp_n_out(const mra_mlp* M);

#define EMPTY_LO 32767

// ||block||_2 in FP64 for the n node blocks then the Step-2 blocks; warp per block
__global__ void k_block_norms(int nb, int n, int k3, const double* s, const double* gblk, double* bn) {
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int b = warp; b < nb; b += nwarps) {
        const double* x = b < n ? s + (size_t)b * k3 : gblk + (size_t)(b - n) * k3;
        double acc = 0.0;
        for (int e = lane; e < k3; e += 32) acc += x[e] * x[e];
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) bn[b] = sqrt(acc);
    }
}

// eta_blk per tree from the pilot: eps sigma_b / sqrt(N_b 216 M)
__global__ void k_eta_blk(Forest F, const double* dv, double eps, int M, double* etab) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < F.ntrees; b += gridDim.x * blockDim.x) {
        const int nb = F.off[b * (F.lm + 1) + F.lm] - F.off[b * (F.lm + 1)];
        etab[b] = eps * dv[4 * b + 1] / sqrt((double)nb * 216.0 * M);
    }
}

__device__ inline int pair_class(const Pair& p) {
    return (abs((int)p.t1) <= 1) + (abs((int)p.t2) <= 1) + (abs((int)p.t3) <= 1);
}

__device__ inline float lg10s(double v) { return (float)(log10(fmax(v, 1e-300)) / 10.0); }

// 16 features per output box (thread per box; pairs in band order)
__global__ void k_sched_features(Forest F, const int32_t* pair_off, const Pair* pairs, const double* bn,
                                 const double* etab, int J, double mu, float* X) {
    for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < F.n; a += gridDim.x * blockDim.x) {
        const int tree = F.node_tree ? F.node_tree[a] : 0;
        const double eta = etab[tree];
        double mx[4] = {0, 0, 0, 0}, sm[4] = {0, 0, 0, 0};
        int cnt[4] = {0, 0, 0, 0};
        for (int p = pair_off[a]; p < pair_off[a + 1]; ++p) {
            const Pair pr = pairs[p];
            const int S = pair_class(pr);
            const double xn = bn[pr.in >= 0 ? pr.in : F.n + (-1 - pr.in)];
            mx[S] = fmax(mx[S], xn / eta);
            sm[S] += xn / eta;
            cnt[S]++;
        }
        float* x = X + (size_t)a * 16;
        x[0] = (float)((double)F.coord[4 * a] / J);
        x[1] = F.leaf[a] ? 1.0f : 0.0f;
        x[2] = lg10s(bn[a] / eta);
        for (int S = 0; S < 4; ++S) {
            x[3 + S] = cnt[S] ? lg10s(mx[S]) : 0.0f;
            x[7 + S] = cnt[S] ? lg10s(sm[S]) : 0.0f;
            x[11 + S] = (float)(cnt[S] / 64.0);
        }
        x[15] = (float)(mu / 2.0);
    }
}

// ---------------------------------------------------------------- range maxima
// The exact test of a pair's term m is P(m) ||x_b|| > eta_blk with the
// operator-only profile P(m) = ((w_m N_F(j,m,t1)) N_F(j,m,t2)) N_F(j,m,t3)
// (the same product, in the same order, as the per-term test, so every
// decision is bitwise the same).  Because x -> fl(x ||x_b||) is monotone,
// some term of an interval passes exactly when the interval's maximum of P
// does: a sparse table of range maxima per (j, t) answers that in O(1), and
// the first / last passing term of an interval by binary search.
#define RMQ_T 343  // translations t in [-3, 3]^3

__host__ __device__ inline int rmq_levels(int M) {
    int L = 1;
    while ((1 << L) <= M) ++L;
    return L;  // floor(log2 M) + 1
}

// block per (t, j): level 0 is P, level l the maximum of P over [m, m + 2^l)
__global__ void k_rmq_build(int M, int L, const double* w, const double* nF, double* rmq) {
    const int tc = blockIdx.x, j = blockIdx.y;
    const int t1 = tc / 49 - 3, t2 = (tc / 7) % 7 - 3, t3 = tc % 7 - 3;
    double* st = rmq + ((size_t)j * RMQ_T + tc) * L * M;
    for (int m = threadIdx.x; m < M; m += blockDim.x) {
        const double* r = nF + ((size_t)j * M + m) * 7;
        st[m] = w[m] * r[t1 + 3] * r[t2 + 3] * r[t3 + 3];
    }
    __syncthreads();
    for (int l = 1; l < L; ++l) {
        const int h = 1 << (l - 1);
        for (int m = threadIdx.x; m + 2 * h <= M; m += blockDim.x)
            st[(size_t)l * M + m] = fmax(st[(size_t)(l - 1) * M + m], st[(size_t)(l - 1) * M + m + h]);
        __syncthreads();
    }
}

// built once per operator, on the first call that needs them (thread-safe)
static int rmq_tables(const mra_op* op, cudaStream_t st, const double** out) {
    static std::mutex mu;
    std::lock_guard<std::mutex> lk(mu);
    if (!op->rmq) {
        mra_op* w = const_cast<mra_op*>(op);  // a cache: the operator's meaning is unchanged
        const int L = rmq_levels(op->M);
        double* t = nullptr;
        MRA_TRY(dalloc(op->A, &t, (size_t)(op->J + 1) * RMQ_T * L * op->M));
        k_rmq_build<<<dim3(RMQ_T, op->J + 1), 128, 0, st>>>(op->M, L, op->w, op->nF, t);
        const cudaError_t e = cudaGetLastError();
        count_launch();
        if (e != cudaSuccess) {
            op->A.put(t);
            set_error("range-maximum tables: %s", cudaGetErrorString(e));
            return MRA_ECUDA;
        }
        w->rmq = t;
        w->rmq_L = L;
    }
    *out = op->rmq;
    return MRA_OK;
}

struct Rmq {
    const double* st;  // this pair's (j, t) table
    int M;
    __device__ double max(int a, int b) const {  // a <= b
        const int l = 31 - __clz(b - a + 1);
        return fmax(st[(size_t)l * M + a], st[(size_t)l * M + b - (1 << l) + 1]);
    }
};

// A pair's candidate terms (those the static schedule keeps before the per-pair
// test) are the terms m of its class range [m1, m2] with J_m >= j, or, for a core
// translation at an internal node, J_m == j.  Per tree, level j and case ci the
// set {m : J_m >= j} (ci = 0) or {m : J_m == j} (ci = 1) is written as at most
// RUNS maximal runs of consecutive terms; a set with more runs is marked -1 and
// its pairs fall back to testing every term.
#define RUNS 4
#define RUN_REC (1 + 2 * RUNS)  // count | (first, last) x RUNS

__global__ void k_term_runs(int ntrees, int M, int lm, const int32_t* sched, int sl, int32_t* runs) {
    const int b = blockIdx.x;
    const int32_t* Jm = sched + (size_t)b * sl;
    for (int e = threadIdx.x; e < lm * 2; e += blockDim.x) {
        const int j = e >> 1, ci = e & 1;
        int32_t* r = runs + ((size_t)b * lm * 2 + e) * RUN_REC;
        int cnt = 0, start = -1;
        for (int m = 0; m <= M; ++m) {
            const bool in = m < M && (ci ? Jm[m] == j : Jm[m] >= j);
            if (in && start < 0) start = m;
            if (!in && start >= 0) {
                if (cnt < RUNS) {
                    r[1 + 2 * cnt] = start;
                    r[2 + 2 * cnt] = m - 1;
                }
                ++cnt;
                start = -1;
            }
        }
        r[0] = cnt <= RUNS ? cnt : -1;
    }
}

struct RangeArgs {
    Forest F;
    int M, sl, npairs, margin;
    Pair* pairs;
    const int32_t* sched;
    const double* w;
    const double* nF;
    const double* bn;
    const double* etab;
    const float* pred;            // [n][12] network outputs (NULL: exact screen)
    int32_t* tlo;                 // [n][4] first / last passing term per class (NULL: not kept)
    int32_t* thi;
    unsigned long long* counts;   // [0] misses (passing items outside the prediction), [1] empty pairs
    const double* rmq;            // range-maximum tables (rmq_L levels)
    int rmq_L;
    const int32_t* runs;          // [ntrees][lm][2] candidate-term runs (k_term_runs)
};

// thread per pair: narrow its term range in place
__global__ void k_pair_ranges(RangeArgs R) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= R.npairs) return;
    Pair p = R.pairs[i];
    const int a = p.out, tree = R.F.node_tree ? R.F.node_tree[a] : 0;
    const int j = R.F.coord[4 * a];
    const int32_t* Jm = R.sched + (size_t)tree * R.sl;
    const double xn = R.bn[p.in >= 0 ? p.in : R.F.n + (-1 - p.in)];
    const double eta = R.etab[tree];
    const int S = pair_class(p);
    const bool core_int = (p.flags & 1) != 0;
    // the prediction for this box and class
    int plo = 0, phi = -1;
    if (R.pred) {
        const float* y = R.pred + (size_t)a * 12 + 3 * S;
        if (!(y[0] > 0.0f)) {  // P(empty) < 1/2
            plo = (int)floorf(y[1] * (R.M - 1)) - R.margin;
            phi = (int)ceilf(y[2] * (R.M - 1)) + R.margin;
        }
        plo = max(plo, (int)p.m_lo);
        phi = min(phi, (int)p.m_hi);
    }
    auto candidate = [&](int m) {
        const int jm = Jm[m];
        return jm >= j && !(core_int && jm > j);
    };
    auto passes_m = [&](int m) {
        const size_t fb = ((size_t)j * R.M + m) * 7;
        return R.w[m] * R.nF[fb + p.t1 + 3] * R.nF[fb + p.t2 + 3] * R.nF[fb + p.t3 + 3] * xn > eta;
    };
    int first = EMPTY_LO, last = -1;
    unsigned long long miss = 0;
    bool need_exact = !R.pred || R.tlo || phi < plo;
    const int32_t* run = R.runs + (((size_t)tree * R.F.lm + j) * 2 + (core_int ? 1 : 0)) * RUN_REC;
    const int nrun = run[0];
    if (nrun >= 0) {
        // candidates: the runs clipped to [m_lo, m_hi]; range maxima answer "does any pass"
        const Rmq Q{R.rmq + ((size_t)j * RMQ_T + (p.t1 + 3) * 49 + (p.t2 + 3) * 7 + (p.t3 + 3)) * R.rmq_L * R.M, R.M};
        auto any = [&](int lo, int hi) { return lo <= hi && Q.max(lo, hi) * xn > eta; };
        // first / last passing term of [A, B] (one exists)
        auto first_in = [&](int A, int B) {
            if (any(A, A)) return A;  // the first candidate passes (no search)
            int lo = A + 1, hi = B;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (any(A, mid)) hi = mid;
                else lo = mid + 1;
            }
            return lo;
        };
        auto last_in = [&](int A, int B) {
            if (any(B, B)) return B;  // the last candidate passes
            int lo = A, hi = B - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (any(mid, B)) lo = mid;
                else hi = mid - 1;
            }
            return lo;
        };
        auto count_in = [&](int A, int B) {  // passing terms of [A, B] (only where a miss was found)
            unsigned long long c = 0;
            if (any(A, B))
                for (int m = A; m <= B; ++m) c += passes_m(m);
            return c;
        };
        const bool judged = R.pred && phi >= plo;
        for (int q = 0; q < nrun; ++q) {
            const int A = max((int)p.m_lo, run[1 + 2 * q]), B = min((int)p.m_hi, run[2 + 2 * q]);
            if (A > B) continue;
            if (judged) {
                // the judge: a passing term outside the prediction is a miss
                const unsigned long long ml = count_in(A, min(B, plo - 1)), mr = count_in(max(A, phi + 1), B);
                if (ml + mr) need_exact = true;
                miss += ml + mr;
            } else if (R.pred) {
                miss += count_in(A, B);  // predicted empty: every passing term is a miss
            }
        }
        if (need_exact)
            for (int q = 0; q < nrun; ++q) {
                const int A = max((int)p.m_lo, run[1 + 2 * q]), B = min((int)p.m_hi, run[2 + 2 * q]);
                if (!any(A, B)) continue;
                first = min(first, first_in(A, B));
                last = max(last, last_in(A, B));
            }
    } else {
        for (int m = p.m_lo; m <= p.m_hi; ++m) {
            if (!candidate(m)) continue;
            if (passes_m(m)) {
                first = min(first, m);
                last = m;
                if (R.pred && (m < plo || m > phi)) ++miss;
            }
        }
        need_exact = true;
    }
    if (R.tlo && last >= 0) {
        atomicMin(&R.tlo[a * 4 + S], first);
        atomicMax(&R.thi[a * 4 + S], last);
    }
    int lo = first, hi = last;
    if (R.pred && phi >= plo) {
        // the prediction, extended to every passing term (first..last when a miss was found)
        lo = need_exact ? min(lo, plo) : plo;
        hi = need_exact ? max(hi, phi) : phi;
    }
    if (hi < lo) {
        lo = EMPTY_LO;
        hi = -1;
        if (R.counts) atomicAdd(&R.counts[1], 1ull);
    }
    p.m_lo = (int16_t)lo;
    p.m_hi = (int16_t)hi;
    R.pairs[i] = p;
    if (R.counts && miss) atomicAdd(&R.counts[0], miss);
}

__global__ void k_targets(int n, int M, const int32_t* tlo, const int32_t* thi, float* T) {
    for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < n; a += gridDim.x * blockDim.x)
        for (int S = 0; S < 4; ++S) {
            const int hi = thi[a * 4 + S];
            float* t = T + (size_t)a * 12 + 3 * S;
            if (hi < 0) {
                t[0] = 1.0f;
                t[1] = 0.0f;
                t[2] = 0.0f;
            } else {
                t[0] = 0.0f;
                t[1] = (float)((double)tlo[a * 4 + S] / (M - 1));
                t[2] = (float)((double)hi / (M - 1));
            }
        }
}

__global__ void k_fill_i32v(int32_t* p, int n, int32_t v) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = v;
}

// Narrow the screened pairs' term ranges (after Step 2: the refined blocks'
// norms are known).  mode 1: exact screen; mode 2: learned screen with the
// exact judge.  X/targets (optional, device): the network's inputs and the
// exact screen's targets.  counts (device, 2): misses, empty pairs.
int schedule_narrow(const mra_op* op, const Forest& F, const ScreenOut& S, const double* gblk, int mode,
                    const void* model, int margin, float* X_out, float* T_out, unsigned long long* counts,
                    const Alloc& A, cudaStream_t st) {
    const int k3 = F.k * F.k * F.k, n = F.n, nb = n + S.nghost;
    const mra_mlp* M = nullptr;
    if (mode == 2) {
        M = mlp_checked(model);
        if (!M) { set_error("the learned screen needs a network handle"); return MRA_EINVAL; }
        if (mlp_n_in(M) != 16 || mlp_n_out(M) != 12) { set_error("the schedule network must map 16 inputs to 12 outputs"); return MRA_EINVAL; }
    }
    Scratch tmp(A);
    double *bn, *etab;
    MRA_TRY(tmp.get(&bn, (size_t)nb));
    MRA_TRY(tmp.get(&etab, (size_t)F.ntrees));
    k_block_norms<<<std::max(1, std::min(num_sms() * 16, (nb * 32 + 255) / 256)), 256, 0, st>>>(nb, n, k3, F.s, gblk, bn);
    MRA_CK_LAUNCH();
    k_eta_blk<<<(F.ntrees + 127) / 128, 128, 0, st>>>(F, S.dv, op->eps, op->M, etab);
    MRA_CK_LAUNCH();
    float* X = X_out;
    float* Y = nullptr;
    if (mode == 2 && !X) MRA_TRY(tmp.get(&X, (size_t)n * 16));
    if (X) {
        k_sched_features<<<(n + 127) / 128, 128, 0, st>>>(F, S.pair_off, S.pairs, bn, etab, op->J, op->mu, X);
        MRA_CK_LAUNCH();
    }
    if (mode == 2) {
        MRA_TRY(tmp.get(&Y, (size_t)n * 12));
        MRA_TRY(mlp_forward(M, X, n, Y, A, st));
    }
    int32_t *tlo = nullptr, *thi = nullptr;
    if (T_out) {
        MRA_TRY(tmp.get(&tlo, (size_t)n * 4));
        MRA_TRY(tmp.get(&thi, (size_t)n * 4));
        k_fill_i32v<<<(n * 4 + 255) / 256, 256, 0, st>>>(tlo, n * 4, EMPTY_LO);
        MRA_CK_LAUNCH();
        k_fill_i32v<<<(n * 4 + 255) / 256, 256, 0, st>>>(thi, n * 4, -1);
        MRA_CK_LAUNCH();
    }
    const double* rmq = nullptr;
    MRA_TRY(rmq_tables(op, st, &rmq));
    int32_t* runs;
    MRA_TRY(tmp.get(&runs, (size_t)F.ntrees * F.lm * 2 * RUN_REC));
    k_term_runs<<<F.ntrees, 64, 0, st>>>(F.ntrees, op->M, F.lm, S.sched, S.sl, runs);
    MRA_CK_LAUNCH();
    RangeArgs R;
    R.F = F; R.M = op->M; R.sl = S.sl; R.npairs = S.npairs; R.margin = margin;
    R.pairs = S.pairs; R.sched = S.sched; R.w = op->w; R.nF = op->nF; R.bn = bn; R.etab = etab;
    R.pred = Y; R.tlo = tlo; R.thi = thi; R.counts = counts;
    R.rmq = rmq; R.rmq_L = op->rmq_L; R.runs = runs;
    if (S.npairs > 0) {
        k_pair_ranges<<<(S.npairs + 255) / 256, 256, 0, st>>>(R);
        MRA_CK_LAUNCH();
    }
    if (T_out) {
        k_targets<<<(n + 127) / 128, 128, 0, st>>>(n, op->M, tlo, thi, T_out);
        MRA_CK_LAUNCH();
    }
    return MRA_OK;
}

int screen_data_impl(const mra_op* op, const mra_tree* f, float* X, float* T, cudaStream_t st) {
    const int k3 = op->k * op->k * op->k;
    if (f->k != op->k) { set_error("tree order k=%d differs from operator k=%d", f->k, op->k); return MRA_EINVAL; }
    if (f->nlev - 1 > op->J) { set_error("tree depth %d exceeds operator max_level %d", f->nlev - 1, op->J); return MRA_EINVAL; }
    if (f->state != MRA_TREE_REDUNDANT) { set_error("screen data needs a compressed (redundant) tree"); return MRA_ESTATE; }
    const Alloc& A = f->A;
    const Forest F = forest_of_tree(f);
    ScreenOut S;
    Scratch tmp(A);
    int rc = screen_forest(op, F, 0, A, st, &S);
    double* gblk = nullptr;
    if (rc == MRA_OK) rc = tmp.get(&gblk, (size_t)(S.nghost + 1) * k3);
    if (rc == MRA_OK) rc = ghost_refine_forest(F, S, gblk, st);
    if (rc == MRA_OK) rc = schedule_narrow(op, F, S, gblk, 1, nullptr, 0, X, T, nullptr, A, st);
    if (rc == MRA_OK) {
        int32_t herr[2] = {0, 0};
        cudaError_t e = cudaMemcpyAsync(herr, S.err, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) { set_error("screen data: %s", cudaGetErrorString(e)); rc = MRA_ECUDA; }
        else if (herr[0] || herr[1]) { set_error("screen/Step-2 error code %d/%d", herr[0], herr[1]); rc = MRA_ECUDA; }
    }
    screen_release(A, &S);
    return rc;
}

}  // namespace mra
