// Algorithm 3 (Sec. 5): the adaptive modified ns-form apply in d = 3.
//
//   pilot      ||T_0 f_0|| (all terms at level 0 on the root block) and ||f||
//   schedule   eta = eps ||T_0 f_0|| / ||f||; J_m (Sec. 4, eq. sep_apply with
//              the estimate of eq. NormEstimateUsing1DBlocks); per scale and
//              Core/Boundary subset the term range [m1, m2]
//   screen     warp per output node: the parity band (eq. fine_scale_band),
//              domain clipping, kept-term test, ballot + popc compaction into a
//              per-node list of (input block, t, m range) pairs; input boxes
//              absent from the tree go into a device hash set (Step 2)
//   ghosts     each missing input box is refined from its ancestor leaf with
//              the d = 0 half of eqs. recon_even / recon_odd
//   apply      per output node: for each pair and kept term,
//              ghat += w_m (F1 x F2 x F3) f_b as three mode products (Step 3)
#include <math.h>

#include <algorithm>
#include <vector>

#include "apply_common.cuh"

namespace mra {

int scan_exclusive(const int32_t* in, int32_t* out, int n, int32_t* total, cudaStream_t st);
int leaf_norm2(const mra_tree* t, double* out, cudaStream_t st);

// ------------------------------------------------------------------ pilot
__global__ void k_pilot(int k, int M, const double* w, const double* F, const double* s0, double* sigma) {
    extern __shared__ double sm[];
    const int k3 = k * k * k, kk = k * k;
    double* x = sm;
    double* z1 = x + k3;
    double* z2 = z1 + k3;
    double* y = z2 + k3;
    double* Fm = y + k3;
    __shared__ double red[32];
    for (int e = threadIdx.x; e < k3; e += blockDim.x) {
        x[e] = s0[e];
        y[e] = 0.0;
    }
    __syncthreads();
    for (int m = 0; m < M; ++m) {
        const double* Fs = F + ((size_t)m * 7 + 3) * kk;  // j = 0, l = 0
        for (int e = threadIdx.x; e < kk; e += blockDim.x) Fm[e] = Fs[e];
        __syncthreads();
        for (int idx = threadIdx.x; idx < k3; idx += blockDim.x) {  // dir 3
            int c = idx % k, base = idx - c;
            double a = 0.0;
            for (int i = 0; i < k; ++i) a += Fm[c * k + i] * x[base + i];
            z1[idx] = a;
        }
        __syncthreads();
        for (int idx = threadIdx.x; idx < k3; idx += blockDim.x) {  // dir 2
            int c3 = idx % k, c2 = (idx / k) % k, i1 = idx / kk;
            double a = 0.0;
            for (int i = 0; i < k; ++i) a += Fm[c2 * k + i] * z1[(i1 * k + i) * k + c3];
            z2[idx] = a;
        }
        __syncthreads();
        for (int idx = threadIdx.x; idx < k3; idx += blockDim.x) {  // dir 1
            int r = idx % kk, c1 = idx / kk;
            double a = 0.0;
            for (int i = 0; i < k; ++i) a += Fm[c1 * k + i] * z2[i * kk + r];
            y[idx] += w[m] * a;
        }
        __syncthreads();
    }
    double acc = 0.0;
    for (int e = threadIdx.x; e < k3; e += blockDim.x) acc += y[e] * y[e];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
        *sigma = sqrt(s);
    }
}

// The same pilot in two steps: block m writes w_m (F x F x F) s0 (F = F^{0;m,0})
// to ym[m], then one block sums the terms in a fixed order (deterministic) and
// takes the norm.
__global__ void k_pilot_terms(int k, int M, const double* w, const double* F, const double* s0, double* ym) {
    extern __shared__ double sm[];
    const int k3 = k * k * k, kk = k * k, m = blockIdx.x;
    double* x = sm;
    double* z1 = x + k3;
    double* z2 = z1 + k3;
    double* Fm = z2 + k3;
    const double* Fs = F + ((size_t)m * 7 + 3) * kk;  // j = 0, l = 0
    for (int e = threadIdx.x; e < k3; e += blockDim.x) x[e] = s0[e];
    for (int e = threadIdx.x; e < kk; e += blockDim.x) Fm[e] = Fs[e];
    __syncthreads();
    for (int idx = threadIdx.x; idx < k3; idx += blockDim.x) {  // dir 3
        int c = idx % k, base = idx - c;
        double a = 0.0;
        for (int i = 0; i < k; ++i) a += Fm[c * k + i] * x[base + i];
        z1[idx] = a;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < k3; idx += blockDim.x) {  // dir 2
        int c3 = idx % k, c2 = (idx / k) % k, i1 = idx / kk;
        double a = 0.0;
        for (int i = 0; i < k; ++i) a += Fm[c2 * k + i] * z1[(i1 * k + i) * k + c3];
        z2[idx] = a;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < k3; idx += blockDim.x) {  // dir 1
        int r = idx % kk, c1 = idx / kk;
        double a = 0.0;
        for (int i = 0; i < k; ++i) a += Fm[c1 * k + i] * z2[i * kk + r];
        ym[(size_t)m * k3 + idx] = w[m] * a;
    }
}

__global__ void k_pilot_reduce(int k3, int M, const double* ym, double* sigma) {
    __shared__ double red[32];
    double acc = 0.0;
    for (int e = threadIdx.x; e < k3; e += blockDim.x) {
        double y = 0.0;
        for (int m = 0; m < M; ++m) y += ym[(size_t)m * k3 + e];
        acc += y * y;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
        *sigma = sqrt(s);
    }
}

// ------------------------------------------------------------------ schedule
// sched layout (int32): Jm[M] | m1[nlev*4] | m2[nlev*4] | cnt[nlev*4*2]
__global__ void k_schedule(int M, int nlev, int unscreened, double eps, const double* w, const double* nF,
                           const double* est, const double* fnorm2, const double* sigma, int32_t* sched,
                           double* eta_out) {
    int32_t* Jm = sched;
    int32_t* m1 = Jm + M;
    int32_t* m2 = m1 + nlev * 4;
    int32_t* cnt = m2 + nlev * 4;
    const double fn = sqrt(*fnorm2);
    const double eta = fn > 0.0 ? eps * (*sigma) / fn : 0.0;
    if (threadIdx.x == 0) *eta_out = eta;
    for (int m = threadIdx.x; m < M; m += blockDim.x) {
        int jm = 0;
        if (unscreened) jm = nlev - 1;
        else
            for (int j = 1; j < nlev; ++j)
                if (w[m] * est[(size_t)j * M + m] > eta / M) jm = j;
        Jm[m] = jm;
    }
    __syncthreads();
    const double budget = eta / (2.0 * 216.0);
    for (int js = threadIdx.x; js < nlev * 4; js += blockDim.x) {
        const int j = js / 4, S = js % 4;
        int lo_m = 0, hi_m = -1;
        if (unscreened) {
            lo_m = 0;
            hi_m = M - 1;
        } else {
            // candidates: terms with J_m >= j, in increasing m
            int first = -1, last = -1, n = 0;
            for (int m = 0; m < M; ++m)
                if (Jm[m] >= j) {
                    if (first < 0) first = m;
                    last = m;
                    ++n;
                }
            if (n > 0) {
                auto e_of = [&](int m) {
                    const double* r = nF + ((size_t)j * M + m) * 7;
                    double c = fmax(fmax(r[2], r[3]), r[4]);
                    double b = fmax(fmax(r[0], r[1]), fmax(r[5], r[6]));
                    double v = w[m];
                    for (int q = 0; q < S; ++q) v *= c;
                    for (int q = S; q < 3; ++q) v *= b;
                    return v;
                };
                double acc = 0.0;
                int lo = first;
                for (; lo <= last; ++lo) {
                    if (Jm[lo] < j) continue;
                    double e = e_of(lo);
                    if (acc + e <= budget) acc += e;
                    else break;
                }
                acc = 0.0;
                int hi = last;
                for (; hi >= lo; --hi) {
                    if (Jm[hi] < j) continue;
                    double e = e_of(hi);
                    if (acc + e <= budget) acc += e;
                    else break;
                }
                if (hi >= lo && lo <= last) {
                    lo_m = lo;
                    hi_m = hi;
                }
            }
        }
        m1[js] = lo_m;
        m2[js] = hi_m;
        // kept-term counts for (j, S, core-at-internal-node)
        for (int ci = 0; ci < 2; ++ci) {
            int c = 0;
            for (int m = lo_m; m <= hi_m; ++m) {
                if (Jm[m] < j) continue;
                if (ci && S == 3 && Jm[m] > j) continue;
                ++c;
            }
            cnt[js * 2 + ci] = c;
        }
    }
}

// ------------------------------------------------------------------ screen
#define GH_EMPTY 0xffffffffffffffffull

__device__ inline uint64_t ghost_key(int j, int b1, int b2, int b3) {
    return ((uint64_t)j << 58) | morton3(b1, b2, b3);
}

__device__ inline uint32_t hash64(uint64_t k) {
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdull;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ull;
    k ^= k >> 33;
    return (uint32_t)k;
}

// returns the slot (>= 0) or -1 when the probe limit is exceeded
__device__ int ghost_insert(uint64_t* tab, uint32_t cap, uint64_t key) {
    uint32_t h = hash64(key) & (cap - 1);
    for (uint32_t it = 0; it < cap && it < 4096; ++it) {
        uint64_t prev = atomicCAS((unsigned long long*)&tab[h], (unsigned long long)GH_EMPTY,
                                  (unsigned long long)key);
        if (prev == GH_EMPTY || prev == key) return (int)h;
        h = (h + 1) & (cap - 1);
    }
    return -1;
}

__device__ int ghost_find(const uint64_t* tab, uint32_t cap, uint64_t key) {
    uint32_t h = hash64(key) & (cap - 1);
    for (uint32_t it = 0; it < cap && it < 4096; ++it) {
        uint64_t v = tab[h];
        if (v == key) return (int)h;
        if (v == GH_EMPTY) return -1;
        h = (h + 1) & (cap - 1);
    }
    return -1;
}

struct ScreenArgs {
    int n, M, nlev;
    const int32_t* coord;
    const int32_t* leaf;
    const uint64_t* key;
    const int32_t* off;
    const int32_t* sched;  // Jm | m1 | m2 | cnt
    uint64_t* gtab;
    uint32_t gcap;
    const int32_t* gid;    // slot -> ghost id (fill pass)
    int32_t* count;        // per node pair count (count pass)
    const int32_t* pair_off;
    Pair* pairs;
    int32_t* err;          // [0] hash overflow
};

// warp per output node; lane q covers band positions q, q+32, ... < 216
template <bool FILL>
__global__ void k_screen(ScreenArgs A) {
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const int32_t* m1 = A.sched + A.M;
    const int32_t* m2 = m1 + A.nlev * 4;
    const int32_t* cnt = m2 + A.nlev * 4;
    for (int i = warp; i < A.n; i += nwarps) {
        const int j = A.coord[4 * i], a1 = A.coord[4 * i + 1], a2 = A.coord[4 * i + 2], a3 = A.coord[4 * i + 3];
        const int leaf = A.leaf[i];
        const int N = 1 << j;
        int running = 0;
        const int base = FILL ? A.pair_off[i] : 0;
        for (int q0 = 0; q0 < 216; q0 += 32) {
            const int q = q0 + lane;
            bool valid = false;
            int t1 = 0, t2 = 0, t3 = 0, S = 0, ci = 0, in = 0;
            if (q < 216) {
                t1 = band_t(a1, q / 36);
                t2 = band_t(a2, (q / 6) % 6);
                t3 = band_t(a3, q % 6);
                const int b1 = a1 - t1, b2 = a2 - t2, b3 = a3 - t3;
                if (b1 >= 0 && b2 >= 0 && b3 >= 0 && b1 < N && b2 < N && b3 < N) {
                    S = (abs(t1) <= 1) + (abs(t2) <= 1) + (abs(t3) <= 1);
                    ci = (S == 3 && !leaf) ? 1 : 0;
                    if (cnt[(j * 4 + S) * 2 + ci] > 0) {
                        valid = true;
                        int idx = find_key_exact(A.key, A.off[j], A.off[j + 1], morton3(b1, b2, b3));
                        if (idx >= 0) in = idx;
                        else {
                            uint64_t gk = ghost_key(j, b1, b2, b3);
                            if (!FILL) {
                                if (ghost_insert(A.gtab, A.gcap, gk) < 0) atomicExch(A.err, 1);
                            } else {
                                int slot = ghost_find(A.gtab, A.gcap, gk);
                                in = slot >= 0 ? -1 - A.gid[slot] : 0;
                                if (slot < 0) atomicExch(A.err, 2);
                            }
                        }
                    }
                }
            }
            const unsigned bal = __ballot_sync(0xffffffffu, valid);
            if (FILL && valid) {
                const int pos = base + running + __popc(bal & ((1u << lane) - 1u));
                Pair p;
                p.out = i;
                p.in = in;
                p.m_lo = (int16_t)m1[j * 4 + S];
                p.m_hi = (int16_t)m2[j * 4 + S];
                p.t1 = (int8_t)t1;
                p.t2 = (int8_t)t2;
                p.t3 = (int8_t)t3;
                p.flags = (uint8_t)ci;
                A.pairs[pos] = p;
            }
            running += __popc(bal);
        }
        if (!FILL && lane == 0) A.count[i] = running;
    }
}

__global__ void k_fill_u64(uint64_t* p, size_t n, uint64_t v) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        p[i] = v;
}

__global__ void k_ghost_ids(const uint64_t* tab, uint32_t cap, int32_t* gid, uint64_t* gkeys, int32_t* ng) {
    for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < cap; s += gridDim.x * blockDim.x) {
        uint64_t v = tab[s];
        if (v != GH_EMPTY) {
            int id = atomicAdd(ng, 1);
            gid[s] = id;
            gkeys[id] = v;
        }
    }
}

__device__ inline uint32_t compact1by2(uint64_t x) {
    x &= 0x1249249249249249ull;
    x = (x ^ (x >> 2)) & 0x10c30c30c30c30c3ull;
    x = (x ^ (x >> 4)) & 0x100f00f00f00f00full;
    x = (x ^ (x >> 8)) & 0x1f0000ff0000ffull;
    x = (x ^ (x >> 16)) & 0x1f00000000ffffull;
    x = (x ^ (x >> 32)) & 0x1fffffull;
    return (uint32_t)x;
}

// Step 2: block per ghost; refine the covering ancestor leaf down to level j.
__global__ void k_ghost_refine(int k, const uint64_t* gkeys, const uint64_t* key, const int32_t* off,
                               const int32_t* leaf, const double* s, const double* filt, double* gblk,
                               int32_t* err) {
    extern __shared__ double sm[];
    const int k3 = k * k * k, kk = k * k;
    double* HT = sm;             // 2 k x k: HT[p][a][i] = H^(p)[i][a]
    double* x = HT + 2 * kk;
    double* y = x + k3;
    double* z = y + k3;
    const uint64_t gk = gkeys[blockIdx.x];
    const int j = (int)(gk >> 58);
    const uint64_t mk = gk & ((1ull << 58) - 1);
    const int b1 = compact1by2(mk >> 2), b2 = compact1by2(mk >> 1), b3 = compact1by2(mk);
    for (int e = threadIdx.x; e < 2 * kk; e += blockDim.x) {
        int p = e / kk, r = e % kk, a = r / k, i = r % k;
        HT[e] = filt[p * kk + i * k + a];
    }
    __shared__ int anc, jj;
    if (threadIdx.x == 0) {
        anc = -1;
        for (int lv = j - 1; lv >= 0 && anc < 0; --lv) {
            int sh = j - lv;
            int idx = find_key_exact(key, off[lv], off[lv + 1], morton3(b1 >> sh, b2 >> sh, b3 >> sh));
            if (idx >= 0) {
                anc = idx;
                jj = lv;
            }
        }
        if (anc < 0 || !leaf[anc]) atomicExch(err, 3);
    }
    __syncthreads();
    if (anc < 0) return;
    for (int e = threadIdx.x; e < k3; e += blockDim.x) x[e] = s[(size_t)anc * k3 + e];
    __syncthreads();
    for (int lv = jj; lv < j; ++lv) {
        const int sh = j - lv - 1;
        const int p1 = (b1 >> sh) & 1, p2 = (b2 >> sh) & 1, p3 = (b3 >> sh) & 1;
        // x <- (H^(p1)T x H^(p2)T x H^(p3)T) x
        for (int idx = threadIdx.x; idx < k3; idx += blockDim.x) {
            int c = idx % k, base = idx - c;
            double a = 0.0;
            for (int i = 0; i < k; ++i) a += HT[p3 * kk + c * k + i] * x[base + i];
            y[idx] = a;
        }
        __syncthreads();
        for (int idx = threadIdx.x; idx < k3; idx += blockDim.x) {
            int c3 = idx % k, c2 = (idx / k) % k, i1 = idx / kk;
            double a = 0.0;
            for (int i = 0; i < k; ++i) a += HT[p2 * kk + c2 * k + i] * y[(i1 * k + i) * k + c3];
            z[idx] = a;
        }
        __syncthreads();
        for (int idx = threadIdx.x; idx < k3; idx += blockDim.x) {
            int r = idx % kk, c1 = idx / kk;
            double a = 0.0;
            for (int i = 0; i < k; ++i) a += HT[p1 * kk + c1 * k + i] * z[i * kk + r];
            x[idx] = a;
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < k3; e += blockDim.x) gblk[(size_t)blockIdx.x * k3 + e] = x[e];
}

// ------------------------------------------------------------------ apply
// Block per output node.  T is the contraction type (double or float); the
// per-pair sum over terms is accumulated in T and added to the FP64 output.
template <class T>
__global__ void __launch_bounds__(128) k_apply_simt(ApplyArgs A) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int k = A.k, k3 = k * k * k, kk = k * k;
    double* y = (double*)smraw;            // k3 FP64 accumulator
    T* x = (T*)(y + k3);
    T* z1 = x + k3;
    T* z2 = z1 + k3;
    T* yp = z2 + k3;                        // per-pair partial
    T* Fs = yp + k3;                        // 3 k x k
    __shared__ double red[32];
    __shared__ unsigned long long items;
    const T* Ftab = (const T*)A.F;
    const int M = A.M;
    for (int i = blockIdx.x; i < A.n; i += gridDim.x) {
        const int j = A.coord[4 * i];
        for (int e = threadIdx.x; e < k3; e += blockDim.x) y[e] = 0.0;
        if (threadIdx.x == 0) items = 0;
        const int p0 = A.pair_off[i], p1 = A.pair_off[i + 1];
        for (int p = p0; p < p1; ++p) {
            const Pair pr = A.pairs[p];
            const double* src = pr.in >= 0 ? A.s + (size_t)pr.in * k3 : A.gblk + (size_t)(-1 - pr.in) * k3;
            double xn2 = 0.0;
            for (int e = threadIdx.x; e < k3; e += blockDim.x) {
                double v = src[e];
                x[e] = (T)v;
                yp[e] = (T)0;
                xn2 += v * v;
            }
            double xnorm = 0.0;
            if (A.eta_blk >= 0.0) {
                for (int o = 16; o > 0; o >>= 1) xn2 += __shfl_xor_sync(0xffffffffu, xn2, o);
                __syncthreads();
                if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = xn2;
                __syncthreads();
                for (int q = 0; q < (int)(blockDim.x >> 5); ++q) xnorm += red[q];
                xnorm = sqrt(xnorm);
            }
            __syncthreads();
            for (int m = pr.m_lo; m <= pr.m_hi; ++m) {
                const int jm = A.Jm[m];
                if (jm < j) continue;
                if ((pr.flags & 1) && jm > j) continue;
                const size_t fb = ((size_t)j * M + m) * 7;
                if (A.eta_blk >= 0.0) {
                    double est = A.w[m] * A.nF[fb + pr.t1 + 3] * A.nF[fb + pr.t2 + 3] * A.nF[fb + pr.t3 + 3] * xnorm;
                    if (!(est > A.eta_blk)) continue;
                }
                const T* F1 = Ftab + (fb + pr.t1 + 3) * kk;
                const T* F2 = Ftab + (fb + pr.t2 + 3) * kk;
                const T* F3 = Ftab + (fb + pr.t3 + 3) * kk;
                for (int e = threadIdx.x; e < kk; e += blockDim.x) {
                    Fs[e] = F1[e];
                    Fs[kk + e] = F2[e];
                    Fs[2 * kk + e] = F3[e];
                }
                __syncthreads();
                for (int idx = threadIdx.x; idx < k3; idx += blockDim.x) {  // direction 3
                    int c = idx % k, base = idx - c;
                    T a = 0;
                    for (int q = 0; q < k; ++q) a += Fs[2 * kk + c * k + q] * x[base + q];
                    z1[idx] = a;
                }
                __syncthreads();
                for (int idx = threadIdx.x; idx < k3; idx += blockDim.x) {  // direction 2
                    int c3 = idx % k, c2 = (idx / k) % k, i1 = idx / kk;
                    T a = 0;
                    for (int q = 0; q < k; ++q) a += Fs[kk + c2 * k + q] * z1[(i1 * k + q) * k + c3];
                    z2[idx] = a;
                }
                __syncthreads();
                const T wm = (T)A.w[m];
                for (int idx = threadIdx.x; idx < k3; idx += blockDim.x) {  // direction 1
                    int r = idx % kk, c1 = idx / kk;
                    T a = 0;
                    for (int q = 0; q < k; ++q) a += Fs[c1 * k + q] * z2[q * kk + r];
                    yp[idx] += wm * a;
                }
                if (threadIdx.x == 0) items++;
                __syncthreads();
            }
            for (int e = threadIdx.x; e < k3; e += blockDim.x) y[e] += (double)yp[e];
            __syncthreads();
        }
        for (int e = threadIdx.x; e < k3; e += blockDim.x) A.out[(size_t)i * k3 + e] = y[e];
        if (threadIdx.x == 0 && A.n_items) atomicAdd(A.n_items, items);
        __syncthreads();
    }
}

// ------------------------------------------------------------------ driver
int apply_impl(const mra_op* op, const mra_tree* f, const mra_apply_opts* o, cudaStream_t st, mra_tree** gout,
               mra_apply_stats* stats) {
    const int k = op->k, k3 = k * k * k, M = op->M, n = f->n, nlev = f->nlev;
    if (f->k != k) { set_error("tree order k=%d differs from operator k=%d", f->k, k); return MRA_EINVAL; }
    if (nlev - 1 > op->J) { set_error("tree depth %d exceeds operator max_level %d", nlev - 1, op->J); return MRA_EINVAL; }
    if (f->state != MRA_TREE_REDUNDANT) { set_error("apply_ns needs a compressed (redundant) tree"); return MRA_ESTATE; }
    const int prec = o ? o->precision : MRA_PREC_FP64;
    if (prec != MRA_PREC_FP64 && prec != MRA_PREC_FP32 && prec != MRA_PREC_TC_SPLIT) {
        set_error("precision %d is not available", prec);
        return MRA_EINVAL;
    }
    if (prec == MRA_PREC_TC_SPLIT && ((o && (o->block_screen || o->itemwise)) || k != 8)) {
        set_error("the tensor-core apply needs k = 8 and the static screen");
        return MRA_EINVAL;
    }
    const Alloc& A = f->A;
    cudaEvent_t ev[4];
    for (int e = 0; e < 4; ++e) MRA_CK(cudaEventCreate(&ev[e]));
    MRA_CK(cudaEventRecord(ev[0], st));

    double* dv;  // [0] ||f||^2 [1] sigma [2] eta
    int32_t *sched, *count, *pair_off, *total, *err;
    MRA_TRY(dalloc(A, &dv, 4));
    MRA_TRY(dalloc(A, &sched, M + nlev * 16));
    MRA_TRY(dalloc(A, &count, n + 1));
    MRA_TRY(dalloc(A, &pair_off, n + 1));
    MRA_TRY(dalloc(A, &total, 2));
    MRA_TRY(dalloc(A, &err, 2));
    MRA_CK(cudaMemsetAsync(dv, 0, 4 * sizeof(double), st));
    MRA_CK(cudaMemsetAsync(err, 0, 2 * sizeof(int32_t), st));
    MRA_CK(cudaMemsetAsync(total, 0, 2 * sizeof(int32_t), st));
    MRA_TRY(leaf_norm2(f, dv, st));
    double* ym;
    MRA_TRY(dalloc(A, &ym, (size_t)M * k3));
    k_pilot_terms<<<M, 128, (3 * (size_t)k3 + k * k) * sizeof(double), st>>>(k, M, op->w, op->F, f->s, ym);
    MRA_CK_LAUNCH();
    k_pilot_reduce<<<1, 256, 0, st>>>(k3, M, ym, dv + 1);
    MRA_CK_LAUNCH();
    A.put(ym);
    const int unscreened = o ? o->unscreened : 0;
    k_schedule<<<1, 256, 0, st>>>(M, nlev, unscreened, op->eps, op->w, op->nF, op->est, dv, dv + 1, sched, dv + 2);
    MRA_CK_LAUNCH();

    // ghost hash set sized for the worst case (every band position missing)
    uint64_t gcap64 = 1024;
    while (gcap64 < (uint64_t)n * 216ull * 2ull && gcap64 < (1ull << 28)) gcap64 <<= 1;
    const uint32_t gcap = (uint32_t)gcap64;
    uint64_t* gtab;
    int32_t* gid;
    MRA_TRY(dalloc(A, &gtab, gcap));
    MRA_TRY(dalloc(A, &gid, gcap));
    k_fill_u64<<<1024, 256, 0, st>>>(gtab, gcap, GH_EMPTY);
    MRA_CK_LAUNCH();

    ScreenArgs sa;
    sa.n = n; sa.M = M; sa.nlev = nlev;
    sa.coord = f->a.coord; sa.leaf = f->a.leaf; sa.key = f->a.key; sa.off = f->a.off;
    sa.sched = sched; sa.gtab = gtab; sa.gcap = gcap; sa.gid = gid;
    sa.count = count; sa.pair_off = pair_off; sa.pairs = nullptr; sa.err = err;
    const int sblocks = (int)std::min<long>(4096, ((long)n * 32 + 255) / 256);
    k_screen<false><<<sblocks, 256, 0, st>>>(sa);
    MRA_CK_LAUNCH();
    MRA_TRY(scan_exclusive(count, pair_off, n, total, st));
    MRA_CK(cudaMemcpyAsync(pair_off + n, total, sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
    uint64_t* gkeys;
    MRA_TRY(dalloc(A, &gkeys, gcap));
    k_ghost_ids<<<1024, 256, 0, st>>>(gtab, gcap, gid, gkeys, total + 1);
    MRA_CK_LAUNCH();
    // the one host synchronisation: pair and ghost counts size the worklist
    int32_t h[2] = {0, 0}, herr[2] = {0, 0};
    MRA_CK(cudaMemcpyAsync(h, total, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    MRA_CK(cudaMemcpyAsync(herr, err, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    MRA_CK(cudaStreamSynchronize(st));
    if (herr[0]) { set_error("ghost hash set overflow"); return MRA_ECUDA; }
    const int npairs = h[0], nghost = h[1];
    Pair* pairs;
    double* gblk;
    MRA_TRY(dalloc(A, &pairs, (size_t)npairs + 1));
    MRA_TRY(dalloc(A, &gblk, (size_t)(nghost + 1) * k3));
    MRA_CK(cudaEventRecord(ev[1], st));
    if (nghost > 0) {
        const size_t gsm = (2 * (size_t)k * k + 3 * (size_t)k3) * sizeof(double);
        k_ghost_refine<<<nghost, 128, gsm, st>>>(k, gkeys, f->a.key, f->a.off, f->a.leaf, f->s, f->filt, gblk, err);
        MRA_CK_LAUNCH();
    }
    sa.pairs = pairs;
    k_screen<true><<<sblocks, 256, 0, st>>>(sa);
    MRA_CK_LAUNCH();
    MRA_CK(cudaEventRecord(ev[2], st));

    mra_tree* g = nullptr;
    MRA_TRY(tree_clone_skeleton(f, &g));
    g->state = MRA_TREE_NSFORM;
    unsigned long long* nitems;
    MRA_TRY(dalloc(A, &nitems, 1));
    MRA_CK(cudaMemsetAsync(nitems, 0, sizeof(unsigned long long), st));

    ApplyArgs aa;
    aa.k = k; aa.M = M; aa.n = n; aa.pairs = pairs; aa.pair_off = pair_off; aa.coord = f->a.coord;
    aa.s = f->s; aa.gblk = gblk; aa.w = op->w; aa.nF = op->nF; aa.Jm = sched; aa.out = g->s; aa.n_items = nitems;
    aa.eta_blk = -1.0;
    if (o && o->block_screen) {
        // eps ||T_0 f_0|| / sqrt(N 216 M), evaluated on the host from the device sigma
        double sig = 0.0;
        MRA_CK(cudaMemcpyAsync(&sig, dv + 1, sizeof(double), cudaMemcpyDeviceToHost, st));
        MRA_CK(cudaStreamSynchronize(st));
        aa.eta_blk = op->eps * sig / sqrt((double)n * 216.0 * M);
    }
    int rc = MRA_OK;
    const bool itemwise = (o && o->itemwise) || aa.eta_blk >= 0.0;
    if (prec == MRA_PREC_TC_SPLIT) {
        // tcgen05 FP16 hi/lo split products (apply_tc.cu)
        rc = launch_apply_tc(aa, nghost, nlev, op, err + 1, st);
        if (rc != MRA_OK) return rc;
    } else if (!itemwise) {
        // Algorithm 3's nested sums, factorised (apply_fact.cu)
        aa.F = prec == MRA_PREC_FP64 ? (const void*)op->F : (const void*)op->F32;
        MRA_TRY(launch_apply_fact(aa, prec, nlev, st));
    } else if (prec == MRA_PREC_FP64) {
        aa.F = op->F;
        size_t smem = (size_t)k3 * sizeof(double) + (4 * (size_t)k3 + 3 * k * k) * sizeof(double);
        MRA_CK(cudaFuncSetAttribute(k_apply_simt<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_apply_simt<double><<<std::min(n, 152 * 16), 128, smem, st>>>(aa);
        MRA_CK_LAUNCH();
    } else {
        aa.F = op->F32;
        size_t smem = (size_t)k3 * sizeof(double) + (4 * (size_t)k3 + 3 * k * k) * sizeof(float);
        MRA_CK(cudaFuncSetAttribute(k_apply_simt<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_apply_simt<float><<<std::min(n, 152 * 16), 128, smem, st>>>(aa);
        MRA_CK_LAUNCH();
    }
    MRA_CK(cudaEventRecord(ev[3], st));

    if (stats) {
        unsigned long long ni = 0;
        double hv[3];
        MRA_CK(cudaMemcpyAsync(&ni, nitems, sizeof(ni), cudaMemcpyDeviceToHost, st));
        MRA_CK(cudaMemcpyAsync(hv, dv, 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
        MRA_CK(cudaMemcpyAsync(herr, err, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        MRA_CK(cudaStreamSynchronize(st));
        stats->n_pairs = npairs;
        stats->n_items = (int64_t)ni;
        stats->n_ghosts = nghost;
        stats->n_out_nodes = n;
        stats->fnorm = sqrt(hv[0]);
        stats->sigma = hv[1];
        stats->eta = hv[2];
        cudaEventElapsedTime(&stats->ms_screen, ev[0], ev[1]);
        cudaEventElapsedTime(&stats->ms_ghost, ev[1], ev[2]);
        cudaEventElapsedTime(&stats->ms_apply, ev[2], ev[3]);
        if (herr[1] == 4) { set_error("tensor-core apply: an MMA completion wait reached its limit"); rc = MRA_ETIMEOUT; }
        else if (herr[0] || herr[1]) { set_error("screen/ghost error code %d/%d", herr[0], herr[1]); rc = MRA_ECUDA; }
    }
    A.put(dv); A.put(sched); A.put(count); A.put(pair_off); A.put(total); A.put(err);
    A.put(gtab); A.put(gid); A.put(gkeys); A.put(pairs); A.put(gblk); A.put(nitems);
    for (int e = 0; e < 4; ++e) cudaEventDestroy(ev[e]);
    *gout = g;
    return rc;
}

}  // namespace mra

// ------------------------------------------------------------------ no-alloc apply
// mra_apply_ns_noalloc: the same screen, Step-2 refinement and SIMT apply as
// apply_impl, for callers that cannot allocate device memory (code running
// where another component owns the allocator, or inside work that must not
// call cudaMalloc/cudaFree).  Its scratch lives in one file-scope device array
// of fixed size that every GPU loading the library keeps until exit.
#include <atomic>
#include <mutex>

namespace mra {

#define NA_MAX_NODES 1024
#define NA_MAX_K 8
#define NA_MAX_GHOSTS 4096
#define NA_HASH_CAP 16384u

struct NaLayout {
    size_t dv, sched, count, pair_off, total, err, gtab, gid, gkeys, pairs, gblk, nitems, bytes;
};

static constexpr size_t na_align(size_t x) { return (x + 255) & ~(size_t)255; }

static NaLayout na_layout() {
    NaLayout L;
    size_t o = 0;
    L.dv = o;       o = na_align(o + 4 * sizeof(double));
    L.sched = o;    o = na_align(o + (MRA_MAX_TERMS + 16 * (MRA_MAX_LEVEL + 1)) * sizeof(int32_t));
    L.count = o;    o = na_align(o + (NA_MAX_NODES + 1) * sizeof(int32_t));
    L.pair_off = o; o = na_align(o + (NA_MAX_NODES + 1) * sizeof(int32_t));
    L.total = o;    o = na_align(o + 2 * sizeof(int32_t));
    L.err = o;      o = na_align(o + 2 * sizeof(int32_t));
    L.gtab = o;     o = na_align(o + NA_HASH_CAP * sizeof(uint64_t));
    L.gid = o;      o = na_align(o + NA_HASH_CAP * sizeof(int32_t));
    L.gkeys = o;    o = na_align(o + NA_HASH_CAP * sizeof(uint64_t));
    L.pairs = o;    o = na_align(o + (size_t)NA_MAX_NODES * 216 * sizeof(Pair));
    L.gblk = o;     o = na_align(o + (size_t)NA_MAX_GHOSTS * NA_MAX_K * NA_MAX_K * NA_MAX_K * sizeof(double));
    L.nitems = o;   o = na_align(o + sizeof(unsigned long long));
    L.bytes = o;
    return L;
}

// 21 MiB: enough for na_layout() (about 20.8 MiB); fixed at compile time.
#define NA_SCRATCH_BYTES (21u * 1024u * 1024u)
static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_SCRATCH_BYTES];

// Host-side device addresses of g_noalloc_scratch, one per device, obtained
// once with cudaGetSymbolAddress while that device is current.  In host code
// the symbol itself is only a host stand-in, never a device address.
static unsigned char* g_na_ptr[256];
static std::mutex g_na_mu;

static int na_scratch(unsigned char** out) {
    int dev = 0;
    MRA_CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 256) { set_error("device index %d out of range", dev); return MRA_EINVAL; }
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            set_error("cudaGetSymbolAddress(scratch) failed: %s", cudaGetErrorString(e));
            return MRA_ECUDA;
        }
        g_na_ptr[dev] = (unsigned char*)p;
    }
    *out = g_na_ptr[dev];
    return MRA_OK;
}

int apply_noalloc_impl(const mra_op* op, const mra_tree* f, int precision, double* ghat, cudaStream_t st,
                       int64_t* n_items_host) {
    const int k = op->k, k3 = k * k * k, M = op->M, n = f->n, nlev = f->nlev;
    static_assert(sizeof(Pair) == 16, "pair size");
    const NaLayout L = na_layout();
    static_assert(NA_SCRATCH_BYTES >= 20u * 1024u * 1024u, "scratch size");
    if (L.bytes > NA_SCRATCH_BYTES) { set_error("internal: no-alloc scratch layout too large"); return MRA_ECUDA; }
    if (f->k != k) { set_error("tree order k=%d differs from operator k=%d", f->k, k); return MRA_EINVAL; }
    if (k > NA_MAX_K) { set_error("no-alloc apply supports k <= %d (got %d)", NA_MAX_K, k); return MRA_EINVAL; }
    if (n > NA_MAX_NODES) { set_error("no-alloc apply supports at most %d nodes (got %d)", NA_MAX_NODES, n); return MRA_EINVAL; }
    if (nlev - 1 > op->J) { set_error("tree depth %d exceeds operator max_level %d", nlev - 1, op->J); return MRA_EINVAL; }
    if (f->state != MRA_TREE_REDUNDANT) { set_error("apply needs a compressed (redundant) tree"); return MRA_ESTATE; }
    if (precision != MRA_PREC_FP64 && precision != MRA_PREC_FP32) { set_error("precision %d is not available", precision); return MRA_EINVAL; }
    if (!ghat) { set_error("output buffer is NULL"); return MRA_EINVAL; }
    unsigned char* base = nullptr;
    MRA_TRY(na_scratch(&base));
    double* dv = (double*)(base + L.dv);
    int32_t* sched = (int32_t*)(base + L.sched);
    int32_t* count = (int32_t*)(base + L.count);
    int32_t* pair_off = (int32_t*)(base + L.pair_off);
    int32_t* total = (int32_t*)(base + L.total);
    int32_t* err = (int32_t*)(base + L.err);
    uint64_t* gtab = (uint64_t*)(base + L.gtab);
    int32_t* gid = (int32_t*)(base + L.gid);
    uint64_t* gkeys = (uint64_t*)(base + L.gkeys);
    Pair* pairs = (Pair*)(base + L.pairs);
    double* gblk = (double*)(base + L.gblk);
    unsigned long long* nitems = (unsigned long long*)(base + L.nitems);

    // the array keeps the previous call's contents: clear what must start at zero
    MRA_CK(cudaMemsetAsync(dv, 0, 4 * sizeof(double), st));
    MRA_CK(cudaMemsetAsync(total, 0, 2 * sizeof(int32_t), st));
    MRA_CK(cudaMemsetAsync(err, 0, 2 * sizeof(int32_t), st));
    MRA_CK(cudaMemsetAsync(nitems, 0, sizeof(unsigned long long), st));
    k_fill_u64<<<64, 256, 0, st>>>(gtab, NA_HASH_CAP, GH_EMPTY);
    MRA_CK_LAUNCH();
    MRA_TRY(leaf_norm2(f, dv, st));
    const size_t pilot_smem = (4 * (size_t)k3 + k * k) * sizeof(double);
    k_pilot<<<1, 128, pilot_smem, st>>>(k, M, op->w, op->F, f->s, dv + 1);
    MRA_CK_LAUNCH();
    k_schedule<<<1, 256, 0, st>>>(M, nlev, 0, op->eps, op->w, op->nF, op->est, dv, dv + 1, sched, dv + 2);
    MRA_CK_LAUNCH();
    ScreenArgs sa;
    sa.n = n; sa.M = M; sa.nlev = nlev;
    sa.coord = f->a.coord; sa.leaf = f->a.leaf; sa.key = f->a.key; sa.off = f->a.off;
    sa.sched = sched; sa.gtab = gtab; sa.gcap = NA_HASH_CAP; sa.gid = gid;
    sa.count = count; sa.pair_off = pair_off; sa.pairs = nullptr; sa.err = err;
    const int sblocks = (int)std::min<long>(4096, ((long)n * 32 + 255) / 256);
    k_screen<false><<<sblocks, 256, 0, st>>>(sa);
    MRA_CK_LAUNCH();
    MRA_TRY(scan_exclusive(count, pair_off, n, total, st));
    MRA_CK(cudaMemcpyAsync(pair_off + n, total, sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
    k_ghost_ids<<<64, 256, 0, st>>>(gtab, NA_HASH_CAP, gid, gkeys, total + 1);
    MRA_CK_LAUNCH();
    int32_t h[2] = {0, 0}, herr[2] = {0, 0};
    MRA_CK(cudaMemcpyAsync(h, total, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    MRA_CK(cudaMemcpyAsync(herr, err, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    MRA_CK(cudaStreamSynchronize(st));
    if (herr[0] || h[1] > NA_MAX_GHOSTS) {
        set_error("no-alloc apply supports at most %d refined input blocks (Step 2)", NA_MAX_GHOSTS);
        return MRA_EINVAL;
    }
    const int nghost = h[1];
    if (nghost > 0) {
        const size_t gsm = (2 * (size_t)k * k + 3 * (size_t)k3) * sizeof(double);
        k_ghost_refine<<<nghost, 128, gsm, st>>>(k, gkeys, f->a.key, f->a.off, f->a.leaf, f->s, f->filt, gblk, err);
        MRA_CK_LAUNCH();
    }
    sa.pairs = pairs;
    k_screen<true><<<sblocks, 256, 0, st>>>(sa);
    MRA_CK_LAUNCH();
    ApplyArgs aa;
    aa.k = k; aa.M = M; aa.n = n; aa.pairs = pairs; aa.pair_off = pair_off; aa.coord = f->a.coord;
    aa.s = f->s; aa.gblk = gblk; aa.w = op->w; aa.nF = op->nF; aa.Jm = sched; aa.out = ghat; aa.n_items = nitems;
    aa.eta_blk = -1.0;
    if (precision == MRA_PREC_FP64) {
        aa.F = op->F;
        size_t smem = (size_t)k3 * sizeof(double) + (4 * (size_t)k3 + 3 * k * k) * sizeof(double);
        k_apply_simt<double><<<std::min(n, 152 * 16), 128, smem, st>>>(aa);
        MRA_CK_LAUNCH();
    } else {
        aa.F = op->F32;
        size_t smem = (size_t)k3 * sizeof(double) + (4 * (size_t)k3 + 3 * k * k) * sizeof(float);
        k_apply_simt<float><<<std::min(n, 152 * 16), 128, smem, st>>>(aa);
        MRA_CK_LAUNCH();
    }
    if (n_items_host) {
        unsigned long long ni = 0;
        MRA_CK(cudaMemcpyAsync(&ni, nitems, sizeof(ni), cudaMemcpyDeviceToHost, st));
        MRA_CK(cudaMemcpyAsync(herr, err, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        MRA_CK(cudaStreamSynchronize(st));
        *n_items_host = (int64_t)ni;
        if (herr[0] || herr[1]) { set_error("screen/ghost error code %d/%d", herr[0], herr[1]); return MRA_ECUDA; }
    }
    return MRA_OK;
}

}  // namespace mra
