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

// ------------------------------------------------------------------ forest
__device__ inline int forest_tree(const Forest& F, int i) { return F.node_tree ? F.node_tree[i] : 0; }

// ||f_b||^2 = sum over the leaves of tree b of ||s||^2 (Parseval).  A warp takes a
// contiguous run of nodes (the trees of a forest are contiguous) and adds its sum to
// its tree's total once per tree it meets, not once per node.
__global__ void k_forest_norm2(Forest F, double* dv) {
    const int k3 = F.k * F.k * F.k, lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nwarps = (gridDim.x * blockDim.x) >> 5;
    const int per = (F.n + nwarps - 1) / nwarps;
    const int i0 = min(F.n, warp * per), i1 = min(F.n, i0 + per);
    // every branch below is uniform over the warp (all lanes walk the same nodes)
    auto flush = [&](double& acc, int tree) {
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0 && acc != 0.0) atomicAdd(&dv[4 * tree], acc);
        acc = 0.0;
    };
    double acc = 0.0;
    int tree = i0 < i1 ? forest_tree(F, i0) : 0;
    for (int i = i0; i < i1; ++i) {
        const int b = forest_tree(F, i);
        if (b != tree) {
            flush(acc, tree);
            tree = b;
        }
        if (!F.leaf[i]) continue;
        const double* s = F.s + (size_t)i * k3;
        for (int e = lane; e < k3; e += 32) acc = fma(s[e], s[e], acc);
    }
    flush(acc, tree);
}

// Pilot ||T_0 f_0|| in two steps: block (m, b) writes w_m (F x F x F) s0_b
// (F = F^{0;m,0}, s0_b the root block of tree b) to ym[b][m]; then the terms are
// summed per coefficient and the squares per tree, in a fixed order, and the norm taken.
__global__ void k_pilot_terms(Forest F, int M, const double* w, const double* Ftab, double* ym) {
    extern __shared__ double sm[];
    const int k = F.k, k3 = k * k * k, kk = k * k, m = blockIdx.x, b = blockIdx.y;
    double* x = sm;
    double* z1 = x + k3;
    double* z2 = z1 + k3;
    double* Fm = z2 + k3;
    const double* s0 = F.s + (size_t)F.off[b * (F.lm + 1)] * k3;
    const double* Fs = Ftab + ((size_t)m * 7 + 3) * kk;  // j = 0, l = 0
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
    double* yo = ym + ((size_t)b * M + m) * k3;
    for (int idx = threadIdx.x; idx < k3; idx += blockDim.x) {  // dir 1
        int r = idx % kk, c1 = idx / kk;
        double a = 0.0;
        for (int i = 0; i < k; ++i) a += Fm[c1 * k + i] * z2[i * kk + r];
        yo[idx] = w[m] * a;
    }
}

// Block (b, q) sums the terms of the 32 coefficients e = 32 q + lane of tree b's
// pilot, eight warps taking every eighth term, and writes the sum of their squares
// to part[b][q]; k_pilot_reduce then adds a tree's parts in order (deterministic).
__global__ void k_pilot_partial(int k3, int M, const double* ym, double* part) {
    __shared__ double sl[8][33];
    const int b = blockIdx.x, q = blockIdx.y, lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
    const int e = q * 32 + lane;
    const double* yb = ym + (size_t)b * M * k3;
    double y = 0.0;
    if (e < k3)
        for (int m = wq; m < M; m += 8) y += yb[(size_t)m * k3 + e];
    sl[wq][lane] = y;
    __syncthreads();
    if (wq == 0) {
        double t = 0.0;
        for (int w8 = 0; w8 < 8; ++w8) t += sl[w8][lane];
        double acc = t * t;
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) part[(size_t)b * gridDim.y + q] = acc;
    }
}

__global__ void k_pilot_reduce(int nq, const double* part, double* dv) {
    const int b = blockIdx.x, lane = threadIdx.x;
    double acc = 0.0;
    for (int q = lane; q < nq; q += 32) acc += part[(size_t)b * nq + q];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) dv[4 * b + 1] = sqrt(acc);
}

// ------------------------------------------------------------------ schedule
// Block per tree.  dv[4b]: ||f_b||^2, dv[4b+1]: sigma_b; writes eta_b to
// dv[4b+2] and the tree's schedule at sched + b * sl, laid out (int32)
//   Jm[M] | m1[lm*4] | m2[lm*4] | cnt[lm*4*2]   (sl = M + 16 lm)
// Levels at or beyond the tree's own depth get empty ranges.
__global__ void k_schedule(int M, int lm, const int32_t* nlev_tab, int unscreened, double eps, const double* w,
                           const double* nF, const double* est, double* dv, int32_t* sched_all, int sl) {
    const int b = blockIdx.x;
    const int nlev = nlev_tab ? nlev_tab[b] : lm;
    int32_t* Jm = sched_all + (size_t)b * sl;
    int32_t* m1 = Jm + M;
    int32_t* m2 = m1 + lm * 4;
    int32_t* cnt = m2 + lm * 4;
    // shared copies of J_m, w_m and, per level, the core / off-core maxima of
    // the 1-D block norms, so the serial range scans below read shared memory
    extern __shared__ double sched_sm[];
    double* ws = sched_sm;                        // M
    double* cmax = ws + M;                        // lm * M: max over |l| <= 1
    double* bmax = cmax + (size_t)lm * M;         // lm * M: max over |l| >= 2
    double* ev = bmax + (size_t)lm * M;           // lm * 4 * M: the bound e_m per (j, S)
    int* Js = (int*)(ev + (size_t)lm * 4 * M);    // M
    const double fn = sqrt(dv[4 * b]);
    const double eta = fn > 0.0 ? eps * dv[4 * b + 1] / fn : 0.0;
    if (threadIdx.x == 0) dv[4 * b + 2] = eta;
    for (int m = threadIdx.x; m < M; m += blockDim.x) {
        int jm = 0;
        if (unscreened) jm = nlev - 1;
        else
            for (int j = 1; j < nlev; ++j)
                if (w[m] * est[(size_t)j * M + m] > eta / M) jm = j;
        Jm[m] = jm;
        Js[m] = jm;
        ws[m] = w[m];
    }
    for (int e = threadIdx.x; e < nlev * M; e += blockDim.x) {
        const double* r = nF + (size_t)e * 7;  // e = j * M + m
        cmax[e] = fmax(fmax(r[2], r[3]), r[4]);
        bmax[e] = fmax(fmax(r[0], r[1]), fmax(r[5], r[6]));
    }
    __syncthreads();
    // the bounds e_m = w_m cmax^S bmax^(3-S) of every (j, S, m) at once (the serial
    // scans below then only add); a term with J_m < j gets 0, which the scans pass over
    // exactly as they skip it (acc + 0 <= budget holds while acc <= budget)
    for (int e = threadIdx.x; e < lm * 4 * M; e += blockDim.x) {
        const int js = e / M, m = e - js * M, j = js >> 2, S = js & 3;
        double v = 0.0;
        if (j < nlev && Js[m] >= j) {
            const double c = cmax[(size_t)j * M + m], bb = bmax[(size_t)j * M + m];
            v = ws[m];
            for (int q = 0; q < S; ++q) v *= c;
            for (int q = S; q < 3; ++q) v *= bb;
        }
        ev[e] = v;
    }
    __syncthreads();
    const double budget = eta / (2.0 * 216.0);
    for (int js = threadIdx.x; js < lm * 4; js += blockDim.x) {
        const int j = js / 4, S = js % 4;
        int lo_m = 0, hi_m = -1;
        if (unscreened) {
            lo_m = 0;
            hi_m = M - 1;
        } else {
            // candidates: terms with J_m >= j, in increasing m
            int first = -1, last = -1, n = 0;
            for (int m = 0; m < M; ++m)
                if (Js[m] >= j) {
                    if (first < 0) first = m;
                    last = m;
                    ++n;
                }
            if (n > 0) {
                const double* e_js = ev + (size_t)js * M;
                double acc = 0.0;
                int lo = first;
                for (; lo <= last; ++lo) {
                    const double e = e_js[lo];
                    if (acc + e <= budget) acc += e;
                    else break;
                }
                acc = 0.0;
                int hi = last;
                for (; hi >= lo; --hi) {
                    const double e = e_js[hi];
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
                if (Js[m] < j) continue;
                if (ci && S == 3 && Js[m] > j) continue;
                ++c;
            }
            cnt[js * 2 + ci] = c;
        }
    }
}

static size_t schedule_smem(int M, int lm) { return ((size_t)M * (1 + 6 * (size_t)lm)) * sizeof(double) + M * sizeof(int); }

static int schedule_smem_attr(int M, int lm) {
    MRA_CK(cudaFuncSetAttribute(k_schedule, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)schedule_smem(M, lm)));
    return MRA_OK;
}

// ------------------------------------------------------------------ screen
#define GH_EMPTY 0xffffffffffffffffull
#define GH_TREE_BITS 22

// level (6 bits) | tree (22 bits) | Morton key of the box (36 bits, level <= 12)
__device__ inline uint64_t ghost_key(int j, int tree, int b1, int b2, int b3) {
    return ((uint64_t)j << 58) | ((uint64_t)tree << 36) | morton3(b1, b2, b3);
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

// The Step-2 set is keyed by the missing box's parent: slot -> parent key, an
// 8-bit mask of the octants needed, and (after k_ghost_ids) the id of the
// parent's first needed child.  A group's children get consecutive ids in
// octant order, so no sort is needed to find siblings.
struct ScreenArgs {
    Forest F;
    int M, sl;
    const int32_t* sched;  // per tree: Jm | m1 | m2 | cnt
    uint64_t* gtab;
    uint32_t gcap;
    uint32_t* gmask;       // slot -> octants needed (count pass)
    const int32_t* gid;    // slot -> id of its first needed child (fill pass)
    int32_t* count;        // per node pair count (count pass)
    const int32_t* pair_off;
    Pair* pairs;
    int32_t* err;          // [0] hash overflow
    // [n][216] (optional): the count pass's lookup per band position -- the input node,
    // or -1 - slot of the missing box's parent in the Step-2 set -- so that the fill
    // pass searches nothing
    int32_t* qin;
};

// warp per output node; lane q covers band positions q, q+32, ... < 216
template <bool FILL>
__global__ void k_screen(ScreenArgs A) {
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const int lm = A.F.lm;
    for (int i = warp; i < A.F.n; i += nwarps) {
        const int b = forest_tree(A.F, i);
        const int32_t* m1 = A.sched + (size_t)b * A.sl + A.M;
        const int32_t* m2 = m1 + lm * 4;
        const int32_t* cnt = m2 + lm * 4;
        const int32_t* off = A.F.off + b * (lm + 1);
        const int j = A.F.coord[4 * i], a1 = A.F.coord[4 * i + 1], a2 = A.F.coord[4 * i + 2],
                  a3 = A.F.coord[4 * i + 3];
        const int leaf = A.F.leaf[i];
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
                        const uint32_t oct = ((b1 & 1) << 2) | ((b2 & 1) << 1) | (b3 & 1);
                        int32_t* qc = A.qin ? A.qin + (size_t)i * 216 + q : nullptr;
                        if (FILL && qc) {
                            const int32_t c = *qc;
                            if (c >= 0) in = c;
                            else {
                                const int slot = -1 - c;
                                in = -1 - (A.gid[slot] + __popc(A.gmask[slot] & ((1u << oct) - 1u)));
                            }
                        } else {
                            int idx = find_key_exact(A.F.key, off[j], off[j + 1], morton3(b1, b2, b3));
                            if (idx >= 0) {
                                in = idx;
                                if (qc) *qc = idx;
                            } else {
                                // keyed by the parent box (the child's level j is kept in the key)
                                const uint64_t pk = ghost_key(j, b, b1 >> 1, b2 >> 1, b3 >> 1);
                                if (!FILL) {
                                    const int slot = ghost_insert(A.gtab, A.gcap, pk);
                                    if (slot < 0) atomicExch(A.err, 1);
                                    else atomicOr(&A.gmask[slot], 1u << oct);
                                    if (qc) *qc = -1 - (slot < 0 ? 0 : slot);
                                } else {
                                    const int slot = ghost_find(A.gtab, A.gcap, pk);
                                    in = slot >= 0 ? -1 - (A.gid[slot] + __popc(A.gmask[slot] & ((1u << oct) - 1u)))
                                                   : 0;
                                    if (slot < 0) atomicExch(A.err, 2);
                                }
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

// ids: each parent slot takes popc(mask) consecutive ids (the order of the slots is
// whatever the atomic gives; every refined block is computed from its own key, so
// the results do not depend on it)
__global__ void k_ghost_ids(const uint64_t* tab, uint32_t cap, const uint32_t* gmask, int32_t* gid, int32_t* ng) {
    for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < cap; s += gridDim.x * blockDim.x)
        if (tab[s] != GH_EMPTY) gid[s] = atomicAdd(ng, __popc(gmask[s]));
}

// the children's keys (level | tree | Morton key of the child) at their ids
__global__ void k_ghost_keys(const uint64_t* tab, uint32_t cap, const uint32_t* gmask, const int32_t* gid,
                             uint64_t* gkeys) {
    const uint64_t lo36 = (1ull << 36) - 1;
    for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < cap; s += gridDim.x * blockDim.x) {
        const uint64_t pk = tab[s];
        if (pk == GH_EMPTY) continue;
        const uint32_t mk = gmask[s];
        int id = gid[s];
        for (uint32_t o = 0; o < 8; ++o)
            if ((mk >> o) & 1u) gkeys[id++] = (pk & ~lo36) | (((pk & lo36) << 3) | o);
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
__global__ void k_ghost_refine(Forest F, const uint64_t* gkeys, double* gblk, int32_t* err) {
    extern __shared__ double sm[];
    const int k = F.k, k3 = k * k * k, kk = k * k;
    double* HT = sm;             // 2 k x k: HT[p][a][i] = H^(p)[i][a]
    double* x = HT + 2 * kk;
    double* y = x + k3;
    double* z = y + k3;
    const uint64_t gk = gkeys[blockIdx.x];
    const int j = (int)(gk >> 58);
    const int tree = (int)((gk >> 36) & ((1ull << GH_TREE_BITS) - 1));
    const uint64_t mk = gk & ((1ull << 36) - 1);
    const int b1 = compact1by2(mk >> 2), b2 = compact1by2(mk >> 1), b3 = compact1by2(mk);
    const int32_t* off = F.off + tree * (F.lm + 1);
    for (int e = threadIdx.x; e < 2 * kk; e += blockDim.x) {
        int p = e / kk, r = e % kk, a = r / k, i = r % k;
        HT[e] = F.filt[p * kk + i * k + a];
    }
    __shared__ int anc, jj;
    if (threadIdx.x == 0) {
        anc = -1;
        for (int lv = j - 1; lv >= 0 && anc < 0; --lv) {
            int sh = j - lv;
            int idx = find_key_exact(F.key, off[lv], off[lv + 1], morton3(b1 >> sh, b2 >> sh, b3 >> sh));
            if (idx >= 0) {
                anc = idx;
                jj = lv;
            }
        }
        if (anc < 0 || !F.leaf[anc]) atomicExch(err, 3);
    }
    __syncthreads();
    if (anc < 0) return;
    for (int e = threadIdx.x; e < k3; e += blockDim.x) x[e] = F.s[(size_t)anc * k3 + e];
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


// out = Mat along dimension `dim` of the k^3 array x (Mat k x k, out[c] = sum_i Mat[c][i] x[i]),
// generic k (row-major k^3 arrays, one output element per thread)
template <typename T>
__device__ void mode_mul(int k, const T* Mat, const T* x, T* out, int dim) {
    const int k3 = k * k * k, kk = k * k;
    for (int idx = threadIdx.x; idx < k3; idx += blockDim.x) {
        const int i1 = idx / kk, i2 = (idx / k) % k, i3 = idx % k;
        const int c = dim == 0 ? i1 : (dim == 1 ? i2 : i3);
        const int st = dim == 0 ? kk : (dim == 1 ? k : 1);
        const T* src = x + idx - c * st;
        T a = 0;
        for (int i = 0; i < k; ++i) a += Mat[c * k + i] * src[i * st];
        out[idx] = a;
    }
    __syncthreads();
}

// The same for k = K fixed at compile time on (K, K, K) arrays whose innermost
// extent is padded to K + 1 (so that fibers along it, one per thread, hit
// distinct banks), for upper-triangular Mat: the refinement matrices H^(p)T and
// their products vanish below the diagonal (H^(p)_{ia} = 0 for a > i, since
// phi_i((u + p)/2) is a polynomial of degree i), so out[c] sums i >= c only.
template <int K, typename T>
__device__ __forceinline__ void mode_mul_tri(const T* Mat, const T* x, T* out, int dim) {
    constexpr int P1 = K + 1, S0 = K * P1;
    const int sf = dim == 0 ? S0 : (dim == 1 ? P1 : 1);             // along the fiber
    const int sa = dim == 0 ? P1 : S0, sb = dim == 2 ? P1 : 1;        // the other two coordinates
    for (int f = threadIdx.x; f < K * K; f += blockDim.x) {
        const int a = f / K, b = f - a * K;
        const T* src = x + a * sa + b * sb;
        T v[K];
#pragma unroll
        for (int i = 0; i < K; ++i) v[i] = src[i * sf];
        T* dst = out + a * sa + b * sb;
#pragma unroll
        for (int c = 0; c < K; ++c) {
            T acc = 0;
#pragma unroll
            for (int i = c; i < K; ++i) acc += Mat[c * K + i] * v[i];
            dst[c * sf] = acc;
        }
    }
    __syncthreads();
}

// Step 2 by sibling groups.  The children of one parent box have consecutive ids
// (k_ghost_ids / k_ghost_keys); the block of a group's first ghost refines the
// ancestor leaf to the parent (the path's per-direction two-scale matrices
// multiplied first, then one three-mode product), then every child of the
// group, sharing the direction-3 and direction-2 partial products among the
// children (d = 0 half of eqs. recon_even / recon_odd).
// T = double, or float where the blocks only feed FP16 hi/lo tensor-core operands.
// KT > 0: k fixed at compile time, padded arrays and triangular contractions.
template <int KT, typename T>
__global__ void k_ghost_refine_groups(Forest F, int ng, const uint64_t* gkeys, double* gblk, int32_t* err) {
    extern __shared__ double sm_raw[];
    T* sm = (T*)sm_raw;
    const int k = KT ? KT : F.k, k3 = k * k * k, kk = k * k;
    const int bs = KT ? KT * KT * (KT + 1) : k3;  // one block's footprint in shared memory
    const int g0 = blockIdx.x;
    const uint64_t key0 = gkeys[g0];
    if (g0 > 0 && (gkeys[g0 - 1] >> 3) == (key0 >> 3)) return;  // not the first child of its group
    T* HT = sm;                // 2 k x k: HT[p][a][i] = H^(p)[i][a]
    T* P = HT + 2 * kk;        // 3 k x k: the path matrices per direction
    T* Q = P + 3 * kk;         // 3 k x k: scratch
    T* x = Q + 3 * kk;         // 1 block: the parent
    T* y = x + bs;             // 2 blocks: direction 3 by p3
    T* z = y + 2 * bs;         // 4 blocks: direction 2 by (p2, p3)
    T* w = z + 4 * bs;         // 1 block
    auto at = [&](int e) { return KT ? (e / KT) * (KT + 1) + e % KT : e; };  // element e of a block
    auto mm = [&](const T* Mat, const T* in, T* out, int dim) {
        if (KT) mode_mul_tri<KT ? KT : 1, T>(Mat, in, out, dim);
        else mode_mul<T>(k, Mat, in, out, dim);
    };
    const int j = (int)(key0 >> 58);
    const int tree = (int)((key0 >> 36) & ((1ull << GH_TREE_BITS) - 1));
    const uint64_t mk = key0 & ((1ull << 36) - 1);
    const int b1 = compact1by2(mk >> 2) >> 1, b2 = compact1by2(mk >> 1) >> 1, b3 = compact1by2(mk) >> 1;  // parent
    const int jp = j - 1;
    const int32_t* off = F.off + tree * (F.lm + 1);
    for (int e = threadIdx.x; e < 2 * kk; e += blockDim.x) {
        int p = e / kk, r = e % kk, a = r / k, i = r % k;
        HT[e] = (T)F.filt[p * kk + i * k + a];
    }
    __shared__ int anc, jj, gn;
    if (threadIdx.x == 0) {
        int n = 1;
        while (g0 + n < ng && n < 8 && (gkeys[g0 + n] >> 3) == (key0 >> 3)) ++n;
        gn = n;
        anc = -1;
        for (int lv = jp; lv >= 0 && anc < 0; --lv) {
            const int sh = jp - lv;
            const int idx = find_key_exact(F.key, off[lv], off[lv + 1], morton3(b1 >> sh, b2 >> sh, b3 >> sh));
            if (idx >= 0) {
                anc = idx;
                jj = lv;
            }
        }
        if (anc < 0 || !F.leaf[anc]) atomicExch(err, 3);
    }
    __syncthreads();
    if (anc < 0) return;
    for (int e = threadIdx.x; e < k3; e += blockDim.x) x[at(e)] = (T)F.s[(size_t)anc * k3 + e];
    if (jj < jp) {
        // P_d = H^(p_last)T ... H^(p_first)T along the path ancestor -> parent
        const int bd[3] = {b1, b2, b3};
        for (int e = threadIdx.x; e < 3 * kk; e += blockDim.x) {
            const int d = e / kk, r = e % kk;
            P[e] = HT[((bd[d] >> (jp - jj - 1)) & 1) * kk + r];
        }
        __syncthreads();
        for (int lv = jj + 1; lv < jp; ++lv) {
            for (int e = threadIdx.x; e < 3 * kk; e += blockDim.x) {
                const int d = e / kk, a = (e % kk) / k, i = e % k;
                const T* H = HT + ((bd[d] >> (jp - lv - 1)) & 1) * kk;
                T acc = 0;
                for (int c = 0; c < k; ++c) acc += H[a * k + c] * P[d * kk + c * k + i];
                Q[e] = acc;
            }
            __syncthreads();
            for (int e = threadIdx.x; e < 3 * kk; e += blockDim.x) P[e] = Q[e];
            __syncthreads();
        }
        mm(P + 2 * kk, x, y, 2);
        mm(P + kk, y, z, 1);
        mm(P, z, x, 0);
    } else {
        __syncthreads();
    }
    // the children: direction 3 for p3 = 0, 1; direction 2 for (p2, p3); direction 1 per child
    mm(HT, x, y, 2);
    mm(HT + kk, x, y + bs, 2);
    for (int q = 0; q < 4; ++q) mm(HT + (q >> 1) * kk, y + (q & 1) * bs, z + q * bs, 1);
    for (int g = 0; g < gn; ++g) {
        const uint64_t cm = gkeys[g0 + g] & 7ull;  // octant (p1 p2 p3) of the child
        const int p1 = (int)(cm >> 2) & 1, p23 = (int)(cm & 3);
        mm(HT + p1 * kk, z + p23 * bs, w, 0);
        for (int e = threadIdx.x; e < k3; e += blockDim.x) gblk[(size_t)(g0 + g) * k3 + e] = (double)w[at(e)];
        __syncthreads();
    }
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
        const int32_t* Jm = A.Jm + (A.node_tree ? A.node_tree[i] * A.jm_stride : 0);
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
                const int jm = Jm[m];
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
        if (threadIdx.x == 0 && A.n_items) atomicAdd(A.n_items + (A.node_tree ? A.node_tree[i] : 0), items);
        __syncthreads();
    }
}

// ------------------------------------------------------------------ driver
void screen_release(const Alloc& A, ScreenOut* S) {
    A.put(S->dv); A.put(S->sched); A.put(S->count); A.put(S->pair_off); A.put(S->total); A.put(S->err);
    A.put(S->gtab); A.put(S->gid); A.put(S->gmask); A.put(S->gkeys); A.put(S->pairs);
    *S = ScreenOut();
}

// Pilot, schedule and the two-pass warp screen over a forest, with the one
// host synchronisation that sizes the worklist.  The ghost hash set starts at
// 64 slots per node; when a probe sequence reaches its limit the count pass
// is redone with a set four times larger.
int screen_forest(const mra_op* op, const Forest& F, int unscreened, const Alloc& A, cudaStream_t st, ScreenOut* S) {
    const int k3 = F.k * F.k * F.k, M = op->M, n = F.n;
    *S = ScreenOut();
    S->sl = M + 16 * F.lm;
    MRA_TRY(dalloc(A, &S->dv, 4 * (size_t)F.ntrees));
    MRA_TRY(dalloc(A, &S->sched, (size_t)F.ntrees * S->sl));
    MRA_TRY(dalloc(A, &S->count, (size_t)n + 1));
    MRA_TRY(dalloc(A, &S->pair_off, (size_t)n + 1));
    MRA_TRY(dalloc(A, &S->total, 2));
    MRA_TRY(dalloc(A, &S->err, 2));
    MRA_CK(cudaMemsetAsync(S->dv, 0, 4 * (size_t)F.ntrees * sizeof(double), st));
    MRA_CK(cudaMemsetAsync(S->err, 0, 2 * sizeof(int32_t), st));
    const int nb_norm = (int)std::max<long>(1, std::min<long>(num_sms() * 16, ((long)n * 32 + 255) / 256));
    k_forest_norm2<<<nb_norm, 256, 0, st>>>(F, S->dv);
    MRA_CK_LAUNCH();
    Scratch tmp(A);
    double *ym, *part;
    const int nq = (k3 + 31) / 32;
    MRA_TRY(tmp.get(&ym, (size_t)F.ntrees * M * k3));
    MRA_TRY(tmp.get(&part, (size_t)F.ntrees * nq));
    k_pilot_terms<<<dim3(M, F.ntrees), 128, (3 * (size_t)k3 + F.k * F.k) * sizeof(double), st>>>(F, M, op->w, op->F, ym);
    MRA_CK_LAUNCH();
    k_pilot_partial<<<dim3(F.ntrees, nq), 256, 0, st>>>(k3, M, ym, part);
    MRA_CK_LAUNCH();
    k_pilot_reduce<<<F.ntrees, 32, 0, st>>>(nq, part, S->dv);
    MRA_CK_LAUNCH();
    MRA_TRY(schedule_smem_attr(M, F.lm));
    k_schedule<<<F.ntrees, 256, schedule_smem(M, F.lm), st>>>(M, F.lm, F.nlev, unscreened, op->eps, op->w, op->nF,
                                                              op->est, S->dv, S->sched, S->sl);
    MRA_CK_LAUNCH();

    ScreenArgs sa;
    sa.F = F; sa.M = M; sa.sl = S->sl; sa.sched = S->sched;
    sa.count = S->count; sa.pair_off = S->pair_off; sa.pairs = nullptr; sa.err = S->err;
    // the count pass's lookups, kept for the fill pass (when they take at most 1 GiB)
    sa.qin = nullptr;
    if ((size_t)n * 216 * sizeof(int32_t) <= ((size_t)1 << 30)) MRA_TRY(tmp.get(&sa.qin, (size_t)n * 216));
    const int sblocks = (int)std::max<long>(1, std::min<long>(num_sms() * 32, ((long)n * 32 + 255) / 256));
    // parents of missing boxes: 16 slots per node to start (a box's band has at most
    // 27 parent boxes, shared with its neighbours), regrown x4 on a probe overflow
    uint64_t cap = 1024;
    while (cap < (uint64_t)n * 16ull) cap <<= 1;
    int32_t h[2] = {0, 0}, herr[2] = {0, 0};
    for (;;) {
        if (cap > (1ull << 30)) { set_error("ghost hash set overflow"); return MRA_ECUDA; }
        S->gcap = (uint32_t)cap;
        MRA_TRY(dalloc(A, &S->gtab, cap));
        MRA_TRY(dalloc(A, &S->gid, cap));
        MRA_TRY(dalloc(A, &S->gmask, cap));
        MRA_CK(cudaMemsetAsync(S->total, 0, 2 * sizeof(int32_t), st));
        MRA_CK(cudaMemsetAsync(S->gmask, 0, cap * sizeof(uint32_t), st));
        k_fill_u64<<<1024, 256, 0, st>>>(S->gtab, cap, GH_EMPTY);
        MRA_CK_LAUNCH();
        sa.gtab = S->gtab; sa.gcap = S->gcap; sa.gid = S->gid; sa.gmask = S->gmask;
        k_screen<false><<<sblocks, 256, 0, st>>>(sa);
        MRA_CK_LAUNCH();
        MRA_TRY(scan_exclusive(S->count, S->pair_off, n, S->total, st));
        MRA_CK(cudaMemcpyAsync(S->pair_off + n, S->total, sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
        k_ghost_ids<<<1024, 256, 0, st>>>(S->gtab, S->gcap, S->gmask, S->gid, S->total + 1);
        MRA_CK_LAUNCH();
        // the one host synchronisation: pair and ghost counts size the worklist
        MRA_CK(cudaMemcpyAsync(h, S->total, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        MRA_CK(cudaMemcpyAsync(herr, S->err, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        MRA_CK(cudaStreamSynchronize(st));
        if (!herr[0]) break;
        A.put(S->gtab); A.put(S->gid); A.put(S->gmask);
        S->gtab = nullptr; S->gid = nullptr; S->gmask = nullptr;
        MRA_CK(cudaMemsetAsync(S->err, 0, 2 * sizeof(int32_t), st));
        cap <<= 2;
    }
    S->npairs = h[0];
    S->nghost = h[1];
    // the children's keys at their ids: siblings (children of one parent box) are consecutive
    MRA_TRY(dalloc(A, &S->gkeys, (size_t)S->nghost + 1));
    if (S->nghost > 0) {
        k_ghost_keys<<<1024, 256, 0, st>>>(S->gtab, S->gcap, S->gmask, S->gid, S->gkeys);
        MRA_CK_LAUNCH();
    }
    MRA_TRY(dalloc(A, &S->pairs, (size_t)S->npairs + 1));
    sa.pairs = S->pairs;
    k_screen<true><<<sblocks, 256, 0, st>>>(sa);
    MRA_CK_LAUNCH();
    return MRA_OK;
}

template <typename T>
static int ghost_refine_launch(const Forest& F, const ScreenOut& S, double* gblk, cudaStream_t st) {
    const int k = F.k, k3 = k * k * k;
    const size_t gsm = (8 * (size_t)k * k + 8 * (size_t)k * k * (k + 1)) * sizeof(T);  // padded blocks
    auto fn = k == 8 ? k_ghost_refine_groups<8, T> : (k == 6 ? k_ghost_refine_groups<6, T> :
                                                    (k == 4 ? k_ghost_refine_groups<4, T> : k_ghost_refine_groups<0, T>));
    MRA_CK(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gsm));
    fn<<<S.nghost, 128, gsm, st>>>(F, S.nghost, S.gkeys, gblk, S.err + 1);
    MRA_CK_LAUNCH();
    return MRA_OK;
}

int ghost_refine_forest(const Forest& F, const ScreenOut& S, double* gblk, cudaStream_t st, bool fp32) {
    if (S.nghost <= 0) return MRA_OK;
    return fp32 ? ghost_refine_launch<float>(F, S, gblk, st) : ghost_refine_launch<double>(F, S, gblk, st);
}

// Precision ladder budget per tree: single-FP16 terms may add at most
// eps sigma_b / (4 sqrt(N_b)) of rounding error to any node of tree b, so
// over its N_b nodes at most eps sigma_b / 4 in the L2 norm (sigma_b =
// ||T_0 f_0||, the pilot of ||g||).
__global__ void k_lp_budget(Forest F, const double* dv, double eps, double* lpb) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < F.ntrees; b += gridDim.x * blockDim.x) {
        const int nb = F.off[b * (F.lm + 1) + F.lm] - F.off[b * (F.lm + 1)];
        lpb[b] = eps * dv[4 * b + 1] / (4.0 * sqrt((double)(nb > 0 ? nb : 1)));
    }
}

int lp_budget(const Forest& F, const ScreenOut& S, double eps, double* lpb, cudaStream_t st) {
    k_lp_budget<<<(F.ntrees + 127) / 128, 128, 0, st>>>(F, S.dv, eps, lpb);
    MRA_CK_LAUNCH();
    return MRA_OK;
}

Forest forest_of_tree(const mra_tree* f) {
    Forest F;
    F.k = f->k; F.ntrees = 1; F.n = f->n; F.lm = f->nlev;
    F.coord = f->a.coord; F.leaf = f->a.leaf; F.key = f->a.key; F.off = f->a.off;
    F.node_tree = nullptr; F.nlev = nullptr; F.s = f->s; F.filt = f->filt;
    return F;
}

int apply_impl(const mra_op* op, const mra_tree* f, const mra_apply_opts* o, cudaStream_t st, mra_tree** gout,
               mra_apply_stats* stats) {
    const int k = op->k, k3 = k * k * k, M = op->M, n = f->n, nlev = f->nlev;
    if (f->k != k) { set_error("tree order k=%d differs from operator k=%d", f->k, k); return MRA_EINVAL; }
    if (nlev - 1 > op->J) { set_error("tree depth %d exceeds operator max_level %d", nlev - 1, op->J); return MRA_EINVAL; }
    if (f->state != MRA_TREE_REDUNDANT) { set_error("apply_ns needs a compressed (redundant) tree"); return MRA_ESTATE; }
    const int prec = o ? o->precision : MRA_PREC_FP64;
    if (prec != MRA_PREC_FP64 && prec != MRA_PREC_FP32 && prec != MRA_PREC_TC_SPLIT && prec != MRA_PREC_TC_LADDER &&
        prec != MRA_PREC_TC_FAST) {
        set_error("precision %d is not available", prec);
        return MRA_EINVAL;
    }
    const bool tc = prec == MRA_PREC_TC_SPLIT || prec == MRA_PREC_TC_LADDER || prec == MRA_PREC_TC_FAST;
    if (o && (o->wait_limit < 0 || (o->test_flags & ~MRA_TEST_WITHHOLD_MMA))) {
        set_error("wait_limit must be >= 0 and test_flags a set of MRA_TEST_* bits");
        return MRA_EINVAL;
    }
    if (tc && ((o && (o->block_screen || o->itemwise)) || k > 8)) {
        set_error("the tensor-core apply needs k <= 8 and the static screen");
        return MRA_EINVAL;
    }
    const Alloc& A = f->A;
    // everything below is released on every return path; the output tree only
    // when the call fails
    struct Guard {
        const Alloc& A;
        ScreenOut S;
        void* p[4] = {nullptr, nullptr, nullptr, nullptr};
        cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
        mra_tree* g = nullptr;
        explicit Guard(const Alloc& a) : A(a) {}
        ~Guard() {
            screen_release(A, &S);
            for (void* q : p) A.put(q);
            for (cudaEvent_t e : ev)
                if (e) cudaEventDestroy(e);
            if (g) mra_free_tree(g);
        }
    } G(A);
    cudaEvent_t* ev = G.ev;
    for (int e = 0; e < 4; ++e) MRA_CK(cudaEventCreate(&ev[e]));
    MRA_CK(cudaEventRecord(ev[0], st));

    const Forest F = forest_of_tree(f);
    ScreenOut& S = G.S;
    const int unscreened = o ? o->unscreened : 0;
    int rc = MRA_OK;
    MRA_TRY(screen_forest(op, F, unscreened, A, st, &S));
    MRA_CK(cudaEventRecord(ev[1], st));
    double* gblk;
    MRA_TRY(dalloc(A, &gblk, (size_t)(S.nghost + 1) * k3));
    G.p[0] = gblk;
    // per-pair term ranges: the exact screen, or the learned one judged by it
    const int smode = o ? o->screen_mode : MRA_SCREEN_STATIC;
    // Step 2 in FP64 (a two-scale transform); MRA_PREC_TC_FAST refines in FP32 when the
    // blocks only become FP16 hi/lo operands (rounding 2^-24, below the operands' 2^-22)
    // and no screen decision reads them
    MRA_TRY(ghost_refine_forest(F, S, gblk, st, prec == MRA_PREC_TC_FAST && smode == MRA_SCREEN_STATIC));
    unsigned long long* scounts = nullptr;
    if (smode != MRA_SCREEN_STATIC) {
        if (smode != MRA_SCREEN_PAIR && smode != MRA_SCREEN_LEARNED) {
            set_error("screen mode %d is not available", smode);
            return MRA_EINVAL;
        }
        MRA_TRY(dalloc(A, &scounts, 2));
        G.p[1] = scounts;
        MRA_CK(cudaMemsetAsync(scounts, 0, 2 * sizeof(unsigned long long), st));
        MRA_TRY(schedule_narrow(op, F, S, gblk, smode, o->schedule, std::max(0, o->margin), nullptr, nullptr,
                                scounts, A, st));
    }
    MRA_CK(cudaEventRecord(ev[2], st));

    MRA_TRY(tree_clone_skeleton(f, &G.g));
    mra_tree* g = G.g;
    g->state = MRA_TREE_NSFORM;
    unsigned long long* nitems;  // [0] items, [1] items with single FP16 operands
    MRA_TRY(dalloc(A, &nitems, 2));
    G.p[2] = nitems;
    MRA_CK(cudaMemsetAsync(nitems, 0, 2 * sizeof(unsigned long long), st));
    double* lpb = nullptr;

    ApplyArgs aa;
    aa.k = k; aa.M = M; aa.n = n; aa.pairs = S.pairs; aa.pair_off = S.pair_off; aa.coord = f->a.coord;
    aa.s = f->s; aa.gblk = gblk; aa.w = op->w; aa.nF = op->nF; aa.Jm = S.sched; aa.out = g->s; aa.n_items = nitems;
    aa.eta_blk = -1.0;
    if (o && o->block_screen) {
        // eps ||T_0 f_0|| / sqrt(N 216 M), evaluated on the host from the device sigma
        double sig = 0.0;
        MRA_CK(cudaMemcpyAsync(&sig, S.dv + 1, sizeof(double), cudaMemcpyDeviceToHost, st));
        MRA_CK(cudaStreamSynchronize(st));
        aa.eta_blk = op->eps * sig / sqrt((double)n * 216.0 * M);
    }
    const bool itemwise = (o && o->itemwise) || aa.eta_blk >= 0.0;
    if (tc) {
        // tcgen05 FP16 hi/lo split products (apply_tc.cu); with the ladder,
        // single FP16 products for the terms the error budget allows
        if (prec == MRA_PREC_TC_LADDER) {
            MRA_TRY(dalloc(A, &lpb, 1));
            G.p[3] = lpb;
            MRA_TRY(lp_budget(F, S, op->eps, lpb, st));
        }
        MRA_TRY(launch_apply_tc(aa, S.nghost, op, S.err + 1, lpb, nitems + 1, o ? (unsigned)o->wait_limit : 0u,
                                o ? (o->test_flags & MRA_TEST_WITHHOLD_MMA) : 0, st));
    } else if (!itemwise) {
        // Algorithm 3's nested sums, factorised (apply_fact.cu)
        aa.F = prec == MRA_PREC_FP64 ? (const void*)op->F : (const void*)op->F32;
        MRA_TRY(launch_apply_fact(aa, prec, st));
    } else if (prec == MRA_PREC_FP64) {
        aa.F = op->F;
        size_t smem = (size_t)k3 * sizeof(double) + (4 * (size_t)k3 + 3 * k * k) * sizeof(double);
        MRA_CK(cudaFuncSetAttribute(k_apply_simt<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_apply_simt<double><<<std::min(n, num_sms() * 16), 128, smem, st>>>(aa);
        MRA_CK_LAUNCH();
    } else {
        aa.F = op->F32;
        size_t smem = (size_t)k3 * sizeof(double) + (4 * (size_t)k3 + 3 * k * k) * sizeof(float);
        MRA_CK(cudaFuncSetAttribute(k_apply_simt<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_apply_simt<float><<<std::min(n, num_sms() * 16), 128, smem, st>>>(aa);
        MRA_CK_LAUNCH();
    }
    MRA_CK(cudaEventRecord(ev[3], st));

    if (stats) {
        unsigned long long ni[2] = {0, 0};
        double hv[3];
        int32_t herr[2] = {0, 0};
        MRA_CK(cudaMemcpyAsync(ni, nitems, sizeof(ni), cudaMemcpyDeviceToHost, st));
        MRA_CK(cudaMemcpyAsync(hv, S.dv, 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
        MRA_CK(cudaMemcpyAsync(herr, S.err, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        MRA_CK(cudaStreamSynchronize(st));
        stats->n_pairs = S.npairs;
        stats->n_items = (int64_t)ni[0];
        stats->n_items_lowp = (int64_t)ni[1];
        unsigned long long sc[2] = {0, 0};
        if (scounts) {
            MRA_CK(cudaMemcpyAsync(sc, scounts, sizeof(sc), cudaMemcpyDeviceToHost, st));
            MRA_CK(cudaStreamSynchronize(st));
        }
        stats->n_misses = (int64_t)sc[0];
        stats->n_pairs_empty = (int64_t)sc[1];
        stats->n_ghosts = S.nghost;
        stats->n_out_nodes = n;
        stats->fnorm = sqrt(hv[0]);
        stats->sigma = hv[1];
        stats->eta = hv[2];
        cudaEventElapsedTime(&stats->ms_screen, ev[0], ev[1]);
        cudaEventElapsedTime(&stats->ms_ghost, ev[1], ev[2]);
        cudaEventElapsedTime(&stats->ms_apply, ev[2], ev[3]);
        if (herr[1] == 4) { set_error("tensor-core apply: an MMA completion wait reached its limit"); rc = MRA_ETIMEOUT; }
        else if (herr[1] == 5) { set_error("tensor-core apply: an output scale is outside the FP32 range (use fp64)"); rc = MRA_EINVAL; }
        else if (herr[0] || herr[1]) { set_error("screen/ghost error code %d/%d", herr[0], herr[1]); rc = MRA_ECUDA; }
    }
    if (rc != MRA_OK) return rc;  // the guard frees the output tree: *gout stays NULL
    G.g = nullptr;  // the caller owns the output from here
    *gout = g;
    return MRA_OK;
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
    size_t dv, sched, count, pair_off, total, err, gtab, gid, gmask, gkeys, pairs, gblk, nitems, bytes;
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
    L.gmask = o;    o = na_align(o + NA_HASH_CAP * sizeof(uint32_t));
    L.gkeys = o;    o = na_align(o + NA_MAX_GHOSTS * sizeof(uint64_t));
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
    uint32_t* gmask = (uint32_t*)(base + L.gmask);
    uint64_t* gkeys = (uint64_t*)(base + L.gkeys);
    Pair* pairs = (Pair*)(base + L.pairs);
    double* gblk = (double*)(base + L.gblk);
    unsigned long long* nitems = (unsigned long long*)(base + L.nitems);

    // the array keeps the previous call's contents: clear what must start at zero
    MRA_CK(cudaMemsetAsync(dv, 0, 4 * sizeof(double), st));
    MRA_CK(cudaMemsetAsync(total, 0, 2 * sizeof(int32_t), st));
    MRA_CK(cudaMemsetAsync(err, 0, 2 * sizeof(int32_t), st));
    MRA_CK(cudaMemsetAsync(nitems, 0, sizeof(unsigned long long), st));
    MRA_CK(cudaMemsetAsync(gmask, 0, NA_HASH_CAP * sizeof(uint32_t), st));
    k_fill_u64<<<64, 256, 0, st>>>(gtab, NA_HASH_CAP, GH_EMPTY);
    MRA_CK_LAUNCH();
    MRA_TRY(leaf_norm2(f, dv, st));
    const size_t pilot_smem = (4 * (size_t)k3 + k * k) * sizeof(double);
    k_pilot<<<1, 128, pilot_smem, st>>>(k, M, op->w, op->F, f->s, dv + 1);
    MRA_CK_LAUNCH();
    const int sl = M + 16 * nlev;
    MRA_TRY(schedule_smem_attr(M, nlev));
    k_schedule<<<1, 256, schedule_smem(M, nlev), st>>>(M, nlev, nullptr, 0, op->eps, op->w, op->nF, op->est, dv,
                                                       sched, sl);
    MRA_CK_LAUNCH();
    const Forest F = forest_of_tree(f);
    ScreenArgs sa;
    sa.F = F; sa.M = M; sa.sl = sl; sa.sched = sched;
    sa.gtab = gtab; sa.gcap = NA_HASH_CAP; sa.gid = gid; sa.gmask = gmask;
    sa.count = count; sa.pair_off = pair_off; sa.pairs = nullptr; sa.err = err; sa.qin = nullptr;
    const int sblocks = (int)std::min<long>(4096, ((long)n * 32 + 255) / 256);
    k_screen<false><<<sblocks, 256, 0, st>>>(sa);
    MRA_CK_LAUNCH();
    MRA_TRY(scan_exclusive(count, pair_off, n, total, st));
    MRA_CK(cudaMemcpyAsync(pair_off + n, total, sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
    k_ghost_ids<<<64, 256, 0, st>>>(gtab, NA_HASH_CAP, gmask, gid, total + 1);
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
        k_ghost_keys<<<64, 256, 0, st>>>(gtab, NA_HASH_CAP, gmask, gid, gkeys);
        MRA_CK_LAUNCH();
        const size_t gsm = (2 * (size_t)k * k + 3 * (size_t)k3) * sizeof(double);
        k_ghost_refine<<<nghost, 128, gsm, st>>>(F, gkeys, gblk, err + 1);
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
        k_apply_simt<double><<<std::min(n, num_sms() * 16), 128, smem, st>>>(aa);
        MRA_CK_LAUNCH();
    } else {
        aa.F = op->F32;
        size_t smem = (size_t)k3 * sizeof(double) + (4 * (size_t)k3 + 3 * k * k) * sizeof(float);
        k_apply_simt<float><<<std::min(n, num_sms() * 16), 128, smem, st>>>(aa);
        MRA_CK_LAUNCH();
    }
    // the device error words are always read back (a missed Step-2 lookup or a
    // refinement without an ancestor leaf leaves ghat wrong); the item count only
    // when asked for
    unsigned long long ni = 0;
    MRA_CK(cudaMemcpyAsync(&ni, nitems, sizeof(ni), cudaMemcpyDeviceToHost, st));
    MRA_CK(cudaMemcpyAsync(herr, err, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    MRA_CK(cudaStreamSynchronize(st));
    if (herr[0] || herr[1]) { set_error("screen/ghost error code %d/%d", herr[0], herr[1]); return MRA_ECUDA; }
    if (n_items_host) *n_items_host = (int64_t)ni;
    return MRA_OK;
}

}  // namespace mra
