// Step 3 of Algorithm 3 on the 5th-generation tensor cores (tcgen05), k <= 8
// (orders below 8 are zero-padded to 8).
//
// Same nested sums as apply_fact.cu, per output node a and chunk of MC terms
// m (w_m, F = F^{j;m,.}):
//   stage I   per (t2,t3) line: W_m[c1][(i2,i3)] = sum_{t1 kept} sum_i1 F^{t1}[c1][i1] x_t[i1][i2][i3]
//             MMA M=64 rows (i3,i2), N=8*MC (m,c1), K=48 (t1,i1); the kept-item
//             mask zeroes whole F^{t1} blocks of the B operand
//   stage II  per line and term: V_m[(c1,i3)][c2] += sum_i2 W_m[c1][i2][i3] F^{t2}[c2][i2]
//             MMA M=64, N=8, K=16 (i2 as hi | lo), accumulated over the plane's lines in TMEM
//   stage III per plane and term: Y_m[(c1,c2)][c3] += sum_i3 V_m F^{t3}[c3][i3]
//             MMA M=64, N=8, K=16 (i3 as hi | lo), read out after each plane
//   ghat_a += w_m Y_m: per plane, an FP32 sum over the chunk's terms, summed in FP32
//             over the chunk's planes; each chunk's sum is added to ghat in FP64 (one
//             FP64 add per chunk and output coefficient, none per item).
// Every operand is FP16 split into hi + lo (v ~= hi + lo to 2^-22), and each
// product is hi*hi + hi*lo + lo*hi into an FP32 accumulator: three MMAs in
// stage I; in stages II and III, whose contraction (8) fills half of an
// MMA's K = 16, two: A = [A_hi | A_lo] against [B_hi ; B_hi] and [B_lo ; 0].
// Power-of-two scales keep every operand in FP16's normal range: per input
// block (x * sx in [2^9, 2^13), sx a power of 16), per (j, m) operator block (F * sF), per node
// (sx_node = the smallest block scale of the neighbourhood), and per term for
// W and V from bounds (|W| <= 48 max|F| max|x|, |V| <= 48 max|F| max|W|).
//
// Five threads issue the MMAs (stage I; stages II/III for a quarter of the terms each)
// and commit them to one mbarrier; warp 0 polls it (bounded) and a block barrier
// releases the rest; the 256 threads read TMEM with tcgen05.ld (16x256b) and
// write the next stage's operand into shared memory in the no-swizzle K-major
// layout (8-row x 16-byte core matrices) with transposing stmatrix stores: the
// input blocks' rows are ordered (i3, i2), so that a warp's TMEM lane quarter
// holds all eight K values of the rows it stores.  The lines of a chunk form one
// software pipeline with one wait per line: stage II of line L and stage I of
// line L+1 go out under one commit, while line L+2's input blocks are copied.
// CTAs are persistent and take nodes from an atomic counter (optionally in a
// given order), so one launch can cover the nodes of many trees.
#include <cfloat>
#include <climits>

#include "apply_common.cuh"
#include "tc_ptx.cuh"

namespace mra {

#define TC_THREADS 256
// polls of one completion wait: the default, and the smallest accepted (far above the
// time one group of MMAs takes)
#define TC_WAIT_LIMIT (1u << 26)
#define TC_WAIT_MIN 4096u
// MMA-issuing threads (lane 0 of warps 0..TC_ISSUERS-1): warps 0-3 issue stages II and III
// for a quarter of a chunk's terms each, warp 4 issues stage I; each commits to the mbarrier
#define TC_ISSUERS 5
// first-order bound on the relative error of one item done with single FP16
// operands: six roundings to FP16 (x, W, V and the three F blocks, 2^-11
// each) plus FP32 accumulation, rounded up to 8 * 2^-11
#define LADDER_U 0.00390625

// ---------------------------------------------------------------- prep
// Input blocks -> FP16 hi/lo in the stage-I A layout: element x[i1][i2][i3]
// (zero for indices >= kr) at half index i3*64 + i2*8 + i1 (core matrix i3,
// row i2, column i1), with a power-of-two scale per block.  Block b is node b
// of s (b < n) or Step-2 block b - n.
#define PREP_WARPS 8
__global__ void __launch_bounds__(32 * PREP_WARPS) k_tc_prep_blocks(int nb, int kr, int n, const double* s,
                                                                  const double* gblk, __half* xh, __half* xl,
                                                                  float* sx, float* xmax, float* xnrm) {
    // warp per block: coalesced FP64 reads, each value rounded to FP32 once (the FP16
    // hi/lo pair keeps 22 bits of it; FP32 keeps 24), then FP32 arithmetic only -- the
    // part's FP64 rate is scarce; each lane writes the 8 values (i1 = 0..7) of two
    // (i3, i2) rows as one 16-byte hi and one 16-byte lo store
    __shared__ float xs[PREP_WARPS][512];
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const int k3 = kr * kr * kr;
    float* x = xs[wl];
    for (int b = blockIdx.x * PREP_WARPS + wl; b < nb; b += gridDim.x * PREP_WARPS) {
        const double* src = b < n ? s + (size_t)b * k3 : gblk + (size_t)(b - n) * k3;
        float s2 = 0.0f, m = 0.0f;
        for (int e = lane; e < k3; e += 32) {
            const float v = (float)src[e];
            x[e] = v;
            m = fmaxf(m, fabsf(v));
            s2 = fmaf(v, v, s2);
        }
        for (int o = 16; o > 0; o >>= 1) {
            m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
            s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        }
        __syncwarp();
        int e = 0;
        if (m > 0.0f) frexpf(m, &e);
        // m * scale in [2^9, 2^13): the exponent is rounded up to a multiple of 4,
        // so that neighbouring blocks mostly share a scale (and the stage-I B
        // operand can be reused from line to line); blocks below 2^-100 keep the
        // scale 2^113 (a finite float) and round to zero in FP16.  Scaling by a
        // power of two is exact.  (Values beyond FP32's range become infinite here;
        // the apply refuses them as outside the FP32 range.)
        const float scale = ldexpf(1.0f, 13 - ((max(e, -100) + 3) & ~3));
        for (int p = lane; p < 64; p += 32) {  // row (i3, i2) of the stage-I layout
            const int i3 = p >> 3, i2 = p & 7;
            uint4 h4, l4;
            __half* hh = (__half*)&h4;
            __half* ll = (__half*)&l4;
#pragma unroll
            for (int i1 = 0; i1 < 8; ++i1) {
                const float v = (i1 < kr && i2 < kr && i3 < kr) ? x[(i1 * kr + i2) * kr + i3] : 0.0f;
                tc::split_h(v * scale, hh[i1], ll[i1]);
            }
            ((uint4*)(xh + (size_t)b * 512))[p] = h4;
            ((uint4*)(xl + (size_t)b * 512))[p] = l4;
        }
        if (lane == 0) {
            sx[b] = scale;
            xmax[b] = m;
            xnrm[b] = sqrtf(s2);
        }
        __syncwarp();
    }
}

// Operator blocks F^{j;m,t}[c][i] (kr x kr) -> FP16 hi/lo 8 x 8 row-major
// (already the core-matrix layout of the B operands), zero-padded, with a
// power-of-two scale per (j, m).
__global__ void k_tc_prep_F(int M, int kr, const double* F, __half* Fh, __half* Fl, float* sF, float* maxF) {
    __shared__ float red[4];
    const int m = blockIdx.x, j = blockIdx.y;
    const double* src = F + ((size_t)j * M + m) * 7 * kr * kr;
    float mx = 0.0f;
    for (int e = threadIdx.x; e < 7 * kr * kr; e += blockDim.x) mx = fmaxf(mx, (float)fabs(src[e]));
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    mx = fmaxf(fmaxf(red[0], red[1]), fmaxf(red[2], red[3]));
    int ex = 0;
    if (mx > 0.0f) frexpf(mx, &ex);
    const double scale = ldexp(1.0, 13 - max(ex, -100));  // a finite float scale, as for the blocks
    for (int e = threadIdx.x; e < 7 * 64; e += blockDim.x) {
        const int t = e / 64, c = (e / 8) % 8, i = e % 8;
        const double v = (c < kr && i < kr) ? src[(t * kr + c) * kr + i] : 0.0;
        __half hi, lo;
        tc::split_h((float)(v * scale), hi, lo);
        Fh[((size_t)j * M + m) * 7 * 64 + e] = hi;
        Fl[((size_t)j * M + m) * 7 * 64 + e] = lo;
    }
    if (threadIdx.x == 0) {
        sF[(size_t)j * M + m] = (float)scale;
        maxF[(size_t)j * M + m] = mx;
    }
}

// shared-memory map (bytes) for MC terms per chunk; every operand region
// starts on a 128-byte boundary
template <int MC>
struct TcSmem {
    static constexpr int XH = 0;                    // 2 buffers x 6 blocks x 1 KB: stage I A (hi); the final y
    static constexpr int XL = 12288;                // (lo); buffer p at + p * 6144
    static constexpr int B1H = 24576;               // MC terms x 6 K groups x 128 B: stage I B
    static constexpr int B1L = B1H + MC * 768;
    // stage II A (K: hi | lo; stage III A aliases it): per term 8 groups of 8 rows, A2_SBO
    // bytes apart (272, not 256, so that the transposed stores of a group hit 32 banks)
    static constexpr int A2_SBO = 272;
    static constexpr int A2_TERM = 8 * A2_SBO;
    static constexpr int A2H = B1L + MC * 768;
    static constexpr int FSH = A2H + MC * A2_TERM;  // MC terms x 7 shifts x 128 B: the chunk's F (hi)
    static constexpr int FSL = FSH + MC * 896;      // (lo)
    static constexpr int FZ = FSL + MC * 896;       // one zero core matrix
    static constexpr int TIN = FZ + 128;            // 216 int: input block per band position
    static constexpr int TLO = TIN + 864;           // 216 int16: term range
    static constexpr int THI = TLO + 432;
    static constexpr int TFL = THI + 432;           // 216 bytes: flags
    static constexpr int TG = (TFL + 216 + 15) / 16 * 16;  // 216 float: g = sx_node / sx_b per band position
    static constexpr int MSK = TG + 864;            // 36 x MC bytes
    static constexpr int TOTAL = (MSK + 36 * MC + 127) / 128 * 128;
    // D_I and D_II (stage III's result reuses D_I's columns)
    static constexpr int TMEM_COLS = (16 * MC <= 64) ? 64 : ((16 * MC <= 128) ? 128 : 256);
};
// three CTAs per SM (the register limit) for either chunk size
static_assert(3 * (TcSmem<8>::TOTAL + 2048) <= 232448, "8 terms per chunk: three CTAs per SM");
static_assert(3 * TcSmem<8>::TMEM_COLS <= 512, "three CTAs' tensor memory");
static_assert(TcSmem<8>::MSK % 8 == 0 && TcSmem<4>::MSK % 4 == 0, "a line's masks are read as one word");

template <int MC, bool LADDER>
__global__ void __launch_bounds__(TC_THREADS, MC == 4 ? 4 : 3) k_apply_tc(TcArgs T) {
    using L = TcSmem<MC>;
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) uint64_t s_mbar;
    __shared__ int s_mlo, s_mhi, s_exp_min, s_node;
    __shared__ unsigned int s_xmax_bits;
    __shared__ unsigned long long s_items;
    __shared__ float s_c2[MC], s_c3[MC];
    __shared__ unsigned char s_lm[36];
    __shared__ unsigned char s_order[36];  // the chunk's lines with a kept item, as cursors
    __shared__ int s_nl;
    __shared__ unsigned long long s_kg[36];  // per line: the g exponents of its six blocks
    __shared__ float s_fin[MC];
    __shared__ int s_cnt[MC];
    __shared__ float s_B[MC];
    __shared__ unsigned char s_low[MC];
    __shared__ int s_all_low;
    __shared__ unsigned long long s_lowi;

    const ApplyArgs& A = T.A;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int kr = T.kr;
    __half* B1H = (__half*)(sm + L::B1H);
    __half* B1L = (__half*)(sm + L::B1L);
    // the operator blocks F (hi, lo) of term m at shift t: uint4 index ((j M + m) 7 + t + 3) 8
    const uint4* FH = (const uint4*)T.Fh;
    const uint4* FL = (const uint4*)T.Fl;
    int* tin = (int*)(sm + L::TIN);
    int16_t* tlo = (int16_t*)(sm + L::TLO);
    int16_t* thi = (int16_t*)(sm + L::THI);
    unsigned char* tfl = sm + L::TFL;
    float* tg = (float*)(sm + L::TG);
    unsigned char* msk = sm + L::MSK;
    // lines in (t3 plane, t2) order: cursor c = q3 * 6 + q2 names line q2 * 6 + q3
    auto line_of = [](int c) { return (c % 6) * 6 + c / 6; };
    // the MC mask bytes of a line as one word (byte mc = term mc's kept-t1 mask)
    auto line_masks = [&](int line) -> unsigned long long {
        if (MC == 8) return *(const unsigned long long*)(msk + line * 8);
        return *(const unsigned int*)(msk + line * MC);
    };

    // zero everything once: the zero core matrix FZ stays zero, and operand buffers that a
    // line leaves unwritten hold finite values (they meet zero B rows)
    for (int e = tid; e < L::TOTAL / 16; e += TC_THREADS) ((uint4*)sm)[e] = make_uint4(0, 0, 0, 0);
    if (warp == 0) tc::tmem_alloc(&s_tmem, L::TMEM_COLS);
    if (tid == 0) tc::mbar_init(&s_mbar, TC_ISSUERS);
    tc::fence_async_smem();
    __syncthreads();
    tc::fence_after();
    const uint32_t tbase = s_tmem;
    // two TMEM blocks of 8 MC columns: D_I and D_II, swapping roles per plane (D_III reuses D_I)
    // warps w and w+4 share TMEM lane quarter w and split the terms of a chunk
    const int quarter = warp & 3, whalf = warp >> 2;
    const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
    const int mc_lo = whalf * (MC / 2), mc_hi = mc_lo + MC / 2;
    const uint32_t idI = tc::idesc_f16(64, 8 * MC), idS = tc::idesc_f16(64, 8);
    // an MMA costs the issuing thread tens of cycles, so five threads issue in parallel,
    // each into its own accumulators (the results stay deterministic)
    const bool issuer = lane == 0 && warp < TC_ISSUERS;
    const int iss_lo = warp * (MC / 4), iss_hi = iss_lo + MC / 4;  // stage II/III terms of warps 0-3
    // this thread's elements e = tid + k TC_THREADS of stage I's B (uint4 e of B1H..B1L, core
    // (mc, q1) of hi or lo): the staged-F source index without the node's t1 offset, and mc, q1
    constexpr int NB1 = (2 * MC * 48 + TC_THREADS - 1) / TC_THREADS;
    int b1_src[NB1], b1_mq[NB1];
#pragma unroll
    for (int k = 0; k < NB1; ++k) {
        const int e = tid + k * TC_THREADS, d48 = e / 48, q1 = (e - 48 * d48) >> 3;
        b1_src[k] = e + 8 * d48;
        b1_mq[k] = (d48 & (MC - 1)) | (q1 << 8);
    }
    uint32_t phase = 0;
    // accumulator rows of this thread in the M=64 layout (16x256b read-outs):
    // 16 quarter + lane/4 and that + 8, columns cA and cA + 1 of each term
    const int rA = quarter * 16 + (lane >> 2), cA = 2 * (lane & 3);
    const uint32_t sbase = tc::smem_u32(sm);
    // B operands of stages II and III read in place from the chunk's staged F: the hi operand
    // [F_hi ; F_hi] has K-group offset 0 (both K groups are the same core matrix), the lo
    // operand [F_lo ; 0] reaches the zero block; a single-FP16 term pairs F_hi with zeros.
    // Operand (mc, t) lies 128 (mc 7 + t + 3) bytes past its table's start: 8 (mc 7 + t + 3)
    // more in the descriptor's start-address field, and as much less in the K-group offset
    // field when that offset reaches the zero block
    auto fdesc = [&](int mc, int t, bool hi, bool low) -> uint64_t {
        const uint64_t k8 = (uint64_t)((mc * 7 + t + 3) * 8);
        if (hi && !low) return tc::sdesc(sbase + L::FSH, 0u, 256) + k8;
        const uint64_t base = hi ? tc::sdesc(sbase + L::FSH, L::FZ - L::FSH, 256)
                                 : tc::sdesc(sbase + L::FSL, L::FZ - L::FSL, 256);
        return base + k8 - (k8 << 16);
    };
    // stage II/III A of term mc: A2_TERM bytes apart
    auto adesc = [&](int mc) -> uint64_t {
        return tc::sdesc(sbase + L::A2H, 128, L::A2_SBO) + (uint64_t)(mc * (L::A2_TERM / 16));
    };
    // this thread's row of the transposed 8x8 stores into A2: matrix lane/8 = (row group
    // 2 quarter + lane/16, K group (lane/8) & 1), row lane % 8 of it
    //   D_I -> stage II A: group c1 = lane % 8 is the row, i3 = 2 quarter + lane/16
    //   D_II -> stage III A: group c1 = 2 quarter + lane/16, row c2 = lane % 8
    const uint32_t a2_row_I = sbase + L::A2H + (lane & 7) * L::A2_SBO + ((lane >> 3) & 1) * 128 +
                              (2 * (warp & 3) + (lane >> 4)) * 16;
    const uint32_t a2_row_II = sbase + L::A2H + (2 * (warp & 3) + (lane >> 4)) * L::A2_SBO +
                               ((lane >> 3) & 1) * 128 + (lane & 7) * 16;

    // the abort decision comes from __syncthreads_or, so it is uniform
    bool aborted = false;
    // warp 0 polls the mbarrier; the block barrier then releases the others
#define TC_WAIT_OR_ABORT()                                                          \
    {                                                                               \
        bool ok_ = true;                                                            \
        if (warp == 0) ok_ = tc::mbar_wait(&s_mbar, phase, T.wait_limit);           \
        phase ^= 1u;                                                                \
        if (__syncthreads_or(!ok_)) {                                               \
            aborted = true;                                                         \
            if (tid == 0) atomicExch(T.err, 4);                                     \
        }                                                                           \
    }

    while (!aborted) {
        if (tid == 0) s_node = atomicAdd(T.counter, 1);
        __syncthreads();
        const int widx = s_node;
        if (widx >= T.nwork) break;
        const int node = T.order ? T.order[widx] : widx;
        const int jm_base = A.node_tree ? A.node_tree[node] * A.jm_stride : 0;
        const double lp_node = T.lpb ? T.lpb[A.node_tree ? A.node_tree[node] : 0] : 0.0;
        const int j = A.coord[4 * node];
        const int a1 = A.coord[4 * node + 1], a2 = A.coord[4 * node + 2], a3 = A.coord[4 * node + 3];
        const int p0 = A.pair_off[node], p1 = A.pair_off[node + 1];
        for (int q = tid; q < 216; q += TC_THREADS) tin[q] = INT_MIN;
        if (tid == 0) {
            s_mlo = INT_MAX;
            s_mhi = -1;
            s_exp_min = INT_MAX;
            s_xmax_bits = 0u;
            s_items = 0;
            s_lowi = 0;
        }
        __syncthreads();
        for (int p = p0 + tid; p < p1; p += TC_THREADS) {
            const Pair pr = A.pairs[p];
            const int q1 = pr.t1 + ((a1 & 1) ? 2 : 3), q2 = pr.t2 + ((a2 & 1) ? 2 : 3),
                      q3 = pr.t3 + ((a3 & 1) ? 2 : 3);
            const int q = q1 * 36 + q2 * 6 + q3;
            tin[q] = pr.in;
            tlo[q] = pr.m_lo;
            thi[q] = pr.m_hi;
            tfl[q] = pr.flags;
            atomicMin(&s_mlo, (int)pr.m_lo);
            atomicMax(&s_mhi, (int)pr.m_hi);
            const int b = pr.in >= 0 ? pr.in : A.n + (-1 - pr.in);
            int e;
            frexpf(T.sx[b], &e);
            atomicMin(&s_exp_min, e);
            atomicMax(&s_xmax_bits, __float_as_uint(T.xmax[b]));  // non-negative floats order as ints
        }
        __syncthreads();
        const int mlo = s_mlo, mhi = s_mhi;
        const float xmax_node = __uint_as_float(s_xmax_bits);
        // input values beyond FP32's range (infinite after the operand prep): refuse
        if (!(xmax_node <= FLT_MAX) && tid == 0) atomicExch(T.err, 5);
        const float sx_node = ldexpf(1.0f, s_exp_min - 1);
        // the power-of-two ratio between the node's scale and each input block's
        for (int q = tid; q < 216; q += TC_THREADS) {
            const int in = tin[q];
            tg[q] = in == INT_MIN ? 0.0f : sx_node / T.sx[in >= 0 ? in : A.n + (-1 - in)];
        }
        // ghat: (row rA + 8 s, column cA + h) at [2 s + h]: yc sums one chunk in FP32, yd
        // the chunks in FP64
        float yc[4];
        double yd[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            yc[c] = 0.0f;
            yd[c] = 0.0;
        }
        unsigned my_items = 0;  // kept (item, term) pairs counted by this thread
        if (mhi >= mlo && xmax_node > 0.0f && xmax_node <= FLT_MAX) {
            for (int m0 = mlo; m0 <= mhi && !aborted; m0 += MC) {
                // the kept-t1 masks per line and the per-term scales of the chunk
                const size_t fbase = ((size_t)j * A.M + m0) * 56;  // uint4 index of F(m0, t = -3)
                // the chunk's F^{j;m,t} (hi, lo) into shared memory, overlapping the set-up below:
                // stages II and III read their B operands there in place, and stage I's B is
                // built from there (terms past mhi get zeros)
                {
                    const int nv = MC * 56, nvalid = min(MC, mhi - m0 + 1) * 56;
                    for (int e = tid; e < 2 * nv; e += TC_THREADS) {
                        const int hl = e >= nv, r = hl ? e - nv : e;
                        uint4* dst = (uint4*)(sm + (hl ? L::FSL : L::FSH)) + r;
                        if (r < nvalid)
                            tc::cp_async16(dst, (hl ? FL : FH) + fbase + r);
                        else
                            *dst = make_uint4(0, 0, 0, 0);
                    }
                    tc::cp_async_commit();
                }
                for (int e = tid; e < 36 * MC; e += TC_THREADS) {
                    const int line = e / MC, mc = e % MC, m = m0 + mc;
                    unsigned char mk = 0;
                    if (m <= mhi) {
                        const int jm = A.Jm[jm_base + m];
                        if (jm >= j)
                            for (int q1 = 0; q1 < 6; ++q1) {
                                const int q = q1 * 36 + line;
                                if (tin[q] == INT_MIN || m < tlo[q] || m > thi[q]) continue;
                                if ((tfl[q] & 1) && jm > j) continue;
                                mk |= (unsigned char)(1u << q1);
                            }
                    }
                    msk[e] = mk;
                    my_items += __popc(mk);
                }
                if (tid < MC) {
                    const int m = m0 + tid;
                    float c2 = 0.0f, c3 = 0.0f, fin = 0.0f;
                    if (m <= mhi) {
                        const float mf = T.maxF[(size_t)j * A.M + m], sf = T.sF[(size_t)j * A.M + m];
                        if (mf > 0.0f) {
                            // power-of-two scales by exponent arithmetic (no FP64 on this path):
                            // sW = 2^eW, the largest power of two <= 8192 / (48 mf xmax), and
                            // sV = 2^eV <= 8192 / (48^2 mf^2 xmax); sf is a power of two
                            int em, ex, ef, e1, e2;
                            const float fm = frexpf(mf, &em), fx = frexpf(xmax_node, &ex);
                            frexpf(sf, &ef);
                            ef -= 1;
                            frexpf(8192.0f / (48.0f * fm * fx), &e1);
                            frexpf(8192.0f / (2304.0f * fm * fm * fx), &e2);
                            const int eW = min(e1 - 1 - em - ex, 126), eV = min(e2 - 1 - 2 * em - ex, 126);
                            if (eW >= -126 && eV >= -126) {
                                c2 = ldexpf(1.0f, eW - ef - (s_exp_min - 1));  // sW / (sf sx_node)
                                c3 = ldexpf(1.0f, eV - eW - ef);                // sV / (sW sf)
                                fin = ldexpf((float)A.w[m], -(eV + ef));        // w_m / (sV sf)
                                if (!(fin <= FLT_MAX)) {  // outputs beyond the FP32 range: refuse
                                    atomicExch(T.err, 5);
                                    fin = 0.0f;
                                }
                            }
                        }
                    }
                    s_c2[tid] = c2;
                    s_c3[tid] = c3;
                    s_fin[tid] = fin;
                    s_B[tid] = 0.0f;
                    s_cnt[tid] = 0;
                }
                tc::cp_async_wait_all();  // this thread's part of the chunk's F
                __syncthreads();
                // precision ladder: B_m = w_m sum over the term's kept items of
                // N_F(t1) N_F(t2) N_F(t3) ||x_b|| bounds its contribution to this node
                if (LADDER)
                    for (int e = tid; e < 36 * MC; e += TC_THREADS) {
                        const unsigned mk = msk[e];
                        if (!mk) continue;
                        const int line = e / MC, mc = e % MC, m = m0 + mc;
                        const double* nf = A.nF + ((size_t)j * A.M + m) * 7;
                        float acc = 0.0f;
                        for (int q1 = 0; q1 < 6; ++q1) {
                            if (!((mk >> q1) & 1u)) continue;
                            const int in = tin[q1 * 36 + line];
                            const int b = in >= 0 ? in : A.n + (-1 - in);
                            acc += (float)nf[band_t(a1, q1) + 3] * T.xnrm[b];
                        }
                        acc *= (float)(nf[band_t(a2, line / 6) + 3] * nf[band_t(a3, line % 6) + 3]);
                        atomicAdd(&s_B[mc], acc);
                        atomicAdd(&s_cnt[mc], __popc(mk));
                    }
                if (tid < 36) {
                    // per line: the union of its terms' kept-t1 masks
                    unsigned long long km = line_masks(tid);
                    km |= km >> 32;
                    km |= km >> 16;
                    km |= km >> 8;
                    s_lm[tid] = (unsigned char)km;
                    if (m0 == mlo) {  // once per node: stage I's B depends on g through these
                        unsigned long long kg = 0;
                        for (int q1 = 0; q1 < 6; ++q1)
                            kg |= (unsigned long long)((__float_as_uint(tg[q1 * 36 + tid]) >> 23) & 0xffu) << (8 * q1);
                        s_kg[tid] = kg;
                    }
                }
                if (warp == 2) {
                    // the visiting order: cursors of the lines with a kept item, ascending
                    const bool h0 = line_masks(line_of(lane)) != 0;
                    const bool h1 = lane < 4 && line_masks(line_of(32 + lane)) != 0;
                    const unsigned b0 = __ballot_sync(0xffffffffu, h0), b1 = __ballot_sync(0xffffffffu, h1);
                    const unsigned below = (1u << lane) - 1u;
                    if (h0) s_order[__popc(b0 & below)] = (unsigned char)lane;
                    if (h1) s_order[__popc(b0) + __popc(b1 & below)] = (unsigned char)(32 + lane);
                    if (lane == 0) s_nl = __popc(b0) + __popc(b1);
                }
                __syncthreads();
                if (LADDER) {
                    if (tid == 32) {
                        // single FP16 products (hi only) for terms whose rounding error,
                        // at most LADDER_U B_m, fits the node's share of the budget
                        int all = 1;
                        const double per_term = lp_node / (double)(mhi - mlo + 1);
                        for (int mc = 0; mc < MC; ++mc) {
                            const int m = m0 + mc;
                            int low = 1;
                            if (m <= mhi) low = T.lpb && LADDER_U * A.w[m] * (double)s_B[mc] <= per_term;
                            s_low[mc] = (unsigned char)low;
                            if (low) s_lowi += s_cnt[mc];
                            all &= low;
                        }
                        s_all_low = all;
                    }
                    __syncthreads();
                }
                const int all_low = LADDER ? s_all_low : 0;
                // masks and g exponents of the line stage I's B was last built for
                unsigned long long built_m = ~0ull, built_g = ~0ull;
                // stage I A (a line's six input blocks) is copied asynchronously into one of two
                // buffers while earlier lines compute
                auto fetch_line = [&](int c, int buf) {
                    const int line = line_of(c);
                    const unsigned lmx = s_lm[line];
                    // element e = (hl, q1, v): uint4 v (of 64) of block q1, hi then lo
                    const int nfe = all_low ? 384 : 768;
#pragma unroll
                    for (int k = 0; k < 768 / TC_THREADS; ++k) {
                        const int e = tid + k * TC_THREADS;
                        if (e >= nfe) continue;
                        const int hl = e >= 384, r = hl ? e - 384 : e, q1 = r >> 6;
                        uint4* dst = (uint4*)(sm + L::XH + hl * (L::XL - L::XH) + buf * 6144) + r;
                        if (lmx & (1u << q1)) {
                            const int in = tin[q1 * 36 + line];
                            const int b = in >= 0 ? in : A.n + (-1 - in);
                            tc::cp_async16(dst, (const uint4*)((hl ? T.xl : T.xh) + (size_t)b * 512) + (r & 63));
                        } else {
                            *dst = make_uint4(0, 0, 0, 0);
                        }
                    }
                    tc::cp_async_commit();
                };
                // stage I's B for a line: core (N group mc, K group q1) = mask ? g F^{t1(q1)} : 0
                // with the power-of-two ratio g = sx_node / sx_b (exact in FP16)
                auto build_B = [&](int c) {
                    const int lineb = line_of(c);
                    // when the line's masks and g equal the last build's, B1 already holds
                    // this line's operand
                    const unsigned long long km = line_masks(lineb), kg = s_kg[lineb];
                    if (km == built_m && kg == built_g) return;
                    built_m = km;
                    built_g = kg;
                    // element e = (hl, mc, q1, v) of B1 (hi then lo, uint4 v of core (mc, q1)) is
                    // uint4 e of B1H..B1L; its source F^{t1(q1)}_mc, t1 + 3 = q1 + (a1 & 1), is
                    // uint4 e + 8 (e / 48 + (a1 & 1)) of the staged F (hi then lo)
                    const int nb1 = all_low ? MC * 48 : 2 * MC * 48;
                    const unsigned char* mline = msk + lineb * MC;
                    const float* gline = tg + lineb;
                    const uint4* fs = (const uint4*)(sm + L::FSH) + 8 * (a1 & 1);
                    // all of this thread's elements at once (predicated, no early exit), so that
                    // their shared-memory loads are in flight together
#pragma unroll
                    for (int k = 0; k < NB1; ++k) {
                        const int e = tid + k * TC_THREADS;
                        const int mc = b1_mq[k] & 0xff, q1 = b1_mq[k] >> 8;
                        const bool keep = e < nb1 && ((mline[mc] >> q1) & 1u);
                        uint4 out = make_uint4(0, 0, 0, 0);
                        if (keep) {
                            const uint4 fin4 = fs[b1_src[k]];
                            const __half2 g2 = __float2half2_rn(gline[q1 * 36]);
                            const __half2* pi = (const __half2*)&fin4;
                            __half2* po = (__half2*)&out;
#pragma unroll
                            for (int h = 0; h < 4; ++h) po[h] = __hmul2(pi[h], g2);
                        }
                        if (e < nb1) ((uint4*)B1H)[e] = out;
                    }
                };
                // stage I from X buffer parx into the TMEM block d (thread 0)
                auto issue_stage1 = [&](int parx, uint32_t d) {
                    const uint64_t a0 = tc::sdesc(sbase + L::XH + parx * 6144, 1024, 128);
                    const uint64_t b0 = tc::sdesc(sbase + L::B1H, 128, 768);
#pragma unroll
                    for (int ks = 0; ks < 3; ++ks) {  // K step: 2048 bytes of X, 256 of B1
                        const uint64_t ah = a0 + ks * 128, al = ah + (L::XL - L::XH) / 16;
                        const uint64_t bh = b0 + ks * 16, bl = bh + (L::B1L - L::B1H) / 16;
                        tc::mma_f16(d, ah, bh, idI, ks > 0);
                        if (!all_low) {
                            tc::mma_f16(d, ah, bl, idI, 1);
                            tc::mma_f16(d, al, bh, idI, 1);
                        }
                    }
                };
                // ghat += w_m Y_m from the TMEM block d: row (c1, c2), column c3; per plane an FP32
                // sum over this warp half's terms, added to the chunk's FP32 sum
                auto accumulate_y = [&](uint32_t d) {
                    float yv[MC / 2][4];
                    tc::tmem_ld16x256_rep<MC / 2>(d + lane_off + mc_lo * 8, yv);
                    float part[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
                    for (int mc = mc_lo; mc < mc_hi; ++mc) {
                        const float* v = yv[mc - mc_lo];
                        const float fin = s_fin[mc];
#pragma unroll
                        for (int q = 0; q < 4; ++q) part[q] = fmaf(fin, v[q], part[q]);
                    }
#pragma unroll
                    for (int q = 0; q < 4; ++q) yc[q] += part[q];
                };
                // Software pipeline over the chunk's lines: one wait and two block barriers per
                // line.  While line L's stage I runs, stage II of the line before runs too; after
                // the wait the block converts D_I(L) and builds line L+1's stage-I B, then the
                // issuing threads send stage II(L) and stage I(L+1) under one commit while the
                // others start the copies of line L+2's input blocks.  After a plane's last
                // line, stage III of the plane and stage I of the next plane's first line go
                // out together: the two TMEM column blocks swap roles (D_I <-> D_II) from plane
                // to plane, and stage III's result, left in the new D_II block, is read after
                // the next wait.
                const int nl = s_nl;  // only lines with a kept item are visited
                if (nl > 0) {
                    int li = 0;
                    int cur = s_order[0];
                    int nxt = nl > 1 ? s_order[1] : 36;
                    int xb = 0;  // X buffer of line L
                    uint32_t dI = tbase, dII = tbase + 8 * MC;
                    bool first = true, y_pending = false;
                    fetch_line(cur, xb);
                    build_B(cur);
                    tc::cp_async_wait_all();
                    if (nxt < 36) fetch_line(nxt, xb ^ 1);
                    tc::fence_async_smem();
                    __syncthreads();
                    // (test hook: with T.withhold nothing is sent, so the first wait can
                    // only end by its limit, with no MMA in flight)
                    if (issuer && !T.withhold) {
                        tc::fence_after();
                        if (warp == 4) issue_stage1(xb, dI);
                        tc::commit(&s_mbar);
                    }
                    for (;;) {
                        // stage I(L) and everything before it complete: D_I, B1, A2 and the X
                        // buffer of line L are free
                        TC_WAIT_OR_ABORT();
                        if (aborted) break;
                        tc::fence_after();
                        if (y_pending) {  // the previous plane's stage III
                            accumulate_y(dII);
                            y_pending = false;
                        }
                        // D_I -> stage II A (rows (c1, i3), K = i2 as hi | lo).  This thread holds D_I
                        // rows (i3, i2) = (2 quarter, lane/4) and (2 quarter + 1, lane/4), columns
                        // c1 = cA, cA + 1: per term, its fragments of the 8x8 matrices [i2][c1] of the
                        // two i3, hi and lo, stored transposed (a memory row = the K values of a (c1, i3))
                        {
                            float vv[MC / 2][4];
                            tc::tmem_ld16x256_rep<MC / 2>(dI + lane_off + mc_lo * 8, vv);
#pragma unroll
                            for (int mc = mc_lo; mc < mc_hi; ++mc) {
                                const float* v = vv[mc - mc_lo];
                                const float c2 = s_c2[mc];
                                uint32_t h0, l0, h1, l1;
                                tc::split_h2(v[0] * c2, v[1] * c2, h0, l0);
                                tc::split_h2(v[2] * c2, v[3] * c2, h1, l1);
                                tc::stmatrix_x4_trans(a2_row_I + mc * L::A2_TERM, h0, l0, h1, l1);
                            }
                        }
                        const int q3 = cur / 6;
                        const bool last = nxt >= 36 || nxt / 6 != q3;  // L ends its plane
                        const int nn = li + 2 < nl ? s_order[li + 2] : 36;
                        if (nxt < 36) {
                            build_B(nxt);
                            tc::cp_async_wait_all();  // line L+1's input blocks
                        }
                        tc::fence_before();
                        tc::fence_async_smem();
                        __syncthreads();
                        if (issuer) {
                            tc::fence_after();
                            if (warp < 4) {
                                // stage II(L): per term, V += A2 (M=64 (c1,i3) x K=16) x F^{t2} (N=8 c2)
                                const int t2 = band_t(a2, cur % 6);
                                for (int mc = iss_lo; mc < iss_hi; ++mc) {
                                    const bool low = LADDER && s_low[mc];
                                    const uint64_t a = adesc(mc);
                                    tc::mma_f16(dII + mc * 8, a, fdesc(mc, t2, true, low), idS, first ? 0u : 1u);
                                    if (!low) tc::mma_f16(dII + mc * 8, a, fdesc(mc, t2, false, false), idS, 1);
                                }
                            } else if (!last) {
                                issue_stage1(xb ^ 1, dI);
                            }
                            tc::commit(&s_mbar);
                        }
                        // line L+2's input blocks into line L's buffer, while the MMAs run
                        if (nn < 36) fetch_line(nn, xb);
                        if (last) {
                            // the plane's last stage II complete: D_II -> stage III A (aliases
                            // stage II A)
                            TC_WAIT_OR_ABORT();
                            if (aborted) break;
                            tc::fence_after();
                            // D_II -> stage III A (rows (c1, c2), K = i3 as hi | lo).  This thread holds
                            // D_II rows (c1, i3) = (2 quarter, lane/4) and (2 quarter + 1, lane/4),
                            // columns c2 = cA, cA + 1: per term, its fragments of the matrices [i3][c2]
                            // of the two c1, hi and lo, stored transposed
                            {
                                float vv[MC / 2][4];
                                tc::tmem_ld16x256_rep<MC / 2>(dII + lane_off + mc_lo * 8, vv);
#pragma unroll
                                for (int mc = mc_lo; mc < mc_hi; ++mc) {
                                    const float* v = vv[mc - mc_lo];
                                    const float c3 = s_c3[mc];
                                    uint32_t h0, l0, h1, l1;
                                    tc::split_h2(v[0] * c3, v[1] * c3, h0, l0);
                                    tc::split_h2(v[2] * c3, v[3] * c3, h1, l1);
                                    tc::stmatrix_x4_trans(a2_row_II + mc * L::A2_TERM, h0, l0, h1, l1);
                                }
                            }
                            tc::fence_before();
                            tc::fence_async_smem();
                            __syncthreads();
                            // stage III: per term, Y += A3 (M=64 (c1,c2) x K=16) x F^{t3} (N=8 c3)
                            // into the D_I block; the next plane's first stage I into D_II
                            if (issuer) {
                                tc::fence_after();
                                if (warp < 4) {
                                    const int t3 = band_t(a3, q3);
                                    for (int mc = iss_lo; mc < iss_hi; ++mc) {
                                        const bool low = LADDER && s_low[mc];
                                        const uint64_t a = adesc(mc);
                                        tc::mma_f16(dI + mc * 8, a, fdesc(mc, t3, true, low), idS, 0);
                                        if (!low) tc::mma_f16(dI + mc * 8, a, fdesc(mc, t3, false, false), idS, 1);
                                    }
                                } else if (nxt < 36) {
                                    issue_stage1(xb ^ 1, dII);
                                }
                                tc::commit(&s_mbar);
                            }
                            const uint32_t d = dI;
                            dI = dII;
                            dII = d;
                            y_pending = true;
                            if (nxt >= 36) {  // the chunk's last plane
                                TC_WAIT_OR_ABORT();
                                if (aborted) break;
                                tc::fence_after();
                                accumulate_y(dII);
                                y_pending = false;
                                tc::fence_before();
                                break;
                            }
                        }
                        first = last;
                        ++li;
                        cur = nxt;
                        nxt = nn;
                        xb ^= 1;
                    }
                    tc::cp_async_wait_all();
                }
                if (aborted) break;
                // the chunk's sum joins ghat in FP64
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    yd[q] += (double)yc[q];
                    yc[q] = 0.0f;
                }
                tc::fence_before();
                __syncthreads();
            }
        }
        // Y rows (c1, c2) = rA + 8 s, columns c3 = cA + h; the two warp halves add up
        double* ysm = (double*)(sm + L::XH);  // every copy into the X buffers is complete here
        if (whalf == 1)
#pragma unroll
            for (int q = 0; q < 4; ++q) ysm[(rA + 8 * (q >> 1)) * 8 + cA + (q & 1)] = yd[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) my_items += __shfl_xor_sync(0xffffffffu, my_items, o);
        if (lane == 0 && my_items) atomicAdd(&s_items, (unsigned long long)my_items);
        __syncthreads();
        if (whalf == 0)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int r = rA + 8 * (q >> 1), c1 = r >> 3, c2 = r & 7, c3 = cA + (q & 1);
                if (c1 < kr && c2 < kr && c3 < kr)
                    A.out[(size_t)node * kr * kr * kr + (c1 * kr + c2) * kr + c3] = yd[q] + ysm[r * 8 + c3];
            }
        if (tid == 0 && A.n_items) atomicAdd(A.n_items + (A.node_tree ? A.node_tree[node] : 0), s_items);
        if (tid == 0 && T.n_lowp && s_lowi) atomicAdd(T.n_lowp, s_lowi);
        __syncthreads();
    }
#undef TC_WAIT_OR_ABORT
    tc::cp_async_wait_all();
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tbase, L::TMEM_COLS);
}

// ---------------------------------------------------------------- host side
int tc_alloc(const mra_op* op, int nb, TcBuffers* B) {
    const Alloc& Al = op->A;
    const size_t JM = (size_t)(op->J + 1) * op->M;
    MRA_TRY(dalloc(Al, &B->xh, (size_t)nb * 512));
    MRA_TRY(dalloc(Al, &B->xl, (size_t)nb * 512));
    MRA_TRY(dalloc(Al, &B->sx, nb));
    MRA_TRY(dalloc(Al, &B->xmax, nb));
    MRA_TRY(dalloc(Al, &B->xnrm, nb));
    MRA_TRY(dalloc(Al, &B->Fh, JM * 7 * 64));
    MRA_TRY(dalloc(Al, &B->Fl, JM * 7 * 64));
    MRA_TRY(dalloc(Al, &B->sF, JM));
    MRA_TRY(dalloc(Al, &B->maxF, JM));
    MRA_TRY(dalloc(Al, &B->counter, 1));
    return MRA_OK;
}

int tc_prep_F(const mra_op* op, const TcBuffers& B, cudaStream_t st) {
    k_tc_prep_F<<<dim3(op->M, op->J + 1), 128, 0, st>>>(op->M, op->k, op->F, B.Fh, B.Fl, B.sF, B.maxF);
    MRA_CK_LAUNCH();
    return MRA_OK;
}

int tc_prep_blocks(int nb, int kr, int n, const double* s, const double* gblk, const TcBuffers& B, cudaStream_t st) {
    if (nb <= 0) return MRA_OK;
    const int grid = std::max(1, std::min(num_sms() * 8, (nb + PREP_WARPS - 1) / PREP_WARPS));
    k_tc_prep_blocks<<<grid, 32 * PREP_WARPS, 0, st>>>(nb, kr, n, s, gblk, B.xh, B.xl, B.sx, B.xmax, B.xnrm);
    MRA_CK_LAUNCH();
    return MRA_OK;
}

void tc_release(const mra_op* op, TcBuffers* B) {
    const Alloc& Al = op->A;
    Al.put(B->xh); Al.put(B->xl); Al.put(B->sx); Al.put(B->xmax); Al.put(B->xnrm);
    Al.put(B->Fh); Al.put(B->Fl); Al.put(B->sF); Al.put(B->maxF); Al.put(B->counter);
    *B = TcBuffers();
}

// dynamic shared memory of both chunk sizes (outside any stream capture)
int tc_configure() {
    MRA_CK(cudaFuncSetAttribute(k_apply_tc<4, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, TcSmem<4>::TOTAL));
    MRA_CK(cudaFuncSetAttribute(k_apply_tc<4, false>, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    MRA_CK(cudaFuncSetAttribute(k_apply_tc<8, false>, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    MRA_CK(cudaFuncSetAttribute(k_apply_tc<4, true>, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    MRA_CK(cudaFuncSetAttribute(k_apply_tc<8, true>, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    MRA_CK(cudaFuncSetAttribute(k_apply_tc<8, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, TcSmem<8>::TOTAL));
    MRA_CK(cudaFuncSetAttribute(k_apply_tc<4, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, TcSmem<4>::TOTAL));
    MRA_CK(cudaFuncSetAttribute(k_apply_tc<8, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, TcSmem<8>::TOTAL));
    return tc3_configure();
}

template <int MC>
static int launch_mc(const TcArgs& T, int ctas_per_sm, cudaStream_t st) {
    const int grid = std::max(1, std::min(T.nwork, num_sms() * ctas_per_sm));
    if (T.lpb) k_apply_tc<MC, true><<<grid, TC_THREADS, TcSmem<MC>::TOTAL, st>>>(T);
    else k_apply_tc<MC, false><<<grid, TC_THREADS, TcSmem<MC>::TOTAL, st>>>(T);
    MRA_CK_LAUNCH();
    return MRA_OK;
}

// variant: terms per chunk (4 or 8) and CTAs per SM (1 to 3 for 8 terms, 1 to 4
// for 4 terms: registers, TMEM and shared memory allow that many); 8 terms at
// two CTAs per SM is the wide-MMA kernel of apply_tc3.cu.
// tc_configure() first.
int tc_launch(const TcArgs& T, int mc, int ctas_per_sm, cudaStream_t st) {
    MRA_CK(cudaMemsetAsync(T.counter, 0, sizeof(int), st));
    if (mc == 4) return launch_mc<4>(T, ctas_per_sm, st);
    // 8 terms at two CTAs per SM: the wide-MMA kernel (apply_tc3.cu)
    if (ctas_per_sm == 2) return tc3_launch(T, st);
    return launch_mc<8>(T, ctas_per_sm, st);
}

TcArgs tc_args(const ApplyArgs& A, const TcBuffers& B, int* err) {
    TcArgs T;
    T.A = A;
    T.xh = B.xh; T.xl = B.xl; T.sx = B.sx; T.xmax = B.xmax; T.xnrm = B.xnrm;
    T.lpb = nullptr;
    T.n_lowp = nullptr;
    T.Fh = B.Fh; T.Fl = B.Fl; T.sF = B.sF; T.maxF = B.maxF;
    T.err = err;  // the apply's error word: a wait that reaches its limit writes 4
    T.wait_limit = TC_WAIT_LIMIT;
    T.withhold = 0;
    T.counter = B.counter;
    T.order = nullptr;
    T.nwork = A.n;
    T.kr = A.k;
    return T;
}

int launch_apply_tc(const ApplyArgs& A, int nghost, const mra_op* op, int* err, const double* lpb,
                    unsigned long long* n_lowp, unsigned wait_limit, int withhold, cudaStream_t st) {
    if (A.k > 8) {
        set_error("the tensor-core apply supports k <= 8 (got k = %d)", A.k);
        return MRA_EINVAL;
    }
    // the operand buffers are released (stream-ordered, after the kernel) on every return
    struct Guard {
        const mra_op* op;
        TcBuffers B;
        ~Guard() { tc_release(op, &B); }
    } G{op, TcBuffers()};
    MRA_TRY(tc_alloc(op, A.n + nghost, &G.B));
    MRA_TRY(tc_prep_F(op, G.B, st));
    MRA_TRY(tc_prep_blocks(A.n + nghost, A.k, A.n, A.s, A.gblk, G.B, st));
    MRA_TRY(tc_configure());
    TcArgs T = tc_args(A, G.B, err);
    T.lpb = lpb;
    T.n_lowp = n_lowp;
    T.wait_limit = wait_limit ? std::max(wait_limit, TC_WAIT_MIN) : TC_WAIT_LIMIT;
    T.withhold = withhold;
    return tc_launch(T, 8, 3, st);
}

}  // namespace mra
