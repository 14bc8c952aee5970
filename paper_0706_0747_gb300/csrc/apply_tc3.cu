// Step 3 of Algorithm 3 on the tcgen05 tensor cores with fewer, wider MMAs
// (8 terms per chunk, two CTAs per SM, k <= 8).
//
// The same nested sums, operands, scales and precision as k_apply_tc
// (apply_tc.cu), and the same software pipeline over a chunk's lines.  On
// this part an MMA costs its SM tens of cycles to issue whatever its size, and
// k_apply_tc issues 25 small ones per line (stage I 3 K steps x 3 hi/lo
// products, stage II 2 per term) and 16 per plane, which bounds its time.
// Here, with 256 TMEM columns per CTA:
//   stage I   per K step: A_hi x [B_hi | B_lo] (N = 128: hi*hi into columns
//             0-63, hi*lo into 64-127) and A_lo x B_hi (N = 64, into 0-63):
//             6 MMAs per line; W is the sum of the two column halves;
//   stage II  per term one MMA with N = 16: [A_hi | A_lo] against
//             [F_hi ; F_hi] (columns 0-7) and [F_lo ; F_lo] (columns 8-15), the
//             B descriptor reaching F_lo through its N-group stride; V is the sum
//             of the two halves (the lo*lo product it adds is harmless);
//   stage III the same per term into D_II's columns (read out after the
//             next wait), so no TMEM block changes role between planes.
// 14 MMAs per line and 8 per plane.  The precision ladder keeps its stage-I
// saving (single FP16 products when every term of the chunk qualifies);
// stages II and III always take the split products, one MMA either way.
#include <cfloat>
#include <climits>

#include "apply_common.cuh"
#include "tc_ptx.cuh"

namespace mra {

#define TC3_THREADS 256
#define TC3_ISSUERS 5
#define LADDER3_U 0.00390625

template <int MC>
struct Tc3Smem {
    static constexpr int XH = 0;                    // 2 buffers x 6 blocks x 1 KB: stage I A (hi); the final y
    static constexpr int XL = 12288;                // (lo); buffer p at + p * 6144
    static constexpr int B1H = 24576;               // MC terms x 6 K groups x 128 B: stage I B (hi)
    static constexpr int B1L = B1H + MC * 768;      // (lo): N groups MC..2MC-1 of the N = 128 operand
    static constexpr int A2_SBO = 272;
    static constexpr int A2_TERM = 8 * A2_SBO;
    static constexpr int A2H = B1L + MC * 768;
    static constexpr int FSH = A2H + MC * A2_TERM;  // MC terms x 7 shifts x 128 B: the chunk's F (hi)
    static constexpr int FSL = FSH + MC * 896;      // (lo)
    static constexpr int FZ = FSL + MC * 896;       // one zero core matrix
    static constexpr int TIN = FZ + 128;
    static constexpr int TLO = TIN + 864;
    static constexpr int THI = TLO + 432;
    static constexpr int TFL = THI + 432;
    static constexpr int TG = (TFL + 216 + 15) / 16 * 16;
    static constexpr int MSK = TG + 864;
    static constexpr int TOTAL = (MSK + 36 * MC + 127) / 128 * 128;
    static constexpr int TMEM_COLS = 256;           // D_I (2 x 8 MC columns), D_II (16 MC columns)
};
static_assert(2 * (Tc3Smem<8>::TOTAL + 2048) <= 232448, "two CTAs per SM");
static_assert(Tc3Smem<8>::MSK % 8 == 0, "a line's masks are read as one word");
static_assert(Tc3Smem<8>::FSL - Tc3Smem<8>::FSH < (1 << 18), "N-group stride of the stage II/III B operand");

template <bool LADDER>
__global__ void __launch_bounds__(TC3_THREADS, 2) k_apply_tc3(TcArgs T) {
    constexpr int MC = 8;
    using L = Tc3Smem<MC>;
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
    for (int e = tid; e < L::TOTAL / 16; e += TC3_THREADS) ((uint4*)sm)[e] = make_uint4(0, 0, 0, 0);
    if (warp == 0) tc::tmem_alloc(&s_tmem, L::TMEM_COLS);
    if (tid == 0) tc::mbar_init(&s_mbar, TC3_ISSUERS);
    tc::fence_async_smem();
    __syncthreads();
    tc::fence_after();
    const uint32_t tbase = s_tmem;
    // TMEM: D_I at columns 0-127 (hi*hi + lo*hi at 8 mc, hi*lo at 64 + 8 mc), D_II (and
    // stage III's result) at 128-255 (term mc at 128 + 16 mc: the F_hi and F_lo halves)
    const uint32_t tDI = tbase, tDII = tbase + 16 * MC;
    // warps w and w+4 share TMEM lane quarter w and split the terms of a chunk
    const int quarter = warp & 3, whalf = warp >> 2;
    const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
    const int mc_lo = whalf * (MC / 2), mc_hi = mc_lo + MC / 2;
    // stage I: N = 128 ([B_hi | B_lo]) and N = 64 (B_hi); stages II / III: N = 16 per term
    const uint32_t idI2 = tc::idesc_f16(64, 16 * MC), idI = tc::idesc_f16(64, 8 * MC), idS = tc::idesc_f16(64, 16);
    // an MMA costs the issuing thread tens of cycles, so five threads issue in parallel,
    // each into its own accumulators (the results stay deterministic)
    const bool issuer = lane == 0 && warp < TC3_ISSUERS;
    const int iss_lo = warp * (MC / 4), iss_hi = iss_lo + MC / 4;  // stage II/III terms of warps 0-3
    // this thread's elements e = tid + k TC3_THREADS of stage I's B (uint4 e of B1H..B1L, core
    // (mc, q1) of hi or lo): the staged-F source index without the node's t1 offset, and mc, q1
    constexpr int NB1 = (2 * MC * 48 + TC3_THREADS - 1) / TC3_THREADS;
    int b1_src[NB1], b1_mq[NB1];
#pragma unroll
    for (int k = 0; k < NB1; ++k) {
        const int e = tid + k * TC3_THREADS, d48 = e / 48, q1 = (e - 48 * d48) >> 3;
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
    // B operand of stages II / III for term mc at shift t: N-group 0 is F_hi, N-group 1
    // F_lo (the N-group stride reaches the lo table), and both K groups of a row read
    // the same core matrix (K-group stride 0): [F_hi ; F_hi] and [F_lo ; F_lo] against
    // A = [A_hi | A_lo].  Operand (mc, t) lies 128 (mc 7 + t + 3) bytes into each table.
    auto fdesc = [&](int mc, int t) -> uint64_t {
        return tc::sdesc(sbase + L::FSH, 0u, L::FSL - L::FSH) + (uint64_t)((mc * 7 + t + 3) * 8);
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
#define TC3_WAIT_OR_ABORT()                                                          \
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
        for (int q = tid; q < 216; q += TC3_THREADS) tin[q] = INT_MIN;
        if (tid == 0) {
            s_mlo = INT_MAX;
            s_mhi = -1;
            s_exp_min = INT_MAX;
            s_xmax_bits = 0u;
            s_items = 0;
            s_lowi = 0;
        }
        __syncthreads();
        for (int p = p0 + tid; p < p1; p += TC3_THREADS) {
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
        for (int q = tid; q < 216; q += TC3_THREADS) {
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
                    for (int e = tid; e < 2 * nv; e += TC3_THREADS) {
                        const int hl = e >= nv, r = hl ? e - nv : e;
                        uint4* dst = (uint4*)(sm + (hl ? L::FSL : L::FSH)) + r;
                        if (r < nvalid)
                            tc::cp_async16(dst, (hl ? FL : FH) + fbase + r);
                        else
                            *dst = make_uint4(0, 0, 0, 0);
                    }
                    tc::cp_async_commit();
                }
                for (int e = tid; e < 36 * MC; e += TC3_THREADS) {
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
                    for (int e = tid; e < 36 * MC; e += TC3_THREADS) {
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
                        // single FP16 stage-I products (hi only) when every term's rounding
                        // error, at most LADDER3_U B_m, fits the node's share of the budget
                        // (stages II and III keep the split products: one MMA either way)
                        int all = 1;
                        unsigned long long cnt = 0;
                        const double per_term = lp_node / (double)(mhi - mlo + 1);
                        for (int mc = 0; mc < MC; ++mc) {
                            const int m = m0 + mc;
                            int low = 1;
                            if (m <= mhi) low = T.lpb && LADDER3_U * A.w[m] * (double)s_B[mc] <= per_term;
                            s_low[mc] = (unsigned char)low;
                            cnt += s_cnt[mc];
                            all &= low;
                        }
                        if (all) s_lowi += cnt;
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
                    for (int k = 0; k < 768 / TC3_THREADS; ++k) {
                        const int e = tid + k * TC3_THREADS;
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
                        const int e = tid + k * TC3_THREADS;
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
                // stage I from X buffer parx into D_I (columns 0-63: hi*hi + lo*hi, 64-127: hi*lo);
                // B1L follows B1H at the N-group stride, so [B_hi | B_lo] is one N = 128 operand
                auto issue_stage1 = [&](int parx) {
                    const uint64_t a0 = tc::sdesc(sbase + L::XH + parx * 6144, 1024, 128);
                    const uint64_t b0 = tc::sdesc(sbase + L::B1H, 128, 768);
#pragma unroll
                    for (int ks = 0; ks < 3; ++ks) {  // K step: 2048 bytes of X, 256 of B1
                        const uint64_t ah = a0 + ks * 128, al = ah + (L::XL - L::XH) / 16;
                        const uint64_t bh = b0 + ks * 16;
                        if (all_low) {
                            tc::mma_f16(tDI, ah, bh, idI, ks > 0);
                        } else {
                            tc::mma_f16(tDI, ah, bh, idI2, ks > 0);
                            tc::mma_f16(tDI, al, bh, idI, 1);
                        }
                    }
                };
                // ghat += w_m Y_m from the TMEM block d: row (c1, c2), column c3; per plane an FP32
                // sum over this warp half's terms, added to the chunk's FP32 sum
                // a D_II read-out: this thread's four terms, the two column halves of each added
                auto read_dii = [&](float (*v)[4]) {
                    float a[4][4], b[4][4];
                    tc::tmem_ld16x256_rep<4>(tDII + lane_off + mc_lo * 16, a);       // terms mc_lo, mc_lo + 1
                    tc::tmem_ld16x256_rep<4>(tDII + lane_off + mc_lo * 16 + 32, b);  // mc_lo + 2, mc_lo + 3
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        v[0][q] = a[0][q] + a[1][q];
                        v[1][q] = a[2][q] + a[3][q];
                        v[2][q] = b[0][q] + b[1][q];
                        v[3][q] = b[2][q] + b[3][q];
                    }
                };
                auto accumulate_y = [&]() {
                    float yv[MC / 2][4];
                    read_dii(yv);
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
                // line, stage III (into D_II, whose values were just read) and stage I of the
                // next plane's first line go out together; stage III's result is read after the
                // next wait, before that plane's first stage II overwrites D_II.
                const int nl = s_nl;  // only lines with a kept item are visited
                if (nl > 0) {
                    int li = 0;
                    int cur = s_order[0];
                    int nxt = nl > 1 ? s_order[1] : 36;
                    int xb = 0;  // X buffer of line L
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
                        if (warp == 4) issue_stage1(xb);
                        tc::commit(&s_mbar);
                    }
                    for (;;) {
                        // stage I(L) and everything before it complete: D_I, B1, A2 and the X
                        // buffer of line L are free
                        TC3_WAIT_OR_ABORT();
                        if (aborted) break;
                        tc::fence_after();
                        if (y_pending) {  // the previous plane's stage III
                            accumulate_y();
                            y_pending = false;
                        }
                        // D_I -> stage II A (rows (c1, i3), K = i2 as hi | lo).  This thread holds D_I
                        // rows (i3, i2) = (2 quarter, lane/4) and (2 quarter + 1, lane/4), columns
                        // c1 = cA, cA + 1: per term, its fragments of the 8x8 matrices [i2][c1] of the
                        // two i3, hi and lo, stored transposed (a memory row = the K values of a (c1, i3))
                        {
                            // W = (hi*hi + lo*hi) + hi*lo: the two column halves of D_I (the
                            // second is not written when the chunk takes single FP16 products)
                            float vv[MC / 2][4], vl[MC / 2][4];
                            tc::tmem_ld16x256_rep<MC / 2>(tDI + lane_off + mc_lo * 8, vv);
                            if (!all_low) {
                                tc::tmem_ld16x256_rep<MC / 2>(tDI + lane_off + 64 + mc_lo * 8, vl);
#pragma unroll
                                for (int r = 0; r < MC / 2; ++r)
#pragma unroll
                                    for (int q = 0; q < 4; ++q) vv[r][q] += vl[r][q];
                            }
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
                                // stage II(L): per term, V += A2 (M=64 (c1,i3) x K=16) x F^{t2} (N=16)
                                const int t2 = band_t(a2, cur % 6);
                                for (int mc = iss_lo; mc < iss_hi; ++mc)
                                    tc::mma_f16(tDII + mc * 16, adesc(mc), fdesc(mc, t2), idS, first ? 0u : 1u);
                            } else if (!last) {
                                issue_stage1(xb ^ 1);
                            }
                            tc::commit(&s_mbar);
                        }
                        // line L+2's input blocks into line L's buffer, while the MMAs run
                        if (nn < 36) fetch_line(nn, xb);
                        if (last) {
                            // the plane's last stage II complete: D_II -> stage III A (aliases
                            // stage II A)
                            TC3_WAIT_OR_ABORT();
                            if (aborted) break;
                            tc::fence_after();
                            // D_II -> stage III A (rows (c1, c2), K = i3 as hi | lo).  This thread holds
                            // D_II rows (c1, i3) = (2 quarter, lane/4) and (2 quarter + 1, lane/4),
                            // columns c2 = cA, cA + 1: per term, its fragments of the matrices [i3][c2]
                            // of the two c1, hi and lo, stored transposed
                            {
                                float vv[MC / 2][4];
                                read_dii(vv);
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
                            // stage III: per term, Y = A3 (M=64 (c1,c2) x K=16) x F^{t3} (N=16) into
                            // D_II; the next plane's first stage I into D_I
                            if (issuer) {
                                tc::fence_after();
                                if (warp < 4) {
                                    const int t3 = band_t(a3, q3);
                                    for (int mc = iss_lo; mc < iss_hi; ++mc)
                                        tc::mma_f16(tDII + mc * 16, adesc(mc), fdesc(mc, t3), idS, 0);
                                } else if (nxt < 36) {
                                    issue_stage1(xb ^ 1);
                                }
                                tc::commit(&s_mbar);
                            }
                            y_pending = true;
                            if (nxt >= 36) {  // the chunk's last plane
                                TC3_WAIT_OR_ABORT();
                                if (aborted) break;
                                tc::fence_after();
                                accumulate_y();
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
#undef TC3_WAIT_OR_ABORT
    tc::cp_async_wait_all();
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tbase, L::TMEM_COLS);
}


int tc3_configure() {
    MRA_CK(cudaFuncSetAttribute(k_apply_tc3<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, Tc3Smem<8>::TOTAL));
    MRA_CK(cudaFuncSetAttribute(k_apply_tc3<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, Tc3Smem<8>::TOTAL));
    MRA_CK(cudaFuncSetAttribute(k_apply_tc3<false>, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    MRA_CK(cudaFuncSetAttribute(k_apply_tc3<true>, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    return MRA_OK;
}

// two persistent CTAs per SM, nodes from the work counter (zeroed by the caller)
int tc3_launch(const TcArgs& T, cudaStream_t st) {
    const int grid = std::max(1, std::min(T.nwork, num_sms() * 2));
    if (T.lpb) k_apply_tc3<true><<<grid, TC3_THREADS, Tc3Smem<8>::TOTAL, st>>>(T);
    else k_apply_tc3<false><<<grid, TC3_THREADS, Tc3Smem<8>::TOTAL, st>>>(T);
    MRA_CK_LAUNCH();
    return MRA_OK;
}

}  // namespace mra
