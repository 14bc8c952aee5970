// Step 3 of Algorithm 3 on the tcgen05 tensor cores: the double-buffered
// pipeline (two CTAs per SM, 8 terms per chunk, k <= 8).
//
// The same nested sums, operands, scales and precision as k_apply_tc
// (apply_tc.cu): stage I per (t2, t3) line with M = 64 rows (i3, i2), N = 64
// (term, c1), K = 48 (t1, i1); stages II and III per term with [hi | lo]
// packed K = 16; FP32 sums per chunk added to the output in FP64.  What
// differs is the schedule inside a CTA.  With 256 TMEM columns per CTA -- two
// stage-I accumulators, D_II and D_III -- and two buffers for each line's input
// blocks and stage-I B operand, stage I of line L+1 is issued as soon as line
// L's wait ends and runs while the block converts line L's result; the input
// blocks and B operand of line L+2 are prepared while the MMAs of lines L and
// L+1 run.  Per line: one completion wait, then
//   issue stage I(L+1) | convert D_I(L) -> stage II A | barrier | issue stage II(L)
//   | fetch + build line L+2 | barrier
// and after a plane's last line a second wait, the D_II -> stage III A
// conversion and stage III into D_III, read out after the next wait.
#include <cfloat>
#include <climits>

#include "apply_common.cuh"
#include "tc_ptx.cuh"

namespace mra {

#define TC2_THREADS 256
#define TC2_ISSUERS 5
#define TC2_MC 8
#define LADDER2_U 0.00390625

struct Tc2Smem {
    static constexpr int MC = TC2_MC;
    static constexpr int XH = 0;                     // 2 buffers x 6 blocks x 1 KB (hi); buffer p at + p 6144
    static constexpr int XL = 12288;                 // (lo)
    static constexpr int B1 = 24576;                 // 2 buffers x (hi MC 768 | lo MC 768)
    static constexpr int B1_BUF = 2 * MC * 768;
    static constexpr int A2_SBO = 272;               // stage II / III A: per term 8 groups of 8 rows
    static constexpr int A2_TERM = 8 * A2_SBO;
    static constexpr int A2H = B1 + 2 * B1_BUF;
    static constexpr int FSH = A2H + MC * A2_TERM;   // the chunk's F (hi), MC terms x 7 shifts x 128 B
    static constexpr int FSL = FSH + MC * 896;       // (lo)
    static constexpr int FZ = FSL + MC * 896;        // one zero core matrix
    static constexpr int TIN = FZ + 128;             // 216 int: input block per band position
    static constexpr int TLO = TIN + 864;            // 216 int16: term range
    static constexpr int THI = TLO + 432;
    static constexpr int TFL = THI + 432;            // 216 bytes: flags
    static constexpr int TG = (TFL + 216 + 15) / 16 * 16;  // 216 float: g per band position
    static constexpr int MSK = TG + 864;             // 36 x MC bytes
    static constexpr int TOTAL = (MSK + 36 * MC + 127) / 128 * 128;
    static constexpr int TMEM_COLS = 256;            // D_I[0], D_I[1], D_II, D_III: 64 columns each
};
static_assert(2 * (Tc2Smem::TOTAL + 2048) <= 232448, "two CTAs per SM");
static_assert(Tc2Smem::MSK % 8 == 0, "a line's masks are read as one word");

template <bool LADDER>
__global__ void __launch_bounds__(TC2_THREADS, 2) k_apply_tc2(TcArgs T) {
    using L = Tc2Smem;
    constexpr int MC = L::MC;
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) uint64_t s_mbar;
    __shared__ int s_mlo, s_mhi, s_exp_min, s_node;
    __shared__ unsigned int s_xmax_bits;
    __shared__ unsigned long long s_items;
    __shared__ float s_c2[MC], s_c3[MC];
    __shared__ unsigned char s_lm[36];
    __shared__ unsigned char s_order[36];
    __shared__ int s_nl;
    __shared__ unsigned long long s_kg[36];
    __shared__ float s_fin[MC];
    __shared__ int s_cnt[MC];
    __shared__ float s_B[MC];
    __shared__ unsigned char s_low[MC];
    __shared__ int s_all_low;
    __shared__ unsigned long long s_lowi;

    const ApplyArgs& A = T.A;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int kr = T.kr;
    const uint4* FH = (const uint4*)T.Fh;
    const uint4* FL = (const uint4*)T.Fl;
    int* tin = (int*)(sm + L::TIN);
    int16_t* tlo = (int16_t*)(sm + L::TLO);
    int16_t* thi = (int16_t*)(sm + L::THI);
    unsigned char* tfl = sm + L::TFL;
    float* tg = (float*)(sm + L::TG);
    unsigned char* msk = sm + L::MSK;
    auto line_of = [](int c) { return (c % 6) * 6 + c / 6; };
    auto line_masks = [&](int line) -> unsigned long long { return *(const unsigned long long*)(msk + line * 8); };

    for (int e = tid; e < L::TOTAL / 16; e += TC2_THREADS) ((uint4*)sm)[e] = make_uint4(0, 0, 0, 0);
    if (warp == 0) tc::tmem_alloc(&s_tmem, L::TMEM_COLS);
    if (tid == 0) tc::mbar_init(&s_mbar, TC2_ISSUERS);
    tc::fence_async_smem();
    __syncthreads();
    tc::fence_after();
    const uint32_t tbase = s_tmem;
    // TMEM columns: D_I of buffer b at 64 b, D_II at 128, D_III at 192
    const uint32_t tDII = tbase + 128, tDIII = tbase + 192;
    const int quarter = warp & 3, whalf = warp >> 2;
    const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
    const int mc_lo = whalf * (MC / 2), mc_hi = mc_lo + MC / 2;
    const uint32_t idI = tc::idesc_f16(64, 8 * MC), idS = tc::idesc_f16(64, 8);
    const bool issuer = lane == 0 && warp < TC2_ISSUERS;
    const int iss_lo = warp * (MC / 4), iss_hi = iss_lo + MC / 4;
    constexpr int NB1 = (2 * MC * 48 + TC2_THREADS - 1) / TC2_THREADS;
    int b1_src[NB1], b1_mq[NB1];
#pragma unroll
    for (int k = 0; k < NB1; ++k) {
        const int e = tid + k * TC2_THREADS, d48 = e / 48, q1 = (e - 48 * d48) >> 3;
        b1_src[k] = e + 8 * d48;
        b1_mq[k] = (d48 & (MC - 1)) | (q1 << 8);
    }
    uint32_t phase = 0;
    const int rA = quarter * 16 + (lane >> 2), cA = 2 * (lane & 3);
    const uint32_t sbase = tc::smem_u32(sm);
    auto fdesc = [&](int mc, int t, bool hi, bool low) -> uint64_t {
        const uint64_t k8 = (uint64_t)((mc * 7 + t + 3) * 8);
        if (hi && !low) return tc::sdesc(sbase + L::FSH, 0u, 256) + k8;
        const uint64_t base = hi ? tc::sdesc(sbase + L::FSH, L::FZ - L::FSH, 256)
                                 : tc::sdesc(sbase + L::FSL, L::FZ - L::FSL, 256);
        return base + k8 - (k8 << 16);
    };
    auto adesc = [&](int mc) -> uint64_t {
        return tc::sdesc(sbase + L::A2H, 128, L::A2_SBO) + (uint64_t)(mc * (L::A2_TERM / 16));
    };
    const uint32_t a2_row_I = sbase + L::A2H + (lane & 7) * L::A2_SBO + ((lane >> 3) & 1) * 128 +
                              (2 * (warp & 3) + (lane >> 4)) * 16;
    const uint32_t a2_row_II = sbase + L::A2H + (2 * (warp & 3) + (lane >> 4)) * L::A2_SBO +
                               ((lane >> 3) & 1) * 128 + (lane & 7) * 16;

    bool aborted = false;
#define TC2_WAIT_OR_ABORT()                                                         \
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
        for (int q = tid; q < 216; q += TC2_THREADS) tin[q] = INT_MIN;
        if (tid == 0) {
            s_mlo = INT_MAX;
            s_mhi = -1;
            s_exp_min = INT_MAX;
            s_xmax_bits = 0u;
            s_items = 0;
            s_lowi = 0;
        }
        __syncthreads();
        for (int p = p0 + tid; p < p1; p += TC2_THREADS) {
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
            atomicMax(&s_xmax_bits, __float_as_uint(T.xmax[b]));
        }
        __syncthreads();
        const int mlo = s_mlo, mhi = s_mhi;
        const float xmax_node = __uint_as_float(s_xmax_bits);
        const float sx_node = ldexpf(1.0f, s_exp_min - 1);
        for (int q = tid; q < 216; q += TC2_THREADS) {
            const int in = tin[q];
            tg[q] = in == INT_MIN ? 0.0f : sx_node / T.sx[in >= 0 ? in : A.n + (-1 - in)];
        }
        float yc[4];
        double yd[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            yc[c] = 0.0f;
            yd[c] = 0.0;
        }
        unsigned my_items = 0;
        if (mhi >= mlo && xmax_node > 0.0f) {
            for (int m0 = mlo; m0 <= mhi && !aborted; m0 += MC) {
                const size_t fbase = ((size_t)j * A.M + m0) * 56;
                {
                    const int nv = MC * 56, nvalid = min(MC, mhi - m0 + 1) * 56;
                    for (int e = tid; e < 2 * nv; e += TC2_THREADS) {
                        const int hl = e >= nv, r = hl ? e - nv : e;
                        uint4* dst = (uint4*)(sm + (hl ? L::FSL : L::FSH)) + r;
                        if (r < nvalid)
                            tc::cp_async16(dst, (hl ? FL : FH) + fbase + r);
                        else
                            *dst = make_uint4(0, 0, 0, 0);
                    }
                    tc::cp_async_commit();
                }
                for (int e = tid; e < 36 * MC; e += TC2_THREADS) {
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
                            int em, ex, ef, e1, e2;
                            const float fm = frexpf(mf, &em), fx = frexpf(xmax_node, &ex);
                            frexpf(sf, &ef);
                            ef -= 1;
                            frexpf(8192.0f / (48.0f * fm * fx), &e1);
                            frexpf(8192.0f / (2304.0f * fm * fm * fx), &e2);
                            const int eW = min(e1 - 1 - em - ex, 126), eV = min(e2 - 1 - 2 * em - ex, 126);
                            if (eW >= -126 && eV >= -126) {
                                c2 = ldexpf(1.0f, eW - ef - (s_exp_min - 1));
                                c3 = ldexpf(1.0f, eV - eW - ef);
                                fin = ldexpf((float)A.w[m], -(eV + ef));
                                if (!(fin <= FLT_MAX)) {
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
                tc::cp_async_wait_all();
                __syncthreads();
                if (LADDER)
                    for (int e = tid; e < 36 * MC; e += TC2_THREADS) {
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
                    unsigned long long km = line_masks(tid);
                    km |= km >> 32;
                    km |= km >> 16;
                    km |= km >> 8;
                    s_lm[tid] = (unsigned char)km;
                    if (m0 == mlo) {
                        unsigned long long kg = 0;
                        for (int q1 = 0; q1 < 6; ++q1)
                            kg |= (unsigned long long)((__float_as_uint(tg[q1 * 36 + tid]) >> 23) & 0xffu) << (8 * q1);
                        s_kg[tid] = kg;
                    }
                }
                if (warp == 2) {
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
                        int all = 1;
                        const double per_term = lp_node / (double)(mhi - mlo + 1);
                        for (int mc = 0; mc < MC; ++mc) {
                            const int m = m0 + mc;
                            int low = 1;
                            if (m <= mhi) low = T.lpb && LADDER2_U * A.w[m] * (double)s_B[mc] <= per_term;
                            s_low[mc] = (unsigned char)low;
                            if (low) s_lowi += s_cnt[mc];
                            all &= low;
                        }
                        s_all_low = all;
                    }
                    __syncthreads();
                }
                const int all_low = LADDER ? s_all_low : 0;
                // per B1 buffer: the masks and g exponents it was last built for
                unsigned long long built_m0 = ~0ull, built_g0 = ~0ull, built_m1 = ~0ull, built_g1 = ~0ull;
                auto fetch_line = [&](int c, int buf) {
                    const int line = line_of(c);
                    const unsigned lmx = s_lm[line];
                    const int nfe = all_low ? 384 : 768;
#pragma unroll
                    for (int k = 0; k < 768 / TC2_THREADS; ++k) {
                        const int e = tid + k * TC2_THREADS;
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
                auto build_B = [&](int c, int buf) {
                    const int lineb = line_of(c);
                    const unsigned long long km = line_masks(lineb), kg = s_kg[lineb];
                    if (buf == 0) {
                        if (km == built_m0 && kg == built_g0) return;
                        built_m0 = km;
                        built_g0 = kg;
                    } else {
                        if (km == built_m1 && kg == built_g1) return;
                        built_m1 = km;
                        built_g1 = kg;
                    }
                    const int nb1 = all_low ? MC * 48 : 2 * MC * 48;
                    const unsigned char* mline = msk + lineb * MC;
                    const float* gline = tg + lineb;
                    const uint4* fs = (const uint4*)(sm + L::FSH) + 8 * (a1 & 1);
                    uint4* b1 = (uint4*)(sm + L::B1 + buf * L::B1_BUF);
#pragma unroll
                    for (int k = 0; k < NB1; ++k) {
                        const int e = tid + k * TC2_THREADS;
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
                        if (e < nb1) b1[e] = out;
                    }
                };
                auto issue_stage1 = [&](int buf, uint32_t d) {
                    const uint64_t a0 = tc::sdesc(sbase + L::XH + buf * 6144, 1024, 128);
                    const uint64_t b0 = tc::sdesc(sbase + L::B1 + buf * L::B1_BUF, 128, 768);
#pragma unroll
                    for (int ks = 0; ks < 3; ++ks) {
                        const uint64_t ah = a0 + ks * 128, al = ah + (L::XL - L::XH) / 16;
                        const uint64_t bh = b0 + ks * 16, bl = bh + (MC * 768) / 16;
                        tc::mma_f16(d, ah, bh, idI, ks > 0);
                        if (!all_low) {
                            tc::mma_f16(d, ah, bl, idI, 1);
                            tc::mma_f16(d, al, bh, idI, 1);
                        }
                    }
                };
                auto accumulate_y = [&]() {
                    float yv[MC / 2][4];
                    tc::tmem_ld16x256_rep<MC / 2>(tDIII + lane_off + mc_lo * 8, yv);
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
                const int nl = s_nl;
                if (nl > 0) {
                    // prologue: lines 0 and 1 prepared, stage I(0) issued
                    fetch_line(s_order[0], 0);
                    build_B(s_order[0], 0);
                    if (nl > 1) {
                        fetch_line(s_order[1], 1);
                        build_B(s_order[1], 1);
                    }
                    tc::cp_async_wait_all();
                    tc::fence_async_smem();
                    __syncthreads();
                    // (test hook: with T.withhold nothing is sent, so the first wait can
                    // only end by its limit, with no MMA in flight)
                    if (issuer && !T.withhold) {
                        tc::fence_after();
                        if (warp == 4) issue_stage1(0, tbase);
                        tc::commit(&s_mbar);
                    }
                    bool first = true, y_pending = false;
                    for (int li = 0; li < nl; ++li) {
                        const int cur = s_order[li];
                        const int nxt = li + 1 < nl ? s_order[li + 1] : 36;
                        const int nn = li + 2 < nl ? s_order[li + 2] : 36;
                        const int bc = li & 1;  // buffers of line L (X, B1, D_I)
                        // stage I(L), and everything issued before it, complete
                        TC2_WAIT_OR_ABORT();
                        if (aborted) break;
                        tc::fence_after();
                        // stage I(L+1) at once: its operands were made ready one line ago
                        if (issuer && warp == 4 && nxt < 36) issue_stage1(bc ^ 1, tbase + 64 * (bc ^ 1));
                        if (y_pending) {  // the previous plane's stage III
                            accumulate_y();
                            y_pending = false;
                        }
                        // D_I(L) -> stage II A (rows (c1, i3), K = i2 as hi | lo)
                        {
                            float vv[MC / 2][4];
                            tc::tmem_ld16x256_rep<MC / 2>(tbase + 64 * bc + lane_off + mc_lo * 8, vv);
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
                        const bool last = nxt >= 36 || nxt / 6 != q3;
                        tc::fence_before();
                        tc::fence_async_smem();
                        __syncthreads();
                        if (issuer) {
                            tc::fence_after();
                            if (warp < 4) {
                                const int t2 = band_t(a2, cur % 6);
                                for (int mc = iss_lo; mc < iss_hi; ++mc) {
                                    const bool low = LADDER && s_low[mc];
                                    const uint64_t a = adesc(mc);
                                    tc::mma_f16(tDII + mc * 8, a, fdesc(mc, t2, true, low), idS, first ? 0u : 1u);
                                    if (!low) tc::mma_f16(tDII + mc * 8, a, fdesc(mc, t2, false, false), idS, 1);
                                }
                            }
                            tc::commit(&s_mbar);  // stage II(L), and warp 4's stage I(L+1)
                        }
                        // line L+2 into line L's buffers while the MMAs run
                        if (nn < 36) {
                            fetch_line(nn, bc);
                            build_B(nn, bc);
                        }
                        if (last) {
                            TC2_WAIT_OR_ABORT();
                            if (aborted) break;
                            tc::fence_after();
                            // D_II -> stage III A (rows (c1, c2), K = i3 as hi | lo)
                            {
                                float vv[MC / 2][4];
                                tc::tmem_ld16x256_rep<MC / 2>(tDII + lane_off + mc_lo * 8, vv);
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
                            if (issuer) {
                                tc::fence_after();
                                if (warp < 4) {
                                    const int t3 = band_t(a3, q3);
                                    for (int mc = iss_lo; mc < iss_hi; ++mc) {
                                        const bool low = LADDER && s_low[mc];
                                        const uint64_t a = adesc(mc);
                                        tc::mma_f16(tDIII + mc * 8, a, fdesc(mc, t3, true, low), idS, 0);
                                        if (!low) tc::mma_f16(tDIII + mc * 8, a, fdesc(mc, t3, false, false), idS, 1);
                                    }
                                }
                                tc::commit(&s_mbar);
                            }
                            y_pending = true;
                        }
                        first = last;
                        tc::cp_async_wait_all();  // line L+2's input blocks
                        tc::fence_async_smem();
                        __syncthreads();
                    }
                    if (!aborted && y_pending) {  // the chunk's last plane
                        TC2_WAIT_OR_ABORT();
                        if (!aborted) {
                            tc::fence_after();
                            accumulate_y();
                        }
                    }
                    tc::cp_async_wait_all();
                }
                if (aborted) break;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    yd[q] += (double)yc[q];
                    yc[q] = 0.0f;
                }
                tc::fence_before();
                __syncthreads();
            }
        }
        double* ysm = (double*)(sm + L::XH);
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
#undef TC2_WAIT_OR_ABORT
    tc::cp_async_wait_all();
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tbase, L::TMEM_COLS);
}

int tc2_configure() {
    MRA_CK(cudaFuncSetAttribute(k_apply_tc2<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, Tc2Smem::TOTAL));
    MRA_CK(cudaFuncSetAttribute(k_apply_tc2<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, Tc2Smem::TOTAL));
    MRA_CK(cudaFuncSetAttribute(k_apply_tc2<false>, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    MRA_CK(cudaFuncSetAttribute(k_apply_tc2<true>, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    return MRA_OK;
}

// one CTA pair per SM (two CTAs of 256 threads), nodes from the work counter
int tc2_launch(const TcArgs& T, cudaStream_t st) {
    const int grid = std::max(1, std::min(T.nwork, num_sms() * 2));
    if (T.lpb) k_apply_tc2<true><<<grid, TC2_THREADS, Tc2Smem::TOTAL, st>>>(T);
    else k_apply_tc2<false><<<grid, TC2_THREADS, Tc2Smem::TOTAL, st>>>(T);
    MRA_CK_LAUNCH();
    return MRA_OK;
}

}  // namespace mra
