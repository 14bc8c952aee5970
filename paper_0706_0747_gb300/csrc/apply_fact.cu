// Step 3 of Algorithm 3 in the factorised order of its own formula:
//
//   ghat_a = sum_m w_m sum_{t3} F^{m,t3} x_3 [ sum_{t2} F^{m,t2} x_2 [ sum_{t1} F^{m,t1} x_1 f_{a-t} ] ]
//
// (the nested sums over l1', l2', l3' written out for d = 3 in Sec. 5).  The
// direction-1 contraction is done once per kept item (a, t, m), the
// direction-2 one once per (t2, t3) line and the direction-3 one once per t3
// plane, instead of all three per item.  The item set is exactly the
// screen's: the kept-item test (pair present, m in its range, J_m rules)
// masks the innermost sum only, so the result equals the per-item sum up to
// the order of additions.
//
// Block per output node (grid-stride).  Per chunk of MC consecutive terms:
// F^{j;m,t} for the chunk, a 36 x MC table of 6-bit masks of kept t1 per
// line, then plane by plane: the line's input blocks are staged once and
// reused by every term of the chunk.
#include <climits>

#include "apply_common.cuh"

namespace mra {

template <class T, int K, int MC, int NT>
__global__ void __launch_bounds__(NT) k_apply_fact(ApplyArgs A) {
    constexpr int K2 = K * K, K3 = K2 * K;
    extern __shared__ __align__(16) unsigned char smraw[];
    double* y = (double*)smraw;              // K3
    T* X = (T*)(y + K3);                      // 6 K3  (one line of input blocks)
    T* W = X + 6 * K3;                        // K3
    T* V = W + K3;                            // MC K3 (per-term plane accumulators)
    T* Fs = V + MC * K3;                      // MC * 7 * K2
    int* tin = (int*)(Fs + MC * 7 * K2);      // 216 input refs (INT_MIN: no pair)
    int* tlo = tin + 216;                     // 216 m_lo
    int* thi = tlo + 216;                     // 216 m_hi
    int* tfl = thi + 216;                     // 216 flags
    unsigned char* msk = (unsigned char*)(tfl + 216);  // 36 * MC
    __shared__ int s_mlo, s_mhi, s_anyv[MC];
    __shared__ unsigned long long s_items;

    const int tid = threadIdx.x;
    const T* Ftab = (const T*)A.F;
    for (int node = blockIdx.x; node < A.n; node += gridDim.x) {
        const int j = A.coord[4 * node];
        const int a1 = A.coord[4 * node + 1], a2 = A.coord[4 * node + 2], a3 = A.coord[4 * node + 3];
        const int p0 = A.pair_off[node], p1 = A.pair_off[node + 1];
        const int32_t* Jm = A.Jm + (A.node_tree ? A.node_tree[node] * A.jm_stride : 0);
        for (int e = tid; e < K3; e += NT) y[e] = 0.0;
        for (int q = tid; q < 216; q += NT) tin[q] = INT_MIN;
        if (tid == 0) {
            s_mlo = INT_MAX;
            s_mhi = -1;
            s_items = 0;
        }
        __syncthreads();
        // scatter the node's pairs into the 6x6x6 band table (q = q1*36+q2*6+q3)
        for (int p = p0 + tid; p < p1; p += NT) {
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
        }
        __syncthreads();
        const int mlo = s_mlo, mhi = s_mhi;
        for (int m0 = mlo; m0 <= mhi; m0 += MC) {
            // operator blocks of the chunk and the kept-t1 masks per line
            for (int e = tid; e < MC * 7 * K2; e += NT) {
                const int mc = e / (7 * K2), r = e % (7 * K2);
                const int m = m0 + mc;
                Fs[e] = (m <= mhi) ? Ftab[((size_t)j * A.M + m) * 7 * K2 + r] : (T)0;
            }
            for (int e = tid; e < 36 * MC; e += NT) {
                const int line = e / MC, mc = e % MC, m = m0 + mc;
                unsigned char mk = 0;
                if (m <= mhi) {
                    const int jm = Jm[m];
                    if (jm >= j)
                        for (int q1 = 0; q1 < 6; ++q1) {
                            const int q = q1 * 36 + line;
                            if (tin[q] == INT_MIN || m < tlo[q] || m > thi[q]) continue;
                            if ((tfl[q] & 1) && jm > j) continue;
                            mk |= (unsigned char)(1u << q1);
                        }
                }
                msk[e] = mk;
            }
            __syncthreads();
            for (int q3 = 0; q3 < 6; ++q3) {
                const int t3 = band_t(a3, q3);
                for (int e = tid; e < MC * K3; e += NT) V[e] = (T)0;
                if (tid < MC) s_anyv[tid] = 0;
                __syncthreads();
                for (int q2 = 0; q2 < 6; ++q2) {
                    const int line = q2 * 6 + q3;
                    unsigned lm = 0;
                    for (int mc = 0; mc < MC; ++mc) lm |= msk[line * MC + mc];
                    if (!lm) continue;  // uniform across the block
                    const int t2 = band_t(a2, q2);
                    // stage the line's input blocks
                    for (int e = tid; e < 6 * K3; e += NT) {
                        const int q1 = e / K3, r = e % K3;
                        T v = (T)0;
                        if (lm & (1u << q1)) {
                            const int in = tin[q1 * 36 + line];
                            const double* src = in >= 0 ? A.s + (size_t)in * K3 : A.gblk + (size_t)(-1 - in) * K3;
                            v = (T)src[r];
                        }
                        X[e] = v;
                    }
                    __syncthreads();
                    for (int mc = 0; mc < MC; ++mc) {
                        const unsigned mk = msk[line * MC + mc];
                        if (!mk) continue;
                        const T* Fm = Fs + mc * 7 * K2;
                        // W[c1][i2][i3] = sum_{kept t1} sum_i1 F^{t1}[c1][i1] X_{t1}[i1][i2][i3]
                        for (int idx = tid; idx < K3; idx += NT) {
                            const int c1 = idx / K2, r = idx % K2;
                            T acc = (T)0;
#pragma unroll
                            for (int q1 = 0; q1 < 6; ++q1) {
                                if (!(mk & (1u << q1))) continue;
                                const T* F1 = Fm + (band_t(a1, q1) + 3) * K2 + c1 * K;
                                const T* x = X + q1 * K3 + r;
#pragma unroll
                                for (int i1 = 0; i1 < K; ++i1) acc += F1[i1] * x[i1 * K2];
                            }
                            W[idx] = acc;
                        }
                        if (tid == 0) {
                            s_items += __popc(mk);
                            s_anyv[mc] = 1;
                        }
                        __syncthreads();
                        // V[c1][c2][i3] += sum_i2 F^{t2}[c2][i2] W[c1][i2][i3]
                        {
                            const T* F2 = Fm + (t2 + 3) * K2;
                            T* Vm = V + mc * K3;
                            for (int idx = tid; idx < K3; idx += NT) {
                                const int c1 = idx / K2, c2 = (idx / K) % K, i3 = idx % K;
                                T acc = (T)0;
#pragma unroll
                                for (int i2 = 0; i2 < K; ++i2) acc += F2[c2 * K + i2] * W[(c1 * K + i2) * K + i3];
                                Vm[idx] += acc;
                            }
                        }
                        __syncthreads();
                    }
                }
                // y[c1][c2][c3] += w_m sum_i3 F^{t3}[c3][i3] V[c1][c2][i3]
                for (int mc = 0; mc < MC; ++mc) {
                    if (!s_anyv[mc]) continue;
                    const T* F3 = Fs + mc * 7 * K2 + (t3 + 3) * K2;
                    const T* Vm = V + mc * K3;
                    const double wm = A.w[m0 + mc];
                    for (int idx = tid; idx < K3; idx += NT) {
                        const int r = idx - idx % K, c3 = idx % K;
                        T acc = (T)0;
#pragma unroll
                        for (int i3 = 0; i3 < K; ++i3) acc += F3[c3 * K + i3] * Vm[r + i3];
                        y[idx] += wm * (double)acc;
                    }
                }
                __syncthreads();
            }
        }
        for (int e = tid; e < K3; e += NT) A.out[(size_t)node * K3 + e] = y[e];
        if (tid == 0 && A.n_items) atomicAdd(A.n_items + (A.node_tree ? A.node_tree[node] : 0), s_items);
        __syncthreads();
    }
}

template <class T, int K>
static int launch_k(const ApplyArgs& A, cudaStream_t st) {
    // terms per chunk: as many as the per-term plane accumulators allow
    constexpr int MC = (K <= 8) ? 8 : (K <= 10 ? 4 : 2), NT = 256;
    constexpr int K2 = K * K, K3 = K2 * K;
    const size_t smem = K3 * sizeof(double) + (size_t)(6 * K3 + K3 + MC * K3 + MC * 7 * K2) * sizeof(T) +
                        4 * 216 * sizeof(int) + 36 * MC;
    auto fn = k_apply_fact<T, K, MC, NT>;
    MRA_CK(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int nb = std::min(A.n, num_sms() * 8);
    fn<<<nb, NT, smem, st>>>(A);
    MRA_CK_LAUNCH();
    return MRA_OK;
}

template <class T>
static int launch_t(const ApplyArgs& A, cudaStream_t st) {
    switch (A.k) {
        case 1: return launch_k<T, 1>(A, st);
        case 2: return launch_k<T, 2>(A, st);
        case 3: return launch_k<T, 3>(A, st);
        case 4: return launch_k<T, 4>(A, st);
        case 5: return launch_k<T, 5>(A, st);
        case 6: return launch_k<T, 6>(A, st);
        case 7: return launch_k<T, 7>(A, st);
        case 8: return launch_k<T, 8>(A, st);
        case 9: return launch_k<T, 9>(A, st);
        case 10: return launch_k<T, 10>(A, st);
        case 11: return launch_k<T, 11>(A, st);
        case 12: return launch_k<T, 12>(A, st);
    }
    set_error("k=%d not supported by the factorised apply", A.k);
    return MRA_EINVAL;
}

int launch_apply_fact(const ApplyArgs& A, int precision, cudaStream_t st) {
    if (precision == MRA_PREC_FP64) return launch_t<double>(A, st);
    return launch_t<float>(A, st);
}

}  // namespace mra
