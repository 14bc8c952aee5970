// Operator construction (make_operator), FP64 on the device.
//
//  * two-scale filters H^(0), H^(1) and their orthonormal completion G
//    (Appendix, two-scale relations);
//  * the Gaussian sum of K_{mu,alpha} (Sec. 3, eqs. IntegralRepr and
//    KernelApproxByGaussians), checked on 4000 log-spaced radii, several
//    candidate steps at once;
//  * the 1-D blocks F^{j;m,l} (eq. KernelFactor) from the cross-correlations
//    (eq. CrossCor).  Route: with Proposition 1 item 2 the integral over
//    [-1, 1] folds onto [0, 1],
//      F_ii' = 2^{-j} int_0^1 Phi+_ii'(x) [g(x+l) + (-1)^{i+i'} g(x-l)] dx,
//    g(u) = exp(-tau u^2 / 4^j) (the Appendix's evaluation formula); Phi+ is
//    a polynomial of degree <= 2k - 1, expanded once per k in the Legendre
//    functions of [0, 1] (exact quadratures), so each block needs only the
//    2k Gaussian-weighted Legendre moments, each integrated on the
//    Gaussian's own window |u| <= sqrt(46/c) by composite 16-point
//    Gauss-Legendre panels no wider than min(1/4, 1/(2 sqrt c)), c = tau/4^j;
//  * block norms (eq. BlockNorms, Frobenius) and the 18-term estimate
//    (eq. NormEstimateUsing1DBlocks) maximised over the coarse core.
#include <math.h>

#include "mra_internal.cuh"

namespace mra {

// ------------------------------------------------------------------ filters
// filt layout: H0 (k*k) | H1 (k*k) | W (2k*2k), all row-major.  One warp:
// lanes < k compute the GL rule and the basis tables, every lane some H
// entries, and lane c owns column c of the Gram-Schmidt vectors (the dot
// products are warp sums).
__global__ void k_filters(int k, double* filt) {
    __shared__ double x[MRA_MAX_K], w[MRA_MAX_K];
    __shared__ double pa[2][MRA_MAX_K][MRA_MAX_K], pb[MRA_MAX_K][MRA_MAX_K];
    const int lane = threadIdx.x;
    if (lane < k) gauss_legendre01_root(k, lane, x, w);
    __syncwarp();
    if (lane < k) {
        phi_all(k, 0.5 * x[lane], pa[0][lane]);
        phi_all(k, 0.5 * (x[lane] + 1.0), pa[1][lane]);
        phi_all(k, x[lane], pb[lane]);
    }
    __syncwarp();
    double* H0 = filt;
    double* W = filt + 2 * k * k;
    const int kk = k * k, n2 = 2 * k;
    const double rs2 = 0.70710678118654752440;
    for (int e = lane; e < 2 * kk; e += 32) {
        const int p = e / kk, i = (e % kk) / k, ip = e % k;
        double h = 0.0;
        for (int q = 0; q < k; ++q) h += rs2 * w[q] * pa[p][q][i] * pb[q][ip];
        H0[e] = h;                                  // H1 follows H0
        W[i * n2 + p * k + ip] = h;
    }
    __threadfence_block();
    __syncwarp();
    // Gram-Schmidt (two passes) of (e_i, -e_i)/sqrt 2 against the H rows and
    // the wavelet rows already built
    for (int i = 0; i < k; ++i) {
        double v = lane == i ? rs2 : (lane == k + i ? -rs2 : 0.0);
        for (int pass = 0; pass < 2; ++pass)
            for (int r = 0; r < k + i; ++r) {
                const double wr = lane < n2 ? W[r * n2 + lane] : 0.0;
                double d = wr * v;
                for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
                v -= d * wr;
            }
        double nn = v * v;
        for (int o = 16; o > 0; o >>= 1) nn += __shfl_xor_sync(0xffffffffu, nn, o);
        if (lane < n2) W[(k + i) * n2 + lane] = v / sqrt(nn);
        __syncwarp();
    }
}

int launch_filters(int k, double* filt, cudaStream_t st) {
    k_filters<<<1, 32, 0, st>>>(k, filt);
    MRA_CK_LAUNCH();
    return MRA_OK;
}

// ------------------------------------------------------------- Gaussian sum
// In R^d (d = 3, and d = 2 for the two-dimensional variant) the integral
// representation has C_alpha = 2 * 2^{-2 alpha} pi^{-d/2} / Gamma(alpha) and the
// exponent (d - 2 alpha) s; the mu = 0 kernel is C_alpha Gamma(d/2 - alpha) /
// (2 r^{d - 2 alpha}).
__device__ double c_alpha_dev(double alpha, int d) {
    return 2.0 * exp2(-2.0 * alpha) * pow(3.14159265358979323846, -0.5 * d) / tgamma(alpha);
}

__device__ double kernel_env(double alpha, double r, int d) {  // K_{0,alpha}(r)
    return tgamma(0.5 * d - alpha) * c_alpha_dev(alpha, d) / (2.0 * pow(r, d - 2.0 * alpha));
}

// K_{mu,alpha}(r): closed forms for mu = 0 and (d = 3) alpha = 1; otherwise the
// integral representation (eq. IntegralRepr) by a trapezoid of step 0.02 over
// the window where the integrand exceeds e^-50 (its error decays like
// exp(-pi^2 / (2 * 0.02))).
__device__ double kernel_value(double mu, double alpha, double r, int d) {
    if (mu == 0.0) return kernel_env(alpha, r, d);
    if (alpha == 1.0 && d == 3) return exp(-mu * r) / (4.0 * 3.14159265358979323846 * r);
    double s_hi = 0.5 * log(50.0 / (r * r)) + 1.0;
    double s_lo = 0.5 * log(mu * mu / 200.0) - 1.0;
    const double hq = 0.02;
    double acc = 0.0;
    for (double s = s_lo; s <= s_hi; s += hq)
        acc += exp(-r * r * exp(2.0 * s) - 0.25 * mu * mu * exp(-2.0 * s) + (d - 2.0 * alpha) * s);
    return c_alpha_dev(alpha, d) * hq * acc;
}

// The step h shrinks by 3 % until the sup-norm test passes (the sequence
// h0, 0.97 h0, ... is formed by repeated multiplication, as a sequential
// search would).  GS_CAND candidate steps are tested at once: block
// (c, chunk) evaluates candidate base + c on 256 of the 4000 radii, and the
// per-candidate maxima meet in err_bits (non-negative doubles order like
// their bit patterns).  k_gs_pick then takes the first candidate in sequence
// order that passes -- the same choice the sequential search makes.  Blocks of
// 64 radii spread the FP64 work over many SMs.
#define GS_CAND 16
#define GS_NPTS 4000
#define GS_ITERS 200

// par = {A, B, h0}
__global__ void k_gs_setup(double mu, double alpha, double eps, double delta, double R, int d, double* par) {
    if (threadIdx.x != 0) return;
    const double L = log(1.0 / eps), q = d - 2.0 * alpha;
    double A = log(0.1 * eps * q * tgamma(0.5 * q) / (2.0 * pow(R, q))) / q;
    if (mu > 0.0) A = fmax(A, -0.5 * log(4.0 * (L + 10.0) / (mu * mu)));
    par[0] = A;
    par[1] = 0.5 * log((L + 5.0) / (delta * delta));
    par[2] = 3.14159265358979323846 * 3.14159265358979323846 / (2.0 * L);
}

__device__ inline double gs_step(double h0, int n) {
    double h = h0;
    for (int t = 0; t < n; ++t) h *= 0.97;
    return h;
}

__global__ void __launch_bounds__(256) k_gs_check(double mu, double alpha, double delta, double R, int d,
                                                  const double* par, int base, unsigned long long* err_bits) {
    __shared__ double w[MRA_MAX_TERMS], tau[MRA_MAX_TERMS], red[8];
    const int c = blockIdx.x, tid = threadIdx.x;
    if (base + c >= GS_ITERS) return;
    const double A = par[0], B = par[1], h = gs_step(par[2], base + c);
    const int M = (int)ceil((B - A) / h);
    if (M > MRA_MAX_TERMS) {
        if (tid == 0) atomicMax(&err_bits[c], (unsigned long long)__double_as_longlong(INFINITY));
        return;
    }
    const double Ca = c_alpha_dev(alpha, d);
    for (int m = tid; m < M; m += blockDim.x) {
        const double s = A + (m + 1) * h;
        tau[m] = exp(2.0 * s);
        w[m] = h * Ca * exp(-0.25 * mu * mu * exp(-2.0 * s) + (d - 2.0 * alpha) * s);
    }
    __syncthreads();
    const double lgd = log(delta), lgR = log(R);
    double err = 0.0;
    const int i = blockIdx.y * blockDim.x + tid;
    if (i < GS_NPTS) {
        const double r = exp(lgd + i * (lgR - lgd) / (GS_NPTS - 1.0));
        double sum = 0.0;
        for (int m = 0; m < M; ++m) sum += w[m] * exp(-tau[m] * r * r);
        err = fabs(kernel_value(mu, alpha, r, d) - sum) / kernel_env(alpha, r, d);
        if (!(err == err)) err = INFINITY;  // a NaN fails the test
    }
    for (int o = 16; o > 0; o >>= 1) err = fmax(err, __shfl_xor_sync(0xffffffffu, err, o));
    if ((tid & 31) == 0) red[tid >> 5] = err;
    __syncthreads();
    if (tid == 0) {
        for (int q = 1; q < (int)(blockDim.x >> 5); ++q) err = fmax(err, red[q]);
        atomicMax(&err_bits[c], (unsigned long long)__double_as_longlong(err));
    }
}

// outM: M on success; -2 when more than MRA_MAX_TERMS terms are needed first;
// -1 when no candidate of this batch passes (the host tries the next batch)
__global__ void k_gs_pick(double mu, double alpha, double eps, int d, const double* par, int base,
                          const unsigned long long* err_bits, double* w, double* tau, int* outM,
                          double* par_out_h) {
    __shared__ int pick, M;
    const int tid = threadIdx.x;
    const double A = par[0], B = par[1];
    if (tid == 0) {
        pick = -1;
        M = -1;
        for (int c = 0; c < GS_CAND && base + c < GS_ITERS; ++c) {
            const int Mc = (int)ceil((B - A) / gs_step(par[2], base + c));
            if (Mc > MRA_MAX_TERMS) {
                M = -2;
                break;
            }
            if (__longlong_as_double((long long)err_bits[c]) <= eps) {
                pick = c;
                M = Mc;
                break;
            }
        }
        outM[0] = M;
    }
    __syncthreads();
    if (pick < 0) return;
    const double h = gs_step(par[2], base + pick), Ca = c_alpha_dev(alpha, d);
    if (tid == 0) par_out_h[0] = h;
    for (int m = tid; m < M; m += blockDim.x) {
        const double s = A + (m + 1) * h;
        tau[m] = exp(2.0 * s);
        w[m] = h * Ca * exp(-0.25 * mu * mu * exp(-2.0 * s) + (d - 2.0 * alpha) * s);
    }
}

// Weights of the term grid s_m = A + (m + 1) h for another mu (tau_m = e^{2 s_m}
// does not depend on mu), and the sup-norm test of eq. KernelApproxByGaussians
// for them on the same 4000 radii.
__global__ void k_gs_weights(double mu, double alpha, int d, double A, double h, int M, double* w) {
    const double Ca = c_alpha_dev(alpha, d);
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < M; m += gridDim.x * blockDim.x) {
        const double s = A + (m + 1) * h;
        w[m] = h * Ca * exp(-0.25 * mu * mu * exp(-2.0 * s) + (d - 2.0 * alpha) * s);
    }
}

__global__ void __launch_bounds__(256) k_gs_check_grid(double mu, double alpha, double delta, double R, int d, int M,
                                                       const double* wg, const double* taug,
                                                       unsigned long long* err_bits) {
    __shared__ double w[MRA_MAX_TERMS], tau[MRA_MAX_TERMS], red[8];
    const int tid = threadIdx.x;
    for (int m = tid; m < M; m += blockDim.x) {
        w[m] = wg[m];
        tau[m] = taug[m];
    }
    __syncthreads();
    const double lgd = log(delta), lgR = log(R);
    double err = 0.0;
    const int i = blockIdx.x * blockDim.x + tid;
    if (i < GS_NPTS) {
        const double r = exp(lgd + i * (lgR - lgd) / (GS_NPTS - 1.0));
        double sum = 0.0;
        for (int m = 0; m < M; ++m) sum += w[m] * exp(-tau[m] * r * r);
        err = fabs(kernel_value(mu, alpha, r, d) - sum) / kernel_env(alpha, r, d);
        if (!(err == err)) err = INFINITY;
    }
    for (int o = 16; o > 0; o >>= 1) err = fmax(err, __shfl_xor_sync(0xffffffffu, err, o));
    if ((tid & 31) == 0) red[tid >> 5] = err;
    __syncthreads();
    if (tid == 0) {
        for (int q = 1; q < (int)(blockDim.x >> 5); ++q) err = fmax(err, red[q]);
        atomicMax(err_bits, (unsigned long long)__double_as_longlong(err));
    }
}

// ------------------------------------------------------------------ F tables
// Phi+_ii'(x) = int_0^{1-x} phi_i(x + y) phi_i'(y) dy is a polynomial of degree
// i + i' + 1 <= 2k - 1 on [0, 1], so it equals its expansion in the first 2k
// Legendre functions phi_p of [0, 1]:  Phi+_ii' = sum_p C[(i k + i') 2k + p] phi_p.
// C by the 2k-point rule in x (exact for the degree 4k - 2 integrands) and
// Phi+ by the k-point rule on [0, 1-x] (exact).  Then
//   F_ii' = 2^{-j} sum_p C_ii'p (G+_p + (-1)^{i+i'} G-_p),
//   G+-_p = int_0^1 phi_p(x) exp(-c (x +- l)^2) dx,
// and a block needs only the 2k Gaussian moments G+-_p, each integrated on
// the Gaussian's own window |u| <= sqrt(46/c) by composite 16-point panels no
// wider than min(1/4, 1/(2 sqrt c)), c = tau/4^j.
// grid k^2: block (i, i'); thread (q, g) < (2k, k) evaluates the inner rule's
// term at x-node q and y-node g; the block then forms Phi+ at the 2k x-nodes
// and their projections on phi_p.
__global__ void __launch_bounds__(2 * MRA_MAX_K * MRA_MAX_K) k_xcorr_coeffs(int k, double* C) {
    __shared__ double xk[MRA_MAX_K], wk[MRA_MAX_K], x2[2 * MRA_MAX_K], w2[2 * MRA_MAX_K];
    __shared__ double term[2 * MRA_MAX_K][MRA_MAX_K], phx[2 * MRA_MAX_K];
    const int tid = threadIdx.x, n2 = 2 * k, e = blockIdx.x;
    const int i = e / k, ip = e % k;
    if (tid < k) gauss_legendre01_root(k, tid, xk, wk);
    if (tid >= 32 && tid < 32 + n2) gauss_legendre01_root(n2, tid - 32, x2, w2);
    __syncthreads();
    if (tid < n2 * k) {
        const int q = tid / k, g = tid % k;
        const double x = x2[q], y = (1.0 - x) * xk[g];
        double ta[MRA_MAX_K], tb[MRA_MAX_K];
        phi_all(k, x + y, ta);
        phi_all(k, y, tb);
        term[q][g] = wk[g] * ta[i] * tb[ip];
    }
    __syncthreads();
    if (tid < n2) {
        double phi = 0.0;
        for (int g = 0; g < k; ++g) phi += term[tid][g];
        phx[tid] = w2[tid] * phi * (1.0 - x2[tid]);
    }
    __syncthreads();
    if (tid < n2) {  // thread p: sum over the x-nodes of phx_q phi_p(x_q)
        double c = 0.0, pp[2 * MRA_MAX_K];
        for (int q = 0; q < n2; ++q) {
            phi_all(n2, x2[q], pp);
            c += phx[q] * pp[tid];
        }
        C[(size_t)e * n2 + tid] = c;
    }
}

#define FT_THREADS 128

// grid (7, M, J+1): block (l+3, m, j)
__global__ void __launch_bounds__(FT_THREADS) k_ftable(int k, int M, const double* tau, const double* C, double* F) {
    __shared__ double gx[16], gw[16];
    __shared__ double Cs[MRA_MAX_K * MRA_MAX_K * 2 * MRA_MAX_K];
    __shared__ double G[2][FT_THREADS / 32][2 * MRA_MAX_K];
    __shared__ int npan[2];
    __shared__ double plo[2], pwd[2];
    const int l = (int)blockIdx.x - 3, m = blockIdx.y, j = blockIdx.z;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int n2 = 2 * k, kk = k * k;
    if (tid < 16) gauss_legendre01_root(16, tid, gx, gw);
    for (int e = tid; e < kk * n2; e += blockDim.x) Cs[e] = C[e];
    const double c = tau[m] / exp2(2.0 * j);
    if (tid == 32) {
        const double half = sqrt(46.0 / c);
        const double width = fmin(0.25, 0.5 / sqrt(c));
        for (int side = 0; side < 2; ++side) {  // side 0: g(x+l) peaks at -l; 1: g(x-l) at +l
            const double xc = side ? (double)l : -(double)l;
            const double a = fmax(0.0, xc - half), b = fmin(1.0, xc + half);
            if (b <= a) {
                npan[side] = 0;
                plo[side] = 0.0;
                pwd[side] = 0.0;
            } else {
                const int n = max(1, (int)ceil((b - a) / width));
                npan[side] = n;
                plo[side] = a;
                pwd[side] = (b - a) / n;
            }
        }
    }
    __syncthreads();
    for (int side = 0; side < 2; ++side) {
        double acc[2 * MRA_MAX_K];
#pragma unroll
        for (int p = 0; p < 2 * MRA_MAX_K; ++p) acc[p] = 0.0;
        const int npts = npan[side] * 16;
        const double sh = side ? -(double)l : (double)l;
        for (int q = tid; q < npts; q += blockDim.x) {
            const double x = plo[side] + pwd[side] * ((q >> 4) + gx[q & 15]);
            const double u = x + sh;
            const double wt = pwd[side] * gw[q & 15] * exp(-c * u * u);
            const double v = 2.0 * x - 1.0;
            double p0 = 1.0, p1 = v;
            acc[0] += wt;
            acc[1] += wt * v;
#pragma unroll
            for (int p = 2; p < 2 * MRA_MAX_K; ++p) {
                if (p < n2) {
                    // Legendre recurrence; p is a constant here, so are a and b
                    const double a = (2.0 * p - 1.0) / p, b = (p - 1.0) / p;
                    const double p2 = a * v * p1 - b * p0;
                    acc[p] += wt * p2;
                    p0 = p1;
                    p1 = p2;
                }
            }
        }
#pragma unroll
        for (int p = 0; p < 2 * MRA_MAX_K; ++p) {
            if (p < n2) {
                double sm = acc[p];
                for (int o = 16; o > 0; o >>= 1) sm += __shfl_xor_sync(0xffffffffu, sm, o);
                if (lane == 0) G[side][warp][p] = sm;
            }
        }
    }
    __syncthreads();
    for (int e = tid; e < kk; e += blockDim.x) {
        const int ii = e / k, ip = e % k;
        const double sgn = ((ii + ip) & 1) ? -1.0 : 1.0;
        double f = 0.0;
        for (int p = 0; p < n2; ++p) {
            double gp = 0.0, gm = 0.0;
            for (int q = 0; q < FT_THREADS / 32; ++q) {
                gp += G[0][q][p];
                gm += G[1][q][p];
            }
            f += Cs[e * n2 + p] * sqrt(2.0 * p + 1.0) * (gp + sgn * gm);
        }
        F[((((size_t)j * M + m) * 7 + (l + 3)) * k + ii) * k + ip] = f / exp2((double)j);
    }
}

// ------------------------------------------------------------------- norms
// grid (M, J+1), one warp: nF for l = -3..3; for j >= 1 the 2x2 fine block
// matrices against U F^{j-1;L} U^T for L = -1..1 and the max over the coarse
// core {-1,0,1}^3 of the symmetrised 18-term estimate.
__device__ inline double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void k_norms(int k, int M, int d, const double* F, const double* filt, double* nF, double* est) {
    __shared__ double R[2][MRA_MAX_K * MRA_MAX_K];  // F^{j-1;L} H^(q)
    const int m = blockIdx.x, j = blockIdx.y, lane = threadIdx.x;
    const int kk = k * k;
    auto Fp = [&](int jj, int l) { return F + (((size_t)jj * M + m) * 7 + (l + 3)) * kk; };
    for (int l = -3; l <= 3; ++l) {
        const double* f = Fp(j, l);
        double s = 0.0;
        for (int e = lane; e < kk; e += 32) s += f[e] * f[e];
        s = warp_sum(s);
        if (lane == 0) nF[((size_t)j * M + m) * 7 + l + 3] = sqrt(s);
    }
    if (j == 0) {
        if (lane == 0) est[m] = 0.0;
        return;
    }
    const double* H[2] = {filt, filt + kk};
    double Nd[3], NF[3], NU[3];
    for (int L = -1; L <= 1; ++L) {
        const double* Fc = Fp(j - 1, L);
        double nu = 0.0;
        for (int e = lane; e < 2 * kk; e += 32) {
            const int q = e / kk, i = (e % kk) / k, b = e % k;
            double r = 0.0;
            for (int i2 = 0; i2 < k; ++i2) r += Fc[i * k + i2] * H[q][i2 * k + b];
            R[q][i * k + b] = r;
            if (q == 0) nu += Fc[e] * Fc[e];
        }
        __syncwarp();
        double nff = 0.0, nd = 0.0;
        for (int e = lane; e < 4 * kk; e += 32) {
            const int pq = e / kk, a = (e % kk) / k, b = e % k, p = pq >> 1, q = pq & 1;
            // (U Fc U^T)_{(p,a),(q,b)} = sum_i H^(p)_{i a} (Fc H^(q))_{i b}
            double up = 0.0;
            for (int i = 0; i < k; ++i) up += H[p][i * k + a] * R[q][i * k + b];
            const double fv = Fp(j, 2 * L + p - q)[a * k + b];
            nff += fv * fv;
            nd += (fv - up) * (fv - up);
        }
        __syncwarp();
        Nd[L + 1] = sqrt(warp_sum(nd));
        NF[L + 1] = sqrt(warp_sum(nff));
        NU[L + 1] = sqrt(warp_sum(nu));
    }
    if (lane != 0) return;
    double best = 0.0;
    if (d == 2) {  // two factors: F1 F2 - G1 G2 = (F1 - G1) F2 + G1 (F2 - G2), both orderings
        for (int L1 = 0; L1 < 3; ++L1)
            for (int L2 = 0; L2 < 3; ++L2) {
                const double tot = Nd[L1] * NF[L2] + NU[L1] * Nd[L2] + Nd[L2] * NF[L1] + NU[L2] * Nd[L1];
                best = fmax(best, tot / 2.0);
            }
        est[(size_t)j * M + m] = best;
        return;
    }
    const int perm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    for (int L1 = 0; L1 < 3; ++L1)
        for (int L2 = 0; L2 < 3; ++L2)
            for (int L3 = 0; L3 < 3; ++L3) {
                int Ls[3] = {L1, L2, L3};
                double tot = 0.0;
                for (int s = 0; s < 6; ++s) {
                    int a = Ls[perm[s][0]], b = Ls[perm[s][1]], c = Ls[perm[s][2]];
                    tot += Nd[a] * NF[b] * NF[c] + NU[a] * Nd[b] * NF[c] + NU[a] * NU[b] * Nd[c];
                }
                best = fmax(best, tot / 6.0);
            }
    est[(size_t)j * M + m] = best;
}

__global__ void k_to_float(const double* src, float* dst, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = (float)src[i];
}

int build_operator(mra_op* op, cudaStream_t st) {
    const int k = op->k, J = op->J;
    const Alloc& A = op->A;
    MRA_TRY(dalloc(A, &op->filt, 6 * k * k));
    MRA_TRY(dalloc(A, &op->scratch_i, 4));
    // w and tau are allocated at their largest size and owned by op from here on
    // (mra_free_op releases them on every error return of the caller)
    MRA_TRY(dalloc(A, &op->w, MRA_MAX_TERMS));
    MRA_TRY(dalloc(A, &op->tau, MRA_MAX_TERMS));
    Scratch tmp(A);
    double *par, *C;
    unsigned long long* err_bits;
    MRA_TRY(tmp.get(&par, 4));
    MRA_TRY(tmp.get(&err_bits, GS_CAND));
    MRA_TRY(tmp.get(&C, (size_t)k * k * 2 * k));
    MRA_TRY(launch_filters(k, op->filt, st));
    k_xcorr_coeffs<<<k * k, 2 * MRA_MAX_K * MRA_MAX_K, 0, st>>>(k, C);
    MRA_CK_LAUNCH();
    const double delta = op->eps / 10.0, R = sqrt((double)op->d);
    k_gs_setup<<<1, 32, 0, st>>>(op->mu, op->alpha, op->eps, delta, R, op->d, par);
    MRA_CK_LAUNCH();
    int M = -1;
    for (int base = 0; base < GS_ITERS && M == -1; base += GS_CAND) {
        MRA_CK(cudaMemsetAsync(err_bits, 0, GS_CAND * sizeof(unsigned long long), st));
        k_gs_check<<<dim3(GS_CAND, (GS_NPTS + 63) / 64), 64, 0, st>>>(op->mu, op->alpha, delta, R, op->d, par,
                                                                        base, err_bits);
        MRA_CK_LAUNCH();
        k_gs_pick<<<1, 256, 0, st>>>(op->mu, op->alpha, op->eps, op->d, par, base, err_bits, op->w, op->tau,
                                     op->scratch_i, par + 3);
        MRA_CK_LAUNCH();
        MRA_CK(cudaMemcpyAsync(&M, op->scratch_i, sizeof(int), cudaMemcpyDeviceToHost, st));
        MRA_CK(cudaStreamSynchronize(st));
    }
    double hpar[4] = {0, 0, 0, 0};
    if (M > 0) {
        MRA_CK(cudaMemcpyAsync(hpar, par, sizeof(hpar), cudaMemcpyDeviceToHost, st));
        MRA_CK(cudaStreamSynchronize(st));
        op->gs_A = hpar[0];
        op->gs_h = hpar[3];
    }
    if (M <= 0) {
        set_error("Gaussian-sum construction failed (code %d): more than %d terms or no convergence", M,
                  MRA_MAX_TERMS);
        return MRA_ECUDA;
    }
    op->M = M;
    const size_t nF = (size_t)(J + 1) * M * 7 * k * k;
    MRA_TRY(dalloc(A, &op->F, nF));
    MRA_TRY(dalloc(A, &op->F32, nF));
    MRA_TRY(dalloc(A, &op->nF, (size_t)(J + 1) * M * 7));
    MRA_TRY(dalloc(A, &op->est, (size_t)(J + 1) * M));
    k_ftable<<<dim3(7, M, J + 1), FT_THREADS, 0, st>>>(k, M, op->tau, C, op->F);
    MRA_CK_LAUNCH();
    k_norms<<<dim3(M, J + 1), 32, 0, st>>>(k, M, op->d, op->F, op->filt, op->nF, op->est);
    MRA_CK_LAUNCH();
    k_to_float<<<256, 256, 0, st>>>(op->F, op->F32, nF);
    MRA_CK_LAUNCH();
    // C is released with the Scratch (stream-ordered after the launches above)
    return MRA_OK;
}

// New weights for mu on op's term grid; the tau-dependent tables (F, F32,
// nF, est) are kept.  The grid must pass the sup-norm test for the new mu;
// if it does not, op is left unchanged and MRA_EINVAL is returned.
int retune_operator(mra_op* op, double mu, cudaStream_t st) {
    Scratch tmp(op->A);
    double* w;
    unsigned long long* err_bits;
    MRA_TRY(tmp.get(&w, op->M));
    MRA_TRY(tmp.get(&err_bits, 1));
    MRA_CK(cudaMemsetAsync(err_bits, 0, sizeof(unsigned long long), st));
    k_gs_weights<<<(op->M + 127) / 128, 128, 0, st>>>(mu, op->alpha, op->d, op->gs_A, op->gs_h, op->M, w);
    MRA_CK_LAUNCH();
    const double delta = op->eps / 10.0, R = sqrt((double)op->d);
    k_gs_check_grid<<<(GS_NPTS + 63) / 64, 64, 0, st>>>(mu, op->alpha, delta, R, op->d, op->M, w, op->tau,
                                                         err_bits);
    MRA_CK_LAUNCH();
    unsigned long long bits = 0;
    MRA_CK(cudaMemcpyAsync(&bits, err_bits, sizeof(bits), cudaMemcpyDeviceToHost, st));
    MRA_CK(cudaStreamSynchronize(st));
    double err;
    memcpy(&err, &bits, sizeof(err));
    if (!(err <= op->eps)) {
        set_error("the operator's term grid gives error %.3g > eps = %.3g for mu = %g", err, op->eps, mu);
        return MRA_EINVAL;
    }
    MRA_CK(cudaMemcpyAsync(op->w, w, op->M * sizeof(double), cudaMemcpyDeviceToDevice, st));
    if (op->rmq) {  // the per-pair screen tables hold w_m: rebuilt on next use
        op->A.put(op->rmq);
        op->rmq = nullptr;
        op->rmq_L = 0;
    }
    op->mu = mu;
    MRA_CK(cudaStreamSynchronize(st));
    return MRA_OK;
}

}  // namespace mra
