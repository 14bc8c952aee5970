// Operator construction (make_operator), FP64 on the device.
//
//  * two-scale filters H^(0), H^(1) and their orthonormal completion G
//    (Appendix, two-scale relations);
//  * the Gaussian sum of K_{mu,alpha} (Sec. 3, eqs. IntegralRepr and
//    KernelApproxByGaussians), checked on 4000 log-spaced radii;
//  * the 1-D blocks F^{j;m,l} (eq. KernelFactor) from the cross-correlations
//    (eq. CrossCor).  Route: with Proposition 1 item 2 the integral over
//    [-1, 1] folds onto [0, 1],
//      F_ii' = 2^{-j} int_0^1 Phi+_ii'(x) [g(x+l) + (-1)^{i+i'} g(x-l)] dx,
//    g(u) = exp(-tau u^2 / 4^j) (the Appendix's evaluation formula); Phi+ is
//    evaluated pointwise by k-point Gauss-Legendre on [0, 1-x] (exact), and
//    each Gaussian factor is integrated on its own window |u| <= sqrt(46/c)
//    by composite 16-point Gauss-Legendre panels no wider than
//    min(1/4, 1/(2 sqrt c)), c = tau/4^j;
//  * block norms (eq. BlockNorms, Frobenius) and the 18-term estimate
//    (eq. NormEstimateUsing1DBlocks) maximised over the coarse core.
#include <math.h>

#include "mra_internal.cuh"

namespace mra {

// ------------------------------------------------------------------ filters
// filt layout: H0 (k*k) | H1 (k*k) | W (2k*2k), all row-major.
__global__ void k_filters(int k, double* filt) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double x[MRA_MAX_K], w[MRA_MAX_K], pa[MRA_MAX_K], pb[MRA_MAX_K];
    gauss_legendre01(k, x, w);
    double* H0 = filt;
    double* H1 = filt + k * k;
    double* W = filt + 2 * k * k;
    const double rs2 = 0.70710678118654752440;
    for (int p = 0; p < 2; ++p) {
        double* H = p ? H1 : H0;
        for (int i = 0; i < k * k; ++i) H[i] = 0.0;
        for (int q = 0; q < k; ++q) {
            phi_all(k, 0.5 * (x[q] + p), pa);
            phi_all(k, x[q], pb);
            for (int i = 0; i < k; ++i)
                for (int ip = 0; ip < k; ++ip) H[i * k + ip] += rs2 * w[q] * pa[i] * pb[ip];
        }
    }
    const int n2 = 2 * k;
    for (int i = 0; i < k; ++i)
        for (int c = 0; c < k; ++c) {
            W[i * n2 + c] = H0[i * k + c];
            W[i * n2 + k + c] = H1[i * k + c];
        }
    // Gram-Schmidt (two passes) of (e_i, -e_i)/sqrt 2 against the H rows and
    // the wavelet rows already built.
    for (int i = 0; i < k; ++i) {
        double v[2 * MRA_MAX_K];
        for (int c = 0; c < n2; ++c) v[c] = 0.0;
        v[i] = rs2;
        v[k + i] = -rs2;
        for (int pass = 0; pass < 2; ++pass)
            for (int r = 0; r < k + i; ++r) {
                double d = 0.0;
                for (int c = 0; c < n2; ++c) d += W[r * n2 + c] * v[c];
                for (int c = 0; c < n2; ++c) v[c] -= d * W[r * n2 + c];
            }
        double nn = 0.0;
        for (int c = 0; c < n2; ++c) nn += v[c] * v[c];
        nn = 1.0 / sqrt(nn);
        for (int c = 0; c < n2; ++c) W[(k + i) * n2 + c] = v[c] * nn;
    }
}

int launch_filters(int k, double* filt, cudaStream_t st) {
    k_filters<<<1, 32, 0, st>>>(k, filt);
    MRA_CK_LAUNCH();
    return MRA_OK;
}

// ------------------------------------------------------------- Gaussian sum
__device__ double c_alpha_dev(double alpha) {
    return 2.0 * exp2(-2.0 * alpha) * pow(3.14159265358979323846, -1.5) / tgamma(alpha);
}

__device__ double kernel_env(double alpha, double r) {  // K_{0,alpha}(r)
    return tgamma(1.5 - alpha) * c_alpha_dev(alpha) / (2.0 * pow(r, 3.0 - 2.0 * alpha));
}

// K_{mu,alpha}(r): closed forms for mu = 0 and for alpha = 1; otherwise the
// integral representation (eq. IntegralRepr) by a trapezoid of step 0.02 over
// the window where the integrand exceeds e^-50 (its error decays like
// exp(-pi^2 / (2 * 0.02))).
__device__ double kernel_value(double mu, double alpha, double r) {
    if (mu == 0.0) return kernel_env(alpha, r);
    if (alpha == 1.0) return exp(-mu * r) / (4.0 * 3.14159265358979323846 * r);
    double s_hi = 0.5 * log(50.0 / (r * r)) + 1.0;
    double s_lo = 0.5 * log(mu * mu / 200.0) - 1.0;
    const double hq = 0.02;
    double acc = 0.0;
    for (double s = s_lo; s <= s_hi; s += hq)
        acc += exp(-r * r * exp(2.0 * s) - 0.25 * mu * mu * exp(-2.0 * s) + (3.0 - 2.0 * alpha) * s);
    return c_alpha_dev(alpha) * hq * acc;
}

__global__ void k_gauss_sum(double mu, double alpha, double eps, double delta, double R,
                            double* w, double* tau, int* outM) {
    __shared__ double red[256];
    __shared__ double A, h, Ca;
    __shared__ int M, done;
    const int tid = threadIdx.x;
    if (tid == 0) {
        double L = log(1.0 / eps);
        double q = 3.0 - 2.0 * alpha;
        A = log(0.1 * eps * q * tgamma(1.5 - alpha) / (2.0 * pow(R, q))) / q;
        if (mu > 0.0) A = fmax(A, -0.5 * log(4.0 * (L + 10.0) / (mu * mu)));
        h = 3.14159265358979323846 * 3.14159265358979323846 / (2.0 * L);
        Ca = c_alpha_dev(alpha);
        done = 0;
        outM[0] = -1;
    }
    __syncthreads();
    const double B = 0.5 * log((log(1.0 / eps) + 5.0) / (delta * delta));
    const double lgd = log(delta), lgR = log(R);
    for (int iter = 0; iter < 200 && !done; ++iter) {
        if (tid == 0) M = (int)ceil((B - A) / h);
        __syncthreads();
        if (M > MRA_MAX_TERMS) {
            if (tid == 0) outM[0] = -2;
            return;
        }
        for (int m = tid; m < M; m += blockDim.x) {
            double s = A + (m + 1) * h;
            tau[m] = exp(2.0 * s);
            w[m] = h * Ca * exp(-0.25 * mu * mu * exp(-2.0 * s) + (3.0 - 2.0 * alpha) * s);
        }
        __syncthreads();
        double err = 0.0;
        for (int i = tid; i < 4000; i += blockDim.x) {
            double r = exp(lgd + i * (lgR - lgd) / 3999.0);
            double sum = 0.0;
            for (int m = 0; m < M; ++m) sum += w[m] * exp(-tau[m] * r * r);
            err = fmax(err, fabs(kernel_value(mu, alpha, r) - sum) / kernel_env(alpha, r));
        }
        red[tid] = err;
        __syncthreads();
        for (int s = blockDim.x / 2; s > 0; s >>= 1) {
            if (tid < s) red[tid] = fmax(red[tid], red[tid + s]);
            __syncthreads();
        }
        if (tid == 0) {
            if (red[0] <= eps) {
                done = 1;
                outM[0] = M;
            } else {
                h *= 0.97;
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ F tables
#define FT_THREADS 160
#define FT_CHUNK 16

// grid (7, M, J+1): block (l+3, m, j).  Thread t < k*k owns entry (i, i').
__global__ void __launch_bounds__(FT_THREADS) k_ftable(int k, int M, const double* tau, double* F) {
    extern __shared__ double sm[];
    double* gx = sm;                    // 16 GL nodes
    double* gw = gx + 16;
    double* kx = gw + 16;               // k GL nodes
    double* kw = kx + MRA_MAX_K;
    double* px = kw + MRA_MAX_K;        // chunk points
    double* pwt = px + FT_CHUNK;        // chunk weights (quadrature * Gaussian)
    double* PA = pwt + FT_CHUNK;        // [p][g][i] phi_i(x + (1-x) y_g)
    double* PB = PA + FT_CHUNK * MRA_MAX_K * MRA_MAX_K;  // [p][g][i'] phi_i'((1-x) y_g)
    __shared__ int npan[2];
    __shared__ double plo[2], pwd[2];

    const int l = (int)blockIdx.x - 3, m = blockIdx.y, j = blockIdx.z;
    const int tid = threadIdx.x;
    if (tid == 0) gauss_legendre01(16, gx, gw);
    if (tid == 32) gauss_legendre01(k, kx, kw);
    const double c = tau[m] / exp2(2.0 * j);
    if (tid == 64) {
        const double half = sqrt(46.0 / c);
        const double width = fmin(0.25, 0.5 / sqrt(c));
        for (int side = 0; side < 2; ++side) {  // side 0: g(x+l) peaks at -l; 1: g(x-l) at +l
            double xc = side ? (double)l : -(double)l;
            double a = fmax(0.0, xc - half), b = fmin(1.0, xc + half);
            if (b <= a) {
                npan[side] = 0;
                plo[side] = 0.0;
                pwd[side] = 0.0;
            } else {
                int n = (int)ceil((b - a) / width);
                if (n < 1) n = 1;
                npan[side] = n;
                plo[side] = a;
                pwd[side] = (b - a) / n;
            }
        }
    }
    __syncthreads();
    const int ii = tid / k, ip = tid % k;
    const bool owner = tid < k * k;
    const double sgn = ((ii + ip) & 1) ? -1.0 : 1.0;
    double acc[2] = {0.0, 0.0};
    for (int side = 0; side < 2; ++side) {
        const int npts = npan[side] * 16;
        const double sh = side ? -(double)l : (double)l;  // g(x + sh)
        for (int base = 0; base < npts; base += FT_CHUNK) {
            const int nc = min(FT_CHUNK, npts - base);
            if (tid < nc) {
                int q = base + tid;
                int pan = q / 16, g = q % 16;
                double x = plo[side] + pwd[side] * (pan + gx[g]);
                double u = x + sh;
                px[tid] = x;
                pwt[tid] = pwd[side] * gw[g] * exp(-c * u * u) * (1.0 - x);
            }
            __syncthreads();
            for (int e = tid; e < nc * k; e += blockDim.x) {
                int p = e / k, g = e % k;
                double x = px[p];
                double y = (1.0 - x) * kx[g];
                double tmp[MRA_MAX_K];
                phi_all(k, x + y, tmp);
                for (int i = 0; i < k; ++i) PA[(p * MRA_MAX_K + g) * MRA_MAX_K + i] = tmp[i] * kw[g];
                phi_all(k, y, tmp);
                for (int i = 0; i < k; ++i) PB[(p * MRA_MAX_K + g) * MRA_MAX_K + i] = tmp[i];
            }
            __syncthreads();
            if (owner) {
                double a = 0.0;
                for (int p = 0; p < nc; ++p) {
                    double phi = 0.0;
                    for (int g = 0; g < k; ++g)
                        phi += PA[(p * MRA_MAX_K + g) * MRA_MAX_K + ii] * PB[(p * MRA_MAX_K + g) * MRA_MAX_K + ip];
                    a += pwt[p] * phi;
                }
                acc[side] += a;
            }
            __syncthreads();
        }
    }
    if (owner) {
        size_t base = ((((size_t)j * M + m) * 7 + (l + 3)) * k + ii) * k + ip;
        F[base] = (acc[0] + sgn * acc[1]) / exp2((double)j);
    }
}

// ------------------------------------------------------------------- norms
// grid (M, J+1), one thread: nF for l = -3..3; for j >= 1 the 2x2 fine block
// matrices against U F^{j-1;L} U^T for L = -1..1 and the max over the coarse
// core {-1,0,1}^3 of the symmetrised 18-term estimate.
__global__ void k_norms(int k, int M, const double* F, const double* filt, double* nF, double* est) {
    if (threadIdx.x != 0) return;
    const int m = blockIdx.x, j = blockIdx.y;
    const int kk = k * k;
    auto Fp = [&](int jj, int l) { return F + (((size_t)jj * M + m) * 7 + (l + 3)) * kk; };
    for (int l = -3; l <= 3; ++l) {
        const double* f = Fp(j, l);
        double s = 0.0;
        for (int e = 0; e < kk; ++e) s += f[e] * f[e];
        nF[((size_t)j * M + m) * 7 + l + 3] = sqrt(s);
    }
    double* E = est + (size_t)j * M + m;
    if (j == 0) {
        *E = 0.0;
        return;
    }
    const double* H[2] = {filt, filt + kk};
    double Nd[3], NF[3], NU[3];
    for (int L = -1; L <= 1; ++L) {
        const double* Fc = Fp(j - 1, L);
        double nu = 0.0;
        for (int e = 0; e < kk; ++e) nu += Fc[e] * Fc[e];
        double nff = 0.0, nd = 0.0;
        for (int p = 0; p < 2; ++p)
            for (int q = 0; q < 2; ++q) {
                const double* Ff = Fp(j, 2 * L + p - q);
                for (int a = 0; a < k; ++a)
                    for (int b = 0; b < k; ++b) {
                        // (U Fc U^T)_{(p,a),(q,b)} = sum_{i,i'} H^(p)_{i a} Fc_{i i'} H^(q)_{i' b}
                        double up = 0.0;
                        for (int i = 0; i < k; ++i) {
                            double r = 0.0;
                            for (int i2 = 0; i2 < k; ++i2) r += Fc[i * k + i2] * H[q][i2 * k + b];
                            up += H[p][i * k + a] * r;
                        }
                        double fv = Ff[a * k + b];
                        nff += fv * fv;
                        nd += (fv - up) * (fv - up);
                    }
            }
        Nd[L + 1] = sqrt(nd);
        NF[L + 1] = sqrt(nff);
        NU[L + 1] = sqrt(nu);
    }
    const int perm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    double best = 0.0;
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
    *E = best;
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
    double *w_tmp = op->w, *tau_tmp = op->tau;
    MRA_TRY(launch_filters(k, op->filt, st));
    const double delta = op->eps / 10.0, R = sqrt(3.0);
    k_gauss_sum<<<1, 256, 0, st>>>(op->mu, op->alpha, op->eps, delta, R, w_tmp, tau_tmp, op->scratch_i);
    MRA_CK_LAUNCH();
    int M = 0;
    MRA_CK(cudaMemcpyAsync(&M, op->scratch_i, sizeof(int), cudaMemcpyDeviceToHost, st));
    MRA_CK(cudaStreamSynchronize(st));
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
    size_t smem = (16 * 2 + 2 * MRA_MAX_K + 2 * FT_CHUNK + 2 * FT_CHUNK * MRA_MAX_K * MRA_MAX_K) * sizeof(double);
    static bool attr = false;
    if (!attr) {
        MRA_CK(cudaFuncSetAttribute(k_ftable, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr = true;
    }
    k_ftable<<<dim3(7, M, J + 1), FT_THREADS, smem, st>>>(k, M, op->tau, op->F);
    MRA_CK_LAUNCH();
    k_norms<<<dim3(M, J + 1), 32, 0, st>>>(k, M, op->F, op->filt, op->nF, op->est);
    MRA_CK_LAUNCH();
    k_to_float<<<256, 256, 0, st>>>(op->F, op->F32, nF);
    MRA_CK_LAUNCH();
    return MRA_OK;
}

}  // namespace mra
