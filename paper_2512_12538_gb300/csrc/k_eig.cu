// k_eig.cu -- leaf solves through the eigenbasis of the column pencil.
//
// A leaf band of b rows and Sx columns, ordered column by column, is block tridiagonal
// (the subdomain matrices A~_i of Eq. (2), Sec. 1-2):
//     D_i = w_i K + (cx_i - i kh bx_i) W,   L_i = U_{i-1} = -W,
// with K = Y - (kh)^2 W - i kh E the band's line operator (Y the second difference
// along the band, E its two edge rows), W = diag(row weights), w_i, cx_i, bx_i the
// column weight, x-stencil diagonal and x-boundary flag.  Every block is a combination
// of K and W, so with the generalised eigenvectors K V = W V Lambda, normalised
// V^T W V = I, the Schur recursion S_i = D_i - L_i S_{i-1}^{-1} U_i of the block
// factorisation keeps the form S_i^{-1} = V diag(xi_i) V^T with the scalar recursions
//     xi_{0,m} = 1 / delta_{0,m},   xi_{i,m} = 1 / (delta_{i,m} - xi_{i-1,m}),
//     delta_{i,m} = w_i lambda_m + cx_i - i kh bx_i,
// i.e. it is the same recursion, evaluated in the basis where it decouples.  The block
// forward/backward substitution then becomes: f^ = V^T f (one dense b x b contraction
// over every column and right-hand side), the scalar recursions
//     y_i = xi_i (f^_i + y_{i-1}),  x_{n-1} = y_{n-1},  x_i = y_i + xi_i x_{i+1},
// and x = V x^ (a second contraction).
//
// Eigenpairs: V = W^{-1/2} Q with Q the eigenvectors of the complex symmetric
// tridiagonal W^{-1/2} K W^{-1/2}; eigenvalues by the Aberth-Ehrlich simultaneous
// iteration on its characteristic polynomial, eigenvectors by inverse iteration with a
// pivoted tridiagonal LU, normalised q^T q = 1 (no conjugation).
#include <algorithm>

#include "kernels.h"

namespace hh {

static constexpr int EIG_BMAX = 136;     // rows of a leaf band supported by the eigenbasis path

// ------------------------------------------------------------ complex helpers
template <typename R> __device__ __forceinline__ R cabs_(cplx<R> z) { return hypot(z.re, z.im); }
template <typename R> __device__ __forceinline__ cplx<R> cdiv_(cplx<R> a, cplx<R> b) {
    // Smith's algorithm for a / b
    if (fabs(b.re) >= fabs(b.im)) {
        const R r = b.im / b.re, den = b.re + b.im * r;
        return {(a.re + a.im * r) / den, (a.im - a.re * r) / den};
    }
    const R r = b.re / b.im, den = b.re * r + b.im;
    return {(a.re * r + a.im) / den, (a.im * r - a.re) / den};
}
// principal square root from |z|: re = sqrt((|z| + x)/2), im = y / (2 re), with the
// cancellation-free branch for x < 0.
template <typename R> __device__ __forceinline__ cplx<R> csqrt_(cplx<R> z) {
    const R r = cabs_(z);
    if (r == (R)0) return {0, 0};
    const R t = sqrt((R)0.5 * (r + fabs(z.re)));
    if (z.re >= (R)0) return {t, z.im / ((R)2 * t)};
    return {fabs(z.im) / ((R)2 * t), copysign(t, z.im)};
}
template <typename R> struct Eps;
template <> struct Eps<float> { static constexpr float v = 1.1920929e-07f; static constexpr float tiny = 1e-5f; };
template <> struct Eps<double> { static constexpr double v = 2.220446049250313e-16; static constexpr double tiny = 1e-12; };

// Complex symmetric tridiagonal line operator of a band (b rows), scaled
// W^{-1/2} K W^{-1/2}: diagonal d_a and coupling e_a between rows a and a+1.
template <typename R>
__device__ __forceinline__ void band_tridiag(int b, double kh, int a, cplx<R>& d, cplx<R>& e) {
    const double wa = wrow(a, b);
    const bool edge = (a == 0 || a == b - 1);
    const double cy = edge ? 1.0 : 2.0;
    d = {(R)((cy - kh * kh * wa) / wa), (R)(-(edge ? kh : 0.0) / wa)};
    e = {(R)(a < b - 1 ? -1.0 / sqrt(wa * wrow(a + 1, b)) : 0.0), (R)0};
}

// Newton correction p(z) / p'(z) of the characteristic polynomial p of the tridiagonal
// matrix, from the ratios r_j = p_j / p_{j-1} of its leading principal minors:
//   r_0 = d_0 - z,  r_j = d_j - z - e_{j-1}^2 / r_{j-1},
//   r'_j = -1 + e_{j-1}^2 r'_{j-1} / r_{j-1}^2,   p'/p = sum_j r'_j / r_j.
// A ratio that vanishes is replaced by a tiny value (the usual Sturm-sequence guard).
template <typename R>
__device__ cplx<R> newton_step(const cplx<R>* d, const cplx<R>* e2, int b, cplx<R> z) {
    const R tiny = Eps<R>::tiny;
    cplx<R> r = d[0] - z;
    if (cabs_(r) < tiny) r = {tiny, 0};
    cplx<R> rp = {(R)-1, 0};
    cplx<R> ir = cdiv_(cplx<R>{1, 0}, r);
    cplx<R> s = rp * ir;
    for (int j = 1; j < b; ++j) {
        const cplx<R> q = e2[j - 1] * ir;          // e^2 / r
        cplx<R> rn = d[j] - z - q;
        if (cabs_(rn) < tiny) rn = {tiny, 0};
        rp = cplx<R>{(R)-1, 0} + q * (rp * ir);
        r = rn;
        ir = cdiv_(cplx<R>{1, 0}, r);
        s = s + rp * ir;
    }
    return cdiv_(cplx<R>{1, 0}, s);
}

// Inverse iteration for the eigenvector of eigenvalue mu: (T - mu) x = x_prev with a
// pivoted tridiagonal LU (row interchanges between neighbours), three iterations,
// normalised q^T q = 1 (complex symmetric, no conjugation).
template <typename R>
__device__ void inverse_iteration(int b, double kh, cplx<R> mu, cplx<R>* x, cplx<R>* ws) {
    using C = cplx<R>;
    C* dg = ws;
    C* up = ws + b;
    C* up2 = ws + 2 * b;
    C* lo = ws + 3 * b;
    R* sw = (R*)(ws + 4 * b);   // interchange flags
    for (int a = 0; a < b; ++a) {
        C d, e;
        band_tridiag<R>(b, kh, a, d, e);
        dg[a] = d - mu;
        up[a] = e;
        up2[a] = {0, 0};
        x[a] = {(R)(1.0 + 1e-3 * a), (R)(1e-3 * (a % 7))};
    }
    for (int j = 0; j < b - 1; ++j) {
        C dsub, esub;
        band_tridiag<R>(b, kh, j, dsub, esub);   // esub = sub-diagonal entry (j+1, j)
        if (cabs_(dg[j]) >= cabs_(esub)) {
            sw[j] = 0;
            const C fact = cabs_(dg[j]) > (R)0 ? cdiv_(esub, dg[j]) : C{0, 0};
            lo[j] = fact;
            dg[j + 1] = dg[j + 1] - fact * up[j];
        } else {
            sw[j] = 1;
            const C fact = cdiv_(dg[j], esub);
            dg[j] = esub;
            lo[j] = fact;
            const C temp = up[j];
            up[j] = dg[j + 1];
            dg[j + 1] = temp - fact * dg[j + 1];
            if (j < b - 2) {
                up2[j] = up[j + 1];
                up[j + 1] = -(fact * up[j + 1]);
            }
        }
    }
    for (int a = 0; a < b; ++a)
        if (cabs_(dg[a]) < Eps<R>::tiny * Eps<R>::v) dg[a] = {Eps<R>::tiny * Eps<R>::v, 0};
    for (int it = 0; it < 3; ++it) {
        for (int j = 0; j < b - 1; ++j) {
            if (sw[j] == (R)0) {
                x[j + 1] = x[j + 1] - lo[j] * x[j];
            } else {
                const C t = x[j];
                x[j] = x[j + 1];
                x[j + 1] = t - lo[j] * x[j];
            }
        }
        x[b - 1] = cdiv_(x[b - 1], dg[b - 1]);
        if (b > 1) x[b - 2] = cdiv_(x[b - 2] - up[b - 2] * x[b - 1], dg[b - 2]);
        for (int j = b - 3; j >= 0; --j) x[j] = cdiv_(x[j] - up[j] * x[j + 1] - up2[j] * x[j + 2], dg[j]);
        R mx = 0;
        for (int a = 0; a < b; ++a) mx = fmax(mx, cabs_(x[a]));
        const R inv = mx > (R)0 ? (R)1 / mx : (R)1;
        for (int a = 0; a < b; ++a) x[a] = inv * x[a];
    }
    C qq = {0, 0};
    for (int a = 0; a < b; ++a) qq = qq + x[a] * x[a];
    const C nr = csqrt_(qq);
    for (int a = 0; a < b; ++a) x[a] = cdiv_(x[a], nr);
}

// Set-up of one leaf per CTA, in the precision of the leaf path (FP32 for the mixed
// form, FP64 for the FP64 form).
// Eigenvalues: Aberth-Ehrlich simultaneous iteration, one thread per eigenvalue,
//   z_j <- z_j - w_j / (1 - w_j sum_{k != j} 1/(z_j - z_k)),  w_j = p(z_j)/p'(z_j),
// started from the closed-form spectrum of the real part, 2 - 2cos(j pi/(b-1)) - (kh)^2
// (the halved-end second difference has the cosine eigenvectors), shifted by the
// first-order effect of the two impedance corners.
template <typename T>
__global__ void __launch_bounds__(256) k_eig_factor(const EigTask* __restrict__ tasks, int Sx, double kh,
                                                    int* err) {
    using C = cplx<T>;
    const EigTask tk = tasks[blockIdx.x];
    const int b = tk.b;
    __shared__ C d[EIG_BMAX], e2[EIG_BMAX], z[EIG_BMAX];
    for (int a = threadIdx.x; a < b; a += blockDim.x) {
        C dd, ee;
        band_tridiag<T>(b, kh, a, dd, ee);
        d[a] = dd;
        e2[a] = ee * ee;
        const double mu = 2.0 - 2.0 * cos(M_PI * a / (b - 1)) - kh * kh;
        z[a] = {(T)mu, (T)(-kh * (a == 0 ? 2.0 : 4.0) / (b - 1))};
    }
    __syncthreads();
    for (int it = 0; it < 48; ++it) {
        C zn = {0, 0};
        bool small = true;
        if (threadIdx.x < b) {
            const int j = threadIdx.x;
            const C zj = z[j];
            const C w = newton_step<T>(d, e2, b, zj);
            C s = {0, 0};
            for (int k = 0; k < b; ++k)
                if (k != j) s = s + cdiv_(C{1, 0}, zj - z[k]);
            const C dz = cdiv_(w, C{1, 0} - w * s);
            zn = zj - dz;
            small = cabs_(dz) <= (T)64 * Eps<T>::v * fmax(cabs_(zj), (T)1);
        }
        __syncthreads();
        if (threadIdx.x < b) z[threadIdx.x] = zn;
        if (__syncthreads_and(small) && it >= 3) break;
    }
    c128* lam = (c128*)tk.lam;
    C* V = (C*)tk.V;
    C* xi = (C*)tk.xi;
    for (int m = threadIdx.x; m < b; m += blockDim.x) {
        const C lm = z[m];
        if (!(isfinite(lm.re) && isfinite(lm.im))) atomicExch(err, DEV_BREAKDOWN);
        lam[m] = cvt<double>(lm);
        C* ws = (C*)tk.work + (size_t)m * 6 * b;
        C* q = ws + 5 * b;
        const C mu = lm + C{(T)(8 * Eps<T>::v) * fmax(cabs_(lm), (T)1), (T)0};
        inverse_iteration<T>(b, kh, mu, q, ws);
        for (int a = 0; a < b; ++a) V[a * b + m] = ((T)(1.0 / sqrt(wrow(a, b)))) * q[a];
        // scalar Schur recursions along the columns
        C prev = {0, 0};
        for (int i = 0; i < Sx; ++i) {
            const T wi = (T)wcol(i, Sx);
            const bool xb = (i == 0 || i == Sx - 1);
            const C delta = C{(T)(xb ? 1.0 : 2.0), (T)(xb ? -kh : 0.0)} + wi * lm;
            const C sdel = delta - prev;
            if (!(abs2(sdel) > (T)0)) atomicExch(err, DEV_BREAKDOWN);
            prev = cdiv_(C{1, 0}, sdel);
            xi[(size_t)i * b + m] = prev;
        }
    }
}

// --------------------------------------------------------------- contractions
// C[r][j] = sum_k op(V)[r][k] B[k][j] for r, k < b and j < J; op = V (out) or V^T (in).
// One CTA per 32 columns; V and B staged through shared memory in k-chunks of 32.
static constexpr int GT_N = 32, GT_K = 32, GT_THREADS = 256, GT_ROWS = 8, GT_RPT = 17;

template <typename T, bool TRANS>
__global__ void __launch_bounds__(GT_THREADS) k_eig_gemm(const EigTask* __restrict__ tasks, int J, int which) {
    const EigTask tk = tasks[blockIdx.y];
    const int b = tk.b;
    const int j0 = blockIdx.x * GT_N;
    if (j0 >= J) return;
    const cplx<T>* V = (const cplx<T>*)tk.V;
    const cplx<T>* B = (const cplx<T>*)(which == 0 ? tk.F : tk.Fh);
    cplx<T>* C = (cplx<T>*)(which == 0 ? tk.Fh : tk.W);
    extern __shared__ __align__(16) unsigned char gsm[];
    cplx<T>* Vs = (cplx<T>*)gsm;              // [r][k-chunk], b x GT_K
    cplx<T>* Bs = Vs + (size_t)b * GT_K;      // [k-chunk][j], GT_K x GT_N
    const int jj = threadIdx.x % GT_N, rg = threadIdx.x / GT_N;
    cplx<T> acc[GT_RPT];
#pragma unroll
    for (int t = 0; t < GT_RPT; ++t) acc[t] = {0, 0};
    for (int k0 = 0; k0 < b; k0 += GT_K) {
        const int kc = min(GT_K, b - k0);
        if (TRANS) {
            // op(V)[r][k] = V[k][r]: read rows of V (consecutive r), store transposed
            for (int e2 = threadIdx.x; e2 < b * GT_K; e2 += GT_THREADS) {
                const int k = e2 / b, r = e2 - k * b;
                Vs[r * GT_K + k] = k < kc ? V[(size_t)(k0 + k) * b + r] : cplx<T>{0, 0};
            }
        } else {
            for (int e2 = threadIdx.x; e2 < b * GT_K; e2 += GT_THREADS) {
                const int r = e2 / GT_K, k = e2 % GT_K;
                Vs[e2] = k < kc ? V[(size_t)r * b + k0 + k] : cplx<T>{0, 0};
            }
        }
        for (int e2 = threadIdx.x; e2 < GT_K * GT_N; e2 += GT_THREADS) {
            const int k = e2 / GT_N, j = e2 % GT_N;
            cplx<T> v = {0, 0};
            if (k < kc && j0 + j < J) v = B[(size_t)(k0 + k) * J + j0 + j];
            Bs[e2] = v;
        }
        __syncthreads();
#pragma unroll
        for (int t = 0; t < GT_RPT; ++t) {
            const int r = rg + t * GT_ROWS;
            if (r < b) {
                cplx<T> a = acc[t];
                for (int k = 0; k < kc; ++k) cfma(a, Vs[r * GT_K + k], Bs[k * GT_N + jj]);
                acc[t] = a;
            }
        }
        __syncthreads();
    }
    if (j0 + jj < J) {
#pragma unroll
        for (int t = 0; t < GT_RPT; ++t) {
            const int r = rg + t * GT_ROWS;
            if (r < b) C[(size_t)r * J + j0 + jj] = acc[t];
        }
    }
}

// Scalar recursions, in place on Fh[m][i][c].  A CTA takes rm modes of one leaf with all
// their right-hand sides: the modes' coefficients xi[i][m] and right-hand sides along the
// whole line are staged in shared memory by all threads (coalesced), one thread per
// (mode, right-hand side) runs the forward/backward recursion out of shared memory, and
// the results are written back cooperatively.  Lines too long to stage use
// k_eig_recur_global (one thread per (mode, right-hand side) straight from memory).
template <typename T>
__global__ void k_eig_recur_global(const EigTask* __restrict__ tasks, int Sx, int nrhs) {
    const EigTask tk = tasks[blockIdx.y];
    const int b = tk.b;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= b * nrhs) return;
    const int m = t / nrhs, c = t % nrhs;
    const cplx<T>* xi = (const cplx<T>*)tk.xi;
    cplx<T>* f = (cplx<T>*)tk.Fh + (size_t)m * Sx * nrhs + c;
    cplx<T> y = {0, 0};
    for (int i = 0; i < Sx; ++i) {
        y = xi[(size_t)i * b + m] * (f[(size_t)i * nrhs] + y);
        f[(size_t)i * nrhs] = y;
    }
    cplx<T> x = y;
    for (int i = Sx - 2; i >= 0; --i) {
        x = f[(size_t)i * nrhs] + xi[(size_t)i * b + m] * x;
        f[(size_t)i * nrhs] = x;
    }
}

static constexpr int RM_THREADS = 256;
template <typename T>
__global__ void __launch_bounds__(RM_THREADS) k_eig_recur(const EigTask* __restrict__ tasks, int Sx, int nrhs,
                                                          int rm) {
    const EigTask tk = tasks[blockIdx.y];
    const int b = tk.b;
    const int m0 = blockIdx.x * rm;
    if (m0 >= b) return;
    const int nm = min(rm, b - m0);
    extern __shared__ __align__(16) unsigned char rsm[];
    cplx<T>* xs = (cplx<T>*)rsm;                      // [Sx][nm]
    cplx<T>* fs = xs + (size_t)Sx * nm;               // [nm][Sx][nrhs]
    const cplx<T>* xi = (const cplx<T>*)tk.xi;
    cplx<T>* fh = (cplx<T>*)tk.Fh;
    const size_t line = (size_t)Sx * nrhs;
    for (size_t e2 = threadIdx.x; e2 < (size_t)Sx * nm; e2 += blockDim.x) {
        const int i = (int)(e2 / nm), mm = (int)(e2 - (size_t)i * nm);
        xs[e2] = xi[(size_t)i * b + m0 + mm];
    }
    for (size_t e2 = threadIdx.x; e2 < (size_t)nm * line; e2 += blockDim.x) fs[e2] = fh[(size_t)m0 * line + e2];
    __syncthreads();
    for (int t = threadIdx.x; t < nm * nrhs; t += blockDim.x) {
        const int mm = t / nrhs, c = t - (t / nrhs) * nrhs;
        cplx<T>* f = fs + (size_t)mm * line + c;
        cplx<T> y = {0, 0};
        for (int i = 0; i < Sx; ++i) {
            y = xs[(size_t)i * nm + mm] * (f[(size_t)i * nrhs] + y);
            f[(size_t)i * nrhs] = y;
        }
        cplx<T> x = y;
        for (int i = Sx - 2; i >= 0; --i) {
            x = f[(size_t)i * nrhs] + xs[(size_t)i * nm + mm] * x;
            f[(size_t)i * nrhs] = x;
        }
    }
    __syncthreads();
    for (size_t e2 = threadIdx.x; e2 < (size_t)nm * line; e2 += blockDim.x) fh[(size_t)m0 * line + e2] = fs[e2];
}

template <typename T>
void launch_eig_factor(const EigTask* d_tasks, int ntasks, int b_max, int Sx, double kh, int* err, cudaStream_t s) {
    if (b_max > EIG_BMAX) {
        int one = DEV_BADARG;
        cudaMemcpyAsync(err, &one, sizeof(int), cudaMemcpyHostToDevice, s);
        return;
    }
    k_eig_factor<T><<<ntasks, 160, 0, s>>>(d_tasks, Sx, kh, err);
    note_launch();
}

// One leaf solve = three launches: f^ = V^T f, the scalar recursions, x = V x^.
// stage 0: transform in, 1: recursions, 2: transform out.
template <typename T>
void launch_eig_sweep_stage(int stage, const EigTask* d_tasks, int ntasks, int b_max, int Sx, int nrhs,
                            cudaStream_t s) {
    const int J = Sx * nrhs;
    dim3 g1((J + GT_N - 1) / GT_N, ntasks);
    const size_t sm = sizeof(cplx<T>) * ((size_t)b_max * GT_K + GT_K * GT_N);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_eig_gemm<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
        cudaFuncSetAttribute(k_eig_gemm<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
        cudaFuncSetAttribute(k_eig_recur<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        attr = true;
    }
    if (stage == 0) {
        k_eig_gemm<T, true><<<g1, GT_THREADS, sm, s>>>(d_tasks, J, 0);
        note_launch();
    } else if (stage == 2) {
        k_eig_gemm<T, false><<<g1, GT_THREADS, sm, s>>>(d_tasks, J, 1);
        note_launch();
    } else {
        // modes per CTA: the staged line (Sx x (1 + nrhs) per mode) within ~96 KB
        const size_t per_mode = sizeof(cplx<T>) * (size_t)Sx * (1 + nrhs);
        if (per_mode > (200u << 10)) {
            dim3 gg((b_max * nrhs + 127) / 128, ntasks);
            k_eig_recur_global<T><<<gg, 128, 0, s>>>(d_tasks, Sx, nrhs);
        } else {
            const int rm = (int)std::max<size_t>(1, std::min<size_t>(32, (96u << 10) / per_mode));
            dim3 g2((b_max + rm - 1) / rm, ntasks);
            k_eig_recur<T><<<g2, RM_THREADS, per_mode * rm, s>>>(d_tasks, Sx, nrhs, rm);
        }
        note_launch();
    }
}

template <typename T>
void launch_eig_sweep(const EigTask* d_tasks, int ntasks, int b_max, int Sx, int nrhs, cudaStream_t s) {
    for (int st = 0; st < 3; ++st) launch_eig_sweep_stage<T>(st, d_tasks, ntasks, b_max, Sx, nrhs, s);
}

int eig_bmax() { return GT_ROWS * GT_RPT < EIG_BMAX ? GT_ROWS * GT_RPT : EIG_BMAX; }
size_t eig_work_elems(int b) { return (size_t)b * 6 * b; }

template void launch_eig_factor<float>(const EigTask*, int, int, int, double, int*, cudaStream_t);
template void launch_eig_factor<double>(const EigTask*, int, int, int, double, int*, cudaStream_t);
template void launch_eig_sweep<float>(const EigTask*, int, int, int, int, cudaStream_t);
template void launch_eig_sweep_stage<float>(int, const EigTask*, int, int, int, int, cudaStream_t);
template void launch_eig_sweep_stage<double>(int, const EigTask*, int, int, int, int, cudaStream_t);
template void launch_eig_sweep<double>(const EigTask*, int, int, int, int, cudaStream_t);

}  // namespace hh
