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
// tridiagonal W^{-1/2} K W^{-1/2}; eigenvalues by the implicit QL algorithm with
// complex orthogonal plane rotations (the symmetric tridiagonal QL method carried over
// to complex symmetric matrices), eigenvectors by inverse iteration with a pivoted
// tridiagonal LU, normalised q^T q = 1 (no conjugation).
#include "kernels.h"

namespace hh {

static constexpr int EIG_BMAX = 136;     // rows of a leaf band supported by the eigenbasis path

// ------------------------------------------------------------ complex helpers (FP64)
__device__ __forceinline__ double cabs_(c128 z) { return hypot(z.re, z.im); }
__device__ __forceinline__ c128 cdiv_(c128 a, c128 b) {
    // Smith's algorithm for a / b
    if (fabs(b.re) >= fabs(b.im)) {
        const double r = b.im / b.re, den = b.re + b.im * r;
        return {(a.re + a.im * r) / den, (a.im - a.re * r) / den};
    }
    const double r = b.re / b.im, den = b.re * r + b.im;
    return {(a.re * r + a.im) / den, (a.im * r - a.re) / den};
}
// principal square root from |z|: re = sqrt((|z| + x)/2), im = y / (2 re), with the
// cancellation-free branch for x < 0.
__device__ __forceinline__ c128 csqrt_(c128 z) {
    const double r = cabs_(z);
    if (r == 0.0) return {0.0, 0.0};
    const double t = sqrt(0.5 * (r + fabs(z.re)));
    if (z.re >= 0.0) return {t, z.im / (2.0 * t)};
    return {fabs(z.im) / (2.0 * t), copysign(t, z.im)};
}

// Complex symmetric tridiagonal line operator of a band (b rows), scaled W^{-1/2} K W^{-1/2}.
__device__ __forceinline__ void band_tridiag(int b, double kh, int a, c128& d, c128& e) {
    const double wa = wrow(a, b);
    const bool edge = (a == 0 || a == b - 1);
    const double cy = edge ? 1.0 : 2.0;
    d = {(cy - kh * kh * wa) / wa, -(edge ? kh : 0.0) / wa};
    e = {a < b - 1 ? -1.0 / sqrt(wa * wrow(a + 1, b)) : 0.0, 0.0};
}

// Implicit QL for a complex symmetric tridiagonal matrix (d diagonal, e[i] couples i
// and i+1, e[n-1] = 0).  Eigenvalues overwrite d.  Returns false if an eigenvalue
// needs more than 60 iterations or a rotation degenerates.
__device__ bool ql_complex_symmetric(c128* d, c128* e, int n) {
    const double eps = 2.220446049250313e-16;
    for (int l = 0; l < n; ++l) {
        int iter = 0;
        for (;;) {
            int m = l;
            for (; m < n - 1; ++m) {
                const double dd = cabs_(d[m]) + cabs_(d[m + 1]);
                if (cabs_(e[m]) <= eps * dd) break;
            }
            if (m == l) break;
            if (++iter > 60) return false;
            c128 g = cdiv_(d[l + 1] - d[l], 2.0 * e[l]);
            c128 r = csqrt_(g * g + c128{1.0, 0.0});
            const c128 gp = g + r, gm = g - r;
            g = d[m] - d[l] + cdiv_(e[l], cabs_(gp) >= cabs_(gm) ? gp : gm);
            c128 s = {1.0, 0.0}, c = {1.0, 0.0}, p = {0.0, 0.0};
            bool early = false;
            for (int i = m - 1; i >= l; --i) {
                const c128 f = s * e[i], bb = c * e[i];
                r = csqrt_(f * f + g * g);
                e[i + 1] = r;
                if (cabs_(r) == 0.0) {
                    d[i + 1] = d[i + 1] - p;
                    e[m] = {0.0, 0.0};
                    early = true;
                    break;
                }
                s = cdiv_(f, r);
                c = cdiv_(g, r);
                g = d[i + 1] - p;
                r = (d[i] - g) * s + 2.0 * (c * bb);
                p = s * r;
                d[i + 1] = g + p;
                g = c * r - bb;
            }
            if (early) continue;
            d[l] = d[l] - p;
            e[l] = g;
            e[m] = {0.0, 0.0};
        }
    }
    return true;
}

// Inverse iteration for the eigenvector of eigenvalue mu: (T - mu) x = x_prev with a
// pivoted tridiagonal LU (row interchanges between neighbours), three iterations.
__device__ void inverse_iteration(int b, double kh, c128 mu, c128* x, c128* ws) {
    // ws: 5 b complex doubles of per-thread workspace (global memory)
    c128* dg = ws;
    c128* up = ws + b;
    c128* up2 = ws + 2 * b;
    c128* lo = ws + 3 * b;
    double* sw = (double*)(ws + 4 * b);   // interchange flags
    for (int a = 0; a < b; ++a) {
        c128 d, e;
        band_tridiag(b, kh, a, d, e);
        dg[a] = d - mu;
        up[a] = e;
        up2[a] = {0.0, 0.0};
        x[a] = {1.0 + 1e-3 * a, 1e-3 * (a % 7)};
    }
    for (int j = 0; j < b - 1; ++j) {
        c128 dsub, esub;
        band_tridiag(b, kh, j, dsub, esub);   // esub = sub-diagonal entry (j+1, j)
        if (cabs_(dg[j]) >= cabs_(esub)) {
            sw[j] = 0.0;
            const c128 fact = cabs_(dg[j]) > 0.0 ? cdiv_(esub, dg[j]) : c128{0.0, 0.0};
            lo[j] = fact;
            dg[j + 1] = dg[j + 1] - fact * up[j];
        } else {
            sw[j] = 1.0;
            const c128 fact = cdiv_(dg[j], esub);
            dg[j] = esub;
            lo[j] = fact;
            const c128 temp = up[j];
            up[j] = dg[j + 1];
            dg[j + 1] = temp - fact * dg[j + 1];
            if (j < b - 2) {
                up2[j] = up[j + 1];
                up[j + 1] = -(fact * up[j + 1]);
            }
        }
    }
    const double tiny = 1e-300;
    for (int a = 0; a < b; ++a)
        if (cabs_(dg[a]) < tiny) dg[a] = {1e-30, 0.0};
    for (int it = 0; it < 3; ++it) {
        for (int j = 0; j < b - 1; ++j) {
            if (sw[j] == 0.0) {
                x[j + 1] = x[j + 1] - lo[j] * x[j];
            } else {
                const c128 t = x[j];
                x[j] = x[j + 1];
                x[j + 1] = t - lo[j] * x[j];
            }
        }
        x[b - 1] = cdiv_(x[b - 1], dg[b - 1]);
        if (b > 1) x[b - 2] = cdiv_(x[b - 2] - up[b - 2] * x[b - 1], dg[b - 2]);
        for (int j = b - 3; j >= 0; --j) x[j] = cdiv_(x[j] - up[j] * x[j + 1] - up2[j] * x[j + 2], dg[j]);
        double mx = 0.0;
        for (int a = 0; a < b; ++a) mx = fmax(mx, cabs_(x[a]));
        const double inv = mx > 0.0 ? 1.0 / mx : 1.0;
        for (int a = 0; a < b; ++a) x[a] = inv * x[a];
    }
    // complex symmetric normalisation q^T q = 1
    c128 qq = {0.0, 0.0};
    for (int a = 0; a < b; ++a) qq = qq + x[a] * x[a];
    const c128 nr = csqrt_(qq);
    for (int a = 0; a < b; ++a) x[a] = cdiv_(x[a], nr);
}

template <typename T>
__global__ void __launch_bounds__(256) k_eig_factor(const EigTask* __restrict__ tasks, int Sx, double kh,
                                                    int* err) {
    const EigTask tk = tasks[blockIdx.x];
    const int b = tk.b;
    __shared__ c128 d[EIG_BMAX], e[EIG_BMAX];
    __shared__ int ok;
    if (threadIdx.x == 0) {
        for (int a = 0; a < b; ++a) band_tridiag(b, kh, a, d[a], e[a]);
        ok = ql_complex_symmetric(d, e, b) ? 1 : 0;
        if (!ok) atomicExch(err, DEV_BREAKDOWN);
    }
    __syncthreads();
    c128* lam = (c128*)tk.lam;
    cplx<T>* V = (cplx<T>*)tk.V;
    cplx<T>* xi = (cplx<T>*)tk.xi;
    for (int m = threadIdx.x; m < b; m += blockDim.x) {
        const c128 lm = d[m];
        lam[m] = lm;
        c128* ws = (c128*)tk.work + (size_t)m * 6 * b;
        c128* q = ws + 5 * b;
        const c128 mu = lm + c128{1e-13 * fmax(1.0, cabs_(lm)), 0.0};
        inverse_iteration(b, kh, mu, q, ws);
        for (int a = 0; a < b; ++a) V[a * b + m] = cvt<T>((1.0 / sqrt(wrow(a, b))) * q[a]);
        // scalar Schur recursions along the columns
        c128 prev = {0.0, 0.0};
        for (int i = 0; i < Sx; ++i) {
            const double wi = wcol(i, Sx);
            const bool xb = (i == 0 || i == Sx - 1);
            const c128 delta = c128{xb ? 1.0 : 2.0, xb ? -kh : 0.0} + wi * lm;
            const c128 s = delta - prev;
            if (!(abs2(s) > 0.0)) atomicExch(err, DEV_BREAKDOWN);
            prev = cdiv_(c128{1.0, 0.0}, s);
            xi[(size_t)i * b + m] = cvt<T>(prev);
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
        for (int e2 = threadIdx.x; e2 < b * GT_K; e2 += GT_THREADS) {
            const int r = e2 / GT_K, k = e2 % GT_K;
            cplx<T> v = {0, 0};
            if (k < kc) v = TRANS ? V[(size_t)(k0 + k) * b + r] : V[(size_t)r * b + k0 + k];
            Vs[e2] = v;
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

// Scalar recursions, one thread per (mode, right-hand side), in place on Fh[m][i][c].
template <typename T>
__global__ void k_eig_recur(const EigTask* __restrict__ tasks, int Sx, int nrhs) {
    const EigTask tk = tasks[blockIdx.y];
    const int b = tk.b;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= b * nrhs) return;
    const int m = t / nrhs, c = t % nrhs;
    const cplx<T>* xi = (const cplx<T>*)tk.xi;
    cplx<T>* f = (cplx<T>*)tk.Fh + (size_t)m * Sx * nrhs + c;
    constexpr int U = 8;
    cplx<T> y = {0, 0};
    for (int i0 = 0; i0 < Sx; i0 += U) {
        cplx<T> fv[U], xv[U];
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (i0 + u < Sx) { fv[u] = f[(size_t)(i0 + u) * nrhs]; xv[u] = xi[(size_t)(i0 + u) * b + m]; }
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (i0 + u < Sx) {
                y = xv[u] * (fv[u] + y);
                f[(size_t)(i0 + u) * nrhs] = y;
            }
    }
    cplx<T> x = y;   // x_{n-1} = y_{n-1}
    for (int i1 = Sx - 2; i1 >= 0; i1 -= U) {
        cplx<T> yv[U], xv[U];
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (i1 - u >= 0) { yv[u] = f[(size_t)(i1 - u) * nrhs]; xv[u] = xi[(size_t)(i1 - u) * b + m]; }
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (i1 - u >= 0) {
                x = yv[u] + xv[u] * x;
                f[(size_t)(i1 - u) * nrhs] = x;
            }
    }
}

template <typename T>
void launch_eig_factor(const EigTask* d_tasks, int ntasks, int b_max, int Sx, double kh, int* err, cudaStream_t s) {
    if (b_max > EIG_BMAX) {
        int one = DEV_BADARG;
        cudaMemcpyAsync(err, &one, sizeof(int), cudaMemcpyHostToDevice, s);
        return;
    }
    k_eig_factor<T><<<ntasks, 128, 0, s>>>(d_tasks, Sx, kh, err);
    note_launch();
}

template <typename T>
void launch_eig_sweep(const EigTask* d_tasks, int ntasks, int b_max, int Sx, int nrhs, cudaStream_t s) {
    const int J = Sx * nrhs;
    dim3 g1((J + GT_N - 1) / GT_N, ntasks);
    const size_t sm = sizeof(cplx<T>) * ((size_t)b_max * GT_K + GT_K * GT_N);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_eig_gemm<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
        cudaFuncSetAttribute(k_eig_gemm<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
        attr = true;
    }
    k_eig_gemm<T, true><<<g1, GT_THREADS, sm, s>>>(d_tasks, J, 0);
    note_launch();
    dim3 g2((b_max * nrhs + 127) / 128, ntasks);
    k_eig_recur<T><<<g2, 128, 0, s>>>(d_tasks, Sx, nrhs);
    note_launch();
    k_eig_gemm<T, false><<<g1, GT_THREADS, sm, s>>>(d_tasks, J, 1);
    note_launch();
}

int eig_bmax() { return GT_ROWS * GT_RPT < EIG_BMAX ? GT_ROWS * GT_RPT : EIG_BMAX; }
size_t eig_work_elems(int b) { return (size_t)b * 6 * b; }

template void launch_eig_factor<float>(const EigTask*, int, int, int, double, int*, cudaStream_t);
template void launch_eig_factor<double>(const EigTask*, int, int, int, double, int*, cudaStream_t);
template void launch_eig_sweep<float>(const EigTask*, int, int, int, int, cudaStream_t);
template void launch_eig_sweep<double>(const EigTask*, int, int, int, int, cudaStream_t);

}  // namespace hh
