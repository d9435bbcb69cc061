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
//
// Bilinear elements (Sec. 3): the blocks are D_i = (X_ii - i kh bx_i) M + M^x_ii K and
// L_i = U_{i-1} = -M + K / 6, with M the consistent 1D mass of the band (tridiagonal),
// K = X - (kh)^2 M - i kh E, and M^x_ii the column's mass (4/6, 2/6 at the ends).  The same
// decoupling holds with K V = M V Lambda, V^T M V = I: delta_{i,m} = M^x_ii lambda_m + X_ii
// - i kh bx_i and the coupling l_m = -1 + lambda_m / 6 (-1 for the 5-point rows), so
//     xi_{i,m} = 1 / (delta_{i,m} - l_m^2 xi_{i-1,m}),
//     y_i = xi_i (f^_i - l y_{i-1}),  x_i = y_i - xi_i l x_{i+1}.
// Written as the 5-point recursions with a_i = -l xi_i and the input f^ / (-l) (the mode's
// scale `sc`), the recursion kernels run unchanged.  The pencil has no diagonal scaling to
// a standard problem (M is not diagonal), so the eigenvalue recurrences and the inverse
// iteration take K - z M directly, and V is normalised V^T M V = I.
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>

#include <cooperative_groups.h>

#include "kernels.h"

namespace cg = cooperative_groups;

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

// 1 / z as conj(z) / |z|^2 (one real reciprocal); the arguments here are differences of
// eigenvalue estimates and Sturm ratios of moderate size, far from over- or underflow.
template <typename R> __device__ __forceinline__ cplx<R> crcp_(cplx<R> z) {
    const R s = (R)1 / (z.re * z.re + z.im * z.im);
    return {z.re * s, -z.im * s};
}

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

// The bilinear elements' pencil of a band: K (diagonal kd, coupling ke between rows a and
// a + 1) and the consistent mass (md, me).
template <typename R>
__device__ __forceinline__ void band_pencil_q1(int b, double kh, int a, cplx<R>& kd, cplx<R>& ke, R& md, R& me) {
    const bool edge = (a == 0 || a == b - 1);
    const double m = edge ? 2.0 / 6.0 : 4.0 / 6.0;
    kd = {(R)((edge ? 1.0 : 2.0) - kh * kh * m), (R)(edge ? -kh : 0.0)};
    ke = {(R)(a < b - 1 ? -1.0 - kh * kh / 6.0 : 0.0), (R)0};
    md = (R)m;
    me = (R)(a < b - 1 ? 1.0 / 6.0 : 0.0);
}

// Newton correction p(z) / p'(z) of p(z) = det(K - z M) for a tridiagonal pencil, from the
// ratios r_j = p_j / p_{j-1} of its leading principal minors, with e_j = ke_{j-1} - z me_{j-1}:
//   r_0 = kd_0 - z md_0,  r_j = kd_j - z md_j - e_j^2 / r_{j-1},
//   r'_j = -md_j + 2 me_{j-1} e_j / r_{j-1} + e_j^2 r'_{j-1} / r_{j-1}^2,   p'/p = sum_j r'_j / r_j.
template <typename R>
__device__ cplx<R> newton_step_pencil(const cplx<R>* kd, const cplx<R>* ke, const R* md, const R* me, int b,
                                      cplx<R> z) {
    const R tiny = Eps<R>::tiny;
    cplx<R> r = kd[0] - md[0] * z;
    if (abs2(r) < tiny * tiny) r = {tiny, 0};
    cplx<R> rp = {-md[0], 0};
    cplx<R> ir = crcp_(r);
    cplx<R> s = rp * ir;
    for (int j = 1; j < b; ++j) {
        const cplx<R> e = ke[j - 1] - me[j - 1] * z;
        const cplx<R> q = (e * e) * ir;           // e^2 / r
        cplx<R> rn = kd[j] - md[j] * z - q;
        if (abs2(rn) < tiny * tiny) rn = {tiny, 0};
        rp = cplx<R>{-md[j], 0} + ((R)2 * me[j - 1]) * (e * ir) + q * (rp * ir);
        r = rn;
        ir = crcp_(r);
        s = s + rp * ir;
    }
    return cdiv_(cplx<R>{1, 0}, s);
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
    if (abs2(r) < tiny * tiny) r = {tiny, 0};
    cplx<R> rp = {(R)-1, 0};
    cplx<R> ir = crcp_(r);
    cplx<R> s = rp * ir;
    for (int j = 1; j < b; ++j) {
        const cplx<R> q = e2[j - 1] * ir;          // e^2 / r
        cplx<R> rn = d[j] - z - q;
        if (abs2(rn) < tiny * tiny) rn = {tiny, 0};
        rp = cplx<R>{(R)-1, 0} + q * (rp * ir);
        r = rn;
        ir = crcp_(r);
        s = s + rp * ir;
    }
    return cdiv_(cplx<R>{1, 0}, s);
}

// Inverse iteration for the eigenvector of eigenvalue mu: (T - mu) x = x_prev with a
// pivoted tridiagonal LU (row interchanges between neighbours), three iterations,
// normalised q^T q = 1 (complex symmetric, no conjugation).
// dd, ee: the band's tridiagonal (band_tridiag), staged once per leaf.
// With a mass (md, me non-null: the bilinear elements' pencil) the matrix is K - mu M and
// the vector is normalised x^T M x = 1.
template <typename R>
__device__ void inverse_iteration(int b, const cplx<R>* dd, const cplx<R>* ee, cplx<R> mu, cplx<R>* x,
                                  cplx<R>* ws, const R* md = nullptr, const R* me = nullptr) {
    using C = cplx<R>;
    C* dg = ws;
    C* up = ws + b;
    C* up2 = ws + 2 * b;
    C* lo = ws + 3 * b;
    R* sw = (R*)(ws + 4 * b);   // interchange flags
    for (int a = 0; a < b; ++a) {
        dg[a] = md ? dd[a] - md[a] * mu : dd[a] - mu;
        up[a] = me ? ee[a] - me[a] * mu : ee[a];
        up2[a] = {0, 0};
        x[a] = {(R)1 + (R)1e-3 * (R)a, (R)1e-3 * (R)(a % 7)};
    }
    for (int j = 0; j < b - 1; ++j) {
        const C esub = me ? ee[j] - me[j] * mu : ee[j];   // sub-diagonal entry (j+1, j)
        if (abs2(dg[j]) >= abs2(esub)) {
            sw[j] = 0;
            const C fact = abs2(dg[j]) > (R)0 ? cdiv_(esub, dg[j]) : C{0, 0};
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
    // the pivots, guarded, then replaced by their reciprocals (the three solves multiply)
    for (int a = 0; a < b; ++a) {
        const R g0 = Eps<R>::tiny * Eps<R>::v;
        const C dv = abs2(dg[a]) < g0 * g0 ? C{g0, 0} : dg[a];
        dg[a] = cdiv_(C{1, 0}, dv);
    }
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
        x[b - 1] = x[b - 1] * dg[b - 1];
        if (b > 1) x[b - 2] = (x[b - 2] - up[b - 2] * x[b - 1]) * dg[b - 2];
        for (int j = b - 3; j >= 0; --j) x[j] = (x[j] - up[j] * x[j + 1] - up2[j] * x[j + 2]) * dg[j];
        R mx2 = 0;
        for (int a = 0; a < b; ++a) mx2 = fmax(mx2, abs2(x[a]));
        const R inv = mx2 > (R)0 ? (R)1 / sqrt(mx2) : (R)1;
        for (int a = 0; a < b; ++a) x[a] = inv * x[a];
    }
    C qq = {0, 0};
    if (md) {
        for (int a = 0; a < b; ++a) {
            C mx = md[a] * x[a];
            if (a > 0) mx = mx + me[a - 1] * x[a - 1];
            if (a < b - 1) mx = mx + me[a] * x[a + 1];
            qq = qq + x[a] * mx;
        }
    } else {
        for (int a = 0; a < b; ++a) qq = qq + x[a] * x[a];
    }
    const C nr = csqrt_(qq);
    for (int a = 0; a < b; ++a) x[a] = cdiv_(x[a], nr);
}

// Set-up of the leaves, in the precision of the leaf path (FP32 for the mixed form, FP64
// for the FP64 form), in two launches: the eigenvalues (one CTA per leaf) and then the
// eigenvectors and recursions (k_eig_modes).
// Eigenvalues: Aberth-Ehrlich simultaneous iteration, one thread per eigenvalue,
//   z_j <- z_j - w_j / (1 - w_j sum_{k != j} 1/(z_j - z_k)),  w_j = p(z_j)/p'(z_j),
// started from the closed-form spectrum of the real part, 2 - 2cos(j pi/(b-1)) - (kh)^2
// (the halved-end second difference has the cosine eigenvectors), shifted by the
// first-order effect of the two impedance corners.
// Bilinear elements (q1): the same iteration on det(K - z M), started from the closed-form
// spectrum of the real part, 6 (1 - cos t) / (2 + cos t) - (kh)^2 with t = j pi / (b - 1) (the
// cosine vectors again; the ends of X and M are halved alike), shifted by the first-order
// effect of the two impedance corners.
template <typename T>
__global__ void __launch_bounds__(256) k_eig_roots(const EigTask* __restrict__ tasks, double kh, int* err, int q1) {
    using C = cplx<T>;
    const EigTask tk = tasks[blockIdx.x];
    const int b = tk.b;
    __shared__ C d[EIG_BMAX], e[EIG_BMAX], e2[EIG_BMAX], z[EIG_BMAX];
    __shared__ T md[EIG_BMAX], me[EIG_BMAX];
    for (int a = threadIdx.x; a < b; a += blockDim.x) {
        C dd, ee;
        if (q1) {
            T m0, m1;
            band_pencil_q1<T>(b, kh, a, dd, ee, m0, m1);
            md[a] = m0;
            me[a] = m1;
            const double ct = cos(M_PI * a / (b - 1));
            const double mu = 6.0 * (1.0 - ct) / (2.0 + ct) - kh * kh;
            z[a] = {(T)mu, (T)(-kh * (a == 0 ? 2.0 : 12.0 / (2.0 + ct)) / (b - 1))};
        } else {
            band_tridiag<T>(b, kh, a, dd, ee);
            const double mu = 2.0 - 2.0 * cos(M_PI * a / (b - 1)) - kh * kh;
            z[a] = {(T)mu, (T)(-kh * (a == 0 ? 2.0 : 4.0) / (b - 1))};
        }
        d[a] = dd;
        e[a] = ee;
        e2[a] = ee * ee;
    }
    __syncthreads();
    // A root is done when its correction is below 64 eps |z|, or when, already below
    // 4096 eps |z|, it no longer halves from one sweep to the next: the correction then
    // measures rounding noise of the recurrences in T, which the strict bound may never
    // pass.  The iteration converges cubically, so this ends it in a few sweeps.
    T dz_prev2 = (T)INFINITY;
    for (int it = 0; it < 48; ++it) {
        C zn = {0, 0};
        bool small = true;
        if (threadIdx.x < b) {
            const int j = threadIdx.x;
            const C zj = z[j];
            const C w = q1 ? newton_step_pencil<T>(d, e, md, me, b, zj) : newton_step<T>(d, e2, b, zj);
            C s = {0, 0};
            for (int k = 0; k < b; ++k)
                if (k != j) s = s + crcp_(zj - z[k]);
            const C dz = cdiv_(w, C{1, 0} - w * s);
            zn = zj - dz;
            const T sc = fmax(abs2(zj), (T)1);
            const T dz2 = abs2(dz);
            const T tight = (T)64 * Eps<T>::v, loose = (T)4096 * Eps<T>::v;
            small = dz2 <= tight * tight * sc || (it >= 3 && dz2 <= loose * loose * sc && dz2 > (T)0.25 * dz_prev2);
            dz_prev2 = dz2;
        }
        __syncthreads();
        if (threadIdx.x < b) z[threadIdx.x] = zn;
        if (__syncthreads_and(small) && it >= 3) break;
    }
    c128* lam = (c128*)tk.lam;
    for (int m = threadIdx.x; m < b; m += blockDim.x) {
        const C lm = z[m];
        if (!(isfinite(lm.re) && isfinite(lm.im))) atomicExch(err, DEV_BREAKDOWN);
        lam[m] = cvt<double>(lm);
    }
}

// Eigenvectors and the scalar recursions, one warp per mode m of one leaf (grid: modes
// in groups of EM_WARPS, leaves): lane 0 runs the inverse iteration with its workspace
// in shared memory (the chains of dependent accesses stay on chip), the warp writes the
// W-orthonormal column V[.][m], then lane 0 runs the chain xi_{m,i} along the columns.
static constexpr int EM_WARPS = 4;
template <typename T>
__global__ void __launch_bounds__(32 * EM_WARPS) k_eig_modes(const EigTask* __restrict__ tasks, int Sx, double kh,
                                                            int* err, int q1) {
    using C = cplx<T>;
    const EigTask tk = tasks[blockIdx.y];
    const int b = tk.b;
    extern __shared__ __align__(16) unsigned char emsm[];
    C* dd = (C*)emsm;                          // [b] tridiagonal of the band
    C* ee = dd + b;                            // [b]
    C* wsall = ee + b;                         // [EM_WARPS][6 b] per-warp workspace
    T* rw = (T*)(wsall + (size_t)EM_WARPS * 6 * b);   // [b] 1 / sqrt(w_a) (1 for q1)
    T* md = rw + b;                            // [b], [b] the consistent mass (q1)
    T* me = md + b;
    for (int a = threadIdx.x; a < b; a += blockDim.x) {
        C d1, e1;
        if (q1) {
            T m0, m1;
            band_pencil_q1<T>(b, kh, a, d1, e1, m0, m1);
            md[a] = m0;
            me[a] = m1;
            rw[a] = (T)1;
        } else {
            band_tridiag<T>(b, kh, a, d1, e1);
            rw[a] = (T)(1.0 / sqrt(wrow(a, b)));
        }
        dd[a] = d1;
        ee[a] = e1;
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m = blockIdx.x * EM_WARPS + warp;
    if (m >= b) return;
    C* ws = wsall + (size_t)warp * 6 * b;
    C* q = ws + 5 * b;
    const c128 l64 = ((const c128*)tk.lam)[m];
    const C lm = {(T)l64.re, (T)l64.im};
    if (lane == 0) {
        const C mu = lm + C{(T)(8 * Eps<T>::v) * fmax(cabs_(lm), (T)1), (T)0};
        if (q1) inverse_iteration<T>(b, dd, ee, mu, q, ws, md, me);
        else inverse_iteration<T>(b, dd, ee, mu, q, ws);
    }
    __syncwarp();
    C* V = (C*)tk.V;
    for (int a = lane; a < b; a += 32) V[a * b + m] = rw[a] * q[a];
    if (lane != 0) return;
    // scalar Schur recursions along the columns (in T: the FP64 pipe is slow here).  q1:
    // nl = -l_m = 1 - lambda_m / 6 couples the columns; the stored coefficient is nl xi
    // (the multiplier of both recursions) and the mode's input scale 1 / nl (a coupling that
    // vanishes to rounding is replaced by a tiny one: the mode's columns then decouple)
    C* xi = (C*)tk.xi;
    const T khT = (T)kh;
    C nl = {1, 0};
    if (q1) {
        nl = C{(T)1, (T)0} - ((T)1 / (T)6) * lm;
        if (abs2(nl) < Eps<T>::tiny * Eps<T>::tiny) nl = {Eps<T>::tiny, 0};
        ((C*)tk.sc)[m] = crcp_(nl);
    }
    const C nl2 = nl * nl;
    C prev = {0, 0};
    for (int i = 0; i < Sx; ++i) {
        const bool xb = (i == 0 || i == Sx - 1);
        const T wi = q1 ? (xb ? (T)(2.0 / 6.0) : (T)(4.0 / 6.0)) : ((Sx > 1 && xb) ? (T)0.5 : (T)1);
        const C delta = C{xb ? (T)1 : (T)2, xb ? -khT : (T)0} + wi * lm;
        const C sdel = delta - nl2 * prev;
        if (!(abs2(sdel) > (T)0)) atomicExch(err, DEV_BREAKDOWN);
        prev = crcp_(sdel);   // |sdel| is of order one here: no scaling needed
        xi[(size_t)m * Sx + i] = q1 ? nl * prev : prev;
    }
}

// --------------------------------------------------------------- contractions
// C[r][j] = sum_k op(V)[r][k] B[k][j] for r, k < b and j < J = Sx * nrhs; op = V^T (in)
// or V (out).  Column j of the node layout is (i, c) = (j / nrhs, j % nrhs); the
// transformed vectors are stored as fh_col says (line by line, [m][c][i], for a few
// right-hand sides, so that each scalar recursion reads one contiguous line).  One CTA per GT_N columns; V and B staged through shared
// memory in k-chunks.
static constexpr int GT_N = 8, GT_K = 32, GT_THREADS = 256, GT_ROWS = 32, GT_RPT = 5;

template <typename T, bool TRANS>
__global__ void __launch_bounds__(GT_THREADS) k_eig_gemm(const EigTask* __restrict__ tasks, int J, int which,
                                                         int Sx, int nrhs, int kchunk, const int* gate) {
    if (gate && *gate) return;   // a set stop word skips the launch (the same for every block)
    const EigTask tk = tasks[blockIdx.y];
    const int b = tk.b;
    const int j0 = blockIdx.x * GT_N;
    if (j0 >= J) return;
    const cplx<T>* V = (const cplx<T>*)tk.V;
    const cplx<T>* B = (const cplx<T>*)(which == 0 ? tk.F : tk.Fh);
    cplx<T>* C = (cplx<T>*)(which == 0 ? tk.Fh : tk.W);
    extern __shared__ __align__(16) unsigned char gsm[];
    cplx<T>* Vs = (cplx<T>*)gsm;              // [r][k-chunk], b x kchunk
    cplx<T>* Bs = Vs + (size_t)b * kchunk;    // [k-chunk][j], kchunk x GT_N
    const int jj = threadIdx.x % GT_N, rg = threadIdx.x / GT_N;
    cplx<T> acc[GT_RPT];
#pragma unroll
    for (int t = 0; t < GT_RPT; ++t) acc[t] = {0, 0};
    for (int k0 = 0; k0 < b; k0 += kchunk) {
        const int kc = min(kchunk, b - k0);
        // stage op(V)[r][k0 + k] (b x kc) and B[k0 + k][j0 .. j0 + GT_N) with 8 loads in
        // flight per thread
        const int nv = b * kc;
        for (int base = threadIdx.x; base < nv; base += 8 * GT_THREADS) {
            cplx<T> tmp[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int e2 = base + u * GT_THREADS;
                if (e2 < nv) {
                    if (TRANS) { const int k = e2 / b, r = e2 - k * b; tmp[u] = V[(size_t)(k0 + k) * b + r]; }
                    else { const int r = e2 / kc, k = e2 - r * kc; tmp[u] = V[(size_t)r * b + k0 + k]; }
                }
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int e2 = base + u * GT_THREADS;
                if (e2 < nv) {
                    if (TRANS) { const int k = e2 / b, r = e2 - k * b; Vs[r * kchunk + k] = tmp[u]; }
                    else { const int r = e2 / kc, k = e2 - r * kc; Vs[r * kchunk + k] = tmp[u]; }
                }
            }
        }
        const int nb2 = kc * GT_N;
        for (int base = threadIdx.x; base < nb2; base += 8 * GT_THREADS) {
            cplx<T> tmp[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int e2 = base + u * GT_THREADS;
                tmp[u] = {0, 0};
                if (e2 < nb2) {
                    const int k = e2 / GT_N, j = e2 - k * GT_N;
                    if (j0 + j < J) {
                        const int jj2 = j0 + j;
                        // which == 1 reads the line-major transformed vectors
                        const size_t col = which == 0 ? (size_t)jj2 : fh_col((size_t)jj2, Sx, nrhs);
                        tmp[u] = B[(size_t)(k0 + k) * J + col];
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int e2 = base + u * GT_THREADS;
                if (e2 < nb2) Bs[e2] = tmp[u];
            }
        }
        __syncthreads();
#pragma unroll
        for (int t = 0; t < GT_RPT; ++t) {
            const int r = rg + t * GT_ROWS;
            if (r < b) {
                cplx<T> a = acc[t];
                for (int k = 0; k < kc; ++k) cfma(a, Vs[r * kchunk + k], Bs[k * GT_N + jj]);
                acc[t] = a;
            }
        }
        __syncthreads();
    }
    if (j0 + jj < J) {
        const int jj2 = j0 + jj;
        const size_t col = which == 0 ? fh_col((size_t)jj2, Sx, nrhs) : (size_t)jj2;
        // x = V x^ keeps rows [w0, w1) (all rows, or the owned rows written into the parent)
        const int rlo = which == 0 ? 0 : tk.w0, rhi = which == 0 ? b : tk.w1;
#pragma unroll
        for (int t = 0; t < GT_RPT; ++t) {
            const int r = rg + t * GT_ROWS;
            if (r >= rlo && r < rhi) C[(size_t)(r - rlo) * J + col] = acc[t];
        }
    }
}

// Register-tiled form of the same contraction for leaves whose V fits in shared memory:
// one CTA per GN columns (GN = 16 CV), V staged once in [k][r] order (op applied) and the
// CTA's B block [k][GN]; thread (rg, cg) accumulates rows rg + 16 u (u < RU) times columns
// cg + 16 v (v < CV): RU + CV shared loads per RU x CV complex multiply-adds.
template <typename T> struct Gemm2Cols { static constexpr int CV = 4; };
template <> struct Gemm2Cols<double> { static constexpr int CV = 2; };

template <typename T, bool TRANS, int RU>
__global__ void __launch_bounds__(256) k_eig_gemm2(const EigTask* __restrict__ tasks, int J, int which, int Sx,
                                                   int nrhs, const int* gate) {
    if (gate && *gate) return;   // a set stop word skips the launch (the same for every block)
    constexpr int CV = Gemm2Cols<T>::CV, GN = 16 * CV;
    using C = cplx<T>;
    const EigTask tk = tasks[blockIdx.y];
    const int b = tk.b;
    const int j0 = blockIdx.x * GN;
    if (j0 >= J) return;
    const C* V = (const C*)tk.V;
    const C* B = (const C*)(which == 0 ? tk.F : tk.Fh);
    C* Cout = (C*)(which == 0 ? tk.Fh : tk.W);
    extern __shared__ __align__(16) unsigned char g2sm[];
    C* Vs = (C*)g2sm;                  // [k][r], ld = b
    C* Bs = Vs + (size_t)b * b;        // [k][GN]
    // stage: eight loads in flight per thread
    const int nv = b * b, nb2 = b * GN;
    for (int e0 = threadIdx.x; e0 < nv + nb2; e0 += 8 * 256) {
        C tmp[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int e = e0 + u * 256;
            tmp[u] = C{0, 0};
            if (e < nv) {
                const int k = e / b, r = e - k * b;
                tmp[u] = TRANS ? V[(size_t)k * b + r] : V[(size_t)r * b + k];
            } else if (e < nv + nb2) {
                const int e2 = e - nv, k = e2 / GN, c = e2 - k * GN, jj = j0 + c;
                if (jj < J) {
                    const size_t col = which == 0 ? (size_t)jj : fh_col((size_t)jj, Sx, nrhs);
                    tmp[u] = B[(size_t)k * J + col];
                }
            }
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int e = e0 + u * 256;
            if (e < nv + nb2) Vs[e] = tmp[u];   // Vs and Bs are contiguous
        }
    }
    __syncthreads();
    const int rg = threadIdx.x >> 4, cg = threadIdx.x & 15;
    C acc[RU][CV];
#pragma unroll
    for (int u = 0; u < RU; ++u)
#pragma unroll
        for (int v = 0; v < CV; ++v) acc[u][v] = C{0, 0};
    for (int k = 0; k < b; ++k) {
        C vr[RU], bc[CV];
#pragma unroll
        for (int u = 0; u < RU; ++u) vr[u] = Vs[k * b + min(rg + 16 * u, b - 1)];
#pragma unroll
        for (int v = 0; v < CV; ++v) bc[v] = Bs[k * GN + cg + 16 * v];
#pragma unroll
        for (int u = 0; u < RU; ++u)
#pragma unroll
            for (int v = 0; v < CV; ++v) cfma(acc[u][v], vr[u], bc[v]);
    }
    // x = V x^ keeps rows [w0, w1) (all rows, or the owned rows written into the parent)
    const int rlo = which == 0 ? 0 : tk.w0, rhi = which == 0 ? b : tk.w1;
#pragma unroll
    for (int v = 0; v < CV; ++v) {
        const int jj = j0 + cg + 16 * v;
        if (jj >= J) continue;
        const size_t col = which == 0 ? fh_col((size_t)jj, Sx, nrhs) : (size_t)jj;
#pragma unroll
        for (int u = 0; u < RU; ++u) {
            const int r = rg + 16 * u;
            if (r >= rlo && r < rhi) Cout[(size_t)(r - rlo) * J + col] = acc[u][v];
        }
    }
}

// Scalar recursions along each line, in place on Fh[m][c][i]: one warp per line (mode m,
// right-hand side c).  Both recursions are affine, y_i = xi_i y_{i-1} + xi_i f_i and
// x_i = xi_i x_{i+1} + y_i (with x_{n-1} = y_{n-1}), so each lane composes the maps of a
// contiguous chunk of the line, a warp scan (shuffles) composes the chunks, and each lane
// then replays its chunk from its entering value.  The line is staged in shared memory.
template <typename T>
__device__ __forceinline__ void affine_shfl(cplx<T>& A, cplx<T>& B, int d, bool up, cplx<T>& A2, cplx<T>& B2) {
    if (up) {
        A2.re = __shfl_up_sync(0xffffffffu, A.re, d); A2.im = __shfl_up_sync(0xffffffffu, A.im, d);
        B2.re = __shfl_up_sync(0xffffffffu, B.re, d); B2.im = __shfl_up_sync(0xffffffffu, B.im, d);
    } else {
        A2.re = __shfl_down_sync(0xffffffffu, A.re, d); A2.im = __shfl_down_sync(0xffffffffu, A.im, d);
        B2.re = __shfl_down_sync(0xffffffffu, B.re, d); B2.im = __shfl_down_sync(0xffffffffu, B.im, d);
    }
}

// Both recursions of one line, in place: on entry fs = f^ (Sx values) and as = xi; on
// exit fs = x^.  One warp; lane l owns the contiguous chunk [l L, (l + 1) L).
template <typename T>
__device__ __forceinline__ void warp_line_solve(const cplx<T>* as, cplx<T>* fs, int Sx, int lane) {
    using C = cplx<T>;
    const int L = (Sx + 31) / 32;
    const int s = lane * L, e = min(Sx, s + L);
    // forward: y_i = a_i (y_{i-1} + f_i)
    C A = {1, 0}, B = {0, 0};
    for (int i = s; i < e; ++i) { A = as[i] * A; B = as[i] * (B + fs[i]); }
    for (int d = 1; d < 32; d <<= 1) {
        C A2, B2;
        affine_shfl(A, B, d, true, A2, B2);
        if (lane >= d) { B = A * B2 + B; A = A * A2; }
    }
    C y;
    y.re = __shfl_up_sync(0xffffffffu, B.re, 1);
    y.im = __shfl_up_sync(0xffffffffu, B.im, 1);
    if (lane == 0) y = {0, 0};
    for (int i = s; i < e; ++i) { y = as[i] * (fs[i] + y); fs[i] = y; }
    __syncwarp();
    // backward: x_i = y_i + a'_i x_{i+1}, a'_{n-1} = 0
    A = {1, 0};
    B = {0, 0};
    for (int i = e - 1; i >= s; --i) {
        const C ap = (i == Sx - 1) ? C{0, 0} : as[i];
        B = ap * B + fs[i];
        A = ap * A;
    }
    for (int d = 1; d < 32; d <<= 1) {
        C A2, B2;
        affine_shfl(A, B, d, false, A2, B2);
        if (lane + d < 32) { B = A * B2 + B; A = A * A2; }
    }
    C x;
    x.re = __shfl_down_sync(0xffffffffu, B.re, 1);
    x.im = __shfl_down_sync(0xffffffffu, B.im, 1);
    if (lane == 31) x = {0, 0};
    for (int i = e - 1; i >= s; --i) {
        const C ap = (i == Sx - 1) ? C{0, 0} : as[i];
        x = fs[i] + ap * x;
        fs[i] = x;
    }
    __syncwarp();
}

template <typename T>
__global__ void __launch_bounds__(256) k_eig_recur(const EigTask* __restrict__ tasks, int Sx, int nrhs, int wpb,
                                                   const int* gate) {
    if (gate && *gate) return;   // a set stop word skips the launch (the same for every block)
    using C = cplx<T>;
    const EigTask tk = tasks[blockIdx.y];
    const int b = tk.b;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int line = blockIdx.x * wpb + warp;
    if (warp >= wpb || line >= b * nrhs) return;
    const int m = line / nrhs;
    extern __shared__ __align__(16) unsigned char ssm[];
    C* as = (C*)ssm + (size_t)warp * 2 * Sx;
    C* fs = as + Sx;
    const C* xi = (const C*)tk.xi + (size_t)m * Sx;
    C* fh = (C*)tk.Fh + (size_t)line * Sx;     // line = m * nrhs + c
    const C sc = tk.sc ? ((const C*)tk.sc)[m] : C{1, 0};   // the mode's input scale (q1)
    if constexpr (sizeof(C) == 8) {
        // complex64: the whole line in flight at once (asynchronous 8-byte copies)
        for (int i = lane; i < Sx; i += 32) {
            cp_async8_zfill(as + i, xi + i, true);
            cp_async8_zfill(fs + i, fh + i, true);
        }
        cp_async_commit();
        cp_async_wait_all();
        __syncwarp();
        if (tk.sc)
            for (int i = lane; i < Sx; i += 32) fs[i] = sc * fs[i];
    } else {
        for (int i0 = lane; i0 < Sx; i0 += 32 * 8) {
            C ta[8], tf[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int i = i0 + 32 * u;
                if (i < Sx) { ta[u] = xi[i]; tf[u] = tk.sc ? sc * fh[i] : fh[i]; }
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int i = i0 + 32 * u;
                if (i < Sx) { as[i] = ta[u]; fs[i] = tf[u]; }
            }
        }
    }
    __syncwarp();
    warp_line_solve(as, fs, Sx, lane);
    for (int i = lane; i < Sx; i += 32) fh[i] = fs[i];
}

// Scalar recursions of many right-hand sides (16 or more), in place on Fh[m][i][c]: one
// warp per (mode m, 32 consecutive right-hand sides), each lane running its line's forward
// and backward recursions along i (the same y_i = xi_i (y_{i-1} + f_i) and
// x_i = y_i + xi_i x_{i+1} as warp_line_solve).  The lanes' Fh accesses are contiguous and
// xi[m][i] is one broadcast load per warp and step.  Each lane loads RB steps of its line
// and of xi at once before running them, so a chain step waits on no load.
template <typename T>
__global__ void __launch_bounds__(256) k_eig_recur_cols(const EigTask* __restrict__ tasks, int Sx, int nrhs,
                                                        const int* gate) {
    if (gate && *gate) return;   // a set stop word skips the launch (the same for every block)
    using C = cplx<T>;
    constexpr int RB = 16;
    const EigTask tk = tasks[blockIdx.y];
    const int cgs = (nrhs + 31) / 32;
    const int wg = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (wg >= tk.b * cgs) return;
    const int m = wg / cgs, c = (wg - m * cgs) * 32 + (threadIdx.x & 31);
    if (c >= nrhs) return;
    const C* xi = (const C*)tk.xi + (size_t)m * Sx;
    C* fh = (C*)tk.Fh + (size_t)m * Sx * nrhs + c;
    const C sc = tk.sc ? ((const C*)tk.sc)[m] : C{1, 0};   // the mode's input scale (q1)
    C y = {0, 0};
    for (int i0 = 0; i0 < Sx; i0 += RB) {
        C a[RB], f[RB];
#pragma unroll
        for (int u = 0; u < RB; ++u) {
            const int i = min(i0 + u, Sx - 1);
            a[u] = xi[i];
            f[u] = fh[(size_t)i * nrhs];
        }
        if (tk.sc) {
#pragma unroll
            for (int u = 0; u < RB; ++u) f[u] = sc * f[u];
        }
#pragma unroll
        for (int u = 0; u < RB; ++u) {
            if (i0 + u < Sx) {
                y = a[u] * (f[u] + y);
                fh[(size_t)(i0 + u) * nrhs] = y;
            }
        }
    }
    // backward from x_{Sx-1} = y_{Sx-1}, in blocks of RB ending at i1 (exclusive)
    C x = y;
    for (int i1 = Sx - 1; i1 > 0; i1 -= RB) {
        C a[RB], yv[RB];
#pragma unroll
        for (int u = 0; u < RB; ++u) {
            const int i = max(i1 - 1 - u, 0);
            a[u] = xi[i];
            yv[u] = fh[(size_t)i * nrhs];
        }
#pragma unroll
        for (int u = 0; u < RB; ++u) {
            const int i = i1 - 1 - u;
            if (i >= 0) {
                x = yv[u] + a[u] * x;
                fh[(size_t)i * nrhs] = x;
            }
        }
    }
}

template <typename T>
void launch_eig_factor(const EigTask* d_tasks, int ntasks, int b_max, int Sx, double kh, int* err, cudaStream_t s,
                       int q1) {
    if (b_max > EIG_BMAX) {
        int one = DEV_BADARG;
        cudaMemcpyAsync(err, &one, sizeof(int), cudaMemcpyHostToDevice, s);
        return;
    }
    k_eig_roots<T><<<ntasks, 160, 0, s>>>(d_tasks, kh, err, q1);
    note_launch();
    const size_t sm = sizeof(cplx<T>) * (size_t)b_max * (2 + 6 * EM_WARPS) + 3 * sizeof(T) * (size_t)b_max;
    static std::atomic<unsigned long long> attr{0};
    smem_limit_once(attr, k_eig_modes<T>, 200 * 1024);
    k_eig_modes<T><<<dim3((b_max + EM_WARPS - 1) / EM_WARPS, ntasks), 32 * EM_WARPS, sm, s>>>(d_tasks, Sx, kh, err, q1);
    note_launch();
}

// One leaf solve = three launches: f^ = V^T f, the scalar recursions, x = V x^.
// stage 0: transform in, 1: recursions, 2: transform out.
template <typename T>
void launch_eig_sweep_stage(int stage, const EigTask* d_tasks, int ntasks, int b_max, int Sx, int nrhs,
                            cudaStream_t s, const int* gate) {
    const int J = Sx * nrhs;
    dim3 g1((J + GT_N - 1) / GT_N, ntasks);
    // stage as much of V as fits in ~96 KB (all of it for complex64 bands up to 136 rows)
    int kchunk = (int)std::min<size_t>((size_t)b_max, (96u << 10) / (sizeof(cplx<T>) * (b_max + GT_N)));
    kchunk = std::max(8, kchunk);
    const size_t sm = sizeof(cplx<T>) * ((size_t)b_max * kchunk + (size_t)kchunk * GT_N);
    static std::atomic<unsigned long long> attr_t{0}, attr_f{0}, attr_r{0};
    smem_limit_once(attr_t, k_eig_gemm<T, true>, 160 * 1024);
    smem_limit_once(attr_f, k_eig_gemm<T, false>, 160 * 1024);
    smem_limit_once(attr_r, k_eig_recur<T>, 200 * 1024);
    // register-tiled contraction where V and the column block fit in shared memory
    constexpr int GN2 = 16 * Gemm2Cols<T>::CV;
    const size_t sm2 = sizeof(cplx<T>) * ((size_t)b_max * b_max + (size_t)b_max * GN2);
    const bool tiled = stage != 1 && b_max <= 144 && sm2 <= (size_t)(220 * 1024);
    if (tiled) {
        static std::atomic<unsigned long long> a_t5{0}, a_f5{0}, a_t9{0}, a_f9{0};
        smem_limit_once(a_t5, k_eig_gemm2<T, true, 5>, 220 * 1024);
        smem_limit_once(a_f5, k_eig_gemm2<T, false, 5>, 220 * 1024);
        smem_limit_once(a_t9, k_eig_gemm2<T, true, 9>, 220 * 1024);
        smem_limit_once(a_f9, k_eig_gemm2<T, false, 9>, 220 * 1024);
        dim3 g2((J + GN2 - 1) / GN2, ntasks);
        const bool small = b_max <= 80;
        if (stage == 0) {
            if (small) k_eig_gemm2<T, true, 5><<<g2, 256, sm2, s>>>(d_tasks, J, 0, Sx, nrhs, gate);
            else k_eig_gemm2<T, true, 9><<<g2, 256, sm2, s>>>(d_tasks, J, 0, Sx, nrhs, gate);
        } else {
            if (small) k_eig_gemm2<T, false, 5><<<g2, 256, sm2, s>>>(d_tasks, J, 1, Sx, nrhs, gate);
            else k_eig_gemm2<T, false, 9><<<g2, 256, sm2, s>>>(d_tasks, J, 1, Sx, nrhs, gate);
        }
    } else if (stage == 0) {
        k_eig_gemm<T, true><<<g1, GT_THREADS, sm, s>>>(d_tasks, J, 0, Sx, nrhs, kchunk, gate);
    } else if (stage == 2) {
        k_eig_gemm<T, false><<<g1, GT_THREADS, sm, s>>>(d_tasks, J, 1, Sx, nrhs, kchunk, gate);
    } else if (!eig_line_major(nrhs)) {
        const int warps = b_max * ((nrhs + 31) / 32);
        dim3 g3((warps + 7) / 8, ntasks);
        k_eig_recur_cols<T><<<g3, 256, 0, s>>>(d_tasks, Sx, nrhs, gate);
    } else {
        const size_t per_warp = 2 * sizeof(cplx<T>) * (size_t)Sx;
        const int wpb = (int)std::max<size_t>(1, std::min<size_t>(8, (200u << 10) / per_warp));
        const int lines = b_max * nrhs;
        dim3 g2((lines + wpb - 1) / wpb, ntasks);
        k_eig_recur<T><<<g2, 32 * wpb, per_warp * wpb, s>>>(d_tasks, Sx, nrhs, wpb, gate);
    }
    note_launch();
}

template <typename T>
void launch_eig_sweep(const EigTask* d_tasks, int ntasks, int b_max, int Sx, int nrhs, cudaStream_t s) {
    for (int st = 0; st < 3; ++st) launch_eig_sweep_stage<T>(st, d_tasks, ntasks, b_max, Sx, nrhs, s);
}

// ------------------------------------------------------- fused one-vector sweep
// The whole leaf solve for one right-hand side in one launch: one cluster of CL CTAs
// per leaf (CL = 16 where the GPU schedules such clusters, else 8).  CTA q of the
// cluster owns the columns [q ncol, (q + 1) ncol) and the modes [q nmode, (q + 1) nmode).
//   1. f^[m][i] = sum_a V[a][m] f[a][i] for all m and the CTA's columns (V and f staged
//      in shared memory);
//   2. cluster barrier; each warp takes one owned mode, gathers its line f^[m][0..Sx)
//      from the CTAs' shared memory (distributed shared memory), runs both recursions
//      and writes x^[m][.] back in place; cluster barrier;
//   3. x[a][i] = sum_m V[a][m] x^[m][i] for the CTA's columns, written to the leaf output
//      (only the rows [w0, w1) the caller asked for: the owned rows, when the output goes
//      straight into the parent's prolongation).
// V stays in shared memory between the two transforms and the transformed vectors never
// leave the cluster.  4 x 2 register tiles: three 16-byte shared loads per eight complex
// multiply-adds (complex64) in phase 1, five loads in phase 3 (rows strided by b/4 so
// that a warp's V reads fall in distinct banks).
static constexpr int FS_THREADS = 256, FS_WARPS = FS_THREADS / 32;

// Shared memory, in elements: V [b][ldv] | f^ / x^ [b][ldf] | xi of the owned modes
// [nmode][Sx] | f of the own columns [b][ldf] (phase 1), reused as one line per warp
// (phase 2).
struct FsGeom {
    int ncol, nmode, ldv, ldf;
    size_t off_xi, off_in, elems;
};
HH_HD FsGeom fs_geom(int b, int Sx, int cl) {
    FsGeom g;
    g.ncol = (Sx + cl - 1) / cl;
    g.nmode = (b + cl - 1) / cl;
    g.ldv = (b + 3) & ~3;
    g.ldf = g.ncol + (g.ncol & 1);
    g.off_xi = (size_t)b * g.ldv + (size_t)b * g.ldf;
    g.off_in = g.off_xi + (((size_t)g.nmode * Sx + 1) & ~(size_t)1);
    const size_t fin = (size_t)b * g.ldf, lines = (size_t)FS_WARPS * Sx;
    g.elems = g.off_in + (fin > lines ? fin : lines);
    return g;
}

// Asynchronous copy of one complex element into shared memory.
template <typename T> __device__ __forceinline__ void cp_async_elem(cplx<T>* smem, const cplx<T>* gmem);
template <> __device__ __forceinline__ void cp_async_elem<float>(c64* smem, const c64* gmem) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(smem)), "l"(gmem) : "memory");
}
template <> __device__ __forceinline__ void cp_async_elem<double>(c128* smem, const c128* gmem) {
    cp_async16(smem, gmem);
}

template <typename T>
__global__ void __launch_bounds__(FS_THREADS) k_eig_sweep_fused(const EigTask* __restrict__ tasks,
                                                                 const int* __restrict__ gate) {
    // a set stop word (written by an earlier launch, so the same for every CTA) skips
    // the launch before any cluster barrier
    if (gate && *gate) return;
    using C = cplx<T>;
    using C2 = cpair<T>;
    cg::cluster_group cluster = cg::this_cluster();
    const int q = (int)cluster.block_rank();
    const int cl = (int)cluster.num_blocks();
    const EigTask tk = tasks[blockIdx.y];
    // a task of a problem that has left (the same word for the whole cluster): return before
    // any cluster barrier and any access to its buffers
    if (tk.gate && *tk.gate) return;
    const int b = tk.b;
    const int Sx = tk.Sx;
    const FsGeom G = fs_geom(b, Sx, cl);
    const int c0 = q * G.ncol;
    const int nown = max(0, min(Sx, c0 + G.ncol) - c0);
    extern __shared__ __align__(128) unsigned char fsm[];
    C* Vs = (C*)fsm;                              // [b][ldv], V[a][m]
    C* Fs = Vs + (size_t)b * G.ldv;               // [b][ldf], f^ then x^ of own columns
    C* XI = (C*)fsm + G.off_xi;                   // [nmode][Sx], xi of the owned modes
    C* Fin = (C*)fsm + G.off_in;                  // [b][ldf], f of own columns (phase 1)
    C* lines = Fin;                               // per warp one line of Sx (phase 2)
    const C* V = (const C*)tk.V;
    const C* F = (const C*)tk.F;
    C* Wout = (C*)tk.W;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int mb = q * G.nmode, me = min(b, mb + G.nmode);

    // stage V, the own columns of f and the owned modes' xi, all copies in flight at once
    for (int e = threadIdx.x; e < b * b; e += FS_THREADS) {
        const int a = e / b, m = e - a * b;
        cp_async_elem<T>(Vs + a * G.ldv + m, V + e);
    }
    for (int e = threadIdx.x; e < b * G.ldf; e += FS_THREADS) {
        const int a = e / G.ldf, il = e - a * G.ldf;
        if (il < nown) cp_async_elem<T>(Fin + e, F + (size_t)a * Sx + c0 + il);
        else Fin[e] = C{0, 0};
    }
    if (me > mb)
        for (int e = threadIdx.x; e < (me - mb) * Sx; e += FS_THREADS)
            cp_async_elem<T>(XI + e, (const C*)tk.xi + (size_t)mb * Sx + e);
    cp_async_commit();
    cp_async_wait_all();
    __syncthreads();

    const int ntc = (nown + 1) / 2, ntm = (b + 3) / 4;
    // phase 1: tiles (modes m0 .. m0 + 3) x (columns i0, i0 + 1)
    for (int t = threadIdx.x; t < ntm * ntc; t += FS_THREADS) {
        const int m0 = 4 * (t / ntc), i0 = 2 * (t % ntc);
        C acc[4][2];
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[u][0] = acc[u][1] = C{0, 0};
        for (int k = 0; k < b; ++k) {
            const C2 v01 = *(const C2*)(Vs + k * G.ldv + m0);
            const C2 v23 = *(const C2*)(Vs + k * G.ldv + m0 + 2);
            const C2 f = *(const C2*)(Fin + k * G.ldf + i0);
            cfma(acc[0][0], v01.x, f.x);
            cfma(acc[0][1], v01.x, f.y);
            cfma(acc[1][0], v01.y, f.x);
            cfma(acc[1][1], v01.y, f.y);
            cfma(acc[2][0], v23.x, f.x);
            cfma(acc[2][1], v23.x, f.y);
            cfma(acc[3][0], v23.y, f.x);
            cfma(acc[3][1], v23.y, f.y);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (m0 + u < b) *(C2*)(Fs + (m0 + u) * G.ldf + i0) = C2{acc[u][0], acc[u][1]};
    }
    cluster.sync();

    // phase 2: the owned modes' lines
    {
        C* fs = lines + (size_t)warp * Sx;
        for (int m = mb + warp; m < me; m += FS_WARPS) {
            const C* as = XI + (size_t)(m - mb) * Sx;
            const C sc = tk.sc ? ((const C*)tk.sc)[m] : C{1, 0};   // the mode's input scale (q1)
            for (int i = lane; i < Sx; i += 32) {
                const int r = i / G.ncol;
                const C* rem = cluster.map_shared_rank(Fs, r);
                const C v = rem[m * G.ldf + (i - r * G.ncol)];
                fs[i] = tk.sc ? sc * v : v;
            }
            __syncwarp();
            warp_line_solve(as, fs, Sx, lane);
            for (int i = lane; i < Sx; i += 32) {
                const int r = i / G.ncol;
                C* rem = cluster.map_shared_rank(Fs, r);
                rem[m * G.ldf + (i - r * G.ncol)] = fs[i];
            }
            __syncwarp();
        }
    }
    cluster.sync();

    // phase 3: tiles (rows g, g + ntm, g + 2 ntm, g + 3 ntm) x (columns i0, i0 + 1): the
    // lanes of a warp read V rows g .. g + 3, which fall in different shared-memory banks
    // (consecutive rows four apart would share one), written to the output
    for (int t = threadIdx.x; t < ntm * ntc; t += FS_THREADS) {
        const int g = t / ntc, i0 = 2 * (t % ntc);
        const C* vr[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) vr[u] = Vs + min(g + u * ntm, b - 1) * G.ldv;
        C acc[4][2];
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[u][0] = acc[u][1] = C{0, 0};
        for (int k = 0; k < b; ++k) {
            const C2 f = *(const C2*)(Fs + k * G.ldf + i0);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const C v = vr[u][k];
                cfma(acc[u][0], v, f.x);
                cfma(acc[u][1], v, f.y);
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int a = g + u * ntm;
            if (a >= tk.w0 && a < tk.w1) {
                C* wr = Wout + (size_t)(a - tk.w0) * Sx + c0 + i0;
                wr[0] = acc[u][0];
                if (i0 + 1 < nown) wr[1] = acc[u][1];
            }
        }
    }
}

template <typename T>
static cudaLaunchConfig_t fs_config(int cl, int ntasks, size_t sm, cudaStream_t s, cudaLaunchAttribute* attr) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cl, ntasks);
    cfg.blockDim = dim3(FS_THREADS);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = s;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cl;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

// The answer depends only on (device, b_max, Sx, T): cached, so that a set-up does not
// pay an occupancy query.
template <typename T>
int eig_sweep_fused_ready_query(int b_max, int Sx);
template <typename T>
int eig_sweep_fused_ready(int b_max, int Sx) {
    static std::mutex mu;
    static std::map<std::tuple<int, int, int>, int> memo;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    const auto key = std::make_tuple(dev, b_max, Sx);
    const auto it = memo.find(key);
    if (it != memo.end()) return it->second;
    const int cl = eig_sweep_fused_ready_query<T>(b_max, Sx);
    memo[key] = cl;
    return cl;
}
template <typename T>
int eig_sweep_fused_ready_query(int b_max, int Sx) {
    static std::atomic<unsigned long long> attr{0};
    const bool ok = once_per_device(attr, [] {
        if (cudaFuncSetAttribute(k_eig_sweep_fused<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, FS_SMEM_MAX) !=
            cudaSuccess)
            return false;
        // clusters of 16 are beyond the portable size; allowed where the GPU supports them
        if (cudaFuncSetAttribute(k_eig_sweep_fused<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
            cudaSuccess)
            cudaGetLastError();
        return true;
    });
    if (!ok) return 0;
    for (int cl : {16, 8}) {
        if (Sx < cl) continue;
        const size_t sm = sizeof(cplx<T>) * fs_geom(b_max, Sx, cl).elems;
        if (sm > (size_t)FS_SMEM_MAX) continue;
        cudaLaunchAttribute at[1];
        cudaLaunchConfig_t cfg = fs_config<T>(cl, 1, sm, nullptr, at);
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, k_eig_sweep_fused<T>, &cfg) == cudaSuccess && n > 0) return cl;
        cudaGetLastError();
    }
    return 0;
}

// Whether clusters of `cl` CTAs can run the one-launch sweep for these sizes (the
// attributes of eig_sweep_fused_ready must have been set on the device).
template <typename T>
bool eig_sweep_fused_feasible(int cl, int b_max, int Sx) {
    if (Sx < cl || eig_sweep_fused_ready<T>(b_max, Sx) == 0) return false;
    const size_t sm = sizeof(cplx<T>) * fs_geom(b_max, Sx, cl).elems;
    if (sm > (size_t)FS_SMEM_MAX) return false;
    cudaLaunchAttribute at[1];
    cudaLaunchConfig_t cfg = fs_config<T>(cl, 1, sm, nullptr, at);
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k_eig_sweep_fused<T>, &cfg) == cudaSuccess && n > 0) return true;
    cudaGetLastError();
    return false;
}

template <typename T>
void launch_eig_sweep_fused(int cl, const EigTask* d_tasks, int ntasks, int b_max, int Sx, cudaStream_t s,
                            const int* gate) {
    const size_t sm = sizeof(cplx<T>) * fs_geom(b_max, Sx, cl).elems;
    cudaLaunchAttribute at[1];
    cudaLaunchConfig_t cfg = fs_config<T>(cl, ntasks, sm, s, at);
    cudaLaunchKernelEx(&cfg, k_eig_sweep_fused<T>, d_tasks, gate);
    note_launch();
}

int eig_bmax() { return GT_ROWS * GT_RPT < EIG_BMAX ? GT_ROWS * GT_RPT : EIG_BMAX; }

template void launch_eig_factor<float>(const EigTask*, int, int, int, double, int*, cudaStream_t, int);
template void launch_eig_factor<double>(const EigTask*, int, int, int, double, int*, cudaStream_t, int);
template void launch_eig_sweep<float>(const EigTask*, int, int, int, int, cudaStream_t);
template void launch_eig_sweep_stage<float>(int, const EigTask*, int, int, int, int, cudaStream_t, const int*);
template void launch_eig_sweep_stage<double>(int, const EigTask*, int, int, int, int, cudaStream_t, const int*);
template void launch_eig_sweep<double>(const EigTask*, int, int, int, int, cudaStream_t);
template void launch_eig_sweep_fused<float>(int, const EigTask*, int, int, int, cudaStream_t, const int*);
template void launch_eig_sweep_fused<double>(int, const EigTask*, int, int, int, cudaStream_t, const int*);
template int eig_sweep_fused_ready<float>(int, int);
template int eig_sweep_fused_ready<double>(int, int);
template bool eig_sweep_fused_feasible<float>(int, int, int);
template bool eig_sweep_fused_feasible<double>(int, int, int);

}  // namespace hh
