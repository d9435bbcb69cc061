// hh_core.cuh -- shared device/host helpers of the CUDA path: complex arithmetic,
// the discrete operator's row coefficients, error flags, bounded mbarrier waits and
// 1D bulk (TMA) copies.  Included by every translation unit of libhh.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#define HH_HD __host__ __device__ __forceinline__

// ------------------------------------------------------------------ complex numbers
template <typename T>
struct alignas(2 * sizeof(T)) cplx {
    T re, im;
};
using c64 = cplx<float>;
using c128 = cplx<double>;

// two consecutive complex values, for one wide shared-memory load
template <typename T>
struct alignas(2 * sizeof(cplx<T>)) cpair {
    cplx<T> x, y;
};

template <typename T> HH_HD cplx<T> mk(T r, T i) { return cplx<T>{r, i}; }
template <typename T> HH_HD cplx<T> operator+(cplx<T> a, cplx<T> b) { return {a.re + b.re, a.im + b.im}; }
template <typename T> HH_HD cplx<T> operator-(cplx<T> a, cplx<T> b) { return {a.re - b.re, a.im - b.im}; }
template <typename T> HH_HD cplx<T> operator-(cplx<T> a) { return {-a.re, -a.im}; }
template <typename T> HH_HD cplx<T> operator*(cplx<T> a, cplx<T> b) {
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename T> HH_HD cplx<T> operator*(T s, cplx<T> a) { return {s * a.re, s * a.im}; }
template <typename T> HH_HD cplx<T> conj(cplx<T> a) { return {a.re, -a.im}; }
template <typename T> HH_HD T abs2(cplx<T> a) { return a.re * a.re + a.im * a.im; }
// acc += a * b
template <typename T> HH_HD void cfma(cplx<T>& acc, cplx<T> a, cplx<T> b) {
    acc.re = fma(a.re, b.re, fma(-a.im, b.im, acc.re));
    acc.im = fma(a.re, b.im, fma(a.im, b.re, acc.im));
}
// acc += conj(a) * b
template <typename T> HH_HD void cfma_cj(cplx<T>& acc, cplx<T> a, cplx<T> b) {
    acc.re = fma(a.re, b.re, fma(a.im, b.im, acc.re));
    acc.im = fma(a.re, b.im, fma(-a.im, b.re, acc.im));
}
template <typename T> HH_HD cplx<T> cinv(cplx<T> a) {
    T d = a.re * a.re + a.im * a.im;
    return {a.re / d, -a.im / d};
}
template <typename D, typename S> HH_HD cplx<D> cvt(cplx<S> a) { return {(D)a.re, (D)a.im}; }

// ------------------------------------------------------------- discrete operator
// Weighted 5-point operator on a band of `b` rows and Sx columns (Sx == 1: 1D):
//   (A u)_ij = w_j X_i(u_.j) + w_i Y_j(u_i.) - (k_j h)^2 w_i w_j u_ij
//              - i k_j h (w_j bx_i + w_i by_j) u_ij,
// with k_j = k, or the wavenumber of row j in a layered medium (Sec. 3.3),
// with w = 1/2 on the band's first/last row and on x = 0, Sx-1 (1 elsewhere), X and Y
// the second differences halved at the ends, bx/by the boundary flags.  A 1D band has
// no x-direction: X = 0, w_i = 1, bx = 0.  Every band edge carries the impedance row
// (zero data on artificial boundaries).
struct OpGeom {
    int b;        // rows in the band
    int Sx;       // columns
    double kh;    // k * h
    const double* khr;   // k h per row of the band (device; layered media, Sec. 3.3) or null: kh
    int q1;       // nonzero: the bilinear elements below instead of the 5-point rows (one k)
};

HH_HD double wrow(int j, int b) { return (j == 0 || j == b - 1) ? 0.5 : 1.0; }
HH_HD double wcol(int i, int Sx) { return Sx == 1 ? 1.0 : ((i == 0 || i == Sx - 1) ? 0.5 : 1.0); }

// Diagonal coefficient of row (j, i) and the off-diagonal weights.
HH_HD c128 op_diag(int j, int i, const OpGeom& g) {
    const double wj = wrow(j, g.b), wi = wcol(i, g.Sx);
    const bool by = (j == 0 || j == g.b - 1);
    const double cy = by ? 1.0 : 2.0;
    double cx = 0.0, bx = 0.0;
    if (g.Sx > 1) {
        const bool xb = (i == 0 || i == g.Sx - 1);
        cx = xb ? 1.0 : 2.0;
        bx = xb ? 1.0 : 0.0;
    }
    const double kh = g.khr ? g.khr[j] : g.kh;
    const double re = wj * cx + wi * cy - kh * kh * wi * wj;
    const double im = -kh * (wj * bx + wi * (by ? 1.0 : 0.0));
    return {re, im};
}
// The same coefficient evaluated in precision R (the weights and stencil counts are
// exact in any precision; R = float keeps single-precision kernels off the FP64 pipe).
template <typename R> HH_HD cplx<R> op_diag_t(int j, int i, const OpGeom& g) {
    const R wj = (j == 0 || j == g.b - 1) ? (R)0.5 : (R)1;
    const R wi = g.Sx == 1 ? (R)1 : ((i == 0 || i == g.Sx - 1) ? (R)0.5 : (R)1);
    const bool by = (j == 0 || j == g.b - 1);
    const R cy = by ? (R)1 : (R)2;
    R cx = 0, bx = 0;
    if (g.Sx > 1) {
        const bool xb = (i == 0 || i == g.Sx - 1);
        cx = xb ? (R)1 : (R)2;
        bx = xb ? (R)1 : (R)0;
    }
    const R kh = (R)(g.khr ? g.khr[j] : g.kh);
    return {wj * cx + wi * cy - kh * kh * wi * wj, -kh * (wj * bx + wi * (by ? (R)1 : (R)0))};
}

// Bilinear (Q1) elements of Sec. 3 on the same grid and band.  Over h, the 1D element
// matrices of a line of n nodes are the mass M = tridiag(1, 4, 1) / 6 (2/6 at the two
// ends) and the stiffness X = tridiag(-1, 2, -1) (1 at the ends); with B the end flags,
//   A = M_y (x) K_x + K'_y (x) M_x,   K_x = X_x - (kh)^2 M_x - i kh B_x,   K'_y = X_y - i kh B_y,
// (y the band's rows, x its columns; the impedance terms are the edge masses of the element
// boundary integrals).  Its row (j, i) couples the 3 x 3 neighbourhood; q1_coef is the
// coefficient of u(j + dj, i + di), for a neighbour inside the band.
HH_HD double q1_mass(int a, int d, int n) { return d != 0 ? 1.0 / 6.0 : ((a == 0 || a == n - 1) ? 2.0 / 6.0 : 4.0 / 6.0); }
HH_HD double q1_stiff(int a, int d, int n) { return d != 0 ? -1.0 : ((a == 0 || a == n - 1) ? 1.0 : 2.0); }
HH_HD c128 q1_coef(int j, int dj, int i, int di, const OpGeom& g) {
    const double q = g.kh;
    const double my = q1_mass(j, dj, g.b), xy = q1_stiff(j, dj, g.b);
    const double mx = q1_mass(i, di, g.Sx), xx = q1_stiff(i, di, g.Sx);
    const double by = (dj == 0 && (j == 0 || j == g.b - 1)) ? 1.0 : 0.0;
    const double bx = (di == 0 && (i == 0 || i == g.Sx - 1)) ? 1.0 : 0.0;
    return {my * (xx - q * q * mx) + xy * mx, -q * (my * bx + by * mx)};
}
// (A u)(j, i) for the bilinear elements, in precision R; at(dj, di) returns u(j + dj, i + di)
// (called for neighbours inside the band only).
template <typename R, typename F> HH_HD cplx<R> q1_row(int j, int i, const OpGeom& g, F&& at) {
    cplx<R> acc = {0, 0};
    for (int dj = -1; dj <= 1; ++dj) {
        if (j + dj < 0 || j + dj >= g.b) continue;
        for (int di = -1; di <= 1; ++di) {
            if (i + di < 0 || i + di >= g.Sx) continue;
            const c128 c = q1_coef(j, dj, i, di, g);
            const cplx<R> v = at(dj, di);
            acc.re += (R)c.re * v.re - (R)c.im * v.im;
            acc.im += (R)c.re * v.im + (R)c.im * v.re;
        }
    }
    return acc;
}

// ------------------------------------------------------------------ error reporting
// Device-side status word (per process): kernels record the first failure here and
// the host reads it after synchronising.  Codes mirror hh_status.
enum DevErr : int { DEV_OK = 0, DEV_BREAKDOWN = 1, DEV_TIMEOUT = 2, DEV_BADARG = 3 };

// ----------------------------------------------------------- mbarrier + bulk copy
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
// Asynchronous 16-byte global -> shared copies (the copy engine of the load/store unit):
// issue, commit, and wait for all of this thread's copies.
// L2 eviction priorities for streamed loads: a policy from createpolicy and a read-only
// load that carries it
__device__ __forceinline__ unsigned long long l2_policy_first() {
    unsigned long long p;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ unsigned long long l2_policy_normal() {
    unsigned long long p;
    asm("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ cplx<float> ld_hint(const cplx<float>* a, unsigned long long pol) {
    cplx<float> v;
    asm("ld.global.nc.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;" : "=f"(v.re), "=f"(v.im) : "l"(a), "l"(pol));
    return v;
}
__device__ __forceinline__ cplx<double> ld_hint(const cplx<double>* a, unsigned long long pol) {
    cplx<double> v;
    asm("ld.global.nc.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;" : "=d"(v.re), "=d"(v.im) : "l"(a), "l"(pol));
    return v;
}
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(smem)), "l"(gmem) : "memory");
}
// 8-byte form; valid = false fills the 8 bytes with zeros (source size 0, nothing read)
__device__ __forceinline__ void cp_async8_zfill(void* smem, const void* gmem, bool valid) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(smem_u32(smem)), "l"(gmem),
                 "r"(valid ? 8 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_group1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: returns false if the phase did not complete within `limit` polls.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint32_t limit) {
    for (uint32_t it = 0; it < limit; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if (it > 64) __nanosleep(64);
    }
    return false;
}
// 1D bulk copy global -> shared (TMA engine), completion signalled on `bar`.
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// --------------------------------------------------------------------- reductions
template <typename T> __device__ __forceinline__ T warp_sum(T v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
template <typename T> __device__ __forceinline__ cplx<T> warp_sum(cplx<T> v) {
    v.re = warp_sum(v.re);
    v.im = warp_sum(v.im);
    return v;
}

HH_HD size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// ------------------------------------------------------ one-time steps per device
// Kernel attributes (the dynamic shared-memory limit, non-portable cluster sizes) belong
// to a device's context, so a process that drives several devices sets them on each.
// `bits` holds one bit per device (ordinals 0..63); f() runs until it succeeds once on
// the current device.  Two threads may both run f() the first time, which is harmless.
inline int current_device() {
    int d = 0;
    cudaGetDevice(&d);
    return d;
}
template <typename F> inline bool once_per_device(std::atomic<unsigned long long>& bits, F&& f) {
    const unsigned long long bit = 1ull << (current_device() & 63);
    if (bits.load(std::memory_order_acquire) & bit) return true;
    if (!f()) return false;
    bits.fetch_or(bit, std::memory_order_release);
    return true;
}
// Raises `fn`'s dynamic shared-memory limit to `bytes` on the current device, once.
template <typename K> inline void smem_limit_once(std::atomic<unsigned long long>& bits, K* fn, int bytes) {
    once_per_device(bits, [&] {
        return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) == cudaSuccess;
    });
}
