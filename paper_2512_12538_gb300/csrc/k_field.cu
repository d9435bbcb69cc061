// k_field.cu -- grid-field kernels: the weighted 5-point operator and residuals
// (Eqs. (2)-(3) need f - A u at every level), right-hand-side assembly (Eq. (1),
// Sec. 3.1), precision casts and restricted prolongation (Sec. 1), the interface
// traces B_s A~_s (Sec. 2), the counter-based sketch and the coarse update C y.
#include <algorithm>
#include <atomic>

#include "kernels.h"

namespace hh {

static int grid_for(size_t n, int threads, int cap = 152 * 16) {
    size_t g = (n + threads - 1) / threads;
    if (g > (size_t)cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

// ------------------------------------------------------------------ operator apply
// One thread per (point, column); grid-stride.  Compute type = TY (the coefficients too,
// so that a complex64 apply stays off the FP64 pipe).  I: the index type, 32-bit when
// the launch's element count fits (the divisions by the sizes are then far shorter).
template <typename TX, typename TV, typename TY, typename I, bool Q1>
__global__ void k_apply(const cplx<TX>* __restrict__ x, const cplx<TV>* __restrict__ v,
                        cplx<TY>* __restrict__ y, OpGeom g, int nc, TY sgn, double* part) {
    const I total = (I)g.b * (I)g.Sx * (I)nc;
    const I ldr = (I)g.Sx * (I)nc;
    double acc2 = 0.0;
    for (I t = blockIdx.x * (I)blockDim.x + threadIdx.x; t < total; t += (I)gridDim.x * blockDim.x) {
        const I pt = t / (I)nc;
        const I jr = pt / (I)g.Sx;
        const int i = (int)(pt - jr * (I)g.Sx);
        const int j = (int)jr;
        cplx<TY> ax;
        if constexpr (Q1) {
            ax = q1_row<TY>(j, i, g, [&](int dj, int di) {
                return cvt<TY>(x[(size_t)((long long)t + (long long)dj * (long long)ldr + (long long)di * nc)]);
            });
        } else {
            ax = op_diag_t<TY>(j, i, g) * cvt<TY>(x[t]);
            const TY wj = (j == 0 || j == g.b - 1) ? (TY)0.5 : (TY)1;
            const TY wi = g.Sx == 1 ? (TY)1 : ((i == 0 || i == g.Sx - 1) ? (TY)0.5 : (TY)1);
            // x-neighbours: coefficient -w_j
            if (g.Sx > 1) {
                if (i > 0) ax = ax - wj * cvt<TY>(x[t - nc]);
                if (i < g.Sx - 1) ax = ax - wj * cvt<TY>(x[t + nc]);
            }
            // y-neighbours: coefficient -w_i
            if (j > 0) ax = ax - wi * cvt<TY>(x[t - ldr]);
            if (j < g.b - 1) ax = ax - wi * cvt<TY>(x[t + ldr]);
        }
        cplx<TY> out = (-sgn) * ax;
        if (v) out = cvt<TY>(v[t]) + out;
        y[t] = out;
        if (part) acc2 += (double)abs2(out);
    }
    if (part) {
        __shared__ double red[32];
        acc2 = warp_sum(acc2);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc2;
        __syncthreads();
        if (threadIdx.x < 32) {
            double s2 = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
            s2 = warp_sum(s2);
            if (threadIdx.x == 0) part[blockIdx.x] = s2;
        }
    }
}

template <typename TX, typename TV, typename TY>
void launch_apply(const cplx<TX>* x, const cplx<TV>* v, cplx<TY>* y, OpGeom g, int nc, double sgn,
                  double* part, int* nblk_out, cudaStream_t s) {
    const size_t total = (size_t)g.b * g.Sx * nc;
    const int th = 256;
    const int grid = grid_for(total, th, 152 * 8);
    // the bilinear elements' 9-point rows are a separate instantiation (their registers
    // would lower the 5-point kernel's occupancy)
    const bool small = total + (size_t)grid * th < (1ull << 32);
    if (g.q1) {
        if (small) k_apply<TX, TV, TY, unsigned, true><<<grid, th, 0, s>>>(x, v, y, g, nc, (TY)sgn, part);
        else k_apply<TX, TV, TY, size_t, true><<<grid, th, 0, s>>>(x, v, y, g, nc, (TY)sgn, part);
    } else {
        if (small) k_apply<TX, TV, TY, unsigned, false><<<grid, th, 0, s>>>(x, v, y, g, nc, (TY)sgn, part);
        else k_apply<TX, TV, TY, size_t, false><<<grid, th, 0, s>>>(x, v, y, g, nc, (TY)sgn, part);
    }
    note_launch();
    if (nblk_out) *nblk_out = grid;
}

// Global residual y = v - A x in FP64 with per-block partial sums of |y|^2, and the
// same residual rounded to the leaf precision (yt), the input of the next ORAS step.
// With stop (the device-tested loop) the last block to finish also adds the partials in
// block order and takes the stopping test the host would take (IEEE division and square
// root in FP64 on both sides), so no second launch is needed: ctl doubles as the gate,
// stop->ticket is zero between launches.
struct ResidStop {
    double* nrm;
    int* ctl;
    unsigned* ticket;
    double tol;
    const int* need;     // may be null: else the launch does nothing while *need is zero
    const int* anchor;   // may be null: else yt is written only while *anchor is nonzero
};
template <typename T, bool Q1>
__global__ void k_residual_cast(const c128* __restrict__ x, const c128* __restrict__ v, c128* __restrict__ y,
                                cplx<T>* __restrict__ yt, OpGeom g, double* part, const int* gate, ResidStop stop) {
    if (gate && *gate) return;
    if (stop.need && !*stop.need) return;
    const bool wt = !stop.anchor || *stop.anchor;
    const size_t total = (size_t)g.b * g.Sx;
    // interior points of a 2D band with one k: the row is (4 - (kh)^2) x minus the four
    // neighbours, formed as v - (4 - (kh)^2) x (one FMA) plus the neighbours' sum, without
    // the weights and impedance terms of the general row below (the FP64 pipe bounds this
    // kernel: 12 FP64 operations per interior point and the two conversions of yt)
    const double d_in = 4.0 - g.kh * g.kh;
    double acc2 = 0.0;
    const unsigned Sx = (unsigned)g.Sx;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    // the point's column and row, advanced by the stride without a division per point
    unsigned i = (unsigned)(t % Sx), j = (unsigned)(t / Sx);
    const unsigned step_r = (unsigned)(stride % Sx), step_q = (unsigned)(stride / Sx);
    for (; t < total; t += stride) {
        c128 out;
        if constexpr (Q1) {
            out = v[t] - q1_row<double>((int)j, (int)i, g, [&](int dj, int di) {
                      return x[(size_t)((long long)t + (long long)dj * Sx + di)];
                  });
        } else if (Sx > 1 && !g.khr && i > 0 && i < Sx - 1 && j > 0 && j < (unsigned)g.b - 1) {
            const c128 xc = x[t], vc = v[t];
            const c128 w = x[t - 1], e = x[t + 1], s = x[t - Sx], n = x[t + Sx];
            out.re = fma(-d_in, xc.re, vc.re) + ((w.re + e.re) + (s.re + n.re));
            out.im = fma(-d_in, xc.im, vc.im) + ((w.im + e.im) + (s.im + n.im));
        } else {
            c128 ax = op_diag((int)j, (int)i, g) * x[t];
            const double wj = wrow((int)j, g.b), wi = wcol((int)i, g.Sx);
            if (Sx > 1) {
                if (i > 0) ax = ax - wj * x[t - 1];
                if (i < Sx - 1) ax = ax - wj * x[t + 1];
            }
            if (j > 0) ax = ax - wi * x[t - Sx];
            if (j < (unsigned)g.b - 1) ax = ax - wi * x[t + Sx];
            out = v[t] - ax;
        }
        if (y) y[t] = out;
        if (wt) yt[t] = cvt<T>(out);
        acc2 = fma(out.re, out.re, acc2);
        acc2 = fma(out.im, out.im, acc2);
        i += step_r;
        j += step_q;
        if (i >= Sx) {
            i -= Sx;
            ++j;
        }
    }
    __shared__ double red[32];
    __shared__ unsigned s_last;
    acc2 = warp_sum(acc2);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc2;
    __syncthreads();
    if (threadIdx.x < 32) {
        double s2 = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        s2 = warp_sum(s2);
        if (threadIdx.x == 0) {
            part[blockIdx.x] = s2;
            if (stop.ctl) {
                __threadfence();
                s_last = atomicAdd(stop.ticket, 1u) == gridDim.x - 1;
            }
        }
    }
    if (!stop.ctl) return;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // the last block: k_sum's order (thread t adds t, t + 256, ..., then the warp and
    // block trees), so ||r||^2 is the value launch_sum would give
    double a = 0.0;
    for (unsigned i = threadIdx.x; i < gridDim.x; i += blockDim.x) a += __ldcg(part + i);
    a = warp_sum(a);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
    __syncthreads();
    if (threadIdx.x < 32) {
        double s2 = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        s2 = warp_sum(s2);
        if (threadIdx.x == 0) {
            *stop.ticket = 0u;
            stop.nrm[0] = s2;
            stop.ctl[1] += 1;
            const double b2 = stop.nrm[2];
            const double rel = b2 > 0 ? sqrt(s2 / b2) : 0.0;
            if (!isfinite(rel)) stop.ctl[0] = 2;
            else if (rel < stop.tol) stop.ctl[0] = 1;
        }
    }
}
// One wave of co-resident blocks (the grid-stride loop takes the rest): a second, partial
// wave left most SMs idle at the end of the launch.
template <typename T, bool Q1>
static int resid_grid(size_t total) {
    static std::atomic<int> cap[64];
    const int dev = current_device();
    int c = cap[dev & 63].load(std::memory_order_relaxed);
    if (!c) {
        int nb = 0, sms = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_residual_cast<T, Q1>, 256, 0);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        c = std::max(1, std::min(nb, 8)) * std::max(sms, 1);
        cap[dev & 63].store(c, std::memory_order_relaxed);
    }
    return grid_for(total, 256, c);
}
template <typename T>
void launch_residual_cast(const c128* x, const c128* v, c128* y, cplx<T>* yt, OpGeom g, double* part, int* nblk_out,
                          cudaStream_t s, const int* gate) {
    const size_t total = (size_t)g.b * g.Sx;
    const int grid = g.q1 ? resid_grid<T, true>(total) : resid_grid<T, false>(total);
    const ResidStop none{nullptr, nullptr, nullptr, 0.0, nullptr, nullptr};
    if (g.q1) k_residual_cast<T, true><<<grid, 256, 0, s>>>(x, v, y, yt, g, part, gate, none);
    else k_residual_cast<T, false><<<grid, 256, 0, s>>>(x, v, y, yt, g, part, gate, none);
    note_launch();
    if (nblk_out) *nblk_out = grid;
}
template <typename T>
void launch_residual_stop(const c128* x, const c128* v, c128* y, cplx<T>* yt, OpGeom g, double* part, double* nrm,
                          int* ctl, unsigned* ticket, double tol, cudaStream_t s, const int* need,
                          const int* anchor) {
    const size_t total = (size_t)g.b * g.Sx;
    const int grid = g.q1 ? resid_grid<T, true>(total) : resid_grid<T, false>(total);
    const ResidStop st{nrm, ctl, ticket, tol, need, anchor};
    if (g.q1) k_residual_cast<T, true><<<grid, 256, 0, s>>>(x, v, y, yt, g, part, ctl, st);
    else k_residual_cast<T, false><<<grid, 256, 0, s>>>(x, v, y, yt, g, part, ctl, st);
    note_launch();
}
template void launch_residual_stop<float>(const c128*, const c128*, c128*, c64*, OpGeom, double*, double*, int*,
                                          unsigned*, double, cudaStream_t, const int*, const int*);
template void launch_residual_stop<double>(const c128*, const c128*, c128*, c128*, OpGeom, double*, double*, int*,
                                           unsigned*, double, cudaStream_t, const int*, const int*);

// y[j N + pt] = (A~ x_j)[pt] for p column-major columns (one thread per (column, point))
template <typename T>
__global__ void k_apply_cols(const cplx<T>* __restrict__ x, cplx<T>* __restrict__ y, OpGeom g, int p) {
    const size_t N = (size_t)g.b * g.Sx, total = N * p;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        const size_t pt = t % N;
        const int i = (int)(pt % g.Sx), j = (int)(pt / g.Sx);
        cplx<T> ax;
        if (g.q1) {
            ax = q1_row<T>(j, i, g, [&](int dj, int di) { return x[(size_t)((long long)t + (long long)dj * g.Sx + di)]; });
        } else {
            ax = op_diag_t<T>(j, i, g) * x[t];
            const T wj = (j == 0 || j == g.b - 1) ? (T)0.5 : (T)1;
            const T wi = g.Sx == 1 ? (T)1 : ((i == 0 || i == g.Sx - 1) ? (T)0.5 : (T)1);
            if (g.Sx > 1) {
                if (i > 0) ax = ax - wj * x[t - 1];
                if (i < g.Sx - 1) ax = ax - wj * x[t + 1];
            }
            if (j > 0) ax = ax - wi * x[t - g.Sx];
            if (j < g.b - 1) ax = ax - wi * x[t + g.Sx];
        }
        y[t] = ax;
    }
}
template <typename T>
void launch_apply_cols(const cplx<T>* x, cplx<T>* y, OpGeom g, int p, cudaStream_t s) {
    const size_t total = (size_t)g.b * g.Sx * p;
    k_apply_cols<T><<<grid_for(total, 256), 256, 0, s>>>(x, y, g, p);
    note_launch();
}
template void launch_apply_cols<float>(const c64*, c64*, OpGeom, int, cudaStream_t);
template void launch_apply_cols<double>(const c128*, c128*, OpGeom, int, cudaStream_t);
template void launch_residual_cast<float>(const c128*, const c128*, c128*, c64*, OpGeom, double*, int*, cudaStream_t,
                                          const int*);
template void launch_residual_cast<double>(const c128*, const c128*, c128*, c128*, OpGeom, double*, int*,
                                           cudaStream_t, const int*);

// Residuals of several problems in one launch (the batched solver): job k owns blocks
// [blk0, blk0 + nblk) and computes y = v - A x, its complex64/128 copy yt and per-block
// |y|^2 partials at part[blockIdx.x]; then one block per job adds its partials in order.
template <typename T>
__global__ void k_residual_batch(ResidBatch bt, double* part) {
    int jb = 0;
    while (jb + 1 < bt.njobs && blockIdx.x >= bt.job[jb + 1].blk0) ++jb;
    const ResidJob& J = bt.job[jb];
    if (J.gate && *J.gate) return;   // a problem that has left: nothing of it is touched
    const OpGeom g = J.g;
    const size_t total = (size_t)g.b * g.Sx;
    const unsigned lb = blockIdx.x - J.blk0;
    double acc2 = 0.0;
    for (size_t t = lb * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)J.nblk * blockDim.x) {
        const int i = (int)(t % g.Sx);
        const int j = (int)(t / g.Sx);
        c128 ax;
        if (g.q1) {
            ax = q1_row<double>(j, i, g, [&](int dj, int di) { return J.x[(size_t)((long long)t + (long long)dj * g.Sx + di)]; });
        } else {
            ax = op_diag(j, i, g) * J.x[t];
            const double wj = wrow(j, g.b), wi = wcol(i, g.Sx);
            if (g.Sx > 1) {
                if (i > 0) ax = ax - wj * J.x[t - 1];
                if (i < g.Sx - 1) ax = ax - wj * J.x[t + 1];
            }
            if (j > 0) ax = ax - wi * J.x[t - g.Sx];
            if (j < g.b - 1) ax = ax - wi * J.x[t + g.Sx];
        }
        const c128 out = J.v[t] - ax;
        J.y[t] = out;
        ((cplx<T>*)J.yt)[t] = cvt<T>(out);
        acc2 += abs2(out);
    }
    __shared__ double red[32];
    acc2 = warp_sum(acc2);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc2;
    __syncthreads();
    if (threadIdx.x < 32) {
        double s2 = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        s2 = warp_sum(s2);
        if (threadIdx.x == 0) part[blockIdx.x] = s2;
    }
}
__global__ void k_sum_batch(ResidBatch bt, const double* part, double* norms) {
    const ResidJob& J = bt.job[blockIdx.x];
    if (J.gate && *J.gate) return;
    double a = 0.0;
    for (unsigned i = threadIdx.x; i < J.nblk; i += blockDim.x) a += part[J.blk0 + i];
    __shared__ double red[32];
    a = warp_sum(a);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
    __syncthreads();
    if (threadIdx.x < 32) {
        double s2 = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        s2 = warp_sum(s2);
        if (threadIdx.x == 0) norms[blockIdx.x] = s2;
    }
}
template <typename T>
void launch_residual_batch(ResidBatch bt, double* part, int part_cap, double* norms, cudaStream_t s) {
    if (bt.njobs < 1) return;
    const int cap = std::max(1, std::min(152 * 2, part_cap / bt.njobs));
    unsigned blk = 0;
    for (int k = 0; k < bt.njobs; ++k) {
        const size_t n = (size_t)bt.job[k].g.b * bt.job[k].g.Sx;
        bt.job[k].blk0 = blk;
        bt.job[k].nblk = (unsigned)grid_for(n, 256, cap);
        blk += bt.job[k].nblk;
    }
    k_residual_batch<T><<<blk, 256, 0, s>>>(bt, part);
    note_launch();
    k_sum_batch<<<bt.njobs, 256, 0, s>>>(bt, part, norms);
    note_launch();
}
template void launch_residual_batch<float>(ResidBatch, double*, int, double*, cudaStream_t);
template void launch_residual_batch<double>(ResidBatch, double*, int, double*, cudaStream_t);

__global__ void k_sum(const double* part, int n, double* out) {
    double a = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) a += part[i];
    __shared__ double red[32];
    a = warp_sum(a);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
    __syncthreads();
    if (threadIdx.x < 32) {
        double s2 = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        s2 = warp_sum(s2);
        if (threadIdx.x == 0) *out = s2;
    }
}
void launch_sum(const double* part, int n, double* out, cudaStream_t s) {
    k_sum<<<1, 256, 0, s>>>(part, n, out);
    note_launch();
}


// --------------------------------------------------------------------------- rhs
// Bilinear elements (q1, 2D): b = h^2 (M_y F M_x^T) + h (the edge masses applied to g), M the
// 1D consistent masses over h (q1_mass): the load vector of the element integrals.
__device__ c128 rhs_q1(const c128* __restrict__ f, const c128* __restrict__ g, int S, double h, int j, int i) {
    c128 v = {0.0, 0.0};
    for (int dj = -1; dj <= 1; ++dj) {
        if (j + dj < 0 || j + dj >= S) continue;
        for (int di = -1; di <= 1; ++di) {
            if (i + di < 0 || i + di >= S) continue;
            v = v + (h * h * q1_mass(j, dj, S) * q1_mass(i, di, S)) * f[(size_t)(j + dj) * S + (i + di)];
        }
    }
    for (int d = -1; d <= 1; ++d) {
        if (j + d >= 0 && j + d < S) {
            if (i == 0) v = v + (h * q1_mass(j, d, S)) * g[0 * S + j + d];
            if (i == S - 1) v = v + (h * q1_mass(j, d, S)) * g[1 * S + j + d];
        }
        if (i + d >= 0 && i + d < S) {
            if (j == 0) v = v + (h * q1_mass(i, d, S)) * g[2 * S + i + d];
            if (j == S - 1) v = v + (h * q1_mass(i, d, S)) * g[3 * S + i + d];
        }
    }
    return v;
}
__global__ void k_rhs(const c128* __restrict__ f, const c128* __restrict__ g, c128* __restrict__ b,
                      int dim, int S, double h, int q1) {
    const int Sx = dim == 2 ? S : 1;
    const size_t total = (size_t)S * Sx;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
         t += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(t % Sx), j = (int)(t / Sx);
        if (q1) {
            b[t] = rhs_q1(f, g, S, h, j, i);
            continue;
        }
        const double wj = wrow(j, S), wi = wcol(i, Sx);
        c128 v = (h * h * wi * wj) * f[t];
        if (dim == 1) {
            if (j == 0) v = v + h * g[0];
            if (j == S - 1) v = v + h * g[1];
        } else {
            if (i == 0) v = v + (h * wj) * g[0 * S + j];
            if (i == Sx - 1) v = v + (h * wj) * g[1 * S + j];
            if (j == 0) v = v + (h * wi) * g[2 * S + i];
            if (j == S - 1) v = v + (h * wi) * g[3 * S + i];
        }
        b[t] = v;
    }
}
void launch_rhs(const c128* f, const c128* g, c128* b, int dim, int S, double h, cudaStream_t s, int q1) {
    const size_t total = (size_t)S * (dim == 2 ? S : 1);
    k_rhs<<<grid_for(total, 256), 256, 0, s>>>(f, g, b, dim, S, h, q1);
    note_launch();
}

// -------------------------------------------------------------------------- copy
template <typename TS, typename TD>
__global__ void k_copy(const cplx<TS>* __restrict__ src, cplx<TD>* __restrict__ dst, size_t n, bool acc,
                       bool cj) {
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
        cplx<TD> v = cvt<TD>(src[t]);
        if (cj) v = conj(v);
        dst[t] = acc ? dst[t] + v : v;
    }
}
template <typename TS, typename TD>
void launch_copy(const cplx<TS>* src, cplx<TD>* dst, size_t n, bool accumulate, bool conjugate,
                 cudaStream_t s) {
    if (n == 0) return;
    k_copy<TS, TD><<<grid_for(n, 256), 256, 0, s>>>(src, dst, n, accumulate, conjugate);
    note_launch();
}

// ------------------------------------------------------------- interface traces
// Boundary row (local row 0 of a band of b_s rows; by symmetry the same for the last
// row) of A~_s: coefficient op_diag on the row itself, -1/2 to the x-neighbours on the
// row (X halved by w_j = 1/2), -w_i to the inward row.
// Bilinear elements: the boundary row couples three columns of the row itself and three of
// the inward row, with q1_coef(0, 0, i, di) and q1_coef(0, 1, i, di) (the same for the last
// row by symmetry).
template <typename T>
__global__ void k_robin_trace(const cplx<T>* __restrict__ uif, const cplx<T>* __restrict__ uin,
                              cplx<T>* __restrict__ Y, int b_s, int Sx, int nc, double kh,
                              const double* khr_row, int q1) {
    const OpGeom g{b_s, Sx, kh, khr_row, q1};
    const size_t total = (size_t)Sx * nc;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
         t += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(t / nc);
        if (q1) {
            c128 y = {0.0, 0.0};
            for (int di = -1; di <= 1; ++di) {
                if (i + di < 0 || i + di >= Sx) continue;
                const size_t tn = (size_t)((long long)t + (long long)di * nc);
                y = y + q1_coef(0, 0, i, di, g) * cvt<double>(uif[tn]) + q1_coef(0, 1, i, di, g) * cvt<double>(uin[tn]);
            }
            Y[t] = cvt<T>(y);
            continue;
        }
        const c128 d = op_diag(0, i, g);
        c128 y = d * cvt<double>(uif[t]);
        if (Sx > 1) {
            if (i > 0) y = y - 0.5 * cvt<double>(uif[t - nc]);
            if (i < Sx - 1) y = y - 0.5 * cvt<double>(uif[t + nc]);
        }
        y = y - wcol(i, Sx) * cvt<double>(uin[t]);
        Y[t] = cvt<T>(y);
    }
}
template <typename T>
void launch_robin_trace(const cplx<T>* u_if, const cplx<T>* u_in, cplx<T>* Y, int b_s, int Sx, int nc,
                        double kh, const double* khr_row, cudaStream_t s, int q1) {
    const size_t total = (size_t)Sx * nc;
    k_robin_trace<T><<<grid_for(total, 256), 256, 0, s>>>(u_if, u_in, Y, b_s, Sx, nc, kh, khr_row, q1);
    note_launch();
}

template <typename T>
__global__ void k_adjoint_place(const cplx<T>* __restrict__ Q, cplx<T>* __restrict__ vif,
                                cplx<T>* __restrict__ vin, int b_s, int Sx, int nc, double kh,
                                const double* khr_row, int q1) {
    const OpGeom g{b_s, Sx, kh, khr_row, q1};
    const size_t total = (size_t)Sx * nc;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
         t += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(t / nc);
        if (q1) {
            // the transposed trace: both coefficient rows are symmetric in (i, i + di)
            c128 yi = {0.0, 0.0}, yn = {0.0, 0.0};
            for (int di = -1; di <= 1; ++di) {
                if (i + di < 0 || i + di >= Sx) continue;
                const c128 q = conj(cvt<double>(Q[(size_t)((long long)t + (long long)di * nc)]));
                yi = yi + q1_coef(0, 0, i, di, g) * q;
                yn = yn + q1_coef(0, 1, i, di, g) * q;
            }
            vif[t] = cvt<T>(yi);
            vin[t] = cvt<T>(yn);
            continue;
        }
        const c128 d = op_diag(0, i, g);
        const c128 q = conj(cvt<double>(Q[t]));
        c128 y = d * q;
        if (Sx > 1) {
            if (i > 0) y = y - 0.5 * conj(cvt<double>(Q[t - nc]));
            if (i < Sx - 1) y = y - 0.5 * conj(cvt<double>(Q[t + nc]));
        }
        vif[t] = cvt<T>(y);
        vin[t] = cvt<T>((-wcol(i, Sx)) * q);
    }
}
template <typename T>
void launch_adjoint_place(const cplx<T>* Q, cplx<T>* v_if, cplx<T>* v_in, int b_s, int Sx, int nc,
                          double kh, const double* khr_row, cudaStream_t s, int q1) {
    const size_t total = (size_t)Sx * nc;
    k_adjoint_place<T><<<grid_for(total, 256), 256, 0, s>>>(Q, v_if, v_in, b_s, Sx, nc, kh, khr_row, q1);
    note_launch();
}

// ------------------------------------------------------------------ sketch (RNG)
// SplitMix64 (Steele, Lea & Flood 2014): n-th output = mix(seed + (n+1) * gamma).
__device__ __forceinline__ unsigned long long splitmix64_at(unsigned long long seed,
                                                            unsigned long long n) {
    unsigned long long z = seed + (n + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
template <typename T>
__global__ void k_sketch(cplx<T>* Om, int Sx, int m, int node, unsigned long long seed) {
    const size_t total = (size_t)Sx * m;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
         t += (size_t)gridDim.x * blockDim.x) {
        const unsigned long long j = t % m, x = t / m;
        const unsigned long long idx = ((unsigned long long)node * 4096ull + j) * (1ull << 20) + x;
        const unsigned long long z1 = splitmix64_at(seed, 2ull * idx);
        const unsigned long long z2 = splitmix64_at(seed, 2ull * idx + 1ull);
        const double u1 = ((double)(z1 >> 11) + 1.0) * 0x1.0p-53;
        const double u2 = (double)(z2 >> 11) * 0x1.0p-53;
        const double rho = sqrt(-2.0 * log(u1)) * 0.70710678118654752440;
        double sn, cs;
        sincospi(2.0 * u2, &sn, &cs);
        Om[t] = cplx<T>{(T)(rho * cs), (T)(rho * sn)};
    }
}
template <typename T>
void launch_sketch(cplx<T>* Om, int Sx, int m, int node, unsigned long long seed, cudaStream_t s) {
    k_sketch<T><<<grid_for((size_t)Sx * m, 256), 256, 0, s>>>(Om, Sx, m, node, seed);
    note_launch();
}

// ---------------------------------------------------------------- coarse update
template <typename TC, typename TW>
__global__ void k_coarse_update(const cplx<TC>* __restrict__ C, const c128* __restrict__ y,
                                cplx<TW>* __restrict__ W, size_t npts, int p, int nc) {
    extern __shared__ c128 ys[];
    for (int t = threadIdx.x; t < p * nc; t += blockDim.x) ys[t] = y[t];
    __syncthreads();
    const size_t total = npts * nc;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
         t += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(t % nc);
        const size_t pt = t / nc;
        // the correction is accumulated in the precision of the basis C
        const cplx<TC>* cr = C + pt * p;
        cplx<TC> acc = {0, 0};
        for (int j = 0; j < p; ++j) cfma(acc, cr[j], cvt<TC>(ys[j * nc + c]));
        W[t] = W[t] + cvt<TW>(acc);
    }
}
// Single column (nc = 1): a warp per point, lanes across the p basis columns, so that
// each row of C is read as one contiguous segment.
template <typename TC, typename TW>
__global__ void k_coarse_update1(const cplx<TC>* __restrict__ C, const c128* __restrict__ y,
                                 cplx<TW>* __restrict__ W, size_t npts, int p) {
    __shared__ cplx<TC> ys[128];
    for (int t = threadIdx.x; t < p; t += blockDim.x) ys[t] = cvt<TC>(y[t]);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const size_t nwarp = (size_t)gridDim.x * (blockDim.x >> 5);
    for (size_t pt = (size_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); pt < npts; pt += nwarp) {
        const cplx<TC>* cr = C + pt * p;
        cplx<TC> acc = {0, 0};
        for (int j = lane; j < p; j += 32) cfma(acc, cr[j], ys[j]);
        acc = warp_sum(acc);
        if (lane == 0) W[pt] = W[pt] + cvt<TW>(acc);
    }
}

template <typename TC, typename TW>
void launch_coarse_update(const cplx<TC>* C, const c128* y, cplx<TW>* W, size_t npts, int p, int nc,
                          cudaStream_t s) {
    if (nc == 1 && p <= 128) {
        k_coarse_update1<TC, TW><<<grid_for(npts, 8), 256, 0, s>>>(C, y, W, npts, p);
        note_launch();
        return;
    }
    const size_t total = npts * nc;
    k_coarse_update<TC, TW><<<grid_for(total, 256), 256, sizeof(c128) * p * nc, s>>>(C, y, W, npts, p, nc);
    note_launch();
}

// --------------------------------------------------------- Krylov basis helpers
// Basis matrices are stored point-major: B[n * ld + j] is entry n of basis vector j.
__global__ void k_col_load(const c128* __restrict__ B, int ld, int col, c128* __restrict__ dst, size_t n) {
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
        dst[t] = B[t * ld + col];
}
void launch_col_load(const c128* B, int ld, int col, c128* dst, size_t n, cudaStream_t s) {
    k_col_load<<<grid_for(n, 256), 256, 0, s>>>(B, ld, col, dst, n);
    note_launch();
}
// B[n][col] = src[n] / sqrt(*nrm2)   (nrm2 read on the device; zero if nrm2 == 0)
__global__ void k_col_store_normalised(c128* __restrict__ B, int ld, int col, const c128* __restrict__ src,
                                       const c128* __restrict__ nrm2, size_t n) {
    const double v = nrm2->re;
    const double sc = v > 0.0 ? 1.0 / sqrt(v) : 0.0;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
        B[t * ld + col] = sc * src[t];
}
void launch_col_store_normalised(c128* B, int ld, int col, const c128* src, const c128* nrm2, size_t n,
                                 cudaStream_t s) {
    k_col_store_normalised<<<grid_for(n, 256), 256, 0, s>>>(B, ld, col, src, nrm2, n);
    note_launch();
}
// w[n] += sgn * sum_{i<j} B[n][i] * c_i, with c_i = conj(coef[i]) if cj else coef[i]
__global__ void k_basis_combine(const c128* __restrict__ B, int ld, int j, const c128* __restrict__ coef, bool cj,
                                double sgn, c128* __restrict__ w, size_t n) {
    __shared__ c128 cs[128];
    for (int i = threadIdx.x; i < j; i += blockDim.x) {
        const c128 c = cj ? conj(coef[i]) : coef[i];
        cs[i] = sgn * c;
    }
    __syncthreads();
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
        c128 a = w[t];
        const c128* br = B + t * ld;
        for (int i = 0; i < j; ++i) cfma(a, br[i], cs[i]);
        w[t] = a;
    }
}
void launch_basis_combine(const c128* B, int ld, int j, const c128* coef, bool cj, double sgn, c128* w, size_t n,
                          cudaStream_t s) {
    k_basis_combine<<<grid_for(n, 256), 256, 0, s>>>(B, ld, j, coef, cj, sgn, w, n);
    note_launch();
}

// ------------------------------------------------------------ instantiations
#define HH_APPLY(TX, TV, TY)                                                                           \
    template void launch_apply<TX, TV, TY>(const cplx<TX>*, const cplx<TV>*, cplx<TY>*, OpGeom, int, \
                                           double, double*, int*, cudaStream_t);
HH_APPLY(double, double, double)
HH_APPLY(float, float, float)
HH_APPLY(float, double, double)
HH_APPLY(double, float, float)

// ------------------------------------------------ GMRES least squares on the device
__global__ void k_gmres_init(GmresLs ls, double beta) {
    if (threadIdx.x != 0) return;
    for (int i = 0; i <= ls.mk; ++i) ls.g[i] = {0.0, 0.0};
    ls.g[0] = {beta, 0.0};
    *ls.st = GmresState{0, 0, 0, 0, 0.0, 0.0};
}
// The steps of a plain Givens QR of the Hessenberg matrix, column by column (the complex
// rotation [c s; -conj(s) c] with real c zeroing the subdiagonal entry hn).
__global__ void k_gmres_rotate(GmresLs ls, const c128* d1, const c128* d2, const c128* dn, int j, double nbv,
                               double tol) {
    if (threadIdx.x != 0 || ls.st->stop) return;
    const int mk = ls.mk;
    c128* H = ls.H;
    for (int i = 0; i <= j; ++i) H[(size_t)i * mk + j] = conj(d1[i]) + conj(d2[i]);
    const double hn = sqrt(fmax(dn->re, 0.0));
    for (int i = 0; i < j; ++i) {
        const c128 a0 = H[(size_t)i * mk + j], a1 = H[(size_t)(i + 1) * mk + j];
        H[(size_t)i * mk + j] = ls.cs[i] * a0 + ls.sn[i] * a1;
        H[(size_t)(i + 1) * mk + j] = ls.cs[i] * a1 - conj(ls.sn[i]) * a0;
    }
    const c128 a = H[(size_t)j * mk + j];
    const double aa = sqrt(abs2(a)), t = sqrt(abs2(a) + hn * hn);
    if (t == 0.0) {
        ls.cs[j] = 1.0;
        ls.sn[j] = {0.0, 0.0};
    } else if (aa == 0.0) {
        ls.cs[j] = 0.0;
        ls.sn[j] = {1.0, 0.0};
        H[(size_t)j * mk + j] = {hn, 0.0};
    } else {
        const c128 ph = (1.0 / aa) * a;
        ls.cs[j] = aa / t;
        ls.sn[j] = (hn / t) * ph;
        H[(size_t)j * mk + j] = t * ph;
    }
    ls.g[j + 1] = -(conj(ls.sn[j]) * ls.g[j]);
    ls.g[j] = ls.cs[j] * ls.g[j];
    GmresState* st = ls.st;
    st->steps = j + 1;
    const double est = nbv > 0 ? sqrt(abs2(ls.g[j + 1])) / nbv : 0.0;
    st->est = est;
    if (!isfinite(est)) {
        st->bad = 1;
        st->stop = 1;
        st->jstop = j + 1;
    } else if (est < 0.5 * tol || hn == 0.0) {
        st->stop = 1;
        st->jstop = j + 1;
    }
}
__global__ void k_gmres_solve(GmresLs ls, int jn, c128* y) {
    if (threadIdx.x != 0) return;
    const int mk = ls.mk;
    for (int i = jn - 1; i >= 0; --i) {
        c128 acc = ls.g[i];
        for (int k = i + 1; k < jn; ++k) acc = acc - ls.H[(size_t)i * mk + k] * y[k];
        const c128 d = ls.H[(size_t)i * mk + i];
        y[i] = abs2(d) > 0 ? acc * cinv(d) : c128{0.0, 0.0};
    }
}
void launch_gmres_init(GmresLs ls, double beta, cudaStream_t s) {
    k_gmres_init<<<1, 32, 0, s>>>(ls, beta);
    note_launch();
}
void launch_gmres_rotate(GmresLs ls, const c128* d1, const c128* d2, const c128* dn, int j, double nbv, double tol,
                         cudaStream_t s) {
    k_gmres_rotate<<<1, 32, 0, s>>>(ls, d1, d2, dn, j, nbv, tol);
    note_launch();
}
void launch_gmres_solve(GmresLs ls, int jn, c128* y, cudaStream_t s) {
    k_gmres_solve<<<1, 32, 0, s>>>(ls, jn, y);
    note_launch();
}

#define HH_COPY(TS, TD) \
    template void launch_copy<TS, TD>(const cplx<TS>*, cplx<TD>*, size_t, bool, bool, cudaStream_t);
HH_COPY(double, double)
HH_COPY(float, float)
HH_COPY(double, float)
HH_COPY(float, double)

#define HH_PREC(T)                                                                                    \
    template void launch_robin_trace<T>(const cplx<T>*, const cplx<T>*, cplx<T>*, int, int, int, double, const double*, \
                                        cudaStream_t, int);                                           \
    template void launch_adjoint_place<T>(const cplx<T>*, cplx<T>*, cplx<T>*, int, int, int, double, const double*,   \
                                          cudaStream_t, int);                                         \
    template void launch_sketch<T>(cplx<T>*, int, int, int, unsigned long long, cudaStream_t);

HH_PREC(float)
HH_PREC(double)
template void launch_coarse_update<float, float>(const c64*, const c128*, c64*, size_t, int, int, cudaStream_t);

template void launch_coarse_update<float, double>(const c64*, const c128*, c128*, size_t, int, int, cudaStream_t);
template void launch_coarse_update<double, double>(const c128*, const c128*, c128*, size_t, int, int,
                                                   cudaStream_t);

}  // namespace hh
