// k_coarse.cu -- the coarse correction of Eq. (3), w <- w + C_p A_c^{-1} C_p^H (v - A~_p w),
// with the coarse basis stored column-major: C[j * N + pt], j < p = 2r, pt < N points of
// the node's band, so that every kernel below reads C with consecutive threads on
// consecutive points.
#include <algorithm>

#include "kernels.h"

namespace hh {

static int blocks_for(size_t n, int threads, int cap) {
    size_t g = (n + threads - 1) / threads;
    if (g > (size_t)cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

// C[(coff + j) * ldc + dst0 + q] = src[(src0 + q) * r + j], q < n, j < r
// (scatter of a child's extension [points][r] into its block of the parent's basis).
template <typename T>
__global__ void k_build_basis(const cplx<T>* __restrict__ src, size_t src0, int r, cplx<T>* __restrict__ C,
                              size_t ldc, int coff, size_t dst0, size_t n) {
    const size_t total = n * r;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(t / n);
        const size_t q = t - (size_t)j * n;
        C[(size_t)(coff + j) * ldc + dst0 + q] = src[(src0 + q) * r + j];
    }
}
template <typename T>
void launch_build_basis(const cplx<T>* src, size_t src0, int r, cplx<T>* C, size_t ldc, int coff, size_t dst0,
                        size_t n, cudaStream_t s) {
    k_build_basis<T><<<blocks_for(n * r, 256, 152 * 8), 256, 0, s>>>(src, src0, r, C, ldc, coff, dst0, n);
    note_launch();
}

// One column.  A block takes 256 consecutive points per step: first every thread forms
// r_pt = v_pt - (A~ w)_pt for one point (w may be null: r = v) in the precision of v and
// w and leaves it in shared memory; then its four groups of 64 threads each accumulate a
// quarter of the p columns over the 256 points (coalesced reads of C along the points).
// Per-block partial sums go to `partial`; the last block to finish (ticket counter) adds
// them in block order (FP64), multiplies by the FP64 inverse Galerkin matrix, writes
// y = A_c^{-1} C^H r and resets the counter.
template <typename TC, typename TV, typename TW, typename ACC>
__global__ void __launch_bounds__(256) k_coarse_proj1(const cplx<TC>* __restrict__ C, const cplx<TV>* __restrict__ v,
                                                      const cplx<TW>* __restrict__ w, OpGeom g, int p,
                                                      c128* __restrict__ partial, unsigned* counter,
                                                      const c128* __restrict__ Minv, c128* __restrict__ y) {
    using CA = cplx<ACC>;
    using R = decltype(TV() + TW());
    __shared__ CA red[8][16];
    __shared__ CA s_r[256];
    __shared__ unsigned ticket;
    __shared__ c128 s_sum[64];
    __shared__ c128 s_m[64 * 64];
    const unsigned N = (unsigned)g.b * (unsigned)g.Sx;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int q = threadIdx.x & 63, jg = threadIdx.x >> 6;        // point in sub-tile, column group
    const int per = (p + 3) / 4, ja = jg * per, jb = min(p, ja + per);
    // the last block needs A_c^{-1}: every block starts its copy into shared memory now,
    // so that it has long arrived when the last block gets there
    for (int t = threadIdx.x; t < p * p; t += blockDim.x) cp_async16(s_m + t, Minv + t);
    cp_async_commit();
    CA acc[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) acc[j] = {0, 0};
    for (unsigned base = blockIdx.x * 256u; base < N; base += gridDim.x * 256u) {
        {
            const unsigned pt = base + threadIdx.x;
            CA ra = {0, 0};
            if (pt < N) {
                cplx<R> rv = cvt<R>(v[pt]);
                if (w) {
                    const int jr = (int)(pt / (unsigned)g.Sx), i = (int)(pt - (unsigned)jr * g.Sx);
                    cplx<R> ax = op_diag_t<R>(jr, i, g) * cvt<R>(w[pt]);
                    const R wj = (jr == 0 || jr == g.b - 1) ? (R)0.5 : (R)1;
                    const R wi = g.Sx == 1 ? (R)1 : ((i == 0 || i == g.Sx - 1) ? (R)0.5 : (R)1);
                    if (g.Sx > 1) {
                        if (i > 0) ax = ax - wj * cvt<R>(w[pt - 1]);
                        if (i < g.Sx - 1) ax = ax - wj * cvt<R>(w[pt + 1]);
                    }
                    if (jr > 0) ax = ax - wi * cvt<R>(w[pt - g.Sx]);
                    if (jr < g.b - 1) ax = ax - wi * cvt<R>(w[pt + g.Sx]);
                    rv = rv - ax;
                }
                ra = cvt<ACC>(rv);
            }
            s_r[threadIdx.x] = ra;
        }
        __syncthreads();
#pragma unroll 2
        for (int sub = 0; sub < 4; ++sub) {
            const unsigned pt = base + sub * 64 + q;
            if (pt < N) {
                cplx<TC> cv[16];
#pragma unroll
                for (int u = 0; u < 16; ++u) cv[u] = (ja + u < jb) ? C[(size_t)(ja + u) * N + pt] : cplx<TC>{0, 0};
                const CA ra = s_r[sub * 64 + q];
#pragma unroll
                for (int u = 0; u < 16; ++u) cfma_cj(acc[u], cvt<ACC>(cv[u]), ra);
            }
        }
        __syncthreads();
    }
    // both warps of a column group hold the group's columns: reduce over lanes, then over
    // the two warps in shared memory
#pragma unroll
    for (int u = 0; u < 16; ++u) {
        const CA t = warp_sum(acc[u]);
        if (lane == 0) red[warp][u] = t;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < p; t += blockDim.x) {
        const int grp = t / per, u = t - grp * per;
        const CA s = red[2 * grp][u] + red[2 * grp + 1][u];
        partial[(size_t)blockIdx.x * p + t] = cvt<double>(s);
    }
    __threadfence();
    cp_async_wait_all();
    __syncthreads();
    if (threadIdx.x == 0) ticket = atomicAdd(counter, 1u);
    __syncthreads();
    if (ticket != gridDim.x - 1) return;
    __threadfence();
    // last block: 8 threads per output add the blocks' partials (fixed order within each
    // thread, then a fixed shuffle tree), loads bypassing L1 (__ldcg)
    // the loop bound is warp-uniform (every lane of a warp reaches the shuffles)
    const int sub = threadIdx.x & 7;
    for (int j0 = 0; j0 < p; j0 += blockDim.x >> 3) {
        const int j = j0 + (threadIdx.x >> 3);
        const bool ok = j < p;
        // partials b = sub, sub + 8, ...: eight loads in flight per thread, added in
        // index order
        c128 t0 = {0.0, 0.0}, t1 = {0.0, 0.0};
        if (ok) {
            for (unsigned b0 = sub; b0 < gridDim.x; b0 += 64) {
                double2 a[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const unsigned bb = b0 + 8u * u;
                    a[u] = bb < gridDim.x ? __ldcg((const double2*)(partial + (size_t)bb * p + j)) : make_double2(0.0, 0.0);
                }
#pragma unroll
                for (int u = 0; u < 8; u += 2) {
                    t0 = t0 + c128{a[u].x, a[u].y};
                    t1 = t1 + c128{a[u + 1].x, a[u + 1].y};
                }
            }
        }
        c128 t = t0 + t1;
        for (int o = 4; o > 0; o >>= 1) {
            t.re += __shfl_xor_sync(0xffffffffu, t.re, o);
            t.im += __shfl_xor_sync(0xffffffffu, t.im, o);
        }
        if (ok && sub == 0) s_sum[j] = t;
    }
    __syncthreads();
    // y = A_c^{-1} s: 8 threads per output (k = sub, sub + 8, ...), fixed shuffle tree
    for (int j0 = 0; j0 < p; j0 += blockDim.x >> 3) {
        const int j = j0 + (threadIdx.x >> 3);
        c128 t = {0.0, 0.0};
        if (j < p)
            for (int k = sub; k < p; k += 8) cfma(t, s_m[j * p + k], s_sum[k]);
        for (int o = 4; o > 0; o >>= 1) {
            t.re += __shfl_xor_sync(0xffffffffu, t.re, o);
            t.im += __shfl_xor_sync(0xffffffffu, t.im, o);
        }
        if (j < p && sub == 0) y[j] = t;
    }
    if (threadIdx.x == 0) *counter = 0u;
}

template <typename TC, typename TV, typename TW>
void launch_coarse_proj1(const cplx<TC>* C, const cplx<TV>* v, const cplx<TW>* w, OpGeom g, int p, c128* partial,
                         unsigned* counter, const c128* Minv, c128* y, cudaStream_t s) {
    const size_t N = (size_t)g.b * g.Sx;
    // one block per SM at most: the last block's reduction reads grid x p partials
    const int grid = blocks_for(N, 256, 152);
    k_coarse_proj1<TC, TV, TW, TC><<<grid, 256, 0, s>>>(C, v, w, g, p, partial, counter, Minv, y);
    note_launch();
}

// ------------------------------------------------------- fused one-column correction
// Barrier over a cooperative grid (all blocks resident): arrive on a counter, the last
// arriver resets it and advances the generation; the others wait on the generation with
// a bounded spin (DEV_TIMEOUT and false after about a second).
__device__ bool grid_barrier(unsigned* bar, int* err) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        volatile unsigned* gen = bar + 1;
        const unsigned g0 = *gen;
        __threadfence();
        if (atomicAdd(bar, 1u) == gridDim.x - 1) {
            bar[0] = 0u;            // no block touches the counter again before the generation moves
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            // spin without sleeping first (the release is usually a few microseconds
            // away), then back off; give up after about a second
            long long it = 0;
            while (*gen == g0) {
                if (++it > (1ll << 24)) {
                    atomicExch(err, DEV_TIMEOUT);
                    ok = 0;
                    break;
                }
                if (it > 4096) __nanosleep(64);
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// One-column coarse corrections of several nodes (Eq. (3)) in one cooperative launch;
// job k owns blocks [blk0, blk0 + nblk).  For each job:
//   phase 1: r = v - A~ w_in (w_in may be null: r = v), formed once per point in shared
//            memory, and per-block partial sums of C^H r in the basis precision (four
//            column groups, coalesced reads of C along the points);
//   grid barrier;
//   phase 2: every block of the job adds the job's partials in the same fixed order and
//            multiplies by A_c^{-1} (basis precision; copied to shared memory with
//            cp.async while phase 1 ran), so all of them hold the same y;
//   phase 3: for the points it projected whose rows lie in [r0, r1):
//            out[pt - r0 Sx] = (acc_out ? out : 0) + (add_w ? w_in[pt] : 0) + (C y)[pt]
//            (in place: out = w_in, acc_out; straight into the parent's solution: the
//            owned rows, add_w).  The barrier separates every read of w_in from the
//            writes.
template <typename TC, typename TV, typename TW, typename TO>
__global__ void __launch_bounds__(256) k_coarse_batch(CoarseBatch bt, int p, cplx<TC>* partial, unsigned* bar,
                                                      int* err) {
    // a set stop word (written by an earlier launch: the same for every block) skips the
    // launch before the grid barrier
    if (bt.gate && *bt.gate) return;
    using CA = cplx<TC>;
    using R = decltype(TV() + TW());
    __shared__ CA red[8][16];
    __shared__ CA s_r[256];
    __shared__ CA s_sum[64];
    __shared__ CA s_y[64];
    __shared__ __align__(16) CA s_m[64 * 64];
    int jb_ = 0;
    while (jb_ + 1 < bt.njobs && blockIdx.x >= bt.job[jb_ + 1].blk0) ++jb_;
    const CoarseJob& J = bt.job[jb_];
    const cplx<TC>* __restrict__ C = (const cplx<TC>*)J.C;
    const cplx<TV>* __restrict__ v = (const cplx<TV>*)J.v;
    const cplx<TW>* w_in = (const cplx<TW>*)J.w_in;
    const OpGeom g = J.g;
    const unsigned lb = blockIdx.x - J.blk0, nblk = J.nblk;
    const unsigned N = (unsigned)g.b * (unsigned)g.Sx;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int q = threadIdx.x & 63, jg = threadIdx.x >> 6;
    const int per = (p + 3) / 4, ja = jg * per, jb = min(p, ja + per);
    {
        const int chunks = (int)(sizeof(CA) * p * p / 16);
        for (int t = threadIdx.x; t < chunks; t += blockDim.x)
            cp_async16((char*)s_m + 16 * t, (const char*)J.Minv + 16 * t);
        cp_async_commit();
    }
    CA acc[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) acc[j] = {0, 0};
    for (unsigned base = lb * 256u; base < N; base += nblk * 256u) {
        {
            const unsigned pt = base + threadIdx.x;
            CA ra = {0, 0};
            if (pt < N) {
                cplx<R> rv = cvt<R>(v[pt]);
                if (w_in) {
                    const int jr = (int)(pt / (unsigned)g.Sx), i = (int)(pt - (unsigned)jr * g.Sx);
                    cplx<R> ax = op_diag_t<R>(jr, i, g) * cvt<R>(w_in[pt]);
                    const R wj = (jr == 0 || jr == g.b - 1) ? (R)0.5 : (R)1;
                    const R wi = g.Sx == 1 ? (R)1 : ((i == 0 || i == g.Sx - 1) ? (R)0.5 : (R)1);
                    if (g.Sx > 1) {
                        if (i > 0) ax = ax - wj * cvt<R>(w_in[pt - 1]);
                        if (i < g.Sx - 1) ax = ax - wj * cvt<R>(w_in[pt + 1]);
                    }
                    if (jr > 0) ax = ax - wi * cvt<R>(w_in[pt - g.Sx]);
                    if (jr < g.b - 1) ax = ax - wi * cvt<R>(w_in[pt + g.Sx]);
                    rv = rv - ax;
                }
                ra = cvt<TC>(rv);
            }
            s_r[threadIdx.x] = ra;
        }
        __syncthreads();
#pragma unroll 2
        for (int sub = 0; sub < 4; ++sub) {
            const unsigned pt = base + sub * 64 + q;
            if (pt < N) {
                // a column whose child does not own this row is zero there: not read
                const int half = J.split < 0 ? -1 : ((int)(pt / (unsigned)g.Sx) < J.split ? 0 : 1);
                cplx<TC> cv[16];
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    const int j = ja + u;
                    const bool need = j < jb && (half < 0 || (j < (p >> 1)) == (half == 0));
                    cv[u] = need ? C[(size_t)j * N + pt] : cplx<TC>{0, 0};
                }
                const CA ra = s_r[sub * 64 + q];
#pragma unroll
                for (int u = 0; u < 16; ++u) cfma_cj(acc[u], cv[u], ra);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 16; ++u) {
        const CA t = warp_sum(acc[u]);
        if (lane == 0) red[warp][u] = t;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < p; t += blockDim.x) {
        const int grp = t / per, u = t - grp * per;
        partial[(size_t)blockIdx.x * p + t] = red[2 * grp][u] + red[2 * grp + 1][u];
    }
    cp_async_wait_all();
    if (!grid_barrier(bar, err)) return;
    // phase 2: the same sums in every block of the job: 8 threads per output, partials
    // b = sub, sub + 8, ... in order, then a fixed shuffle tree
    const int sub = threadIdx.x & 7;
    const CA* jp = partial + (size_t)J.blk0 * p;
    for (int j0 = 0; j0 < p; j0 += blockDim.x >> 3) {
        const int j = j0 + (threadIdx.x >> 3);
        // all of a thread's partials requested at once (one round trip for up to
        // 8 PU blocks), then added in index order
        constexpr int PU = sizeof(TC) == 4 ? 24 : 12;
        CA t0 = {0, 0}, t1 = {0, 0};
        if (j < p) {
            for (unsigned b0 = sub; b0 < nblk; b0 += 8 * PU) {
                CA a[PU];
#pragma unroll
                for (int u = 0; u < PU; ++u) {
                    const unsigned bb = b0 + 8u * u;
                    a[u] = bb < nblk ? jp[(size_t)bb * p + j] : CA{0, 0};
                }
#pragma unroll
                for (int u = 0; u < PU; u += 2) {
                    t0 = t0 + a[u];
                    t1 = t1 + a[u + 1];
                }
            }
        }
        CA t = t0 + t1;
        for (int o = 4; o > 0; o >>= 1) {
            t.re += __shfl_xor_sync(0xffffffffu, t.re, o);
            t.im += __shfl_xor_sync(0xffffffffu, t.im, o);
        }
        if (j < p && sub == 0) s_sum[j] = t;
    }
    __syncthreads();
    for (int j0 = 0; j0 < p; j0 += blockDim.x >> 3) {
        const int j = j0 + (threadIdx.x >> 3);
        CA t = {0, 0};
        if (j < p)
            for (int k = sub; k < p; k += 8) cfma(t, s_m[j * p + k], s_sum[k]);
        for (int o = 4; o > 0; o >>= 1) {
            t.re += __shfl_xor_sync(0xffffffffu, t.re, o);
            t.im += __shfl_xor_sync(0xffffffffu, t.im, o);
        }
        if (j < p && sub == 0) {
            s_y[j] = t;
            if (lb == 0 && J.y) J.y[j] = cvt<double>(t);
        }
    }
    __syncthreads();
    // phase 3: one point per thread, all p columns (coalesced along the points)
    cplx<TO>* out = (cplx<TO>*)J.out;
    const unsigned lo = (unsigned)J.r0 * g.Sx, hi = (unsigned)J.r1 * g.Sx;
    for (unsigned base = lb * 256u; base < N; base += nblk * 256u) {
        const unsigned pt = base + threadIdx.x;
        if (pt < lo || pt >= hi) continue;
        CA a = {0, 0};
        // only the columns of the child that owns this row are nonzero
        int j = 0, je = p;
        if (J.split >= 0) {
            if ((int)(pt / (unsigned)g.Sx) < J.split) je = p >> 1;
            else j = p >> 1;
        }
        for (; j + 8 <= je; j += 8) {
            cplx<TC> cv[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) cv[u] = C[(size_t)(j + u) * N + pt];
#pragma unroll
            for (int u = 0; u < 8; ++u) cfma(a, cv[u], s_y[j + u]);
        }
        for (; j < je; ++j) cfma(a, C[(size_t)j * N + pt], s_y[j]);
        cplx<TO> val = cvt<TO>(a);
        if (J.add_w) val = val + cvt<TO>(w_in[pt]);
        cplx<TO>& o = out[pt - lo];
        o = J.acc_out ? o + val : val;
    }
}

template <typename TC, typename TV, typename TW, typename TO>
int coarse_batch_max_grid() {
    static int mg = 0;
    if (!mg) {
        int dev = 0, sms = 0, nb = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_coarse_batch<TC, TV, TW, TO>, 256, 0);
        mg = std::max(1, std::min(nb, 2) * sms);
    }
    return mg;
}

template <typename TC, typename TV, typename TW, typename TO>
void launch_coarse_batch(CoarseBatch bt, int p, void* partial, unsigned* bar, int* err, cudaStream_t s) {
    if (bt.njobs < 1) return;
    // blocks per job: one per 256 points, at most 152 per job (phase 2 reads every partial
    // of the job), within the co-resident total
    const int mg = coarse_batch_max_grid<TC, TV, TW, TO>();
    const int cap = std::max(1, std::min(152, mg / bt.njobs));
    unsigned blk = 0;
    for (int k = 0; k < bt.njobs; ++k) {
        const size_t N = (size_t)bt.job[k].g.b * bt.job[k].g.Sx;
        bt.job[k].blk0 = blk;
        bt.job[k].nblk = (unsigned)blocks_for(N, 256, cap);
        blk += bt.job[k].nblk;
    }
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    cfg.gridDim = dim3(blk);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, k_coarse_batch<TC, TV, TW, TO>, bt, p, (cplx<TC>*)partial, bar, err);
    note_launch();
}

// W[pt] += sum_j C[j][pt] y[j]  (one column; accumulated in the basis precision).
// A block takes 64 consecutive points; its four groups of 64 threads each sum a quarter
// of the p columns (coalesced reads of C along the points), combined in shared memory.
template <typename TC, typename TW>
__global__ void __launch_bounds__(256) k_coarse_upd1(const cplx<TC>* __restrict__ C, const c128* __restrict__ y,
                                                     cplx<TW>* __restrict__ W, size_t N, int p) {
    __shared__ cplx<TC> ys[64];
    __shared__ cplx<TC> part[4][64];
    // entries past p are multiplied by zero columns: they must be finite, so zero them
    for (int j = threadIdx.x; j < 64; j += blockDim.x) ys[j] = j < p ? cvt<TC>(y[j]) : cplx<TC>{0, 0};
    __syncthreads();
    const int q = threadIdx.x & 63, jg = threadIdx.x >> 6;
    const int per = (p + 3) / 4, ja = jg * per, jb = min(p, ja + per);
    for (size_t base = (size_t)blockIdx.x * 64; base < N; base += (size_t)gridDim.x * 64) {
        const size_t pt = base + q;
        cplx<TC> acc = {0, 0};
        if (pt < N) {
            cplx<TC> cv[16];
#pragma unroll
            for (int u = 0; u < 16; ++u) cv[u] = (ja + u < jb) ? C[(size_t)(ja + u) * N + pt] : cplx<TC>{0, 0};
            asm volatile("" ::: "memory");
#pragma unroll
            for (int u = 0; u < 16; ++u) cfma(acc, cv[u], ys[(ja + u) & 63]);
        }
        part[jg][q] = acc;
        __syncthreads();
        if (jg == 0 && pt < N) W[pt] = W[pt] + cvt<TW>((part[0][q] + part[1][q]) + (part[2][q] + part[3][q]));
        __syncthreads();
    }
}
template <typename TC, typename TW>
void launch_coarse_upd1(const cplx<TC>* C, const c128* y, cplx<TW>* W, size_t N, int p, cudaStream_t s) {
    k_coarse_upd1<TC, TW><<<blocks_for(N, 64, 152 * 16), 256, 0, s>>>(C, y, W, N, p);
    note_launch();
}

// Several columns (set-up): W[pt][c] += sum_j C[j][pt] y[j][c].  One thread per point
// and 16 columns at a time: each C[j][pt] is read once per chunk (coalesced along the
// points) and used for all the chunk's columns; y staged in shared memory in the basis
// precision.
template <typename TC, typename TW>
__global__ void __launch_bounds__(256) k_coarse_updn(const cplx<TC>* __restrict__ C, const c128* __restrict__ y,
                                                     cplx<TW>* __restrict__ W, size_t N, int p, int nc) {
    extern __shared__ __align__(16) unsigned char ysm[];
    cplx<TC>* ys = (cplx<TC>*)ysm;   // [p][nc]
    for (int t = threadIdx.x; t < p * nc; t += blockDim.x) ys[t] = cvt<TC>(y[t]);
    __syncthreads();
    for (size_t pt = blockIdx.x * (size_t)blockDim.x + threadIdx.x; pt < N; pt += (size_t)gridDim.x * blockDim.x) {
        for (int c0 = 0; c0 < nc; c0 += 16) {
            const int cn = min(16, nc - c0);
            cplx<TC> acc[16];
#pragma unroll
            for (int c = 0; c < 16; ++c) acc[c] = {0, 0};
            for (int j = 0; j < p; ++j) {
                const cplx<TC> cv = C[(size_t)j * N + pt];
                const cplx<TC>* yr = ys + j * nc + c0;
#pragma unroll
                for (int c = 0; c < 16; ++c)
                    if (c < cn) cfma(acc[c], cv, yr[c]);
            }
            cplx<TW>* wr = W + pt * nc + c0;
#pragma unroll
            for (int c = 0; c < 16; ++c)
                if (c < cn) wr[c] = wr[c] + cvt<TW>(acc[c]);
        }
    }
}
template <typename TC, typename TW>
void launch_coarse_updn(const cplx<TC>* C, const c128* y, cplx<TW>* W, size_t N, int p, int nc, cudaStream_t s) {
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_coarse_updn<TC, TW>, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
        attr = true;
    }
    k_coarse_updn<TC, TW><<<blocks_for(N, 256, 152 * 8), 256, sizeof(cplx<TC>) * p * nc, s>>>(C, y, W, N, p, nc);
    note_launch();
}

template void launch_build_basis<float>(const c64*, size_t, int, c64*, size_t, int, size_t, size_t, cudaStream_t);
template void launch_build_basis<double>(const c128*, size_t, int, c128*, size_t, int, size_t, size_t, cudaStream_t);
template void launch_coarse_proj1<float, float, float>(const c64*, const c64*, const c64*, OpGeom, int, c128*,
                                                       unsigned*, const c128*, c128*, cudaStream_t);
template void launch_coarse_proj1<float, double, double>(const c64*, const c128*, const c128*, OpGeom, int, c128*,
                                                         unsigned*, const c128*, c128*, cudaStream_t);
template void launch_coarse_proj1<double, double, double>(const c128*, const c128*, const c128*, OpGeom, int,
                                                          c128*, unsigned*, const c128*, c128*, cudaStream_t);
template void launch_coarse_batch<float, float, float, float>(CoarseBatch, int, void*, unsigned*, int*, cudaStream_t);
template void launch_coarse_batch<float, float, float, double>(CoarseBatch, int, void*, unsigned*, int*, cudaStream_t);
template void launch_coarse_batch<float, double, double, double>(CoarseBatch, int, void*, unsigned*, int*,
                                                                 cudaStream_t);
template void launch_coarse_batch<double, double, double, double>(CoarseBatch, int, void*, unsigned*, int*,
                                                                  cudaStream_t);
template void launch_coarse_upd1<float, float>(const c64*, const c128*, c64*, size_t, int, cudaStream_t);
template void launch_coarse_upd1<float, double>(const c64*, const c128*, c128*, size_t, int, cudaStream_t);
template void launch_coarse_upd1<double, double>(const c128*, const c128*, c128*, size_t, int, cudaStream_t);
template void launch_coarse_updn<float, float>(const c64*, const c128*, c64*, size_t, int, int, cudaStream_t);
template void launch_coarse_updn<double, double>(const c128*, const c128*, c128*, size_t, int, int, cudaStream_t);

}  // namespace hh
