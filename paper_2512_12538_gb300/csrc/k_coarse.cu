// k_coarse.cu -- the coarse correction of Eq. (3), w <- w + C_p A_c^{-1} C_p^H (v - A~_p w),
// with the coarse basis stored column-major: C[j * N + pt], j < p = 2r, pt < N points of
// the node's band, so that every kernel below reads C with consecutive threads on
// consecutive points.
#include <algorithm>

#include <atomic>

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

// ------------------------------------------------------------- bounded waits
static std::atomic<long long> g_wait_polls{-1};
void set_wait_polls(long long polls) { g_wait_polls.store(polls); }
long long wait_polls(long long dflt) {
    const long long v = g_wait_polls.load();
    return v < 0 ? dflt : v;
}

// ------------------------------------------------------- fused one-column correction
// Barrier over a cooperative grid (all blocks resident): arrive on a counter, the last
// arriver resets it and advances the generation; the others wait on the generation with
// a bounded spin (DEV_TIMEOUT and false after `limit` polls, by default about a second).
__device__ bool grid_barrier(unsigned* bar, int* err, long long limit) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        volatile unsigned* gen = bar + 1;
        const unsigned g0 = *gen;
        __threadfence();
        if (atomicAdd(bar, 1u) == gridDim.x - 1) {
            // the last arriver releases the others (also when some have given up: the
            // counter and generation are consistent again for the next launch)
            bar[0] = 0u;            // no block touches the counter again before the generation moves
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            // spin without sleeping first (the release is usually a few microseconds
            // away), then back off; give up after about a second
            long long it = 0;
            while (limit == 0 || *gen == g0) {   // limit 0: give up at once (testing form)
                if (++it > limit) {
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

// CoarseRecur's end of phase 3: the block's |next residual|^2, then in the last block to
// finish the fixed-order sum and the control words.  The norm only decides when the FP64
// residual is formed, so it is summed in FP32 (the FP64 pipe is slow here).
__device__ __forceinline__ void coarse_recur_tail(const CoarseRecur& R, float rr2, unsigned lb, unsigned nblk) {
    __shared__ float rred[8];
    __shared__ unsigned s_last;
    rr2 = warp_sum(rr2);
    if ((threadIdx.x & 31) == 0) rred[threadIdx.x >> 5] = rr2;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += rred[w];
        ((float*)R.part)[lb] = t;
        __threadfence();
        s_last = atomicAdd(R.ticket, 1u) == nblk - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    float a = 0.f;
    for (unsigned k = threadIdx.x; k < nblk; k += blockDim.x) a += __ldcg((const float*)R.part + k);
    a = warp_sum(a);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) rred[threadIdx.x >> 5] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += rred[w];
        *R.ticket = 0u;
        R.nrm[1] = (double)t;
        const int steps = R.ctl[3] + 1;
        R.ctl[3] = steps;
        const int anchor = (steps % R.anchor) == 0;
        const float b2 = (float)R.nrm[2];
        const float rel = b2 > 0.f ? sqrtf(t / b2) : 0.f;
        R.ctl[4] = anchor;
        R.ctl[2] = (anchor || !isfinite(rel) || rel < 2.f * (float)R.tol) ? 1 : 0;
    }
}

// One-column coarse corrections of several nodes (Eq. (3)) in one cooperative launch;
// job k owns blocks [blk0, blk0 + nblk).  A node's basis has p = 2r columns: those of its
// first child [0, p/2) vanish on the rows at and below `split`, the second child's
// [p/2, p) above it (split < 0: dense).  The launcher cuts each half's columns into
// groups of at most CB_COLS and gives every (half, group) set s = h G + g the job's blocks
// [sb[s], sb[s + 1]); the set's blocks cover the half's points.  For each job:
//   phase 1: each thread takes one point at a time of its block's set: it issues the
//            loads of the set's basis columns at that point together with those of
//            r = v - A~ w_in (w_in may be null: r = v), then accumulates conj(C) r; the
//            block's sums go to partial[block][CB_COLS];
//   grid barrier;
//   phase 2: every block of the job adds, for each column, the partials of the blocks
//            of that column's set in the same fixed order and multiplies by A_c^{-1}
//            (basis precision; copied to shared memory with cp.async while phase 1
//            ran), so all of them hold the same y;
//   phase 3: for the points whose rows lie in [r0, r1):
//            out[pt - r0 Sx] = (acc_out ? out : 0) + (add_w ? w_in[pt] : 0) + (C y)[pt]
//            (in place: out = w_in, acc_out; straight into the parent's solution: the
//            owned rows, add_w), and the added value alone into dout when given.  The
//            barrier separates every read of w_in from the writes.
// Q1: the jobs' operators are the bilinear elements' 9-point rows (a separate instantiation:
// the 5-point kernel keeps its registers).
template <typename TC, typename TV, typename TW, typename TO, bool Q1>
__global__ void __launch_bounds__(256, sizeof(TC) == 4 ? 2 : 1) k_coarse_batch(CoarseBatch bt, int p, cplx<TC>* partial, unsigned* bar,
                                                      int* err) {
    // a set stop word (written by an earlier launch: the same for every block) skips the
    // launch before the grid barrier
    if (bt.gate && *bt.gate) return;
    using CA = cplx<TC>;
    using R = decltype(TV() + TW());
    __shared__ CA red[8][CB_COLS];
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
    const int ph = p >> 1, G = J.ngrp;
    // a job of a problem that has left (the same word for all its blocks): its blocks take
    // part in the grid barrier only, touching none of its buffers
    if (J.gate && *J.gate) {
        grid_barrier(bar, err, bt.wait_polls);
        return;
    }
    {
        const int chunks = (int)(sizeof(CA) * p * p / 16);
        for (int t = threadIdx.x; t < chunks; t += blockDim.x)
            cp_async16((char*)s_m + 16 * t, (const char*)J.Minv + 16 * t);
        cp_async_commit();
    }
    // this block's set: half h, column group gi, columns [c0, c0 + nc), points [P0, P1)
    int st = 0;
    while (st + 1 < 2 * G && lb >= J.sb[st + 1]) ++st;
    const int h = st / G, gi = st - h * G;
    const int c0 = h * ph + gi * CB_COLS, nc = min(CB_COLS, ph - gi * CB_COLS);
    const unsigned nsplit = J.split < 0 ? 0u : (unsigned)J.split * (unsigned)g.Sx;
    const unsigned P0 = (J.split < 0 || h == 0) ? 0u : nsplit;
    const unsigned P1 = (J.split < 0 || h == 1) ? N : nsplit;
    const unsigned ls = lb - J.sb[st], ns = J.sb[st + 1] - J.sb[st];
    CA acc[CB_COLS];
#pragma unroll
    for (int u = 0; u < CB_COLS; ++u) acc[u] = {0, 0};
    // r = v - A~ w_in at one point (w_in null: r = v), in the basis precision
    auto resid_at = [&](unsigned pt) -> CA {
        cplx<R> rv = cvt<R>(v[pt]);
        if (Q1 && w_in) {
            const int jr = (int)(pt / (unsigned)g.Sx), i = (int)(pt - (unsigned)jr * g.Sx);
            rv = rv - q1_row<R>(jr, i, g, [&](int dj, int di) {
                     return cvt<R>(w_in[(size_t)((long long)pt + (long long)dj * g.Sx + di)]);
                 });
        } else if (w_in) {
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
        const CA ra = cvt<TC>(rv);
        if (bt.rr.AC && gi == 0) ((CA*)bt.rr.rp)[pt] = ra;   // r' for the next residual
        return ra;
    };
    // When the launch's basis exceeds the L2, the lines phase 1 reads last are kept for
    // phase 3 (which reads them first): the first (1 - keep) of each sweep is loaded with
    // evict-first priority, the rest with normal priority, and phase 3's loads are
    // evict-first (nothing reads them again in this launch).
    const bool hint = bt.keep < 1.f;
    const unsigned long long pol_first = l2_policy_first(), pol_normal = l2_policy_normal();
    const unsigned pkeep = hint ? P0 + (unsigned)((1.f - bt.keep) * (float)(P1 - P0)) : 0u;
    // two points per iteration: their basis and vector loads are in flight together
    const unsigned stride = ns * 256u;
    unsigned pt = P0 + ls * 256u + threadIdx.x;
    for (; pt + stride < P1; pt += 2u * stride) {
        const unsigned pb = pt + stride;
        const unsigned long long pol = pt < pkeep ? pol_first : pol_normal;
        cplx<TC> ca[CB_COLS], cb[CB_COLS];
#pragma unroll
        for (int u = 0; u < CB_COLS; ++u) {
            ca[u] = u < nc ? ld_hint(C + (size_t)(c0 + u) * N + pt, pol) : CA{0, 0};
            cb[u] = u < nc ? ld_hint(C + (size_t)(c0 + u) * N + pb, pol) : CA{0, 0};
        }
        const CA ra = resid_at(pt), rb = resid_at(pb);
#pragma unroll
        for (int u = 0; u < CB_COLS; ++u) {
            cfma_cj(acc[u], ca[u], ra);
            cfma_cj(acc[u], cb[u], rb);
        }
    }
    if (pt < P1) {
        cplx<TC> cv[CB_COLS];
#pragma unroll
        for (int u = 0; u < CB_COLS; ++u) cv[u] = u < nc ? C[(size_t)(c0 + u) * N + pt] : CA{0, 0};
        const CA ra = resid_at(pt);
#pragma unroll
        for (int u = 0; u < CB_COLS; ++u) cfma_cj(acc[u], cv[u], ra);
    }
#pragma unroll
    for (int u = 0; u < CB_COLS; ++u) {
        const CA t = warp_sum(acc[u]);
        if (lane == 0) red[warp][u] = t;
    }
    __syncthreads();
    if (threadIdx.x < CB_COLS) {
        CA t = red[0][threadIdx.x];
        for (int w = 1; w < 8; ++w) t = t + red[w][threadIdx.x];
        partial[(size_t)blockIdx.x * CB_COLS + threadIdx.x] = t;
    }
    cp_async_wait_all();
    if (!grid_barrier(bar, err, bt.wait_polls)) return;
    // phase 2: the same sums in every block of the job: 8 threads per column, the
    // partials of the column's set b = sub, sub + 8, ... in order, then a fixed shuffle
    // tree
    const int sub = threadIdx.x & 7;
    for (int j0 = 0; j0 < p; j0 += blockDim.x >> 3) {
        const int j = j0 + (threadIdx.x >> 3);
        // all of a thread's partials requested at once (one round trip for up to
        // 8 PU blocks), then added in index order
        constexpr int PU = sizeof(TC) == 4 ? 24 : 12;
        CA t0 = {0, 0}, t1 = {0, 0};
        if (j < p) {
            const int hj = j < ph ? 0 : 1;
            const int gj = (j - hj * ph) / CB_COLS, u = j - hj * ph - gj * CB_COLS;
            const int sj = hj * G + gj;
            const unsigned nbs = J.sb[sj + 1] - J.sb[sj];
            const CA* jp = partial + (size_t)(J.blk0 + J.sb[sj]) * CB_COLS + u;
            for (unsigned b0 = sub; b0 < nbs; b0 += 8 * PU) {
                CA a[PU];
#pragma unroll
                for (int q = 0; q < PU; ++q) {
                    const unsigned bb = b0 + 8u * q;
                    a[q] = bb < nbs ? jp[(size_t)bb * CB_COLS] : CA{0, 0};
                }
#pragma unroll
                for (int q = 0; q < PU; q += 2) {
                    t0 = t0 + a[q];
                    t1 = t1 + a[q + 1];
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
    // phase 3: one point per thread, all p columns (coalesced along the points).  Phase 1
    // swept each half upwards, so the basis lines it read last (the top of each half) are
    // the ones still in the L2: phase 3 takes 256-point chunks from the top of both halves
    // downwards, alternating between the halves while both have chunks left.
    cplx<TO>* out = (cplx<TO>*)J.out;
    const unsigned lo = (unsigned)J.r0 * g.Sx, hi = (unsigned)J.r1 * g.Sx;
    const unsigned n0 = J.split < 0 ? N : nsplit;
    const unsigned nc0 = (n0 + 255u) / 256u, nc1 = (N - n0 + 255u) / 256u;
    const unsigned ncm = min(nc0, nc1), nct = nc0 + nc1;
    float rr2 = 0.f;   // |next residual|^2 of the thread's points (CoarseRecur)
    for (unsigned c = lb; c < nct; c += nblk) {
        unsigned hh, k;
        if (c < 2u * ncm) {
            hh = c & 1u;
            k = c >> 1;
        } else {
            hh = nc0 > nc1 ? 0u : 1u;
            k = c - ncm;
        }
        const unsigned pt = hh == 0 ? (nc0 - 1u - k) * 256u + threadIdx.x : n0 + (nc1 - 1u - k) * 256u + threadIdx.x;
        if (pt >= (hh == 0 ? n0 : N) || pt < lo || pt >= hi) continue;
        CA a = {0, 0};
        // only the columns of the child that owns this row are nonzero
        int j = 0, je = p;
        if (J.split >= 0) {
            if ((int)(pt / (unsigned)g.Sx) < J.split) je = p >> 1;
            else j = p >> 1;
        }
        // sixteen or more basis loads in flight per thread (the columns are far apart in
        // memory)
        const unsigned long long pol3 = hint ? pol_first : pol_normal;
        for (; j + 32 <= je; j += 32) {
            cplx<TC> cv[32];
#pragma unroll
            for (int u = 0; u < 32; ++u) cv[u] = ld_hint(C + (size_t)(j + u) * N + pt, pol3);
#pragma unroll
            for (int u = 0; u < 32; ++u) cfma(a, cv[u], s_y[j + u]);
        }
        for (; j + 16 <= je; j += 16) {
            cplx<TC> cv[16];
#pragma unroll
            for (int u = 0; u < 16; ++u) cv[u] = ld_hint(C + (size_t)(j + u) * N + pt, pol3);
#pragma unroll
            for (int u = 0; u < 16; ++u) cfma(a, cv[u], s_y[j + u]);
        }
        for (; j + 8 <= je; j += 8) {
            cplx<TC> cv[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) cv[u] = ld_hint(C + (size_t)(j + u) * N + pt, pol3);
#pragma unroll
            for (int u = 0; u < 8; ++u) cfma(a, cv[u], s_y[j + u]);
        }
        for (; j < je; ++j) cfma(a, ld_hint(C + (size_t)j * N + pt, pol3), s_y[j]);
        cplx<TO> val = cvt<TO>(a);
        if (J.add_w) val = val + cvt<TO>(w_in[pt]);
        if (J.dout) ((cplx<TC>*)J.dout)[pt - lo] = J.add_w ? a + cvt<TC>(w_in[pt]) : a;
        cplx<TO>& o = out[pt - lo];
        o = J.acc_out ? o + val : val;
        if (bt.rr.AC) {
            // the next residual r' - (A C) y; A C's columns of one child reach one row into
            // the other child's rows (the stencil), so both halves count next to the split
            const int jr = (int)(pt / (unsigned)g.Sx);
            int k0 = 0, k1 = p;
            if (J.split >= 0) {
                if (jr < J.split - 1) k1 = p >> 1;
                else if (jr > J.split) k0 = p >> 1;
            }
            const CA* AC = (const CA*)bt.rr.AC;
            CA rn = ((const CA*)bt.rr.rp)[pt];
            for (; k0 + 8 <= k1; k0 += 8) {
                CA av[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) av[u] = AC[(size_t)(k0 + u) * N + pt];
#pragma unroll
                for (int u = 0; u < 8; ++u) rn = rn - av[u] * s_y[k0 + u];
            }
            for (; k0 < k1; ++k0) rn = rn - AC[(size_t)k0 * N + pt] * s_y[k0];
            ((CA*)bt.rr.rt)[pt] = rn;
            rr2 += (float)abs2(rn);
        }
    }
    if (bt.rr.AC) coarse_recur_tail(bt.rr, rr2, lb, nblk);
}

template <typename TC, typename TV, typename TW, typename TO>
int coarse_batch_max_grid() {
    static std::atomic<int> mg[64];   // per device ordinal; 0 until queried
    const int dev = current_device();
    int g = mg[dev & 63].load(std::memory_order_relaxed);
    if (!g) {
        int sms = 0, nb = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_coarse_batch<TC, TV, TW, TO, false>, 256, 0);
        g = std::max(1, std::min(nb, 2) * sms);
        mg[dev & 63].store(g, std::memory_order_relaxed);
    }
    return g;
}

template <typename TC, typename TV, typename TW, typename TO>
void launch_coarse_batch(CoarseBatch bt, int p, void* partial, unsigned* bar, int* err, cudaStream_t s) {
    if (bt.njobs < 1) return;
    bt.wait_polls = wait_polls(1ll << 24);
    // blocks per job: one per 256 points, at most 152 per job (phase 2 reads every partial
    // of the job), within the co-resident total
    const int mg = coarse_batch_max_grid<TC, TV, TW, TO>();
    // jobs too large for the L2 (the basis streams from HBM) take every co-resident block:
    // there the launch is bound by memory parallelism, not by phase 2's reads
    size_t nmax = 0;
    for (int k = 0; k < bt.njobs; ++k) nmax = std::max(nmax, (size_t)bt.job[k].g.b * bt.job[k].g.Sx);
    const int per_job = nmax * (size_t)p * sizeof(cplx<TC>) > ((size_t)64 << 20) ? 1 << 30 : 152;
    const int cap = std::max(1, std::min(per_job, mg / bt.njobs));
    // each job's blocks shared out among its (half, column group) sets in proportion to
    // the points each set covers, at least one block per set
    const int ph = p / 2, G = (ph + CB_COLS - 1) / CB_COLS, nsets = 2 * G;
    unsigned blk = 0;
    for (int k = 0; k < bt.njobs; ++k) {
        CoarseJob& J = bt.job[k];
        const size_t N = (size_t)J.g.b * J.g.Sx;
        const size_t n0 = J.split < 0 ? N : std::min(N, (size_t)J.split * J.g.Sx);
        const size_t n1 = J.split < 0 ? N : N - n0;
        const int nb = std::max(nsets, blocks_for(N, 256, cap));
        const double tot = (double)G * (double)(n0 + n1);
        J.ngrp = G;
        J.sb[0] = 0;
        for (int st = 0; st < nsets; ++st) {
            const size_t pts = st < G ? n0 : n1;
            const int left = nsets - st - 1;
            int want = tot > 0 ? (int)std::lround(nb * (double)pts / tot) : 1;
            want = std::max(1, std::min(want, nb - (int)J.sb[st] - left));
            J.sb[st + 1] = J.sb[st] + (st == nsets - 1 ? std::max(1, nb - (int)J.sb[st]) : want);
        }
        J.blk0 = blk;
        J.nblk = J.sb[nsets];
        blk += J.nblk;
    }
    // bytes of basis one phase streams, against the L2
    {
        double bytes = 0.0;
        for (int k = 0; k < bt.njobs; ++k) {
            const CoarseJob& J = bt.job[k];
            bytes += (double)J.g.b * J.g.Sx * (J.split < 0 ? p : p / 2) * sizeof(cplx<TC>);
        }
        static std::atomic<long long> l2b[64];
        const int dev = current_device();
        long long l2 = l2b[dev & 63].load(std::memory_order_relaxed);
        if (!l2) {
            int v = 0;
            cudaDeviceGetAttribute(&v, cudaDevAttrL2CacheSize, dev);
            l2 = std::max(1, v);
            l2b[dev & 63].store(l2, std::memory_order_relaxed);
        }
        // the part of each sweep kept at normal priority: 0.8 of the L2's size (on the 1023^2
        // workload 0.5, 0.8 and 1.0 of it give the same launch time, about 5% shorter than
        // the reversed update order without priorities)
        bt.keep = bytes > (double)l2 ? (float)(0.8 * (double)l2 / bytes) : 1.f;
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
    if (bt.job[0].g.q1) cudaLaunchKernelEx(&cfg, k_coarse_batch<TC, TV, TW, TO, true>, bt, p, (cplx<TC>*)partial, bar, err);
    else cudaLaunchKernelEx(&cfg, k_coarse_batch<TC, TV, TW, TO, false>, bt, p, (cplx<TC>*)partial, bar, err);
    note_launch();
}


// Several columns (set-up): W[pt][c] += sum_j C[j][pt] y[j][c].  One thread per point
// and per chunk of UPD_COLS columns (chunk = blockIdx.y): each C[j][pt] is read once per
// chunk (coalesced along the points) and used for all the chunk's columns; y staged in
// shared memory in the basis precision.  The chunks in separate blocks keep several blocks
// per SM in flight (the loop over j waits on L2 loads).
// split_pt >= 0: the basis's first p/2 columns vanish from point split_pt on and the
// others before it (a node's two children), so each point reads only its child's half.
static constexpr int UPD_COLS = 16;
template <typename TC, typename TW>
__global__ void __launch_bounds__(256) k_coarse_updn(const cplx<TC>* __restrict__ C, const c128* __restrict__ y,
                                                     cplx<TW>* __restrict__ W, size_t N, int p, int nc,
                                                     long long split_pt) {
    extern __shared__ __align__(16) unsigned char ysm[];
    cplx<TC>* ys = (cplx<TC>*)ysm;   // [p][UPD_COLS]: this chunk's columns of y
    const int c0 = blockIdx.y * UPD_COLS, cn = min(UPD_COLS, nc - c0);
    for (int t = threadIdx.x; t < p * UPD_COLS; t += blockDim.x) {
        const int j = t / UPD_COLS, c = t - j * UPD_COLS;
        ys[t] = c < cn ? cvt<TC>(y[j * nc + c0 + c]) : cplx<TC>{0, 0};
    }
    __syncthreads();
    for (size_t pt = blockIdx.x * (size_t)blockDim.x + threadIdx.x; pt < N; pt += (size_t)gridDim.x * blockDim.x) {
        cplx<TC> acc[UPD_COLS];
#pragma unroll
        for (int c = 0; c < UPD_COLS; ++c) acc[c] = {0, 0};
        int j = 0, je = p;
        if (split_pt >= 0) {
            if ((long long)pt < split_pt) je = p / 2;
            else j = p / 2;
        }
        for (; j < je; ++j) {
            const cplx<TC> cv = C[(size_t)j * N + pt];
            const cplx<TC>* yr = ys + j * UPD_COLS;
#pragma unroll
            for (int c = 0; c < UPD_COLS; ++c) cfma(acc[c], cv, yr[c]);
        }
        cplx<TW>* wr = W + pt * nc + c0;
#pragma unroll
        for (int c = 0; c < UPD_COLS; ++c)
            if (c < cn) wr[c] = wr[c] + cvt<TW>(acc[c]);
    }
}
// The complex64 form of the same update with the basis staged and the output tile
// written whole: a block owns UPD_SP consecutive points (their rows of W are one contiguous
// span), one thread per point and chunk of 16 right-hand sides (up to four chunks at once);
// it stages the points' basis values, 32 columns at a time, with
// asynchronous 8-byte copies (the whole group in flight at once), runs every chunk of 16
// right-hand sides from shared memory into a shared output tile, and adds the tile to W
// with coalesced loads and stores.  (Per-thread row updates of W left partial sectors that
// the memory system wrote back several times over.)  A block whose points straddle the
// split stages both halves in turn (the vanishing half is stored as zeros).
static constexpr int UPD_SP = 64;
__global__ void __launch_bounds__(UPD_SP * 4) k_coarse_updn_s(const c64* __restrict__ C, const c128* __restrict__ y,
                                                              c64* __restrict__ W, size_t N, int p, int nc,
                                                              long long split_pt) {
    extern __shared__ __align__(16) unsigned char usm[];
    const int ncp = (nc + 15) / 16 * 16;        // right-hand sides padded to whole chunks
    c64* ys = (c64*)usm;                        // [p][ncp]
    c64* cs = ys + (size_t)p * ncp;             // [32][UPD_SP] one column group of the basis
    c64* ot = cs + 32 * UPD_SP;                 // [UPD_SP][ncp] the block's output tile
    const int t = threadIdx.x, nth = blockDim.x;
    const int pl = t % UPD_SP, ch = t / UPD_SP; // a thread's point and first chunk of 16
    for (int e = t; e < p * ncp; e += nth) {
        const int j = e / ncp, c = e - j * ncp;
        ys[e] = c < nc ? cvt<float>(y[j * nc + c]) : c64{0.f, 0.f};
    }
    for (size_t p0 = (size_t)blockIdx.x * UPD_SP; p0 < N; p0 += (size_t)gridDim.x * UPD_SP) {
        const int np = (int)min((size_t)UPD_SP, N - p0);
        const size_t plast = p0 + np - 1;
        int jlo = 0, jhi = p;
        if (split_pt >= 0) {
            if ((long long)plast < split_pt) jhi = p / 2;
            else if ((long long)p0 >= split_pt) jlo = p / 2;
        }
        __syncthreads();   // the previous span's tile is written out
        for (int e = t; e < UPD_SP * ncp; e += nth) ot[e] = {0.f, 0.f};
        for (int g0 = jlo; g0 < jhi; g0 += 32) {
            const int gn = min(32, jhi - g0);
            __syncthreads();   // the previous group's values are no longer read
            for (int e = t; e < gn * UPD_SP; e += nth) {
                const int j = e / UPD_SP, k = e - j * UPD_SP;
                const size_t x = p0 + k;
                cp_async8_zfill(cs + e, C + (size_t)(g0 + j) * N + (x < N ? x : 0), x < N);
            }
            cp_async_commit();
            cp_async_wait_all();
            __syncthreads();
            for (int c0 = 16 * ch; c0 < nc; c0 += 16 * (nth / UPD_SP)) {
                c64 acc[16];
#pragma unroll
                for (int c = 0; c < 16; ++c) acc[c] = {0.f, 0.f};
                for (int j = 0; j < gn; ++j) {
                    const c64 cv = cs[j * UPD_SP + pl];
                    const cpair<float>* yr = (const cpair<float>*)(ys + (size_t)(g0 + j) * ncp + c0);
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        const cpair<float> yy = yr[c];
                        cfma(acc[2 * c], cv, yy.x);
                        cfma(acc[2 * c + 1], cv, yy.y);
                    }
                }
                c64* orow = ot + (size_t)pl * ncp + c0;
#pragma unroll
                for (int c = 0; c < 16; ++c) orow[c] = orow[c] + acc[c];
            }
        }
        __syncthreads();
        // W's rows p0 .. p0 + np - 1 are one span of np nc values
        c64* wspan = W + p0 * nc;
        for (int e = t; e < np * nc; e += nth) {
            const int r = e / nc, c = e - r * nc;
            wspan[e] = wspan[e] + ot[(size_t)r * ncp + c];
        }
    }
}

template <typename TC, typename TW>
void launch_coarse_updn(const cplx<TC>* C, const c128* y, cplx<TW>* W, size_t N, int p, int nc, cudaStream_t s,
                        long long split_pt) {
    if constexpr (sizeof(TC) == 4 && sizeof(TW) == 4) {
        const int ncp = (nc + 15) / 16 * 16;
        const size_t sm = sizeof(c64) * ((size_t)p * ncp + 32 * UPD_SP + (size_t)UPD_SP * ncp);
        if (sm <= (size_t)(200 * 1024)) {
            static std::atomic<unsigned long long> attr{0};
            smem_limit_once(attr, k_coarse_updn_s, 200 * 1024);
            const int grid = blocks_for(N, UPD_SP, 152 * 16);
            // one group of UPD_SP threads per chunk of 16 right-hand sides (up to four), so
            // that every thread has the same number of chunks
            const int groups = std::min(4, ncp / 16);
            k_coarse_updn_s<<<grid, UPD_SP * groups, sm, s>>>(C, y, W, N, p, nc, split_pt);
            note_launch();
            return;
        }
    }
    const dim3 grid(blocks_for(N, 256, 152 * 8), (nc + UPD_COLS - 1) / UPD_COLS);
    k_coarse_updn<TC, TW><<<grid, 256, sizeof(cplx<TC>) * p * UPD_COLS, s>>>(C, y, W, N, p, nc, split_pt);
    note_launch();
}

template void launch_build_basis<float>(const c64*, size_t, int, c64*, size_t, int, size_t, size_t, cudaStream_t);
template void launch_build_basis<double>(const c128*, size_t, int, c128*, size_t, int, size_t, size_t, cudaStream_t);
template void launch_coarse_batch<float, float, float, float>(CoarseBatch, int, void*, unsigned*, int*, cudaStream_t);
template void launch_coarse_batch<float, float, float, double>(CoarseBatch, int, void*, unsigned*, int*, cudaStream_t);
template void launch_coarse_batch<float, double, double, double>(CoarseBatch, int, void*, unsigned*, int*,
                                                                 cudaStream_t);
template void launch_coarse_batch<double, double, double, double>(CoarseBatch, int, void*, unsigned*, int*,
                                                                  cudaStream_t);
template void launch_coarse_updn<float, float>(const c64*, const c128*, c64*, size_t, int, int, cudaStream_t, long long);
template void launch_coarse_updn<double, double>(const c128*, const c128*, c128*, size_t, int, int, cudaStream_t, long long);

}  // namespace hh
