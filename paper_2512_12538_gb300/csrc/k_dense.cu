// k_dense.cu -- small dense steps of the set-up and the coarse solve:
//  * tall-skinny inner products A^H B in FP64 (coarse projection C^H r of Eq. (3), the
//    Gram matrix of the sketch);
//  * the Galerkin product A_c = C^H A~ C (Sec. 1) fused with the 5-point operator;
//  * orthonormalisation of the sketch Y = T Omega (Sec. 2, randomised SVD);
//  * the small SVD: Hermitian eigenproblem of Z^H Z in FP64 (tridiagonal reduction,
//    bisection, inverse iteration) and V = Z U Sigma^{-1};
//  * Gauss-Jordan inversion with partial pivoting of A_c (FP64).
#include <cooperative_groups.h>

#include "kernels.h"

namespace hh {

static constexpr int IP_TILE = 32;
static constexpr int IP_THREADS = 256;
static constexpr int IP_MAXOUT = 16;   // outputs per thread when p*q >= IP_THREADS
static constexpr int GAL_FLUSH = 4;     // Galerkin tiles summed in FP32 before the FP64 add

// Accumulate conj(As[n][i]) * Bs[n][j] over a tile of `rows` rows held in shared memory.
// Rows i outside [ilo, ihi) contribute nothing for this tile (ihi = 0: no restriction).
template <typename ACC, int KMAX = IP_MAXOUT>
__device__ __forceinline__ void ip_tile_accumulate(const cplx<ACC>* As, const cplx<ACC>* Bs, int rows, int p, int q,
                                                   int split, cplx<ACC>* acc, int ilo, int ihi, int jlo = 0,
                                                   int jhi = 0) {
    const int nout = p * q;
    if (split == 1) {
        // output o = threadIdx.x + k IP_THREADS; k is a compile-time index, so acc stays
        // in registers.  Columns j outside [jlo, jhi) contribute nothing for this tile
        // (jhi = 0: no restriction); with q a multiple of 32 the skipped ones are whole warps
#pragma unroll
        for (int k = 0; k < KMAX; ++k) {
            const int o = threadIdx.x + k * IP_THREADS;
            if (o >= nout) continue;
            const int i = o / q, j = o % q;
            if (ihi > 0 && (i < ilo || i >= ihi)) continue;
            if (jhi > 0 && (j < jlo || j >= jhi)) continue;
            cplx<ACC> a = acc[k];
            for (int n = 0; n < rows; ++n) cfma_cj(a, As[n * p + i], Bs[n * q + j]);
            acc[k] = a;
        }
    } else {
        const int s = threadIdx.x / nout, o = threadIdx.x % nout;
        if (s < split) {
            const int i = o / q, j = o % q;
            if (ihi > 0 && (i < ilo || i >= ihi)) return;
            if (jhi > 0 && (j < jlo || j >= jhi)) return;
            cplx<ACC> a = acc[0];
            for (int n = s; n < rows; n += split) cfma_cj(a, As[n * p + i], Bs[n * q + j]);
            acc[0] = a;
        }
    }
}

template <typename ACC, int KMAX = IP_MAXOUT>
__device__ __forceinline__ void ip_store_partial(cplx<ACC>* acc, int p, int q, int split, cplx<ACC>* red,
                                                 c128* out) {
    const int nout = p * q;
    if (split == 1) {
#pragma unroll
        for (int k = 0; k < KMAX; ++k) {
            const int o = threadIdx.x + k * IP_THREADS;
            if (o < nout) out[o] = cvt<double>(acc[k]);
        }
    } else {
        const int s = threadIdx.x / nout, o = threadIdx.x % nout;
        if (s < split) red[s * nout + o] = acc[0];
        __syncthreads();
        for (int o2 = threadIdx.x; o2 < nout; o2 += IP_THREADS) {
            c128 t = {0.0, 0.0};
            for (int s2 = 0; s2 < split; ++s2) t = t + cvt<double>(red[s2 * nout + o2]);
            out[o2] = t;
        }
    }
}

// ACOL: A column-major (column i at A + i lda), staged along the points (coalesced).
// split_pt >= 0 (ACOL, a node's coarse basis): A's columns [0, p/2) vanish at points
// >= split_pt and [p/2, p) below it, so a tile on one side skips the other half.
template <typename TA, typename TB, typename ACC, bool ACOL>
__global__ void __launch_bounds__(IP_THREADS) k_ip_partial(const cplx<TA>* __restrict__ A, size_t lda,
                                                           const cplx<TB>* __restrict__ B, int ldb,
                                                           size_t N, int p, int q, c128* partial,
                                                           long long split_pt = -1) {
    extern __shared__ __align__(16) unsigned char ipsm[];
    using CA = cplx<ACC>;
    CA* As = (CA*)ipsm;
    CA* Bs = As + IP_TILE * p;
    CA* red = Bs + IP_TILE * q;
    const int nout = p * q;
    const int split = nout >= IP_THREADS ? 1 : IP_THREADS / nout;
    CA acc[IP_MAXOUT];
    for (int k = 0; k < IP_MAXOUT; ++k) acc[k] = {0, 0};
    const size_t chunk = (N + gridDim.x - 1) / gridDim.x;
    const size_t n0 = blockIdx.x * chunk, n1 = min(N, n0 + chunk);
    for (size_t t0 = n0; t0 < n1; t0 += IP_TILE) {
        const int rows = (int)min((size_t)IP_TILE, n1 - t0);
        // columns of A that can be nonzero on this tile: [ilo, ihi) (ihi = 0: all)
        int ilo = 0, ihi = 0, c_lo = 0, c_n = p;
        if (ACOL && split_pt >= 0) {
            if ((long long)(t0 + rows) <= split_pt) { ihi = p / 2; c_n = p / 2; }
            else if ((long long)t0 >= split_pt) { ilo = p / 2; ihi = p; c_lo = p / 2; c_n = p - p / 2; }
        }
        {
            // 8 loads in flight per thread before the shared-memory stores; a column-major
            // A is read along the points (element e: column c_lo + e / rows, point e % rows)
            const int na = rows * c_n, nbq = rows * q;
            for (int base = threadIdx.x; base < na + nbq; base += 8 * IP_THREADS) {
                cplx<ACC> tmp[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int e = base + u * IP_THREADS;
                    if (e < na) tmp[u] = ACOL ? cvt<ACC>(A[(size_t)(c_lo + e / rows) * lda + t0 + e % rows])
                                              : cvt<ACC>(A[(t0 + e / p) * lda + e % p]);
                    else if (e < na + nbq) { const int e2 = e - na; tmp[u] = cvt<ACC>(B[(t0 + e2 / q) * ldb + e2 % q]); }
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int e = base + u * IP_THREADS;
                    if (e < na) {
                        if (ACOL) As[(e % rows) * p + c_lo + e / rows] = tmp[u];
                        else As[e] = tmp[u];
                    } else if (e < na + nbq) Bs[e - na] = tmp[u];
                }
            }
        }
        __syncthreads();
        ip_tile_accumulate<ACC>(As, Bs, rows, p, q, split, acc, ilo, ihi);
        __syncthreads();
    }
    ip_store_partial<ACC>(acc, p, q, split, red, partial + (size_t)blockIdx.x * nout);
}

// Skinny products (p * q <= 64): each lane owns at most two outputs; warps stride over
// rows with several rows in flight; the block's warps are combined in shared memory.
template <typename TA, typename TB, typename ACC>
__global__ void __launch_bounds__(256) k_ip_skinny(const cplx<TA>* __restrict__ A, int lda,
                                                   const cplx<TB>* __restrict__ B, int ldb, size_t N, int p,
                                                   int q, c128* partial) {
    using CA = cplx<ACC>;
    __shared__ CA red[8][64];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nout = p * q;
    const int o0 = lane, o1 = lane + 32;
    const int i0 = o0 / q, j0 = o0 - (o0 / q) * q;
    const int i1 = o1 / q, j1 = o1 - (o1 / q) * q;
    const bool h0 = o0 < nout, h1 = o1 < nout;
    CA a0 = {0, 0}, a1 = {0, 0};
    const size_t gw = (size_t)gridDim.x * 8;
    size_t n = (size_t)blockIdx.x * 8 + warp;
    constexpr int U = 4;
    for (; n + (U - 1) * gw < N; n += U * gw) {
        CA x0[U], y0[U], x1[U], y1[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const size_t r = n + u * gw;
            if (h0) { x0[u] = cvt<ACC>(A[r * lda + i0]); y0[u] = cvt<ACC>(B[r * ldb + j0]); }
            if (h1) { x1[u] = cvt<ACC>(A[r * lda + i1]); y1[u] = cvt<ACC>(B[r * ldb + j1]); }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (h0) cfma_cj(a0, x0[u], y0[u]);
            if (h1) cfma_cj(a1, x1[u], y1[u]);
        }
    }
    for (; n < N; n += gw) {
        if (h0) cfma_cj(a0, cvt<ACC>(A[n * lda + i0]), cvt<ACC>(B[n * ldb + j0]));
        if (h1) cfma_cj(a1, cvt<ACC>(A[n * lda + i1]), cvt<ACC>(B[n * ldb + j1]));
    }
    red[warp][o0] = a0;
    red[warp][o1] = a1;
    __syncthreads();
    for (int o = threadIdx.x; o < nout; o += blockDim.x) {
        c128 t = {0.0, 0.0};
        for (int w = 0; w < 8; ++w) t = t + cvt<double>(red[w][o]);
        partial[(size_t)blockIdx.x * nout + o] = t;
    }
}

static size_t ip_smem(int p, int q, size_t esz = sizeof(c128)) {
    const int nout = p * q;
    const int split = nout >= IP_THREADS ? 1 : IP_THREADS / nout;
    return esz * ((size_t)IP_TILE * (p + q) + (split > 1 ? (size_t)split * nout : 0));
}

template <typename TA, typename TB, typename ACC>
int launch_ip_partial(const cplx<TA>* A, int lda, const cplx<TB>* B, int ldb, size_t N, int p, int q,
                      c128* partial, int max_blocks, cudaStream_t s) {
    if (p * q <= 64) {
        int grid = (int)((N + 63) / 64);
        if (grid > max_blocks) grid = max_blocks;
        if (grid < 1) grid = 1;
        k_ip_skinny<TA, TB, ACC><<<grid, 256, 0, s>>>(A, lda, B, ldb, N, p, q, partial);
        note_launch();
        return grid;
    }
    // one block per IP_TILE rows up to one per SM: the outputs are many and the rows few
    // (Gram matrices of sketch blocks), so the work per row is what needs spreading
    int grid = (int)((N + IP_TILE - 1) / IP_TILE);
    if (grid > 152) grid = 152;
    if (grid > max_blocks) grid = max_blocks;
    if (grid < 1) grid = 1;
    const size_t sm = ip_smem(p, q, sizeof(cplx<ACC>));
    static std::atomic<unsigned long long> attr{0};   // per instantiation
    smem_limit_once(attr, k_ip_partial<TA, TB, ACC, false>, 200 * 1024);
    k_ip_partial<TA, TB, ACC, false><<<grid, IP_THREADS, sm, s>>>(A, lda, B, ldb, N, p, q, partial);
    note_launch();
    return grid;
}

// The complex64 form for a node's basis (the set-up's multi-column projections), as dense
// products: rows [ilo, ilo + ni) of A (the columns that can be nonzero on the points
// [pa, pb)) against all q columns of B.  Register-tiled: a thread owns 4 x 4 outputs and a
// share (KG groups) of each 32-point tile's points; per point it reads 4 values of A and 4
// of B from shared memory for 16 complex multiply-adds.  The tiles are double-buffered
// with cp.async (8-byte copies, zero-filled past the range).  The groups' sums are added in
// shared memory, and the block writes its whole [p][q] partial (zeros outside the rows).
static constexpr int RT_TP = 32;
// The two halves of a node's basis share one launch: blocks [0, nb0) take rows [ilo0, ilo0 +
// ni) on the points [pa0, pb0), the others rows [ilo1, ilo1 + ni) on [pa1, pb1).
template <int KG>
__global__ void __launch_bounds__(256) k_ip_colA_rt(const c64* __restrict__ A, size_t lda, const c64* __restrict__ B,
                                                    int ldb, int p, int q, int ni, int nb0, int ilo0, size_t pa0,
                                                    size_t pb0, int ilo1, size_t pa1, size_t pb1, c128* partial) {
    const bool second = (int)blockIdx.x >= nb0;
    const int ilo = second ? ilo1 : ilo0;
    const size_t pa = second ? pa1 : pa0, pb = second ? pb1 : pb0;
    const unsigned blk = second ? blockIdx.x - nb0 : blockIdx.x;
    const unsigned nblk = second ? gridDim.x - nb0 : nb0;
    extern __shared__ __align__(16) unsigned char rtsm[];
    const int IT = (ni + 3) / 4, CT = (q + 3) / 4, nt = IT * CT;
    const int nr = 4 * IT, qp = 4 * CT;          // padded tile rows and columns
    c64* As = (c64*)rtsm;                        // [2][nr][RT_TP]
    c64* Bs = As + 2 * nr * RT_TP;               // [2][RT_TP][qp]
    const int tid = threadIdx.x;
    const int o = tid % nt, kg = tid / nt;
    const int it = o / CT, ct = o - it * CT;
    // this block's points: whole tiles of the range
    const size_t ntiles_all = (pb - pa + RT_TP - 1) / RT_TP;
    const size_t t0b = ntiles_all * blk / nblk, t1b = ntiles_all * (blk + 1) / nblk;
    // padding rows / columns stay zero
    for (int e = tid; e < 2 * nr * RT_TP; e += blockDim.x) As[e] = {0.f, 0.f};
    for (int e = tid; e < 2 * RT_TP * qp; e += blockDim.x) Bs[e] = {0.f, 0.f};
    __syncthreads();
    auto stage = [&](size_t tile, int buf) {
        const size_t x0 = pa + tile * RT_TP;
        c64* as = As + (size_t)buf * nr * RT_TP;
        c64* bs = Bs + (size_t)buf * RT_TP * qp;
        for (int e = tid; e < ni * RT_TP; e += blockDim.x) {
            const int i = e / RT_TP, k = e - i * RT_TP;
            const size_t x = x0 + k;
            const bool ok = x < pb;
            cp_async8_zfill(as + i * RT_TP + k, A + (size_t)(ilo + i) * lda + (ok ? x : pa), ok);
        }
        for (int e = tid; e < RT_TP * q; e += blockDim.x) {
            const int k = e / q, c = e - k * q;
            const size_t x = x0 + k;
            const bool ok = x < pb;
            cp_async8_zfill(bs + k * qp + c, B + (ok ? x : pa) * ldb + c, ok);
        }
        cp_async_commit();
    };
    c64 acc[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = {0.f, 0.f};
    if (t0b < t1b) stage(t0b, 0);
    for (size_t tile = t0b; tile < t1b; ++tile) {
        const int buf = (int)((tile - t0b) & 1);
        if (tile + 1 < t1b) {
            stage(tile + 1, buf ^ 1);
            cp_async_wait_group1();
        } else {
            cp_async_wait_all();
        }
        __syncthreads();
        if (kg < KG) {
            const c64* as = As + (size_t)buf * nr * RT_TP + (size_t)(4 * it) * RT_TP;
            const c64* bs = Bs + (size_t)buf * RT_TP * qp + 4 * ct;
            for (int k = kg; k < RT_TP; k += KG) {
                c64 a[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) a[u] = as[u * RT_TP + k];
                const cpair<float> b01 = *(const cpair<float>*)(bs + k * qp);
                const cpair<float> b23 = *(const cpair<float>*)(bs + k * qp + 2);
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    cfma_cj(acc[u][0], a[u], b01.x);
                    cfma_cj(acc[u][1], a[u], b01.y);
                    cfma_cj(acc[u][2], a[u], b23.x);
                    cfma_cj(acc[u][3], a[u], b23.y);
                }
            }
        }
        __syncthreads();
    }
    // the groups' sums (the tile buffers are free now), then the block's [p][q] partial
    c64* red = As;                               // [KG][nt][16]
    if (kg < KG)
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) red[((size_t)kg * nt + o) * 16 + u * 4 + v] = acc[u][v];
    __syncthreads();
    c128* out = partial + (size_t)blockIdx.x * p * q;
    for (int e = tid; e < p * q; e += blockDim.x) {
        const int i = e / q, c = e - i * q;
        c128 t = {0.0, 0.0};
        const int ir = i - ilo;
        if (ir >= 0 && ir < ni) {
            const int oo = (ir >> 2) * CT + (c >> 2), uv = (ir & 3) * 4 + (c & 3);
            for (int g = 0; g < KG; ++g) t = t + cvt<double>(red[((size_t)g * nt + oo) * 16 + uv]);
        }
        out[e] = t;
    }
}

// nb0 blocks for the first set, nb1 for the second (nb1 = 0: one set)
static int ip_colA_rt_launch(const c64* A, size_t lda, const c64* B, int ldb, int p, int q, int ni, int nb0,
                             int ilo0, size_t pa0, size_t pb0, int nb1, int ilo1, size_t pa1, size_t pb1,
                             c128* partial, cudaStream_t s) {
    const int IT = (ni + 3) / 4, CT = (q + 3) / 4, nt = IT * CT;
    const int kg = std::max(1, std::min(4, 256 / nt));
    const size_t sm = sizeof(c64) * std::max<size_t>((size_t)2 * (4 * IT * RT_TP + RT_TP * 4 * CT),
                                                     (size_t)kg * nt * 16);
    const int threads = nt * kg, nblk = nb0 + nb1;
#define HH_COLA_ARGS A, lda, B, ldb, p, q, ni, nb0, ilo0, pa0, pb0, ilo1, pa1, pb1, partial
    switch (kg) {
        case 1: k_ip_colA_rt<1><<<nblk, threads, sm, s>>>(HH_COLA_ARGS); break;
        case 2: k_ip_colA_rt<2><<<nblk, threads, sm, s>>>(HH_COLA_ARGS); break;
        case 3: k_ip_colA_rt<3><<<nblk, threads, sm, s>>>(HH_COLA_ARGS); break;
        default: k_ip_colA_rt<4><<<nblk, threads, sm, s>>>(HH_COLA_ARGS); break;
    }
#undef HH_COLA_ARGS
    note_launch();
    return nblk;
}

// partial[blk][i][j] = sum conj(A[i * N + n]) B[n * ldb + j] with A column-major (p x N).
template <typename TA, typename TB, typename ACC>
int launch_ip_partial_colA(const cplx<TA>* A, const cplx<TB>* B, int ldb, size_t N, int p, int q, c128* partial,
                           int max_blocks, cudaStream_t s, long long split_pt) {
    if constexpr (sizeof(TA) == 4 && sizeof(TB) == 4 && sizeof(ACC) == 4) {
        // complex64, at most 64 columns of B (the 4 x 4 tiles of a block fit 256 threads)
        const int half = p / 2;
        if (q <= 64 && p <= 64 && N > 0) {
            const size_t sp = split_pt < 0 ? 0 : std::min<size_t>((size_t)split_pt, N);
            if (split_pt < 0 || half == 0 || sp == 0 || sp == N) {
                // one set: every row on every point
                const int nb = std::max(1, std::min(max_blocks, (int)((N + 255) / 256)));
                return ip_colA_rt_launch((const c64*)A, N, (const c64*)B, ldb, p, q, p, nb, 0, 0, N, 0, 0, 0, 0,
                                         partial, s);
            }
            // the two halves of the basis on their own points, in one launch, blocks in
            // proportion to the points
            int nb1 = std::max(1, (int)std::lround((double)max_blocks * sp / N));
            const int nb2 = std::max(1, max_blocks - nb1);
            if (nb1 + nb2 > max_blocks) nb1 = max_blocks - nb2;
            return ip_colA_rt_launch((const c64*)A, N, (const c64*)B, ldb, p, q, half, nb1, 0, 0, sp, nb2, half, sp,
                                     N, partial, s);
        }
    }
    int grid = (int)((N + 255) / 256);
    if (grid > max_blocks) grid = max_blocks;
    if (grid < 1) grid = 1;
    const size_t sm = ip_smem(p, q, sizeof(cplx<ACC>));
    static std::atomic<unsigned long long> attr{0};
    smem_limit_once(attr, k_ip_partial<TA, TB, ACC, true>, 200 * 1024);
    k_ip_partial<TA, TB, ACC, true><<<grid, IP_THREADS, sm, s>>>(A, N, B, ldb, N, p, q, partial, split_pt);
    note_launch();
    return grid;
}

// out = sum over blocks (one warp per output, lanes across blocks: fixed order, so
// deterministic); optional out2 = Minv * out computed by the same (single) block.
__global__ void __launch_bounds__(1024) k_ip_reduce(const c128* __restrict__ partial, int nblk, int p, int q,
                                                    c128* out, const c128* __restrict__ Minv, c128* out2) {
    extern __shared__ c128 s_out[];          // [nout] sums, then [p*p] Minv when present
    const int nout = p * q;
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    c128* s_m = s_out + nout;
    if (Minv)
        for (int t = threadIdx.x; t < p * p; t += blockDim.x) s_m[t] = Minv[t];
    for (int o = blockIdx.x * nw + (threadIdx.x >> 5); o < nout; o += gridDim.x * nw) {
        c128 t0 = {0.0, 0.0}, t1 = {0.0, 0.0}, t2 = {0.0, 0.0}, t3 = {0.0, 0.0};
        int b = lane;
        for (; b + 96 < nblk; b += 128) {
            t0 = t0 + partial[(size_t)b * nout + o];
            t1 = t1 + partial[(size_t)(b + 32) * nout + o];
            t2 = t2 + partial[(size_t)(b + 64) * nout + o];
            t3 = t3 + partial[(size_t)(b + 96) * nout + o];
        }
        for (; b < nblk; b += 32) t0 = t0 + partial[(size_t)b * nout + o];
        c128 t = (t0 + t1) + (t2 + t3);
        t = warp_sum(t);
        if (lane == 0) {
            if (Minv) s_out[o] = t;
            if (out) out[o] = t;
        }
    }
    if (!Minv) return;
    __syncthreads();
    for (int o = threadIdx.x; o < nout; o += blockDim.x) {
        const int i = o / q, j = o % q;
        c128 t = {0.0, 0.0};
        for (int k = 0; k < p; ++k) cfma(t, s_m[i * p + k], s_out[k * q + j]);
        out2[o] = t;
    }
}
// y = M x for a p x p matrix and a p x q block.  Eight threads per output, each adding
// every eighth term, then a fixed shuffle tree: the FP64 products spread over eight
// times the SMs of one thread per output.
__global__ void k_small_matmul(const c128* __restrict__ M, const c128* __restrict__ x, int p, int q, c128* y) {
    const int o = (blockIdx.x * blockDim.x + threadIdx.x) >> 3, sub = threadIdx.x & 7;
    const bool ok = o < p * q;
    c128 t = {0.0, 0.0};
    if (ok) {
        const int i = o / q, j = o - (o / q) * q;
        for (int k = sub; k < p; k += 8) cfma(t, M[i * p + k], x[k * q + j]);
    }
    for (int d = 4; d > 0; d >>= 1) {
        t.re += __shfl_xor_sync(0xffffffffu, t.re, d);
        t.im += __shfl_xor_sync(0xffffffffu, t.im, d);
    }
    if (ok && sub == 0) y[o] = t;
}

void launch_ip_reduce(const c128* partial, int nblk, int p, int q, c128* out, const c128* Minv, c128* out2,
                      cudaStream_t s) {
    static std::atomic<unsigned long long> attr{0};
    smem_limit_once(attr, k_ip_reduce, 200 * 1024);
    const int nout = p * q;
    if (Minv && nout > 64) {
        // many outputs: reduce over blocks with the whole GPU, then apply Minv separately
        // the sums go just past the partials (the scratch holds nblk * nout + nout values)
        c128* sums = const_cast<c128*>(partial) + (size_t)nblk * nout;
        int grid = (nout + 7) / 8;
        if (grid > 304) grid = 304;
        k_ip_reduce<<<grid, 256, 0, s>>>(partial, nblk, p, q, sums, nullptr, nullptr);
        note_launch();
        k_small_matmul<<<(8 * nout + 255) / 256, 256, 0, s>>>(Minv, sums, p, q, out2);
        note_launch();
        if (out) cudaMemcpyAsync(out, sums, sizeof(c128) * nout, cudaMemcpyDeviceToDevice, s);
        return;
    }
    if (Minv) {
        k_ip_reduce<<<1, 1024, sizeof(c128) * (nout + (size_t)p * p), s>>>(partial, nblk, p, q, out, Minv, out2);
    } else {
        int grid = (nout + 7) / 8;
        if (grid > 304) grid = 304;
        k_ip_reduce<<<grid, 256, 0, s>>>(partial, nblk, p, q, out, nullptr, nullptr);
    }
    note_launch();
}

// ------------------------------------------------------------------- Galerkin
// Points of block `blk` of `nblk` in a Galerkin launch over N = b Sx points, shared out by
// cost: with a split row the two rows next to it (split - 1 and split) need every column of
// A~ C against one half of conj(C), twice a point's work elsewhere, so they count twice.
// An even split of the points left the blocks on those rows with twice the mean work.
__device__ __forceinline__ void gal_range(size_t N, int Sx, int split_row, unsigned blk, unsigned nblk,
                                          size_t& n0, size_t& n1) {
    size_t s0 = 0, s1 = 0;   // the rows of double cost: [s0, s1)
    if (split_row >= 0) {
        s0 = min(N, (size_t)max(split_row - 1, 0) * Sx);
        s1 = min(N, (size_t)(split_row + 1) * Sx);
    }
    const size_t T = N + (s1 - s0);
    auto inv = [&](size_t c) -> size_t {   // the point at cost c (monotone in c)
        if (c <= s0) return c;
        if (c <= s0 + 2 * (s1 - s0)) return s0 + (c - s0) / 2;
        return c - (s1 - s0);
    };
    n0 = inv(T * blk / nblk);
    n1 = blk + 1 == nblk ? N : inv(T * (blk + 1) / nblk);
}

// partial[blk][a][l] = sum over the block's points of conj(C[pt][a]) * (A~ C)[pt][l].
// C is stored in TI (complex64 in the mixed form); the stencil and the products run in
// T.  T = double: FP64 arithmetic on the basis values (a complex64 basis widens exactly),
// so A_c = C^H A~ C is the FP64 Galerkin matrix of the stored basis.  T = float (the
// opt-in FP32 coarse variant of the mixed form): the products of GAL_FLUSH 32-point
// tiles are summed in FP32, then added to FP64 accumulators, so the FP32 rounding stays
// at the level of 128 points' sum (only the outputs a thread owns are flushed; FP64 on
// this GPU runs at 1/64 of the FP32 rate).
template <typename TI, typename T, int KMAX>
__global__ void __launch_bounds__(IP_THREADS) k_galerkin_partial(const cplx<TI>* __restrict__ C, OpGeom g, int p,
                                                                 int split_row, c128* partial) {
    using CT = cplx<T>;
    extern __shared__ __align__(16) unsigned char gsm_[];
    CT* As = (CT*)gsm_;
    CT* Bs = As + IP_TILE * p;
    c128* red = (c128*)(Bs + IP_TILE * p);
    const int nout = p * p;
    const int split = nout >= IP_THREADS ? 1 : IP_THREADS / nout;
    c128 acc[KMAX];
    for (int k = 0; k < KMAX; ++k) acc[k] = {0.0, 0.0};
    CT tacc[KMAX];
    for (int k = 0; k < KMAX; ++k) tacc[k] = {0, 0};
    const int nk = split > 1 ? 1 : (nout + IP_THREADS - 1) / IP_THREADS;   // outputs owned
    int ntile = 0;
    const size_t N = (size_t)g.b * g.Sx;
    size_t n0, n1;
    gal_range(N, g.Sx, split_row, blockIdx.x, gridDim.x, n0, n1);
    for (size_t t0 = n0; t0 < n1; t0 += IP_TILE) {
        const int rows = (int)min((size_t)IP_TILE, n1 - t0);
        // C's columns [0, p/2) live on rows < split_row, [p/2, p) on the others, and A~ C
        // reaches one row further (the stencil).  A tile inside one row range needs one half
        // of conj(C) (rows i of A_c: [ilo, ihi)) and, away from the rows next to the split,
        // one half of A~ C (columns l: [jlo, jhi)); 0 as the upper end: every column.
        int ilo = 0, ihi = 0, jlo = 0, jhi = 0;
        if (split_row >= 0) {
            const int j0 = (int)(t0 / g.Sx), j1 = (int)((t0 + rows - 1) / g.Sx);
            if (j1 < split_row) { ilo = 0; ihi = p / 2; }
            else if (j0 >= split_row) { ilo = p / 2; ihi = p; }
            if (j1 < split_row - 1) { jlo = 0; jhi = p / 2; }
            else if (j0 > split_row) { jlo = p / 2; jhi = p; }
        }
        for (int e = threadIdx.x; e < rows * p; e += IP_THREADS) {
            const size_t pt = t0 + e / p;
            const int l = e % p;
            const bool need_a = ihi == 0 || (l >= ilo && l < ihi);
            const bool need_b = jhi == 0 || (l >= jlo && l < jhi);
            if (!need_a && !need_b) continue;
            const int i = (int)(pt % g.Sx), j = (int)(pt / g.Sx);
            const size_t t = (size_t)l * N + pt;          // column-major basis
            const CT cv = cvt<T>(C[t]);
            CT ax;
            if (g.q1) {
                ax = q1_row<T>(j, i, g, [&](int dj, int di) {
                    return cvt<T>(C[(size_t)((long long)t + (long long)dj * g.Sx + di)]);
                });
            } else {
                ax = op_diag_t<T>(j, i, g) * cv;
                const T wj = (j == 0 || j == g.b - 1) ? (T)0.5 : (T)1;
                const T wi = g.Sx == 1 ? (T)1 : ((i == 0 || i == g.Sx - 1) ? (T)0.5 : (T)1);
                if (g.Sx > 1) {
                    if (i > 0) ax = ax - wj * cvt<T>(C[t - 1]);
                    if (i < g.Sx - 1) ax = ax - wj * cvt<T>(C[t + 1]);
                }
                if (j > 0) ax = ax - wi * cvt<T>(C[t - g.Sx]);
                if (j < g.b - 1) ax = ax - wi * cvt<T>(C[t + g.Sx]);
            }
            As[e] = cv;
            Bs[e] = ax;
        }
        __syncthreads();
        if (sizeof(T) == sizeof(double)) {
            ip_tile_accumulate<double, KMAX>((const c128*)As, (const c128*)Bs, rows, p, p, split, acc, ilo, ihi, jlo,
                                             jhi);
        } else {
            ip_tile_accumulate<T, KMAX>(As, Bs, rows, p, p, split, tacc, ilo, ihi, jlo, jhi);
            if (++ntile == GAL_FLUSH || t0 + IP_TILE >= n1) {
#pragma unroll
                for (int k = 0; k < KMAX; ++k)
                    if (k < nk) {
                        acc[k] = acc[k] + cvt<double>(tacc[k]);
                        tacc[k] = {0, 0};
                    }
                ntile = 0;
            }
        }
        __syncthreads();
    }
    ip_store_partial<double, KMAX>(acc, p, p, split, red, partial + (size_t)blockIdx.x * nout);
}

// The FP64 form of the same partial sums with three real products per complex product
// (the 3M method: Higham, "Accuracy and Stability of Numerical Algorithms", 2nd ed.,
// Sec. 23.2.4).  For conj(a) b, with the staged sums a- = ar - ai, b- = bi - br and
// b+ = br + bi,
//   Re = br a- + ai b+,   Im = br a- + ar b-,
// so a thread accumulates S1 = sum br a-, S2 = sum ar b-, S3 = sum ai b+ and forms
// (S1 + S3, S1 + S2) at the end: 3 FP64 multiply-adds per product instead of 4, the
// additions done once per staged element.  Each staged value is one FP64 rounding of an
// exact sum (a complex64 basis widens exactly), so the error stays at FP64 level,
// bounded like the 4-product form's by a few ulps of (|ar| + |ai|)(|br| + |bi|).
// Block of G3_THREADS threads (one per SM: the three sums of KMAX outputs a thread fit the
// registers of one such block), each thread owning KMAX whole outputs (p * p >= G3_THREADS).
static constexpr int G3_THREADS = 512;
template <typename TI, int KMAX>
__global__ void __launch_bounds__(G3_THREADS, 1) k_galerkin_partial3(const cplx<TI>* __restrict__ C, OpGeom g, int p,
                                                                     int split_row, c128* partial) {
    extern __shared__ __align__(16) unsigned char gsm_[];
    double* As = (double*)gsm_;                      // [IP_TILE][p] x {ar, ai, ar - ai}
    double* Bs = As + 3 * (size_t)IP_TILE * p;       // [IP_TILE][p] x {br, bi - br, br + bi}
    const int nout = p * p;
    double s1[KMAX], s2[KMAX], s3[KMAX];
#pragma unroll
    for (int k = 0; k < KMAX; ++k) s1[k] = s2[k] = s3[k] = 0.0;
    const size_t N = (size_t)g.b * g.Sx;
    size_t n0, n1;
    gal_range(N, g.Sx, split_row, blockIdx.x, gridDim.x, n0, n1);
    for (size_t t0 = n0; t0 < n1; t0 += IP_TILE) {
        const int rows = (int)min((size_t)IP_TILE, n1 - t0);
        // the half-block skipping of k_galerkin_partial
        int ilo = 0, ihi = 0, jlo = 0, jhi = 0;
        if (split_row >= 0) {
            const int j0 = (int)(t0 / g.Sx), j1 = (int)((t0 + rows - 1) / g.Sx);
            if (j1 < split_row) { ilo = 0; ihi = p / 2; }
            else if (j0 >= split_row) { ilo = p / 2; ihi = p; }
            if (j1 < split_row - 1) { jlo = 0; jhi = p / 2; }
            else if (j0 > split_row) { jlo = p / 2; jhi = p; }
        }
        for (int e = threadIdx.x; e < rows * p; e += G3_THREADS) {
            const size_t pt = t0 + e / p;
            const int l = e % p;
            const bool need_a = ihi == 0 || (l >= ilo && l < ihi);
            const bool need_b = jhi == 0 || (l >= jlo && l < jhi);
            if (!need_a && !need_b) continue;
            const int i = (int)(pt % g.Sx), j = (int)(pt / g.Sx);
            const size_t t = (size_t)l * N + pt;          // column-major basis
            const c128 cv = cvt<double>(C[t]);
            c128 ax;
            if (g.q1) {
                ax = q1_row<double>(j, i, g, [&](int dj, int di) {
                    return cvt<double>(C[(size_t)((long long)t + (long long)dj * g.Sx + di)]);
                });
            } else if (g.Sx > 1 && i > 0 && i < g.Sx - 1 && j > 0 && j < g.b - 1) {
                // interior row: unit weights, no impedance term, real diagonal 4 - (kh)^2
                const double kr = g.khr ? g.khr[j] : g.kh;
                const double d = 4.0 - kr * kr;
                const c128 n1 = cvt<double>(C[t - 1]), n2 = cvt<double>(C[t + 1]);
                const c128 n3 = cvt<double>(C[t - g.Sx]), n4 = cvt<double>(C[t + g.Sx]);
                ax.re = d * cv.re - n1.re - n2.re - n3.re - n4.re;
                ax.im = d * cv.im - n1.im - n2.im - n3.im - n4.im;
            } else {
                ax = op_diag(j, i, g) * cv;
                const double wj = wrow(j, g.b), wi = wcol(i, g.Sx);
                if (g.Sx > 1) {
                    if (i > 0) ax = ax - wj * cvt<double>(C[t - 1]);
                    if (i < g.Sx - 1) ax = ax - wj * cvt<double>(C[t + 1]);
                }
                if (j > 0) ax = ax - wi * cvt<double>(C[t - g.Sx]);
                if (j < g.b - 1) ax = ax - wi * cvt<double>(C[t + g.Sx]);
            }
            double* a = As + 3 * (size_t)e;
            double* b = Bs + 3 * (size_t)e;
            a[0] = cv.re;
            a[1] = cv.im;
            a[2] = cv.re - cv.im;
            b[0] = ax.re;
            b[1] = ax.im - ax.re;
            b[2] = ax.re + ax.im;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < KMAX; ++k) {
            const int o = threadIdx.x + k * G3_THREADS;
            if (o >= nout) continue;
            const int i = o / p, j = o % p;
            if (ihi > 0 && (i < ilo || i >= ihi)) continue;
            if (jhi > 0 && (j < jlo || j >= jhi)) continue;
            double x1 = s1[k], x2 = s2[k], x3 = s3[k];
            for (int n = 0; n < rows; ++n) {
                const double* a = As + 3 * ((size_t)n * p + i);
                const double* b = Bs + 3 * ((size_t)n * p + j);
                x1 = fma(b[0], a[2], x1);
                x2 = fma(a[0], b[1], x2);
                x3 = fma(a[1], b[2], x3);
            }
            s1[k] = x1;
            s2[k] = x2;
            s3[k] = x3;
        }
        __syncthreads();
    }
    c128* out = partial + (size_t)blockIdx.x * nout;
#pragma unroll
    for (int k = 0; k < KMAX; ++k) {
        const int o = threadIdx.x + k * G3_THREADS;
        if (o < nout) out[o] = {s1[k] + s3[k], s1[k] + s2[k]};
    }
}

// ------------------------------------------------ Hermitian-packed FP64 Galerkin matrix
// For the 5-point rows A~ is complex symmetric with real couplings: A~ = S + i D, S = Re A~
// real symmetric and D = Im A~ diagonal, nonzero only on the band's boundary points (the
// impedance terms).  So A_c = C^H S C + i C^H D C with both terms Hermitian, and for i < j
//   A_c[j][i] = conj(A_c[i][j]) + 2i conj(H_D[i][j]),   H_D = C^H D C.
// k_galerkin_herm sums A_c[i][j] over its points for i <= j only (about half the products
// of the full matrix) into slot [i][j] of the block's partial, zero below the diagonal;
// k_galerkin_bdry sums 2i conj(H_D[i][j]) over boundary points into the slots [j][i]; after
// the fixed-order sum over blocks k_herm_fill forms A_c[j][i] = conj(A_c[i][j]) + slot[j][i].
// The sums of a pair are the 3M products of k_galerkin_partial3, in FP64.

// Block point ranges of equal cost for k_galerkin_herm: a point of row split_row - 1 (the
// only row where the first child's columns meet the second child's, through the stencil)
// costs wgt, any other point 1.
__device__ __forceinline__ void gal_range_w(size_t N, int Sx, int split_row, int wgt, unsigned blk, unsigned nblk,
                                            size_t& n0, size_t& n1) {
    size_t s0 = 0, s1 = 0;
    if (split_row >= 1) {
        s0 = min(N, (size_t)(split_row - 1) * Sx);
        s1 = min(N, (size_t)split_row * Sx);
    }
    const size_t w = (size_t)wgt;
    const size_t T = N + (w - 1) * (s1 - s0);
    auto inv = [&](size_t c) -> size_t {
        if (c <= s0) return c;
        if (c <= s0 + w * (s1 - s0)) return s0 + (c - s0) / w;
        return c - (w - 1) * (s1 - s0);
    };
    n0 = inv(T * blk / nblk);
    n1 = blk + 1 == nblk ? N : inv(T * (blk + 1) / nblk);
}

// Pair t of the upper triangle (diagonal included) of an m x m block, rows folded in
// pairs (r, m - 1 - r) so that consecutive t run along one row: t = r (m + 1) + c.
__device__ __forceinline__ void tri_pair(int t, int m, int& i, int& j) {
    const int r = t / (m + 1), c = t - r * (m + 1);
    if (c < m - r) {
        i = r;
        j = r + c;
    } else {
        i = m - 1 - r;
        j = c - 1;
    }
}

static constexpr int GH_SLOTS = 6;
template <typename TI>
__global__ void __launch_bounds__(G3_THREADS, 1) k_galerkin_herm(const cplx<TI>* __restrict__ C, OpGeom g, int p,
                                                                 int split_row, int wgt, c128* partial) {
    extern __shared__ __align__(16) unsigned char gsm_[];
    const int plane = IP_TILE * p;
    double* A0 = (double*)gsm_;   // ar, ai, ar - ai of conj(C)'s factor
    double* A1 = A0 + plane;
    double* A2 = A1 + plane;
    double* B0 = A2 + plane;      // br, bi - br, br + bi of A~ C
    double* B1 = B0 + plane;
    double* B2 = B1 + plane;
    const int ph = p / 2, T = ph * (ph + 1) / 2, X = ph * ph;
    const int RT = (T + G3_THREADS - 1) / G3_THREADS, RC = (X + G3_THREADS - 1) / G3_THREADS;
    // the thread's pairs: slot k belongs to set 0 (first half's triangle), 1 (second
    // half's) or 2 (first half's rows against the second half's columns), one round of
    // G3_THREADS pairs each.  A warp's FP64 instruction costs the same however many of its
    // lanes are active, so the pairs of a partial round are shared out over all sixteen
    // warps, and the lanes given one pair split the tile's points between them (sn0: first
    // point, snst: step); their sums are added across those lanes at the end.
    int si[GH_SLOTS], sj[GH_SLOTS], ss[GH_SLOTS], sn0[GH_SLOTS], snst[GH_SLOTS];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < GH_SLOTS; ++k) {
        int set, rnd;
        if (k < RT) { set = 0; rnd = k; }
        else if (k < 2 * RT) { set = 1; rnd = k - RT; }
        else { set = 2; rnd = k - 2 * RT; }
        const int size = set == 2 ? X : T;
        const int rem = k < 2 * RT + RC ? size - rnd * G3_THREADS : 0;
        int e = -1;
        sn0[k] = 0;
        snst[k] = 1;
        if (rem >= G3_THREADS) {
            e = rnd * G3_THREADS + threadIdx.x;
        } else if (rem > 0) {
            const int ppw = (rem + 15) / 16, L = max(1, 32 / ppw);
            const int gq = lane / L, m = w * ppw + gq;
            sn0[k] = lane - gq * L;
            snst[k] = L;
            if (gq < ppw && m < rem) e = rnd * G3_THREADS + m;
        }
        ss[k] = e < 0 ? -1 : set;
        si[k] = sj[k] = 0;
        if (e >= 0) {
            if (set == 2) {
                si[k] = e / ph;
                sj[k] = ph + e % ph;
            } else {
                tri_pair(e, ph, si[k], sj[k]);
                si[k] += set * ph;
                sj[k] += set * ph;
            }
        }
    }
    double s1[GH_SLOTS], s2[GH_SLOTS], s3[GH_SLOTS];
#pragma unroll
    for (int k = 0; k < GH_SLOTS; ++k) s1[k] = s2[k] = s3[k] = 0.0;
    const size_t N = (size_t)g.b * g.Sx;
    size_t n0, n1;
    gal_range_w(N, g.Sx, split_row, wgt, blockIdx.x, gridDim.x, n0, n1);
    for (size_t t0 = n0; t0 < n1; t0 += IP_TILE) {
        const int rows = (int)min((size_t)IP_TILE, n1 - t0);
        // the sets with nonzero terms on this tile's rows: the first half's columns of C
        // live on rows < split_row, the second's on the others, and A~ C reaches one row
        // further
        bool act0 = true, act1 = true, actx = true;
        if (split_row >= 0) {
            const int j0 = (int)(t0 / g.Sx), j1 = (int)((t0 + rows - 1) / g.Sx);
            act0 = j0 < split_row;
            act1 = j1 >= split_row;
            actx = j0 <= split_row - 1 && j1 >= split_row - 1;
        }
        for (int e = threadIdx.x; e < rows * p; e += G3_THREADS) {
            const size_t pt = t0 + e / p;
            const int l = e % p;
            const bool lo = l < ph;
            const bool need_a = lo ? (act0 || actx) : act1;
            const bool need_b = lo ? act0 : (act1 || actx);
            if (!need_a && !need_b) continue;
            const int i = (int)(pt % g.Sx), j = (int)(pt / g.Sx);
            const size_t t = (size_t)l * N + pt;
            const c128 cv = cvt<double>(C[t]);
            c128 ax;
            if (g.Sx > 1 && i > 0 && i < g.Sx - 1 && j > 0 && j < g.b - 1) {
                const double kr = g.khr ? g.khr[j] : g.kh;
                const double d = 4.0 - kr * kr;
                const c128 q1 = cvt<double>(C[t - 1]), q2 = cvt<double>(C[t + 1]);
                const c128 q3 = cvt<double>(C[t - g.Sx]), q4 = cvt<double>(C[t + g.Sx]);
                ax.re = d * cv.re - q1.re - q2.re - q3.re - q4.re;
                ax.im = d * cv.im - q1.im - q2.im - q3.im - q4.im;
            } else {
                ax = op_diag(j, i, g) * cv;
                const double wj = wrow(j, g.b), wi = wcol(i, g.Sx);
                if (g.Sx > 1) {
                    if (i > 0) ax = ax - wj * cvt<double>(C[t - 1]);
                    if (i < g.Sx - 1) ax = ax - wj * cvt<double>(C[t + 1]);
                }
                if (j > 0) ax = ax - wi * cvt<double>(C[t - g.Sx]);
                if (j < g.b - 1) ax = ax - wi * cvt<double>(C[t + g.Sx]);
            }
            A0[e] = cv.re;
            A1[e] = cv.im;
            A2[e] = cv.re - cv.im;
            B0[e] = ax.re;
            B1[e] = ax.im - ax.re;
            B2[e] = ax.re + ax.im;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < GH_SLOTS; ++k) {
            const int set = ss[k];
            if (set < 0 || !(set == 0 ? act0 : (set == 1 ? act1 : actx))) continue;
            const int i = si[k], j = sj[k];
            double x1 = s1[k], x2 = s2[k], x3 = s3[k];
            for (int n = sn0[k]; n < rows; n += snst[k]) {
                const int ai = n * p + i, bj = n * p + j;
                x1 = fma(B0[bj], A2[ai], x1);
                x2 = fma(A0[ai], B1[bj], x2);
                x3 = fma(A1[ai], B2[bj], x3);
            }
            s1[k] = x1;
            s2[k] = x2;
            s3[k] = x3;
        }
        __syncthreads();
    }
    // the lanes that shared a pair's points: their sums added in lane order (the step is
    // the same for the whole warp)
#pragma unroll
    for (int k = 0; k < GH_SLOTS; ++k) {
        const int L = snst[k];
        if (L > 1) {
            const int base = lane - sn0[k];
            double t1 = 0.0, t2 = 0.0, t3 = 0.0;
            for (int d = 0; d < L; ++d) {
                const int src = (base + d) & 31;
                t1 += __shfl_sync(0xffffffffu, s1[k], src);
                t2 += __shfl_sync(0xffffffffu, s2[k], src);
                t3 += __shfl_sync(0xffffffffu, s3[k], src);
            }
            s1[k] = t1;
            s2[k] = t2;
            s3[k] = t3;
            if (sn0[k] != 0) ss[k] = -1;   // one lane of the group writes
        }
    }
    c128* out = partial + (size_t)blockIdx.x * p * p;
    for (int o = threadIdx.x; o < p * p; o += G3_THREADS)
        if (o / p > o % p) out[o] = {0.0, 0.0};
#pragma unroll
    for (int k = 0; k < GH_SLOTS; ++k)
        if (ss[k] >= 0) out[(size_t)si[k] * p + sj[k]] = {s1[k] + s3[k], s1[k] + s2[k]};
}

// Boundary points of a band (those with an impedance term): rows 0 and b - 1, then the
// first and last column of the rows between (Sx > 1).
__host__ __device__ inline int band_boundary_points(int b, int Sx) {
    if (b <= 1) return Sx;
    return 2 * Sx + (Sx > 1 ? 2 * (b - 2) : 0);
}
__device__ __forceinline__ void band_boundary_point(int q, int b, int Sx, int& j, int& i) {
    if (q < Sx) { j = 0; i = q; return; }
    if (q < 2 * Sx) { j = b - 1; i = q - Sx; return; }
    const int k = q - 2 * Sx;
    j = 1 + k / 2;
    i = (k & 1) ? Sx - 1 : 0;
}

// slot [j][i] (i < j) of block blockIdx.x's partial: 2i conj(sum conj(C_i) D C_j) over the
// block's `chunk` boundary points; zero elsewhere (and for i, j in different halves of a
// split basis, whose columns never meet at one point)
template <typename TI>
__global__ void __launch_bounds__(256) k_galerkin_bdry(const cplx<TI>* __restrict__ C, OpGeom g, int p, int split_row,
                                                       int chunk, c128* partial) {
    extern __shared__ c128 bsm_[];
    c128* Cs = bsm_;                // [chunk][p] C
    c128* Ds = bsm_ + (size_t)chunk * p;   // [chunk][p] D C
    const size_t N = (size_t)g.b * g.Sx;
    const int nbp = band_boundary_points(g.b, g.Sx);
    const int q0 = blockIdx.x * chunk, nq = max(0, min(nbp, q0 + chunk) - q0);
    for (int e = threadIdx.x; e < nq * p; e += blockDim.x) {
        const int n = e / p, l = e % p;
        int j, i;
        band_boundary_point(q0 + n, g.b, g.Sx, j, i);
        const c128 cv = cvt<double>(C[(size_t)l * N + (size_t)j * g.Sx + i]);
        const double d = op_diag(j, i, g).im;
        Cs[e] = cv;
        Ds[e] = {d * cv.re, d * cv.im};
    }
    __syncthreads();
    const int ph = p / 2;
    c128* out = partial + (size_t)blockIdx.x * p * p;
    for (int o = threadIdx.x; o < p * p; o += blockDim.x) {
        const int jr = o / p, ic = o % p;   // slot [j][i]
        c128 h = {0.0, 0.0};
        if (jr > ic && !(split_row >= 0 && (ic < ph) != (jr < ph)))
            for (int n = 0; n < nq; ++n) cfma_cj(h, Cs[n * p + ic], Ds[n * p + jr]);
        out[o] = jr > ic ? c128{2.0 * h.im, 2.0 * h.re} : c128{0.0, 0.0};
    }
}

__global__ void k_herm_fill(c128* A, int p) {
    for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < p * p; o += gridDim.x * blockDim.x) {
        const int r = o / p, c = o % p;
        if (r > c) A[o] = conj(A[(size_t)c * p + r]) + A[o];
    }
}
void launch_herm_fill(c128* A, int p, cudaStream_t s) {
    k_herm_fill<<<(p * p + 255) / 256, 256, 0, s>>>(A, p);
    note_launch();
}

template <typename TI, typename T>
int launch_galerkin_partial(const cplx<TI>* C, OpGeom g, int p, int split_row, c128* partial, int max_blocks,
                            cudaStream_t s, bool* herm) {
    const size_t N = (size_t)g.b * g.Sx;
    if (herm) *herm = false;
    int grid = (int)((N + 127) / 128);
    if (grid > max_blocks) grid = max_blocks;
    if (grid < 1) grid = 1;
    const int nout = p * p;
    const int split = nout >= IP_THREADS ? 1 : IP_THREADS / nout;
    const size_t sm = sizeof(cplx<T>) * (size_t)IP_TILE * 2 * p + (split > 1 ? sizeof(c128) * split * nout : 0);
    static std::atomic<unsigned long long> attr4{0}, attrmax{0};
    smem_limit_once(attr4, k_galerkin_partial<TI, T, 4>, 200 * 1024);
    smem_limit_once(attrmax, k_galerkin_partial<TI, T, IP_MAXOUT>, 200 * 1024);
    if (sizeof(T) == sizeof(double) && herm && !g.q1 && p % 2 == 0 && p <= 64 && nout >= G3_THREADS) {
        // FP64 products of the 5-point rows: the Hermitian-packed form, the blocks' point
        // ranges balanced with the rows' costs (the row before the split also pairs the
        // first half's columns with the second's); the boundary terms go to the blocks
        // after those (at most max_blocks + 1 - g3 of them)
        const int g3 = std::min(grid, max_blocks / 2 > 0 ? max_blocks / 2 : 1);
        const int nbp = band_boundary_points(g.b, g.Sx);
        const int room = std::max(1, max_blocks + 1 - g3);
        const int chunk = std::max(16, (nbp + room - 1) / room);
        const int maxchunk = (int)((96 * 1024) / (2 * sizeof(c128) * p));
        if (chunk <= maxchunk) {
            const int ph = p / 2, T3 = ph * (ph + 1) / 2;
            const int wgt = split_row >= 1 ? (T3 + ph * ph + T3 / 2) / T3 : 1;
            const size_t smh = sizeof(double) * 6 * (size_t)IP_TILE * p;
            static std::atomic<unsigned long long> ah{0}, ab{0};
            smem_limit_once(ah, k_galerkin_herm<TI>, 200 * 1024);
            smem_limit_once(ab, k_galerkin_bdry<TI>, 200 * 1024);
            k_galerkin_herm<TI><<<g3, G3_THREADS, smh, s>>>(C, g, p, split_row, wgt, partial);
            note_launch();
            const int nbx = (nbp + chunk - 1) / chunk;
            const size_t smb = 2 * sizeof(c128) * (size_t)chunk * p;
            k_galerkin_bdry<TI><<<nbx, 256, smb, s>>>(C, g, p, split_row, chunk, partial + (size_t)g3 * nout);
            note_launch();
            *herm = true;
            return g3 + nbx;
        }
    }
    if (sizeof(T) == sizeof(double) && nout >= G3_THREADS && nout <= 8 * G3_THREADS) {
        // FP64 products, whole outputs per thread: the 3M form, one block per SM
        const size_t sm3 = sizeof(double) * 6 * (size_t)IP_TILE * p;
        static std::atomic<unsigned long long> a32{0}, a34{0}, a38{0};
        smem_limit_once(a32, k_galerkin_partial3<TI, 2>, 200 * 1024);
        smem_limit_once(a34, k_galerkin_partial3<TI, 4>, 200 * 1024);
        smem_limit_once(a38, k_galerkin_partial3<TI, 8>, 200 * 1024);
        const int g3 = std::min(grid, max_blocks / 2 > 0 ? max_blocks / 2 : 1);
        if (nout <= 2 * G3_THREADS)
            k_galerkin_partial3<TI, 2><<<g3, G3_THREADS, sm3, s>>>(C, g, p, split_row, partial);
        else if (nout <= 4 * G3_THREADS)
            k_galerkin_partial3<TI, 4><<<g3, G3_THREADS, sm3, s>>>(C, g, p, split_row, partial);
        else
            k_galerkin_partial3<TI, 8><<<g3, G3_THREADS, sm3, s>>>(C, g, p, split_row, partial);
        note_launch();
        return g3;
    }
    // accumulators sized to the outputs a thread owns (p <= 32: at most 4), so that the
    // registers allow two blocks per SM and the grid runs in one wave
    if (nout <= 4 * IP_THREADS)
        k_galerkin_partial<TI, T, 4><<<grid, IP_THREADS, sm, s>>>(C, g, p, split_row, partial);
    else
        k_galerkin_partial<TI, T, IP_MAXOUT><<<grid, IP_THREADS, sm, s>>>(C, g, p, split_row, partial);
    note_launch();
    return grid;
}

// ------------------------------------------------------------------------ QR
// Classical Gram-Schmidt applied twice per column (orthogonal to working precision
// for full-rank input); column j of Y becomes q_j with r_jj > 0 real.  One CTA per
// block; the block stays in global memory (L2).
// The block is staged in shared memory when it fits (every step of the sequential
// column loop then waits on shared rather than global memory latency).
template <typename T>
__global__ void __launch_bounds__(512) k_qr(cplx<T>* const* Yp, int Sx, int m, int staged) {
    cplx<T>* Yg = Yp[blockIdx.x];
    extern __shared__ __align__(16) unsigned char qsm[];
    cplx<T>* Y = staged ? (cplx<T>*)qsm : Yg;
    __shared__ cplx<T> dots[128];
    __shared__ T red[32];
    __shared__ T s_inv;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const size_t tot = (size_t)Sx * m;
    // the staged copy's rows are m + 1 apart: a warp reading one column of consecutive
    // rows then spreads over the shared-memory banks
    const int ld = staged ? m + 1 : m;
    if (staged) {
        for (size_t e0 = threadIdx.x; e0 < tot; e0 += 4 * blockDim.x) {
            cplx<T> t[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const size_t e = e0 + (size_t)u * blockDim.x;
                if (e < tot) t[u] = Yg[e];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const size_t e = e0 + (size_t)u * blockDim.x;
                if (e < tot) Y[(e / m) * ld + e % m] = t[u];
            }
        }
        __syncthreads();
    }
    for (int j = 0; j < m; ++j) {
        for (int pass = 0; pass < 2 && j > 0; ++pass) {
            for (int k = warp; k < j; k += nw) {
                cplx<T> a = {0, 0};
                for (int x = lane; x < Sx; x += 32) cfma_cj(a, Y[(size_t)x * ld + k], Y[(size_t)x * ld + j]);
                a = warp_sum(a);
                if (lane == 0) dots[k] = a;
            }
            __syncthreads();
            for (int x = threadIdx.x; x < Sx; x += blockDim.x) {
                cplx<T> v = Y[(size_t)x * ld + j];
                for (int k = 0; k < j; ++k) v = v - Y[(size_t)x * ld + k] * dots[k];
                Y[(size_t)x * ld + j] = v;
            }
            __syncthreads();
        }
        T a2 = 0;
        for (int x = threadIdx.x; x < Sx; x += blockDim.x) a2 += abs2(Y[(size_t)x * ld + j]);
        a2 = warp_sum(a2);
        if (lane == 0) red[warp] = a2;
        __syncthreads();
        if (warp == 0) {
            T v = lane < nw ? red[lane] : (T)0;
            v = warp_sum(v);
            if (lane == 0) {
                const T nrm = sqrt(v);
                s_inv = nrm > (T)0 ? (T)1 / nrm : (T)0;
            }
        }
        __syncthreads();
        const T inv = s_inv;
        for (int x = threadIdx.x; x < Sx; x += blockDim.x) Y[(size_t)x * ld + j] = inv * Y[(size_t)x * ld + j];
        __syncthreads();
    }
    if (staged)
        for (size_t e = threadIdx.x; e < tot; e += blockDim.x) Yg[e] = Y[(e / m) * ld + e % m];
}
// The same orthogonalisation for a block too large for one CTA's shared memory: a cluster
// of QR_CL CTAs per block, each holding a slice of the rows in shared memory.  Each dot
// product and norm is a sum of the CTAs' partial sums, added in rank order from
// distributed shared memory, so every CTA takes the same coefficients; the partial-sum
// arrays alternate between two buffers, and the cluster barrier after each write keeps a
// CTA from overwriting a buffer another is still reading.
static constexpr int QR_CL = 8;
template <typename T>
__global__ void __launch_bounds__(512) k_qr_cluster(cplx<T>* const* Yp, int Sx, int m) {
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    cplx<T>* Yg = Yp[blockIdx.x / QR_CL];
    extern __shared__ __align__(16) unsigned char qcs[];
    const int ld = m + 1;                       // padded rows (bank spread)
    const int rows = (Sx + QR_CL - 1) / QR_CL;
    const int r0 = min(Sx, rank * rows), r1 = min(Sx, r0 + rows), nr = r1 - r0;
    cplx<T>* Y = (cplx<T>*)qcs;                 // [rows][ld]
    __shared__ cplx<T> pd[2][128];              // partial dot products (two buffers)
    __shared__ T pn[2];                         // partial squared norms
    __shared__ cplx<T> dots[128];
    __shared__ T red[32];
    __shared__ T s_inv;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int e = threadIdx.x; e < nr * m; e += blockDim.x) {
        const int x = e / m, c = e - x * m;
        Y[x * ld + c] = Yg[(size_t)(r0 + x) * m + c];
    }
    __syncthreads();
    int buf = 0;
    for (int j = 0; j < m; ++j) {
        for (int pass = 0; pass < 2 && j > 0; ++pass) {
            for (int k = warp; k < j; k += nw) {
                cplx<T> a = {0, 0};
                for (int x = lane; x < nr; x += 32) cfma_cj(a, Y[x * ld + k], Y[x * ld + j]);
                a = warp_sum(a);
                if (lane == 0) pd[buf][k] = a;
            }
            cluster.sync();
            for (int k = threadIdx.x; k < j; k += blockDim.x) {
                cplx<T> a = {0, 0};
                for (int r = 0; r < QR_CL; ++r) a = a + cluster.map_shared_rank(&pd[buf][0], r)[k];
                dots[k] = a;
            }
            buf ^= 1;
            __syncthreads();
            for (int x = threadIdx.x; x < nr; x += blockDim.x) {
                cplx<T> v = Y[x * ld + j];
                for (int k = 0; k < j; ++k) v = v - Y[x * ld + k] * dots[k];
                Y[x * ld + j] = v;
            }
            __syncthreads();
        }
        T a2 = 0;
        for (int x = threadIdx.x; x < nr; x += blockDim.x) a2 += abs2(Y[x * ld + j]);
        a2 = warp_sum(a2);
        if (lane == 0) red[warp] = a2;
        __syncthreads();
        if (warp == 0) {
            T v = lane < nw ? red[lane] : (T)0;
            v = warp_sum(v);
            if (lane == 0) pn[buf] = v;
        }
        cluster.sync();
        if (threadIdx.x == 0) {
            T v = 0;
            for (int r = 0; r < QR_CL; ++r) v += *cluster.map_shared_rank(&pn[buf], r);
            const T nrm = sqrt(v);
            s_inv = nrm > (T)0 ? (T)1 / nrm : (T)0;
        }
        buf ^= 1;
        __syncthreads();
        const T inv = s_inv;
        for (int x = threadIdx.x; x < nr; x += blockDim.x) Y[x * ld + j] = inv * Y[x * ld + j];
        __syncthreads();
    }
    for (int e = threadIdx.x; e < nr * m; e += blockDim.x) {
        const int x = e / m, c = e - x * m;
        Yg[(size_t)(r0 + x) * m + c] = Y[x * ld + c];
    }
    // no CTA leaves while another may still read its partial sums
    cluster.sync();
}

template <typename T>
void launch_qr(cplx<T>* const* Y, int nq, int Sx, int m, cplx<T>** dev_ptr_scratch, cudaStream_t s) {
    cudaMemcpyAsync(dev_ptr_scratch, Y, sizeof(cplx<T>*) * nq, cudaMemcpyHostToDevice, s);
    static std::atomic<unsigned long long> attr{0};
    smem_limit_once(attr, k_qr<T>, 200 * 1024);
    const size_t bytes = sizeof(cplx<T>) * (size_t)Sx * (m + 1);   // padded rows
    const int staged = bytes <= (size_t)(200 * 1024) - 2048;
    const size_t cbytes = sizeof(cplx<T>) * (size_t)((Sx + QR_CL - 1) / QR_CL) * (m + 1);
    if (!staged && m <= 128 && cbytes <= (size_t)(200 * 1024) - 4096) {
        static std::atomic<unsigned long long> attr_c{0};
        smem_limit_once(attr_c, k_qr_cluster<T>, 200 * 1024);
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[1];
        cfg.gridDim = dim3(nq * QR_CL);
        cfg.blockDim = dim3(512);
        cfg.dynamicSmemBytes = cbytes;
        cfg.stream = s;
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = QR_CL;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        cudaLaunchKernelEx(&cfg, k_qr_cluster<T>, dev_ptr_scratch, Sx, m);
        note_launch();
        return;
    }
    k_qr<T><<<nq, 512, staged ? bytes : 0, s>>>(dev_ptr_scratch, Sx, m, staged);
    note_launch();
}

// ------------------------------------------------------ Hermitian eigen (FP64)
// Eigenvalues (all, descending) and the r leading eigenvectors of the m x m Hermitian
// Gram matrix G = Z^H Z of the sketch, in FP64, in two launches:
//  1. (one CTA per matrix) Householder reduction to tridiagonal form, H_k = I - tau v v^H
//     applied on both sides of the trailing block (w = tau A v, q = w - (tau/2)(v^H w) v,
//     A <- A - v q^H - q v^H); a diagonal unitary scaling makes the tridiagonal real
//     symmetric;
//  2. (one warp per eigenvalue and matrix, spread over the SMs: FP64 is throughput-bound
//     per SM) each eigenvalue by multisection on Sturm counts; the r leading eigenvectors
//     by inverse iteration on the tridiagonal (pivoted LU), mapped back through the
//     scaling and the reflectors.
static constexpr int HE_MAX = 64;

// Number of eigenvalues below x: sign changes of the leading principal minors
// p_0 = 1, p_i = (d_{i-1} - x) p_{i-1} - e_{i-2}^2 p_{i-2} (Sturm sequence).  Three FP64
// operations per step: the sign test and the range check read the sign and exponent
// bits with integer instructions, and the pair (p_i, p_{i-1}) is rescaled by an exact
// power of two when it leaves [2^-400, 2^400].  A vanishing minor needs no special
// case: p_{i+1} = -e^2 p_{i-1} then has the opposite sign of p_{i-1}, so the triple
// counts one change whichever sign the zero is given.
__device__ int sturm_count(const double* d, const double* e2, int m, double x) {
    double pm = 1.0, p = d[0] - x;
    int hp = __double2hiint(p);
    int c = hp < 0;
    for (int i = 1; i < m; ++i) {
        const double pn = fma(d[i] - x, p, -(e2[i - 1] * pm));
        const int hn = __double2hiint(pn);
        c += (hn ^ hp) < 0;
        pm = p;
        p = pn;
        hp = hn;
        const int ex = max((hn >> 20) & 0x7ff, (__double2hiint(pm) >> 20) & 0x7ff);
        if (ex > 1023 + 400) {
            p *= 0x1p-400;
            pm *= 0x1p-400;
        } else if (ex < 1023 - 400 && ex > 0) {
            p *= 0x1p+400;
            pm *= 0x1p+400;
        }
    }
    return c;
}

// Stage 1, one block per matrix: Householder reduction of the Hermitian G to a real
// symmetric tridiagonal T = D^H Q^H G Q D (d diagonal, eb >= 0 off-diagonal, D = diag
// of unit phases).  Overwrites G with the workspace read by stage 2: reflector k in
// row k (tau_k = 2 / ||v_k||^2), then d, eb, eb^2, tau (m doubles each) and D (m
// complex) from offset m^2.
//
// FP64 issue on one SM bounds this kernel, so each column's step is laid out by FP64
// instruction count. Only the lower triangle of the trailing matrix is kept, and the
// rank-2 update touches only that triangle. The product A'v reads an upper entry as
// the conjugate of its mirror, with the sign of the imaginary part flipped by an
// integer operation. The product is formed as four column-interleaved partial sums
// per row, one warp per SM sub-partition, then added in a fixed order. The scalar
// work of a column (the reflector, K and q) runs in warp 0 alone, with four block
// barriers per column.
__global__ void __launch_bounds__(256) k_heig_tri(c128* const* Gp, int m) {
    extern __shared__ __align__(16) unsigned char hsm[];
    c128* A = (c128*)hsm;                    // m x m working matrix (lower triangle)
    c128* Vr = A + m * m;                    // reflector k stored in row k (length m-k-1)
    c128* w = Vr + m * m;                    // m: q = tau A'v - K v
    double* tau = (double*)(w + m);          // m
    double* d = tau + m;                     // m   diagonal of the real tridiagonal
    double* eb = d + m;                      // m   |subdiagonal|
    double* e2 = eb + m;                     // m   squared
    c128* delta = (c128*)(e2 + m);           // m   diagonal unitary scaling
    c128* part = delta + m;                  // 4 x m partial sums of A'v; phases at the end
    __shared__ c128 s_beta;
    c128* G = Gp[blockIdx.x];
    for (int t = threadIdx.x; t < m * m; t += blockDim.x) A[t] = G[t];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = 0; k + 2 < m; ++k) {
        const int n = m - k - 1;             // length of the column below the diagonal
        c128* v = Vr + k * m;
        const c128* a0 = A + (k + 1) * m + (k + 1);   // trailing block, row stride m
        // v = x - beta e_1 with beta = -|x| x_0 / |x_0|, and tau = 2 / ||v||^2; every lane
        // of warp 0 forms the same scalars
        if (warp == 0) {
            double a2 = 0.0;
            for (int i = lane; i < n; i += 32) a2 += abs2(A[(k + 1 + i) * m + k]);
            a2 = warp_sum(a2);
            const c128 x0 = A[(k + 1) * m + k];
            const double alpha = sqrt(a2);
            const double ax02 = abs2(x0);
            double ax0 = 0.0;
            c128 ph = {1.0, 0.0};
            if (ax02 > 0.0) {
                const double r0 = rsqrt(ax02);
                ax0 = ax02 * r0;
                ph = r0 * x0;
            }
            const c128 beta = (-alpha) * ph;
            const double tk = alpha > 0.0 ? 1.0 / (alpha * (alpha + ax0)) : 0.0;
            for (int i = lane; i < n; i += 32) {
                c128 x = A[(k + 1 + i) * m + k];
                if (i == 0) x = x - beta;
                v[i] = x;
            }
            if (lane == 0) {
                tau[k] = tk;
                s_beta = beta;
            }
        }
        __syncthreads();
        const double tk = tau[k];
        // thread (q, i) adds columns q, q + 4, ... of row i of A'v (4 n <= 252 threads)
        for (int t = threadIdx.x; t < 4 * n; t += blockDim.x) {
            const int q = t / n, i = t - q * n;
            c128 acc = {0.0, 0.0};
            for (int j = q; j < n; j += 4) {
                const bool lo = j <= i;
                c128 a = a0[lo ? i * m + j : j * m + i];
                a.im = __hiloint2double(__double2hiint(a.im) ^ (lo ? 0 : (int)0x80000000), __double2loint(a.im));
                cfma(acc, a, v[j]);
            }
            part[q * m + i] = acc;
        }
        __syncthreads();
        // warp 0: w = tau A'v, K = (tau / 2) v^H w, q = w - K v (rows lane and lane + 32)
        if (warp == 0) {
            c128 wl[2];
            c128 kp = {0.0, 0.0};
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int i = lane + 32 * h;
                c128 s = {0.0, 0.0};
                if (i < n) {
                    s = tk * (((part[i] + part[m + i]) + part[2 * m + i]) + part[3 * m + i]);
                    cfma_cj(kp, v[i], s);
                }
                wl[h] = s;
            }
            const c128 K = (0.5 * tk) * warp_sum(kp);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int i = lane + 32 * h;
                if (i < n) w[i] = wl[h] - K * v[i];
            }
        }
        __syncthreads();
        // A' -= v q^H + q v^H on the lower triangle; thread t takes element t of the
        // row-major triangle, i from the triangular root and two exact integer corrections
        const int nt = n * (n + 1) / 2;
        for (int t = threadIdx.x; t < nt; t += blockDim.x) {
            int i = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
            while (i * (i + 1) / 2 > t) --i;
            while ((i + 1) * (i + 2) / 2 <= t) ++i;
            const int j = t - i * (i + 1) / 2;
            c128& a = A[(k + 1 + i) * m + (k + 1 + j)];
            const c128 vi = v[i], vj = v[j], wi = w[i], wj = w[j];
            a.re = fma(-vi.re, wj.re, fma(-vi.im, wj.im, fma(-wi.re, vj.re, fma(-wi.im, vj.im, a.re))));
            a.im = fma(-vi.im, wj.re, fma(vi.re, wj.im, fma(-wi.im, vj.re, fma(wi.re, vj.im, a.im))));
        }
        const c128 beta = s_beta;
        for (int i = threadIdx.x; i < n; i += blockDim.x)
            A[(k + 1 + i) * m + k] = (i == 0) ? beta : c128{0.0, 0.0};
        __syncthreads();
    }
    // d, eb, eb^2 and the unit phases of the subdiagonal, one thread per index; the
    // phases' prefix product (D) by thread 0
    c128* phs = part;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        d[i] = A[i * m + i].re;
        if (i + 1 < m) {
            const c128 e = A[(i + 1) * m + i];
            const double ae = sqrt(abs2(e));
            eb[i] = ae;
            e2[i] = ae * ae;
            phs[i] = ae > 0.0 ? (1.0 / ae) * e : c128{1.0, 0.0};
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        c128 dl = {1.0, 0.0};
        for (int i = 0; i < m; ++i) {
            delta[i] = dl;
            if (i + 1 < m) dl = dl * phs[i];
        }
    }
    // the Gershgorin interval of T, warp 1
    double* ws = (double*)(G + (size_t)m * m);
    if (warp == 1) {
        double lo0 = 0.0, hi0 = 0.0;
        bool any = false;
        for (int i = lane; i < m; i += 32) {
            const double rad = (i > 0 ? eb[i - 1] : 0.0) + (i + 1 < m ? eb[i] : 0.0);
            lo0 = any ? fmin(lo0, d[i] - rad) : d[i] - rad;
            hi0 = any ? fmax(hi0, d[i] + rad) : d[i] + rad;
            any = true;
        }
        if (!any) { lo0 = 1e300; hi0 = -1e300; }
        for (int o = 16; o > 0; o >>= 1) {
            lo0 = fmin(lo0, __shfl_xor_sync(0xffffffffu, lo0, o));
            hi0 = fmax(hi0, __shfl_xor_sync(0xffffffffu, hi0, o));
        }
        if (lane == 0) {
            ws[6 * m] = lo0;
            ws[6 * m + 1] = hi0;
        }
    }
    __syncthreads();
    // write the workspace (G is no longer needed)
    for (int t = threadIdx.x; t < m * m; t += blockDim.x) G[t] = Vr[t];
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        ws[i] = d[i];
        ws[m + i] = eb[i];
        ws[2 * m + i] = e2[i];
        ws[3 * m + i] = tau[i];
        ((c128*)(ws + 4 * m))[i] = delta[i];
    }
}

// Stage 2, one block of four warps per (eigenvalue, matrix): the kk-th largest
// eigenvalue of T by multisection (128 Sturm-count probes per round, one per thread, so
// that each SM's four FP64 pipes work); for kk < r also its eigenvector (warp 0):
// inverse iteration with a pivoted tridiagonal LU (two steps from a fixed start),
// then u = Q D y by the reflectors in reverse.
static constexpr int HV_THREADS = 128;
__global__ void __launch_bounds__(HV_THREADS) k_heig_vec(c128* const* Gp, c128* const* Up, double* const* lamp,
                                                         int m, int r) {
    __shared__ double d[HE_MAX], eb[HE_MAX], e2[HE_MAX], tau[HE_MAX];
    __shared__ c128 delta[HE_MAX], u[HE_MAX];
    __shared__ double dg[HE_MAX], up[HE_MAX], up2[HE_MAX], lo[HE_MAX], y[HE_MAX];
    __shared__ bool sw[HE_MAX];
    __shared__ unsigned s_mask[HV_THREADS / 32];
    const int kk = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const c128* Vr = Gp[blockIdx.y];
    const double* ws = (const double*)(Vr + (size_t)m * m);
    for (int i = tid; i < m; i += HV_THREADS) {
        d[i] = ws[i];
        eb[i] = ws[m + i];
        e2[i] = ws[2 * m + i];
        tau[i] = ws[3 * m + i];
        delta[i] = ((const c128*)(ws + 4 * m))[i];
    }
    const double lo0 = ws[6 * m], hi0 = ws[6 * m + 1];
    __syncthreads();
    const double span = fmax(hi0 - lo0, 1e-300);
    double blo = lo0 - 1e-12 * span, bhi = hi0 + 1e-12 * span;
    // thread t probes lo + (t + 1) (hi - lo) / 129; the bracket shrinks 129x per round.
    // Absolute accuracy 2e-16 ||T|| is what the selection and the singular values need.
    // Rounds also stop once the bracket is within two ulps of its end points: for the
    // largest eigenvalues 2e-16 ||T|| is below one ulp, and further rounds cannot narrow
    // the bracket.
    const int j = m - 1 - kk;                 // ascending index of the kk-th largest
    for (int it = 0; it < 12 && bhi - blo > fmax(2e-16 * span, 0x1p-51 * fmax(fabs(blo), fabs(bhi))); ++it) {
        const double step = (bhi - blo) * (1.0 / (HV_THREADS + 1));
        const bool above = sturm_count(d, e2, m, blo + step * (tid + 1)) > j;   // eigenvalue below x
        const unsigned mask = __ballot_sync(0xffffffffu, above);
        if (lane == 0) s_mask[warp] = mask;
        __syncthreads();
        int first = HV_THREADS;
        for (int w = HV_THREADS / 32 - 1; w >= 0; --w)
            if (s_mask[w]) first = w * 32 + __ffs(s_mask[w]) - 1;
        __syncthreads();
        const double nlo = blo + step * first;
        const double nhi = first < HV_THREADS ? blo + step * (first + 1) : bhi;
        blo = nlo;
        bhi = nhi;
    }
    const double l = 0.5 * (blo + bhi);
    if (tid == 0) lamp[blockIdx.y][kk] = l;
    if (kk >= r || warp != 0) return;
    if (lane == 0) {
        const double mu = l + 1e-14 * fmax(fabs(l), span * 1e-3);
        for (int i = 0; i < m; ++i) {
            dg[i] = d[i] - mu;
            up[i] = i + 1 < m ? eb[i] : 0.0;
            up2[i] = 0.0;
            y[i] = 1.0 + 1e-3 * i;
        }
        for (int i = 0; i + 1 < m; ++i) {
            const double sub = eb[i];
            if (fabs(dg[i]) >= fabs(sub)) {
                sw[i] = false;
                const double f = dg[i] != 0.0 ? sub * __drcp_rn(dg[i]) : 0.0;
                lo[i] = f;
                dg[i + 1] -= f * up[i];
            } else {
                sw[i] = true;
                const double f = dg[i] * __drcp_rn(sub);
                dg[i] = sub;
                lo[i] = f;
                const double t = up[i];
                up[i] = dg[i + 1];
                dg[i + 1] = t - f * dg[i + 1];
                if (i + 2 < m) {
                    up2[i] = up[i + 1];
                    up[i + 1] = -f * up[i + 1];
                }
            }
        }
        for (int i = 0; i < m; ++i) dg[i] = __drcp_rn(fabs(dg[i]) < 1e-300 ? 1e-300 : dg[i]);   // reciprocals
        for (int it = 0; it < 2; ++it) {
            for (int i = 0; i + 1 < m; ++i) {
                if (!sw[i]) y[i + 1] -= lo[i] * y[i];
                else { const double t = y[i]; y[i] = y[i + 1]; y[i + 1] = t - lo[i] * y[i]; }
            }
            y[m - 1] *= dg[m - 1];
            if (m > 1) y[m - 2] = (y[m - 2] - up[m - 2] * y[m - 1]) * dg[m - 2];
            for (int i = m - 3; i >= 0; --i) y[i] = (y[i] - up[i] * y[i + 1] - up2[i] * y[i + 2]) * dg[i];
            double nr = 0.0;
            for (int i = 0; i < m; ++i) nr += y[i] * y[i];
            nr = nr > 0.0 ? rsqrt(nr) : 1.0;
            for (int i = 0; i < m; ++i) y[i] *= nr;
        }
    }
    __syncwarp();
    for (int i = lane; i < m; i += 32) u[i] = y[i] * delta[i];
    __syncwarp();
    // u = Q D y with Q = H_0 ... H_{m-3}: reflectors applied in reverse
    for (int k = m - 3; k >= 0; --k) {
        const int n = m - k - 1;
        const c128* v = Vr + (size_t)k * m;
        c128 s = {0.0, 0.0};
        for (int i = lane; i < n; i += 32) cfma_cj(s, v[i], u[k + 1 + i]);
        s = tau[k] * warp_sum(s);
        __syncwarp();
        for (int i = lane; i < n; i += 32) u[k + 1 + i] = u[k + 1 + i] - v[i] * s;
        __syncwarp();
    }
    c128* U = Up[blockIdx.y];
    for (int i = lane; i < m; i += 32) U[(size_t)i * m + kk] = u[i];
}

void launch_heig(c128* const* G, c128* const* U, double* const* lam, int nq, int m, int r, void** scratch,
                 cudaStream_t s) {
    void* hp[3 * 64];
    for (int i = 0; i < nq; ++i) { hp[i] = G[i]; hp[nq + i] = U[i]; hp[2 * nq + i] = lam[i]; }
    cudaMemcpyAsync(scratch, hp, sizeof(void*) * 3 * nq, cudaMemcpyHostToDevice, s);
    const size_t sm = sizeof(c128) * (2 * (size_t)m * m + m) + sizeof(double) * 4 * m + sizeof(c128) * 5 * m + 64;
    static std::atomic<unsigned long long> attr{0};
    smem_limit_once(attr, k_heig_tri, 200 * 1024);
    k_heig_tri<<<nq, 256, sm, s>>>((c128* const*)scratch, m);
    note_launch();
    k_heig_vec<<<dim3(m, nq), HV_THREADS, 0, s>>>((c128* const*)scratch, (c128* const*)(scratch + nq),
                                          (double* const*)(scratch + 2 * nq), m, r);
    note_launch();
}

// V[x][j] = sum_k Z[x][k] U[k][j] / sqrt(lam_j), in FP64.  Eight threads per output,
// each adding every eighth term, then a fixed shuffle tree (the FP64 products spread over
// the SMs); the r scales 1 / sqrt(lam_j) formed once per block.
template <typename T>
__global__ void k_form_v(const cplx<T>* __restrict__ Z, const c128* __restrict__ U, const double* lam,
                         cplx<T>* __restrict__ V, int Sx, int m, int r) {
    __shared__ double sc[64];
    for (int j = threadIdx.x; j < r && j < 64; j += blockDim.x) {
        const double l = lam[j];
        sc[j] = l > 0.0 ? 1.0 / sqrt(l) : 0.0;
    }
    __syncthreads();
    const unsigned total = (unsigned)Sx * (unsigned)r;
    const unsigned t = (blockIdx.x * blockDim.x + threadIdx.x) >> 3;
    const int sub = threadIdx.x & 7;
    const bool ok = t < total;
    c128 a = {0.0, 0.0};
    unsigned x = 0;
    int j = 0;
    if (ok) {
        x = t / (unsigned)r;
        j = (int)(t - x * (unsigned)r);
        for (int k = sub; k < m; k += 8) cfma(a, cvt<double>(Z[(size_t)x * m + k]), U[k * m + j]);
    }
    for (int d = 4; d > 0; d >>= 1) {
        a.re += __shfl_xor_sync(0xffffffffu, a.re, d);
        a.im += __shfl_xor_sync(0xffffffffu, a.im, d);
    }
    if (ok && sub == 0) V[t] = cvt<T>(sc[j] * a);
}
template <typename T>
void launch_form_v(const cplx<T>* Z, const c128* U, const double* lam, cplx<T>* V, int Sx, int m, int r,
                   cudaStream_t s) {
    const size_t total = (size_t)Sx * r;   // r <= 64 (the basis width)
    const int grid = (int)((8 * total + 255) / 256);
    k_form_v<T><<<grid, 256, 0, s>>>(Z, U, lam, V, Sx, m, r);
    note_launch();
}

// ------------------------------------------------------- Gauss-Jordan (FP64)
// In-place inverse with partial pivoting: row interchanges during elimination, the
// inverse's columns unscrambled in reverse order at the end.
// One block per matrix, in arithmetic R: FP64, or FP32 for the opt-in FP32 coarse variant
// of the complex64 form.  The pivot's reciprocal is formed once per step (thread 0) and
// shared.  The inverse is written back to A in complex128 and, where AT is given, in
// complex64.  Matrices of 16 to 64 rows take the cluster form below.
template <typename R>
__global__ void __launch_bounds__(256) k_gj_inverse(GjBatch bt) {
    using C = cplx<R>;
    extern __shared__ __align__(16) unsigned char gjs[];
    c128* A = bt.A[blockIdx.x];
    const int n = bt.n;
    C* M = (C*)gjs;
    C* col = M + n * n;
    C* row = col + n;
    int* perm = (int*)(row + n);
    __shared__ int piv;
    __shared__ C pv, akk, s_ip;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) M[e] = cvt<R>(A[e]);
    __syncthreads();
    for (int k = 0; k < n; ++k) {
        if (threadIdx.x < 32) {
            R best = -1;
            int bi = k;
            for (int r = k + threadIdx.x; r < n; r += 32) {
                const R a = abs2(M[r * n + k]);
                if (a > best) { best = a; bi = r; }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const R ob = __shfl_xor_sync(0xffffffffu, best, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
            }
            if (threadIdx.x == 0) {
                piv = bi;
                perm[k] = bi;
                C pk = M[bi * n + k];
                akk = M[k * n + k];
                if (!(best > 0) || !isfinite(best)) {
                    atomicExch(bt.err, DEV_BREAKDOWN);
                    pk = C{1, 0};
                }
                pv = pk;
                s_ip = cinv(pk);
            }
        }
        __syncthreads();
        const int p = piv;
        const C ip = s_ip;
        for (int t = threadIdx.x; t < n; t += blockDim.x) {
            col[t] = (t == k) ? pv : (t == p ? akk : M[t * n + k]);
            const C rp = M[p * n + t];
            if (p != k) { M[p * n + t] = M[k * n + t]; M[k * n + t] = rp; }
            row[t] = rp * ip;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
            const int r = e / n, c = e - r * n;
            if (r == k) {
                M[e] = (c == k) ? ip : row[c];
            } else {
                const C f = col[r];
                M[e] = (c == k) ? -(f * ip) : M[e] - f * row[c];
            }
        }
        __syncthreads();
    }
    // unscramble columns: position c holds original column pos[c]
    if (threadIdx.x == 0) {
        int* pos = perm + n;
        for (int c = 0; c < n; ++c) pos[c] = c;
        for (int k = n - 1; k >= 0; --k) {
            const int t = pos[k]; pos[k] = pos[perm[k]]; pos[perm[k]] = t;
        }
    }
    __syncthreads();
    const int* pos = perm + n;
    c64* AT = (c64*)bt.AT[blockIdx.x];
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const int r = e / n, c = e - r * n;
        const C v = M[r * n + pos[c]];
        A[e] = cvt<double>(v);
        if (AT) AT[e] = cvt<float>(v);
    }
}
// The same elimination on a cluster of GJ_CL CTAs per matrix, each holding a slice of the
// rows: per step every CTA proposes its best pivot row (cluster barrier), all take the
// same pivot from the proposals (largest magnitude, then lowest row), read the pivot row
// (and the owner of the pivot row, the old row k) from distributed shared memory, and
// after a second barrier update their own rows.  The FP64 updates of a step spread over
// GJ_CL SMs (FP64 issues at 2 multiply-adds per SM and clock on this GPU).
static constexpr int GJ_CL = 8;
template <typename R>
__global__ void __launch_bounds__(256) k_gj_cluster(GjBatch bt) {
    namespace cg = cooperative_groups;
    using C = cplx<R>;
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int mat = blockIdx.x / GJ_CL;
    c128* A = bt.A[mat];
    const int n = bt.n;
    const int rpc = (n + GJ_CL - 1) / GJ_CL;
    const int r0 = min(n, rank * rpc), r1 = min(n, r0 + rpc), nr = r1 - r0;
    extern __shared__ __align__(16) unsigned char gjc[];
    C* M = (C*)gjc;                 // [rpc][n] own rows
    C* row = M + rpc * n;           // [n] the normalised pivot row
    C* tmp = row + n;               // [n] the old row k (the pivot row's owner)
    C* colk = tmp + n;              // [rpc] column k of the own rows, before the step
    int* perm = (int*)(colk + rpc); // [n]
    int* pos = perm + n;            // [n]
    __shared__ R s_best;
    __shared__ int s_idx, s_p;
    __shared__ C s_ip, s_akk;
    for (int e = threadIdx.x; e < nr * n; e += blockDim.x) M[e] = cvt<R>(A[(size_t)r0 * n + e]);
    __syncthreads();
    for (int k = 0; k < n; ++k) {
        if (threadIdx.x == 0) {
            R best = -1;
            int bi = n;
            for (int r = max(k, r0); r < r1; ++r) {
                const R a = abs2(M[(r - r0) * n + k]);
                if (a > best) { best = a; bi = r; }
            }
            s_best = best;
            s_idx = bi;
        }
        cluster.sync();
        if (threadIdx.x == 0) {
            R best = -1;
            int bi = n;
            for (int q = 0; q < GJ_CL; ++q) {
                const R ob = *cluster.map_shared_rank(&s_best, q);
                const int oi = *cluster.map_shared_rank(&s_idx, q);
                if (oi < n && (ob > best || (ob == best && oi < bi))) { best = ob; bi = oi; }
            }
            s_p = bi < n ? bi : k;
            perm[k] = s_p;
            const int ok_ = (bi < n) && (best > 0) && isfinite(best);
            if (!ok_ && rank == 0) atomicExch(bt.err, DEV_BREAKDOWN);
            const int ob = s_p / rpc, ok2 = k / rpc;
            const C pk = ok_ ? cluster.map_shared_rank(M, ob)[(s_p - ob * rpc) * n + k] : C{1, 0};
            s_ip = cinv(pk);
            s_akk = cluster.map_shared_rank(M, ok2)[(k - ok2 * rpc) * n + k];
        }
        __syncthreads();
        const int p = s_p;
        const C ip = s_ip;
        {
            const int ob = p / rpc, okk = k / rpc;
            const C* prow = cluster.map_shared_rank(M, ob) + (size_t)(p - ob * rpc) * n;
            for (int c = threadIdx.x; c < n; c += blockDim.x) row[c] = prow[c] * ip;
            if (p != k && p >= r0 && p < r1) {
                const C* krow = cluster.map_shared_rank(M, okk) + (size_t)(k - okk * rpc) * n;
                for (int c = threadIdx.x; c < n; c += blockDim.x) tmp[c] = krow[c];
            }
            for (int rl = threadIdx.x; rl < nr; rl += blockDim.x) colk[rl] = M[rl * n + k];
        }
        cluster.sync();   // every read of another CTA's rows is done before the updates
        const C akk = s_akk;
        for (int e = threadIdx.x; e < nr * n; e += blockDim.x) {
            const int rl = e / n, c = e - rl * n, r = r0 + rl;
            C v;
            if (r == k) {
                v = (c == k) ? ip : row[c];
            } else {
                const C f = (r == p) ? akk : colk[rl];
                const C cur = (r == p) ? tmp[c] : M[e];
                v = (c == k) ? -(f * ip) : cur - f * row[c];
            }
            M[e] = v;
        }
        __syncthreads();
    }
    // unscramble columns: position c holds original column pos[c]
    if (threadIdx.x == 0) {
        for (int c = 0; c < n; ++c) pos[c] = c;
        for (int k = n - 1; k >= 0; --k) {
            const int t = pos[k]; pos[k] = pos[perm[k]]; pos[perm[k]] = t;
        }
    }
    __syncthreads();
    c64* AT = (c64*)bt.AT[mat];
    for (int e = threadIdx.x; e < nr * n; e += blockDim.x) {
        const int rl = e / n, c = e - rl * n;
        const C v = M[rl * n + pos[c]];
        A[(size_t)(r0 + rl) * n + c] = cvt<double>(v);
        if (AT) AT[(size_t)(r0 + rl) * n + c] = cvt<float>(v);
    }
}

void launch_gj_inverse(const GjBatch& bt, int count, bool fp32, cudaStream_t s) {
    if (count < 1) return;
    if (bt.n >= 16 && bt.n <= 64) {
        const int n = bt.n, rpc = (n + GJ_CL - 1) / GJ_CL;
        const size_t es = fp32 ? sizeof(c64) : sizeof(c128);
        const size_t sm = es * ((size_t)rpc * n + 2 * n + rpc) + sizeof(int) * 2 * n;
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[1];
        cfg.gridDim = dim3(count * GJ_CL);
        cfg.blockDim = dim3(256);
        cfg.dynamicSmemBytes = sm;
        cfg.stream = s;
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = GJ_CL;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        if (fp32) cudaLaunchKernelEx(&cfg, k_gj_cluster<float>, bt);
        else cudaLaunchKernelEx(&cfg, k_gj_cluster<double>, bt);
        note_launch();
        return;
    }
    const int n = bt.n;
    const size_t es = fp32 ? sizeof(c64) : sizeof(c128);
    const size_t sm = es * (n * n + 2 * n) + sizeof(int) * 2 * n;
    static std::atomic<unsigned long long> attr64{0}, attr32{0};
    smem_limit_once(attr64, k_gj_inverse<double>, 200 * 1024);
    smem_limit_once(attr32, k_gj_inverse<float>, 200 * 1024);
    if (fp32) k_gj_inverse<float><<<count, 256, sm, s>>>(bt);
    else k_gj_inverse<double><<<count, 256, sm, s>>>(bt);
    note_launch();
}

// ------------------------------------------------------------ instantiations
template int launch_ip_partial<float, float, float>(const c64*, int, const c64*, int, size_t, int, int, c128*, int,
                                                    cudaStream_t);
template int launch_ip_partial<float, float, double>(const c64*, int, const c64*, int, size_t, int, int, c128*,
                                                     int, cudaStream_t);
template int launch_ip_partial<double, double, double>(const c128*, int, const c128*, int, size_t, int, int, c128*,
                                                       int, cudaStream_t);
template int launch_ip_partial<float, double, float>(const c64*, int, const c128*, int, size_t, int, int, c128*,
                                                     int, cudaStream_t);
template int launch_ip_partial<float, double, double>(const c64*, int, const c128*, int, size_t, int, int, c128*,
                                                      int, cudaStream_t);
template int launch_ip_partial_colA<float, float, float>(const c64*, const c64*, int, size_t, int, int, c128*, int,
                                                        cudaStream_t, long long);
template int launch_ip_partial_colA<double, double, double>(const c128*, const c128*, int, size_t, int, int, c128*,
                                                            int, cudaStream_t, long long);
template int launch_galerkin_partial<float, float>(const c64*, OpGeom, int, int, c128*, int, cudaStream_t, bool*);
template int launch_galerkin_partial<float, double>(const c64*, OpGeom, int, int, c128*, int, cudaStream_t, bool*);
template int launch_galerkin_partial<double, double>(const c128*, OpGeom, int, int, c128*, int, cudaStream_t, bool*);
template void launch_qr<float>(c64* const*, int, int, int, c64**, cudaStream_t);
template void launch_qr<double>(c128* const*, int, int, int, c128**, cudaStream_t);
template void launch_form_v<float>(const c64*, const c128*, const double*, c64*, int, int, int, cudaStream_t);
template void launch_form_v<double>(const c128*, const c128*, const double*, c128*, int, int, int, cudaStream_t);

}  // namespace hh
