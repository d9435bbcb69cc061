// k_dense.cu -- small dense steps of the set-up and the coarse solve:
//  * tall-skinny inner products A^H B in FP64 (coarse projection C^H r of Eq. (3), the
//    Gram matrix of the sketch);
//  * the Galerkin product A_c = C^H A~ C (Sec. 1) fused with the 5-point operator;
//  * orthonormalisation of the sketch Y = T Omega (Sec. 2, randomised SVD);
//  * the small SVD: Hermitian Jacobi on Z^H Z in FP64 and V = Z U Sigma^{-1};
//  * Gauss-Jordan inversion with partial pivoting of A_c (FP64).
#include "kernels.h"

namespace hh {

static constexpr int IP_TILE = 32;
static constexpr int IP_THREADS = 256;
static constexpr int IP_MAXOUT = 16;   // outputs per thread when p*q >= IP_THREADS

// Accumulate conj(As[n][i]) * Bs[n][j] over a tile of `rows` rows held in shared memory.
// Rows i outside [ilo, ihi) contribute nothing for this tile (ihi = 0: no restriction).
template <typename ACC>
__device__ __forceinline__ void ip_tile_accumulate(const cplx<ACC>* As, const cplx<ACC>* Bs, int rows, int p, int q,
                                                   int split, cplx<ACC>* acc, int ilo, int ihi) {
    const int nout = p * q;
    if (split == 1) {
        int k = 0;
        for (int o = threadIdx.x; o < nout; o += IP_THREADS, ++k) {
            const int i = o / q, j = o % q;
            if (ihi > 0 && (i < ilo || i >= ihi)) continue;
            cplx<ACC> a = acc[k];
            for (int n = 0; n < rows; ++n) cfma_cj(a, As[n * p + i], Bs[n * q + j]);
            acc[k] = a;
        }
    } else {
        const int s = threadIdx.x / nout, o = threadIdx.x % nout;
        if (s < split) {
            const int i = o / q, j = o % q;
            if (ihi > 0 && (i < ilo || i >= ihi)) return;
            cplx<ACC> a = acc[0];
            for (int n = s; n < rows; n += split) cfma_cj(a, As[n * p + i], Bs[n * q + j]);
            acc[0] = a;
        }
    }
}

template <typename ACC>
__device__ __forceinline__ void ip_store_partial(cplx<ACC>* acc, int p, int q, int split, cplx<ACC>* red,
                                                 c128* out) {
    const int nout = p * q;
    if (split == 1) {
        int k = 0;
        for (int o = threadIdx.x; o < nout; o += IP_THREADS, ++k) out[o] = cvt<double>(acc[k]);
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

template <typename TA, typename TB, typename ACC>
__global__ void __launch_bounds__(IP_THREADS) k_ip_partial(const cplx<TA>* __restrict__ A, int lda,
                                                           const cplx<TB>* __restrict__ B, int ldb,
                                                           size_t N, int p, int q, c128* partial) {
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
        for (int e = threadIdx.x; e < rows * p; e += IP_THREADS)
            As[e] = cvt<ACC>(A[(t0 + e / p) * lda + e % p]);
        for (int e = threadIdx.x; e < rows * q; e += IP_THREADS)
            Bs[e] = cvt<ACC>(B[(t0 + e / q) * ldb + e % q]);
        __syncthreads();
        ip_tile_accumulate<ACC>(As, Bs, rows, p, q, split, acc, 0, 0);
        __syncthreads();
    }
    ip_store_partial<ACC>(acc, p, q, split, red, partial + (size_t)blockIdx.x * nout);
}

static size_t ip_smem(int p, int q, size_t esz = sizeof(c128)) {
    const int nout = p * q;
    const int split = nout >= IP_THREADS ? 1 : IP_THREADS / nout;
    return esz * ((size_t)IP_TILE * (p + q) + (split > 1 ? (size_t)split * nout : 0));
}

template <typename TA, typename TB, typename ACC>
int launch_ip_partial(const cplx<TA>* A, int lda, const cplx<TB>* B, int ldb, size_t N, int p, int q,
                      c128* partial, int max_blocks, cudaStream_t s) {
    // rows per block: enough work per block to amortise the reduction over blocks
    const size_t per = (size_t)p * q >= 256 ? 256 : 1024;
    int grid = (int)((N + per - 1) / per);
    if (grid > max_blocks) grid = max_blocks;
    if (grid < 1) grid = 1;
    const size_t sm = ip_smem(p, q, sizeof(cplx<ACC>));
    static bool attr_set = false;  // per instantiation
    if (!attr_set) {
        cudaFuncSetAttribute(k_ip_partial<TA, TB, ACC>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        attr_set = true;
    }
    k_ip_partial<TA, TB, ACC><<<grid, IP_THREADS, sm, s>>>(A, lda, B, ldb, N, p, q, partial);
    note_launch();
    return grid;
}

// out = sum over blocks (one warp per output, lanes across blocks: fixed order, so
// deterministic); optional out2 = Minv * out computed by the same (single) block.
__global__ void __launch_bounds__(1024) k_ip_reduce(const c128* __restrict__ partial, int nblk, int p, int q,
                                                    c128* out, const c128* __restrict__ Minv, c128* out2) {
    extern __shared__ c128 s_out[];
    const int nout = p * q;
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int o = blockIdx.x * nw + (threadIdx.x >> 5); o < nout; o += gridDim.x * nw) {
        c128 t = {0.0, 0.0};
        for (int b = lane; b < nblk; b += 32) t = t + partial[(size_t)b * nout + o];
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
        for (int k = 0; k < p; ++k) cfma(t, Minv[i * p + k], s_out[k * q + j]);
        out2[o] = t;
    }
}
void launch_ip_reduce(const c128* partial, int nblk, int p, int q, c128* out, const c128* Minv, c128* out2,
                      cudaStream_t s) {
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_ip_reduce, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        attr = true;
    }
    const int nout = p * q;
    if (Minv) {
        k_ip_reduce<<<1, 1024, sizeof(c128) * nout, s>>>(partial, nblk, p, q, out, Minv, out2);
    } else {
        int grid = (nout + 7) / 8;
        if (grid > 304) grid = 304;
        k_ip_reduce<<<grid, 256, 0, s>>>(partial, nblk, p, q, out, nullptr, nullptr);
    }
    note_launch();
}

// ------------------------------------------------------------------- Galerkin
// partial[blk][a][l] = sum over the block's points of conj(C[pt][a]) * (A~ C)[pt][l].
template <typename T>
__global__ void __launch_bounds__(IP_THREADS) k_galerkin_partial(const cplx<T>* __restrict__ C, OpGeom g, int p,
                                                                 int split_row, c128* partial) {
    extern __shared__ c128 sm[];
    c128* As = sm;
    c128* Bs = As + IP_TILE * p;
    c128* red = Bs + IP_TILE * p;
    const int nout = p * p;
    const int split = nout >= IP_THREADS ? 1 : IP_THREADS / nout;
    c128 acc[IP_MAXOUT];
    for (int k = 0; k < IP_MAXOUT; ++k) acc[k] = {0.0, 0.0};
    const size_t N = (size_t)g.b * g.Sx;
    const size_t ldr = (size_t)g.Sx * p;
    const size_t chunk = (N + gridDim.x - 1) / gridDim.x;
    const size_t n0 = blockIdx.x * chunk, n1 = min(N, n0 + chunk);
    for (size_t t0 = n0; t0 < n1; t0 += IP_TILE) {
        const int rows = (int)min((size_t)IP_TILE, n1 - t0);
        for (int e = threadIdx.x; e < rows * p; e += IP_THREADS) {
            const size_t pt = t0 + e / p;
            const int l = e % p;
            const int i = (int)(pt % g.Sx), j = (int)(pt / g.Sx);
            const size_t t = pt * p + l;
            const c128 cv = cvt<double>(C[t]);
            c128 ax = op_diag(j, i, g) * cv;
            const double wj = wrow(j, g.b), wi = wcol(i, g.Sx);
            if (g.Sx > 1) {
                if (i > 0) ax = ax - wj * cvt<double>(C[t - p]);
                if (i < g.Sx - 1) ax = ax - wj * cvt<double>(C[t + p]);
            }
            if (j > 0) ax = ax - wi * cvt<double>(C[t - ldr]);
            if (j < g.b - 1) ax = ax - wi * cvt<double>(C[t + ldr]);
            As[e] = cv;
            Bs[e] = ax;
        }
        __syncthreads();
        // C's columns [0, p/2) live on rows < split_row, [p/2, p) on the others; a tile
        // inside one row touches one block of conj(C)
        int ilo = 0, ihi = 0;
        if (split_row >= 0) {
            const int j0 = (int)(t0 / g.Sx), j1 = (int)((t0 + rows - 1) / g.Sx);
            if (j1 < split_row) { ilo = 0; ihi = p / 2; }
            else if (j0 >= split_row) { ilo = p / 2; ihi = p; }
        }
        ip_tile_accumulate<double>(As, Bs, rows, p, p, split, acc, ilo, ihi);
        __syncthreads();
    }
    ip_store_partial<double>(acc, p, p, split, red, partial + (size_t)blockIdx.x * nout);
}

template <typename T>
int launch_galerkin_partial(const cplx<T>* C, OpGeom g, int p, int split_row, c128* partial, int max_blocks,
                            cudaStream_t s) {
    const size_t N = (size_t)g.b * g.Sx;
    int grid = (int)((N + 127) / 128);
    if (grid > max_blocks) grid = max_blocks;
    if (grid < 1) grid = 1;
    const size_t sm = ip_smem(p, p);
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(k_galerkin_partial<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        attr_set = true;
    }
    k_galerkin_partial<T><<<grid, IP_THREADS, sm, s>>>(C, g, p, split_row, partial);
    note_launch();
    return grid;
}

// ------------------------------------------------------------------------ QR
// Classical Gram-Schmidt applied twice per column (orthogonal to working precision
// for full-rank input); column j of Y becomes q_j with r_jj > 0 real.  One CTA per
// block; the block stays in global memory (L2).
template <typename T>
__global__ void __launch_bounds__(512) k_qr(cplx<T>* const* Yp, int Sx, int m) {
    cplx<T>* Y = Yp[blockIdx.x];
    __shared__ cplx<T> dots[128];
    __shared__ T red[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int j = 0; j < m; ++j) {
        for (int pass = 0; pass < 2 && j > 0; ++pass) {
            for (int k = warp; k < j; k += nw) {
                cplx<T> a = {0, 0};
                for (int x = lane; x < Sx; x += 32) cfma_cj(a, Y[(size_t)x * m + k], Y[(size_t)x * m + j]);
                a = warp_sum(a);
                if (lane == 0) dots[k] = a;
            }
            __syncthreads();
            for (int x = threadIdx.x; x < Sx; x += blockDim.x) {
                cplx<T> v = Y[(size_t)x * m + j];
                for (int k = 0; k < j; ++k) v = v - Y[(size_t)x * m + k] * dots[k];
                Y[(size_t)x * m + j] = v;
            }
            __syncthreads();
        }
        T a2 = 0;
        for (int x = threadIdx.x; x < Sx; x += blockDim.x) a2 += abs2(Y[(size_t)x * m + j]);
        a2 = warp_sum(a2);
        if (lane == 0) red[warp] = a2;
        __syncthreads();
        if (warp == 0) {
            T v = lane < nw ? red[lane] : (T)0;
            v = warp_sum(v);
            if (lane == 0) red[0] = v;
        }
        __syncthreads();
        const T nrm = sqrt(red[0]);
        const T inv = nrm > (T)0 ? (T)1 / nrm : (T)0;
        for (int x = threadIdx.x; x < Sx; x += blockDim.x) Y[(size_t)x * m + j] = inv * Y[(size_t)x * m + j];
        __syncthreads();
    }
}
template <typename T>
void launch_qr(cplx<T>* const* Y, int nq, int Sx, int m, cplx<T>** dev_ptr_scratch, cudaStream_t s) {
    cudaMemcpyAsync(dev_ptr_scratch, Y, sizeof(cplx<T>*) * nq, cudaMemcpyHostToDevice, s);
    k_qr<T><<<nq, 512, 0, s>>>(dev_ptr_scratch, Sx, m);
    note_launch();
}

// -------------------------------------------------------------- Jacobi (FP64)
// Cyclic Jacobi with round-robin ordering: each round applies m/2 disjoint unitary
// plane rotations J = diag(1, e^{-i phi}) * [[c, s], [-s, c]] that annihilate G[p][q].
__device__ __forceinline__ int rr_index(int i, int round, int n) {
    return i == 0 ? 0 : 1 + (i - 1 + round) % (n - 1);
}

__global__ void __launch_bounds__(256) k_jacobi(c128* const* Gp, c128* const* Up, double* const* lamp, int m) {
    extern __shared__ c128 sj[];
    const int n = m + (m & 1);          // padded to even
    c128* G = sj;                       // m x m
    c128* U = G + m * m;                // m x m
    double* rot = (double*)(U + m * m); // per pair: c, s, cos(phi), sin(phi)
    int* pq = (int*)(rot + 4 * (n / 2));
    __shared__ double off_s, diag_s;
    c128* Gg = Gp[blockIdx.x];
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
        G[e] = Gg[e];
        U[e] = c128{(e / m == e % m) ? 1.0 : 0.0, 0.0};
    }
    __syncthreads();
    const int npair = n / 2;
    for (int sweep = 0; sweep < 40; ++sweep) {
        // convergence test on the off-diagonal mass
        if (threadIdx.x == 0) { off_s = 0.0; diag_s = 0.0; }
        __syncthreads();
        double off = 0.0, dg = 0.0;
        for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
            if (e / m == e % m) dg += abs2(G[e]); else off += abs2(G[e]);
        }
        off = warp_sum(off);
        dg = warp_sum(dg);
        if ((threadIdx.x & 31) == 0) { atomicAdd(&off_s, off); atomicAdd(&diag_s, dg); }
        __syncthreads();
        if (off_s <= 1e-24 * diag_s || off_s == 0.0) break;   // off-diagonal <= 1e-12 relative
        __syncthreads();
        for (int round = 0; round < n - 1; ++round) {
            if (threadIdx.x < npair) {
                const int k = threadIdx.x;
                int a = rr_index(k, round, n), b = rr_index(n - 1 - k, round, n);
                if (a > b) { int t = a; a = b; b = t; }
                pq[2 * k] = a;
                pq[2 * k + 1] = b;
                double c = 1.0, s = 0.0, cph = 1.0, sph = 0.0;
                if (b < m) {
                    const c128 g = G[a * m + b];
                    const double ag = sqrt(abs2(g));
                    const double app = G[a * m + a].re, aqq = G[b * m + b].re;
                    if (ag > 1e-300 && ag > 1e-18 * sqrt(fabs(app * aqq))) {
                        cph = g.re / ag;
                        sph = g.im / ag;
                        const double zeta = (aqq - app) / (2.0 * ag);
                        const double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                        c = 1.0 / sqrt(1.0 + t * t);
                        s = t * c;
                    }
                }
                rot[4 * k] = c; rot[4 * k + 1] = s; rot[4 * k + 2] = cph; rot[4 * k + 3] = sph;
            }
            __syncthreads();
            // columns: (G J) and (U J): col_p' = c col_p - s e^{-i phi} col_q ; col_q' = s col_p + c e^{-i phi} col_q
            for (int e = threadIdx.x; e < npair * m * 2; e += blockDim.x) {
                const int which = e / (npair * m);
                const int k = (e / m) % npair, r = e % m;
                const int a = pq[2 * k], b = pq[2 * k + 1];
                if (b >= m) continue;
                const double c = rot[4 * k], s = rot[4 * k + 1];
                const c128 em = {rot[4 * k + 2], -rot[4 * k + 3]};   // e^{-i phi}
                c128* X = which ? U : G;
                const c128 xp = X[r * m + a], xq = X[r * m + b];
                const c128 eq = em * xq;
                X[r * m + a] = c * xp - s * eq;
                X[r * m + b] = s * xp + c * eq;
            }
            __syncthreads();
            // rows: row_p' = c row_p - s e^{i phi} row_q ; row_q' = s row_p + c e^{i phi} row_q
            for (int e = threadIdx.x; e < npair * m; e += blockDim.x) {
                const int k = e / m, col = e % m;
                const int a = pq[2 * k], b = pq[2 * k + 1];
                if (b >= m) continue;
                const double c = rot[4 * k], s = rot[4 * k + 1];
                const c128 ep = {rot[4 * k + 2], rot[4 * k + 3]};
                const c128 xp = G[a * m + col], xq = G[b * m + col];
                const c128 eq = ep * xq;
                G[a * m + col] = c * xp - s * eq;
                G[b * m + col] = s * xp + c * eq;
            }
            __syncthreads();
        }
    }
    // sort eigenvalues descending (selection by one thread), permute U's columns
    int* perm = pq;
    if (threadIdx.x == 0) {
        for (int i = 0; i < m; ++i) perm[i] = i;
        for (int i = 0; i < m; ++i) {
            int best = i;
            for (int j = i + 1; j < m; ++j)
                if (G[perm[j] * m + perm[j]].re > G[perm[best] * m + perm[best]].re) best = j;
            int t = perm[i]; perm[i] = perm[best]; perm[best] = t;
        }
    }
    __syncthreads();
    double* lam = lamp[blockIdx.x];
    c128* Uo = Up[blockIdx.x];
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
        const int r = e / m, j = e % m;
        Uo[e] = U[r * m + perm[j]];
    }
    for (int j = threadIdx.x; j < m; j += blockDim.x) lam[j] = G[perm[j] * m + perm[j]].re;
}

void launch_jacobi(c128* const* G, c128* const* U, double* const* lam, int nq, int m, void** scratch,
                   cudaStream_t s) {
    // scratch holds 3*nq device pointers
    void* hp[3 * 64];
    for (int i = 0; i < nq; ++i) { hp[i] = G[i]; hp[nq + i] = U[i]; hp[2 * nq + i] = lam[i]; }
    cudaMemcpyAsync(scratch, hp, sizeof(void*) * 3 * nq, cudaMemcpyHostToDevice, s);
    const int n = m + (m & 1);
    const size_t sm = sizeof(c128) * 2 * m * m + sizeof(double) * 4 * (n / 2) + sizeof(int) * (n + 2);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_jacobi, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        attr = true;
    }
    k_jacobi<<<nq, 256, sm, s>>>((c128* const*)scratch, (c128* const*)(scratch + nq),
                                 (double* const*)(scratch + 2 * nq), m);
    note_launch();
}

// V[x][j] = sum_k Z[x][k] U[k][j] / sqrt(lam_j)
template <typename T>
__global__ void k_form_v(const cplx<T>* __restrict__ Z, const c128* __restrict__ U, const double* lam,
                         cplx<T>* __restrict__ V, int Sx, int m, int r) {
    const size_t total = (size_t)Sx * r;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(t % r);
        const size_t x = t / r;
        c128 a = {0.0, 0.0};
        for (int k = 0; k < m; ++k) cfma(a, cvt<double>(Z[x * m + k]), U[k * m + j]);
        const double l = lam[j];
        const double sc = l > 0.0 ? 1.0 / sqrt(l) : 0.0;
        V[t] = cvt<T>(sc * a);
    }
}
template <typename T>
void launch_form_v(const cplx<T>* Z, const c128* U, const double* lam, cplx<T>* V, int Sx, int m, int r,
                   cudaStream_t s) {
    const size_t total = (size_t)Sx * r;
    int grid = (int)((total + 255) / 256);
    k_form_v<T><<<grid, 256, 0, s>>>(Z, U, lam, V, Sx, m, r);
    note_launch();
}

// ------------------------------------------------------- Gauss-Jordan (FP64)
// In-place inverse with partial pivoting: row interchanges during elimination, the
// inverse's columns unscrambled in reverse order at the end.
__global__ void __launch_bounds__(256) k_gj_inverse(c128* A, int n, int* err) {
    extern __shared__ c128 sg[];
    c128* M = sg;
    c128* col = M + n * n;
    c128* row = col + n;
    int* perm = (int*)(row + n);
    __shared__ int piv;
    __shared__ c128 pv, akk;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) M[e] = A[e];
    __syncthreads();
    for (int k = 0; k < n; ++k) {
        if (threadIdx.x < 32) {
            double best = -1.0;
            int bi = k;
            for (int r = k + threadIdx.x; r < n; r += 32) {
                const double a = abs2(M[r * n + k]);
                if (a > best) { best = a; bi = r; }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const double ob = __shfl_xor_sync(0xffffffffu, best, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
            }
            if (threadIdx.x == 0) {
                piv = bi;
                perm[k] = bi;
                pv = M[bi * n + k];
                akk = M[k * n + k];
                if (!(best > 0.0) || !isfinite(best)) {
                    atomicExch(err, DEV_BREAKDOWN);
                    pv = c128{1.0, 0.0};
                }
            }
        }
        __syncthreads();
        const int p = piv;
        const c128 ip = cinv(pv);
        for (int t = threadIdx.x; t < n; t += blockDim.x) {
            col[t] = (t == k) ? pv : (t == p ? akk : M[t * n + k]);
            const c128 rp = M[p * n + t];
            if (p != k) { M[p * n + t] = M[k * n + t]; M[k * n + t] = rp; }
            row[t] = rp * ip;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
            const int r = e / n, c = e % n;
            if (r == k) {
                M[e] = (c == k) ? ip : row[c];
            } else {
                const c128 f = col[r];
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
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const int r = e / n, c = e % n;
        A[e] = M[r * n + pos[c]];
    }
}
void launch_gj_inverse(c128* A, int n, int* err, cudaStream_t s) {
    const size_t sm = sizeof(c128) * (n * n + 2 * n) + sizeof(int) * 2 * n;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_gj_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        attr = true;
    }
    k_gj_inverse<<<1, 256, sm, s>>>(A, n, err);
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
template int launch_galerkin_partial<float>(const c64*, OpGeom, int, int, c128*, int, cudaStream_t);
template int launch_galerkin_partial<double>(const c128*, OpGeom, int, int, c128*, int, cudaStream_t);
template void launch_qr<float>(c64* const*, int, int, int, c64**, cudaStream_t);
template void launch_qr<double>(c128* const*, int, int, int, c128**, cudaStream_t);
template void launch_form_v<float>(const c64*, const c128*, const double*, c64*, int, int, int, cudaStream_t);
template void launch_form_v<double>(const c128*, const c128*, const double*, c128*, int, int, int, cudaStream_t);

}  // namespace hh
