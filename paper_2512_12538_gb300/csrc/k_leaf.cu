// k_leaf.cu -- leaf subdomain solves A~_leaf^{-1} v (the subdomain solves of Eq. (2),
// the sketches and the basis extension of Sec. 2).
//
// 2D leaf = band of b rows x Sx columns.  Ordered column by column (block index i
// along x), A~_leaf is block tridiagonal with b x b blocks:
//     D_i  (tridiagonal: the y-coupling inside column i, plus the diagonal terms),
//     L_i = U_{i-1} = -W (W = diag of the row weights w_a: 1/2 on the band edges).
// Factorisation (Schur recursion): S_0 = D_0, S_i = D_i - W S_{i-1}^{-1} W; the kernel
// stores X_i = S_i^{-1} (dense, explicit inverse by Gauss-Jordan with partial pivoting).
// Solve: forward  y_0 = X_0 f_0,  y_i = X_i (f_i + W y_{i-1});
//        backward x_{n-1} = y_{n-1}, x_i = y_i + X_i W x_{i+1}.
// 1D leaf (Sx = 1): the same recursion with 1 x 1 blocks along the band's rows.
#include "kernels.h"

namespace hh {

int leaf_ldx(int b, int elem_bytes) {
    // every row of a stored X_i is a multiple of 16 bytes (bulk-copy granularity)
    const int per16 = 16 / elem_bytes;      // elements per 16 bytes: 2 (c64) or 1 (c128)
    return (b + per16 - 1) / per16 * per16;
}

static constexpr uint32_t WAIT_LIMIT = 1u << 21;   // bounded mbarrier polls (~0.1-0.3 s)
static constexpr int MAXP = 4;                       // row pieces per step in the sweep

// ------------------------------------------------------------- factorisation (2D)
template <typename T>
__device__ void gj_invert(cplx<T>* M, int ld, int b, cplx<T>* col, cplx<T>* row, int* perm, int* err) {
    __shared__ int s_piv;
    __shared__ cplx<T> s_pv, s_akk;
    for (int k = 0; k < b; ++k) {
        if (threadIdx.x < 32) {
            T best = (T)-1;
            int bi = k;
            for (int r = k + threadIdx.x; r < b; r += 32) {
                const T a = abs2(M[r * ld + k]);
                if (a > best) { best = a; bi = r; }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const T ob = __shfl_xor_sync(0xffffffffu, best, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
            }
            if (threadIdx.x == 0) {
                s_piv = bi;
                perm[k] = bi;
                s_pv = M[bi * ld + k];
                s_akk = M[k * ld + k];
                if (!(best > (T)0) || !isfinite(best)) {
                    atomicExch(err, DEV_BREAKDOWN);
                    s_pv = cplx<T>{(T)1, (T)0};
                }
            }
        }
        __syncthreads();
        const int p = s_piv;
        const cplx<T> pv = s_pv, ip = cinv(pv);
        for (int t = threadIdx.x; t < b; t += blockDim.x) {
            col[t] = (t == k) ? pv : (t == p ? s_akk : M[t * ld + k]);
            const cplx<T> rp = M[p * ld + t];
            if (p != k) { M[p * ld + t] = M[k * ld + t]; M[k * ld + t] = rp; }
            row[t] = rp * ip;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
            const int r = e / b, c = e - r * b;
            cplx<T>& m = M[r * ld + c];
            if (r == k) {
                m = (c == k) ? ip : row[c];
            } else {
                const cplx<T> f = col[r];
                m = (c == k) ? -(f * ip) : m - f * row[c];
            }
        }
        __syncthreads();
    }
    // unscramble columns in reverse pivot order; one thread per row, in place
    for (int r = threadIdx.x; r < b; r += blockDim.x) {
        for (int k = b - 1; k >= 0; --k) {
            const int p = perm[k];
            if (p != k) {
                const cplx<T> t = M[r * ld + k];
                M[r * ld + k] = M[r * ld + p];
                M[r * ld + p] = t;
            }
        }
    }
    __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(256) k_factor2d(const LeafTask* __restrict__ tasks, int Sx, double kh, int* err) {
    const LeafTask tk = tasks[blockIdx.x];
    const int b = tk.b, ldx = tk.ldx;
    cplx<T>* X = (cplx<T>*)tk.X;
    extern __shared__ __align__(16) unsigned char smf[];
    cplx<T>* M = (cplx<T>*)smf;      // b x b, leading dimension b
    cplx<T>* col = M + b * b;
    cplx<T>* row = col + b;
    int* perm = (int*)(row + b);
    const OpGeom g{b, Sx, kh, tk.khr};
    const size_t step = (size_t)b * ldx;
    for (int i = 0; i < Sx; ++i) {
        // S_i = D_i - W X_{i-1} W, built in place over X_{i-1}
        const T wi = (T)wcol(i, Sx);
        for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
            const int r = e / b, c = e - r * b;
            cplx<T> v = {0, 0};
            if (i > 0) v = (-(T)(wrow(r, b) * wrow(c, b))) * M[e];
            if (r == c) {
                const c128 d = op_diag(r, i, g);
                v = v + cplx<T>{(T)d.re, (T)d.im};
            } else if (r - c == 1 || c - r == 1) {
                v.re -= wi;
            }
            M[e] = v;
        }
        __syncthreads();
        gj_invert(M, b, b, col, row, perm, err);
        cplx<T>* Xi = X + (size_t)i * step;
        for (int e = threadIdx.x; e < b * ldx; e += blockDim.x) {
            const int r = e / ldx, c = e - r * ldx;
            Xi[e] = c < b ? M[r * b + c] : cplx<T>{0, 0};
        }
        // no barrier needed: each thread rebuilds exactly the elements it owns?  Not
        // guaranteed (different index maps), so synchronise.
        __syncthreads();
    }
}

// ---------------------------------------------------------- factorisation (1D)
template <typename T>
__global__ void k_factor1d(const LeafTask* __restrict__ tasks, int ntasks, double kh, int* err) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntasks) return;
    const LeafTask tk = tasks[t];
    cplx<T>* X = (cplx<T>*)tk.X;
    const OpGeom g{tk.b, 1, kh, tk.khr};
    cplx<double> prev_inv = {0.0, 0.0};
    for (int j = 0; j < tk.b; ++j) {
        // S_j = D_j - (-1) S_{j-1}^{-1} (-1)
        const c128 s = op_diag(j, 0, g) - prev_inv;
        if (!(abs2(s) > 0.0)) atomicExch(err, DEV_BREAKDOWN);
        prev_inv = cinv(s);
        X[j] = cvt<T>(prev_inv);
    }
}

// Tallest band whose b x b inverse and pivot workspace fit one block's shared memory
// (227 KiB) in k_factor2d: 119 rows in complex128, 169 in complex64.
int leaf_block_bmax(int elem_bytes) {
    const long long cap = 227 * 1024;
    int b = 1;
    while ((long long)elem_bytes * ((long long)(b + 1) * (b + 1) + 2 * (b + 1)) + 4ll * (b + 1) <= cap) ++b;
    return b;
}

template <typename T>
void launch_factor(const LeafTask* d_tasks, int ntasks, int b_max, int Sx, double kh, int* err, cudaStream_t s) {
    if (Sx == 1) {
        k_factor1d<T><<<(ntasks + 31) / 32, 32, 0, s>>>(d_tasks, ntasks, kh, err);
        note_launch();
        return;
    }
    const size_t sm = sizeof(cplx<T>) * ((size_t)b_max * b_max + 2 * b_max) + sizeof(int) * b_max;
    cudaFuncSetAttribute(k_factor2d<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_factor2d<T><<<ntasks, 256, sm, s>>>(d_tasks, Sx, kh, err);
    note_launch();
}

// ------------------------------------------------------------------ sweep (2D)
// One CTA per (leaf, chunk of NC right-hand sides).  X_i pieces (row blocks of a step's
// inverse) stream through a ring of shared-memory slots by 1D bulk copies (TMA engine)
// completing on mbarriers; the chain vector lives in shared memory.  G lanes split
// every row's dot product.
template <typename T, int NC, int G>
__global__ void k_sweep2d(const LeafTask* __restrict__ tasks, int Sx, int nrhs, int nslot, int prow,
                          size_t slot_elems, int* err) {
    const LeafTask tk = tasks[blockIdx.y];
    const int b = tk.b, ldx = tk.ldx;
    const int c0 = blockIdx.x * NC;
    if (c0 >= nrhs) return;
    const int ncol = min(NC, nrhs - c0);
    const cplx<T>* X = (const cplx<T>*)tk.X;
    const cplx<T>* F = (const cplx<T>*)tk.F;
    cplx<T>* W = (cplx<T>*)tk.W;
    const size_t ldrow = (size_t)Sx * nrhs;   // stride between rows of F / W
    const size_t step = (size_t)b * ldx;

    extern __shared__ __align__(128) unsigned char sms[];
    cplx<T>* slots = (cplx<T>*)sms;
    cplx<T>* vbuf = slots + (size_t)nslot * slot_elems;          // [2][b][NC]
    uint64_t* bars = (uint64_t*)(vbuf + 2 * (size_t)b * NC);
    __shared__ int s_abort;

    const int npiece = (b + prow - 1) / prow;
    const int nsteps = 2 * Sx - 1;
    const int total = nsteps * npiece;
    auto step_col = [&](int s) { return s < Sx ? s : 2 * Sx - 2 - s; };
    auto issue = [&](int q) {
        const int s = q / npiece, p = q - s * npiece;
        const int r0 = p * prow;
        const int rows = min(prow, b - r0);
        const uint32_t bytes = (uint32_t)(rows * ldx * sizeof(cplx<T>));
        const int slot = q % nslot;
        mbar_arrive_expect_tx(&bars[slot], bytes);
        bulk_g2s(slots + (size_t)slot * slot_elems, X + (size_t)step_col(s) * step + (size_t)r0 * ldx, bytes,
                 &bars[slot]);
    };

    if (threadIdx.x == 0) {
        s_abort = 0;
        for (int k = 0; k < nslot; ++k) mbar_init(&bars[k], 1);
        fence_barrier_init();
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int q = 0; q < nslot && q < total; ++q) issue(q);
    // v for the first forward step: f_0
    for (int e = threadIdx.x; e < b * NC; e += blockDim.x) {
        const int a = e / NC, c = e - a * NC;
        vbuf[e] = c < ncol ? F[a * ldrow + c0 + c] : cplx<T>{0, 0};
    }
    __syncthreads();

    const int lr = threadIdx.x / G, g = threadIdx.x - (threadIdx.x / G) * G;
    // Per-thread registers for the rows this thread finalises (g == 0): `cur` holds
    // y_i for the current backward step, `nxt` the data the next step needs (f_{i+1}
    // forward, y_{i-1} backward), loaded one step ahead to hide the memory latency.
    cplx<T> cur[MAXP][NC], nxt[MAXP][NC];
    for (int p = 0; p < MAXP; ++p)
        for (int c = 0; c < NC; ++c) cur[p][c] = nxt[p][c] = cplx<T>{0, 0};
    int q = 0;
    for (int s = 0; s < nsteps; ++s) {
        const int i = step_col(s);
        const bool fwd = s < Sx;
        const cplx<T>* v = vbuf + (size_t)(s & 1) * b * NC;
        cplx<T>* vn = vbuf + (size_t)((s + 1) & 1) * b * NC;
        if (g == 0 && s + 1 < nsteps) {
            const int i1 = step_col(s + 1);
            const cplx<T>* src = (s + 1 < Sx) ? F : W;     // y_{i1} was written by this thread
            for (int p = 0; p < npiece; ++p) {
                const int a = p * prow + lr;
                if (lr < prow && a < b)
                    for (int c = 0; c < NC; ++c)
                        if (c < ncol) nxt[p][c] = src[a * ldrow + (size_t)i1 * nrhs + c0 + c];
            }
        }
        for (int p = 0; p < npiece; ++p, ++q) {
            const int slot = q % nslot;
            if (!mbar_wait_bounded(&bars[slot], (uint32_t)((q / nslot) & 1), WAIT_LIMIT)) {
                atomicExch(err, DEV_TIMEOUT);
                s_abort = 1;
            }
            const int r0 = p * prow;
            const int rows = min(prow, b - r0);
            const cplx<T>* Xs = slots + (size_t)slot * slot_elems;
            cplx<T> acc[NC];
            for (int c = 0; c < NC; ++c) acc[c] = {0, 0};
            if (lr < rows) {
                const cplx<T>* xr = Xs + (size_t)lr * ldx;
                for (int k = g; k < b; k += G) {
                    const cplx<T> xv = xr[k];
                    for (int c = 0; c < NC; ++c) cfma(acc[c], xv, v[k * NC + c]);
                }
            }
            for (int o = G / 2; o > 0; o >>= 1)
                for (int c = 0; c < NC; ++c) {
                    acc[c].re += __shfl_xor_sync(0xffffffffu, acc[c].re, o);
                    acc[c].im += __shfl_xor_sync(0xffffffffu, acc[c].im, o);
                }
            if (g == 0 && lr < rows) {
                const int a = r0 + lr;
                const T wa = (T)wrow(a, b);
                for (int c = 0; c < NC; ++c) {
                    cplx<T> res = acc[c];
                    if (!fwd) res = res + cur[p][c];          // x_i = y_i + X_i W x_{i+1}
                    if (c < ncol) W[a * ldrow + (size_t)i * nrhs + c0 + c] = res;
                    cplx<T> nv = wa * res;                     // W y_i  or  W x_i
                    if (s + 1 < Sx) nv = nv + nxt[p][c];        // + f_{i+1}
                    vn[a * NC + c] = nv;
                }
            }
            __syncthreads();
            if (s_abort) break;
            if (threadIdx.x == 0 && q + nslot < total) issue(q + nslot);
        }
        if (s_abort) break;
        for (int p = 0; p < MAXP; ++p)
            for (int c = 0; c < NC; ++c) cur[p][c] = nxt[p][c];
    }
    if (s_abort && threadIdx.x == 0) {
        // drain copies still in flight before the CTA's shared memory is released
        for (int k = q; k < total && k < q + nslot; ++k)
            mbar_wait_bounded(&bars[k % nslot], (uint32_t)((k / nslot) & 1), WAIT_LIMIT);
    }
}

// --------------------------------------------------------------------- sweep (1D)
template <typename T>
__global__ void k_sweep1d(const LeafTask* __restrict__ tasks, int nrhs) {
    const LeafTask tk = tasks[blockIdx.y];
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nrhs) return;
    const cplx<T>* X = (const cplx<T>*)tk.X;
    const cplx<T>* F = (const cplx<T>*)tk.F;
    cplx<T>* W = (cplx<T>*)tk.W;
    cplx<T> y = {0, 0};
    for (int j = 0; j < tk.b; ++j) {
        y = X[j] * (F[(size_t)j * nrhs + c] + y);
        W[(size_t)j * nrhs + c] = y;
    }
    cplx<T> x = y;
    for (int j = tk.b - 2; j >= 0; --j) {
        x = W[(size_t)j * nrhs + c] + X[j] * x;
        W[(size_t)j * nrhs + c] = x;
    }
}

template <typename T, int NC, int G>
static void sweep_cfg(const LeafTask* d_tasks, int ntasks, int b_max, int Sx, int nrhs, int* err, cudaStream_t s) {
    const int esz = (int)sizeof(cplx<T>);
    const int ldx = leaf_ldx(b_max, esz);
    const size_t budget = 220 * 1024;
    const size_t vbytes = 2 * (size_t)b_max * NC * esz + 8 * 8 + 128;
    int prow = b_max < 1024 / G ? b_max : 1024 / G, nslot = 3;
    size_t slot_bytes = align_up((size_t)prow * ldx * esz, 128);
    while (nslot * slot_bytes + vbytes > budget && prow > 8) {
        prow = (prow + 1) / 2;
        slot_bytes = align_up((size_t)prow * ldx * esz, 128);
    }
    while ((nslot + 1) * slot_bytes + vbytes <= budget && nslot < 6) ++nslot;
    const size_t sm = nslot * slot_bytes + vbytes;
    if ((b_max + prow - 1) / prow > MAXP) {          // band too tall for this kernel
        int one = DEV_BADARG;
        cudaMemcpyAsync(err, &one, sizeof(int), cudaMemcpyHostToDevice, s);
        return;
    }
    int threads = ((prow * G + 31) / 32) * 32;
    if (threads > 1024) threads = 1024;
    cudaFuncSetAttribute(k_sweep2d<T, NC, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    dim3 grid((nrhs + NC - 1) / NC, ntasks);
    k_sweep2d<T, NC, G><<<grid, threads, sm, s>>>(d_tasks, Sx, nrhs, nslot, prow, slot_bytes / esz, err);
    note_launch();
}

template <typename T>
void launch_sweep(const LeafTask* d_tasks, int ntasks, int b_max, int Sx, int nrhs, int* err, cudaStream_t s) {
    if (Sx == 1) {
        dim3 grid((nrhs + 63) / 64, ntasks);
        k_sweep1d<T><<<grid, 64, 0, s>>>(d_tasks, nrhs);
        note_launch();
        return;
    }
    // prow * G threads must fit in one CTA; rows beyond are handled as further pieces
    if (nrhs == 1) sweep_cfg<T, 1, 8>(d_tasks, ntasks, b_max, Sx, nrhs, err, s);
    else sweep_cfg<T, 2, 8>(d_tasks, ntasks, b_max, Sx, nrhs, err, s);
}

template void launch_factor<float>(const LeafTask*, int, int, int, double, int*, cudaStream_t);
template void launch_factor<double>(const LeafTask*, int, int, int, double, int*, cudaStream_t);
template void launch_sweep<float>(const LeafTask*, int, int, int, int, int*, cudaStream_t);
template void launch_sweep<double>(const LeafTask*, int, int, int, int, int*, cudaStream_t);

}  // namespace hh
