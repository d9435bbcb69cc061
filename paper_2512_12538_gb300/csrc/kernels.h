// kernels.h -- host-side launchers of the libhh CUDA kernels (internal header).
#pragma once
#include <cuda_runtime.h>
#include "hh_core.cuh"

namespace hh {

// Counts kernel launches made by this library (process-wide); see hh_launch_count().
void note_launch();

// ---- field kernels (k_field.cu) ----------------------------------------------------
// y = (v ? v : 0) - sgn * A~ x  on a band (b rows, Sx cols, nc columns per point).
// With `v` null and sgn = -1 this is y = A~ x.  If `part` is non-null each block writes
// its partial sum of |y|^2 to part[blockIdx.x] (nblk_out receives the block count).
template <typename TX, typename TV, typename TY>
void launch_apply(const cplx<TX>* x, const cplx<TV>* v, cplx<TY>* y, OpGeom g, int nc, double sgn,
                  double* part, int* nblk_out, cudaStream_t s);

// y = v - A x (FP64, one column) with per-block |y|^2 partials, and yt = y rounded to T.
// gate (may be null): when the device word is nonzero at launch, nothing is done.
template <typename T>
void launch_residual_cast(const c128* x, const c128* v, c128* y, cplx<T>* yt, OpGeom g, double* part, int* nblk_out,
                          cudaStream_t s, const int* gate = nullptr);

// Residuals of up to RB_MAX_JOBS problems in one launch: per job y = v - A x (FP64) and
// yt = y in T; norms[k] = ||y_k||^2 (fixed-order sums).  part: scratch of part_cap doubles.
constexpr int RB_MAX_JOBS = 32;
struct ResidJob {
    const c128* x;
    const c128* v;
    c128* y;
    void* yt;
    OpGeom g;
    unsigned blk0, nblk;   // set by the launcher
    const int* gate;       // may be null: while the word is nonzero the job touches nothing
};
struct ResidBatch {
    ResidJob job[RB_MAX_JOBS];
    int njobs;
};
template <typename T>
void launch_residual_batch(ResidBatch bt, double* part, int part_cap, double* norms, cudaStream_t s);

// out = sum of n doubles (deterministic single-block reduction)
void launch_sum(const double* part, int n, double* out, cudaStream_t s);
// A~ applied to p column-major columns of a node's band: y[j N + pt] = (A~ x_j)[pt].
template <typename T>
void launch_apply_cols(const cplx<T>* x, cplx<T>* y, OpGeom g, int p, cudaStream_t s);

// launch_residual_cast with the stopping test of the stationary iteration kept on the
// device, in the same launch.  Unless ctl[0] is already set, or need is given and zero
// (then nothing is done); yt is written only when anchor is null or nonzero:
// y (may be null: not stored), yt and the partials as launch_residual_cast, then
// nrm[0] = ||y||^2 (launch_sum's
// order), ctl[1] += 1, and with rel = sqrt(nrm[0] / nrm[2]) (0 when nrm[2] <= 0)
// ctl[0] = 2 if rel is not finite, 1 if rel < tol.  ctl[0] is the gate of the next
// step's launches; ticket is a device counter that is zero between launches.
template <typename T>
void launch_residual_stop(const c128* x, const c128* v, c128* y, cplx<T>* yt, OpGeom g, double* part, double* nrm,
                          int* ctl, unsigned* ticket, double tol, cudaStream_t s, const int* need = nullptr,
                          const int* anchor = nullptr);

// b = h^2 w_i w_j f + h (w_j gx + w_i gy) for the global problem (q1: the bilinear
// elements' load vector, h^2 M_y F M_x^T + h (edge masses) g).
void launch_rhs(const c128* f, const c128* g, c128* b, int dim, int S, double h, cudaStream_t s, int q1 = 0);

// dst[i] (+)= (TD) src[i], i < n
template <typename TS, typename TD>
void launch_copy(const cplx<TS>* src, cplx<TD>* dst, size_t n, bool accumulate, bool conjugate,
                 cudaStream_t s);

// Y[x][c] = boundary row of A~_s applied to u: u_if = row on the sibling's artificial
// boundary, u_in = the next row inward (both rows of the child's solution).
template <typename T>
void launch_robin_trace(const cplx<T>* u_if, const cplx<T>* u_in, cplx<T>* Y, int b_s, int Sx, int nc,
                        double kh, const double* khr_row, cudaStream_t s, int q1 = 0);

// v_if/v_in = rows of A~_s B_s^T conj(Q) (the adjoint trace, conjugated for the
// conj o solve o conj adjoint); other rows untouched.
template <typename T>
void launch_adjoint_place(const cplx<T>* Q, cplx<T>* v_if, cplx<T>* v_in, int b_s, int Sx, int nc,
                          double kh, const double* khr_row, cudaStream_t s, int q1 = 0);

// Omega[x][j] (Sx x m) for child `node`: SplitMix64 + Box-Muller, re/im ~ N(0,1/2).
template <typename T>
void launch_sketch(cplx<T>* Om, int Sx, int m, int node, unsigned long long seed, cudaStream_t s);

// W[n][c] += sum_j C[n][j] y[j][c]   (n < npts, j < p, c < nc), y FP64 [p][nc]
template <typename TC, typename TW>
void launch_coarse_update(const cplx<TC>* C, const c128* y, cplx<TW>* W, size_t npts, int p, int nc,
                          cudaStream_t s);

// ---- coarse correction with a column-major basis C[j * N + pt] (k_coarse.cu) --------
template <typename T>
void launch_build_basis(const cplx<T>* src, size_t src0, int r, cplx<T>* C, size_t ldc, int coff, size_t dst0,
                        size_t n, cudaStream_t s);
// One-column coarse corrections of up to CB_MAX_JOBS nodes in one cooperative launch
// (k_coarse.cu).  Per job: basis C [p][N] (TC), right-hand side v (TV), iterate w_in
// (TW, may be null), output out (TO) for the rows [r0, r1) of the node:
//   out[pt - r0 Sx] = (acc_out ? out : 0) + (add_w ? w_in[pt] : 0) + (C y)[pt],
//   y = Minv C^H (v - A~ w_in)  (Minv in TC; y also stored in FP64 when non-null).
// partial: (total blocks) x p scratch entries of TC; bar: two zeroed words (grid
// barrier); err: the device status word (DEV_TIMEOUT if the barrier wait gives up).
constexpr int CB_MAX_JOBS = 16;
constexpr int CB_COLS = 16;   // basis columns one block of k_coarse_batch projects on (p <= 64)
struct CoarseJob {
    const void* C;
    const void* v;
    const void* w_in;
    void* out;
    const void* Minv;
    c128* y;
    OpGeom g;
    int r0, r1;
    int acc_out, add_w;
    int split;             // >= 0: columns [0, p/2) vanish on rows >= split, [p/2, p) on rows
                           // below (each child's basis lives on its owned rows); -1: dense
    unsigned blk0, nblk;   // set by the launcher
    void* dout;            // may be null: also receives the correction added to out (without
                           // out's old value), in the basis precision, at out's index
    int ngrp;              // set by the launcher: column groups per half (p/2 / CB_COLS, rounded up)
    unsigned sb[5];        // set by the launcher: blocks of set s are [sb[s], sb[s + 1])
    const int* gate;       // may be null: while the word is nonzero the job's blocks only take
                           // part in the grid barrier and touch none of the job's buffers
};
// Optional extras of a one-job launch on the root in the device-tested stationary loop.
// Phase 1 keeps r' = v - A~ w (the residual after the level-1 update) in rp; phase 3
// forms the next residual r' - (A C) y (AC: A applied to the basis, laid out as C) into
// rt, with its |.|^2 per block in part, and the last block to finish (ticket: zero
// between launches) adds those in block order and sets the loop's control words:
//   ctl[3] += 1 (steps done); ctl[4] = 1 when ctl[3] is a multiple of `anchor` (the FP64
//   residual then replaces rt), else 0; ctl[2] = 1 when the FP64 residual must be formed
//   (an anchor step, or sqrt(sum / nrm[2]) < 2 tol, or the sum not finite), else 0;
//   nrm[1] = the sum.
struct CoarseRecur {
    const void* AC;        // null: none of this
    void* rp;
    void* rt;
    double* part;
    unsigned* ticket;
    double* nrm;
    int* ctl;
    double tol;
    int anchor;
};
struct CoarseBatch {
    CoarseJob job[CB_MAX_JOBS];
    int njobs;
    const int* gate;       // may be null: when the word is nonzero at launch, nothing is done
    CoarseRecur rr;
    long long wait_polls;  // polls of the grid barrier's wait before it gives up (set by the launcher)
    float keep;            // set by the launcher: < 1 when the launch's basis exceeds the L2 (see the kernel)
};

// Polls a bounded device-side wait makes before giving up with DEV_TIMEOUT: the
// cooperative grid barrier of the coarse corrections and the tensor-core transforms'
// waits for their operands and MMAs.  Negative: each wait's default (about a second).
// Read when a kernel is launched (a captured graph keeps the value of its capture).
// The drains after a wait gave up always use the default.
void set_wait_polls(long long polls);
long long wait_polls(long long dflt);
template <typename TC, typename TV, typename TW, typename TO>
void launch_coarse_batch(CoarseBatch bt, int p, void* partial, unsigned* bar, int* err, cudaStream_t s);
// W[pt][c] += sum_j C[j][pt] y[j][c] (nc columns); split_pt as launch_ip_partial_colA
template <typename TC, typename TW>
void launch_coarse_updn(const cplx<TC>* C, const c128* y, cplx<TW>* W, size_t N, int p, int nc, cudaStream_t s,
                        long long split_pt = -1);
// tiled inner products with a column-major A (p x N); split_pt >= 0: A's first p/2
// columns vanish from point split_pt on and the others before it (a node's coarse basis)
template <typename TA, typename TB, typename ACC>
int launch_ip_partial_colA(const cplx<TA>* A, const cplx<TB>* B, int ldb, size_t N, int p, int q, c128* partial,
                           int max_blocks, cudaStream_t s, long long split_pt = -1);

// Krylov bases, point-major B[n * ld + j]:
void launch_col_load(const c128* B, int ld, int col, c128* dst, size_t n, cudaStream_t s);
void launch_col_store_normalised(c128* B, int ld, int col, const c128* src, const c128* nrm2, size_t n,
                                 cudaStream_t s);
// w += sgn * B[:, :j] c   (c = conj(coef) if cj), coef on the device, j <= 128
void launch_basis_combine(const c128* B, int ld, int j, const c128* coef, bool cj, double sgn, c128* w, size_t n,
                          cudaStream_t s);

// Flexible GMRES's least-squares problem on the device (one thread): the Hessenberg
// matrix H (entry (i, j) at H[i * mk + j], mk + 1 rows), the Givens rotations (cs, sn) and
// the rotated right-hand side g of one restart cycle.
struct GmresState {
    int stop;      // 1 once the estimate is below tol / 2, the new column vanished, or not finite
    int jstop;     // columns of the cycle when it stopped
    int bad;       // 1: the estimate was not finite
    int steps;     // columns done
    double est;    // |g[steps]| / ||b||, the residual estimate
    double pad;
};
struct GmresLs {
    c128* H;       // [(mk + 1) * mk]
    double* cs;    // [mk]
    c128* sn;      // [mk]
    c128* g;       // [mk + 1]
    GmresState* st;
    int mk;
};
// start a cycle: g = (beta, 0, ...), state cleared
void launch_gmres_init(GmresLs ls, double beta, cudaStream_t s);
// column j from the dot products of the two Gram-Schmidt passes (d1, d2: conj(h_ij)) and
// ||w||^2 (dn.re): rotations, g, the estimate and the stop test; does nothing once stopped
void launch_gmres_rotate(GmresLs ls, const c128* d1, const c128* d2, const c128* dn, int j, double nbv, double tol,
                         cudaStream_t s);
// y = R^{-1} g over the first jn columns (R the rotated H)
void launch_gmres_solve(GmresLs ls, int jn, c128* y, cudaStream_t s);

// ---- dense kernels (k_dense.cu) ----------------------------------------------------
// partial[blk][i][j] = sum_{n in blk} conj(A[n*lda+i]) * B[n*ldb+j]; returns nblk.
// ACC is the accumulation precision (double, or float for complex64 working data).
template <typename TA, typename TB, typename ACC = double>
int launch_ip_partial(const cplx<TA>* A, int lda, const cplx<TB>* B, int ldb, size_t N, int p, int q,
                      c128* partial, int max_blocks, cudaStream_t s);
// out[i][j] = sum_blk partial; if Minv != null, out2 = Minv (p x p) * out  (p x q).
void launch_ip_reduce(const c128* partial, int nblk, int p, int q, c128* out, const c128* Minv,
                      c128* out2, cudaStream_t s);
// Galerkin partials: partial[blk][a][l] = sum_pts conj(C[a][pt]) (A~ C)[l][pt]  (p = 2r,
// C column-major).
// split_row >= 0: columns [0, p/2) of C vanish on rows >= split_row and [p/2, p) below it.
// Galerkin partial sums of A_c = C^H A~ C: basis stored in TI, stencil and products in T
// Returns the number of partial blocks written (partial holds max_blocks + 1 blocks of p x p).
// *herm set: the partials are in the Hermitian-packed form (FP64 products of the 5-point
// rows), and launch_herm_fill completes the summed matrix.
template <typename TI, typename T>
int launch_galerkin_partial(const cplx<TI>* C, OpGeom g, int p, int split_row, c128* partial, int max_blocks,
                            cudaStream_t s, bool* herm = nullptr);
// A[j][i] = conj(A[i][j]) + A[j][i] for i < j (p x p, row-major)
void launch_herm_fill(c128* A, int p, cudaStream_t s);
// In-place QR (classical Gram-Schmidt, two passes) of nq independent Sx x m blocks.
template <typename T>
void launch_qr(cplx<T>* const* Y, int nq, int Sx, int m, cplx<T>** dev_ptr_scratch, cudaStream_t s);
// Hermitian eigenproblems of nq m x m FP64 matrices (m <= 64): all eigenvalues
// descending in lam, the r leading eigenvectors in columns 0..r-1 of U (m x m).  Each G
// holds m^2 + 4m complex entries; the matrix is destroyed (used as workspace).
void launch_heig(c128* const* G, c128* const* U, double* const* lam, int nq, int m, int r,
                 void** dev_ptr_scratch, cudaStream_t s);
// V[x][j] = sum_k Z[x][k] U[k][j] / sqrt(lam_j)  for j < r
template <typename T>
void launch_form_v(const cplx<T>* Z, const c128* U, const double* lam, cplx<T>* V, int Sx, int m, int r,
                   cudaStream_t s);
// In-place Gauss-Jordan inverses with partial pivoting of `count` n x n FP64 matrices
// A[0..count) (count <= GJ_MAX_BATCH), one launch.
constexpr int GJ_MAX_BATCH = 32;
struct GjBatch {
    c128* A[GJ_MAX_BATCH];
    void* AT[GJ_MAX_BATCH];   // complex64 copies of the inverses (entries may be NULL)
    int n;
    int* err;
};
// fp32: eliminate in FP32 (the complex64 form), else FP64.
void launch_gj_inverse(const GjBatch& bt, int count, bool fp32, cudaStream_t s);

// ---- leaf kernels (k_leaf.cu) ------------------------------------------------------
struct LeafTask {
    void* X;          // factor store: Sx steps of b x ldx blocks (2D) or b diagonal inverses (1D)
    const void* F;    // right-hand sides [b][Sx][nrhs]
    void* W;          // solutions [b][Sx][nrhs]
    int b;
    int ldx;
    const double* khr;   // k h per row of the band (layered media) or null: the launch's kh
};
template <typename T>
void launch_factor(const LeafTask* d_tasks, int ntasks, int b_max, int Sx, double kh, int* err,
                   cudaStream_t s);
template <typename T>
void launch_sweep(const LeafTask* d_tasks, int ntasks, int b_max, int Sx, int nrhs, int* err,
                  cudaStream_t s);
int leaf_ldx(int b, int elem_bytes);
// tallest band the explicit-inverse path factors (shared-memory bound of k_factor2d)
int leaf_block_bmax(int elem_bytes);

// ---- eigenbasis leaf path (k_eig.cu) -------------------------------------------------
struct EigTask {
    void* V;          // [b][b] generalised eigenvectors of the column pencil (V^T W V = I)
    void* xi;         // [Sx][b] scalar Schur recursion coefficients
    void* lam;        // [b] eigenvalues (complex128)
    const void* F;    // right-hand sides [b][Sx][nrhs]
    void* Fh;         // transformed right-hand sides / solutions [b][Sx][nrhs]
    void* W;          // solutions [b][Sx][nrhs]
    int b;
    int Sx;           // columns of the leaf's problem (tasks of several problems may share a launch)
    int w0, w1;       // the sweep writes local rows [w0, w1) only, row a to W + (a - w0) Sx nrhs
                      // (all rows: w0 = 0, w1 = b)
    const void* vt_emb;   // complex64 form: V^T and V as the tensor-core transforms' B operand
    const void* vn_emb;   // (tc_prepare_v layout; null where the transforms run on CUDA cores)
    const int* gate;      // one-launch sweep: may be null; while the word is nonzero the task's
                          // cluster returns at once, touching none of the task's buffers
    void* sc;             // bilinear elements: [b] per-mode scale of the recursions' input
                          // (null: the 5-point rows, scale 1)
};

// Layout of the transformed vectors Fh of a multi-vector sweep (b rows of J = Sx nrhs):
// up to 15 right-hand sides line by line, [m][c][i] (each scalar recursion reads one
// contiguous line; one warp per line); from 16 on in the node order [m][i][c] (one lane
// per right-hand side, a warp's loads contiguous).  fh_col: the Fh column of node column jj.
HH_HD bool eig_line_major(int nrhs) { return nrhs <= 15; }
HH_HD size_t fh_col(size_t jj, int Sx, int nrhs) {
    return eig_line_major(nrhs) ? (jj % (size_t)nrhs) * (size_t)Sx + jj / (size_t)nrhs : jj;
}

// ---- tensor-core transforms (k_tc.cu) -----------------------------------------------
// Bytes of one B operand (one leaf, one transform) for bands of up to b_max rows.
size_t tc_vemb_bytes(int b_max);
// Fills every task's vt_emb / vn_emb from its V (complex64).
void launch_tc_prepare_v(const EigTask* d_tasks, int ntasks, int b_max, cudaStream_t s);
// 1 when the transform kernel can run on the current device (its shared-memory limit set).
int tc_transform_ready();
// The complex64 sweep transforms on the tensor cores: which = 0, Fh = V^T F; which = 1,
// W = V Fh (layouts as the three-stage sweep).  err: device status word (DEV_TIMEOUT on a
// bounded wait that gave up).  gate (may be null): a device word; when it is nonzero at launch
// the launch does nothing.
void launch_tc_transform(int which, const EigTask* d_tasks, int ntasks, int b_max, int Sx, int nrhs, int* err,
                         cudaStream_t s, const int* gate = nullptr);
template <typename T>
void launch_eig_factor(const EigTask* d_tasks, int ntasks, int b_max, int Sx, double kh, int* err,
                       cudaStream_t s, int q1 = 0);
template <typename T>
void launch_eig_sweep(const EigTask* d_tasks, int ntasks, int b_max, int Sx, int nrhs, cudaStream_t s);
// One right-hand side (nrhs = 1, F/W [b][Sx]): the three stages in one launch, one
// thread-block cluster per leaf.  eig_sweep_fused_ready (call outside stream capture)
// prepares the kernel and returns the cluster size to launch with (16 or 8), or 0 when
// leaves of up to b_max rows do not fit a cluster's shared memory; the caller then runs
// the three stages instead.
constexpr int FS_SMEM_MAX = 220 * 1024;
template <typename T>
int eig_sweep_fused_ready(int b_max, int Sx);
// whether clusters of `cl` CTAs can run the one-launch sweep for these sizes
template <typename T>
bool eig_sweep_fused_feasible(int cl, int b_max, int Sx);
// b_max, Sx: the largest band and column count among the tasks (shared-memory size).
// gate (may be null): a device word; when it is nonzero at launch the launch does nothing.
template <typename T>
void launch_eig_sweep_fused(int cl, const EigTask* d_tasks, int ntasks, int b_max, int Sx, cudaStream_t s,
                            const int* gate = nullptr);
// stage 0: f^ = V^T f; 1: scalar recursions; 2: x = V x^.  gate as launch_eig_sweep_fused.
template <typename T>
void launch_eig_sweep_stage(int stage, const EigTask* d_tasks, int ntasks, int b_max, int Sx, int nrhs,
                            cudaStream_t s, const int* gate = nullptr);
int eig_bmax();

}  // namespace hh
