/*
 * hh.h -- C-ABI of the GB300 hierarchical ORAS Helmholtz library (libhh.so).
 *
 * Problem (Gander, Jiang & Zhang, "Hierarchical Coarse Basis by Randomised SVD: the
 * Helmholtz Problem", Eq. (1) in 1D and Sec. 3.1 in 2D):
 *
 *     -Delta u - k^2 u = f  in (0,1)^d,     d_n u - i k u = g  on the boundary,
 *
 * discretised by second-order finite differences on S = n + 2 nodes per side
 * (n interior nodes plus the two impedance boundary nodes, h = 1/(n+1)), rows scaled
 * by h^2 and the nodal weights (1/2 on boundary nodes) so that A is complex symmetric.
 * The solver is the hierarchical optimised restricted additive Schwarz iteration of
 * Eqs. (2)-(3) over a binary hierarchy of row bands (Sec. 1), with coarse spaces built
 * per level from a randomised SVD of the interface maps (Sec. 2).
 *
 * Conventions for every entry point below
 * ---------------------------------------
 * - Complex numbers are interleaved (re, im) pairs of double ("complex128").
 * - Grid vectors (f, u, b, residuals) are row-major [S_y][S_x], x fastest; a 1D
 *   problem has S_x = 1 and S_y = S.  Multi-column node vectors are
 *   [rows][S_x][ncols] with the column index fastest.
 * - g (impedance data): 2D [4][S], sides x=0, x=1, y=0, y=1, each indexed along the
 *   side; 1D [2] = (g0, g1) with -(u'+iku)(0) = g0 and (u'-iku)(1) = g1 (Eq. (1)).
 * - Pointers named d_* are DEVICE pointers on the current CUDA device; pointers named
 *   h_* are HOST pointers.  The caller owns every pointer it passes; the library never
 *   frees them and keeps no reference after the call returns.
 * - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls enqueue their
 *   work on it and return; calls that return host scalars or hh_stats synchronise it.
 * - The library owns its factors, bases and work buffers.  It obtains them in one
 *   block per handle from the allocator set by hh_set_allocator (default: a
 *   stream-ordered memory pool of the library's own per device, on the handle's
 *   stream) and returns it in hh_destroy.
 * - Errors are returned as hh_status; no call exits, traps or prints.  A handle is not
 *   thread-safe: use one host thread and one stream per handle.
 */
#ifndef HH_H
#define HH_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HH_OK = 0,
    HH_EINVAL = -1,       /* invalid parameter, pointer, node index or size            */
    HH_ENOMEM = -2,       /* the allocator returned NULL                              */
    HH_ENOCONV = -3,      /* max_iter reached or the residual stopped being finite;   */
                          /* u holds the last iterate, stats the achieved residual    */
    HH_EBREAKDOWN = -4,   /* zero pivot in a subdomain or coarse factorisation        */
    HH_ETIMEOUT = -5,     /* a bounded device-side wait gave up                       */
    HH_ECUDA = -6,        /* a CUDA runtime call failed                               */
    HH_ENOTIMPL = -7,
    HH_ETOOLARGE = -8,    /* the problem does not fit a fixed-size static scratch     */
                          /* (hh_residual_noalloc: n + 2 > HH_NOALLOC_MAX_ROWS)       */
    HH_EPENDING = -9      /* hh_server_poll: the request has not finished yet         */
} hh_status;

typedef enum {
    HH_PREC_FP64 = 0,     /* complex128 everywhere, FP64 CUDA-core arithmetic          */
    HH_PREC_MIXED = 1     /* complex64 subdomain factors, sweeps, sketches and bases  */
                          /* (the sweeps' multi-vector transforms on the tensor cores);*/
                          /* FP64 residual, Galerkin matrices A_c (FP64 products of   */
                          /* the complex64 basis), their elimination and the sketch   */
                          /* SVD; the outer iteration refines against the FP64        */
                          /* residual (HH_FLAG_COARSE_FP32: A_c from FP32 products,   */
                          /* eliminated in FP32)                                      */
} hh_precision;

typedef struct {
    int dim;              /* 1 or 2                                                      */
    int n;                /* interior nodes per side; S = n + 2, h = 1/(n+1); n >= 4     */
    double k;             /* wavenumber k > 0 (Eq. (1)); see k_rows for layered media     */
    int levels;           /* hierarchy depth L >= 1: 2^L leaf bands (Sec. 1)             */
    int overlap;          /* rows shared by two siblings; even, >= 2; e = overlap/2 rows */
                          /* added on each side of a non-overlapping split (Sec. 3)      */
    int rank;             /* r: coarse vectors per child (n_c of Sec. 3), >= 1           */
    int oversample;       /* p: extra random samples (Sec. 3 uses n_c + 5 samples)       */
    int n_inner;          /* n_i: sub-level iterations (Sec. 3), >= 1                    */
    double tol;           /* stop when ||b - A u||_2 < tol ||b||_2 (FP64)                */
    int max_iter;         /* outer iterations, >= 1                                      */
    int precision;        /* hh_precision                                                */
    unsigned long long seed;  /* sketch generator seed                                  */
    int leaf_solver;      /* hh_leaf_solver                                              */
    int outer;            /* hh_outer                                                    */
    int restart;          /* Krylov vectors per GMRES cycle (outer = HH_OUTER_GMRES), 1..64 */
    unsigned flags;       /* HH_FLAG_* bits; 0 for the defaults                           */
    const double* k_rows; /* layered media (Sec. 3.3): HOST array of S = n + 2 wavenumbers, */
                          /* one per grid row (k = omega / c(y)), or NULL for the constant k; */
                          /* copied by hh_setup (hh_server_submit: keep it valid until the    */
                          /* request has finished).  Each k_rows[j] > 0 and finite.  2D      */
                          /* problems then need leaf_solver = HH_LEAF_BLOCK (the eigenbasis  */
                          /* path takes one k per band); the paper solves them with GMRES    */
} hh_params;

/* hh_params.flags: the mixed form forms the Galerkin matrices A_c = C^H A~ C from FP32
 * products (FP64 partial sums) and inverts them in FP32, instead of FP64 products and
 * FP64 elimination.  Ignored by the FP64 form. */
#define HH_FLAG_COARSE_FP32 1u
/* hh_params.flags: the mixed form runs its leaf sweeps' dense transforms (f^ = V^T f,
 * x = V x^ over several right-hand sides) on the CUDA cores (FP32 FMA) instead of the
 * tensor cores (TF32 with a three-term split, FP32 accumulation).  Ignored by the FP64
 * form, which always uses the CUDA cores. */
#define HH_FLAG_CUDA_CORE_SWEEPS 2u
/* hh_params.flags: the mixed form runs those transforms on the tensor cores wherever it
 * can, without timing the alternatives (the choice the autotuner otherwise makes per
 * shape).  Not together with HH_FLAG_CUDA_CORE_SWEEPS. */
#define HH_FLAG_TENSOR_CORE_SWEEPS 4u
/* hh_params.flags: discretise with the paper's bilinear (Q1) finite elements on the same
 * nodes (Sec. 3: mass-weighted 9-point rows A = M_y (x) (X_x - (kh)^2 M_x - i kh B_x) +
 * (X_y - i kh B_y) (x) M_x, with the consistent 1D masses M and stiffnesses X over h, and
 * the load vector b = h^2 M_y F M_x^T + h (edge masses) g) instead of the weighted 5-point
 * differences (which are these elements with lumped masses).  2D only, with
 * leaf_solver = HH_LEAF_EIGEN and one wavenumber (k_rows NULL); otherwise HH_EINVAL.
 * The lockstep engine takes 5-point problems only: hh_solve_batch and a server solve these
 * one at a time. */
#define HH_FLAG_BILINEAR 8u

typedef enum {
    HH_LEAF_EIGEN = 0,    /* 2D leaves: the block Schur recursion evaluated in the eigenbasis */
                          /* of the column pencil (scalar recursions + two b x b transforms)  */
    HH_LEAF_BLOCK = 1     /* 2D leaves: the block Schur recursion with explicit b x b inverses */
                          /* S_j^{-1} (Gauss-Jordan, partial pivoting) and block substitution; */
                          /* bands of at most 119 rows (FP64) or 169 rows (mixed), else       */
                          /* hh_setup returns HH_EINVAL                                       */
} hh_leaf_solver;         /* 1D leaves always use the scalar recursion along the line         */

typedef enum {
    HH_OUTER_ORAS = 0,    /* stationary iteration u <- u + M (b - A u) (Eqs. (2)-(3))          */
    HH_OUTER_GMRES = 1    /* flexible GMRES right-preconditioned by M (Sec. 3), FP64 Arnoldi   */
} hh_outer;

typedef struct {
    int iters;            /* outer iterations taken                                      */
    double rel_res;       /* final ||b - A u|| / ||b|| (FP64)                            */
    double t_setup_ms;    /* device time of hh_setup (CUDA events)                       */
    double t_solve_ms;    /* device time of the last hh_solve                            */
    size_t footprint_bytes;
    double t_queue_ms;    /* served requests: submission to admission (host clock)       */
    double t_total_ms;    /* served requests: submission to completion (host clock)      */
} hh_stats;

typedef struct hh_handle hh_handle;

/* Device allocator hook.  alloc(bytes, stream, ctx) returns device memory usable on
 * `stream` or NULL; free_(ptr, bytes, stream, ctx) returns it.  Passing alloc = NULL
 * restores the default: a stream-ordered memory pool of the library's own per device,
 * which keeps memory freed by hh_destroy for later handles (until the process exits).
 * Affects handles created afterwards. */
hh_status hh_set_allocator(void* (*alloc)(size_t bytes, void* stream, void* ctx),
                           void (*free_)(void* ptr, size_t bytes, void* stream, void* ctx),
                           void* ctx);

/* Host-only: device bytes hh_setup will allocate for these parameters (admission). */
hh_status hh_footprint(const hh_params* params, size_t* bytes);

/* Set-up (Sec. 1-2): build the hierarchy, factor every leaf band (block-tridiagonal
 * Schur recursion S_j = D_j - L_j S_{j-1}^{-1} U_j over grid columns), sketch every
 * interface map T_c by the randomised SVD, extend the leading right singular vectors
 * into the coarse bases C_c = P_c A~_c^{-1} B_c^T V_c, and form and invert the Galerkin
 * matrices A_c = C^H A~ C, children before parents.  Synchronises `stream`.
 * Errors: HH_EINVAL (parameters; e.g. odd overlap, a band owning fewer than overlap+2
 * rows, levels < 1), HH_ENOMEM, HH_EBREAKDOWN, HH_ECUDA. */
hh_status hh_setup(const hh_params* params, void* stream, hh_handle** out,
                   size_t* footprint_out);

/* Solve A u = b(f, g) from u = 0 until the FP64 relative residual is below params.tol,
 * by the outer iteration params.outer selects: the coarse-corrected ORAS iteration of
 * Eqs. (2)-(3), or flexible GMRES preconditioned by one step of it (Sec. 3).  d_f
 * [S_y][S_x], d_g [4][S] (or [2]), d_u [S_y][S_x] complex128 device arrays.
 * Synchronises.  Returns HH_ENOCONV (u = last iterate, stats->rel_res its residual) if
 * max_iter is reached or the residual stops being finite. */
hh_status hh_solve(hh_handle* h, const void* d_f, const void* d_g, void* d_u,
                   void* stream, hh_stats* stats);

/* Same as hh_solve with HOST arrays (pinned or pageable): copies f and g in, solves,
 * copies u out, all on `stream`.  Synchronises. */
hh_status hh_solve_host(hh_handle* h, const void* h_f, const void* h_g, void* h_u,
                        void* stream, hh_stats* stats);

/* ||b(f,g) - A u||_2 / ||b||_2 in FP64 (the stopping test of hh_solve).  Synchronises. */
hh_status hh_residual(hh_handle* h, const void* d_f, const void* d_g, const void* d_u,
                      void* stream, double* rel_res);

/* --------------------------------------------------------------------------------
 * Batching form: many independent problems (each with its own parameters and grid
 * size) set up and solved together.
 * -------------------------------------------------------------------------------- */
/* Sets up count problems (params[k] for out[k]): the set-ups run concurrently, up to
 * eight at a time, each on a stream and host thread of its own; returns when all are
 * done.  On any failure every handle created so far is destroyed, out[] is NULL and the
 * first failing status is returned.  The handles are ordinary handles (hh_solve,
 * hh_destroy, ...); their stream is set to `stream`. */
hh_status hh_setup_batch(const hh_params* params, int count, void* stream, hh_handle** out);

/* Solves count set-up problems: u[k] = solution of problem h[k] for d_f[k], d_g[k]
 * (layouts as hh_solve).  When every handle uses the stationary outer iteration with
 * n_inner = 1, the eigenbasis leaf path and at least two levels, in one precision, the
 * problems iterate in lockstep: each iteration is one residual launch, one leaf-sweep
 * launch, one coarse-correction launch per hierarchy height and one for the roots, for
 * all problems together, and a problem drops out when its residual meets its own tol.
 * Otherwise the problems are solved one after another.  stats[k] (may be NULL) gets
 * problem k's iterations and residual; t_solve_ms is the time of the whole batch.
 * Synchronises.  Returns HH_OK if all converged, else the first failing status. */
hh_status hh_solve_batch(hh_handle* const* h, const void* const* d_f, const void* const* d_g, void* const* d_u,
                         int count, void* stream, hh_stats* stats);

/* --------------------------------------------------------------------------------
 * Serving form: a request loop with continuous batching.  Requests (any grid size,
 * wavenumber and hierarchy) are admitted while the sum of their footprints
 * (hh_footprint) stays within hbm_budget bytes and fewer than max_slots are in flight.
 * Four set-up workers set admitted requests up concurrently, each on a stream of its own;
 * one engine thread iterates all set-up requests together (the lockstep iteration of
 * hh_solve_batch), taking new ones in between iterations and retiring each as soon as
 * its residual meets its tol.  Requests the lockstep iteration cannot take are solved by
 * their worker; requests whose stationary iteration does not converge are re-solved by
 * flexible GMRES.  Server problems allocate from the library's own stream-ordered pool
 * on the current device (the default of hh_set_allocator), never through an installed
 * hook.
 * -------------------------------------------------------------------------------- */
typedef struct hh_server hh_server;

/* Starts the server threads on the current device.  HH_EINVAL for max_slots outside
 * [1, 4096] or a zero budget. */
hh_status hh_server_create(size_t hbm_budget, int max_slots, hh_server** out);

/* Queues one request and returns at once with its ticket.  d_f, d_g (read) and d_u
 * (written) are device arrays laid out as for hh_solve; they must stay valid, and d_f,
 * d_g unchanged, until the ticket has finished, and must hold their data (the caller's
 * stream synchronised) before the call.  HH_EINVAL for invalid parameters, HH_ENOMEM
 * when the request's footprint alone exceeds the budget. */
hh_status hh_server_submit(hh_server* srv, const hh_params* params, const void* d_f, const void* d_g, void* d_u,
                           unsigned long long* ticket);

/* Non-blocking.  HH_EPENDING while the request is queued or in flight; HH_OK once it has
 * finished, with *result its status (as hh_solve's) and *stats (may be NULL) its
 * iterations, residual, set-up and solve times, footprint, queueing and total latency;
 * d_u then holds the solution.  A finished ticket is forgotten after it has been polled
 * (polling it again gives HH_EINVAL). */
hh_status hh_server_poll(hh_server* srv, unsigned long long ticket, hh_status* result, hh_stats* stats);

/* Stops the threads (queued and in-flight requests are abandoned) and frees everything. */
void hh_server_destroy(hh_server* srv);

void hh_destroy(hh_handle* h);
const char* hh_status_string(hh_status s);

/* --------------------------------------------------------------------------------
 * Allocation-free residual.  The paper has no counterpart: this is a service entry
 * point of the library, not a step of the method.
 *
 * Who needs it: a caller that may not allocate device memory at the moment it wants
 * the residual.  cudaMalloc and cudaFree can synchronise the whole device, which a
 * caller overlapping latency-bound work on other streams cannot afford; a process whose
 * device memory is already claimed by a pooling allocator (a framework's caching pool,
 * a serving engine that reserves the HBM up front) may see a fresh cudaMalloc fail
 * although its own pool has room; and a caller with a fixed memory plan (a health check
 * run after a solve, next to other jobs' buffers) must not fail half-way for want of
 * memory.  hh_residual needs a handle, and hh_setup allocates.
 * -------------------------------------------------------------------------------- */
/* Largest number of grid rows (S = n + 2) hh_residual_noalloc accepts. */
#define HH_NOALLOC_MAX_ROWS 16384

/* ||b(f,g) - A u||_2 / ||b||_2 in FP64, the same quantity as hh_residual, for the
 * problem (dim, n, k) of Eq. (1) / Sec. 3.1 (h = 1/(n+1)), without a handle and
 * without allocating: no cudaMalloc, cudaFree or allocating library call.
 * d_f [S_y][S_x], d_g [4][S] (or [2]) and d_u [S_y][S_x] are complex128 device arrays
 * on the current device, owned by the caller and only read; rel_res is a host double.
 * Enqueues one memset of a 4-byte counter, one kernel and one 16-byte device-to-host
 * copy on `stream`, and synchronises it.  b = 0 gives 0.
 * Scratch: a file-scope device array of HH_NOALLOC_MAX_ROWS x 16 bytes (256 KiB)
 * plus 256 bytes, which every GPU that loads libhh holds until the process exits.  It
 * holds one (sum |r|^2, sum |b|^2) pair per grid row, the total and a counter; the
 * counter, the one part that must start at zero, is cleared on `stream` by every call.
 * The first call on a device (the device current at the call) looks the array's address
 * up (cudaGetSymbolAddress) and caches it.  Under CUDA's lazy module loading that first
 * call may also be the moment the library's device code is loaded on that device and the
 * array's memory reserved, so the promise of no allocation is firm only from the second
 * call on: a caller that must not allocate later makes one warm-up call at start-up (any
 * small problem), before any stream capture.  Calls that overlap in time on one device share the array and race: issue
 * them from one host thread on one stream (or otherwise serialise them).
 * Errors: HH_EINVAL for dim not 1 or 2, n < 1, k negative or not finite, or a NULL
 * pointer; HH_ETOOLARGE when n + 2 > HH_NOALLOC_MAX_ROWS (checked before any pointer
 * or the device is touched); HH_ECUDA when a CUDA call fails (including the address
 * look-up). */
hh_status hh_residual_noalloc(int dim, int n, double k, const void* d_f, const void* d_g,
                              const void* d_u, void* stream, double* rel_res);

/* --------------------------------------------------------------------------------
 * Step-level entry points.  Each runs one step of the path on device arrays so that it
 * can be checked on its own.  Nodes are numbered as in Sec. 1: root 0, children of i
 * are 2i+1 and 2i+2.  Node vectors are complex128 [b_node][S_x][ncols] over the node's
 * band of rows (hh_node_info).  Asynchronous on `stream` unless stated.
 * -------------------------------------------------------------------------------- */

/* info[0..9] = owned rows [oa, ob), region rows [ra, rb), level, parent, child0,
 * child1, S_x, interface row (global row of the band's artificial boundary facing its
 * sibling, -1 for the root).  Host-only. */
hh_status hh_node_info(const hh_handle* h, int node, int info[10]);

/* d_y = A~_node d_x for ncols columns (A for the root), the weighted 5-point operator
 * with impedance rows on the band's artificial boundaries (Sec. 1, Sec. 2). */
hh_status hh_apply_operator(hh_handle* h, int node, const void* d_x, void* d_y, int ncols,
                            void* stream);

/* d_x = A~_leaf^{-1} d_v by the leaf's block forward and backward substitution
 * (the subdomain solves of Eq. (2)).  ncols >= 1 columns. */
hh_status hh_leaf_solve(hh_handle* h, int leaf, const void* d_v, void* d_x, int ncols,
                        void* stream);

/* Interface map of child c (Sec. 2): adjoint = 0: d_out = T_c d_in; adjoint = 1:
 * d_out = T_c^* d_in.  T_c = B_s A~_s R_s R_c^T M_c B_c^T with s the sibling and M_c the
 * leaf solve (leaves) or n_i sub-level iterations (internal children); the adjoint of
 * M_c is taken as conj o M_c o conj.  d_in, d_out: [S_x][ncols] complex128. */
hh_status hh_interface_map(hh_handle* h, int child, int adjoint, const void* d_in,
                           void* d_out, int ncols, void* stream);

/* Copies child c's coarse modes V_c ([S_x][r] complex128) and the singular values of
 * its sketch (r + p doubles, descending) to HOST arrays.  Synchronises. */
hh_status hh_get_basis(hh_handle* h, int child, void* h_V, double* h_sigma);

/* d_z = C_p A_c^{-1} C_p^H d_r on node p's band (Eq. (3)), one column. */
hh_status hh_coarse_apply(hh_handle* h, int node, const void* d_r, void* d_z, void* stream);

/* d_z = one coarse-corrected ORAS step from zero applied to the global residual d_r
 * (Eqs. (2)-(3) with u^(n-1) = 0): the preconditioner of the outer iteration. */
hh_status hh_precondition(hh_handle* h, const void* d_r, void* d_z, void* stream);

/* Writes the counter-based complex Gaussian sketch of child c ([S_x][r+p]) used by
 * the randomised SVD (SplitMix64 + Box-Muller, re/im ~ N(0, 1/2)). */
hh_status hh_sketch_samples(hh_handle* h, int child, void* d_out, void* stream);

/* --------------------------------------------------------------------------------
 * Tracing.  With profiling enabled a handle records CUDA events on its stream around
 * the kernels of each category below (events cost a few microseconds of stream time
 * each); totals accumulate over hh_setup/hh_solve calls until the next enable.
 * Categories: 0 leaf factorisation, 1 leaf sweep transform into the column eigenbasis,
 * 2 leaf sweep recursions along the line (scalar recursions, or the block substitution
 * of the explicit-inverse path), 3 leaf sweep transform back, 4 FP64 global residual,
 * 5 one-column coarse corrections (C^H r, A_c^{-1}, C y: one launch per level), 6 Galerkin
 * product, 7 sketch orthonormalisation, 8 sketch SVD, 9 leaf sweep of a single
 * right-hand side on the eigenbasis path (categories 1-3 fused into one launch; 1-3 then
 * count the multi-vector sweeps of the set-up), 10 multi-column coarse projections of the
 * set-up's sub-level solves.
 * -------------------------------------------------------------------------------- */
/* h != NULL: (re)start profiling of that handle, clearing its totals; h == NULL: set
 * whether handles created afterwards profile from their first set-up kernel. */
hh_status hh_profile_enable(hh_handle* h, int enable);
/* Which categories the profiler times: bit c of mask for category c (default: all).
 * Each timed category costs events on the stream, so a caller timing one kernel family
 * selects only that one.  h != NULL: that handle, from its next launch; h == NULL:
 * handles created afterwards.  Within one outer step the coarse corrections of all
 * levels run back to back and share one event pair (counted as that many launches). */
hh_status hh_profile_categories(hh_handle* h, unsigned mask);
/* total_ms: summed event time; launches: timed launches; alg_bytes / alg_flops: the
 * algorithmic memory traffic and floating-point work of those launches (formulas in the
 * library: e.g. a band transform of b rows, S_x columns and nc right-hand sides counts
 * 8 b^2 S_x nc flops and (b^2 + 2 b S_x nc) elements; a one-column coarse correction of
 * a node of n points and rank r counts 2 r n elements of the basis: its r basis columns
 * read once for C^H r and once for C y).  Any output may be NULL. */
hh_status hh_profile_read(const hh_handle* h, int category, double* total_ms, long long* launches,
                          double* alg_bytes, double* alg_flops);
/* Number of CUDA kernels this library has launched in the calling process. */
unsigned long long hh_launch_count(void);

/* Decisions of the library's autotuner in this process, as a JSON array: for each shape
 * met so far, the candidates' measured milliseconds per launch and the one chosen.  The
 * candidates are the complex64 multi-vector sweep transforms on the tensor cores or the
 * CUDA cores (per transform, band height, columns and right-hand sides) and the cluster
 * size (16 or 8) of the one-launch single-vector sweep; each is timed on the first use of
 * its shape, outside any stream capture, and kept until exit.  The text (NUL-terminated,
 * cut at cap - 1 bytes) goes to buf when buf is not NULL; *len (may be NULL) gets its
 * full length.  An engineering aid: the paper has no counterpart. */
hh_status hh_autotune_report(char* buf, size_t cap, size_t* len);

/* --------------------------------------------------------------------------------
 * Failure detection (testing aid; the paper has no counterpart).  Every device-side
 * wait of the library is bounded: a wait that runs out records HH_ETIMEOUT, its kernel
 * stops issuing work, drains what it has in flight and returns, and the call that
 * synchronises reports HH_ETIMEOUT with the context still usable.
 * -------------------------------------------------------------------------------- */
/* Caps the polls of the give-up waits of the kernels launched from now on in this
 * process: the coarse corrections' cooperative grid barrier and the tensor-core
 * transforms' waits for their operands and MMAs.  polls = 0 makes every such wait give
 * up at once (how a test makes a wait run out without a fault); polls < 0 restores the
 * defaults (about a second).  CUDA graphs captured meanwhile keep the value of their
 * capture, so a test sets it before creating the handle it checks.  Process-wide. */
hh_status hh_debug_set_wait_limit(long long polls);

#ifdef __cplusplus
}
#endif
#endif /* HH_H */
