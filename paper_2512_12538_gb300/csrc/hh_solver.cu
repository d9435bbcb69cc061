// hh_solver.cu -- host driver and C-ABI of libhh.
//
// Method (Gander, Jiang & Zhang): hierarchical ORAS with randomised-SVD coarse spaces.
//  * Hierarchy (Sec. 1): binary bands of grid rows, node i has children 2i+1, 2i+2;
//    a node owning rows [oa, ob) splits at mid = oa + (ob-oa)/2, every non-root region
//    is its owned rows extended by e = overlap/2 rows each side (Sec. 3), clipped; the
//    first child owns [parent.ra, mid) inside its parent, the second [mid, parent.rb).
//  * Sub-level solve M_p (Sec. 1, Sec. 3 "n_i"): n_i iterations from zero of
//        w~ = w + sum_c P_c M_c R_c (v - A~_p w)          (Eq. (2))
//        w  = w~ + C_p A_c^{-1} C_p^H (v - A~_p w~)         (Eq. (3))
//    with exact leaf solves.  The outer iteration is the same step at the root in FP64:
//        u <- u + M_root(b - A u) until ||b - A u|| < tol ||b||.
//  * Coarse space of p (Sec. 2): for each child c, randomised SVD of the interface map
//    T_c = B_s A~_s R_s R_c^T M_c B_c^T (s = sibling), V_c = leading right singular
//    vectors, C_c = P_c M_c B_c^T V_c, A_c = C_p^H A~_p C_p, children before parents.
//
// Every level is processed in batch: all nodes of a level run each step together.
// Storage: node vectors [rows][Sx][ncols] (column index fastest); a child's input is a
// contiguous row window of its parent's residual buffer.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "../../include/hh.h"
#include "kernels.h"

namespace hh {

// ------------------------------------------------------------------ launch counter
static std::atomic<unsigned long long> g_launches{0};
static bool g_prof_default = false;   // profiling state of newly created handles
static unsigned g_prof_mask_default = ~0u;   // their timed categories
static thread_local unsigned long long t_launches = 0;   // this thread's launches (captures)
void note_launch() {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    ++t_launches;
}

// ------------------------------------------------------------ pinned host blocks
// The per-handle host copies of norms and dot products live in 8 KiB pinned blocks kept
// in a process-wide free list: page-locking memory per handle (and releasing it, which
// synchronises the device) cost more than a whole set-up's kernels on small problems.
// Blocks are returned only once nothing can still copy into them, and are held until
// the process exits.
static constexpr size_t PIN_BLOCK = 8192;
static std::mutex g_pin_mu;
static std::vector<void*> g_pin_free;
static void* pinned_get() {
    {
        std::lock_guard<std::mutex> lk(g_pin_mu);
        if (!g_pin_free.empty()) {
            void* p = g_pin_free.back();
            g_pin_free.pop_back();
            return p;
        }
    }
    void* p = nullptr;
    if (cudaHostAlloc(&p, PIN_BLOCK, cudaHostAllocPortable) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}
static void pinned_put(void* p) {
    if (!p) return;
    std::lock_guard<std::mutex> lk(g_pin_mu);
    g_pin_free.push_back(p);
}

// Kernel categories timed by the optional event profiler (hh_profile_*).
enum ProfCat {
    PC_FACTOR = 0,   // leaf factorisation (eigen set-up or explicit block inverses)
    PC_TIN,          // leaf sweep: transform into the eigenbasis
    PC_RECUR,        // leaf sweep: recursions along the line (scalar, or the block substitution)
    PC_TOUT,         // leaf sweep: transform back
    PC_SPMV,         // FP64 global residual
    PC_COARSE,       // one-column coarse corrections (C^H r, A_c^{-1}, C y; one launch per level)
    PC_GALERKIN,     // Galerkin product
    PC_QR,           // sketch orthonormalisation
    PC_JACOBI,       // sketch SVD
    PC_SWEEP,        // leaf sweep for one right-hand side, all three stages in one launch
    PC_COARSE_MC,    // multi-column coarse projections C^H r of the set-up's sub-level solves
    PC_NCAT
};

// ----------------------------------------------------------------- allocator hook
struct AllocHook {
    void* (*alloc)(size_t, void*, void*) = nullptr;
    void (*free_)(void*, size_t, void*, void*) = nullptr;
    void* ctx = nullptr;
};
static AllocHook g_alloc;

// Without a hook, handles draw from a stream-ordered memory pool of the library's own,
// one per device, that keeps freed memory for later set-ups. (The device's default pool
// returns freed memory to the driver at every synchronisation, so each set-up mapped its
// block afresh.) The memory stays with the pool until the process exits.
static cudaMemPool_t lib_pool(int dev) {
    static std::mutex mu;
    static std::map<int, cudaMemPool_t> pools;
    std::lock_guard<std::mutex> lk(mu);
    const auto it = pools.find(dev);
    if (it != pools.end()) return it->second;
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
        cudaGetLastError();
        pool = nullptr;
    } else {
        unsigned long long keep = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    pools[dev] = pool;
    return pool;
}
static void* dev_alloc(size_t bytes, cudaStream_t s, const AllocHook& a) {
    if (a.alloc) return a.alloc(bytes, (void*)s, a.ctx);
    void* p = nullptr;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    const cudaMemPool_t pool = lib_pool(dev);
    const cudaError_t e = pool ? cudaMallocFromPoolAsync(&p, bytes, pool, s) : cudaMallocAsync(&p, bytes, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}
static void dev_free(void* p, size_t bytes, cudaStream_t s, const AllocHook& a) {
    if (!p) return;
    if (a.alloc) {
        if (a.free_) a.free_(p, bytes, (void*)s, a.ctx);
        return;
    }
    cudaFreeAsync(p, s);
}

// ---------------------------------------------------------------------- autotuner
// Schedules of the leaf sweep are chosen by timing the candidates on the first use of
// each shape, on the device and with the data of that use, and kept for the process:
//   kind 0: the complex64 multi-vector transforms (f^ = V^T f, x = V x^) on the tensor
//           cores (choice 1) or the CUDA cores (choice 0), per (transform, b_max, Sx, nrhs);
//   kind 1: the cluster size of the one-launch single-vector sweep (16 or 8 CTAs per
//           leaf), per (b_max, Sx), where both fit.
// Candidates compute the same quantities (up to rounding), so the choice changes speed,
// not the method.  Timing never runs inside a stream capture.
struct TuneKey {
    int dev, kind, a, b, c, d;
    bool operator<(const TuneKey& o) const {
        return std::tie(dev, kind, a, b, c, d) < std::tie(o.dev, o.kind, o.a, o.b, o.c, o.d);
    }
};
struct TuneEntry {
    int choice;
    float ms[2];   // per launch: candidate 0, candidate 1
};
static std::mutex g_tune_mu;
static std::map<TuneKey, TuneEntry> g_tune;
static bool tune_find(const TuneKey& k, int& choice) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    const auto it = g_tune.find(k);
    if (it == g_tune.end()) return false;
    choice = it->second.choice;
    return true;
}
static void tune_store(const TuneKey& k, const TuneEntry& e) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune.emplace(k, e);
}
static bool stream_capturing(cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    return cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone;
}
// Times two candidates on `s` (each `reps` times after one warm-up run), returns the
// faster (0 or 1) and their milliseconds per launch.  run(c) enqueues candidate c.
template <typename F> static int tune_pair(cudaStream_t s, F&& run, float ms[2], int reps = 3) {
    cudaEvent_t ev[3];
    for (auto& e : ev) cudaEventCreate(&e);
    run(0);
    run(1);
    cudaEventRecord(ev[0], s);
    for (int i = 0; i < reps; ++i) run(0);
    cudaEventRecord(ev[1], s);
    for (int i = 0; i < reps; ++i) run(1);
    cudaEventRecord(ev[2], s);
    cudaEventSynchronize(ev[2]);
    float a = 0.f, b = 0.f;
    cudaEventElapsedTime(&a, ev[0], ev[1]);
    cudaEventElapsedTime(&b, ev[1], ev[2]);
    for (auto& e : ev) cudaEventDestroy(e);
    ms[0] = a / reps;
    ms[1] = b / reps;
    return ms[1] < ms[0] ? 1 : 0;
}

// ---------------------------------------------------------------------- hierarchy
struct Node {
    int id = 0, level = 0, oa = 0, ob = 0, ra = 0, rb = 0, parent = -1;
    int child[2] = {-1, -1};
    int own_a = 0, own_b = 0;   // rows owned inside the parent's region (global)
    int ifrow = -1;             // artificial boundary row facing the sibling (global)
    int inward = -1;            // the row next to ifrow, inside the band
    int sib = -1;
    int b() const { return rb - ra; }
    bool leaf() const { return child[0] < 0; }
};

static hh_status build_tree(int S, int L, int e, std::vector<Node>& nodes) {
    nodes.assign((size_t)(1 << (L + 1)) - 1, Node());
    nodes[0].ob = S;
    nodes[0].rb = S;
    for (int id = 0; id < (1 << L) - 1; ++id) {
        Node& p = nodes[id];
        const int mid = p.oa + (p.ob - p.oa) / 2;
        for (int k = 0; k < 2; ++k) {
            const int cid = 2 * id + 1 + k;
            Node& c = nodes[cid];
            c.id = cid;
            c.level = p.level + 1;
            c.parent = id;
            c.oa = k ? mid : p.oa;
            c.ob = k ? p.ob : mid;
            if (c.ob - c.oa < 2 * e + 2) return HH_EINVAL;
            c.ra = std::max(0, c.oa - e);
            c.rb = std::min(S, c.ob + e);
            c.own_a = k ? mid : p.ra;
            c.own_b = k ? p.rb : mid;
            c.ifrow = k ? c.ra : c.rb - 1;
            c.inward = k ? c.ra + 1 : c.rb - 2;
            c.sib = 2 * id + 2 - k;
            p.child[k] = cid;
        }
    }
    return HH_OK;
}

static hh_status validate(const hh_params* P) {
    if (!P) return HH_EINVAL;
    if (P->dim != 1 && P->dim != 2) return HH_EINVAL;
    if (P->n < 4 || P->n > 1 << 20) return HH_EINVAL;
    if (!(P->k > 0.0) || !std::isfinite(P->k)) return HH_EINVAL;
    if (P->levels < 1 || P->levels > 10) return HH_EINVAL;
    if (P->overlap < 2 || (P->overlap & 1)) return HH_EINVAL;
    if (P->rank < 1 || P->oversample < 0 || P->n_inner < 1) return HH_EINVAL;
    if (!(P->tol > 0.0) || P->max_iter < 1) return HH_EINVAL;
    if (P->precision != HH_PREC_FP64 && P->precision != HH_PREC_MIXED) return HH_EINVAL;
    if (P->leaf_solver != HH_LEAF_EIGEN && P->leaf_solver != HH_LEAF_BLOCK) return HH_EINVAL;
    if (P->outer != HH_OUTER_ORAS && P->outer != HH_OUTER_GMRES) return HH_EINVAL;
    if (P->outer == HH_OUTER_GMRES && (P->restart < 1 || P->restart > 64)) return HH_EINVAL;
    if (P->flags & ~(HH_FLAG_COARSE_FP32 | HH_FLAG_CUDA_CORE_SWEEPS | HH_FLAG_TENSOR_CORE_SWEEPS | HH_FLAG_BILINEAR))
        return HH_EINVAL;
    if ((P->flags & HH_FLAG_CUDA_CORE_SWEEPS) && (P->flags & HH_FLAG_TENSOR_CORE_SWEEPS)) return HH_EINVAL;
    // bilinear elements: the eigenbasis leaves of a 2D problem with one wavenumber
    if ((P->flags & HH_FLAG_BILINEAR) && (P->dim != 2 || P->leaf_solver != HH_LEAF_EIGEN || P->k_rows))
        return HH_EINVAL;
    if (P->k_rows) {
        // layered media: the wavenumber varies across the rows of a band, which the
        // column-pencil eigenbasis of the 2D leaves does not take (explicit inverses do)
        if (P->dim == 2 && P->leaf_solver == HH_LEAF_EIGEN) return HH_EINVAL;
        for (int j = 0; j < P->n + 2; ++j)
            if (!(P->k_rows[j] > 0.0) || !std::isfinite(P->k_rows[j])) return HH_EINVAL;
    }
    if (P->levels > 6) return HH_EINVAL;
    const int Sx = P->dim == 2 ? P->n + 2 : 1;
    if ((long long)(P->n + 2) * Sx >= (1ll << 31)) return HH_EINVAL;   // grid points index in 32 bits
    const int m = std::min(P->rank + P->oversample, Sx);
    if (2 * std::min(P->rank, m) > 64 || m > 64) return HH_EINVAL;   // dense coarse kernels
    std::vector<Node> nodes;
    const hh_status st = build_tree(P->n + 2, P->levels, P->overlap / 2, nodes);
    if (st != HH_OK) return st;
    if (P->dim == 2 && P->leaf_solver == HH_LEAF_EIGEN)
        for (auto& nd : nodes)
            if (nd.leaf() && nd.b() > eig_bmax()) return HH_EINVAL;   // band too tall for this path
    if (P->dim == 2 && P->leaf_solver == HH_LEAF_BLOCK) {
        const int bmax = leaf_block_bmax(P->precision == HH_PREC_FP64 ? 16 : 8);
        for (auto& nd : nodes)
            if (nd.leaf() && nd.b() > bmax) return HH_EINVAL;         // inverse does not fit shared memory
    }
    return HH_OK;
}

// ----------------------------------------------------------------- arena planning
struct Arena {
    char* base = nullptr;
    size_t off = 0;
    template <class X> X* take(size_t count) {
        off = align_up(off, 256);
        X* p = base ? (X*)(base + off) : nullptr;
        off += sizeof(X) * std::max<size_t>(count, 1);
        return p;
    }
};

static inline cudaError_t ck(cudaError_t e, cudaError_t& first) {
    if (e != cudaSuccess && first == cudaSuccess) first = e;
    return e;
}

static const int MAX_PART_BLOCKS = 304;   // 2 x 152 SMs
static const int COARSE_BLOCKS = 64;      // partial blocks of a one-column coarse projection

struct SolverBase {
    hh_params P{};
    AllocHook hook;
    void* block = nullptr;
    size_t footprint = 0;
    cudaStream_t stream = nullptr;
    double t_setup_ms = 0.0, t_solve_ms = 0.0;
    // event profiler: pairs recorded around the kernels of one category
    // nl: launches between a and b (adjacent launches of one category share a pair)
    struct EvPair { cudaEvent_t a, b; int cat; double bytes, flops; int nl; };
    bool prof_on = false;
    unsigned prof_mask = ~0u;   // categories timed while prof_on
    std::vector<EvPair> prof_pending;
    std::vector<cudaEvent_t> prof_pool;
    double prof_ms[PC_NCAT] = {0};
    long long prof_n[PC_NCAT] = {0};
    double prof_bytes[PC_NCAT] = {0}, prof_flops[PC_NCAT] = {0};   // algorithmic work
    cudaEvent_t prof_ev() {
        if (!prof_pool.empty()) { cudaEvent_t e = prof_pool.back(); prof_pool.pop_back(); return e; }
        cudaEvent_t e;
        cudaEventCreate(&e);
        return e;
    }
    // While the stream is being captured into a graph, the records become external
    // event-record nodes, so replays of the graph stamp the same events again.
    void ev_record(cudaEvent_t e) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        cudaStreamIsCapturing(stream, &cs);
        if (cs == cudaStreamCaptureStatusActive) cudaEventRecordWithFlags(e, stream, cudaEventRecordExternal);
        else cudaEventRecord(e, stream);
    }
    // bytes / flops: algorithmic work of the kernels between pbeg and pend
    bool prof_cat(int cat) const { return prof_on && ((prof_mask >> cat) & 1u); }
    void pbeg(int cat, double bytes = 0.0, double flops = 0.0) {
        if (!prof_cat(cat)) return;
        EvPair p{prof_ev(), nullptr, cat, bytes, flops, 1};
        ev_record(p.a);
        prof_pending.push_back(p);
    }
    // like pbeg, but a launch that directly follows an open pair of the same category
    // joins it (one pair, two events, for a run of adjacent launches)
    void pjoin(int cat, double bytes, double flops) {
        if (!prof_cat(cat)) return;
        if (!prof_pending.empty() && !prof_pending.back().b && prof_pending.back().cat == cat) {
            EvPair& p = prof_pending.back();
            p.bytes += bytes;
            p.flops += flops;
            p.nl += 1;
            return;
        }
        pbeg(cat, bytes, flops);
    }
    void pend(int cat) {
        if (!prof_cat(cat) || prof_pending.empty() || prof_pending.back().b || prof_pending.back().cat != cat) return;
        prof_pending.back().b = prof_ev();
        ev_record(prof_pending.back().b);
    }
    // event pairs owned by captured graphs: read after every synchronised replay
    void prof_account(const EvPair& p) {
        float ms = 0.f;
        if (p.b && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            prof_ms[p.cat] += ms;
            prof_n[p.cat] += p.nl;
            prof_bytes[p.cat] += p.bytes;
            prof_flops[p.cat] += p.flops;
        }
    }
    void prof_read_pairs(const std::vector<EvPair>& v) {
        for (auto& p : v) prof_account(p);
    }
    void prof_collect() {   // call after synchronising the stream
        for (auto& p : prof_pending) {
            prof_account(p);
            prof_pool.push_back(p.a);
            if (p.b) prof_pool.push_back(p.b);
        }
        prof_pending.clear();
    }
    void prof_reset(bool on, unsigned mask) {
        prof_on = on;
        prof_mask = mask;
        for (int i = 0; i < PC_NCAT; ++i) { prof_ms[i] = 0; prof_n[i] = 0; prof_bytes[i] = 0; prof_flops[i] = 0; }
    }
    virtual ~SolverBase() {
        for (auto& p : prof_pending) { prof_pool.push_back(p.a); if (p.b) prof_pool.push_back(p.b); }
        for (auto e : prof_pool) cudaEventDestroy(e);
    }
    // forget captured graphs (their event-record nodes follow the profiler settings of
    // the capture); the next step captures again
    virtual void drop_graphs() {}
    // profiler settings of this handle; captured graphs are dropped when they change
    void prof_configure(bool on, unsigned mask, bool clear) {
        if (on != prof_on || mask != prof_mask) drop_graphs();
        if (clear) prof_reset(on, mask);
        prof_on = on;
        prof_mask = mask;
    }
    virtual size_t plan(char* base) = 0;
    virtual hh_status setup() = 0;
    virtual hh_status solve(const c128* f, const c128* g, c128* u, hh_stats* st) = 0;
    virtual hh_status residual(const c128* f, const c128* g, const c128* u, double* rel) = 0;
    virtual hh_status node_info(int node, int info[10]) const = 0;
    virtual hh_status apply_operator(int node, const c128* x, c128* y, int nc) = 0;
    virtual hh_status leaf_solve(int leaf, const c128* v, c128* x, int nc) = 0;
    virtual hh_status interface_map(int child, int adj, const c128* in, c128* out, int nc) = 0;
    virtual hh_status get_basis(int child, void* hV, double* hsig) = 0;
    virtual hh_status coarse_apply(int node, const c128* r, c128* z) = 0;
    virtual hh_status precondition(const c128* r, c128* z) = 0;
    virtual hh_status sketch_samples(int child, c128* out) = 0;
    virtual c128* staging_f() = 0;
    virtual c128* staging_g() = 0;
    virtual c128* iterate() = 0;
    virtual int npoints() const = 0;
};

template <typename T>
struct Solver final : SolverBase {
    using CT = cplx<T>;
    int S = 0, Sx = 0, Sy = 0, L = 0, e = 0, m = 0, r = 0, nmax = 0, nn = 0;
    double h = 0, kh = 0;
    std::vector<Node> nodes;
    std::vector<std::vector<int>> lev;
    // device buffers
    std::vector<CT*> W, R, Vs, C, X, Om, Z, Vc;
    std::vector<c128*> Ainv, ycoef, Gm, U;
    std::vector<CT*> AinvT;      // A_c^{-1} in the basis precision (the one-column correction)
    std::vector<double*> lam;
    std::vector<int> ldx;
    c128 *u = nullptr, *ut = nullptr, *bvec = nullptr, *res = nullptr, *gbuf = nullptr;
    double* khr_dev = nullptr;  // layered media: k h per grid row (device), else null
    CT* RT = nullptr;
    CT* dlt = nullptr;          // the level-1 update of the current step (leaf precision)
    CT* AC0 = nullptr;          // A~_0 C_0: the root's operator on its basis (column-major)
    CT* RP = nullptr;           // r' of the current step (the root's input residual)
    c128* partial = nullptr;
    double *npart = nullptr, *dnorm = nullptr;
    int* derr = nullptr;
    unsigned* dcounter = nullptr;   // ticket counter of the last-block reductions (zero between launches)
    LeafTask *d_tasks_view = nullptr, *d_tasks_own = nullptr, *d_task_one = nullptr, *d_tasks_pre = nullptr;
    // inputs of the nodes in the current apply (with n_i = 1 a child reads its parent's
    // input directly: R_c of the parent's input, no copy into the parent's buffer)
    std::vector<const CT*> cur_in;
    bool in_pre = false;        // inside the preconditioner step (oras_step)
    c128* root_out = nullptr;   // with n_i = 1 the level-1 corrections write into the root's
    bool root_acc = false;      // output directly (accumulating onto a base iterate)
    bool pre_direct = false;    // its leaf sweeps write the owned rows into the parents
    const int* step_gate = nullptr;   // gate of the launches of the step being enqueued
    std::vector<const void*> view_key, eview_key;
    std::vector<EigTask> h_pre;   // host copy of the preconditioner's leaf tasks (batched solves)
    // eigenbasis leaf path
    bool eig = false;
    int eig_fused = 0;          // cluster size of the one-launch single-vector sweep (0: off)
    std::vector<CT*> EV, EXI, EFh, ESC;   // ESC: per-mode input scales (bilinear elements)
    std::vector<c128*> ELAM;
    // complex64 form: the sweep transforms' B operands for the tensor cores (V^T and V)
    bool tc = false;
    std::vector<void*> EVT, EVN;
    EigTask *d_etasks_view = nullptr, *d_etasks_own = nullptr, *d_etask_one = nullptr, *d_etasks_pre = nullptr;
    // flexible GMRES
    int mk = 0;                                   // restart length
    c128 *Vb = nullptr, *Zb = nullptr, *gw = nullptr, *gv = nullptr, *gz = nullptr, *gdots = nullptr,
         *gy = nullptr;
    c128* h_dots = nullptr;                       // pinned host copy of the dot products
    GmresLs gls{};                                // the cycle's least-squares problem (device)
    GmresState* h_gst = nullptr;                  // pinned snapshots of its state, GM_SLOTS
    static constexpr int GM_SLOTS = 4, GM_LAG = 2;
    cudaEvent_t gm_ev[GM_SLOTS] = {};
    // captured graphs of the preconditioner step (slot 0: gv -> gz for GMRES, slot 1:
    // the stationary update of u, slot 2: one step of the device-tested loop, update and
    // residual)
    struct Graph {
        cudaGraph_t graph = nullptr;   // kept: its event-record nodes address the exec's
        cudaGraphExec_t exec = nullptr;
        bool failed = false;
        bool replayed = false;
        unsigned long long nkern = 0;  // kernels in the graph
        std::vector<EvPair> prof;      // pairs stamped by the captured event-record nodes
        // event-record nodes of the profiler pairs: (node, 2 * pair + (0: a, 1: b))
        std::vector<std::pair<cudaGraphNode_t, int>> evnode;
        // replays launched with fresh events (replay_fresh), in launch order
        std::vector<std::vector<EvPair>> runs;
    };
    Graph graphs[3];
    cudaStream_t cap_stream = nullptr;   // private stream the graphs are captured on
    void** d_ptrs = nullptr;
    void* h_pin = nullptr;      // pinned block holding h_norm and h_dots
    double* h_norm = nullptr;   // pinned host
    int b_max = 0;
    cudaError_t cerr = cudaSuccess;

    ~Solver() override {
        for (auto& g : graphs) {
            if (g.exec) cudaGraphExecDestroy(g.exec);
            if (g.graph) cudaGraphDestroy(g.graph);
            for (auto& p : g.prof) { prof_pool.push_back(p.a); if (p.b) prof_pool.push_back(p.b); }
            runs_release(g, 0);
        }
        if (cap_stream) cudaStreamDestroy(cap_stream);
        if (block) dev_free(block, footprint, stream, hook);
        if (stream) cudaStreamSynchronize(stream);
        pinned_put(h_pin);   // nothing copies into it any more
        for (auto& e : gm_ev)
            if (e) cudaEventDestroy(e);
    }

    // the mixed form's opt-in FP32 Galerkin products and coarse elimination
    bool coarse_fp32() const { return sizeof(CT) != sizeof(c128) && (P.flags & HH_FLAG_COARSE_FP32); }
    int q1() const { return (P.flags & HH_FLAG_BILINEAR) ? 1 : 0; }   // bilinear elements
    OpGeom geom(int id) const { return OpGeom{nodes[id].b(), Sx, kh, khr_at(nodes[id].ra), q1()}; }
    const double* khr_at(int grow) const { return khr_dev ? khr_dev + grow : nullptr; }
    size_t pts(int id) const { return (size_t)nodes[id].b() * Sx; }
    size_t row_off(int id, int grow, int nc) const { return (size_t)(grow - nodes[id].ra) * Sx * nc; }

    void init_geometry() {
        S = P.n + 2;
        Sy = S;
        Sx = P.dim == 2 ? S : 1;
        h = 1.0 / (P.n + 1);
        kh = P.k * h;
        L = P.levels;
        e = P.overlap / 2;
        m = std::min(P.rank + P.oversample, Sx);
        r = std::min(P.rank, m);
        nmax = std::max(m, 4);   // columns of every node buffer (>= r + p)
        build_tree(S, L, e, nodes);
        nn = (int)nodes.size();
        lev.assign(L + 1, {});
        for (auto& nd : nodes) lev[nd.level].push_back(nd.id);
        b_max = 0;
        for (auto& nd : nodes)
            if (nd.leaf()) b_max = std::max(b_max, nd.b());
        eig = (Sx > 1 && P.leaf_solver == HH_LEAF_EIGEN);
        tc = eig && sizeof(CT) == sizeof(c64) && !(P.flags & HH_FLAG_CUDA_CORE_SWEEPS);
        mk = P.outer == HH_OUTER_GMRES ? P.restart : 0;
    }

    size_t plan(char* base) override {
        Arena a;
        a.base = base;
        W.assign(nn, nullptr); R.assign(nn, nullptr); Vs.assign(nn, nullptr); C.assign(nn, nullptr);
        X.assign(nn, nullptr); Om.assign(nn, nullptr); Z.assign(nn, nullptr); Vc.assign(nn, nullptr);
        Ainv.assign(nn, nullptr); ycoef.assign(nn, nullptr); Gm.assign(nn, nullptr); U.assign(nn, nullptr);
        AinvT.assign(nn, nullptr);
        lam.assign(nn, nullptr); ldx.assign(nn, 0);
        EV.assign(nn, nullptr); EXI.assign(nn, nullptr); EFh.assign(nn, nullptr); ESC.assign(nn, nullptr);
        EVT.assign(nn, nullptr); EVN.assign(nn, nullptr);
        ELAM.assign(nn, nullptr);
        const size_t N = (size_t)Sy * Sx;
        u = a.take<c128>(N); ut = a.take<c128>(N); bvec = a.take<c128>(N); res = a.take<c128>(N);
        dlt = a.take<CT>(N);
        if (recur_possible()) {
            AC0 = a.take<CT>(N * 2 * (size_t)r);
            RP = a.take<CT>(N);
        }
        gbuf = a.take<c128>(4 * (size_t)S);
        khr_dev = P.k_rows ? a.take<double>(S) : nullptr;
        RT = a.take<CT>(N * nmax);
        for (auto& nd : nodes) {
            const int id = nd.id;
            const size_t np = pts(id);
            if (id != 0) {
                W[id] = a.take<CT>(np * nmax);
                Vs[id] = a.take<CT>(np * nmax);
                Om[id] = a.take<CT>((size_t)Sx * nmax);
                Z[id] = a.take<CT>((size_t)Sx * nmax);
                Vc[id] = a.take<CT>((size_t)Sx * std::max(r, 1));
                Gm[id] = a.take<c128>((size_t)m * m + 4 * (size_t)m);   // + eigensolver workspace
                U[id] = a.take<c128>((size_t)m * m);
                lam[id] = a.take<double>(m);
            }
            if (!nd.leaf()) {
                if (id != 0) R[id] = a.take<CT>(np * nmax);
                C[id] = a.take<CT>(np * 2 * r);
                Ainv[id] = a.take<c128>((size_t)4 * r * r);
                AinvT[id] = sizeof(CT) == sizeof(c128) ? (CT*)Ainv[id] : a.take<CT>((size_t)4 * r * r);
                ycoef[id] = a.take<c128>((size_t)2 * r * nmax);
            } else if (eig) {
                const int b = nd.b();
                EV[id] = a.take<CT>((size_t)b * b);
                EXI[id] = a.take<CT>((size_t)Sx * b);
                ELAM[id] = a.take<c128>(b);
                EFh[id] = a.take<CT>(np * nmax);
                if (q1()) ESC[id] = a.take<CT>(b);
                if (tc) {
                    EVT[id] = a.take<unsigned char>(tc_vemb_bytes(b_max));
                    EVN[id] = a.take<unsigned char>(tc_vemb_bytes(b_max));
                }
            } else {
                ldx[id] = leaf_ldx(nd.b(), (int)sizeof(CT));
                X[id] = a.take<CT>(Sx == 1 ? (size_t)nd.b() : (size_t)Sx * nd.b() * ldx[id]);
            }
        }
        R[0] = RT;
        cur_in.assign(nn, nullptr);
        cur_in[0] = RT;
        // per-block partial sums of up to 64 x 64 outputs, plus the block of sums that
        // launch_ip_reduce writes just past the partials
        partial = a.take<c128>((size_t)(MAX_PART_BLOCKS + 1) * 64 * 64);
        npart = a.take<double>(2048);
        // [0] ||r||^2 (FP64 residual), [1] ||r||^2 (recursive residual), [2..4) ||b||^2,
        // [4..6) the device status words, [6..10) the device-tested loop's control words
        dnorm = a.take<double>(10);
        derr = (int*)(dnorm + 4);
        dcounter = a.take<unsigned>(4);
        const int nleaf = 1 << L;
        d_tasks_view = a.take<LeafTask>(nleaf);
        d_tasks_own = a.take<LeafTask>(nleaf);
        d_task_one = a.take<LeafTask>(1);
        d_tasks_pre = a.take<LeafTask>(nleaf);
        d_etasks_pre = a.take<EigTask>(nleaf);
        d_etasks_view = a.take<EigTask>(nleaf);
        d_etasks_own = a.take<EigTask>(nleaf);
        d_etask_one = a.take<EigTask>(1);
        if (mk > 0) {
            Vb = a.take<c128>(N * (mk + 1));
            Zb = a.take<c128>(N * mk);
            gw = a.take<c128>(N);
            gv = a.take<c128>(N);
            gz = a.take<c128>(N);
            gdots = a.take<c128>(4 * 80);
            gy = a.take<c128>(80);
            gls.mk = mk;
            gls.H = a.take<c128>((size_t)(mk + 1) * mk);
            gls.cs = a.take<double>(mk);
            gls.sn = a.take<c128>(mk);
            gls.g = a.take<c128>(mk + 1);
            gls.st = a.take<GmresState>(1);
        }
        d_ptrs = a.take<void*>(3 * 64);
        return align_up(a.off, 256);
    }

    // ------------------------------------------------------------- small helpers
    bool sync_check(hh_status& st) {
        ck(cudaGetLastError(), cerr);
        ck(cudaStreamSynchronize(stream), cerr);
        if (cerr != cudaSuccess) { st = HH_ECUDA; return false; }
        int e2 = 0;
        ck(cudaMemcpy(&e2, derr, sizeof(int), cudaMemcpyDeviceToHost), cerr);
        if (e2 == DEV_BREAKDOWN) { st = HH_EBREAKDOWN; return false; }
        if (e2 == DEV_TIMEOUT) { st = HH_ETIMEOUT; return false; }
        if (e2 == DEV_BADARG) { st = HH_EINVAL; return false; }
        st = HH_OK;
        return true;
    }
    void zero(void* p, size_t bytes) { ck(cudaMemsetAsync(p, 0, bytes, stream), cerr); }
    void d2d(void* dst, const void* src, size_t bytes) {
        ck(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, stream), cerr);
    }

    std::vector<LeafTask> leaf_tasks(bool own) const {
        std::vector<LeafTask> t;
        for (int id : lev[L]) {
            const Node& nd = nodes[id];
            LeafTask k{};
            k.X = X[id];
            k.W = W[id];
            k.b = nd.b();
            k.ldx = ldx[id];
            k.khr = khr_at(nd.ra);
            if (own) k.F = Vs[id];
            else k.F = R[nd.parent] + (size_t)(nd.ra - nodes[nd.parent].ra) * Sx * 0;  // fixed per call
            t.push_back(k);
        }
        return t;
    }
    // The view tasks depend on the column count (row stride = Sx * nc).
    // Leaf input of the current apply: R_leaf of the parent's input (n_i = 1) or of the
    // parent's residual buffer.
    const CT* leaf_input(int id, int nc) const {
        const int p = nodes[id].parent;
        return src_of(p) + row_off(p, nodes[id].ra, nc);
    }
    void upload_view_tasks(int nc) {
        std::vector<LeafTask> t;
        std::vector<const void*> key{(const void*)(size_t)nc};
        for (int id : lev[L]) {
            const Node& nd = nodes[id];
            LeafTask k{};
            k.X = X[id];
            k.W = W[id];
            k.b = nd.b();
            k.ldx = ldx[id];
            k.khr = khr_at(nd.ra);
            k.F = leaf_input(id, nc);
            key.push_back(k.F);
            t.push_back(k);
        }
        if (key == view_key) return;
        view_key = key;
        ck(cudaMemcpyAsync(d_tasks_view, t.data(), sizeof(LeafTask) * t.size(), cudaMemcpyHostToDevice, stream),
           cerr);
    }
    EigTask eig_task(int id, const void* F, void* Wout) const {
        EigTask k{};
        k.V = EV[id];
        k.xi = EXI[id];
        k.lam = ELAM[id];
        k.F = F;
        k.Fh = EFh[id];
        k.W = Wout;
        k.b = nodes[id].b();
        k.Sx = Sx;
        k.w0 = 0;
        k.w1 = k.b;
        k.vt_emb = EVT[id];
        k.vn_emb = EVN[id];
        k.sc = ESC[id];
        return k;
    }
    // Cluster size of the one-launch single-vector sweep, 16 or 8 CTAs per leaf, timed on
    // this handle's preconditioner tasks at the end of its set-up (their outputs are scratch
    // there) where both fit.
    void tune_fused_cluster() {
        if (!eig || !eig_fused || !pre_direct || stream_capturing(stream)) return;
        const int nl = (int)lev[L].size();
        const TuneKey key{current_device(), 1, b_max, Sx, nl, (int)sizeof(T)};
        int choice = 0;
        if (!tune_find(key, choice)) {
            if (!eig_sweep_fused_feasible<T>(16, b_max, Sx) || !eig_sweep_fused_feasible<T>(8, b_max, Sx)) return;
            TuneEntry e{};
            e.choice = tune_pair(stream, [&](int c) {
                launch_eig_sweep_fused<T>(c ? 8 : 16, d_etasks_pre, nl, b_max, Sx, stream);
            }, e.ms);
            tune_store(key, e);
            choice = e.choice;
        }
        eig_fused = choice ? 8 : 16;
    }
    // The three-stage sweep of several right-hand sides: transforms on the tensor cores
    // in the complex64 form, else on the CUDA cores; the line recursions in between.
    void eig_sweep_stage(int stg, const EigTask* tasks, int ntasks, int nc) {
        // inside a gated step (step_gate set) every launch is skipped once the stop word is set
        if (!tc || stg == 1) {
            launch_eig_sweep_stage<T>(stg, tasks, ntasks, b_max, Sx, nc, stream, step_gate);
            return;
        }
        // transforms: tensor cores or CUDA cores, as the autotuner found faster for this shape
        auto run = [&](int c) {
            if (c) launch_tc_transform(stg == 0 ? 0 : 1, tasks, ntasks, b_max, Sx, nc, derr, stream, step_gate);
            else launch_eig_sweep_stage<T>(stg, tasks, ntasks, b_max, Sx, nc, stream, step_gate);
        };
        const TuneKey key{current_device(), 0, stg, b_max, Sx, nc * 64 + std::min(ntasks, 63)};
        int choice = 1;
        if (P.flags & HH_FLAG_TENSOR_CORE_SWEEPS) choice = 1;
        else if (!tune_find(key, choice)) {
            if (stream_capturing(stream)) choice = 1;
            else {
                TuneEntry e{};
                e.choice = tune_pair(stream, run, e.ms);
                tune_store(key, e);
                choice = e.choice;
            }
        }
        run(choice);   // the outputs are those of the chosen candidate
    }
    void upload_eig_view_tasks(int nc) {
        std::vector<EigTask> t;
        std::vector<const void*> key{(const void*)(size_t)nc};
        for (int id : lev[L]) {
            t.push_back(eig_task(id, leaf_input(id, nc), W[id]));
            key.push_back(t.back().F);
        }
        if (key == eview_key) return;
        eview_key = key;
        ck(cudaMemcpyAsync(d_etasks_view, t.data(), sizeof(EigTask) * t.size(), cudaMemcpyHostToDevice, stream),
           cerr);
    }
    // Leaf tasks of the preconditioner step (one vector, from the root's residual RT),
    // fixed after set-up so that captured graphs can read them.  With n_i = 1 each leaf
    // writes its owned rows straight into its parent's solution (restricted prolongation
    // without a copy).
    void upload_pre_tasks() {
        const bool direct_in = P.n_inner == 1;
        pre_direct = eig && direct_in && L >= 2;
        std::vector<EigTask> et;
        std::vector<LeafTask> lt;
        for (int id : lev[L]) {
            const Node& nd = nodes[id];
            const int p = nd.parent;
            const CT* F = direct_in ? RT + row_off(0, nd.ra, 1) : R[p] + row_off(p, nd.ra, 1);
            if (eig) {
                EigTask k = eig_task(id, F, W[id]);
                if (pre_direct) {
                    k.W = W[p] + row_off(p, nd.own_a, 1);
                    k.w0 = nd.own_a - nd.ra;
                    k.w1 = nd.own_b - nd.ra;
                }
                et.push_back(k);
            } else {
                LeafTask k{};
                k.X = X[id];
                k.W = W[id];
                k.b = nd.b();
                k.ldx = ldx[id];
                k.khr = khr_at(nd.ra);
                k.F = F;
                lt.push_back(k);
            }
        }
        if (eig) {
            h_pre = et;
            ck(cudaMemcpyAsync(d_etasks_pre, et.data(), sizeof(EigTask) * et.size(), cudaMemcpyHostToDevice, stream),
               cerr);
        }
        else
            ck(cudaMemcpyAsync(d_tasks_pre, lt.data(), sizeof(LeafTask) * lt.size(), cudaMemcpyHostToDevice, stream),
               cerr);
    }
    // all leaves: W[leaf] = A~_leaf^{-1} F (F = own buffers or views into the parents)
    void leaf_sweep_all(int nc, bool own) {
        const int nl = (int)lev[L].size();
        if (eig) {
            const EigTask* tasks = d_etasks_own;
            if (!own) {
                if (in_pre && nc == 1) {
                    tasks = d_etasks_pre;
                } else {
                    upload_eig_view_tasks(nc);
                    tasks = d_etasks_view;
                }
            }
            if (nc == 1 && eig_fused) {
                // both transforms (16 b^2 Sx flops) and the recursions; V, f, xi read and
                // x written once: b^2 + 3 b Sx elements
                double by = 0.0, fl = 0.0;
                for (int id : lev[L]) {
                    const double b = nodes[id].b(), sx = Sx;
                    fl += 16.0 * b * b * sx;
                    by += sizeof(CT) * (b * b + 3.0 * b * sx);
                }
                pbeg(PC_SWEEP, by, fl);
                launch_eig_sweep_fused<T>(eig_fused, tasks, nl, b_max, Sx, stream, step_gate);
                pend(PC_SWEEP);
                return;
            }
            for (int stg = 0; stg < 3; ++stg) {
                // per leaf b x Sx x nc: transforms 8 b^2 Sx nc flops and (b^2 + 2 b Sx nc)
                // elements; recursions read xi (Sx b) and read/write the lines (2 b Sx nc)
                double by = 0.0, fl = 0.0;
                for (int id : lev[L]) {
                    const double b = nodes[id].b(), sx = Sx;
                    if (stg == 1) by += sizeof(CT) * (b * sx + 2.0 * b * sx * nc);
                    else { fl += 8.0 * b * b * sx * nc; by += sizeof(CT) * (b * b + 2.0 * b * sx * nc); }
                }
                pbeg(PC_TIN + stg, by, fl);
                eig_sweep_stage(stg, tasks, nl, nc);
                pend(PC_TIN + stg);
            }
            return;
        }
        const LeafTask* tasks = d_tasks_own;
        if (!own) {
            if (in_pre && nc == 1) {
                tasks = d_tasks_pre;
            } else {
                upload_view_tasks(nc);
                tasks = d_tasks_view;
            }
        }
        pbeg(PC_RECUR);
        launch_sweep<T>(tasks, nl, b_max, Sx, nc, derr, stream);
        pend(PC_RECUR);
    }

    // Buffer holding node p's input during the current apply: with n_i = 1 its input
    // itself (nothing is subtracted from it), else its residual buffer R[p].
    const CT* src_of(int p) const { return (P.n_inner == 1 && cur_in[p]) ? cur_in[p] : R[p]; }

    // Input of node id in an apply: its own buffer (top level of a multi-vector apply)
    // or its rows of the parent's input buffer.
    const CT* input(int id, int nc, bool own) const {
        if (own) return Vs[id];
        const int p = nodes[id].parent;
        return src_of(p) + row_off(p, nodes[id].ra, nc);
    }

    // ------------------------------------------------- sub-level solve M at level l
    void apply_M(int l, int nc, bool own) {
        if (l == L) {
            leaf_sweep_all(nc, own);
            return;
        }
        for (int p : lev[l]) cur_in[p] = input(p, nc, own);
        // preconditioner step with n_i = 1: every level's corrections in one launch, each
        // node writing its owned rows straight into its parent's solution
        const bool batch = in_pre && nc == 1 && P.n_inner == 1;
        const bool children_direct = batch && (l + 1 < L || pre_direct);
        for (int it = 0; it < P.n_inner; ++it) {
            for (int p : lev[l]) {
                if (it == 0) {
                    if (P.n_inner > 1) d2d(R[p], cur_in[p], sizeof(CT) * pts(p) * nc);
                } else {
                    launch_apply<T, T, T>(W[p], cur_in[p], R[p], geom(p), nc, 1.0, nullptr, nullptr, stream);
                }
            }
            apply_M(l + 1, nc, false);
            if (!children_direct) {
                for (int p : lev[l]) {
                    for (int c : nodes[p].child) {
                        const Node& cn = nodes[c];
                        const size_t n = (size_t)(cn.own_b - cn.own_a) * Sx * nc;
                        launch_copy<T, T>(W[c] + row_off(c, cn.own_a, nc), W[p] + row_off(p, cn.own_a, nc), n,
                                          it > 0, false, stream);
                    }
                }
            }
            if (batch) coarse_level_direct(l);
            else
                for (int p : lev[l]) coarse_correct(p, cur_in[p], nc);
        }
    }

    // The one-column corrections of all level-l nodes of the preconditioner step, each
    // written (owned rows, plus the node's own solution) into the parent: the root's
    // output for level 1, else the parent's W.
    void coarse_level_direct(int l) {
        const std::vector<int>& ps = lev[l];
        for (size_t k0 = 0; k0 < ps.size(); k0 += CB_MAX_JOBS) {
            CoarseBatch bt{};
            bt.gate = step_gate;
            double by = 0.0, fl = 0.0;
            for (size_t k = k0; k < ps.size() && k < k0 + CB_MAX_JOBS; ++k) {
                const int p = ps[k];
                const Node& nd = nodes[p];
                CoarseJob& j = bt.job[bt.njobs++];
                j.C = C[p];
                j.v = cur_in[p];
                j.w_in = W[p];
                j.out = l == 1 ? (void*)(root_out + row_off(0, nd.own_a, 1))
                               : (void*)(W[nd.parent] + row_off(nd.parent, nd.own_a, 1));
                j.Minv = AinvT[p];
                j.y = ycoef[p];
                j.g = geom(p);
                j.r0 = nd.own_a - nd.ra;
                j.r1 = nd.own_b - nd.ra;
                j.acc_out = l == 1 && root_acc;
                j.add_w = 1;
                j.split = split_row(p);
                // level 1 also keeps its update delta_1 for the root's correction
                j.dout = l == 1 ? (void*)(dlt + row_off(0, nd.own_a, 1)) : nullptr;
                by += coarse_bytes(p);
                fl += 2.0 * 8.0 * 2 * r * pts(p);
            }
            // the pair stays open: the step's next launches are the coarse corrections of
            // the levels above and the root's, which closes it (oras_step)
            pjoin(PC_COARSE, by, fl);
            if (l == 1) launch_coarse_batch<T, T, T, double>(bt, 2 * r, partial, dcounter + 2, derr, stream);
            else launch_coarse_batch<T, T, T, T>(bt, 2 * r, partial, dcounter + 2, derr, stream);
        }
    }

    // Algorithmic bytes of one one-column coarse correction of node p: each point of its
    // band lies in one child's owned rows and carries that child's r basis columns, read
    // once for C^H r and once for C y: 2 r n c bytes (n points, c bytes per element of the
    // basis precision).  The residual and update vectors are not counted.
    double coarse_bytes(int p) const { return 2.0 * r * (double)pts(p) * sizeof(CT); }

    // local row of node p where its second child's owned rows (and basis columns) begin
    int split_row(int p) const { return nodes[nodes[p].child[1]].own_a - nodes[p].ra; }

    // out (+)= C_p A_c^{-1} C_p^H (v - A~_p w) over node p's band, one column
    CoarseBatch one_job(int p, const void* v, const void* w, void* out, bool acc) const {
        CoarseBatch bt{};
        CoarseJob& j = bt.job[0];
        j.C = C[p];
        j.v = v;
        j.w_in = w;
        j.out = out;
        j.Minv = AinvT[p];
        j.y = ycoef[p];
        j.g = geom(p);
        j.r0 = 0;
        j.r1 = nodes[p].b();
        j.acc_out = acc;
        j.add_w = 0;
        j.split = split_row(p);
        bt.njobs = 1;
        return bt;
    }

    // W[p] += C_p A_c^{-1} C_p^H (v - A~_p W[p])
    void coarse_correct(int p, const CT* vin, int nc) {
        if (nc == 1) {
            pbeg(PC_COARSE, coarse_bytes(p), 2.0 * 8.0 * 2 * r * pts(p));
            launch_coarse_batch<T, T, T, T>(one_job(p, vin, W[p], W[p], true), 2 * r, partial, dcounter + 2, derr,
                                            stream);
            pend(PC_COARSE);
            return;
        }
        launch_apply<T, T, T>(W[p], vin, R[p], geom(p), nc, 1.0, nullptr, nullptr, stream);
        pbeg(PC_COARSE_MC, (double)pts(p) * (2.0 * r + nc) * sizeof(CT), 8.0 * 2 * r * nc * pts(p));
        const int nb = launch_ip_partial_colA<T, T, T>(C[p], R[p], nc, pts(p), 2 * r, nc, partial, MAX_PART_BLOCKS,
                                                       stream, (long long)split_row(p) * Sx);
        pend(PC_COARSE_MC);
        launch_ip_reduce(partial, nb, 2 * r, nc, nullptr, Ainv[p], ycoef[p], stream);
        launch_coarse_updn<T, T>(C[p], ycoef[p], W[p], pts(p), 2 * r, nc, stream, (long long)split_row(p) * Sx);
    }

    // ------------------------------------------------------------------ set-up
    void sketch_level(int l) {   // children at level l of the nodes at level l-1
        const std::vector<int>& cs = lev[l];
        // Y = T_c Omega
        for (int c : cs) {
            const Node& cn = nodes[c];
            launch_sketch<T>(Om[c], Sx, m, c, P.seed, stream);
            zero(Vs[c], sizeof(CT) * pts(c) * m);
            d2d(Vs[c] + row_off(c, cn.ifrow, m), Om[c], sizeof(CT) * Sx * m);
        }
        apply_M(l, m, true);
        for (int c : cs) {
            const Node& cn = nodes[c];
            const Node& sn = nodes[cn.sib];
            launch_robin_trace<T>(W[c] + row_off(c, sn.ifrow, m), W[c] + row_off(c, sn.inward, m), Om[c], sn.b(), Sx,
                                  m, kh, khr_at(sn.ifrow), stream, q1());
        }
        // Q = orth(Y)
        std::vector<CT*> ys;
        for (int c : cs) ys.push_back(Om[c]);
        pbeg(PC_QR);
        launch_qr<T>(ys.data(), (int)ys.size(), Sx, m, (CT**)d_ptrs, stream);
        pend(PC_QR);
        // Z = T_c^* Q = B_c conj(M_c conj(A~_s B_s^T ... )) ; here as conj(M_c(A~_s B_s^T conj Q))
        for (int c : cs) {
            const Node& cn = nodes[c];
            const Node& sn = nodes[cn.sib];
            zero(Vs[c], sizeof(CT) * pts(c) * m);
            launch_adjoint_place<T>(Om[c], Vs[c] + row_off(c, sn.ifrow, m), Vs[c] + row_off(c, sn.inward, m), sn.b(),
                                    Sx, m, kh, khr_at(sn.ifrow), stream, q1());
        }
        apply_M(l, m, true);
        for (int c : cs)
            launch_copy<T, T>(W[c] + row_off(c, nodes[c].ifrow, m), Z[c], (size_t)Sx * m, false, true, stream);
        // SVD of Z^H = Q^H T: Gram Z^H Z (FP64), its Hermitian eigenproblem, V = Z U Sigma^{-1}
        for (int c : cs) {
            // Gram matrix Z^H Z of the stored sketch in FP64 (the complex64 sketch widens
            // exactly), so that forming it squares no FP32 rounding into the small singular
            // values; the SVD that follows is FP64 as well
            const int nb = launch_ip_partial<T, T, double>(Z[c], m, Z[c], m, Sx, m, m, partial, MAX_PART_BLOCKS,
                                                           stream);
            launch_ip_reduce(partial, nb, m, m, Gm[c], nullptr, nullptr, stream);
        }
        std::vector<c128*> gs, us;
        std::vector<double*> ls;
        for (int c : cs) { gs.push_back(Gm[c]); us.push_back(U[c]); ls.push_back(lam[c]); }
        pbeg(PC_JACOBI);
        launch_heig(gs.data(), us.data(), ls.data(), (int)cs.size(), m, r, d_ptrs, stream);
        pend(PC_JACOBI);
        for (int c : cs) launch_form_v<T>(Z[c], U[c], lam[c], Vc[c], Sx, m, r, stream);
        // C_c = P_c M_c B_c^T V_c
        for (int c : cs) {
            zero(Vs[c], sizeof(CT) * pts(c) * r);
            d2d(Vs[c] + row_off(c, nodes[c].ifrow, r), Vc[c], sizeof(CT) * Sx * r);
        }
        apply_M(l, r, true);
        for (int p : lev[l - 1]) {
            zero(C[p], sizeof(CT) * pts(p) * 2 * r);
            for (int k = 0; k < 2; ++k) {
                const int c = nodes[p].child[k];
                const Node& cn = nodes[c];
                launch_build_basis<T>(W[c], (size_t)(cn.own_a - cn.ra) * Sx, r, C[p], pts(p), k * r,
                                      (size_t)(cn.own_a - nodes[p].ra) * Sx, (size_t)(cn.own_b - cn.own_a) * Sx,
                                      stream);
            }
            // A_c = C_p^H A~_p C_p, then its inverse.  Algorithmic work: a point in one child's
            // rows pairs that child's r columns of conj(C) with r columns of A~ C, complex
            // products of 8 real flops: r^2 of them (the two rows next to the split pair r with
            // 2r), or r (r + 1) / 2 in the Hermitian-packed form of the FP64 5-point products
            // (the row before the split adds r^2)
            const bool herm_form = !coarse_fp32() && !q1();
            pbeg(PC_GALERKIN, (double)pts(p) * 2 * r * sizeof(CT),
                 herm_form ? 8.0 * (0.5 * r * (r + 1.0) * pts(p) + (double)r * r * Sx)
                           : 8.0 * r * r * (pts(p) + 2.0 * Sx));
            const int split = nodes[nodes[p].child[1]].own_a - nodes[p].ra;
            // FP64 products from the stored basis, or FP32 ones in the opt-in FP32 coarse
            // variant of the mixed form
            bool herm = false;
            const int nb = coarse_fp32()
                               ? launch_galerkin_partial<T, T>(C[p], geom(p), 2 * r, split, partial, MAX_PART_BLOCKS,
                                                               stream)
                               : launch_galerkin_partial<T, double>(C[p], geom(p), 2 * r, split, partial,
                                                                    MAX_PART_BLOCKS, stream, &herm);
            pend(PC_GALERKIN);
            launch_ip_reduce(partial, nb, 2 * r, 2 * r, Ainv[p], nullptr, nullptr, stream);
            if (herm) launch_herm_fill(Ainv[p], 2 * r, stream);
        }
        // the level's Galerkin matrices inverted together
        GjBatch bt{};
        bt.n = 2 * r;
        bt.err = derr;
        int cnt = 0;
        // FP64 elimination in both forms (the opt-in FP32 coarse variant eliminates in
        // FP32); the complex64 form also gets the inverse rounded to complex64 for its
        // one-column corrections
        const bool c64 = sizeof(CT) != sizeof(c128);
        for (int p : lev[l - 1]) {
            bt.A[cnt] = Ainv[p];
            bt.AT[cnt++] = c64 ? (void*)AinvT[p] : nullptr;
        }
        launch_gj_inverse(bt, cnt, coarse_fp32(), stream);
    }

    hh_status setup() override {
        if (khr_dev) {
            // layered media: k h per grid row (the caller's k_rows times h)
            std::vector<double> khr(S);
            for (int j = 0; j < S; ++j) khr[j] = P.k_rows[j] * h;
            ck(cudaMemcpyAsync(khr_dev, khr.data(), sizeof(double) * S, cudaMemcpyHostToDevice, stream), cerr);
            ck(cudaStreamSynchronize(stream), cerr);
        }
        eig_fused = eig ? eig_sweep_fused_ready<T>(b_max, Sx) : 0;
        if (tc && !tc_transform_ready()) return HH_ECUDA;
        zero(derr, sizeof(int) * 4);
        zero(dcounter, sizeof(unsigned) * 4);
        for (int id = 1; id < nn; ++id) zero(Vs[id], sizeof(CT) * pts(id) * nmax);
        if (eig) {
            std::vector<EigTask> own;
            for (int id : lev[L]) own.push_back(eig_task(id, Vs[id], W[id]));
            ck(cudaMemcpyAsync(d_etasks_own, own.data(), sizeof(EigTask) * own.size(), cudaMemcpyHostToDevice,
                               stream),
               cerr);
        } else {
            std::vector<LeafTask> own = leaf_tasks(true);
            ck(cudaMemcpyAsync(d_tasks_own, own.data(), sizeof(LeafTask) * own.size(), cudaMemcpyHostToDevice,
                               stream),
               cerr);
        }
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        cudaEventRecord(e0, stream);
        pbeg(PC_FACTOR);
        if (eig) launch_eig_factor<T>(d_etasks_own, (int)lev[L].size(), b_max, Sx, kh, derr, stream, q1());
        else launch_factor<T>(d_tasks_own, (int)lev[L].size(), b_max, Sx, kh, derr, stream);
        if (tc) launch_tc_prepare_v(d_etasks_own, (int)lev[L].size(), b_max, stream);
        pend(PC_FACTOR);
        for (int l = L; l >= 1; --l) sketch_level(l);
        upload_pre_tasks();
        tune_fused_cluster();
        if (device_test_path() && recur_possible()) launch_apply_cols<T>(C[0], AC0, geom(0), 2 * r, stream);
        cudaEventRecord(e1, stream);
        hh_status st;
        const bool ok = sync_check(st);
        prof_collect();
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        t_setup_ms = ms;
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (!ok) return st;
        // one pinned block: the norms (8 doubles) at 0, the dot products (320 complex) at 256
        // and GM_SLOTS snapshots of the GMRES state after them
        static_assert(256 + 4 * 80 * sizeof(c128) + GM_SLOTS * sizeof(GmresState) <= PIN_BLOCK,
                      "pinned block too small");
        h_pin = pinned_get();
        if (!h_pin) return HH_ENOMEM;
        h_norm = (double*)h_pin;
        if (mk > 0) {
            h_dots = (c128*)((char*)h_pin + 256);
            h_gst = (GmresState*)((char*)h_pin + 256 + 4 * 80 * sizeof(c128));
            for (auto& e : gm_ev)
                if (!e) ck(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), cerr);
        }
        return cerr == cudaSuccess ? HH_OK : HH_ECUDA;
    }

    // --------------------------------------------------------- the outer iteration
    // One coarse-corrected ORAS step from the FP64 residual kept in res (and already in
    // RT, the leaf precision, when rt_ready):
    // out = base + sum_c P_c M_c R_c res (base null: zero; base may be out), then
    // out += C A_c^{-1} C^H (rhs - A out).
    // recur: the root's extras forming the next residual recursively (null: none)
    void oras_step(const c128* base, const c128* rhs, c128* out, bool rt_ready = false, const int* gate = nullptr,
                   const CoarseRecur* recur = nullptr) {
        const size_t N = (size_t)Sy * Sx;
        step_gate = gate;
        if (!rt_ready) launch_copy<double, T>(res, RT, N, false, false, stream);
        // with n_i = 1 (and a level below the root's children) the level-1 corrections
        // write out = base + sum_c P_c M_c R_c res themselves
        const bool direct = P.n_inner == 1 && L >= 2;
        if (base && base != out) d2d(out, base, sizeof(c128) * N);
        root_out = out;
        root_acc = base != nullptr;
        in_pre = true;
        apply_M(1, 1, false);
        in_pre = false;
        if (!direct) {
            // the level-1 owned rows partition the grid, so with no base the copies
            // initialise out
            for (int c : lev[1]) {
                const Node& cn = nodes[c];
                launch_copy<T, double>(W[c] + row_off(c, cn.own_a, 1), out + row_off(0, cn.own_a, 1),
                                       (size_t)(cn.own_b - cn.own_a) * Sx, base != nullptr, false, stream);
            }
        }
        if (direct) {
            // The root corrects on the residual after the level-1 update, rhs - A(base +
            // delta_1) = res - A delta_1: the step's input residual (RT, in the leaf
            // precision) less A applied to the update the level-1 kernel kept in dlt.
            // Both terms are in the leaf precision, like the correction computed from them;
            // the FP64 residual of the new iterate is formed afterwards as before.
            // with the recursive residual also r' kept, the r columns of A C_0 at each point
            // read and the next residual written; r complex multiply-adds per point
            pjoin(PC_COARSE, coarse_bytes(0), 2.0 * 8.0 * 2 * r * N + (recur ? 8.0 * r * N : 0.0));
            CoarseBatch rb = one_job(0, RT, dlt, out, true);
            rb.gate = gate;
            if (recur) rb.rr = *recur;
            launch_coarse_batch<T, T, T, double>(rb, 2 * r, partial, dcounter + 2, derr, stream);
        } else {
            pjoin(PC_COARSE, coarse_bytes(0), 2.0 * 8.0 * 2 * r * N);
            CoarseBatch rb = one_job(0, rhs, out, out, true);
            rb.gate = gate;
            launch_coarse_batch<T, double, double, double>(rb, 2 * r, partial, dcounter + 2, derr, stream);
        }
        pend(PC_COARSE);
        step_gate = nullptr;
    }

    hh_status norm_sq(const c128* x, double* dst) {
        const size_t N = (size_t)Sy * Sx;
        const int nb = launch_ip_partial<double, double>(x, 1, x, 1, N, 1, 1, partial, MAX_PART_BLOCKS, stream);
        launch_ip_reduce(partial, nb, 1, 1, (c128*)dst, nullptr, nullptr, stream);
        return HH_OK;
    }

    // z = M v: one coarse-corrected ORAS step from zero (v, z distinct from res and ut)
    void precond(const c128* v, c128* z) {
        d2d(res, v, sizeof(c128) * (size_t)Sy * Sx);
        oras_step(nullptr, v, z);
    }

    // Runs `body` through a CUDA graph: the first call runs it directly (which also
    // performs any one-time uploads and attribute settings) and then captures it; later
    // calls replay the graph.  Buffers used by `body` must not change between calls.
    template <class F> void via_graph(int slot, F body) {
        Graph& g = graphs[slot];
        if (g.exec) {
            cudaGraphLaunch(g.exec, stream);
            g_launches.fetch_add(g.nkern, std::memory_order_relaxed);
            g.replayed = true;
            return;
        }
        body();
        if (g.failed) return;
        cudaGraph_t graph = nullptr;
        const size_t npend = prof_pending.size();
        const unsigned long long l0 = t_launches;
        // captured on a private stream (the caller's may be the legacy default stream,
        // which cannot be captured); replays go to the caller's stream
        if (!cap_stream && cudaStreamCreateWithFlags(&cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            cap_stream = nullptr;
            g.failed = true;
            return;
        }
        const cudaStream_t user = stream;
        stream = cap_stream;
        if (cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaGetLastError();
            stream = user;
            g.failed = true;
            return;
        }
        body();
        const cudaError_t e1 = cudaStreamEndCapture(stream, &graph);
        stream = user;
        if (e1 != cudaSuccess || !graph || cudaGraphInstantiate(&g.exec, graph, 0) != cudaSuccess) {
            cudaGetLastError();
            g.failed = true;
            g.exec = nullptr;
        }
        // the captured body launched nothing: its kernels count at each replay
        g.nkern = t_launches - l0;
        g_launches.fetch_sub(g.nkern, std::memory_order_relaxed);
        // the pairs recorded during capture belong to the graph
        g.prof.assign(prof_pending.begin() + npend, prof_pending.end());
        prof_pending.resize(npend);
        if (g.exec && !g.prof.empty()) {
            // find the event-record nodes, so that replays can stamp fresh events
            size_t cnt = 0;
            cudaGraphGetNodes(graph, nullptr, &cnt);
            std::vector<cudaGraphNode_t> nd(cnt);
            if (cnt && cudaGraphGetNodes(graph, nd.data(), &cnt) == cudaSuccess) {
                for (size_t i = 0; i < cnt; ++i) {
                    cudaGraphNodeType ty;
                    cudaEvent_t ev = nullptr;
                    if (cudaGraphNodeGetType(nd[i], &ty) != cudaSuccess || ty != cudaGraphNodeTypeEventRecord ||
                        cudaGraphEventRecordNodeGetEvent(nd[i], &ev) != cudaSuccess)
                        continue;
                    for (size_t k = 0; k < g.prof.size(); ++k) {
                        if (g.prof[k].a == ev) g.evnode.push_back({nd[i], (int)(2 * k)});
                        else if (g.prof[k].b == ev) g.evnode.push_back({nd[i], (int)(2 * k + 1)});
                    }
                }
            }
            cudaGetLastError();
        }
        if (g.exec) g.graph = graph;
        else if (graph) cudaGraphDestroy(graph);
    }

    // Replay of graph slot `slot` whose profiler pairs get fresh events (several replays
    // may then be in flight before the host reads them); the pairs are kept in g.runs.
    // The first call for a slot runs `body` and captures it, as via_graph does.
    template <class F> void replay_fresh(int slot, F body) {
        Graph& g = graphs[slot];
        if (!g.exec) {
            via_graph(slot, body);
            return;
        }
        if (prof_on && !g.prof.empty() && g.evnode.size() == 2 * g.prof.size()) {
            std::vector<EvPair> v = g.prof;
            for (auto& p : v) {
                p.a = prof_ev();
                p.b = prof_ev();
            }
            bool ok = true;
            for (auto& [node, k] : g.evnode)
                ok = ok && cudaGraphExecEventRecordNodeSetEvent(g.exec, node, (k & 1) ? v[k >> 1].b : v[k >> 1].a) ==
                               cudaSuccess;
            if (ok) {
                g.runs.push_back(std::move(v));
            } else {
                // not settable: replays keep stamping the captured events (only the last
                // replay before a read is then timed)
                cudaGetLastError();
                g.evnode.clear();
                for (auto& p : v) { prof_pool.push_back(p.a); prof_pool.push_back(p.b); }
            }
        }
        cudaGraphLaunch(g.exec, stream);
        g_launches.fetch_add(g.nkern, std::memory_order_relaxed);
    }
    void drop_graphs() override {
        if (stream) cudaStreamSynchronize(stream);
        for (auto& g : graphs) {
            if (g.exec) cudaGraphExecDestroy(g.exec);
            if (g.graph) cudaGraphDestroy(g.graph);
            for (auto& p : g.prof) { prof_pool.push_back(p.a); if (p.b) prof_pool.push_back(p.b); }
            runs_release(g, 0);
            g = Graph{};
        }
    }
    // after a synchronisation: account the first `keep` replays of g.runs (those that
    // did work) and return every event of g.runs to the pool
    void runs_release(Graph& g, size_t keep) {
        for (size_t i = 0; i < g.runs.size(); ++i) {
            for (auto& p : g.runs[i]) {
                if (i < keep) prof_account(p);
                prof_pool.push_back(p.a);
                if (p.b) prof_pool.push_back(p.b);
            }
        }
        g.runs.clear();
    }
    // after a synchronisation: account the graphs' profiler events of the last replay
    void graphs_collect() {
        for (auto& g : graphs) {
            if (g.replayed && prof_on) prof_read_pairs(g.prof);
            g.replayed = false;
        }
    }

    // ||b - A u||^2 into h_norm[0] (synchronises); ||b||^2 must be in dnorm[2].
    bool true_residual(c128* dst, hh_status& st, CT* dst_t = nullptr) {
        int nb = 0;
        pbeg(PC_SPMV, 48.0 * (double)Sy * Sx);
        if (dst_t) launch_residual_cast<T>(u, bvec, dst, dst_t, geom(0), npart, &nb, stream);
        else launch_apply<double, double, double>(u, bvec, dst, geom(0), 1, 1.0, npart, &nb, stream);
        pend(PC_SPMV);
        launch_sum(npart, nb, dnorm, stream);
        // the norms and the device status words in one copy
        ck(cudaMemcpyAsync(h_norm, dnorm, 8 * sizeof(double), cudaMemcpyDeviceToHost, stream), cerr);
        ck(cudaGetLastError(), cerr);
        ck(cudaStreamSynchronize(stream), cerr);
        bool ok = cerr == cudaSuccess;
        if (!ok) st = HH_ECUDA;
        else {
            const int e2 = *(const int*)(h_norm + 4);
            st = e2 == DEV_BREAKDOWN ? HH_EBREAKDOWN : e2 == DEV_TIMEOUT ? HH_ETIMEOUT : e2 == DEV_BADARG ? HH_EINVAL
                                                                                                     : HH_OK;
            ok = st == HH_OK;
        }
        graphs_collect();
        return ok;
    }

    // The launches of one stationary step on the fast path (n_i = 1, fused eigenbasis
    // leaf sweeps writing into the parents, L >= 2) are the leaf sweep and the batched
    // coarse corrections: all of them, and the residual that follows, take a gate.
    // (the one-launch sweep and the three-stage one both take the stop word)
    bool device_test_path() const {
        return eig && pre_direct && P.n_inner == 1 && L >= 2 && P.outer == HH_OUTER_ORAS;
    }

    // residual b - A u into RT (the step's input; the FP64 vector itself is not kept), its
    // norm and the device stopping test (ctl), one launch; dcounter[0] is its ticket
    void gated_residual(int* ctl, const int* need = nullptr, const int* anchor = nullptr) {
        pbeg(PC_SPMV, 48.0 * (double)Sy * Sx);
        launch_residual_stop<T>(u, bvec, nullptr, RT, geom(0), npart, dnorm, ctl, dcounter, P.tol, stream, need, anchor);
        pend(PC_SPMV);
    }

    // the norms, the status words and the stop words (dnorm[0..8)) to the host
    bool read_norms(hh_status& st) {
        ck(cudaMemcpyAsync(h_norm, dnorm, 10 * sizeof(double), cudaMemcpyDeviceToHost, stream), cerr);
        ck(cudaGetLastError(), cerr);
        ck(cudaStreamSynchronize(stream), cerr);
        if (cerr != cudaSuccess) { st = HH_ECUDA; return false; }
        const int e2 = *(const int*)(h_norm + 4);
        st = e2 == DEV_BREAKDOWN ? HH_EBREAKDOWN : e2 == DEV_TIMEOUT ? HH_ETIMEOUT : e2 == DEV_BADARG ? HH_EINVAL
                                                                                                 : HH_OK;
        return st == HH_OK;
    }

    // Stationary iteration u <- u + M (b - A u) (Eqs. (2)-(3)) with the stopping test on
    // the device.  Each step (update, residual, test) is gated by the stop word the
    // previous test sets, so the host queues several steps per synchronisation: a step
    // queued after the test passed does nothing, and u, the iteration count and the
    // final residual are those of the loop that tests after every step.  The number of
    // steps queued follows the contraction observed so far.
    //
    // In the complex64 form the residual that drives the steps is formed recursively by
    // the root's correction, r_{k+1} = (r_k - A delta_1) - (A C_0) y_0 in the leaf
    // precision, and replaced by the FP64 residual b - A u every RECUR_ANCHOR steps.  The FP64 residual is formed at those
    // steps and wherever the recursive one comes within 2 tol: the stopping test always
    // takes the FP64 residual, and the anchors depend on the step count only, so the
    // iterates do not depend on when the test ran.
    static constexpr int RECUR_ANCHOR = 8;
    // The recursive residual serves the complex64 form: the FP64 form's residual is already
    // in its working precision, and there the recursion's extra FP64 work costs more than
    // the residual launch it saves.
    // It reads the root's A~_0 C_0 (r columns at each point) in every step: worth it while
    // that stays in the L2, not when it is read from HBM, where it costs about as much as the
    // FP64 residual it replaces.
    bool recur_possible() const {
        const size_t ac_bytes = 2 * (size_t)r * Sy * Sx * sizeof(CT);
        return sizeof(T) == sizeof(float) && eig && L >= 2 && P.n_inner == 1 && P.outer == HH_OUTER_ORAS &&
               ac_bytes <= ((size_t)64 << 20) && !q1();
    }
    hh_status loop_oras_device_test(int& it, double& rel) {
        // [0] stop (1 converged, 2 not finite), [1] FP64 tests run, [2] FP64 residual due,
        // [3] steps done, [4] anchor step
        int* ctl = (int*)(dnorm + 6);
        const int* hctl = (const int*)(h_norm + 6);
        hh_status st = HH_OK;
        zero(ctl, 8 * sizeof(int));
        zero(dcounter, 2 * sizeof(unsigned));   // the residual's and the root's tickets
        gated_residual(ctl);
        if (!read_norms(st)) return st;
        const bool recur = recur_possible();
        CoarseRecur rr{};
        rr.AC = recur ? AC0 : nullptr;
        rr.rp = RP;
        rr.rt = RT;
        rr.part = npart;
        rr.ticket = dcounter + 1;
        rr.nrm = dnorm;
        rr.ctl = ctl;
        rr.tol = P.tol;
        rr.anchor = RECUR_ANCHOR;
        double rel_prev = -1.0;
        int it_prev = 0, chunks = 0;
        for (;;) {
            rel = h_norm[2] > 0 ? std::sqrt(h_norm[0] / h_norm[2]) : 0.0;   // last FP64 residual
            if (hctl[0] == 2 || !std::isfinite(rel)) return HH_ENOCONV;
            if (hctl[0] == 1) return HH_OK;
            if (it >= P.max_iter) {
                // the FP64 residual of the last iterate, for the report
                gated_residual(ctl);
                if (!read_norms(st)) return st;
                rel = h_norm[2] > 0 ? std::sqrt(h_norm[0] / h_norm[2]) : 0.0;
                return hctl[0] == 1 ? HH_OK : HH_ENOCONV;
            }
            // the current residual: the recursive one once steps have run
            const double relc =
                (it == 0 || !recur) ? rel : (h_norm[2] > 0 ? std::sqrt(h_norm[1] / h_norm[2]) : 0.0);
            // Two chunks of 8 first: the residual of the first steps may grow before it
            // settles into its asymptotic rate, so a rate measured from step 0 overshoots.
            // Then the steps still needed at the rate of the last chunk, none to spare (a
            // short estimate costs one more synchronisation, a long one gated steps).
            int chunk = 8;
            if (chunks >= 2 && it > it_prev && relc < rel_prev && relc > 0) {
                const double rho = std::pow(relc / rel_prev, 1.0 / (it - it_prev));
                const double need = std::log(P.tol / relc) / std::log(rho);
                chunk = need < 64.0 ? std::max(1, (int)std::ceil(need)) : 64;
            }
            ++chunks;
            rel_prev = relc;
            it_prev = it;
            const int n = std::max(1, std::min(chunk, P.max_iter - it));
            // steps done: counted by the root's correction (recursive residual), else by
            // the FP64 tests, one per step
            const int count0 = recur ? hctl[3] : hctl[1];
            const bool fresh = graphs[2].exec == nullptr;
            for (int k = 0; k < n; ++k)
                replay_fresh(2, [&] {
                    oras_step(u, bvec, u, true, ctl, recur ? &rr : nullptr);
                    if (recur) gated_residual(ctl, ctl + 2, ctl + 4);
                    else gated_residual(ctl);
                });
            const bool ok = read_norms(st);
            const int ran = (recur ? hctl[3] : hctl[1]) - count0;
            // the first step of a new handle ran directly (its pairs are pending); the
            // replays that did work are the next ran - 1
            runs_release(graphs[2], (size_t)std::max(0, ran - (fresh ? 1 : 0)));
            if (!ok) return st;
            it += ran;
        }
    }

    // Stationary iteration u <- u + M (b - A u)  (Eqs. (2)-(3)).
    hh_status loop_oras(int& it, double& rel) {
        if (device_test_path()) return loop_oras_device_test(it, rel);
        hh_status st = HH_OK;
        for (;;) {
            if (!true_residual(res, st, RT)) return st;
            rel = h_norm[2] > 0 ? std::sqrt(h_norm[0] / h_norm[2]) : 0.0;
            if (!std::isfinite(rel)) return HH_ENOCONV;
            if (rel < P.tol) return HH_OK;
            if (it >= P.max_iter) return HH_ENOCONV;
            via_graph(1, [&] { oras_step(u, bvec, u, true); });
            ++it;
        }
    }

    // Flexible GMRES(mk) right-preconditioned by M (Sec. 3 solves the preconditioned
    // system by GMRES).  Arnoldi in FP64 with classical Gram-Schmidt applied twice; the
    // preconditioned directions z_j = M v_j are kept, so M may vary between steps (the
    // complex64 form).  The least-squares problem (Hessenberg column, Givens rotations,
    // residual estimate and stopping test) is updated on the device after each step, so
    // the host does not wait on a step: it queues step j once it has read the state after
    // step j - GM_LAG (a pinned snapshot behind an event).  A step queued after the test
    // stopped the cycle works on columns past the stopping one and changes nothing the
    // update reads (g and H up to the stopping column).  Convergence is confirmed on the
    // true residual at every restart.
    hh_status loop_gmres(int& it, double& rel) {
        const size_t N = (size_t)Sy * Sx;
        const int ld = mk + 1;
        hh_status st = HH_OK;
        const c128 one = {1.0, 0.0};
        c128* gone = gdots + 3 * 80;
        ck(cudaMemcpyAsync(gone, &one, sizeof(c128), cudaMemcpyHostToDevice, stream), cerr);
        const double nbv = std::sqrt(std::max(h_norm[2], 0.0));
        // with the profiler on, the captured preconditioner's events are read after every
        // step, which needs a synchronisation per step
        const int lag = prof_on ? 0 : GM_LAG;
        for (;;) {
            if (!true_residual(gw, st)) return st;
            const double beta = std::sqrt(std::max(h_norm[0], 0.0));
            rel = nbv > 0 ? beta / nbv : 0.0;
            if (!std::isfinite(rel)) return HH_ENOCONV;
            if (rel < P.tol) return HH_OK;
            if (it >= P.max_iter) return HH_ENOCONV;
            launch_col_store_normalised(Vb, ld, 0, gw, (const c128*)dnorm, N, stream);
            launch_gmres_init(gls, beta, stream);
            const int nsteps = std::min(mk, P.max_iter - it);
            int launched = 0;
            for (int j = 0; j < nsteps; ++j) {
                if (j >= lag && lag > 0) {
                    // the state after step j - lag
                    const int sl = (j - lag) % GM_SLOTS;
                    ck(cudaEventSynchronize(gm_ev[sl]), cerr);
                    if (cerr != cudaSuccess) return HH_ECUDA;
                    if (h_gst[sl].stop) break;
                }
                launch_col_load(Vb, ld, j, gv, N, stream);
                via_graph(0, [&] { precond(gv, gz); });
                launch_col_store_normalised(Zb, mk, j, gz, gone, N, stream);
                launch_apply<double, double, double>(gz, nullptr, gw, geom(0), 1, -1.0, nullptr, nullptr, stream);
                for (int pass = 0; pass < 2; ++pass) {
                    const int nbk = launch_ip_partial<double, double>(gw, 1, Vb, ld, N, 1, j + 1, partial,
                                                                      MAX_PART_BLOCKS, stream);
                    launch_ip_reduce(partial, nbk, 1, j + 1, gdots + pass * 80, nullptr, nullptr, stream);
                    launch_basis_combine(Vb, ld, j + 1, gdots + pass * 80, true, -1.0, gw, N, stream);
                }
                const int nbn = launch_ip_partial<double, double>(gw, 1, gw, 1, N, 1, 1, partial, MAX_PART_BLOCKS,
                                                                  stream);
                launch_ip_reduce(partial, nbn, 1, 1, gdots + 160, nullptr, nullptr, stream);
                launch_col_store_normalised(Vb, ld, j + 1, gw, gdots + 160, N, stream);
                launch_gmres_rotate(gls, gdots, gdots + 80, gdots + 160, j, nbv, P.tol, stream);
                const int sl = j % GM_SLOTS;
                ck(cudaMemcpyAsync(&h_gst[sl], gls.st, sizeof(GmresState), cudaMemcpyDeviceToHost, stream), cerr);
                ck(cudaEventRecord(gm_ev[sl], stream), cerr);
                ++launched;
                if (lag == 0) {
                    if (!sync_check(st)) return st;
                    graphs_collect();
                    if (h_gst[sl].stop) break;
                }
            }
            if (!sync_check(st)) return st;
            graphs_collect();
            GmresState fin{};
            ck(cudaMemcpy(&fin, gls.st, sizeof(GmresState), cudaMemcpyDeviceToHost), cerr);
            if (cerr != cudaSuccess) return HH_ECUDA;
            if (fin.bad) return HH_ENOCONV;
            const int jn = fin.stop ? fin.jstop : launched;
            it += jn;
            // y = R^{-1} g  (jn x jn upper triangular), u += Z y
            launch_gmres_solve(gls, jn, gy, stream);
            launch_basis_combine(Zb, mk, jn, gy, false, 1.0, u, N, stream);
        }
    }

    hh_status solve(const c128* f, const c128* g, c128* uo, hh_stats* stt) override {
        const size_t N = (size_t)Sy * Sx;
        zero(derr, sizeof(int) * 4);
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        cudaEventRecord(e0, stream);
        launch_rhs(f, g, bvec, P.dim, S, h, stream, q1());
        norm_sq(bvec, dnorm + 2);   // dnorm[2..3] = ||b||^2 as a complex
        ck(cudaMemcpyAsync(h_norm, dnorm, 4 * sizeof(double), cudaMemcpyDeviceToHost, stream), cerr);
        zero(u, sizeof(c128) * N);
        int it = 0;
        double rel = 0.0;
        hh_status st = HH_OK;
        if (sync_check(st)) st = mk > 0 ? loop_gmres(it, rel) : loop_oras(it, rel);
        d2d(uo, u, sizeof(c128) * N);
        cudaEventRecord(e1, stream);
        hh_status st2;
        sync_check(st2);
        prof_collect();
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        t_solve_ms = ms;
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (stt) {
            stt->iters = it;
            stt->rel_res = rel;
            stt->t_setup_ms = t_setup_ms;
            stt->t_solve_ms = t_solve_ms;
            stt->footprint_bytes = footprint;
        }
        if (st != HH_OK) return st;
        return st2;
    }

    hh_status residual(const c128* f, const c128* g, const c128* uu, double* rel) override {
        launch_rhs(f, g, bvec, P.dim, S, h, stream, q1());
        norm_sq(bvec, dnorm + 2);
        int nb = 0;
        launch_apply<double, double, double>(uu, bvec, res, geom(0), 1, 1.0, npart, &nb, stream);
        launch_sum(npart, nb, dnorm, stream);
        ck(cudaMemcpyAsync(h_norm, dnorm, 4 * sizeof(double), cudaMemcpyDeviceToHost, stream), cerr);
        hh_status st;
        if (!sync_check(st)) return st;
        *rel = h_norm[2] > 0 ? std::sqrt(h_norm[0] / h_norm[2]) : 0.0;
        return HH_OK;
    }

    // --------------------------------------------------------- step-level access
    bool valid_node(int id) const { return id >= 0 && id < nn; }

    hh_status node_info(int id, int info[10]) const override {
        if (!valid_node(id) || !info) return HH_EINVAL;
        const Node& nd = nodes[id];
        const int v[10] = {nd.oa, nd.ob, nd.ra, nd.rb, nd.level, nd.parent, nd.child[0], nd.child[1], Sx,
                           nd.ifrow};
        std::memcpy(info, v, sizeof(v));
        return HH_OK;
    }

    hh_status apply_operator(int id, const c128* x, c128* y, int nc) override {
        if (!valid_node(id) || nc < 1 || !x || !y) return HH_EINVAL;
        launch_apply<double, double, double>(x, nullptr, y, geom(id), nc, -1.0, nullptr, nullptr, stream);
        ck(cudaGetLastError(), cerr);
        return cerr == cudaSuccess ? HH_OK : HH_ECUDA;
    }

    hh_status leaf_solve(int id, const c128* v, c128* x, int nc) override {
        if (!valid_node(id) || !nodes[id].leaf() || nc < 1 || nc > nmax || !v || !x) return HH_EINVAL;
        const size_t n = pts(id) * nc;
        launch_copy<double, T>(v, Vs[id], n, false, false, stream);
        if (eig) {
            EigTask k = eig_task(id, Vs[id], W[id]);
            ck(cudaMemcpyAsync(d_etask_one, &k, sizeof(k), cudaMemcpyHostToDevice, stream), cerr);
            // the same kernels as inside a solve: one launch for a single vector
            if (nc == 1 && eig_fused) launch_eig_sweep_fused<T>(eig_fused, d_etask_one, 1, nodes[id].b(), Sx, stream);
            else
                for (int stg = 0; stg < 3; ++stg) eig_sweep_stage(stg, d_etask_one, 1, nc);
        } else {
            LeafTask k{};
            k.X = X[id];
            k.F = Vs[id];
            k.W = W[id];
            k.b = nodes[id].b();
            k.ldx = ldx[id];
            k.khr = khr_at(nodes[id].ra);
            ck(cudaMemcpyAsync(d_task_one, &k, sizeof(k), cudaMemcpyHostToDevice, stream), cerr);
            launch_sweep<T>(d_task_one, 1, nodes[id].b(), Sx, nc, derr, stream);
        }
        launch_copy<T, double>(W[id], x, n, false, false, stream);
        hh_status st;
        sync_check(st);
        return st;
    }

    hh_status interface_map(int c, int adj, const c128* in, c128* out, int nc) override {
        if (!valid_node(c) || c == 0 || nc < 1 || nc > m || !in || !out) return HH_EINVAL;
        const Node& cn = nodes[c];
        const Node& sn = nodes[cn.sib];
        const int l = cn.level;
        for (int o : lev[l]) zero(Vs[o], sizeof(CT) * pts(o) * nc);
        if (!adj) {
            launch_copy<double, T>(in, Vs[c] + row_off(c, cn.ifrow, nc), (size_t)Sx * nc, false, false, stream);
            apply_M(l, nc, true);
            launch_robin_trace<T>(W[c] + row_off(c, sn.ifrow, nc), W[c] + row_off(c, sn.inward, nc), Om[c], sn.b(), Sx,
                                  nc, kh, khr_at(sn.ifrow), stream, q1());
            launch_copy<T, double>(Om[c], out, (size_t)Sx * nc, false, false, stream);
        } else {
            launch_copy<double, T>(in, Om[c], (size_t)Sx * nc, false, false, stream);
            launch_adjoint_place<T>(Om[c], Vs[c] + row_off(c, sn.ifrow, nc), Vs[c] + row_off(c, sn.inward, nc), sn.b(),
                                    Sx, nc, kh, khr_at(sn.ifrow), stream, q1());
            apply_M(l, nc, true);
            launch_copy<T, double>(W[c] + row_off(c, cn.ifrow, nc), out, (size_t)Sx * nc, false, true, stream);
        }
        hh_status st;
        sync_check(st);
        return st;
    }

    hh_status get_basis(int c, void* hV, double* hsig) override {
        if (!valid_node(c) || c == 0) return HH_EINVAL;
        hh_status st;
        if (hV) {
            launch_copy<T, double>(Vc[c], res, (size_t)Sx * r, false, false, stream);
            if (!sync_check(st)) return st;
            ck(cudaMemcpy(hV, res, sizeof(c128) * Sx * r, cudaMemcpyDeviceToHost), cerr);
        }
        if (hsig) {
            if (!sync_check(st)) return st;
            ck(cudaMemcpy(hsig, lam[c], sizeof(double) * m, cudaMemcpyDeviceToHost), cerr);
            for (int j = 0; j < m; ++j) hsig[j] = std::sqrt(std::max(0.0, hsig[j]));
        }
        return cerr == cudaSuccess ? HH_OK : HH_ECUDA;
    }

    hh_status coarse_apply(int p, const c128* rr, c128* z) override {
        if (!valid_node(p) || nodes[p].leaf() || !rr || !z) return HH_EINVAL;
        launch_coarse_batch<T, double, double, double>(one_job(p, rr, nullptr, z, false), 2 * r, partial, dcounter + 2,
                                                       derr, stream);
        hh_status st;
        sync_check(st);
        return st;
    }

    hh_status precondition(const c128* rr, c128* z) override {
        if (!rr || !z) return HH_EINVAL;
        d2d(res, rr, sizeof(c128) * (size_t)Sy * Sx);
        d2d(bvec, rr, sizeof(c128) * (size_t)Sy * Sx);   // residual of the second half: rr - A ut
        oras_step(nullptr, bvec, z);
        hh_status st;
        sync_check(st);
        return st;
    }

    hh_status sketch_samples(int c, c128* out) override {
        if (!valid_node(c) || c == 0 || !out) return HH_EINVAL;
        launch_sketch<double>(out, Sx, m, c, P.seed, stream);
        hh_status st;
        sync_check(st);
        return st;
    }

    c128* staging_f() override { return res; }
    c128* staging_g() override { return gbuf; }
    c128* iterate() override { return u; }
    int npoints() const override { return Sy * Sx; }
};

static SolverBase* make_solver(const hh_params* P) {
    SolverBase* s = nullptr;
    if (P->precision == HH_PREC_MIXED) {
        auto* x = new Solver<float>();
        x->P = *P;
        x->init_geometry();
        s = x;
    } else {
        auto* x = new Solver<double>();
        x->P = *P;
        x->init_geometry();
        s = x;
    }
    return s;
}

// A solver set up in one call (validation, allocation through the hook, set-up).
static hh_status setup_one(const hh_params* p, cudaStream_t s, SolverBase** out, const AllocHook& hook) {
    *out = nullptr;
    const hh_status v = validate(p);
    if (v != HH_OK) return v;
    std::unique_ptr<SolverBase> sb(make_solver(p));
    sb->stream = s;
    sb->hook = hook;
    sb->footprint = sb->plan(nullptr);
    sb->block = dev_alloc(sb->footprint, sb->stream, sb->hook);
    if (!sb->block) return HH_ENOMEM;
    sb->plan((char*)sb->block);
    sb->prof_reset(g_prof_default, g_prof_mask_default);
    const hh_status st = sb->setup();
    if (st != HH_OK) return st;
    *out = sb.release();
    return HH_OK;
}

// ------------------------------------------------------------------ batched solves
// Several set-up problems solved together in lockstep (the batching form): per iteration
// one residual launch and one norm launch for all of them, one one-launch leaf sweep over
// all their leaves, one cooperative coarse launch per height of the hierarchy over all
// their nodes, and one for all roots; a problem leaves the batch when it converges.
// Requires the stationary outer iteration, n_i = 1, the eigenbasis leaf path with the
// one-launch sweep and at least two levels, for every problem, in one precision.
template <typename T>
static bool batchable(const Solver<T>* p) {
    return p->eig && p->eig_fused && p->pre_direct && p->P.n_inner == 1 && p->P.outer == HH_OUTER_ORAS && p->L >= 2 &&
           !p->q1();
}

// Lockstep iteration of several set-up problems: the engine of the batching and serving
// forms.  Problems are added with their right-hand sides and leave when they converge (or
// when the stationary iteration stops contracting for them); each step() is one
// iteration for all current problems: one residual launch and one norm launch, one
// one-launch leaf sweep over all their leaves, one cooperative coarse launch per
// hierarchy height and one for the roots.
template <typename T>
struct BatchEngine {
    struct Prob {
        Solver<T>* p = nullptr;
        c128* uo = nullptr;          // where the solution goes when the problem leaves
        void* tag = nullptr;
        unsigned long long serial = 0;   // unique per add(): the key of the task upload
        int it = 0, chk_it = 0;
        double rel = 0.0, best = 0.0, chk = 0.0;
        hh_status st = HH_OK;
        bool live = true;                // false once it has left (its jobs gated off)
    };
    cudaStream_t stream = nullptr;
    int cap_probs = 0, cap_tasks = 0;
    AllocHook hook;
    char* base = nullptr;
    size_t bytes = 0;
    EigTask* d_tasks = nullptr;
    double* part = nullptr;
    double* norms = nullptr;
    c128* cpart = nullptr;
    unsigned* bar = nullptr;
    int* berr = nullptr;
    double* h_norms = nullptr;       // pinned
    int part_cap = RB_MAX_JOBS * 304;
    std::vector<Prob> act;
    // serials of the problems whose leaf tasks are in d_tasks (a freed solver's address
    // can come back for a new problem, so addresses are no key)
    std::vector<unsigned long long> uploaded;
    unsigned long long next_serial = 1;
    int cl = 0, bmax = 0, sxmax = 0;
    cudaError_t cerr = cudaSuccess;
    // One lockstep iteration after the first (the preconditioner step of every current
    // problem, then their residuals for the next test) is a CUDA graph, captured on a
    // private stream for the current set of problems and replayed while the set stays.
    cudaStream_t cap_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    std::vector<unsigned long long> graph_key;
    bool resid_pending = false;   // the current problems' residuals are already enqueued
    unsigned long long replays = 0, captures = 0;
    // Gate word per position of act: a problem that leaves keeps its place in the captured
    // graph with its word set, so that its jobs return at once; the set is compacted (and
    // the graph captured again) when a quarter of it has left or a problem joins.
    int* gates = nullptr;
    bool joined = false;

    hh_status init(cudaStream_t s, int probs, int tasks, const AllocHook& h) {
        stream = s;
        cap_probs = std::max(probs, 1);
        cap_tasks = std::max(tasks, 1);
        hook = h;
        bytes = align_up(sizeof(EigTask) * cap_tasks, 256) + align_up(sizeof(double) * part_cap, 256) +
                align_up(sizeof(double) * (cap_probs + 8), 256) + align_up(sizeof(c128) * 304 * 64, 256) + 256 +
                align_up(sizeof(int) * cap_probs, 256);
        base = (char*)dev_alloc(bytes, stream, hook);
        if (!base) return HH_ENOMEM;
        size_t off = 0;
        auto take = [&](size_t b) { char* q = base + off; off += align_up(b, 256); return q; };
        d_tasks = (EigTask*)take(sizeof(EigTask) * cap_tasks);
        part = (double*)take(sizeof(double) * part_cap);
        norms = (double*)take(sizeof(double) * (cap_probs + 8));
        cpart = (c128*)take(sizeof(c128) * 304 * 64);
        bar = (unsigned*)take(256);
        berr = (int*)(bar + 4);
        gates = (int*)take(sizeof(int) * cap_probs);
        ck(cudaMemsetAsync(gates, 0, sizeof(int) * cap_probs, stream), cerr);
        ck(cudaMallocHost(&h_norms, sizeof(double) * (cap_probs + 8)), cerr);
        ck(cudaMemsetAsync(bar, 0, 256, stream), cerr);
        return cerr == cudaSuccess ? HH_OK : HH_ECUDA;
    }
    void drop_graph() {
        if (gexec) cudaGraphExecDestroy(gexec);
        if (graph) cudaGraphDestroy(graph);
        gexec = nullptr;
        graph = nullptr;
        graph_key.clear();
    }
    void release() {
        drop_graph();
        if (cap_stream) cudaStreamDestroy(cap_stream);
        cap_stream = nullptr;
        if (h_norms) cudaFreeHost(h_norms);
        h_norms = nullptr;
        if (base) dev_free(base, bytes, stream, hook);
        base = nullptr;
    }
    int tasks_in_use() const {
        int n = 0;
        for (auto& q : act)
            if (q.live) n += (int)q.p->h_pre.size();
        return n;
    }
    int live_count() const {
        int n = 0;
        for (auto& q : act) n += q.live;
        return n;
    }
    // whether p can join: lockstep-able, room left, and a fused-sweep cluster size that
    // serves every member
    bool can_add(Solver<T>* p) const {
        if (!batchable(p) || live_count() >= cap_probs) return false;
        if (tasks_in_use() + (int)p->h_pre.size() > cap_tasks) return false;
        int bm = p->b_max, sx = p->Sx, smin = p->Sx;
        for (auto& q : act) {
            if (!q.live) continue;
            bm = std::max(bm, q.p->b_max);
            sx = std::max(sx, q.p->Sx);
            smin = std::min(smin, q.p->Sx);
        }
        const int c = eig_sweep_fused_ready<T>(bm, sx);
        return c && c <= smin;
    }
    // enqueue the right-hand side, ||b||^2 and u = 0 of a problem that joins
    void add(Solver<T>* p, const c128* f, const c128* g, c128* uo, void* tag) {
        p->stream = stream;
        p->zero(p->derr, sizeof(int) * 4);
        launch_rhs(f, g, p->bvec, p->P.dim, p->S, p->h, stream, p->q1());
        p->norm_sq(p->bvec, p->dnorm + 2);
        ck(cudaMemcpyAsync(p->h_norm + 2, p->dnorm + 2, sizeof(double), cudaMemcpyDeviceToHost, stream), cerr);
        p->zero(p->u, sizeof(c128) * (size_t)p->Sy * p->Sx);
        Prob q;
        q.p = p;
        q.uo = uo;
        q.tag = tag;
        q.serial = next_serial++;
        q.it = -1;   // the first step reads ||b||^2
        compact();   // a joining problem takes its place in a set without departed ones
        act.push_back(q);
        ck(cudaMemsetAsync(gates, 0, sizeof(int) * act.size(), stream), cerr);
        resid_pending = false;   // the next step enqueues every current problem's residual
        joined = true;
    }
    // drop the departed problems from the set (positions change: the gate words are reset)
    void compact() {
        std::vector<Prob> keep;
        for (auto& q : act)
            if (q.live) keep.push_back(q);
        if (keep.size() == act.size()) return;
        act.swap(keep);
        ck(cudaMemsetAsync(gates, 0, sizeof(int) * std::max<size_t>(act.size(), 1), stream), cerr);
    }
    // One iteration for every current problem; problems that leave are appended to `done`
    // (their solution already copied to uo, the copy complete).
    // Residuals of every current problem (norms[k] for act[k]), enqueued on `stream`.
    void enqueue_residuals() {
        const int na = (int)act.size();
        for (int c0 = 0; c0 < na; c0 += RB_MAX_JOBS) {
            ResidBatch rb{};
            for (int k = c0; k < na && k < c0 + RB_MAX_JOBS; ++k) {
                Solver<T>* p = act[k].p;
                ResidJob& j = rb.job[rb.njobs++];
                j.x = p->u;
                j.v = p->bvec;
                j.y = p->res;
                j.yt = p->RT;
                j.g = p->geom(0);
                j.gate = gates + k;
            }
            launch_residual_batch<T>(rb, part, part_cap, norms + c0, stream);
        }
    }
    hh_status step(std::vector<Prob>& done) {
        if (act.empty()) return HH_OK;
        const int na = (int)act.size();
        if (!resid_pending) enqueue_residuals();
        resid_pending = false;
        ck(cudaMemcpyAsync(h_norms, norms, sizeof(double) * na, cudaMemcpyDeviceToHost, stream), cerr);
        ck(cudaMemcpyAsync(h_norms + cap_probs, berr, sizeof(int), cudaMemcpyDeviceToHost, stream), cerr);
        ck(cudaStreamSynchronize(stream), cerr);
        if (cerr != cudaSuccess) return HH_ECUDA;
        if (*(const int*)(h_norms + cap_probs) == DEV_TIMEOUT) return HH_ETIMEOUT;
        bool left = false;
        for (int k = 0; k < na; ++k) {
            Prob& q = act[k];
            if (!q.live) continue;
            if (q.it < 0) q.it = 0;
            const double b2 = q.p->h_norm[2];
            q.rel = b2 > 0 ? std::sqrt(h_norms[k] / b2) : 0.0;
            if (q.it == 0) q.best = q.chk = q.rel;
            q.best = std::min(q.best, q.rel);
            // the stationary iteration is not a contraction for every problem: one whose
            // residual has grown a hundredfold past its best, or fell less than tenfold over
            // the last 25 steps, leaves early (its owner solves it by GMRES)
            bool slow = false;
            if (q.it - q.chk_it >= 25) {
                slow = q.rel > 0.1 * q.chk;
                q.chk = q.rel;
                q.chk_it = q.it;
            }
            bool out = true;
            if (!std::isfinite(q.rel) || q.rel > 100.0 * q.best || (slow && q.rel >= q.p->P.tol)) q.st = HH_ENOCONV;
            else if (q.rel < q.p->P.tol) q.st = HH_OK;
            else if (q.it >= q.p->P.max_iter) q.st = HH_ENOCONV;
            else out = false;
            if (out) {
                ck(cudaMemcpyAsync(q.uo, q.p->u, sizeof(c128) * (size_t)q.p->Sy * q.p->Sx, cudaMemcpyDeviceToDevice,
                                   stream),
                   cerr);
                // its jobs in the captured graph return at once from now on
                const int one = 1;
                ck(cudaMemcpyAsync(gates + k, &one, sizeof(int), cudaMemcpyHostToDevice, stream), cerr);
                q.live = false;
                done.push_back(q);
                left = true;
            }
        }
        if (left) ck(cudaStreamSynchronize(stream), cerr);
        const int nl = live_count();
        if (nl == 0) {
            act.clear();
            drop_graph();
            return cerr == cudaSuccess ? HH_OK : HH_ECUDA;
        }
        // compact once a quarter of the set has left (the graph is captured again)
        if (4 * (na - nl) >= na) compact();
        joined = false;
        // one preconditioner step for every current problem
        std::vector<Solver<T>*> ids;
        std::vector<unsigned long long> key;
        for (auto& q : act) {
            ids.push_back(q.p);
            key.push_back(q.serial);
        }
        if (key != uploaded) {
            std::vector<EigTask> tk;
            bmax = sxmax = 0;
            int smin = 1 << 30;
            for (size_t k = 0; k < ids.size(); ++k) {
                Solver<T>* p = ids[k];
                for (EigTask t : p->h_pre) {
                    t.gate = gates + k;
                    tk.push_back(t);
                }
                bmax = std::max(bmax, p->b_max);
                sxmax = std::max(sxmax, p->Sx);
                smin = std::min(smin, p->Sx);
            }
            cl = eig_sweep_fused_ready<T>(bmax, sxmax);
            if (!cl || cl > smin) return HH_ENOTIMPL;
            ck(cudaMemcpyAsync(d_tasks, tk.data(), sizeof(EigTask) * tk.size(), cudaMemcpyHostToDevice, stream),
               cerr);
            // the pageable source must stay alive until the copy has read it
            ck(cudaStreamSynchronize(stream), cerr);
            uploaded = key;
        }
        if (key != graph_key) {
            // capture the iteration for this set of problems: the preconditioner step and
            // the residuals of the next test (launches only: no host synchronisation inside)
            drop_graph();
            if (!cap_stream) ck(cudaStreamCreateWithFlags(&cap_stream, cudaStreamNonBlocking), cerr);
            cudaStream_t user = stream;
            bool ok = cerr == cudaSuccess &&
                      cudaStreamBeginCapture(cap_stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
            if (ok) {
                stream = cap_stream;
                enqueue_precond(ids);
                enqueue_residuals();
                stream = user;
                ok = cudaStreamEndCapture(cap_stream, &graph) == cudaSuccess && graph &&
                     cudaGraphInstantiate(&gexec, graph, 0) == cudaSuccess;
            }
            stream = user;
            if (!ok) {
                cudaGetLastError();
                drop_graph();
                return HH_ECUDA;
            }
            graph_key = key;
            ++captures;
        }
        ck(cudaGraphLaunch(gexec, stream), cerr);
        ++replays;
        resid_pending = true;
        for (auto& q : act)
            if (q.live) ++q.it;
        ck(cudaGetLastError(), cerr);
        return cerr == cudaSuccess ? HH_OK : HH_ECUDA;
    }

    // One preconditioner step for the problems `ids` (the current set, in order).
    void enqueue_precond(const std::vector<Solver<T>*>& ids) {
        int nt = 0, lmax = 0;
        for (auto* p : ids) {
            nt += (int)p->h_pre.size();
            lmax = std::max(lmax, p->L);
        }
        launch_eig_sweep_fused<T>(cl, d_tasks, nt, bmax, sxmax, stream);
        // internal nodes, deepest first: height = L - level; level 1 writes into u (FP64)
        for (int hgt = 1; hgt < lmax; ++hgt) {
            for (int to64 = 0; to64 < 2; ++to64) {
                struct NodeJob {
                    Solver<T>* p;
                    int id, k;   // node, position of the problem in the set
                };
                std::vector<NodeJob> jobs;
                for (size_t k = 0; k < ids.size(); ++k) {
                    Solver<T>* p = ids[k];
                    const int l = p->L - hgt;
                    if (l < 1 || (l == 1) != (to64 == 1)) continue;
                    for (int id : p->lev[l]) jobs.push_back({p, id, (int)k});
                }
                std::vector<int> widths;   // one launch per basis width and per CB_MAX_JOBS nodes
                for (auto& jn : jobs)
                    if (std::find(widths.begin(), widths.end(), 2 * jn.p->r) == widths.end())
                        widths.push_back(2 * jn.p->r);
                for (int w : widths) {
                    CoarseBatch bt{};
                    auto flush = [&]() {
                        if (!bt.njobs) return;
                        if (to64) launch_coarse_batch<T, T, T, double>(bt, w, cpart, bar, berr, stream);
                        else launch_coarse_batch<T, T, T, T>(bt, w, cpart, bar, berr, stream);
                        bt = CoarseBatch{};
                    };
                    for (auto& jn : jobs) {
                        Solver<T>* p = jn.p;
                        if (2 * p->r != w) continue;
                        const int id = jn.id;
                        const Node& nd = p->nodes[id];
                        CoarseJob& j = bt.job[bt.njobs++];
                        j.C = p->C[id];
                        j.v = p->RT + p->row_off(0, nd.ra, 1);
                        j.w_in = p->W[id];
                        j.out = to64 ? (void*)(p->u + p->row_off(0, nd.own_a, 1))
                                     : (void*)(p->W[nd.parent] + p->row_off(nd.parent, nd.own_a, 1));
                        j.Minv = p->AinvT[id];
                        j.y = p->ycoef[id];
                        j.g = p->geom(id);
                        j.r0 = nd.own_a - nd.ra;
                        j.r1 = nd.own_b - nd.ra;
                        j.acc_out = to64;
                        j.add_w = 1;
                        j.split = p->split_row(id);
                        j.gate = gates + jn.k;
                        if (bt.njobs == CB_MAX_JOBS) flush();
                    }
                    flush();
                }
            }
        }
        // the roots: u += C A_c^{-1} C^H (b - A u)
        std::vector<int> widths;
        for (auto* p : ids)
            if (std::find(widths.begin(), widths.end(), 2 * p->r) == widths.end()) widths.push_back(2 * p->r);
        for (int w : widths) {
            CoarseBatch bt{};
            for (size_t k = 0; k < ids.size(); ++k) {
                Solver<T>* p = ids[k];
                if (2 * p->r != w) continue;
                bt.job[bt.njobs] = p->one_job(0, p->bvec, p->u, p->u, true).job[0];
                bt.job[bt.njobs++].gate = gates + k;
                if (bt.njobs == CB_MAX_JOBS) {
                    launch_coarse_batch<T, double, double, double>(bt, w, cpart, bar, berr, stream);
                    bt = CoarseBatch{};
                }
            }
            if (bt.njobs) launch_coarse_batch<T, double, double, double>(bt, w, cpart, bar, berr, stream);
        }
    }
};

template <typename T>
static hh_status batch_solve(std::vector<Solver<T>*>& ps, const c128* const* f, const c128* const* g,
                             c128* const* uo, cudaStream_t stream, hh_stats* stats, std::vector<hh_status>& res) {
    const int np = (int)ps.size();
    int nleaf = 0;
    for (auto* p : ps) nleaf += (int)p->h_pre.size();
    BatchEngine<T> eng;
    eng.cap_probs = np;
    eng.cap_tasks = nleaf;
    for (auto* p : ps) {
        if (!eng.can_add(p)) return HH_ENOTIMPL;
        eng.act.push_back({});   // capacity and cluster checks against the members so far
        eng.act.back().p = p;
    }
    eng.act.clear();
    hh_status st = eng.init(stream, np, nleaf, g_alloc);
    if (st != HH_OK) {
        eng.release();
        return st;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, stream);
    for (int k = 0; k < np; ++k) eng.add(ps[k], f[k], g[k], uo[k], (void*)(size_t)k);
    std::vector<typename BatchEngine<T>::Prob> done;
    while (st == HH_OK && !eng.act.empty()) st = eng.step(done);
    cudaEventRecord(e1, stream);
    cudaStreamSynchronize(stream);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    eng.release();
    res.assign(np, HH_ECUDA);
    for (auto& q : done) {
        const int k = (int)(size_t)q.tag;
        res[k] = q.st;
        if (stats) {
            stats[k].iters = q.it;
            stats[k].rel_res = q.rel;
            stats[k].t_setup_ms = ps[k]->t_setup_ms;
            stats[k].t_solve_ms = ms;
            stats[k].footprint_bytes = ps[k]->footprint;
        }
    }
    if (st != HH_OK) return st;
    for (auto s1 : res)
        if (s1 != HH_OK) return s1;
    return HH_OK;
}

// All handles in one precision and batchable: solve them together in lockstep.  Problems
// the stationary iteration does not converge are then solved by flexible GMRES (the
// paper's outer solver) on handles set up for it, several at a time from host threads.
// Handles that cannot join the lockstep batch are solved one by one.
static hh_status setup_one(const hh_params* p, cudaStream_t s, SolverBase** out, const AllocHook& hook);

static hh_status solve_many(SolverBase* const* hs, const c128* const* f, const c128* const* g, c128* const* u, int n,
                            cudaStream_t stream, hh_stats* stats) {
    std::vector<Solver<float>*> pf;
    std::vector<Solver<double>*> pd;
    for (int k = 0; k < n; ++k) {
        if (auto* a = dynamic_cast<Solver<float>*>(hs[k])) { if (batchable(a)) pf.push_back(a); }
        else if (auto* b = dynamic_cast<Solver<double>*>(hs[k])) { if (batchable(b)) pd.push_back(b); }
    }
    std::vector<hh_status> per;
    hh_status st = HH_ENOTIMPL;
    if ((int)pf.size() == n) st = batch_solve<float>(pf, f, g, u, stream, stats, per);
    else if ((int)pd.size() == n) st = batch_solve<double>(pd, f, g, u, stream, stats, per);
    if (st == HH_ENOTIMPL) {
        hh_status first = HH_OK;
        for (int k = 0; k < n; ++k) {
            hs[k]->stream = stream;
            const hh_status s1 = hs[k]->solve(f[k], g[k], u[k], stats ? stats + k : nullptr);
            if (s1 != HH_OK && first == HH_OK) first = s1;
        }
        return first;
    }
    if (st != HH_OK && st != HH_ENOCONV) return st;
    std::vector<int> rescue;
    for (int k = 0; k < n; ++k)
        if (per[k] == HH_ENOCONV) rescue.push_back(k);
    if (rescue.empty()) return st;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return HH_ECUDA;
    std::vector<hh_status> rs(rescue.size(), HH_OK);
    const int nw = std::min((int)rescue.size(), 8);
    auto worker = [&](int w) {
        cudaSetDevice(dev);
        cudaStream_t ws = nullptr;
        if (cudaStreamCreateWithFlags(&ws, cudaStreamNonBlocking) != cudaSuccess) {
            for (size_t i = w; i < rescue.size(); i += nw) rs[i] = HH_ECUDA;
            return;
        }
        for (size_t i = w; i < rescue.size(); i += nw) {
            const int k = rescue[i];
            hh_params q = hs[k]->P;
            q.outer = HH_OUTER_GMRES;
            if (q.restart < 1 || q.restart > 64) q.restart = 40;
            SolverBase* g2 = nullptr;
            rs[i] = setup_one(&q, ws, &g2, g_alloc);
            if (rs[i] != HH_OK) continue;
            hh_stats s2{};
            rs[i] = g2->solve(f[k], g[k], u[k], &s2);
            if (stats) {
                stats[k].iters += s2.iters;
                stats[k].rel_res = s2.rel_res;
            }
            cudaStreamSynchronize(ws);
            delete g2;
        }
        cudaStreamSynchronize(ws);
        cudaStreamDestroy(ws);
    };
    // the batch wrote its last iterates on `stream`: the rescues overwrite them on theirs
    cudaStreamSynchronize(stream);
    std::vector<std::thread> th;
    for (int w = 1; w < nw; ++w) th.emplace_back(worker, w);
    worker(0);
    for (auto& t : th) t.join();
    for (auto s1 : rs)
        if (s1 != HH_OK) return s1;
    return HH_OK;
}

// ------------------------------------------------------------------ serving form
// Continuous batching: requests are admitted while the sum of their footprints stays
// within the HBM budget and a slot is free; set-up workers set them up concurrently; an
// engine thread iterates every set-up problem in lockstep (BatchEngine), taking in new
// problems between iterations and retiring converged ones at once.  Problems the
// lockstep iteration cannot take (other outer solvers, n_i > 1, one level, 1D, the
// explicit-inverse leaf path) are solved by the worker that set them up; problems whose
// stationary iteration does not converge go back to a worker for flexible GMRES.
struct ServerReq {
    unsigned long long ticket = 0;
    hh_params P{};
    const c128* f = nullptr;
    const c128* g = nullptr;
    c128* u = nullptr;
    size_t fp = 0;
    hh_status st = HH_OK;
    hh_stats stats{};
    bool done = false, rescued = false;
    std::chrono::steady_clock::time_point t_submit, t_admit, t_join;
    SolverBase* s = nullptr;
};

static double ms_since(std::chrono::steady_clock::time_point a) {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - a).count();
}

struct Server {
    size_t budget = 0, used = 0;
    int max_slots = 0, slots = 0, dev = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_engine;
    std::deque<ServerReq*> pending, ready, rescue;
    std::map<unsigned long long, ServerReq*> all;
    unsigned long long next = 1;
    bool stop = false;
    std::vector<std::thread> threads;

    // called with the lock held
    void finish(ServerReq* r) {
        r->done = true;
        used -= r->fp;
        --slots;
        cv_work.notify_all();
    }
    void complete(ServerReq* r, hh_status st, cudaStream_t s) {
        if (r->s) {
            r->s->stream = s;
            delete r->s;
            r->s = nullptr;
        }
        std::lock_guard<std::mutex> lk(mu);
        r->st = st;
        r->stats.t_total_ms = ms_since(r->t_submit);
        r->stats.t_queue_ms = std::chrono::duration<double, std::milli>(r->t_admit - r->t_submit).count();
        finish(r);
    }

    void worker() {
        cudaSetDevice(dev);
        cudaStream_t ws = nullptr;
        cudaStreamCreateWithFlags(&ws, cudaStreamNonBlocking);
        const AllocHook rt{};   // no hook: server problems allocate from the library's pool, on this stream
        for (;;) {
            ServerReq* r = nullptr;
            bool is_rescue = false;
            {
                std::unique_lock<std::mutex> lk(mu);
                for (;;) {
                    if (stop) break;
                    if (!rescue.empty()) {
                        r = rescue.front();
                        rescue.pop_front();
                        is_rescue = true;
                        break;
                    }
                    if (!pending.empty() && slots < max_slots && used + pending.front()->fp <= budget) {
                        r = pending.front();
                        pending.pop_front();
                        used += r->fp;
                        ++slots;
                        r->t_admit = std::chrono::steady_clock::now();
                        break;
                    }
                    cv_work.wait(lk);
                }
            }
            if (!r) break;
            if (is_rescue) {
                gmres_rescue(r, ws, rt);
                continue;
            }
            SolverBase* sb = nullptr;
            hh_status st = setup_one(&r->P, ws, &sb, rt);
            r->s = sb;
            if (st != HH_OK) {
                complete(r, st, ws);
                continue;
            }
            r->stats.t_setup_ms = sb->t_setup_ms;
            r->stats.footprint_bytes = sb->footprint;
            bool lock = false;
            if (auto* a = dynamic_cast<Solver<float>*>(sb)) lock = batchable(a);
            else if (auto* b = dynamic_cast<Solver<double>*>(sb)) lock = batchable(b);
            if (lock) {
                cudaStreamSynchronize(ws);
                std::lock_guard<std::mutex> lk(mu);
                ready.push_back(r);
                cv_engine.notify_one();
                continue;
            }
            const auto t0 = std::chrono::steady_clock::now();
            st = sb->solve(r->f, r->g, r->u, &r->stats);
            cudaStreamSynchronize(ws);
            r->stats.t_solve_ms = ms_since(t0);
            if (st == HH_ENOCONV && r->P.outer == HH_OUTER_ORAS) {
                sb->stream = ws;
                delete sb;
                r->s = nullptr;
                gmres_rescue(r, ws, rt);
                continue;
            }
            complete(r, st, ws);
        }
        cudaStreamSynchronize(ws);
        cudaStreamDestroy(ws);
    }

    // Re-solves a request by flexible GMRES on a handle set up for it.  Its footprint
    // replaces the request's in the budget (waiting until it fits, unless nothing else is
    // in flight).
    void gmres_rescue(ServerReq* r, cudaStream_t ws, const AllocHook& rt) {
        r->rescued = true;
        hh_params q = r->P;
        q.outer = HH_OUTER_GMRES;
        if (q.restart < 1 || q.restart > 64) q.restart = 40;
        size_t fpg = 0;
        {
            std::unique_ptr<SolverBase> tmp(make_solver(&q));
            fpg = tmp->plan(nullptr);
        }
        {
            std::unique_lock<std::mutex> lk(mu);
            cv_work.wait(lk, [&] { return stop || used - r->fp + fpg <= budget || slots == 1; });
            used = used - r->fp + fpg;
            r->fp = fpg;
        }
        SolverBase* g2 = nullptr;
        hh_status st = setup_one(&q, ws, &g2, rt);
        hh_stats s2{};
        if (st == HH_OK) {
            st = g2->solve(r->f, r->g, r->u, &s2);
            cudaStreamSynchronize(ws);
            g2->stream = ws;
            delete g2;
        }
        r->stats.iters += s2.iters;
        r->stats.rel_res = s2.rel_res;
        complete(r, st, ws);
    }

    template <typename T>
    void retire(BatchEngine<T>& eng, std::vector<typename BatchEngine<T>::Prob>& done) {
        for (auto& q : done) {
            ServerReq* r = (ServerReq*)q.tag;
            r->stats.iters = q.it;
            r->stats.rel_res = q.rel;
            r->stats.t_solve_ms = ms_since(r->t_join);
            if (q.st == HH_ENOCONV && !r->rescued) {
                // hand to a worker for GMRES; the handle of the stationary run goes now
                r->s->stream = eng.stream;
                delete r->s;
                r->s = nullptr;
                std::lock_guard<std::mutex> lk(mu);
                rescue.push_back(r);
                cv_work.notify_all();
            } else {
                complete(r, q.st, eng.stream);
            }
        }
        done.clear();
    }

    void engine() {
        cudaSetDevice(dev);
        cudaStream_t es = nullptr;
        cudaStreamCreateWithFlags(&es, cudaStreamNonBlocking);
        BatchEngine<float> e32;
        BatchEngine<double> e64;
        const AllocHook rt{};
        const bool ok = e32.init(es, max_slots, max_slots * 64, rt) == HH_OK &&
                        e64.init(es, max_slots, max_slots * 64, rt) == HH_OK;
        std::vector<BatchEngine<float>::Prob> d32;
        std::vector<BatchEngine<double>::Prob> d64;
        for (;;) {
            std::vector<ServerReq*> take;
            {
                std::unique_lock<std::mutex> lk(mu);
                if (e32.act.empty() && e64.act.empty())
                    cv_engine.wait(lk, [&] { return stop || !ready.empty(); });
                if (stop) break;
                while (!ready.empty()) {
                    take.push_back(ready.front());
                    ready.pop_front();
                }
            }
            std::vector<ServerReq*> later;
            for (ServerReq* r : take) {
                bool added = false;
                if (ok) {
                    r->t_join = std::chrono::steady_clock::now();
                    if (auto* a = dynamic_cast<Solver<float>*>(r->s)) {
                        if (e32.can_add(a)) { e32.add(a, r->f, r->g, r->u, r); added = true; }
                    } else if (auto* b = dynamic_cast<Solver<double>*>(r->s)) {
                        if (e64.can_add(b)) { e64.add(b, r->f, r->g, r->u, r); added = true; }
                    }
                }
                if (!added) {
                    if (!ok || (e32.act.empty() && e64.act.empty())) {
                        // cannot join even an empty engine: solve it here on its own
                        r->s->stream = es;
                        const auto t0 = std::chrono::steady_clock::now();
                        const hh_status st = r->s->solve(r->f, r->g, r->u, &r->stats);
                        cudaStreamSynchronize(es);
                        r->stats.t_solve_ms = ms_since(t0);
                        complete(r, st, es);
                    } else {
                        later.push_back(r);
                    }
                }
            }
            if (!later.empty()) {
                std::lock_guard<std::mutex> lk(mu);
                for (auto it2 = later.rbegin(); it2 != later.rend(); ++it2) ready.push_front(*it2);
            }
            hh_status st32 = e32.step(d32);
            retire(e32, d32);
            hh_status st64 = e64.step(d64);
            retire(e64, d64);
            if (st32 != HH_OK) {
                for (auto& q : e32.act)
                    if (q.live) complete((ServerReq*)q.tag, st32, es);
                e32.act.clear();
                e32.uploaded.clear();
            }
            if (st64 != HH_OK) {
                for (auto& q : e64.act)
                    if (q.live) complete((ServerReq*)q.tag, st64, es);
                e64.act.clear();
                e64.uploaded.clear();
            }
        }
        // shutting down: requests still iterating are dropped (their handles freed); the
        // entries that have left were completed when they left
        for (auto& q : e32.act)
            if (q.live) complete((ServerReq*)q.tag, HH_ECUDA, es);
        for (auto& q : e64.act)
            if (q.live) complete((ServerReq*)q.tag, HH_ECUDA, es);
        cudaStreamSynchronize(es);
        e32.release();
        e64.release();
        cudaStreamDestroy(es);
    }
};

}  // namespace hh

// ============================================================================= C-ABI
struct hh_handle {
    hh::SolverBase* s;
};

extern "C" {

hh_status hh_set_allocator(void* (*alloc)(size_t, void*, void*), void (*free_)(void*, size_t, void*, void*),
                           void* ctx) {
    if (alloc && !free_) return HH_EINVAL;
    hh::g_alloc.alloc = alloc;
    hh::g_alloc.free_ = alloc ? free_ : nullptr;
    hh::g_alloc.ctx = alloc ? ctx : nullptr;
    return HH_OK;
}

hh_status hh_footprint(const hh_params* params, size_t* bytes) {
    if (!bytes) return HH_EINVAL;
    const hh_status v = hh::validate(params);
    if (v != HH_OK) return v;
    std::unique_ptr<hh::SolverBase> s(hh::make_solver(params));
    *bytes = s->plan(nullptr);
    return HH_OK;
}

hh_status hh_setup(const hh_params* params, void* stream, hh_handle** out, size_t* footprint_out) {
    if (!out) return HH_EINVAL;
    *out = nullptr;
    const hh_status v = hh::validate(params);
    if (v != HH_OK) return v;
    std::unique_ptr<hh::SolverBase> s(hh::make_solver(params));
    s->stream = (cudaStream_t)stream;
    s->hook = hh::g_alloc;
    s->footprint = s->plan(nullptr);
    s->block = hh::dev_alloc(s->footprint, s->stream, s->hook);
    if (!s->block) return HH_ENOMEM;
    s->plan((char*)s->block);
    s->prof_reset(hh::g_prof_default, hh::g_prof_mask_default);
    const hh_status st = s->setup();
    if (footprint_out) *footprint_out = s->footprint;
    if (st != HH_OK) return st;
    *out = new hh_handle{s.release()};
    return HH_OK;
}

hh_status hh_setup_batch(const hh_params* params, int count, void* stream, hh_handle** out) {
    if (!params || !out || count < 1) return HH_EINVAL;
    for (int k = 0; k < count; ++k) {
        out[k] = nullptr;
        const hh_status v = hh::validate(params + k);
        if (v != HH_OK) return v;
    }
    // set-ups are latency-bound chains of small kernels: run several at once, each on its
    // own stream from its own host thread
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return HH_ECUDA;
    const int nw = std::min(count, 8);
    std::vector<hh_status> st(count, HH_OK);
    auto worker = [&](int w) {
        cudaSetDevice(dev);
        cudaStream_t ws = nullptr;
        if (cudaStreamCreateWithFlags(&ws, cudaStreamNonBlocking) != cudaSuccess) {
            for (int k = w; k < count; k += nw) st[k] = HH_ECUDA;
            return;
        }
        for (int k = w; k < count; k += nw) {
            size_t fp = 0;
            st[k] = hh_setup(params + k, ws, &out[k], &fp);
            if (out[k]) out[k]->s->stream = (cudaStream_t)stream;
        }
        cudaStreamSynchronize(ws);
        cudaStreamDestroy(ws);
    };
    std::vector<std::thread> th;
    for (int w = 1; w < nw; ++w) th.emplace_back(worker, w);
    worker(0);
    for (auto& t : th) t.join();
    for (int k = 0; k < count; ++k)
        if (st[k] != HH_OK) {
            for (int j = 0; j < count; ++j) {
                hh_destroy(out[j]);
                out[j] = nullptr;
            }
            return st[k];
        }
    return HH_OK;
}

hh_status hh_solve_batch(hh_handle* const* h, const void* const* d_f, const void* const* d_g, void* const* d_u,
                         int count, void* stream, hh_stats* stats) {
    if (!h || !d_f || !d_g || !d_u || count < 1) return HH_EINVAL;
    std::vector<hh::SolverBase*> hs(count);
    for (int k = 0; k < count; ++k) {
        if (!h[k] || !d_f[k] || !d_g[k] || !d_u[k]) return HH_EINVAL;
        hs[k] = h[k]->s;
    }
    return hh::solve_many(hs.data(), (const c128* const*)d_f, (const c128* const*)d_g, (c128* const*)d_u, count,
                          (cudaStream_t)stream, stats);
}

struct hh_server {
    hh::Server* sv;
};

hh_status hh_server_create(size_t hbm_budget, int max_slots, hh_server** out) {
    if (!out || max_slots < 1 || max_slots > 4096 || hbm_budget == 0) return HH_EINVAL;
    *out = nullptr;
    auto* sv = new hh::Server();
    sv->budget = hbm_budget;
    sv->max_slots = max_slots;
    if (cudaGetDevice(&sv->dev) != cudaSuccess) {
        delete sv;
        return HH_ECUDA;
    }
    sv->threads.emplace_back([sv] { sv->engine(); });
    for (int w = 0; w < 4; ++w) sv->threads.emplace_back([sv] { sv->worker(); });
    *out = new hh_server{sv};
    return HH_OK;
}

hh_status hh_server_submit(hh_server* srv, const hh_params* params, const void* d_f, const void* d_g, void* d_u,
                           unsigned long long* ticket) {
    if (!srv || !params || !d_f || !d_g || !d_u || !ticket) return HH_EINVAL;
    const hh_status v = hh::validate(params);
    if (v != HH_OK) return v;
    size_t fp = 0;
    {
        std::unique_ptr<hh::SolverBase> s(hh::make_solver(params));
        fp = s->plan(nullptr);
    }
    hh::Server* sv = srv->sv;
    if (fp > sv->budget) return HH_ENOMEM;
    auto* r = new hh::ServerReq();
    r->P = *params;
    r->f = (const c128*)d_f;
    r->g = (const c128*)d_g;
    r->u = (c128*)d_u;
    r->fp = fp;
    r->t_submit = r->t_admit = std::chrono::steady_clock::now();
    std::lock_guard<std::mutex> lk(sv->mu);
    r->ticket = sv->next++;
    sv->all[r->ticket] = r;
    sv->pending.push_back(r);
    sv->cv_work.notify_all();
    *ticket = r->ticket;
    return HH_OK;
}

hh_status hh_server_poll(hh_server* srv, unsigned long long ticket, hh_status* result, hh_stats* stats) {
    if (!srv || !result) return HH_EINVAL;
    hh::Server* sv = srv->sv;
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->all.find(ticket);
    if (it == sv->all.end()) return HH_EINVAL;
    hh::ServerReq* r = it->second;
    if (!r->done) return HH_EPENDING;
    *result = r->st;
    if (stats) *stats = r->stats;
    sv->all.erase(it);
    delete r;
    return HH_OK;
}

void hh_server_destroy(hh_server* srv) {
    if (!srv) return;
    hh::Server* sv = srv->sv;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
        sv->cv_work.notify_all();
        sv->cv_engine.notify_all();
    }
    for (auto& t : sv->threads) t.join();
    for (auto& kv : sv->all) {
        if (kv.second->s) delete kv.second->s;
        delete kv.second;
    }
    delete sv;
    delete srv;
}

hh_status hh_solve(hh_handle* h, const void* d_f, const void* d_g, void* d_u, void* stream, hh_stats* stats) {
    if (!h || !d_f || !d_g || !d_u) return HH_EINVAL;
    h->s->stream = (cudaStream_t)stream;
    return h->s->solve((const c128*)d_f, (const c128*)d_g, (c128*)d_u, stats);
}

hh_status hh_solve_host(hh_handle* h, const void* h_f, const void* h_g, void* h_u, void* stream,
                        hh_stats* stats) {
    if (!h || !h_f || !h_g || !h_u) return HH_EINVAL;
    hh::SolverBase* s = h->s;
    s->stream = (cudaStream_t)stream;
    const size_t N = (size_t)s->npoints();
    const size_t ng = s->P.dim == 2 ? 4 * (size_t)(s->P.n + 2) : 2;
    if (cudaMemcpyAsync(s->staging_f(), h_f, sizeof(c128) * N, cudaMemcpyHostToDevice, s->stream) != cudaSuccess ||
        cudaMemcpyAsync(s->staging_g(), h_g, sizeof(c128) * ng, cudaMemcpyHostToDevice, s->stream) != cudaSuccess)
        return HH_ECUDA;
    const hh_status st = s->solve(s->staging_f(), s->staging_g(), s->iterate(), stats);
    if (cudaMemcpyAsync(h_u, s->iterate(), sizeof(c128) * N, cudaMemcpyDeviceToHost, s->stream) != cudaSuccess ||
        cudaStreamSynchronize(s->stream) != cudaSuccess)
        return HH_ECUDA;
    return st;
}

hh_status hh_residual(hh_handle* h, const void* d_f, const void* d_g, const void* d_u, void* stream,
                      double* rel_res) {
    if (!h || !d_f || !d_g || !d_u || !rel_res) return HH_EINVAL;
    h->s->stream = (cudaStream_t)stream;
    return h->s->residual((const c128*)d_f, (const c128*)d_g, (const c128*)d_u, rel_res);
}

void hh_destroy(hh_handle* h) {
    if (!h) return;
    delete h->s;
    delete h;
}

const char* hh_status_string(hh_status s) {
    switch (s) {
        case HH_OK: return "ok";
        case HH_EINVAL: return "invalid argument";
        case HH_ENOMEM: return "out of device memory";
        case HH_ENOCONV: return "iteration did not converge";
        case HH_EBREAKDOWN: return "zero pivot in a factorisation";
        case HH_ETIMEOUT: return "bounded device wait gave up";
        case HH_ECUDA: return "CUDA runtime error";
        case HH_ENOTIMPL: return "not implemented";
        case HH_ETOOLARGE: return "problem larger than the fixed static scratch (n + 2 > HH_NOALLOC_MAX_ROWS)";
        case HH_EPENDING: return "request not finished yet";
    }
    return "unknown status";
}

hh_status hh_node_info(const hh_handle* h, int node, int info[10]) {
    if (!h) return HH_EINVAL;
    return h->s->node_info(node, info);
}
hh_status hh_apply_operator(hh_handle* h, int node, const void* d_x, void* d_y, int ncols, void* stream) {
    if (!h) return HH_EINVAL;
    h->s->stream = (cudaStream_t)stream;
    return h->s->apply_operator(node, (const c128*)d_x, (c128*)d_y, ncols);
}
hh_status hh_leaf_solve(hh_handle* h, int leaf, const void* d_v, void* d_x, int ncols, void* stream) {
    if (!h) return HH_EINVAL;
    h->s->stream = (cudaStream_t)stream;
    return h->s->leaf_solve(leaf, (const c128*)d_v, (c128*)d_x, ncols);
}
hh_status hh_interface_map(hh_handle* h, int child, int adjoint, const void* d_in, void* d_out, int ncols,
                           void* stream) {
    if (!h) return HH_EINVAL;
    h->s->stream = (cudaStream_t)stream;
    return h->s->interface_map(child, adjoint, (const c128*)d_in, (c128*)d_out, ncols);
}
hh_status hh_get_basis(hh_handle* h, int child, void* h_V, double* h_sigma) {
    if (!h) return HH_EINVAL;
    return h->s->get_basis(child, h_V, h_sigma);
}
hh_status hh_coarse_apply(hh_handle* h, int node, const void* d_r, void* d_z, void* stream) {
    if (!h) return HH_EINVAL;
    h->s->stream = (cudaStream_t)stream;
    return h->s->coarse_apply(node, (const c128*)d_r, (c128*)d_z);
}
hh_status hh_precondition(hh_handle* h, const void* d_r, void* d_z, void* stream) {
    if (!h) return HH_EINVAL;
    h->s->stream = (cudaStream_t)stream;
    return h->s->precondition((const c128*)d_r, (c128*)d_z);
}
hh_status hh_profile_enable(hh_handle* h, int enable) {
    if (!h) {
        hh::g_prof_default = enable != 0;
        return HH_OK;
    }
    h->s->prof_configure(enable != 0, h->s->prof_mask, true);
    return HH_OK;
}
hh_status hh_profile_categories(hh_handle* h, unsigned mask) {
    if (!h) {
        hh::g_prof_mask_default = mask;
        return HH_OK;
    }
    // the totals so far stay; graphs captured under the old selection are dropped
    h->s->prof_configure(h->s->prof_on, mask, false);
    return HH_OK;
}
hh_status hh_profile_read(const hh_handle* h, int category, double* total_ms, long long* launches,
                          double* alg_bytes, double* alg_flops) {
    if (!h || category < 0 || category >= hh::PC_NCAT) return HH_EINVAL;
    if (total_ms) *total_ms = h->s->prof_ms[category];
    if (launches) *launches = h->s->prof_n[category];
    if (alg_bytes) *alg_bytes = h->s->prof_bytes[category];
    if (alg_flops) *alg_flops = h->s->prof_flops[category];
    return HH_OK;
}
unsigned long long hh_launch_count(void) { return hh::g_launches.load(); }

hh_status hh_autotune_report(char* buf, size_t cap, size_t* len) {
    std::string out = "[";
    {
        std::lock_guard<std::mutex> lk(hh::g_tune_mu);
        bool first = true;
        for (const auto& kv : hh::g_tune) {
            const hh::TuneKey& k = kv.first;
            const hh::TuneEntry& e = kv.second;
            char line[320];
            if (k.kind == 0)
                std::snprintf(line, sizeof line,
                              "{\"device\":%d,\"what\":\"%s\",\"b_max\":%d,\"Sx\":%d,\"nrhs\":%d,\"leaves\":%d,"
                              "\"cuda_cores_ms\":%.4f,\"tensor_cores_ms\":%.4f,\"chosen\":\"%s\"}",
                              k.dev, k.a == 0 ? "transform_in" : "transform_out", k.b, k.c, k.d / 64, k.d % 64,
                              e.ms[0], e.ms[1], e.choice ? "tensor_cores" : "cuda_cores");
            else
                std::snprintf(line, sizeof line,
                              "{\"device\":%d,\"what\":\"fused_sweep_cluster\",\"b_max\":%d,\"Sx\":%d,"
                              "\"leaves\":%d,\"precision\":\"%s\",\"cluster16_ms\":%.4f,\"cluster8_ms\":%.4f,"
                              "\"chosen\":%d}",
                              k.dev, k.a, k.b, k.c, k.d == 4 ? "mixed" : "fp64", e.ms[0], e.ms[1], e.choice ? 8 : 16);
            if (!first) out += ",";
            out += line;
            first = false;
        }
    }
    out += "]";
    if (len) *len = out.size();
    if (buf && cap > 0) {
        const size_t n = std::min(cap - 1, out.size());
        std::memcpy(buf, out.data(), n);
        buf[n] = 0;
    }
    return HH_OK;
}

hh_status hh_debug_set_wait_limit(long long polls) {
    hh::set_wait_polls(polls < 0 ? -1 : polls);
    return HH_OK;
}

hh_status hh_sketch_samples(hh_handle* h, int child, void* d_out, void* stream) {
    if (!h) return HH_EINVAL;
    h->s->stream = (cudaStream_t)stream;
    return h->s->sketch_samples(child, (c128*)d_out);
}

}  // extern "C"
