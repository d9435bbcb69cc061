// k_tc.cu -- the eigenbasis leaf sweep's dense transforms on the tensor cores (tcgen05).
//
// The subdomain solves of Eq. (2) on the eigenbasis leaf path (k_eig.cu) spend their
// arithmetic in two complex contractions per sweep, over every column of the band's
// right-hand sides:
//     f^ = V^T f   (into the column-pencil eigenbasis)   and   x = V x^   (back),
// V the b x b generalised eigenvectors, f a b x J block (J = Sx nrhs).  In the complex64
// form they run here, on the 5th-generation tensor cores, with FP32 accuracy from the
// TF32 pipe by the three-term split a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi (a_hi the
// TF32 rounding of a, a_lo the TF32 rounding of a - a_hi; the dropped a_lo b_lo is below
// FP32 rounding), accumulated in FP32 in tensor memory.
//
// Real form of one complex product.  A tile of 64 complex columns of f is the MMA's A
// operand, M = 128 rows: row 2j + c holds part c (0 real, 1 imaginary) of column j.  The
// B operand holds the transform's matrix split by parts: rows [0, NB) its real part,
// rows [NB, 2 NB) its imaginary part (NB = b rounded up to 16, zero rows beyond b).
// Two accumulators: D0 = A * B[0, NB)^T and D1 = A * B[NB, 2NB)^T, so that lane 2j holds
// (Re f . Re V, Re f . Im V) and lane 2j + 1 holds (Im f . Re V, Im f . Im V); the
// epilogue pairs the two lanes: Re = rr - ii, Im = ri + ir.
//
// Shared-memory operands are K-major without swizzle, in 8-row x 16-byte core matrices:
// element (row, k) of a 16-wide K chunk at (row / 8) * 512 + (k / 4) * 128 +
// (row % 8) * 16 + (k % 4) * 4 bytes (leading-dimension offset 128 B between core
// matrices along K, stride offset 512 B between 8-row groups).  The B operand is laid
// out that way once per leaf in global memory (tc_prepare_v) and each K chunk reaches
// shared memory by one bulk copy (TMA engine); the A tile is split and transposed by
// the threads on its way in.  One CTA per SM (209 KB of shared memory in four pipeline
// stages, all 512 tensor-memory columns), persistent over the (leaf, column tile) pairs,
// warp-specialised: sixteen staging warps, one warp issuing the MMAs and one issuing the
// bulk copies, handing the stages over by mbarriers.
//
// Every wait is bounded: a wait that gives up records DEV_TIMEOUT, the CTA stops
// issuing work, waits (bounded) for its tensor-core operations in flight, frees its
// tensor memory and returns.
#include <algorithm>
#include <atomic>
#include <cstdint>

#include "kernels.h"

namespace hh {

namespace {

constexpr int TC_STAGERS = 512;          // 16 warps stage A and run the epilogue (four per 32-lane quarter of tensor memory)
constexpr int TC_THREADS = TC_STAGERS + 64;   // + the MMA-issuer warp and the B-producer warp
constexpr int TC_ISSUER = TC_STAGERS;         // lane 0 of warp 16
constexpr int TC_PRODUCER = TC_STAGERS + 32;  // lane 0 of warp 17
constexpr int TC_COLS = 64;              // complex columns per tile (M = 128 real rows)
constexpr int TC_KC = 16;                // K per pipeline chunk (2 MMAs of K = 8)
constexpr int TC_STAGES = 4;             // pipeline stages (A tile and B operand each)
constexpr uint32_t TC_SBO = 8u * TC_KC * 4u;   // bytes between 8-row groups of a chunk
constexpr int TC_NB_MAX = 144;           // N per accumulator (b <= 136 rounded up to 16)
constexpr int TC_TMEM_COLS = 512;
constexpr int TC_D1_COL = 256;           // tensor-memory column of the second accumulator
constexpr uint32_t TC_A_BYTES = 2u * 128u * TC_KC * 4u;                    // hi + lo: 16 KiB
constexpr uint32_t TC_B_BYTES_MAX = 2u * 2u * TC_NB_MAX * TC_KC * 4u;      // hi + lo: 36 KiB
constexpr uint32_t TC_STAGE_BYTES = TC_A_BYTES + TC_B_BYTES_MAX;
constexpr uint32_t TC_SMEM = TC_STAGES * TC_STAGE_BYTES + 1024u + 256u;   // + alignment, barriers
constexpr uint32_t TC_WAIT_LIMIT = 1u << 22;                               // polls (~0.3-1 s)
static_assert(TC_SMEM <= 227u * 1024u, "tensor-core transform stages exceed shared memory");
static_assert(TC_STAGERS == 64 * (TC_KC / 4) * 2, "one (column, K quad, part) per staging thread");

__device__ __forceinline__ uint32_t tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}
// (hi, lo) with hi = tf32(x), lo = tf32(x - hi), as the 32-bit containers the MMA reads
__device__ __forceinline__ void tf32_split(float x, uint32_t& hi, uint32_t& lo) {
    hi = tf32_rna(x);
    lo = tf32_rna(x - __uint_as_float(hi));
}

// byte offset of element (row, k) inside one K chunk of a K-major operand
__device__ __forceinline__ uint32_t kmaj_off(int row, int kk) {
    return (uint32_t)((row >> 3) * (int)TC_SBO + (kk >> 2) * 128 + (row & 7) * 16 + (kk & 3) * 4);
}

// Shared-memory matrix descriptor: K-major, no swizzle, leading-dimension byte offset
// 128 (next core matrix along K), stride byte offset TC_SBO (next 8-row group).
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((128u >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((TC_SBO >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;                 // descriptor version of this architecture
    return d;                               // base offset 0, layout: no swizzle
}

// Instruction descriptor: kind::tf32, FP32 accumulator, A and B TF32, both K-major,
// M = 128, N = n.
__host__ __device__ __forceinline__ uint32_t idesc_tf32(int n) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 16 consecutive 32-bit tensor-memory columns of this thread's lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Bounded wait (thread 0): false, and the error word set, after `limit` polls (limit 0:
// give up at once, the testing form of a wait that runs out).
__device__ __forceinline__ bool tc_wait(uint64_t* bar, uint32_t parity, uint32_t limit, int* err) {
    if (limit > 0 && mbar_wait_bounded(bar, parity, limit)) return true;
    atomicCAS(err, DEV_OK, DEV_TIMEOUT);
    return false;
}
// The pipeline roles' wait: false after `limit` polls (the error word set and the shared
// abort word raised, so that the other roles stop too) or as soon as another role has raised
// the abort word.
__device__ __forceinline__ bool role_wait(uint64_t* bar, uint32_t parity, uint32_t limit, int* err,
                                          volatile int* abort_word) {
    for (uint32_t it = 0; it < limit; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*abort_word) return false;
        if (it > 64) __nanosleep(32);
    }
    atomicCAS(err, DEV_OK, DEV_TIMEOUT);
    *abort_word = 1;
    return false;
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

}  // namespace

// Geometry of a launch (every task padded to the largest band).
struct TcGeom {
    int nb;      // N per accumulator: b_max rounded up to 16
    int ks;      // K steps of 8: b_max rounded up to 8, over 8
    int nq;      // K chunks of TC_KC
    uint32_t b_bytes;   // bytes of one chunk of the B operand (hi + lo)
};
HH_HD TcGeom tc_geom(int b_max) {
    TcGeom g;
    g.nb = (b_max + 15) & ~15;
    g.ks = (b_max + 7) / 8;
    g.nq = (g.ks + TC_KC / 8 - 1) / (TC_KC / 8);
    g.b_bytes = 2u * 2u * (uint32_t)g.nb * TC_KC * 4u;
    return g;
}

size_t tc_vemb_bytes(int b_max) {
    const TcGeom g = tc_geom(b_max);
    return (size_t)g.nq * g.b_bytes;
}

// B operand of one leaf and one transform in the chunked K-major layout:
// trans = 1: B[h NB + m][k] = part_h(V[k][m]) (f^ = V^T f);
// trans = 0: B[h NB + a][k] = part_h(V[a][k]) (x = V x^).
// Row n of split s of chunk q starts at q b_bytes + s (b_bytes / 2).
__global__ void k_tc_prepare_v(const EigTask* __restrict__ tasks, int b_max) {
    const EigTask tk = tasks[blockIdx.y];
    const TcGeom g = tc_geom(b_max);
    const int b = tk.b;
    const c64* V = (const c64*)tk.V;
    const int nt = 2 * g.nb, kp = g.nq * TC_KC;
    for (int trans = 0; trans < 2; ++trans) {
        unsigned char* out = (unsigned char*)(trans ? tk.vt_emb : tk.vn_emb);
        for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nt * kp; e += gridDim.x * blockDim.x) {
            const int n = e / kp, k = e - n * kp;
            const int h = n >= g.nb, r = n - h * g.nb;
            float x = 0.f;
            if (r < b && k < b) {
                const c64 v = trans ? V[(size_t)k * b + r] : V[(size_t)r * b + k];
                x = h ? v.im : v.re;
            }
            uint32_t hi, lo;
            tf32_split(x, hi, lo);
            const int q = k / TC_KC, kk = k - q * TC_KC;
            unsigned char* base = out + (size_t)q * g.b_bytes + kmaj_off(n, kk);
            *(uint32_t*)base = hi;
            *(uint32_t*)(base + g.b_bytes / 2) = lo;
        }
    }
}

void launch_tc_prepare_v(const EigTask* d_tasks, int ntasks, int b_max, cudaStream_t s) {
    dim3 grid(16, ntasks);
    k_tc_prepare_v<<<grid, 256, 0, s>>>(d_tasks, b_max);
    note_launch();
}

// which = 0: Fh = V^T F (input F in node order [b][J], output Fh as fh_col says);
// which = 1: W = V Fh (input Fh, output W in node order).  The tiles run along the
// input's contiguous column index p.
//
// Warp-specialised pipeline over the CTA's chunks c = 0, 1, ... (stage c % TC_STAGES),
// with no block barrier inside the loop:
//   staging warps 0-15: wait until the MMAs of chunk c - TC_STAGES have finished (the
//       stage is free), split and transpose their part of A(c) into the stage, arrive on
//       a_full; after a tile's last chunk, wait for its MMAs, read the accumulators out of
//       tensor memory, write the tile and arrive on tfree;
//   producer (warp 17, lane 0): wait until the stage is free, bulk-copy B(c) into it
//       (b_full), up to TC_STAGES chunks ahead of the MMAs;
//   issuer (warp 16, lane 0): before a tile's first chunk wait for tfree (the previous
//       tile's accumulators read out), then per chunk wait for a_full and b_full, issue
//       the MMAs and commit them to done.
// Every wait is bounded and also ends when another role has raised the abort word; the
// roles then leave their loops, the issuer waits (bounded) for its MMAs and the producer
// for its copies, and the tensor memory is freed.
__global__ void __launch_bounds__(TC_THREADS, 1) k_tc_transform(const EigTask* __restrict__ tasks, int ntasks,
                                                                int which, int Sx, int nrhs, int b_max,
                                                                int tiles_per_task, uint32_t limit, int* err,
                                                                const int* gate) {
    // a set stop word (written by an earlier launch: the same for every CTA) skips the
    // launch before the tensor memory is allocated
    if (gate && *gate) return;
    extern __shared__ __align__(1024) unsigned char tsm_raw[];
    unsigned char* tsm = (unsigned char*)(((uintptr_t)tsm_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* a_full = (uint64_t*)(tsm + TC_STAGES * TC_STAGE_BYTES);   // A part of a stage staged
    uint64_t* b_full = a_full + TC_STAGES;                               // B operand of a stage landed
    uint64_t* done = b_full + TC_STAGES;                                 // MMAs of a stage finished
    uint64_t* tfree = done + TC_STAGES;                                  // accumulators read out
    uint32_t* tmem_slot = (uint32_t*)(tfree + 1);
    volatile int* abort_word = (volatile int*)(tmem_slot + 1);
    const TcGeom g = tc_geom(b_max);
    const int J = Sx * nrhs;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t lim = limit > 0 ? limit : 1u;

    if (tid == 0) {
        for (int s = 0; s < TC_STAGES; ++s) {
            mbar_init(&a_full[s], TC_STAGERS);
            mbar_init(&b_full[s], 1);
            mbar_init(&done[s], 1);
        }
        mbar_init(tfree, TC_STAGERS);
        *abort_word = 0;
        fence_barrier_init();
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TC_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int ntiles = ntasks * tiles_per_task;
    // the testing form of a wait that runs out (limit 0): the first wait of each role gives up
    const bool give_up = limit == 0;

    if (tid < TC_STAGERS) {
        // ------------------------------------------------------------ staging warps
        // part (re or im) of four consecutive K of one column: column tid % 64, K quad
        // (tid / 64) % 4, part tid / 256; loaded into registers one chunk ahead
        const int jcol = tid & 63, kq = (tid >> 6) & 3, part = tid >> 8;
        float pre[4];
        auto load_chunk = [&](int t, int q) {
            const EigTask& tq = tasks[t / tiles_per_task];
            const int p = (t % tiles_per_task) * TC_COLS + jcol;
            const c64* src = (const c64*)(which == 0 ? tq.F : tq.Fh);
            const int bb = tq.b;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int k = q * TC_KC + kq * 4 + i;
                pre[i] = (p < J && k < bb) ? __ldg((const float*)(src + (size_t)k * J + p) + part) : 0.f;
            }
        };
        uint32_t c = 0;
        bool ok = !give_up;
        if (give_up) {
            atomicCAS(err, DEV_OK, DEV_TIMEOUT);
            *abort_word = 1;
        }
        if (ok && blockIdx.x < ntiles) load_chunk(blockIdx.x, 0);
        for (int tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x) {
            const EigTask tk = tasks[tile / tiles_per_task];
            const int p0 = (tile % tiles_per_task) * TC_COLS;
            const int b = tk.b;
            c64* outp = (c64*)(which == 0 ? tk.Fh : tk.W);
            // x = V x^ keeps rows [w0, w1) (all rows, or the owned rows written into the parent)
            const int rlo = which == 0 ? 0 : tk.w0, rhi = which == 0 ? b : tk.w1;
            for (int q = 0; q < g.nq; ++q, ++c) {
                const int s = (int)(c % TC_STAGES);
                if (c >= TC_STAGES && !role_wait(&done[s], ((c - TC_STAGES) / TC_STAGES) & 1u, lim, err, abort_word)) {
                    ok = false;
                    break;
                }
                unsigned char* As = tsm + s * TC_STAGE_BYTES;
                uint4 hi, lo;
                tf32_split(pre[0], hi.x, lo.x);
                tf32_split(pre[1], hi.y, lo.y);
                tf32_split(pre[2], hi.z, lo.z);
                tf32_split(pre[3], hi.w, lo.w);
                const uint32_t o = kmaj_off(2 * jcol + part, kq * 4);
                *(uint4*)(As + o) = hi;
                *(uint4*)(As + TC_A_BYTES / 2 + o) = lo;
                // the next chunk's loads (this tile's next, or the next tile's first)
                if (q + 1 < g.nq) load_chunk(tile, q + 1);
                else if (tile + (int)gridDim.x < ntiles) load_chunk(tile + gridDim.x, 0);
                fence_async_smem();
                mbar_arrive(&a_full[s]);
            }
            if (!ok) break;
            // epilogue: the tile's last MMAs, then the lanes 2j, 2j + 1 of each warp pair up
            const uint32_t cl = c - 1;
            if (!role_wait(&done[cl % TC_STAGES], (cl / TC_STAGES) & 1u, lim, err, abort_word)) {
                ok = false;
                break;
            }
            tc_fence_after();
            // the warps w, w + 4, ... share the tensor-memory lanes 32 (w % 4) .. + 31 and take
            // interleaved 16-column groups of the accumulators
            const int wq = warp & 3, wh = warp >> 2;
            const int jl = wq * 16 + (lane >> 1);        // complex column of this lane pair
            const bool even = (lane & 1) == 0;
            const int p = p0 + jl;
            size_t col = 0;
            // which = 0 writes Fh (fh_col of node column p); which = 1 reads Fh along p and
            // writes the node column p (node order) or (p % Sx) nrhs + p / Sx (line-major Fh)
            if (p < J)
                col = which == 0 ? fh_col((size_t)p, Sx, nrhs)
                                 : (eig_line_major(nrhs) ? (size_t)(p % Sx) * nrhs + p / Sx : (size_t)p);
            const uint32_t lane_base = tmem + ((uint32_t)(wq * 32) << 16);
            for (int m0 = 16 * wh; m0 < g.nb; m0 += 16 * (TC_STAGERS / 128)) {
                float d0[16], d1[16];
                tmem_ld16(lane_base + (uint32_t)m0, d0);
                tmem_ld16(lane_base + (uint32_t)(TC_D1_COL + m0), d1);
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    const float v0 = __shfl_xor_sync(0xffffffffu, even ? d0[8 + t] : d0[t], 1);
                    const float v1 = __shfl_xor_sync(0xffffffffu, even ? d1[8 + t] : d1[t], 1);
                    const int m = even ? m0 + t : m0 + 8 + t;
                    c64 o;
                    if (even) o = c64{d0[t] - v1, d1[t] + v0};          // rr - ii, ri + ir
                    else o = c64{v0 - d1[8 + t], v1 + d0[8 + t]};
                    if (p < J && m >= rlo && m < rhi) outp[(size_t)(m - rlo) * J + col] = o;
                }
            }
            // the next tile's MMAs may overwrite the accumulators
            tc_fence_before();
            mbar_arrive(tfree);
        }
    } else if (tid == TC_ISSUER) {
        // ------------------------------------------------------------ MMA issuer
        const uint32_t idesc = idesc_tf32(g.nb);
        uint32_t c = 0, ntile = 0;
        bool ok = !give_up;
        for (int tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x, ++ntile) {
            if (ntile > 0 && !role_wait(tfree, (ntile - 1) & 1u, lim, err, abort_word)) break;
            for (int q = 0; q < g.nq; ++q, ++c) {
                const int s = (int)(c % TC_STAGES);
                const uint32_t par = (c / TC_STAGES) & 1u;
                if (!role_wait(&a_full[s], par, lim, err, abort_word) ||
                    !role_wait(&b_full[s], par, lim, err, abort_word)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                unsigned char* As = tsm + s * TC_STAGE_BYTES;
                const uint32_t a_addr = smem_u32(As), b_addr = a_addr + TC_A_BYTES;
                // descriptors advanced by address offsets (the 14-bit address field holds
                // every shared-memory offset)
                const uint64_t da_hi = smem_desc(a_addr), da_lo = smem_desc(a_addr + TC_A_BYTES / 2);
                const uint64_t db_hi = smem_desc(b_addr), db_lo = smem_desc(b_addr + g.b_bytes / 2);
                const uint64_t half = (uint64_t)((g.nb / 8) * TC_SBO) >> 4;
                const int nks = min(TC_KC / 8, g.ks - (TC_KC / 8) * q);
#pragma unroll
                for (int kk = 0; kk < TC_KC / 8; ++kk) {
                    if (kk < nks) {
                        const uint64_t ko = (uint64_t)(kk * 256) >> 4;
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const uint32_t d = tmem + (h ? TC_D1_COL : 0);
                            const uint64_t bo = (h ? half : 0) + ko;
                            const uint32_t acc0 = (q > 0 || kk > 0) ? 1u : 0u;
                            mma_tf32(d, da_hi + ko, db_hi + bo, idesc, acc0);
                            mma_tf32(d, da_hi + ko, db_lo + bo, idesc, 1u);
                            mma_tf32(d, da_lo + ko, db_hi + bo, idesc, 1u);
                        }
                    }
                }
                mma_commit(&done[s]);
            }
        }
        // no MMA may be in flight when the block's tensor memory is freed: they complete in
        // order, so the last commit covers them all
        if (c > 0) mbar_wait_bounded(&done[(c - 1) % TC_STAGES], ((c - 1) / TC_STAGES) & 1u, TC_WAIT_LIMIT);
    } else if (tid == TC_PRODUCER) {
        // ------------------------------------------------------------ B producer
        uint32_t c = 0;
        bool ok = !give_up;
        for (int tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x) {
            const EigTask& tq = tasks[tile / tiles_per_task];
            const unsigned char* src = (const unsigned char*)(which == 0 ? tq.vt_emb : tq.vn_emb);
            for (int q = 0; q < g.nq; ++q, ++c) {
                const int s = (int)(c % TC_STAGES);
                if (c >= TC_STAGES && !role_wait(&done[s], ((c - TC_STAGES) / TC_STAGES) & 1u, lim, err, abort_word)) {
                    ok = false;
                    break;
                }
                mbar_arrive_expect_tx(&b_full[s], g.b_bytes);
                bulk_g2s(tsm + s * TC_STAGE_BYTES + TC_A_BYTES, src + (size_t)q * g.b_bytes, g.b_bytes, &b_full[s]);
            }
        }
        // no bulk copy may be in flight when the block exits: wait for the last ones issued
        for (uint32_t k = 0; k < (uint32_t)TC_STAGES && k < c; ++k) {
            const uint32_t ck = c - 1 - k;
            mbar_wait_bounded(&b_full[ck % TC_STAGES], (ck / TC_STAGES) & 1u, TC_WAIT_LIMIT);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS)
                     : "memory");
    }
}

int tc_transform_ready() {
    static std::atomic<unsigned long long> attr{0};
    const bool ok = once_per_device(attr, [] {
        return cudaFuncSetAttribute(k_tc_transform, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM) ==
               cudaSuccess;
    });
    return ok ? 1 : 0;
}

void launch_tc_transform(int which, const EigTask* d_tasks, int ntasks, int b_max, int Sx, int nrhs, int* err,
                         cudaStream_t s, const int* gate) {
    const int J = Sx * nrhs;
    const int tiles_per_task = (J + TC_COLS - 1) / TC_COLS;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int grid = ntasks * tiles_per_task;
    if (grid > sms) grid = sms > 0 ? sms : 1;     // one block per SM (shared and tensor memory)
    const uint32_t limit = (uint32_t)std::min<long long>(wait_polls(TC_WAIT_LIMIT), 0xFFFFFFFFll);
    k_tc_transform<<<grid, TC_THREADS, TC_SMEM, s>>>(d_tasks, ntasks, which, Sx, nrhs, b_max, tiles_per_task, limit,
                                                     err, gate);
    note_launch();
}

}  // namespace hh
