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
// element (row, k) of a 32-wide K chunk at (row / 8) * 1024 + (k / 4) * 128 +
// (row % 8) * 16 + (k % 4) * 4 bytes (leading-dimension offset 128 B between core
// matrices along K, stride offset 1024 B between 8-row groups).  The B operand is laid
// out that way once per leaf in global memory (tc_prepare_v) and each K chunk reaches
// shared memory by one bulk copy (TMA engine); the A tile is split and transposed by
// the threads on its way in.  One CTA per SM (212 KB of shared memory, all 512 tensor-
// memory columns), persistent over the (leaf, column tile) pairs, two pipeline stages.
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

constexpr int TC_THREADS = 512;          // 16 warps: four per 32-lane quarter of tensor memory
constexpr int TC_KQ_T = TC_THREADS / 64;  // K quads of a chunk a thread does not stage between its own
constexpr int TC_COLS = 64;              // complex columns per tile (M = 128 real rows)
constexpr int TC_KC = 32;                // K per pipeline chunk (4 MMAs of K = 8)
constexpr int TC_NB_MAX = 144;           // N per accumulator (b <= 136 rounded up to 16)
constexpr int TC_TMEM_COLS = 512;
constexpr int TC_D1_COL = 256;           // tensor-memory column of the second accumulator
constexpr uint32_t TC_A_BYTES = 2u * 128u * TC_KC * 4u;                    // hi + lo: 32 KiB
constexpr uint32_t TC_B_BYTES_MAX = 2u * 2u * TC_NB_MAX * TC_KC * 4u;      // hi + lo: 72 KiB
constexpr uint32_t TC_STAGE_BYTES = TC_A_BYTES + TC_B_BYTES_MAX;
constexpr uint32_t TC_SMEM = 2u * TC_STAGE_BYTES + 1024u + 256u;          // + alignment, barriers
constexpr uint32_t TC_WAIT_LIMIT = 1u << 22;                               // polls (~0.3-1 s)

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
    return (uint32_t)((row >> 3) * 1024 + (kk >> 2) * 128 + (row & 7) * 16 + (kk & 3) * 4);
}

// Shared-memory matrix descriptor: K-major, no swizzle, leading-dimension byte offset
// 128 (next core matrix along K), stride byte offset 1024 (next 8-row group).
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((128u >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((1024u >> 4) & 0x3FFFu) << 32;
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

}  // namespace

// Geometry of a launch (every task padded to the largest band).
struct TcGeom {
    int nb;      // N per accumulator: b_max rounded up to 16
    int ks;      // K steps of 8: b_max rounded up to 8, over 8
    int nq;      // K chunks of 32
    uint32_t b_bytes;   // bytes of one chunk of the B operand (hi + lo)
};
HH_HD TcGeom tc_geom(int b_max) {
    TcGeom g;
    g.nb = (b_max + 15) & ~15;
    g.ks = (b_max + 7) / 8;
    g.nq = (g.ks + 3) / 4;
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
__global__ void __launch_bounds__(TC_THREADS, 1) k_tc_transform(const EigTask* __restrict__ tasks, int ntasks,
                                                                int which, int Sx, int nrhs, int b_max,
                                                                int tiles_per_task, uint32_t limit, int* err,
                                                                const int* gate) {
    // a set stop word (written by an earlier launch: the same for every CTA) skips the
    // launch before the tensor memory is allocated
    if (gate && *gate) return;
    extern __shared__ __align__(1024) unsigned char tsm_raw[];
    unsigned char* tsm = (unsigned char*)(((uintptr_t)tsm_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* full = (uint64_t*)(tsm + 2 * TC_STAGE_BYTES);       // bulk copy of B landed, per stage
    uint64_t* done = full + 2;                                     // MMAs of a stage finished, per stage
    uint32_t* tmem_slot = (uint32_t*)(done + 2);
    int* abort_flag = (int*)(tmem_slot + 1);
    const TcGeom g = tc_geom(b_max);
    const int J = Sx * nrhs;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (tid == 0) {
        mbar_init(&full[0], 1);
        mbar_init(&full[1], 1);
        mbar_init(&done[0], 1);
        mbar_init(&done[1], 1);
        abort_flag[0] = abort_flag[1] = abort_flag[2] = 0;
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

    const uint32_t idesc = idesc_tf32(g.nb);
    uint32_t use[2] = {0u, 0u};     // committed uses of each stage (this CTA)
    bool copy_pending[2] = {false, false};   // thread 0: a bulk copy issued, not yet seen landed
    uint32_t chunk = 0;             // chunks issued so far (stage = chunk & 1)
    bool ok = true;
    const int ntiles = ntasks * tiles_per_task;

    // Only thread 0 waits on the barriers (and issues the MMAs); the others learn the
    // outcome through the shared abort word after a block barrier, so every thread takes
    // the same path and the block barriers stay matched.
    //
    // Each thread stages column j = tid % 64 of the tile and the K quads kq = tid / 64,
    // tid / 64 + TC_KQ_T, ...: 8 complex values per chunk, loaded into registers one chunk
    // ahead (the loads of chunk q + 1, or of the next tile's first chunk, are in flight
    // while chunk q's MMAs are issued and run).
    const int jcol = tid & 63, kq0 = tid >> 6;
    constexpr int NU = TC_KC / 4 / TC_KQ_T;   // K quads a thread stages per chunk
    c64 pre[NU][4];
    auto load_chunk = [&](int t, int q) {
        const EigTask& tq = tasks[t / tiles_per_task];
        const int p = (t % tiles_per_task) * TC_COLS + jcol;
        const c64* src = (const c64*)(which == 0 ? tq.F : tq.Fh);
        const int bb = tq.b;
#pragma unroll
        for (int u = 0; u < NU; ++u)
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int k = q * TC_KC + (kq0 + TC_KQ_T * u) * 4 + i;
                float2 v = make_float2(0.f, 0.f);
                if (p < J && k < bb) v = __ldg((const float2*)(src + (size_t)k * J + p));
                pre[u][i] = c64{v.x, v.y};
            }
    };
    // thread 0: the bulk copy of chunk (t, q)'s B operand into stage s
    auto issue_b = [&](int t, int q, int s) {
        const EigTask& tq = tasks[t / tiles_per_task];
        const unsigned char* src = (const unsigned char*)(which == 0 ? tq.vt_emb : tq.vn_emb);
        mbar_arrive_expect_tx(&full[s], g.b_bytes);
        bulk_g2s(tsm + s * TC_STAGE_BYTES + TC_A_BYTES, src + (size_t)q * g.b_bytes, g.b_bytes, &full[s]);
        copy_pending[s] = true;
    };
    if (blockIdx.x < ntiles) {
        load_chunk(blockIdx.x, 0);
        if (tid == 0) issue_b(blockIdx.x, 0, 0);
    }
    for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        const EigTask tk = tasks[tile / tiles_per_task];
        const int p0 = (tile % tiles_per_task) * TC_COLS;
        const int b = tk.b;
        c64* outp = (c64*)(which == 0 ? tk.Fh : tk.W);
        // x = V x^ keeps rows [w0, w1) (all rows, or the owned rows written into the parent)
        const int rlo = which == 0 ? 0 : tk.w0, rhi = which == 0 ? b : tk.w1;
        for (int q = 0; q < g.nq; ++q, ++chunk) {
            const int s = chunk & 1;
            unsigned char* As = tsm + s * TC_STAGE_BYTES;
            unsigned char* Bs = As + TC_A_BYTES;
            // The stage's previous chunk (two back) must have finished its MMAs before its A
            // tile is overwritten: every thread waits on that commit itself, so the staging
            // below runs while thread 0 still issues the previous chunk's MMAs.  (Its B
            // operand was requested into the stage after the same wait.)  A thread whose
            // wait runs out raises this iteration's abort word.
            if (chunk >= 2 && !mbar_wait_bounded(&done[s], ((chunk - 2) >> 1) & 1u, limit > 0 ? limit : 1u)) {
                atomicCAS(err, DEV_OK, DEV_TIMEOUT);
                abort_flag[chunk & 1] = 1;
            }
            // A tile chunk from the registers: rows 2j + c, split and transposed
#pragma unroll
            for (int u = 0; u < NU; ++u) {
                uint4 hr, lr, hm, lm;
                tf32_split(pre[u][0].re, hr.x, lr.x);
                tf32_split(pre[u][1].re, hr.y, lr.y);
                tf32_split(pre[u][2].re, hr.z, lr.z);
                tf32_split(pre[u][3].re, hr.w, lr.w);
                tf32_split(pre[u][0].im, hm.x, lm.x);
                tf32_split(pre[u][1].im, hm.y, lm.y);
                tf32_split(pre[u][2].im, hm.z, lm.z);
                tf32_split(pre[u][3].im, hm.w, lm.w);
                const int kq = kq0 + TC_KQ_T * u;
                const uint32_t o_re = kmaj_off(2 * jcol, kq * 4), o_im = kmaj_off(2 * jcol + 1, kq * 4);
                *(uint4*)(As + o_re) = hr;
                *(uint4*)(As + o_im) = hm;
                *(uint4*)(As + TC_A_BYTES / 2 + o_re) = lr;
                *(uint4*)(As + TC_A_BYTES / 2 + o_im) = lm;
            }
            // prefetch the next chunk (this tile's next, or the next tile's first)
            if (q + 1 < g.nq) load_chunk(tile, q + 1);
            else if (tile + (int)gridDim.x < ntiles) load_chunk(tile + gridDim.x, 0);
            fence_async_smem();
            __syncthreads();
            // Thread 0 writes only the next iteration's abort word after this barrier, so
            // every thread reads the same value here.
            if (abort_flag[chunk & 1]) { ok = false; break; }
            if (tid == 0) {
                if (tc_wait(&full[s], use[s] & 1, limit, err)) {
                    copy_pending[s] = false;
                    tc_fence_after();
                    // descriptors of the stage's operands, advanced by address offsets (the
                    // 14-bit address field holds every shared-memory offset)
                    const uint64_t da_hi = smem_desc(smem_u32(As)), da_lo = smem_desc(smem_u32(As) + TC_A_BYTES / 2);
                    const uint64_t db_hi = smem_desc(smem_u32(Bs)), db_lo = smem_desc(smem_u32(Bs) + g.b_bytes / 2);
                    const uint32_t half = (uint32_t)(g.nb / 8) * 1024u;
                    const int nks = min(4, g.ks - 4 * q);
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) {
                        if (kk < nks) {
                            const uint64_t ko = (uint64_t)(kk * 256) >> 4;
#pragma unroll
                            for (int h = 0; h < 2; ++h) {
                                const uint32_t d = tmem + (h ? TC_D1_COL : 0);
                                const uint64_t bo = ((uint64_t)(h * half) >> 4) + ko;
                                const uint32_t acc0 = (q > 0 || kk > 0) ? 1u : 0u;
                                mma_tf32(d, da_hi + ko, db_hi + bo, idesc, acc0);
                                mma_tf32(d, da_hi + ko, db_lo + bo, idesc, 1u);
                                mma_tf32(d, da_lo + ko, db_hi + bo, idesc, 1u);
                            }
                        }
                    }
                    mma_commit(&done[s]);
                    ++use[s];
                    // the next chunk's B operand into the other stage, once that stage's
                    // MMAs (the previous chunk's) have finished reading it: the copy runs
                    // while the next chunk's A tile is staged
                    int nt = tile, nq = q + 1;
                    if (nq == g.nq) {
                        nt = tile + (int)gridDim.x;
                        nq = 0;
                    }
                    if (nt < ntiles) {
                        const int s2 = s ^ 1;
                        if (use[s2] > 0 && !tc_wait(&done[s2], (use[s2] - 1) & 1, limit, err))
                            abort_flag[(chunk + 1) & 1] = 1;
                        else issue_b(nt, nq, s2);
                    }
                } else {
                    abort_flag[(chunk + 1) & 1] = 1;   // the bulk copy may still land: drained below
                }
            }
        }
        if (!ok) break;
        // epilogue: thread 0 waits for the tile's last MMAs; then the lanes 2j, 2j + 1
        // of each warp pair up.  (An abort raised by thread 0 after the last chunk is in
        // the word of the next iteration.)
        if (tid == 0) {
            const int sl = (chunk - 1) & 1;
            if (abort_flag[chunk & 1] || !tc_wait(&done[sl], (use[sl] - 1) & 1, limit, err)) abort_flag[2] = 1;
        }
        __syncthreads();
        if (abort_flag[2]) { ok = false; break; }
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
        for (int m0 = 16 * wh; m0 < g.nb; m0 += 16 * (TC_THREADS / 128)) {
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
        // the next tile's MMAs overwrite the accumulators
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
    }
    // drain after a failed wait: no tensor-core operation or bulk copy may be in flight
    // when the block exits and its memory is freed (bounded as well)
    if (!ok && tid == 0) {
        for (int s = 0; s < 2; ++s) {
            if (use[s] > 0) mbar_wait_bounded(&done[s], (use[s] - 1) & 1, TC_WAIT_LIMIT);
            if (copy_pending[s]) mbar_wait_bounded(&full[s], use[s] & 1, TC_WAIT_LIMIT);
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
