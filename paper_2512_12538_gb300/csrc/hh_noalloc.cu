// hh_noalloc.cu -- hh_residual_noalloc: the relative residual ||b - A u|| / ||b|| of
// the global impedance problem without any device allocation.
//
// The handle-based hh_residual assembles b into a handle buffer (k_rhs), forms r in
// another (k_apply, with per-block norm partials in handle scratch) and reduces the
// partials with k_sum.  This variant fuses the three: every warp assembles b and r for
// one grid row on the fly and leaves the row's (sum |r|^2, sum |b|^2) in a file-scope
// device array; the last block to finish adds the rows in a fixed order.  The array
// is the only scratch, its size is fixed at compile time, and it caps the number of
// grid rows a call can take.
#include <cmath>
#include <mutex>

#include "hh.h"
#include "kernels.h"

namespace hh {
namespace {

constexpr int kNaMaxRows = HH_NOALLOC_MAX_ROWS;
constexpr int kNaMaxDevices = 64;
constexpr size_t kNaRowBytes = sizeof(double2) * kNaMaxRows;          // 256 KiB
constexpr size_t kNaBytes = kNaRowBytes + 256;                        // + total and ticket

// Per-device scratch: [0, kNaRowBytes) row pairs, then the total (double2) and the
// ticket counter (unsigned) of the last-block reduction.  Every GPU that loads the
// library holds it until the process exits.
static __device__ __align__(256) unsigned char g_na_scratch[kNaBytes];

void* g_na_base[kNaMaxDevices] = {};
std::mutex g_na_mu;

// One warp per grid row j (grid-stride over rows).  Per point: b from Eq. (1) with the
// rows of A scaled by h^2 w_i w_j (the same assembly as k_rhs), then r = b - A u with
// the weighted 5-point row (the same as k_apply with v = b, sgn = 1).
__global__ void __launch_bounds__(256) k_residual_rows(const c128* __restrict__ f, const c128* __restrict__ g,
                                                       const c128* __restrict__ u, int dim, int S, double h,
                                                       double kh, double2* rows, double2* total,
                                                       unsigned* ticket) {
    const int Sx = dim == 2 ? S : 1;
    const OpGeom geo{S, Sx, kh};
    const int lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    for (int j = blockIdx.x * wpb + (threadIdx.x >> 5); j < S; j += gridDim.x * wpb) {
        double r2 = 0.0, b2 = 0.0;
        for (int i = lane; i < Sx; i += 32) {
            const size_t t = (size_t)j * Sx + i;
            const double wj = wrow(j, S), wi = wcol(i, Sx);
            c128 bv = (h * h * wi * wj) * f[t];
            if (dim == 1) {
                if (j == 0) bv = bv + h * g[0];
                if (j == S - 1) bv = bv + h * g[1];
            } else {
                if (i == 0) bv = bv + (h * wj) * g[0 * S + j];
                if (i == Sx - 1) bv = bv + (h * wj) * g[1 * S + j];
                if (j == 0) bv = bv + (h * wi) * g[2 * S + i];
                if (j == S - 1) bv = bv + (h * wi) * g[3 * S + i];
            }
            c128 ax = op_diag(j, i, geo) * u[t];
            if (Sx > 1) {
                if (i > 0) ax = ax - wj * u[t - 1];
                if (i < Sx - 1) ax = ax - wj * u[t + 1];
            }
            if (j > 0) ax = ax - wi * u[t - Sx];
            if (j < S - 1) ax = ax - wi * u[t + Sx];
            const c128 r = bv - ax;
            r2 += abs2(r);
            b2 += abs2(bv);
        }
        r2 = warp_sum(r2);
        b2 = warp_sum(b2);
        if (lane == 0) rows[j] = make_double2(r2, b2);
    }
    __threadfence();
    __syncthreads();
    __shared__ unsigned s_ticket;
    if (threadIdx.x == 0) s_ticket = atomicAdd(ticket, 1u);
    __syncthreads();
    if (s_ticket != gridDim.x - 1) return;
    __threadfence();
    // last block: thread t adds rows t, t + 256, ... in order, then a fixed tree, so the
    // result does not depend on the grid size or on which block finished last
    double a = 0.0, c = 0.0;
    for (int j = threadIdx.x; j < S; j += blockDim.x) {
        const double2 v = __ldcg(rows + j);
        a += v.x;
        c += v.y;
    }
    __shared__ double red[2][8];
    a = warp_sum(a);
    c = warp_sum(c);
    if (lane == 0) {
        red[0][threadIdx.x >> 5] = a;
        red[1][threadIdx.x >> 5] = c;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double sa = 0.0, sc = 0.0;
        for (int w = 0; w < wpb; ++w) {
            sa += red[0][w];
            sc += red[1][w];
        }
        *total = make_double2(sa, sc);
        *ticket = 0u;
    }
}

// Address of this device's scratch; looked up once per device with that device current.
hh_status na_scratch(void** base) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return HH_ECUDA;
    if (dev < 0 || dev >= kNaMaxDevices) return HH_EINVAL;
    std::lock_guard<std::mutex> lock(g_na_mu);
    if (!g_na_base[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_na_scratch) != cudaSuccess || !p) return HH_ECUDA;
        g_na_base[dev] = p;
    }
    *base = g_na_base[dev];
    return HH_OK;
}

}  // namespace
}  // namespace hh

extern "C" hh_status hh_residual_noalloc(int dim, int n, double k, const void* d_f, const void* d_g,
                                         const void* d_u, void* stream, double* rel_res) {
    using namespace hh;
    if ((dim != 1 && dim != 2) || n < 1 || !std::isfinite(k) || k < 0.0) return HH_EINVAL;
    if ((long long)n + 2 > (long long)kNaMaxRows) return HH_ETOOLARGE;
    if (!d_f || !d_g || !d_u || !rel_res) return HH_EINVAL;
    void* base = nullptr;
    const hh_status st = na_scratch(&base);
    if (st != HH_OK) return st;
    unsigned char* b = (unsigned char*)base;
    double2* rows = (double2*)b;
    double2* total = (double2*)(b + kNaRowBytes);
    unsigned* ticket = (unsigned*)(b + kNaRowBytes + sizeof(double2));
    const cudaStream_t s = (cudaStream_t)stream;
    const int S = n + 2;
    const double h = 1.0 / (n + 1);
    // the ticket must start at zero; the row pairs and the total are overwritten
    if (cudaMemsetAsync(ticket, 0, sizeof(unsigned), s) != cudaSuccess) return HH_ECUDA;
    int grid = (S + 7) / 8;
    if (grid > 152 * 8) grid = 152 * 8;
    k_residual_rows<<<grid, 256, 0, s>>>((const c128*)d_f, (const c128*)d_g, (const c128*)d_u, dim, S, h, k * h,
                                         rows, total, ticket);
    note_launch();
    if (cudaGetLastError() != cudaSuccess) return HH_ECUDA;
    double out[2] = {0.0, 0.0};
    if (cudaMemcpyAsync(out, total, sizeof(out), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return HH_ECUDA;
    *rel_res = out[1] > 0 ? std::sqrt(out[0] / out[1]) : 0.0;
    return HH_OK;
}
