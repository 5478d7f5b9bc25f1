// rlb_stream.cu -- the FP32 deviation step with TMA-staged pull streaming.
//
// Persistent CTAs walk the lattice in tiles of R consecutive x-rows of one z
// plane.  For plane q (velocity i of f or g) the populations that arrive at a
// tile come from the rows y - e_iy of plane z - e_iz, shifted by -e_ix along
// x: one contiguous block of R rows in global memory (two when the window
// wraps in y).  One thread copies those blocks into shared memory with 1-D
// bulk asynchronous copies (cp.async.bulk, the TMA unit) completing on an
// mbarrier; a ring of K stages keeps K-1 tiles in flight while the CTA
// collides the current one from shared memory (reads shifted by -e_ix, bank
// conflict free).  Every population is still read from HBM exactly once and
// written once; what changes is that the loads are issued a tile ahead by
// the copy engine instead of one cell at a time by the threads.
//
// Conditions: nx * 4 bytes a multiple of 16 (nx % 4 == 0) and K stages of
// 38 * R * nx floats fitting in shared memory; otherwise the caller falls
// back to the one-cell-per-thread kernel.  Waits are bounded (rlb_tma.cuh):
// a CTA that gives up sets Counters::pipe_err, waits (bounded) for its own
// copies still in flight, and returns.
#include <cuda.h>  // CUcontext type only; cuCtxGetCurrent is taken through the runtime
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>

#include <mutex>

#include "rlb_collide.cuh"
#include "rlb_device.cuh"
#include "rlb_tma.cuh"

namespace rlb {

struct TmaCfg {
    int stages;  // K
    int rows;    // R
    int tiles_per_z;
    int ntiles;
};

template <int XBC, bool SOLID, int MINB>
__global__ void __launch_bounds__(256, MINB)
    k_step_f32_tma(const float* __restrict__ A, float* __restrict__ B, Geom g, Dev32 c, Counters cnt, int count,
                   long long step_index, TmaCfg tc) {
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
    float* stages = reinterpret_cast<float*>(smem + 128);
    const int K = tc.stages, R = tc.rows, nx = g.nx, ny = g.ny, nz = g.nz;
    const int plane_elems = R * nx;
    const int stage_elems = 38 * plane_elems;
    const long long S = g.S;

    if (threadIdx.x == 0) {
        for (int s = 0; s < K; ++s) mbar_init(&bars[s], 1);
        fence_mbar_init();
    }
    __syncthreads();

    // Producer (warp 0, all lanes): bulk copies of the source rows of every
    // plane of tile 'tile' into stage 's'.  Lane i (< 19) copies velocity i of
    // both f and g (same source rows); wraps use compares, not divisions.
    auto issue = [&](int tile, int s) {
        const int z = tile / tc.tiles_per_z;
        const int y0 = (tile - z * tc.tiles_per_z) * R;
        const int rr = min(R, ny - y0);
        float* st = stages + (size_t)s * stage_elems;
        if (threadIdx.x == 0) mbar_arrive_expect_tx(&bars[s], (unsigned)(38 * rr * nx * 4));
        __syncwarp();
        const int i = threadIdx.x;
        if (i < 19) {
            int zs = z - vel_z(i);
            zs = zs < 0 ? zs + nz : (zs >= nz ? zs - nz : zs);
            int ys = y0 - vel_y(i);
            ys = ys < 0 ? ys + ny : (ys >= ny ? ys - ny : ys);
            const int seg = min(rr, ny - ys);
            const long long row0 = ((long long)zs * ny + ys) * nx;
            const long long wrap0 = (long long)zs * ny * nx;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int q = i + 19 * h;
                bulk_g2s(st + q * plane_elems, RLB_CHK_PTR(A, q * S + row0, 38ll * S), (unsigned)(seg * nx * 4), &bars[s]);
                if (seg < rr)
                    bulk_g2s(st + q * plane_elems + seg * nx, RLB_CHK_PTR(A, q * S + wrap0, 38ll * S), (unsigned)((rr - seg) * nx * 4),
                             &bars[s]);
            }
        }
    };

    // pend[s]: phase parity pending on stage s, or -1 (warp 0 bookkeeping)
    int pend[4] = {-1, -1, -1, -1};
    if (threadIdx.x < 32) {
        for (int s = 0; s < K; ++s) {
            const int tile = blockIdx.x + s * gridDim.x;
            if (tile < tc.ntiles) {
                issue(tile, s);
                pend[s] = 0;
            }
        }
    }
    bool ok = true;
    int k = 0;
    for (int tile = blockIdx.x; tile < tc.ntiles; tile += gridDim.x, ++k) {
        const int s = k % K;
        const unsigned parity = (unsigned)((k / K) & 1);
        const bool got = mbar_wait(&bars[s], parity);
        ok = __syncthreads_and(got) != 0;
        if (!ok) break;
        pend[s] = -1;
        const float* st = stages + (size_t)s * stage_elems;
        const int z = tile / tc.tiles_per_z;
        const int y0 = (tile - z * tc.tiles_per_z) * R;
        const int rr = min(R, ny - y0);
        for (int cidx = threadIdx.x; cidx < rr * nx; cidx += blockDim.x) {
            const int r = cidx / nx;
            const int x = cidx - r * nx;
            const int idx = (z * ny + y0 + r) * nx + x;
            if (XBC != XBC_PERIODIC && (x == 0 || x == nx - 1)) {
                if (XBC == XBC_INFLOW_OUTFLOW && x == 0) {
#pragma unroll
                    for (int q = 0; q < 38; ++q) B[RLB_CHK(q * S + idx, 38ll * S)] = __ldg(RLB_CHK_PTR(A, q * S + idx, 38ll * S));
                }
                continue;
            }
            if (SOLID && is_solid(st[19 * plane_elems + r * nx + x])) {
                const float m = solid_marker_f();
#pragma unroll
                for (int q = 0; q < 38; ++q) B[RLB_CHK(q * S + idx, 38ll * S)] = m;
                continue;
            }
            const int xm = (x == 0) ? nx - 1 : x - 1;
            const int xp = (x == nx - 1) ? 0 : x + 1;
            const float* row = st + r * nx;
            auto fetch = [&](int q, int i) {
                const int ex = vel_x(i);
                return row[q * plane_elems + (ex > 0 ? xm : (ex < 0 ? xp : x))];
            };
            auto bounce = [&](int q, int i) { return __ldg(RLB_CHK_PTR(A, (q - i + opp(i)) * S + idx, 38ll * S)); };  // link bounce-back
            const int dup = (XBC != XBC_PERIODIC && x == nx - 2) ? 1 : ((XBC == XBC_OUTFLOW_BOTH && x == 1) ? -1 : 0);
            float* Bc = B + idx;
            auto put = [&](int q, float v) {
                Bc[RLB_CHK_OFF(q * S, idx, 38ll * S)] = v;
                if (dup) Bc[RLB_CHK_OFF(q * S + dup, idx, 38ll * S)] = v;
            };
            bool unphys, nonpos;
            collide_cell_f32<SOLID>(fetch, bounce, put, c, unphys, nonpos);
            if (count) count_flags(cnt, unphys, nonpos, (unsigned long long)step_index * (unsigned long long)g.N + idx);
        }
        __syncthreads();  // every thread is done reading stage s
        if (threadIdx.x < 32) {
            const int next = tile + K * gridDim.x;
            if (next < tc.ntiles) {
                fence_proxy_async_smem();
                issue(next, s);
                pend[s] = (int)(((k + K) / K) & 1);
            }
        }
    }
    if (!ok && threadIdx.x == 0) {
        atomicAdd(cnt.pipe_err, 1ull);
        // let this CTA's copies still in flight land before its shared memory goes away
        for (int s = 0; s < K; ++s)
            if (pend[s] >= 0) mbar_wait(&bars[s], (unsigned)pend[s]);
    }
}

namespace {
int env_int(const char* name, int dflt) {
    const char* v = getenv(name);
    return (v && *v) ? atoi(v) : dflt;
}

// The calling thread's current context, through the driver entry point the
// runtime hands out (no link against the driver library).
CUcontext current_context() {
    using Fn = CUresult (*)(CUcontext*);
    static Fn fn = nullptr;
    static bool looked = false;
    if (!looked) {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 4000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<Fn>(f);
        looked = true;
    }
    CUcontext c = nullptr;
    if (fn) fn(&c);
    return c;
}

// The dynamic shared memory opt-in of a kernel, per context and kernel (the
// attribute belongs to the kernel in a context), raised when a launch needs
// more than was set.
std::mutex g_optin_mu;
struct OptIn {
    CUcontext ctx;
    const void* kern;
    size_t bytes;
};
OptIn g_optin[32];
int g_optin_n = 0;

void smem_opt_in(const void* kern, size_t bytes) {
    const CUcontext ctx = current_context();
    std::lock_guard<std::mutex> lock(g_optin_mu);
    int k = 0;
    while (k < g_optin_n && !(g_optin[k].ctx == ctx && g_optin[k].kern == kern)) ++k;
    if (k < g_optin_n && g_optin[k].bytes >= bytes) return;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess) return;
    if (k < g_optin_n)
        g_optin[k].bytes = bytes;
    else if (g_optin_n < 32)
        g_optin[g_optin_n++] = {ctx, kern, bytes};
}
}  // namespace

cudaError_t launch_step_f32_tma(const Geom& g, const Dev32& c, const float* A, float* B, Counters cnt, bool count,
                                long long step_index, cudaStream_t st) {
    if ((g.nx * 4) % 16 != 0) return cudaErrorNotSupported;
    static int dev_smem = -1, nsm = 0;
    if (dev_smem < 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&dev_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    }
    const size_t row_bytes = (size_t)38 * g.nx * 4;
    const size_t budget = (size_t)env_int("RLB_TMA_SMEM_KB", 200) * 1024;
    int K = env_int("RLB_TMA_STAGES", 3);
    if (K < 2) K = 2;
    if (K > 4) K = 4;
    int R = env_int("RLB_TMA_ROWS", 0);
    if (R <= 0) R = (int)(budget / (K * row_bytes));
    if (R < 1 && K > 2) {
        K = 2;
        R = (int)(budget / (K * row_bytes));
    }
    if (R < 1) return cudaErrorNotSupported;
    if (R > g.ny) R = g.ny;
    const size_t smem = 128 + (size_t)K * R * row_bytes;
    if ((int)smem > dev_smem) return cudaErrorNotSupported;
    TmaCfg tc;
    tc.stages = K;
    tc.rows = R;
    tc.tiles_per_z = (g.ny + R - 1) / R;
    tc.ntiles = g.nz * tc.tiles_per_z;
    int threads = ((R * g.nx + 31) / 32) * 32;
    if (threads > 256) threads = 256;
    const int minb = env_int("RLB_TMA_MINB", 2) >= 3 ? 3 : 2;
    const int ctas_per_sm = env_int("RLB_TMA_CTAS", 1);
    int grid = nsm * ctas_per_sm;
    if (grid > tc.ntiles) grid = tc.ntiles;
    auto run = [&](auto kern, int) {
        smem_opt_in((const void*)kern, smem);  // a failure shows at the launch
        kern<<<grid, threads, smem, st>>>(A, B, g, c, cnt, count ? 1 : 0, step_index, tc);
    };
    if (minb == 3) {
        switch (g.xbc) {
            case XBC_PERIODIC: run(k_step_f32_tma<XBC_PERIODIC, true, 3>, 3); break;
            case XBC_INFLOW_OUTFLOW: run(k_step_f32_tma<XBC_INFLOW_OUTFLOW, true, 3>, 4); break;
            default: run(k_step_f32_tma<XBC_OUTFLOW_BOTH, true, 3>, 5); break;
        }
    } else {
        switch (g.xbc) {
            case XBC_PERIODIC: run(k_step_f32_tma<XBC_PERIODIC, true, 2>, 0); break;
            case XBC_INFLOW_OUTFLOW: run(k_step_f32_tma<XBC_INFLOW_OUTFLOW, true, 2>, 1); break;
            default: run(k_step_f32_tma<XBC_OUTFLOW_BOTH, true, 2>, 2); break;
        }
    }
    return cudaGetLastError();
}

// Bounds-check count of this translation unit (0 in the release build).
RLB_OOB_TAKE_FN(oob_take_stream)

}  // namespace rlb
