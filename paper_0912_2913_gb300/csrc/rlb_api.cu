// rlb_api.cu -- the C ABI of librlb (include/rlb.h): parameter checks,
// workspace layout, host<->device marshalling and kernel launches on the
// context's stream.  No arithmetic of the scheme lives here; every step of
// the method runs in the kernels of rlb_forward.cu and rlb_adjoint.cu.
#include <nvtx3/nvToolsExt.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <new>

#include "../../include/rlb.h"
#include "rlb_internal.h"

using namespace rlb;

struct rlb_ctx {
    rlb_params p;
    Geom g;
    Phys ph;
    cudaStream_t stream;
    int device;
    void* ws;
    size_t ws_bytes;
    bool own_ws;
    void* A;  // current state
    void* B;  // the other buffer
    Counters cnt;
    double* red;  // adjoint partial sums
    double* inflow_d;  // d eq_in / d beta_in, 38 x 3 doubles, then the same as floats
    size_t state_bytes;
    int elem;
    int64_t steps;
    bool inited;
    int64_t launches;
    cudaError_t err;
    char msg[320];
};

namespace {

// NVTX range around an entry point (visible in profilers; no cost without one).
struct Nvtx {
    explicit Nvtx(const char* name) { nvtxRangePushA(name); }
    ~Nvtx() { nvtxRangePop(); }
};

// Allocation-failure injection for tests of the error path (host side only):
// with RLB_INJECT_ALLOC_FAILURE=1 in the environment, rlb_create reports
// RLB_ERR_OOM instead of allocating its workspace.
bool inject_alloc_failure() {
    const char* v = getenv("RLB_INJECT_ALLOC_FAILURE");
    return v && v[0] == '1';
}

thread_local char g_msg[320] = "";

rlb_status fail(rlb_ctx* c, rlb_status s, const char* fmt, ...) {
    char buf[320];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    snprintf(g_msg, sizeof g_msg, "%s", buf);
    if (c) snprintf(c->msg, sizeof c->msg, "%s", buf);
    return s;
}

rlb_status cuda_fail(rlb_ctx* c, cudaError_t e, const char* where) {
    if (c && c->err == cudaSuccess) c->err = e;
    return fail(c, RLB_ERR_CUDA, "%s: %s (%s)", where, cudaGetErrorString(e), cudaGetErrorName(e));
}

#define RLB_LATCHED(c)                                                                          \
    do {                                                                                        \
        if (!(c)) return fail(nullptr, RLB_ERR_ARG, "null context");                            \
        if ((c)->err != cudaSuccess) return fail((c), RLB_ERR_CUDA, "latched CUDA error: %s",   \
                                                 cudaGetErrorString((c)->err));                 \
    } while (0)

#define RLB_CUDA(c, expr, where)                          \
    do {                                                  \
        cudaError_t e_ = (expr);                          \
        if (e_ != cudaSuccess) return cuda_fail((c), e_, (where)); \
    } while (0)

constexpr size_t kAlign = 256;
size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

rlb_status check_params(const rlb_params* p) {
    if (!p) return fail(nullptr, RLB_ERR_ARG, "params is NULL");
    if (p->nx < 1 || p->ny < 1 || p->nz < 1) return fail(nullptr, RLB_ERR_ARG, "lattice sizes must be >= 1");
    const long long N = (long long)p->nx * p->ny * p->nz;
    // Cell indices are 32-bit in the kernels; the limit leaves 2^21 of room
    // above the last cell for the thread indices of the last block and of a
    // grid-stride step.
    if (N > (1ll << 31) - (1ll << 21))
        return fail(nullptr, RLB_ERR_ARG, "lattice too large (N must be <= 2^31 - 2^21)");
    if (p->prec != RLB_FP64 && p->prec != RLB_FP32_DEV) return fail(nullptr, RLB_ERR_ARG, "bad precision %d", p->prec);
    if (p->xbc < RLB_BC_PERIODIC || p->xbc > RLB_BC_OUTFLOW_BOTH) return fail(nullptr, RLB_ERR_ARG, "bad xbc %d", p->xbc);
    if (p->xbc != RLB_BC_PERIODIC && p->nx < 3) return fail(nullptr, RLB_ERR_ARG, "ghost planes need nx >= 3");
    if (p->eos != RLB_EOS_ULTRA && p->eos != RLB_EOS_GAMMA_LAW) return fail(nullptr, RLB_ERR_ARG, "bad eos %d", p->eos);
    if (p->eos == RLB_EOS_GAMMA_LAW) {
        if (p->prec != RLB_FP64) return fail(nullptr, RLB_ERR_ARG, "the general equation of state runs in FP64");
        if (!(p->eos_gamma > 1.0 && p->eos_gamma <= 2.0)) return fail(nullptr, RLB_ERR_ARG, "eos_gamma must be in (1, 2]");
        if (!(p->eos_mass >= 0.0) || !isfinite(p->eos_mass)) return fail(nullptr, RLB_ERR_ARG, "eos_mass must be >= 0");
    }
    if (!(p->tau > 0.5) || !isfinite(p->tau)) return fail(nullptr, RLB_ERR_ARG, "tau must be > 1/2");
    if (!(p->c_l > 0.0) || !isfinite(p->c_l)) return fail(nullptr, RLB_ERR_ARG, "c_l must be > 0");
    if (p->xbc == RLB_BC_INFLOW_OUTFLOW) {
        const double b2 = p->beta_in[0] * p->beta_in[0] + p->beta_in[1] * p->beta_in[1] + p->beta_in[2] * p->beta_in[2];
        if (!(p->n_in > 0) || !(p->eps_in > 0) || !(b2 < 1.0)) return fail(nullptr, RLB_ERR_ARG, "bad inflow state");
    }
    if (p->prec == RLB_FP32_DEV && (!(p->n_ref > 0) || !(p->eps_ref > 0)))
        return fail(nullptr, RLB_ERR_ARG, "FP32 deviation storage needs n_ref > 0 and eps_ref > 0");
    if (p->zbc != RLB_ZBC_PERIODIC && p->zbc != RLB_ZBC_HALO) return fail(nullptr, RLB_ERR_ARG, "bad zbc %d", p->zbc);
    if (p->reserved != 0) return fail(nullptr, RLB_ERR_ARG, "rlb_params.reserved must be 0");
    if (p->zbc == RLB_ZBC_HALO) {
        if (p->nz < 3) return fail(nullptr, RLB_ERR_ARG, "a z slab with halo planes needs nz >= 3");
        if (p->eos != RLB_EOS_ULTRA) return fail(nullptr, RLB_ERR_ARG, "z slabs cover the eps = 3P equation of state");
    }
    return RLB_OK;
}

void layout(const rlb_params* p, long long* S, int* elem, size_t* state_bytes) {
    const long long N = (long long)p->nx * p->ny * p->nz;
    *S = (N + 63) / 64 * 64;
    *elem = p->prec == RLB_FP64 ? 8 : 4;
    *state_bytes = (size_t)38 * (size_t)(*S) * (size_t)(*elem);
}

size_t counters_bytes() {
    return align_up(sizeof(unsigned long long) * (2 * kCounterSlots + 3), kAlign) + align_up((sizeof(double) + sizeof(float)) * kInflowTable, kAlign);
}
size_t red_bytes(const rlb_params* p) {
    return align_up(sizeof(double) * adj_red_doubles((long long)p->nx * p->ny * p->nz), kAlign);
}

size_t workspace_size(const rlb_params* p) {
    long long S;
    int elem;
    size_t sb;
    layout(p, &S, &elem, &sb);
    return 2 * align_up(sb, kAlign) + counters_bytes() + red_bytes(p);
}

rlb_status reset_counters(rlb_ctx* c) {
    RLB_CUDA(c, cudaMemsetAsync(c->cnt.slots, 0, sizeof(unsigned long long) * 2 * kCounterSlots, c->stream),
             "reset counters");
    RLB_CUDA(c, cudaMemsetAsync(c->cnt.first_bad, 0xff, sizeof(unsigned long long), c->stream), "reset counters");
    RLB_CUDA(c, cudaMemsetAsync(c->cnt.macro_bad, 0, 2 * sizeof(unsigned long long), c->stream), "reset counters");
    return RLB_OK;
}

rlb_status after_launch(rlb_ctx* c, cudaError_t e, const char* where) {
    c->launches += last_launch_count();
    if (e != cudaSuccess) return cuda_fail(c, e, where);
    return RLB_OK;
}

}  // namespace

extern "C" {

rlb_status rlb_state_layout(const rlb_params* p, int64_t* plane_stride, int32_t* elem_bytes, size_t* bytes) {
    rlb_status s = check_params(p);
    if (s != RLB_OK) return s;
    long long S;
    int elem;
    size_t sb;
    layout(p, &S, &elem, &sb);
    if (plane_stride) *plane_stride = S;
    if (elem_bytes) *elem_bytes = elem;
    if (bytes) *bytes = sb;
    return RLB_OK;
}

rlb_status rlb_workspace_bytes(const rlb_params* p, size_t* bytes) {
    rlb_status s = check_params(p);
    if (s != RLB_OK) return s;
    if (!bytes) return fail(nullptr, RLB_ERR_ARG, "bytes is NULL");
    *bytes = workspace_size(p);
    return RLB_OK;
}

rlb_status rlb_create(const rlb_params* p, void* stream, void* workspace, size_t workspace_bytes, rlb_ctx** out) {
    rlb_status s = check_params(p);
    if (s != RLB_OK) return s;
    if (!out) return fail(nullptr, RLB_ERR_ARG, "out is NULL");
    *out = nullptr;
    const size_t need = workspace_size(p);
    if (workspace && workspace_bytes < need)
        return fail(nullptr, RLB_ERR_ARG, "workspace too small: %zu < %zu bytes", workspace_bytes, need);
    if (workspace && ((uintptr_t)workspace % kAlign) != 0)
        return fail(nullptr, RLB_ERR_ARG, "workspace must be %zu-byte aligned", kAlign);
    if (!workspace && inject_alloc_failure())
        return fail(nullptr, RLB_ERR_OOM, "injected allocation failure (RLB_INJECT_ALLOC_FAILURE)");
    rlb_ctx* c = new (std::nothrow) rlb_ctx();
    if (!c) return fail(nullptr, RLB_ERR_OOM, "host allocation of the context failed");
    c->p = *p;
    c->stream = (cudaStream_t)stream;
    c->err = cudaSuccess;
    cudaError_t e = cudaGetDevice(&c->device);
    if (e != cudaSuccess) {
        delete c;
        return cuda_fail(nullptr, e, "cudaGetDevice");
    }
    long long S;
    layout(p, &S, &c->elem, &c->state_bytes);
    Geom& g = c->g;
    g.nx = p->nx;
    g.ny = p->ny;
    g.nz = p->nz;
    g.nxy = p->nx * p->ny;
    g.N = p->nx * p->ny * p->nz;
    g.S = S;
    g.xbc = p->xbc;
    g.div_nx = make_fast_div((unsigned)g.nx);
    g.div_ny = make_fast_div((unsigned)g.ny);
    g.zhalo = p->zbc == RLB_ZBC_HALO ? 1 : 0;
    {
        // Tuning knobs (no effect on results beyond rounding): RLB_TMA=1
        // selects the TMA-staged FP32 step, RLB_F32_VARIANT the launch variant
        // of the plain one, RLB_ADJ_PIPE the FP32 adjoint kernel (0: one cell
        // per thread, 1: persistent, 2: persistent shared-memory staged;
        // RLB_ADJ_COOP=0 stages lambda per thread instead of per block).
        const char* t = getenv("RLB_TMA");
        g.tma = (t && t[0] == '1' && !g.zhalo) ? 1 : 0;  // the TMA-staged step updates every z plane
        const char* v = getenv("RLB_F32_VARIANT");
        g.variant = v ? atoi(v) : -1;  // -1: chosen by timing at the first step
        const char* ap = getenv("RLB_ADJ_PIPE");
        g.adj_pipe = ap ? atoi(ap) : 2;
        const char* ac = getenv("RLB_ADJ_COOP");
        g.adj_coop = (ac && ac[0] == '0') ? 0 : 1;
        const char* pb = getenv("RLB_PIPE_BLOCKS");
        g.pipe_blocks = pb ? atoi(pb) : 3;
        // RLB_F64_ARITH=df: the FP64 step with its arithmetic in compensated
        // binary32 pairs (binary64 storage and recovery root; an ablation of
        // the all-FP64 step, which stays the default)
        const char* fa = getenv("RLB_F64_ARITH");
        g.f64df = (fa && fa[0] == 'd' && fa[1] == 'f') ? 1 : 0;
        const char* fs = getenv("RLB_F64_SPLIT");
        g.f64split = fs ? (fs[0] == '1' ? 1 : 0) : -1;
    }
    Phys& ph = c->ph;
    ph.tau = p->tau;
    ph.omega = 1.0 / p->tau;
    ph.c_l = p->c_l;
    ph.inv_cl = 1.0 / p->c_l;
    ph.inv_cl2 = 1.0 / (p->c_l * p->c_l);
    ph.n_in = p->n_in;
    ph.eps_in = p->eps_in;
    for (int a = 0; a < 3; ++a) ph.beta_in[a] = p->beta_in[a];
    ph.n_ref = p->n_ref;
    ph.eps_ref = p->eps_ref;
    for (int cl = 0; cl < 2; ++cl) {
        const double w = cl == 0 ? 1.0 / 18.0 : 1.0 / 36.0;
        ph.c_k1[cl] = ph.omega * w * ph.inv_cl2;
        ph.c_k2[cl] = 6.0 * ph.omega * w * ph.inv_cl2;
        ph.c_k3[cl] = 4.0 * ph.omega * w * ph.inv_cl;
        ph.c_fs[cl] = ph.omega * w;
        ph.c_fa[cl] = 3.0 * ph.omega * w * ph.inv_cl;
    }
    ph.c_f0 = ph.omega / 3.0;
    ph.c_g0[0] = 4.0 * ph.omega / 3.0;
    ph.c_g0[1] = -(ph.omega / 3.0) * (2.0 * ph.inv_cl2 + 1.0);
    ph.c_g0[2] = -2.0 * (ph.omega / 3.0) * ph.inv_cl2;
    ph.m3cl2 = -3.0 * p->c_l * p->c_l;
    ph.three_cl = 3.0 * p->c_l;
    ph.eos = p->eos;
    ph.eos_gamma = p->eos == RLB_EOS_GAMMA_LAW ? p->eos_gamma : 4.0 / 3.0;
    ph.eos_mass = p->eos == RLB_EOS_GAMMA_LAW ? p->eos_mass : 0.0;
    if (workspace) {
        c->ws = workspace;
        c->own_ws = false;
    } else {
        e = cudaMallocAsync(&c->ws, need, c->stream);
        if (e != cudaSuccess) {
            cudaGetLastError();
            delete c;
            return fail(nullptr, e == cudaErrorMemoryAllocation ? RLB_ERR_OOM : RLB_ERR_CUDA,
                        "cudaMallocAsync of %zu bytes: %s", need, cudaGetErrorString(e));
        }
        c->own_ws = true;
    }
    c->ws_bytes = need;
    char* base = (char*)c->ws;
    const size_t sb = align_up(c->state_bytes, kAlign);
    c->A = base;
    c->B = base + sb;
    c->cnt.slots = (unsigned long long*)(base + 2 * sb);
    c->cnt.first_bad = c->cnt.slots + 2 * kCounterSlots;
    c->cnt.macro_bad = c->cnt.first_bad + 1;
    c->cnt.pipe_err = c->cnt.first_bad + 2;
    c->inflow_d = (double*)(base + 2 * sb + align_up(sizeof(unsigned long long) * (2 * kCounterSlots + 3), kAlign));
    c->red = (double*)(base + 2 * sb + counters_bytes());
    s = reset_counters(c);
    if (s == RLB_OK) s = after_launch(c, launch_inflow_derivs(c->ph, c->inflow_d, c->stream), "inflow table");
    if (s != RLB_OK) {
        rlb_destroy(c);
        return s;
    }
    *out = c;
    return RLB_OK;
}

rlb_status rlb_destroy(rlb_ctx* c) {
    if (!c) return RLB_OK;
    rlb_status s = RLB_OK;
    if (c->own_ws && c->ws) {
        cudaError_t e = cudaFreeAsync(c->ws, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) s = cuda_fail(nullptr, e, "cudaFreeAsync");
    }
    delete c;
    return s;
}

rlb_status rlb_init_fields(rlb_ctx* c, const double* n, const double* eps, const double* beta, const uint8_t* solid,
                           rlb_where where) {
    Nvtx nvtx_("rlb_init_fields");
    RLB_LATCHED(c);
    if (!n || !eps || !beta) return fail(c, RLB_ERR_ARG, "n, eps and beta are required");
    if (where != RLB_HOST && where != RLB_DEVICE) return fail(c, RLB_ERR_ARG, "bad 'where'");
    const Geom& g = c->g;
    const size_t N = (size_t)g.N;
    const double *dn = n, *de = eps, *db = beta;
    const uint8_t* ds = solid;
    void* tmp = nullptr;
    if (where == RLB_HOST) {
        if (solid && g.xbc != RLB_BC_PERIODIC) {
            for (int z = 0; z < g.nz; ++z)
                for (int y = 0; y < g.ny; ++y) {
                    const size_t row = ((size_t)z * g.ny + y) * g.nx;
                    if (solid[row] || solid[row + 1] || solid[row + g.nx - 2] || solid[row + g.nx - 1])
                        return fail(c, RLB_ERR_ARG, "solid cells on a ghost plane or its neighbour (x = 0, 1, nx-2, nx-1)");
                }
        }
        const size_t bytes = N * 5 * sizeof(double) + (solid ? N : 0);
        RLB_CUDA(c, cudaMallocAsync(&tmp, bytes, c->stream), "cudaMallocAsync (init staging)");
        char* t = (char*)tmp;
        RLB_CUDA(c, cudaMemcpyAsync(t, n, N * sizeof(double), cudaMemcpyHostToDevice, c->stream), "copy n");
        RLB_CUDA(c, cudaMemcpyAsync(t + N * 8, eps, N * sizeof(double), cudaMemcpyHostToDevice, c->stream), "copy eps");
        RLB_CUDA(c, cudaMemcpyAsync(t + N * 16, beta, 3 * N * sizeof(double), cudaMemcpyHostToDevice, c->stream),
                 "copy beta");
        if (solid)
            RLB_CUDA(c, cudaMemcpyAsync(t + N * 40, solid, N, cudaMemcpyHostToDevice, c->stream), "copy solid");
        dn = (const double*)t;
        de = (const double*)(t + N * 8);
        db = (const double*)(t + N * 16);
        ds = solid ? (const uint8_t*)(t + N * 40) : nullptr;
    } else if (solid && g.xbc != RLB_BC_PERIODIC) {
        RLB_CUDA(c, cudaMemsetAsync(c->cnt.macro_bad, 0, sizeof(unsigned long long), c->stream), "memset");
        rlb_status s = after_launch(c, launch_check_solid_planes(g, solid, c->cnt.macro_bad, c->stream), "check solid");
        if (s != RLB_OK) return s;
        unsigned long long bad = 0;
        RLB_CUDA(c, cudaMemcpyAsync(&bad, c->cnt.macro_bad, sizeof bad, cudaMemcpyDeviceToHost, c->stream), "copy flag");
        RLB_CUDA(c, cudaStreamSynchronize(c->stream), "sync");
        if (bad) return fail(c, RLB_ERR_ARG, "solid cells on a ghost plane or its neighbour (x = 0, 1, nx-2, nx-1)");
    }
    rlb_status s = after_launch(c,
                                c->ph.eos ? launch_init_eos(g, c->ph, dn, de, db, ds, c->A, c->B, c->stream)
                                          : launch_init(c->p.prec, g, c->ph, dn, de, db, ds, c->A, c->B, c->stream),
                                "init");
    if (s != RLB_OK) return s;
    if (tmp) {
        RLB_CUDA(c, cudaFreeAsync(tmp, c->stream), "cudaFreeAsync (init staging)");
        RLB_CUDA(c, cudaStreamSynchronize(c->stream), "sync");
    }
    s = reset_counters(c);
    if (s != RLB_OK) return s;
    c->steps = 0;
    c->inited = true;
    return RLB_OK;
}

// Launch variants of the FP32 step compute bit-identical results; which one
// is fastest depends on the lattice.  The candidates: 2 (256-thread blocks,
// 64 registers), 7 and 8 (the f populations loaded before the g arithmetic,
// 128 x 7 blocks at 72 registers, 64 x 12 at 80; measured fastest on the
// 512^3 box and the 200x100x100 sphere).  The first FP32 rlb_step times
// each on the context's second buffer (which the step then overwrites) and
// keeps the fastest.  This first call synchronises the stream once.
static rlb_status autotune_f32(rlb_ctx* c) {
    const int cand[3] = {2, 7, 8};
    float best = 1e30f;
    int pick = 2;
    cudaEvent_t e0, e1;
    RLB_CUDA(c, cudaEventCreate(&e0), "event");
    RLB_CUDA(c, cudaEventCreate(&e1), "event");
    for (int k = 0; k < 3; ++k) {
        c->g.variant = cand[k];
        cudaError_t e = launch_step(c->p.prec, c->g, c->ph, c->A, c->B, c->cnt, false, 0, c->stream);
        if (e == cudaSuccess) e = cudaEventRecord(e0, c->stream);
        for (int r = 0; r < 3 && e == cudaSuccess; ++r)
            e = launch_step(c->p.prec, c->g, c->ph, c->A, c->B, c->cnt, false, 0, c->stream);
        if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return cuda_fail(c, e, "autotune");
        }
        c->launches += 4;
        if (ms < best) {
            best = ms;
            pick = cand[k];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->g.variant = pick;
    return RLB_OK;
}

rlb_status rlb_step(rlb_ctx* c, int32_t nsteps) {
    Nvtx nvtx_("rlb_step");
    RLB_LATCHED(c);
    if (nsteps < 0) return fail(c, RLB_ERR_ARG, "nsteps must be >= 0");
    if (!c->inited) return fail(c, RLB_ERR_STATE, "rlb_step before rlb_init_fields");
    if (c->g.variant < 0 && nsteps > 0) {
        if (c->p.prec == RLB_FP32_DEV && !c->g.tma) {
            rlb_status s = autotune_f32(c);
            if (s != RLB_OK) return s;
        } else {
            c->g.variant = 7;
        }
    }
    for (int32_t t = 0; t < nsteps; ++t) {
        rlb_status s = after_launch(c,
                                    c->ph.eos ? launch_step_eos(c->g, c->ph, c->A, c->B, c->cnt, true, c->steps, c->stream)
                                              : launch_step(c->p.prec, c->g, c->ph, c->A, c->B, c->cnt, true, c->steps,
                                                            c->stream),
                                    "step");
        if (s != RLB_OK) return s;
        void* tmp = c->A;
        c->A = c->B;
        c->B = tmp;
        c->steps += 1;
    }
    return RLB_OK;
}

rlb_status rlb_step_into(rlb_ctx* c, const void* src, void* dst) {
    Nvtx nvtx_("rlb_step_into");
    RLB_LATCHED(c);
    if (!src || !dst || src == dst) return fail(c, RLB_ERR_ARG, "src and dst must be distinct device buffers");
    if (c->g.variant < 0) c->g.variant = 7;  // untuned: the shape measured fastest on the benchmark lattices
    return after_launch(c,
                        c->ph.eos ? launch_step_eos(c->g, c->ph, src, dst, c->cnt, false, 0, c->stream)
                                  : launch_step(c->p.prec, c->g, c->ph, src, dst, c->cnt, false, 0, c->stream),
                        "step_into");
}

rlb_status rlb_step_into_counted(rlb_ctx* c, const void* src, void* dst) {
    Nvtx nvtx_("rlb_step_into_counted");
    RLB_LATCHED(c);
    if (!src || !dst || src == dst) return fail(c, RLB_ERR_ARG, "src and dst must be distinct device buffers");
    if (!c->inited) return fail(c, RLB_ERR_STATE, "rlb_step_into_counted before rlb_init_fields");
    if (c->g.variant < 0) c->g.variant = 7;  // untuned: the shape measured fastest on the benchmark lattices
    rlb_status s = after_launch(c,
                                c->ph.eos ? launch_step_eos(c->g, c->ph, src, dst, c->cnt, true, c->steps, c->stream)
                                          : launch_step(c->p.prec, c->g, c->ph, src, dst, c->cnt, true, c->steps,
                                                        c->stream),
                                "step_into_counted");
    if (s == RLB_OK) c->steps += 1;
    return s;
}

rlb_status rlb_state_ptr(rlb_ctx* c, void** state) {
    RLB_LATCHED(c);
    if (!state) return fail(c, RLB_ERR_ARG, "state is NULL");
    *state = c->A;
    return RLB_OK;
}

rlb_status rlb_save_state(rlb_ctx* c, void* dst) {
    RLB_LATCHED(c);
    if (!dst) return fail(c, RLB_ERR_ARG, "dst is NULL");
    RLB_CUDA(c, cudaMemcpyAsync(dst, c->A, c->state_bytes, cudaMemcpyDeviceToDevice, c->stream), "save_state");
    return RLB_OK;
}

rlb_status rlb_load_state(rlb_ctx* c, const void* src) {
    RLB_LATCHED(c);
    if (!src) return fail(c, RLB_ERR_ARG, "src is NULL");
    RLB_CUDA(c, cudaMemcpyAsync(c->A, src, c->state_bytes, cudaMemcpyDeviceToDevice, c->stream), "load_state");
    c->inited = true;
    return RLB_OK;
}

rlb_status rlb_macro(rlb_ctx* c, const void* state, double* n, double* eps, double* beta, rlb_where where) {
    Nvtx nvtx_("rlb_macro");
    RLB_LATCHED(c);
    if (!n || !eps || !beta) return fail(c, RLB_ERR_ARG, "outputs are required");
    if (where != RLB_HOST && where != RLB_DEVICE) return fail(c, RLB_ERR_ARG, "bad 'where'");
    if (!state && !c->inited) return fail(c, RLB_ERR_STATE, "rlb_macro before rlb_init_fields");
    const void* A = state ? state : c->A;
    const size_t N = (size_t)c->g.N;
    double *dn = n, *de = eps, *db = beta;
    void* tmp = nullptr;
    if (where == RLB_HOST) {
        RLB_CUDA(c, cudaMallocAsync(&tmp, N * 5 * sizeof(double), c->stream), "cudaMallocAsync (macro staging)");
        dn = (double*)tmp;
        de = dn + N;
        db = dn + 2 * N;
    }
    RLB_CUDA(c, cudaMemsetAsync(c->cnt.macro_bad, 0, sizeof(unsigned long long), c->stream), "memset");
    rlb_status s = after_launch(c,
                                c->ph.eos ? launch_macro_eos(c->g, c->ph, A, dn, de, db, c->cnt, c->stream)
                                          : launch_macro(c->p.prec, c->g, c->ph, A, dn, de, db, c->cnt, c->stream),
                                "macro");
    if (s != RLB_OK) return s;
    if (tmp) {
        RLB_CUDA(c, cudaMemcpyAsync(n, dn, N * 8, cudaMemcpyDeviceToHost, c->stream), "copy n");
        RLB_CUDA(c, cudaMemcpyAsync(eps, de, N * 8, cudaMemcpyDeviceToHost, c->stream), "copy eps");
        RLB_CUDA(c, cudaMemcpyAsync(beta, db, 3 * N * 8, cudaMemcpyDeviceToHost, c->stream), "copy beta");
        RLB_CUDA(c, cudaFreeAsync(tmp, c->stream), "cudaFreeAsync (macro staging)");
    }
    unsigned long long bad = 0, first = 0;
    RLB_CUDA(c, cudaMemcpyAsync(&bad, c->cnt.macro_bad, sizeof bad, cudaMemcpyDeviceToHost, c->stream), "copy count");
    RLB_CUDA(c, cudaMemcpyAsync(&first, c->cnt.first_bad, sizeof first, cudaMemcpyDeviceToHost, c->stream), "copy count");
    RLB_CUDA(c, cudaStreamSynchronize(c->stream), "sync");
    if (bad || first != ~0ull) return fail(c, RLB_ERR_UNPHYSICAL, "unphysical cells: %llu in the output state%s", bad,
                                           first != ~0ull ? " (and during the run)" : "");
    return RLB_OK;
}

rlb_status rlb_stats(rlb_ctx* c, int64_t* steps, int64_t* n_unphysical, int64_t* first_bad, int64_t* n_nonpositive_eq) {
    RLB_LATCHED(c);
    unsigned long long* h = (unsigned long long*)malloc(sizeof(unsigned long long) * (2 * kCounterSlots + 3));
    if (!h) return fail(c, RLB_ERR_OOM, "host allocation failed");
    cudaError_t e = cudaMemcpyAsync(h, c->cnt.slots, sizeof(unsigned long long) * (2 * kCounterSlots + 3),
                                    cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        free(h);
        return cuda_fail(c, e, "stats");
    }
    unsigned long long u = 0, p = 0;
    for (int i = 0; i < kCounterSlots; ++i) {
        u += h[i];
        p += h[kCounterSlots + i];
    }
    const unsigned long long fb = h[2 * kCounterSlots];
    const unsigned long long perr = h[2 * kCounterSlots + 2];
    free(h);
    if (perr) {
        c->err = cudaErrorLaunchTimeout;
        return fail(c, RLB_ERR_CUDA, "a staged kernel timed out waiting for its bulk copies (%llu CTAs)", perr);
    }
    if (steps) *steps = c->steps;
    if (n_unphysical) *n_unphysical = (int64_t)u;
    if (first_bad) *first_bad = fb == ~0ull ? -1 : (int64_t)fb;
    if (n_nonpositive_eq) *n_nonpositive_eq = (int64_t)p;
    return RLB_OK;
}

rlb_status rlb_adjoint_macro(rlb_ctx* c, const void* state, const double* dL_dn, const double* dL_deps,
                             const double* dL_dbeta, void* lam_out) {
    RLB_LATCHED(c);
    if (c->ph.eos) return fail(c, RLB_ERR_ARG, "the discrete adjoint covers the eps = 3P equation of state");
    if (c->g.zhalo) return fail(c, RLB_ERR_ARG, "the discrete adjoint covers whole lattices (no z slabs)");
    if (!state || !dL_dn || !dL_deps || !dL_dbeta || !lam_out) return fail(c, RLB_ERR_ARG, "null pointer");
    return after_launch(c, launch_adjoint_macro(c->p.prec, c->g, c->ph, state, dL_dn, dL_deps, dL_dbeta, lam_out,
                                                c->stream),
                        "adjoint_macro");
}

rlb_status rlb_adjoint_step(rlb_ctx* c, const void* state_t, const void* lam_in, void* lam_out, double* dL_dtau_accum,
                            double* dL_dbeta_in_accum) {
    Nvtx nvtx_("rlb_adjoint_step");
    RLB_LATCHED(c);
    if (c->ph.eos) return fail(c, RLB_ERR_ARG, "the discrete adjoint covers the eps = 3P equation of state");
    if (c->g.zhalo) return fail(c, RLB_ERR_ARG, "the discrete adjoint covers whole lattices (no z slabs)");
    if (!state_t || !lam_in || !lam_out || lam_in == lam_out) return fail(c, RLB_ERR_ARG, "bad buffers");
    if (!dL_dtau_accum || !dL_dbeta_in_accum) return fail(c, RLB_ERR_ARG, "accumulators are required");
    return after_launch(c, launch_adjoint_step(c->p.prec, c->g, c->ph, state_t, lam_in, lam_out, c->red, c->inflow_d,
                                               dL_dtau_accum, dL_dbeta_in_accum, c->stream),
                        "adjoint_step");
}

rlb_status rlb_adjoint_step_noalloc(rlb_ctx* c, const void* state_t, const void* lam_in, void* lam_out,
                                    double* dL_dtau_accum, double* dL_dbeta_in_accum) {
    RLB_LATCHED(c);
    if (c->ph.eos) return fail(c, RLB_ERR_ARG, "the discrete adjoint covers the eps = 3P equation of state");
    if (c->g.zhalo) return fail(c, RLB_ERR_ARG, "the discrete adjoint covers whole lattices (no z slabs)");
    if (!state_t || !lam_in || !lam_out || lam_in == lam_out) return fail(c, RLB_ERR_ARG, "bad buffers");
    if (!dL_dtau_accum || !dL_dbeta_in_accum) return fail(c, RLB_ERR_ARG, "accumulators are required");
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaGetDevice");
    if (dev != c->device)
        return fail(c, RLB_ERR_STATE, "rlb_adjoint_step_noalloc: the context's device %d is not current (%d is)",
                    c->device, dev);
    long long need = 0;
    e = launch_adjoint_step_noalloc(c->p.prec, c->g, c->ph, state_t, lam_in, lam_out, c->inflow_d, dL_dtau_accum,
                                    dL_dbeta_in_accum, c->stream, &need);
    if (e == cudaErrorInvalidValue && need > kAdjScratchDoubles)
        return fail(c, RLB_ERR_ARG,
                    "rlb_adjoint_step_noalloc: the launch needs %lld scratch doubles, the static maximum is %lld",
                    need, kAdjScratchDoubles);
    return after_launch(c, e, "adjoint_step_noalloc");
}

rlb_status rlb_adjoint_fields(rlb_ctx* c, const double* n0, const double* eps0, const double* beta0, const void* lam0,
                              double* dL_dn0, double* dL_deps0, double* dL_dbeta0, double* dL_dbeta_in_accum) {
    RLB_LATCHED(c);
    if (c->ph.eos) return fail(c, RLB_ERR_ARG, "the discrete adjoint covers the eps = 3P equation of state");
    if (c->g.zhalo) return fail(c, RLB_ERR_ARG, "the discrete adjoint covers whole lattices (no z slabs)");
    if (!n0 || !eps0 || !beta0 || !lam0 || !dL_dn0 || !dL_deps0 || !dL_dbeta0 || !dL_dbeta_in_accum)
        return fail(c, RLB_ERR_ARG, "null pointer");
    if (!c->inited) return fail(c, RLB_ERR_STATE, "rlb_adjoint_fields needs the solid layout of rlb_init_fields");
    return after_launch(c, launch_adjoint_fields(c->p.prec, c->g, c->ph, n0, eps0, beta0, c->A, lam0, dL_dn0, dL_deps0,
                                                 dL_dbeta0, c->red, dL_dbeta_in_accum, c->stream),
                        "adjoint_fields");
}

rlb_status rlb_halo_exchange(rlb_ctx* lo, rlb_ctx* up) {
    Nvtx nvtx_("rlb_halo_exchange");
    RLB_LATCHED(lo);
    RLB_LATCHED(up);
    if (!lo->g.zhalo || !up->g.zhalo) return fail(lo, RLB_ERR_ARG, "rlb_halo_exchange needs contexts with zbc = RLB_ZBC_HALO");
    if (lo->g.nx != up->g.nx || lo->g.ny != up->g.ny || lo->p.prec != up->p.prec || lo->p.xbc != up->p.xbc ||
        lo->device != up->device)
        return fail(lo, RLB_ERR_ARG, "slabs of one lattice need the same nx, ny, precision, x boundary and device");
    if (!lo->inited || !up->inited) return fail(lo, RLB_ERR_STATE, "rlb_halo_exchange before rlb_init_fields");
    int dev = -1;
    RLB_CUDA(lo, cudaGetDevice(&dev), "cudaGetDevice");
    if (dev != lo->device) return fail(lo, RLB_ERR_STATE, "the slabs' device %d is not current (%d is)", lo->device, dev);
    cudaEvent_t ev = nullptr;
    const bool two = up->stream != lo->stream;
    if (two) {
        // lower's stream waits for upper's earlier work; upper's later work
        // waits for the copy
        RLB_CUDA(lo, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "event");
        cudaError_t e = cudaEventRecord(ev, up->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(lo->stream, ev, 0);
        if (e != cudaSuccess) {
            cudaEventDestroy(ev);
            return cuda_fail(lo, e, "halo exchange ordering");
        }
    }
    rlb_status s = after_launch(lo, launch_halo_exchange(lo->elem, (long long)lo->g.nxy, lo->A, lo->g.S, lo->g.nz, up->A,
                                                         up->g.S, lo->stream),
                                "halo exchange");
    if (two) {
        cudaError_t e = cudaEventRecord(ev, lo->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(up->stream, ev, 0);
        cudaEventDestroy(ev);
        if (e != cudaSuccess && s == RLB_OK) s = cuda_fail(lo, e, "halo exchange ordering");
    }
    return s;
}

rlb_status rlb_selftest_conversions(const float* f_in, const double* d_in, int64_t n, double* f2d_out,
                                    float* d2f_out) {
    if (n < 0 || (n > 0 && (!f_in || !d_in || !f2d_out || !d2f_out))) return fail(nullptr, RLB_ERR_ARG, "bad arguments");
    cudaError_t e = launch_conversions(f_in, d_in, n, f2d_out, d2f_out);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "selftest_conversions");
    return RLB_OK;
}

rlb_status rlb_debug_bounds_violations(int64_t* count) {
    if (!count) return fail(nullptr, RLB_ERR_ARG, "count is NULL");
#ifdef RLB_CHECK_BOUNDS
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaDeviceSynchronize");
    const unsigned long long a = oob_take_forward(), b = oob_take_adjoint(), d = oob_take_eos(), e2 = oob_take_stream();
    if (a == ~0ull || b == ~0ull || d == ~0ull || e2 == ~0ull) return fail(nullptr, RLB_ERR_CUDA, "reading the bounds counters failed");
    *count = (int64_t)(a + b + d + e2);
    return RLB_OK;
#else
    *count = -1;
    return fail(nullptr, RLB_ERR_STATE, "librlb was built without RLB_CHECK_BOUNDS");
#endif
}

rlb_status rlb_debug_bounds_selftest(int64_t index, int64_t n, int64_t* checked) {
    if (!checked) return fail(nullptr, RLB_ERR_ARG, "checked is NULL");
#ifdef RLB_CHECK_BOUNDS
    *checked = (int64_t)bounds_selftest((long long)index, (long long)n, 0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "bounds self-test");
    return RLB_OK;
#else
    (void)index;
    (void)n;
    *checked = -1;
    return fail(nullptr, RLB_ERR_STATE, "librlb was built without RLB_CHECK_BOUNDS");
#endif
}

rlb_status rlb_sync(rlb_ctx* c) {
    RLB_LATCHED(c);
    RLB_CUDA(c, cudaStreamSynchronize(c->stream), "sync");
    RLB_CUDA(c, cudaGetLastError(), "sync");
    return RLB_OK;
}

const char* rlb_status_str(rlb_status s) {
    switch (s) {
        case RLB_OK: return "RLB_OK";
        case RLB_ERR_ARG: return "RLB_ERR_ARG";
        case RLB_ERR_OOM: return "RLB_ERR_OOM";
        case RLB_ERR_CUDA: return "RLB_ERR_CUDA";
        case RLB_ERR_UNPHYSICAL: return "RLB_ERR_UNPHYSICAL";
        case RLB_ERR_STATE: return "RLB_ERR_STATE";
    }
    return "RLB_UNKNOWN";
}

const char* rlb_last_error(rlb_ctx* c) { return c ? c->msg : g_msg; }

int64_t rlb_launch_count(rlb_ctx* c) { return c ? c->launches : 0; }

}  // extern "C"
