// rlb_internal.h -- types shared by the host API and the kernels of librlb.
//
// Kernel argument blocks and the launcher functions that each .cu file
// exports to the C-ABI layer (rlb_api.cu).  Nothing here is part of the
// public ABI (include/rlb.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace rlb {

enum : int { XBC_PERIODIC = 0, XBC_INFLOW_OUTFLOW = 1, XBC_OUTFLOW_BOTH = 2 };

// Number of counter slots that warps spread their statistics over.
constexpr int kCounterSlots = 4096;

// n / d = (umulhi(n, mul) + n) >> shift for 0 <= n < 2^31, 1 <= d < 2^31.
struct FastDiv {
    unsigned mul, shift;
};
inline FastDiv make_fast_div(unsigned d) {
    unsigned l = 0;
    while (l < 32 && (1ull << l) < d) ++l;  // l = ceil(log2 d)
    const unsigned long long m = ((1ull << 32) * ((1ull << l) - d)) / d + 1;
    return FastDiv{(unsigned)m, l};
}

// Lattice geometry.  Populations of plane q (0..37) of a state start at
// element q * S; cell index c = (z*ny + y)*nx + x.
struct Geom {
    int nx, ny, nz;
    int nxy;     // nx * ny
    int N;       // nx * ny * nz (< 2^31)
    long long S; // plane stride in elements (N rounded up to a multiple of 64)
    int xbc;
    int tma;     // 1: use the TMA-staged FP32 step where the lattice allows it
    int variant; // launch variant of the one-cell-per-thread FP32 step (tuning)
    int pipe_blocks;  // resident blocks per SM of the persistent variant (tuning)
    FastDiv div_nx, div_ny;
    int adj_pipe;   // FP32 adjoint kernel: 0 one cell per thread, 1 persistent, 2 staged (tuning)
    int adj_coop;   // staged FP32 adjoint: 1 lambda copied by the whole block (default), 0 per thread
    int zhalo;      // 1: planes z = 0 and z = nz-1 are halo copies, not updated by a step
    int f64df;      // 1: the FP64 step computes in compensated binary32 pairs (ablation)
    int f64split;   // FP64 step with eight lanes per cell: -1 small lattices, 0 never, 1 always (tests)
};

// Physical parameters, with the derived constants the kernels use.
struct Phys {
    double tau, omega, c_l;
    double inv_cl, inv_cl2;
    double n_in, eps_in, beta_in[3];
    double n_ref, eps_ref;  // FP32 deviation reference (beta = 0)
    int eos;                // 0: eps = 3P; 1: P = (eos_gamma - 1)(eps - n eos_mass)
    double eos_gamma, eos_mass;
    // Products of the run's constants that the FP64 step multiplies its
    // per-cell values by, formed once on the host (w_cl: the pair weights
    // 1/18, 1/36; w0 = 1/3): omega w_cl / c_l^2, 6 omega w_cl / c_l^2,
    // 4 omega w_cl / c_l, omega w_cl, 3 omega w_cl / c_l, omega w0, and for
    // omega g_0^eq: 4 omega w0, -omega w0 (2/c_l^2 + 1), -2 omega w0 / c_l^2;
    // -3 c_l^2 and 3 c_l for the recovery from M / c_l.
    double c_k1[2], c_k2[2], c_k3[2], c_fs[2], c_fa[2], c_f0, c_g0[3], m3cl2, three_cl;
};

// Binary32 constants of the FP32 deviation step.
struct Dev32 {
    float omega, omw, c_l, inv_cl, inv_cl2, n_ref;
    float g0a, g0b;  // 3 - 2/c_l^2 and 4 - 2/c_l^2
    double eps_ref;
    double n_ref_d, c_l_d, inv_cl_d, inv_cl2_d;  // binary64 copies (compensated collision)
};

// Device-side statistics of a run (see rlb_stats).
struct Counters {
    unsigned long long* slots;      // [2][kCounterSlots]: unphysical, non-positive equilibria
    unsigned long long* first_bad;  // min over flagged updates of step*N + cell
    unsigned long long* macro_bad;  // cells flagged by the last macro evaluation
    unsigned long long* pipe_err;   // set when a staged kernel gave up waiting for its copies
};

// Launchers (return the launch error, enqueue on 'stream').
cudaError_t launch_init(int prec, const Geom& g, const Phys& ph, const double* n, const double* eps,
                        const double* beta, const uint8_t* solid, void* A, void* B, cudaStream_t stream);
cudaError_t launch_step(int prec, const Geom& g, const Phys& ph, const void* A, void* B, Counters cnt,
                        bool count, long long step_index, cudaStream_t stream);
cudaError_t launch_macro(int prec, const Geom& g, const Phys& ph, const void* A, double* n, double* eps,
                         double* beta, Counters cnt, cudaStream_t stream);
// FP64 step with its arithmetic in compensated binary32 pairs (rlb_f64df.cu).
cudaError_t launch_step_f64_df(const Geom& g, const Phys& ph, const void* A, void* B, Counters cnt, bool count,
                               long long step_index, cudaStream_t stream, int threads);
// TMA-staged FP32 step; returns cudaErrorNotSupported when the lattice does
// not meet its alignment / shared-memory conditions (caller falls back).
cudaError_t launch_step_f32_tma(const Geom& g, const Dev32& c, const float* A, float* B, Counters cnt, bool count,
                                long long step_index, cudaStream_t stream);
Dev32 make_dev32(const Phys& ph);

cudaError_t launch_conversions(const float* fi, const double* di, long long n, double* fo, float* dout);

cudaError_t launch_check_solid_planes(const Geom& g, const uint8_t* solid, unsigned long long* flag,
                                      cudaStream_t stream);

// Halo exchange between the current states of two z slabs (elem: 4 or 8
// bytes): the e_z = +1 populations of lower's plane z = nz_l - 2 into upper's
// plane 0, the e_z = -1 populations of upper's plane 1 into lower's plane
// nz_l - 1.
cudaError_t launch_halo_exchange(int elem, long long nxy, void* lower, long long S_lower, int nz_lower, void* upper,
                                 long long S_upper, cudaStream_t stream);

// Adjoint.  'red' holds 4 doubles of partial sums per 32-cell warp.
inline long long adj_red_doubles(long long N) { return 4 * 4 * ((N + 127) / 128); }
cudaError_t launch_adjoint_macro(int prec, const Geom& g, const Phys& ph, const void* A, const double* dn,
                                 const double* deps, const double* dbeta, void* lam, cudaStream_t stream);
cudaError_t launch_adjoint_step(int prec, const Geom& g, const Phys& ph, const void* A, const void* lam_in,
                                void* lam_out, double* red, const double* inflow_d, double* dtau, double* dbeta_in,
                                cudaStream_t stream);
// Allocation-free variant of launch_adjoint_step (same kernels, persistent
// grid): partial sums in a static device array of kAdjScratchDoubles doubles,
// set up once per device on first use.  Needs 16 doubles per block of the
// grid (reported in *need_doubles); returns cudaErrorInvalidValue, launching
// nothing, when that exceeds the array.
constexpr long long kAdjScratchDoubles = 32768;  // 256 KiB
cudaError_t launch_adjoint_step_noalloc(int prec, const Geom& g, const Phys& ph, const void* A, const void* lam_in,
                                        void* lam_out, const double* inflow_d, double* dtau, double* dbeta_in,
                                        cudaStream_t stream, long long* need_doubles);
// d eq_in / d beta_in table of the inflow state: kInflowTable doubles
// followed by the same kInflowTable values rounded to binary32 (the FP32
// adjoint kernels read the float copy, so their ghost cells convert nothing).
constexpr int kInflowTable = 38 * 3;
cudaError_t launch_inflow_derivs(const Phys& ph, double* out, cudaStream_t stream);
cudaError_t launch_adjoint_fields(int prec, const Geom& g, const Phys& ph, const double* n0, const double* eps0,
                                  const double* beta0, const void* A0, const void* lam0, double* dn0,
                                  double* deps0, double* dbeta0, double* red, double* dbeta_in,
                                  cudaStream_t stream);

// General equation of state (FP64): initialisation, step and macro output.
cudaError_t launch_init_eos(const Geom& g, const Phys& ph, const double* n, const double* eps, const double* beta,
                            const uint8_t* solid, void* A, void* B, cudaStream_t stream);
cudaError_t launch_step_eos(const Geom& g, const Phys& ph, const void* A, void* B, Counters cnt, bool count,
                            long long step_index, cudaStream_t stream);
cudaError_t launch_macro_eos(const Geom& g, const Phys& ph, const void* A, double* n, double* eps, double* beta,
                             Counters cnt, cudaStream_t stream);

// Out-of-range state indices counted by the bounds-checking build since the
// last call, per translation unit (always 0 in the release build).
unsigned long long oob_take_forward();
unsigned long long oob_take_adjoint();
unsigned long long oob_take_eos();
unsigned long long oob_take_stream();
#ifdef RLB_CHECK_BOUNDS
// Runs the index check on (i, n) in a kernel; returns the checked index.
long long bounds_selftest(long long i, long long n, cudaStream_t s);
#endif

// Kernel launches issued by the last launcher call (for accounting).
int last_launch_count();
void set_last_launch_count(int n);

}  // namespace rlb
