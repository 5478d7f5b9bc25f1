// gb300_probes.cu -- throughput microbenchmarks behind the kernel design of
// librlb on GB300: FP64 FMA/add, binary32<->binary64 conversion, FP32 FMA,
// rsqrt, IEEE FP64 sqrt/div, and 1-D bulk asynchronous copies (TMA) of
// various sizes.  Pure register arithmetic or bounded copies; every wait is
// bounded.  Prints one JSON object per line.
#include <cstdint>
#include <cstdio>
#include <cuda_runtime.h>

#define ITERS 2048

__global__ void k_dfma(double* out, double a, double b) {
    double x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
    for (int i = 0; i < ITERS; ++i) {
        x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
        x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}
__global__ void k_ffma(float* out, float a, float b) {
    float x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
    for (int i = 0; i < ITERS; ++i) {
        x0 = fmaf(x0, a, b); x1 = fmaf(x1, a, b); x2 = fmaf(x2, a, b); x3 = fmaf(x3, a, b);
        x4 = fmaf(x4, a, b); x5 = fmaf(x5, a, b); x6 = fmaf(x6, a, b); x7 = fmaf(x7, a, b);
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}
// cvt.f64.f32 and cvt.rn.f32.f64 in chains the compiler cannot remove
__global__ void k_cvt(float* out, float a) {
    float x0 = threadIdx.x * 1e-3f, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3;
    double d0, d1, d2, d3;
    for (int i = 0; i < ITERS; ++i) {
        asm volatile("cvt.f64.f32 %0, %1;" : "=d"(d0) : "f"(x0)); asm volatile("cvt.f64.f32 %0, %1;" : "=d"(d1) : "f"(x1));
        asm volatile("cvt.f64.f32 %0, %1;" : "=d"(d2) : "f"(x2)); asm volatile("cvt.f64.f32 %0, %1;" : "=d"(d3) : "f"(x3));
        asm volatile("cvt.rn.f32.f64 %0, %1;" : "=f"(x0) : "d"(d0)); asm volatile("cvt.rn.f32.f64 %0, %1;" : "=f"(x1) : "d"(d1));
        asm volatile("cvt.rn.f32.f64 %0, %1;" : "=f"(x2) : "d"(d2)); asm volatile("cvt.rn.f32.f64 %0, %1;" : "=f"(x3) : "d"(d3));
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + a;
}
__global__ void k_rsq(float* out) {
    float x0 = threadIdx.x + 1.f, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3;
    for (int i = 0; i < ITERS; ++i) { x0 = rsqrtf(x0) + 1.f; x1 = rsqrtf(x1) + 1.f; x2 = rsqrtf(x2) + 1.f; x3 = rsqrtf(x3) + 1.f; }
    out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3;
}
__global__ void k_dsqrt(double* out) {
    double x0 = threadIdx.x + 1., x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3;
    for (int i = 0; i < ITERS / 8; ++i) { x0 = sqrt(x0) + 1.; x1 = sqrt(x1) + 1.; x2 = sqrt(x2) + 1.; x3 = sqrt(x3) + 1.; }
    out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3;
}
__global__ void k_ddiv(double* out, double a) {
    double x0 = threadIdx.x + 1., x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3;
    for (int i = 0; i < ITERS / 8; ++i) { x0 = a / x0 + 1.; x1 = a / x1 + 1.; x2 = a / x2 + 1.; x3 = a / x3 + 1.; }
    out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3;
}

__device__ __forceinline__ unsigned su(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ bool try_wait(uint64_t* bar, unsigned par) {
    unsigned ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok) : "r"(su(bar)), "r"(par) : "memory");
    return ok;
}
// One CTA per SM; thread 0 issues NC bulk copies of SZ bytes into distinct
// shared-memory slots completing on one mbarrier, all threads wait; ITERS rounds.
__global__ void k_bulk(const char* __restrict__ src, long long src_bytes, int SZ, int NC, int iters, unsigned* err) {
    extern __shared__ __align__(128) unsigned char sm[];
    uint64_t* bar = (uint64_t*)sm;
    unsigned char* buf = sm + 128;
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su(bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    long long off = (long long)blockIdx.x * NC * SZ;
    for (int it = 0; it < iters; ++it) {
        const long long base = (off % (src_bytes - 64ll * 200 * 1024)) & ~127ll;
        if (threadIdx.x == 0) {
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su(bar)), "r"(NC * SZ) : "memory");
            for (int c = 0; c < NC; ++c) {
                const long long o = base + (long long)c * ((SZ + 127) & ~127);
                asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                             ::"r"(su(buf + c * SZ)), "l"(src + o), "r"(SZ), "r"(su(bar)) : "memory");
            }
        }
        __syncwarp();
        bool ok = false;
        for (unsigned k = 0; k < (1u << 24); ++k)
            if (try_wait(bar, it & 1)) { ok = true; break; }
        if (!ok) atomicAdd(err, 1u);
        __syncthreads();
        off += (long long)gridDim.x * NC * SZ;
    }
}

int main() {
    int sms, clk;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
    cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, 0);
    const int blocks = sms * 8, threads = 256, n = blocks * threads;
    double* d; float* f;
    cudaMalloc(&d, n * sizeof(double));
    cudaMalloc(&f, n * sizeof(float));
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    float ms;
    auto report = [&](const char* name, double ops_per_thread) {
        cudaEventElapsedTime(&ms, a, b);
        const double ops = ops_per_thread * n;
        printf("{\"op\": \"%s\", \"gops\": %.1f, \"per_sm_per_clk\": %.3f}\n", name, ops / (ms * 1e-3) / 1e9,
               ops / (ms * 1e-3) / (sms * (clk * 1e3)));
    };
#define TIME(name, ops, launch)                                   \
    launch;                                                       \
    cudaEventRecord(a); launch; cudaEventRecord(b);               \
    cudaEventSynchronize(b); report(name, ops);
    TIME("dfma", 8.0 * ITERS, (k_dfma<<<blocks, threads>>>(d, 0.999, 1e-3)));
    TIME("ffma", 8.0 * ITERS, (k_ffma<<<blocks, threads>>>(f, 0.999f, 1e-3f)));
    TIME("cvt f32<->f64 (each counted)", 8.0 * ITERS, (k_cvt<<<blocks, threads>>>(f, 1.f)));
    TIME("rsqrtf", 4.0 * ITERS, (k_rsq<<<blocks, threads>>>(f)));
    TIME("dsqrt (IEEE)", 4.0 * ITERS / 8, (k_dsqrt<<<blocks, threads>>>(d)));
    TIME("ddiv (IEEE)", 4.0 * ITERS / 8, (k_ddiv<<<blocks, threads>>>(d, 3.0)));
    const long long src_bytes = 2ll << 30;
    char* src;
    cudaMalloc(&src, src_bytes);
    cudaMemset(src, 1, src_bytes);
    unsigned* err;
    cudaMalloc(&err, 4);
    cudaMemset(err, 0, 4);
    cudaFuncSetAttribute(k_bulk, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    const int sizes[] = {800, 1600, 4096, 8192};
    const int ncs[] = {1, 8, 38};
    for (int si = 0; si < 4; ++si)
        for (int ni = 0; ni < 3; ++ni) {
            const int SZ = sizes[si], NC = ncs[ni], it = 200;
            if ((long long)SZ * NC > 190 * 1024) continue;
            k_bulk<<<sms, 256, 128 + SZ * NC>>>(src, src_bytes, SZ, NC, 2, err);
            cudaEventRecord(a);
            k_bulk<<<sms, 256, 128 + SZ * NC>>>(src, src_bytes, SZ, NC, it, err);
            cudaEventRecord(b);
            cudaEventSynchronize(b);
            cudaEventElapsedTime(&ms, a, b);
            printf("{\"op\": \"bulk copy\", \"bytes\": %d, \"copies_per_round\": %d, \"us_per_round\": %.3f, \"GBs\": %.1f}\n",
                   SZ, NC, ms * 1e3 / it, (double)sms * it * NC * SZ / (ms * 1e-3) / 1e9);
        }
    unsigned h;
    cudaMemcpy(&h, err, 4, cudaMemcpyDeviceToHost);
    printf("{\"sms\": %d, \"clock_khz\": %d, \"bulk_wait_timeouts\": %u, \"err\": \"%s\"}\n", sms, clk, h,
           cudaGetErrorString(cudaGetLastError()));
    return 0;
}
