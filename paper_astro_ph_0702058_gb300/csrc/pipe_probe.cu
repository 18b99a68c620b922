// Throughput probes of the GPU pipes that bound the pair loop: chains of
// FP32 FMA, ADD and MUL, the packed FP32x2 FMA, and the MUFU reciprocal
// square root; and of the pipes that bound the FP64 predictor and corrector:
// FP64 FMA and the double -> float -> double conversions.  Then the latency of
// one dependent FP64 chain (FMA, square root + add, division + add) in one
// block of 1, 4 or 16 warps with 1 or 32 active lanes: the cycles each
// operation of a chain costs when the SM's FP64 unit is shared.  A standalone program (not part of libnbody.so); prints one
// JSON line with results per SM and clock, the clock taken from clock64()
// over the kernel's own duration.
#include <cstdio>
#include <cuda_runtime.h>

namespace {

constexpr int kChains = 8;    // independent accumulators per thread
constexpr int kInner = 16;    // unrolled repetitions per loop trip

__device__ __forceinline__ float rsqrt_approx(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ unsigned long long pack2(float lo, float hi)
{
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}

__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b, unsigned long long c)
{
    unsigned long long d;
    asm volatile("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// KIND 0: FFMA, 1: FADD, 2: FMUL; results kept alive through a data-dependent store
template <int KIND>
__global__ void scalar_chain(float *out, long long *cyc, int iters, float a, float b)
{
    const long long c0 = clock64();
    float r[kChains];
    for (int i = 0; i < kChains; ++i) r[i] = threadIdx.x * 1e-3f + i;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kInner; ++u)
#pragma unroll
            for (int i = 0; i < kChains; ++i) {
                if (KIND == 0) r[i] = fmaf(r[i], a, b);
                else if (KIND == 1) r[i] = r[i] + a;
                else r[i] = r[i] * a;
            }
    }
    float s = 0.f;
    for (int i = 0; i < kChains; ++i) s += r[i];
    if (s == 1234.5f) out[0] = s;
    if (threadIdx.x == 0) cyc[blockIdx.x] = clock64() - c0;
}

__global__ void packed_chain(float *out, long long *cyc, int iters, float a, float b)
{
    const long long c0 = clock64();
    unsigned long long r[kChains];
    for (int i = 0; i < kChains; ++i) r[i] = pack2(threadIdx.x * 1e-3f + i, i * 0.5f);
    const unsigned long long A = pack2(a, a), B = pack2(b, b);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kInner; ++u)
#pragma unroll
            for (int i = 0; i < kChains; ++i) r[i] = fma2(r[i], A, B);
    }
    unsigned long long s = 0;
    for (int i = 0; i < kChains; ++i) s ^= r[i];
    if (s == 12345ull) out[0] = 1.f;
    if (threadIdx.x == 0) cyc[blockIdx.x] = clock64() - c0;
}

__global__ void mufu_chain(float *out, long long *cyc, int iters)
{
    const long long c0 = clock64();
    float r[kChains];
    for (int i = 0; i < kChains; ++i) r[i] = 1.0f + threadIdx.x * 1e-3f + i;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kInner; ++u)
#pragma unroll
            for (int i = 0; i < kChains; ++i) r[i] = rsqrt_approx(r[i]) + 1.0f;  // 1 MUFU + 1 FADD
    }
    float s = 0.f;
    for (int i = 0; i < kChains; ++i) s += r[i];
    if (s == 1234.5f) out[0] = s;
    if (threadIdx.x == 0) cyc[blockIdx.x] = clock64() - c0;
}

// FP64 FMA chains (KIND 0) and double -> float -> double conversion chains (KIND 1, two conversions)
template <int KIND>
__global__ void fp64_chain(float *out, long long *cyc, int iters, double a, double b)
{
    const long long c0 = clock64();
    double r[kChains];
    for (int i = 0; i < kChains; ++i) r[i] = threadIdx.x * 1e-3 + i + 0.25;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kInner; ++u)
#pragma unroll
            for (int i = 0; i < kChains; ++i) {
                if (KIND == 0) r[i] = fma(r[i], a, b);
                else r[i] = static_cast<double>(__double2float_rn(r[i]));
            }
    }
    double s = 0.0;
    for (int i = 0; i < kChains; ++i) s += r[i];
    if (s == 1234.5) out[0] = 1.f;
    if (threadIdx.x == 0) cyc[blockIdx.x] = clock64() - c0;
}

// One dependent chain per active lane (lanes < `lanes` of every warp); cycles per operation in cyc[0].
template <int KIND>
__global__ void fp64_dep(float *out, long long *cyc, int iters, int lanes, double a, double b)
{
    double r = 1.0 + threadIdx.x * 1e-3;
    __syncthreads();
    const long long c0 = clock64();
    if (static_cast<int>(threadIdx.x & 31) < lanes) {
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int u = 0; u < kInner; ++u) {
                if (KIND == 0) r = fma(r, a, b);
                else if (KIND == 1) r = sqrt(r) + b;
                else r = b / r + a;
            }
        }
    }
    __syncthreads();
    const long long c1 = clock64();
    if (r == 12345.0) out[0] = 1.f;
    if (threadIdx.x == 0) cyc[0] = c1 - c0;
}

}  // namespace

int main()
{
    int sm = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = sm * 8, threads = 256, iters = 2000;
    float *out = nullptr;
    long long *cyc = nullptr;
    if (cudaMalloc(&out, 16) != cudaSuccess || cudaMalloc(&cyc, blocks * sizeof(long long)) != cudaSuccess) {
        std::printf("{\"error\": \"allocation failed\"}\n");
        return 1;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double ops_per_thread = static_cast<double>(iters) * kInner * kChains;
    const double threads_total = static_cast<double>(blocks) * threads;
    long long *cyc_h = new long long[blocks];
    auto run = [&](const char *name, double results_per_op, auto launch) {
        launch();  // warm-up
        cudaDeviceSynchronize();
        cudaEventRecord(e0);
        launch();
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        cudaMemcpy(cyc_h, cyc, blocks * sizeof(long long), cudaMemcpyDeviceToHost);
        long long cmax = 0;
        for (int i = 0; i < blocks; ++i) cmax = cyc_h[i] > cmax ? cyc_h[i] : cmax;
        const double clk = static_cast<double>(cmax) / (ms * 1e-3);  // SM clock seen by the busiest block
        const double per_sm_clk = ops_per_thread * threads_total * results_per_op / (ms * 1e-3) / sm / clk;
        std::printf("\"%s\": {\"per_sm_per_clk\": %.2f, \"sm_mhz\": %.0f}, ", name, per_sm_clk, clk * 1e-6);
    };
    std::printf("{");
    run("ffma", 1.0, [&] { scalar_chain<0><<<blocks, threads>>>(out, cyc, iters, 1.0001f, 1e-6f); });
    run("fadd", 1.0, [&] { scalar_chain<1><<<blocks, threads>>>(out, cyc, iters, 1e-6f, 1e-6f); });
    run("fmul", 1.0, [&] { scalar_chain<2><<<blocks, threads>>>(out, cyc, iters, 1.0000001f, 1e-6f); });
    run("ffma2_fp32_results", 2.0, [&] { packed_chain<<<blocks, threads>>>(out, cyc, iters, 1.0001f, 1e-6f); });
    run("mufu_rsqrt", 1.0, [&] { mufu_chain<<<blocks, threads>>>(out, cyc, iters); });
    const int iters64 = iters / 20;  // the FP64 pipes are narrow: fewer trips
    ops_per_thread = static_cast<double>(iters64) * kInner * kChains;
    run("dfma", 1.0, [&] { fp64_chain<0><<<blocks, threads>>>(out, cyc, iters64, 1.0000001, 1e-9); });
    run("f64_f32_f64_conversions", 2.0, [&] { fp64_chain<1><<<blocks, threads>>>(out, cyc, iters64, 0.0, 0.0); });
    // dependent FP64 chains in one block: cycles per operation
    const int dep_iters = 64;
    auto dep = [&](const char *name, int warps, int lanes, auto launch) {
        launch(warps, lanes);  // warm-up
        launch(warps, lanes);
        long long c = 0;
        cudaMemcpy(&c, cyc, sizeof(long long), cudaMemcpyDeviceToHost);
        std::printf("\"%s_%dw_%dl_clk_per_op\": %.1f, ", name, warps, lanes,
                    static_cast<double>(c) / (dep_iters * kInner));
    };
    for (int wl : {1, 32, 4, 16}) {  // 1 warp with 1 or 32 lanes, 4 and 16 warps with 32 lanes
        const int warps = wl == 32 ? 1 : wl, lanes = wl == 1 ? 1 : 32;
        dep("dfma_dep", warps, lanes, [&](int w, int l) {
            fp64_dep<0><<<1, 32 * w>>>(out, cyc, dep_iters, l, 1.0000001, 1e-9);
        });
    }
    dep("dsqrt_plus_dadd_dep", 1, 32, [&](int w, int l) { fp64_dep<1><<<1, 32 * w>>>(out, cyc, dep_iters, l, 1.0, 1e-9); });
    dep("ddiv_plus_dadd_dep", 1, 32, [&](int w, int l) { fp64_dep<2><<<1, 32 * w>>>(out, cyc, dep_iters, l, 1.0000001, 1e-9); });
    const cudaError_t err = cudaGetLastError();
    std::printf("\"sms\": %d, \"status\": \"%s\"}\n", sm, cudaGetErrorString(err));
    delete[] cyc_h;
    return err == cudaSuccess ? 0 : 1;
}
