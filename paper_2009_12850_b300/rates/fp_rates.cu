// Rate microbenchmark of the arithmetic the FP64 design depends on: FP64 FMA and
// add, f64<->f32 conversions, FP32 FMA and packed FP32x2 FMA.  Each kernel runs
// 8 independent dependency chains per thread over 8 CTAs per SM; results are
// written only under a runtime flag that is 0, so nothing is optimised away.
// Prints one JSON object: operations per second and per clock per SM.
#include <cstdio>
#include <cuda_runtime.h>

constexpr int IT = 4096;
typedef unsigned long long u64;

__device__ __forceinline__ u64 fma2(u64 a, u64 b, u64 c) {
    u64 d;
    asm volatile("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__global__ void k_dfma(double *o, double a, double b, int f) {
    double x[8];
    for (int j = 0; j < 8; j++) x[j] = threadIdx.x + j;
    for (int i = 0; i < IT / 8; i++)
#pragma unroll
        for (int j = 0; j < 8; j++) x[j] = fma(x[j], a, b);
    if (f) o[threadIdx.x] = x[0] + x[1] + x[2] + x[3] + x[4] + x[5] + x[6] + x[7];
}
__global__ void k_ffma(float *o, float a, float b, int f) {
    float x[8];
    for (int j = 0; j < 8; j++) x[j] = threadIdx.x + j;
    for (int i = 0; i < IT; i++)
#pragma unroll
        for (int j = 0; j < 8; j++) x[j] = fmaf(x[j], a, b);
    if (f) o[threadIdx.x] = x[0] + x[1] + x[2] + x[3] + x[4] + x[5] + x[6] + x[7];
}
__global__ void k_ffma2(u64 *o, u64 a, u64 b, int f) {
    u64 x[8];
    for (int j = 0; j < 8; j++) x[j] = threadIdx.x + j;
    for (int i = 0; i < IT; i++)
#pragma unroll
        for (int j = 0; j < 8; j++) x[j] = fma2(x[j], a, b);
    if (f) o[threadIdx.x] = x[0] ^ x[1] ^ x[2] ^ x[3] ^ x[4] ^ x[5] ^ x[6] ^ x[7];
}
__global__ void k_d2f(float *o, int f) {
    double x[8];
    float acc[8];
    for (int j = 0; j < 8; j++) { x[j] = threadIdx.x + j; acc[j] = 0.f; }
    for (int i = 0; i < IT / 8; i++) {
#pragma unroll
        for (int j = 0; j < 8; j++) acc[j] += __double2float_rn(x[j]);
#pragma unroll
        for (int j = 0; j < 8; j++) x[j] = __hiloint2double(__double2hiint(x[j]) ^ (int)acc[j], __double2loint(x[j]));
    }
    if (f) o[threadIdx.x] = acc[0] + acc[1] + acc[2] + acc[3] + acc[4] + acc[5] + acc[6] + acc[7];
}

int main() {
    int sms = 0, clk = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
    cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, 0);
    const int blocks = sms * 8, thr = 256;
    void *o = nullptr;
    if (cudaMalloc(&o, (size_t)blocks * thr * 8) != cudaSuccess) return 1;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    const double threads = (double)blocks * thr;
    struct R { const char *name; double ops; float ms; } r[5] = {
        {"dfma", threads * IT, 0}, {"ffma", threads * IT * 8, 0}, {"ffma2_lanes", threads * IT * 16, 0},
        {"cvt_f64_f32", threads * IT, 0}, {"none", 0, 0}};
    for (int rep = 0; rep < 2; rep++) {
        cudaEventRecord(a); k_dfma<<<blocks, thr>>>((double *)o, 1.0000001, 1e-9, 0); cudaEventRecord(b);
        cudaEventSynchronize(b); cudaEventElapsedTime(&r[0].ms, a, b);
        cudaEventRecord(a); k_ffma<<<blocks, thr>>>((float *)o, 1.0000001f, 1e-9f, 0); cudaEventRecord(b);
        cudaEventSynchronize(b); cudaEventElapsedTime(&r[1].ms, a, b);
        cudaEventRecord(a); k_ffma2<<<blocks, thr>>>((u64 *)o, 0x3f8000013f800001ull, 0x3000000030000000ull, 0);
        cudaEventRecord(b); cudaEventSynchronize(b); cudaEventElapsedTime(&r[2].ms, a, b);
        cudaEventRecord(a); k_d2f<<<blocks, thr>>>((float *)o, 0); cudaEventRecord(b);
        cudaEventSynchronize(b); cudaEventElapsedTime(&r[3].ms, a, b);
    }
    if (cudaGetLastError() != cudaSuccess) return 2;
    printf("{\"sms\": %d, \"clock_khz\": %d", sms, clk);
    for (int q = 0; q < 4; q++)
        printf(", \"%s_per_s\": %.4e, \"%s_per_clk_sm\": %.3f", r[q].name, r[q].ops / (r[q].ms * 1e-3), r[q].name,
               r[q].ops / (r[q].ms * 1e-3) / sms / (clk * 1e3));
    printf("}\n");
    return 0;
}
