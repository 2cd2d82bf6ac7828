// Throughput micro-benchmark of the min-plus update c = min(c, a + b) on the ALU/FMA
// pipes, for the roofline of the Floyd-Warshall kernels (which are bound by it: min-plus
// has no tensor-core form).  Every operand is a register; each thread keeps 16
// independent accumulators and feeds them back as the next step's operands, so nothing
// is loop-invariant and no memory traffic is involved.
#include <cuda_runtime.h>
#include <stdint.h>

#include "spq_bench.h"

namespace {

__device__ __forceinline__ float fmin3(float a, float b, float c) {
    float d;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

__device__ __forceinline__ void add2(float& r0, float& r1, float a0, float a1, float b0, float b1) {
    unsigned long long x, y, z;
    asm("mov.b64 %0, {%1, %2};" : "=l"(x) : "f"(a0), "f"(a1));
    asm("mov.b64 %0, {%1, %2};" : "=l"(y) : "f"(b0), "f"(b1));
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(z) : "l"(x), "l"(y));
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r0), "=f"(r1) : "l"(z));
}

// MODE 0: f32 add + 2-input min (1 update / step); 1: f32 add + 3-input min over two
// k steps; 2: packed f32x2 add + 3-input min; 3: int32 add + min; 4: int32
// __viaddmin_s32; 5: int32 add, add, min, min over two k steps.
template <int MODE>
__global__ void __launch_bounds__(256) k_peak(const float* __restrict__ in, float* __restrict__ out, int iters) {
    float c[16], a0[4], a1[4], b0[4], b1[4];
    const int t = threadIdx.x & 63;
#pragma unroll
    for (int i = 0; i < 16; ++i) c[i] = in[(t + i) & 63];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        a0[i] = in[(t + 16 + i) & 63];
        a1[i] = in[(t + 20 + i) & 63];
        b0[i] = in[(t + 24 + i) & 63];
        b1[i] = in[(t + 28 + i) & 63];
    }
    if (MODE <= 2) {
#pragma unroll 1
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; j += 2) {
                    float& x = c[i * 4 + j];
                    float& y = c[i * 4 + j + 1];
                    if (MODE == 0) {
                        x = fminf(x, a0[i] + b0[j]);
                        y = fminf(y, a0[i] + b0[j + 1]);
                    } else if (MODE == 1) {
                        x = fmin3(x, a0[i] + b0[j], a1[i] + b1[j]);
                        y = fmin3(y, a0[i] + b0[j + 1], a1[i] + b1[j + 1]);
                    } else {
                        float s0, s1, u0, u1;
                        add2(s0, s1, a0[i], a0[i], b0[j], b0[j + 1]);
                        add2(u0, u1, a1[i], a1[i], b1[j], b1[j + 1]);
                        x = fmin3(x, s0, u0);
                        y = fmin3(y, s1, u1);
                    }
                }
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                a0[i] = c[i * 4];
                a1[i] = c[i * 4 + 1];
                b0[i] = c[i];
                b1[i] = c[4 + i];
            }
        }
    } else {
        int ci[16], ia0[4], ia1[4], ib0[4], ib1[4];
#pragma unroll
        for (int i = 0; i < 16; ++i) ci[i] = (int)c[i];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            ia0[i] = (int)a0[i];
            ia1[i] = (int)a1[i];
            ib0[i] = (int)b0[i];
            ib1[i] = (int)b1[i];
        }
#pragma unroll 1
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    int& x = ci[i * 4 + j];
                    if (MODE == 3)
                        x = min(x, ia0[i] + ib0[j]);
                    else if (MODE == 4)
                        x = __viaddmin_s32(ia0[i], ib0[j], x);
                    else
                        x = min(x, min(ia0[i] + ib0[j], ia1[i] + ib1[j]));
                }
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                ia0[i] = ci[i * 4];
                ia1[i] = ci[i * 4 + 1];
                ib0[i] = ci[i];
                ib1[i] = ci[4 + i];
            }
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) c[i] = (float)ci[i];
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < 16; ++i) s += c[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <int MODE>
cudaError_t run(int blocks, const float* in, float* out, int iters, cudaStream_t st) {
    k_peak<MODE><<<blocks, 256, 0, st>>>(in, out, iters);
    return cudaGetLastError();
}

}  // namespace

extern "C" int spq_peak_minplus(int mode, int iters, int blocks_per_sm, double* updates_per_s, double* ms) {
    if (mode < 0 || mode > 5 || iters <= 0 || blocks_per_sm <= 0) return (int)cudaErrorInvalidValue;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return (int)e;
    const int blocks = sms * blocks_per_sm;
    float *in = nullptr, *out = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess) return (int)e;
    if ((e = cudaMalloc(&in, 64 * sizeof(float))) != cudaSuccess) goto done;
    if ((e = cudaMalloc(&out, (size_t)blocks * 256 * sizeof(float))) != cudaSuccess) goto done;
    {
        float h[64];
        for (int i = 0; i < 64; ++i) h[i] = (float)((i * 37) % 61 + 1);
        if ((e = cudaMemcpy(in, h, sizeof(h), cudaMemcpyHostToDevice)) != cudaSuccess) goto done;
    }
    if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) goto done;
    for (int rep = 0; rep < 2; ++rep) {  // first launch warms up
        cudaEventRecord(e0, st);
        switch (mode) {
            case 0: e = run<0>(blocks, in, out, iters, st); break;
            case 1: e = run<1>(blocks, in, out, iters, st); break;
            case 2: e = run<2>(blocks, in, out, iters, st); break;
            case 3: e = run<3>(blocks, in, out, iters, st); break;
            case 4: e = run<4>(blocks, in, out, iters, st); break;
            default: e = run<5>(blocks, in, out, iters, st); break;
        }
        if (e != cudaSuccess) goto done;
        cudaEventRecord(e1, st);
        if ((e = cudaEventSynchronize(e1)) != cudaSuccess) goto done;
    }
    {
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        const double per_iter = (mode == 0 || mode == 3 || mode == 4) ? 16.0 : 32.0;
        const double upd = (double)blocks * 256.0 * iters * per_iter;
        if (ms) *ms = t;
        if (updates_per_s) *updates_per_s = upd / (t * 1e-3);
    }
done:
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (in) cudaFree(in);
    if (out) cudaFree(out);
    cudaStreamDestroy(st);
    return (int)e;
}
