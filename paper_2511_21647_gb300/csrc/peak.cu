// FP32 issue-rate probe: the denominator of the FP32 roofline, measured on the
// device that runs the library instead of derived from a clock and a lane
// count.  Every thread runs 16 independent dependent chains of FP32 FMAs
// (scalar `fma.rn.f32`, or eight chains of packed `fma.rn.f32x2` pairs), so
// the FMA pipe is the only thing that can bind; the launch fills every SM
// with 64 warps.  The chains' final values feed one conditional store, so no
// FMA is dead code.  No counterpart in the paper: a measurement aid.
#include "rca_internal.cuh"

namespace {

#define PK_THREADS 256
#define PK_BLOCKS_PER_SM 8
#define PK_CHAINS 16

template <bool PACKED>
__global__ void __launch_bounds__(PK_THREADS) k_fp32_probe(float* __restrict__ sink, int iters, float b, float c)
{
    const float seed = (float)threadIdx.x * 1e-3f;
    if constexpr (PACKED) {
        uint64_t a[PK_CHAINS / 2];
        const uint64_t bb = f2_pack(b, b), cc = f2_pack(c, c);
#pragma unroll
        for (int j = 0; j < PK_CHAINS / 2; ++j) a[j] = f2_pack(seed + (float)(2 * j), seed + (float)(2 * j + 1));
#pragma unroll 1
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int j = 0; j < PK_CHAINS / 2; ++j) a[j] = f2_fma(a[j], bb, cc);
        }
        float s = 0.f;
#pragma unroll
        for (int j = 0; j < PK_CHAINS / 2; ++j) {
            const float2 v = f2_unpack(a[j]);
            s += v.x + v.y;
        }
        if (s == 1234.5f) sink[blockIdx.x] = s;
    } else {
        float a[PK_CHAINS];
#pragma unroll
        for (int j = 0; j < PK_CHAINS; ++j) a[j] = seed + (float)j;
#pragma unroll 1
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int j = 0; j < PK_CHAINS; ++j) a[j] = fmaf(a[j], b, c);
        }
        float s = 0.f;
#pragma unroll
        for (int j = 0; j < PK_CHAINS; ++j) s += a[j];
        if (s == 1234.5f) sink[blockIdx.x] = s;
    }
}

}  // namespace

rca_status launch_fp32_probe(rca_handle* h, int packed, int iters, float* sink, double* flops)
{
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
    const int blocks = sms * PK_BLOCKS_PER_SM;
    // b slightly below 1 and c small keep every chain finite for any length
    if (packed)
        k_fp32_probe<true><<<blocks, PK_THREADS, 0, h->stream>>>(sink, iters, 0.999999f, 1e-6f);
    else
        k_fp32_probe<false><<<blocks, PK_THREADS, 0, h->stream>>>(sink, iters, 0.999999f, 1e-6f);
    if (flops) *flops = 2.0 * PK_CHAINS * (double)iters * (double)blocks * PK_THREADS;
    return cuda_check(h, cudaGetLastError(), "fp32 probe");
}

int fp32_probe_blocks(int sms) { return sms * PK_BLOCKS_PER_SM; }
