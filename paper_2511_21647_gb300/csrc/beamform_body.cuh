// beamform_body.cuh -- device bodies of the beamforming stages, shared by the
// single-ensemble kernels (beamform.cu) and the persistent batched kernel
// (batch_impl.cuh).
//
// Sec. II-A1 (two-stage RCA beamforming, Fig. 1b-c), Sec. II-A4/II-A5
// (P x P x N sub-blocks sum-projected onto x-z and y-z planes), Sec. II-A2
// (clutter removal before Stage 2; here the ensemble-mean filter).
#pragma once
#include <algorithm>
#include <type_traits>

#include "rca_internal.cuh"

namespace {


struct Fir {
    float h[31];
};

__device__ __forceinline__ float rf_value(const void* rf, int rf_t, size_t i)
{
    if (rf_t == RCA_F32) return reinterpret_cast<const float*>(rf)[i];
    if (rf_t == RCA_F16) return __half2float(reinterpret_cast<const __half*>(rf)[i]);
    return (float)reinterpret_cast<const int16_t*>(rf)[i];
}

// ---------------------------------------------------------------------------
// Ingest: ensemble mean of every (tx, element, sample), then mixing by
// exp(-j 2 pi fc t_n) and the half-band low-pass (x2).
// ---------------------------------------------------------------------------

// Four adjacent (tx, element, sample) columns per thread; frames strided by
// ncol, loaded four frames at a time.  float / half input: Neumaier-
// compensated float sums; int16: exact integer sums.
__device__ __forceinline__ void rf_load4(const void* rf, int rf_t, size_t i, float v[4])
{
    if (rf_t == RCA_F32) {
        float4 x = __ldcs(reinterpret_cast<const float4*>(reinterpret_cast<const float*>(rf) + i));
        v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
    } else if (rf_t == RCA_F16) {
        uint2 x = __ldcs(reinterpret_cast<const uint2*>(reinterpret_cast<const __half*>(rf) + i));
        float2 a = __half22float2(*reinterpret_cast<__half2*>(&x.x)), b = __half22float2(*reinterpret_cast<__half2*>(&x.y));
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    } else {
        uint2 x = __ldcs(reinterpret_cast<const uint2*>(reinterpret_cast<const int16_t*>(rf) + i));
        v[0] = (float)(short)(x.x & 0xffff); v[1] = (float)(short)(x.x >> 16);
        v[2] = (float)(short)(x.y & 0xffff); v[3] = (float)(short)(x.y >> 16);
    }
}

__device__ __forceinline__ void mean_body(int bx, const void* __restrict__ rf, int rf_t,
                                          const float* __restrict__ scale, int F, int ns, int ncol,
                                          float* __restrict__ mean)
{
    const int c4 = (bx * blockDim.x + threadIdx.x) * 4;
    if (c4 >= ncol) return;
    const size_t stride = (size_t)ncol;
    if (rf_t == RCA_I16 && F <= 65535) {
        // int16 samples summed exactly in 32-bit integers (|sum| < 65535 * 32768),
        // eight frames' loads in flight
        const int16_t* p = reinterpret_cast<const int16_t*>(rf) + c4;
        int qs[4] = {0, 0, 0, 0};
        int f = 0;
        for (; f + 8 <= F; f += 8) {
            uint2 x[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) x[u] = __ldcs(reinterpret_cast<const uint2*>(p + (size_t)(f + u) * stride));
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                qs[0] += (int)(short)(x[u].x & 0xffffu);
                qs[1] += (int)(short)(x[u].x >> 16);
                qs[2] += (int)(short)(x[u].y & 0xffffu);
                qs[3] += (int)(short)(x[u].y >> 16);
            }
        }
        for (; f < F; ++f) {
            const uint2 x = __ldcs(reinterpret_cast<const uint2*>(p + (size_t)f * stride));
            qs[0] += (int)(short)(x.x & 0xffffu);
            qs[1] += (int)(short)(x.x >> 16);
            qs[2] += (int)(short)(x.y & 0xffffu);
            qs[3] += (int)(short)(x.y >> 16);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int col = c4 + j;
            mean[col] = (float)((double)qs[j] / (double)F * (double)scale[col / ns]);
        }
        return;
    }
    float s[4] = {0.f, 0.f, 0.f, 0.f}, cmp[4] = {0.f, 0.f, 0.f, 0.f};
    long long qs[4] = {0, 0, 0, 0};
    int f = 0;
    for (; f + 4 <= F; f += 4) {
        float v[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u) rf_load4(rf, rf_t, (size_t)(f + u) * stride + c4, v[u]);
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (rf_t == RCA_I16) {
                    qs[j] += (long long)v[u][j];
                } else {
                    const float x = v[u][j], tt = s[j] + x;
                    cmp[j] += (fabsf(s[j]) >= fabsf(x)) ? ((s[j] - tt) + x) : ((x - tt) + s[j]);
                    s[j] = tt;
                }
            }
    }
    for (; f < F; ++f) {
        float v[4];
        rf_load4(rf, rf_t, (size_t)f * stride + c4, v);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (rf_t == RCA_I16) {
                qs[j] += (long long)v[j];
            } else {
                const float x = v[j], tt = s[j] + x;
                cmp[j] += (fabsf(s[j]) >= fabsf(x)) ? ((s[j] - tt) + x) : ((x - tt) + s[j]);
                s[j] = tt;
            }
        }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int col = c4 + j;
        mean[col] = (rf_t == RCA_I16) ? (float)((double)qs[j] / (double)F * (double)scale[col / ns])
                                      : (s[j] + cmp[j]) / (float)F;
    }
}

#define DM_NT 128           // samples per CTA
#define DM_NE 32            // elements per CTA
#define DM_PITCH (DM_NT + 31)  // odd float2 pitch: conflict-free column reads

// CTA = (128 samples, 32 elements, one frame-transmission).  Reads RF rows
// [e][n] coalesced along n (warps over elements, lanes over samples), writes
// IQ [n][e] coalesced along e (lanes over elements).  Each thread filters
// DM_OB consecutive samples of one element from a register window, so every
// staged sample is read DM_OB + 30 times per DM_OB outputs instead of 17 times
// per output.
#define DM_OB 16            // consecutive outputs per thread
// four consecutive channel samples n .. n + 3 (n a multiple of 4) as floats
template <int RT>
__device__ __forceinline__ float4 rf_quad(const void* __restrict__ rf, size_t i)
{
    if constexpr (RT == RCA_F32) {
        return __ldg(reinterpret_cast<const float4*>(reinterpret_cast<const float*>(rf) + i));
    } else if constexpr (RT == RCA_F16) {
        const uint2 x = __ldg(reinterpret_cast<const uint2*>(reinterpret_cast<const __half*>(rf) + i));
        const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&x.x));
        const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&x.y));
        return make_float4(a.x, a.y, b.x, b.y);
    } else {
        const uint2 x = __ldg(reinterpret_cast<const uint2*>(reinterpret_cast<const int16_t*>(rf) + i));
        return make_float4((float)(short)(x.x & 0xffff), (float)(short)(x.x >> 16), (float)(short)(x.y & 0xffff),
                           (float)(short)(x.y >> 16));
    }
}

template <int RT>
__device__ __forceinline__ void demod_body(int bx, int by, int bz, float2* __restrict__ xs,
                                           const void* __restrict__ rf, const float* __restrict__ scale,
                                           const float* __restrict__ mean, const float2* __restrict__ mix,
                                           const Fir& fir, int nt, int E, int ns, void* __restrict__ iq, int iq_t)
{
    constexpr int rf_t = RT;
    const int n0 = bx * DM_NT;
    const int e0 = by * DM_NE;
    const int fk = bz;
    const int k = fk % nt;
    const size_t chan0 = (size_t)fk * E;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    // stage (rf - mean) * exp(-j 2 pi fc t_n) for samples n0-15 .. n0+DM_NT+14
    const bool quads = (ns & 3) == 0 && (reinterpret_cast<uintptr_t>(rf) & 15) == 0 &&
                       (reinterpret_cast<uintptr_t>(mean) & 15) == 0;
    if (quads) {
        // whole aligned quads n0-16+4q .. n0-13+4q (q < NQ): each inside or outside [0, ns).
        // Items (element, quad) in blocks of 4 elements x 4 quads per 16 consecutive
        // threads: a half-warp's four stores of sample j then hit 16 different bank
        // pairs (element rows 159 = 15 mod 16 float2 apart, quads 4 apart), and
        // its loads are four 64-byte runs.  Two items per thread in flight: both
        // items' loads are issued before either is converted and stored.
        constexpr int NQ = (DM_NT + 32) / 4;
        constexpr int ITEMS = DM_NE * NQ;
        static_assert(NQ % 4 == 0 && DM_NE % 4 == 0, "4 x 4 item blocks");
        auto item = [](int idx, int& el, int& q) {
            const int grp = idx >> 4, sub = idx & 15;
            el = (grp % (DM_NE / 4)) * 4 + (sub >> 2);
            q = (grp / (DM_NE / 4)) * 4 + (sub & 3);
        };
        for (int i0 = threadIdx.x; i0 < ITEMS; i0 += 2 * blockDim.x) {
            float4 r[2], mu[2], ma[2], mb[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int idx = i0 + u * blockDim.x;
                int el, q;
                item(idx, el, q);
                const int e = e0 + el, nb = n0 - 16 + 4 * q;
                r[u] = mu[u] = ma[u] = mb[u] = make_float4(0.f, 0.f, 0.f, 0.f);
                if (idx < ITEMS && nb >= 0 && nb < ns && e < E) {
                    r[u] = rf_quad<RT>(rf, (chan0 + e) * ns + nb);
                    if (mean) mu[u] = __ldg(reinterpret_cast<const float4*>(mean + ((size_t)k * E + e) * ns + nb));
                    ma[u] = __ldg(reinterpret_cast<const float4*>(mix + nb));
                    mb[u] = __ldg(reinterpret_cast<const float4*>(mix + nb + 2));
                }
            }
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int idx = i0 + u * blockDim.x;
                if (idx >= ITEMS) continue;
                int el, q;
                item(idx, el, q);
                const int e = e0 + el;
                const float sc = (rf_t == RCA_I16 && e < E) ? scale[k * E + e] : 1.f;
                const float x0 = r[u].x * sc - mu[u].x, x1 = r[u].y * sc - mu[u].y;
                const float x2 = r[u].z * sc - mu[u].z, x3 = r[u].w * sc - mu[u].w;
                const float2 v[4] = {make_float2(x0 * ma[u].x, x0 * ma[u].y), make_float2(x1 * ma[u].z, x1 * ma[u].w),
                                     make_float2(x2 * mb[u].x, x2 * mb[u].y), make_float2(x3 * mb[u].z, x3 * mb[u].w)};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int sidx = 4 * q - 1 + j;
                    if (sidx >= 0 && sidx < DM_NT + 30) xs[el * DM_PITCH + sidx] = v[j];
                }
            }
        }
    } else {
        for (int el = warp; el < DM_NE; el += nwarp) {
            const int e = e0 + el;
            const float sc = (rf_t == RCA_I16 && e < E) ? scale[k * E + e] : 1.f;
            const float* mrow = mean ? mean + ((size_t)k * E + e) * ns : nullptr;
            for (int sidx = lane; sidx < DM_NT + 30; sidx += 32) {
                const int n = n0 - 15 + sidx;
                float2 v = make_float2(0.f, 0.f);
                if (n >= 0 && n < ns && e < E) {
                    float x = rf_value(rf, rf_t, (chan0 + e) * ns + n) * sc;
                    if (mrow) x -= mrow[n];
                    const float2 m = mix[n];
                    v = make_float2(x * m.x, x * m.y);
                }
                xs[el * DM_PITCH + sidx] = v;
            }
        }
    }
    __syncthreads();
    // half-band low-pass x2: out[n] = 2 (h15 x[n] + sum_{odd m} h[15+m] (x[n-m] + x[n+m])).
    // Each staged sample is read once and added into the DM_OB outputs it feeds.
    uint64_t hp[16];                                  // 2 h[15 + d], d = 0 .. 15 (even d > 0 are zero)
#pragma unroll
    for (int d = 0; d < 16; ++d) hp[d] = f2_pack(2.f * fir.h[15 + d], 2.f * fir.h[15 + d]);
    const int e = e0 + lane;
    const unsigned row = smem_u32(xs + lane * DM_PITCH);
    for (int ob = warp; ob < DM_NT / DM_OB; ob += nwarp) {
        const int s0 = ob * DM_OB;                    // output o sits at window sample o + 15
        uint64_t acc[DM_OB];
#pragma unroll
        for (int o = 0; o < DM_OB; ++o) acc[o] = 0ull;
#pragma unroll
        for (int j = 0; j < DM_OB + 30; ++j) {
            const uint64_t w = lds_u64(row + (unsigned)((s0 + j) * 8));
#pragma unroll
            for (int o = 0; o < DM_OB; ++o) {
                const int d = j - o - 15 < 0 ? o + 15 - j : j - o - 15;
                if (d <= 15 && (d == 0 || (d & 1))) acc[o] = f2_fma(hp[d], w, acc[o]);
            }
        }
        if (e >= E) continue;
#pragma unroll
        for (int o = 0; o < DM_OB; ++o) {
            const int n = n0 + s0 + o;
            if (n < ns) store_c(iq, ((size_t)fk * ns + n) * E + e, iq_t, f2_unpack(acc[o]));
        }
    }
}


// ---------------------------------------------------------------------------
// Stage 1: reference slices
//   S_k(l, r) = sum_d W[r][d] (IQ_{k, l-d}(xi) + IQ_{k, l+d}(xi)),  (d = 0 once)
//   xi = (tx_q16[k][r] + rx_q16[r][d]) / 2^16 samples.
// For a fixed (r, d) the sample position is the same for every lateral pixel,
// so each warp (32 consecutive pixels) reads 32 consecutive elements of one
// sample row of the [ns][E] IQ block: the delay, its fraction and the weight
// are warp-uniform and are precomputed per (row, d) once per chunk.  The
// linear interpolation is folded into the weights and the two mirror
// elements are summed before the complex multiply:
//   term = a (IQ_{l-d}[n] + IQ_{l+d}[n]) + b (IQ_{l-d}[n+1] + IQ_{l+d}[n+1]),
//   a = w (1 - fr),  b = w fr   (both halved at d = 0, where the two
//   elements coincide).
// The chunk's sample window is one contiguous block of the IQ array, fetched
// by a TMA bulk copy into a double buffer while the previous chunk is
// processed.  Each warp splits its lateral distances into ranges where the
// mirror element l - d (and l + d) exists for all of its lanes, for some of
// them (predicated loads) or for none (skipped), so full ranges run without
// predicates and no shared-memory bandwidth goes to lanes with nothing to add.
// A thread owns MAXR consecutive slice rows; the per-(d, row) records are
// stored d-major so that its rows sit at fixed offsets from one address.
// ---------------------------------------------------------------------------
// per-(d, row) weights, 16 bytes.  FP32 arithmetic: Re a, Re b, Im a, Im b
// as floats, with the byte offset of the window row in a separate array.
// FP16 arithmetic: {Re a, Re b} and {Im a, Im b} as half pairs, then the
// row offset.
template <typename TS>
struct S1Rec {
    static constexpr bool HALF = std::is_same<TS, __half2>::value;
    static constexpr int BYTES = 16;
};

// one complex sample as a packed float pair (FP32 arithmetic)
template <typename TS>
__device__ __forceinline__ uint64_t s1_ld(unsigned addr);
template <>
__device__ __forceinline__ uint64_t s1_ld<float2>(unsigned addr) { return lds_u64(addr); }
template <>
__device__ __forceinline__ uint64_t s1_ld<__nv_bfloat162>(unsigned addr)
{
    const unsigned u = lds_u32(addr);
    // bf16 -> f32 is a 16-bit shift of each half
    return f2_pack(__uint_as_float(u << 16), __uint_as_float(u & 0xffff0000u));
}

__device__ __forceinline__ unsigned h2_add(unsigned a, unsigned b)
{
    unsigned d;
    asm("add.rn.f16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}

__device__ __forceinline__ void lds_u32x4(unsigned addr, unsigned& a, unsigned& b, unsigned& c, unsigned& d)
{
    asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];" : "=r"(a), "=r"(b), "=r"(c), "=r"(d) : "r"(addr));
}

// FP16 samples, FP32 accumulators: A1 += Re a * s0 + Re b * s1, A2 += Im a * s0 + Im b * s1
// with mixed-precision FMAs (f16 x f16 + f32), s0 / s1 packed {re, im} halves.
__device__ __forceinline__ void s1_mfma(float& a1x, float& a1y, float& a2x, float& a2y, unsigned wr, unsigned wi,
                                        unsigned s0, unsigned s1)
{
    asm("{\n\t.reg .f16 ar, br, ai, bi, s0r, s0i, s1r, s1i;\n\t"
        "mov.b32 {ar, br}, %4;\n\t"
        "mov.b32 {ai, bi}, %5;\n\t"
        "mov.b32 {s0r, s0i}, %6;\n\t"
        "mov.b32 {s1r, s1i}, %7;\n\t"
        "fma.rn.f32.f16 %0, ar, s0r, %0;\n\t"
        "fma.rn.f32.f16 %0, br, s1r, %0;\n\t"
        "fma.rn.f32.f16 %1, ar, s0i, %1;\n\t"
        "fma.rn.f32.f16 %1, br, s1i, %1;\n\t"
        "fma.rn.f32.f16 %2, ai, s0r, %2;\n\t"
        "fma.rn.f32.f16 %2, bi, s1r, %2;\n\t"
        "fma.rn.f32.f16 %3, ai, s0i, %3;\n\t"
        "fma.rn.f32.f16 %3, bi, s1i, %3;\n\t}"
        : "+f"(a1x), "+f"(a1y), "+f"(a2x), "+f"(a2y)
        : "r"(wr), "r"(wi), "r"(s0), "r"(s1));
}

enum { S1_NONE = 0, S1_FULL = 1, S1_PRED = 2 };

// One pixel's update for one (row, d) record: A = {A1.x, A1.y, A2.x, A2.y}
// += the folded term of the mirror elements at window offsets ox (l - d) and
// oy (l + d), sample rows at `row` and row + RS.  Modes XM / YM and the
// per-lane predicates hx / hy say which of the two elements exist.
// HALF: r0 / r1 = {Re a, Re b} / {Im a, Im b} half pairs; else r0..r3 =
// Re a, Re b, Im a, Im b as floats.
template <typename TS, int XM, int YM>
__device__ __forceinline__ void s1_pixel(float (&A)[4], unsigned row, unsigned ox, unsigned oy, int RS, bool hx,
                                         bool hy, unsigned r0, unsigned r1, unsigned r2, unsigned r3)
{
    if constexpr (S1Rec<TS>::HALF) {
        unsigned x0 = 0u, x1 = 0u, y0 = 0u, y1 = 0u;
        if (XM != S1_NONE && hx) {
            x0 = lds_u32(row + ox);
            x1 = lds_u32(row + ox + RS);
        }
        if (YM != S1_NONE && hy) {
            y0 = lds_u32(row + oy);
            y1 = lds_u32(row + oy + RS);
        }
        unsigned s0, s1;
        if constexpr (XM == S1_NONE) {
            s0 = y0;
            s1 = y1;
        } else if constexpr (YM == S1_NONE) {
            s0 = x0;
            s1 = x1;
        } else {
            s0 = h2_add(x0, y0);
            s1 = h2_add(x1, y1);
        }
        s1_mfma(A[0], A[1], A[2], A[3], r0, r1, s0, s1);
    } else {
        uint64_t x0 = 0ull, x1 = 0ull, y0 = 0ull, y1 = 0ull;
        if (XM != S1_NONE && hx) {
            x0 = s1_ld<TS>(row + ox);
            x1 = s1_ld<TS>(row + ox + RS);
        }
        if (YM != S1_NONE && hy) {
            y0 = s1_ld<TS>(row + oy);
            y1 = s1_ld<TS>(row + oy + RS);
        }
        uint64_t s0, s1;
        if constexpr (XM == S1_NONE) {
            s0 = y0;
            s1 = y1;
        } else if constexpr (YM == S1_NONE) {
            s0 = x0;
            s1 = x1;
        } else {
            s0 = f2_add(x0, y0);
            s1 = f2_add(x1, y1);
        }
        const float2 u = f2_unpack(s0), v = f2_unpack(s1);
        const float fax = __uint_as_float(r0), fbx = __uint_as_float(r1);
        const float fay = __uint_as_float(r2), fby = __uint_as_float(r3);
        A[0] = fmaf(fax, u.x, fmaf(fbx, v.x, A[0]));
        A[1] = fmaf(fax, u.y, fmaf(fbx, v.y, A[1]));
        A[2] = fmaf(fay, u.x, fmaf(fby, v.x, A[2]));
        A[3] = fmaf(fay, u.y, fmaf(fby, v.y, A[3]));
    }
}

// One range [d0, d1) of lateral distances with fixed modes for the two mirror
// elements: S1_FULL (every lane has the element), S1_PRED (some do: the others
// load zeros), S1_NONE (no lane does: skipped).  nrow: rows of this thread
// (MAXR when EXACT).  H[j] = {A1.x, A1.y, A2.x, A2.y}: sums of the
// Re-weight and Im-weight products of row j for pixel l.
// PAIR: the thread also owns the mirror pixel m = N - 1 - l, whose elements
// m - d and m + d exist exactly when l + d and l - d do, so it runs in the
// same range with the modes swapped and accumulates into G; each record read
// then serves both pixels.
template <typename TS, int MAXR, bool EXACT, bool PAIR, int XM, int YM>
__device__ __forceinline__ void stage1_range(float (&H)[MAXR][4], float (&G)[MAXR][4], int d0, int d1, int cz, int zt,
                                             int l, int m, int Lx, int Ly, int row0, int nrow, unsigned rbase,
                                             unsigned obase, unsigned wbase, int RS, int dc, unsigned rmax,
                                             unsigned* __restrict__ status)
{
    constexpr bool HALF = S1Rec<TS>::HALF;
    constexpr int RB = S1Rec<TS>::BYTES, ESZ = (int)sizeof(TS);
#pragma unroll 1
    for (int d = d0; d < d1; ++d) {
        if (!chk(d - cz >= 0 && d - cz < dc, status)) break;   // record block of the chunk
        const bool hx = XM == S1_FULL || (XM == S1_PRED && d <= Lx);
        const bool hy = YM == S1_FULL || (YM == S1_PRED && d <= Ly);
        // window offsets of the two mirror elements (records hold the row offset)
        const unsigned ox = wbase + (unsigned)((l - d) * ESZ), oy = wbase + (unsigned)((l + d) * ESZ);
        const unsigned mx = wbase + (unsigned)((m - d) * ESZ), my = wbase + (unsigned)((m + d) * ESZ);
        const int base = (d - cz) * zt + row0;    // record index of the thread's first row
        const unsigned rp = rbase + base * RB, op = obase + base * 4;
        unsigned rowq[4];
#pragma unroll
        for (int j = 0; j < MAXR; ++j) {
            if (EXACT || j < nrow) {
                unsigned r0, r1, r2, r3, row;
                if constexpr (HALF) {
                    lds_u32x4(rp + j * RB, r0, r1, row, r3);
                    r2 = 0u;
                } else {
                    lds_u32x4(rp + j * RB, r0, r1, r2, r3);
                    // row addresses of four consecutive rows in one load (16-byte
                    // aligned: the thread's first row and zt are multiples of 4)
                    constexpr bool QUAD = EXACT && MAXR >= 4;
                    if (!QUAD || (j & 3) == 0) {
                        if constexpr (QUAD)
                            lds_u32x4(op + j * 4, rowq[0], rowq[1], rowq[2], rowq[3]);
                        else
                            rowq[0] = lds_u32(op + j * 4);
                    }
                    // FP32-weight records hold offsets for 8-byte samples: halve for 4-byte ones
                    row = rowq[QUAD ? (j & 3) : 0] >> (ESZ == 4 ? 1 : 0);
                }
                // the two sample rows read lie inside the ring: row <= (ring - 1) RS
                if (!chk(row <= rmax, status)) continue;
                s1_pixel<TS, XM, YM>(H[j], row, ox, oy, RS, hx, hy, r0, r1, r2, r3);
                if constexpr (PAIR) s1_pixel<TS, YM, XM>(G[j], row, mx, my, RS, hy, hx, r0, r1, r2, r3);
            }
        }
    }
}

// Returns false if a bounded wait ran out (the CTA must stop).  The thread
// owns rows [rg * per, rg * per + per) of the tile, per = ceil(zt / RG)
// (per <= MAXR; EXACT: per == MAXR and zt == RG * MAXR, or MAXR == 1), and
// pixel l (plus N - 1 - l when PAIR).
// rtab: the plan's record table for this arithmetic (FP16 weights for FP16
// samples, FP32 weights otherwise), one block of rblk bytes per chunk.
template <typename TS, int MAXR, bool EXACT, bool PAIR = false>
__device__ __forceinline__ bool stage1_body(int tile, int k, int f, unsigned char* __restrict__ smraw,
                                            uint64_t* bars, const GeomDev& g, const void* __restrict__ iq,
                                            const unsigned char* __restrict__ rtab, int rblk,
                                            const int* __restrict__ dmax, const int4* __restrict__ chunks, int zt,
                                            int dc, int n_tiles, int nch, int ring, float2* __restrict__ slices,
                                            unsigned* __restrict__ status)
{
    constexpr int ESZ = (int)sizeof(TS);
    const int E = g.N, N = g.N;
    const int RS = E * ESZ;                                   // sample row (bytes)
    unsigned char* rng = smraw;                               // [ring + 1][RS]
    unsigned char* recs = rng + (size_t)(ring + 1) * RS;      // [2][rblk]
    const int nt = 2 * g.K;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int LW = PAIR ? N >> 6 : (N + 31) >> 5;
    const int RG = (blockDim.x >> 5) / LW;
    const int lw = warp % LW, rg = warp / LW;
    const int lb = lw * 32;
    const int l = lb + lane;
    const int m = N - 1 - l;                                   // mirror pixel (PAIR)
    const int per = (zt + RG - 1) / RG;
    const int row0 = rg * per;                                 // first tile row of this thread
    const int nrow = max(0, min(per, zt - row0));
    const int r0 = tile * zt;
    const int rend = min(r0 + zt, g.nzs);
    const int4* ch = chunks + ((size_t)k * n_tiles + tile) * nch;
    const unsigned char* rsrc = rtab + ((size_t)k * n_tiles + tile) * nch * rblk;
    const unsigned char* blk = reinterpret_cast<const unsigned char*>(iq) + ((size_t)f * nt + k) * g.ns * RS;
    // largest (aperture limit + 1) over this thread's rows: its distance count in a chunk
    int dmx = 0;
    for (int j = 0; j < nrow; ++j)
        if (r0 + row0 + j < rend) dmx = max(dmx, __ldg(dmax + r0 + row0 + j) + 1);

    if (threadIdx.x == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        mbar_fence_init();
    }
    __syncthreads();

    // fetch the rows of chunk c that are not resident: [a, a + cnt) into ring
    // slots sa.. (wrapping to slot 0 after c1 rows); rows outside [0, ns) are
    // zeroed by all threads, the rest bulk-copied by thread 0 with the
    // chunk's record block on one barrier.  The row in slot 0 is also
    // written to slot `ring`.
    auto issue = [&](int c, int b) {
        const int4 cc = ch[c];
        const int a = cc.x, cnt = cc.y & 0xffff, sa = cc.y >> 16;
        const int c1 = min(cnt, ring - sa);
        const int v16 = RS / 16;
        if (a < 0 || a + cnt > g.ns) {
            for (int idx = threadIdx.x; idx < cnt * v16; idx += blockDim.x) {
                const int q = idx / v16, u = idx - q * v16, n = a + q;
                if (n >= 0 && n < g.ns) continue;
                const int sl = q < c1 ? sa + q : q - c1;
                if (!chk(sl >= 0 && sl <= ring, status)) continue;
                reinterpret_cast<uint4*>(rng + (size_t)sl * RS)[u] = make_uint4(0u, 0u, 0u, 0u);
                if (sl == 0) reinterpret_cast<uint4*>(rng + (size_t)ring * RS)[u] = make_uint4(0u, 0u, 0u, 0u);
            }
        }
        if (threadIdx.x == 0) {
            fence_proxy_async();
            // in-sample parts of the two runs, and the row that lands in slot 0
            const int lo1 = max(a, 0), hi1 = max(lo1, min(a + c1, g.ns));
            const int lo2 = max(a + c1, 0), hi2 = max(lo2, min(a + cnt, g.ns));
            const int n0 = c1 < cnt ? a + c1 : (sa == 0 && cnt > 0 ? a : -1);
            const bool dup = n0 >= 0 && n0 < g.ns;
            // both runs land inside slots [0, ring): the first from slot sa, the second from slot 0
            if (!chk(sa >= 0 && (hi1 <= lo1 || sa + hi1 - a <= ring) && (hi2 <= lo2 || hi2 - (a + c1) <= ring) &&
                         c >= 0 && c < nch, status)) {
                // nothing is copied; the phase completes at once (results invalid, status set)
                mbar_arrive_expect_tx(&bars[b], 0u);
                return;
            }
            const unsigned bytes = (unsigned)((hi1 - lo1) + (hi2 - lo2) + (dup ? 1 : 0)) * (unsigned)RS;
            mbar_arrive_expect_tx(&bars[b], bytes + (unsigned)rblk);
            if (hi1 > lo1)
                bulk_g2s(rng + (size_t)(sa + lo1 - a) * RS, blk + (size_t)lo1 * RS, (unsigned)((hi1 - lo1) * RS),
                         &bars[b]);
            if (hi2 > lo2)
                bulk_g2s(rng + (size_t)(lo2 - (a + c1)) * RS, blk + (size_t)lo2 * RS, (unsigned)((hi2 - lo2) * RS),
                         &bars[b]);
            if (dup) bulk_g2s(rng + (size_t)ring * RS, blk + (size_t)n0 * RS, (unsigned)RS, &bars[b]);
            bulk_g2s(recs + (size_t)b * rblk, rsrc + (size_t)c * rblk, (unsigned)rblk, &bars[b]);
        }
    };

    // H[j] = {A1.x, A1.y, A2.x, A2.y} of pixel l (G[j]: of pixel m);
    // slice value = (A1.x - A2.y, A1.y + A2.x)
    float H[MAXR][4], G[MAXR][4];
#pragma unroll
    for (int j = 0; j < MAXR; ++j) {
        H[j][0] = H[j][1] = H[j][2] = H[j][3] = 0.f;
        G[j][0] = G[j][1] = G[j][2] = G[j][3] = 0.f;
    }
    // per-lane reach of the mirror elements: l - d needs d <= Lx, l + d needs d <= Ly
    // (for the mirror pixel m the two swap: m - d needs d <= Ly, m + d needs d <= Lx)
    const int Lx = l < N ? l : -1;
    const int Ly = N - 1 - l;
    // warp-uniform range limits: x (e = l - d) for every lane up to xf, for some up to xe;
    // y (e = l + d) for every lane up to yf, for some up to ye
    const int xf = lb + 31 < N ? lb : -1, xe = min(lb + 31, N - 1);
    const int yf = N - 32 - lb, ye = N - 1 - lb;
    unsigned phase = 0;
    issue(0, 0);
    for (int c = 0; c < nch; ++c) {
        const int b = c & 1;
        const int4 cc = ch[c];
        if (!cta_wait_copies(&bars[b], (phase >> b) & 1u, status)) return false;
        phase ^= 1u << b;
        if (c + 1 < nch) issue(c + 1, b ^ 1);
        if (cc.w <= cc.z || nrow == 0) continue;
        const unsigned wbase = smem_u32(rng);
        const unsigned rbase = smem_u32(recs + (size_t)b * rblk);
        const unsigned obase = rbase + (unsigned)(zt * dc * 16);
        // the thread's rows advance together: each d step updates its rows'
        // independent accumulators (records past a row's aperture have zero weights)
        const int ndw = max(0, min(cc.w, dmx) - cc.z);
        const int dend = cc.z + min(ndw, max(xe, ye) - cc.z + 1);
        for (int d = cc.z; d < dend;) {
            const int xm = d <= xf ? S1_FULL : (d <= xe ? S1_PRED : S1_NONE);
            const int ym = d <= yf ? S1_FULL : (d <= ye ? S1_PRED : S1_NONE);
            int nx = dend;
            if (xf + 1 > d) nx = min(nx, xf + 1);
            if (xe + 1 > d) nx = min(nx, xe + 1);
            if (yf + 1 > d) nx = min(nx, yf + 1);
            if (ye + 1 > d) nx = min(nx, ye + 1);
#define RCA_S1_RANGE(XM, YM)                                                                                     \
    stage1_range<TS, MAXR, EXACT, PAIR, XM, YM>(H, G, d, nx, cc.z, zt, l, m, Lx, Ly, row0, nrow, rbase, obase, wbase, \
                                                RS, dc, (unsigned)((ring - 1) * RS), status)
            switch (xm * 3 + ym) {
            case S1_FULL * 3 + S1_FULL: RCA_S1_RANGE(S1_FULL, S1_FULL); break;
            case S1_FULL * 3 + S1_PRED: RCA_S1_RANGE(S1_FULL, S1_PRED); break;
            case S1_FULL * 3 + S1_NONE: RCA_S1_RANGE(S1_FULL, S1_NONE); break;
            case S1_PRED * 3 + S1_FULL: RCA_S1_RANGE(S1_PRED, S1_FULL); break;
            case S1_PRED * 3 + S1_PRED: RCA_S1_RANGE(S1_PRED, S1_PRED); break;
            case S1_PRED * 3 + S1_NONE: RCA_S1_RANGE(S1_PRED, S1_NONE); break;
            case S1_NONE * 3 + S1_FULL: RCA_S1_RANGE(S1_NONE, S1_FULL); break;
            case S1_NONE * 3 + S1_PRED: RCA_S1_RANGE(S1_NONE, S1_PRED); break;
            default: break;
            }
#undef RCA_S1_RANGE
            d = nx;
        }
    }
    float2* out = slices + ((size_t)f * nt + k) * g.nzs * N;
#pragma unroll
    for (int j = 0; j < MAXR; ++j) {
        const int r = r0 + row0 + j;
        if ((EXACT || j < nrow) && r < rend && l < N) {
            out[(size_t)r * N + l] = make_float2(H[j][0] - H[j][3], H[j][1] + H[j][2]);
            if (PAIR) out[(size_t)r * N + m] = make_float2(G[j][0] - G[j][3], G[j][1] + G[j][2]);
        }
    }
    return true;
}

// ---------------------------------------------------------------------------
// Stage 2 + block sum-projection, written straight to the planes.
// For a family, the "transverse-slab" plane sums over the transverse
// coordinate u inside slab b: each u shifts the slice by its own dz_k(u), so
// the per-(k, b) sum of P linear interpolations is a short filter along the
// slice rows.  Its taps are the same for every plane row up to the row's
// carrier, coef[k][b][i][t] = ec[k][i] c2[k][b][t], except in the few rows
// near the slice ends where a shifted row leaves the slice (there the exact
// per-row taps are used).  The "lateral-slab" plane sums over lateral pixels
// inside slab b: the shift does not depend on the lateral pixel, so the
// slice is first summed over the slab and interpolated once per u.
// RC: transverse = y -> XZ planes (axis 0), lateral-slab -> YZ (axis 1).
// CR: transverse = x -> YZ planes (axis 1), lateral-slab -> XZ (axis 0).
// A CTA covers one frame and family, up to S2_ZP plane rows and one group of
// GW lateral pixels: it stages the group's slice columns for all K
// transmissions, then its warps write the transverse-slab planes of every
// slab at those pixels and the lateral-slab planes of the group's slabs at
// every u, S2_RH plane rows per warp task.
// ---------------------------------------------------------------------------
#define S2_RH 8        // plane rows per warp task

// Streaming stores of n (<= S2_RH) plane values at ob, ob + N, ...: the
// dtype is chosen once for the group.
__device__ __forceinline__ void s2_store_rows(void* __restrict__ planes, int pt, size_t ob, int N, const float2* v,
                                              int n)
{
    if (pt == RCA_C32) {
        float2* p = reinterpret_cast<float2*>(planes) + ob;
#pragma unroll
        for (int q = 0; q < S2_RH; ++q)
            if (q < n) __stcs(p + (size_t)q * N, v[q]);
    } else if (pt == RCA_C16F) {
        unsigned* p = reinterpret_cast<unsigned*>(planes) + ob;
#pragma unroll
        for (int q = 0; q < S2_RH; ++q) {
            if (q < n) {
                __half2 hv = __float22half2_rn(v[q]);
                __stcs(p + (size_t)q * N, *reinterpret_cast<unsigned*>(&hv));
            }
        }
    } else {
        unsigned* p = reinterpret_cast<unsigned*>(planes) + ob;
#pragma unroll
        for (int q = 0; q < S2_RH; ++q) {
            if (q < n) {
                __nv_bfloat162 bv = __float22bfloat162_rn(v[q]);
                __stcs(p + (size_t)q * N, *reinterpret_cast<unsigned*>(&bv));
            }
        }
    }
}

// Complex products on packed FP32 pairs: with a complex coefficient c held as
// (c.re, c.re) and (c.im, c.im), A1 += (c.re, c.re) * v and A2 += (c.im, c.im) * v
// give c v = (A1.x - A2.y, A1.y + A2.x) after any number of terms.
__device__ __forceinline__ uint64_t s2_join(uint64_t A1, uint64_t A2)
{
    const float2 p1 = f2_unpack(A1), p2 = f2_unpack(A2);
    return f2_pack(p1.x - p2.y, p1.y + p2.x);
}

// transverse-slab plane rows [q0, q0 + S2_RH) of slab b at lateral pixel g0 + lane.
// TT: tap count (0: t->T at run time, up to 16); US: slice rows per plane row
// (0: g.us at run time).  INTERIOR: every row of the tile has
// carrier-separable taps.  With TT and US fixed, the rows of consecutive
// plane rows overlap by TT - US and are loaded once.
template <int TT, int US, bool INTERIOR>
__device__ __forceinline__ void s2_transverse(int b, int q0, int nrow, int ia, int ib, int lane, int gw, int fam,
                                              int f, int i0, int axT, const GeomDev& g, int T, int rows,
                                              const uint64_t* __restrict__ sS64, const uint64_t* __restrict__ sC2q,
                                              const int* __restrict__ sTb, const float2* __restrict__ coef,
                                              void* __restrict__ planes, int pt, int g0, unsigned* __restrict__ status)
{
    const int K = g.K, S = g.S, N = g.N;
    const int us = US > 0 ? US : g.us;
    constexpr int TMX = TT > 0 ? TT : 16;
    const int nT = TT > 0 ? TT : T;
    // the slices are carrier-rotated, so the taps carry each row's carrier:
    // the sum over transmissions and taps accumulates straight into
    // out = (O1.x - O2.y, O1.y + O2.x)
    uint64_t O1[S2_RH], O2[S2_RH];
#pragma unroll
    for (int q = 0; q < S2_RH; ++q) O1[q] = O2[q] = 0ull;
    const int qlast = min(q0 + S2_RH, nrow) - 1;       // last plane row of the task read below
    for (int kk = 0; kk < K; ++kk) {
        const int tb = sTb[kk * S + b];
        if (!chk(tb >= 0 && tb + us * qlast + nT - 1 < rows, status)) continue;   // staged window rows
        // this lane's column in transmission kk from the window row of plane row q0
        const uint64_t* col = sS64 + (size_t)(kk * rows + tb + us * q0) * 32 + lane;
        const uint64_t* cp = sC2q + 2 * (size_t)(kk * S + b) * T;
        if constexpr (TT > 0 && US > 0 && INTERIOR) {
            uint64_t cx[TT], cy[TT], v[TT];
#pragma unroll
            for (int t = 0; t < TT; ++t) {
                cx[t] = cp[2 * t];
                cy[t] = cp[2 * t + 1];
                v[t] = col[t * 32];
            }
#pragma unroll
            for (int q = 0; q < S2_RH; ++q) {
                if (q > 0) {
#pragma unroll
                    for (int t = 0; t < TT; ++t) v[t] = t + US < TT ? v[t + US] : col[(US * q + t) * 32];
                }
#pragma unroll
                for (int t = 0; t < TT; ++t) {
                    O1[q] = f2_fma(cx[t], v[t], O1[q]);
                    O2[q] = f2_fma(cy[t], v[t], O2[q]);
                }
            }
        } else {
            // taps read per use (a run-time tap count would hold up to 32 coefficient registers)
#pragma unroll
            for (int q = 0; q < S2_RH; ++q) {
                const int ii = q0 + q;
                if (INTERIOR || (ii >= ia && ii < ib)) {
#pragma unroll
                    for (int t = 0; t < TMX; ++t) {
                        if (TT > 0 || t < nT) {
                            const uint64_t v = col[(us * q + t) * 32];
                            O1[q] = f2_fma(cp[2 * t], v, O1[q]);
                            O2[q] = f2_fma(cp[2 * t + 1], v, O2[q]);
                        }
                    }
                } else if (ii < nrow) {
                    // rows near the slice ends: exact per-row taps (carrier included)
                    const float2* cf = coef + (((size_t)(fam * K + kk) * S + b) * g.nz + i0 + ii) * T;
                    float2 y = make_float2(0.f, 0.f);
                    for (int t = 0; t < T; ++t) {
                        const float2 sv = f2_unpack(col[(us * q + t) * 32]);
                        cfma(y, __ldg(cf + t), sv);
                    }
                    O1[q] = f2_add(O1[q], f2_pack(y.x, y.y));
                }
            }
        }
    }
    if (lane < gw) {
        const size_t plane_sz = (size_t)g.nz * N;
        const size_t ob = ((((size_t)f * 2 + axT) * 2 + fam) * S + b) * plane_sz + (size_t)(i0 + q0) * N + g0 + lane;
        float2 v[S2_RH];
#pragma unroll
        for (int q = 0; q < S2_RH; ++q) v[q] = f2_unpack(s2_join(O1[q], O2[q]));
        s2_store_rows(planes, pt, ob, N, v, INTERIOR ? S2_RH : min(S2_RH, nrow - q0));
    }
}

// lateral-slab plane rows [q0, q0 + S2_RH) of group slab sb at transverse position u
template <int US, bool INTERIOR>
__device__ __forceinline__ void s2_lateral(int sb, int u, int q0, int nrow, int ia, int ib, int fam, int f, int i0,
                                           int axL, int rlo, int grp, int SG, const GeomDev& g, int rows,
                                           const float4* __restrict__ sLw, const int* __restrict__ sSh,
                                           const uint64_t* __restrict__ sSum64, const float* __restrict__ sfr,
                                           void* __restrict__ planes, int pt, unsigned* __restrict__ status)
{
    const int K = g.K, S = g.S, N = g.N;
    const int us = US > 0 ? US : g.us;
    uint64_t O1[S2_RH], O2[S2_RH];
#pragma unroll
    for (int q = 0; q < S2_RH; ++q) O1[q] = O2[q] = 0ull;
#pragma unroll 2
    for (int kk = 0; kk < K; ++kk) {
        const float4 w = sLw[kk * N + u];            // a, b: interpolation weights with the carrier folded in
        const uint64_t ax = f2_pack(w.x, w.x), ay = f2_pack(w.y, w.y);
        const uint64_t bx = f2_pack(w.z, w.z), by = f2_pack(w.w, w.w);
        const int sh = sSh[kk * N + u];
        // the two slab-sum rows of the task's plane rows lie inside the window
        if (!chk(sh >= 0 && sh + us * (min(q0 + S2_RH, nrow) - 1) + 1 < rows, status)) continue;
        const float fr = INTERIOR ? 0.f : __ldg(sfr + (size_t)(fam * K + kk) * N + u);
        const uint64_t* src = sSum64 + (size_t)(kk * SG + sb) * rows + sh + us * q0;
#pragma unroll
        for (int q = 0; q < S2_RH; ++q) {
            const int ii = q0 + q;
            bool valid = true;
            if (!INTERIOR) {
                // zero where the interpolation point leaves [0, nzs - 1]
                const int n0 = rlo + sh + us * ii;
                valid = ii < nrow && ((ii >= ia && ii < ib) ||
                                      (n0 >= 0 && (n0 < g.nzs - 1 || (n0 == g.nzs - 1 && fr == 0.f))));
            }
            if (valid) {
                const uint64_t s0 = src[us * q], s1 = src[us * q + 1];
                O1[q] = f2_fma(bx, s1, f2_fma(ax, s0, O1[q]));
                O2[q] = f2_fma(by, s1, f2_fma(ay, s0, O2[q]));
            }
        }
    }
    const size_t plane_sz = (size_t)g.nz * N;
    const size_t ob = ((((size_t)f * 2 + axL) * 2 + fam) * S + grp * SG + sb) * plane_sz + (size_t)(i0 + q0) * N + u;
    float2 v[S2_RH];
#pragma unroll
    for (int q = 0; q < S2_RH; ++q) v[q] = f2_unpack(s2_join(O1[q], O2[q]));
    s2_store_rows(planes, pt, ob, N, v, INTERIOR ? S2_RH : min(S2_RH, nrow - q0));
}

template <int TT, int US>
__device__ __forceinline__ bool stage2_body(int tile, int grp, int fam, int f, unsigned char* __restrict__ smraw,
                                            uint64_t* barp, const GeomDev& g, const float2* __restrict__ slices,
                                            const int* __restrict__ sfl, const float* __restrict__ sfr,
                                            const float4* __restrict__ lw, const float2* __restrict__ rot,
                                            const float2* __restrict__ coef, const float2* __restrict__ c2,
                                            const int* __restrict__ tmin, int T, int iA, int iB, int zp, int rows,
                                            int smin0, int smin1, void* __restrict__ planes, int pt,
                                            unsigned* __restrict__ status)
{
    uint64_t& bar = *barp;
    const int N = g.N, K = g.K, S = g.S, P = g.P;
    const int us = US > 0 ? US : g.us;
    const int nt = 2 * K;
    const int GW = s2_group_width(P), SG = GW / P;
    const int g0 = grp * GW;                           // first lateral pixel of the group
    const int gw = min(GW, N - g0);                    // pixels in this group
    const int sg = gw / P;                             // slabs in this group
    const int i0 = tile * zp;
    const int nrow = min(zp, g.nz - i0);
    const int smin = fam ? smin1 : smin0;
    const int rlo = us * i0 + smin;                    // slice row of window row 0
    float2* sS = reinterpret_cast<float2*>(smraw);                    // [K][rows][32]
    float4* sLw = reinterpret_cast<float4*>(sS + (size_t)K * rows * 32); // [K][N] {a, b}
    float4* sC2 = sLw + (size_t)K * N;                                 // [K][S][T] {x, x, y, y}
    float2* sSum = reinterpret_cast<float2*>(sC2 + (size_t)K * S * T); // [K][SG][rows]
    int* sSh = reinterpret_cast<int*>(sSum + (size_t)K * SG * rows);   // [K][N] floor shift - smin
    int* sTb = sSh + (size_t)K * N;                                    // [K][S] tmin - smin
    const int lo = max(rlo, 0), hi = max(lo, min(rlo + rows, g.nzs));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const unsigned cbytes = (unsigned)(gw * sizeof(float2));       // one row segment
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_fence_init();
        mbar_arrive_expect_tx(&bar, cbytes * (unsigned)(K * (hi - lo)));
    }
    // window rows outside the slice (and columns past the group) read zero
    if (gw < 32 || lo > rlo || hi < rlo + rows) {
        for (int kk = 0; kk < K; ++kk)
            for (int rr = warp; rr < rows; rr += nwarp) {
                const int r = rlo + rr;
                if (lane >= gw || r < lo || r >= hi) sS[((size_t)kk * rows + rr) * 32 + lane] = make_float2(0.f, 0.f);
            }
    }
    __syncthreads();
    // one bulk copy per (k, in-slice row): the group's gw pixels
    {
        const int nr = hi - lo;
        bool fenced = false;
        for (int idx = threadIdx.x; idx < K * nr; idx += blockDim.x) {
            const int kk = idx / nr, r = lo + (idx - kk * nr);
            if (!fenced) {
                fence_proxy_async();
                fenced = true;
            }
            bulk_g2s(sS + ((size_t)kk * rows + (r - rlo)) * 32,
                     slices + (((size_t)f * nt + fam * K + kk) * g.nzs + r) * N + g0, cbytes, &bar);
        }
    }
    // per-CTA tables while the copies are in flight
    for (int idx = threadIdx.x; idx < K * S * T; idx += blockDim.x) {
        const float2 c = __ldg(c2 + (size_t)fam * K * S * T + idx);
        sC2[idx] = make_float4(c.x, c.x, c.y, c.y);
    }
    for (int idx = threadIdx.x; idx < K * N; idx += blockDim.x) {
        const int k = fam * K + idx / N, u = idx % N;
        sLw[idx] = __ldg(lw + (size_t)k * N + u);
        sSh[idx] = __ldg(sfl + (size_t)k * N + u) - smin;
    }
    for (int idx = threadIdx.x; idx < K * S; idx += blockDim.x) sTb[idx] = __ldg(tmin + fam * K * S + idx) - smin;
    if (!cta_wait_copies(&bar, 0, status)) return false;
    // carrier rotation of the staged slice rows: w = v rot[k][r] (rows outside
    // the slice and columns past the group are zero and stay zero)
    // carrier rotation and slab sums of the group's slabs, one thread per
    // (k, window row, slab): each staged value of the slab becomes w = v
    // rot[k][r] in place (zero rows stay zero) and the rotated values are
    // summed; for a power-of-two P the pixels are visited in a row-rotated
    // order so that the lanes of a warp (consecutive slabs, then rows) spread
    // over the banks
    {
        const int nsum = K * rows * sg;
        const unsigned magic = sg > 1 ? 0xffffffffu / (unsigned)sg + 1u : 0u;   // idx / sg for idx < 2^16
        const bool pow2 = (P & (P - 1)) == 0;
        for (int idx = threadIdx.x; idx < nsum; idx += blockDim.x) {
            const int rk = sg == 1 ? idx : (int)__umulhi((unsigned)idx, magic);   // nsum == 0 when sg == 0
            const int sb = idx - rk * sg;
            const int kk = rk / rows, rr = rk - kk * rows;
            const int r = min(max(rlo + rr, 0), g.nzs - 1);      // rows outside the slice hold zeros
            const float2 e = __ldg(rot + (size_t)(fam * K + kk) * g.nzs + r);
            float2* px = sS + (size_t)rk * 32 + sb * P;
            float2 a = make_float2(0.f, 0.f);
            for (int j0 = 0; j0 < P; ++j0) {
                const int j = pow2 ? (j0 + rk) & (P - 1) : j0;
                const float2 v = px[j];
                const float2 w = make_float2(fmaf(v.x, e.x, -v.y * e.y), fmaf(v.x, e.y, v.y * e.x));
                px[j] = w;
                a.x += w.x;
                a.y += w.y;
            }
            sSum[((size_t)kk * SG + sb) * rows + rr] = a;
        }
    }
    __syncthreads();
    const int axT = fam == 0 ? 0 : 1;
    const int axL = 1 - axT;
    // the tile's rows with carrier-separable taps: [ia, ib) (tile-relative)
    const int ia = min(nrow, max(0, iA - i0)), ib = max(ia, min(nrow, iB - i0 + 1));
    const bool interior = ia == 0 && ib == nrow && nrow == S2_ZP;
    // tasks: S2_RH plane rows of one transverse slab (lanes over the group's
    // pixels) or of one lateral slab and 32 transverse positions; zp <= S2_ZP = 2 S2_RH
    const int H = nrow > S2_RH ? 2 : 1;
    const int LU = (N + 31) >> 5;
    const int nTt = S * H, nTl = sg * LU * H;
    const uint64_t* sS64 = reinterpret_cast<const uint64_t*>(sS);
    const uint64_t* sC2q = reinterpret_cast<const uint64_t*>(sC2);
    const uint64_t* sSum64 = reinterpret_cast<const uint64_t*>(sSum);
    for (int task = warp; task < nTt + nTl; task += nwarp) {
        if (task < nTt) {
            const int b = H == 2 ? task >> 1 : task, q0 = H == 2 ? (task & 1) * S2_RH : 0;
            if (interior)
                s2_transverse<TT, US, true>(b, q0, nrow, ia, ib, lane, gw, fam, f, i0, axT, g, T, rows, sS64, sC2q,
                                            sTb, coef, planes, pt, g0, status);
            else
                s2_transverse<TT, US, false>(b, q0, nrow, ia, ib, lane, gw, fam, f, i0, axT, g, T, rows, sS64, sC2q,
                                             sTb, coef, planes, pt, g0, status);
        } else {
            const int o = task - nTt;
            const int hq = H == 2 ? o & 1 : 0, rest = H == 2 ? o >> 1 : o;
            const int sb = rest / LU, u = (rest - sb * LU) * 32 + lane;
            if (u < N) {
                if (interior)
                    s2_lateral<US, true>(sb, u, hq * S2_RH, nrow, ia, ib, fam, f, i0, axL, rlo, grp, SG, g, rows, sLw,
                                         sSh, sSum64, sfr, planes, pt, status);
                else
                    s2_lateral<US, false>(sb, u, hq * S2_RH, nrow, ia, ib, fam, f, i0, axL, rlo, grp, SG, g, rows, sLw,
                                          sSh, sSum64, sfr, planes, pt, status);
            }
        }
    }
    return true;
}

inline bool complex_dtype(rca_dtype t) { return t == RCA_C32 || t == RCA_C16F || t == RCA_C16BF; }

}  // namespace
