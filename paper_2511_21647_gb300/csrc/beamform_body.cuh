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
// [e][n] coalesced along n, writes IQ [n][e] coalesced along e.
__device__ __forceinline__ void demod_body(int bx, int by, int bz, float2* __restrict__ xs,
                                           const void* __restrict__ rf, int rf_t, const float* __restrict__ scale,
                                           const float* __restrict__ mean, const float2* __restrict__ mix,
                                           const Fir& fir, int nt, int E, int ns, void* __restrict__ iq, int iq_t)
{
    const int n0 = bx * DM_NT;
    const int e0 = by * DM_NE;
    const int fk = bz;
    const int k = fk % nt;
    const size_t chan0 = (size_t)fk * E;
#pragma unroll 4
    for (int idx = threadIdx.x; idx < DM_NE * (DM_NT + 30); idx += blockDim.x) {
        int el = idx / (DM_NT + 30), s = idx - el * (DM_NT + 30);
        int n = n0 - 15 + s, e = e0 + el;
        float2 v = make_float2(0.f, 0.f);
        if (n >= 0 && n < ns && e < E) {
            float x = rf_value(rf, rf_t, (chan0 + e) * ns + n);
            if (rf_t == RCA_I16) x *= scale[k * E + e];
            if (mean) x -= mean[((size_t)k * E + e) * ns + n];
            float2 m = mix[n];
            v = make_float2(x * m.x, x * m.y);
        }
        xs[el * DM_PITCH + s] = v;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < DM_NE * DM_NT; idx += blockDim.x) {
        int el = idx % DM_NE, s = idx / DM_NE;
        int n = n0 + s, e = e0 + el;
        if (n >= ns || e >= E) continue;
        const float2* x = xs + el * DM_PITCH + s + 15;
        float re = fir.h[15] * x[0].x, im = fir.h[15] * x[0].y;
#pragma unroll
        for (int m = 1; m <= 15; m += 2) {  // even taps are zero (half-band)
            float hm = fir.h[15 + m];
            re = fmaf(hm, x[-m].x + x[m].x, re);
            im = fmaf(hm, x[-m].y + x[m].y, im);
        }
        store_c(iq, ((size_t)fk * ns + n) * E + e, iq_t, make_float2(2.f * re, 2.f * im));
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

// One range [d0, d1) of lateral distances with fixed modes for the two mirror
// elements: S1_FULL (every lane has the element), S1_PRED (some do: the others
// load zeros), S1_NONE (no lane does: skipped).  nrow: rows of this thread
// (MAXR when EXACT).  H[j] = {A1.x, A1.y, A2.x, A2.y}: sums of the
// Re-weight and Im-weight products of row j.
template <typename TS, int MAXR, bool EXACT, int XM, int YM>
__device__ __forceinline__ void stage1_range(float (&H)[MAXR][4], int d0,
                                             int d1, int cz, int zt, int l, int Lx, int Ly, int row0, int nrow,
                                             unsigned rbase, unsigned obase, unsigned wbase, int RS)
{
    constexpr bool HALF = S1Rec<TS>::HALF;
    constexpr int RB = S1Rec<TS>::BYTES, ESZ = (int)sizeof(TS);
#pragma unroll 1
    for (int d = d0; d < d1; ++d) {
        const bool hx = XM == S1_FULL || (XM == S1_PRED && d <= Lx);
        const bool hy = YM == S1_FULL || (YM == S1_PRED && d <= Ly);
        // window offsets of the two mirror elements (records hold the row offset)
        const unsigned ox = wbase + (unsigned)((l - d) * ESZ), oy = wbase + (unsigned)((l + d) * ESZ);
        const unsigned ox1 = ox + RS, oy1 = oy + RS;
        const int base = (d - cz) * zt + row0;    // record index of the thread's first row
        const unsigned rp = rbase + base * RB, op = obase + base * 4;
        unsigned rowq[4];
#pragma unroll
        for (int j = 0; j < MAXR; ++j) {
            if (EXACT || j < nrow) {
                if constexpr (HALF) {
                    unsigned wr, wi, row, pad;
                    lds_u32x4(rp + j * RB, wr, wi, row, pad);
                    unsigned x0 = 0u, x1 = 0u, y0 = 0u, y1 = 0u;
                    if (XM != S1_NONE && hx) {
                        x0 = lds_u32(row + ox);
                        x1 = lds_u32(row + ox1);
                    }
                    if (YM != S1_NONE && hy) {
                        y0 = lds_u32(row + oy);
                        y1 = lds_u32(row + oy1);
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
                    s1_mfma(H[j][0], H[j][1], H[j][2], H[j][3], wr, wi, s0, s1);
                } else {
                    unsigned ax, bx, ay, by;
                    lds_u32x4(rp + j * RB, ax, bx, ay, by);
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
                    const unsigned row = rowq[QUAD ? (j & 3) : 0] >> (ESZ == 4 ? 1 : 0);
                    uint64_t x0 = 0ull, x1 = 0ull, y0 = 0ull, y1 = 0ull;
                    if (XM != S1_NONE && hx) {
                        x0 = s1_ld<TS>(row + ox);
                        x1 = s1_ld<TS>(row + ox1);
                    }
                    if (YM != S1_NONE && hy) {
                        y0 = s1_ld<TS>(row + oy);
                        y1 = s1_ld<TS>(row + oy1);
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
                    const float fax = __uint_as_float(ax), fbx = __uint_as_float(bx);
                    const float fay = __uint_as_float(ay), fby = __uint_as_float(by);
                    H[j][0] = fmaf(fax, u.x, fmaf(fbx, v.x, H[j][0]));
                    H[j][1] = fmaf(fax, u.y, fmaf(fbx, v.y, H[j][1]));
                    H[j][2] = fmaf(fay, u.x, fmaf(fby, v.x, H[j][2]));
                    H[j][3] = fmaf(fay, u.y, fmaf(fby, v.y, H[j][3]));
                }
            }
        }
    }
}

// Returns false if a bounded wait ran out (the CTA must stop).  The thread
// owns rows [rg * per, rg * per + per) of the tile, per = ceil(zt / RG)
// (per <= MAXR; EXACT: per == MAXR and zt == RG * MAXR, or MAXR == 1).
// rtab: the plan's record table for this arithmetic (FP16 weights for FP16
// samples, FP32 weights otherwise), one block of rblk bytes per chunk.
template <typename TS, int MAXR, bool EXACT>
__device__ __forceinline__ bool stage1_body(int tile, int k, int f, unsigned char* __restrict__ smraw,
                                            uint64_t* bars, const GeomDev& g, const void* __restrict__ iq,
                                            const unsigned char* __restrict__ rtab, int rblk,
                                            const int* __restrict__ dmax, const int4* __restrict__ chunks, int zt,
                                            int dc, int n_tiles, int nch, int win, float2* __restrict__ slices,
                                            unsigned* __restrict__ status)
{
    constexpr int ESZ = (int)sizeof(TS);
    const int E = g.N, N = g.N;
    const int RS = E * ESZ;                                   // window row (bytes)
    unsigned char* bufs = smraw;                              // [2][win][RS]
    unsigned char* recs = bufs + 2 * (size_t)win * RS;        // [2][rblk]
    const int nt = 2 * g.K;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int LW = (N + 31) >> 5;
    const int RG = (blockDim.x >> 5) / LW;
    const int lw = warp % LW, rg = warp / LW;
    const int lb = lw * 32;
    const int l = lb + lane;
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

    // zero the window rows outside the record, then (thread 0) bulk-copy the
    // rest and the chunk's record block on one barrier
    auto issue = [&](int c, int b) {
        const int4 cc = ch[c];
        unsigned char* dst = bufs + (size_t)b * win * RS;
        const int lo = max(cc.x, 0), hi = max(lo, min(cc.x + cc.y, g.ns));
        const int z0 = min(lo - cc.x, cc.y), z1 = hi - cc.x;
        const int v16 = RS / 16;
        for (int idx = threadIdx.x; idx < z0 * v16; idx += blockDim.x)
            reinterpret_cast<uint4*>(dst)[idx] = make_uint4(0u, 0u, 0u, 0u);
        for (int idx = threadIdx.x; idx < (cc.y - z1) * v16; idx += blockDim.x)
            reinterpret_cast<uint4*>(dst + (size_t)z1 * RS)[idx] = make_uint4(0u, 0u, 0u, 0u);
        if (threadIdx.x == 0) {
            fence_proxy_async();
            const unsigned bytes = (unsigned)((hi - lo) * RS);
            mbar_arrive_expect_tx(&bars[b], bytes + (unsigned)rblk);
            if (bytes) bulk_g2s(dst + (size_t)(lo - cc.x) * RS, blk + (size_t)lo * RS, bytes, &bars[b]);
            bulk_g2s(recs + (size_t)b * rblk, rsrc + (size_t)c * rblk, (unsigned)rblk, &bars[b]);
        }
    };

    // H[j] = {A1.x, A1.y, A2.x, A2.y}; slice value = (A1.x - A2.y, A1.y + A2.x)
    float H[MAXR][4];
#pragma unroll
    for (int j = 0; j < MAXR; ++j) H[j][0] = H[j][1] = H[j][2] = H[j][3] = 0.f;
    // per-lane reach of the mirror elements: l - d needs d <= Lx, l + d needs d <= Ly
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
        if (cc.y == 0 || nrow == 0) continue;
        const unsigned wbase = smem_u32(bufs + (size_t)b * win * RS);
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
    stage1_range<TS, MAXR, EXACT, XM, YM>(H, d, nx, cc.z, zt, l, Lx, Ly, row0, nrow, rbase, obase, wbase, RS)
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
#pragma unroll
    for (int j = 0; j < MAXR; ++j) {
        const int r = r0 + row0 + j;
        if ((EXACT || j < nrow) && r < rend && l < N)
            slices[(((size_t)f * nt + k) * g.nzs + r) * N + l] = make_float2(H[j][0] - H[j][3], H[j][1] + H[j][2]);
    }
    return true;
}

// ---------------------------------------------------------------------------
// Stage 2 + block sum-projection, written straight to the planes.
// For a family, the "transverse-slab" plane sums over the transverse
// coordinate u inside slab b: each u shifts the slice by its own dz_k(u), so
// the per-(k, b, i) sum of P linear interpolations is a short filter along
// the slice rows with precomputed coefficients.  The "lateral-slab" plane sums
// over lateral pixels inside slab b: the shift does not depend on the lateral
// pixel, so the slice is first summed over the slab and interpolated once.
// RC: transverse = y -> XZ planes (axis 0), lateral-slab -> YZ (axis 1).
// CR: transverse = x -> YZ planes (axis 1), lateral-slab -> XZ (axis 0).
// ---------------------------------------------------------------------------
template <int ZP>
__device__ __forceinline__ bool stage2_body(int tile, int fam, int f, int zp, float2* __restrict__ sm, uint64_t* barp,
                                            const GeomDev& g, const float2* __restrict__ slices,
                                            const int* __restrict__ sfl, const float* __restrict__ sfr,
                                            const float2* __restrict__ psi, const float2* __restrict__ ec,
                                            const float2* __restrict__ coef, const int* __restrict__ tmin, int T,
                                            int rows, int smin0, int smin1, void* __restrict__ planes, int pt,
                                            unsigned* __restrict__ status)
{
    uint64_t& bar = *barp;
    const int N = g.N, K = g.K, S = g.S, P = g.P, us = g.us;
    const int nt = 2 * K;
    const int i0 = tile * zp;          // zp <= ZP plane rows per tile
    const int nrow = min(zp, g.nz - i0);
    const int smin = fam ? smin1 : smin0;
    const int rlo = us * i0 + smin;
    float2* sS = sm;                                 // [K][rows][N]
    float2* sSum = sS + (size_t)K * rows * N;        // [K][S][rows]
    float2* sCoef = sSum + (size_t)K * S * rows;     // [K][S][ZP][T]
    float2* sPsi = sCoef + (size_t)K * S * ZP * T;   // [K][N]
    float2* sEc = sPsi + (size_t)K * N;              // [K][ZP]
    float* sSfr = reinterpret_cast<float*>(sEc + (size_t)K * ZP);  // [K][N]
    int* sSfl = reinterpret_cast<int*>(sSfr + (size_t)K * N);       // [K][N]  (row offset - smin)
    int* sTb = sSfl + (size_t)K * N;                                 // [K][S]  (tmin - smin)
    const int lo = max(rlo, 0), hi = max(lo, min(rlo + rows, g.nzs));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_fence_init();
    }
    __syncthreads();
    {
        const int z0 = min(lo - rlo, rows), z1 = hi - rlo;
        const int nzr = z0 + (rows - z1);
        for (int idx = threadIdx.x; idx < K * nzr * N; idx += blockDim.x) {
            const int kk = idx / (nzr * N), q = idx - kk * nzr * N, zr = q / N, l = q - zr * N;
            const int rr = zr < z0 ? zr : z1 + (zr - z0);
            sS[((size_t)kk * rows + rr) * N + l] = make_float2(0.f, 0.f);
        }
    }
    if (threadIdx.x == 0) {
        fence_proxy_async();
        const unsigned bytes = (unsigned)((hi - lo) * N * sizeof(float2));
        mbar_arrive_expect_tx(&bar, bytes * K);
        if (bytes)
            for (int kk = 0; kk < K; ++kk)
                bulk_g2s(sS + ((size_t)kk * rows + (lo - rlo)) * N,
                         slices + (((size_t)f * nt + fam * K + kk) * g.nzs + lo) * N, bytes, &bar);
    }
    // per-CTA table slices while the copy is in flight
    for (int idx = threadIdx.x; idx < K * S * ZP * T; idx += blockDim.x) {
        const int t = idx % T, ii = (idx / T) % ZP, kb = idx / (T * ZP);
        const int kk = kb / S, b = kb % S, i = min(i0 + ii, g.nz - 1);
        sCoef[idx] = __ldg(coef + (((size_t)(fam * K + kk) * S + b) * g.nz + i) * T + t);
    }
    for (int idx = threadIdx.x; idx < K * N; idx += blockDim.x) {
        const int k = fam * K + idx / N, u = idx % N;
        sPsi[idx] = __ldg(psi + (size_t)k * N + u);
        sSfr[idx] = __ldg(sfr + (size_t)k * N + u);
        sSfl[idx] = __ldg(sfl + (size_t)k * N + u) - smin;
    }
    for (int idx = threadIdx.x; idx < K * ZP; idx += blockDim.x) {
        const int kk = idx / ZP, ii = idx % ZP;
        sEc[idx] = __ldg(ec + (size_t)(fam * K + kk) * g.nz + min(i0 + ii, g.nz - 1));
    }
    for (int idx = threadIdx.x; idx < K * S; idx += blockDim.x) sTb[idx] = __ldg(tmin + fam * K * S + idx) - smin;
    if (!cta_wait_copies(&bar, 0, status)) return false;
    // slab sums over the lateral pixels: one warp per (k, row)
    for (int o = warp; o < K * rows; o += nwarp) {
        const int kk = o / rows, rr = o - kk * rows;
        const float2* src = sS + ((size_t)kk * rows + rr) * N;
        if ((32 % P) == 0) {
            for (int c0 = 0; c0 < N; c0 += 32) {
                const int l = c0 + lane;
                float2 v = l < N ? src[l] : make_float2(0.f, 0.f);
                for (int m = 1; m < P; m <<= 1) {
                    v.x += __shfl_xor_sync(0xffffffffu, v.x, m);
                    v.y += __shfl_xor_sync(0xffffffffu, v.y, m);
                }
                if ((lane % P) == 0 && l < N) sSum[((size_t)kk * S + l / P) * rows + rr] = v;
            }
        } else {
            for (int b = lane; b < S; b += 32) {
                float2 a = make_float2(0.f, 0.f);
                for (int q = 0; q < P; ++q) {
                    a.x += src[b * P + q].x;
                    a.y += src[b * P + q].y;
                }
                sSum[((size_t)kk * S + b) * rows + rr] = a;
            }
        }
    }
    __syncthreads();
    const int axT = fam == 0 ? 0 : 1;
    const int axL = 1 - axT;
    const size_t plane_sz = (size_t)g.nz * N;
    const int LW = (N + 31) >> 5;
    // transverse-slab planes: out[b][i][l] = sum_k sum_t coef[k][b][i][t] S_k(l, us i + tmin[k][b] + t)
    for (int o = warp; o < S * LW; o += nwarp) {
        const int lw = o % LW, b = o / LW;
        const int l = lw * 32 + lane, lc = l < N ? l : 0;
        uint64_t a1[ZP], a2[ZP];
#pragma unroll
        for (int ii = 0; ii < ZP; ++ii) a1[ii] = a2[ii] = 0ull;
        for (int kk = 0; kk < K; ++kk) {
            const int tb = sTb[kk * S + b];
            const float2* cf = sCoef + (size_t)(kk * S + b) * ZP * T;
            const uint64_t* col = reinterpret_cast<const uint64_t*>(sS + ((size_t)kk * rows + tb) * N + lc);
            for (int t = 0; t < T; ++t) {
#pragma unroll
                for (int ii = 0; ii < ZP; ++ii) {
                    if (ii < nrow) {
                        const float2 c = cf[ii * T + t];
                        const uint64_t v = col[(size_t)(us * ii + t) * N];
                        a1[ii] = f2_fma(f2_pack(c.x, c.x), v, a1[ii]);
                        a2[ii] = f2_fma(f2_pack(c.y, c.y), v, a2[ii]);
                    }
                }
            }
        }
        if (l < N) {
            const size_t ob = ((((size_t)f * 2 + axT) * 2 + fam) * S + b) * plane_sz + (size_t)i0 * N + l;
#pragma unroll
            for (int ii = 0; ii < ZP; ++ii) {
                if (ii < nrow) {
                    const float2 p1 = f2_unpack(a1[ii]), p2 = f2_unpack(a2[ii]);
                    store_c_cs(planes, ob + (size_t)ii * N, pt, make_float2(p1.x - p2.y, p1.y + p2.x));
                }
            }
        }
    }
    // lateral-slab planes: out[b][i][u] = sum_k ec[k][i] psi[k][u] lerp(sum_{l in b} S_k(l, .), us i + s_k(u))
    for (int o = warp; o < S * LW; o += nwarp) {
        const int lw = o % LW, b = o / LW;
        const int u = lw * 32 + lane;
        if (u >= N) continue;
        float2 acc[ZP];
#pragma unroll
        for (int ii = 0; ii < ZP; ++ii) acc[ii] = make_float2(0.f, 0.f);
        for (int kk = 0; kk < K; ++kk) {
            const int n0r = sSfl[kk * N + u];     // row offset relative to rlo at ii = 0
            const float fr = sSfr[kk * N + u];
            const float2 ps = sPsi[kk * N + u];
            const float2* src = sSum + ((size_t)kk * S + b) * rows;
#pragma unroll
            for (int ii = 0; ii < ZP; ++ii) {
                const int nr = us * ii + n0r;
                const int n0 = rlo + nr;          // slice row
                const bool valid = ii < nrow && n0 >= 0 && (n0 < g.nzs - 1 || (n0 == g.nzs - 1 && fr == 0.f));
                if (valid) {
                    const float2 s0 = src[nr], s1 = src[nr + 1];
                    const float2 v = make_float2(fmaf(fr, s1.x - s0.x, s0.x), fmaf(fr, s1.y - s0.y, s0.y));
                    cfma(acc[ii], cmul(sEc[kk * ZP + ii], ps), v);
                }
            }
        }
        const size_t ob = ((((size_t)f * 2 + axL) * 2 + fam) * S + b) * plane_sz + (size_t)i0 * N + u;
#pragma unroll
        for (int ii = 0; ii < ZP; ++ii)
            if (ii < nrow) store_c_cs(planes, ob + (size_t)ii * N, pt, acc[ii]);
    }
    return true;
}

inline bool complex_dtype(rca_dtype t) { return t == RCA_C32 || t == RCA_C16F || t == RCA_C16BF; }

}  // namespace
