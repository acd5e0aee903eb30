// beamform.cu -- channel data -> IQ -> Stage-1 slices -> projection planes.
//
// Sec. II-A1 (two-stage RCA beamforming, Fig. 1b-c), Sec. II-A4/II-A5
// (P x P x N sub-blocks sum-projected onto x-z and y-z planes), Sec. II-A2
// (clutter removal before Stage 2; here the ensemble-mean filter).
#include <algorithm>

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

__global__ void __launch_bounds__(256) k_mean(const void* __restrict__ rf, int rf_t, const float* __restrict__ scale,
                                              int F, int ns, int ncol, float* __restrict__ mean)
{
    mean_body(blockIdx.x, rf, rf_t, scale, F, ns, ncol, mean);
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

__global__ void __launch_bounds__(256) k_demod(const void* __restrict__ rf, int rf_t, const float* __restrict__ scale,
                                               const float* __restrict__ mean, const float2* __restrict__ mix, Fir fir,
                                               int nt, int E, int ns, void* __restrict__ iq, int iq_t)
{
    __shared__ float2 xs[DM_NE * DM_PITCH];
    demod_body(blockIdx.x, blockIdx.y, blockIdx.z, xs, rf, rf_t, scale, mean, mix, fir, nt, E, ns, iq, iq_t);
}

// ---------------------------------------------------------------------------
// Stage 1: reference slices
//   S_k(l, r) = sum_d W[r][d] (IQ_{k, l-d}(xi) + IQ_{k, l+d}(xi)),  (d = 0 once)
//   xi = (tx_q16[k][r] + rx_q16[r][d]) / 2^16 samples.
// For a fixed (r, d) the sample position is the same for every lateral pixel,
// so each warp (32 consecutive pixels) reads 32 consecutive elements of one
// sample row of the [ns][E] IQ block: the delay, its fraction and the weight
// are warp-uniform and are precomputed per (row, d) once per chunk.  The
// chunk's sample window is one contiguous block of the IQ array, fetched by a
// TMA bulk copy into a double buffer while the previous chunk is processed.
// ---------------------------------------------------------------------------
// per-(row, d) record, 32 bytes: the interpolation fraction and the
// apodised carrier weight (0 where the delay leaves the record) duplicated
// into packed pairs, and the element offset of the sample row in the window
struct __align__(16) RowD {
    float fr0, fr1;  // fraction, fraction
    float wx0, wx1;  // Re w, Re w
    float wy0, wy1;  // Im w, Im w
    int off;         // sample row * E
    int pad;
};

// one complex IQ sample from shared memory (byte address) as a packed float pair
template <typename TS>
__device__ __forceinline__ uint64_t ld_sa(unsigned addr);
template <>
__device__ __forceinline__ uint64_t ld_sa<float2>(unsigned addr) { return lds_u64(addr); }
template <>
__device__ __forceinline__ uint64_t ld_sa<__half2>(unsigned addr)
{
    unsigned u = lds_u32(addr);
    const float2 v = __half22float2(*reinterpret_cast<__half2*>(&u));
    return f2_pack(v.x, v.y);
}
template <>
__device__ __forceinline__ uint64_t ld_sa<__nv_bfloat162>(unsigned addr)
{
    unsigned u = lds_u32(addr);
    // bf16 -> f32 is a 16-bit shift of each half
    return f2_pack(__uint_as_float(u << 16), __uint_as_float(u & 0xffff0000u));
}

// one complex IQ sample (shared memory) as a packed float pair
template <typename TS>
__device__ __forceinline__ uint64_t ld_sp(const unsigned char* p);
template <>
__device__ __forceinline__ uint64_t ld_sp<float2>(const unsigned char* p) { return *reinterpret_cast<const uint64_t*>(p); }
template <>
__device__ __forceinline__ uint64_t ld_sp<__half2>(const unsigned char* p)
{
    const float2 v = __half22float2(*reinterpret_cast<const __half2*>(p));
    return f2_pack(v.x, v.y);
}
template <>
__device__ __forceinline__ uint64_t ld_sp<__nv_bfloat162>(const unsigned char* p)
{
    const unsigned u = *reinterpret_cast<const unsigned*>(p);
    return f2_pack(__uint_as_float(u << 16), __uint_as_float(u & 0xffff0000u));
}

// v = b0 + fr (b1 - b0);  A1 += wx * v;  A2 += wy * v   (all packed pairs).
// The complex product w * v is recovered at the end as
// (A1.x - A2.y, A1.y + A2.x).
template <typename TS>
__device__ __forceinline__ void lerp_acc2(uint64_t& A1, uint64_t& A2, unsigned a0, unsigned rowbytes, uint64_t frp,
                                          uint64_t wxp, uint64_t wyp)
{
    const uint64_t b0 = ld_sa<TS>(a0), b1 = ld_sa<TS>(a0 + rowbytes);
    const uint64_t v = f2_fma(frp, f2_sub(b1, b0), b0);
    A1 = f2_fma(wxp, v, A1);
    A2 = f2_fma(wyp, v, A2);
}

// returns false if a bounded wait ran out (the CTA must stop)
template <typename TS, int MAXR>
__device__ __forceinline__ bool stage1_body(int tile, int k, int f, unsigned char* __restrict__ smraw,
                                            uint64_t* bars, const GeomDev& g, const void* __restrict__ iq,
                                            const int* __restrict__ tx_q16, const int* __restrict__ rx_q16,
                                            const float2* __restrict__ W, const int* __restrict__ dmax,
                                            const int4* __restrict__ chunks, int zt, int dc, int n_tiles, int nch,
                                            int win, float2* __restrict__ slices, unsigned* __restrict__ status)
{
    const int E = g.N, N = g.N;
    TS* bufs = reinterpret_cast<TS*>(smraw);                  // [2][win][E]
    RowD* recs = reinterpret_cast<RowD*>(bufs + 2 * (size_t)win * E);  // [2][zt][dc]
    int* dcnt = reinterpret_cast<int*>(recs + 2 * zt * dc);  // [2][zt]
    const int nt = 2 * g.K;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int LW = (N + 31) >> 5;
    const int RG = (blockDim.x >> 5) / LW;
    const int lw = warp % LW, rg = warp / LW;
    const int lb = lw * 32;
    const int l = lb + lane;
    const int r0 = tile * zt;
    const int rend = min(r0 + zt, g.nzs);
    const int qmax = (g.ns - 1) << 16;
    const int4* ch = chunks + ((size_t)k * n_tiles + tile) * nch;
    const TS* blk = reinterpret_cast<const TS*>(iq) + ((size_t)f * nt + k) * g.ns * E;
    const TS zero = TS();

    if (threadIdx.x == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        mbar_fence_init();
    }
    __syncthreads();

    // zero the window rows outside the record, then (thread 0) bulk-copy the rest
    auto issue = [&](int c, int b) {
        const int4 cc = ch[c];
        TS* dst = bufs + (size_t)b * win * E;
        const int lo = max(cc.x, 0), hi = max(lo, min(cc.x + cc.y, g.ns));
        const int z0 = min(lo - cc.x, cc.y), z1 = hi - cc.x;
        for (int idx = threadIdx.x; idx < z0 * E; idx += blockDim.x) dst[idx] = zero;
        for (int idx = threadIdx.x; idx < (cc.y - z1) * E; idx += blockDim.x) dst[(size_t)z1 * E + idx] = zero;
        if (threadIdx.x == 0) {
            fence_proxy_async();
            const unsigned bytes = (unsigned)((hi - lo) * E * sizeof(TS));
            mbar_arrive_expect_tx(&bars[b], bytes);
            if (bytes) bulk_g2s(dst + (size_t)(lo - cc.x) * E, blk + (size_t)lo * E, bytes, &bars[b]);
        }
    };

    uint64_t acc1[MAXR], acc2[MAXR];
#pragma unroll
    for (int j = 0; j < MAXR; ++j) acc1[j] = acc2[j] = 0ull;
    unsigned phase = 0;
    issue(0, 0);
    for (int c = 0; c < nch; ++c) {
        const int b = c & 1;
        const int4 cc = ch[c];
        RowD* rc = recs + b * zt * dc;
        for (int idx = threadIdx.x; idx < zt * dc; idx += blockDim.x) {
            const int rr = idx / dc, dd = idx - rr * dc;
            const int r = r0 + rr, d = cc.z + dd;
            RowD rec;
            rec.off = 0;
            rec.pad = 0;
            rec.fr0 = rec.fr1 = rec.wx0 = rec.wx1 = rec.wy0 = rec.wy1 = 0.f;
            if (r < rend && d < cc.w && d <= __ldg(dmax + r)) {
                const int q = __ldg(tx_q16 + (size_t)k * g.nzs + r) + __ldg(rx_q16 + (size_t)r * N + d);
                if (q >= 0 && q <= qmax) {
                    const float2 w = __ldg(W + (size_t)r * N + d);
                    rec.off = ((q >> 16) - cc.x) * E * (int)sizeof(TS);   // byte offset of the row
                    rec.fr0 = rec.fr1 = (float)(q & 0xffff) * (1.0f / 65536.0f);
                    rec.wx0 = rec.wx1 = w.x;
                    rec.wy0 = rec.wy1 = w.y;
                }
            }
            rc[idx] = rec;
        }
        for (int rr = threadIdx.x; rr < zt; rr += blockDim.x) {
            const int r = r0 + rr;
            dcnt[b * zt + rr] = r < rend ? max(0, min(cc.w, __ldg(dmax + r) + 1) - cc.z) : 0;
        }
        if (!cta_wait_copies(&bars[b], (phase >> b) & 1u, status)) return false;
        phase ^= 1u << b;
        if (c + 1 < nch) issue(c + 1, b ^ 1);
        if (cc.y == 0) continue;
        const unsigned char* wbase = reinterpret_cast<const unsigned char*>(bufs + (size_t)b * win * E);
        const int rowbytes = E * (int)sizeof(TS);
        const int lim1 = lb + 31 - cc.z;     // warp-uniform: e = l - d reachable for dd <= lim1
        const int lim2 = N - 1 - lb - cc.z;  // warp-uniform: e = l + d reachable for dd <= lim2
        const int L1 = l - cc.z;             // this lane: e = l - d >= 0 for dd <= L1
        const int L2 = N - 1 - l - cc.z;     // this lane: e = l + d < N for dd <= L2
        // the thread's rows advance together: each d step updates MAXR
        // independent accumulators (records past a row's aperture have w = 0);
        // lanes outside the element range load zeros instead of branching
        int ndw = 0;
#pragma unroll
        for (int j = 0; j < MAXR; ++j) {
            const int rr = rg + j * RG;
            if (rr < zt) ndw = max(ndw, dcnt[b * zt + rr]);
        }
        const int n1 = min(ndw, lim1 + 1);
        const int s2 = cc.z == 0 ? 1 : 0;   // d = 0 is counted once
        const int n2 = min(ndw, lim2 + 1);
        const int nmax = max(n1, n2);
        for (int dd = 0; dd < nmax; ++dd) {
            const bool h1 = dd < n1 && dd <= L1 && l < N;
            const bool h2 = dd >= s2 && dd < n2 && dd <= L2;
            const int o1 = (L1 - dd) * (int)sizeof(TS);
            const int o2 = (l + cc.z + dd) * (int)sizeof(TS);
#pragma unroll
            for (int j = 0; j < MAXR; ++j) {
                const int rr = rg + j * RG;
                if (rr < zt) {
                    const ulonglong2* rp = reinterpret_cast<const ulonglong2*>(rc + rr * dc + dd);
                    const ulonglong2 ra = rp[0], rb = rp[1];   // {fr, fr | wx, wx}, {wy, wy | off}
                    const unsigned char* row = wbase + (int)(unsigned)rb.y;
                    uint64_t x0 = 0ull, x1 = 0ull, y0 = 0ull, y1 = 0ull;
                    if (h1) {
                        x0 = ld_sp<TS>(row + o1);
                        x1 = ld_sp<TS>(row + o1 + rowbytes);
                    }
                    if (h2) {
                        y0 = ld_sp<TS>(row + o2);
                        y1 = ld_sp<TS>(row + o2 + rowbytes);
                    }
                    const uint64_t v1 = f2_fma(ra.x, f2_sub(x1, x0), x0);
                    const uint64_t v2 = f2_fma(ra.x, f2_sub(y1, y0), y0);
                    acc1[j] = f2_fma(ra.y, v1, acc1[j]);
                    acc2[j] = f2_fma(rb.x, v1, acc2[j]);
                    acc1[j] = f2_fma(ra.y, v2, acc1[j]);
                    acc2[j] = f2_fma(rb.x, v2, acc2[j]);
                }
            }
        }
    }
#pragma unroll
    for (int j = 0; j < MAXR; ++j) {
        const int r = r0 + rg + j * RG;
        if (r < rend && (rg + j * RG) < zt && l < N) {
            const float2 p1 = f2_unpack(acc1[j]), p2 = f2_unpack(acc2[j]);
            slices[(((size_t)f * nt + k) * g.nzs + r) * N + l] = make_float2(p1.x - p2.y, p1.y + p2.x);
        }
    }
    return true;
}

template <typename TS, int MAXR>
__global__ void __launch_bounds__(256, 2) k_stage1(GeomDev g, const void* __restrict__ iq,
                                                const int* __restrict__ tx_q16, const int* __restrict__ rx_q16,
                                                const float2* __restrict__ W, const int* __restrict__ dmax,
                                                const int4* __restrict__ chunks, int zt, int dc, int n_tiles, int nch,
                                                int win, float2* __restrict__ slices, unsigned* __restrict__ status)
{
    extern __shared__ __align__(128) unsigned char smraw[];
    __shared__ uint64_t bars[2];
    stage1_body<TS, MAXR>(blockIdx.x, blockIdx.y, blockIdx.z, smraw, bars, g, iq, tx_q16, rx_q16, W, dmax, chunks,
                          zt, dc, n_tiles, nch, win, slices, status);
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

template <int ZP>
__global__ void __launch_bounds__(512) k_stage2(GeomDev g, const float2* __restrict__ slices,
                                                const int* __restrict__ sfl, const float* __restrict__ sfr,
                                                const float2* __restrict__ psi, const float2* __restrict__ ec,
                                                const float2* __restrict__ coef, const int* __restrict__ tmin, int T,
                                                int rows, int smin0, int smin1, void* __restrict__ planes, int pt,
                                                unsigned* __restrict__ status)
{
    extern __shared__ __align__(128) float2 sm[];
    __shared__ uint64_t bar;
    stage2_body<ZP>(blockIdx.x, blockIdx.y, blockIdx.z, ZP, sm, &bar, g, slices, sfl, sfr, psi, ec, coef, tmin, T,
                    rows, smin0, smin1, planes, pt, status);
}

// ---------------------------------------------------------------------------
// Direct projection of conventional 3D DAS (no volume).  CTA = (plane-row
// tile, transverse slab bt, frame x family); for every transmission of the
// family and every transverse position u of the slab it beamforms the voxels
// V(l, u, i) of its rows (DAS with the delay of position u), then
//   transverse-slab plane  out[bt][i][l] += V(l, u, i)
//   lateral-slab plane     out[l / P][i][u] += sum over the P lanes of a slab.
// ---------------------------------------------------------------------------
template <int MAXR>
__global__ void __launch_bounds__(256) k_direct(GeomDev g, const void* __restrict__ iq, int iq_t,
                                                    const int* __restrict__ dtx_q16, const float2* __restrict__ dtx_ph,
                                                    const int* __restrict__ rx_q16, const float2* __restrict__ W,
                                                    const int* __restrict__ dmax, int dzt, int win,
                                                    void* __restrict__ planes, int pt)
{
    extern __shared__ float2 sm[];
    const int E = g.N, N = g.N, S = g.S, P = g.P, K = g.K, nt = 2 * K;
    float2* sw = sm;                          // [win][E]
    float2* accL = sm + (size_t)win * E;      // [S][dzt][P]
    const int tile = blockIdx.x, bt = blockIdx.y, f = blockIdx.z >> 1, fam = blockIdx.z & 1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int LW = (N + 31) >> 5;
    const int RG = (blockDim.x >> 5) / LW;
    const int lw = warp % LW, rg = warp / LW;
    const int l = lw * 32 + lane;
    const int i0 = tile * dzt;
    const int iend = min(i0 + dzt, g.nz);
    const int qmax = (g.ns - 1) << 16;
    for (int idx = threadIdx.x; idx < S * dzt * P; idx += blockDim.x) accL[idx] = make_float2(0.f, 0.f);
    float2 accT[MAXR];
#pragma unroll
    for (int j = 0; j < MAXR; ++j) accT[j] = make_float2(0.f, 0.f);
    for (int kk = 0; kk < K; ++kk) {
        const int k = fam * K + kk;
        const size_t blk = ((size_t)f * nt + k) * g.ns;
        for (int u = bt * P; u < bt * P + P; ++u) {
            const int* txr = dtx_q16 + ((size_t)k * N + u) * g.nz;
            int lo = 1 << 30;
            for (int i = i0; i < iend; ++i) lo = min(lo, (__ldg(txr + i) + __ldg(rx_q16 + (size_t)i * g.us * N)) >> 16);
            __syncthreads();
            for (int idx = threadIdx.x; idx < win * E; idx += blockDim.x) {
                int rr = idx / E, e = idx - rr * E;
                int n = lo + rr;
                float2 v = make_float2(0.f, 0.f);
                if (n >= 0 && n < g.ns) v = load_c(iq, (blk + n) * E + e, iq_t);
                sw[idx] = v;
            }
            __syncthreads();
#pragma unroll
            for (int j = 0; j < MAXR; ++j) {
                const int i = i0 + rg + j * RG;
                float2 v = make_float2(0.f, 0.f);
                if (i < iend) {
                    const int r = i * g.us;
                    const int tq = __ldg(txr + i);
                    const int dend = __ldg(dmax + r) + 1;
                    const int* rxr = rx_q16 + (size_t)r * N;
                    const float2* wr = W + (size_t)r * N;
                    for (int d = 0; d < dend; ++d) {
                        const int q = tq + __ldg(rxr + d);
                        if (q < 0 || q > qmax) continue;
                        const int n = (q >> 16) - lo;
                        const float fr = (float)(q & 0xffff) * (1.0f / 65536.0f);
                        const float2 w = __ldg(wr + d);
                        const float2* row0 = sw + n * E;
                        const int e1 = l - d;
                        if (e1 >= 0 && l < N) {
                            float2 b0 = row0[e1], b1 = row0[E + e1];
                            cfma(v, w, make_float2(fmaf(fr, b1.x - b0.x, b0.x), fmaf(fr, b1.y - b0.y, b0.y)));
                        }
                        const int e2 = l + d;
                        if (d > 0 && e2 < E) {
                            float2 b0 = row0[e2], b1 = row0[E + e2];
                            cfma(v, w, make_float2(fmaf(fr, b1.x - b0.x, b0.x), fmaf(fr, b1.y - b0.y, b0.y)));
                        }
                    }
                    v = cmul(v, __ldg(dtx_ph + ((size_t)k * N + u) * g.nz + i));
                }
                if (l >= N) v = make_float2(0.f, 0.f);
                accT[j].x += v.x;
                accT[j].y += v.y;
                // sum over the P lateral pixels of each lateral slab (P divides 32)
                float2 sv = v;
                for (int o = 1; o < P; o <<= 1) {
                    sv.x += __shfl_xor_sync(0xffffffffu, sv.x, o);
                    sv.y += __shfl_xor_sync(0xffffffffu, sv.y, o);
                }
                if (i < iend && (lane % P) == 0 && l < N) {
                    float2* dst = accL + ((size_t)(l / P) * dzt + (i - i0)) * P + (u - bt * P);
                    dst->x += sv.x;
                    dst->y += sv.y;
                }
            }
        }
    }
    __syncthreads();
    const int axT = fam == 0 ? 0 : 1;
    const int axL = 1 - axT;
    const size_t plane_sz = (size_t)g.nz * N;
#pragma unroll
    for (int j = 0; j < MAXR; ++j) {
        const int i = i0 + rg + j * RG;
        if (i < iend && l < N)
            store_c(planes, ((((size_t)f * 2 + axT) * 2 + fam) * S + bt) * plane_sz + (size_t)i * N + l, pt, accT[j]);
    }
    for (int idx = threadIdx.x; idx < S * dzt * P; idx += blockDim.x) {
        const int uu = idx % P, ii = (idx / P) % dzt, bl = idx / (P * dzt);
        const int i = i0 + ii;
        if (i >= iend) continue;
        store_c(planes, ((((size_t)f * 2 + axL) * 2 + fam) * S + bl) * plane_sz + (size_t)i * N + bt * P + uu, pt,
                accL[idx]);
    }
}

inline bool complex_dtype(rca_dtype t) { return t == RCA_C32 || t == RCA_C16F || t == RCA_C16BF; }


// ---------------------------------------------------------------------------
// Persistent batched beamforming.  Every CTA repeatedly takes the next work
// unit from a device queue (mean units of all ensembles first, then per
// ensemble demodulation, Stage 1 and Stage 2 units), waits -- bounded -- until
// the unit's inputs are complete (per-ensemble counters), runs the same body
// as the standalone kernel, and publishes its completion.  Units only wait
// on units earlier in the queue, which were taken by CTAs already running,
// so the queue always drains.  A wait that runs out sets ST_TIMEOUT and an
// abort flag that stops every CTA at its next unit.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int ld_acquire(const int* p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void mbar_inval(uint64_t* bar)
{
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}

template <typename TS, int MAXR, int ZP>
__global__ void __launch_bounds__(256, 2) k_batch(const BatchEns* __restrict__ ens, const int4* __restrict__ segs,
                                                 int nseg, int total, int* __restrict__ cnt, int n_counters,
                                                 long long wait_limit, Fir fir, int rf_t, int iq_t, int pt,
                                                 unsigned* __restrict__ status)
{
    extern __shared__ __align__(128) unsigned char smraw[];
    __shared__ uint64_t bars[2];
    __shared__ int s_unit, s_ok;
    int* next = cnt + n_counters;
    int* abort_flag = cnt + n_counters + 1;
    for (;;) {
        if (threadIdx.x == 0) s_unit = atomicAdd(next, 1);
        __syncthreads();
        const int u = s_unit;
        if (u >= total) break;
        int sg = 0;
        while (sg + 1 < nseg && segs[sg + 1].z <= u) ++sg;
        const int4 SG = segs[sg];
        const int stage = SG.x, e = SG.y, loc = u - SG.z;
        const BatchEns& E = ens[e];
        const GeomDev& g = E.g;
        const int nt = 2 * g.K;
        // decode the unit, its dependency and the counter it completes
        int dep = -1, dep_target = 0, done = -1;
        int a0 = 0, a1 = 0, a2 = 0;
        if (stage == BS_MEAN) {
            a0 = loc;
            done = E.cA;
        } else if (stage == BS_DEMOD) {
            const int nbx = (g.ns + DM_NT - 1) / DM_NT, nby = (g.N + DM_NE - 1) / DM_NE;
            a0 = loc % nbx;
            a1 = (loc / nbx) % nby;
            a2 = loc / (nbx * nby);  // f * nt + k
            dep = E.cA;
            dep_target = E.nA;
            done = E.cB0 + a2;
        } else if (stage == BS_STAGE1) {
            a0 = loc % E.n_tiles;                // tile
            a1 = (loc / E.n_tiles) % nt;         // k
            a2 = loc / (E.n_tiles * nt);         // f
            dep = E.cB0 + a2 * nt + a1;
            dep_target = E.nB_fk;
            done = E.cC0 + a2;
        } else {
            a0 = loc % E.n_tiles2;               // tile
            a1 = (loc / E.n_tiles2) % 2;         // family
            a2 = loc / (E.n_tiles2 * 2);         // f
            dep = E.cC0 + a2;
            dep_target = E.n_tiles * nt;
        }
        if (threadIdx.x == 0) {
            int ok = 1;
            if (dep >= 0) {
                const long long t0 = clock64();
                while (ld_acquire(cnt + dep) < dep_target) {
                    if (*(volatile int*)abort_flag) {
                        ok = 0;
                        break;
                    }
                    if (clock64() - t0 > wait_limit) {
                        atomicOr(status, ST_TIMEOUT);
                        atomicExch(abort_flag, 1);
                        ok = 0;
                        break;
                    }
                    __nanosleep(200);
                }
                // order the producers' global writes before this CTA's TMA reads
                asm volatile("fence.proxy.async.global;" ::: "memory");
            }
            if (*(volatile int*)abort_flag) ok = 0;
            s_ok = ok;
        }
        __syncthreads();
        if (!s_ok) break;
        bool ok = true;
        if (stage == BS_MEAN) {
            mean_body(a0, E.rf, rf_t, E.scale, E.F, g.ns, nt * g.N * g.ns, E.mean);
        } else if (stage == BS_DEMOD) {
            demod_body(a0, a1, a2, reinterpret_cast<float2*>(smraw), E.rf, rf_t, E.scale, E.mean, E.mix, fir, nt, g.N,
                       g.ns, E.iq, iq_t);
        } else if (stage == BS_STAGE1) {
            ok = stage1_body<TS, MAXR>(a0, a1, a2, smraw, bars, g, E.iq, E.tx_q16, E.rx_q16, E.W, E.dmax, E.chunks,
                                       E.zt, E.dc, E.n_tiles, E.nch, E.win, E.slices, status);
        } else {
            ok = stage2_body<ZP>(a0, a1, a2, E.zp, reinterpret_cast<float2*>(smraw), &bars[0], g, E.slices, E.sfl,
                                 E.sfr, E.psi, E.ec, E.coef, E.tmin, E.T, E.rows, E.smin0, E.smin1, E.planes, pt,
                                 status);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            if (stage == BS_STAGE1) {
                mbar_inval(&bars[0]);
                mbar_inval(&bars[1]);
            } else if (stage == BS_STAGE2) {
                mbar_inval(&bars[0]);
            }
            if (!ok) {
                atomicExch(abort_flag, 1);
            } else if (done >= 0) {
                __threadfence();
                atomicAdd(cnt + done, 1);
            }
        }
        if (!ok) break;
    }
}

}  // namespace

rca_status launch_ingest(rca_handle* h, const rca_tables* t, const void* rf, rca_dtype rf_t, const float* scale, int F,
                         int clutter, void* iq, rca_dtype iq_t)
{
    const GeomDev& g = t->gd;
    const int nt = 2 * g.K;
    rca_status st = RCA_OK;
    float* mean = nullptr;
    if (clutter == RCA_CLUTTER_MEAN) {
        const int ncol = nt * g.N * g.ns;
        mean = (float*)ws_get(h, WS_MEAN, (size_t)ncol * sizeof(float), &st);
        if (!mean) return st;
        k_mean<<<(ncol / 4 + 255) / 256, 256, 0, h->stream>>>(rf, rf_t, scale, F, g.ns, ncol, mean);
    }
    Fir fir;
    for (int q = 0; q < 31; ++q) fir.h[q] = t->fir[q];
    dim3 grid((g.ns + DM_NT - 1) / DM_NT, (g.N + DM_NE - 1) / DM_NE, F * nt);
    k_demod<<<grid, 256, 0, h->stream>>>(rf, rf_t, scale, mean, t->mix, fir, nt, g.N, g.ns, iq, iq_t);
    return cuda_check(h, cudaGetLastError(), "ingest kernels");
}

// Lateral pixels across the lanes of LW warps, rows across RG warp groups:
// 32 * LW * RG <= 256 threads, each thread owning ceil(zt / RG) rows.
static void warp_layout(int N, int zt, int* LW, int* RG, int* per)
{
    *LW = (N + 31) / 32;
    *RG = std::max(1, 8 / *LW);
    *per = (zt + *RG - 1) / *RG;
}

template <typename TS, int MAXR>
static rca_status stage1_launch(rca_handle* h, const rca_tables* t, const void* iq, int F, float2* slices,
                                int threads)
{
    const GeomDev& g = t->gd;
    const Stage1Plan& p = t->s1;
    size_t smem = 2 * (size_t)p.win * g.N * sizeof(TS) + 2 * (size_t)p.zt * p.dc * sizeof(RowD) +
                  2 * (size_t)p.zt * sizeof(int);
    auto kern = k_stage1<TS, MAXR>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_check(h, e, "stage1 smem attribute");
    dim3 grid(p.n_tiles, 2 * g.K, F);
    kern<<<grid, threads, smem, h->stream>>>(g, iq, t->tx_q16, t->rx_q16, t->W, t->dmax, p.d_chunks, p.zt, p.dc,
                                             p.n_tiles, p.nch, p.win, slices, h->d_status);
    return cuda_check(h, cudaGetLastError(), "stage1 kernel");
}

template <typename TS>
static rca_status stage1_dispatch(rca_handle* h, const rca_tables* t, const void* iq, int F, float2* slices)
{
    const GeomDev& g = t->gd;
    int LW, RG, per;
    warp_layout(g.N, t->s1.zt, &LW, &RG, &per);
    if (LW > 8) return set_error(h, RCA_ERR_UNSUPPORTED, "n_el > 256 is not supported");
    const int threads = 32 * LW * RG;
    if (per <= 2) return stage1_launch<TS, 2>(h, t, iq, F, slices, threads);
    if (per <= 4) return stage1_launch<TS, 4>(h, t, iq, F, slices, threads);
    if (per <= 8) return stage1_launch<TS, 8>(h, t, iq, F, slices, threads);
    if (per <= 16) return stage1_launch<TS, 16>(h, t, iq, F, slices, threads);
    return set_error(h, RCA_ERR_UNSUPPORTED, "Stage-1 row tile too tall");
}

rca_status launch_stage1(rca_handle* h, const rca_tables* t, const void* iq, rca_dtype iq_t, int F, float2* slices)
{
    if (iq_t == RCA_C32) return stage1_dispatch<float2>(h, t, iq, F, slices);
    if (iq_t == RCA_C16F) return stage1_dispatch<__half2>(h, t, iq, F, slices);
    if (iq_t == RCA_C16BF) return stage1_dispatch<__nv_bfloat162>(h, t, iq, F, slices);
    return set_error(h, RCA_ERR_UNSUPPORTED, "iq dtype must be C32, C16F or C16BF");
}

template <int ZP>
static rca_status stage2_launch(rca_handle* h, const rca_tables* t, const float2* slices, int F, void* planes,
                                rca_dtype pt)
{
    const GeomDev& g = t->gd;
    const int rows = t->s2.rows, K = g.K, S = g.S, T = t->T;
    size_t smem = ((size_t)K * rows * g.N + (size_t)K * S * rows + (size_t)K * S * ZP * T + (size_t)K * g.N +
                   (size_t)K * ZP) * sizeof(float2) +
                  ((size_t)2 * K * g.N + (size_t)K * S) * sizeof(int);
    auto kern = k_stage2<ZP>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_check(h, e, "stage2 smem attribute");
    dim3 grid(t->s2.n_tiles, 2, F);
    kern<<<grid, 512, smem, h->stream>>>(g, slices, t->s2_sfl, t->s2_sfr, t->s2_psi, t->s2_ec, t->s2_coef, t->s2_tmin,
                                         T, rows, t->s2.smin[0], t->s2.smin[1], planes, (int)pt, h->d_status);
    return cuda_check(h, cudaGetLastError(), "stage2 kernel");
}

rca_status launch_stage2(rca_handle* h, const rca_tables* t, const float2* slices, int F, void* planes, rca_dtype pt)
{
    if (!complex_dtype(pt)) return set_error(h, RCA_ERR_UNSUPPORTED, "planes dtype must be C32, C16F or C16BF");
    switch (t->s2.zp) {
    case 1: return stage2_launch<1>(h, t, slices, F, planes, pt);
    case 2: return stage2_launch<2>(h, t, slices, F, planes, pt);
    case 4: return stage2_launch<4>(h, t, slices, F, planes, pt);
    case 8: return stage2_launch<8>(h, t, slices, F, planes, pt);
    default: return stage2_launch<16>(h, t, slices, F, planes, pt);
    }
}

template <int MAXR>
static rca_status direct_launch(rca_handle* h, const rca_tables* t, const void* iq, rca_dtype iq_t, int F,
                                void* planes, rca_dtype pt, int threads)
{
    const GeomDev& g = t->gd;
    const int dzt = t->direct_zt, win = t->direct_win;
    size_t smem = ((size_t)win * g.N + (size_t)g.S * dzt * g.P) * sizeof(float2);
    auto kern = k_direct<MAXR>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_check(h, e, "direct smem attribute");
    dim3 grid((g.nz + dzt - 1) / dzt, g.S, 2 * F);
    kern<<<grid, threads, smem, h->stream>>>(g, iq, iq_t, t->dtx_q16, t->dtx_ph, t->rx_q16, t->W, t->dmax, dzt, win,
                                             planes, (int)pt);
    return cuda_check(h, cudaGetLastError(), "direct kernel");
}

rca_status launch_direct(rca_handle* h, const rca_tables* t, const void* iq, rca_dtype iq_t, int F, void* planes,
                         rca_dtype pt)
{
    const GeomDev& g = t->gd;
    if (!complex_dtype(pt)) return set_error(h, RCA_ERR_UNSUPPORTED, "planes dtype must be C32, C16F or C16BF");
    if (32 % g.P != 0) return set_error(h, RCA_ERR_UNSUPPORTED, "direct mode needs P dividing 32");
    int LW, RG, per;
    warp_layout(g.N, t->direct_zt, &LW, &RG, &per);
    if (LW > 8) return set_error(h, RCA_ERR_UNSUPPORTED, "n_el > 256 is not supported");
    const int threads = 32 * LW * RG;
    if (per <= 2) return direct_launch<2>(h, t, iq, iq_t, F, planes, pt, threads);
    if (per <= 4) return direct_launch<4>(h, t, iq, iq_t, F, planes, pt, threads);
    if (per <= 8) return direct_launch<8>(h, t, iq, iq_t, F, planes, pt, threads);
    if (per <= 16) return direct_launch<16>(h, t, iq, iq_t, F, planes, pt, threads);
    return set_error(h, RCA_ERR_UNSUPPORTED, "direct row tile too tall");
}

// ---------------------------------------------------------------------------
// batched launch
// ---------------------------------------------------------------------------
template <typename TS, int MAXR, int ZP>
static rca_status batch_launch(rca_handle* h, rca_batch* b)
{
    auto kern = k_batch<TS, MAXR, ZP>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem);
    if (e != cudaSuccess) return cuda_check(h, e, "batch smem attribute");
    if (b->grid == 0) {
        int per_sm = 0, dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, b->smem);
        b->grid = std::max(1, per_sm) * sms;
    }
    Fir fir;
    for (int q = 0; q < 31; ++q) fir.h[q] = b->fir[q];
    cudaMemsetAsync(b->d_cnt, 0, sizeof(int) * (b->n_counters + 2), h->stream);
    kern<<<b->grid, 256, b->smem, h->stream>>>(b->d_ens, b->d_segs, (int)b->segs.size(), b->total, b->d_cnt,
                                               b->n_counters, b->wait_limit, fir, (int)b->rf_t, (int)b->iq_t,
                                               (int)b->pl_t, h->d_status);
    return cuda_check(h, cudaGetLastError(), "batch kernel");
}

template <typename TS, int MAXR>
static rca_status batch_zp(rca_handle* h, rca_batch* b)
{
    switch (b->zpmax) {
    case 1: return batch_launch<TS, MAXR, 1>(h, b);
    case 2: return batch_launch<TS, MAXR, 2>(h, b);
    case 4: return batch_launch<TS, MAXR, 4>(h, b);
    case 8: return batch_launch<TS, MAXR, 8>(h, b);
    default: return batch_launch<TS, MAXR, 16>(h, b);
    }
}

template <typename TS>
static rca_status batch_maxr(rca_handle* h, rca_batch* b)
{
    if (b->maxr <= 2) return batch_zp<TS, 2>(h, b);
    if (b->maxr <= 4) return batch_zp<TS, 4>(h, b);
    if (b->maxr <= 8) return batch_zp<TS, 8>(h, b);
    return batch_zp<TS, 16>(h, b);
}

rca_status launch_batch(rca_handle* h, rca_batch* b)
{
    if (b->iq_t == RCA_C32) return batch_maxr<float2>(h, b);
    if (b->iq_t == RCA_C16F) return batch_maxr<__half2>(h, b);
    return batch_maxr<__nv_bfloat162>(h, b);
}
