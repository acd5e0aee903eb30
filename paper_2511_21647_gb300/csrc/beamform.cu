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

// One thread per (tx, element, sample) column; frames are strided by ncol.
// float / half input: Neumaier-compensated float sum; int16: exact integer sum.
__global__ void k_mean(const void* __restrict__ rf, int rf_t, const float* __restrict__ scale, int F, int ns,
                       int ncol, float* __restrict__ mean)
{
    int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= ncol) return;
    const size_t stride = (size_t)ncol;
    if (rf_t == RCA_I16) {
        const int16_t* q = reinterpret_cast<const int16_t*>(rf);
        long long acc = 0;
        for (int f = 0; f < F; ++f) acc += q[(size_t)f * stride + col];
        mean[col] = (float)((double)acc / (double)F * (double)scale[col / ns]);
        return;
    }
    float s = 0.f, c = 0.f;
    for (int f = 0; f < F; ++f) {
        float x = rf_value(rf, rf_t, (size_t)f * stride + col);
        float t = s + x;
        c += (fabsf(s) >= fabsf(x)) ? ((s - t) + x) : ((x - t) + s);
        s = t;
    }
    mean[col] = (s + c) / (float)F;
}

#define DM_NT 128           // samples per CTA
#define DM_NE 32            // elements per CTA
#define DM_PITCH (DM_NT + 31)  // odd float2 pitch: conflict-free column reads

// CTA = (128 samples, 32 elements, one frame-transmission).  Reads RF rows
// [e][n] coalesced along n, writes IQ [n][e] coalesced along e.
__global__ void __launch_bounds__(256) k_demod(const void* __restrict__ rf, int rf_t, const float* __restrict__ scale,
                                               const float* __restrict__ mean, const float2* __restrict__ mix, Fir fir,
                                               int nt, int E, int ns, void* __restrict__ iq, int iq_t)
{
    __shared__ float2 xs[DM_NE * DM_PITCH];
    const int n0 = blockIdx.x * DM_NT;
    const int e0 = blockIdx.y * DM_NE;
    const int fk = blockIdx.z;
    const int k = fk % nt;
    const size_t chan0 = (size_t)fk * E;
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
// sample row: the delay, its fraction and the weight are warp-uniform.
// ---------------------------------------------------------------------------
template <int MAXR>
__global__ void __launch_bounds__(256) k_stage1(GeomDev g, const void* __restrict__ iq, int iq_t,
                                                    const int* __restrict__ tx_q16, const int* __restrict__ rx_q16,
                                                    const float2* __restrict__ W, const int* __restrict__ dmax,
                                                    const int4* __restrict__ chunks, int zt, int n_tiles, int nch,
                                                    float2* __restrict__ slices)
{
    extern __shared__ float2 sw[];  // [nrows][E]
    const int E = g.N, N = g.N;
    const int tile = blockIdx.x, k = blockIdx.y, f = blockIdx.z;
    const int nt = 2 * g.K;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int LW = (N + 31) >> 5;
    const int RG = (blockDim.x >> 5) / LW;
    const int lw = warp % LW, rg = warp / LW;
    const int l = lw * 32 + lane;
    const int r0 = tile * zt;
    const int rend = min(r0 + zt, g.nzs);
    float2 acc[MAXR];
#pragma unroll
    for (int j = 0; j < MAXR; ++j) acc[j] = make_float2(0.f, 0.f);
    const size_t blk = ((size_t)f * nt + k) * g.ns;
    const int qmax = (g.ns - 1) << 16;
    const int4* ch = chunks + ((size_t)k * n_tiles + tile) * nch;
    for (int c = 0; c < nch; ++c) {
        const int4 cc = ch[c];  // {nlo, nrows, d0, d1}
        if (cc.y == 0) continue;
        __syncthreads();
        const int total = cc.y * E;
        for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
            int rr = idx / E, e = idx - rr * E;
            int n = cc.x + rr;
            float2 v = make_float2(0.f, 0.f);
            if (n >= 0 && n < g.ns) v = load_c(iq, (blk + n) * E + e, iq_t);
            sw[idx] = v;
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < MAXR; ++j) {
            const int r = r0 + rg + j * RG;
            if (r < rend) {
                const int tq = __ldg(tx_q16 + (size_t)k * g.nzs + r);
                const int dend = min(cc.w, __ldg(dmax + r) + 1);
                const int* rxr = rx_q16 + (size_t)r * N;
                const float2* wr = W + (size_t)r * N;
                float2 a = acc[j];
                for (int d = cc.z; d < dend; ++d) {
                    const int q = tq + __ldg(rxr + d);
                    if (q < 0 || q > qmax) continue;
                    const int n = (q >> 16) - cc.x;
                    const float fr = (float)(q & 0xffff) * (1.0f / 65536.0f);
                    const float2 w = __ldg(wr + d);
                    const float2* row0 = sw + n * E;
                    const int e1 = l - d;
                    if (e1 >= 0 && l < N) {
                        float2 b0 = row0[e1], b1 = row0[E + e1];
                        float2 v = make_float2(fmaf(fr, b1.x - b0.x, b0.x), fmaf(fr, b1.y - b0.y, b0.y));
                        cfma(a, w, v);
                    }
                    const int e2 = l + d;
                    if (d > 0 && e2 < E) {
                        float2 b0 = row0[e2], b1 = row0[E + e2];
                        float2 v = make_float2(fmaf(fr, b1.x - b0.x, b0.x), fmaf(fr, b1.y - b0.y, b0.y));
                        cfma(a, w, v);
                    }
                }
                acc[j] = a;
            }
        }
    }
#pragma unroll
    for (int j = 0; j < MAXR; ++j) {
        const int r = r0 + rg + j * RG;
        if (r < rend && l < N) slices[(((size_t)f * nt + k) * g.nzs + r) * N + l] = acc[j];
    }
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
__global__ void __launch_bounds__(256) k_stage2(GeomDev g, const float2* __restrict__ slices,
                                                const int* __restrict__ sfl, const float* __restrict__ sfr,
                                                const float2* __restrict__ psi, const float2* __restrict__ ec,
                                                const float2* __restrict__ coef, const int* __restrict__ tmin, int T,
                                                int zp, int rows, int smin0, int smin1, void* __restrict__ planes,
                                                int pt)
{
    extern __shared__ float2 sm[];
    const int N = g.N, K = g.K, S = g.S, P = g.P, us = g.us;
    const int tile = blockIdx.x, fam = blockIdx.y, f = blockIdx.z;
    const int nt = 2 * K;
    const int i0 = tile * zp;
    const int iend = min(i0 + zp, g.nz);
    const int rlo = us * i0 + (fam ? smin1 : smin0);
    float2* sS = sm;                            // [K][rows][N]
    float2* sSum = sm + (size_t)K * rows * N;   // [K][S][rows]
    for (int idx = threadIdx.x; idx < K * rows * N; idx += blockDim.x) {
        int kk = idx / (rows * N), rr = (idx / N) % rows, l = idx % N;
        int row = rlo + rr;
        float2 v = make_float2(0.f, 0.f);
        if (row >= 0 && row < g.nzs) v = slices[(((size_t)f * nt + fam * K + kk) * g.nzs + row) * N + l];
        sS[idx] = v;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < K * S * rows; idx += blockDim.x) {
        int kk = idx / (S * rows), b = (idx / rows) % S, rr = idx % rows;
        const float2* src = sS + ((size_t)kk * rows + rr) * N + b * P;
        float2 a = make_float2(0.f, 0.f);
        for (int q = 0; q < P; ++q) {
            a.x += src[q].x;
            a.y += src[q].y;
        }
        sSum[idx] = a;
    }
    __syncthreads();
    const int axT = fam == 0 ? 0 : 1;
    const int axL = 1 - axT;
    const size_t plane_sz = (size_t)g.nz * N;
    const int nout = S * zp * N;
    for (int idx = threadIdx.x; idx < nout; idx += blockDim.x) {
        const int l = idx % N, ii = (idx / N) % zp, b = idx / (N * zp);
        const int i = i0 + ii;
        if (i >= iend) continue;
        float2 acc = make_float2(0.f, 0.f);
        for (int kk = 0; kk < K; ++kk) {
            const int k = fam * K + kk;
            const int base = us * i + __ldg(tmin + k * S + b) - rlo;
            const float2* cf = coef + (((size_t)k * S + b) * g.nz + i) * T;
            const float2* src = sS + ((size_t)kk * rows + base) * N + l;
            for (int t = 0; t < T; ++t) cfma(acc, __ldg(cf + t), src[(size_t)t * N]);
        }
        store_c(planes, ((((size_t)f * 2 + axT) * 2 + fam) * S + b) * plane_sz + (size_t)i * N + l, pt, acc);
    }
    for (int idx = threadIdx.x; idx < nout; idx += blockDim.x) {
        const int u = idx % N, ii = (idx / N) % zp, b = idx / (N * zp);
        const int i = i0 + ii;
        if (i >= iend) continue;
        float2 acc = make_float2(0.f, 0.f);
        for (int kk = 0; kk < K; ++kk) {
            const int k = fam * K + kk;
            const int n0 = us * i + __ldg(sfl + k * N + u);
            const float fr = __ldg(sfr + k * N + u);
            const bool valid = n0 >= 0 && (n0 < g.nzs - 1 || (n0 == g.nzs - 1 && fr == 0.f));
            if (!valid) continue;
            const float2* src = sSum + ((size_t)kk * S + b) * rows + (n0 - rlo);
            const float2 s0 = src[0], s1 = src[1];
            const float2 v = make_float2(fmaf(fr, s1.x - s0.x, s0.x), fmaf(fr, s1.y - s0.y, s0.y));
            cfma(acc, cmul(__ldg(ec + (size_t)k * g.nz + i), __ldg(psi + (size_t)k * N + u)), v);
        }
        store_c(planes, ((((size_t)f * 2 + axL) * 2 + fam) * S + b) * plane_sz + (size_t)i * N + u, pt, acc);
    }
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
        k_mean<<<(ncol + 255) / 256, 256, 0, h->stream>>>(rf, rf_t, scale, F, g.ns, ncol, mean);
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

template <int MAXR>
static rca_status stage1_launch(rca_handle* h, const rca_tables* t, const void* iq, rca_dtype iq_t, int F,
                                float2* slices, int threads)
{
    const GeomDev& g = t->gd;
    size_t smem = (size_t)t->s1.win * g.N * sizeof(float2);
    auto kern = k_stage1<MAXR>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_check(h, e, "stage1 smem attribute");
    dim3 grid(t->s1.n_tiles, 2 * g.K, F);
    kern<<<grid, threads, smem, h->stream>>>(g, iq, iq_t, t->tx_q16, t->rx_q16, t->W, t->dmax, t->s1.d_chunks,
                                             t->s1.zt, t->s1.n_tiles, t->s1.nch, slices);
    return cuda_check(h, cudaGetLastError(), "stage1 kernel");
}

rca_status launch_stage1(rca_handle* h, const rca_tables* t, const void* iq, rca_dtype iq_t, int F, float2* slices)
{
    const GeomDev& g = t->gd;
    int LW, RG, per;
    warp_layout(g.N, t->s1.zt, &LW, &RG, &per);
    if (LW > 8) return set_error(h, RCA_ERR_UNSUPPORTED, "n_el > 256 is not supported");
    const int threads = 32 * LW * RG;
    if (per <= 2) return stage1_launch<2>(h, t, iq, iq_t, F, slices, threads);
    if (per <= 4) return stage1_launch<4>(h, t, iq, iq_t, F, slices, threads);
    if (per <= 8) return stage1_launch<8>(h, t, iq, iq_t, F, slices, threads);
    if (per <= 16) return stage1_launch<16>(h, t, iq, iq_t, F, slices, threads);
    return set_error(h, RCA_ERR_UNSUPPORTED, "Stage-1 row tile too tall");
}

rca_status launch_stage2(rca_handle* h, const rca_tables* t, const float2* slices, int F, void* planes, rca_dtype pt)
{
    const GeomDev& g = t->gd;
    if (!complex_dtype(pt)) return set_error(h, RCA_ERR_UNSUPPORTED, "planes dtype must be C32, C16F or C16BF");
    const int rows = t->s2.rows;
    size_t smem = ((size_t)g.K * rows * g.N + (size_t)g.K * g.S * rows) * sizeof(float2);
    cudaError_t e = cudaFuncSetAttribute(k_stage2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_check(h, e, "stage2 smem attribute");
    dim3 grid(t->s2.n_tiles, 2, F);
    k_stage2<<<grid, 256, smem, h->stream>>>(g, slices, t->s2_sfl, t->s2_sfr, t->s2_psi, t->s2_ec, t->s2_coef,
                                             t->s2_tmin, t->T, t->s2.zp, rows, t->s2.smin[0], t->s2.smin[1], planes,
                                             (int)pt);
    return cuda_check(h, cudaGetLastError(), "stage2 kernel");
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
