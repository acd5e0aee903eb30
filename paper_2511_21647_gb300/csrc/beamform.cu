// beamform.cu -- channel data -> IQ -> Stage-1 slices -> projection planes.
//
// Sec. II-A1 (two-stage RCA beamforming, Fig. 1b-c), Sec. II-A4/II-A5
// (P x P x N sub-blocks sum-projected onto x-z and y-z planes), Sec. II-A2
// (clutter removal before Stage 2; here the ensemble-mean filter).
#include "beamform_body.cuh"

namespace {

__global__ void __launch_bounds__(256) k_mean(const void* __restrict__ rf, int rf_t, const float* __restrict__ scale,
                                              int F, int ns, int ncol, float* __restrict__ mean)
{
    mean_body(blockIdx.x, rf, rf_t, scale, F, ns, ncol, mean);
}

template <int RT>
__global__ void __launch_bounds__(256, 4) k_demod(const void* __restrict__ rf, const float* __restrict__ scale,
                                                  const float* __restrict__ mean, const float2* __restrict__ mix,
                                                  Fir fir, int nt, int E, int ns, void* __restrict__ iq, int iq_t)
{
    __shared__ float2 xs[DM_NE * DM_PITCH];
    demod_body<RT>(blockIdx.x, blockIdx.y, blockIdx.z, xs, rf, scale, mean, mix, fir, nt, E, ns, iq, iq_t);
}

template <typename TS, int MAXR, bool PAIR>
__global__ void __launch_bounds__(256, 2) k_stage1(GeomDev g, const void* __restrict__ iq,
                                                const unsigned char* __restrict__ rtab, int rblk,
                                                const int* __restrict__ dmax, const int4* __restrict__ chunks, int zt,
                                                int dc, int n_tiles, int nch, int ring, float2* __restrict__ slices,
                                                unsigned* __restrict__ status)
{
    extern __shared__ __align__(128) unsigned char smraw[];
    __shared__ uint64_t bars[2];
    stage1_body<TS, MAXR, true, PAIR>(blockIdx.x, blockIdx.y, blockIdx.z, smraw, bars, g, iq, rtab, rblk, dmax, chunks, zt,
                                dc, n_tiles, nch, ring, slices, status);
}

template <int TM, int US>
__global__ void __launch_bounds__(S2_THREADS, 3) k_stage2(GeomDev g, const float2* __restrict__ slices,
                                                       const int* __restrict__ sfl, const float* __restrict__ sfr,
                                                       const float4* __restrict__ lw, const float2* __restrict__ rot,
                                                       const float2* __restrict__ coef, const float2* __restrict__ c2,
                                                       const int* __restrict__ tmin, int T, int iA, int iB, int zp,
                                                       int rows, int smin0, int smin1, void* __restrict__ planes,
                                                       int pt, unsigned* __restrict__ status)
{
    extern __shared__ __align__(128) unsigned char smraw[];
    __shared__ uint64_t bar;
    stage2_body<TM, US>(blockIdx.x, blockIdx.y, blockIdx.z & 1, blockIdx.z >> 1, smraw, &bar, g, slices, sfl, sfr, lw, rot,
                    coef, c2, tmin, T, iA, iB, zp, rows, smin0, smin1, planes, pt, status);
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
    if (rf_t == RCA_F32)
        k_demod<RCA_F32><<<grid, 256, 0, h->stream>>>(rf, scale, mean, t->mix, fir, nt, g.N, g.ns, iq, iq_t);
    else if (rf_t == RCA_F16)
        k_demod<RCA_F16><<<grid, 256, 0, h->stream>>>(rf, scale, mean, t->mix, fir, nt, g.N, g.ns, iq, iq_t);
    else
        k_demod<RCA_I16><<<grid, 256, 0, h->stream>>>(rf, scale, mean, t->mix, fir, nt, g.N, g.ns, iq, iq_t);
    return cuda_check(h, cudaGetLastError(), "ingest kernels");
}

template <typename TS, int MAXR, bool PAIR>
static rca_status stage1_launch(rca_handle* h, const rca_tables* t, const void* iq, int F, float2* slices,
                                int threads)
{
    const GeomDev& g = t->gd;
    const Stage1Plan& p = t->s1;
    const size_t smem = stage1_smem_bytes(t, p.zt, p.dc, p.ring, sizeof(TS));
    auto kern = k_stage1<TS, MAXR, PAIR>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_check(h, e, "stage1 smem attribute");
    dim3 grid(p.n_tiles, 2 * g.K, F);
    const unsigned char* rtab = std::is_same<TS, __half2>::value ? p.d_rec16 : p.d_rec32;
    kern<<<grid, threads, smem, h->stream>>>(g, iq, rtab, p.rblk, t->dmax, p.d_chunks, p.zt, p.dc, p.n_tiles, p.nch,
                                             p.ring, slices, h->d_status);
    return cuda_check(h, cudaGetLastError(), "stage1 kernel");
}

template <typename TS>
static rca_status stage1_dispatch(rca_handle* h, const rca_tables* t, const void* iq, int F, float2* slices)
{
    const GeomDev& g = t->gd;
    const S1Layout L = stage1_layout(g.N, t->s1.zt, true);
    if (L.LW > 8) return set_error(h, RCA_ERR_UNSUPPORTED, "n_el > 256 is not supported");
    const int threads = 32 * L.LW * L.RG;
    // the kernel's row loop is exact: every thread owns exactly MAXR rows
    // (or one row, with some warps idle, when the tile has fewer rows than warps)
    if (!(L.per == 1 || L.per * L.RG == t->s1.zt))
        return set_error(h, RCA_ERR_UNSUPPORTED, "Stage-1 row tile %d is not a multiple of %d row groups", t->s1.zt,
                         L.RG);
    if (L.pair) {
        if (L.per == 1) return stage1_launch<TS, 1, true>(h, t, iq, F, slices, threads);
        if (L.per == 2) return stage1_launch<TS, 2, true>(h, t, iq, F, slices, threads);
        if (L.per == 4) return stage1_launch<TS, 4, true>(h, t, iq, F, slices, threads);
        if (L.per == 8) return stage1_launch<TS, 8, true>(h, t, iq, F, slices, threads);
    } else {
        if (L.per == 1) return stage1_launch<TS, 1, false>(h, t, iq, F, slices, threads);
        if (L.per == 2) return stage1_launch<TS, 2, false>(h, t, iq, F, slices, threads);
        if (L.per == 4) return stage1_launch<TS, 4, false>(h, t, iq, F, slices, threads);
        if (L.per == 8) return stage1_launch<TS, 8, false>(h, t, iq, F, slices, threads);
        if (L.per == 16) return stage1_launch<TS, 16, false>(h, t, iq, F, slices, threads);
    }
    return set_error(h, RCA_ERR_UNSUPPORTED, "Stage-1 row tile too tall");
}

rca_status launch_stage1(rca_handle* h, const rca_tables* t, const void* iq, rca_dtype iq_t, int F, float2* slices)
{
    if (iq_t == RCA_C32) return stage1_dispatch<float2>(h, t, iq, F, slices);
    if (iq_t == RCA_C16F) return stage1_dispatch<__half2>(h, t, iq, F, slices);
    if (iq_t == RCA_C16BF) return stage1_dispatch<__nv_bfloat162>(h, t, iq, F, slices);
    return set_error(h, RCA_ERR_UNSUPPORTED, "iq dtype must be C32, C16F or C16BF");
}

template <int TM, int US>
static rca_status stage2_launch(rca_handle* h, const rca_tables* t, const float2* slices, int F, void* planes,
                                rca_dtype pt)
{
    const GeomDev& g = t->gd;
    const int GW = s2_group_width(g.P);
    if (GW == 0) return set_error(h, RCA_ERR_UNSUPPORTED, "Stage 2 needs an even multiple of P (%d) up to 32", g.P);
    if (2 * (long long)F > 65535) return set_error(h, RCA_ERR_UNSUPPORTED, "more than 32767 frames in one call");
    const size_t smem = stage2_smem_bytes(t, t->s2.zp);
    auto kern = k_stage2<TM, US>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_check(h, e, "stage2 smem attribute");
    dim3 grid(t->s2.n_tiles, (g.N + GW - 1) / GW, 2 * F);
    kern<<<grid, S2_THREADS, smem, h->stream>>>(g, slices, t->s2_sfl, t->s2_sfr, t->s2_lw, t->s2_rot, t->s2_coefr,
                                                t->s2_c2r, t->s2_tmin, t->T, t->s2_iA, t->s2_iB, t->s2.zp, t->s2.rows,
                                                t->s2.smin[0], t->s2.smin[1], planes, (int)pt, h->d_status);
    return cuda_check(h, cudaGetLastError(), "stage2 kernel");
}

rca_status launch_stage2(rca_handle* h, const rca_tables* t, const float2* slices, int F, void* planes, rca_dtype pt)
{
    if (!complex_dtype(pt)) return set_error(h, RCA_ERR_UNSUPPORTED, "planes dtype must be C32, C16F or C16BF");
    // exact tap counts of the usual steering ranges with two slice rows per
    // plane row; any other combination runs the generic loop
    if (t->gd.us == 2) {
        if (t->T == 2) return stage2_launch<2, 2>(h, t, slices, F, planes, pt);
        if (t->T == 3) return stage2_launch<3, 2>(h, t, slices, F, planes, pt);
        if (t->T == 4) return stage2_launch<4, 2>(h, t, slices, F, planes, pt);
    }
    return stage2_launch<0, 0>(h, t, slices, F, planes, pt);
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
    const S1Layout L = stage1_layout(g.N, t->direct_zt, false);
    if (L.LW > 8) return set_error(h, RCA_ERR_UNSUPPORTED, "n_el > 256 is not supported");
    const int threads = 32 * L.LW * L.RG;
    const int per = L.per;
    if (per <= 2) return direct_launch<2>(h, t, iq, iq_t, F, planes, pt, threads);
    if (per <= 4) return direct_launch<4>(h, t, iq, iq_t, F, planes, pt, threads);
    if (per <= 8) return direct_launch<8>(h, t, iq, iq_t, F, planes, pt, threads);
    if (per <= 16) return direct_launch<16>(h, t, iq, iq_t, F, planes, pt, threads);
    return set_error(h, RCA_ERR_UNSUPPORTED, "direct row tile too tall");
}

rca_status launch_batch(rca_handle* h, rca_batch* b)
{
    if (b->iq_t == RCA_C32) return launch_batch_c32(h, b);
    if (b->iq_t == RCA_C16F) return launch_batch_c16f(h, b);
    return launch_batch_c16bf(h, b);
}
