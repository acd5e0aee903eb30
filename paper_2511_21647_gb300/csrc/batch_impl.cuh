// batch_impl.cuh -- the persistent batched beamforming kernel, instantiated
// once per IQ dtype (batch_c32.cu, batch_c16f.cu, batch_c16bf.cu) so the
// translation units compile in parallel.
#pragma once
#include "beamform_body.cuh"

namespace {

// ---------------------------------------------------------------------------
// Persistent batched beamforming.  Every CTA repeatedly takes the next work
// unit from a device queue (stage-major: the mean units of all ensembles,
// then all demodulation, all Stage 1 and all Stage 2 units), waits -- bounded -- until
// the unit's inputs are complete (per-ensemble counters), runs the same body
// as the standalone kernel, and publishes its completion.  Units only wait
// on units earlier in the queue, which were taken by CTAs already running,
// so the queue always drains.  A wait that runs out sets ST_TIMEOUT and an
// abort flag that stops every CTA at its next unit.  nowait != 0 (staged
// mode: the queue holds the units of one stage, whose inputs earlier
// launches on the stream completed) skips the waits and the counters.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int ld_acquire(const int* p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}


template <typename TS, int MAXR, int TM, int US>
__global__ void __launch_bounds__(256, 3) k_batch(const BatchEns* __restrict__ ens, const int4* __restrict__ segs,
                                                 int nseg, int total, int* __restrict__ cnt, int n_counters,
                                                 long long wait_limit, Fir fir, int rf_t, int iq_t, int pt,
                                                 int nowait, unsigned* __restrict__ status)
{
    extern __shared__ __align__(128) unsigned char smraw[];
    __shared__ uint64_t bars[2];
    __shared__ int s_unit, s_ok, s_sg, s_cur;
    __shared__ int4 s_seg;
    // the current ensemble's descriptor, copied once per ensemble change
    __shared__ __align__(16) BatchEns sE;
    int* next = cnt + n_counters;
    int* abort_flag = cnt + n_counters + 1;
    if (threadIdx.x == 0) {
        s_sg = 0;
        s_cur = -1;
    }
    for (;;) {
        if (threadIdx.x == 0) {
            const int u = atomicAdd(next, 1);
            s_unit = u;
            if (u < total) {
                // units are taken in increasing order: advance from the last segment
                int sg = s_sg;
                while (sg + 1 < nseg && segs[sg + 1].y <= u) ++sg;
                s_sg = sg;
                s_seg = segs[sg];
            }
        }
        __syncthreads();
        const int u = s_unit;
        if (u >= total) break;
        const int4 SG = s_seg;
        const int stage = SG.x & 15, e = SG.x >> 4, loc = u - SG.y + SG.w;
        // queue segment and ensemble of the unit (checked build)
        if (!chk(SG.y <= u && loc >= 0 && e >= 0 && stage <= BS_STAGE2, status)) break;
        if (e != s_cur) {
            const int* src = reinterpret_cast<const int*>(ens + e);
            int* dst = reinterpret_cast<int*>(&sE);
            for (int i = threadIdx.x; i < (int)(sizeof(BatchEns) / sizeof(int)); i += blockDim.x) dst[i] = src[i];
            __syncthreads();
            if (threadIdx.x == 0) s_cur = e;
        }
        const BatchEns& E = sE;
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
            a1 = (loc / E.n_tiles2) % (2 * E.LG);  // lateral group * 2 + family
            a2 = loc / (E.n_tiles2 * 2 * E.LG);  // f
            dep = E.cC0 + a2;
            dep_target = E.n_tiles * nt;
        }
        if (threadIdx.x == 0) {
            int ok = 1;
            // the counters the unit waits on and completes (checked build)
            if (!chk(dep < n_counters && done < n_counters, status)) ok = 0;
            if (ok && dep >= 0 && !nowait) {
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
            float2* xs = reinterpret_cast<float2*>(smraw);
            if (rf_t == RCA_F32)
                demod_body<RCA_F32>(a0, a1, a2, xs, E.rf, E.scale, E.mean, E.mix, fir, nt, g.N, g.ns, E.iq, iq_t);
            else if (rf_t == RCA_F16)
                demod_body<RCA_F16>(a0, a1, a2, xs, E.rf, E.scale, E.mean, E.mix, fir, nt, g.N, g.ns, E.iq, iq_t);
            else
                demod_body<RCA_I16>(a0, a1, a2, xs, E.rf, E.scale, E.mean, E.mix, fir, nt, g.N, g.ns, E.iq, iq_t);
        } else if (stage == BS_STAGE1) {
            ok = stage1_body<TS, MAXR, false>(a0, a1, a2, smraw, bars, g, E.iq, E.rtab, E.rblk, E.dmax, E.chunks,
                                              E.zt, E.dc, E.n_tiles, E.nch, E.ring, E.slices, status);
        } else {
            ok = stage2_body<TM, US>(a0, a1 >> 1, a1 & 1, a2, smraw, &bars[0], g, E.slices, E.sfl, E.sfr, E.lw, E.rot,
                                 E.coef, E.c2, E.tmin, E.T, E.iA, E.iB, E.zp, E.rows, E.smin0, E.smin1, E.planes, pt,
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
            } else if (done >= 0 && !nowait) {
                __threadfence();
                atomicAdd(cnt + done, 1);
            }
        }
        if (!ok) break;
    }
}


}  // namespace

// ---------------------------------------------------------------------------
// batched launch
// ---------------------------------------------------------------------------
template <typename TS, int MAXR, int TM, int US>
static rca_status batch_launch(rca_handle* h, rca_batch* b)
{
    auto kern = k_batch<TS, MAXR, TM, US>;
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
    if (b->mode == RCA_BATCH_STAGED) {
        // one launch per stage, each sized by its own shared memory
        for (int s = BS_MEAN; s <= BS_STAGE2; ++s) {
            if (b->stotal[s] == 0) continue;
            if (b->sgrid[s] == 0) {
                int per_sm = 0, dev = 0, sms = 0;
                cudaGetDevice(&dev);
                cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, b->ssmem[s]);
                b->sgrid[s] = std::max(1, std::min(b->stotal[s], std::max(1, per_sm) * sms));
            }
            cudaMemsetAsync(b->d_cnt + b->n_counters, 0, sizeof(int) * 2, h->stream);
            kern<<<b->sgrid[s], 256, b->ssmem[s], h->stream>>>(
                b->d_ens, b->d_ssegs + b->sseg0[s], b->sseg0[s + 1] - b->sseg0[s], b->stotal[s], b->d_cnt,
                b->n_counters, b->wait_limit, fir, (int)b->rf_t, (int)b->iq_t, (int)b->pl_t, 1, h->d_status);
            rca_status st = cuda_check(h, cudaGetLastError(), "batch stage kernel");
            if (st != RCA_OK) return st;
        }
        return RCA_OK;
    }
    cudaMemsetAsync(b->d_cnt, 0, sizeof(int) * (b->n_counters + 2), h->stream);
    kern<<<b->grid, 256, b->smem, h->stream>>>(b->d_ens, b->d_segs, (int)b->segs.size(), b->total, b->d_cnt,
                                               b->n_counters, b->wait_limit, fir, (int)b->rf_t, (int)b->iq_t,
                                               (int)b->pl_t, 0, h->d_status);
    return cuda_check(h, cudaGetLastError(), "batch kernel");
}

template <typename TS, int MAXR>
static rca_status batch_tm(rca_handle* h, rca_batch* b)
{
    // one tap count and two slice rows per plane row in every ensemble: exact,
    // else the generic loop
    if (b->tmax == 3 && b->tmin_all == 3 && b->us2) return batch_launch<TS, MAXR, 3, 2>(h, b);
    return batch_launch<TS, MAXR, 0, 0>(h, b);
}

template <typename TS>
static rca_status batch_maxr(rca_handle* h, rca_batch* b)
{
    if (b->maxr <= 2) return batch_tm<TS, 2>(h, b);
    if (b->maxr <= 4) return batch_tm<TS, 4>(h, b);
    if (b->maxr <= 8) return batch_tm<TS, 8>(h, b);
    return batch_tm<TS, 16>(h, b);
}
