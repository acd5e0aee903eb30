// localize.cu -- XDoppler enhancement, separable NCC, sub-pixel peaks and
// XZ / YZ pairing (Sec. II-A4, Fig. 1e, Fig. 1g).
#include <algorithm>
#include <cmath>
#include <mutex>

#include "rca_internal.cuh"

namespace {

// ---------------------------------------------------------------------------
// XDoppler: each thread owns one pixel (axis, slab, row, lateral) and walks
// the frames with a sliding 3-frame window, so every plane is read once:
//   Q_t = P_RC,t conj(P_CR,t),  A_t = sqrt(|Q_{t-1} + Q_t + Q_{t+1}|).
// The planes of frame t+2 are loaded while frame t is finished.  Frames are
// split into chunks across blockIdx.y (each chunk re-reads the frame before
// it) when the planes alone would give too few blocks.  M_t = max A_t: warp
// max, shared-memory atomicMax per frame, one global atomicMax per block and
// frame at the end (non-negative floats order like their bits).
// ---------------------------------------------------------------------------
// plane element i of compile-time dtype PT as float2 (read-only path)
template <int PT>
__device__ __forceinline__ float2 ld_plane(const void* __restrict__ p, size_t i)
{
    if constexpr (PT == RCA_C32) {
        return __ldg(reinterpret_cast<const float2*>(p) + i);
    } else {
        const unsigned u = __ldg(reinterpret_cast<const unsigned*>(p) + i);
        if constexpr (PT == RCA_C16F) return __half22float2(*reinterpret_cast<const __half2*>(&u));
        else return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u));
    }
}

template <int PT>
__global__ void __launch_bounds__(256) k_enhance(const void* __restrict__ planes, int F, int S, size_t plane_sz,
                                                 int enh, int tf, float* __restrict__ A, unsigned* __restrict__ M)
{
    extern __shared__ unsigned mx[];  // [tf] maxima of this chunk's frames
    const int t0 = blockIdx.y * tf, t1 = min(F, t0 + tf);
    for (int t = threadIdx.x; t < t1 - t0; t += blockDim.x) mx[t] = 0u;
    __syncthreads();
    const size_t per_axis = (size_t)S * plane_sz;
    const size_t npx = 2 * per_axis;
    const size_t FS = 2 * npx;                       // elements per frame: [axis][family][S][nz][N]
    const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool act = p < npx;
    const size_t axis = act ? p / per_axis : 0, rest = act ? p % per_axis : 0;
    const int lane = threadIdx.x & 31;
    // element of the RC plane of frame t is t FS + oR; its CR plane lies per_axis further
    const size_t oR = axis * 2 * per_axis + rest;
    auto ld = [&](int t, int fam) {
        return (act && t < F) ? ld_plane<PT>(planes, (size_t)t * FS + oR + (fam ? per_axis : 0))
                              : make_float2(0.f, 0.f);
    };
    auto xq = [](float2 a, float2 b) { return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y); };
    float2 r0 = ld(t0, 0), c0 = ld(t0, 1), r1 = ld(t0 + 1, 0), c1 = ld(t0 + 1, 1);
    float2 r2 = ld(t0 + 2, 0), c2 = ld(t0 + 2, 1);
    float2 qm = make_float2(0.f, 0.f);
    if (t0 > 0 && enh == ULM_ENH_XDOPPLER) qm = xq(ld(t0 - 1, 0), ld(t0 - 1, 1));
    // prefetch index of frame t + 3 and output pointer of frame t, advanced per frame
    size_t i3 = (size_t)(t0 + 3) * FS + oR;
    float* out = A + (size_t)t0 * npx + p;
    for (int t = t0; t < t1; ++t) {
        float2 r3 = make_float2(0.f, 0.f), c3 = r3;
        if (act && t + 3 < F) {
            r3 = ld_plane<PT>(planes, i3);
            c3 = ld_plane<PT>(planes, i3 + per_axis);
        }
        i3 += FS;
        float a;
        if (enh == ULM_ENH_XDOPPLER) {
            const float2 q0 = xq(r0, c0), qp = xq(r1, c1);
            const float re = qm.x + q0.x + qp.x, im = qm.y + q0.y + qp.y;
            a = sqrtf(sqrtf(re * re + im * im));
            qm = q0;
        } else {
            const float re = r0.x + c0.x, im = r0.y + c0.y;
            a = sqrtf(re * re + im * im);
        }
        if (act) __stcs(out, a);
        out += npx;
        // warp maximum on the bits (non-negative floats order like their bits)
        const unsigned m = __reduce_max_sync(0xffffffffu, act ? __float_as_uint(a) : 0u);
        if (lane == 0) atomicMax(mx + (t - t0), m);
        r0 = r1; c0 = c1; r1 = r2; c1 = c2; r2 = r3; c2 = c3;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < t1 - t0; t += blockDim.x) atomicMax(M + t0 + t, mx[t]);
}

// ---------------------------------------------------------------------------
// NCC + regional peaks.  CTA = (row strip of NCC_RS rows, plane).  NCC via
// separable 1D correlations (Fig. 1g):
//   s1 = box(A), s2 = box(A^2), sg = (g_z x g_l) * A,
//   NCC = (sg - mu_G s1) / sqrt((s2 - s1^2 / d^2) * ss_G),
// computed on the strip plus one row above and below for the 3x3 test.
// Candidates are compacted in raster order into a fixed-capacity slot of
// the strip; the true count is kept.
//
// Box sums by split points: for a run of B <= d consecutive outputs every
// window contains the run's last first-row m, so
//   box(r) = Suf(r) + Pre(r + d - 1),  Suf(r) = x_r + ... + x_{m-1},
//   Pre(k) = x_m + ... + x_k,
// about three adds per output instead of d, and every output is the sum of
// two partial sums over its own window only (no running sum carries the
// rounding of values that have left the window).  The Gaussian-weighted sums
// keep their d taps.
//
// Vertical pass first, on column pairs (one 64-bit shared load gives two
// columns of an input row; thread task = column pair x VB output rows); its
// three sums are stored transposed into row pairs, so the horizontal pass
// works on two output rows at once (thread task = row pair x HB output
// columns).  Thread-to-data maps keep both passes free of bank conflicts:
// consecutive lanes take consecutive column pairs in the vertical pass and
// consecutive row pairs (row-pair stride of N + 1 pairs) in the horizontal
// pass.
// ---------------------------------------------------------------------------
#define NCC_THREADS 256

// float2 columns of one padded vertical-sum row pair (see k_detect)
__host__ __device__ inline int det_npad(int N, int H, int HB)
{
    const int w = (N + HB - 1) / HB * HB + 2 * H;
    return w | 1;
}
__host__ __device__ inline int det_hb(int H) { return H >= 4 ? 8 : 2 * H; }

// split-point box sums of NB consecutive outputs from the NB + 2H inputs
// in[0 ..]: out[r] = in[r] + ... + in[r + 2H]  (NB <= 2H + 1)
template <int H, int NB, typename LOAD>
__device__ __forceinline__ void split_box(LOAD in, uint64_t (&out)[NB])
{
    static_assert(NB >= 1 && NB <= 2 * H + 1, "a run of outputs must share a split row");
    constexpr int m = NB - 1;
    uint64_t suf[NB];
    if constexpr (m >= 1) {
        suf[m - 1] = in(m - 1);
#pragma unroll
        for (int k = m - 2; k >= 0; --k) suf[k] = f2_add(in(k), suf[k + 1]);
    }
    uint64_t pre = in(m);
#pragma unroll
    for (int k = m + 1; k <= m + 2 * H; ++k) {
        pre = f2_add(pre, in(k));
        const int r = k - 2 * H;
        if (r >= 0) out[r] = r < m ? f2_add(suf[r], pre) : pre;
    }
}

template <int H, int NC>
__global__ void __launch_bounds__(NCC_THREADS, 2) k_detect(const float* __restrict__ A, const float* __restrict__ Mf,
                                                          int S, int nz, int Nrt, int nplanes, NccConst nc,
                                                          ulm_loc2d* __restrict__ cand, int* __restrict__ cnt,
                                                          float* __restrict__ ncc_out, unsigned* __restrict__ status)
{
    constexpr int D = 2 * H + 1;
    constexpr int RN = NCC_RS + 2;          // NCC rows: the strip and one row above and below
    constexpr int RP = RN / 2;              // row pairs
    constexpr int VB = H >= 4 ? 8 : (H >= 2 ? 4 : 2);   // output rows per vertical task
    constexpr int HB = H >= 4 ? 8 : 2 * H;  // output columns per horizontal task (det_hb)
    constexpr int NW = (NCC_RS * 256 + 31) / 32;   // bitmap words of the strip's pixels (N <= 256)
    static_assert(RN % VB == 0 && VB % 2 == 0 && VB <= D, "vertical runs must tile the NCC rows in pairs");
    const int N = NC > 0 ? NC : Nrt;        // lateral pixels (compile-time for the usual widths)
    extern __shared__ __align__(128) float sm[];
    const int nstrip = (nz + NCC_RS - 1) / NCC_RS;
    const int items = nplanes * nstrip;
    const int rin = RN + 2 * H;
    // columns of a padded vertical-sum row pair: column c at c + H, zero pads on
    // both sides, room for the last horizontal block's overhang, odd (conflict-free)
    const int NPAD = det_npad(N, H, HB);
    const int VS = 2 * NPAD;                // floats per row pair of a vertical-sum array
    const int NS = N + 1;                   // NCC row stride
    const size_t abuf = max((size_t)rin * N, (size_t)RN * NS);
    // sm + bb abuf (bb = 0, 1): [rin][N] amplitude rows i0-1-H ..., double-buffered
    float* sV = sm + 2 * abuf;              // [3][RP][NPAD][2]; column c at c + H
    // [RN][N] flags A >= alpha M_t of the NCC rows' pixels, set by the vertical pass
    // (which holds the amplitudes), so that no phase after it reads global memory
    unsigned char* aflag = reinterpret_cast<unsigned char*>(sV + (size_t)3 * RP * NPAD * 2);
    __shared__ unsigned bits[NW];           // candidate pixels of the strip, raster order
    __shared__ int wsum[NCC_THREADS / 32];
    __shared__ uint64_t bar[2];
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_fence_init();
    }
    {
        const int npad = NPAD - N;          // H on the left, the rest on the right
        for (int idx = threadIdx.x; idx < 3 * RP * npad; idx += blockDim.x) {
            const int ar = idx / npad, q = idx - ar * npad;
            const int col = q < H ? q : N + q;
            reinterpret_cast<float2*>(sV)[(size_t)ar * NPAD + col] = make_float2(0.f, 0.f);
        }
    }
    __syncthreads();
    // rows [i0-1-H, i0+NCC_RS+1+H) of item `it`'s plane into buffer bb: zero
    // outside the plane (all threads), one bulk copy inside (thread 0)
    auto fetch = [&](int it, int bb) {
        const int plane = it / nstrip, strip = it - plane * nstrip;
        const int rlo = strip * NCC_RS - 1 - H;
        const int lo = max(rlo, 0), hi = max(lo, min(rlo + rin, nz));
        const int z0 = min(lo - rlo, rin), z1 = hi - rlo;
        float* sA = sm + bb * abuf;
        for (int idx = threadIdx.x; idx < z0 * N; idx += blockDim.x) sA[idx] = 0.f;
        for (int idx = threadIdx.x; idx < (rin - z1) * N; idx += blockDim.x) sA[(size_t)z1 * N + idx] = 0.f;
        if (threadIdx.x == 0) {
            fence_proxy_async();
            // the copied rows land inside the buffer's rin rows (checked build; else nothing is copied)
            const bool in = chk(lo >= rlo && hi - rlo <= rin && plane < nplanes, status);
            const unsigned bytes = in ? (unsigned)((hi - lo) * N * sizeof(float)) : 0u;
            mbar_arrive_expect_tx(&bar[bb], bytes);
            if (bytes)
                bulk_g2s(sA + (size_t)(lo - rlo) * N, A + ((size_t)plane * nz + lo) * N, bytes, &bar[bb]);
        }
    };
    // packed Gaussian taps, held for every item
    uint64_t gz[D], gl[D];
#pragma unroll
    for (int q = 0; q < D; ++q) {
        gz[q] = f2_pack(nc.gz[q], nc.gz[q]);
        gl[q] = f2_pack(nc.gl[q], nc.gl[q]);
    }
    int it = blockIdx.x;
    if (it < items) fetch(it, 0);
    for (int k = 0; it < items; it += gridDim.x, ++k) {
        const int bb = k & 1;
        const int next = it + gridDim.x;
        // the other buffer was released by the barrier that ended the previous item
        if (next < items) fetch(next, bb ^ 1);
        if (!cta_wait_copies(&bar[bb], (unsigned)(k >> 1) & 1u, status)) {
            if (next < items) mbar_wait_bounded(&bar[bb ^ 1], (unsigned)((k + 1) >> 1) & 1u);
            return;
        }
        float* sA = sm + bb * abuf;
        float* sN = sA;                     // NCC rows over the amplitude rows once the vertical pass is done
        const int plane = it / nstrip, strip = it - plane * nstrip;
        const int t = plane / (2 * S), axis = (plane / S) % 2, b = plane % S;
        const int i0 = strip * NCC_RS;
        const float Mt = Mf[t];
        const float athr = nc.alpha * Mt;
        for (int idx = threadIdx.x; idx < NW; idx += blockDim.x) bits[idx] = 0u;
        // ---- vertical pass: thread = (column pair, VB output rows)
        {
            const int NP = N / 2;
            const unsigned sAa = smem_u32(sA), sVa = smem_u32(sV);
            for (int task = threadIdx.x; task < NP * (RN / VB); task += blockDim.x) {
                const int cp = task % NP, rb = task / NP;
                const int ro0 = rb * VB;
                // NCC rows ro0 .. ro0 + VB - 1 use amplitude rows ro0 .. ro0 + VB - 1 + 2H
                uint64_t x[VB + 2 * H];
                const unsigned src = sAa + (unsigned)((ro0 * N + 2 * cp) * 4);
#pragma unroll
                for (int m = 0; m < VB + 2 * H; ++m) x[m] = lds_u64(src + (unsigned)(m * N * 4));
#pragma unroll
                for (int r = 0; r < VB; ++r) {
                    // the centre amplitude of NCC row ro0 + r, both columns of the pair
                    const float2 ac = f2_unpack(x[r + H]);
                    const unsigned short fl = (unsigned short)((ac.x >= athr ? 1u : 0u) | (ac.y >= athr ? 0x100u : 0u));
                    if (chk((ro0 + r) * N + 2 * cp + 1 < RN * N, status))
                        *reinterpret_cast<unsigned short*>(aflag + (ro0 + r) * N + 2 * cp) = fl;
                }
                uint64_t v1[VB], v2[VB], vg[VB];
                split_box<H, VB>([&](int q) { return x[q]; }, v1);
                split_box<H, VB>([&](int q) { return f2_mul(x[q], x[q]); }, v2);
#pragma unroll
                for (int r = 0; r < VB; ++r) {
                    uint64_t a = f2_mul(gz[0], x[r]);
#pragma unroll
                    for (int q = 1; q < D; ++q) a = f2_fma(gz[q], x[r + q], a);
                    vg[r] = a;
                }
                // transpose 2 x 2 blocks into row pairs: [arr][rp][H + column][row parity]
                const unsigned dst0 = sVa + (unsigned)(((ro0 / 2) * VS + 2 * (2 * cp + H)) * 4);
#pragma unroll
                for (int j = 0; j < VB; j += 2) {
                    const uint64_t* arrs[3] = {v1, v2, vg};
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        const float2 r0 = f2_unpack(arrs[a][j]), r1 = f2_unpack(arrs[a][j + 1]);
                        const unsigned dst = dst0 + (unsigned)(((a * RP + j / 2) * VS) * 4);
                        asm volatile("st.shared.v2.f32 [%0], {%1, %2};" ::"r"(dst), "f"(r0.x), "f"(r1.x) : "memory");
                        asm volatile("st.shared.v2.f32 [%0], {%1, %2};" ::"r"(dst + 8u), "f"(r0.y), "f"(r1.y) : "memory");
                    }
                }
            }
        }
        __syncthreads();
        // ---- horizontal pass + NCC: thread = (row pair, HB output columns);
        // the amplitude rows are no longer read, so the NCC rows take their place
        {
            const float flat = nc.flat_coef * Mt * Mt;
            const float inv_d2 = 1.0f / (float)(D * D);
            const int ncb = (N + HB - 1) / HB;
            const uint64_t nid2 = f2_pack(-inv_d2, -inv_d2), nmu = f2_pack(-nc.muG, -nc.muG);
            const unsigned sVa = smem_u32(sV);
            for (int task = threadIdx.x; task < RP * ncb; task += blockDim.x) {
                const int rp = task % RP, cb = task / RP;
                const int c0 = cb * HB;
                // padded input columns c0 - H .. c0 + HB - 1 + H start at pad index c0; past N they
                // read the right pad (zero) or feed only outputs past N
                const unsigned at = sVa + (unsigned)((rp * VS + 2 * c0) * 4);
                uint64_t s1[HB], s2[HB], sg[HB];
                {
                    uint64_t a[HB + 2 * H];
#pragma unroll
                    for (int m = 0; m < HB + 2 * H; ++m) a[m] = lds_u64(at + (unsigned)(m * 8));
                    split_box<H, HB>([&](int q) { return a[q]; }, s1);
#pragma unroll
                    for (int m = 0; m < HB + 2 * H; ++m) a[m] = lds_u64(at + (unsigned)(RP * VS * 4 + m * 8));
                    split_box<H, HB>([&](int q) { return a[q]; }, s2);
#pragma unroll
                    for (int m = 0; m < HB + 2 * H; ++m) a[m] = lds_u64(at + (unsigned)(2 * RP * VS * 4 + m * 8));
#pragma unroll
                    for (int r = 0; r < HB; ++r) {
                        uint64_t g = f2_mul(gl[0], a[r]);
#pragma unroll
                        for (int q = 1; q < D; ++q) g = f2_fma(gl[q], a[r + q], g);
                        sg[r] = g;
                    }
                }
                const int ia = i0 - 1 + 2 * rp;    // plane row of the pair's first row
                const bool row0 = ia >= H && ia < nz - H && Mt > 0.f;
                const bool row1 = ia + 1 >= H && ia + 1 < nz - H && Mt > 0.f;
                float* nrow = sN + (2 * rp) * NS + c0;
#pragma unroll
                for (int j = 0; j < HB; ++j) {
                    const int c = c0 + j;
                    if (c >= N) break;
                    // ssA = s2 - s1^2 / d^2, numerator = sg - mu_G s1 (both rows of the pair)
                    const float2 ss = f2_unpack(f2_fma(f2_mul(s1[j], s1[j]), nid2, s2[j]));
                    const float2 nu = f2_unpack(f2_fma(nmu, s1[j], sg[j]));
                    const bool colok = c >= H && c < N - H;
                    const float v0 = (colok && row0 && ss.x > flat) ? nu.x * nc.inv_ssG_sqrt * rsqrtf(ss.x) : 0.f;
                    const float v1 = (colok && row1 && ss.y > flat) ? nu.y * nc.inv_ssG_sqrt * rsqrtf(ss.y) : 0.f;
                    nrow[j] = v0;
                    nrow[NS + j] = v1;
                    if (ncc_out) {
                        if (2 * rp >= 1 && 2 * rp <= NCC_RS && ia < nz) ncc_out[((size_t)plane * nz + ia) * N + c] = v0;
                        if (2 * rp + 1 <= NCC_RS && ia + 1 < nz) ncc_out[((size_t)plane * nz + ia + 1) * N + c] = v1;
                    }
                }
            }
        }
        __syncthreads();
        // ---- peaks: test every strip pixel (thread = column, rows in steps), mark
        // the candidates in a raster-order bitmap, then compact the bitmap words
        // (consecutive words per thread, a block-wide exclusive scan of their
        // counts) so the strip's candidates come out in raster order
        {
            const int RG = NCC_THREADS / N > 0 ? NCC_THREADS / N : 1;   // row groups (N <= 256)
            const int l = threadIdx.x % N, rg = threadIdx.x / N;
            // NCC rows whose plane row i = i0 - 1 + ro lies in [1, nz - 2]
            const int ro_lo = max(1, 2 - i0), ro_hi = min(NCC_RS, nz - 1 - i0);
            if (rg < RG && l >= 1 && l < N - 1) {
                int ro = ro_lo + rg;
                const float* np_ = sN + ro * NS + l;
#pragma unroll 5
                for (; ro <= ro_hi; ro += RG, np_ += RG * NS) {
                    const float c = *np_;
                    if (!(c >= nc.ncc_min)) continue;
                    bool pk = aflag[ro * N + l] != 0;
#pragma unroll
                    for (int a = -1; a <= 1; ++a)
#pragma unroll
                        for (int bq = -1; bq <= 1; ++bq) {
                            if (a == 0 && bq == 0) continue;
                            const float q = sN[(ro + a) * NS + l + bq];
                            const bool earlier = (a < 0) || (a == 0 && bq < 0);
                            pk = pk && (earlier ? (c > q) : (c >= q));
                        }
                    if (pk) {
                        const int p = (ro - 1) * N + l;
                        if (chk(p >= 0 && (p >> 5) < NW && ro + 1 < RN, status)) atomicOr(&bits[p >> 5], 1u << (p & 31));
                    }
                }
            }
        }
        __syncthreads();
        ulm_loc2d* slot = cand + (size_t)it * CAND_CAP;
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        // each thread compacts wpt consecutive bitmap words (wpt = 2 only when N > 273)
        const int nwords = (NCC_RS * N + 31) / 32;
        const int wpt = (nwords + NCC_THREADS - 1) / NCC_THREADS;
        const int w0 = threadIdx.x * wpt;
        unsigned long long mask = 0ull;
        if (w0 < nwords) mask = bits[w0];
        if (wpt == 2 && w0 + 1 < nwords) mask |= (unsigned long long)bits[w0 + 1] << 32;
        const int mine = __popcll(mask);
        int x = mine;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[warp] = x;
        __syncthreads();
        int before = x - mine;
        for (int w = 0; w < warp; ++w) before += wsum[w];
        while (mask) {
            const int bit = __ffsll(mask) - 1;
            mask &= mask - 1;
            if (before < CAND_CAP) {
                const int p = w0 * 32 + bit;
                const int ro = 1 + p / N, l = p - (ro - 1) * N, i = i0 - 1 + ro;
                const float c = sN[ro * NS + l];
                auto para = [](float fm, float f0, float fp) {
                    const float den = fm - 2.f * f0 + fp;
                    if (den >= 0.f) return 0.f;
                    const float dl = (fm - fp) / (2.f * den);
                    return fminf(0.5f, fmaxf(-0.5f, dl));
                };
                ulm_loc2d e;
                e.frame = t;
                e.axis = axis;
                e.slab = b;
                e.iz = i;
                e.ilat = l;
                e.z = (float)i + para(sN[(ro - 1) * NS + l], c, sN[(ro + 1) * NS + l]);
                e.lat = (float)l + para(sN[ro * NS + l - 1], c, sN[ro * NS + l + 1]);
                e.ncc = c;
                e.amp = 0.f;        // filled from A by the gather (no global load in this phase)
                e.reserved = 0;
                slot[before] = e;
            }
            ++before;
        }
        // the last thread's running index is the strip's count
        if (threadIdx.x == blockDim.x - 1) {
            cnt[it] = before;
            if (before > CAND_CAP) atomicOr(status, ST_CAPACITY);
        }
        // the next iteration fetches into this buffer and rewrites the bitmap
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        mbar_inval(&bar[0]);
        mbar_inval(&bar[1]);
    }
}

// ---------------------------------------------------------------------------
// Peaks of score maps on a finer grid (the learned localiser's heatmaps).
// CTA = (strip of DET_RS fine rows, plane); same raster-order compaction as
// k_detect.  Positions are converted to plane pixels for pairing.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_detect_map(const float* __restrict__ map, int up, const float* __restrict__ A,
                                                    const float* __restrict__ Mf, int S, int nz, int N, float score_min,
                                                    float alpha, ulm_loc2d* __restrict__ cand, int* __restrict__ cnt,
                                                    unsigned* __restrict__ status)
{
    extern __shared__ __align__(128) float smf[];
    __shared__ int wsum[32];
    __shared__ uint64_t bar;
    const int H4 = nz * up, W4 = N * up;
    const int strip = blockIdx.x, plane = blockIdx.y, nstrip = gridDim.x;
    const int t = plane / (2 * S), axis = (plane / S) % 2, b = plane % S;
    const int i0 = strip * DET_RS, rin = DET_RS + 2;
    const float* mp = map + (size_t)plane * H4 * W4;
    const float* Ap = A + (size_t)plane * nz * N;
    const float Mt = Mf[t];
    {
        const int rlo = i0 - 1;
        const int lo = max(rlo, 0), hi = max(lo, min(rlo + rin, H4));
        if (threadIdx.x == 0) {
            mbar_init(&bar, 1);
            mbar_fence_init();
        }
        __syncthreads();
        const int z0 = min(lo - rlo, rin), z1 = hi - rlo;
        for (int idx = threadIdx.x; idx < z0 * W4; idx += blockDim.x) smf[idx] = 0.f;
        for (int idx = threadIdx.x; idx < (rin - z1) * W4; idx += blockDim.x) smf[(size_t)z1 * W4 + idx] = 0.f;
        if (threadIdx.x == 0) {
            fence_proxy_async();
            const unsigned bytes = (unsigned)((hi - lo) * W4 * sizeof(float));
            mbar_arrive_expect_tx(&bar, bytes);
            if (bytes) bulk_g2s(smf + (size_t)(lo - rlo) * W4, mp + (size_t)lo * W4, bytes, &bar);
        }
        if (!cta_wait_copies(&bar, 0, status)) return;
    }
    const float athr = alpha * Mt;
    ulm_loc2d* slot = cand + ((size_t)plane * nstrip + strip) * CAND_CAP;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int npx = DET_RS * W4;
    const int nwords = (npx + 31) / 32;
    // candidate bitmap of the strip's pixels in raster order (cleared, then set by
    // the test: consecutive lanes take consecutive pixels, conflict-free on the rows)
    unsigned* bits = reinterpret_cast<unsigned*>(smf + (size_t)rin * W4);
    for (int w = threadIdx.x; w < nwords; w += blockDim.x) bits[w] = 0u;
    __syncthreads();
    // rows in turn, consecutive lanes on consecutive columns (no division per pixel)
    const int ro_lo = max(1, 2 - i0), ro_hi = min(DET_RS, H4 - 1 - i0);   // rows with 1 <= i <= H4 - 2
    for (int ro = ro_lo; ro <= ro_hi; ++ro) {
#pragma unroll 2
        for (int j = threadIdx.x; j < W4; j += blockDim.x) {
            const int i = i0 - 1 + ro, p = (ro - 1) * W4 + j;
            if (j < 1 || j >= W4 - 1) continue;
            const float c = smf[ro * W4 + j];
            if (!(c >= score_min)) continue;
            bool pk = true;
#pragma unroll
            for (int a = -1; a <= 1; ++a)
#pragma unroll
                for (int bb = -1; bb <= 1; ++bb) {
                    if (a == 0 && bb == 0) continue;
                    const float q = smf[(ro + a) * W4 + j + bb];
                    const bool earlier = (a < 0) || (a == 0 && bb < 0);
                    pk = pk && (earlier ? (c > q) : (c >= q));
                }
            // the amplitude (global memory) only for regional maxima
            if (pk && Ap[(size_t)(i / up) * N + j / up] >= athr) atomicOr(&bits[p >> 5], 1u << (p & 31));
        }
    }
    __syncthreads();
    // compaction: consecutive bitmap words per thread, a block-wide exclusive scan of their counts
    const int wpt = (nwords + blockDim.x - 1) / blockDim.x;
    const int w0 = threadIdx.x * wpt, w1 = min(nwords, w0 + wpt);
    int mine = 0;
    for (int w = w0; w < w1; ++w) mine += __popc(bits[w]);
    int x = mine;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    int before = x - mine;
    for (int w = 0; w < warp; ++w) before += wsum[w];
    const float half = 0.5f * (float)(up - 1), inv = 1.f / (float)up;
    for (int w = w0; w < w1; ++w) {
        unsigned m = bits[w];
        while (m) {
            const int bit = __ffs(m) - 1;
            m &= m - 1;
            if (before < CAND_CAP) {
                const int p = w * 32 + bit;
                const int ro = 1 + p / W4, j = p - (ro - 1) * W4, i = i0 - 1 + ro;
                const float c = smf[ro * W4 + j];
                auto para = [](float fm, float f0, float fp) {
                    const float den = fm - 2.f * f0 + fp;
                    if (den >= 0.f) return 0.f;
                    const float dl = (fm - fp) / (2.f * den);
                    return fminf(0.5f, fmaxf(-0.5f, dl));
                };
                ulm_loc2d e;
                e.frame = t;
                e.axis = axis;
                e.slab = b;
                e.iz = i / up;
                e.ilat = j / up;
                e.z = ((float)i + para(smf[(ro - 1) * W4 + j], c, smf[(ro + 1) * W4 + j]) - half) * inv;
                e.lat = ((float)j + para(smf[ro * W4 + j - 1], c, smf[ro * W4 + j + 1]) - half) * inv;
                e.ncc = c;
                e.amp = Ap[(size_t)e.iz * N + e.ilat];
                e.reserved = 0;
                slot[before] = e;
            }
            ++before;
        }
    }
    // the last thread's running index is the strip's count
    if (threadIdx.x == blockDim.x - 1) {
        cnt[(size_t)plane * nstrip + strip] = before;
        if (before > CAND_CAP) atomicOr(status, ST_CAPACITY);
    }
}

// Multi-block exclusive scan of min(cnt[i], cap_each) (cap_each <= 0: no cap)
// over n entries (n = min(n, *n_dev) when n_dev is given).  off[n] = kept
// total; *total_true = sum of the uncapped counts.
#define SCAN_CHUNK 4096
#define SCAN_THREADS 512

__device__ __forceinline__ int scan_n(int n, const int* n_dev) { return n_dev ? min(n, *n_dev) : n; }

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_part(const int* __restrict__ cnt, int n, const int* __restrict__ n_dev,
                                                            int cap_each, long long* __restrict__ part)
{
    __shared__ long long red[2][SCAN_THREADS / 32];
    n = scan_n(n, n_dev);
    const int lo = blockIdx.x * SCAN_CHUNK, hi = min(n, lo + SCAN_CHUNK);
    long long s = 0, st = 0;
    for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const int c = cnt[i];
        st += c;
        s += (cap_each > 0) ? min(c, cap_each) : c;
    }
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        st += __shfl_xor_sync(0xffffffffu, st, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = s;
        red[1][threadIdx.x >> 5] = st;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        long long a = 0, b = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            a += red[0][w];
            b += red[1][w];
        }
        part[2 * blockIdx.x] = a;
        part[2 * blockIdx.x + 1] = b;
    }
}

// one block: exclusive scan of the per-chunk totals (nb <= 1024 chunks)
__global__ void __launch_bounds__(1024) k_scan_top(long long* __restrict__ part, int nb, int n,
                                                   const int* __restrict__ n_dev, int* __restrict__ off,
                                                   int* __restrict__ total_true)
{
    __shared__ long long a[1024], b[1024];
    n = scan_n(n, n_dev);
    const int used = (n + SCAN_CHUNK - 1) / SCAN_CHUNK;
    const int i = threadIdx.x;
    a[i] = (i < nb && i < used) ? part[2 * i] : 0;
    b[i] = (i < nb && i < used) ? part[2 * i + 1] : 0;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        long long va = i >= o ? a[i - o] : 0, vb = i >= o ? b[i - o] : 0;
        __syncthreads();
        a[i] += va;
        b[i] += vb;
        __syncthreads();
    }
    if (i < nb) part[2 * i] = i ? a[i - 1] : 0;  // exclusive chunk offset
    if (i == 1023) {
        off[n] = (int)min(a[1023], (long long)0x7fffffff);
        if (total_true) *total_true = (int)min(b[1023], (long long)0x7fffffff);
    }
}

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_apply(const int* __restrict__ cnt, int n,
                                                             const int* __restrict__ n_dev, int cap_each,
                                                             const long long* __restrict__ part, int* __restrict__ off)
{
    constexpr int PER = SCAN_CHUNK / SCAN_THREADS;
    __shared__ int wsum[SCAN_THREADS / 32];
    n = scan_n(n, n_dev);
    const int lo = blockIdx.x * SCAN_CHUNK;
    if (lo >= n) return;
    const int base = lo + threadIdx.x * PER;
    int v[PER], s = 0;
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        const int i = base + q;
        const int c = i < n ? cnt[i] : 0;
        v[q] = (cap_each > 0) ? min(c, cap_each) : c;
        s += v[q];
    }
    // block exclusive scan of the per-thread sums
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = s;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    int wpre = 0;
    for (int w = 0; w < warp; ++w) wpre += wsum[w];
    int run = (int)part[2 * blockIdx.x] + wpre + x - s;
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        const int i = base + q;
        if (i < n) off[i] = run;
        run += v[q];
    }
}

// Copy each strip's kept candidates to their place in the output list.
// A non-null: each entry's amplitude is read here from A [plane][nz][N] at its
// pixel (the detection kernel leaves it to this highly parallel pass)
__global__ void k_gather(const ulm_loc2d* __restrict__ cand, const int* __restrict__ cnt, const int* __restrict__ off,
                         int nslots, ulm_loc2d* __restrict__ out, int cap, const float* __restrict__ A, int S, int nz,
                         int N, unsigned* __restrict__ status)
{
    const int s = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (s >= nslots) return;
    const int lane = threadIdx.x & 31;
    const int c = min(cnt[s], CAND_CAP);
    for (int r = lane; r < c; r += 32) {
        int dst = off[s] + r;
        if (dst < cap) {
            ulm_loc2d e = cand[(size_t)s * CAND_CAP + r];
            if (A && chk(e.iz >= 0 && e.iz < nz && e.ilat >= 0 && e.ilat < N && e.slab >= 0 && e.slab < S, status))
                e.amp = __ldg(A + (((size_t)(e.frame * 2 + e.axis) * S + e.slab) * nz + e.iz) * N + e.ilat);
            out[dst] = e;
        } else {
            atomicOr(status, ST_CAPACITY);
        }
    }
}

// plane offsets of the (frame, axis, slab)-sorted list: first entry of each plane
__global__ void k_strip_to_plane(const int* __restrict__ off, int nstrip, int nplanes, int* __restrict__ poff)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p <= nplanes) poff[p] = off[(size_t)p * nstrip];
}

// ---------------------------------------------------------------------------
// pairing
// ---------------------------------------------------------------------------
__device__ __forceinline__ int plane_key(const ulm_loc2d& e, int S) { return (e.frame * 2 + e.axis) * S + e.slab; }

__global__ void k_list_plane_offsets(const ulm_loc2d* __restrict__ L, const int* __restrict__ n2d, int cap2d, int S,
                                     int nplanes, int* __restrict__ poff)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p > nplanes) return;
    int n = min(*n2d, cap2d);
    int lo = 0, hi = n;  // first index with key >= p
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (plane_key(L[mid], S) < p) lo = mid + 1;
        else hi = mid;
    }
    poff[p] = lo;
}

// XZ / YZ eligibility and cost in double precision: same frame and
// sub-block, |dz| <= 1 pixel, ratio I_xz / I_yz in [0.9, 1.11];
// cost max(I) / min(I) (orders pairs like |ln ratio|).
// The decisions are those of FP64 arithmetic on the FP32 inputs (the oracle's).
// GB300's FP64 rate is low, so each test is first taken in FP32 where that
// provably gives the same answer (rounding to nearest is monotonic, so
// fl32(e) > 1 implies e > 1 and fl32(e) < 1 implies e < 1; a ratio more than
// 0.01 inside or outside a bound is on the same side in FP64), and in FP64
// only when the FP32 value sits at the bound.
__device__ __forceinline__ bool pair_ok(const ulm_loc2d& x, const ulm_loc2d& y, int P, double* cost)
{
    if (x.frame != y.frame) return false;
    // x.ilat / P == y.slab and y.ilat / P == x.slab (non-negative indexes), without divisions
    const int xl = y.slab * P, yl = x.slab * P;
    if (x.ilat < xl || x.ilat >= xl + P || y.ilat < yl || y.ilat >= yl + P) return false;
    const float dz = fabsf(x.z - y.z);
    if (dz > 1.0f) return false;
    if (dz == 1.0f && fabs((double)x.z - (double)y.z) > 1.0) return false;
    const float r32 = x.amp / y.amp;
    const bool lo_sure = r32 >= 0.91f, hi_sure = r32 <= 1.10f;
    if (r32 <= 0.89f || r32 >= 1.12f || !(r32 == r32)) return false;
    const double ax = x.amp, ay = y.amp;
    if (!(lo_sure && hi_sure)) {
        const double r = ax / ay;
        if (!(r >= 0.9 && r <= 1.11)) return false;
    }
    *cost = ax > ay ? ax / ay : ay / ax;
    return true;
}

__global__ void k_pair_match(const ulm_loc2d* __restrict__ L, const int* __restrict__ n2d, int cap2d, int S, int P,
                             const int* __restrict__ poff, int* __restrict__ match)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = min(*n2d, cap2d);
    if (a >= n) return;
    const ulm_loc2d x = L[a];
    int m = -1;
    if (x.axis == 0) {
        const int py = (x.frame * 2 + 1) * S + x.ilat / P;
        int best = -1;
        double bc = 0.0;
        for (int q = poff[py]; q < min(poff[py + 1], n); ++q) {
            double c;
            if (pair_ok(x, L[q], P, &c) && (best < 0 || c < bc)) {
                best = q;
                bc = c;
            }
        }
        if (best >= 0) {
            const ulm_loc2d y = L[best];
            const int px = (y.frame * 2 + 0) * S + y.ilat / P;
            int back = -1;
            double bc2 = 0.0;
            for (int q = poff[px]; q < min(poff[px + 1], n); ++q) {
                double c;
                if (pair_ok(L[q], y, P, &c) && (back < 0 || c < bc2)) {
                    back = q;
                    bc2 = c;
                }
            }
            if (back == a) m = best;
        }
    }
    match[a] = m;
}

__global__ void k_match_flags(const int* __restrict__ match, const int* __restrict__ n2d, int cap2d,
                              int* __restrict__ flags)
{
    // every slot the scan reads, max(cap2d, 1) of them, is written (0 past the list)
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= max(cap2d, 1)) return;
    const int n = min(*n2d, cap2d);
    flags[a] = (a < n && match[a] >= 0) ? 1 : 0;
}

__global__ void k_pair_write(const ulm_loc2d* __restrict__ L, const int* __restrict__ n2d, int cap2d,
                             const int* __restrict__ match, const int* __restrict__ off, ulm_loc3d* __restrict__ out,
                             int cap3d, unsigned* __restrict__ status)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = min(*n2d, cap2d);
    if (a >= n || match[a] < 0) return;
    const int dst = off[a];
    if (dst >= cap3d) {
        atomicOr(status, ST_CAPACITY);
        return;
    }
    const ulm_loc2d x = L[a], y = L[match[a]];
    ulm_loc3d o;
    o.frame = x.frame;
    o.i_xz = a;
    o.i_yz = match[a];
    o.reserved = 0;
    o.x = x.lat;
    o.y = y.lat;
    o.z = 0.5f * (x.z + y.z);
    o.amp_xz = x.amp;
    o.amp_yz = y.amp;
    o.reserved2 = 0.f;
    out[dst] = o;
}

}  // namespace

// exclusive scan on the device; part: workspace of 2 * ceil(n_max / SCAN_CHUNK) long longs
static rca_status device_scan(rca_handle* h, const int* cnt, int n_max, const int* n_dev, int cap_each, int* off,
                              int* total_true, long long* part)
{
    const int nb = std::max(1, (n_max + SCAN_CHUNK - 1) / SCAN_CHUNK);
    if (nb > 1024) return set_error(h, RCA_ERR_UNSUPPORTED, "scan over more than %d entries", 1024 * SCAN_CHUNK);
    k_scan_part<<<nb, SCAN_THREADS, 0, h->stream>>>(cnt, n_max, n_dev, cap_each, part);
    k_scan_top<<<1, 1024, 0, h->stream>>>(part, nb, n_max, n_dev, off, total_true);
    k_scan_apply<<<nb, SCAN_THREADS, 0, h->stream>>>(cnt, n_max, n_dev, cap_each, part, off);
    return cuda_check(h, cudaGetLastError(), "scan kernels");
}

rca_status launch_enhance(rca_handle* h, const rca_tables* t, const void* planes, rca_dtype pt, int F, int enh,
                          float* A, float* M)
{
    const GeomDev& g = t->gd;
    if (enh != ULM_ENH_XDOPPLER && enh != ULM_ENH_COHERENT) return set_error(h, RCA_ERR_INVALID_ARG, "bad enhancement mode");
    const size_t plane_sz = (size_t)g.nz * g.N;
    const size_t npx = 2 * (size_t)g.S * plane_sz;
    if (F > 48 * 1024) return set_error(h, RCA_ERR_UNSUPPORTED, "more than 49152 frames in one call");
    cudaMemsetAsync(M, 0, sizeof(float) * F, h->stream);
    // Every block walks all frames of its chunk, so the last wave of blocks
    // sets the tail: split the frames into chunks until the grid holds at
    // least eight waves of resident blocks (each chunk re-reads one frame;
    // at least 16 frames per chunk)
    const unsigned pblocks = (unsigned)((npx + 255) / 256);
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    auto kern = pt == RCA_C32 ? k_enhance<RCA_C32> : pt == RCA_C16F ? k_enhance<RCA_C16F> : k_enhance<RCA_C16BF>;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, (size_t)std::min(F, 16) * sizeof(unsigned));
    const unsigned resident = (unsigned)(std::max(1, per_sm) * sms);
    const int want = std::max(1, (int)((8u * resident + pblocks - 1) / pblocks));
    const int nchunk = std::min(want, std::max(1, F / 16));
    const int tf = (F + nchunk - 1) / nchunk;
    const size_t smem = (size_t)tf * sizeof(unsigned);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_check(h, e, "enhance smem attribute");
    dim3 grid(pblocks, (unsigned)((F + tf - 1) / tf));
    kern<<<grid, 256, smem, h->stream>>>(planes, F, g.S, plane_sz, enh, tf, A, reinterpret_cast<unsigned*>(M));
    return cuda_check(h, cudaGetLastError(), "enhance kernel");
}

rca_status launch_detect2d(rca_handle* h, const rca_tables* t, const float* A, const float* M, int F,
                           const ulm_params* prm, ulm_loc2d* out, int cap, int* n2d, float* ncc_out, int* plane_off)
{
    const GeomDev& g = t->gd;
    const int d = prm->d, hh = (d - 1) / 2;
    NccConst nc;
    nc.d = d;
    nc.h = hh;
    double G[RCA_MAX_NCC_D * RCA_MAX_NCC_D];
    double muG = 0.0;
    for (int a = -hh; a <= hh; ++a) {
        nc.gz[a + hh] = (float)std::exp(-(double)(a * a) / (2.0 * (double)prm->sig_z * prm->sig_z));
        nc.gl[a + hh] = (float)std::exp(-(double)(a * a) / (2.0 * (double)prm->sig_lat * prm->sig_lat));
    }
    for (int a = 0; a < d; ++a)
        for (int b = 0; b < d; ++b) {
            G[a * d + b] = (double)nc.gz[a] * (double)nc.gl[b];
            muG += G[a * d + b];
        }
    muG /= (double)(d * d);
    double ssG = 0.0;
    for (int q = 0; q < d * d; ++q) ssG += (G[q] - muG) * (G[q] - muG);
    nc.muG = (float)muG;
    nc.inv_ssG_sqrt = (float)(1.0 / std::sqrt(ssG));
    nc.flat_coef = (float)(1e-5 * d * d);
    nc.alpha = prm->alpha;
    nc.ncc_min = prm->ncc_min;

    const int nstrip = (g.nz + NCC_RS - 1) / NCC_RS;
    const int nplanes = F * 2 * g.S;
    const int nslots = nplanes * nstrip;
    rca_status st = RCA_OK;
    ulm_loc2d* cand = (ulm_loc2d*)ws_get(h, WS_CAND, (size_t)nslots * CAND_CAP * sizeof(ulm_loc2d), &st);
    if (!cand) return st;
    int* cnt = (int*)ws_get(h, WS_CANDCNT, (size_t)nslots * sizeof(int), &st);
    if (!cnt) return st;
    int* off = (int*)ws_get(h, WS_SCAN, (size_t)(nslots + 1) * sizeof(int), &st);
    if (!off) return st;
    if (g.N % 2 != 0 || g.N > 256) return set_error(h, RCA_ERR_UNSUPPORTED, "NCC detection needs an even N <= 256");
    const int rin = NCC_RS + 2 + 2 * hh;
    // two buffers of amplitude rows (later the NCC rows, stride N + 1) + three
    // padded vertical-sum arrays of row pairs
    // + the amplitude flags of the NCC rows ([NCC_RS + 2][N] bytes)
    size_t smem = (2 * std::max((size_t)rin * g.N, (size_t)(NCC_RS + 2) * (g.N + 1)) +
                   (size_t)3 * ((NCC_RS + 2) / 2) * det_npad(g.N, hh, det_hb(hh)) * 2) * sizeof(float) +
                  (size_t)(NCC_RS + 2) * g.N;
    // persistent CTAs (as many as fit on an SM, each walking (plane, strip)
    // items with the next item's rows in flight), never more CTAs than items
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = cudaSuccess;
    switch (hh) {
#define RCA_DETECT_LAUNCH(HV, NV)                                                                          \
    do {                                                                                                   \
        e = cudaFuncSetAttribute(k_detect<HV, NV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
        if (e != cudaSuccess) return cuda_check(h, e, "detect smem attribute");                          \
        int per_sm = 0;                                                                                    \
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_detect<HV, NV>, NCC_THREADS, smem);       \
        const dim3 grid((unsigned)std::max(1, std::min(nslots, std::max(1, per_sm) * sms)));               \
        k_detect<HV, NV><<<grid, NCC_THREADS, smem, h->stream>>>(A, M, g.S, g.nz, g.N, nplanes, nc, cand, cnt, \
                                                                 ncc_out, h->d_status);                   \
    } while (0)
#define RCA_DETECT_CASE(HV)                                                                                \
    case HV:                                                                                               \
        if (g.N == 128) RCA_DETECT_LAUNCH(HV, 128);                                                        \
        else if (g.N == 32) RCA_DETECT_LAUNCH(HV, 32);                                                     \
        else RCA_DETECT_LAUNCH(HV, 0);                                                                     \
        break;
        RCA_DETECT_CASE(1)
        RCA_DETECT_CASE(2)
        RCA_DETECT_CASE(3)
        RCA_DETECT_CASE(4)
        RCA_DETECT_CASE(5)
        RCA_DETECT_CASE(6)
        RCA_DETECT_CASE(7)
#undef RCA_DETECT_CASE
#undef RCA_DETECT_LAUNCH
    default: return set_error(h, RCA_ERR_INVALID_ARG, "NCC kernel length out of range");
    }
    long long* part = (long long*)ws_get(h, WS_N2D, (size_t)2 * 1024 * sizeof(long long), &st);
    if (!part) return st;
    if ((st = device_scan(h, cnt, nslots, nullptr, CAND_CAP, off, n2d, part)) != RCA_OK) return st;
    k_gather<<<(nslots + 7) / 8, 256, 0, h->stream>>>(cand, cnt, off, nslots, out, cap, A, g.S, g.nz, g.N,
                                                      h->d_status);
    if (plane_off) k_strip_to_plane<<<(nplanes + 1 + 255) / 256, 256, 0, h->stream>>>(off, nstrip, nplanes, plane_off);
    return cuda_check(h, cudaGetLastError(), "detect kernels");
}

rca_status launch_pair3d(rca_handle* h, const rca_tables* t, const ulm_loc2d* L, const int* n2d, int cap2d, int F,
                         ulm_loc3d* out, int cap3d, int* n3d)
{
    const GeomDev& g = t->gd;
    const int nplanes = F * 2 * g.S;
    rca_status st = RCA_OK;
    int* poff = (int*)ws_get(h, WS_PLANEOFF, (size_t)(nplanes + 1) * sizeof(int), &st);
    if (!poff) return st;
    const int nn = std::max(cap2d, 1);
    int* match = (int*)ws_get(h, WS_FLAGS, (size_t)nn * 2 * sizeof(int), &st);
    if (!match) return st;
    int* flags = match + nn;
    int* off = (int*)ws_get(h, WS_MISC, (size_t)(nn + 1) * sizeof(int), &st);
    if (!off) return st;
    k_list_plane_offsets<<<(nplanes + 1 + 255) / 256, 256, 0, h->stream>>>(L, n2d, cap2d, g.S, nplanes, poff);
    k_pair_match<<<(nn + 255) / 256, 256, 0, h->stream>>>(L, n2d, cap2d, g.S, g.P, poff, match);
    k_match_flags<<<(nn + 255) / 256, 256, 0, h->stream>>>(match, n2d, cap2d, flags);
    long long* part = (long long*)ws_get(h, WS_N2D, (size_t)2 * 1024 * sizeof(long long), &st);
    if (!part) return st;
    if ((st = device_scan(h, flags, nn, n2d, 0, off, n3d, part)) != RCA_OK) return st;
    k_pair_write<<<(nn + 255) / 256, 256, 0, h->stream>>>(L, n2d, cap2d, match, off, out, cap3d, h->d_status);
    return cuda_check(h, cudaGetLastError(), "pair kernels");
}

// ---------------------------------------------------------------------------
// Pairing without allocation (ulm_pair3d_noalloc).
//
// ulm_pair3d takes its scratch from the handle's workspace, which grows with
// cudaMalloc the first time a longer list arrives.  Some callers must not
// allocate once they are running: an acquisition loop that sized its device
// memory before the first ensemble cannot afford the device-wide stall of an
// allocation, or its failure, in the middle of a scan; a program whose own
// memory pool already holds the free HBM would see the allocation fail.
// For them the same kernels run on a fixed scratch array compiled into this
// file.  Being a file-scope __device__ variable, the array exists once per
// device, shared by every handle and call on it: calls whose work overlaps
// on the GPU race on it.  Its address is looked up once per device, on the
// first call made with that device current, and kept for the life of the
// process (a device reset makes the kept address stale; rca.h says so).
//
// Nothing in it needs clearing between calls: each call writes every entry
// it reads (plane offsets for all planes, flags for all list slots, match
// indices and scan offsets for all live entries, one partial per scan
// chunk), so the previous call's contents are never seen.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t na_round(size_t b) { return (b + 255) & ~(size_t)255; }
constexpr int NA_CHUNKS = (ULM_PAIR3D_NOALLOC_MAX_2D + SCAN_CHUNK - 1) / SCAN_CHUNK;
constexpr size_t NA_POFF = 0;
constexpr size_t NA_MATCH = NA_POFF + na_round((size_t)(ULM_PAIR3D_NOALLOC_MAX_PLANES + 1) * sizeof(int));
constexpr size_t NA_FLAGS = NA_MATCH + na_round((size_t)ULM_PAIR3D_NOALLOC_MAX_2D * sizeof(int));
constexpr size_t NA_OFF = NA_FLAGS + na_round((size_t)ULM_PAIR3D_NOALLOC_MAX_2D * sizeof(int));
constexpr size_t NA_PART = NA_OFF + na_round((size_t)(ULM_PAIR3D_NOALLOC_MAX_2D + 1) * sizeof(int));
constexpr size_t NA_BYTES = NA_PART + na_round((size_t)2 * NA_CHUNKS * sizeof(long long));
static_assert(NA_BYTES == ULM_PAIR3D_NOALLOC_SCRATCH_BYTES, "scratch size stated in rca.h is stale");
static_assert(NA_CHUNKS <= 1024, "device_scan handles at most 1024 chunks");

constexpr int NA_MAX_DEVICES = 64;

}  // namespace

static __device__ __align__(256) unsigned char g_pair_scratch[NA_BYTES];

static std::mutex g_pair_scratch_mu;
static unsigned char* g_pair_scratch_dev[NA_MAX_DEVICES];  // per device, null until looked up

// device address of g_pair_scratch on the handle's device (which is current)
static rca_status pair_scratch(rca_handle* h, unsigned char** base)
{
    if (h->device < 0 || h->device >= NA_MAX_DEVICES)
        return set_error(h, RCA_ERR_UNSUPPORTED, "ulm_pair3d_noalloc: device %d beyond %d", h->device, NA_MAX_DEVICES);
    std::lock_guard<std::mutex> lock(g_pair_scratch_mu);
    if (!g_pair_scratch_dev[h->device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_pair_scratch);
        if (e != cudaSuccess) return cuda_check(h, e, "ulm_pair3d_noalloc scratch address");
        if (!p) return set_error(h, RCA_ERR_CUDA, "ulm_pair3d_noalloc: null scratch address");
        g_pair_scratch_dev[h->device] = static_cast<unsigned char*>(p);
    }
    *base = g_pair_scratch_dev[h->device];
    return RCA_OK;
}

rca_status launch_pair3d_noalloc(rca_handle* h, const rca_tables* t, const ulm_loc2d* L, const int* n2d, int cap2d,
                                 int F, ulm_loc3d* out, int cap3d, int* n3d)
{
    const GeomDev& g = t->gd;
    const long long nplanes = (long long)F * 2 * g.S;
    if (cap2d > ULM_PAIR3D_NOALLOC_MAX_2D)
        return set_error(h, RCA_ERR_UNSUPPORTED, "ulm_pair3d_noalloc: cap2d %d exceeds its fixed scratch of %d entries",
                         cap2d, ULM_PAIR3D_NOALLOC_MAX_2D);
    if (nplanes > ULM_PAIR3D_NOALLOC_MAX_PLANES)
        return set_error(h, RCA_ERR_UNSUPPORTED, "ulm_pair3d_noalloc: %lld planes exceed its fixed scratch of %d planes",
                         nplanes, ULM_PAIR3D_NOALLOC_MAX_PLANES);
    unsigned char* base = nullptr;
    rca_status st = pair_scratch(h, &base);
    if (st != RCA_OK) return st;
    int* poff = reinterpret_cast<int*>(base + NA_POFF);
    int* match = reinterpret_cast<int*>(base + NA_MATCH);
    int* flags = reinterpret_cast<int*>(base + NA_FLAGS);
    int* off = reinterpret_cast<int*>(base + NA_OFF);
    long long* part = reinterpret_cast<long long*>(base + NA_PART);
    const int nn = std::max(cap2d, 1);
    const int np = (int)nplanes;
    k_list_plane_offsets<<<(np + 1 + 255) / 256, 256, 0, h->stream>>>(L, n2d, cap2d, g.S, np, poff);
    k_pair_match<<<(nn + 255) / 256, 256, 0, h->stream>>>(L, n2d, cap2d, g.S, g.P, poff, match);
    k_match_flags<<<(nn + 255) / 256, 256, 0, h->stream>>>(match, n2d, cap2d, flags);
    if ((st = device_scan(h, flags, nn, n2d, 0, off, n3d, part)) != RCA_OK) return st;
    k_pair_write<<<(nn + 255) / 256, 256, 0, h->stream>>>(L, n2d, cap2d, match, off, out, cap3d, h->d_status);
    return cuda_check(h, cudaGetLastError(), "pair kernels (no-alloc)");
}

rca_status launch_detect_map(rca_handle* h, const rca_tables* t, const float* map, int up, const float* A, const float* M,
                             int F, float score_min, float alpha, ulm_loc2d* out, int cap, int* n2d)
{
    const GeomDev& g = t->gd;
    const int H4 = g.nz * up, W4 = g.N * up;
    const int nstrip = (H4 + DET_RS - 1) / DET_RS;
    const int nplanes = F * 2 * g.S;
    const int nslots = nplanes * nstrip;
    rca_status st = RCA_OK;
    ulm_loc2d* cand = (ulm_loc2d*)ws_get(h, WS_CAND, (size_t)nslots * CAND_CAP * sizeof(ulm_loc2d), &st);
    if (!cand) return st;
    int* cnt = (int*)ws_get(h, WS_CANDCNT, (size_t)nslots * sizeof(int), &st);
    if (!cnt) return st;
    int* off = (int*)ws_get(h, WS_SCAN, (size_t)(nslots + 1) * sizeof(int), &st);
    if (!off) return st;
    long long* part = (long long*)ws_get(h, WS_N2D, (size_t)2 * 1024 * sizeof(long long), &st);
    if (!part) return st;
    // the strip's rows plus the candidate bitmap of its pixels
    const size_t smem = (size_t)(DET_RS + 2) * W4 * sizeof(float) + (size_t)((DET_RS * W4 + 31) / 32) * sizeof(unsigned);
    if (smem > 200 * 1024) return set_error(h, RCA_ERR_UNSUPPORTED, "map rows of %d fine pixels exceed shared memory", W4);
    cudaError_t e = cudaFuncSetAttribute(k_detect_map, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_check(h, e, "detect_map smem attribute");
    dim3 grid(nstrip, nplanes);
    k_detect_map<<<grid, 256, smem, h->stream>>>(map, up, A, M, g.S, g.nz, g.N, score_min, alpha, cand, cnt, h->d_status);
    if ((st = device_scan(h, cnt, nslots, nullptr, CAND_CAP, off, n2d, part)) != RCA_OK) return st;
    k_gather<<<(nslots + 7) / 8, 256, 0, h->stream>>>(cand, cnt, off, nslots, out, cap, nullptr, 0, 0, 0,
                                                      h->d_status);
    return cuda_check(h, cudaGetLastError(), "detect_map kernels");
}
