// Eigen-based SVD clutter filter on the Stage-1 slices (Sec. II-A2): for each
// transmission k, the frames' slices form the Casorati matrix X_k (pixels x
// frames); the filter removes the subspace of the n_c largest eigenvalues of
// the frame covariance C_k = X_k^H X_k:  X_k <- X_k - X_k Q Q^H.
//   k_svd_cov_tc   partial covariance tiles of 128 x 128 frames over one split
//                  of the pixels on the tensor cores (tcgen05, kind::tf32, FP32
//                  accumulators in TMEM), FP32-accurate by three TF32 products
//   k_svd_covsum   deterministic sum of the splits, Hermitian completion
//   k_svd_cq, k_svd_orth  orthogonal iteration Q <- orth(C Q) towards the
//                  n_c-dim dominant eigenspace: the product over many CTAs, the
//                  orthonormalisation (classical Gram-Schmidt applied twice) in
//                  one CTA per transmission; the projection needs the subspace only
//   k_svd_project  thread per pixel: t = X[p] Q, then X[p] -= t Q^H (in place)
//   k_svd_info     (on request) Rayleigh quotients of the removed basis and of
//                  one extra iterated vector, and the invariance residual
//                  ||C Q - Q (Q^H C Q)||_F of the removed subspace
// The iteration carries nc + 1 vectors (one beyond the rank, when F allows):
// Gram-Schmidt keeps the first nc columns independent of the last, so the
// removed subspace is that of an nc-vector iteration, and the extra column's
// Rayleigh quotient estimates the first eigenvalue left in the data.
#include <algorithm>
#include <cmath>

#include "rca_internal.cuh"

namespace {

#define SV_THREADS 512     // subspace CTA

__device__ __forceinline__ float2 sv_cmul(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }

// ---------------------------------------------------------------------------
// Covariance on the tensor cores.  With X = Xr + i Xi (pixels x frames),
//   Re C = Xr^T Xr + Xi^T Xi,   Im C = Xr^T Xi - Xi^T Xr,
// four real products per frame-tile pair, each a K-major GEMM over the pixels
// (a frame's slice is contiguous in pixels).  FP32 accuracy from TF32 operands:
// x = hi + lo with hi = tf32(x), lo = tf32(x - hi), and a product a b taken as
// hi hi + hi lo + lo hi (the dropped lo lo term is 2^-22 of it).  CTA = (frame
// tile pair ta <= tb of 128 frames each, transmission, pixel split), 160
// threads.  Converter thread r < 128 owns frame row a0 + r of the A tile and
// b0 + r of the B tile: per 16-pixel chunk it writes its rows into eight
// operand tiles (A / B x re / im x hi / lo, 128 rows x 16 TF32 each, K-major,
// no swizzle: core matrix (k group kg of 4, row group mg of 8 rows) at byte
// kg 2048 + mg 128, row r % 8 at + 16 (r % 8)) of one of three stages and
// arrives on the stage's `full` barrier; the first thread of the fifth warp
// waits for it, issues the chunk's 24 MMAs (M = N = 128, K = 8) and commits
// them to the stage's `empty` barrier, which the converters wait on before
// reusing the stage.  Each converter loads the next chunk into registers
// meanwhile.  Accumulators in TMEM (lane = A row, column = B row): Re at
// columns 0-127, Xr^T Xi at 128-255, Xi^T Xr at 256-383; the epilogue
// writes Re + i (the difference) into part[k][split][a][b] (a in tile ta, b in
// tile tb).
// Every mbarrier wait is bounded; on a timeout the CTA records ST_TIMEOUT,
// waits once more (bounded) for the commit of its MMAs in flight, frees TMEM
// and returns.  If that second wait also runs out, MMAs may still be in
// flight when TMEM is freed: nothing then guarantees the CTA's accumulators,
// and the status word says the call failed.
// ---------------------------------------------------------------------------
#define SVT_M 128
#define SVT_PC 16                           // pixels per chunk
#define SVT_TILE (SVT_M * SVT_PC * 4)       // one operand tile, bytes
#define SVT_STAGE (8 * SVT_TILE)
#define SVT_STAGES 3
#define SVT_SMEM (SVT_STAGES * SVT_STAGE)
#define SVT_CONV 128                        // converter threads (one per tile row)
#define SVT_THREADS (SVT_CONV + 32)         // + one warp whose first thread issues the MMAs
#define SVT_TMEM_COLS 512
#define SVT_KMAX 1024                       // pixels per split at most
enum { SVT_ARH = 0, SVT_ARL, SVT_AIH, SVT_AIL, SVT_BRH, SVT_BRL, SVT_BIH, SVT_BIL };

__device__ __forceinline__ unsigned svt_tf32(float x)
{
    unsigned r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// hi and lo TF32 parts of four values
__device__ __forceinline__ void svt_split(float x0, float x1, float x2, float x3, uint4& hi, uint4& lo)
{
    hi = make_uint4(svt_tf32(x0), svt_tf32(x1), svt_tf32(x2), svt_tf32(x3));
    lo = make_uint4(svt_tf32(x0 - __uint_as_float(hi.x)), svt_tf32(x1 - __uint_as_float(hi.y)),
                    svt_tf32(x2 - __uint_as_float(hi.z)), svt_tf32(x3 - __uint_as_float(hi.w)));
}

__device__ __forceinline__ void svt_st16(unsigned addr, uint4 v)
{
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w)
                 : "memory");
}

// shared-memory matrix descriptor: start, leading (K) and stride (M / N) byte
// offsets in 16-byte units, descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t svt_sdesc(unsigned saddr, unsigned lbo, unsigned sbo)
{
    return (uint64_t)((saddr >> 4) & 0x3fff) | ((uint64_t)((lbo >> 4) & 0x3fff) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3fff) << 32) | (1ull << 46);
}

// instruction descriptor of kind::tf32: D FP32, A and B TF32 (format 2), both
// K-major, M = N = 128
__host__ __device__ constexpr unsigned svt_idesc()
{
    return (1u << 4) | (2u << 7) | (2u << 10) | ((unsigned)(SVT_M >> 3) << 17) | ((unsigned)(SVT_M >> 4) << 24);
}

__device__ __forceinline__ void svt_mma(unsigned tmem_d, uint64_t da, uint64_t db, int accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(tmem_d), "l"(da), "l"(db), "r"(svt_idesc()), "r"(accumulate)
        : "memory");
}

// 32 consecutive FP32 accumulator columns of this warp's 32 TMEM lanes
__device__ __forceinline__ void svt_ld32(unsigned taddr, float* v)
{
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        unsigned r[16];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
            "%14, %15}, [%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(taddr + 16u * h));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int q = 0; q < 16; ++q) v[16 * h + q] = __uint_as_float(r[q]);
    }
}

__device__ __forceinline__ void svt_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__global__ void __launch_bounds__(SVT_THREADS, 1) k_svd_cov_tc(const float2* __restrict__ sl, int F, int nt, int P,
                                                               int ntile, int psplit, float2* __restrict__ part,
                                                               unsigned* __restrict__ status)
{
    extern __shared__ __align__(128) unsigned char svsm[];
    __shared__ uint64_t full[SVT_STAGES], empty[SVT_STAGES], done;
    __shared__ unsigned s_tmem;
    __shared__ volatile int abort_flag;
    int pair = blockIdx.x, ta = 0;
    while (pair >= ntile - ta) {
        pair -= ntile - ta;
        ++ta;
    }
    const int tb = ta + pair;
    const int k = blockIdx.y, split = blockIdx.z;
    const int a0 = ta * SVT_M, b0 = tb * SVT_M;
    const int p0 = split * psplit, p1 = min(P, p0 + psplit);
    const int nch = p1 > p0 ? (p1 - p0 + SVT_PC - 1) / SVT_PC : 0;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(SVT_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        for (int q = 0; q < SVT_STAGES; ++q) {
            mbar_init(&full[q], SVT_CONV);
            mbar_init(&empty[q], 1);
        }
        mbar_init(&done, 1);
        abort_flag = 0;
        mbar_fence_init();
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = s_tmem;
    const unsigned sbase = smem_u32(svsm);
    if (threadIdx.x < SVT_CONV) {
        // converter: row r of the A tile (frame a0 + r) and of the B tile (b0 + r)
        const int r = threadIdx.x;
        const int fa = a0 + r, fb = b0 + r;
        const float4* ga = fa < F ? reinterpret_cast<const float4*>(sl + ((size_t)fa * nt + k) * P) : nullptr;
        const float4* gb = fb < F ? reinterpret_cast<const float4*>(sl + ((size_t)fb * nt + k) * P) : nullptr;
        const unsigned roff = (unsigned)(r * 16);   // (r / 8) 128 + (r % 8) 16
        // float4 j of a raw chunk row holds pixels 2 j, 2 j + 1 (re, im, re, im)
        auto load = [&](int c, float4 (&xa)[8], float4 (&xb)[8]) {
            const int pc = p0 + c * SVT_PC;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int p = pc + 2 * j;   // pixel pairs are either inside [p0, p1) or outside (P % 4 == 0)
                const bool in = c < nch && p < p1;
                xa[j] = (ga && in) ? __ldg(ga + p / 2) : make_float4(0.f, 0.f, 0.f, 0.f);
                xb[j] = (gb && in) ? __ldg(gb + p / 2) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
        };
        float4 ra[8], rb[8];
        load(0, ra, rb);
        for (int c = 0; c < nch; ++c) {
            const int q = c % SVT_STAGES, u = c / SVT_STAGES;
            float4 na[8], nb[8];
            load(c + 1, na, nb);
            // use u of stage q waits until the MMAs of use u - 1 have read it
            if (u > 0 && !mbar_wait_bounded(&empty[q], (unsigned)(u - 1) & 1u)) abort_flag = 1;
            if (abort_flag) break;
            const unsigned st = sbase + (unsigned)(q * SVT_STAGE) + roff;
#pragma unroll
            for (int i = 0; i < 4; ++i) {   // k group i: pixels 4 i .. 4 i + 3 of the chunk
                uint4 h, l;
                const float4 x0 = ra[2 * i], x1 = ra[2 * i + 1];
                svt_split(x0.x, x0.z, x1.x, x1.z, h, l);
                svt_st16(st + SVT_ARH * SVT_TILE + i * 2048, h);
                svt_st16(st + SVT_ARL * SVT_TILE + i * 2048, l);
                svt_split(x0.y, x0.w, x1.y, x1.w, h, l);
                svt_st16(st + SVT_AIH * SVT_TILE + i * 2048, h);
                svt_st16(st + SVT_AIL * SVT_TILE + i * 2048, l);
                const float4 y0 = rb[2 * i], y1 = rb[2 * i + 1];
                svt_split(y0.x, y0.z, y1.x, y1.z, h, l);
                svt_st16(st + SVT_BRH * SVT_TILE + i * 2048, h);
                svt_st16(st + SVT_BRL * SVT_TILE + i * 2048, l);
                svt_split(y0.y, y0.w, y1.y, y1.w, h, l);
                svt_st16(st + SVT_BIH * SVT_TILE + i * 2048, h);
                svt_st16(st + SVT_BIL * SVT_TILE + i * 2048, l);
            }
            // this thread's generic-proxy writes before the tensor cores read them
            fence_proxy_async();
            svt_arrive(&full[q]);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                ra[j] = na[j];
                rb[j] = nb[j];
            }
        }
    } else if (lane == 0) {
        // MMA issue (first thread of the fifth warp; the rest of the warp waits
        // at the __syncwarp below): the 24 MMAs of chunk c once its stage is
        // full, committed to the stage's empty barrier; the final commit (all
        // MMAs) to `done`
        const unsigned dRe = tmem, dP = tmem + 128, dN = tmem + 256;
        for (int c = 0; c < nch; ++c) {
            const int q = c % SVT_STAGES, u = c / SVT_STAGES;
            if (!mbar_wait_bounded(&full[q], (unsigned)u & 1u)) abort_flag = 1;
            if (abort_flag) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const unsigned sq = sbase + (unsigned)(q * SVT_STAGE);
            auto d = [&](int t, int s) { return svt_sdesc(sq + t * SVT_TILE + s * 4096, 2048, 128); };
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                const int acc = (c | s) != 0;
                svt_mma(dRe, d(SVT_ARH, s), d(SVT_BRH, s), acc);
                svt_mma(dRe, d(SVT_ARH, s), d(SVT_BRL, s), 1);
                svt_mma(dRe, d(SVT_ARL, s), d(SVT_BRH, s), 1);
                svt_mma(dRe, d(SVT_AIH, s), d(SVT_BIH, s), 1);
                svt_mma(dRe, d(SVT_AIH, s), d(SVT_BIL, s), 1);
                svt_mma(dRe, d(SVT_AIL, s), d(SVT_BIH, s), 1);
                svt_mma(dP, d(SVT_ARH, s), d(SVT_BIH, s), acc);
                svt_mma(dP, d(SVT_ARH, s), d(SVT_BIL, s), 1);
                svt_mma(dP, d(SVT_ARL, s), d(SVT_BIH, s), 1);
                svt_mma(dN, d(SVT_AIH, s), d(SVT_BRH, s), acc);
                svt_mma(dN, d(SVT_AIH, s), d(SVT_BRL, s), 1);
                svt_mma(dN, d(SVT_AIL, s), d(SVT_BRH, s), 1);
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&empty[q]))
                         : "memory");
        }
        // arrives once every MMA issued above has completed (none issued: at once)
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(&done))
                     : "memory");
    }
    if (warp == SVT_CONV / 32) __syncwarp();
    // every thread: the MMAs complete (bounded) before the accumulators are read or freed
    const bool fin = mbar_wait_bounded(&done, 0u);
    if (__syncthreads_or(!fin || abort_flag)) {
        if (threadIdx.x == 0) atomicOr(status, ST_TIMEOUT);
        // one more bounded wait for the MMAs still in flight before the
        // barriers are invalidated and TMEM is freed (the MMA thread commits
        // `done` after its last issue even when it stopped early)
        if (!fin) mbar_wait_bounded(&done, 0u);
        __syncthreads();
    } else if (nch > 0 && warp < SVT_CONV / 32) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        float2* dst = part + (((size_t)k * gridDim.z + split) * F) * F;
        const int a = a0 + 32 * warp + lane;
        const unsigned lrow = (unsigned)(32 * warp) << 16;
#pragma unroll 1
        for (int cg = 0; cg < 4; ++cg) {
            float re[32], ip[32], in[32];
            svt_ld32(tmem + lrow + (unsigned)(32 * cg), re);
            svt_ld32(tmem + lrow + 128u + (unsigned)(32 * cg), ip);
            svt_ld32(tmem + lrow + 256u + (unsigned)(32 * cg), in);
            if (a < F) {
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int b = b0 + 32 * cg + j;
                    if (b < F) dst[(size_t)a * F + b] = make_float2(re[j], ip[j] - in[j]);
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 0; q < SVT_STAGES; ++q) {
            asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(&full[q])) : "memory");
            asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(&empty[q])) : "memory");
        }
        asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(&done)) : "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(SVT_TMEM_COLS)
                     : "memory");
    }
}

// C[k][a][b] = sum over splits for a <= b, C[b][a] = conj(C[a][b]): the lower
// half of the diagonal tiles is computed but not used, so C is exactly Hermitian
__global__ void k_svd_covsum(const float2* __restrict__ part, int F, int nsplit, float2* __restrict__ C)
{
    const int k = blockIdx.y;
    float2* Ck = C + (size_t)k * F * F;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < F * F; idx += gridDim.x * blockDim.x) {
        const int a = idx / F, b = idx - a * F;
        if (a > b) continue;
        float2 s = make_float2(0.f, 0.f);
        for (int q = 0; q < nsplit; ++q) {
            const float2 v = part[(((size_t)k * nsplit + q) * F + a) * F + b];
            s.x += v.x;
            s.y += v.y;
        }
        Ck[(size_t)a * F + b] = s;
        if (a < b) Ck[(size_t)b * F + a] = make_float2(s.x, -s.y);
    }
}

// deterministic start vectors in [-1, 1]
__device__ __forceinline__ float sv_hash(unsigned x)
{
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return (float)(x & 0xffffff) * (2.0f / 16777216.0f) - 1.0f;
}

// block sum of one float (all threads get the result)
__device__ __forceinline__ float sv_bsum(float v, float* red)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    float s = 0.f;
    for (int w = 0; w < nw; ++w) s += red[w];
    return s;
}

// Orthonormalise the nc columns of Y (pitch ld) into Q by classical
// Gram-Schmidt applied twice per column.
__device__ void sv_orth(float2* Y, float2* Q, int F, int nc, int ld, float2* rbuf, float* red)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int j = 0; j < nc; ++j) {
        for (int pass = 0; pass < 2; ++pass) {
            // r_i = Q_i^H y_j, one warp per previous column
            for (int i = warp; i < j; i += nw) {
                float2 s = make_float2(0.f, 0.f);
                for (int g = lane; g < F; g += 32) {
                    const float2 q = Q[g * ld + i], y = Y[g * ld + j];
                    s.x += q.x * y.x + q.y * y.y;
                    s.y += q.x * y.y - q.y * y.x;
                }
                for (int o = 16; o > 0; o >>= 1) {
                    s.x += __shfl_xor_sync(0xffffffffu, s.x, o);
                    s.y += __shfl_xor_sync(0xffffffffu, s.y, o);
                }
                if (lane == 0) rbuf[i] = s;
            }
            __syncthreads();
            for (int g = threadIdx.x; g < F; g += blockDim.x) {
                float2 y = Y[g * ld + j];
                for (int i = 0; i < j; ++i) {
                    const float2 t = sv_cmul(rbuf[i], Q[g * ld + i]);
                    y.x -= t.x;
                    y.y -= t.y;
                }
                Y[g * ld + j] = y;
            }
            __syncthreads();
        }
        float e = 0.f;
        for (int g = threadIdx.x; g < F; g += blockDim.x) {
            const float2 y = Y[g * ld + j];
            e += y.x * y.x + y.y * y.y;
        }
        const float nrm = sqrtf(sv_bsum(e, red));
        const float inv = nrm > 0.f ? 1.0f / nrm : 0.f;
        for (int g = threadIdx.x; g < F; g += blockDim.x) {
            const float2 y = Y[g * ld + j];
            Q[g * ld + j] = make_float2(y.x * inv, y.y * inv);
        }
        __syncthreads();
    }
}

// Orthogonal iteration for the nc-dimensional dominant eigenspace of each
// C_k, one step = k_svd_cq (Y = C Q over many CTAs) then k_svd_orth (one CTA
// per transmission: Y -> orthonormal Q); k_svd_orth with `start` set builds
// the fixed start basis.  Q, Y: [k][F][nc] in global memory.
__global__ void __launch_bounds__(SV_THREADS) k_svd_orth(float2* __restrict__ Yg, float2* __restrict__ Qg, int F,
                                                         int nc, int start)
{
    extern __shared__ float2 ssv[];
    __shared__ float red[32];
    __shared__ float2 rbuf[32];
    const int ld = nc + 1;                             // padded: lanes over g spread over the banks
    float2* Q = ssv;                                   // [F][ld]
    float2* Y = ssv + (size_t)F * ld;                  // [F][ld]
    const int k = blockIdx.x;
    for (int idx = threadIdx.x; idx < F * nc; idx += blockDim.x) {
        const int g = idx / nc, j = idx - g * nc;
        Y[g * ld + j] = start ? make_float2(sv_hash(2u * (unsigned)idx + 1u), sv_hash(2u * (unsigned)idx + 2u))
                              : Yg[((size_t)k * F + g) * nc + j];
    }
    __syncthreads();
    sv_orth(Y, Q, F, nc, ld, rbuf, red);
    for (int idx = threadIdx.x; idx < F * nc; idx += blockDim.x) {
        const int g = idx / nc, j = idx - g * nc;
        Qg[((size_t)k * F + g) * nc + j] = Q[g * ld + j];
    }
}

// Y[k] = C_k Q[k]: a thread per (row, column) of Y, rows in blocks of
// SV_THREADS / nc per CTA; Q[k] staged in shared memory
__global__ void __launch_bounds__(SV_THREADS) k_svd_cq(const float2* __restrict__ C, const float2* __restrict__ Qg,
                                                       int F, int nc, float2* __restrict__ Yg)
{
    extern __shared__ float2 ssv[];                    // Q[k] [F][nc]
    const int k = blockIdx.y;
    const float2* Qk = Qg + (size_t)k * F * nc;
    for (int idx = threadIdx.x; idx < F * nc; idx += blockDim.x) ssv[idx] = Qk[idx];
    __syncthreads();
    const int rows = blockDim.x / nc;
    const int f = blockIdx.x * rows + threadIdx.x / nc, j = threadIdx.x % nc;
    if (threadIdx.x >= rows * nc || f >= F) return;
    const float2* Crow = C + ((size_t)k * F + f) * F;
    float2 acc = make_float2(0.f, 0.f);
    for (int g = 0; g < F; ++g) {
        const float2 c = __ldg(Crow + g), q = ssv[g * nc + j];
        acc.x = fmaf(c.x, q.x, fmaf(-c.y, q.y, acc.x));
        acc.y = fmaf(c.x, q.y, fmaf(c.y, q.x, acc.y));
    }
    Yg[((size_t)k * F + f) * nc + j] = acc;
}

// thread per pixel: t = sum_f X[p][f] Q[f][:], X[p][f] -= sum_j t_j conj(Q[f][j]);
// frames in blocks of four, the block's loads issued before its arithmetic
#define SV_FB 4
__global__ void __launch_bounds__(128) k_svd_project(float2* __restrict__ sl, int F, int nt, int P, int nc, int nb,
                                                     const float2* __restrict__ Qall)
{
    extern __shared__ float2 ssv[];
    const int k = blockIdx.y;
    const float2* Qk = Qall + (size_t)k * F * nb;          // [F][nb]; the first nc columns are removed
    for (int idx = threadIdx.x; idx < F * nc; idx += blockDim.x) ssv[idx] = Qk[(idx / nc) * nb + idx % nc];
    __syncthreads();
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    const size_t fs = (size_t)nt * P;                  // frame stride
    float2* base = sl + (size_t)k * P + p;
    float2 t[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) t[j] = make_float2(0.f, 0.f);
    for (int f0 = 0; f0 < F; f0 += SV_FB) {
        float2 x[SV_FB];
#pragma unroll
        for (int u = 0; u < SV_FB; ++u) x[u] = f0 + u < F ? base[(size_t)(f0 + u) * fs] : make_float2(0.f, 0.f);
#pragma unroll
        for (int u = 0; u < SV_FB; ++u) {
            if (f0 + u >= F) break;
            const float2* qf = ssv + (f0 + u) * nc;
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                if (j < nc) {
                    const float2 q = qf[j];
                    t[j].x = fmaf(x[u].x, q.x, fmaf(-x[u].y, q.y, t[j].x));
                    t[j].y = fmaf(x[u].x, q.y, fmaf(x[u].y, q.x, t[j].y));
                }
            }
        }
    }
    for (int f0 = 0; f0 < F; f0 += SV_FB) {
        float2 x[SV_FB];
#pragma unroll
        for (int u = 0; u < SV_FB; ++u) x[u] = f0 + u < F ? base[(size_t)(f0 + u) * fs] : make_float2(0.f, 0.f);
#pragma unroll
        for (int u = 0; u < SV_FB; ++u) {
            if (f0 + u >= F) break;
            const float2* qf = ssv + (f0 + u) * nc;
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                if (j < nc) {
                    const float2 q = qf[j];
                    // t_j conj(q)
                    x[u].x = fmaf(-t[j].x, q.x, fmaf(-t[j].y, q.y, x[u].x));
                    x[u].y = fmaf(-t[j].y, q.x, fmaf(t[j].x, q.y, x[u].y));
                }
            }
            base[(size_t)(f0 + u) * fs] = x[u];
        }
    }
}

// One CTA per transmission, after Y = C Q (nb columns): H = Q^H Y, the
// Rayleigh quotients theta_j = Re H_jj, and the residual of the removed
// subspace R = Y_nc - Q_nc H_nc (first nc columns).  info[k] = {max and min
// theta_j over j < nc, theta_nc of the extra column (0 without one),
// ||R||_F / min_j theta_j}.
__global__ void __launch_bounds__(SV_THREADS) k_svd_info(const float2* __restrict__ Qg, const float2* __restrict__ Yg,
                                                        int F, int nc, int nb, float* __restrict__ info)
{
    extern __shared__ float2 ssv[];
    __shared__ float red[32];
    __shared__ float2 H[33 * 33];
    const int ld = nb + 1;
    float2* Q = ssv;                                   // [F][ld]
    float2* Y = ssv + (size_t)F * ld;                  // [F][ld]
    const int k = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int idx = threadIdx.x; idx < F * nb; idx += blockDim.x) {
        const int g = idx / nb, j = idx - g * nb;
        Q[g * ld + j] = Qg[((size_t)k * F + g) * nb + j];
        Y[g * ld + j] = Yg[((size_t)k * F + g) * nb + j];
    }
    __syncthreads();
    for (int e = warp; e < nb * nb; e += nw) {
        const int i = e / nb, j = e - i * nb;
        float2 acc = make_float2(0.f, 0.f);
        for (int g = lane; g < F; g += 32) {
            const float2 q = Q[g * ld + i], y = Y[g * ld + j];    // conj(q) y
            acc.x += q.x * y.x + q.y * y.y;
            acc.y += q.x * y.y - q.y * y.x;
        }
        for (int o = 16; o > 0; o >>= 1) {
            acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
            acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
        }
        if (lane == 0) H[i * nb + j] = acc;
    }
    __syncthreads();
    float r2 = 0.f;
    for (int idx = threadIdx.x; idx < F * nc; idx += blockDim.x) {
        const int g = idx / nc, j = idx - g * nc;
        float2 r = Y[g * ld + j];
        for (int i = 0; i < nc; ++i) {
            const float2 t = sv_cmul(Q[g * ld + i], H[i * nb + j]);
            r.x -= t.x;
            r.y -= t.y;
        }
        r2 += r.x * r.x + r.y * r.y;
    }
    r2 = sv_bsum(r2, red);
    if (threadIdx.x == 0) {
        float tmax = -INFINITY, tmin = INFINITY;
        for (int j = 0; j < nc; ++j) {
            tmax = fmaxf(tmax, H[j * nb + j].x);
            tmin = fminf(tmin, H[j * nb + j].x);
        }
        info[4 * k + 0] = tmax;
        info[4 * k + 1] = tmin;
        info[4 * k + 2] = nb > nc ? H[nc * nb + nc].x : 0.f;
        info[4 * k + 3] = tmin > 0.f ? sqrtf(r2) / tmin : INFINITY;
    }
}

}  // namespace

size_t svd_subspace_smem(int F, int nb) { return 2 * (size_t)F * (nb + 1) * sizeof(float2); }

rca_status launch_clutter_svd(rca_handle* h, const rca_tables* t, float2* slices, int F, int nc, int iters,
                              float* info)
{
    const GeomDev& g = t->gd;
    const int nt = 2 * g.K, P = g.nzs * g.N;
    if (nc < 0 || nc > 32) return set_error(h, RCA_ERR_INVALID_ARG, "clutter rank %d outside [0, 32]", nc);
    if (nc >= F) return set_error(h, RCA_ERR_INVALID_ARG, "clutter rank %d must be below the frame count %d", nc, F);
    if (iters < 1 || iters > 1000) return set_error(h, RCA_ERR_INVALID_ARG, "iterations %d outside [1, 1000]", iters);
    if (nc == 0) {
        if (info) {
            cudaError_t e0 = cudaMemsetAsync(info, 0, (size_t)4 * nt * sizeof(float), h->stream);
            if (e0 != cudaSuccess) return cuda_check(h, e0, "clutter info clear");
        }
        return RCA_OK;
    }
    const int nb = std::min(nc + 1, F);                 // iterated vectors: the rank plus one
    const size_t smem_sub = svd_subspace_smem(F, nb);
    if (smem_sub > 200 * 1024)
        return set_error(h, RCA_ERR_UNSUPPORTED, "frames x (rank + 2) = %d x %d exceeds the subspace kernel", F, nb + 1);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // the covariance's pixel quads stay whole: N is a multiple of 4 (geometry rule)
    if (P % 4 != 0) return set_error(h, RCA_ERR_UNSUPPORTED, "slice pixel count %d not a multiple of 4", P);
    // (tile pair, transmission, pixel split) CTAs, at least one wave, and at
    // most SVT_KMAX pixels per split, added on the CUDA cores (k_svd_covsum):
    // the error of one TMEM accumulation grows with its length (measured on the
    // 300-frame paper stack: 2.6e-5 of the input with 21 280 pixels per split,
    // 1.6e-6 with 1 024; 5.7e-7 for the CUDA-core FP32 covariance it replaced)
    const int ntile = (F + SVT_M - 1) / SVT_M, npair = ntile * (ntile + 1) / 2;
    int nsplit = std::max({1, sms / (npair * nt), (P + SVT_KMAX - 1) / SVT_KMAX});
    nsplit = std::min(nsplit, (P + SVT_PC - 1) / SVT_PC);
    const int psplit = ((P + nsplit - 1) / nsplit + SVT_PC - 1) / SVT_PC * SVT_PC;
    nsplit = (P + psplit - 1) / psplit;
    auto up = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t n_part = (size_t)nt * nsplit * F * F, n_C = (size_t)nt * F * F, n_Q = (size_t)nt * F * nb;
    const size_t bytes = up(n_part * 8) + up(n_C * 8) + 2 * up(n_Q * 8);
    rca_status st = RCA_OK;
    char* ws = (char*)ws_get(h, WS_SVD, bytes, &st);
    if (!ws) return st;
    float2* part = reinterpret_cast<float2*>(ws);
    float2* C = reinterpret_cast<float2*>(ws + up(n_part * 8));
    float2* Q = reinterpret_cast<float2*>((char*)C + up(n_C * 8));
    float2* Y = reinterpret_cast<float2*>((char*)Q + up(n_Q * 8));
    cudaError_t ea = cudaFuncSetAttribute(k_svd_cov_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, SVT_SMEM);
    if (ea != cudaSuccess) return cuda_check(h, ea, "covariance smem attribute");
    k_svd_cov_tc<<<dim3(npair, nt, nsplit), SVT_THREADS, SVT_SMEM, h->stream>>>(slices, F, nt, P, ntile, psplit,
                                                                                 part, h->d_status);
    k_svd_covsum<<<dim3((unsigned)std::min<size_t>(((size_t)F * F + 255) / 256, 1024), nt), 256, 0, h->stream>>>(
        part, F, nsplit, C);
    cudaError_t e = cudaFuncSetAttribute(k_svd_orth, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_sub);
    if (e != cudaSuccess) return cuda_check(h, e, "subspace smem attribute");
    const size_t smem_q = (size_t)F * nb * sizeof(float2);
    e = cudaFuncSetAttribute(k_svd_cq, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_q);
    if (e != cudaSuccess) return cuda_check(h, e, "subspace product smem attribute");
    const int rows_cq = SV_THREADS / nb;
    k_svd_orth<<<nt, SV_THREADS, smem_sub, h->stream>>>(Y, Q, F, nb, 1);
    for (int it = 0; it < iters; ++it) {
        k_svd_cq<<<dim3((F + rows_cq - 1) / rows_cq, nt), SV_THREADS, smem_q, h->stream>>>(C, Q, F, nb, Y);
        k_svd_orth<<<nt, SV_THREADS, smem_sub, h->stream>>>(Y, Q, F, nb, 0);
    }
    if (info) {
        k_svd_cq<<<dim3((F + rows_cq - 1) / rows_cq, nt), SV_THREADS, smem_q, h->stream>>>(C, Q, F, nb, Y);
        e = cudaFuncSetAttribute(k_svd_info, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_sub);
        if (e != cudaSuccess) return cuda_check(h, e, "clutter info smem attribute");
        k_svd_info<<<nt, SV_THREADS, smem_sub, h->stream>>>(Q, Y, F, nc, nb, info);
    }
    const size_t smem_proj = (size_t)F * nc * sizeof(float2);
    e = cudaFuncSetAttribute(k_svd_project, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_proj);
    if (e != cudaSuccess) return cuda_check(h, e, "projection smem attribute");
    k_svd_project<<<dim3((P + 127) / 128, nt), 128, smem_proj, h->stream>>>(slices, F, nt, P, nc, nb, Q);
    return cuda_check(h, cudaGetLastError(), "clutter filter kernels");
}
