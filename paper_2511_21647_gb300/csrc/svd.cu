// Eigen-based SVD clutter filter on the Stage-1 slices (Sec. II-A2): for each
// transmission k, the frames' slices form the Casorati matrix X_k (pixels x
// frames); the filter removes the subspace of the n_c largest eigenvalues of
// the frame covariance C_k = X_k^H X_k:  X_k <- X_k - X_k Q Q^H.
//   k_svd_cov      partial covariance tiles: 64 x 64 frames, 8 x 4 per thread,
//                  over one split of the pixels; slices staged frame-innermost
//                  in shared memory (double buffered); complex products on
//                  packed FP32 pairs
//   k_svd_covsum   deterministic sum of the splits, Hermitian completion
//   k_svd_cq, k_svd_orth  orthogonal iteration Q <- orth(C Q) towards the
//                  n_c-dim dominant eigenspace: the product over many CTAs, the
//                  orthonormalisation (classical Gram-Schmidt applied twice) in
//                  one CTA per transmission; the projection needs the subspace only
//   k_svd_project  thread per pixel: t = X[p] Q, then X[p] -= t Q^H (in place)
#include <algorithm>
#include <cmath>

#include "rca_internal.cuh"

namespace {

#define SV_T 64            // covariance tile (frames)
#define SV_PC 32           // pixels per staged chunk
#define SV_SP 68           // staged row pitch in float2 (frames + 4: 16-byte aligned, shifts banks)
#define SV_THREADS 512     // subspace CTA

__device__ __forceinline__ float2 sv_cmul(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }

// C_k partial sums for the frame tile pair (ta <= tb) over pixels [p0, p1):
// part[k][split][a][b] for a in tile ta, b in tile tb.  128 threads: thread
// (ty, tx) in 8 x 16 owns rows a0 + 8 ty .. + 7 and columns b0 + 4 tx .. + 3
// (32 complex accumulators); the staged chunk is double buffered.
__global__ void __launch_bounds__(128) k_svd_cov(const float2* __restrict__ sl, int F, int nt, int P, int ntile,
                                                 int psplit, float2* __restrict__ part)
{
    __shared__ __align__(16) float2 As[2][SV_PC][SV_SP];
    __shared__ __align__(16) float2 Bs[2][SV_PC][SV_SP];
    // tile pair from the linear upper-triangle index
    int pair = blockIdx.x, ta = 0;
    while (pair >= ntile - ta) {
        pair -= ntile - ta;
        ++ta;
    }
    const int tb = ta + pair;
    const int k = blockIdx.y, split = blockIdx.z;
    const int a0 = ta * SV_T, b0 = tb * SV_T;
    const int p0 = split * psplit, p1 = min(P, p0 + psplit);
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    // acc[i][j] = sum conj(X[a0 + 8 ty + i]) X[b0 + 4 tx + j] as (re, im) packed
    uint64_t acc[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0ull;
    // stage [pixel][frame] for chunk pc into buffer q with asynchronous 8-byte
    // copies (zero-filled outside the slice or the frame range): lanes over
    // pixels, so each warp reads slice rows contiguously
    auto stage = [&](int pc, int q) {
        for (int idx = threadIdx.x; idx < SV_T * SV_PC; idx += blockDim.x) {
            const int r = idx / SV_PC, c = idx - r * SV_PC;
            const int p = pc + c;
            const int fa = a0 + r, fb = b0 + r;
            const bool va = p < p1 && fa < F, vb = p < p1 && fb < F;
            const float2* ga = va ? sl + ((size_t)fa * nt + k) * P + p : sl;
            const float2* gb = vb ? sl + ((size_t)fb * nt + k) * P + p : sl;
            asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(smem_u32(&As[q][c][r])), "l"(ga),
                         "r"(va ? 8 : 0)
                         : "memory");
            asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(smem_u32(&Bs[q][c][r])), "l"(gb),
                         "r"(vb ? 8 : 0)
                         : "memory");
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    int q = 0;
    if (p0 < p1) stage(p0, 0);
    for (int pc = p0; pc < p1; pc += SV_PC) {
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        __syncthreads();                       // chunk pc staged in q; q ^ 1 free
        if (pc + SV_PC < p1) stage(pc + SV_PC, q ^ 1);
#pragma unroll 2
        for (int c = 0; c < SV_PC; ++c) {
            const float4 b01 = *reinterpret_cast<const float4*>(&Bs[q][c][4 * tx]);
            const float4 b23 = *reinterpret_cast<const float4*>(&Bs[q][c][4 * tx + 2]);
            // conj(a) b = a.re (b.re, b.im) + a.im (b.im, -b.re)
            const uint64_t bb[4] = {f2_pack(b01.x, b01.y), f2_pack(b01.z, b01.w), f2_pack(b23.x, b23.y),
                                    f2_pack(b23.z, b23.w)};
            const uint64_t bs[4] = {f2_pack(b01.y, -b01.x), f2_pack(b01.w, -b01.z), f2_pack(b23.y, -b23.x),
                                    f2_pack(b23.w, -b23.z)};
#pragma unroll
            for (int i2 = 0; i2 < 4; ++i2) {
                const float4 a = *reinterpret_cast<const float4*>(&As[q][c][8 * ty + 2 * i2]);
                const uint64_t ar0 = f2_pack(a.x, a.x), ai0 = f2_pack(a.y, a.y);
                const uint64_t ar1 = f2_pack(a.z, a.z), ai1 = f2_pack(a.w, a.w);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    acc[2 * i2][j] = f2_fma(ai0, bs[j], f2_fma(ar0, bb[j], acc[2 * i2][j]));
                    acc[2 * i2 + 1][j] = f2_fma(ai1, bs[j], f2_fma(ar1, bb[j], acc[2 * i2 + 1][j]));
                }
            }
        }
        q ^= 1;
    }
    float2* dst = part + (((size_t)k * gridDim.z + split) * F) * F;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int a = a0 + 8 * ty + i;
        if (a >= F) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int b = b0 + 4 * tx + j;
            if (b < F) dst[(size_t)a * F + b] = f2_unpack(acc[i][j]);
        }
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
__global__ void __launch_bounds__(128) k_svd_project(float2* __restrict__ sl, int F, int nt, int P, int nc,
                                                     const float2* __restrict__ Qall)
{
    extern __shared__ float2 ssv[];
    const int k = blockIdx.y;
    const float2* Qk = Qall + (size_t)k * F * nc;
    for (int idx = threadIdx.x; idx < F * nc; idx += blockDim.x) ssv[idx] = Qk[idx];
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

}  // namespace

size_t svd_subspace_smem(int F, int nc) { return 2 * (size_t)F * (nc + 1) * sizeof(float2); }

rca_status launch_clutter_svd(rca_handle* h, const rca_tables* t, float2* slices, int F, int nc, int iters)
{
    const GeomDev& g = t->gd;
    const int nt = 2 * g.K, P = g.nzs * g.N;
    if (nc < 0 || nc > 32) return set_error(h, RCA_ERR_INVALID_ARG, "clutter rank %d outside [0, 32]", nc);
    if (nc >= F) return set_error(h, RCA_ERR_INVALID_ARG, "clutter rank %d must be below the frame count %d", nc, F);
    if (iters < 1 || iters > 1000) return set_error(h, RCA_ERR_INVALID_ARG, "iterations %d outside [1, 1000]", iters);
    if (nc == 0) return RCA_OK;
    const size_t smem_sub = svd_subspace_smem(F, nc);
    if (smem_sub > 200 * 1024)
        return set_error(h, RCA_ERR_UNSUPPORTED, "frames x (rank + 1) = %d x %d exceeds the subspace kernel", F, nc + 1);
    const int ntile = (F + SV_T - 1) / SV_T, npair = ntile * (ntile + 1) / 2;
    // pixel splits: about 8 CTAs per SM in total
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int nsplit = std::max(1, std::min((P + SV_PC - 1) / SV_PC, (8 * sms + npair * nt - 1) / (npair * nt)));
    const int psplit = ((P + nsplit - 1) / nsplit + SV_PC - 1) / SV_PC * SV_PC;
    nsplit = (P + psplit - 1) / psplit;
    auto up = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t n_part = (size_t)nt * nsplit * F * F, n_C = (size_t)nt * F * F, n_Q = (size_t)nt * F * nc;
    const size_t bytes = up(n_part * 8) + up(n_C * 8) + 2 * up(n_Q * 8);
    rca_status st = RCA_OK;
    char* ws = (char*)ws_get(h, WS_SVD, bytes, &st);
    if (!ws) return st;
    float2* part = reinterpret_cast<float2*>(ws);
    float2* C = reinterpret_cast<float2*>(ws + up(n_part * 8));
    float2* Q = reinterpret_cast<float2*>((char*)C + up(n_C * 8));
    float2* Y = reinterpret_cast<float2*>((char*)Q + up(n_Q * 8));
    k_svd_cov<<<dim3(npair, nt, nsplit), 128, 0, h->stream>>>(slices, F, nt, P, ntile, psplit, part);
    k_svd_covsum<<<dim3((unsigned)std::min<size_t>(((size_t)F * F + 255) / 256, 1024), nt), 256, 0, h->stream>>>(
        part, F, nsplit, C);
    cudaError_t e = cudaFuncSetAttribute(k_svd_orth, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_sub);
    if (e != cudaSuccess) return cuda_check(h, e, "subspace smem attribute");
    const size_t smem_q = (size_t)F * nc * sizeof(float2);
    e = cudaFuncSetAttribute(k_svd_cq, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_q);
    if (e != cudaSuccess) return cuda_check(h, e, "subspace product smem attribute");
    const int rows_cq = SV_THREADS / nc;
    k_svd_orth<<<nt, SV_THREADS, smem_sub, h->stream>>>(Y, Q, F, nc, 1);
    for (int it = 0; it < iters; ++it) {
        k_svd_cq<<<dim3((F + rows_cq - 1) / rows_cq, nt), SV_THREADS, smem_q, h->stream>>>(C, Q, F, nc, Y);
        k_svd_orth<<<nt, SV_THREADS, smem_sub, h->stream>>>(Y, Q, F, nc, 0);
    }
    const size_t smem_proj = (size_t)F * nc * sizeof(float2);
    e = cudaFuncSetAttribute(k_svd_project, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_proj);
    if (e != cudaSuccess) return cuda_check(h, e, "projection smem attribute");
    k_svd_project<<<dim3((P + 127) / 128, nt), 128, smem_proj, h->stream>>>(slices, F, nt, P, nc, Q);
    return cuda_check(h, cudaGetLastError(), "clutter filter kernels");
}
