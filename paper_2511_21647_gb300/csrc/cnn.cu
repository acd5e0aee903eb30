// cnn.cu -- learned localiser: a 4-layer 3x3 convolutional network mapping a
// projection plane (XDoppler amplitude / frame maximum) to a microbubble
// heatmap on a 4x finer grid, with BF16 tensor-core forward, input-gradient
// and weight-gradient kernels (FP32 accumulation), MSE loss, Adam on FP32
// master weights.  The paper names learned localisation as future work
// (Sec. IV); the network is the build's reading of that form.
//
//   L1 conv3x3(1 -> 32) + ReLU     FP32 CUDA cores (K = 9)
//   L2 conv3x3(32 -> 32) + ReLU    tcgen05 MMA (BF16, FP32 accumulators in TMEM)
//   L3 conv3x3(32 -> 32) + ReLU    idem
//   L4 conv3x3(32 -> 16)           idem, epilogue = pixel shuffle to 4x
// The input gradients run the same tcgen05 kernel on flipped weights; the
// weight gradients (M = COUT is below the tcgen05 minimum of 64) use
// mma.sync m16n8k16.
//
// Activations NHWC BF16; weights [Cout][9 taps][Cin] (tap = 3 (dy+1) + dx+1).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>
#include <vector>

#include "rca_internal.cuh"

#define CNN_C 32
#define CNN_UP 4
#define CONV_TH 8   // tile rows (one warp each)
#define CONV_TW 16  // tile columns (the 16 rows of one mma A fragment)

namespace {

struct ParamLayout {
    // offsets (floats) into the flat parameter vector
    int w[4], b[4], total;
};

inline ParamLayout param_layout()
{
    ParamLayout p;
    const int cin[4] = {1, CNN_C, CNN_C, CNN_C}, cout[4] = {CNN_C, CNN_C, CNN_C, CNN_UP * CNN_UP};
    int o = 0;
    for (int l = 0; l < 4; ++l) {
        p.w[l] = o;
        o += cout[l] * 9 * cin[l];
        p.b[l] = o;
        o += cout[l];
    }
    p.total = o;
    return p;
}

__device__ __forceinline__ unsigned pack_bf2(float a, float b)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<unsigned*>(&v);
}

__device__ __forceinline__ float2 unpack_bf2(unsigned u)
{
    return make_float2(__uint_as_float(u << 16), __uint_as_float(u & 0xffff0000u));
}

__device__ __forceinline__ void mma_bf16(float c[4], const unsigned a[4], const unsigned b[2])
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// ---------------------------------------------------------------------------
// input: x[b][i][j] = A[b][i][j] / M[b / planes_per_frame]
// ---------------------------------------------------------------------------
__global__ void k_cnn_input(const float* __restrict__ A, const float* __restrict__ M, int ppf, int B, int HW,
                            float* __restrict__ x)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)B * HW) return;
    const int b = (int)(i / HW);
    float s = 1.f;
    if (M) {
        const float m = M[b / ppf];
        s = m > 0.f ? 1.f / m : 0.f;
    }
    x[i] = A[i] * s;
}

// L1 forward (Cin = 1): direct 3x3, FP32, + bias + ReLU -> BF16 NHWC.
__global__ void k_conv1_fwd(const float* __restrict__ x, const float* __restrict__ w1, const float* __restrict__ b1,
                            int B, int H, int W, __nv_bfloat16* __restrict__ y)
{
    __shared__ float sw[CNN_C * 9], sb[CNN_C];
    for (int q = threadIdx.x; q < CNN_C * 9; q += blockDim.x) sw[q] = w1[q];
    for (int q = threadIdx.x; q < CNN_C; q += blockDim.x) sb[q] = b1[q];
    __syncthreads();
    const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= (size_t)B * H * W) return;
    const int b = (int)(p / ((size_t)H * W)), ij = (int)(p % ((size_t)H * W)), i = ij / W, j = ij % W;
    float v[9];
#pragma unroll
    for (int t = 0; t < 9; ++t) {
        const int ii = i + t / 3 - 1, jj = j + t % 3 - 1;
        v[t] = (ii >= 0 && ii < H && jj >= 0 && jj < W) ? x[((size_t)b * H + ii) * W + jj] : 0.f;
    }
    // all CNN_C outputs in registers, written as 16-byte vectors (the pixel's
    // 2 CNN_C bytes in CNN_C / 8 stores instead of CNN_C / 2)
    unsigned pk[CNN_C / 2];
#pragma unroll
    for (int o = 0; o < CNN_C; o += 2) {
        float a0 = sb[o], a1 = sb[o + 1];
#pragma unroll
        for (int t = 0; t < 9; ++t) {
            a0 = fmaf(sw[o * 9 + t], v[t], a0);
            a1 = fmaf(sw[(o + 1) * 9 + t], v[t], a1);
        }
        pk[o / 2] = pack_bf2(fmaxf(a0, 0.f), fmaxf(a1, 0.f));
    }
    uint4* out = reinterpret_cast<uint4*>(y + p * CNN_C);
#pragma unroll
    for (int q = 0; q < CNN_C / 8; ++q) out[q] = make_uint4(pk[4 * q], pk[4 * q + 1], pk[4 * q + 2], pk[4 * q + 3]);
}

// ---------------------------------------------------------------------------
// Epilogue modes of the 3x3 convolution kernels:
//   MODE 0: + bias, ReLU, BF16 NHWC out
//   MODE 1: + bias, pixel shuffle (COUT = 16) to the FP32 4x heatmap
//   MODE 2: no bias, times (mask > 0) of a BF16 NHWC tensor, BF16 out (dgrad)
// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// 3x3 convolution on the 5th-generation tensor cores (tcgen05, TMEM).
// A CTA of 128 threads owns a tile of 8 rows x 16 columns (M = 128 pixels,
// ordered column-major: pixel m = 8 x + y), so that one image column of the
// tile is one 8-row core matrix of the MMA's A operand.  The input tile with
// its one-pixel halo (10 x 18 pixels, CIN channels) sits in shared memory in
// the K-major, no-swizzle core-matrix layout
//   [CIN / 8][18 columns][10 rows][8 channels] (16-byte rows),
// so the A operand of tap (dy, dx) is the same array seen from start offset
// dx x 160 + dy x 16 bytes: a column step is 160 bytes (SBO) and an 8-channel
// step 18 x 160 bytes (LBO).  No im2col copy is made.  The weights of all nine
// taps (B operand, [9][CIN / 8][COUT / 8][8 outputs][8 channels]) are staged
// once per CTA.  One thread issues the 9 x CIN / 16 MMAs (M = 128, N = COUT,
// K = 16, BF16 in, FP32 accumulators in TMEM) and commits them to an
// mbarrier; each warp then reads its 32 pixels' rows of the accumulator with
// tcgen05.ld for the epilogue.
// ---------------------------------------------------------------------------
#define TC_HALO_C 18                        // tile columns + halo
#define TC_HALO_R 10                        // tile rows + halo
#define TC_CM_BYTES (TC_HALO_R * 16)        // one column of the halo tile: 10 rows x 16 bytes

__device__ __forceinline__ uint64_t tc_sdesc(unsigned saddr, unsigned lbo, unsigned sbo)
{
    // shared-memory matrix descriptor: start, leading (K) and stride (M/N) byte
    // offsets in 16-byte units, descriptor version 1, no swizzle
    return (uint64_t)((saddr >> 4) & 0x3fff) | ((uint64_t)((lbo >> 4) & 0x3fff) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3fff) << 32) | (1ull << 46);
}

// instruction descriptor of kind::f16: D FP32, A and B BF16, both K-major
__host__ __device__ constexpr unsigned tc_idesc(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(N >> 3) << 17) | ((unsigned)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(unsigned tmem_d, uint64_t da, uint64_t db, unsigned idesc, int accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(tmem_d), "l"(da), "l"(db), "r"(idesc), "r"(accumulate)
        : "memory");
}

template <int NC>
__device__ __forceinline__ void tc_ld(unsigned taddr, float* v);
template <>
__device__ __forceinline__ void tc_ld<16>(unsigned taddr, float* v)
{
    unsigned r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}
template <>
__device__ __forceinline__ void tc_ld<32>(unsigned taddr, float* v)
{
    tc_ld<16>(taddr, v);
    tc_ld<16>(taddr + 16, v + 16);
}

template <int CIN, int COUT, int MODE>
__global__ void __launch_bounds__(128) k_conv_tc(const __nv_bfloat16* __restrict__ x,
                                                 const __nv_bfloat16* __restrict__ wt,
                                                 const float* __restrict__ bias,
                                                 const __nv_bfloat16* __restrict__ mask, int B, int H, int W,
                                                 void* __restrict__ out, unsigned* __restrict__ status)
{
    static_assert(CIN % 16 == 0 && COUT % 16 == 0 && COUT <= 32, "shapes of the 3x3 layers");
    constexpr int KC = CIN / 8, NG = COUT / 8;
    constexpr int TAPB = KC * NG * 128;                 // bytes of one tap's weights
    constexpr int ABYTES = KC * TC_HALO_C * TC_CM_BYTES;
    constexpr unsigned IDESC = tc_idesc(128, COUT);
    constexpr unsigned TMEM_COLS = 64;                  // two 32-column accumulators
    extern __shared__ __align__(16) unsigned char smtc[];
    unsigned char* sB = smtc;                           // [9][KC][NG][8][8] bf16
    unsigned char* sA = smtc + 9 * TAPB;                // [3][KC][18][10][8] bf16
    __shared__ uint64_t bars[2];
    __shared__ unsigned s_tmem;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // weights: element (o, t, c) of [COUT][9][CIN] -> tap t, core (c / 8, o / 8), row o % 8, column c % 8
    for (int q = threadIdx.x; q < COUT * 9 * KC; q += blockDim.x) {
        const int o = q / (9 * KC), r = q % (9 * KC), t = r / KC, kc = r % KC;
        const uint4 v = reinterpret_cast<const uint4*>(wt)[q];   // 8 channels kc*8 .. of (o, t)
        *reinterpret_cast<uint4*>(sB + t * TAPB + (kc * NG + o / 8) * 128 + (o % 8) * 16) = v;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        mbar_fence_init();
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = s_tmem;
    const unsigned sAa = smem_u32(sA), sBa = smem_u32(sB);
    const int tiles_i = (H + CONV_TH - 1) / CONV_TH, tiles_j = (W + CONV_TW - 1) / CONV_TW;
    const int ntiles = B * tiles_i * tiles_j;
    auto coords = [&](int tile, int& b, int& i0, int& j0) {
        b = tile / (tiles_i * tiles_j);
        const int tij = tile % (tiles_i * tiles_j);
        i0 = (tij / tiles_j) * CONV_TH;
        j0 = (tij % tiles_j) * CONV_TW;
    };
    // halo tile of `tile` into buffer `buf` by 16-byte cp.async copies (zero-filled
    // outside the plane), one commit group per call (empty when tile >= ntiles):
    // 8-channel chunk kc of pixel (row yr, column xg)
    auto load = [&](int tile, int buf) {
        if (tile < ntiles) {
            int b, i0, j0;
            coords(tile, b, i0, j0);
            const unsigned dst = sAa + (unsigned)(buf * ABYTES);
            for (int q = threadIdx.x; q < TC_HALO_R * TC_HALO_C * KC; q += blockDim.x) {
                const int kc = q % KC, p = q / KC, xg = p % TC_HALO_C, yr = p / TC_HALO_C;
                const int ii = i0 - 1 + yr, jj = j0 - 1 + xg;
                const bool in = ii >= 0 && ii < H && jj >= 0 && jj < W;
                const void* src = in ? (const void*)(x + (((size_t)b * H + ii) * W + jj) * CIN + kc * 8) : (const void*)x;
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(
                                 dst + (unsigned)((kc * TC_HALO_C + xg) * TC_CM_BYTES + yr * 16)),
                             "l"(src), "r"(in ? 16u : 0u)
                             : "memory");
            }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    // this thread's copies of every group but the newest are done; then the
    // generic-proxy writes are ordered before the tensor cores read the tile
    auto wait_older = [&]() {
        asm volatile("cp.async.wait_group 1;" ::: "memory");
        fence_proxy_async();
    };
    // the 9 x CIN / 16 MMAs of halo buffer `ab` into accumulator `buf` (one thread)
    auto issue = [&](int ab, int buf) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const unsigned aB = sAa + ab * ABYTES, dcol = tmem + (unsigned)(32 * buf);
#pragma unroll
        for (int t = 0; t < 9; ++t) {
            const int dy = t / 3, dx = t % 3;
#pragma unroll
            for (int kk = 0; kk < CIN / 16; ++kk) {
                const uint64_t da = tc_sdesc(aB + (2 * kk * TC_HALO_C + dx) * TC_CM_BYTES + dy * 16,
                                             TC_HALO_C * TC_CM_BYTES, TC_CM_BYTES);
                const uint64_t db = tc_sdesc(sBa + t * TAPB + 2 * kk * NG * 128, NG * 128, 128);
                tc_mma(dcol, da, db, IDESC, (t | kk) != 0);
            }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(&bars[buf]))
                     : "memory");
    };
    // software pipeline over three halo buffers and two accumulators: the copies
    // of tile k + 2 and the MMAs of tile k + 1 run while tile k's epilogue drains
    unsigned phase = 0;   // bit b: parity of the next completion of bars[b]
    bool ok = true;
    int tile = blockIdx.x;
    load(tile, 0);
    load(tile + gridDim.x, 1);
    if (tile < ntiles) {
        wait_older();
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        if (threadIdx.x == 0) issue(0, 0);
    }
    for (int k = 0; tile < ntiles; ++k, tile += gridDim.x) {
        const int cur = k & 1, nxt = cur ^ 1;
        const int ntile = tile + gridDim.x;
        // buffer (k + 2) mod 3 held tile k - 1, whose MMAs completed before its epilogue
        load(ntile + gridDim.x, (k + 2) % 3);
        wait_older();
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        if (ntile < ntiles && threadIdx.x == 0) issue((k + 1) % 3, nxt);
        // bounded wait for tile k's accumulators
        if (!mbar_wait_bounded(&bars[cur], (phase >> cur) & 1u)) ok = false;
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0) atomicOr(status, ST_TIMEOUT);
            // the MMAs in flight finish (bounded) before the accumulators are freed
            mbar_wait_bounded(&bars[cur], (phase >> cur) & 1u);
            if (ntile < ntiles) mbar_wait_bounded(&bars[nxt], (phase >> nxt) & 1u);
            asm volatile("cp.async.wait_all;" ::: "memory");
            break;
        }
        phase ^= 1u << cur;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        int b, i0, j0;
        coords(tile, b, i0, j0);
        // epilogue: warp w reads TMEM lanes 32 w .. 32 w + 31 = pixels m of the tile
        float v[COUT];
        tc_ld<COUT>(tmem + ((unsigned)(32 * warp) << 16) + (unsigned)(32 * cur), v);
        const int m = 32 * warp + lane;
        const int i = i0 + (m & 7), j = j0 + (m >> 3);
        if (i < H && j < W) {
            const size_t pix = ((size_t)b * H + i) * W + j;
            if (MODE == 0) {
                unsigned pk[COUT / 2];
#pragma unroll
                for (int o = 0; o < COUT; o += 2)
                    pk[o / 2] = pack_bf2(fmaxf(v[o] + bias[o], 0.f), fmaxf(v[o + 1] + bias[o + 1], 0.f));
#pragma unroll
                for (int q = 0; q < COUT / 8; ++q)
                    reinterpret_cast<uint4*>(out)[pix * (COUT / 8) + q] =
                        make_uint4(pk[4 * q], pk[4 * q + 1], pk[4 * q + 2], pk[4 * q + 3]);
            } else if (MODE == 1) {
                // channel c = 4 a + s -> heatmap pixel (4 i + a, 4 j + s)
                float* heat = reinterpret_cast<float*>(out);
                const size_t W4 = (size_t)W * CNN_UP;
#pragma unroll
                for (int a = 0; a < CNN_UP; ++a) {
                    const float4 r4 = make_float4(v[4 * a] + bias[4 * a], v[4 * a + 1] + bias[4 * a + 1],
                                                  v[4 * a + 2] + bias[4 * a + 2], v[4 * a + 3] + bias[4 * a + 3]);
                    __stcs(reinterpret_cast<float4*>(heat + ((size_t)b * H * CNN_UP + (size_t)i * CNN_UP + a) * W4 +
                                                     (size_t)j * CNN_UP),
                           r4);
                }
            } else {
                const unsigned* mk = reinterpret_cast<const unsigned*>(mask) + pix * (COUT / 2);
                unsigned pk[COUT / 2];
#pragma unroll
                for (int o = 0; o < COUT; o += 2) {
                    const float2 mm = unpack_bf2(mk[o / 2]);
                    pk[o / 2] = pack_bf2(mm.x > 0.f ? v[o] : 0.f, mm.y > 0.f ? v[o + 1] : 0.f);
                }
#pragma unroll
                for (int q = 0; q < COUT / 8; ++q)
                    reinterpret_cast<uint4*>(out)[pix * (COUT / 8) + q] =
                        make_uint4(pk[4 * q], pk[4 * q + 1], pk[4 * q + 2], pk[4 * q + 3]);
            }
        }
        // every warp's reads of accumulator `cur` are done before MMAs write it again
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_inval(&bars[0]);
        mbar_inval(&bars[1]);
    }
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

// ---------------------------------------------------------------------------
// Weight gradient on tensor cores: dW[o][t][c] = sum_p dY[p][o] X[p + t][c],
// a GEMM with M = COUT, N = 9 x CIN and the reduction over pixels.  Each CTA
// accumulates its tiles in registers and writes one partial [COUT][9 CIN]
// (plus the bias partial) to scratch; a second kernel adds the partials in a
// fixed order (deterministic).  dY and X are staged transposed (channel-major)
// so that pixel pairs are contiguous for the fragments.
// ---------------------------------------------------------------------------
template <int CIN, int COUT>
__global__ void __launch_bounds__(256) k_wgrad_mma(const __nv_bfloat16* __restrict__ x, const __nv_bfloat16* __restrict__ dy,
                                                   int B, int H, int W, float* __restrict__ part)
{
    constexpr int TP = CONV_TH * CONV_TW;          // 128 pixels per tile
    constexpr int DS = TP + 8;                      // dY^T row stride
    constexpr int HH = CONV_TH + 2, HW2 = CONV_TW + 2;
    constexpr int XS = HH * HW2 + 8;                // X^T row stride (halo'd tile)
    constexpr int MT = COUT / 16;                   // m-tiles
    constexpr int NTT = 9 * CIN / 8;                // n-tiles in total
    constexpr int NPW = (MT * NTT + 7) / 8;         // (m, n) tiles per warp
    extern __shared__ __align__(16) unsigned char smraw[];
    __nv_bfloat16* dYT = reinterpret_cast<__nv_bfloat16*>(smraw);   // [COUT][DS]
    __nv_bfloat16* XT = dYT + COUT * DS;                            // [CIN][XS]
    float* dbs = reinterpret_cast<float*>(XT + CIN * XS);           // [COUT]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, tig = lane & 3;
    float acc[NPW][4];
#pragma unroll
    for (int q = 0; q < NPW; ++q) acc[q][0] = acc[q][1] = acc[q][2] = acc[q][3] = 0.f;
    float dbacc = 0.f;  // thread o < COUT accumulates the bias gradient of channel o
    const int tiles_i = (H + CONV_TH - 1) / CONV_TH, tiles_j = (W + CONV_TW - 1) / CONV_TW;
    const int ntiles = B * tiles_i * tiles_j;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int b = tile / (tiles_i * tiles_j), tij = tile % (tiles_i * tiles_j);
        const int i0 = (tij / tiles_j) * CONV_TH, j0 = (tij % tiles_j) * CONV_TW;
        __syncthreads();
        for (int q = threadIdx.x; q < TP * COUT; q += blockDim.x) {
            const int p = q / COUT, o = q % COUT;
            const int ii = i0 + p / CONV_TW, jj = j0 + p % CONV_TW;
            __nv_bfloat16 v = __float2bfloat16(0.f);
            if (ii < H && jj < W) v = dy[(((size_t)b * H + ii) * W + jj) * COUT + o];
            dYT[o * DS + p] = v;
        }
        for (int q = threadIdx.x; q < HH * HW2 * CIN; q += blockDim.x) {
            const int pix = q / CIN, c = q % CIN;
            const int ii = i0 - 1 + pix / HW2, jj = j0 - 1 + pix % HW2;
            __nv_bfloat16 v = __float2bfloat16(0.f);
            if (ii >= 0 && ii < H && jj >= 0 && jj < W) v = x[(((size_t)b * H + ii) * W + jj) * CIN + c];
            XT[c * XS + pix] = v;
        }
        __syncthreads();
        if (threadIdx.x < COUT) {
            float s = 0.f;
            for (int p = 0; p < TP; ++p) s += __bfloat162float(dYT[threadIdx.x * DS + p]);
            dbacc += s;
        }
        // k-steps: each tile row of 16 pixels
#pragma unroll 1
        for (int rr = 0; rr < CONV_TH; ++rr) {
#pragma unroll
            for (int q = 0; q < NPW; ++q) {
                const int mn = warp + 8 * q;
                if (mn >= MT * NTT) break;
                const int mt = mn % MT, nt = mn / MT;
                unsigned a[4];
                const __nv_bfloat16* ya = dYT + (mt * 16 + g) * DS + rr * CONV_TW + 2 * tig;
                a[0] = *reinterpret_cast<const unsigned*>(ya);
                a[1] = *reinterpret_cast<const unsigned*>(ya + 8 * DS);
                a[2] = *reinterpret_cast<const unsigned*>(ya + 8);
                a[3] = *reinterpret_cast<const unsigned*>(ya + 8 * DS + 8);
                // column n = nt * 8 + g of N = (tap, cin): tap = n / CIN, c = n % CIN
                const int n = nt * 8 + g, tap = n / CIN, c = n % CIN;
                const int dyy = tap / 3, dxx = tap % 3;
                const __nv_bfloat16* xb = XT + c * XS + (rr + dyy) * HW2 + dxx + 2 * tig;
                // B(k, n) for pixels k = 2 tig, 2 tig + 1 (and + 8): two bf16 that may be
                // unaligned in the halo row, so they are gathered as scalars
                unsigned bb[2];
                bb[0] = (unsigned)__bfloat16_as_ushort(xb[0]) | ((unsigned)__bfloat16_as_ushort(xb[1]) << 16);
                bb[1] = (unsigned)__bfloat16_as_ushort(xb[8]) | ((unsigned)__bfloat16_as_ushort(xb[9]) << 16);
                mma_bf16(acc[q], a, bb);
            }
        }
    }
    // partial of this CTA: rows (o) g, g + 8 of m-tile, columns n = nt*8 + 2 tig (+1)
    float* dst = part + (size_t)blockIdx.x * (COUT * 9 * CIN + COUT);
#pragma unroll
    for (int q = 0; q < NPW; ++q) {
        const int mn = warp + 8 * q;
        if (mn >= MT * NTT) break;
        const int mt = mn % MT, nt = mn / MT;
        const int o0 = mt * 16 + g, n0 = nt * 8 + 2 * tig;
        dst[o0 * 9 * CIN + n0] = acc[q][0];
        dst[o0 * 9 * CIN + n0 + 1] = acc[q][1];
        dst[(o0 + 8) * 9 * CIN + n0] = acc[q][2];
        dst[(o0 + 8) * 9 * CIN + n0 + 1] = acc[q][3];
    }
    (void)dbs;
    if (threadIdx.x < COUT) dst[COUT * 9 * CIN + threadIdx.x] = dbacc;
}

// L1 weight gradient (CIN = 1), FP32: per-CTA partials of dW1[o][t], db1[o].
__global__ void k_wgrad1(const float* __restrict__ x, const __nv_bfloat16* __restrict__ dy, int B, int H, int W,
                         float* __restrict__ part)
{
    // thread (o, t) for o < 32, t < 10 (t = 9: bias); CTA strides over pixels
    __shared__ float red[CNN_C * 10];
    const int o = threadIdx.x / 10, t = threadIdx.x % 10;
    float s = 0.f;
    if (threadIdx.x < CNN_C * 10) {
        const size_t np = (size_t)B * H * W;
        for (size_t p = blockIdx.x; p < np; p += gridDim.x) {
            const int b = (int)(p / ((size_t)H * W)), ij = (int)(p % ((size_t)H * W)), i = ij / W, j = ij % W;
            const float d = __bfloat162float(dy[p * CNN_C + o]);
            if (t == 9) {
                s += d;
            } else {
                const int ii = i + t / 3 - 1, jj = j + t % 3 - 1;
                if (ii >= 0 && ii < H && jj >= 0 && jj < W) s = fmaf(d, x[((size_t)b * H + ii) * W + jj], s);
            }
        }
        red[threadIdx.x] = s;
    }
    __syncthreads();
    if (threadIdx.x < CNN_C * 10) {
        float* dst = part + (size_t)blockIdx.x * (CNN_C * 9 + CNN_C);
        if (t < 9) dst[o * 9 + t] = red[threadIdx.x];
        else dst[CNN_C * 9 + o] = red[threadIdx.x];
    }
}

// sum CTA partials in a fixed order: out[k] = sum_c part[c][k]
__global__ void k_reduce_partials(const float* __restrict__ part, int nparts, int len, float* __restrict__ out)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= len) return;
    float s = 0.f;
    for (int c = 0; c < nparts; ++c) s += part[(size_t)c * len + k];
    out[k] = s;
}

// MSE loss: per-CTA partial sums of (heat - target)^2 and dZ4 (un-shuffled
// 2 (heat - target) / n, BF16 NHWC with 16 channels).
__global__ void k_loss(const float* __restrict__ heat, const float* __restrict__ target, int B, int H, int W,
                       __nv_bfloat16* __restrict__ dz, float* __restrict__ part)
{
    __shared__ float red[32];
    const size_t n = (size_t)B * H * W * CNN_UP * CNN_UP;
    const float scale = 2.0f / (float)n;
    float s = 0.f;
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
        const size_t W4 = (size_t)W * CNN_UP;
        const size_t b = q / ((size_t)H * CNN_UP * W4), rem = q % ((size_t)H * CNN_UP * W4);
        const int y = (int)(rem / W4), xq = (int)(rem % W4);
        const float d = heat[q] - target[q];
        s = fmaf(d, d, s);
        const int i = y / CNN_UP, a = y % CNN_UP, j = xq / CNN_UP, c = xq % CNN_UP;
        dz[(((b * H + i) * W + j) * (CNN_UP * CNN_UP)) + a * CNN_UP + c] = __float2bfloat16(d * scale);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        part[blockIdx.x] = t;
    }
}

__global__ void k_loss_final(const float* __restrict__ part, int nparts, float inv_n, float* __restrict__ loss)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        float s = 0.f;
        for (int c = 0; c < nparts; ++c) s += part[c];
        *loss = s * inv_n;
    }
}

// Adam on the FP32 masters (bias-corrected step sizes computed on the host)
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ gr, float* __restrict__ m, float* __restrict__ v,
                       int n, float lr_t, float b1, float b2, float eps_t)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float g = gr[i];
    const float mi = b1 * m[i] + (1.f - b1) * g;
    const float vi = b2 * v[i] + (1.f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr_t * mi / (sqrtf(vi) + eps_t);
}

// BF16 copies of the weights: forward layout [O][9][I] and, for the input
// gradient, the transposed and tap-flipped [I][9][O] (tap 8 - t).
__global__ void k_pack_weights(const float* __restrict__ w, int O, int I, __nv_bfloat16* __restrict__ fwd,
                               __nv_bfloat16* __restrict__ flip)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= O * 9 * I) return;
    const int o = q / (9 * I), t = (q / I) % 9, c = q % I;
    const __nv_bfloat16 v = __float2bfloat16(w[q]);
    fwd[q] = v;
    if (flip) flip[((size_t)c * 9 + (8 - t)) * O + o] = v;
}

// Gaussian targets: target[b][y][x] = sum over the plane's points of
// exp(-((y - z4)^2 + (x - x4)^2) / (2 sigma^2)); pts [n][3] = (plane, z4, x4),
// grouped by plane with offsets off[B + 1].
__global__ void k_target(const float* __restrict__ pts, const int* __restrict__ off, int H4, int W4, float sigma,
                         float* __restrict__ target)
{
    const int b = blockIdx.y;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= H4 * W4) return;
    const int y = q / W4, x = q % W4;
    const float inv = 1.f / (2.f * sigma * sigma);
    float s = 0.f;
    for (int k = off[b]; k < off[b + 1]; ++k) {
        const float dz = (float)y - pts[3 * k + 1], dx = (float)x - pts[3 * k + 2];
        s += __expf(-(dz * dz + dx * dx) * inv);
    }
    target[(size_t)b * H4 * W4 + q] = s;
}

__global__ void k_count_offsets(const float* __restrict__ pts, int n, int B, int* __restrict__ off)
{
    // off[b] = first point with plane >= b (points sorted by plane)
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b > B) return;
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if ((int)pts[3 * mid] < b) lo = mid + 1;
        else hi = mid;
    }
    off[b] = lo;
}

}  // namespace

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct ulm_cnn {
    rca_handle* h = nullptr;
    ulm_cnn_desc desc{};
    ParamLayout lay{};
    float* params = nullptr;   // FP32 masters
    float* grads = nullptr;
    float* m = nullptr;
    float* v = nullptr;
    __nv_bfloat16* wbf[4] = {nullptr, nullptr, nullptr, nullptr};  // forward copies (layers 2..4)
    __nv_bfloat16* wfl[4] = {nullptr, nullptr, nullptr, nullptr};  // flipped copies (layers 2..4)
    long long step = 0;
    // activations for the largest batch
    size_t cap_px = 0;
    float* x0 = nullptr;
    __nv_bfloat16 *a1 = nullptr, *a2 = nullptr, *a3 = nullptr;
    __nv_bfloat16 *g1 = nullptr, *g2 = nullptr, *g3 = nullptr, *gz = nullptr;
    float* heat = nullptr;
    float* part = nullptr;  // scratch for per-CTA partials
    size_t part_len = 0;
    int grid_conv = 0;
    int grid_conv_tc = 0;
};

static rca_status cnn_check_shape(ulm_cnn* c, int B, int H, int W)
{
    if (B <= 0 || H <= 0 || W <= 0) return set_error(c->h, RCA_ERR_SHAPE, "batch and plane sizes must be positive");
    if ((size_t)B * H * W > c->cap_px)
        return set_error(c->h, RCA_ERR_SHAPE, "batch of %d planes %dx%d exceeds the network's capacity (%zu pixels)", B, H, W,
                         c->cap_px);
    return RCA_OK;
}

static rca_status cnn_pack(ulm_cnn* c)
{
    const int cin[4] = {1, CNN_C, CNN_C, CNN_C}, cout[4] = {CNN_C, CNN_C, CNN_C, CNN_UP * CNN_UP};
    for (int l = 1; l < 4; ++l) {
        const int n = cout[l] * 9 * cin[l];
        k_pack_weights<<<(n + 255) / 256, 256, 0, c->h->stream>>>(c->params + c->lay.w[l], cout[l], cin[l], c->wbf[l],
                                                                c->wfl[l]);
    }
    return cuda_check(c->h, cudaGetLastError(), "cnn pack");
}

template <int CIN, int COUT, int MODE>
static rca_status conv_launch(ulm_cnn* c, const __nv_bfloat16* x, const __nv_bfloat16* w, const float* bias,
                              const __nv_bfloat16* mask, int B, int H, int W, void* out)
{
    // weights of the nine taps + three halo tiles
    constexpr size_t smem = (size_t)9 * CIN * COUT * 2 + (size_t)3 * (CIN / 8) * TC_HALO_C * TC_CM_BYTES;
    static_assert(smem <= 100 * 1024, "conv tile exceeds its shared-memory budget");
    auto kern = k_conv_tc<CIN, COUT, MODE>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_check(c->h, e, "conv smem attribute");
    const int ntiles = B * ((H + CONV_TH - 1) / CONV_TH) * ((W + CONV_TW - 1) / CONV_TW);
    const int grid = std::min(ntiles, c->grid_conv_tc);
    kern<<<grid, 128, smem, c->h->stream>>>(x, w, bias, mask, B, H, W, out, c->h->d_status);
    return cuda_check(c->h, cudaGetLastError(), "conv kernel");
}

template <int CIN, int COUT>
static rca_status wgrad_launch(ulm_cnn* c, const __nv_bfloat16* x, const __nv_bfloat16* dy, int B, int H, int W,
                               float* dw)
{
    constexpr int DS = CONV_TH * CONV_TW + 8, XS = (CONV_TH + 2) * (CONV_TW + 2) + 8;
    const size_t smem = ((size_t)COUT * DS + (size_t)CIN * XS) * sizeof(__nv_bfloat16) + COUT * sizeof(float);
    auto kern = k_wgrad_mma<CIN, COUT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_check(c->h, e, "wgrad smem attribute");
    const int ntiles = B * ((H + CONV_TH - 1) / CONV_TH) * ((W + CONV_TW - 1) / CONV_TW);
    const int grid = std::min(ntiles, c->grid_conv);
    const int len = COUT * 9 * CIN + COUT;
    if ((size_t)grid * len > c->part_len) return set_error(c->h, RCA_ERR_CAPACITY, "cnn scratch too small");
    kern<<<grid, 256, smem, c->h->stream>>>(x, dy, B, H, W, c->part);
    k_reduce_partials<<<(len + 255) / 256, 256, 0, c->h->stream>>>(c->part, grid, len, dw);
    return cuda_check(c->h, cudaGetLastError(), "wgrad kernels");
}

static rca_status cnn_forward(ulm_cnn* c, const float* A, const float* M, int ppf, int B, int H, int W)
{
    cudaStream_t s = c->h->stream;
    const size_t np = (size_t)B * H * W;
    k_cnn_input<<<(unsigned)((np + 255) / 256), 256, 0, s>>>(A, M, ppf > 0 ? ppf : 1, B, H * W, c->x0);
    k_conv1_fwd<<<(unsigned)((np + 255) / 256), 256, 0, s>>>(c->x0, c->params + c->lay.w[0], c->params + c->lay.b[0], B,
                                                             H, W, c->a1);
    rca_status st;
    if ((st = conv_launch<CNN_C, CNN_C, 0>(c, c->a1, c->wbf[1], c->params + c->lay.b[1], nullptr, B, H, W, c->a2)) != RCA_OK)
        return st;
    if ((st = conv_launch<CNN_C, CNN_C, 0>(c, c->a2, c->wbf[2], c->params + c->lay.b[2], nullptr, B, H, W, c->a3)) != RCA_OK)
        return st;
    return conv_launch<CNN_C, CNN_UP * CNN_UP, 1>(c, c->a3, c->wbf[3], c->params + c->lay.b[3], nullptr, B, H, W, c->heat);
}

extern "C" rca_status ulm_cnn_create(rca_handle* h, const ulm_cnn_desc* d, ulm_cnn** out)
{
    if (!h) return RCA_ERR_INVALID_ARG;
    if (!d || !out) return set_error(h, RCA_ERR_INVALID_ARG, "null descriptor or output");
    *out = nullptr;
    if (d->channels != CNN_C) return set_error(h, RCA_ERR_UNSUPPORTED, "only %d channels are built", CNN_C);
    if (d->max_pixels <= 0) return set_error(h, RCA_ERR_INVALID_ARG, "max_pixels must be positive");
    ulm_cnn* c = new (std::nothrow) ulm_cnn();
    if (!c) return set_error(h, RCA_ERR_CUDA, "out of host memory");
    c->h = h;
    c->desc = *d;
    c->lay = param_layout();
    c->cap_px = (size_t)d->max_pixels;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    c->grid_conv = 4 * sms;
    c->grid_conv_tc = 4 * sms;   // four CTAs per SM (64 TMEM columns each)
    c->part_len = (size_t)c->grid_conv * (CNN_C * 9 * CNN_C + CNN_C) + 4096;
    const size_t P = c->lay.total, px = c->cap_px;
    bool ok = cudaMalloc(&c->params, P * 4) == cudaSuccess && cudaMalloc(&c->grads, P * 4) == cudaSuccess &&
              cudaMalloc(&c->m, P * 4) == cudaSuccess && cudaMalloc(&c->v, P * 4) == cudaSuccess &&
              cudaMalloc(&c->x0, px * 4) == cudaSuccess && cudaMalloc(&c->a1, px * CNN_C * 2) == cudaSuccess &&
              cudaMalloc(&c->a2, px * CNN_C * 2) == cudaSuccess && cudaMalloc(&c->a3, px * CNN_C * 2) == cudaSuccess &&
              cudaMalloc(&c->g1, px * CNN_C * 2) == cudaSuccess && cudaMalloc(&c->g2, px * CNN_C * 2) == cudaSuccess &&
              cudaMalloc(&c->g3, px * CNN_C * 2) == cudaSuccess &&
              cudaMalloc(&c->gz, px * CNN_UP * CNN_UP * 2) == cudaSuccess &&
              cudaMalloc(&c->heat, px * CNN_UP * CNN_UP * 4) == cudaSuccess &&
              cudaMalloc(&c->part, c->part_len * 4) == cudaSuccess;
    for (int l = 1; l < 4 && ok; ++l) {
        const int n = (l == 3 ? CNN_UP * CNN_UP : CNN_C) * 9 * CNN_C;
        ok = cudaMalloc(&c->wbf[l], n * 2) == cudaSuccess && cudaMalloc(&c->wfl[l], n * 2) == cudaSuccess;
    }
    if (!ok) {
        ulm_cnn_destroy(c);
        return set_error(h, RCA_ERR_CUDA, "cnn allocation failed");
    }
    // He-normal initial weights, zero biases (seeded, host generated)
    std::vector<float> init(P, 0.f);
    std::mt19937_64 rng(d->seed);
    std::normal_distribution<double> nd(0.0, 1.0);
    const int cin[4] = {1, CNN_C, CNN_C, CNN_C}, cout[4] = {CNN_C, CNN_C, CNN_C, CNN_UP * CNN_UP};
    for (int l = 0; l < 4; ++l) {
        const double sd = std::sqrt(2.0 / (9.0 * cin[l]));
        for (int q = 0; q < cout[l] * 9 * cin[l]; ++q) init[c->lay.w[l] + q] = (float)(nd(rng) * sd);
    }
    rca_status st = ulm_cnn_set_params(c, init.data(), P);
    if (st != RCA_OK) {
        ulm_cnn_destroy(c);
        return st;
    }
    *out = c;
    return RCA_OK;
}

extern "C" rca_status ulm_cnn_destroy(ulm_cnn* c)
{
    if (!c) return RCA_ERR_INVALID_ARG;
    cudaStreamSynchronize(c->h->stream);
    void* ptrs[] = {c->params, c->grads, c->m, c->v, c->x0, c->a1, c->a2, c->a3, c->g1, c->g2, c->g3, c->gz, c->heat,
                    c->part, c->wbf[1], c->wbf[2], c->wbf[3], c->wfl[1], c->wfl[2], c->wfl[3]};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete c;
    return RCA_OK;
}

extern "C" rca_status ulm_cnn_param_count(const ulm_cnn* c, size_t* n)
{
    if (!c || !n) return RCA_ERR_INVALID_ARG;
    *n = (size_t)c->lay.total;
    return RCA_OK;
}

extern "C" rca_status ulm_cnn_set_params(ulm_cnn* c, const float* host, size_t n)
{
    if (!c || !host) return RCA_ERR_INVALID_ARG;
    if (n != (size_t)c->lay.total) return set_error(c->h, RCA_ERR_SHAPE, "expected %d parameters", c->lay.total);
    rca_status st = cuda_check(c->h, cudaMemcpy(c->params, host, n * 4, cudaMemcpyHostToDevice), "set params");
    if (st != RCA_OK) return st;
    cudaMemset(c->m, 0, n * 4);
    cudaMemset(c->v, 0, n * 4);
    cudaMemset(c->grads, 0, n * 4);
    c->step = 0;
    return cnn_pack(c);
}

extern "C" rca_status ulm_cnn_get_params(const ulm_cnn* c, float* host, size_t n)
{
    if (!c || !host) return RCA_ERR_INVALID_ARG;
    if (n != (size_t)c->lay.total) return set_error(c->h, RCA_ERR_SHAPE, "expected %d parameters", c->lay.total);
    cudaStreamSynchronize(c->h->stream);
    return cuda_check(c->h, cudaMemcpy(host, c->params, n * 4, cudaMemcpyDeviceToHost), "get params");
}

extern "C" rca_status ulm_cnn_get_grads(const ulm_cnn* c, float* host, size_t n)
{
    if (!c || !host) return RCA_ERR_INVALID_ARG;
    if (n != (size_t)c->lay.total) return set_error(c->h, RCA_ERR_SHAPE, "expected %d parameters", c->lay.total);
    cudaStreamSynchronize(c->h->stream);
    return cuda_check(c->h, cudaMemcpy(host, c->grads, n * 4, cudaMemcpyDeviceToHost), "get grads");
}

extern "C" rca_status ulm_cnn_forward(ulm_cnn* c, const float* A, const float* M, int ppf, int B, int H, int W,
                                      float* heat)
{
    if (!c) return RCA_ERR_INVALID_ARG;
    if (!A || !heat) return set_error(c->h, RCA_ERR_INVALID_ARG, "null input or heatmap");
    rca_status st = cnn_check_shape(c, B, H, W);
    if (st != RCA_OK) return st;
    if ((st = cnn_forward(c, A, M, ppf, B, H, W)) != RCA_OK) return st;
    return cuda_check(c->h,
                      cudaMemcpyAsync(heat, c->heat, (size_t)B * H * W * CNN_UP * CNN_UP * 4, cudaMemcpyDeviceToDevice,
                                      c->h->stream),
                      "heatmap copy");
}

extern "C" rca_status ulm_cnn_infer(ulm_cnn* c, const float* A, const float* M, int ppf, int B, int H, int W,
                                    float* heat)
{
    return ulm_cnn_forward(c, A, M, ppf, B, H, W, heat);
}

extern "C" rca_status ulm_cnn_train_step(ulm_cnn* c, const float* A, const float* M, int ppf, int B, int H, int W,
                                         const float* target, float* loss_dev, int apply_update)
{
    if (!c) return RCA_ERR_INVALID_ARG;
    if (!A || !target || !loss_dev) return set_error(c->h, RCA_ERR_INVALID_ARG, "null input, target or loss");
    rca_status st = cnn_check_shape(c, B, H, W);
    if (st != RCA_OK) return st;
    cudaStream_t s = c->h->stream;
    if ((st = cnn_forward(c, A, M, ppf, B, H, W)) != RCA_OK) return st;
    const size_t n = (size_t)B * H * W * CNN_UP * CNN_UP;
    const int lgrid = (int)std::min<size_t>((n + 255) / 256, 1024);
    k_loss<<<lgrid, 256, 0, s>>>(c->heat, target, B, H, W, c->gz, c->part);
    k_loss_final<<<1, 32, 0, s>>>(c->part, lgrid, 1.0f / (float)n, loss_dev);
    const ParamLayout& L = c->lay;
    // layer 4: dW4 from (a3, dz); dgrad -> g3 masked by a3 > 0
    if ((st = wgrad_launch<CNN_C, CNN_UP * CNN_UP>(c, c->a3, c->gz, B, H, W, c->grads + L.w[3])) != RCA_OK) return st;
    if ((st = conv_launch<CNN_UP * CNN_UP, CNN_C, 2>(c, c->gz, c->wfl[3], nullptr, c->a3, B, H, W, c->g3)) != RCA_OK) return st;
    // layer 3
    if ((st = wgrad_launch<CNN_C, CNN_C>(c, c->a2, c->g3, B, H, W, c->grads + L.w[2])) != RCA_OK) return st;
    if ((st = conv_launch<CNN_C, CNN_C, 2>(c, c->g3, c->wfl[2], nullptr, c->a2, B, H, W, c->g2)) != RCA_OK) return st;
    // layer 2
    if ((st = wgrad_launch<CNN_C, CNN_C>(c, c->a1, c->g2, B, H, W, c->grads + L.w[1])) != RCA_OK) return st;
    if ((st = conv_launch<CNN_C, CNN_C, 2>(c, c->g2, c->wfl[1], nullptr, c->a1, B, H, W, c->g1)) != RCA_OK) return st;
    // layer 1 (FP32)
    const int g1grid = std::min(c->grid_conv, (int)std::max<size_t>(1, (size_t)B * H * W / 64));
    k_wgrad1<<<g1grid, 320, 0, s>>>(c->x0, c->g1, B, H, W, c->part);
    k_reduce_partials<<<(CNN_C * 10 + 255) / 256, 256, 0, s>>>(c->part, g1grid, CNN_C * 10, c->grads + L.w[0]);
    if ((st = cuda_check(c->h, cudaGetLastError(), "backward kernels")) != RCA_OK) return st;
    if (!apply_update) return RCA_OK;
    c->step += 1;
    const double b1 = c->desc.beta1, b2 = c->desc.beta2;
    const double bc1 = 1.0 - std::pow(b1, (double)c->step), bc2 = 1.0 - std::pow(b2, (double)c->step);
    // p -= lr * (m / bc1) / (sqrt(v / bc2) + eps)  ==  lr_t * m / (sqrt(v) + eps_t)
    const float lr_t = (float)(c->desc.lr * std::sqrt(bc2) / bc1);
    const float eps_t = (float)(c->desc.eps * std::sqrt(bc2));
    k_adam<<<(L.total + 255) / 256, 256, 0, s>>>(c->params, c->grads, c->m, c->v, L.total, lr_t, (float)b1, (float)b2,
                                                eps_t);
    if ((st = cuda_check(c->h, cudaGetLastError(), "adam")) != RCA_OK) return st;
    return cnn_pack(c);
}

extern "C" rca_status ulm_cnn_target(rca_handle* h, const float* pts, int n, int B, int H4, int W4, float sigma,
                                     float* target)
{
    if (!h) return RCA_ERR_INVALID_ARG;
    if (!target || (n > 0 && !pts) || n < 0 || B <= 0 || H4 <= 0 || W4 <= 0 || !(sigma > 0))
        return set_error(h, RCA_ERR_INVALID_ARG, "bad target arguments");
    rca_status st = RCA_OK;
    int* off = (int*)ws_get(h, WS_MISC, (size_t)(B + 1) * sizeof(int), &st);
    if (!off) return st;
    k_count_offsets<<<(B + 1 + 255) / 256, 256, 0, h->stream>>>(pts, n, B, off);
    dim3 grid((H4 * W4 + 255) / 256, B);
    k_target<<<grid, 256, 0, h->stream>>>(pts, off, H4, W4, sigma, target);
    return cuda_check(h, cudaGetLastError(), "target kernels");
}

extern "C" rca_status ulm_cnn_save(const ulm_cnn* c, const char* path)
{
    if (!c || !path) return RCA_ERR_INVALID_ARG;
    const size_t P = c->lay.total;
    std::vector<float> buf(4 * P);
    cudaStreamSynchronize(c->h->stream);
    cudaMemcpy(buf.data(), c->params, P * 4, cudaMemcpyDeviceToHost);
    cudaMemcpy(buf.data() + P, c->m, P * 4, cudaMemcpyDeviceToHost);
    cudaMemcpy(buf.data() + 2 * P, c->v, P * 4, cudaMemcpyDeviceToHost);
    FILE* f = fopen(path, "wb");
    if (!f) return set_error(c->h, RCA_ERR_INVALID_ARG, "cannot open %s", path);
    const char magic[8] = {'U', 'L', 'M', 'C', 'N', 'N', '1', 0};
    long long hdr[3] = {(long long)P, c->step, CNN_C};
    bool ok = fwrite(magic, 1, 8, f) == 8 && fwrite(hdr, sizeof hdr, 1, f) == 1 && fwrite(buf.data(), 4, 3 * P, f) == 3 * P;
    fclose(f);
    return ok ? RCA_OK : set_error(c->h, RCA_ERR_INVALID_ARG, "write failed: %s", path);
}

extern "C" rca_status ulm_cnn_load(ulm_cnn* c, const char* path)
{
    if (!c || !path) return RCA_ERR_INVALID_ARG;
    const size_t P = c->lay.total;
    FILE* f = fopen(path, "rb");
    if (!f) return set_error(c->h, RCA_ERR_INVALID_ARG, "cannot open %s", path);
    char magic[8];
    long long hdr[3];
    std::vector<float> buf(3 * P);
    bool ok = fread(magic, 1, 8, f) == 8 && memcmp(magic, "ULMCNN1", 7) == 0 && fread(hdr, sizeof hdr, 1, f) == 1 &&
              hdr[0] == (long long)P && hdr[2] == CNN_C && fread(buf.data(), 4, 3 * P, f) == 3 * P;
    fclose(f);
    if (!ok) return set_error(c->h, RCA_ERR_SHAPE, "%s is not a checkpoint of this network", path);
    cudaMemcpy(c->params, buf.data(), P * 4, cudaMemcpyHostToDevice);
    cudaMemcpy(c->m, buf.data() + P, P * 4, cudaMemcpyHostToDevice);
    cudaMemcpy(c->v, buf.data() + 2 * P, P * 4, cudaMemcpyHostToDevice);
    c->step = hdr[1];
    return cnn_pack(c);
}
