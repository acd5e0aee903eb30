// Microbubble separation on the projection planes (Sec. II-A5): each plane
// pixel's slow-time signal over the F frames is Fourier transformed, split by
// rectangular masks into 2 nb speed / direction subsets and transformed back.
//
// k_separate<MX, OUT> is persistent.  A CTA loops over groups of SP_TL
// consecutive lateral pixels of one plane row; the group's 2 SP_TL slow-time
// signals (RC and CR family of each pixel, interleaved: signal 2 l + fam) sit
// in shared memory as [F][SP_G] complex.  Transforms are mixed-radix Stockham
// passes (self-sorting, ping-pong between two buffers) whose radices (2, 3,
// 4, 5 and products of two of them up to 20) are evaluated in registers:
//   forward transform, spectrum kept in registers (MX values per thread);
//   per subset: the masked spectrum, scaled by 1/F, is written back and
//   transformed inversely; then either the complex subset is stored
//   (SP_OUT_COMPLEX) or its XDoppler / coherent amplitude and per-frame maxima
//   (SP_OUT_ENHANCE), which is what a subset's localisation reads.
// Shared-memory traffic per subset and group: one write of the masked
// spectrum, two accesses per element per pass, one read for the output.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>

#include "rca_internal.cuh"

namespace {

#define SP_TL 8                 // lateral pixels per group
#define SP_G (2 * SP_TL)        // signals per group
#define SP_THREADS 256
#define SP_MAXP 10              // passes
#define SP_MAXF 512
#define SP_OUT_COMPLEX 0
#define SP_OUT_ENHANCE 1

struct SepConst {
    int F, npass, nsub, enh;
    int radix[SP_MAXP];
    float s3, c51, c52, s51, s52;   // sin(2pi/3); cos, sin of 2pi/5 and 4pi/5
    signed char bin[SP_MAXF];       // subset of DFT bin j, -1 none
};

struct Codelet {
    float s3, c51, c52, s51, s52;
};

__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 f2sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 f2scale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 f2fma(float2 a, float s, float2 b) { return make_float2(fmaf(a.x, s, b.x), fmaf(a.y, s, b.y)); }
__device__ __forceinline__ float2 f2mul(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// -i v (forward) / +i v (inverse)
template <bool INV>
__device__ __forceinline__ float2 rot(float2 v) { return INV ? make_float2(-v.y, v.x) : make_float2(v.y, -v.x); }
// twiddle exp(-+ 2 pi i m / F) from the forward table
template <bool INV>
__device__ __forceinline__ float2 twid(const float2* tw, int m)
{
    const float2 w = tw[m];
    return INV ? make_float2(w.x, -w.y) : w;
}

// R-point DFT in registers, y_k = sum_n x_n exp(-+2 pi i n k / R)
template <int R, bool INV> struct Dft;

template <bool INV> struct Dft<2, INV> {
    static __device__ __forceinline__ void run(float2 (&v)[2], const Codelet&, const float2*, int)
    {
        const float2 a = v[0];
        v[0] = f2add(a, v[1]);
        v[1] = f2sub(a, v[1]);
    }
};

template <bool INV> struct Dft<3, INV> {
    static __device__ __forceinline__ void run(float2 (&v)[3], const Codelet& c, const float2*, int)
    {
        const float2 t = f2add(v[1], v[2]);
        const float2 m = f2fma(t, -0.5f, v[0]);
        const float2 r = f2scale(rot<INV>(f2sub(v[1], v[2])), c.s3);
        v[0] = f2add(v[0], t);
        v[1] = f2add(m, r);
        v[2] = f2sub(m, r);
    }
};

template <bool INV> struct Dft<4, INV> {
    static __device__ __forceinline__ void run(float2 (&v)[4], const Codelet&, const float2*, int)
    {
        const float2 t0 = f2add(v[0], v[2]), t1 = f2sub(v[0], v[2]);
        const float2 t2 = f2add(v[1], v[3]), t3 = rot<INV>(f2sub(v[1], v[3]));
        v[0] = f2add(t0, t2);
        v[2] = f2sub(t0, t2);
        v[1] = f2add(t1, t3);
        v[3] = f2sub(t1, t3);
    }
};

template <bool INV> struct Dft<5, INV> {
    static __device__ __forceinline__ void run(float2 (&v)[5], const Codelet& c, const float2*, int)
    {
        const float2 a1 = f2add(v[1], v[4]), b1 = f2sub(v[1], v[4]);
        const float2 a2 = f2add(v[2], v[3]), b2 = f2sub(v[2], v[3]);
        const float2 m1 = f2fma(a2, c.c52, f2fma(a1, c.c51, v[0]));
        const float2 m2 = f2fma(a2, c.c51, f2fma(a1, c.c52, v[0]));
        const float2 r1 = rot<INV>(f2fma(b2, c.s52, f2scale(b1, c.s51)));
        const float2 r2 = rot<INV>(f2fma(b2, -c.s51, f2scale(b1, c.s52)));
        v[0] = f2add(v[0], f2add(a1, a2));
        v[1] = f2add(m1, r1);
        v[4] = f2sub(m1, r1);
        v[2] = f2add(m2, r2);
        v[3] = f2sub(m2, r2);
    }
};

// R = R1 R2 by one Cooley-Tukey split in registers: n = R2 n1 + n2,
// k = k1 + R1 k2; inner twiddles W_R^(n2 k1) = tw[n2 k1 F / R] (twr = F / R).
template <int R1, int R2, bool INV> struct DftC {
    static __device__ __forceinline__ void run(float2 (&v)[R1 * R2], const Codelet& c, const float2* tw, int twr)
    {
#pragma unroll
        for (int n2 = 0; n2 < R2; ++n2) {
            float2 a[R1];
#pragma unroll
            for (int n1 = 0; n1 < R1; ++n1) a[n1] = v[R2 * n1 + n2];
            Dft<R1, INV>::run(a, c, tw, twr);
#pragma unroll
            for (int k1 = 0; k1 < R1; ++k1)
                v[R2 * k1 + n2] = (n2 * k1 == 0) ? a[k1] : f2mul(a[k1], twid<INV>(tw, n2 * k1 * twr));
        }
        float2 o[R1 * R2];
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) {
            float2 b[R2];
#pragma unroll
            for (int n2 = 0; n2 < R2; ++n2) b[n2] = v[R2 * k1 + n2];
            Dft<R2, INV>::run(b, c, tw, twr);
#pragma unroll
            for (int k2 = 0; k2 < R2; ++k2) o[k1 + R1 * k2] = b[k2];
        }
#pragma unroll
        for (int k = 0; k < R1 * R2; ++k) v[k] = o[k];
    }
};

template <int R, bool INV> struct Radix { using T = Dft<R, INV>; };
template <bool INV> struct Radix<6, INV> { using T = DftC<2, 3, INV>; };
template <bool INV> struct Radix<8, INV> { using T = DftC<2, 4, INV>; };
template <bool INV> struct Radix<10, INV> { using T = DftC<2, 5, INV>; };
template <bool INV> struct Radix<12, INV> { using T = DftC<4, 3, INV>; };
template <bool INV> struct Radix<15, INV> { using T = DftC<3, 5, INV>; };
template <bool INV> struct Radix<16, INV> { using T = DftC<4, 4, INV>; };
template <bool INV> struct Radix<20, INV> { using T = DftC<4, 5, INV>; };

// One Stockham pass of radix R over the SP_G signals: after the passes with
// radices before this one (product Ns), butterfly idx (k = idx mod Ns) takes
// in[idx + r F / R], twiddles them by W_F^(k r F / (Ns R)), transforms and
// stores output u at (idx - k) R + k + u Ns.
template <int R, bool INV>
__device__ __noinline__ void sp_pass(const float2* __restrict__ in, float2* __restrict__ out, int F, int Ns,
                                     const float2* __restrict__ tw, Codelet c)
{
    const int nb = F / R, step = F / (Ns * R), twr = F / R;
    for (int it = threadIdx.x; it < nb * SP_G; it += SP_THREADS) {
        const int g = it & (SP_G - 1), idx = it / SP_G;
        const int k = idx % Ns;
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = in[(idx + r * nb) * SP_G + g];
        if (k != 0) {
#pragma unroll
            for (int r = 1; r < R; ++r) v[r] = f2mul(v[r], twid<INV>(tw, k * r * step));
        }
        Radix<R, INV>::T::run(v, c, tw, twr);
        const int o = (idx - k) * R + k;
#pragma unroll
        for (int u = 0; u < R; ++u) out[(o + u * Ns) * SP_G + g] = v[u];
    }
}

// all passes; returns the buffer that holds the result
template <bool INV>
__device__ float2* sp_fft(float2* a, float2* b, const SepConst& sc, const float2* tw, Codelet c)
{
    int Ns = 1;
    for (int p = 0; p < sc.npass; ++p) {
        const int R = sc.radix[p], F = sc.F;
        switch (R) {
            case 2: sp_pass<2, INV>(a, b, F, Ns, tw, c); break;
            case 3: sp_pass<3, INV>(a, b, F, Ns, tw, c); break;
            case 4: sp_pass<4, INV>(a, b, F, Ns, tw, c); break;
            case 5: sp_pass<5, INV>(a, b, F, Ns, tw, c); break;
            case 6: sp_pass<6, INV>(a, b, F, Ns, tw, c); break;
            case 8: sp_pass<8, INV>(a, b, F, Ns, tw, c); break;
            case 10: sp_pass<10, INV>(a, b, F, Ns, tw, c); break;
            case 12: sp_pass<12, INV>(a, b, F, Ns, tw, c); break;
            case 15: sp_pass<15, INV>(a, b, F, Ns, tw, c); break;
            case 16: sp_pass<16, INV>(a, b, F, Ns, tw, c); break;
            default: sp_pass<20, INV>(a, b, F, Ns, tw, c); break;
        }
        __syncthreads();
        float2* t = a;
        a = b;
        b = t;
        Ns *= R;
    }
    return a;
}

// planes [F][2][2][S][nz][N] -> OUT_COMPLEX: sub [nsub][F][2][2][S][nz][N] C32;
// OUT_ENHANCE: A [nsub][F][2][S][nz][N], M [nsub][F] (float bits, >= 0)
template <int MX, int OUT>
__global__ void __launch_bounds__(SP_THREADS, MX <= 20 ? 2 : 1)
    k_separate(const void* __restrict__ planes, int pt, const __grid_constant__ SepConst sc, int S, int nz, int N,
               float2* __restrict__ sub, float* __restrict__ A, unsigned* __restrict__ M)
{
    extern __shared__ __align__(16) float2 smem[];
    const int F = sc.F, nsub = sc.nsub;
    float2* B0 = smem;
    float2* B1 = B0 + (size_t)F * SP_G;
    float2* tw = B1 + (size_t)F * SP_G;
    unsigned* mx = reinterpret_cast<unsigned*>(tw + F);                       // [nsub][F] (OUT_ENHANCE)
    signed char* sbin = reinterpret_cast<signed char*>(mx + (OUT == SP_OUT_ENHANCE ? nsub * F : 0));
    const Codelet c{sc.s3, sc.c51, sc.c52, sc.s51, sc.s52};

    for (int m = threadIdx.x; m < F; m += SP_THREADS) {
        double s, co;
        sincospi(-2.0 * (double)m / (double)F, &s, &co);
        tw[m] = make_float2((float)co, (float)s);
        sbin[m] = sc.bin[m];
    }
    if (OUT == SP_OUT_ENHANCE)
        for (int i = threadIdx.x; i < nsub * F; i += SP_THREADS) mx[i] = 0u;
    __syncthreads();

    const int ngl = (N + SP_TL - 1) / SP_TL;
    const size_t rows_axis = (size_t)S * nz, per_axis = rows_axis * N;
    const long long ngroups = 2LL * (long long)rows_axis * ngl;
    const int n_el = F * SP_G;
    const float invF = 1.0f / (float)F;

    for (long long grp = blockIdx.x; grp < ngroups; grp += gridDim.x) {
        const int lg = (int)(grp % ngl);
        const long long row = grp / ngl;
        const int axis = (int)(row / (long long)rows_axis);
        const int lat0 = lg * SP_TL;
        const size_t rest0 = (size_t)(row % (long long)rows_axis) * N + lat0;

        // slow-time signals of the group: element t * SP_G + 2 l + fam
#pragma unroll 4
        for (int i = threadIdx.x; i < n_el; i += SP_THREADS) {
            const int t = i / SP_G, gg = i & (SP_G - 1), l = gg >> 1, fam = gg & 1;
            float2 v = make_float2(0.f, 0.f);
            if (lat0 + l < N) v = load_c(planes, (((size_t)t * 2 + axis) * 2 + fam) * per_axis + rest0 + l, pt);
            B0[i] = v;
        }
        __syncthreads();
        const float2* X = sp_fft<false>(B0, B1, sc, tw, c);
        float2 xr[MX];
#pragma unroll
        for (int m = 0; m < MX; ++m) {
            const int e = threadIdx.x + m * SP_THREADS;
            xr[m] = e < n_el ? X[e] : make_float2(0.f, 0.f);
        }
        __syncthreads();

        for (int s = 0; s < nsub; ++s) {
#pragma unroll
            for (int m = 0; m < MX; ++m) {
                const int e = threadIdx.x + m * SP_THREADS;
                if (e < n_el) B0[e] = sbin[e / SP_G] == s ? f2scale(xr[m], invF) : make_float2(0.f, 0.f);
            }
            __syncthreads();
            const float2* Y = sp_fft<true>(B0, B1, sc, tw, c);
            if (OUT == SP_OUT_COMPLEX) {
                float2* dst = sub + (size_t)s * F * 4 * per_axis;
                for (int i = threadIdx.x; i < n_el; i += SP_THREADS) {
                    const int t = i / SP_G, gg = i & (SP_G - 1), l = gg >> 1, fam = gg & 1;
                    if (lat0 + l < N) dst[(((size_t)t * 2 + axis) * 2 + fam) * per_axis + rest0 + l] = Y[i];
                }
            } else {
                // one lateral pixel per lane, a run of `per` frames per group of 8 lanes;
                // (RC, CR) of a pixel are adjacent: one 16-byte load
                const int l = threadIdx.x & (SP_TL - 1), ch = threadIdx.x / SP_TL;
                const int per = (F + SP_THREADS / SP_TL - 1) / (SP_THREADS / SP_TL), tb = ch * per;
                const float4* Y4 = reinterpret_cast<const float4*>(Y);
                auto q = [&](int t) -> float2 {
                    if (t < 0 || t >= F) return make_float2(0.f, 0.f);
                    const float4 v = Y4[t * SP_TL + l];   // (RC re, RC im, CR re, CR im)
                    return make_float2(v.x * v.z + v.y * v.w, v.y * v.z - v.x * v.w);
                };
                float* dstA = A + (size_t)s * F * 2 * per_axis;
                const bool lat_ok = lat0 + l < N;
                float2 qm = make_float2(0.f, 0.f), q0 = make_float2(0.f, 0.f);
                if (sc.enh == ULM_ENH_XDOPPLER) {
                    qm = q(tb - 1);
                    q0 = q(tb);
                }
                for (int i = 0; i < per; ++i) {
                    const int t = tb + i;
                    float a = 0.f;
                    if (sc.enh == ULM_ENH_XDOPPLER) {
                        const float2 qp = q(t + 1);
                        const float re = qm.x + q0.x + qp.x, im = qm.y + q0.y + qp.y;
                        a = sqrtf(sqrtf(re * re + im * im));
                        qm = q0;
                        q0 = qp;
                    } else if (t < F) {
                        const float4 v = Y4[t * SP_TL + l];
                        const float re = v.x + v.z, im = v.y + v.w;
                        a = sqrtf(re * re + im * im);
                    }
                    const bool ok = t < F && lat_ok;
                    if (ok) __stcs(dstA + ((size_t)t * 2 + axis) * per_axis + rest0 + l, a);
                    float mm = ok ? a : 0.f;
                    mm = fmaxf(mm, __shfl_xor_sync(0xffffffffu, mm, 1));
                    mm = fmaxf(mm, __shfl_xor_sync(0xffffffffu, mm, 2));
                    mm = fmaxf(mm, __shfl_xor_sync(0xffffffffu, mm, 4));
                    if (l == 0 && t < F) atomicMax(mx + s * F + t, __float_as_uint(mm));
                }
            }
            __syncthreads();
        }
    }
    if (OUT == SP_OUT_ENHANCE)
        for (int i = threadIdx.x; i < nsub * F; i += SP_THREADS)
            if (mx[i]) atomicMax(M + i, mx[i]);
}

// radix plan: F = product of the passes' radices, largest first from the menu
bool plan_radices(int F, int* radix, int* npass)
{
    static const int menu[] = {20, 16, 15, 12, 10, 8, 6, 5, 4, 3, 2};
    int n = 0, rem = F;
    while (rem > 1) {
        int pick = 0;
        for (int r : menu)
            if (rem % r == 0) {
                pick = r;
                break;
            }
        if (!pick || n == SP_MAXP) return false;
        radix[n++] = pick;
        rem /= pick;
    }
    *npass = n;
    return true;
}

template <int MX, int OUT>
rca_status launch_mx(rca_handle* h, const void* planes, int pt, const SepConst& sc, int S, int nz, int N,
                     float2* sub, float* A, unsigned* M, size_t smem, long long ngroups)
{
    auto kern = k_separate<MX, OUT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_check(h, e, "separation smem attribute");
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, SP_THREADS, smem);
    if (e != cudaSuccess) return cuda_check(h, e, "separation occupancy");
    if (per_sm < 1) return set_error(h, RCA_ERR_UNSUPPORTED, "separation kernel does not fit an SM");
    const long long grid = std::min<long long>(ngroups, (long long)per_sm * sms);
    if (grid > 0) kern<<<(unsigned)grid, SP_THREADS, smem, h->stream>>>(planes, pt, sc, S, nz, N, sub, A, M);
    return cuda_check(h, cudaGetLastError(), "separation kernel");
}

}  // namespace

rca_status launch_separate(rca_handle* h, const rca_tables* t, const void* planes, rca_dtype pt, int F,
                           const ulm_sep_params* prm, int enh, float2* sub, float* A, float* M)
{
    const GeomDev& g = t->gd;
    const int nb = prm->n_bands;
    if (!(prm->prf_hz > 0.0) || nb < 1 || nb > ULM_SEP_MAX_BANDS)
        return set_error(h, RCA_ERR_INVALID_ARG, "separation needs prf_hz > 0 and 1 .. %d bands", ULM_SEP_MAX_BANDS);
    if (!(prm->edges_hz[0] >= 0.0)) return set_error(h, RCA_ERR_INVALID_ARG, "band edges must start at >= 0");
    for (int b = 0; b < nb; ++b)
        if (!(prm->edges_hz[b + 1] > prm->edges_hz[b]))
            return set_error(h, RCA_ERR_INVALID_ARG, "band edges must increase");
    if (A && enh != ULM_ENH_XDOPPLER && enh != ULM_ENH_COHERENT)
        return set_error(h, RCA_ERR_INVALID_ARG, "bad enhancement mode");
    if (F > SP_MAXF) return set_error(h, RCA_ERR_UNSUPPORTED, "separation supports at most %d frames", SP_MAXF);
    SepConst sc;
    std::memset(&sc, 0, sizeof(sc));
    sc.F = F;
    sc.nsub = 2 * nb;
    sc.enh = enh;
    if (!plan_radices(F, sc.radix, &sc.npass))
        return set_error(h, RCA_ERR_UNSUPPORTED, "separation needs a frame count with prime factors 2, 3, 5 (F = %d)", F);
    const double pi = 3.14159265358979323846;
    sc.s3 = (float)std::sin(2.0 * pi / 3.0);
    sc.c51 = (float)std::cos(2.0 * pi / 5.0);
    sc.c52 = (float)std::cos(4.0 * pi / 5.0);
    sc.s51 = (float)std::sin(2.0 * pi / 5.0);
    sc.s52 = (float)std::sin(4.0 * pi / 5.0);
    // bin -> subset: signed index k, |k| prf / F against the edges (upper edge
    // inclusive), k > 0 up (subsets 0 .. nb-1), k < 0 down (nb .. 2 nb - 1);
    // DC and the Nyquist bin in none
    for (int j = 0; j < F; ++j) {
        sc.bin[j] = -1;
        if (j == 0 || 2 * j == F) continue;
        const int k = 2 * j < F ? j : j - F;
        const double f = (double)std::abs(k) * prm->prf_hz / (double)F;
        for (int b = 0; b < nb; ++b)
            if (prm->edges_hz[b] < f && f <= prm->edges_hz[b + 1]) {
                sc.bin[j] = (signed char)((k > 0 ? 0 : 1) * nb + b);
                break;
            }
    }
    const int out = A ? SP_OUT_ENHANCE : SP_OUT_COMPLEX;
    const size_t smem = (size_t)2 * F * SP_G * sizeof(float2) + (size_t)F * sizeof(float2) +
                        (out == SP_OUT_ENHANCE ? (size_t)sc.nsub * F * sizeof(unsigned) : 0) + (size_t)F;
    const long long ngroups = 2LL * g.S * g.nz * ((g.N + SP_TL - 1) / SP_TL);
    unsigned* Mu = reinterpret_cast<unsigned*>(M);
    if (out == SP_OUT_ENHANCE) {
        cudaError_t e = cudaMemsetAsync(M, 0, sizeof(float) * (size_t)sc.nsub * F, h->stream);
        if (e != cudaSuccess) return cuda_check(h, e, "separation maxima");
    }
    const int mx = (F * SP_G + SP_THREADS - 1) / SP_THREADS;
#define SP_LAUNCH(MXV)                                                                                        \
    return out == SP_OUT_ENHANCE                                                                              \
               ? launch_mx<MXV, SP_OUT_ENHANCE>(h, planes, (int)pt, sc, g.S, g.nz, g.N, sub, A, Mu, smem, ngroups) \
               : launch_mx<MXV, SP_OUT_COMPLEX>(h, planes, (int)pt, sc, g.S, g.nz, g.N, sub, A, Mu, smem, ngroups)
    if (mx <= 4) SP_LAUNCH(4);
    if (mx <= 8) SP_LAUNCH(8);
    if (mx <= 12) SP_LAUNCH(12);
    if (mx <= 16) SP_LAUNCH(16);
    if (mx <= 20) SP_LAUNCH(20);
    SP_LAUNCH(32);
#undef SP_LAUNCH
}
