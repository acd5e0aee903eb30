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
//   (SP_OUT_COMPLEX) or its XDoppler (SP_OUT_XDOPPLER) or coherent
//   (SP_OUT_COHERENT) amplitude and per-frame maxima, which is what a
//   subset's localisation reads.
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
#define SP_WR 87                // W_R^m tables of the composite radices 6, 8, 10, 12, 15, 16, 20
#define SP_OUT_COMPLEX 0
#define SP_OUT_XDOPPLER 1
#define SP_OUT_COHERENT 2

struct SepConst {
    int F, npass, nsub, enh;
    int radix[SP_MAXP];
    int twoff[SP_MAXP];             // pass p's twiddle table in shared memory (float2 offset)
    int ntw;                        // entries of all pass tables
    float s3, c51, c52, s51, s52;   // sin(2pi/3); cos, sin of 2pi/5 and 4pi/5
    float2 wr[SP_WR];               // exp(-2 pi i m / R) of each composite radix R, m < R
    signed char bin[SP_MAXF];       // subset of DFT bin j, -1 none
};

// offset of radix R's table in SepConst::wr
__host__ __device__ constexpr int wr_off(int R)
{
    return R == 6 ? 0 : R == 8 ? 6 : R == 10 ? 14 : R == 12 ? 24 : R == 15 ? 36 : R == 16 ? 51 : R == 20 ? 67 : -1;
}

__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 f2sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 f2scale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 f2fma(float2 a, float s, float2 b) { return make_float2(fmaf(a.x, s, b.x), fmaf(a.y, s, b.y)); }
// a w (forward) or a conj(w) (inverse)
template <bool INV>
__device__ __forceinline__ float2 twmul(float2 a, float2 w)
{
    return INV ? make_float2(fmaf(a.x, w.x, a.y * w.y), fmaf(a.y, w.x, -a.x * w.y))
               : make_float2(fmaf(a.x, w.x, -a.y * w.y), fmaf(a.x, w.y, a.y * w.x));
}
// sqrt.approx (relative error about 2^-23; 0 -> 0)
__device__ __forceinline__ float sqrt_approx(float x)
{
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
// -i v (forward) / +i v (inverse)
template <bool INV>
__device__ __forceinline__ float2 rot(float2 v) { return INV ? make_float2(-v.y, v.x) : make_float2(v.y, -v.x); }

// R-point DFT in registers, y_k = sum_n x_n exp(-+2 pi i n k / R)
template <int R, bool INV> struct Dft;

template <bool INV> struct Dft<2, INV> {
    static __device__ __forceinline__ void run(float2 (&v)[2], const SepConst&)
    {
        const float2 a = v[0];
        v[0] = f2add(a, v[1]);
        v[1] = f2sub(a, v[1]);
    }
};

template <bool INV> struct Dft<3, INV> {
    static __device__ __forceinline__ void run(float2 (&v)[3], const SepConst& c)
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
    static __device__ __forceinline__ void run(float2 (&v)[4], const SepConst&)
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
    static __device__ __forceinline__ void run(float2 (&v)[5], const SepConst& c)
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
// k = k1 + R1 k2; the inner twiddles W_R^(n2 k1) are kernel-parameter
// constants at compile-time offsets.
template <int R1, int R2, bool INV> struct DftC {
    static __device__ __forceinline__ void run(float2 (&v)[R1 * R2], const SepConst& c)
    {
        constexpr int W0 = wr_off(R1 * R2);
#pragma unroll
        for (int n2 = 0; n2 < R2; ++n2) {
            float2 a[R1];
#pragma unroll
            for (int n1 = 0; n1 < R1; ++n1) a[n1] = v[R2 * n1 + n2];
            Dft<R1, INV>::run(a, c);
#pragma unroll
            for (int k1 = 0; k1 < R1; ++k1)
                v[R2 * k1 + n2] = (n2 * k1 == 0) ? a[k1] : twmul<INV>(a[k1], c.wr[W0 + n2 * k1]);
        }
        float2 o[R1 * R2];
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) {
            float2 b[R2];
#pragma unroll
            for (int n2 = 0; n2 < R2; ++n2) b[n2] = v[R2 * k1 + n2];
            Dft<R2, INV>::run(b, c);
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

// twiddle-table row pitch of a radix-R pass (R - 1 entries, even for 16-byte pairs)
__host__ __device__ constexpr int tw_pitch(int R) { return (R - 1 + 1) & ~1; }

// One Stockham pass of radix R over the SP_G signals: after the passes with
// radices before this one (product Ns), butterfly idx (k = idx mod Ns) takes
// in[idx + r F / R], twiddles them by W_F^(k r F / (Ns R)) = T[k pitch + r - 1],
// transforms and stores output u at (idx - k) R + k + u Ns.  FT / NS: the
// frame count and Ns at compile time (0: the run-time values).
template <int R, bool INV, int FT, int NS>
__device__ __forceinline__ void sp_pass(const float2* __restrict__ in, float2* __restrict__ out, int Frt, int Nsrt,
                                        const float2* __restrict__ T, const SepConst& c)
{
    const int F = FT ? FT : Frt, Ns = NS ? NS : Nsrt;
    constexpr int P = tw_pitch(R);
    const int nb = F / R;
    for (int it = threadIdx.x; it < nb * SP_G; it += SP_THREADS) {
        const int g = it & (SP_G - 1), idx = it / SP_G;
        const int k = NS == 1 ? 0 : idx % Ns;
        const float2* src = in + idx * SP_G + g;
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = src[r * nb * SP_G];
        if (NS != 1 && k != 0) {
            const float4* t4 = reinterpret_cast<const float4*>(T + k * P);
#pragma unroll
            for (int r = 1; r < R; r += 2) {
                const float4 w = t4[(r - 1) / 2];
                v[r] = twmul<INV>(v[r], make_float2(w.x, w.y));
                if (r + 1 < R) v[r + 1] = twmul<INV>(v[r + 1], make_float2(w.z, w.w));
            }
        }
        Radix<R, INV>::T::run(v, c);
        float2* dst = out + ((idx - k) * R + k) * SP_G + g;
#pragma unroll
        for (int u = 0; u < R; ++u) dst[u * Ns * SP_G] = v[u];
    }
}

// all passes; returns the buffer that holds the result.  FT = 300: the plan
// 20 x 15 at compile time; FT = 0: the run-time plan.
template <bool INV, int FT>
__device__ float2* sp_fft(float2* a, float2* b, const SepConst& sc, const float2* tws)
{
    if constexpr (FT == 300) {
        sp_pass<20, INV, 300, 1>(a, b, 0, 0, nullptr, sc);
        __syncthreads();
        sp_pass<15, INV, 300, 20>(b, a, 0, 0, tws + sc.twoff[1], sc);
        __syncthreads();
        return a;
    } else {
        int Ns = 1;
        const int F = sc.F;
        for (int p = 0; p < sc.npass; ++p) {
            const int R = sc.radix[p];
            const float2* T = tws + sc.twoff[p];
            switch (R) {
                case 2: sp_pass<2, INV, 0, 0>(a, b, F, Ns, T, sc); break;
                case 3: sp_pass<3, INV, 0, 0>(a, b, F, Ns, T, sc); break;
                case 4: sp_pass<4, INV, 0, 0>(a, b, F, Ns, T, sc); break;
                case 5: sp_pass<5, INV, 0, 0>(a, b, F, Ns, T, sc); break;
                case 6: sp_pass<6, INV, 0, 0>(a, b, F, Ns, T, sc); break;
                case 8: sp_pass<8, INV, 0, 0>(a, b, F, Ns, T, sc); break;
                case 10: sp_pass<10, INV, 0, 0>(a, b, F, Ns, T, sc); break;
                case 12: sp_pass<12, INV, 0, 0>(a, b, F, Ns, T, sc); break;
                case 15: sp_pass<15, INV, 0, 0>(a, b, F, Ns, T, sc); break;
                case 16: sp_pass<16, INV, 0, 0>(a, b, F, Ns, T, sc); break;
                default: sp_pass<20, INV, 0, 0>(a, b, F, Ns, T, sc); break;
            }
            __syncthreads();
            float2* t = a;
            a = b;
            b = t;
            Ns *= R;
        }
        return a;
    }
}

// planes [F][2][2][S][nz][N] -> OUT_COMPLEX: sub [nsub][F][2][2][S][nz][N] C32;
// OUT_XDOPPLER / OUT_COHERENT: A [nsub][F][2][S][nz][N], M [nsub][F] (float bits, >= 0)
template <int MX, int OUT, int FT>
__global__ void __launch_bounds__(SP_THREADS, MX <= 19 ? 2 : 1)
    k_separate(const void* __restrict__ planes, int pt, const __grid_constant__ SepConst sc, int S, int nz, int N,
               float2* __restrict__ sub, float* __restrict__ A, unsigned* __restrict__ M)
{
    extern __shared__ __align__(16) float2 smem[];
    const int F = FT ? FT : sc.F, nsub = sc.nsub;
    float2* B0 = smem;
    float2* B1 = B0 + (size_t)F * SP_G;
    float2* tws = B1 + (size_t)F * SP_G;                                      // pass twiddle tables
    unsigned* mx = reinterpret_cast<unsigned*>(tws + sc.ntw);                 // [nsub][F] frame maxima (amplitude outputs)
    signed char* sbin = reinterpret_cast<signed char*>(mx + (OUT != SP_OUT_COMPLEX ? nsub * F : 0));

    // pass p (Ns > 1): T_p[k pitch + r - 1] = exp(-2 pi i k r / (Ns R)), double then rounded
    {
        int Ns = 1;
        for (int p = 0; p < sc.npass; ++p) {
            const int R = sc.radix[p], P = tw_pitch(R);
            if (Ns > 1)
                for (int e = threadIdx.x; e < Ns * P; e += SP_THREADS) {
                    const int k = e / P, r = e % P + 1;
                    float2 w = make_float2(0.f, 0.f);
                    if (r < R) {
                        double sn, cs;
                        sincospi(-2.0 * (double)(k * r) / (double)(Ns * R), &sn, &cs);
                        w = make_float2((float)cs, (float)sn);
                    }
                    tws[sc.twoff[p] + e] = w;
                }
            Ns *= R;
        }
    }
    for (int m = threadIdx.x; m < F; m += SP_THREADS) sbin[m] = sc.bin[m];
    if (OUT != SP_OUT_COMPLEX)
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

        // slow-time signals of the group: element t * SP_G + 2 l + fam; all of a
        // thread's loads are issued before its shared-memory stores
        float2 xr[MX];
#pragma unroll
        for (int m = 0; m < MX; ++m) {
            const int i = threadIdx.x + m * SP_THREADS;
            const int t = i / SP_G, gg = i & (SP_G - 1), l = gg >> 1, fam = gg & 1;
            xr[m] = make_float2(0.f, 0.f);
            if (i < n_el && lat0 + l < N)
                xr[m] = load_c(planes, (((size_t)t * 2 + axis) * 2 + fam) * per_axis + rest0 + l, pt);
        }
#pragma unroll
        for (int m = 0; m < MX; ++m) {
            const int i = threadIdx.x + m * SP_THREADS;
            if (i < n_el) B0[i] = xr[m];
        }
        __syncthreads();
        const float2* X = sp_fft<false, FT>(B0, B1, sc, tws);
        // FT = 300: each of the first 240 threads keeps the 20 spectrum values
        // that its butterfly of the first inverse pass (radix 20, Ns = 1, no
        // twiddles) reads, with their subsets (4-bit codes, subset + 1), so the
        // masking and that pass run from registers; otherwise the thread keeps
        // elements threadIdx.x + m SP_THREADS and the masked spectrum is
        // written back for the inverse transform
        constexpr int R0 = 20, NB0 = 15;
        const int g0 = threadIdx.x & (SP_G - 1), idx0 = threadIdx.x / SP_G;
        const bool bf0 = threadIdx.x < NB0 * SP_G;
        float2 xs[FT == 300 ? R0 : 1];
        unsigned long long code_lo = 0ull;
        unsigned code_hi = 0u;
        if constexpr (FT == 300) {
            if (bf0) {
#pragma unroll
                for (int r = 0; r < R0; ++r) {
                    const int j = idx0 + NB0 * r;
                    xs[r] = X[j * SP_G + g0];
                    const unsigned cj = (unsigned)(sbin[j] + 1);
                    if (r < 16)
                        code_lo |= (unsigned long long)cj << (4 * r);
                    else
                        code_hi |= cj << (4 * (r - 16));
                }
            }
        } else {
#pragma unroll
            for (int m = 0; m < MX; ++m) {
                const int e = threadIdx.x + m * SP_THREADS;
                xr[m] = e < n_el ? X[e] : make_float2(0.f, 0.f);
            }
        }
        __syncthreads();

        for (int s = 0; s < nsub; ++s) {
            const float2* Y;
            if constexpr (FT == 300) {
                if (bf0) {
                    float2 v[R0];
#pragma unroll
                    for (int r = 0; r < R0; ++r) {
                        const unsigned cj = r < 16 ? (unsigned)(code_lo >> (4 * r)) & 15u : (code_hi >> (4 * (r - 16))) & 15u;
                        v[r] = cj == (unsigned)(s + 1) ? f2scale(xs[r], invF) : make_float2(0.f, 0.f);
                    }
                    Radix<R0, true>::T::run(v, sc);
                    float2* dst = B1 + idx0 * R0 * SP_G + g0;
#pragma unroll
                    for (int u = 0; u < R0; ++u) dst[u * SP_G] = v[u];
                }
                __syncthreads();
                sp_pass<15, true, 300, 20>(B1, B0, 0, 0, tws + sc.twoff[1], sc);
                __syncthreads();
                Y = B0;
            } else {
#pragma unroll
                for (int m = 0; m < MX; ++m) {
                    const int e = threadIdx.x + m * SP_THREADS;
                    if (e < n_el) B0[e] = sbin[e / SP_G] == s ? f2scale(xr[m], invF) : make_float2(0.f, 0.f);
                }
                __syncthreads();
                Y = sp_fft<true, FT>(B0, B1, sc, tws);
            }
            if (OUT == SP_OUT_COMPLEX) {
                float2* dst = sub + (size_t)s * F * 4 * per_axis;
                for (int i = threadIdx.x; i < n_el; i += SP_THREADS) {
                    const int t = i / SP_G, gg = i & (SP_G - 1), l = gg >> 1, fam = gg & 1;
                    if (lat0 + l < N) dst[(((size_t)t * 2 + axis) * 2 + fam) * per_axis + rest0 + l] = Y[i];
                }
            } else {
                // thread = (frame chunk ch, lateral pair lp): frames [ch per, ch per + per)
                // of lateral pixels la = lp + 4 (ch & 1) and lb = lp + 4 (1 - (ch & 1))
                // (the two chunks of a quarter-warp read opposite halves of their rows);
                // the three-frame window slides along the chunk.  Y4[t SP_TL + l] =
                // (RC, CR) of pixel l at frame t.
                constexpr int NLP = SP_TL / 2, NCH = SP_THREADS / NLP;
                const float4* Y4 = reinterpret_cast<const float4*>(Y);
                float* dstA = A + (size_t)s * F * 2 * per_axis;
                const int lp = threadIdx.x & (NLP - 1), ch = threadIdx.x / NLP;
                const int la = lp + NLP * (ch & 1), lb = lp + NLP * (1 - (ch & 1));
                const bool oka = lat0 + la < N, okb = lat0 + lb < N;
                const int per = (F + NCH - 1) / NCH, t0 = ch * per;
                auto ld = [&](int t, int l) -> float4 {
                    return (t >= 0 && t < F) ? Y4[t * SP_TL + l] : make_float4(0.f, 0.f, 0.f, 0.f);
                };
                auto qf = [](float4 v) { return make_float2(v.x * v.z + v.y * v.w, v.y * v.z - v.x * v.w); };
                float2 qma = qf(ld(t0 - 1, la)), qmb = qf(ld(t0 - 1, lb));
                float2 q0a = qf(ld(t0, la)), q0b = qf(ld(t0, lb));
                float4 ya = ld(t0, la), yb = ld(t0, lb);
#pragma unroll
                for (int i = 0; i < per; ++i) {
                    const int t = t0 + i;
                    float aa, ab;
                    if (OUT == SP_OUT_XDOPPLER) {
                        const float2 qpa = qf(ld(t + 1, la)), qpb = qf(ld(t + 1, lb));
                        const float ra = qma.x + q0a.x + qpa.x, ia = qma.y + q0a.y + qpa.y;
                        const float rb = qmb.x + q0b.x + qpb.x, ib = qmb.y + q0b.y + qpb.y;
                        aa = sqrt_approx(sqrt_approx(ra * ra + ia * ia));
                        ab = sqrt_approx(sqrt_approx(rb * rb + ib * ib));
                        qma = q0a;
                        q0a = qpa;
                        qmb = q0b;
                        q0b = qpb;
                    } else {
                        const float ra = ya.x + ya.z, ia = ya.y + ya.w, rb = yb.x + yb.z, ib = yb.y + yb.w;
                        aa = sqrt_approx(ra * ra + ia * ia);
                        ab = sqrt_approx(rb * rb + ib * ib);
                        ya = ld(t + 1, la);
                        yb = ld(t + 1, lb);
                    }
                    float mm = 0.f;
                    if (t < F) {
                        float* d = dstA + ((size_t)t * 2 + axis) * per_axis + rest0;
                        if (oka) {
                            __stcs(d + la, aa);
                            mm = aa;
                        }
                        if (okb) {
                            __stcs(d + lb, ab);
                            mm = fmaxf(mm, ab);
                        }
                    }
                    mm = fmaxf(mm, __shfl_xor_sync(0xffffffffu, mm, 1));
                    mm = fmaxf(mm, __shfl_xor_sync(0xffffffffu, mm, 2));
                    if (lp == 0 && t < F) atomicMax(mx + s * F + t, __float_as_uint(mm));
                }
            }
            __syncthreads();
        }
    }
    if (OUT != SP_OUT_COMPLEX)
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

template <int MX, int OUT, int FT>
rca_status launch_mx(rca_handle* h, const void* planes, int pt, const SepConst& sc, int S, int nz, int N,
                     float2* sub, float* A, unsigned* M, size_t smem, long long ngroups)
{
    auto kern = k_separate<MX, OUT, FT>;
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
    for (int R : {6, 8, 10, 12, 15, 16, 20})
        for (int m = 0; m < R; ++m)
            sc.wr[wr_off(R) + m] = make_float2((float)std::cos(2.0 * pi * m / R), (float)-std::sin(2.0 * pi * m / R));
    // pass twiddle tables: rows of tw_pitch(R) entries per k < Ns (passes with Ns > 1)
    {
        int Ns = 1, off = 0;
        for (int p = 0; p < sc.npass; ++p) {
            sc.twoff[p] = off;
            if (Ns > 1) off += Ns * tw_pitch(sc.radix[p]);
            Ns *= sc.radix[p];
        }
        sc.ntw = off;
    }
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
    const int out = !A ? SP_OUT_COMPLEX : enh == ULM_ENH_XDOPPLER ? SP_OUT_XDOPPLER : SP_OUT_COHERENT;
    const size_t smem = (size_t)2 * F * SP_G * sizeof(float2) + (size_t)sc.ntw * sizeof(float2) +
                        (out != SP_OUT_COMPLEX ? (size_t)sc.nsub * F * sizeof(unsigned) : 0) + (size_t)F;
    const long long ngroups = 2LL * g.S * g.nz * ((g.N + SP_TL - 1) / SP_TL);
    unsigned* Mu = reinterpret_cast<unsigned*>(M);
    if (out != SP_OUT_COMPLEX) {
        cudaError_t e = cudaMemsetAsync(M, 0, sizeof(float) * (size_t)sc.nsub * F, h->stream);
        if (e != cudaSuccess) return cuda_check(h, e, "separation maxima");
    }
    const int mx = (F * SP_G + SP_THREADS - 1) / SP_THREADS;
#define SP_LAUNCH(MXV, FTV)                                                                                     \
    return out == SP_OUT_XDOPPLER                                                                               \
               ? launch_mx<MXV, SP_OUT_XDOPPLER, FTV>(h, planes, (int)pt, sc, g.S, g.nz, g.N, sub, A, Mu, smem, ngroups) \
           : out == SP_OUT_COHERENT                                                                              \
               ? launch_mx<MXV, SP_OUT_COHERENT, FTV>(h, planes, (int)pt, sc, g.S, g.nz, g.N, sub, A, Mu, smem, ngroups) \
               : launch_mx<MXV, SP_OUT_COMPLEX, FTV>(h, planes, (int)pt, sc, g.S, g.nz, g.N, sub, A, Mu, smem, ngroups)
    if (F == 300) SP_LAUNCH(19, 300);   // the paper's ensemble: plan 20 x 15 at compile time
    if (mx <= 8) SP_LAUNCH(8, 0);
    if (mx <= 19) SP_LAUNCH(19, 0);
    SP_LAUNCH(32, 0);
#undef SP_LAUNCH
}
