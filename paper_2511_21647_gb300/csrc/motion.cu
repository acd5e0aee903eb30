// Projection-based rigid motion estimation (Sec. II-A3, Fig. 1d): Fourier-
// domain cross-correlation of every frame's Stage-1 slices with frame 0.
//
// The slices are zero-padded to Zp x Xp (Zp the next power of two >= nzs,
// Xp = N) and transformed by hand-written radix-4 / radix-2 FFTs in shared
// memory; forward transforms leave the spectra in bit-reversed order, which
// the pointwise product and the inverse transforms take as they are:
//   k_mo_twiddles   exp(-2 pi i k / n) tables for both axes (double, rounded)
//   k_mo_rows       forward FFT of every slice row (one warp per row) and the
//                   row energies
//   k_mo_cols       per 32-column tile of one slice: forward FFT of each column;
//                   for frame 0 the 2D spectrum is kept as the reference,
//                   otherwise it is multiplied by the reference's conjugate and
//                   transformed back along the columns
//   k_mo_peak       one CTA per (frame, transmission): inverse FFT of every row,
//                   the peak of |R| (first in row-major order on ties), its four
//                   neighbours for the parabolic sub-pixel refinement, the NCC
//   k_mo_combine    RC / CR averaging into one 3D displacement per frame
// No scaling in either direction: R comes out Zp Xp times the correlation.
#include <algorithm>
#include <cmath>

#include "rca_internal.cuh"

namespace {

#define MO_TILE 16        // columns per k_mo_cols CTA (three CTAs per SM at 512 rows)
#define MO_TP (MO_TILE + 1)  // padded tile row: a warp's column walk spreads over the banks

__device__ __forceinline__ float2 c_mul(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ float2 c_mulc(float2 a, float2 b) { return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y); }

// twiddles w_n^k = exp(-2 pi i k / n), k < n / 2, for n = Xp (first Xp / 2
// entries) and n = Zp (next Zp / 2)
__global__ void k_mo_twiddles(int xp, int zp, float2* __restrict__ tw)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int nx = xp / 2, nz = zp / 2;
    if (i >= nx + nz) return;
    const int n = i < nx ? xp : zp, k = i < nx ? i : i - nx;
    double s, c;
    sincospi(-2.0 * (double)k / (double)n, &s, &c);
    tw[i] = make_float2((float)c, (float)s);
}

// In-place FFTs of n = 2^logn points buf[i * st] by the 32 lanes of one warp,
// no scaling.  The forward transform is decimation in frequency (natural
// order in, bit-reversed order out) and the inverse decimation in time
// (bit-reversed in, natural out), so a spectrum is only ever multiplied
// pointwise in bit-reversed order and no reordering pass is needed.  Two
// radix-2 stages run as one radix-4 butterfly on four points held in
// registers (one shared-memory pass per two stages); an odd stage count adds
// one radix-2 stage.  tw[k] = exp(-2 pi i k / n), k < n / 2; the inverse uses
// the conjugates.

// -i v (forward) or +i v (inverse)
__device__ __forceinline__ float2 rot_q(float2 v, bool inverse)
{
    return inverse ? make_float2(-v.y, v.x) : make_float2(v.y, -v.x);
}

__device__ __forceinline__ float2 tw_get(const float2* tw, int i, bool inverse)
{
    float2 w = tw[i];
    if (inverse) w.y = -w.y;
    return w;
}

// natural -> bit-reversed
__device__ __forceinline__ void warp_fft_dif(float2* buf, int st, int logn, const float2* tw, bool inverse, int lane)
{
    const int n = 1 << logn;
    int s = logn;
    if (s & 1) {
        // single radix-2 stage, half = 2^(s-1)
        const int half = 1 << (s - 1), tstep = n >> s;
        for (int bf = lane; bf < n / 2; bf += 32) {
            const int pos = bf & (half - 1), i0 = (bf >> (s - 1)) * 2 * half + pos, i1 = i0 + half;
            const float2 u = buf[i0 * st], v = buf[i1 * st];
            buf[i0 * st] = make_float2(u.x + v.x, u.y + v.y);
            buf[i1 * st] = c_mul(make_float2(u.x - v.x, u.y - v.y), tw_get(tw, pos * tstep, inverse));
        }
        __syncwarp();
        --s;
    }
    for (; s >= 2; s -= 2) {
        // stages s (half 2h) then s - 1 (half h) on a, b, c, d at i0 + {0, h, 2h, 3h}
        const int h = 1 << (s - 2);
        for (int g = lane; g < n / 4; g += 32) {
            const int pos = g & (h - 1), i0 = (g >> (s - 2)) * 4 * h + pos;
            const float2 a = buf[i0 * st], b = buf[(i0 + h) * st], c = buf[(i0 + 2 * h) * st],
                         d = buf[(i0 + 3 * h) * st];
            const float2 w2 = tw_get(tw, pos * (n >> s), inverse);            // w_{4h}^pos
            const float2 w1 = tw_get(tw, pos * (n >> (s - 1)), inverse);      // w_{2h}^pos
            const float2 a1 = make_float2(a.x + c.x, a.y + c.y);
            const float2 c1 = c_mul(make_float2(a.x - c.x, a.y - c.y), w2);
            const float2 b1 = make_float2(b.x + d.x, b.y + d.y);
            const float2 d1 = rot_q(c_mul(make_float2(b.x - d.x, b.y - d.y), w2), inverse);
            buf[i0 * st] = make_float2(a1.x + b1.x, a1.y + b1.y);
            buf[(i0 + h) * st] = c_mul(make_float2(a1.x - b1.x, a1.y - b1.y), w1);
            buf[(i0 + 2 * h) * st] = make_float2(c1.x + d1.x, c1.y + d1.y);
            buf[(i0 + 3 * h) * st] = c_mul(make_float2(c1.x - d1.x, c1.y - d1.y), w1);
        }
        __syncwarp();
    }
}

// bit-reversed -> natural
__device__ __forceinline__ void warp_fft_dit(float2* buf, int st, int logn, const float2* tw, bool inverse, int lane)
{
    const int n = 1 << logn;
    int s = 1;
    for (; s + 1 <= logn; s += 2) {
        // stages s (half h) then s + 1 (half 2h) on a, b, c, d at i0 + {0, h, 2h, 3h}
        const int h = 1 << (s - 1);
        for (int g = lane; g < n / 4; g += 32) {
            const int pos = g & (h - 1), i0 = (g >> (s - 1)) * 4 * h + pos;
            const float2 a = buf[i0 * st], b = buf[(i0 + h) * st], c = buf[(i0 + 2 * h) * st],
                         d = buf[(i0 + 3 * h) * st];
            const float2 w1 = tw_get(tw, pos * (n >> s), inverse);            // w_{2h}^pos
            const float2 w2 = tw_get(tw, pos * (n >> (s + 1)), inverse);      // w_{4h}^pos
            const float2 tb = c_mul(b, w1), td = c_mul(d, w1);
            const float2 a1 = make_float2(a.x + tb.x, a.y + tb.y), b1 = make_float2(a.x - tb.x, a.y - tb.y);
            const float2 c1 = make_float2(c.x + td.x, c.y + td.y), d1 = make_float2(c.x - td.x, c.y - td.y);
            const float2 tc = c_mul(c1, w2), tdd = rot_q(c_mul(d1, w2), inverse);
            buf[i0 * st] = make_float2(a1.x + tc.x, a1.y + tc.y);
            buf[(i0 + 2 * h) * st] = make_float2(a1.x - tc.x, a1.y - tc.y);
            buf[(i0 + h) * st] = make_float2(b1.x + tdd.x, b1.y + tdd.y);
            buf[(i0 + 3 * h) * st] = make_float2(b1.x - tdd.x, b1.y - tdd.y);
        }
        __syncwarp();
    }
    if (s == logn) {
        const int half = 1 << (s - 1);
        for (int bf = lane; bf < n / 2; bf += 32) {
            const int pos = bf & (half - 1), i0 = (bf >> (s - 1)) * 2 * half + pos, i1 = i0 + half;
            const float2 u = buf[i0 * st], v = c_mul(buf[i1 * st], tw_get(tw, pos * (n >> s), inverse));
            buf[i0 * st] = make_float2(u.x + v.x, u.y + v.y);
            buf[i1 * st] = make_float2(u.x - v.x, u.y - v.y);
        }
        __syncwarp();
    }
}

// forward FFT of every slice row; B[f][k][z][Xp], E[f][k][z] = sum |s|^2
__global__ void __launch_bounds__(256) k_mo_rows(const float2* __restrict__ sl, int nt, int nzs, int xp, int logx,
                                                 const float2* __restrict__ tw, float2* __restrict__ B,
                                                 float* __restrict__ E)
{
    extern __shared__ float2 smo[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float2* stw = smo;                                  // twiddles [xp / 2]
    float2* buf = smo + xp / 2 + (size_t)warp * xp;
    for (int i = threadIdx.x; i < xp / 2; i += blockDim.x) stw[i] = tw[i];
    __syncthreads();
    const int z = blockIdx.x * 8 + warp;
    const size_t fk = (size_t)blockIdx.z * nt + blockIdx.y;
    if (z >= nzs) return;
    const float2* src = sl + (fk * nzs + z) * xp;
    float e = 0.f;
    for (int x = lane; x < xp; x += 32) {
        const float2 v = src[x];
        buf[x] = v;
        e = fmaf(v.x, v.x, fmaf(v.y, v.y, e));
    }
    for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
    __syncwarp();
    warp_fft_dif(buf, 1, logx, stw, false, lane);
    float2* dst = B + (fk * nzs + z) * xp;
    for (int x = lane; x < xp; x += 32) dst[x] = buf[x];
    if (lane == 0) E[fk * nzs + z] = e;
}

// Column pass over a 32-column tile of one slice.  ref == nullptr: frame 0,
// keep the 2D spectrum in REF.  Otherwise multiply by conj(REF) and inverse
// FFT the columns into C[f][k][Zp][Xp].
__global__ void __launch_bounds__(256) k_mo_cols(const float2* __restrict__ B, int nt, int nzs, int xp, int zp, int logz,
                                                 const float2* __restrict__ twz, int frame_base,
                                                 const float2* __restrict__ ref, float2* __restrict__ out)
{
    extern __shared__ float2 smo[];
    float2* stw = smo;                                 // twiddles [zp / 2]
    float2* tile = smo + zp / 2;                       // [zp][MO_TP]
    const int nth = blockDim.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const int x0 = blockIdx.x * MO_TILE;
    const int k = blockIdx.y, f = frame_base + blockIdx.z;
    const size_t fk = (size_t)f * nt + k;
    for (int i = threadIdx.x; i < zp / 2; i += nth) stw[i] = twz[i];
    // element i of the tile: row i / MO_TILE, column i % MO_TILE (a warp covers two rows)
    for (int i = threadIdx.x; i < zp * MO_TILE; i += nth) {
        const int z = i / MO_TILE, c = i - z * MO_TILE;
        tile[z * MO_TP + c] = z < nzs ? B[(fk * nzs + z) * xp + x0 + c] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    for (int c = warp; c < MO_TILE; c += nwarp) warp_fft_dif(tile + c, MO_TP, logz, stw, false, lane);
    __syncthreads();
    if (!ref) {
        float2* dst = out + (size_t)k * zp * xp;
        for (int i = threadIdx.x; i < zp * MO_TILE; i += nth) {
            const int z = i / MO_TILE, c = i - z * MO_TILE;
            dst[(size_t)z * xp + x0 + c] = tile[z * MO_TP + c];
        }
        return;
    }
    const float2* rk = ref + (size_t)k * zp * xp;
    for (int i = threadIdx.x; i < zp * MO_TILE; i += nth) {
        const int z = i / MO_TILE, c = i - z * MO_TILE;
        tile[z * MO_TP + c] = c_mulc(tile[z * MO_TP + c], rk[(size_t)z * xp + x0 + c]);
    }
    __syncthreads();
    for (int c = warp; c < MO_TILE; c += nwarp) warp_fft_dit(tile + c, MO_TP, logz, stw, true, lane);
    __syncthreads();
    float2* dst = out + ((size_t)blockIdx.z * nt + k) * zp * xp;
    for (int i = threadIdx.x; i < zp * MO_TILE; i += nth) {
        const int z = i / MO_TILE, c = i - z * MO_TILE;
        dst[(size_t)z * xp + x0 + c] = tile[z * MO_TP + c];
    }
}

// |R|^2 of one inverse-transformed row into the caller's buffer
__device__ __forceinline__ void mo_row_mag(const float2* __restrict__ Crow, float2* buf, int xp, int logx,
                                           const float2* __restrict__ twx, int lane)
{
    for (int x = lane; x < xp; x += 32) buf[x] = Crow[x];
    __syncwarp();
    warp_fft_dit(buf, 1, logx, twx, true, lane);
}

// one CTA per (frame, transmission): peak, sub-pixel, NCC
__global__ void __launch_bounds__(256) k_mo_peak(const float2* __restrict__ C, const float* __restrict__ E, int nt,
                                                 int nzs, int xp, int zp, int logx, const float2* __restrict__ twx,
                                                 int frame_base, float* __restrict__ shifts, int* __restrict__ peaks)
{
    extern __shared__ float2 smo[];
    __shared__ float s_best[8];
    __shared__ int s_idx[8];
    __shared__ float s_nb[4];
    __shared__ float s_e[2];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    float2* stw = smo;                                  // twiddles [xp / 2]
    float2* buf = smo + xp / 2 + (size_t)warp * xp;
    for (int i = threadIdx.x; i < xp / 2; i += blockDim.x) stw[i] = twx[i];
    __syncthreads();
    const int k = blockIdx.x, fl = blockIdx.y, f = frame_base + fl;
    const float2* Cfk = C + ((size_t)fl * nt + k) * zp * xp;
    float best = -1.f;
    int bidx = 0x7fffffff;
    for (int z = warp; z < zp; z += nwarp) {
        mo_row_mag(Cfk + (size_t)z * xp, buf, xp, logx, stw, lane);
        for (int x = lane; x < xp; x += 32) {
            const float2 v = buf[x];
            const float m = v.x * v.x + v.y * v.y;
            const int idx = z * xp + x;
            if (m > best || (m == best && idx < bidx)) {
                best = m;
                bidx = idx;
            }
        }
        __syncwarp();
    }
    for (int o = 16; o > 0; o >>= 1) {
        const float ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bidx, o);
        if (ob > best || (ob == best && oi < bidx)) {
            best = ob;
            bidx = oi;
        }
    }
    if (lane == 0) {
        s_best[warp] = best;
        s_idx[warp] = bidx;
    }
    // frame energies (row sums of |s|^2)
    if (warp == nwarp - 1) {
        float e0 = 0.f, e1 = 0.f;
        for (int z = lane; z < nzs; z += 32) {
            e0 += E[((size_t)f * nt + k) * nzs + z];
            e1 += E[(size_t)k * nzs + z];
        }
        for (int o = 16; o > 0; o >>= 1) {
            e0 += __shfl_xor_sync(0xffffffffu, e0, o);
            e1 += __shfl_xor_sync(0xffffffffu, e1, o);
        }
        if (lane == 0) {
            s_e[0] = e0;
            s_e[1] = e1;
        }
    }
    __syncthreads();
    if (warp != 0) return;
    best = s_best[0];
    bidx = s_idx[0];
    for (int w = 1; w < nwarp; ++w)
        if (s_best[w] > best || (s_best[w] == best && s_idx[w] < bidx)) {
            best = s_best[w];
            bidx = s_idx[w];
        }
    const int iz = bidx / xp, ix = bidx - iz * xp;
    // neighbours: rows iz - 1 and iz + 1 at ix, row iz at ix - 1 and ix + 1 (circular)
    const int rows[3] = {(iz + zp - 1) & (zp - 1), iz, (iz + 1) & (zp - 1)};
    for (int r = 0; r < 3; ++r) {
        mo_row_mag(Cfk + (size_t)rows[r] * xp, buf, xp, logx, stw, lane);
        if (lane == 0) {
            auto mag = [&](int x) {
                const float2 v = buf[x];
                return sqrtf(v.x * v.x + v.y * v.y);
            };
            if (r == 0) s_nb[0] = mag(ix);
            if (r == 2) s_nb[1] = mag(ix);
            if (r == 1) {
                s_nb[2] = mag((ix + xp - 1) & (xp - 1));
                s_nb[3] = mag((ix + 1) & (xp - 1));
            }
        }
        __syncwarp();
    }
    if (lane == 0) {
        const float m0 = sqrtf(best);
        auto para = [](float mm, float m, float mp) {
            const float den = mm - 2.f * m + mp;
            if (den >= 0.f) return 0.f;
            return fminf(0.5f, fmaxf(-0.5f, (mm - mp) / (2.f * den)));
        };
        const int dz = iz < zp / 2 ? iz : iz - zp, dx = ix < xp / 2 ? ix : ix - xp;
        const float sz = (float)dz + para(s_nb[0], m0, s_nb[1]);
        const float sx = (float)dx + para(s_nb[2], m0, s_nb[3]);
        const float den = sqrtf(s_e[0]) * sqrtf(s_e[1]) * (float)zp * (float)xp;
        float* o = shifts + ((size_t)f * nt + k) * 3;
        o[0] = sz;
        o[1] = sx;
        o[2] = den > 0.f ? m0 / den : 0.f;
        if (peaks) {
            peaks[((size_t)f * nt + k) * 2] = dz;
            peaks[((size_t)f * nt + k) * 2 + 1] = dx;
        }
    }
}

// motion[f] = (x_RC pitch, y_CR pitch, (z_RC + z_CR) / 2 dz / us), averages over each family's K
__global__ void k_mo_combine(const float* __restrict__ shifts, int F, int K, double pitch, double row_m,
                             float* __restrict__ motion)
{
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= F) return;
    const float* s = shifts + (size_t)f * 2 * K * 3;
    double zr = 0.0, xr = 0.0, zc = 0.0, yc = 0.0;
    for (int k = 0; k < K; ++k) {
        zr += s[k * 3];
        xr += s[k * 3 + 1];
        zc += s[(K + k) * 3];
        yc += s[(K + k) * 3 + 1];
    }
    motion[f * 3] = (float)(xr / K * pitch);
    motion[f * 3 + 1] = (float)(yc / K * pitch);
    motion[f * 3 + 2] = (float)(0.5 * (zr + zc) / K * row_m);
}

int ilog2(int v)
{
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
}

}  // namespace

rca_status launch_motion(rca_handle* h, const rca_tables* t, const float2* slices, int F, float* motion,
                         float* shifts_out, int* peaks)
{
    const GeomDev& g = t->gd;
    const int nt = 2 * g.K, nzs = g.nzs, xp = g.N;
    if (xp < 32 || xp > 256 || (xp & (xp - 1)))
        return set_error(h, RCA_ERR_UNSUPPORTED, "motion estimation needs a power-of-two N in [32, 256] (N = %d)", xp);
    const int logz = ilog2(nzs), zp = 1 << logz, logx = ilog2(xp);
    // the column pass holds Zp x 33 complex values in shared memory
    if (zp > 512) return set_error(h, RCA_ERR_UNSUPPORTED, "motion estimation supports at most 512 slice rows");
    // workspace: twiddles, B [F][2K][nzs][Xp], REF [2K][Zp][Xp], C [chunk][2K][Zp][Xp], E [F][2K][nzs],
    // shifts [F][2K][3]; frames are correlated in chunks so that C stays bounded
    const int chunk = std::min(F, 64);
    const size_t n_tw = (size_t)(xp + zp) / 2;
    const size_t nB = (size_t)F * nt * nzs * xp, nR = (size_t)nt * zp * xp, nC = (size_t)chunk * nt * zp * xp;
    const size_t nE = (size_t)F * nt * nzs, nS = (size_t)F * nt * 3;
    auto up = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t bytes = up(n_tw * 8) + up(nB * 8) + up(nR * 8) + up(nC * 8) + up(nE * 4) + up(nS * 4);
    rca_status st = RCA_OK;
    char* ws = (char*)ws_get(h, WS_MOTION, bytes, &st);
    if (!ws) return st;
    float2* tw = reinterpret_cast<float2*>(ws);
    float2* B = reinterpret_cast<float2*>(ws + up(n_tw * 8));
    float2* REF = reinterpret_cast<float2*>((char*)B + up(nB * 8));
    float2* Cb = reinterpret_cast<float2*>((char*)REF + up(nR * 8));
    float* E = reinterpret_cast<float*>((char*)Cb + up(nC * 8));
    float* S = reinterpret_cast<float*>((char*)E + up(nE * 4));
    float* shifts = shifts_out ? shifts_out : S;

    const size_t smem_cols = ((size_t)zp * MO_TP + zp / 2) * sizeof(float2);
    const size_t smem_rows = ((size_t)8 * xp + xp / 2) * sizeof(float2);
    cudaError_t e = cudaFuncSetAttribute(k_mo_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_cols);
    if (e != cudaSuccess) return cuda_check(h, e, "motion column smem attribute");
    k_mo_twiddles<<<(unsigned)((n_tw + 255) / 256), 256, 0, h->stream>>>(xp, zp, tw);
    k_mo_rows<<<dim3((nzs + 7) / 8, nt, F), 256, smem_rows, h->stream>>>(slices, nt, nzs, xp, logx, tw, B, E);
    // reference spectrum (frame 0)
    k_mo_cols<<<dim3(xp / MO_TILE, nt, 1), 256, smem_cols, h->stream>>>(B, nt, nzs, xp, zp, logz, tw + xp / 2, 0,
                                                                         nullptr, REF);
    for (int f0 = 0; f0 < F; f0 += chunk) {
        const int nf = std::min(chunk, F - f0);
        k_mo_cols<<<dim3(xp / MO_TILE, nt, nf), 256, smem_cols, h->stream>>>(B, nt, nzs, xp, zp, logz, tw + xp / 2,
                                                                              f0, REF, Cb);
        k_mo_peak<<<dim3(nt, nf), 256, smem_rows, h->stream>>>(Cb, E, nt, nzs, xp, zp, logx, tw, f0, shifts, peaks);
    }
    k_mo_combine<<<(F + 127) / 128, 128, 0, h->stream>>>(shifts, F, g.K, g.pitch, g.dz / g.us, motion);
    return cuda_check(h, cudaGetLastError(), "motion kernels");
}
