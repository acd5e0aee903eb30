// tables.cu -- per-geometry delay / weight tables, computed on the GPU in FP64.
//
// Built with -fmad=false so every double expression rounds exactly as
// written (the transmit / receive delays are then bit-reproducible).
//
// Geometry (Sec. II-A1, Sec. II-C): element / pixel centres
// u = (e - (N-1)/2) pitch; RC transmission k has the plane-wave delay
// (z cos th + trans sin th + (L/2)|sin th|)/c and receives on line elements
// with sqrt(off^2 + z^2)/c.  Stage 1 works on slice rows z_r = z0 + r dz/us;
// the planes on rows z_i = z0 + i dz.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "rca_internal.cuh"

#define TWO_PI_D 6.283185307179586476925286766559
#define PI_D 3.1415926535897932384626433832795

namespace {

__device__ __forceinline__ double elem_pos(const GeomDev& g, int e)
{
    return ((double)e - 0.5 * (g.N - 1)) * g.pitch;
}

__device__ __forceinline__ double slice_z(const GeomDev& g, int r) { return g.z0 + (double)r * (g.dz / (double)g.us); }

__device__ __forceinline__ double plane_z(const GeomDev& g, int i) { return g.z0 + (double)i * g.dz; }

__device__ __forceinline__ double tau_tx(const GeomDev& g, int k, double trans, double z)
{
    return (z * g.cos_th[k] + trans * g.sin_th[k] + 0.5 * g.L * fabs(g.sin_th[k])) / g.c;
}

__device__ __forceinline__ double tau_rx(const GeomDev& g, double off, double z) { return sqrt(off * off + z * z) / g.c; }

__device__ __forceinline__ double tau_c(const GeomDev& g, int k, double z)
{
    return (z * (1.0 + g.cos_th[k]) + 0.5 * g.L * fabs(g.sin_th[k])) / g.c;
}

__device__ __forceinline__ double hann(const GeomDev& g, double off, double z)
{
    double a = z / g.fnum;
    if (fabs(off) > 0.5 * a) return 0.0;
    double ct = cos(PI_D * off / a);
    return ct * ct;
}

__device__ __forceinline__ float2 cis(double ph)
{
    double s, c;
    sincos(ph, &s, &c);
    return make_float2((float)c, (float)s);
}

__device__ __forceinline__ int q16(double samples) { return __double2int_rn(samples * 65536.0); }

// Stage-1 / DAS tables.  One thread per (r, d) of the [nzs][N] grid also
// fills the [2K][nzs] transmit tables and dmax for d == 0.
__global__ void k_tables_das(GeomDev g, double* tx_f64, double* rx_f64, int* tx_q16, int* rx_q16, float2* W,
                             int* dmax)
{
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= g.nzs * g.N) return;
    int r = idx / g.N, d = idx % g.N;
    double z = slice_z(g, r);
    double off = (double)d * g.pitch;
    double trx = tau_rx(g, off, z);
    rx_f64[(size_t)d * g.nzs + r] = trx * g.fs;
    rx_q16[idx] = q16(trx * g.fs);
    double w = hann(g, off, z);
    float2 ph = cis(TWO_PI_D * g.fc * (trx - z / g.c));
    W[idx] = make_float2((float)(w * (double)ph.x), (float)(w * (double)ph.y));
    if (d == 0) {
        double t0 = 2.0 * g.z0 / g.c;
        for (int k = 0; k < 2 * g.K; ++k) {
            double x = (tau_tx(g, k, 0.0, z) - t0) * g.fs;
            tx_f64[(size_t)k * g.nzs + r] = x;
            tx_q16[(size_t)k * g.nzs + r] = q16(x);
        }
        // largest lateral distance inside the aperture (hann() is non-zero there)
        double a = z / g.fnum;
        int m = -1;
        for (int dd = 0; dd < g.N; ++dd)
            if (!(fabs((double)dd * g.pitch) > 0.5 * a)) m = dd;
        dmax[r] = m;
    }
}

// Stage-2 per-(k, u) shift and carrier, per-(k, i) carrier.
// Stage-2 shift, lateral weights and carriers.  With rot[k][r] = exp(j 2 pi
// fc (1 + cos th_k) z_r / c) at slice row r and kappa_k the constant carrier
// phase exp(j 2 pi fc (L/2) |sin th_k| / c), the carrier of plane row i is
// ec[k][i] = kappa_k rot[k][us i]; the lateral-slab weights of transverse
// position u on the rotated slab sums (slice rows us i + sfl, us i + sfl + 1)
// are a = (1 - fr) exp(j ph), b = fr exp(j (ph - beta_k)),
// ph = 2 pi fc ((1 + cos th_k)(dz_k(u) - sfl dz / us) + (L/2)|sin th_k|) / c,
// beta_k = 2 pi fc (1 + cos th_k)(dz / us) / c.
__global__ void k_tables_s2(GeomDev g, double* shift, int* sfl, float* sfr, float2* psi, float2* ec, float2* rot,
                            float4* lw)
{
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    int nt = 2 * g.K;
    if (idx < nt * g.N) {
        int k = idx / g.N, m = idx % g.N;
        double u = elem_pos(g, m);
        double sh = u * g.sin_th[k] / (1.0 + g.cos_th[k]);
        double s = sh * (double)g.us / g.dz;
        double fl = floor(s);
        double fr = s - fl;
        shift[idx] = s;
        sfl[idx] = (int)fl;
        sfr[idx] = (float)fr;
        psi[idx] = cis(TWO_PI_D * g.fc * ((1.0 + g.cos_th[k]) * sh / g.c));
        double ph = TWO_PI_D * g.fc * ((1.0 + g.cos_th[k]) * (sh - fl * g.dz / (double)g.us) + 0.5 * g.L * fabs(g.sin_th[k])) / g.c;
        double beta = TWO_PI_D * g.fc * (1.0 + g.cos_th[k]) * (g.dz / (double)g.us) / g.c;
        double sa, ca, sb, cb;
        sincos(ph, &sa, &ca);
        sincos(ph - beta, &sb, &cb);
        lw[idx] = make_float4((float)((1.0 - fr) * ca), (float)((1.0 - fr) * sa), (float)(fr * cb), (float)(fr * sb));
    }
    if (idx < nt * g.nz) {
        int k = idx / g.nz, i = idx % g.nz;
        ec[idx] = cis(TWO_PI_D * g.fc * tau_c(g, k, plane_z(g, i)));
    }
    if (idx < nt * g.nzs) {
        int k = idx / g.nzs, r = idx % g.nzs;
        rot[idx] = cis(TWO_PI_D * g.fc * (1.0 + g.cos_th[k]) * slice_z(g, r) / g.c);
    }
}

// Transverse-slab sum coefficients: for plane row i of slab b,
//   sum_{u in slab} valid(zeta) exp(j 2 pi fc tau_c,k(z_i + dz_k(u))) lerp_weights(zeta)
// gathered onto slice rows us*i + tmin[k][b] + t, t < T.
// coefr: the same taps for the carrier-rotated slices, each contribution at
// slice row n times conj(rot[k][n]): the phase 2 pi fc ((1 + cos th_k)
// (z_i + dz_k(u) - z_n) + (L/2)|sin th_k|) / c.
__global__ void k_tables_coef(GeomDev g, const double* shift, const int* tmin, int T, float2* coef, float2* coefr,
                              unsigned* status)
{
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    int nt = 2 * g.K;
    if (idx >= nt * g.S * g.nz) return;
    int i = idx % g.nz;
    int b = (idx / g.nz) % g.S;
    int k = idx / (g.nz * g.S);
    double accr[16], acci[16], rotr[16], roti[16];
    for (int t = 0; t < T; ++t) accr[t] = acci[t] = rotr[t] = roti[t] = 0.0;
    int base = g.us * i + tmin[k * g.S + b];
    for (int m = b * g.P; m < (b + 1) * g.P; ++m) {
        double s = shift[(size_t)k * g.N + m];
        double zeta = (double)(g.us * i) + s;
        if (!(zeta >= 0.0) || zeta > (double)(g.nzs - 1)) continue;
        // slice row and fraction from us*i + floor(s) (equal to floor(zeta)
        // except within rounding of an integer, where the interpolant is continuous)
        double fl = floor(s);
        int n0 = g.us * i + (int)fl;
        double fr = s - fl;
        double sh = elem_pos(g, m) * g.sin_th[k] / (1.0 + g.cos_th[k]);
        double ph = TWO_PI_D * g.fc * tau_c(g, k, plane_z(g, i) + sh);
        double sn, cs;
        sincos(ph, &sn, &cs);
        int t = n0 - base;
        if (t < 0 || t + (fr > 0.0 ? 1 : 0) >= T) {
            atomicOr(status, ST_BOUNDS);
            continue;
        }
        accr[t] += (1.0 - fr) * cs;
        acci[t] += (1.0 - fr) * sn;
        if (fr > 0.0) {
            accr[t + 1] += fr * cs;
            acci[t + 1] += fr * sn;
        }
        // rotated: z_i + dz_k(u) - z_n = (fr - j) dz / us at slice rows n0 + j
        const double kap = 0.5 * g.L * fabs(g.sin_th[k]);
        const double a1 = 1.0 + g.cos_th[k];
        const double step = g.dz / (double)g.us;
        double s0, c0;
        sincos(TWO_PI_D * g.fc * (a1 * fr * step + kap) / g.c, &s0, &c0);
        rotr[t] += (1.0 - fr) * c0;
        roti[t] += (1.0 - fr) * s0;
        if (fr > 0.0) {
            double s1, c1;
            sincos(TWO_PI_D * g.fc * (a1 * (fr - 1.0) * step + kap) / g.c, &s1, &c1);
            rotr[t + 1] += fr * c1;
            roti[t + 1] += fr * s1;
        }
    }
    for (int t = 0; t < T; ++t) {
        coef[(size_t)idx * T + t] = make_float2((float)accr[t], (float)acci[t]);
        coefr[(size_t)idx * T + t] = make_float2((float)rotr[t], (float)roti[t]);
    }
}

// Row-independent transverse-slab taps: for slab b,
//   c2[k][b][t] = sum_{u in slab} exp(j 2 pi fc (1 + cos th_k) dz_k(u) / c) lerp_weights,
// so that coef[k][b][i][t] = ec[k][i] c2[k][b][t] wherever every shifted row
// of the slab lies inside the slice (the carrier phase of tau_c is linear in z).
// c2r = c2 kappa_k exp(-j beta_k (tmin + t)): the taps on the carrier-rotated
// slices, ec[k][i] conj(rot[k][us i + tmin + t]) being independent of i.
__global__ void k_tables_coef2(GeomDev g, const double* shift, const int* tmin, int T, float2* c2, float2* c2r,
                               unsigned* status)
{
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    int nt = 2 * g.K;
    if (idx >= nt * g.S) return;
    int b = idx % g.S, k = idx / g.S;
    double accr[16], acci[16];
    for (int t = 0; t < T; ++t) accr[t] = acci[t] = 0.0;
    for (int m = b * g.P; m < (b + 1) * g.P; ++m) {
        double s = shift[(size_t)k * g.N + m];
        double fl = floor(s);
        double fr = s - fl;
        double sh = elem_pos(g, m) * g.sin_th[k] / (1.0 + g.cos_th[k]);
        double sn, cs;
        sincos(TWO_PI_D * g.fc * (1.0 + g.cos_th[k]) * sh / g.c, &sn, &cs);
        int t = (int)fl - tmin[idx];
        if (t < 0 || t + (fr > 0.0 ? 1 : 0) >= T) {
            atomicOr(status, ST_BOUNDS);
            continue;
        }
        accr[t] += (1.0 - fr) * cs;
        acci[t] += (1.0 - fr) * sn;
        if (fr > 0.0) {
            accr[t + 1] += fr * cs;
            acci[t + 1] += fr * sn;
        }
    }
    const double kap = TWO_PI_D * g.fc * 0.5 * g.L * fabs(g.sin_th[k]) / g.c;
    const double beta = TWO_PI_D * g.fc * (1.0 + g.cos_th[k]) * (g.dz / (double)g.us) / g.c;
    for (int t = 0; t < T; ++t) {
        c2[(size_t)idx * T + t] = make_float2((float)accr[t], (float)acci[t]);
        double sn, cs;
        sincos(kap - beta * (double)(tmin[idx] + t), &sn, &cs);
        c2r[(size_t)idx * T + t] = make_float2((float)(accr[t] * cs - acci[t] * sn), (float)(accr[t] * sn + acci[t] * cs));
    }
}

// Conventional-DAS transmit tables at every transverse position and plane row.
__global__ void k_tables_direct(GeomDev g, int* dtx_q16, float2* dtx_ph)
{
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    int nt = 2 * g.K;
    if (idx >= nt * g.N * g.nz) return;
    int i = idx % g.nz;
    int m = (idx / g.nz) % g.N;
    int k = idx / (g.nz * g.N);
    double z = plane_z(g, i);
    double ttx = tau_tx(g, k, elem_pos(g, m), z);
    double t0 = 2.0 * g.z0 / g.c;
    dtx_q16[idx] = q16((ttx - t0) * g.fs);
    dtx_ph[idx] = cis(TWO_PI_D * g.fc * (ttx + z / g.c));
}

__global__ void k_tables_mix(GeomDev g, float2* mix)
{
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= g.ns) return;
    double t0 = 2.0 * g.z0 / g.c;
    mix[n] = cis(-TWO_PI_D * g.fc * (t0 + (double)n / g.fs));
}

// Half-band Hamming low-pass, 31 taps, cut-off fs/4: centre 1/2, even
// offsets 0, odd offsets sinc(m/2) * hamming(m) scaled to sum to 1/2.
void fir_taps(float out[31])
{
    double h[31];
    double odd = 0.0;
    for (int m = -15; m <= 15; ++m) {
        double v = 0.0;
        if (m % 2 != 0) {
            double x = 0.5 * PI_D * m;
            v = 0.5 * (std::sin(x) / x) * (0.54 + 0.46 * std::cos(PI_D * m / 15.0));
            odd += v;
        }
        h[m + 15] = v;
    }
    for (int m = -15; m <= 15; ++m) out[m + 15] = (m == 0) ? 0.5f : (float)(h[m + 15] * (0.5 / odd));
}

template <typename T>
T* dalloc(rca_handle* h, size_t n, rca_status* st)
{
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, n * sizeof(T) + 16);
    if (e != cudaSuccess) {
        *st = cuda_check(h, e, "cudaMalloc(tables)");
        return nullptr;
    }
    return (T*)p;
}

}  // namespace

rca_status launch_tables(rca_handle* h, rca_tables* t)
{
    const GeomDev& g = t->gd;
    const int nt = 2 * g.K;
    rca_status st = RCA_OK;
    t->tx_f64 = dalloc<double>(h, (size_t)nt * g.nzs, &st);
    t->rx_f64 = dalloc<double>(h, (size_t)g.N * g.nzs, &st);
    t->tx_q16 = dalloc<int>(h, (size_t)nt * g.nzs, &st);
    t->rx_q16 = dalloc<int>(h, (size_t)g.N * g.nzs, &st);
    t->W = dalloc<float2>(h, (size_t)g.N * g.nzs, &st);
    t->dmax = dalloc<int>(h, (size_t)g.nzs, &st);
    t->s2_shift = dalloc<double>(h, (size_t)nt * g.N, &st);
    t->s2_sfl = dalloc<int>(h, (size_t)nt * g.N, &st);
    t->s2_sfr = dalloc<float>(h, (size_t)nt * g.N, &st);
    t->s2_psi = dalloc<float2>(h, (size_t)nt * g.N, &st);
    t->s2_ec = dalloc<float2>(h, (size_t)nt * g.nz, &st);
    t->s2_rot = dalloc<float2>(h, (size_t)nt * g.nzs, &st);
    t->s2_lw = dalloc<float4>(h, (size_t)nt * g.N, &st);
    t->s2_tmin = dalloc<int>(h, (size_t)nt * g.S, &st);
    t->dtx_q16 = dalloc<int>(h, (size_t)nt * g.N * g.nz, &st);
    t->dtx_ph = dalloc<float2>(h, (size_t)nt * g.N * g.nz, &st);
    t->mix = dalloc<float2>(h, (size_t)g.ns, &st);
    if (st != RCA_OK) return st;
    fir_taps(t->fir);

    cudaStream_t s = h->stream;
    const int B = 256;
    k_tables_das<<<(g.nzs * g.N + B - 1) / B, B, 0, s>>>(g, t->tx_f64, t->rx_f64, t->tx_q16, t->rx_q16, t->W,
                                                          t->dmax);
    int n2 = std::max({nt * g.N, nt * g.nz, nt * g.nzs});
    k_tables_s2<<<(n2 + B - 1) / B, B, 0, s>>>(g, t->s2_shift, t->s2_sfl, t->s2_sfr, t->s2_psi, t->s2_ec, t->s2_rot,
                                               t->s2_lw);
    k_tables_direct<<<(nt * g.N * g.nz + B - 1) / B, B, 0, s>>>(g, t->dtx_q16, t->dtx_ph);
    k_tables_mix<<<(g.ns + B - 1) / B, B, 0, s>>>(g, t->mix);
    if ((st = cuda_check(h, cudaGetLastError(), "table kernels")) != RCA_OK) return st;

    // Download what the host needs to size the launches.
    std::vector<int> txq((size_t)nt * g.nzs), rxq((size_t)g.N * g.nzs), dm(g.nzs), sfl((size_t)nt * g.N),
        dtx((size_t)nt * g.N * g.nz);
    cudaMemcpyAsync(txq.data(), t->tx_q16, txq.size() * 4, cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(rxq.data(), t->rx_q16, rxq.size() * 4, cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(dm.data(), t->dmax, dm.size() * 4, cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(sfl.data(), t->s2_sfl, sfl.size() * 4, cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(dtx.data(), t->dtx_q16, dtx.size() * 4, cudaMemcpyDeviceToHost, s);
    if ((st = cuda_check(h, cudaStreamSynchronize(s), "table download")) != RCA_OK) return st;

    // Stage-2: slab coefficient offsets and the shift range per family.
    std::vector<int> tmin((size_t)nt * g.S);
    int T = 2;
    for (int k = 0; k < nt; ++k)
        for (int b = 0; b < g.S; ++b) {
            int lo = 1 << 30, hi = -(1 << 30);
            for (int m = b * g.P; m < (b + 1) * g.P; ++m) {
                lo = std::min(lo, sfl[(size_t)k * g.N + m]);
                hi = std::max(hi, sfl[(size_t)k * g.N + m]);
            }
            tmin[(size_t)k * g.S + b] = lo;
            T = std::max(T, hi - lo + 2);
        }
    if (T > 16) return set_error(h, RCA_ERR_UNSUPPORTED, "Stage-2 shift spans %d slice rows within one slab (max 14)", T - 2);
    t->T = T;
    for (int fam = 0; fam < 2; ++fam) {
        int lo = 1 << 30, hi = -(1 << 30);
        for (int k = fam * g.K; k < (fam + 1) * g.K; ++k)
            for (int m = 0; m < g.N; ++m) {
                lo = std::min(lo, sfl[(size_t)k * g.N + m]);
                hi = std::max(hi, sfl[(size_t)k * g.N + m]);
            }
        t->s2.smin[fam] = lo;
        t->s2.smax[fam] = hi + 1;
    }
    t->s2_coef = dalloc<float2>(h, (size_t)nt * g.S * g.nz * T, &st);
    t->s2_coefr = dalloc<float2>(h, (size_t)nt * g.S * g.nz * T, &st);
    if (st != RCA_OK) return st;
    cudaMemcpyAsync(t->s2_tmin, tmin.data(), tmin.size() * 4, cudaMemcpyHostToDevice, s);
    k_tables_coef<<<(nt * g.S * g.nz + B - 1) / B, B, 0, s>>>(g, t->s2_shift, t->s2_tmin, T, t->s2_coef,
                                                                 t->s2_coefr, h->d_status);
    if ((st = cuda_check(h, cudaGetLastError(), "coef kernel")) != RCA_OK) return st;
    t->s2_c2 = dalloc<float2>(h, (size_t)nt * g.S * T, &st);
    t->s2_c2r = dalloc<float2>(h, (size_t)nt * g.S * T, &st);
    if (st != RCA_OK) return st;
    k_tables_coef2<<<(nt * g.S + B - 1) / B, B, 0, s>>>(g, t->s2_shift, t->s2_tmin, T, t->s2_c2, t->s2_c2r,
                                                          h->d_status);
    if ((st = cuda_check(h, cudaGetLastError(), "coef2 kernel")) != RCA_OK) return st;
    // plane rows whose shifted slice rows (floor(shift) .. floor(shift) + 1
    // around us * i) all lie inside [0, nzs - 1]
    {
        int iA = 0, iB = g.nz - 1;
        for (int v : sfl) {
            iA = std::max(iA, v < 0 ? (-v + g.us - 1) / g.us : 0);
            const int room = g.nzs - 2 - v;
            iB = std::min(iB, room >= 0 ? room / g.us : -1);
        }
        t->s2_iA = iA;
        t->s2_iB = iB;
    }

    t->h_txq = txq;
    t->h_rxq = rxq;
    t->h_dm = dm;
    t->h_sfl = sfl;
    // Stage 1: the tallest row tile / widest distance chunk whose double
    // buffer leaves room for two CTAs per SM (the autotuner may replace it)
    const size_t budget = 104 * 1024;
    const int shapes[][2] = {{16, 16}, {16, 8}, {8, 8}, {8, 4}, {4, 4}, {4, 2}, {2, 2}, {1, 1}};
    int zt = 1, dc = 1;
    for (auto& sh : shapes) {
        zt = sh[0];
        dc = sh[1];
        if (stage1_smem_bytes(t, zt, dc, stage1_ring(t, zt, dc, nullptr, nullptr), sizeof(float2)) <= budget) break;
    }
    if ((st = plan_stage1(h, t, zt, dc)) != RCA_OK) return st;
    // Stage 2: the tallest plane-row tile that fits the same budget
    int zp = S2_ZP;
    while (zp > 1 && stage2_smem_bytes(t, zp) > 100 * 1024) zp /= 2;
    if (stage2_smem_bytes(t, zp) > 200 * 1024) return set_error(h, RCA_ERR_UNSUPPORTED, "Stage-2 tile exceeds shared memory");
    plan_stage2(t, zp);

    // Direct mode windows (per transverse position; rows of plane depth).
    {
        int dzt = 16, win = 0;
        for (;;) {
            win = 0;
            int tiles = (g.nz + dzt - 1) / dzt;
            for (int k = 0; k < nt; ++k)
                for (int m = 0; m < g.N; ++m)
                    for (int tt = 0; tt < tiles; ++tt) {
                        long lo = 1L << 40, hi = -(1L << 40);
                        for (int i = tt * dzt; i < std::min(g.nz, (tt + 1) * dzt); ++i) {
                            int r = i * g.us;
                            long tq = dtx[((size_t)k * g.N + m) * g.nz + i];
                            lo = std::min(lo, (tq + rxq[(size_t)r * g.N]) >> 16);
                            hi = std::max(hi, (tq + rxq[(size_t)r * g.N + std::max(0, dm[r])]) >> 16);
                        }
                        win = std::max(win, (int)(hi - lo + 2));
                    }
            if ((size_t)win * g.N * sizeof(float2) <= budget || dzt == 1) break;
            dzt /= 2;
        }
        t->direct_zt = dzt;
        t->direct_win = win;
    }
    return cuda_check(h, cudaStreamSynchronize(s), "table build");
}

// ---------------------------------------------------------------------------
// launch-shape planning from the host copies of the tables
// ---------------------------------------------------------------------------
// Stage-1 chunks: row tiles of zt slice rows, lateral distances in chunks of
// dc.  A chunk needs the contiguous sample rows [lo, hi] of the [ns][E] IQ
// block (its delays' integer parts plus the interpolation neighbour); lo and
// hi only grow from one chunk of a tile to the next.  The CTA keeps the rows
// in a ring of R rows: sample row n sits in slot (n - base) mod R (base: the
// tile's first row), and while chunk c runs, the rows of chunk c + 1 that
// are not resident yet are fetched into slots that chunk c does not read.
// That holds when R >= hi(c + 1) - lo(c) + 1 for consecutive chunks with
// work; R is the largest such span over all tiles.  Slot R repeats slot 0,
// so that a row and its successor are always R-adjacent.
// Returns R; fills the chunk table and the per-(k, tile) base rows.
int stage1_ring(const rca_tables* t, int zt, int dc, std::vector<int4>* out, std::vector<int>* bases)
{
    const GeomDev& g = t->gd;
    const int nt = 2 * g.K;
    const int tiles = (g.nzs + zt - 1) / zt, nch = (g.N + dc - 1) / dc;
    std::vector<long> lo_v((size_t)nt * tiles * nch), hi_v((size_t)nt * tiles * nch);
    int R = 1;
    for (int k = 0; k < nt; ++k)
        for (int tt = 0; tt < tiles; ++tt) {
            long plo = 0;
            bool prev = false;
            for (int c = 0; c < nch; ++c) {
                const int d0 = c * dc, d1 = std::min(g.N, d0 + dc);
                long lo = 1L << 40, hi = -(1L << 40);
                for (int r = tt * zt; r < std::min(g.nzs, (tt + 1) * zt); ++r) {
                    if (t->h_dm[r] < d0) continue;
                    const long tq = t->h_txq[(size_t)k * g.nzs + r];
                    lo = std::min(lo, (tq + t->h_rxq[(size_t)r * g.N + d0]) >> 16);
                    hi = std::max(hi, ((tq + t->h_rxq[(size_t)r * g.N + std::min(d1 - 1, t->h_dm[r])]) >> 16) + 1);
                }
                const size_t i = ((size_t)k * tiles + tt) * nch + c;
                lo_v[i] = lo;
                hi_v[i] = hi;
                if (hi < lo) continue;
                R = std::max(R, (int)(hi - lo + 1));
                if (prev) R = std::max(R, (int)(hi - plo + 1));
                plo = lo;
                prev = true;
            }
        }
    if (out) out->assign((size_t)nt * tiles * nch, make_int4(0, 0, 0, 0));
    if (bases) bases->assign((size_t)nt * tiles, 0);
    if (!out) return R;
    for (int k = 0; k < nt; ++k)
        for (int tt = 0; tt < tiles; ++tt) {
            bool first = true;
            long base = 0, top = 0;           // top: last resident row
            for (int c = 0; c < nch; ++c) {
                const size_t i = ((size_t)k * tiles + tt) * nch + c;
                const int d0 = c * dc, d1 = std::min(g.N, d0 + dc);
                const long lo = lo_v[i], hi = hi_v[i];
                if (hi < lo) {
                    (*out)[i] = make_int4(0, 0, d0, d0);
                    continue;
                }
                if (first) {
                    base = lo;
                    top = lo - 1;
                    first = false;
                }
                const long a = std::max(lo, top + 1);
                const int cnt = (int)std::max(0L, hi - a + 1);
                const int slot = (int)((a - base) % R);
                (*out)[i] = make_int4((int)a, cnt | (slot << 16), d0, d1);
                top = std::max(top, hi);
            }
            if (bases) (*bases)[(size_t)k * tiles + tt] = (int)base;
        }
    return R;
}

// bytes of one chunk's record block: [dc][zt] 16-byte records + [dc][zt]
// 4-byte ring offsets, rounded up to 16 (a TMA bulk copy unit)
static int stage1_rblk(int zt, int dc) { return ((zt * dc * 20) + 15) / 16 * 16; }

// double-buffered sample windows and record blocks
size_t stage1_smem_bytes(const rca_tables* t, int zt, int dc, int ring, size_t esz)
{
    return (size_t)(ring + 1) * t->gd.N * esz + 2 * (size_t)stage1_rblk(zt, dc);
}

// Stage-1 records of every (k, tile, chunk): one thread per (d, row) slot.
// HALF: FP16 weights {Re a, Re b}, {Im a, Im b}, then the window offset for
// 4-byte samples; otherwise FP32 {Re a, Re b, Im a, Im b} with the offsets
// (for 8-byte samples) in the block's second array.  a = w (1 - fr),
// b = w fr, halved at d = 0 (the two mirror elements coincide there); zero
// (and offset 0, a slot the tile's first chunk fills) where the distance is
// outside the row's aperture or the delay leaves the record.
template <bool HALF>
__global__ void k_s1_records(GeomDev g, const int* __restrict__ tx_q16, const int* __restrict__ rx_q16,
                             const float2* __restrict__ W, const int* __restrict__ dmax,
                             const int4* __restrict__ chunks, const int* __restrict__ bases, int ring, int zt,
                             int dc, int n_tiles, int nch, int rblk, unsigned char* __restrict__ out)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int per_blk = zt * dc;
    const long long total = (long long)2 * g.K * n_tiles * nch * per_blk;
    if (idx >= total) return;
    const int slot = (int)(idx % per_blk);
    const long long cb = idx / per_blk;             // (k * n_tiles + tile) * nch + c
    const int tile = (int)((cb / nch) % n_tiles), k = (int)(cb / ((long long)nch * n_tiles));
    const int dd = slot / zt, rr = slot - dd * zt;
    const int4 cc = chunks[cb];
    const int r = tile * zt + rr, d = cc.z + dd;
    const int RS = g.N * (HALF ? 4 : 8);
    const int qmax = (g.ns - 1) << 16;
    float ax = 0.f, bx = 0.f, ay = 0.f, by = 0.f;
    int off = 0;
    if (r < g.nzs && d < cc.w && d <= dmax[r]) {
        const int q = tx_q16[(size_t)k * g.nzs + r] + rx_q16[(size_t)r * g.N + d];
        if (q >= 0 && q <= qmax) {
            const float2 w = W[(size_t)r * g.N + d];
            const float fr = (float)(q & 0xffff) * (1.0f / 65536.0f);
            const float h = d == 0 ? 0.5f : 1.0f;
            ax = h * w.x * (1.0f - fr);
            bx = h * w.x * fr;
            ay = h * w.y * (1.0f - fr);
            by = h * w.y * fr;
            off = (((q >> 16) - bases[cb / nch]) % ring) * RS;
        }
    }
    unsigned char* blk = out + cb * rblk;
    uint4 rec;
    if (HALF) {
        const __half2 re = __floats2half2_rn(ax, bx), im = __floats2half2_rn(ay, by);
        rec = make_uint4(*reinterpret_cast<const unsigned*>(&re), *reinterpret_cast<const unsigned*>(&im),
                         (unsigned)off, 0u);
    } else {
        rec = make_uint4(__float_as_uint(ax), __float_as_uint(bx), __float_as_uint(ay), __float_as_uint(by));
    }
    reinterpret_cast<uint4*>(blk)[slot] = rec;
    reinterpret_cast<int*>(blk + (size_t)per_blk * 16)[slot] = off;
}

rca_status plan_stage1(rca_handle* h, rca_tables* t, int zt, int dc)
{
    std::vector<int4> chunks;
    std::vector<int> bases;
    const int ring = stage1_ring(t, zt, dc, &chunks, &bases);
    if (stage1_smem_bytes(t, zt, dc, ring, sizeof(float2)) > 200 * 1024)
        return set_error(h, RCA_ERR_UNSUPPORTED, "Stage-1 sample ring of %d samples x %d elements exceeds shared memory",
                         ring, t->gd.N);
    rca_status st = RCA_OK;
    int4* d = dalloc<int4>(h, chunks.size(), &st);
    int* db = st == RCA_OK ? dalloc<int>(h, bases.size(), &st) : nullptr;
    if (st == RCA_OK)
        st = cuda_check(h, cudaMemcpyAsync(d, chunks.data(), chunks.size() * sizeof(int4), cudaMemcpyHostToDevice,
                                           h->stream), "chunk upload");
    if (st == RCA_OK)
        st = cuda_check(h, cudaMemcpyAsync(db, bases.data(), bases.size() * sizeof(int), cudaMemcpyHostToDevice,
                                           h->stream), "ring base upload");
    if (st == RCA_OK) st = cuda_check(h, cudaStreamSynchronize(h->stream), "chunk upload sync");
    if (st != RCA_OK) {
        if (d) cudaFree(d);
        if (db) cudaFree(db);
        return st;
    }
    const int n_tiles = (t->gd.nzs + zt - 1) / zt, nch = (t->gd.N + dc - 1) / dc;
    const int rblk = stage1_rblk(zt, dc);
    const size_t nblk = (size_t)2 * t->gd.K * n_tiles * nch;
    unsigned char* r32 = dalloc<unsigned char>(h, nblk * rblk, &st);
    unsigned char* r16 = st == RCA_OK ? dalloc<unsigned char>(h, nblk * rblk, &st) : nullptr;
    if (st != RCA_OK) {
        cudaFree(d);
        cudaFree(db);
        if (r32) cudaFree(r32);
        return st;
    }
    const long long slots = (long long)nblk * zt * dc;
    const unsigned grid = (unsigned)((slots + 255) / 256);
    k_s1_records<false><<<grid, 256, 0, h->stream>>>(t->gd, t->tx_q16, t->rx_q16, t->W, t->dmax, d, db, ring, zt, dc,
                                                      n_tiles, nch, rblk, r32);
    k_s1_records<true><<<grid, 256, 0, h->stream>>>(t->gd, t->tx_q16, t->rx_q16, t->W, t->dmax, d, db, ring, zt, dc,
                                                     n_tiles, nch, rblk, r16);
    st = cuda_check(h, cudaGetLastError(), "Stage-1 record kernels");
    if (st == RCA_OK) st = cuda_check(h, cudaStreamSynchronize(h->stream), "Stage-1 record build");
    cudaFree(db);
    if (st != RCA_OK) {
        cudaFree(d);
        cudaFree(r32);
        cudaFree(r16);
        return st;
    }
    if (t->s1.d_chunks) cudaFree(t->s1.d_chunks);
    if (t->s1.d_rec32) cudaFree(t->s1.d_rec32);
    if (t->s1.d_rec16) cudaFree(t->s1.d_rec16);
    t->s1.d_chunks = d;
    t->s1.d_rec32 = r32;
    t->s1.d_rec16 = r16;
    t->s1.rblk = rblk;
    t->s1.zt = zt;
    t->s1.dc = dc;
    t->s1.ring = ring;
    t->s1.n_tiles = n_tiles;
    t->s1.nch = nch;
    return RCA_OK;
}

size_t stage2_smem_bytes(const rca_tables* t, int zp)
{
    const int span = std::max(t->s2.smax[0] - t->s2.smin[0], t->s2.smax[1] - t->s2.smin[1]) + 2;
    const int rows = t->gd.us * (zp - 1) + span;
    return s2_smem_bytes(t->gd.K, t->gd.S, t->gd.N, t->gd.P, t->T, rows);
}

void plan_stage2(rca_tables* t, int zp)
{
    const int span = std::max(t->s2.smax[0] - t->s2.smin[0], t->s2.smax[1] - t->s2.smin[1]) + 2;
    t->s2.zp = zp;
    t->s2.rows = t->gd.us * (zp - 1) + span;
    t->s2.n_tiles = (t->gd.nz + zp - 1) / zp;
}
