/*
 * rca_oracle.c -- FP64 CPU oracle (TEST INFRASTRUCTURE ONLY; see rca_oracle.h).
 *
 * Plain loops, double precision, no blocking or reordering beyond what each
 * definition states.  Compiled with -ffp-contract=off so that the geometry
 * expressions round exactly as written.
 */
#include "rca_oracle.h"

#include <math.h>
#include <omp.h>
#include <stdlib.h>
#include <string.h>

#define TWO_PI 6.283185307179586476925286766559
#define OR_PI 3.1415926535897932384626433832795

/* ------------------------------------------------------------------------ */
/* Geometry (Sec. II-A1; acquisition constants Sec. II-C)                    */
/* ------------------------------------------------------------------------ */

/* element / lateral pixel centre u_e = (e - (N-1)/2) * pitch */
double or_elem_pos(const or_geom* g, int e) { return ((double)e - 0.5 * (g->n_el - 1)) * g->pitch; }

/* pixel depth z_i = z0 + i dz */
double or_depth(const or_geom* g, int i) { return g->z0 + (double)i * g->dz; }

/* Stage-1 slice row r lies at depth z0 + r dz/us (us-fold finer than the planes) */
double or_slice_depth(const or_geom* g, int r) { return g->z0 + (double)r * (g->dz / (double)g->us); }

int or_slice_rows(const or_geom* g) { return (g->nz - 1) * g->us + 1; }

/* time of the first sample: round trip to the top of the imaging region */
double or_t0(const or_geom* g) { return 2.0 * g->z0 / g->c; }

static double aperture_len(const or_geom* g) { return (double)g->n_el * g->pitch; }

/* Plane-wave transmit delay of transmission k at transverse coordinate `trans`
 * (y for RC: rows transmit, steering in y-z; x for CR) and depth z.  The
 * (L/2)|sin th| term starts the clock when the first element fires. */
double or_tau_tx(const or_geom* g, int k, double trans, double z)
{
    double th = g->ang[k];
    return (z * cos(th) + trans * sin(th) + 0.5 * aperture_len(g) * fabs(sin(th))) / g->c;
}

/* Receive delay to a line element at lateral offset lat_off (the element is a
 * strip along the transverse axis, so only the lateral offset and depth count). */
double or_tau_rx(const or_geom* g, double lat_off, double z)
{
    return sqrt(lat_off * lat_off + z * z) / g->c;
}

/* Receive apodisation (the paper does not state one): Hann over the F-number
 * aperture a = z / F#, w = cos^2(pi * lat_off / a) for |lat_off| <= a/2. */
double or_apod(const or_geom* g, double lat_off, double z)
{
    double a = z / g->fnum;
    if (fabs(lat_off) > 0.5 * a) return 0.0;
    double cth = cos(OR_PI * lat_off / a);
    return cth * cth;
}

/* Carrier reference delay of transmission k at depth z on the reference slice:
 * the on-axis round trip (z cos th + (L/2)|sin th|)/c + z/c.  Stage 1 removes
 * it (baseband slices), Stage 2 re-applies it at the shifted depth. */
double or_tau_c(const or_geom* g, int k, double z)
{
    double th = g->ang[k];
    return (z * (1.0 + cos(th)) + 0.5 * aperture_len(g) * fabs(sin(th))) / g->c;
}

/* Stage-2 rigid axial shift (Sec. II-A1: slices along the transmit direction
 * differ by an axial shift set by the steering angle).  Reading: the shift
 * that keeps the on-axis round-trip delay equal, dz = u sin th / (1 + cos th). */
double or_shift_dz(const or_geom* g, int k, double u)
{
    double th = g->ang[k];
    return u * sin(th) / (1.0 + cos(th));
}

/* ------------------------------------------------------------------------ */
/* RF -> IQ                                                                  */
/* ------------------------------------------------------------------------ */

/* Half-band low-pass (cut-off fs/4), 31 taps, Hamming window: h[0] = 1/2,
 * even offsets 0, odd offsets proportional to sinc(m/2) * hamming(m) and
 * scaled so that they sum to 1/2 (DC gain exactly 1, gain at fs/2 exactly 0).
 * h[15 + m] holds tap m, m = -15..15. */
void or_fir_taps(double h[OR_FIR_TAPS])
{
    const int half = (OR_FIR_TAPS - 1) / 2;
    double odd_sum = 0.0;
    for (int m = -half; m <= half; ++m) {
        double v = 0.0;
        if (m != 0 && (m % 2) != 0) {
            double x = 0.5 * OR_PI * m;
            double sinc = sin(x) / x;
            double ham = 0.54 + 0.46 * cos(OR_PI * m / half);
            v = 0.5 * sinc * ham;
            odd_sum += v;
        }
        h[m + half] = v;
    }
    for (int m = -half; m <= half; ++m)
        if (m != 0) h[m + half] *= 0.5 / odd_sum;
    h[half] = 0.5;
}

/* Clutter removal + IQ demodulation (the paper beamforms IQ, Sec. II-C, and
 * filters clutter before Stage 2, Sec. II-A2).  Reading: the temporal mean of
 * every (tx, element, sample) over the ensemble is removed (exact for static
 * tissue), then
 *   b[n] = 2 sum_m h[m] r~[n-m] exp(-j 2 pi fc t_{n-m}),  t_n = t0 + n / fs,
 * with samples outside [0, ns) taken as zero. */
void or_demod(const or_geom* g, int F, const float* rf, int remove_mean, int n_sel, const int* sel,
              double* iq)
{
    const int nt = 2 * g->K, E = g->n_el, ns = g->ns;
    const int half = (OR_FIR_TAPS - 1) / 2;
    double h[OR_FIR_TAPS];
    or_fir_taps(h);
    const double t0 = or_t0(g);
    double* mean = (double*)calloc((size_t)nt * E * ns, sizeof(double));
    if (remove_mean) {
        for (int f = 0; f < F; ++f)
            for (size_t q = 0; q < (size_t)nt * E * ns; ++q) mean[q] += (double)rf[(size_t)f * nt * E * ns + q];
        for (size_t q = 0; q < (size_t)nt * E * ns; ++q) mean[q] /= (double)F;
    }
    if (!sel) n_sel = F;
#pragma omp parallel for collapse(3) schedule(static)
    for (int q = 0; q < n_sel; ++q)
        for (int k = 0; k < nt; ++k)
            for (int e = 0; e < E; ++e) {
                int f = sel ? sel[q] : q;
                double* mre = (double*)malloc(sizeof(double) * ns);
                double* mim = (double*)malloc(sizeof(double) * ns);
                size_t ich = (((size_t)q * nt + k) * E + e) * ns;
                size_t ch = (((size_t)f * nt + k) * E + e) * ns;
                size_t mch = ((size_t)k * E + e) * ns;
                for (int n = 0; n < ns; ++n) {
                    double r = (double)rf[ch + n] - mean[mch + n];
                    double ph = -TWO_PI * g->fc * (t0 + (double)n / g->fs);
                    mre[n] = r * cos(ph);
                    mim[n] = r * sin(ph);
                }
                for (int n = 0; n < ns; ++n) {
                    double re = 0.0, im = 0.0;
                    for (int m = -half; m <= half; ++m) {
                        int s = n - m;
                        if (s < 0 || s >= ns) continue;
                        re += h[m + half] * mre[s];
                        im += h[m + half] * mim[s];
                    }
                    iq[2 * (ich + n)] = 2.0 * re;
                    iq[2 * (ich + n) + 1] = 2.0 * im;
                }
                free(mre);
                free(mim);
            }
    free(mean);
}

/* Linear interpolation of one channel's IQ at fractional sample xi; zero
 * outside [0, ns-1] (the paper does not name its interpolator). */
static void iq_at(const double* ch, int ns, double xi, double* re, double* im)
{
    *re = 0.0;
    *im = 0.0;
    if (!(xi >= 0.0) || xi > (double)(ns - 1)) return;
    int n0 = (int)floor(xi);
    double fr = xi - (double)n0;
    double r = ch[2 * n0], i = ch[2 * n0 + 1];
    if (fr > 0.0) {
        r = (1.0 - fr) * r + fr * ch[2 * (n0 + 1)];
        i = (1.0 - fr) * i + fr * ch[2 * (n0 + 1) + 1];
    }
    *re = r;
    *im = i;
}

/* ------------------------------------------------------------------------ */
/* Conventional 3D DAS and block sum-projection                              */
/* ------------------------------------------------------------------------ */

/* One voxel of transmission k: sum over receive elements of
 *   w(lat - u_e, z) * IQ_{k,e}(tau) * exp(j 2 pi fc tau),
 *   tau = tau_tx(k, trans, z) + tau_rx(lat - u_e, z).
 * RC (k < K): lat = x, trans = y.  CR: lat = y, trans = x. */
static void das_voxel(const or_geom* g, const double* iq_frame, int k, double lat, double trans,
                      double z, double* out_re, double* out_im)
{
    const int E = g->n_el, ns = g->ns;
    const double t0 = or_t0(g);
    double re = 0.0, im = 0.0;
    double ttx = or_tau_tx(g, k, trans, z);
    for (int e = 0; e < E; ++e) {
        double off = lat - or_elem_pos(g, e);
        double w = or_apod(g, off, z);
        if (w == 0.0) continue;
        double tau = ttx + or_tau_rx(g, off, z);
        double br, bi;
        iq_at(iq_frame + 2 * ((size_t)k * E + e) * ns, ns, (tau - t0) * g->fs, &br, &bi);
        double ph = TWO_PI * g->fc * tau;
        double cr = cos(ph), ci = sin(ph);
        re += w * (br * cr - bi * ci);
        im += w * (br * ci + bi * cr);
    }
    *out_re = re;
    *out_im = im;
}

/* V_fam(x_j, y_m, z_i) = sum over the family's K transmissions (coherent
 * compounding, Sec. II-A1), computed voxel by voxel. */
void or_das_volume(const or_geom* g, const double* iq_frame, int fam, double* V)
{
    const int N = g->n_el, nz = g->nz, K = g->K;
#pragma omp parallel for collapse(2) schedule(static)
    for (int j = 0; j < N; ++j)
        for (int m = 0; m < N; ++m)
            for (int i = 0; i < nz; ++i) {
                double x = or_elem_pos(g, j), y = or_elem_pos(g, m), z = or_depth(g, i);
                double sr = 0.0, si = 0.0;
                for (int kk = 0; kk < K; ++kk) {
                    int k = fam * K + kk;
                    double r, im;
                    if (fam == 0) das_voxel(g, iq_frame, k, x, y, z, &r, &im);
                    else das_voxel(g, iq_frame, k, y, x, z, &r, &im);
                    sr += r;
                    si += im;
                }
                size_t o = 2 * (((size_t)j * N + m) * nz + i);
                V[o] = sr;
                V[o + 1] = si;
            }
}

static size_t plane_index(const or_geom* g, int axis, int fam, int b, int i, int l)
{
    const int S = g->n_el / g->P;
    return 2 * ((((((size_t)axis * 2 + fam) * S + b) * g->nz + i) * g->n_el) + l);
}

/* Block sum-projection (Sec. II-A4/A5): the N x N x nz volume is cut into
 * P x P x nz sub-blocks; XZ plane b sums the P y-positions of y-slab b,
 * YZ plane b sums the P x-positions of x-slab b. */
void or_project_volume(const or_geom* g, const double* V, int fam, double* planes_frame)
{
    const int N = g->n_el, nz = g->nz, P = g->P, S = N / P;
    for (int b = 0; b < S; ++b)
        for (int i = 0; i < nz; ++i)
            for (int l = 0; l < N; ++l) {
                double xr = 0, xi = 0, yr = 0, yi = 0;
                for (int t = b * P; t < b * P + P; ++t) {
                    size_t ox = 2 * (((size_t)l * N + t) * nz + i); /* x = l, y = t */
                    size_t oy = 2 * (((size_t)t * N + l) * nz + i); /* x = t, y = l */
                    xr += V[ox];
                    xi += V[ox + 1];
                    yr += V[oy];
                    yi += V[oy + 1];
                }
                size_t px = plane_index(g, 0, fam, b, i, l), py = plane_index(g, 1, fam, b, i, l);
                planes_frame[px] = xr;
                planes_frame[px + 1] = xi;
                planes_frame[py] = yr;
                planes_frame[py + 1] = yi;
            }
}

/* The same projection computed pixel by pixel straight from channel data,
 * with no volume: each plane pixel sums the DAS voxels of its slab. */
void or_project_direct(const or_geom* g, const double* iq_frame, int fam, double* planes_frame)
{
    const int N = g->n_el, nz = g->nz, P = g->P, S = N / P, K = g->K;
#pragma omp parallel for collapse(3) schedule(static)
    for (int axis = 0; axis < 2; ++axis)
        for (int b = 0; b < S; ++b)
            for (int i = 0; i < nz; ++i)
                for (int l = 0; l < N; ++l) {
                    double sr = 0.0, si = 0.0;
                    for (int t = b * P; t < b * P + P; ++t) {
                        /* axis 0 (XZ): x = l, y = t;  axis 1 (YZ): x = t, y = l */
                        double x = or_elem_pos(g, axis == 0 ? l : t);
                        double y = or_elem_pos(g, axis == 0 ? t : l);
                        double z = or_depth(g, i);
                        for (int kk = 0; kk < K; ++kk) {
                            int k = fam * K + kk;
                            double r, im;
                            if (fam == 0) das_voxel(g, iq_frame, k, x, y, z, &r, &im);
                            else das_voxel(g, iq_frame, k, y, x, z, &r, &im);
                            sr += r;
                            si += im;
                        }
                    }
                    size_t o = plane_index(g, axis, fam, b, i, l);
                    planes_frame[o] = sr;
                    planes_frame[o + 1] = si;
                }
}

/* ------------------------------------------------------------------------ */
/* Two-stage beamforming (Sec. II-A1, Fig. 1b-c)                             */
/* ------------------------------------------------------------------------ */

/* Stage 1: reference slice S_k (lateral x for RC, y for CR) at transverse
 * coordinate 0, per transmission, with the carrier of the on-axis delay
 * removed (baseband slices, so Stage 2 can interpolate them along z):
 *   S_k(l, i) = sum_e w * IQ(tau0) * exp(j 2 pi fc (tau0 - tau_c,k(z_i))),
 *   tau0 = tau_tx(k, 0, z_i) + tau_rx(u_l - u_e, z_i). */
void or_stage1(const or_geom* g, const double* iq_frame, double* S)
{
    const int N = g->n_el, nz = or_slice_rows(g), E = g->n_el, ns = g->ns, nt = 2 * g->K;
    const double t0 = or_t0(g);
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < nt; ++k)
        for (int i = 0; i < nz; ++i)
            for (int l = 0; l < N; ++l) {
                double z = or_slice_depth(g, i), lat = or_elem_pos(g, l);
                double ttx = or_tau_tx(g, k, 0.0, z), tc = or_tau_c(g, k, z);
                double re = 0.0, im = 0.0;
                for (int e = 0; e < E; ++e) {
                    double off = lat - or_elem_pos(g, e);
                    double w = or_apod(g, off, z);
                    if (w == 0.0) continue;
                    double tau0 = ttx + or_tau_rx(g, off, z);
                    double br, bi;
                    iq_at(iq_frame + 2 * ((size_t)k * E + e) * ns, ns, (tau0 - t0) * g->fs, &br, &bi);
                    double ph = TWO_PI * g->fc * (tau0 - tc);
                    double cr = cos(ph), ci = sin(ph);
                    re += w * (br * cr - bi * ci);
                    im += w * (br * ci + bi * cr);
                }
                size_t o = 2 * (((size_t)k * nz + i) * N + l);
                S[o] = re;
                S[o + 1] = im;
            }
}

/* Stage 2 for one voxel of transmission k: the reference slice is shifted
 * axially by dz_k(u) (u = transverse coordinate) and the carrier re-applied:
 *   V_k(l, u, z_i) = S~_k(l, zeta) * exp(j 2 pi fc tau_c,k(z')),
 *   z' = z_i + dz_k(u), zeta = us i + dz_k(u) us / dz (slice-row units),
 * S~ linear in zeta and zero for zeta outside [0, nzs-1]. */
static void stage2_voxel(const or_geom* g, const double* S, int k, int l, double u, int i,
                         double* re, double* im)
{
    const int N = g->n_el, nz = or_slice_rows(g);
    double sh = or_shift_dz(g, k, u);
    double zeta = (double)(g->us * i) + sh * (double)g->us / g->dz;
    *re = 0.0;
    *im = 0.0;
    if (!(zeta >= 0.0) || zeta > (double)(nz - 1)) return;
    int n0 = (int)floor(zeta);
    double fr = zeta - (double)n0;
    const double* s0 = S + 2 * (((size_t)k * nz + n0) * N + l);
    double sr = s0[0], si = s0[1];
    if (fr > 0.0) {
        const double* s1 = S + 2 * (((size_t)k * nz + n0 + 1) * N + l);
        sr = (1.0 - fr) * sr + fr * s1[0];
        si = (1.0 - fr) * si + fr * s1[1];
    }
    double ph = TWO_PI * g->fc * or_tau_c(g, k, or_depth(g, i) + sh);
    double cr = cos(ph), ci = sin(ph);
    *re = sr * cr - si * ci;
    *im = sr * ci + si * cr;
}

/* Stage-2 volume of one family: V_fam = sum_k V_k (compounding). */
void or_stage2_volume(const or_geom* g, const double* S, int fam, double* V)
{
    const int N = g->n_el, nz = g->nz, K = g->K;
#pragma omp parallel for collapse(2) schedule(static)
    for (int j = 0; j < N; ++j)
        for (int m = 0; m < N; ++m)
            for (int i = 0; i < nz; ++i) {
                double sr = 0.0, si = 0.0;
                for (int kk = 0; kk < K; ++kk) {
                    int k = fam * K + kk;
                    double r, im;
                    /* RC: slice lateral = x (j), transverse = y (m); CR: swapped */
                    if (fam == 0) stage2_voxel(g, S, k, j, or_elem_pos(g, m), i, &r, &im);
                    else stage2_voxel(g, S, k, m, or_elem_pos(g, j), i, &r, &im);
                    sr += r;
                    si += im;
                }
                size_t o = 2 * (((size_t)j * N + m) * nz + i);
                V[o] = sr;
                V[o + 1] = si;
            }
}

/* Stage 2 straight into the projection planes of both families: the
 * extrapolated volume of each family is built and block sum-projected. */
void or_stage2_project(const or_geom* g, const double* S, double* planes_frame)
{
    const int N = g->n_el, nz = g->nz;
    double* V = (double*)malloc(sizeof(double) * 2 * (size_t)N * N * nz);
    for (int fam = 0; fam < 2; ++fam) {
        or_stage2_volume(g, S, fam, V);
        or_project_volume(g, V, fam, planes_frame);
    }
    free(V);
}

/* ------------------------------------------------------------------------ */
/* Localisation (Sec. II-A4)                                                 */
/* ------------------------------------------------------------------------ */

/* XDoppler enhancement (Sec. II-A4, ref. [40]; formula not printed).
 * Reading: on each projection pixel, the RC and CR planes of the same axis
 * and slab are cross-correlated over a centred 3-frame window (clipped at the
 * ensemble ends) and the amplitude is
 *   A_t = sqrt(| sum_{t'} P_RC,t' * conj(P_CR,t') |).
 * M_t is the maximum of A over all planes of frame t (thresholding, Sec. II-A4). */
void or_xdoppler(int F, int S, int nz, int N, const double* planes, double* A, double* M)
{
    const size_t plane = (size_t)nz * N;
    for (int t = 0; t < F; ++t) {
        double mx = 0.0;
        for (int axis = 0; axis < 2; ++axis)
            for (int b = 0; b < S; ++b)
                for (size_t p = 0; p < plane; ++p) {
                    double qr = 0.0, qi = 0.0;
                    for (int tt = t - 1; tt <= t + 1; ++tt) {
                        if (tt < 0 || tt >= F) continue;
                        size_t rc = 2 * (((((size_t)tt * 2 + axis) * 2 + 0) * S + b) * plane + p);
                        size_t cr = 2 * (((((size_t)tt * 2 + axis) * 2 + 1) * S + b) * plane + p);
                        double ar = planes[rc], ai = planes[rc + 1];
                        double br = planes[cr], bi = -planes[cr + 1];
                        qr += ar * br - ai * bi;
                        qi += ar * bi + ai * br;
                    }
                    double a = sqrt(sqrt(qr * qr + qi * qi));
                    A[(((size_t)t * 2 + axis) * S + b) * plane + p] = a;
                    if (a > mx) mx = a;
                }
        M[t] = mx;
    }
}

/* Normalised cross-correlation of one plane with a d x d Gaussian kernel
 * G(qz, ql) = exp(-qz^2 / 2 sz^2) exp(-ql^2 / 2 sl^2) (the Gaussian-fitted PSF,
 * Sec. II-A4), evaluated directly in 2D:
 *   NCC(p) = sum_q (A(p+q) - mu_p)(G(q) - mu_G)
 *            / sqrt( sum_q (A(p+q) - mu_p)^2 * sum_q (G(q) - mu_G)^2 ).
 * NCC = 0 within h = (d-1)/2 of the plane border, and where the local sum of
 * squares sum_q (A - mu_p)^2 <= 1e-5 d^2 Mt^2 (flat window; Mt = frame max). */
void or_ncc_plane(int nz, int N, const double* A, int d, double sig_z, double sig_l, double Mt,
                  double* ncc)
{
    const int h = (d - 1) / 2;
    const int dd = d * d;
    double* G = (double*)malloc(sizeof(double) * dd);
    double muG = 0.0;
    for (int a = -h; a <= h; ++a)
        for (int b = -h; b <= h; ++b) {
            double v = exp(-(double)(a * a) / (2.0 * sig_z * sig_z)) * exp(-(double)(b * b) / (2.0 * sig_l * sig_l));
            G[(a + h) * d + (b + h)] = v;
            muG += v;
        }
    muG /= dd;
    double ssG = 0.0;
    for (int q = 0; q < dd; ++q) ssG += (G[q] - muG) * (G[q] - muG);
    const double flat = 1e-5 * dd * Mt * Mt;
    for (int i = 0; i < nz; ++i)
        for (int l = 0; l < N; ++l) {
            double v = 0.0;
            if (i >= h && i < nz - h && l >= h && l < N - h && Mt > 0.0) {
                double mu = 0.0;
                for (int a = -h; a <= h; ++a)
                    for (int b = -h; b <= h; ++b) mu += A[(size_t)(i + a) * N + (l + b)];
                mu /= dd;
                double num = 0.0, ssA = 0.0;
                for (int a = -h; a <= h; ++a)
                    for (int b = -h; b <= h; ++b) {
                        double da = A[(size_t)(i + a) * N + (l + b)] - mu;
                        num += da * (G[(a + h) * d + (b + h)] - muG);
                        ssA += da * da;
                    }
                if (ssA > flat) v = num / sqrt(ssA * ssG);
            }
            ncc[(size_t)i * N + l] = v;
        }
    free(G);
}

/* three-point parabolic vertex offset, clamped to [-1/2, 1/2]; 0 when the
 * three values are not strictly concave. */
static double parabolic(double fm, double f0, double fp)
{
    double den = fm - 2.0 * f0 + fp;
    if (den >= 0.0) return 0.0;
    double dlt = (fm - fp) / (2.0 * den);
    if (dlt < -0.5) dlt = -0.5;
    if (dlt > 0.5) dlt = 0.5;
    return dlt;
}

/* Sub-pixel regional peaks of one NCC map (Sec. II-A4).  Reading:
 * p is a localisation iff NCC(p) >= ncc_min, A(p) >= alpha * Mt, and NCC(p)
 * is a 3x3 regional maximum with raster-order tie-break (strictly greater than
 * neighbours that come earlier in z-major order, not smaller than later ones).
 * Sub-pixel offsets: parabolic fit of NCC along each axis.  Output in raster
 * order; returns the number found (entries beyond cap are not written). */
int or_peaks_plane(int nz, int N, const double* A, const double* ncc, double Mt, double alpha,
                   double ncc_min, int cap, or_loc2d* out)
{
    int n = 0;
    for (int i = 1; i < nz - 1; ++i)
        for (int l = 1; l < N - 1; ++l) {
            size_t p = (size_t)i * N + l;
            double c = ncc[p];
            if (!(c >= ncc_min) || !(A[p] >= alpha * Mt)) continue;
            int ok = 1;
            for (int a = -1; a <= 1 && ok; ++a)
                for (int b = -1; b <= 1 && ok; ++b) {
                    if (a == 0 && b == 0) continue;
                    double q = ncc[(size_t)(i + a) * N + (l + b)];
                    int earlier = (a < 0) || (a == 0 && b < 0);
                    if (earlier ? !(c > q) : !(c >= q)) ok = 0;
                }
            if (!ok) continue;
            if (n < cap) {
                out[n].frame = 0;
                out[n].axis = 0;
                out[n].slab = 0;
                out[n].iz = i;
                out[n].ilat = l;
                out[n].z = (double)i + parabolic(ncc[p - N], c, ncc[p + N]);
                out[n].lat = (double)l + parabolic(ncc[p - 1], c, ncc[p + 1]);
                out[n].ncc = c;
                out[n].amp = A[p];
            }
            ++n;
        }
    return n;
}

/* All planes of an ensemble, in (frame, axis, slab, iz, ilat) order. */
int or_localize2d(int F, int S, int nz, int N, const double* A, const double* M, int d,
                  double sig_z, double sig_l, double alpha, double ncc_min, int cap, or_loc2d* out)
{
    const size_t plane = (size_t)nz * N;
    double* ncc = (double*)malloc(sizeof(double) * plane);
    int n = 0;
    for (int t = 0; t < F; ++t)
        for (int axis = 0; axis < 2; ++axis)
            for (int b = 0; b < S; ++b) {
                const double* Ap = A + (((size_t)t * 2 + axis) * S + b) * plane;
                or_ncc_plane(nz, N, Ap, d, sig_z, sig_l, M[t], ncc);
                int room = n < cap ? cap - n : 0;
                int m = or_peaks_plane(nz, N, Ap, ncc, M[t], alpha, ncc_min, room,
                                       out + (n < cap ? n : 0));
                for (int q = 0; q < m && q < room; ++q) {
                    out[n + q].frame = t;
                    out[n + q].axis = axis;
                    out[n + q].slab = b;
                }
                n += m;
            }
    free(ncc);
    return n;
}

/* XZ / YZ pairing (Sec. II-A4).  Readings: an XZ localisation in y-slab by at
 * lateral pixel jx belongs to sub-block (jx / P, by); a YZ localisation in
 * x-slab bx at lateral pixel jy to (bx, jy / P).  Within a frame and
 * sub-block, a pair is eligible iff |z_xz - z_yz| <= 1 pixel and the intensity
 * ratio r = I_xz / I_yz lies in [0.9, 1.11].  The cost is |ln r|, evaluated as
 * max(I)/min(I) (same order); each XZ picks its cheapest eligible YZ, each YZ
 * its cheapest eligible XZ (ties to the lower list index), and mutual choices
 * are kept.  3D position: x from XZ, y from YZ, z the mean.  Output ordered by
 * XZ index; returns the number of pairs (entries beyond cap not written). */
int or_pair3d(int n2d, const or_loc2d* L, int P, int cap, or_loc3d* out)
{
    int* best_yz = (int*)malloc(sizeof(int) * (n2d > 0 ? n2d : 1));
    int* best_xz = (int*)malloc(sizeof(int) * (n2d > 0 ? n2d : 1));
    for (int a = 0; a < n2d; ++a) {
        best_yz[a] = -1;
        best_xz[a] = -1;
    }
    for (int a = 0; a < n2d; ++a) {
        if (L[a].axis != 0) continue;
        double bestc = 0.0;
        for (int b = 0; b < n2d; ++b) {
            if (L[b].axis != 1 || L[b].frame != L[a].frame) continue;
            if (L[a].ilat / P != L[b].slab || L[b].ilat / P != L[a].slab) continue;
            if (fabs(L[a].z - L[b].z) > 1.0) continue;
            double r = L[a].amp / L[b].amp;
            if (!(r >= 0.9 && r <= 1.11)) continue;
            double c = L[a].amp > L[b].amp ? L[a].amp / L[b].amp : L[b].amp / L[a].amp;
            if (best_yz[a] < 0 || c < bestc) {
                best_yz[a] = b;
                bestc = c;
            }
        }
    }
    for (int b = 0; b < n2d; ++b) {
        if (L[b].axis != 1) continue;
        double bestc = 0.0;
        for (int a = 0; a < n2d; ++a) {
            if (L[a].axis != 0 || L[a].frame != L[b].frame) continue;
            if (L[a].ilat / P != L[b].slab || L[b].ilat / P != L[a].slab) continue;
            if (fabs(L[a].z - L[b].z) > 1.0) continue;
            double r = L[a].amp / L[b].amp;
            if (!(r >= 0.9 && r <= 1.11)) continue;
            double c = L[a].amp > L[b].amp ? L[a].amp / L[b].amp : L[b].amp / L[a].amp;
            if (best_xz[b] < 0 || c < bestc) {
                best_xz[b] = a;
                bestc = c;
            }
        }
    }
    int n = 0;
    for (int a = 0; a < n2d; ++a) {
        int b = best_yz[a];
        if (b < 0 || best_xz[b] != a) continue;
        if (n < cap) {
            out[n].frame = L[a].frame;
            out[n].i_xz = a;
            out[n].i_yz = b;
            out[n].x = L[a].lat;
            out[n].y = L[b].lat;
            out[n].z = 0.5 * (L[a].z + L[b].z);
            out[n].amp_xz = L[a].amp;
            out[n].amp_yz = L[b].amp;
        }
        ++n;
    }
    free(best_yz);
    free(best_xz);
    return n;
}

/* ------------------------------------------------------------------------ */
/* Fixed-length tracking, smoothing, rejection and accumulation (Sec. II-A6, */
/* Fig. 1f)                                                                  */
/* ------------------------------------------------------------------------ */
/* Readings (the paper names a bipartite pairing [41] and the rules, not the
 * formulas):
 *  - positions in metres: x, y lateral pixel -> (p - (N-1)/2) pitch, depth
 *    pixel -> z0 + p dz;
 *  - pairing between frames t and t+1: mutual nearest neighbours (Euclidean,
 *    within max_step; ties to the lower list index) -- a one-to-one partial
 *    matching of the bipartite graph of the two frames' localisations;
 *  - every localisation of every frame starts a search; it becomes a track
 *    when its successor chain reaches len points;
 *  - smoothing: least-squares quadratic per axis over tau = 0 .. len-1, in the
 *    orthogonal basis 1, phi1 = tau - m, phi2 = (tau - m)^2 - q, m = (len-1)/2,
 *    q = (len^2 - 1)/12;
 *  - rejection: the direction change is the angle between the first and the
 *    last smoothed segment (kept when its cosine >= cos_max_turn); the speed
 *    change is max - min of the smoothed segment lengths (kept when <=
 *    max_speed_change x their mean); a track with zero mean speed is dropped;
 *  - accumulation: the smoothed track sampled at tau = s / substeps,
 *    s = 0 .. (len-1) substeps, adds one count per sample to the voxel that
 *    holds it; the grid starts half a pixel before the first lateral pixel and
 *    the first depth row. */

static void or_track_pos(const or_geom* g, double xp, double yp, double zp, double p[3])
{
    p[0] = (xp - 0.5 * (g->n_el - 1)) * g->pitch;
    p[1] = (yp - 0.5 * (g->n_el - 1)) * g->pitch;
    p[2] = g->z0 + zp * g->dz;
}

static double or_d2(const double a[3], const double b[3])
{
    const double dx = a[0] - b[0], dy = a[1] - b[1], dz = a[2] - b[2];
    return dx * dx + dy * dy + dz * dz;
}

/* succ[i] = the localisation of frame[i] + 1 paired with i, or -1 */
void or_track_link(const or_geom* g, int n, const int* frame, const double* x, const double* y, const double* z,
                   double max_step, int* succ)
{
    int* nxt = (int*)malloc(sizeof(int) * (n > 0 ? n : 1));
    int* prv = (int*)malloc(sizeof(int) * (n > 0 ? n : 1));
    const double r2 = max_step * max_step;
    for (int i = 0; i < n; ++i) {
        double pi[3], pj[3], best = 0.0;
        or_track_pos(g, x[i], y[i], z[i], pi);
        nxt[i] = -1;
        prv[i] = -1;
        for (int j = 0; j < n; ++j) {
            if (frame[j] != frame[i] + 1) continue;
            or_track_pos(g, x[j], y[j], z[j], pj);
            const double d2 = or_d2(pi, pj);
            if (d2 <= r2 && (nxt[i] < 0 || d2 < best)) {
                nxt[i] = j;
                best = d2;
            }
        }
        best = 0.0;
        for (int j = 0; j < n; ++j) {
            if (frame[j] != frame[i] - 1) continue;
            or_track_pos(g, x[j], y[j], z[j], pj);
            const double d2 = or_d2(pi, pj);
            if (d2 <= r2 && (prv[i] < 0 || d2 < best)) {
                prv[i] = j;
                best = d2;
            }
        }
    }
    for (int i = 0; i < n; ++i) succ[i] = (nxt[i] >= 0 && prv[nxt[i]] == i) ? nxt[i] : -1;
    free(nxt);
    free(prv);
}

/* Tracks in list order of their first point; returns the count (entries
 * beyond cap are counted, not written). */
int or_track_build(const or_geom* g, int n, const int* frame, const double* x, const double* y, const double* z,
                   const int* succ, const or_track_params* prm, int cap, or_track* out)
{
    const int L = prm->len;
    const double m = 0.5 * (double)(L - 1), q = ((double)L * (double)L - 1.0) / 12.0;
    /* sums of phi1^2 and phi2^2 over tau = 0 .. L-1 */
    double n1 = 0.0, n2 = 0.0;
    for (int t = 0; t < L; ++t) {
        const double f1 = (double)t - m, f2 = f1 * f1 - q;
        n1 += f1 * f1;
        n2 += f2 * f2;
    }
    int* idx = (int*)malloc(sizeof(int) * (L > 0 ? L : 1));
    int cnt = 0;
    for (int i = 0; i < n; ++i) {
        idx[0] = i;
        int ok = 1;
        for (int s = 1; s < L && ok; ++s) {
            idx[s] = succ[idx[s - 1]];
            ok = idx[s] >= 0;
        }
        if (!ok) continue;
        or_track tr;
        tr.first = i;
        tr.frame0 = frame[i];
        for (int ax = 0; ax < 3; ++ax) {
            double s0 = 0.0, s1 = 0.0, s2 = 0.0;
            for (int t = 0; t < L; ++t) {
                double p[3];
                or_track_pos(g, x[idx[t]], y[idx[t]], z[idx[t]], p);
                const double f1 = (double)t - m, f2 = f1 * f1 - q;
                s0 += p[ax];
                s1 += p[ax] * f1;
                s2 += p[ax] * f2;
            }
            tr.a[ax][0] = s0 / (double)L;
            tr.a[ax][1] = s1 / n1;
            tr.a[ax][2] = s2 / n2;
        }
        /* smoothed segment s -> s+1: a1 + a2 (phi2(s+1) - phi2(s)) = a1 + a2 (2 (s - m) + 1) */
        double vfirst[3] = {0.0, 0.0, 0.0}, vlast[3] = {0.0, 0.0, 0.0}, sum = 0.0, vmax = 0.0, vmin = 0.0;
        for (int s = 0; s + 1 < L; ++s) {
            double v[3];
            const double dphi2 = 2.0 * ((double)s - m) + 1.0;
            for (int ax = 0; ax < 3; ++ax) v[ax] = tr.a[ax][1] + tr.a[ax][2] * dphi2;
            const double sp = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
            sum += sp;
            if (s == 0 || sp > vmax) vmax = sp;
            if (s == 0 || sp < vmin) vmin = sp;
            if (s == 0)
                for (int ax = 0; ax < 3; ++ax) vfirst[ax] = v[ax];
            if (s + 2 == L)
                for (int ax = 0; ax < 3; ++ax) vlast[ax] = v[ax];
        }
        tr.mean_speed = sum / (double)(L - 1);
        tr.speed_range = vmax - vmin;
        const double nf = sqrt(vfirst[0] * vfirst[0] + vfirst[1] * vfirst[1] + vfirst[2] * vfirst[2]);
        const double nl = sqrt(vlast[0] * vlast[0] + vlast[1] * vlast[1] + vlast[2] * vlast[2]);
        const double dot = vfirst[0] * vlast[0] + vfirst[1] * vlast[1] + vfirst[2] * vlast[2];
        tr.cos_turn = (nf > 0.0 && nl > 0.0) ? dot / (nf * nl) : -2.0;
        tr.accepted = tr.mean_speed > 0.0 && tr.cos_turn >= prm->cos_max_turn &&
                      tr.speed_range <= prm->max_speed_change * tr.mean_speed;
        if (cnt < cap) out[cnt] = tr;
        ++cnt;
    }
    free(idx);
    return cnt;
}

/* density grid [nz_v][ny_v][nx_v] covering the lateral pixels and the depth rows */
void or_track_grid(const or_geom* g, double voxel, int dims[3])
{
    dims[0] = (int)ceil((double)g->n_el * g->pitch / voxel);
    dims[1] = dims[0];
    dims[2] = (int)ceil((double)g->nz * g->dz / voxel);
}

void or_track_accumulate(const or_geom* g, int ntr, const or_track* tr, const or_track_params* prm,
                         unsigned* grid)
{
    int dims[3];
    or_track_grid(g, prm->voxel, dims);
    const int L = prm->len;
    const double m = 0.5 * (double)(L - 1), q = ((double)L * (double)L - 1.0) / 12.0;
    const double lo[3] = {-0.5 * (double)g->n_el * g->pitch, -0.5 * (double)g->n_el * g->pitch,
                          g->z0 - 0.5 * g->dz};
    for (int k = 0; k < ntr; ++k) {
        if (!tr[k].accepted) continue;
        for (int s = 0; s <= (L - 1) * prm->substeps; ++s) {
            const double tau = (double)s / (double)prm->substeps;
            const double f1 = tau - m, f2 = f1 * f1 - q;
            int iv[3], inside = 1;
            for (int ax = 0; ax < 3; ++ax) {
                const double p = tr[k].a[ax][0] + tr[k].a[ax][1] * f1 + tr[k].a[ax][2] * f2;
                const double c = floor((p - lo[ax]) / prm->voxel);
                inside = inside && c >= 0.0 && c < (double)dims[ax];
                iv[ax] = inside ? (int)c : 0;
            }
            if (inside) grid[((size_t)iv[2] * dims[1] + iv[1]) * dims[0] + iv[0]] += 1u;
        }
    }
}

/* Velocity volumes (Sec. II-C: density and velocity volumes on the 50 um grid):
 * at every accumulation sample of an accepted track (the samples and voxels of
 * or_track_accumulate) the smoothed track's velocity is the derivative of its
 * quadratic, v = a1 + 2 a2 phi1(tau) per axis (metres per frame interval).  The
 * voxel adds the speed |v| and the axial component v_z (positive = deeper),
 * each rounded to a whole nanometre per frame interval, to two integer sums;
 * mean values are the sums over the density count (times the frame rate for
 * metres per second). */
void or_track_velocity(const or_geom* g, int ntr, const or_track* tr, const or_track_params* prm,
                       long long* speed_sum, long long* vz_sum)
{
    int dims[3];
    or_track_grid(g, prm->voxel, dims);
    const int L = prm->len;
    const double m = 0.5 * (double)(L - 1), q = ((double)L * (double)L - 1.0) / 12.0;
    const double lo[3] = {-0.5 * (double)g->n_el * g->pitch, -0.5 * (double)g->n_el * g->pitch,
                          g->z0 - 0.5 * g->dz};
    for (int k = 0; k < ntr; ++k) {
        if (!tr[k].accepted) continue;
        for (int s = 0; s <= (L - 1) * prm->substeps; ++s) {
            const double tau = (double)s / (double)prm->substeps;
            const double f1 = tau - m, f2 = f1 * f1 - q;
            int iv[3], inside = 1;
            double v[3];
            for (int ax = 0; ax < 3; ++ax) {
                const double p = tr[k].a[ax][0] + tr[k].a[ax][1] * f1 + tr[k].a[ax][2] * f2;
                const double c = floor((p - lo[ax]) / prm->voxel);
                inside = inside && c >= 0.0 && c < (double)dims[ax];
                iv[ax] = inside ? (int)c : 0;
                v[ax] = tr[k].a[ax][1] + 2.0 * tr[k].a[ax][2] * f1;
            }
            if (inside) {
                const size_t at = ((size_t)iv[2] * dims[1] + iv[1]) * dims[0] + iv[0];
                const double sp = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
                speed_sum[at] += llrint(sp * 1e9);
                vz_sum[at] += llrint(v[2] * 1e9);
            }
        }
    }
}

/* Thread count of the OpenMP loops above (timing of the CPU baseline with one
 * thread and with all cores); no arithmetic. */
void or_set_threads(int n) { omp_set_num_threads(n > 0 ? n : 1); }
int or_max_threads(void) { return omp_get_max_threads(); }
