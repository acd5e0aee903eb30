// api.cu -- host side of the librca C ABI (argument checks, workspace,
// launches).  Every entry point validates on the host before enqueuing.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "rca_internal.cuh"

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
rca_status set_error(rca_handle* h, rca_status s, const char* fmt, ...)
{
    if (h) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        h->last_error = buf;
    }
    return s;
}

rca_status cuda_check(rca_handle* h, cudaError_t e, const char* what)
{
    if (e == cudaSuccess) return RCA_OK;
    return set_error(h, RCA_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

static bool capturing(rca_handle* h)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(h->stream, &cs);
    return cs != cudaStreamCaptureStatusNone;
}

void* ws_get(rca_handle* h, WsSlot slot, size_t bytes, rca_status* st)
{
    WsBuf& b = h->ws[slot];
    if (b.bytes >= bytes && b.p) return b.p;
    if (capturing(h)) {
        *st = set_error(h, RCA_ERR_CAPACITY, "workspace slot %d needs %zu bytes during stream capture; call rca_reserve first",
                        (int)slot, bytes);
        return nullptr;
    }
    if (b.p) {
        cudaStreamSynchronize(h->stream);
        cudaFree(b.p);
        b.p = nullptr;
        b.bytes = 0;
    }
    size_t want = bytes + bytes / 8 + 256;
    cudaError_t e = cudaMalloc(&b.p, want);
    if (e != cudaSuccess) {
        b.p = nullptr;
        *st = cuda_check(h, e, "workspace cudaMalloc");
        return nullptr;
    }
    b.bytes = want;
    return b.p;
}

size_t dtype_size(rca_dtype t)
{
    switch (t) {
    case RCA_F32: return 4;
    case RCA_I16: return 2;
    case RCA_F16: return 2;
    case RCA_C32: return 8;
    case RCA_C16F: return 4;
    case RCA_C16BF: return 4;
    }
    return 0;
}

static bool is_complex(int t) { return t == RCA_C32 || t == RCA_C16F || t == RCA_C16BF; }
static bool is_real_rf(int t) { return t == RCA_F32 || t == RCA_F16 || t == RCA_I16; }

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

#define CHECK_HANDLE(h)                                                                                     \
    do {                                                                                                     \
        if (!(h)) return RCA_ERR_INVALID_ARG;                                                                \
    } while (0)

// ---------------------------------------------------------------------------
// handle
// ---------------------------------------------------------------------------
extern "C" int rca_version(void) { return (RCA_VERSION_MAJOR << 16) | RCA_VERSION_MINOR; }

extern "C" const char* rca_status_string(rca_status s)
{
    switch (s) {
    case RCA_OK: return "ok";
    case RCA_ERR_INVALID_ARG: return "invalid argument";
    case RCA_ERR_SHAPE: return "shape mismatch";
    case RCA_ERR_UNSUPPORTED: return "unsupported";
    case RCA_ERR_CUDA: return "CUDA error";
    case RCA_ERR_CAPACITY: return "output capacity exceeded";
    case RCA_ERR_TIMEOUT: return "bounded wait timed out";
    case RCA_ERR_BOUNDS: return "index out of bounds";
    }
    return "unknown status";
}

extern "C" rca_status rca_create(rca_handle** out, int device)
{
    if (!out) return RCA_ERR_INVALID_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return RCA_ERR_CUDA;
    rca_handle* h = new (std::nothrow) rca_handle();
    if (!h) return RCA_ERR_CUDA;
    h->device = device;
    DeviceGuard dg(device);
    if (cudaMalloc(&h->d_status, sizeof(unsigned)) != cudaSuccess || cudaMemset(h->d_status, 0, sizeof(unsigned)) != cudaSuccess) {
        delete h;
        return RCA_ERR_CUDA;
    }
    *out = h;
    return RCA_OK;
}

extern "C" rca_status rca_destroy(rca_handle* h)
{
    CHECK_HANDLE(h);
    DeviceGuard dg(h->device);
    cudaStreamSynchronize(h->stream);
    for (auto& b : h->ws)
        if (b.p) cudaFree(b.p);
    cudaFree(h->d_status);
    delete h;
    return RCA_OK;
}

extern "C" rca_status rca_set_stream(rca_handle* h, void* stream)
{
    CHECK_HANDLE(h);
    h->stream = (cudaStream_t)stream;
    return RCA_OK;
}

extern "C" const char* rca_last_error(const rca_handle* h) { return h ? h->last_error.c_str() : "null handle"; }

extern "C" rca_status rca_sync_status(rca_handle* h, rca_status* dev)
{
    CHECK_HANDLE(h);
    DeviceGuard dg(h->device);
    if (dev) *dev = RCA_OK;
    rca_status st = cuda_check(h, cudaStreamSynchronize(h->stream), "stream synchronize");
    if (st != RCA_OK) return st;
    unsigned w = 0;
    st = cuda_check(h, cudaMemcpy(&w, h->d_status, sizeof w, cudaMemcpyDeviceToHost), "status read");
    if (st != RCA_OK) return st;
    st = cuda_check(h, cudaMemset(h->d_status, 0, sizeof(unsigned)), "status clear");
    if (dev) {
        if (w & ST_BOUNDS) *dev = RCA_ERR_BOUNDS;
        else if (w & ST_TIMEOUT) *dev = RCA_ERR_TIMEOUT;
        else if (w & ST_CAPACITY) *dev = RCA_ERR_CAPACITY;
    }
    return st;
}

// ---------------------------------------------------------------------------
// geometry and tables
// ---------------------------------------------------------------------------
extern "C" rca_status rca_geometry_create(rca_handle* h, const rca_geometry_desc* d, rca_geometry** out)
{
    CHECK_HANDLE(h);
    if (!d || !out) return set_error(h, RCA_ERR_INVALID_ARG, "null descriptor or output");
    *out = nullptr;
    if (d->n_el <= 0 || d->nz <= 1 || d->ns <= 1 || d->P <= 0 || d->K <= 0 || d->us <= 0)
        return set_error(h, RCA_ERR_INVALID_ARG, "sizes must be positive (nz, ns > 1)");
    if (d->K > RCA_MAX_K) return set_error(h, RCA_ERR_UNSUPPORTED, "K = %d > %d transmissions per family", d->K, RCA_MAX_K);
    if (d->us > 8) return set_error(h, RCA_ERR_UNSUPPORTED, "us = %d > 8", d->us);
    if (d->n_el % d->P != 0) return set_error(h, RCA_ERR_INVALID_ARG, "n_el %% P != 0");
    if (d->n_el > 256) return set_error(h, RCA_ERR_UNSUPPORTED, "n_el > 256");
    if (d->n_el % 4 != 0) return set_error(h, RCA_ERR_UNSUPPORTED, "n_el must be a multiple of 4 (16-byte sample rows)");
    if ((long)d->ns * 65536L >= (1L << 31)) return set_error(h, RCA_ERR_UNSUPPORTED, "ns too large for Q16 delays");
    if (!(d->pitch_m > 0) || !(d->fc_hz > 0) || !(d->fs_hz > 0) || !(d->c_mps > 0) || !(d->dz_m > 0) || !(d->fnum > 0) ||
        !(d->z0_m > 0))
        return set_error(h, RCA_ERR_INVALID_ARG, "physical parameters must be positive");
    if (!d->ang_rc_rad || !d->ang_cr_rad) return set_error(h, RCA_ERR_INVALID_ARG, "null angle arrays");
    rca_geometry* g = new (std::nothrow) rca_geometry();
    if (!g) return set_error(h, RCA_ERR_CUDA, "out of host memory");
    g->desc = *d;
    g->ang.assign(d->ang_rc_rad, d->ang_rc_rad + d->K);
    g->ang.insert(g->ang.end(), d->ang_cr_rad, d->ang_cr_rad + d->K);
    g->desc.ang_rc_rad = g->ang.data();
    g->desc.ang_cr_rad = g->ang.data() + d->K;
    GeomDev& gd = g->gd;
    gd.N = d->n_el;
    gd.nz = d->nz;
    gd.us = d->us;
    gd.nzs = (d->nz - 1) * d->us + 1;
    gd.ns = d->ns;
    gd.P = d->P;
    gd.S = d->n_el / d->P;
    gd.K = d->K;
    gd.pitch = d->pitch_m;
    gd.fc = d->fc_hz;
    gd.fs = d->fs_hz;
    gd.c = d->c_mps;
    gd.z0 = d->z0_m;
    gd.dz = d->dz_m;
    gd.fnum = d->fnum;
    gd.t0 = 2.0 * d->z0_m / d->c_mps;
    gd.L = (double)d->n_el * d->pitch_m;
    for (int k = 0; k < 2 * d->K; ++k) {
        double a = g->ang[k];
        if (!(std::fabs(a) < 1.4)) {
            delete g;
            return set_error(h, RCA_ERR_INVALID_ARG, "steering angle %d out of range", k);
        }
        gd.sin_th[k] = std::sin(a);
        gd.cos_th[k] = std::cos(a);
    }
    *out = g;
    return RCA_OK;
}

extern "C" rca_status rca_geometry_destroy(rca_geometry* g)
{
    delete g;
    return RCA_OK;
}

static void free_tables(rca_tables* t)
{
    void* ptrs[] = {t->tx_f64, t->rx_f64, t->tx_q16, t->rx_q16, t->W, t->dmax, t->s2_shift, t->s2_sfl,
                    t->s2_sfr, t->s2_psi, t->s2_ec, t->s2_coef, t->s2_tmin, t->s2_c2, t->s2_rot, t->s2_c2r,
                    t->s2_coefr, t->s2_lw, t->dtx_q16, t->dtx_ph, t->mix,
                    t->s1.d_chunks, t->s1.d_rec32, t->s1.d_rec16};
    for (void* p : ptrs)
        if (p) cudaFree(p);
}

extern "C" rca_status rca_delay_tables(rca_handle* h, const rca_geometry* g, rca_tables** out)
{
    CHECK_HANDLE(h);
    if (!g || !out) return set_error(h, RCA_ERR_INVALID_ARG, "null geometry or output");
    *out = nullptr;
    if (capturing(h)) return set_error(h, RCA_ERR_INVALID_ARG, "rca_delay_tables cannot run during stream capture");
    DeviceGuard dg(h->device);
    rca_tables* t = new (std::nothrow) rca_tables();
    if (!t) return set_error(h, RCA_ERR_CUDA, "out of host memory");
    t->h = h;
    t->gd = g->gd;
    rca_status st = launch_tables(h, t);
    if (st != RCA_OK) {
        free_tables(t);
        delete t;
        return st;
    }
    *out = t;
    return RCA_OK;
}

extern "C" rca_status rca_tables_destroy(rca_tables* t)
{
    if (!t) return RCA_ERR_INVALID_ARG;
    DeviceGuard dg(t->h->device);
    cudaStreamSynchronize(t->h->stream);
    free_tables(t);
    delete t;
    return RCA_OK;
}

static rca_status table_info(const rca_tables* t, int id, const void** ptr, size_t* bytes, int dims[4])
{
    const GeomDev& g = t->gd;
    const int nt = 2 * g.K;
    int d[4] = {0, 0, 0, 0};
    size_t es = 0;
    const void* p = nullptr;
    switch (id) {
    case RCA_TAB_TX_F64: p = t->tx_f64; es = 8; d[0] = nt; d[1] = g.nzs; break;
    case RCA_TAB_RX_F64: p = t->rx_f64; es = 8; d[0] = g.N; d[1] = g.nzs; break;
    case RCA_TAB_TX_Q16: p = t->tx_q16; es = 4; d[0] = nt; d[1] = g.nzs; break;
    case RCA_TAB_RX_Q16: p = t->rx_q16; es = 4; d[0] = g.nzs; d[1] = g.N; break;
    case RCA_TAB_W: p = t->W; es = 8; d[0] = g.nzs; d[1] = g.N; break;
    case RCA_TAB_DMAX: p = t->dmax; es = 4; d[0] = g.nzs; break;
    case RCA_TAB_S2_SHIFT: p = t->s2_shift; es = 8; d[0] = nt; d[1] = g.N; break;
    case RCA_TAB_S2_PSI: p = t->s2_psi; es = 8; d[0] = nt; d[1] = g.N; break;
    case RCA_TAB_S2_EC: p = t->s2_ec; es = 8; d[0] = nt; d[1] = g.nz; break;
    case RCA_TAB_S2_COEF: p = t->s2_coef; es = 8; d[0] = nt; d[1] = g.S; d[2] = g.nz; d[3] = t->T; break;
    case RCA_TAB_S2_TMIN: p = t->s2_tmin; es = 4; d[0] = nt; d[1] = g.S; break;
    default: return RCA_ERR_INVALID_ARG;
    }
    size_t n = 1;
    for (int q = 0; q < 4; ++q)
        if (d[q]) n *= (size_t)d[q];
    if (ptr) *ptr = p;
    if (bytes) *bytes = n * es;
    if (dims)
        for (int q = 0; q < 4; ++q) dims[q] = d[q];
    return RCA_OK;
}

extern "C" rca_status rca_tables_query(const rca_tables* t, int id, size_t* bytes, int dims[4])
{
    if (!t) return RCA_ERR_INVALID_ARG;
    return table_info(t, id, nullptr, bytes, dims);
}

extern "C" rca_status rca_tables_download(const rca_tables* t, int id, void* dst, size_t bytes)
{
    if (!t || !dst) return RCA_ERR_INVALID_ARG;
    const void* p = nullptr;
    size_t need = 0;
    rca_status st = table_info(t, id, &p, &need, nullptr);
    if (st != RCA_OK) return set_error(t->h, st, "unknown table id %d", id);
    if (bytes < need) return set_error(t->h, RCA_ERR_SHAPE, "table %d needs %zu bytes, got %zu", id, need, bytes);
    DeviceGuard dg(t->h->device);
    st = cuda_check(t->h, cudaStreamSynchronize(t->h->stream), "sync before download");
    if (st != RCA_OK) return st;
    return cuda_check(t->h, cudaMemcpy(dst, p, need, cudaMemcpyDeviceToHost), "table download");
}

extern "C" rca_status rca_reserve(rca_handle* h, const rca_geometry* g, int F)
{
    CHECK_HANDLE(h);
    if (!g || F <= 0) return set_error(h, RCA_ERR_INVALID_ARG, "null geometry or F <= 0");
    DeviceGuard dg(h->device);
    const GeomDev& gd = g->gd;
    const size_t nt = 2 * gd.K;
    rca_status st = RCA_OK;
    const int nstrip = (gd.nz + NCC_RS - 1) / NCC_RS;
    const size_t nslots = (size_t)F * 2 * gd.S * nstrip;
    struct {
        WsSlot s;
        size_t b;
    } want[] = {
        {WS_MEAN, nt * gd.N * gd.ns * sizeof(float)},
        {WS_IQ, (size_t)F * nt * gd.N * gd.ns * sizeof(float2)},
        {WS_SLICES, (size_t)F * nt * gd.nzs * gd.N * sizeof(float2)},
        {WS_A, (size_t)F * 2 * gd.S * gd.nz * gd.N * sizeof(float)},
        {WS_M, (size_t)F * sizeof(float)},
        {WS_CAND, nslots * CAND_CAP * sizeof(ulm_loc2d)},
        {WS_CANDCNT, nslots * sizeof(int)},
        {WS_SCAN, (nslots + 1) * sizeof(int)},
        {WS_PLANEOFF, ((size_t)F * 2 * gd.S + 1) * sizeof(int)},
    };
    for (auto& w : want)
        if (!ws_get(h, w.s, w.b, &st)) return st;
    return cuda_check(h, cudaStreamSynchronize(h->stream), "reserve");
}

// ---------------------------------------------------------------------------
// beamforming
// ---------------------------------------------------------------------------
static rca_status check_tables(rca_handle* h, const rca_tables* t, int F)
{
    if (!t) return set_error(h, RCA_ERR_INVALID_ARG, "null tables");
    if (t->h->device != h->device) return set_error(h, RCA_ERR_INVALID_ARG, "tables belong to another device");
    if (F <= 0) return set_error(h, RCA_ERR_SHAPE, "n_frames must be positive");
    return RCA_OK;
}

extern "C" rca_status rca_ingest(rca_handle* h, const rca_tables* t, const void* rf, rca_dtype rf_t, const float* scale,
                                 int F, int clutter, void* iq, rca_dtype iq_t)
{
    CHECK_HANDLE(h);
    rca_status st = check_tables(h, t, F);
    if (st != RCA_OK) return st;
    if (!rf || !iq) return set_error(h, RCA_ERR_INVALID_ARG, "null rf or iq");
    if (!is_real_rf(rf_t)) return set_error(h, RCA_ERR_UNSUPPORTED, "rf dtype must be F32, F16 or I16");
    if (rf_t == RCA_I16 && !scale) return set_error(h, RCA_ERR_INVALID_ARG, "int16 rf needs a scale array");
    if (!is_complex(iq_t)) return set_error(h, RCA_ERR_UNSUPPORTED, "iq dtype must be C32, C16F or C16BF");
    if (clutter != RCA_CLUTTER_NONE && clutter != RCA_CLUTTER_MEAN) return set_error(h, RCA_ERR_INVALID_ARG, "bad clutter mode");
    DeviceGuard dg(h->device);
    return launch_ingest(h, t, rf, rf_t, scale, F, clutter, iq, iq_t);
}

extern "C" rca_status rca_stage1(rca_handle* h, const rca_tables* t, const void* iq, rca_dtype iq_t, int F, void* slices)
{
    CHECK_HANDLE(h);
    rca_status st = check_tables(h, t, F);
    if (st != RCA_OK) return st;
    if (!iq || !slices) return set_error(h, RCA_ERR_INVALID_ARG, "null iq or slices");
    if (!is_complex(iq_t)) return set_error(h, RCA_ERR_UNSUPPORTED, "iq dtype must be C32, C16F or C16BF");
    if (reinterpret_cast<uintptr_t>(iq) % 16 != 0) return set_error(h, RCA_ERR_INVALID_ARG, "iq must be 16-byte aligned");
    DeviceGuard dg(h->device);
    return launch_stage1(h, t, iq, iq_t, F, (float2*)slices);
}

extern "C" rca_status rca_stage2_project(rca_handle* h, const rca_tables* t, const void* slices, int F, void* planes,
                                         rca_dtype pt)
{
    CHECK_HANDLE(h);
    rca_status st = check_tables(h, t, F);
    if (st != RCA_OK) return st;
    if (!slices || !planes) return set_error(h, RCA_ERR_INVALID_ARG, "null slices or planes");
    if (!is_complex(pt)) return set_error(h, RCA_ERR_UNSUPPORTED, "planes dtype must be C32, C16F or C16BF");
    DeviceGuard dg(h->device);
    return launch_stage2(h, t, (const float2*)slices, F, planes, pt);
}

extern "C" rca_status rca_direct_project(rca_handle* h, const rca_tables* t, const void* iq, rca_dtype iq_t, int F,
                                         void* planes, rca_dtype pt)
{
    CHECK_HANDLE(h);
    rca_status st = check_tables(h, t, F);
    if (st != RCA_OK) return st;
    if (!iq || !planes) return set_error(h, RCA_ERR_INVALID_ARG, "null iq or planes");
    if (!is_complex(iq_t) || !is_complex(pt)) return set_error(h, RCA_ERR_UNSUPPORTED, "complex dtypes required");
    DeviceGuard dg(h->device);
    return launch_direct(h, t, iq, iq_t, F, planes, pt);
}

extern "C" rca_status rca_beamform_projections(rca_handle* h, const rca_tables* t, const void* rf, rca_dtype rf_t,
                                               const float* scale, int F, const rca_bf_params* prm, void* planes,
                                               rca_dtype pt)
{
    CHECK_HANDLE(h);
    rca_status st = check_tables(h, t, F);
    if (st != RCA_OK) return st;
    if (!rf || !planes || !prm) return set_error(h, RCA_ERR_INVALID_ARG, "null rf, planes or params");
    if (prm->mode != RCA_MODE_TWO_STAGE && prm->mode != RCA_MODE_DIRECT) return set_error(h, RCA_ERR_INVALID_ARG, "bad mode");
    if (!is_real_rf(rf_t)) return set_error(h, RCA_ERR_UNSUPPORTED, "rf dtype must be F32, F16 or I16");
    if (rf_t == RCA_I16 && !scale) return set_error(h, RCA_ERR_INVALID_ARG, "int16 rf needs a scale array");
    if (!is_complex(prm->iq_dtype) || !is_complex(pt)) return set_error(h, RCA_ERR_UNSUPPORTED, "complex dtypes required");
    if (prm->clutter != RCA_CLUTTER_NONE && prm->clutter != RCA_CLUTTER_MEAN && prm->clutter != RCA_CLUTTER_SVD)
        return set_error(h, RCA_ERR_INVALID_ARG, "bad clutter mode");
    const bool svd = prm->clutter == RCA_CLUTTER_SVD;
    if (svd && prm->mode != RCA_MODE_TWO_STAGE)
        return set_error(h, RCA_ERR_INVALID_ARG, "the SVD clutter filter acts on Stage-1 slices (TWO_STAGE only)");
    if (svd && (prm->svd_rank < 0 || prm->svd_rank > 32 || prm->svd_rank >= F || prm->svd_iterations < 0 ||
                prm->svd_iterations > 1000))
        return set_error(h, RCA_ERR_INVALID_ARG, "SVD rank %d / iterations %d out of range", prm->svd_rank,
                         prm->svd_iterations);
    DeviceGuard dg(h->device);
    const GeomDev& g = t->gd;
    const rca_dtype iq_t = (rca_dtype)prm->iq_dtype;
    void* iq = ws_get(h, WS_IQ, (size_t)F * 2 * g.K * g.N * g.ns * dtype_size(iq_t), &st);
    if (!iq) return st;
    if ((st = launch_ingest(h, t, rf, rf_t, scale, F, svd ? RCA_CLUTTER_NONE : prm->clutter, iq, iq_t)) != RCA_OK)
        return st;
    if (prm->mode == RCA_MODE_DIRECT) return launch_direct(h, t, iq, iq_t, F, planes, pt);
    float2* slices = (float2*)ws_get(h, WS_SLICES, (size_t)F * 2 * g.K * g.nzs * g.N * sizeof(float2), &st);
    if (!slices) return st;
    if ((st = launch_stage1(h, t, iq, iq_t, F, slices)) != RCA_OK) return st;
    if (svd && (st = launch_clutter_svd(h, t, slices, F, prm->svd_rank,
                                        prm->svd_iterations > 0 ? prm->svd_iterations : 30, nullptr)) != RCA_OK)
        return st;
    return launch_stage2(h, t, slices, F, planes, pt);
}

// ---------------------------------------------------------------------------
// localisation
// ---------------------------------------------------------------------------
static rca_status check_ulm(rca_handle* h, const ulm_params* p)
{
    if (!p) return set_error(h, RCA_ERR_INVALID_ARG, "null ulm_params");
    if (p->d < 3 || p->d > RCA_MAX_NCC_D || p->d % 2 == 0) return set_error(h, RCA_ERR_INVALID_ARG, "d must be odd in [3, 15]");
    if (!(p->sig_z > 0) || !(p->sig_lat > 0)) return set_error(h, RCA_ERR_INVALID_ARG, "PSF sigmas must be positive");
    if (!(p->alpha >= 0) || !(p->ncc_min > -1.0f)) return set_error(h, RCA_ERR_INVALID_ARG, "bad thresholds");
    if (p->enh != ULM_ENH_XDOPPLER && p->enh != ULM_ENH_COHERENT) return set_error(h, RCA_ERR_INVALID_ARG, "bad enhancement mode");
    return RCA_OK;
}

extern "C" rca_status ulm_enhance(rca_handle* h, const rca_tables* t, const void* planes, rca_dtype pt, int F, int enh,
                                  float* A, float* M)
{
    CHECK_HANDLE(h);
    rca_status st = check_tables(h, t, F);
    if (st != RCA_OK) return st;
    if (!planes || !A || !M) return set_error(h, RCA_ERR_INVALID_ARG, "null planes, A or M");
    if (!is_complex(pt)) return set_error(h, RCA_ERR_UNSUPPORTED, "planes dtype must be C32, C16F or C16BF");
    DeviceGuard dg(h->device);
    return launch_enhance(h, t, planes, pt, F, enh, A, M);
}

extern "C" rca_status ulm_detect2d(rca_handle* h, const rca_tables* t, const float* A, const float* M, int F,
                                   const ulm_params* prm, ulm_loc2d* out, int cap, int* n2d, float* ncc_out,
                                   int* plane_off)
{
    CHECK_HANDLE(h);
    rca_status st = check_tables(h, t, F);
    if (st != RCA_OK) return st;
    if ((st = check_ulm(h, prm)) != RCA_OK) return st;
    if (!A || !M || !n2d || (cap > 0 && !out) || cap < 0) return set_error(h, RCA_ERR_INVALID_ARG, "null A, M, list or count");
    if (t->gd.N < prm->d || t->gd.nz < prm->d) return set_error(h, RCA_ERR_SHAPE, "plane smaller than the NCC kernel");
    DeviceGuard dg(h->device);
    return launch_detect2d(h, t, A, M, F, prm, out, cap, n2d, ncc_out, plane_off);
}

extern "C" rca_status ulm_pair3d(rca_handle* h, const rca_tables* t, const ulm_loc2d* L, const int* n2d, int cap2d, int F,
                                 ulm_loc3d* out, int cap3d, int* n3d)
{
    CHECK_HANDLE(h);
    rca_status st = check_tables(h, t, F);
    if (st != RCA_OK) return st;
    if (!n2d || !n3d || cap2d < 0 || cap3d < 0 || (cap2d > 0 && !L) || (cap3d > 0 && !out))
        return set_error(h, RCA_ERR_INVALID_ARG, "null list or count");
    DeviceGuard dg(h->device);
    return launch_pair3d(h, t, L, n2d, cap2d, F, out, cap3d, n3d);
}

extern "C" rca_status ulm_pair3d_noalloc(rca_handle* h, const rca_tables* t, const ulm_loc2d* L, const int* n2d,
                                         int cap2d, int F, ulm_loc3d* out, int cap3d, int* n3d)
{
    CHECK_HANDLE(h);
    rca_status st = check_tables(h, t, F);
    if (st != RCA_OK) return st;
    if (!n2d || !n3d || cap2d < 0 || cap3d < 0 || (cap2d > 0 && !L) || (cap3d > 0 && !out))
        return set_error(h, RCA_ERR_INVALID_ARG, "null list or count");
    DeviceGuard dg(h->device);
    return launch_pair3d_noalloc(h, t, L, n2d, cap2d, F, out, cap3d, n3d);
}

extern "C" rca_status rca_clutter_svd(rca_handle* h, const rca_tables* t, void* slices, int F, int rank,
                                      int iterations)
{
    CHECK_HANDLE(h);
    rca_status st = check_tables(h, t, F);
    if (st != RCA_OK) return st;
    if (!slices) return set_error(h, RCA_ERR_INVALID_ARG, "null slices");
    if (F > 65535) return set_error(h, RCA_ERR_UNSUPPORTED, "more than 65535 frames in one call");
    DeviceGuard dg(h->device);
    return launch_clutter_svd(h, t, (float2*)slices, F, rank, iterations, nullptr);
}

extern "C" rca_status rca_clutter_svd_info(rca_handle* h, const rca_tables* t, void* slices, int F, int rank,
                                           int iterations, float* info)
{
    CHECK_HANDLE(h);
    rca_status st = check_tables(h, t, F);
    if (st != RCA_OK) return st;
    if (!slices || !info) return set_error(h, RCA_ERR_INVALID_ARG, "null slices or info");
    if (F > 65535) return set_error(h, RCA_ERR_UNSUPPORTED, "more than 65535 frames in one call");
    DeviceGuard dg(h->device);
    return launch_clutter_svd(h, t, (float2*)slices, F, rank, iterations, info);
}

extern "C" rca_status rca_motion_estimate(rca_handle* h, const rca_tables* t, const void* slices, int F,
                                          float* motion, float* shifts, int* peaks)
{
    CHECK_HANDLE(h);
    rca_status st = check_tables(h, t, F);
    if (st != RCA_OK) return st;
    if (!slices || !motion) return set_error(h, RCA_ERR_INVALID_ARG, "null slices or motion");
    if (F > 65535) return set_error(h, RCA_ERR_UNSUPPORTED, "more than 65535 frames in one call");
    DeviceGuard dg(h->device);
    return launch_motion(h, t, (const float2*)slices, F, motion, shifts, peaks);
}

extern "C" rca_status ulm_separate(rca_handle* h, const rca_tables* t, const void* planes, rca_dtype pt, int F,
                                   const ulm_sep_params* prm, void* subsets)
{
    CHECK_HANDLE(h);
    rca_status st = check_tables(h, t, F);
    if (st != RCA_OK) return st;
    if (!planes || !prm || !subsets) return set_error(h, RCA_ERR_INVALID_ARG, "null planes, parameters or subsets");
    if (!is_complex(pt)) return set_error(h, RCA_ERR_UNSUPPORTED, "planes dtype must be C32, C16F or C16BF");
    DeviceGuard dg(h->device);
    return launch_separate(h, t, planes, pt, F, prm, ULM_ENH_XDOPPLER, (float2*)subsets, nullptr, nullptr);
}

extern "C" rca_status ulm_separate_enhance(rca_handle* h, const rca_tables* t, const void* planes, rca_dtype pt, int F,
                                           const ulm_sep_params* prm, int enh, float* A, float* M)
{
    CHECK_HANDLE(h);
    rca_status st = check_tables(h, t, F);
    if (st != RCA_OK) return st;
    if (!planes || !prm || !A || !M) return set_error(h, RCA_ERR_INVALID_ARG, "null planes, parameters, A or M");
    if (!is_complex(pt)) return set_error(h, RCA_ERR_UNSUPPORTED, "planes dtype must be C32, C16F or C16BF");
    DeviceGuard dg(h->device);
    return launch_separate(h, t, planes, pt, F, prm, enh, nullptr, A, M);
}

extern "C" rca_status ulm_density_shape(const rca_tables* t, double voxel_m, int32_t dims[3])
{
    if (!t || !dims || !(voxel_m > 0.0)) return RCA_ERR_INVALID_ARG;
    int d[3];
    density_shape(t->gd, voxel_m, d);
    for (int k = 0; k < 3; ++k) dims[k] = d[k];
    return RCA_OK;
}

extern "C" rca_status ulm_track(rca_handle* h, const rca_tables* t, const ulm_loc3d* L, const int* n3d, int cap3d,
                                int F, const ulm_track_params* prm, ulm_track_rec* out, int cap_tracks, int* n_tracks,
                                uint32_t* density)
{
    CHECK_HANDLE(h);
    rca_status st = check_tables(h, t, F);
    if (st != RCA_OK) return st;
    if (!prm) return set_error(h, RCA_ERR_INVALID_ARG, "null tracking parameters");
    if (prm->len < 2 || prm->len > ULM_TRACK_MAX_LEN)
        return set_error(h, RCA_ERR_INVALID_ARG, "track length %d outside [2, %d]", prm->len, ULM_TRACK_MAX_LEN);
    if (prm->substeps < 1 || prm->substeps > 1024)
        return set_error(h, RCA_ERR_INVALID_ARG, "substeps %d outside [1, 1024]", prm->substeps);
    if (!(prm->max_step_m > 0.0) || !(prm->voxel_m > 0.0) || !(prm->max_speed_change >= 0.0) ||
        !(prm->cos_max_turn >= -1.0 && prm->cos_max_turn <= 1.0))
        return set_error(h, RCA_ERR_INVALID_ARG, "tracking radius, voxel, speed change or turn cosine out of range");
    if (!n3d || !n_tracks || cap3d < 0 || cap_tracks < 0 || (cap3d > 0 && !L) || (cap_tracks > 0 && !out))
        return set_error(h, RCA_ERR_INVALID_ARG, "null list or count");
    if (density) {
        int d[3];
        density_shape(t->gd, prm->voxel_m, d);
        if (d[0] <= 0 || d[2] <= 0 || (double)d[0] * d[1] * d[2] > 4.0e9)
            return set_error(h, RCA_ERR_INVALID_ARG, "density grid of %d x %d x %d voxels", d[0], d[1], d[2]);
    }
    DeviceGuard dg(h->device);
    return launch_track(h, t, L, n3d, cap3d, F, prm, out, cap_tracks, n_tracks, density);
}

extern "C" rca_status ulm_track_velocity(rca_handle* h, const rca_tables* t, const ulm_track_rec* tracks,
                                         const int* n_tracks, int cap_tracks, const ulm_track_params* prm,
                                         int64_t* speed_sum, int64_t* vz_sum)
{
    CHECK_HANDLE(h);
    if (!t || !prm) return set_error(h, RCA_ERR_INVALID_ARG, "null tables or tracking parameters");
    if (prm->len < 2 || prm->len > ULM_TRACK_MAX_LEN || prm->substeps < 1 || prm->substeps > 1024 ||
        !(prm->voxel_m > 0.0))
        return set_error(h, RCA_ERR_INVALID_ARG, "track length, substeps or voxel out of range");
    if (!n_tracks || !speed_sum || !vz_sum || cap_tracks < 0 || (cap_tracks > 0 && !tracks))
        return set_error(h, RCA_ERR_INVALID_ARG, "null tracks, count or velocity sums");
    int d[3];
    density_shape(t->gd, prm->voxel_m, d);
    if (d[0] <= 0 || d[2] <= 0 || (double)d[0] * d[1] * d[2] > 4.0e9)
        return set_error(h, RCA_ERR_INVALID_ARG, "velocity grid of %d x %d x %d voxels", d[0], d[1], d[2]);
    DeviceGuard dg(h->device);
    return launch_track_velocity(h, t, tracks, n_tracks, cap_tracks, prm, speed_sum, vz_sum);
}

extern "C" rca_status ulm_localize(rca_handle* h, const rca_tables* t, const void* planes, rca_dtype pt, int F,
                                   const ulm_params* prm, ulm_loc2d* out2d, int cap2d, int* n2d, ulm_loc3d* out3d,
                                   int cap3d, int* n3d)
{
    CHECK_HANDLE(h);
    rca_status st = check_tables(h, t, F);
    if (st != RCA_OK) return st;
    if ((st = check_ulm(h, prm)) != RCA_OK) return st;
    if (!planes || !n2d || !n3d || cap2d < 0 || cap3d < 0 || (cap2d > 0 && !out2d) || (cap3d > 0 && !out3d))
        return set_error(h, RCA_ERR_INVALID_ARG, "null planes, list or count");
    if (!is_complex(pt)) return set_error(h, RCA_ERR_UNSUPPORTED, "planes dtype must be C32, C16F or C16BF");
    if (t->gd.N < prm->d || t->gd.nz < prm->d) return set_error(h, RCA_ERR_SHAPE, "plane smaller than the NCC kernel");
    DeviceGuard dg(h->device);
    const GeomDev& g = t->gd;
    float* A = (float*)ws_get(h, WS_A, (size_t)F * 2 * g.S * g.nz * g.N * sizeof(float), &st);
    if (!A) return st;
    float* M = (float*)ws_get(h, WS_M, (size_t)F * sizeof(float), &st);
    if (!M) return st;
    if ((st = launch_enhance(h, t, planes, pt, F, prm->enh, A, M)) != RCA_OK) return st;
    if ((st = launch_detect2d(h, t, A, M, F, prm, out2d, cap2d, n2d, nullptr, nullptr)) != RCA_OK) return st;
    return launch_pair3d(h, t, out2d, n2d, cap2d, F, out3d, cap3d, n3d);
}

extern "C" rca_status ulm_detect_map(rca_handle* h, const rca_tables* t, const float* map, int up, const float* A,
                                     const float* M, int F, float score_min, float alpha, ulm_loc2d* out2d, int cap2d,
                                     int* n2d)
{
    CHECK_HANDLE(h);
    rca_status st = check_tables(h, t, F);
    if (st != RCA_OK) return st;
    if (!map || !A || !M || !n2d || cap2d < 0 || (cap2d > 0 && !out2d))
        return set_error(h, RCA_ERR_INVALID_ARG, "null map, A, M, list or count");
    if (up < 1 || up > 8) return set_error(h, RCA_ERR_INVALID_ARG, "up must be in [1, 8]");
    if (!(alpha >= 0)) return set_error(h, RCA_ERR_INVALID_ARG, "bad alpha");
    DeviceGuard dg(h->device);
    return launch_detect_map(h, t, map, up, A, M, F, score_min, alpha, out2d, cap2d, n2d);
}

// ---------------------------------------------------------------------------
// batched form
// ---------------------------------------------------------------------------
static void batch_free(rca_batch* b)
{
    for (rca_handle* lh : b->lhs) {
        for (auto& w : lh->ws)
            if (w.p) cudaFree(w.p);
        delete lh;  // its status word belongs to the caller's handle
    }
    b->lhs.clear();
    for (cudaStream_t st : b->lstreams)
        if (st) cudaStreamDestroy(st);
    b->lstreams.clear();
    for (cudaEvent_t ev : b->ldone)
        if (ev) cudaEventDestroy(ev);
    b->ldone.clear();
    if (b->bf_done) cudaEventDestroy(b->bf_done);
    b->bf_done = nullptr;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    for (void* p : b->owned)
        if (p) cudaFree(p);
    if (b->d_ens) cudaFree(b->d_ens);
    if (b->d_segs) cudaFree(b->d_segs);
    if (b->d_ssegs) cudaFree(b->d_ssegs);
    if (b->d_cnt) cudaFree(b->d_cnt);
}

extern "C" rca_status rca_batch_create(rca_handle* h, int n, const rca_batch_item* items, rca_dtype rf_t,
                                       rca_dtype iq_t, rca_dtype pl_t, const ulm_params* prm, rca_batch** out)
{
    CHECK_HANDLE(h);
    if (!items || !out || n <= 0) return set_error(h, RCA_ERR_INVALID_ARG, "null items/output or n <= 0");
    *out = nullptr;
    if (!is_real_rf(rf_t) || !is_complex(iq_t) || !is_complex(pl_t))
        return set_error(h, RCA_ERR_UNSUPPORTED, "rf must be F32/F16/I16, iq and planes complex");
    if (prm && check_ulm(h, prm) != RCA_OK) return RCA_ERR_INVALID_ARG;
    for (int e = 0; e < n; ++e) {
        const rca_batch_item& it = items[e];
        if (!it.tables || !it.rf || !it.planes || it.n_frames <= 0)
            return set_error(h, RCA_ERR_INVALID_ARG, "item %d: null tables/rf/planes or n_frames <= 0", e);
        if (it.tables->h->device != h->device) return set_error(h, RCA_ERR_INVALID_ARG, "item %d on another device", e);
        if (rf_t == RCA_I16 && !it.scale) return set_error(h, RCA_ERR_INVALID_ARG, "item %d: int16 rf needs a scale", e);
        if (prm && (!it.n2d_dev || !it.n3d_dev || it.cap2d < 0 || it.cap3d < 0 || (it.cap2d && !it.out2d) ||
                    (it.cap3d && !it.out3d)))
            return set_error(h, RCA_ERR_INVALID_ARG, "item %d: localisation outputs missing", e);
        if (prm && (it.tables->gd.N < prm->d || it.tables->gd.nz < prm->d))
            return set_error(h, RCA_ERR_SHAPE, "item %d: plane smaller than the NCC kernel", e);
    }
    DeviceGuard dg(h->device);
    rca_batch* b = new (std::nothrow) rca_batch();
    if (!b) return set_error(h, RCA_ERR_CUDA, "out of host memory");
    b->h = h;
    b->n = n;
    b->rf_t = rf_t;
    b->iq_t = iq_t;
    b->pl_t = pl_t;
    for (int q = 0; q < 31; ++q) b->fir[q] = items[0].tables->fir[q];
    const size_t esz = dtype_size(iq_t);
    rca_status st = RCA_OK;
    auto alloc = [&](size_t bytes) -> void* {
        void* p = nullptr;
        if (cudaMalloc(&p, bytes + 256) != cudaSuccess) {
            st = set_error(h, RCA_ERR_CUDA, "batch workspace cudaMalloc(%zu) failed", bytes);
            return nullptr;
        }
        b->owned.push_back(p);
        return p;
    };
    int counters = 0;
    size_t smem = (size_t)32 * 159 * 8;  // demodulation tile (DM_NE x DM_PITCH float2)
    int maxr = 1, tmax = 1, tmin_all = 1 << 30;
    // Queue order: the mean units of every ensemble, then ensemble by ensemble
    // a software pipeline over chunks of BQ_CHUNK frames -- demodulation of
    // chunk c, Stage 1 of chunk c - BQ_LAG1, Stage 2 of chunk c - BQ_LAG2 --
    // so a unit's inputs are normally complete when it is taken and the IQ and
    // slices in flight stay small enough to be passed on through L2.  Every
    // unit depends only on units earlier in the queue.
    std::vector<int4> segA;
    int unit = 0;
    b->ens.resize(n);
    for (int e = 0; e < n && st == RCA_OK; ++e) {
        const rca_batch_item& it = items[e];
        const rca_tables* t = it.tables;
        const GeomDev& g = t->gd;
        const int nt = 2 * g.K, F = it.n_frames;
        BatchEns& E = b->ens[e];
        E.g = g;
        E.rf = it.rf;
        E.scale = it.scale;
        E.F = F;
        E.planes = it.planes;
        E.mean = (float*)alloc((size_t)nt * g.N * g.ns * 4);
        E.iq = alloc((size_t)F * nt * g.ns * g.N * esz);
        E.slices = (float2*)alloc((size_t)F * nt * g.nzs * g.N * 8);
        E.tx_q16 = t->tx_q16;
        E.rx_q16 = t->rx_q16;
        E.W = t->W;
        E.dmax = t->dmax;
        E.chunks = t->s1.d_chunks;
        E.rtab = iq_t == RCA_C16F ? t->s1.d_rec16 : t->s1.d_rec32;
        E.rblk = t->s1.rblk;
        E.zt = t->s1.zt;
        E.dc = t->s1.dc;
        E.n_tiles = t->s1.n_tiles;
        E.nch = t->s1.nch;
        E.ring = t->s1.ring;
        E.mix = t->mix;
        E.sfl = t->s2_sfl;
        E.sfr = t->s2_sfr;
        E.lw = t->s2_lw;
        E.rot = t->s2_rot;
        E.coef = t->s2_coefr;
        E.tmin = t->s2_tmin;
        E.T = t->T;
        E.zp = t->s2.zp;
        E.rows = t->s2.rows;
        E.smin0 = t->s2.smin[0];
        E.smin1 = t->s2.smin[1];
        E.n_tiles2 = t->s2.n_tiles;
        E.c2 = t->s2_c2r;
        E.iA = t->s2_iA;
        E.iB = t->s2_iB;
        {
            const int GW = s2_group_width(g.P);
            if (GW == 0) {
                st = set_error(h, RCA_ERR_UNSUPPORTED, "Stage 2 needs an even multiple of P (%d) up to 32", g.P);
                break;
            }
            E.LG = (g.N + GW - 1) / GW;
        }
        const int ncol = nt * g.N * g.ns;
        const int nbx = (g.ns + 127) / 128, nby = (g.N + 31) / 32;
        E.nA = (ncol / 4 + 255) / 256;
        E.nB_fk = nbx * nby;
        E.nB = E.nB_fk * F * nt;
        E.nC = E.n_tiles * nt * F;
        E.nD = E.n_tiles2 * E.LG * 2 * F;
        E.cA = counters;
        E.cB0 = counters + 1;
        E.cC0 = counters + 1 + F * nt;
        counters += 1 + F * nt + F;
        segA.push_back(make_int4(BS_MEAN, e, 0, E.nA));

        int LW = (g.N + 31) / 32, RG = std::max(1, 8 / LW);
        maxr = std::max(maxr, (E.zt + RG - 1) / RG);
        tmax = std::max(tmax, t->T);
        tmin_all = std::min(tmin_all, t->T);
        if (g.us != 2) b->us2 = false;
        smem = std::max(smem, stage1_smem_bytes(t, E.zt, E.dc, E.ring, esz));
        smem = std::max(smem, stage2_smem_bytes(t, E.zp));
        if (prm) {
            b->A.push_back((float*)alloc((size_t)F * 2 * g.S * g.nz * g.N * 4));
            b->M.push_back((float*)alloc((size_t)F * 4));
        }
    }
    if (st != RCA_OK) {
        batch_free(b);
        delete b;
        return st;
    }
    if (maxr > 16 || smem > 200 * 1024) {
        batch_free(b);
        delete b;
        return set_error(h, RCA_ERR_UNSUPPORTED, "batch tile shapes exceed the persistent kernel limits");
    }
    // segment = {stage | ensemble << 4, first unit, units, first stage-local unit}
    auto push = [&](int stage, int e, int loc0, int count) {
        if (count <= 0) return;
        b->segs.push_back(make_int4(stage | (e << 4), unit, count, loc0));
        unit += count;
    };
    for (auto& sg : segA) push(sg.x, sg.y, 0, sg.w);
    constexpr int BQ_CHUNK = 16, BQ_LAG1 = 2, BQ_LAG2 = 4;
    for (int e = 0; e < n; ++e) {
        const BatchEns& E = b->ens[e];
        const int F = E.F, nt = 2 * E.g.K, nc = (F + BQ_CHUNK - 1) / BQ_CHUNK;
        const int perB = E.nB / F, perC = E.nC / F, perD = E.nD / F;   // units per frame
        for (int c = 0; c < nc + BQ_LAG2; ++c) {
            auto frames = [&](int cc, int* f0, int* f1) {
                *f0 = cc * BQ_CHUNK;
                *f1 = std::min(F, *f0 + BQ_CHUNK);
            };
            int f0, f1;
            if (c < nc) {
                frames(c, &f0, &f1);
                push(BS_DEMOD, e, f0 * perB, (f1 - f0) * perB);
            }
            if (c - BQ_LAG1 >= 0 && c - BQ_LAG1 < nc) {
                frames(c - BQ_LAG1, &f0, &f1);
                push(BS_STAGE1, e, f0 * perC, (f1 - f0) * perC);
            }
            if (c - BQ_LAG2 >= 0 && c - BQ_LAG2 < nc) {
                frames(c - BQ_LAG2, &f0, &f1);
                push(BS_STAGE2, e, f0 * perD, (f1 - f0) * perD);
            }
        }
        (void)nt;
    }
    b->total = unit;
    // staged mode: per stage, every ensemble's units of that stage in one segment each
    std::vector<int4> ssegs;
    size_t s1max = 0, s2max = 0;
    for (int e = 0; e < n; ++e) {
        s1max = std::max(s1max, stage1_smem_bytes(items[e].tables, b->ens[e].zt, b->ens[e].dc, b->ens[e].ring, esz));
        s2max = std::max(s2max, stage2_smem_bytes(items[e].tables, b->ens[e].zp));
    }
    for (int stage = BS_MEAN; stage <= BS_STAGE2; ++stage) {
        b->sseg0[stage] = (int)ssegs.size();
        int u = 0;
        for (int e = 0; e < n; ++e) {
            const BatchEns& E = b->ens[e];
            const int cntu = stage == BS_MEAN ? E.nA : stage == BS_DEMOD ? E.nB : stage == BS_STAGE1 ? E.nC : E.nD;
            if (cntu <= 0) continue;
            ssegs.push_back(make_int4(stage | (e << 4), u, cntu, 0));
            u += cntu;
        }
        b->stotal[stage] = u;
    }
    b->sseg0[4] = (int)ssegs.size();
    b->ssmem[BS_MEAN] = 0;
    b->ssmem[BS_DEMOD] = (size_t)32 * 159 * 8;
    b->ssmem[BS_STAGE1] = s1max;
    b->ssmem[BS_STAGE2] = s2max;
    b->n_counters = counters;
    b->maxr = maxr;
    b->tmax = tmax;
    b->tmin_all = tmin_all;
    b->smem = smem;
    if (cudaMalloc(&b->d_ens, sizeof(BatchEns) * n) != cudaSuccess ||
        cudaMalloc(&b->d_segs, sizeof(int4) * b->segs.size()) != cudaSuccess ||
        cudaMalloc(&b->d_cnt, sizeof(int) * (counters + 2)) != cudaSuccess ||
        cudaMalloc(&b->d_ssegs, sizeof(int4) * ssegs.size()) != cudaSuccess) {
        batch_free(b);
        delete b;
        return set_error(h, RCA_ERR_CUDA, "batch descriptor cudaMalloc failed");
    }
    cudaMemcpy(b->d_ens, b->ens.data(), sizeof(BatchEns) * n, cudaMemcpyHostToDevice);
    cudaMemcpy(b->d_segs, b->segs.data(), sizeof(int4) * b->segs.size(), cudaMemcpyHostToDevice);
    cudaMemcpy(b->d_ssegs, ssegs.data(), sizeof(int4) * ssegs.size(), cudaMemcpyHostToDevice);
    if (prm) {
        b->localise = true;
        b->prm = *prm;
        bool okh = cudaEventCreateWithFlags(&b->bf_done, cudaEventDisableTiming) == cudaSuccess;
        for (int e = 0; e < n && okh; ++e) {
            rca_handle* lh = new (std::nothrow) rca_handle();
            if (!lh) {
                okh = false;
                break;
            }
            lh->device = h->device;
            lh->d_status = h->d_status;
            b->lhs.push_back(lh);
            cudaStream_t ls = nullptr;
            cudaEvent_t ev = nullptr;
            okh = cudaStreamCreateWithFlags(&ls, cudaStreamNonBlocking) == cudaSuccess;
            b->lstreams.push_back(ls);
            okh = okh && cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess;
            b->ldone.push_back(ev);
        }
        if (!okh) {
            batch_free(b);
            delete b;
            return set_error(h, RCA_ERR_CUDA, "localisation streams / handles for the batch");
        }
        for (int e = 0; e < n; ++e) {
            b->tabs.push_back(items[e].tables);
            b->out2d.push_back(items[e].out2d);
            b->out3d.push_back(items[e].out3d);
            b->cap2d.push_back(items[e].cap2d);
            b->cap3d.push_back(items[e].cap3d);
            b->n2d.push_back(items[e].n2d_dev);
            b->n3d.push_back(items[e].n3d_dev);
        }
    }
    *out = b;
    return RCA_OK;
}

static rca_status batch_enqueue(rca_batch* b)
{
    rca_status st = launch_batch(b->h, b);
    if (st != RCA_OK || !b->localise) return st;
    // fork: every ensemble's localisation on its own stream after the beamforming
    cudaStream_t main = b->h->stream;
    if ((st = cuda_check(b->h, cudaEventRecord(b->bf_done, main), "batch fork")) != RCA_OK) return st;
    for (int e = 0; e < b->n && st == RCA_OK; ++e) {
        rca_handle* h = b->lhs[e];
        h->stream = b->lstreams[e];
        const rca_tables* t = b->tabs[e];
        const int F = b->ens[e].F;
        st = cuda_check(b->h, cudaStreamWaitEvent(h->stream, b->bf_done, 0), "batch fork wait");
        if (st == RCA_OK) st = launch_enhance(h, t, b->ens[e].planes, b->pl_t, F, b->prm.enh, b->A[e], b->M[e]);
        if (st == RCA_OK)
            st = launch_detect2d(h, t, b->A[e], b->M[e], F, &b->prm, b->out2d[e], b->cap2d[e], b->n2d[e], nullptr,
                                 nullptr);
        if (st == RCA_OK)
            st = launch_pair3d(h, t, b->out2d[e], b->n2d[e], b->cap2d[e], F, b->out3d[e], b->cap3d[e], b->n3d[e]);
        if (!h->last_error.empty()) b->h->last_error = h->last_error;
        // join (also after a failed launch, so a capture stays well formed)
        cudaEventRecord(b->ldone[e], h->stream);
        cudaStreamWaitEvent(main, b->ldone[e], 0);
    }
    return st;
}

extern "C" rca_status rca_batch_run(rca_batch* b, int use_graph)
{
    if (!b) return RCA_ERR_INVALID_ARG;
    rca_handle* h = b->h;
    DeviceGuard dg(h->device);
    if (!use_graph) return batch_enqueue(b);
    if (!b->exec) {
        // one plain run sizes every workspace, then the same work is captured
        rca_status st = batch_enqueue(b);
        if (st != RCA_OK) return st;
        if ((st = cuda_check(h, cudaStreamSynchronize(h->stream), "batch warm-up")) != RCA_OK) return st;
        if (!b->cap_stream &&
            (st = cuda_check(h, cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking), "capture stream")) != RCA_OK)
            return st;
        cudaStream_t user = h->stream;
        h->stream = b->cap_stream;
        cudaGraph_t graph = nullptr;
        st = cuda_check(h, cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal), "begin capture");
        if (st == RCA_OK) {
            rca_status st2 = batch_enqueue(b);
            st = cuda_check(h, cudaStreamEndCapture(b->cap_stream, &graph), "end capture");
            if (st2 != RCA_OK) st = st2;
        }
        h->stream = user;
        if (st == RCA_OK) st = cuda_check(h, cudaGraphInstantiate(&b->exec, graph, 0), "graph instantiate");
        if (graph) cudaGraphDestroy(graph);
        if (st != RCA_OK) return st;
        return RCA_OK;  // the warm-up run already produced this run's results
    }
    return cuda_check(h, cudaGraphLaunch(b->exec, h->stream), "graph launch");
}

extern "C" rca_status rca_batch_set_mode(rca_batch* b, int mode)
{
    if (!b || (mode != RCA_BATCH_PERSISTENT && mode != RCA_BATCH_STAGED)) return RCA_ERR_INVALID_ARG;
    DeviceGuard dg(b->h->device);
    b->mode = mode;
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    return RCA_OK;
}

extern "C" rca_status rca_batch_set_wait_limit(rca_batch* b, long long cycles, int block_ensemble)
{
    if (!b || cycles <= 0 || block_ensemble >= b->n) return RCA_ERR_INVALID_ARG;
    DeviceGuard dg(b->h->device);
    b->wait_limit = cycles;
    if (block_ensemble >= 0) {
        BatchEns E = b->ens[block_ensemble];
        E.nB_fk += 1;  // Stage-1 units now wait for a demodulation unit that does not exist
        cudaMemcpy(b->d_ens + block_ensemble, &E, sizeof(BatchEns), cudaMemcpyHostToDevice);
    }
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    return RCA_OK;
}

extern "C" rca_status rca_batch_destroy(rca_batch* b)
{
    if (!b) return RCA_ERR_INVALID_ARG;
    DeviceGuard dg(b->h->device);
    cudaStreamSynchronize(b->h->stream);
    batch_free(b);
    delete b;
    return RCA_OK;
}

// ---------------------------------------------------------------------------
// autotuner
// ---------------------------------------------------------------------------
extern "C" rca_status rca_autotune(rca_handle* h, rca_tables* t, const void* iq, rca_dtype iq_t, int F, int* zt_out,
                                   int* dc_out, int* zp_out)
{
    CHECK_HANDLE(h);
    rca_status st = check_tables(h, t, F);
    if (st != RCA_OK) return st;
    if (!iq || !is_complex(iq_t)) return set_error(h, RCA_ERR_INVALID_ARG, "null or non-complex IQ");
    if (capturing(h)) return set_error(h, RCA_ERR_INVALID_ARG, "rca_autotune cannot run during stream capture");
    DeviceGuard dg(h->device);
    const GeomDev& g = t->gd;
    float2* slices = (float2*)ws_get(h, WS_SLICES, (size_t)F * 2 * g.K * g.nzs * g.N * sizeof(float2), &st);
    if (!slices) return st;
    void* planes = ws_get(h, WS_A, (size_t)F * 4 * g.S * g.nz * g.N * sizeof(float2), &st);
    if (!planes) return st;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    auto time_it = [&](auto fn) -> float {
        fn();  // warm-up
        cudaEventRecord(e0, h->stream);
        for (int r = 0; r < 3; ++r) fn();
        cudaEventRecord(e1, h->stream);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        return ms;
    };
    const size_t esz = dtype_size(iq_t);
    const int shapes[][2] = {{32, 8}, {16, 16}, {16, 8}, {16, 4}, {8, 16}, {8, 8}, {8, 4}, {4, 8}, {4, 4}};
    float best = 1e30f;
    int bz = t->s1.zt, bd = t->s1.dc;
    for (auto& sh : shapes) {
        const int zt = sh[0], dc = sh[1];
        const int ring = stage1_ring(t, zt, dc, nullptr, nullptr);
        if (stage1_smem_bytes(t, zt, dc, ring, esz) > 200 * 1024) continue;
        if (stage1_layout(g.N, zt, true).per > 16) continue;
        if ((st = plan_stage1(h, t, zt, dc)) != RCA_OK) break;
        const float ms = time_it([&] { launch_stage1(h, t, iq, iq_t, F, slices); });
        if (ms < best) {
            best = ms;
            bz = zt;
            bd = dc;
        }
    }
    if (st == RCA_OK) st = plan_stage1(h, t, bz, bd);
    // Stage 2 on the slices of the chosen shape
    if (st == RCA_OK) st = launch_stage1(h, t, iq, iq_t, F, slices);
    float best2 = 1e30f;
    int bzp = t->s2.zp;
    for (int zp = 1; zp <= 16 && st == RCA_OK; zp <<= 1) {
        if (stage2_smem_bytes(t, zp) > 200 * 1024) break;
        plan_stage2(t, zp);
        const float ms = time_it([&] { launch_stage2(h, t, slices, F, planes, RCA_C32); });
        if (ms < best2) {
            best2 = ms;
            bzp = zp;
        }
    }
    plan_stage2(t, bzp);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != RCA_OK) return st;
    st = cuda_check(h, cudaStreamSynchronize(h->stream), "autotune");
    if (zt_out) *zt_out = bz;
    if (dc_out) *dc_out = bd;
    if (zp_out) *zp_out = bzp;
    return st;
}

extern "C" rca_status rca_beamform_projections_batched(rca_handle* h, int n, const rca_batch_item* items,
                                                       rca_dtype rf_t, rca_dtype pl_t, const ulm_params* prm)
{
    CHECK_HANDLE(h);
    rca_batch* b = nullptr;
    rca_status st = rca_batch_create(h, n, items, rf_t, RCA_C32, pl_t, prm, &b);
    if (st != RCA_OK) return st;
    st = rca_batch_run(b, 0);
    DeviceGuard dg(h->device);
    const cudaError_t e = cudaStreamSynchronize(h->stream);
    const rca_status sd = rca_batch_destroy(b);
    if (st != RCA_OK) return st;
    if (e != cudaSuccess) return cuda_check(h, e, "batched beamforming");
    return sd;
}

extern "C" rca_status rca_fp32_probe(rca_handle* h, int packed, int iterations, float* sink, double* flops)
{
    CHECK_HANDLE(h);
    if (!sink) return set_error(h, RCA_ERR_INVALID_ARG, "null sink");
    if (iterations < 1 || iterations > (1 << 24))
        return set_error(h, RCA_ERR_INVALID_ARG, "iterations %d outside [1, 2^24]", iterations);
    DeviceGuard dg(h->device);
    return launch_fp32_probe(h, packed ? 1 : 0, iterations, sink, flops);
}
