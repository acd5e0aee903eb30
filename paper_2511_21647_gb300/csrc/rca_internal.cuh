// rca_internal.cuh -- internal types shared by librca's translation units.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/rca.h"

// ---------------------------------------------------------------------------
// device status word bits (read by rca_sync_status)
// ---------------------------------------------------------------------------
enum : unsigned {
    ST_CAPACITY = 1u << 0,
    ST_TIMEOUT = 1u << 1,
    ST_BOUNDS = 1u << 2,
};

// Geometry as seen by kernels (plain values, passed by value).
struct GeomDev {
    int N;       // elements per array = lateral pixels
    int nz;      // plane rows
    int nzs;     // slice rows = (nz - 1) * us + 1
    int ns;      // samples per channel
    int P;       // slab size
    int S;       // slabs per axis = N / P
    int K;       // transmissions per family
    int us;      // slice oversampling
    double pitch, fc, fs, c, z0, dz, fnum, t0, L;
    double sin_th[2 * RCA_MAX_K];
    double cos_th[2 * RCA_MAX_K];
};

// Workspace slots owned by a handle.
enum WsSlot {
    WS_MEAN = 0,   // float [2K][E][ns] clutter mean
    WS_IQ,         // IQ of the current ensemble
    WS_SLICES,     // float2 [F][2K][nzs][N]
    WS_A,          // float [F][2][S][nz][N]
    WS_M,          // float [F]
    WS_CAND,       // ulm_loc2d [strips][CAND_CAP]
    WS_CANDCNT,    // int [strips]
    WS_PLANEOFF,   // int [planes + 1]
    WS_FLAGS,      // int [n]
    WS_SCAN,       // int [n + 1]
    WS_N2D,        // int [1]
    WS_MISC,       // small scratch
    WS_TRACK,      // tracking: frame offsets, links, flags, positions, per-localisation tracks
    WS_MOTION,     // motion estimation: twiddles, row spectra, reference spectrum, correlations
    WS_SVD,        // clutter filter: partial covariances, covariances, subspace bases
    WS_COUNT
};

struct WsBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

struct rca_handle {
    int device = 0;
    cudaStream_t stream = nullptr;
    unsigned* d_status = nullptr;
    std::string last_error;
    WsBuf ws[WS_COUNT];
};

struct rca_geometry {
    rca_geometry_desc desc{};
    std::vector<double> ang;  // 2K angles, RC first
    GeomDev gd{};
};

// Stage-1 launch shape chosen at table-build time.  A CTA owns `zt` slice
// rows of one (frame, transmission) and walks the lateral distance d in
// chunks of `dc`; chunk c of row tile t needs the contiguous sample rows
// [nlo, nlo + nrows) of the [ns][E] IQ block (element innermost).
struct Stage1Plan {
    int zt = 0;               // slice rows per CTA
    int dc = 0;               // lateral distances per chunk
    int n_tiles = 0;
    int nch = 0;              // chunks per tile
    int ring = 0;             // sample rows of the shared-memory ring (plus one duplicate row)
    // [2K][n_tiles][nch] {first new sample row n, new row count | ring slot of n << 16, d0, d1}:
    // the rows a chunk needs that earlier chunks of its tile did not load; d1 == d0 for a
    // chunk without work
    int4* d_chunks = nullptr;
    // per-(d, row) weight records of every chunk, one block of rblk bytes per
    // (k, tile, chunk): [dc][zt] 16-byte records, then [dc][zt] ring byte
    // offsets.  rec32: FP32 weights, offsets for 8-byte samples (4-byte
    // samples use half of them); rec16: FP16 weights, offsets for 4-byte samples.
    int rblk = 0;
    unsigned char* d_rec32 = nullptr;
    unsigned char* d_rec16 = nullptr;
};

struct Stage2Plan {
    int zp = 0;           // plane rows per CTA
    int n_tiles = 0;
    int rows = 0;         // slice rows held per transmission
    int smin[2] = {0, 0}; // per family: min floor shift (slice rows)
    int smax[2] = {0, 0};
};

struct rca_tables {
    rca_handle* h = nullptr;
    GeomDev gd{};
    // Stage-1 / DAS tables
    double* tx_f64 = nullptr;   // [2K][nzs]
    double* rx_f64 = nullptr;   // [N][nzs]
    int* tx_q16 = nullptr;      // [2K][nzs]
    int* rx_q16 = nullptr;      // [nzs][N]
    float2* W = nullptr;        // [nzs][N]
    int* dmax = nullptr;        // [nzs]
    // Stage-2 tables
    double* s2_shift = nullptr; // [2K][N]
    int* s2_sfl = nullptr;      // [2K][N] floor of the shift
    float* s2_sfr = nullptr;    // [2K][N] fractional part
    float2* s2_psi = nullptr;   // [2K][N]
    float2* s2_ec = nullptr;    // [2K][nz]
    float2* s2_coef = nullptr;  // [2K][S][nz][T]
    int* s2_tmin = nullptr;     // [2K][S]
    int T = 0;
    // the same taps without the row's carrier: coef[k][b][i][t] = ec[k][i] c2[k][b][t]
    // for every plane row i in [s2_iA, s2_iB] (all of the slab's shifted rows
    // inside the slice)
    float2* s2_c2 = nullptr;    // [2K][S][T]
    int s2_iA = 0, s2_iB = -1;
    // Stage 2 on carrier-rotated slices w_r = v_r rot[k][r] (rot: the carrier
    // phase of tau_c at slice row r without its constant part; tau_c is
    // linear in depth, so each output's carrier becomes a constant factor of
    // the taps and no longer multiplies the output): the same taps and
    // lateral weights times that factor
    float2* s2_rot = nullptr;   // [2K][nzs] exp(j 2 pi fc (1 + cos th_k) z_r / c)
    float2* s2_c2r = nullptr;   // [2K][S][T] c2 kappa_k exp(-j beta_k (tmin + t))
    float2* s2_coefr = nullptr; // [2K][S][nz][T] coef conj(rot) at each tap's slice row
    float4* s2_lw = nullptr;    // [2K][N] {a, b}: lateral interpolation weights with the carrier folded in
    // direct (conventional 3D) tables
    int* dtx_q16 = nullptr;     // [2K][N][nz] transmit delay at transverse u, plane depth
    float2* dtx_ph = nullptr;   // [2K][N][nz] exp(j 2 pi fc (tau_tx + z / c))
    // demodulation
    float2* mix = nullptr;      // [ns] exp(-j 2 pi fc t_n)
    float fir[31] = {0};        // half-band taps (host copy; passed by value)
    Stage1Plan s1;
    Stage2Plan s2;
    int direct_win = 0;         // window for direct mode (rows of samples)
    int direct_zt = 0;
    // host copies used to (re)plan launch shapes
    std::vector<int> h_txq, h_rxq, h_dm, h_sfl;
};

// Stage-2 CTA geometry (shared by the planner and the kernels)
// Thread layout of a Stage-1 CTA (256 threads): LW warps across the lateral
// pixels times RG row groups of `per` rows each.  Paired (N a multiple of 64,
// at most 8 rows per thread): a lane owns pixel l < N / 2 and its mirror
// N - 1 - l, so LW = N / 64; otherwise one pixel per lane, LW = ceil(N / 32).
struct S1Layout {
    int LW, RG, per;
    bool pair;
};
__host__ __device__ inline S1Layout stage1_layout(int N, int zt, bool allow_pair)
{
    S1Layout s;
    s.pair = false;
    if (allow_pair && N % 64 == 0 && N <= 512) {
        s.LW = N / 64;
        s.RG = s.LW >= 8 ? 1 : 8 / s.LW;
        s.per = (zt + s.RG - 1) / s.RG;
        if (s.per <= 8) {
            s.pair = true;
            return s;
        }
    }
    s.LW = (N + 31) / 32;
    s.RG = s.LW >= 8 ? 1 : 8 / s.LW;
    s.per = (zt + s.RG - 1) / s.RG;
    return s;
}

#define S2_ZP 16       // plane rows per CTA (at most)
#define S2_THREADS 256

// lateral pixels per CTA: the largest even multiple of P up to 32 (even, so
// that a row segment of complex FP32 values is a whole number of 16-byte
// units); 0 where no such multiple exists (P odd above 15, or P > 32)
inline __host__ __device__ int s2_group_width(int P)
{
    if (P > 32) return 0;
    int m = 32 / P;
    if (P & 1) m &= ~1;
    return m * P;
}

// shared-memory bytes of one Stage-2 CTA
inline __host__ __device__ size_t s2_smem_bytes(int K, int S, int N, int P, int T, int rows)
{
    const int GW = s2_group_width(P), SG = GW > 0 ? GW / P : 1;
    return (size_t)K * rows * 32 * 8          // slice columns [K][rows][32]
           + (size_t)K * N * 16               // lateral weights [K][N] {a, b}
           + (size_t)K * S * T * 16           // row-independent taps [K][S][T] {x, x, y, y}
           + (size_t)K * SG * rows * 8        // slab sums [K][SG][rows]
           + (size_t)K * N * 4 + (size_t)K * S * 4;  // shift rows [K][N], tap rows [K][S]
}


// launch-shape planning (tables.cu)
int stage1_ring(const rca_tables* t, int zt, int dc, std::vector<int4>* chunks, std::vector<int>* bases);
size_t stage1_smem_bytes(const rca_tables* t, int zt, int dc, int ring, size_t esz);
rca_status plan_stage1(rca_handle* h, rca_tables* t, int zt, int dc);
size_t stage2_smem_bytes(const rca_tables* t, int zp);
void plan_stage2(rca_tables* t, int zp);

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
#define RCA_MAX_NCC_D 15
#define CAND_CAP 96       // 2D candidates per (plane, row strip)
#define DET_RS 30         // rows per strip of the heatmap peak search (ulm_detect_map)
#define NCC_RS 30         // rows per strip of the NCC detection (+ one row above and below: 32 = 8 x 4)

struct NccConst {
    int d, h;
    float gz[RCA_MAX_NCC_D];
    float gl[RCA_MAX_NCC_D];
    float muG, inv_ssG_sqrt, flat_coef;  // flat_coef = 1e-5 d^2
    float alpha, ncc_min;
};

rca_status set_error(rca_handle* h, rca_status s, const char* fmt, ...);
rca_status cuda_check(rca_handle* h, cudaError_t e, const char* what);
void* ws_get(rca_handle* h, WsSlot slot, size_t bytes, rca_status* st);

// size in bytes of one element of a dtype
size_t dtype_size(rca_dtype t);

// launchers (implemented in the .cu files)
rca_status launch_tables(rca_handle* h, rca_tables* t);
rca_status launch_ingest(rca_handle* h, const rca_tables* t, const void* rf, rca_dtype rf_t,
                         const float* scale, int F, int clutter, void* iq, rca_dtype iq_t);
rca_status launch_stage1(rca_handle* h, const rca_tables* t, const void* iq, rca_dtype iq_t, int F,
                         float2* slices);
void density_shape(const GeomDev& g, double voxel, int dims[3]);
rca_status launch_clutter_svd(rca_handle* h, const rca_tables* t, float2* slices, int F, int nc, int iters,
                              float* info);
rca_status launch_separate(rca_handle* h, const rca_tables* t, const void* planes, rca_dtype pt, int F,
                           const ulm_sep_params* prm, int enh, float2* sub, float* A, float* M);
rca_status launch_motion(rca_handle* h, const rca_tables* t, const float2* slices, int F, float* motion,
                         float* shifts, int* peaks);
rca_status launch_track_velocity(rca_handle* h, const rca_tables* t, const ulm_track_rec* tracks,
                                 const int* n_tracks, int cap_tracks, const ulm_track_params* prm, int64_t* speed,
                                 int64_t* vz);
rca_status launch_track(rca_handle* h, const rca_tables* t, const ulm_loc3d* L, const int* n3d, int cap3d, int F,
                        const ulm_track_params* prm, ulm_track_rec* out, int cap_tracks, int* n_tracks, unsigned* density);
rca_status launch_stage2(rca_handle* h, const rca_tables* t, const float2* slices, int F, void* planes,
                         rca_dtype pt);
rca_status launch_direct(rca_handle* h, const rca_tables* t, const void* iq, rca_dtype iq_t, int F,
                         void* planes, rca_dtype pt);
rca_status launch_enhance(rca_handle* h, const rca_tables* t, const void* planes, rca_dtype pt, int F,
                          int enh, float* A, float* M);
rca_status launch_detect2d(rca_handle* h, const rca_tables* t, const float* A, const float* M, int F,
                           const ulm_params* prm, ulm_loc2d* out, int cap, int* n2d, float* ncc_out,
                           int* plane_off);
rca_status launch_detect_map(rca_handle* h, const rca_tables* t, const float* map, int up, const float* A, const float* M,
                             int F, float score_min, float alpha, ulm_loc2d* out, int cap, int* n2d);
rca_status launch_pair3d(rca_handle* h, const rca_tables* t, const ulm_loc2d* L, const int* n2d, int cap2d,
                         int F, ulm_loc3d* out, int cap3d, int* n3d);
rca_status launch_fp32_probe(rca_handle* h, int packed, int iters, float* sink, double* flops);
rca_status launch_pair3d_noalloc(rca_handle* h, const rca_tables* t, const ulm_loc2d* L, const int* n2d,
                                 int cap2d, int F, ulm_loc3d* out, int cap3d, int* n3d);

// ---------------------------------------------------------------------------
// device-side element access for the supported complex / real dtypes
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 load_c(const void* p, size_t i, int dt)
{
    if (dt == RCA_C32) return reinterpret_cast<const float2*>(p)[i];
    if (dt == RCA_C16F) return __half22float2(reinterpret_cast<const __half2*>(p)[i]);
    return __bfloat1622float2(reinterpret_cast<const __nv_bfloat162*>(p)[i]);
}

__device__ __forceinline__ void store_c(void* p, size_t i, int dt, float2 v)
{
    if (dt == RCA_C32) {
        reinterpret_cast<float2*>(p)[i] = v;
    } else if (dt == RCA_C16F) {
        reinterpret_cast<__half2*>(p)[i] = __float22half2_rn(v);
    } else {
        reinterpret_cast<__nv_bfloat162*>(p)[i] = __float22bfloat162_rn(v);
    }
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__device__ __forceinline__ void cfma(float2& acc, float2 w, float2 v)
{
    acc.x = fmaf(w.x, v.x, acc.x);
    acc.x = fmaf(-w.y, v.y, acc.x);
    acc.y = fmaf(w.x, v.y, acc.y);
    acc.y = fmaf(w.y, v.x, acc.y);
}

// ---------------------------------------------------------------------------
// TMA bulk copies (cp.async.bulk, global -> shared) completed on an mbarrier.
// Every wait is bounded by a clock budget; a wait that runs out reports
// ST_TIMEOUT through the status word and the caller returns.
// ---------------------------------------------------------------------------
#define RCA_WAIT_CYCLES (4ll * 1000 * 1000 * 1000)  // ~2 s at 2 GHz

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// make mbarrier initialisation visible to the async (TMA) proxy
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// order this thread's earlier generic shared-memory accesses before later
// async-proxy (TMA) accesses to the same memory
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// bytes and both addresses must be multiples of 16
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// Checked build (compiled with -DRCA_CHECKED, library librca_checked.so):
// index checks on shared-memory ring slots, staged rows, detection strip
// rows, flag and candidate-bitmap indexes, gathered pixels and queue indexes
// that record ST_BOUNDS in the status word and skip the access instead of
// trapping.  In the release build chk() is constant true and compiles away.
#ifdef RCA_CHECKED
#define RCA_CHECKED_BUILD 1
#else
#define RCA_CHECKED_BUILD 0
#endif
__device__ __forceinline__ bool chk(bool ok, unsigned* status)
{
    if constexpr (RCA_CHECKED_BUILD) {
        if (!ok) atomicOr(status, ST_BOUNDS);
        return ok;
    }
    return true;
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned phase)
{
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void mbar_inval(uint64_t* bar)
{
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// bounded wait for the given phase parity; false if the budget ran out
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned phase)
{
    long long t0 = clock64();
    while (!mbar_try_wait(bar, phase)) {
        if (clock64() - t0 > RCA_WAIT_CYCLES) return false;
    }
    return true;
}

// All threads wait for `phase` of `bar`, then synchronise.  Returns false
// (after recording ST_TIMEOUT and waiting once more, bounded, for the copy
// still in flight) if any thread's wait ran out; the CTA must then return.
__device__ __forceinline__ bool cta_wait_copies(uint64_t* bar, unsigned phase, unsigned* status)
{
    bool ok = mbar_wait_bounded(bar, phase);
    if (__syncthreads_or(!ok)) {
        if (threadIdx.x == 0) atomicOr(status, ST_TIMEOUT);
        mbar_wait_bounded(bar, phase);
        __syncthreads();
        return false;
    }
    return true;
}

// Streaming store (evict-first): outputs that are not re-read soon.
__device__ __forceinline__ void store_c_cs(void* p, size_t i, int dt, float2 v)
{
    if (dt == RCA_C32) {
        __stcs(reinterpret_cast<float2*>(p) + i, v);
    } else if (dt == RCA_C16F) {
        __half2 h = __float22half2_rn(v);
        __stcs(reinterpret_cast<unsigned*>(p) + i, *reinterpret_cast<unsigned*>(&h));
    } else {
        __nv_bfloat162 b = __float22bfloat162_rn(v);
        __stcs(reinterpret_cast<unsigned*>(p) + i, *reinterpret_cast<unsigned*>(&b));
    }
}

// ---------------------------------------------------------------------------
// packed FP32 pairs (Blackwell f32x2 FMA): two lanes of float math per instruction
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t f2_pack(float a, float b)
{
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}

__device__ __forceinline__ float2 f2_unpack(uint64_t v)
{
    float a, b;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
    return make_float2(a, b);
}

__device__ __forceinline__ uint64_t f2_fma(uint64_t a, uint64_t b, uint64_t c)
{
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

__device__ __forceinline__ uint64_t f2_sub(uint64_t a, uint64_t b)
{
    uint64_t d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

__device__ __forceinline__ uint64_t f2_mul(uint64_t a, uint64_t b)
{
    uint64_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

__device__ __forceinline__ uint64_t f2_add(uint64_t a, uint64_t b)
{
    uint64_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// 32-bit shared-memory loads by byte address
__device__ __forceinline__ uint64_t lds_u64(unsigned addr)
{
    uint64_t v;
    asm volatile("ld.shared.b64 %0, [%1];" : "=l"(v) : "r"(addr));
    return v;
}

__device__ __forceinline__ unsigned lds_u32(unsigned addr)
{
    unsigned v;
    asm volatile("ld.shared.b32 %0, [%1];" : "=r"(v) : "r"(addr));
    return v;
}

__device__ __forceinline__ void lds_u64x2(unsigned addr, uint64_t& a, uint64_t& b)
{
    asm volatile("ld.shared.v2.b64 {%0, %1}, [%2];" : "=l"(a), "=l"(b) : "r"(addr));
}

// ---------------------------------------------------------------------------
// batched form: one persistent launch over the beamforming work of many
// ensembles (ingest mean, demodulation, Stage 1, Stage 2), ordered by a
// device work queue with per-ensemble dependency counters
// ---------------------------------------------------------------------------
enum BatchStage { BS_MEAN = 0, BS_DEMOD = 1, BS_STAGE1 = 2, BS_STAGE2 = 3 };

struct BatchEns {
    GeomDev g;
    const void* rf;
    const float* scale;
    int F;
    float* mean;
    void* iq;
    float2* slices;
    void* planes;
    // tables
    const int* tx_q16;
    const int* rx_q16;
    const float2* W;
    const int* dmax;
    const int4* chunks;
    const unsigned char* rtab;  // Stage-1 record table for the batch's IQ dtype
    int rblk;
    int zt, dc, n_tiles, nch, ring;
    const float2* mix;
    const int* sfl;
    const float* sfr;
    const float4* lw;           // Stage-2 tables for carrier-rotated slices (rca_tables::s2_lw, s2_rot,
    const float2* rot;          // s2_coefr, s2_c2r)
    const float2* coef;
    const int* tmin;
    int T, zp, rows, smin0, smin1, n_tiles2;
    const float2* c2;
    int iA, iB, LG;
    // work units and counters
    int nA, nB, nC, nD;      // units per stage
    int nB_fk;               // demodulation units per (frame, transmission)
    int cA, cB0, cC0;        // counter indices: mean done, demod done per (f, k), Stage 1 done per f
};

struct rca_batch {
    rca_handle* h = nullptr;
    int n = 0;
    rca_dtype rf_t = RCA_F32, iq_t = RCA_C32, pl_t = RCA_C32;
    std::vector<BatchEns> ens;
    std::vector<int4> segs;       // {stage | ensemble << 4, first unit, count, first stage-local unit}
    int total = 0;                // work units
    int n_counters = 0;
    BatchEns* d_ens = nullptr;
    int4* d_segs = nullptr;
    int* d_cnt = nullptr;         // [n_counters + 2]: counters, next-unit, abort
    std::vector<void*> owned;     // per-ensemble workspace
    float fir[31];
    long long wait_limit = RCA_WAIT_CYCLES;
    int maxr = 2, tmax = 1, tmin_all = 1 << 30;
    bool us2 = true;              // every ensemble has two slice rows per plane row
    size_t smem = 0;
    int grid = 0;
    // launch mode: RCA_BATCH_PERSISTENT (one launch, dependency-ordered queue)
    // or RCA_BATCH_STAGED (one launch per stage over every ensemble's units
    // of that stage; stream order replaces the dependency waits)
    int mode = 0;
    int4* d_ssegs = nullptr;      // staged mode: segments of stage s at [sseg0[s], sseg0[s + 1]), units from 0
    int sseg0[5] = {0, 0, 0, 0, 0};
    int stotal[4] = {0, 0, 0, 0}; // units per stage
    size_t ssmem[4] = {0, 0, 0, 0};
    int sgrid[4] = {0, 0, 0, 0};
    // optional localisation
    bool localise = false;
    ulm_params prm{};
    std::vector<const rca_tables*> tabs;
    std::vector<ulm_loc2d*> out2d;
    std::vector<ulm_loc3d*> out3d;
    std::vector<int> cap2d, cap3d;
    std::vector<int*> n2d, n3d;
    std::vector<float*> A, M;
    // private handles for the localisation workspace, one per ensemble (they
    // share the caller's status word), so a captured graph never points at
    // buffers that other calls on the caller's handle could reallocate, and
    // the ensembles' localisations can run concurrently on their own streams
    std::vector<rca_handle*> lhs;
    std::vector<cudaStream_t> lstreams;
    std::vector<cudaEvent_t> ldone;
    cudaEvent_t bf_done = nullptr;
    // CUDA graph of one batch run
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap_stream = nullptr;
};

rca_status launch_batch(rca_handle* h, rca_batch* b);
// one per IQ dtype (separate translation units)
rca_status launch_batch_c32(rca_handle* h, rca_batch* b);
rca_status launch_batch_c16f(rca_handle* h, rca_batch* b);
rca_status launch_batch_c16bf(rca_handle* h, rca_batch* b);
