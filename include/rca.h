/*
 * rca.h -- C ABI of librca: projection-based row-column-array (RCA) 3D
 * ultrasound localization microscopy on one GPU (sm_103a).
 *
 * Method (arXiv 2511.21647):
 *   Sec. II-A1  two-stage RCA beamforming: Stage 1 beamforms one reference
 *               slice per steered RC / CR transmission from channel data;
 *               Stage 2 extrapolates it along the transmit direction by a
 *               rigid axial shift and compounds (Fig. 1b-c).
 *   Sec. II-A4  the volume is cut into P x P x N sub-blocks and sum-projected
 *               onto x-z and y-z planes (Sec. II-A5 counts 2N/P planes); the
 *               RC and CR stacks are combined by XDoppler (3-frame window);
 *               each plane is normalised-cross-correlated with a Gaussian PSF
 *               using separable 1D correlations (Fig. 1g); sub-pixel regional
 *               peaks are paired across the XZ and YZ planes into 3D by an
 *               axial tolerance of one pixel and an intensity ratio in
 *               [0.9, 1.11] with mutual minimum ratio.
 *   Sec. II-C   acquisition constants (pitch 0.214 mm, 128 + 128 elements,
 *               400 Hz, P = 8, 11-tap 1D kernels).
 * The library never materialises the N x N x nz volume.
 *
 * Conventions for every entry point
 *   Ownership   the caller owns all data buffers (channel data, scales,
 *               planes, lists, counts): plain device pointers, 256-byte
 *               alignment recommended, 16 bytes required.  The library owns
 *               handles, geometries, tables, CNNs and its internal workspace
 *               and frees them in the matching *_destroy call.
 *   Execution   all GPU work is enqueued on the handle's stream (the legacy
 *               default stream until rca_set_stream) and returns without
 *               synchronising, except where a function says it synchronises.
 *   Errors      argument, shape and dtype errors are detected on the host
 *               before anything is enqueued: the call returns a non-zero
 *               rca_status and rca_last_error() describes it.  Conditions
 *               only the GPU can see (output capacity overflow, a bounded
 *               wait that ran out, a checked-build bounds violation) set bits
 *               of a device status word that rca_sync_status() reads and
 *               clears; no kernel traps or asserts.
 *   Threads     one handle per host thread.
 *
 * Array layouts (row-major; complex = interleaved re, im):
 *   rf      [F][2K][E][ns]           F frames, 2K transmissions (RC first),
 *                                    E = n_el receive elements, ns samples
 *   iq      [F][2K][ns][E] complex   baseband IQ after clutter removal
 *                                    (element innermost: one sample row of
 *                                    all elements is contiguous)
 *   slices  [F][2K][nzs][N] complex  Stage-1 reference slices, N = n_el
 *                                    lateral pixels, nzs = (nz-1)*us + 1
 *   planes  [F][2][2][S][nz][N] complex   [axis][family][slab]:
 *                                    axis 0 = XZ (slab over y, lateral x),
 *                                    axis 1 = YZ (slab over x, lateral y),
 *                                    family 0 = RC, 1 = CR, S = N / P
 *   A       [F][2][S][nz][N] float   XDoppler amplitude
 */
#ifndef RCA_H
#define RCA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RCA_VERSION_MAJOR 0
#define RCA_VERSION_MINOR 1
#define RCA_MAX_K 8            /* transmissions per family */

typedef enum {
    RCA_OK = 0,
    RCA_ERR_INVALID_ARG = 1,  /* null pointer, bad enum, value out of range */
    RCA_ERR_SHAPE = 2,        /* sizes inconsistent with the geometry */
    RCA_ERR_UNSUPPORTED = 3,  /* valid but not implemented (dtype combination, K > 8) */
    RCA_ERR_CUDA = 4,         /* a CUDA runtime call failed; see rca_last_error */
    RCA_ERR_CAPACITY = 5,     /* (device) an output list overflowed its capacity */
    RCA_ERR_TIMEOUT = 6,      /* (device) a bounded wait gave up */
    RCA_ERR_BOUNDS = 7        /* (device, checked builds) an index left its buffer */
} rca_status;

typedef enum {
    RCA_F32 = 0,    /* float */
    RCA_I16 = 1,    /* int16 with a per-channel float scale */
    RCA_F16 = 2,    /* IEEE half */
    RCA_C32 = 3,    /* complex float (8 bytes) */
    RCA_C16F = 4,   /* complex half (4 bytes) */
    RCA_C16BF = 5   /* complex bfloat16 (4 bytes) */
} rca_dtype;

typedef struct rca_handle rca_handle;
typedef struct rca_geometry rca_geometry;
typedef struct rca_tables rca_tables;

/* ---------------------------------------------------------------------- */
/* Handle, stream, status                                                  */
/* ---------------------------------------------------------------------- */

/* Library version as (major << 16) | minor. */
int rca_version(void);

/* Static text for a status code; never NULL. */
const char* rca_status_string(rca_status s);

/* Create a handle bound to CUDA device `device` (made current for the call).
 * Allocates the device status word.  Errors: INVALID_ARG (h NULL), CUDA. */
rca_status rca_create(rca_handle** h, int device);

/* Free the handle and its workspace (synchronises its stream first). */
rca_status rca_destroy(rca_handle* h);

/* Use a caller-owned cudaStream_t (passed as void*) for all later work;
 * NULL selects the legacy default stream.  The library never destroys it. */
rca_status rca_set_stream(rca_handle* h, void* cuda_stream);

/* Host-side text of the last error on this handle ("" if none). */
const char* rca_last_error(const rca_handle* h);

/* Synchronise the handle's stream, then read and clear the device status
 * word.  *device_status receives RCA_OK or the first device-side error
 * (CAPACITY, TIMEOUT, BOUNDS).  Returns CUDA if the stream reported a fault. */
rca_status rca_sync_status(rca_handle* h, rca_status* device_status);

/* Reserve workspace for ensembles of up to n_frames frames of `g` so that no
 * allocation happens later (needed before CUDA graph capture). Synchronises. */
rca_status rca_reserve(rca_handle* h, const rca_geometry* g, int n_frames);

/* ---------------------------------------------------------------------- */
/* Geometry and delay tables (Sec. II-A1, Sec. II-C)                       */
/* ---------------------------------------------------------------------- */

typedef struct {
    int n_el;          /* elements per array (rows = columns); N lateral pixels;
                          a multiple of 4 (16-byte sample rows), at most 256 */
    int nz;            /* axial pixels of the projection planes */
    int ns;            /* RF samples per channel */
    int P;             /* sub-block / slab size in pixels (paper: 8); n_el % P == 0 */
    int K;             /* transmissions per family: K RC then K CR (1..8) */
    int us;            /* Stage-1 axial oversampling (slice rows per plane pixel, 1..8) */
    double pitch_m;    /* element pitch = lateral pixel size */
    double fc_hz;      /* demodulation / carrier frequency */
    double fs_hz;      /* RF sampling rate */
    double c_mps;      /* speed of sound */
    double z0_m;       /* depth of plane row 0; first RF sample at t0 = 2 z0 / c */
    double dz_m;       /* axial pixel size of the planes */
    double fnum;       /* receive F-number (Hann apodisation over z / fnum) */
    const double* ang_rc_rad;  /* K steering angles of the RC transmissions */
    const double* ang_cr_rad;  /* K steering angles of the CR transmissions */
} rca_geometry_desc;

/* Copy and validate a geometry (host only; nothing is enqueued).
 * Model: element / pixel centres u_e = (e - (N-1)/2) pitch; RC transmission
 * k delays (z cos th + y sin th + (L/2)|sin th|)/c and receives on columns
 * with sqrt((x-u_e)^2 + z^2)/c (CR swaps x and y), L = N pitch.
 * Errors: INVALID_ARG (non-positive sizes, n_el % P != 0), UNSUPPORTED (K > 8). */
rca_status rca_geometry_create(rca_handle* h, const rca_geometry_desc* desc, rca_geometry** out);
rca_status rca_geometry_destroy(rca_geometry* g);

/* Build the per-geometry tables on the GPU in FP64 (sub-nanosecond delays)
 * and store them as Q16 fixed-point sample delays and FP32 complex weights:
 * transmit and receive delays, Hann x carrier weights, aperture limits,
 * Stage-2 axial shifts and carrier terms, and the Stage-2 slab-sum
 * coefficients.  Synchronises once (to size the Stage-1 sample windows). */
rca_status rca_delay_tables(rca_handle* h, const rca_geometry* g, rca_tables** out);
rca_status rca_tables_destroy(rca_tables* t);

/* Table identifiers for rca_tables_query / rca_tables_download. */
typedef enum {
    RCA_TAB_TX_F64 = 0,   /* double [2K][nzs]: (tau_tx(k, 0, z_r) - t0) fs, samples */
    RCA_TAB_RX_F64 = 1,   /* double [N][nzs] : tau_rx(d pitch, z_r) fs, d = |lateral - element| */
    RCA_TAB_TX_Q16 = 2,   /* int32  [2K][nzs]: rint(TX_F64 * 65536) */
    RCA_TAB_RX_Q16 = 3,   /* int32  [nzs][N] : rint(RX_F64 * 65536), row-major by r */
    RCA_TAB_W = 4,        /* float2 [nzs][N] : hann(d pitch, z_r) exp(j 2 pi fc (tau_rx - z_r / c)) */
    RCA_TAB_DMAX = 5,     /* int32  [nzs]    : largest d inside the F-number aperture */
    RCA_TAB_S2_SHIFT = 6, /* double [2K][N]  : Stage-2 shift in slice rows, dz_k(u) us / dz */
    RCA_TAB_S2_PSI = 7,   /* float2 [2K][N]  : exp(j 2 pi fc (1 + cos th) dz_k(u) / c) */
    RCA_TAB_S2_EC = 8,    /* float2 [2K][nz] : exp(j 2 pi fc tau_c,k(z_i)) */
    RCA_TAB_S2_COEF = 9,  /* float2 [2K][S][nz][T]: transverse-slab sum coefficients */
    RCA_TAB_S2_TMIN = 10, /* int32  [2K][S]  : first slice-row offset of the coefficients */
    RCA_TAB_COUNT = 11
} rca_table_id;

/* Size in bytes and up to 4 dimensions (unused = 0) of one table. */
rca_status rca_tables_query(const rca_tables* t, int table_id, size_t* bytes, int dims[4]);
/* Copy one table to host memory (synchronises).  SHAPE if bytes is too small. */
rca_status rca_tables_download(const rca_tables* t, int table_id, void* host_dst, size_t bytes);

/* ---------------------------------------------------------------------- */
/* Beamforming into projection planes (Sec. II-A1, II-A4, II-A5)           */
/* ---------------------------------------------------------------------- */

typedef enum { RCA_MODE_TWO_STAGE = 0, RCA_MODE_DIRECT = 1 } rca_bf_mode;
typedef enum { RCA_CLUTTER_NONE = 0, RCA_CLUTTER_MEAN = 1, RCA_CLUTTER_SVD = 2 } rca_clutter;

typedef struct {
    int mode;      /* rca_bf_mode: TWO_STAGE (the method) or DIRECT (exact slab
                      sums of conventional 3D DAS, no volume; validation and
                      the "what it replaces" baseline) */
    int clutter;   /* rca_clutter: MEAN removes each channel sample's mean over
                      the ensemble's frames before demodulation; SVD (TWO_STAGE
                      only) runs rca_clutter_svd on the Stage-1 slices before
                      Stage 2, as the paper places its filter (Sec. II-A2) */
    int iq_dtype;  /* internal IQ storage: RCA_C32, RCA_C16F or RCA_C16BF */
    int svd_rank;        /* SVD: tissue eigenvectors removed (0 .. 32) */
    int svd_iterations;  /* SVD: orthogonal-iteration steps (0: 30) */
    int reserved[3];
} rca_bf_params;

/* Channel data -> IQ: optional mean clutter removal over the F frames, then
 * demodulation b[n] = 2 sum_m h[m] r~[n-m] exp(-j 2 pi fc t_{n-m}) with a
 * 31-tap half-band Hamming low-pass h (cut-off fs/4).
 *   rf: [F][2K][E][ns] RCA_F32, RCA_F16 or RCA_I16 (then scale[2K][E] float,
 *       value = q * scale); iq: [F][2K][ns][E] RCA_C32 / C16F / C16BF. */
rca_status rca_ingest(rca_handle* h, const rca_tables* t, const void* rf, rca_dtype rf_dtype,
                      const float* scale, int n_frames, int clutter, void* iq, rca_dtype iq_dtype);

/* Stage 1 (Sec. II-A1): one baseband reference slice per transmission,
 *   S_k(l, r) = sum_e w * IQ_{k,e}(tau0) * exp(j 2 pi fc (tau0 - tau_c,k(z_r))),
 *   tau0 = tau_tx(k, 0, z_r) + tau_rx(u_l - u_e, z_r), IQ linear in time and
 *   zero outside the record.  slices: [F][2K][nzs][N] RCA_C32. */
rca_status rca_stage1(rca_handle* h, const rca_tables* t, const void* iq, rca_dtype iq_dtype,
                      int n_frames, void* slices);

/* Stage 2 + block sum-projection (Sec. II-A1, II-A4): each slice is shifted
 * axially by dz_k(u) = u sin th / (1 + cos th), the carrier exp(j 2 pi fc
 * tau_c,k(z')) re-applied, the K transmissions of a family summed and the
 * result sum-projected over P-pixel slabs, written straight to the planes.
 * slices: [F][2K][nzs][N] RCA_C32; planes: RCA_C32, RCA_C16F or RCA_C16BF. */
rca_status rca_stage2_project(rca_handle* h, const rca_tables* t, const void* slices, int n_frames,
                              void* planes, rca_dtype planes_dtype);

/* Exact projection of conventional 3D DAS: every plane pixel sums the DAS
 * voxels of its slab, computed from IQ with no volume (Sec. II-A1's
 * "conventional" path).  iq as for rca_stage1; planes as for stage 2. */
rca_status rca_direct_project(rca_handle* h, const rca_tables* t, const void* iq, rca_dtype iq_dtype,
                              int n_frames, void* planes, rca_dtype planes_dtype);

/* The whole beamforming path: ingest -> Stage 1 -> [SVD clutter filter] ->
 * Stage 2 + projection (or ingest -> direct) using library workspace for IQ
 * and slices.
 *   rf: [F][2K][E][ns] (F32, F16, or I16 + scale[2K][E]); planes as above.
 * Errors: INVALID_ARG / SHAPE / UNSUPPORTED on the host. */
rca_status rca_beamform_projections(rca_handle* h, const rca_tables* t, const void* rf,
                                    rca_dtype rf_dtype, const float* scale, int n_frames,
                                    const rca_bf_params* prm, void* planes, rca_dtype planes_dtype);

/* ---------------------------------------------------------------------- */
/* Localisation (Sec. II-A4, Fig. 1e, Fig. 1g)                             */
/* ---------------------------------------------------------------------- */

typedef enum { ULM_ENH_XDOPPLER = 0, ULM_ENH_COHERENT = 1 } ulm_enhance_mode;

typedef struct {
    int d;            /* NCC kernel length (odd, 3..15; paper 11) */
    float sig_z;      /* Gaussian PSF sigma along z, pixels */
    float sig_lat;    /* Gaussian PSF sigma along the lateral axis, pixels */
    float alpha;      /* amplitude threshold as a fraction of the frame maximum */
    float ncc_min;    /* NCC threshold */
    int enh;          /* ulm_enhance_mode */
    int reserved[4];
} ulm_params;

/* One 2D localisation.  Lists are ordered by (frame, axis, slab, iz, ilat). */
typedef struct {
    int32_t frame, axis, slab;  /* plane */
    int32_t iz, ilat;           /* integer peak pixel */
    float z, lat;               /* sub-pixel position (pixels) */
    float ncc, amp;             /* NCC value and amplitude A at the peak pixel */
    int32_t reserved;
} ulm_loc2d;                    /* 40 bytes */

/* One paired 3D localisation; ordered by i_xz. */
typedef struct {
    int32_t frame, i_xz, i_yz;  /* indices into the 2D list */
    int32_t reserved;
    float x, y, z;              /* x from the XZ entry, y from YZ, z the mean (pixels) */
    float amp_xz, amp_yz;
    float reserved2;
} ulm_loc3d;                    /* 40 bytes */

/* XDoppler enhancement: A_t = sqrt(| sum_{t' = t-1}^{t+1} P_RC,t' conj(P_CR,t') |)
 * over a centred 3-frame window clipped at the ensemble ends (or the
 * coherent |P_RC + P_CR|), and the per-frame maximum M_t of A.
 * planes: [F][2][2][S][nz][N] (C32 / C16F / C16BF); A: [F][2][S][nz][N]
 * float; M: [F] float.  Geometry sizes come from t. */
rca_status ulm_enhance(rca_handle* h, const rca_tables* t, const void* planes, rca_dtype planes_dtype,
                       int n_frames, int enh, float* A, float* M);

/* NCC against the d x d Gaussian PSF via separable 1D correlations, then
 * sub-pixel 3x3 regional peaks with NCC >= ncc_min and A >= alpha M_t (ties
 * to the earlier raster pixel), parabolic sub-pixel refinement.
 *   out: capacity cap2d; *n2d_dev (device int) receives the true count even
 *   when it exceeds cap2d (then the status word gets CAPACITY).
 *   ncc_out: optional [F][2][S][nz][N] float copy of the NCC maps (NULL = none).
 *   plane_offsets: optional device int [F*2*S + 1] list offset of each plane. */
rca_status ulm_detect2d(rca_handle* h, const rca_tables* t, const float* A, const float* M,
                        int n_frames, const ulm_params* prm, ulm_loc2d* out2d, int cap2d,
                        int* n2d_dev, float* ncc_out, int* plane_offsets);

/* Pair XZ and YZ localisations into 3D (sub-block membership by integer
 * pixel, |z_xz - z_yz| <= 1 pixel, I_xz / I_yz in [0.9, 1.11], mutual minimum
 * of max(I)/min(I), ties to the lower index; decisions in double precision).
 *   list2d: sorted as ulm_detect2d writes it; n2d_dev: device count (entries
 *   beyond cap2d are ignored).  out3d: capacity cap3d; *n3d_dev true count. */
rca_status ulm_pair3d(rca_handle* h, const rca_tables* t, const ulm_loc2d* list2d, const int* n2d_dev,
                      int cap2d, int n_frames, ulm_loc3d* out3d, int cap3d, int* n3d_dev);

/* ulm_pair3d without allocation.  The paper has no counterpart: this entry
 * point serves callers that must not allocate device memory once they are
 * running.  An acquisition loop that sized its memory before the first
 * ensemble cannot take the device-wide stall of an allocation, or its
 * failure, in the middle of a scan; a program whose own memory pool already
 * holds the free device memory would see an allocation fail.  ulm_pair3d
 * takes its scratch from the handle's workspace, which grows with cudaMalloc
 * when a longer list arrives; this call uses a fixed scratch array compiled
 * into the library instead (ULM_PAIR3D_NOALLOC_SCRATCH_BYTES, 6.3 MiB, one
 * per device) and allocates nothing.
 *   Arguments, results and status rules: as ulm_pair3d (same kernels, same
 *   lists bit for bit), with two limits: cap2d <= ULM_PAIR3D_NOALLOC_MAX_2D
 *   and n_frames * 2 * S <= ULM_PAIR3D_NOALLOC_MAX_PLANES.  Beyond them it
 *   returns RCA_ERR_UNSUPPORTED (message in rca_last_error) before anything
 *   is enqueued.
 *   Set-up: the first call on a device looks up the array's device address
 *   with that device current, which can make the CUDA runtime load the
 *   library's device code; make that first call before any stream capture.
 *   The address is kept for the life of the process: after cudaDeviceReset
 *   (or a reset of the device's primary context) the kept address is stale,
 *   so do not call this entry point again on that device in this process.
 *   Sharing: every handle and every call on a device uses the one array.
 *   Calls in order on one stream are fine (each call writes every scratch
 *   entry it reads, so nothing is cleared or carried over); calls whose work
 *   overlaps on the GPU (two streams, two threads) race and give wrong lists. */
#define ULM_PAIR3D_NOALLOC_MAX_2D (1 << 19)
#define ULM_PAIR3D_NOALLOC_MAX_PLANES (1 << 16)
#define ULM_PAIR3D_NOALLOC_SCRATCH_BYTES 6556160
rca_status ulm_pair3d_noalloc(rca_handle* h, const rca_tables* t, const ulm_loc2d* list2d, const int* n2d_dev,
                              int cap2d, int n_frames, ulm_loc3d* out3d, int cap3d, int* n3d_dev);

/* The whole localisation path: ulm_enhance -> ulm_detect2d -> ulm_pair3d with
 * library workspace for A and M. */
rca_status ulm_localize(rca_handle* h, const rca_tables* t, const void* planes, rca_dtype planes_dtype,
                        int n_frames, const ulm_params* prm, ulm_loc2d* out2d, int cap2d, int* n2d_dev,
                        ulm_loc3d* out3d, int cap3d, int* n3d_dev);

/* ---------------------------------------------------------------------- */
/* Eigen-based SVD clutter filter on the Stage-1 slices (Sec. II-A2)       */
/* ---------------------------------------------------------------------- */

/* In place on slices [F][2K][nzs][N] C32 (as rca_stage1 writes them; use
 * slices of channel data ingested with RCA_CLUTTER_NONE).  For each
 * transmission k the frames' slices are the columns of the Casorati matrix
 * X_k (nzs N pixels x F frames); the filter removes the subspace of the
 * `rank` largest eigenvalues of the frame covariance C_k = X_k^H X_k:
 * X_k <- X_k - X_k Q Q^H, Q an orthonormal basis of that subspace found by
 * `iterations` steps of orthogonal iteration Q <- orth(C_k Q) from fixed
 * start vectors (the projection depends on the subspace only).  The paper
 * gives no rank or threshold: `rank` is the caller's (0 leaves the slices
 * unchanged).  FP32 arithmetic throughout.
 *   Limits: rank in [0, 32] and below F; iterations in [1, 1000]
 *   (INVALID_ARG); F x (rank + 2) complex values twice must fit the
 *   eigenspace kernel's shared memory (F (rank + 2) <= 12 800, UNSUPPORTED). */
rca_status rca_clutter_svd(rca_handle* h, const rca_tables* t, void* slices, int n_frames, int rank, int iterations);

/* rca_clutter_svd plus a report of how well the removed subspace is
 * determined (Sec. II-A2 removes the leading eigenvectors; whether FP32
 * arithmetic resolves them depends on the spectrum).  The iteration carries
 * one vector beyond the rank (when F allows); after the last step, with
 * Q the removed basis and q' the extra vector, per transmission k:
 *   info[4k + 0]  largest Rayleigh quotient q_j^H C_k q_j over the removed j
 *   info[4k + 1]  smallest such quotient (the rank-th eigenvalue, when converged)
 *   info[4k + 2]  q'^H C_k q' (the next eigenvalue, when converged; 0 if F
 *                 leaves no room for the extra vector)
 *   info[4k + 3]  ||C_k Q - Q (Q^H C_k Q)||_F / info[4k + 1]: zero for an
 *                 exactly invariant subspace.
 * The split between the removed and the kept subspace is determined by the
 * FP32 covariance only where (info[1] - info[2]) / info[0] is well above
 * the covariance's relative rounding (about 1e-7 here); where it is not,
 * info[3] stays large for any iteration count and the removed subspace
 * differs from the exact one among the eigenvectors near the split.
 * info: caller-owned device array [2K][4] floats, written on the stream
 * before the projection (zeros at rank 0).  Other arguments and errors as
 * rca_clutter_svd; a null info is INVALID_ARG. */
rca_status rca_clutter_svd_info(rca_handle* h, const rca_tables* t, void* slices, int n_frames, int rank,
                                int iterations, float* info);

/* ---------------------------------------------------------------------- */
/* Microbubble separation on the projection planes (Sec. II-A5, Fig. 1c)   */
/* ---------------------------------------------------------------------- */

#define ULM_SEP_MAX_BANDS 4

/* Speed bands of the separation.  Bin j of the F-point slow-time DFT has the
 * signed index k = j (2 j < F) or j - F (2 j > F) and the Doppler frequency
 * k prf_hz / F; band b holds the bins with
 *   edges_hz[b] < |k| prf_hz / F <= edges_hz[b + 1]      (b < n_bands),
 * evaluated in double precision.  k > 0 (flow toward the array, decreasing
 * depth: the planes' phase grows as the echo delay shrinks) is "up", k < 0
 * "down"; DC and, for even F, the Nyquist bin belong to no subset.  The
 * paper separates into three speed ranges and two directions but prints no
 * band edges: equal bands over (0, prf/2] are edges_hz[i] = i prf / (2 n). */
typedef struct {
    double prf_hz;                            /* frame rate (Hz, > 0) */
    int32_t n_bands;                          /* 1 .. ULM_SEP_MAX_BANDS (paper: 3) */
    int32_t reserved;
    double edges_hz[ULM_SEP_MAX_BANDS + 1];   /* n_bands + 1 increasing edges, edges_hz[0] >= 0 */
} ulm_sep_params;

/* Subsets of the planes: for every plane pixel, the F-frame signal is
 * transformed, each subset keeps its bins (rectangular mask) and is
 * transformed back (1/F on the inverse).  Subset index = direction n_bands +
 * band, direction 0 up, 1 down.
 *   planes: [F][2][2][S][nz][N] (C32 / C16F / C16BF); subsets: device
 *   [2 n_bands][F][2][2][S][nz][N] C32.  FP32 transforms.
 * Limits: F <= 512 with prime factors 2, 3 and 5 only (UNSUPPORTED
 * otherwise); bad bands or prf: INVALID_ARG. */
rca_status ulm_separate(rca_handle* h, const rca_tables* t, const void* planes, rca_dtype planes_dtype, int n_frames,
                        const ulm_sep_params* prm, void* subsets);

/* Separation fused with each subset's enhancement: the subsets are never
 * stored; for each subset the XDoppler (or coherent) amplitude of
 * ulm_enhance and its per-frame maxima are written, ready for ulm_detect2d
 * on A + s F 2 S nz N and M + s F.
 *   A: device [2 n_bands][F][2][S][nz][N] float; M: device [2 n_bands][F]
 *   float.  Limits as ulm_separate; enh as ulm_enhance. */
rca_status ulm_separate_enhance(rca_handle* h, const rca_tables* t, const void* planes, rca_dtype planes_dtype,
                                int n_frames, const ulm_sep_params* prm, int enh, float* A, float* M);

/* ---------------------------------------------------------------------- */
/* Projection-based rigid motion estimation (Sec. II-A3, Fig. 1d)          */
/* ---------------------------------------------------------------------- */

/* Rigid displacement of every frame against frame 0 from the Stage-1 slices.
 * For each transmission k, slice k of frame f and of frame 0 are
 * zero-padded to Zp x N (Zp: next power of two >= nzs) and correlated by 2D
 * FFT: R = IFFT2(FFT2(S_f) conj(FFT2(S_0))), R[dz, dx] = sum_p S_f[p + (dz,
 * dx)] conj(S_0[p]) (circular).  The displacement is the peak of |R| (first
 * in row-major order on ties; indices at or past half the padded size are
 * negative), refined per axis by a 3-point parabola through |R| at the peak
 * and its circular neighbours (clamped to +-1/2, none when not concave).
 * RC transmissions (k < K) resolve (x, z), CR (k >= K) resolve (y, z); each
 * family is averaged over its K transmissions and the two combine into
 * motion[f] = (x_RC pitch, y_CR pitch, (z_RC + z_CR) / 2 dz / us) metres.
 *   slices: [F][2K][nzs][N] C32 (as rca_stage1 writes them; pass unfiltered
 *   slices, whose tissue carries the motion).  motion: device [F][3] float.
 *   shifts (nullable): device [F][2K][3] float (z in slice rows, x in
 *   lateral pixels, NCC = |R| / (||S_f|| ||S_0||) at the peak).  peaks
 *   (nullable): device [F][2K][2] int, the integer (dz, dx).
 * Limits: N a power of two in [32, 256], nzs <= 512 (UNSUPPORTED beyond). */
rca_status rca_motion_estimate(rca_handle* h, const rca_tables* t, const void* slices, int n_frames, float* motion,
                               float* shifts, int* peaks);

/* ---------------------------------------------------------------------- */
/* Fixed-length tracking and accumulation (Sec. II-A6, Fig. 1f)            */
/* ---------------------------------------------------------------------- */

/* Tracking parameters.  The paper keeps MBs tracked across ten consecutive
 * volumes, smooths each track by a least-squares quadratic and drops tracks
 * whose direction changes by more than 45 degrees or whose speed changes by
 * more than half their mean speed (Sec. II-A6). */
typedef struct {
    int32_t len;               /* points per track (10); 2 .. ULM_TRACK_MAX_LEN */
    int32_t substeps;          /* density samples per frame interval (>= 1) */
    double max_step_m;         /* link radius between consecutive frames (metres, > 0) */
    double cos_max_turn;       /* cosine of the largest direction change kept (cos 45 deg) */
    double max_speed_change;   /* largest (max - min) smoothed segment speed kept, as a fraction of the mean (0.5) */
    double voxel_m;            /* density grid spacing (metres, > 0) */
} ulm_track_params;
#define ULM_TRACK_MAX_LEN 64

/* One fixed-length track. */
typedef struct {
    int32_t first;             /* track id: 3D-list index of its first point */
    int32_t frame0;            /* frame of the first point */
    int32_t accepted;          /* 1: kept by the turn and speed tests */
    int32_t reserved;
    double a[3][3];            /* per axis x, y, z (metres): least-squares quadratic in the basis
                                  1, tau - m, (tau - m)^2 - (len^2 - 1)/12, tau = 0 .. len-1, m = (len-1)/2 */
    double mean_speed;         /* mean smoothed segment length (metres per frame) */
    double cos_turn;           /* cosine of the angle between the first and last smoothed segment (-2: undefined) */
    double speed_range;        /* max - min smoothed segment length (metres per frame) */
} ulm_track_rec;               /* 112 bytes */

/* Density grid of a geometry: dims = {nx, ny, nz} voxels of voxel_m covering
 * the N lateral pixels (x, y from -N pitch / 2) and the nz depth rows (from
 * z0 - dz / 2); the grid is [nz][ny][nx] uint32. */
rca_status ulm_density_shape(const rca_tables* t, double voxel_m, int32_t dims[3]);

/* Fixed-length tracking of a 3D localisation list (Sec. II-A6).  Positions
 * in metres: x, y -> (p - (N-1)/2) pitch, z -> z0 + p dz.
 *  1. Pairing of consecutive frames: i (frame t) and j (frame t + 1) are
 *     linked when each is the other's nearest neighbour within max_step_m
 *     (ties to the lower index) -- a one-to-one matching of the two frames.
 *  2. Every localisation starts a search; it becomes a track when its chain
 *     of links reaches len points (tracks may overlap in time).
 *  3. Least-squares quadratic per axis; rejection as in ulm_track_params;
 *     a track with zero mean speed is rejected.
 *  4. If density is non-NULL, every accepted track written to out, sampled
 *     at tau = s / substeps (s = 0 .. (len-1) substeps), adds 1 to the voxel
 *     holding each sample (accumulated INTO density: zero it first, or sum
 *     ensembles).
 * All decisions and coefficients in double precision.
 *   list3d: frame-major (as ulm_pair3d writes it); *n3d_dev: its length
 *   (entries beyond cap3d ignored).  out: capacity cap_tracks, tracks in
 *   order of their first point; *n_tracks_dev (device int) receives the true
 *   count (beyond cap_tracks: status word CAPACITY).  density: device
 *   [nz][ny][nx] uint32 as from ulm_density_shape.
 * Host-side errors: invalid parameters or sizes (INVALID_ARG) before any launch. */
rca_status ulm_track(rca_handle* h, const rca_tables* t, const ulm_loc3d* list3d, const int* n3d_dev, int cap3d,
                     int n_frames, const ulm_track_params* prm, ulm_track_rec* out, int cap_tracks, int* n_tracks_dev,
                     uint32_t* density);

/* Velocity volumes of the tracks ulm_track wrote (Sec. II-C: density and
 * velocity volumes): at every accumulation sample of an accepted track (the
 * samples and voxels of the density), the smoothed track's velocity is the
 * derivative of its quadratic, v = a1 + 2 a2 phi1(tau) per axis (metres per
 * frame interval); the voxel adds |v| and v_z (positive = deeper), each
 * rounded to a whole nanometre per frame interval, to two 64-bit integer sums
 * (exact in any order).  Mean speed of a voxel = speed_sum / density count x
 * frame rate (m/s).  Accumulated INTO the sums (zero them first).
 *   tracks, *n_tracks_dev, cap_tracks: as ulm_track wrote them; prm: the same
 *   parameters; speed_sum, vz_sum: device int64 [nz][ny][nx] (ulm_density_shape).
 * Host-side errors: invalid parameters or sizes (INVALID_ARG). */
rca_status ulm_track_velocity(rca_handle* h, const rca_tables* t, const ulm_track_rec* tracks, const int* n_tracks_dev,
                              int cap_tracks, const ulm_track_params* prm, int64_t* speed_sum, int64_t* vz_sum);

/* ---------------------------------------------------------------------- */
/* Learned localiser (the paper's future-work form, Sec. IV)               */
/* ---------------------------------------------------------------------- */

/* conv3x3(1->C)+ReLU, conv3x3(C->C)+ReLU x2, conv3x3(C->16), pixel shuffle
 * to a 4x heatmap; BF16 tensor-core kernels with FP32 accumulation and FP32
 * master weights, MSE loss against Gaussian targets, Adam. */
typedef struct ulm_cnn ulm_cnn;

typedef struct {
    int channels;        /* C (only 32 is built) */
    int max_pixels;      /* largest batch * H * W the network will see */
    float lr, beta1, beta2, eps;  /* Adam (1e-3, 0.9, 0.999, 1e-8) */
    unsigned long long seed;      /* He-normal initial weights */
} ulm_cnn_desc;

/* Parameter vector (FP32, host order): w1 [C][9][1], b1 [C], w2 [C][9][C],
 * b2, w3 [C][9][C], b3, w4 [16][9][C], b4 [16]; tap = 3 (dy+1) + (dx+1). */
rca_status ulm_cnn_create(rca_handle* h, const ulm_cnn_desc* desc, ulm_cnn** out);
rca_status ulm_cnn_destroy(ulm_cnn* c);
rca_status ulm_cnn_param_count(const ulm_cnn* c, size_t* n);
/* copy parameters from host memory (resets the Adam state; synchronises) */
rca_status ulm_cnn_set_params(ulm_cnn* c, const float* host, size_t n);
/* copy parameters / the last step's gradients to host memory (synchronises) */
rca_status ulm_cnn_get_params(const ulm_cnn* c, float* host, size_t n);
rca_status ulm_cnn_get_grads(const ulm_cnn* c, float* host, size_t n);

/* Forward pass.  Input plane b is A[b][H][W] / M[b / planes_per_frame]
 * (M NULL: A as is); heat: [B][4H][4W] float (device). */
rca_status ulm_cnn_forward(ulm_cnn* c, const float* A, const float* M, int planes_per_frame, int B, int H, int W,
                           float* heat);

/* Inference: the same computation as ulm_cnn_forward (the name of the
 * learned form's inference step). */
rca_status ulm_cnn_infer(ulm_cnn* c, const float* A, const float* M, int planes_per_frame, int B, int H, int W,
                         float* heat);

/* One training step on a batch: forward, MSE against target [B][4H][4W],
 * backward (gradients kept for ulm_cnn_get_grads) and, if apply_update, an
 * Adam update.  loss_dev: device float receiving the mean squared error. */
rca_status ulm_cnn_train_step(ulm_cnn* c, const float* A, const float* M, int planes_per_frame, int B, int H, int W,
                              const float* target, float* loss_dev, int apply_update);

/* Gaussian training targets: target[b][y][x] = sum over the points of plane
 * b of exp(-((y - z4)^2 + (x - x4)^2) / (2 sigma^2)).  pts: [n][3] device
 * floats (plane, z4, x4) sorted by plane; target: [B][H4][W4]. */
rca_status ulm_cnn_target(rca_handle* h, const float* pts, int n, int B, int H4, int W4, float sigma, float* target);

/* Checkpoint (weights and Adam state) to / from a file (synchronises). */
rca_status ulm_cnn_save(const ulm_cnn* c, const char* path);
rca_status ulm_cnn_load(ulm_cnn* c, const char* path);

/* 2D localisations from score maps on an up-times finer grid (the CNN
 * heatmap): a fine pixel is a localisation iff its score >= score_min,
 * A >= alpha M_t at the plane pixel that contains it, and it is a 3x3
 * regional maximum (ties to the earlier raster pixel); parabolic sub-pixel
 * refinement.  Positions are returned in plane pixels, (fine - (up-1)/2)/up;
 * iz / ilat are the plane pixel; amp = A there; ncc = the score.
 *   map: [F][2][S][up nz][up N]; A, M as from ulm_enhance.  Output as for
 *   ulm_detect2d (same order and capacity rules), ready for ulm_pair3d. */
rca_status ulm_detect_map(rca_handle* h, const rca_tables* t, const float* map, int up, const float* A, const float* M,
                          int n_frames, float score_min, float alpha, ulm_loc2d* out2d, int cap2d, int* n2d_dev);

/* ---------------------------------------------------------------------- */
/* Batched form and launch-shape autotuning                                */
/* ---------------------------------------------------------------------- */

typedef struct rca_batch rca_batch;

/* One ensemble of a batch.  Buffers are caller-owned device memory and must
 * stay valid (and at the same address) for the life of the batch plan. */
typedef struct {
    const rca_tables* tables;  /* the ensemble's geometry (ensembles may differ in K) */
    const void* rf;            /* [F][2K][E][ns] channel data, dtype of the batch */
    const float* scale;        /* [2K][E] per-channel scale when the batch rf dtype is RCA_I16 */
    int n_frames;              /* F */
    void* planes;              /* [F][2][2][S][nz][N] output planes, dtype of the batch */
    ulm_loc2d* out2d;          /* localisation outputs (used when the batch has ulm_params) */
    int cap2d;
    int* n2d_dev;
    ulm_loc3d* out3d;
    int cap3d;
    int* n3d_dev;
} rca_batch_item;

/* Plan a batch of n ensembles of uneven frame counts and transmission sets.
 * Beamforming of the whole batch (mean clutter removal, demodulation,
 * Stage 1, Stage 2 + projection) runs by default as ONE persistent launch
 * (see rca_batch_set_mode for one launch per stage instead): a device
 * work queue of units, ordered so that every unit only waits for earlier
 * ones through per-ensemble completion counters (bounded waits: a wait that
 * runs out sets RCA_ERR_TIMEOUT in the status word and stops the launch).
 * With prm non-NULL each ensemble is then localised (ulm_localize).
 * Allocates the per-ensemble IQ and slice workspace (owned by the plan).
 * Errors: INVALID_ARG / SHAPE / UNSUPPORTED on the host. */
rca_status rca_batch_create(rca_handle* h, int n, const rca_batch_item* items, rca_dtype rf_dtype,
                            rca_dtype iq_dtype, rca_dtype planes_dtype, const ulm_params* prm, rca_batch** out);

/* Enqueue one run of the batch on the handle's stream.  use_graph != 0:
 * the first call runs the batch once, then captures it into a CUDA graph
 * (on a private stream); every call launches that graph. */
rca_status rca_batch_run(rca_batch* b, int use_graph);

/* One-shot form of the batch plan: rca_batch_create, one rca_batch_run
 * without a graph, a synchronisation of the handle's stream and
 * rca_batch_destroy.  Same items and errors as rca_batch_create; the IQ is
 * kept as RCA_C32.  Synchronises (the plan's workspace is freed); for
 * repeated batches build the plan once and run it (optionally as a graph). */
rca_status rca_beamform_projections_batched(rca_handle* h, int n, const rca_batch_item* items, rca_dtype rf_dtype,
                                            rca_dtype planes_dtype, const ulm_params* prm);

/* Launch mode of later runs.  RCA_BATCH_PERSISTENT (the default): the whole
 * beamforming as one persistent launch with the dependency-ordered queue
 * described at rca_batch_create.  RCA_BATCH_STAGED: one launch per stage
 * (mean, demodulation, Stage 1, Stage 2), each over the units of that stage
 * of every ensemble, sized by that stage's shared memory; the stream orders
 * the stages, so no unit waits.  Same bodies, same results bit for bit.
 * Discards a captured graph (the next rca_batch_run with use_graph captures
 * again).  Errors: INVALID_ARG. */
#define RCA_BATCH_PERSISTENT 0
#define RCA_BATCH_STAGED 1
rca_status rca_batch_set_mode(rca_batch* b, int mode);

/* Bound of every dependency wait in the persistent launch, in SM clock
 * cycles (default ~4e9).  block_ensemble >= 0 makes that ensemble's Stage-1
 * units wait for one demodulation unit that never exists -- a host-built
 * impossible queue used to test that the launch ends with RCA_ERR_TIMEOUT. */
rca_status rca_batch_set_wait_limit(rca_batch* b, long long cycles, int block_ensemble);

rca_status rca_batch_destroy(rca_batch* b);

/* Time the Stage-1 (row tile x distance chunk) and Stage-2 (plane-row tile)
 * launch shapes that fit shared memory on the given IQ (n_frames frames of
 * t's geometry, RCA_C32 / C16F / C16BF) and keep the fastest in t.
 * Synchronises.  zt, dc, zp (optional) receive the chosen shapes. */
rca_status rca_autotune(rca_handle* h, rca_tables* t, const void* iq, rca_dtype iq_dtype, int n_frames,
                        int* zt, int* dc, int* zp);

/* ---------------------------------------------------------------------- */
/* Measurement aid (no counterpart in the paper)                           */
/* ---------------------------------------------------------------------- */

/* FP32 issue-rate probe: the denominator of an FP32 roofline, measured on
 * this device rather than derived from a clock and a lane count.  Enqueues
 * one launch that fills every SM (8 CTAs of 256 threads each), every thread
 * running 16 independent chains of `iterations` dependent FP32 FMAs
 * (packed = 0: scalar fma.rn.f32; packed = 1: eight chains of packed
 * fma.rn.f32x2 pairs, the same 16 FMAs).  The caller times the launch on the
 * handle's stream.  sink: caller-owned device buffer of at least
 * 8 x (SM count) floats, written only by a chain whose result hits a value
 * no chain reaches (it keeps the work live).  *flops (host, optional) gets
 * 2 x 16 x iterations x threads, the launch's FP32 operations.
 *   Errors: iterations outside [1, 1 << 24] or a null sink: INVALID_ARG. */
rca_status rca_fp32_probe(rca_handle* h, int packed, int iterations, float* sink, double* flops);

#ifdef __cplusplus
}
#endif
#endif /* RCA_H */
