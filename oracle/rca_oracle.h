/*
 * rca_oracle.h -- FP64 CPU oracle for projection-based RCA beamforming and
 * NCC microbubble localisation.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this code.  It shares nothing with the
 * CUDA library (no headers, tables or helpers); both sides read the same
 * seeded inputs and nothing else.
 *
 * Everything is plain loops in double precision, written to be checked
 * against the paper by eye:
 *   Sec. II-A1 (two-stage RCA beamforming, Fig. 1b-c), Sec. II-A4 (block
 *   sum-projection, separable NCC with a Gaussian PSF, XZ/YZ pairing),
 *   Sec. II-C (acquisition constants), Fig. 1g (separable NCC).
 * Where the paper is silent the reading is stated at the function.
 *
 * Array layouts (row-major, complex = interleaved re,im):
 *   rf      [F][2K][E][ns]               real
 *   iq      [F][2K][E][ns][2]            baseband IQ
 *   S       [2K][nzs][N][2]              Stage-1 reference slices of one frame,
 *                                        nzs = (nz-1)*us + 1
 *   V       [N(x)][N(y)][nz][2]          one family's volume of one frame
 *   planes  [F][2 axis][2 fam][S][nz][N][2]  axis 0 = XZ (slab over y, lateral x),
 *                                            axis 1 = YZ (slab over x, lateral y);
 *                                            fam 0 = RC, fam 1 = CR
 *   A       [F][2 axis][S][nz][N]        XDoppler amplitude
 */
#ifndef RCA_ORACLE_H
#define RCA_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

#define OR_MAX_K 8
#define OR_FIR_TAPS 31

typedef struct {
    int n_el;      /* elements per array (rows = columns) = lateral pixels N */
    int nz;        /* axial pixels */
    int ns;        /* samples per channel */
    int P;         /* slab thickness in pixels (Sec. II-C: 8) */
    int K;         /* transmissions per family (RC and CR) */
    int us;        /* Stage-1 axial oversampling: slices have (nz-1)*us+1 rows
                      at depth z0 + r dz/us (the paper's slice pixel is finer
                      axially than its volume voxel, Sec. II-C) */
    double pitch, fc, fs, c, z0, dz, fnum;
    double ang[2 * OR_MAX_K]; /* first K: RC angles, next K: CR angles (rad) */
} or_geom;

typedef struct {
    int frame, axis, slab, iz, ilat;
    double z, lat, ncc, amp;
} or_loc2d;

typedef struct {
    int frame, i_xz, i_yz;
    double x, y, z, amp_xz, amp_yz;
} or_loc3d;

/* geometry definitions (Sec. II-A1, Sec. II-C) */
double or_elem_pos(const or_geom* g, int e);
double or_depth(const or_geom* g, int i);
double or_slice_depth(const or_geom* g, int r);
int or_slice_rows(const or_geom* g);
double or_t0(const or_geom* g);
double or_tau_tx(const or_geom* g, int k, double trans, double z);
double or_tau_rx(const or_geom* g, double lat_off, double z);
double or_apod(const or_geom* g, double lat_off, double z);
double or_tau_c(const or_geom* g, int k, double z);
double or_shift_dz(const or_geom* g, int k, double u);

/* RF -> IQ (mean clutter removal + demodulation).  The mean always runs over
 * all F frames; IQ is produced for the n_sel frames listed in sel (all F
 * frames, in order, when sel is NULL), iq [n_sel][2K][E][ns][2]. */
void or_fir_taps(double h[OR_FIR_TAPS]);
void or_demod(const or_geom* g, int F, const float* rf, int remove_mean, int n_sel, const int* sel,
              double* iq);

/* conventional full 3D DAS of one family, one frame */
void or_das_volume(const or_geom* g, const double* iq_frame, int fam, double* V);
/* block sum-projection of a family volume into planes_frame[axis][fam] */
void or_project_volume(const or_geom* g, const double* V, int fam, double* planes_frame);
/* exact projection of the full 3D DAS computed per plane pixel (no volume) */
void or_project_direct(const or_geom* g, const double* iq_frame, int fam, double* planes_frame);

/* two-stage beamforming */
void or_stage1(const or_geom* g, const double* iq_frame, double* S);
void or_stage2_volume(const or_geom* g, const double* S, int fam, double* V);
void or_stage2_project(const or_geom* g, const double* S, double* planes_frame);

/* localisation */
void or_xdoppler(int F, int S, int nz, int N, const double* planes, double* A, double* M);
void or_ncc_plane(int nz, int N, const double* A, int d, double sig_z, double sig_l,
                  double Mt, double* ncc);
int or_peaks_plane(int nz, int N, const double* A, const double* ncc, double Mt,
                   double alpha, double ncc_min, int cap, or_loc2d* out);
int or_localize2d(int F, int S, int nz, int N, const double* A, const double* M,
                  int d, double sig_z, double sig_l, double alpha, double ncc_min,
                  int cap, or_loc2d* out);
int or_pair3d(int n2d, const or_loc2d* list, int P, int cap, or_loc3d* out);

/* OpenMP thread count of the loops (timing only). */
void or_set_threads(int n);
int or_max_threads(void);

/* fixed-length tracking and accumulation (Sec. II-A6, Fig. 1f) */
typedef struct {
    int len;                  /* points per track (the paper: ten consecutive volumes) */
    int substeps;             /* accumulation samples per frame interval */
    double max_step;          /* link radius between consecutive frames (m) */
    double cos_max_turn;      /* cosine of the largest direction change kept (45 deg) */
    double max_speed_change;  /* largest (max - min) segment speed kept, fraction of the mean (0.5) */
    double voxel;             /* density grid spacing (m) */
} or_track_params;

typedef struct {
    int first;                /* track id: list index of the first point */
    int frame0;               /* its frame */
    int accepted;             /* 1 if the turn and speed tests pass */
    double a[3][3];           /* per axis x, y, z: coefficients of 1, phi1(tau), phi2(tau) (m) */
    double mean_speed;        /* mean smoothed segment length (m per frame) */
    double cos_turn;          /* cosine of the angle between the first and last segment */
    double speed_range;       /* max - min smoothed segment length (m per frame) */
} or_track;

void or_track_link(const or_geom* g, int n, const int* frame, const double* x, const double* y, const double* z,
                   double max_step, int* succ);
int or_track_build(const or_geom* g, int n, const int* frame, const double* x, const double* y, const double* z,
                   const int* succ, const or_track_params* prm, int cap, or_track* out);
void or_track_grid(const or_geom* g, double voxel, int dims[3]);
void or_track_accumulate(const or_geom* g, int ntr, const or_track* tr, const or_track_params* prm,
                         unsigned* grid);
void or_track_velocity(const or_geom* g, int ntr, const or_track* tr, const or_track_params* prm,
                       long long* speed_sum, long long* vz_sum);

#ifdef __cplusplus
}
#endif
#endif
