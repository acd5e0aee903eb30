// Fixed-length tracking, quadratic smoothing, rejection and accumulation of
// 3D localisations (Sec. II-A6, Fig. 1f).
//
// One thread per localisation throughout, as the paper assigns one thread
// per MB:
//   k_track_offsets   frame boundaries of the frame-major 3D list
//   k_track_link      each localisation's nearest neighbour in the next and
//                     in the previous frame within the link radius
//   k_track_build     follow the mutual-nearest links len - 1 times; fit the
//                     least-squares quadratic, apply the turn and speed tests
//   k_track_scan / k_track_write   compaction in order of the first point
//   k_track_accumulate one thread per (track, sample): density counts
//   k_track_velocity   one thread per (track, sample): velocity sums (speed and
//                      axial component, whole nanometres per frame interval)
// Every decision and coefficient is computed in double precision with the
// operations in a fixed order; this unit is compiled without fused
// multiply-add contraction, so each double result rounds exactly as written.
#include <algorithm>
#include <cmath>

#include "rca_internal.cuh"

namespace {

#define TR_THREADS 256

struct TrackConst {
    double half_span;      // (N - 1) / 2 pixels
    double pitch, dz, z0;
    double r2;             // link radius squared
    double m, q;           // basis centre (len - 1) / 2 and (len^2 - 1) / 12
    double n1, n2;         // sums of phi1^2 and phi2^2 over tau = 0 .. len - 1
    double lo[3];          // grid origin
    double voxel;
    double cos_max_turn, max_speed_change;
    int dims[3];
    int len, substeps;
};

__device__ __forceinline__ void tr_pos(const TrackConst& c, const ulm_loc3d& p, double v[3])
{
    v[0] = ((double)p.x - c.half_span) * c.pitch;
    v[1] = ((double)p.y - c.half_span) * c.pitch;
    v[2] = c.z0 + (double)p.z * c.dz;
}

__device__ __forceinline__ double tr_d2(const double a[3], const double b[3])
{
    const double dx = a[0] - b[0], dy = a[1] - b[1], dz = a[2] - b[2];
    return dx * dx + dy * dy + dz * dz;
}

// offs[f] = first list index with frame >= f, f = 0 .. F + 1 (binary search;
// the list is frame-major)
__global__ void k_track_offsets(const ulm_loc3d* __restrict__ L, const int* __restrict__ n3d, int cap3d, int F,
                                int* __restrict__ offs)
{
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f > F + 1) return;
    const int n = min(max(*n3d, 0), cap3d);
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (L[mid].frame < f) lo = mid + 1;
        else hi = mid;
    }
    offs[f] = lo;
}

// nearest neighbour of i among [j0, j1) within the link radius (ties to the lower index)
__device__ __forceinline__ int tr_nearest(const TrackConst& c, const ulm_loc3d* __restrict__ L, const double pi[3],
                                          int j0, int j1)
{
    int best = -1;
    double bd = 0.0;
    for (int j = j0; j < j1; ++j) {
        double pj[3];
        tr_pos(c, L[j], pj);
        const double d2 = tr_d2(pi, pj);
        if (d2 <= c.r2 && (best < 0 || d2 < bd)) {
            best = j;
            bd = d2;
        }
    }
    return best;
}

__global__ void k_track_link(TrackConst c, const ulm_loc3d* __restrict__ L, const int* __restrict__ n3d, int cap3d,
                             int F, const int* __restrict__ offs, int* __restrict__ nxt, int* __restrict__ prv)
{
    const int n = min(max(*n3d, 0), cap3d);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int t = L[i].frame;
        double pi[3];
        tr_pos(c, L[i], pi);
        nxt[i] = (t >= 0 && t + 1 < F) ? tr_nearest(c, L, pi, offs[t + 1], offs[t + 2]) : -1;
        prv[i] = (t >= 1 && t <= F) ? tr_nearest(c, L, pi, offs[t - 1], offs[t]) : -1;
    }
}

__global__ void k_track_build(TrackConst c, const ulm_loc3d* __restrict__ L, const int* __restrict__ n3d, int cap3d,
                              const int* __restrict__ nxt, const int* __restrict__ prv, ulm_track_rec* __restrict__ rec,
                              int* __restrict__ flag)
{
    const int n = min(max(*n3d, 0), cap3d);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int idx[ULM_TRACK_MAX_LEN];
        idx[0] = i;
        bool ok = true;
        for (int s = 1; s < c.len && ok; ++s) {
            const int j = nxt[idx[s - 1]];
            ok = j >= 0 && prv[j] == idx[s - 1];
            idx[s] = ok ? j : -1;
        }
        flag[i] = ok ? 1 : 0;
        if (!ok) continue;
        ulm_track_rec tr;
        tr.first = i;
        tr.frame0 = L[i].frame;
        tr.reserved = 0;
        for (int ax = 0; ax < 3; ++ax) {
            double s0 = 0.0, s1 = 0.0, s2 = 0.0;
            for (int t = 0; t < c.len; ++t) {
                double p[3];
                tr_pos(c, L[idx[t]], p);
                const double f1 = (double)t - c.m, f2 = f1 * f1 - c.q;
                s0 += p[ax];
                s1 += p[ax] * f1;
                s2 += p[ax] * f2;
            }
            tr.a[ax][0] = s0 / (double)c.len;
            tr.a[ax][1] = s1 / c.n1;
            tr.a[ax][2] = s2 / c.n2;
        }
        // smoothed segment s -> s + 1: a1 + a2 (2 (s - m) + 1)
        double vf[3] = {0.0, 0.0, 0.0}, vl[3] = {0.0, 0.0, 0.0}, sum = 0.0, vmax = 0.0, vmin = 0.0;
        for (int s = 0; s + 1 < c.len; ++s) {
            double v[3];
            const double dphi2 = 2.0 * ((double)s - c.m) + 1.0;
            for (int ax = 0; ax < 3; ++ax) v[ax] = tr.a[ax][1] + tr.a[ax][2] * dphi2;
            const double sp = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
            sum += sp;
            if (s == 0 || sp > vmax) vmax = sp;
            if (s == 0 || sp < vmin) vmin = sp;
            if (s == 0)
                for (int ax = 0; ax < 3; ++ax) vf[ax] = v[ax];
            if (s + 2 == c.len)
                for (int ax = 0; ax < 3; ++ax) vl[ax] = v[ax];
        }
        tr.mean_speed = sum / (double)(c.len - 1);
        tr.speed_range = vmax - vmin;
        const double nf = sqrt(vf[0] * vf[0] + vf[1] * vf[1] + vf[2] * vf[2]);
        const double nl = sqrt(vl[0] * vl[0] + vl[1] * vl[1] + vl[2] * vl[2]);
        const double dot = vf[0] * vl[0] + vf[1] * vl[1] + vf[2] * vl[2];
        tr.cos_turn = (nf > 0.0 && nl > 0.0) ? dot / (nf * nl) : -2.0;
        tr.accepted = (tr.mean_speed > 0.0 && tr.cos_turn >= c.cos_max_turn &&
                       tr.speed_range <= c.max_speed_change * tr.mean_speed) ? 1 : 0;
        rec[i] = tr;
    }
}

// Exclusive scan of flag[0 .. n) into pos (one CTA: each thread sums a
// contiguous chunk, a block scan places the chunks); pos[n] = total.
__global__ void __launch_bounds__(1024) k_track_scan(const int* __restrict__ n3d, int cap3d,
                                                     const int* __restrict__ flag, int* __restrict__ pos,
                                                     int* __restrict__ n_tracks, int cap_tracks,
                                                     unsigned* __restrict__ status)
{
    __shared__ int part[1024];
    const int n = min(max(*n3d, 0), cap3d);
    const int per = (n + blockDim.x - 1) / blockDim.x;
    const int a = min(n, (int)threadIdx.x * per), b = min(n, a + per);
    int s = 0;
    for (int i = a; i < b; ++i) s += flag[i];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int o = 1; o < (int)blockDim.x; o <<= 1) {
        const int v = threadIdx.x >= (unsigned)o ? part[threadIdx.x - o] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    int run = part[threadIdx.x] - s;
    for (int i = a; i < b; ++i) {
        pos[i] = run;
        run += flag[i];
    }
    if (threadIdx.x == blockDim.x - 1) {
        pos[n] = part[threadIdx.x];
        *n_tracks = part[threadIdx.x];
        if (part[threadIdx.x] > cap_tracks) atomicOr(status, ST_CAPACITY);
    }
}

__global__ void k_track_write(const int* __restrict__ n3d, int cap3d, const int* __restrict__ flag,
                              const int* __restrict__ pos, const ulm_track_rec* __restrict__ rec,
                              ulm_track_rec* __restrict__ out, int cap_tracks)
{
    const int n = min(max(*n3d, 0), cap3d);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        if (flag[i] && pos[i] < cap_tracks) out[pos[i]] = rec[i];
}

// one thread per (track, sample): the smoothed position at tau = s / substeps
// adds one count to the voxel that holds it
__global__ void k_track_accumulate(TrackConst c, const ulm_track_rec* __restrict__ tr, const int* __restrict__ n_tracks,
                                   int cap_tracks, unsigned* __restrict__ grid)
{
    const int nt = min(*n_tracks, cap_tracks);
    const int ns = (c.len - 1) * c.substeps + 1;
    const long long total = (long long)nt * ns;
    for (long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x; w < total;
         w += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(w / ns), s = (int)(w - (long long)k * ns);
        if (!tr[k].accepted) continue;
        const double tau = (double)s / (double)c.substeps;
        const double f1 = tau - c.m, f2 = f1 * f1 - c.q;
        int iv[3];
        bool inside = true;
        for (int ax = 0; ax < 3; ++ax) {
            const double p = tr[k].a[ax][0] + tr[k].a[ax][1] * f1 + tr[k].a[ax][2] * f2;
            const double cv = floor((p - c.lo[ax]) / c.voxel);
            inside = inside && cv >= 0.0 && cv < (double)c.dims[ax];
            iv[ax] = inside ? (int)cv : 0;
        }
        if (inside) atomicAdd(grid + ((size_t)iv[2] * c.dims[1] + iv[1]) * c.dims[0] + iv[0], 1u);
    }
}

// Velocity at every accumulation sample of an accepted track: the derivative
// of the smoothed quadratic, v = a1 + 2 a2 phi1(tau) per axis (metres per frame
// interval); the voxel of the sample (as for the density) adds |v| and v_z,
// each rounded to a whole nanometre, to 64-bit integer sums, so the result is
// exact whatever the order of the atomic additions.
__global__ void k_track_velocity(TrackConst c, const ulm_track_rec* __restrict__ tr, const int* __restrict__ n_tracks,
                                 int cap_tracks, unsigned long long* __restrict__ speed,
                                 unsigned long long* __restrict__ vz)
{
    const int nt = min(*n_tracks, cap_tracks);
    const int ns = (c.len - 1) * c.substeps + 1;
    const long long total = (long long)nt * ns;
    for (long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x; w < total;
         w += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(w / ns), s = (int)(w - (long long)k * ns);
        if (!tr[k].accepted) continue;
        const double tau = (double)s / (double)c.substeps;
        const double f1 = tau - c.m, f2 = f1 * f1 - c.q;
        int iv[3];
        double v[3];
        bool inside = true;
        for (int ax = 0; ax < 3; ++ax) {
            const double p = tr[k].a[ax][0] + tr[k].a[ax][1] * f1 + tr[k].a[ax][2] * f2;
            const double cv = floor((p - c.lo[ax]) / c.voxel);
            inside = inside && cv >= 0.0 && cv < (double)c.dims[ax];
            iv[ax] = inside ? (int)cv : 0;
            v[ax] = tr[k].a[ax][1] + 2.0 * tr[k].a[ax][2] * f1;
        }
        if (inside) {
            const size_t at = ((size_t)iv[2] * c.dims[1] + iv[1]) * c.dims[0] + iv[0];
            const double sp = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
            atomicAdd(speed + at, (unsigned long long)llrint(sp * 1e9));
            atomicAdd(vz + at, (unsigned long long)llrint(v[2] * 1e9));
        }
    }
}

}  // namespace

void density_shape(const GeomDev& g, double voxel, int dims[3])
{
    dims[0] = (int)std::ceil((double)g.N * g.pitch / voxel);
    dims[1] = dims[0];
    dims[2] = (int)std::ceil((double)g.nz * g.dz / voxel);
}

static TrackConst track_const(const GeomDev& g, const ulm_track_params* prm)
{
    TrackConst c;
    c.half_span = 0.5 * (double)(g.N - 1);
    c.pitch = g.pitch;
    c.dz = g.dz;
    c.z0 = g.z0;
    c.r2 = prm->max_step_m * prm->max_step_m;
    c.len = prm->len;
    c.substeps = prm->substeps;
    c.m = 0.5 * (double)(c.len - 1);
    c.q = ((double)c.len * (double)c.len - 1.0) / 12.0;
    c.n1 = 0.0;
    c.n2 = 0.0;
    for (int tt = 0; tt < c.len; ++tt) {
        const double f1 = (double)tt - c.m, f2 = f1 * f1 - c.q;
        c.n1 += f1 * f1;
        c.n2 += f2 * f2;
    }
    c.lo[0] = -0.5 * (double)g.N * g.pitch;
    c.lo[1] = c.lo[0];
    c.lo[2] = g.z0 - 0.5 * g.dz;
    c.voxel = prm->voxel_m;
    c.cos_max_turn = prm->cos_max_turn;
    c.max_speed_change = prm->max_speed_change;
    density_shape(g, prm->voxel_m, c.dims);
    return c;
}

rca_status launch_track_velocity(rca_handle* h, const rca_tables* t, const ulm_track_rec* tracks,
                                 const int* n_tracks, int cap_tracks, const ulm_track_params* prm, int64_t* speed,
                                 int64_t* vz)
{
    const TrackConst c = track_const(t->gd, prm);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t samples = (size_t)std::max(cap_tracks, 1) * ((size_t)(c.len - 1) * c.substeps + 1);
    const int grid_a = (int)std::min<size_t>((samples + TR_THREADS - 1) / TR_THREADS, (size_t)sms * 16);
    k_track_velocity<<<grid_a, TR_THREADS, 0, h->stream>>>(c, tracks, n_tracks, cap_tracks,
                                                           reinterpret_cast<unsigned long long*>(speed),
                                                           reinterpret_cast<unsigned long long*>(vz));
    return cuda_check(h, cudaGetLastError(), "velocity kernel");
}

rca_status launch_track(rca_handle* h, const rca_tables* t, const ulm_loc3d* L, const int* n3d, int cap3d, int F,
                        const ulm_track_params* prm, ulm_track_rec* out, int cap_tracks, int* n_tracks, unsigned* density)
{
    const TrackConst c = track_const(t->gd, prm);
    rca_status st = RCA_OK;
    const size_t nmax = (size_t)std::max(cap3d, 1);
    // workspace: offsets [F + 2], nxt, prv, flag [n], pos [n + 1], records [n]
    const size_t ints = (size_t)(F + 2) + 4 * nmax + 1;
    const size_t bytes = ((ints * sizeof(int) + 15) / 16) * 16 + nmax * sizeof(ulm_track_rec);
    char* ws = (char*)ws_get(h, WS_TRACK, bytes, &st);
    if (!ws) return st;
    int* offs = reinterpret_cast<int*>(ws);
    int* nxt = offs + (F + 2);
    int* prv = nxt + nmax;
    int* flag = prv + nmax;
    int* pos = flag + nmax;
    ulm_track_rec* rec = reinterpret_cast<ulm_track_rec*>(ws + ((ints * sizeof(int) + 15) / 16) * 16);

    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid_n = (int)std::min<size_t>((nmax + TR_THREADS - 1) / TR_THREADS, (size_t)sms * 8);
    k_track_offsets<<<(F + 2 + TR_THREADS - 1) / TR_THREADS, TR_THREADS, 0, h->stream>>>(L, n3d, cap3d, F, offs);
    k_track_link<<<grid_n, TR_THREADS, 0, h->stream>>>(c, L, n3d, cap3d, F, offs, nxt, prv);
    k_track_build<<<grid_n, TR_THREADS, 0, h->stream>>>(c, L, n3d, cap3d, nxt, prv, rec, flag);
    k_track_scan<<<1, 1024, 0, h->stream>>>(n3d, cap3d, flag, pos, n_tracks, cap_tracks, h->d_status);
    k_track_write<<<grid_n, TR_THREADS, 0, h->stream>>>(n3d, cap3d, flag, pos, rec, out, cap_tracks);
    if (density) {
        const size_t samples = (size_t)std::max(cap_tracks, 1) * ((size_t)(c.len - 1) * c.substeps + 1);
        const int grid_a = (int)std::min<size_t>((samples + TR_THREADS - 1) / TR_THREADS, (size_t)sms * 16);
        k_track_accumulate<<<grid_a, TR_THREADS, 0, h->stream>>>(c, out, n_tracks, cap_tracks, density);
    }
    return cuda_check(h, cudaGetLastError(), "tracking kernels");
}
