// localize.cu -- XDoppler enhancement, separable NCC, sub-pixel peaks and
// XZ / YZ pairing (Sec. II-A4, Fig. 1e, Fig. 1g).
#include <algorithm>
#include <cmath>

#include "rca_internal.cuh"

namespace {

__device__ __forceinline__ float block_max_256(float v, float* red)
{
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) red[warp] = v;
    __syncthreads();
    float m = 0.f;
    if (threadIdx.x < 32) {
        m = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    }
    __syncthreads();
    return m;  // valid in thread 0
}

// ---------------------------------------------------------------------------
// XDoppler: each thread owns one pixel (axis, slab, row, lateral) and walks
// the frames with a sliding 3-frame window, so every plane is read once:
//   Q_t = P_RC,t conj(P_CR,t),  A_t = sqrt(|Q_{t-1} + Q_t + Q_{t+1}|).
// M_t = max A_t through a block max and one atomicMax per block and frame
// (non-negative floats order like their bit patterns).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_enhance(const void* __restrict__ planes, int pt, int F, int S,
                                                 size_t plane_sz, int enh, float* __restrict__ A,
                                                 unsigned* __restrict__ M)
{
    __shared__ float red[8];
    const size_t per_axis = (size_t)S * plane_sz;
    const size_t npx = 2 * per_axis;
    const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool act = p < npx;
    const size_t axis = act ? p / per_axis : 0, rest = act ? p % per_axis : 0;
    auto at = [&](int t, int fam) { return (((size_t)t * 2 + axis) * 2 + fam) * per_axis + rest; };
    auto q_of = [&](int t) {
        float2 a = load_c(planes, at(t, 0), pt), b = load_c(planes, at(t, 1), pt);
        return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);  // a * conj(b)
    };
    float2 qm = make_float2(0.f, 0.f), q0 = act ? q_of(0) : make_float2(0.f, 0.f);
    for (int t = 0; t < F; ++t) {
        float a = 0.f;
        if (act) {
            if (enh == ULM_ENH_XDOPPLER) {
                float2 qp = (t + 1 < F) ? q_of(t + 1) : make_float2(0.f, 0.f);
                float re = qm.x + q0.x + qp.x, im = qm.y + q0.y + qp.y;
                a = sqrtf(sqrtf(re * re + im * im));
                qm = q0;
                q0 = qp;
            } else {
                float2 x = load_c(planes, at(t, 0), pt), y = load_c(planes, at(t, 1), pt);
                float re = x.x + y.x, im = x.y + y.y;
                a = sqrtf(re * re + im * im);
            }
            A[(size_t)t * npx + p] = a;
        }
        float m = block_max_256(a, red);
        if (threadIdx.x == 0) atomicMax(M + t, __float_as_uint(m));
    }
}

// ---------------------------------------------------------------------------
// NCC + regional peaks.  CTA = (row strip of DET_RS rows, plane).  NCC via
// separable 1D correlations (Fig. 1g):
//   s1 = box(A), s2 = box(A^2), sg = (g_z x g_l) * A,
//   NCC = (sg - mu_G s1) / sqrt((s2 - s1^2 / d^2) * ss_G),
// computed on the strip plus one row above and below for the 3x3 test.
// Candidates are compacted in raster order into a fixed-capacity slot of
// the strip; the true count is kept.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_detect(const float* __restrict__ A, const float* __restrict__ Mf, int S,
                                                int nz, int N, NccConst nc, ulm_loc2d* __restrict__ cand,
                                                int* __restrict__ cnt, float* __restrict__ ncc_out,
                                                unsigned* __restrict__ status)
{
    extern __shared__ float sm[];
    const int h = nc.h, d = nc.d;
    const int strip = blockIdx.x, plane = blockIdx.y;
    const int nstrip = gridDim.x;
    const int t = plane / (2 * S), axis = (plane / S) % 2, b = plane % S;
    const int i0 = strip * DET_RS;
    const int rin = DET_RS + 2 + 2 * h, rn = DET_RS + 2;
    float* sA = sm;
    float* H1 = sA + rin * N;
    float* H2 = H1 + rin * N;
    float* HG = H2 + rin * N;
    float* sN = HG + rin * N;
    __shared__ int wsum[8];
    __shared__ int base_count;
    const float* Ap = A + (size_t)plane * nz * N;
    const float Mt = Mf[t];
    for (int idx = threadIdx.x; idx < rin * N; idx += blockDim.x) {
        int rr = idx / N, l = idx - rr * N;
        int row = i0 - 1 - h + rr;
        sA[idx] = (row >= 0 && row < nz) ? Ap[(size_t)row * N + l] : 0.f;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < rin * N; idx += blockDim.x) {
        int rr = idx / N, l = idx - rr * N;
        float s1 = 0.f, s2 = 0.f, sg = 0.f;
        if (l >= h && l < N - h) {
            const float* x = sA + rr * N + l - h;
            for (int q = 0; q < d; ++q) {
                float v = x[q];
                s1 += v;
                s2 = fmaf(v, v, s2);
                sg = fmaf(nc.gl[q], v, sg);
            }
        }
        H1[idx] = s1;
        H2[idx] = s2;
        HG[idx] = sg;
    }
    __syncthreads();
    const float flat = nc.flat_coef * Mt * Mt;
    const float inv_d2 = 1.0f / (float)(d * d);
    for (int idx = threadIdx.x; idx < rn * N; idx += blockDim.x) {
        int ro = idx / N, l = idx - ro * N;
        int i = i0 - 1 + ro;
        float v = 0.f;
        if (i >= h && i < nz - h && l >= h && l < N - h && Mt > 0.f) {
            float s1 = 0.f, s2 = 0.f, sg = 0.f;
            for (int a = 0; a <= 2 * h; ++a) {
                int o = (ro + a) * N + l;
                s1 += H1[o];
                s2 += H2[o];
                sg = fmaf(nc.gz[a], HG[o], sg);
            }
            float ssA = s2 - s1 * s1 * inv_d2;
            if (ssA > flat) v = (sg - nc.muG * s1) * nc.inv_ssG_sqrt * rsqrtf(ssA);
        }
        sN[idx] = v;
        if (ncc_out && ro >= 1 && ro <= DET_RS && i < nz) ncc_out[((size_t)plane * nz + i) * N + l] = v;
    }
    if (threadIdx.x == 0) base_count = 0;
    __syncthreads();
    const float athr = nc.alpha * Mt;
    ulm_loc2d* slot = cand + ((size_t)plane * nstrip + strip) * CAND_CAP;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int base = 0; base < DET_RS * N; base += blockDim.x) {
        const int p = base + threadIdx.x;
        const int ro = 1 + p / N, l = p % N;
        const int i = i0 - 1 + ro;
        bool pk = false;
        float c = 0.f;
        if (p < DET_RS * N && i >= 1 && i < nz - 1 && l >= 1 && l < N - 1) {
            c = sN[ro * N + l];
            float amp = sA[(ro + h) * N + l];
            if (c >= nc.ncc_min && amp >= athr) {
                pk = true;
                for (int a = -1; a <= 1; ++a)
                    for (int bb = -1; bb <= 1; ++bb) {
                        if (a == 0 && bb == 0) continue;
                        float q = sN[(ro + a) * N + l + bb];
                        bool earlier = (a < 0) || (a == 0 && bb < 0);
                        if (earlier ? !(c > q) : !(c >= q)) pk = false;
                    }
            }
        }
        unsigned bal = __ballot_sync(0xffffffffu, pk);
        if (lane == 0) wsum[warp] = __popc(bal);
        __syncthreads();
        int before = base_count;
        for (int w = 0; w < warp; ++w) before += wsum[w];
        before += __popc(bal & ((1u << lane) - 1u));
        if (pk && before < CAND_CAP) {
            auto para = [](float fm, float f0, float fp) {
                float den = fm - 2.f * f0 + fp;
                if (den >= 0.f) return 0.f;
                float dl = (fm - fp) / (2.f * den);
                return fminf(0.5f, fmaxf(-0.5f, dl));
            };
            ulm_loc2d e;
            e.frame = t;
            e.axis = axis;
            e.slab = b;
            e.iz = i;
            e.ilat = l;
            e.z = (float)i + para(sN[(ro - 1) * N + l], c, sN[(ro + 1) * N + l]);
            e.lat = (float)l + para(sN[ro * N + l - 1], c, sN[ro * N + l + 1]);
            e.ncc = c;
            e.amp = sA[(ro + h) * N + l];
            e.reserved = 0;
            slot[before] = e;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int tot = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += wsum[w];
            base_count += tot;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        cnt[(size_t)plane * nstrip + strip] = base_count;
        if (base_count > CAND_CAP) atomicOr(status, ST_CAPACITY);
    }
}

// Single-CTA exclusive scan of min(cnt[i], cap_each) (cap_each <= 0: no cap).
// off[n] = total kept; *total_true = sum of cnt (may exceed the kept total).
__global__ void __launch_bounds__(1024) k_scan(const int* __restrict__ cnt, int n, int cap_each,
                                               int* __restrict__ off, int* __restrict__ total_true,
                                               const int* __restrict__ n_dev)
{
    __shared__ int part[1024];
    __shared__ long long tpart[1024];
    if (n_dev) n = min(n, *n_dev);
    const int T = blockDim.x;
    const int per = (n + T - 1) / T;
    const int lo = threadIdx.x * per, hi = min(n, lo + per);
    int s = 0;
    long long st = 0;
    for (int i = lo; i < hi; ++i) {
        int c = cnt[i];
        st += c;
        s += (cap_each > 0) ? min(c, cap_each) : c;
    }
    part[threadIdx.x] = s;
    tpart[threadIdx.x] = st;
    __syncthreads();
    for (int o = 1; o < T; o <<= 1) {
        int v = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
        long long tv = threadIdx.x >= o ? tpart[threadIdx.x - o] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        tpart[threadIdx.x] += tv;
        __syncthreads();
    }
    int run = threadIdx.x ? part[threadIdx.x - 1] : 0;
    for (int i = lo; i < hi; ++i) {
        off[i] = run;
        int c = cnt[i];
        run += (cap_each > 0) ? min(c, cap_each) : c;
    }
    if (threadIdx.x == T - 1) {
        off[n] = part[T - 1];
        if (total_true) *total_true = (int)(tpart[T - 1] < 0x7fffffffLL ? tpart[T - 1] : 0x7fffffffLL);
    }
}

// Copy each strip's kept candidates to their place in the output list.
__global__ void k_gather(const ulm_loc2d* __restrict__ cand, const int* __restrict__ cnt, const int* __restrict__ off,
                         int nslots, ulm_loc2d* __restrict__ out, int cap, unsigned* __restrict__ status)
{
    const int s = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (s >= nslots) return;
    const int lane = threadIdx.x & 31;
    const int c = min(cnt[s], CAND_CAP);
    for (int r = lane; r < c; r += 32) {
        int dst = off[s] + r;
        if (dst < cap) out[dst] = cand[(size_t)s * CAND_CAP + r];
        else atomicOr(status, ST_CAPACITY);
    }
}

// plane offsets of the (frame, axis, slab)-sorted list: first entry of each plane
__global__ void k_strip_to_plane(const int* __restrict__ off, int nstrip, int nplanes, int* __restrict__ poff)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p <= nplanes) poff[p] = off[(size_t)p * nstrip];
}

// ---------------------------------------------------------------------------
// pairing
// ---------------------------------------------------------------------------
__device__ __forceinline__ int plane_key(const ulm_loc2d& e, int S) { return (e.frame * 2 + e.axis) * S + e.slab; }

__global__ void k_list_plane_offsets(const ulm_loc2d* __restrict__ L, const int* __restrict__ n2d, int cap2d, int S,
                                     int nplanes, int* __restrict__ poff)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p > nplanes) return;
    int n = min(*n2d, cap2d);
    int lo = 0, hi = n;  // first index with key >= p
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (plane_key(L[mid], S) < p) lo = mid + 1;
        else hi = mid;
    }
    poff[p] = lo;
}

// XZ / YZ eligibility and cost in double precision: same frame and
// sub-block, |dz| <= 1 pixel, ratio I_xz / I_yz in [0.9, 1.11];
// cost max(I) / min(I) (orders pairs like |ln ratio|).
__device__ __forceinline__ bool pair_ok(const ulm_loc2d& x, const ulm_loc2d& y, int P, double* cost)
{
    if (x.frame != y.frame) return false;
    if (x.ilat / P != y.slab || y.ilat / P != x.slab) return false;
    if (fabs((double)x.z - (double)y.z) > 1.0) return false;
    double ax = x.amp, ay = y.amp;
    double r = ax / ay;
    if (!(r >= 0.9 && r <= 1.11)) return false;
    *cost = ax > ay ? ax / ay : ay / ax;
    return true;
}

__global__ void k_pair_match(const ulm_loc2d* __restrict__ L, const int* __restrict__ n2d, int cap2d, int S, int P,
                             const int* __restrict__ poff, int* __restrict__ match)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = min(*n2d, cap2d);
    if (a >= n) return;
    const ulm_loc2d x = L[a];
    int m = -1;
    if (x.axis == 0) {
        const int py = (x.frame * 2 + 1) * S + x.ilat / P;
        int best = -1;
        double bc = 0.0;
        for (int q = poff[py]; q < min(poff[py + 1], n); ++q) {
            double c;
            if (pair_ok(x, L[q], P, &c) && (best < 0 || c < bc)) {
                best = q;
                bc = c;
            }
        }
        if (best >= 0) {
            const ulm_loc2d y = L[best];
            const int px = (y.frame * 2 + 0) * S + y.ilat / P;
            int back = -1;
            double bc2 = 0.0;
            for (int q = poff[px]; q < min(poff[px + 1], n); ++q) {
                double c;
                if (pair_ok(L[q], y, P, &c) && (back < 0 || c < bc2)) {
                    back = q;
                    bc2 = c;
                }
            }
            if (back == a) m = best;
        }
    }
    match[a] = m;
}

__global__ void k_match_flags(const int* __restrict__ match, const int* __restrict__ n2d, int cap2d,
                              int* __restrict__ flags)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= cap2d) return;
    const int n = min(*n2d, cap2d);
    flags[a] = (a < n && match[a] >= 0) ? 1 : 0;
}

__global__ void k_pair_write(const ulm_loc2d* __restrict__ L, const int* __restrict__ n2d, int cap2d,
                             const int* __restrict__ match, const int* __restrict__ off, ulm_loc3d* __restrict__ out,
                             int cap3d, unsigned* __restrict__ status)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = min(*n2d, cap2d);
    if (a >= n || match[a] < 0) return;
    const int dst = off[a];
    if (dst >= cap3d) {
        atomicOr(status, ST_CAPACITY);
        return;
    }
    const ulm_loc2d x = L[a], y = L[match[a]];
    ulm_loc3d o;
    o.frame = x.frame;
    o.i_xz = a;
    o.i_yz = match[a];
    o.reserved = 0;
    o.x = x.lat;
    o.y = y.lat;
    o.z = 0.5f * (x.z + y.z);
    o.amp_xz = x.amp;
    o.amp_yz = y.amp;
    o.reserved2 = 0.f;
    out[dst] = o;
}

}  // namespace

rca_status launch_enhance(rca_handle* h, const rca_tables* t, const void* planes, rca_dtype pt, int F, int enh,
                          float* A, float* M)
{
    const GeomDev& g = t->gd;
    if (enh != ULM_ENH_XDOPPLER && enh != ULM_ENH_COHERENT) return set_error(h, RCA_ERR_INVALID_ARG, "bad enhancement mode");
    const size_t plane_sz = (size_t)g.nz * g.N;
    const size_t npx = 2 * (size_t)g.S * plane_sz;
    cudaMemsetAsync(M, 0, sizeof(float) * F, h->stream);
    k_enhance<<<(unsigned)((npx + 255) / 256), 256, 0, h->stream>>>(planes, (int)pt, F, g.S, plane_sz, enh, A,
                                                                   reinterpret_cast<unsigned*>(M));
    return cuda_check(h, cudaGetLastError(), "enhance kernel");
}

rca_status launch_detect2d(rca_handle* h, const rca_tables* t, const float* A, const float* M, int F,
                           const ulm_params* prm, ulm_loc2d* out, int cap, int* n2d, float* ncc_out, int* plane_off)
{
    const GeomDev& g = t->gd;
    const int d = prm->d, hh = (d - 1) / 2;
    NccConst nc;
    nc.d = d;
    nc.h = hh;
    double G[RCA_MAX_NCC_D * RCA_MAX_NCC_D];
    double muG = 0.0;
    for (int a = -hh; a <= hh; ++a) {
        nc.gz[a + hh] = (float)std::exp(-(double)(a * a) / (2.0 * (double)prm->sig_z * prm->sig_z));
        nc.gl[a + hh] = (float)std::exp(-(double)(a * a) / (2.0 * (double)prm->sig_lat * prm->sig_lat));
    }
    for (int a = 0; a < d; ++a)
        for (int b = 0; b < d; ++b) {
            G[a * d + b] = (double)nc.gz[a] * (double)nc.gl[b];
            muG += G[a * d + b];
        }
    muG /= (double)(d * d);
    double ssG = 0.0;
    for (int q = 0; q < d * d; ++q) ssG += (G[q] - muG) * (G[q] - muG);
    nc.muG = (float)muG;
    nc.inv_ssG_sqrt = (float)(1.0 / std::sqrt(ssG));
    nc.flat_coef = (float)(1e-5 * d * d);
    nc.alpha = prm->alpha;
    nc.ncc_min = prm->ncc_min;

    const int nstrip = (g.nz + DET_RS - 1) / DET_RS;
    const int nplanes = F * 2 * g.S;
    const int nslots = nplanes * nstrip;
    rca_status st = RCA_OK;
    ulm_loc2d* cand = (ulm_loc2d*)ws_get(h, WS_CAND, (size_t)nslots * CAND_CAP * sizeof(ulm_loc2d), &st);
    if (!cand) return st;
    int* cnt = (int*)ws_get(h, WS_CANDCNT, (size_t)nslots * sizeof(int), &st);
    if (!cnt) return st;
    int* off = (int*)ws_get(h, WS_SCAN, (size_t)(nslots + 1) * sizeof(int), &st);
    if (!off) return st;
    const int rin = DET_RS + 2 + 2 * hh;
    size_t smem = ((size_t)4 * rin * g.N + (size_t)(DET_RS + 2) * g.N) * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(k_detect, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_check(h, e, "detect smem attribute");
    dim3 grid(nstrip, nplanes);
    k_detect<<<grid, 256, smem, h->stream>>>(A, M, g.S, g.nz, g.N, nc, cand, cnt, ncc_out, h->d_status);
    k_scan<<<1, 1024, 0, h->stream>>>(cnt, nslots, CAND_CAP, off, n2d, nullptr);
    k_gather<<<(nslots + 7) / 8, 256, 0, h->stream>>>(cand, cnt, off, nslots, out, cap, h->d_status);
    if (plane_off) k_strip_to_plane<<<(nplanes + 1 + 255) / 256, 256, 0, h->stream>>>(off, nstrip, nplanes, plane_off);
    return cuda_check(h, cudaGetLastError(), "detect kernels");
}

rca_status launch_pair3d(rca_handle* h, const rca_tables* t, const ulm_loc2d* L, const int* n2d, int cap2d, int F,
                         ulm_loc3d* out, int cap3d, int* n3d)
{
    const GeomDev& g = t->gd;
    const int nplanes = F * 2 * g.S;
    rca_status st = RCA_OK;
    int* poff = (int*)ws_get(h, WS_PLANEOFF, (size_t)(nplanes + 1) * sizeof(int), &st);
    if (!poff) return st;
    const int nn = std::max(cap2d, 1);
    int* match = (int*)ws_get(h, WS_FLAGS, (size_t)nn * 2 * sizeof(int), &st);
    if (!match) return st;
    int* flags = match + nn;
    int* off = (int*)ws_get(h, WS_MISC, (size_t)(nn + 1) * sizeof(int), &st);
    if (!off) return st;
    k_list_plane_offsets<<<(nplanes + 1 + 255) / 256, 256, 0, h->stream>>>(L, n2d, cap2d, g.S, nplanes, poff);
    k_pair_match<<<(nn + 255) / 256, 256, 0, h->stream>>>(L, n2d, cap2d, g.S, g.P, poff, match);
    k_match_flags<<<(nn + 255) / 256, 256, 0, h->stream>>>(match, n2d, cap2d, flags);
    k_scan<<<1, 1024, 0, h->stream>>>(flags, nn, 0, off, n3d, n2d);
    k_pair_write<<<(nn + 255) / 256, 256, 0, h->stream>>>(L, n2d, cap2d, match, off, out, cap3d, h->d_status);
    return cuda_check(h, cudaGetLastError(), "pair kernels");
}
