// Create-time work of fmmbem_create, all on the device:
//   panel geometry and K-point Gauss points (Sec. 2.3, eqs. gauss:1st-kind/2nd-kind),
//   Morton keys and a radix sort of panels by centroid,
//   a top-down octree whose leaves hold at most ncrit Gauss points (Sec. 2.5),
//   a dual-tree traversal with the acceptance criterion (R_a + R_b) < theta |c_a - c_b|
//   producing M2L and P2P lists (Sec. 2.5),
//   the near-singular search (|c_i - c_j| < f sqrt(2 S_j)) and the FP64 correction
//   table: 20-point rule minus K-point rule for near panels, the semi-analytic
//   integral for the self panel (Sec. 2.3, Hess-Smith decomposition).
#include <algorithm>
#include <cstring>
#include <vector>
#include "handle.cuh"
#include "harmonics.cuh"

namespace fmmbem {

namespace {

template <typename P>
int dalloc(P** p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    FMM_CU(fmm_malloc((void**)p, count * sizeof(P)));
    return 0;
}

// ---------------------------------------------------------------- quadrature
// Far rules from their published definitions (area-normalised weights):
// K=1 centroid; K=3 Strang-Fix (2/3,1/6,1/6); K=4 Strang-Fix degree 3 (centroid
// -27/48, (3/5,1/5,1/5) 25/48); K=7 Radon degree 5.
int far_rule_host(int K, double* q /* K x 4: l1,l2,l3,w */) {
    if (K == 1) {
        q[0] = q[1] = q[2] = 1.0 / 3.0; q[3] = 1.0;
        return 0;
    }
    if (K == 3) {
        const double a = 2.0 / 3.0, b = 1.0 / 6.0;
        double pts[3][3] = {{a, b, b}, {b, a, b}, {b, b, a}};
        for (int k = 0; k < 3; ++k) { for (int d = 0; d < 3; ++d) q[4 * k + d] = pts[k][d]; q[4 * k + 3] = 1.0 / 3.0; }
        return 0;
    }
    if (K == 4) {
        double pts[4][3] = {{1.0 / 3, 1.0 / 3, 1.0 / 3}, {0.6, 0.2, 0.2}, {0.2, 0.6, 0.2}, {0.2, 0.2, 0.6}};
        double w[4] = {-27.0 / 48.0, 25.0 / 48.0, 25.0 / 48.0, 25.0 / 48.0};
        for (int k = 0; k < 4; ++k) { for (int d = 0; d < 3; ++d) q[4 * k + d] = pts[k][d]; q[4 * k + 3] = w[k]; }
        return 0;
    }
    if (K == 7) {
        const double s15 = sqrt(15.0);
        const double a[2] = {(6.0 - s15) / 21.0, (6.0 + s15) / 21.0};
        const double w[2] = {(155.0 - s15) / 1200.0, (155.0 + s15) / 1200.0};
        q[0] = q[1] = q[2] = 1.0 / 3.0; q[3] = 9.0 / 40.0;
        int k = 1;
        for (int g = 0; g < 2; ++g) {
            const double b = 1.0 - 2.0 * a[g];
            double pts[3][3] = {{b, a[g], a[g]}, {a[g], b, a[g]}, {a[g], a[g], b}};
            for (int r = 0; r < 3; ++r, ++k) { for (int d = 0; d < 3; ++d) q[4 * k + d] = pts[r][d]; q[4 * k + 3] = w[g]; }
        }
        return 0;
    }
    return FMMBEM_EINVAL;
}

// Near-singular rule: collapsed coordinates l1 = 1-u, l2 = u(1-v), l3 = uv with
// nu Gauss-Legendre nodes in u (weight multiplied by the Jacobian u) and nv = nu - 1 in v
// (5 x 4 = 20 points by default, the K ~ 20 of Sec. 2.3), scaled so the weights sum to
// one; exact to total degree 2 nv - 1. Legendre roots by Newton's method on P_n.
__device__ void legendre_rule01(int n, double* x, double* w) {
    for (int i = 0; i < n; ++i) {
        double t = cos(3.14159265358979323846 * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = t;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2 * k - 1) * t * p1 - (k - 1) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            double pn = (n == 1) ? t : p1, pnm1 = (n == 1) ? 1.0 : p0;
            dp = n * (t * pn - pnm1) / (t * t - 1.0);
            double dt = pn / dp;
            t -= dt;
            if (fabs(dt) < 1e-16) break;
        }
        x[i] = 0.5 * (1.0 - t);
        w[i] = 1.0 / ((1.0 - t * t) * dp * dp);  // = 0.5 * 2/((1-t^2) P_n'(t)^2)
    }
}

__global__ void k_near_rule(int nu, int nv, double* q /* nu nv x 4 */) {
    double xu[8], wu[8], xv[8], wv[8];
    legendre_rule01(nu, xu, wu);
    legendre_rule01(nv, xv, wv);
    for (int i = 0; i < nu; ++i)
        for (int j = 0; j < nv; ++j) {
            double* o = q + 4 * (nv * i + j);
            o[0] = 1.0 - xu[i];
            o[1] = xu[i] * (1.0 - xv[j]);
            o[2] = xu[i] * xv[j];
            o[3] = 2.0 * wu[i] * wv[j] * xu[i];
        }
}

// ---------------------------------------------------------------- geometry
__device__ __forceinline__ unsigned long long dbits(double x) { return (unsigned long long)__double_as_longlong(x); }

__global__ void k_bbox(const double* v, int64_t nv, double* out /* lo[3], hi[3] */) {
    __shared__ double slo[3][256], shi[3][256];
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int64_t i = threadIdx.x; i < nv; i += blockDim.x)
        for (int d = 0; d < 3; ++d) {
            double x = v[3 * i + d];
            lo[d] = fmin(lo[d], x);
            hi[d] = fmax(hi[d], x);
        }
    for (int d = 0; d < 3; ++d) { slo[d][threadIdx.x] = lo[d]; shi[d][threadIdx.x] = hi[d]; }
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int d = 0; d < 3; ++d) {
                slo[d][threadIdx.x] = fmin(slo[d][threadIdx.x], slo[d][threadIdx.x + s]);
                shi[d][threadIdx.x] = fmax(shi[d][threadIdx.x], shi[d][threadIdx.x + s]);
            }
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int d = 0; d < 3; ++d) { out[d] = slo[d][0]; out[3 + d] = shi[d][0]; }
}

// Per panel in the caller's order: centroid, unit normal, area; the largest
// centroid-to-vertex distance and the largest area (as ordered bit patterns of
// non-negative doubles); a flag for degenerate panels or bad indices.
__global__ void k_panel_geom(const double* v, int64_t nv, const int* tri, int64_t n, double4* cen, double4* nrm,
                             unsigned long long* spill_bits, unsigned long long* amax_bits, int* bad) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double P[3][3];
    for (int a = 0; a < 3; ++a) {
        int vi = tri[3 * i + a];
        if (vi < 0 || vi >= nv) { atomicExch(bad, 1); return; }
        for (int d = 0; d < 3; ++d) P[a][d] = v[3 * (int64_t)vi + d];
    }
    double c[3], e1[3], e2[3];
    for (int d = 0; d < 3; ++d) {
        c[d] = (P[0][d] + P[1][d] + P[2][d]) / 3.0;
        e1[d] = P[1][d] - P[0][d];
        e2[d] = P[2][d] - P[0][d];
    }
    double cr[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
    double len = sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
    if (!(len > 0.0)) { atomicExch(bad, 2); return; }
    double S = 0.5 * len;
    cen[i] = make_double4(c[0], c[1], c[2], S);
    nrm[i] = make_double4(cr[0] / len, cr[1] / len, cr[2] / len, S);
    double sp = 0.0;
    for (int a = 0; a < 3; ++a) {
        double d2 = 0.0;
        for (int d = 0; d < 3; ++d) d2 += (P[a][d] - c[d]) * (P[a][d] - c[d]);
        sp = fmax(sp, sqrt(d2));
    }
    atomicMax(spill_bits, dbits(sp));
    atomicMax(amax_bits, dbits(S));
}

__device__ __forceinline__ uint64_t spread3(uint64_t x) {
    x &= 0x1fffffULL;
    x = (x | x << 32) & 0x1f00000000ffffULL;
    x = (x | x << 16) & 0x1f0000ff0000ffULL;
    x = (x | x << 8) & 0x100f00f00f00f00fULL;
    x = (x | x << 4) & 0x10c30c30c30c30c3ULL;
    x = (x | x << 2) & 0x1249249249249249ULL;
    return x;
}

// 63-bit Morton key of each centroid in the root cube: bits (3l+2, 3l+1, 3l) = (z, y, x).
__global__ void k_morton(const double4* cen, int64_t n, double lox, double loy, double loz, double side,
                         uint64_t* key, int* idx) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double scale = 2097152.0 / side;  // 2^21
    double4 c = cen[i];
    int64_t q[3] = {(int64_t)floor((c.x - lox) * scale), (int64_t)floor((c.y - loy) * scale),
                    (int64_t)floor((c.z - loz) * scale)};
    for (int d = 0; d < 3; ++d) q[d] = q[d] < 0 ? 0 : (q[d] > 2097151 ? 2097151 : q[d]);
    key[i] = spread3(q[0]) | (spread3(q[1]) << 1) | (spread3(q[2]) << 2);
    idx[i] = (int)i;
}

// Sorted-order copies: centroids, normals, vertices and the K Gauss points of each panel.
__global__ void k_gather_sorted(const int* perm, int64_t n, const double* v, const int* tri, const double4* cen,
                                const double4* nrm, const double* quad, int K, double4* tgt_d, float4* tgt_f,
                                double4* nrm_d, float4* nrm_f, double* verts, double4* src_d, float4* src_f) {
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= n) return;
    int i = perm[s];
    double4 c = cen[i];
    tgt_d[s] = c;
    tgt_f[s] = make_float4((float)c.x, (float)c.y, (float)c.z, (float)c.w);
    const double4 nv = nrm[i];
    nrm_d[s] = nv;
    nrm_f[s] = make_float4((float)nv.x, (float)nv.y, (float)nv.z, (float)nv.w);
    double P[3][3];
    for (int a = 0; a < 3; ++a)
        for (int d = 0; d < 3; ++d) {
            P[a][d] = v[3 * (int64_t)tri[3 * i + a] + d];
            verts[9 * s + 3 * a + d] = P[a][d];
        }
    for (int k = 0; k < K; ++k) {
        const double* q = quad + 4 * k;
        double y[3];
        for (int d = 0; d < 3; ++d) y[d] = q[0] * P[0][d] + q[1] * P[1][d] + q[2] * P[2][d];
        double w = q[3] * c.w;
        src_d[s * K + k] = make_double4(y[0], y[1], y[2], w);
        src_f[s * K + k] = make_float4((float)y[0], (float)y[1], (float)y[2], (float)w);
    }
}

// ---------------------------------------------------------------- octree
__device__ __forceinline__ int lower_bound_key(const uint64_t* key, int lo, int hi, uint64_t prefix, int shift) {
    // first index in [lo, hi) whose key >> shift >= prefix
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if ((key[mid] >> shift) < prefix) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// For each cell of one level: split if it holds more than ncrit Gauss points.
__global__ void k_split_count(int lb, int le, int level, const int2* range, const uint64_t* key, int K, int ncrit,
                              int* nch, int* bounds /* [cells][9] */) {
    int c = lb + blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= le) return;
    int2 r = range[c];
    int cnt = 0;
    int* b = bounds + 9 * (int64_t)(c - lb);
    if ((int64_t)K * (r.y - r.x) > ncrit && level < MAX_LEVELS) {
        const int shift = 3 * (MAX_LEVELS - level - 1);
        const uint64_t base = (key[r.x] >> shift) & ~7ULL;
        b[0] = r.x;
        for (int o = 1; o < 8; ++o) b[o] = lower_bound_key(key, r.x, r.y, base + o, shift);
        b[8] = r.y;
        for (int o = 0; o < 8; ++o) cnt += (b[o + 1] > b[o]);
    }
    nch[c - lb] = cnt;
}

__global__ void k_split_emit(int lb, int le, int next_start, int level, const int* nch, const int* off,
                             const int* bounds, double4* cs, int2* range, int2* child, int* clevel, int* parent) {
    int c = lb + blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= le) return;
    int n = nch[c - lb];
    int first = next_start + off[c - lb];
    child[c] = make_int2(n ? first : -1, n);
    if (!n) return;
    const int* b = bounds + 9 * (int64_t)(c - lb);
    double4 pc = cs[c];
    const double q = 0.25 * pc.w;
    int k = first;
    for (int o = 0; o < 8; ++o) {
        if (b[o + 1] <= b[o]) continue;
        cs[k] = make_double4(pc.x + ((o & 1) ? q : -q), pc.y + ((o & 2) ? q : -q), pc.z + ((o & 4) ? q : -q), 0.5 * pc.w);
        range[k] = make_int2(b[o], b[o + 1]);
        child[k] = make_int2(-1, 0);
        clevel[k] = level + 1;
        parent[k] = c;
        ++k;
    }
}

// Cluster radii of every cell about its box centre: .x = the farthest collocation point
// (targets), .y = the farthest Gauss point (sources). The MAC uses them as the cluster
// sizes, the a of eq. multipole_error.
// Each cell's range is cut into gridDim.y slices; each block reduces the squared distances of
// its slice and raises the cell's maximum with an integer max on the bit patterns (squared
// distances are non-negative, and non-negative doubles order like their bits). rad2 must
// be zero on entry; k_cell_radii_sqrt then takes the square roots.
__global__ void k_cell_radii(int ncells, const double4* cs, const int2* range, const double4* tgt, const double4* src,
                             int K, unsigned long long* rad2) {
    __shared__ double st[128], ss[128];
    const int c = blockIdx.x;
    if (c >= ncells) return;
    const double4 cc = cs[c];
    const int2 r = range[c];
    const int nsl = (int)gridDim.y, sl = (int)blockIdx.y;
    double mt = 0.0, ms = 0.0;
    const int nt = r.y - r.x, t0 = r.x + (int)((long long)nt * sl / nsl), t1 = r.x + (int)((long long)nt * (sl + 1) / nsl);
    for (int i = t0 + threadIdx.x; i < t1; i += blockDim.x) {
        const double4 t = tgt[i];
        mt = fmax(mt, (t.x - cc.x) * (t.x - cc.x) + (t.y - cc.y) * (t.y - cc.y) + (t.z - cc.z) * (t.z - cc.z));
    }
    const int ns = nt * K, g0 = r.x * K + (int)((long long)ns * sl / nsl), g1 = r.x * K + (int)((long long)ns * (sl + 1) / nsl);
    for (int g = g0 + threadIdx.x; g < g1; g += blockDim.x) {
        const double4 y = src[g];
        ms = fmax(ms, (y.x - cc.x) * (y.x - cc.x) + (y.y - cc.y) * (y.y - cc.y) + (y.z - cc.z) * (y.z - cc.z));
    }
    st[threadIdx.x] = mt;
    ss[threadIdx.x] = ms;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            st[threadIdx.x] = fmax(st[threadIdx.x], st[threadIdx.x + o]);
            ss[threadIdx.x] = fmax(ss[threadIdx.x], ss[threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        atomicMax(rad2 + 2 * c, (unsigned long long)__double_as_longlong(st[0]));
        atomicMax(rad2 + 2 * c + 1, (unsigned long long)__double_as_longlong(ss[0]));
    }
}

__global__ void k_cell_radii_sqrt(int ncells, const unsigned long long* rad2, double2* rad) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncells) return;
    rad[c] = make_double2(sqrt(__longlong_as_double((long long)rad2[2 * c])),
                          sqrt(__longlong_as_double((long long)rad2[2 * c + 1])));
}

// ---------------------------------------------------------------- dual-tree traversal
// One round over a frontier of (target cell, source cell) pairs: accepted pairs go
// to M2L, leaf-leaf pairs to P2P, the rest are split (both cells when they have the
// same size, else the larger / the non-leaf one). Acceptance: R_a + R_b < theta |c_a - c_b|
// with R_a the target radius of a and R_b the source radius of b.
__global__ void k_dtt_round(const int2* in, int n_in, const double4* cs, const int2* child, const int* clevel,
                            double theta, const double2* rad, int2* m2l, long long cap_m2l, int2* p2p, long long cap_p2p,
                            int2* next, long long cap_next, unsigned long long* cnt, int* overflow) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_in) return;
    const int a = in[i].x, b = in[i].y;
    const double4 ca = cs[a], cb = cs[b];
    const double Ra = rad[a].x, Rb = rad[b].y;
    const double dx = ca.x - cb.x, dy = ca.y - cb.y, dz = ca.z - cb.z;
    const double d = sqrt(dx * dx + dy * dy + dz * dz);
    // the multipole acceptance criterion with the cluster radii, and centres at least the
    // larger cell's side apart: the translation operator's entries grow like
    // rho^n (n + j)! / |v|^(n + j + 1) with v the offset in units of the target's side, and
    // a coarse cell holding a small piece of surface could otherwise pass with |v| << 1 and
    // carry entries beyond the FP32 range at p = 16 (on a closed surface mesh the cluster
    // radii already keep |v| above 2)
    if (Ra + Rb < theta * d && d >= fmax(ca.w, cb.w)) {
        unsigned long long k = atomicAdd(&cnt[0], 1ULL);
        if ((long long)k < cap_m2l) m2l[k] = make_int2(a, b); else atomicExch(overflow, 1);
        return;
    }
    const int2 cha = child[a], chb = child[b];
    if (cha.y == 0 && chb.y == 0) {
        unsigned long long k = atomicAdd(&cnt[1], 1ULL);
        if ((long long)k < cap_p2p) p2p[k] = make_int2(a, b); else atomicExch(overflow, 1);
        return;
    }
    bool sa, sb;
    if (cha.y == 0) { sa = false; sb = true; }
    else if (chb.y == 0) { sa = true; sb = false; }
    else if (clevel[a] == clevel[b]) { sa = sb = true; }
    else if (clevel[a] < clevel[b]) { sa = true; sb = false; }
    else { sa = false; sb = true; }
    const int na = sa ? cha.y : 1, nb = sb ? chb.y : 1;
    unsigned long long k0 = atomicAdd(&cnt[2], (unsigned long long)(na * nb));
    if ((long long)(k0 + na * nb) > cap_next) { atomicExch(overflow, 1); return; }
    for (int x = 0; x < na; ++x)
        for (int y = 0; y < nb; ++y)
            next[k0 + x * nb + y] = make_int2(sa ? cha.x + x : a, sb ? chb.x + y : b);
}

__global__ void k_pack_pairs(const int2* pr, long long n, long long ncells, unsigned long long* key) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    key[i] = (unsigned long long)pr[i].x * (unsigned long long)ncells + (unsigned long long)pr[i].y;
}

__global__ void k_unpack_src(const unsigned long long* key, long long n, long long ncells, int* src) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    src[i] = (int)(key[i] % (unsigned long long)ncells);
}

// ptr[c] = first sorted pair whose target >= c, for c = 0..ncells.
__global__ void k_csr_ptr(const unsigned long long* key, long long n, long long ncells, int* ptr) {
    long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c > ncells) return;
    const unsigned long long bound = (unsigned long long)c * (unsigned long long)ncells;
    long long lo = 0, hi = n;
    while (lo < hi) {
        long long mid = (lo + hi) >> 1;
        if (key[mid] < bound) lo = mid + 1; else hi = mid;
    }
    ptr[c] = (int)lo;
}

// Pair counts of the lists, and the shallowest levels holding an M2L source (lmin[0]) and an
// M2L target (lmin[1]): M2M above the first and L2L above the second carry nothing.
__global__ void k_list_stats(const int* m2l_ptr, const int* m2l_src, const int* p2p_ptr, const int* p2p_src,
                             const int* clevel, const int2* range, int ncells, int K,
                             unsigned long long* same_level, unsigned long long* p2p_inter, int* lmin) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncells) return;
    unsigned long long same = 0, inter = 0;
    int ls = 1 << 30;
    for (int e = m2l_ptr[c]; e < m2l_ptr[c + 1]; ++e) {
        same += (clevel[m2l_src[e]] == clevel[c]);
        ls = min(ls, clevel[m2l_src[e]]);
    }
    if (m2l_ptr[c + 1] > m2l_ptr[c]) {
        atomicMin(lmin, ls);
        atomicMin(lmin + 1, clevel[c]);
    }
    const int nt = range[c].y - range[c].x;
    for (int e = p2p_ptr[c]; e < p2p_ptr[c + 1]; ++e) {
        const int2 r = range[p2p_src[e]];
        inter += (unsigned long long)nt * (unsigned long long)(K * (r.y - r.x));
    }
    if (same) atomicAdd(same_level, same);
    if (inter) atomicAdd(p2p_inter, inter);
}

// Leaf-relative FP32 copies of the targets and Gauss points (the P2P operands in
// mixed precision): offsets from the leaf centre keep FP32 rounding relative to the
// leaf size instead of the domain size.
__global__ void k_relative(const int* leaves, const double4* cs, const int2* range, const double4* tgt,
                           const double4* src, int K, float4* tgt_rel, float4* src_rel) {
    const int cell = leaves[blockIdx.x];
    const double4 c = cs[cell];
    const int2 r = range[cell];
    for (int i = r.x + threadIdx.x; i < r.y; i += blockDim.x) {
        const double4 t = tgt[i];
        tgt_rel[i] = make_float4((float)(t.x - c.x), (float)(t.y - c.y), (float)(t.z - c.z), (float)t.w);
    }
    for (int g = r.x * K + threadIdx.x; g < r.y * K; g += blockDim.x) {
        const double4 y = src[g];
        src_rel[g] = make_float4((float)(y.x - c.x), (float)(y.y - c.y), (float)(y.z - c.z), (float)y.w);
    }
}

// Static P2P records per target leaf: the other leaves of its list form one stream
// of Gauss points; each pair stores its FP32 leaf-to-leaf shift, first Gauss point and
// offset in the stream (the self pair contributes nothing to the stream).
__global__ void k_p2p_records(const int* pptr, const int* psrc, const double4* cs, const int2* range, int ncells,
                              int K, float4* rec, int* off, int* len) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncells) return;
    const double4 ct = cs[c];
    int acc = 0;
    for (int e = pptr[c]; e < pptr[c + 1]; ++e) {
        const int s = psrc[e];
        const double4 cv = cs[s];
        const int2 r = range[s];
        rec[e] = make_float4((float)(cv.x - ct.x), (float)(cv.y - ct.y), (float)(cv.z - ct.z), __int_as_float(r.x * K));
        off[e] = acc;
        if (s != c) acc += K * (r.y - r.x);
    }
    len[c] = acc;
}

// Static stage plans of the bulk-copy near field: whole pairs, at most `tile` Gauss
// points and 64 pairs per stage, in list order. COUNT pass counts stages; FILL pass writes them.
template <bool FILL>
__global__ void k_p2p_plan(const int* pptr, const int* psrc, const int2* range, int ncells, int K, int tile,
                           int* nst, const int* sptr, int* cnt, int* toff, int* sfirst, int* sbytes) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncells) return;
    int ns = 0, fill = 0, npair = 0, out = FILL ? sptr[c] : 0;
    for (int e = pptr[c]; e < pptr[c + 1]; ++e) {
        const int2 r = range[psrc[e]];
        const int n = K * (r.y - r.x);
        if (ns == 0 || fill + n > tile || npair == 64) {
            if (FILL) {
                if (ns > 0) sbytes[out + ns - 1] = fill * 16;
                sfirst[out + ns] = e;
            }
            ++ns;
            fill = 0;
            npair = 0;
        }
        if (FILL) { cnt[e] = n; toff[e] = fill; }
        fill += n;
        ++npair;
    }
    if (FILL && ns > 0) sbytes[out + ns - 1] = fill * 16;
    if (!FILL) nst[c] = ns;
}

__global__ void k_leaf_class_key(const int* leaves, const int2* range, int n, int* key, int* counts) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int2 r = range[leaves[i]];
    const int nt = r.y - r.x;
    const int c = nt <= 32 ? 0 : (nt <= 64 ? 1 : 2);
    key[i] = c;
    atomicAdd(&counts[c], 1);
}

__global__ void k_leaves(const int2* child, const int2* range, int ncells, int* leaves, int* nleaf, int* maxp) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncells) return;
    if (child[c].y == 0) {
        leaves[atomicAdd(nleaf, 1)] = c;
        atomicMax(maxp, range[c].y - range[c].x);
    }
}

// ---------------------------------------------------------------- near-singular search
// For sorted target panel i: every panel j with j == i or |c_i - c_j|^2 < f^2 2 S_j,
// found by a depth-first walk that prunes cells farther than f sqrt(2 S_max).
template <bool FILL>
__global__ void k_near_search(const double4* tgt, int n, const double4* cs, const int2* child, const int2* range,
                              double f2, double r2max, int* count, const int* ptr, int* col, int* row) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double4 ci = tgt[i];
    int stack[8 * MAX_LEVELS + 8];
    int sp = 0;
    stack[sp++] = 0;
    int k = 0;
    int out = FILL ? ptr[i] : 0;
    while (sp > 0) {
        const int c = stack[--sp];
        const double4 b = cs[c];
        const double h = 0.5 * b.w;
        const double ex = fmax(fabs(ci.x - b.x) - h, 0.0), ey = fmax(fabs(ci.y - b.y) - h, 0.0),
                     ez = fmax(fabs(ci.z - b.z) - h, 0.0);
        if (ex * ex + ey * ey + ez * ez > r2max) continue;
        const int2 ch = child[c];
        if (ch.y == 0) {
            const int2 r = range[c];
            for (int j = r.x; j < r.y; ++j) {
                const double4 cj = tgt[j];
                const double dx = ci.x - cj.x, dy = ci.y - cj.y, dz = ci.z - cj.z;
                if (j == i || dx * dx + dy * dy + dz * dz < f2 * 2.0 * cj.w) {
                    if (FILL) { col[out + k] = j; row[out + k] = i; }
                    ++k;
                }
            }
        } else {
            for (int x = ch.y - 1; x >= 0; --x) stack[sp++] = ch.x + x;
        }
    }
    if (!FILL) count[i] = k;
}

// Semi-analytic self-panel integrals for a point c inside a flat triangle and in its
// plane (Sec. 2.3, Hess & Smith): the panel splits into three triangles (c, P_a, P_b);
// in polar coordinates about c the radial integral is exact, and for an edge at
// perpendicular distance h with end coordinates s1 < s2 along it the angular part is
//   int 1/r dA = h [asinh(s/h)],
//   int e e^T R(psi) dpsi = h { [sin] u u^T - [cos] (u w^T + w u^T) + [asinh(s/h) - sin] w w^T },
// u = unit vector from c to the foot of the perpendicular, w = edge direction.
__device__ void self_integrals(const double* P, const double* c, double* I1, double* D) {
    double acc = 0.0;
    for (int q = 0; q < 9; ++q) D[q] = 0.0;
    for (int a = 0; a < 3; ++a) {
        const double* A = P + 3 * a;
        const double* B = P + 3 * ((a + 1) % 3);
        double w[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]};
        const double L = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
        for (int d = 0; d < 3; ++d) w[d] /= L;
        const double t = (c[0] - A[0]) * w[0] + (c[1] - A[1]) * w[1] + (c[2] - A[2]) * w[2];
        double u[3];
        for (int d = 0; d < 3; ++d) u[d] = A[d] + t * w[d] - c[d];
        const double h = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        for (int d = 0; d < 3; ++d) u[d] /= h;
        const double s1 = -t, s2 = L - t;
        const double q1 = sqrt(s1 * s1 + h * h), q2 = sqrt(s2 * s2 + h * h);
        const double as = asinh(s2 / h) - asinh(s1 / h);
        const double ds = s2 / q2 - s1 / q1;  // sin(psi2) - sin(psi1)
        const double dc = h / q2 - h / q1;    // cos(psi2) - cos(psi1)
        acc += h * as;
        for (int x = 0; x < 3; ++x)
            for (int y = 0; y < 3; ++y)
                D[3 * x + y] += h * (ds * u[x] * u[y] - dc * (u[x] * w[y] + w[x] * u[y]) + (as - ds) * w[x] * w[y]);
    }
    *I1 = acc;
}

// Kernel sums of one rule over panel j seen from target c (unscaled):
//   sl[0]     : sum w / r                      (Laplace single layer)
//   dl[0]     : sum w n.(c - y) / r^3          (Laplace double layer)
//   sl[9]     : sum w (I/r + d d^T/r^3)        (Stokeslet)
//   dl[9]     : sum w 6 d d^T (e.n) / r^5, e = y - c = -d   (stresslet)
__device__ void rule_sums(const double* P, const double4 nj, const double* c, const double* quad, int nq,
                          bool stokes, double* sl, double* dl) {
    const int nout = stokes ? 9 : 1;
    for (int q = 0; q < nout; ++q) { sl[q] = 0.0; dl[q] = 0.0; }
    for (int k = 0; k < nq; ++k) {
        const double* g = quad + 4 * k;
        double d[3];
        for (int x = 0; x < 3; ++x) d[x] = c[x] - (g[0] * P[x] + g[1] * P[3 + x] + g[2] * P[6 + x]);
        const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        // one FP64 reciprocal square root per point instead of a square root and divisions
        // (FP64 throughput is scarce on this GPU); rsqrt is within 1 ulp
        const double ir = rsqrt(r2), ir2 = ir * ir, ir3 = ir2 * ir;
        const double w = g[3] * nj.w;
        const double dn = d[0] * nj.x + d[1] * nj.y + d[2] * nj.z;
        if (!stokes) {
            sl[0] += w * ir;
            dl[0] += w * dn * ir3;
        } else {
            const double ir5 = ir3 * ir2;
            for (int x = 0; x < 3; ++x)
                for (int y = 0; y < 3; ++y) {
                    sl[3 * x + y] += w * ((x == y ? ir : 0.0) + d[x] * d[y] * ir3);
                    dl[3 * x + y] += w * 6.0 * d[x] * d[y] * (-dn) * ir5;
                }
        }
    }
}

// The FP32 normal of each Gauss point's panel (sorted order: Gauss point g lies on panel g / K).
__global__ void k_point_normals(const float4* nrm_f, int K, int64_t ns, float4* out) {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g < ns) out[g] = nrm_f[g / K];
}

// Round FP64 values to FP32 (the mixed-precision correction pass reads the rounded table).
__global__ void k_round_f32(const double* in, int64_t n, float* out) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        out[e] = (float)in[e];
}

// Correction entries: self -> analytic single layer (double layer 0); near ->
// (20-point rule) - (K-point rule), so that P2P's K-point sum plus the entry gives
// the accurate integral.
__global__ void k_corrections(int64_t nnz, const int* row, const int* col, const double4* tgt, const double4* nrm,
                              const double* verts, const double* farq, int K, const double* nearq, int nq, bool stokes,
                              double* csl, double* cdl) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= nnz) return;
    const int i = row[e], j = col[e];
    const double4 ti = tgt[i];
    const double c[3] = {ti.x, ti.y, ti.z};
    double P[9];
    for (int q = 0; q < 9; ++q) P[q] = verts[9 * (int64_t)j + q];
    const int nout = stokes ? 9 : 1;
    if (i == j) {
        double I1, D[9];
        self_integrals(P, c, &I1, D);
        if (!stokes) {
            csl[e] = I1;
            cdl[e] = 0.0;
        } else {
            for (int q = 0; q < 9; ++q) { csl[9 * e + q] = D[q] + ((q % 4) == 0 ? I1 : 0.0); cdl[9 * e + q] = 0.0; }
        }
        return;
    }
    double sn[9], dn[9], sf[9], df[9];
    rule_sums(P, nrm[j], c, nearq, nq, stokes, sn, dn);
    rule_sums(P, nrm[j], c, farq, K, stokes, sf, df);
    for (int q = 0; q < nout; ++q) {
        csl[(int64_t)nout * e + q] = sn[q] - sf[q];
        cdl[(int64_t)nout * e + q] = dn[q] - df[q];
    }
}

int sort_pairs_to_csr(fmmbem_handle* h, int2* pairs, long long n, int** ptr_out, int** src_out) {
    cudaStream_t st = h->stream;
    const long long nc = h->n_cells;
    unsigned long long *k1 = nullptr, *k2 = nullptr;
    FMM_TRY(dalloc(&k1, n));
    FMM_TRY(dalloc(&k2, n));
    const int T = 256;
    if (n > 0) { k_pack_pairs<<<(unsigned)((n + T - 1) / T), T, 0, st>>>(pairs, n, nc, k1); FMM_LAUNCHED(); }
    int end_bit = 1;
    while (end_bit < 64 && ((unsigned long long)nc * (unsigned long long)nc >> end_bit) != 0) ++end_bit;
    FMM_TRY(radix_sort(reinterpret_cast<const uint64_t*>(k1), reinterpret_cast<uint64_t*>(k2), nullptr, nullptr, n,
                       end_bit, st));
    FMM_TRY(dalloc(ptr_out, nc + 1));
    FMM_TRY(dalloc(src_out, n));
    k_csr_ptr<<<(unsigned)((nc + 1 + T - 1) / T), T, 0, st>>>(k2, n, nc, *ptr_out);
    FMM_LAUNCHED();
    if (n > 0) { k_unpack_src<<<(unsigned)((n + T - 1) / T), T, 0, st>>>(k2, n, nc, *src_out); FMM_LAUNCHED(); }
    FMM_CU(cudaStreamSynchronize(st));
    fmm_free(k1);
    fmm_free(k2);
    return 0;
}

}  // namespace

int build_geometry_tree_lists(fmmbem_handle* h, const fmmbem_mesh* mesh) {
    cudaStream_t st = h->stream;
    const int64_t n = mesh->n_panels, nv = mesh->n_vertices;
    const int K = h->K;
    const int T = 256;
    const unsigned gn = (unsigned)((n + T - 1) / T);
    h->N = n;
    h->NS = (int64_t)K * n;

    // quadrature tables: [far K x 4 | near near_k x 4]
    double farq_h[7 * 4];
    if (far_rule_host(K, farq_h) != 0) {
        fmmbem_set_error("unsupported gauss_k=%d (use 1, 3, 4 or 7)", K);
        return FMMBEM_EINVAL;
    }
    const int nq = h->opts.near_k;
    int nu = 3;
    while (nu * (nu - 1) < nq) ++nu;
    if (nu * (nu - 1) != nq || nu > 7) {
        fmmbem_set_error("near_k=%d is not nu (nu - 1) for nu in 3..7", nq);
        return FMMBEM_EINVAL;
    }
    double* quad = nullptr;
    FMM_TRY(dalloc(&quad, 4 * (K + nq)));
    FMM_CU(cudaMemcpyAsync(quad, farq_h, sizeof(double) * 4 * K, cudaMemcpyHostToDevice, st));
    k_near_rule<<<1, 1, 0, st>>>(nu, nu - 1, quad + 4 * K);
    FMM_LAUNCHED();

    // upload mesh
    double* dv = nullptr;
    int* dt = nullptr;
    FMM_TRY(dalloc(&dv, 3 * nv));
    FMM_TRY(dalloc(&dt, 3 * n));
    FMM_CU(cudaMemcpyAsync(dv, mesh->vertices, sizeof(double) * 3 * nv, cudaMemcpyHostToDevice, st));
    FMM_CU(cudaMemcpyAsync(dt, mesh->triangles, sizeof(int) * 3 * n, cudaMemcpyHostToDevice, st));

    // geometry in the caller's order
    double4 *cen = nullptr, *nrm = nullptr;
    FMM_TRY(dalloc(&cen, n));
    FMM_TRY(dalloc(&nrm, n));
    unsigned long long* scal = nullptr;  // spill bits, max area bits, bad flag
    FMM_TRY(dalloc(&scal, 3));
    FMM_CU(cudaMemsetAsync(scal, 0, 3 * sizeof(unsigned long long), st));
    double* bbox = nullptr;
    FMM_TRY(dalloc(&bbox, 6));
    k_bbox<<<1, 256, 0, st>>>(dv, nv, bbox);
    FMM_LAUNCHED();
    k_panel_geom<<<gn, T, 0, st>>>(dv, nv, dt, n, cen, nrm, scal, scal + 1, (int*)(scal + 2));
    FMM_LAUNCHED();
    unsigned long long scal_h[3];
    double bbox_h[6];
    FMM_CU(cudaMemcpyAsync(scal_h, scal, sizeof(scal_h), cudaMemcpyDeviceToHost, st));
    FMM_CU(cudaMemcpyAsync(bbox_h, bbox, sizeof(bbox_h), cudaMemcpyDeviceToHost, st));
    FMM_CU(cudaStreamSynchronize(st));
    if ((int)scal_h[2] != 0) {
        fmmbem_set_error(scal_h[2] == 1 ? "triangle vertex index out of range" : "degenerate (zero-area) panel");
        return FMMBEM_EINVAL;
    }
    double spill, amax;
    memcpy(&spill, &scal_h[0], 8);
    memcpy(&amax, &scal_h[1], 8);
    h->spill = spill;
    double ext = 0.0;
    for (int d = 0; d < 3; ++d) {
        h->origin[d] = 0.5 * (bbox_h[d] + bbox_h[3 + d]);
        ext = std::max(ext, bbox_h[3 + d] - bbox_h[d]);
    }
    h->half = 0.5 * ext * (1.0 + 1e-9) + 1e-300;

    // Morton order
    uint64_t *key = nullptr, *key_s = nullptr;
    int *idx = nullptr;
    FMM_TRY(dalloc(&key, n));
    FMM_TRY(dalloc(&key_s, n));
    FMM_TRY(dalloc(&idx, n));
    FMM_TRY(dalloc(&h->perm, n));
    k_morton<<<gn, T, 0, st>>>(cen, n, h->origin[0] - h->half, h->origin[1] - h->half, h->origin[2] - h->half,
                               2.0 * h->half, key, idx);
    FMM_LAUNCHED();
    FMM_TRY(radix_sort(key, key_s, idx, h->perm, n, 63, st));

    FMM_TRY(dalloc(&h->tgt_d, n));
    FMM_TRY(dalloc(&h->tgt_f, n));
    FMM_TRY(dalloc(&h->nrm_d, n));
    FMM_TRY(dalloc(&h->nrm_f, n));
    FMM_TRY(dalloc(&h->verts, 9 * n));
    FMM_TRY(dalloc(&h->src_d, h->NS));
    FMM_TRY(dalloc(&h->src_f, h->NS));
    k_gather_sorted<<<gn, T, 0, st>>>(h->perm, n, dv, dt, cen, nrm, quad, K, h->tgt_d, h->tgt_f, h->nrm_d, h->nrm_f,
                                      h->verts, h->src_d, h->src_f);
    FMM_LAUNCHED();
    if (h->kernel == FMMBEM_STOKES) {  // the stresslet near field reads each source's normal with it
        FMM_TRY(dalloc(&h->nrm_pt, h->NS));
        k_point_normals<<<(unsigned)((h->NS + T - 1) / T), T, 0, st>>>(h->nrm_f, K, h->NS, h->nrm_pt);
        FMM_LAUNCHED();
    }

    // ---- octree, level by level
    {
        long long cap = std::max<long long>(64, 4 * (n / std::max(1, h->ncrit / K)) + 64);
        double4* cs = nullptr;
        int2 *range = nullptr, *child = nullptr;
        int *clevel = nullptr, *parent = nullptr;
        int *nch = nullptr, *off = nullptr, *bounds = nullptr;
        auto alloc_cells = [&](long long c) -> int {
            FMM_TRY(dalloc(&cs, c));
            FMM_TRY(dalloc(&range, c));
            FMM_TRY(dalloc(&child, c));
            FMM_TRY(dalloc(&clevel, c));
            FMM_TRY(dalloc(&parent, c));
            return 0;
        };
        FMM_TRY(alloc_cells(cap));
        double4 root = make_double4(h->origin[0], h->origin[1], h->origin[2], 2.0 * h->half);
        int2 rr = make_int2(0, (int)n), rc = make_int2(-1, 0);
        int zero = 0, minus1 = -1;
        FMM_CU(cudaMemcpyAsync(cs, &root, sizeof(root), cudaMemcpyHostToDevice, st));
        FMM_CU(cudaMemcpyAsync(range, &rr, sizeof(rr), cudaMemcpyHostToDevice, st));
        FMM_CU(cudaMemcpyAsync(child, &rc, sizeof(rc), cudaMemcpyHostToDevice, st));
        FMM_CU(cudaMemcpyAsync(clevel, &zero, sizeof(int), cudaMemcpyHostToDevice, st));
        FMM_CU(cudaMemcpyAsync(parent, &minus1, sizeof(int), cudaMemcpyHostToDevice, st));
        h->level_start.assign(1, 0);
        int lb = 0, le = 1, level = 0;
        long long scan_cap = 0;
        while (le > lb) {
            h->level_start.push_back(le);
            const int nl = le - lb;
            if (nl > scan_cap) {
                if (nch) { fmm_free(nch); fmm_free(off); fmm_free(bounds); }
                scan_cap = std::max<long long>(2 * nl, 1024);
                FMM_TRY(dalloc(&nch, scan_cap));
                FMM_TRY(dalloc(&off, scan_cap));
                FMM_TRY(dalloc(&bounds, 9 * scan_cap));
            }
            k_split_count<<<(nl + T - 1) / T, T, 0, st>>>(lb, le, level, range, key_s, K, h->ncrit, nch, bounds);
            FMM_LAUNCHED();
            FMM_TRY(exclusive_scan(nch, off, nl, st));
            int last[2];
            FMM_CU(cudaMemcpyAsync(&last[0], off + nl - 1, sizeof(int), cudaMemcpyDeviceToHost, st));
            FMM_CU(cudaMemcpyAsync(&last[1], nch + nl - 1, sizeof(int), cudaMemcpyDeviceToHost, st));
            FMM_CU(cudaStreamSynchronize(st));
            const int nnext = last[0] + last[1];
            if ((long long)le + nnext > cap) {
                long long ncap = std::max<long long>(2 * cap, (long long)le + nnext + 64);
                double4* cs2; int2 *r2, *c2; int *l2, *p2;
                FMM_TRY(dalloc(&cs2, ncap)); FMM_TRY(dalloc(&r2, ncap)); FMM_TRY(dalloc(&c2, ncap));
                FMM_TRY(dalloc(&l2, ncap)); FMM_TRY(dalloc(&p2, ncap));
                FMM_CU(cudaMemcpyAsync(cs2, cs, sizeof(double4) * le, cudaMemcpyDeviceToDevice, st));
                FMM_CU(cudaMemcpyAsync(r2, range, sizeof(int2) * le, cudaMemcpyDeviceToDevice, st));
                FMM_CU(cudaMemcpyAsync(c2, child, sizeof(int2) * le, cudaMemcpyDeviceToDevice, st));
                FMM_CU(cudaMemcpyAsync(l2, clevel, sizeof(int) * le, cudaMemcpyDeviceToDevice, st));
                FMM_CU(cudaMemcpyAsync(p2, parent, sizeof(int) * le, cudaMemcpyDeviceToDevice, st));
                FMM_CU(cudaStreamSynchronize(st));
                fmm_free(cs); fmm_free(range); fmm_free(child); fmm_free(clevel); fmm_free(parent);
                cs = cs2; range = r2; child = c2; clevel = l2; parent = p2;
                cap = ncap;
            }
            k_split_emit<<<(nl + T - 1) / T, T, 0, st>>>(lb, le, le, level, nch, off, bounds, cs, range, child, clevel,
                                                        parent);
            FMM_LAUNCHED();
            lb = le;
            le = le + nnext;
            ++level;
        }
        FMM_CU(cudaStreamSynchronize(st));
        fmm_free(nch); fmm_free(off); fmm_free(bounds);
        h->n_cells = le;
        h->n_levels = level;  // level_start has n_levels + 1 entries
        h->cell_cs = cs; h->cell_range = range; h->cell_child = child; h->cell_level = clevel; h->cell_parent = parent;
    }
    {
        // non-leaf cells by level: one M2M / L2L block each
        std::vector<int2> ch_h(h->n_cells);
        FMM_CU(cudaMemcpyAsync(ch_h.data(), h->cell_child, sizeof(int2) * h->n_cells, cudaMemcpyDeviceToHost, st));
        FMM_CU(cudaStreamSynchronize(st));
        std::vector<int> par;
        h->parent_start.assign(1, 0);
        for (int l = 0; l < h->n_levels; ++l) {
            for (int c = h->level_start[l]; c < h->level_start[l + 1]; ++c)
                if (ch_h[c].y > 0) par.push_back(c);
            h->parent_start.push_back((int)par.size());
        }
        FMM_TRY(dalloc(&h->parents, par.size()));
        if (!par.empty())
            FMM_CU(cudaMemcpyAsync(h->parents, par.data(), sizeof(int) * par.size(), cudaMemcpyHostToDevice, st));
        FMM_CU(cudaStreamSynchronize(st));
    }
    const int nc = h->n_cells;
    {
        int* cnt = nullptr;
        FMM_TRY(dalloc(&cnt, 2));
        FMM_CU(cudaMemsetAsync(cnt, 0, 2 * sizeof(int), st));
        FMM_TRY(dalloc(&h->leaves, nc));
        k_leaves<<<(nc + T - 1) / T, T, 0, st>>>(h->cell_child, h->cell_range, nc, h->leaves, cnt, cnt + 1);
        FMM_LAUNCHED();
        int cnt_h[2];
        FMM_CU(cudaMemcpyAsync(cnt_h, cnt, sizeof(cnt_h), cudaMemcpyDeviceToHost, st));
        FMM_CU(cudaStreamSynchronize(st));
        h->n_leaves = cnt_h[0];
        h->max_leaf_panels = cnt_h[1];
        fmm_free(cnt);
        // deterministic leaf order (ascending cell id)
        int* ls = nullptr;
        FMM_TRY(dalloc(&ls, h->n_leaves));
        // cell ids are non-negative, so their unsigned order is their order
        FMM_TRY(radix_sort(reinterpret_cast<const uint32_t*>(h->leaves), reinterpret_cast<uint32_t*>(ls), nullptr,
                           nullptr, h->n_leaves, 32, st));
        FMM_CU(cudaStreamSynchronize(st));
        fmm_free(h->leaves);
        h->leaves = ls;
        // leaves ordered by target-count class for the near-field kernels
        {
            int *ckey = nullptr, *ckey_s = nullptr, *counts = nullptr;
            FMM_TRY(dalloc(&ckey, h->n_leaves));
            FMM_TRY(dalloc(&ckey_s, h->n_leaves));
            FMM_TRY(dalloc(&counts, 3));
            FMM_TRY(dalloc(&h->leaf_class, h->n_leaves));
            FMM_CU(cudaMemsetAsync(counts, 0, 3 * sizeof(int), st));
            k_leaf_class_key<<<(h->n_leaves + T - 1) / T, T, 0, st>>>(h->leaves, h->cell_range, h->n_leaves, ckey, counts);
            FMM_LAUNCHED();
            FMM_TRY(radix_sort(reinterpret_cast<const uint32_t*>(ckey), reinterpret_cast<uint32_t*>(ckey_s), h->leaves,
                               h->leaf_class, h->n_leaves, 2, st));
            int c_h[3];
            FMM_CU(cudaMemcpyAsync(c_h, counts, sizeof(c_h), cudaMemcpyDeviceToHost, st));
            FMM_CU(cudaStreamSynchronize(st));
            fmm_free(ckey); fmm_free(ckey_s); fmm_free(counts);
            h->leaf_class_start[0] = 0;
            h->leaf_class_start[1] = c_h[0];
            h->leaf_class_start[2] = c_h[0] + c_h[1];
            h->leaf_class_start[3] = h->n_leaves;
        }
        FMM_TRY(dalloc(&h->tgt_rel, n));
        FMM_TRY(dalloc(&h->src_rel, h->NS));
        if (h->n_leaves > 0) {
            k_relative<<<h->n_leaves, 256, 0, st>>>(h->leaves, h->cell_cs, h->cell_range, h->tgt_d, h->src_d, K,
                                                    h->tgt_rel, h->src_rel);
            FMM_LAUNCHED();
        }
    }

    // ---- dual-tree traversal
    {
        FMM_TRY(dalloc(&h->cell_rad, nc));
        {
            unsigned long long* rad2 = nullptr;
            FMM_TRY(dalloc(&rad2, 2 * (size_t)nc));
            FMM_CU(cudaMemsetAsync(rad2, 0, sizeof(unsigned long long) * 2 * nc, st));
            k_cell_radii<<<dim3(nc, 16), 128, 0, st>>>(nc, h->cell_cs, h->cell_range, h->tgt_d, h->src_d, K, rad2);
            FMM_LAUNCHED();
            k_cell_radii_sqrt<<<(nc + T - 1) / T, T, 0, st>>>(nc, rad2, h->cell_rad);
            FMM_LAUNCHED();
            fmm_free(rad2);
        }
        long long cap_m2l = std::max<long long>(1024, 256LL * nc), cap_p2p = std::max<long long>(1024, 64LL * nc);
        long long cap_f = std::max<long long>(4096, 64LL * nc);
        int2 *m2l = nullptr, *p2p = nullptr, *fa = nullptr, *fb = nullptr;
        FMM_TRY(dalloc(&m2l, cap_m2l));
        FMM_TRY(dalloc(&p2p, cap_p2p));
        FMM_TRY(dalloc(&fa, cap_f));
        FMM_TRY(dalloc(&fb, cap_f));
        unsigned long long* cnt = nullptr;
        int* ovf = nullptr;
        FMM_TRY(dalloc(&cnt, 3));
        FMM_TRY(dalloc(&ovf, 1));
        int2 root = make_int2(0, 0);
        FMM_CU(cudaMemcpyAsync(fa, &root, sizeof(root), cudaMemcpyHostToDevice, st));
        unsigned long long done[3] = {0, 0, 0};
        long long nf = 1;
        int rounds = 0;
        while (nf > 0) {
            if (++rounds > 4 * MAX_LEVELS + 8) { fmmbem_set_error("dual-tree traversal did not terminate"); return FMMBEM_EDEVICE; }
            for (;;) {
                unsigned long long c0[3] = {done[0], done[1], 0};
                FMM_CU(cudaMemcpyAsync(cnt, c0, sizeof(c0), cudaMemcpyHostToDevice, st));
                FMM_CU(cudaMemsetAsync(ovf, 0, sizeof(int), st));
                k_dtt_round<<<(unsigned)((nf + T - 1) / T), T, 0, st>>>(fa, (int)nf, h->cell_cs, h->cell_child,
                                                                       h->cell_level, h->theta, h->cell_rad, m2l, cap_m2l,
                                                                       p2p, cap_p2p, fb, cap_f, cnt, ovf);
                FMM_LAUNCHED();
                unsigned long long c1[3];
                int o;
                FMM_CU(cudaMemcpyAsync(c1, cnt, sizeof(c1), cudaMemcpyDeviceToHost, st));
                FMM_CU(cudaMemcpyAsync(&o, ovf, sizeof(int), cudaMemcpyDeviceToHost, st));
                FMM_CU(cudaStreamSynchronize(st));
                if (!o) { done[0] = c1[0]; done[1] = c1[1]; nf = (long long)c1[2]; break; }
                // grow whichever list overflowed, keeping the pairs already written
                auto grow = [&](int2** buf, long long& cap, long long need, long long keep) -> int {
                    if (need <= cap) return 0;
                    long long ncap = std::max(2 * cap, need + need / 4);
                    int2* nb = nullptr;
                    FMM_TRY(dalloc(&nb, ncap));
                    if (keep) FMM_CU(cudaMemcpyAsync(nb, *buf, keep * sizeof(int2), cudaMemcpyDeviceToDevice, st));
                    FMM_CU(cudaStreamSynchronize(st));
                    fmm_free(*buf);
                    *buf = nb;
                    cap = ncap;
                    return 0;
                };
                FMM_TRY(grow(&m2l, cap_m2l, (long long)c1[0], (long long)done[0]));
                FMM_TRY(grow(&p2p, cap_p2p, (long long)c1[1], (long long)done[1]));
                if ((long long)c1[2] > cap_f) {
                    long long ncap = (long long)c1[2] + (long long)c1[2] / 4;
                    int2 *na = nullptr, *nb = nullptr;
                    FMM_TRY(dalloc(&na, ncap));
                    FMM_TRY(dalloc(&nb, ncap));
                    FMM_CU(cudaMemcpyAsync(na, fa, nf * sizeof(int2), cudaMemcpyDeviceToDevice, st));
                    FMM_CU(cudaStreamSynchronize(st));
                    fmm_free(fa); fmm_free(fb);
                    fa = na; fb = nb; cap_f = ncap;
                }
            }
            std::swap(fa, fb);
        }
        h->n_m2l = (int64_t)done[0];
        h->n_p2p = (int64_t)done[1];
        FMM_TRY(sort_pairs_to_csr(h, m2l, (long long)done[0], &h->m2l_ptr, &h->m2l_src));
        FMM_TRY(sort_pairs_to_csr(h, p2p, (long long)done[1], &h->p2p_ptr, &h->p2p_src));
        fmm_free(m2l); fmm_free(p2p); fmm_free(fa); fmm_free(fb); fmm_free(ovf);
        FMM_CU(cudaMemsetAsync(cnt, 0, 2 * sizeof(unsigned long long), st));
        int* lmin = reinterpret_cast<int*>(cnt + 2);
        const int lmin_init[2] = {1 << 30, 1 << 30};
        FMM_CU(cudaMemcpyAsync(lmin, lmin_init, sizeof(lmin_init), cudaMemcpyHostToDevice, st));
        k_list_stats<<<(nc + T - 1) / T, T, 0, st>>>(h->m2l_ptr, h->m2l_src, h->p2p_ptr, h->p2p_src, h->cell_level,
                                                    h->cell_range, nc, K, cnt, cnt + 1, lmin);
        FMM_LAUNCHED();
        unsigned long long s_h[3];
        FMM_CU(cudaMemcpyAsync(s_h, cnt, sizeof(s_h), cudaMemcpyDeviceToHost, st));
        FMM_CU(cudaStreamSynchronize(st));
        h->n_m2l_same = (int64_t)s_h[0];
        h->n_p2p_inter = (int64_t)s_h[1];
        int lmin_h[2];
        memcpy(lmin_h, &s_h[2], sizeof(lmin_h));
        h->m2m_lmin = std::min(lmin_h[0], h->n_levels);
        h->l2l_lmin = std::min(lmin_h[1], h->n_levels);
        fmm_free(cnt);
        FMM_TRY(dalloc(&h->p2p_rec, h->n_p2p));
        FMM_TRY(dalloc(&h->p2p_off, h->n_p2p));
        FMM_TRY(dalloc(&h->p2p_len, nc));
        k_p2p_records<<<(nc + T - 1) / T, T, 0, st>>>(h->p2p_ptr, h->p2p_src, h->cell_cs, h->cell_range, nc, K,
                                                     h->p2p_rec, h->p2p_off, h->p2p_len);
        FMM_LAUNCHED();
        {
            // source-lane kernel work in decreasing order (targets x stream length), so that its
            // blocks, issued in order, finish together
            const int nl = h->n_leaves;
            std::vector<int> lv(nl), len(nc);
            std::vector<int2> rg(nc);
            FMM_CU(cudaMemcpyAsync(lv.data(), h->leaves, sizeof(int) * nl, cudaMemcpyDeviceToHost, st));
            FMM_CU(cudaMemcpyAsync(len.data(), h->p2p_len, sizeof(int) * nc, cudaMemcpyDeviceToHost, st));
            FMM_CU(cudaMemcpyAsync(rg.data(), h->cell_range, sizeof(int2) * nc, cudaMemcpyDeviceToHost, st));
            FMM_CU(cudaStreamSynchronize(st));
            // work items of the source-lane kernel: (leaf, first target, target count), a leaf's
            // targets split evenly into chunks of at most tmax, largest work first
            std::vector<int4> items;
            std::vector<long long> cost;
            const int tmax = h->kernel == FMMBEM_STOKES ? P2P_SRC_TMAX_STOKES
                                                        : (h->nrhs > 1 ? P2P_SRC_TMAX_BATCH : P2P_SRC_TMAX);
            for (int c : lv) {
                const int t = rg[c].y - rg[c].x;
                const int nchk = (t + tmax - 1) / tmax;
                for (int q = 0; q < nchk; ++q) {
                    const int b = rg[c].x + (int)((long long)t * q / nchk), e = rg[c].x + (int)((long long)t * (q + 1) / nchk);
                    items.push_back(make_int4(c, b, e - b, 0));
                    cost.push_back((long long)(e - b) * ((long long)len[c] + (long long)t * K));
                }
            }
            std::vector<int> idx(items.size());
            for (size_t q = 0; q < idx.size(); ++q) idx[q] = (int)q;
            std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return cost[a] > cost[b]; });
            std::vector<int4> sorted(items.size());
            for (size_t q = 0; q < idx.size(); ++q) sorted[q] = items[idx[q]];
            h->n_p2p_items = (int)sorted.size();
            FMM_TRY(dalloc(&h->p2p_items, sorted.size()));
            FMM_CU(cudaMemcpyAsync(h->p2p_items, sorted.data(), sizeof(int4) * sorted.size(), cudaMemcpyHostToDevice, st));
            FMM_CU(cudaStreamSynchronize(st));
        }
        // stage plans of the bulk-copy near field (leaves of at most 1024 Gauss points)
        if ((int64_t)K * h->max_leaf_panels <= 1024) {
            int* nst = nullptr;
            FMM_TRY(dalloc(&nst, nc + 1));
            FMM_CU(cudaMemsetAsync(nst, 0, sizeof(int) * (nc + 1), st));
            k_p2p_plan<false><<<(nc + T - 1) / T, T, 0, st>>>(h->p2p_ptr, h->p2p_src, h->cell_range, nc, K, 1024, nst,
                                                            nullptr, nullptr, nullptr, nullptr, nullptr);
            FMM_LAUNCHED();
            FMM_TRY(dalloc(&h->stage_ptr, nc + 1));
            FMM_TRY(exclusive_scan(nst, h->stage_ptr, nc + 1, st));
            int nstages = 0;
            FMM_CU(cudaMemcpyAsync(&nstages, h->stage_ptr + nc, sizeof(int), cudaMemcpyDeviceToHost, st));
            FMM_CU(cudaStreamSynchronize(st));
            fmm_free(nst);
            h->n_stages = nstages;
            FMM_TRY(dalloc(&h->stage_first, nstages));
            FMM_TRY(dalloc(&h->stage_bytes, nstages));
            FMM_TRY(dalloc(&h->p2p_cnt, h->n_p2p));
            FMM_TRY(dalloc(&h->p2p_toff, h->n_p2p));
            k_p2p_plan<true><<<(nc + T - 1) / T, T, 0, st>>>(h->p2p_ptr, h->p2p_src, h->cell_range, nc, K, 1024, nullptr,
                                                           h->stage_ptr, h->p2p_cnt, h->p2p_toff, h->stage_first,
                                                           h->stage_bytes);
            FMM_LAUNCHED();
        }
    }

    // ---- near-singular table
    {
        const double f2 = h->opts.near_factor * h->opts.near_factor;
        const double r2max = f2 * 2.0 * amax * (1.0 + 1e-12);
        int *count = nullptr;
        FMM_TRY(dalloc(&count, n + 1));
        FMM_CU(cudaMemsetAsync(count, 0, sizeof(int) * (n + 1), st));
        k_near_search<false><<<gn, T, 0, st>>>(h->tgt_d, (int)n, h->cell_cs, h->cell_child, h->cell_range, f2, r2max,
                                               count, nullptr, nullptr, nullptr);
        FMM_LAUNCHED();
        FMM_TRY(dalloc(&h->corr_ptr, n + 1));
        FMM_TRY(exclusive_scan(count, h->corr_ptr, n + 1, st));
        int nnz = 0;
        FMM_CU(cudaMemcpyAsync(&nnz, h->corr_ptr + n, sizeof(int), cudaMemcpyDeviceToHost, st));
        FMM_CU(cudaStreamSynchronize(st));
        h->n_corr = nnz;
        int* row = nullptr;
        FMM_TRY(dalloc(&row, nnz));
        FMM_TRY(dalloc(&h->corr_col, nnz));
        k_near_search<true><<<gn, T, 0, st>>>(h->tgt_d, (int)n, h->cell_cs, h->cell_child, h->cell_range, f2, r2max,
                                              nullptr, h->corr_ptr, h->corr_col, row);
        FMM_LAUNCHED();
        const bool stokes = h->kernel == FMMBEM_STOKES;
        const int per = stokes ? 9 : 1;
        FMM_TRY(dalloc(&h->corr_sl, (int64_t)per * nnz));
        FMM_TRY(dalloc(&h->corr_dl, (int64_t)per * nnz));
        if (nnz > 0) {
            k_corrections<<<(unsigned)((nnz + 127) / 128), 128, 0, st>>>(nnz, row, h->corr_col, h->tgt_d, h->nrm_d,
                                                                       h->verts, quad, K, quad + 4 * K, nq, stokes,
                                                                       h->corr_sl, h->corr_dl);
            FMM_LAUNCHED();
        }
        FMM_TRY(dalloc(&h->corr_sl_f, (int64_t)per * nnz));
        FMM_TRY(dalloc(&h->corr_dl_f, (int64_t)per * nnz));
        if (nnz > 0) {
            const int64_t m = (int64_t)per * nnz;
            k_round_f32<<<(unsigned)std::min<int64_t>((m + 255) / 256, 4096), 256, 0, st>>>(h->corr_sl, m, h->corr_sl_f);
            k_round_f32<<<(unsigned)std::min<int64_t>((m + 255) / 256, 4096), 256, 0, st>>>(h->corr_dl, m, h->corr_dl_f);
            FMM_LAUNCHED();
        }
        FMM_CU(cudaStreamSynchronize(st));
        fmm_free(row);
        fmm_free(count);
    }

    fmm_free(quad); fmm_free(dv); fmm_free(dt); fmm_free(cen); fmm_free(nrm); fmm_free(scal); fmm_free(bbox);
    fmm_free(key); fmm_free(key_s); fmm_free(idx);
    return 0;
}

}  // namespace fmmbem
