// M2L as batched dense products against precomputed translation operators.
//
// With expansions scaled by the cell side (M~_n = M_n / s^n, L^_j = L_j s^{j+1}), the
// M2L operator of a pair depends only on v = (c_t - c_s) / s_t and on the size ratio
// rho = s_s / s_t = 2^dl:
//   L^_j^k = (-1)^j conj( sum_{n,m} rho^n M~_n^m I_{n+j}^{m+k}(v) )
// (Sec. 2.5; the complex form is derived in harmonics.cuh). For cells of one octree v
// is a multiple of 1/256 for dl >= -7, so every pair of the dual-tree traversal maps to
// one of a few thousand distinct operators. Each operator is stored once as a real
// matrix acting on the interleaved (Re, Im) coefficients, ordered by degree so that the
// leading 2 ncoef(p) x 2 ncoef(p) block is the order-p operator for every p <= p_max.
// The pairs of one operator form a GEMM: L[t_i] += T X[s_i] over the pairs i of the group.
// Reflections of the coordinate axes map solid harmonics to themselves up to signs and
// conjugation (z -> -z: (-1)^{n+m}; y -> -y: conj; x -> -x: (-1)^m conj), so in real
// form T_v = D_Q T_{Qv} D_Q with D_Q diagonal +-1. Operators are stored only for
// v with non-negative components; each pair carries the reflection Q (3 bits) that maps
// its v there, and the products apply D_Q to the gathered input and to the output.
#include <algorithm>
#include <type_traits>
#include "handle.cuh"
#include "harmonics.cuh"

namespace fmmbem {

namespace {

// Operator key: 4 bits of level difference dl + 8 (dl in [-8, 7]) above three coordinates of
// KEY_BITS bits, each KEY_RES v + KEY_BIAS. A centre offset is a multiple of 2^(dl - 1) target
// sides when the source is the smaller cell (dl < 0) and of 1/2 otherwise, so a resolution of
// 1/256 represents every offset exactly for dl >= -7, up to |v| < 2048.
constexpr int KEY_BITS = 20;
constexpr int KEY_BIAS = 1 << (KEY_BITS - 1);
constexpr double KEY_RES = 256.0;
constexpr int GEMM_THREADS = 256;     // 16 x 16 threads
constexpr int GEMM_COLS = 64;         // (pair, component) columns per tile
constexpr int GEMM_KC = 16;           // inputs per shared-memory stage

template <typename P>
int dalloc(P** p, size_t count) {
    *p = nullptr;
    FMM_CU(fmm_malloc((void**)p, (count ? count : 1) * sizeof(P)));
    return 0;
}

// Rows per thread of the 16 x 16 thread grid for order p: 16 RPT >= 2 ncoef(p).
int rpt_for(int p) {
    const int rows = 2 * ncoef(p);
    const int opts[] = {1, 2, 4, 8, 12, 16, 20};
    for (int r : opts)
        if (16 * r >= rows) return r;
    return 20;
}

__global__ void k_expand_pairs(const int* ptr, const int* src, int ncells, int* pt, int* ps) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncells) return;
    for (int e = ptr[c]; e < ptr[c + 1]; ++e) { pt[e] = c; ps[e] = src[e]; }
}

__global__ void k_pair_keys(const int* pt, const int* ps, long long n, const double4* cs, const int* lev,
                            unsigned long long* key, int* idx, int* refl, int* bad) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int t = pt[i], s = ps[i];
    const double4 ct = cs[t], cv = cs[s];
    const int dl = lev[t] - lev[s];
    const double is = KEY_RES / ct.w;
    long long kx = llrint((ct.x - cv.x) * is), ky = llrint((ct.y - cv.y) * is), kz = llrint((ct.z - cv.z) * is);
    const int q = (kx < 0 ? 1 : 0) | (ky < 0 ? 2 : 0) | (kz < 0 ? 4 : 0);  // reflection to the canonical octant
    kx = llabs(kx);
    ky = llabs(ky);
    kz = llabs(kz);
    if (dl < -7 || dl > 7 || kx >= KEY_BIAS || ky >= KEY_BIAS || kz >= KEY_BIAS) atomicExch(bad, 1);
    key[i] = ((unsigned long long)(dl + 8) << (3 * KEY_BITS)) | ((unsigned long long)(kx + KEY_BIAS) << (2 * KEY_BITS)) |
             ((unsigned long long)(ky + KEY_BIAS) << KEY_BITS) | (unsigned long long)(kz + KEY_BIAS);
    idx[i] = (int)i;
    refl[i] = q;
}

__global__ void k_mark_heads(const unsigned long long* key, long long n, int* head) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    head[i] = (i == 0 || key[i] != key[i - 1]) ? 1 : 0;
}

// After an inclusive scan of the head flags: table id of each sorted pair, the
// permuted pair arrays, and the first pair / key of each table.
__global__ void k_assign_tables(const unsigned long long* key, const int* idx, const int* scan, long long n,
                                const int* pt, const int* ps, const int* refl, int* st, int* ss, int* sr, int* tab_first,
                                unsigned long long* tab_key) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i > n) return;
    if (i == n) { tab_first[scan[n - 1]] = (int)n; return; }
    const int id = scan[i] - 1;
    st[i] = pt[idx[i]];
    ss[i] = ps[idx[i]];
    sr[i] = refl[idx[i]];
    if (i == 0 || key[i] != key[i - 1]) { tab_first[id] = (int)i; tab_key[id] = key[i]; }
}

__global__ void k_tile_counts(const int* tab_first, int ntab, int per_tile, int* cnt) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ntab) return;
    cnt[g] = (tab_first[g + 1] - tab_first[g] + per_tile - 1) / per_tile;
}

__global__ void k_tile_emit(const int* tab_first, const int* off, int ntab, int per_tile, int4* tiles) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ntab) return;
    const int a = tab_first[g], b = tab_first[g + 1];
    int k = off[g];
    for (int p0 = a; p0 < b; p0 += per_tile, ++k) tiles[k] = make_int4(g, p0, min(per_tile, b - p0), 0);
}

// Real matrix of one operator, stored input-major: T[k * ld + r], k = input real
// index 2 cidx(n, mu) + {0: Re, 1: Im}, r = output real index 2 cidx(j, kk) + {0, 1}.
// With A = I_{n+j}^{mu+kk}, B = (-1)^mu I_{n+j}^{kk-mu} (mu > 0; B = 0 for mu = 0)
// and s = (-1)^j, the contribution of M = a + i b to L is
//   Re L += s [a (A_r + B_r) + b (B_i - A_i)],  Im L -= s [a (A_i + B_i) + b (A_r - B_r)],
// scaled by rho^n.
__global__ void k_gen_tables(const unsigned long long* tab_key, int pmax, int ld, double* Td, float* Tf) {
    __shared__ cpx<double> sI[NI_MAX];
    const int g = blockIdx.x;
    const unsigned long long key = tab_key[g];
    const int mask = (1 << KEY_BITS) - 1;
    const int dl = (int)(key >> (3 * KEY_BITS)) - 8;
    const double vx = ((int)((key >> (2 * KEY_BITS)) & mask) - KEY_BIAS) / KEY_RES;
    const double vy = ((int)((key >> KEY_BITS) & mask) - KEY_BIAS) / KEY_RES;
    const double vz = ((int)(key & mask) - KEY_BIAS) / KEY_RES;
    if (threadIdx.x <= 2 * pmax) irregular_column<double>(vx, vy, vz, threadIdx.x, 2 * pmax, sI);
    __syncthreads();
    const int nr = 2 * ncoef(pmax);
    const size_t base = (size_t)g * nr * ld;
    for (int e = threadIdx.x; e < nr * ld; e += blockDim.x) {
        const int k = e / ld, r = e % ld;
        double val = 0.0;
        if (r < nr) {
            const int qi = k >> 1, qo = r >> 1;
            int n = 0, j = 0;
            while ((n + 1) * (n + 2) / 2 <= qi) ++n;
            while ((j + 1) * (j + 2) / 2 <= qo) ++j;
            const int mu = qi - n * (n + 1) / 2, kk = qo - j * (j + 1) / 2;
            const cpx<double> A = sI[cidx(n + j, mu + kk)];
            cpx<double> B = mk(0.0, 0.0);
            if (mu > 0) {
                B = coef_any(sI, n + j, kk - mu);
                if (mu & 1) B = mk(-B.re, -B.im);
            }
            const double s = (j & 1) ? -1.0 : 1.0;
            double d;
            if ((r & 1) == 0) d = (k & 1) == 0 ? s * (A.re + B.re) : s * (B.im - A.im);
            else d = (k & 1) == 0 ? -s * (A.im + B.im) : -s * (A.re - B.re);
            val = ldexp(d, dl * n);
        }
        Td[base + e] = val;
        Tf[base + e] = (float)val;
    }
}

// sign[q][k] of real coefficient k = 2 cidx(n, m) + part under reflection q (bit 0: x,
// bit 1: y, bit 2: z): z -> (-1)^{n+m}; y -> conj (Im negated); x -> (-1)^m conj.
__global__ void k_refl_signs(float* sf, double* sd) {
    const int q = blockIdx.x;
    for (int k = threadIdx.x; k < ESTRIDE; k += blockDim.x) {
        double v = 0.0;
        if (k < 2 * NCOEF_MAX) {
            const int c = k >> 1, part = k & 1;
            int n = 0;
            while ((n + 1) * (n + 2) / 2 <= c) ++n;
            const int m = c - n * (n + 1) / 2;
            v = 1.0;
            if (q & 4) v *= ((n + m) & 1) ? -1.0 : 1.0;
            if ((q & 2) && part) v = -v;
            if (q & 1) {
                if (m & 1) v = -v;
                if (part) v = -v;
            }
        }
        sf[q * ESTRIDE + k] = (float)v;
        sd[q * ESTRIDE + k] = v;
    }
}

template <typename T> struct Vec4;
template <> struct Vec4<float> { typedef float4 type; };
template <> struct Vec4<double> { typedef double4 type; };

// One tile = up to GEMM_COLS (pair, component) columns of one operator. Thread
// (ty, tx) of the 16 x 16 grid owns rows [ty RPT, ty RPT + RPT) and columns
// [4 tx, 4 tx + 4). Inputs beyond 2 ncoef(p) are masked to zero (the M array keeps
// stale higher degrees from earlier calls at larger p).
template <typename T, int RPT, int NC>
__global__ void __launch_bounds__(GEMM_THREADS) k_m2l_gemm(int p, const int4* tiles, const int* pt, const int* ps,
                                                          const int* prefl, const T* sign, const T* tables,
                                                          size_t tab_stride, int ld, const T* M, T* L, size_t msys) {
    constexpr int RP = 16 * RPT;
    M += blockIdx.y * msys;  // copy blockIdx.y of a Stokes batch
    L += blockIdx.y * msys;
    __shared__ __align__(16) T sA[GEMM_KC][RP];
    __shared__ __align__(16) T sB[GEMM_KC][GEMM_COLS];
    const int4 tile = tiles[blockIdx.x];
    const int ncols = tile.z * NC;
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
    const int kmax = 2 * ncoef(p);
    const T* Tg = tables + (size_t)tile.x * tab_stride;
    T acc[RPT][4];
#pragma unroll
    for (int i = 0; i < RPT; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
    for (int k0 = 0; k0 < kmax; k0 += GEMM_KC) {
        __syncthreads();
        for (int e = tid; e < GEMM_KC * RP; e += GEMM_THREADS) {
            const int kk = e / RP, r = e % RP;
            const int k = k0 + kk;
            sA[kk][r] = (k < kmax) ? Tg[(size_t)k * ld + r] : T(0);
        }
        for (int e = tid; e < GEMM_KC * GEMM_COLS; e += GEMM_THREADS) {
            const int col = e / GEMM_KC, kk = e % GEMM_KC;
            const int k = k0 + kk;
            T v = T(0);
            if (col < ncols && k < kmax) {
                const int pr = tile.y + col / NC, c = col % NC;
                v = M[((size_t)ps[pr] * NC + c) * ESTRIDE + k] * sign[prefl[pr] * ESTRIDE + k];
            }
            sB[kk][col] = v;
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < GEMM_KC; ++kk) {
            T a[RPT], b[4];
#pragma unroll
            for (int i = 0; i < RPT; ++i) a[i] = sA[kk][ty * RPT + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = sB[kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < RPT; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
        }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int col = tx * 4 + j;
        if (col >= ncols) continue;
        const int pr = tile.y + col / NC, c = col % NC;
        T* dst = L + ((size_t)pt[pr] * NC + c) * ESTRIDE;
        const int r0 = ty * RPT;
        const T* sg = sign + prefl[pr] * ESTRIDE;
#pragma unroll
        for (int i = 0; i < RPT; ++i) acc[i][j] *= sg[r0 + i];
        if (std::is_same<T, float>::value && (RPT % 4) == 0) {
#pragma unroll
            for (int i = 0; i < RPT; i += 4) {
                if (r0 + i >= kmax) break;
                float4 v = make_float4((float)acc[i][j], (float)acc[i + 1][j], (float)acc[i + 2][j], (float)acc[i + 3][j]);
                atomicAdd(reinterpret_cast<float4*>(reinterpret_cast<float*>(dst) + r0 + i), v);
            }
        } else {
#pragma unroll
            for (int i = 0; i < RPT; ++i)
                if (r0 + i < kmax) atomicAdd(dst + r0 + i, acc[i][j]);
        }
    }
}

}  // namespace

int build_m2l_tables(fmmbem_handle* h) {
    cudaStream_t st = h->stream;
    const long long n = h->n_m2l;
    h->m2l_tables = false;
    if (n == 0) return 0;
    const int T = 256;
    const unsigned gp = (unsigned)((n + T - 1) / T);
    int *pt = nullptr, *ps = nullptr, *idx = nullptr, *idx_s = nullptr, *head = nullptr, *scan = nullptr, *bad = nullptr;
    int* refl = nullptr;
    unsigned long long *key = nullptr, *key_s = nullptr;
    FMM_TRY(dalloc(&pt, n)); FMM_TRY(dalloc(&ps, n)); FMM_TRY(dalloc(&idx, n)); FMM_TRY(dalloc(&idx_s, n));
    FMM_TRY(dalloc(&head, n)); FMM_TRY(dalloc(&scan, n)); FMM_TRY(dalloc(&bad, 1));
    FMM_TRY(dalloc(&key, n)); FMM_TRY(dalloc(&key_s, n)); FMM_TRY(dalloc(&refl, n));
    FMM_CU(cudaMemsetAsync(bad, 0, sizeof(int), st));
    k_expand_pairs<<<(h->n_cells + T - 1) / T, T, 0, st>>>(h->m2l_ptr, h->m2l_src, h->n_cells, pt, ps);
    FMM_LAUNCHED();
    k_pair_keys<<<gp, T, 0, st>>>(pt, ps, n, h->cell_cs, h->cell_level, key, idx, refl, bad);
    FMM_LAUNCHED();
    FMM_TRY(radix_sort(reinterpret_cast<const uint64_t*>(key), reinterpret_cast<uint64_t*>(key_s), idx, idx_s, n,
                       3 * KEY_BITS + 4, st));
    k_mark_heads<<<gp, T, 0, st>>>(key_s, n, head);
    FMM_LAUNCHED();
    FMM_TRY(inclusive_scan(head, scan, n, st));
    int ntab = 0, bad_h = 0;
    FMM_CU(cudaMemcpyAsync(&ntab, scan + n - 1, sizeof(int), cudaMemcpyDeviceToHost, st));
    FMM_CU(cudaMemcpyAsync(&bad_h, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
    FMM_CU(cudaStreamSynchronize(st));
    const int pmax = h->opts.p_max;
    const int ld = 16 * rpt_for(pmax);
    const size_t per = (size_t)2 * ncoef(pmax) * ld;
    const size_t bytes = (size_t)ntab * per * (sizeof(double) + sizeof(float));
    if (bad_h || bytes > ((size_t)16 << 30)) {
        // keys out of range or tables too large: the gather kernel (k_m2l) handles M2L
        fmm_free(pt); fmm_free(ps); fmm_free(idx); fmm_free(idx_s); fmm_free(head); fmm_free(scan); fmm_free(bad);
        fmm_free(key); fmm_free(key_s); fmm_free(refl);
        return 0;
    }
    int* tab_first = nullptr;
    unsigned long long* tab_key = nullptr;
    FMM_TRY(dalloc(&h->m2l_pt, n));
    FMM_TRY(dalloc(&h->m2l_ps, n));
    FMM_TRY(dalloc(&h->m2l_refl, n));
    FMM_TRY(dalloc(&h->sign_f, 8 * ESTRIDE));
    FMM_TRY(dalloc(&h->sign_d, 8 * ESTRIDE));
    k_refl_signs<<<8, 128, 0, st>>>(h->sign_f, h->sign_d);
    FMM_LAUNCHED();
    FMM_TRY(dalloc(&tab_first, ntab + 1));
    FMM_TRY(dalloc(&tab_key, ntab));
    k_assign_tables<<<(unsigned)((n + 1 + T - 1) / T), T, 0, st>>>(key_s, idx_s, scan, n, pt, ps, refl, h->m2l_pt,
                                                                  h->m2l_ps, h->m2l_refl, tab_first, tab_key);
    FMM_LAUNCHED();
    // tiles for Laplace (64 pairs) and Stokes (16 pairs x 4 expansions)
    const int per_tile = GEMM_COLS / h->ncomp;
    int *cnt = nullptr, *off = nullptr;
    FMM_TRY(dalloc(&cnt, ntab + 1));
    FMM_TRY(dalloc(&off, ntab + 1));
    FMM_CU(cudaMemsetAsync(cnt, 0, sizeof(int) * (ntab + 1), st));
    k_tile_counts<<<(ntab + T - 1) / T, T, 0, st>>>(tab_first, ntab, per_tile, cnt);
    FMM_LAUNCHED();
    FMM_TRY(exclusive_scan(cnt, off, ntab + 1, st));
    int ntiles = 0;
    FMM_CU(cudaMemcpyAsync(&ntiles, off + ntab, sizeof(int), cudaMemcpyDeviceToHost, st));
    FMM_CU(cudaStreamSynchronize(st));
    FMM_TRY(dalloc(&h->m2l_tiles, ntiles));
    k_tile_emit<<<(ntab + T - 1) / T, T, 0, st>>>(tab_first, off, ntab, per_tile, h->m2l_tiles);
    FMM_LAUNCHED();
    // tiles of 128 rows for the tensor-core path (128 pairs Laplace, 32 pairs x 4 Stokes)
    {
        const int per_tc = 128 / (h->ncomp * h->nsys);  // rows of a pair: every component of every copy
        FMM_CU(cudaMemsetAsync(cnt, 0, sizeof(int) * (ntab + 1), st));
        k_tile_counts<<<(ntab + T - 1) / T, T, 0, st>>>(tab_first, ntab, per_tc, cnt);
        FMM_LAUNCHED();
        FMM_TRY(exclusive_scan(cnt, off, ntab + 1, st));
        int ntc = 0;
        FMM_CU(cudaMemcpyAsync(&ntc, off + ntab, sizeof(int), cudaMemcpyDeviceToHost, st));
        FMM_CU(cudaStreamSynchronize(st));
        FMM_TRY(dalloc(&h->m2l_tiles_tc, ntc));
        k_tile_emit<<<(ntab + T - 1) / T, T, 0, st>>>(tab_first, off, ntab, per_tc, h->m2l_tiles_tc);
        FMM_LAUNCHED();
        h->n_tiles_tc = ntc;
    }
    FMM_TRY(dalloc(&h->tab_d, (size_t)ntab * per));
    FMM_TRY(dalloc(&h->tab_f, (size_t)ntab * per));
    k_gen_tables<<<ntab, 256, 0, st>>>(tab_key, pmax, ld, h->tab_d, h->tab_f);
    FMM_LAUNCHED();
    FMM_CU(cudaStreamSynchronize(st));
    h->n_tables = ntab;
    h->n_tiles = ntiles;
    h->tab_ld = ld;
    h->tab_stride = per;
    h->m2l_tables = true;
    fmm_free(pt); fmm_free(ps); fmm_free(idx); fmm_free(idx_s); fmm_free(head); fmm_free(scan); fmm_free(bad);
    fmm_free(key); fmm_free(key_s); fmm_free(refl); fmm_free(tab_first); fmm_free(tab_key); fmm_free(cnt); fmm_free(off);
    return 0;
}

template <typename T, int NC>
int m2l_gemm_t(fmmbem_handle* h, int p) {
    T* L = reinterpret_cast<T*>(h->L);
    const T* M = reinterpret_cast<const T*>(h->M);
    const T* tab = std::is_same<T, float>::value ? reinterpret_cast<const T*>(h->tab_f) : reinterpret_cast<const T*>(h->tab_d);
    const T* sign = std::is_same<T, float>::value ? reinterpret_cast<const T*>(h->sign_f) : reinterpret_cast<const T*>(h->sign_d);
    FMM_CU(cudaMemsetAsync(L, 0, sizeof(T) * h->esys * h->nsys, h->stream));
    const int rpt = rpt_for(p);
    const dim3 g(h->n_tiles, h->nsys), b(GEMM_THREADS);
#define M2L_CASE(R) \
    case R: k_m2l_gemm<T, R, NC><<<g, b, 0, h->stream>>>(p, h->m2l_tiles, h->m2l_pt, h->m2l_ps, h->m2l_refl, sign, tab, h->tab_stride, h->tab_ld, M, L, h->esys); break;
    switch (rpt) {
        M2L_CASE(1) M2L_CASE(2) M2L_CASE(4) M2L_CASE(8) M2L_CASE(12) M2L_CASE(16) M2L_CASE(20)
        default: fmmbem_set_error("no M2L kernel for p=%d", p); return FMMBEM_EINVAL;
    }
#undef M2L_CASE
    FMM_LAUNCHED();
    return 0;
}

int m2l_gemm(fmmbem_handle* h, int p, bool fp64) {
    if (h->ncomp == 1) return fp64 ? m2l_gemm_t<double, 1>(h, p) : m2l_gemm_t<float, 1>(h, p);
    return fp64 ? m2l_gemm_t<double, 4>(h, p) : m2l_gemm_t<float, 4>(h, p);
}

}  // namespace fmmbem
