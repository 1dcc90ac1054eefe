// M2L on the 5th-generation tensor cores (tcgen05, TMEM accumulators, bulk-copy
// operand staging), the high-order path of the mixed-precision mat-vec.
//
// Per tile: D[128 x N] = X[128 x K] * T^T, where the 128 rows are (pair, expansion)
// columns of one translation operator (one M2L geometry, m2l.cu), K = N = 2 ncoef(p)
// real coefficients, X holds the gathered source expansions and T the operator
// (row r = output coefficient). Both operands are K-major in the no-swizzle
// core-matrix layout (8 rows x 16 bytes per core matrix; 128 bytes between core
// matrices along K, 1024 bytes between 8-row groups for 32-wide K chunks).
// FP32 accuracy comes from the 3xTF32 split: x = x_hi + x_lo with x_hi rounded to
// TF32, D = X_hi T_hi + X_hi T_lo + X_lo T_hi (the X_lo T_lo term is below FP32
// rounding). T_hi/T_lo are precomputed; X is split while it is staged.
// The accumulator rows are read back with tcgen05.ld (warp w owns TMEM lanes
// 32w..32w+31) and added to the target expansions with vector atomics.
#include <algorithm>
#include <type_traits>
#include "handle.cuh"

namespace fmmbem {

namespace {

constexpr int TC_ROWS = 128;  // rows per tile (MMA M)
constexpr int TC_KC = 32;     // K per staged chunk
constexpr uint32_t WAIT_LIMIT = 1u << 24;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start, leading-dimension byte offset (between
// core matrices along K), stride byte offset (between 8-row groups), version 1,
// no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((uint64_t)((lbo & 0x3FFFF) >> 4) << 16) |
           ((uint64_t)((sbo & 0x3FFFF) >> 4) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::tf32: D F32, A/B TF32, both K-major.
__device__ __forceinline__ uint32_t idesc_tf32(int m, int n) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

// element (r, k) of a K-major operand chunk with TC_KC columns, in floats
__device__ __forceinline__ int cm_index(int r, int k) {
    return ((r >> 3) * (TC_KC / 4) + (k >> 2)) * 32 + (r & 7) * 4 + (k & 3);
}

__device__ __forceinline__ float tf32_hi(float x) {
    return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
    for (uint32_t it = 0; it < WAIT_LIMIT; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred q;\n\tmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n\tselp.u32 %0, 1, 0, q;\n\t}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// Operator tables for this path: per operator, per 32-wide input chunk c, the hi and
// lo parts of rows [0, rows_max) in the core-matrix layout:
//   tab[g][c][h][cm_index(r, k mod 32)], h = 0 (hi) or 1 (lo).
__global__ void k_tc_tables(const double* Td, int ntab, int nr, int ld, int nch, int rows_max, float* out) {
    const size_t per_tab = (size_t)nch * 2 * rows_max * TC_KC;
    const size_t total = (size_t)ntab * per_tab;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const size_t g = e / per_tab;
        size_t rem = e % per_tab;
        const int c = (int)(rem / (2 * (size_t)rows_max * TC_KC));
        rem %= 2 * (size_t)rows_max * TC_KC;
        const int h = (int)(rem / ((size_t)rows_max * TC_KC));
        const int q = (int)(rem % ((size_t)rows_max * TC_KC));
        // invert cm_index: q = ((r/8)*8 + kq)*32 + (r%8)*4 + k%4
        const int blk = q >> 5, w = q & 31;
        const int r = (blk >> 3) * 8 + (w >> 2), k = c * TC_KC + (blk & 7) * 4 + (w & 3);
        double v = 0.0;
        if (r < nr && k < nr) v = Td[g * (size_t)nr * ld + (size_t)k * ld + r];
        const float hi = (float)v;
        const float hi32 = __uint_as_float((__float_as_uint(hi) + 0x1000u) & 0xFFFFE000u);
        out[e] = h == 0 ? hi32 : (float)(v - (double)hi32);
    }
}

// Persistent: each CTA allocates its TMEM columns and initializes its barriers once,
// then takes tiles blockIdx.x, blockIdx.x + gridDim.x, ...; the barrier parities run
// on across tiles (one load phase and one MMA phase per chunk).
template <int NC>
__global__ void __launch_bounds__(128) k_m2l_tc(int p, const int4* tiles, int ntiles, const int* pt, const int* ps,
                                               const int* prefl, const float* sign, const float* tab,
                                               size_t tab_stride, int rows_max, const float* M, float* L, int* err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    const int R = 2 * ncoef(p);                // outputs = inputs
    const int Np = (R + 15) & ~15;             // MMA N (multiple of 16)
    const int nch = (R + TC_KC - 1) / TC_KC;   // K chunks
    float* sX_hi = reinterpret_cast<float*>(smem);
    float* sX_lo = sX_hi + TC_ROWS * TC_KC;
    float* sT_hi = sX_lo + TC_ROWS * TC_KC;
    float* sT_lo = sT_hi + Np * TC_KC;
    uint64_t* bars = reinterpret_cast<uint64_t*>(sT_lo + Np * TC_KC);
    uint32_t* taddr_slot = reinterpret_cast<uint32_t*>(bars + 2);
    const uint32_t mbar_load = smem_u32(&bars[0]), mbar_mma = smem_u32(&bars[1]);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t tcols = Np <= 32 ? 32 : (Np <= 64 ? 64 : (Np <= 128 ? 128 : (Np <= 256 ? 256 : 512)));

    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar_load), "r"(1));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar_mma), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(taddr_slot)),
                     "r"(tcols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t taddr = *taddr_slot;
    uint32_t ph = 0;  // completed phases of each barrier (both advance once per chunk)
    bool ok = true;
    for (int ti = blockIdx.x; ti < ntiles && ok; ti += gridDim.x) {
    const int4 tile = tiles[ti];
    const int nrows = tile.z * NC;
    // source expansion of each of this thread's gather rows (row = tid/8 + 16 i), read once
    const float* rowsrc[8];
    const float* rowsgn[8];  // reflection signs of the row's pair (see m2l.cu)
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int row = (tid >> 3) + 16 * i;
        rowsrc[i] = nullptr;
        rowsgn[i] = sign + (tid & 7) * 4;
        if (row < nrows) {
            const int pr = tile.y + row / NC;
            rowsrc[i] = M + ((size_t)ps[pr] * NC + row % NC) * ESTRIDE + (tid & 7) * 4;
            rowsgn[i] = sign + prefl[pr] * ESTRIDE + (tid & 7) * 4;
        }
    }
    const float* Tg = tab + (size_t)tile.x * tab_stride;
    const uint32_t chunk_bytes = (uint32_t)Np * TC_KC * 4;
    for (int c = 0; c < nch && ok; ++c) {
        // operator chunk (hi, lo) by bulk copy
        if (tid == 0) {
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar_load), "r"(2 * chunk_bytes)
                         : "memory");
            const float* src = Tg + (size_t)c * 2 * rows_max * TC_KC;
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    smem_u32(sT_hi)),
                "l"(src), "r"(chunk_bytes), "r"(mbar_load)
                : "memory");
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    smem_u32(sT_lo)),
                "l"(src + (size_t)rows_max * TC_KC), "r"(chunk_bytes), "r"(mbar_load)
                : "memory");
        }
        // gathered source expansions, split into TF32 hi/lo (8 independent loads per thread)
        const int kq = (tid & 7) * 4, k = c * TC_KC + kq;
        float4 v[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            v[i] = rowsrc[i] ? *reinterpret_cast<const float4*>(rowsrc[i] + c * TC_KC) : make_float4(0.f, 0.f, 0.f, 0.f);
            const float4 sg = *reinterpret_cast<const float4*>(rowsgn[i] + c * TC_KC);
            v[i].x *= sg.x; v[i].y *= sg.y; v[i].z *= sg.z; v[i].w *= sg.w;
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int row = (tid >> 3) + 16 * i;
            if (k + 0 >= R) v[i].x = 0.f;
            if (k + 1 >= R) v[i].y = 0.f;
            if (k + 2 >= R) v[i].z = 0.f;
            if (k + 3 >= R) v[i].w = 0.f;
            const float4 hi = make_float4(tf32_hi(v[i].x), tf32_hi(v[i].y), tf32_hi(v[i].z), tf32_hi(v[i].w));
            const float4 lo = make_float4(v[i].x - hi.x, v[i].y - hi.y, v[i].z - hi.z, v[i].w - hi.w);
            *reinterpret_cast<float4*>(sX_hi + cm_index(row, kq)) = hi;
            *reinterpret_cast<float4*>(sX_lo + cm_index(row, kq)) = lo;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        if (!mbar_wait(mbar_load, ph & 1)) { atomicExch(err, 1); ok = false; }
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (tid == 0 && ok) {
            const uint32_t xh = smem_u32(sX_hi), xl = smem_u32(sX_lo), th = smem_u32(sT_hi), tl = smem_u32(sT_lo);
            const int n1 = Np <= 256 ? Np : 256;
            const uint32_t id1 = idesc_tf32(TC_ROWS, n1);
            const uint32_t id2 = Np > 256 ? idesc_tf32(TC_ROWS, Np - 256) : 0u;
            for (int ks = 0; ks < TC_KC / 8; ++ks) {
                const uint32_t off = 256u * ks;
                const uint64_t a_hi = smem_desc(xh + off, 128, 1024), a_lo = smem_desc(xl + off, 128, 1024);
                const uint64_t b_hi = smem_desc(th + off, 128, 1024), b_lo = smem_desc(tl + off, 128, 1024);
                const uint32_t first = (c == 0 && ks == 0) ? 0u : 1u;
                mma_tf32(taddr, a_hi, b_hi, id1, first);
                mma_tf32(taddr, a_hi, b_lo, id1, 1u);
                mma_tf32(taddr, a_lo, b_hi, id1, 1u);
                if (Np > 256) {
                    const uint32_t boff = 32u * 1024u;  // rows 256.. start 32 row groups later
                    const uint64_t b2_hi = smem_desc(th + off + boff, 128, 1024), b2_lo = smem_desc(tl + off + boff, 128, 1024);
                    mma_tf32(taddr + 256, a_hi, b2_hi, id2, first);
                    mma_tf32(taddr + 256, a_hi, b2_lo, id2, 1u);
                    mma_tf32(taddr + 256, a_lo, b2_hi, id2, 1u);
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar_mma)
                         : "memory");
        }
        if (ok && !mbar_wait(mbar_mma, ph & 1)) { atomicExch(err, 2); ok = false; }
        ++ph;
        asm volatile("tcgen05.fence::after_thread_sync;");
        __syncthreads();
    }
    if (ok) {
        const int row = 32 * warp + lane;
        float* dst = nullptr;
        const float* sg = sign;
        if (row < nrows) {
            dst = L + ((size_t)pt[tile.y + row / NC] * NC + row % NC) * ESTRIDE;
            sg = sign + prefl[tile.y + row / NC] * ESTRIDE;
        }
        for (int col0 = 0; col0 < R; col0 += 16) {
            uint32_t r[16];
            const uint32_t a = taddr + ((uint32_t)(32 * warp) << 16) + (uint32_t)col0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                : "r"(a));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (dst) {
#pragma unroll
                for (int j = 0; j < 16; j += 4)
                    atomicAdd(reinterpret_cast<float4*>(dst + col0 + j),
                              make_float4(__uint_as_float(r[j]) * sg[col0 + j], __uint_as_float(r[j + 1]) * sg[col0 + j + 1],
                                          __uint_as_float(r[j + 2]) * sg[col0 + j + 2],
                                          __uint_as_float(r[j + 3]) * sg[col0 + j + 3]));
            }
        }
    }
    // the epilogue's TMEM reads finish before the next tile's MMAs overwrite the accumulator
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(tcols));
}

}  // namespace

size_t m2l_tc_smem(int p) {
    const int R = 2 * ncoef(p);
    const int Np = (R + 15) & ~15;
    return (size_t)(2 * TC_ROWS * TC_KC + 2 * Np * TC_KC) * sizeof(float) + 64;
}

int build_m2l_tc(fmmbem_handle* h) {
    if (!h->m2l_tables) return 0;
    const int pmax = h->opts.p_max;
    const int nr = 2 * ncoef(pmax);
    const int rows_max = (nr + 15) & ~15;
    const int nch = (nr + TC_KC - 1) / TC_KC;
    const size_t per_tab = (size_t)nch * 2 * rows_max * TC_KC;
    FMM_CU(cudaMalloc((void**)&h->tab_tc, sizeof(float) * per_tab * (size_t)h->n_tables));
    k_tc_tables<<<2048, 256, 0, h->stream>>>(h->tab_d, h->n_tables, nr, h->tab_ld, nch, rows_max, h->tab_tc);
    FMM_LAUNCHED();
    h->tc_stride = per_tab;
    h->tc_rows_max = rows_max;
    FMM_CU(cudaMalloc((void**)&h->tc_err, sizeof(int)));
    FMM_CU(cudaMemsetAsync(h->tc_err, 0, sizeof(int), h->stream));
    const size_t smax = m2l_tc_smem(pmax);
    FMM_CU(cudaFuncSetAttribute(k_m2l_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smax));
    FMM_CU(cudaFuncSetAttribute(k_m2l_tc<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smax));
    int dev = 0;
    FMM_CU(cudaGetDevice(&dev));
    FMM_CU(cudaDeviceGetAttribute(&h->n_sm, cudaDevAttrMultiProcessorCount, dev));
    h->m2l_tc_ready = true;
    return 0;
}

int m2l_tc(fmmbem_handle* h, int p) {
    float* L = reinterpret_cast<float*>(h->L);
    const float* M = reinterpret_cast<const float*>(h->M);
    FMM_CU(cudaMemsetAsync(L, 0, sizeof(float) * (size_t)h->n_cells * h->ncomp * ESTRIDE, h->stream));
    const size_t sm = m2l_tc_smem(p);
    const int R = 2 * ncoef(p), Np = (R + 15) & ~15;
    const int tcols = Np <= 32 ? 32 : (Np <= 64 ? 64 : (Np <= 128 ? 128 : (Np <= 256 ? 256 : 512)));
    const int per_sm = std::max(1, std::min({4, (int)((220u << 10) / sm), 512 / tcols}));
    const int grid = std::min(h->n_tiles_tc, h->n_sm * per_sm);
    if (h->ncomp == 1)
        k_m2l_tc<1><<<grid, 128, sm, h->stream>>>(p, h->m2l_tiles_tc, h->n_tiles_tc, h->m2l_pt, h->m2l_ps, h->m2l_refl, h->sign_f, h->tab_tc,
                                                           h->tc_stride, h->tc_rows_max, M, L, h->tc_err);
    else
        k_m2l_tc<4><<<grid, 128, sm, h->stream>>>(p, h->m2l_tiles_tc, h->n_tiles_tc, h->m2l_pt, h->m2l_ps, h->m2l_refl, h->sign_f, h->tab_tc,
                                                           h->tc_stride, h->tc_rows_max, M, L, h->tc_err);
    FMM_LAUNCHED();
    return 0;
}

}  // namespace fmmbem
