// M2L on the 5th-generation tensor cores (tcgen05, TMEM accumulators, bulk-copy
// operand staging), the high-order path of the mixed-precision mat-vec.
//
// Per tile: D[128 x N] = X[128 x K] * T^T, where the 128 rows are (pair, expansion)
// columns of one translation operator (one M2L geometry, m2l.cu), K = N = 2 ncoef(p)
// real coefficients, X holds the gathered source expansions and T the operator
// (row r = output coefficient). Both operands are K-major in the no-swizzle
// core-matrix layout (8 rows x 16 bytes per core matrix; 128 bytes between core
// matrices along K, 32 KC bytes between 8-row groups of a KC-wide K chunk).
// FP32 accuracy comes from the 3xTF32 split: x = x_hi + x_lo with x_hi rounded to
// TF32, D = X_hi T_hi + X_hi T_lo + X_lo T_hi (the X_lo T_lo term is below FP32
// rounding). T_hi/T_lo are precomputed; X is split while it is staged.
// The accumulator rows are read back with tcgen05.ld (warps w and w + 4 own TMEM lanes
// 32 (w mod 4) .. +31 and split the columns), transposed through padded shared memory
// and added to the target expansions with row-contiguous float4 atomics.
#include <algorithm>
#include <type_traits>
#include <vector>
#include "handle.cuh"
#include "harmonics.cuh"
#include "tc_ptx.cuh"

namespace fmmbem {

namespace {

constexpr int TC_ROWS = 128;  // rows per tile (MMA M)
// K per staged chunk (a kernel template parameter): 16 for every handle. Against 32-wide
// chunks a lone M2L at p <= 12 is a few percent slower, but p = 16 keeps three stages in flight
// instead of one, the split tree levels get more K ranges, and at low p the CTA's smaller
// footprint leaves room for a near-field block beside it: the concurrent solve is faster.
constexpr int TC_KC = 16;
template <int KC> struct Kc {
    static_assert(KC % 16 == 0, "a gather lane covers whole k-quads of 16-wide steps");
    static constexpr int KQ = KC / 4;           // k-quads (core matrices along K) per chunk
    static constexpr int E = KC / 16;           // k-quads per gather lane and item
    static constexpr uint32_t SBO = 32u * KC;   // bytes between 8-row groups of an operand chunk
};
constexpr uint32_t WAIT_LIMIT = 1u << 24;

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) { return mbar_wait_bounded(mbar, parity, WAIT_LIMIT); }

// element (r, k) of a K-major operand chunk with KC columns, in floats
template <int KC> __device__ __forceinline__ int cm_index(int r, int k) {
    return ((r >> 3) * (KC / 4) + (k >> 2)) * 32 + (r & 7) * 4 + (k & 3);
}

__device__ __forceinline__ float tf32_hi(float x) {
    return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

// Operator tables for this path: per operator, per KC-wide input chunk c, the hi and
// lo parts of rows [0, rows_max) in the core-matrix layout:
//   tab[g][c][h][cm_index<KC>(r, k mod KC)], h = 0 (hi) or 1 (lo).
template <int KC>
__global__ void k_tc_tables(const double* Td, int ntab, int nr, int ld, int nch, int rows_max, float* out) {
    const size_t per_tab = (size_t)nch * 2 * rows_max * KC;
    const size_t total = (size_t)ntab * per_tab;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const size_t g = e / per_tab;
        size_t rem = e % per_tab;
        const int c = (int)(rem / (2 * (size_t)rows_max * KC));
        rem %= 2 * (size_t)rows_max * KC;
        const int h = (int)(rem / ((size_t)rows_max * KC));
        const int q = (int)(rem % ((size_t)rows_max * KC));
        // invert cm_index: q = ((r/8)*8 + kq)*32 + (r%8)*4 + k%4
        const int blk = q >> 5, w = q & 31;
        const int r = (blk / Kc<KC>::KQ) * 8 + (w >> 2), k = c * KC + (blk % Kc<KC>::KQ) * 4 + (w & 3);
        double v = 0.0;
        if (r < nr && k < nr) v = Td[g * (size_t)nr * ld + (size_t)k * ld + r];
        const float hi = (float)v;
        const float hi32 = __uint_as_float((__float_as_uint(hi) + 0x1000u) & 0xFFFFE000u);
        out[e] = h == 0 ? hi32 : (float)(v - (double)hi32);
    }
}

// Persistent and warp-specialized: one CTA per SM takes work units blockIdx.x, blockIdx.x +
// gridDim.x, ... (a unit is a tile, or with split-K a range of its K chunks); its work items
// are (unit, K chunk) pairs in that order. Roles:
//   warp 0      : bulk-copies the operator chunk of item i into smem stage i % NST;
//   warp 1      : issues the MMAs of item i into TMEM accumulator (unit) % NB and commits;
//   warps 2-9   : gather producers; each stages 16 rows of every item (rows of the
//                 tile's pairs, reflection signs applied, split into TF32 hi/lo),
//                 keeping the loads of the next item in flight while storing this one;
//   warps 10-17 : two epilogue groups of four (one per TMEM lane quadrant); group g
//                 drains the accumulators of units j = g mod 2 (all units by group 0
//                 when there is one accumulator) through a padded smem transpose into
//                 row-contiguous float4 atomics.
// mbarriers: full[s] (8 producer arrivals + the copy's transaction bytes), empty[s]
// (MMA commit), acc_full[b] (commit after a unit's last chunk), acc_empty[b] (the
// four warps of the draining group). Use k of a barrier completes phase k; a role
// waits on phase k only before the use k + 1 that it gates can begin, so parities
// never alias. Every wait is bounded: on timeout the CTA records an error code,
// raises an abort flag that the other roles' waits observe, drains what it
// issued (bounded again), frees TMEM and returns.
constexpr int TC_WARPS = 18;
constexpr int TC_THREADS = 32 * TC_WARPS;
constexpr int TC_PROD0 = 2, TC_NPROD = 8, TC_EPI0 = 10;
constexpr int EPI_LD = 33;  // padded row length of the epilogue transpose buffer
constexpr int TC_SMEM_BUDGET = 222 * 1024;
constexpr int TC_SIGN_TAB = 16 * 8;  // k-quad entries: 512 reals cover 2 ncoef(P_MAX) <= 320

// Stages, accumulators and TMEM columns of one order. With atm (A in TMEM) a stage's gathered
// rows (TF32 hi and lo, 2 kc columns) live in the last nst * 2 kc TMEM columns and shared
// memory holds only the operator chunks; the accumulators take what is left.
struct TcLayout {
    int nst, nb, np, kc, buf_cols;
    bool atm;
    __host__ __device__ int a_floats() const { return atm ? 0 : 2 * TC_ROWS * kc; }
    __host__ __device__ int stage_floats() const { return a_floats() + 2 * np * kc; }
    __host__ __device__ int epi_floats() const { return 8 * 32 * EPI_LD; }
    __host__ __device__ int a_col0() const { return 512 - nst * 2 * kc; }  // first A column (atm)
    __host__ __device__ size_t bytes() const {
        return (size_t)(nst * stage_floats() + epi_floats()) * sizeof(float) + 16 * 8 + 64 + 2 * TC_SIGN_TAB * 4;
    }
};

__host__ __device__ inline TcLayout tc_layout(int p, int kc, bool atm) {
    TcLayout t;
    t.kc = kc;
    t.atm = atm;
    const int R = 2 * ncoef(p);
    t.np = (R + 15) & ~15;
    t.nb = t.np <= 128 ? 4 : (t.np <= 256 ? 2 : 1);
    t.buf_cols = 512 / t.nb;
    t.nst = 1;
    for (int n = 4; n >= 1; --n) {
        t.nst = n;
        if (t.bytes() <= (size_t)TC_SMEM_BUDGET) break;
    }
    if (atm) {
        // accumulators of 32-column multiples beside the A stages; fewer stages (down to two)
        // when that keeps a second accumulator. The count stays 1, 2 or 4: with two epilogue
        // groups, group g drains units j = g mod 2, and an even count keeps each accumulator
        // with one group (whose waits then follow its phases in order).
        t.buf_cols = (t.np + 31) & ~31;
        auto nb_of = [&](int nst) { return (512 - nst * 2 * kc) / t.buf_cols; };
        while (t.nst > 2 && nb_of(t.nst) < 2 && t.np <= 256) --t.nst;
        const int nb = nb_of(t.nst);
        t.nb = nb >= 4 ? 4 : (nb >= 2 ? 2 : nb);
    }
    return t;
}

// The TMEM-operand variant where it keeps as many accumulators as the shared-memory one (up
// to two) and at least three stages where that one has them. Measured alone, p = 12: 277
// against 303 us; p = 16: 747 against 806 us; p = 13, where two accumulators leave two
// stages: 411 against 369 us (p = 13 and 14 keep the shared-memory variant).
__host__ __device__ inline bool tc_atm_at(int p, int kc) {
    const TcLayout a = tc_layout(p, kc, true), s = tc_layout(p, kc, false);
    return a.nb >= 1 && a.nb >= (s.nb < 2 ? s.nb : 2) && a.nst >= (s.nst < 3 ? s.nst : 3);
}

// Reflection sign bits of a float4 of real coefficients (re_a, im_a, re_b, im_b),
// coefficients a and a + 1: bit e set = element e changes sign under reflection q
// (bit 0: x, bit 1: y, bit 2: z). z -> (-1)^{n+m}; y -> conj; x -> (-1)^m conj.
__device__ __forceinline__ uint32_t coef_nm_bits(int c) {
    int n = (int)((sqrtf(8.f * c + 1.f) - 1.f) * 0.5f);
    if ((n + 1) * (n + 2) / 2 <= c) ++n;
    if (n * (n + 1) / 2 > c) --n;
    const int m = c - n * (n + 1) / 2;
    return (uint32_t)(((n + m) & 1) | ((m & 1) << 1));  // bit 0: z parity, bit 1: x parity
}
__device__ __forceinline__ uint32_t sign_bits(uint32_t nm_a, uint32_t nm_b, int q) {
    const uint32_t z = (q >> 2) & 1, y = (q >> 1) & 1, x = q & 1;
    const uint32_t ra = (z & nm_a) ^ (x & (nm_a >> 1)), rb = (z & nm_b) ^ (x & (nm_b >> 1));
    const uint32_t ia = ra ^ y ^ x, ib = rb ^ y ^ x;
    return ra | (ia << 1) | (rb << 2) | (ib << 3);
}
__device__ __forceinline__ float4 apply_zero(float4 v, uint32_t z) {
    if (z & 1u) v.x = 0.f;
    if (z & 2u) v.y = 0.f;
    if (z & 4u) v.z = 0.f;
    if (z & 8u) v.w = 0.f;
    return v;
}
__device__ __forceinline__ float4 apply_signs(float4 v, uint32_t b) {
    v.x = __uint_as_float(__float_as_uint(v.x) ^ ((b & 1u) << 31));
    v.y = __uint_as_float(__float_as_uint(v.y) ^ (((b >> 1) & 1u) << 31));
    v.z = __uint_as_float(__float_as_uint(v.z) ^ (((b >> 2) & 1u) << 31));
    v.w = __uint_as_float(__float_as_uint(v.w) ^ (((b >> 3) & 1u) << 31));
    return v;
}

// Bounded wait that also gives up once another role has raised the abort flag.
__device__ __forceinline__ bool mbar_wait_ab(uint32_t mbar, uint32_t parity, volatile int* abort_flag) {
    for (uint32_t it = 0; it < WAIT_LIMIT; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred q;\n\tmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n\tselp.u32 %0, 1, 0, q;\n\t}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
        if ((it & 255) == 255 && *abort_flag) return false;
    }
    return false;
}

__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
}

// rinfo[t * 128 + r] = (row offset of pair row r of tile t in the expansion array) * 8 + reflection,
// -1 past the tile's rows; one table for the sources (gather) and one for the targets (epilogue).
template <int KC, bool SPLIT, bool ATM>
__global__ void __launch_bounds__(TC_THREADS, 1) k_m2l_tc(int p, int prods, const int4* tiles, int ntiles, int ksplit_arg,
                                                         const int* src_info, const int* dst_info, const float* tab,
                                                         size_t tab_stride, int rows_max, const float* M, float* L,
                                                         int* err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    const TcLayout lay = tc_layout(p, KC, ATM);
    const int R = 2 * ncoef(p);
    const int R8 = (R + 7) & ~7;  // K extent the MMAs read: k-steps of 8 that start below R
    const int Np = lay.np, NST = lay.nst, NB = lay.nb;
    const int nch = (R + KC - 1) / KC;
    const uint32_t chunk_bytes = (uint32_t)Np * KC * 4;
    float* stage0 = reinterpret_cast<float*>(smem);
    const int sf = lay.stage_floats();
    float* epi = stage0 + NST * sf;
    uint64_t* bar = reinterpret_cast<uint64_t*>(epi + lay.epi_floats());  // full[4], empty[4], acc_full[4], acc_empty[4]
    uint32_t* taddr_slot = reinterpret_cast<uint32_t*>(bar + 16);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(taddr_slot + 1);
    // sgn_tab[k / 4]: bits 4q..4q+3 = sign flips of the 4 reals at k = 4 (k / 4) .. under
    // reflection q; zm_tab: bit e set when k + e >= R (coefficient of degree > p, zeroed)
    uint32_t* sgn_tab = reinterpret_cast<uint32_t*>(smem) + (lay.bytes() - 2 * TC_SIGN_TAB * 4) / 4;
    uint32_t* zm_tab = sgn_tab + TC_SIGN_TAB;
    auto full = [&](int st) { return smem_u32(&bar[st]); };
    auto empty = [&](int st) { return smem_u32(&bar[4 + st]); };
    auto acc_full = [&](int b) { return smem_u32(&bar[8 + b]); };
    auto acc_empty = [&](int b) { return smem_u32(&bar[12 + b]); };
    auto xh = [&](int st) { return stage0 + st * sf; };
    auto xl = [&](int st) { return stage0 + st * sf + TC_ROWS * KC; };
    auto th = [&](int st) { return stage0 + st * sf + lay.a_floats(); };
    auto tl = [&](int st) { return stage0 + st * sf + lay.a_floats() + Np * KC; };

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int e = tid; e < TC_SIGN_TAB; e += blockDim.x) {
        const int k0 = 4 * e;  // entry e holds the k-quad of reals k0 .. k0 + 3
        const uint32_t nm_a = coef_nm_bits(k0 >> 1), nm_b = coef_nm_bits((k0 >> 1) + 1);
        uint32_t sg = 0;
        for (int q = 0; q < 8; ++q) sg |= sign_bits(nm_a, nm_b, q) << (4 * q);
        sgn_tab[e] = sg;
        zm_tab[e] = (k0 >= R ? 1u : 0u) | (k0 + 1 >= R ? 2u : 0u) | (k0 + 2 >= R ? 4u : 0u) | (k0 + 3 >= R ? 8u : 0u);
    }
    if (tid == 0) {
        for (int st = 0; st < 4; ++st) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(full(st)), "r"(TC_NPROD + 1));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(empty(st)), "r"(1));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(acc_full(st)), "r"(1));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(acc_empty(st)), "r"(4));
        }
        asm volatile("fence.mbarrier_init.release.cluster;");
        *abort_flag = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(taddr_slot)),
                     "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t taddr = *taddr_slot;
    // everything above (barriers, sign tables, TMEM) may overlap the previous kernel of the
    // stream; the expansions it writes are read and accumulated only after it has completed
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const uint32_t buf_cols = (uint32_t)lay.buf_cols;
    // Work units are (tile, range of K chunks): the nch chunks of a tile are cut into ksplit
    // ranges (split-K for launches with fewer tiles than SMs; the epilogue adds each range's
    // partial product like any other). Unit u covers tile u / ksplit, range u mod ksplit; the
    // CTA takes units blockIdx.x, blockIdx.x + gridDim.x, ... and its items are (unit, chunk).
    const int ksplit = SPLIT ? ksplit_arg : 1;  // the unsplit kernel has none of the unit arithmetic
    const int nunits = ntiles * ksplit;
    const int my_units = (int)blockIdx.x < nunits ? (nunits - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    auto unit_of = [&](int j) { return (int)blockIdx.x + j * (int)gridDim.x; };
    // (the divisions only run with split-K, and only when a role moves to its next unit)
    auto tile_of = [&](int j) { return ksplit == 1 ? unit_of(j) : unit_of(j) / ksplit; };
    auto c_begin = [&](int j) { return ksplit == 1 ? 0 : (unit_of(j) % ksplit) * nch / ksplit; };
    auto c_end = [&](int j) { return ksplit == 1 ? nch : (unit_of(j) % ksplit + 1) * nch / ksplit; };
    int n_items = ksplit == 1 ? my_units * nch : 0;
    if (ksplit > 1)
        for (int j = 0; j < my_units; ++j) n_items += c_end(j) - c_begin(j);
    auto fail = [&](int code) {
        atomicExch(err, code);
        *abort_flag = 1;
    };
    int issued_tma = 0, issued_mma = 0;  // items issued by the copy and MMA roles (for the final drain)

    if (warp == 0) {
        // ---------------- operator copies
        if (lane == 0) {
            // the tile record of the next unit is loaded one unit ahead, and the next unit's
            // operator chunks are prefetched into L2 when this unit starts, so neither the
            // record load nor a DRAM miss sits between a free stage and its refill
            const uint32_t bytes = prods == 3 ? 2 * chunk_bytes : chunk_bytes;
            int4 tile = my_units > 0 ? tiles[tile_of(0)] : make_int4(0, 0, 0, 0);
            int4 next_tile = my_units > 1 ? tiles[tile_of(1)] : tile;
            int4 next2_tile = my_units > 2 ? tiles[tile_of(2)] : next_tile;
            int c0 = c_begin(0), c1 = c_end(0), c = c0, st = 0, k = 0, j = 0;
            for (int i = 0; i < n_items; ++i) {
                if (c == c0 && j + 1 < my_units) {
                    const float* nt = tab + (size_t)next_tile.x * tab_stride;
                    for (int cc = c_begin(j + 1); cc < c_end(j + 1); ++cc) {
                        const float* q = nt + (size_t)cc * 2 * rows_max * KC;
                        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(q), "r"(chunk_bytes) : "memory");
                        if (prods == 3)
                            asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(q + (size_t)rows_max * KC),
                                         "r"(chunk_bytes)
                                         : "memory");
                    }
                }
                if (k > 0 && !mbar_wait_ab(empty(st), (uint32_t)((k - 1) & 1), abort_flag)) { fail(1); break; }
                if (*abort_flag) break;
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(full(st)), "r"(bytes) : "memory");
                const float* src = tab + (size_t)tile.x * tab_stride + (size_t)c * 2 * rows_max * KC;
                asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                                 smem_u32(th(st))),
                             "l"(src), "r"(chunk_bytes), "r"(full(st))
                             : "memory");
                if (prods == 3)
                    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                                     smem_u32(tl(st))),
                                 "l"(src + (size_t)rows_max * KC), "r"(chunk_bytes), "r"(full(st))
                                 : "memory");
                issued_tma = i + 1;
                if (++st == NST) { st = 0; ++k; }
                if (++c == c1) {
                    ++j;
                    c0 = c_begin(j);
                    c1 = c_end(j);
                    c = c0;
                    tile = next_tile;
                    next_tile = next2_tile;
                    if (j + 2 < my_units) next2_tile = tiles[tile_of(j + 2)];
                }
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issue
        if (lane == 0) {
            const int n1 = Np <= 256 ? Np : 256;
            const uint32_t id1 = idesc_tf32(TC_ROWS, n1);
            const uint32_t id2 = Np > 256 ? idesc_tf32(TC_ROWS, Np - 256) : 0u;
            // stage, stage use, unit, chunk and the unit's chunk range, accumulator, accumulator use
            int st = 0, k = 0, j = 0, c0 = c_begin(0), c1 = c_end(0), c = c0, b = 0, u = 0;
            for (int i = 0; i < n_items; ++i) {
                if (c == c0 && u > 0 && !mbar_wait_ab(acc_empty(b), (uint32_t)((u - 1) & 1), abort_flag)) { fail(3); break; }
                if (!mbar_wait_ab(full(st), (uint32_t)(k & 1), abort_flag)) { fail(4); break; }
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t acc = taddr + (uint32_t)b * buf_cols;
                const uint32_t ah = smem_u32(xh(st)), al = smem_u32(xl(st)), bh = smem_u32(th(st)), bl = smem_u32(tl(st));
                const uint32_t at = taddr + (uint32_t)(lay.a_col0() + st * 2 * KC);  // the stage's A columns (ATM)
                // D (+)= A B^T with k-step ks of A's hi or lo part, from TMEM or shared memory
                auto mma_a = [&](uint32_t d, bool lo, int ks, uint64_t bdesc, uint32_t id, uint32_t accum) {
                    if constexpr (ATM)
                        mma_tf32_ts(d, at + (lo ? (uint32_t)KC : 0u) + 8u * ks, bdesc, id, accum);
                    else
                        mma_tf32(d, smem_desc((lo ? al : ah) + 256u * ks, 128, Kc<KC>::SBO), bdesc, id, accum);
                };
                for (int ks = 0; ks < KC / 8; ++ks) {
                    if (c * KC + 8 * ks >= R) break;  // the rest of the chunk lies past degree p
                    const uint32_t off = 256u * ks;
                    const uint64_t b_hi = smem_desc(bh + off, 128, Kc<KC>::SBO);
                    const uint32_t first = (c == c0 && ks == 0) ? 0u : 1u;
                    mma_a(acc, false, ks, b_hi, id1, first);
                    if (prods == 3) {
                        mma_a(acc, false, ks, smem_desc(bl + off, 128, Kc<KC>::SBO), id1, 1u);
                        mma_a(acc, true, ks, b_hi, id1, 1u);
                    }
                    if (Np > 256) {
                        const uint32_t boff = 32u * Kc<KC>::SBO;  // operator rows 256.. start 32 row groups later
                        const uint64_t b2_hi = smem_desc(bh + off + boff, 128, Kc<KC>::SBO);
                        mma_a(acc + 256, false, ks, b2_hi, id2, first);
                        if (prods == 3) {
                            mma_a(acc + 256, false, ks, smem_desc(bl + off + boff, 128, Kc<KC>::SBO), id2, 1u);
                            mma_a(acc + 256, true, ks, b2_hi, id2, 1u);
                        }
                    }
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(empty(st))
                             : "memory");
                if (c == c1 - 1)
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                     acc_full(b))
                                 : "memory");
                issued_mma = i + 1;
                if (++st == NST) { st = 0; ++k; }
                if (++c == c1) {
                    ++j;
                    c0 = c_begin(j);
                    c1 = c_end(j);
                    c = c0;
                    if (++b == NB) { b = 0; ++u; }
                }
            }
        }
    } else if (warp < TC_EPI0) {
        // ---------------- gather producers: rows 16 pw + 8 h + (lane & 7), k-quads (lane >> 3) + 4 e.
        // Software pipeline over three register slots (the loop is unrolled by three so the
        // slot indices are constants): while item i is stored from slot i % 3, the inputs of
        // item i + 2 are issued into slot (i + 2) % 3. A row table belongs to a unit's tile, not
        // to an item: each lane keeps its two rows' entries for the units j .. j + 3 in registers
        // (ti[0] = unit j of item i; item i + 2 lies at most two units ahead) and loads those of
        // unit j + 3 when item i starts unit j, a whole unit before the gathers that use them.
        // Item counters (unit, chunk, stage, phase) advance incrementally; signs and the order-p
        // mask come from the CTA's tables.
      if constexpr (ATM) {
        // ---------------- gather producers, A operand in TMEM: warp w may write TMEM lanes
        // 32 (w mod 4) .. + 31 only, so lane l of warp w gathers tile row 32 (w mod 4) + l, and
        // the two warps of a quadrant take the chunk's columns 0-7 and 8-15. Each item stores
        // the row's 8 TF32 hi values and 8 lo values with one tcgen05.st each. The software
        // pipeline, row tables and counters are those of the shared-memory variant below.
        const int pw = warp - TC_PROD0, qd = warp & 3, half = pw >> 2;
        const int row = 32 * qd + lane;
        const uint32_t ta_row = taddr + ((uint32_t)(32 * qd) << 16) + (uint32_t)(lay.a_col0() + 8 * half);
        float4 d[3][2];
        int ti[4] = {-1, -1, -1, -1};
        struct Ctr {
            int j, c, c1;
        };
        auto adv = [&](Ctr& t) {
            if (++t.c < t.c1) return false;
            ++t.j;
            t.c = c_begin(t.j);
            t.c1 = c_end(t.j);
            return true;
        };
        auto load_info = [&](int j) { return j < my_units ? src_info[(size_t)tile_of(j) * TC_ROWS + row] : -1; };
        // one 32-byte load per lane and item: rows start at multiples of 320 floats and k at
        // multiples of 8, and the 8 reals stay inside the row's 320 (the ones past degree p
        // are zeroed with the sign table's mask)
        auto load_data = [&](const Ctr& t, int dj, float4 (&v)[2]) {
            const int info = dj == 0 ? ti[0] : (dj == 1 ? ti[1] : ti[2]);
            const int k = t.c * KC + 8 * half;
            if (t.j < my_units && info >= 0 && k < R) {
                asm volatile("ld.global.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                             : "=f"(v[0].x), "=f"(v[0].y), "=f"(v[0].z), "=f"(v[0].w), "=f"(v[1].x), "=f"(v[1].y),
                               "=f"(v[1].z), "=f"(v[1].w)
                             : "l"(M + (size_t)(info >> 3) + k));
            } else {
                v[0] = make_float4(0.f, 0.f, 0.f, 0.f);
                v[1] = v[0];
            }
        };
#pragma unroll
        for (int q = 0; q < 4; ++q) ti[q] = load_info(q);
        Ctr ci{0, c_begin(0), c_end(0)};
        Ctr c2 = ci;
        {
            Ctr c1 = ci;
            adv(c1);
            load_data(ci, 0, d[0]);
            load_data(c1, c1.j, d[1]);
            c2 = c1;
            adv(c2);
        }
        int st = 0, ph = 0;
        bool stop = false;
        for (int base = 0; base < n_items && !stop; base += 3) {
#pragma unroll
            for (int u = 0; u < 3; ++u) {
                const int i = base + u;
                if (i >= n_items || stop) break;
                const int sa = u, sc = (u + 2) % 3;
                load_data(c2, c2.j - ci.j, d[sc]);
                const bool okw = ph == 0 || mbar_wait_ab(empty(st), (uint32_t)((ph - 1) & 1), abort_flag);
                if (!__all_sync(0xffffffffu, okw)) {
                    if (lane == 0) fail(2);
                    stop = true;
                    break;
                }
                if (__any_sync(0xffffffffu, *abort_flag != 0)) { stop = true; break; }
                uint32_t hv[8], lv[8];
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int te = ((ci.c * KC + 8 * half) >> 2) + e;
                    const uint32_t sg = sgn_tab[te], zm = zm_tab[te];
                    const float4 x = apply_zero(apply_signs(d[sa][e], (sg >> (4 * (ti[0] & 7))) & 15u), zm);
                    const float4 hi = make_float4(tf32_hi(x.x), tf32_hi(x.y), tf32_hi(x.z), tf32_hi(x.w));
                    hv[4 * e + 0] = __float_as_uint(hi.x);
                    hv[4 * e + 1] = __float_as_uint(hi.y);
                    hv[4 * e + 2] = __float_as_uint(hi.z);
                    hv[4 * e + 3] = __float_as_uint(hi.w);
                    lv[4 * e + 0] = __float_as_uint(x.x - hi.x);
                    lv[4 * e + 1] = __float_as_uint(x.y - hi.y);
                    lv[4 * e + 2] = __float_as_uint(x.z - hi.z);
                    lv[4 * e + 3] = __float_as_uint(x.w - hi.w);
                }
                const uint32_t ta = ta_row + (uint32_t)(st * 2 * KC);
                tmem_st8(ta, hv);
                if (prods == 3) tmem_st8(ta + KC, lv);
                asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                asm volatile("tcgen05.fence::before_thread_sync;");
                __syncwarp();
                if (lane == 0) mbar_arrive(full(st));
                const bool new_unit = adv(ci);
                adv(c2);
                if (new_unit) {
                    ti[0] = ti[1];
                    ti[1] = ti[2];
                    ti[2] = ti[3];
                    ti[3] = load_info(ci.j + 3);
                }
                if (++st == NST) { st = 0; ++ph; }
            }
        }
      } else {
        const int pw = warp - TC_PROD0, r7 = lane & 7, kq0 = lane >> 3;
        const int row0 = 16 * pw + r7;
        float4 d[3][2][Kc<KC>::E];
        int ti[4][2];
        struct Ctr {
            int j, c, c1;  // unit, chunk, end of the unit's chunk range
        };
        // next item; true when it starts a new unit
        auto adv = [&](Ctr& t) {
            if (++t.c < t.c1) return false;
            ++t.j;
            t.c = c_begin(t.j);
            t.c1 = c_end(t.j);
            return true;
        };
        auto load_info = [&](int j, int (&info)[2]) {
#pragma unroll
            for (int h = 0; h < 2; ++h)
                info[h] = j < my_units ? src_info[(size_t)tile_of(j) * TC_ROWS + row0 + 8 * h] : -1;
        };
        // the row entries of tile t.j, which lies dj = t.j - (tile of item i) in {0, 1, 2} tiles ahead
        auto load_data = [&](const Ctr& t, int dj, float4 (&v)[2][Kc<KC>::E]) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int info = dj == 0 ? ti[0][h] : (dj == 1 ? ti[1][h] : ti[2][h]);
#pragma unroll
                for (int e = 0; e < Kc<KC>::E; ++e) {
                    const int k = t.c * KC + 4 * (kq0 + 4 * e);
                    v[h][e] = (t.j < my_units && info >= 0 && k < R)
                                  ? *reinterpret_cast<const float4*>(M + (size_t)(info >> 3) + k)
                                  : make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
        };
#pragma unroll
        for (int q = 0; q < 4; ++q) load_info(q, ti[q]);
        Ctr ci{0, c_begin(0), c_end(0)};  // item i
        Ctr c2 = ci;            // item i + 2
        {
            Ctr c1 = ci;
            adv(c1);
            load_data(ci, 0, d[0]);
            load_data(c1, c1.j, d[1]);
            c2 = c1;
            adv(c2);
        }
        int st = 0, ph = 0;  // stage of item i and the number of earlier uses of that stage
        bool stop = false;
        for (int base = 0; base < n_items && !stop; base += 3) {
#pragma unroll
            for (int u = 0; u < 3; ++u) {
                const int i = base + u;
                if (i >= n_items || stop) break;
                const int sa = u, sc = (u + 2) % 3;
                load_data(c2, c2.j - ci.j, d[sc]);
                // warp-uniform decisions: the warp's lanes take every branch together
                const bool okw = ph == 0 || mbar_wait_ab(empty(st), (uint32_t)((ph - 1) & 1), abort_flag);
                if (!__all_sync(0xffffffffu, okw)) {
                    if (lane == 0) fail(2);
                    stop = true;
                    break;
                }
                if (__any_sync(0xffffffffu, *abort_flag != 0)) { stop = true; break; }
                float* xh_s = xh(st);
                float* xl_s = xl(st);
#pragma unroll
                for (int e = 0; e < Kc<KC>::E; ++e) {
                    const int kq = 4 * (kq0 + 4 * e);
                    if (ci.c * KC + kq >= R8) continue;  // past the last 8-wide k-step any MMA reads
                    const int te = ci.c * Kc<KC>::KQ + kq0 + 4 * e;
                    const uint32_t sg = sgn_tab[te], zm = zm_tab[te];
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int row = row0 + 8 * h;
                        const float4 x = apply_zero(apply_signs(d[sa][h][e], (sg >> (4 * (ti[0][h] & 7))) & 15u), zm);
                        const float4 hi = make_float4(tf32_hi(x.x), tf32_hi(x.y), tf32_hi(x.z), tf32_hi(x.w));
                        *reinterpret_cast<float4*>(xh_s + cm_index<KC>(row, kq)) = hi;
                        if (prods == 3)
                            *reinterpret_cast<float4*>(xl_s + cm_index<KC>(row, kq)) =
                                make_float4(x.x - hi.x, x.y - hi.y, x.z - hi.z, x.w - hi.w);
                    }
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(full(st));
                const bool new_unit = adv(ci);
                adv(c2);
                if (new_unit) {  // item i + 1 starts unit ci.j: shift the row tables, fetch unit ci.j + 3
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        ti[0][h] = ti[1][h];
                        ti[1][h] = ti[2][h];
                        ti[2][h] = ti[3][h];
                    }
                    load_info(ci.j + 3, ti[3]);
                }
                if (++st == NST) { st = 0; ++ph; }
            }
        }
      }
    } else {
        // ---------------- epilogue groups
        // with one accumulator a single group drains every tile, so that each group waits
        // on the phases of its buffers in order
        const int EG = NB >= 2 ? 2 : 1;
        const int eg = (warp - TC_EPI0) >> 2;  // group 0 or 1
        const int quad = warp & 3;             // TMEM lane quadrant of this warp
        float* E = epi + (warp - TC_EPI0) * 32 * EPI_LD;
        // destination row table of this warp's 32 accumulator rows, one per lane (shuffled per
        // pass); the next tile's entries are fetched before this tile's accumulator wait
        auto dst_of = [&](int j) { return j < my_units ? dst_info[(size_t)tile_of(j) * TC_ROWS + 32 * quad + lane] : -1; };
        int next_info = eg < EG ? dst_of(eg) : -1;
        for (int j = eg; eg < EG && j < my_units; j += EG) {
            const int b = j % NB, u = j / NB;
            const int my_info = next_info;
            next_info = dst_of(j + EG);
            const bool okw = mbar_wait_ab(acc_full(b), (uint32_t)(u & 1), abort_flag);
            if (!__all_sync(0xffffffffu, okw)) {
                if (lane == 0) fail(5);
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
            for (int cb = 0; cb < R; cb += 32) {
                uint32_t v[32];
                const uint32_t a = taddr + (uint32_t)b * buf_cols + ((uint32_t)(32 * quad) << 16) + (uint32_t)cb;
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                    "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                      "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                      "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
                      "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
                      "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                    : "r"(a));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int q = 0; q < 32; ++q) E[lane * EPI_LD + q] = __uint_as_float(v[q]);
                __syncwarp();
                const int col = cb + 4 * (lane & 7);
                const int te = (cb >> 5) * 8 + (lane & 7);
                const uint32_t sg = sgn_tab[te], zm = zm_tab[te];
#pragma unroll
                for (int pass = 0; pass < 8; ++pass) {
                    const int rr = 4 * pass + (lane >> 3);
                    const int info = __shfl_sync(0xffffffffu, my_info, rr);
                    if (info >= 0 && col < R) {
                        const float* e = E + rr * EPI_LD + 4 * (lane & 7);
                        const float4 w =
                            apply_zero(apply_signs(make_float4(e[0], e[1], e[2], e[3]), (sg >> (4 * (info & 7))) & 15u), zm);
                        atomicAdd(reinterpret_cast<float4*>(L + (size_t)(info >> 3) + col), w);
                    }
                }
                __syncwarp();
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncwarp();
            if (lane == 0) mbar_arrive(acc_empty(b));
        }
    }
    __syncthreads();
    // drain what this CTA issued before TMEM is released (waits on completed phases return at once)
    if (tid == 0) {
        for (int i = issued_tma - NST > 0 ? issued_tma - NST : 0; i < issued_tma; ++i)
            mbar_wait(full(i % NST), (uint32_t)((i / NST) & 1));
    }
    if (tid == 32) {
        for (int i = issued_mma - NST > 0 ? issued_mma - NST : 0; i < issued_mma; ++i)
            mbar_wait(empty(i % NST), (uint32_t)((i / NST) & 1));
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(512));
}

// Row tables of the tensor-core tiles (see k_m2l_tc). A pair has nc * nsys rows: component c
// of copy q (a Stokes batch keeps one copy of the expansions per vector, esys reals apart).
__global__ void k_tc_rowinfo(const int4* tiles, int ntiles, const int* pt, const int* ps, const int* prefl, int nc,
                             int nsys, size_t esys, int* src_info, int* dst_info) {
    const int t = blockIdx.x, r = threadIdx.x;
    if (t >= ntiles || r >= TC_ROWS) return;
    const int4 tile = tiles[t];
    const int rows = nc * nsys;
    int si = -1, di = -1;
    if (r < tile.z * rows) {
        const int pr = tile.y + r / rows, q = (r % rows) / nc, comp = r % nc;
        si = (int)(q * esys + ((size_t)ps[pr] * nc + comp) * ESTRIDE) * 8 + prefl[pr];
        di = (int)(q * esys + ((size_t)pt[pr] * nc + comp) * ESTRIDE) * 8 + prefl[pr];
    }
    src_info[(size_t)t * TC_ROWS + r] = si;
    dst_info[(size_t)t * TC_ROWS + r] = di;
}

// Real operators of the tree translations between a cell and a child in the canonical
// octant, in the layout of the M2L operators (input-major [nr][nr], nr = 2 ncoef(pmax)):
//   op 0, M2M (child -> parent), d = c_child - c_parent = (-1/4, -1/4, -1/4) s_parent:
//     M~_n^m(P) = sum_{j,k} 2^{-j} M~_j^k(c) conj(R_{n-j}^{m-k}(d / s_parent));
//   op 1, L2L (parent -> child), d = (+1/4, +1/4, +1/4) s_parent:
//     L^_j^k(c) = 2^{-(j+1)} sum_{n >= j, m} L^_n^m(P) R_{n-j}^{m-k}(d / s_parent).
// Column kin is the image of the unit input (Re or Im of one m >= 0 coefficient; its
// m < 0 partner follows from X_n^{-m} = (-1)^m conj(X_n^m)). Other octants are reached by
// the axis reflections of the M2L path (target - source >= 0 in the canonical octant).
__global__ void k_tree_ops(int pmax, double* Td) {
    __shared__ cpx<double> R[NCOEF_MAX];
    const int op = blockIdx.y, kin = blockIdx.x;
    const int nr = 2 * ncoef(pmax);
    if (threadIdx.x == 0) {
        const double d = op == 0 ? -0.25 : 0.25;
        regular_table<double>(d, d, d, pmax, R);
    }
    __syncthreads();
    auto rnm = [&](int n, int m) -> cpx<double> {  // R_n^m for any m, |m| <= n
        if (m >= 0) return R[cidx(n, m)];
        const cpx<double> v = R[cidx(n, -m)];
        return (m & 1) ? mk(-v.re, v.im) : mk(v.re, -v.im);
    };
    const int cin = kin >> 1, pin = kin & 1;
    int n0 = 0;
    while ((n0 + 1) * (n0 + 2) / 2 <= cin) ++n0;
    const int m0 = cin - n0 * (n0 + 1) / 2;
    // the unit input at m0 and, for m0 > 0, its partner at -m0
    const cpx<double> v_pos = pin == 0 ? mk(1.0, 0.0) : mk(0.0, 1.0);
    const cpx<double> v_neg = (m0 & 1) ? mk(-v_pos.re, v_pos.im) : mk(v_pos.re, -v_pos.im);
    for (int rout = threadIdx.x; rout < nr; rout += blockDim.x) {
        const int cout = rout >> 1, pout = rout & 1;
        int n = 0;
        while ((n + 1) * (n + 2) / 2 <= cout) ++n;
        const int m = cout - n * (n + 1) / 2;
        cpx<double> acc = mk(0.0, 0.0);
        for (int sgn = 0; sgn < (m0 > 0 ? 2 : 1); ++sgn) {
            const int mi = sgn ? -m0 : m0;
            const cpx<double> v = sgn ? v_neg : v_pos;
            if (op == 0) {  // input degree j = n0 feeds output degree n >= n0
                if (n0 <= n && abs(m - mi) <= n - n0) acc = acc + ldexp(1.0, -n0) * (v * conj(rnm(n - n0, m - mi)));
            } else {        // input degree n0 feeds output degree j = n <= n0
                if (n <= n0 && abs(mi - m) <= n0 - n) acc = acc + ldexp(1.0, -(n + 1)) * (v * rnm(n0 - n, mi - m));
            }
        }
        Td[(size_t)op * nr * nr + (size_t)kin * nr + rout] = pout == 0 ? acc.re : acc.im;
    }
}

// Zero the first R reals of every expansion of the listed cells (M2M accumulates into them).
__global__ void k_zero_cells(const int* cells, int n, int nc, int R, float* X, size_t esys) {
    const int c = blockIdx.x;
    if (c >= n) return;
    float* row = X + blockIdx.y * esys + (size_t)cells[c] * nc * ESTRIDE;  // copy blockIdx.y of a Stokes batch
    for (int e = threadIdx.x; e < nc * R; e += blockDim.x) row[(e / R) * ESTRIDE + e % R] = 0.f;
}

}  // namespace

// Orders whose tensor-core passes keep the gathered rows in TMEM (tc_atm_at).
static bool atm_at(const fmmbem_handle* h, int p) { return tc_atm_at(p, h->tc_kc); }

size_t m2l_tc_smem(const fmmbem_handle* h, int p) { return tc_layout(p, h->tc_kc, atm_at(h, p)).bytes(); }

// The operator tables in the handle's chunk layout.
static void launch_tc_tables(const fmmbem_handle* h, unsigned grid, const double* Td, int ntab, int nr, int ld, int nch,
                             int rows_max, float* out, cudaStream_t st) {
    k_tc_tables<TC_KC><<<grid, 256, 0, st>>>(Td, ntab, nr, ld, nch, rows_max, out);
}

// M2M and L2L of each level as tensor-core products: the pairs (parent at level l, child)
// in tiles of 128 rows with the row tables of the M2L path; op 0 (M2M) reads the children
// and accumulates into the parents, op 1 (L2L) reads the parents and accumulates into the
// children.
static int build_tree_tc(fmmbem_handle* h, int nr, int rows_max, int nch) {
    cudaStream_t st = h->stream;
    const int nc = h->n_cells, NC = h->ncomp;
    double* Td = nullptr;
    FMM_CU(fmm_malloc((void**)&Td, sizeof(double) * 2 * (size_t)nr * nr));
    k_tree_ops<<<dim3(nr, 2), 128, 0, st>>>(h->opts.p_max, Td);
    FMM_LAUNCHED();
    const size_t per_tab = (size_t)nch * 2 * rows_max * h->tc_kc;
    FMM_CU(fmm_malloc((void**)&h->tree_tab_tc, sizeof(float) * 2 * per_tab));
    launch_tc_tables(h, 256, Td, 2, nr, nr, nch, rows_max, h->tree_tab_tc, st);
    FMM_LAUNCHED();
    std::vector<double4> cs(nc);
    std::vector<int2> ch(nc);
    std::vector<int> par(h->parent_start.back());
    FMM_CU(cudaMemcpyAsync(cs.data(), h->cell_cs, sizeof(double4) * nc, cudaMemcpyDeviceToHost, st));
    FMM_CU(cudaMemcpyAsync(ch.data(), h->cell_child, sizeof(int2) * nc, cudaMemcpyDeviceToHost, st));
    if (!par.empty())
        FMM_CU(cudaMemcpyAsync(par.data(), h->parents, sizeof(int) * par.size(), cudaMemcpyDeviceToHost, st));
    FMM_CU(cudaStreamSynchronize(st));
    fmm_free(Td);
    std::vector<int4> tiles;
    std::vector<int> m_src, m_dst, l_src, l_dst;
    h->tree_tile_start.assign(1, 0);
    for (int l = 0; l + 1 < h->n_levels; ++l) {
        std::vector<int> rows_ms, rows_md, rows_ls, rows_ld;
        for (int pi = h->parent_start[l]; pi < h->parent_start[l + 1]; ++pi) {
            const int pc = par[pi];
            for (int x = 0; x < ch[pc].y; ++x) {
                const int cc = ch[pc].x + x;
                const int o = (cs[cc].x > cs[pc].x ? 1 : 0) | (cs[cc].y > cs[pc].y ? 2 : 0) | (cs[cc].z > cs[pc].z ? 4 : 0);
                for (int q = 0; q < h->nsys; ++q)  // every copy of a Stokes batch
                    for (int comp = 0; comp < NC; ++comp) {
                        const int prow = (int)(q * h->esys) + (pc * NC + comp) * ESTRIDE;
                        const int crow = (int)(q * h->esys) + (cc * NC + comp) * ESTRIDE;
                        rows_ms.push_back(crow * 8 + o);
                        rows_md.push_back(prow * 8 + o);
                        rows_ls.push_back(prow * 8 + (7 - o));
                        rows_ld.push_back(crow * 8 + (7 - o));
                    }
            }
        }
        const int nt = ((int)rows_ms.size() + TC_ROWS - 1) / TC_ROWS;
        for (int t = 0; t < nt; ++t) {
            tiles.push_back(make_int4(0, 0, 0, 0));
            for (int r = 0; r < TC_ROWS; ++r) {
                const size_t e = (size_t)t * TC_ROWS + r;
                const bool in = e < rows_ms.size();
                m_src.push_back(in ? rows_ms[e] : -1);
                m_dst.push_back(in ? rows_md[e] : -1);
                l_src.push_back(in ? rows_ls[e] : -1);
                l_dst.push_back(in ? rows_ld[e] : -1);
            }
        }
        h->tree_tile_start.push_back((int)tiles.size());
    }
    const size_t ntl = tiles.size();
    FMM_CU(fmm_malloc((void**)&h->tree_tiles, sizeof(int4) * (ntl ? 2 * ntl : 1)));
    FMM_CU(fmm_malloc((void**)&h->tree_info, sizeof(int) * (ntl ? 4 * ntl * TC_ROWS : 1)));
    if (ntl) {
        std::vector<int4> both(tiles);
        for (auto& t : tiles) both.push_back(make_int4(1, 0, 0, 0));  // L2L tiles use op 1
        FMM_CU(cudaMemcpyAsync(h->tree_tiles, both.data(), sizeof(int4) * 2 * ntl, cudaMemcpyHostToDevice, st));
        const size_t rw = ntl * TC_ROWS;
        FMM_CU(cudaMemcpyAsync(h->tree_info, m_src.data(), sizeof(int) * rw, cudaMemcpyHostToDevice, st));
        FMM_CU(cudaMemcpyAsync(h->tree_info + rw, m_dst.data(), sizeof(int) * rw, cudaMemcpyHostToDevice, st));
        FMM_CU(cudaMemcpyAsync(h->tree_info + 2 * rw, l_src.data(), sizeof(int) * rw, cudaMemcpyHostToDevice, st));
        FMM_CU(cudaMemcpyAsync(h->tree_info + 3 * rw, l_dst.data(), sizeof(int) * rw, cudaMemcpyHostToDevice, st));
        FMM_CU(cudaStreamSynchronize(st));  // the host vectors go out of scope
    }
    h->n_tree_tiles = (int)ntl;
    return 0;
}

int build_m2l_tc(fmmbem_handle* h) {
    if (!h->m2l_tables) return 0;
    // row tables pack (offset * 8 + reflection) into an int
    if ((double)h->esys * h->nsys * 8.0 >= 2147483647.0) return 0;
    const int pmax = h->opts.p_max;
    const int nr = 2 * ncoef(pmax);
    const int rows_max = (nr + 15) & ~15;
    h->tc_kc = TC_KC;
    const int nch = (nr + h->tc_kc - 1) / h->tc_kc;
    const size_t per_tab = (size_t)nch * 2 * rows_max * h->tc_kc;
    FMM_CU(fmm_malloc((void**)&h->tab_tc, sizeof(float) * per_tab * (size_t)h->n_tables));
    launch_tc_tables(h, 2048, h->tab_d, h->n_tables, nr, h->tab_ld, nch, rows_max, h->tab_tc, h->stream);
    FMM_LAUNCHED();
    h->tc_stride = per_tab;
    h->tc_rows_max = rows_max;
    FMM_CU(fmm_malloc((void**)&h->tc_src_info, sizeof(int) * (size_t)h->n_tiles_tc * TC_ROWS));
    FMM_CU(fmm_malloc((void**)&h->tc_dst_info, sizeof(int) * (size_t)h->n_tiles_tc * TC_ROWS));
    if (h->n_tiles_tc > 0) {
        k_tc_rowinfo<<<h->n_tiles_tc, TC_ROWS, 0, h->stream>>>(h->m2l_tiles_tc, h->n_tiles_tc, h->m2l_pt, h->m2l_ps,
                                                               h->m2l_refl, h->ncomp, h->nsys, h->esys, h->tc_src_info,
                                                               h->tc_dst_info);
        FMM_LAUNCHED();
    }
    FMM_CU(fmm_malloc((void**)&h->tc_err, sizeof(int)));
    FMM_CU(cudaMemsetAsync(h->tc_err, 0, sizeof(int), h->stream));
    FMM_TRY(build_tree_tc(h, nr, rows_max, nch));
    size_t smax = 0;
    for (int q = 1; q <= pmax; ++q)
        smax = std::max({smax, tc_layout(q, h->tc_kc, false).bytes(), tc_layout(q, h->tc_kc, true).bytes()});
    FMM_CU(cudaFuncSetAttribute(k_m2l_tc<TC_KC, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smax));
    FMM_CU(cudaFuncSetAttribute(k_m2l_tc<TC_KC, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smax));
    FMM_CU(cudaFuncSetAttribute(k_m2l_tc<TC_KC, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smax));
    FMM_CU(cudaFuncSetAttribute(k_m2l_tc<TC_KC, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smax));
    int dev = 0;
    FMM_CU(cudaGetDevice(&dev));
    FMM_CU(cudaDeviceGetAttribute(&h->n_sm, cudaDevAttrMultiProcessorCount, dev));
    h->m2l_tc_ready = true;
    return 0;
}

// Zero the multipole expansions of every non-leaf cell (the M2M products accumulate into them).
int tree_tc_zero(fmmbem_handle* h, int p) {
    const int np = h->parent_start.back();
    if (np <= 0) return 0;
    k_zero_cells<<<dim3(np, h->nsys), 128, 0, h->stream>>>(h->parents, np, h->ncomp, 2 * ncoef(p),
                                                            reinterpret_cast<float*>(h->M), h->esys);
    FMM_LAUNCHED();
    return 0;
}

// Launch of the tensor-core kernel with programmatic stream serialization: consecutive
// tensor-core passes of a mat-vec (tree levels, M2L) overlap each launch's set-up with the
// previous one's tail (the kernel waits for its predecessor before reading expansions).
template <int KC, bool SPLIT, bool ATM>
static cudaError_t launch_tc1(int grid, size_t smem, cudaStream_t st, int p, int prods, const int4* tiles, int nt,
                              int ks, const int* src, const int* dst, const float* tab, size_t stride, int rows_max,
                              const float* M, float* L, int* err) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(TC_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_m2l_tc<KC, SPLIT, ATM>, p, prods, tiles, nt, ks, src, dst, tab, stride, rows_max,
                              M, L, err);
}

template <bool SPLIT>
static cudaError_t launch_tc(const fmmbem_handle* h, int grid, cudaStream_t st, int p, int prods, const int4* tiles,
                             int nt, int ks, const int* src, const int* dst, const float* tab, size_t stride,
                             int rows_max, const float* M, float* L, int* err) {
    const size_t smem = m2l_tc_smem(h, p);
    return atm_at(h, p) ? launch_tc1<TC_KC, SPLIT, true>(grid, smem, st, p, prods, tiles, nt, ks, src, dst, tab, stride,
                                                          rows_max, M, L, err)
                        : launch_tc1<TC_KC, SPLIT, false>(grid, smem, st, p, prods, tiles, nt, ks, src, dst, tab, stride,
                                                           rows_max, M, L, err);
}

// One level of M2M (which = 0: children of level l into their parents, zeroed beforehand
// by tree_tc_zero) or L2L (which = 1: parents of level l into their children) on the
// tensor cores.
int tree_tc(fmmbem_handle* h, int p, int level, int which) {
    const int t0 = h->tree_tile_start[level], t1 = h->tree_tile_start[level + 1];
    const int nt = t1 - t0;
    if (nt <= 0) return 0;
    float* X = reinterpret_cast<float*>(which == 0 ? h->M : h->L);
    const size_t rw = (size_t)h->n_tree_tiles * TC_ROWS;
    const int* src = h->tree_info + (which == 0 ? 0 : 2 * rw) + (size_t)t0 * TC_ROWS;
    const int* dst = h->tree_info + (which == 0 ? rw : 3 * rw) + (size_t)t0 * TC_ROWS;
    const int4* tiles = h->tree_tiles + (which == 0 ? 0 : h->n_tree_tiles) + t0;
    // a level has few tiles (tens against 152 SMs): split each tile's K chunks over several
    // CTAs so that more SMs share the level and each CTA's chain of chunks is shorter
    const int nch = (2 * ncoef(p) + h->tc_kc - 1) / h->tc_kc;
    const int ks = std::max(1, std::min(nch, h->n_sm / nt));
    const int grid = std::min(nt * ks, h->n_sm);
    FMM_CU((launch_tc<true>(h, grid, h->stream, p, 3, tiles, nt, ks, src, dst, h->tree_tab_tc, h->tc_stride,
                            h->tc_rows_max, X, X, h->tc_err)));
    return 0;
}

// The local expansions are zeroed ahead of the upward pass (nothing reads or writes them until
// the M2L), so that the M2L launch follows the last M2M level directly and its set-up overlaps
// that level's tail.
int m2l_tc_zero(fmmbem_handle* h) {
    FMM_CU(cudaMemsetAsync(h->L, 0, sizeof(float) * h->esys * h->nsys, h->stream));
    return 0;
}

int m2l_tc(fmmbem_handle* h, int p) {
    float* L = reinterpret_cast<float*>(h->L);
    const float* M = reinterpret_cast<const float*>(h->M);
    const int grid = std::min(h->n_tiles_tc, h->n_sm);  // persistent: one CTA per SM (512 TMEM columns each)
    const int prods = 3;
    if (grid <= 0) return 0;
    FMM_CU((launch_tc<false>(h, grid, h->stream, p, prods, h->m2l_tiles_tc, h->n_tiles_tc, 1, h->tc_src_info,
                             h->tc_dst_info, h->tab_tc, h->tc_stride, h->tc_rows_max, M, L, h->tc_err)));
    return 0;
}

}  // namespace fmmbem
