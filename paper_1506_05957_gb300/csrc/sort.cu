// Device-wide sorts and scans of the create step: the Morton sort of the panels, the
// sorts of the M2L pair keys and of the interaction-list pairs into CSR, the leaf order,
// and the prefix sums that turn counts into offsets.
//
// Radix sort: least-significant-digit first, 8-bit digits, stable (equal keys keep their
// input order, which every pass relies on). Per pass:
//   1. k_rs_hist    : each block counts the digits of its tile of RS_TILE keys;
//   2. exclusive scan of the counts laid out digit-major ([digit][block]), so that
//      offset[d][b] is where block b's first key of digit d goes;
//   3. k_rs_scatter : each block walks its tile in rounds of one key per thread, in input
//      order; a key's place among the round's equal digits comes from the warp's match of
//      digits and a per-warp count table, and the block keeps a running count per digit.
// Scan: a block sums each tile, the tile sums are scanned (recursively), and each block
// rescans its tile from its offset.
#include <stdint.h>
#include "handle.cuh"

namespace fmmbem {

namespace {

constexpr int RS_THREADS = 256;
constexpr int RS_ITEMS = 8;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;
constexpr int RS_BINS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;

template <typename K>
__global__ void __launch_bounds__(RS_THREADS) k_rs_hist(const K* keys, int64_t n, int shift, int* hist) {
    __shared__ int h[RS_BINS];
    const int tid = threadIdx.x;
    h[tid] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
#pragma unroll
    for (int i = 0; i < RS_ITEMS; ++i) {
        const int64_t idx = base + i * RS_THREADS + tid;
        if (idx < n) atomicAdd(&h[(int)((keys[idx] >> shift) & (RS_BINS - 1))], 1);
    }
    __syncthreads();
    hist[(int64_t)tid * gridDim.x + blockIdx.x] = h[tid];
}

template <typename K>
__global__ void __launch_bounds__(RS_THREADS) k_rs_scatter(const K* kin, const int* vin, K* kout, int* vout, int64_t n,
                                                           int shift, const int* off, int* err) {
    __shared__ int s_cnt[RS_WARPS][RS_BINS];  // per warp: keys of each digit in this round (then their prefix)
    __shared__ int s_run[RS_BINS];            // keys of each digit this block has placed in earlier rounds
    __shared__ int s_tot[RS_BINS];            // keys of each digit in this round
    __shared__ int s_base[RS_BINS];           // the block's first place for each digit
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    s_run[tid] = 0;
    s_base[tid] = off[(int64_t)tid * gridDim.x + blockIdx.x];
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
    const unsigned lt = (1u << lane) - 1u;
    for (int round = 0; round < RS_ITEMS; ++round) {
#pragma unroll
        for (int w = 0; w < RS_WARPS; ++w) s_cnt[w][tid] = 0;
        __syncthreads();
        const int64_t idx = base + round * RS_THREADS + tid;
        const bool valid = idx < n;
        const K k = valid ? kin[idx] : K(0);
        const int v = (valid && vin) ? vin[idx] : 0;
        // past the end each lane gets a digit of its own, so it has no peers
        const int d = valid ? (int)((k >> shift) & (RS_BINS - 1)) : RS_BINS + lane;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int rank = __popc(peers & lt);
        if (valid && rank == 0) s_cnt[warp][d] = __popc(peers);
        __syncthreads();
        {  // digit tid: exclusive prefix over the warps, in place
            int run = 0;
#pragma unroll
            for (int w = 0; w < RS_WARPS; ++w) {
                const int c = s_cnt[w][tid];
                s_cnt[w][tid] = run;
                run += c;
            }
            s_tot[tid] = run;
        }
        __syncthreads();
        if (valid) {
            const int pos = s_base[d] + s_run[d] + s_cnt[warp][d] + rank;
            if (pos >= 0 && pos < n) {  // always, by construction; a place outside is flagged, never written
                kout[pos] = k;
                if (vout) vout[pos] = v;
            } else {
                atomicExch(err, 1);
            }
        }
        __syncthreads();
        s_run[tid] += s_tot[tid];
    }
}

constexpr int SC_THREADS = 512;
constexpr int SC_ITEMS = 4;
constexpr int SC_TILE = SC_THREADS * SC_ITEMS;

// Exclusive prefix of v over the block (512 threads) and the block total.
__device__ __forceinline__ int block_excl_scan(int v, int* s_warp, int* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = lane < SC_THREADS / 32 ? s_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < SC_THREADS / 32) s_warp[lane] = w;  // inclusive prefix of the warp sums
    }
    __syncthreads();
    *total = s_warp[SC_THREADS / 32 - 1];
    const int before = warp > 0 ? s_warp[warp - 1] : 0;
    __syncthreads();
    return before + x - v;
}

__global__ void __launch_bounds__(SC_THREADS) k_scan_sums(const int* in, int64_t n, int* sums) {
    __shared__ int s_warp[SC_THREADS / 32];
    const int64_t base = (int64_t)blockIdx.x * SC_TILE + (int64_t)threadIdx.x * SC_ITEMS;
    int t = 0;
#pragma unroll
    for (int i = 0; i < SC_ITEMS; ++i)
        if (base + i < n) t += in[base + i];
    int total = 0;
    block_excl_scan(t, s_warp, &total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// out = exclusive (or inclusive) prefix of in, offset by the scanned tile sums (or 0)
__global__ void __launch_bounds__(SC_THREADS) k_scan_apply(const int* in, int* out, int64_t n, const int* tile_off,
                                                           int inclusive) {
    __shared__ int s_warp[SC_THREADS / 32];
    const int64_t base = (int64_t)blockIdx.x * SC_TILE + (int64_t)threadIdx.x * SC_ITEMS;
    int v[SC_ITEMS], t = 0;
#pragma unroll
    for (int i = 0; i < SC_ITEMS; ++i) {
        v[i] = base + i < n ? in[base + i] : 0;
        t += v[i];
    }
    int total = 0;
    int run = block_excl_scan(t, s_warp, &total) + (tile_off ? tile_off[blockIdx.x] : 0);
#pragma unroll
    for (int i = 0; i < SC_ITEMS; ++i) {
        if (base + i < n) out[base + i] = inclusive ? run + v[i] : run;
        run += v[i];
    }
}

int scan_i32(const int* in, int* out, int64_t n, bool inclusive, cudaStream_t st) {
    if (n <= 0) return 0;
    const int64_t nb = (n + SC_TILE - 1) / SC_TILE;
    if (nb > INT32_MAX) { fmmbem_set_error("scan: %lld elements", (long long)n); return FMMBEM_EINVAL; }
    if (nb == 1) {
        k_scan_apply<<<1, SC_THREADS, 0, st>>>(in, out, n, nullptr, inclusive ? 1 : 0);
        FMM_LAUNCHED();
        return 0;
    }
    int* sums = nullptr;
    FMM_CU(fmm_malloc(&sums, sizeof(int) * 2 * nb));
    int* offs = sums + nb;
    k_scan_sums<<<(unsigned)nb, SC_THREADS, 0, st>>>(in, n, sums);
    cudaError_t e = cudaGetLastError();
    int rc = e == cudaSuccess ? scan_i32(sums, offs, nb, false, st) : FMMBEM_EDEVICE;
    if (rc == 0) {
        k_scan_apply<<<(unsigned)nb, SC_THREADS, 0, st>>>(in, out, n, offs, inclusive ? 1 : 0);
        e = cudaGetLastError();
        if (e != cudaSuccess) rc = FMMBEM_EDEVICE;
    }
    if (e != cudaSuccess) fmmbem_set_error("scan: %s", cudaGetErrorString(e));
    fmm_free(sums);
    return rc;
}

template <typename K>
int radix_sort_t(const K* kin, K* kout, const int* vin, int* vout, int64_t n, int end_bit, cudaStream_t st) {
    if (n <= 0) return 0;
    if (n > INT32_MAX / 2) { fmmbem_set_error("radix sort: %lld keys", (long long)n); return FMMBEM_EINVAL; }
    const int maxbit = (int)(8 * sizeof(K));
    if (end_bit <= 0 || end_bit > maxbit) end_bit = maxbit;
    const int passes = (end_bit + 7) / 8;
    const int64_t nb = (n + RS_TILE - 1) / RS_TILE;
    K* ktmp = nullptr;
    int *vtmp = nullptr, *hist = nullptr;
    FMM_CU(fmm_malloc(&ktmp, sizeof(K) * n));
    FMM_CU(fmm_malloc(&hist, sizeof(int) * (RS_BINS * nb + 1)));
    int* err = hist + RS_BINS * nb;
    FMM_CU(cudaMemsetAsync(err, 0, sizeof(int), st));
    if (vin) FMM_CU(fmm_malloc(&vtmp, sizeof(int) * n));
    const K* ks = kin;
    const int* vs = vin;
    int rc = 0;
    for (int pass = 0; pass < passes && rc == 0; ++pass) {
        // the last pass writes the outputs; earlier passes alternate so that it does
        const bool to_out = ((passes - pass) & 1) == 1;
        K* kd = to_out ? kout : ktmp;
        int* vd = vin ? (to_out ? vout : vtmp) : nullptr;
        k_rs_hist<K><<<(unsigned)nb, RS_THREADS, 0, st>>>(ks, n, 8 * pass, hist);
        if (cudaGetLastError() != cudaSuccess) { rc = FMMBEM_EDEVICE; break; }
        rc = scan_i32(hist, hist, RS_BINS * nb, false, st);
        if (rc < 0) break;
        k_rs_scatter<K><<<(unsigned)nb, RS_THREADS, 0, st>>>(ks, vs, kd, vd, n, 8 * pass, hist, err);
        if (cudaGetLastError() != cudaSuccess) { rc = FMMBEM_EDEVICE; break; }
        ks = kd;
        vs = vd;
    }
    if (rc == FMMBEM_EDEVICE) fmmbem_set_error("radix sort: %s", cudaGetErrorString(cudaGetLastError()));
    if (rc == 0) {
        int herr = 0;
        if (cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            fmmbem_set_error("radix sort: %s", cudaGetErrorString(cudaGetLastError()));
            rc = FMMBEM_EDEVICE;
        } else if (herr) {
            fmmbem_set_error("radix sort: a key's place fell outside the output");
            rc = FMMBEM_EDEVICE;
        }
    }
    fmm_free(ktmp);
    fmm_free(hist);
    if (vtmp) fmm_free(vtmp);
    return rc;
}

}  // namespace

int radix_sort(const uint64_t* kin, uint64_t* kout, const int* vin, int* vout, int64_t n, int end_bit, cudaStream_t st) {
    return radix_sort_t<unsigned long long>(reinterpret_cast<const unsigned long long*>(kin),
                                            reinterpret_cast<unsigned long long*>(kout), vin, vout, n, end_bit, st);
}

int radix_sort(const uint32_t* kin, uint32_t* kout, const int* vin, int* vout, int64_t n, int end_bit, cudaStream_t st) {
    return radix_sort_t<unsigned int>(reinterpret_cast<const unsigned int*>(kin), reinterpret_cast<unsigned int*>(kout),
                                      vin, vout, n, end_bit, st);
}

int exclusive_scan(const int* in, int* out, int64_t n, cudaStream_t st) { return scan_i32(in, out, n, false, st); }

int inclusive_scan(const int* in, int* out, int64_t n, cudaStream_t st) { return scan_i32(in, out, n, true, st); }

}  // namespace fmmbem

// The exported forms (stream-ordered scratch on the caller's stream; arguments checked first).
extern "C" int fmmbem_sort_pairs_u64(const uint64_t* keys_in, uint64_t* keys_out, const int32_t* vals_in,
                                     int32_t* vals_out, int64_t n, int end_bit, void* stream) {
    if (n < 0 || end_bit < 0 || end_bit > 64 || (n > 0 && (!keys_in || !keys_out)) || ((vals_in == nullptr) != (vals_out == nullptr)) ||
        (n > 0 && (keys_in == keys_out || (vals_in && vals_in == vals_out)))) {
        fmmbem_set_error("sort_pairs_u64: need n >= 0, 0 <= end_bit <= 64, distinct input and output buffers, both or neither value buffer");
        return FMMBEM_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    cudaStream_t keep = fmm_alloc_stream();
    fmm_alloc_stream() = st;
    const int rc = fmmbem::radix_sort(keys_in, keys_out, vals_in, vals_out, n, end_bit, st);
    fmm_alloc_stream() = keep;
    return rc;
}

extern "C" int fmmbem_scan_i32(const int32_t* in, int32_t* out, int64_t n, int inclusive, void* stream) {
    if (n < 0 || (n > 0 && (!in || !out))) {
        fmmbem_set_error("scan_i32: need n >= 0 and device buffers");
        return FMMBEM_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    cudaStream_t keep = fmm_alloc_stream();
    fmm_alloc_stream() = st;
    int rc = inclusive ? fmmbem::inclusive_scan(in, out, n, st) : fmmbem::exclusive_scan(in, out, n, st);
    if (rc == 0 && cudaStreamSynchronize(st) != cudaSuccess) {
        fmmbem_set_error("scan_i32: %s", cudaGetErrorString(cudaGetLastError()));
        rc = FMMBEM_EDEVICE;
    }
    fmm_alloc_stream() = keep;
    return rc;
}
