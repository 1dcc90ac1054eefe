// Peak-rate kernels: the denominators of the near-field, far-field and FP64 rooflines,
// measured on the running GPU at its current clocks instead of derived from unit counts.
//   FFMA  : fma.rn.f32, 2 flop each (the FP32 pipe);
//   FFMA2 : fma.rn.f32x2, 4 flop each (the paired FP32 instruction of sm_100-family GPUs);
//   RSQRT : rsqrt.approx.ftz.f32 results (the special-function unit; the near field issues
//           this instruction once per pair);
//   DFMA  : FP64 fma, 2 flop each;
//   TF32  : tcgen05.mma.kind::tf32 of M = 128, N = 256, K = 8 on shared-memory operands into
//           TMEM, 2 M N K flop each (one issuing thread per CTA, one CTA per SM).
// Every thread runs eight independent dependency chains so that the pipe, not the latency
// of one chain, bounds the rate. The chains' values are kept live by a store that the
// compiler cannot prove dead.
#include "handle.cuh"
#include "tc_ptx.cuh"

namespace fmmbem {

namespace {

constexpr int PK_THREADS = 256;
constexpr int PK_BLOCKS_PER_SM = 4;
constexpr int PK_CHAINS = 8;

__global__ void __launch_bounds__(PK_THREADS) k_peak_ffma(int64_t iters, float a, float b, float* sink) {
    float x[PK_CHAINS];
#pragma unroll
    for (int c = 0; c < PK_CHAINS; ++c) x[c] = 1e-3f * (float)(threadIdx.x + c);
    for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < PK_CHAINS; ++c) x[c] = fmaf(x[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < PK_CHAINS; ++c) s += x[c];
    if (s == -1.f) sink[blockIdx.x] = s;
}

__global__ void __launch_bounds__(PK_THREADS) k_peak_ffma2(int64_t iters, float a, float b, float* sink) {
    f32x2 x[PK_CHAINS];
    const f32x2 va = f2_pack(a, a), vb = f2_pack(b, b);
#pragma unroll
    for (int c = 0; c < PK_CHAINS; ++c) x[c] = f2_pack(1e-3f * (float)(threadIdx.x + c), 2e-3f * (float)c);
    for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < PK_CHAINS; ++c) x[c] = f2_fma(x[c], va, vb);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < PK_CHAINS; ++c) {
        float u, v;
        f2_unpack(x[c], u, v);
        s += u + v;
    }
    if (s == -1.f) sink[blockIdx.x] = s;
}

__global__ void __launch_bounds__(PK_THREADS) k_peak_rsqrt(int64_t iters, float a, float b, float* sink) {
    float x[PK_CHAINS];
#pragma unroll
    for (int c = 0; c < PK_CHAINS; ++c) x[c] = 1.f + 1e-3f * (float)(threadIdx.x + c);
    for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < PK_CHAINS; ++c) {  // one add on the FMA pipe beside it
            float y;
            asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x[c] + b));
            x[c] = y;
        }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < PK_CHAINS; ++c) s += x[c];
    if (s == -1.f) sink[blockIdx.x] = s + a;
}

__global__ void __launch_bounds__(PK_THREADS) k_peak_dfma(int64_t iters, double a, double b, float* sink) {
    double x[PK_CHAINS];
#pragma unroll
    for (int c = 0; c < PK_CHAINS; ++c) x[c] = 1e-3 * (double)(threadIdx.x + c);
    for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < PK_CHAINS; ++c) x[c] = fma(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < PK_CHAINS; ++c) s += x[c];
    if (s == -1.0) sink[blockIdx.x] = (float)s;
}

// TF32 tensor-core rate. A (128 x 32) and B (256 x 32) sit in shared memory in the K-major
// no-swizzle core-matrix layout of the M2L kernel (8 rows x 16 bytes per core matrix, 128 B
// between core matrices along K, 1024 B between 8-row groups); each iteration issues the
// four K = 8 steps of that chunk into one of two TMEM accumulators of 256 columns. One
// thread issues; the issue queue's back-pressure paces it. A final commit to an mbarrier
// and a bounded wait for it precede the TMEM release; a wait that gives up sets *err.
constexpr int TF_M = 128, TF_N = 256, TF_KC = 32;
constexpr uint32_t TF_WAIT_LIMIT = 1u << 26;
constexpr size_t TF_SMEM = (size_t)(TF_M + TF_N) * TF_KC * 4 + 64;

__global__ void __launch_bounds__(128, 1) k_peak_tf32(int64_t iters, int* err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    float* A = reinterpret_cast<float*>(smem);
    float* B = A + TF_M * TF_KC;
    uint64_t* bar = reinterpret_cast<uint64_t*>(B + TF_N * TF_KC);
    uint32_t* slot = reinterpret_cast<uint32_t*>(bar + 1);
    const int tid = threadIdx.x, warp = tid >> 5;
    for (int i = tid; i < (TF_M + TF_N) * TF_KC; i += blockDim.x) A[i] = 1e-3f * (float)(i % 13);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    // the operands were written through the generic proxy and are read by the tensor cores
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t taddr = *slot;
    if (tid == 0) {
        const uint32_t id = idesc_tf32(TF_M, TF_N);
        const uint32_t a0 = smem_u32(A), b0 = smem_u32(B);
        for (int64_t it = 0; it < iters; ++it) {
            const uint32_t acc = taddr + (uint32_t)(it & 1) * TF_N;
#pragma unroll
            for (int ks = 0; ks < TF_KC / 8; ++ks) {
                const uint32_t off = 256u * ks;
                mma_tf32(acc, smem_desc(a0 + off, 128, 1024), smem_desc(b0 + off, 128, 1024), id,
                         (it >= 2 || ks > 0) ? 1u : 0u);
            }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                     : "memory");
        if (!mbar_wait_bounded(smem_u32(bar), 0u, TF_WAIT_LIMIT)) atomicExch(err, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(512));
}

}  // namespace

int peak_rate(int kind, int blocks, int64_t iters, double* ops, double* ms, cudaStream_t st) {
    int dev = 0, sms = 0;
    FMM_CU(cudaGetDevice(&dev));
    FMM_CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const bool tc = kind == FMMBEM_PEAK_TF32;
    if (blocks <= 0) blocks = tc ? sms : sms * PK_BLOCKS_PER_SM;
    if (tc && blocks > sms) {
        fmmbem_set_error("the TF32 rate runs at most one CTA per SM (%d)", sms);
        return FMMBEM_EINVAL;
    }
    float* sink = nullptr;
    int* err = nullptr;
    FMM_CU(cudaMallocAsync((void**)&sink, sizeof(float) * blocks + sizeof(int), st));
    err = reinterpret_cast<int*>(sink + blocks);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = 0;
    auto done = [&](int code) {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        cudaFreeAsync(sink, st);
        cudaStreamSynchronize(st);
        return code;
    };
    if (cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess) {
        fmmbem_set_error("peak_rate: set-up failed: %s", cudaGetErrorString(cudaGetLastError()));
        return done(FMMBEM_EDEVICE);
    }
    if (tc && cudaFuncSetAttribute(k_peak_tf32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TF_SMEM) != cudaSuccess) {
        fmmbem_set_error("peak_rate: %s", cudaGetErrorString(cudaGetLastError()));
        return done(FMMBEM_EDEVICE);
    }
    cudaEventRecord(e0, st);
    double per = 0.0;  // operations per thread-iteration (ALU) or per CTA-iteration (TF32)
    switch (kind) {
        case FMMBEM_PEAK_FFMA:
            k_peak_ffma<<<blocks, PK_THREADS, 0, st>>>(iters, 0.9999f, 1e-4f, sink);
            per = 2.0 * PK_CHAINS;
            break;
        case FMMBEM_PEAK_FFMA2:
            k_peak_ffma2<<<blocks, PK_THREADS, 0, st>>>(iters, 0.9999f, 1e-4f, sink);
            per = 4.0 * PK_CHAINS;
            break;
        case FMMBEM_PEAK_RSQRT:
            k_peak_rsqrt<<<blocks, PK_THREADS, 0, st>>>(iters, 0.f, 0.5f, sink);
            per = 1.0 * PK_CHAINS;
            break;
        case FMMBEM_PEAK_DFMA:
            k_peak_dfma<<<blocks, PK_THREADS, 0, st>>>(iters, 0.9999, 1e-4, sink);
            per = 2.0 * PK_CHAINS;
            break;
        case FMMBEM_PEAK_TF32:
            k_peak_tf32<<<blocks, 128, TF_SMEM, st>>>(iters, err);
            per = 2.0 * TF_M * TF_N * 8 * (TF_KC / 8);
            break;
        default:
            fmmbem_set_error("unknown peak kind %d", kind);
            return done(FMMBEM_EINVAL);
    }
    if (cudaGetLastError() != cudaSuccess) {
        fmmbem_set_error("peak_rate launch: %s", cudaGetErrorString(cudaGetLastError()));
        return done(FMMBEM_EDEVICE);
    }
    cudaEventRecord(e1, st);
    int herr = 0;
    if (cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        fmmbem_set_error("peak_rate: %s", cudaGetErrorString(cudaGetLastError()));
        return done(FMMBEM_EDEVICE);
    }
    if (herr) {
        fmmbem_set_error("peak_rate: the tensor-core completion wait gave up");
        rc = FMMBEM_ETIMEOUT;
    }
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    if (ms) *ms = t;
    if (ops) *ops = per * (double)iters * (double)blocks * (tc ? 1.0 : (double)PK_THREADS);
    return done(rc);
}

}  // namespace fmmbem

extern "C" int fmmbem_peak(int kind, int blocks, int64_t iters, double* ops, double* ms, void* stream) {
    if (iters < 1 || blocks < 0) {
        fmmbem_set_error("peak: need iters >= 1 and blocks >= 0");
        return FMMBEM_EINVAL;
    }
    return fmmbem::peak_rate(kind, blocks, iters, ops, ms, (cudaStream_t)stream);
}
