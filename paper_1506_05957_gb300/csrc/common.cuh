// Shared definitions of the CUDA path: complex helpers, coefficient indexing,
// error reporting and launch checks.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include "fmmbem.h"

#define FMM_HD __host__ __device__ __forceinline__

namespace fmmbem {

constexpr int PMAX = FMMBEM_P_MAX;
// Expansions keep degrees n = 0..p and orders m = 0..n (the m < 0 half follows
// from X_n^{-m} = (-1)^m conj(X_n^m)): (p+1)(p+2)/2 complex coefficients.
constexpr int NCOEF_MAX = (PMAX + 1) * (PMAX + 2) / 2;
// Irregular harmonics needed by M2L reach degree 2p.
constexpr int NI_MAX = (2 * PMAX + 1) * (2 * PMAX + 2) / 2;
// Stride, in reals, of one expansion in the global M and L arrays: 2 * NCOEF_MAX = 306
// padded to a multiple of 32 so every expansion starts on a 128-byte boundary.
constexpr int ESTRIDE = 320;
constexpr int MAX_LEVELS = 21;  // 63-bit Morton keys, 21 bits per axis
constexpr int P2P_SRC_TMAX = 24;  // targets per block of the source-lane near-field kernel
constexpr int P2P_SRC_TMAX_STOKES = 8;   // the same for the Stokeslet (three accumulators per target)
constexpr int P2P_SRC_TMAX_BATCH = 8;    // the same for a batch of four vectors (four accumulators per target;
                                         // the per-lane partial sums stay within 48 KB of shared memory)

FMM_HD int cidx(int n, int m) { return (n * (n + 1)) / 2 + m; }
FMM_HD int ncoef(int p) { return (p + 1) * (p + 2) / 2; }

template <typename T> struct cpx { T re, im; };
template <typename T> FMM_HD cpx<T> mk(T r, T i) { cpx<T> z; z.re = r; z.im = i; return z; }
template <typename T> FMM_HD cpx<T> operator+(cpx<T> a, cpx<T> b) { return mk(a.re + b.re, a.im + b.im); }
template <typename T> FMM_HD cpx<T> operator-(cpx<T> a, cpx<T> b) { return mk(a.re - b.re, a.im - b.im); }
template <typename T> FMM_HD cpx<T> operator*(cpx<T> a, cpx<T> b) {
    return mk(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <typename T> FMM_HD cpx<T> operator*(T s, cpx<T> a) { return mk(s * a.re, s * a.im); }
template <typename T> FMM_HD cpx<T> conj(cpx<T> a) { return mk(a.re, -a.im); }
// acc += a * b
template <typename T> FMM_HD void cfma(cpx<T>& acc, cpx<T> a, cpx<T> b) {
    acc.re += a.re * b.re - a.im * b.im;
    acc.im += a.re * b.im + a.im * b.re;
}
// acc += conj(a) * b
template <typename T> FMM_HD void cfma_conja(cpx<T>& acc, cpx<T> a, cpx<T> b) {
    acc.re += a.re * b.re + a.im * b.im;
    acc.im += a.re * b.im - a.im * b.re;
}

// Two FP32 values in one 64-bit register, operated on by the paired FP32 instructions of
// sm_100-family GPUs (PTX .f32x2): one instruction applies the same operation to both halves,
// each rounded as the scalar FP32 operation, which halves the issue slots of the arithmetic.
typedef unsigned long long f32x2;
__device__ __forceinline__ f32x2 f2_pack(float a, float b) {
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void f2_unpack(f32x2 v, float& a, float& b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ f32x2 f2_sub(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 f2_mul(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 f2_fma(f32x2 a, f32x2 b, f32x2 c) {
    f32x2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// 4-wide vector of the arithmetic type (positions + weight).
template <typename T> struct V4;
template <> struct V4<float> { typedef float4 type; };
template <> struct V4<double> { typedef double4 type; };

template <typename T> FMM_HD T rsqrt_t(T x);
template <> FMM_HD float rsqrt_t<float>(float x) {
#ifdef __CUDA_ARCH__
    return rsqrtf(x);
#else
    return 1.0f / sqrtf(x);
#endif
}
template <> FMM_HD double rsqrt_t<double>(double x) {
#ifdef __CUDA_ARCH__
    return rsqrt(x);
#else
    return 1.0 / sqrt(x);
#endif
}

}  // namespace fmmbem

// Device memory of a handle is stream-ordered (cudaMallocAsync / cudaFreeAsync on the
// handle's stream, from the device's default memory pool, which keeps freed blocks for
// reuse), so creating or destroying a handle never waits for other handles' work.
// fmm_alloc_stream() is the stream of the handle being built or torn down on this thread.
cudaStream_t& fmm_alloc_stream();
inline cudaError_t fmm_malloc_bytes(void** p, size_t bytes) { return cudaMallocAsync(p, bytes ? bytes : 16, fmm_alloc_stream()); }
template <typename P> inline cudaError_t fmm_malloc(P** p, size_t bytes) {
    return fmm_malloc_bytes(reinterpret_cast<void**>(p), bytes);
}
inline cudaError_t fmm_free(void* p) { return p ? cudaFreeAsync(p, fmm_alloc_stream()) : cudaSuccess; }

// Thread-local message of the last failure (fmmbem_last_error).
void fmmbem_set_error(const char* fmt, ...);

#define FMM_CU(call)                                                                        \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess) {                                                            \
            fmmbem_set_error("%s:%d %s: %s", __FILE__, __LINE__, #call, cudaGetErrorString(e_)); \
            return e_ == cudaErrorMemoryAllocation ? FMMBEM_ENOMEM : FMMBEM_EDEVICE;        \
        }                                                                                   \
    } while (0)

#define FMM_LAUNCHED()                                                                      \
    do {                                                                                    \
        cudaError_t e_ = cudaGetLastError();                                                \
        if (e_ != cudaSuccess) {                                                            \
            fmmbem_set_error("%s:%d launch: %s", __FILE__, __LINE__, cudaGetErrorString(e_)); \
            return FMMBEM_EDEVICE;                                                          \
        }                                                                                   \
    } while (0)

// Programmatic dependent launch. A kernel launched by launch_pdl may be scheduled while its
// predecessor in the stream drains; it calls pdl_wait() before anything else, which returns
// once that predecessor has completed and its writes are visible (at once for a plain launch).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KP, typename... A>
inline cudaError_t launch_pdl(void (*kernel)(KP...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              A&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<A&&>(args)...);
}

#define FMM_TRY(expr)              \
    do {                           \
        int r_ = (expr);           \
        if (r_ < 0) return r_;     \
    } while (0)
