// Near field of the FMM mat-vec and the direct (all-pairs) operators.
//
// P2P (Sec. 2.5): for every target leaf, the K-point sums (eq. gauss:1st-kind) over
// the Gauss points of the leaves in its P2P list, skipping the target's own panel;
// then the FP64 correction row (near-singular 20-point rule minus K-point rule, and
// the semi-analytic self integral, Sec. 2.3) is added. Sources are staged in
// shared memory per tile; each target is shared by several threads ("slices")
// that take interleaved sources, so small leaves still fill the block. Tile sums
// run in the arithmetic type and are accumulated in FP64.
//
// Direct: the same sums over every Gauss point (the Appendix mat-vec algorithm),
// for the single layers and for the double layers used by the right-hand side
// (eq. laplace_bem_dGdn) and the stresslet operator (eq. stresslet).
#include <type_traits>
#include "handle.cuh"

namespace fmmbem {

namespace {

constexpr int P2P_THREADS = 128;
constexpr int P2P_TILE = 512;

// LAP_B4: the Laplace single layer for a batch of FMMBEM_BATCH vectors ([4][N] input,
// [N][4] near-field output).
enum Op { LAP_SL = 0, LAP_DL = 1, STK_SL = 2, STK_DL = 3, LAP_B4 = 4 };

template <int OP> struct OpDof { static constexpr int v = (OP == STK_SL || OP == STK_DL) ? 3 : (OP == LAP_B4 ? 4 : 1); };

// Accumulate one source into acc (unscaled kernel sums).
//   LAP_SL : w / r
//   LAP_DL : w n.d / r^3                      (d = x - y)
//   STK_SL : f / r + d (d.f) / r^3            (f = w t)
//   STK_DL : 6 d (d.u)(e.n) / r^5, e = -d     (w folded into u)
template <typename T, int OP>
__device__ __forceinline__ void interact(T dx, T dy, T dz, const T* s, T* acc) {
    const T r2 = dx * dx + dy * dy + dz * dz;
    const T ir = rsqrt_t<T>(r2);
    if (OP == LAP_SL) {
        acc[0] += s[0] * ir;
    } else if (OP == LAP_B4) {
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[c] += s[c] * ir;
    } else if (OP == LAP_DL) {
        const T ir3 = ir * ir * ir;
        acc[0] += s[0] * (dx * s[1] + dy * s[2] + dz * s[3]) * ir3;
    } else if (OP == STK_SL) {
        const T ir3 = ir * ir * ir;
        const T df = (dx * s[0] + dy * s[1] + dz * s[2]) * ir3;
        acc[0] += s[0] * ir + dx * df;
        acc[1] += s[1] * ir + dy * df;
        acc[2] += s[2] * ir + dz * df;
    } else {
        const T ir2 = ir * ir;
        const T ir5 = ir2 * ir2 * ir;
        const T du = dx * s[0] + dy * s[1] + dz * s[2];
        const T en = -(dx * s[3] + dy * s[4] + dz * s[5]);
        const T f = T(6) * du * en * ir5;
        acc[0] += dx * f;
        acc[1] += dy * f;
        acc[2] += dz * f;
    }
}

template <int OP> struct SrcWidth {
    static constexpr int v = (OP == LAP_SL) ? 1 : (OP == LAP_DL || OP == LAP_B4 ? 4 : (OP == STK_SL ? 3 : 6));
};

// Stage source q (global Gauss-point index) into shared memory: position + strength terms.
// bstride: LAP_B4's distance between the batch's vectors in xs (N).
template <typename T, int OP>
__device__ __forceinline__ void stage(int g, const typename V4<T>::type* src, const double* xs, const double4* nrm, int K,
                                      T* spos, T* sval, int slot, int64_t bstride = 0) {
    const auto y = src[g];
    const int pj = g / K;
    spos[3 * slot] = y.x;
    spos[3 * slot + 1] = y.y;
    spos[3 * slot + 2] = y.z;
    constexpr int W = SrcWidth<OP>::v;
    T* v = sval + W * slot;
    const double w = (double)y.w;
    if (OP == LAP_SL) {
        v[0] = T(w * xs[pj]);
    } else if (OP == LAP_B4) {
#pragma unroll
        for (int c = 0; c < 4; ++c) v[c] = T(w * xs[c * bstride + pj]);
    } else if (OP == LAP_DL) {
        const double4 n = nrm[pj];
        v[0] = T(w * xs[pj]);
        v[1] = T(n.x); v[2] = T(n.y); v[3] = T(n.z);
    } else if (OP == STK_SL) {
        v[0] = T(w * xs[3 * pj]); v[1] = T(w * xs[3 * pj + 1]); v[2] = T(w * xs[3 * pj + 2]);
    } else {
        const double4 n = nrm[pj];
        v[0] = T(w * xs[3 * pj]); v[1] = T(w * xs[3 * pj + 1]); v[2] = T(w * xs[3 * pj + 2]);
        v[3] = T(n.x); v[4] = T(n.y); v[5] = T(n.z);
    }
}

// Add the correction row of target i: sum_e C_e x_{col_e} (1x1 or 3x3 blocks), FP64. DOF 4:
// one scalar entry applied to each vector of a batch (vector c at xs + c * bstride).
template <int DOF>
__device__ __forceinline__ void add_correction(int i, const int* cptr, const int* ccol, const double* cval,
                                               const double* xs, double* out, int64_t bstride = 0) {
    for (int e = cptr[i]; e < cptr[i + 1]; ++e) {
        const int j = ccol[e];
        if (DOF == 1) {
            out[0] += cval[e] * xs[j];
        } else if (DOF == 4) {
            const double c0 = cval[e];
#pragma unroll
            for (int c = 0; c < 4; ++c) out[c] += c0 * xs[c * bstride + j];
        } else {
            const double* B = cval + 9 * (int64_t)e;
            const double x0 = xs[3 * j], x1 = xs[3 * j + 1], x2 = xs[3 * j + 2];
            out[0] += B[0] * x0 + B[1] * x1 + B[2] * x2;
            out[1] += B[3] * x0 + B[4] * x1 + B[5] * x2;
            out[2] += B[6] * x0 + B[7] * x1 + B[8] * x2;
        }
    }
}

// The correction rows of every target as their own pass of the mixed-precision near field:
// yc[DOF i + a] = sum_e (C_e x_{col_e})_a with the FP32-rounded table and x rounded to FP32
// (products and sums in FP32, like the P2P sums they are added to), written in FP64 in the
// layout of the near-field output (DOF 4: a batch, vector c of the input at xs + c * bstride;
// gridDim.y: the vectors of a Stokes batch, xsys apart). CR_LANES lanes share a row and each
// takes U of its entries per pass (8; 4 for the 3x3 blocks) with every load issued before the
// first product, so a row of up to CR_LANES * U entries costs three dependent loads (row
// start, entry, input); a shuffle reduction adds the lanes' sums.
constexpr int CR_LANES = 4;
template <int DOF> struct CorrUnroll { static constexpr int U = DOF == 3 ? 4 : 8; };

template <int DOF>
__global__ void k_corr_rows(int n, const int* cptr, const int* ccol, const float* cval, const double* xs, double* yc,
                            int64_t bstride, int64_t xsys) {
    constexpr int U = CorrUnroll<DOF>::U, NV = DOF == 3 ? 9 : 1;
    xs += blockIdx.y * xsys;
    yc += blockIdx.y * xsys;
    const int i = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / CR_LANES);
    const int sub = threadIdx.x % CR_LANES;
    float out[DOF];
#pragma unroll
    for (int a = 0; a < DOF; ++a) out[a] = 0.f;
    if (i < n) {
        const int e1 = cptr[i + 1];
        for (int eb = cptr[i] + sub; eb < e1; eb += CR_LANES * U) {
            int j[U];
            float c[U][NV];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int e = eb + CR_LANES * u;
                j[u] = e < e1 ? ccol[e] : -1;
#pragma unroll
                for (int v = 0; v < NV; ++v) c[u][v] = e < e1 ? cval[(int64_t)NV * e + v] : 0.f;
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (j[u] < 0) continue;
                if (DOF == 1) {
                    out[0] = fmaf(c[u][0], (float)xs[j[u]], out[0]);
                } else if (DOF == 4) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) out[q] = fmaf(c[u][0], (float)xs[q * bstride + j[u]], out[q]);
                } else {
                    const float x0 = (float)xs[3 * j[u]], x1 = (float)xs[3 * j[u] + 1], x2 = (float)xs[3 * j[u] + 2];
#pragma unroll
                    for (int a = 0; a < 3; ++a)
                        out[a] = fmaf(c[u][3 * a], x0, fmaf(c[u][3 * a + 1], x1, fmaf(c[u][3 * a + 2], x2, out[a])));
                }
            }
        }
    }
    // every lane of the warp takes part (blockDim is a multiple of 32); rows past n add zeros
#pragma unroll
    for (int o = CR_LANES / 2; o >= 1; o >>= 1)
#pragma unroll
        for (int a = 0; a < DOF; ++a) out[a] += __shfl_xor_sync(0xffffffffu, out[a], o, CR_LANES);
    if (i < n && sub == 0)
#pragma unroll
        for (int a = 0; a < DOF; ++a) yc[(int64_t)DOF * i + a] = (double)out[a];
}

// Near field: one block per target leaf. In FP32 the operands are leaf-relative:
// target offsets from its leaf centre, source offsets from theirs, and the
// leaf-to-leaf shift (FP64 difference of the centres) is added while staging, so
// close pairs keep their relative precision. Partial sums run over at most 32
// sources in the arithmetic type before they are added to the FP64 accumulator.
constexpr int P2P_FLUSH = 32;

template <typename T, int OP>
__global__ void __launch_bounds__(P2P_THREADS) k_p2p(const int* leaves, const double4* cs, const int2* range,
                                                     const int* pptr, const int* psrc, const typename V4<T>::type* src,
                                                     const typename V4<T>::type* tgt, bool relative, const double* xs,
                                                     const double4* nrm, int K, const int* cptr, const int* ccol,
                                                     const double* cval, double* ynear, int64_t bstride) {
    constexpr int DOF = OpDof<OP>::v;
    constexpr int W = SrcWidth<OP>::v;
    __shared__ T spos[3 * P2P_TILE];
    __shared__ T sval[W * P2P_TILE];
    __shared__ double sred[P2P_THREADS * DOF];
    const int cell = leaves[blockIdx.x];
    const int2 r = range[cell];
    const double4 ccell = cs[cell];
    const int tid = threadIdx.x;
    for (int tb = r.x; tb < r.y; tb += P2P_THREADS) {
        const int chunk = min(P2P_THREADS, r.y - tb);
        const int nsl = max(1, P2P_THREADS / chunk);
        const int ti = tid % chunk, sl = tid / chunk;
        const bool active = sl < nsl;
        const int i = tb + ti;
        const auto xi = tgt[i];
        const T tx = xi.x, ty = xi.y, tz = xi.z;
        double acc[DOF];
#pragma unroll
        for (int a = 0; a < DOF; ++a) acc[a] = 0.0;
        for (int e = pptr[cell]; e < pptr[cell + 1]; ++e) {
            const int sc = psrc[e];
            const int2 sr = range[sc];
            const int g0 = sr.x * K, g1 = sr.y * K;
            const bool self_leaf = (sc == cell);
            T shx = 0, shy = 0, shz = 0;
            if (relative) {
                const double4 cc = cs[sc];
                shx = T(cc.x - ccell.x);
                shy = T(cc.y - ccell.y);
                shz = T(cc.z - ccell.z);
            }
            for (int gb = g0; gb < g1; gb += P2P_TILE) {
                const int nt = min(P2P_TILE, g1 - gb);
                __syncthreads();
                for (int q = tid; q < nt; q += P2P_THREADS) {
                    stage<T, OP>(gb + q, src, xs, nrm, K, spos, sval, q, bstride);
                    spos[3 * q] += shx;
                    spos[3 * q + 1] += shy;
                    spos[3 * q + 2] += shz;
                }
                __syncthreads();
                if (active) {
                    const int own0 = self_leaf ? i * K - gb : -(1 << 30);  // the target's own Gauss points are skipped
                    for (int q0 = sl; q0 < nt; q0 += P2P_FLUSH * nsl) {
                        const int q1 = min(nt, q0 + P2P_FLUSH * nsl);
                        T part[DOF];
#pragma unroll
                        for (int a = 0; a < DOF; ++a) part[a] = T(0);
                        if (!self_leaf) {
                            for (int q = q0; q < q1; q += nsl)
                                interact<T, OP>(tx - spos[3 * q], ty - spos[3 * q + 1], tz - spos[3 * q + 2], sval + W * q, part);
                        } else {
                            for (int q = q0; q < q1; q += nsl) {
                                if ((unsigned)(q - own0) < (unsigned)K) continue;
                                interact<T, OP>(tx - spos[3 * q], ty - spos[3 * q + 1], tz - spos[3 * q + 2], sval + W * q, part);
                            }
                        }
#pragma unroll
                        for (int a = 0; a < DOF; ++a) acc[a] += (double)part[a];
                    }
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int a = 0; a < DOF; ++a) sred[tid * DOF + a] = active ? acc[a] : 0.0;
        __syncthreads();
        if (sl == 0 && ti < chunk) {
            double out[DOF];
#pragma unroll
            for (int a = 0; a < DOF; ++a) out[a] = 0.0;
            for (int s = 0; s < nsl; ++s)
#pragma unroll
                for (int a = 0; a < DOF; ++a) out[a] += sred[(s * chunk + ti) * DOF + a];
            add_correction<DOF>(i, cptr, ccol, cval, xs, out, bstride);
#pragma unroll
            for (int a = 0; a < DOF; ++a) ynear[(int64_t)DOF * i + a] = out[a];
        }
    }
}

// Laplace single layer in FP32, the near-field pass of every mixed-precision mat-vec.
// Per mat-vec each Gauss point is packed once as (leaf-relative position, w = q_k S_j x_j)
// (k_pack_sources). A block takes one target leaf; each lane holds TPL targets in
// registers (lane l: targets l, l+32, ...), the four warps split every staged source
// tile into contiguous quarters, so one 128-bit broadcast shared load feeds TPL
// interactions. FP32 partial sums over 32 sources are added to FP64 accumulators.
constexpr int LAP_TILE = 1024;

// One thread per panel converts x_j to FP32 once and writes its K Gauss points as
// (leaf-relative position, q_k S_j x_j): FP64 throughput is scarce on this GPU, so the
// conversion is done once per panel, not per Gauss point or per pass.
__global__ void k_pack_sources(const float4* src_rel, const double* xs, int K, int64_t n, float4* out) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= n) return;
    const float x = (float)xs[j];
    for (int k = 0; k < K; ++k) {
        const float4 y = src_rel[j * K + k];
        out[j * K + k] = make_float4(y.x, y.y, y.z, y.w * x);
    }
}

__device__ __forceinline__ float rsqrt_approx(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Compensated (Kahan) FP32 accumulation: hi + lo carries the sum of the partials to
// about FP64 accuracy without FP64 arithmetic in the interaction loop.
__device__ __forceinline__ void kahan_add(float& hi, float& lo, float v) {
    const float y = v - lo;
    const float t = hi + y;
    lo = (t - hi) - y;
    hi = t;
}

// Each source of a staged tile carries its global Gauss-point index in .w of a
// companion int array only for the target leaf's own sources (the own panel is
// skipped there); other leaves are merged into shared tiles of up to LAP_TILE
// sources, so one barrier pair serves many small leaves. Two partial sums per
// target alternate between sources to break the FMA dependency chain.
template <int TPL>
__device__ __forceinline__ void lap_tile(const float4* s, int q0, int q1, const float* tx, const float* ty,
                                         const float* tz, float* hi, float* lo) {
    for (int qb = q0; qb < q1; qb += 64) {
        const int qe = min(q1, qb + 64);
        float pa[TPL], pb[TPL];
#pragma unroll
        for (int t = 0; t < TPL; ++t) { pa[t] = 0.f; pb[t] = 0.f; }
        int q = qb;
        for (; q + 1 < qe; q += 2) {
            const float4 u = s[q], v = s[q + 1];
#pragma unroll
            for (int t = 0; t < TPL; ++t) {
                const float ux = tx[t] - u.x, uy = ty[t] - u.y, uz = tz[t] - u.z;
                const float vx = tx[t] - v.x, vy = ty[t] - v.y, vz = tz[t] - v.z;
                pa[t] = fmaf(u.w, rsqrt_approx(fmaf(ux, ux, fmaf(uy, uy, uz * uz))), pa[t]);
                pb[t] = fmaf(v.w, rsqrt_approx(fmaf(vx, vx, fmaf(vy, vy, vz * vz))), pb[t]);
            }
        }
        if (q < qe) {
            const float4 u = s[q];
#pragma unroll
            for (int t = 0; t < TPL; ++t) {
                const float ux = tx[t] - u.x, uy = ty[t] - u.y, uz = tz[t] - u.z;
                pa[t] = fmaf(u.w, rsqrt_approx(fmaf(ux, ux, fmaf(uy, uy, uz * uz))), pa[t]);
            }
        }
#pragma unroll
        for (int t = 0; t < TPL; ++t) kahan_add(hi[t], lo[t], pa[t] + pb[t]);
    }
}

template <int TPL>
__device__ __forceinline__ void lap_tile_self(const float4* s, int q0, int q1, int gb, const int* own, int K,
                                              const float* tx, const float* ty, const float* tz, float* hi,
                                              float* lo) {
    for (int qb = q0; qb < q1; qb += 32) {
        const int qe = min(q1, qb + 32);
        float part[TPL];
#pragma unroll
        for (int t = 0; t < TPL; ++t) part[t] = 0.f;
        for (int q = qb; q < qe; ++q) {
            const float4 v = s[q];
#pragma unroll
            for (int t = 0; t < TPL; ++t) {
                if ((unsigned)(gb + q - own[t]) < (unsigned)K) continue;
                const float dx = tx[t] - v.x, dy = ty[t] - v.y, dz = tz[t] - v.z;
                part[t] = fmaf(v.w, rsqrt_approx(fmaf(dx, dx, fmaf(dy, dy, dz * dz))), part[t]);
            }
        }
#pragma unroll
        for (int t = 0; t < TPL; ++t) kahan_add(hi[t], lo[t], part[t]);
    }
}

// Per target leaf the sources of every other leaf of its P2P list form one
// concatenated stream; the static per-pair records (leaf-to-leaf FP32 shift, first
// Gauss point, offset in the stream) are loaded into shared memory once, and each
// slot of a staged tile finds its pair by a binary search over the offsets, so
// staging runs in parallel with no dependent global-load chains.
constexpr int LAP_MAXE = 512;

template <int TPL>
__global__ void __launch_bounds__(128) k_p2p_lap(const int* leaves, const int2* range, const int* pptr,
                                                 const float4* prec, const int* poff, const int* plen,
                                                 const float4* srcw, const float4* tgt, int K, const int* cptr,
                                                 const int* ccol, const double* cval, const double* xs,
                                                 double* ynear) {
    __shared__ float4 sS[LAP_TILE];
    __shared__ float4 sRec[LAP_MAXE];
    __shared__ int sOff[LAP_MAXE];
    __shared__ double sred[4 * 128];
    const int cell = leaves[blockIdx.x];
    const int2 r = range[cell];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int e0 = pptr[cell], e1 = pptr[cell + 1];
    const int total = plen[cell];
    for (int tb = r.x; tb < r.y; tb += 32 * TPL) {
        const int nt = min(32 * TPL, r.y - tb);
        float tx[TPL], ty[TPL], tz[TPL], hi[TPL], lo[TPL];
        int own[TPL];
#pragma unroll
        for (int t = 0; t < TPL; ++t) {
            const int li = lane + 32 * t;
            const float4 x = li < nt ? tgt[tb + li] : make_float4(1e30f, 0.f, 0.f, 0.f);
            tx[t] = x.x; ty[t] = x.y; tz[t] = x.z;
            own[t] = (tb + li) * K;
            hi[t] = 0.f;
            lo[t] = 0.f;
        }
        // the target leaf's own sources, with the own-panel skip
        {
            const int g0 = r.x * K, g1 = r.y * K;
            for (int gb = g0; gb < g1; gb += LAP_TILE) {
                const int n = min(LAP_TILE, g1 - gb);
                __syncthreads();
                for (int q = threadIdx.x; q < n; q += blockDim.x) sS[q] = srcw[gb + q];
                __syncthreads();
                const int per = (n + 3) >> 2;
                const int q0 = min(n, warp * per), q1 = min(n, q0 + per);
                lap_tile_self<TPL>(sS, q0, q1, gb, own, K, tx, ty, tz, hi, lo);
            }
        }
        // the other leaves, as one stream of Gauss points
        for (int eb = e0; eb < e1; eb += LAP_MAXE) {
            const int ne = min(LAP_MAXE, e1 - eb);
            __syncthreads();
            for (int j = threadIdx.x; j < ne; j += blockDim.x) {
                sRec[j] = prec[eb + j];
                sOff[j] = poff[eb + j];
            }
            __syncthreads();
            const int s_beg = sOff[0];
            const int s_end = (eb + LAP_MAXE < e1) ? poff[eb + LAP_MAXE] : total;
            for (int s0 = s_beg; s0 < s_end; s0 += LAP_TILE) {
                const int n = min(LAP_TILE, s_end - s0);
                for (int q = threadIdx.x; q < n; q += blockDim.x) {
                    const int sp = s0 + q;
                    int lo_i = 0, hi_i = ne;  // last j with sOff[j] <= sp
                    while (hi_i - lo_i > 1) {
                        const int mid = (lo_i + hi_i) >> 1;
                        if (sOff[mid] <= sp) lo_i = mid; else hi_i = mid;
                    }
                    const float4 rc = sRec[lo_i];
                    float4 v = srcw[__float_as_int(rc.w) + (sp - sOff[lo_i])];
                    v.x += rc.x; v.y += rc.y; v.z += rc.z;
                    sS[q] = v;
                }
                __syncthreads();
                const int per = (n + 3) >> 2;
                const int q0 = min(n, warp * per), q1 = min(n, q0 + per);
                lap_tile<TPL>(sS, q0, q1, tx, ty, tz, hi, lo);
                __syncthreads();
            }
        }
        __syncthreads();
#pragma unroll
        for (int t = 0; t < TPL; ++t) sred[warp * 128 + lane + 32 * t] = (double)hi[t] - (double)lo[t];
        __syncthreads();
        if (warp == 0) {
#pragma unroll
            for (int t = 0; t < TPL; ++t) {
                const int li = lane + 32 * t;
                if (li >= nt) continue;
                double out = sred[li] + sred[128 + li] + sred[256 + li] + sred[384 + li];
                add_correction<1>(tb + li, cptr, ccol, cval, xs, &out);
                ynear[tb + li] = out;
            }
        }
        __syncthreads();
    }
}

// Sliced variant: thread tid of the block takes target tid % nt and source slice
// tid / nt (S = 128 / nt slices), so small leaves still keep every lane busy. Each
// slice walks whole P2P pairs (pair e goes to slice (e - e0) % S) and reads the Gauss
// points straight through L1: all lanes of a slice read the same address, so every
// load is a broadcast. No shared staging, no barriers inside the sums.
__device__ __forceinline__ float lap_pair(float px, float py, float pz, float4 u) {
    const float ux = px - u.x, uy = py - u.y, uz = pz - u.z;
    return u.w * rsqrt_approx(fmaf(ux, ux, fmaf(uy, uy, uz * uz)));
}

// One pair's Gauss points for one target: loads are issued 8 at a time ahead of the
// arithmetic (8 independent 128-bit requests in flight per thread), partial sums of
// at most 64 sources are folded into the compensated accumulator.
__device__ __forceinline__ void lap_run(const float4* __restrict__ srcw, int g0, int n, float shx, float shy,
                                        float shz, float tx, float ty, float tz, int skip0, int K, float& hi,
                                        float& lo) {
    const float px = tx - shx, py = ty - shy, pz = tz - shz;
    const float4* p = srcw + g0;
    for (int qb = 0; qb < n; qb += 64) {
        const int qe = min(n, qb + 64);
        float pa = 0.f, pb = 0.f;
        int q = qb;
        if (skip0 < 0) {
            for (; q + 7 < qe; q += 8) {
                float4 u[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) u[j] = __ldg(p + q + j);
#pragma unroll
                for (int j = 0; j < 8; j += 2) {
                    pa += lap_pair(px, py, pz, u[j]);
                    pb += lap_pair(px, py, pz, u[j + 1]);
                }
            }
            for (; q + 1 < qe; q += 2) {
                const float4 u = __ldg(p + q), v = __ldg(p + q + 1);
                pa += lap_pair(px, py, pz, u);
                pb += lap_pair(px, py, pz, v);
            }
            if (q < qe) pa += lap_pair(px, py, pz, __ldg(p + q));
            q = qe;
        }
        for (; q < qe; ++q) {
            if ((unsigned)(q - skip0) < (unsigned)K) continue;
            pa += lap_pair(px, py, pz, __ldg(p + q));
        }
        kahan_add(hi, lo, pa + pb);
    }
}

__global__ void __launch_bounds__(128) k_p2p_lap_sliced(const int* leaves, const int2* range, const int* pptr,
                                                        const int* psrc, const float4* prec, const float4* srcw,
                                                        const float4* tgt, int K, const int* cptr, const int* ccol,
                                                        const double* cval, const double* xs, double* ynear) {
    __shared__ double sred[128];
    const int cell = leaves[blockIdx.x];
    const int2 r = range[cell];
    const int e0 = pptr[cell], e1 = pptr[cell + 1];
    const int tid = threadIdx.x;
    for (int tb = r.x; tb < r.y; tb += 128) {
        const int nt = min(128, r.y - tb);
        const int S = 128 / nt;
        const int t = tid % nt, slice = tid / nt;
        const bool active = slice < S;
        float hi = 0.f, lo = 0.f;
        if (active) {
            const float4 x = tgt[tb + t];
            for (int e = e0 + slice; e < e1; e += S) {
                const int sc = psrc[e];
                const float4 rc = prec[e];
                const int2 sr = range[sc];
                const int g0 = __float_as_int(rc.w), n = K * (sr.y - sr.x);
                const int skip0 = (sc == cell) ? (tb + t) * K - g0 : -(1 << 30);
                lap_run(srcw, g0, n, rc.x, rc.y, rc.z, x.x, x.y, x.z, skip0, K, hi, lo);
            }
        }
        __syncthreads();
        sred[tid] = active ? (double)hi - (double)lo : 0.0;
        __syncthreads();
        if (slice == 0) {
            double out = 0.0;
            for (int sl = 0; sl < S; ++sl) out += sred[sl * nt + t];
            add_correction<1>(tb + t, cptr, ccol, cval, xs, &out);
            ynear[tb + t] = out;
        }
        __syncthreads();
    }
}

// Bulk-copy variant: the Gauss points of each P2P pair are one contiguous range, so a
// stage of up to BK_TILE sources is filled by one cp.async.bulk per pair (issued by
// thread 0, completing on the stage's mbarrier) while the block computes the other
// stage. Within a stage, pair j goes to slice j % S; every thread of a slice reads the
// same shared-memory source (broadcast). Thread = (target, slice) as in the sliced
// variant.
constexpr int BK_TILE = 1024;
constexpr int BK_MAXP = 64;  // pairs per stage

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool bk_wait(uint32_t mbar, uint32_t parity) {
    for (uint32_t it = 0; it < (1u << 24); ++it) {
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

// Warp 0: arm stage buffer `buf` with stage k's byte count, issue one bulk copy per
// pair, and leave the pairs' records (shift, stage offset, count, own-leaf flag) in
// shared memory for the consumers (visible to them after the next block barrier).
__device__ __forceinline__ void bk_issue(int k, int s1, int e1, int cell, const int* sfirst, const int* sbytes,
                                         const int* ptoff, const int* pcnt, const int* psrc, const float4* prec,
                                         const float4* srcw, float4* dst, float4* rec, int2* info, int* np_out,
                                         uint32_t bar, int lane) {
    const int fa = sfirst[k], fb = (k + 1 < s1) ? sfirst[k + 1] : e1;
    if (lane == 0) {
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"((uint32_t)sbytes[k])
                     : "memory");
        *np_out = fb - fa;
    }
    __syncwarp();
    for (int e = fa + lane; e < fb; e += 32) {
        const float4 rc = prec[e];
        const int to = ptoff[e], n = pcnt[e];
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                smem_addr(dst + to)),
            "l"(srcw + __float_as_int(rc.w)), "r"((uint32_t)n * 16u), "r"(bar)
            : "memory");
        rec[e - fa] = rc;
        info[e - fa] = make_int2(to | (psrc[e] == cell ? (1 << 30) : 0), n);
    }
}

// Stage plans are static (create time): stage k of a target leaf covers pairs
// [first_k, first_{k+1}) with at most BK_TILE Gauss points; pair e sits at offset
// toff[e] of its stage and holds cnt[e] points. Warp 0 arms the stage barrier with the
// stage's byte count, then its lanes issue one bulk copy per pair in parallel.
__global__ void __launch_bounds__(128) k_p2p_lap_bulk(const int* leaves, const int2* range, const int* pptr,
                                                      const int* psrc, const float4* prec, const int* pcnt,
                                                      const int* ptoff, const int* sptr, const int* sfirst,
                                                      const int* sbytes, const float4* srcw, const float4* tgt, int K,
                                                      const int* cptr, const int* ccol, const double* cval,
                                                      const double* xs, double* ynear, int* err) {
    __shared__ __align__(128) float4 sS[2][BK_TILE];
    __shared__ float4 sRec[2][BK_MAXP];
    __shared__ int2 sInfo[2][BK_MAXP];
    __shared__ int sNp[2];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ double sred[128];
    const int cell = leaves[blockIdx.x];
    const int2 r = range[cell];
    const int e1 = pptr[cell + 1];
    const int s0 = sptr[cell], s1 = sptr[cell + 1];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        for (int i = 0; i < 2; ++i) asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&bar[i])), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    __syncthreads();
    int use0 = 0, use1 = 0;  // completed phases of each stage barrier
    bool ok = true;
    for (int tb = r.x; tb < r.y; tb += 128) {
        const int nt = min(128, r.y - tb);
        const int S = 128 / nt;
        const int t = tid % nt, slice = tid / nt;
        const bool active = slice < S;
        float tx = 0.f, ty = 0.f, tz = 0.f;
        if (active) {
            const float4 x = tgt[tb + t];
            tx = x.x; ty = x.y; tz = x.z;
        }
        const int own = (tb + t) * K;
        float hi = 0.f, lo = 0.f;
        if (warp == 0 && s0 < s1)
            bk_issue(s0, s1, e1, cell, sfirst, sbytes, ptoff, pcnt, psrc, prec, srcw, sS[0], sRec[0], sInfo[0], &sNp[0],
                     smem_addr(&bar[0]), lane);
        __syncthreads();
        for (int k = s0; k < s1; ++k) {
            const int buf = (k - s0) & 1;
            if (warp == 0 && k + 1 < s1)  // the other buffer was released by the previous barrier
                bk_issue(k + 1, s1, e1, cell, sfirst, sbytes, ptoff, pcnt, psrc, prec, srcw, sS[buf ^ 1], sRec[buf ^ 1],
                         sInfo[buf ^ 1], &sNp[buf ^ 1], smem_addr(&bar[buf ^ 1]), lane);
            const uint32_t par = (uint32_t)((buf ? use1 : use0) & 1);
            if (ok && !bk_wait(smem_addr(&bar[buf]), par)) { atomicExch(err, 4); ok = false; }
            if (buf) ++use1; else ++use0;
            if (active && ok) {
                const int np = sNp[buf];
                for (int j = slice; j < np; j += S) {
                    const float4 rc = sRec[buf][j];
                    const int2 in = sInfo[buf][j];
                    const int to = in.x & ((1 << 30) - 1), cnt = in.y;
                    const float px = tx - rc.x, py = ty - rc.y, pz = tz - rc.z;
                    const float4* sp = &sS[buf][to];
                    const int skip = (in.x >> 30) ? own - __float_as_int(rc.w) : -(1 << 30);
                    for (int qb = 0; qb < cnt; qb += 64) {
                        const int qe = min(cnt, qb + 64);
                        float pa = 0.f, pb = 0.f;
                        int q = qb;
                        if (skip < 0) {
                            for (; q + 1 < qe; q += 2) {
                                pa += lap_pair(px, py, pz, sp[q]);
                                pb += lap_pair(px, py, pz, sp[q + 1]);
                            }
                        }
                        for (; q < qe; ++q) {
                            if ((unsigned)(q - skip) < (unsigned)K) continue;
                            pa += lap_pair(px, py, pz, sp[q]);
                        }
                        kahan_add(hi, lo, pa + pb);
                    }
                }
            }
            __syncthreads();
        }
        sred[tid] = active ? (double)hi - (double)lo : 0.0;
        __syncthreads();
        if (slice == 0) {
            double out = 0.0;
            for (int sl = 0; sl < S; ++sl) out += sred[sl * nt + t];
            add_correction<1>(tb + t, cptr, ccol, cval, xs, &out);
            ynear[tb + t] = out;
        }
        __syncthreads();
    }
}

// Source-lane variant: one block of PS_WARPS warps per work item, a chunk of at most
// PS_TMAX targets of one leaf (items in order of decreasing work).
// - The leaf's source stream is its own Gauss points (own panel skipped), then those of
//   every other leaf of its P2P list.
// - The stream is cut into rounds of 128 positions; round r goes to warp r mod
//   PS_WARPS, and each lane takes four positions of the round, so lanes stay full
//   whatever the leaf sizes.
// - Each lane loops over the leaf's targets (shared memory, broadcast reads) with one
//   FP32 accumulator per target in registers.
// - Every PS_FOLD rounds the accumulators are folded into per-lane compensated (hi, lo)
//   sums in shared memory.
// - At the end lane i of every warp adds target i's partials of the warp's lanes, then
//   thread i adds the warp sums (both compensated), applies the FP64 correction row and
//   writes the result.
constexpr int PS_WARPS = 4;
constexpr int PS_TMAX = P2P_SRC_TMAX;  // targets per block (a leaf's targets are split into chunks of at most this)
constexpr int PS_EMAX = 64;   // pair records per shared-memory chunk
constexpr int PS_FOLD = 8;    // rounds between folds (32 terms per lane and target)
static_assert(PS_TMAX <= 32, "the epilogue gives each target of a block one lane per warp");

// Positions base + 32 h + lane (h < NS) of a warp's source stream (woff: the stream offsets of
// the staged pair records, woff[ne] = s_end): rec[h] = the record holding position h (-1 past
// the stream end) and g[h] = the position's offset inside that record's sources. The lane's
// cursor only moves forward; the caller issues the loads.
template <int NS>
__device__ __forceinline__ void stream_slots(int base, int lane, int s_end, const int* woff, int& cur, int (&rec)[NS],
                                             int (&g)[NS]) {
#pragma unroll
    for (int h = 0; h < NS; ++h) {
        const int pos = base + 32 * h + lane;
        rec[h] = -1;
        g[h] = 0;
        if (pos < s_end) {
            while (woff[cur + 1] <= pos) ++cur;
            rec[h] = cur;
            g[h] = pos - woff[cur];
        }
    }
}

// Pair records are staged per warp, so the warps of a block never wait for one another
// between the target load and the epilogue. Targets are stored in pairs: (x_a, x_b, y_a, y_b)
// and (z_a, z_b).
struct PsShared {
    float4 txy[PS_TMAX / 2];
    float2 tz[PS_TMAX / 2];
    float2 hl[PS_WARPS][PS_TMAX][32];
    float4 rec[PS_WARPS][PS_EMAX];
    int off[PS_WARPS][PS_EMAX + 1];
    float2 wsum[PS_WARPS][PS_TMAX];
};
constexpr int PS_GRP = 4;  // targets per group of the unrolled target loop (a multiple of the pair)
static_assert(PS_TMAX % PS_GRP == 0 && PS_GRP % 2 == 0, "targets are processed in groups of whole pairs");

// A source of the round, each component repeated in both halves.
struct PsSrc {
    f32x2 x, y, z, w;
};
__device__ __forceinline__ PsSrc ps_src(float4 u) {
    return {f2_pack(u.x, u.x), f2_pack(u.y, u.y), f2_pack(u.z, u.z), f2_pack(u.w, u.w)};
}

// acc[j] holds the running sums of targets 2j and 2j + 1.
__device__ __forceinline__ void ps_fold(f32x2* acc, float2* hl, int ntb, int lane) {
#pragma unroll
    for (int j = 0; j < PS_TMAX / 2; ++j) {
        float a0, a1;
        f2_unpack(acc[j], a0, a1);
        if (2 * j < ntb) {
            float2 v = hl[2 * j * 32 + lane];
            kahan_add(v.x, v.y, a0);
            hl[2 * j * 32 + lane] = v;
        }
        if (2 * j + 1 < ntb) {
            float2 v = hl[(2 * j + 1) * 32 + lane];
            kahan_add(v.x, v.y, a1);
            hl[(2 * j + 1) * 32 + lane] = v;
        }
        acc[j] = 0ull;
        asm volatile("" ::: "memory");
    }
}

// The target loop runs over groups of PS_GRP targets (whole pairs), fully unrolled (so the
// accumulators stay in registers) with one uniform branch per group; the target count of a
// pass is padded to a multiple of PS_GRP with far-away dummy targets whose sums are never read.
// Each lane holds PS_SRC sources per round; per source and target pair: 3 paired
// subtractions, the squared distances (paired mul + 2 paired fma), two rsqrt and one paired
// fma into the accumulators.
constexpr int PS_SRC = 4;

__device__ __forceinline__ void ps_round(const float4* sXY, const float2* sZ, int ntb, const PsSrc (&u)[PS_SRC],
                                         f32x2* acc) {
#pragma unroll
    for (int g = 0; g < PS_TMAX; g += PS_GRP) {
        if (g < ntb) {
#pragma unroll
            for (int j = g / 2; j < (g + PS_GRP) / 2; ++j) {
                const float4 A = sXY[j];
                const float2 B = sZ[j];
                const f32x2 tx = f2_pack(A.x, A.y), ty = f2_pack(A.z, A.w), tz = f2_pack(B.x, B.y);
                f32x2 a = acc[j];
#pragma unroll
                for (int h = 0; h < PS_SRC; ++h) {
                    const f32x2 dx = f2_sub(tx, u[h].x), dy = f2_sub(ty, u[h].y), dz = f2_sub(tz, u[h].z);
                    float r0, r1;
                    f2_unpack(f2_fma(dx, dx, f2_fma(dy, dy, f2_mul(dz, dz))), r0, r1);
                    a = f2_fma(u[h].w, f2_pack(rsqrt_approx(r0), rsqrt_approx(r1)), a);
                }
                acc[j] = a;
            }
        }
        asm volatile("" ::: "memory");  // keeps the next group's target loads from being hoisted (register pressure)
    }
}

// The own leaf: a source on the target's own panel contributes nothing.
__device__ __forceinline__ void ps_round_self(const float4* sXY, const float2* sZ, int ntb, int tb,
                                              const PsSrc (&u)[PS_SRC], const int (&gp)[PS_SRC], f32x2* acc) {
#pragma unroll
    for (int g = 0; g < PS_TMAX; g += PS_GRP) {
        if (g < ntb) {
#pragma unroll
            for (int j = g / 2; j < (g + PS_GRP) / 2; ++j) {
                const float4 A = sXY[j];
                const float2 B = sZ[j];
                const f32x2 tx = f2_pack(A.x, A.y), ty = f2_pack(A.z, A.w), tz = f2_pack(B.x, B.y);
                const int own = tb + 2 * j;
                f32x2 a = acc[j];
#pragma unroll
                for (int h = 0; h < PS_SRC; ++h) {
                    const f32x2 dx = f2_sub(tx, u[h].x), dy = f2_sub(ty, u[h].y), dz = f2_sub(tz, u[h].z);
                    float r0, r1;
                    f2_unpack(f2_fma(dx, dx, f2_fma(dy, dy, f2_mul(dz, dz))), r0, r1);
                    const bool s0 = gp[h] == own, s1 = gp[h] == own + 1;
                    const float i0 = rsqrt_approx(s0 ? 1.f : r0), i1 = rsqrt_approx(s1 ? 1.f : r1);
                    a = f2_fma(u[h].w, f2_pack(s0 ? 0.f : i0, s1 ? 0.f : i1), a);
                }
                acc[j] = a;
            }
        }
        asm volatile("" ::: "memory");
    }
}

__global__ void __launch_bounds__(32 * PS_WARPS, 7) k_p2p_lap_src(const int4* items, const int2* range, const int* pptr,
                                                                 const float4* prec, const int* poff, const int* plen,
                                                                 const float4* srcw, const float4* tgt, int K,
                                                                 const double* yc, double* ynear) {
    __shared__ PsShared sh;
    constexpr int RND = 32 * PS_SRC;  // stream positions per warp round
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int4 item = items[blockIdx.x];
    const int cell = item.x;
    const int2 r = range[cell];
    const int e0 = pptr[cell], e1 = pptr[cell + 1];
    const int total = plen[cell];
    float2* sHL = &sh.hl[warp][0][0];
    const float4 far_src = make_float4(1e18f, 0.f, 0.f, 0.f);  // padding: contributes 0 * rsqrt(1e36)
    {
        const int tb = item.y;
        const int ntb = item.z;
        __syncthreads();
        for (int i = threadIdx.x; i < (ntb + PS_GRP - 1) / PS_GRP * PS_GRP; i += blockDim.x) {
            const float4 x = i < ntb ? tgt[tb + i] : make_float4(1e18f, 1e18f, 1e18f, 0.f);
            float* xy = reinterpret_cast<float*>(&sh.txy[i >> 1]);
            float* z = reinterpret_cast<float*>(&sh.tz[i >> 1]);
            xy[i & 1] = x.x;
            xy[2 + (i & 1)] = x.y;
            z[i & 1] = x.z;
        }
        for (int i = 0; i < ntb; ++i) sHL[i * 32 + lane] = make_float2(0.f, 0.f);
        f32x2 acc[PS_TMAX / 2];
#pragma unroll
        for (int j = 0; j < PS_TMAX / 2; ++j) acc[j] = 0ull;
        int rounds = 0;
        __syncthreads();
        // own leaf: positions relative to the same centre; the target's own panel is skipped
        {
            const int g0 = r.x * K, n = (r.y - r.x) * K;
            for (int base = RND * warp; base < n; base += RND * PS_WARPS) {
                PsSrc u[PS_SRC];
                int gp[PS_SRC];
#pragma unroll
                for (int h = 0; h < PS_SRC; ++h) {
                    const int q = base + 32 * h + lane;
                    u[h] = ps_src(q < n ? srcw[g0 + q] : far_src);
                    gp[h] = q < n ? (g0 + q) / K : -1;
                }
                ps_round_self(sh.txy, sh.tz, ntb, tb, u, gp, acc);
                if (++rounds == PS_FOLD) { ps_fold(acc, sHL, ntb, lane); rounds = 0; }
            }
        }
        // the other leaves, as one stream of Gauss points in chunks of PS_EMAX pair records,
        // each warp staging its own copy of a chunk's records
        float4* wrec = sh.rec[warp];
        int* woff = sh.off[warp];
        for (int eb = e0; eb < e1; eb += PS_EMAX) {
            const int ne = min(PS_EMAX, e1 - eb);
            __syncwarp();
            for (int j = lane; j < ne; j += 32) {
                wrec[j] = prec[eb + j];
                woff[j] = poff[eb + j];
            }
            if (lane == 0) woff[ne] = (eb + PS_EMAX < e1) ? poff[eb + PS_EMAX] : total;
            __syncwarp();
            const int s_beg = woff[0], s_end = woff[ne];
            int cur = 0;  // per-lane cursor: the pair record holding the lane's next position
            // the records of the lane's positions first (the cursor walk), then every source
            // load of the round back to back, so that their latencies overlap
            auto fetch = [&](int base, PsSrc (&u)[PS_SRC]) {
                int rec[PS_SRC], g[PS_SRC];
                stream_slots<PS_SRC>(base, lane, s_end, woff, cur, rec, g);
                float4 rc[PS_SRC], v[PS_SRC];
#pragma unroll
                for (int h = 0; h < PS_SRC; ++h) rc[h] = wrec[max(rec[h], 0)];
#pragma unroll
                for (int h = 0; h < PS_SRC; ++h) v[h] = rec[h] >= 0 ? srcw[__float_as_int(rc[h].w) + g[h]] : far_src;
#pragma unroll
                for (int h = 0; h < PS_SRC; ++h) {
                    if (rec[h] >= 0) { v[h].x += rc[h].x; v[h].y += rc[h].y; v[h].z += rc[h].z; }
                    u[h] = ps_src(v[h]);
                }
            };
            for (int base = s_beg + RND * warp; base < s_end; base += RND * PS_WARPS) {
                PsSrc u[PS_SRC];
                fetch(base, u);
                ps_round(sh.txy, sh.tz, ntb, u, acc);
                if (++rounds == PS_FOLD) { ps_fold(acc, sHL, ntb, lane); rounds = 0; }
            }
        }
        ps_fold(acc, sHL, ntb, lane);
        __syncwarp();
        // lane i of each warp adds target i's compensated partials of the warp's 32 lanes,
        // then thread i adds the PS_WARPS warp sums
        if (lane < ntb) {
            float hi = 0.f, lo = 0.f;
            for (int k = 0; k < 32; ++k) {
                const float2 v = sHL[lane * 32 + ((k + lane) & 31)];
                kahan_add(hi, lo, v.x);
                kahan_add(hi, lo, -v.y);
            }
            sh.wsum[warp][lane] = make_float2(hi, lo);
        }
        __syncthreads();
        if (threadIdx.x < ntb) {
            const int i = threadIdx.x;
            float hi = 0.f, lo = 0.f;
#pragma unroll
            for (int w = 0; w < PS_WARPS; ++w) {
                const float2 v = sh.wsum[w][i];
                kahan_add(hi, lo, v.x);
                kahan_add(hi, lo, -v.y);
            }
            ynear[tb + i] = ((double)hi - (double)lo) + yc[tb + i];
        }
    }
}

// Two-float4 source lanes, the same schedule as k_p2p_lap_src for kernels whose sources
// carry a vector: per mat-vec each Gauss point is packed as (leaf-relative position, v_x)
// and (v_y, v_z, -, -).
// - Stokeslet (eq. stokeslet): v = f = q_k S_J t_J; three FP32 accumulators per target,
//   at most P2P_SRC_TMAX_STOKES targets per work item; per pair d = x - y, r^-1 by rsqrt,
//   u += f / r + d (d.f) / r^3.
// - Laplace double layer (eq. gauss:2nd-kind): v = q_k S_j x_j n_j; one accumulator per
//   target, at most P2P_SRC_TMAX targets per item; per pair phi += (d.v) / r^3.
// - Stresslet double layer (eq. stresslet): v = u = q_k S_J u_J, and a third float4 per Gauss
//   point, the source panel's normal n; three accumulators per target, at most
//   P2P_SRC_TMAX_STOKES targets per item; per pair u += -6 (d.u)(d.n) d / r^5.
// Accumulators are folded every PS_FOLD rounds into compensated per-lane sums.
constexpr int SS_SRC = 2;  // sources per lane per round

template <int OP> struct VecLane;
// DOF accumulators per target, at most TM targets per item, MINB resident blocks per SM the
// register budget is set for.
template <> struct VecLane<STK_SL> { static constexpr int DOF = 3, TM = P2P_SRC_TMAX_STOKES, MINB = 7; };
template <> struct VecLane<LAP_DL> { static constexpr int DOF = 1, TM = P2P_SRC_TMAX, MINB = 7; };
template <> struct VecLane<LAP_B4> { static constexpr int DOF = 4, TM = P2P_SRC_TMAX_BATCH, MINB = 6; };
template <> struct VecLane<STK_DL> { static constexpr int DOF = 3, TM = P2P_SRC_TMAX_STOKES, MINB = 6; };

// Both pack per panel (one FP64-to-FP32 conversion per unknown, as k_pack_sources).
__global__ void k_pack_sources_stokes(const float4* src_rel, const double* xs, int K, int64_t n, float4* out) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= n) return;
    xs += blockIdx.y * 3 * n;  // vector blockIdx.y of a Stokes batch
    out += blockIdx.y * 2 * (int64_t)K * n;
    const float t0 = (float)xs[3 * j], t1 = (float)xs[3 * j + 1], t2 = (float)xs[3 * j + 2];
    for (int k = 0; k < K; ++k) {
        const int64_t g = j * K + k;
        const float4 y = src_rel[g];
        out[2 * g] = make_float4(y.x, y.y, y.z, y.w * t0);
        out[2 * g + 1] = make_float4(y.w * t1, y.w * t2, 0.f, 0.f);
    }
}

// A batch of four vectors ([4][n] in xs): (position, w x_0) and (w x_1, w x_2, w x_3, 0).
__global__ void k_pack_sources_b4(const float4* src_rel, const double* xs, int K, int64_t n, float4* out) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= n) return;
    const float x0 = (float)xs[j], x1 = (float)xs[n + j], x2 = (float)xs[2 * n + j], x3 = (float)xs[3 * n + j];
    for (int k = 0; k < K; ++k) {
        const int64_t g = j * K + k;
        const float4 y = src_rel[g];
        out[2 * g] = make_float4(y.x, y.y, y.z, y.w * x0);
        out[2 * g + 1] = make_float4(y.w * x1, y.w * x2, y.w * x3, 0.f);
    }
}

__global__ void k_pack_sources_dipole(const float4* src_rel, const float4* nrm_f, const double* xs, int K, int64_t n,
                                      float4* out) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= n) return;
    const float x = (float)xs[j];
    const float4 nv = nrm_f[j];
    for (int k = 0; k < K; ++k) {
        const int64_t g = j * K + k;
        const float4 y = src_rel[g];
        const float w = y.w * x;
        out[2 * g] = make_float4(y.x, y.y, y.z, w * nv.x);
        out[2 * g + 1] = make_float4(w * nv.y, w * nv.z, 0.f, 0.f);
    }
}

// Pair records are staged per warp (VS_EMAX per chunk), so warps do not wait for one another
// in the main loop; the epilogue's warp sums reuse the record area.
constexpr int VS_EMAX = 32;
static_assert(P2P_SRC_TMAX % 2 == 0 && P2P_SRC_TMAX_STOKES % 2 == 0 && P2P_SRC_TMAX_BATCH % 2 == 0,
              "targets are processed in pairs");
template <int OP> struct VlShared {
    float4 txy[VecLane<OP>::TM / 2];  // target pairs (x_a, x_b, y_a, y_b) and (z_a, z_b)
    float2 tz[VecLane<OP>::TM / 2];
    float2 hl[PS_WARPS][VecLane<OP>::TM * VecLane<OP>::DOF][32];
    union {
        struct {
            float4 rec[PS_WARPS][VS_EMAX];
            int off[PS_WARPS][VS_EMAX + 1];
        } s;
        float2 wsum[PS_WARPS][VecLane<OP>::TM * VecLane<OP>::DOF];
    } u;
};

// One source against a target pair (paired FP32, as in the Laplace kernel). The source's
// position and strength components are repeated in both halves; sk0/sk1 drop the pair's
// first/second target (the source lies on that target's own panel).
struct VlSrc {
    f32x2 x, y, z, v0, v1, v2, v3, n0, n1, n2;
};
__device__ __forceinline__ VlSrc vl_src(float4 a, float4 b, float4 c) {
    return {f2_pack(a.x, a.x), f2_pack(a.y, a.y), f2_pack(a.z, a.z), f2_pack(a.w, a.w),
            f2_pack(b.x, b.x), f2_pack(b.y, b.y), f2_pack(b.z, b.z), f2_pack(c.x, c.x),
            f2_pack(c.y, c.y), f2_pack(c.z, c.z)};
}

template <int OP>
__device__ __forceinline__ void vl_pair(f32x2 tx, f32x2 ty, f32x2 tz, const VlSrc& u, bool sk0, bool sk1,
                                        f32x2* acc) {
    const f32x2 dx = f2_sub(tx, u.x), dy = f2_sub(ty, u.y), dz = f2_sub(tz, u.z);
    float r0, r1;
    f2_unpack(f2_fma(dx, dx, f2_fma(dy, dy, f2_mul(dz, dz))), r0, r1);
    const float i0 = rsqrt_approx(sk0 ? 1.f : r0), i1 = rsqrt_approx(sk1 ? 1.f : r1);
    const f32x2 ir = f2_pack(sk0 ? 0.f : i0, sk1 ? 0.f : i1);
    if (OP == LAP_B4) {
        acc[0] = f2_fma(u.v0, ir, acc[0]);
        acc[1] = f2_fma(u.v1, ir, acc[1]);
        acc[2] = f2_fma(u.v2, ir, acc[2]);
        acc[3] = f2_fma(u.v3, ir, acc[3]);
        return;
    }
    const f32x2 ir3 = f2_mul(ir, f2_mul(ir, ir));
    const f32x2 dv = f2_fma(dx, u.v0, f2_fma(dy, u.v1, f2_mul(dz, u.v2)));
    if (OP == STK_SL) {
        const f32x2 df = f2_mul(dv, ir3);
        acc[0] = f2_fma(u.v0, ir, f2_fma(dx, df, acc[0]));
        acc[1] = f2_fma(u.v1, ir, f2_fma(dy, df, acc[1]));
        acc[2] = f2_fma(u.v2, ir, f2_fma(dz, df, acc[2]));
    } else if (OP == STK_DL) {
        // 6 d (d.u)(e.n) / r^5 with e = -d: f = -6 (d.u)(d.n) / r^5
        const f32x2 dn = f2_fma(dx, u.n0, f2_fma(dy, u.n1, f2_mul(dz, u.n2)));
        const f32x2 ir5 = f2_mul(ir3, f2_mul(ir, ir));
        const f32x2 f = f2_mul(f2_mul(dv, dn), f2_mul(f2_pack(-6.f, -6.f), ir5));
        acc[0] = f2_fma(dx, f, acc[0]);
        acc[1] = f2_fma(dy, f, acc[1]);
        acc[2] = f2_fma(dz, f, acc[2]);
    } else {
        acc[0] = f2_fma(dv, ir3, acc[0]);
    }
}

template <int OP>
__global__ void __launch_bounds__(32 * PS_WARPS, VecLane<OP>::MINB) k_p2p_vec_src(const int4* items, const int2* range, const int* pptr,
                                                                 const float4* prec, const int* poff, const int* plen,
                                                                 const float4* srcw, const float4* snrm,
                                                                 const float4* tgt, int K, const double* yc,
                                                                 double* ynear, int64_t ssys, int64_t xsys) {
    constexpr int DOF = VecLane<OP>::DOF, TM = VecLane<OP>::TM;
    srcw += blockIdx.y * ssys;  // vector blockIdx.y of a Stokes batch: its strengths, corrections and output
    yc += blockIdx.y * xsys;
    ynear += blockIdx.y * xsys;
    __shared__ VlShared<OP> sh;
    constexpr int RND = 32 * SS_SRC;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int4 item = items[blockIdx.x];
    const int cell = item.x, tb = item.y, ntb = item.z;
    const int2 r = range[cell];
    const int e0 = pptr[cell], e1 = pptr[cell + 1];
    const int total = plen[cell];
    float2* sHL = &sh.hl[warp][0][0];
    const float4 far_a = make_float4(1e18f, 0.f, 0.f, 0.f), zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    // the third float4 of a source: its panel's normal (stresslet only)
    auto nrm_of = [&](int q) { return OP == STK_DL ? snrm[q] : zero4; };
    // targets in pairs; an odd count is padded with a far-away target whose sums are never read
    for (int i = threadIdx.x; i < ((ntb + 1) & ~1); i += blockDim.x) {
        const float4 x = i < ntb ? tgt[tb + i] : make_float4(1e18f, 1e18f, 1e18f, 0.f);
        float* xy = reinterpret_cast<float*>(&sh.txy[i >> 1]);
        float* z = reinterpret_cast<float*>(&sh.tz[i >> 1]);
        xy[i & 1] = x.x;
        xy[2 + (i & 1)] = x.y;
        z[i & 1] = x.z;
    }
    for (int i = 0; i < DOF * ntb; ++i) sHL[i * 32 + lane] = make_float2(0.f, 0.f);
    f32x2 acc[TM / 2][DOF];  // acc[j][a]: component a of targets 2j and 2j + 1
#pragma unroll
    for (int j = 0; j < TM / 2; ++j)
#pragma unroll
        for (int a = 0; a < DOF; ++a) acc[j][a] = 0ull;
    int rounds = 0;
    auto fold = [&]() {
#pragma unroll
        for (int j = 0; j < TM / 2; ++j) {
#pragma unroll
            for (int a = 0; a < DOF; ++a) {
                float a0, a1;
                f2_unpack(acc[j][a], a0, a1);
                if (2 * j < ntb) {
                    float2 v = sHL[(DOF * 2 * j + a) * 32 + lane];
                    kahan_add(v.x, v.y, a0);
                    sHL[(DOF * 2 * j + a) * 32 + lane] = v;
                }
                if (2 * j + 1 < ntb) {
                    float2 v = sHL[(DOF * (2 * j + 1) + a) * 32 + lane];
                    kahan_add(v.x, v.y, a1);
                    sHL[(DOF * (2 * j + 1) + a) * 32 + lane] = v;
                }
                acc[j][a] = 0ull;
            }
            asm volatile("" ::: "memory");
        }
    };
    auto round = [&](const VlSrc (&u)[SS_SRC], const int (&gp)[SS_SRC], bool self) {
#pragma unroll
        for (int j = 0; j < TM / 2; ++j) {
            if (2 * j < ntb) {
                const float4 A = sh.txy[j];
                const float2 B = sh.tz[j];
                const f32x2 tx = f2_pack(A.x, A.y), ty = f2_pack(A.z, A.w), tz = f2_pack(B.x, B.y);
#pragma unroll
                for (int h = 0; h < SS_SRC; ++h)
                    vl_pair<OP>(tx, ty, tz, u[h], self && gp[h] == tb + 2 * j, self && gp[h] == tb + 2 * j + 1,
                                acc[j]);
            }
            asm volatile("" ::: "memory");
        }
    };
    __syncthreads();
    // own leaf (own panel skipped)
    {
        const int g0 = r.x * K, n = (r.y - r.x) * K;
        for (int base = RND * warp; base < n; base += RND * PS_WARPS) {
            VlSrc u[SS_SRC];
            int gp[SS_SRC];
#pragma unroll
            for (int h = 0; h < SS_SRC; ++h) {
                const int q = base + 32 * h + lane;
                u[h] = vl_src(q < n ? srcw[2 * (g0 + q)] : far_a, q < n ? srcw[2 * (g0 + q) + 1] : zero4,
                              q < n ? nrm_of(g0 + q) : zero4);
                gp[h] = q < n ? (g0 + q) / K : -1;
            }
            round(u, gp, true);
            if (++rounds == PS_FOLD) { fold(); rounds = 0; }
        }
    }
    // the other leaves of the P2P list, as one stream
    float4* wrec = sh.u.s.rec[warp];
    int* woff = sh.u.s.off[warp];
    for (int eb = e0; eb < e1; eb += VS_EMAX) {
        const int ne = min(VS_EMAX, e1 - eb);
        __syncwarp();
        if (lane < ne) {
            wrec[lane] = prec[eb + lane];
            woff[lane] = poff[eb + lane];
        }
        if (lane == 0) woff[ne] = (eb + VS_EMAX < e1) ? poff[eb + VS_EMAX] : total;
        __syncwarp();
        const int s_beg = woff[0], s_end = woff[ne];
        int cur = 0;
        for (int base = s_beg + RND * warp; base < s_end; base += RND * PS_WARPS) {
            VlSrc u[SS_SRC];
            int gp[SS_SRC];
            // records first, then the round's source loads back to back (as k_p2p_lap_src)
            int rec[SS_SRC], g[SS_SRC];
            stream_slots<SS_SRC>(base, lane, s_end, woff, cur, rec, g);
            float4 rc[SS_SRC], a[SS_SRC], b[SS_SRC], c[SS_SRC];
#pragma unroll
            for (int h = 0; h < SS_SRC; ++h) rc[h] = wrec[max(rec[h], 0)];
#pragma unroll
            for (int h = 0; h < SS_SRC; ++h) {
                const int q = __float_as_int(rc[h].w) + g[h];
                a[h] = rec[h] >= 0 ? srcw[2 * q] : far_a;
                b[h] = rec[h] >= 0 ? srcw[2 * q + 1] : zero4;
                c[h] = rec[h] >= 0 ? nrm_of(q) : zero4;
            }
#pragma unroll
            for (int h = 0; h < SS_SRC; ++h) {
                if (rec[h] >= 0) { a[h].x += rc[h].x; a[h].y += rc[h].y; a[h].z += rc[h].z; }
                u[h] = vl_src(a[h], b[h], c[h]);
                gp[h] = -1;
            }
            round(u, gp, false);
            if (++rounds == PS_FOLD) { fold(); rounds = 0; }
        }
    }
    fold();
    __syncthreads();  // every warp is done with its records before the warp sums overwrite them
    // each warp adds, per (target, component) row, the compensated partials of its 32 lanes
    for (int row = lane; row < DOF * ntb; row += 32) {
        float hi = 0.f, lo = 0.f;
        for (int k = 0; k < 32; ++k) {
            const float2 v = sHL[row * 32 + ((k + row) & 31)];
            kahan_add(hi, lo, v.x);
            kahan_add(hi, lo, -v.y);
        }
        sh.u.wsum[warp][row] = make_float2(hi, lo);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < ntb; i += blockDim.x) {
        double out[DOF];
#pragma unroll
        for (int a = 0; a < DOF; ++a) {
            float hi = 0.f, lo = 0.f;
#pragma unroll
            for (int w = 0; w < PS_WARPS; ++w) {
                const float2 v = sh.u.wsum[w][DOF * i + a];
                kahan_add(hi, lo, v.x);
                kahan_add(hi, lo, -v.y);
            }
            out[a] = (double)hi - (double)lo;
        }
#pragma unroll
        for (int a = 0; a < DOF; ++a) ynear[DOF * (int64_t)(tb + i) + a] = out[a] + yc[DOF * (int64_t)(tb + i) + a];
    }
}

// Direct: one thread per target, every Gauss point staged through shared memory.
template <typename T, int OP>
__global__ void __launch_bounds__(P2P_THREADS) k_direct(int n, int ns, const typename V4<T>::type* src,
                                                        const double4* tgt, const double* xs, const double4* nrm, int K,
                                                        const int* cptr, const int* ccol, const double* cval,
                                                        double scale, double* y) {
    constexpr int DOF = OpDof<OP>::v;
    constexpr int W = SrcWidth<OP>::v;
    __shared__ T spos[3 * P2P_TILE];
    __shared__ T sval[W * P2P_TILE];
    const int i = blockIdx.x * P2P_THREADS + threadIdx.x;
    const bool active = i < n;
    double4 xi = active ? tgt[i] : make_double4(0, 0, 0, 0);
    const T tx = T(xi.x), ty = T(xi.y), tz = T(xi.z);
    double acc[DOF];
#pragma unroll
    for (int a = 0; a < DOF; ++a) acc[a] = 0.0;
    const int own0 = i * K;
    for (int gb = 0; gb < ns; gb += P2P_TILE) {
        const int nt = min(P2P_TILE, ns - gb);
        __syncthreads();
        for (int q = threadIdx.x; q < nt; q += P2P_THREADS) stage<T, OP>(gb + q, src, xs, nrm, K, spos, sval, q);
        __syncthreads();
        if (active) {
            T part[DOF];
#pragma unroll
            for (int a = 0; a < DOF; ++a) part[a] = T(0);
            for (int q = 0; q < nt; ++q) {
                if ((unsigned)(gb + q - own0) < (unsigned)K) continue;
                interact<T, OP>(tx - spos[3 * q], ty - spos[3 * q + 1], tz - spos[3 * q + 2], sval + W * q, part);
            }
#pragma unroll
            for (int a = 0; a < DOF; ++a) acc[a] += (double)part[a];
        }
    }
    if (!active) return;
    add_correction<DOF>(i, cptr, ccol, cval, xs, acc);
#pragma unroll
    for (int a = 0; a < DOF; ++a) y[(int64_t)DOF * i + a] = scale * acc[a];
}

template <typename T, int OP>
int launch_p2p(fmmbem_handle* h, const double* cval) {
    const bool rel = std::is_same<T, float>::value;
    const typename V4<T>::type* src = rel ? reinterpret_cast<const typename V4<T>::type*>(h->src_rel)
                                          : reinterpret_cast<const typename V4<T>::type*>(h->src_d);
    const typename V4<T>::type* tgt = rel ? reinterpret_cast<const typename V4<T>::type*>(h->tgt_rel)
                                          : reinterpret_cast<const typename V4<T>::type*>(h->tgt_d);
    k_p2p<T, OP><<<h->n_leaves, P2P_THREADS, 0, h->stream>>>(h->leaves, h->cell_cs, h->cell_range, h->p2p_ptr,
                                                             h->p2p_src, src, tgt, rel, h->xin, h->nrm_d, h->K,
                                                             h->corr_ptr, h->corr_col, cval, h->ynear, h->N);
    FMM_LAUNCHED();
    return 0;
}

template <typename T, int OP>
int launch_direct(fmmbem_handle* h, const double* xs, double* y, const double* cval, double scale) {
    const typename V4<T>::type* src = std::is_same<T, float>::value
                                          ? reinterpret_cast<const typename V4<T>::type*>(h->src_f)
                                          : reinterpret_cast<const typename V4<T>::type*>(h->src_d);
    const int n = (int)h->N;
    k_direct<T, OP><<<(n + P2P_THREADS - 1) / P2P_THREADS, P2P_THREADS, 0, h->stream>>>(
        n, (int)h->NS, src, h->tgt_d, xs, h->nrm_d, h->K, h->corr_ptr, h->corr_col, cval, scale, y);
    FMM_LAUNCHED();
    return 0;
}

}  // namespace

int near_field_on(fmmbem_handle* h, bool fp64);

// Per-mat-vec FP32 source data of the mixed-precision passes (P2M and the near field read
// it), on the handle's stream before the near and far fields fork.
int pack_sources(fmmbem_handle* h) {
    const unsigned g = (unsigned)((h->N + 255) / 256);
    if (h->nrhs > 1 && h->kernel == FMMBEM_LAPLACE)
        k_pack_sources_b4<<<g, 256, 0, h->stream>>>(h->src_rel, h->xin, h->K, h->N, h->src_w);
    else if (h->kernel == FMMBEM_STOKES)
        k_pack_sources_stokes<<<dim3(g, h->nsys), 256, 0, h->stream>>>(h->src_rel, h->xin, h->K, h->N, h->src_w);
    else if (h->layer == FMMBEM_LAYER_DOUBLE)
        k_pack_sources_dipole<<<g, 256, 0, h->stream>>>(h->src_rel, h->nrm_f, h->xin, h->K, h->N, h->src_w);
    else
        k_pack_sources<<<g, 256, 0, h->stream>>>(h->src_rel, h->xin, h->K, h->N, h->src_w);
    FMM_LAUNCHED();
    h->launches += 1;
    return 0;
}

int near_field(fmmbem_handle* h, bool fp64, cudaStream_t st) {
    cudaStream_t keep = h->stream;
    h->stream = st;
    const int rc = near_field_on(h, fp64);
    h->stream = keep;
    return rc;
}

// The source-lane kernels' resident blocks (seven of 30.8 KB for the Laplace single layer,
// five to seven of 27-36 KB for the others) fit on an SM only with the largest shared-memory
// carveout.
int init_near_attrs() {
    const int c = (int)cudaSharedmemCarveoutMaxShared;
    FMM_CU(cudaFuncSetAttribute(k_p2p_lap_src, cudaFuncAttributePreferredSharedMemoryCarveout, c));
    FMM_CU(cudaFuncSetAttribute(k_p2p_vec_src<STK_SL>, cudaFuncAttributePreferredSharedMemoryCarveout, c));
    FMM_CU(cudaFuncSetAttribute(k_p2p_vec_src<LAP_DL>, cudaFuncAttributePreferredSharedMemoryCarveout, c));
    FMM_CU(cudaFuncSetAttribute(k_p2p_vec_src<LAP_B4>, cudaFuncAttributePreferredSharedMemoryCarveout, c));
    FMM_CU(cudaFuncSetAttribute(k_p2p_vec_src<STK_DL>, cudaFuncAttributePreferredSharedMemoryCarveout, c));
    return 0;
}

// The work-item (source-lane) near-field kernel of this handle's operator over every item.
static int launch_items(fmmbem_handle* h) {
    const int4* it = h->p2p_items;
    const unsigned nb = (unsigned)h->n_p2p_items;
    if (nb == 0) return 0;
    // the correction rows first, into h->ycorr; the item kernel adds one value per target
    const int n = (int)h->N;
    const unsigned gc = (unsigned)(((int64_t)n * CR_LANES + 255) / 256);
    if (h->nrhs > 1 && h->kernel == FMMBEM_LAPLACE) {
        k_corr_rows<4><<<gc, 256, 0, h->stream>>>(n, h->corr_ptr, h->corr_col, h->corr_sl_f, h->xin, h->ycorr, h->N, 0);
        FMM_LAUNCHED();
        k_p2p_vec_src<LAP_B4><<<nb, 32 * PS_WARPS, 0, h->stream>>>(it, h->cell_range, h->p2p_ptr, h->p2p_rec, h->p2p_off,
                                                                   h->p2p_len, h->src_w, nullptr, h->tgt_rel, h->K,
                                                                   h->ycorr, h->ynear, 0, 0);
    } else if (h->kernel == FMMBEM_LAPLACE && h->layer == FMMBEM_LAYER_DOUBLE) {
        k_corr_rows<1><<<gc, 256, 0, h->stream>>>(n, h->corr_ptr, h->corr_col, h->corr_dl_f, h->xin, h->ycorr, 0, 0);
        FMM_LAUNCHED();
        k_p2p_vec_src<LAP_DL><<<nb, 32 * PS_WARPS, 0, h->stream>>>(it, h->cell_range, h->p2p_ptr, h->p2p_rec, h->p2p_off,
                                                                   h->p2p_len, h->src_w, nullptr, h->tgt_rel, h->K,
                                                                   h->ycorr, h->ynear, 0, 0);
    } else if (h->kernel == FMMBEM_LAPLACE) {
        k_corr_rows<1><<<gc, 256, 0, h->stream>>>(n, h->corr_ptr, h->corr_col, h->corr_sl_f, h->xin, h->ycorr, 0, 0);
        FMM_LAUNCHED();
        k_p2p_lap_src<<<nb, 32 * PS_WARPS, 0, h->stream>>>(it, h->cell_range, h->p2p_ptr, h->p2p_rec, h->p2p_off,
                                                          h->p2p_len, h->src_w, h->tgt_rel, h->K, h->ycorr, h->ynear);
    } else if (h->layer == FMMBEM_LAYER_DOUBLE) {  // the stresslet (one vector)
        k_corr_rows<3><<<gc, 256, 0, h->stream>>>(n, h->corr_ptr, h->corr_col, h->corr_dl_f, h->xin, h->ycorr, 0, 0);
        FMM_LAUNCHED();
        k_p2p_vec_src<STK_DL><<<nb, 32 * PS_WARPS, 0, h->stream>>>(it, h->cell_range, h->p2p_ptr, h->p2p_rec, h->p2p_off,
                                                                   h->p2p_len, h->src_w, h->nrm_pt, h->tgt_rel, h->K,
                                                                   h->ycorr, h->ynear, 0, 0);
    } else {  // the Stokeslet: one launch for every vector of a batch (blockIdx.y)
        k_corr_rows<3><<<dim3(gc, h->nsys), 256, 0, h->stream>>>(n, h->corr_ptr, h->corr_col, h->corr_sl_f, h->xin,
                                                                 h->ycorr, 0, 3 * h->N);
        FMM_LAUNCHED();
        k_p2p_vec_src<STK_SL><<<dim3(nb, h->nsys), 32 * PS_WARPS, 0, h->stream>>>(
            it, h->cell_range, h->p2p_ptr, h->p2p_rec, h->p2p_off, h->p2p_len, h->src_w, nullptr, h->tgt_rel, h->K,
            h->ycorr, h->ynear, 2 * h->NS, 3 * h->N);
    }
    FMM_LAUNCHED();
    h->launches += 2;
    return 0;
}

// The near field of one mat-vec (P2P plus the correction rows) on h->stream. The
// mixed-precision kernels read the sources packed by pack_sources.
int near_field_on(fmmbem_handle* h, bool fp64) {
    prof_begin(h, FMMBEM_PASS_P2P);
    const int64_t l0 = h->launches;
    const bool items = !fp64 && h->p2p_variant == 3 && h->p2p_items;
    if (h->nrhs > 1 && h->kernel == FMMBEM_LAPLACE) {
        if (items) FMM_TRY(launch_items(h));
        else {
            FMM_TRY((fp64 ? launch_p2p<double, LAP_B4>(h, h->corr_sl) : launch_p2p<float, LAP_B4>(h, h->corr_sl)));
            h->launches += 1;
        }
    } else if (h->kernel == FMMBEM_STOKES && h->layer == FMMBEM_LAYER_DOUBLE) {
        // the stresslet double layer: the work-item kernel (mixed precision), else the
        // shared-tile schedule with the FP64 3x3 correction rows
        if (items && h->nrm_pt) FMM_TRY(launch_items(h));
        else {
            FMM_TRY((fp64 ? launch_p2p<double, STK_DL>(h, h->corr_dl) : launch_p2p<float, STK_DL>(h, h->corr_dl)));
            h->launches += 1;
        }
    } else if (h->kernel == FMMBEM_LAPLACE && h->layer == FMMBEM_LAYER_DOUBLE) {
        if (items) FMM_TRY(launch_items(h));
        else {
            FMM_TRY((fp64 ? launch_p2p<double, LAP_DL>(h, h->corr_dl) : launch_p2p<float, LAP_DL>(h, h->corr_dl)));
            h->launches += 1;
        }
    } else if (h->kernel == FMMBEM_LAPLACE && !fp64) {
        if (items) {
            FMM_TRY(launch_items(h));
        } else if (h->p2p_variant == 2 && h->stage_ptr) {
            k_p2p_lap_bulk<<<h->n_leaves, 128, 0, h->stream>>>(
                h->leaves, h->cell_range, h->p2p_ptr, h->p2p_src, h->p2p_rec, h->p2p_cnt, h->p2p_toff, h->stage_ptr,
                h->stage_first, h->stage_bytes, h->src_w, h->tgt_rel, h->K, h->corr_ptr, h->corr_col, h->corr_sl,
                h->xin, h->ynear, h->kerr);
            FMM_LAUNCHED();
            h->launches += 1;
        } else if (h->p2p_variant == 1) {
            k_p2p_lap_sliced<<<h->n_leaves, 128, 0, h->stream>>>(h->leaves, h->cell_range, h->p2p_ptr, h->p2p_src,
                                                                h->p2p_rec, h->src_w, h->tgt_rel, h->K, h->corr_ptr,
                                                                h->corr_col, h->corr_sl, h->xin, h->ynear);
            FMM_LAUNCHED();
            h->launches += 1;
        } else {
            // leaves grouped by target count: <= 32, <= 64, more (targets per lane 1, 2, 4)
            const int* cls = h->leaf_class;
            const int n1 = h->leaf_class_start[1], n2 = h->leaf_class_start[2] - n1, n3 = h->n_leaves - n1 - n2;
            if (n1 > 0)
                k_p2p_lap<1><<<n1, 128, 0, h->stream>>>(cls, h->cell_range, h->p2p_ptr, h->p2p_rec, h->p2p_off,
                                                        h->p2p_len, h->src_w, h->tgt_rel, h->K, h->corr_ptr,
                                                        h->corr_col, h->corr_sl, h->xin, h->ynear);
            if (n2 > 0)
                k_p2p_lap<2><<<n2, 128, 0, h->stream>>>(cls + n1, h->cell_range, h->p2p_ptr, h->p2p_rec, h->p2p_off,
                                                        h->p2p_len, h->src_w, h->tgt_rel, h->K, h->corr_ptr,
                                                        h->corr_col, h->corr_sl, h->xin, h->ynear);
            if (n3 > 0)
                k_p2p_lap<4><<<n3, 128, 0, h->stream>>>(cls + n1 + n2, h->cell_range, h->p2p_ptr, h->p2p_rec,
                                                        h->p2p_off, h->p2p_len, h->src_w, h->tgt_rel, h->K,
                                                        h->corr_ptr, h->corr_col, h->corr_sl, h->xin, h->ynear);
            FMM_LAUNCHED();
            h->launches += (n1 > 0) + (n2 > 0) + (n3 > 0);
        }
    } else if (h->kernel == FMMBEM_LAPLACE) {
        FMM_TRY((launch_p2p<double, LAP_SL>(h, h->corr_sl)));
        h->launches += 1;
    } else if (items) {
        FMM_TRY(launch_items(h));
    } else {
        // the shared-tile schedule takes one vector per launch: each vector of a batch in turn
        const double* x0 = h->xin;
        double* y0 = h->ynear;
        for (int q = 0; q < h->nsys; ++q) {
            h->xin = x0 + q * 3 * h->N;
            h->ynear = y0 + q * 3 * h->N;
            const int rc = fp64 ? launch_p2p<double, STK_SL>(h, h->corr_sl) : launch_p2p<float, STK_SL>(h, h->corr_sl);
            h->xin = x0;
            h->ynear = y0;
            FMM_TRY(rc);
            h->launches += 1;
        }
    }
    prof_end(h, FMMBEM_PASS_P2P, (int)(h->launches - l0));
    return 0;
}

// which: 0 single layer (scale of the operator), 1 double layer / stresslet.
int direct_field(fmmbem_handle* h, bool fp64, int which, const double* xsorted, double* ysorted) {
    const double pi = 3.14159265358979323846;
    h->launches += 1;
    if (h->kernel == FMMBEM_LAPLACE) {
        const double sc = 1.0 / (4.0 * pi);
        if (which == 0)
            return fp64 ? launch_direct<double, LAP_SL>(h, xsorted, ysorted, h->corr_sl, sc)
                        : launch_direct<float, LAP_SL>(h, xsorted, ysorted, h->corr_sl, sc);
        return launch_direct<double, LAP_DL>(h, xsorted, ysorted, h->corr_dl, sc);
    }
    if (which == 0) {
        const double sc = -1.0 / (8.0 * pi * h->opts.mu);
        return fp64 ? launch_direct<double, STK_SL>(h, xsorted, ysorted, h->corr_sl, sc)
                    : launch_direct<float, STK_SL>(h, xsorted, ysorted, h->corr_sl, sc);
    }
    return launch_direct<double, STK_DL>(h, xsorted, ysorted, h->corr_dl, 1.0 / (8.0 * pi));
}

}  // namespace fmmbem
