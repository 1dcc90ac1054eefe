// Far-field passes of the FMM mat-vec at a runtime expansion order p (Sec. 2.5):
// P2M at the leaves, M2M up the tree, M2L over the dual-tree-traversal list,
// L2L down the tree, L2P at the collocation points. Expansions are stored
// scaled by the cell side s (M~_n = M_n / s^n, L^_n = L_n s^{n+1}) so that
// magnitudes stay O(1) at every level in FP32 and the translation operators
// between same-size cells depend only on the offset in units of s.
//
// Laplace uses one expansion per cell with strengths w = q_k S_j x_j (eq.
// matvec-onerow). Stokes uses four (Sec. 3.2: "four Laplace expansions"):
// strengths f_1, f_2, f_3 and y.f with f = q_k S_J t_J, and the Stokeslet sum
// u_a = phi_a - x_b d_a phi_b + d_a phi_4 at each target.
#include <mutex>
#include <type_traits>
#include "handle.cuh"
#include "harmonics.cuh"

namespace fmmbem {

namespace {

__constant__ unsigned char c_deg[NCOEF_MAX];  // degree n of each stored coefficient index

template <typename T> FMM_HD cpx<T> ld(const T* base, int q) { return mk(base[2 * q], base[2 * q + 1]); }
template <typename T> FMM_HD void st(T* base, int q, cpx<T> v) { base[2 * q] = v.re; base[2 * q + 1] = v.im; }

// any-order coefficient from a stored (m >= 0) complex array
template <typename T> __device__ __forceinline__ cpx<T> ld_any(const T* base, int n, int m) {
    if (m >= 0) return ld(base, cidx(n, m));
    cpx<T> v = ld(base, cidx(n, -m));
    return (m & 1) ? mk(-v.re, v.im) : mk(v.re, -v.im);
}

__device__ __forceinline__ void decode(int q, int& n, int& m) {
    n = c_deg[q];
    m = q - (n * (n + 1)) / 2;
}

template <typename T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ int octant_of(double4 c, double4 par) {
    return (c.x > par.x ? 1 : 0) | (c.y > par.y ? 2 : 0) | (c.z > par.z ? 4 : 0);
}

constexpr int P2M_WARPS = 4;

// P2M: one block per leaf. Each lane of a warp takes one Gauss point; the solid
// harmonics are generated column by column and every coefficient is reduced
// across the warp by shuffles into a per-warp shared-memory accumulator.
template <typename T, int NC>
__global__ void __launch_bounds__(32 * P2M_WARPS) k_p2m(int p, const int* leaves, const double4* cs, const int2* range,
                                                       const typename V4<T>::type* src, const double* xs, int K,
                                                       double ox, double oy, double oz, T* M, int64_t bstride,
                                                       int64_t xsys, size_t msys) {
    extern __shared__ unsigned char smem_raw[];
    T* acc = reinterpret_cast<T*>(smem_raw);  // [warps][NC][ncoef][2]
    xs += blockIdx.y * xsys;  // copy blockIdx.y of a Stokes batch
    M += blockIdx.y * msys;
    const int nco = ncoef(p);
    const int cell = leaves[blockIdx.x];
    const double4 cc = cs[cell];
    const int2 r = range[cell];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int q = threadIdx.x; q < P2M_WARPS * NC * nco * 2; q += blockDim.x) acc[q] = T(0);
    __shared__ double s_inv;  // 1 / side: one FP64 division per block (FP64 is scarce on this GPU)
    if (threadIdx.x == 0) s_inv = 1.0 / cc.w;
    __syncthreads();
    T* wacc = acc + warp * NC * nco * 2;
    const double inv_s = s_inv;
    const int s0 = r.x * K, s1 = r.y * K;
    for (int base = s0 + warp * 32; base < s1; base += P2M_WARPS * 32) {
        const int s = base + lane;
        T vx = 0, vy = 0, vz = 0, q[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) q[c] = 0;
        if (s < s1) {
            const auto y = src[s];
            const int pj = s / K;
            vx = T(((double)y.x - cc.x) * inv_s);
            vy = T(((double)y.y - cc.y) * inv_s);
            vz = T(((double)y.z - cc.z) * inv_s);
            if (NC == 1) {
                q[0] = T((double)y.w * xs[pj]);
            } else if (bstride) {  // a batch of vectors: plain strengths, vector c at xs + c * bstride
#pragma unroll
                for (int c = 0; c < NC; ++c) q[c] = T((double)y.w * xs[c * bstride + pj]);
            } else {
                const double t0 = xs[3 * pj], t1 = xs[3 * pj + 1], t2 = xs[3 * pj + 2];
                const double w = (double)y.w;
                q[0] = T(w * t0);
                q[1] = T(w * t1);
                q[2] = T(w * t2);
                q[NC - 1] = T(w * (((double)y.x - ox) * t0 + ((double)y.y - oy) * t1 + ((double)y.z - oz) * t2));
            }
        }
        const T r2 = vx * vx + vy * vy + vz * vz;
        const cpx<T> xy = mk(vx, vy);
        cpx<T> diag = mk(T(1), T(0));
        auto emit = [&](int n, int m, cpx<T> R) {
            const int qi = cidx(n, m);
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                T re = warp_sum(q[c] * R.re), im = warp_sum(-q[c] * R.im);
                if (lane == 0) {
                    wacc[(c * nco + qi) * 2] += re;
                    wacc[(c * nco + qi) * 2 + 1] += im;
                }
            }
        };
        for (int m = 0; m <= p; ++m) {
            if (m > 0) diag = (T(-0.5) / T(m)) * (xy * diag);
            emit(m, m, diag);
            if (m + 1 > p) break;
            cpx<T> prev2 = diag, prev1 = vz * diag;
            emit(m + 1, m, prev1);
            for (int n = m + 2; n <= p; ++n) {
                const T inv = T(1) / T((n - m) * (n + m));
                cpx<T> cur = mk((T(2 * n - 1) * vz * prev1.re - r2 * prev2.re) * inv,
                                (T(2 * n - 1) * vz * prev1.im - r2 * prev2.im) * inv);
                emit(n, m, cur);
                prev2 = prev1;
                prev1 = cur;
            }
        }
    }
    __syncthreads();
    T* out = M + (size_t)cell * NC * ESTRIDE;
    for (int idx = threadIdx.x; idx < NC * nco * 2; idx += blockDim.x) {
        const int c = idx / (nco * 2), rest = idx % (nco * 2);
        T v = 0;
#pragma unroll
        for (int w = 0; w < P2M_WARPS; ++w) v += acc[w * NC * nco * 2 + idx];
        out[c * ESTRIDE + rest] = v;
    }
}

// Mixed-precision P2M from the packed sources (pack_sources): each Gauss point is a float4
// (position relative to its leaf centre, strength), so the pass does no FP64 arithmetic
// (FP64 throughput is scarce on this GPU). Each lane carries SPL Gauss points and runs
// their harmonic recurrences side by side; every coefficient is summed over the lane's
// points in registers and then across the warp by one shuffle reduction, so a reduction
// serves 32 SPL points. The block's warps split the harmonic columns m (every warp walks
// all of the leaf's points and runs the cheap diagonal recurrence, but only the owner of
// column m runs and reduces its n-recurrence): a leaf holds one or two chunks of points, so
// splitting the points left one warp doing all the work while the others waited (ncu:
// barrier stalls, 14 of 64 warps active).
// MODE 1: the double layer's dipoles (two float4 per Gauss point, the moment w n in .w of
// the first and .x, .y of the second), scattered as in k_p2m_dl. MODE 2: a batch of four
// vectors (strengths in .w of the first float4 and .x, .y, .z of the second), four
// expansions per cell. MODE 3: the Stokeslet's four Laplace expansions (Sec. 2.5 for Stokes:
// strengths w t_x, w t_y, w t_z packed as for the near field, and w t.(y - o), o the handle's
// origin, formed here from the cell centre's offset to o and the point's position in the
// leaf); the vector of a Stokes batch is blockIdx.y (its sources ssys float4 apart, its
// expansions msys reals apart).
constexpr int P2MP_WARPS = 4;
template <int MODE> struct P2mSpl { static constexpr int v = MODE >= 2 ? 2 : 4; };

template <int MODE>
__global__ void __launch_bounds__(32 * P2MP_WARPS) k_p2m_packed(int p, const int* leaves, const double4* cs,
                                                               const int2* range, const float4* srcw, int K, float* M,
                                                               double ox = 0.0, double oy = 0.0, double oz = 0.0,
                                                               int64_t ssys = 0, size_t msys = 0) {
    constexpr bool DL = MODE == 1;
    constexpr bool QUAD = MODE >= 2;  // four strengths per point, four expansions per cell
    constexpr int NC = QUAD ? 4 : 1;
    srcw += blockIdx.y * ssys;
    M += blockIdx.y * msys;
    constexpr int SPL = P2mSpl<MODE>::v;
    extern __shared__ unsigned char smem_raw[];
    float* acc = reinterpret_cast<float*>(smem_raw);  // [warps][NC][ncoef][2]
    const int nco = ncoef(p);
    const int cell = leaves[blockIdx.x];
    const int2 r = range[cell];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int q = threadIdx.x; q < P2MP_WARPS * NC * nco * 2; q += blockDim.x) acc[q] = 0.f;
    __shared__ float s_inv;  // 1 / side: one FP64 division per block (FP64 is scarce on this GPU)
    __shared__ float s_co[3];  // MODE 3: the cell centre minus the origin
    if (threadIdx.x == 0) {
        const double4 cc = cs[cell];
        s_inv = (float)(1.0 / cc.w);
        s_co[0] = (float)(cc.x - ox);
        s_co[1] = (float)(cc.y - oy);
        s_co[2] = (float)(cc.z - oz);
    }
    __syncthreads();
    float* wacc = acc + warp * NC * nco * 2;
    const float inv_s = s_inv;
    const int s0 = r.x * K, s1 = r.y * K;
    auto add = [&](int comp, int n, int m, cpx<float> d) {  // M~_comp(n, m) += conj(d), summed over the warp
        const int qi = comp * nco + cidx(n, m);
        const float re = warp_sum(d.re), im = warp_sum(-d.im);
        if (lane == 0) {
            wacc[2 * qi] += re;
            wacc[2 * qi + 1] += im;
        }
    };
    // column m belongs to warp w in a snake order (0 1 2 3 3 2 1 0 0 ...), which balances the
    // column lengths p - m + 1 between the warps
    auto owns = [&](int m) {
        const int qd = m / P2MP_WARPS, rm = m - qd * P2MP_WARPS;
        return ((qd & 1) ? P2MP_WARPS - 1 - rm : rm) == warp;
    };
    constexpr int NP = SPL / 2;  // pairs of points per lane
    static_assert(SPL % 2 == 0, "points are processed in pairs");
    for (int base = s0; base < s1; base += 32 * SPL) {
        float vx[SPL], vy[SPL], vz[SPL], q[SPL], c[SPL], qb[SPL][4];
        cpx<float> a[SPL], b[SPL];
#pragma unroll
        for (int h = 0; h < SPL; ++h) {
            const int s = base + 32 * h + lane;
            vx[h] = vy[h] = vz[h] = q[h] = c[h] = 0.f;
            qb[h][0] = qb[h][1] = qb[h][2] = qb[h][3] = 0.f;
            a[h] = b[h] = mk(0.f, 0.f);
            if (s < s1) {
                if (MODE == 2) {
                    const float4 u = srcw[2 * s], u2 = srcw[2 * s + 1];
                    vx[h] = u.x * inv_s; vy[h] = u.y * inv_s; vz[h] = u.z * inv_s;
                    qb[h][0] = u.w; qb[h][1] = u2.x; qb[h][2] = u2.y; qb[h][3] = u2.z;
                } else if (MODE == 3) {
                    const float4 u = srcw[2 * s], u2 = srcw[2 * s + 1];
                    vx[h] = u.x * inv_s; vy[h] = u.y * inv_s; vz[h] = u.z * inv_s;
                    qb[h][0] = u.w; qb[h][1] = u2.x; qb[h][2] = u2.y;
                    qb[h][3] = u.w * (s_co[0] + u.x) + u2.x * (s_co[1] + u.y) + u2.y * (s_co[2] + u.z);
                } else if (DL) {
                    const float4 u = srcw[2 * s], u2 = srcw[2 * s + 1];
                    vx[h] = u.x * inv_s; vy[h] = u.y * inv_s; vz[h] = u.z * inv_s;
                    const float mx = u.w * inv_s, my = u2.x * inv_s, mz = u2.y * inv_s;
                    c[h] = mz;
                    a[h] = mk(0.5f * mx, -0.5f * my);
                    b[h] = mk(0.5f * mx, 0.5f * my);
                } else {
                    const float4 u = srcw[s];
                    vx[h] = u.x * inv_s; vy[h] = u.y * inv_s; vz[h] = u.z * inv_s;
                    q[h] = u.w;
                }
            }
        }
        f32x2 q2[NP];
#pragma unroll
        for (int k = 0; k < NP; ++k) q2[k] = f2_pack(q[2 * k], q[2 * k + 1]);
        // R_n^m of the lane's points, held as pairs of points (re and im of points 2k, 2k + 1)
        auto emit = [&](int n, int m, const f32x2 (&Rre)[NP], const f32x2 (&Rim)[NP]) {
            if (!DL && !QUAD) {  // single layer: sum_h q_h R_h with paired multiply-adds
                f32x2 sre = f2_mul(q2[0], Rre[0]), sim = f2_mul(q2[0], Rim[0]);
#pragma unroll
                for (int k = 1; k < NP; ++k) {
                    sre = f2_fma(q2[k], Rre[k], sre);
                    sim = f2_fma(q2[k], Rim[k], sim);
                }
                float a0, a1, b0, b1;
                f2_unpack(sre, a0, a1);
                f2_unpack(sim, b0, b1);
                add(0, n, m, mk(a0 + a1, b0 + b1));
                return;
            }
            cpx<float> R[SPL];
#pragma unroll
            for (int k = 0; k < NP; ++k) {
                f2_unpack(Rre[k], R[2 * k].re, R[2 * k + 1].re);
                f2_unpack(Rim[k], R[2 * k].im, R[2 * k + 1].im);
            }
            if (DL) {  // R = R_n^m, n < p: feeds degree n + 1
                cpx<float> t0 = mk(0.f, 0.f), t1 = t0, t2 = t0, t3 = t0;
#pragma unroll
                for (int h = 0; h < SPL; ++h) {
                    cfma(t0, mk(c[h], 0.f), R[h]);
                    cfma(t1, a[h], R[h]);
                    cfma(t2, b[h], R[h]);
                    cfma(t3, b[h], conj(R[h]));
                }
                add(0, n + 1, m, t0);
                if (m >= 1) add(0, n + 1, m - 1, t1);
                add(0, n + 1, m + 1, mk(-t2.re, -t2.im));
                if (m == 1) add(0, n + 1, 0, t3);
            } else if (QUAD) {
#pragma unroll
                for (int cc = 0; cc < 4; ++cc) {
                    cpx<float> t = mk(0.f, 0.f);
#pragma unroll
                    for (int h = 0; h < SPL; ++h) t = t + qb[h][cc] * R[h];
                    add(cc, n, m, t);
                }
            }
        };
        const int nmax = DL ? p - 1 : p;  // highest degree generated
        // The recurrences run on pairs of points with paired FP32 instructions:
        //   R_m^m = (-(x + iy) / (2m)) R_{m-1}^{m-1},  R_{m+1}^m = z R_m^m,
        //   R_n^m = ((2n - 1) z R_{n-1}^m - r^2 R_{n-2}^m) / ((n - m)(n + m)).
        f32x2 vz2[NP], nr2[NP], xre[NP], xim[NP], nxim[NP], dre[NP], dim[NP], p1re[NP], p1im[NP], p2re[NP], p2im[NP];
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            const int h0 = 2 * k, h1 = 2 * k + 1;
            vz2[k] = f2_pack(vz[h0], vz[h1]);
            nr2[k] = f2_pack(-(vx[h0] * vx[h0] + vy[h0] * vy[h0] + vz[h0] * vz[h0]),
                             -(vx[h1] * vx[h1] + vy[h1] * vy[h1] + vz[h1] * vz[h1]));
            xre[k] = f2_pack(vx[h0], vx[h1]);
            xim[k] = f2_pack(vy[h0], vy[h1]);
            nxim[k] = f2_pack(-vy[h0], -vy[h1]);
            dre[k] = f2_pack(1.f, 1.f);
            dim[k] = 0ull;
        }
        for (int m = 0; m <= nmax; ++m) {
            if (m > 0) {
                const float f = -0.5f / (float)m;
                const f32x2 f2 = f2_pack(f, f);
#pragma unroll
                for (int k = 0; k < NP; ++k) {
                    const f32x2 re = f2_fma(xre[k], dre[k], f2_mul(nxim[k], dim[k]));
                    const f32x2 im = f2_fma(xre[k], dim[k], f2_mul(xim[k], dre[k]));
                    dre[k] = f2_mul(f2, re);
                    dim[k] = f2_mul(f2, im);
                }
            }
            if (!owns(m)) continue;
            emit(m, m, dre, dim);
            if (m + 1 > nmax) continue;
#pragma unroll
            for (int k = 0; k < NP; ++k) {
                p2re[k] = dre[k];
                p2im[k] = dim[k];
                p1re[k] = f2_mul(vz2[k], dre[k]);
                p1im[k] = f2_mul(vz2[k], dim[k]);
            }
            emit(m + 1, m, p1re, p1im);
            for (int n = m + 2; n <= nmax; ++n) {
                const float inv = 1.f / (float)((n - m) * (n + m)), tn = (float)(2 * n - 1);
                const f32x2 inv2 = f2_pack(inv, inv), tn2 = f2_pack(tn, tn);
#pragma unroll
                for (int k = 0; k < NP; ++k) {
                    const f32x2 tz = f2_mul(tn2, vz2[k]);
                    const f32x2 cre = f2_mul(f2_fma(tz, p1re[k], f2_mul(nr2[k], p2re[k])), inv2);
                    const f32x2 cim = f2_mul(f2_fma(tz, p1im[k], f2_mul(nr2[k], p2im[k])), inv2);
                    p2re[k] = p1re[k];
                    p2im[k] = p1im[k];
                    p1re[k] = cre;
                    p1im[k] = cim;
                }
                emit(n, m, p1re, p1im);
            }
        }
    }
    __syncthreads();
    float* out = M + (size_t)cell * NC * ESTRIDE;
    for (int idx = threadIdx.x; idx < NC * nco * 2; idx += blockDim.x) {
        const int cc = idx / (nco * 2), rest = idx % (nco * 2);
        float v = 0.f;
#pragma unroll
        for (int w = 0; w < P2MP_WARPS; ++w) v += acc[w * NC * nco * 2 + idx];
        out[cc * ESTRIDE + rest] = v;
    }
}

// P2M of the double layer (eq. laplace_bem_dGdn): Gauss point y carries a dipole of
// moment w n_j (w = q_k S_j x_j, n_j its panel's normal), whose potential is
// w n_j . grad_y (1/|x - y|). Its multipole coefficients are the conjugated directional
// derivatives of the regular solid harmonics,
//   M_n^m += w conj(n_z R_{n-1}^m + (n_x - i n_y)/2 R_{n-1}^{m+1} - (n_x + i n_y)/2 R_{n-1}^{m-1}),
// which follow from dR_n^m/dz = R_{n-1}^m and (d/dx + i d/dy) R_n^m = R_{n-1}^{m+1},
// (d/dx - i d/dy) R_n^m = -R_{n-1}^{m-1} for R_n^m = r^n P_n^m(cos theta) e^{i m phi} / (n+m)!,
// with R_{n-1}^{-1} = -conj(R_{n-1}^1). In the scaled storage (M~_n = M_n / s^n, argument
// (y - c)/s) the derivative brings one factor 1/s. M_0^0 is zero. Each R_k^j (k < p) a lane
// generates is scattered into the coefficients of degree k + 1 it feeds, each reduced
// across the warp as in k_p2m.
template <typename T>
__global__ void __launch_bounds__(32 * P2M_WARPS) k_p2m_dl(int p, const int* leaves, const double4* cs, const int2* range,
                                                          const typename V4<T>::type* src, const double4* nrm,
                                                          const double* xs, int K, T* M) {
    extern __shared__ unsigned char smem_raw[];
    T* acc = reinterpret_cast<T*>(smem_raw);  // [warps][ncoef][2]
    const int nco = ncoef(p);
    const int cell = leaves[blockIdx.x];
    const double4 cc = cs[cell];
    const int2 r = range[cell];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int q = threadIdx.x; q < P2M_WARPS * nco * 2; q += blockDim.x) acc[q] = T(0);
    __syncthreads();
    T* wacc = acc + warp * nco * 2;
    const double inv_s = 1.0 / cc.w;
    const int s0 = r.x * K, s1 = r.y * K;
    for (int base = s0 + warp * 32; base < s1; base += P2M_WARPS * 32) {
        const int s = base + lane;
        T vx = 0, vy = 0, vz = 0, c = 0;
        cpx<T> a = mk(T(0), T(0)), b = mk(T(0), T(0));  // w (n_x -+ i n_y) / 2
        if (s < s1) {
            const auto y = src[s];
            const int pj = s / K;
            const double4 n = nrm[pj];
            vx = T(((double)y.x - cc.x) * inv_s);
            vy = T(((double)y.y - cc.y) * inv_s);
            vz = T(((double)y.z - cc.z) * inv_s);
            const double w = (double)y.w * xs[pj] * inv_s;
            c = T(w * n.z);
            a = mk(T(0.5 * w * n.x), T(-0.5 * w * n.y));
            b = mk(T(0.5 * w * n.x), T(0.5 * w * n.y));
        }
        auto add = [&](int n, int m, cpx<T> d) {  // M~(n, m) += conj(d), summed over the warp
            const int qi = cidx(n, m);
            const T re = warp_sum(d.re), im = warp_sum(-d.im);
            if (lane == 0) {
                wacc[2 * qi] += re;
                wacc[2 * qi + 1] += im;
            }
        };
        auto emit = [&](int k, int j, cpx<T> R) {  // R = R_k^j(v), k < p
            add(k + 1, j, c * R);
            if (j >= 1) add(k + 1, j - 1, a * R);
            const cpx<T> bR = b * R;
            add(k + 1, j + 1, mk(-bR.re, -bR.im));
            if (j == 1) add(k + 1, 0, b * conj(R));  // the R_k^{-1} term of M_{k+1}^0
        };
        const T r2 = vx * vx + vy * vy + vz * vz;
        const cpx<T> xy = mk(vx, vy);
        cpx<T> diag = mk(T(1), T(0));
        for (int m = 0; m < p; ++m) {
            if (m > 0) diag = (T(-0.5) / T(m)) * (xy * diag);
            emit(m, m, diag);
            if (m + 1 >= p) break;
            cpx<T> prev2 = diag, prev1 = vz * diag;
            emit(m + 1, m, prev1);
            for (int n = m + 2; n < p; ++n) {
                const T inv = T(1) / T((n - m) * (n + m));
                cpx<T> cur = mk((T(2 * n - 1) * vz * prev1.re - r2 * prev2.re) * inv,
                                (T(2 * n - 1) * vz * prev1.im - r2 * prev2.im) * inv);
                emit(n, m, cur);
                prev2 = prev1;
                prev1 = cur;
            }
        }
    }
    __syncthreads();
    T* out = M + (size_t)cell * ESTRIDE;
    for (int idx = threadIdx.x; idx < nco * 2; idx += blockDim.x) {
        T v = 0;
#pragma unroll
        for (int w = 0; w < P2M_WARPS; ++w) v += acc[w * nco * 2 + idx];
        out[idx] = v;
    }
}

// P2M of the stresslet double layer (eq. stresslet) as four Laplace dipole expansions.
// With r = x - y, a = q_k S_j u_j (the density times the quadrature weight) and n_j the
// panel normal,
//   sum (a.r)(n.r) r_i / |r|^5 = (1/6) [ S_i - x_b d_i S_b + d_i S_0 ],
// where S_b (b = 1..3) is the potential of dipoles of moment a_b n + n_b a and S_0 that of
// moments (a.y') n + (n.y') a (y' = y - origin, x likewise in the evaluation): the sum is
// the Stokeslet's four-potential evaluation of L2P applied to these dipole expansions.
// The moments are stored negated so that the far field carries the near-field kernel's
// sign (-6 (r.a)(r.n) r / |r|^5). Component c of a cell: c < 3 -> S_{c+1}, c = 3 -> S_0.
// Each harmonic R_k^j (k < p) a lane generates feeds degree k + 1 of every component, as in
// k_p2m_dl. FP32 path: packed sources (position relative to the leaf centre, a) and the
// FP32 normals; FP64 path: absolute Gauss points, x and the FP64 normals.
template <typename T, bool PACKED>
__global__ void __launch_bounds__(32 * P2M_WARPS) k_p2m_sdl(int p, const int* leaves, const double4* cs,
                                                           const int2* range, const typename V4<T>::type* src,
                                                           const float4* srcw, const double4* nrm_d,
                                                           const float4* nrm_f, const double* xs, int K, double ox,
                                                           double oy, double oz, T* M) {
    extern __shared__ unsigned char smem_raw[];
    T* acc = reinterpret_cast<T*>(smem_raw);  // [warps][4][ncoef][2]
    const int nco = ncoef(p);
    const int cell = leaves[blockIdx.x];
    const double4 cc = cs[cell];
    const int2 r = range[cell];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int q = threadIdx.x; q < P2M_WARPS * 4 * nco * 2; q += blockDim.x) acc[q] = T(0);
    __syncthreads();
    T* wacc = acc + warp * 4 * nco * 2;
    const double inv_s = 1.0 / cc.w;
    const T co_x = T(cc.x - ox), co_y = T(cc.y - oy), co_z = T(cc.z - oz);  // leaf centre from the origin
    const int s0 = r.x * K, s1 = r.y * K;
    auto add = [&](int comp, int n, int m, cpx<T> d) {  // M~_comp(n, m) += conj(d), summed over the warp
        const int qi = comp * nco + cidx(n, m);
        const T re = warp_sum(d.re), im = warp_sum(-d.im);
        if (lane == 0) {
            wacc[2 * qi] += re;
            wacc[2 * qi + 1] += im;
        }
    };
    for (int base = s0 + warp * 32; base < s1; base += P2M_WARPS * 32) {
        const int s = base + lane;
        T vx = 0, vy = 0, vz = 0;
        T mom[4][3];
#pragma unroll
        for (int c = 0; c < 4; ++c) mom[c][0] = mom[c][1] = mom[c][2] = T(0);
        if (s < s1) {
            T rx, ry, rz, a[3], nn[3];
            const int pj = s / K;
            if (PACKED) {
                const float4 u = srcw[2 * s], u2 = srcw[2 * s + 1];
                const float4 nv = nrm_f[pj];
                rx = u.x; ry = u.y; rz = u.z;
                a[0] = u.w; a[1] = u2.x; a[2] = u2.y;
                nn[0] = nv.x; nn[1] = nv.y; nn[2] = nv.z;
            } else {
                const auto y = src[s];
                const double4 nv = nrm_d[pj];
                rx = T((double)y.x - cc.x); ry = T((double)y.y - cc.y); rz = T((double)y.z - cc.z);
                const double w = (double)y.w;
                a[0] = T(w * xs[3 * pj]); a[1] = T(w * xs[3 * pj + 1]); a[2] = T(w * xs[3 * pj + 2]);
                nn[0] = T(nv.x); nn[1] = T(nv.y); nn[2] = T(nv.z);
            }
            vx = rx * T(inv_s); vy = ry * T(inv_s); vz = rz * T(inv_s);
            const T yx = co_x + rx, yy = co_y + ry, yz = co_z + rz;  // y - origin
            const T ay = a[0] * yx + a[1] * yy + a[2] * yz, ny = nn[0] * yx + nn[1] * yy + nn[2] * yz;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
#pragma unroll
                for (int b = 0; b < 3; ++b) mom[b][d] = -(a[b] * nn[d] + nn[b] * a[d]);
                mom[3][d] = -(ay * nn[d] + ny * a[d]);
            }
        }
        // per component: c = m_z / s, a = (m_x - i m_y) / 2s, b = (m_x + i m_y) / 2s
        T cz[4];
        cpx<T> ca[4], cb[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const T mx = mom[c][0] * T(inv_s), my = mom[c][1] * T(inv_s), mz = mom[c][2] * T(inv_s);
            cz[c] = mz;
            ca[c] = mk(T(0.5) * mx, T(-0.5) * my);
            cb[c] = mk(T(0.5) * mx, T(0.5) * my);
        }
        auto emit = [&](int k, int j, cpx<T> R) {  // R = R_k^j(v), k < p
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                add(c, k + 1, j, cz[c] * R);
                if (j >= 1) add(c, k + 1, j - 1, ca[c] * R);
                const cpx<T> bR = cb[c] * R;
                add(c, k + 1, j + 1, mk(-bR.re, -bR.im));
                if (j == 1) add(c, k + 1, 0, cb[c] * conj(R));
            }
        };
        const T r2 = vx * vx + vy * vy + vz * vz;
        const cpx<T> xy = mk(vx, vy);
        cpx<T> diag = mk(T(1), T(0));
        for (int m = 0; m < p; ++m) {
            if (m > 0) diag = (T(-0.5) / T(m)) * (xy * diag);
            emit(m, m, diag);
            if (m + 1 >= p) break;
            cpx<T> prev2 = diag, prev1 = vz * diag;
            emit(m + 1, m, prev1);
            for (int n = m + 2; n < p; ++n) {
                const T inv = T(1) / T((n - m) * (n + m));
                cpx<T> cur = mk((T(2 * n - 1) * vz * prev1.re - r2 * prev2.re) * inv,
                                (T(2 * n - 1) * vz * prev1.im - r2 * prev2.im) * inv);
                emit(n, m, cur);
                prev2 = prev1;
                prev1 = cur;
            }
        }
    }
    __syncthreads();
    T* out = M + (size_t)cell * 4 * ESTRIDE;
    for (int idx = threadIdx.x; idx < 4 * nco * 2; idx += blockDim.x) {
        const int c = idx / (nco * 2), rest = idx % (nco * 2);
        T v = 0;
#pragma unroll
        for (int w = 0; w < P2M_WARPS; ++w) v += acc[w * 4 * nco * 2 + idx];
        out[c * ESTRIDE + rest] = v;
    }
}

// M2M for the non-leaf cells of one level: M~_n^m(P) = sum_children sum_{j,k}
// M~_j^k(c) 2^{-j} conj(R_{n-j}^{m-k}(d)), d = (c_child - c_parent)/s_parent.
// One block per parent. The children's expansions and octant tables are staged in
// shared memory; thread (child x, coefficient q) forms one child's contribution and
// the children are summed in a fixed order, so the result is deterministic.
constexpr int TREE_THREADS = 256;

template <typename T, int NC>
__global__ void __launch_bounds__(TREE_THREADS) k_m2m(int p, const int* parents, const double4* cs, const int2* child,
                                                      const T* oct, T* M, size_t msys) {
    pdl_wait();
    M += blockIdx.y * msys;  // copy blockIdx.y of a Stokes batch
    extern __shared__ unsigned char smem_raw[];
    const int nco = ncoef(p);
    const int cell = parents[blockIdx.x];
    const int2 ch = child[cell];
    const int per = NC * nco * 2;  // reals of one cell's expansions
    T* sM = reinterpret_cast<T*>(smem_raw);  // [8][NC][nco][2]
    T* sR = sM + 8 * per;                    // [8][nco][2]
    T* sP = sR + 8 * nco * 2;                // [8][NC][nco][2] per-child contributions
    const double4 pc = cs[cell];
    for (int idx = threadIdx.x; idx < ch.y * per; idx += blockDim.x) {
        const int x = idx / per, rem = idx % per, c = rem / (2 * nco), q2 = rem % (2 * nco);
        sM[idx] = M[(size_t)(ch.x + x) * NC * ESTRIDE + c * ESTRIDE + q2];
    }
    for (int idx = threadIdx.x; idx < ch.y * nco * 2; idx += blockDim.x) {
        const int x = idx / (2 * nco), q2 = idx % (2 * nco);
        sR[idx] = oct[octant_of(cs[ch.x + x], pc) * NCOEF_MAX * 2 + q2];
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < ch.y * nco; idx += blockDim.x) {
        const int x = idx / nco, q = idx % nco;
        int n, m;
        decode(q, n, m);
        const T* Rt = sR + x * nco * 2;
        const T* Mc = sM + x * per;
        cpx<T> acc[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[c] = mk(T(0), T(0));
        T sc = T(1);
        for (int j = 0; j <= n; ++j) {
            const int klo = max(-j, m - (n - j)), khi = min(j, m + (n - j));
            for (int k = klo; k <= khi; ++k) {
                const cpx<T> R = conj(ld_any(Rt, n - j, m - k));
#pragma unroll
                for (int c = 0; c < NC; ++c) cfma(acc[c], sc * ld_any(Mc + c * nco * 2, j, k), R);
            }
            sc *= T(0.5);
        }
#pragma unroll
        for (int c = 0; c < NC; ++c) st(sP + x * per + c * nco * 2, q, acc[c]);
    }
    __syncthreads();
    T* out = M + (size_t)cell * NC * ESTRIDE;
    for (int idx = threadIdx.x; idx < per; idx += blockDim.x) {
        T v = T(0);
        for (int x = 0; x < ch.y; ++x) v += sP[x * per + idx];
        const int c = idx / (2 * nco), q2 = idx % (2 * nco);
        out[c * ESTRIDE + q2] = v;
    }
}

// M2L, gathered per target cell over its interaction list:
//   L^_j^k += (-1)^j conj( sum_{n,m} rho^n M~_n^m I_{n+j}^{m+k}(t / s_t) ),
// t = c_target - c_source, rho = s_source / s_target (a power of two).
// One thread per output coefficient (j, k); the irregular table of each pair is
// built in shared memory, one column per thread.
// The gather form computes in FP64 whatever the storage type T: its irregular harmonics reach
// degree 2p, and their magnitudes ((n - m)! P_n^m / r^(n+1), n up to 32) leave the FP32 range
// for offsets of about one cell side and below. It is the fallback of trees whose operators
// are not tabulated, so its speed matters less than its range.
template <typename T, int NC>
__global__ void k_m2l(int p, const int* ptr, const int* srcl, const double4* cs, const T* M, T* L, size_t msys) {
    M += blockIdx.y * msys;  // copy blockIdx.y of a Stokes batch
    L += blockIdx.y * msys;
    __shared__ double sI[NI_MAX * 2];
    __shared__ double sM[NC * NCOEF_MAX * 2];
    const int tc = blockIdx.x;
    const int nco = ncoef(p);
    const int t = threadIdx.x;
    int j = 0, k = 0;
    if (t < nco) decode(t, j, k);
    const double4 ct = cs[tc];
    cpx<double> acc[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[c] = mk(0.0, 0.0);
    const int e0 = ptr[tc], e1 = ptr[tc + 1];
    for (int e = e0; e < e1; ++e) {
        const int sc = srcl[e];
        const double4 cv = cs[sc];
        const double is = 1.0 / ct.w;
        const double vx = (ct.x - cv.x) * is, vy = (ct.y - cv.y) * is, vz = (ct.z - cv.z) * is;
        const int dl = ilogb(cv.w * is);  // log2(rho), exact for cells of the same tree
        __syncthreads();
        if (t <= 2 * p) irregular_column<double>(vx, vy, vz, t, 2 * p, reinterpret_cast<cpx<double>*>(sI));
        const T* Ms = M + (size_t)sc * NC * ESTRIDE;
        for (int idx = t; idx < NC * nco; idx += blockDim.x) {
            const int c = idx / nco, q = idx % nco;
            const double f = (dl == 0) ? 1.0 : ldexp(1.0, dl * (int)c_deg[q]);
            sM[(c * NCOEF_MAX + q) * 2] = f * (double)Ms[c * ESTRIDE + 2 * q];
            sM[(c * NCOEF_MAX + q) * 2 + 1] = f * (double)Ms[c * ESTRIDE + 2 * q + 1];
        }
        __syncthreads();
        if (t < nco) {
            for (int n = 0; n <= p; ++n) {
                const int nj = n + j;
                const int base = cidx(n, 0);
                // m >= 0: M_n^m I_{n+j}^{m+k}
                for (int m = 0; m <= n; ++m) {
                    const cpx<double> I = ld(sI, cidx(nj, m + k));
#pragma unroll
                    for (int c = 0; c < NC; ++c) cfma(acc[c], ld(sM + c * NCOEF_MAX * 2, base + m), I);
                }
                // m = -mu, 1 <= mu <= min(n, k): (-1)^mu conj(M_n^mu) I_{n+j}^{k-mu}
                const int mk1 = min(n, k);
                for (int mu = 1; mu <= mk1; ++mu) {
                    cpx<double> I = ld(sI, cidx(nj, k - mu));
                    if (mu & 1) I = mk(-I.re, -I.im);
#pragma unroll
                    for (int c = 0; c < NC; ++c) cfma_conja(acc[c], ld(sM + c * NCOEF_MAX * 2, base + mu), I);
                }
                // m = -mu, k < mu <= n: (-1)^k conj(M_n^mu I_{n+j}^{mu-k})
                for (int mu = k + 1; mu <= n; ++mu) {
                    const cpx<double> I = ld(sI, cidx(nj, mu - k));
#pragma unroll
                    for (int c = 0; c < NC; ++c) {
                        const cpx<double> v = ld(sM + c * NCOEF_MAX * 2, base + mu) * I;
                        if (k & 1) { acc[c].re -= v.re; acc[c].im += v.im; }
                        else { acc[c].re += v.re; acc[c].im -= v.im; }
                    }
                }
            }
        }
    }
    if (t < nco) {
        T* out = L + (size_t)tc * NC * ESTRIDE;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            cpx<double> v = conj(acc[c]);
            if (j & 1) v = mk(-v.re, -v.im);
            st(out + c * ESTRIDE, t, mk(T(v.re), T(v.im)));
        }
    }
}

// L2L from the non-leaf cells of one level to their children:
//   L^_j^k(c) += sum_{n>=j, m} L^_n^m(P) R_{n-j}^{m-k}(d) 2^{-(j+1)}.
// One block per parent: the parent's expansions and the children's octant tables are
// staged in shared memory; thread (child x, coefficient q) writes one output.
template <typename T, int NC>
__global__ void __launch_bounds__(TREE_THREADS) k_l2l(int p, const int* parents, const double4* cs, const int2* child,
                                                      const T* oct, T* L, size_t msys) {
    pdl_wait();
    L += blockIdx.y * msys;  // copy blockIdx.y of a Stokes batch
    extern __shared__ unsigned char smem_raw[];
    const int nco = ncoef(p);
    const int cell = parents[blockIdx.x];
    const int2 ch = child[cell];
    const int per = NC * nco * 2;
    T* sL = reinterpret_cast<T*>(smem_raw);  // [NC][nco][2]
    T* sR = sL + per;                        // [8][nco][2]
    const double4 pc = cs[cell];
    const T* Lp = L + (size_t)cell * NC * ESTRIDE;
    for (int idx = threadIdx.x; idx < per; idx += blockDim.x) {
        const int c = idx / (2 * nco), q2 = idx % (2 * nco);
        sL[idx] = Lp[c * ESTRIDE + q2];
    }
    for (int idx = threadIdx.x; idx < ch.y * nco * 2; idx += blockDim.x) {
        const int x = idx / (2 * nco), q2 = idx % (2 * nco);
        sR[idx] = oct[octant_of(cs[ch.x + x], pc) * NCOEF_MAX * 2 + q2];
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < ch.y * nco; idx += blockDim.x) {
        const int x = idx / nco, q = idx % nco;
        int j, k;
        decode(q, j, k);
        const T* Rt = sR + x * nco * 2;
        cpx<T> acc[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[c] = mk(T(0), T(0));
        for (int n = j; n <= p; ++n) {
            const int mlo = max(-n, k - (n - j)), mhi = min(n, k + (n - j));
            for (int m = mlo; m <= mhi; ++m) {
                const cpx<T> R = ld_any(Rt, n - j, m - k);
#pragma unroll
                for (int c = 0; c < NC; ++c) cfma(acc[c], ld_any(sL + c * nco * 2, n, m), R);
            }
        }
        const T f = T(ldexp(1.0, -(j + 1)));
        T* out = L + (size_t)(ch.x + x) * NC * ESTRIDE;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            cpx<T> v = ld(out + c * ESTRIDE, q);
            st(out + c * ESTRIDE, q, v + f * acc[c]);
        }
    }
}

// L2P at the collocation points of each leaf, plus the near-field sum, times the
// operator's scale; written in the caller's order or in sorted order.
//   phi(x) = (1/s) sum_{n,m} L^_n^m R_n^m(v), v = (x - c)/s
//   grad phi = (1/s^2) sum L^_n^m grad R_n^m(v) with d_z R_n^m = R_{n-1}^m and
//   (d_x + i d_y) R_n^m = R_{n-1}^{m+1}.
template <typename T, int NC>
__global__ void k_l2p(int p, const int* leaves, const double4* cs, const int2* range, const double4* tgt, const T* L,
                      const double* ynear, double scale, double ox, double oy, double oz, const double* xs_half,
                      const float4* tgt_rel, double* yout, int64_t bstride, size_t msys, int64_t ysys) {
    __shared__ T sL[NC * NCOEF_MAX * 2];
    L += blockIdx.y * msys;  // copy blockIdx.y of a Stokes batch and its output vector
    ynear += blockIdx.y * ysys;
    yout += blockIdx.y * ysys;
    const int cell = leaves[blockIdx.x];
    const double4 cc = cs[cell];
    const int2 r = range[cell];
    const int nco = ncoef(p);
    const T* Lc = L + (size_t)cell * NC * ESTRIDE;
    for (int idx = threadIdx.x; idx < NC * nco; idx += blockDim.x) {
        const int c = idx / nco, q = idx % nco;
        sL[(c * NCOEF_MAX + q) * 2] = Lc[c * ESTRIDE + 2 * q];
        sL[(c * NCOEF_MAX + q) * 2 + 1] = Lc[c * ESTRIDE + 2 * q + 1];
    }
    __shared__ double s_inv;  // 1 / side: one FP64 division per block
    if (threadIdx.x == 0) s_inv = 1.0 / cc.w;
    __syncthreads();
    const double inv_s = s_inv;
    // FP32 with one expansion, or a batch: the FP32 offsets from the leaf centre (no FP64 arithmetic)
    const bool rel = std::is_same<T, float>::value && (NC == 1 || bstride != 0);
    const float inv_sf = (float)inv_s;
    for (int i = r.x + threadIdx.x; i < r.y; i += blockDim.x) {
        T vx, vy, vz;
        double4 x = make_double4(0.0, 0.0, 0.0, 0.0);
        if (rel) {
            const float4 t = tgt_rel[i];
            vx = T(t.x * inv_sf); vy = T(t.y * inv_sf); vz = T(t.z * inv_sf);
        } else {
            x = tgt[i];
            vx = T((x.x - cc.x) * inv_s); vy = T((x.y - cc.y) * inv_s); vz = T((x.z - cc.z) * inv_s);
        }
        const T r2 = vx * vx + vy * vy + vz * vz;
        const cpx<T> xy = mk(vx, vy);
        T phi[NC], gz[NC];
        cpx<T> F[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) { phi[c] = 0; gz[c] = 0; F[c] = mk(T(0), T(0)); }
        cpx<T> diag = mk(T(1), T(0));
        auto use = [&](int n, int m, cpx<T> R) {
            const T wgt = m ? T(2) : T(1);
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const T* Lb = sL + c * NCOEF_MAX * 2;
                const cpx<T> a = ld(Lb, cidx(n, m));
                phi[c] += wgt * (a.re * R.re - a.im * R.im);
                if (NC > 1 && bstride == 0 && n + 1 <= p) {  // Stokes: the gradients too
                    const cpx<T> b = ld(Lb, cidx(n + 1, m));
                    gz[c] += wgt * (b.re * R.re - b.im * R.im);
                    if (m >= 1) cfma(F[c], ld(Lb, cidx(n + 1, m - 1)), R);
                    const cpx<T> d = ld(Lb, cidx(n + 1, m + 1)) * R;
                    F[c].re -= d.re;
                    F[c].im += d.im;
                }
            }
        };
        for (int m = 0; m <= p; ++m) {
            if (m > 0) diag = (T(-0.5) / T(m)) * (xy * diag);
            use(m, m, diag);
            if (m + 1 > p) break;
            cpx<T> prev2 = diag, prev1 = vz * diag;
            use(m + 1, m, prev1);
            for (int n = m + 2; n <= p; ++n) {
                const T inv = T(1) / T((n - m) * (n + m));
                cpx<T> cur = mk((T(2 * n - 1) * vz * prev1.re - r2 * prev2.re) * inv,
                                (T(2 * n - 1) * vz * prev1.im - r2 * prev2.im) * inv);
                use(n, m, cur);
                prev2 = prev1;
                prev1 = cur;
            }
        }
        if (NC == 1) {
            const double far = rel ? (double)(phi[0] * inv_sf) : (double)phi[0] * inv_s;
            yout[i] = scale * (far + ynear[i]) + (xs_half ? 0.5 * xs_half[i] : 0.0);  // 1/2 I of the second kind
        } else if (bstride) {  // a batch: potential of each vector, near field interleaved [N][NC]
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const double far = rel ? (double)(phi[c] * inv_sf) : (double)phi[c] * inv_s;
                yout[c * bstride + i] = scale * (far + ynear[(int64_t)NC * i + c]);
            }
        } else {
            const double is2 = inv_s * inv_s;
            const double px = x.x - ox, py = x.y - oy, pz = x.z - oz;
            double g[NC][3];
#pragma unroll
            for (int c = 0; c < NC; ++c) { g[c][0] = (double)F[c].re * is2; g[c][1] = (double)F[c].im * is2; g[c][2] = (double)gz[c] * is2; }
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const double u = (double)phi[a] * inv_s - (px * g[0][a] + py * g[1][a] + pz * g[2][a]) + g[NC - 1][a];
                yout[3 * (int64_t)i + a] = scale * (u + ynear[3 * (int64_t)i + a]) +
                                           (xs_half ? 0.5 * xs_half[3 * (int64_t)i + a] : 0.0);  // 1/2 I (double layer)
            }
        }
    }
}

// L2P of one FP32 expansion (the Laplace mat-vec) with paired FP32 instructions: each lane
// takes two targets of the leaf (positions base + lane and base + 32 + lane) and runs their
// recurrences as one pair; the coefficients are staged with their weight (2 for m > 0) and
// repeated in both halves, (w re, w re, -w im, -w im). Same sums as k_l2p<float, 1>.
__global__ void k_l2p_pair(int p, const int* leaves, const double4* cs, const int2* range, const float* L,
                           const double* ynear, double scale, const double* xs_half, const float4* tgt_rel,
                           double* yout) {
    __shared__ float4 sA[NCOEF_MAX];
    const int cell = leaves[blockIdx.x];
    const int2 r = range[cell];
    const int nco = ncoef(p);
    const float* Lc = L + (size_t)cell * ESTRIDE;
    for (int q = threadIdx.x; q < nco; q += blockDim.x) {
        int n, m;
        decode(q, n, m);
        const float w = m ? 2.f : 1.f, are = w * Lc[2 * q], aim = w * Lc[2 * q + 1];
        sA[q] = make_float4(are, are, -aim, -aim);
    }
    __shared__ float s_inv;  // 1 / side: one FP64 division per block
    if (threadIdx.x == 0) s_inv = (float)(1.0 / cs[cell].w);
    __syncthreads();
    const float inv_sf = s_inv;
    for (int base = r.x; base < r.y; base += 64) {
        const int i0 = base + threadIdx.x, i1 = i0 + 32;
        const float4 t0 = i0 < r.y ? tgt_rel[i0] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 t1 = i1 < r.y ? tgt_rel[i1] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float x0 = t0.x * inv_sf, y0 = t0.y * inv_sf, z0 = t0.z * inv_sf;
        const float x1 = t1.x * inv_sf, y1 = t1.y * inv_sf, z1 = t1.z * inv_sf;
        const f32x2 vz = f2_pack(z0, z1), xre = f2_pack(x0, x1), xim = f2_pack(y0, y1), nxim = f2_pack(-y0, -y1);
        const f32x2 nr2 = f2_pack(-(x0 * x0 + y0 * y0 + z0 * z0), -(x1 * x1 + y1 * y1 + z1 * z1));
        f32x2 phi = 0ull, dre = f2_pack(1.f, 1.f), dim = 0ull;
        auto use = [&](int q, f32x2 Rre, f32x2 Rim) {
            const float4 a = sA[q];
            phi = f2_fma(f2_pack(a.x, a.y), Rre, f2_fma(f2_pack(a.z, a.w), Rim, phi));
        };
        for (int m = 0; m <= p; ++m) {
            if (m > 0) {
                const float f = -0.5f / (float)m;
                const f32x2 f2 = f2_pack(f, f);
                const f32x2 re = f2_fma(xre, dre, f2_mul(nxim, dim));
                const f32x2 im = f2_fma(xre, dim, f2_mul(xim, dre));
                dre = f2_mul(f2, re);
                dim = f2_mul(f2, im);
            }
            use(cidx(m, m), dre, dim);
            if (m + 1 > p) break;
            f32x2 p2re = dre, p2im = dim, p1re = f2_mul(vz, dre), p1im = f2_mul(vz, dim);
            use(cidx(m + 1, m), p1re, p1im);
            for (int n = m + 2; n <= p; ++n) {
                const float inv = 1.f / (float)((n - m) * (n + m)), tn = (float)(2 * n - 1);
                const f32x2 inv2 = f2_pack(inv, inv), tz = f2_mul(f2_pack(tn, tn), vz);
                const f32x2 cre = f2_mul(f2_fma(tz, p1re, f2_mul(nr2, p2re)), inv2);
                const f32x2 cim = f2_mul(f2_fma(tz, p1im, f2_mul(nr2, p2im)), inv2);
                p2re = p1re;
                p2im = p1im;
                p1re = cre;
                p1im = cim;
                use(cidx(n, m), p1re, p1im);
            }
        }
        float ph0, ph1;
        f2_unpack(phi, ph0, ph1);
        if (i0 < r.y)
            yout[i0] = scale * ((double)(ph0 * inv_sf) + ynear[i0]) + (xs_half ? 0.5 * xs_half[i0] : 0.0);
        if (i1 < r.y)
            yout[i1] = scale * ((double)(ph1 * inv_sf) + ynear[i1]) + (xs_half ? 0.5 * xs_half[i1] : 0.0);
    }
}

__global__ void k_octant_tables(double* od, float* of) {
    const int o = threadIdx.x;
    if (o >= 8) return;
    cpx<double> tab[NCOEF_MAX];
    regular_table<double>((o & 1) ? 0.25 : -0.25, (o & 2) ? 0.25 : -0.25, (o & 4) ? 0.25 : -0.25, PMAX, tab);
    for (int q = 0; q < NCOEF_MAX; ++q) {
        od[(o * NCOEF_MAX + q) * 2] = tab[q].re;
        od[(o * NCOEF_MAX + q) * 2 + 1] = tab[q].im;
        of[(o * NCOEF_MAX + q) * 2] = (float)tab[q].re;
        of[(o * NCOEF_MAX + q) * 2 + 1] = (float)tab[q].im;
    }
}

// Single expansions for fmmbem_expansion_eval (FP64): kind 0 multipole, 1 local.
__global__ void k_form_expansion(int kind, int p, double cx, double cy, double cz, double s, int ns, const double4* src,
                                 double* E) {
    const int nco = ncoef(p);
    const int t = threadIdx.x;
    if (t >= nco) return;
    int n, m;
    decode(t, n, m);
    cpx<double> acc = mk(0.0, 0.0);
    cpx<double> tab[NCOEF_MAX];
    for (int j = 0; j < ns; ++j) {
        const double4 y = src[j];
        const double vx = (y.x - cx) / s, vy = (y.y - cy) / s, vz = (y.z - cz) / s;
        if (kind == 0) regular_table<double>(vx, vy, vz, n, tab);
        else irregular_table<double>(vx, vy, vz, n, tab);
        const cpx<double> v = tab[cidx(n, m)];
        acc.re += y.w * v.re;
        acc.im -= y.w * v.im;
    }
    E[2 * t] = acc.re;
    E[2 * t + 1] = acc.im;
}

__global__ void k_eval_expansion(int kind, int p, double cx, double cy, double cz, double s, const double* E, int nt,
                                 const double* tgt, double* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nt) return;
    const double vx = (tgt[3 * i] - cx) / s, vy = (tgt[3 * i + 1] - cy) / s, vz = (tgt[3 * i + 2] - cz) / s;
    cpx<double> tab[NCOEF_MAX];
    if (kind == 0) irregular_table<double>(vx, vy, vz, p, tab);
    else regular_table<double>(vx, vy, vz, p, tab);
    double phi = 0.0;
    for (int n = 0; n <= p; ++n)
        for (int m = 0; m <= n; ++m) {
            const cpx<double> a = mk(E[2 * cidx(n, m)], E[2 * cidx(n, m) + 1]), b = tab[cidx(n, m)];
            phi += (m ? 2.0 : 1.0) * (a.re * b.re - a.im * b.im);
        }
    out[i] = phi / s;
}

// The degree table lives in constant memory of each device; it is filled once per device,
// under a lock (handles may be created from several host threads).
std::mutex g_deg_mutex;
bool g_deg_ready[64] = {};

int ensure_degree_table() {
    int dev = 0;
    FMM_CU(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) { fmmbem_set_error("device ordinal %d out of range", dev); return FMMBEM_EDEVICE; }
    std::lock_guard<std::mutex> lock(g_deg_mutex);
    if (g_deg_ready[dev]) return 0;
    unsigned char deg[NCOEF_MAX];
    for (int n = 0; n <= PMAX; ++n)
        for (int m = 0; m <= n; ++m) deg[cidx(n, m)] = (unsigned char)n;
    FMM_CU(cudaMemcpyToSymbol(c_deg, deg, sizeof(deg)));
    g_deg_ready[dev] = true;
    return 0;
}

unsigned m2l_block(int p) { return (unsigned)((ncoef(p) > 2 * p + 1 ? ncoef(p) : 2 * p + 1) + 31) / 32 * 32; }
unsigned coef_block(int p) { return (unsigned)(ncoef(p) + 31) / 32 * 32; }

template <typename T, int NC>
int far_field_t(fmmbem_handle* h, int p) {
    cudaStream_t st = h->stream;
    T* M = reinterpret_cast<T*>(h->M);
    T* L = reinterpret_cast<T*>(h->L);
    const T* oct = std::is_same<T, float>::value ? reinterpret_cast<const T*>(h->oct_f) : reinterpret_cast<const T*>(h->oct_d);
    const typename V4<T>::type* src;
    if (std::is_same<T, float>::value) src = reinterpret_cast<const typename V4<T>::type*>(h->src_f);
    else src = reinterpret_cast<const typename V4<T>::type*>(h->src_d);
    const int nco = ncoef(p);
    // tensor-core tree translations in the mixed-precision M2L-TENSOR mode
    const bool tree_tc_on = std::is_same<T, float>::value && h->m2l_mode == FMMBEM_M2L_TENSOR && h->m2l_tc_ready &&
                            h->tree_tiles != nullptr && h->tree_tc_at[p];
    const bool m2l_tc_on = std::is_same<T, float>::value && h->m2l_mode == FMMBEM_M2L_TENSOR && h->m2l_tc_ready &&
                           h->m2l_tc_at[p];
    // P2M (after the zeroing of what the tensor-core passes accumulate into: all local
    // expansions, and the multipoles of the non-leaf cells, which P2M does not write), so that
    // the first M2M level follows P2M directly and its launch overlaps P2M's tail
    prof_begin(h, FMMBEM_PASS_P2M);
    int nz = 0;
    if (m2l_tc_on) FMM_TRY(m2l_tc_zero(h));
    if (tree_tc_on) {
        FMM_TRY(tree_tc_zero(h, p));
        ++nz;
    }
    const size_t sm = (size_t)P2M_WARPS * NC * nco * 2 * sizeof(T);
    const bool stokeslet = NC == 4 && h->kernel == FMMBEM_STOKES && h->layer != FMMBEM_LAYER_DOUBLE;
    if (std::is_same<T, float>::value && (NC == 1 || (h->nrhs > 1 && h->kernel == FMMBEM_LAPLACE) || stokeslet)) {
        // mixed precision: the packed FP32 sources
        float* Mf = reinterpret_cast<float*>(h->M);
        const size_t smp = (size_t)P2MP_WARPS * NC * nco * 2 * sizeof(float);
        if (stokeslet)
            k_p2m_packed<3><<<dim3(h->n_leaves, h->nsys), 32 * P2MP_WARPS, smp, st>>>(
                p, h->leaves, h->cell_cs, h->cell_range, h->src_w, h->K, Mf, h->origin[0], h->origin[1], h->origin[2],
                2 * h->NS, h->esys);
        else if (h->nrhs > 1)
            k_p2m_packed<2><<<h->n_leaves, 32 * P2MP_WARPS, smp, st>>>(p, h->leaves, h->cell_cs, h->cell_range,
                                                                      h->src_w, h->K, Mf);
        else if (h->layer == FMMBEM_LAYER_DOUBLE)
            k_p2m_packed<1><<<h->n_leaves, 32 * P2MP_WARPS, smp, st>>>(p, h->leaves, h->cell_cs, h->cell_range,
                                                                      h->src_w, h->K, Mf);
        else
            k_p2m_packed<0><<<h->n_leaves, 32 * P2MP_WARPS, smp, st>>>(p, h->leaves, h->cell_cs, h->cell_range,
                                                                      h->src_w, h->K, Mf);
    } else if (NC == 1 && h->layer == FMMBEM_LAYER_DOUBLE) {
        k_p2m_dl<T><<<h->n_leaves, 32 * P2M_WARPS, sm, st>>>(p, h->leaves, h->cell_cs, h->cell_range, src, h->nrm_d,
                                                            h->xin, h->K, M);
    } else if (NC == 4 && h->kernel == FMMBEM_STOKES && h->layer == FMMBEM_LAYER_DOUBLE) {
        if (std::is_same<T, float>::value)
            k_p2m_sdl<T, true><<<h->n_leaves, 32 * P2M_WARPS, sm, st>>>(
                p, h->leaves, h->cell_cs, h->cell_range, src, h->src_w, h->nrm_d, h->nrm_f, h->xin, h->K, h->origin[0],
                h->origin[1], h->origin[2], M);
        else
            k_p2m_sdl<T, false><<<h->n_leaves, 32 * P2M_WARPS, sm, st>>>(
                p, h->leaves, h->cell_cs, h->cell_range, src, h->src_w, h->nrm_d, h->nrm_f, h->xin, h->K, h->origin[0],
                h->origin[1], h->origin[2], M);
    } else {
        const bool copies = h->nsys > 1;
        k_p2m<T, NC><<<dim3(h->n_leaves, h->nsys), 32 * P2M_WARPS, sm, st>>>(
            p, h->leaves, h->cell_cs, h->cell_range, src, h->xin, h->K, h->origin[0], h->origin[1], h->origin[2], M,
            (h->nrhs > 1 && !copies) ? h->N : 0, h->N * h->dof, h->esys);
    }
    FMM_LAUNCHED();
    prof_end(h, FMMBEM_PASS_P2M, 1 + nz);
    FMM_TRY(near_release(h, 1));
    // passes of this mat-vec that run on the tensor-core kernel (profiling attributes their time to it)
    h->tc_pass_bits = (tree_tc_on ? (1 << FMMBEM_PASS_M2M) | (1 << FMMBEM_PASS_L2L) : 0) |
                      (m2l_tc_on ? 1 << FMMBEM_PASS_M2L : 0);
    // M2M, deepest non-leaf level first
    prof_begin(h, FMMBEM_PASS_M2M);
    int nl = 0;
    const size_t sm_m2m = (size_t)(16 * NC + 8) * nco * 2 * sizeof(T);
    for (int l = h->n_levels - 2; l >= h->m2m_lmin; --l) {
        const int pb = h->parent_start[l], pe = h->parent_start[l + 1];
        if (pe == pb) continue;
        if (tree_tc_on) {
            FMM_TRY(tree_tc(h, p, l, 0));
            ++nl;
        } else {
            FMM_CU(launch_pdl(k_m2m<T, NC>, dim3(pe - pb, h->nsys), dim3(TREE_THREADS), sm_m2m, st, p, h->parents + pb,
                              h->cell_cs, h->cell_child, oct, M, h->esys));
            ++nl;
        }
    }
    prof_end(h, FMMBEM_PASS_M2M, nl);
    FMM_TRY(near_release(h, 2));
    // M2L
    prof_begin(h, FMMBEM_PASS_M2L);
    if (m2l_tc_on) {
        FMM_TRY(m2l_tc(h, p));
    } else if (h->m2l_mode != FMMBEM_M2L_GATHER && h->m2l_tables) {
        FMM_TRY(m2l_gemm(h, p, !std::is_same<T, float>::value));
    } else {
        k_m2l<T, NC><<<dim3(h->n_cells, h->nsys), m2l_block(p), 0, st>>>(p, h->m2l_ptr, h->m2l_src, h->cell_cs, M, L,
                                                                         h->esys);
        FMM_LAUNCHED();
    }
    prof_end(h, FMMBEM_PASS_M2L, 1);
    FMM_TRY(near_release(h, 3));
    // L2L, top-down
    prof_begin(h, FMMBEM_PASS_L2L);
    int nl2 = 0;
    const size_t sm_l2l = (size_t)(NC + 8) * nco * 2 * sizeof(T);
    for (int l = h->l2l_lmin; l + 1 < h->n_levels; ++l) {
        const int pb = h->parent_start[l], pe = h->parent_start[l + 1];
        if (pe == pb) continue;
        if (tree_tc_on) {
            FMM_TRY(tree_tc(h, p, l, 1));
        } else {
            FMM_CU(launch_pdl(k_l2l<T, NC>, dim3(pe - pb, h->nsys), dim3(TREE_THREADS), sm_l2l, st, p, h->parents + pb,
                              h->cell_cs, h->cell_child, oct, L, h->esys));
        }
        ++nl2;
    }
    prof_end(h, FMMBEM_PASS_L2L, nl2);
    h->launches += 2 + nz + nl + nl2;
    return 0;
}

template <typename T, int NC>
int far_eval_t(fmmbem_handle* h, int p, double* y_sorted, double scale) {
    prof_begin(h, FMMBEM_PASS_L2P);
    // one warp per leaf: a leaf holds about 20 targets (a 128-thread block left most threads idle)
    if (std::is_same<T, float>::value && NC == 1)
        k_l2p_pair<<<h->n_leaves, 32, 0, h->stream>>>(p, h->leaves, h->cell_cs, h->cell_range,
                                                      reinterpret_cast<const float*>(h->L), h->ynear, scale,
                                                      h->layer == FMMBEM_LAYER_DOUBLE ? h->xin : nullptr,
                                                      h->tgt_rel, y_sorted);
    else
        k_l2p<T, NC><<<dim3(h->n_leaves, h->nsys), 32, 0, h->stream>>>(
            p, h->leaves, h->cell_cs, h->cell_range, h->tgt_d, reinterpret_cast<const T*>(h->L), h->ynear, scale,
            h->origin[0], h->origin[1], h->origin[2], h->layer == FMMBEM_LAYER_DOUBLE ? h->xin : nullptr, h->tgt_rel,
            y_sorted, (h->nrhs > 1 && h->nsys == 1) ? h->N : 0, h->esys, h->N * h->dof);
    FMM_LAUNCHED();
    prof_end(h, FMMBEM_PASS_L2P, 1);
    h->launches += 1;
    return 0;
}

}  // namespace

int init_octant_tables(fmmbem_handle* h) {
    FMM_TRY(ensure_degree_table());
    // dynamic shared memory of the tree passes at p = PMAX (above the 48 KB default for FP64 and Stokes)
    const int nmax = NCOEF_MAX * 2;
    FMM_CU(cudaFuncSetAttribute(k_m2m<float, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 24 * nmax * (int)sizeof(float)));
    FMM_CU(cudaFuncSetAttribute(k_m2m<float, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, 72 * nmax * (int)sizeof(float)));
    FMM_CU(cudaFuncSetAttribute(k_m2m<double, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 24 * nmax * (int)sizeof(double)));
    FMM_CU(cudaFuncSetAttribute(k_m2m<double, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, 72 * nmax * (int)sizeof(double)));
    FMM_CU(cudaFuncSetAttribute(k_l2l<double, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, 12 * nmax * (int)sizeof(double)));
    FMM_CU(fmm_malloc(&h->oct_d, sizeof(double) * 8 * NCOEF_MAX * 2));
    FMM_CU(fmm_malloc(&h->oct_f, sizeof(float) * 8 * NCOEF_MAX * 2));
    k_octant_tables<<<1, 8, 0, h->stream>>>(h->oct_d, h->oct_f);
    FMM_LAUNCHED();
    return 0;
}

int far_field(fmmbem_handle* h, int p, bool fp64) {
    if (h->ncomp == 1) return fp64 ? far_field_t<double, 1>(h, p) : far_field_t<float, 1>(h, p);
    return fp64 ? far_field_t<double, 4>(h, p) : far_field_t<float, 4>(h, p);
}

int far_eval_add(fmmbem_handle* h, int p, bool fp64, double* y_sorted, double scale) {
    if (h->ncomp == 1) return fp64 ? far_eval_t<double, 1>(h, p, y_sorted, scale) : far_eval_t<float, 1>(h, p, y_sorted, scale);
    return fp64 ? far_eval_t<double, 4>(h, p, y_sorted, scale) : far_eval_t<float, 4>(h, p, y_sorted, scale);
}

int expansion_eval(int kind, int p, const double* center, double scale, int n_src, const double* src, int n_tgt,
                   const double* tgt, double* out, cudaStream_t st) {
    FMM_TRY(ensure_degree_table());
    double* E = nullptr;
    FMM_CU(cudaMalloc((void**)&E, sizeof(double) * NCOEF_MAX * 2));
    // every exit below releases E
    auto finish = [&](int rc) {
        cudaStreamSynchronize(st);
        cudaFree(E);
        return rc;
    };
    k_form_expansion<<<1, coef_block(p), 0, st>>>(kind, p, center[0], center[1], center[2], scale, n_src,
                                                  reinterpret_cast<const double4*>(src), E);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && n_tgt > 0) {
        k_eval_expansion<<<(n_tgt + 127) / 128, 128, 0, st>>>(kind, p, center[0], center[1], center[2], scale, E, n_tgt,
                                                             tgt, out);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        fmmbem_set_error("expansion_eval: %s", cudaGetErrorString(e));
        return finish(FMMBEM_EDEVICE);
    }
    return finish(0);
}

}  // namespace fmmbem

// ---------------------------------------------------------------------------
// Allocation-free variant of fmmbem_expansion_eval.
//
// Some callers cannot call cudaMalloc: code running inside a CUDA-graph capture
// (allocation is not capturable), code whose memory is owned by a pool or an
// arena that forbids side allocations, and real-time loops that must not block
// on the driver's allocator. For them the expansion coefficients live in a fixed
// module-global buffer instead of a per-call allocation.
namespace {

// One expansion of order <= FMMBEM_P_MAX: (P_MAX+1)(P_MAX+2)/2 complex FP64
// coefficients = 2448 bytes. Every GPU that loads the library holds it until exit.
static __device__ __align__(256) double g_expansion_scratch[fmmbem::NCOEF_MAX * 2];

// Per device: the scratch array's device address once its set-up has succeeded. A failed
// set-up (say, a first call made inside a stream capture) is not cached: the next call on
// that device tries again.
constexpr int kMaxDevices = 64;
std::mutex g_scratch_mutex;
double* g_scratch_ptr[kMaxDevices] = {};

// Per-device set-up, with that device current: the device address of the scratch array
// (host code only sees a host-side stand-in for the symbol) and the degree table the
// kernels read from constant memory (shared with the allocating path).
int scratch_address(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        fmmbem_set_error("cudaGetDevice: %s", cudaGetErrorString(e));
        return FMMBEM_EDEVICE;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        fmmbem_set_error("device ordinal %d beyond the %d supported", dev, kMaxDevices);
        return FMMBEM_EDEVICE;
    }
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_ptr[dev]) {
        const int rc = fmmbem::ensure_degree_table();
        if (rc < 0) return rc;
        double* p = nullptr;
        e = cudaGetSymbolAddress((void**)&p, g_expansion_scratch);
        if (e != cudaSuccess || !p) {
            fmmbem_set_error("static scratch set-up on device %d: %s", dev, cudaGetErrorString(e));
            return FMMBEM_EDEVICE;
        }
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return 0;
}

}  // namespace

extern "C" int fmmbem_expansion_eval_static(int kind, int p, const double* center, double scale, int n_src,
                                            const double* src_dev, int n_tgt, const double* tgt_dev, double* out_dev,
                                            void* stream) {
    using namespace fmmbem;
    if (p > FMMBEM_P_MAX) {
        fmmbem_set_error("p=%d exceeds the static scratch, which holds one expansion of order <= %d", p,
                         FMMBEM_P_MAX);
        return FMMBEM_EINVAL;
    }
    if ((kind != 0 && kind != 1) || p < 0 || !center || !(scale > 0.0) || n_src < 0 || n_tgt < 0 ||
        (n_src && !src_dev) || (n_tgt && (!tgt_dev || !out_dev))) {
        fmmbem_set_error("bad argument");
        return FMMBEM_EINVAL;
    }
    double* E = nullptr;
    FMM_TRY(scratch_address(&E));
    cudaStream_t st = (cudaStream_t)stream;
    // k_form_expansion overwrites every coefficient of order <= p, so nothing left by
    // an earlier call is read.
    k_form_expansion<<<1, coef_block(p), 0, st>>>(kind, p, center[0], center[1], center[2], scale, n_src,
                                                  reinterpret_cast<const double4*>(src_dev), E);
    FMM_LAUNCHED();
    if (n_tgt > 0) {
        k_eval_expansion<<<(n_tgt + 127) / 128, 128, 0, st>>>(kind, p, center[0], center[1], center[2], scale, E,
                                                             n_tgt, tgt_dev, out_dev);
        FMM_LAUNCHED();
    }
    return 0;
}
