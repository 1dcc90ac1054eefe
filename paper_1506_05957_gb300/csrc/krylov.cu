// Relaxed restarted GMRES(m) (Sec. 2.4 and 2.6) with the Krylov recurrence in FP64.
// Arnoldi: classical Gram-Schmidt with selective reorthogonalization (a second pass only
// when the first one cancels more than half of ||w||^2), as batched dot products and a
// fused update-and-normalize sweep, all on the device; the (m+1) x m Hessenberg column,
// Givens rotations and the residual estimate rho_k = |g_{k+1}| / ||b|| live on the
// host (k+3 doubles cross per step). Step k runs the mat-vec at
//   p_k = min(p_initial, max(p_min, ceil(-log2 eps_k))),
//   eps_k = min(tol / min(rho_{k-1}, 1), 1)                (eqs. matrix-perturbation, fmm_p)
// when relaxation is on, else at p_initial. Restart residuals and the final true
// residual use p_initial.
#include <math.h>
#include <algorithm>
#include <cmath>
#include <vector>
#include "handle.cuh"

namespace fmmbem {

namespace {

constexpr int DOT_BLOCKS = 96;
constexpr int DOT_THREADS = 256;

// partial[j * gridDim.x + bx] = sum over this block's rows of V_j[i] w[i]
__global__ void k_dots(const double* V, int64_t ldv, const double* w, int64_t n, double* partial) {
    __shared__ double red[DOT_THREADS];
    const int j = blockIdx.y;
    const double* v = V + (int64_t)j * ldv;
    const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
    const int64_t i0 = (int64_t)blockIdx.x * chunk, i1 = min(n, i0 + chunk);
    double s = 0.0;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += DOT_THREADS) s += v[i] * w[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = DOT_THREADS / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[(int64_t)j * gridDim.x + blockIdx.x] = red[0];
}

__global__ void k_reduce(const double* partial, int nb, int nv, double* out) {
    const int j = threadIdx.x;
    if (j >= nv) return;
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += partial[j * nb + b];
    out[j] = s;
}

// w[i] -= sum_j c[j] V_j[i]
__global__ void k_sub_combo(double* w, const double* V, int64_t ldv, int nv, const double* c, int64_t n) {
    __shared__ double sc[64];
    if (threadIdx.x < nv) sc[threadIdx.x] = c[threadIdx.x];
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int j = 0; j < nv; ++j) s += sc[j] * V[(int64_t)j * ldv + i];
        w[i] -= s;
    }
}

// x[i] += sum_j c[j] V_j[i]
__global__ void k_add_combo(double* x, const double* V, int64_t ldv, int nv, const double* c, int64_t n) {
    __shared__ double sc[64];
    if (threadIdx.x < nv) sc[threadIdx.x] = c[threadIdx.x];
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int j = 0; j < nv; ++j) s += sc[j] * V[(int64_t)j * ldv + i];
        x[i] += s;
    }
}

// dst = a src, and a second copy in dst2 (the fixed input buffer of the next mat-vec)
__global__ void k_scale(double* dst, double* dst2, const double* src, double a, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = a * src[i];
        dst[i] = v;
        dst2[i] = v;
    }
}

// x += d
__global__ void k_add(double* x, const double* d, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] += d[i];
}

__global__ void k_sub(double* r, const double* b, const double* ax, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        r[i] = b[i] - ax[i];
}

// ---- fused Arnoldi step: the projections, the norm and the new basis vector in one
// cooperative launch (all blocks co-resident). Between phases the blocks
// meet at a sense-reversal grid barrier whose wait is bounded: on timeout the kernel
// flags an error and stops. Each block reduces the per-block partial dots itself in a
// fixed order (results are deterministic); block 0 writes h1, h2 and ||w||^2 to out
// (mapped pinned host memory).
constexpr int ARN_THREADS = 512;
constexpr int ARN_MAXV = 64;

__device__ __forceinline__ bool grid_barrier(unsigned* count, volatile unsigned* gen, unsigned nb, int* err,
                                             unsigned limit) {
    __syncthreads();
    bool ok = true;
    if (threadIdx.x == 0) {
        const unsigned g = *gen;
        __threadfence();
        if (atomicAdd(count, 1u) == nb - 1) {
            *count = 0;
            __threadfence();
            atomicAdd((unsigned*)gen, 1u);
        } else {
            unsigned it = 0;
            while (*gen == g) {
                if (++it > limit) { atomicExch(err, 5); ok = false; break; }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    __shared__ int s_ok;
    if (threadIdx.x == 0) s_ok = ok;
    __syncthreads();
    return s_ok != 0;
}

// FP64 throughput is scarce on this GPU: two FP64 operations per clock per SM, so a warp-wide
// FP64 instruction holds its sub-partition's FP64 unit for 64 clocks. The helpers below spend
// about one FP64 operation per vector element, keep the reductions short (one entry per
// vector per block) and leave scalar FP64 work to a single thread.

// partial[j * nbk + bk] = sum over the block's rows of V_j w. One warp per vector: its lanes
// stride over the block's rows with four independent accumulators (eight loads in flight per
// lane), then one five-level shuffle reduction. With with_self the vector after the last V_j
// is w itself (entry nv is w.w), so ||w||^2 comes from the same sweep. When the block has more
// warps than vectors, each vector's rows are cut into ns slices (one warp each) whose sums are
// added in shared memory (sred, one double per warp) before the block writes its entry.
// Fixed summation order: deterministic.
__device__ __forceinline__ int arn_slices(int nt) {
    const int nw = (int)(blockDim.x >> 5);
    return nw > nt ? nw / nt : 1;
}

// nbk, bk: the blocks that share this system and this block's index among them.
__device__ void arn_partials(const double* V, int64_t ldv, int nv, const double* w, int64_t i0, int64_t i1,
                             double* partial, int nbk, int bk, bool with_self, double* sred) {
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
    const int nt = nv + (with_self ? 1 : 0);
    const int ns = arn_slices(nt);
    const int64_t len = (i1 - i0 + ns - 1) / ns;
    for (int item = wp; item < nt * ns; item += nw) {
        const int j = item / ns, sl = item - j * ns;
        const double* vj = j < nv ? V + (int64_t)j * ldv : w;
        const int64_t a = i0 + sl * len, e = min(i1, a + len);
        double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
        int64_t i = a + lane;
        for (; i + 96 < e; i += 128) {
            s0 = fma(vj[i], w[i], s0);
            s1 = fma(vj[i + 32], w[i + 32], s1);
            s2 = fma(vj[i + 64], w[i + 64], s2);
            s3 = fma(vj[i + 96], w[i + 96], s3);
        }
        for (; i < e; i += 32) s0 = fma(vj[i], w[i], s0);
        double t = (s0 + s1) + (s2 + s3);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (ns == 1) {
            if (lane == 0) partial[(int64_t)j * nbk + bk] = t;
        } else if (lane == 0) {
            sred[item] = t;
        }
    }
    if (ns > 1) {
        __syncthreads();
        if ((int)threadIdx.x < nt) {
            const int j = threadIdx.x;
            double t = sred[j * ns];
            for (int sl = 1; sl < ns; ++sl) t += sred[j * ns + sl];
            partial[(int64_t)j * nbk + bk] = t;
        }
    }
}

// hs[j] = sum over the system's blocks of partial[j][.] (one warp per j, fixed order); every block forms
// the same hs. With sq != nullptr, *sq = sum_{j < nsq} hs[j]^2, by one warp.
__device__ void arn_reduce(const double* partial, int nv, int nbk, double* hs, int nsq = 0, double* sq = nullptr) {
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    for (int j = wp; j < nv; j += (int)(blockDim.x >> 5)) {
        double t = 0.0;
        for (int b = lane; b < nbk; b += 32) t += partial[(int64_t)j * nbk + b];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) hs[j] = t;
    }
    __syncthreads();
    if (sq && wp == 0) {
        double t = 0.0;
        for (int j = lane; j < nsq; j += 32) t = fma(hs[j], hs[j], t);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) *sq = t;
    }
    if (sq) __syncthreads();
}

// w[i] -= sum_j hs[j] V_j[i] over the block's rows (eight independent loads per full group,
// then the remaining vectors one by one: exactly nv FP64 multiply-adds per row); with
// scale != 0 the result is also multiplied by scale and written to V_{k+1} and xfix.
__device__ void arn_update(const double* V, int64_t n, int nv, const double* hs, double* w, int64_t i0, int64_t i1,
                           double scale, double* vk1, double* xfix) {
    const int full = nv & ~7;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        double t = 0.0;
        for (int j0 = 0; j0 < full; j0 += 8) {
            double v[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) v[q] = V[(int64_t)(j0 + q) * n + i];
#pragma unroll
            for (int q = 0; q < 8; ++q) t = fma(hs[j0 + q], v[q], t);
        }
        for (int j = full; j < nv; ++j) t = fma(hs[j], V[(int64_t)j * n + i], t);
        const double r = w[i] - t;
        if (scale != 0.0) {
            const double u = r * scale;
            vk1[i] = u;
            xfix[i] = u;
        } else {
            w[i] = r;
        }
    }
}

// Classical Gram-Schmidt with selective reorthogonalization (the criterion of Daniel,
// Gragg, Kaufman and Stewart): one sweep gives h = V^T w and ||w||^2; when
// ||w - V h||^2 = ||w||^2 - ||h||^2 stays above ||w||^2 / 2 the projected vector is
// normalized and written as V_{k+1} in the same sweep that forms it (one grid barrier).
// Otherwise a second projection pass follows (the CGS2 step), whose sweep also gives the
// explicit ||w - V h||^2 (two grid barriers in all).
// A launch may carry several systems of a batch: the grid is cut into nsys equal groups of
// blocks, group q working on system q (its basis at V + q * vstride, its vectors at
// w + q * wstride and xfix + q * wstride, its partial sums, barrier pair and output areas
// offset likewise). A system whose bit in active is clear does nothing (its whole group
// returns at once, so barrier counts stay consistent).
__global__ void __launch_bounds__(ARN_THREADS) k_arnoldi(double* V, int64_t n, int k, double* w, double* xfix,
                                                         double* partial, unsigned* bar, double* out, int* err,
                                                         int nsys, int64_t vstride, int64_t wstride,
                                                         unsigned active, unsigned wait_limit, const int* kdev) {
    if (kdev) k = *kdev;  // the device-resident cycle keeps the step index on the device
    __shared__ double hs[ARN_MAXV];
    __shared__ double h1[ARN_MAXV];
    const int nbk = (int)gridDim.x / nsys;
    const int sys = (int)blockIdx.x / nbk, bk = (int)blockIdx.x - sys * nbk;
    if (sys >= nsys || !((active >> sys) & 1u)) return;
    V += sys * vstride;
    w += sys * wstride;
    xfix += sys * wstride;
    const size_t parea = (size_t)ARN_MAXV * nbk;
    partial += (size_t)sys * 2 * parea;
    unsigned* bar_count = bar + 2 * sys;
    unsigned* bar_gen = bar + 2 * sys + 1;
    out += (size_t)sys * (2 * (ARN_MAXV + 1) + 1);
    const int nv = k + 1;
    const int64_t chunk = (n + nbk - 1) / nbk;
    const int64_t i0 = (int64_t)bk * chunk, i1 = min(n, i0 + chunk);
    // each phase has its own partial-sum area, so one grid barrier per phase suffices:
    // a block's w rows are read and written by that block alone
    double* vk1 = V + (int64_t)(k + 1) * n;
    // phase 1: h = V^T w and ||w||^2
    __shared__ double s_sq, s_scale;
    __shared__ int s_direct;
    __shared__ double sred[ARN_THREADS / 32];
    arn_partials(V, n, nv, w, i0, i1, partial, nbk, bk, true, sred);
    // a barrier that gives up marks the step's norm NaN in the output: the host stops there
    // and reports the flag set in err
    if (!grid_barrier(bar_count, bar_gen, (unsigned)nbk, err, wait_limit)) {
        if (threadIdx.x == 0) out[2 * (ARN_MAXV + 1)] = __longlong_as_double(0x7ff8000000000000ll);
        return;
    }
    arn_reduce(partial, nv + 1, nbk, hs, nv, &s_sq);
    // the scalar decisions in FP64 by one thread, broadcast through shared memory
    if (threadIdx.x == 0) {
        const double ww = hs[nv];
        const double nn2 = ww - s_sq;
        s_direct = nn2 > 0.5 * ww && nn2 > 0.0 && isfinite(nn2);
        s_scale = s_direct ? 1.0 / sqrt(nn2) : 0.0;
        if (bk == 0 && s_direct) out[2 * (ARN_MAXV + 1)] = nn2;
    }
    __syncthreads();
    if (bk == 0)
        for (int j = threadIdx.x; j < nv; j += blockDim.x) out[j] = hs[j];
    if (s_direct) {
        if (bk == 0)
            for (int j = threadIdx.x; j < nv; j += blockDim.x) out[(ARN_MAXV + 1) + j] = 0.0;
        arn_update(V, n, nv, hs, w, i0, i1, s_scale, vk1, xfix);
        return;
    }
    // phase 2: reorthogonalize. The sweep that projects w1 = w - V h1 again also gives
    // ||w1||^2 explicitly, so ||w1 - V h2||^2 = ||w1||^2 - ||h2||^2 has no cancellation to
    // fear (h2 is the small correction) and the new basis vector is normalized in the same
    // pass that forms it.
    for (int j = threadIdx.x; j < nv; j += blockDim.x) h1[j] = hs[j];
    __syncthreads();
    arn_update(V, n, nv, h1, w, i0, i1, 0.0, nullptr, nullptr);
    __syncthreads();  // arn_partials reads rows of w that other threads of the block updated
    double* part2 = partial + parea;
    arn_partials(V, n, nv, w, i0, i1, part2, nbk, bk, true, sred);
    if (!grid_barrier(bar_count, bar_gen, (unsigned)nbk, err, wait_limit)) {
        if (threadIdx.x == 0) out[2 * (ARN_MAXV + 1)] = __longlong_as_double(0x7ff8000000000000ll);
        return;
    }
    arn_reduce(part2, nv + 1, nbk, hs, nv, &s_sq);
    if (threadIdx.x == 0) {
        const double w1w1 = hs[nv];
        const double nrm2 = fmax(w1w1 - s_sq, 0.0);  // rounding below zero: w1 lies in the span (breakdown)
        const double hn = sqrt(nrm2);
        s_direct = hn > 0.0 && isfinite(hn);
        s_scale = s_direct ? 1.0 / hn : 0.0;
        if (bk == 0) out[2 * (ARN_MAXV + 1)] = nrm2;
    }
    __syncthreads();
    if (bk == 0)
        for (int j = threadIdx.x; j < nv; j += blockDim.x) out[(ARN_MAXV + 1) + j] = hs[j];
    if (s_direct) {
        arn_update(V, n, nv, hs, w, i0, i1, s_scale, vk1, xfix);
    } else {
        arn_update(V, n, nv, hs, w, i0, i1, 0.0, nullptr, nullptr);
    }
}

struct Kr {
    fmmbem_handle* h;
    int64_t n;
    unsigned gs;  // grid for streaming kernels
    int dots(const double* V, int nv, const double* w, double* out) {
        dim3 g(DOT_BLOCKS, nv);
        k_dots<<<g, DOT_THREADS, 0, h->stream>>>(V, n, w, n, h->kpart);
        FMM_LAUNCHED();
        k_reduce<<<1, 64, 0, h->stream>>>(h->kpart, DOT_BLOCKS, nv, out);
        FMM_LAUNCHED();
        h->launches += 2;
        return 0;
    }
    int sub(double* w, const double* V, int nv, const double* c) {
        k_sub_combo<<<gs, 256, 0, h->stream>>>(w, V, n, nv, c, n);
        FMM_LAUNCHED();
        h->launches += 1;
        return 0;
    }
};

__host__ __device__ int relaxed_p_int(double eta, double rho_prev, int p_initial, int p_min) {
    double eps = eta / (rho_prev < 1.0 ? rho_prev : 1.0);
    if (eps > 1.0) eps = 1.0;
    int p;
    if (eps >= 1.0) {
        p = 0;
    } else {
        int e;
        frexp(eps, &e);
        p = 1 - e;
    }
    if (p < p_min) p = p_min;
    if (p > p_initial) p = p_initial;
    return p;
}

// State of one device-resident GMRES cycle (the host loop's scalars, Hessenberg matrix,
// rotations and per-step records), written by k_dloop_begin and advanced by k_dloop_step.
struct KrylovDev {
    int k, it, m, max_iter, p_initial, p_min, relax, status;  // status: 0 running, 1 converged, 2 NaN, 3 cycle or budget ended
    int k_done, p_cur, pad0, pad1;
    double rho, bnorm, tol, pad2;
    double g[ARN_MAXV + 1], cs[ARN_MAXV], sn[ARN_MAXV];
    double H[(ARN_MAXV + 1) * ARN_MAXV];  // (i, j) at i * ARN_MAXV + j
    double res_c[ARN_MAXV];               // rho after each step of the cycle
    int p_c[ARN_MAXV];                    // order of each step's mat-vec
};

__global__ void k_dloop_begin(KrylovDev* s, int it, int m, int max_iter, int p_initial, int p_min, int relax, double tol,
                              double bnorm, double beta, double rho) {
    for (int i = threadIdx.x; i < (ARN_MAXV + 1) * ARN_MAXV; i += blockDim.x) s->H[i] = 0.0;
    for (int i = threadIdx.x; i <= ARN_MAXV; i += blockDim.x) s->g[i] = 0.0;
    __syncthreads();
    if (threadIdx.x == 0) {
        s->k = 0;
        s->it = it;
        s->m = m;
        s->max_iter = max_iter;
        s->p_initial = p_initial;
        s->p_min = p_min;
        s->relax = relax;
        s->status = 0;
        s->k_done = 0;
        s->rho = rho;
        s->bnorm = bnorm;
        s->tol = tol;
        s->g[0] = beta;
        s->p_cur = relax ? relaxed_p_int(tol, rho, p_initial, p_min) : p_initial;
    }
}

// First node of the cycle graph: the switch takes the first step's order.
__global__ void k_dloop_init(const KrylovDev* s, cudaGraphConditionalHandle hs) {
    if (threadIdx.x == 0) cudaGraphSetConditional(hs, (unsigned)s->p_cur);
}

// After each Arnoldi step: the host loop's column update, done by one thread in the same
// order and FP64 operations (Givens rotations, residual estimate, stopping tests, next order),
// then the switch's next order and whether the while node runs again.
__global__ void k_dloop_step(KrylovDev* s, const double* ao, cudaGraphConditionalHandle hw,
                             cudaGraphConditionalHandle hs) {
    if (threadIdx.x != 0) return;
    const int k = s->k;
    auto Hc = [&](int i, int j) -> double& { return s->H[i * ARN_MAXV + j]; };
    s->p_c[k] = s->p_cur;
    s->it += 1;
    for (int i = 0; i <= k; ++i) Hc(i, k) = ao[i] + ao[(ARN_MAXV + 1) + i];
    const double hn = sqrt(ao[2 * (ARN_MAXV + 1)]);
    Hc(k + 1, k) = hn;
    bool stop = false;
    if (!isfinite(hn)) {
        s->status = 2;
        s->k_done = k;
        stop = true;
    } else {
        for (int i = 0; i < k; ++i) {
            const double t = s->cs[i] * Hc(i, k) + s->sn[i] * Hc(i + 1, k);
            Hc(i + 1, k) = -s->sn[i] * Hc(i, k) + s->cs[i] * Hc(i + 1, k);
            Hc(i, k) = t;
        }
        const double den = hypot(Hc(k, k), Hc(k + 1, k));
        s->cs[k] = Hc(k, k) / den;
        s->sn[k] = Hc(k + 1, k) / den;
        Hc(k, k) = den;
        Hc(k + 1, k) = 0.0;
        s->g[k + 1] = -s->sn[k] * s->g[k];
        s->g[k] = s->cs[k] * s->g[k];
        const double rho = fabs(s->g[k + 1]) / s->bnorm;
        s->rho = rho;
        s->res_c[k] = rho;
        s->k_done = k + 1;
        if (!isfinite(rho)) {
            s->status = 2;
            stop = true;
        } else if (rho <= s->tol || hn == 0.0) {  // converged, or the exact solution is in the space
            s->status = 1;
            stop = true;
        } else if (s->it >= s->max_iter || k + 1 >= s->m) {
            s->status = 3;
            stop = true;
        }
        if (!stop) {
            s->k = k + 1;
            s->p_cur = s->relax ? relaxed_p_int(s->tol, rho, s->p_initial, s->p_min) : s->p_initial;
            cudaGraphSetConditional(hs, (unsigned)s->p_cur);
        }
    }
    cudaGraphSetConditional(hw, stop ? 0u : 1u);
}

}  // namespace

int arnoldi_blocks() {
    int dev = 0, sms = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_arnoldi, ARN_THREADS, 0) != cudaSuccess || per < 1) return 0;
    return sms;  // one block per SM: co-resident for the cooperative launch (more blocks make
                 // the grid barriers dearer than the extra loads in flight gain)
}

// Threads per Arnoldi block (one block per SM).
int arnoldi_threads(int64_t, int) { return ARN_THREADS; }

int relaxed_p(double eta, double rho_prev, int p_initial, int p_min) {
    return relaxed_p_int(eta, rho_prev, p_initial, p_min);
}

void dloop_free(fmmbem_handle* h) {
    if (h->dloop_exec) cudaGraphExecDestroy(h->dloop_exec);
    if (h->dloop_state) cudaFree(h->dloop_state);
    if (h->dloop_out) cudaFree(h->dloop_out);
    if (h->dloop_host) cudaFreeHost(h->dloop_host);
    h->dloop_exec = nullptr;
    h->dloop_state = h->dloop_host = nullptr;
    h->dloop_out = nullptr;
}

// The cycle graph: k_dloop_init, then a while node whose body is a switch over the orders
// (body p: the mat-vec xfix -> kw at order p, as matvec_sorted's graph), the Arnoldi step
// (its index read from the state) and k_dloop_step. Rebuilt when the kernel selection of
// any order changed.
static int dloop_build(fmmbem_handle* h) {
    const uint64_t key = matvec_modes_key(h);
    if (h->dloop_exec && h->dloop_key == key) return 0;
    if (h->dloop_exec) {
        cudaGraphExecDestroy(h->dloop_exec);
        h->dloop_exec = nullptr;
    }
    if (!h->dloop_state) {
        FMM_CU(cudaMalloc(&h->dloop_state, sizeof(KrylovDev)));
        FMM_CU(cudaMalloc((void**)&h->dloop_out, sizeof(double) * (2 * (ARN_MAXV + 1) + 1)));
        FMM_CU(cudaMallocHost(&h->dloop_host, sizeof(KrylovDev)));
    }
    cudaStream_t st = h->stream;
    KrylovDev* state = reinterpret_cast<KrylovDev*>(h->dloop_state);
    cudaGraph_t g = nullptr;
    FMM_CU(cudaGraphCreate(&g, 0));
    // every exit below destroys the graph under construction
    auto fail_with = [&](cudaError_t e, const char* what) {
        cudaGraph_t dummy = nullptr;
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
            cudaStreamEndCapture(st, &dummy);
        cudaGetLastError();
        cudaGraphDestroy(g);
        fmmbem_set_error("device loop: %s: %s", what, cudaGetErrorString(e));
        return FMMBEM_EDEVICE;
    };
    cudaGraphConditionalHandle hw, hs;
    cudaError_t e = cudaGraphConditionalHandleCreate(&hw, g, 1, cudaGraphCondAssignDefault);
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&hs, g, 0, 0);
    if (e != cudaSuccess) return fail_with(e, "conditional handles");
    cudaGraph_t out = nullptr;
    e = cudaStreamBeginCaptureToGraph(st, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return fail_with(e, "capture");
    k_dloop_init<<<1, 32, 0, st>>>(state, hs);
    e = cudaGetLastError();
    cudaError_t e2 = cudaStreamEndCapture(st, &out);
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) return fail_with(e, "init node");
    size_t nn = 0;
    cudaGraphNode_t init = nullptr;
    e = cudaGraphGetNodes(g, nullptr, &nn);
    if (e != cudaSuccess || nn != 1) return fail_with(e, "init node count");
    e = cudaGraphGetNodes(g, &init, &nn);
    if (e != cudaSuccess) return fail_with(e, "init node");
    cudaGraphNodeParams wp = {};
    wp.type = cudaGraphNodeTypeConditional;
    wp.conditional.handle = hw;
    wp.conditional.type = cudaGraphCondTypeWhile;
    wp.conditional.size = 1;
    cudaGraphNode_t wn;
    e = cudaGraphAddNode(&wn, g, &init, nullptr, 1, &wp);
    if (e != cudaSuccess) return fail_with(e, "while node");
    cudaGraph_t body = wp.conditional.phGraph_out[0];
    cudaGraphNodeParams sp = {};
    sp.type = cudaGraphNodeTypeConditional;
    sp.conditional.handle = hs;
    sp.conditional.type = cudaGraphCondTypeSwitch;
    sp.conditional.size = (unsigned)h->opts.p_max + 1;
    cudaGraphNode_t sn;
    e = cudaGraphAddNode(&sn, body, nullptr, nullptr, 0, &sp);
    if (e != cudaSuccess) return fail_with(e, "switch node");
    for (int q = 1; q <= h->opts.p_max; ++q) {
        e = cudaStreamBeginCaptureToGraph(st, sp.conditional.phGraph_out[q], nullptr, nullptr, 0,
                                          cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return fail_with(e, "mat-vec capture");
        const int rc = matvec_capture_body(h, q);
        e = cudaStreamEndCapture(st, &out);
        if (rc < 0) {
            cudaGraphDestroy(g);
            return rc;
        }
        if (e != cudaSuccess) return fail_with(e, "mat-vec body");
    }
    e = cudaStreamBeginCaptureToGraph(st, body, &sn, nullptr, 1, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return fail_with(e, "step capture");
    {
        double* dV = h->V;
        int64_t nn64 = h->N * h->dof;
        int kk = 0;
        double* dw = h->kw;
        double* dx = h->xfix;
        double* dp = h->kpart;
        unsigned* bar = h->arn_bar;
        double* dout = h->dloop_out;
        int* de = h->kerr;
        int nsys = 1;
        int64_t vstride = 0, wstride = 0;
        unsigned active = 1u;
        unsigned wl = h->wait_limit;
        const int* kdev = &state->k;
        void* args[] = {&dV, &nn64, &kk, &dw, &dx, &dp, &bar, &dout, &de, &nsys, &vstride, &wstride, &active, &wl, &kdev};
        e = cudaLaunchCooperativeKernel((const void*)k_arnoldi, dim3(h->arn_blocks),
                                        dim3(arnoldi_threads(nn64, h->arn_blocks)), args, 0, st);
        if (e == cudaSuccess) {
            k_dloop_step<<<1, 32, 0, st>>>(state, h->dloop_out, hw, hs);
            e = cudaGetLastError();
        }
    }
    e2 = cudaStreamEndCapture(st, &out);
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) return fail_with(e, "Arnoldi and step nodes");
    e = cudaGraphInstantiate(&h->dloop_exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        h->dloop_exec = nullptr;
        cudaGetLastError();
        fmmbem_set_error("device loop: instantiate: %s", cudaGetErrorString(e));
        return FMMBEM_EDEVICE;
    }
    h->dloop_key = key;
    return 0;
}

// One restart cycle on the device: the state is set, the cycle graph runs until the cycle
// converges, fails or ends, and the state comes back in one copy. Outputs as in the host loop.
static int dloop_cycle(fmmbem_handle* h, int& it, int m, int max_iter, int relax, int p_initial, int p_min, double tol,
                       double bnorm, double beta, double& rho, std::vector<double>& H, int m_max, std::vector<double>& g,
                       int& k_done, int& status, bool& converged, int* p_hist, double* res_hist) {
    FMM_TRY(dloop_build(h));
    cudaStream_t st = h->stream;
    KrylovDev* state = reinterpret_cast<KrylovDev*>(h->dloop_state);
    k_dloop_begin<<<1, 256, 0, st>>>(state, it, m, max_iter, p_initial, p_min, relax, tol, bnorm, beta, rho);
    FMM_LAUNCHED();
    FMM_CU(cudaGraphLaunch(h->dloop_exec, st));
    FMM_CU(cudaMemcpyAsync(h->dloop_host, state, sizeof(KrylovDev), cudaMemcpyDeviceToHost, st));
    FMM_CU(cudaStreamSynchronize(st));
    const KrylovDev* s = reinterpret_cast<const KrylovDev*>(h->dloop_host);
    const int steps = s->it - it;
    h->launches += 2;  // k_dloop_begin, k_dloop_init
    for (int j = 0; j < steps; ++j) {
        if (p_hist) p_hist[it + j] = s->p_c[j];
        if (res_hist && j < s->k_done) res_hist[it + j + 1] = s->res_c[j];
        h->launches += h->dloop_mv_launches[s->p_c[j]] + 2;
    }
    it = s->it;
    k_done = s->k_done;
    rho = s->rho;
    for (int i = 0; i <= k_done && i <= m_max; ++i) {
        g[i] = s->g[i];
        for (int j = 0; j < k_done; ++j) H[(size_t)i * m_max + j] = s->H[i * ARN_MAXV + j];
    }
    if (s->status == 1) converged = true;
    if (s->status == 2) status = FMMBEM_ENAN;
    return 0;
}

static int gmres_solve_on(fmmbem_handle* h, const double* b, double tol, int relax, int p_initial, int p_min, double* x,
                          int* iters, int* p_hist, double* res_hist, double* true_res);
static int gmres_refine_on(fmmbem_handle* h, const double* b, double tol, int relax, int p_initial, int p_min,
                           double* x, int* iters, int* p_hist, double* res_hist, double* true_res);

// The solve runs on the handle's internal stream (capturable, so the mat-vec graphs can
// be recorded), ordered after the caller's stream on entry and before it on exit.
static int gmres_batch_on(fmmbem_handle* h, const double* b, double tol, int relax, int p_initial, int p_min,
                          double* x, int* iters, int* p_hist, double* res_hist, double* true_res);

// Read and clear the handle's bounded-wait flags after the work queued on st: 0 when no
// wait gave up, FMMBEM_ETIMEOUT otherwise (the grid-barrier counters are then reset too,
// so the handle stays usable).
int read_wait_flags(fmmbem_handle* h, cudaStream_t st) {
    int flags[2] = {0, 0};
    FMM_CU(cudaMemcpyAsync(&flags[0], h->kerr, sizeof(int), cudaMemcpyDeviceToHost, st));
    if (h->tc_err) FMM_CU(cudaMemcpyAsync(&flags[1], h->tc_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    FMM_CU(cudaStreamSynchronize(st));
    if (!flags[0] && !flags[1]) return 0;
    fmmbem_set_error("a bounded device wait gave up (code %d/%d); results are invalid", flags[0], flags[1]);
    FMM_CU(cudaMemsetAsync(h->kerr, 0, sizeof(int), st));
    if (h->tc_err) FMM_CU(cudaMemsetAsync(h->tc_err, 0, sizeof(int), st));
    FMM_CU(cudaMemsetAsync(h->arn_bar, 0, 2 * h->nrhs * sizeof(unsigned), st));
    FMM_CU(cudaStreamSynchronize(st));
    return FMMBEM_ETIMEOUT;
}

// Batched handles (nrhs > 1): b, x are [nrhs][n]; iters, true_res hold nrhs entries,
// res_hist [nrhs][max_iter + 1]; p_hist (one order per mat-vec) is shared.
int gmres_solve(fmmbem_handle* h, const double* b, double tol, int relax, int p_initial, int p_min, double* x,
                int* iters, int* p_hist, double* res_hist, double* true_res) {
    cudaStream_t user = h->stream;
    FMM_CU(cudaEventRecord(h->ev_in, user));
    FMM_CU(cudaStreamWaitEvent(h->istream, h->ev_in, 0));
    // a flag left by an earlier mat-vec of this handle must not fail this solve: its waits
    // are cleared here (earlier mat-vecs report through fmmbem_check_waits)
    FMM_CU(cudaMemsetAsync(h->kerr, 0, sizeof(int), h->istream));
    if (h->tc_err) FMM_CU(cudaMemsetAsync(h->tc_err, 0, sizeof(int), h->istream));
    h->stream = h->istream;
    const int rc = h->nrhs > 1 ? gmres_batch_on(h, b, tol, relax, p_initial, p_min, x, iters, p_hist, res_hist, true_res)
                   : h->precision == FMMBEM_MIXED_REFINED
                       ? gmres_refine_on(h, b, tol, relax, p_initial, p_min, x, iters, p_hist, res_hist, true_res)
                       : gmres_solve_on(h, b, tol, relax, p_initial, p_min, x, iters, p_hist, res_hist, true_res);
    h->stream = user;
    if (rc == FMMBEM_EDEVICE || rc == FMMBEM_ENOMEM) return rc;
    // bounded device waits (grid barrier, bulk-copy and tensor-core barriers) report here,
    // ahead of a NaN status that a wait giving up may have caused
    const int wr = read_wait_flags(h, h->istream);
    if (wr < 0) return wr;
    if (rc < 0) return rc;
    FMM_CU(cudaEventRecord(h->ev_out, h->istream));
    FMM_CU(cudaStreamWaitEvent(user, h->ev_out, 0));
    return rc;
}

static int gmres_solve_on(fmmbem_handle* h, const double* b, double tol, int relax, int p_initial, int p_min, double* x,
                          int* iters, int* p_hist, double* res_hist, double* true_res) {
    const int64_t n = h->N * h->dof;
    const int m_max = h->kr_m;
    const int max_iter = h->opts.max_iter;
    cudaStream_t st = h->stream;
    Kr kr{h, n, (unsigned)std::min<int64_t>((n + 255) / 256, 2048)};
    double* hb = h->kh_host;  // [3 * (m+2)] pinned
    double* kh1 = h->kh;
    double* kh2 = h->kh + (m_max + 2);
    double* knr = h->kh + 2 * (m_max + 2);

    FMM_CU(cudaMemsetAsync(x, 0, sizeof(double) * n, st));
    FMM_TRY(kr.dots(b, 1, b, knr));
    FMM_CU(cudaMemcpyAsync(hb, knr, sizeof(double), cudaMemcpyDeviceToHost, st));
    FMM_CU(cudaStreamSynchronize(st));
        prof_harvest(h);
    const double bnorm = sqrt(hb[0]);
    if (iters) *iters = 0;
    if (res_hist) res_hist[0] = 1.0;
    if (!(bnorm > 0.0)) {
        if (true_res) *true_res = 0.0;
        return bnorm == 0.0 ? 0 : FMMBEM_ENAN;
    }
    std::vector<double> H((size_t)(m_max + 1) * m_max), cs(m_max), sn(m_max), g(m_max + 1), y(m_max);
    auto Hc = [&](int i, int k) -> double& { return H[(size_t)i * m_max + k]; };
    int it = 0;
    double rho = 1.0;
    double beta = bnorm;
    // r0 = b (x0 = 0)
    FMM_CU(cudaMemcpyAsync(h->kr, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    bool converged = false;
    int status = 0;
    while (true) {
        const int m = std::min(m_max, max_iter - it);
        if (m <= 0) break;
        k_scale<<<kr.gs, 256, 0, st>>>(h->V, h->xfix, h->kr, 1.0 / beta, n);
        FMM_LAUNCHED();
        h->launches += 1;
        std::fill(H.begin(), H.end(), 0.0);
        std::fill(g.begin(), g.end(), 0.0);
        g[0] = beta;
        int k_done = 0;
        bool stop = false;
        // the device-resident cycle (fmmbem_set_device_loop) runs the same steps on the device
        const bool dloop = h->dloop_on && h->use_graphs && !h->prof_on && h->stream != nullptr && m <= ARN_MAXV;
        if (dloop)
            FMM_TRY(dloop_cycle(h, it, m, max_iter, relax, p_initial, p_min, tol, bnorm, beta, rho, H, m_max, g, k_done,
                                status, converged, p_hist, res_hist));
        for (int k = 0; k < m && !dloop; ++k) {
            const int p = relax ? relaxed_p_int(tol, rho, p_initial, p_min) : p_initial;
            // v_k is also in xfix, the fixed input of the per-order mat-vec graphs
            FMM_TRY(matvec_sorted(h, p, h->xfix, h->kw));
            if (p_hist) p_hist[it] = p;
            ++it;
            prof_begin(h, FMMBEM_PASS_KRYLOV);
            {
                // fused Arnoldi step; results in mapped pinned memory
                double* dV = h->V;
                int64_t nn = n;
                int kk = k;
                double* dw = h->kw;
                double* dx = h->xfix;
                double* dp = h->kpart;
                unsigned* bar = h->arn_bar;
                double* dout = h->arn_out_dev;
                int* de = h->kerr;
                int nsys = 1;
                int64_t vstride = 0, wstride = 0;
                unsigned active = 1u;
                unsigned wl = h->wait_limit;
                const int* kdev = nullptr;
                void* args[] = {&dV, &nn, &kk, &dw, &dx, &dp, &bar, &dout, &de, &nsys, &vstride, &wstride, &active, &wl, &kdev};
                FMM_CU(cudaLaunchCooperativeKernel((const void*)k_arnoldi, dim3(h->arn_blocks), dim3(arnoldi_threads(n, h->arn_blocks)), args, 0,
                                                   st));
                h->launches += 1;
            }
            FMM_CU(cudaStreamSynchronize(st));
            prof_harvest(h);
            const volatile double* ao = h->arn_out_host;
            for (int i = 0; i <= k; ++i) Hc(i, k) = ao[i] + ao[(ARN_MAXV + 1) + i];
            const double hn = sqrt(ao[2 * (ARN_MAXV + 1)]);
            Hc(k + 1, k) = hn;
            if (!std::isfinite(hn)) { status = FMMBEM_ENAN; stop = true; k_done = k; prof_end(h, FMMBEM_PASS_KRYLOV, 1); break; }
            for (int i = 0; i < k; ++i) {
                const double t = cs[i] * Hc(i, k) + sn[i] * Hc(i + 1, k);
                Hc(i + 1, k) = -sn[i] * Hc(i, k) + cs[i] * Hc(i + 1, k);
                Hc(i, k) = t;
            }
            const double den = hypot(Hc(k, k), Hc(k + 1, k));
            cs[k] = Hc(k, k) / den;
            sn[k] = Hc(k + 1, k) / den;
            Hc(k, k) = den;
            Hc(k + 1, k) = 0.0;
            g[k + 1] = -sn[k] * g[k];
            g[k] = cs[k] * g[k];
            rho = fabs(g[k + 1]) / bnorm;
            if (res_hist) res_hist[it] = rho;
            prof_end(h, FMMBEM_PASS_KRYLOV, 1);
            k_done = k + 1;
            if (!std::isfinite(rho)) { status = FMMBEM_ENAN; stop = true; break; }
            if (rho <= tol) { converged = true; break; }
            if (hn == 0.0) { converged = true; break; }  // happy breakdown: exact solution in the space
            if (it >= max_iter) break;
        }
        if (status < 0) break;
        // y = H^{-1} g (upper triangular), x += V y
        for (int i = k_done - 1; i >= 0; --i) {
            double s = g[i];
            for (int j = i + 1; j < k_done; ++j) s -= Hc(i, j) * y[j];
            y[i] = s / Hc(i, i);
        }
        if (k_done > 0) {
            FMM_CU(cudaMemcpyAsync(h->kyv, y.data(), sizeof(double) * k_done, cudaMemcpyHostToDevice, st));
            k_add_combo<<<kr.gs, 256, 0, st>>>(x, h->V, n, k_done, h->kyv, n);
            FMM_LAUNCHED();
            h->launches += 1;
        }
        if (converged || it >= max_iter || stop) break;
        // restart: r = b - A x at p_initial
        FMM_CU(cudaMemcpyAsync(h->xfix, x, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
        FMM_TRY(matvec_sorted(h, p_initial, h->xfix, h->kw));
        k_sub<<<kr.gs, 256, 0, st>>>(h->kr, b, h->kw, n);
        FMM_LAUNCHED();
        h->launches += 1;
        FMM_TRY(kr.dots(h->kr, 1, h->kr, knr));
        FMM_CU(cudaMemcpyAsync(hb, knr, sizeof(double), cudaMemcpyDeviceToHost, st));
        FMM_CU(cudaStreamSynchronize(st));
        prof_harvest(h);
        beta = sqrt(hb[0]);
        rho = beta / bnorm;
        if (res_hist) res_hist[it] = rho;
        if (rho <= tol) { converged = true; break; }
        if (!(beta > 0.0)) { converged = beta == 0.0; break; }
    }
    if (iters) *iters = it;
    if (status < 0) return status;
    if (true_res) {
        FMM_CU(cudaMemcpyAsync(h->xfix, x, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
        FMM_TRY(matvec_sorted(h, p_initial, h->xfix, h->kw));
        k_sub<<<kr.gs, 256, 0, st>>>(h->kr, b, h->kw, n);
        FMM_LAUNCHED();
        h->launches += 1;
        FMM_TRY(kr.dots(h->kr, 1, h->kr, knr));
        FMM_CU(cudaMemcpyAsync(hb, knr, sizeof(double), cudaMemcpyDeviceToHost, st));
        FMM_CU(cudaStreamSynchronize(st));
        prof_harvest(h);
        *true_res = sqrt(hb[0]) / bnorm;
    }
    return converged ? 0 : FMMBEM_NOT_CONVERGED;
}

// Iterative refinement around the mixed-precision relaxed GMRES: the FP32 passes resolve the
// operator to about 1e-6, so each outer step solves A d = r with mixed mat-vecs only to a
// relative RF_INNER_TOL (or to the final tolerance when that is looser), then x += d and
// r = b - A x with an FP64 mat-vec at p_initial. The error of one step is about the inner
// tolerance plus the mixed operator's relative error times the conditioning, so two or three
// outer steps reach 1e-8 where an all-FP64 solve runs every mat-vec at a few times the cost.
constexpr double RF_INNER_TOL = 1e-5;
constexpr int RF_MAX_OUTER = 8;

static int gmres_refine_on(fmmbem_handle* h, const double* b, double tol, int relax, int p_initial, int p_min,
                           double* x, int* iters, int* p_hist, double* res_hist, double* true_res) {
    const int64_t n = h->N * h->dof;
    const int max_iter = h->opts.max_iter;
    cudaStream_t st = h->stream;
    Kr kr{h, n, (unsigned)std::min<int64_t>((n + 255) / 256, 2048)};
    double* hb = h->kh_host;
    double* knr = h->kh + 2 * (h->kr_m + 2);
    double* r = h->rf_r;
    double* d = h->rf_d;
    auto norm_of = [&](const double* v, double* out) -> int {
        FMM_TRY(kr.dots(v, 1, v, knr));
        FMM_CU(cudaMemcpyAsync(hb, knr, sizeof(double), cudaMemcpyDeviceToHost, st));
        FMM_CU(cudaStreamSynchronize(st));
        prof_harvest(h);
        *out = sqrt(hb[0]);
        return 0;
    };
    FMM_CU(cudaMemsetAsync(x, 0, sizeof(double) * n, st));
    double bnorm = 0.0;
    FMM_TRY(norm_of(b, &bnorm));
    if (iters) *iters = 0;
    if (res_hist) res_hist[0] = 1.0;
    if (!(bnorm > 0.0)) {
        if (true_res) *true_res = 0.0;
        return bnorm == 0.0 ? 0 : FMMBEM_ENAN;
    }
    FMM_CU(cudaMemcpyAsync(r, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    std::vector<int> ph(max_iter + 1);
    std::vector<double> rh(max_iter + 2);
    double rho = 1.0;
    int it = 0, rc = 0;
    bool converged = false;
    for (int outer = 0; outer < RF_MAX_OUTER && it < max_iter; ++outer) {
        // inner: A d = r, mixed mat-vecs, relaxed by the inner tolerance
        const double tin = std::min(0.5, std::max(RF_INNER_TOL, tol / rho));
        int it_in = 0;
        const int keep_max = h->opts.max_iter;
        h->opts.max_iter = max_iter - it;
        h->precision = FMMBEM_MIXED;
        rc = gmres_solve_on(h, r, tin, relax, p_initial, p_min, d, &it_in, ph.data(), rh.data(), nullptr);
        h->precision = FMMBEM_MIXED_REFINED;
        h->opts.max_iter = keep_max;
        if (rc < 0) return rc;
        for (int k = 0; k < it_in; ++k) {
            if (p_hist) p_hist[it + k] = ph[k];
            if (res_hist) res_hist[it + k + 1] = rh[k + 1] * rho;  // the inner estimate, relative to ||b||
        }
        it += it_in;
        k_add<<<kr.gs, 256, 0, st>>>(x, d, n);
        FMM_LAUNCHED();
        h->launches += 1;
        // outer: r = b - A x with an FP64 mat-vec at p_initial
        FMM_CU(cudaMemcpyAsync(h->xfix, x, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
        h->precision = FMMBEM_FP64;
        rc = matvec_sorted(h, p_initial, h->xfix, h->kw);
        h->precision = FMMBEM_MIXED_REFINED;
        if (rc < 0) return rc;
        k_sub<<<kr.gs, 256, 0, st>>>(r, b, h->kw, n);
        FMM_LAUNCHED();
        h->launches += 1;
        double rn = 0.0;
        FMM_TRY(norm_of(r, &rn));
        rho = rn / bnorm;
        if (res_hist && it > 0) res_hist[it] = rho;
        if (!std::isfinite(rho)) return FMMBEM_ENAN;
        if (rho <= tol) { converged = true; break; }
        if (it_in == 0) break;  // no progress possible (the inner solve met its tolerance at once)
    }
    if (iters) *iters = it;
    if (true_res) *true_res = rho;
    return converged ? 0 : FMMBEM_NOT_CONVERGED;
}

// Restarted GMRES for the nrhs systems of a batched handle, in lockstep: each mat-vec
// evaluates every system's current basis vector at once, at the largest order any active
// system's relaxation rule asks for (a higher order than a system needs only makes its
// product more accurate, so each system still meets its own bound). Each system keeps its
// own Hessenberg matrix, Givens rotations, residual and restart state, and leaves the
// lockstep once converged (its input vector is then zero). One cooperative launch runs the
// Arnoldi steps of all active systems, one group of blocks per system.
static int gmres_batch_on(fmmbem_handle* h, const double* b, double tol, int relax, int p_initial, int p_min,
                          double* x, int* iters, int* p_hist, double* res_hist, double* true_res) {
    const int nb = h->nrhs;
    const int64_t n = h->N * h->dof;  // per system
    const int m_max = h->kr_m;
    const int max_iter = h->opts.max_iter;
    cudaStream_t st = h->stream;
    Kr kr{h, n, (unsigned)std::min<int64_t>((n + 255) / 256, 2048)};
    double* hb = h->kh_host;
    double* knr = h->kh + 2 * (m_max + 2) * nb;
    const int64_t vstride = (int64_t)(m_max + 1) * n;
    FMM_CU(cudaMemsetAsync(x, 0, sizeof(double) * n * nb, st));
    for (int q = 0; q < nb; ++q) FMM_TRY(kr.dots(b + q * n, 1, b + q * n, knr + q));
    FMM_CU(cudaMemcpyAsync(hb, knr, sizeof(double) * nb, cudaMemcpyDeviceToHost, st));
    FMM_CU(cudaStreamSynchronize(st));
    prof_harvest(h);
    struct Sys {
        double bnorm = 0, beta = 0, rho = 1;
        bool active = false, converged = false;
        int it = 0, k_done = 0;
        std::vector<double> H, cs, sn, g, y;
    };
    std::vector<Sys> sy(nb);
    for (int q = 0; q < nb; ++q) {
        Sys& S = sy[q];
        S.bnorm = S.beta = sqrt(hb[q]);
        S.H.assign((size_t)(m_max + 1) * m_max, 0.0);
        S.cs.assign(m_max, 0.0);
        S.sn.assign(m_max, 0.0);
        S.g.assign(m_max + 1, 0.0);
        S.y.assign(m_max, 0.0);
        if (iters) iters[q] = 0;
        if (res_hist) res_hist[(size_t)q * (max_iter + 1)] = 1.0;
        if (!std::isfinite(S.bnorm)) return FMMBEM_ENAN;
        S.converged = S.bnorm == 0.0;
        S.active = !S.converged;
    }
    // r0 = b (x0 = 0)
    FMM_CU(cudaMemcpyAsync(h->kr, b, sizeof(double) * n * nb, cudaMemcpyDeviceToDevice, st));
    int it = 0, status = 0;
    auto any_active = [&]() {
        for (const Sys& S : sy) if (S.active) return true;
        return false;
    };
    while (any_active() && it < max_iter) {
        const int m = std::min(m_max, max_iter - it);
        // v_0 = r / beta for the active systems; inactive inputs are zero
        for (int q = 0; q < nb; ++q) {
            Sys& S = sy[q];
            if (S.active) {
                k_scale<<<kr.gs, 256, 0, st>>>(h->V + q * vstride, h->xfix + q * n, h->kr + q * n, 1.0 / S.beta, n);
                FMM_LAUNCHED();
                h->launches += 1;
                std::fill(S.H.begin(), S.H.end(), 0.0);
                std::fill(S.g.begin(), S.g.end(), 0.0);
                S.g[0] = S.beta;
                S.k_done = 0;
            } else {
                FMM_CU(cudaMemsetAsync(h->xfix + q * n, 0, sizeof(double) * n, st));
            }
        }
        unsigned cycle = 0;  // systems taking part in this cycle
        for (int q = 0; q < nb; ++q) cycle |= (sy[q].active ? 1u : 0u) << q;
        for (int k = 0; k < m; ++k) {
            int p = p_min;
            for (const Sys& S : sy)
                if (S.active) p = std::max(p, relax ? relaxed_p_int(tol, S.rho, p_initial, p_min) : p_initial);
            FMM_TRY(matvec_sorted(h, p, h->xfix, h->kw));
            if (p_hist) p_hist[it] = p;
            ++it;
            unsigned active = 0;
            for (int q = 0; q < nb; ++q) active |= (sy[q].active ? 1u : 0u) << q;
            prof_begin(h, FMMBEM_PASS_KRYLOV);
            {
                double* dV = h->V;
                int64_t nn = n;
                int kk = k;
                double* dw = h->kw;
                double* dx = h->xfix;
                double* dp = h->kpart;
                unsigned* bar = h->arn_bar;
                double* dout = h->arn_out_dev;
                int* de = h->kerr;
                int nsys = nb;
                int64_t vs = vstride, ws = n;
                unsigned wl = h->wait_limit;
                const int* kdev = nullptr;
                void* args[] = {&dV, &nn, &kk, &dw, &dx, &dp, &bar, &dout, &de, &nsys, &vs, &ws, &active, &wl, &kdev};
                const int grid = (h->arn_blocks / nb) * nb;
                FMM_CU(cudaLaunchCooperativeKernel((const void*)k_arnoldi, dim3(grid),
                                                   dim3(arnoldi_threads(n, grid)), args, 0, st));
                h->launches += 1;
            }
            FMM_CU(cudaStreamSynchronize(st));
            prof_harvest(h);
            for (int q = 0; q < nb; ++q) {
                Sys& S = sy[q];
                if (!S.active) continue;
                auto Hc = [&](int i, int c) -> double& { return S.H[(size_t)i * m_max + c]; };
                const volatile double* ao = h->arn_out_host + (size_t)q * (2 * (ARN_MAXV + 1) + 1);
                for (int i = 0; i <= k; ++i) Hc(i, k) = ao[i] + ao[(ARN_MAXV + 1) + i];
                const double hn = sqrt(ao[2 * (ARN_MAXV + 1)]);
                Hc(k + 1, k) = hn;
                if (!std::isfinite(hn)) { status = FMMBEM_ENAN; break; }
                for (int i = 0; i < k; ++i) {
                    const double t = S.cs[i] * Hc(i, k) + S.sn[i] * Hc(i + 1, k);
                    Hc(i + 1, k) = -S.sn[i] * Hc(i, k) + S.cs[i] * Hc(i + 1, k);
                    Hc(i, k) = t;
                }
                const double den = hypot(Hc(k, k), Hc(k + 1, k));
                S.cs[k] = Hc(k, k) / den;
                S.sn[k] = Hc(k + 1, k) / den;
                Hc(k, k) = den;
                Hc(k + 1, k) = 0.0;
                S.g[k + 1] = -S.sn[k] * S.g[k];
                S.g[k] = S.cs[k] * S.g[k];
                S.rho = fabs(S.g[k + 1]) / S.bnorm;
                S.it = it;
                S.k_done = k + 1;
                if (res_hist) res_hist[(size_t)q * (max_iter + 1) + it] = S.rho;
                if (!std::isfinite(S.rho)) { status = FMMBEM_ENAN; break; }
                if (S.rho <= tol || hn == 0.0) {
                    S.converged = true;
                    S.active = false;  // its basis stays as is; x is updated at the end of the cycle
                    FMM_CU(cudaMemsetAsync(h->xfix + q * n, 0, sizeof(double) * n, st));
                }
            }
            prof_end(h, FMMBEM_PASS_KRYLOV, 1);
            if (status < 0) break;
            if (!any_active() || it >= max_iter) break;
        }
        if (status < 0) break;
        // y = H^{-1} g, x += V y for every system of this cycle
        for (int q = 0; q < nb; ++q) {
            Sys& S = sy[q];
            if (!((cycle >> q) & 1u) || S.k_done == 0) continue;
            auto Hc = [&](int i, int c) -> double& { return S.H[(size_t)i * m_max + c]; };
            for (int i = S.k_done - 1; i >= 0; --i) {
                double t = S.g[i];
                for (int j = i + 1; j < S.k_done; ++j) t -= Hc(i, j) * S.y[j];
                S.y[i] = t / Hc(i, i);
            }
            FMM_CU(cudaMemcpyAsync(h->kyv + q * (m_max + 2), S.y.data(), sizeof(double) * S.k_done,
                                   cudaMemcpyHostToDevice, st));
            k_add_combo<<<kr.gs, 256, 0, st>>>(x + q * n, h->V + q * vstride, n, S.k_done, h->kyv + q * (m_max + 2), n);
            FMM_LAUNCHED();
            h->launches += 1;
        }
        if (!any_active() || it >= max_iter) break;
        // restart the active systems: r = b - A x at p_initial (the batch mat-vec, inactive inputs zero)
        for (int q = 0; q < nb; ++q) {
            if (sy[q].active) FMM_CU(cudaMemcpyAsync(h->xfix + q * n, x + q * n, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
            else FMM_CU(cudaMemsetAsync(h->xfix + q * n, 0, sizeof(double) * n, st));
        }
        FMM_TRY(matvec_sorted(h, p_initial, h->xfix, h->kw));
        for (int q = 0; q < nb; ++q) {
            if (!sy[q].active) continue;
            k_sub<<<kr.gs, 256, 0, st>>>(h->kr + q * n, b + q * n, h->kw + q * n, n);
            FMM_LAUNCHED();
            h->launches += 1;
            FMM_TRY(kr.dots(h->kr + q * n, 1, h->kr + q * n, knr + q));
        }
        FMM_CU(cudaMemcpyAsync(hb, knr, sizeof(double) * nb, cudaMemcpyDeviceToHost, st));
        FMM_CU(cudaStreamSynchronize(st));
        prof_harvest(h);
        for (int q = 0; q < nb; ++q) {
            Sys& S = sy[q];
            if (!S.active) continue;
            S.beta = sqrt(hb[q]);
            S.rho = S.beta / S.bnorm;
            if (res_hist) res_hist[(size_t)q * (max_iter + 1) + it] = S.rho;
            if (S.rho <= tol || !(S.beta > 0.0)) {
                S.converged = S.rho <= tol || S.beta == 0.0;
                S.active = false;
            }
        }
    }
    for (int q = 0; q < nb; ++q)
        if (iters) iters[q] = sy[q].it;
    if (status < 0) return status;
    if (true_res) {
        FMM_CU(cudaMemcpyAsync(h->xfix, x, sizeof(double) * n * nb, cudaMemcpyDeviceToDevice, st));
        FMM_TRY(matvec_sorted(h, p_initial, h->xfix, h->kw));
        for (int q = 0; q < nb; ++q) {
            k_sub<<<kr.gs, 256, 0, st>>>(h->kr + q * n, b + q * n, h->kw + q * n, n);
            FMM_LAUNCHED();
            h->launches += 1;
            FMM_TRY(kr.dots(h->kr + q * n, 1, h->kr + q * n, knr + q));
        }
        FMM_CU(cudaMemcpyAsync(hb, knr, sizeof(double) * nb, cudaMemcpyDeviceToHost, st));
        FMM_CU(cudaStreamSynchronize(st));
        prof_harvest(h);
        for (int q = 0; q < nb; ++q) true_res[q] = sy[q].bnorm > 0.0 ? sqrt(hb[q]) / sy[q].bnorm : 0.0;
    }
    bool all = true;
    for (const Sys& S : sy) all = all && S.converged;
    return all ? 0 : FMMBEM_NOT_CONVERGED;
}

}  // namespace fmmbem
