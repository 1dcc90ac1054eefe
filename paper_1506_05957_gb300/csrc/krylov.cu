// Relaxed restarted GMRES(m) (Sec. 2.4 and 2.6) with the Krylov recurrence in FP64.
// Arnoldi: classical Gram-Schmidt applied twice (CGS2), as batched dot products and
// one fused update per pass, all on the device; the (m+1) x m Hessenberg column,
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

__global__ void k_sub(double* r, const double* b, const double* ax, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        r[i] = b[i] - ax[i];
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

int relaxed_p_int(double eta, double rho_prev, int p_initial, int p_min) {
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

}  // namespace

int relaxed_p(double eta, double rho_prev, int p_initial, int p_min) {
    return relaxed_p_int(eta, rho_prev, p_initial, p_min);
}

static int gmres_solve_on(fmmbem_handle* h, const double* b, double tol, int relax, int p_initial, int p_min, double* x,
                          int* iters, int* p_hist, double* res_hist, double* true_res);

// The solve runs on the handle's internal stream (capturable, so the mat-vec graphs can
// be recorded), ordered after the caller's stream on entry and before it on exit.
int gmres_solve(fmmbem_handle* h, const double* b, double tol, int relax, int p_initial, int p_min, double* x,
                int* iters, int* p_hist, double* res_hist, double* true_res) {
    cudaStream_t user = h->stream;
    FMM_CU(cudaEventRecord(h->ev_in, user));
    FMM_CU(cudaStreamWaitEvent(h->istream, h->ev_in, 0));
    h->stream = h->istream;
    const int rc = gmres_solve_on(h, b, tol, relax, p_initial, p_min, x, iters, p_hist, res_hist, true_res);
    h->stream = user;
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
        for (int k = 0; k < m; ++k) {
            const int p = relax ? relaxed_p_int(tol, rho, p_initial, p_min) : p_initial;
            // v_k is also in xfix, the fixed input of the per-order mat-vec graphs
            FMM_TRY(matvec_sorted(h, p, h->xfix, h->kw));
            if (p_hist) p_hist[it] = p;
            ++it;
            prof_begin(h, FMMBEM_PASS_KRYLOV);
            FMM_TRY(kr.dots(h->V, k + 1, h->kw, kh1));
            FMM_TRY(kr.sub(h->kw, h->V, k + 1, kh1));
            FMM_TRY(kr.dots(h->V, k + 1, h->kw, kh2));
            FMM_TRY(kr.sub(h->kw, h->V, k + 1, kh2));
            FMM_TRY(kr.dots(h->kw, 1, h->kw, knr));
            FMM_CU(cudaMemcpyAsync(hb, h->kh, sizeof(double) * 3 * (m_max + 2), cudaMemcpyDeviceToHost, st));
            FMM_CU(cudaStreamSynchronize(st));
        prof_harvest(h);
            for (int i = 0; i <= k; ++i) Hc(i, k) = hb[i] + hb[(m_max + 2) + i];
            const double hn = sqrt(hb[2 * (m_max + 2)]);
            Hc(k + 1, k) = hn;
            if (!std::isfinite(hn)) { status = FMMBEM_ENAN; stop = true; k_done = k; prof_end(h, FMMBEM_PASS_KRYLOV, 9); break; }
            if (hn > 0.0) {
                k_scale<<<kr.gs, 256, 0, st>>>(h->V + (int64_t)(k + 1) * n, h->xfix, h->kw, 1.0 / hn, n);
                FMM_LAUNCHED();
                h->launches += 1;
            }
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
            prof_end(h, FMMBEM_PASS_KRYLOV, 9);
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

}  // namespace fmmbem
