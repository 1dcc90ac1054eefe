// C ABI of libfmmbem.so (declared in include/fmmbem.h): handle life cycle, the
// mat-vec pipeline (near field, far field, evaluation) in Morton-sorted order,
// permutations to and from the caller's panel order, solves and profiling.
#include <stdarg.h>
#include <mutex>
#include <string.h>
#include <algorithm>
#include <chrono>
#include <vector>
#include "handle.cuh"

namespace {
thread_local char g_err[1024] = "";
}

cudaStream_t& fmm_alloc_stream() {
    thread_local cudaStream_t s = nullptr;
    return s;
}

void fmmbem_set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

namespace fmmbem {

namespace {

// Caller order <-> Morton-sorted order; blockIdx.y selects the vector of a batch ([nrhs][n][dof]).
__global__ void k_perm_in(const double* x, const int* perm, int64_t n, int dof, double* xs) {
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int64_t off = (int64_t)blockIdx.y * n * dof;
    const int64_t i = perm[s];
    for (int a = 0; a < dof; ++a) xs[off + dof * s + a] = x[off + dof * i + a];
}

__global__ void k_perm_out(const double* ys, const int* perm, int64_t n, int dof, double* y) {
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int64_t off = (int64_t)blockIdx.y * n * dof;
    const int64_t i = perm[s];
    for (int a = 0; a < dof; ++a) y[off + dof * i + a] = ys[off + dof * s + a];
}

// out[body][a] += S_s x[perm[s]][a] over the sorted panels s (FP64 atomics; the order of the
// additions is not fixed, so the sums agree with a serial sum to rounding)
__global__ void k_body_sums(const double* x, const int* perm, const double4* tgt, const int* body, int64_t n, int dof,
                            double* out) {
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int64_t i = perm[s];
    const int b = body ? body[s] : 0;
    const double S = tgt[s].w;
    for (int a = 0; a < dof; ++a) atomicAdd(out + (int64_t)b * dof + a, S * x[dof * i + a]);
}

__global__ void k_axpy_half(double* y, const double* x, int64_t n) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) y[i] += 0.5 * x[i];
}

struct ProfRec {
    int pass;
    int launches;
    cudaEvent_t a, b;
    bool tc;  // the pass ran on the tensor-core kernel
};
struct ProfState {
    std::vector<cudaEvent_t> pool;
    size_t used = 0;
    std::vector<ProfRec> recs;
    cudaEvent_t open[FMMBEM_N_PASSES] = {};
};
ProfState* prof_state(fmmbem_handle* h);

double operator_scale(const fmmbem_handle* h) {
    const double pi = 3.14159265358979323846;
    if (h->kernel == FMMBEM_LAPLACE) return 1.0 / (4.0 * pi);
    return h->layer == FMMBEM_LAYER_DOUBLE ? 1.0 / (8.0 * pi) : -1.0 / (8.0 * pi * h->opts.mu);
}

int perm_in(fmmbem_handle* h, const double* x, double* xs) {
    const int64_t n = h->N;
    k_perm_in<<<dim3((unsigned)((n + 255) / 256), h->nrhs), 256, 0, h->stream>>>(x, h->perm, n, h->dof, xs);
    FMM_LAUNCHED();
    h->launches += 1;
    return 0;
}

int perm_out(fmmbem_handle* h, const double* ys, double* y) {
    const int64_t n = h->N;
    k_perm_out<<<dim3((unsigned)((n + 255) / 256), h->nrhs), 256, 0, h->stream>>>(ys, h->perm, n, h->dof, y);
    FMM_LAUNCHED();
    h->launches += 1;
    return 0;
}

template <typename P>
int dalloc(P** p, size_t count) {
    *p = nullptr;
    FMM_CU(fmm_malloc(p, (count ? count : 1) * sizeof(P)));
    return 0;
}

// Pinned host buffers (the solver's small result areas) are recycled through a free list
// instead of being released, because freeing pinned memory synchronizes the device.
std::mutex g_pinned_mu;
std::vector<std::pair<size_t, void*>> g_pinned_free;

void* pinned_get(size_t bytes, unsigned flags) {
    {
        std::lock_guard<std::mutex> lock(g_pinned_mu);
        for (size_t i = 0; i < g_pinned_free.size(); ++i)
            if (g_pinned_free[i].first >= bytes) {
                void* p = g_pinned_free[i].second;
                g_pinned_free.erase(g_pinned_free.begin() + i);
                return p;
            }
    }
    void* p = nullptr;
    // every recycled buffer is mapped, so any request can take any of them
    if (cudaHostAlloc(&p, bytes < 4096 ? 4096 : bytes, flags | cudaHostAllocMapped) != cudaSuccess) return nullptr;
    return p;
}

void pinned_put(void* p, size_t bytes) {
    if (!p) return;
    std::lock_guard<std::mutex> lock(g_pinned_mu);
    g_pinned_free.push_back({bytes < 4096 ? 4096 : bytes, p});
}

}  // namespace

// Profiling state lives in the handle (allocated on first use), so handles driven from
// different host threads share nothing.
namespace {
ProfState* prof_state(fmmbem_handle* h) {
    if (!h->prof_state) h->prof_state = new ProfState();
    return reinterpret_cast<ProfState*>(h->prof_state);
}
void prof_free(fmmbem_handle* h) {
    ProfState* s = reinterpret_cast<ProfState*>(h->prof_state);
    if (!s) return;
    for (auto ev : s->pool) cudaEventDestroy(ev);
    delete s;
    h->prof_state = nullptr;
}
cudaEvent_t prof_event(ProfState* s) {
    if (s->used == s->pool.size()) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        s->pool.push_back(e);
    }
    return s->pool[s->used++];
}
}  // namespace

// While a mat-vec graph is being captured with profiling on, pass boundaries become
// external event-record nodes of that graph (one event pair per pass, owned by the
// graph); prof_harvest reads them after each replay, once the stream has synchronized.
void prof_begin(fmmbem_handle* h, int pass) {
    if (!h->prof_on) return;
    if (h->capturing >= 0) {
        cudaEvent_t& e = h->gev[h->capturing][2 * pass];
        if (!e) cudaEventCreate(&e);
        cudaEventRecordWithFlags(e, h->stream, cudaEventRecordExternal);
        return;
    }
    ProfState* s = prof_state(h);
    cudaEvent_t e = prof_event(s);
    cudaEventRecord(e, h->stream);
    s->open[pass] = e;
}

void prof_end(fmmbem_handle* h, int pass, int launches) {
    if (!h->prof_on) return;
    if (h->capturing >= 0) {
        cudaEvent_t& e = h->gev[h->capturing][2 * pass + 1];
        if (!e) cudaEventCreate(&e);
        cudaEventRecordWithFlags(e, h->stream, cudaEventRecordExternal);
        h->gev_launches[h->capturing][pass] = launches;
        h->gev_tc[h->capturing] = h->tc_pass_bits;
        return;
    }
    ProfState* s = prof_state(h);
    if (!s->open[pass]) return;
    cudaEvent_t e = prof_event(s);
    cudaEventRecord(e, h->stream);
    s->recs.push_back({pass, launches, s->open[pass], e, ((h->tc_pass_bits >> pass) & 1) != 0});
    s->open[pass] = nullptr;
}

void prof_harvest(fmmbem_handle* h) {
    const int p = h->pending_graph;
    if (p < 0) return;
    h->pending_graph = -1;
    for (int pass = 0; pass < FMMBEM_N_PASSES; ++pass) {
        cudaEvent_t a = h->gev[p][2 * pass], b = h->gev[p][2 * pass + 1];
        if (!a || !b) continue;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, a, b) != cudaSuccess) continue;
        h->prof.ms[pass] += ms;
        h->prof.launches[pass] += h->gev_launches[p][pass];
        h->prof.calls[pass] += 1;
        if ((h->gev_tc[p] >> pass) & 1) h->prof.tc_ms += ms;
    }
}

// Algorithmic flops of the passes of one mat-vec at order p that run on the tensor-core
// kernel: 2 (p+1)^4 per M2L pair and expansion, the same per M2M and per L2L translation
// (one per non-root cell).
static double tc_flops(const fmmbem_handle* h, int p) {
    if (h->precision == FMMBEM_FP64 || h->m2l_mode != FMMBEM_M2L_TENSOR || !h->m2l_tc_ready) return 0.0;
    const double q = (double)(p + 1) * (p + 1), per = 2.0 * q * q * h->ncomp * h->nsys;
    double f = 0.0;
    if (h->m2l_tc_at[p]) f += per * (double)h->n_m2l;
    if (h->tree_tc_at[p] && h->tree_tiles) f += 2.0 * per * (double)(h->n_cells - 1);
    return f;
}

static int matvec_launch(fmmbem_handle* h, int p, const double* xs, double* ys);


// Mat-vecs of the solver (fixed buffers xfix -> kw, not profiling) replay one CUDA graph
// per order p; the graph is recaptured when the arithmetic or kernel selection changed.
uint64_t matvec_modes_key(const fmmbem_handle* h) {
    uint64_t key = 1469598103934665603ull;
    for (int q = 0; q <= h->opts.p_max; ++q) {
        const int mode = h->precision * 16 + h->m2l_mode + 4 * h->p2p_variant + 128 * h->layer + 256 * h->m2l_tc_at[q] +
                         512 * h->tree_tc_at[q] + 2048 * h->near_at;
        key = (key ^ (uint64_t)mode) * 1099511628211ull;
    }
    return key;
}

int matvec_capture_body(fmmbem_handle* h, int p) {
    const int64_t keep = h->launches;
    const int rc = matvec_launch(h, p, h->xfix, h->kw);
    h->dloop_mv_launches[p] = h->launches - keep;
    h->launches = keep;
    return rc;
}

int matvec_sorted(fmmbem_handle* h, int p, const double* xs, double* ys) {
    const int mode = h->precision * 16 + h->m2l_mode + 4 * h->p2p_variant + 64 * (h->prof_on ? 1 : 0) + 128 * h->layer +
                     256 * h->m2l_tc_at[p] + 512 * h->tree_tc_at[p] + 1024 * (h->prof_serial ? 1 : 0) +
                     2048 * h->near_at;
    if (!h->use_graphs || xs != h->xfix || ys != h->kw || h->stream == nullptr)
        return matvec_launch(h, p, xs, ys);
    prof_harvest(h);
    const int g_i = p + (h->precision == FMMBEM_FP64 ? FMMBEM_P_MAX + 1 : 0);  // graph slot
    if (h->mv_graph[g_i] && h->mv_graph_mode[g_i] != mode) {
        cudaGraphExecDestroy(h->mv_graph[g_i]);
        h->mv_graph[g_i] = nullptr;
    }
    if (!h->mv_graph[g_i]) {
        cudaGraph_t g = nullptr;
        const int64_t keep = h->launches;
        FMM_CU(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
        h->capturing = g_i;
        const int rc = matvec_launch(h, p, xs, ys);
        h->capturing = -1;
        cudaError_t e = cudaStreamEndCapture(h->stream, &g);
        if (rc < 0) { if (g) cudaGraphDestroy(g); return rc; }
        FMM_CU(e);
        e = cudaGraphInstantiate(&h->mv_graph[g_i], g, 0);
        cudaGraphDestroy(g);
        FMM_CU(e);
        h->mv_graph_mode[g_i] = mode;
        h->graph_launches[g_i] = h->launches - keep;
        h->launches = keep;
    }
    FMM_CU(cudaGraphLaunch(h->mv_graph[g_i], h->stream));
    h->launches += h->graph_launches[g_i];
    if (h->prof_on) h->pending_graph = g_i;
    if (h->prof_on) {
        const double q = (double)(p + 1) * (p + 1);
        h->prof.m2l_flops += 2.0 * q * q * h->ncomp * h->nsys * (double)h->n_m2l;
        h->prof.p2p_interactions += (double)h->n_p2p_inter * h->nsys;
        h->prof.tc_flops += tc_flops(h, p);
    }
    return 0;
}

// Forks the pending near field onto the second stream when the far field reaches stage
// (see near_at); ev_join follows it there.
int near_release(fmmbem_handle* h, int stage) {
    // FP64 mat-vecs release it before their P2M, which is long (FP64 recurrences) and would
    // otherwise run alone
    const int at = h->near_fp64 ? 0 : h->near_at;
    if (!h->near_pending || stage < at) return 0;
    h->near_pending = false;
    FMM_CU(cudaEventRecord(h->ev_fork, h->stream));
    FMM_CU(cudaStreamWaitEvent(h->stream2, h->ev_fork, 0));
    FMM_TRY(near_field(h, h->near_fp64, h->stream2));
    FMM_CU(cudaEventRecord(h->ev_join, h->stream2));
    return 0;
}

static int matvec_launch(fmmbem_handle* h, int p, const double* xs, double* ys) {
    const bool fp64 = h->precision == FMMBEM_FP64;
    h->xin = xs;
    prof_begin(h, FMMBEM_PASS_MATVEC);
    // near field on the second stream, released once P2M is queued (near_at), far field on the
    // handle's stream, joined before L2P; in serial profiling the near field runs first on the
    // handle's stream, so that every pass's events time its kernels alone (no wait for SMs held
    // by the other field)
    if (!fp64) FMM_TRY(pack_sources(h));
    if (h->prof_on && h->prof_serial) {
        FMM_TRY(near_field(h, fp64, h->stream));
        FMM_TRY(far_field(h, p, fp64));
    } else {
        h->near_pending = true;
        h->near_fp64 = fp64;
        FMM_TRY(near_release(h, 0));
        FMM_TRY(far_field(h, p, fp64));  // releases the near field at stage near_at
        FMM_TRY(near_release(h, 4));
        FMM_CU(cudaStreamWaitEvent(h->stream, h->ev_join, 0));
    }
    FMM_TRY(far_eval_add(h, p, fp64, ys, operator_scale(h)));
    prof_end(h, FMMBEM_PASS_MATVEC, 0);
    if (h->prof_on && h->capturing < 0) {  // a captured graph counts its work at each replay
        const double q = (double)(p + 1) * (p + 1);
        h->prof.m2l_flops += 2.0 * q * q * h->ncomp * h->nsys * (double)h->n_m2l;
        h->prof.p2p_interactions += (double)h->n_p2p_inter * h->nsys;
        h->prof.tc_flops += tc_flops(h, p);
    }
    return 0;
}

}  // namespace fmmbem

using namespace fmmbem;

extern "C" {

const char* fmmbem_last_error(void) { return g_err; }

int fmmbem_default_opts(fmmbem_opts* o) {
    if (!o) return FMMBEM_EINVAL;
    o->p_max = FMMBEM_P_MAX;
    o->near_factor = 2.0;
    o->mu = 1.0;
    o->precision = FMMBEM_MIXED;
    o->restart = 50;
    o->max_iter = 100;
    o->stream = nullptr;
    o->nrhs = 1;
    o->near_k = 20;
    return 0;
}

int fmmbem_relaxed_p(double eta, double rho_prev, int p_initial, int p_min) {
    return fmmbem::relaxed_p(eta, rho_prev, p_initial, p_min);
}

void fmmbem_destroy(fmmbem_handle* h) {
    if (!h) return;
    // the handle's own streams finish first; then its memory goes back to the pool in
    // stream order (no device-wide synchronization)
    if (h->stream2) cudaStreamSynchronize(h->stream2);
    if (h->istream) cudaStreamSynchronize(h->istream);
    fmm_alloc_stream() = h->stream;
    void* bufs[] = {h->perm, h->body, h->body_acc, h->rf_r, h->rf_d, h->tgt_d, h->tgt_f, h->nrm_d, h->nrm_f, h->nrm_pt, h->verts, h->src_d, h->src_f, h->src_rel, h->tgt_rel, h->src_w, h->cell_cs, h->cell_range, h->cell_rad,
                    h->cell_child, h->cell_level, h->cell_parent, h->leaves, h->parents, h->leaf_class, h->m2l_ptr, h->m2l_src, h->p2p_ptr,
                    h->p2p_src, h->p2p_rec, h->p2p_off, h->p2p_len, h->p2p_items, h->p2p_cnt, h->p2p_toff, h->stage_ptr, h->stage_first, h->stage_bytes, h->corr_ptr, h->corr_col, h->corr_sl, h->corr_dl, h->corr_sl_f, h->corr_dl_f, h->oct_d, h->oct_f, h->M, h->L,
                    h->xs, h->ys, h->ynear, h->ycorr, h->m2l_pt, h->m2l_ps, h->m2l_refl, h->sign_f, h->sign_d, h->m2l_tiles, h->tab_d, h->tab_f, h->tab_tc, h->m2l_tiles_tc, h->tc_src_info, h->tc_dst_info, h->tree_tab_tc, h->tree_tiles, h->tree_info, h->tc_err, h->kerr, h->V, h->kw, h->xfix, h->kb, h->kx, h->kr, h->kpart, h->kh, h->kyv, h->arn_bar};
    for (void* b : bufs)
        if (b) fmm_free(b);
    pinned_put(h->kh_host, sizeof(double) * 3 * (h->kr_m + 2) * h->nrhs);
    pinned_put(h->arn_out_host, sizeof(double) * (2 * 65 + 1) * h->nrhs);
    for (int q = 0; q < fmmbem_handle::NGRAPH; ++q) {
        if (h->mv_graph[q]) cudaGraphExecDestroy(h->mv_graph[q]);
        for (int e = 0; e < 2 * FMMBEM_N_PASSES; ++e)
            if (h->gev[q][e]) cudaEventDestroy(h->gev[q][e]);
    }
    if (h->ev_in) cudaEventDestroy(h->ev_in);
    if (h->ev_out) cudaEventDestroy(h->ev_out);
    if (h->istream) cudaStreamDestroy(h->istream);
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    dloop_free(h);
    if (h->stream2) cudaStreamDestroy(h->stream2);
    prof_free(h);
    delete h;
}

int fmmbem_create(const fmmbem_mesh* mesh, int kernel, int gauss_k, int ncrit, double theta, const fmmbem_opts* opts,
                  fmmbem_handle** out) {
    const auto t0 = std::chrono::steady_clock::now();
    if (!out) { fmmbem_set_error("out is NULL"); return FMMBEM_EINVAL; }
    *out = nullptr;
    if (!mesh || !mesh->vertices || !mesh->triangles || mesh->n_panels <= 0 || mesh->n_vertices < 3) {
        fmmbem_set_error("empty or NULL mesh");
        return FMMBEM_EINVAL;
    }
    if (mesh->n_panels > (int64_t)1 << 28) { fmmbem_set_error("too many panels"); return FMMBEM_EINVAL; }
    if (kernel != FMMBEM_LAPLACE && kernel != FMMBEM_STOKES) { fmmbem_set_error("unknown kernel %d", kernel); return FMMBEM_EINVAL; }
    if (!(theta > 0.0 && theta < 1.0)) { fmmbem_set_error("theta must lie in (0, 1)"); return FMMBEM_EINVAL; }
    if (ncrit < gauss_k || ncrit < 1) { fmmbem_set_error("ncrit must be >= gauss_k"); return FMMBEM_EINVAL; }
    fmmbem_opts o;
    fmmbem_default_opts(&o);
    if (opts) o = *opts;
    if (o.p_max < 1 || o.p_max > FMMBEM_P_MAX) { fmmbem_set_error("p_max outside [1, %d]", FMMBEM_P_MAX); return FMMBEM_EINVAL; }
    if (o.restart < 1 || o.restart > 60) { fmmbem_set_error("restart outside [1, 60]"); return FMMBEM_EINVAL; }
    if (o.max_iter < 1) { fmmbem_set_error("max_iter < 1"); return FMMBEM_EINVAL; }
    if (!(o.near_factor >= 0.0)) { fmmbem_set_error("near_factor < 0"); return FMMBEM_EINVAL; }
    if (!(o.mu > 0.0)) { fmmbem_set_error("mu must be > 0"); return FMMBEM_EINVAL; }
    if (o.precision != FMMBEM_FP64 && o.precision != FMMBEM_MIXED && o.precision != FMMBEM_MIXED_REFINED) {
        fmmbem_set_error("bad precision");
        return FMMBEM_EINVAL;
    }
    if (o.precision == FMMBEM_MIXED_REFINED && o.nrhs > 1) {
        fmmbem_set_error("refined solves take one right-hand side");
        return FMMBEM_EINVAL;
    }
    if (kernel == FMMBEM_LAPLACE && o.nrhs != 1 && o.nrhs != FMMBEM_BATCH) {
        fmmbem_set_error("a Laplace handle takes nrhs 1 or %d", FMMBEM_BATCH);
        return FMMBEM_EINVAL;
    }
    if (kernel == FMMBEM_STOKES && (o.nrhs < 1 || o.nrhs > FMMBEM_STOKES_BATCH_MAX)) {
        fmmbem_set_error("a Stokes handle takes nrhs in [1, %d]", FMMBEM_STOKES_BATCH_MAX);
        return FMMBEM_EINVAL;
    }
    if (o.near_k == 0) o.near_k = 20;  // callers that fill the options themselves get the default rule
    if (o.near_k != 6 && o.near_k != 12 && o.near_k != 20 && o.near_k != 30 && o.near_k != 42) {
        fmmbem_set_error("near_k must be 6, 12, 20, 30 or 42 (collapsed products of nu x (nu - 1) points)");
        return FMMBEM_EINVAL;
    }
    if (mesh->n_bodies > 1) {
        if (!mesh->body_of_panel) { fmmbem_set_error("n_bodies > 1 needs body_of_panel"); return FMMBEM_EINVAL; }
        for (int64_t j = 0; j < mesh->n_panels; ++j)
            if (mesh->body_of_panel[j] < 0 || mesh->body_of_panel[j] >= mesh->n_bodies) {
                fmmbem_set_error("body_of_panel[%lld] = %d outside [0, %d)", (long long)j, mesh->body_of_panel[j],
                                 mesh->n_bodies);
                return FMMBEM_EINVAL;
            }
    }

    fmmbem_handle* h = new fmmbem_handle();
    fmm_alloc_stream() = (cudaStream_t)o.stream;
    {
        // freed device blocks stay in the default pool for the next handle
        static std::once_flag pool_once;
        std::call_once(pool_once, []() {
            int dev = 0;
            cudaMemPool_t pool;
            if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
                uint64_t keep = UINT64_MAX;
                cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
            }
        });
    }
    h->kernel = kernel;
    for (int q = 0; q <= FMMBEM_P_MAX; ++q) {  // defaults measured on the 81920-panel sphere
        h->m2l_tc_at[q] = 1;
        h->tree_tc_at[q] = q >= 6;
    }
    h->dof = kernel == FMMBEM_STOKES ? 3 : 1;
    h->nrhs = o.nrhs;
    h->ncomp = kernel == FMMBEM_STOKES ? 4 : o.nrhs;
    h->K = gauss_k;
    h->ncrit = ncrit;
    h->theta = theta;
    h->opts = o;
    h->precision = o.precision;
    h->stream = (cudaStream_t)o.stream;
    auto fail = [&](int rc) { fmmbem_destroy(h); return rc; };
    // the near field (stream2) runs at the lowest priority and the solver's far-field chain
    // (istream) at the highest, so that blocks of the short, dependent far-field kernels are
    // dispatched ahead of queued near-field blocks as SMs free up
    int prio_lo = 0, prio_hi = 0;
    cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
    if (cudaStreamCreateWithPriority(&h->stream2, cudaStreamNonBlocking, prio_lo) != cudaSuccess ||
        cudaStreamCreateWithPriority(&h->istream, cudaStreamNonBlocking, prio_hi) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming) != cudaSuccess) {
        fmmbem_set_error("stream/event creation failed: %s", cudaGetErrorString(cudaGetLastError()));
        return fail(FMMBEM_EDEVICE);
    }
    int rc = build_geometry_tree_lists(h, mesh);
    if (rc < 0) return fail(rc);
    // a Stokes batch keeps one copy of the expansions per vector (see handle.cuh)
    h->nsys = kernel == FMMBEM_STOKES ? o.nrhs : 1;
    h->esys = (size_t)h->n_cells * h->ncomp * ESTRIDE;
    h->n_bodies = mesh->n_bodies > 1 ? mesh->n_bodies : 1;
    if ((rc = dalloc(&h->body_acc, (size_t)h->n_bodies * h->dof)) < 0) return fail(rc);
    if (mesh->n_bodies > 1) {  // each sorted panel's body: body[s] = body_of_panel[perm[s]]
        std::vector<int> perm_h(h->N), body_h(h->N);
        if (cudaMemcpyAsync(perm_h.data(), h->perm, sizeof(int) * h->N, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
            cudaStreamSynchronize(h->stream) != cudaSuccess) {
            fmmbem_set_error("create: %s", cudaGetErrorString(cudaGetLastError()));
            return fail(FMMBEM_EDEVICE);
        }
        for (int64_t s_ = 0; s_ < h->N; ++s_) body_h[s_] = mesh->body_of_panel[perm_h[s_]];
        if ((rc = dalloc(&h->body, h->N)) < 0) return fail(rc);
        if (cudaMemcpyAsync(h->body, body_h.data(), sizeof(int) * h->N, cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
            cudaStreamSynchronize(h->stream) != cudaSuccess) {
            fmmbem_set_error("create: %s", cudaGetErrorString(cudaGetLastError()));
            return fail(FMMBEM_EDEVICE);
        }
    }
    rc = init_octant_tables(h);
    if (rc < 0) return fail(rc);
    rc = init_near_attrs();
    if (rc < 0) return fail(rc);
    rc = build_m2l_tables(h);
    if (rc < 0) return fail(rc);
    rc = build_m2l_tc(h);
    if (rc < 0) return fail(rc);
    h->m2l_mode = h->m2l_tc_ready ? FMMBEM_M2L_TENSOR : (h->m2l_tables ? FMMBEM_M2L_TABLES : FMMBEM_M2L_GATHER);
    const size_t ex = h->esys * h->nsys;
    const int64_t n = h->N * h->dof * h->nrhs;  // every work vector holds the nrhs vectors of a batch
    const int nb = h->nrhs;
    h->kr_m = o.restart;
    if ((rc = dalloc((double**)&h->M, ex)) < 0) return fail(rc);
    if ((rc = dalloc((double**)&h->L, ex)) < 0) return fail(rc);
    // per-mat-vec packed sources: one float4 per Gauss point (Laplace single layer), two
    // (Stokeslet strengths, or the Laplace double layer's moment w n)
    if ((rc = dalloc(&h->src_w, (size_t)h->NS * 2 * h->nsys)) < 0) return fail(rc);
    if ((rc = dalloc(&h->xs, n)) < 0 || (rc = dalloc(&h->ys, n)) < 0 || (rc = dalloc(&h->ynear, n)) < 0 ||
        (rc = dalloc(&h->ycorr, n)) < 0)
        return fail(rc);
    if ((rc = dalloc(&h->V, (size_t)(o.restart + 1) * n)) < 0) return fail(rc);
    if ((rc = dalloc(&h->xfix, n)) < 0) return fail(rc);
    if ((rc = dalloc(&h->kerr, 1)) < 0) return fail(rc);
    if (cudaMemsetAsync(h->kerr, 0, sizeof(int), h->stream) != cudaSuccess) return fail(FMMBEM_EDEVICE);
    if ((rc = dalloc(&h->kw, n)) < 0 || (rc = dalloc(&h->kb, n)) < 0 || (rc = dalloc(&h->kx, n)) < 0 ||
        (rc = dalloc(&h->kr, n)) < 0)
        return fail(rc);
    h->arn_blocks = arnoldi_blocks();
    if (h->arn_blocks < 1) { fmmbem_set_error("cooperative Arnoldi kernel cannot be resident"); return fail(FMMBEM_EDEVICE); }
    // partial dots: the fused Arnoldi step uses three areas of [64][blocks]; the restart dots [m+2][96]
    if ((rc = dalloc(&h->kpart, std::max((size_t)96 * (o.restart + 2), (size_t)3 * 64 * h->arn_blocks * nb))) < 0) return fail(rc);
    if ((rc = dalloc(&h->arn_bar, 2 * nb)) < 0) return fail(rc);  // one barrier pair per system of a batch
    if (cudaMemsetAsync(h->arn_bar, 0, 2 * nb * sizeof(unsigned), h->stream) != cudaSuccess) return fail(FMMBEM_EDEVICE);
    h->arn_out_host = reinterpret_cast<double*>(pinned_get(sizeof(double) * (2 * 65 + 1) * nb, cudaHostAllocMapped));
    if (!h->arn_out_host || cudaHostGetDevicePointer((void**)&h->arn_out_dev, h->arn_out_host, 0) != cudaSuccess) {
        fmmbem_set_error("mapped pinned allocation failed");
        return fail(FMMBEM_ENOMEM);
    }
    if ((rc = dalloc(&h->kh, (size_t)3 * (o.restart + 2) * nb)) < 0) return fail(rc);
    if ((rc = dalloc(&h->kyv, (size_t)(o.restart + 2) * nb)) < 0) return fail(rc);
    if (nb == 1 && ((rc = dalloc(&h->rf_r, n)) < 0 || (rc = dalloc(&h->rf_d, n)) < 0)) return fail(rc);
    h->kh_host = reinterpret_cast<double*>(pinned_get(sizeof(double) * 3 * (o.restart + 2) * nb, cudaHostAllocDefault));
    if (!h->kh_host) {
        fmmbem_set_error("pinned allocation failed");
        return fail(FMMBEM_ENOMEM);
    }
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) {
        fmmbem_set_error("create: %s", cudaGetErrorString(cudaGetLastError()));
        return fail(FMMBEM_EDEVICE);
    }
    h->setup_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    *out = h;
    return 0;
}

int64_t fmmbem_n_unknowns(const fmmbem_handle* h) { return h ? h->N * h->dof : -1; }

int fmmbem_n_bodies(const fmmbem_handle* h) { return h ? h->n_bodies : -1; }

int fmmbem_body_integrals(fmmbem_handle* h, const double* x_dev, double* out_host) {
    if (!h || !x_dev || !out_host) { fmmbem_set_error("NULL argument"); return FMMBEM_EINVAL; }
    const size_t bytes = sizeof(double) * h->n_bodies * h->dof;
    FMM_CU(cudaMemsetAsync(h->body_acc, 0, bytes, h->stream));
    k_body_sums<<<(unsigned)((h->N + 255) / 256), 256, 0, h->stream>>>(x_dev, h->perm, h->tgt_d, h->body, h->N, h->dof,
                                                                       h->body_acc);
    FMM_LAUNCHED();
    h->launches += 1;
    FMM_CU(cudaMemcpyAsync(out_host, h->body_acc, bytes, cudaMemcpyDeviceToHost, h->stream));
    FMM_CU(cudaStreamSynchronize(h->stream));
    return 0;
}

int fmmbem_set_precision(fmmbem_handle* h, int precision) {
    if (!h || (precision != FMMBEM_FP64 && precision != FMMBEM_MIXED && precision != FMMBEM_MIXED_REFINED)) {
        fmmbem_set_error("bad precision");
        return FMMBEM_EINVAL;
    }
    if (precision == FMMBEM_MIXED_REFINED && h->nrhs > 1) {
        fmmbem_set_error("refined solves take one right-hand side");
        return FMMBEM_ESTATE;
    }
    h->precision = precision;
    return 0;
}

int fmmbem_set_layer(fmmbem_handle* h, int layer) {
    if (!h || (layer != FMMBEM_LAYER_SINGLE && layer != FMMBEM_LAYER_DOUBLE)) { fmmbem_set_error("bad layer"); return FMMBEM_EINVAL; }
    if (layer == FMMBEM_LAYER_DOUBLE && h->nrhs > 1) {
        fmmbem_set_error("the double-layer operator is not built for batched handles");
        return FMMBEM_ESTATE;
    }
    h->layer = layer;
    return 0;
}

int fmmbem_set_tc_thresholds(fmmbem_handle* h, int m2l_min_p, int tree_min_p) {
    if (!h || m2l_min_p < 1 || tree_min_p < 1) { fmmbem_set_error("bad tensor-core threshold"); return FMMBEM_EINVAL; }
    for (int q = 0; q <= FMMBEM_P_MAX; ++q) {
        h->m2l_tc_at[q] = q >= m2l_min_p;
        h->tree_tc_at[q] = q >= tree_min_p;
    }
    return 0;
}

// Milliseconds of the handle's mat-vec at order p (its captured graph on the fixed buffers),
// summed over three runs after a capture run.
static int time_matvec(fmmbem_handle* h, int p, cudaEvent_t e0, cudaEvent_t e1, float* ms_out) {
    float ms = 0.f;
    for (int rep = 0; rep < 4; ++rep) {
        FMM_CU(cudaEventRecord(e0, h->stream));
        FMM_TRY(matvec_sorted(h, p, h->xfix, h->kw));
        FMM_CU(cudaEventRecord(e1, h->stream));
        FMM_CU(cudaEventSynchronize(e1));
        float t = 0.f;
        FMM_CU(cudaEventElapsedTime(&t, e0, e1));
        if (rep > 0) ms += t;
    }
    *ms_out = ms;
    return 0;
}

int fmmbem_autotune(fmmbem_handle* h, int p_lo, int p_hi, int* choice) {
    if (!h || p_lo < 1 || p_hi > h->opts.p_max || p_lo > p_hi) { fmmbem_set_error("need 1 <= p_lo <= p_hi <= p_max"); return FMMBEM_EINVAL; }
    if (choice) choice[0] = h->p2p_variant;
    if (h->precision == FMMBEM_FP64 || !h->m2l_tc_ready || h->m2l_mode != FMMBEM_M2L_TENSOR) {
        for (int p = p_lo; p <= p_hi; ++p)
            if (choice) choice[p] = 2 * h->m2l_tc_at[p] + h->tree_tc_at[p];
        return 0;  // nothing to choose: the tensor-core paths are not in use
    }
    // the solver's fixed mat-vec buffers carry the timed products (zero input: no kernel has a
    // data-dependent path, so the timing is that of any input)
    FMM_CU(cudaMemsetAsync(h->xfix, 0, sizeof(double) * h->N * h->dof * h->nrhs, h->stream));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    FMM_CU(cudaEventCreate(&e0));
    FMM_CU(cudaEventCreate(&e1));
    int rc = 0;
    {  // the near-field schedule, at the highest order (the near field does not depend on p)
        const int keep = h->p2p_variant;
        float best = 0.f;
        int best_v = keep;
        for (int v : {3, 1, 0, 2}) {
            h->p2p_variant = v;
            float ms = 0.f;
            rc = time_matvec(h, p_hi, e0, e1, &ms);
            if (rc < 0) break;
            if (v == 3 || ms < best) { best = ms; best_v = v; }
        }
        h->p2p_variant = rc < 0 ? keep : best_v;
        if (choice) choice[0] = h->p2p_variant;
    }
    for (int p = p_lo; p <= p_hi && rc == 0; ++p) {
        float best = 0.f;
        int best_cfg = 3;
        for (int cfg = 3; cfg >= 0 && rc == 0; --cfg) {  // bit 1: M2L, bit 0: M2M/L2L on the tensor cores
            h->m2l_tc_at[p] = (cfg >> 1) & 1;
            h->tree_tc_at[p] = cfg & 1;
            float ms = 0.f;
            for (int rep = 0; rep < 4 && rc == 0; ++rep) {  // the first run captures the graph
                if (cudaEventRecord(e0, h->stream) != cudaSuccess) { rc = FMMBEM_EDEVICE; break; }
                rc = matvec_sorted(h, p, h->xfix, h->kw);
                if (rc < 0) break;
                if (cudaEventRecord(e1, h->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
                    rc = FMMBEM_EDEVICE;
                    break;
                }
                float t = 0.f;
                cudaEventElapsedTime(&t, e0, e1);
                if (rep > 0) ms += t;
            }
            if (rc == 0 && (cfg == 3 || ms < best)) {
                best = ms;
                best_cfg = cfg;
            }
        }
        h->m2l_tc_at[p] = (best_cfg >> 1) & 1;
        h->tree_tc_at[p] = best_cfg & 1;
        if (choice) choice[p] = best_cfg;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc < 0 ? rc : 0;
}

int fmmbem_create_tuned(const fmmbem_mesh* mesh, int kernel, int gauss_k, int n_cand, const int* ncrit_cand,
                        double theta, const fmmbem_opts* opts, int p_lo, int p_hi, fmmbem_handle** out, int* ncrit_out,
                        double* ms_out) {
    if (!out || !ncrit_cand || n_cand < 1 || p_lo < 1 || p_lo > p_hi) {
        fmmbem_set_error("need candidates and 1 <= p_lo <= p_hi");
        return FMMBEM_EINVAL;
    }
    *out = nullptr;
    fmmbem_handle* best = nullptr;
    double best_ms = 0.0;
    int best_nc = 0;
    for (int i = 0; i < n_cand; ++i) {
        fmmbem_handle* h = nullptr;
        int rc = fmmbem_create(mesh, kernel, gauss_k, ncrit_cand[i], theta, opts, &h);
        if (rc == 0 && p_hi > h->opts.p_max) {
            fmmbem_set_error("p_hi beyond p_max");
            rc = FMMBEM_EINVAL;
        }
        if (rc == 0) rc = fmmbem_autotune(h, p_lo, p_hi, nullptr);
        double total = 0.0;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (rc == 0 && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)) rc = FMMBEM_EDEVICE;
        if (rc == 0 && cudaMemsetAsync(h->xfix, 0, sizeof(double) * h->N * h->dof * h->nrhs, h->stream) != cudaSuccess)
            rc = FMMBEM_EDEVICE;
        for (int p = p_lo; p <= p_hi && rc == 0; ++p) {
            float ms = 0.f;
            rc = time_matvec(h, p, e0, e1, &ms);
            total += ms / 3.0;
        }
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (rc < 0) {
            fmmbem_destroy(h);
            fmmbem_destroy(best);
            return rc;
        }
        if (!best || total < best_ms) {
            fmmbem_destroy(best);
            best = h;
            best_ms = total;
            best_nc = ncrit_cand[i];
        } else {
            fmmbem_destroy(h);
        }
    }
    *out = best;
    if (ncrit_out) *ncrit_out = best_nc;
    if (ms_out) *ms_out = best_ms;
    return 0;
}

int fmmbem_set_p2p_variant(fmmbem_handle* h, int variant) {
    if (!h || variant < 0 || variant > 3) { fmmbem_set_error("bad P2P variant"); return FMMBEM_EINVAL; }
    h->p2p_variant = variant;
    return 0;
}

int fmmbem_set_device_loop(fmmbem_handle* h, int on) {
    if (!h || (on != 0 && on != 1)) { fmmbem_set_error("device loop: on must be 0 or 1"); return FMMBEM_EINVAL; }
    h->dloop_on = on != 0;
    return 0;
}

int fmmbem_set_m2l_mode(fmmbem_handle* h, int mode) {
    if (!h || (mode != FMMBEM_M2L_TABLES && mode != FMMBEM_M2L_GATHER && mode != FMMBEM_M2L_TENSOR)) {
        fmmbem_set_error("bad M2L mode");
        return FMMBEM_EINVAL;
    }
    if (mode == FMMBEM_M2L_TABLES && !h->m2l_tables) { fmmbem_set_error("M2L operator tables were not built"); return FMMBEM_ESTATE; }
    if (mode == FMMBEM_M2L_TENSOR && !h->m2l_tc_ready) { fmmbem_set_error("tensor-core M2L tables were not built"); return FMMBEM_ESTATE; }
    h->m2l_mode = mode;
    return 0;
}

int fmmbem_matvec(fmmbem_handle* h, int p, const double* x_dev, double* y_dev) {
    if (!h || !x_dev || !y_dev) { fmmbem_set_error("NULL argument"); return FMMBEM_EINVAL; }
    if (p < 1 || p > h->opts.p_max) { fmmbem_set_error("p=%d outside [1, %d]", p, h->opts.p_max); return FMMBEM_EINVAL; }
    if (x_dev == y_dev) { fmmbem_set_error("x and y alias"); return FMMBEM_EINVAL; }
    FMM_TRY(perm_in(h, x_dev, h->xs));
    FMM_TRY(matvec_sorted(h, p, h->xs, h->ys));
    FMM_TRY(perm_out(h, h->ys, y_dev));
    return 0;
}

int fmmbem_matvec_direct(fmmbem_handle* h, const double* x_dev, double* y_dev) {
    if (!h || !x_dev || !y_dev || x_dev == y_dev) { fmmbem_set_error("bad argument"); return FMMBEM_EINVAL; }
    FMM_TRY(perm_in(h, x_dev, h->xs));
    if (h->layer == FMMBEM_LAYER_DOUBLE) {  // 1/2 x + K x, in FP64
        const int64_t nd = h->N * h->dof;
        FMM_TRY(direct_field(h, true, 1, h->xs, h->ys));
        k_axpy_half<<<(unsigned)((nd + 255) / 256), 256, 0, h->stream>>>(h->ys, h->xs, nd);
        FMM_LAUNCHED();
    } else {
        for (int q = 0; q < h->nrhs; ++q)  // a batch: each vector in turn
            FMM_TRY(direct_field(h, h->precision == FMMBEM_FP64, 0, h->xs + q * h->N * h->dof, h->ys + q * h->N * h->dof));
    }
    FMM_TRY(perm_out(h, h->ys, y_dev));
    return 0;
}

int fmmbem_rhs(fmmbem_handle* h, const double* known_dev, double* b_dev) {
    if (!h || !known_dev || !b_dev || known_dev == b_dev) { fmmbem_set_error("bad argument"); return FMMBEM_EINVAL; }
    if (h->kernel != FMMBEM_LAPLACE) { fmmbem_set_error("fmmbem_rhs needs a Laplace handle"); return FMMBEM_ESTATE; }
    FMM_TRY(perm_in(h, known_dev, h->xs));
    for (int q = 0; q < h->nrhs; ++q) {  // a batch: each vector in turn
        FMM_TRY(direct_field(h, true, 1, h->xs + q * h->N, h->ys + q * h->N));
        k_axpy_half<<<(unsigned)((h->N + 255) / 256), 256, 0, h->stream>>>(h->ys + q * h->N, h->xs + q * h->N, h->N);
        FMM_LAUNCHED();
    }
    FMM_TRY(perm_out(h, h->ys, b_dev));
    return 0;
}

int fmmbem_stokes_dl_apply(fmmbem_handle* h, const double* u_dev, double* y_dev) {
    if (!h || !u_dev || !y_dev || u_dev == y_dev) { fmmbem_set_error("bad argument"); return FMMBEM_EINVAL; }
    if (h->kernel != FMMBEM_STOKES) { fmmbem_set_error("needs a Stokes handle"); return FMMBEM_ESTATE; }
    FMM_TRY(perm_in(h, u_dev, h->xs));
    FMM_TRY(direct_field(h, true, 1, h->xs, h->ys));
    FMM_TRY(perm_out(h, h->ys, y_dev));
    return 0;
}

static int solve_checked(fmmbem_handle* h, const double* rhs_dev, double tol, int relax, int p_initial, int p_min,
                         double* x_dev, int* iters, int* p_hist, double* res_hist, double* true_res);

int fmmbem_solve(fmmbem_handle* h, const double* rhs_dev, double tol, int relax, int p_initial, int p_min,
                 double* x_dev, int* iters, int* p_hist, double* res_hist, double* true_res) {
    if (h && h->nrhs > 1) { fmmbem_set_error("batched handle: use fmmbem_solve_batch"); return FMMBEM_ESTATE; }
    return solve_checked(h, rhs_dev, tol, relax, p_initial, p_min, x_dev, iters, p_hist, res_hist, true_res);
}

int fmmbem_solve_batch(fmmbem_handle* h, const double* rhs_dev, double tol, int relax, int p_initial, int p_min,
                       double* x_dev, int* iters, int* p_hist, double* res_hist, double* true_res) {
    if (h && h->nrhs == 1) { fmmbem_set_error("fmmbem_solve_batch needs a batched handle (opts.nrhs)"); return FMMBEM_ESTATE; }
    return solve_checked(h, rhs_dev, tol, relax, p_initial, p_min, x_dev, iters, p_hist, res_hist, true_res);
}

static int solve_checked(fmmbem_handle* h, const double* rhs_dev, double tol, int relax, int p_initial, int p_min,
                         double* x_dev, int* iters, int* p_hist, double* res_hist, double* true_res) {
    if (!h || !rhs_dev || !x_dev) { fmmbem_set_error("NULL argument"); return FMMBEM_EINVAL; }
    if (p_initial < 1 || p_initial > h->opts.p_max || p_min < 1 || p_min > p_initial) {
        fmmbem_set_error("need 1 <= p_min <= p_initial <= p_max");
        return FMMBEM_EINVAL;
    }
    if (!(tol > 0.0 && tol < 1.0)) { fmmbem_set_error("tol must lie in (0, 1)"); return FMMBEM_EINVAL; }
    FMM_TRY(perm_in(h, rhs_dev, h->kb));
    int rc = gmres_solve(h, h->kb, tol, relax, p_initial, p_min, h->kx, iters, p_hist, res_hist, true_res);
    if (rc < 0) return rc;
    FMM_TRY(perm_out(h, h->kx, x_dev));
    return rc;
}

int fmmbem_solve_host(fmmbem_handle* h, const double* rhs_host, double tol, int relax, int p_initial, int p_min,
                      double* x_host, int* iters, int* p_hist, double* res_hist, double* true_res) {
    if (!h || !rhs_host || !x_host) { fmmbem_set_error("NULL argument"); return FMMBEM_EINVAL; }
    if (h->nrhs > 1) { fmmbem_set_error("batched handle: use fmmbem_solve_batch"); return FMMBEM_ESTATE; }
    const int64_t n = h->N * h->dof;
    FMM_CU(cudaMemcpyAsync(h->ys, rhs_host, sizeof(double) * n, cudaMemcpyHostToDevice, h->stream));
    int rc = fmmbem_solve(h, h->ys, tol, relax, p_initial, p_min, h->xs, iters, p_hist, res_hist, true_res);
    if (rc < 0) return rc;
    FMM_CU(cudaMemcpyAsync(x_host, h->xs, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream));
    FMM_CU(cudaStreamSynchronize(h->stream));
    return rc;
}

int fmmbem_expansion_eval(int kind, int p, const double* center, double scale, int n_src, const double* src_dev,
                          int n_tgt, const double* tgt_dev, double* out_dev, void* stream) {
    if ((kind != 0 && kind != 1) || p < 0 || p > FMMBEM_P_MAX || !center || !(scale > 0.0) || n_src < 0 ||
        n_tgt < 0 || (n_src && !src_dev) || (n_tgt && (!tgt_dev || !out_dev))) {
        fmmbem_set_error("bad argument");
        return FMMBEM_EINVAL;
    }
    return fmmbem::expansion_eval(kind, p, center, scale, n_src, src_dev, n_tgt, tgt_dev, out_dev, (cudaStream_t)stream);
}

int fmmbem_check_waits(fmmbem_handle* h) {
    if (!h) { fmmbem_set_error("NULL handle"); return FMMBEM_EINVAL; }
    FMM_CU(cudaStreamSynchronize(h->stream2));
    FMM_CU(cudaStreamSynchronize(h->istream));
    return read_wait_flags(h, h->stream);
}

int fmmbem_set_wait_limit(fmmbem_handle* h, unsigned limit) {
    if (!h) { fmmbem_set_error("NULL handle"); return FMMBEM_EINVAL; }
    h->wait_limit = limit ? limit : (1u << 26);
    return 0;
}


int fmmbem_get_stats(const fmmbem_handle* h, fmmbem_stats* s) {
    if (!h || !s) { fmmbem_set_error("NULL argument"); return FMMBEM_EINVAL; }
    s->n_panels = h->N;
    s->n_sources = h->NS;
    s->n_cells = h->n_cells;
    s->n_leaves = h->n_leaves;
    s->n_levels = h->n_levels;
    s->n_m2l_pairs = h->n_m2l;
    s->n_m2l_same_level = h->n_m2l_same;
    s->n_p2p_pairs = h->n_p2p;
    s->n_p2p_interactions = h->n_p2p_inter;
    s->n_corrections = h->n_corr;
    s->n_m2l_tables = h->n_tables;
    s->n_m2l_tiles = h->n_tiles;
    s->setup_seconds = h->setup_seconds;
    s->n_m2l_tiles_tc = h->n_tiles_tc;
    return 0;
}

int fmmbem_profile_enable(fmmbem_handle* h, int enable) {
    if (!h) { fmmbem_set_error("NULL handle"); return FMMBEM_EINVAL; }
    FMM_CU(cudaStreamSynchronize(h->stream));
    ProfState* s = prof_state(h);
    s->recs.clear();
    s->used = 0;
    for (auto& e : s->open) e = nullptr;
    memset(&h->prof, 0, sizeof(h->prof));
    h->launches = 0;
    h->pending_graph = -1;
    h->prof_on = enable != 0;
    h->prof_serial = enable == 2;
    return 0;
}

int fmmbem_profile_get(fmmbem_handle* h, fmmbem_profile* out) {
    if (!h || !out) { fmmbem_set_error("NULL argument"); return FMMBEM_EINVAL; }
    FMM_CU(cudaStreamSynchronize(h->stream));
    FMM_CU(cudaStreamSynchronize(h->istream));
    prof_harvest(h);
    ProfState* s = prof_state(h);
    for (const auto& r : s->recs) {
        float ms = 0.f;
        FMM_CU(cudaEventElapsedTime(&ms, r.a, r.b));
        h->prof.ms[r.pass] += ms;
        h->prof.launches[r.pass] += r.launches;
        h->prof.calls[r.pass] += 1;
        if (r.tc) h->prof.tc_ms += ms;
    }
    s->recs.clear();
    s->used = 0;
    h->prof.kernel_launches = h->launches;
    *out = h->prof;
    return 0;
}

}  // extern "C"
