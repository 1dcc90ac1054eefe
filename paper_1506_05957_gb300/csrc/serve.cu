// Serving runtime: many relaxed BEM solves of different meshes, operators and tolerances
// on one GPU at once (the paper solves one problem at a time; this is the request loop
// around its solver).
//
// fmmbem_server_submit copies the request (mesh, right-hand side, solver settings) into a
// queue and returns a ticket. max_active worker threads take requests in arrival order;
// a request is admitted once a worker is free and its device-memory estimate fits in
// what the HBM budget has left, so later small requests go ahead of a large one that
// does not fit yet (continuous admission, not a FIFO of whole batches). An admitted
// request gets its own handle (tree, lists, operators, expansions and Krylov basis stay
// resident for the request's lifetime) and its own CUDA stream; the workers' relaxed
// mat-vecs are independent kernel streams that interleave on the device. When a solve
// ends its memory returns to the budget and the next queued request is admitted.
// fmmbem_server_wait blocks until a ticket's result (solution, iterations, timings) is in.
//
// Handles of finished requests are kept in an idle cache (least recently used first out,
// up to fmmbem_server_set_cache's count and always inside the HBM budget): a later request
// on the same mesh with the same operator and settings takes the cached handle (tree, lists,
// operators, correction rows and captured mat-vec graphs) and skips fmmbem_create. The
// cache is keyed by a hash of the mesh and settings and confirmed by comparing the mesh.
#include <math.h>
#include <string.h>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>
#include "handle.cuh"

namespace {

using clk = std::chrono::steady_clock;

struct Request {
    int64_t ticket = 0;
    std::vector<double> vertices;
    std::vector<int32_t> triangles;
    std::vector<double> rhs;
    int kernel = FMMBEM_LAPLACE, gauss_k = 4, ncrit = 150;
    double theta = 0.5;
    fmmbem_opts opts{};
    double tol = 1e-6;
    int relax = 1, p_initial = 10, p_min = 3;
    double* x_host = nullptr;
    int64_t bytes = 0;  // admission estimate
    uint64_t key = 0;   // hash of the mesh and the handle settings (the handle cache's key)
    clk::time_point t_submit;
    fmmbem_result res{};
    bool done = false;
};

// An idle handle of a finished request, with what it was created from.
struct CacheEntry {
    uint64_t key = 0;
    std::vector<double> vertices;
    std::vector<int32_t> triangles;
    int kernel = 0, gauss_k = 0, ncrit = 0;
    double theta = 0.0;
    fmmbem_opts opts{};
    fmmbem_handle* h = nullptr;
    int64_t bytes = 0;
    uint64_t last_use = 0;
};

// 64-bit FNV-1a over a byte range, continuing from h.
uint64_t fnv1a(const void* data, size_t n, uint64_t h) {
    const unsigned char* b = static_cast<const unsigned char*>(data);
    for (size_t i = 0; i < n; ++i) {
        h ^= b[i];
        h *= 1099511628211ull;
    }
    return h;
}

// The settings that decide a handle's contents (the stream excluded).
bool same_opts(const fmmbem_opts& a, const fmmbem_opts& b) {
    return a.p_max == b.p_max && a.near_factor == b.near_factor && a.mu == b.mu && a.precision == b.precision &&
           a.restart == b.restart && a.max_iter == b.max_iter && a.nrhs == b.nrhs && a.near_k == b.near_k;
}

uint64_t request_key(const Request& r) {
    uint64_t h = 1469598103934665603ull;
    h = fnv1a(r.vertices.data(), r.vertices.size() * sizeof(double), h);
    h = fnv1a(r.triangles.data(), r.triangles.size() * sizeof(int32_t), h);
    const int ints[] = {r.kernel, r.gauss_k, r.ncrit, r.opts.p_max, r.opts.precision, r.opts.restart,
                        r.opts.max_iter, r.opts.nrhs, r.opts.near_k};
    const double dbl[] = {r.theta, r.opts.near_factor, r.opts.mu};
    h = fnv1a(ints, sizeof(ints), h);
    return fnv1a(dbl, sizeof(dbl), h);
}

bool entry_matches(const CacheEntry& e, const Request& r) {
    return e.key == r.key && e.kernel == r.kernel && e.gauss_k == r.gauss_k && e.ncrit == r.ncrit &&
           e.theta == r.theta && same_opts(e.opts, r.opts) && e.vertices == r.vertices && e.triangles == r.triangles;
}

}  // namespace

struct fmmbem_server {
    int device = 0;
    int64_t budget = 0, in_use = 0;  // in_use counts running requests and cached handles
    int n_workers = 0;
    bool stop = false;
    int64_t next_ticket = 1;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request*> queue;
    std::map<int64_t, Request*> all;
    std::vector<std::thread> workers;
    std::vector<cudaStream_t> streams;  // one per worker; they outlive every handle created on them
    std::vector<CacheEntry*> idle;      // cached handles of finished requests
    int max_cached = 0;
    uint64_t use_clock = 0;
    int64_t hits = 0;
};

namespace {

// Remove the least recently used idle entry (caller holds the lock); the caller destroys it.
CacheEntry* pop_lru(fmmbem_server* s) {
    if (s->idle.empty()) return nullptr;
    size_t v = 0;
    for (size_t i = 1; i < s->idle.size(); ++i)
        if (s->idle[i]->last_use < s->idle[v]->last_use) v = i;
    CacheEntry* e = s->idle[v];
    s->idle.erase(s->idle.begin() + (long)v);
    s->in_use -= e->bytes;
    return e;
}

void destroy_entries(std::vector<CacheEntry*>& v) {
    for (CacheEntry* e : v) {
        fmmbem_destroy(e->h);
        delete e;
    }
    v.clear();
}

void worker_main(fmmbem_server* s, int idx) {
    cudaSetDevice(s->device);
    cudaStream_t st = s->streams[idx];
    for (;;) {
        Request* r = nullptr;
        CacheEntry* hit = nullptr;
        std::vector<CacheEntry*> evicted;
        {
            std::unique_lock<std::mutex> lock(s->mu);
            for (;;) {
                if (s->stop && s->queue.empty()) break;
                // the first queued request that has a cached handle or whose estimate fits in the
                // remaining budget once idle handles are given up
                auto it = s->queue.begin();
                for (; it != s->queue.end(); ++it) {
                    for (size_t i = 0; i < s->idle.size(); ++i)
                        if (entry_matches(*s->idle[i], **it)) {
                            hit = s->idle[i];
                            s->idle.erase(s->idle.begin() + (long)i);
                            break;
                        }
                    if (hit) {
                        r = *it;
                        r->bytes = hit->bytes;  // already counted in in_use
                    } else {
                        int64_t idle_bytes = 0;
                        for (CacheEntry* e : s->idle) idle_bytes += e->bytes;
                        if (s->in_use - idle_bytes + (*it)->bytes <= s->budget || s->in_use == idle_bytes) {
                            r = *it;
                            while (!s->idle.empty() && s->in_use + r->bytes > s->budget) evicted.push_back(pop_lru(s));
                            s->in_use += r->bytes;
                        }
                    }
                    if (r) break;
                }
                if (r) {
                    s->queue.erase(it);
                    break;
                }
                s->cv_work.wait(lock);
            }
            if (!r) break;
        }
        destroy_entries(evicted);
        const auto t_adm = clk::now();
        r->res.queue_s = std::chrono::duration<double>(t_adm - r->t_submit).count();
        fmmbem_handle* h = hit ? hit->h : nullptr;
        int rc = 0;
        if (!h) {
            fmmbem_mesh mesh{(int64_t)(r->vertices.size() / 3), r->vertices.data(), (int64_t)(r->triangles.size() / 3),
                             r->triangles.data()};
            fmmbem_opts o = r->opts;
            o.stream = st;
            rc = fmmbem_create(&mesh, r->kernel, r->gauss_k, r->ncrit, r->theta, &o, &h);
        }
        const auto t_set = clk::now();
        r->res.setup_s = std::chrono::duration<double>(t_set - t_adm).count();
        r->res.handle_reused = hit ? 1 : 0;
        if (rc == 0) {
            int iters = 0;
            double true_res = 0.0;
            rc = fmmbem_solve_host(h, r->rhs.data(), r->tol, r->relax, r->p_initial, r->p_min, r->x_host, &iters,
                                   nullptr, nullptr, &true_res);
            r->res.iters = iters;
            r->res.true_res = true_res;
        }
        const auto t_end = clk::now();
        r->res.solve_s = std::chrono::duration<double>(t_end - t_set).count();
        r->res.latency_s = std::chrono::duration<double>(t_end - r->t_submit).count();
        r->res.status = rc;
        r->res.device_bytes = r->bytes;
        // a handle that solved cleanly goes to the idle cache; a failed one is destroyed
        CacheEntry* keep = nullptr;
        if (h && rc >= 0 && s->max_cached > 0) {
            keep = hit ? hit : new CacheEntry();
            if (!hit) {
                keep->key = r->key;
                keep->kernel = r->kernel;
                keep->gauss_k = r->gauss_k;
                keep->ncrit = r->ncrit;
                keep->theta = r->theta;
                keep->opts = r->opts;
                keep->h = h;
                keep->bytes = r->bytes;
                keep->vertices.swap(r->vertices);
                keep->triangles.swap(r->triangles);
            }
        } else if (h) {
            fmmbem_destroy(h);
            if (hit) delete hit;
        }
        {
            std::lock_guard<std::mutex> lock(s->mu);
            if (keep) {
                keep->last_use = ++s->use_clock;
                s->idle.push_back(keep);
                while ((int)s->idle.size() > s->max_cached) evicted.push_back(pop_lru(s));
            } else {
                s->in_use -= r->bytes;
            }
            if (hit) ++s->hits;
            r->done = true;
            r->vertices.clear();
            r->triangles.clear();
            r->rhs.clear();
        }
        destroy_entries(evicted);
        s->cv_done.notify_all();
        s->cv_work.notify_all();
    }
}

}  // namespace

extern "C" {

int64_t fmmbem_estimate_bytes(int64_t n_panels, int kernel, int gauss_k, int ncrit, const fmmbem_opts* opts) {
    if (n_panels <= 0 || gauss_k < 1 || ncrit < 1) return -1;
    fmmbem_opts o;
    fmmbem_default_opts(&o);
    if (opts) o = *opts;
    const double dof = kernel == FMMBEM_STOKES ? 3.0 : 1.0, nc = kernel == FMMBEM_STOKES ? 4.0 : 1.0;
    const double n = (double)n_panels, ns = n * gauss_k;
    const double cells = 2.6 * ns / ncrit + 64.0;
    const double q = (double)fmmbem::ncoef(o.p_max) / fmmbem::NCOEF_MAX;
    double b = 0.0;
    b += n * (32 + 16 + 32 + 72 + 16 + 8 * 4) + ns * (32 + 16 + 16 + 16 * dof);  // geometry, sources, packed strengths
    b += cells * (nc * 2 * 2560.0 + 256.0);                                        // expansions, cell data
    const double tables = fmin(1100.0, 60.0 + 0.3 * cells);                       // distinct M2L geometries
    b += tables * 2.0e6 * q * q;                                                  // M2L operators (FP64, FP32, TF32 hi/lo)
    b += cells * 300.0 * 32.0;                                                     // interaction lists and row tables
    b += n * 30.0 * 12.0 * dof * dof;                                              // near-singular corrections
    b += (double)(o.restart + 10) * n * dof * 8.0;                                // Krylov basis and work vectors
    return (int64_t)(1.25 * b);                                                   // margin
}

int fmmbem_server_create(int max_active, int64_t hbm_budget, fmmbem_server** out) {
    if (!out || max_active < 1 || max_active > 64 || hbm_budget <= 0) {
        fmmbem_set_error("bad server arguments");
        return FMMBEM_EINVAL;
    }
    fmmbem_server* s = new fmmbem_server();
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        delete s;
        fmmbem_set_error("no CUDA device");
        return FMMBEM_EDEVICE;
    }
    s->budget = hbm_budget;
    s->n_workers = max_active;
    s->max_cached = 4 * max_active;
    for (int i = 0; i < max_active; ++i) {
        cudaStream_t st = nullptr;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            for (cudaStream_t q : s->streams) cudaStreamDestroy(q);
            delete s;
            fmmbem_set_error("cannot create the workers' streams");
            return FMMBEM_EDEVICE;
        }
        s->streams.push_back(st);
    }
    for (int i = 0; i < max_active; ++i) s->workers.emplace_back(worker_main, s, i);
    *out = s;
    return 0;
}

int fmmbem_server_set_cache(fmmbem_server* s, int max_handles) {
    if (!s || max_handles < 0) {
        fmmbem_set_error("bad cache size");
        return FMMBEM_EINVAL;
    }
    std::vector<CacheEntry*> evicted;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->max_cached = max_handles;
        while ((int)s->idle.size() > max_handles) evicted.push_back(pop_lru(s));
    }
    destroy_entries(evicted);
    s->cv_work.notify_all();
    return 0;
}

int64_t fmmbem_server_cache_hits(fmmbem_server* s) {
    if (!s) return 0;
    std::lock_guard<std::mutex> lock(s->mu);
    return s->hits;
}

int fmmbem_server_submit(fmmbem_server* s, const fmmbem_mesh* mesh, int kernel, int gauss_k, int ncrit, double theta,
                         const fmmbem_opts* opts, const double* rhs_host, double tol, int relax, int p_initial,
                         int p_min, double* x_host, int64_t* ticket) {
    if (!s || !mesh || !mesh->vertices || !mesh->triangles || mesh->n_panels <= 0 || mesh->n_vertices < 3 || !rhs_host ||
        !x_host || !ticket) {
        fmmbem_set_error("bad request");
        return FMMBEM_EINVAL;
    }
    if (opts && opts->nrhs != 1) {
        fmmbem_set_error("served requests carry one right-hand side (opts.nrhs = 1)");
        return FMMBEM_EINVAL;
    }
    Request* r = new Request();
    r->vertices.assign(mesh->vertices, mesh->vertices + 3 * mesh->n_vertices);
    r->triangles.assign(mesh->triangles, mesh->triangles + 3 * mesh->n_panels);
    const int64_t n = mesh->n_panels * (kernel == FMMBEM_STOKES ? 3 : 1);
    r->rhs.assign(rhs_host, rhs_host + n);
    r->kernel = kernel;
    r->gauss_k = gauss_k;
    r->ncrit = ncrit;
    r->theta = theta;
    fmmbem_default_opts(&r->opts);
    if (opts) r->opts = *opts;
    r->tol = tol;
    r->relax = relax;
    r->p_initial = p_initial;
    r->p_min = p_min;
    r->x_host = x_host;
    r->bytes = fmmbem_estimate_bytes(mesh->n_panels, kernel, gauss_k, ncrit, &r->opts);
    r->opts.stream = nullptr;  // each worker has its own
    r->key = request_key(*r);
    r->t_submit = clk::now();
    {
        std::lock_guard<std::mutex> lock(s->mu);
        if (s->stop) {
            delete r;
            fmmbem_set_error("server is shutting down");
            return FMMBEM_ESTATE;
        }
        r->ticket = s->next_ticket++;
        r->res.ticket = r->ticket;
        s->all[r->ticket] = r;
        s->queue.push_back(r);
        *ticket = r->ticket;
    }
    s->cv_work.notify_all();
    return 0;
}

int fmmbem_server_wait(fmmbem_server* s, int64_t ticket, fmmbem_result* out) {
    if (!s || !out) { fmmbem_set_error("NULL argument"); return FMMBEM_EINVAL; }
    std::unique_lock<std::mutex> lock(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) { fmmbem_set_error("unknown ticket %lld", (long long)ticket); return FMMBEM_EINVAL; }
    Request* r = it->second;
    s->cv_done.wait(lock, [&] { return r->done; });
    *out = r->res;
    s->all.erase(it);
    delete r;
    return 0;
}

int fmmbem_server_destroy(fmmbem_server* s) {
    if (!s) return 0;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    for (auto& w : s->workers) w.join();
    for (auto& e : s->all) delete e.second;
    destroy_entries(s->idle);  // before the streams the handles were created on
    for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
    delete s;
    return 0;
}

}  // extern "C"
