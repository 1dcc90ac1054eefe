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
#include <math.h>
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
    clk::time_point t_submit;
    fmmbem_result res{};
    bool done = false;
};

}  // namespace

struct fmmbem_server {
    int device = 0;
    int64_t budget = 0, in_use = 0;
    int n_workers = 0;
    bool stop = false;
    int64_t next_ticket = 1;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request*> queue;
    std::map<int64_t, Request*> all;
    std::vector<std::thread> workers;
};

namespace {

void worker_main(fmmbem_server* s) {
    cudaSetDevice(s->device);
    cudaStream_t st = nullptr;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    for (;;) {
        Request* r = nullptr;
        {
            std::unique_lock<std::mutex> lock(s->mu);
            for (;;) {
                if (s->stop && s->queue.empty()) break;
                // the first queued request whose estimate fits in the remaining budget
                for (auto it = s->queue.begin(); it != s->queue.end(); ++it) {
                    if (s->in_use + (*it)->bytes <= s->budget || s->in_use == 0) {
                        r = *it;
                        s->queue.erase(it);
                        break;
                    }
                }
                if (r) break;
                s->cv_work.wait(lock);
            }
            if (!r) break;
            s->in_use += r->bytes;
        }
        const auto t_adm = clk::now();
        r->res.queue_s = std::chrono::duration<double>(t_adm - r->t_submit).count();
        fmmbem_mesh mesh{(int64_t)(r->vertices.size() / 3), r->vertices.data(), (int64_t)(r->triangles.size() / 3),
                         r->triangles.data()};
        fmmbem_opts o = r->opts;
        o.stream = st;
        fmmbem_handle* h = nullptr;
        int rc = fmmbem_create(&mesh, r->kernel, r->gauss_k, r->ncrit, r->theta, &o, &h);
        const auto t_set = clk::now();
        r->res.setup_s = std::chrono::duration<double>(t_set - t_adm).count();
        if (rc == 0) {
            int iters = 0;
            double true_res = 0.0;
            rc = fmmbem_solve_host(h, r->rhs.data(), r->tol, r->relax, r->p_initial, r->p_min, r->x_host, &iters,
                                   nullptr, nullptr, &true_res);
            r->res.iters = iters;
            r->res.true_res = true_res;
            fmmbem_destroy(h);
        }
        const auto t_end = clk::now();
        r->res.solve_s = std::chrono::duration<double>(t_end - t_set).count();
        r->res.latency_s = std::chrono::duration<double>(t_end - r->t_submit).count();
        r->res.status = rc;
        r->res.device_bytes = r->bytes;
        {
            std::lock_guard<std::mutex> lock(s->mu);
            s->in_use -= r->bytes;
            r->done = true;
            r->vertices.clear();
            r->triangles.clear();
            r->rhs.clear();
        }
        s->cv_done.notify_all();
        s->cv_work.notify_all();
    }
    cudaStreamDestroy(st);
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
    for (int i = 0; i < max_active; ++i) s->workers.emplace_back(worker_main, s);
    *out = s;
    return 0;
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
    delete s;
    return 0;
}

}  // extern "C"
