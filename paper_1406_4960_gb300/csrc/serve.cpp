// Continuous-batching solve server.
//
// Requests (a slab problem + nbands + tolerance + precision) are queued on
// submission.  A fixed set of worker threads ("slots") admits them as slots
// and device memory free up: a request is admitted when a slot is idle and
// its device footprint fits in the remaining budget (first fit over the
// queue, so one large request does not hold back smaller ones behind it).
// Each admitted request gets its own handle (basis, potential and Krylov
// state stay resident until it completes) and its own stream, so the work of
// concurrent requests overlaps on the device.  A request's result does not
// depend on what else runs: handles, workspaces and streams are private and
// every reduction in the library has a fixed order.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "mb_internal.h"

namespace mb {

namespace {

using clk = std::chrono::steady_clock;

struct Job {
    long long ticket = 0;
    mb_cell cell;
    std::vector<double> kpts, breaks;
    std::vector<mb_atom> atoms;
    int nk = 0, order = 0;
    double ecut = 0;
    mb_opts opts;
    int nbands = 0, prec = 0;
    double tol = 0;
    size_t footprint = 0;
    std::unique_ptr<mb_handle> host;   // host tables, built once at submission
    clk::time_point submitted, started, setup_done, finished;
    // results
    bool done = false;
    int rc = MB_OK;
    std::vector<double> evals;
    mb_solve_info info{};
};

// Device bytes a request will hold: handle tables (FP64 + FP32 copies),
// apply scratch, and the eigensolver workspace (vectors + small matrices).
size_t footprint_of(const mb_handle &h, int nbands, int prec) {
    const size_t NN = (size_t)h.n1 * h.n2;
    // V: the natural FP64 table, permuted + natural (FP64 + FP32), per column
    // (FP32); the transient buffers of its build
    size_t tables = (size_t)h.nq * NN * (8 + (8 + 4) * 2 + 4) + vloc_build_scratch_bytes(&h);
    tables += (size_t)h.nq * h.order * 12 + (size_t)h.nb * (2 * h.order - 1) * 12 * 2 + (size_t)h.nb * h.order * 12 +
              (size_t)h.nb * band_pad(h.order) * 12;   // the padded S band
    size_t vec_bytes = 0, pf = 0;
    int maxldg = 0;
    for (auto &k : h.kp) {
        tables += (size_t)k.ldg * (12 + 4) + (size_t)h.nterm * k.ldg * 24;
        pf += (size_t)k.ldg * h.nb * h.order * 12;
        vec_bytes += (size_t)h.nb * k.ldg * 16;
        maxldg = std::max(maxldg, k.ldg);
    }
    tables += pf;
    const int guard = std::max(2, (nbands + 7) / 8), M = nbands + guard;
    const int kd = kDefaultKrylovDepth, b = kDefaultBlock;
    const int nblk = (M + b - 1) / b, mA = M + kd, mB = b + kd, nc = std::max(1, nblk);
    const size_t nvecs = 3 * (size_t)std::max(mA, nblk * b) + 2 * (size_t)nblk * mB + 4 * nc + 3 * (size_t)mA +
                         (size_t)nblk * mB;
    size_t work = nvecs * vec_bytes + 2 * (size_t)std::max(M, nc) * vec_bytes / 2;
    // FP32 vectors of the mixed solver: X, SX, HX, the chain inputs, K, SK and
    // HK of every chain, two scratch sets
    if (prec != MB_FP64)
        work += (size_t)(3 * M + nc * (1 + 3 * kd) + 2 * std::max(M, nblk * b)) * vec_bytes / 2;
    const size_t LD = 128;
    work += (size_t)h.kp.size() * nc * LD * LD * 16 * (prec != MB_FP64 ? 6 : 3) + (size_t)h.kp.size() * LD * LD * 16 * 3;
    work += (size_t)std::max<size_t>(304, h.kp.size() * nc) * 112 * 112 * 16;
    // apply scratch: boundary rows + projector overlaps (generous bound)
    size_t scratch = (size_t)h.kp.size() *
                     ((size_t)M * 40 * 2 * (h.order - 1) * maxldg * 16 +
                      2 * (size_t)M * std::max((size_t)16 * std::max(1, h.nzf) * maxldg,
                                               (size_t)h.nb * std::max(1, h.nterm)) * 16);
    return tables + work + scratch + (64u << 20);   // + context-side slack per request
}

}  // namespace

}  // namespace mb

using namespace mb;

struct mb_server {
    int device = 0;
    size_t budget = 0, in_use = 0, peak_in_use = 0;
    int running = 0, peak_running = 0;
    long long next_ticket = 1;
    bool stopping = false;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<Job>> queue;
    std::map<long long, std::shared_ptr<Job>> jobs;
    std::vector<std::thread> workers;

    void worker_loop() {
        cudaSetDevice(device);
        for (;;) {
            std::shared_ptr<Job> job;
            {
                std::unique_lock<std::mutex> lock(mu);
                for (;;) {
                    if (stopping && queue.empty()) return;
                    auto it = queue.begin();
                    for (; it != queue.end(); ++it)
                        if ((*it)->footprint + in_use <= budget) break;
                    if (it != queue.end()) {
                        job = *it;
                        queue.erase(it);
                        in_use += job->footprint;
                        peak_in_use = std::max(peak_in_use, in_use);
                        ++running;
                        peak_running = std::max(peak_running, running);
                        break;
                    }
                    cv_work.wait(lock);
                }
            }
            job->started = clk::now();
            run(*job);
            job->finished = clk::now();
            {
                std::lock_guard<std::mutex> lock(mu);
                in_use -= job->footprint;
                --running;
                job->done = true;
            }
            cv_work.notify_all();
            cv_done.notify_all();
        }
    }

    // The device half of the request's set-up (its host tables were built at
    // submission), the solve, and the teardown; allocations and frees are
    // stream-ordered on the request's own streams, so none of this waits for
    // the other requests' work on the device.
    void run(Job &j) {
        mb_handle *h = j.host.release();
        j.rc = setup_device(h);
        j.setup_done = clk::now();
        if (j.rc == MB_OK) {
            j.evals.assign((size_t)j.nk * j.nbands, 0.0);
            j.rc = mb_eigsolve(h, j.nbands, j.tol, j.prec, j.evals.data(), nullptr, nullptr, &j.info, nullptr);
        }
        mb_destroy(h);
    }
};

extern "C" {

int mb_server_create(int device, int slots, double hbm_budget_bytes, mb_server **out) {
    if (!out || slots < 1 || slots > 64 || !(hbm_budget_bytes > 0)) return MB_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return MB_ECUDA;
    mb_server *s = new (std::nothrow) mb_server();
    if (!s) return MB_ENOMEM;
    s->device = device;
    s->budget = (size_t)hbm_budget_bytes;
    for (int i = 0; i < slots; ++i) s->workers.emplace_back([s] { s->worker_loop(); });
    *out = s;
    return MB_OK;
}

int mb_server_submit(mb_server *s, const mb_request *r, long long *ticket) {
    if (!s || !r || !ticket || !r->kpts || r->nk <= 0 || !r->breaks || r->nbreaks < 2) return MB_EINVAL;
    if (r->natoms < 0 || (r->natoms > 0 && !r->atoms) || r->nbands < 1 || !(r->tol > 0)) return MB_EINVAL;
    auto job = std::make_shared<Job>();
    job->cell = r->cell;
    job->kpts.assign(r->kpts, r->kpts + 2 * (size_t)r->nk);
    job->breaks.assign(r->breaks, r->breaks + r->nbreaks);
    if (r->natoms > 0) job->atoms.assign(r->atoms, r->atoms + r->natoms);
    job->nk = r->nk;
    job->order = r->order;
    job->ecut = r->ecut;
    job->opts = r->opts;
    job->opts.device = s->device;
    job->nbands = r->nbands;
    job->prec = r->prec;
    job->tol = r->tol;
    // the request's host tables (kept for its set-up) give its exact sizes
    {
        job->host.reset(new (std::nothrow) mb_handle());
        if (!job->host) return MB_ENOMEM;
        job->host->device = s->device;
        int rc = build_host_tables(job->host.get(), &job->cell, job->kpts.data(), job->nk, job->ecut,
                                   job->breaks.data(), (int)job->breaks.size(), job->order,
                                   job->atoms.empty() ? nullptr : job->atoms.data(), (int)job->atoms.size(),
                                   &job->opts);
        if (rc != MB_OK) return rc;
        job->footprint = footprint_of(*job->host, job->nbands, job->prec);
    }
    if (job->footprint > s->budget) return MB_ENOMEM;     // could never be admitted
    {
        std::lock_guard<std::mutex> lock(s->mu);
        if (s->stopping) return MB_EINVAL;
        job->ticket = s->next_ticket++;
        job->submitted = clk::now();
        s->jobs[job->ticket] = job;
        s->queue.push_back(job);
        *ticket = job->ticket;
    }
    s->cv_work.notify_all();
    return MB_OK;
}

int mb_server_wait(mb_server *s, long long ticket, double *evals, mb_solve_info *info, double *latency_s,
                   double *phases, double timeout_s) {
    if (!s) return MB_EINVAL;
    std::shared_ptr<Job> job;
    {
        std::unique_lock<std::mutex> lock(s->mu);
        auto it = s->jobs.find(ticket);
        if (it == s->jobs.end()) return MB_EINVAL;
        job = it->second;
        auto pred = [&] { return job->done; };
        if (timeout_s > 0) {
            if (!s->cv_done.wait_for(lock, std::chrono::duration<double>(timeout_s), pred)) return MB_ETIMEOUT;
        } else {
            s->cv_done.wait(lock, pred);
        }
        s->jobs.erase(it);
    }
    if (evals && !job->evals.empty()) std::memcpy(evals, job->evals.data(), sizeof(double) * job->evals.size());
    if (info) *info = job->info;
    if (latency_s) *latency_s = std::chrono::duration<double>(job->finished - job->submitted).count();
    if (phases) {
        phases[0] = std::chrono::duration<double>(job->started - job->submitted).count();
        phases[1] = std::chrono::duration<double>(job->setup_done - job->started).count();
        phases[2] = std::chrono::duration<double>(job->finished - job->setup_done).count();
    }
    return job->rc;
}

int mb_server_stats(mb_server *s, int *queued, int *running, int *peak_running, double *bytes_in_use,
                    double *peak_bytes) {
    if (!s) return MB_EINVAL;
    std::lock_guard<std::mutex> lock(s->mu);
    if (queued) *queued = (int)s->queue.size();
    if (running) *running = s->running;
    if (peak_running) *peak_running = s->peak_running;
    if (bytes_in_use) *bytes_in_use = (double)s->in_use;
    if (peak_bytes) *peak_bytes = (double)s->peak_in_use;
    return MB_OK;
}

void mb_server_destroy(mb_server *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stopping = true;
    }
    s->cv_work.notify_all();
    for (auto &t : s->workers) t.join();
    delete s;
}

}  // extern "C"
