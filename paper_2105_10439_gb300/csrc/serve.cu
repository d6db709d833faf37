// Serving loop: continuous batching of independent CoFEM fits.
//
// A server owns `max_slots` worker threads, each with its own CUDA stream.
// Requests enter a FIFO queue; a worker takes the request at the head as soon
// as it is idle and the request's device-memory estimate fits in what is left
// of the HBM budget, then runs the whole fit (create -> one graph launch ->
// results -> destroy) on its stream.  Fits of different workers overlap on the
// GPU; a request that arrives while others run is admitted as soon as a slot
// and memory free up.  Handle memory is stream-ordered, so finishing one
// request never synchronises the device under the others.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "cofem_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct Job {
    cofem_request req;
    unsigned long long ticket = 0;
    long long estimate = 0;
    bool done = false;
    cofem_result result{};
    Clock::time_point t_submit, t_start, t_end;
};

long long round_up_ll(long long x, long long m) { return (x + m - 1) / m * m; }

}  // namespace

struct cofem_server {
    int device = 0;
    long long budget = 0, in_use = 0;
    int max_slots = 0;
    bool stop = false;
    unsigned long long next_ticket = 1;
    std::deque<Job*> queue;
    std::map<unsigned long long, Job*> jobs;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::vector<std::thread> workers;
    int running = 0;
};

extern "C" long long cofem_estimate_bytes(int kind, long long N, long long D, long long L, int precision, int K) {
    const long long Np = round_up_ll(N, 128), Dp = round_up_ll(D, 128), Q = K + 1;
    const long long QP = (Q + 7) / 8 * 8;
    long long b = 0;
    if (kind == COFEM_OP_DENSE) {
        // tensor-core images of the dictionary and of its transpose (rows rounded to 512)
        const long long img = round_up_ll(Np, 512) * Dp + round_up_ll(Dp, 512) * Np;
        if (precision == COFEM_BF16) {
            b += Np * Dp * 4 + Np * Dp * 2 + img * 2;          // FP32 staging, bf16 copy, images
        } else if (precision == COFEM_F32_TF32X3) {
            b += Np * Dp * 4 + img * 4;                        // FP32 copy, images
        } else {
            b += Np * Dp * 4 + 9 * Np * QP * 4 + 8 * Q * Dp * 4;   // FP32 copy, T and slices, U slices
        }
        if (precision != COFEM_F32)
            b += 2 * 200 * Q * 512 * 4 + 2 * 3 * Q * (Np + Dp) * 4;   // segment partials, split blocks
    } else {
        b += L * 4 + Q * Dp * 4;
    }
    b += 4 * Q * Dp * 4 + 8 * Dp * 4 + Np * 4 + (1 << 20);  // X R P U, vectors, y, small buffers
    return b;
}

namespace {

void worker_loop(cofem_server* s) {
    cudaSetDevice(s->device);
    cudaStream_t st = nullptr;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    for (;;) {
        Job* job = nullptr;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_work.wait(lk, [&] {
                return s->stop || (!s->queue.empty() && s->in_use + s->queue.front()->estimate <= s->budget);
            });
            if (s->queue.empty() || s->in_use + s->queue.front()->estimate > s->budget) {
                if (s->stop) break;
                continue;
            }
            job = s->queue.front();
            s->queue.pop_front();
            s->in_use += job->estimate;
            ++s->running;
        }
        job->t_start = Clock::now();
        const cofem_request& r = job->req;
        cofem_opts o;
        cofem_default_opts(&o);
        o.precision = r.precision;
        o.precond = r.precond;
        o.conv = r.conv;
        o.rr_period = r.rr_period;
        o.alpha_max = r.alpha_max > 0.0 ? r.alpha_max : 1e12;
        o.seed = r.seed;
        o.stream = st;
        o.use_graph = 1;
        // no SM cap by default: on the serving mix (D up to 16384) capping each
        // request at 2 SMs / slots halved throughput (the GEMMs are the bound)
        o.max_sms = r.max_sms > 0 ? r.max_sms : 0;
        o.prior = r.prior;
        cofem_ctx* h = nullptr;
        unsigned flags = 0;
        cofem_status stat = cofem_create(&h, r.N, r.D, r.kind, r.phi, r.L, &o);
        if (stat == COFEM_OK)
            stat = cofem_fit(h, r.y, r.beta, r.alpha0, r.K, r.T_em, r.cg_tol, r.cg_maxit, r.mu, r.s, r.alpha,
                             r.cg_iters, &flags);
        if (stat != COFEM_OK) snprintf(job->result.message, sizeof(job->result.message), "%s", cofem_last_error());
        cofem_destroy(h);
        job->t_end = Clock::now();
        {
            std::lock_guard<std::mutex> lk(s->mu);
            job->result.status = stat;
            job->result.flags = flags;
            job->result.queue_ms = std::chrono::duration<double, std::milli>(job->t_start - job->t_submit).count();
            job->result.run_ms = std::chrono::duration<double, std::milli>(job->t_end - job->t_start).count();
            job->done = true;
            s->in_use -= job->estimate;
            --s->running;
        }
        s->cv_done.notify_all();
        s->cv_work.notify_all();
    }
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
}

}  // namespace

extern "C" {

cofem_status cofem_server_create(cofem_server** out, long long hbm_budget_bytes, int max_slots) {
    if (!out || hbm_budget_bytes <= 0 || max_slots < 1 || max_slots > 256)
        return cofem_set_error(COFEM_ERR_INVALID_ARG, "need out, hbm_budget_bytes > 0 and 1 <= max_slots <= 256");
    cofem_server* s = new cofem_server();
    cudaError_t e = cudaGetDevice(&s->device);
    if (e != cudaSuccess) {
        delete s;
        return cofem_set_error(COFEM_ERR_CUDA, cudaGetErrorString(e));
    }
    s->budget = hbm_budget_bytes;
    s->max_slots = max_slots;
    for (int i = 0; i < max_slots; ++i) s->workers.emplace_back(worker_loop, s);
    *out = s;
    return COFEM_OK;
}

cofem_status cofem_submit(cofem_server* s, const cofem_request* r, unsigned long long* ticket) {
    if (!s || !r || !ticket) return cofem_set_error(COFEM_ERR_INVALID_ARG, "NULL argument");
    if (!r->phi || !r->y || !r->mu || !r->s || !r->alpha || r->N < 1 || r->D < 1 || r->K < 1 || r->T_em < 1)
        return cofem_set_error(COFEM_ERR_INVALID_ARG, "incomplete request");
    Job* job = new Job();
    job->req = *r;
    job->estimate = cofem_estimate_bytes(r->kind, r->N, r->D, r->L, r->precision, r->K);
    if (job->estimate > s->budget) {
        delete job;
        return cofem_set_error(COFEM_ERR_NOMEM, "request needs more device memory than the server's whole budget");
    }
    job->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) {
            delete job;
            return cofem_set_error(COFEM_ERR_INVALID_ARG, "server is shutting down");
        }
        job->ticket = s->next_ticket++;
        s->jobs[job->ticket] = job;
        s->queue.push_back(job);
        *ticket = job->ticket;
    }
    s->cv_work.notify_all();
    return COFEM_OK;
}

cofem_status cofem_poll(cofem_server* s, unsigned long long ticket, int* done) {
    if (!s || !done) return cofem_set_error(COFEM_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->jobs.find(ticket);
    if (it == s->jobs.end()) return cofem_set_error(COFEM_ERR_NOT_FOUND, "unknown ticket");
    *done = it->second->done ? 1 : 0;
    return COFEM_OK;
}

cofem_status cofem_wait(cofem_server* s, unsigned long long ticket, cofem_result* out) {
    if (!s || !out) return cofem_set_error(COFEM_ERR_INVALID_ARG, "NULL argument");
    Job* job = nullptr;
    {
        std::unique_lock<std::mutex> lk(s->mu);
        auto it = s->jobs.find(ticket);
        if (it == s->jobs.end()) return cofem_set_error(COFEM_ERR_NOT_FOUND, "unknown ticket");
        job = it->second;
        s->cv_done.wait(lk, [&] { return job->done; });
        s->jobs.erase(it);
    }
    *out = job->result;
    delete job;
    return COFEM_OK;
}

cofem_status cofem_server_destroy(cofem_server* s) {
    if (!s) return COFEM_OK;
    {
        std::unique_lock<std::mutex> lk(s->mu);
        s->cv_done.wait(lk, [&] { return s->queue.empty() && s->running == 0; });
        s->stop = true;
    }
    s->cv_work.notify_all();
    for (auto& t : s->workers) t.join();
    for (auto& kv : s->jobs) delete kv.second;
    delete s;
    return COFEM_OK;
}

}  // extern "C"
