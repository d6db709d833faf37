// Serving loop: continuous batching of CoFEM fits, in two modes.
//
// Independent (cofem_server_create): a server owns `max_slots` worker
// threads, each with its own CUDA stream.  Requests enter a FIFO queue; a
// worker takes the request at the head as soon as it is idle and the
// request's device-memory estimate fits in what is left of the HBM budget,
// then runs the whole fit (create -> one graph launch -> results -> destroy)
// on its stream.  Fits of different workers overlap on the GPU; a request
// that arrives while others run is admitted as soon as a slot and memory free
// up.  Handle memory is stream-ordered, so finishing one request never
// synchronises the device under the others.
//
// Packed (cofem_server_create_packed): the CG steps of all admitted fits run
// in shared launches.  Preparation threads create each request's handle and
// run its prologue (dictionary images, b = beta Phi^T y, the first E-step's
// initialisation) on the handle's own stream; an engine thread keeps the
// prepared fits in one step: the packed GEMM applies the operator's first
// product to every fit (each fit's units cut into fixed segments, the
// segments of all fits spread over the CTAs), one kernel sums and splits T of
// every fit, the packed GEMM applies the second product, and one launch each
// of the CG update, the direction, the M-step (fits whose CG loop ended) and
// the next E-step's initialisation follow.  The step is a CUDA graph whose
// WHILE node repeats it on the device until a fit finishes, the host has new
// fits to admit (a mapped host flag), or a step budget is spent; every fit
// keeps its alpha, mu and CG state on the device throughout.  A fit's
// segments do not depend on the others, so its results are the same bits
// alone and in any mix.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <queue>
#include <string>
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

namespace {

// A prepared fit of the packed engine.
struct PFit {
    Job* job = nullptr;
    cofem_ctx* h = nullptr;
    cudaStream_t st = nullptr;   // the handle's stream (high priority: preparation is not starved by the step)
    PackedFit pf;
    VSlot vs{};
};

// Device tables of the packed step, sized for a capacity: the step's CUDA
// graph is built for the capacities and reads the counts, so admitting or
// retiring a fit only rewrites the tables (the graph is rebuilt only when a
// capacity grows).
struct StepTables {
    int cap_fits = 0, cap_blk[3] = {}, cap_seg[2][2] = {}, cap_sl[2][2] = {};
    TcSlot* sl[2][2] = {};   // [precision group][product]
    TcSeg* sg[2][2] = {};
    int* cta[2][2] = {};     // num_sms + 1 entries each
    VSlot* vs = nullptr;
    int4* map[3] = {};       // vector blocks, T blocks, M-step blocks
    int* counts = nullptr;   // blocks of each map, then fits
    int* status = nullptr;
    unsigned* steps = nullptr;   // steps of the current launch
    unsigned* flags = nullptr;   // COFEM_FLAG_DEVICE_TIMEOUT of the packed GEMMs
};

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
    // packed mode
    bool packed = false;
    int max_fits = 0;          // fits in a step (preparing, ready and active together)
    int num_sms = 0;
    int in_flight = 0;         // preparing + ready + active
    std::deque<PFit*> ready;   // prepared, waiting to join the step
    std::thread engine;
    std::condition_variable cv_engine;
    volatile int* pending_h = nullptr;   // mapped host flag: new fits are ready
    int* pending_d = nullptr;
    bool host_loop = false;    // COFEM_SERVE_HOST_LOOP: one step per host launch, no graph
    cofem_server_stats stats{};
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

namespace {

// ---------------------------------------------------------------------------
// Packed mode
// ---------------------------------------------------------------------------
bool packed_eligible(const cofem_request& r, const char** why) {
    if (r.kind != COFEM_OP_DENSE) return *why = "packed serving takes dense dictionaries", false;
    if (r.precision != COFEM_BF16 && r.precision != COFEM_F32_TF32X3)
        return *why = "packed serving takes COFEM_BF16 or COFEM_F32_TF32X3 dictionaries", false;
    if (r.rr_period != 0) return *why = "packed serving runs without residual replacement", false;
    const int Q = r.K + 1;
    const int QS = r.precision == COFEM_BF16 ? (3 * Q + 15) / 16 * 16 : 2 * ((Q + 15) / 16 * 16);
    if (QS > 128) return *why = "packed serving needs the split block in 128 rows (BF16: K <= 41)", false;
    return true;
}

long long packed_estimate(const cofem_request& r) {
    const long long Np = round_up_ll(r.N, 128), Dp = round_up_ll(r.D, 128), Q = r.K + 1;
    const long long segs = (round_up_ll(Np, 512) / 512) * ((Dp / 64 + PK_SEGK - 1) / PK_SEGK) +
                           (round_up_ll(Dp, 512) / 512) * ((Np / 64 + PK_SEGK - 1) / PK_SEGK);
    return cofem_estimate_bytes(r.kind, r.N, r.D, r.L, r.precision, r.K) + segs * Q * 512 * 4;
}

void finish_job(cofem_server* s, Job* job, cofem_status stat, unsigned flags, const char* msg) {
    job->t_end = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        job->result.status = stat;
        job->result.flags = flags;
        if (stat != COFEM_OK && msg) snprintf(job->result.message, sizeof(job->result.message), "%s", msg);
        job->result.queue_ms = std::chrono::duration<double, std::milli>(job->t_start - job->t_submit).count();
        job->result.run_ms = std::chrono::duration<double, std::milli>(job->t_end - job->t_start).count();
        job->done = true;
        s->in_use -= job->estimate;
        --s->running;
        --s->in_flight;
    }
    s->cv_done.notify_all();
    s->cv_work.notify_all();
}

// Preparation thread: create the handle, run the prologue, hand it to the engine.
void prep_loop(cofem_server* s) {
    cudaSetDevice(s->device);
    for (;;) {
        Job* job = nullptr;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_work.wait(lk, [&] {
                return s->stop || (!s->queue.empty() && s->in_use + s->queue.front()->estimate <= s->budget &&
                                   s->in_flight < s->max_fits);
            });
            if (s->queue.empty() || s->in_use + s->queue.front()->estimate > s->budget ||
                s->in_flight >= s->max_fits) {
                if (s->stop) break;
                continue;
            }
            job = s->queue.front();
            s->queue.pop_front();
            s->in_use += job->estimate;
            ++s->running;
            ++s->in_flight;
        }
        job->t_start = Clock::now();
        const cofem_request& r = job->req;
        cofem_opts o;
        cofem_default_opts(&o);
        o.precision = r.precision;
        o.precond = r.precond;
        o.conv = r.conv;
        o.alpha_max = r.alpha_max > 0.0 ? r.alpha_max : 1e12;
        o.seed = r.seed;
        o.use_graph = 0;
        o.prior = r.prior;
        PFit* f = new PFit();
        f->job = job;
        // the preparation's kernels run while the step loop keeps every SM
        // busy: a stream of the highest priority gets them scheduled first
        int lo = 0, hi = 0;
        cudaDeviceGetStreamPriorityRange(&lo, &hi);
        cofem_status stat = COFEM_OK;
        if (cudaStreamCreateWithPriority(&f->st, cudaStreamNonBlocking, hi) != cudaSuccess) {
            (void)cudaGetLastError();
            f->st = nullptr;
            stat = cofem_set_error(COFEM_ERR_CUDA, "cudaStreamCreateWithPriority");
        }
        o.stream = f->st;
        if (stat == COFEM_OK) stat = cofem_create(&f->h, r.N, r.D, r.kind, r.phi, r.L, &o);
        if (stat == COFEM_OK) stat = packed_prepare(f->h, r);
        if (stat != COFEM_OK) {
            const std::string msg = cofem_last_error();
            cofem_destroy(f->h);
            if (f->st) cudaStreamDestroy(f->st);
            delete f;
            finish_job(s, job, stat, 0u, msg.c_str());
            continue;
        }
        tc_pack_describe(f->h, &f->pf);
        tc_pack_vslot(f->h, &f->vs);
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->ready.push_back(f);
            *s->pending_h = 1;
        }
        s->cv_engine.notify_all();
    }
}

// Segments to CTAs, longest first to the least loaded CTA (the LPT rule:
// every CTA within one segment's cost of the others); `seg` is reordered so
// that CTA c's segments are seg[r[c] .. r[c + 1]).
std::vector<int> assign_ctas(std::vector<TcSeg>& seg, const std::vector<double>& cost, int nCTA) {
    std::vector<int> order(seg.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    using Load = std::pair<double, int>;   // (bytes so far, CTA)
    std::priority_queue<Load, std::vector<Load>, std::greater<Load>> heap;
    for (int c = 0; c < nCTA; ++c) heap.push({0.0, c});
    std::vector<std::vector<int>> mine(nCTA);
    for (int i : order) {
        Load l = heap.top();
        heap.pop();
        mine[l.second].push_back(i);
        l.first += cost[i];
        heap.push(l);
    }
    std::vector<TcSeg> out;
    out.reserve(seg.size());
    std::vector<int> r(nCTA + 1, 0);
    for (int c = 0; c < nCTA; ++c) {
        std::sort(mine[c].begin(), mine[c].end());   // a fit's segments in their order
        for (int i : mine[c]) out.push_back(seg[i]);
        r[c + 1] = (int)out.size();
    }
    seg.swap(out);
    return r;
}

struct StepGraph {
    cudaGraph_t g = nullptr;
    cudaGraphExec_t x = nullptr;
    void reset() {
        if (x) cudaGraphExecDestroy(x);
        if (g) cudaGraphDestroy(g);
        x = nullptr;
        g = nullptr;
    }
};

constexpr int PK_QSMAX = 128;   // the packed GEMM's split tile ring fits every admitted fit

template <typename T>
cudaError_t realloc_dev(T** p, size_t n) {
    if (*p) cudaFree(*p);
    *p = nullptr;
    return cudaMalloc((void**)p, std::max<size_t>(n, 1) * sizeof(T));
}

void free_tables(StepTables& tb) {
    for (int gi = 0; gi < 2; ++gi)
        for (int pr = 0; pr < 2; ++pr) {
            if (tb.sl[gi][pr]) cudaFree(tb.sl[gi][pr]);
            if (tb.sg[gi][pr]) cudaFree(tb.sg[gi][pr]);
            if (tb.cta[gi][pr]) cudaFree(tb.cta[gi][pr]);
        }
    if (tb.vs) cudaFree(tb.vs);
    for (auto* m : tb.map)
        if (m) cudaFree(m);
    for (void* p : {(void*)tb.counts, (void*)tb.status, (void*)tb.steps, (void*)tb.flags})
        if (p) cudaFree(p);
    tb = StepTables{};
}

// Host copy of a step's tables.
struct StepHost {
    std::vector<TcSlot> sl[2][2];
    std::vector<TcSeg> seg[2][2];
    std::vector<int> cta[2][2];
    std::vector<VSlot> vs;
    std::vector<int4> map[3];
    int mask = 0;   // 1: BF16 fits, 2: 3xTF32 fits
};

void compose(const std::vector<PFit*>& fits, int num_sms, StepHost& h) {
    h = StepHost{};
    std::vector<double> cost[2][2];
    for (size_t i = 0; i < fits.size(); ++i) {
        const PackedFit& pf = fits[i]->pf;
        const int gi = pf.tf ? 1 : 0;
        h.mask |= 1 << gi;
        for (int pr = 0; pr < 2; ++pr) {
            const int idx = (int)h.sl[gi][pr].size();
            h.sl[gi][pr].push_back(pr == 0 ? pf.g1 : pf.g2);
            const std::vector<TcSeg>& src = pr == 0 ? pf.s1 : pf.s2;
            const std::vector<double>& cs = pr == 0 ? pf.c1 : pf.c2;
            for (size_t k = 0; k < src.size(); ++k) {
                TcSeg x = src[k];
                x.slot = idx;
                h.seg[gi][pr].push_back(x);
                cost[gi][pr].push_back(cs[k]);
            }
        }
        const VSlot& v = fits[i]->vs;
        h.vs.push_back(v);
        const int ii = (int)i;
        for (int q = 0; q < v.Q; ++q)
            for (int ch = 0; ch < v.nch; ++ch) h.map[0].push_back(make_int4(ii, q, ch, v.nch * v.Q));
        const int nblk = (int)((v.Np + 1023) / 1024);
        for (int q = 0; q < v.Q; ++q)
            for (int ib = 0; ib < nblk; ++ib) h.map[1].push_back(make_int4(ii, q, ib, 0));
        const int mb = (int)((v.Dp + COFEM_VEC_THREADS - 1) / COFEM_VEC_THREADS);
        for (int jb = 0; jb < mb; ++jb) h.map[2].push_back(make_int4(ii, jb, mb, 0));
    }
    for (int gi = 0; gi < 2; ++gi)
        for (int pr = 0; pr < 2; ++pr) h.cta[gi][pr] = assign_ctas(h.seg[gi][pr], cost[gi][pr], num_sms);
}

// Grow the device tables to hold `h` (false: the graphs must be rebuilt).
cudaError_t ensure_capacity(StepTables& tb, const StepHost& h, int num_sms, bool* kept) {
    *kept = true;
    cudaError_t e;
    const int nf = (int)h.vs.size();
    if (nf > tb.cap_fits || !tb.vs) {
        const int cap = std::max(nf, std::max(16, 2 * tb.cap_fits));
        if ((e = realloc_dev(&tb.vs, cap)) || (e = realloc_dev(&tb.status, cap))) return e;
        tb.cap_fits = cap;
        *kept = false;
    }
    for (int k = 0; k < 3; ++k)
        if ((int)h.map[k].size() > tb.cap_blk[k] || !tb.map[k]) {
            const int cap = std::max((int)h.map[k].size(), std::max(1024, 2 * tb.cap_blk[k]));
            if ((e = realloc_dev(&tb.map[k], cap))) return e;
            tb.cap_blk[k] = cap;
            *kept = false;
        }
    for (int gi = 0; gi < 2; ++gi)
        for (int pr = 0; pr < 2; ++pr) {
            if ((int)h.seg[gi][pr].size() > tb.cap_seg[gi][pr] || !tb.sg[gi][pr]) {
                const int cap = std::max((int)h.seg[gi][pr].size(), std::max(1024, 2 * tb.cap_seg[gi][pr]));
                if ((e = realloc_dev(&tb.sg[gi][pr], cap))) return e;
                tb.cap_seg[gi][pr] = cap;
                *kept = false;
            }
            if (!tb.sl[gi][pr] || (int)h.sl[gi][pr].size() > tb.cap_sl[gi][pr]) {
                const int cap = std::max(tb.cap_fits, nf);
                if ((e = realloc_dev(&tb.sl[gi][pr], cap))) return e;
                tb.cap_sl[gi][pr] = cap;
                *kept = false;
            }
            if (!tb.cta[gi][pr]) {
                if ((e = realloc_dev(&tb.cta[gi][pr], num_sms + 1))) return e;
                *kept = false;
            }
        }
    if (!tb.counts) {
        if ((e = realloc_dev(&tb.counts, 4)) || (e = realloc_dev(&tb.steps, 1)) || (e = realloc_dev(&tb.flags, 1)))
            return e;
        *kept = false;
    }
    return cudaSuccess;
}

template <typename T>
cudaError_t put(T* dst, const std::vector<T>& v, cudaStream_t st) {
    if (v.empty()) return cudaSuccess;
    return cudaMemcpyAsync(dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st);
}

cudaError_t upload(StepTables& tb, const StepHost& h, cudaStream_t st) {
    cudaError_t e;
    for (int gi = 0; gi < 2; ++gi)
        for (int pr = 0; pr < 2; ++pr) {
            if ((e = put(tb.sl[gi][pr], h.sl[gi][pr], st))) return e;
            if ((e = put(tb.sg[gi][pr], h.seg[gi][pr], st))) return e;
            if ((e = put(tb.cta[gi][pr], h.cta[gi][pr], st))) return e;
        }
    if ((e = put(tb.vs, h.vs, st))) return e;
    for (int k = 0; k < 3; ++k)
        if ((e = put(tb.map[k], h.map[k], st))) return e;
    const std::vector<int> counts = {(int)h.map[0].size(), (int)h.map[1].size(), (int)h.map[2].size(),
                                     (int)h.vs.size()};
    if ((e = put(tb.counts, counts, st))) return e;
    if ((e = cudaMemsetAsync(tb.status, 0, h.vs.size() * sizeof(int), st))) return e;
    if ((e = cudaMemsetAsync(tb.flags, 0, sizeof(unsigned), st))) return e;
    return cudaMemsetAsync(tb.steps, 0, sizeof(unsigned), st);
}

// One packed step's launches into `body` (a graph's loop body, or a stream
// when the host drives the loop); h is the loop's condition (0: none).
void record_step(cofem_server* s, const StepTables& tb, int mask, Sink& body, cudaGraphConditionalHandle h) {
    for (int pr = 0; pr < 2; ++pr) {
        for (int gi = 0; gi < 2; ++gi) {
            if (!(mask & (1 << gi))) continue;
            TcBatch b{};
            b.slots = tb.sl[gi][pr];
            b.segs = tb.sg[gi][pr];
            b.cta_seg = tb.cta[gi][pr];
            b.G = 4;
            b.acc_stride = 128;
            b.QSmax = PK_QSMAX;
            b.flags = tb.flags;   // a timeout fails every fit of the step
            launch_gemm_packed(body, gi == 1, b, s->num_sms, tc_packed_smem(gi == 1, PK_QSMAX));
        }
        if (pr == 0) launch_reduce_T_packed(body, tb.vs, tb.map[1], tb.counts + 1, tb.cap_blk[1]);
    }
    launch_update_packed(body, tb.vs, tb.map[0], tb.counts + 0, tb.cap_blk[0]);
    launch_direction_packed(body, tb.vs, tb.map[0], tb.counts + 0, tb.cap_blk[0]);
    launch_mstep_packed(body, tb.vs, tb.map[2], tb.counts + 2, tb.cap_blk[2]);
    launch_init_packed(body, tb.vs, tb.map[0], tb.counts + 0, tb.cap_blk[0]);
    // a launch runs at most 4096 steps before the host looks again
    launch_packed_status(body, tb.vs, tb.counts + 3, tb.status, s->pending_d, tb.steps, 4096u, h);
}

// The step graph for the fits of the groups in `mask`, at the tables' capacities.
cudaError_t build_graph(cofem_server* s, const StepTables& tb, int mask, StepGraph& sg, cudaStream_t st, bool pdl) {
    sg.reset();
    cudaError_t e = cudaGraphCreate(&sg.g, 0);
    if (e) return e;
    Sink root;
    root.stream = st;
    root.graph = sg.g;
    root.pdl = pdl;
    const cudaGraphConditionalHandle h = root.make_handle(1u, true);
    Sink body = root.conditional(h, cudaGraphCondTypeWhile);
    record_step(s, tb, mask, body, h);
    e = root.err ? root.err : body.err;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&sg.x, sg.g, 0);
    if (e != cudaSuccess) sg.reset();
    return e;
}

void retire(cofem_server* s, std::vector<PFit*>& done) {
    for (PFit* f : done) {
        unsigned flags = 0;
        const cofem_status stat = packed_finish(f->h, f->job->req, &flags);
        const std::string msg = stat != COFEM_OK ? cofem_last_error() : "";
        cofem_destroy(f->h);
        if (f->st) cudaStreamDestroy(f->st);
        finish_job(s, f->job, stat, flags, msg.c_str());
        delete f;
    }
    done.clear();
}

void engine_loop(cofem_server* s) {
    cudaSetDevice(s->device);
    cudaStream_t st = nullptr;
    int lo = 0, hi = 0;
    cudaDeviceGetStreamPriorityRange(&lo, &hi);
    cudaStreamCreateWithPriority(&st, cudaStreamNonBlocking, lo);   // the step loop yields to preparation
    StepTables tb;
    StepGraph graphs[4];
    StepHost host;
    std::vector<PFit*> active, done;
    std::vector<int> status;
    bool pdl = true;
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_engine.wait(lk, [&] {
                return !s->ready.empty() || !active.empty() || !done.empty() || (s->stop && s->in_flight == 0);
            });
            if (active.empty() && s->ready.empty() && done.empty() && s->stop && s->in_flight == 0) break;
            while (!s->ready.empty()) {
                active.push_back(s->ready.front());
                s->ready.pop_front();
            }
            *s->pending_h = 0;
        }
        cudaError_t e = cudaSuccess;
        const bool run = !active.empty();
        if (run) {
            compose(active, s->num_sms, host);
            bool kept = true;
            e = ensure_capacity(tb, host, s->num_sms, &kept);
            if (!kept)
                for (auto& g : graphs) g.reset();
            if (e == cudaSuccess) e = upload(tb, host, st);
            if (e == cudaSuccess && s->host_loop) {   // one step from the host (profilers see each launch)
                Sink direct;
                direct.stream = st;
                direct.pdl = pdl;
                record_step(s, tb, host.mask, direct, 0);
                e = direct.err;
            } else if (e == cudaSuccess && !graphs[host.mask].x) {
                e = build_graph(s, tb, host.mask, graphs[host.mask], st, pdl);
                if (e != cudaSuccess && pdl) {   // programmatic edges refused: plain ones
                    (void)cudaGetLastError();
                    pdl = false;
                    e = build_graph(s, tb, host.mask, graphs[host.mask], st, pdl);
                }
                if (e == cudaSuccess) {
                    std::lock_guard<std::mutex> lk(s->mu);
                    ++s->stats.graphs_built;
                }
            }
            if (e == cudaSuccess && !s->host_loop) e = cudaGraphLaunch(graphs[host.mask].x, st);
        }
        retire(s, done);   // the fits that finished in the previous launch, while this one runs
        if (!run) continue;
        status.assign(active.size(), PH_NONE);
        unsigned dflags = 0, steps = 0;
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(status.data(), tb.status, active.size() * sizeof(int), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&dflags, tb.flags, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&steps, tb.steps, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess || (dflags & COFEM_FLAG_DEVICE_TIMEOUT)) {   // every fit of the step fails
            const char* msg = e != cudaSuccess ? cudaGetErrorString(e)
                                               : "a bounded on-device wait timed out (packed tensor-core pipeline)";
            (void)cudaGetLastError();
            for (PFit* f : active) {
                cofem_destroy(f->h);
                if (f->st) cudaStreamDestroy(f->st);
                finish_job(s, f->job, COFEM_ERR_CUDA, dflags, msg);
                delete f;
            }
            active.clear();
            for (auto& g : graphs) g.reset();
            continue;
        }
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->stats.launches += 1;
            s->stats.steps += steps;
            s->stats.fit_steps += (long long)steps * (long long)active.size();
        }
        std::vector<PFit*> keep;
        for (size_t i = 0; i < active.size(); ++i) (status[i] == PH_DONE ? done : keep).push_back(active[i]);
        active.swap(keep);
    }
    for (auto& g : graphs) g.reset();
    free_tables(tb);
    cudaStreamDestroy(st);
}

}  // namespace

extern "C" {

cofem_status cofem_server_create_packed(cofem_server** out, long long hbm_budget_bytes, int max_fits,
                                        int prep_threads, int flags) {
    if (!out || hbm_budget_bytes <= 0 || max_fits < 1 || max_fits > 1024 || prep_threads < 1 || prep_threads > 64 ||
        (flags & ~COFEM_SERVE_HOST_LOOP))
        return cofem_set_error(COFEM_ERR_INVALID_ARG,
                               "need out, hbm_budget_bytes > 0, 1 <= max_fits <= 1024, 1 <= prep_threads <= 64 "
                               "and flags in COFEM_SERVE_HOST_LOOP");
    cofem_server* s = new cofem_server();
    cudaError_t e = cudaGetDevice(&s->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, s->device);
    int* hp = nullptr;
    if (e == cudaSuccess) e = cudaHostAlloc((void**)&hp, sizeof(int), cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer((void**)&s->pending_d, hp, 0);
    if (e != cudaSuccess) {
        if (hp) cudaFreeHost(hp);
        delete s;
        return cofem_set_error(COFEM_ERR_CUDA, cudaGetErrorString(e));
    }
    *hp = 0;
    s->pending_h = hp;
    s->packed = true;
    s->host_loop = (flags & COFEM_SERVE_HOST_LOOP) != 0;
    s->budget = hbm_budget_bytes;
    s->max_fits = max_fits;
    s->max_slots = prep_threads;
    for (int i = 0; i < prep_threads; ++i) s->workers.emplace_back(prep_loop, s);
    s->engine = std::thread(engine_loop, s);
    *out = s;
    return COFEM_OK;
}

cofem_status cofem_server_get_stats(cofem_server* s, cofem_server_stats* out) {
    if (!s || !out) return cofem_set_error(COFEM_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->stats;
    return COFEM_OK;
}

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
    if (s->packed) {
        const char* why = nullptr;
        if (!packed_eligible(*r, &why)) return cofem_set_error(COFEM_ERR_UNSUPPORTED, why);
    }
    Job* job = new Job();
    job->req = *r;
    job->estimate = s->packed ? packed_estimate(*r)
                              : cofem_estimate_bytes(r->kind, r->N, r->D, r->L, r->precision, r->K);
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
    s->cv_engine.notify_all();
    for (auto& t : s->workers) t.join();
    if (s->engine.joinable()) s->engine.join();
    for (auto& kv : s->jobs) delete kv.second;
    if (s->pending_h) cudaFreeHost((void*)s->pending_h);
    delete s;
    return COFEM_OK;
}

}  // extern "C"
