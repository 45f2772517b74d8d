// Request server: MLMC level estimates (mlmc_level_estimate, §3.4) served to
// a stream of requests of different grid sizes and covariances, with
// continuous batching.
//
//   - `slots` worker threads, each with its own non-blocking CUDA stream,
//     take requests from one arrival-ordered queue as soon as a slot and
//     enough of the HBM budget are free, so the work of requests that
//     arrived at different times overlaps on the device.
//   - Admission by footprint: a request reserves an upper bound of the
//     device memory its level estimate allocates (fields, field intermediate,
//     solver hierarchy of the fine and coarse grids, per chunk) and is
//     admitted only while the reserved total stays within the budget.  The
//     queue is served first-fit in arrival order; once later requests have
//     overtaken a blocked head 8 times, only the head is admitted, so large
//     requests are not starved.
//   - Embedding cache: set-up (eigenvalues, masks, sqrt(Lambda~) tables) is
//     keyed by (covariance, n, padding, smoothing rule) and stays resident;
//     unused entries are evicted least-recently-used beyond max_embeddings.
//     Concurrent requests for a key that is being built wait for it.
//   - Results are bit-identical to a call of mlmc_level_estimate alone
//     (every reduction has a fixed order; no state is shared between
//     requests other than the immutable handles).
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "sce_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct EmbKey {
    int kind;
    double nu, lam, sigma2;
    int n, pad_mode, pad_J, pad_max_P, smoothing, finest;
    auto tie() const {
        return std::tie(kind, nu, lam, sigma2, n, pad_mode, pad_J, pad_max_P, smoothing, finest);
    }
    bool operator<(const EmbKey &o) const { return tie() < o.tie(); }
};

struct EmbEntry {
    ce_embedding_t e = nullptr;
    int refs = 0;
    unsigned long long last = 0;
    bool ready = false;
    int status = CE_OK;
};

struct Job {
    sce_request r{};
    sce_result res{};
    long long fp = 0;
    bool done = false;
    // a slice of a sliced request (parent != 0): slice index within it
    unsigned long long parent = 0;
    int slice = 0;
    // a sliced request: slices, the next one to queue, those done, samples
    // per slice, and each slice's sums and status (added in slice order)
    int nslices = 0, next_slice = 0, slices_done = 0, per_slice = 0;
    std::vector<sce_result> part;
};

constexpr int kMaxHeadSkips = 8;
// queued or running slices of one request: with every slot open to them, a
// large request's slices held all slots and small requests waited a slice
// (measured p99 of small requests 172 ms against 56 ms with two)
constexpr int kSlicesInFlight = 2;

bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

// Upper bound of the device memory one level estimate allocates at a time
// (it works in chunks of at most 2^27 fine vertices).
long long request_footprint(const sce_request &r, int precision) {
    const long long n = r.n, nc = n / 2;
    const long long Vf = (n + 1) * (n + 1), Vc = (nc + 1) * (nc + 1);
    const long long chunk =
        std::max(1LL, std::min<long long>({(long long)r.count, (1LL << 27) / Vf, 65535LL}));
    const long long es = precision == 64 ? 8 : 4;
    const long long P = 8 * n;   // embedding side bound (padding doubles J = n at most once)
    const long long inter = std::min(512LL << 20, chunk * (n + 1) * P * 2 * es);
    const bool coarse = r.level > 0;
    const long long fields = chunk * (Vf + (coarse ? Vc : 0)) * es;
    // hierarchy (cx, cy, b, z, zpre: 5 arrays x 4/3) + d, p, q in T, FP64 u, r,
    // conductances, partial sums
    auto solver = [&](long long V) { return chunk * V * (12 * es + 48); };
    return inter + fields + solver(Vf) + (coarse ? solver(Vc) : 0) + chunk * 64 + (1LL << 20);
}

}  // namespace

struct sce_server_s {
    sce_server_config cfg{};
    Clock::time_point t0;
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done, cv_emb;
    std::deque<unsigned long long> queue;
    std::deque<unsigned long long> sliced;   // sliced requests, oldest first
    std::unordered_map<unsigned long long, Job> jobs;
    unsigned long long next_id = 1;
    long long budget = 0, reserved = 0, peak_reserved = 0;
    long long submitted = 0, completed = 0, in_flight = 0, peak_in_flight = 0;
    int head_skips = 0;
    bool stop = false;
    std::map<EmbKey, EmbEntry> cache;
    unsigned long long use_clock = 0;
    long long hits = 0, misses = 0;
    std::vector<std::thread> workers;

    double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }

    // Queues the next slice of sliced request `pid` at the back (caller holds mu).
    void enqueue_slice(unsigned long long pid) {
        Job &P = jobs.at(pid);
        const int k = P.next_slice++;
        Job j;
        j.r = P.r;
        j.r.first_sample = P.r.first_sample + (uint64_t)k * P.per_slice;
        j.r.count = std::min(P.per_slice, P.r.count - k * P.per_slice);
        if (P.r.Y) j.r.Y = P.r.Y + (size_t)k * P.per_slice;
        j.fp = std::min(request_footprint(j.r, cfg.precision), budget);
        j.res.footprint = j.fp;
        j.res.t_submit = P.res.t_submit;
        j.parent = pid;
        j.slice = k;
        const unsigned long long id = next_id++;
        jobs.emplace(id, j);
        queue.push_back(id);
    }

    // A finished slice: keep its results, queue the next slice, and complete
    // the request once every slice is done (caller holds mu).  Returns true
    // when the request completed.
    bool slice_done(unsigned long long sid) {
        Job &sj = jobs.at(sid);
        const unsigned long long pid = sj.parent;
        Job &P = jobs.at(pid);
        P.part[sj.slice] = sj.res;
        P.res.footprint = std::max(P.res.footprint, sj.fp);
        jobs.erase(sid);
        ++P.slices_done;
        if (P.next_slice < P.nslices) enqueue_slice(pid);
        if (P.slices_done < P.nslices) return false;
        mlmc_level_sums tot{};
        int status = CE_OK, hit = 1;
        for (int k = 0; k < P.nslices; ++k) {   // fixed order: independent of timing
            const sce_result &r = P.part[k];
            tot.N += r.sums.N;
            tot.sumY += r.sums.sumY;
            tot.sumY2 += r.sums.sumY2;
            tot.sumQf += r.sums.sumQf;
            tot.sumQf2 += r.sums.sumQf2;
            tot.n_failed += r.sums.n_failed;
            tot.max_iters = std::max(tot.max_iters, r.sums.max_iters);
            tot.total_iters += r.sums.total_iters;
            if (status == CE_OK || status == CE_ERR_NOT_CONVERGED)
                if (r.status != CE_OK) status = r.status;
            hit &= r.cache_hit;
        }
        P.res.sums = tot;
        P.res.status = status;
        P.res.cache_hit = hit;
        P.res.t_admit = P.part[0].t_admit;
        P.res.t_setup_done = P.part[0].t_setup_done;
        P.res.t_done = now();
        P.done = true;
        P.part.clear();
        return true;
    }

    // Next admissible job (caller holds mu); 0 if none.  With nothing
    // admissible queued, another slice of the oldest sliced request with
    // slices left is started -- while at least one slot stays free for the
    // requests that arrive meanwhile -- so that an otherwise idle server gives
    // a large request more of the GPU.
    unsigned long long pick() {
        for (size_t i = 0; i < queue.size(); ++i) {
            const unsigned long long id = queue[i];
            if (jobs.at(id).fp > budget - reserved) continue;
            if (i > 0) {
                if (head_skips >= kMaxHeadSkips) return 0;
                ++head_skips;
            } else {
                head_skips = 0;
            }
            queue.erase(queue.begin() + (long)i);
            return id;
        }
        if (!queue.empty() || in_flight + 1 >= cfg.slots) return 0;
        while (!sliced.empty()) {
            const unsigned long long pid = sliced.front();
            auto it = jobs.find(pid);
            if (it == jobs.end() || it->second.next_slice >= it->second.nslices) {
                sliced.pop_front();
                continue;
            }
            enqueue_slice(pid);
            const unsigned long long id = queue.back();
            if (jobs.at(id).fp > budget - reserved) return 0;   // stays queued
            queue.pop_back();
            return id;
        }
        return 0;
    }

    int build_embedding(const EmbKey &k, cudaStream_t st, ce_embedding_t *out) {
        const ce_cov cov{k.kind, k.nu, k.lam, k.sigma2};
        const ce_pad pad{k.pad_mode, k.pad_J, k.pad_max_P};
        if (!k.smoothing) return ce_setup_embedding(&cov, k.n, &pad, nullptr, st, out, nullptr);
        const ce_smoothing sm{k.finest ? (long long)CE_KEEP_ALL : (long long)CE_KEEP_TAU_SQRT_S,
                              (long long)CE_KEEP_TAU_SQRT_S, 0.0};
        return ce_setup_embedding(&cov, k.n, &pad, &sm, st, out, nullptr);
    }

    // Evicts least-recently-used unused entries beyond max_embeddings (caller
    // holds mu); returns the handles to destroy after unlocking.
    std::vector<ce_embedding_t> evict() {
        std::vector<ce_embedding_t> victims;
        while ((int)cache.size() > cfg.max_embeddings) {
            auto best = cache.end();
            for (auto it = cache.begin(); it != cache.end(); ++it)
                if (it->second.ready && it->second.refs == 0 &&
                    (best == cache.end() || it->second.last < best->second.last))
                    best = it;
            if (best == cache.end()) break;
            victims.push_back(best->second.e);
            cache.erase(best);
        }
        return victims;
    }

    int acquire(const EmbKey &k, cudaStream_t st, ce_embedding_t *out, int *hit) {
        std::unique_lock<std::mutex> lk(mu);
        auto it = cache.find(k);
        if (it != cache.end()) {
            EmbEntry &en = it->second;
            ++en.refs;
            cv_emb.wait(lk, [&] { return en.ready; });
            if (en.status != CE_OK) {
                const int rc = en.status;
                if (--en.refs == 0) cache.erase(k);
                return rc;
            }
            en.last = ++use_clock;
            ++hits;
            *out = en.e;
            *hit = 1;
            return CE_OK;
        }
        EmbEntry &en = cache[k];
        en.refs = 1;
        ++misses;
        lk.unlock();
        ce_embedding_t e = nullptr;
        const int rc = build_embedding(k, st, &e);
        lk.lock();
        en.ready = true;
        en.status = rc;
        en.e = e;
        en.last = ++use_clock;
        cv_emb.notify_all();
        if (rc != CE_OK) {
            if (--en.refs == 0) cache.erase(k);
            return rc;
        }
        std::vector<ce_embedding_t> victims = evict();
        lk.unlock();
        for (ce_embedding_t v : victims) ce_destroy(v);
        *out = e;
        *hit = 0;
        return CE_OK;
    }

    void release(const EmbKey &k) {
        std::vector<ce_embedding_t> victims;
        {
            std::lock_guard<std::mutex> lk(mu);
            auto it = cache.find(k);
            if (it != cache.end()) --it->second.refs;
            victims = evict();
        }
        for (ce_embedding_t v : victims) ce_destroy(v);
    }

    void run(Job &j, cudaStream_t st) {
        const sce_request &r = j.r;
        const EmbKey key{r.cov.kind, r.cov.nu,   r.cov.lambda, r.cov.sigma2, r.n,
                         r.pad.mode, r.pad.J,    r.pad.max_P,  r.smoothing,  r.finest};
        ce_embedding_t e = nullptr;
        int hit = 0;
        int rc = acquire(key, st, &e, &hit);
        j.res.cache_hit = hit;
        j.res.t_setup_done = now();
        if (rc == CE_OK) {
            const darcy_problem p{r.n, r.f, cfg.rtol, cfg.maxit, cfg.precision};
            rc = mlmc_level_estimate(e, &p, r.seed, r.level, r.first_sample, r.count, r.qoi_index,
                                     &j.res.sums, r.Y, nullptr, nullptr, st);
            release(key);
        }
        j.res.status = rc;
    }

    void worker() {
        cudaSetDevice(device);
        cudaStream_t st = nullptr;
        const bool have_stream = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess;
        for (;;) {
            unsigned long long id = 0;
            Job *j = nullptr;
            {
                std::unique_lock<std::mutex> lk(mu);
                cv_work.wait(lk, [&] { return (id = pick()) != 0 || (stop && queue.empty()); });
                if (id == 0) break;
                j = &jobs.at(id);
                reserved += j->fp;
                peak_reserved = std::max(peak_reserved, reserved);
                ++in_flight;
                peak_in_flight = std::max(peak_in_flight, in_flight);
                j->res.t_admit = now();
            }
            if (have_stream) run(*j, st);
            else j->res.status = CE_ERR_CUDA;
            {
                std::lock_guard<std::mutex> lk(mu);
                j->res.t_done = now();
                reserved -= j->fp;
                --in_flight;
                if (j->parent) {
                    if (slice_done(id)) ++completed;
                } else {
                    j->done = true;
                    ++completed;
                }
            }
            cv_done.notify_all();
            cv_work.notify_all();
        }
        if (st) cudaStreamDestroy(st);
    }
};

extern "C" int sce_server_create(const sce_server_config *cfg, sce_server_t *out) {
    if (!cfg || !out || cfg->slots < 1 || cfg->slots > 64 || cfg->max_embeddings < 1 ||
        (cfg->precision != 32 && cfg->precision != 64) || !(cfg->rtol > 0))
        return CE_ERR_INVALID_ARG;
    *out = nullptr;
    sce_server_s *S = new (std::nothrow) sce_server_s;
    if (!S) return CE_ERR_OOM;
    S->cfg = *cfg;
    S->t0 = Clock::now();
    if (cudaGetDevice(&S->device) != cudaSuccess) {
        delete S;
        return CE_ERR_CUDA;
    }
    S->budget = cfg->hbm_budget;
    if (S->budget <= 0) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
            delete S;
            return CE_ERR_CUDA;
        }
        S->budget = (long long)(fr / 4 * 3);
    }
    for (int i = 0; i < cfg->slots; ++i) S->workers.emplace_back([S] { S->worker(); });
    *out = S;
    return CE_OK;
}

extern "C" int sce_server_submit(sce_server_t S, const sce_request *r, uint64_t *ticket) {
    if (!S || !r || !ticket) return CE_ERR_INVALID_ARG;
    if (!is_pow2(r->n) || r->n < 4 || r->n > 4096 || r->count < 0 || r->level > 30 ||
        r->qoi_index < 0 || r->qoi_index > 2 || (r->smoothing != 0 && r->smoothing != 1) ||
        (r->cov.kind != CE_COV_MATERN && r->cov.kind != CE_COV_SEP_EXP))
        return CE_ERR_INVALID_ARG;
    Job j;
    j.r = *r;
    const long long Vf = (long long)(r->n + 1) * (r->n + 1);
    const long long sv = S->cfg.slice_vertices == 0 ? (1LL << 24) : S->cfg.slice_vertices;
    const long long per = sv > 0 ? std::max(1LL, sv / Vf) : (long long)r->count;
    const bool sliced = sv > 0 && (long long)r->count > per;
    if (sliced) {
        j.per_slice = (int)per;
        j.nslices = (int)(((long long)r->count + per - 1) / per);
        j.part.assign(j.nslices, sce_result{});
    } else {
        j.fp = std::min(request_footprint(*r, S->cfg.precision), S->budget);
        j.res.footprint = j.fp;
    }
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->stop) return CE_ERR_INVALID_ARG;
        const unsigned long long id = S->next_id++;
        j.res.t_submit = S->now();
        S->jobs.emplace(id, j);
        if (sliced) {
            // each finished slice queues the next one behind the requests that
            // arrived meanwhile
            for (int k = 0; k < std::min(kSlicesInFlight, j.nslices); ++k) S->enqueue_slice(id);
            S->sliced.push_back(id);
        } else {
            S->queue.push_back(id);
        }
        ++S->submitted;
        *ticket = id;
    }
    S->cv_work.notify_all();
    return CE_OK;
}

extern "C" int sce_server_wait(sce_server_t S, uint64_t ticket, double timeout_s,
                               sce_result *out) {
    if (!S || !out) return CE_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->jobs.find(ticket);
    if (it == S->jobs.end()) return CE_ERR_INVALID_ARG;
    // element references survive rehashing by later submissions; iterators do not
    const Job *j = &it->second;
    auto ready = [&] { return j->done; };
    if (timeout_s < 0) {
        S->cv_done.wait(lk, ready);
    } else if (!S->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), ready)) {
        return CE_ERR_TIMEOUT;
    }
    *out = j->res;
    S->jobs.erase(ticket);
    return CE_OK;
}

extern "C" int sce_server_stats(sce_server_t S, sce_server_stats_t *out) {
    if (!S || !out) return CE_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    out->submitted = S->submitted;
    out->completed = S->completed;
    out->queued = (long long)S->queue.size();
    out->in_flight = S->in_flight;
    out->peak_in_flight = S->peak_in_flight;
    out->cache_hits = S->hits;
    out->cache_misses = S->misses;
    out->cached = (long long)S->cache.size();
    out->reserved = S->reserved;
    out->peak_reserved = S->peak_reserved;
    out->budget = S->budget;
    out->now = S->now();
    return CE_OK;
}

extern "C" void sce_server_destroy(sce_server_t S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    for (std::thread &t : S->workers) t.join();
    for (auto &kv : S->cache)
        if (kv.second.e) ce_destroy(kv.second.e);
    delete S;
}
