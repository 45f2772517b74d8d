// One MLMC level of Algorithm 1 (Algorithm 2 with a smoothed handle):
// fields -> fine and coarse Darcy solves -> Y_l = Q_f - Q_c (Y_0 = Q_f) ->
// level sums (N, sum Y, sum Y^2, sum Q_f, sum Q_f^2) for Eq. (3.5).
//
// mlmc_estimate_levels runs several levels at once: one host worker thread
// per level in flight, each level on its own CUDA streams (the coarse solve
// of a level on a second stream, driven by a second host thread, once the
// fields of the chunk exist).  The solvers' convergence checks synchronise
// only their own stream, so the phases of one level that leave SMs idle
// (coarse-grid cycles, reductions, host checks) are filled by the others.
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <future>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "sce_internal.cuh"

namespace {

__global__ void level_diff_kernel(const double *__restrict__ qf, const double *__restrict__ qc,
                                  int count, int qi, double *__restrict__ Y) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= count) return;
    Y[s] = qf[3 * s + qi] - (qc ? qc[3 * s + qi] : 0.0);
}

// One block, fixed-order: per-thread strided sums, then a shared-memory tree.
__global__ void level_sums_kernel(const double *__restrict__ Y, const double *__restrict__ qf,
                                  int count, int qi, double *__restrict__ out4) {
    __shared__ double sh[4][256];
    double a = 0, b = 0, c = 0, d = 0;
    for (int s = threadIdx.x; s < count; s += blockDim.x) {
        const double y = Y[s], q = qf[3 * s + qi];
        a += y;
        b += y * y;
        c += q;
        d += q * q;
    }
    sh[0][threadIdx.x] = a;
    sh[1][threadIdx.x] = b;
    sh[2][threadIdx.x] = c;
    sh[3][threadIdx.x] = d;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int r = 0; r < 4; ++r) sh[r][threadIdx.x] += sh[r][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 4) out4[threadIdx.x] = sh[threadIdx.x][0];
}


struct LevelArgs {
    ce_embedding_t e;
    uint32_t level;
    uint64_t first_sample;
    int count;
    double *Y, *qoi_f, *qoi_c;
    mlmc_level_sums *out;
    const QmcArgs *qa = nullptr;   // lattice sampler (nullptr: Philox)
    const void *kf_pre = nullptr;  // fields computed beforehand (count of them), or nullptr
    const void *kc_pre = nullptr;
};

// One level on stream st; the coarse solves go to stream stc (a second host
// thread) when stc != st, otherwise they follow the fine solve on st.
static int level_run(const LevelArgs &a, const darcy_problem *p, uint64_t seed, int qoi_index,
                     cudaStream_t st, cudaStream_t stc) {
    ce_embedding_t e = a.e;
    const int count = a.count;
    *a.out = mlmc_level_sums{};
    if (count == 0) return CE_OK;
    const int n = e->n, nc = n / 2;
    const bool coarse = a.level > 0;
    // nested iteration: on levels with a coarse grid the coarse solve runs
    // first and its prolonged solution is the fine solve's first iterate
    // (SCE_NESTED=0: both start from the lifting, the coarse solve on a second
    // stream; SCE_NESTED_SMALL=0: only where the fine solve is the batched
    // solver, not the one-block solver of the small grids)
    const bool fine_batched = !(p->precision == 32 && n <= sce_small_max_n() && n <= 64);
    bool nested = coarse;
    if (!fine_batched)
        if (const char *ev = getenv("SCE_NESTED_SMALL")) nested = nested && atoi(ev) != 0;
    if (const char *ev = getenv("SCE_NESTED")) nested = nested && atoi(ev) != 0;
    const bool split = coarse && stc != st && !nested;
    const size_t es = p->precision == 64 ? sizeof(double) : sizeof(float);
    const long long Vf = (long long)(n + 1) * (n + 1), Vc = (long long)(nc + 1) * (nc + 1);
    // chunk: bound the number of fine vertices resident at once
    // (SCE_MLMC_CHUNK_VERTICES lowers the bound, to exercise the chunk loop)
    long long max_vertices = 1LL << 27;
    if (const char *ev = getenv("SCE_MLMC_CHUNK_VERTICES"))
        max_vertices = std::max(1LL, std::min(max_vertices, atoll(ev)));
    int chunk = (int)std::max<long long>(1, std::min<long long>(count, max_vertices / Vf));
    chunk = std::min(chunk, 65535);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CE_ERR_CUDA;

    void *kf = nullptr, *kc = nullptr;
    double *qf = nullptr, *qc = nullptr, *Yd = nullptr, *sums = nullptr;
    double *ucs = nullptr;   // nested iteration: the coarse solution
    // FP32 problems hand it over as float-float pairs (8 bytes per vertex, as a double)
    const bool ff_hand = p->precision == 32;
    cudaEvent_t ev_field = nullptr, ev_coarse = nullptr;
    std::vector<void *> owned;
    auto cleanup = [&]() {
        // coarse kernels of the split path may still be in flight on stc
        // after an error return: the stream-ordered frees on st must not
        // hand their buffers to the next allocation before they finish
        if (split) cudaStreamSynchronize(stc);
        for (void *q : owned) sce_free(q, st);
        if (ev_field) cudaEventDestroy(ev_field);
        if (ev_coarse) cudaEventDestroy(ev_coarse);
    };
    int rc = CE_OK;
    auto A = [&](void **ptr, size_t bytes) {
        int r = sce_alloc(ptr, bytes, st);
        if (r == CE_OK) owned.push_back(*ptr);
        return r;
    };
    const bool pre = a.kf_pre != nullptr;
    if (!pre && (rc = A(&kf, (size_t)chunk * Vf * es)) != CE_OK) { cleanup(); return rc; }
    if (!pre && coarse && (rc = A(&kc, (size_t)chunk * Vc * es)) != CE_OK) { cleanup(); return rc; }
    if (!a.qoi_f && (rc = A((void **)&qf, (size_t)chunk * 3 * sizeof(double))) != CE_OK) { cleanup(); return rc; }
    if (coarse && !a.qoi_c && (rc = A((void **)&qc, (size_t)chunk * 3 * sizeof(double))) != CE_OK) { cleanup(); return rc; }
    if (!a.Y && (rc = A((void **)&Yd, (size_t)chunk * sizeof(double))) != CE_OK) { cleanup(); return rc; }
    if ((rc = A((void **)&sums, 4 * sizeof(double))) != CE_OK) { cleanup(); return rc; }
    if (nested && (rc = A((void **)&ucs, (size_t)chunk * Vc * sizeof(double))) != CE_OK) {
        cleanup();
        return rc;
    }
    if (split && (cudaEventCreateWithFlags(&ev_field, cudaEventDisableTiming) != cudaSuccess ||
                  cudaEventCreateWithFlags(&ev_coarse, cudaEventDisableTiming) != cudaSuccess)) {
        cleanup();
        return CE_ERR_CUDA;
    }

    darcy_problem pf = *p, pc = *p;
    pf.n = n;
    pc.n = nc;
    const int qmask_f = a.qoi_f ? 7 : (1 << qoi_index);
    const int qmask_c = a.qoi_c ? 7 : (1 << qoi_index);
    double acc[4] = {0, 0, 0, 0};
    int n_failed = 0, max_it = 0;
    long long tot_it = 0;
    int result = CE_OK;
    auto account = [&](int r, const int *mi, int nf) {
        if (r == CE_ERR_NOT_CONVERGED) result = r;
        n_failed += nf;
        max_it = std::max(max_it, mi[0]);
        tot_it += mi[1];
    };
    for (int c0 = 0; c0 < count; c0 += chunk) {
        const int cn = std::min(chunk, count - c0);
        double *qf_c = a.qoi_f ? a.qoi_f + 3 * (size_t)c0 : qf;
        double *qc_c = coarse ? (a.qoi_c ? a.qoi_c + 3 * (size_t)c0 : qc) : nullptr;
        double *Y_c = a.Y ? a.Y + c0 : Yd;
        if (pre) {
            kf = (char *)a.kf_pre + (size_t)c0 * Vf * es;
            kc = coarse ? (char *)a.kc_pre + (size_t)c0 * Vc * es : nullptr;
        } else {
            rc = sce_sample_batch_impl(e, seed, a.level, a.first_sample + (uint64_t)c0, cn,
                                       p->precision, kf, coarse ? kc : nullptr, st, a.qa);
            if (rc != CE_OK) { cleanup(); return rc; }
        }
        int mi_c[2] = {0, 0}, nf_c = 0;
        char coarse_err[512] = {0};
        std::future<int> fut;
        if (split) {
            if (cudaEventRecord(ev_field, st) != cudaSuccess) { cleanup(); return CE_ERR_CUDA; }
            fut = std::async(std::launch::async, [&, cn]() {
                if (cudaSetDevice(dev) != cudaSuccess ||
                    cudaStreamWaitEvent(stc, ev_field, 0) != cudaSuccess)
                    return (int)CE_ERR_CUDA;
                const int r = sce_darcy_solve_impl(&pc, kc, cn, qc_c, nullptr, nullptr, nullptr,
                                                   stc, mi_c, &nf_c, qmask_c);
                if (r != CE_OK && r != CE_ERR_NOT_CONVERGED) snprintf(coarse_err, sizeof(coarse_err), "%s", sce_last_error());
                if (cudaEventRecord(ev_coarse, stc) != cudaSuccess) return (int)CE_ERR_CUDA;
                return r;
            });
        }
        int mi[2] = {0, 0}, nf = 0;
        if (nested) {
            rc = sce_darcy_solve_impl(&pc, kc, cn, qc_c, nullptr, nullptr, ucs, st, mi_c, &nf_c,
                                      qmask_c, nullptr, ff_hand);
            if (rc != CE_OK && rc != CE_ERR_NOT_CONVERGED) { cleanup(); return rc; }
            account(rc, mi_c, nf_c);
        }
        rc = sce_darcy_solve_impl(&pf, kf, cn, qf_c, nullptr, nullptr, nullptr, st, mi, &nf,
                                  qmask_f, nested ? ucs : nullptr, ff_hand);
        const int rc_c = split ? fut.get() : CE_OK;
        if (split && rc_c != CE_OK && rc_c != CE_ERR_NOT_CONVERGED) sce_set_last_error_text(coarse_err);
        if (rc != CE_OK && rc != CE_ERR_NOT_CONVERGED) { cleanup(); return rc; }
        account(rc, mi, nf);
        if (split) {
            if (rc_c != CE_OK && rc_c != CE_ERR_NOT_CONVERGED) { cleanup(); return rc_c; }
            account(rc_c, mi_c, nf_c);
            if (cudaStreamWaitEvent(st, ev_coarse, 0) != cudaSuccess) { cleanup(); return CE_ERR_CUDA; }
        } else if (coarse && !nested) {
            rc = sce_darcy_solve_impl(&pc, kc, cn, qc_c, nullptr, nullptr, nullptr, st, mi, &nf,
                                      qmask_c);
            if (rc != CE_OK && rc != CE_ERR_NOT_CONVERGED) { cleanup(); return rc; }
            account(rc, mi, nf);
        }
        {
            SceProf pr(KP_LEVEL, st, (double)cn * 32.0);
            level_diff_kernel<<<(cn + 255) / 256, 256, 0, st>>>(qf_c, qc_c, cn, qoi_index, Y_c);
        }
        {
            SceProf pr(KP_LEVEL, st, (double)cn * 16.0);
            level_sums_kernel<<<1, 256, 0, st>>>(Y_c, qf_c, cn, qoi_index, sums);
        }
        if (cudaGetLastError() != cudaSuccess) { cleanup(); return CE_ERR_CUDA; }
        double h[4];
        if (cudaMemcpyAsync(h, sums, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            cleanup();
            return CE_ERR_CUDA;
        }
        for (int r = 0; r < 4; ++r) acc[r] += h[r];
    }
    cleanup();
    mlmc_level_sums &o = *a.out;
    o.N = count;
    o.sumY = acc[0];
    o.sumY2 = acc[1];
    o.sumQf = acc[2];
    o.sumQf2 = acc[3];
    o.n_failed = n_failed;
    o.max_iters = max_it;
    o.total_iters = tot_it;
    return result;
}

static bool valid_problem(const darcy_problem *p, int qoi_index) {
    return p && qoi_index >= 0 && qoi_index <= 2 && (p->precision == 32 || p->precision == 64);
}

}  // namespace

extern "C" int mlmc_level_estimate(ce_embedding_t e, const darcy_problem *p, uint64_t seed,
                                   uint32_t level, uint64_t first_sample, int count,
                                   int qoi_index, mlmc_level_sums *out, double *Y, double *qoi_f,
                                   double *qoi_c, void *stream) {
    if (!e || !out || count < 0 || !valid_problem(p, qoi_index) || p->n != e->n)
        return CE_ERR_INVALID_ARG;
    const cudaStream_t st = as_stream(stream);
    return level_run(LevelArgs{e, level, first_sample, count, Y, qoi_f, qoi_c, out}, p, seed,
                     qoi_index, st, st);
}

// All levels of a step; pre_f / pre_c: per task, fields computed beforehand
// (or nullptr: each level samples its own).
static int estimate_levels(const darcy_problem *p, uint64_t seed, int qoi_index,
                           mlmc_level_task *tasks, int ntasks, int max_concurrency,
                           cudaStream_t st, void *const *pre_f, void *const *pre_c) {
    auto args_of = [&](int i) {
        mlmc_level_task &t = tasks[i];
        LevelArgs a{t.emb, t.level, t.first_sample, t.count, t.Y, t.qoi_f, t.qoi_c, &t.sums};
        if (pre_f) {
            a.kf_pre = pre_f[i];
            a.kc_pre = pre_c[i];
        }
        return a;
    };
    auto combine = [&]() {
        int worst = CE_OK;
        for (int i = 0; i < ntasks; ++i) {
            const int r = tasks[i].status;
            if (r != CE_OK && r != CE_ERR_NOT_CONVERGED) return r;
            if (r == CE_ERR_NOT_CONVERGED) worst = r;
        }
        return worst;
    };
    if (max_concurrency <= 1 || ntasks == 0) {
        for (int i = 0; i < ntasks; ++i) {
            tasks[i].status = level_run(args_of(i), p, seed, qoi_index, st, st);
            if (tasks[i].status != CE_OK && tasks[i].status != CE_ERR_NOT_CONVERGED) break;
        }
        return combine();
    }

    int dev = 0;
    SCE_CUDA(cudaGetDevice(&dev));
    // streams: [2 i] fine, [2 i + 1] coarse of task i; all start after the
    // work already queued on the caller's stream and the caller's stream
    // waits for all of them at the end
    std::vector<cudaStream_t> ss(2 * (size_t)ntasks, nullptr);
    std::vector<cudaEvent_t> evs;
    auto release = [&]() {
        for (cudaStream_t s : ss)
            if (s) cudaStreamDestroy(s);
        for (cudaEvent_t ev : evs) cudaEventDestroy(ev);
    };
    auto new_event = [&](cudaEvent_t *ev) {
        cudaError_t err = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
        if (err == cudaSuccess) evs.push_back(*ev);
        return err;
    };
    cudaEvent_t ev0;
    if (new_event(&ev0) != cudaSuccess || cudaEventRecord(ev0, st) != cudaSuccess) {
        release();
        return CE_ERR_CUDA;
    }
    // largest levels first: they bound the makespan
    std::vector<int> order(ntasks);
    for (int i = 0; i < ntasks; ++i) order[i] = i;
    auto work = [&](int i) {
        const long long n = tasks[i].emb->n;
        return (double)tasks[i].count * (double)((n + 1) * (n + 1)) * (tasks[i].level ? 1.25 : 1.0);
    };
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return work(x) > work(y); });
    // SCE_LEVEL_PRIORITY=1: the levels' streams get priorities by rank of work
    // (the largest the highest), so the other levels fill the gaps of the largest
    int lo_prio = 0, hi_prio = 0;
    std::vector<int> prio(ntasks, 0);
    {
        const char *e = getenv("SCE_LEVEL_PRIORITY");
        if (e && atoi(e) != 0 && cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio) == cudaSuccess)
            for (int k = 0; k < ntasks; ++k) prio[order[k]] = std::min(lo_prio, hi_prio + k);
    }
    for (int i = 0; i < ntasks; ++i) {
        for (int k = 0; k < (tasks[i].level > 0 ? 2 : 1); ++k) {
            cudaStream_t &s = ss[2 * (size_t)i + k];
            if (cudaStreamCreateWithPriority(&s, cudaStreamNonBlocking, prio[i]) != cudaSuccess ||
                cudaStreamWaitEvent(s, ev0, 0) != cudaSuccess) {
                release();
                return CE_ERR_CUDA;
            }
        }
    }
    std::atomic<int> next{0};
    // a failing task's error text (the workers' sce_last_error is thread-local)
    std::mutex err_mu;
    std::string err_text;
    auto worker = [&]() {
        if (cudaSetDevice(dev) != cudaSuccess) return;
        for (int k; (k = next.fetch_add(1)) < ntasks;) {
            const int i = order[k];
            cudaStream_t sf = ss[2 * (size_t)i], sc = ss[2 * (size_t)i + 1];
            tasks[i].status = level_run(args_of(i), p, seed, qoi_index, sf, sc ? sc : sf);
            if (tasks[i].status != CE_OK && tasks[i].status != CE_ERR_NOT_CONVERGED) {
                std::lock_guard<std::mutex> lk(err_mu);
                if (err_text.empty()) err_text = sce_last_error();
            }
        }
    };
    const int nthreads = std::min(max_concurrency, ntasks);
    std::vector<std::thread> pool;
    for (int t = 0; t < nthreads; ++t) pool.emplace_back(worker);
    for (std::thread &t : pool) t.join();
    if (!err_text.empty()) sce_set_last_error_text(err_text.c_str());
    for (cudaStream_t s : ss) {
        if (!s) continue;
        cudaEvent_t ev;
        if (new_event(&ev) != cudaSuccess || cudaEventRecord(ev, s) != cudaSuccess ||
            cudaStreamWaitEvent(st, ev, 0) != cudaSuccess) {
            release();
            return CE_ERR_CUDA;
        }
    }
    release();
    return combine();
}

extern "C" int mlmc_estimate_levels(const darcy_problem *p, uint64_t seed, int qoi_index,
                                    mlmc_level_task *tasks, int ntasks, int max_concurrency,
                                    void *stream) {
    if (!valid_problem(p, qoi_index) || ntasks < 0 || (ntasks > 0 && !tasks))
        return CE_ERR_INVALID_ARG;
    for (int i = 0; i < ntasks; ++i)
        if (!tasks[i].emb || tasks[i].count < 0) return CE_ERR_INVALID_ARG;
    for (int i = 0; i < ntasks; ++i) {
        tasks[i].sums = mlmc_level_sums{};
        tasks[i].status = CE_OK;
    }
    return estimate_levels(p, seed, qoi_index, tasks, ntasks, max_concurrency, as_stream(stream),
                           nullptr, nullptr);
}

extern "C" int mlmc_estimate_levels_persistent(const darcy_problem *p, uint64_t seed,
                                               int qoi_index, mlmc_level_task *tasks, int ntasks,
                                               int max_concurrency, void *stream) {
    if (!valid_problem(p, qoi_index) || p->precision != 32 || ntasks < 1 || ntasks > 16 || !tasks)
        return CE_ERR_INVALID_ARG;
    for (int i = 0; i < ntasks; ++i)
        if (!tasks[i].emb || tasks[i].count < 0 || tasks[i].emb->P > 4096)
            return CE_ERR_INVALID_ARG;
    for (int i = 0; i < ntasks; ++i) {
        tasks[i].sums = mlmc_level_sums{};
        tasks[i].status = CE_OK;
    }
    const cudaStream_t st = as_stream(stream);
    // every level's fields in one persistent launch on the caller's stream
    std::vector<void *> pf(ntasks, nullptr), pc(ntasks, nullptr);
    std::vector<ce_field_task> ft(ntasks);
    int rc = CE_OK;
    for (int i = 0; i < ntasks && rc == CE_OK; ++i) {
        const mlmc_level_task &t = tasks[i];
        const long long n = t.emb->n, nc = n / 2;
        const size_t cnt = (size_t)std::max(t.count, 1);
        rc = sce_alloc(&pf[i], cnt * (n + 1) * (n + 1) * sizeof(float), st);
        if (rc == CE_OK && t.level > 0)
            rc = sce_alloc(&pc[i], cnt * (nc + 1) * (nc + 1) * sizeof(float), st);
        ft[i] = ce_field_task{t.emb, t.level, t.first_sample, t.count, pf[i], pc[i]};
    }
    if (rc == CE_OK) rc = ce_sample_levels(ft.data(), ntasks, seed, nullptr, st);
    if (rc == CE_OK)
        rc = estimate_levels(p, seed, qoi_index, tasks, ntasks, max_concurrency, st, pf.data(),
                             pc.data());
    for (int i = 0; i < ntasks; ++i) {
        if (pf[i]) sce_free(pf[i], st);
        if (pc[i]) sce_free(pc[i], st);
    }
    return rc;
}

extern "C" int mlmc_level_estimate_qmc(ce_qmc_t q, const darcy_problem *p, uint64_t seed,
                                       uint32_t level, uint32_t shift, uint32_t first_point,
                                       int count, int qoi_index, mlmc_level_sums *out, double *Y,
                                       double *qoi_f, double *qoi_c, void *stream) {
    if (!q || !out || count < 0 || !valid_problem(p, qoi_index) || p->n != q->e->n ||
        (uint64_t)first_point + (uint64_t)count > q->N)
        return CE_ERR_INVALID_ARG;
    const QmcArgs qa{q->zr, q->N, ((uint64_t)level << 32) | shift};
    LevelArgs a{q->e, level, first_point, count, Y, qoi_f, qoi_c, out};
    a.qa = &qa;
    const cudaStream_t st = as_stream(stream);
    return level_run(a, p, seed, qoi_index, st, st);
}
