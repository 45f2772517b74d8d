// Optional launch profiler: CUDA events around each kernel launch, per kernel
// family, with the algorithmic bytes the caller attributes to the launch.
// Off by default (no events are recorded); sce_profile_enable(1) resets and
// turns it on, sce_profile_read() waits for the recorded events and returns
// per-family totals.
#include <mutex>
#include <vector>

#include "sce_internal.cuh"

namespace {
struct Rec {
    int id;
    cudaEvent_t a, b;
    double bytes;
    cudaStream_t st;
};
std::mutex g_mu;
bool g_on = false;
long long g_gen = 0;   // bumped whenever the records are folded into the totals
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_free;
double g_ms[KP_COUNT_], g_bytes[KP_COUNT_];
long long g_launches[KP_COUNT_];

cudaEvent_t get_event() {
    if (!g_free.empty()) {
        cudaEvent_t e = g_free.back();
        g_free.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void resolve_locked() {
    for (Rec &r : g_recs) {
        float ms = 0.f;
        if (r.b && cudaEventSynchronize(r.b) == cudaSuccess &&
            cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            g_ms[r.id] += ms;
            g_bytes[r.id] += r.bytes;
            g_launches[r.id] += 1;
        }
        g_free.push_back(r.a);
        if (r.b) g_free.push_back(r.b);
    }
    g_recs.clear();
    ++g_gen;
}

const char *kNames[KP_COUNT_] = {
    "ce_row", "ce_col", "cond", "coarsen", "mg_smooth", "mg_restrict", "mg_prolong",
    "mg_coarsest", "cg_spmv_dot", "cg_axpy", "cg_dot", "cg_pupdate", "cg_copy", "reduce",
    "ir_residual", "ir_update", "qoi", "setup", "normals", "level_sums", "darcy_small", "mg_down", "mg_up", "mg_tail",
    "ce3_x", "ce3_y", "ce3_z", "cond3", "mg3_smooth", "mg3_resid", "mg3_restrict", "mg3_prolong",
    "cg3_spmv_dot", "cg3_vec", "ir3", "mg_v64", "ce_levels", "coarsen_tail", "mg_down3",
    "mg_up3"};
}  // namespace

bool sce_prof_on() { return g_on; }

SceProf::SceProf(int kernel, cudaStream_t s, double bytes) {
    if (!g_on) return;
    std::lock_guard<std::mutex> lk(g_mu);
    id = kernel;
    st = s;
    Rec r{kernel, get_event(), nullptr, bytes, s};
    cudaEventRecord(r.a, s);
    g_recs.push_back(r);
    slot = (int)g_recs.size() - 1;
}

SceProf::~SceProf() {
    if (slot < 0) return;
    std::lock_guard<std::mutex> lk(g_mu);
    if (slot < (int)g_recs.size() && g_recs[slot].id == id && g_recs[slot].b == nullptr) {
        g_recs[slot].b = get_event();
        cudaEventRecord(g_recs[slot].b, st);
    }
}

SceProfMark sce_prof_mark() {
    std::lock_guard<std::mutex> lk(g_mu);
    return SceProfMark{g_gen, (long long)g_recs.size()};
}

void sce_prof_scale(const SceProfMark &m, cudaStream_t st, const int *ids, int nids, double f) {
    if (!g_on || !(f >= 0.0)) return;
    std::lock_guard<std::mutex> lk(g_mu);
    if (m.gen != g_gen) return;   // the records were folded in since the mark
    for (size_t i = (size_t)m.idx; i < g_recs.size(); ++i) {
        Rec &r = g_recs[i];
        if (r.st != st) continue;
        for (int k = 0; k < nids; ++k)
            if (r.id == ids[k]) {
                r.bytes *= f;
                break;
            }
    }
}

extern "C" void sce_profile_enable(int on) {
    std::lock_guard<std::mutex> lk(g_mu);
    resolve_locked();
    for (int i = 0; i < KP_COUNT_; ++i) {
        g_ms[i] = 0;
        g_bytes[i] = 0;
        g_launches[i] = 0;
    }
    g_on = on != 0;
}

extern "C" int sce_profile_read(int id, double *ms, double *bytes, long long *launches) {
    if (id < 0 || id >= KP_COUNT_) return CE_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    resolve_locked();
    if (ms) *ms = g_ms[id];
    if (bytes) *bytes = g_bytes[id];
    if (launches) *launches = g_launches[id];
    return CE_OK;
}

extern "C" int sce_profile_count(void) { return KP_COUNT_; }

extern "C" const char *sce_profile_name(int id) {
    return (id >= 0 && id < KP_COUNT_) ? kNames[id] : "";
}
