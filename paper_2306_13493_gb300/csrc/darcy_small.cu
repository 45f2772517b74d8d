// One-block-per-sample Darcy solver for small grids (n <= 64), mixed precision.
//
// The same discrete problem and the same algorithm as the batched solver in
// darcy.cu (float-float iterative refinement around FP32 CG preconditioned
// with one symmetric multigrid cycle, here V(1,1)), but the whole solve of one sample --
// conductances, hierarchy, every CG iteration and V-cycle, the QoIs -- runs in
// one thread block with all state in shared memory: the coefficient field is
// read from HBM once and three doubles per sample are written back.  Many
// independent samples in flight per SM hide the block barriers.
#include <algorithm>

#include "block_mg.cuh"
#include "sce_internal.cuh"
#include "stencil.cuh"

using namespace sce;

namespace {

constexpr int ilog2c(int v) { return v <= 1 ? 0 : 1 + ilog2c(v / 2); }

// Shared-memory layout of one sample: every level-0 array in rows of PW
// values (N + 2 with PAD on grids of at least 32 cells, see mg_pitch), V
// vertices, VP values per array.
template <int N, bool PAD> struct SmallLayout {
    using MG = MGPackedLayout<N, PAD>;
    static constexpr int W = N + 1;
    static constexpr int PW = MG::pitch(0);
    static constexpr int V = W * W;
    static constexpr int VP = W * PW;
    static constexpr int NL = ilog2c(N);            // levels N, N/2, ..., 2
    // float2: u as float-float; doubles: reduction scratch (64); floats: the
    // multigrid hierarchy (level 0 holds the conductances' hi parts), their lo
    // parts, d, p
    static constexpr size_t bytes = sizeof(float2) * (size_t)VP + sizeof(double) * 64 +
                                    sizeof(float) * (MG::total() + 4 * (size_t)VP);
};

// Sum over the block, returned to every thread (fixed order: warp trees,
// then the warp partials in index order by every thread).  One barrier: the
// partials alternate between two buffers (`par` flips per call), so a thread
// that runs ahead writes the other buffer while the slower ones still read
// this one, and the next call's barrier orders the reuse.
template <int NT, typename R>
__device__ __forceinline__ R bsum1(R v, R *sh, int &par) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if constexpr (NT == 32) {   // one warp: the tree's result, from lane 0 to every lane
        return __shfl_sync(0xffffffffu, v, 0);
    }
    R *buf = sh + (par ? 16 : 0);
    par ^= 1;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) buf[w] = v;
    __syncthreads();
    R t = R(0);
#pragma unroll
    for (int i = 0; i < NT / 32; ++i) t += buf[i];
    return t;
}

template <int N, int NT, int NU = 1, bool PAD = false>
__global__ void __launch_bounds__(NT, N >= 16 ? 1024 / NT : 1) small_solve_kernel(
    const float *__restrict__ kin, double f, double rtol2, double in_rel2, int maxit,
    double *__restrict__ qoi, int *__restrict__ iters_out, int *__restrict__ status_out,
    double *__restrict__ u_out, int *__restrict__ nfail, int *__restrict__ maxits, int qmask,
    const float2 *__restrict__ u0f, const double *__restrict__ u0d) {
    using Lay = SmallLayout<N, PAD>;
    using MG = typename Lay::MG;
    constexpr int W = Lay::W, PW = Lay::PW, V = Lay::V, VP = Lay::VP, NL = Lay::NL;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *u = reinterpret_cast<float2 *>(smem_raw);
    double *sh = reinterpret_cast<double *>(u + VP);
    // FP32 region: the multigrid hierarchy (level 0 = [cx | cy | r | z]), then
    // the lo parts of the level-0 conductances, d, p
    float *mg = reinterpret_cast<float *>(sh + 64);
    float *cx0 = mg + MG::off(0, 0), *cy0 = mg + MG::off(0, 1);
    float *r = mg + MG::off(0, 2), *z = mg + MG::off(0, 3);
    float *cxl = mg + MG::total();
    float *cyl = cxl + VP;
    float *d = cyl + VP;
    float *p = d + VP;
    const int s = blockIdx.x;
    const int tid = threadIdx.x;
    const float *ks = kin + (size_t)s * V;
    int pard = 0, parf = 0;   // buffer parity of the FP64 and FP32 block sums

    // operator: float-float conductances, hi = the FP32 operator of the inner solve
    // (v: the vertex in the dense layout of k and of the outputs; q: its slot
    // in the shared-memory arrays of row pitch PW)
    for (int v = tid; v < V; v += NT) {
        const int j = v / W, i = v - j * W, q = j * PW + i;
        ff gx, gy;
        cond_at_ff(ks, i, j, N, &gx, &gy);
        cx0[q] = gx.hi;
        cy0[q] = gy.hi;
        cxl[q] = gx.lo;
        cyl[q] = gy.lo;
        u[q] = make_float2(i == 0 ? 1.0f : 0.0f, 0.0f);
    }
    block_sync<NT>();
    block_coarsen<float, N, NT, MG, 1>(mg);

    // load F = f h^2/6 x (triangles at the vertex): 3 on the rows j = 0, N, 6 inside
    const double h2_6 = f / (6.0 * (double)N * (double)N);
    ff Fv[2];
    for (int q = 0; q < 2; ++q) Fv[q] = ff_from_double(h2_6 * (q ? 6.0 : 3.0));
    // float-float residual r = F - A u, rounded into the FP32 rhs; returns |r|^2
    auto outer_residual = [&]() {
        float acc = 0.f;
        for (int v = tid; v < V; v += NT) {
            const int j = v / W, i = v - j * W;
            float rv = 0.f;
            if (i > 0 && i < N) {
                rv = resid_at_ff((j > 0 && j < N) ? Fv[1] : Fv[0], cx0, cxl, cy0, cyl, u, i, j, N,
                                 PW);
                acc += rv * rv;
            }
            r[j * PW + i] = rv;
        }
        return bsum1<NT>((double)acc, sh, pard);
    };

    // one symmetric V(NU,NU) cycle: z[0] = M^-1 r (one sweep per side by
    // default: every half-sweep of this solver is a block barrier, and V(2,2)
    // measured slower here than the iterations it saves)
    static_assert(NL == mg_levels(N), "level count");
    auto vcycle = [&]() { block_vcycle<float, N, NT, MG, 0, NU>(mg); };

    // residual of the lifting in closed form: r0 = F + [i = 1] cx(0, j)
    double orr;
    {
        float acc = 0.f;
        for (int v = tid; v < V; v += NT) {
            const int j = v / W, i = v - j * W, q = j * PW + i;
            float rv = 0.f;
            if (i > 0 && i < N) {
                ff rf = (j > 0 && j < N) ? Fv[1] : Fv[0];
                if (i == 1) rf = ff_add(rf, ff{cx0[q - 1], cxl[q - 1]});
                rv = rf.hi;
                acc += rv * rv;
            }
            r[q] = rv;
        }
        orr = bsum1<NT>((double)acc, sh, pard);
    }
    const double orr0 = orr;
    // a first iterate from the n/2 solution (nested iteration): u = P u_c with
    // float-float additions and exact halvings, then its float-float residual
    if (u0f || u0d) {
        constexpr int NCc = N / 2, WCc = NCc + 1;
        const size_t cb = (size_t)s * WCc * WCc;
        auto U = [&](int jj, int ii) {
            const size_t q = cb + (size_t)jj * WCc + ii;
            if (u0f) {
                const float2 t = u0f[q];
                return ff{t.x, t.y};
            }
            return ff_from_double(u0d[q]);
        };
        for (int v = tid; v < V; v += NT) {
            const int j = v / W, i = v - j * W;
            const int i0 = i >> 1, i1 = (i + 1) >> 1, j0 = j >> 1, j1 = (j + 1) >> 1;
            ff a = U(j0, i0);
            float sc = 1.0f;
            if (i1 != i0) {
                a = ff_add(a, U(j0, i1));
                sc = 0.5f;
            }
            if (j1 != j0) {
                ff b = U(j1, i0);
                if (i1 != i0) b = ff_add(b, U(j1, i1));
                a = ff_add(a, b);
                sc *= 0.5f;
            }
            u[j * PW + i] = make_float2(a.hi * sc, a.lo * sc);
        }
        block_sync<NT>();
        orr = outer_residual();
    }
    float *shf = reinterpret_cast<float *>(sh + 40);
    int its = 0;
    for (int outer = 0; outer < 64 && orr > rtol2 * orr0 && its < maxit; ++outer) {
        // inner CG on A d = r, entirely in FP32 (dot products included)
        float rr0 = 0.f;
        for (int v = tid; v < V; v += NT) {
            const int j = v / W, q = j * PW + (v - j * W);
            d[q] = 0.f;
            rr0 += r[q] * r[q];
        }
        rr0 = bsum1<NT>(rr0, shf, parf);
        const float thr = (float)fmax(in_rel2 * (double)rr0, 0.0625 * rtol2 * orr0);
        vcycle();
        float rz = 0.f;
        for (int v = tid; v < V; v += NT) {
            const int j = v / W, q = j * PW + (v - j * W);
            p[q] = z[q];
            rz += r[q] * z[q];
        }
        rz = bsum1<NT>(rz, shf, parf);
        for (int it = 0; it < 40 && its < maxit; ++it) {
            // q = A p, kept in the multigrid z array (free until the next cycle)
            float pq = 0.f;
            for (int v = tid; v < V; v += NT) {
                const int j = v / W, i = v - j * W, q = j * PW + i;
                if (i > 0 && i < N) {
                    const float ap = apply_at(cx0, cy0, p, i, j, N, PW);
                    z[q] = ap;
                    pq += p[q] * ap;
                }
            }
            pq = bsum1<NT>(pq, shf, parf);
            const float alpha = pq > 0.f ? rz / pq : 0.f;
            float rr = 0.f;
            for (int v = tid; v < V; v += NT) {
                const int j = v / W, i = v - j * W, q = j * PW + i;
                if (i > 0 && i < N) {
                    const float ap = z[q];
                    d[q] += alpha * p[q];
                    const float rv = r[q] - alpha * ap;
                    r[q] = rv;
                    rr += rv * rv;
                }
            }
            rr = bsum1<NT>(rr, shf, parf);
            ++its;
            if (rr <= thr) break;
            vcycle();
            float rzn = 0.f;
            for (int v = tid; v < V; v += NT) {
                const int j = v / W, q = j * PW + (v - j * W);
                rzn += r[q] * z[q];
            }
            rzn = bsum1<NT>(rzn, shf, parf);
            const float beta = rz > 0.f ? rzn / rz : 0.f;
            rz = rzn;
            for (int v = tid; v < V; v += NT) {
                const int j = v / W, q = j * PW + (v - j * W);
                p[q] = z[q] + beta * p[q];
            }
            block_sync<NT>();
        }
        for (int v = tid; v < V; v += NT) {
            const int j = v / W, q = j * PW + (v - j * W);
            const ff t = ff_add_f(ff{u[q].x, u[q].y}, d[q]);
            u[q] = make_float2(t.hi, t.lo);
        }
        block_sync<NT>();
        orr = outer_residual();
    }

    // QoIs (FP64): the outflow (bit 0 of qmask) and L2 norm (bit 2) need a
    // pass over the grid, the point value (bit 1) does not
    double qo = 0.0, l2 = 0.0;
    const bool want_out = qmask & 1, want_l2 = qmask & 4;
    auto ud = [&](int q) { return (double)u[q].x + (double)u[q].y; };
    if (want_out || want_l2 || u_out) {
        for (int v = tid; v < V; v += NT) {
            const int j = v / W, i = v - j * W, q = j * PW + i;
            if (want_out && i == N - 1) qo += ((double)cx0[q] + (double)cxl[q]) * ud(q);
            if (want_l2 && i < N && j < N) {
                const double a = ud(q), b = ud(q + 1), c = ud(q + PW + 1), e = ud(q + PW);
                const double s1 = a + b + c, s2 = a + e + c;
                l2 += s1 * s1 + a * a + b * b + c * c + s2 * s2 + a * a + e * e + c * c;
            }
            if (u_out) {
                if (qmask & 8) reinterpret_cast<float2 *>(u_out)[(size_t)s * V + v] = u[q];
                else u_out[(size_t)s * V + v] = ud(q);
            }
        }
        qo = bsum1<NT>(qo, sh, pard);
        l2 = bsum1<NT>(l2, sh, pard);
    }
    if (tid == 0) {
        const double h = 1.0 / (double)N;
        const double q_out = want_out ? qo + f * h * 0.5 : 0.0;
        const double q_l2 = want_l2 ? sqrt(l2 * h * h / 24.0) : 0.0;
        const double xs = 7.0 / 15.0 * (double)N, ys = 7.0 / 15.0 * (double)N;
        const int ca = min((int)floor(xs), N - 1), cb = min((int)floor(ys), N - 1);
        const double xi = xs - ca, et = ys - cb;
        const double uab = ud(cb * PW + ca), ua1b = ud(cb * PW + ca + 1);
        const double uab1 = ud((cb + 1) * PW + ca), ua1b1 = ud((cb + 1) * PW + ca + 1);
        const double q_pt = !(qmask & 2) ? 0.0
                            : xi >= et ? uab + xi * (ua1b - uab) + et * (ua1b1 - ua1b)
                                       : uab + et * (uab1 - uab) + xi * (ua1b1 - uab1);
        qoi[3 * s + 0] = q_out;
        qoi[3 * s + 1] = q_pt;
        qoi[3 * s + 2] = q_l2;
        int st = 0;
        if (!(fabs(q_out) < 1e300 && fabs(q_pt) < 1e300 && fabs(q_l2) < 1e300)) st = CE_ERR_NONFINITE;
        else if (!(orr <= rtol2 * orr0)) st = CE_ERR_NOT_CONVERGED;
        if (status_out) status_out[s] = st;
        if (iters_out) iters_out[s] = its;
        if (st) atomicAdd(nfail, 1);
        atomicMax(maxits, its);
        atomicAdd(maxits + 1, its);
    }
}

template <int N, int NT, int NU = 1, bool PAD = false>
int launch_small(const darcy_problem *p, const float *k, int count, double *qoi, int *iters,
                 int *status, double *u_out, int *misc, int qmask, const float2 *u0f,
                 const double *u0d, cudaStream_t st) {
    using Lay = SmallLayout<N, PAD>;
    const size_t smem = Lay::bytes;
    SCE_TRY(sce_raise_smem_limit((const void *)small_solve_kernel<N, NT, NU, PAD>, smem));
    const double in_rel = sce_inner_rel_f32();
    SceProf pr(KP_SMALL, st, (double)count * Lay::V * (sizeof(float) + 0.0) + 24.0 * count);
    small_solve_kernel<N, NT, NU, PAD><<<count, NT, smem, st>>>(
        k, p->f, p->rtol * p->rtol, in_rel * in_rel, p->maxit > 0 ? p->maxit : 1000, qoi, iters,
        status, u_out, misc, misc + 1, qmask, u0f, u0d);
    SCE_CUDA(cudaGetLastError());
    return CE_OK;
}

}  // namespace

// n = 16: two warps per sample; SCE_SMALL16_NT=32 runs one warp per sample with
// warp synchronisation only (measured slower: 7.89 vs 7.31 ms per sweep)
static int small16_threads() {
    const char *e = getenv("SCE_SMALL16_NT");
    return e && atoi(e) == 32 ? 32 : 64;
}

// Sweeps per side of the n = 16 solver's cycle (SCE_SMALL16_NU: 1 or 2; its
// two-warp blocks make a barrier cheap).
static int small16_nu() {
    const char *e = getenv("SCE_SMALL16_NU");
    return e && atoi(e) == 2 ? 2 : 1;
}

// Threads per block of the n = 32 solver (SCE_SMALL32_NT: 128 or 256).
static int small32_threads() {
    const char *e = getenv("SCE_SMALL32_NT");
    return e && atoi(e) == 128 ? 128 : 256;
}

// Largest n solved one block per sample (SCE_SMALL_MAX_N overrides; 0 = never).
int sce_small_max_n() {
    const char *e = getenv("SCE_SMALL_MAX_N");
    return e ? atoi(e) : 32;
}

int sce_darcy_small(const darcy_problem *p, const float *k, int count, double *qoi, int *iters,
                    int *status, double *u_out, cudaStream_t st, int *max_iters_out,
                    int *n_failed_out, int qmask, const void *u_init, bool u_init_ff) {
    const float2 *u0f = u_init_ff ? static_cast<const float2 *>(u_init) : nullptr;
    const double *u0d = u_init_ff ? nullptr : static_cast<const double *>(u_init);
    int *misc = nullptr;   // [0] failed samples, [1] max iterations, [2] total iterations
    SCE_TRY(sce_alloc_t(&misc, 3, st));
    SCE_CUDA(cudaMemsetAsync(misc, 0, 3 * sizeof(int), st));
    int rc = CE_ERR_INVALID_ARG;
#define SCE_SMALL(NN, TT) \
    rc = launch_small<NN, TT>(p, k, count, qoi, iters, status, u_out, misc, qmask, u0f, u0d, st)
    switch (p->n) {
        case 4: SCE_SMALL(4, 32); break;
        case 8: SCE_SMALL(8, 64); break;
        case 16:
            if (small16_threads() == 32) SCE_SMALL(16, 32);
            else if (small16_nu() == 2)
                rc = launch_small<16, 64, 2>(p, k, count, qoi, iters, status, u_out, misc, qmask,
                                             u0f, u0d, st);
            else SCE_SMALL(16, 64);
            break;
        case 32:
            if (small32_threads() == 128) SCE_SMALL(32, 128);
            else if (sce_small_pad())
                rc = launch_small<32, 256, 1, true>(p, k, count, qoi, iters, status, u_out, misc,
                                                    qmask, u0f, u0d, st);
            else SCE_SMALL(32, 256);
            break;
        case 64:
            if (sce_small_pad())
                rc = launch_small<64, 512, 1, true>(p, k, count, qoi, iters, status, u_out, misc,
                                                    qmask, u0f, u0d, st);
            else SCE_SMALL(64, 512);
            break;
        default: break;
    }
#undef SCE_SMALL
    if (rc != CE_OK) {
        sce_free(misc, st);
        return rc;
    }
    int h[3] = {0, 0, 0};
    SCE_CUDA(cudaMemcpyAsync(h, misc, sizeof(h), cudaMemcpyDeviceToHost, st));
    SCE_CUDA(cudaStreamSynchronize(st));
    sce_free(misc, st);
    if (n_failed_out) *n_failed_out = h[0];
    if (max_iters_out) {
        max_iters_out[0] = h[1];
        max_iters_out[1] = h[2];
    }
    return h[0] > 0 ? CE_ERR_NOT_CONVERGED : CE_OK;
}
