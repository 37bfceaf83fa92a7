// tune.cu -- autotuners for the layout and launch schedule of a workload.
//
// gpe_autotune: for an analytic potential, cutoff, state type and step kind,
// builds the grid with each candidate brick shape (8x8x8, 8x8x4, 8x4x4) and
// schedule (staged; wavefront with 2 or 8 bricks per task; for real time also
// the RK4 stages fused in pairs), times `nsteps` steps with CUDA events after
// one warm-up step, and returns the fastest in active-cell-steps per second.
// Results are cached per (state type, step kind, size class = round(2 log2
// n_active)) for the life of the process.
//
// gpe_batch_autotune: the brick shape of a batch of shells (the batch kernels
// run the staged schedule), timed on the batch itself.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>
#include <vector>

#include "gpe_internal.cuh"

namespace gpe {

// a smooth, finite test state: psi = exp(-|V| * w) on active cells (real
// part of a complex state, or the value of a real one)
template <typename CT>
__global__ void k_tune_fill(CT *psi, const double *V, int64_t n, double w)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double f = V[i] < INFINITY ? exp(-fabs(V[i]) * w) : 0.0;
        if constexpr (std::is_arithmetic<CT>::value) {
            psi[i] = (CT)f;
        } else {
            CT v;
            v.x = f;
            v.y = 0;
            psi[i] = v;
        }
    }
}

static void tune_fill(gpe_state *st, double w, cudaStream_t s)
{
    const gpe_grid *g = st->grid;
    switch (st->dtype) {
    case GPE_C128: k_tune_fill<double2><<<g->nsm * 8, 256, 0, s>>>((double2 *)st->d_psi, g->d_V[0], g->n_packed, w); break;
    case GPE_C64: k_tune_fill<float2><<<g->nsm * 8, 256, 0, s>>>((float2 *)st->d_psi, g->d_V[0], g->n_packed, w); break;
    case GPE_R64: k_tune_fill<double><<<g->nsm * 8, 256, 0, s>>>((double *)st->d_psi, g->d_V[0], g->n_packed, w); break;
    default: k_tune_fill<float><<<g->nsm * 8, 256, 0, s>>>((float *)st->d_psi, g->d_V[0], g->n_packed, w); break;
    }
    count_launch();
}

static std::mutex g_tune_mu;
static std::map<std::tuple<int, int, int, int>, gpe_tune_result> g_tune_cache;

}  // namespace gpe

using namespace gpe;

extern "C" int gpe_autotune(const gpe_box *box, const gpe_potential *pot, double V_cut, int dtype, int mode,
                            int nsteps, gpe_tune_result *best, gpe_tune_result *all, int *n_all, gpe_stream stream)
{
    if (!box || !pot || !best) return fail(GPE_ERR_ARG, "NULL argument");
    if (mode != GPE_TUNE_REAL && mode != GPE_TUNE_IMAG) return fail(GPE_ERR_ARG, "mode must be GPE_TUNE_REAL or GPE_TUNE_IMAG");
    if (dtype != GPE_C128 && dtype != GPE_C64 && !(mode == GPE_TUNE_IMAG && (dtype == GPE_R64 || dtype == GPE_R32)))
        return fail(GPE_ERR_ARG, "dtype must be GPE_C128 or GPE_C64 (or GPE_R64 / GPE_R32 for imaginary time)");
    if (nsteps < 1) return fail(GPE_ERR_ARG, "nsteps must be >= 1");
    cudaStream_t s = S(stream);
    int dev = 0;
    GPE_TRY_CUDA(cudaGetDevice(&dev));
    struct Cand {
        int bx, by, bz, sched, chunk;
    };
    // the last candidate, RK4 stages fused in pairs (fusion depth 2), applies
    // to real-time steps only
    const Cand cands[] = {{8, 8, 8, GPE_SCHED_STAGED, 0}, {8, 8, 4, GPE_SCHED_STAGED, 0}, {8, 4, 4, GPE_SCHED_STAGED, 0},
                          {8, 8, 8, GPE_SCHED_WAVE, 2},   {8, 8, 8, GPE_SCHED_WAVE, 8},   {8, 8, 4, GPE_SCHED_WAVE, 4},
                          {8, 4, 4, GPE_SCHED_WAVE, 8},   {8, 8, 4, GPE_SCHED_PAIR, 0}};
    const int nc = (int)(sizeof cands / sizeof cands[0]) - (mode == GPE_TUNE_REAL ? 0 : 1);
    std::vector<gpe_tune_result> res;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    GPE_TRY_CUDA(cudaEventCreate(&e0));
    GPE_TRY_CUDA(cudaEventCreate(&e1));
    int rc = GPE_OK;
    int64_t n_active = 0;
    for (int c = 0; c < nc && rc == GPE_OK; ++c) {
        gpe_grid_opts o{};
        o.bx = cands[c].bx;
        o.by = cands[c].by;
        o.bz = cands[c].bz;
        o.sched = cands[c].sched;
        o.chunk = cands[c].chunk;
        o.order = GPE_ORDER_ZMAJOR;
        gpe_grid *g = nullptr;
        gpe_state *st = nullptr;
        rc = gpe_grid_create_analytic(box, pot, V_cut, &o, &g, stream);
        if (rc != GPE_OK) break;
        n_active = g->n_active;
        if (c == 0 && !all) {
            // a cached answer for this size class needs no timing
            const auto key = std::make_tuple(dev, dtype, mode, (int)std::lround(2.0 * std::log2((double)n_active)));
            std::lock_guard<std::mutex> lk(g_tune_mu);
            auto it = g_tune_cache.find(key);
            if (it != g_tune_cache.end()) {
                *best = it->second;
                gpe_grid_destroy(g);
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                if (n_all) *n_all = 0;
                return GPE_OK;
            }
        }
        rc = gpe_state_create(g, dtype, &st);
        if (rc == GPE_OK) {
            const double h2 = 2.0 / (box->hx * box->hx) + 2.0 / (box->hy * box->hy) + 2.0 / (box->hz * box->hz);
            const double dt = 0.2 / (h2 + g->v_max + 1e-300);
            const double w = g->v_max > 0 ? 1.0 / g->v_max : 1.0;
            tune_fill(st, w, s);
            gpe_real_params rp{};
            rp.g = 1.0;
            rp.dt = dt;
            rp.integrator = GPE_RK4;
            rp.potential = GPE_V_STATIC;
            gpe_imag_params ip{1.0, dt, 1.0};
            auto run = [&](int n) {
                return mode == GPE_TUNE_REAL ? gpe_step_real(st, &rp, n, 0.0, stream) : gpe_step_imag(st, &ip, n, stream);
            };
            rc = run(1);
            if (rc == GPE_OK && cudaEventRecord(e0, s) != cudaSuccess) rc = fail(GPE_ERR_CUDA, "event record failed");
            if (rc == GPE_OK) rc = run(nsteps);
            if (rc == GPE_OK && cudaEventRecord(e1, s) != cudaSuccess) rc = fail(GPE_ERR_CUDA, "event record failed");
            float ms = 0.f;
            if (rc == GPE_OK && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
                rc = fail(GPE_ERR_CUDA, "event timing failed");
            if (rc == GPE_OK) {
                gpe_tune_result r{};
                r.bx = cands[c].bx;
                r.by = cands[c].by;
                r.bz = cands[c].bz;
                r.sched = cands[c].sched;
                r.chunk = cands[c].chunk;
                r.ms_per_step = ms / nsteps;
                r.cell_steps_per_s = (double)g->n_active * nsteps / (ms * 1e-3);
                res.push_back(r);
            }
            gpe_state_destroy(st);
        }
        gpe_grid_destroy(g);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != GPE_OK) return rc;
    int bi = 0;
    for (int i = 1; i < (int)res.size(); ++i)
        if (res[i].cell_steps_per_s > res[bi].cell_steps_per_s) bi = i;
    *best = res[bi];
    if (all)
        for (size_t i = 0; i < res.size(); ++i) all[i] = res[i];
    if (n_all) *n_all = (int)res.size();
    const auto key = std::make_tuple(dev, dtype, mode, (int)std::lround(2.0 * std::log2((double)n_active)));
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = res[bi];
    return GPE_OK;
}

extern "C" int gpe_batch_autotune(const gpe_box *boxes, const gpe_potential *pots, const double *V_cuts, int n,
                                  int dtype, int nsteps, gpe_tune_result *best, gpe_tune_result *all, int *n_all,
                                  gpe_stream stream)
{
    if (!boxes || !pots || !V_cuts || !best) return fail(GPE_ERR_ARG, "NULL argument");
    if (n < 1 || n > 1000000) return fail(GPE_ERR_ARG, "need 1 <= n <= 1e6 shells");
    if (dtype != GPE_C128 && dtype != GPE_C64 && dtype != GPE_R64 && dtype != GPE_R32)
        return fail(GPE_ERR_ARG, "unknown state type %d", dtype);
    if (nsteps < 1) return fail(GPE_ERR_ARG, "nsteps must be >= 1");
    static const int shapes[3][3] = {{8, 8, 8}, {8, 8, 4}, {8, 4, 4}};
    std::vector<gpe_tune_result> res;
    int rc = GPE_OK;
    for (int c = 0; c < 3 && rc == GPE_OK; ++c) {
        std::vector<gpe_grid *> grids(n, nullptr);
        std::vector<gpe_state *> states(n, nullptr);
        std::vector<gpe_imag_params> ip(n);
        gpe_batch *B = nullptr;
        int64_t active = 0;
        gpe_grid_opts o{};
        o.bx = shapes[c][0];
        o.by = shapes[c][1];
        o.bz = shapes[c][2];
        o.sched = GPE_SCHED_STAGED;
        o.order = GPE_ORDER_ZMAJOR;
        o.stencil = 7;
        for (int i = 0; i < n && rc == GPE_OK; ++i) {
            rc = gpe_grid_create_analytic(&boxes[i], &pots[i], V_cuts[i], &o, &grids[i], stream);
            if (rc == GPE_OK) rc = gpe_state_create(grids[i], dtype, &states[i]);
            if (rc != GPE_OK) break;
            const gpe_grid *g = grids[i];
            const gpe_box &b = boxes[i];
            const double h2 = 2.0 / (b.hx * b.hx) + 2.0 / (b.hy * b.hy) + 2.0 / (b.hz * b.hz);
            tune_fill(states[i], g->v_max > 0 ? 1.0 / g->v_max : 1.0, S(stream));
            ip[i] = gpe_imag_params{1.0, 0.2 / (h2 + g->v_max + 1e-300), 1.0};
            active += g->n_active;
        }
        if (rc == GPE_OK) rc = gpe_batch_create(states.data(), n, &B);
        // an unreachable tolerance: every shell runs max_steps steps.  One
        // block of nsteps records the graph; then one and two blocks are
        // timed, and their difference is nsteps steps of the batch alone.
        double sec[2] = {0.0, 0.0};
        for (int k = 0; k < 3 && rc == GPE_OK; ++k) {
            const int64_t m = k == 2 ? 2 * (int64_t)nsteps : (int64_t)nsteps;
            const auto t0 = std::chrono::steady_clock::now();
            int r = gpe_batch_ground_state(B, ip.data(), 1e-300, nsteps, m, nullptr, nullptr, nullptr, stream);
            const auto t1 = std::chrono::steady_clock::now();
            if (r == GPE_ERR_NOT_CONVERGED) r = GPE_OK;
            rc = r;
            if (k > 0) sec[k - 1] = std::chrono::duration<double>(t1 - t0).count();
        }
        if (rc == GPE_OK) {
            const double dtm = std::max(sec[1] - sec[0], 1e-9);
            gpe_tune_result r{};
            r.bx = shapes[c][0];
            r.by = shapes[c][1];
            r.bz = shapes[c][2];
            r.sched = GPE_SCHED_STAGED;
            r.ms_per_step = dtm * 1e3 / nsteps;
            r.cell_steps_per_s = (double)active * nsteps / dtm;
            res.push_back(r);
        }
        if (B) gpe_batch_destroy(B);
        for (int i = 0; i < n; ++i) {
            if (states[i]) gpe_state_destroy(states[i]);
            if (grids[i]) gpe_grid_destroy(grids[i]);
        }
    }
    if (rc != GPE_OK) return rc;
    int bi = 0;
    for (int i = 1; i < (int)res.size(); ++i)
        if (res[i].cell_steps_per_s > res[bi].cell_steps_per_s) bi = i;
    *best = res[bi];
    if (all)
        for (size_t i = 0; i < res.size(); ++i) all[i] = res[i];
    if (n_all) *n_all = (int)res.size();
    return GPE_OK;
}
