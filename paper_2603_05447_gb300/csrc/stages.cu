// stages.cu -- multi-stage potential ramps (Sec. V): each stage blends two
// precomputed potentials linearly in time; at the start of each stage the
// region of interest is selected again from the Thomas-Fermi chemical
// potentials of the stage's endpoints, and the wavefunction is remapped from
// the previous stage's grid.  Host orchestration of the library's own calls.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>

#include "gpe_internal.cuh"

using namespace gpe;

namespace {

bool is_analytic(const gpe_ramp_pot &P) { return P.analytic != nullptr; }

int tf_mu_of(const gpe_box &box, const gpe_ramp_pot &P, double g, double N, double *mu, gpe_stream s)
{
    if (is_analytic(P)) return gpe_tf_mu_analytic(&box, P.analytic, g, N, mu, s);
    return gpe_tf_mu_dense(&box, P.V, P.V_dtype, P.V_on_device, g, N, mu, s);
}

// Grid of one stage: the union {A < cut} U {B < cut} (slots A, B), or
// {A < cut} alone (slot A) for the hold.
int stage_grid(const gpe_box &box, const gpe_ramp_pot &A, const gpe_ramp_pot *B, double cut,
               const gpe_grid_opts &o, gpe_grid **out, gpe_stream s)
{
    if (is_analytic(A)) {
        if (!B) return gpe_grid_create_analytic(&box, A.analytic, cut, &o, out, s);
        return gpe_grid_create_blend(&box, A.analytic, cut, B->analytic, cut, &o, out, s);
    }
    if (!B) return gpe_grid_create_dense(&box, A.V, A.V_dtype, A.V_on_device, cut, &o, out, s);
    return gpe_grid_create_blend_dense(&box, A.V, B->V, A.V_dtype, A.V_on_device, cut, cut, &o, out, s);
}

gpe_grid_opts opts_of(const gpe_grid *g)
{
    gpe_grid_opts o{};
    o.bx = g->bx;
    o.by = g->by;
    o.bz = g->bz;
    o.mask_mode = g->mask_mode;
    o.order = g->order;
    o.sched = g->sched;
    o.chunk = g->cb;
    o.stencil = g->stencil;
    return o;
}

}  // namespace

extern "C" int gpe_ramp_stages(const gpe_state *psi0, const gpe_ramp_pot *pots, int n_pots,
                               const double *durations, const gpe_stage_params *p,
                               const gpe_grid_opts *opts, gpe_grid **grid_out, gpe_state **state_out,
                               gpe_stage_report *report, gpe_stream stream)
{
    if (!grid_out || !state_out) return fail(GPE_ERR_ARG, "grid_out / state_out is NULL");
    *grid_out = nullptr;
    *state_out = nullptr;
    if (!psi0 || !psi0->grid || !pots || !p || !durations) return fail(GPE_ERR_ARG, "NULL argument");
    if (n_pots < 2) return fail(GPE_ERR_ARG, "a ramp needs at least two potentials");
    if (psi0->dtype != GPE_C64 && psi0->dtype != GPE_C128)
        return fail(GPE_ERR_ARG, "ramp stages need a complex state");
    if (!(std::isfinite(p->dt) && p->dt > 0.0)) return fail(GPE_ERR_ARG, "dt must be finite and > 0");
    if (!(std::isfinite(p->cut_factor) && p->cut_factor > 0.0)) return fail(GPE_ERR_ARG, "cut_factor must be > 0");
    if (!(std::isfinite(p->t_hold) && p->t_hold >= 0.0)) return fail(GPE_ERR_ARG, "t_hold must be >= 0");
    if (!(std::isfinite(p->N) && p->N > 0.0) || !std::isfinite(p->g)) return fail(GPE_ERR_ARG, "bad g or N");
    for (int i = 0; i + 1 < n_pots; ++i)
        if (!(std::isfinite(durations[i]) && durations[i] > 0.0))
            return fail(GPE_ERR_ARG, "durations[%d] must be finite and > 0", i);
    for (int i = 0; i < n_pots; ++i) {
        const gpe_ramp_pot &P = pots[i];
        if (!is_analytic(P) && !P.V) return fail(GPE_ERR_ARG, "pots[%d] has neither an analytic form nor V", i);
        if (is_analytic(P) != is_analytic(pots[0]))
            return fail(GPE_ERR_ARG, "the potentials must be all analytic or all dense");
        if (!is_analytic(P) && (P.V_dtype != pots[0].V_dtype || P.V_on_device != pots[0].V_on_device))
            return fail(GPE_ERR_ARG, "dense potentials must share V_dtype and V_on_device");
    }
    const gpe_grid_opts o = opts ? *opts : opts_of(psi0->grid);
    const gpe_box box = psi0->grid->box;

    // Thomas-Fermi chemical potential of every potential (Eq. (5))
    std::vector<double> mu(n_pots);
    for (int i = 0; i < n_pots; ++i) GPE_TRY(tf_mu_of(box, pots[i], p->g, p->N, &mu[i], stream));

    gpe_grid *cur_g = nullptr;
    gpe_state *cur_s = nullptr;
    auto drop = [&]() {
        if (cur_s) gpe_state_destroy(cur_s);
        if (cur_g) gpe_grid_destroy(cur_g);
        cur_s = nullptr;
        cur_g = nullptr;
    };
    const int n_stages = n_pots - 1 + (p->t_hold > 0.0 ? 1 : 0);
    for (int i = 0; i < n_stages; ++i) {
        const bool hold = i == n_pots - 1;
        const gpe_ramp_pot &A = pots[hold ? n_pots - 1 : i];
        const gpe_ramp_pot *B = hold ? nullptr : &pots[i + 1];
        const double mu_a = mu[hold ? n_pots - 1 : i], mu_b = hold ? mu_a : mu[i + 1];
        const double cut = p->cut_factor * std::max(mu_a, mu_b);

        // select the region again and carry the wavefunction over
        const auto t_regrid = std::chrono::steady_clock::now();
        gpe_grid *ng = nullptr;
        gpe_state *ns = nullptr;
        int rc = stage_grid(box, A, B, cut, o, &ng, stream);
        if (rc == GPE_OK) rc = gpe_state_create(ng, psi0->dtype, &ns);
        if (rc == GPE_OK) rc = gpe_state_remap(ns, cur_s ? cur_s : psi0, stream);
        if (rc != GPE_OK) {
            if (ns) gpe_state_destroy(ns);
            if (ng) gpe_grid_destroy(ng);
            drop();
            return rc;
        }
        drop();  // the previous stage's state and grid are no longer needed
        cur_g = ng;
        cur_s = ns;

        gpe_obs ob{};
        if (report) {
            const cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
            if (e != cudaSuccess) {
                drop();
                return cuda_fail(e, "cudaStreamSynchronize", __FILE__, __LINE__);
            }
            report[i].regrid_s =
                std::chrono::duration<double>(std::chrono::steady_clock::now() - t_regrid).count();
            rc = gpe_observables(cur_s, p->g, 0.0, &ob, stream);
            if (rc != GPE_OK) {
                drop();
                return rc;
            }
            report[i].norm_kept = ob.norm;
        }

        // the stage's real-time steps: equal steps of at most dt covering
        // the duration, V(t) blended linearly from A (t = 0) to B (t = d)
        const double d = hold ? p->t_hold : durations[i];
        const int64_t n = std::max<int64_t>(1, (int64_t)std::ceil(d / p->dt * (1.0 - 1e-12)));
        gpe_real_params rp{};
        rp.g = p->g;
        rp.dt = d / (double)n;
        rp.integrator = p->integrator;
        if (hold) {
            rp.potential = GPE_V_STATIC;
        } else {
            rp.potential = GPE_V_BLEND;
            rp.n_knots = 2;
            rp.T_ramp = d;
            rp.knots[0] = 0.0;
            rp.knots[1] = 1.0;
        }
        rc = gpe_step_real(cur_s, &rp, n, 0.0, stream);
        if (rc == GPE_OK && report) rc = gpe_observables(cur_s, p->g, hold ? 0.0 : 1.0, &ob, stream);
        if (rc != GPE_OK) {
            drop();
            return rc;
        }
        if (report) {
            report[i].mu_a = mu_a;
            report[i].mu_b = mu_b;
            report[i].cut = cut;
            report[i].n_active = cur_g->n_active;
            report[i].steps = n;
            report[i].dt = rp.dt;
            report[i].norm_end = ob.norm;
        }
    }
    if (!report) {
        // the steps are asynchronous: report their errors here
        const cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
        if (e != cudaSuccess) {
            drop();
            return cuda_fail(e, "cudaStreamSynchronize", __FILE__, __LINE__);
        }
    }
    *grid_out = cur_g;
    *state_out = cur_s;
    return GPE_OK;
}
