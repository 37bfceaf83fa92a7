// trace.cu -- real-time steps with an observables trace at a cadence (the
// norm, energy and chemical potential of a run over time).  Host
// orchestration of the library's own step and reduction calls.
#include <algorithm>
#include <cmath>

#include "gpe_internal.cuh"

using namespace gpe;

namespace {

// s(t) of a ramp: piecewise linear through the knots at uniform times on
// [0, T], held constant outside (the blend between potentials of Sec. V)
double ramp_fraction(const gpe_real_params &p, double t)
{
    if (p.potential != GPE_V_BLEND) return 0.0;
    if (t <= 0.0) return p.knots[0];
    if (t >= p.T_ramp) return p.knots[p.n_knots - 1];
    const double u = t / p.T_ramp * (double)(p.n_knots - 1);
    int k = (int)std::floor(u);
    if (k >= p.n_knots - 1) k = p.n_knots - 2;
    const double w = u - (double)k;
    return (1.0 - w) * p.knots[k] + w * p.knots[k + 1];
}

}  // namespace

extern "C" int gpe_step_real_traced(gpe_state *st, const gpe_real_params *p, int64_t nsteps, double t0,
                                    int64_t every, gpe_obs *log, int64_t *n_logged, gpe_stream stream)
{
    if (!p || !log || !n_logged) return fail(GPE_ERR_ARG, "NULL argument");
    *n_logged = 0;
    if (nsteps < 0) return fail(GPE_ERR_ARG, "nsteps < 0");
    if (every < 1) return fail(GPE_ERR_ARG, "every must be >= 1");
    if (p->potential == GPE_V_BLEND && (p->n_knots < 2 || p->n_knots > GPE_MAX_KNOTS))
        return fail(GPE_ERR_ARG, "n_knots must be in [2, 16]");
    int64_t done = 0;
    while (done < nsteps) {
        const int64_t n = std::min(every, nsteps - done);
        GPE_TRY(gpe_step_real(st, p, n, t0 + (double)done * p->dt, stream));
        done += n;
        const double t = t0 + (double)done * p->dt;
        const int rc = gpe_observables(st, p->g, ramp_fraction(*p, t), &log[*n_logged], stream);
        if (rc != GPE_OK && rc != GPE_ERR_NONFINITE) return rc;
        ++*n_logged;
        if (rc == GPE_ERR_NONFINITE) return rc;
    }
    return GPE_OK;
}
