// step19.cu -- the step drivers of 19-point grids (App. B's higher-order
// compact Laplacian): RK4 (stages of App. A), imaginary time and the
// observables, staged schedule, one launch per stage.  A separate
// translation unit so that the 19-point kernel instances build in parallel
// with the 7-point ones.
#include <algorithm>

#include "kernels.cuh"

namespace gpe {

namespace {

__global__ void k_set_scalar19(double *p, double v) { *p = v; }

// resident blocks over all SMs, at most one warp per brick
template <typename K>
int grid_blocks(K kernel, const gpe_grid *g, size_t smem, int nw)
{
    const int per = prepare_kernel(kernel, 32 * nw, smem);
    const int64_t need = (g->nb + nw - 1) / nw;
    return (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)g->nsm * per, need));
}

template <typename R, int BX, int BY, int BZ>
int rk4_19(gpe_state *st, const gpe_real_params *p, int64_t nsteps, double t0, cudaStream_t s)
{
    using CT = typename Cx<R>::T;
    const gpe_grid *g = st->grid;
    const bool blend = p->potential == GPE_V_BLEND;
    RkArgs<R> a{};
    a.V0 = (const R *)potential_ptr(st, 0);
    a.V1 = blend ? (const R *)potential_ptr(st, 1) : nullptr;
    if (!a.V0 || (blend && !a.V1)) return fail(GPE_ERR_STATE, "potential slot missing");
    a.y0 = (CT *)st->d_psi;
    a.y2 = (CT *)st->d_work[0];
    a.y3 = (CT *)st->d_work[1];
    a.y4 = (CT *)st->d_work[0];  // y2 is dead once stage 1 is done
    a.w = (CT *)st->d_work[2];
    a.ihx2 = (R)(1.0 / (g->box.hx * g->box.hx));
    a.ihy2 = (R)(1.0 / (g->box.hy * g->box.hy));
    a.ihz2 = (R)(1.0 / (g->box.hz * g->box.hz));
    a.g = (R)p->g;
    a.dt = (R)p->dt;
    a.dtd = p->dt;
    a.ramp.clock = st->d_clock;
    a.ramp.T = p->T_ramp;
    a.ramp.n_knots = p->n_knots;
    for (int k = 0; k < GPE_MAX_KNOTS; ++k) a.ramp.knots[k] = p->knots[k];
    if (blend) {
        k_set_scalar19<<<1, 1, 0, s>>>(st->d_clock, t0);
        GPE_LAUNCH_CHECK();
    }
    using RS = Rk4Stages<R, BX, BY, BZ, 19>;
    typename RS::K k[4];
    int nblk[4];
    for (int stg = 0; stg < 4; ++stg) {
        k[stg] = RS::get(blend, stg);
        nblk[stg] = grid_blocks(k[stg], g, RS::smem(), RS::NW);
    }
    const GridView G = view(g);
    for (int64_t n = 0; n < nsteps; ++n) {
        a.t_off = (double)n * p->dt;
        for (int stg = 0; stg < 4; ++stg) {
            k[stg]<<<nblk[stg], RS::THREADS, RS::smem(), s>>>(a, G);
            GPE_LAUNCH_CHECK();
        }
    }
    return GPE_OK;
}

template <typename R, int BX, int BY, int BZ, typename CT>
int itp_19(gpe_state *st, const gpe_imag_params *p, int64_t nsteps, cudaStream_t s)
{
    const gpe_grid *g = st->grid;
    if (st->E_dt != p->dt) {
        k_make_E<R><<<g->nsm * 8, 256, 0, s>>>(g->d_V[0], (R *)st->d_E, g->n_packed, p->dt);
        GPE_LAUNCH_CHECK();
        st->E_dt = p->dt;
    }
    ItpArgs<R, CT> a{};
    a.psi = (CT *)st->d_psi;
    a.tmp = (CT *)st->d_work[0];
    a.E = (const R *)st->d_E;
    a.ihx2 = (R)(1.0 / (g->box.hx * g->box.hx));
    a.ihy2 = (R)(1.0 / (g->box.hy * g->box.hy));
    a.ihz2 = (R)(1.0 / (g->box.hz * g->box.hz));
    a.g = (R)p->g;
    a.dt = (R)p->dt;
    a.scalars = st->red.scalars;
    a.N = p->N;
    a.dV = g->box.hx * g->box.hy * g->box.hz;
    k_set_scalar19<<<1, 1, 0, s>>>(st->red.scalars, 1.0);
    GPE_LAUNCH_CHECK();
    const GridView G = view(g);
    const int th = KernelCfg<R>::THREADS;
    const size_t smem = smem_bytes<R, BX, BY, BZ, CT, 19>();
    auto ka = k_itp_a<R, BX, BY, BZ, CT, 19>;
    auto kb = k_itp_b<R, BX, BY, BZ, CT, 19>;
    const int nba = grid_blocks(ka, g, smem, KernelCfg<R>::NW), nbb = grid_blocks(kb, g, smem, KernelCfg<R>::NW);
    for (int64_t n = 0; n < nsteps; ++n) {
        ka<<<nba, th, smem, s>>>(a, G);
        GPE_LAUNCH_CHECK();
        kb<<<nbb, th, smem, s>>>(a, G, st->red.partials, st->red.counter);
        GPE_LAUNCH_CHECK();
    }
    k_apply_scale<CT><<<g->nsm * 8, 256, 0, s>>>((CT *)st->d_psi, g->n_packed, st->red.scalars);
    GPE_LAUNCH_CHECK();
    return GPE_OK;
}

template <typename R, int BX, int BY, int BZ, typename CT>
int obs_19(const gpe_state *stc, double gg, double sb, cudaStream_t s)
{
    gpe_state *st = const_cast<gpe_state *>(stc);
    const gpe_grid *g = st->grid;
    ObsArgs<R, CT> a{};
    a.psi = (const CT *)st->d_psi;
    a.V0 = (const R *)potential_ptr(st, 0);
    a.V1 = (sb != 0.0) ? (const R *)potential_ptr(st, 1) : nullptr;
    if (sb != 0.0 && !a.V1) return fail(GPE_ERR_ARG, "s_blend != 0 needs potential slot 1");
    a.s = (R)sb;
    a.ihx2 = (R)(1.0 / (g->box.hx * g->box.hx));
    a.ihy2 = (R)(1.0 / (g->box.hy * g->box.hy));
    a.ihz2 = (R)(1.0 / (g->box.hz * g->box.hz));
    a.g = (R)gg;
    a.dV = g->box.hx * g->box.hy * g->box.hz;
    a.partials = st->red.partials;
    a.counter = st->red.counter;
    a.out = (gpe_obs *)(st->red.scalars + 2);
    const size_t smem = smem_bytes<R, BX, BY, BZ, CT, 19>();
    auto k = k_obs<R, BX, BY, BZ, CT, 19>;
    k<<<grid_blocks(k, g, smem, KernelCfg<R>::NW), KernelCfg<R>::THREADS, smem, s>>>(a, view(g));
    GPE_LAUNCH_CHECK();
    return GPE_OK;
}

}  // namespace

int rk4_run19(gpe_state *st, const gpe_real_params *p, int64_t nsteps, double t0, cudaStream_t s)
{
    const bool c128 = st->dtype == GPE_C128;
#define RK19(id, X, Y, Z) \
    case id: return c128 ? rk4_19<double, X, Y, Z>(st, p, nsteps, t0, s) : rk4_19<float, X, Y, Z>(st, p, nsteps, t0, s);
    switch (st->grid->shape) { GPE_SHAPES(RK19) }
#undef RK19
    return fail(GPE_ERR_STATE, "bad brick shape");
}

int itp_run19(gpe_state *st, const gpe_imag_params *p, int64_t nsteps, cudaStream_t s)
{
    const int dt_ = st->dtype;
#define ITP19(id, X, Y, Z)                                                      \
    case id:                                                                    \
        switch (dt_) {                                                          \
        case GPE_C128: return itp_19<double, X, Y, Z, double2>(st, p, nsteps, s); \
        case GPE_C64: return itp_19<float, X, Y, Z, float2>(st, p, nsteps, s);    \
        case GPE_R64: return itp_19<double, X, Y, Z, double>(st, p, nsteps, s);   \
        default: return itp_19<float, X, Y, Z, float>(st, p, nsteps, s);          \
        }
    switch (st->grid->shape) { GPE_SHAPES(ITP19) }
#undef ITP19
    return fail(GPE_ERR_STATE, "bad brick shape");
}

int obs_run19(const gpe_state *st, double g, double s_blend, cudaStream_t s)
{
    const int dt_ = st->dtype;
#define OBS19(id, X, Y, Z)                                                       \
    case id:                                                                     \
        switch (dt_) {                                                           \
        case GPE_C128: return obs_19<double, X, Y, Z, double2>(st, g, s_blend, s); \
        case GPE_C64: return obs_19<float, X, Y, Z, float2>(st, g, s_blend, s);    \
        case GPE_R64: return obs_19<double, X, Y, Z, double>(st, g, s_blend, s);   \
        default: return obs_19<float, X, Y, Z, float>(st, g, s_blend, s);          \
        }
    switch (st->grid->shape) { GPE_SHAPES(OBS19) }
#undef OBS19
    return fail(GPE_ERR_STATE, "bad brick shape");
}

}  // namespace gpe
