// step.cu -- wavefunction states, the real-time RK4 step, the imaginary-time
// split step with renormalisation, and the FP64 observables of libgpeshell.
//
// Every stencil kernel stages one brick plus its face halo in shared memory
// (the paper's per-block tile of Sec. II B, gathered here from the six face
// neighbours through the brick-neighbour table), evaluates the 7-point
// Laplacian of Eq. (B1) from the tile, applies the pointwise terms of the
// equation and writes only active cells.  Blocks walk the brick list with a
// fixed stride (block b handles bricks b, b + gridDim, ...), so per-block
// partial sums, and therefore every FP64 reduction, are deterministic.
#include <cmath>
#include <mutex>
#include <unordered_map>

#include "gpe_internal.cuh"

namespace gpe {

// ------------------------------------------------------------ small kernels
__global__ void k_d2f(const double *s, float *d, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        d[i] = (float)s[i];
}

int convert_to_float(const double *src, float *dst, int64_t n)
{
    k_d2f<<<1024, 256>>>(src, dst, n);
    GPE_LAUNCH_CHECK();
    GPE_TRY_CUDA(cudaStreamSynchronize(0));
    return GPE_OK;
}

__global__ void k_set_scalar(double *p, double v) { *p = v; }
__global__ void k_add_scalar(double *p, double v) { *p += v; }

// E = exp(-V dt/2) in the state precision (Eq. (7): the diagonal propagator
// is precomputed once per dt)
template <typename R>
__global__ void k_make_E(const double *V, R *E, int64_t n, double dt)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        E[i] = (R)exp(-V[i] * dt / 2.0);
}

// ------------------------------------------------------------ launch helper
static std::mutex g_occ_mu;
static std::unordered_map<const void *, int> g_occ;

template <typename K>
static int blocks_for(K kernel, const gpe_grid *g, int threads)
{
    int per_sm = 0;
    {
        std::lock_guard<std::mutex> lk(g_occ_mu);
        auto it = g_occ.find((const void *)kernel);
        if (it != g_occ.end()) per_sm = it->second;
    }
    if (per_sm == 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess || per_sm < 1) {
            cudaGetLastError();
            per_sm = 1;
        }
        std::lock_guard<std::mutex> lk(g_occ_mu);
        g_occ[(const void *)kernel] = per_sm;
    }
    int64_t b = (int64_t)g->nsm * per_sm;
    if (b > g->nb) b = g->nb;
    if (b < 1) b = 1;
    return (int)b;
}

static inline int brick_threads(const gpe_grid *g) { return g->bc < 256 ? g->bc : 256; }

#define GPE_SHAPES(M) \
    M(0, 8, 8, 8)     \
    M(1, 8, 8, 4)     \
    M(2, 8, 4, 4)     \
    M(3, 4, 4, 4)

// ------------------------------------------------------------ ramp schedule
struct Ramp {
    const double *clock;  // device time base
    double t_off;         // stage time = *clock + t_off
    double T;
    int n_knots;
    double knots[GPE_MAX_KNOTS];
};

// s(t): piecewise linear through n_knots values at t_k = k T/(n_knots-1),
// held constant outside [0, T] (linear interpolation between potentials, Sec. V)
__device__ __forceinline__ double ramp_s(const Ramp &r, double t)
{
    if (t <= 0.0) return r.knots[0];
    if (t >= r.T) return r.knots[r.n_knots - 1];
    double u = t / r.T * (double)(r.n_knots - 1);
    int k = (int)floor(u);
    if (k >= r.n_knots - 1) k = r.n_knots - 2;
    double w = u - (double)k;
    return (1.0 - w) * r.knots[k] + w * r.knots[k + 1];
}

// ------------------------------------------------------------ RK4 stages
// Memory-optimised RK4 (App. A, RK4 a* and b*): the stage states are stored
// instead of the k_i, so stage i reads only the state it differentiates (with
// halo) plus the own-cell values of earlier states:
//   ST1: y2 = y0 + dt/2 f(t, y0)
//   ST2: y3 = y0 + dt/2 f(t + dt/2, y2)
//   ST3: y4 = y0 + dt   f(t + dt/2, y3)
//   ST4: y1 = (-y0 + y2 + 2 y3 + y4)/3 + dt/6 f(t + dt, y4)   (in place of y0)
// with f(t, y) = -i [ -1/2 lap y + (V(t) + g|y|^2) y ]  (Eq. (8)).
template <typename R>
struct RkArgs {
    using CT = typename Cx<R>::T;
    const CT *yin;
    const CT *y0;
    const CT *y2;
    const CT *y3;
    CT *yout;
    const R *V0;
    const R *V1;
    const int32_t *nbr;
    const uint32_t *mask;
    int64_t nb;
    R ihx2, ihy2, ihz2, g, dt;
    Ramp ramp;
};

template <typename R, int BX, int BY, int BZ, int ST, bool BLEND>
__global__ void __launch_bounds__(256) k_rk4(const RkArgs<R> a)
{
    using B = Brick<BX, BY, BZ>;
    using CT = typename Cx<R>::T;
    __shared__ CT tile[B::TN];
    R s = 0;
    if (BLEND) s = (R)ramp_s(a.ramp, *a.ramp.clock + a.ramp.t_off);
    const R c = (ST == 3) ? a.dt : (ST == 4 ? a.dt / (R)6 : a.dt / (R)2);
    for (int64_t b = blockIdx.x; b < a.nb; b += gridDim.x) {
        load_tile<BX, BY, BZ>(tile, a.yin, b, a.nbr, a.mask, [](CT v, int64_t) { return v; });
        __syncthreads();
        for (int l = threadIdx.x; l < B::BC; l += blockDim.x) {
            const int64_t slot = b * B::BC + l;
            if (!mask_bit(a.mask, slot)) continue;
            const int x = l % BX, y = (l / BX) % BY, z = l / (BX * BY);
            const CT L = tile_laplacian<BX, BY, BZ, R>(tile, x, y, z, a.ihx2, a.ihy2, a.ihz2);
            const CT yc = tile[B::t(x, y, z)];
            R V;
            if (BLEND) V = ((R)1 - s) * a.V0[slot] + s * a.V1[slot];
            else V = a.V0[slot];
            const R w = V + a.g * (yc.x * yc.x + yc.y * yc.y);
            const R hr = (R)(-0.5) * L.x + w * yc.x;
            const R hi = (R)(-0.5) * L.y + w * yc.y;
            CT o;  // f = -i (hr + i hi) = hi - i hr
            if (ST == 1) {
                o.x = yc.x + c * hi;
                o.y = yc.y - c * hr;
            } else if (ST < 4) {
                const CT y0 = a.y0[slot];
                o.x = y0.x + c * hi;
                o.y = y0.y - c * hr;
            } else {
                const CT y0 = a.y0[slot], y2 = a.y2[slot], y3 = a.y3[slot];
                o.x = (-y0.x + y2.x + (R)2 * y3.x + yc.x) / (R)3 + c * hi;
                o.y = (-y0.y + y2.y + (R)2 * y3.y + yc.y) / (R)3 - c * hr;
            }
            a.yout[slot] = o;
        }
        __syncthreads();
    }
}

template <typename R, int BX, int BY, int BZ, int ST>
static int launch_rk4(const gpe_grid *g, const RkArgs<R> &a, bool blend, cudaStream_t s)
{
    const int th = brick_threads(g);
    if (blend) {
        auto k = k_rk4<R, BX, BY, BZ, ST, true>;
        k<<<blocks_for(k, g, th), th, 0, s>>>(a);
    } else {
        auto k = k_rk4<R, BX, BY, BZ, ST, false>;
        k<<<blocks_for(k, g, th), th, 0, s>>>(a);
    }
    GPE_LAUNCH_CHECK();
    return GPE_OK;
}

template <typename R, int BX, int BY, int BZ>
static int rk4_run(gpe_state *st, const gpe_real_params *p, int64_t nsteps, double t0, cudaStream_t s)
{
    using CT = typename Cx<R>::T;
    const gpe_grid *g = st->grid;
    const bool blend = p->potential == GPE_V_BLEND;
    RkArgs<R> a{};
    a.V0 = (const R *)potential_ptr(st, 0);
    a.V1 = blend ? (const R *)potential_ptr(st, 1) : nullptr;
    if (!a.V0 || (blend && !a.V1)) return fail(GPE_ERR_STATE, "potential slot missing");
    a.nbr = g->d_nbr;
    a.mask = g->d_mask;
    a.nb = g->nb;
    a.ihx2 = (R)(1.0 / (g->box.hx * g->box.hx));
    a.ihy2 = (R)(1.0 / (g->box.hy * g->box.hy));
    a.ihz2 = (R)(1.0 / (g->box.hz * g->box.hz));
    a.g = (R)p->g;
    a.dt = (R)p->dt;
    a.ramp.clock = st->d_clock;
    a.ramp.T = p->T_ramp;
    a.ramp.n_knots = p->n_knots;
    for (int k = 0; k < GPE_MAX_KNOTS; ++k) a.ramp.knots[k] = p->knots[k];
    CT *psi = (CT *)st->d_psi, *w0 = (CT *)st->d_work[0], *w1 = (CT *)st->d_work[1], *w2 = (CT *)st->d_work[2];
    if (blend) {
        k_set_scalar<<<1, 1, 0, s>>>(st->d_clock, t0);
        GPE_LAUNCH_CHECK();
    }
    const double dt = p->dt;
    for (int64_t n = 0; n < nsteps; ++n) {
        const double tn = (double)n * dt;
        a.yin = psi; a.y0 = psi; a.yout = w0; a.ramp.t_off = tn;
        GPE_TRY((launch_rk4<R, BX, BY, BZ, 1>(g, a, blend, s)));
        a.yin = w0; a.yout = w1; a.ramp.t_off = tn + 0.5 * dt;
        GPE_TRY((launch_rk4<R, BX, BY, BZ, 2>(g, a, blend, s)));
        a.yin = w1; a.yout = w2; a.ramp.t_off = tn + 0.5 * dt;
        GPE_TRY((launch_rk4<R, BX, BY, BZ, 3>(g, a, blend, s)));
        a.yin = w2; a.y2 = w0; a.y3 = w1; a.yout = psi; a.ramp.t_off = tn + dt;
        GPE_TRY((launch_rk4<R, BX, BY, BZ, 4>(g, a, blend, s)));
    }
    return GPE_OK;
}

// ------------------------------------------------------------ imaginary time
// Sec. II A/B, Eqs. (6)-(7).  K-ITP-A stages psi with its halo, applying on
// load the pending renormalisation factor and the diagonal half step
// psi * E * (1 - g|psi|^2 dt/2), E = exp(-V dt/2); then the first Euler
// kinetic substep psi - (dt/2) T psi = psi + (dt/4) lap psi -> tmp.
// K-ITP-B stages tmp, takes the second Euler substep, applies the diagonal
// half step again, writes psi and reduces sum |psi|^2 in FP64; the last block
// stores the next factor sqrt(N / (sum |psi|^2 dV)).
template <typename R>
struct ItpArgs {
    using CT = typename Cx<R>::T;
    const CT *in;
    CT *out;
    const R *E;
    const int32_t *nbr;
    const uint32_t *mask;
    int64_t nb;
    R ihx2, ihy2, ihz2, g, dt;
    double *scalars;  // [0] scale to apply on load / next scale, [1] last norm
    double *partials;
    unsigned int *counter;
    double N, dV;
};

template <typename R, int BX, int BY, int BZ>
__global__ void __launch_bounds__(256) k_itp_a(const ItpArgs<R> a)
{
    using B = Brick<BX, BY, BZ>;
    using CT = typename Cx<R>::T;
    __shared__ CT tile[B::TN];
    const R sc = (R)a.scalars[0];
    const R hg = a.g * a.dt / (R)2;
    const R q = a.dt / (R)4;
    const R *E = a.E;
    auto diag = [sc, hg, E](CT v, int64_t s) {
        v.x *= sc;
        v.y *= sc;
        const R f = E[s] * ((R)1 - hg * (v.x * v.x + v.y * v.y));
        v.x *= f;
        v.y *= f;
        return v;
    };
    for (int64_t b = blockIdx.x; b < a.nb; b += gridDim.x) {
        load_tile<BX, BY, BZ>(tile, a.in, b, a.nbr, a.mask, diag);
        __syncthreads();
        for (int l = threadIdx.x; l < B::BC; l += blockDim.x) {
            const int64_t slot = b * B::BC + l;
            if (!mask_bit(a.mask, slot)) continue;
            const int x = l % BX, y = (l / BX) % BY, z = l / (BX * BY);
            const CT L = tile_laplacian<BX, BY, BZ, R>(tile, x, y, z, a.ihx2, a.ihy2, a.ihz2);
            const CT yc = tile[B::t(x, y, z)];
            CT o;
            o.x = yc.x + q * L.x;
            o.y = yc.y + q * L.y;
            a.out[slot] = o;
        }
        __syncthreads();
    }
}

template <typename R, int BX, int BY, int BZ>
__global__ void __launch_bounds__(256) k_itp_b(const ItpArgs<R> a)
{
    using B = Brick<BX, BY, BZ>;
    using CT = typename Cx<R>::T;
    __shared__ CT tile[B::TN];
    const R hg = a.g * a.dt / (R)2;
    const R q = a.dt / (R)4;
    double acc[1] = {0.0};
    for (int64_t b = blockIdx.x; b < a.nb; b += gridDim.x) {
        load_tile<BX, BY, BZ>(tile, a.in, b, a.nbr, a.mask, [](CT v, int64_t) { return v; });
        __syncthreads();
        for (int l = threadIdx.x; l < B::BC; l += blockDim.x) {
            const int64_t slot = b * B::BC + l;
            if (!mask_bit(a.mask, slot)) continue;
            const int x = l % BX, y = (l / BX) % BY, z = l / (BX * BY);
            const CT L = tile_laplacian<BX, BY, BZ, R>(tile, x, y, z, a.ihx2, a.ihy2, a.ihz2);
            const CT yc = tile[B::t(x, y, z)];
            CT o;
            o.x = yc.x + q * L.x;
            o.y = yc.y + q * L.y;
            const R f = a.E[slot] * ((R)1 - hg * (o.x * o.x + o.y * o.y));
            o.x *= f;
            o.y *= f;
            a.out[slot] = o;
            acc[0] += (double)(o.x * o.x + o.y * o.y);
        }
        __syncthreads();
    }
    double tot[1];
    if (reduce_finish<1>(acc, a.partials, a.counter, tot) && threadIdx.x == 0) {
        const double nrm = tot[0] * a.dV;
        a.scalars[0] = sqrt(a.N / nrm);
        a.scalars[1] = nrm;
    }
}

template <typename CT>
__global__ void k_apply_scale(CT *psi, const uint32_t *mask, int64_t ns, const double *scalars)
{
    const double sc = scalars[0];
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < ns; s += (int64_t)gridDim.x * blockDim.x) {
        if ((mask[s >> 5] >> (s & 31)) & 1u) {
            CT v = psi[s];
            v.x = v.x * sc;
            v.y = v.y * sc;
            psi[s] = v;
        }
    }
}

template <typename R, int BX, int BY, int BZ>
static int itp_run(gpe_state *st, const gpe_imag_params *p, int64_t nsteps, cudaStream_t s)
{
    using CT = typename Cx<R>::T;
    const gpe_grid *g = st->grid;
    if (st->E_dt != p->dt) {
        k_make_E<R><<<g->nsm * 8, 256, 0, s>>>(g->d_V[0], (R *)st->d_E, g->n_stored, p->dt);
        GPE_LAUNCH_CHECK();
        st->E_dt = p->dt;
    }
    ItpArgs<R> a{};
    a.E = (const R *)st->d_E;
    a.nbr = g->d_nbr;
    a.mask = g->d_mask;
    a.nb = g->nb;
    a.ihx2 = (R)(1.0 / (g->box.hx * g->box.hx));
    a.ihy2 = (R)(1.0 / (g->box.hy * g->box.hy));
    a.ihz2 = (R)(1.0 / (g->box.hz * g->box.hz));
    a.g = (R)p->g;
    a.dt = (R)p->dt;
    a.scalars = st->red.scalars;
    a.partials = st->red.partials;
    a.counter = st->red.counter;
    a.N = p->N;
    a.dV = g->box.hx * g->box.hy * g->box.hz;
    CT *psi = (CT *)st->d_psi, *tmp = (CT *)st->d_work[0];
    k_set_scalar<<<1, 1, 0, s>>>(st->red.scalars, 1.0);
    GPE_LAUNCH_CHECK();
    const int th = brick_threads(g);
    auto ka = k_itp_a<R, BX, BY, BZ>;
    auto kb = k_itp_b<R, BX, BY, BZ>;
    const int nba = blocks_for(ka, g, th), nbb = blocks_for(kb, g, th);
    for (int64_t n = 0; n < nsteps; ++n) {
        a.in = psi;
        a.out = tmp;
        ka<<<nba, th, 0, s>>>(a);
        GPE_LAUNCH_CHECK();
        a.in = tmp;
        a.out = psi;
        kb<<<nbb, th, 0, s>>>(a);
        GPE_LAUNCH_CHECK();
    }
    if (nsteps > 0) {
        k_apply_scale<CT><<<g->nsm * 8, 256, 0, s>>>(psi, g->d_mask, g->n_stored, st->red.scalars);
        GPE_LAUNCH_CHECK();
    }
    return GPE_OK;
}

// ------------------------------------------------------------ observables
template <typename R>
struct ObsArgs {
    using CT = typename Cx<R>::T;
    const CT *psi;
    const R *V0;
    const R *V1;
    R s;
    const int32_t *nbr;
    const uint32_t *mask;
    int64_t nb;
    R ihx2, ihy2, ihz2, g;
    double dV;
    double *partials;
    unsigned int *counter;
    gpe_obs *out;
};

template <typename R, int BX, int BY, int BZ>
__global__ void __launch_bounds__(256) k_obs(const ObsArgs<R> a)
{
    using B = Brick<BX, BY, BZ>;
    using CT = typename Cx<R>::T;
    __shared__ CT tile[B::TN];
    double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};  // norm, ekin, epot, eint, nonfinite
    for (int64_t b = blockIdx.x; b < a.nb; b += gridDim.x) {
        load_tile<BX, BY, BZ>(tile, a.psi, b, a.nbr, a.mask, [](CT v, int64_t) { return v; });
        __syncthreads();
        for (int l = threadIdx.x; l < B::BC; l += blockDim.x) {
            const int64_t slot = b * B::BC + l;
            if (!mask_bit(a.mask, slot)) continue;
            const int x = l % BX, y = (l / BX) % BY, z = l / (BX * BY);
            const CT L = tile_laplacian<BX, BY, BZ, R>(tile, x, y, z, a.ihx2, a.ihy2, a.ihz2);
            const CT yc = tile[B::t(x, y, z)];
            const R V = a.V1 ? ((R)1 - a.s) * a.V0[slot] + a.s * a.V1[slot] : a.V0[slot];
            const R rho = yc.x * yc.x + yc.y * yc.y;
            acc[0] += (double)rho;
            acc[1] += (double)((R)(-0.5) * (yc.x * L.x + yc.y * L.y));
            acc[2] += (double)(V * rho);
            acc[3] += (double)((R)0.5 * a.g * rho * rho);
            acc[4] += (isfinite(yc.x) && isfinite(yc.y)) ? 0.0 : 1.0;
        }
        __syncthreads();
    }
    double tot[5];
    if (reduce_finish<5>(acc, a.partials, a.counter, tot) && threadIdx.x == 0) {
        gpe_obs o;
        o.norm = tot[0] * a.dV;
        o.e_kin = tot[1] * a.dV;
        o.e_pot = tot[2] * a.dV;
        o.e_int = tot[3] * a.dV;
        o.energy = o.e_kin + o.e_pot + o.e_int;
        o.mu = (o.e_kin + o.e_pot + 2.0 * o.e_int) / o.norm;
        o.nonfinite = tot[4];
        *a.out = o;
    }
}

template <typename R, int BX, int BY, int BZ>
static int obs_run(const gpe_state *stc, double gg, double sb, cudaStream_t s)
{
    gpe_state *st = const_cast<gpe_state *>(stc);
    const gpe_grid *g = st->grid;
    ObsArgs<R> a{};
    a.psi = (const typename Cx<R>::T *)st->d_psi;
    a.V0 = (const R *)potential_ptr(st, 0);
    a.V1 = (sb != 0.0) ? (const R *)potential_ptr(st, 1) : nullptr;
    if (sb != 0.0 && !a.V1) return fail(GPE_ERR_ARG, "s_blend != 0 needs potential slot 1");
    a.s = (R)sb;
    a.nbr = g->d_nbr;
    a.mask = g->d_mask;
    a.nb = g->nb;
    a.ihx2 = (R)(1.0 / (g->box.hx * g->box.hx));
    a.ihy2 = (R)(1.0 / (g->box.hy * g->box.hy));
    a.ihz2 = (R)(1.0 / (g->box.hz * g->box.hz));
    a.g = (R)gg;
    a.dV = g->box.hx * g->box.hy * g->box.hz;
    a.partials = st->red.partials;
    a.counter = st->red.counter;
    a.out = (gpe_obs *)(st->red.scalars + 2);
    const int th = brick_threads(g);
    auto k = k_obs<R, BX, BY, BZ>;
    k<<<blocks_for(k, g, th), th, 0, s>>>(a);
    GPE_LAUNCH_CHECK();
    return GPE_OK;
}

// <a|b> = sum conj(a) b dV
template <typename CT>
__global__ void k_overlap(const CT *a, const CT *b, const uint32_t *mask, int64_t ns, double dV, double *partials,
                          unsigned int *counter, double *out)
{
    double acc[2] = {0.0, 0.0};
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < ns; s += (int64_t)gridDim.x * blockDim.x) {
        if ((mask[s >> 5] >> (s & 31)) & 1u) {
            const CT u = a[s], v = b[s];
            acc[0] += (double)(u.x * v.x + u.y * v.y);
            acc[1] += (double)(u.x * v.y - u.y * v.x);
        }
    }
    double tot[2];
    if (reduce_finish<2>(acc, partials, counter, tot) && threadIdx.x == 0) {
        out[0] = tot[0] * dV;
        out[1] = tot[1] * dV;
    }
}

// ------------------------------------------------------------ load / store
struct BoxI {
    int64_t nx, ny, nz;
    int BX, BY, BZ;
};

template <typename CT>
__global__ void k_load_dense(const CT *dense, CT *psi, const int32_t *org, const uint32_t *mask, int64_t ns, BoxI b)
{
    const int BC = b.BX * b.BY * b.BZ;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < ns; s += (int64_t)gridDim.x * blockDim.x) {
        CT v;
        v.x = 0;
        v.y = 0;
        if ((mask[s >> 5] >> (s & 31)) & 1u) {
            const int64_t br = s / BC;
            const int l = (int)(s % BC);
            const int64_t i = org[3 * br] + l % b.BX, j = org[3 * br + 1] + (l / b.BX) % b.BY,
                          k = org[3 * br + 2] + l / (b.BX * b.BY);
            v = dense[i + b.nx * (j + b.ny * k)];
        }
        psi[s] = v;
    }
}

template <typename CT>
__global__ void k_store_dense(const CT *psi, CT *dense, const int32_t *org, const uint32_t *mask, int64_t ns, BoxI b)
{
    const int BC = b.BX * b.BY * b.BZ;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < ns; s += (int64_t)gridDim.x * blockDim.x) {
        if ((mask[s >> 5] >> (s & 31)) & 1u) {
            const int64_t br = s / BC;
            const int l = (int)(s % BC);
            const int64_t i = org[3 * br] + l % b.BX, j = org[3 * br + 1] + (l / b.BX) % b.BY,
                          k = org[3 * br + 2] + l / (b.BX * b.BY);
            dense[i + b.nx * (j + b.ny * k)] = psi[s];
        }
    }
}

template <typename CT>
__global__ void k_mask_compact(CT *psi, const uint32_t *mask, int64_t ns)
{
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < ns; s += (int64_t)gridDim.x * blockDim.x) {
        if (!((mask[s >> 5] >> (s & 31)) & 1u)) {
            CT v;
            v.x = 0;
            v.y = 0;
            psi[s] = v;
        }
    }
}

// ------------------------------------------------------------ state helpers
int ensure_work(gpe_state *st, int n)
{
    for (int i = 0; i < n; ++i) {
        if (st->d_work[i]) continue;
        GPE_TRY(dev_alloc(&st->d_work[i], st->grid->n_stored * st->elem));
        GPE_TRY_CUDA(cudaMemset(st->d_work[i], 0, st->grid->n_stored * st->elem));
    }
    return GPE_OK;
}

const void *potential_ptr(gpe_state *st, int slot)
{
    gpe_grid *g = st->grid;
    if (!g->d_V[slot]) return nullptr;
    if (st->dtype == GPE_C128) return g->d_V[slot];
    if (ensure_vf(g, slot) != GPE_OK) return nullptr;
    return g->d_Vf[slot];
}

static int check_state(const gpe_state *st)
{
    if (!st) return fail(GPE_ERR_ARG, "state is NULL");
    int dev = -1;
    GPE_TRY_CUDA(cudaGetDevice(&dev));
    if (dev != st->grid->device)
        return fail(GPE_ERR_STATE, "state lives on device %d but device %d is current", st->grid->device, dev);
    return GPE_OK;
}

}  // namespace gpe

using namespace gpe;

// ------------------------------------------------------------ C ABI
extern "C" int gpe_state_create(gpe_grid *g, int dtype, gpe_state **out)
{
    if (!g || !out) return fail(GPE_ERR_ARG, "NULL argument");
    *out = nullptr;
    if (dtype != GPE_C128 && dtype != GPE_C64) return fail(GPE_ERR_ARG, "dtype must be GPE_C128 or GPE_C64");
    gpe_state *st = new gpe_state();
    st->grid = g;
    st->dtype = dtype;
    st->elem = dtype == GPE_C128 ? 16 : 8;
    int rc = dev_alloc(&st->d_psi, g->n_stored * st->elem);
    if (rc == GPE_OK && cudaMemset(st->d_psi, 0, g->n_stored * st->elem) != cudaSuccess)
        rc = fail(GPE_ERR_CUDA, "cudaMemset(psi) failed");
    if (rc == GPE_OK) rc = dev_alloc(&st->d_E, g->n_stored * st->elem / 2);
    if (rc == GPE_OK) rc = dev_alloc_t(&st->d_clock, 1);
    if (rc == GPE_OK) rc = red_alloc(st->red, g->nsm * 32);
    if (rc == GPE_OK && cudaMallocHost(&st->h_obs, sizeof(gpe_obs)) != cudaSuccess)
        rc = fail(GPE_ERR_CUDA, "cudaMallocHost failed");
    if (rc != GPE_OK) {
        dev_free(st->d_psi);
        dev_free(st->d_E);
        dev_free(st->d_clock);
        red_free(st->red);
        if (st->h_obs) cudaFreeHost(st->h_obs);
        delete st;
        return rc;
    }
    g->n_states++;
    *out = st;
    return GPE_OK;
}

extern "C" int gpe_state_destroy(gpe_state *st)
{
    if (!st) return GPE_OK;
    cudaDeviceSynchronize();
    dev_free(st->d_psi);
    for (int i = 0; i < 3; ++i) dev_free(st->d_work[i]);
    dev_free(st->d_E);
    dev_free(st->d_clock);
    red_free(st->red);
    if (st->h_obs) cudaFreeHost(st->h_obs);
    st->grid->n_states--;
    delete st;
    return GPE_OK;
}

extern "C" int gpe_state_device_ptr(gpe_state *st, void **dptr)
{
    GPE_TRY(check_state(st));
    if (!dptr) return fail(GPE_ERR_ARG, "dptr is NULL");
    *dptr = st->d_psi;
    return GPE_OK;
}

extern "C" int gpe_state_load(gpe_state *st, const void *psi, int layout, int on_device, gpe_stream stream)
{
    GPE_TRY(check_state(st));
    if (!psi) return fail(GPE_ERR_ARG, "psi is NULL");
    const gpe_grid *g = st->grid;
    cudaStream_t s = S(stream);
    const BoxI bi{g->box.nx, g->box.ny, g->box.nz, g->bx, g->by, g->bz};
    if (layout == GPE_LAYOUT_COMPACT) {
        GPE_TRY_CUDA(cudaMemcpyAsync(st->d_psi, psi, g->n_stored * st->elem,
                                     on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
        if (st->dtype == GPE_C128) k_mask_compact<double2><<<g->nsm * 8, 256, 0, s>>>((double2 *)st->d_psi, g->d_mask, g->n_stored);
        else k_mask_compact<float2><<<g->nsm * 8, 256, 0, s>>>((float2 *)st->d_psi, g->d_mask, g->n_stored);
        GPE_LAUNCH_CHECK();
        if (!on_device) GPE_TRY_CUDA(cudaStreamSynchronize(s));
        return GPE_OK;
    }
    if (layout != GPE_LAYOUT_DENSE) return fail(GPE_ERR_ARG, "unknown layout %d", layout);
    const size_t dbytes = (size_t)g->box.nx * g->box.ny * g->box.nz * st->elem;
    const void *src = psi;
    void *owned = nullptr;
    if (!on_device) {
        GPE_TRY(dev_alloc(&owned, dbytes));
        cudaError_t e = cudaMemcpyAsync(owned, psi, dbytes, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) {
            dev_free(owned);
            return cuda_fail(e, "cudaMemcpyAsync(psi)", __FILE__, __LINE__);
        }
        src = owned;
    }
    if (st->dtype == GPE_C128)
        k_load_dense<double2><<<g->nsm * 8, 256, 0, s>>>((const double2 *)src, (double2 *)st->d_psi, g->d_org, g->d_mask, g->n_stored, bi);
    else
        k_load_dense<float2><<<g->nsm * 8, 256, 0, s>>>((const float2 *)src, (float2 *)st->d_psi, g->d_org, g->d_mask, g->n_stored, bi);
    cudaError_t e = cudaGetLastError();
    if (owned) {
        cudaStreamSynchronize(s);
        dev_free(owned);
    }
    if (e != cudaSuccess) return cuda_fail(e, "k_load_dense", __FILE__, __LINE__);
    return GPE_OK;
}

extern "C" int gpe_state_store(const gpe_state *st, void *psi, int layout, int on_device, gpe_stream stream)
{
    GPE_TRY(check_state(st));
    if (!psi) return fail(GPE_ERR_ARG, "psi is NULL");
    const gpe_grid *g = st->grid;
    cudaStream_t s = S(stream);
    if (layout == GPE_LAYOUT_COMPACT) {
        GPE_TRY_CUDA(cudaMemcpyAsync(psi, st->d_psi, g->n_stored * st->elem,
                                     on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
        if (!on_device) GPE_TRY_CUDA(cudaStreamSynchronize(s));
        return GPE_OK;
    }
    if (layout != GPE_LAYOUT_DENSE) return fail(GPE_ERR_ARG, "unknown layout %d", layout);
    const BoxI bi{g->box.nx, g->box.ny, g->box.nz, g->bx, g->by, g->bz};
    const size_t dbytes = (size_t)g->box.nx * g->box.ny * g->box.nz * st->elem;
    void *dst = psi;
    void *owned = nullptr;
    if (!on_device) {
        GPE_TRY(dev_alloc(&owned, dbytes));
        dst = owned;
    }
    cudaError_t e = cudaMemsetAsync(dst, 0, dbytes, s);
    if (e == cudaSuccess) {
        if (st->dtype == GPE_C128)
            k_store_dense<double2><<<g->nsm * 8, 256, 0, s>>>((const double2 *)st->d_psi, (double2 *)dst, g->d_org, g->d_mask, g->n_stored, bi);
        else
            k_store_dense<float2><<<g->nsm * 8, 256, 0, s>>>((const float2 *)st->d_psi, (float2 *)dst, g->d_org, g->d_mask, g->n_stored, bi);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && owned) e = cudaMemcpyAsync(psi, owned, dbytes, cudaMemcpyDeviceToHost, s);
    if (owned) {
        cudaError_t e2 = cudaStreamSynchronize(s);
        if (e == cudaSuccess) e = e2;
        dev_free(owned);
    }
    if (e != cudaSuccess) return cuda_fail(e, "gpe_state_store", __FILE__, __LINE__);
    return GPE_OK;
}

extern "C" int gpe_state_copy(gpe_state *dst, const gpe_state *src, gpe_stream stream)
{
    GPE_TRY(check_state(dst));
    GPE_TRY(check_state(src));
    if (dst->grid != src->grid || dst->dtype != src->dtype)
        return fail(GPE_ERR_ARG, "states differ in grid or dtype");
    GPE_TRY_CUDA(cudaMemcpyAsync(dst->d_psi, src->d_psi, src->grid->n_stored * src->elem, cudaMemcpyDeviceToDevice, S(stream)));
    return GPE_OK;
}

extern "C" int gpe_step_real(gpe_state *st, const gpe_real_params *p, int64_t nsteps, double t0, gpe_stream stream)
{
    GPE_TRY(check_state(st));
    if (!p) return fail(GPE_ERR_ARG, "params is NULL");
    if (nsteps < 0) return fail(GPE_ERR_ARG, "nsteps < 0");
    if (p->integrator != GPE_RK4) return fail(GPE_ERR_ARG, "unknown integrator %d", p->integrator);
    if (!(p->dt > 0) || !std::isfinite(p->dt)) return fail(GPE_ERR_ARG, "dt must be finite and > 0");
    if (!std::isfinite(p->g)) return fail(GPE_ERR_ARG, "g must be finite");
    if (p->potential == GPE_V_BLEND) {
        if (p->n_knots < 2 || p->n_knots > GPE_MAX_KNOTS) return fail(GPE_ERR_ARG, "n_knots must be in [2, 16]");
        if (!(p->T_ramp > 0)) return fail(GPE_ERR_ARG, "T_ramp must be > 0");
        if (!st->grid->d_V[1]) return fail(GPE_ERR_STATE, "blend needs potential slot 1");
    } else if (p->potential != GPE_V_STATIC) {
        return fail(GPE_ERR_ARG, "unknown potential mode %d", p->potential);
    }
    const gpe_box &b = st->grid->box;
    const double lam = 2.0 / (b.hx * b.hx) + 2.0 / (b.hy * b.hy) + 2.0 / (b.hz * b.hz) + st->grid->v_max;
    if (p->dt * lam > 2.0 * std::sqrt(2.0))
        return fail(GPE_ERR_UNSTABLE, "dt*lambda_max = %.3g exceeds RK4's limit 2*sqrt(2)", p->dt * lam);
    if (nsteps == 0) return GPE_OK;
    GPE_TRY(ensure_work(st, 3));
    cudaStream_t s = S(stream);
    const bool c128 = st->dtype == GPE_C128;
#define RK_CASE(id, X, Y, Z) \
    case id: return c128 ? rk4_run<double, X, Y, Z>(st, p, nsteps, t0, s) : rk4_run<float, X, Y, Z>(st, p, nsteps, t0, s);
    switch (st->grid->shape) { GPE_SHAPES(RK_CASE) }
#undef RK_CASE
    return fail(GPE_ERR_STATE, "bad brick shape");
}

extern "C" int gpe_step_imag(gpe_state *st, const gpe_imag_params *p, int64_t nsteps, gpe_stream stream)
{
    GPE_TRY(check_state(st));
    if (!p) return fail(GPE_ERR_ARG, "params is NULL");
    if (nsteps < 0) return fail(GPE_ERR_ARG, "nsteps < 0");
    if (!(p->dt > 0) || !std::isfinite(p->dt)) return fail(GPE_ERR_ARG, "dt must be finite and > 0");
    if (!(p->N > 0) || !std::isfinite(p->N)) return fail(GPE_ERR_ARG, "N must be finite and > 0");
    if (!std::isfinite(p->g)) return fail(GPE_ERR_ARG, "g must be finite");
    const gpe_box &b = st->grid->box;
    const double lam = 2.0 / (b.hx * b.hx) + 2.0 / (b.hy * b.hy) + 2.0 / (b.hz * b.hz);
    if (p->dt * lam > 4.0)
        return fail(GPE_ERR_UNSTABLE, "dt*lambda_max(T) = %.3g exceeds the Euler substep limit 4", p->dt * lam);
    if (nsteps == 0) return GPE_OK;
    GPE_TRY(ensure_work(st, 1));
    cudaStream_t s = S(stream);
    const bool c128 = st->dtype == GPE_C128;
#define ITP_CASE(id, X, Y, Z) \
    case id: return c128 ? itp_run<double, X, Y, Z>(st, p, nsteps, s) : itp_run<float, X, Y, Z>(st, p, nsteps, s);
    switch (st->grid->shape) { GPE_SHAPES(ITP_CASE) }
#undef ITP_CASE
    return fail(GPE_ERR_STATE, "bad brick shape");
}

extern "C" int gpe_observables(const gpe_state *st, double g, double s_blend, gpe_obs *out, gpe_stream stream)
{
    GPE_TRY(check_state(st));
    if (!out) return fail(GPE_ERR_ARG, "out is NULL");
    if (!std::isfinite(g) || !std::isfinite(s_blend)) return fail(GPE_ERR_ARG, "g and s_blend must be finite");
    cudaStream_t s = S(stream);
    const bool c128 = st->dtype == GPE_C128;
    int rc = GPE_ERR_STATE;
#define OBS_CASE(id, X, Y, Z) \
    case id: rc = c128 ? obs_run<double, X, Y, Z>(st, g, s_blend, s) : obs_run<float, X, Y, Z>(st, g, s_blend, s); break;
    switch (st->grid->shape) { GPE_SHAPES(OBS_CASE) }
#undef OBS_CASE
    if (rc != GPE_OK) return rc;
    GPE_TRY_CUDA(cudaMemcpyAsync(st->h_obs, st->red.scalars + 2, sizeof(gpe_obs), cudaMemcpyDeviceToHost, s));
    GPE_TRY_CUDA(cudaStreamSynchronize(s));
    *out = *st->h_obs;
    if (out->nonfinite > 0) return fail(GPE_ERR_NONFINITE, "%.0f active cells hold NaN or Inf", out->nonfinite);
    return GPE_OK;
}

extern "C" int gpe_overlap(const gpe_state *a, const gpe_state *b, double out[2], gpe_stream stream)
{
    GPE_TRY(check_state(a));
    GPE_TRY(check_state(b));
    if (!out) return fail(GPE_ERR_ARG, "out is NULL");
    if (a->grid != b->grid || a->dtype != b->dtype) return fail(GPE_ERR_ARG, "states differ in grid or dtype");
    const gpe_grid *g = a->grid;
    cudaStream_t s = S(stream);
    gpe_state *w = const_cast<gpe_state *>(a);
    const int blocks = g->nsm * 4;
    const double dV = g->box.hx * g->box.hy * g->box.hz;
    if (a->dtype == GPE_C128)
        k_overlap<double2><<<blocks, 256, 0, s>>>((const double2 *)a->d_psi, (const double2 *)b->d_psi, g->d_mask,
                                                   g->n_stored, dV, w->red.partials, w->red.counter, w->red.scalars + 10);
    else
        k_overlap<float2><<<blocks, 256, 0, s>>>((const float2 *)a->d_psi, (const float2 *)b->d_psi, g->d_mask,
                                                  g->n_stored, dV, w->red.partials, w->red.counter, w->red.scalars + 10);
    GPE_LAUNCH_CHECK();
    double h[2];
    GPE_TRY_CUDA(cudaMemcpyAsync(h, w->red.scalars + 10, sizeof h, cudaMemcpyDeviceToHost, s));
    GPE_TRY_CUDA(cudaStreamSynchronize(s));
    out[0] = h[0];
    out[1] = h[1];
    return GPE_OK;
}

extern "C" int gpe_ground_state(gpe_state *st, const gpe_imag_params *p, double tol_dmu, int64_t check_every,
                                int64_t max_steps, int64_t *steps_done, gpe_obs *obs, gpe_stream stream)
{
    GPE_TRY(check_state(st));
    if (!p) return fail(GPE_ERR_ARG, "params is NULL");
    if (check_every < 1 || max_steps < 1 || !(tol_dmu > 0))
        return fail(GPE_ERR_ARG, "need check_every >= 1, max_steps >= 1, tol_dmu > 0");
    double mu_prev = NAN;
    int64_t done = 0;
    gpe_obs o{};
    int rc = GPE_ERR_NOT_CONVERGED;
    while (done < max_steps) {
        int64_t n = check_every < max_steps - done ? check_every : max_steps - done;
        GPE_TRY(gpe_step_imag(st, p, n, stream));
        done += n;
        int r = gpe_observables(st, p->g, 0.0, &o, stream);
        if (r != GPE_OK) {
            rc = r;
            break;
        }
        if (std::isfinite(mu_prev) && std::fabs(o.mu - mu_prev) < tol_dmu) {
            rc = GPE_OK;
            break;
        }
        mu_prev = o.mu;
    }
    if (steps_done) *steps_done = done;
    if (obs) *obs = o;
    if (rc == GPE_ERR_NOT_CONVERGED)
        return fail(GPE_ERR_NOT_CONVERGED, "|dmu| >= %g after %lld steps", tol_dmu, (long long)done);
    return rc;
}
