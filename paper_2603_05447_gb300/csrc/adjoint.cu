// adjoint.cu -- gradient of a ramp's final-state infidelity with respect to
// the knots of the potential schedule, by the discrete adjoint of the RK4 step.
//
// The forward pass (gpe_ramp_forward) is the real-time RK4 ramp of Eq. (8)
// with V(t) = (1 - s(t)) V0 + s(t) V1 (the linear interpolation between
// potentials of Sec. V) and keeps a checkpoint of psi every K steps.  The
// backward pass (gpe_ramp_backward) seeds dL/dpsi(T) for
// L = 1 - |<psi_t|psi(T)>|^2, then walks the segments from the last: it
// recomputes the segment's step-start states from its checkpoint, and for
// each step (last first) recomputes the stage states Y2, Y3, Y4 and runs four
// adjoint-stage kernels.  With psi as the real pair (Re, Im), a gradient G is
// stored as dL/dRe + i dL/dIm, and the transposed Jacobian of
// f(y) = -i [(T + V) y + g|y|^2 y] acting on G is
//   J^T G = i (T + V) G + 2 i g |y|^2 G - i g y^2 conj(G).
// Reversing y1 = y0 + dt (k1 + 2 k2 + 2 k3 + k4)/6:
//   mu4 = dt/6 lam'             nu4 = J4^T mu4
//   mu3 = dt/3 lam' + dt nu4     nu3 = J3^T mu3
//   mu2 = dt/3 lam' + dt/2 nu3   nu2 = J2^T mu2
//   mu1 = dt/6 lam' + dt/2 nu2   nu1 = J1^T mu1
//   lam = lam' + nu1 + nu2 + nu3 + nu4
// and every stage adds Re<mu_i, -i (V1 - V0) Y_i> = sum (V1 - V0) Im(conj(mu_i) Y_i),
// reduced in FP64, to the two knots whose hat functions cover its time.
// Bulk arithmetic runs in the state's precision; the gradient accumulates in
// FP64.
#include <algorithm>
#include <cmath>
#include <vector>

#include "gpe_internal.cuh"
#include "stencil.cuh"

namespace gpe {

template <typename R>
struct AdjArgs {
    using CT = typename Cx<R>::T;
    const CT *mu_in;  // gathered: mu_i (stage 4: lam', scaled by m_scale)
    R m_scale;
    const CT *Y;      // stage state Y_i
    const CT *lam;    // lam' (own cells)
    CT *lam_out;      // lam, written by the last stage (may alias lam)
    CT *acc;          // running lam' + sum nu
    CT *mu_out;       // mu_{i-1} = cl lam' + cn nu_i
    const R *V0;
    const R *V1;
    R s;              // schedule value at the stage time
    R cl, cn;
    int first, last;
    R ihx2, ihy2, ihz2, g;
    double *partials;
    unsigned int *counter;
    double *grad;     // [16] FP64 knot gradient
    int k0;
    double w0, w1;    // hat weights of knots k0, k0+1 at the stage time
};

template <typename R>
struct Scale {
    R s;
    template <typename CT>
    __device__ __forceinline__ CT operator()(CT v, uint32_t) const
    {
        v.x *= s;
        v.y *= s;
        return v;
    }
};

template <typename R, int BX, int BY, int BZ, bool BLEND>
__global__ void GPE_BOUNDS(R) k_adj_stage(const AdjArgs<R> a, const GridView G)
{
    using CT = typename Cx<R>::T;
    constexpr int NW = KernelCfg<R>::NW;
    auto &ws = warp_space<R, BX, BY, BZ>();
    const int warp = threadIdx.x >> 5;
    double dot[1] = {0.0};
    const int64_t stride = (int64_t)gridDim.x * NW;
    for (int64_t b = (int64_t)blockIdx.x * NW + warp; b < G.nb; b += stride) {
        brick_apply<BX, BY, BZ, false>(ws, G, b, b + stride < G.nb ? b + stride : -1, a.mu_in, Scale<R>{a.m_scale}, a.ihx2, a.ihy2, a.ihz2,
                                       [&](uint32_t idx, const CT(&M)[4], const CT(&L)[4]) {
            R V0[4], V1[4];
            CT Y[4], lam[4], acc[4];
            ldr4(a.V0 + idx, V0);
            if (BLEND) ldr4(a.V1 + idx, V1);
            ld4<false>(a.Y + idx, Y);
            ld4<false>(a.lam + idx, lam);
            if (!a.first) ld4<false>(a.acc + idx, acc);
            CT nacc[4], mo[4];
            R d4 = (R)0;  // the segment's share of the knot derivative, added in FP64 once
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                if (!(V0[i] < (R)INFINITY)) {  // inactive cell of a stored segment
                    nacc[i] = czero<CT>();
                    mo[i] = czero<CT>();
                    continue;
                }
                const R dV = BLEND ? V1[i] - V0[i] : (R)0;
                const R Vt = BLEND ? ((R)1 - a.s) * V0[i] + a.s * V1[i] : V0[i];
                const R rho = Y[i].x * Y[i].x + Y[i].y * Y[i].y;
                // C = (T + Vt + 2 g rho) M - g Y^2 conj(M);  nu = i C
                const R w = Vt + (R)2 * a.g * rho;
                const R y2r = Y[i].x * Y[i].x - Y[i].y * Y[i].y, y2i = (R)2 * Y[i].x * Y[i].y;
                const R br = y2r * M[i].x + y2i * M[i].y;   // Re(Y^2 conj(M))
                const R bi = y2i * M[i].x - y2r * M[i].y;   // Im(Y^2 conj(M))
                const R cr = (R)(-0.5) * L[i].x + w * M[i].x - a.g * br;
                const R ci = (R)(-0.5) * L[i].y + w * M[i].y - a.g * bi;
                CT nu;
                nu.x = -ci;
                nu.y = cr;
                if (BLEND) d4 += dV * (M[i].x * Y[i].y - M[i].y * Y[i].x);
                const CT base = a.first ? lam[i] : acc[i];
                nacc[i].x = base.x + nu.x;
                nacc[i].y = base.y + nu.y;
                mo[i].x = a.cl * lam[i].x + a.cn * nu.x;
                mo[i].y = a.cl * lam[i].y + a.cn * nu.y;
            }
            if (BLEND) dot[0] += (double)d4;
            if (a.last) {
                st4(a.lam_out + idx, nacc);
            } else {
                st4(a.acc + idx, nacc);
                st4(a.mu_out + idx, mo);
            }
        });
    }
    double tot[1];
    if (reduce_finish<1>(dot, a.partials, a.counter, tot) && threadIdx.x == 0 && BLEND) {
        a.grad[a.k0] += a.w0 * tot[0];
        a.grad[a.k0 + 1] += a.w1 * tot[0];
    }
}

// seed of the reverse sweep: lam = dL/dpsi(T) = -2 dV c psi_t for
// L = 1 - |c|^2, c = <psi_t|psi(T)>
template <typename CT>
__global__ void k_seed(CT *lam, const CT *tgt, int64_t n, double cr, double ci, double dV)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const CT t = tgt[i];
        CT o;
        o.x = (-2.0 * dV) * (cr * t.x - ci * t.y);
        o.y = (-2.0 * dV) * (cr * t.y + ci * t.x);
        lam[i] = o;
    }
}

// s(t) on the host, the same piecewise-linear schedule as ramp_s
static double ramp_s_host(const gpe_real_params &p, double t)
{
    const int nk = p.n_knots;
    if (t <= 0.0) return p.knots[0];
    if (t >= p.T_ramp) return p.knots[nk - 1];
    const double u = t / p.T_ramp * (double)(nk - 1);
    int k = (int)std::floor(u);
    if (k >= nk - 1) k = nk - 2;
    const double w = u - (double)k;
    return (1.0 - w) * p.knots[k] + w * p.knots[k + 1];
}

// hat weights of the knots at time t (the interpolation of the schedule)
static void hat(const gpe_real_params &p, double t, int &k0, double &w0, double &w1)
{
    const int nk = p.n_knots;
    if (t <= 0.0) {
        k0 = 0;
        w0 = 1.0;
        w1 = 0.0;
        return;
    }
    if (t >= p.T_ramp) {
        k0 = nk - 2;
        w0 = 0.0;
        w1 = 1.0;
        return;
    }
    const double u = t / p.T_ramp * (double)(nk - 1);
    k0 = (int)std::floor(u);
    if (k0 >= nk - 1) k0 = nk - 2;
    const double w = u - (double)k0;
    w0 = 1.0 - w;
    w1 = w;
}

}  // namespace gpe

using namespace gpe;

struct gpe_tape {
    gpe_state *st = nullptr;
    gpe_real_params p{};
    int64_t nsteps = 0, nck = 0;
    double t0 = 0.0;
    int K = 0;
    void *d_ckpt = nullptr;  // [nck * n_packed]
    void *d_seg = nullptr;   // [K * n_packed]
    void *d_lam = nullptr, *d_mu[2] = {nullptr, nullptr}, *d_acc = nullptr;
    void *d_w[4] = {nullptr, nullptr, nullptr, nullptr};  // Y2, Y3, Y4, RK4 partial sum
    double *d_grad = nullptr;
    double *d_clock = nullptr;
    RedScratch red;
};

static void tape_free(gpe_tape *t)
{
    if (!t) return;
    dev_free(t->d_ckpt);
    dev_free(t->d_seg);
    dev_free(t->d_lam);
    dev_free(t->d_mu[0]);
    dev_free(t->d_mu[1]);
    dev_free(t->d_acc);
    for (int i = 0; i < 4; ++i) dev_free(t->d_w[i]);
    dev_free(t->d_grad);
    dev_free(t->d_clock);
    red_free(t->red);
    if (t->st) t->st->grid->n_states--;
    delete t;
}

extern "C" int gpe_tape_destroy(gpe_tape *t)
{
    cudaDeviceSynchronize();
    tape_free(t);
    return GPE_OK;
}

extern "C" int gpe_ramp_forward(gpe_state *st, const gpe_real_params *p, int64_t nsteps, double t0, int K,
                                gpe_tape **out, gpe_stream stream)
{
    if (!st || !p || !out) return fail(GPE_ERR_ARG, "NULL argument");
    *out = nullptr;
    if (nsteps < 1 || K < 1) return fail(GPE_ERR_ARG, "need nsteps >= 1 and K >= 1");
    if (p->potential != GPE_V_BLEND) return fail(GPE_ERR_ARG, "the ramp gradient needs potential = GPE_V_BLEND");
    if (p->integrator != GPE_RK4) return fail(GPE_ERR_ARG, "the ramp gradient is the adjoint of the RK4 step");
    if (st->dtype != GPE_C128 && st->dtype != GPE_C64) return fail(GPE_ERR_ARG, "the ramp gradient needs a complex state");
    if (st->grid->stencil != 7) return fail(GPE_ERR_ARG, "the ramp gradient is built for the 7-point stencil");
    const gpe_grid *g = st->grid;
    const size_t bytes = (size_t)g->n_packed * st->elem;
    gpe_tape *t = new gpe_tape();
    t->p = *p;
    t->nsteps = nsteps;
    t->t0 = t0;
    t->K = (int)std::min<int64_t>(K, nsteps);
    t->nck = (nsteps + t->K - 1) / t->K;
    int rc = GPE_OK;
    rc = dev_alloc(&t->d_ckpt, bytes * t->nck);
    if (rc == GPE_OK) rc = dev_alloc(&t->d_seg, bytes * t->K);
    for (void **b : {&t->d_lam, &t->d_mu[0], &t->d_mu[1], &t->d_acc, &t->d_w[0], &t->d_w[1], &t->d_w[2], &t->d_w[3]})
        if (rc == GPE_OK && (rc = dev_alloc(b, bytes)) == GPE_OK) rc = dev_zero(*b, bytes);
    if (rc == GPE_OK) rc = dev_alloc_t(&t->d_grad, GPE_MAX_KNOTS);
    if (rc == GPE_OK) rc = dev_alloc_t(&t->d_clock, 1);
    if (rc == GPE_OK) rc = dev_zero(t->d_clock, sizeof(double));
    if (rc == GPE_OK) rc = red_alloc(t->red, g->nsm * 32);
    if (rc != GPE_OK) {
        tape_free(t);
        return rc;
    }
    t->st = st;
    st->grid->n_states++;
    cudaStream_t s = S(stream);
    for (int64_t j = 0; j < t->nck; ++j) {
        const int64_t n = std::min<int64_t>(t->K, nsteps - j * t->K);
        cudaError_t e = cudaMemcpyAsync((char *)t->d_ckpt + j * bytes, st->d_psi, bytes, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) {
            tape_free(t);
            return cuda_fail(e, "checkpoint copy", __FILE__, __LINE__);
        }
        rc = gpe_step_real(st, p, n, t0 + (double)(j * t->K) * p->dt, stream);
        if (rc != GPE_OK) {
            tape_free(t);
            return rc;
        }
    }
    *out = t;
    return GPE_OK;
}

namespace gpe {

template <typename R, typename K>
static int adj_blocks(K kernel, const gpe_grid *g, size_t smem, int nw = KernelCfg<R>::NW)
{
    const int per = prepare_kernel(kernel, 32 * nw, smem);
    const int64_t need = (g->nb + nw - 1) / nw;
    return (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)g->nsm * per, need));
}

template <typename R, int BX, int BY, int BZ>
static int backward_impl(gpe_tape *t, const gpe_state *target, double *grad, double *loss, cudaStream_t s)
{
    using CT = typename Cx<R>::T;
    gpe_state *st = t->st;
    const gpe_grid *g = st->grid;
    const gpe_real_params &p = t->p;
    const size_t np = (size_t)g->n_packed;
    const GridView G = view(g);
    // loss and seed
    double c[2];
    GPE_TRY(gpe_overlap(target, st, c, (gpe_stream)s));
    *loss = 1.0 - (c[0] * c[0] + c[1] * c[1]);
    const double dV = g->box.hx * g->box.hy * g->box.hz;
    CT *lam = (CT *)t->d_lam;
    k_seed<CT><<<g->nsm * 8, 256, 0, s>>>(lam, (const CT *)target->d_psi, (int64_t)np, c[0], c[1], dV);
    GPE_LAUNCH_CHECK();
    GPE_TRY_CUDA(cudaMemsetAsync(t->d_grad, 0, GPE_MAX_KNOTS * sizeof(double), s));
    // forward stage kernels on tape buffers
    RkArgs<R> f{};
    f.V0 = (const R *)potential_ptr(st, 0);
    f.V1 = (const R *)potential_ptr(st, 1);
    if (!f.V0 || !f.V1) return fail(GPE_ERR_STATE, "ramp needs potential slots 0 and 1");
    f.y2 = (CT *)t->d_w[0];
    f.y3 = (CT *)t->d_w[1];
    f.y4 = (CT *)t->d_w[2];  // kept apart from Y2: the reverse sweep reads all three
    f.w = (CT *)t->d_w[3];
    f.ihx2 = (R)(1.0 / (g->box.hx * g->box.hx));
    f.ihy2 = (R)(1.0 / (g->box.hy * g->box.hy));
    f.ihz2 = (R)(1.0 / (g->box.hz * g->box.hz));
    f.g = (R)p.g;
    f.dt = (R)p.dt;
    f.dtd = p.dt;
    f.ramp.clock = t->d_clock;  // holds 0: stage times are absolute
    f.ramp.T = p.T_ramp;
    f.ramp.n_knots = p.n_knots;
    for (int k = 0; k < GPE_MAX_KNOTS; ++k) f.ramp.knots[k] = p.knots[k];
    using RS = Rk4Stages<R, BX, BY, BZ>;
    typename RS::K kf[4];
    auto ka = k_adj_stage<R, BX, BY, BZ, true>;
    const size_t smem = smem_bytes<R, BX, BY, BZ>();
    const int th = KernelCfg<R>::THREADS;
    int nbf[4];
    for (int stg = 0; stg < 4; ++stg) {
        kf[stg] = RS::get(true, stg);
        nbf[stg] = adj_blocks<R>(kf[stg], g, RS::smem(), RS::NW);
    }
    const int nba = adj_blocks<R>(ka, g, smem);
    AdjArgs<R> a{};
    a.lam = lam;
    a.lam_out = lam;
    a.acc = (CT *)t->d_acc;
    a.V0 = f.V0;
    a.V1 = f.V1;
    a.ihx2 = f.ihx2;
    a.ihy2 = f.ihy2;
    a.ihz2 = f.ihz2;
    a.g = f.g;
    a.partials = t->red.partials;
    a.counter = t->red.counter;
    a.grad = t->d_grad;
    const R dt = (R)p.dt;
    CT *seg = (CT *)t->d_seg, *ck = (CT *)t->d_ckpt;
    for (int64_t j = t->nck - 1; j >= 0; --j) {
        const int64_t len = std::min<int64_t>(t->K, t->nsteps - j * t->K);
        GPE_TRY_CUDA(cudaMemcpyAsync(seg, ck + j * np, np * sizeof(CT), cudaMemcpyDeviceToDevice, s));
        // step-start states of the segment
        for (int64_t m = 0; m + 1 < len; ++m) {
            GPE_TRY_CUDA(cudaMemcpyAsync(seg + (m + 1) * np, seg + m * np, np * sizeof(CT), cudaMemcpyDeviceToDevice, s));
            f.y0 = seg + (m + 1) * np;
            f.t_off = t->t0 + (double)(j * t->K + m) * p.dt;
            for (int stg = 0; stg < 4; ++stg) {
                kf[stg]<<<nbf[stg], RS::THREADS, RS::smem(), s>>>(f, G);
                GPE_LAUNCH_CHECK();
            }
        }
        for (int64_t m = len - 1; m >= 0; --m) {
            const double tm = t->t0 + (double)(j * t->K + m) * p.dt;
            f.y0 = seg + m * np;
            f.t_off = tm;
            for (int stg = 0; stg < 3; ++stg) {  // Y2, Y3, Y4
                kf[stg]<<<nbf[stg], RS::THREADS, RS::smem(), s>>>(f, G);
                GPE_LAUNCH_CHECK();
            }
            // stages 4, 3, 2, 1 of the reverse sweep
            const double ts[4] = {tm + p.dt, tm + 0.5 * p.dt, tm + 0.5 * p.dt, tm};
            const CT *Ys[4] = {f.y4, f.y3, f.y2, f.y0};
            const R cl[4] = {dt / (R)3, dt / (R)3, dt / (R)6, (R)0};
            const R cn[4] = {dt, dt / (R)2, dt / (R)2, (R)0};
            CT *mu[2] = {(CT *)t->d_mu[0], (CT *)t->d_mu[1]};
            for (int r = 0; r < 4; ++r) {
                a.mu_in = r == 0 ? lam : mu[(r - 1) & 1];
                a.m_scale = r == 0 ? dt / (R)6 : (R)1;
                a.mu_out = mu[r & 1];
                a.Y = Ys[r];
                a.s = (R)ramp_s_host(p, ts[r]);
                a.cl = cl[r];
                a.cn = cn[r];
                a.first = r == 0;
                a.last = r == 3;
                hat(p, ts[r], a.k0, a.w0, a.w1);
                ka<<<nba, th, smem, s>>>(a, G);
                GPE_LAUNCH_CHECK();
            }
        }
    }
    double h[GPE_MAX_KNOTS];
    GPE_TRY_CUDA(cudaMemcpyAsync(h, t->d_grad, sizeof h, cudaMemcpyDeviceToHost, s));
    GPE_TRY_CUDA(cudaStreamSynchronize(s));
    for (int k = 0; k < p.n_knots; ++k) grad[k] = h[k];
    return GPE_OK;
}

}  // namespace gpe

extern "C" int gpe_ramp_backward(gpe_tape *t, const gpe_state *target, double *grad_knots, double *loss,
                                 gpe_stream stream)
{
    if (!t || !target || !grad_knots || !loss) return fail(GPE_ERR_ARG, "NULL argument");
    if (target->grid != t->st->grid || target->dtype != t->st->dtype)
        return fail(GPE_ERR_ARG, "target must share the tape state's grid and dtype");
    const bool c128 = t->st->dtype == GPE_C128;
    cudaStream_t s = S(stream);
#define ADJ_CASE(id, X, Y, Z) \
    case id: return c128 ? backward_impl<double, X, Y, Z>(t, target, grad_knots, loss, s) : backward_impl<float, X, Y, Z>(t, target, grad_knots, loss, s);
    switch (t->st->grid->shape) { GPE_SHAPES(ADJ_CASE) }
#undef ADJ_CASE
    return fail(GPE_ERR_STATE, "bad brick shape");
}
