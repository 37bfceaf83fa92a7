// kernels.cuh -- device kernels shared by the step translation units (the
// 7-point and 19-point builds): the imaginary-time stencil passes, the
// propagator table, the deferred renormalisation and the observables.  Not
// part of the ABI.
#pragma once

#include "stencil.cuh"

namespace gpe {

// a + b rounded once and never fused with the product that feeds it, so that
// the per-segment sums of a real state and of a complex state with zero
// imaginary part round identically
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }

// E = exp(-V dt/2) in the state precision (Eq. (7): the diagonal propagator
// is precomputed once per dt); E = -1 marks the inactive cells of stored
// segments (V = +inf there)
template <typename R>
__global__ void k_make_E(const double *V, R *E, int64_t n, double dt)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        E[i] = V[i] < INFINITY ? (R)exp(-V[i] * dt / 2.0) : (R)-1;
}

// ------------------------------------------------------------ imaginary time
// Sec. II A/B, Eqs. (6)-(7).  Stage A gathers psi with its neighbours,
// applying on load the pending renormalisation factor and the diagonal half
// step psi * E * (1 - g|psi|^2 dt/2), E = exp(-V dt/2); then the first Euler
// kinetic substep psi - (dt/2) T psi = psi + (dt/4) lap psi -> tmp.
// Stage B gathers tmp, takes the second Euler substep, applies the diagonal
// half step again, writes psi and sums |psi|^2 in FP64; the factor
// sqrt(N / (sum |psi|^2 dV)) is stored for the next step's stage A (or the
// end of the call).  E = -1 marks the inactive cells of stored segments
// (V = +inf), which are set to zero.
template <typename R, typename CT = typename Cx<R>::T>
struct ItpArgs {
    CT *psi;
    CT *tmp;
    const R *E;
    R ihx2, ihy2, ihz2, g, dt;
    double *scalars;  // [0] scale to apply on load / next scale, [1] last norm
    double N, dV;
};

// The propagator table E of a segment (E < 0 marks an inactive cell), loaded
// ahead of the segment's update
template <typename R>
struct ELoad {
    const R *E;
    struct P {
        R e[4];
    };
    __device__ __forceinline__ P operator()(uint32_t idx) const
    {
        P p;
        ldr4(E + idx, p.e);
        return p;
    }
};

template <typename R, typename CT, int BX, int BY, int BZ, bool CG, int NP = 7>
__device__ __forceinline__ void itp_brick_a(const ItpArgs<R, CT> &a, const GridView &G, int64_t b, int64_t next,
                                            WarpSpace<CT, BX, BY, BZ, NP> &ws, R sc)
{
    const R q4 = a.dt / (R)4;
    const DiagLoad<R, CT> diag{sc, a.g * a.dt / (R)2, a.E};
    brick_apply<BX, BY, BZ, CG>(ws, G, b, next, a.psi, diag, a.ihx2, a.ihy2, a.ihz2, ELoad<R>{a.E},
                                [&](uint32_t idx, const typename ELoad<R>::P &p, const CT(&c)[4], const CT(&L)[4]) {
        CT o[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const bool act = p.e[i] >= (R)0;  // E < 0 marks an inactive cell of a stored segment
            o[i] = act ? axpy(c[i], q4, L[i]) : czero<CT>();
        }
        st4(a.tmp + idx, o);
    });
}

template <typename R, typename CT, int BX, int BY, int BZ, bool CG, int NP = 7>
__device__ __forceinline__ void itp_brick_b(const ItpArgs<R, CT> &a, const GridView &G, int64_t b, int64_t next,
                                            WarpSpace<CT, BX, BY, BZ, NP> &ws, double &acc)
{
    const R hg = a.g * a.dt / (R)2;
    const R q4 = a.dt / (R)4;
    brick_apply<BX, BY, BZ, CG>(ws, G, b, next, a.tmp, Identity(), a.ihx2, a.ihy2, a.ihz2, ELoad<R>{a.E},
                                [&](uint32_t idx, const typename ELoad<R>::P &p, const CT(&c)[4], const CT(&L)[4]) {
        CT o[4];
        R n4 = (R)0;  // the segment's |psi|^2, added to the FP64 sum once
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            o[i] = axpy(c[i], q4, L[i]);
            const R f = p.e[i] >= (R)0 ? p.e[i] * ((R)1 - hg * norm2(o[i])) : (R)0;
            o[i] = scale(o[i], f);
            n4 = add_rn(n4, norm2(o[i]));
        }
        acc += (double)n4;
        st4(a.psi + idx, o);
    });
}

template <typename R, int BX, int BY, int BZ, typename CT = typename Cx<R>::T, int NP = 7>
__global__ void GPE_BOUNDS_NP(R) k_itp_a(const ItpArgs<R, CT> a, const GridView G)
{
    pdl_enter();
    constexpr int NW = KernelCfg<R>::NW;
    auto &ws = warp_space<R, BX, BY, BZ, CT, NP>();
    const int warp = threadIdx.x >> 5;
    const R sc = (R)a.scalars[0];
    const int64_t stride = (int64_t)gridDim.x * NW;
    for (int64_t b = (int64_t)blockIdx.x * NW + warp; b < G.nb; b += stride)
        itp_brick_a<R, CT, BX, BY, BZ, false, NP>(a, G, b, b + stride < G.nb ? b + stride : -1, ws, sc);
}

template <typename R, int BX, int BY, int BZ, typename CT = typename Cx<R>::T, int NP = 7>
__global__ void GPE_BOUNDS_NP(R) k_itp_b(const ItpArgs<R, CT> a, const GridView G, double *partials,
                                          unsigned int *counter)
{
    pdl_enter();
    constexpr int NW = KernelCfg<R>::NW;
    auto &ws = warp_space<R, BX, BY, BZ, CT, NP>();
    const int warp = threadIdx.x >> 5;
    double acc[1] = {0.0};
    const int64_t stride = (int64_t)gridDim.x * NW;
    for (int64_t b = (int64_t)blockIdx.x * NW + warp; b < G.nb; b += stride)
        itp_brick_b<R, CT, BX, BY, BZ, false, NP>(a, G, b, b + stride < G.nb ? b + stride : -1, ws, acc[0]);
    double tot[1];
    if (reduce_finish<1>(acc, partials, counter, tot) && threadIdx.x == 0) {
        const double nrm = tot[0] * a.dV;
        a.scalars[0] = sqrt(a.N / nrm);
        a.scalars[1] = nrm;
    }
}

// the pending renormalisation applied at the end of a call, rounded exactly as
// the next step's load would apply it (factor in the state's precision), so
// that a run split across calls or resumed from a dump is bit-identical
template <typename CT>
__global__ void k_apply_scale(CT *psi, int64_t n, const double *scalars)
{
    const auto sc = (typename RealOf<CT>::T)scalars[0];
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
        psi[s] = scale(psi[s], sc);
    }
}

// ------------------------------------------------------------ observables
template <typename R, typename CT = typename Cx<R>::T>
struct ObsArgs {
    const CT *psi;
    const R *V0;
    const R *V1;
    R s;
    R ihx2, ihy2, ihz2, g;
    double dV;
    double *partials;
    unsigned int *counter;
    gpe_obs *out;
};

template <typename R, int BX, int BY, int BZ, typename CT = typename Cx<R>::T, int NP = 7>
__global__ void GPE_BOUNDS_NP(R) k_obs(const ObsArgs<R, CT> a, const GridView G)
{
    constexpr int NW = KernelCfg<R>::NW;
    auto &ws = warp_space<R, BX, BY, BZ, CT, NP>();
    const int warp = threadIdx.x >> 5;
    double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};  // norm, ekin, epot, eint, nonfinite
    const int64_t stride = (int64_t)gridDim.x * NW;
    for (int64_t b = (int64_t)blockIdx.x * NW + warp; b < G.nb; b += stride) {
        brick_apply<BX, BY, BZ, false>(ws, G, b, b + stride < G.nb ? b + stride : -1, a.psi, Identity(), a.ihx2, a.ihy2, a.ihz2,
                                       [&](uint32_t idx, const CT(&c)[4], const CT(&L)[4]) {
            R V0[4], V1[4];
            ldr4(a.V0 + idx, V0);
            if (a.V1) ldr4(a.V1 + idx, V1);
            // the segment's four terms summed in the state precision, then
            // added to the FP64 sums once (one FP64 add per segment and term)
            R t[4] = {(R)0, (R)0, (R)0, (R)0};
            int nf = 0;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                if (!(V0[i] < (R)INFINITY)) continue;
                const R V = a.V1 ? ((R)1 - a.s) * V0[i] + a.s * V1[i] : V0[i];
                const R rho = norm2(c[i]);
                t[0] = add_rn(t[0], rho);
                t[1] = add_rn(t[1], (R)(-0.5) * dotre(c[i], L[i]));
                t[2] = add_rn(t[2], V * rho);
                t[3] = add_rn(t[3], (R)0.5 * a.g * rho * rho);
                nf += finite_v(c[i]) ? 0 : 1;
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[k] += (double)t[k];
            acc[4] += (double)nf;
        });
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

}  // namespace gpe
