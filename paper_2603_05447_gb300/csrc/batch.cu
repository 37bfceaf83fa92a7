// batch.cu -- many independent shells in one persistent launch: imaginary-time
// ground-state solves (Sec. II A, Eqs. (6)-(7), iterated to a tolerance as in
// Sec. III) for a batch of states whose grids differ in size and shape.  The
// states are complex or, since the imaginary-time step keeps a real
// wavefunction real, real (half the bytes).
//
// The batch concatenates the shells' brick lists, records and packed arrays
// into one layout (neighbour ids and packed offsets shifted by each shell's
// base; a brick record carries its shell id), so one launch of each kernel
// covers every shell.  Per-shell parameters (g, dt, N, spacings, the pending
// renormalisation factor, mu and the convergence flag) live in a device table.
// Norms and observables are reduced per brick, then per shell in brick order
// (deterministic).  Converged shells are skipped brick by brick.  Each block
// of `check_every` steps plus the convergence test is captured once in a CUDA
// graph and replayed; the host polls the number of unconverged shells between
// replays.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "gpe_internal.cuh"
#include "kernels.cuh"
#include "stencil.cuh"

namespace gpe {

struct ShellParams {
    double g, dt, N, dV;
    double ihx2, ihy2, ihz2;
    double scale;     // pending renormalisation factor (applied by the next stage A)
    double mu, mu_prev, energy, norm, e_kin, e_pot, e_int, nonfinite;
    double tol;
    long long steps;  // steps taken
    int converged;
    int has_prev;
};

template <typename R, typename CT = typename Cx<R>::T>
struct BatchArgs {
    CT *psi;
    CT *tmp;
    const R *E;       // exp(-V dt_s/2) per shell, -1 on inactive cells of stored segments
    const R *V;       // potential (for observables), +inf on inactive cells
    ShellParams *sh;
    double *part;     // [nb*5] per-brick partial sums
    const int64_t *brick_base;  // [n+1]
    int n;
};

__device__ __forceinline__ int shell_of(const BrickRec &r) { return (int)r.pad[0]; }

// CT: complex (float2 / double2) or real (float / double) values; a real
// state stays real under the imaginary-time step
template <typename R, typename CT, int BX, int BY, int BZ, int STAGE>
__global__ void GPE_BOUNDS(R) k_batch_itp(const BatchArgs<R, CT> a, const GridView G)
{
    constexpr int NW = KernelCfg<R>::NW;
    auto &ws = warp_space<R, BX, BY, BZ, CT>();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * NW;
    for (int64_t b = (int64_t)blockIdx.x * NW + warp; b < G.nb; b += stride) {
        const ShellParams &P = a.sh[shell_of(G.rec[b])];
        if (P.converged) continue;  // uniform across the warp
        const int64_t nx = b + stride < G.nb ? b + stride : -1;
        const R g = (R)P.g, dt = (R)P.dt;
        const R ihx2 = (R)P.ihx2, ihy2 = (R)P.ihy2, ihz2 = (R)P.ihz2;
        const R q4 = dt / (R)4, hg = g * dt / (R)2;
        double acc = 0.0;
        // E of each segment is loaded ahead (while the tile is in flight)
        auto body = [&](uint32_t idx, const typename ELoad<R>::P &p, const CT(&c)[4], const CT(&L)[4]) {
            const R(&E)[4] = p.e;
            CT o[4];
            R n4 = (R)0;  // the segment's |psi|^2, added to the FP64 sum once
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const bool act = E[i] >= (R)0;
                o[i] = axpy(c[i], q4, L[i]);
                if (STAGE == 1) {
                    const R f = act ? E[i] * ((R)1 - hg * norm2(o[i])) : (R)0;
                    o[i] = scale(o[i], f);
                    n4 = add_rn(n4, norm2(o[i]));
                } else if (!act) {
                    o[i] = czero<CT>();
                }
            }
            if (STAGE == 1) acc += (double)n4;
            st4((STAGE == 0 ? a.tmp : a.psi) + idx, o);
        };
        if (STAGE == 0)
            brick_apply<BX, BY, BZ, false>(ws, G, b, nx, a.psi, DiagLoad<R, CT>{(R)P.scale, hg, a.E}, ihx2, ihy2, ihz2,
                                           ELoad<R>{a.E}, body);
        else
            brick_apply<BX, BY, BZ, false>(ws, G, b, nx, a.tmp, Identity(), ihx2, ihy2, ihz2, ELoad<R>{a.E}, body);
        if (STAGE == 1) {
            for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
            if (lane == 0) a.part[b * 5] = acc;
        }
    }
    cp_async_wait_all();  // a fetched-ahead record row of a skipped brick
}

// per shell: norm from the brick partials (brick order), next factor
__global__ void k_batch_norm_finish(ShellParams *sh, const double *part, const int64_t *brick_base)
{
    const int s = blockIdx.x;
    if (sh[s].converged) return;
    double x = 0.0;
    for (int64_t b = brick_base[s] + threadIdx.x; b < brick_base[s + 1]; b += blockDim.x) x += part[b * 5];
    x = block_sum(x);
    if (threadIdx.x == 0) {
        const double nrm = x * sh[s].dV;
        sh[s].norm = nrm;
        sh[s].scale = sqrt(sh[s].N / nrm);
        sh[s].steps += 1;
    }
}

// apply each shell's pending factor to its bricks (rounded to the state's
// precision, as the next load would apply it), then reset it to 1
template <typename CT>
__global__ void k_batch_apply_scale(CT *psi, const BrickRec *rec, const ShellParams *sh, int64_t nb, int nseg)
{
    for (int64_t b = blockIdx.x; b < nb; b += gridDim.x) {
        const BrickRec r = rec[b];
        const ShellParams &P = sh[shell_of(r)];
        const auto sc = (typename RealOf<CT>::T)P.scale;
        int n = 0;
        for (int w = 0; w < 4; ++w) n += __popc(r.m[w]);
        for (int i = threadIdx.x; i < 4 * n; i += blockDim.x) psi[r.off + i] = scale(psi[r.off + i], sc);
    }
}

__global__ void k_batch_reset_scale(ShellParams *sh, int n)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < n) sh[s].scale = 1.0;
}

template <typename R, typename CT, int BX, int BY, int BZ>
__global__ void GPE_BOUNDS(R) k_batch_obs(const BatchArgs<R, CT> a, const GridView G)
{
    constexpr int NW = KernelCfg<R>::NW;
    auto &ws = warp_space<R, BX, BY, BZ, CT>();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * NW;
    for (int64_t b = (int64_t)blockIdx.x * NW + warp; b < G.nb; b += stride) {
        const ShellParams &P = a.sh[shell_of(G.rec[b])];
        if (P.converged) continue;
        const int64_t nx = b + stride < G.nb ? b + stride : -1;
        const R g = (R)P.g;
        double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
        brick_apply<BX, BY, BZ, false>(ws, G, b, nx, a.psi, Identity(), (R)P.ihx2, (R)P.ihy2, (R)P.ihz2,
                                       [&](uint32_t idx, const CT(&c)[4], const CT(&L)[4]) {
            R V[4];
            ldr4(a.V + idx, V);
            R t[4] = {(R)0, (R)0, (R)0, (R)0};  // the segment's terms, added to the FP64 sums once
            int nf = 0;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                if (!(V[i] < (R)INFINITY)) continue;
                const R rho = norm2(c[i]);
                t[0] = add_rn(t[0], rho);
                t[1] = add_rn(t[1], (R)(-0.5) * dotre(c[i], L[i]));
                t[2] = add_rn(t[2], V[i] * rho);
                t[3] = add_rn(t[3], (R)0.5 * g * rho * rho);
                nf += finite_v(c[i]) ? 0 : 1;
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[k] += (double)t[k];
            acc[4] += (double)nf;
        });
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            double x = acc[k];
            for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
            if (lane == 0) a.part[b * 5 + k] = x;
        }
    }
    cp_async_wait_all();  // a fetched-ahead record row of a skipped brick
}

// per shell: observables from the brick partials, then the convergence test
// |mu - mu_prev| < tol against the previous check
__global__ void k_batch_obs_finish(ShellParams *sh, const double *part, const int64_t *brick_base,
                                   int *n_unconverged)
{
    const int s = blockIdx.x;
    if (sh[s].converged) return;
    double t[5];
    for (int k = 0; k < 5; ++k) {
        double x = 0.0;
        for (int64_t b = brick_base[s] + threadIdx.x; b < brick_base[s + 1]; b += blockDim.x) x += part[b * 5 + k];
        t[k] = block_sum(x);
    }
    if (threadIdx.x == 0) {
        ShellParams &P = sh[s];
        P.norm = t[0] * P.dV;
        P.e_kin = t[1] * P.dV;
        P.e_pot = t[2] * P.dV;
        P.e_int = t[3] * P.dV;
        P.nonfinite = t[4];
        P.energy = P.e_kin + P.e_pot + P.e_int;
        P.mu = (P.e_kin + P.e_pot + 2.0 * P.e_int) / P.norm;
        if (P.has_prev && fabs(P.mu - P.mu_prev) < P.tol) P.converged = 1;
        if (P.nonfinite > 0) P.converged = 1;  // stop a shell that blew up
        P.mu_prev = P.mu;
        P.has_prev = 1;
        if (!P.converged) atomicAdd(n_unconverged, 1);
    }
}

__global__ void k_zero_int(int *p) { *p = 0; }

template <typename R>
__global__ void k_batch_make_E(const double *V, R *E, const BrickRec *rec, const ShellParams *sh, int64_t nb)
{
    for (int64_t b = blockIdx.x; b < nb; b += gridDim.x) {
        const BrickRec r = rec[b];
        const double dt = sh[shell_of(r)].dt;
        int n = 0;
        for (int w = 0; w < 4; ++w) n += __popc(r.m[w]);
        for (int i = threadIdx.x; i < 4 * n; i += blockDim.x) {
            const double v = V[r.off + i];
            E[r.off + i] = v < INFINITY ? (R)exp(-v * dt / 2.0) : (R)-1;
        }
    }
}

template <typename R>
__global__ void k_d2r(const double *s, R *d, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        d[i] = (R)s[i];
}

}  // namespace gpe

using namespace gpe;

struct gpe_batch {
    int n = 0;
    int dtype = 0, shape = 0, device = 0, nsm = 0;
    size_t elem = 0;   // bytes per value of the state type
    size_t relem = 0;  // bytes per real of its precision (E and V tables)
    std::vector<gpe_state *> states;
    std::vector<int64_t> brick_base, packed_base;
    int64_t nb = 0, np = 0;
    int32_t *d_nbr = nullptr;
    BrickRec *d_rec = nullptr;
    BrickRec *d_rec7 = nullptr;
    void *d_psi = nullptr, *d_tmp = nullptr, *d_E = nullptr, *d_Vr = nullptr;
    double *d_V = nullptr;
    ShellParams *d_sh = nullptr;
    double *d_part = nullptr;
    int64_t *d_bb = nullptr;
    int *d_unconv = nullptr;
    int *h_unconv = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap = nullptr;
    uint64_t key = 0;
};

static void batch_free(gpe_batch *B)
{
    if (!B) return;
    if (B->exec) cudaGraphExecDestroy(B->exec);
    if (B->cap) cudaStreamDestroy(B->cap);
    dev_free(B->d_nbr);
    dev_free(B->d_rec);
    dev_free(B->d_rec7);
    dev_free(B->d_psi);
    dev_free(B->d_tmp);
    dev_free(B->d_E);
    dev_free(B->d_Vr);
    dev_free(B->d_V);
    dev_free(B->d_sh);
    dev_free(B->d_part);
    dev_free(B->d_bb);
    dev_free(B->d_unconv);
    if (B->h_unconv) cudaFreeHost(B->h_unconv);
    delete B;
}

extern "C" int gpe_batch_create(gpe_state *const *states, int n, gpe_batch **out)
{
    if (!states || !out || n < 1) return fail(GPE_ERR_ARG, "need n >= 1 states and an output pointer");
    *out = nullptr;
    if (n > 1000000) return fail(GPE_ERR_ARG, "too many shells");
    for (int i = 0; i < n; ++i)
        if (!states[i]) return fail(GPE_ERR_ARG, "state %d is NULL", i);
    const int dtype = states[0]->dtype, shape = states[0]->grid->shape;
    for (int i = 1; i < n; ++i)
        if (states[i]->dtype != dtype || states[i]->grid->shape != shape)
            return fail(GPE_ERR_ARG, "batch states must share dtype and brick shape (state %d differs)", i);
    if (dtype != GPE_C128 && dtype != GPE_C64 && dtype != GPE_R64 && dtype != GPE_R32)
        return fail(GPE_ERR_ARG, "unknown state type %d", dtype);
    for (int i = 0; i < n; ++i)
        if (states[i]->grid->stencil != 7) return fail(GPE_ERR_ARG, "batches run the 7-point stencil (state %d)", i);
    gpe_batch *B = new gpe_batch();
    B->n = n;
    B->dtype = dtype;
    B->shape = shape;
    B->elem = states[0]->elem;
    B->relem = (dtype == GPE_C128 || dtype == GPE_R64) ? sizeof(double) : sizeof(float);
    B->states.assign(states, states + n);
    B->device = states[0]->grid->device;
    B->nsm = states[0]->grid->nsm;
    B->brick_base.resize(n + 1);
    B->packed_base.resize(n + 1);
    for (int i = 0; i < n; ++i) {
        B->brick_base[i + 1] = B->brick_base[i] + states[i]->grid->nb;
        B->packed_base[i + 1] = B->packed_base[i] + states[i]->grid->n_packed;
    }
    B->nb = B->brick_base[n];
    B->np = B->packed_base[n];
    int rc = GPE_OK;
#define BT(x)                  \
    do {                       \
        rc = (x);              \
        if (rc != GPE_OK) {    \
            batch_free(B);     \
            return rc;         \
        }                      \
    } while (0)
    if (B->np >= 0xffffffffLL) BT(fail(GPE_ERR_ARG, "batch too large for 32-bit packed offsets"));
    BT(dev_alloc_t(&B->d_nbr, B->nb * 6));
    BT(dev_alloc_t(&B->d_rec, B->nb));
    BT(dev_alloc_t(&B->d_rec7, B->nb * 7));
    BT(dev_alloc(&B->d_psi, B->np * B->elem));
    BT(dev_alloc(&B->d_tmp, B->np * B->elem));
    BT(dev_alloc(&B->d_E, B->np * B->relem));
    BT(dev_alloc(&B->d_Vr, B->np * B->relem));
    BT(dev_alloc_t(&B->d_V, B->np));
    BT(dev_alloc_t(&B->d_sh, n));
    BT(dev_alloc_t(&B->d_part, B->nb * 5));
    BT(dev_alloc_t(&B->d_bb, n + 1));
    BT(dev_alloc_t(&B->d_unconv, 1));
    if (cudaMallocHost(&B->h_unconv, sizeof(int)) != cudaSuccess) BT(fail(GPE_ERR_CUDA, "cudaMallocHost failed"));
    // combined tables, built on the host from each grid's
    std::vector<int32_t> nbr(B->nb * 6);
    std::vector<BrickRec> rec(B->nb);
    for (int i = 0; i < n; ++i) {
        const gpe_grid *g = states[i]->grid;
        const int64_t b0 = B->brick_base[i];
        if (cudaMemcpy(nbr.data() + b0 * 6, g->d_nbr, g->nb * 6 * sizeof(int32_t), cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(rec.data() + b0, g->d_rec, g->nb * sizeof(BrickRec), cudaMemcpyDeviceToHost) != cudaSuccess)
            BT(fail(GPE_ERR_CUDA, "batch table copy failed"));
        for (int64_t b = b0; b < b0 + g->nb; ++b) {
            for (int d = 0; d < 6; ++d)
                if (nbr[b * 6 + d] >= 0) nbr[b * 6 + d] += (int32_t)b0;
            rec[b].off += (uint32_t)B->packed_base[i];
            rec[b].pad[0] = (uint32_t)i;
        }
        if (cudaMemcpy(B->d_V + B->packed_base[i], g->d_V[0], g->n_packed * sizeof(double), cudaMemcpyDeviceToDevice) !=
            cudaSuccess)
            BT(fail(GPE_ERR_CUDA, "batch potential copy failed"));
    }
    std::vector<BrickRec> rec7;
    build_rec7(rec, nbr, rec7);
    if (cudaMemcpy(B->d_rec7, rec7.data(), rec7.size() * sizeof(BrickRec), cudaMemcpyHostToDevice) != cudaSuccess)
        BT(fail(GPE_ERR_CUDA, "batch table upload failed"));
    if (cudaMemcpy(B->d_nbr, nbr.data(), nbr.size() * sizeof(int32_t), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(B->d_rec, rec.data(), rec.size() * sizeof(BrickRec), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(B->d_bb, B->brick_base.data(), (n + 1) * sizeof(int64_t), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(B->d_tmp, 0, B->np * B->elem) != cudaSuccess)
        BT(fail(GPE_ERR_CUDA, "batch table upload failed"));
    if (B->relem == sizeof(double)) k_d2r<double><<<B->nsm * 8, 256>>>(B->d_V, (double *)B->d_Vr, B->np);
    else k_d2r<float><<<B->nsm * 8, 256>>>(B->d_V, (float *)B->d_Vr, B->np);
    count_launch();
    if (cudaDeviceSynchronize() != cudaSuccess) BT(fail(GPE_ERR_CUDA, "batch setup kernel failed"));
#undef BT
    for (int i = 0; i < n; ++i) states[i]->grid->n_states++;  // the batch keeps the grids alive
    *out = B;
    return GPE_OK;
}

extern "C" int gpe_batch_destroy(gpe_batch *B)
{
    if (!B) return GPE_OK;
    cudaDeviceSynchronize();
    for (gpe_state *s : B->states) s->grid->n_states--;
    batch_free(B);
    return GPE_OK;
}

namespace gpe {

template <typename R, typename CT, int BX, int BY, int BZ>
static int batch_record_block(gpe_batch *B, int64_t nsteps, cudaStream_t s)
{
    BatchArgs<R, CT> a;
    a.psi = (CT *)B->d_psi;
    a.tmp = (CT *)B->d_tmp;
    a.E = (const R *)B->d_E;
    a.V = (const R *)B->d_Vr;
    a.sh = B->d_sh;
    a.part = B->d_part;
    a.brick_base = B->d_bb;
    a.n = B->n;
    const GridView G{B->d_nbr, B->d_rec, B->d_rec7, B->nb};
    auto ka = k_batch_itp<R, CT, BX, BY, BZ, 0>;
    auto kb = k_batch_itp<R, CT, BX, BY, BZ, 1>;
    auto ko = k_batch_obs<R, CT, BX, BY, BZ>;
    const int th = KernelCfg<R>::THREADS;
    const size_t smem = smem_bytes<R, BX, BY, BZ, CT>();
    const int per = std::min(prepare_kernel(ka, th, smem), std::min(prepare_kernel(kb, th, smem), prepare_kernel(ko, th, smem)));
    const int64_t need = (B->nb + KernelCfg<R>::NW - 1) / KernelCfg<R>::NW;
    const int nblk = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)B->nsm * per, need));
    for (int64_t k = 0; k < nsteps; ++k) {
        ka<<<nblk, th, smem, s>>>(a, G);
        GPE_LAUNCH_CHECK();
        kb<<<nblk, th, smem, s>>>(a, G);
        GPE_LAUNCH_CHECK();
        k_batch_norm_finish<<<B->n, 256, 0, s>>>(B->d_sh, B->d_part, B->d_bb);
        GPE_LAUNCH_CHECK();
    }
    const int nseg = Seg<BX, BY, BZ>::NSEG;
    k_batch_apply_scale<CT><<<B->nsm * 8, 256, 0, s>>>((CT *)B->d_psi, B->d_rec, B->d_sh, B->nb, nseg);
    GPE_LAUNCH_CHECK();
    k_batch_reset_scale<<<(B->n + 255) / 256, 256, 0, s>>>(B->d_sh, B->n);
    GPE_LAUNCH_CHECK();
    k_zero_int<<<1, 1, 0, s>>>(B->d_unconv);
    GPE_LAUNCH_CHECK();
    ko<<<nblk, th, smem, s>>>(a, G);
    GPE_LAUNCH_CHECK();
    k_batch_obs_finish<<<B->n, 256, 0, s>>>(B->d_sh, B->d_part, B->d_bb, B->d_unconv);
    GPE_LAUNCH_CHECK();
    return GPE_OK;
}

static int batch_record(gpe_batch *B, int64_t nsteps, cudaStream_t s)
{
#define BATCH_CASE(id, X, Y, Z)                                                              \
    case id:                                                                                 \
        switch (B->dtype) {                                                                  \
        case GPE_C128: return batch_record_block<double, double2, X, Y, Z>(B, nsteps, s);    \
        case GPE_C64: return batch_record_block<float, float2, X, Y, Z>(B, nsteps, s);       \
        case GPE_R64: return batch_record_block<double, double, X, Y, Z>(B, nsteps, s);      \
        case GPE_R32: return batch_record_block<float, float, X, Y, Z>(B, nsteps, s);        \
        }                                                                                    \
        break;
    switch (B->shape) { GPE_SHAPES(BATCH_CASE) }
#undef BATCH_CASE
    return fail(GPE_ERR_STATE, "bad brick shape");
}

template <typename R>
static int batch_make_E(gpe_batch *B)
{
    k_batch_make_E<R><<<B->nsm * 8, 256>>>(B->d_V, (R *)B->d_E, B->d_rec, B->d_sh, B->nb);
    GPE_LAUNCH_CHECK();
    return GPE_OK;
}

}  // namespace gpe

extern "C" int gpe_batch_ground_state(gpe_batch *B, const gpe_imag_params *per_shell, double tol_dmu,
                                      int64_t check_every, int64_t max_steps, int32_t *converged, int64_t *steps,
                                      gpe_obs *obs, gpe_stream stream)
{
    if (!B || !per_shell) return fail(GPE_ERR_ARG, "NULL argument");
    if (check_every < 1 || max_steps < 1 || !(tol_dmu > 0))
        return fail(GPE_ERR_ARG, "need check_every >= 1, max_steps >= 1, tol_dmu > 0");
    int dev = -1;
    GPE_TRY_CUDA(cudaGetDevice(&dev));
    if (dev != B->device) return fail(GPE_ERR_STATE, "batch lives on device %d but device %d is current", B->device, dev);
    std::vector<ShellParams> sh(B->n);
    for (int i = 0; i < B->n; ++i) {
        const gpe_imag_params &p = per_shell[i];
        const gpe_box &b = B->states[i]->grid->box;
        if (!(p.dt > 0) || !(p.N > 0) || !std::isfinite(p.g) || !std::isfinite(p.dt) || !std::isfinite(p.N))
            return fail(GPE_ERR_ARG, "shell %d: need finite g, dt > 0, N > 0", i);
        const double lam = 2.0 / (b.hx * b.hx) + 2.0 / (b.hy * b.hy) + 2.0 / (b.hz * b.hz);
        if (p.dt * lam > 4.0) return fail(GPE_ERR_UNSTABLE, "shell %d: dt*lambda_max(T) = %.3g exceeds 4", i, p.dt * lam);
        ShellParams &P = sh[i];
        memset(&P, 0, sizeof P);
        P.g = p.g;
        P.dt = p.dt;
        P.N = p.N;
        P.dV = b.hx * b.hy * b.hz;
        P.ihx2 = 1.0 / (b.hx * b.hx);
        P.ihy2 = 1.0 / (b.hy * b.hy);
        P.ihz2 = 1.0 / (b.hz * b.hz);
        P.scale = 1.0;
        P.tol = tol_dmu;
    }
    cudaStream_t s = S(stream);
    GPE_TRY_CUDA(cudaMemcpyAsync(B->d_sh, sh.data(), B->n * sizeof(ShellParams), cudaMemcpyHostToDevice, s));
    for (int i = 0; i < B->n; ++i)
        GPE_TRY_CUDA(cudaMemcpyAsync((char *)B->d_psi + B->packed_base[i] * B->elem, B->states[i]->d_psi,
                                     B->states[i]->grid->n_packed * B->elem, cudaMemcpyDeviceToDevice, s));
    GPE_TRY_CUDA(cudaStreamSynchronize(s));
    GPE_TRY(B->relem == sizeof(double) ? batch_make_E<double>(B) : batch_make_E<float>(B));
    GPE_TRY_CUDA(cudaDeviceSynchronize());
    // one graph per (block length) replayed until every shell converged
    const uint64_t key = (uint64_t)check_every;
    if (!B->exec || B->key != key) {
        if (B->exec) {
            cudaGraphExecDestroy(B->exec);
            B->exec = nullptr;
        }
        if (!B->cap) GPE_TRY_CUDA(cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking));
        GPE_TRY_CUDA(cudaStreamBeginCapture(B->cap, cudaStreamCaptureModeThreadLocal));
        int rc = batch_record(B, check_every, B->cap);
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(B->cap, &graph);
        if (rc != GPE_OK) {
            if (graph) cudaGraphDestroy(graph);
            return rc;
        }
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture", __FILE__, __LINE__);
        e = cudaGraphInstantiate(&B->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate", __FILE__, __LINE__);
        B->key = key;
    }
    int64_t done = 0;
    const int nodes = (int)(3 * check_every + 5);
    int unconv = B->n;
    while (done < max_steps && unconv > 0) {
        GPE_TRY_CUDA(cudaGraphLaunch(B->exec, s));
        for (int k = 0; k < nodes; ++k) count_launch();
        done += check_every;
        GPE_TRY_CUDA(cudaMemcpyAsync(B->h_unconv, B->d_unconv, sizeof(int), cudaMemcpyDeviceToHost, s));
        GPE_TRY_CUDA(cudaStreamSynchronize(s));
        unconv = *B->h_unconv;
    }
    // results back to the states and to the caller
    for (int i = 0; i < B->n; ++i)
        GPE_TRY_CUDA(cudaMemcpyAsync(B->states[i]->d_psi, (char *)B->d_psi + B->packed_base[i] * B->elem,
                                     B->states[i]->grid->n_packed * B->elem, cudaMemcpyDeviceToDevice, s));
    GPE_TRY_CUDA(cudaMemcpyAsync(sh.data(), B->d_sh, B->n * sizeof(ShellParams), cudaMemcpyDeviceToHost, s));
    GPE_TRY_CUDA(cudaStreamSynchronize(s));
    int n_bad = 0, n_unconv = 0;
    for (int i = 0; i < B->n; ++i) {
        const ShellParams &P = sh[i];
        if (converged) converged[i] = P.converged && P.nonfinite == 0;
        if (steps) steps[i] = P.steps;
        if (obs) {
            obs[i].norm = P.norm;
            obs[i].energy = P.energy;
            obs[i].mu = P.mu;
            obs[i].nonfinite = P.nonfinite;
            obs[i].e_kin = P.e_kin;
            obs[i].e_pot = P.e_pot;
            obs[i].e_int = P.e_int;
        }
        if (P.nonfinite > 0) ++n_bad;
        else if (!P.converged) ++n_unconv;
    }
    (void)done;
    if (n_bad) return fail(GPE_ERR_NONFINITE, "%d shell(s) hold NaN or Inf", n_bad);
    if (n_unconv) return fail(GPE_ERR_NOT_CONVERGED, "%d shell(s) did not reach |dmu| < %g", n_unconv, tol_dmu);
    return GPE_OK;
}
