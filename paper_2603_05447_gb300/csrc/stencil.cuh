// stencil.cuh -- device building blocks shared by the stencil kernels of
// libgpeshell (steps, batches, adjoint): the packed segment layout, the
// warp-per-brick gather of a segment's 7-point Laplacian (Eq. (B1)), the ramp
// schedule and small reductions.  Not part of the ABI.
#pragma once

#include "gpe_internal.cuh"

namespace gpe {

// The warps of a block share the per-warp record slots below.
constexpr int WARPS = 8;  // blocks of 256 threads, one brick per warp at a time

// Minimum resident blocks per SM requested from the register allocator for
// the stencil kernels (complex64 / complex128 bulk).
#ifndef GPE_MINB_F
#define GPE_MINB_F 2
#endif
#ifndef GPE_MINB_D
#define GPE_MINB_D 1
#endif
#define GPE_BOUNDS(R) __launch_bounds__(256, (sizeof(R) == 4 ? GPE_MINB_F : GPE_MINB_D))

// ------------------------------------------------------------ packed layout
// supported brick shapes (shape id, BX, BY, BZ)
#define GPE_SHAPES(M) \
    M(0, 8, 8, 8)     \
    M(1, 8, 8, 4)     \
    M(2, 8, 4, 4)

struct GridView {
    const int32_t *nbr;
    const BrickRec *rec;
    int64_t nb;
};

inline GridView view(const gpe_grid *g) { return GridView{g->d_nbr, g->d_rec, g->nb}; }

// segment geometry of a brick shape (BX must be 8: two segments per row)
template <int BX, int BY, int BZ>
struct Seg {
    static_assert(BX == 8, "bricks are 8 cells long in x");
    static constexpr int SX = BX / 4;          // segments per x-row
    static constexpr int PLANE = SX * BY;      // segments per z-plane (divides 32)
    static constexpr int NSEG = PLANE * BZ;    // segments per brick
    static constexpr int NIT = NSEG / 32;      // warp iterations per brick
    static_assert(32 % PLANE == 0 && NSEG % 32 == 0, "brick shape must tile the warp");
};

template <typename CT>
__device__ __forceinline__ CT czero()
{
    CT z;
    z.x = 0;
    z.y = 0;
    return z;
}

__device__ __forceinline__ float2 shfl_up(float2 v, int d)
{
    v.x = __shfl_up_sync(0xffffffffu, v.x, d);
    v.y = __shfl_up_sync(0xffffffffu, v.y, d);
    return v;
}
__device__ __forceinline__ double2 shfl_up(double2 v, int d)
{
    v.x = __shfl_up_sync(0xffffffffu, v.x, d);
    v.y = __shfl_up_sync(0xffffffffu, v.y, d);
    return v;
}
__device__ __forceinline__ float2 shfl_down(float2 v, int d)
{
    v.x = __shfl_down_sync(0xffffffffu, v.x, d);
    v.y = __shfl_down_sync(0xffffffffu, v.y, d);
    return v;
}
__device__ __forceinline__ double2 shfl_down(double2 v, int d)
{
    v.x = __shfl_down_sync(0xffffffffu, v.x, d);
    v.y = __shfl_down_sync(0xffffffffu, v.y, d);
    return v;
}
__device__ __forceinline__ float2 shfl_xor(float2 v, int d)
{
    v.x = __shfl_xor_sync(0xffffffffu, v.x, d);
    v.y = __shfl_xor_sync(0xffffffffu, v.y, d);
    return v;
}
__device__ __forceinline__ double2 shfl_xor(double2 v, int d)
{
    v.x = __shfl_xor_sync(0xffffffffu, v.x, d);
    v.y = __shfl_xor_sync(0xffffffffu, v.y, d);
    return v;
}

// 4 consecutive complex values (one segment); CG: read through L2 only
// (data written by other blocks of the same launch)
template <bool CG>
__device__ __forceinline__ void ld4(const float2 *p, float2 (&v)[4])
{
    const float4 *q = reinterpret_cast<const float4 *>(p);
    const float4 a = CG ? __ldcg(q) : q[0], b = CG ? __ldcg(q + 1) : q[1];
    v[0] = make_float2(a.x, a.y);
    v[1] = make_float2(a.z, a.w);
    v[2] = make_float2(b.x, b.y);
    v[3] = make_float2(b.z, b.w);
}
template <bool CG>
__device__ __forceinline__ void ld4(const double2 *p, double2 (&v)[4])
{
#pragma unroll
    for (int i = 0; i < 4; ++i) v[i] = CG ? __ldcg(p + i) : p[i];
}
__device__ __forceinline__ void st4(float2 *p, const float2 (&v)[4])
{
    float4 *q = reinterpret_cast<float4 *>(p);
    q[0] = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
    q[1] = make_float4(v[2].x, v[2].y, v[3].x, v[3].y);
}
__device__ __forceinline__ void st4(double2 *p, const double2 (&v)[4])
{
#pragma unroll
    for (int i = 0; i < 4; ++i) p[i] = v[i];
}
__device__ __forceinline__ void ldr4(const float *p, float (&v)[4])
{
    const float4 a = __ldg(reinterpret_cast<const float4 *>(p));
    v[0] = a.x;
    v[1] = a.y;
    v[2] = a.z;
    v[3] = a.w;
}
__device__ __forceinline__ void ldr4(const double *p, double (&v)[4])
{
    const double2 a = __ldg(reinterpret_cast<const double2 *>(p)), b = __ldg(reinterpret_cast<const double2 *>(p) + 1);
    v[0] = a.x;
    v[1] = a.y;
    v[2] = b.x;
    v[3] = b.y;
}

struct Identity {
    template <typename CT>
    __device__ __forceinline__ CT operator()(CT v, uint32_t) const { return v; }
};

// Records of brick b (slot 0) and of its six face neighbours (slots 1..6,
// order -x +x -y +y -z +z; an absent neighbour gets an empty record), loaded by
// one warp into its shared-memory slots.
__device__ __forceinline__ void load_recs(BrickRec *R, const GridView &G, int64_t b)
{
    const int lane = threadIdx.x & 31;
    __syncwarp();
    if (lane < 7) {
        const int64_t id = lane == 0 ? b : (int64_t)__ldg(&G.nbr[b * 6 + lane - 1]);
        uint4 a = make_uint4(0, 0, 0, 0), c = make_uint4(0, 0, 0, 0);
        if (id >= 0) {
            const uint4 *p = reinterpret_cast<const uint4 *>(G.rec + id);
            a = __ldg(p);
            c = __ldg(p + 1);
        }
        uint4 *d = reinterpret_cast<uint4 *>(R + lane);
        d[0] = a;
        d[1] = c;
    }
    __syncwarp();
}

// One lane's segment q of a brick: its four values c[] and their 7-point
// Laplacians L[] (Eq. (B1)), every loaded value passed through xf first.
// All 32 lanes must call this together: x and y neighbours inside the brick
// come from other lanes by shuffles; z neighbours and brick-boundary
// neighbours are loaded.  Every load of the lane is issued before the first
// shuffle so that they are in flight together.
template <bool CG, typename CT>
__device__ __forceinline__ CT ld1(const CT *p)
{
    return CG ? __ldcg(p) : *p;
}

template <int BX, int BY, int BZ, bool CG, typename CT, typename R, typename XF>
__device__ __forceinline__ void gather(const CT *src, const BrickRec *Rr, int q, bool stored, uint32_t idx, XF xf,
                                       R ihx2, R ihy2, R ihz2, CT (&c)[4], CT (&L)[4])
{
    using S = Seg<BX, BY, BZ>;
    const int hx = q % S::SX, y = (q / S::SX) % BY, z = q / S::PLANE;
    // neighbour segments that live in memory
    uint32_t jzm = 0, jzp = 0, jy = 0, jx = 0;
    const bool hzm = stored && (z == 0 ? seg_index(Rr[5], q + S::PLANE * (BZ - 1), jzm)
                                       : seg_index(Rr[0], q - S::PLANE, jzm));
    const bool hzp = stored && (z == BZ - 1 ? seg_index(Rr[6], q - S::PLANE * (BZ - 1), jzp)
                                            : seg_index(Rr[0], q + S::PLANE, jzp));
    const bool ylo = (y == 0), yhi = (y == BY - 1);
    const bool hy = stored && (ylo ? seg_index(Rr[3], hx + S::SX * (BY - 1) + S::PLANE * z, jy)
                                   : (yhi && seg_index(Rr[4], hx + S::PLANE * z, jy)));
    // x: segment (1, y, z) of the -x brick (cell x = 7) or (0, y, z) of the +x brick (cell x = 0)
    const bool hxb = stored && (hx == 0 ? seg_index(Rr[1], q + 1, jx) : seg_index(Rr[2], q - 1, jx));
    if (hx == 0) jx += 3;
    CT zm[4], zp[4], yb[4], xb = czero<CT>();
#pragma unroll
    for (int i = 0; i < 4; ++i) c[i] = zm[i] = zp[i] = yb[i] = czero<CT>();
    if (stored) ld4<CG>(src + idx, c);
    if (hzm) ld4<CG>(src + jzm, zm);
    if (hzp) ld4<CG>(src + jzp, zp);
    if (hy) ld4<CG>(src + jy, yb);
    if (hxb) xb = ld1<CG>(src + jx);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        if (stored) c[i] = xf(c[i], idx + i);
        if (hzm) zm[i] = xf(zm[i], jzm + i);
        if (hzp) zp[i] = xf(zp[i], jzp + i);
        if (hy) yb[i] = xf(yb[i], jy + i);
    }
    if (hxb) xb = xf(xb, jx);
    CT ym[4], yp[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        ym[i] = shfl_up(c[i], S::SX);
        yp[i] = shfl_down(c[i], S::SX);
        if (ylo) ym[i] = yb[i];
        if (yhi) yp[i] = yb[i];
    }
    const CT p0 = shfl_xor(c[0], 1), p3 = shfl_xor(c[3], 1);
    const CT xm = hx == 0 ? xb : p3;  // left of cell 0
    const CT xp = hx == 0 ? p0 : xb;  // right of cell 3
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const CT l = i == 0 ? xm : c[i - 1];
        const CT r = i == 3 ? xp : c[i + 1];
        L[i].x = (r.x - 2 * c[i].x + l.x) * ihx2 + (yp[i].x - 2 * c[i].x + ym[i].x) * ihy2 +
                 (zp[i].x - 2 * c[i].x + zm[i].x) * ihz2;
        L[i].y = (r.y - 2 * c[i].y + l.y) * ihx2 + (yp[i].y - 2 * c[i].y + ym[i].y) * ihy2 +
                 (zp[i].y - 2 * c[i].y + zm[i].y) * ihz2;
    }
}

// ------------------------------------------------------------ ramp schedule
struct Ramp {
    const double *clock;  // device time base
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

template <typename R>
struct DiagLoad {
    using CT = typename Cx<R>::T;
    R sc, hg;
    const R *E;
    __device__ __forceinline__ CT operator()(CT v, uint32_t idx) const
    {
        v.x *= sc;
        v.y *= sc;
        const R e = __ldg(E + idx);
        const R f = e >= (R)0 ? e * ((R)1 - hg * (v.x * v.x + v.y * v.y)) : (R)0;
        v.x *= f;
        v.y *= f;
        return v;
    }
};

// deterministic block sum (result valid in thread 0)
__device__ __forceinline__ double block_sum(double x)
{
    __shared__ double sm[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
    __syncthreads();
    if (lane == 0) sm[warp] = x;
    __syncthreads();
    x = 0.0;
    if (warp == 0) {
        x = lane < nw ? sm[lane] : 0.0;
        for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
    }
    return x;
}

// ------------------------------------------------------------ RK4 stages
// Memory-optimised RK4 (App. A, RK4 a* and b*): the stage states are stored
// instead of the k_i, so stage i reads only the state it differentiates (with
// halo) plus the own-cell values of earlier states:
//   stage 0: y2 = y0 + dt/2 f(t, y0)
//   stage 1: y3 = y0 + dt/2 f(t + dt/2, y2)
//   stage 2: y4 = y0 + dt   f(t + dt/2, y3)
//   stage 3: y1 = (-y0 + y2 + 2 y3 + y4)/3 + dt/6 f(t + dt, y4)  (in place of y0)
// with f(t, y) = -i [ -1/2 lap y + (V(t) + g|y|^2) y ]  (Eq. (8)).
template <typename R>
struct RkArgs {
    using CT = typename Cx<R>::T;
    CT *y0;
    CT *y2;
    CT *y3;
    CT *y4;
    const R *V0;
    const R *V1;
    R ihx2, ihy2, ihz2, g, dt;
    Ramp ramp;
    double t_off;  // stage-0 time of this step relative to *ramp.clock
    double dtd;    // dt in FP64 for stage times
};

template <typename R, bool BLEND>
__device__ __forceinline__ R stage_s(const RkArgs<R> &a, int st)
{
    if (!BLEND) return (R)0;
    const double c = (st == 0) ? 0.0 : (st == 3 ? 1.0 : 0.5);
    return (R)ramp_s(a.ramp, *a.ramp.clock + a.t_off + c * a.dtd);
}

// One RK4 stage on brick b, one warp, lane = segment within each group of 32.
template <typename R, int BX, int BY, int BZ, bool BLEND, bool CG>
__device__ __forceinline__ void rk4_brick(const RkArgs<R> &a, const GridView &G, int st, int64_t b, BrickRec *Rr,
                                          R s)
{
    using S = Seg<BX, BY, BZ>;
    using CT = typename Cx<R>::T;
    const CT *yin = st == 0 ? a.y0 : st == 1 ? a.y2 : st == 2 ? a.y3 : a.y4;
    CT *yout = st == 0 ? a.y2 : st == 1 ? a.y3 : st == 2 ? a.y4 : a.y0;
    const R k = (st == 2) ? a.dt : (st == 3 ? a.dt / (R)6 : a.dt / (R)2);
    load_recs(Rr, G, b);
    const int lane = threadIdx.x & 31;
#pragma unroll 1
    for (int it = 0; it < S::NIT; ++it) {
        const int q = it * 32 + lane;
        uint32_t idx = 0;
        const bool stored = seg_index(Rr[0], q, idx);
        R V0[4], V1[4];
        CT y0[4], y2[4], y3[4];
        if (stored) {
            ldr4(a.V0 + idx, V0);
            if (BLEND) ldr4(a.V1 + idx, V1);
            if (st > 0) ld4<CG>(a.y0 + idx, y0);
            if (st == 3) {
                ld4<CG>(a.y2 + idx, y2);
                ld4<CG>(a.y3 + idx, y3);
            }
        }
        CT c[4], L[4];
        gather<BX, BY, BZ, CG>(yin, Rr, q, stored, idx, Identity(), a.ihx2, a.ihy2, a.ihz2, c, L);
        if (!stored) continue;
        CT o[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            if (!(V0[i] < (R)INFINITY)) {  // inactive cell of a stored segment
                o[i] = czero<CT>();
                continue;
            }
            const R V = BLEND ? ((R)1 - s) * V0[i] + s * V1[i] : V0[i];
            const R w = V + a.g * (c[i].x * c[i].x + c[i].y * c[i].y);
            const R hr = (R)(-0.5) * L[i].x + w * c[i].x;
            const R hi = (R)(-0.5) * L[i].y + w * c[i].y;
            // f = -i (hr + i hi) = hi - i hr
            if (st == 0) {
                o[i].x = c[i].x + k * hi;
                o[i].y = c[i].y - k * hr;
            } else if (st < 3) {
                o[i].x = y0[i].x + k * hi;
                o[i].y = y0[i].y - k * hr;
            } else {
                o[i].x = (-y0[i].x + y2[i].x + (R)2 * y3[i].x + c[i].x) / (R)3 + k * hi;
                o[i].y = (-y0[i].y + y2[i].y + (R)2 * y3[i].y + c[i].y) / (R)3 - k * hr;
            }
        }
        st4(yout + idx, o);
    }
}

template <typename R, int BX, int BY, int BZ, bool BLEND>
__global__ void GPE_BOUNDS(R) k_rk4_staged(const RkArgs<R> a, const GridView G, int st)
{
    __shared__ BrickRec s_rec[WARPS][7];
    const int warp = threadIdx.x >> 5;
    const R s = stage_s<R, BLEND>(a, st);
    for (int64_t b = (int64_t)blockIdx.x * WARPS + warp; b < G.nb; b += (int64_t)gridDim.x * WARPS)
        rk4_brick<R, BX, BY, BZ, BLEND, false>(a, G, st, b, s_rec[warp], s);
}

}  // namespace gpe
