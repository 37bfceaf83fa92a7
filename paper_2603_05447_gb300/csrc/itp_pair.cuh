// itp_pair.cuh -- the imaginary-time step (Sec. II A, Eqs. (6)-(7)) in one
// pass per step instead of two.
//
// The staged step makes two stencil passes over the state (kernels.cuh):
// pass A applies the pending renormalisation factor and the first diagonal
// half step while it gathers psi, then takes the first Euler substep of the
// kinetic part into tmp; pass B takes the second Euler substep, the second
// diagonal half step and the FP64 norm.  Pass B's Laplacian needs the first
// substep on the brick's one-cell face halo, which needs psi on a two-cell
// face halo and the one-cell edge halo: the tile of the fused-pair RK4 block
// (pair.cuh).  One block of two warps per brick:
//  * stages psi in that tile and, beside it, the propagator table E of the
//    same cells, by cp.async;
//  * applies the factor and the half step to the whole tile in place;
//  * takes the first substep on the brick and its one-deep face halo into
//    the second tile (zero on inactive cells, as pass A writes them);
//  * takes the second substep, the half step and the norm on the brick.
// Compulsory traffic per stored cell: psi and E in, psi out (20 bytes in
// complex64) against 40 for the two passes.  psi is read at halo cells of
// other bricks, so the result goes to a second buffer and the state
// alternates between two buffers from step to step.
//
// The per-cell arithmetic is the staged kernels' (DiagLoad::apply, lapv,
// axpy), so before the final factor the two schedules agree bit for bit;
// the norm is summed in another order, so the factor can differ in its last
// bit.  Complex states only (a real float segment is a single 16-byte unit,
// which the tile's x halo layout does not split).
#pragma once

#include "kernels.cuh"
#include "pair.cuh"

namespace gpe {

// 8-byte asynchronous global -> shared copy (valid == false writes zeros)
__device__ __forceinline__ void cp_async8(void *dst, const void *src, bool valid)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 8 : 0) : "memory");
}

template <typename CT, int BX, int BY, int BZ>
struct ItpPairSpace {
    using R = typename RealOf<CT>::T;
    using PS = PairSpace<CT, BX, BY, BZ>;
    static constexpr int EUPS = (int)(4 * sizeof(R) / 16);  // 16-byte units of E per segment
    static constexpr int NROW = PS::TY * PS::TZ;
    PS ps;
    uint4 e[EUPS][PS::PSTR];      // E of the u slots (zero where u was zeroed)
    alignas(16) R exl[NROW][2];   // E at x = -2, -1 of each u row
    alignas(16) R exr[NROW][2];   // E at x = BX, BX + 1
    __device__ __forceinline__ void eget(int s, R (&e4)[4]) const
    {
#pragma unroll
        for (int k = 0; k < EUPS; ++k) {
            const uint4 w = e[k][s];
            const R *p = reinterpret_cast<const R *>(&w);
#pragma unroll
            for (int i = 0; i < 4 / EUPS; ++i) e4[k * (4 / EUPS) + i] = p[i];
        }
    }
};

// pair_fill hook: E of every staged segment and x halo pair of cells
template <typename CT, int BX, int BY, int BZ>
struct EFill {
    using SP = ItpPairSpace<CT, BX, BY, BZ>;
    using R = typename SP::R;
    SP *sp;
    const R *E;
    __device__ __forceinline__ void units(int sl, bool ok, uint32_t j) const
    {
        const char *g = reinterpret_cast<const char *>(E + (ok ? j : 0u));
#pragma unroll
        for (int k = 0; k < SP::EUPS; ++k) cp_async16(&sp->e[k][sl], g + 16 * k, ok);
    }
    __device__ __forceinline__ void own(int sl, bool ok, uint32_t j) const { units(sl, ok, j); }
    __device__ __forceinline__ void seg(int sl, const BrickRec &r, int q) const
    {
        uint32_t j = 0;
        const bool ok = seg_index(r, q, j);
        units(sl, ok, j);
    }
    // side 0: cells 2, 3 of the segment (x = -2, -1); side 1: cells 0, 1
    __device__ __forceinline__ void xh(int side, int row, const BrickRec &r, int q) const
    {
        uint32_t j = 0;
        const bool ok = seg_index(r, q, j);
        const R *g = E + (ok ? j + (side == 0 ? 2u : 0u) : 0u);
        R *dst = side == 0 ? sp->exl[row] : sp->exr[row];
        if constexpr (sizeof(R) == 4)
            cp_async8(dst, g, ok);
        else
            cp_async16(dst, g, ok);
    }
};

// One imaginary-time step of brick b: src -> out, the norm of its cells
// added to acc
template <typename R, int BX, int BY, int BZ>
__device__ __forceinline__ void itp_pair_brick(ItpPairSpace<typename Cx<R>::T, BX, BY, BZ> &sp, const PairView &P,
                                               const ItpArgs<R> &a, int64_t b, R sc, double &acc)
{
    using CT = typename Cx<R>::T;
    using SP = ItpPairSpace<CT, BX, BY, BZ>;
    using PS = PairSpace<CT, BX, BY, BZ>;
    constexpr int SX = PS::SX, PL = PS::PLANE_B;
    auto &ps = sp.ps;
    const int t = threadIdx.x;
    const R c6 = (R)2 * (a.ihx2 + a.ihy2 + a.ihz2);
    const R q4 = a.dt / (R)4, hg = a.g * a.dt / (R)2;
    pair_fill(ps, P, b, a.psi, EFill<CT, BX, BY, BZ>{&sp, a.E});
    for (int i = t; i < PS::UPS * PS::VPSTR; i += PAIR_THREADS) (&ps.v[0][0])[i] = make_uint4(0, 0, 0, 0);
    for (int i = t; i < BY * BZ; i += PAIR_THREADS) {
        ps.vxl[i] = czero<CT>();
        ps.vxr[i] = czero<CT>();
    }
    cp_async_wait_all();
    __syncthreads();
    // the pending factor and the first diagonal half step on every staged
    // cell (slots and rows the fill left unwritten are never read)
    const DiagLoad<R, CT> diag{sc, hg, a.E};
    for (int s = t; s < PS::NSLOT; s += PAIR_THREADS) {
        CT c[4];
        R e4[4];
        ps.uget(s, c);
        sp.eget(s, e4);
#pragma unroll
        for (int k = 0; k < PS::UPS; ++k) {
            uint4 w;
            CT *p = reinterpret_cast<CT *>(&w);
#pragma unroll
            for (int i = 0; i < PS::CPU_; ++i) p[i] = diag.apply(c[k * PS::CPU_ + i], e4[k * PS::CPU_ + i]);
            ps.u[k][s] = w;
        }
    }
    for (int i = t; i < 2 * SP::NROW; i += PAIR_THREADS) {
        const int side = i / SP::NROW, r = i % SP::NROW;
        CT *u = side == 0 ? ps.uxl[r] : ps.uxr[r];
        const R *e = side == 0 ? sp.exl[r] : sp.exr[r];
        u[0] = diag.apply(u[0], e[0]);
        u[1] = diag.apply(u[1], e[1]);
    }
    __syncthreads();
    const int nst = ps.nst;
    const BrickRec &R0 = ps.rec[0];
    // first Euler substep on the brick's stored segments and on the stored
    // segments of the one-deep z and y face layers
    const int ntask = nst + 2 * PL + 2 * SX * BZ;
    for (int i = t; i < ntask; i += PAIR_THREADS) {
        int hx, y, z;
        bool ok = true;
        uint32_t j = 0;
        if (i < nst) {
            const int q = ps.list[i];
            hx = q % SX;
            y = (q / SX) % BY;
            z = q / PL;
        } else if (i < nst + 2 * PL) {
            const int s = (i - nst) % PL, f = (i - nst) / PL;
            hx = s % SX;
            y = s / SX;
            z = f == 0 ? -1 : BZ;
            ok = seg_index(ps.rec[5 + f], hx + SX * y + PL * (f == 0 ? BZ - 1 : 0), j);
        } else {
            const int s = (i - nst - 2 * PL) % (SX * BZ), f = (i - nst - 2 * PL) / (SX * BZ);
            hx = s % SX;
            z = s / SX;
            y = f == 0 ? -1 : BY;
            ok = seg_index(ps.rec[3 + f], hx + SX * (f == 0 ? BY - 1 : 0) + PL * z, j);
        }
        if (!ok) continue;
        CT c[4], L[4], o[4];
        R e4[4];
        pair_lap_u(ps, hx, y, z, c, L, a.ihx2, a.ihy2, a.ihz2, c6);
        sp.eget(PS::slot(hx, y, z), e4);
#pragma unroll
        for (int k = 0; k < 4; ++k) o[k] = e4[k] >= (R)0 ? axpy(c[k], q4, L[k]) : czero<CT>();
        ps.vput(PS::vslot(hx, y, z), o);
    }
    // the same on the single cells of the one-deep x face layers
    for (int i = t; i < 2 * BY * BZ; i += PAIR_THREADS) {
        const int side = i / (BY * BZ), rr = i % (BY * BZ);
        const int y = rr % BY, z = rr / BY;
        uint32_t j;
        if (!seg_index(ps.rec[1 + side], (side == 0 ? SX - 1 : 0) + SX * y + PL * z, j)) continue;
        CT c0, xm, xp, ym, yp, zm, zp;
        R e;
        const int h = PS::row(y, z);
        if (side == 0) {
            c0 = ps.uxl[h][1];
            e = sp.exl[h][1];
            xm = ps.uxl[h][0];
            xp = ps.ucell(PS::slot(0, y, z), 0);
            ym = ps.uxl[PS::row(y - 1, z)][1];
            yp = ps.uxl[PS::row(y + 1, z)][1];
            zm = ps.uxl[PS::row(y, z - 1)][1];
            zp = ps.uxl[PS::row(y, z + 1)][1];
        } else {
            c0 = ps.uxr[h][0];
            e = sp.exr[h][0];
            xm = ps.ucell(PS::slot(SX - 1, y, z), 3);
            xp = ps.uxr[h][1];
            ym = ps.uxr[PS::row(y - 1, z)][0];
            yp = ps.uxr[PS::row(y + 1, z)][0];
            zm = ps.uxr[PS::row(y, z - 1)][0];
            zp = ps.uxr[PS::row(y, z + 1)][0];
        }
        const CT L = lapv(xp, xm, yp, ym, zp, zm, c0, a.ihx2, a.ihy2, a.ihz2, c6);
        (side == 0 ? ps.vxl : ps.vxr)[PS::vrow(y, z)] = e >= (R)0 ? axpy(c0, q4, L) : czero<CT>();
    }
    __syncthreads();
    // second Euler substep, second half step and the norm on the brick
    for (int i = t; i < nst; i += PAIR_THREADS) {
        const int q = ps.list[i];
        const int hx = q % SX, y = (q / SX) % BY, z = q / PL;
        CT c[4], L[4], o[4];
        R e4[4];
        R n4 = (R)0;  // the segment's |psi|^2, added to the FP64 sum once
        pair_lap_v(ps, hx, y, z, c, L, a.ihx2, a.ihy2, a.ihz2, c6);
        sp.eget(PS::slot(hx, y, z), e4);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            o[k] = axpy(c[k], q4, L[k]);
            const R f = e4[k] >= (R)0 ? e4[k] * ((R)1 - hg * norm2(o[k])) : (R)0;
            o[k] = scale(o[k], f);
            n4 = add_rn(n4, norm2(o[k]));
        }
        acc += (double)n4;
        st4(a.tmp + R0.off + 4u * (uint32_t)i, o);
    }
    __syncthreads();  // the tiles are reused for the next brick
}

// One imaginary-time step over every brick: a.psi -> a.tmp (the caller
// swaps the buffers between steps); the last block to finish stores the
// next factor sqrt(N / norm) and the norm in a.scalars
template <typename R, int BX, int BY, int BZ>
__global__ void __launch_bounds__(PAIR_THREADS) k_itp_fused(const ItpArgs<R> a, const PairView P, double *partials,
                                                            unsigned int *counter)
{
    using CT = typename Cx<R>::T;
    extern __shared__ __align__(16) unsigned char gpe_smem[];
    auto &sp = *reinterpret_cast<ItpPairSpace<CT, BX, BY, BZ> *>(gpe_smem);
    const R sc = (R)a.scalars[0];
    double acc[1] = {0.0};
    for (int64_t b = blockIdx.x; b < P.nb; b += gridDim.x) itp_pair_brick<R, BX, BY, BZ>(sp, P, a, b, sc, acc[0]);
    double tot[1];
    if (reduce_finish<1>(acc, partials, counter, tot) && threadIdx.x == 0) {
        const double nrm = tot[0] * a.dV;
        a.scalars[0] = sqrt(a.N / nrm);
        a.scalars[1] = nrm;
    }
}

}  // namespace gpe
