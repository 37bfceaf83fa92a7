// pair.cuh -- RK4 with two stages fused per pass: stages 0+1, then 2+3.
//
// The staged kernels make four passes over the state per RK4 step, and their
// compulsory traffic is 112 bytes per stored cell (complex64): each stage
// reads its input with a halo, the potential and one or two own-cell states,
// and writes its output.  A pass that computes two stages keeps the middle
// stage in shared memory instead:
//   pass 1: u = y0;  stage A: y2 = y0 + dt/2 f(t, y0)        (brick + face halo)
//                    stage B: y3 = y0 + dt/2 f(t + dt/2, y2), w = -y0 + y2 + 2 y3
//   pass 2: u = y3;  stage A: y4 = y0 + dt f(t + dt/2, y3)   (brick + face halo)
//                    stage B: y1 = (w + y4)/3 + dt/6 f(t + dt, y4)
// (the memory-optimised stages of App. A, as in Rk4Body).  Stage B's
// Laplacian needs stage A on the brick and its one-cell face halo, which in
// turn needs u on a two-cell face halo and the one-cell edge halo; the halo
// values of stage A are recomputed by every brick that needs them.  The
// compulsory traffic falls to 28 + 36 = 64 bytes per stored cell.  Pass 2
// reads y0 at halo cells of other bricks, so y1 goes to a second buffer (the
// state alternates between two buffers from step to step).
//
// One block of two warps per brick.  The block stages in shared memory:
//  * u: the brick's segments with a two-deep face halo in y and z (whole
//    segments, from the face neighbours) and the one-deep y-z edge rows; per
//    row the two cells on either side in x (x = -2, -1 and BX, BX+1, from the
//    x-face and the xy/xz-edge neighbours); filled by cp.async;
//  * v: stage A on the brick and its one-deep face halo (the layout of the
//    staged kernels' tile), written by the block's threads;
//  * the records of the brick, its 6 face and 12 edge neighbours, looked up
//    through the per-brick neighbour ids (the 32-byte records stay in L2).
// Stage A runs as three task sets: the brick's stored segments, the stored
// segments of the one-deep z and y face layers, and the single cells of the
// one-deep x face layers.  The arithmetic per cell is that of the staged
// kernels (lapv, Rk4Body::compute), so both schedules give identical bits.
#pragma once

#include "stencil.cuh"

namespace gpe {

constexpr int PAIR_THREADS = 64;  // threads (two warps) per brick

struct PairView {
    const BrickRec *rec;    // per-brick records
    const int32_t *nbr18;   // per brick: -x +x -y +y -z +z, then the 12 edges (build_rec19 order); -1 = none
    int64_t nb;
};

template <typename CT, int BX, int BY, int BZ>
struct PairSpace {
    using S = Seg<BX, BY, BZ>;
    static constexpr int SX = S::SX, PLANE_B = S::PLANE;
    static constexpr int UPS = (int)(4 * sizeof(CT) / 16);  // 16-byte units per segment
    static constexpr int CPU_ = 4 / UPS;                    // cells per unit
    static constexpr int NXU = 2 / CPU_;                    // units holding two cells
    // u: y in [-2, BY+1], z in [-2, BZ+1]
    static constexpr int TY = BY + 4, TZ = BZ + 4, NSLOT = SX * TY * TZ;
    static constexpr int PSTR = NSLOT + (((UPS == 2 ? 4 : 2) - NSLOT % 8) + 8) % 8;
    static constexpr int ROW = SX, PLANE = SX * TY;
    // v: y in [-1, BY], z in [-1, BZ]
    static constexpr int VTY = BY + 2, VTZ = BZ + 2, VNSLOT = SX * VTY * VTZ;
    static constexpr int VPSTR = VNSLOT + (((UPS == 2 ? 4 : 2) - VNSLOT % 8) + 8) % 8;
    static constexpr int VROW = SX, VPLANE = SX * VTY;
    __device__ __forceinline__ static int slot(int hx, int y, int z) { return hx + SX * ((y + 2) + TY * (z + 2)); }
    __device__ __forceinline__ static int row(int y, int z) { return (y + 2) + TY * (z + 2); }
    __device__ __forceinline__ static int vslot(int hx, int y, int z) { return hx + SX * ((y + 1) + VTY * (z + 1)); }
    __device__ __forceinline__ static int vrow(int y, int z) { return y + BY * z; }

    uint4 u[UPS][PSTR];
    CT uxl[TY * TZ][2];  // per u row: x = -2, -1
    CT uxr[TY * TZ][2];  // per u row: x = BX, BX + 1
    uint4 v[UPS][VPSTR];
    CT vxl[BY * BZ];     // v at x = -1 (brick rows)
    CT vxr[BY * BZ];     // v at x = BX
    alignas(16) BrickRec rec[19];
    uint16_t list[S::NSEG];  // the brick's stored segments in order (local segment number)
    int nst;

    __device__ __forceinline__ void get(const uint4 (*t)[PSTR], int s, CT (&c)[4]) const
    {
#pragma unroll
        for (int k = 0; k < UPS; ++k) {
            const uint4 w = t[k][s];
            const CT *p = reinterpret_cast<const CT *>(&w);
#pragma unroll
            for (int i = 0; i < CPU_; ++i) c[k * CPU_ + i] = p[i];
        }
    }
    __device__ __forceinline__ void uget(int s, CT (&c)[4]) const { get(u, s, c); }
    __device__ __forceinline__ void vget(int s, CT (&c)[4]) const
    {
#pragma unroll
        for (int k = 0; k < UPS; ++k) {
            const uint4 w = v[k][s];
            const CT *p = reinterpret_cast<const CT *>(&w);
#pragma unroll
            for (int i = 0; i < CPU_; ++i) c[k * CPU_ + i] = p[i];
        }
    }
    __device__ __forceinline__ void vput(int s, const CT (&c)[4])
    {
#pragma unroll
        for (int k = 0; k < UPS; ++k) {
            uint4 w;
            CT *p = reinterpret_cast<CT *>(&w);
#pragma unroll
            for (int i = 0; i < CPU_; ++i) p[i] = c[k * CPU_ + i];
            v[k][s] = w;
        }
    }
    __device__ __forceinline__ CT ucell(int s, int i) const  // cell i of u slot s
    {
        return reinterpret_cast<const CT *>(&u[i / CPU_][s])[i % CPU_];
    }
    __device__ __forceinline__ CT vcell(int s, int i) const
    {
        return reinterpret_cast<const CT *>(&v[i / CPU_][s])[i % CPU_];
    }
};

template <typename R, int BX, int BY, int BZ>
constexpr size_t pair_smem()
{
    return sizeof(PairSpace<typename Cx<R>::T, BX, BY, BZ>);
}

// 16-byte unit k of segment q of the brick with record r into dst (zeros if
// that segment is not stored)
template <typename CT>
__device__ __forceinline__ void seg_unit_async(void *dst, const BrickRec &r, int q, int k, const CT *src)
{
    uint32_t j = 0;
    const bool ok = seg_index(r, q, j);
    cp_async16(dst, reinterpret_cast<const char *>(src + (ok ? j : 0u)) + 16 * k, ok);
}

// A fill hook stages per-cell data of the same cells beside u (the
// imaginary-time pass stages the propagator table E): own(slot, stored, j)
// for each of the brick's segments, seg(slot, r, q) for each halo segment
// (segment q of the brick with record r) and xh(side, row, r, q) for each x
// halo row.  The RK4 passes use none.
struct NoFillHook {
    __device__ __forceinline__ void own(int, bool, uint32_t) const {}
    __device__ __forceinline__ void seg(int, const BrickRec &, int) const {}
    __device__ __forceinline__ void xh(int, int, const BrickRec &, int) const {}
};

// Stage u of brick b: records, the own stored segments, the two-deep y and z
// face layers, the one-deep y-z edge rows and the x halo cells of every row
// with y in [-1, BY], z in [-1, BZ] (no y-z corner rows).
template <typename CT, int BX, int BY, int BZ, typename HOOK = NoFillHook>
__device__ __forceinline__ void pair_fill(PairSpace<CT, BX, BY, BZ> &ps, const PairView &P, int64_t b, const CT *src,
                                          const HOOK &hook = HOOK())
{
    using PS = PairSpace<CT, BX, BY, BZ>;
    constexpr int SX = PS::SX, PL = PS::PLANE_B, UPS = PS::UPS, NXU = PS::NXU;
    const int t = threadIdx.x;
    // records: own (0), faces -x +x -y +y -z +z (1-6), edges (7-18)
    if (t < 19) {
        uint4 r0 = make_uint4(0, 0, 0, 0), r1 = make_uint4(0, 0, 0, 0);
        const int64_t id = t == 0 ? b : (int64_t)__ldg(P.nbr18 + 18 * b + (t - 1));
        if (id >= 0) {
            const uint4 *p = reinterpret_cast<const uint4 *>(P.rec + id);
            r0 = __ldg(p);
            r1 = __ldg(p + 1);
        }
        reinterpret_cast<uint4 *>(&ps.rec[t])[0] = r0;
        reinterpret_cast<uint4 *>(&ps.rec[t])[1] = r1;
    }
    __syncthreads();
    const BrickRec &R0 = ps.rec[0];
    // own segments: stored ones by cp.async, unstored interior slots zeroed
    for (int q = t; q < PS::S::NSEG; q += PAIR_THREADS) {
        const int hx = q % SX, y = (q / SX) % BY, z = q / PL;
        const int sl = PS::slot(hx, y, z);
        const int w = q >> 5, bit = q & 31;
        const uint32_t m = R0.m[w];
        if ((m >> bit) & 1u) {
            const uint32_t rank = ((R0.pre >> (8 * w)) & 0xffu) + (uint32_t)__popc(m & ((1u << bit) - 1u));
            ps.list[rank] = (uint16_t)q;
            const char *g = reinterpret_cast<const char *>(src + R0.off + 4u * rank);
#pragma unroll
            for (int k = 0; k < UPS; ++k) cp_async16(&ps.u[k][sl], g + 16 * k, true);
            hook.own(sl, true, R0.off + 4u * rank);
        } else {
#pragma unroll
            for (int k = 0; k < UPS; ++k) ps.u[k][sl] = make_uint4(0, 0, 0, 0);
            hook.own(sl, false, 0u);
        }
    }
    if (t == 0) ps.nst = __popc(R0.m[0]) + __popc(R0.m[1]) + __popc(R0.m[2]) + __popc(R0.m[3]);
    // z face layers: planes -2, -1 (planes BZ-2, BZ-1 of the -z brick), BZ, BZ+1
    // (planes 0, 1 of the +z brick); in-plane y in [0, BY)
    for (int i = t; i < 4 * PL * UPS; i += PAIR_THREADS) {
        const int k = i % UPS, s = (i / UPS) % PL, pz = i / (UPS * PL);  // pz 0..3
        const int hx = s % SX, y = s / SX;
        const int z = pz < 2 ? pz - 2 : BZ + (pz - 2);
        const int zs = pz < 2 ? BZ - 2 + pz : pz - 2;
        seg_unit_async(&ps.u[k][PS::slot(hx, y, z)], ps.rec[pz < 2 ? 5 : 6], hx + SX * y + PL * zs, k, src);
        if (k == 0) hook.seg(PS::slot(hx, y, z), ps.rec[pz < 2 ? 5 : 6], hx + SX * y + PL * zs);
    }
    // y face layers: rows -2, -1 (rows BY-2, BY-1 of the -y brick), BY, BY+1
    // (rows 0, 1 of the +y brick); z in [0, BZ)
    for (int i = t; i < 4 * SX * BZ * UPS; i += PAIR_THREADS) {
        const int k = i % UPS, s = (i / UPS) % (SX * BZ), py = i / (UPS * SX * BZ);
        const int hx = s % SX, z = s / SX;
        const int y = py < 2 ? py - 2 : BY + (py - 2);
        const int ys = py < 2 ? BY - 2 + py : py - 2;
        seg_unit_async(&ps.u[k][PS::slot(hx, y, z)], ps.rec[py < 2 ? 3 : 4], hx + SX * ys + PL * z, k, src);
        if (k == 0) hook.seg(PS::slot(hx, y, z), ps.rec[py < 2 ? 3 : 4], hx + SX * ys + PL * z);
    }
    // y-z edge rows (y, z) in {-1, BY} x {-1, BZ}: records 15-18 are the edge
    // neighbours (0,-1,-1) (0,+1,-1) (0,-1,+1) (0,+1,+1)
    for (int i = t; i < 4 * SX * UPS; i += PAIR_THREADS) {
        const int k = i % UPS, hx = (i / UPS) % SX, e = i / (UPS * SX);
        const bool yp = e & 1, zp = e & 2;
        seg_unit_async(&ps.u[k][PS::slot(hx, yp ? BY : -1, zp ? BZ : -1)], ps.rec[15 + e],
                       hx + SX * (yp ? 0 : BY - 1) + PL * (zp ? 0 : BZ - 1), k, src);
        if (k == 0)
            hook.seg(PS::slot(hx, yp ? BY : -1, zp ? BZ : -1), ps.rec[15 + e],
                     hx + SX * (yp ? 0 : BY - 1) + PL * (zp ? 0 : BZ - 1));
    }
    // x halo cells: rows with y in [-1, BY], z in [-1, BZ] except the four y-z
    // corners; the -x side takes cells 2, 3 of the source's last segment of the
    // row, the +x side cells 0, 1 of its first.  Sources: the x-face bricks for
    // rows of the brick, the xy-edge bricks (records 7-10: (-1,-1,0) (+1,-1,0)
    // (-1,+1,0) (+1,+1,0)) for y = -1, BY, the xz-edge bricks (11-14: (-1,0,-1)
    // (+1,0,-1) (-1,0,+1) (+1,0,+1)) for z = -1, BZ.
    constexpr int NR = (BY + 2) * (BZ + 2);
    for (int i = t; i < 2 * NR * NXU; i += PAIR_THREADS) {
        const int k = i % NXU, rr = (i / NXU) % NR, side = i / (NXU * NR);
        const int y = rr % (BY + 2) - 1, z = rr / (BY + 2) - 1;
        const bool yin = y >= 0 && y < BY, zin = z >= 0 && z < BZ;
        if (!yin && !zin) continue;
        int rec = 1 + side, ys = y, zs = z;
        if (!yin) {
            rec = 7 + side + (y == BY ? 2 : 0);
            ys = y < 0 ? BY - 1 : 0;
        } else if (!zin) {
            rec = 11 + side + (z == BZ ? 2 : 0);
            zs = z < 0 ? BZ - 1 : 0;
        }
        const int q = (side == 0 ? SX - 1 : 0) + SX * ys + PL * zs;
        CT *dst = side == 0 ? &ps.uxl[PS::row(y, z)][k * (2 / NXU)] : &ps.uxr[PS::row(y, z)][k * (2 / NXU)];
        seg_unit_async(dst, ps.rec[rec], q, side == 0 ? UPS - NXU + k : k, src);
        if (k == 0) hook.xh(side, PS::row(y, z), ps.rec[rec], q);
    }
}

// The 7-point Laplacian (Eq. (B1)) of the 4 cells of u slot (hx, y, z); the
// x neighbours at the row ends come from the row's x halo cells
template <typename CT, int BX, int BY, int BZ, typename R>
__device__ __forceinline__ void pair_lap_u(const PairSpace<CT, BX, BY, BZ> &ps, int hx, int y, int z, CT (&c)[4],
                                           CT (&L)[4], R ihx2, R ihy2, R ihz2, R c6)
{
    using PS = PairSpace<CT, BX, BY, BZ>;
    const int s = PS::slot(hx, y, z);
    CT ym[4], yp[4], zm[4], zp[4];
    ps.uget(s, c);
    ps.uget(s - PS::ROW, ym);
    ps.uget(s + PS::ROW, yp);
    ps.uget(s - PS::PLANE, zm);
    ps.uget(s + PS::PLANE, zp);
    const int h = PS::row(y, z);
    const CT xm = hx == 0 ? ps.uxl[h][1] : ps.ucell(s - 1, 3);
    const CT xp = hx == PS::SX - 1 ? ps.uxr[h][0] : ps.ucell(s + 1, 0);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const CT l = i == 0 ? xm : c[i - 1];
        const CT rr = i == 3 ? xp : c[i + 1];
        L[i] = lapv(rr, l, yp[i], ym[i], zp[i], zm[i], c[i], ihx2, ihy2, ihz2, c6);
    }
}

// The same on the v tile (the brick's own slots only)
template <typename CT, int BX, int BY, int BZ, typename R>
__device__ __forceinline__ void pair_lap_v(const PairSpace<CT, BX, BY, BZ> &ps, int hx, int y, int z, CT (&c)[4],
                                           CT (&L)[4], R ihx2, R ihy2, R ihz2, R c6)
{
    using PS = PairSpace<CT, BX, BY, BZ>;
    const int s = PS::vslot(hx, y, z);
    CT ym[4], yp[4], zm[4], zp[4];
    ps.vget(s, c);
    ps.vget(s - PS::VROW, ym);
    ps.vget(s + PS::VROW, yp);
    ps.vget(s - PS::VPLANE, zm);
    ps.vget(s + PS::VPLANE, zp);
    const int h = PS::vrow(y, z);
    const CT xm = hx == 0 ? ps.vxl[h] : ps.vcell(s - 1, 3);
    const CT xp = hx == PS::SX - 1 ? ps.vxr[h] : ps.vcell(s + 1, 0);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const CT l = i == 0 ? xm : c[i - 1];
        const CT rr = i == 3 ? xp : c[i + 1];
        L[i] = lapv(rr, l, yp[i], ym[i], zp[i], zm[i], c[i], ihx2, ihy2, ihz2, c6);
    }
}

// Two RK4 stages of one brick.  PASS 0: stages 0 and 1 (u = y0); PASS 1:
// stages 2 and 3 (u = y3), y1 written to y1out.
template <typename R, int BX, int BY, int BZ, bool BLEND, int PASS>
__device__ __forceinline__ void pair_brick(PairSpace<typename Cx<R>::T, BX, BY, BZ> &ps, const PairView &P,
                                           const RkArgs<R> &a, int64_t b, R sA, R sB,
                                           typename Cx<R>::T *y1out)
{
    using CT = typename Cx<R>::T;
    using PS = PairSpace<CT, BX, BY, BZ>;
    constexpr int STA = PASS == 0 ? 0 : 2, STB = STA + 1;
    using BA = Rk4Body<R, BLEND, false, STA>;
    using BB = Rk4Body<R, BLEND, false, STB>;
    constexpr int SX = PS::SX, PL = PS::PLANE_B;
    const int t = threadIdx.x;
    const CT *usrc = PASS == 0 ? a.y0 : a.y3;
    const R c6 = (R)2 * (a.ihx2 + a.ihy2 + a.ihz2);
    pair_fill(ps, P, b, usrc);
    // v: zero (slots no task writes stay zero: cells outside the region)
    for (int i = t; i < PS::UPS * PS::VPSTR; i += PAIR_THREADS)
        (&ps.v[0][0])[i] = make_uint4(0, 0, 0, 0);
    for (int i = t; i < BY * BZ; i += PAIR_THREADS) {
        ps.vxl[i] = czero<CT>();
        ps.vxr[i] = czero<CT>();
    }
    cp_async_wait_all();
    __syncthreads();
    const BA bodyA(a, sA);
    const int nst = ps.nst;
    const BrickRec &R0 = ps.rec[0];
    // stage A on the stored segments of the brick, then of the one-deep z and
    // y face layers (tasks nst .. nst + 2*PL - 1: z = -1, BZ; then y = -1, BY)
    const int ntask = nst + 2 * PL + 2 * SX * BZ;
    for (int i = t; i < ntask; i += PAIR_THREADS) {
        int hx, y, z;
        uint32_t j;
        bool ok = true;
        if (i < nst) {
            const int q = ps.list[i];
            hx = q % SX;
            y = (q / SX) % BY;
            z = q / PL;
            j = R0.off + 4u * (uint32_t)i;
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
        const typename BA::P pa = bodyA.load(j);
        CT c[4], L[4], o[4], wv[4];
        pair_lap_u(ps, hx, y, z, c, L, a.ihx2, a.ihy2, a.ihz2, c6);
        bodyA.compute(pa, c, L, o, wv);
        ps.vput(PS::vslot(hx, y, z), o);
    }
    // stage A on the single cells of the one-deep x face layers
    for (int i = t; i < 2 * BY * BZ; i += PAIR_THREADS) {
        const int side = i / (BY * BZ), rr = i % (BY * BZ);
        const int y = rr % BY, z = rr / BY;
        uint32_t j;
        if (!seg_index(ps.rec[1 + side], (side == 0 ? SX - 1 : 0) + SX * y + PL * z, j)) continue;
        j += side == 0 ? 3u : 0u;  // the cell at x = -1 or x = BX
        // the cell's value and its six neighbours
        CT c0, xm, xp, ym, yp, zm, zp;
        const int h = PS::row(y, z);
        if (side == 0) {
            c0 = ps.uxl[h][1];
            xm = ps.uxl[h][0];
            xp = ps.ucell(PS::slot(0, y, z), 0);
            ym = ps.uxl[PS::row(y - 1, z)][1];
            yp = ps.uxl[PS::row(y + 1, z)][1];
            zm = ps.uxl[PS::row(y, z - 1)][1];
            zp = ps.uxl[PS::row(y, z + 1)][1];
        } else {
            c0 = ps.uxr[h][0];
            xm = ps.ucell(PS::slot(SX - 1, y, z), 3);
            xp = ps.uxr[h][1];
            ym = ps.uxr[PS::row(y - 1, z)][0];
            yp = ps.uxr[PS::row(y + 1, z)][0];
            zm = ps.uxr[PS::row(y, z - 1)][0];
            zp = ps.uxr[PS::row(y, z + 1)][0];
        }
        // operands of that cell only; the other three lanes of the update are
        // inactive (V = +inf)
        typename BA::P pa{};
        pa.V0[0] = a.V0[j];
        pa.V0[1] = pa.V0[2] = pa.V0[3] = (R)INFINITY;
        if constexpr (BLEND) pa.V1[0] = a.V1[j];
        if constexpr (STA == 2) pa.y[0] = a.y0[j];
        CT c[4] = {c0, czero<CT>(), czero<CT>(), czero<CT>()}, L[4], o[4], wv[4];
        L[0] = lapv(xp, xm, yp, ym, zp, zm, c0, a.ihx2, a.ihy2, a.ihz2, c6);
        L[1] = L[2] = L[3] = czero<CT>();
        bodyA.compute(pa, c, L, o, wv);
        (side == 0 ? ps.vxl : ps.vxr)[PS::vrow(y, z)] = o[0];
    }
    __syncthreads();
    // stage B on the brick's stored segments
    RkArgs<R> ab = a;
    if constexpr (PASS == 1) ab.y0 = y1out;  // stage 3 writes y1 to the other buffer
    const BB bodyB(ab, sB);
    for (int i = t; i < nst; i += PAIR_THREADS) {
        const int q = ps.list[i];
        const int hx = q % SX, y = (q / SX) % BY, z = q / PL;
        const uint32_t j = R0.off + 4u * (uint32_t)i;
        typename BB::P pb;
        ldr4(a.V0 + j, pb.V0);
        if constexpr (BLEND) ldr4(a.V1 + j, pb.V1);
        if constexpr (STB == 1) ps.uget(PS::slot(hx, y, z), pb.y);  // y0 of the cell (u = y0)
        if constexpr (STB == 3) ld4<false>(a.w + j, pb.y);
        CT c[4], L[4];
        pair_lap_v(ps, hx, y, z, c, L, a.ihx2, a.ihy2, a.ihz2, c6);
        bodyB(j, pb, c, L);
    }
    __syncthreads();  // the tiles are reused for the next brick
}

template <typename R, int BX, int BY, int BZ, bool BLEND, int PASS>
__global__ void __launch_bounds__(PAIR_THREADS) k_rk4_fused(const RkArgs<R> a, const PairView P,
                                                            typename Cx<R>::T *y1out)
{
    using CT = typename Cx<R>::T;
    extern __shared__ __align__(16) unsigned char gpe_smem[];
    auto &ps = *reinterpret_cast<PairSpace<CT, BX, BY, BZ> *>(gpe_smem);
    const R sA = stage_s<R, BLEND>(a, PASS == 0 ? 0 : 2);
    const R sB = stage_s<R, BLEND>(a, PASS == 0 ? 1 : 3);
    for (int64_t b = blockIdx.x; b < P.nb; b += gridDim.x) pair_brick<R, BX, BY, BZ, BLEND, PASS>(ps, P, a, b, sA, sB, y1out);
}

template <typename R, int BX, int BY, int BZ>
struct Rk4Fused {
    using K = void (*)(RkArgs<R>, PairView, typename Cx<R>::T *);
    static K get(bool blend, int pass)
    {
        static const K t[2][2] = {{k_rk4_fused<R, BX, BY, BZ, false, 0>, k_rk4_fused<R, BX, BY, BZ, false, 1>},
                                  {k_rk4_fused<R, BX, BY, BZ, true, 0>, k_rk4_fused<R, BX, BY, BZ, true, 1>}};
        return t[blend ? 1 : 0][pass];
    }
};

}  // namespace gpe
