// flat.cuh -- segment-parallel RK4 stage kernels for 7-point grids.
//
// The tile kernels (stencil.cuh) give one warp a brick: they stage the brick
// and its face halo in shared memory and then let the lanes take the brick's
// stored segments.  A brick of the thin shells holds about 35 stored segments,
// so the per-brick staging and the second, nearly empty pass over the lanes
// cost more issue slots than the stencil itself.  Here every thread takes one
// stored segment of the packed run (4 cells along x, the unit of the compact
// layout) and gathers its six neighbours directly:
//  * a segment table gives each stored segment its brick and local segment
//    number q (written once per grid);
//  * the brick's record and, at a brick face, the neighbour's record come
//    from the per-brick block of seven records (own, -x +x -y +y -z +z);
//  * the +-y and +-z neighbours are whole segments (256-bit loads), the +-x
//    neighbours single cells; absent segments read as zero (the rows and
//    columns deleted from the Laplacian, Sec. II A).
// Neighbour loads hit L1/L2: the lanes of a block take consecutive stored
// segments, so a segment's in-brick neighbours are loaded by the same or an
// adjacent warp, and the neighbour bricks' faces by recent blocks.  Lanes are
// always fully used, and no shared memory or barrier is needed.  The
// arithmetic per cell is the tile kernels' own (same expressions, same
// order), Eq. (B1) for the Laplacian and the memory-optimised RK4 stages of
// App. A (Rk4Body).
#pragma once

#include "stencil.cuh"

namespace gpe {

struct FlatView {
    const uint32_t *segtab;  // per stored segment: brick << 7 | local segment q
    const BrickRec *rec7;    // per brick: its record, then -x +x -y +y -z +z neighbours'
    int64_t nseg;            // stored segments (n_packed / 4)
};

// the parts of a brick record the gather needs: stored-segment bits of the
// NWRD mask words in use, packed offset, per-word prefix counts
template <int NWRD>
struct SegRec {
    uint32_t m[NWRD];
    uint32_t off, pre;
    __device__ __forceinline__ void load(const BrickRec *p)
    {
        const uint4 a = __ldg(reinterpret_cast<const uint4 *>(p));
        const uint4 b = __ldg(reinterpret_cast<const uint4 *>(p) + 1);
        m[0] = a.x;
        if constexpr (NWRD > 1) m[1] = a.y;
        if constexpr (NWRD > 2) {
            m[2] = a.z;
            m[3] = a.w;
        }
        off = b.x;
        pre = b.y;
    }
    // packed index of the first cell of segment q, if stored
    __device__ __forceinline__ bool at(int q, uint32_t &idx) const
    {
        const int w = q >> 5, bit = q & 31;
        uint32_t mw = m[0];
        if constexpr (NWRD > 1) mw = w == 1 ? m[1] : mw;
        if constexpr (NWRD > 2) mw = w == 2 ? m[2] : (w == 3 ? m[3] : mw);
        if (!((mw >> bit) & 1u)) return false;
        idx = off + 4u * (((pre >> (8 * w)) & 0xffu) + (uint32_t)__popc(mw & ((1u << bit) - 1u)));
        return true;
    }
};

// segment q_in of the own brick when `inside`, else segment q_out of the face
// neighbour whose record sits in slot k of the brick's record block; zero if
// that segment is not stored (or the neighbour is absent: empty record)
template <int NWRD, typename CT>
__device__ __forceinline__ void gather_seg(const SegRec<NWRD> &own, const BrickRec *blk, int k, bool inside, int q_in,
                                           int q_out, const CT *src, CT (&v)[4])
{
    uint32_t j = 0;
    bool ok;
    if (inside) {
        ok = own.at(q_in, j);
    } else {
        SegRec<NWRD> r;
        r.load(blk + k);
        ok = r.at(q_out, j);
    }
    if (ok) {
        ld4<false>(src + j, v);
    } else {
#pragma unroll
        for (int i = 0; i < 4; ++i) v[i] = czero<CT>();
    }
}

// one cell (cell `cell` of a segment) in the same way
template <int NWRD, typename CT>
__device__ __forceinline__ CT gather_cell(const SegRec<NWRD> &own, const BrickRec *blk, int k, bool inside, int q_in,
                                          int q_out, int cell, const CT *src)
{
    uint32_t j = 0;
    bool ok;
    if (inside) {
        ok = own.at(q_in, j);
    } else {
        SegRec<NWRD> r;
        r.load(blk + k);
        ok = r.at(q_out, j);
    }
    return ok ? ld1<false>(src + j + cell) : czero<CT>();
}

// The 7-point Laplacians L[4] (Eq. (B1)) of the four cells of stored segment
// sg of `src`, with the segment's own values c[4].  Returns the brick.
template <int BX, int BY, int BZ, typename CT, typename R>
__device__ __forceinline__ void flat_laplacian(const FlatView &F, int64_t sg, const CT *src, R ihx2, R ihy2, R ihz2,
                                               CT (&c)[4], CT (&L)[4])
{
    using S = Seg<BX, BY, BZ>;
    constexpr int NWRD = (S::NSEG + 31) / 32;
    const uint32_t info = __ldg(F.segtab + sg);
    const int64_t b = (int64_t)(info >> 7);
    const int q = (int)(info & 127u);
    const int hx = q % S::SX, y = (q / S::SX) % BY, z = q / S::PLANE;
    const BrickRec *blk = F.rec7 + 7 * b;
    SegRec<NWRD> own;
    own.load(blk);
    ld4<false>(src + 4 * sg, c);
    CT ym[4], yp[4], zm[4], zp[4];
    // record slots: 1 -x, 2 +x, 3 -y, 4 +y, 5 -z, 6 +z
    gather_seg(own, blk, 3, y > 0, q - S::SX, q + S::SX * (BY - 1), src, ym);
    gather_seg(own, blk, 4, y < BY - 1, q + S::SX, q - S::SX * (BY - 1), src, yp);
    gather_seg(own, blk, 5, z > 0, q - S::PLANE, q + S::PLANE * (BZ - 1), src, zm);
    gather_seg(own, blk, 6, z < BZ - 1, q + S::PLANE, q - S::PLANE * (BZ - 1), src, zp);
    // x neighbours: cell 3 of the segment to the left, cell 0 of the one to the right
    const CT xm = gather_cell(own, blk, 1, hx > 0, q - 1, q + (S::SX - 1), 3, src);
    const CT xp = gather_cell(own, blk, 2, hx < S::SX - 1, q + 1, q - (S::SX - 1), 0, src);
    const R c6 = (R)2 * (ihx2 + ihy2 + ihz2);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const CT l = i == 0 ? xm : c[i - 1];
        const CT rr = i == 3 ? xp : c[i + 1];
        L[i] = lapv(rr, l, yp[i], ym[i], zp[i], zm[i], c[i], ihx2, ihy2, ihz2, c6);
    }
}

// One memory-optimised RK4 stage (App. A; the stage body of the tile
// kernels): one thread per stored segment.
template <typename R, int BX, int BY, int BZ, bool BLEND, int ST>
__global__ void __launch_bounds__(256) k_rk4_flat(const RkArgs<R> a, const FlatView F)
{
    using CT = typename Cx<R>::T;
    using B = Rk4Body<R, BLEND, false, ST>;
    const int64_t sg = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (sg >= F.nseg) return;
    const B body(a, stage_s<R, BLEND>(a, ST));
    const uint32_t idx = 4u * (uint32_t)sg;
    const typename B::P pre = body.load(idx);
    CT c[4], L[4];
    flat_laplacian<BX, BY, BZ>(F, sg, body.yin(), a.ihx2, a.ihy2, a.ihz2, c, L);
    body(idx, pre, c, L);
}

template <typename R, int BX, int BY, int BZ>
struct Rk4Flat {
    using K = void (*)(RkArgs<R>, FlatView);
    static constexpr int THREADS = 256;
    static K get(bool blend, int st)
    {
        static const K t[2][4] = {
            {k_rk4_flat<R, BX, BY, BZ, false, 0>, k_rk4_flat<R, BX, BY, BZ, false, 1>,
             k_rk4_flat<R, BX, BY, BZ, false, 2>, k_rk4_flat<R, BX, BY, BZ, false, 3>},
            {k_rk4_flat<R, BX, BY, BZ, true, 0>, k_rk4_flat<R, BX, BY, BZ, true, 1>,
             k_rk4_flat<R, BX, BY, BZ, true, 2>, k_rk4_flat<R, BX, BY, BZ, true, 3>}};
        return t[blend ? 1 : 0][st];
    }
};

}  // namespace gpe
