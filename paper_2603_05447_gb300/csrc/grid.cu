// grid.cu -- region-of-interest selection and brick compaction (Sec. II A and
// Sec. II B of the paper), built on the device.
//
// Steps: (1) brick occupancy over the brick grid covering the box (a brick is
// kept if any of its in-box cells has V < V_cut); (2) enumeration of the brick
// grid in Morton or z-major key order with an order-preserving compaction (two
// passes: per-block counts, then emission at scanned offsets); (3) a dense
// brick-id volume and the 6-entry face-neighbour table; (4) per-cell potential
// values and the active-cell bit mask.  The paper's GPU variant keeps a
// 488-entry halo index list per 8^3 block (Sec. II B); here six neighbour ids
// per brick are enough because the halo is gathered from neighbour bricks at
// fixed offsets inside the step kernels.
#include <algorithm>
#include <cmath>
#include <vector>

#include "gpe_internal.cuh"

namespace gpe {

struct PotDesc {
    int kind;
    double p[8];
};

// V source for the builder: a dense array, one analytic potential, or two
// potentials (ramp endpoints, analytic or dense) whose union mask is taken.
struct VSource {
    int mode;  // 0 dense, 1 analytic, 2 analytic blend, 3 dense blend
    const void *dense, *dense1;
    int dtype;
    PotDesc p0, p1;
    double cut0, cut1;
};

__device__ __forceinline__ double eval_pot(const PotDesc &P, double x, double y, double z)
{
    if (P.kind == GPE_POT_HARMONIC)
        return 0.5 * (P.p[0] * P.p[0] * x * x + P.p[1] * P.p[1] * y * y + P.p[2] * P.p[2] * z * z);
    if (P.kind == GPE_POT_ELLIPSOID_SHELL) {
        double rho = sqrt(x * x / (P.p[1] * P.p[1]) + y * y / (P.p[2] * P.p[2]) +
                          z * z / (P.p[3] * P.p[3]));
        double d = rho - 1.0;
        return 0.5 * P.p[0] * P.p[0] * d * d;
    }
    return 0.0;
}

struct BoxD {
    int64_t nx, ny, nz;
    double hx, hy, hz, x0, y0, z0;
};

__device__ __forceinline__ void cell_values(const VSource &src, const BoxD &bx, int64_t i,
                                            int64_t j, int64_t k, double &v0, double &v1,
                                            bool &sel)
{
    if (src.mode == 0 || src.mode == 3) {
        int64_t lin = i + bx.nx * (j + bx.ny * k);
        auto at = [&](const void *p) {
            return src.dtype == GPE_F64 ? ((const double *)p)[lin] : (double)((const float *)p)[lin];
        };
        v0 = at(src.dense);
        if (src.mode == 3) {
            v1 = at(src.dense1);
            sel = (v0 < src.cut0) || (v1 < src.cut1);
        } else {
            v1 = 0.0;
            sel = v0 < src.cut0;
        }
        return;
    }
    double x = bx.x0 + i * bx.hx, y = bx.y0 + j * bx.hy, z = bx.z0 + k * bx.hz;
    v0 = eval_pot(src.p0, x, y, z);
    if (src.mode == 2) {
        v1 = eval_pot(src.p1, x, y, z);
        sel = (v0 < src.cut0) || (v1 < src.cut1);
    } else {
        v1 = 0.0;
        sel = v0 < src.cut0;
    }
}

// May an analytic potential fall below `cut` somewhere in the axis-aligned
// box [xl,xh] x [yl,yh] x [zl,zh]?  (true for an unknown kind.)  Both
// potentials are separable in the squares of the coordinates, so the extremes
// of each square over an interval give the exact range: the harmonic
// potential's minimum directly, and for the ellipsoidal shell the range
// [rmin, rmax] of the scaled radius, from which the smallest |rho - 1|
// follows.  Evaluated in FP32 with wide margins: it only has to be
// conservative, the per-cell FP64 test decides.
__device__ __forceinline__ bool pot_may_select(const PotDesc &P, double cut, float xl, float xh, float yl, float yh,
                                               float zl, float zh)
{
    auto sqmin = [](float l, float h) { return (l <= 0.f && h >= 0.f) ? 0.f : fminf(l * l, h * h); };
    auto sqmax = [](float l, float h) { return fmaxf(l * l, h * h); };
    if (P.kind == GPE_POT_HARMONIC) {
        const float wx = (float)P.p[0], wy = (float)P.p[1], wz = (float)P.p[2];
        const float vmin = 0.5f * (wx * wx * sqmin(xl, xh) + wy * wy * sqmin(yl, yh) + wz * wz * sqmin(zl, zh));
        return vmin <= (float)cut * 1.0001f + 1e-30f;
    }
    if (P.kind == GPE_POT_ELLIPSOID_SHELL) {
        const float w = (float)P.p[0];
        const float ia = 1.f / (float)(P.p[1] * P.p[1]), ib = 1.f / (float)(P.p[2] * P.p[2]),
                    ic = 1.f / (float)(P.p[3] * P.p[3]);
        const float rmin = sqrtf(sqmin(xl, xh) * ia + sqmin(yl, yh) * ib + sqmin(zl, zh) * ic);
        const float rmax = sqrtf(sqmax(xl, xh) * ia + sqmax(yl, yh) * ib + sqmax(zl, zh) * ic);
        const float d = (rmin <= 1.f && rmax >= 1.f) ? 0.f : fminf(fabsf(rmin - 1.f), fabsf(rmax - 1.f));
        // V = w^2 d^2 / 2 < cut  <=>  |w| d < sqrt(2 cut)
        return fabsf(w) * d <= sqrtf(2.f * (float)cut) * 1.0001f + 1e-4f * (1.f + rmax) * fabsf(w);
    }
    return true;
}

// (1) occupancy of every brick-grid position (lexicographic q), 256 brick
// positions a block.  Analytic sources: one thread a position tests the
// brick's cell-centre box against the bound above; then the block tests the
// cells of each candidate brick exactly.
__global__ void k_occupancy(VSource src, BoxD box, int BX, int BY, int BZ, int64_t nbx, int64_t nby, int64_t nbz,
                            uint8_t *occ)
{
    __shared__ int64_t cand[256];
    __shared__ int ncand;
    const int64_t nq = nbx * nby * nbz;
    const int64_t q = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (threadIdx.x == 0) ncand = 0;
    __syncthreads();
    if (q < nq) {
        const int64_t qx = q % nbx, qy = (q / nbx) % nby, qz = q / (nbx * nby);
        bool may = true;
        if (src.mode == 1 || src.mode == 2) {
            const int64_t i0 = qx * BX, j0 = qy * BY, k0 = qz * BZ;
            const int64_t i1 = min(i0 + BX, box.nx) - 1, j1 = min(j0 + BY, box.ny) - 1, k1 = min(k0 + BZ, box.nz) - 1;
            const float xl = (float)(box.x0 + i0 * box.hx), xh = (float)(box.x0 + i1 * box.hx);
            const float yl = (float)(box.y0 + j0 * box.hy), yh = (float)(box.y0 + j1 * box.hy);
            const float zl = (float)(box.z0 + k0 * box.hz), zh = (float)(box.z0 + k1 * box.hz);
            may = pot_may_select(src.p0, src.cut0, xl, xh, yl, yh, zl, zh);
            if (src.mode == 2) may = may || pot_may_select(src.p1, src.cut1, xl, xh, yl, yh, zl, zh);
        }
        if (may)
            cand[atomicAdd(&ncand, 1)] = q;
        else
            occ[q] = 0;
    }
    __syncthreads();
    const int nc = ncand;
    const int BC = BX * BY * BZ;
    for (int c = 0; c < nc; ++c) {
        const int64_t qq = cand[c];
        const int64_t qx = qq % nbx, qy = (qq / nbx) % nby, qz = qq / (nbx * nby);
        int sel_any = 0;
        for (int l = threadIdx.x; l < BC; l += blockDim.x) {
            const int64_t i = qx * BX + l % BX, j = qy * BY + (l / BX) % BY, k = qz * BZ + l / (BX * BY);
            if (i < box.nx && j < box.ny && k < box.nz) {
                double v0, v1;
                bool sel;
                cell_values(src, box, i, j, k, v0, v1, sel);
                sel_any |= sel;
            }
        }
        sel_any = __syncthreads_or(sel_any);
        if (threadIdx.x == 0) occ[qq] = (uint8_t)(sel_any != 0);
    }
}

__device__ __forceinline__ uint32_t compact3(uint64_t m)
{
    // keep every third bit of m (bit 3n -> bit n)
    uint64_t x = m & 0x1249249249249249ull;
    x = (x ^ (x >> 2)) & 0x10c30c30c30c30c3ull;
    x = (x ^ (x >> 4)) & 0x100f00f00f00f00full;
    x = (x ^ (x >> 8)) & 0x1f0000ff0000ffull;
    x = (x ^ (x >> 16)) & 0x1f00000000ffffull;
    x = (x ^ (x >> 32)) & 0x1fffffull;
    return (uint32_t)x;
}

struct Enum {
    int order;  // GPE_ORDER_*
    int64_t nbx, nby, nbz;
    uint64_t nkeys;
};

__device__ __forceinline__ bool key_brick(const Enum &E, const uint8_t *occ, uint64_t key,
                                          int64_t &bx, int64_t &by, int64_t &bz)
{
    if (E.order == GPE_ORDER_MORTON) {
        bx = compact3(key);
        by = compact3(key >> 1);
        bz = compact3(key >> 2);
        if (bx >= E.nbx || by >= E.nby || bz >= E.nbz) return false;
    } else {
        bx = key % E.nbx;
        by = (key / E.nbx) % E.nby;
        bz = key / (E.nbx * E.nby);
    }
    return occ[bx + E.nbx * (by + E.nby * bz)] != 0;
}

constexpr int ENUM_THREADS = 256, ENUM_PER_THREAD = 4;
constexpr int ENUM_PER_BLOCK = ENUM_THREADS * ENUM_PER_THREAD;

// (2a) number of kept bricks per enumeration block
__global__ void k_enum_count(Enum E, const uint8_t *occ, int64_t *bsum)
{
    const uint64_t base = (uint64_t)blockIdx.x * ENUM_PER_BLOCK + threadIdx.x * ENUM_PER_THREAD;
    int c = 0;
    for (int r = 0; r < ENUM_PER_THREAD; ++r) {
        uint64_t key = base + r;
        int64_t bx, by, bz;
        if (key < E.nkeys && key_brick(E, occ, key, bx, by, bz)) ++c;
    }
    __shared__ int warp_tot[ENUM_THREADS / 32];
    for (int off = 16; off > 0; off >>= 1) c += __shfl_down_sync(0xffffffffu, c, off);
    if ((threadIdx.x & 31) == 0) warp_tot[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int s = 0;
        for (int w = 0; w < ENUM_THREADS / 32; ++w) s += warp_tot[w];
        bsum[blockIdx.x] = s;
    }
}

// (2b) emit kept bricks in key order at the scanned block offsets
__global__ void k_enum_emit(Enum E, const uint8_t *occ, const int64_t *boff, int32_t *coords)
{
    __shared__ int warp_tot[ENUM_THREADS / 32];
    const uint64_t base = (uint64_t)blockIdx.x * ENUM_PER_BLOCK + threadIdx.x * ENUM_PER_THREAD;
    int c = 0;
    for (int r = 0; r < ENUM_PER_THREAD; ++r) {
        uint64_t key = base + r;
        int64_t bx, by, bz;
        if (key < E.nkeys && key_brick(E, occ, key, bx, by, bz)) ++c;
    }
    // exclusive scan of c over threads (in thread order = key order)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = c;
    for (int off = 1; off < 32; off <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += y;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    int wpre = 0;
    for (int w = 0; w < warp; ++w) wpre += warp_tot[w];
    int64_t pos = boff[blockIdx.x] + wpre + incl - c;
    for (int r = 0; r < ENUM_PER_THREAD; ++r) {
        uint64_t key = base + r;
        int64_t bx, by, bz;
        if (key < E.nkeys && key_brick(E, occ, key, bx, by, bz)) {
            coords[3 * pos + 0] = (int32_t)bx;
            coords[3 * pos + 1] = (int32_t)by;
            coords[3 * pos + 2] = (int32_t)bz;
            ++pos;
        }
    }
}

// (3) brick-id volume, origins, neighbour table
__global__ void k_bricks(int64_t nb, const int32_t *coords, int BX, int BY, int BZ,
                         int64_t nbx, int64_t nby, int32_t *bvol, int32_t *org)
{
    int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (id >= nb) return;
    int64_t bx = coords[3 * id], by = coords[3 * id + 1], bz = coords[3 * id + 2];
    bvol[bx + nbx * (by + nby * bz)] = (int32_t)id;
    org[3 * id + 0] = (int32_t)(bx * BX);
    org[3 * id + 1] = (int32_t)(by * BY);
    org[3 * id + 2] = (int32_t)(bz * BZ);
}

__global__ void k_neighbors(int64_t nb, const int32_t *coords, int64_t nbx, int64_t nby,
                            int64_t nbz, const int32_t *bvol, int32_t *nbr)
{
    int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (id >= nb) return;
    const int64_t c[3] = {coords[3 * id], coords[3 * id + 1], coords[3 * id + 2]};
    const int64_t n[3] = {nbx, nby, nbz};
    for (int d = 0; d < 6; ++d) {
        int64_t q[3] = {c[0], c[1], c[2]};
        q[d >> 1] += (d & 1) ? 1 : -1;
        int32_t r = -1;
        if (q[d >> 1] >= 0 && q[d >> 1] < n[d >> 1]) r = bvol[q[0] + nbx * (q[1] + nby * q[2])];
        nbr[6 * id + d] = r;
    }
}

// (4) per-cell potential values and active bits; one block per brick
__global__ void k_cells(VSource src, BoxD box, int BX, int BY, int BZ, int mask_mode,
                        const int32_t *org, double *V0, double *V1, uint32_t *mask,
                        unsigned long long *n_active, unsigned long long *vmax_bits)
{
    const int64_t id = blockIdx.x;
    const int BC = BX * BY * BZ;
    unsigned long long cnt = 0;
    double vm = 0.0;
    for (int l = threadIdx.x; l < BC; l += blockDim.x) {  // BC % 32 == 0, blockDim % 32 == 0
        int64_t i = org[3 * id] + l % BX, j = org[3 * id + 1] + (l / BX) % BY,
                k = org[3 * id + 2] + l / (BX * BY);
        bool inbox = i < box.nx && j < box.ny && k < box.nz;
        double v0 = 0.0, v1 = 0.0;
        bool sel = false;
        if (inbox) cell_values(src, box, i, j, k, v0, v1, sel);
        bool act = inbox && (mask_mode == GPE_MASK_BRICK ? true : sel);
        const int64_t slot = id * BC + l;
        V0[slot] = v0;
        if (V1) V1[slot] = v1;
        unsigned bits = __ballot_sync(0xffffffffu, act);
        if ((threadIdx.x & 31) == 0) mask[slot >> 5] = bits;
        if (act) {
            ++cnt;
            vm = fmax(vm, fabs(v0));
            if (V1) vm = fmax(vm, fabs(v1));
        }
    }
    for (int off = 16; off > 0; off >>= 1) {
        cnt += __shfl_down_sync(0xffffffffu, cnt, off);
        vm = fmax(vm, __shfl_down_sync(0xffffffffu, vm, off));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(n_active, cnt);
        atomicMax(vmax_bits, (unsigned long long)__double_as_longlong(vm));
    }
}

// Segment layout: a segment is 4 consecutive cells along x inside a brick
// (one 32-byte sector of complex64).  A brick stores exactly its segments that
// hold at least one active cell.  k_seg_records builds each brick's record:
// the segment bit mask, the number of stored segments before each mask word,
// and (after the host scan) the packed offset.
__global__ void k_seg_records(int64_t nb, int BC, const uint32_t *mask, BrickRec *rec, uint32_t *cnt)
{
    int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= nb) return;
    const int W = BC / 32, nseg = BC / 4;
    BrickRec r{};
    uint32_t c = 0;
    for (int q = 0; q < nseg; ++q) {
        // cells 4q..4q+3 of the brick: nibble (q & 7) of mask word q/8
        const uint32_t word = mask[b * W + (q >> 3)];
        if ((word >> (4 * (q & 7))) & 0xfu) r.m[q >> 5] |= 1u << (q & 31);
    }
    for (int w = 0; w < 4; ++w) {
        r.pre |= (c & 0xffu) << (8 * w);
        c += __popc(r.m[w]);
    }
    rec[b] = r;
    cnt[b] = c;
}

// scatter stored-lattice values to the packed layout: active cells get their
// value, inactive cells of stored segments get `fill`
__global__ void k_pack(int64_t ns, int BC, const uint32_t *mask, const BrickRec *rec, const double *src,
                       double *dst, double fill)
{
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < ns; s += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = s / BC;
        const int l = (int)(s % BC);
        uint32_t idx;
        if (!seg_index(rec[b], l >> 2, idx)) continue;
        const bool act = (mask[s >> 5] >> (s & 31)) & 1u;
        dst[idx + (l & 3)] = act ? src[s] : fill;
    }
}

// replace a potential slot from a dense array (region unchanged)
__global__ void k_set_potential(const void *dense, int dtype, BoxD box, int BX, int BY, int BZ,
                                const int32_t *org, const uint32_t *mask, const BrickRec *rec, double *V)
{
    const int64_t id = blockIdx.x;
    const int BC = BX * BY * BZ, W = BC / 32;
    for (int l = threadIdx.x; l < BC; l += blockDim.x) {
        const uint32_t word = mask[id * W + (l >> 5)];
        if (!((word >> (l & 31)) & 1u)) continue;   // active cells are always inside the box
        uint32_t idx;
        if (!seg_index(rec[id], l >> 2, idx)) continue;
        int64_t i = org[3 * id] + l % BX, j = org[3 * id + 1] + (l / BX) % BY,
                k = org[3 * id + 2] + l / (BX * BY);
        int64_t lin = i + box.nx * (j + box.ny * k);
        V[idx + (l & 3)] = dtype == GPE_F64 ? ((const double *)dense)[lin] : (double)((const float *)dense)[lin];
    }
}

// max |V| over the active cells of the packed arrays (inactive cells of
// stored segments hold +inf in V0 and are skipped)
__global__ void k_vmax(int64_t np, const double *V0, const double *V1, unsigned long long *vmax_bits)
{
    double vm = 0.0;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < np;
         s += (int64_t)gridDim.x * blockDim.x) {
        if (!(V0[s] < INFINITY)) continue;
        vm = fmax(vm, fabs(V0[s]));
        if (V1) vm = fmax(vm, fabs(V1[s]));
    }
    for (int off = 16; off > 0; off >>= 1) vm = fmax(vm, __shfl_down_sync(0xffffffffu, vm, off));
    if ((threadIdx.x & 31) == 0) atomicMax(vmax_bits, (unsigned long long)__double_as_longlong(vm));
}

}  // namespace gpe

void gpe::build_rec7(const std::vector<BrickRec> &rec, const std::vector<int32_t> &nbr, std::vector<BrickRec> &out)
{
    const size_t nb = rec.size();
    out.assign(nb * 7, BrickRec{});
    for (size_t b = 0; b < nb; ++b) {
        out[7 * b] = rec[b];
        for (int d = 0; d < 6; ++d)
            if (nbr[6 * b + d] >= 0) out[7 * b + 1 + d] = rec[nbr[6 * b + d]];
    }
}

void gpe::build_rec19(const std::vector<BrickRec> &rec, const std::vector<int32_t> &nbr,
                      const std::vector<int32_t> &nbr_e, std::vector<BrickRec> &out)
{
    const size_t nb = rec.size();
    out.assign(nb * 19, BrickRec{});
    for (size_t b = 0; b < nb; ++b) {
        out[19 * b] = rec[b];
        for (int d = 0; d < 6; ++d)
            if (nbr[6 * b + d] >= 0) out[19 * b + 1 + d] = rec[nbr[6 * b + d]];
        for (int e = 0; e < 12; ++e)
            if (nbr_e[12 * b + e] >= 0) out[19 * b + 7 + e] = rec[nbr_e[12 * b + e]];
    }
}

namespace gpe {

// the 12 edge neighbours of each brick (order as in build_rec19), -1 if absent
__global__ void k_edge_neighbors(int64_t nb, const int32_t *coords, int64_t nbx, int64_t nby, int64_t nbz,
                                 const int32_t *bvol, int32_t *nbr_e)
{
    const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (id >= nb) return;
    const int8_t d[12][3] = {{-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}, {1, 1, 0}, {-1, 0, -1}, {1, 0, -1},
                             {-1, 0, 1},  {1, 0, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}, {0, 1, 1}};
    for (int e = 0; e < 12; ++e) {
        const int64_t x = coords[3 * id] + d[e][0], y = coords[3 * id + 1] + d[e][1], z = coords[3 * id + 2] + d[e][2];
        int32_t r = -1;
        if (x >= 0 && x < nbx && y >= 0 && y < nby && z >= 0 && z < nbz) r = bvol[x + nbx * (y + nby * z)];
        nbr_e[12 * id + e] = r;
    }
}

static BoxD boxd(const gpe_box &b)
{
    return BoxD{b.nx, b.ny, b.nz, b.hx, b.hy, b.hz, b.x0, b.y0, b.z0};
}

static int check_box(const gpe_box *box)
{
    if (!box) return fail(GPE_ERR_ARG, "box is NULL");
    if (box->nx < 1 || box->ny < 1 || box->nz < 1)
        return fail(GPE_ERR_ARG, "box dimensions must be >= 1 (got %lld x %lld x %lld)",
                    (long long)box->nx, (long long)box->ny, (long long)box->nz);
    if (!(box->hx > 0) || !(box->hy > 0) || !(box->hz > 0))
        return fail(GPE_ERR_ARG, "grid spacings must be > 0");
    if (box->nx > (1 << 24) || box->ny > (1 << 24) || box->nz > (1 << 24))
        return fail(GPE_ERR_ARG, "box dimension above 2^24");
    return GPE_OK;
}

static int check_pot(const gpe_potential *p)
{
    if (!p) return fail(GPE_ERR_ARG, "potential is NULL");
    if (p->kind != GPE_POT_HARMONIC && p->kind != GPE_POT_ELLIPSOID_SHELL)
        return fail(GPE_ERR_ARG, "unknown potential kind %d", p->kind);
    if (p->kind == GPE_POT_ELLIPSOID_SHELL && (!(p->p[1] > 0) || !(p->p[2] > 0) || !(p->p[3] > 0)))
        return fail(GPE_ERR_ARG, "ellipsoid semi-axes must be > 0");
    return GPE_OK;
}

static PotDesc potdesc(const gpe_potential &p)
{
    PotDesc d;
    d.kind = p.kind;
    for (int i = 0; i < 8; ++i) d.p[i] = p.p[i];
    return d;
}

static void grid_free(gpe_grid *g)
{
    if (!g) return;
    dev_free(g->d_rec);
    dev_free(g->d_rec7);
    dev_free(g->d_rec19);
    dev_free(g->d_nbr18);
    dev_free(g->d_chunk_lohi);
    dev_free(g->d_tasks);
    dev_free(g->d_dep_off);
    dev_free(g->d_dep_ids);
    dev_free(g->d_tasks_w);
    dev_free(g->d_org);
    dev_free(g->d_nbr);
    dev_free(g->d_mask);
    dev_free(g->d_bvol);
    for (int s = 0; s < 2; ++s) {
        dev_free(g->d_V[s]);
        dev_free(g->d_Vf[s]);
    }
    delete g;
}

// Build the grid; `src.dense` (mode 0) is a device pointer here.
static int build_grid(const gpe_box *box, const VSource &src, const gpe_grid_opts *opts,
                      gpe_grid **out, cudaStream_t st)
{
    gpe_grid_opts o{};
    if (opts) o = *opts;
    if (o.bx == 0 && o.by == 0 && o.bz == 0) o.bx = o.by = o.bz = 8;
    const int shape = shape_id(o.bx, o.by, o.bz);
    if (shape < 0)
        return fail(GPE_ERR_ARG, "unsupported brick shape %dx%dx%d (use 8x8x8, 8x8x4 or 8x4x4)", o.bx, o.by,
                    o.bz);
    if (o.mask_mode != GPE_MASK_CELL && o.mask_mode != GPE_MASK_BRICK)
        return fail(GPE_ERR_ARG, "unknown mask mode %d", o.mask_mode);
    if (o.order != GPE_ORDER_MORTON && o.order != GPE_ORDER_ZMAJOR)
        return fail(GPE_ERR_ARG, "unknown brick order %d", o.order);
    if (o.stencil != 0 && o.stencil != 7 && o.stencil != 19) return fail(GPE_ERR_ARG, "stencil must be 7 or 19");
    if (o.sched != GPE_SCHED_WAVE && o.sched != GPE_SCHED_WAVE2 && o.sched != GPE_SCHED_STAGED &&
        o.sched != GPE_SCHED_PAIR)
        return fail(GPE_ERR_ARG, "unknown schedule %d", o.sched);
    if (o.chunk < 0 || o.chunk > 4096) return fail(GPE_ERR_ARG, "chunk must be in [0, 4096]");

    gpe_grid *g = new gpe_grid();
    GPE_TRY_CUDA(cudaGetDevice(&g->device));
    g->nsm = sm_count(g->device);
    g->box = *box;
    g->bx = o.bx;
    g->by = o.by;
    g->bz = o.bz;
    g->bc = o.bx * o.by * o.bz;
    g->shape = shape;
    g->mask_mode = o.mask_mode;
    g->order = o.order;
    g->sched = o.sched;
    g->stencil = o.stencil == 19 ? 19 : 7;
    // bricks per wavefront task: about 2048 lattice cells for block tasks,
    // about 1024 for the warp tasks of WAVE2
    g->cb = o.chunk > 0 ? o.chunk : std::max(1, (o.sched == GPE_SCHED_WAVE2 ? 1024 : 2048) / g->bc);
    g->nbx = (box->nx + o.bx - 1) / o.bx;
    g->nby = (box->ny + o.by - 1) / o.by;
    g->nbz = (box->nz + o.bz - 1) / o.bz;
    const int64_t nq = g->nbx * g->nby * g->nbz;
    const BoxD bd = boxd(*box);

    uint8_t *occ = nullptr;
    int64_t *bsum = nullptr;
    int32_t *coords = nullptr;
    unsigned long long *counters = nullptr;
    double *tmpV[2] = {nullptr, nullptr};
    uint32_t *cnt = nullptr;
    int rc = GPE_OK;
    auto cleanup = [&]() {
        dev_free(occ);
        dev_free(bsum);
        dev_free(coords);
        dev_free(counters);
        dev_free(tmpV[0]);
        dev_free(tmpV[1]);
        dev_free(cnt);
        occ = nullptr;
        bsum = nullptr;
        coords = nullptr;
        counters = nullptr;
        tmpV[0] = tmpV[1] = nullptr;
        cnt = nullptr;
    };
#define BUILD_TRY(x)                 \
    do {                             \
        rc = (x);                    \
        if (rc != GPE_OK) {          \
            cleanup();               \
            grid_free(g);            \
            return rc;               \
        }                            \
    } while (0)
#define BUILD_CUDA(x)                                                        \
    do {                                                                     \
        cudaError_t e__ = (x);                                               \
        if (e__ != cudaSuccess) {                                            \
            rc = cuda_fail(e__, #x, __FILE__, __LINE__);                     \
            cleanup();                                                       \
            grid_free(g);                                                    \
            return rc;                                                       \
        }                                                                    \
    } while (0)

    BUILD_TRY(dev_alloc_t(&occ, nq));
    {
        const int64_t nblk_occ = (nq + 255) / 256;
        if (nblk_occ > 0x7fffffffLL) BUILD_TRY(fail(GPE_ERR_ARG, "brick grid too large"));
        k_occupancy<<<(unsigned)nblk_occ, 256, 0, st>>>(src, bd, o.bx, o.by, o.bz, g->nbx, g->nby, g->nbz, occ);
        BUILD_CUDA(cudaGetLastError());
    }
    Enum E;
    E.order = o.order;
    E.nbx = g->nbx;
    E.nby = g->nby;
    E.nbz = g->nbz;
    if (o.order == GPE_ORDER_MORTON) {
        int64_t m = std::max(g->nbx, std::max(g->nby, g->nbz));
        int L = 0;
        while ((int64_t(1) << L) < m) ++L;
        if (3 * L > 62) BUILD_TRY(fail(GPE_ERR_ARG, "brick grid too large for Morton keys"));
        E.nkeys = uint64_t(1) << (3 * L);
    } else {
        E.nkeys = (uint64_t)nq;
    }
    const int64_t nblk = (int64_t)((E.nkeys + ENUM_PER_BLOCK - 1) / ENUM_PER_BLOCK);
    if (nblk > 0x7fffffffLL) BUILD_TRY(fail(GPE_ERR_ARG, "brick grid too large"));
    BUILD_TRY(dev_alloc_t(&bsum, nblk));
    k_enum_count<<<(unsigned)nblk, ENUM_THREADS, 0, st>>>(E, occ, bsum);
    BUILD_CUDA(cudaGetLastError());
    std::vector<int64_t> h(nblk);
    BUILD_CUDA(cudaMemcpyAsync(h.data(), bsum, nblk * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    BUILD_CUDA(cudaStreamSynchronize(st));
    int64_t total = 0;
    for (int64_t i = 0; i < nblk; ++i) {
        int64_t c = h[i];
        h[i] = total;
        total += c;
    }
    if (total == 0) BUILD_TRY(fail(GPE_ERR_ARG, "region of interest is empty (no cell with V < V_cut)"));
    if (total * g->bc > 0x7fffffffLL * 32LL)
        BUILD_TRY(fail(GPE_ERR_ARG, "too many stored cells"));
    g->nb = total;
    g->n_stored = total * g->bc;
    BUILD_CUDA(cudaMemcpyAsync(bsum, h.data(), nblk * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    BUILD_TRY(dev_alloc_t(&coords, 3 * total));
    k_enum_emit<<<(unsigned)nblk, ENUM_THREADS, 0, st>>>(E, occ, bsum, coords);
    BUILD_CUDA(cudaGetLastError());

    BUILD_TRY(dev_alloc_t(&g->d_bvol, nq));
    BUILD_CUDA(cudaMemsetAsync(g->d_bvol, 0xff, nq * sizeof(int32_t), st));
    BUILD_TRY(dev_alloc_t(&g->d_org, 3 * total));
    BUILD_TRY(dev_alloc_t(&g->d_nbr, 6 * total));
    const unsigned nbb = (unsigned)((total + 255) / 256);
    k_bricks<<<nbb, 256, 0, st>>>(total, coords, o.bx, o.by, o.bz, g->nbx, g->nby, g->d_bvol, g->d_org);
    BUILD_CUDA(cudaGetLastError());
    k_neighbors<<<nbb, 256, 0, st>>>(total, coords, g->nbx, g->nby, g->nbz, g->d_bvol, g->d_nbr);
    BUILD_CUDA(cudaGetLastError());

    BUILD_TRY(dev_alloc_t(&g->d_mask, g->n_stored / 32));
    BUILD_TRY(dev_alloc_t(&tmpV[0], g->n_stored));
    if (src.mode == 2 || src.mode == 3) {
        BUILD_TRY(dev_alloc_t(&tmpV[1], g->n_stored));
        g->n_slots = 2;
    }
    BUILD_TRY(dev_alloc_t(&counters, 2));
    BUILD_CUDA(cudaMemsetAsync(counters, 0, 2 * sizeof(unsigned long long), st));
    if (total > 0x7fffffffLL) BUILD_TRY(fail(GPE_ERR_ARG, "too many bricks"));
    k_cells<<<(unsigned)total, std::min(g->bc, 256), 0, st>>>(src, bd, o.bx, o.by, o.bz, o.mask_mode,
                                                            g->d_org, tmpV[0], tmpV[1], g->d_mask,
                                                            counters, counters + 1);
    BUILD_CUDA(cudaGetLastError());
    unsigned long long hc[2];
    BUILD_CUDA(cudaMemcpyAsync(hc, counters, sizeof hc, cudaMemcpyDeviceToHost, st));
    BUILD_CUDA(cudaStreamSynchronize(st));
    g->n_active = (int64_t)hc[0];
    long long vb = (long long)hc[1];
    memcpy(&g->v_max, &vb, sizeof(double));

    // packed layout: every brick stores its segments (4 cells along x) that
    // hold an active cell, in lattice order, as one run
    BUILD_TRY(dev_alloc_t(&g->d_rec, total));
    BUILD_TRY(dev_alloc_t(&cnt, total));
    k_seg_records<<<nbb, 256, 0, st>>>(total, g->bc, g->d_mask, g->d_rec, cnt);
    BUILD_CUDA(cudaGetLastError());
    std::vector<uint32_t> hcnt(total);
    std::vector<BrickRec> hrec(total);
    BUILD_CUDA(cudaMemcpyAsync(hcnt.data(), cnt, total * sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    BUILD_CUDA(cudaMemcpyAsync(hrec.data(), g->d_rec, total * sizeof(BrickRec), cudaMemcpyDeviceToHost, st));
    BUILD_CUDA(cudaStreamSynchronize(st));
    uint64_t acc = 0;
    for (int64_t b = 0; b < total; ++b) {
        hrec[b].off = (uint32_t)acc;
        acc += 4ull * hcnt[b];
        if (acc >= 0xffffffffull) BUILD_TRY(fail(GPE_ERR_ARG, "too many stored cells for 32-bit offsets"));
    }
    g->n_packed = (int64_t)acc;
    BUILD_CUDA(cudaMemcpyAsync(g->d_rec, hrec.data(), total * sizeof(BrickRec), cudaMemcpyHostToDevice, st));
    {
        std::vector<int32_t> hnbr(total * 6);
        BUILD_CUDA(cudaMemcpyAsync(hnbr.data(), g->d_nbr, total * 6 * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        BUILD_CUDA(cudaStreamSynchronize(st));
        std::vector<BrickRec> h7;
        build_rec7(hrec, hnbr, h7);
        BUILD_TRY(dev_alloc_t(&g->d_rec7, total * 7));
        BUILD_CUDA(cudaMemcpyAsync(g->d_rec7, h7.data(), h7.size() * sizeof(BrickRec), cudaMemcpyHostToDevice, st));
        BUILD_CUDA(cudaStreamSynchronize(st));
        if (g->stencil == 19) {
            int32_t *d_e = nullptr;
            BUILD_TRY(dev_alloc_t(&d_e, total * 12));
            k_edge_neighbors<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(total, coords, g->nbx, g->nby, g->nbz,
                                                                            g->d_bvol, d_e);
            std::vector<int32_t> he(total * 12);
            cudaError_t e1 = cudaGetLastError();
            if (e1 == cudaSuccess) e1 = cudaMemcpyAsync(he.data(), d_e, he.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, st);
            if (e1 == cudaSuccess) e1 = cudaStreamSynchronize(st);
            dev_free(d_e);
            BUILD_CUDA(e1);
            std::vector<BrickRec> h19;
            build_rec19(hrec, hnbr, he, h19);
            BUILD_TRY(dev_alloc_t(&g->d_rec19, total * 19));
            BUILD_CUDA(cudaMemcpyAsync(g->d_rec19, h19.data(), h19.size() * sizeof(BrickRec), cudaMemcpyHostToDevice, st));
            BUILD_CUDA(cudaStreamSynchronize(st));
        }
    }
    for (int sl = 0; sl < g->n_slots; ++sl) {
        BUILD_TRY(dev_alloc_t(&g->d_V[sl], g->n_packed));
        k_pack<<<g->nsm * 8, 256, 0, st>>>(g->n_stored, g->bc, g->d_mask, g->d_rec, tmpV[sl], g->d_V[sl],
                                          sl == 0 ? (double)INFINITY : 0.0);
        BUILD_CUDA(cudaGetLastError());
    }
    BUILD_CUDA(cudaStreamSynchronize(st));
    cleanup();
#undef BUILD_TRY
#undef BUILD_CUDA
    *out = g;
    return GPE_OK;
}

static int stage_dense(const gpe_box *box, const void *V, int V_dtype, int on_device,
                       const void **dptr, void **owned, cudaStream_t st)
{
    *owned = nullptr;
    if (!V) return fail(GPE_ERR_ARG, "V is NULL");
    if (V_dtype != GPE_F64 && V_dtype != GPE_F32) return fail(GPE_ERR_ARG, "V_dtype must be GPE_F64 or GPE_F32");
    if (on_device) {
        *dptr = V;
        return GPE_OK;
    }
    size_t bytes = (size_t)box->nx * box->ny * box->nz * (V_dtype == GPE_F64 ? 8 : 4);
    GPE_TRY(dev_alloc(owned, bytes));
    cudaError_t e = cudaMemcpyAsync(*owned, V, bytes, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) {
        dev_free(*owned);
        *owned = nullptr;
        return cuda_fail(e, "cudaMemcpyAsync(V)", __FILE__, __LINE__);
    }
    *dptr = *owned;
    return GPE_OK;
}

int ensure_vf(gpe_grid *g, int slot)
{
    if (g->d_Vf[slot]) return GPE_OK;
    GPE_TRY(dev_alloc_t(&g->d_Vf[slot], g->n_packed));
    // conversion is ordered on the legacy stream; synchronise so that any
    // stream sees the finished copy
    extern int convert_to_float(const double *src, float *dst, int64_t n);
    GPE_TRY(convert_to_float(g->d_V[slot], g->d_Vf[slot], g->n_packed));
    return GPE_OK;
}

}  // namespace gpe

using namespace gpe;

extern "C" int gpe_grid_create_dense(const gpe_box *box, const void *V, int V_dtype, int V_on_device,
                                     double V_cut, const gpe_grid_opts *opts, gpe_grid **out,
                                     gpe_stream stream)
{
    if (!out) return fail(GPE_ERR_ARG, "out is NULL");
    *out = nullptr;
    GPE_TRY(check_box(box));
    cudaStream_t st = S(stream);
    const void *dptr = nullptr;
    void *owned = nullptr;
    GPE_TRY(stage_dense(box, V, V_dtype, V_on_device, &dptr, &owned, st));
    VSource src{};
    src.mode = 0;
    src.dense = dptr;
    src.dtype = V_dtype;
    src.cut0 = V_cut;
    int rc = build_grid(box, src, opts, out, st);
    if (owned) {
        cudaStreamSynchronize(st);
        dev_free(owned);
    }
    return rc;
}

extern "C" int gpe_grid_create_analytic(const gpe_box *box, const gpe_potential *pot, double V_cut,
                                        const gpe_grid_opts *opts, gpe_grid **out, gpe_stream stream)
{
    if (!out) return fail(GPE_ERR_ARG, "out is NULL");
    *out = nullptr;
    GPE_TRY(check_box(box));
    GPE_TRY(check_pot(pot));
    VSource src{};
    src.mode = 1;
    src.p0 = potdesc(*pot);
    src.cut0 = V_cut;
    return build_grid(box, src, opts, out, S(stream));
}

extern "C" int gpe_grid_create_blend(const gpe_box *box, const gpe_potential *pot0, double cut0,
                                     const gpe_potential *pot1, double cut1, const gpe_grid_opts *opts,
                                     gpe_grid **out, gpe_stream stream)
{
    if (!out) return fail(GPE_ERR_ARG, "out is NULL");
    *out = nullptr;
    GPE_TRY(check_box(box));
    GPE_TRY(check_pot(pot0));
    GPE_TRY(check_pot(pot1));
    VSource src{};
    src.mode = 2;
    src.p0 = potdesc(*pot0);
    src.p1 = potdesc(*pot1);
    src.cut0 = cut0;
    src.cut1 = cut1;
    return build_grid(box, src, opts, out, S(stream));
}

extern "C" int gpe_grid_create_blend_dense(const gpe_box *box, const void *V0, const void *V1, int V_dtype,
                                           int V_on_device, double cut0, double cut1,
                                           const gpe_grid_opts *opts, gpe_grid **out, gpe_stream stream)
{
    if (!out) return fail(GPE_ERR_ARG, "out is NULL");
    *out = nullptr;
    GPE_TRY(check_box(box));
    cudaStream_t st = S(stream);
    const void *d0 = nullptr, *d1 = nullptr;
    void *own0 = nullptr, *own1 = nullptr;
    GPE_TRY(stage_dense(box, V0, V_dtype, V_on_device, &d0, &own0, st));
    int rc = stage_dense(box, V1, V_dtype, V_on_device, &d1, &own1, st);
    if (rc == GPE_OK) {
        VSource src{};
        src.mode = 3;
        src.dense = d0;
        src.dense1 = d1;
        src.dtype = V_dtype;
        src.cut0 = cut0;
        src.cut1 = cut1;
        rc = build_grid(box, src, opts, out, st);
    }
    if (own0 || own1) {
        cudaStreamSynchronize(st);
        dev_free(own0);
        dev_free(own1);
    }
    return rc;
}

extern "C" int gpe_grid_set_potential(gpe_grid *g, int slot, const void *V, int V_dtype, int V_on_device,
                                      gpe_stream stream)
{
    if (!g) return fail(GPE_ERR_ARG, "grid is NULL");
    if (slot != 0 && slot != 1) return fail(GPE_ERR_ARG, "slot must be 0 or 1");
    cudaStream_t st = S(stream);
    const void *dptr = nullptr;
    void *owned = nullptr;
    GPE_TRY(stage_dense(&g->box, V, V_dtype, V_on_device, &dptr, &owned, st));
    int rc = GPE_OK;
    if (!g->d_V[slot]) {
        rc = dev_alloc_t(&g->d_V[slot], g->n_packed);
        if (rc == GPE_OK) rc = dev_zero(g->d_V[slot], g->n_packed * sizeof(double));
    }
    if (rc == GPE_OK) {
        k_set_potential<<<(unsigned)g->nb, std::min(g->bc, 256), 0, st>>>(dptr, V_dtype, boxd(g->box), g->bx,
                                                                        g->by, g->bz, g->d_org, g->d_mask,
                                                                        g->d_rec, g->d_V[slot]);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) rc = cuda_fail(e, "k_set_potential", __FILE__, __LINE__);
    }
    if (rc == GPE_OK && slot == 1) g->n_slots = 2;
    unsigned long long *vb = nullptr;
    if (rc == GPE_OK) rc = dev_alloc_t(&vb, 1);
    if (rc == GPE_OK) {
        cudaMemsetAsync(vb, 0, sizeof(unsigned long long), st);
        k_vmax<<<g->nsm * 4, 256, 0, st>>>(g->n_packed, g->d_V[0], g->n_slots > 1 ? g->d_V[1] : nullptr, vb);
        unsigned long long h = 0;
        cudaMemcpyAsync(&h, vb, sizeof h, cudaMemcpyDeviceToHost, st);
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = cuda_fail(e, "set_potential", __FILE__, __LINE__);
        long long hv = (long long)h;
        memcpy(&g->v_max, &hv, sizeof(double));
    }
    dev_free(vb);
    if (owned) {
        cudaStreamSynchronize(st);
        dev_free(owned);
    }
    if (g->d_Vf[slot]) {
        dev_free(g->d_Vf[slot]);
        g->d_Vf[slot] = nullptr;
    }
    return rc;
}

extern "C" int gpe_grid_get_info(const gpe_grid *g, gpe_grid_info *out)
{
    if (!g || !out) return fail(GPE_ERR_ARG, "NULL argument");
    out->n_active = g->n_active;
    out->n_bricks = g->nb;
    out->n_stored = g->n_stored;
    out->n_packed = g->n_packed;
    out->bx = g->bx;
    out->by = g->by;
    out->bz = g->bz;
    out->mask_mode = g->mask_mode;
    out->order = g->order;
    out->n_slots = g->n_slots;
    out->v_max = g->v_max;
    out->box = g->box;
    return GPE_OK;
}

extern "C" int gpe_grid_bricks(const gpe_grid *g, int32_t *origins, int32_t *nbr)
{
    if (!g) return fail(GPE_ERR_ARG, "grid is NULL");
    if (origins) GPE_TRY_CUDA(cudaMemcpy(origins, g->d_org, g->nb * 3 * sizeof(int32_t), cudaMemcpyDeviceToHost));
    if (nbr) GPE_TRY_CUDA(cudaMemcpy(nbr, g->d_nbr, g->nb * 6 * sizeof(int32_t), cudaMemcpyDeviceToHost));
    return GPE_OK;
}

extern "C" int gpe_grid_mask(const gpe_grid *g, uint32_t *bits)
{
    if (!g || !bits) return fail(GPE_ERR_ARG, "NULL argument");
    GPE_TRY_CUDA(cudaMemcpy(bits, g->d_mask, g->n_stored / 32 * sizeof(uint32_t), cudaMemcpyDeviceToHost));
    return GPE_OK;
}

extern "C" int gpe_grid_potential(const gpe_grid *g, int slot, double *V)
{
    if (!g || !V) return fail(GPE_ERR_ARG, "NULL argument");
    if (slot < 0 || slot > 1 || !g->d_V[slot]) return fail(GPE_ERR_ARG, "potential slot %d not set", slot);
    GPE_TRY_CUDA(cudaMemcpy(V, g->d_V[slot], g->n_packed * sizeof(double), cudaMemcpyDeviceToHost));
    return GPE_OK;
}

extern "C" int gpe_grid_destroy(gpe_grid *g)
{
    if (!g) return GPE_OK;
    if (g->n_states > 0) return fail(GPE_ERR_STATE, "grid still has %d live states", g->n_states);
    grid_free(g);
    return GPE_OK;
}

// ------------------------------------------------------------ Thomas-Fermi mu
namespace gpe {

// One pass of the Thomas-Fermi solve: over the cells with V < mu, the sum of
// V and their count (result[0], result[1]).  Blocks take whole x-rows, so a
// cell's coordinates need no division; dense sources read V directly.
__global__ void k_tf_pass(VSource src, BoxD box, double mu, double *partials, unsigned int *counter,
                          double *result)
{
    double acc[2] = {0.0, 0.0};
    const int64_t rows = box.ny * box.nz;
    for (int64_t r = blockIdx.x; r < rows; r += gridDim.x) {
        const int64_t j = r % box.ny, k = r / box.ny;
        for (int64_t i = threadIdx.x; i < box.nx; i += blockDim.x) {
            double v0, v1;
            bool sel;
            cell_values(src, box, i, j, k, v0, v1, sel);
            if (v0 < mu) {
                acc[0] += v0;
                acc[1] += 1.0;
            }
        }
    }
    double tot[2];
    if (reduce_finish<2>(acc, partials, counter, tot) && threadIdx.x == 0) {
        result[0] = tot[0];
        result[1] = tot[1];
    }
}

// Eq. (5): the mu at which the Thomas-Fermi atom number
//   F(mu) = sum over the box of max(mu - V, 0) / g dV
// equals N.  F is convex, increasing and piecewise linear in mu, so Newton's
// method started above the root stays above it and reaches the root exactly
// once the set {V < mu} stops changing:
//   mu <- (g N / dV + sum_{V < mu} V) / #{V < mu}.
// The first pass takes every cell (mu = +inf), whose line lies below F, so
// its root already bounds the true one from above.
static int tf_mu_impl(const gpe_box *box, const VSource &src, double g, double N, double *mu, cudaStream_t st)
{
    if (!(g > 0)) return fail(GPE_ERR_ARG, "g must be > 0 for the Thomas-Fermi estimate");
    if (!(N > 0)) return fail(GPE_ERR_ARG, "N must be > 0");
    if (!mu) return fail(GPE_ERR_ARG, "mu is NULL");
    int dev = 0;
    GPE_TRY_CUDA(cudaGetDevice(&dev));
    const int64_t rows = box->ny * box->nz;
    const int blocks = (int)std::min<int64_t>(rows, (int64_t)sm_count(dev) * 8);
    RedScratch r;
    GPE_TRY(red_alloc(r, blocks));
    double *res = nullptr, h[2];
    int rc = dev_alloc_t(&res, 2);
    const BoxD bd = boxd(*box);
    const double dV = box->hx * box->hy * box->hz;
    const double target = g * N / dV;
    auto pass = [&](double m) -> int {
        k_tf_pass<<<blocks, 256, 0, st>>>(src, bd, m, r.partials, r.counter, res);
        GPE_TRY_CUDA(cudaGetLastError());
        GPE_TRY_CUDA(cudaMemcpyAsync(h, res, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
        GPE_TRY_CUDA(cudaStreamSynchronize(st));
        return GPE_OK;
    };
    double m = INFINITY;
    double count = -1.0;
    for (int it = 0; it < 200 && rc == GPE_OK; ++it) {
        rc = pass(m);
        if (rc != GPE_OK) break;
        if (!(h[1] > 0.0)) {
            rc = fail(GPE_ERR_ARG, "Thomas-Fermi solve found no cell below mu (V not finite?)");
            break;
        }
        const double next = (target + h[0]) / h[1];
        const bool same_set = h[1] == count;
        count = h[1];
        if (!std::isfinite(next)) {
            rc = fail(GPE_ERR_ARG, "Thomas-Fermi solve: non-finite mu (V not finite?)");
            break;
        }
        if (same_set || !(next < m)) {
            m = std::min(m, next);
            break;
        }
        m = next;
    }
    if (rc == GPE_OK) *mu = m;
    dev_free(res);
    red_free(r);
    return rc;
}

}  // namespace gpe

extern "C" int gpe_tf_mu_dense(const gpe_box *box, const void *V, int V_dtype, int V_on_device, double g,
                               double N, double *mu, gpe_stream stream)
{
    GPE_TRY(check_box(box));
    cudaStream_t st = S(stream);
    const void *dptr = nullptr;
    void *owned = nullptr;
    GPE_TRY(stage_dense(box, V, V_dtype, V_on_device, &dptr, &owned, st));
    VSource src{};
    src.mode = 0;
    src.dense = dptr;
    src.dtype = V_dtype;
    src.cut0 = 0.0;
    int rc = tf_mu_impl(box, src, g, N, mu, st);
    if (owned) {
        cudaStreamSynchronize(st);
        dev_free(owned);
    }
    return rc;
}

extern "C" int gpe_tf_mu_analytic(const gpe_box *box, const gpe_potential *pot, double g, double N, double *mu,
                                  gpe_stream stream)
{
    GPE_TRY(check_box(box));
    GPE_TRY(check_pot(pot));
    VSource src{};
    src.mode = 1;
    src.p0 = potdesc(*pot);
    return tf_mu_impl(box, src, g, N, mu, S(stream));
}
