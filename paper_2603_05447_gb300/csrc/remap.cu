// remap.cu -- a state carried from one grid to another over the same box:
// the wavefunction remapped between the old and new grids when the region
// of interest is selected again between ramp stages (Sec. V).
#include "stencil.cuh"

namespace gpe {

struct RemapSide {
    const int32_t *org;    // brick origins (3 per brick)
    const BrickRec *rec;
    const uint32_t *mask;  // bc bits per brick
    const int32_t *bvol;   // brick grid -> brick id or -1
    int bx, by, bz;
    int64_t nbx, nby, nbz;
};

// One thread per stored lattice cell of dst (brick b, local cell l): its
// value is src's at the same box cell when that cell is active in both
// grids, else 0.  Cells of stored segments only: the others are not stored.
template <typename CT>
__global__ void k_remap(CT *dst, const CT *src, RemapSide D, RemapSide S, int64_t n_lattice)
{
    const int dbc = D.bx * D.by * D.bz;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n_lattice;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = t / dbc;
        const int l = (int)(t % dbc);
        uint32_t jd;
        if (!seg_index(D.rec[b], l >> 2, jd)) continue;
        jd += (uint32_t)(l & 3);
        CT v = czero<CT>();
        if ((D.mask[b * (dbc / 32) + (l >> 5)] >> (l & 31)) & 1u) {
            const int64_t i = D.org[3 * b] + l % D.bx;
            const int64_t j = D.org[3 * b + 1] + (l / D.bx) % D.by;
            const int64_t k = D.org[3 * b + 2] + l / (D.bx * D.by);
            const int64_t qx = i / S.bx, qy = j / S.by, qz = k / S.bz;
            if (qx < S.nbx && qy < S.nby && qz < S.nbz) {
                const int32_t sb = S.bvol[qx + S.nbx * (qy + S.nby * qz)];
                if (sb >= 0) {
                    const int ls = (int)((i - qx * S.bx) + S.bx * ((j - qy * S.by) + S.by * (k - qz * S.bz)));
                    uint32_t js;
                    if (seg_index(S.rec[sb], ls >> 2, js)) v = src[js + (uint32_t)(ls & 3)];  // 0 where inactive
                }
            }
        }
        dst[jd] = v;
    }
}

static RemapSide side(const gpe_grid *g)
{
    return RemapSide{g->d_org, g->d_rec, g->d_mask, g->d_bvol, g->bx, g->by, g->bz, g->nbx, g->nby, g->nbz};
}

static bool same_box(const gpe_box &a, const gpe_box &b)
{
    return a.nx == b.nx && a.ny == b.ny && a.nz == b.nz && a.hx == b.hx && a.hy == b.hy && a.hz == b.hz &&
           a.x0 == b.x0 && a.y0 == b.y0 && a.z0 == b.z0;
}

}  // namespace gpe

using namespace gpe;

extern "C" int gpe_state_remap(gpe_state *dst, const gpe_state *src, gpe_stream stream)
{
    if (!dst || !src) return fail(GPE_ERR_ARG, "NULL state");
    if (dst == src) return fail(GPE_ERR_ARG, "dst and src are the same state");
    if (dst->dtype != src->dtype) return fail(GPE_ERR_ARG, "states differ in dtype");
    const gpe_grid *dg = dst->grid, *sg = src->grid;
    if (dg->device != sg->device) return fail(GPE_ERR_ARG, "states live on different devices");
    if (!same_box(dg->box, sg->box)) return fail(GPE_ERR_ARG, "grids differ in box sizes, spacings or origin");
    int dev = -1;
    GPE_TRY_CUDA(cudaGetDevice(&dev));
    if (dev != dg->device) return fail(GPE_ERR_STATE, "states live on device %d but device %d is current", dg->device, dev);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int64_t n_lattice = dg->nb * (int64_t)dg->bc;
    const int blocks = (int)std::min<int64_t>((n_lattice + 255) / 256, (int64_t)dg->nsm * 16);
    if (n_lattice == 0) return GPE_OK;
    switch (dst->dtype) {
    case GPE_C128:
        k_remap<double2><<<blocks, 256, 0, s>>>((double2 *)dst->d_psi, (const double2 *)src->d_psi, side(dg), side(sg),
                                                n_lattice);
        break;
    case GPE_C64:
        k_remap<float2><<<blocks, 256, 0, s>>>((float2 *)dst->d_psi, (const float2 *)src->d_psi, side(dg), side(sg),
                                               n_lattice);
        break;
    case GPE_R64:
        k_remap<double><<<blocks, 256, 0, s>>>((double *)dst->d_psi, (const double *)src->d_psi, side(dg), side(sg),
                                               n_lattice);
        break;
    default:
        k_remap<float><<<blocks, 256, 0, s>>>((float *)dst->d_psi, (const float *)src->d_psi, side(dg), side(sg),
                                              n_lattice);
        break;
    }
    GPE_LAUNCH_CHECK();
    return GPE_OK;
}
