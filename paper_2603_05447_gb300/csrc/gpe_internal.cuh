// gpe_internal.cuh -- shared internals of libgpeshell (not part of the ABI).
//
// Layout of a grid in device memory.  Bricks of BC = BX*BY*BZ lattice cells,
// local index l = x + BX*(y + BY*z); "slot" = brick * BC + l addresses the
// lattice.  A segment is 4 consecutive cells along x (local segment q = l/4).
// Only segments holding an active cell are stored ("packed" layout):
//   d_org  [nb*3]  int32    brick origin in cells (i0, j0, k0)
//   d_nbr  [nb*6]  int32    face-neighbour brick ids (-x +x -y +y -z +z), -1 = none
//   d_mask [ns/32] uint32   active-cell bits of the lattice, bit slot&31 of word slot/32
//   d_rec  [nb]    BrickRec stored-segment bits, per-word prefix counts, packed offset
//   d_V[s] [n_packed] double potential slot s (0: V or V0, 1: V1); the inactive
//                           cells of stored segments hold +inf in slot 0
// Packed index of cell l of brick b (if its segment is stored):
//   rec.off + 4*(rank of segment l/4 among the brick's stored segments) + l%4.
// Inactive cells of stored segments hold psi = 0 and are never updated (the
// +inf potential marks them); cells of absent segments and bricks are not
// stored and read as psi = 0: Dirichlet zero on the rows/columns deleted
// from the Laplacian (Sec. II A).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <vector>

#include "gpe.h"

namespace gpe {

// ------------------------------------------------------------ errors
int fail(int code, const char *fmt, ...);
int cuda_fail(cudaError_t e, const char *expr, const char *file, int line);

#define GPE_TRY_CUDA(x)                                                      \
    do {                                                                     \
        cudaError_t e__ = (x);                                               \
        if (e__ != cudaSuccess)                                              \
            return ::gpe::cuda_fail(e__, #x, __FILE__, __LINE__);            \
    } while (0)
#define GPE_TRY(x)                                                           \
    do {                                                                     \
        int r__ = (x);                                                       \
        if (r__ != GPE_OK) return r__;                                       \
    } while (0)
// every kernel launch of the library is followed by GPE_LAUNCH_CHECK(), which
// also counts it (gpe_launch_count)
void count_launch();
#define GPE_LAUNCH_CHECK()                                                   \
    do {                                                                     \
        ::gpe::count_launch();                                               \
        GPE_TRY_CUDA(cudaGetLastError());                                    \
    } while (0)

int dev_alloc(void **p, size_t bytes);
template <typename T>
inline int dev_alloc_t(T **p, size_t count)
{
    return dev_alloc(reinterpret_cast<void **>(p), count * sizeof(T));
}
void dev_free(void *p);
int dev_zero(void *p, size_t bytes);  // memset 0 and wait (any stream may use it next)

inline cudaStream_t S(gpe_stream s) { return reinterpret_cast<cudaStream_t>(s); }

// supported brick shapes; the kernels are instantiated for each
int shape_id(int bx, int by, int bz);  // 0: 8x8x8, 1: 8x8x4, 2: 8x4x4

int sm_count(int device);

// per-brick record of the packed layout (32 bytes)
struct BrickRec {
    uint32_t m[4];  // bit q: segment q is stored
    uint32_t off;   // packed index of the brick's first stored cell
    uint32_t pre;   // byte w: stored segments in mask words < w
    uint32_t pad[2];
};

// per brick: its record followed by its six face neighbours' (-x +x -y +y -z
// +z; empty records for absent neighbours), built on the host
void build_rec7(const std::vector<BrickRec> &rec, const std::vector<int32_t> &nbr, std::vector<BrickRec> &out);
// records of each brick, its 6 face and 12 edge neighbours (edge order: xy
// (-1,-1,0) (+1,-1,0) (-1,+1,0) (+1,+1,0); xz (-1,0,-1) (+1,0,-1) (-1,0,+1)
// (+1,0,+1); yz (0,-1,-1) (0,+1,-1) (0,-1,+1) (0,+1,+1))
void build_rec19(const std::vector<BrickRec> &rec, const std::vector<int32_t> &nbr,
                 const std::vector<int32_t> &nbr_e, std::vector<BrickRec> &out);

// packed index of the first cell of segment q, if stored
__host__ __device__ __forceinline__ bool seg_index(const BrickRec &r, int q, uint32_t &idx)
{
    const int w = q >> 5, bit = q & 31;
    const uint32_t m = r.m[w];
    if (!((m >> bit) & 1u)) return false;
#ifdef __CUDA_ARCH__
    const uint32_t below = __popc(m & ((1u << bit) - 1u));
#else
    const uint32_t below = (uint32_t)__builtin_popcount(m & ((1u << bit) - 1u));
#endif
    idx = r.off + 4u * (((r.pre >> (8 * w)) & 0xffu) + below);
    return true;
}

// ------------------------------------------------------------ complex types
template <typename R> struct Cx;
template <> struct Cx<float> { using T = float2; };
template <> struct Cx<double> { using T = double2; };

template <typename R>
__device__ __forceinline__ typename Cx<R>::T cmk(R x, R y)
{
    typename Cx<R>::T c;
    c.x = x;
    c.y = y;
    return c;
}

// ------------------------------------------------------------ brick tiles
// A tile holds one brick plus a one-cell face halo (edges/corners unused by
// the 7-point stencil), (BX+2)(BY+2)(BZ+2) entries, x fastest.
template <int BX, int BY, int BZ>
struct Brick {
    static constexpr int BC = BX * BY * BZ;
    static constexpr int TX = BX + 2, TY = BY + 2, TZ = BZ + 2;
    static constexpr int TN = TX * TY * TZ;
    static constexpr int NXF = BY * BZ, NYF = BX * BZ, NZF = BX * BY;
    static constexpr int NH = 2 * (NXF + NYF + NZF);
    __device__ __forceinline__ static int t(int x, int y, int z)
    {
        return (x + 1) + TX * ((y + 1) + TY * (z + 1));
    }
};

__device__ __forceinline__ bool mask_bit(const uint32_t *__restrict__ mask, int64_t slot)
{
    return (__ldg(&mask[slot >> 5]) >> (slot & 31)) & 1u;
}

// Stage brick b of `src` and its six face halos into shared memory, passing
// each loaded value through xf(value, slot).  Interior loads are predicated on
// the active mask (inactive slots are zero in memory; skipping them saves
// DRAM sectors).  xf(0, slot) must be 0.
template <int BX, int BY, int BZ, typename CT, typename XF>
__device__ __forceinline__ void load_tile(CT *tile, const CT *src, int64_t b,
                                          const int32_t *__restrict__ nbr,
                                          const uint32_t *__restrict__ mask, XF xf)
{
    using B = Brick<BX, BY, BZ>;
    const int64_t base = b * B::BC;
    CT zero;
    zero.x = 0;
    zero.y = 0;
    for (int l = threadIdx.x; l < B::BC; l += blockDim.x) {
        const int64_t s = base + l;
        CT v = zero;
        if (mask_bit(mask, s)) v = xf(src[s], s);
        const int x = l % BX, y = (l / BX) % BY, z = l / (BX * BY);
        tile[B::t(x, y, z)] = v;
    }
    for (int h = threadIdx.x; h < B::NH; h += blockDim.x) {
        int face, u, lx, ly, lz, tx, ty, tz;
        if (h < 2 * B::NXF) {
            face = h / B::NXF;  // 0: -x, 1: +x
            u = h % B::NXF;
            ly = u % BY;
            lz = u / BY;
            lx = face ? 0 : BX - 1;
            tx = face ? BX : -1;
            ty = ly;
            tz = lz;
        } else if (h < 2 * (B::NXF + B::NYF)) {
            const int hh = h - 2 * B::NXF;
            face = 2 + hh / B::NYF;  // 2: -y, 3: +y
            u = hh % B::NYF;
            lx = u % BX;
            lz = u / BX;
            ly = (face == 3) ? 0 : BY - 1;
            tx = lx;
            ty = (face == 3) ? BY : -1;
            tz = lz;
        } else {
            const int hh = h - 2 * (B::NXF + B::NYF);
            face = 4 + hh / B::NZF;  // 4: -z, 5: +z
            u = hh % B::NZF;
            lx = u % BX;
            ly = u / BX;
            lz = (face == 5) ? 0 : BZ - 1;
            tx = lx;
            ty = ly;
            tz = (face == 5) ? BZ : -1;
        }
        const int nb = __ldg(&nbr[b * 6 + face]);
        CT v = zero;
        if (nb >= 0) {
            const int64_t s = (int64_t)nb * B::BC + lx + BX * (ly + BY * lz);
            v = xf(src[s], s);
        }
        tile[B::t(tx, ty, tz)] = v;
    }
}

// 7-point Laplacian (Eq. (B1)) of tile entry (x, y, z).
template <int BX, int BY, int BZ, typename R, typename CT>
__device__ __forceinline__ CT tile_laplacian(const CT *tile, int x, int y, int z,
                                             R ihx2, R ihy2, R ihz2)
{
    using B = Brick<BX, BY, BZ>;
    const int c = B::t(x, y, z);
    const CT p = tile[c];
    const CT xm = tile[c - 1], xp = tile[c + 1];
    const CT ym = tile[c - B::TX], yp = tile[c + B::TX];
    const CT zm = tile[c - B::TX * B::TY], zp = tile[c + B::TX * B::TY];
    CT r;
    r.x = (xp.x - 2 * p.x + xm.x) * ihx2 + (yp.x - 2 * p.x + ym.x) * ihy2 +
          (zp.x - 2 * p.x + zm.x) * ihz2;
    r.y = (xp.y - 2 * p.y + xm.y) * ihx2 + (yp.y - 2 * p.y + ym.y) * ihy2 +
          (zp.y - 2 * p.y + zm.y) * ihz2;
    return r;
}

// ------------------------------------------------------------ reductions
// Deterministic FP64 block reduction of NV values with a "last block
// finishes" epilogue: every block writes its partial sums to
// partials[blockIdx.x*NV + k]; the last block to arrive sums all partials in
// a fixed order.  Returns true in the one block that holds the totals, whose
// thread 0 then has them in tot[].  The counter is reset to 0 by that block.
template <int NV>
__device__ __forceinline__ bool reduce_finish(double (&v)[NV], double *partials,
                                              unsigned int *counter, double (&tot)[NV])
{
    __shared__ double sm[NV][32];
    __shared__ bool is_last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double x = v[k];
        for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
        if (lane == 0) sm[k][warp] = x;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double x = lane < nwarps ? sm[k][lane] : 0.0;
            for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
            if (lane == 0) partials[(int64_t)blockIdx.x * NV + k] = x;
        }
    }
    if (threadIdx.x == 0) {
        __threadfence();
        unsigned int ticket = atomicAdd(counter, 1u);
        is_last = (ticket == gridDim.x - 1);
    }
    __syncthreads();
    if (!is_last) return false;
    __threadfence();
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double x = 0.0;
        for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x)
            x += __ldcg(&partials[(int64_t)i * NV + k]);
        for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
        __syncthreads();
        if (lane == 0) sm[k][warp] = x;
        __syncthreads();
        if (warp == 0) {
            x = lane < nwarps ? sm[k][lane] : 0.0;
            for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
            if (lane == 0) tot[k] = x;
        }
    }
    if (threadIdx.x == 0) *counter = 0u;
    return true;
}

// Per-launch scratch for reductions: partial sums (max_blocks * 8 doubles),
// a completion counter and a few FP64 scalars (ITP scale, results).
struct RedScratch {
    double *partials = nullptr;
    unsigned int *counter = nullptr;
    double *scalars = nullptr;  // [0] ITP scale, [1] last norm, [2..9] observables
    int max_blocks = 0;
};
int red_alloc(RedScratch &r, int max_blocks);
void red_free(RedScratch &r);

}  // namespace gpe

// ------------------------------------------------------------ handles
// launch the staged stage kernels with programmatic dependent launch (off:
// measured no gain for RK4 and a slower imaginary-time step on GB300)
#ifndef GPE_PDL
#define GPE_PDL 0
#endif

struct gpe_grid {
    int device = 0;
    gpe_box box{};
    int bx = 8, by = 8, bz = 8, bc = 512, shape = 0;
    int mask_mode = 0, order = 0;
    int64_t nbx = 0, nby = 0, nbz = 0;
    int64_t nb = 0, n_stored = 0, n_active = 0;
    int64_t n_packed = 0;
    int32_t *d_org = nullptr;
    int32_t *d_nbr = nullptr;
    uint32_t *d_mask = nullptr;
    gpe::BrickRec *d_rec = nullptr;
    gpe::BrickRec *d_rec7 = nullptr;  // [nb*7] record of each brick and of its six face neighbours
    gpe::BrickRec *d_rec19 = nullptr; // [nb*19] ... and of its 12 edge neighbours (19-point grids)
    int stencil = 7;                  // 7 or 19 points
    int32_t *d_nbr18 = nullptr;       // [nb*18] face then edge neighbour ids (PAIR schedule, built on first use)
    int32_t *d_bvol = nullptr;  // brick-grid volume nbx*nby*nbz -> brick id or -1
    double *d_V[2] = {nullptr, nullptr};
    float *d_Vf[2] = {nullptr, nullptr};  // float copies, made on first use
    // wavefront schedule (built on first use): chunks of `cb` consecutive
    // bricks, the chunk range each chunk's stencils touch, and the task order
    // for 2-stage (imaginary time) and 4-stage (RK4) steps
    int cb = 0;
    int64_t n_chunks = 0;
    int32_t *d_chunk_lohi = nullptr;  // [n_chunks*2]
    int32_t *d_tasks = nullptr;       // [2*n_chunks] for 2 stages, then [4*n_chunks] for 4
    // warp-task schedule of the two-stage RK4 launches (GPE_SCHED_WAVE2): per
    // chunk the sorted chunks its stencils read (CSR), and the task order
    int32_t *d_dep_off = nullptr;     // [n_chunks + 1]
    int32_t *d_dep_ids = nullptr;
    int32_t *d_tasks_w = nullptr;     // [2*n_chunks]
    int sched = -1;                   // GPE_SCHED_* used by the step calls
    int n_slots = 1;
    double v_max = 0.0;
    int nsm = 0;
    int n_states = 0;
};

struct gpe_state {
    gpe_grid *grid = nullptr;
    int dtype = GPE_C128;
    size_t elem = 16;       // bytes per complex element
    void *d_psi = nullptr;  // n_packed complex
    void *d_work[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};  // RK stage states / ITP tmp
    void *d_E = nullptr;    // ITP exp(-V dt/2), state precision
    double E_dt = -1.0;     // dt that d_E was made for
    double *d_clock = nullptr;  // device time base for ramps
    gpe::RedScratch red;
    gpe_obs *h_obs = nullptr;   // pinned host landing buffer
    // wavefront bookkeeping: per-chunk completion stamps (monotonic), the
    // dynamic ticket counter, the finish counter and a device error word
    uint32_t *d_done = nullptr;
    unsigned long long *d_ctr = nullptr;  // [0] tickets, [1] finished ITP chunks, [2] error
    double *d_chunk_norm = nullptr;       // per-chunk FP64 partial norms (ITP)
    uint32_t epoch = 0;                   // stages completed so far (flags compare to it)
    unsigned long long ticket_base = 0, finish_base = 0;
    // CUDA graphs of `graph_steps` staged steps ([0] real time, [1] imaginary)
    int graph_steps = 32;
    bool pdl = GPE_PDL != 0;  // stage kernels launched with programmatic dependent launch
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    unsigned long long gkey[2] = {0, 0};
    int gnodes[2] = {0, 0};
    cudaStream_t gcap = nullptr;
};

namespace gpe {
int ensure_work(gpe_state *st, int n);          // allocate d_work[0..n-1] (zeroed)
// step drivers of 19-point grids (step19.cu)
int rk4_run19(gpe_state *st, const gpe_real_params *p, int64_t nsteps, double t0, cudaStream_t s);
int itp_run19(gpe_state *st, const gpe_imag_params *p, int64_t nsteps, cudaStream_t s);
int obs_run19(const gpe_state *st, double g, double s_blend, cudaStream_t s);
int ensure_vf(gpe_grid *g, int slot);           // float copy of a potential slot
const void *potential_ptr(gpe_state *st, int slot);  // V slot in state precision
int launch_blocks(const gpe_grid *g, int threads, int per_sm);
}  // namespace gpe
