// step.cu -- wavefunction states, the real-time RK4 step, the imaginary-time
// split step with renormalisation, and the FP64 observables of libgpeshell.
//
// Every stencil kernel stages one brick plus its face halo in shared memory
// (the paper's per-block tile of Sec. II B, gathered here from the six face
// neighbours through the brick-neighbour table and the packed-layout ranks),
// evaluates the 7-point Laplacian of Eq. (B1) from the tile, applies the
// pointwise terms of the equation and writes the active cells.
//
// Two schedules run the same per-brick arithmetic:
//  * STAGED: one launch per stage; blocks walk the brick list with a fixed
//    stride, so per-block partial sums (and every FP64 reduction) are
//    deterministic.
//  * WAVE: one persistent launch per time step.  The work is split into
//    (stage, chunk) tasks, a chunk being `cb` consecutive bricks.  Tasks are
//    handed out from an atomic ticket counter in an order where every
//    dependency of a task has a smaller ticket (stage s of chunk c needs stage
//    s-1 of every chunk its stencils read), and a task waits for those
//    completion stamps before it reads.  The live window of intermediate
//    stage states is a few brick layers wide, so it stays in L2 instead of
//    making a round trip through HBM per stage.  Waits are bounded (about 2 s);
//    a wait that runs out sets the state's error word and the call that reads
//    results reports GPE_ERR_CUDA.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "gpe_internal.cuh"
#include "kernels.cuh"
#include "itp_pair.cuh"
#include "pair.cuh"

namespace gpe {

// ------------------------------------------------------------ small kernels
__global__ void k_d2f(const double *s, float *d, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        d[i] = (float)s[i];
}

int convert_to_float(const double *src, float *dst, int64_t n)
{
    k_d2f<<<1024, 256>>>(src, dst, n);
    GPE_LAUNCH_CHECK();
    GPE_TRY_CUDA(cudaStreamSynchronize(0));
    return GPE_OK;
}

__global__ void k_set_scalar(double *p, double v) { *p = v; }

// ------------------------------------------------------------ launch helper
static std::mutex g_occ_mu;
static std::unordered_map<const void *, int> g_occ;

// resident blocks per SM of a stencil kernel (prepared once: dynamic shared
// memory opt-in and occupancy query)
template <typename K>
static int per_sm_for(K kernel, int threads, size_t smem)
{
    {
        std::lock_guard<std::mutex> lk(g_occ_mu);
        auto it = g_occ.find((const void *)kernel);
        if (it != g_occ.end()) return it->second;
    }
    const int per = prepare_kernel(kernel, threads, smem);
    std::lock_guard<std::mutex> lk(g_occ_mu);
    g_occ[(const void *)kernel] = per;
    return per;
}

// a grid of resident blocks of nw warps, no more than one warp per brick
template <typename K>
static int blocks_for_nw(K kernel, const gpe_grid *g, size_t smem, int nw)
{
    int64_t b = (int64_t)g->nsm * per_sm_for(kernel, 32 * nw, smem);
    const int64_t need = (g->nb + nw - 1) / nw;
    if (b > need) b = need;
    if (b < 1) b = 1;
    return (int)b;
}
template <typename R, typename K>
static int blocks_for(K kernel, const gpe_grid *g, size_t smem)
{
    return blocks_for_nw(kernel, g, smem, KernelCfg<R>::NW);
}

// Launch a stage kernel; with pdl, with programmatic stream serialisation so
// that it can become resident during the previous kernel's tail (the kernel
// itself waits for that grid before reading its output: pdl_enter).
template <typename... KArgs, typename... Args>
static cudaError_t launch_stage(void (*k)(KArgs...), unsigned grid, unsigned threads, size_t smem, cudaStream_t s,
                                bool pdl, Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, k, args...);
}

// ------------------------------------------------------------ wavefront sync
__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(uint32_t *p, uint32_t v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

constexpr unsigned long long WAIT_NS = 2000000000ull;  // 2 s
constexpr long long WAIT_ITERS = 40000000LL;           // backstop if the timer stalls

// Called by all 32 lanes of one warp: wait until done[c] >= target for every
// chunk c in [lo, hi].  Returns false (and sets *err) if the wait runs out
// after limit_ns.
__device__ bool wait_chunks(const uint32_t *done, int lo, int hi, uint32_t target, unsigned long long *err,
                            unsigned long long limit_ns = WAIT_NS)
{
    const int lane = threadIdx.x & 31;
    const unsigned long long t0 = global_ns();
    for (long long it = 0; it < WAIT_ITERS; ++it) {
        bool ok = true;
        for (int i = lo + lane; i <= hi; i += 32) ok = ok && (ld_acquire(done + i) >= target);
        if (__all_sync(0xffffffffu, ok)) return true;
        if (global_ns() - t0 > limit_ns) break;
        __nanosleep(200);
    }
    if (lane == 0) atomicOr(err, 1ull);
    return false;
}

// Self-test of the bounded wait: one warp waits for a completion stamp that
// nothing sets; the wait must give up after limit_ns and report it.
__global__ void k_wait_selftest(const uint32_t *flags, unsigned long long *err, unsigned long long limit_ns,
                                unsigned long long *elapsed)
{
    const unsigned long long t0 = global_ns();
    wait_chunks(flags, 0, 0, 1u, err, limit_ns);
    if (threadIdx.x == 0) *elapsed = global_ns() - t0;
}

// Invalidate, without write-back, the L2 lines lying wholly inside
// [p, p + bytes): the data is dead (every reader has finished).
__device__ __forceinline__ void discard_range(const void *p, size_t bytes)
{
    const uintptr_t a = reinterpret_cast<uintptr_t>(p);
    const uintptr_t first = (a + 127) & ~uintptr_t(127);
    const uintptr_t last = (a + bytes) & ~uintptr_t(127);
    for (uintptr_t q = first + (uintptr_t)threadIdx.x * 128; q + 128 <= last; q += (uintptr_t)blockDim.x * 128)
        asm volatile("discard.global.L2 [%0], 128;" ::"l"(q) : "memory");
}

struct Wave {
    const int32_t *tasks;      // packed (stage << 28) | chunk, in dependency-safe order
    const int32_t *lohi;       // chunk range read by each chunk's stencils
    uint32_t *done;            // completion stamp per chunk
    unsigned long long *ctr;   // [0] tickets, [1] finished chunks, [2] error word
    unsigned long long ticket_base;
    unsigned long long finish_base;
    uint32_t epoch;            // stamp before this launch
    int ntasks;
    int cb;                    // bricks per chunk
    int nchunks;
    uint32_t n_packed;
};

// grab the next task of this launch; -1 when none is left
__device__ __forceinline__ int next_task(const Wave &w)
{
    __shared__ int s_task;
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned long long t = atomicAdd(&w.ctr[0], 1ull) - w.ticket_base;
        s_task = t < (unsigned long long)w.ntasks ? w.tasks[t] : -1;
    }
    __syncthreads();
    return s_task;
}

__device__ __forceinline__ void wait_for(const Wave &w, int st, int c)
{
    if (st > 0 && threadIdx.x < 32)
        wait_chunks(w.done, w.lohi[2 * c], w.lohi[2 * c + 1], w.epoch + (uint32_t)st, &w.ctr[2]);
    __syncthreads();
}

__device__ __forceinline__ void publish(const Wave &w, int st, int c)
{
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) st_release(w.done + c, w.epoch + (uint32_t)st + 1u);
}

// ------------------------------------------------------------ warp-task wavefront (WAVE2)
// Each warp takes its own tasks (a stage of a chunk of cb bricks) in ticket
// order, one ticket ahead; a second-stage task waits until the first stage
// has finished on every chunk its stencils read (a per-chunk list), then
// publishes its own completion stamp.  No block-wide barrier is involved.
struct WaveW {
    const int32_t *tasks;      // packed (stage << 28) | chunk
    const int32_t *dep_off;    // [nchunks + 1]
    const int32_t *dep_ids;    // chunks read by each chunk's stencils (itself included)
    uint32_t *done;            // completion stamp per chunk
    unsigned long long *ctr;   // [0] tickets, [2] error word
    unsigned long long ticket_base;
    uint32_t epoch;
    int ntasks;
    int cb;
};

// one ticket for the calling warp (-1 past the last task)
__device__ __forceinline__ int grab_ticket(const WaveW &w)
{
    unsigned long long t = 0;
    if ((threadIdx.x & 31) == 0) t = atomicAdd(&w.ctr[0], 1ull) - w.ticket_base;
    t = __shfl_sync(0xffffffffu, t, 0);
    return t < (unsigned long long)w.ntasks ? (int)t : -1;
}

// Wait (all 32 lanes) until every chunk in c's list has stamp >= target; at
// most 64 entries.  Bounded like wait_chunks; once the error word is set,
// no further wait is started.
__device__ bool wait_deps(const WaveW &w, int c, uint32_t target)
{
    const int lane = threadIdx.x & 31;
    const int d0 = w.dep_off[c], n = w.dep_off[c + 1] - d0;
    const int i0 = lane < n ? w.dep_ids[d0 + lane] : -1;
    const int i1 = lane + 32 < n ? w.dep_ids[d0 + lane + 32] : -1;
    const volatile unsigned long long *err = &w.ctr[2];
    if (*err != 0ull) return false;
    const unsigned long long t0 = global_ns();
    for (long long it = 0; it < WAIT_ITERS; ++it) {
        const bool ok = (i0 < 0 || ld_acquire(w.done + i0) >= target) && (i1 < 0 || ld_acquire(w.done + i1) >= target);
        if (__all_sync(0xffffffffu, ok)) return true;
        if (global_ns() - t0 > WAIT_NS || *err != 0ull) break;
        __nanosleep(100);
    }
    if (lane == 0) atomicOr(&w.ctr[2], 1ull);
    return false;
}

// RK4 stages first and first + 1 (first = 0 or 2) of one step, warp tasks
template <typename R, int BX, int BY, int BZ, bool BLEND>
__global__ void GPE_BOUNDS(R) k_rk4_pair(const RkArgs<R> a, const GridView G, const WaveW w, int first)
{
    auto &ws = warp_space<R, BX, BY, BZ>();
    const int lane = threadIdx.x & 31;
    const R s0 = stage_s<R, BLEND>(a, first), s1 = stage_s<R, BLEND>(a, first + 1);
    int t = grab_ticket(w);
    while (t >= 0) {
        const int task = w.tasks[t];
        const int tn = grab_ticket(w);  // the next ticket, in flight during this task
        const int ls = task >> 28, c = task & 0x0fffffff, st = first + ls;
        if (ls == 1) {
            wait_deps(w, c, w.epoch + 1u);
            __syncwarp();
        }
        const int64_t b0 = (int64_t)c * w.cb;
        const int64_t b1 = b0 + w.cb < G.nb ? b0 + w.cb : G.nb;
        for (int64_t b = b0; b < b1; ++b) {
            const int64_t nx = b + 1 < b1 ? b + 1 : -1;
            switch (st) {
            case 0: rk4_brick<R, BX, BY, BZ, BLEND, true, 0>(a, G, b, nx, ws, s0); break;
            case 1: rk4_brick<R, BX, BY, BZ, BLEND, true, 1>(a, G, b, nx, ws, s1); break;
            case 2: rk4_brick<R, BX, BY, BZ, BLEND, true, 2>(a, G, b, nx, ws, s0); break;
            default: rk4_brick<R, BX, BY, BZ, BLEND, true, 3>(a, G, b, nx, ws, s1); break;
            }
        }
        // every lane's stores reach device scope before the warp publishes
        __threadfence();
        __syncwarp();
        if (lane == 0) st_release(w.done + c, w.epoch + (uint32_t)ls + 1u);
        t = tn;
    }
}

// RK4 stages first .. first + (tasks' stage count) - 1 of one step in one
// persistent launch: first = 0 with the 4-stage task list (WAVE), or 0 and
// then 2 with the 2-stage list (WAVE2).
template <typename R, int BX, int BY, int BZ, bool BLEND>
__global__ void GPE_BOUNDS(R) k_rk4_wave(const RkArgs<R> a, const GridView G, const Wave w, int first)
{
    using CT = typename Cx<R>::T;
    constexpr int NW = KernelCfg<R>::NW;
    auto &ws = warp_space<R, BX, BY, BZ>();
    const int warp = threadIdx.x >> 5;
    R s[4];
#pragma unroll
    for (int st = 0; st < 4; ++st) s[st] = stage_s<R, BLEND>(a, st);
    for (;;) {
        const int task = next_task(w);
        if (task < 0) break;
        const int ls = task >> 28, c = task & 0x0fffffff;  // stage within this launch
        const int st = first + ls;
        wait_for(w, ls, c);
        const int64_t b0 = (int64_t)c * w.cb;
        const int64_t b1 = b0 + w.cb < G.nb ? b0 + w.cb : G.nb;
        for (int64_t b = b0 + warp; b < b1; b += NW) {
            const int64_t nx = b + NW < b1 ? b + NW : -1;
            switch (st) {
            case 0: rk4_brick<R, BX, BY, BZ, BLEND, true, 0>(a, G, b, nx, ws, s[0]); break;
            case 1: rk4_brick<R, BX, BY, BZ, BLEND, true, 1>(a, G, b, nx, ws, s[1]); break;
            case 2: rk4_brick<R, BX, BY, BZ, BLEND, true, 2>(a, G, b, nx, ws, s[2]); break;
            default: rk4_brick<R, BX, BY, BZ, BLEND, true, 3>(a, G, b, nx, ws, s[3]); break;
            }
        }
        publish(w, ls, c);
        if (st == 3) {
            // y3 and w of this chunk have no reader left in this step (y4,
            // in y2's buffer, is still read by the neighbour chunks' stage 3)
            const uint32_t p0 = __ldg(&G.rec[b0].off);
            const uint32_t p1 = b1 < G.nb ? __ldg(&G.rec[b1].off) : w.n_packed;
            discard_range(a.y3 + p0, (size_t)(p1 - p0) * sizeof(CT));
            discard_range(a.w + p0, (size_t)(p1 - p0) * sizeof(CT));
        }
    }
}


template <typename R, int BX, int BY, int BZ>
__global__ void GPE_BOUNDS(R) k_itp_wave(const ItpArgs<R> a, const GridView G, const Wave w, double *chunk_norm)
{
    constexpr int NW = KernelCfg<R>::NW;
    auto &ws = warp_space<R, BX, BY, BZ>();
    __shared__ bool s_last;
    const int warp = threadIdx.x >> 5;
    const R sc = (R)a.scalars[0];
    for (;;) {
        const int task = next_task(w);
        if (task < 0) break;
        const int st = task >> 28, c = task & 0x0fffffff;
        wait_for(w, st, c);
        const int64_t b0 = (int64_t)c * w.cb;
        const int64_t b1 = b0 + w.cb < G.nb ? b0 + w.cb : G.nb;
        if (st == 0) {
            for (int64_t b = b0 + warp; b < b1; b += NW)
                itp_brick_a<R, typename Cx<R>::T, BX, BY, BZ, true>(a, G, b, b + NW < b1 ? b + NW : -1, ws, sc);
            publish(w, st, c);
            continue;
        }
        double acc = 0.0;
        for (int64_t b = b0 + warp; b < b1; b += NW)
            itp_brick_b<R, typename Cx<R>::T, BX, BY, BZ, true>(a, G, b, b + NW < b1 ? b + NW : -1, ws, acc);
        const double part = block_sum(acc);
        if (threadIdx.x == 0) chunk_norm[c] = part;
        publish(w, st, c);
        if (threadIdx.x == 0) {
            const unsigned long long k = atomicAdd(&w.ctr[1], 1ull) - w.finish_base;
            s_last = (k == (unsigned long long)w.nchunks - 1);
        }
        __syncthreads();
        if (s_last) {
            // every chunk has finished both stages: fold the chunk norms in
            // chunk order and store the next renormalisation factor
            __threadfence();
            double x = 0.0;
            for (int i = threadIdx.x; i < w.nchunks; i += blockDim.x) x += __ldcg(chunk_norm + i);
            x = block_sum(x);
            if (threadIdx.x == 0) {
                const double nrm = x * a.dV;
                a.scalars[0] = sqrt(a.N / nrm);
                a.scalars[1] = nrm;
            }
        }
    }
}



// <a|b> = sum conj(a) b dV over the packed arrays (inactive entries are zero)
template <typename CT>
__global__ void k_overlap(const CT *a, const CT *b, int64_t n, double dV, double *partials, unsigned int *counter,
                          double *out)
{
    double acc[2] = {0.0, 0.0};
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
        const CT u = a[s], v = b[s];
        acc[0] += (double)(u.x * v.x + u.y * v.y);
        acc[1] += (double)(u.x * v.y - u.y * v.x);
    }
    double tot[2];
    if (reduce_finish<2>(acc, partials, counter, tot) && threadIdx.x == 0) {
        out[0] = tot[0] * dV;
        out[1] = tot[1] * dV;
    }
}

// ------------------------------------------------------------ load / store
struct BoxI {
    int64_t nx, ny, nz;
    int BX, BY, BZ;
};

template <typename CT, bool STORE>
__global__ void k_dense_io(CT *psi, CT *dense, const int32_t *org, const uint32_t *mask, GridView G, int64_t ns,
                           BoxI bi)
{
    const int BC = bi.BX * bi.BY * bi.BZ;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < ns; s += (int64_t)gridDim.x * blockDim.x) {
        if (!((mask[s >> 5] >> (s & 31)) & 1u)) continue;
        const int64_t br = s / BC;
        const int l = (int)(s % BC);
        uint32_t idx;
        if (!seg_index(G.rec[br], l >> 2, idx)) continue;  // cannot happen for an active cell
        const int64_t i = org[3 * br] + l % bi.BX, j = org[3 * br + 1] + (l / bi.BX) % bi.BY,
                      k = org[3 * br + 2] + l / (bi.BX * bi.BY);
        const int64_t lin = i + bi.nx * (j + bi.ny * k);
        if (STORE) dense[lin] = psi[idx + (l & 3)];
        else psi[idx + (l & 3)] = dense[lin];
    }
}

// zero the inactive cells of stored segments (V0 = +inf there)
template <typename CT>
__global__ void k_zero_inactive(CT *psi, const double *V0, int64_t n)
{
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x)
        if (!(V0[s] < INFINITY)) psi[s] = czero<CT>();
}

// psi = src, zero on the inactive cells of stored segments, in one pass; src
// may be page-locked host memory read in place by the GPU (its device view)
template <typename CT>
__global__ void k_load_zero(CT *psi, const CT *src, const double *V0, int64_t n)
{
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x)
        psi[s] = V0[s] < INFINITY ? src[s] : czero<CT>();
}

// The device view of page-locked host memory (NULL for pageable memory).
// The driver is asked (cuPointerGetAttribute through its entry point): memory
// page-locked by another CUDA runtime in the process (a framework's pinned
// allocator) is known to the driver but not to this library's runtime.
typedef int (*ptr_attr_fn)(void *data, int attribute, unsigned long long ptr);
static const void *pinned_view(const void *p)
{
    static ptr_attr_fn fn = nullptr;
    static bool looked = false;
    if (!looked) {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuPointerGetAttribute", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<ptr_attr_fn>(f);
        cudaGetLastError();
        looked = true;
    }
    if (!fn) return nullptr;
    const unsigned long long a = (unsigned long long)(uintptr_t)p;
    unsigned int type = 0;
    unsigned long long dptr = 0;
    // attributes 2 (memory type; 1 = host) and 3 (device pointer)
    if (fn(&type, 2, a) != 0 || type != 1u || fn(&dptr, 3, a) != 0 || dptr == 0) return nullptr;
    return reinterpret_cast<const void *>((uintptr_t)dptr);
}

// ------------------------------------------------------------ state helpers
int ensure_work(gpe_state *st, int n)
{
    for (int i = 0; i < n; ++i) {
        if (st->d_work[i]) continue;
        GPE_TRY(dev_alloc(&st->d_work[i], st->grid->n_packed * st->elem));
        GPE_TRY(dev_zero(st->d_work[i], st->grid->n_packed * st->elem));
    }
    return GPE_OK;
}

const void *potential_ptr(gpe_state *st, int slot)
{
    gpe_grid *g = st->grid;
    if (!g->d_V[slot]) return nullptr;
    if (st->dtype == GPE_C128 || st->dtype == GPE_R64) return g->d_V[slot];
    if (ensure_vf(g, slot) != GPE_OK) return nullptr;
    return g->d_Vf[slot];
}

static int check_state(const gpe_state *st)
{
    if (!st) return fail(GPE_ERR_ARG, "state is NULL");
    int dev = -1;
    GPE_TRY_CUDA(cudaGetDevice(&dev));
    if (dev != st->grid->device)
        return fail(GPE_ERR_STATE, "state lives on device %d but device %d is current", st->grid->device, dev);
    return GPE_OK;
}

// ------------------------------------------------------------ wavefront schedule
// Chunk c = bricks [c*cb, (c+1)*cb).  lo/hi: the lowest and highest chunk that
// holds a face neighbour of one of c's bricks (c included).  Task order: with
// H(c) = max over c' <= c of hi(c'), tau(0, c) = c and
// tau(s, c) = tau(s-1, H(c)) + 1; tasks sorted by (tau, s, c).  Every
// dependency (s-1, c'), c' <= hi(c) <= H(c), then has a smaller tau, so it was
// handed out earlier and the holder of the smallest unfinished ticket never
// waits.
static int build_schedule(gpe_grid *g)
{
    if (g->d_tasks) return GPE_OK;
    // lag between a dependency's position and the task's: about one
    // launch's worth of resident blocks, so that a task's dependencies were
    // handed out a full wave of tasks earlier and have usually finished
    int64_t lag = (int64_t)g->nsm * 2;
    if (const char *e = getenv("GPE_WAVE_LAG")) lag = std::max<int64_t>(1, atoll(e));
    const int64_t nb = g->nb, cb = g->cb;
    const int64_t nch = (nb + cb - 1) / cb;
    if (nch >= (1 << 28)) return fail(GPE_ERR_ARG, "too many chunks for the wavefront schedule");
    std::vector<int32_t> nbr(nb * 6);
    GPE_TRY_CUDA(cudaMemcpy(nbr.data(), g->d_nbr, nb * 6 * sizeof(int32_t), cudaMemcpyDeviceToHost));
    std::vector<int32_t> lohi(nch * 2);
    for (int64_t c = 0; c < nch; ++c) {
        int64_t lo = c, hi = c;
        for (int64_t b = c * cb; b < std::min(nb, (c + 1) * cb); ++b)
            for (int d = 0; d < 6; ++d) {
                const int32_t n = nbr[b * 6 + d];
                if (n < 0) continue;
                lo = std::min<int64_t>(lo, n / cb);
                hi = std::max<int64_t>(hi, n / cb);
            }
        lohi[2 * c] = (int32_t)lo;
        lohi[2 * c + 1] = (int32_t)hi;
    }
    std::vector<int64_t> H(nch);
    int64_t run = 0;
    for (int64_t c = 0; c < nch; ++c) {
        run = std::max<int64_t>(run, lohi[2 * c + 1]);
        H[c] = run;
    }
    std::vector<int64_t> tau[4];
    tau[0].resize(nch);
    for (int64_t c = 0; c < nch; ++c) tau[0][c] = c;
    for (int s = 1; s < 4; ++s) {
        tau[s].resize(nch);
        for (int64_t c = 0; c < nch; ++c) tau[s][c] = tau[s - 1][H[c]] + lag;
    }
    std::vector<int32_t> tasks;
    tasks.reserve(6 * nch);
    for (int S : {2, 4}) {
        std::vector<std::pair<std::pair<int64_t, int>, int64_t>> v;
        v.reserve(S * nch);
        for (int s = 0; s < S; ++s)
            for (int64_t c = 0; c < nch; ++c) v.push_back({{tau[s][c], s}, c});
        std::sort(v.begin(), v.end());
        for (auto &e : v) tasks.push_back((int32_t)((e.first.second << 28) | e.second));
    }
    int32_t *d_lohi = nullptr, *d_tasks = nullptr;
    GPE_TRY(dev_alloc_t(&d_lohi, nch * 2));
    int rc = dev_alloc_t(&d_tasks, tasks.size());
    if (rc != GPE_OK) {
        dev_free(d_lohi);
        return rc;
    }
    if (cudaMemcpy(d_lohi, lohi.data(), lohi.size() * sizeof(int32_t), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(d_tasks, tasks.data(), tasks.size() * sizeof(int32_t), cudaMemcpyHostToDevice) != cudaSuccess) {
        dev_free(d_lohi);
        dev_free(d_tasks);
        return fail(GPE_ERR_CUDA, "schedule upload failed");
    }
    g->n_chunks = nch;
    g->d_chunk_lohi = d_lohi;
    g->d_tasks = d_tasks;
    return GPE_OK;
}

static int ensure_wave(gpe_state *st)
{
    gpe_grid *g = st->grid;
    GPE_TRY(build_schedule(g));
    if (!st->d_done) {
        GPE_TRY(dev_alloc_t(&st->d_done, g->n_chunks));
        GPE_TRY(dev_zero(st->d_done, g->n_chunks * sizeof(uint32_t)));
        GPE_TRY(dev_alloc_t(&st->d_ctr, 4));
        GPE_TRY(dev_zero(st->d_ctr, 4 * sizeof(unsigned long long)));
        GPE_TRY(dev_alloc_t(&st->d_chunk_norm, g->n_chunks));
        st->epoch = 0;
        st->ticket_base = 0;
        st->finish_base = 0;
    }
    return GPE_OK;
}

// Warp-task schedule of the two-stage RK4 launches: per chunk the sorted set
// of chunks holding its bricks' face neighbours (and itself), H(c) the running
// maximum of those sets, tau(0, c) = c and tau(1, c) = H(c) + lag; tasks
// sorted by (tau, stage, chunk).  A second-stage task's dependencies then
// hold earlier tickets, so the holder of the smallest unfinished ticket never
// waits.  lag: about half the resident warps, the number of first-stage
// tasks in flight.
static int build_schedule_w(gpe_grid *g, int64_t lag)
{
    if (g->d_tasks_w) return GPE_OK;
    if (const char *e = getenv("GPE_WAVE_LAG")) lag = std::max<int64_t>(1, atoll(e));
    const int64_t nb = g->nb, cb = g->cb;
    const int64_t nch = (nb + cb - 1) / cb;
    if (nch >= (1 << 28)) return fail(GPE_ERR_ARG, "too many chunks for the wavefront schedule");
    std::vector<int32_t> nbr(nb * 6);
    GPE_TRY_CUDA(cudaMemcpy(nbr.data(), g->d_nbr, nb * 6 * sizeof(int32_t), cudaMemcpyDeviceToHost));
    std::vector<int32_t> off(nch + 1, 0), ids;
    std::vector<int64_t> H(nch);
    int64_t run = 0;
    for (int64_t c = 0; c < nch; ++c) {
        std::vector<int32_t> d{(int32_t)c};
        for (int64_t b = c * cb; b < std::min(nb, (c + 1) * cb); ++b)
            for (int k = 0; k < 6; ++k)
                if (nbr[b * 6 + k] >= 0) d.push_back((int32_t)(nbr[b * 6 + k] / cb));
        std::sort(d.begin(), d.end());
        d.erase(std::unique(d.begin(), d.end()), d.end());
        if (d.size() > 64) return fail(GPE_ERR_ARG, "chunk too large for the two-stage wavefront (at most 64 neighbour chunks)");
        ids.insert(ids.end(), d.begin(), d.end());
        off[c + 1] = (int32_t)ids.size();
        run = std::max<int64_t>(run, d.back());
        H[c] = run;
    }
    std::vector<std::pair<std::pair<int64_t, int>, int64_t>> v;
    v.reserve(2 * nch);
    for (int64_t c = 0; c < nch; ++c) {
        v.push_back({{c, 0}, c});
        v.push_back({{H[c] + lag, 1}, c});
    }
    std::sort(v.begin(), v.end());
    std::vector<int32_t> tasks;
    tasks.reserve(2 * nch);
    for (auto &e : v) tasks.push_back((int32_t)((e.first.second << 28) | e.second));
    int rc = dev_alloc_t(&g->d_dep_off, nch + 1);
    if (rc == GPE_OK) rc = dev_alloc_t(&g->d_dep_ids, ids.size());
    if (rc == GPE_OK) rc = dev_alloc_t(&g->d_tasks_w, tasks.size());
    if (rc == GPE_OK &&
        (cudaMemcpy(g->d_dep_off, off.data(), off.size() * sizeof(int32_t), cudaMemcpyHostToDevice) != cudaSuccess ||
         cudaMemcpy(g->d_dep_ids, ids.data(), ids.size() * sizeof(int32_t), cudaMemcpyHostToDevice) != cudaSuccess ||
         cudaMemcpy(g->d_tasks_w, tasks.data(), tasks.size() * sizeof(int32_t), cudaMemcpyHostToDevice) != cudaSuccess))
        rc = fail(GPE_ERR_CUDA, "schedule upload failed");
    if (rc != GPE_OK) {
        dev_free(g->d_dep_off);
        dev_free(g->d_dep_ids);
        dev_free(g->d_tasks_w);
        g->d_dep_off = g->d_dep_ids = g->d_tasks_w = nullptr;
    }
    return rc;
}

static WaveW make_wave_w(gpe_state *st)
{
    const gpe_grid *g = st->grid;
    WaveW w;
    w.tasks = g->d_tasks_w;
    w.dep_off = g->d_dep_off;
    w.dep_ids = g->d_dep_ids;
    w.done = st->d_done;
    w.ctr = st->d_ctr;
    w.ticket_base = st->ticket_base;
    w.epoch = st->epoch;
    w.ntasks = (int)(2 * g->n_chunks);
    w.cb = g->cb;
    return w;
}

static Wave make_wave(gpe_state *st, int stages)
{
    const gpe_grid *g = st->grid;
    Wave w;
    w.tasks = g->d_tasks + (stages == 2 ? 0 : 2 * g->n_chunks);
    w.lohi = g->d_chunk_lohi;
    w.done = st->d_done;
    w.ctr = st->d_ctr;
    w.ticket_base = st->ticket_base;
    w.finish_base = st->finish_base;
    w.epoch = st->epoch;
    w.ntasks = (int)(stages * g->n_chunks);
    w.cb = g->cb;
    w.nchunks = (int)g->n_chunks;
    w.n_packed = (uint32_t)g->n_packed;
    return w;
}

// after a wave launch with `grid` blocks: every block took one ticket past
// the end, so the counter advanced by ntasks + grid
static void advance_wave(gpe_state *st, int stages, int grid_blocks, bool itp)
{
    st->ticket_base += (unsigned long long)stages * st->grid->n_chunks + (unsigned long long)grid_blocks;
    if (itp) st->finish_base += (unsigned long long)st->grid->n_chunks;
    st->epoch += (uint32_t)stages;
}

// ------------------------------------------------------------ CUDA graphs
static uint64_t fnv1a(const void *p, size_t n, uint64_t h = 1469598103934665603ull)
{
    const unsigned char *c = static_cast<const unsigned char *>(p);
    for (size_t i = 0; i < n; ++i) h = (h ^ c[i]) * 1099511628211ull;
    return h;
}

// Graphs replay on the caller's stream; the legacy default stream cannot be
// captured, so steps issued there run eagerly.
static bool use_graph(const gpe_state *st, cudaStream_t s, int64_t nsteps)
{
    return st->graph_steps > 0 && nsteps >= st->graph_steps && s != nullptr && s != cudaStreamLegacy &&
           s != cudaStreamPerThread;
}

// Replay graph `which` (capturing it first if its key changed) `reps` times.
template <typename F>
static int replay_graph(gpe_state *st, int which, uint64_t key, int nodes, int64_t reps, cudaStream_t s, F record)
{
    if (!st->gexec[which] || st->gkey[which] != key) {
        if (st->gexec[which]) {
            cudaGraphExecDestroy(st->gexec[which]);
            st->gexec[which] = nullptr;
        }
        if (!st->gcap) GPE_TRY_CUDA(cudaStreamCreateWithFlags(&st->gcap, cudaStreamNonBlocking));
        GPE_TRY_CUDA(cudaStreamBeginCapture(st->gcap, cudaStreamCaptureModeThreadLocal));
        const int rc = record(st->gcap);
        cudaGraph_t graph = nullptr;
        const cudaError_t e = cudaStreamEndCapture(st->gcap, &graph);
        if (rc != GPE_OK) {
            if (graph) cudaGraphDestroy(graph);
            return rc;
        }
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture", __FILE__, __LINE__);
        const cudaError_t e2 = cudaGraphInstantiate(&st->gexec[which], graph, 0);
        cudaGraphDestroy(graph);
        if (e2 != cudaSuccess) return cuda_fail(e2, "cudaGraphInstantiate", __FILE__, __LINE__);
        st->gkey[which] = key;
        st->gnodes[which] = nodes;
    }
    for (int64_t r = 0; r < reps; ++r) {
        GPE_TRY_CUDA(cudaGraphLaunch(st->gexec[which], s));
        for (int k = 0; k < nodes; ++k) count_launch();
    }
    return GPE_OK;
}

__global__ void k_add_scalar(double *p, double v) { *p += v; }

// ------------------------------------------------------------ neighbour ids (PAIR schedule)
// nbr18[18 b + k]: the face neighbours (-x +x -y +y -z +z) and the 12 edge
// neighbours (xy (-1,-1,0) (+1,-1,0) (-1,+1,0) (+1,+1,0); xz (-1,0,-1)
// (+1,0,-1) (-1,0,+1) (+1,0,+1); yz (0,-1,-1) (0,+1,-1) (0,-1,+1) (0,+1,+1))
// of brick b, -1 if absent
__global__ void k_nbr18(int64_t nb, const int32_t *org, int bx, int by, int bz, int64_t nbx, int64_t nby, int64_t nbz,
                        const int32_t *bvol, const int32_t *nbr6, int32_t *out)
{
    const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (id >= nb) return;
    const int8_t d[12][3] = {{-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}, {1, 1, 0}, {-1, 0, -1}, {1, 0, -1},
                             {-1, 0, 1},  {1, 0, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}, {0, 1, 1}};
    for (int k = 0; k < 6; ++k) out[18 * id + k] = nbr6[6 * id + k];
    const int64_t cx = org[3 * id] / bx, cy = org[3 * id + 1] / by, cz = org[3 * id + 2] / bz;
    for (int e = 0; e < 12; ++e) {
        const int64_t x = cx + d[e][0], y = cy + d[e][1], z = cz + d[e][2];
        int32_t r = -1;
        if (x >= 0 && x < nbx && y >= 0 && y < nby && z >= 0 && z < nbz) r = bvol[x + nbx * (y + nby * z)];
        out[18 * id + 6 + e] = r;
    }
}

static int ensure_nbr18(gpe_grid *g)
{
    if (g->d_nbr18) return GPE_OK;
    int32_t *t = nullptr;
    GPE_TRY(dev_alloc_t(&t, (size_t)std::max<int64_t>(1, 18 * g->nb)));
    if (g->nb > 0) {
        k_nbr18<<<(unsigned)((g->nb + 255) / 256), 256, 0, cudaStreamLegacy>>>(
            g->nb, g->d_org, g->bx, g->by, g->bz, g->nbx, g->nby, g->nbz, g->d_bvol, g->d_nbr, t);
        count_launch();
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(cudaStreamLegacy);
        if (e != cudaSuccess) {
            dev_free(t);
            return cuda_fail(e, "k_nbr18", __FILE__, __LINE__);
        }
    }
    g->d_nbr18 = t;
    return GPE_OK;
}

// ------------------------------------------------------------ step drivers
template <typename R, int BX, int BY, int BZ>
static int rk4_run(gpe_state *st, const gpe_real_params *p, int64_t nsteps, double t0, cudaStream_t s)
{
    using CT = typename Cx<R>::T;
    const gpe_grid *g = st->grid;
    const bool blend = p->potential == GPE_V_BLEND;
    RkArgs<R> a{};
    a.V0 = (const R *)potential_ptr(st, 0);
    a.V1 = blend ? (const R *)potential_ptr(st, 1) : nullptr;
    if (!a.V0 || (blend && !a.V1)) return fail(GPE_ERR_STATE, "potential slot missing");
    a.y0 = (CT *)st->d_psi;
    a.y2 = (CT *)st->d_work[0];
    a.y3 = (CT *)st->d_work[1];
    a.y4 = (CT *)st->d_work[0];  // y2 is dead once stage 1 is done
    a.w = (CT *)st->d_work[2];
    a.ihx2 = (R)(1.0 / (g->box.hx * g->box.hx));
    a.ihy2 = (R)(1.0 / (g->box.hy * g->box.hy));
    a.ihz2 = (R)(1.0 / (g->box.hz * g->box.hz));
    a.g = (R)p->g;
    a.dt = (R)p->dt;
    a.dtd = p->dt;
    a.ramp.clock = st->d_clock;
    a.ramp.T = p->T_ramp;
    a.ramp.n_knots = p->n_knots;
    for (int k = 0; k < GPE_MAX_KNOTS; ++k) a.ramp.knots[k] = p->knots[k];
    if (blend) {
        k_set_scalar<<<1, 1, 0, s>>>(st->d_clock, t0);
        GPE_LAUNCH_CHECK();
    }
    const GridView G = view(g);
    const int th = KernelCfg<R>::THREADS;
    const size_t smem = smem_bytes<R, BX, BY, BZ>();
    if (g->sched == GPE_SCHED_WAVE) {
        GPE_TRY(ensure_wave(st));
        auto k = blend ? k_rk4_wave<R, BX, BY, BZ, true> : k_rk4_wave<R, BX, BY, BZ, false>;
        const int nblk = (int)std::min<int64_t>((int64_t)g->nsm * per_sm_for(k, th, smem), 4 * g->n_chunks);
        for (int64_t n = 0; n < nsteps; ++n) {
            a.t_off = (double)n * p->dt;
            k<<<nblk, th, smem, s>>>(a, G, make_wave(st, 4), 0);
            GPE_LAUNCH_CHECK();
            advance_wave(st, 4, nblk, false);
        }
        return GPE_OK;
    }
    if (g->sched == GPE_SCHED_WAVE2) {
        GPE_TRY(ensure_wave(st));
        auto k = blend ? k_rk4_pair<R, BX, BY, BZ, true> : k_rk4_pair<R, BX, BY, BZ, false>;
        const int nblk = g->nsm * per_sm_for(k, th, smem);
        const int nwarps = nblk * KernelCfg<R>::NW;
        GPE_TRY(build_schedule_w(st->grid, std::max(1, nwarps / 2)));
        for (int64_t n = 0; n < nsteps; ++n) {
            a.t_off = (double)n * p->dt;
            for (int first = 0; first < 4; first += 2) {
                k<<<nblk, th, smem, s>>>(a, G, make_wave_w(st), first);
                GPE_LAUNCH_CHECK();
                // every warp took one ticket past the last task
                st->ticket_base += 2ull * (unsigned long long)g->n_chunks + (unsigned long long)nwarps;
                st->epoch += 2u;
            }
        }
        return GPE_OK;
    }
    if (g->sched == GPE_SCHED_PAIR) {
        // two launches per step (stages 0+1, 2+3); the state alternates between
        // the psi buffer and work buffer 0 (unused by this schedule otherwise)
        GPE_TRY(ensure_nbr18(const_cast<gpe_grid *>(g)));
        const PairView P{g->d_rec, g->d_nbr18, g->nb};
        using RP = Rk4Fused<R, BX, BY, BZ>;
        typename RP::K kp[2] = {RP::get(blend, 0), RP::get(blend, 1)};
        const size_t psm = pair_smem<R, BX, BY, BZ>();
        int nbp[2];
        for (int i = 0; i < 2; ++i)
            nbp[i] = (int)std::max<int64_t>(
                1, std::min<int64_t>(g->nb, (int64_t)g->nsm * per_sm_for(kp[i], PAIR_THREADS, psm)));
        CT *bufA = (CT *)st->d_psi, *bufB = (CT *)st->d_work[0];
        // cnt steps from bufA; after an odd count psi is copied back to bufA
        auto record = [&](cudaStream_t cs, int64_t cnt) -> int {
            for (int64_t n = 0; n < cnt; ++n) {
                RkArgs<R> an = a;
                an.t_off = (double)n * p->dt;
                an.y0 = (n % 2 == 0) ? bufA : bufB;
                CT *out = (n % 2 == 0) ? bufB : bufA;
                for (int pass = 0; pass < 2; ++pass) {
                    kp[pass]<<<nbp[pass], PAIR_THREADS, psm, cs>>>(an, P, out);
                    GPE_LAUNCH_CHECK();
                }
            }
            if (cnt % 2)
                GPE_TRY_CUDA(cudaMemcpyAsync(bufA, bufB, (size_t)g->n_packed * sizeof(CT), cudaMemcpyDeviceToDevice, cs));
            return GPE_OK;
        };
        int64_t left = nsteps;
        if (use_graph(st, s, nsteps)) {
            const int G_ = st->graph_steps;
            uint64_t key = fnv1a(p, sizeof *p);
            const void *ptrs[2] = {a.V0, a.V1};
            key = fnv1a(ptrs, sizeof ptrs, key);
            key = fnv1a(&G_, sizeof G_, key);
            auto rec_block = [&](cudaStream_t cs) -> int {
                GPE_TRY(record(cs, G_));
                if (blend) {
                    k_add_scalar<<<1, 1, 0, cs>>>(st->d_clock, (double)G_ * p->dt);
                    GPE_LAUNCH_CHECK();
                }
                return GPE_OK;
            };
            GPE_TRY(replay_graph(st, 0, key, 2 * G_ + (blend ? 1 : 0), nsteps / G_, s, rec_block));
            left = nsteps % G_;
        }
        return record(s, left);
    }
    using RS = Rk4Stages<R, BX, BY, BZ>;
    typename RS::K k[4];
    int nblk[4];
    for (int stg = 0; stg < 4; ++stg) {
        k[stg] = RS::get(blend, stg);
        nblk[stg] = blocks_for_nw(k[stg], g, RS::smem(), RS::NW);
    }
    // steps n0 .. n0+cnt-1 with stage times relative to the device clock
    auto record = [&](cudaStream_t cs, int64_t cnt) -> int {
        for (int64_t n = 0; n < cnt; ++n) {
            a.t_off = (double)n * p->dt;
            for (int stg = 0; stg < 4; ++stg) {
                // stage 0 follows the scalar kernels of a ramp (no programmatic edge)
                const bool pdl = st->pdl && !(blend && n == 0 && stg == 0);
                GPE_TRY_CUDA(launch_stage(k[stg], (unsigned)nblk[stg], RS::THREADS, RS::smem(), cs, pdl, a, G));
                GPE_LAUNCH_CHECK();
            }
        }
        return GPE_OK;
    };
    int64_t left = nsteps;
    if (use_graph(st, s, nsteps)) {
        const int G_ = st->graph_steps;
        uint64_t key = fnv1a(p, sizeof *p);
        const void *ptrs[2] = {a.V0, a.V1};
        key = fnv1a(ptrs, sizeof ptrs, key);
        key = fnv1a(&G_, sizeof G_, key);
        auto rec_block = [&](cudaStream_t cs) -> int {
            GPE_TRY(record(cs, G_));
            if (blend) {
                k_add_scalar<<<1, 1, 0, cs>>>(st->d_clock, (double)G_ * p->dt);
                GPE_LAUNCH_CHECK();
            }
            return GPE_OK;
        };
        GPE_TRY(replay_graph(st, 0, key, 4 * G_ + (blend ? 1 : 0), nsteps / G_, s, rec_block));
        left = nsteps % G_;
    }
    return record(s, left);
}

// ------------------------------------------------------------ general explicit RK (RKHE3, RKCK)
// Memory-optimised form of App. A, Eqs. (A6)-(A7): with y^(1) = y0,
//   y^(i+1) = sum_{j<=i} a*_ij y^(j) + dt a_{i+1,i} f(t + c_i dt, y^(i)),
//   y1      = sum_{j<=s} b*_j  y^(j) + dt b_s     f(t + c_s dt, y^(s)).
// Stage i reads y^(i) with its halo and the own cells of the earlier states
// whose coefficient is not zero.
struct RkTable {
    int s;                 // stages
    double c[6];           // stage times
    double sub[6];         // a_{i+1,i} (i < s), then b_s
    double a_star[5][5];   // rows for y^(2) .. y^(s) (App. A printed tables)
    double b_star[6];
    double ylim;           // dt * lambda_max accepted by gpe_step_real
};

// Heun's third-order method (RKHE3): App. A, a* = [[1],[1, 0]],
// b* = (1/4, 3/4, 0); a_21 = 1/3, a_32 = 2/3, b_3 = 3/4; c = (0, 1/3, 2/3).
// |R(iy)| <= 1 up to y = sqrt(3).
static const RkTable RK_HE3 = {3,
                               {0.0, 1.0 / 3.0, 2.0 / 3.0},
                               {1.0 / 3.0, 2.0 / 3.0, 3.0 / 4.0},
                               {{1.0}, {1.0, 0.0}},
                               {1.0 / 4.0, 3.0 / 4.0, 0.0},
                               1.7320508075688772};
// Cash-Karp, fifth-order solution (RKCK): App. A's a* rows and b*; the
// tableau's sub-diagonal a_21 = 1/5, a_32 = 9/40, a_43 = 6/5, a_54 = 35/27,
// a_65 = 253/4096, b_6 = 512/1771; c = (0, 1/5, 3/10, 3/5, 1, 7/8).  Its
// stability function exceeds 1 on the whole imaginary axis, |R(iy)| ~ 1 +
// 1.39e-4 y^6; steps are accepted while that growth stays below 1e-6 per
// step (y <= 0.43).
static const RkTable RK_CK = {6,
                              {0.0, 1.0 / 5.0, 3.0 / 10.0, 3.0 / 5.0, 1.0, 7.0 / 8.0},
                              {1.0 / 5.0, 9.0 / 40.0, 6.0 / 5.0, 35.0 / 27.0, 253.0 / 4096.0, 512.0 / 1771.0},
                              {{1.0},
                               {5.0 / 8.0, 3.0 / 8.0},
                               {2.0, 3.0, -4.0},
                               {-49.0 / 81.0, 35.0 / 27.0, 200.0 / 81.0, -175.0 / 81.0},
                               {253.0 / 12288.0, -3795.0 / 4096.0, 1375.0 / 1536.0, 2875.0 / 4096.0, 1265.0 / 4096.0}},
                              {-991.0 / 15939.0, -3865.0 / 5313.0, 5000.0 / 5313.0, 3125.0 / 4554.0, 25.0 / 154.0, 0.0},
                              0.43};

static const RkTable *rk_table(int integrator)
{
    return integrator == GPE_RKHE3 ? &RK_HE3 : integrator == GPE_RKCK ? &RK_CK : nullptr;
}
double rk_stability_limit(int integrator)
{
    const RkTable *t = rk_table(integrator);
    return t ? t->ylim : 2.0 * std::sqrt(2.0);
}

template <typename R>
struct RkGenArgs {
    using CT = typename Cx<R>::T;
    CT *y[6];        // y^(1) = psi, y^(2..6) = work buffers
    const R *V0;
    const R *V1;
    R ihx2, ihy2, ihz2, g;
    Ramp ramp;
    double t_off;    // step start relative to *ramp.clock
    double tc;       // c_i dt
    int tile, out;   // y^(i) and the state written (y^(i+1), or y^(1) for y1)
    int nsrc;        // own-cell terms
    int src[5];
    R coef[5];
    R ctile;         // coefficient of y^(i) itself
    R kdt;           // dt a_{i+1,i} (dt b_s in the last stage)
};

template <typename R, int BX, int BY, int BZ, bool BLEND>
__global__ void GPE_BOUNDS(R) k_rk_stage(const RkGenArgs<R> a, const GridView G)
{
    using CT = typename Cx<R>::T;
    constexpr int NW = KernelCfg<R>::NW;
    auto &ws = warp_space<R, BX, BY, BZ>();
    const int warp = threadIdx.x >> 5;
    const R s = BLEND ? (R)ramp_s(a.ramp, *a.ramp.clock + a.t_off + a.tc) : (R)0;
    const int64_t stride = (int64_t)gridDim.x * NW;
    for (int64_t b = (int64_t)blockIdx.x * NW + warp; b < G.nb; b += stride) {
        brick_apply<BX, BY, BZ, false>(ws, G, b, b + stride < G.nb ? b + stride : -1, a.y[a.tile], Identity(), a.ihx2,
                                       a.ihy2, a.ihz2, [&](uint32_t idx, const CT(&c)[4], const CT(&L)[4]) {
            R V0[4], V1[4];
            ldr4(a.V0 + idx, V0);
            if (BLEND) ldr4(a.V1 + idx, V1);
            CT acc[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                acc[i].x = a.ctile * c[i].x;
                acc[i].y = a.ctile * c[i].y;
            }
            for (int j = 0; j < a.nsrc; ++j) {
                CT yj[4];
                ld4<false>(a.y[a.src[j]] + idx, yj);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    acc[i].x += a.coef[j] * yj[i].x;
                    acc[i].y += a.coef[j] * yj[i].y;
                }
            }
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
                o[i].x = acc[i].x + a.kdt * hi;
                o[i].y = acc[i].y - a.kdt * hr;
            }
            st4(a.y[a.out] + idx, o);
        });
    }
}

template <typename R, int BX, int BY, int BZ>
static int rkgen_run(gpe_state *st, const gpe_real_params *p, int64_t nsteps, double t0, cudaStream_t s)
{
    using CT = typename Cx<R>::T;
    const gpe_grid *g = st->grid;
    const RkTable &T = *rk_table(p->integrator);
    const bool blend = p->potential == GPE_V_BLEND;
    RkGenArgs<R> a{};
    a.y[0] = (CT *)st->d_psi;
    for (int i = 1; i < 6; ++i) a.y[i] = (CT *)st->d_work[i - 1];
    a.V0 = (const R *)potential_ptr(st, 0);
    a.V1 = blend ? (const R *)potential_ptr(st, 1) : nullptr;
    if (!a.V0 || (blend && !a.V1)) return fail(GPE_ERR_STATE, "potential slot missing");
    a.ihx2 = (R)(1.0 / (g->box.hx * g->box.hx));
    a.ihy2 = (R)(1.0 / (g->box.hy * g->box.hy));
    a.ihz2 = (R)(1.0 / (g->box.hz * g->box.hz));
    a.g = (R)p->g;
    a.ramp.clock = st->d_clock;
    a.ramp.T = p->T_ramp;
    a.ramp.n_knots = p->n_knots;
    for (int k = 0; k < GPE_MAX_KNOTS; ++k) a.ramp.knots[k] = p->knots[k];
    if (blend) {
        k_set_scalar<<<1, 1, 0, s>>>(st->d_clock, t0);
        GPE_LAUNCH_CHECK();
    }
    auto k = blend ? k_rk_stage<R, BX, BY, BZ, true> : k_rk_stage<R, BX, BY, BZ, false>;
    const size_t smem = smem_bytes<R, BX, BY, BZ>();
    const int nblk = blocks_for<R>(k, g, smem);
    for (int64_t n = 0; n < nsteps; ++n) {
        a.t_off = (double)n * p->dt;
        for (int i = 0; i < T.s; ++i) {  // stage i + 1 of App. A
            const bool last = i == T.s - 1;
            const double *row = last ? T.b_star : T.a_star[i];
            a.tile = i;
            a.out = last ? 0 : i + 1;
            a.tc = T.c[i] * p->dt;
            a.kdt = (R)(T.sub[i] * p->dt);
            a.ctile = (R)row[i];
            a.nsrc = 0;
            for (int j = 0; j < i; ++j)
                if (row[j] != 0.0) {
                    a.src[a.nsrc] = j;
                    a.coef[a.nsrc] = (R)row[j];
                    ++a.nsrc;
                }
            k<<<nblk, KernelCfg<R>::THREADS, smem, s>>>(a, view(g));
            GPE_LAUNCH_CHECK();
        }
    }
    return GPE_OK;
}

template <typename R, int BX, int BY, int BZ, typename CT = typename Cx<R>::T>
static int itp_run(gpe_state *st, const gpe_imag_params *p, int64_t nsteps, cudaStream_t s)
{
    const gpe_grid *g = st->grid;
    if (st->E_dt != p->dt) {
        k_make_E<R><<<g->nsm * 8, 256, 0, s>>>(g->d_V[0], (R *)st->d_E, g->n_packed, p->dt);
        GPE_LAUNCH_CHECK();
        st->E_dt = p->dt;
    }
    ItpArgs<R, CT> a{};
    a.psi = (CT *)st->d_psi;
    a.tmp = (CT *)st->d_work[0];
    a.E = (const R *)st->d_E;
    a.ihx2 = (R)(1.0 / (g->box.hx * g->box.hx));
    a.ihy2 = (R)(1.0 / (g->box.hy * g->box.hy));
    a.ihz2 = (R)(1.0 / (g->box.hz * g->box.hz));
    a.g = (R)p->g;
    a.dt = (R)p->dt;
    a.scalars = st->red.scalars;
    a.N = p->N;
    a.dV = g->box.hx * g->box.hy * g->box.hz;
    k_set_scalar<<<1, 1, 0, s>>>(st->red.scalars, 1.0);
    GPE_LAUNCH_CHECK();
    const GridView G = view(g);
    const int th = KernelCfg<R>::THREADS;
    const size_t smem = smem_bytes<R, BX, BY, BZ, CT>();
    // real-valued states run the staged schedule whatever the grid's
    if constexpr (is_cplx<CT>()) if (g->sched == GPE_SCHED_WAVE || g->sched == GPE_SCHED_WAVE2) {
        GPE_TRY(ensure_wave(st));
        auto k = k_itp_wave<R, BX, BY, BZ>;
        const int nblk = (int)std::min<int64_t>((int64_t)g->nsm * per_sm_for(k, th, smem), 2 * g->n_chunks);
        for (int64_t n = 0; n < nsteps; ++n) {
            k<<<nblk, th, smem, s>>>(a, G, make_wave(st, 2), st->d_chunk_norm);
            GPE_LAUNCH_CHECK();
            advance_wave(st, 2, nblk, true);
        }
        k_apply_scale<CT><<<g->nsm * 8, 256, 0, s>>>((CT *)st->d_psi, g->n_packed, st->red.scalars);
        GPE_LAUNCH_CHECK();
        return GPE_OK;
    }
    if constexpr (is_cplx<CT>()) if (g->sched == GPE_SCHED_PAIR) {
        // one pass per step; the state alternates between the psi buffer and
        // work buffer 0
        GPE_TRY(ensure_nbr18(const_cast<gpe_grid *>(g)));
        const PairView P{g->d_rec, g->d_nbr18, g->nb};
        auto k = k_itp_fused<R, BX, BY, BZ>;
        const size_t psm = sizeof(ItpPairSpace<CT, BX, BY, BZ>);
        const int64_t res = (int64_t)g->nsm * per_sm_for(k, PAIR_THREADS, psm);
        const int nbk = (int)std::max<int64_t>(1, std::min<int64_t>(std::min<int64_t>(g->nb, res), st->red.max_blocks));
        CT *bufA = (CT *)st->d_psi, *bufB = (CT *)st->d_work[0];
        // cnt steps from bufA; after an odd count psi is copied back to bufA
        auto record = [&](cudaStream_t cs, int64_t cnt) -> int {
            for (int64_t n = 0; n < cnt; ++n) {
                ItpArgs<R, CT> an = a;
                an.psi = (n % 2 == 0) ? bufA : bufB;
                an.tmp = (n % 2 == 0) ? bufB : bufA;
                k<<<nbk, PAIR_THREADS, psm, cs>>>(an, P, st->red.partials, st->red.counter);
                GPE_LAUNCH_CHECK();
            }
            if (cnt % 2)
                GPE_TRY_CUDA(cudaMemcpyAsync(bufA, bufB, (size_t)g->n_packed * sizeof(CT), cudaMemcpyDeviceToDevice, cs));
            return GPE_OK;
        };
        int64_t left = nsteps;
        if (use_graph(st, s, nsteps)) {
            const int G_ = st->graph_steps;
            uint64_t key = fnv1a(p, sizeof *p);
            key = fnv1a(&G_, sizeof G_, key);
            key = fnv1a(&a.E, sizeof a.E, key);
            GPE_TRY(replay_graph(st, 1, key, G_, nsteps / G_, s, [&](cudaStream_t cs) { return record(cs, G_); }));
            left = nsteps % G_;
        }
        GPE_TRY(record(s, left));
        k_apply_scale<CT><<<g->nsm * 8, 256, 0, s>>>((CT *)st->d_psi, g->n_packed, st->red.scalars);
        GPE_LAUNCH_CHECK();
        return GPE_OK;
    }
    {
        auto ka = k_itp_a<R, BX, BY, BZ, CT>;
        auto kb = k_itp_b<R, BX, BY, BZ, CT>;
        const int nba = blocks_for<R>(ka, g, smem), nbb = blocks_for<R>(kb, g, smem);
        auto record = [&](cudaStream_t cs, int64_t cnt) -> int {
            for (int64_t n = 0; n < cnt; ++n) {
                GPE_TRY_CUDA(launch_stage(ka, (unsigned)nba, th, smem, cs, st->pdl && n > 0, a, G));
                GPE_LAUNCH_CHECK();
                GPE_TRY_CUDA(launch_stage(kb, (unsigned)nbb, th, smem, cs, st->pdl, a, G, st->red.partials,
                                          st->red.counter));
                GPE_LAUNCH_CHECK();
            }
            return GPE_OK;
        };
        int64_t left = nsteps;
        if (use_graph(st, s, nsteps)) {
            const int G_ = st->graph_steps;
            uint64_t key = fnv1a(p, sizeof *p);
            key = fnv1a(&G_, sizeof G_, key);
            key = fnv1a(&a.E, sizeof a.E, key);
            GPE_TRY(replay_graph(st, 1, key, 2 * G_, nsteps / G_, s, [&](cudaStream_t cs) { return record(cs, G_); }));
            left = nsteps % G_;
        }
        GPE_TRY(record(s, left));
    }
    k_apply_scale<CT><<<g->nsm * 8, 256, 0, s>>>((CT *)st->d_psi, g->n_packed, st->red.scalars);
    GPE_LAUNCH_CHECK();
    return GPE_OK;
}

template <typename R, int BX, int BY, int BZ, typename CT = typename Cx<R>::T>
static int obs_run(const gpe_state *stc, double gg, double sb, cudaStream_t s)
{
    gpe_state *st = const_cast<gpe_state *>(stc);
    const gpe_grid *g = st->grid;
    ObsArgs<R, CT> a{};
    a.psi = (const CT *)st->d_psi;
    a.V0 = (const R *)potential_ptr(st, 0);
    a.V1 = (sb != 0.0) ? (const R *)potential_ptr(st, 1) : nullptr;
    if (sb != 0.0 && !a.V1) return fail(GPE_ERR_ARG, "s_blend != 0 needs potential slot 1");
    a.s = (R)sb;
    a.ihx2 = (R)(1.0 / (g->box.hx * g->box.hx));
    a.ihy2 = (R)(1.0 / (g->box.hy * g->box.hy));
    a.ihz2 = (R)(1.0 / (g->box.hz * g->box.hz));
    a.g = (R)gg;
    a.dV = g->box.hx * g->box.hy * g->box.hz;
    a.partials = st->red.partials;
    a.counter = st->red.counter;
    a.out = (gpe_obs *)(st->red.scalars + 2);
    const size_t smem = smem_bytes<R, BX, BY, BZ, CT>();
    auto k = k_obs<R, BX, BY, BZ, CT>;
    k<<<blocks_for<R>(k, g, smem), KernelCfg<R>::THREADS, smem, s>>>(a, view(g));
    GPE_LAUNCH_CHECK();
    return GPE_OK;
}

// dense <-> packed copy in the state's value type
template <bool STORE>
static void dense_io(const gpe_state *st, void *dense, const GridView &G, const BoxI &bi, cudaStream_t s)
{
    const gpe_grid *g = st->grid;
    const int nb = g->nsm * 8;
    switch (st->dtype) {
    case GPE_C128:
        k_dense_io<double2, STORE><<<nb, 256, 0, s>>>((double2 *)st->d_psi, (double2 *)dense, g->d_org, g->d_mask, G, g->n_stored, bi);
        break;
    case GPE_C64:
        k_dense_io<float2, STORE><<<nb, 256, 0, s>>>((float2 *)st->d_psi, (float2 *)dense, g->d_org, g->d_mask, G, g->n_stored, bi);
        break;
    case GPE_R64:
        k_dense_io<double, STORE><<<nb, 256, 0, s>>>((double *)st->d_psi, (double *)dense, g->d_org, g->d_mask, G, g->n_stored, bi);
        break;
    default:
        k_dense_io<float, STORE><<<nb, 256, 0, s>>>((float *)st->d_psi, (float *)dense, g->d_org, g->d_mask, G, g->n_stored, bi);
        break;
    }
}

static bool is_real_dtype(int dtype) { return dtype == GPE_R64 || dtype == GPE_R32; }

// device error word of the wavefront schedule (0 = fine)
static int wave_error(const gpe_state *st, cudaStream_t s)
{
    if (!st->d_ctr) return GPE_OK;
    unsigned long long e = 0;
    GPE_TRY_CUDA(cudaMemcpyAsync(&e, st->d_ctr + 2, sizeof e, cudaMemcpyDeviceToHost, s));
    GPE_TRY_CUDA(cudaStreamSynchronize(s));
    if (e) return fail(GPE_ERR_CUDA, "a wavefront dependency wait timed out (results are invalid)");
    return GPE_OK;
}

}  // namespace gpe

using namespace gpe;

// ------------------------------------------------------------ C ABI
extern "C" int gpe_state_create(gpe_grid *g, int dtype, gpe_state **out)
{
    if (!g || !out) return fail(GPE_ERR_ARG, "NULL argument");
    *out = nullptr;
    if (dtype != GPE_C128 && dtype != GPE_C64 && dtype != GPE_R64 && dtype != GPE_R32)
        return fail(GPE_ERR_ARG, "dtype must be GPE_C128, GPE_C64, GPE_R64 or GPE_R32");
    gpe_state *st = new gpe_state();
    st->grid = g;
    st->dtype = dtype;
    st->elem = dtype == GPE_C128 ? 16 : (dtype == GPE_R32 ? 4 : 8);
    int rc = dev_alloc(&st->d_psi, g->n_packed * st->elem);
    if (rc == GPE_OK) rc = dev_zero(st->d_psi, g->n_packed * st->elem);
    // E = exp(-V dt/2) in the state's real type (8 bytes for C128 and R64)
    const size_t real_bytes = (dtype == GPE_C128 || dtype == GPE_R64) ? 8 : 4;
    if (rc == GPE_OK) rc = dev_alloc(&st->d_E, g->n_packed * real_bytes);
    if (rc == GPE_OK) rc = dev_alloc_t(&st->d_clock, 1);
    if (rc == GPE_OK) rc = red_alloc(st->red, g->nsm * 32);
    if (rc == GPE_OK && cudaMallocHost(&st->h_obs, sizeof(gpe_obs)) != cudaSuccess)
        rc = fail(GPE_ERR_CUDA, "cudaMallocHost failed");
    if (rc != GPE_OK) {
        dev_free(st->d_psi);
        dev_free(st->d_E);
        dev_free(st->d_clock);
        red_free(st->red);
        if (st->h_obs) cudaFreeHost(st->h_obs);
        delete st;
        return rc;
    }
    g->n_states++;
    *out = st;
    return GPE_OK;
}

extern "C" int gpe_state_destroy(gpe_state *st)
{
    if (!st) return GPE_OK;
    cudaDeviceSynchronize();
    dev_free(st->d_psi);
    for (int i = 0; i < 6; ++i) dev_free(st->d_work[i]);
    dev_free(st->d_E);
    dev_free(st->d_clock);
    dev_free(st->d_done);
    dev_free(st->d_ctr);
    dev_free(st->d_chunk_norm);
    for (int i = 0; i < 2; ++i)
        if (st->gexec[i]) cudaGraphExecDestroy(st->gexec[i]);
    if (st->gcap) cudaStreamDestroy(st->gcap);
    red_free(st->red);
    if (st->h_obs) cudaFreeHost(st->h_obs);
    st->grid->n_states--;
    delete st;
    return GPE_OK;
}

extern "C" int gpe_wait_selftest(double limit_s, int *timed_out, double *waited_s)
{
    if (!timed_out || !(limit_s > 0) || limit_s > 10.0) return fail(GPE_ERR_ARG, "need 0 < limit_s <= 10 and timed_out");
    uint32_t *flags = nullptr;
    unsigned long long *w = nullptr;
    GPE_TRY(dev_alloc_t(&flags, 1));
    int rc = dev_alloc_t(&w, 2);
    if (rc == GPE_OK) rc = dev_zero(flags, sizeof(uint32_t));
    if (rc == GPE_OK) rc = dev_zero(w, 2 * sizeof(unsigned long long));
    unsigned long long h[2] = {0, 0};
    if (rc == GPE_OK) {
        k_wait_selftest<<<1, 32>>>(flags, w, (unsigned long long)(limit_s * 1e9), w + 1);
        count_launch();
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpy(h, w, sizeof h, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) rc = cuda_fail(e, "wait self-test", __FILE__, __LINE__);
    }
    dev_free(flags);
    dev_free(w);
    if (rc != GPE_OK) return rc;
    *timed_out = h[0] != 0;
    if (waited_s) *waited_s = (double)h[1] * 1e-9;
    return GPE_OK;
}

extern "C" int gpe_state_set_graph(gpe_state *st, int steps_per_graph)
{
    GPE_TRY(check_state(st));
    if (steps_per_graph < 0 || steps_per_graph > 4096) return fail(GPE_ERR_ARG, "steps_per_graph must be in [0, 4096]");
    st->graph_steps = steps_per_graph;
    return GPE_OK;
}

extern "C" int gpe_state_device_ptr(gpe_state *st, void **dptr)
{
    GPE_TRY(check_state(st));
    if (!dptr) return fail(GPE_ERR_ARG, "dptr is NULL");
    *dptr = st->d_psi;
    return GPE_OK;
}

extern "C" int gpe_state_load(gpe_state *st, const void *psi, int layout, int on_device, gpe_stream stream)
{
    GPE_TRY(check_state(st));
    if (!psi) return fail(GPE_ERR_ARG, "psi is NULL");
    const gpe_grid *g = st->grid;
    cudaStream_t s = S(stream);
    const GridView G = view(g);
    if (layout == GPE_LAYOUT_COMPACT) {
        // page-locked host input: read in place over the host link by one
        // copy-and-zero kernel, which is faster than a staged memcpy there
        const void *hv = on_device ? nullptr : pinned_view(psi);
        if (hv) {
            const unsigned nbk = (unsigned)g->nsm * 8;
            switch (st->dtype) {
            case GPE_C128: k_load_zero<double2><<<nbk, 256, 0, s>>>((double2 *)st->d_psi, (const double2 *)hv, g->d_V[0], g->n_packed); break;
            case GPE_C64: k_load_zero<float2><<<nbk, 256, 0, s>>>((float2 *)st->d_psi, (const float2 *)hv, g->d_V[0], g->n_packed); break;
            case GPE_R64: k_load_zero<double><<<nbk, 256, 0, s>>>((double *)st->d_psi, (const double *)hv, g->d_V[0], g->n_packed); break;
            default: k_load_zero<float><<<nbk, 256, 0, s>>>((float *)st->d_psi, (const float *)hv, g->d_V[0], g->n_packed); break;
            }
            GPE_LAUNCH_CHECK();
            GPE_TRY_CUDA(cudaStreamSynchronize(s));
            return GPE_OK;
        }
        GPE_TRY_CUDA(cudaMemcpyAsync(st->d_psi, psi, g->n_packed * st->elem,
                                     on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
        switch (st->dtype) {
        case GPE_C128: k_zero_inactive<double2><<<g->nsm * 8, 256, 0, s>>>((double2 *)st->d_psi, g->d_V[0], g->n_packed); break;
        case GPE_C64: k_zero_inactive<float2><<<g->nsm * 8, 256, 0, s>>>((float2 *)st->d_psi, g->d_V[0], g->n_packed); break;
        case GPE_R64: k_zero_inactive<double><<<g->nsm * 8, 256, 0, s>>>((double *)st->d_psi, g->d_V[0], g->n_packed); break;
        default: k_zero_inactive<float><<<g->nsm * 8, 256, 0, s>>>((float *)st->d_psi, g->d_V[0], g->n_packed); break;
        }
        GPE_LAUNCH_CHECK();
        if (!on_device) GPE_TRY_CUDA(cudaStreamSynchronize(s));
        return GPE_OK;
    }
    if (layout != GPE_LAYOUT_DENSE) return fail(GPE_ERR_ARG, "unknown layout %d", layout);
    const BoxI bi{g->box.nx, g->box.ny, g->box.nz, g->bx, g->by, g->bz};
    const size_t dbytes = (size_t)g->box.nx * g->box.ny * g->box.nz * st->elem;
    const void *src = psi;
    void *owned = nullptr;
    if (!on_device) {
        GPE_TRY(dev_alloc(&owned, dbytes));
        cudaError_t e = cudaMemcpyAsync(owned, psi, dbytes, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) {
            dev_free(owned);
            return cuda_fail(e, "cudaMemcpyAsync(psi)", __FILE__, __LINE__);
        }
        src = owned;
    }
    cudaError_t e = cudaMemsetAsync(st->d_psi, 0, g->n_packed * st->elem, s);
    if (e == cudaSuccess) {
        dense_io<false>(st, const_cast<void *>(src), G, bi, s);
        count_launch();
        e = cudaGetLastError();
    }
    if (owned) {
        cudaStreamSynchronize(s);
        dev_free(owned);
    }
    if (e != cudaSuccess) return cuda_fail(e, "gpe_state_load", __FILE__, __LINE__);
    return GPE_OK;
}

extern "C" int gpe_state_store(const gpe_state *st, void *psi, int layout, int on_device, gpe_stream stream)
{
    GPE_TRY(check_state(st));
    if (!psi) return fail(GPE_ERR_ARG, "psi is NULL");
    const gpe_grid *g = st->grid;
    cudaStream_t s = S(stream);
    GPE_TRY(wave_error(st, s));
    if (layout == GPE_LAYOUT_COMPACT) {
        GPE_TRY_CUDA(cudaMemcpyAsync(psi, st->d_psi, g->n_packed * st->elem,
                                     on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
        if (!on_device) GPE_TRY_CUDA(cudaStreamSynchronize(s));
        return GPE_OK;
    }
    if (layout != GPE_LAYOUT_DENSE) return fail(GPE_ERR_ARG, "unknown layout %d", layout);
    const BoxI bi{g->box.nx, g->box.ny, g->box.nz, g->bx, g->by, g->bz};
    const size_t dbytes = (size_t)g->box.nx * g->box.ny * g->box.nz * st->elem;
    void *dst = psi;
    void *owned = nullptr;
    if (!on_device) {
        GPE_TRY(dev_alloc(&owned, dbytes));
        dst = owned;
    }
    const GridView G = view(g);
    cudaError_t e = cudaMemsetAsync(dst, 0, dbytes, s);
    if (e == cudaSuccess) {
        dense_io<true>(st, dst, G, bi, s);
        count_launch();
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && owned) e = cudaMemcpyAsync(psi, owned, dbytes, cudaMemcpyDeviceToHost, s);
    if (owned) {
        cudaError_t e2 = cudaStreamSynchronize(s);
        if (e == cudaSuccess) e = e2;
        dev_free(owned);
    }
    if (e != cudaSuccess) return cuda_fail(e, "gpe_state_store", __FILE__, __LINE__);
    return GPE_OK;
}

extern "C" int gpe_state_copy(gpe_state *dst, const gpe_state *src, gpe_stream stream)
{
    GPE_TRY(check_state(dst));
    GPE_TRY(check_state(src));
    if (dst->grid != src->grid || dst->dtype != src->dtype)
        return fail(GPE_ERR_ARG, "states differ in grid or dtype");
    GPE_TRY_CUDA(cudaMemcpyAsync(dst->d_psi, src->d_psi, src->grid->n_packed * src->elem, cudaMemcpyDeviceToDevice,
                                 S(stream)));
    return GPE_OK;
}

extern "C" int gpe_step_real(gpe_state *st, const gpe_real_params *p, int64_t nsteps, double t0, gpe_stream stream)
{
    GPE_TRY(check_state(st));
    if (is_real_dtype(st->dtype)) return fail(GPE_ERR_ARG, "real-time steps need a complex state");
    if (!p) return fail(GPE_ERR_ARG, "params is NULL");
    if (nsteps < 0) return fail(GPE_ERR_ARG, "nsteps < 0");
    if (p->integrator != GPE_RK4 && p->integrator != GPE_RKHE3 && p->integrator != GPE_RKCK)
        return fail(GPE_ERR_ARG, "unknown integrator %d", p->integrator);
    if (!(p->dt > 0) || !std::isfinite(p->dt)) return fail(GPE_ERR_ARG, "dt must be finite and > 0");
    if (!std::isfinite(p->g)) return fail(GPE_ERR_ARG, "g must be finite");
    if (p->potential == GPE_V_BLEND) {
        if (p->n_knots < 2 || p->n_knots > GPE_MAX_KNOTS) return fail(GPE_ERR_ARG, "n_knots must be in [2, 16]");
        if (!(p->T_ramp > 0)) return fail(GPE_ERR_ARG, "T_ramp must be > 0");
        if (!st->grid->d_V[1]) return fail(GPE_ERR_STATE, "blend needs potential slot 1");
    } else if (p->potential != GPE_V_STATIC) {
        return fail(GPE_ERR_ARG, "unknown potential mode %d", p->potential);
    }
    const gpe_box &b = st->grid->box;
    const double lam = 2.0 / (b.hx * b.hx) + 2.0 / (b.hy * b.hy) + 2.0 / (b.hz * b.hz) + st->grid->v_max;
    const double ylim = rk_stability_limit(p->integrator);
    if (p->dt * lam > ylim)
        return fail(GPE_ERR_UNSTABLE, "dt*lambda_max = %.3g exceeds the integrator's limit %.3g", p->dt * lam, ylim);
    if (nsteps == 0) return GPE_OK;
    cudaStream_t s = S(stream);
    const bool c128 = st->dtype == GPE_C128;
    if (st->grid->stencil == 19) {
        if (p->integrator != GPE_RK4) return fail(GPE_ERR_ARG, "19-point grids step with RK4");
        GPE_TRY(ensure_work(st, 3));
        return rk4_run19(st, p, nsteps, t0, s);
    }
    if (p->integrator != GPE_RK4) {
        GPE_TRY(ensure_work(st, rk_table(p->integrator)->s - 1));
#define RKG_CASE(id, X, Y, Z) \
    case id: return c128 ? rkgen_run<double, X, Y, Z>(st, p, nsteps, t0, s) : rkgen_run<float, X, Y, Z>(st, p, nsteps, t0, s);
        switch (st->grid->shape) { GPE_SHAPES(RKG_CASE) }
#undef RKG_CASE
        return fail(GPE_ERR_STATE, "bad brick shape");
    }
    GPE_TRY(ensure_work(st, 3));
#define RK_CASE(id, X, Y, Z) \
    case id: return c128 ? rk4_run<double, X, Y, Z>(st, p, nsteps, t0, s) : rk4_run<float, X, Y, Z>(st, p, nsteps, t0, s);
    switch (st->grid->shape) { GPE_SHAPES(RK_CASE) }
#undef RK_CASE
    return fail(GPE_ERR_STATE, "bad brick shape");
}

extern "C" int gpe_step_imag(gpe_state *st, const gpe_imag_params *p, int64_t nsteps, gpe_stream stream)
{
    GPE_TRY(check_state(st));
    if (!p) return fail(GPE_ERR_ARG, "params is NULL");
    if (nsteps < 0) return fail(GPE_ERR_ARG, "nsteps < 0");
    if (!(p->dt > 0) || !std::isfinite(p->dt)) return fail(GPE_ERR_ARG, "dt must be finite and > 0");
    if (!(p->N > 0) || !std::isfinite(p->N)) return fail(GPE_ERR_ARG, "N must be finite and > 0");
    if (!std::isfinite(p->g)) return fail(GPE_ERR_ARG, "g must be finite");
    const gpe_box &b = st->grid->box;
    const double lam = 2.0 / (b.hx * b.hx) + 2.0 / (b.hy * b.hy) + 2.0 / (b.hz * b.hz);
    if (p->dt * lam > 4.0)
        return fail(GPE_ERR_UNSTABLE, "dt*lambda_max(T) = %.3g exceeds the Euler substep limit 4", p->dt * lam);
    if (nsteps == 0) return GPE_OK;
    GPE_TRY(ensure_work(st, 1));
    cudaStream_t s = S(stream);
    if (st->grid->stencil == 19) return itp_run19(st, p, nsteps, s);
    const int dt_ = st->dtype;
#define ITP_CASE(id, X, Y, Z)                                                                         \
    case id:                                                                                          \
        switch (dt_) {                                                                                \
        case GPE_C128: return itp_run<double, X, Y, Z>(st, p, nsteps, s);                             \
        case GPE_C64: return itp_run<float, X, Y, Z>(st, p, nsteps, s);                               \
        case GPE_R64: return itp_run<double, X, Y, Z, double>(st, p, nsteps, s);                      \
        default: return itp_run<float, X, Y, Z, float>(st, p, nsteps, s);                             \
        }
    switch (st->grid->shape) { GPE_SHAPES(ITP_CASE) }
#undef ITP_CASE
    return fail(GPE_ERR_STATE, "bad brick shape");
}

extern "C" int gpe_observables(const gpe_state *st, double g, double s_blend, gpe_obs *out, gpe_stream stream)
{
    GPE_TRY(check_state(st));
    if (!out) return fail(GPE_ERR_ARG, "out is NULL");
    if (!std::isfinite(g) || !std::isfinite(s_blend)) return fail(GPE_ERR_ARG, "g and s_blend must be finite");
    cudaStream_t s = S(stream);
    const int dt_ = st->dtype;
    int rc = GPE_ERR_STATE;
#define OBS_CASE(id, X, Y, Z)                                                         \
    case id:                                                                          \
        switch (dt_) {                                                                \
        case GPE_C128: rc = obs_run<double, X, Y, Z>(st, g, s_blend, s); break;       \
        case GPE_C64: rc = obs_run<float, X, Y, Z>(st, g, s_blend, s); break;         \
        case GPE_R64: rc = obs_run<double, X, Y, Z, double>(st, g, s_blend, s); break; \
        default: rc = obs_run<float, X, Y, Z, float>(st, g, s_blend, s); break;       \
        }                                                                             \
        break;
    if (st->grid->stencil == 19) {
        rc = obs_run19(st, g, s_blend, s);
    } else {
        switch (st->grid->shape) { GPE_SHAPES(OBS_CASE) }
    }
#undef OBS_CASE
    if (rc != GPE_OK) return rc;
    GPE_TRY_CUDA(cudaMemcpyAsync(st->h_obs, st->red.scalars + 2, sizeof(gpe_obs), cudaMemcpyDeviceToHost, s));
    GPE_TRY_CUDA(cudaStreamSynchronize(s));
    GPE_TRY(wave_error(st, s));
    *out = *st->h_obs;
    if (out->nonfinite > 0) return fail(GPE_ERR_NONFINITE, "%.0f active cells hold NaN or Inf", out->nonfinite);
    return GPE_OK;
}

extern "C" int gpe_overlap(const gpe_state *a, const gpe_state *b, double out[2], gpe_stream stream)
{
    GPE_TRY(check_state(a));
    GPE_TRY(check_state(b));
    if (!out) return fail(GPE_ERR_ARG, "out is NULL");
    if (a->grid != b->grid || a->dtype != b->dtype) return fail(GPE_ERR_ARG, "states differ in grid or dtype");
    if (is_real_dtype(a->dtype)) return fail(GPE_ERR_ARG, "the overlap is computed for complex states");
    const gpe_grid *g = a->grid;
    cudaStream_t s = S(stream);
    gpe_state *w = const_cast<gpe_state *>(a);
    const int blocks = g->nsm * 4;
    const double dV = g->box.hx * g->box.hy * g->box.hz;
    if (a->dtype == GPE_C128)
        k_overlap<double2><<<blocks, 256, 0, s>>>((const double2 *)a->d_psi, (const double2 *)b->d_psi, g->n_packed,
                                                   dV, w->red.partials, w->red.counter, w->red.scalars + 10);
    else
        k_overlap<float2><<<blocks, 256, 0, s>>>((const float2 *)a->d_psi, (const float2 *)b->d_psi, g->n_packed, dV,
                                                  w->red.partials, w->red.counter, w->red.scalars + 10);
    GPE_LAUNCH_CHECK();
    double h[2];
    GPE_TRY_CUDA(cudaMemcpyAsync(h, w->red.scalars + 10, sizeof h, cudaMemcpyDeviceToHost, s));
    GPE_TRY_CUDA(cudaStreamSynchronize(s));
    out[0] = h[0];
    out[1] = h[1];
    return GPE_OK;
}

extern "C" int gpe_ground_state(gpe_state *st, const gpe_imag_params *p, double tol_dmu, int64_t check_every,
                                int64_t max_steps, int64_t *steps_done, gpe_obs *obs, gpe_stream stream)
{
    GPE_TRY(check_state(st));
    if (!p) return fail(GPE_ERR_ARG, "params is NULL");
    if (check_every < 1 || max_steps < 1 || !(tol_dmu > 0))
        return fail(GPE_ERR_ARG, "need check_every >= 1, max_steps >= 1, tol_dmu > 0");
    double mu_prev = NAN;
    int64_t done = 0;
    gpe_obs o{};
    int rc = GPE_ERR_NOT_CONVERGED;
    while (done < max_steps) {
        int64_t n = check_every < max_steps - done ? check_every : max_steps - done;
        GPE_TRY(gpe_step_imag(st, p, n, stream));
        done += n;
        int r = gpe_observables(st, p->g, 0.0, &o, stream);
        if (r != GPE_OK) {
            rc = r;
            break;
        }
        if (std::isfinite(mu_prev) && std::fabs(o.mu - mu_prev) < tol_dmu) {
            rc = GPE_OK;
            break;
        }
        mu_prev = o.mu;
    }
    if (steps_done) *steps_done = done;
    if (obs) *obs = o;
    if (rc == GPE_ERR_NOT_CONVERGED)
        return fail(GPE_ERR_NOT_CONVERGED, "|dmu| >= %g after %lld steps", tol_dmu, (long long)done);
    return rc;
}
