// noalloc.cu -- an overlap reduction that allocates no device memory.
//
// Some callers cannot call cudaMalloc at the point where they need a result:
// a host application whose memory pool has already reserved the device's free
// HBM for its own arrays, or a loop that must not allocate per call because
// cudaMalloc/cudaFree can synchronise the device and stall work on other
// streams.  gpe_overlap_noalloc serves them: it reads two caller-owned device
// arrays and writes the result to caller memory, and keeps its per-block
// partial sums in a fixed-size array that is part of the library's device
// image (every GPU that loads the library holds it until the process exits).
#include <mutex>

#include "gpe_internal.cuh"

namespace gpe {

// The scratch holds one pair of FP64 partial sums per reduction block, a
// completion counter and the two result values.  One block reduces
// NOALLOC_CHUNK elements, so the array bounds the input size.
constexpr int NOALLOC_THREADS = 256;
constexpr int64_t NOALLOC_CHUNK = 8192;
constexpr int NOALLOC_MAX_BLOCKS = 32768;
constexpr int64_t NOALLOC_MAX_ELEMS = NOALLOC_CHUNK * NOALLOC_MAX_BLOCKS;  // 268,435,456

struct NoallocScratch {
    double partials[2 * NOALLOC_MAX_BLOCKS];
    double result[2];
    unsigned int counter;
};

static __device__ __align__(256) NoallocScratch g_noalloc_scratch;  // 512 KiB + 24 B

// Device address of the scratch array, looked up per device and per CUDA
// context (in host code the symbol name is only a stand-in for it).  The
// array lives in the library's module, which is loaded into each context: if
// a device's context is destroyed and made again (cudaDeviceReset, or a
// framework tearing its context down), the array gets a new address, so the
// cache is keyed on the context's process-unique id and the lookup repeats
// when it changes.
typedef int (*ctx_get_current_fn)(void **ctx);
typedef int (*ctx_get_id_fn)(void *ctx, unsigned long long *id);

struct NoallocSlot {
    unsigned long long ctx_id;
    NoallocScratch *ptr;
};

static std::mutex g_noalloc_mu;
static NoallocSlot g_noalloc_slot[64] = {};
static ctx_get_current_fn g_ctx_current = nullptr;
static ctx_get_id_fn g_ctx_id = nullptr;

// id of the calling thread's current context
static int current_ctx_id(unsigned long long *id)
{
    if (!g_ctx_current || !g_ctx_id) {
        void *f1 = nullptr, *f2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        GPE_TRY_CUDA(cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1));
        GPE_TRY_CUDA(cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2));
        if (q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
            return fail(GPE_ERR_CUDA, "driver entry points cuCtxGetCurrent/cuCtxGetId not available");
        g_ctx_current = reinterpret_cast<ctx_get_current_fn>(f1);
        g_ctx_id = reinterpret_cast<ctx_get_id_fn>(f2);
    }
    void *ctx = nullptr;
    if (g_ctx_current(&ctx) != 0) return fail(GPE_ERR_CUDA, "cuCtxGetCurrent failed");
    if (!ctx) {
        // nothing current on this thread yet: cudaSetDevice initialises the
        // device's primary context and makes it current
        int dev = 0;
        GPE_TRY_CUDA(cudaGetDevice(&dev));
        GPE_TRY_CUDA(cudaSetDevice(dev));
        if (g_ctx_current(&ctx) != 0 || !ctx) return fail(GPE_ERR_CUDA, "no current CUDA context");
    }
    if (g_ctx_id(ctx, id) != 0) return fail(GPE_ERR_CUDA, "cuCtxGetId failed");
    return GPE_OK;
}

static int noalloc_scratch(NoallocScratch **out)
{
    int dev = 0;
    GPE_TRY_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(GPE_ERR_STATE, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    unsigned long long id = 0;
    GPE_TRY(current_ctx_id(&id));
    NoallocSlot &sl = g_noalloc_slot[dev];
    if (!sl.ptr || sl.ctx_id != id) {
        void *p = nullptr;
        GPE_TRY_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        sl.ptr = static_cast<NoallocScratch *>(p);
        sl.ctx_id = id;
    }
    *out = sl.ptr;
    return GPE_OK;
}

// One block per NOALLOC_CHUNK consecutive elements; partial sums of
// conj(a) b in FP64, then the last block to finish adds the per-block partials
// in a fixed order (strided per thread, then a warp and block tree), so the
// result is the same from run to run.
template <typename CT>
__global__ void __launch_bounds__(NOALLOC_THREADS)
    k_overlap_noalloc(const CT *a, const CT *b, int64_t n, double dV, NoallocScratch *scr)
{
    double acc[2] = {0.0, 0.0};
    const int64_t lo = (int64_t)blockIdx.x * NOALLOC_CHUNK;
    const int64_t hi = lo + NOALLOC_CHUNK < n ? lo + NOALLOC_CHUNK : n;
    for (int64_t i = lo + threadIdx.x; i < hi; i += NOALLOC_THREADS) {
        const CT u = a[i], v = b[i];
        acc[0] += (double)(u.x * v.x + u.y * v.y);
        acc[1] += (double)(u.x * v.y - u.y * v.x);
    }
    double tot[2];
    if (reduce_finish<2>(acc, scr->partials, &scr->counter, tot) && threadIdx.x == 0) {
        scr->result[0] = tot[0] * dV;
        scr->result[1] = tot[1] * dV;
    }
}

}  // namespace gpe

using namespace gpe;

extern "C" int gpe_overlap_noalloc(const void *a, const void *b, int64_t n, int dtype, double dV,
                                   double out[2], gpe_stream stream)
{
    if (!a || !b || !out) return fail(GPE_ERR_ARG, "NULL argument");
    if (dtype != GPE_C128 && dtype != GPE_C64) return fail(GPE_ERR_ARG, "dtype must be GPE_C128 or GPE_C64");
    if (n < 1) return fail(GPE_ERR_ARG, "n must be >= 1");
    if (n > NOALLOC_MAX_ELEMS)
        return fail(GPE_ERR_ARG, "n = %lld exceeds the static scratch limit of %lld elements",
                    (long long)n, (long long)NOALLOC_MAX_ELEMS);
    NoallocScratch *scr = nullptr;
    GPE_TRY(noalloc_scratch(&scr));
    cudaStream_t s = S(stream);
    // the completion counter must start at zero; a previous call leaves it at
    // zero, but clear it anyway in case that call did not finish
    GPE_TRY_CUDA(cudaMemsetAsync(&scr->counter, 0, sizeof(unsigned int), s));
    const unsigned blocks = (unsigned)((n + NOALLOC_CHUNK - 1) / NOALLOC_CHUNK);
    if (dtype == GPE_C128)
        k_overlap_noalloc<double2><<<blocks, NOALLOC_THREADS, 0, s>>>((const double2 *)a, (const double2 *)b, n, dV, scr);
    else
        k_overlap_noalloc<float2><<<blocks, NOALLOC_THREADS, 0, s>>>((const float2 *)a, (const float2 *)b, n, dV, scr);
    GPE_LAUNCH_CHECK();
    GPE_TRY_CUDA(cudaMemcpyAsync(out, scr->result, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    GPE_TRY_CUDA(cudaStreamSynchronize(s));
    return GPE_OK;
}
