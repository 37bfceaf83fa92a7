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

// Device address of the scratch array on each device, looked up once per
// device (in host code the symbol name is only a stand-in for it).
static std::mutex g_noalloc_mu;
static NoallocScratch *g_noalloc_ptr[64] = {nullptr};

static int noalloc_scratch(NoallocScratch **out)
{
    int dev = 0;
    GPE_TRY_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(GPE_ERR_STATE, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        GPE_TRY_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_noalloc_ptr[dev] = static_cast<NoallocScratch *>(p);
    }
    *out = g_noalloc_ptr[dev];
    return GPE_OK;
}

// One block per NOALLOC_CHUNK consecutive elements; partial sums of
// conj(a) b in FP64, then the last block adds them in block order.
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
