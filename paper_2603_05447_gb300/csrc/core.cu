// core.cu -- error reporting, allocation and small utilities of libgpeshell.
#include <atomic>
#include <cstdarg>
#include <cstring>
#include <string>

#include "gpe_internal.cuh"

namespace gpe {

static thread_local std::string g_last_error;
static std::atomic<unsigned long long> g_launches{0};

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char *expr, const char *file, int line)
{
    const char *base = strrchr(file, '/');
    return fail(e == cudaErrorMemoryAllocation ? GPE_ERR_OOM : GPE_ERR_CUDA,
                "%s failed: %s (%s:%d)", expr, cudaGetErrorString(e),
                base ? base + 1 : file, line);
}

int dev_alloc(void **p, size_t bytes)
{
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();  // clear the sticky-free allocation error
        *p = nullptr;
        return fail(e == cudaErrorMemoryAllocation ? GPE_ERR_OOM : GPE_ERR_CUDA,
                    "cudaMalloc(%zu bytes): %s", bytes, cudaGetErrorString(e));
    }
    return GPE_OK;
}

void dev_free(void *p)
{
    if (p) cudaFree(p);
}

// Zero freshly allocated memory and wait for it: the caller's stream may be a
// non-blocking stream that does not order itself after the legacy stream.
int dev_zero(void *p, size_t bytes)
{
    GPE_TRY_CUDA(cudaMemsetAsync(p, 0, bytes, cudaStreamLegacy));
    GPE_TRY_CUDA(cudaStreamSynchronize(cudaStreamLegacy));
    return GPE_OK;
}

int shape_id(int bx, int by, int bz)
{
    if (bx == 8 && by == 8 && bz == 8) return 0;
    if (bx == 8 && by == 8 && bz == 4) return 1;
    if (bx == 8 && by == 4 && bz == 4) return 2;
    return -1;
}

int sm_count(int device)
{
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
        cudaGetLastError();
        n = 1;
    }
    return n;
}

int red_alloc(RedScratch &r, int max_blocks)
{
    if (r.max_blocks >= max_blocks) return GPE_OK;
    red_free(r);
    GPE_TRY(dev_alloc_t(&r.partials, (size_t)max_blocks * 8));
    GPE_TRY(dev_alloc_t(&r.counter, 1));
    GPE_TRY(dev_alloc_t(&r.scalars, 16));
    GPE_TRY(dev_zero(r.counter, sizeof(unsigned int)));
    GPE_TRY(dev_zero(r.scalars, 16 * sizeof(double)));
    r.max_blocks = max_blocks;
    return GPE_OK;
}

void red_free(RedScratch &r)
{
    dev_free(r.partials);
    dev_free(r.counter);
    dev_free(r.scalars);
    r = RedScratch{};
}

int launch_blocks(const gpe_grid *g, int threads, int per_sm)
{
    (void)threads;
    int64_t want = (int64_t)g->nsm * per_sm;
    if (want > g->nb) want = g->nb;
    if (want < 1) want = 1;
    return (int)want;
}

}  // namespace gpe

extern "C" int gpe_version(void) { return 100; }

extern "C" int gpe_launch_count(uint64_t *out)
{
    if (!out) return gpe::fail(GPE_ERR_ARG, "out is NULL");
    *out = (uint64_t)gpe::g_launches.load(std::memory_order_relaxed);
    return GPE_OK;
}

extern "C" int gpe_last_error(char *buf, size_t n)
{
    const std::string &s = gpe::g_last_error;
    if (buf && n > 0) {
        size_t m = s.size() < n - 1 ? s.size() : n - 1;
        memcpy(buf, s.data(), m);
        buf[m] = '\0';
    }
    return (int)s.size();
}
