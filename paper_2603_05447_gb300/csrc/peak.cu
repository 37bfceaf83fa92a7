// peak.cu -- arithmetic-throughput microbenchmarks of the GPU (diagnostics).
//
// The complex128 step of this library is bound by the GPU's FP64 arithmetic,
// not by HBM, so its roofline needs the FP64 fused multiply-add rate of the
// device it runs on.  k_fma_peak runs long chains of independent fused
// multiply-adds (enough chains per thread to cover the pipeline latency,
// enough resident warps per SM to fill every issue slot) and the host side
// times them with CUDA events.  The same kernel in FP32 gives the CUDA-core
// single-precision rate, the other arithmetic roof of the single-precision
// step.
#include "gpe_internal.cuh"

namespace gpe {

constexpr int PEAK_CHAINS = 8;  // independent dependency chains per thread

static __device__ double g_peak_sink;

template <typename T>
__global__ void __launch_bounds__(256) k_fma_peak(int iters, T b, T c)
{
    T acc[PEAK_CHAINS];
#pragma unroll
    for (int k = 0; k < PEAK_CHAINS; ++k) acc[k] = (T)(threadIdx.x + k) * (T)1e-3;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int k = 0; k < PEAK_CHAINS; ++k) acc[k] = fma(acc[k], b, c);
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < PEAK_CHAINS; ++k) s += acc[k];
    // never true for the arguments the host passes; keeps the chains live
    if (s == (T)-12345.0) g_peak_sink = (double)s;
}

template <typename T>
static int fma_peak(int iters, double *tflops, double *seconds)
{
    int dev = 0;
    GPE_TRY_CUDA(cudaGetDevice(&dev));
    const int nsm = sm_count(dev);
    int per = 0;
    GPE_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_fma_peak<T>, 256, 0));
    if (per < 1) per = 1;
    const int blocks = nsm * per;
    cudaStream_t s = nullptr;
    GPE_TRY_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = GPE_OK;
    float ms = 0.f;
    // b slightly below 1 and c small: the chains converge to c / (1 - b)
    // and stay finite, normal numbers
    const T b = (T)0.999999, c = (T)1e-6;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        rc = fail(GPE_ERR_CUDA, "cudaEventCreate failed");
    } else {
        k_fma_peak<T><<<blocks, 256, 0, s>>>(iters / 8 + 1, b, c);  // warm-up
        count_launch();
        cudaEventRecord(e0, s);
        k_fma_peak<T><<<blocks, 256, 0, s>>>(iters, b, c);
        count_launch();
        cudaEventRecord(e1, s);
        const cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess || cudaGetLastError() != cudaSuccess) {
            rc = cuda_fail(e != cudaSuccess ? e : cudaErrorUnknown, "k_fma_peak", __FILE__, __LINE__);
        } else {
            cudaEventElapsedTime(&ms, e0, e1);
            const double flops = 2.0 * 16.0 * PEAK_CHAINS * (double)iters * 256.0 * (double)blocks;
            *seconds = ms * 1e-3;
            *tflops = flops / (*seconds) / 1e12;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaStreamDestroy(s);
    return rc;
}

}  // namespace gpe

using namespace gpe;

extern "C" int gpe_fma_peak(int dtype, int iters, double *tflops, double *seconds)
{
    if (!tflops || !seconds) return fail(GPE_ERR_ARG, "NULL output");
    if (iters < 1 || iters > (1 << 24)) return fail(GPE_ERR_ARG, "iters must be in [1, 2^24]");
    if (dtype == GPE_F64) return fma_peak<double>(iters, tflops, seconds);
    if (dtype == GPE_F32) return fma_peak<float>(iters, tflops, seconds);
    return fail(GPE_ERR_ARG, "dtype must be GPE_F64 or GPE_F32");
}
