// dl_bench_fma: the FP64 and FP32 fused-multiply-add rate of this GPU.
//
// The plain FP64 solve is bound by FP64 arithmetic, not by memory, so its
// roofline needs the device's FP64 rate.  The vendor figure is nominal; this
// kernel measures it.  Every thread runs 8 independent FMA chains (a = a*b + c)
// so the pipes stay full, and writes one value to keep the compiler from
// removing the work.
#include <cuda_runtime.h>

#include "dloops.h"

__attribute__((visibility("hidden"))) int dl_record_error(int code, const char *msg);

namespace {

constexpr int kChains = 8;
constexpr int kBlock = 256;

template <typename T>
__global__ void __launch_bounds__(kBlock) fma_chain_kernel(T b, T c, int iters, T *out) {
    T a[kChains];
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = (T)(tid + k) * (T)1e-7;
#pragma unroll 4
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    out[tid] = s;
}

template <typename T>
int run(int iters, int grid, cudaStream_t s, T *out, float *ms) {
    // b slightly below 1 and c small keep every chain finite and normal.
    const T b = (T)0.999999, c = (T)1e-6;
    fma_chain_kernel<T><<<grid, kBlock, 0, s>>>(b, c, iters / 8, out);  // warm-up
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
    fma_chain_kernel<T><<<grid, kBlock, 0, s>>>(b, c, iters, out);
    cudaEventRecord(e1, s);
    cudaError_t err = cudaStreamSynchronize(s);
    if (err == cudaSuccess) err = cudaGetLastError();
    cudaEventElapsedTime(ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return err == cudaSuccess ? DL_OK : dl_record_error(DL_ECUDA, cudaGetErrorString(err));
}

}  // namespace

extern "C" int dl_bench_fma(int precision, void *cuda_stream, double *tflops, double *ms) {
    if ((precision != DL_PREC_F64 && precision != DL_PREC_F32) || !tflops)
        return dl_record_error(DL_EINVAL, "dl_bench_fma: precision must be F64 or F32, tflops non-null");
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return dl_record_error(DL_ECUDA, "dl_bench_fma: no CUDA device");
    const int grid = sms * 8;
    const size_t n = (size_t)grid * kBlock;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    void *out = nullptr;
    if (cudaMalloc(&out, n * sizeof(double)) != cudaSuccess) return dl_record_error(DL_ENOMEM, "dl_bench_fma: cudaMalloc");
    // Iteration counts sized for a few milliseconds on a GPU of this class.
    const int iters = precision == DL_PREC_F64 ? 2048 : 65536;
    float t = 0.f;
    const int rc = precision == DL_PREC_F64 ? run<double>(iters, grid, s, (double *)out, &t)
                                            : run<float>(iters, grid, s, (float *)out, &t);
    cudaFree(out);
    if (rc != DL_OK) return rc;
    const double flops = 2.0 * kChains * (double)iters * (double)n;
    *tflops = t > 0.f ? flops / (t * 1e-3) / 1e12 : 0.0;
    if (ms) *ms = t;
    return DL_OK;
}
