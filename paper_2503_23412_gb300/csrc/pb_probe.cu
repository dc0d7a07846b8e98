// Read-bandwidth probe of the memory hierarchy (pb_read_bandwidth): the
// denominators of the traversal kernels' roofline. A buffer smaller than the
// L2 cache, read over and over with loads that bypass L1 (ld.global.cg),
// gives the L2 read rate; a buffer many times the L2 size gives the HBM read
// rate. The paper has no counterpart; it is measurement infrastructure.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "../../include/proxybdpt.h"

namespace {

__global__ void __launch_bounds__(256) k_read(const float4 *__restrict__ p, size_t n4, int reps, float *sink) {
    float acc = 0.0f;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (int r = 0; r < reps; ++r)
        for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
            float4 v = __ldcg(p + i);
            acc += v.x + v.y + v.z + v.w;
        }
    if (acc == 123.456f) *sink = acc;   // keeps the loads; never true for the zero-filled buffer
}

}  // namespace

extern "C" pb_status pb_read_bandwidth(int device, size_t bytes, int reps, double *gbs) {
    if (!gbs || bytes < 4096 || reps < 1) return PB_ERR_ARG;
    if (cudaSetDevice(device) != cudaSuccess) return PB_ERR_CUDA;
    int sms = 1;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    const size_t n4 = bytes / 16;
    float4 *buf = nullptr;
    float *sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    pb_status st = PB_OK;
    float ms = 0.0f;
    if (cudaMalloc(&buf, n4 * 16) != cudaSuccess || cudaMalloc(&sink, sizeof(float)) != cudaSuccess) {
        st = PB_ERR_OOM;
    } else if (cudaMemset(buf, 0, n4 * 16) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
               cudaEventCreate(&e1) != cudaSuccess) {
        st = PB_ERR_CUDA;
    } else {
        const int blocks = sms * 8;
        k_read<<<blocks, 256>>>(buf, n4, 1, sink);   // warm-up (and, for a small buffer, fill L2)
        cudaEventRecord(e0);
        k_read<<<blocks, 256>>>(buf, n4, reps, sink);
        cudaEventRecord(e1);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) st = PB_ERR_CUDA;
        else cudaEventElapsedTime(&ms, e0, e1);
    }
    if (st == PB_OK) *gbs = ms > 0.0f ? (double)n4 * 16.0 * reps / (ms * 1e-3) / 1e9 : 0.0;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (buf) cudaFree(buf);
    if (sink) cudaFree(sink);
    return st;
}
