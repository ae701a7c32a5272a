// Measured device peaks for the roofline of the PatchMatch kernels (no
// counterpart in the paper): the FP32 FMA rate, the rate of 8-byte gathers
// served from L1 in the access pattern of the window samples, and the L2
// read bandwidth.  Each is timed with CUDA events on a private stream after
// one warm-up launch.
#include <algorithm>
#include <cstdint>

#include "../../include/mvs.h"
#include "mvs_internal.h"

namespace {

constexpr int kPeakBlock = 256;

// 16 independent FMA chains per thread; `flag` is never set by the caller,
// so the store only keeps the compiler from dropping the arithmetic.
__global__ void __launch_bounds__(kPeakBlock) k_peak_ffma(int iters, float a, float b, int flag, float* out) {
    float acc[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) acc[k] = (float)(threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 16; ++k) acc[k] = fmaf(acc[k], a, b);
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < 16; ++k) s += acc[k];
    if (flag) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// 8-byte gathers from an L1-resident table in the phase kernel's pattern:
// two groups of 16 lanes per warp, lane g of a group reads texel 2 g of a
// row (dilation 2), every load of a thread independent of the others.
__global__ void __launch_bounds__(kPeakBlock) k_peak_gather(const uint2* __restrict__ tab, uint32_t mask, int iters,
                                                            int flag, uint2* out) {
    const int lane = threadIdx.x & 31;
    uint32_t base = (uint32_t)(lane & 15) * 2u + (uint32_t)(lane >> 4) * 97u + blockIdx.x * 131u;
    uint32_t x = 0, y = 0;
    for (int i = 0; i < iters; ++i) {
        uint2 q[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) q[k] = __ldg(tab + ((base + (uint32_t)k * 67u) & mask));
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            x ^= q[k].x;
            y += q[k].y;
        }
        base += 8u * 67u + 5u;
    }
    if (flag) out[blockIdx.x * blockDim.x + threadIdx.x] = make_uint2(x, y);
}

// Coalesced 16-byte reads of an L2-resident buffer (larger than the L1s,
// smaller than L2), grid-stride, `passes` times over it.
__global__ void __launch_bounds__(kPeakBlock) k_peak_l2(const float4* __restrict__ buf, long long n, int passes,
                                                        int flag, float* out) {
    float s = 0.0f;
    for (int p = 0; p < passes; ++p)
        for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
             i += (long long)gridDim.x * blockDim.x) {
            const float4 v = __ldcg(buf + i);
            s += v.x + v.y + v.z + v.w;
        }
    if (flag) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" mvs_status mvs_measure_peaks(int32_t device, double* fp32_flops, double* gathers, double* l2_bytes) {
    if (!fp32_flops && !gathers && !l2_bytes) return MVS_EINVAL;
    int n_dev = 0;
    if (cudaGetDeviceCount(&n_dev) != cudaSuccess || device < 0 || device >= n_dev) return MVS_EINVAL;
    int prev = 0;
    cudaGetDevice(&prev);
    if (cudaSetDevice(device) != cudaSuccess) return MVS_ECUDA;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    struct {
        void* p = nullptr;
    } out, tab, l2;
    mvs_status st = MVS_OK;
    auto ck = [&](cudaError_t e) {
        if (e != cudaSuccess && st == MVS_OK) st = e == cudaErrorMemoryAllocation ? MVS_ENOMEM : MVS_ECUDA;
        return e == cudaSuccess;
    };
    // times `launch` (after one warm-up run) and returns the shortest of
    // five runs in seconds (a peak: the least disturbed run)
    auto timed = [&](auto launch) -> double {
        launch();
        if (!ck(cudaGetLastError())) return 0.0;
        float best = 3.0e38f;
        for (int rep = 0; rep < 5; ++rep) {
            ck(cudaEventRecord(e0, s));
            launch();
            ck(cudaEventRecord(e1, s));
            ck(cudaGetLastError());
            ck(cudaEventSynchronize(e1));
            float ms = 0.0f;
            ck(cudaEventElapsedTime(&ms, e0, e1));
            best = std::min(best, ms);
        }
        count_launch(6);
        return best * 1e-3;
    };
    const unsigned grid = (unsigned)sms * 8u;   // 8 blocks of 8 warps per SM
    if (ck(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) && ck(cudaEventCreate(&e0)) &&
        ck(cudaEventCreate(&e1)) && ck(cudaMalloc(&out.p, (size_t)grid * kPeakBlock * sizeof(uint2)))) {
        if (fp32_flops) {
            const int iters = 4096;
            const double t = timed([&] { k_peak_ffma<<<grid, kPeakBlock, 0, s>>>(iters, 0.999f, 1e-3f, 0, (float*)out.p); });
            *fp32_flops = st == MVS_OK && t > 0 ? 2.0 * 16.0 * iters * (double)grid * kPeakBlock / t : 0.0;
        }
        if (gathers && st == MVS_OK) {
            const uint32_t n = 1u << 12;   // 32 KB of texels
            if (ck(cudaMalloc(&tab.p, n * sizeof(uint2))) && ck(cudaMemsetAsync(tab.p, 1, n * sizeof(uint2), s))) {
                const int iters = 1024;
                const double t = timed([&] {
                    k_peak_gather<<<grid, kPeakBlock, 0, s>>>((const uint2*)tab.p, n - 1u, iters, 0, (uint2*)out.p);
                });
                *gathers = st == MVS_OK && t > 0 ? 8.0 * iters * (double)grid * kPeakBlock / t : 0.0;
            }
        }
        if (l2_bytes && st == MVS_OK) {
            const long long n = (64LL << 20) / (long long)sizeof(float4);   // 64 MB
            if (ck(cudaMalloc(&l2.p, n * sizeof(float4))) && ck(cudaMemsetAsync(l2.p, 0, n * sizeof(float4), s))) {
                const int passes = 8;
                const double t = timed(
                    [&] { k_peak_l2<<<grid, kPeakBlock, 0, s>>>((const float4*)l2.p, n, passes, 0, (float*)out.p); });
                *l2_bytes = st == MVS_OK && t > 0 ? (double)passes * n * sizeof(float4) / t : 0.0;
            }
        }
    }
    if (s) cudaStreamSynchronize(s);
    cudaFree(out.p);
    cudaFree(tab.p);
    cudaFree(l2.p);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    cudaSetDevice(prev);
    return st;
}
