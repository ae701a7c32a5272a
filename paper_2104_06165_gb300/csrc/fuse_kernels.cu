// Depth-map fusion (Sec. III-F): the depth maps of several views are merged
// into one point cloud.  Views are taken in the given order; every pixel of
// view a that is still present (depth > 0, kept, not merged before) is
// back-projected to X, projected into each later view b, and when the pixel
// it lands on is present and its back-projection X' differs from X by less
// than tol times the depth of X, that pixel is merged into X's point and
// removed from view b.
//
// The sequential statement is order dependent only through which pixel of
// view a takes a pixel of view b first (the lowest in raster order), so view
// a is processed in parallel in two passes: every pixel claims its
// consistent targets with an atomicMin of its index, then every pixel
// averages the targets it won and removes them.  Every claimed target is
// removed, so the claim arrays are reset once for the whole fusion.  The points of view a are
// written in raster order after those of the earlier views (a block count,
// a one-block scan, a block-local rank).
//
// The decisions are integers and the paper fixes no precision, so they are
// taken in single precision with every operation rounded on its own
// (__fmul_rn / __fadd_rn / __fsub_rn / __fdiv_rn, no contraction):
//   back-projection of pixel (x, y) with depth d (pinhole K, x_cam = R X + t):
//     yc = (y - cy) / fy, xc = ((x - cx) - s yc) / fx,
//     X = R^T ((d xc, d yc, d) - t), component k = ((R0k e0 + R1k e1) + R2k e2)
//   projection: c = R X + t, component k = ((Rk0 X0 + Rk1 X1) + Rk2 X2) + tk,
//     u = ((fx c0 + s c1) + cx c2) / c2, v = (fy c1 + cy c2) / c2,
//     pixel (floor(u + 1/2), floor(v + 1/2)) when c2 > 0 and inside the image
//   agreement: ((e0 e0 + e1 e1) + e2 e2) < (tol d)^2 with e = X - X'
//   point: (X + X'_b1 + X'_b2 + ...) / count, summed in view order.
#include <algorithm>

#include "mvs_internal.h"

namespace {

constexpr int kFuseBlock = 256;

__device__ __forceinline__ void fuse_backproject(const FuseView& c, int x, int y, float d, float X[3]) {
    const float yc = __fdiv_rn(__fsub_rn((float)y, c.cy), c.fy);
    const float xc = __fdiv_rn(__fsub_rn(__fsub_rn((float)x, c.cx), __fmul_rn(c.sk, yc)), c.fx);
    const float e0 = __fsub_rn(__fmul_rn(d, xc), c.t[0]);
    const float e1 = __fsub_rn(__fmul_rn(d, yc), c.t[1]);
    const float e2 = __fsub_rn(d, c.t[2]);
#pragma unroll
    for (int k = 0; k < 3; ++k)
        X[k] = __fadd_rn(__fadd_rn(__fmul_rn(c.R[k], e0), __fmul_rn(c.R[3 + k], e1)), __fmul_rn(c.R[6 + k], e2));
}

// pixel index of the projection of X into view c, or -1
__device__ __forceinline__ long long fuse_project(const FuseView& c, const float X[3]) {
    float q[3];
#pragma unroll
    for (int k = 0; k < 3; ++k)
        q[k] = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(c.R[3 * k], X[0]), __fmul_rn(c.R[3 * k + 1], X[1])),
                                   __fmul_rn(c.R[3 * k + 2], X[2])),
                         c.t[k]);
    if (!(q[2] > 0.0f)) return -1;
    const float u = __fdiv_rn(__fadd_rn(__fadd_rn(__fmul_rn(c.fx, q[0]), __fmul_rn(c.sk, q[1])), __fmul_rn(c.cx, q[2])), q[2]);
    const float v = __fdiv_rn(__fadd_rn(__fmul_rn(c.fy, q[1]), __fmul_rn(c.cy, q[2])), q[2]);
    const float fu = floorf(__fadd_rn(u, 0.5f)), fv = floorf(__fadd_rn(v, 0.5f));
    if (!(fu >= 0.0f && fu <= (float)(c.W - 1) && fv >= 0.0f && fv <= (float)(c.H - 1))) return -1;
    return (long long)fv * c.W + (long long)fu;
}

__device__ __forceinline__ bool fuse_agree(const float X[3], const float Y[3], float thr) {
    const float e0 = __fsub_rn(X[0], Y[0]), e1 = __fsub_rn(X[1], Y[1]), e2 = __fsub_rn(X[2], Y[2]);
    const float d2 = __fadd_rn(__fadd_rn(__fmul_rn(e0, e0), __fmul_rn(e1, e1)), __fmul_rn(e2, e2));
    return d2 < __fmul_rn(thr, thr);
}

// present pixels of a view: depth > 0 and kept
__global__ void k_fuse_present(FuseView v, const uint8_t* __restrict__ keep) {
    const long long n = (long long)v.W * v.H;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        v.alive[i] = (uint8_t)(v.plane[i].w > 0.0f && (!keep || keep[i]));
}

// pass 1: every present pixel of view a claims the pixels of later views it
// agrees with (the lowest index wins, as in the raster-order statement)
__global__ void __launch_bounds__(kFuseBlock) k_fuse_claim(const FuseView* __restrict__ views, int n, int a, float tol) {
    const FuseView& va = views[a];
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)va.W * va.H || !va.alive[i]) return;
    const int x = (int)(i % va.W), y = (int)(i / va.W);
    const float d = va.plane[i].w;
    float X[3];
    fuse_backproject(va, x, y, d, X);
    const float thr = __fmul_rn(tol, d);
    for (int b = a + 1; b < n; ++b) {
        const FuseView& vb = views[b];
        const long long t = fuse_project(vb, X);
        if (t < 0 || !vb.alive[t]) continue;
        float Y[3];
        fuse_backproject(vb, (int)(t % vb.W), (int)(t / vb.W), vb.plane[t].w, Y);
        if (fuse_agree(X, Y, thr)) atomicMin(vb.claim + t, (int)i);
    }
}

// present pixels of view a per block
__global__ void __launch_bounds__(kFuseBlock) k_fuse_count(FuseView va, int* __restrict__ block_count) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const bool p = i < (long long)va.W * va.H && va.alive[i];
    const int c = __syncthreads_count(p);
    if (threadIdx.x == 0) block_count[blockIdx.x] = c;
}

// exclusive scan of the block counts (one block of 1024 threads, any
// number of blocks), offset by the points already written; the running
// total is updated
__global__ void __launch_bounds__(1024) k_fuse_scan(const int* __restrict__ block_count, long long* __restrict__ block_off,
                                                    int nblk, long long* __restrict__ total) {
    __shared__ long long part[1024];
    const int per = (nblk + 1023) / 1024;
    const int lo = min(nblk, threadIdx.x * per), hi = min(nblk, lo + per);
    long long s = 0;
    for (int k = lo; k < hi; ++k) s += block_count[k];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {   // inclusive Hillis-Steele scan
        long long v = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    long long base = *total + (threadIdx.x ? part[threadIdx.x - 1] : 0);
    for (int k = lo; k < hi; ++k) {
        block_off[k] = base;
        base += block_count[k];
    }
    __syncthreads();
    if (threadIdx.x == 1023) *total += part[1023];
}

// pass 2: every present pixel of view a averages the pixels it won, removes
// them from their views and writes its point at its raster rank
__global__ void __launch_bounds__(kFuseBlock) k_fuse_merge(const FuseView* __restrict__ views, int n, int a,
                                                           const long long* __restrict__ block_off,
                                                           float4* __restrict__ points, int2* __restrict__ src,
                                                           long long cap) {
    __shared__ int warp_count[kFuseBlock / 32];
    const FuseView& va = views[a];
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const bool p = i < (long long)va.W * va.H && va.alive[i];
    // rank of this pixel among the present pixels of the block
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned m = __ballot_sync(0xffffffffu, p);
    if (lane == 0) warp_count[warp] = __popc(m);
    __syncthreads();
    int rank = __popc(m & ((1u << lane) - 1u));
    for (int w = 0; w < warp; ++w) rank += warp_count[w];
    if (!p) return;
    const int x = (int)(i % va.W), y = (int)(i / va.W);
    const float d = va.plane[i].w;
    float X[3], sum[3];
    fuse_backproject(va, x, y, d, X);
    sum[0] = X[0]; sum[1] = X[1]; sum[2] = X[2];
    int cnt = 1;
    for (int b = a + 1; b < n; ++b) {
        const FuseView& vb = views[b];
        const long long t = fuse_project(vb, X);
        // a claim won in this view's pass implies a present, agreeing pixel;
        // claims left from earlier views sit on pixels already removed
        if (t < 0 || vb.claim[t] != (int)i || !vb.alive[t]) continue;
        float Y[3];
        fuse_backproject(vb, (int)(t % vb.W), (int)(t / vb.W), vb.plane[t].w, Y);
        sum[0] = __fadd_rn(sum[0], Y[0]);
        sum[1] = __fadd_rn(sum[1], Y[1]);
        sum[2] = __fadd_rn(sum[2], Y[2]);
        cnt++;
        vb.alive[t] = 0;
        if (vb.owner) vb.owner[t] = block_off[blockIdx.x] + rank;
    }
    const long long k = block_off[blockIdx.x] + rank;
    if (va.owner) va.owner[i] = k;
    if (k < cap) {
        const float fc = (float)cnt;
        points[k] = make_float4(__fdiv_rn(sum[0], fc), __fdiv_rn(sum[1], fc), __fdiv_rn(sum[2], fc), fc);
        if (src) src[k] = make_int2(va.index, (int)i);
    }
}

unsigned blocks_of(long long n, int block) { return (unsigned)((n + block - 1) / block); }

}  // namespace

cudaError_t launch_fuse(const FuseView* host_views, FuseView* dev_views, int n, const uint8_t* const* keep, float tol,
                        int* block_count, long long* block_off, long long* total, float4* points, int2* src,
                        long long cap, cudaStream_t s) {
    cudaError_t e = cudaMemcpyAsync(dev_views, host_views, sizeof(FuseView) * n, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(total, 0, sizeof(long long), s)) != cudaSuccess) return e;
    for (int a = 0; a < n; ++a) {
        const long long np = (long long)host_views[a].W * host_views[a].H;
        k_fuse_present<<<std::min<long long>(blocks_of(np, 256), 152LL * 16), 256, 0, s>>>(host_views[a],
                                                                                           keep ? keep[a] : nullptr);
        count_launch();
        // unclaimed: 0x7f7f7f7f, above every pixel index
        if ((e = cudaMemsetAsync(host_views[a].claim, 0x7f, sizeof(int) * np, s)) != cudaSuccess) return e;
        // pixels never present keep owner -1
        if (host_views[a].owner &&
            (e = cudaMemsetAsync(host_views[a].owner, 0xff, sizeof(long long) * np, s)) != cudaSuccess)
            return e;
    }
    for (int a = 0; a < n; ++a) {
        const long long np = (long long)host_views[a].W * host_views[a].H;
        const unsigned nb = blocks_of(np, kFuseBlock);
        if (a + 1 < n) {
            k_fuse_claim<<<nb, kFuseBlock, 0, s>>>(dev_views, n, a, tol);
            count_launch();
        }
        k_fuse_count<<<nb, kFuseBlock, 0, s>>>(host_views[a], block_count);
        k_fuse_scan<<<1, 1024, 0, s>>>(block_count, block_off, (int)nb, total);
        k_fuse_merge<<<nb, kFuseBlock, 0, s>>>(dev_views, n, a, block_off, points, src, cap);
        count_launch(3);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaGetLastError();
}
