// Learned plane proposals: a small U-Net that maps the reference image and an
// early PatchMatch state to K = 4 plane hypotheses per pixel, trained on the
// depth maps the plain pipeline produces.  (No counterpart in the paper; the
// proposals only add candidates to the propagation step, the ZNCC cost of
// Eq. 4/5 still decides.)
//
// Tensors are channels-last bfloat16 (pixel-major, channels contiguous, a
// multiple of 16 channels); convolutions are implicit GEMMs on the
// fifth-generation tensor cores (conv_tc.cu: TMA-staged operands,
// tcgen05.mma bf16 x bf16 -> fp32 in tensor memory): M = pixels, N = output
// channels, K = taps x input channels.  The data gradient is the same kernel
// run on the output gradient with flipped, transposed weights; the weight
// gradient is a shared-memory-tiled reduction over pixels.  Master weights,
// gradients and Adam moments are fp32.
#include <atomic>
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/mvs.h"
#include "conv_tc.h"
#include "mvs_internal.h"
#include "pm_device.cuh"

namespace {

typedef __nv_bfloat16 bf16;

struct Mat3 {
    float m[9];
};

// Weight gradient: dw[co][tap][ci] += sum_p dy[p][co] * x[p + tap][ci],
// db[co] += sum_p dy[p][co].  A block of 16 x 16 threads owns 16 output x 16
// input channels and `rows` image rows; rows are staged in shared memory.
__global__ void __launch_bounds__(256) k_conv_wgrad(const bf16* __restrict__ x, int Cin, const bf16* __restrict__ dy,
                                                    int Cout, int W, int H, int taps, int rows, float* __restrict__ dw,
                                                    float* __restrict__ db) {
    extern __shared__ float sm[];
    float* dys = sm;                    // [W][16]
    float* xs = sm + W * 16;            // [3][W + 2][16]
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int co = blockIdx.x * 16 + ty, ci = blockIdx.y * 16 + tx;
    float acc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    float bacc = 0.0f;
    const int y0 = blockIdx.z * rows;
    for (int y = y0; y < min(H, y0 + rows); ++y) {
        __syncthreads();
        for (int i = threadIdx.x; i < W * 16; i += 256) {
            int px = i >> 4, c = i & 15;
            dys[i] = __bfloat162float(dy[((long long)y * W + px) * Cout + blockIdx.x * 16 + c]);
        }
        const int nr = taps == 9 ? 3 : 1;
        for (int i = threadIdx.x; i < nr * (W + 2) * 16; i += 256) {
            int c = i & 15, rest = i >> 4, px = rest % (W + 2) - 1, r = rest / (W + 2);
            int yy = taps == 9 ? y + r - 1 : y;
            float v = 0.0f;
            if (yy >= 0 && yy < H && px >= 0 && px < W) v = __bfloat162float(x[((long long)yy * W + px) * Cin + blockIdx.y * 16 + c]);
            xs[i] = v;
        }
        __syncthreads();
        for (int px = 0; px < W; ++px) {
            float d = dys[px * 16 + ty];
            bacc += d;
            if (taps == 9) {
#pragma unroll
                for (int tap = 0; tap < 9; ++tap) {
                    int r = tap / 3, dx = tap % 3;   // x index px + dx - 1, stored at +1
                    acc[tap] = fmaf(d, xs[(r * (W + 2) + px + dx) * 16 + tx], acc[tap]);
                }
            } else {
                acc[0] = fmaf(d, xs[(px + 1) * 16 + tx], acc[0]);
            }
        }
    }
    for (int tap = 0; tap < taps; ++tap) atomicAdd(&dw[((long long)co * taps + tap) * Cin + ci], acc[tap]);
    if (db && blockIdx.y == 0 && tx == 0) atomicAdd(&db[co], bacc);
}

// ---------------------------------------------------------------------------
// elementwise pieces
// ---------------------------------------------------------------------------
// din (W x H, C) += 1/4 of dout at the parent pixel (accumulate when add != 0)
__global__ void k_pool_bwd(const bf16* __restrict__ dout, int W, int H, int C, bf16* __restrict__ din, int add) {
    long long n = (long long)W * H * C;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        int c = (int)(i % C);
        long long p = i / C;
        int x = (int)(p % W), y = (int)(p / W);
        float v = 0.25f * __bfloat162float(dout[((long long)(y / 2) * (W / 2) + x / 2) * C + c]);
        if (add) v += __bfloat162float(din[i]);
        din[i] = __float2bfloat16(v);
    }
}

// gradient of the up-sampling: din (W/2 x H/2, C) = sum of the four children
// of channels [0, C) of dout (W x H, dout_ch)
__global__ void k_up_bwd(const bf16* __restrict__ dout, int W, int H, int C, int dout_ch, bf16* __restrict__ din) {
    long long n = (long long)(W / 2) * (H / 2) * C;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        int c = (int)(i % C);
        long long p = i / C;
        int x = (int)(p % (W / 2)), y = (int)(p / (W / 2));
        float s = 0.0f;
        for (int j = 0; j < 2; ++j)
            for (int k = 0; k < 2; ++k) s += __bfloat162float(dout[((long long)(2 * y + j) * W + 2 * x + k) * dout_ch + c]);
        din[i] = __float2bfloat16(s);
    }
}

// copy channels: dst[p][d_off + c] = src[p][s_off + c], c < C; add != 0 adds
__global__ void k_copy_ch(const bf16* __restrict__ src, int s_ch, int s_off, bf16* __restrict__ dst, int d_ch, int d_off,
                          int C, long long npix, int add) {
    long long n = npix * C;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        int c = (int)(i % C);
        long long p = i / C;
        float v = __bfloat162float(src[p * s_ch + s_off + c]);
        if (add) v += __bfloat162float(dst[p * d_ch + d_off + c]);
        dst[p * d_ch + d_off + c] = __float2bfloat16(v);
    }
}

// Forward-pass data movement in 16-byte vectors (8 channels per thread,
// channel counts are multiples of 16, rows of pixels at most 8192 wide).
// 2 x 2 average pooling: out (W/2 x H/2, C) from in (W x H, C), summed in
// the order (0,0), (0,1), (1,0), (1,1) and scaled by 1/4 in fp32.
__global__ void k_pool_fwd_v(const uint4* __restrict__ in, int W, int H, int C, uint4* __restrict__ out) {
    const int cv = C / 8, Wo = W / 2;
    const long long n = (long long)Wo * (H / 2) * cv;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % cv);
        const int p = (int)(i / cv), x = p % Wo, y = p / Wo;
        const uint4 q[4] = {in[((long long)(2 * y) * W + 2 * x) * cv + c], in[((long long)(2 * y) * W + 2 * x + 1) * cv + c],
                            in[((long long)(2 * y + 1) * W + 2 * x) * cv + c],
                            in[((long long)(2 * y + 1) * W + 2 * x + 1) * cv + c]};
        uint32_t r[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            float2 s = make_float2(0.0f, 0.0f);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const uint32_t w = (&q[j].x)[k];
                const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w));
                s.x += f.x;
                s.y += f.y;
            }
            __nv_bfloat162 h = __floats2bfloat162_rn(0.25f * s.x, 0.25f * s.y);
            r[k] = *reinterpret_cast<uint32_t*>(&h);
        }
        out[i] = make_uint4(r[0], r[1], r[2], r[3]);
    }
}

// decoder input: out (W x H, up_ch + C) = [nearest up-sampling of prev
// (W/2 x H/2, up_ch) | skip (W x H, C)], copies of 16-byte vectors
__global__ void k_concat_up(const uint4* __restrict__ prev, int up_ch, const uint4* __restrict__ skip, int C, int W,
                            int H, uint4* __restrict__ out) {
    const int uv = up_ch / 8, sv = C / 8, ov = uv + sv;
    const long long n = (long long)W * H * ov;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % ov);
        const long long p = i / ov;
        const int x = (int)(p % W), y = (int)(p / W);
        out[i] = c < uv ? prev[((long long)(y / 2) * (W / 2) + x / 2) * uv + c] : skip[p * sv + (c - uv)];
    }
}

// gradient through ReLU: g *= (y > 0)
__global__ void k_relu_mask(bf16* __restrict__ g, const bf16* __restrict__ y, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        if (!(__bfloat162float(y[i]) > 0.0f)) g[i] = __float2bfloat16(0.0f);
}

__global__ void k_f32_to_bf16(const float* __restrict__ a, bf16* __restrict__ b, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        b[i] = __float2bfloat16(a[i]);
}

__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       long long n, float lr, float b1, float b2, float eps, float c1, float c2) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float gi = g[i];
        float mi = b1 * m[i] + (1.0f - b1) * gi, vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// ---------------------------------------------------------------------------
// proposal head: 16 outputs per pixel = 4 x (a, nx, ny, nz); inverse depth
// rho = 1/d_hi + (1/d_lo - 1/d_hi) sigmoid(a), normal = (nx, ny, nz) / norm
// ---------------------------------------------------------------------------
struct HeadConst {
    float rho_lo, rho_hi;   // 1/d_hi, 1/d_lo
    float lambda_n;         // weight of the normal term
};

__device__ __forceinline__ void decode(const float* o, const HeadConst& hc, float& rho, float n[3], float& len,
                                       float& sig) {
    sig = 1.0f / (1.0f + expf(-o[0]));
    rho = hc.rho_lo + (hc.rho_hi - hc.rho_lo) * sig;
    len = sqrtf(o[1] * o[1] + o[2] * o[2] + o[3] * o[3]) + 1e-12f;
    n[0] = o[1] / len; n[1] = o[2] / len; n[2] = o[3] / len;
}

// per pixel with a target: loss = min_k |rho_k - rho_t| / (rho_hi - rho_lo)
// + lambda (1 - |n_k . n_t|), rho_t = 1 / target depth; the first k wins
// ties.  L = scale * sum over target pixels; writes dL/d out and adds L to
// *loss_sum.
__global__ void k_proposal_loss(const float* __restrict__ out, const float4* __restrict__ target,
                                const uint8_t* __restrict__ mask, long long npix, HeadConst hc, float scale,
                                float* __restrict__ grad, float* __restrict__ loss_sum) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    float lsum = 0.0f;
    if (i < npix) {
        float* gp = grad + 16 * i;
        for (int k = 0; k < 16; ++k) gp[k] = 0.0f;
        if (mask[i]) {
            const float4 t4 = target[i];
            const float tp[4] = {1.0f / t4.w, t4.x, t4.y, t4.z};
            const float span = hc.rho_hi - hc.rho_lo;
            int best = 0;
            float bl = 3.0e38f;
            for (int k = 0; k < 4; ++k) {
                float rho, n[3], len, sig;
                decode(out + 16 * i + 4 * k, hc, rho, n, len, sig);
                float l = fabsf(rho - tp[0]) / span + hc.lambda_n * (1.0f - fabsf(n[0] * tp[1] + n[1] * tp[2] + n[2] * tp[3]));
                if (l < bl) { bl = l; best = k; }
            }
            float rho, n[3], len, sig;
            const float* o = out + 16 * i + 4 * best;
            decode(o, hc, rho, n, len, sig);
            float sgn = rho > tp[0] ? 1.0f : (rho < tp[0] ? -1.0f : 0.0f);
            gp[4 * best] = scale * sgn * sig * (1.0f - sig);
            float dot = n[0] * tp[1] + n[1] * tp[2] + n[2] * tp[3];
            float sd = dot > 0.0f ? 1.0f : (dot < 0.0f ? -1.0f : 0.0f);
            for (int c = 0; c < 3; ++c)
                gp[4 * best + 1 + c] = scale * hc.lambda_n * (-sd) * (tp[1 + c] - dot * n[c]) / len;
            lsum = bl * scale;
        }
    }
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    if ((threadIdx.x & 31) == 0 && lsum != 0.0f) atomicAdd(loss_sum, lsum);
}

// decode the head into K = 4 planes per pixel (n facing the camera, depth)
__global__ void k_decode_proposals(const float* __restrict__ out, long long npix, int W, HeadConst hc, Mat3 Kinv,
                                   float4* __restrict__ props) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= npix) return;
    int x = (int)(i % W), y = (int)(i / W);
    float r0 = Kinv.m[0] * x + Kinv.m[1] * y + Kinv.m[2], r1 = Kinv.m[3] * x + Kinv.m[4] * y + Kinv.m[5];
    float r2 = Kinv.m[6] * x + Kinv.m[7] * y + Kinv.m[8];
    for (int k = 0; k < 4; ++k) {
        float rho, n[3], len, sig;
        decode(out + 16 * i + 4 * k, hc, rho, n, len, sig);
        if (n[0] * r0 + n[1] * r1 + n[2] * r2 > 0.0f) { n[0] = -n[0]; n[1] = -n[1]; n[2] = -n[2]; }
        props[4 * i + k] = make_float4(n[0], n[1], n[2], 1.0f / rho);
    }
}

// network input (16 channels, bf16): image / 255, normalised inverse depth,
// normal (3), cost / 2, zeros
__global__ void k_make_input(const uint8_t* __restrict__ img, const float4* __restrict__ plane,
                             const float* __restrict__ cost, long long npix, HeadConst hc, bf16* __restrict__ in) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= npix) return;
    float4 p = plane[i];
    float rho = p.w > 0.0f ? 1.0f / p.w : hc.rho_lo;
    float v[6] = {img[i] / 255.0f, (rho - hc.rho_lo) / (hc.rho_hi - hc.rho_lo), p.x, p.y, p.z, cost[i] * 0.5f};
    uint32_t w[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * c], v[2 * c + 1]);
        w[c] = *reinterpret_cast<uint32_t*>(&h);
    }
    uint4* o = reinterpret_cast<uint4*>(in + 16 * i);
    o[0] = make_uint4(w[0], w[1], w[2], 0u);
    o[1] = make_uint4(0u, 0u, 0u, 0u);
}

unsigned blocks(long long n, int b = 256) {
    long long g = (n + b - 1) / b;
    return (unsigned)(g > 152LL * 32 ? 152LL * 32 : (g < 1 ? 1 : g));
}

}  // namespace

// ===========================================================================
// host side: the network, its buffers and the C ABI
// ===========================================================================
namespace {

struct Layer {
    int cin, cout, taps;
    bool relu;
    size_t nw;                     // cout * taps * cin
    float *w, *b, *gw, *gb, *mw, *vw, *mb, *vb;
    bf16 *wt, *wtf;                // bf16 B operands of the tensor-core convolution: forward, data gradient
};

// channel plan (level l has 1/2^l resolution)
enum { E0, E1, E2, E3, E4, D3, D2, D1, D0, HEAD, NL };
const int kLayerCin[NL] = {16, 32, 48, 64, 96, 224, 160, 112, 80, 32};
const int kLayerCout[NL] = {32, 48, 64, 96, 128, 96, 64, 48, 32, 16};

cudaError_t g_cnn_err = cudaSuccess;

// widest level-0 image the weight-gradient kernel stages in shared memory
// (256 B per column)
constexpr int kMaxTrainWidth = 768;

}  // namespace

struct mvs_cnn {
    int maxW = 0, maxH = 0;
    cudaStream_t stream = nullptr;
    HeadConst hc;
    Layer L[NL];
    // activations (bf16, channels last)
    bf16 *x = nullptr, *e[5] = {}, *p[4] = {}, *c[4] = {}, *d[4] = {};
    float* y = nullptr;            // head output, 16 channels fp32
    // gradients
    bf16 *gyb = nullptr, *gd[4] = {}, *gc[4] = {}, *ge[5] = {}, *gp[4] = {};
    float* gy = nullptr;
    float* loss = nullptr;
    int* status = nullptr;         // device word: MVS_DEV_TIMEOUT once a bounded wait of a convolution ran out
    int steps = 0;
    int lastW = 0, lastH = 0;      // size of the last forward pass
    std::string err;
    std::vector<void*> allocs;
};

namespace {

template <typename T>
cudaError_t cnn_alloc(mvs_cnn* n, T** p, size_t count) {
    cudaError_t e = cudaMalloc((void**)p, count * sizeof(T) + 256);
    if (e == cudaSuccess) n->allocs.push_back((void*)*p);
    return e;
}

// wait limit of the convolutions' mbarriers (polls, with a 64 ns back-off):
// about a second
constexpr unsigned kConvWaitLimit = 1u << 24;

// One tensor-core convolution; `status` collects a timed-out wait.
cudaError_t conv_launch(mvs_cnn* n, const bf16* in, int Cin, int W, int H, const bf16* wt, const float* bias,
                        int taps, int Cout, bool relu, bool out_f32, void* out, int out_ch, int out_off,
                        cudaStream_t s);

cudaError_t wgrad_launch(const bf16* x, int Cin, const bf16* dy, int Cout, int W, int H, int taps, float* dw, float* db,
                         cudaStream_t s) {
    const int rows = 4;
    dim3 grid(Cout / 16, Cin / 16, (H + rows - 1) / rows);
    size_t smem = (size_t)(W * 16 + 3 * (W + 2) * 16) * sizeof(float);
    // the shared-memory opt-in is a property of the current device
    static std::atomic<bool> attr[128];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
    if (!attr[dev].load()) {
        if ((e = cudaFuncSetAttribute(k_conv_wgrad, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024)) !=
            cudaSuccess)
            return e;
        attr[dev].store(true);
    }
    k_conv_wgrad<<<grid, 256, smem, s>>>(x, Cin, dy, Cout, W, H, taps, rows, dw, db);
    count_launch();
    return cudaGetLastError();
}

#define CUK(call)                         \
    do {                                  \
        cudaError_t _e = (call);          \
        if (_e != cudaSuccess) return _e; \
    } while (0)

cudaError_t refresh_bf16(mvs_cnn* n) {
    for (int i = 0; i < NL; ++i) {
        Layer& L = n->L[i];
        CUK(conv_tc_weights(L.w, L.cout, L.taps, L.cin, 0, L.wt, n->stream));
        CUK(conv_tc_weights(L.w, L.cout, L.taps, L.cin, 1, L.wtf, n->stream));
    }
    return cudaGetLastError();
}

cudaError_t conv_launch(mvs_cnn* n, const bf16* in, int Cin, int W, int H, const bf16* wt, const float* bias,
                        int taps, int Cout, bool relu, bool out_f32, void* out, int out_ch, int out_off,
                        cudaStream_t s) {
    return conv_tc_launch(in, Cin, W, H, wt, bias, taps, Cout, relu, out_f32, out, out_ch, out_off, n->status, 0,
                          kConvWaitLimit, s);
}

// forward pass; x must hold the 16-channel input of a W x H image
cudaError_t cnn_forward(mvs_cnn* n, int W, int H) {
    cudaStream_t s = n->stream;
    auto C = [&](int l) -> const Layer& { return n->L[l]; };
    int Ws[5], Hs[5];
    for (int l = 0; l < 5; ++l) { Ws[l] = W >> l; Hs[l] = H >> l; }
    // encoder
    const bf16* in = n->x;
    for (int l = 0; l <= 4; ++l) {
        const Layer& L = C(E0 + l);
        if (l > 0) {
            k_pool_fwd_v<<<blocks((long long)Ws[l] * Hs[l] * C(E0 + l - 1).cout / 8), 256, 0, s>>>(
                reinterpret_cast<const uint4*>(n->e[l - 1]), Ws[l - 1], Hs[l - 1], C(E0 + l - 1).cout,
                reinterpret_cast<uint4*>(n->p[l - 1]));
            count_launch();
            in = n->p[l - 1];
        }
        CUK(conv_launch(n, in, L.cin, Ws[l], Hs[l], L.wt, L.b, 9, L.cout, true, false, n->e[l], L.cout, 0, s));
    }
    // decoder: level l = 3..0, c[l] = [up(prev) | e[l]]
    const bf16* prev = n->e[4];
    int prev_ch = C(E4).cout;
    for (int l = 3; l >= 0; --l) {
        const Layer& L = C(D3 + (3 - l));
        int ch = L.cin;
        k_concat_up<<<blocks((long long)Ws[l] * Hs[l] * ch / 8), 256, 0, s>>>(
            reinterpret_cast<const uint4*>(prev), prev_ch, reinterpret_cast<const uint4*>(n->e[l]), C(E0 + l).cout,
            Ws[l], Hs[l], reinterpret_cast<uint4*>(n->c[l]));
        count_launch();
        CUK(conv_launch(n, n->c[l], ch, Ws[l], Hs[l], L.wt, L.b, 9, L.cout, true, false, n->d[l], L.cout, 0, s));
        prev = n->d[l];
        prev_ch = L.cout;
    }
    const Layer& Hd = C(HEAD);
    CUK(conv_launch(n, n->d[0], Hd.cin, W, H, Hd.wt, Hd.b, 1, Hd.cout, false, true, n->y, Hd.cout, 0, s));
    return cudaGetLastError();
}

// backward pass from gy (fp32, 16 channels); fills every layer's gw / gb
cudaError_t cnn_backward(mvs_cnn* n, int W, int H) {
    cudaStream_t s = n->stream;
    int Ws[5], Hs[5];
    for (int l = 0; l < 5; ++l) { Ws[l] = W >> l; Hs[l] = H >> l; }
    for (int i = 0; i < NL; ++i) {
        CUK(cudaMemsetAsync(n->L[i].gw, 0, n->L[i].nw * sizeof(float), s));
        CUK(cudaMemsetAsync(n->L[i].gb, 0, n->L[i].cout * sizeof(float), s));
    }
    const long long np0 = (long long)W * H;
    k_f32_to_bf16<<<blocks(np0 * 16), 256, 0, s>>>(n->gy, n->gyb, np0 * 16);
    count_launch();
    Layer& Hd = n->L[HEAD];
    CUK(wgrad_launch(n->d[0], Hd.cin, n->gyb, Hd.cout, W, H, 1, Hd.gw, Hd.gb, s));
    CUK(conv_launch(n, n->gyb, Hd.cout, W, H, Hd.wtf, nullptr, 1, Hd.cin, false, false, n->gd[0], Hd.cin, 0, s));
    // decoder levels 0..3: gd[l] is the gradient of d[l]
    for (int l = 0; l <= 3; ++l) {
        Layer& L = n->L[D3 + (3 - l)];
        long long np = (long long)Ws[l] * Hs[l];
        k_relu_mask<<<blocks(np * L.cout), 256, 0, s>>>(n->gd[l], n->d[l], np * L.cout);
        count_launch();
        CUK(wgrad_launch(n->c[l], L.cin, n->gd[l], L.cout, Ws[l], Hs[l], 9, L.gw, L.gb, s));
        CUK(conv_launch(n, n->gd[l], L.cout, Ws[l], Hs[l], L.wtf, nullptr, 9, L.cin, false, false, n->gc[l], L.cin, 0,
                        s));
        // split gc[l] = [g up(prev) | g e[l] (skip)]
        int up_ch = L.cin - n->L[E0 + l].cout;
        k_copy_ch<<<blocks(np * n->L[E0 + l].cout), 256, 0, s>>>(n->gc[l], L.cin, up_ch, n->ge[l], n->L[E0 + l].cout,
                                                                 0, n->L[E0 + l].cout, np, 0);
        count_launch();
        bf16* dst = l < 3 ? n->gd[l + 1] : n->ge[4];
        long long npc = (long long)Ws[l + 1] * Hs[l + 1];
        k_up_bwd<<<blocks(npc * up_ch), 256, 0, s>>>(n->gc[l], Ws[l], Hs[l], up_ch, L.cin, dst);
        count_launch();
    }
    // encoder levels 4..0: ge[l] is the gradient of e[l]
    for (int l = 4; l >= 0; --l) {
        Layer& L = n->L[E0 + l];
        long long np = (long long)Ws[l] * Hs[l];
        k_relu_mask<<<blocks(np * L.cout), 256, 0, s>>>(n->ge[l], n->e[l], np * L.cout);
        count_launch();
        const bf16* in = l > 0 ? n->p[l - 1] : n->x;
        CUK(wgrad_launch(in, L.cin, n->ge[l], L.cout, Ws[l], Hs[l], 9, L.gw, L.gb, s));
        if (l > 0) {
            CUK(conv_launch(n, n->ge[l], L.cout, Ws[l], Hs[l], L.wtf, nullptr, 9, L.cin, false, false, n->gp[l - 1],
                            L.cin, 0, s));
            long long npf = (long long)Ws[l - 1] * Hs[l - 1];
            k_pool_bwd<<<blocks(npf * L.cin), 256, 0, s>>>(n->gp[l - 1], Ws[l - 1], Hs[l - 1], L.cin, n->ge[l - 1], 1);
            count_launch();
        }
    }
    return cudaGetLastError();
}

uint64_t splitmix(uint64_t& s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

mvs_status cnn_fail(mvs_cnn* n, mvs_status st, const char* msg, cudaError_t e = cudaSuccess) {
    if (n) n->err = std::string(msg) + (e != cudaSuccess ? std::string(": ") + cudaGetErrorString(e) : "");
    return st;
}

#define CNK(n, call)                                                                        \
    do {                                                                                    \
        cudaError_t _e = (call);                                                            \
        if (_e != cudaSuccess)                                                              \
            return cnn_fail((n), _e == cudaErrorMemoryAllocation ? MVS_ENOMEM : MVS_ECUDA, #call, _e); \
    } while (0)

bool shape_ok(const mvs_cnn* n, int W, int H) {
    return W >= 16 && H >= 16 && W % 16 == 0 && H % 16 == 0 && W <= n->maxW && H <= n->maxH;
}

}  // namespace

// network input from a PatchMatch state, forward pass, decode (the steps
// mvs_propose in mvs_api.cu runs on a context's view)
cudaError_t cnn_propose(mvs_cnn* n, const uint8_t* img, const float4* plane, const float* cost, int W, int H,
                        const double Kinv[9], float4* props, cudaStream_t s) {
    cudaStream_t keep = n->stream;
    n->stream = s;
    const long long np = (long long)W * H;
    k_make_input<<<(unsigned)((np + 255) / 256), 256, 0, s>>>(img, plane, cost, np, n->hc, n->x);
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cnn_forward(n, W, H);
    if (e == cudaSuccess) {
        Mat3 K;
        for (int i = 0; i < 9; ++i) K.m[i] = (float)Kinv[i];
        k_decode_proposals<<<(unsigned)((np + 255) / 256), 256, 0, s>>>(n->y, np, W, n->hc, K, props);
        count_launch();
        e = cudaGetLastError();
    }
    n->stream = keep;
    return e;
}

bool cnn_shape_ok(const mvs_cnn* n, int W, int H) { return shape_ok(n, W, H); }

extern "C" {

mvs_status mvs_cnn_create(int32_t max_width, int32_t max_height, float d_lo, float d_hi, uint64_t seed,
                          void* cuda_stream, mvs_cnn** out) {
    if (!out) return MVS_EINVAL;
    *out = nullptr;
    if (max_width < 16 || max_height < 16 || max_width % 16 || max_height % 16 || max_width > 8192 ||
        max_height > 8192 || !(d_lo > 0) || !(d_hi > d_lo))
        return MVS_EINVAL;
    mvs_cnn* n = new (std::nothrow) mvs_cnn();
    if (!n) return MVS_ENOMEM;
    n->maxW = max_width;
    n->maxH = max_height;
    n->stream = (cudaStream_t)cuda_stream;
    n->hc.rho_lo = 1.0f / d_hi;
    n->hc.rho_hi = 1.0f / d_lo;
    n->hc.lambda_n = 0.1f;
    const long long np = (long long)max_width * max_height;
    cudaError_t e = cudaSuccess;
    uint64_t rs = seed ^ 0x6A09E667F3BCC909ULL;
    for (int i = 0; i < NL && e == cudaSuccess; ++i) {
        Layer& L = n->L[i];
        L.cin = kLayerCin[i];
        L.cout = kLayerCout[i];
        L.taps = i == HEAD ? 1 : 9;
        L.relu = i != HEAD;
        L.nw = (size_t)L.cout * L.taps * L.cin;
        e = cnn_alloc(n, &L.w, L.nw);
        if (e == cudaSuccess) e = cnn_alloc(n, &L.gw, L.nw);
        if (e == cudaSuccess) e = cnn_alloc(n, &L.mw, L.nw);
        if (e == cudaSuccess) e = cnn_alloc(n, &L.vw, L.nw);
        if (e == cudaSuccess) e = cnn_alloc(n, &L.b, L.cout);
        if (e == cudaSuccess) e = cnn_alloc(n, &L.gb, L.cout);
        if (e == cudaSuccess) e = cnn_alloc(n, &L.mb, L.cout);
        if (e == cudaSuccess) e = cnn_alloc(n, &L.vb, L.cout);
        if (e == cudaSuccess) e = cnn_alloc(n, &L.wt, L.nw);
        if (e == cudaSuccess) e = cnn_alloc(n, &L.wtf, L.nw);
        if (e != cudaSuccess) break;
        // He initialisation (Box-Muller on a splitmix64 stream); the first
        // layer's padding channels (6..15) and the head start small
        std::vector<float> hw(L.nw);
        const int fan_in = L.taps * (i == E0 ? 6 : L.cin);
        const float sd = (i == HEAD ? 0.1f : 1.0f) * sqrtf(2.0f / fan_in);
        for (size_t k = 0; k < L.nw; ++k) {
            double u1 = ((splitmix(rs) >> 11) + 1.0) * (1.0 / 9007199254740993.0);
            double u2 = (splitmix(rs) >> 11) * (1.0 / 9007199254740992.0);
            float v = (float)(sqrt(-2.0 * log(u1)) * cos(2.0 * 3.14159265358979323846 * u2)) * sd;
            if (i == E0 && (int)(k % L.cin) >= 6) v = 0.0f;
            hw[k] = v;
        }
        e = cudaMemcpy(L.w, hw.data(), L.nw * sizeof(float), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemset(L.b, 0, L.cout * sizeof(float));
        if (e == cudaSuccess) e = cudaMemset(L.mw, 0, L.nw * sizeof(float));
        if (e == cudaSuccess) e = cudaMemset(L.vw, 0, L.nw * sizeof(float));
        if (e == cudaSuccess) e = cudaMemset(L.mb, 0, L.cout * sizeof(float));
        if (e == cudaSuccess) e = cudaMemset(L.vb, 0, L.cout * sizeof(float));
    }
    // activations and gradients at the maximum size
    for (int l = 0; l < 5 && e == cudaSuccess; ++l) {
        long long npl = np >> (2 * l);
        e = cnn_alloc(n, &n->e[l], npl * kLayerCout[E0 + l]);
        if (e == cudaSuccess) e = cnn_alloc(n, &n->ge[l], npl * kLayerCout[E0 + l]);
        if (e == cudaSuccess && l < 4) e = cnn_alloc(n, &n->p[l], (npl / 4) * kLayerCout[E0 + l]);
        if (e == cudaSuccess && l < 4) e = cnn_alloc(n, &n->gp[l], (npl / 4) * kLayerCout[E0 + l]);
        if (e == cudaSuccess && l < 4) e = cnn_alloc(n, &n->c[l], npl * kLayerCin[D3 + (3 - l)]);
        if (e == cudaSuccess && l < 4) e = cnn_alloc(n, &n->gc[l], npl * kLayerCin[D3 + (3 - l)]);
        if (e == cudaSuccess && l < 4) e = cnn_alloc(n, &n->d[l], npl * kLayerCout[D3 + (3 - l)]);
        if (e == cudaSuccess && l < 4) e = cnn_alloc(n, &n->gd[l], npl * kLayerCout[D3 + (3 - l)]);
    }
    if (e == cudaSuccess) e = cnn_alloc(n, &n->x, np * 16);
    if (e == cudaSuccess) e = cnn_alloc(n, &n->y, np * 16);
    if (e == cudaSuccess) e = cnn_alloc(n, &n->gy, np * 16);
    if (e == cudaSuccess) e = cnn_alloc(n, &n->gyb, np * 16);
    if (e == cudaSuccess) e = cnn_alloc(n, &n->loss, 1);
    if (e == cudaSuccess) e = cnn_alloc(n, &n->status, 1);
    if (e == cudaSuccess) e = cudaMemsetAsync(n->status, 0, sizeof(int), n->stream);
    if (e == cudaSuccess) e = refresh_bf16(n);
    if (e == cudaSuccess) e = cudaStreamSynchronize(n->stream);
    if (e != cudaSuccess) {
        g_cnn_err = e;
        mvs_cnn_destroy(n);
        return e == cudaErrorMemoryAllocation ? MVS_ENOMEM : MVS_ECUDA;
    }
    *out = n;
    return MVS_OK;
}

void mvs_cnn_destroy(mvs_cnn* n) {
    if (!n) return;
    cudaStreamSynchronize(n->stream);
    for (void* p : n->allocs) cudaFree(p);
    delete n;
}

const char* mvs_cnn_last_error(const mvs_cnn* n) {
    return n ? n->err.c_str() : (g_cnn_err != cudaSuccess ? cudaGetErrorString(g_cnn_err) : "");
}

mvs_status mvs_cnn_n_params(const mvs_cnn* n, int64_t* count) {
    if (!n || !count) return MVS_EINVAL;
    int64_t t = 0;
    for (int i = 0; i < NL; ++i) t += (int64_t)n->L[i].nw + n->L[i].cout;
    *count = t;
    return MVS_OK;
}

// MVS_ETIMEOUT once a convolution's bounded wait ran out since the last
// check (the status word is cleared); call after synchronising the stream
static mvs_status check_status(mvs_cnn* n) {
    int st = 0;
    CNK(n, cudaMemcpyAsync(&st, n->status, sizeof st, cudaMemcpyDeviceToHost, n->stream));
    CNK(n, cudaStreamSynchronize(n->stream));
    if (st == 0) return MVS_OK;
    CNK(n, cudaMemsetAsync(n->status, 0, sizeof(int), n->stream));
    return cnn_fail(n, MVS_ETIMEOUT, "a tensor-core convolution gave up waiting for its operands");
}

static mvs_status copy_params(mvs_cnn* n, float* host, bool grads, bool set) {
    size_t off = 0;
    for (int i = 0; i < NL; ++i) {
        Layer& L = n->L[i];
        float* w = grads ? L.gw : L.w;
        float* b = grads ? L.gb : L.b;
        if (set) {
            CNK(n, cudaMemcpyAsync(w, host + off, L.nw * sizeof(float), cudaMemcpyHostToDevice, n->stream));
            CNK(n, cudaMemcpyAsync(b, host + off + L.nw, L.cout * sizeof(float), cudaMemcpyHostToDevice, n->stream));
        } else {
            CNK(n, cudaMemcpyAsync(host + off, w, L.nw * sizeof(float), cudaMemcpyDeviceToHost, n->stream));
            CNK(n, cudaMemcpyAsync(host + off + L.nw, b, L.cout * sizeof(float), cudaMemcpyDeviceToHost, n->stream));
        }
        off += L.nw + L.cout;
    }
    if (set) CNK(n, refresh_bf16(n));
    CNK(n, cudaStreamSynchronize(n->stream));
    return check_status(n);
}

mvs_status mvs_cnn_get_params(mvs_cnn* n, float* host_out) {
    if (!n || !host_out) return MVS_EINVAL;
    return copy_params(n, host_out, false, false);
}

mvs_status mvs_cnn_set_params(mvs_cnn* n, const float* host_in) {
    if (!n || !host_in) return MVS_EINVAL;
    return copy_params(n, const_cast<float*>(host_in), false, true);
}

mvs_status mvs_cnn_get_grads(mvs_cnn* n, float* host_out) {
    if (!n || !host_out) return MVS_EINVAL;
    return copy_params(n, host_out, true, false);
}

static mvs_status run_forward(mvs_cnn* n, const uint8_t* img, const float4* plane, const float* cost, int W, int H) {
    if (!shape_ok(n, W, H))
        return cnn_fail(n, MVS_EINVAL, "width and height must be multiples of 16 within the capacity");
    if (((uintptr_t)plane & 15u) || ((uintptr_t)cost & 3u))
        return cnn_fail(n, MVS_EINVAL, "plane must be 16-byte and cost 4-byte aligned");
    const long long np = (long long)W * H;
    k_make_input<<<(unsigned)((np + 255) / 256), 256, 0, n->stream>>>(img, plane, cost, np, n->hc, n->x);
    count_launch();
    CNK(n, cudaGetLastError());
    CNK(n, cnn_forward(n, W, H));
    n->lastW = W;
    n->lastH = H;
    return MVS_OK;
}

mvs_status mvs_cnn_forward(mvs_cnn* n, const uint8_t* img, const float* plane, const float* cost, int32_t W,
                           int32_t H, float* out) {
    if (!n || !img || !plane || !cost || !out) return MVS_EINVAL;
    mvs_status st = run_forward(n, img, (const float4*)plane, cost, W, H);
    if (st != MVS_OK) return st;
    CNK(n, cudaMemcpyAsync(out, n->y, (size_t)W * H * 16 * sizeof(float), cudaMemcpyDeviceToDevice, n->stream));
    return MVS_OK;
}

mvs_status mvs_cnn_backward(mvs_cnn* n, const uint8_t* img, const float* plane, const float* cost, int32_t W,
                            int32_t H, const float* target, const uint8_t* mask, float* loss_out) {
    if (!n || !img || !plane || !cost || !target || !mask) return MVS_EINVAL;
    if (W > kMaxTrainWidth) return cnn_fail(n, MVS_EINVAL, "training width above the weight-gradient kernel's limit");
    if ((uintptr_t)target & 15u) return cnn_fail(n, MVS_EINVAL, "target must be 16-byte aligned");
    mvs_status st = run_forward(n, img, (const float4*)plane, cost, W, H);
    if (st != MVS_OK) return st;
    const long long np = (long long)W * H;
    CNK(n, cudaMemsetAsync(n->loss, 0, sizeof(float), n->stream));
    k_proposal_loss<<<(unsigned)((np + 255) / 256), 256, 0, n->stream>>>(n->y, (const float4*)target, mask, np, n->hc,
                                                                         1.0f / (float)np, n->gy, n->loss);
    count_launch();
    CNK(n, cudaGetLastError());
    CNK(n, cnn_backward(n, W, H));
    if (loss_out) {
        CNK(n, cudaMemcpyAsync(loss_out, n->loss, sizeof(float), cudaMemcpyDeviceToHost, n->stream));
        CNK(n, cudaStreamSynchronize(n->stream));
        return check_status(n);
    }
    return MVS_OK;
}

mvs_status mvs_cnn_propose(mvs_cnn* n, const uint8_t* img, const float* plane, const float* cost, int32_t W,
                           int32_t H, const double Kinv[9], float* proposals) {
    if (!n || !img || !plane || !cost || !Kinv || !proposals) return MVS_EINVAL;
    if (!shape_ok(n, W, H))
        return cnn_fail(n, MVS_EINVAL, "width and height must be multiples of 16 within the capacity");
    if (((uintptr_t)plane & 15u) || ((uintptr_t)cost & 3u) || ((uintptr_t)proposals & 15u))
        return cnn_fail(n, MVS_EINVAL, "plane and proposals must be 16-byte, cost 4-byte aligned");
    CNK(n, cnn_propose(n, img, (const float4*)plane, cost, W, H, Kinv, (float4*)proposals, n->stream));
    return MVS_OK;
}

mvs_status mvs_cnn_read(mvs_cnn* n, int32_t tensor, int32_t level, void* host_out, int64_t bytes) {
    if (!n || !host_out) return MVS_EINVAL;
    if (!n->lastW) return cnn_fail(n, MVS_EINVAL, "no forward pass yet");
    const void* src = nullptr;
    int ch = 0, lv = level;
    size_t elem = sizeof(bf16);
    auto in_range = [&](int hi) { return level >= 0 && level <= hi; };
    switch (tensor) {
        case MVS_CNN_T_INPUT: if (level == 0) { src = n->x; ch = 16; } break;
        case MVS_CNN_T_ENC: if (in_range(4)) { src = n->e[level]; ch = kLayerCout[E0 + level]; } break;
        case MVS_CNN_T_POOL: if (in_range(3)) { src = n->p[level]; ch = kLayerCout[E0 + level]; lv = level + 1; } break;
        case MVS_CNN_T_CAT: if (in_range(3)) { src = n->c[level]; ch = kLayerCin[D3 + (3 - level)]; } break;
        case MVS_CNN_T_DEC: if (in_range(3)) { src = n->d[level]; ch = kLayerCout[D3 + (3 - level)]; } break;
        case MVS_CNN_T_HEAD: if (level == 0) { src = n->y; ch = 16; elem = sizeof(float); } break;
        case MVS_CNN_T_GRAD_HEAD: if (level == 0) { src = n->gyb; ch = 16; } break;
        case MVS_CNN_T_GRAD_DEC: if (in_range(3)) { src = n->gd[level]; ch = kLayerCout[D3 + (3 - level)]; } break;
        case MVS_CNN_T_GRAD_CAT: if (in_range(3)) { src = n->gc[level]; ch = kLayerCin[D3 + (3 - level)]; } break;
        case MVS_CNN_T_GRAD_ENC: if (in_range(4)) { src = n->ge[level]; ch = kLayerCout[E0 + level]; } break;
        case MVS_CNN_T_GRAD_POOL:
            if (in_range(3)) { src = n->gp[level]; ch = kLayerCout[E0 + level]; lv = level + 1; }
            break;
        default: break;
    }
    if (!src) return cnn_fail(n, MVS_EINVAL, "no such tensor");
    const size_t need = (size_t)(n->lastW >> lv) * (size_t)(n->lastH >> lv) * ch * elem;
    if ((int64_t)need != bytes) return cnn_fail(n, MVS_EINVAL, "size mismatch");
    CNK(n, cudaMemcpyAsync(host_out, src, need, cudaMemcpyDeviceToHost, n->stream));
    CNK(n, cudaStreamSynchronize(n->stream));
    return check_status(n);
}

mvs_status mvs_cnn_test_timeout(mvs_cnn* n) {
    if (!n) return MVS_EINVAL;
    // one 16 x 16 convolution of the input buffer whose first wait targets a
    // barrier that nothing completes, with a wait limit of about 0.1 ms
    CNK(n, conv_tc_launch(n->x, 16, 16, 16, n->L[E0].wt, n->L[E0].b, 9, n->L[E0].cout, true, false, n->e[0],
                          n->L[E0].cout, 0, n->status, 1, 1500u, n->stream));
    CNK(n, cudaStreamSynchronize(n->stream));
    return check_status(n);
}

mvs_status mvs_cnn_adam_step(mvs_cnn* n, float lr) {
    if (!n || !(lr > 0)) return MVS_EINVAL;
    n->steps++;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - powf(b1, (float)n->steps), c2 = 1.0f - powf(b2, (float)n->steps);
    for (int i = 0; i < NL; ++i) {
        Layer& L = n->L[i];
        k_adam<<<blocks((long long)L.nw), 256, 0, n->stream>>>(L.w, L.gw, L.mw, L.vw, (long long)L.nw, lr, b1, b2, 1e-8f,
                                                               c1, c2);
        k_adam<<<1, 256, 0, n->stream>>>(L.b, L.gb, L.mb, L.vb, L.cout, lr, b1, b2, 1e-8f, c1, c2);
        count_launch(2);
    }
    CNK(n, cudaGetLastError());
    CNK(n, refresh_bf16(n));
    return MVS_OK;
}

}  // extern "C"
