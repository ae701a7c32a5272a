// Convolutions of the proposal network on the fifth-generation tensor cores
// (no counterpart in the paper; the network proposes extra plane
// hypotheses).  One CTA of four warps computes an implicit GEMM tile:
//   M = 128 pixels (a Wt x Ht block of the image, Wt Ht = 128),
//   N = all output channels (16..224, one MMA width),
//   K = taps x input channels, in k-steps of one chunk of up to 64 input
//   channels (all nine taps, halo tiles) or of one tap and one chunk.
// Operands are staged in shared memory by the tensor-memory accelerator in
// the K-major, non-swizzled core-matrix layout of tcgen05 (8 rows x 16 bytes
// per core matrix), taps that leave the image reading the copy's zero fill
// (the convolution's padding):
//  - rows of at least 128 pixels (3 x 3 filters): a tile is 128 pixels of
//    one row and each group of 8 input channels is copied once with its
//    halo, box 8 x 130 x 3; the nine taps are nine descriptors into that box
//    (start shifted by the tap's row and column), so the activations are
//    read three times instead of nine;
//  - narrower images and 1 x 1 filters: a tile is a Wt x Ht block and each
//    tap and group of 8 channels is one box 8 x Wt x Ht.
// The weights come by one bulk copy per k-step from a layout prepared in the
// operand's order, chunk-major: [chunk][tap][channels of the chunk / 8][N][8].
// One thread (warp 0) issues the copies and another (warp 1) the tcgen05.mma
// instructions (bf16 x bf16, fp32 accumulation in tensor memory), through a
// ring of 2-8 stages guarded by mbarriers: a copy waits only for the MMAs
// that last read its stage, an MMA only for its copies.  Then every thread
// reads its pixel's accumulators with tcgen05.ld, adds the bias, applies
// ReLU and stores bf16 (or fp32).
// Every wait on an mbarrier is bounded: past the limit the CTA records
// MVS_DEV_TIMEOUT in *status, drains what it issued (again bounded), frees
// its tensor memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <mutex>

#include "mvs_internal.h"
#include "conv_tc.h"

namespace {

constexpr int kTcThreads = 128;
constexpr int kTileM = 128;
constexpr uint32_t kBoxBytes = kTileM * 16;  // one 8-channel box of a block tile
constexpr int kHaloW = kTileM + 2, kHaloH = 3;
constexpr uint32_t kHaloBytes = kHaloW * kHaloH * 16;            // one 8-channel box with its halo
constexpr uint32_t kHaloStride = (kHaloBytes + 127u) & ~127u;     // boxes 128-byte aligned
// shared memory per CTA: chunks small enough that two stages take at most
// kChunkBudget, and at most kStageBudget of stages in all, so that two to
// four CTAs (one tile each) share an SM and hide each other's prologue,
// copies and epilogue
constexpr size_t kChunkBudget = 32 * 1024;
constexpr size_t kStageBudget = 44 * 1024;

struct TcArgs {
    int W, H, Cin, Cout, taps;
    int Wt, Ht, tiles_x;
    int halo;                        // 1: 128-pixel row tiles with a shared halo box
    int kc, nchunk, stages;          // input channels per chunk, chunks, pipeline stages
    uint32_t stage_bytes, a_bytes;   // per stage: A part then B part (both 1024-aligned offsets)
    int relu, out_f32;
    const __nv_bfloat16* wt;         // [chunk][tap][chunk channels / 8][Cout][8]
    const float* bias;               // Cout, or null
    void* out;
    int out_ch, out_off;
    int* status;
    int force_timeout;
    unsigned wait_limit;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n"
        ".reg .pred p;\n"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait: true when the phase with the given parity completed
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, unsigned limit) {
    for (unsigned it = 0; it < limit; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if (it > 32) __nanosleep(64);
    }
    return false;
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(bar)
                 : "memory");
}

// shared-memory matrix descriptor: K-major, no swizzle; lbo = byte step
// between core matrices along K, sbo = along M (or N)
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// instruction descriptor of kind::f16: fp32 accumulator, bf16 A and B, both
// K-major, M = 128, N = n
__host__ __device__ constexpr uint32_t mma_idesc(uint32_t n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((n >> 3) << 17) | ((uint32_t)(kTileM >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n"
        ".reg .pred p;\n"
        "setp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
        "}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__global__ void __launch_bounds__(kTcThreads, 1)
    k_conv_tc(const __grid_constant__ CUtensorMap amap, const __grid_constant__ TcArgs a) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-aligned base for the stages (the dynamic allocation holds 1 KB of slack)
    unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    const int S = a.stages;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + (size_t)S * a.stage_bytes);   // full[S], empty[S], done
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * S + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t ncols = a.Cout <= 32 ? 32u : (a.Cout <= 64 ? 64u : (a.Cout <= 128 ? 128u : 256u));

    if (threadIdx.x == 0) {
        for (int s = 0; s < 2 * S + 1; ++s) mbar_init(smem_u32(bars + s), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    const int tile = blockIdx.x;
    const int x0 = (tile % a.tiles_x) * a.Wt, y0 = (tile / a.tiles_x) * a.Ht;
    const int ksteps = a.halo ? a.nchunk : a.taps * a.nchunk;
    const uint32_t idesc = mma_idesc((uint32_t)a.Cout);
    const uint32_t done_bar = smem_u32(bars + 2 * S);
    int* consumed_sm = reinterpret_cast<int*>(tmem_slot + 1);
    bool failed = false;
    int issued = 0;

    if (warp == 0 && lane == 0) {
        // producer: k-step i into stage i % S once the MMAs of k-step i - S
        // have read that stage
        if (a.force_timeout) {
            // a wait on a barrier that nothing completes (checks the timeout path)
            failed = !mbar_wait(smem_u32(bars), 0, a.wait_limit);
        }
        for (int i = 0; i < ksteps && !failed; ++i) {
            const int s = i % S;
            if (i >= S && !mbar_wait(smem_u32(bars + S + s), (uint32_t)((i / S - 1) & 1), a.wait_limit)) {
                failed = true;
                break;
            }
            const int tap = a.halo ? 0 : i / a.nchunk, chunk = a.halo ? i : i % a.nchunk;
            const int kc = min(a.kc, a.Cin - chunk * a.kc);
            const uint32_t sa = smem_u32(smem + (size_t)s * a.stage_bytes);
            const uint32_t sb = sa + a.a_bytes;
            const uint32_t full = smem_u32(bars + s);
            // weights of the chunk (all taps with halo tiles, else one tap)
            const __nv_bfloat16* wsrc = a.wt + (size_t)chunk * a.taps * a.kc * a.Cout + (size_t)tap * kc * a.Cout;
            const uint32_t bbytes = (uint32_t)((a.halo ? a.taps : 1) * kc) * (uint32_t)a.Cout * 2u;
            if (a.halo) {
                mbar_expect_tx(full, (uint32_t)(kc / 8) * kHaloBytes + bbytes);
                for (int b = 0; b < kc / 8; ++b)
                    tma_load_3d(sa + (uint32_t)b * kHaloStride, &amap, chunk * a.kc + 8 * b, x0 - 1, y0 - 1, full);
            } else {
                const int dy = a.taps == 9 ? tap / 3 - 1 : 0, dx = a.taps == 9 ? tap % 3 - 1 : 0;
                mbar_expect_tx(full, (uint32_t)(kc / 8) * kBoxBytes + bbytes);
                for (int b = 0; b < kc / 8; ++b)
                    tma_load_3d(sa + (uint32_t)b * kBoxBytes, &amap, chunk * a.kc + 8 * b, x0 + dx, y0 + dy, full);
            }
            bulk_load(sb, wsrc, bbytes, full);
            issued = i + 1;
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer: k-step j once its copies have landed; the commit frees
        // the stage for the producer when these MMAs have read it
        int consumed = 0;
        for (int j = 0; j < ksteps; ++j) {
            const int s = j % S;
            if (!mbar_wait(smem_u32(bars + s), (uint32_t)((j / S) & 1), a.wait_limit)) {
                failed = true;
                break;
            }
            tc_fence_after();
            const int chunk = a.halo ? j : j % a.nchunk;
            const int kc = min(a.kc, a.Cin - chunk * a.kc);
            const uint32_t sa = smem_u32(smem + (size_t)s * a.stage_bytes);
            const uint32_t sb = sa + a.a_bytes;
            const uint32_t nb = (uint32_t)a.Cout * 16u;   // bytes of one 8-channel group of the weights
            if (a.halo) {
                // tap (dy, dx): the 128 rows starting at halo row (dy + 1, dx + 1)
                for (int t = 0; t < 9; ++t) {
                    const uint32_t shift = (uint32_t)((t / 3) * kHaloW + t % 3) * 16u;
                    for (int kk = 0; kk < kc / 16; ++kk) {
                        const uint64_t ad = smem_desc(sa + (uint32_t)kk * 2u * kHaloStride + shift, kHaloStride, 128u);
                        const uint64_t bd = smem_desc(sb + ((uint32_t)t * (uint32_t)(kc / 8) + 2u * kk) * nb, nb, 128u);
                        mma_bf16(tmem, ad, bd, idesc, (j > 0 || t > 0 || kk > 0) ? 1u : 0u);
                    }
                }
            } else {
                for (int kk = 0; kk < kc / 16; ++kk) {
                    const uint64_t ad = smem_desc(sa + (uint32_t)kk * 2u * kBoxBytes, kBoxBytes, 128u);
                    const uint64_t bd = smem_desc(sb + 2u * kk * nb, nb, 128u);
                    mma_bf16(tmem, ad, bd, idesc, (j > 0 || kk > 0) ? 1u : 0u);
                }
            }
            mma_commit(smem_u32(bars + S + s));   // stage s free once these MMAs have read it
            consumed = j + 1;
        }
        *consumed_sm = consumed;
        mma_commit(done_bar);   // arrives when every MMA issued above has completed
    }
    __syncwarp();   // lanes 1..31 wait for their lane 0 before the block barrier
    __syncthreads();
    if (warp == 0 && lane == 0 && issued > *consumed_sm) {
        // the MMA issuer gave up: wait (bounded) for the copies it did not
        // consume, so that none lands after the CTA has exited
        failed = true;
        for (int j = *consumed_sm; j < issued; ++j)
            mbar_wait(smem_u32(bars + (j % S)), (uint32_t)((j / S) & 1), a.wait_limit);
    }
    if (failed) atomicExch(a.status, MVS_DEV_TIMEOUT);
    __syncwarp();
    // all threads: the accumulators are complete (or the CTA gave up)
    const bool ok = mbar_wait(done_bar, 0, a.wait_limit);
    if (!ok && lane == 0) atomicExch(a.status, MVS_DEV_TIMEOUT);
    tc_fence_after();
    const bool err = __syncthreads_or(failed || !ok) != 0;
    if (!err) {
        const int m = threadIdx.x;   // TMEM lane = tile row = pixel of the tile
        const int px = x0 + m % a.Wt, py = y0 + m / a.Wt;
        const bool valid = px < a.W && py < a.H;
        const long long pix = (long long)py * a.W + px;
        const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
        for (int n0 = 0; n0 < a.Cout; n0 += 16) {
            float v[16];
            tmem_ld16(trow + (uint32_t)n0, v);   // warp-wide: every lane takes part
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                if (a.bias) v[i] += a.bias[n0 + i];
                if (a.relu) v[i] = fmaxf(v[i], 0.0f);
            }
            if (!valid) continue;
            if (a.out_f32) {
                float4* o = reinterpret_cast<float4*>((float*)a.out + pix * a.out_ch + a.out_off + n0);
#pragma unroll
                for (int q = 0; q < 4; ++q) o[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
            } else {
                uint32_t w[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);
                    w[q] = *reinterpret_cast<uint32_t*>(&h);
                }
                uint4* o = reinterpret_cast<uint4*>((__nv_bfloat16*)a.out + pix * a.out_ch + a.out_off + n0);
                o[0] = make_uint4(w[0], w[1], w[2], w[3]);
                o[1] = make_uint4(w[4], w[5], w[6], w[7]);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
    }
}

// weights [co][tap][ci] (fp32) -> the B operand as bf16 in the order
// conv_tc_launch reads: chunk-major over the convolution's input channels K
// (chunks of kc, the last one shorter), then tap, then groups of 8 input
// channels, output channels N, 8 input channels: element (t, k, n) at
//   c taps kc N + t kcc N + ((k - c kc) / 8) N 8 + n 8 + (k - c kc) % 8,
// c = k / kc, kcc = the size of chunk c.  `flip` gives the data-gradient
// filter: N = ci, K = co, taps reversed.
__global__ void k_weights_tc(const float* __restrict__ w, int co_n, int taps, int ci_n, int flip, int kc,
                             __nv_bfloat16* __restrict__ out) {
    const long long n = (long long)co_n * taps * ci_n;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int ci = (int)(i % ci_n);
        const long long r = i / ci_n;
        const int tap = (int)(r % taps), co = (int)(r / taps);
        const int nn = flip ? ci : co, kk = flip ? co : ci, t = flip ? taps - 1 - tap : tap;
        const int N = flip ? ci_n : co_n, K = flip ? co_n : ci_n;
        const int c = kk / kc, kin = kk - c * kc, kcc = min(kc, K - c * kc);
        const long long o = (long long)c * taps * kc * N + (long long)t * kcc * N + (long long)(kin / 8) * N * 8 +
                            (long long)nn * 8 + kin % 8;
        out[o] = __float2bfloat16(w[i]);
    }
}

using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn encode_fn() {
    static EncodeFn fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return (EncodeFn) nullptr;
        return reinterpret_cast<EncodeFn>(p);
    }();
    return fn;
}

int next_pow2(int v) {
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}

}  // namespace

// input channels per chunk of a convolution with K input and N output
// channels: the largest of 64, 32, 16 whose halo-tile stage (taps = 9) or
// block-tile stage fits twice in the chunk budget
int conv_tc_chunk(int K, int N, int taps) {
    for (int kc : {64, 32, 16}) {
        const int k = std::min(kc, K);
        const size_t a = taps == 9 ? (size_t)(k / 8) * kHaloStride : (size_t)(k / 8) * kBoxBytes;
        const size_t b = (size_t)taps * k * N * 2;
        const size_t stage = ((a + 1023) & ~(size_t)1023) + ((b + 1023) & ~(size_t)1023);
        if (2 * stage <= kChunkBudget || kc == 16) return std::min(kc, K);
    }
    return 16;
}

cudaError_t conv_tc_weights(const float* w, int co_n, int taps, int ci_n, int flip, __nv_bfloat16* out,
                            cudaStream_t s) {
    const long long n = (long long)co_n * taps * ci_n;
    const int kc = flip ? conv_tc_chunk(co_n, ci_n, taps) : conv_tc_chunk(ci_n, co_n, taps);
    k_weights_tc<<<(unsigned)std::min<long long>((n + 255) / 256, 152LL * 16), 256, 0, s>>>(w, co_n, taps, ci_n,
                                                                                           flip, kc, out);
    count_launch();
    return cudaGetLastError();
}

// per-stage bytes (A part, whole stage) of a launch
static void stage_bytes(int Cin, int Cout, int taps, int kc, bool halo, uint32_t* a_bytes, uint32_t* stage) {
    const size_t a = halo ? (size_t)(kc / 8) * kHaloStride : (size_t)(kc / 8) * kBoxBytes;
    const size_t b = (size_t)(halo ? taps : 1) * kc * Cout * 2;
    *a_bytes = (uint32_t)((a + 1023) & ~(size_t)1023);
    *stage = *a_bytes + (uint32_t)((b + 1023) & ~(size_t)1023);
    (void)Cin;
}

cudaError_t conv_tc_launch(const __nv_bfloat16* in, int Cin, int W, int H, const __nv_bfloat16* wt, const float* bias,
                           int taps, int Cout, bool relu, bool out_f32, void* out, int out_ch, int out_off,
                           int* status, int force_timeout, unsigned wait_limit, cudaStream_t s) {
    if (Cin % 16 || Cout % 16 || Cout < 16 || Cout > 256 || (taps != 9 && taps != 1) || W < 1 || H < 1)
        return cudaErrorInvalidValue;
    if (((uintptr_t)in & 15u) || ((uintptr_t)wt & 15u) || ((uintptr_t)out & 15u) || (out_off % 16) ||
        (out_ch % 16))
        return cudaErrorInvalidValue;
    EncodeFn enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    TcArgs a{};
    a.W = W; a.H = H; a.Cin = Cin; a.Cout = Cout; a.taps = taps;
    a.halo = taps == 9 && W >= kTileM;
    a.Wt = a.halo ? kTileM : std::min(kTileM, next_pow2(W));
    a.Ht = kTileM / a.Wt;
    a.tiles_x = (W + a.Wt - 1) / a.Wt;
    const int tiles_y = (H + a.Ht - 1) / a.Ht;
    a.kc = conv_tc_chunk(Cin, Cout, taps);
    a.nchunk = (Cin + a.kc - 1) / a.kc;
    stage_bytes(Cin, Cout, taps, a.kc, a.halo, &a.a_bytes, &a.stage_bytes);
    a.stages = (int)std::max<size_t>(2, std::min<size_t>(8, kStageBudget / a.stage_bytes));
    const size_t smem = (size_t)a.stages * a.stage_bytes + (2 * a.stages + 1) * 8 + 16 + 1024;   // + TMEM slot, count
    a.relu = relu; a.out_f32 = out_f32;
    a.wt = wt; a.bias = bias; a.out = out; a.out_ch = out_ch; a.out_off = out_off;
    a.status = status; a.force_timeout = force_timeout; a.wait_limit = wait_limit;
    // activations: channels-last [H][W][Cin] bf16 as a 3D tensor (C, W, H)
    CUtensorMap map;
    const cuuint64_t dims[3] = {(cuuint64_t)Cin, (cuuint64_t)W, (cuuint64_t)H};
    const cuuint64_t strides[2] = {(cuuint64_t)Cin * 2, (cuuint64_t)W * Cin * 2};
    const cuuint32_t box[3] = {8, (cuuint32_t)(a.halo ? kHaloW : a.Wt), (cuuint32_t)(a.halo ? kHaloH : a.Ht)};
    const cuuint32_t estr[3] = {1, 1, 1};
    if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<__nv_bfloat16*>(in), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    // the shared-memory opt-in is a property of the current device
    static std::atomic<bool> attr[128];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
    if (!attr[dev].load()) {
        if ((e = cudaFuncSetAttribute(k_conv_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024)) !=
            cudaSuccess)
            return e;
        attr[dev].store(true);
    }
    const unsigned grid = (unsigned)(a.tiles_x * tiles_y);
    k_conv_tc<<<grid, kTcThreads, smem, s>>>(map, a);
    count_launch();
    return cudaGetLastError();
}
