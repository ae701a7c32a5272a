// Device building blocks of the PatchMatch path: Philox4x64-10, the dilated
// support window, the plane-induced homography and the weighted ZNCC of one
// plane hypothesis against all source views (Sec. III-C, Eq. 4, Eq. 5).
//
// Work layout: one warp owns one reference pixel.  The warp is split into
// 32/G groups of G lanes; the n*n window samples are dealt round-robin to the
// G lanes of a group (S slots per lane, sample k = slot * G + lane_in_group)
// and every group keeps the reference side of the window (bilateral weights,
// centred intensities) in registers.  The (hypothesis, view) pairs of a
// batch of hypotheses whose window lands inside the source image are listed
// first, then each group evaluates one listed pair at a time: S bilinear
// gathers per lane and one group reduction phase of three moments.  Pairs that
// fall outside a source and pixels with a flat reference patch therefore
// cost no gathers and leave no lane idle.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_fp16.h>
#include "mvs_internal.h"

namespace mvsdev {

constexpr float kCmax = 2.0f;                       // C_max = 1 - Z_min, Z_min = -1
constexpr float kEpsC = 1e-6f;                      // floor of C(x,j) in the weights of Eq. 5
constexpr float kTauVar = 1e-6f * 1020.0f * 1020.0f;  // flat-patch variance limit, texel units (4 x [0,255])
constexpr float kGraze = 1e-3f;                     // grazing-plane limit |n.r| / |r|
constexpr float kMagic2 = 25165824.0f;              // 1.5 * 2^24: float -> nearest even integer
constexpr int kMagic2Bits = 0x4BC00000;
constexpr float kPi = 3.14159265358979323846f;

__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// float(h) + c for an fp16 h, rounded once (mixed-precision add of sm_100+).
__device__ __forceinline__ float add_f16_f32(__half h, float c) {
    float d;
    asm("add.rn.f32.f16 %0, %1, %2;" : "=f"(d) : "h"(__half_as_ushort(h)), "f"(c));
    return d;
}

// Philox4x64-10 (Salmon et al., SC'11).
__device__ __forceinline__ void philox4x64(unsigned long long c[4], unsigned long long k0,
                                           unsigned long long k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const unsigned long long M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
        unsigned long long hi0 = __umul64hi(M0, c[0]), lo0 = M0 * c[0];
        unsigned long long hi1 = __umul64hi(M1, c[2]), lo1 = M1 * c[2];
        unsigned long long n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
        k0 += 0x9E3779B97F4A7C15ULL;
        k1 += 0xBB67AE8584CAA73BULL;
    }
}

// Uniform in [0, 1) from the top 24 bits of a Philox word (exact in float).
__device__ __forceinline__ float u24(unsigned long long w) {
    return (float)(unsigned)(w >> 40) * (1.0f / 16777216.0f);
}

// Three uniforms for pixel `pix` in phase `phase` (-1 = initialisation):
// counter (pix, phase + 1, 0, 0), key (seed, reference index).
__device__ __forceinline__ void draws3(const RefConst& rc, long long pix, int phase, float u[3]) {
    unsigned long long c[4] = {(unsigned long long)pix, (unsigned long long)(long long)(phase + 1), 0ULL, 0ULL};
    philox4x64(c, rc.seed, (unsigned long long)rc.ref_index);
    u[0] = u24(c[0]);
    u[1] = u24(c[1]);
    u[2] = u24(c[2]);
}

template <int G>
__device__ __forceinline__ float gsum(float v) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <int G>
__device__ __forceinline__ unsigned group_mask(int lane) {
    return G == 32 ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
}

// Four times the bilinear value of a coefficient texture at (x + 1/2, y + 1/2)
// given xs2 = 2x, ys2 = 2y (the caller folds the shift and the factor 2 into
// its homography).  Adding 1.5 * 2^24 rounds 2x to the nearest even integer
// 2i, so U = 2x - 2i lies in [-1, 1] and the bits of the sum give i.  The
// texel index is clamped into the array, so any input (even NaN) reads
// inside the buffer.
__device__ __forceinline__ float tex_sample(const uint2* __restrict__ tex, int pitch, uint32_t n_tex, float xs2,
                                            float ys2) {
    float tx = __fadd_rn(xs2, kMagic2), ty = __fadd_rn(ys2, kMagic2);
    float U = __fsub_rn(xs2, __fsub_rn(tx, kMagic2));
    float V = __fsub_rn(ys2, __fsub_rn(ty, kMagic2));
    uint32_t idx = (uint32_t)__float_as_int(ty) * (uint32_t)pitch + (uint32_t)__float_as_int(tx) +
                   (uint32_t)(pitch + 1) * (uint32_t)(1 - kMagic2Bits);
    idx = min(idx, n_tex - 1u);
    uint2 q = __ldg(tex + idx);
    float2 ab = __half22float2(*reinterpret_cast<const __half2*>(&q.x));
    float2 cd = __half22float2(*reinterpret_cast<const __half2*>(&q.y));
    return fmaf(V, fmaf(U, cd.y, cd.x), fmaf(U, ab.y, ab.x));
}

// The warp-uniform part of one pixel's window: the corners of the included
// sample rectangle, the viewing ray and the reference moments (48 bytes; the
// phase kernel keeps it in shared memory, read where a stage or a round needs
// it).
struct __align__(16) WinGeo {
    float cu_lo, cu_hi, cv_lo, cv_hi;  // corners of the included sample rectangle
    float rx0, rx1, rx2;  // K^-1 (x, y, 1)
    float rlen;           // |K^-1 (x, y, 1)|
    float inv_wsum;       // 1 / sum w
    float srr;            // sum w (I_ref - mean)^2
    float wr_sum;         // sum w (I_ref - mean) (zero up to rounding)
    float wsum;
};

// Reference side of the window of one pixel.  Every group of G lanes of the
// warp holds the same pixel's window (sample k = slot * G + lane_in_group).
template <int S>
struct PixWin {
    float ou[S], ov[S];   // sample offsets (the first included sample for padding / excluded samples)
    float w[S];           // bilateral weights (0 for padding / excluded)
    float wr[S];          // w * (I_ref - weighted mean)
    float mean;           // weighted mean of the reference samples
    WinGeo geo;
    bool ok;              // pixel exists and its reference patch is not flat
};

// Window offsets s*(k - r_now) (Sec. III-C); samples outside the reference
// image are left out of the window.
template <int G, int S>
__device__ __forceinline__ void build_window(const RefConst& rc, int px, int py, bool exists, PixWin<S>& pw) {
    const int lane = threadIdx.x & 31, lg = lane & (G - 1);
    const int n = rc.n;
    const float half = 0.5f * (float)(n - 1);
    // window rows / columns inside the reference image: lane k tests offset k
    // (n <= 22 < 32)
    int ku_lo, ku_hi, kv_lo, kv_hi;
    {
        const float o = rc.step * ((float)lane - half);
        const float eu = (float)px + o, ev = (float)py + o;
        const unsigned mu = __ballot_sync(0xffffffffu, lane < n && eu >= 0.0f && eu <= (float)(rc.W - 1));
        const unsigned mv = __ballot_sync(0xffffffffu, lane < n && ev >= 0.0f && ev <= (float)(rc.H - 1));
        ku_lo = mu ? __ffs(mu) - 1 : n;
        ku_hi = mu ? 31 - __clz(mu) : -1;
        kv_lo = mv ? __ffs(mv) - 1 : n;
        kv_hi = mv ? 31 - __clz(mv) : -1;
    }
    // excluded and padding samples sit on the first included sample (weight 0)
    const float ou_pad = rc.step * ((float)ku_lo - half), ov_pad = rc.step * ((float)kv_lo - half);
    const float rcen = exists ? 4.0f * (float)__ldg(rc.img + (long long)py * rc.W + px) : 0.0f;
    const float inv_n = rcp_approx((float)n);   // (k + 1/2) / n stays 1/(2n) away from integers
    float sw = 0.0f, swr = 0.0f;
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const int k = s * G + lg;
        const int kv = (int)(((float)k + 0.5f) * inv_n), ku = k - kv * n;   // exact for k < 2^20
        bool in = exists && k < n * n && ku >= ku_lo && ku <= ku_hi && kv >= kv_lo && kv <= kv_hi;
        float ou = rc.step * ((float)ku - half), ov = rc.step * ((float)kv - half);
        float r = 0.0f, w = 0.0f;
        if (in) {
            r = tex_sample(rc.tex, rc.pitch, rc.n_tex, 2.0f * ((float)px + ou) - 1.0f, 2.0f * ((float)py + ov) - 1.0f);
            float dc = r - rcen;
            w = __expf(fmaf(rc.sp_coef, ou * ou + ov * ov, rc.col_coef * dc * dc));
        }
        pw.ou[s] = in ? ou : ou_pad;
        pw.ov[s] = in ? ov : ov_pad;
        pw.w[s] = w;
        pw.wr[s] = r;   // temporarily the intensity
        sw += w;
        swr = fmaf(w, r, swr);
    }
    sw = gsum<G>(sw);
    swr = gsum<G>(swr);
    const float inv_sw = sw > 0.0f ? rcp_approx(sw) : 0.0f;
    float mu = swr * inv_sw;
    float srr = 0.0f, wrs = 0.0f;
#pragma unroll
    for (int s = 0; s < S; ++s) {
        float d = pw.wr[s] - mu;
        float t = pw.w[s] * d;
        pw.wr[s] = t;
        wrs += t;
        srr = fmaf(t, d, srr);
    }
    srr = gsum<G>(srr);
    pw.geo.wr_sum = gsum<G>(wrs);
    pw.geo.wsum = sw;
    pw.mean = mu;
    pw.geo.inv_wsum = inv_sw;
    pw.geo.srr = srr;
    pw.ok = exists && sw > 0.0f && srr >= kTauVar * sw && ku_hi >= 0 && kv_hi >= 0;
    WinGeo& g = pw.geo;
    g.cu_lo = rc.step * ((float)ku_lo - half);
    g.cu_hi = rc.step * ((float)ku_hi - half);
    g.cv_lo = rc.step * ((float)kv_lo - half);
    g.cv_hi = rc.step * ((float)kv_hi - half);
    const float* Ki = rc.Kinv;
    float x = (float)px, y = (float)py;
    g.rx0 = fmaf(Ki[0], x, fmaf(Ki[1], y, Ki[2]));
    g.rx1 = fmaf(Ki[3], x, fmaf(Ki[4], y, Ki[5]));
    g.rx2 = fmaf(Ki[6], x, fmaf(Ki[7], y, Ki[8]));
    g.rlen = sqrtf(g.rx0 * g.rx0 + g.rx1 * g.rx1 + g.rx2 * g.rx2);
}

// Source-view constants copied to shared memory once per block (80 bytes,
// read as 16-byte words).
struct __align__(16) ViewSm {
    const uint2* tex;
    // index of texel (i + 1, j + 1) = bits(1.5 * 2^24 + 2 j) * pitch
    // + bits(1.5 * 2^24 + 2 i) + toff (mod 2^32), see tex_sample
    uint32_t pitch, toff;
    uint32_t last, pad_;  // last texel index (W + 1) (H + 1) - 1
    float wm1, hm1;       // W - 1, H - 1
    float A[9];
    float b[3];
};

static_assert(sizeof(ViewSm) == 80 && offsetof(ViewSm, pitch) == 8 && offsetof(ViewSm, toff) == 12 &&
                  offsetof(ViewSm, last) == 16 && offsetof(ViewSm, wm1) == 24 && offsetof(ViewSm, A) == 32 &&
                  offsetof(ViewSm, b) == 68,
              "eval_batch reads ViewSm as 128-bit words");

__device__ __forceinline__ void load_views(const RefConst& rc, ViewSm* sv) {
    for (int j = threadIdx.x; j < rc.n_src; j += blockDim.x) {
        const PairConst& P = rc.pair[j];
        for (int i = 0; i < 9; ++i) sv[j].A[i] = P.A[i];
        for (int i = 0; i < 3; ++i) sv[j].b[i] = P.b[i];
        sv[j].wm1 = (float)(P.W - 1);
        sv[j].hm1 = (float)(P.H - 1);
        sv[j].pitch = (uint32_t)P.pitch;
        sv[j].last = P.n_tex - 1u;
        sv[j].tex = P.tex;
        sv[j].toff = (uint32_t)(P.pitch + 1) * (uint32_t)(1 - kMagic2Bits);
    }
    __syncthreads();
}

// A plane hypothesis held by one lane: (n, d), validity and the homography
// factors m = K^-T n / rho, 1/d.
struct Cand {
    float n0, n1, n2, d;
    float m0, m1, invd;
    bool ok;
};

// Reading of the paper's silent points: a hypothesis is usable only if
// d > 0, n.r < -1e-3 |r| at the pixel and n.r < 0 at every window sample (the
// plane lies in front of the reference camera; n.r is affine in the sample
// position, so the four corners decide).
template <int S>
__device__ __forceinline__ Cand make_cand(const RefConst& rc, const PixWin<S>& pw, const WinGeo& g, float n0,
                                          float n1, float n2, float d, bool want) {
    Cand c;
    c.n0 = n0; c.n1 = n1; c.n2 = n2; c.d = d;
    const float* Ki = rc.Kinv;
    float nr = n0 * g.rx0 + n1 * g.rx1 + n2 * g.rx2;
    float k0 = Ki[0] * n0 + Ki[3] * n1 + Ki[6] * n2;
    float k1 = Ki[1] * n0 + Ki[4] * n1 + Ki[7] * n2;
    bool corners = fmaf(g.cu_lo, k0, fmaf(g.cv_lo, k1, nr)) < 0.0f && fmaf(g.cu_hi, k0, fmaf(g.cv_lo, k1, nr)) < 0.0f &&
                   fmaf(g.cu_lo, k0, fmaf(g.cv_hi, k1, nr)) < 0.0f && fmaf(g.cu_hi, k0, fmaf(g.cv_hi, k1, nr)) < 0.0f;
    c.ok = want && pw.ok && d > 0.0f && d < 3.0e38f && nr < -kGraze * g.rlen && corners;
    float inv_rho = c.ok ? rcp_approx(d * nr) : 0.0f;
    c.m0 = k0 * inv_rho;
    c.m1 = k1 * inv_rho;
    c.invd = c.ok ? rcp_approx(d) : 0.0f;
    return c;
}

// One listed (hypothesis, view) pair in shared memory (three 16-byte
// words): the homography columns H e1, H e2 and H x (x, y rows shifted by
// -1/2 and doubled for tex_sample), the view, and after evaluation its
// per-view cost C(x, j) (C_max when excluded), the hypothesis and the view.
struct __align__(16) PairSm {
    float h0x, h0y, h0z, h1x;
    float h1y, h1z, p0x, p0y;
    float p0z, res;
    int c, j;
};

static_assert(sizeof(PairSm) == 48 && offsetof(PairSm, h1y) == 16 && offsetof(PairSm, p0z) == 32 &&
                  offsetof(PairSm, res) == 36 && offsetof(PairSm, c) == 40 && offsetof(PairSm, j) == 44,
              "eval_batch reads and writes PairSm as 128-bit words");

// Shared-memory bytes of a block: the view table and, per warp, room for
// 8 hypotheses x n_src pairs followed by their 8 x n_src Eq. 5 weights.
__host__ __device__ constexpr size_t smem_views_bytes(int n_src) {
    return ((size_t)n_src * sizeof(ViewSm) + 15) & ~(size_t)15;
}
__host__ __device__ constexpr size_t smem_warp_bytes(int n_src) {
    return (size_t)8 * n_src * (sizeof(PairSm) + sizeof(float));   // 416 n_src: a multiple of 16
}
__host__ __device__ constexpr size_t smem_block_bytes(int n_src, int warps) {
    return smem_views_bytes(n_src) + (size_t)warps * smem_warp_bytes(n_src);
}
// pair list of warp `warp` in a block's dynamic shared memory
__device__ __forceinline__ PairSm* warp_pairs(unsigned char* smem, int n_src, int warp) {
    return reinterpret_cast<PairSm*>(smem + smem_views_bytes(n_src) + (size_t)warp * smem_warp_bytes(n_src));
}

// Two planes (n, depth at the pixel) equal up to float rounding (1e-6
// relative in depth, 1e-6 per normal component); such planes score the same
// cost to within rounding.
__device__ __forceinline__ bool same_plane(const float4& a, const float4& b) {
    return fabsf(a.w - b.w) <= 1e-6f * b.w && fabsf(a.x - b.x) <= 1e-6f && fabsf(a.y - b.y) <= 1e-6f &&
           fabsf(a.z - b.z) <= 1e-6f;
}

// Costs C(x) (Eq. 5) of up to 8 hypotheses of the warp's pixel: lane c < nc
// holds hypothesis c on entry and its cost on return.
//   1. the (hypothesis, view) pairs of the usable hypotheses whose window
//      maps inside the source image (corner test: the image of the window is
//      convex, w > 0 included) are listed in `pairs` (per-warp shared memory,
//      nc * n_src entries) in hypothesis-major, view-minor order, with their
//      homography;
//   2. each group of G lanes takes the next pair: S bilinear gathers per
//      lane, the weighted mean, then the centred moments (group reductions),
//      ZNCC (Eq. 4),
//      C(x,j) = 1 - Z; a view is excluded when its weighted variance is below
//      1e-6 on the [0,1] scale (reading);
//   3. lane c folds the per-view results of hypothesis c in view order
//      (Eq. 5, weights 1/max(C, 1e-6)).
// Must be called by all 32 lanes with the same nc (warp-uniform).
// OFF_SM: the window's sample offsets are read from shared memory, (ou, ov)
// of slot k and lane-in-group lg at off_sm[k * G + lg] (pw.ou / pw.ov are not
// read, so they need not stay in registers).
template <int G, int S, bool VIEWS, bool MIXED = false, bool OFF_SM = false>
__device__ __forceinline__ float eval_batch(const RefConst& rc, const ViewSm* __restrict__ sv, const PixWin<S>& pw,
                                            const WinGeo& geo, int px, int py, const Cand& my, int nc, PairSm* pairs,
                                            float* view_cost, unsigned& n_evals, const float2* off_sm = nullptr) {
    constexpr int NG = 32 / G;
    const int lane = threadIdx.x & 31, lg = lane & (G - 1), grp = lane / G;
    const int V = rc.n_src;
    const float x = (float)px, y = (float)py;
    // ---- 1. list the pairs that map inside the source images, over the
    // usable hypotheses only: lane r < nok holds the lane of the r-th one
    const unsigned okm = __ballot_sync(0xffffffffu, lane < nc && my.ok);
    const int nok = __popc(okm);
    int hyp_of;
    {
        unsigned m = okm;   // drop the lowest set bit `lane` times (nc <= 8)
#pragma unroll
        for (int t = 0; t < 7; ++t)
            if (t < lane) m &= m - 1u;
        hyp_of = m ? __ffs(m) - 1 : 0;
    }
    // Pairs are listed view-major (all usable hypotheses of view 0, then of
    // view 1, ...): the groups of a round then gather from the same source,
    // usually around the same place (neighbouring planes).  Their Eq. 5
    // weights go to tab[hypothesis][view], so that each hypothesis still
    // folds its views in view order.
    float* tab = reinterpret_cast<float*>(pairs + 8 * V);
    const int P = nok * V;
    int count = 0;
    // floor(i / nok) = (i * ceil(2^16 / nok)) >> 16 exactly for i < 2^16 / nok
    // (i < 8 * MVS_MAX_SRC here)
    const uint32_t kmagic = nok ? 0xffffu / (uint32_t)nok + 1u : 0u;
    for (int base = 0; base < P; base += 32) {
        int i = base + lane;
        bool act = i < P;
        int j = act ? (int)(((uint32_t)i * kmagic) >> 16) : 0;
        int cr = act ? i - j * nok : 0;
        int c = __shfl_sync(0xffffffffu, hyp_of, cr);
        float m0 = __shfl_sync(0xffffffffu, my.m0, c);
        float m1 = __shfl_sync(0xffffffffu, my.m1, c);
        float invd = __shfl_sync(0xffffffffu, my.invd, c);
        // the view record as 128-bit words: (wm1, hm1) in word 1, A and b in 2..4
        const float4* vw = reinterpret_cast<const float4*>(sv + j);
        const float4 w1 = vw[1], w2 = vw[2], w3 = vw[3], w4 = vw[4];
        const float A0 = w2.x, A1 = w2.y, A2 = w2.z, A3 = w2.w, A4 = w3.x, A5 = w3.y, A6 = w3.z, A7 = w3.w;
        const float A8 = w4.x, b0 = w4.y, b1 = w4.z, b2 = w4.w;
        float h0z = fmaf(b2, m0, A6), h1z = fmaf(b2, m1, A7);
        float p0z = fmaf(b2, invd, fmaf(A6, x, fmaf(A7, y, A8)));
        // coordinates shifted by -1/2 (tex_sample's convention)
        float h0x = fmaf(-0.5f, h0z, fmaf(b0, m0, A0));
        float h0y = fmaf(-0.5f, h0z, fmaf(b1, m0, A3));
        float h1x = fmaf(-0.5f, h1z, fmaf(b0, m1, A1));
        float h1y = fmaf(-0.5f, h1z, fmaf(b1, m1, A4));
        float p0x = fmaf(-0.5f, p0z, fmaf(b0, invd, fmaf(A0, x, fmaf(A1, y, A2))));
        float p0y = fmaf(-0.5f, p0z, fmaf(b1, invd, fmaf(A3, x, fmaf(A4, y, A5))));
        bool ok = act;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            float cu = (k & 1) ? geo.cu_hi : geo.cu_lo, cv = (k & 2) ? geo.cv_hi : geo.cv_lo;
            float cx = fmaf(cu, h0x, fmaf(cv, h1x, p0x));
            float cy = fmaf(cu, h0y, fmaf(cv, h1y, p0y));
            float cz = fmaf(cu, h0z, fmaf(cv, h1z, p0z));
            float icz = rcp_approx(cz);
            float xs = cx * icz, ys = cy * icz;
            ok = ok && cz > 0.0f && xs >= -0.5f && xs <= w1.z - 0.5f && ys >= -0.5f && ys <= w1.w - 0.5f;
        }
        unsigned m = __ballot_sync(0xffffffffu, ok);
        if (ok) {   // stored with x and y doubled (tex_sample's convention)
            float4* qw = reinterpret_cast<float4*>(pairs + count + __popc(m & ((1u << lane) - 1u)));
            qw[0] = make_float4(2.0f * h0x, 2.0f * h0y, h0z, 2.0f * h1x);
            qw[1] = make_float4(2.0f * h1y, h1z, 2.0f * p0x, 2.0f * p0y);
            qw[2] = make_float4(p0z, 0.0f, __int_as_float(c), __int_as_float(j));
        } else if (act) {
            tab[c * V + j] = 0.0f;   // view excluded for this hypothesis
        }
        count += __popc(m);
    }
    __syncwarp();
    // ---- 2. evaluate the listed pairs, NG at a time
    for (int r = 0; r < count; r += NG) {
        int it = r + grp;
        bool has = it < count;
        const float4* qw = reinterpret_cast<const float4*>(pairs + (has ? it : 0));
        const float4 qa = qw[0], qb = qw[1], qc = qw[2];
        const float h0x = qa.x, h0y = qa.y, h0z = qa.z, h1x = qa.w;
        const float h1y = qb.x, h1z = qb.y, p0x = qb.z, p0y = qb.w, p0z = qc.x;
        // view words 0 (texels, pitch, toff) and 1 (last texel)
        const uint4 v0 = reinterpret_cast<const uint4*>(sv + __float_as_int(qc.w))[0];
        const uint32_t v_last = reinterpret_cast<const uint4*>(sv + __float_as_int(qc.w))[1].x;
        const uint2* v_tex = reinterpret_cast<const uint2*>(((unsigned long long)v0.y << 32) | v0.x);
        float sa = 0.0f, sb = 0.0f, se = 0.0f;
        float sval[S], c0 = 0.0f;   // mixed precision only: the samples and their shift
        if constexpr (!MIXED) {
            // Sample k at doubled, half-shifted source coordinates (X/Z, Y/Z).
            // One FMA rounds X/Z + 1.5 * 2^24 to the nearest even integer 2i
            // (its bits give i), a second gives U = X/Z - 2i in [-1, 1]
            // rounded once.  The texel index is clamped into the array: the
            // listed window corners lie inside the source, but FP32 positions
            // of other samples of a plane seen almost edge-on by the source
            // need not.
            const uint2* tex = v_tex;
            const uint32_t pitch = v0.z, toff = v0.w, last = v_last;
            // gathers in chunks of up to 8 slots (registers); the intensities
            // are shifted by c0 = the 2 x 2 texel sum at the group's first
            // sample (an intensity of this source patch), which enters through
            // the fp16 coefficient a (one mixed add)
            constexpr int CH = S <= 9 ? S : 8;
            float nc0 = 0.0f, dv[S];
#pragma unroll
            for (int k0 = 0; k0 < S; k0 += CH) {
                uint2 tq[CH];
                float Us[CH], Vs[CH];
#pragma unroll
                for (int kk = 0; kk < CH; ++kk) {
                    const int k = k0 + kk;
                    if (k < S) {
                        const float2 o = OFF_SM ? off_sm[k * G + lg] : make_float2(pw.ou[k], pw.ov[k]);
                        float X = fmaf(o.x, h0x, fmaf(o.y, h1x, p0x));
                        float Y = fmaf(o.x, h0y, fmaf(o.y, h1y, p0y));
                        float Z = fmaf(o.x, h0z, fmaf(o.y, h1z, p0z));
                        float iz = rcp_approx(Z);
                        float tx = fmaf(X, iz, kMagic2), ty = fmaf(Y, iz, kMagic2);
                        Us[kk] = fmaf(X, iz, kMagic2 - tx);
                        Vs[kk] = fmaf(Y, iz, kMagic2 - ty);
                        uint32_t idx = (uint32_t)__float_as_int(ty) * pitch + (uint32_t)__float_as_int(tx) + toff;
                        tq[kk] = __ldg(tex + min(idx, last));
                    }
                }
                if (k0 == 0)
                    nc0 = -__half2float(
                        __ushort_as_half((unsigned short)(__shfl_sync(0xffffffffu, tq[0].x, grp * G) & 0xffffu)));
#pragma unroll
                for (int kk = 0; kk < CH; ++kk) {
                    const int k = k0 + kk;
                    if (k < S) {
                        const __half2 ab = *reinterpret_cast<const __half2*>(&tq[kk].x);
                        const __half2 cd = *reinterpret_cast<const __half2*>(&tq[kk].y);
                        const float am = add_f16_f32(__low2half(ab), nc0);
                        dv[k] = fmaf(Vs[kk], fmaf(Us[kk], __high2float(cd), __low2float(cd)),
                                     fmaf(Us[kk], __high2float(ab), am));
                        sa = fmaf(pw.w[k], dv[k], sa);
                        se = fmaf(pw.wr[k], dv[k], se);
                    }
                }
            }
            // two-pass weighted variance (the form of Eq. 4): the weighted
            // mean first, then the centred second moment
            sa = gsum<G>(sa);
            const float mu = sa * geo.inv_wsum;
#pragma unroll
            for (int k = 0; k < S; ++k) {
                const float e = dv[k] - mu;
                sb = fmaf(pw.w[k] * e, e, sb);
            }
        } else {
            const uint2* tex = v_tex;
            const uint32_t pitch = v0.z, toff = v0.w, last = v_last;
            // mixed precision: positions and fractions in FP32 (as above), the
            // bilinear interpolation of two samples per half2 instruction, on
            // intensities shifted by the reference patch mean
            const __half2 mu2 = __float2half2_rn(pw.mean);
#pragma unroll
            for (int k = 0; k < S; k += 2) {
                float Us[2], Vs[2];
                uint2 q[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int kk = k + h < S ? k + h : k;
                    const float2 o = OFF_SM ? off_sm[kk * G + lg] : make_float2(pw.ou[kk], pw.ov[kk]);
                    float X = fmaf(o.x, h0x, fmaf(o.y, h1x, p0x));
                    float Y = fmaf(o.x, h0y, fmaf(o.y, h1y, p0y));
                    float Z = fmaf(o.x, h0z, fmaf(o.y, h1z, p0z));
                    float iz = rcp_approx(Z);
                    float tx = fmaf(X, iz, kMagic2), ty = fmaf(Y, iz, kMagic2);
                    Us[h] = fmaf(X, iz, kMagic2 - tx);
                    Vs[h] = fmaf(Y, iz, kMagic2 - ty);
                    uint32_t idx = (uint32_t)__float_as_int(ty) * pitch + (uint32_t)__float_as_int(tx) + toff;
                    q[h] = __ldg(tex + min(idx, last));
                }
                uint32_t ab = __byte_perm(q[0].x, q[1].x, 0x5410), bb = __byte_perm(q[0].x, q[1].x, 0x7632);
                uint32_t cb = __byte_perm(q[0].y, q[1].y, 0x5410), db = __byte_perm(q[0].y, q[1].y, 0x7632);
                __half2 A = __hsub2(*reinterpret_cast<__half2*>(&ab), mu2);
                __half2 B = *reinterpret_cast<__half2*>(&bb), Cc = *reinterpret_cast<__half2*>(&cb);
                __half2 D = *reinterpret_cast<__half2*>(&db);
                __half2 U2 = __floats2half2_rn(Us[0], Us[1]), V2 = __floats2half2_rn(Vs[0], Vs[1]);
                float2 s2 = __half22float2(__hfma2(V2, __hfma2(U2, D, Cc), __hfma2(U2, B, A)));
                sval[k] = s2.x;
                if (k + 1 < S) sval[k + 1] = s2.y;
            }
            // weighted moments in one pass, shifted by the group's first
            // sample (an intensity of this source patch): with d = s - c0,
            // sum w (s - mu)^2 = sum w d^2 - (sum w d)^2 / W; near the flat
            // limit the denominator is recomputed in FP64 below
            c0 = __shfl_sync(0xffffffffu, sval[0], grp * G);
#pragma unroll
            for (int k = 0; k < S; ++k) {
                float dv = sval[k] - c0;
                float t = pw.w[k] * dv;
                sa += t;
                sb = fmaf(t, dv, sb);
                se = fmaf(pw.wr[k], dv, se);
            }
        }
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) {
            if constexpr (MIXED) sa += __shfl_xor_sync(0xffffffffu, sa, o);
            sb += __shfl_xor_sync(0xffffffffu, sb, o);
            se += __shfl_xor_sync(0xffffffffu, se, o);
        }
        const float mean_d = sa * geo.inv_wsum;
        // sum w (s - mu)^2 (FP32: already centred; mixed: one-pass, shifted)
        float sdd = MIXED ? fmaf(-mean_d, sa, sb) : sb;
        // sum w r' (s - mu) = sum w r' d - mu_d sum w r'
        const float srd = fmaf(-mean_d, geo.wr_sum, se);
        if constexpr (MIXED) {
            // a source patch near the flat limit (where the exclusion decision
            // is taken): recompute the variance denominator in FP64
            const bool near_flat = sdd < 2.0f * kTauVar * geo.wsum && sdd > 0.5f * kTauVar * geo.wsum;
            if (__any_sync(0xffffffffu, near_flat)) {
                const double mu_d = (double)c0 + (double)sa / (double)geo.wsum;
                double v = 0.0;
#pragma unroll
                for (int k = 0; k < S; ++k) {
                    double dd = (double)sval[k] - mu_d;
                    v = fma((double)pw.w[k] * dd, dd, v);
                }
#pragma unroll
                for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (near_flat) sdd = (float)v;
            }
        }
        // ZNCC, C(x, j) = 1 - Z, and its Eq. 5 weight (all lanes compute,
        // the group's first lane stores)
        const bool flat = !(sdd >= kTauVar * geo.wsum);
        const float z = fminf(1.0f, fmaxf(-1.0f, srd * rsqrtf(geo.srr * sdd)));
        const float cj = flat ? kCmax : fminf(1.0f - z, kCmax);
        if (has && lg == 0) {
            if (VIEWS) pairs[it].res = cj;
            tab[__float_as_int(qc.z) * V + __float_as_int(qc.w)] = cj < kCmax ? rcp_approx(fmaxf(cj, kEpsC)) : 0.0f;
            n_evals++;
        }
    }
    __syncwarp();
    // ---- 3. fold hypothesis `lane`'s views in view order
    int cnt = 0;
    float inv_sum = 0.0f;
    if ((okm >> lane) & 1u)
        for (int j = 0; j < V; ++j) {
            const float wv = tab[lane * V + j];
            cnt += wv > 0.0f;
            inv_sum += wv;
        }
    if (VIEWS && view_cost) {
        if (lane < V) view_cost[lane] = kCmax;
        __syncwarp();
        for (int p = lane; p < count; p += 32) view_cost[pairs[p].j] = pairs[p].res;
    }
    __syncwarp();
    return (lane < nc && my.ok && cnt > 0) ? (float)cnt * rcp_approx(inv_sum) : kCmax;
}

// adds the warp's evaluated (pixel, hypothesis, view) count to the counter
__device__ __forceinline__ void flush_evals(unsigned long long* counter, unsigned n) {
    unsigned t = __reduce_add_sync(0xffffffffu, n);
    if (counter && (threadIdx.x & 31) == 0 && t) atomicAdd(counter, (unsigned long long)t);
}

// index of the lowest cost among lanes 0..nc-1 (lowest lane on a tie); costs
// of the other lanes are ignored
__device__ __forceinline__ int warp_argmin(float cost, int nc, float& best) {
    const int lane = threadIdx.x & 31;
    float c = lane < nc ? cost : 3.0e38f;
    int i = lane;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        float oc = __shfl_xor_sync(0xffffffffu, c, o);
        int oi = __shfl_xor_sync(0xffffffffu, i, o);
        if (oc < c || (oc == c && oi < i)) { c = oc; i = oi; }
    }
    best = c;
    return i;
}

// Sec. III-B: n = (cos t sin p, sin t sin p, cos p), turned to face the camera.
__device__ __forceinline__ void normal_from_angles(float th, float ph, float rx0, float rx1, float rx2, float& n0,
                                                   float& n1, float& n2) {
    float st, ct, sp, cp;
    sincosf(th, &st, &ct);
    sincosf(ph, &sp, &cp);
    n0 = ct * sp;
    n1 = st * sp;
    n2 = cp;
    if (n0 * rx0 + n1 * rx1 + n2 * rx2 > 0.0f) {
        n0 = -n0;
        n1 = -n1;
        n2 = -n2;
    }
}

}  // namespace mvsdev
