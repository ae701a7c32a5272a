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
// given the doubled coordinates 2x = rx + ax, 2y = ry + ay, split into a small
// part (rx, ry) and an even integer (ax, ay) passed as 1.5 * 2^24 + ax (the
// caller folds the shift by 1/2 and the factor 2 into its coordinates).
// Adding the magic number rounds 2x to the nearest even integer 2i in one
// FMA-free add, so U = 2x - 2i lies in [-1, 1] and the bits of the sum give
// i; carrying the large integer part in the magic number keeps rx, and with
// it U, exact to a float ulp of a small number.  The texel index is clamped
// into the array, so any input (even NaN) reads inside the buffer.
__device__ __forceinline__ float tex_sample(const uint2* __restrict__ tex, int pitch, uint32_t n_tex, float rx,
                                            float ry, float mag_x, float mag_y) {
    float tx = __fadd_rn(rx, mag_x), ty = __fadd_rn(ry, mag_y);
    float U = __fadd_rn(rx, __fsub_rn(mag_x, tx));
    float V = __fadd_rn(ry, __fsub_rn(mag_y, ty));
    uint32_t idx = (uint32_t)__float_as_int(ty) * (uint32_t)pitch + (uint32_t)__float_as_int(tx) +
                   (uint32_t)(pitch + 1) * (uint32_t)(1 - kMagic2Bits);
    idx = min(idx, n_tex - 1u);
    uint2 q = __ldg(tex + idx);
    float2 ab = __half22float2(*reinterpret_cast<const __half2*>(&q.x));
    float2 cd = __half22float2(*reinterpret_cast<const __half2*>(&q.y));
    return fmaf(V, fmaf(U, cd.y, cd.x), fmaf(U, ab.y, ab.x));
}

// Error-free transformations (Knuth's TwoSum, the FMA TwoProduct) for the
// double-float evaluation of source positions; the _rn intrinsics keep the
// compiler from contracting or reassociating them.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// (h0 + l0) x + (h1 + l1) y + (h2 + l2) as hi + lo for integers x, y < 2^24:
// the large products and sums are carried exactly, the lo parts and the
// rounding errors are summed in float.
__device__ __forceinline__ void df_affine(float h0, float h1, float h2, float l0, float l1, float l2, float x,
                                          float y, float& hi, float& lo) {
    const float p0 = __fmul_rn(h0, x), e0 = fmaf(h0, x, -p0);
    const float p1 = __fmul_rn(h1, y), e1 = fmaf(h1, y, -p1);
    float s, es, s2, es2;
    two_sum(p0, p1, s, es);
    two_sum(s, h2, s2, es2);
    const float rest = __fadd_rn(__fadd_rn(__fadd_rn(e0, e1), __fadd_rn(es, es2)), fmaf(l0, x, fmaf(l1, y, l2)));
    hi = __fadd_rn(s2, rest);
    lo = __fsub_rn(rest, __fsub_rn(hi, s2));
}

// Numerator of an anchored source coordinate: (g - a gz) + (B - a Bz) / d,
// for g, gz, B, Bz given as hi + lo, an integer a (|a| < 2^15) and the
// depth d with invd ~ 1/d.  g - a gz and B - a Bz are carried exactly as
// sums (TwoProduct, TwoSum); their large parts cancel against each other
// (the anchor sits next to the projection), and B / d is split as q + r / d
// with the exact remainder r = B - q d, so the result is accurate to a few
// ulps of itself.
__device__ __forceinline__ float anchored_num(float gh, float gl, float gzh, float gzl, float Bh, float Bl,
                                              float Bzh, float Bzl, float a, float d, float invd) {
    float s, es, sb, esb;
    const float p = __fmul_rn(a, gzh), ep = fmaf(a, gzh, -p);
    two_sum(gh, -p, s, es);
    const float tl = __fsub_rn(__fadd_rn(__fsub_rn(es, ep), gl), __fmul_rn(a, gzl));
    const float pb = __fmul_rn(a, Bzh), epb = fmaf(a, Bzh, -pb);
    two_sum(Bh, -pb, sb, esb);
    const float bl = __fsub_rn(__fadd_rn(__fsub_rn(esb, epb), Bl), __fmul_rn(a, Bzl));
    const float q = __fmul_rn(sb, invd), r = fmaf(-q, d, sb);
    return __fadd_rn(__fadd_rn(s, q), fmaf(__fadd_rn(r, bl), invd, tl));
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
    __half2 o2[S];        // sample offsets / step: (k_u - r_now, k_v - r_now), exact in fp16 (the first
                          // included sample for padding / excluded samples)
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
    const __half2 o2_pad = __floats2half2_rn((float)ku_lo - half, (float)kv_lo - half);
    const float rcen = exists ? 4.0f * (float)__ldg(rc.img + (long long)py * rc.W + px) : 0.0f;
    const float inv_n = rcp_approx((float)n);   // (k + 1/2) / n stays 1/(2n) away from integers
    float sw = 0.0f, swr = 0.0f;
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const int k = s * G + lg;
        const int kv = (int)(((float)k + 0.5f) * inv_n), ku = k - kv * n;   // exact for k < 2^20
        bool in = exists && k < n * n && ku >= ku_lo && ku <= ku_hi && kv >= kv_lo && kv <= kv_hi;
        const float ku_f = (float)ku - half, kv_f = (float)kv - half;
        float ou = rc.step * ku_f, ov = rc.step * kv_f;
        float r = 0.0f, w = 0.0f;
        if (in) {
            r = tex_sample(rc.tex, rc.pitch, rc.n_tex, fmaf(2.0f, ou, -1.0f), fmaf(2.0f, ov, -1.0f),
                           kMagic2 + 2.0f * (float)px, kMagic2 + 2.0f * (float)py);
            float dc = r - rcen;
            w = __expf(fmaf(rc.sp_coef, ou * ou + ov * ov, rc.col_coef * dc * dc));
        }
        pw.o2[s] = in ? __floats2half2_rn(ku_f, kv_f) : o2_pad;
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

// Source-view constants copied to shared memory once per block (128 bytes,
// read as 16-byte words, and 16 bytes of padding: lanes that read different
// views' records at the same offset then fall on different banks): the
// texture, and the doubled, half-shifted homography rows G and B of
// PairConst with their hi and lo parts.
struct __align__(16) ViewSm {
    const uint2* tex;
    uint32_t pitch;
    float fold_x;         // 2 + 2 alpha: the guard texel and tex_fold's alpha in doubled coordinates
    uint32_t last;        // last texel index pitch (H + 1) - 1
    float fold_y;         // 2 + 2 beta
    float xmax2, ymax2;   // 2 W - 3, 2 H - 3: doubled, half-shifted image bounds
    float gx0, gx1, gy0, gy1;   // G_0, G_1 columns 0 and 1 (hi)
    float gz0, gz1, bxh, byh;   // G_2 columns 0 and 1 (hi); B_0, B_1 (hi)
    float bzh, bxl, byl, bzl;   // B_2 (hi); B (lo)
    float gx2, gy2, gz2, gz2l;  // column 2 of G (hi), G_2 column 2 (lo)
    float gx0l, gx1l, gx2l, gy0l;
    float gy1l, gy2l, gz0l, gz1l;
    float pad_[4];
};

static_assert(sizeof(ViewSm) == 144 && offsetof(ViewSm, pitch) == 8 && offsetof(ViewSm, fold_x) == 12 &&
                  offsetof(ViewSm, last) == 16 && offsetof(ViewSm, fold_y) == 20 && offsetof(ViewSm, xmax2) == 24 &&
                  offsetof(ViewSm, gx0) == 32 &&
                  offsetof(ViewSm, gz0) == 48 && offsetof(ViewSm, bzh) == 64 && offsetof(ViewSm, gx2) == 80 &&
                  offsetof(ViewSm, gx0l) == 96 && offsetof(ViewSm, gy1l) == 112,
              "eval_batch and pix_views read ViewSm as 128-bit words");

__device__ __forceinline__ void load_views(const RefConst& rc, ViewSm* sv) {
    for (int j = threadIdx.x; j < rc.n_src; j += blockDim.x) {
        const PairConst& P = rc.pair[j];
        ViewSm& v = sv[j];
        v.tex = P.tex;
        v.pitch = (uint32_t)P.pitch;
        uint32_t alpha, beta;
        tex_fold(P.pitch, &alpha, &beta);
        v.fold_x = 2.0f + 2.0f * (float)alpha;
        v.fold_y = 2.0f + 2.0f * (float)beta;
        v.last = P.n_tex - 1u;
        v.xmax2 = (float)(2 * P.W - 3);
        v.ymax2 = (float)(2 * P.H - 3);
        v.gx0 = P.Gh[0]; v.gx1 = P.Gh[1]; v.gx2 = P.Gh[2];
        v.gy0 = P.Gh[3]; v.gy1 = P.Gh[4]; v.gy2 = P.Gh[5];
        v.gz0 = P.Gh[6]; v.gz1 = P.Gh[7]; v.gz2 = P.Gh[8];
        v.gx0l = P.Gl[0]; v.gx1l = P.Gl[1]; v.gx2l = P.Gl[2];
        v.gy0l = P.Gl[3]; v.gy1l = P.Gl[4]; v.gy2l = P.Gl[5];
        v.gz0l = P.Gl[6]; v.gz1l = P.Gl[7]; v.gz2l = P.Gl[8];
        v.bxh = P.Bh[0]; v.byh = P.Bh[1]; v.bzh = P.Bh[2];
        v.bxl = P.Bl[0]; v.byl = P.Bl[1]; v.bzl = P.Bl[2];
    }
    __syncthreads();
}

// Per (reference pixel, source view): G x~ of the pixel (the source point at
// infinite depth in doubled, half-shifted homogeneous coordinates) as hi + lo
// floats, computed once per pixel by lane j for view j (48 bytes: lanes
// reading eight different views' records touch eight different bank groups).
struct __align__(16) PixView {
    float gxh, gxl, gyh, gyl;
    float gzh, gzl, pad0_, pad1_;
    float pad2_[4];
};

__device__ __forceinline__ void pix_views(const RefConst& rc, const ViewSm* __restrict__ sv, int px, int py,
                                          PixView* pv) {
    const int j = threadIdx.x & 31;
    if (j < rc.n_src) {
        const float4* w = reinterpret_cast<const float4*>(sv + j);
        const float4 w2 = w[2], w3 = w[3], w5 = w[5], w6 = w[6], w7 = w[7];
        const float x = (float)px, y = (float)py;
        PixView r;
        df_affine(w2.x, w2.y, w5.x, w6.x, w6.y, w6.z, x, y, r.gxh, r.gxl);
        df_affine(w2.z, w2.w, w5.y, w6.w, w7.x, w7.y, x, y, r.gyh, r.gyl);
        df_affine(w3.x, w3.y, w5.z, w7.z, w7.w, w5.w, x, y, r.gzh, r.gzl);
        float4* o = reinterpret_cast<float4*>(pv + j);   // the padding is never read
        o[0] = make_float4(r.gxh, r.gxl, r.gyh, r.gyl);
        o[1] = make_float4(r.gzh, r.gzl, 0.0f, 0.0f);
    }
    __syncwarp();
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
    // approximate reciprocals: 1/d enters the anchored source positions
    // only through a correction term of anchored_num's exact-remainder
    // division, and m only through the window's (small) derivatives
    float inv_rho = c.ok ? rcp_approx(d * nr) : 0.0f;
    c.m0 = k0 * inv_rho;
    c.m1 = k1 * inv_rho;
    c.invd = c.ok ? rcp_approx(d) : 0.0f;
    return c;
}

// One listed (hypothesis, view) pair in shared memory (three 16-byte
// words).  Its source positions are anchored: with (ax, ay) even integers
// next to the doubled, half-shifted projection of the window centre, a
// sample at offset (ou, ov) from the pixel lands at
//   xs2 = ax + (nx + ou j0x + ov j1x) / (pz + ou h0z + ov h1z),
//   ys2 = ay + (ny + ou j0y + ov j1y) / (pz + ou h0z + ov h1z),
// so the float arithmetic per sample works on numbers of the size of the
// window's image, not of the source image.  The record holds the columns
// per sample step, s j0 and s j1 (and s h0z, s h1z), so that a sample at
// (k_u - r_now, k_v - r_now) steps from the pixel multiplies them by its
// step counts directly; it also holds the magic numbers 1.5 * 2^24 +
// (ax, ay) of tex_sample and (hypothesis | view << 8).
struct __align__(16) PairSm {
    float j0x, j0y, h0z, j1x;
    float j1y, h1z, nx, ny;
    float pz, mx, my;
    int cj;
};

static_assert(sizeof(PairSm) == 48 && offsetof(PairSm, j1y) == 16 && offsetof(PairSm, pz) == 32 &&
                  offsetof(PairSm, cj) == 44,
              "eval_batch reads and writes PairSm as 128-bit words");

// Shared-memory bytes of a block: the view table and, per warp, room for
// 8 hypotheses x n_src pairs, their 8 x n_src Eq. 5 weights and the pixel's
// n_src PixView records.
__host__ __device__ constexpr size_t smem_views_bytes(int n_src) {
    return (size_t)n_src * sizeof(ViewSm);
}
__host__ __device__ constexpr size_t smem_warp_bytes(int n_src) {
    return (size_t)8 * n_src * (sizeof(PairSm) + sizeof(float)) + (size_t)n_src * sizeof(PixView);   // 464 n_src
}
__host__ __device__ constexpr size_t smem_block_bytes(int n_src, int warps) {
    return smem_views_bytes(n_src) + (size_t)warps * smem_warp_bytes(n_src);
}
// pair list of warp `warp` in a block's dynamic shared memory
__device__ __forceinline__ PairSm* warp_pairs(unsigned char* smem, int n_src, int warp) {
    return reinterpret_cast<PairSm*>(smem + smem_views_bytes(n_src) + (size_t)warp * smem_warp_bytes(n_src));
}
// the PixView records of warp `warp`'s current pixel
__device__ __forceinline__ PixView* warp_pixviews(unsigned char* smem, int n_src, int warp) {
    return reinterpret_cast<PixView*>(smem + smem_views_bytes(n_src) + (size_t)warp * smem_warp_bytes(n_src) +
                                      (size_t)8 * n_src * (sizeof(PairSm) + sizeof(float)));
}

// Two planes (n, depth at the pixel) equal up to float rounding (1e-6
// relative in depth, 1e-6 per normal component); such planes score the same
// cost to within rounding.
__device__ __forceinline__ bool same_plane(const float4& a, const float4& b) {
    return fabsf(a.w - b.w) <= 1e-6f * b.w && fabsf(a.x - b.x) <= 1e-6f && fabsf(a.y - b.y) <= 1e-6f &&
           fabsf(a.z - b.z) <= 1e-6f;
}

// The anchored homography of one listed pair (PairSm words 0..2 without the
// (hypothesis, view) word).
struct PairGeo {
    float j0x, j0y, h0z, j1x, j1y, h1z, nx, ny, pz, mx, my;
};

// One pass over a group's window samples of a listed pair (S slots per lane).
// Sample k: anchored numerators (X, Y) and depth Z; one FMA adds X/Z to the
// pair's magic number 1.5 * 2^24 + ax, rounding to the nearest even integer
// 2i (its bits give i), a second gives U = ax + X/Z - 2i in [-1, 1] rounded
// once.  The texel index is clamped into the array: the listed window
// corners lie inside the source, but float positions of other samples of a
// plane seen almost edge-on by the source need not.  The bilinear values
// are shifted by c0 = the 2 x 2 texel sum at the pair's anchor, next to the
// image of the window centre (an intensity of this source patch, which
// enters through the fp16 coefficient a in one mixed add): the bilateral
// weights favour samples like the centre, so the weighted mean lies near c0
// and the one-pass moments rarely cancel.
//   CENTRED = false: nc0 = -c0 out; sa, sb, se += sum w d, sum w d^2,
//     sum w r' d over the lane's samples, d = s - c0;
//   CENTRED = true: nc0 in (from the first pass, so every d is the same
//     float); sa += sum w (d - mean_d)^2.
// The gathers run in chunks of up to 8 slots (registers).
template <int G, int S, bool CENTRED, int CH = (S <= 9 ? S : 8)>
__device__ __forceinline__ void window_pass(const PixWin<S>& pw, int grp,
                                            const uint2* __restrict__ tex, uint32_t pitch, uint32_t last,
                                            const PairGeo& g, float& nc0, float mean_d, float& sa, float& sb,
                                            float& se) {
    if (!CENTRED) {
        // the texel at the anchor: X / Z = 0 in the sample formula below
        const uint32_t ia = (uint32_t)__float_as_int(g.my) * pitch + (uint32_t)__float_as_int(g.mx);
        const uint2 qa = __ldg(tex + min(ia, last));
        nc0 = -__half2float(__ushort_as_half((unsigned short)(qa.x & 0xffffu)));
    }
#pragma unroll
    for (int k0 = 0; k0 < S; k0 += CH) {
        uint2 tq[CH];
        float Us[CH], Vs[CH];
#pragma unroll
        for (int kk = 0; kk < CH; ++kk) {
            const int k = k0 + kk;
            if (k < S) {
                const float2 o = __half22float2(pw.o2[k]);
                const float X = fmaf(o.x, g.j0x, fmaf(o.y, g.j1x, g.nx));
                const float Y = fmaf(o.x, g.j0y, fmaf(o.y, g.j1y, g.ny));
                const float Z = fmaf(o.x, g.h0z, fmaf(o.y, g.h1z, g.pz));
                const float iz = rcp_approx(Z);
                const float tx = fmaf(X, iz, g.mx), ty = fmaf(Y, iz, g.my);
                Us[kk] = fmaf(X, iz, g.mx - tx);
                Vs[kk] = fmaf(Y, iz, g.my - ty);
                // (j + 1) pitch + (i + 1) modulo 2^32 (tex_fold)
                const uint32_t idx = (uint32_t)__float_as_int(ty) * pitch + (uint32_t)__float_as_int(tx);
                tq[kk] = __ldg(tex + min(idx, last));
            }
        }
#pragma unroll
        for (int kk = 0; kk < CH; ++kk) {
            const int k = k0 + kk;
            if (k < S) {
                const __half2 ab = *reinterpret_cast<const __half2*>(&tq[kk].x);
                const __half2 cd = *reinterpret_cast<const __half2*>(&tq[kk].y);
                const float am = add_f16_f32(__low2half(ab), nc0);
                const float dv = fmaf(Vs[kk], fmaf(Us[kk], __high2float(cd), __low2float(cd)),
                                      fmaf(Us[kk], __high2float(ab), am));
                if (CENTRED) {
                    const float e = dv - mean_d;
                    sa = fmaf(pw.w[k] * e, e, sa);
                } else {
                    // first and second moments in one pass
                    const float t = pw.w[k] * dv;
                    sa += t;
                    sb = fmaf(t, dv, sb);
                    se = fmaf(pw.wr[k], dv, se);
                }
            }
        }
    }
}

// Mixed-precision form of window_pass: positions, fractions and texel
// indices in FP32 exactly as there, the bilinear value of two slots per
// half2 instruction (fp16 products of the exact fp16 coefficients), moments
// accumulated in FP32.  The coefficient a is shifted by c0 in fp16 (both
// are integers up to 1020, so a - c0 is exact); c0 is the anchor texel's a,
// as in window_pass.
//   MODE 0: nc0 = -c0 out; sa, sb, se += sum w d, sum w d^2, sum w r' d;
//   MODE 1: sa += sum w (d - mean_d)^2 in FP32;
//   MODE 2: sd += the same in FP64 (the variance denominator near the
//           flat-patch limit).
// d is the same value in every mode (the same half2 operations).
template <int G, int S, int MODE, int CH = (S <= 9 ? S : 8)>
__device__ __forceinline__ void window_pass_h2(const PixWin<S>& pw, const uint2* __restrict__ tex, uint32_t pitch,
                                               uint32_t last, const PairGeo& g, float& nc0, float mean_d, float& sa,
                                               float& sb, float& se, double& sd) {
    const uint32_t ia = (uint32_t)__float_as_int(g.my) * pitch + (uint32_t)__float_as_int(g.mx);
    if (MODE == 0) {
        const uint2 qa = __ldg(tex + min(ia, last));
        nc0 = -__half2float(__ushort_as_half((unsigned short)(qa.x & 0xffffu)));
    }
    const __half2 c2 = __float2half2_rn(-nc0);   // exact: an integer <= 1020
#pragma unroll
    for (int k0 = 0; k0 < S; k0 += CH) {
        uint2 tq[CH];
        float Us[CH], Vs[CH];
#pragma unroll
        for (int kk = 0; kk < CH; ++kk) {
            const int k = k0 + kk;
            if (k < S) {
                const float2 o = __half22float2(pw.o2[k]);
                const float X = fmaf(o.x, g.j0x, fmaf(o.y, g.j1x, g.nx));
                const float Y = fmaf(o.x, g.j0y, fmaf(o.y, g.j1y, g.ny));
                const float Z = fmaf(o.x, g.h0z, fmaf(o.y, g.h1z, g.pz));
                const float iz = rcp_approx(Z);
                const float tx = fmaf(X, iz, g.mx), ty = fmaf(Y, iz, g.my);
                Us[kk] = fmaf(X, iz, g.mx - tx);
                Vs[kk] = fmaf(Y, iz, g.my - ty);
                const uint32_t idx = (uint32_t)__float_as_int(ty) * pitch + (uint32_t)__float_as_int(tx);
                tq[kk] = __ldg(tex + min(idx, last));
            }
        }
#pragma unroll
        for (int kk = 0; kk < CH; kk += 2) {
            const int k = k0 + kk;
            if (k < S) {
                const bool two = k + 1 < S;   // compile-time
                const uint2 q0 = tq[kk], q1 = two ? tq[kk + 1] : tq[kk];
                uint32_t ab = __byte_perm(q0.x, q1.x, 0x5410), bb = __byte_perm(q0.x, q1.x, 0x7632);
                uint32_t cb = __byte_perm(q0.y, q1.y, 0x5410), db = __byte_perm(q0.y, q1.y, 0x7632);
                const __half2 A = __hsub2(*reinterpret_cast<__half2*>(&ab), c2);
                const __half2 B = *reinterpret_cast<__half2*>(&bb), C = *reinterpret_cast<__half2*>(&cb);
                const __half2 D = *reinterpret_cast<__half2*>(&db);
                const __half2 U2 = __floats2half2_rn(Us[kk], two ? Us[kk + 1] : Us[kk]);
                const __half2 V2 = __floats2half2_rn(Vs[kk], two ? Vs[kk + 1] : Vs[kk]);
                const float2 dv = __half22float2(__hfma2(V2, __hfma2(U2, D, C), __hfma2(U2, B, A)));
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    if (h == 1 && !two) break;
                    const float d = h ? dv.y : dv.x;
                    const float w = pw.w[k + h];
                    if (MODE == 0) {
                        const float t = w * d;
                        sa += t;
                        sb = fmaf(t, d, sb);
                        se = fmaf(pw.wr[k + h], d, se);
                    } else if (MODE == 1) {
                        const float e = d - mean_d;
                        sa = fmaf(w * e, e, sa);
                    } else {
                        // e and w e rounded once each in FP32; their product
                        // and the sum exact or in FP64
                        const float e = d - mean_d;
                        sd = fma((double)(w * e), (double)e, sd);
                    }
                }
            }
        }
    }
}

// Costs C(x) (Eq. 5) of up to 8 hypotheses of the warp's pixel: lane c < nc
// holds hypothesis c on entry and its cost on return.
//   1. the (hypothesis, view) pairs of the usable hypotheses whose window
//      maps inside the source image (corner test: the image of the window is
//      convex, w > 0 included) are listed in `pairs` (per-warp shared memory,
//      nc * n_src entries) in view-major order, with their anchored
//      homography (PairSm);
//   2. each group of G lanes takes the next pair: S bilinear gathers per
//      lane, the weighted moments in one pass (group reductions; a centred
//      second pass where the one-pass form would cancel); then one lane per
//      pair: ZNCC (Eq. 4), C(x,j) = 1 - Z; a view is excluded when its
//      weighted variance is below 1e-6 on the [0,1] scale (reading);
//   3. lane c folds the per-view results of hypothesis c in view order
//      (Eq. 5, weights 1/max(C, 1e-6)).
// pv: the pixel's PixView records (pix_views).  Must be called by all 32
// lanes with the same nc (warp-uniform); VIEWS (per-view costs out) needs
// nc == 1.
template <int G, int S, bool VIEWS, bool MIXED = false>
__device__ __forceinline__ float eval_batch(const RefConst& rc, const ViewSm* __restrict__ sv, const PixWin<S>& pw,
                                            const WinGeo& geo, const PixView* __restrict__ pv, const Cand& my, int nc,
                                            PairSm* pairs, float* view_cost, unsigned& n_evals) {
    constexpr int NG = 32 / G;
    const int lane = threadIdx.x & 31, lg = lane & (G - 1), grp = lane / G;
    const int V = rc.n_src;
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
    // folds its views in view order; with VIEWS the per-view costs go to
    // row 1 of the same table.
    float* tab = reinterpret_cast<float*>(pairs + 8 * V);
    if (VIEWS) {
        if (lane < V) tab[V + lane] = kCmax;
        __syncwarp();
    }
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
        const float m0 = __shfl_sync(0xffffffffu, my.m0, c);
        const float m1 = __shfl_sync(0xffffffffu, my.m1, c);
        const float invd = __shfl_sync(0xffffffffu, my.invd, c);
        const float dd = __shfl_sync(0xffffffffu, my.d, c);
        // the view record (ViewSm words 1..4) and the pixel's G x~ for view j
        const float4* vw = reinterpret_cast<const float4*>(sv + j);
        const float4 w1 = vw[1], w2 = vw[2], w3 = vw[3], w4 = vw[4];
        const float4 g0 = reinterpret_cast<const float4*>(pv + j)[0];   // gxh, gxl, gyh, gyl
        const float4 g1 = reinterpret_cast<const float4*>(pv + j)[1];   // gzh, gzl
        // columns of H = A + b m^T (doubled, half-shifted rows) for offsets
        // along x and y, and the window centre's homogeneous depth
        const float h0z = fmaf(w4.x, m0, w3.x), h1z = fmaf(w4.x, m1, w3.y);
        const float h0x = fmaf(w3.z, m0, w2.x), h1x = fmaf(w3.z, m1, w2.y);
        const float h0y = fmaf(w3.w, m0, w2.z), h1y = fmaf(w3.w, m1, w2.w);
        const float pz = fmaf(w4.x, invd, __fadd_rn(g1.x, g1.y));
        // anchors: the centre's doubled coordinates rounded to even integers
        // (clamped, so that a pair rejected below still computes finite values)
        const float ipz = rcp_approx(pz);
        const float xc = fmaf(w3.z, invd, g0.x) * ipz, yc = fmaf(w3.w, invd, g0.z) * ipz;
        const float ax = fminf(fmaxf(__fsub_rn(__fadd_rn(xc, kMagic2), kMagic2), -4.0f), w1.z + 5.0f);
        const float ay = fminf(fmaxf(__fsub_rn(__fadd_rn(yc, kMagic2), kMagic2), -4.0f), w1.w + 5.0f);
        const float nx = anchored_num(g0.x, g0.y, g1.x, g1.y, w3.z, w4.y, w4.x, w4.w, ax, dd, invd);
        const float ny = anchored_num(g0.z, g0.w, g1.x, g1.y, w3.w, w4.z, w4.x, w4.w, ay, dd, invd);
        const float j0x = fmaf(-ax, h0z, h0x), j1x = fmaf(-ax, h1z, h1x);
        const float j0y = fmaf(-ay, h0z, h0y), j1y = fmaf(-ay, h1z, h1y);
        // every corner in front of the source and inside its image:
        // doubled coordinates in [-1, 2W - 3] x [-1, 2H - 3]
        bool ok = act;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            float cu = (k & 1) ? geo.cu_hi : geo.cu_lo, cv = (k & 2) ? geo.cv_hi : geo.cv_lo;
            float cx = fmaf(cu, j0x, fmaf(cv, j1x, nx));
            float cy = fmaf(cu, j0y, fmaf(cv, j1y, ny));
            float cz = fmaf(cu, h0z, fmaf(cv, h1z, pz));
            float icz = rcp_approx(cz);
            float xs = cx * icz, ys = cy * icz;
            ok = ok && cz > 0.0f && xs >= -1.0f - ax && xs <= w1.z - ax && ys >= -1.0f - ay && ys <= w1.w - ay;
        }
        unsigned m = __ballot_sync(0xffffffffu, ok);
        if (ok) {
            float4* qw = reinterpret_cast<float4*>(pairs + count + __popc(m & ((1u << lane) - 1u)));
            // derivatives per sample step (the offsets are in steps)
            const float st = rc.step;
            qw[0] = make_float4(j0x * st, j0y * st, h0z * st, j1x * st);
            qw[1] = make_float4(j1y * st, h1z * st, nx, ny);
            // magic numbers with the anchor, the texture's guard texel and the
            // index fold (tex_fold): bits(ty) pitch + bits(tx) = texel index
            const float fx = reinterpret_cast<const float4*>(sv + j)[0].w;
            qw[2] = make_float4(pz, kMagic2 + (ax + fx), kMagic2 + (ay + w1.y), __int_as_float(c | (j << 8)));
        } else if (act) {
            tab[c * V + j] = 0.0f;   // view excluded for this hypothesis
        }
        count += __popc(m);
    }
    __syncwarp();
    // ---- 2. evaluate the listed pairs, NG at a time: the weighted moments
    // of each pair (group reductions), which the group's first lane writes
    // over the pair's first record word (the record is not read again)
    const float inv_wsum = geo.inv_wsum;
    for (int r = 0; r < count; r += NG) {
        const int it = r + grp;
        const bool has = it < count;
        float4* qw = reinterpret_cast<float4*>(pairs + (has ? it : 0));
        const float4 qa = qw[0], qb = qw[1], qc = qw[2];
        const PairGeo pg{qa.x, qa.y, qa.z, qa.w, qb.x, qb.y, qb.z, qb.w, qc.x, qc.y, qc.z};
        const int cj = __float_as_int(qc.w), pj = cj >> 8;
        // view words 0 (texels, pitch) and 1 (last texel)
        const uint4 v0 = reinterpret_cast<const uint4*>(sv + pj)[0];
        const uint32_t v_last = reinterpret_cast<const uint4*>(sv + pj)[1].x;
        const uint2* v_tex = reinterpret_cast<const uint2*>(((unsigned long long)v0.y << 32) | v0.x);
        float sa = 0.0f, sb = 0.0f, se = 0.0f, sdd, mean_d;
        if constexpr (!MIXED) {
            float nc0 = 0.0f;
            window_pass<G, S, false>(pw, grp, v_tex, v0.z, v_last, pg, nc0, 0.0f, sa, sb, se);
#pragma unroll
            for (int o = G / 2; o > 0; o >>= 1) {
                sa += __shfl_xor_sync(0xffffffffu, sa, o);
                sb += __shfl_xor_sync(0xffffffffu, sb, o);
                se += __shfl_xor_sync(0xffffffffu, se, o);
            }
            mean_d = sa * inv_wsum;
            // sum w (s - mu)^2 = sum w d^2 - mu_d sum w d (one pass)
            sdd = fmaf(-mean_d, sa, sb);
            // when the shift lies far from the patch mean, W mu_d^2 > 8 sum
            // w (d - mu_d)^2, the one-pass form loses bits to cancellation:
            // the samples are taken again for the centred second moment (the
            // two-pass form of Eq. 4)
            const bool centre = has && sa * mean_d > 8.0f * sdd;
            if (__any_sync(0xffffffffu, centre)) {
                float s2 = 0.0f, u0 = 0.0f, u1 = 0.0f;
                window_pass<G, S, true>(pw, grp, v_tex, v0.z, v_last, pg, nc0, mean_d, s2, u0,
                                                u1);
                s2 = gsum<G>(s2);
                if (centre) sdd = s2;
            }
        } else {
            float nc0 = 0.0f;
            {
                double unused = 0.0;
                window_pass_h2<G, S, 0>(pw, v_tex, v0.z, v_last, pg, nc0, 0.0f, sa, sb, se, unused);
            }
#pragma unroll
            for (int o = G / 2; o > 0; o >>= 1) {
                sa += __shfl_xor_sync(0xffffffffu, sa, o);
                sb += __shfl_xor_sync(0xffffffffu, sb, o);
                se += __shfl_xor_sync(0xffffffffu, se, o);
            }
            mean_d = sa * inv_wsum;
            sdd = fmaf(-mean_d, sa, sb);
            // the shift far from the patch mean: the centred second moment in
            // FP32 from a second gather pass, as in the FP32 path
            const bool centre = has && sa * mean_d > 8.0f * sdd;
            if (__any_sync(0xffffffffu, centre)) {
                float s2 = 0.0f, u0 = 0.0f, u1 = 0.0f;
                double unused = 0.0;
                window_pass_h2<G, S, 1>(pw, v_tex, v0.z, v_last, pg, nc0, mean_d, s2, u0, u1, unused);
                s2 = gsum<G>(s2);
                if (centre) sdd = s2;
            }
            // a source patch within 1 % of the flat limit (where the exclusion
            // decision is taken): the variance denominator in FP64
            const bool near_flat = has && sdd < 1.01f * kTauVar * geo.wsum && sdd > 0.99f * kTauVar * geo.wsum;
            if (__any_sync(0xffffffffu, near_flat)) {
                double v = 0.0;
                float s0 = 0.0f, u0 = 0.0f, u1 = 0.0f;
                window_pass_h2<G, S, 2, 2>(pw, v_tex, v0.z, v_last, pg, nc0, mean_d, s0, u0, u1, v);
#pragma unroll
                for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (near_flat) sdd = (float)v;
            }
        }
        if (has && lg == 0) qw[0] = make_float4(sdd, se, mean_d, __int_as_float(cj));
    }
    __syncwarp();
    // ---- 2b. per evaluated pair, one per lane: ZNCC (Eq. 4), C(x, j) = 1 - Z
    // and its Eq. 5 weight
    for (int i = lane; i < count; i += 32) {
        const float4 q = reinterpret_cast<const float4*>(pairs + i)[0];
        const int cj = __float_as_int(q.w), pj = cj >> 8, pc = cj & 255;
        // sum w r' (s - mu) = sum w r' d - mu_d sum w r'
        const float srd = fmaf(-q.z, geo.wr_sum, q.y);
        const bool flat = !(q.x >= kTauVar * geo.wsum);
        const float z = fminf(1.0f, fmaxf(-1.0f, srd * rsqrtf(geo.srr * q.x)));
        const float cjv = flat ? kCmax : fminf(1.0f - z, kCmax);
        if (VIEWS) tab[V + pj] = cjv;
        tab[pc * V + pj] = cjv < kCmax ? rcp_approx(fmaxf(cjv, kEpsC)) : 0.0f;
        n_evals++;
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
        __syncwarp();
        if (lane < V) view_cost[lane] = tab[V + lane];
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
