// PatchMatch kernels: texture build, random initialisation, plane-map cost
// and one checkerboard phase (propagation + random refinement).
//   Sec. III-B  random initialisation
//   Sec. III-C  Eq. 4 weighted ZNCC, Eq. 5 aggregation, refinement
//   Sec. III    red-black checkerboard updating
#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <unordered_map>

#include "pm_device.cuh"

using namespace mvsdev;

namespace {

constexpr int kBlock = 128;

// ---------------------------------------------------------------------------
// bilinear-coefficient texture (layout documented in mvs_internal.h)
// ---------------------------------------------------------------------------
__global__ void k_build_texture(const uint8_t* __restrict__ img, int W, int H, int pitch, uint2* __restrict__ tex) {
    long long n = (long long)(W + 1) * (H + 1);
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x) {
        int i = (int)(t % (W + 1)) - 1, j = (int)(t / (W + 1)) - 1;
        int x0 = min(max(i, 0), W - 1), x1 = min(max(i + 1, 0), W - 1);
        int y0 = min(max(j, 0), H - 1), y1 = min(max(j + 1, 0), H - 1);
        float p00 = img[(long long)y0 * W + x0], p01 = img[(long long)y0 * W + x1];
        float p10 = img[(long long)y1 * W + x0], p11 = img[(long long)y1 * W + x1];
        __half2 ab = __floats2half2_rn(p00 + p01 + p10 + p11, (p01 - p00) + (p11 - p10));
        __half2 cd = __floats2half2_rn((p10 - p00) + (p11 - p01), p00 - p01 - p10 + p11);
        uint2 q;
        q.x = *reinterpret_cast<const uint32_t*>(&ab);
        q.y = *reinterpret_cast<const uint32_t*>(&cd);
        tex[(long long)(j + 1) * pitch + (i + 1)] = q;
    }
}

// Per-block shared memory: the source-view table and one pair list per warp.
constexpr int kWarps = kBlock / 32;
// Checkerboard-phase blocks cover a tile of kTileX x kTileY pixels of the
// active colour, one warp per pixel, so that the warps sharing an SM's L1
// gather overlapping windows.  20 warps at 96 registers a thread hide more
// gather latency than 16 at 128 (4 % less time per phase at 3072 x 2048
// with 11 x 11 samples; 12, 21 and 24 warps were slower), and a tall tile
// of 2 x 10 warps (4 x 10 pixels) shares more of the L1 than 4 x 5 (4 %
// less again; 10 x 2 and 5 x 4 were slower, 1 x 20 the same).
#ifndef MVS_TILE_X
#define MVS_TILE_X 2
#endif
#ifndef MVS_TILE_Y
#define MVS_TILE_Y 10
#endif
// Windows of 16 slots per lane need more than 128 registers: their blocks
// keep to one row of kTileX pixels (12 warps per SM).
template <int S>
struct PhaseTile {
    static constexpr int TX = MVS_TILE_X;
    static constexpr int TY = S >= 16 ? 1 : MVS_TILE_Y;
    static constexpr int WARPS = TX * TY;
    static constexpr int BLOCK = 32 * WARPS;
    static constexpr int MIN_BLOCKS = (S >= 16 ? 384 : 512) / BLOCK > 0 ? (S >= 16 ? 384 : 512) / BLOCK : 1;
};

// Blocks of the one-hypothesis kernels per SM: 5 (96 registers, no spills)
// for windows of up to 9 slots per lane; 16 slots need more registers.
template <int S>
constexpr int one_hyp_blocks() { return S >= 16 ? 1 : 5; }

// ---------------------------------------------------------------------------
// Sec. III-B: random initialisation, then the cost of the initial plane.
// One warp per pixel, grid-stride over the pixels.
// ---------------------------------------------------------------------------
template <int G, int S, bool MIXED>
__global__ void __launch_bounds__(kBlock, one_hyp_blocks<S>()) k_init(const __grid_constant__ RefConst rc, float* view_cost) {
    extern __shared__ __align__(16) unsigned char smem[];
    ViewSm* views = reinterpret_cast<ViewSm*>(smem);
    load_views(rc, views);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long npix = (long long)rc.W * rc.H;
    unsigned nev = 0;
    for (long long a = (long long)blockIdx.x * kWarps + warp; a < npix; a += (long long)gridDim.x * kWarps) {
        const int px = (int)(a % rc.W), py = (int)(a / rc.W);
        PixWin<S> pw;
        build_window<G, S>(rc, px, py, true, pw);
        float u[3];
        draws3(rc, a, -1, u);
        float d = rc.d_lo + (rc.d_hi - rc.d_lo) * u[0];
        if (rc.init_range) {   // Sec. III-B: a depth between the nearest sparse features
            const float2 r = rc.init_range[a];
            if (r.x == r.x) d = r.x + (r.y - r.x) * u[0];
        }
        float th = 2.0f * kPi * u[1];
        float ph = kPi * (u[2] - 0.5f);
        float n0, n1, n2;
        normal_from_angles(th, ph, pw.geo.rx0, pw.geo.rx1, pw.geo.rx2, n0, n1, n2);
        float* vc = view_cost ? view_cost + a * rc.n_src : nullptr;
        float c = kCmax;
        if (pw.ok) {
            PixView* pv = warp_pixviews(smem, rc.n_src, warp);
            pix_views(rc, views, px, py, pv);
            Cand my = make_cand(rc, pw, pw.geo, n0, n1, n2, d, lane == 0);
            c = eval_batch<G, S, true, MIXED>(rc, views, pw, pw.geo, pv, my, 1, warp_pairs(smem, rc.n_src, warp), vc,
                                              nev);
        } else if (vc && lane < rc.n_src) {
            vc[lane] = kCmax;
        }
        if (lane == 0) {
            rc.plane[a] = make_float4(n0, n1, n2, d);
            rc.cost[a] = c;
        }
    }
    flush_evals(rc.eval_counter, nev);
}

// cost of a given plane map
template <int G, int S, bool MIXED>
__global__ void __launch_bounds__(kBlock, one_hyp_blocks<S>()) k_cost(const __grid_constant__ RefConst rc, const float4* __restrict__ plane,
                                                  float* __restrict__ cost, float* view_cost) {
    extern __shared__ __align__(16) unsigned char smem[];
    ViewSm* views = reinterpret_cast<ViewSm*>(smem);
    load_views(rc, views);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long npix = (long long)rc.W * rc.H;
    unsigned nev = 0;
    for (long long a = (long long)blockIdx.x * kWarps + warp; a < npix; a += (long long)gridDim.x * kWarps) {
        const int px = (int)(a % rc.W), py = (int)(a / rc.W);
        PixWin<S> pw;
        build_window<G, S>(rc, px, py, true, pw);
        float4 pl = plane[a];
        float* vc = view_cost ? view_cost + a * rc.n_src : nullptr;
        float c = kCmax;
        if (pw.ok) {
            PixView* pv = warp_pixviews(smem, rc.n_src, warp);
            pix_views(rc, views, px, py, pv);
            Cand my = make_cand(rc, pw, pw.geo, pl.x, pl.y, pl.z, pl.w, lane == 0);
            c = eval_batch<G, S, true, MIXED>(rc, views, pw, pw.geo, pv, my, 1, warp_pairs(smem, rc.n_src, warp), vc,
                                              nev);
        } else if (vc && lane < rc.n_src) {
            vc[lane] = kCmax;
        }
        if (lane == 0) cost[a] = c;
    }
    flush_evals(rc.eval_counter, nev);
}

// ---------------------------------------------------------------------------
// Checkerboard phase.  Reading of the cited (undescribed) sampling pattern:
// eight groups of other-colour neighbours, the member with the lowest stored
// cost of each group is a candidate (first listed wins a tie).
//   groups 0..3: near V-shapes up / down / left / right, six members
//   groups 4..7: far lines up / down / left / right at distances 5, 7, .., 25
// ---------------------------------------------------------------------------
// offset of member k of group g (members past the group's size: any in-range
// shift value, masked by the caller)
__device__ __forceinline__ void group_member(int g, int k, int& dx, int& dy) {
    if (g < 4) {
        k = min(k, 5);
        // up-pointing V {(0,-1), (-1,-2), (1,-2), (-2,-3), (0,-3), (2,-3)},
        // packed 3 bits per member (x + 2, y + 3), rotated per group
        const int a = (int)((0x220CAu >> (3 * k)) & 7u) - 2;   // x + 2: 2, 1, 3, 0, 2, 4
        const int b = (int)((0x4Au >> (3 * k)) & 7u) - 3;      // y + 3: 2, 1, 1, 0, 0, 0
        switch (g) {
            case 0: dx = a; dy = b; break;
            case 1: dx = a; dy = -b; break;
            case 2: dx = b; dy = a; break;
            default: dx = -b; dy = a; break;
        }
    } else {
        const int dist = 5 + 2 * k;
        dx = g == 6 ? -dist : (g == 7 ? dist : 0);
        dy = g == 4 ? -dist : (g == 5 ? dist : 0);
    }
}

// Member of group g with the lowest stored cost (in-image members only, the
// first listed wins a tie), as a pixel index on lane g < 8, or -1.  The 8
// groups x 16 member slots are spread over 4 registers of the warp (register
// r, lane l: group 2r + l / 16, member l % 16), each half warp takes the
// minimum of its register, and the lowest member holding it wins; stored
// costs are >= 0, so their bit patterns order like the values.  The members
// have the other colour, which this phase does not write.
__device__ __forceinline__ int best_members(const RefConst& rc, int px, int py, int& member) {
    const int lane = threadIdx.x & 31, half = lane >> 4, k = lane & 15;
    unsigned first[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int g = 2 * r + half;
        int dx, dy;
        group_member(g, k, dx, dy);
        const int x2 = px + dx, y2 = py + dy;
        const bool in = k < (g < 4 ? 6 : 11) && x2 >= 0 && x2 < rc.W && y2 >= 0 && y2 < rc.H;
        const unsigned bits = in ? __float_as_uint(__ldg(rc.cost + (long long)y2 * rc.W + x2) + 0.0f) : 0xffffffffu;
        const unsigned mn0 = __reduce_min_sync(0xffffffffu, half ? 0xffffffffu : bits);
        const unsigned mn1 = __reduce_min_sync(0xffffffffu, half ? bits : 0xffffffffu);
        first[r] = __ballot_sync(0xffffffffu, in && bits == (half ? mn1 : mn0));
    }
    int q = -1;
    member = -1;
    if (lane < 8) {
        const int g = lane;
        const unsigned m = (first[g >> 1] >> (16 * (g & 1))) & 0xffffu;
        if (m) {
            int dx, dy;
            member = __ffs(m) - 1;
            group_member(g, member, dx, dy);
            q = (py + dy) * rc.W + px + dx;
        }
    }
    return q;
}

// Refinement perturbations of one pixel, drawn ahead for the next 32 pixels
// of a warp (one lane each): delta_d, and cos / sin of delta_theta and of
// delta_phi.  20 bytes per pixel, after the pair lists; then each warp's
// PhaseWarp record.
// Per-warp state of the current pixel kept in shared memory rather than in
// registers through the evaluation rounds: its window geometry, its plane and
// cost so far, and the hypothesis each lane proposes in the current stage.
struct __align__(16) PhaseWarp {
    WinGeo geo;
    float4 cur;
    float cur_c, pad_[3];
    float4 hyp[8];     // the stage's hypotheses (at most 8: propagation groups, proposals, refinement)
};
// Shared memory of a phase block (the same for both precisions).
__host__ __device__ constexpr size_t phase_smem_bytes(int n_src, int warps, bool mixed) {
    return (void)mixed,
           smem_block_bytes(n_src, warps) + (size_t)warps * (32 * (sizeof(float4) + sizeof(float)) + sizeof(PhaseWarp));
}

// Rows of warps of a phase block: PhaseTile<S>::TY, or fewer when the
// block's pair lists (which grow with the number of sources) would exceed the
// per-block shared memory.
// The limit is a property of the current device (queried once per device;
// a failed query leaves 48 KB, the limit without the opt-in).
int max_block_smem() {
    static std::atomic<int> bytes[128];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) return 48 * 1024;
    int v = bytes[dev].load();
    if (v == 0) {
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess || v <= 0)
            return 48 * 1024;
        bytes[dev].store(v);
    }
    return v;
}
template <int S>
int phase_rows(int n_src, bool mixed) {
    int ty = PhaseTile<S>::TY;
    while (ty > 1 && phase_smem_bytes(n_src, PhaseTile<S>::TX * ty, mixed) > (size_t)max_block_smem()) --ty;
    return ty;
}

// Tiles are visited in super-tiles of 8 x 16 tiles so that the pixels in
// flight at once form a compact region (a smaller source footprint in L2;
// within a phase the order of the pixels does not change the result).
// Pixel of the active colour that warp `warp` takes in tile t, or -1.
template <int TX>
__device__ __forceinline__ long long phase_pixel(const RefConst& rc, long long t, int warp, int color, int TY,
                                                 int& px, int& py) {
    constexpr int kSTX = 8, kSTY = 16;
    const int Wa = (rc.W + 1) >> 1;
    const int ntx = (Wa + TX - 1) / TX, nty = (rc.H + TY - 1) / TY;
    const int nstx = (ntx + kSTX - 1) / kSTX;
    const int sti = (int)(t / (kSTX * kSTY)), r = (int)(t % (kSTX * kSTY));
    const int tx = (sti % nstx) * kSTX + r % kSTX, ty = (sti / nstx) * kSTY + r / kSTX;
    const int ax = tx * TX + warp % TX;
    py = ty * TY + warp / TX;
    px = 2 * ax + ((py + color) & 1);
    if (tx >= ntx || ty >= nty || ax >= Wa || py >= rc.H || px >= rc.W) return -1;
    return (long long)py * rc.W + px;
}

template <int G, int S, bool MIXED>
__global__ void __launch_bounds__(PhaseTile<S>::BLOCK, PhaseTile<S>::MIN_BLOCKS)
    k_phase(const __grid_constant__ RefConst rc, int phase) {
    // the block is kTileX x kTileY warps, kTileY <= PhaseTile<S>::TY chosen by
    // the host so that the block's shared memory fits
    constexpr int kTileX = PhaseTile<S>::TX;
    const int kTileY = (int)(blockDim.x >> 5) / kTileX;
    const int kWarpsB = kTileX * kTileY;
    extern __shared__ __align__(16) unsigned char smem[];   // phase_smem_bytes(n_src, kWarpsB, MIXED)
    ViewSm* views = reinterpret_cast<ViewSm*>(smem);
    load_views(rc, views);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int color = phase & 1;
    float4* draw4 = reinterpret_cast<float4*>(smem + smem_block_bytes(rc.n_src, kWarpsB)) + warp * 32;
    float* draw1 = reinterpret_cast<float*>(reinterpret_cast<float4*>(smem + smem_block_bytes(rc.n_src, kWarpsB)) +
                                            kWarpsB * 32) + warp * 32;
    PhaseWarp* ws = reinterpret_cast<PhaseWarp*>(smem + smem_block_bytes(rc.n_src, kWarpsB) +
                                                 (size_t)kWarpsB * 32 * (sizeof(float4) + sizeof(float))) + warp;
    const int Wa = (rc.W + 1) >> 1;
    const int ntx = (Wa + kTileX - 1) / kTileX, nty = (rc.H + kTileY - 1) / kTileY;
    const int nstx = (ntx + 7) / 8, nsty = (nty + 15) / 16;
    const long long ntiles = (long long)nstx * nsty * (8 * 16);
    unsigned nev = 0, it = 0;
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
        if ((it & 31u) == 0) {
            // refinement perturbations (Sec. III-C) of this warp's next 32
            // pixels, one per lane: delta_d in [-d_hi/4, d_hi/4],
            // delta_theta in [-pi/2, pi/2], delta_phi in [-pi/12, pi/12]
            int qx, qy;
            const long long q = phase_pixel<kTileX>(rc, t + (long long)lane * gridDim.x, warp, color, kTileY, qx, qy);
            float u[3];
            draws3(rc, q < 0 ? 0 : q, phase, u);
            float sdt, cdt, sdp, cdp;
            sincosf((2.0f * u[1] - 1.0f) * (kPi * 0.5f), &sdt, &cdt);
            sincosf((2.0f * u[2] - 1.0f) * (kPi / 12.0f), &sdp, &cdp);
            __syncwarp();
            draw4[lane] = make_float4((2.0f * u[0] - 1.0f) * (rc.d_hi * 0.25f), cdt, sdt, cdp);
            draw1[lane] = sdp;
            __syncwarp();
        }
        int px, py;
        const long long pix = phase_pixel<kTileX>(rc, t, warp, color, kTileY, px, py);
        if (pix < 0) continue;   // warp-uniform
        PixWin<S> pw;
        build_window<G, S>(rc, px, py, true, pw);
        if (!pw.ok) continue;                           // flat patch: every hypothesis costs C_max
        // the window geometry and the pixel's state wait in shared memory
        // (fewer live registers through the evaluation rounds)
        __syncwarp();
        if (lane == 0) {
            ws->geo = pw.geo;
            ws->cur = rc.plane[pix];
            ws->cur_c = rc.cost[pix];
        }
        PixView* pv = warp_pixviews(smem, rc.n_src, warp);
        pix_views(rc, views, px, py, pv);   // (ends with a warp barrier)
        const WinGeo& geo = ws->geo;

        // ---- propagation: lane g < 8 takes group g's cheapest member and
        // carries its plane over
        int member;
        const int q = best_members(rc, px, py, member);
        // candidate memo: group g's (member, plane generation) now and at this
        // pixel's last visit in this call; an unchanged one was scored then
        uint32_t key = 0xfffffffeu;
        bool repeat = false;
        if (lane < 8) {
            if (q >= 0) key = ((uint32_t)member << 28) | (__ldg(rc.gen + q) & 0x0fffffffu);
            repeat = q >= 0 && key == rc.memo[pix * MVS_MEMO_WORDS + lane];
        }
        float4 np = make_float4(0.f, 0.f, -1.f, 1.f);
        float d = 0.0f;
        bool ok = q >= 0;
        if (ok) {
            // the neighbour's plane carried over as a plane (reading)
            np = rc.plane[q];
            int x2 = q % rc.W, y2 = q / rc.W;
            const float* Ki = rc.Kinv;
            float r0 = fmaf(Ki[0], (float)x2, fmaf(Ki[1], (float)y2, Ki[2]));
            float r1 = fmaf(Ki[3], (float)x2, fmaf(Ki[4], (float)y2, Ki[5]));
            float r2 = fmaf(Ki[6], (float)x2, fmaf(Ki[7], (float)y2, Ki[8]));
            float rho = np.w * (np.x * r0 + np.y * r1 + np.z * r2);
            float den = np.x * geo.rx0 + np.y * geo.rx1 + np.z * geo.rx2;
            ok = den < 0.0f;
            d = ok ? rho * rcp_approx(den) : 0.0f;
            ok = ok && d >= rc.d_lo && d <= rc.d_hi;
        }
        // A carried-over plane equal (to float rounding) to the pixel's own
        // plane or to an earlier group's plane scores the same cost, so it
        // cannot be strictly cheaper than that plane: it is not evaluated.
        {
            const float4 mine = make_float4(np.x, np.y, np.z, d);
            bool dup = ok && same_plane(mine, ws->cur);
#pragma unroll
            for (int g2 = 0; g2 < 7; ++g2) {
                const float4 o = make_float4(__shfl_sync(0xffffffffu, np.x, g2), __shfl_sync(0xffffffffu, np.y, g2),
                                             __shfl_sync(0xffffffffu, np.z, g2), __shfl_sync(0xffffffffu, d, g2));
                const bool ook = __shfl_sync(0xffffffffu, (int)ok, g2) != 0;
                dup = dup || (ok && ook && lane > g2 && same_plane(mine, o));
            }
            ok = ok && !dup;
        }
        ok = ok && !repeat;
        // stage 0: the eight propagated planes; stage 1: the learned
        // proposals of this pixel (when given); stage 2: the three refinement
        // candidates built from the state after stages 0 and 1.  One call
        // site keeps a single copy of the evaluation in the instruction cache.
        float4 hyp4 = make_float4(np.x, np.y, np.z, d);
        bool want = ok;
        bool changed = false;
#pragma unroll 1
        for (int stage = 0; stage < 3; ++stage) {
            if (stage == 1) {
                if (rc.n_prop == 0) continue;
                // proposals already scored at this pixel in this call (the
                // memo word holds the complement of their mask)
                const uint32_t scored = ~rc.memo[pix * MVS_MEMO_WORDS + 8];
                const bool has = lane < rc.n_prop;
                hyp4 = has ? rc.props[pix * rc.n_prop + lane] : make_float4(0.f, 0.f, -1.f, 0.f);
                want = has && !((scored >> lane) & 1u) && hyp4.w >= rc.d_lo && hyp4.w <= rc.d_hi &&
                       !same_plane(hyp4, ws->cur);
            } else if (stage == 2) {
                const float4 cur = ws->cur;
                // refinement (Sec. III-C): d + delta_d clamped to the range;
                // the normal's angles theta = atan2(m1, m0), phi = acos(m2)
                // (after flipping to m2 >= 0) move by delta_theta, delta_phi,
                // taken through the angle-addition formulas
                const float4 r4 = draw4[it & 31u];
                const float sdp = draw1[it & 31u];
                float d_new = fminf(fmaxf(cur.w + r4.x, rc.d_lo), rc.d_hi);
                float m0 = cur.x, m1 = cur.y, m2 = cur.z;
                if (m2 < 0.0f) { m0 = -m0; m1 = -m1; m2 = -m2; }
                const float rr = sqrtf(m0 * m0 + m1 * m1);
                // cos / sin of atan2(m1, m0); atan2(+-0, x) is 0 for x = +0 and pi for x = -0
                const float irr = rr > 0.0f ? 1.0f / rr : 0.0f;
                const float ct = rr > 0.0f ? m0 * irr : (signbit(m0) ? -1.0f : 1.0f), st = m1 * irr;
                const float cp = fminf(1.0f, fmaxf(-1.0f, m2)), sp = sqrtf(fmaxf(0.0f, 1.0f - cp * cp));
                const float ct2 = ct * r4.y - st * r4.z, st2 = st * r4.y + ct * r4.z;
                const float cp2 = cp * r4.w - sp * sdp, sp2 = sp * r4.w + cp * sdp;
                float nn0 = ct2 * sp2, nn1 = st2 * sp2, nn2 = cp2;
                if (nn0 * geo.rx0 + nn1 * geo.rx1 + nn2 * geo.rx2 > 0.0f) {   // face the camera
                    nn0 = -nn0;
                    nn1 = -nn1;
                    nn2 = -nn2;
                }
                // candidates (d_new, n_old), (d_old, n_new), (d_new, n_new) in lanes 0..2
                hyp4 = lane == 0 ? make_float4(cur.x, cur.y, cur.z, d_new)
                     : (lane == 1 ? make_float4(nn0, nn1, nn2, cur.w) : make_float4(nn0, nn1, nn2, d_new));
                want = lane < 3;
            }
            const int nc = stage == 0 ? 8 : (stage == 1 ? rc.n_prop : 3);
            if (lane < 8) ws->hyp[lane] = hyp4;
            Cand my = make_cand(rc, pw, geo, hyp4.x, hyp4.y, hyp4.z, hyp4.w, want);
            float c = eval_batch<G, S, false, MIXED>(rc, views, pw, geo, pv, my, nc,
                                                     warp_pairs(smem, rc.n_src, warp), nullptr,
                                                     nev);   // (ends with a warp barrier)
            float bc;
            int bi = warp_argmin(my.ok ? c : 3.0e38f, nc, bc);
            if (bc < ws->cur_c && lane == 0) {
                ws->cur = ws->hyp[bi];
                ws->cur_c = bc;
                changed = true;
            }
            __syncwarp();
        }
        if (lane == 0) {
            rc.plane[pix] = ws->cur;
            rc.cost[pix] = ws->cur_c;
            if (changed) rc.gen[pix] = rc.gen[pix] + 1u;
        }
        if (lane < 8) rc.memo[pix * MVS_MEMO_WORDS + lane] = key;
        if (lane == 8 && rc.n_prop > 0)
            rc.memo[pix * MVS_MEMO_WORDS + 8] = rc.n_prop >= 32 ? 0u : ~((1u << rc.n_prop) - 1u);
    }
    flush_evals(rc.eval_counter, nev);
}

// grid of the grid-stride kernels: as many blocks as fit on the device at
// once (occupancy query, cached per kernel), at most one warp per unit
}  // namespace

namespace {
thread_local cudaError_t t_grid_err = cudaSuccess;
}

// Launch-shape cache per (device, kernel): the SM count, the dynamic shared
// memory opt-in and the occupancy query are all properties of the current
// device.  A failed query leaves grid 0 (the launch then fails) and the
// query's own error for pm_grid_error().
unsigned pm_grid_for(const void* kernel, long long units, size_t smem, int block) {
    static std::mutex mu;
    struct Cfg { size_t smem; int block, per_sm; };
    static std::map<std::pair<int, const void*>, Cfg> cache;
    static std::map<int, int> sms_of;
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        t_grid_err = e;
        return 0;
    }
    {
        std::lock_guard<std::mutex> lk(mu);
        auto si = sms_of.find(dev);
        if (si == sms_of.end()) {
            if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) {
                t_grid_err = e;
                return 0;
            }
            sms_of[dev] = sms;
        } else {
            sms = si->second;
        }
        const auto key = std::make_pair(dev, kernel);
        auto it = cache.find(key);
        if (it != cache.end() && it->second.smem == smem && it->second.block == block) {
            per_sm = it->second.per_sm;
        } else {
            if (smem > 48 * 1024 &&
                (e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
                    cudaSuccess) {
                t_grid_err = e;
                return 0;
            }
            if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, smem)) != cudaSuccess) {
                t_grid_err = e;
                return 0;
            }
            per_sm = std::max(per_sm, 1);
            cache[key] = {smem, block, per_sm};
        }
    }
    long long need = units;   // blocks of work
    long long full = (long long)sms * per_sm;
    return (unsigned)std::max<long long>(1, std::min(need, full));
}

cudaError_t pm_grid_error() {
    const cudaError_t e = t_grid_err;
    t_grid_err = cudaSuccess;
    return e;
}

// the error of the launch-shape queries of this thread, else of the launches
static cudaError_t launch_status() {
    const cudaError_t g = pm_grid_error();
    const cudaError_t l = cudaGetLastError();
    return g != cudaSuccess ? g : l;
}

// Lanes per pixel group (G) and slots per lane (S) for an n x n window:
// G * S >= n * n.  lanes_hint 0 picks the default; 4, 8, 16 or 32 picks G.
// The mixed-precision kernels exist for the default layout of each window
// size only.
#define MVS_DISPATCH_DEFAULT(n, CALL)                                                     \
    do {                                                                                  \
        int _s = (n) * (n);                                                               \
        if (_s <= 16) { CALL(4, 4); }                                                     \
        else if (_s <= 36) { CALL(4, 9); }                                                \
        else if (_s <= 64) { CALL(8, 8); }                                                \
        else if (_s <= 128) { CALL(16, 8); }                                              \
        else if (_s <= 256) { CALL(16, 16); }                                             \
        else { CALL(32, 16); }                                                            \
    } while (0)

#define MVS_DISPATCH(n, hint, CALL)                                                       \
    do {                                                                                  \
        int _s = (n) * (n), _h = (hint);                                                  \
        if (_s <= 16) { CALL(4, 4); }                                                     \
        else if (_s <= 36) { if (_h == 8) { CALL(8, 5); } else { CALL(4, 9); } }          \
        else if (_s <= 64) { if (_h == 16) { CALL(16, 4); } else { CALL(8, 8); } }        \
        else if (_s <= 128) {                                                             \
            if (_h == 8) { CALL(8, 16); } else if (_h == 32) { CALL(32, 4); }             \
            else { CALL(16, 8); }                                                         \
        }                                                                                 \
        else if (_s <= 256) { if (_h == 32) { CALL(32, 8); } else { CALL(16, 16); } }     \
        else { CALL(32, 16); }                                                            \
    } while (0)

// Resolves (and caches) the grid sizes of the init / cost / phase kernels of
// this configuration without launching anything, so that a later stream
// capture contains kernel launches only.
cudaError_t prime_launch_configs(const RefConst& rc) {
    const size_t smem = smem_block_bytes(rc.n_src, kWarps);
#define CALL(G, S)                                                                                    \
    do {                                                                                              \
        pm_grid_for((const void*)k_init<G, S, MX>, 1, smem, kBlock);                                  \
        pm_grid_for((const void*)k_cost<G, S, MX>, 1, smem, kBlock);                                  \
        pm_grid_for((const void*)k_phase<G, S, MX>, 1,                                                \
                    phase_smem_bytes(rc.n_src, PhaseTile<S>::TX * phase_rows<S>(rc.n_src, MX), MX),  \
                    32 * PhaseTile<S>::TX * phase_rows<S>(rc.n_src, MX));                              \
    } while (0)
    if (rc.precision) {
        constexpr bool MX = true;
        MVS_DISPATCH_DEFAULT(rc.n, CALL);
    } else {
        constexpr bool MX = false;
        MVS_DISPATCH(rc.n, rc.lanes_hint, CALL);
    }
#undef CALL
    return launch_status();
}

cudaError_t launch_build_texture(const uint8_t* img, int W, int H, uint2* tex, cudaStream_t s) {
    long long n = (long long)(W + 1) * (H + 1);
    unsigned blocks = (unsigned)std::min<long long>((n + 255) / 256, 152LL * 16);
    k_build_texture<<<blocks, 256, 0, s>>>(img, W, H, tex_pitch(W), tex);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_init(const RefConst& rc, float* view_cost, cudaStream_t s) {
    long long npix = (long long)rc.W * rc.H;
    const size_t smem = smem_block_bytes(rc.n_src, kWarps);
    const unsigned units = (unsigned)((npix + kWarps - 1) / kWarps);
#define CALL(G, S) \
    k_init<G, S, MX><<<pm_grid_for((const void*)k_init<G, S, MX>, units, smem, kBlock), kBlock, smem, s>>>(rc, view_cost)
    if (rc.precision) {
        constexpr bool MX = true;
        MVS_DISPATCH_DEFAULT(rc.n, CALL);
    } else {
        constexpr bool MX = false;
        MVS_DISPATCH(rc.n, rc.lanes_hint, CALL);
    }
#undef CALL
    count_launch();
    return launch_status();
}

cudaError_t launch_cost(const RefConst& rc, const float4* plane, float* cost, float* view_cost, cudaStream_t s) {
    long long npix = (long long)rc.W * rc.H;
    const size_t smem = smem_block_bytes(rc.n_src, kWarps);
    const unsigned units = (unsigned)((npix + kWarps - 1) / kWarps);
#define CALL(G, S)                                                                                         \
    k_cost<G, S, MX><<<pm_grid_for((const void*)k_cost<G, S, MX>, units, smem, kBlock), kBlock, smem, s>>>( \
        rc, plane, cost, view_cost)
    if (rc.precision) {
        constexpr bool MX = true;
        MVS_DISPATCH_DEFAULT(rc.n, CALL);
    } else {
        constexpr bool MX = false;
        MVS_DISPATCH(rc.n, rc.lanes_hint, CALL);
    }
#undef CALL
    count_launch();
    return launch_status();
}

template <int G, int S, bool MX>
void phase_launch(const RefConst& rc, int phase, cudaStream_t s) {
    using T = PhaseTile<S>;
    const int ty = phase_rows<S>(rc.n_src, MX), block = 32 * T::TX * ty;
    const long long ntiles = (long long)(((rc.W + 1) / 2 + T::TX - 1) / T::TX) * ((rc.H + ty - 1) / ty);
    const size_t smem = phase_smem_bytes(rc.n_src, T::TX * ty, MX);
    k_phase<G, S, MX><<<pm_grid_for((const void*)k_phase<G, S, MX>, ntiles, smem, block), block, smem, s>>>(rc,
                                                                                                           phase);
}

cudaError_t launch_memo_reset(const RefConst& rc, cudaStream_t s) {
    return cudaMemsetAsync(rc.memo, 0xff, (size_t)rc.W * rc.H * MVS_MEMO_WORDS * sizeof(uint32_t), s);
}

cudaError_t launch_phase(const RefConst& rc, int phase, cudaStream_t s) {
    if (rc.precision) {
#define CALL(G, S) phase_launch<G, S, true>(rc, phase, s)
        MVS_DISPATCH_DEFAULT(rc.n, CALL);
#undef CALL
    } else {
#define CALL(G, S) phase_launch<G, S, false>(rc, phase, s)
        MVS_DISPATCH(rc.n, rc.lanes_hint, CALL);
#undef CALL
    }
    count_launch();
    return launch_status();
}
