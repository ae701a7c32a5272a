// Geometric-consistency filter (Sec. III-D) and plane hypothesis inference
// (Sec. III-E): four-direction line-fit hypotheses, their matching cost, the
// pairwise MRF of Eq. 6-9 decoded by tree-reweighted message passing at half
// resolution, closest-hypothesis selection and Eq. 10 normals.
#include <cooperative_groups.h>

#include <algorithm>
#include <mutex>

#include "../../include/mvs.h"
#include "pm_device.cuh"

using namespace mvsdev;

namespace {

// ---------------------------------------------------------------------------
// Sec. III-D: geometric consistency.  Reading: the z-depth of X in view j is
// compared with the bilinear depth of view j at x'_j (a tap without depth
// makes the view inconsistent); the normal of view j at the rounded x'_j is
// rotated into the reference frame and compared sign-agnostically; the
// reprojection goes back through d_j(x'_j).  Kept with >= min_consistent.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void mat3v(const float* M, float a, float b, float c, float& o0, float& o1, float& o2) {
    o0 = fmaf(M[0], a, fmaf(M[1], b, M[2] * c));
    o1 = fmaf(M[3], a, fmaf(M[4], b, M[5] * c));
    o2 = fmaf(M[6], a, fmaf(M[7], b, M[8] * c));
}

__global__ void k_geo_filter(const __grid_constant__ FilterConst fc, uint8_t* __restrict__ keep,
                             int32_t* __restrict__ count) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)fc.W * fc.H) return;
    int x = (int)(i % fc.W), y = (int)(i / fc.W);
    float4 pl = fc.plane[i];
    int cnt = 0;
    if (pl.w > 0.0f) {
        float r0, r1, r2;
        mat3v(fc.Kinv, (float)x, (float)y, 1.0f, r0, r1, r2);
        float X0 = pl.w * r0, X1 = pl.w * r1, X2 = pl.w * r2;
        for (int jj = 0; jj < fc.n_src; ++jj) {
            const FilterConst::Src& S = fc.src[jj];
            float Y0, Y1, Y2;
            mat3v(S.R, X0, X1, X2, Y0, Y1, Y2);
            Y0 += S.t[0]; Y1 += S.t[1]; Y2 += S.t[2];
            if (!(Y2 > 0.0f)) continue;
            float q0, q1, q2;
            mat3v(S.K, Y0, Y1, Y2, q0, q1, q2);
            float u = q0 / q2, v = q1 / q2;
            if (!(u >= 0.0f && u <= (float)(S.W - 1) && v >= 0.0f && v <= (float)(S.H - 1))) continue;
            int x0 = (int)floorf(u), y0 = (int)floorf(v);
            int x1 = min(x0 + 1, S.W - 1), y1 = min(y0 + 1, S.H - 1);
            float da = S.plane[(long long)y0 * S.W + x0].w, db = S.plane[(long long)y0 * S.W + x1].w;
            float dc = S.plane[(long long)y1 * S.W + x0].w, de = S.plane[(long long)y1 * S.W + x1].w;
            if (!(da > 0.0f && db > 0.0f && dc > 0.0f && de > 0.0f)) continue;
            float fx = u - (float)x0, fy = v - (float)y0;
            float dj = (1.0f - fy) * ((1.0f - fx) * da + fx * db) + fy * ((1.0f - fx) * dc + fx * de);
            float diff = fabsf(dj - Y2);
            if (fc.depth_relative) diff /= Y2;
            if (!(diff < fc.depth_tol)) continue;
            int xn = min((int)floorf(u + 0.5f), S.W - 1), yn = min((int)floorf(v + 0.5f), S.H - 1);
            float4 nj = S.plane[(long long)yn * S.W + xn];
            // R^T n_j
            float m0 = S.R[0] * nj.x + S.R[3] * nj.y + S.R[6] * nj.z;
            float m1 = S.R[1] * nj.x + S.R[4] * nj.y + S.R[7] * nj.z;
            float m2 = S.R[2] * nj.x + S.R[5] * nj.y + S.R[8] * nj.z;
            float cs = fabsf(pl.x * m0 + pl.y * m1 + pl.z * m2) /
                       sqrtf((pl.x * pl.x + pl.y * pl.y + pl.z * pl.z) * (m0 * m0 + m1 * m1 + m2 * m2));
            if (!(cs > fc.cos_max)) continue;
            float s0, s1, s2;
            mat3v(S.Kinv, u, v, 1.0f, s0, s1, s2);
            float Z0 = dj * s0 - S.t[0], Z1 = dj * s1 - S.t[1], Z2 = dj * s2 - S.t[2];
            float B0 = S.R[0] * Z0 + S.R[3] * Z1 + S.R[6] * Z2;
            float B1 = S.R[1] * Z0 + S.R[4] * Z1 + S.R[7] * Z2;
            float B2 = S.R[2] * Z0 + S.R[5] * Z1 + S.R[8] * Z2;
            if (!(B2 > 0.0f)) continue;
            float e0, e1, e2;
            mat3v(fc.K, B0, B1, B2, e0, e1, e2);
            float eu = e0 / e2 - (float)x, ev = e1 / e2 - (float)y;
            if (!(sqrtf(eu * eu + ev * ev) < fc.max_reproj)) continue;
            cnt++;
        }
    }
    if (count) count[i] = cnt;
    keep[i] = (uint8_t)(pl.w > 0.0f && cnt >= fc.min_consistent);
}

// ---------------------------------------------------------------------------
// Sec. III-E hypotheses.  Direction k: 0 horizontal (1,0), 1 vertical (0,1),
// 2 diagonal 45 deg below (1,1), 3 diagonal 45 deg above (1,-1).  A line of
// direction k is indexed by its first pixel; gap[k][side][p] holds the
// distance in steps from p to the nearest reconstructed pixel strictly
// before (side 0) or after (side 1) p along the line, 0 if there is none.
// ---------------------------------------------------------------------------
__constant__ int c_dir[4][2] = {{1, 0}, {0, 1}, {1, 1}, {1, -1}};

__device__ __forceinline__ int n_lines(int k, int W, int H) { return k == 0 ? H : (k == 1 ? W : W + H - 1); }

// start pixel of line l of direction k
__device__ __forceinline__ void line_start(int k, int l, int W, int H, int& x, int& y) {
    if (k == 0) { x = 0; y = l; }
    else if (k == 1) { x = l; y = 0; }
    else if (k == 2) {          // step (1,1): starts on the left column (bottom up) then the top row
        if (l < H) { x = 0; y = H - 1 - l; } else { x = l - H + 1; y = 0; }
    } else {                    // step (1,-1): starts on the left column then the bottom row
        if (l < H) { x = 0; y = l; } else { x = l - H + 1; y = H - 1; }
    }
}

__global__ void k_line_gaps(int W, int H, const uint8_t* __restrict__ known, int32_t* __restrict__ gaps) {
    const long long N = (long long)W * H;
    int k = blockIdx.y;
    int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= n_lines(k, W, H)) return;
    int sx = c_dir[k][0], sy = c_dir[k][1];
    int x0, y0;
    line_start(k, l, W, H, x0, y0);
    int32_t* before = gaps + (long long)(2 * k) * N;
    int32_t* after = gaps + (long long)(2 * k + 1) * N;
    // forward walk: distance to the previous reconstructed pixel
    int last = -1, t = 0;
    for (int x = x0, y = y0; x >= 0 && x < W && y >= 0 && y < H; x += sx, y += sy, ++t) {
        long long p = (long long)y * W + x;
        before[p] = last >= 0 ? t - last : 0;
        if (known[p]) last = t;
    }
    // backward walk: distance to the next reconstructed pixel
    int len = t;
    last = -1;
    for (int s = len - 1; s >= 0; --s) {
        int x = x0 + s * sx, y = y0 + s * sy;
        long long p = (long long)y * W + x;
        after[p] = last >= 0 ? last - s : 0;
        if (known[p]) last = s;
    }
}

// least-squares line v = a + b t through the n_fit reconstructed pixels
// nearest along the line (negative side first at equal distance), value at
// t = 0; centred normal equations in float
__global__ void k_line_fit(int W, int H, const float* __restrict__ depth, const uint8_t* __restrict__ known,
                           const int32_t* __restrict__ gaps, int n_fit, int inverse, float d_lo, float d_hi,
                           float* __restrict__ hyp, uint8_t* __restrict__ valid) {
    const long long N = (long long)W * H;
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    int x = (int)(i % W), y = (int)(i / W);
    bool hole = !known[i];
    for (int k = 0; k < 4; ++k) {
        float h = 0.0f;
        bool ok = false;
        if (hole) {
            const int32_t* before = gaps + (long long)(2 * k) * N;
            const int32_t* after = gaps + (long long)(2 * k + 1) * N;
            int sx = c_dir[k][0], sy = c_dir[k][1];
            int dl = before[i], dr = after[i];   // distances of the next candidates on each side (0 = none)
            float ts[32], vs[32];
            int m = 0;
            float tsum = 0.0f;
            while (m < n_fit && (dl > 0 || dr > 0)) {
                bool take_left = dl > 0 && (dr == 0 || dl <= dr);
                int dist = take_left ? dl : dr;
                int side = take_left ? -1 : 1;
                long long q = (long long)(y + side * dist * sy) * W + (x + side * dist * sx);
                float dv = depth[q];
                ts[m] = (float)(side * dist);
                vs[m] = inverse ? 1.0f / dv : dv;
                tsum += ts[m];
                m++;
                if (take_left) {
                    int g = before[q];
                    dl = g > 0 ? dl + g : 0;
                } else {
                    int g = after[q];
                    dr = g > 0 ? dr + g : 0;
                }
            }
            if (m >= 2) {
                float tm = tsum / (float)m, vm = 0.0f;
                for (int a = 0; a < m; ++a) vm += vs[a];
                vm /= (float)m;
                float stt = 0.0f, stv = 0.0f;
                for (int a = 0; a < m; ++a) {
                    float dt = ts[a] - tm;
                    stt = fmaf(dt, dt, stt);
                    stv = fmaf(dt, vs[a] - vm, stv);
                }
                float b = stv / stt;
                float av = vm - b * tm;
                h = inverse ? 1.0f / av : av;
                ok = h >= d_lo && h <= d_hi;
            }
        }
        hyp[4 * i + k] = ok ? h : 0.0f;
        valid[4 * i + k] = ok ? 1 : 0;
    }
}

// ---------------------------------------------------------------------------
// hypothesis cost: fronto-parallel plane z = h, n = (0, 0, -1) (Sec. III-E)
// ---------------------------------------------------------------------------
constexpr int kBlock = 128;
constexpr int kWarps = kBlock / 32;

// one warp per pixel, the four hypotheses of a pixel in lanes 0..3
template <int G, int S>
__global__ void __launch_bounds__(kBlock, 3) k_phi_cost(const __grid_constant__ RefConst rc, const float* __restrict__ hyp,
                                                      const uint8_t* __restrict__ valid, float* __restrict__ hcost) {
    extern __shared__ __align__(16) unsigned char smem[];
    ViewSm* views = reinterpret_cast<ViewSm*>(smem);
    load_views(rc, views);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long npix = (long long)rc.W * rc.H;
    unsigned nev = 0;
    for (long long a = (long long)blockIdx.x * kWarps + warp; a < npix; a += (long long)gridDim.x * kWarps) {
        bool v = lane < 4 && valid[4 * a + lane] != 0;
        if (!__any_sync(0xffffffffu, v)) {
            if (lane < 4) hcost[4 * a + lane] = kCmax;
            continue;
        }
        const int px = (int)(a % rc.W), py = (int)(a / rc.W);
        PixWin<S> pw;
        build_window<G, S>(rc, px, py, true, pw);
        float h = lane < 4 ? hyp[4 * a + lane] : 1.0f;
        float c = kCmax;
        if (pw.ok) {
            PixView* pv = warp_pixviews(smem, rc.n_src, warp);
            pix_views(rc, views, px, py, pv);
            Cand my = make_cand(rc, pw, pw.geo, 0.0f, 0.0f, -1.0f, h, v);
            c = eval_batch<G, S, false>(rc, views, pw, pw.geo, pv, my, 4, warp_pairs(smem, rc.n_src, warp), nullptr,
                                        nev);
        }
        if (lane < 4) hcost[4 * a + lane] = v ? c : kCmax;
    }
}

// ---------------------------------------------------------------------------
// MRF (Eq. 6-9) at half resolution (node (gx, gy) <- pixel (2gx, 2gy)).
// Reading: TRW = sequential tree-reweighted min-sum message passing with
// rows and columns as monotonic chains (node weight 1 / max(#earlier,
// #later present neighbours)); one iteration = forward pass in raster order +
// backward pass; decode = per-node argmin of the belief (lowest label on a
// tie).  The raster order is run as anti-diagonal wavefronts (a node only
// depends on its up / left neighbours in the forward pass and on its down /
// right neighbours in the backward pass), which gives the same messages as
// the sequential sweep.  One cooperative launch per pass pipelines strips of
// kTrwRows node rows: a block owns strips b, b + gridDim.x, ... and walks each
// in tiles of kTrwCols columns; at stage k strip s takes tile k - s, whose
// upper neighbour tile (strip s - 1) was finished at stage k - 1 and whose
// left neighbour tile by the same block at stage k - 1.  Stages are separated
// by a grid barrier (ns + nb - 1 of them instead of gw + gh - 1), and the
// anti-diagonals of a tile by a block barrier.  Inside a tile one warp takes
// one node: lane (d, lq, l) evaluates the min-sum term of own label l towards
// label lq of the d-th outgoing neighbour.  At the start of a stage the block
// stages its tile in shared memory (unaries, label depths, the messages that
// do not change during the pass, the messages entering the tile from the
// tiles finished at the previous stage, written by other multiprocessors and
// read at L2); inside the stage a message to the lower node passes through
// shared memory and one to the right node stays in the warp's registers, so
// the anti-diagonal steps wait on no global memory.  Every message is also
// written to global memory (.cg) for the other pass and the decoding.  The
// backward pass runs the same schedule on the mirrored grid.
// ---------------------------------------------------------------------------
constexpr int kTrwRows = 32, kTrwCols = 32, kTrwBlock = 32 * kTrwRows;

struct MrfBufs {
    int gw, gh;
    int8_t* nlab;     // labels per node (0 = absent)
    int8_t* lmap;     // [4] hypothesis index of each label (-1 = reconstructed pixel)
    float* lab;       // [4] label depths
    float* un;        // [4] unary energies -log phi_n
    float* msg;       // [4 dir][4 lab] incoming messages (dir 0 up, 1 down, 2 left, 3 right)
};

__global__ void k_mrf_setup(int W, int H, MrfBufs mb, const uint8_t* __restrict__ known,
                            const float* __restrict__ depth, const float* __restrict__ hyp,
                            const uint8_t* __restrict__ valid, const float* __restrict__ hcost, float k1, float k2) {
    long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= (long long)mb.gw * mb.gh) return;
    int gx = (int)(g % mb.gw), gy = (int)(g / mb.gw);
    long long i = (long long)(2 * gy) * W + 2 * gx;
    int L = 0;
    if (known[i]) {
        mb.lab[4 * g] = depth[i];
        mb.un[4 * g] = 0.0f;
        mb.lmap[4 * g] = -1;
        L = 1;
    } else {
        for (int k = 0; k < 4; ++k)
            if (valid[4 * i + k]) {
                mb.lab[4 * g + L] = hyp[4 * i + k];
                mb.un[4 * g + L] = -logf((kCmax - hcost[4 * i + k]) / k1 + k2);   // Eq. 6
                mb.lmap[4 * g + L] = (int8_t)k;
                L++;
            }
    }
    mb.nlab[g] = (int8_t)L;
    for (int k = 0; k < 16; ++k) mb.msg[16 * g + k] = 0.0f;
}

// ((((a + b) + c) + d) + e): the belief sum in message-slot order
__device__ __forceinline__ float un_add4(float a, float b, float c, float d, float e) {
    return (((a + b) + c) + d) + e;
}

// -log of Eq. 7: phi_e = [k3 - min(1, relative difference)]^2
__device__ __forceinline__ float pair_energy(float h1, float h2, float k3) {
    float rel = h1 > h2 ? (h1 - h2) / h2 : (h2 - h1) / h1;
    return -2.0f * logf(k3 - fminf(1.0f, rel));
}

// Per-stage tile record in dynamic shared memory: the static data of the
// tile's 32 x 32 nodes (pass-local row-major), of the targets just below and
// right of it, the messages entering its first row and column from the
// tiles finished at the previous stage, and the wavefront's downward
// messages (double-buffered by step parity).
struct TrwTileSm {
    float4 un[kTrwRows * kTrwCols];    // unaries of the four labels
    float4 lab[kTrwRows * kTrwCols];   // label depths
    float4 msv[kTrwRows * kTrwCols];   // static message from the pass-local lower neighbour
    float4 msh[kTrwRows * kTrwCols];   // static message from the pass-local right neighbour
    float gamma[kTrwRows * kTrwCols];
    int nl[kTrwRows * kTrwCols];       // labels (0: absent or outside the grid)
    float4 lab_d[kTrwCols], lab_r[kTrwRows];   // targets below the last row / right of the last column
    int nl_d[kTrwCols], nl_r[kTrwRows];
    float4 up_b[kTrwCols], left_b[kTrwRows];   // messages into the first row / first column
    float4 up_w[2][kTrwRows + 1];              // downward messages of the current wavefront
};

__global__ void __launch_bounds__(kTrwBlock, 1) k_trw_strips(MrfBufs mb, bool forward, float k3) {
    cooperative_groups::grid_group grid = cooperative_groups::this_grid();
    extern __shared__ __align__(16) unsigned char trw_smem[];
    TrwTileSm& T = *reinterpret_cast<TrwTileSm*>(trw_smem);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ns = (mb.gh + kTrwRows - 1) / kTrwRows, nb = (mb.gw + kTrwCols - 1) / kTrwCols;
    // message slots (dir 0 up, 1 down, 2 left, 3 right) in pass-local terms:
    // the static ones come from the lower / right neighbours, the dynamic
    // ones from the upper / left neighbours updated earlier in this pass
    const int sv = forward ? 1 : 0, sh = forward ? 3 : 2, dv = forward ? 0 : 1, dh = forward ? 2 : 3;
    // original node index of pass-local (xf, yf), or -1 outside the grid
    auto node = [&](int xf, int yf) -> long long {
        if (xf < 0 || yf < 0 || xf >= mb.gw || yf >= mb.gh) return -1;
        const int x = forward ? xf : mb.gw - 1 - xf, y = forward ? yf : mb.gh - 1 - yf;
        return (long long)y * mb.gw + x;
    };
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int k = 0; k < ns + nb - 1; ++k) {
        for (int st = blockIdx.x; st < ns; st += gridDim.x) {
            const int c = k - st;
            if (c < 0 || c >= nb) continue;              // block-uniform
            const int x0 = c * kTrwCols, y0 = st * kTrwRows;
            // ---- load the tile (one node per thread) and its borders
            {
                const int r = tid / kTrwCols, cc = tid % kTrwCols;
                const long long i = node(x0 + cc, y0 + r);
                int L = 0;
                float gm = 1.0f;
                float4 un = z4, lb = z4, mv = z4, mh = z4;
                if (i >= 0) {
                    L = mb.nlab[i];
                    const int x = (int)(i % mb.gw), y = (int)(i / mb.gw);
                    const int nbx[4] = {0, 0, -1, 1}, nby[4] = {-1, 1, 0, 0};
                    int before = 0, after = 0;
#pragma unroll
                    for (int d = 0; d < 4; ++d) {
                        const int qx = x + nbx[d], qy = y + nby[d];
                        const bool in = qx >= 0 && qx < mb.gw && qy >= 0 && qy < mb.gh;
                        const int nq = in ? mb.nlab[(long long)qy * mb.gw + qx] : 0;
                        if (nq > 0) { if (d == 0 || d == 2) before++; else after++; }
                    }
                    const int mx = max(before, after);
                    gm = mx > 0 ? 1.0f / (float)mx : 1.0f;
                    un = reinterpret_cast<const float4*>(mb.un)[i];
                    lb = reinterpret_cast<const float4*>(mb.lab)[i];
                    mv = __ldcg(reinterpret_cast<const float4*>(mb.msg + 16 * i + 4 * sv));
                    mh = __ldcg(reinterpret_cast<const float4*>(mb.msg + 16 * i + 4 * sh));
                }
                T.nl[tid] = L;
                T.gamma[tid] = gm;
                T.un[tid] = un;
                T.lab[tid] = lb;
                T.msv[tid] = mv;
                T.msh[tid] = mh;
                if (tid < kTrwCols) {                     // targets below the tile
                    const long long q = node(x0 + tid, y0 + kTrwRows);
                    T.nl_d[tid] = q >= 0 ? mb.nlab[q] : 0;
                    T.lab_d[tid] = q >= 0 ? reinterpret_cast<const float4*>(mb.lab)[q] : z4;
                } else if (tid < kTrwCols + kTrwRows) {   // targets right of the tile
                    const int rr = tid - kTrwCols;
                    const long long q = node(x0 + kTrwCols, y0 + rr);
                    T.nl_r[rr] = q >= 0 ? mb.nlab[q] : 0;
                    T.lab_r[rr] = q >= 0 ? reinterpret_cast<const float4*>(mb.lab)[q] : z4;
                } else if (tid < 2 * kTrwCols + kTrwRows) {   // into the first row (previous stage)
                    const int c2 = tid - kTrwCols - kTrwRows;
                    const long long q = node(x0 + c2, y0);
                    T.up_b[c2] = q >= 0 ? __ldcg(reinterpret_cast<const float4*>(mb.msg + 16 * q + 4 * dv)) : z4;
                } else if (tid < 2 * kTrwCols + 2 * kTrwRows) {   // into the first column
                    const int r2 = tid - 2 * kTrwCols - kTrwRows;
                    const long long q = node(x0, y0 + r2);
                    T.left_b[r2] = q >= 0 ? __ldcg(reinterpret_cast<const float4*>(mb.msg + 16 * q + 4 * dh)) : z4;
                }
            }
            __syncthreads();
            // ---- the tile's anti-diagonals: warp = row, lane (dsel, lq, l)
            // evaluates the min-sum term of own label l towards label lq of
            // the lower (dsel 0) or right (dsel 1) neighbour
            const int dsel = lane >> 4, lq = (lane >> 2) & 3, l = lane & 3;
            const int dir = forward ? (dsel ? 3 : 1) : (dsel ? 2 : 0);
            float left_in = 0.0f;                         // message from the left node, kept by this warp
            for (int t = 0; t < kTrwRows + kTrwCols - 1; ++t) {
                const int u = t - warp;                   // tile column of this warp's node
                float out_v = 0.0f, out_h = 0.0f;         // messages sent down / right (0: none)
                if (u >= 0 && u < kTrwCols) {
                    const int n = warp * kTrwCols + u;
                    const int L = T.nl[n];
                    if (L > 0) {                          // warp-uniform
                        const float4 un4 = T.un[n], mv4 = T.msv[n], mh4 = T.msh[n], lb4 = T.lab[n];
                        const float unl = l == 0 ? un4.x : l == 1 ? un4.y : l == 2 ? un4.z : un4.w;
                        const float mvl = l == 0 ? mv4.x : l == 1 ? mv4.y : l == 2 ? mv4.z : mv4.w;
                        const float mhl = l == 0 ? mh4.x : l == 1 ? mh4.y : l == 2 ? mh4.z : mh4.w;
                        const float labl = l == 0 ? lb4.x : l == 1 ? lb4.y : l == 2 ? lb4.z : lb4.w;
                        const float4 upv = warp == 0 ? T.up_b[u] : T.up_w[(t - 1) & 1][warp];
                        const float dynv = l == 0 ? upv.x : l == 1 ? upv.y : l == 2 ? upv.z : upv.w;
                        float dynh = left_in;
                        if (u == 0) {
                            const float4 lf = T.left_b[warp];
                            dynh = l == 0 ? lf.x : l == 1 ? lf.y : l == 2 ? lf.z : lf.w;
                        }
                        // belief of own label l: unary + the four incoming messages in slot order
                        const float bel = forward ? un_add4(unl, dynv, mvl, dynh, mhl) : un_add4(unl, mvl, dynv, mhl, dynh);
                        int Lq;
                        float4 lq4;
                        if (dsel == 0) {
                            Lq = warp + 1 < kTrwRows ? T.nl[n + kTrwCols] : T.nl_d[u];
                            lq4 = warp + 1 < kTrwRows ? T.lab[n + kTrwCols] : T.lab_d[u];
                        } else {
                            Lq = u + 1 < kTrwCols ? T.nl[n + 1] : T.nl_r[warp];
                            lq4 = u + 1 < kTrwCols ? T.lab[n + 1] : T.lab_r[warp];
                        }
                        const float labq = lq == 0 ? lq4.x : lq == 1 ? lq4.y : lq == 2 ? lq4.z : lq4.w;
                        const float mdir = dsel ? mhl : mvl;
                        float e = 3.0e38f;
                        if (l < L && lq < Lq) e = T.gamma[n] * bel - mdir + pair_energy(labl, labq, k3);
                        // minimum over own labels, then over the target's labels (normalisation)
                        e = fminf(e, __shfl_xor_sync(0xffffffffu, e, 1));
                        e = fminf(e, __shfl_xor_sync(0xffffffffu, e, 2));
                        float mn = fminf(e, __shfl_xor_sync(0xffffffffu, e, 4));
                        mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, 8));
                        const float o = lq < Lq ? e - mn : 0.0f;
                        if (l == 0 && lq < Lq) {
                            const long long q = dsel == 0 ? node(x0 + u, y0 + warp + 1) : node(x0 + u + 1, y0 + warp);
                            __stcg(mb.msg + 16 * q + 4 * (dir ^ 1) + lq, o);
                        }
                        // lane j < 4: the message to label j of the node below
                        // (sent by lane 4 j); every lane: the message to label l
                        // of the right node (sent by lane 16 + 4 l)
                        out_v = __shfl_sync(0xffffffffu, o, 4 * l);
                        out_h = __shfl_sync(0xffffffffu, o, 16 + 4 * l);
                    }
                }
                // the node below reads the downward message at the next step
                // (lanes 0..3 write its four labels), the right node is this
                // warp's next node
                if (lane < 4) {
                    float* w = reinterpret_cast<float*>(&T.up_w[t & 1][warp + 1]);
                    w[lane] = out_v;
                }
                left_in = out_h;
                __syncthreads();
            }
        }
        grid.sync();                                      // every block runs the same number of stages
    }
}

__global__ void k_trw_decode(MrfBufs mb, int32_t* __restrict__ label) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)mb.gw * mb.gh) return;
    int L = mb.nlab[i];
    if (!L) { label[i] = -2; return; }
    int best = 0;
    float bv = 3.0e38f;
    for (int l = 0; l < L; ++l) {
        float b = mb.un[4 * i + l];
        for (int d = 0; d < 4; ++d) b += mb.msg[16 * i + 4 * d + l];
        if (b < bv) { bv = b; best = l; }
    }
    label[i] = mb.lmap[4 * i + best];
}

// ---------------------------------------------------------------------------
// selection: nearest up-sampled decoded depth is the reference; the closest
// valid hypothesis (lowest k on a tie) becomes the new depth of a hole
// ---------------------------------------------------------------------------
__global__ void k_select(int W, int H, const uint8_t* __restrict__ known, const float* __restrict__ hyp,
                         const uint8_t* __restrict__ valid, const int32_t* __restrict__ label,
                         const float4* __restrict__ plane, float* __restrict__ newd) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)W * H) return;
    int x = (int)(i % W), y = (int)(i / W);
    if (known[i]) { newd[i] = plane[i].w; return; }
    int gw = (W + 1) / 2;
    long long g = (long long)(y / 2) * gw + (x / 2);
    int lb = label[g];
    float nd = 0.0f;
    if (lb >= -1) {
        long long ni = (long long)(2 * (y / 2)) * W + 2 * (x / 2);
        float rd = lb == -1 ? plane[ni].w : hyp[4 * ni + lb];
        float bd = 3.0e38f;
        for (int k = 0; k < 4; ++k)
            if (valid[4 * i + k]) {
                float e = fabsf(hyp[4 * i + k] - rd);
                if (e < bd) { bd = e; nd = hyp[4 * i + k]; }
            }
    }
    newd[i] = nd;
}

// PHI-MVS/M (Sec. IV, Table I: the MRF removed): each hole takes its valid
// hypothesis of minimal matching cost, the lowest k on a tie; a hole without
// a valid hypothesis gets no depth
__global__ void k_select_min_cost(long long n, const uint8_t* __restrict__ known, const float* __restrict__ hyp,
                                  const uint8_t* __restrict__ valid, const float* __restrict__ hcost,
                                  const float4* __restrict__ plane, float* __restrict__ newd) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (known[i]) { newd[i] = plane[i].w; return; }
    const float4 h = reinterpret_cast<const float4*>(hyp)[i];
    const float4 c = reinterpret_cast<const float4*>(hcost)[i];
    const uchar4 v = reinterpret_cast<const uchar4*>(valid)[i];
    const float hv[4] = {h.x, h.y, h.z, h.w}, cv[4] = {c.x, c.y, c.z, c.w};
    const bool ok[4] = {v.x != 0, v.y != 0, v.z != 0, v.w != 0};
    int bk = -1;
#pragma unroll
    for (int k = 0; k < 4; ++k)
        if (ok[k] && (bk < 0 || cv[k] < cv[bk])) bk = k;
    newd[i] = bk >= 0 ? hv[bk] : 0.0f;
}

// Eq. 10 normal from the back-projected 4-neighbours (reading: unit length,
// oriented towards the camera); a hole without all four neighbours stays
// empty
__global__ void k_eq10(const __grid_constant__ RefConst rc, const uint8_t* __restrict__ known,
                       const float* __restrict__ newd, float4* __restrict__ plane) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int W = rc.W, H = rc.H;
    if (i >= (long long)W * H) return;
    if (known[i]) return;
    int x = (int)(i % W), y = (int)(i / W);
    float4 out = make_float4(0.f, 0.f, 0.f, 0.f);
    float d = newd[i];
    if (d > 0.0f && x >= 1 && y >= 1 && x <= W - 2 && y <= H - 2) {
        const int nx[4] = {x, x, x - 1, x + 1}, ny[4] = {y - 1, y + 1, y, y};
        float P[4][3];
        bool ok = true;
        for (int k = 0; k < 4; ++k) {
            float dk = newd[(long long)ny[k] * W + nx[k]];
            if (!(dk > 0.0f)) { ok = false; break; }
            float r0, r1, r2;
            mat3v(rc.Kinv, (float)nx[k], (float)ny[k], 1.0f, r0, r1, r2);
            P[k][0] = dk * r0; P[k][1] = dk * r1; P[k][2] = dk * r2;
        }
        if (ok) {
            float a0 = P[0][0] - P[1][0], a1 = P[0][1] - P[1][1], a2 = P[0][2] - P[1][2];
            float b0 = P[2][0] - P[3][0], b1 = P[2][1] - P[3][1], b2 = P[2][2] - P[3][2];
            float n0 = a1 * b2 - a2 * b1, n1 = a2 * b0 - a0 * b2, n2 = a0 * b1 - a1 * b0;
            float len = sqrtf(n0 * n0 + n1 * n1 + n2 * n2);
            if (len > 0.0f) {
                n0 /= len; n1 /= len; n2 /= len;
                float r0, r1, r2;
                mat3v(rc.Kinv, (float)x, (float)y, 1.0f, r0, r1, r2);
                if (n0 * r0 + n1 * r1 + n2 * r2 > 0.0f) { n0 = -n0; n1 = -n1; n2 = -n2; }
                out = make_float4(n0, n1, n2, d);
            }
        }
    }
    plane[i] = out;
}

__global__ void k_known_from_cost(long long n, const float4* __restrict__ plane, const float* __restrict__ cost,
                                  float hole_cost, uint8_t* __restrict__ known, float* __restrict__ depth) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float d = plane[i].w;
    bool k = d > 0.0f && cost[i] < hole_cost;
    known[i] = k ? 1 : 0;
    depth[i] = k ? d : 0.0f;
}

__global__ void k_depth_of(long long n, const float4* __restrict__ plane, const uint8_t* __restrict__ known,
                           float* __restrict__ depth) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    depth[i] = known[i] ? plane[i].w : 0.0f;
}

unsigned blocks_for(long long n, int b) { return (unsigned)((n + b - 1) / b); }

}  // namespace

cudaError_t launch_geo_filter(const FilterConst& fc, uint8_t* keep, int32_t* count, cudaStream_t s) {
    long long n = (long long)fc.W * fc.H;
    k_geo_filter<<<blocks_for(n, 256), 256, 0, s>>>(fc, keep, count);
    count_launch();
    return cudaGetLastError();
}

// Fixed line-gap scratch of mvs_phi_hypotheses_static: 8 int32 per pixel for
// up to MVS_PHI_STATIC_MAX_PIXELS pixels, in the library's own device memory.
static __device__ __align__(256) int32_t g_phi_gaps_static[8 * (size_t)MVS_PHI_STATIC_MAX_PIXELS];

// Device address of g_phi_gaps_static on the current device, looked up once
// per device with that device current (host code only sees a stand-in for the
// symbol, never its device address).
cudaError_t phi_static_scratch(int32_t** out) {
    static std::mutex mu;
    static int32_t* ptr[128] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(mu);
    if (!ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_phi_gaps_static);
        if (e != cudaSuccess) return e;
        ptr[dev] = (int32_t*)p;
    }
    *out = ptr[dev];
    return cudaSuccess;
}

cudaError_t launch_phi_hypotheses(int W, int H, const float* depth, const uint8_t* known, int n_fit, int inverse,
                                  float d_lo, float d_hi, float* hyp, uint8_t* valid, int32_t* scratch,
                                  cudaStream_t s) {
    int maxl = W + H - 1;
    dim3 grid(blocks_for(maxl, 128), 4);
    k_line_gaps<<<grid, 128, 0, s>>>(W, H, known, scratch);
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    long long n = (long long)W * H;
    k_line_fit<<<blocks_for(n, 128), 128, 0, s>>>(W, H, depth, known, scratch, n_fit, inverse, d_lo, d_hi, hyp,
                                                  valid);
    count_launch();
    return cudaGetLastError();
}

#define MVS_DISPATCH(n, CALL)                       \
    do {                                            \
        int _s = (n) * (n);                         \
        if (_s <= 16) { CALL(4, 4); }               \
        else if (_s <= 36) { CALL(4, 9); }          \
        else if (_s <= 64) { CALL(8, 8); }          \
        else if (_s <= 128) { CALL(16, 8); }        \
        else if (_s <= 256) { CALL(16, 16); }       \
        else { CALL(32, 16); }                      \
    } while (0)

cudaError_t launch_phi_cost(const RefConst& rc, const float* hyp, const uint8_t* valid, float* hcost,
                            cudaStream_t s) {
    long long npix = (long long)rc.W * rc.H;
    const size_t smem = smem_block_bytes(rc.n_src, kWarps);
#define CALL(G, S) k_phi_cost<G, S><<<pm_grid_for((const void*)k_phi_cost<G, S>, (npix + kWarps - 1) / kWarps, smem, kBlock), kBlock, smem, s>>>(rc, hyp, valid, hcost)
    MVS_DISPATCH(rc.n, CALL);
#undef CALL
    count_launch();
    const cudaError_t g = pm_grid_error();
    return g != cudaSuccess ? g : cudaGetLastError();
}

size_t phi_mrf_work_floats(int W, int H) {
    size_t g = (size_t)((W + 1) / 2) * ((H + 1) / 2);
    // msg 16, lab 4, un 4 floats; nlab 1 + lmap 4 bytes (rounded up to 2 floats)
    return g * (16 + 4 + 4 + 2) + 64;
}

cudaError_t launch_phi_mrf(int W, int H, const uint8_t* known, const float* depth, const float* hyp,
                           const uint8_t* valid, const float* hcost, float k1, float k2, float k3, int iters,
                           int32_t* label, float* work, cudaStream_t s) {
    MrfBufs mb;
    mb.gw = (W + 1) / 2;
    mb.gh = (H + 1) / 2;
    long long g = (long long)mb.gw * mb.gh;
    mb.msg = work;
    mb.lab = mb.msg + 16 * g;
    mb.un = mb.lab + 4 * g;
    mb.lmap = (int8_t*)(mb.un + 4 * g);
    mb.nlab = mb.lmap + 4 * g;
    k_mrf_setup<<<blocks_for(g, 256), 256, 0, s>>>(W, H, mb, known, depth, hyp, valid, hcost, k1, k2);
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // one block per strip, at most as many as are co-resident; the shared-
    // memory opt-in and the occupancy belong to the current device
    int max_blocks = 0;
    {
        static std::mutex mu;
        static int per_dev[128] = {};
        int dev = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
        if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
        std::lock_guard<std::mutex> lk(mu);
        if (!per_dev[dev]) {
            int sms = 0, per_sm = 0;
            if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
            if ((e = cudaFuncSetAttribute(k_trw_strips, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)sizeof(TrwTileSm))) != cudaSuccess)
                return e;
            if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_trw_strips, kTrwBlock,
                                                                   sizeof(TrwTileSm))) != cudaSuccess)
                return e;
            if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
            per_dev[dev] = sms * per_sm;
        }
        max_blocks = per_dev[dev];
    }
    const int want = (mb.gh + kTrwRows - 1) / kTrwRows;
    dim3 grid(std::max(1, std::min(want, max_blocks))), block(kTrwBlock);
    for (int it = 0; it < iters; ++it)
        for (int pass = 0; pass < 2; ++pass) {
            bool forward = pass == 0;
            void* args[] = {(void*)&mb, (void*)&forward, (void*)&k3};
            e = cudaLaunchCooperativeKernel((const void*)k_trw_strips, grid, block, args, sizeof(TrwTileSm), s);
            count_launch();
            if (e != cudaSuccess) return e;
        }
    k_trw_decode<<<blocks_for(g, 256), 256, 0, s>>>(mb, label);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_phi_select(const RefConst& rc, const uint8_t* known, const float* hyp, const uint8_t* valid,
                              const int32_t* label, float4* plane, float* newdepth, cudaStream_t s) {
    long long n = (long long)rc.W * rc.H;
    k_select<<<blocks_for(n, 256), 256, 0, s>>>(rc.W, rc.H, known, hyp, valid, label, plane, newdepth);
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_eq10<<<blocks_for(n, 256), 256, 0, s>>>(rc, known, newdepth, plane);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_phi_select_min_cost(const RefConst& rc, const uint8_t* known, const float* hyp,
                                       const uint8_t* valid, const float* hcost, float4* plane, float* newdepth,
                                       cudaStream_t s) {
    long long n = (long long)rc.W * rc.H;
    k_select_min_cost<<<blocks_for(n, 256), 256, 0, s>>>(n, known, hyp, valid, hcost, plane, newdepth);
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_eq10<<<blocks_for(n, 256), 256, 0, s>>>(rc, known, newdepth, plane);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_known_from_cost(int W, int H, const float4* plane, const float* cost, float hole_cost,
                                   uint8_t* known, float* depth, cudaStream_t s) {
    long long n = (long long)W * H;
    k_known_from_cost<<<blocks_for(n, 256), 256, 0, s>>>(n, plane, cost, hole_cost, known, depth);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_depth_of(int W, int H, const float4* plane, const uint8_t* known, float* depth, cudaStream_t s) {
    long long n = (long long)W * H;
    k_depth_of<<<blocks_for(n, 256), 256, 0, s>>>(n, plane, known, depth);
    count_launch();
    return cudaGetLastError();
}
