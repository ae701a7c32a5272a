// PatchMatch kernels: texture build, random initialisation, plane-map cost
// and one checkerboard phase (propagation + random refinement).
//   Sec. III-B  random initialisation
//   Sec. III-C  Eq. 4 weighted ZNCC, Eq. 5 aggregation, refinement
//   Sec. III    red-black checkerboard updating
#include "pm_device.cuh"

using namespace mvsdev;

namespace {

constexpr int kBlock = 128;

// ---------------------------------------------------------------------------
// bilinear-coefficient texture (layout documented in mvs_internal.h)
// ---------------------------------------------------------------------------
__global__ void k_build_texture(const uint8_t* __restrict__ img, int W, int H, float4* __restrict__ tex) {
    long long n = (long long)(W + 1) * (H + 1);
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x) {
        int i = (int)(t % (W + 1)) - 1, j = (int)(t / (W + 1)) - 1;
        int x0 = min(max(i, 0), W - 1), x1 = min(max(i + 1, 0), W - 1);
        int y0 = min(max(j, 0), H - 1), y1 = min(max(j + 1, 0), H - 1);
        float p00 = img[(long long)y0 * W + x0], p01 = img[(long long)y0 * W + x1];
        float p10 = img[(long long)y1 * W + x0], p11 = img[(long long)y1 * W + x1];
        float4 c;
        c.x = 0.25f * (p00 + p01 + p10 + p11);
        c.y = 0.5f * ((p01 - p00) + (p11 - p10));
        c.z = 0.5f * ((p10 - p00) + (p11 - p01));
        c.w = p00 - p01 - p10 + p11;
        tex[t] = c;
    }
}

// ---------------------------------------------------------------------------
// Sec. III-B: random initialisation, then the cost of the initial plane
// ---------------------------------------------------------------------------
template <int G, int S>
__global__ void __launch_bounds__(kBlock) k_init(const __grid_constant__ RefConst rc, float* view_cost) {
    const int lane = threadIdx.x & 31;
    const long long npix = (long long)rc.W * rc.H;
    const long long a = ((long long)blockIdx.x * kBlock + threadIdx.x) / G;
    if (((long long)blockIdx.x * kBlock + (threadIdx.x & ~31)) / G >= npix) return;  // whole warp past the end
    const bool exists = a < npix;
    const int px = exists ? (int)(a % rc.W) : 0, py = exists ? (int)(a / rc.W) : 0;
    PixWin<S> pw;
    build_window<G, S>(rc, px, py, exists, pw);
    float u[3];
    draws3(rc, exists ? a : 0, -1, u);
    float d = rc.d_lo + (rc.d_hi - rc.d_lo) * u[0];
    float th = 2.0f * kPi * u[1];
    float ph = kPi * (u[2] - 0.5f);
    float n0, n1, n2;
    normal_from_angles(th, ph, pw.rx0, pw.rx1, pw.rx2, n0, n1, n2);
    float* vc = (view_cost && exists) ? view_cost + a * rc.n_src : nullptr;
    unsigned nev = 0;
    float c = eval_hyp<G, S, true>(rc, pw, px, py, n0, n1, n2, d, exists, vc, nev);
    flush_evals(rc.eval_counter, nev);
    if (exists && (lane & (G - 1)) == 0) {
        rc.plane[a] = make_float4(n0, n1, n2, d);
        rc.cost[a] = c;
    }
}

// cost of a given plane map
template <int G, int S>
__global__ void __launch_bounds__(kBlock) k_cost(const __grid_constant__ RefConst rc, const float4* __restrict__ plane,
                                                  float* __restrict__ cost, float* view_cost) {
    const int lane = threadIdx.x & 31;
    const long long npix = (long long)rc.W * rc.H;
    const long long a = ((long long)blockIdx.x * kBlock + threadIdx.x) / G;
    if (((long long)blockIdx.x * kBlock + (threadIdx.x & ~31)) / G >= npix) return;
    const bool exists = a < npix;
    const int px = exists ? (int)(a % rc.W) : 0, py = exists ? (int)(a / rc.W) : 0;
    PixWin<S> pw;
    build_window<G, S>(rc, px, py, exists, pw);
    float4 pl = exists ? plane[a] : make_float4(0.f, 0.f, -1.f, 1.f);
    float* vc = (view_cost && exists) ? view_cost + a * rc.n_src : nullptr;
    unsigned nev = 0;
    float c = eval_hyp<G, S, true>(rc, pw, px, py, pl.x, pl.y, pl.z, pl.w, exists, vc, nev);
    flush_evals(rc.eval_counter, nev);
    if (exists && (lane & (G - 1)) == 0) cost[a] = c;
}

// ---------------------------------------------------------------------------
// Checkerboard phase.  Reading of the cited (undescribed) sampling pattern:
// eight groups of other-colour neighbours, the member with the lowest stored
// cost of each group is a candidate (first listed wins a tie).
//   groups 0..3: near V-shapes up / down / left / right, six members
//   groups 4..7: far lines up / down / left / right at distances 5, 7, .., 25
// ---------------------------------------------------------------------------
__device__ __forceinline__ void near_member(int g, int k, int& dx, int& dy) {
    // up-pointing pattern, rotated per group
    const int ux[6] = {0, -1, 1, -2, 0, 2};
    const int uy[6] = {-1, -2, -2, -3, -3, -3};
    int a = ux[k], b = uy[k];
    switch (g) {
        case 0: dx = a; dy = b; break;
        case 1: dx = a; dy = -b; break;
        case 2: dx = b; dy = a; break;
        default: dx = -b; dy = a; break;
    }
}

template <int G, int S>
__global__ void __launch_bounds__(kBlock) k_phase(const __grid_constant__ RefConst rc, int phase) {
    const int lane = threadIdx.x & 31, lg = lane & (G - 1), gbase = lane & ~(G - 1);
    const int color = phase & 1;
    const int Wa = (rc.W + 1) >> 1;
    const long long nact = (long long)Wa * rc.H;
    const long long a = ((long long)blockIdx.x * kBlock + threadIdx.x) / G;
    if (((long long)blockIdx.x * kBlock + (threadIdx.x & ~31)) / G >= nact) return;
    const int py = (int)(a / Wa);
    const int px = 2 * (int)(a % Wa) + ((py + color) & 1);
    const bool exists = a < nact && px < rc.W;
    const int qx = exists ? px : 0, qy = exists ? py : 0;
    const long long pix = (long long)qy * rc.W + qx;
    PixWin<S> pw;
    build_window<G, S>(rc, qx, qy, exists, pw);

    float4 cur = exists ? rc.plane[pix] : make_float4(0.f, 0.f, -1.f, 1.f);
    float cur_c = exists ? rc.cost[pix] : kCmax;
    unsigned nev = 0;

    // ---- candidate search: lane lg scans groups lg, lg + G, ...
    constexpr int kSlots = (8 + G - 1) / G;
    int cand[kSlots];
#pragma unroll
    for (int s = 0; s < kSlots; ++s) {
        int g = s * G + lg;
        int best = -1;
        float bc = 0.0f;
        if (g < 8 && exists) {
            int cnt = g < 4 ? 6 : 11;
            for (int k = 0; k < cnt; ++k) {
                int dx, dy;
                if (g < 4) near_member(g, k, dx, dy);
                else {
                    int dist = 5 + 2 * k;
                    dx = g == 6 ? -dist : (g == 7 ? dist : 0);
                    dy = g == 4 ? -dist : (g == 5 ? dist : 0);
                }
                int x2 = qx + dx, y2 = qy + dy;
                if (x2 < 0 || x2 >= rc.W || y2 < 0 || y2 >= rc.H) continue;
                int q = y2 * rc.W + x2;
                float c = rc.cost[q];
                if (best < 0 || c < bc) { best = q; bc = c; }
            }
        }
        cand[s] = best;
    }

    // ---- propagation: evaluate the transferred candidate planes
    float best_c = cur_c;
    float4 best = cur;
    bool changed = false;
#pragma unroll
    for (int g = 0; g < 8; ++g) {
        int q = __shfl_sync(0xffffffffu, cand[g / G], gbase + (g % G));
        bool ok = exists && q >= 0;
        float4 np = ok ? rc.plane[q] : make_float4(0.f, 0.f, -1.f, 1.f);
        float d = 0.0f;
        if (ok) {
            // the neighbour's plane carried over as a plane (reading)
            int x2 = q % rc.W, y2 = q / rc.W;
            const float* Ki = rc.Kinv;
            float r0 = fmaf(Ki[0], (float)x2, fmaf(Ki[1], (float)y2, Ki[2]));
            float r1 = fmaf(Ki[3], (float)x2, fmaf(Ki[4], (float)y2, Ki[5]));
            float r2 = fmaf(Ki[6], (float)x2, fmaf(Ki[7], (float)y2, Ki[8]));
            float rho = np.w * (np.x * r0 + np.y * r1 + np.z * r2);
            float den = np.x * pw.rx0 + np.y * pw.rx1 + np.z * pw.rx2;
            ok = den < 0.0f;
            d = ok ? rho / den : 0.0f;
            ok = ok && d >= rc.d_lo && d <= rc.d_hi;
        }
        float c = eval_hyp<G, S, false>(rc, pw, qx, qy, np.x, np.y, np.z, d, ok, nullptr, nev);
        if (ok && c < best_c) {
            best_c = c;
            best = make_float4(np.x, np.y, np.z, d);
            changed = true;
        }
    }
    if (changed) {
        cur = best;
        cur_c = best_c;
    }

    // ---- refinement (Sec. III-C): delta_d in [-d_hi/4, d_hi/4],
    // delta_theta in [-pi/2, pi/2], delta_phi in [-pi/12, pi/12]
    float u[3];
    draws3(rc, pix, phase, u);
    float dd = (2.0f * u[0] - 1.0f) * (rc.d_hi * 0.25f);
    float dth = (2.0f * u[1] - 1.0f) * (kPi * 0.5f);
    float dph = (2.0f * u[2] - 1.0f) * (kPi / 12.0f);
    float d_new = fminf(fmaxf(cur.w + dd, rc.d_lo), rc.d_hi);
    float m0 = cur.x, m1 = cur.y, m2 = cur.z;
    if (m2 < 0.0f) { m0 = -m0; m1 = -m1; m2 = -m2; }
    float th = atan2f(m1, m0);
    float ph = acosf(fminf(1.0f, fmaxf(-1.0f, m2)));
    float nn0, nn1, nn2;
    normal_from_angles(th + dth, ph + dph, pw.rx0, pw.rx1, pw.rx2, nn0, nn1, nn2);
    float4 rcand[3] = {make_float4(cur.x, cur.y, cur.z, d_new), make_float4(nn0, nn1, nn2, cur.w),
                       make_float4(nn0, nn1, nn2, d_new)};
    best_c = cur_c;
    best = cur;
    changed = false;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float c = eval_hyp<G, S, false>(rc, pw, qx, qy, rcand[k].x, rcand[k].y, rcand[k].z, rcand[k].w, exists,
                                         nullptr, nev);
        if (exists && c < best_c) {
            best_c = c;
            best = rcand[k];
            changed = true;
        }
    }
    if (changed) {
        cur = best;
        cur_c = best_c;
    }
    if (exists && lg == 0) {
        rc.plane[pix] = cur;
        rc.cost[pix] = cur_c;
    }
    flush_evals(rc.eval_counter, nev);
}

template <int G, int S>
unsigned grid_for(long long units) {
    long long threads = units * G;
    return (unsigned)((threads + kBlock - 1) / kBlock);
}

}  // namespace

// lanes per pixel and slots per lane for a window of n x n samples
int pm_group_lanes(int n) {
    int s = n * n;
    if (s <= 36) return 4;
    if (s <= 128) return 8;
    if (s <= 256) return 16;
    return 32;
}

#define MVS_DISPATCH(n, CALL)                       \
    do {                                            \
        int _s = (n) * (n);                         \
        if (_s <= 16) { CALL(4, 4); }               \
        else if (_s <= 36) { CALL(4, 9); }          \
        else if (_s <= 64) { CALL(8, 8); }          \
        else if (_s <= 128) { CALL(8, 16); }        \
        else if (_s <= 256) { CALL(16, 16); }       \
        else { CALL(32, 16); }                      \
    } while (0)

cudaError_t launch_build_texture(const uint8_t* img, int W, int H, float4* tex, cudaStream_t s) {
    long long n = (long long)(W + 1) * (H + 1);
    unsigned blocks = (unsigned)std::min<long long>((n + 255) / 256, 152LL * 16);
    k_build_texture<<<blocks, 256, 0, s>>>(img, W, H, tex);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_init(const RefConst& rc, float* view_cost, cudaStream_t s) {
    long long npix = (long long)rc.W * rc.H;
#define CALL(G, S) k_init<G, S><<<grid_for<G, S>(npix), kBlock, 0, s>>>(rc, view_cost)
    MVS_DISPATCH(rc.n, CALL);
#undef CALL
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_cost(const RefConst& rc, const float4* plane, float* cost, float* view_cost, cudaStream_t s) {
    long long npix = (long long)rc.W * rc.H;
#define CALL(G, S) k_cost<G, S><<<grid_for<G, S>(npix), kBlock, 0, s>>>(rc, plane, cost, view_cost)
    MVS_DISPATCH(rc.n, CALL);
#undef CALL
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_phase(const RefConst& rc, int phase, cudaStream_t s) {
    long long nact = (long long)((rc.W + 1) / 2) * rc.H;
#define CALL(G, S) k_phase<G, S><<<grid_for<G, S>(nact), kBlock, 0, s>>>(rc, phase)
    MVS_DISPATCH(rc.n, CALL);
#undef CALL
    count_launch();
    return cudaGetLastError();
}
