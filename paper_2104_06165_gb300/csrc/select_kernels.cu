// Kernels on the sparse points of a structure-from-motion step: neighbouring-
// image selection (Sec. III-A) and the depth initialisation from sparse
// features (Sec. III-B, at the end of this file).
//
// Neighbouring-image selection (Sec. III-A, Eqs. 1-3).  For every ordered
// pair (reference i, source j) one block walks the sparse points: a point
// visible in both counts towards N_A, and Eq. 1 moves it along the ray from
// the reference centre, X^ = (1 + eps) X - eps C_i, so that Eq. 2 averages
// the displacement |x^'_j - x'_j| of its projection into j (FP64, block
// reduction in a fixed order).  Then one thread per reference image scores
// the sources with Eq. 3, zeta = (1 / N_A) min(b_ij, 0.1) min(theta_ij, 0.05)
// (baselines and principal-axis angles are FP64 per-pair constants from the
// host), removes those with tau < t_tau or no shared point and keeps the k
// smallest (tie: lower index).
#include <algorithm>
#include <cmath>

#include "mvs_internal.h"

namespace {

constexpr int kNbrBlock = 256;

__device__ __forceinline__ void proj(const NbrView& v, const double X[3], double& u, double& w) {
    double c[3], q[3];
    for (int a = 0; a < 3; ++a) c[a] = v.R[3 * a] * X[0] + v.R[3 * a + 1] * X[1] + v.R[3 * a + 2] * X[2] + v.t[a];
    for (int a = 0; a < 3; ++a) q[a] = v.K[3 * a] * c[0] + v.K[3 * a + 1] * c[1] + v.K[3 * a + 2] * c[2];
    u = q[0] / q[2];
    w = q[1] / q[2];
}

__global__ void __launch_bounds__(kNbrBlock) k_nbr_pairs(const NbrView* __restrict__ views, int n,
                                                        const double* __restrict__ X,
                                                        const unsigned long long* __restrict__ vis, long long n_pts,
                                                        double eps, double* __restrict__ tau, int* __restrict__ na) {
    const int i = blockIdx.x / n, j = blockIdx.x % n;
    __shared__ double s_sum[kNbrBlock / 32];
    __shared__ long long s_cnt[kNbrBlock / 32];
    double sum = 0.0;
    long long cnt = 0;
    if (i != j) {
        const NbrView& vi = views[i];
        const NbrView& vj = views[j];
        const double Ci[3] = {vi.C[0], vi.C[1], vi.C[2]};
        const unsigned long long both = (1ULL << i) | (1ULL << j);
        for (long long p = threadIdx.x; p < n_pts; p += blockDim.x) {
            if ((vis[p] & both) != both) continue;
            const double Xp[3] = {X[3 * p], X[3 * p + 1], X[3 * p + 2]};
            double Xh[3];
            for (int a = 0; a < 3; ++a) Xh[a] = (1.0 + eps) * Xp[a] - eps * Ci[a];
            double u, w, uh, wh;
            proj(vj, Xp, u, w);
            proj(vj, Xh, uh, wh);
            const double du = uh - u, dv = wh - w;
            sum += sqrt(du * du + dv * dv);
            cnt++;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        sum += __shfl_down_sync(0xffffffffu, sum, o);
        cnt += __shfl_down_sync(0xffffffffu, cnt, o);
    }
    if ((threadIdx.x & 31) == 0) {
        s_sum[threadIdx.x >> 5] = sum;
        s_cnt[threadIdx.x >> 5] = cnt;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        long long c = 0;
        for (int w = 0; w < kNbrBlock / 32; ++w) {
            s += s_sum[w];
            c += s_cnt[w];
        }
        na[blockIdx.x] = (int)c;
        tau[blockIdx.x] = c ? s / (double)c : 0.0;
    }
}

// one thread per reference image: Eq. 3 scores and the k smallest
__global__ void k_nbr_select(int n, int k, const double* __restrict__ base, const double* __restrict__ angle,
                             const int* __restrict__ na, const double* __restrict__ tau, double t_tau,
                             double* __restrict__ zeta, int* __restrict__ nbr) {
    const int i = threadIdx.x;
    if (i >= n) return;
    int cand[MVS_MAX_VIEWS_SELECT];
    double zc[MVS_MAX_VIEWS_SELECT];
    int nc = 0;
    for (int j = 0; j < n; ++j) {
        const long long e = (long long)i * n + j;
        double z = INFINITY;
        if (j != i && na[e] > 0 && tau[e] >= t_tau) {
            z = (1.0 / (double)na[e]) * fmin(base[e], 0.1) * fmin(angle[e], 0.05);
            // insertion by (zeta, index)
            int b = nc - 1;
            while (b >= 0 && zc[b] > z) {
                cand[b + 1] = cand[b];
                zc[b + 1] = zc[b];
                b--;
            }
            cand[b + 1] = j;
            zc[b + 1] = z;
            nc++;
        }
        if (zeta) zeta[e] = z;
    }
    for (int r = 0; r < k; ++r) nbr[(long long)i * k + r] = r < nc ? cand[r] : -1;
}

}  // namespace

cudaError_t launch_select_neighbors(const NbrView* dev_views, int n, const double* X, const unsigned long long* vis,
                                    long long n_pts, double eps, double t_tau, int k, const double* base,
                                    const double* angle, double* tau, int* na, double* zeta, int* nbr,
                                    cudaStream_t s) {
    k_nbr_pairs<<<n * n, kNbrBlock, 0, s>>>(dev_views, n, X, vis, n_pts, eps, tau, na);
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_nbr_select<<<1, 64, 0, s>>>(n, k, base, angle, na, tau, t_tau, zeta, nbr);
    count_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Depth initialisation from sparse features (Sec. III-B).  Features of the
// reference view: the sparse points visible in it whose re-projection error
// is below max_reproj and that are visible in at least floor(v - 1) images
// (v = mean images per point); each keeps its observation in the reference
// and its z-depth there (FP64, rounded to float).  Per pixel, the closest
// feature in each of four quadrants within W / 10 px gives [d_min, d_max],
// clamped to the depth range; the closest-feature choice is taken in single
// precision, each operation rounded on its own, the first feature winning a
// tie.
// ---------------------------------------------------------------------------
namespace {

constexpr int kRangeTile = 16;   // 16 x 16 pixels per block

__global__ void k_sparse_count(const unsigned long long* __restrict__ vis, long long n_pts,
                               unsigned long long views_mask, unsigned long long* __restrict__ total) {
    unsigned long long s = 0;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n_pts; p += (long long)gridDim.x * blockDim.x)
        s += __popcll(vis[p] & views_mask);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(total, s);
}

__global__ void k_sparse_features(const double* __restrict__ X, const unsigned long long* __restrict__ vis,
                                  const double* __restrict__ reproj, const double* __restrict__ obs, long long n_pts,
                                  unsigned long long views_mask, const unsigned long long* __restrict__ total,
                                  int ref, double R6, double R7, double R8, double t2, double max_reproj,
                                  float2* __restrict__ uv, float* __restrict__ depth) {
    const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= n_pts) return;
    const double vbar = (double)*total / (double)n_pts;
    const int min_views = (int)floor(__dsub_rn(vbar, 1.0));
    const unsigned long long m = vis[p];
    const bool keep = ((m >> ref) & 1ULL) && reproj[p] < max_reproj && __popcll(m & views_mask) >= min_views;
    double z = __dadd_rn(__dadd_rn(__dadd_rn(__dmul_rn(R6, X[3 * p]), __dmul_rn(R7, X[3 * p + 1])),
                                   __dmul_rn(R8, X[3 * p + 2])),
                         t2);
    uv[p] = make_float2((float)obs[2 * p], (float)obs[2 * p + 1]);
    depth[p] = keep ? (float)z : __int_as_float(0x7fc00000);   // NaN: not a feature
}

__global__ void __launch_bounds__(kRangeTile * kRangeTile) k_sparse_range(
    const float2* __restrict__ uv, const float* __restrict__ depth, long long n_pts, int W, int H, float d_lo,
    float d_hi, float2* __restrict__ range) {
    constexpr int NT = kRangeTile * kRangeTile;
    __shared__ float2 s_uv[NT];
    __shared__ float s_d[NT];
    __shared__ int s_wc[NT / 32];
    const int x = blockIdx.x * kRangeTile + (threadIdx.x % kRangeTile);
    const int y = blockIdx.y * kRangeTile + (threadIdx.x / kRangeTile);
    const float r = __fdiv_rn((float)W, 10.0f), r2 = __fmul_rn(r, r);
    // the tile's pixel box widened by the radius (a conservative candidate test)
    const float bx0 = (float)(blockIdx.x * kRangeTile) - r, bx1 = (float)(blockIdx.x * kRangeTile + kRangeTile - 1) + r;
    const float by0 = (float)(blockIdx.y * kRangeTile) - r, by1 = (float)(blockIdx.y * kRangeTile + kRangeTile - 1) + r;
    float best[4] = {INFINITY, INFINITY, INFINITY, INFINITY}, bd[4] = {0.f, 0.f, 0.f, 0.f};
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (long long base = 0; base < n_pts; base += NT) {
        const long long p = base + threadIdx.x;
        float2 f = make_float2(0.f, 0.f);
        float fd = 0.f;
        bool cand = false;
        if (p < n_pts) {
            fd = depth[p];
            f = uv[p];
            cand = fd == fd && f.x >= bx0 && f.x <= bx1 && f.y >= by0 && f.y <= by1;
        }
        // compact the candidates in point order
        const unsigned m = __ballot_sync(0xffffffffu, cand);
        if (lane == 0) s_wc[warp] = __popc(m);
        __syncthreads();
        int off = __popc(m & ((1u << lane) - 1u)), cnt = 0;
        for (int w = 0; w < NT / 32; ++w) {
            if (w < warp) off += s_wc[w];
            cnt += s_wc[w];
        }
        if (cand) {
            s_uv[off] = f;
            s_d[off] = fd;
        }
        __syncthreads();
        for (int k = 0; k < cnt; ++k) {
            const float dx = __fsub_rn(s_uv[k].x, (float)x), dy = __fsub_rn(s_uv[k].y, (float)y);
            const float d2 = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
            if (!(d2 < r2)) continue;
            const int q = dx >= 0.0f ? (dy >= 0.0f ? 0 : 3) : (dy >= 0.0f ? 1 : 2);
            if (d2 < best[q]) {
                best[q] = d2;
                bd[q] = s_d[k];
            }
        }
        __syncthreads();
    }
    if (x >= W || y >= H) return;
    float lo = INFINITY, hi = -INFINITY;
    for (int q = 0; q < 4; ++q)
        if (best[q] < INFINITY) {
            lo = bd[q] < lo ? bd[q] : lo;
            hi = bd[q] > hi ? bd[q] : hi;
        }
    const float nan = __int_as_float(0x7fc00000);
    range[(long long)y * W + x] = lo <= hi ? make_float2(fminf(fmaxf(lo, d_lo), d_hi), fminf(fmaxf(hi, d_lo), d_hi))
                                           : make_float2(nan, nan);
}

}  // namespace

cudaError_t launch_sparse_range(int ref, int n_views, const double Rrow2[3], double t2, const double* X,
                                const unsigned long long* vis, const double* reproj, const double* obs,
                                long long n_pts, double max_reproj, int W, int H, float d_lo, float d_hi,
                                unsigned long long* total, float2* uv, float* depth, float2* range, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(total, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    const unsigned long long views_mask = n_views >= 64 ? ~0ULL : ((1ULL << n_views) - 1ULL);
    if (n_pts > 0) {
        const unsigned nb = (unsigned)std::min<long long>((n_pts + 255) / 256, 152LL * 8);
        k_sparse_count<<<nb, 256, 0, s>>>(vis, n_pts, views_mask, total);
        k_sparse_features<<<(unsigned)((n_pts + 255) / 256), 256, 0, s>>>(X, vis, reproj, obs, n_pts, views_mask, total,
                                                                         ref, Rrow2[0], Rrow2[1], Rrow2[2], t2,
                                                                         max_reproj, uv, depth);
        count_launch(2);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    dim3 grid((W + kRangeTile - 1) / kRangeTile, (H + kRangeTile - 1) / kRangeTile);
    k_sparse_range<<<grid, kRangeTile * kRangeTile, 0, s>>>(uv, depth, n_pts, W, H, d_lo, d_hi, range);
    count_launch();
    return cudaGetLastError();
}
