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
