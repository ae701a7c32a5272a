// Internal data layout shared by the host and device translation units of
// the library (not part of the C ABI).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#define MVS_MAX_SRC 32
#define MVS_MAX_WIN 22
#define MVS_MEMO_WORDS 9

// One source view as seen from a reference view.
//   A = K_j R_rel K_ref^-1, b = K_j t_rel, so that the plane-induced
//   homography of a plane (n, d) at reference pixel x is H = A + b m^T with
//   m = K_ref^-T n / rho, rho = d n.K_ref^-1 x (Sec. III-C homography
//   mapping), and m^T x = 1 / d at the pixel itself.  Kernels work in
//   doubled, half-shifted source coordinates xs2 = 2 u - 1, ys2 = 2 v - 1 of
//   a source point (u, v) = (q_x, q_y) / q_z, q = H x, i.e. with the rows
//     G = (2 A_0 - A_2, 2 A_1 - A_2, A_2),  B = (2 b_0 - b_2, 2 b_1 - b_2, b_2):
//   (xs2, ys2) = (G_0 x + B_0 m^T x, G_1 x + B_1 m^T x) / (G_2 x + B_2 m^T x).
//   Each entry is held as an unevaluated sum hi + lo of floats that equals its
//   double value (computed on the host) to about 2^-48 relative, so that the
//   kernels can evaluate source positions to far below a float ulp of an
//   image coordinate.
struct PairConst {
    float Gh[9], Gl[9];  // G row-major, hi and lo parts
    float Bh[3], Bl[3];  // B, hi and lo parts
    const uint2* tex;    // bilinear-coefficient texels of the source, see below
    int W, H;            // source image size
    int pitch;           // texel row pitch, tex_pitch(W)
    uint32_t n_tex;      // pitch * (H + 1)
};

// Per reference-view launch constants (kernel parameter, < 4 KB).
struct RefConst {
    int W, H;
    int ref_index;
    int n_src;
    float Kinv[9];
    const uint2* tex;          // reference bilinear-coefficient texels
    const uint8_t* img;        // reference image (uint8)
    int pitch;                 // tex_pitch(W)
    uint32_t n_tex;            // pitch * (H + 1)
    // window (Sec. III-C): n samples per axis, offsets step * (k - (n-1)/2)
    int n;
    float step;
    float sp_coef;             // -1 / (2 sigma_s^2) (0 = no spatial weight)
    float col_coef;            // -1 / (2 (4 * 255 sigma_c)^2) (0 = no colour weight), texel units
    float d_lo, d_hi;
    unsigned long long seed;
    float4* plane;             // state: (n.x, n.y, n.z, depth) per pixel
    float* cost;               // state: aggregated cost per pixel
    // Candidate memo of the checkerboard phases (exact work skipping): per
    // pixel MVS_MEMO_WORDS words, word g < 8 the key (member << 28 | plane
    // generation of that member) of the plane propagation group g offered
    // at the pixel's last visit, word 8 the mask of learned proposals scored
    // so far; all ones = nothing recorded.  gen: per pixel, a counter bumped
    // whenever the pixel's plane changes.  A pixel's cost never rises, so a
    // plane it scored (or found equal to a scored one) at an earlier visit of
    // the same call cannot be strictly cheaper now: such candidates are not
    // scored again, and the results are the same as without the memo.
    uint32_t* memo;
    uint32_t* gen;
    unsigned long long* eval_counter;  // measurement: evaluated (pixel, hypothesis, view) triples, or null
    int lanes_hint;            // lanes per pixel group (0 = default)
    int precision;             // 0 = FP32, 1 = mixed (half2 bilinear, FP32 moments)
    int n_prop;                // learned proposals per pixel (0 = none)
    const float4* props;       // H*W*n_prop planes (n, depth), or null
    const float2* init_range;  // H*W (d_min, d_max) of the sparse-feature initialisation (NaN: none), or null
    PairConst pair[MVS_MAX_SRC];
};
static_assert(sizeof(RefConst) <= 4096, "RefConst is passed as a kernel parameter (4 KB)");

// Row pitch (texels) of a bilinear-coefficient texture and the offsets that
// let the kernels form a texel index in one integer multiply-add.  A sample
// at doubled, half-shifted coordinates rounds to texel (i + 1, j + 1)
// through the sums 1.5 * 2^24 + 2 (i + 1 + alpha) and 1.5 * 2^24 +
// 2 (j + 1 + beta) (bits M + i + 1 + alpha and M + j + 1 + beta); their
// product-sum bits(y) p + bits(x) equals the index (j + 1) p + (i + 1)
// modulo 2^32 when beta p + alpha = -M (p + 1) modulo 2^32.  For p >= 1029
// that holds with beta < 2^22 - 2^14 and alpha < p, so both sums stay in the
// binade of 1.5 * 2^24 (exact integers); narrower images take the smallest
// p >= W + 1 with p + 1 a multiple of 1024, where M (p + 1) vanishes modulo
// 2^32 (M = 2^22 times an odd number) and alpha = beta = 0.  Wide images keep
// p = W + 1: a padded pitch near a power of two would alias the rows of a
// window in the L1 sets.
constexpr uint32_t kMagicBits = 0x4BC00000u;   // bits of 1.5 * 2^24
__host__ __device__ inline int tex_pitch(int W) { return W + 1 >= 1029 ? W + 1 : ((W + 2 + 1023) / 1024) * 1024 - 1; }
__host__ __device__ inline void tex_fold(int pitch, uint32_t* alpha, uint32_t* beta) {
    const uint32_t k = 0u - kMagicBits * (uint32_t)(pitch + 1);
    *beta = k / (uint32_t)pitch;
    *alpha = k - *beta * (uint32_t)pitch;
}

// Bilinear-coefficient texel layout.  Texel (i, j), i in [-1, W-1],
// j in [-1, H-1], stored at ((j + 1) * pitch + (i + 1)), holds four fp16
// numbers computed from the clamped taps p00 = I(i, j), p01 = I(i+1, j),
// p10 = I(i, j+1), p11 = I(i+1, j+1) on the [0, 255] scale:
//   a = p00 + p01 + p10 + p11                 (integer in [0, 1020])
//   b = (p01 - p00) + (p11 - p10)             (integer in [-510, 510])
//   c = (p10 - p00) + (p11 - p01)
//   d = p00 - p01 - p10 + p11
// all exact in fp16, so that four times the bilinear value at
// (i + 1/2 + U/2, j + 1/2 + V/2), |U|, |V| <= 1, is a + U b + V c + U V d.
// Kernels therefore work with intensities scaled by 4 (the ZNCC is
// scale-free; the colour weight and the flat limit are scaled to match).

// Status word written by kernels (bounded waits, bounds checks).
enum { MVS_DEV_OK = 0, MVS_DEV_TIMEOUT = 1, MVS_DEV_BOUNDS = 2 };

// Number of kernels the library has launched (all contexts); every launcher
// adds its launches so that a caller can count the kernels of a timed region.
#include <atomic>
extern std::atomic<long long> g_kernel_launches;
inline void count_launch(long long n = 1) { g_kernel_launches.fetch_add(n, std::memory_order_relaxed); }

// Host-side launchers (pm_kernels.cu / phi_kernels.cu).
cudaError_t launch_build_texture(const uint8_t* img, int W, int H, uint2* tex, cudaStream_t s);   // pitch tex_pitch(W)
cudaError_t launch_init(const RefConst& rc, float* view_cost, cudaStream_t s);
cudaError_t launch_cost(const RefConst& rc, const float4* plane, float* cost, float* view_cost, cudaStream_t s);
cudaError_t launch_phase(const RefConst& rc, int phase, cudaStream_t s);
// clears the candidate memo of rc's view (before the first phase of a call)
cudaError_t launch_memo_reset(const RefConst& rc, cudaStream_t s);
cudaError_t prime_launch_configs(const RefConst& rc);
int pm_group_lanes(int n_samples);
// grid of a grid-stride kernel: `units` blocks of work, capped at the blocks
// of `block` threads and `smem_bytes` shared memory that fit the device at once
unsigned pm_grid_for(const void* kernel, long long units, size_t smem_bytes, int block);
// error of this thread's last failed pm_grid_for query (cleared on read)
cudaError_t pm_grid_error();

struct FilterConst {
    int W, H;
    float K[9], Kinv[9];
    const float4* plane;
    int n_src;
    struct Src {
        float R[9], t[3];      // X_j = R X_ref + t
        float K[9], Kinv[9];
        const float4* plane;
        int W, H;
    } src[MVS_MAX_SRC];
    float depth_tol;
    int depth_relative;
    float cos_max;
    float max_reproj;
    int min_consistent;
};
cudaError_t launch_geo_filter(const FilterConst& fc, uint8_t* keep, int32_t* count, cudaStream_t s);

cudaError_t launch_phi_hypotheses(int W, int H, const float* depth, const uint8_t* known, int n_fit, int inverse,
                                  float d_lo, float d_hi, float* hyp, uint8_t* valid, int32_t* scratch,
                                  cudaStream_t s);
cudaError_t phi_static_scratch(int32_t** out);
cudaError_t launch_phi_cost(const RefConst& rc, const float* hyp, const uint8_t* valid, float* hcost,
                            cudaStream_t s);
cudaError_t launch_phi_mrf(int W, int H, const uint8_t* known, const float* depth, const float* hyp,
                           const uint8_t* valid, const float* hcost, float k1, float k2, float k3, int iters,
                           int32_t* label, float* work, cudaStream_t s);
size_t phi_mrf_work_floats(int W, int H);
cudaError_t launch_phi_select(const RefConst& rc, const uint8_t* known, const float* hyp, const uint8_t* valid,
                              const int32_t* label, float4* plane, float* newdepth, cudaStream_t s);
cudaError_t launch_phi_select_min_cost(const RefConst& rc, const uint8_t* known, const float* hyp,
                                       const uint8_t* valid, const float* hcost, float4* plane, float* newdepth,
                                       cudaStream_t s);
cudaError_t launch_known_from_cost(int W, int H, const float4* plane, const float* cost, float hole_cost,
                                   uint8_t* known, float* depth, cudaStream_t s);
cudaError_t launch_depth_of(int W, int H, const float4* plane, const uint8_t* known, float* depth, cudaStream_t s);

// depth-map fusion (fuse_kernels.cu): one view as seen by the fusion kernels
struct FuseView {
    float fx, sk, cx, fy, cy;    // pinhole K = [fx sk cx; 0 fy cy; 0 0 1]
    float R[9], t[3];            // x_cam = R X + t
    int W, H;
    int index;                   // context view index (reported with each point)
    const float4* plane;         // depth map (depth in .w, 0 = none)
    uint8_t* alive;              // W*H: 1 = still present
    int* claim;                  // W*H: lowest claiming pixel of the view being fused
    long long* owner;            // W*H or NULL: index of the point the pixel went into, -1 if absent
};
cudaError_t launch_fuse(const FuseView* host_views, FuseView* dev_views, int n, const uint8_t* const* keep, float tol,
                        int* block_count, long long* block_off, long long* total, float4* points, int2* src,
                        long long cap, cudaStream_t s);

// neighbouring-image selection (select_kernels.cu): at most 64 views (one
// visibility bit per view in a 64-bit mask per sparse point)
#define MVS_MAX_VIEWS_SELECT 64
struct NbrView {
    double K[9], R[9], t[3];     // x_cam = R X + t
    double C[3];                 // camera centre -R^T t
};
cudaError_t launch_select_neighbors(const NbrView* dev_views, int n, const double* X, const unsigned long long* vis,
                                    long long n_pts, double eps, double t_tau, int k, const double* base,
                                    const double* angle, double* tau, int* na, double* zeta, int* nbr,
                                    cudaStream_t s);

cudaError_t launch_sparse_range(int ref, int n_views, const double Rrow2[3], double t2, const double* X,
                                const unsigned long long* vis, const double* reproj, const double* obs,
                                long long n_pts, double max_reproj, int W, int H, float d_lo, float d_hi,
                                unsigned long long* total, float2* uv, float* depth, float2* range, cudaStream_t s);

// learned proposals (cnn_kernels.cu)
struct mvs_cnn;
cudaError_t cnn_propose(mvs_cnn* n, const uint8_t* img, const float4* plane, const float* cost, int W, int H,
                        const double Kinv[9], float4* props, cudaStream_t s);
bool cnn_shape_ok(const mvs_cnn* n, int W, int H);
