/*
 * PHI-MVS oracle: a plain, slow, single-threaded FP64 CPU implementation of the
 * depth-map path of PHI-MVS (Sun et al., arXiv 2104.06165).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark load this file.  It shares no code, header,
 * table or constant with the CUDA library: every step below is written out
 * from the paper's text in the paper's order, in double precision, with no
 * blocking, fusion or reordering.
 *
 * Passages followed (section / equation of the paper):
 *   Sec. III-B   random initialisation of depth and normal (theta, phi form),
 *                or the depth drawn between the nearest sparse features in
 *                four quadrants
 *   Sec. III-C   dilated window (scale s = r_orig / r_now), Eq. 4 ZNCC with
 *                bilinear samples and homography mapping, C(x,j) = 1 - Z,
 *                C_max for out-of-border samples, Eq. 5 aggregation with
 *                weights C(x,j)^-1, refinement with four candidates
 *   Sec. III     red-black checkerboard updating
 *   Sec. III-D   geometric-consistency filter (0.02, 30 deg, 1 px, > 1 view)
 *   Sec. III-E   four-direction line-fit hypotheses from the six closest
 *                reconstructed pixels, Eq. 6 unary, Eq. 7 pairwise, Eq. 8/9
 *                MAP via tree-reweighted message passing at half resolution,
 *                closest-hypothesis selection, Eq. 10 normals
 *   Sec. III-A   neighbouring-image selection: Eq. 1 disturbance, Eq. 2 tau,
 *                Eq. 3 zeta over the sparse points two images share
 *   Sec. III-F   depth-map fusion: greedy merging of back-projected pixels
 *                whose relative difference is below 0.01, image by image
 *   Sec. IV      parameters {r_now, r_orig, k1, k2, k3} = {5, 7, 4, 0.5, 2},
 *                one TRW iteration
 *
 * Readings where the paper is silent or ambiguous are marked "reading:".
 * The readings are the same ones the CUDA library implements; they are
 * listed in the project's design notes.
 *
 * Parity status: every function here is pinned by the CPU test-suite
 * (closed forms, library routines, brute force); none is "parity unpinned".
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* constants fixed by the paper or by the readings                      */
/* ------------------------------------------------------------------ */
#define OR_ZMIN (-1.0)                 /* ZNCC lower bound                 */
#define OR_CMAX (1.0 - OR_ZMIN)        /* Sec. III-C: C_max = 1 - Z_min    */
#define OR_EPS_C 1e-6                  /* reading: floor of C(x,j) in Eq.5 */
#define OR_TAU_VAR 1e-6                /* reading: flat-patch variance     */
#define OR_GRAZE 1e-3                  /* reading: grazing-plane limit     */
#define OR_PI 3.14159265358979323846

/* ------------------------------------------------------------------ */
/* scene                                                                */
/* ------------------------------------------------------------------ */
typedef struct {
    double K[9], Kinv[9], R[9], t[3];  /* x_cam = R X_world + t           */
    int W, H;
    const double* img;                 /* H*W intensities in [0,1]        */
} or_view;

typedef struct {
    int n;
    or_view* v;
} or_scene;

typedef struct {
    double win_radius;   /* r_orig                                          */
    int win_samples;     /* samples per axis n = 2 r_now + 1                */
    double sigma_s;      /* bilateral spatial sigma in px (<= 0: none)      */
    double sigma_c;      /* bilateral colour sigma, [0,1] scale (<= 0: none)*/
    double d_lo, d_hi;   /* depth range                                     */
    uint64_t seed;
    int n_prop;          /* learned proposals per pixel (0: none)           */
    const double* props; /* H*W*n_prop*4 planes (nx, ny, nz, d) or NULL     */
    const float* init_range; /* H*W*2 (d_min, d_max) of the sparse-feature
                                initialisation (NaN: none) or NULL          */
} or_pm;

static void m3_mul(const double* A, const double* B, double* C) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += A[3 * i + k] * B[3 * k + j];
            C[3 * i + j] = s;
        }
}
static void m3_vec(const double* A, const double* x, double* y) {
    for (int i = 0; i < 3; ++i) y[i] = A[3 * i] * x[0] + A[3 * i + 1] * x[1] + A[3 * i + 2] * x[2];
}
static void m3_tr(const double* A, double* T) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) T[3 * j + i] = A[3 * i + j];
}
static void m3_inv(const double* A, double* B) {
    double c00 = A[4] * A[8] - A[5] * A[7], c01 = A[5] * A[6] - A[3] * A[8], c02 = A[3] * A[7] - A[4] * A[6];
    double det = A[0] * c00 + A[1] * c01 + A[2] * c02;
    B[0] = c00 / det; B[1] = (A[2] * A[7] - A[1] * A[8]) / det; B[2] = (A[1] * A[5] - A[2] * A[4]) / det;
    B[3] = c01 / det; B[4] = (A[0] * A[8] - A[2] * A[6]) / det; B[5] = (A[2] * A[3] - A[0] * A[5]) / det;
    B[6] = c02 / det; B[7] = (A[1] * A[6] - A[0] * A[7]) / det; B[8] = (A[0] * A[4] - A[1] * A[3]) / det;
}
static double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void cross3(const double* a, const double* b, double* c) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

or_scene* or_scene_create(int n, const double* K, const double* R, const double* t,
                          const int* W, const int* H, const double* const* imgs) {
    or_scene* s = (or_scene*)calloc(1, sizeof(or_scene));
    s->n = n;
    s->v = (or_view*)calloc((size_t)n, sizeof(or_view));
    for (int i = 0; i < n; ++i) {
        memcpy(s->v[i].K, K + 9 * i, sizeof(double) * 9);
        memcpy(s->v[i].R, R + 9 * i, sizeof(double) * 9);
        memcpy(s->v[i].t, t + 3 * i, sizeof(double) * 3);
        m3_inv(s->v[i].K, s->v[i].Kinv);
        s->v[i].W = W[i];
        s->v[i].H = H[i];
        s->v[i].img = imgs ? imgs[i] : NULL;
    }
    return s;
}
void or_scene_destroy(or_scene* s) {
    if (!s) return;
    free(s->v);
    free(s);
}

/* relative pose of view j with respect to view r: X_j = Rr X_r + tr */
static void rel_pose(const or_scene* s, int r, int j, double* Rr, double* tr) {
    double RrT[9];
    m3_tr(s->v[r].R, RrT);
    m3_mul(s->v[j].R, RrT, Rr);
    double Rt[3];
    m3_vec(Rr, s->v[r].t, Rt);
    for (int i = 0; i < 3; ++i) tr[i] = s->v[j].t[i] - Rt[i];
}

/* ------------------------------------------------------------------ */
/* Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11), own implementation */
/* ------------------------------------------------------------------ */
void or_philox4x64(const uint64_t ctr_in[4], const uint64_t key_in[2], uint64_t out[4]) {
    uint64_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint64_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        unsigned __int128 p0 = (unsigned __int128)0xD2E7470EE14C6C93ULL * c0;
        unsigned __int128 p1 = (unsigned __int128)0xCA5A826395121157ULL * c2;
        uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
        uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
        uint64_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B97F4A7C15ULL;
        k1 += 0xBB67AE8584CAA73BULL;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* reading: a uniform draw uses the top 24 bits of a Philox word, so it is
 * exactly representable in single and double precision alike */
static double u24(uint64_t w) { return (double)(w >> 40) * (1.0 / 16777216.0); }

/* reading: counter = (pixel linear index, phase + 1, 0, 0) with phase = -1
 * for the initialisation, key = (seed, reference view index) */
static void draws(const or_pm* p, int ref, long pix, int phase, double u[3]) {
    uint64_t ctr[4] = {(uint64_t)pix, (uint64_t)(int64_t)(phase + 1), 0, 0};
    uint64_t key[2] = {p->seed, (uint64_t)ref};
    uint64_t o[4];
    or_philox4x64(ctr, key, o);
    u[0] = u24(o[0]);
    u[1] = u24(o[1]);
    u[2] = u24(o[2]);
}

/* ------------------------------------------------------------------ */
/* Sec. III-C: bilinear interpolation                                   */
/* ------------------------------------------------------------------ */
/* reading: pixel centres at integer coordinates; (u, v) must satisfy
 * 0 <= u <= W-1, 0 <= v <= H-1; taps past the last row/column are clamped
 * (they carry weight 0 there) */
static double bilin(const double* I, int W, int H, double u, double v) {
    int x0 = (int)floor(u), y0 = (int)floor(v);
    double fx = u - x0, fy = v - y0;
    int x1 = x0 + 1 < W ? x0 + 1 : W - 1;
    int y1 = y0 + 1 < H ? y0 + 1 : H - 1;
    double a = I[(long)y0 * W + x0], b = I[(long)y0 * W + x1];
    double c = I[(long)y1 * W + x0], d = I[(long)y1 * W + x1];
    return (1 - fy) * ((1 - fx) * a + fx * b) + fy * ((1 - fx) * c + fx * d);
}
double or_bilinear(const double* I, int W, int H, double u, double v) { return bilin(I, W, H, u, v); }

/* ------------------------------------------------------------------ */
/* Sec. III-C: the dilated support window                               */
/* ------------------------------------------------------------------ */
/* offsets s*k, k = -r_now..r_now in unit steps, s = r_orig / r_now,
 * n = 2 r_now + 1 samples per axis (r_now may be a half integer) */
void or_window_offsets(const or_pm* p, double* off) {
    int n = p->win_samples;
    double r_now = 0.5 * (n - 1);
    double s = p->win_radius / r_now;
    for (int k = 0; k < n; ++k) off[k] = s * ((double)k - r_now);
}

#define OR_MAXS 64   /* samples per axis */

typedef struct {
    int m;                          /* included samples                  */
    double ou[OR_MAXS * OR_MAXS];   /* offsets                           */
    double ov[OR_MAXS * OR_MAXS];
    double r[OR_MAXS * OR_MAXS];    /* I_ref(eta)                        */
    double w[OR_MAXS * OR_MAXS];    /* bilateral weight                  */
    double sum_w, mean_r, var_r;    /* weighted moments of the ref patch */
} or_window;

/* reading: samples of the window that fall outside the reference image are
 * left out of the window; reading: bilateral weight
 * w = exp(-|eta-x|^2 / 2 sigma_s^2) exp(-(I(eta)-I(x))^2 / 2 sigma_c^2) */
static void ref_window(const or_scene* s, int ref, const or_pm* p, int x, int y, or_window* win) {
    const or_view* V = &s->v[ref];
    double off[OR_MAXS];
    or_window_offsets(p, off);
    int n = p->win_samples;
    double rc = V->img[(long)y * V->W + x];
    win->m = 0;
    for (int kv = 0; kv < n; ++kv)
        for (int ku = 0; ku < n; ++ku) {
            double eu = x + off[ku], ev = y + off[kv];
            if (eu < 0 || eu > V->W - 1 || ev < 0 || ev > V->H - 1) continue;
            double rv = bilin(V->img, V->W, V->H, eu, ev);
            double w = 1.0;
            if (p->sigma_s > 0) w *= exp(-(off[ku] * off[ku] + off[kv] * off[kv]) / (2 * p->sigma_s * p->sigma_s));
            if (p->sigma_c > 0) w *= exp(-(rv - rc) * (rv - rc) / (2 * p->sigma_c * p->sigma_c));
            int i = win->m++;
            win->ou[i] = off[ku];
            win->ov[i] = off[kv];
            win->r[i] = rv;
            win->w[i] = w;
        }
    double sw = 0, swr = 0;
    for (int i = 0; i < win->m; ++i) { sw += win->w[i]; swr += win->w[i] * win->r[i]; }
    double mr = swr / sw, vr = 0;
    for (int i = 0; i < win->m; ++i) vr += win->w[i] * (win->r[i] - mr) * (win->r[i] - mr);
    win->sum_w = sw;
    win->mean_r = mr;
    win->var_r = vr / sw;
}

/* reading: a plane hypothesis (n, d) at pixel x is usable only if d > 0, the
 * normal faces the camera away from grazing (n.r < -1e-3 |r|) and the plane
 * lies in front of the reference camera at every included window sample */
static int hyp_valid(const or_scene* s, int ref, int x, int y, const double n[3], double d, const or_window* win) {
    const or_view* V = &s->v[ref];
    if (!(d > 0) || !isfinite(d)) return 0;
    double xt[3] = {(double)x, (double)y, 1.0}, r[3];
    m3_vec(V->Kinv, xt, r);
    if (!(dot3(n, r) < -OR_GRAZE * sqrt(dot3(r, r)))) return 0;
    for (int i = 0; i < win->m; ++i) {
        double et[3] = {x + win->ou[i], y + win->ov[i], 1.0}, re[3];
        m3_vec(V->Kinv, et, re);
        if (!(dot3(n, re) < 0)) return 0;
    }
    return 1;
}

/* plane-induced homography H = K_j (R + t n^T / rho) K_ref^-1, with
 * rho = n . X and X = d K_ref^-1 x (reading: d is the z-depth) */
void or_homography(const or_scene* s, int ref, int j, int x, int y, const double n[3], double d, double Hm[9]) {
    const or_view* V = &s->v[ref];
    double Rr[9], tr[3];
    rel_pose(s, ref, j, Rr, tr);
    double xt[3] = {(double)x, (double)y, 1.0}, r[3];
    m3_vec(V->Kinv, xt, r);
    double rho = d * dot3(n, r);
    double M[9], T[9];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) M[3 * a + b] = Rr[3 * a + b] + tr[a] * n[b] / rho;
    m3_mul(s->v[j].K, M, T);
    m3_mul(T, V->Kinv, Hm);
}

/* per-view cost C(x,j) = 1 - Z(x,j) (Eq. 4, two-pass weighted form).
 * Returns 1 when the view counts in Eq. 5, 0 when it is excluded:
 * a sample maps outside source j or behind it (Sec. III-C: C = C_max),
 * or (reading) either weighted variance is below 1e-6. */
static int view_cost(const or_scene* s, int ref, int j, const or_pm* p, int x, int y,
                     const double n[3], double d, const or_window* win, double* cj, double* margin) {
    (void)p;
    const or_view* S = &s->v[j];
    double Hm[9];
    or_homography(s, ref, j, x, y, n, d, Hm);
    double* sv = (double*)malloc(sizeof(double) * (size_t)(win->m > 0 ? win->m : 1));
    double mg = 1e300;
    int ok = 1;
    for (int i = 0; i < win->m && ok; ++i) {
        double et[3] = {x + win->ou[i], y + win->ov[i], 1.0}, q[3];
        m3_vec(Hm, et, q);
        if (!(q[2] > 0)) { ok = 0; break; }
        double u = q[0] / q[2], v = q[1] / q[2];
        double dm = fmin(fmin(u, S->W - 1 - u), fmin(v, S->H - 1 - v));
        if (fabs(dm) < mg) mg = fabs(dm);
        if (!(u >= 0 && u <= S->W - 1 && v >= 0 && v <= S->H - 1)) { ok = 0; break; }
        sv[i] = bilin(S->img, S->W, S->H, u, v);
    }
    if (ok) {
        double sw = win->sum_w, ss = 0;
        for (int i = 0; i < win->m; ++i) ss += win->w[i] * sv[i];
        double ms = ss / sw, vs = 0, cv = 0;
        for (int i = 0; i < win->m; ++i) {
            vs += win->w[i] * (sv[i] - ms) * (sv[i] - ms);
            cv += win->w[i] * (win->r[i] - win->mean_r) * (sv[i] - ms);
        }
        vs /= sw;
        cv /= sw;
        double fr = fabs(vs / OR_TAU_VAR - 1.0);
        if (fr < mg) mg = fr;
        if (vs < OR_TAU_VAR) ok = 0;
        else {
            double z = cv / sqrt(win->var_r * vs);
            if (z > 1) z = 1;
            if (z < -1) z = -1;
            *cj = 1.0 - z;
            /* decision margin of the delta(C, C_max) exclusion of Eq. 5: a view
             * within 1e-4 of C_max is a fragile decision (contributes < 1e-3) */
            double fc = (OR_CMAX - *cj) * 10.0;
            if (fc < mg) mg = fc;
        }
    }
    free(sv);
    if (margin) *margin = mg;
    if (!ok) *cj = OR_CMAX;
    return ok;
}

/* Eq. 5 with omega = 1 (reading), weight C(x,j)^-1 floored at 1e-6
 * (reading), views at C_max excluded by the delta term */
static double aggregate(int nv, const double* cj, const int* ok) {
    int cnt = 0;
    double inv = 0;
    for (int j = 0; j < nv; ++j)
        if (ok[j] && cj[j] < OR_CMAX) {
            cnt++;
            inv += 1.0 / fmax(cj[j], OR_EPS_C);
        }
    return cnt ? (double)cnt / inv : OR_CMAX;
}

/* cost of hypothesis (n, d) at pixel (x, y); also the smallest decision
 * margin met on the way (distance of a sample to a border in px, relative
 * distance of a variance to the flat limit, grazing distance) */
static double pixel_cost(const or_scene* s, int ref, const int* srcs, int ns, const or_pm* p, int x, int y,
                         const double n[3], double d, const or_window* win, double* cj_out, double* margin) {
    double cj[64];
    int ok[64];
    double mg = 1e300;
    if (win->var_r < OR_TAU_VAR || !hyp_valid(s, ref, x, y, n, d, win)) {
        for (int j = 0; j < ns; ++j) if (cj_out) cj_out[j] = OR_CMAX;
        if (margin) {
            double fr = fabs(win->var_r / OR_TAU_VAR - 1.0);
            *margin = fr;
        }
        return OR_CMAX;
    }
    for (int j = 0; j < ns; ++j) {
        double m1;
        ok[j] = view_cost(s, ref, srcs[j], p, x, y, n, d, win, &cj[j], &m1);
        if (m1 < mg) mg = m1;
        if (cj_out) cj_out[j] = cj[j];
    }
    if (margin) *margin = mg;
    return aggregate(ns, cj, ok);
}

/* Eq. 4/5 cost of n given planes (nx, ny, nz, d) at the pixels (xs[k], ys[k])
 * of the reference: the same as or_plane_cost at those pixels, without
 * touching the others (for sampled checks on large images) */
void or_cost_at(const or_scene* s, int ref, const int* srcs, int ns, const or_pm* p, int n, const int* xs,
                const int* ys, const double* planes, double* cost, double* margin_out) {
    or_window* win = (or_window*)malloc(sizeof(or_window));
    for (int k = 0; k < n; ++k) {
        double mg;
        ref_window(s, ref, p, xs[k], ys[k], win);
        cost[k] = pixel_cost(s, ref, srcs, ns, p, xs[k], ys[k], planes + 4 * k, planes[4 * k + 3], win, NULL, &mg);
        if (margin_out) margin_out[k] = mg;
    }
    free(win);
}

/* cost map of a given plane map; plane = H*W*4 (nx, ny, nz, d) */
void or_plane_cost(const or_scene* s, int ref, const int* srcs, int ns, const or_pm* p, const double* plane,
                   double* cost, double* view_cost_out, double* margin_out) {
    const or_view* V = &s->v[ref];
    or_window* win = (or_window*)malloc(sizeof(or_window));
    for (int y = 0; y < V->H; ++y)
        for (int x = 0; x < V->W; ++x) {
            long i = (long)y * V->W + x;
            ref_window(s, ref, p, x, y, win);
            double mg;
            cost[i] = pixel_cost(s, ref, srcs, ns, p, x, y, plane + 4 * i, plane[4 * i + 3], win,
                                 view_cost_out ? view_cost_out + (long)ns * i : NULL, &mg);
            if (margin_out) margin_out[i] = mg;
        }
    free(win);
}

/* Extent of each view's image of the window (a comparison diagnostic, not
 * part of the method): for every pixel and source view, the largest
 * distance max(|u_i - u_c|, |v_i - v_c|) in source pixels between the
 * projection of an included window sample and that of the pixel itself,
 * under the pixel's plane; 0 when the plane is not usable there or a sample
 * falls behind the source.  An implementation that evaluates the samples
 * relative to the projected centre in single precision carries position
 * errors proportional to this extent.  extent = H*W*ns. */
void or_window_extent(const or_scene* s, int ref, const int* srcs, int ns, const or_pm* p, const double* plane,
                      double* extent) {
    const or_view* V = &s->v[ref];
    or_window* win = (or_window*)malloc(sizeof(or_window));
    for (int y = 0; y < V->H; ++y)
        for (int x = 0; x < V->W; ++x) {
            long i = (long)y * V->W + x;
            ref_window(s, ref, p, x, y, win);
            const double* n = plane + 4 * i;
            const double d = plane[4 * i + 3];
            const int usable = hyp_valid(s, ref, x, y, n, d, win);
            for (int j = 0; j < ns; ++j) {
                double e = 0.0;
                if (usable) {
                    double Hm[9], c[3], q[3];
                    const double xc[3] = {(double)x, (double)y, 1.0};
                    or_homography(s, ref, srcs[j], x, y, n, d, Hm);
                    m3_vec(Hm, xc, c);
                    for (int k = 0; k < win->m; ++k) {
                        const double et[3] = {x + win->ou[k], y + win->ov[k], 1.0};
                        m3_vec(Hm, et, q);
                        if (!(q[2] > 0.0) || !(c[2] > 0.0)) {
                            e = 0.0;
                            break;
                        }
                        const double du = fabs(q[0] / q[2] - c[0] / c[2]), dv = fabs(q[1] / q[2] - c[1] / c[2]);
                        e = fmax(e, fmax(du, dv));
                    }
                }
                extent[(long)ns * i + j] = e;
            }
        }
    free(win);
}

/* weighted ZNCC of two given patches (Eq. 4 with weights); for tests */
double or_wzncc(int m, const double* w, const double* a, const double* b) {
    double sw = 0, sa = 0, sb = 0;
    for (int i = 0; i < m; ++i) { sw += w[i]; sa += w[i] * a[i]; sb += w[i] * b[i]; }
    double ma = sa / sw, mb = sb / sw, va = 0, vb = 0, cv = 0;
    for (int i = 0; i < m; ++i) {
        va += w[i] * (a[i] - ma) * (a[i] - ma);
        vb += w[i] * (b[i] - mb) * (b[i] - mb);
        cv += w[i] * (a[i] - ma) * (b[i] - mb);
    }
    return cv / sqrt(va * vb);
}
double or_aggregate(int nv, const double* cj, const int* ok) { return aggregate(nv, cj, ok); }

/* ------------------------------------------------------------------ */
/* Sec. III-B: random initialisation                                    */
/* ------------------------------------------------------------------ */
/* reading: normals are stored facing the camera (n . K^-1 x < 0) */
static void orient(const double r[3], double n[3]) {
    if (dot3(n, r) > 0) { n[0] = -n[0]; n[1] = -n[1]; n[2] = -n[2]; }
}
static void normal_from_angles(double th, double ph, double n[3]) {
    n[0] = cos(th) * sin(ph);
    n[1] = sin(th) * sin(ph);
    n[2] = cos(ph);
}

void or_init(const or_scene* s, int ref, const int* srcs, int ns, const or_pm* p, double* plane, double* cost) {
    const or_view* V = &s->v[ref];
    or_window* win = (or_window*)malloc(sizeof(or_window));
    for (int y = 0; y < V->H; ++y)
        for (int x = 0; x < V->W; ++x) {
            long i = (long)y * V->W + x;
            double u[3];
            draws(p, ref, i, -1, u);
            double d = p->d_lo + (p->d_hi - p->d_lo) * u[0];
            /* Sec. III-B: a depth drawn in [d_min, d_max] of the sparse features */
            if (p->init_range && p->init_range[2 * i] == p->init_range[2 * i]) {
                double lo = p->init_range[2 * i], hi = p->init_range[2 * i + 1];
                d = lo + (hi - lo) * u[0];
            }
            double th = 2 * OR_PI * u[1];
            double ph = OR_PI * (u[2] - 0.5);
            double n[3], xt[3] = {(double)x, (double)y, 1.0}, r[3];
            normal_from_angles(th, ph, n);
            m3_vec(V->Kinv, xt, r);
            orient(r, n);
            plane[4 * i] = n[0];
            plane[4 * i + 1] = n[1];
            plane[4 * i + 2] = n[2];
            plane[4 * i + 3] = d;
            if (cost) {
                ref_window(s, ref, p, x, y, win);
                cost[i] = pixel_cost(s, ref, srcs, ns, p, x, y, n, d, win, NULL, NULL);
            }
        }
    free(win);
}

/* ------------------------------------------------------------------ */
/* Sec. III / III-C: checkerboard propagation and random refinement      */
/* ------------------------------------------------------------------ */
/* reading (the cited improved red-black sampling is not described): eight
 * groups of other-colour neighbours; in each group the member with the
 * lowest stored cost is the candidate (first listed wins a tie).
 * Groups 0..3: near V-shapes towards up, down, left, right.
 * Groups 4..7: far lines at odd distances 5..25 towards up, down, left, right. */
static const int OR_NEAR_UP[6][2] = {{0, -1}, {-1, -2}, {1, -2}, {-2, -3}, {0, -3}, {2, -3}};

static int group_members(int g, int mem[16][2]) {
    if (g < 4) {
        for (int k = 0; k < 6; ++k) {
            int dx = OR_NEAR_UP[k][0], dy = OR_NEAR_UP[k][1];
            switch (g) {
                case 0: mem[k][0] = dx; mem[k][1] = dy; break;    /* up    */
                case 1: mem[k][0] = dx; mem[k][1] = -dy; break;   /* down  */
                case 2: mem[k][0] = dy; mem[k][1] = dx; break;    /* left  */
                default: mem[k][0] = -dy; mem[k][1] = dx; break;  /* right */
            }
        }
        return 6;
    }
    for (int k = 0; k < 11; ++k) {
        int dist = 5 + 2 * k;
        switch (g) {
            case 4: mem[k][0] = 0; mem[k][1] = -dist; break;
            case 5: mem[k][0] = 0; mem[k][1] = dist; break;
            case 6: mem[k][0] = -dist; mem[k][1] = 0; break;
            default: mem[k][0] = dist; mem[k][1] = 0; break;
        }
    }
    return 11;
}
int or_group_members(int g, int* out) {
    int mem[16][2];
    int c = group_members(g, mem);
    for (int k = 0; k < c; ++k) { out[2 * k] = mem[k][0]; out[2 * k + 1] = mem[k][1]; }
    return c;
}

/* one phase (half iteration): colour c = phase & 1, red = (x + y) even.
 * Only pixels of colour c change; they read the other colour's state.
 * Outputs (optional): per pixel the propagation winner (-1 keep, 0..7 group)
 * and refinement winner (-1 keep, 0..2), the gap between the two lowest
 * competing costs of each decision, and the smallest decision margin. */
void or_phase(const or_scene* s, int ref, const int* srcs, int ns, const or_pm* p, int phase,
              double* plane, double* cost, int* win_prop, double* gap_prop, int* win_ref, double* gap_ref,
              double* margin_out) {
    const or_view* V = &s->v[ref];
    int c = phase & 1;
    or_window* win = (or_window*)malloc(sizeof(or_window));
    for (int y = 0; y < V->H; ++y)
        for (int x = 0; x < V->W; ++x) {
            if (((x + y) & 1) != c) continue;
            long i = (long)y * V->W + x;
            ref_window(s, ref, p, x, y, win);
            double xt[3] = {(double)x, (double)y, 1.0}, rx[3];
            m3_vec(V->Kinv, xt, rx);
            double cur_n[3] = {plane[4 * i], plane[4 * i + 1], plane[4 * i + 2]};
            double cur_d = plane[4 * i + 3], cur_c = cost[i];
            double mg_all = 1e300, mg;

            /* propagation */
            double cand_c[8];
            int cand_ok[8];
            double cand_n[8][3], cand_d[8];
            for (int g = 0; g < 8; ++g) {
                int mem[16][2];
                int cnt = group_members(g, mem), best = -1;
                double bc = 0;
                for (int k = 0; k < cnt; ++k) {
                    int qx = x + mem[k][0], qy = y + mem[k][1];
                    if (qx < 0 || qx >= V->W || qy < 0 || qy >= V->H) continue;
                    double qc = cost[(long)qy * V->W + qx];
                    if (best < 0 || qc < bc) { best = k; bc = qc; }
                }
                cand_ok[g] = 0;
                if (best < 0) continue;
                long q = (long)(y + mem[best][1]) * V->W + (x + mem[best][0]);
                double nq[3] = {plane[4 * q], plane[4 * q + 1], plane[4 * q + 2]};
                double qt[3] = {(double)(x + mem[best][0]), (double)(y + mem[best][1]), 1.0}, rq[3];
                m3_vec(V->Kinv, qt, rq);
                /* reading: the neighbour's plane is carried over as a plane:
                 * rho_q = d_q n_q . K^-1 q, depth at x = rho_q / (n_q . K^-1 x);
                 * a transfer that does not face the camera or leaves the
                 * depth range is dropped */
                double rho = plane[4 * q + 3] * dot3(nq, rq);
                double den = dot3(nq, rx);
                if (!(den < 0)) continue;
                double dx = rho / den;
                if (!(dx >= p->d_lo && dx <= p->d_hi)) continue;
                cand_ok[g] = 1;
                memcpy(cand_n[g], nq, sizeof nq);
                cand_d[g] = dx;
                cand_c[g] = pixel_cost(s, ref, srcs, ns, p, x, y, nq, dx, win, NULL, &mg);
                if (mg < mg_all) mg_all = mg;
            }
            int bw = -1;
            double lo1 = cur_c, lo2 = 1e300;   /* two lowest competing values */
            double bestc = cur_c;
            for (int g = 0; g < 8; ++g) {
                if (!cand_ok[g]) continue;
                double v = cand_c[g];
                if (v < lo1) { lo2 = lo1; lo1 = v; } else if (v < lo2) lo2 = v;
                if (v < bestc) { bestc = v; bw = g; }
            }
            double gap = lo2 - lo1;
            if (bw >= 0) {
                memcpy(cur_n, cand_n[bw], sizeof cur_n);
                cur_d = cand_d[bw];
                cur_c = cand_c[bw];
            }

            /* learned proposals (no counterpart in the paper): the pixel's
             * n_prop given planes compete after the propagated ones, in
             * slot order, and replace the state only if strictly cheaper; a
             * slot whose depth lies outside [d_lo, d_hi] is skipped */
            if (p->n_prop > 0 && p->props) {
                int pw = -1;
                double pbest = cur_c, pn[3] = {0, 0, 0}, pd = 0;
                lo1 = cur_c; lo2 = 1e300;
                for (int k = 0; k < p->n_prop; ++k) {
                    const double* pr = p->props + 4 * ((long)i * p->n_prop + k);
                    if (!(pr[3] >= p->d_lo && pr[3] <= p->d_hi)) continue;
                    double v = pixel_cost(s, ref, srcs, ns, p, x, y, pr, pr[3], win, NULL, &mg);
                    if (mg < mg_all) mg_all = mg;
                    if (v < lo1) { lo2 = lo1; lo1 = v; } else if (v < lo2) lo2 = v;
                    if (v < pbest) { pbest = v; pw = k; memcpy(pn, pr, sizeof pn); pd = pr[3]; }
                }
                if (lo2 - lo1 < gap) gap = lo2 - lo1;
                if (pw >= 0) {
                    bw = 8 + pw;
                    memcpy(cur_n, pn, sizeof cur_n);
                    cur_d = pd;
                    cur_c = pbest;
                }
            }
            if (win_prop) win_prop[i] = bw;
            if (gap_prop) gap_prop[i] = gap;

            /* refinement (Sec. III-C): delta_d in [-d_max/4, d_max/4]
             * (reading: d_max = upper end of the depth range), delta_theta
             * in [-pi/2, pi/2], delta_phi in [-pi/12, pi/12] */
            double u[3];
            draws(p, ref, i, phase, u);
            double dd = (2 * u[0] - 1) * (p->d_hi / 4);
            double dth = (2 * u[1] - 1) * (OR_PI / 2);
            double dph = (2 * u[2] - 1) * (OR_PI / 12);
            double d_new = cur_d + dd;
            if (d_new < p->d_lo) d_new = p->d_lo;
            if (d_new > p->d_hi) d_new = p->d_hi;
            double m[3] = {cur_n[0], cur_n[1], cur_n[2]};
            if (m[2] < 0) { m[0] = -m[0]; m[1] = -m[1]; m[2] = -m[2]; }
            double th = atan2(m[1], m[0]);
            double ph = acos(m[2] > 1 ? 1 : (m[2] < -1 ? -1 : m[2]));
            double n_new[3];
            normal_from_angles(th + dth, ph + dph, n_new);
            orient(rx, n_new);
            double rn[3][3];
            double rd[3];
            memcpy(rn[0], cur_n, sizeof cur_n); rd[0] = d_new;
            memcpy(rn[1], n_new, sizeof n_new); rd[1] = cur_d;
            memcpy(rn[2], n_new, sizeof n_new); rd[2] = d_new;
            int rw = -1;
            double rbest = cur_c;
            lo1 = cur_c; lo2 = 1e300;
            double rc[3];
            for (int k = 0; k < 3; ++k) {
                rc[k] = pixel_cost(s, ref, srcs, ns, p, x, y, rn[k], rd[k], win, NULL, &mg);
                if (mg < mg_all) mg_all = mg;
                if (rc[k] < lo1) { lo2 = lo1; lo1 = rc[k]; } else if (rc[k] < lo2) lo2 = rc[k];
                if (rc[k] < rbest) { rbest = rc[k]; rw = k; }
            }
            if (win_ref) win_ref[i] = rw;
            if (gap_ref) gap_ref[i] = lo2 - lo1;
            if (margin_out) margin_out[i] = mg_all;
            if (rw >= 0) {
                memcpy(cur_n, rn[rw], sizeof cur_n);
                cur_d = rd[rw];
                cur_c = rc[rw];
            }
            plane[4 * i] = cur_n[0];
            plane[4 * i + 1] = cur_n[1];
            plane[4 * i + 2] = cur_n[2];
            plane[4 * i + 3] = cur_d;
            cost[i] = cur_c;
        }
    free(win);
}

/* full run: initialisation, then iterations of (red phase, black phase) */
void or_patchmatch(const or_scene* s, int ref, const int* srcs, int ns, const or_pm* p, int iters,
                   double* plane, double* cost) {
    or_init(s, ref, srcs, ns, p, plane, cost);
    for (int ph = 0; ph < 2 * iters; ++ph)
        or_phase(s, ref, srcs, ns, p, ph, plane, cost, NULL, NULL, NULL, NULL, NULL);
}

/* ------------------------------------------------------------------ */
/* Sec. III-D: geometric-consistency filter                             */
/* ------------------------------------------------------------------ */
typedef struct {
    double depth_tol;     /* 0.02                                           */
    int depth_relative;   /* reading: 0 = absolute difference (paper)       */
    double max_angle_deg; /* 30                                             */
    double max_reproj;    /* 1 px                                           */
    int min_consistent;   /* reading of "more than one": 2                  */
} or_filter;

/* planes[j] = H_j*W_j*4 map of view j (depth 0 = no depth).
 * reading: z-depth of X in view j is compared with the bilinear depth of
 * view j at x'_j; a tap without depth makes the view inconsistent; the
 * normal of view j is taken at the rounded coordinate, brought into the
 * reference frame and compared sign-agnostically */
/* Test support: margin_out (or NULL) receives per pixel the smallest
 * distance of any decision taken for it to that decision's boundary, in
 * units of a band: 1e-3 px for positions (image bounds, the reprojection
 * limit), 1e-5 for the depth test (in its own units), 1e-5 for the cosine of
 * the angle test.  A position within 1e-3 px of a pixel boundary of the
 * bilinear depth's tap cell, or of the nearest-pixel rounding of the normal
 * lookup, counts only where the neighbouring choice would change a decision
 * (a tap without depth, an angle test on the other side).  A pixel whose
 * margin is below 1 can be decided either way by a float evaluation of the
 * same tests. */
static double frac_dist(double a) {     /* distance of a to the nearest integer */
    double t = a - floor(a);
    return t < 0.5 ? t : 1.0 - t;
}

/* all four taps of the cell with corner (x0, y0) (clamped) have depth */
static int cell_has_depth(const double* Pj, int W, int H, int x0, int y0) {
    x0 = x0 < 0 ? 0 : (x0 > W - 1 ? W - 1 : x0);
    y0 = y0 < 0 ? 0 : (y0 > H - 1 ? H - 1 : y0);
    int x1 = x0 + 1 < W ? x0 + 1 : W - 1, y1 = y0 + 1 < H ? y0 + 1 : H - 1;
    return Pj[4 * ((long)y0 * W + x0) + 3] > 0 && Pj[4 * ((long)y0 * W + x1) + 3] > 0 &&
           Pj[4 * ((long)y1 * W + x0) + 3] > 0 && Pj[4 * ((long)y1 * W + x1) + 3] > 0;
}

void or_geo_filter(const or_scene* s, int ref, const int* srcs, int ns, const or_filter* f,
                   const double* const* planes, unsigned char* keep, int* count_out, double* margin_out) {
    const or_view* V = &s->v[ref];
    const double* P = planes[ref];
    double cos_max = cos(f->max_angle_deg * OR_PI / 180.0);
    for (int y = 0; y < V->H; ++y)
        for (int x = 0; x < V->W; ++x) {
            long i = (long)y * V->W + x;
            double d = P[4 * i + 3];
            int cnt = 0;
            double mg = 1e300;
#define OR_MG(v) do { double m_ = (v); if (m_ < mg) mg = m_; } while (0)
            if (d > 0) {
                double xt[3] = {(double)x, (double)y, 1.0}, r[3], X[3];
                m3_vec(V->Kinv, xt, r);
                for (int a = 0; a < 3; ++a) X[a] = d * r[a];
                for (int jj = 0; jj < ns; ++jj) {
                    int j = srcs[jj];
                    const or_view* S = &s->v[j];
                    const double* Pj = planes[j];
                    double Rr[9], tr[3], Xj[3], q[3];
                    rel_pose(s, ref, j, Rr, tr);
                    m3_vec(Rr, X, Xj);
                    for (int a = 0; a < 3; ++a) Xj[a] += tr[a];
                    if (!(Xj[2] > 0)) continue;
                    m3_vec(S->K, Xj, q);
                    double u = q[0] / q[2], v = q[1] / q[2];
                    OR_MG(fmin(fmin(fabs(u), fabs(S->W - 1 - u)), fmin(fabs(v), fabs(S->H - 1 - v))) / 1e-3);
                    if (!(u >= 0 && u <= S->W - 1 && v >= 0 && v <= S->H - 1)) continue;
                    int x0 = (int)floor(u), y0 = (int)floor(v);
                    {   /* a float position on the other side of a pixel boundary picks the
                         * neighbouring cell: fragile where its taps' depth presence differs */
                        const int here = cell_has_depth(Pj, S->W, S->H, x0, y0);
                        const int ax = u - x0 < 0.5 ? x0 - 1 : x0 + 1, ay = v - y0 < 0.5 ? y0 - 1 : y0 + 1;
                        if (frac_dist(u) < 1e-3 && cell_has_depth(Pj, S->W, S->H, ax, y0) != here) OR_MG(0.0);
                        if (frac_dist(v) < 1e-3 && cell_has_depth(Pj, S->W, S->H, x0, ay) != here) OR_MG(0.0);
                        if (frac_dist(u) < 1e-3 && frac_dist(v) < 1e-3 &&
                            cell_has_depth(Pj, S->W, S->H, ax, ay) != here) OR_MG(0.0);
                    }
                    int x1 = x0 + 1 < S->W ? x0 + 1 : S->W - 1, y1 = y0 + 1 < S->H ? y0 + 1 : S->H - 1;
                    double da = Pj[4 * ((long)y0 * S->W + x0) + 3], db = Pj[4 * ((long)y0 * S->W + x1) + 3];
                    double dc = Pj[4 * ((long)y1 * S->W + x0) + 3], de = Pj[4 * ((long)y1 * S->W + x1) + 3];
                    if (!(da > 0 && db > 0 && dc > 0 && de > 0)) continue;
                    double fx = u - x0, fy = v - y0;
                    double dj = (1 - fy) * ((1 - fx) * da + fx * db) + fy * ((1 - fx) * dc + fx * de);
                    double diff = fabs(dj - Xj[2]);
                    if (f->depth_relative) diff /= Xj[2];
                    OR_MG(fabs(diff - f->depth_tol) / 1e-5);
                    if (!(diff < f->depth_tol)) continue;
                    int xn = (int)floor(u + 0.5), yn = (int)floor(v + 0.5);
                    if (xn > S->W - 1) xn = S->W - 1;
                    if (yn > S->H - 1) yn = S->H - 1;
                    const double* nj = Pj + 4 * ((long)yn * S->W + xn);
                    double RrT[9], nr[3];
                    m3_tr(Rr, RrT);
                    m3_vec(RrT, nj, nr);
                    const double* nx = P + 4 * i;
                    double cs = fabs(dot3(nx, nr)) / sqrt(dot3(nx, nx) * dot3(nr, nr));
                    OR_MG(fabs(cs - cos_max) / 1e-5);
                    /* a float position on the other side of a rounding boundary takes the
                     * neighbouring pixel's normal: its angle test counts too */
                    for (int alt = 1; alt <= 3; ++alt) {
                        const int bx = (alt & 1) && frac_dist(u + 0.5) < 1e-3, by = (alt & 2) && frac_dist(v + 0.5) < 1e-3;
                        if (((alt & 1) && !bx) || ((alt & 2) && !by)) continue;
                        int xa = xn, ya = yn;
                        if (bx) xa = u + 0.5 - xn < 0.5 ? xn - 1 : xn + 1;
                        if (by) ya = v + 0.5 - yn < 0.5 ? yn - 1 : yn + 1;
                        xa = xa < 0 ? 0 : (xa > S->W - 1 ? S->W - 1 : xa);
                        ya = ya < 0 ? 0 : (ya > S->H - 1 ? S->H - 1 : ya);
                        double na[3];
                        m3_vec(RrT, Pj + 4 * ((long)ya * S->W + xa), na);
                        const double ca = fabs(dot3(nx, na)) / sqrt(dot3(nx, nx) * dot3(na, na));
                        OR_MG((ca > cos_max) != (cs > cos_max) ? 0.0 : fabs(ca - cos_max) / 1e-5);
                    }
                    if (!(cs > cos_max)) continue;
                    /* reprojection: back-project x'_j with d_j, into the reference */
                    double ut[3] = {u, v, 1.0}, rj[3], Y[3], Yr[3], qr[3];
                    m3_vec(S->Kinv, ut, rj);
                    for (int a = 0; a < 3; ++a) Y[a] = dj * rj[a] - tr[a];
                    m3_vec(RrT, Y, Yr);
                    if (!(Yr[2] > 0)) continue;
                    m3_vec(V->K, Yr, qr);
                    double eu = qr[0] / qr[2] - x, ev = qr[1] / qr[2] - y;
                    OR_MG(fabs(sqrt(eu * eu + ev * ev) - f->max_reproj) / 1e-3);
                    if (!(sqrt(eu * eu + ev * ev) < f->max_reproj)) continue;
                    cnt++;
                }
            }
#undef OR_MG
            if (margin_out) margin_out[i] = mg;
            if (count_out) count_out[i] = cnt;
            keep[i] = (unsigned char)(d > 0 && cnt >= f->min_consistent);
        }
}

/* ------------------------------------------------------------------ */
/* Sec. III-E: plane hypothesis inference                               */
/* ------------------------------------------------------------------ */
/* direction k of the 1D arrays: 0 horizontal, 1 vertical, 2 diagonal at
 * 45 degrees below (step (1,1)), 3 diagonal at 45 degrees above (step (1,-1)) */
static const int OR_DIR[4][2] = {{1, 0}, {0, 1}, {1, 1}, {1, -1}};

/* hypothesis of direction k at a hole: least-squares line depth = a + b t
 * through the n_fit reconstructed pixels closest along the line (t = step
 * index, hole at t = 0; reading: at equal distance the negative side comes
 * first); reading: invalid with fewer than two points or outside [d_lo, d_hi];
 * inverse != 0 fits 1/depth instead (option) */
static int line_hyp(const double* depth, const unsigned char* known, int W, int H, int x, int y, int k,
                    int n_fit, int inverse, double d_lo, double d_hi, double* h) {
    double ts[64], vs[64];
    int m = 0;
    int sx = OR_DIR[k][0], sy = OR_DIR[k][1];
    int lim = W > H ? W : H;
    for (int dist = 1; dist < lim && m < n_fit; ++dist)
        for (int side = -1; side <= 1 && m < n_fit; side += 2) {
            int qx = x + side * dist * sx, qy = y + side * dist * sy;
            if (qx < 0 || qx >= W || qy < 0 || qy >= H) continue;
            long q = (long)qy * W + qx;
            if (!known[q]) continue;
            ts[m] = side * dist;
            vs[m] = inverse ? 1.0 / depth[q] : depth[q];
            m++;
        }
    if (m < 2) return 0;
    double st = 0, sv = 0, stt = 0, stv = 0;
    for (int i = 0; i < m; ++i) { st += ts[i]; sv += vs[i]; stt += ts[i] * ts[i]; stv += ts[i] * vs[i]; }
    double den = m * stt - st * st;
    double b = (m * stv - st * sv) / den;
    double a = (sv - b * st) / m;
    double hv = inverse ? 1.0 / a : a;
    if (!(hv >= d_lo && hv <= d_hi)) return 0;
    *h = hv;
    return 1;
}

/* hyp: H*W*4 depths, valid: H*W*4 flags; only holes (known == 0) get
 * hypotheses */
void or_phi_hypotheses(int W, int H, const double* depth, const unsigned char* known, int n_fit, int inverse,
                       double d_lo, double d_hi, double* hyp, unsigned char* valid) {
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            long i = (long)y * W + x;
            for (int k = 0; k < 4; ++k) {
                double h = 0;
                int ok = !known[i] && line_hyp(depth, known, W, H, x, y, k, n_fit, inverse, d_lo, d_hi, &h);
                hyp[4 * i + k] = ok ? h : 0.0;
                valid[4 * i + k] = (unsigned char)ok;
            }
        }
}
double or_line_fit_at(const double* depth, const unsigned char* known, int W, int H, int x, int y, int k,
                      int n_fit, int inverse, double d_lo, double d_hi, int* ok) {
    double h = 0;
    *ok = line_hyp(depth, known, W, H, x, y, k, n_fit, inverse, d_lo, d_hi, &h);
    return h;
}

/* matching cost of each hypothesis: the back-projected point at depth h is
 * projected into the sources (Sec. III-E); this is the homography of the
 * fronto-parallel plane z = h, n = (0, 0, -1) (reading) */
void or_phi_cost(const or_scene* s, int ref, const int* srcs, int ns, const or_pm* p, const double* hyp,
                 const unsigned char* valid, double* hcost, double* margin_out) {
    const or_view* V = &s->v[ref];
    or_window* win = (or_window*)malloc(sizeof(or_window));
    double n[3] = {0, 0, -1};
    for (int y = 0; y < V->H; ++y)
        for (int x = 0; x < V->W; ++x) {
            long i = (long)y * V->W + x;
            int any = 0;
            for (int k = 0; k < 4; ++k) any |= valid[4 * i + k];
            if (any) ref_window(s, ref, p, x, y, win);
            for (int k = 0; k < 4; ++k) {
                double mg = 1e300;
                hcost[4 * i + k] = valid[4 * i + k]
                    ? pixel_cost(s, ref, srcs, ns, p, x, y, n, hyp[4 * i + k], win, NULL, &mg)
                    : OR_CMAX;
                if (margin_out) margin_out[4 * i + k] = mg;
            }
        }
    free(win);
}

/* Eq. 6 unary and Eq. 7 pairwise potentials */
double or_phi_unary(double c, double k1, double k2) { return (OR_CMAX - c) / k1 + k2; }
double or_phi_pair(double h1, double h2, double k3) {
    double rel = h1 > h2 ? (h1 - h2) / h2 : (h2 - h1) / h1;
    double t = k3 - (rel < 1 ? rel : 1);
    return t * t;
}

/* MRF over a grid of nodes (gw x gh), up to 4 labels per node.
 * nlab[i] = number of labels (0 = node absent), lab[4i+k] = depth of label k,
 * un[4i+k] = unary energy -log phi_n.  Pairwise energy -log phi_e (Eq. 7).
 * MAP of Eq. 8 = minimum of E = sum unary + sum pairwise.
 * reading: TRW is sequential tree-reweighted min-sum message passing
 * (monotonic chains = rows and columns, node weight 1 / max(#earlier
 * neighbours, #later neighbours)); one iteration = a forward pass in raster
 * order then a backward pass; decoding takes the argmin of each node's
 * belief (lowest label on a tie). msg[(4i+dir)*4 + l] = message INTO node i
 * from its neighbour in direction dir (0 up, 1 down, 2 left, 3 right). */
static const int OR_NB[4][2] = {{0, -1}, {0, 1}, {-1, 0}, {1, 0}};
static int opp(int dir) { return dir ^ 1; }

static void trw_node(int gw, int gh, const int* nlab, const double* lab, const double* un, double k3,
                     double* msg, int x, int y, int forward) {
    long i = (long)y * gw + x;
    int L = nlab[i];
    if (!L) return;
    double bel[4];
    for (int l = 0; l < L; ++l) {
        bel[l] = un[4 * i + l];
        for (int dir = 0; dir < 4; ++dir) bel[l] += msg[(4 * i + dir) * 4 + l];
    }
    int nb_before = 0, nb_after = 0;
    for (int dir = 0; dir < 4; ++dir) {
        int qx = x + OR_NB[dir][0], qy = y + OR_NB[dir][1];
        if (qx < 0 || qx >= gw || qy < 0 || qy >= gh || !nlab[(long)qy * gw + qx]) continue;
        if (dir == 0 || dir == 2) nb_before++; else nb_after++;
    }
    int mx = nb_before > nb_after ? nb_before : nb_after;
    double gamma = mx > 0 ? 1.0 / mx : 1.0;
    for (int dir = 0; dir < 4; ++dir) {
        int later = (dir == 1 || dir == 3);
        if (later != forward) continue;
        int qx = x + OR_NB[dir][0], qy = y + OR_NB[dir][1];
        if (qx < 0 || qx >= gw || qy < 0 || qy >= gh) continue;
        long q = (long)qy * gw + qx;
        int Lq = nlab[q];
        if (!Lq) continue;
        double out[4], mn = 1e300;
        for (int lq = 0; lq < Lq; ++lq) {
            double best = 1e300;
            for (int l = 0; l < L; ++l) {
                double e = gamma * bel[l] - msg[(4 * i + dir) * 4 + l]
                         - log(or_phi_pair(lab[4 * i + l], lab[4 * q + lq], k3));
                if (e < best) best = e;
            }
            out[lq] = best;
            if (best < mn) mn = best;
        }
        for (int lq = 0; lq < Lq; ++lq) msg[(4 * q + opp(dir)) * 4 + lq] = out[lq] - mn;
    }
}

void or_trw(int gw, int gh, const int* nlab, const double* lab, const double* un, double k3, int iters,
            double* msg, int* label) {
    memset(msg, 0, sizeof(double) * (size_t)gw * gh * 16);
    for (int it = 0; it < iters; ++it) {
        for (int y = 0; y < gh; ++y)
            for (int x = 0; x < gw; ++x) trw_node(gw, gh, nlab, lab, un, k3, msg, x, y, 1);
        for (int y = gh - 1; y >= 0; --y)
            for (int x = gw - 1; x >= 0; --x) trw_node(gw, gh, nlab, lab, un, k3, msg, x, y, 0);
    }
    for (long i = 0; i < (long)gw * gh; ++i) {
        int L = nlab[i];
        if (!L) { label[i] = -1; continue; }
        int best = 0;
        double bv = 1e300;
        for (int l = 0; l < L; ++l) {
            double b = un[4 * i + l];
            for (int dir = 0; dir < 4; ++dir) b += msg[(4 * i + dir) * 4 + l];
            if (b < bv) { bv = b; best = l; }
        }
        label[i] = best;
    }
}

double or_mrf_energy(int gw, int gh, const int* nlab, const double* lab, const double* un, double k3,
                     const int* label) {
    double e = 0;
    for (int y = 0; y < gh; ++y)
        for (int x = 0; x < gw; ++x) {
            long i = (long)y * gw + x;
            if (!nlab[i]) continue;
            e += un[4 * i + label[i]];
            for (int dir = 1; dir <= 3; dir += 2) {   /* down and right: each edge once */
                int qx = x + OR_NB[dir][0], qy = y + OR_NB[dir][1];
                if (qx >= gw || qy >= gh) continue;
                long q = (long)qy * gw + qx;
                if (!nlab[q]) continue;
                e -= log(or_phi_pair(lab[4 * i + label[i]], lab[4 * q + label[q]], k3));
            }
        }
    return e;
}

/* Eq. 10 normal at pixel (x,y) from the back-projected 4-neighbours;
 * reading: the norm in the denominator is taken unsquared, so the normal has
 * unit length, and it is oriented towards the camera.  Returns 0 if a
 * neighbour has no depth. */
static int eq10_normal(const or_view* V, const double* depth, int x, int y, double n[3]) {
    if (x < 1 || y < 1 || x > V->W - 2 || y > V->H - 2) return 0;
    int nx[4] = {x, x, x - 1, x + 1}, ny[4] = {y - 1, y + 1, y, y};   /* u, d, l, r */
    double P[4][3];
    for (int k = 0; k < 4; ++k) {
        double d = depth[(long)ny[k] * V->W + nx[k]];
        if (!(d > 0)) return 0;
        double xt[3] = {(double)nx[k], (double)ny[k], 1.0}, r[3];
        m3_vec(V->Kinv, xt, r);
        for (int a = 0; a < 3; ++a) P[k][a] = d * r[a];
    }
    double a[3], b[3];
    for (int k = 0; k < 3; ++k) { a[k] = P[0][k] - P[1][k]; b[k] = P[2][k] - P[3][k]; }
    cross3(a, b, n);
    double len = sqrt(dot3(n, n));
    if (!(len > 0)) return 0;
    for (int k = 0; k < 3; ++k) n[k] /= len;
    double xt[3] = {(double)x, (double)y, 1.0}, r[3];
    m3_vec(V->Kinv, xt, r);
    orient(r, n);
    return 1;
}
int or_eq10_normal(const or_scene* s, int ref, const double* depth, int x, int y, double* n) {
    return eq10_normal(&s->v[ref], depth, x, y, n);
}

typedef struct {
    double k1, k2, k3;     /* Eq. 6 / Eq. 7: 4, 0.5, 2                       */
    int n_fit;             /* six closest reconstructed pixels               */
    int inverse;           /* 0: fit depth (paper), 1: fit inverse depth     */
    int trw_iters;         /* 1                                              */
    int min_cost;          /* 0: MRF selection (PHI-MVS); 1: each hole takes
                              its valid hypothesis of minimal matching cost,
                              no MRF (PHI-MVS/M of Sec. IV, Table I)        */
} or_phi;

/* MRF stage of Sec. III-E from full-resolution inputs: nodes at pixels
 * (2i, 2j) (reading: half resolution by sub-sampling); a reconstructed pixel
 * is a one-label node carrying its depth, a hole carries its valid
 * hypotheses with unary -log phi_n (Eq. 6), a hole without hypotheses is
 * absent.  label_out[g] = chosen hypothesis index (0..3), -1 for a
 * reconstructed node, -2 for an absent node; gap_out[g] (optional) = belief
 * difference between the best and the second-best label (1e300 for one
 * label). */
void or_phi_mrf(int W, int H, const unsigned char* known, const double* depth, const double* hyp,
                const unsigned char* valid, const double* hcost, double k1, double k2, double k3, int iters,
                int* label_out, double* gap_out) {
    int gw = (W + 1) / 2, gh = (H + 1) / 2;
    long G = (long)gw * gh;
    int* nlab = (int*)calloc((size_t)G, sizeof(int));
    double* lab = (double*)calloc((size_t)G * 4, sizeof(double));
    double* un = (double*)calloc((size_t)G * 4, sizeof(double));
    int* lmap = (int*)calloc((size_t)G * 4, sizeof(int));
    for (int gy = 0; gy < gh; ++gy)
        for (int gx = 0; gx < gw; ++gx) {
            long g = (long)gy * gw + gx, i = (long)(2 * gy) * W + 2 * gx;
            if (known[i]) {
                nlab[g] = 1;
                lab[4 * g] = depth[i];
                un[4 * g] = 0.0;
                lmap[4 * g] = -1;
                continue;
            }
            int L = 0;
            for (int k = 0; k < 4; ++k)
                if (valid[4 * i + k]) {
                    lab[4 * g + L] = hyp[4 * i + k];
                    un[4 * g + L] = -log(or_phi_unary(hcost[4 * i + k], k1, k2));
                    lmap[4 * g + L] = k;
                    L++;
                }
            nlab[g] = L;
        }
    double* msg = (double*)malloc(sizeof(double) * G * 16);
    int* label = (int*)malloc(sizeof(int) * G);
    or_trw(gw, gh, nlab, lab, un, k3, iters, msg, label);
    for (long g = 0; g < G; ++g) {
        label_out[g] = nlab[g] ? lmap[4 * g + label[g]] : -2;
        if (gap_out) {
            double b1 = 1e300, b2 = 1e300;
            for (int l = 0; l < nlab[g]; ++l) {
                double b = un[4 * g + l];
                for (int dir = 0; dir < 4; ++dir) b += msg[(4 * g + dir) * 4 + l];
                if (b < b1) { b2 = b1; b1 = b; } else if (b < b2) b2 = b;
            }
            gap_out[g] = b2 - b1;
        }
    }
    free(nlab); free(lab); free(un); free(lmap); free(msg); free(label);
}

/* Last step of Sec. III-E for the chosen depths newd: each hole with a
 * depth and four neighbours with depth gets its Eq. 10 normal and becomes a
 * plane (n, d); any other hole is zeroed.  Reconstructed pixels keep their
 * plane. */
static void phi_fill_holes(const or_view* V, const unsigned char* known, const double* newd, double* plane,
                           unsigned char* filled_out) {
    int W = V->W, H = V->H;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            long i = (long)y * W + x;
            unsigned char filled = 0;
            if (!known[i]) {
                double n[3];
                if (newd[i] > 0 && eq10_normal(V, newd, x, y, n)) {
                    plane[4 * i] = n[0]; plane[4 * i + 1] = n[1]; plane[4 * i + 2] = n[2];
                    plane[4 * i + 3] = newd[i];
                    filled = 1;
                } else {
                    plane[4 * i] = plane[4 * i + 1] = plane[4 * i + 2] = plane[4 * i + 3] = 0.0;
                }
            }
            if (filled_out) filled_out[i] = filled;
        }
}

/* Selection stage of Sec. III-E: the decoded depth of node (x/2, y/2)
 * (nearest up-sampling) is the reference; each hole takes its valid
 * hypothesis closest to it (lowest k on a tie); then Eq. 10 normals for the
 * filled pixels.  plane (in/out): reconstructed pixels keep their plane,
 * holes get (n, d) or zeros. */
void or_phi_select(const or_scene* s, int ref, const unsigned char* known, const double* hyp,
                   const unsigned char* valid, const int* label, double* plane, unsigned char* filled_out,
                   double* refdepth_out) {
    const or_view* V = &s->v[ref];
    int W = V->W, H = V->H, gw = (W + 1) / 2;
    long N = (long)W * H;
    double* newd = (double*)calloc((size_t)N, sizeof(double));
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            long i = (long)y * W + x, g = (long)(y / 2) * gw + (x / 2);
            long ni = (long)(2 * (y / 2)) * W + 2 * (x / 2);
            int lb = label[g];
            double rd = lb == -1 ? plane[4 * ni + 3] : (lb >= 0 ? hyp[4 * ni + lb] : 0.0);
            if (refdepth_out) refdepth_out[i] = rd;
            if (known[i]) { newd[i] = plane[4 * i + 3]; continue; }
            if (lb < -1) continue;
            int bk = -1;
            double bd = 1e300;
            for (int k = 0; k < 4; ++k)
                if (valid[4 * i + k]) {
                    double e = fabs(hyp[4 * i + k] - rd);
                    if (e < bd) { bd = e; bk = k; }
                }
            if (bk >= 0) newd[i] = hyp[4 * i + bk];
        }
    phi_fill_holes(V, known, newd, plane, filled_out);
    free(newd);
}

/* Selection of PHI-MVS/M (Sec. IV, Table I: the MRF removed): each hole
 * takes, among its valid hypotheses, the one of minimal matching cost hcost
 * (the lowest k on a tie); a hole without a valid hypothesis stays empty.
 * Then Eq. 10 normals as in or_phi_select. */
void or_phi_select_min_cost(const or_scene* s, int ref, const unsigned char* known, const double* hyp,
                            const unsigned char* valid, const double* hcost, double* plane,
                            unsigned char* filled_out) {
    const or_view* V = &s->v[ref];
    long N = (long)V->W * V->H;
    double* newd = (double*)calloc((size_t)N, sizeof(double));
    for (long i = 0; i < N; ++i) {
        if (known[i]) { newd[i] = plane[4 * i + 3]; continue; }
        int bk = -1;
        for (int k = 0; k < 4; ++k)
            if (valid[4 * i + k] && (bk < 0 || hcost[4 * i + k] < hcost[4 * i + bk])) bk = k;
        if (bk >= 0) newd[i] = hyp[4 * i + bk];
    }
    phi_fill_holes(V, known, newd, plane, filled_out);
    free(newd);
}


/* The whole PHI step for one reference view: hypotheses, their costs, MRF,
 * selection and Eq. 10 normals (q->min_cost: the minimal-cost selection in
 * place of MRF and closest-hypothesis selection; label_out is then -3
 * everywhere).  plane (in/out) H*W*4; known H*W (1 = reconstructed, kept).
 * Intermediate results go to the optional outputs. */
void or_plane_infer(const or_scene* s, int ref, const int* srcs, int ns, const or_pm* p, const or_phi* q,
                    const unsigned char* known, double* plane, double* hyp_out, unsigned char* valid_out,
                    double* hcost_out, int* label_out, double* refdepth_out, unsigned char* filled_out) {
    const or_view* V = &s->v[ref];
    int W = V->W, H = V->H;
    long N = (long)W * H;
    long G = (long)((W + 1) / 2) * ((H + 1) / 2);
    double* depth = (double*)malloc(sizeof(double) * N);
    for (long i = 0; i < N; ++i) depth[i] = known[i] ? plane[4 * i + 3] : 0.0;
    double* hyp = (double*)malloc(sizeof(double) * 4 * N);
    unsigned char* valid = (unsigned char*)malloc(4 * N);
    double* hcost = (double*)malloc(sizeof(double) * 4 * N);
    int* label = (int*)malloc(sizeof(int) * G);
    or_phi_hypotheses(W, H, depth, known, q->n_fit, q->inverse, p->d_lo, p->d_hi, hyp, valid);
    or_phi_cost(s, ref, srcs, ns, p, hyp, valid, hcost, NULL);
    for (long i = 0; i < N; ++i)
        if (known[i]) plane[4 * i + 3] = depth[i];
    if (q->min_cost) {
        for (long g = 0; g < G; ++g) label[g] = -3;      /* no MRF */
        if (refdepth_out) memset(refdepth_out, 0, sizeof(double) * N);
        or_phi_select_min_cost(s, ref, known, hyp, valid, hcost, plane, filled_out);
    } else {
        or_phi_mrf(W, H, known, depth, hyp, valid, hcost, q->k1, q->k2, q->k3, q->trw_iters, label, NULL);
        or_phi_select(s, ref, known, hyp, valid, label, plane, filled_out, refdepth_out);
    }
    if (hyp_out) memcpy(hyp_out, hyp, sizeof(double) * 4 * N);
    if (valid_out) memcpy(valid_out, valid, 4 * N);
    if (hcost_out) memcpy(hcost_out, hcost, sizeof(double) * 4 * N);
    if (label_out) memcpy(label_out, label, sizeof(int) * G);
    free(depth); free(hyp); free(valid); free(hcost); free(label);
}

/* ------------------------------------------------------------------ */
/* Sec. III-F: depth-map fusion                                         */
/* ------------------------------------------------------------------ */
/* Everything is computed in double precision:
 *   back-projection of pixel (x, y) of view v with z-depth d (pinhole,
 *   x_cam = R X + t): X = R^T (d K^-1 (x, y, 1)^T - t);
 *   projection into view j: c = R X + t, (u, v) = (K c)_{0,1} / c_2 when
 *   c_2 > 0, pixel [x'_j] = (floor(u + 1/2), floor(v + 1/2)) (reading: the
 *   nearest pixel) when it lies in the image;
 *   relative difference (reading: distance over the z-depth d_i of X_i in
 *   view i): |X_i - X'_j| < rel_tol d_i;
 *   merged point: (X_i + X'_j1 + X'_j2 + ...) / count, summed in view order.
 *
 * Fragile decisions.  Another implementation that rounds differently can
 * take a decision the other way when it lies within rounding of its
 * boundary: a projection whose u + 1/2 or v + 1/2 is within band_px of an
 * integer (two or four candidate pixels), or a distance within
 * band_rel rel_tol d_i of the threshold (merge or not).  Such a decision is
 * counted.  When `hint` gives that implementation's result (the point index
 * each pixel went into, laid out as `owner` below), a fragile decision takes
 * the outcome the hint shows, if that outcome is one of the possible ones;
 * every other decision is this function's own. */
static void fuse_backproject(const or_view* V, int x, int y, double d, double X[3]) {
    const double xt[3] = {(double)x, (double)y, 1.0};
    double r[3], e[3];
    m3_vec(V->Kinv, xt, r);
    for (int k = 0; k < 3; ++k) e[k] = d * r[k] - V->t[k];
    for (int k = 0; k < 3; ++k) X[k] = V->R[k] * e[0] + V->R[3 + k] * e[1] + V->R[6 + k] * e[2];
}

/* candidate pixels of the projection of X into view V: cand[0] is the
 * nearest pixel, the others the alternatives within band_px of a rounding
 * boundary; -1 = outside the image or behind the camera.  Returns the number
 * of candidates (1, 2 or 4). */
static int fuse_candidates(const or_view* V, const double X[3], double band_px, long cand[4]) {
    double c[3], q[3];
    m3_vec(V->R, X, c);
    for (int k = 0; k < 3; ++k) c[k] += V->t[k];
    if (!(c[2] > 0.0)) {
        cand[0] = -1;
        return 1;
    }
    m3_vec(V->K, c, q);
    const double uu = q[0] / q[2] + 0.5, vv = q[1] / q[2] + 0.5;
    const double fu = floor(uu), fv = floor(vv);
    double cu[2] = {fu, fu}, cv[2] = {fv, fv};
    int nu = 1, nv = 1;
    if (uu - fu < band_px) cu[nu++] = fu - 1.0;
    else if (fu + 1.0 - uu < band_px) cu[nu++] = fu + 1.0;
    if (vv - fv < band_px) cv[nv++] = fv - 1.0;
    else if (fv + 1.0 - vv < band_px) cv[nv++] = fv + 1.0;
    int m = 0;
    for (int b = 0; b < nv; ++b)
        for (int a = 0; a < nu; ++a) {
            const double px = cu[a], py = cv[b];
            cand[m++] = (px >= 0.0 && px <= (double)(V->W - 1) && py >= 0.0 && py <= (double)(V->H - 1))
                            ? (long)py * V->W + (long)px
                            : -1;
        }
    return m;
}

/* Fusion of the depth maps of views order[0..n-1], in that order (Sec. III-F):
 * every remaining pixel x of image i (depth > 0, kept by keep[a] when given,
 * not merged before) is back-projected to X_i; for every remaining image j
 * the pixel [x'_j] that X_i projects to is back-projected to X'_j, and when
 * the relative difference is below rel_tol that pixel is merged (removed
 * from image j) and X'_j joins the average; after its pixels, image i is
 * removed.  planes[a] and keep[a] belong to view order[a] (keep NULL or
 * keep[a] NULL: every pixel with depth).  Points are emitted in view order,
 * then raster order: pts[4k..4k+3] = (x, y, z, number of merged pixels),
 * src_view[k], src_pix[k] = the emitting pixel; at most cap points are
 * written and the number of points is returned.  owner (optional): one
 * entry per pixel of the views, view after view in `order`, the index of
 * the point the pixel went into, -1 if never present.  hint (optional): the
 * same layout from another implementation, consulted at fragile decisions
 * only.  stats (optional): [0] projections tested, [1] fragile decisions,
 * [2] fragile decisions resolved by the hint. */
long or_fuse(const or_scene* s, int n, const int* order, const double* const* planes,
             const unsigned char* const* keep, double rel_tol, double band_px, double band_rel, const long* hint,
             double* pts, int* src_view, long* src_pix, long* owner, long cap, long* stats) {
    unsigned char** alive = (unsigned char**)calloc((size_t)n, sizeof(unsigned char*));
    long* base = (long*)calloc((size_t)n + 1, sizeof(long));
    for (int a = 0; a < n; ++a) {
        const or_view* V = &s->v[order[a]];
        long N = (long)V->W * V->H;
        base[a + 1] = base[a] + N;
        alive[a] = (unsigned char*)malloc((size_t)N);
        for (long i = 0; i < N; ++i)
            alive[a][i] = (unsigned char)(planes[a][4 * i + 3] > 0.0 && (!keep || !keep[a] || keep[a][i]));
    }
    if (owner)
        for (long i = 0; i < base[n]; ++i) owner[i] = -1;
    long st[3] = {0, 0, 0};
    long np = 0;
    for (int a = 0; a < n; ++a) {
        const or_view* V = &s->v[order[a]];
        for (int y = 0; y < V->H; ++y)
            for (int x = 0; x < V->W; ++x) {
                long i = (long)y * V->W + x;
                if (!alive[a][i]) continue;
                double d = planes[a][4 * i + 3];
                double X[3], sum[3];
                fuse_backproject(V, x, y, d, X);
                for (int k = 0; k < 3; ++k) sum[k] = X[k];
                int cnt = 1;
                const double thr = rel_tol * d;
                for (int b = a + 1; b < n; ++b) {
                    const or_view* S = &s->v[order[b]];
                    long cand[4];
                    const int m = fuse_candidates(S, X, band_px, cand);
                    /* outcome of each candidate: merge it (firm or fragile)
                     * or not (firm or fragile) */
                    int can_merge[4], can_skip[4];
                    double Ys[4][3];
                    int n_merge = 0, any_skip = 0;
                    for (int c = 0; c < m; ++c) {
                        can_merge[c] = can_skip[c] = 0;
                        const long t = cand[c];
                        if (t < 0 || !alive[b][t]) {
                            can_skip[c] = 1;
                        } else {
                            fuse_backproject(S, (int)(t % S->W), (int)(t / S->W), planes[b][4 * t + 3], Ys[c]);
                            const double e0 = X[0] - Ys[c][0], e1 = X[1] - Ys[c][1], e2 = X[2] - Ys[c][2];
                            const double dist = sqrt(e0 * e0 + e1 * e1 + e2 * e2);
                            can_merge[c] = dist < thr + band_rel * thr;
                            can_skip[c] = !(dist < thr - band_rel * thr);
                        }
                        n_merge += can_merge[c];
                        any_skip |= can_skip[c];
                    }
                    st[0]++;
                    /* this function's own outcome: the nearest pixel, its
                     * distance against the threshold itself */
                    int pick = -1;
                    if (cand[0] >= 0 && alive[b][cand[0]]) {
                        const double e0 = X[0] - Ys[0][0], e1 = X[1] - Ys[0][1], e2 = X[2] - Ys[0][2];
                        if (sqrt(e0 * e0 + e1 * e1 + e2 * e2) < thr) pick = 0;
                    }
                    if (n_merge + any_skip > 1) {
                        st[1]++;
                        if (hint) {
                            int h = -2;
                            for (int c = 0; c < m && h == -2; ++c)
                                if (can_merge[c] && hint[base[b] + cand[c]] == np) h = c;
                            if (h == -2 && any_skip) {
                                int taken = 0;
                                for (int c = 0; c < m; ++c)
                                    if (cand[c] >= 0 && hint[base[b] + cand[c]] == np) taken = 1;
                                if (!taken) h = -1;
                            }
                            if (h != -2) {
                                if (h != pick) st[2]++;
                                pick = h;
                            }
                        }
                    }
                    if (pick < 0) continue;
                    const long t = cand[pick];
                    alive[b][t] = 0;
                    if (owner) owner[base[b] + t] = np;
                    for (int k = 0; k < 3; ++k) sum[k] = sum[k] + Ys[pick][k];
                    cnt++;
                }
                alive[a][i] = 0;
                if (owner) owner[base[a] + i] = np;
                if (np < cap) {
                    for (int k = 0; k < 3; ++k) pts[4 * np + k] = sum[k] / (double)cnt;
                    pts[4 * np + 3] = (double)cnt;
                    if (src_view) src_view[np] = order[a];
                    if (src_pix) src_pix[np] = i;
                }
                np++;
            }
    }
    if (stats)
        for (int k = 0; k < 3; ++k) stats[k] = st[k];
    for (int a = 0; a < n; ++a) free(alive[a]);
    free(alive);
    free(base);
    return np;
}

/* ------------------------------------------------------------------ */
/* Sec. III-A: neighbouring-image selection (Eqs. 1-3)                  */
/* ------------------------------------------------------------------ */
/* For reference image i and every other image j, A = the sparse points
 * visible in both; Eq. 1 disturbs each X in A along the ray from the
 * centre C_i, X^ = (1 + eps) X - eps C_i; Eq. 2 averages the displacement
 * of its projection into j, tau = mean |x^'_j - x'_j|; Eq. 3 scores
 * zeta = (1 / N_A) min(b_ij, 0.1) min(theta_ij, 0.05) with b_ij the
 * baseline and theta_ij the angle between the principal axes (reading:
 * radians).  Images with tau < t_tau or no shared point are removed (zeta
 * reported as +inf); the rest are sorted by zeta from small to large (tie:
 * lower index) and the first k kept.  X: 3 doubles per point; vis[p * n + v]
 * = 1 when point p is visible in view v.  Outputs: nbr[i * k + r] (-1 past
 * the kept ones), tau / zeta / n_shared [i * n + j] (NULL: not written). */
void or_select_neighbors(const or_scene* s, long n_pts, const double* X, const unsigned char* vis, double eps,
                         double t_tau, int k, int* nbr, double* tau_out, int* na_out, double* zeta_out) {
    const int n = s->n;
    double* C = (double*)malloc(sizeof(double) * 3 * n);
    for (int v = 0; v < n; ++v) {
        const double* R = s->v[v].R;
        const double* t = s->v[v].t;
        for (int a = 0; a < 3; ++a) C[3 * v + a] = -(R[a] * t[0] + R[3 + a] * t[1] + R[6 + a] * t[2]);
    }
    double* zeta = (double*)malloc(sizeof(double) * n);
    int* cand = (int*)malloc(sizeof(int) * n);
    for (int i = 0; i < n; ++i) {
        const double* Ci = C + 3 * i;
        const double* Ri = s->v[i].R;
        int nc = 0;
        for (int j = 0; j < n; ++j) {
            zeta[j] = INFINITY;
            if (j == i) continue;
            const or_view* Vj = &s->v[j];
            long na = 0;
            double sum = 0.0;
            for (long p = 0; p < n_pts; ++p) {
                if (!vis[p * n + i] || !vis[p * n + j]) continue;
                const double* Xp = X + 3 * p;
                double Xh[3], c[3], ch[3], q[3], qh[3];
                for (int a = 0; a < 3; ++a) Xh[a] = (1.0 + eps) * Xp[a] - eps * Ci[a];
                m3_vec(Vj->R, Xp, c);
                m3_vec(Vj->R, Xh, ch);
                for (int a = 0; a < 3; ++a) { c[a] += Vj->t[a]; ch[a] += Vj->t[a]; }
                m3_vec(Vj->K, c, q);
                m3_vec(Vj->K, ch, qh);
                double du = qh[0] / qh[2] - q[0] / q[2], dv = qh[1] / qh[2] - q[1] / q[2];
                sum += sqrt(du * du + dv * dv);
                na++;
            }
            double tau = na ? sum / (double)na : 0.0;
            const double* Cj = C + 3 * j;
            double db[3] = {Ci[0] - Cj[0], Ci[1] - Cj[1], Ci[2] - Cj[2]};
            double b = sqrt(dot3(db, db));
            double cs = Ri[6] * Vj->R[6] + Ri[7] * Vj->R[7] + Ri[8] * Vj->R[8];
            double th = acos(cs > 1.0 ? 1.0 : (cs < -1.0 ? -1.0 : cs));
            if (na > 0 && tau >= t_tau) {
                zeta[j] = (1.0 / (double)na) * (b < 0.1 ? b : 0.1) * (th < 0.05 ? th : 0.05);
                cand[nc++] = j;
            }
            if (tau_out) tau_out[(long)i * n + j] = tau;
            if (na_out) na_out[(long)i * n + j] = (int)na;
            if (zeta_out) zeta_out[(long)i * n + j] = zeta[j];
        }
        if (tau_out) tau_out[(long)i * n + i] = 0.0;
        if (na_out) na_out[(long)i * n + i] = 0;
        if (zeta_out) zeta_out[(long)i * n + i] = INFINITY;
        /* sort by (zeta, index): insertion sort */
        for (int a = 1; a < nc; ++a) {
            int c = cand[a], b = a - 1;
            while (b >= 0 && (zeta[cand[b]] > zeta[c] || (zeta[cand[b]] == zeta[c] && cand[b] > c))) {
                cand[b + 1] = cand[b];
                b--;
            }
            cand[b + 1] = c;
        }
        for (int r = 0; r < k; ++r) nbr[(long)i * k + r] = r < nc ? cand[r] : -1;
    }
    free(C); free(zeta); free(cand);
}

/* ------------------------------------------------------------------ */
/* Sec. III-B: depth initialisation from sparse feature points           */
/* ------------------------------------------------------------------ */
/* Features of view ref: the sparse 3D points visible in it whose
 * re-projection error is below max_reproj (reading: the point's mean error
 * over its views) and that are visible in at least floor(v - 1) images, v
 * the mean number of images per point.  Each keeps its observation in ref
 * (uv) and its z-depth in ref.  vis[p * n + v] = 1 when point p is visible
 * in view v; obs[2p..2p+1] = its observation in ref.  Writes uv[2k..],
 * depth[k] in point order and returns the number of features. */
long or_sparse_features(const or_scene* s, int ref, long n_pts, const double* X, const unsigned char* vis,
                        const double* reproj, const double* obs, double max_reproj, double* uv, double* depth) {
    const int n = s->n;
    long total = 0;
    for (long p = 0; p < n_pts; ++p)
        for (int v = 0; v < n; ++v) total += vis[p * n + v] ? 1 : 0;
    const double vbar = n_pts ? (double)total / (double)n_pts : 0.0;
    const int min_views = (int)floor(vbar - 1.0);
    const double* R = s->v[ref].R;
    const double* t = s->v[ref].t;
    long k = 0;
    for (long p = 0; p < n_pts; ++p) {
        int cnt = 0;
        for (int v = 0; v < n; ++v) cnt += vis[p * n + v] ? 1 : 0;
        if (!vis[p * n + ref] || !(reproj[p] < max_reproj) || cnt < min_views) continue;
        const double* Xp = X + 3 * p;
        uv[2 * k] = obs[2 * p];
        uv[2 * k + 1] = obs[2 * p + 1];
        depth[k] = R[6] * Xp[0] + R[7] * Xp[1] + R[8] * Xp[2] + t[2];
        k++;
    }
    return k;
}

/* Per pixel of a W x H view, the closest feature in each of the four
 * quadrants around it (dx >= 0, dy >= 0 / dx < 0, dy >= 0 / dx < 0, dy < 0 /
 * dx >= 0, dy < 0 with dx = u - x, dy = v - y) within w / 10 pixels, and the
 * minimum and maximum depth over those features, clamped to [d_lo, d_hi]
 * (reading); NaN when no feature is that close.  The first feature wins a
 * tie.  range[2i], range[2i+1] = d_min, d_max.
 * fragile[i] (optional) = 1 when the pixel's choice lies within band_px of
 * a boundary, where an implementation that rounds the positions or the
 * distances differently may decide otherwise: a feature within band_px of
 * the radius, a counted feature within band_px of a quadrant border, or a
 * quadrant whose two closest features are within band_px in distance. */
void or_sparse_range(int W, int H, long n_feat, const double* uv, const double* depth, double d_lo, double d_hi,
                     double band_px, double* range, unsigned char* fragile) {
    const double r = (double)W / 10.0;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            double best[4] = {INFINITY, INFINITY, INFINITY, INFINITY};
            double second[4] = {INFINITY, INFINITY, INFINITY, INFINITY};
            double bd[4] = {0, 0, 0, 0};
            int frag = 0;
            for (long f = 0; f < n_feat; ++f) {
                const double dx = uv[2 * f] - (double)x, dy = uv[2 * f + 1] - (double)y;
                const double d2 = dx * dx + dy * dy;
                const double dist = sqrt(d2);
                if (fabs(dist - r) < band_px) frag = 1;
                if (!(d2 < r * r)) continue;
                if (fabs(dx) < band_px || fabs(dy) < band_px) frag = 1;
                const int q = dx >= 0.0 ? (dy >= 0.0 ? 0 : 3) : (dy >= 0.0 ? 1 : 2);
                if (dist < best[q]) {
                    second[q] = best[q];
                    best[q] = dist;
                    bd[q] = depth[f];
                } else if (dist < second[q]) {
                    second[q] = dist;
                }
            }
            double lo = INFINITY, hi = -INFINITY;
            for (int q = 0; q < 4; ++q)
                if (best[q] < INFINITY) {
                    lo = bd[q] < lo ? bd[q] : lo;
                    hi = bd[q] > hi ? bd[q] : hi;
                    if (second[q] - best[q] < band_px) frag = 1;
                }
            long i = (long)y * W + x;
            if (lo <= hi) {
                lo = lo < d_lo ? d_lo : (lo > d_hi ? d_hi : lo);
                hi = hi < d_lo ? d_lo : (hi > d_hi ? d_hi : hi);
                range[2 * i] = lo;
                range[2 * i + 1] = hi;
            } else {
                range[2 * i] = range[2 * i + 1] = NAN;
            }
            if (fragile) fragile[i] = (unsigned char)frag;
        }
}
