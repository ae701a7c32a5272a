// C ABI of the library (declared in include/mvs.h): context management,
// argument checking, per-view constants in double precision, and the
// stream-ordered sequencing of the kernels.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "../../include/mvs.h"
#include "mvs_internal.h"

namespace {

struct ViewData {
    mvs_camera cam;
    double Kinv[9];
    uint8_t* img = nullptr;
    uint2* tex = nullptr;      // bilinear-coefficient texels (fp16 x 4)
    float4* plane = nullptr;   // depth map state (library-owned)
    float* cost = nullptr;
    uint32_t* memo = nullptr;  // per pixel: candidates scored at the last visit (RefConst::memo)
    uint32_t* gen = nullptr;   // per pixel: plane generation (RefConst::gen)
    bool has_map = false;
};

struct Scratch {
    void* p = nullptr;
    size_t bytes = 0;
};

thread_local std::string g_create_error;

}  // namespace

std::atomic<long long> g_kernel_launches{0};

// A captured batch of PatchMatch kernels and the call it was captured for.
struct BatchGraph {
    std::vector<int32_t> refs, srcs;
    mvs_pm_params params;
    int lanes = 0;
    cudaGraphExec_t exec = nullptr;
    long long kernels = 0;
    unsigned long long used = 0;   // call counter of the last use (least recently used is replaced)
};
constexpr int kBatchGraphs = 4;   // captured batches kept per context

struct mvs_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::vector<ViewData> views;
    std::string err;
    Scratch scratch[8];
    // measurement hooks
    bool prof = false;
    std::vector<cudaEvent_t> ev;
    size_t ev_used = 0;
    long long launches0 = 0;
    unsigned long long* evals = nullptr;   // device counter of evaluated (pixel, hypothesis, view)
    // batched path
    cudaStream_t gstream = nullptr;        // private stream for graph capture / replay
    cudaEvent_t gev[2] = {nullptr, nullptr};
    BatchGraph batch[kBatchGraphs];
    unsigned long long batch_calls = 0;
    std::map<long long, int> tuned_lanes;  // (win_samples, n_src) -> lanes per pixel
};

namespace {

mvs_status fail(mvs_ctx* c, mvs_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    else g_create_error = buf;
    return st;
}

#define CK(c, call)                                                                                     \
    do {                                                                                                \
        cudaError_t _e = (call);                                                                        \
        if (_e != cudaSuccess)                                                                          \
            return fail((c), _e == cudaErrorMemoryAllocation ? MVS_ENOMEM : MVS_ECUDA, "%s: %s (%s:%d)", \
                        #call, cudaGetErrorString(_e), __FILE__, __LINE__);                             \
    } while (0)

void m3_mul(const double* A, const double* B, double* C) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0;
            for (int k = 0; k < 3; ++k) s += A[3 * i + k] * B[3 * k + j];
            C[3 * i + j] = s;
        }
}
void m3_inv(const double* A, double* B) {
    double c00 = A[4] * A[8] - A[5] * A[7], c01 = A[5] * A[6] - A[3] * A[8], c02 = A[3] * A[7] - A[4] * A[6];
    double det = A[0] * c00 + A[1] * c01 + A[2] * c02;
    B[0] = c00 / det; B[1] = (A[2] * A[7] - A[1] * A[8]) / det; B[2] = (A[1] * A[5] - A[2] * A[4]) / det;
    B[3] = c01 / det; B[4] = (A[0] * A[8] - A[2] * A[6]) / det; B[5] = (A[2] * A[3] - A[0] * A[5]) / det;
    B[6] = c02 / det; B[7] = (A[1] * A[6] - A[0] * A[7]) / det; B[8] = (A[0] * A[4] - A[1] * A[3]) / det;
}
// X_j = Rr X_ref + tr
void rel_pose(const mvs_camera& r, const mvs_camera& j, double* Rr, double* tr) {
    double RrT[9];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) RrT[3 * b + a] = r.R[3 * a + b];
    m3_mul(j.R, RrT, Rr);
    for (int a = 0; a < 3; ++a) tr[a] = j.t[a] - (Rr[3 * a] * r.t[0] + Rr[3 * a + 1] * r.t[1] + Rr[3 * a + 2] * r.t[2]);
}

void* scratch(mvs_ctx* c, int slot, size_t bytes, cudaError_t* e) {
    Scratch& s = c->scratch[slot];
    *e = cudaSuccess;
    if (s.bytes >= bytes) return s.p;
    if (s.p) {
        cudaStreamSynchronize(c->stream);
        cudaFree(s.p);
        s.p = nullptr;
        s.bytes = 0;
    }
    *e = cudaMalloc(&s.p, bytes);
    if (*e != cudaSuccess) { s.p = nullptr; return nullptr; }
    s.bytes = bytes;
    return s.p;
}

// true when p is device (or managed) memory the kernels can read
bool is_device_ptr(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

mvs_status check_view(mvs_ctx* c, int32_t v) {
    if (!c) return MVS_EINVAL;
    if (v < 0 || v >= (int32_t)c->views.size()) return fail(c, MVS_EINVAL, "view index %d out of range", v);
    return MVS_OK;
}

mvs_status check_pm(mvs_ctx* c, int32_t ref, const int32_t* srcs, int32_t n_src, const mvs_pm_params* p) {
    mvs_status st = check_view(c, ref);
    if (st != MVS_OK) return st;
    if (!p) return fail(c, MVS_EINVAL, "params is NULL");
    if (!srcs || n_src < 1 || n_src > MVS_MAX_SRC)
        return fail(c, MVS_EINVAL, "need 1..%d source views (got %d)", MVS_MAX_SRC, n_src);
    for (int i = 0; i < n_src; ++i) {
        if (srcs[i] < 0 || srcs[i] >= (int32_t)c->views.size() || srcs[i] == ref)
            return fail(c, MVS_EINVAL, "bad source view %d", srcs[i]);
        for (int k = 0; k < i; ++k)
            if (srcs[k] == srcs[i]) return fail(c, MVS_EINVAL, "duplicate source view %d", srcs[i]);
    }
    if (p->win_samples < 2 || p->win_samples > MVS_MAX_WIN)
        return fail(c, MVS_EINVAL, "win_samples must be in 2..%d", MVS_MAX_WIN);
    if (!(p->win_radius > 0.0f) || !(p->win_radius <= 64.0f))
        return fail(c, MVS_EINVAL, "win_radius must be in (0, 64]");
    if (!(p->d_lo > 0.0f) || !(p->d_hi > p->d_lo) || !std::isfinite(p->d_hi))
        return fail(c, MVS_EINVAL, "need 0 < d_lo < d_hi");
    if (p->precision != 0 && p->precision != 1) return fail(c, MVS_EUNSUPPORTED, "precision %d not built", p->precision);
    if (p->iters < 0) return fail(c, MVS_EINVAL, "iters < 0");
    if (p->lanes_per_pixel != 0 && p->lanes_per_pixel != 4 && p->lanes_per_pixel != 8 &&
        p->lanes_per_pixel != 16 && p->lanes_per_pixel != 32)
        return fail(c, MVS_EINVAL, "lanes_per_pixel must be 0, 4, 8, 16 or 32");
    if (p->n_prop < 0 || p->n_prop > 8) return fail(c, MVS_EINVAL, "n_prop must be in 0..8");
    if ((p->n_prop > 0) != (p->proposals != nullptr))
        return fail(c, MVS_EINVAL, "proposals must be given exactly when n_prop > 0");
    if ((uintptr_t)p->proposals & 15u) return fail(c, MVS_EINVAL, "proposals must be 16-byte aligned");
    if (p->proposals && !is_device_ptr(p->proposals)) return fail(c, MVS_EINVAL, "proposals must be device memory");
    return MVS_OK;
}

void make_refconst(const mvs_ctx* c, int32_t ref, const int32_t* srcs, int32_t n_src, const mvs_pm_params* p,
                   RefConst& rc) {
    std::memset(&rc, 0, sizeof rc);
    const ViewData& R = c->views[ref];
    rc.W = R.cam.width;
    rc.H = R.cam.height;
    rc.ref_index = ref;
    rc.n_src = n_src;
    for (int i = 0; i < 9; ++i) rc.Kinv[i] = (float)R.Kinv[i];
    rc.tex = R.tex;
    rc.img = R.img;
    rc.pitch = tex_pitch(rc.W);
    rc.n_tex = (uint32_t)rc.pitch * (uint32_t)(rc.H + 1);
    rc.n = p->win_samples;
    double r_now = 0.5 * (p->win_samples - 1);
    rc.step = (float)(p->win_radius / r_now);
    rc.sp_coef = p->sigma_s > 0 ? (float)(-1.0 / (2.0 * (double)p->sigma_s * p->sigma_s)) : 0.0f;
    double sc = 4.0 * 255.0 * p->sigma_c;   // texel units are 4 x [0, 255]
    rc.col_coef = p->sigma_c > 0 ? (float)(-1.0 / (2.0 * sc * sc)) : 0.0f;
    rc.d_lo = p->d_lo;
    rc.d_hi = p->d_hi;
    rc.seed = p->seed;
    rc.lanes_hint = p->lanes_per_pixel;
    rc.precision = p->precision;
    rc.n_prop = p->n_prop;
    rc.props = reinterpret_cast<const float4*>(p->proposals);
    rc.init_range = p->init_mode == MVS_INIT_RANGE ? reinterpret_cast<const float2*>(p->init_range) : nullptr;
    rc.plane = R.plane;
    rc.cost = R.cost;
    rc.memo = R.memo;
    rc.gen = R.gen;
    for (int j = 0; j < n_src; ++j) {
        const ViewData& S = c->views[srcs[j]];
        double Rr[9], tr[3], T[9], A[9];
        rel_pose(R.cam, S.cam, Rr, tr);
        m3_mul(S.cam.K, Rr, T);
        m3_mul(T, R.Kinv, A);
        PairConst& P = rc.pair[j];
        double b[3];
        for (int a = 0; a < 3; ++a) b[a] = S.cam.K[3 * a] * tr[0] + S.cam.K[3 * a + 1] * tr[1] + S.cam.K[3 * a + 2] * tr[2];
        // doubled, half-shifted rows (see PairConst), split into hi + lo floats
        auto split = [](double v, float& hi, float& lo) {
            hi = (float)v;
            lo = (float)(v - (double)hi);
        };
        for (int k = 0; k < 3; ++k) {
            split(2.0 * A[k] - A[6 + k], P.Gh[k], P.Gl[k]);
            split(2.0 * A[3 + k] - A[6 + k], P.Gh[3 + k], P.Gl[3 + k]);
            split(A[6 + k], P.Gh[6 + k], P.Gl[6 + k]);
        }
        split(2.0 * b[0] - b[2], P.Bh[0], P.Bl[0]);
        split(2.0 * b[1] - b[2], P.Bh[1], P.Bl[1]);
        split(b[2], P.Bh[2], P.Bl[2]);
        P.tex = S.tex;
        P.W = S.cam.width;
        P.H = S.cam.height;
        P.pitch = tex_pitch(P.W);
        P.n_tex = (uint32_t)P.pitch * (uint32_t)(P.H + 1);
    }
}

mvs_status ensure_map(mvs_ctx* c, int32_t v) {
    ViewData& V = c->views[v];
    if (V.plane) return MVS_OK;
    size_t n = (size_t)V.cam.width * V.cam.height;
    CK(c, cudaMalloc(&V.plane, n * sizeof(float4)));
    CK(c, cudaMalloc(&V.cost, n * sizeof(float)));
    CK(c, cudaMalloc(&V.memo, n * MVS_MEMO_WORDS * sizeof(uint32_t)));
    CK(c, cudaMalloc(&V.gen, n * sizeof(uint32_t)));
    CK(c, cudaMemsetAsync(V.gen, 0, n * sizeof(uint32_t), c->stream));
    return MVS_OK;
}

// fills n floats with v
__global__ void k_fill(float* __restrict__ a, size_t n, float v) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) a[i] = v;
}

cudaMemcpyKind kind_in(int32_t mem) { return mem == MVS_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice; }
cudaMemcpyKind kind_out(int32_t mem) { return mem == MVS_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice; }

}  // namespace

extern "C" {

mvs_status mvs_create(const mvs_camera* cams, const uint8_t* const* images, int32_t n_views, void* cuda_stream,
                      mvs_ctx** out) {
    if (!out) return fail(nullptr, MVS_EINVAL, "out is NULL");
    *out = nullptr;
    if (!cams || !images) return fail(nullptr, MVS_EINVAL, "cams or images is NULL");
    if (n_views < 2) return fail(nullptr, MVS_EINVAL, "need at least 2 views");
    for (int i = 0; i < n_views; ++i) {
        if (!images[i]) return fail(nullptr, MVS_EINVAL, "image %d is NULL", i);
        if (cams[i].width < 2 || cams[i].height < 2 || cams[i].width > 32768 || cams[i].height > 32768)
            return fail(nullptr, MVS_EINVAL, "view %d: size %dx%d outside 2..32768", i, cams[i].width,
                        cams[i].height);
        const double* K = cams[i].K;
        double det = K[0] * (K[4] * K[8] - K[5] * K[7]) - K[1] * (K[3] * K[8] - K[5] * K[6]) +
                     K[2] * (K[3] * K[7] - K[4] * K[6]);
        if (!(std::fabs(det) > 0) || !std::isfinite(det))
            return fail(nullptr, MVS_EINVAL, "view %d: singular or non-finite K", i);
        for (int k = 0; k < 9; ++k)
            if (!std::isfinite(cams[i].R[k])) return fail(nullptr, MVS_EINVAL, "view %d: non-finite R", i);
        for (int k = 0; k < 3; ++k)
            if (!std::isfinite(cams[i].t[k])) return fail(nullptr, MVS_EINVAL, "view %d: non-finite t", i);
    }
    mvs_ctx* c = new (std::nothrow) mvs_ctx();
    if (!c) return fail(nullptr, MVS_ENOMEM, "host allocation failed");
    cudaError_t e = cudaGetDevice(&c->device);
    if (e != cudaSuccess) {
        delete c;
        return fail(nullptr, MVS_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    }
    c->stream = (cudaStream_t)cuda_stream;
    c->views.resize(n_views);
    for (int i = 0; i < n_views; ++i) {
        ViewData& V = c->views[i];
        V.cam = cams[i];
        m3_inv(V.cam.K, V.Kinv);
        size_t n = (size_t)V.cam.width * V.cam.height;
        size_t nt = (size_t)tex_pitch(V.cam.width) * (V.cam.height + 1);
        e = cudaMalloc(&V.img, n);
        if (e == cudaSuccess) e = cudaMalloc(&V.tex, nt * sizeof(uint2));
        if (e == cudaSuccess) e = cudaMemsetAsync(V.tex, 0, nt * sizeof(uint2), c->stream);   // row padding
        if (e == cudaSuccess) e = cudaMemcpyAsync(V.img, images[i], n, cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) e = launch_build_texture(V.img, V.cam.width, V.cam.height, V.tex, c->stream);
        if (e != cudaSuccess) {
            mvs_status st = e == cudaErrorMemoryAllocation ? MVS_ENOMEM : MVS_ECUDA;
            fail(nullptr, st, "view %d upload: %s", i, cudaGetErrorString(e));
            mvs_destroy(c);
            return st;
        }
    }
    e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        fail(nullptr, MVS_ECUDA, "upload: %s", cudaGetErrorString(e));
        mvs_destroy(c);
        return MVS_ECUDA;
    }
    *out = c;
    return MVS_OK;
}

void mvs_destroy(mvs_ctx* c) {
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    for (auto& V : c->views) {
        cudaFree(V.img);
        cudaFree(V.tex);
        cudaFree(V.plane);
        cudaFree(V.cost);
        cudaFree(V.memo);
        cudaFree(V.gen);
    }
    for (auto& s : c->scratch) cudaFree(s.p);
    for (auto e : c->ev) cudaEventDestroy(e);
    cudaFree(c->evals);
    for (auto& b : c->batch)
        if (b.exec) cudaGraphExecDestroy(b.exec);
    for (auto e : c->gev) if (e) cudaEventDestroy(e);
    if (c->gstream) cudaStreamDestroy(c->gstream);
    delete c;
}

const char* mvs_last_error(const mvs_ctx* c) { return c ? c->err.c_str() : g_create_error.c_str(); }

// the initialisation mode and its depth-range buffer
static mvs_status check_init(mvs_ctx* c, const mvs_pm_params* p) {
    if (p->init_mode < MVS_INIT_RANDOM || p->init_mode > MVS_INIT_RANGE) return fail(c, MVS_EINVAL, "bad init_mode");
    if ((p->init_mode == MVS_INIT_RANGE) != (p->init_range != nullptr) || ((uintptr_t)p->init_range & 7u))
        return fail(c, MVS_EINVAL, "init_range (8-byte aligned) must be given exactly with MVS_INIT_RANGE");
    if (p->init_range && !is_device_ptr(p->init_range)) return fail(c, MVS_EINVAL, "init_range must be device memory");
    return MVS_OK;
}

mvs_status mvs_patchmatch(mvs_ctx* c, int32_t ref, const int32_t* srcs, int32_t n_src, const mvs_pm_params* p,
                          mvs_depth_map* out) {
    mvs_status st = check_pm(c, ref, srcs, n_src, p);
    if (st != MVS_OK) return st;
    if (!out || !out->plane || !out->cost) return fail(c, MVS_EINVAL, "out buffers are NULL");
    if (((uintptr_t)out->plane & 15u) || ((uintptr_t)out->cost & 3u))
        return fail(c, MVS_EINVAL, "plane must be 16-byte and cost 4-byte aligned");
    if (out->mem != MVS_MEM_DEVICE && out->mem != MVS_MEM_HOST) return fail(c, MVS_EINVAL, "bad mem kind");
    if ((st = check_init(c, p)) != MVS_OK) return st;
    int pend = p->phase_end < 0 ? 2 * p->iters : p->phase_end;
    if (p->phase_begin < 0 || pend < p->phase_begin) return fail(c, MVS_EINVAL, "bad phase range");
    CK(c, cudaSetDevice(c->device));
    if ((st = ensure_map(c, ref)) != MVS_OK) return st;
    ViewData& V = c->views[ref];
    size_t n = (size_t)V.cam.width * V.cam.height;
    RefConst rc;
    make_refconst(c, ref, srcs, n_src, p, rc);
    if (p->init_mode == MVS_INIT_RANDOM || p->init_mode == MVS_INIT_RANGE) {
        CK(c, launch_init(rc, nullptr, c->stream));
    } else {
        CK(c, cudaMemcpyAsync(V.plane, out->plane, n * sizeof(float4), kind_in(out->mem), c->stream));
        if (p->init_mode == MVS_INIT_GIVEN)
            CK(c, cudaMemcpyAsync(V.cost, out->cost, n * sizeof(float), kind_in(out->mem), c->stream));
        else
            CK(c, launch_cost(rc, V.plane, V.cost, nullptr, c->stream));
    }
    RefConst rcp = rc;
    if (c->prof) rcp.eval_counter = c->evals;
    CK(c, launch_memo_reset(rc, c->stream));
    for (int ph = p->phase_begin; ph < pend; ++ph) {
        if (c->prof) {
            while (c->ev.size() < c->ev_used + 2) {
                cudaEvent_t e;
                CK(c, cudaEventCreate(&e));
                c->ev.push_back(e);
            }
            CK(c, cudaEventRecord(c->ev[c->ev_used], c->stream));
        }
        CK(c, launch_phase(rcp, ph, c->stream));
        if (c->prof) {
            CK(c, cudaEventRecord(c->ev[c->ev_used + 1], c->stream));
            c->ev_used += 2;
        }
    }
    V.has_map = true;
    CK(c, cudaMemcpyAsync(out->plane, V.plane, n * sizeof(float4), kind_out(out->mem), c->stream));
    CK(c, cudaMemcpyAsync(out->cost, V.cost, n * sizeof(float), kind_out(out->mem), c->stream));
    if (out->mem == MVS_MEM_HOST) CK(c, cudaStreamSynchronize(c->stream));
    return MVS_OK;
}

// Times two iterations (four phases) of `ref` with each candidate work
// layout, each from the same freshly initialised state, and returns the
// fastest lanes per pixel.
static mvs_status autotune_lanes(mvs_ctx* c, int32_t ref, const int32_t* srcs, int32_t n_src,
                                 const mvs_pm_params* p, int* lanes_out) {
    long long key = (long long)p->win_samples * 64 + n_src;
    auto it = c->tuned_lanes.find(key);
    if (it != c->tuned_lanes.end()) { *lanes_out = it->second; return MVS_OK; }
    const int s = p->win_samples * p->win_samples;
    std::vector<int> cand;
    if (s <= 16) cand = {4};
    else if (s <= 36) cand = {4, 8};
    else if (s <= 64) cand = {8, 16};
    else if (s <= 128) cand = {8, 16, 32};
    else if (s <= 256) cand = {16, 32};
    else cand = {32};
    ViewData& V = c->views[ref];
    size_t n = (size_t)V.cam.width * V.cam.height;
    mvs_pm_params q = *p;
    q.lanes_per_pixel = 0;
    RefConst rc;
    make_refconst(c, ref, srcs, n_src, &q, rc);
    cudaError_t e;
    char* keep = (char*)scratch(c, 5, n * (sizeof(float4) + sizeof(float)), &e);
    CK(c, e);
    CK(c, launch_init(rc, nullptr, c->stream));
    CK(c, cudaMemcpyAsync(keep, V.plane, n * sizeof(float4), cudaMemcpyDeviceToDevice, c->stream));
    CK(c, cudaMemcpyAsync(keep + n * sizeof(float4), V.cost, n * sizeof(float), cudaMemcpyDeviceToDevice, c->stream));
    cudaEvent_t t0, t1;
    CK(c, cudaEventCreate(&t0));
    CK(c, cudaEventCreate(&t1));
    float best_ms = 3.0e38f;
    int best = cand[0];
    for (int lanes : cand) {
        rc.lanes_hint = lanes;
        for (int rep = 0; rep < 2; ++rep) {   // the first run warms caches and launch configuration
            CK(c, cudaMemcpyAsync(V.plane, keep, n * sizeof(float4), cudaMemcpyDeviceToDevice, c->stream));
            CK(c, cudaMemcpyAsync(V.cost, keep + n * sizeof(float4), n * sizeof(float), cudaMemcpyDeviceToDevice,
                                  c->stream));
            CK(c, cudaEventRecord(t0, c->stream));
            CK(c, launch_memo_reset(rc, c->stream));
            for (int ph = 0; ph < 4; ++ph) CK(c, launch_phase(rc, ph, c->stream));
            CK(c, cudaEventRecord(t1, c->stream));
        }
        CK(c, cudaEventSynchronize(t1));
        float ms = 0.0f;
        CK(c, cudaEventElapsedTime(&ms, t0, t1));
        if (ms < best_ms) { best_ms = ms; best = lanes; }
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    c->tuned_lanes[key] = best;
    *lanes_out = best;
    return MVS_OK;
}

mvs_status mvs_patchmatch_batch(mvs_ctx* c, int32_t n_ref, const int32_t* refs, const int32_t* srcs, int32_t n_src,
                                const mvs_pm_params* p, mvs_depth_map* outs) {
    if (!c) return MVS_EINVAL;
    if (n_ref < 1 || !refs || !srcs || !outs || !p) return fail(c, MVS_EINVAL, "bad batch arguments");
    mvs_pm_params q = *p;
    const bool tune = p->lanes_per_pixel == -1;
    if (tune) q.lanes_per_pixel = 0;
    for (int r = 0; r < n_ref; ++r) {
        mvs_status st = check_pm(c, refs[r], srcs + (size_t)r * n_src, n_src, &q);
        if (st != MVS_OK) return st;
        for (int k = 0; k < r; ++k)
            if (refs[k] == refs[r]) return fail(c, MVS_EINVAL, "reference view %d repeated", refs[r]);
        if (!outs[r].plane || !outs[r].cost) return fail(c, MVS_EINVAL, "out buffers of entry %d are NULL", r);
        if (((uintptr_t)outs[r].plane & 15u) || ((uintptr_t)outs[r].cost & 3u))
            return fail(c, MVS_EINVAL, "plane must be 16-byte and cost 4-byte aligned");
        if (outs[r].mem != outs[0].mem || (outs[r].mem != MVS_MEM_DEVICE && outs[r].mem != MVS_MEM_HOST))
            return fail(c, MVS_EINVAL, "all outputs must be in the same memory kind");
    }
    mvs_status st = check_init(c, p);
    if (st != MVS_OK) return st;
    int pend = p->phase_end < 0 ? 2 * p->iters : p->phase_end;
    if (p->phase_begin < 0 || pend < p->phase_begin) return fail(c, MVS_EINVAL, "bad phase range");
    CK(c, cudaSetDevice(c->device));
    for (int r = 0; r < n_ref; ++r)
        if ((st = ensure_map(c, refs[r])) != MVS_OK) return st;
    if (tune && (st = autotune_lanes(c, refs[0], srcs, n_src, p, &q.lanes_per_pixel)) != MVS_OK) return st;
    const int32_t mem = outs[0].mem;
    if (p->init_mode == MVS_INIT_GIVEN || p->init_mode == MVS_INIT_GIVEN_RECOST)
        for (int r = 0; r < n_ref; ++r) {
            ViewData& V = c->views[refs[r]];
            size_t n = (size_t)V.cam.width * V.cam.height;
            CK(c, cudaMemcpyAsync(V.plane, outs[r].plane, n * sizeof(float4), kind_in(mem), c->stream));
            if (p->init_mode == MVS_INIT_GIVEN)
                CK(c, cudaMemcpyAsync(V.cost, outs[r].cost, n * sizeof(float), kind_in(mem), c->stream));
        }
    if (!c->gstream) {
        CK(c, cudaStreamCreateWithFlags(&c->gstream, cudaStreamNonBlocking));
        CK(c, cudaEventCreateWithFlags(&c->gev[0], cudaEventDisableTiming));
        CK(c, cudaEventCreateWithFlags(&c->gev[1], cudaEventDisableTiming));
    }
    std::vector<RefConst> rcs(n_ref);
    size_t range_off = 0;   // MVS_INIT_RANGE: the views' ranges lie back to back in refs order
    size_t prop_off = 0;    // learned proposals: likewise, H * W * n_prop planes per view
    for (int r = 0; r < n_ref; ++r) {
        make_refconst(c, refs[r], srcs + (size_t)r * n_src, n_src, &q, rcs[r]);
        if (rcs[r].init_range) {
            rcs[r].init_range += range_off;
            range_off += (size_t)rcs[r].W * rcs[r].H;
        }
        if (rcs[r].props) {
            rcs[r].props += prop_off;
            prop_off += (size_t)rcs[r].W * rcs[r].H * rcs[r].n_prop;
        }
    }
    std::vector<int32_t> kr(refs, refs + n_ref), ks(srcs, srcs + (size_t)n_ref * n_src);
    // a graph captured for the same call, else the least recently used slot
    BatchGraph* hit = nullptr;
    BatchGraph* lru = &c->batch[0];
    for (auto& b : c->batch) {
        if (b.exec && b.refs == kr && b.srcs == ks && b.lanes == q.lanes_per_pixel &&
            std::memcmp(&b.params, &q, sizeof q) == 0)
            hit = &b;
        if (!b.exec || (lru->exec && b.used < lru->used)) lru = &b;
    }
    BatchGraph& B = hit ? *hit : *lru;
    B.used = ++c->batch_calls;
    bool same = hit != nullptr;
    if (!same) {
        if (B.exec) { cudaGraphExecDestroy(B.exec); B.exec = nullptr; }
        for (auto& rc : rcs) CK(c, prime_launch_configs(rc));
        long long k0 = g_kernel_launches.load();
        cudaGraph_t g = nullptr;
        CK(c, cudaStreamBeginCapture(c->gstream, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = cudaSuccess;
        // view after view: consecutive launches share their source textures in L2
        for (int r = 0; r < n_ref && e == cudaSuccess; ++r) {
            if (p->init_mode == MVS_INIT_RANDOM || p->init_mode == MVS_INIT_RANGE)
                e = launch_init(rcs[r], nullptr, c->gstream);
            else if (p->init_mode == MVS_INIT_GIVEN_RECOST)
                e = launch_cost(rcs[r], rcs[r].plane, rcs[r].cost, nullptr, c->gstream);
            if (e == cudaSuccess) e = launch_memo_reset(rcs[r], c->gstream);
            for (int ph = p->phase_begin; ph < pend && e == cudaSuccess; ++ph) e = launch_phase(rcs[r], ph, c->gstream);
        }
        cudaError_t e2 = cudaStreamEndCapture(c->gstream, &g);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&B.exec, g, 0);
        if (g) cudaGraphDestroy(g);
        CK(c, e);
        B.kernels = g_kernel_launches.load() - k0;
        g_kernel_launches.fetch_sub(B.kernels);   // counted when the graph runs
        B.refs = kr;
        B.srcs = ks;
        B.params = q;
        B.lanes = q.lanes_per_pixel;
    }
    // order the private stream after the caller's stream, replay, and back
    CK(c, cudaEventRecord(c->gev[0], c->stream));
    CK(c, cudaStreamWaitEvent(c->gstream, c->gev[0], 0));
    CK(c, cudaGraphLaunch(B.exec, c->gstream));
    count_launch(B.kernels);
    CK(c, cudaEventRecord(c->gev[1], c->gstream));
    CK(c, cudaStreamWaitEvent(c->stream, c->gev[1], 0));
    for (int r = 0; r < n_ref; ++r) {
        ViewData& V = c->views[refs[r]];
        size_t n = (size_t)V.cam.width * V.cam.height;
        V.has_map = true;
        CK(c, cudaMemcpyAsync(outs[r].plane, V.plane, n * sizeof(float4), kind_out(mem), c->stream));
        CK(c, cudaMemcpyAsync(outs[r].cost, V.cost, n * sizeof(float), kind_out(mem), c->stream));
    }
    if (mem == MVS_MEM_HOST) CK(c, cudaStreamSynchronize(c->stream));
    return MVS_OK;
}

mvs_status mvs_plane_cost(mvs_ctx* c, int32_t ref, const int32_t* srcs, int32_t n_src, const mvs_pm_params* p,
                          const float* plane, float* cost, float* view_cost, int32_t mem) {
    mvs_status st = check_pm(c, ref, srcs, n_src, p);
    if (st != MVS_OK) return st;
    if (!plane || !cost) return fail(c, MVS_EINVAL, "plane or cost is NULL");
    if (((uintptr_t)plane & 15u) || ((uintptr_t)cost & 3u) || ((uintptr_t)view_cost & 3u))
        return fail(c, MVS_EINVAL, "plane must be 16-byte and costs 4-byte aligned");
    if (mem != MVS_MEM_DEVICE && mem != MVS_MEM_HOST) return fail(c, MVS_EINVAL, "bad mem kind");
    CK(c, cudaSetDevice(c->device));
    ViewData& V = c->views[ref];
    size_t n = (size_t)V.cam.width * V.cam.height;
    RefConst rc;
    make_refconst(c, ref, srcs, n_src, p, rc);
    const float4* pl_d = (const float4*)plane;
    float* cost_d = cost;
    float* vc_d = view_cost;
    cudaError_t e;
    if (mem == MVS_MEM_HOST) {
        char* buf = (char*)scratch(c, 0, n * (sizeof(float4) + sizeof(float) * (1 + n_src)), &e);
        CK(c, e);
        pl_d = (const float4*)buf;
        cost_d = (float*)(buf + n * sizeof(float4));
        vc_d = view_cost ? cost_d + n : nullptr;
        CK(c, cudaMemcpyAsync((void*)pl_d, plane, n * sizeof(float4), cudaMemcpyHostToDevice, c->stream));
    }
    CK(c, launch_cost(rc, pl_d, cost_d, vc_d, c->stream));
    if (mem == MVS_MEM_HOST) {
        CK(c, cudaMemcpyAsync(cost, cost_d, n * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
        if (view_cost)
            CK(c, cudaMemcpyAsync(view_cost, vc_d, n * n_src * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
        CK(c, cudaStreamSynchronize(c->stream));
    }
    return MVS_OK;
}

mvs_status mvs_set_depth_map(mvs_ctx* c, int32_t view, const float* plane, const float* cost, int32_t mem) {
    if (!c) return MVS_EINVAL;
    if (view < 0 || view >= (int32_t)c->views.size()) return fail(c, MVS_EINVAL, "bad view %d", view);
    if (!plane) return fail(c, MVS_EINVAL, "plane is NULL");
    if (((uintptr_t)plane & 15u) || ((uintptr_t)cost & 3u))
        return fail(c, MVS_EINVAL, "plane must be 16-byte and cost 4-byte aligned");
    if (mem != MVS_MEM_DEVICE && mem != MVS_MEM_HOST) return fail(c, MVS_EINVAL, "bad mem kind");
    CK(c, cudaSetDevice(c->device));
    mvs_status st = ensure_map(c, view);
    if (st != MVS_OK) return st;
    ViewData& V = c->views[view];
    const size_t n = (size_t)V.cam.width * V.cam.height;
    CK(c, cudaMemcpyAsync(V.plane, plane, n * sizeof(float4), kind_in(mem), c->stream));
    if (cost) {
        CK(c, cudaMemcpyAsync(V.cost, cost, n * sizeof(float), kind_in(mem), c->stream));
    } else {
        k_fill<<<(unsigned)std::min<size_t>((n + 255) / 256, 152 * 16), 256, 0, c->stream>>>(V.cost, n, 2.0f);
        count_launch();
        CK(c, cudaGetLastError());
    }
    V.has_map = true;
    if (mem == MVS_MEM_HOST) CK(c, cudaStreamSynchronize(c->stream));
    return MVS_OK;
}

mvs_status mvs_geo_filter(mvs_ctx* c, int32_t ref, const int32_t* srcs, int32_t n_src, const mvs_filter_params* fp,
                          uint8_t* keep_mask, int32_t* count, int32_t mem) {
    mvs_status st = check_view(c, ref);
    if (st != MVS_OK) return st;
    if (!fp || !keep_mask) return fail(c, MVS_EINVAL, "params or keep_mask is NULL");
    if (!srcs || n_src < 1 || n_src > MVS_MAX_SRC) return fail(c, MVS_EINVAL, "need 1..%d sources", MVS_MAX_SRC);
    if (mem != MVS_MEM_DEVICE && mem != MVS_MEM_HOST) return fail(c, MVS_EINVAL, "bad mem kind");
    for (int i = 0; i < n_src; ++i)
        if (srcs[i] < 0 || srcs[i] >= (int32_t)c->views.size() || srcs[i] == ref)
            return fail(c, MVS_EINVAL, "bad source view %d", srcs[i]);
    if (!c->views[ref].has_map) return fail(c, MVS_ESTATE, "view %d has no depth map", ref);
    for (int i = 0; i < n_src; ++i)
        if (!c->views[srcs[i]].has_map) return fail(c, MVS_ESTATE, "source view %d has no depth map", srcs[i]);
    CK(c, cudaSetDevice(c->device));
    const ViewData& V = c->views[ref];
    FilterConst fc;
    std::memset(&fc, 0, sizeof fc);
    fc.W = V.cam.width;
    fc.H = V.cam.height;
    for (int i = 0; i < 9; ++i) { fc.K[i] = (float)V.cam.K[i]; fc.Kinv[i] = (float)V.Kinv[i]; }
    fc.plane = V.plane;
    fc.n_src = n_src;
    for (int j = 0; j < n_src; ++j) {
        const ViewData& S = c->views[srcs[j]];
        double Rr[9], tr[3];
        rel_pose(V.cam, S.cam, Rr, tr);
        auto& s = fc.src[j];
        for (int i = 0; i < 9; ++i) { s.R[i] = (float)Rr[i]; s.K[i] = (float)S.cam.K[i]; s.Kinv[i] = (float)S.Kinv[i]; }
        for (int i = 0; i < 3; ++i) s.t[i] = (float)tr[i];
        s.plane = S.plane;
        s.W = S.cam.width;
        s.H = S.cam.height;
    }
    fc.depth_tol = fp->depth_tol;
    fc.depth_relative = fp->depth_relative;
    fc.cos_max = (float)std::cos(fp->max_angle_deg * 3.14159265358979323846 / 180.0);
    fc.max_reproj = fp->max_reproj_px;
    fc.min_consistent = fp->min_consistent;
    size_t n = (size_t)fc.W * fc.H;
    uint8_t* keep_d = keep_mask;
    int32_t* cnt_d = count;
    cudaError_t e;
    if (mem == MVS_MEM_HOST) {
        char* buf = (char*)scratch(c, 0, n * (1 + sizeof(int32_t)) + 16, &e);
        CK(c, e);
        cnt_d = (int32_t*)buf;
        keep_d = (uint8_t*)(buf + n * sizeof(int32_t));
    }
    CK(c, launch_geo_filter(fc, keep_d, cnt_d, c->stream));
    if (mem == MVS_MEM_HOST) {
        CK(c, cudaMemcpyAsync(keep_mask, keep_d, n, cudaMemcpyDeviceToHost, c->stream));
        if (count) CK(c, cudaMemcpyAsync(count, cnt_d, n * sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
        CK(c, cudaStreamSynchronize(c->stream));
    }
    return MVS_OK;
}

mvs_status mvs_fuse(mvs_ctx* c, int32_t n_views, const int32_t* views, const uint8_t* const* keep_masks, float rel_tol,
                    float* points, int32_t* src, int64_t* owner, int64_t capacity, int64_t* n_points, int32_t mem) {
    if (!c) return MVS_EINVAL;
    if (!views || n_views < 1 || n_views > (int32_t)c->views.size())
        return fail(c, MVS_EINVAL, "need 1..%d views", (int)c->views.size());
    if (!n_points || capacity < 0 || (capacity > 0 && !points)) return fail(c, MVS_EINVAL, "bad output arguments");
    if (!(rel_tol > 0.0f)) return fail(c, MVS_EINVAL, "rel_tol must be > 0");
    if (mem != MVS_MEM_DEVICE && mem != MVS_MEM_HOST) return fail(c, MVS_EINVAL, "bad mem kind");
    std::vector<char> seen(c->views.size(), 0);
    for (int a = 0; a < n_views; ++a) {
        const int v = views[a];
        if (v < 0 || v >= (int32_t)c->views.size() || seen[v]) return fail(c, MVS_EINVAL, "bad or repeated view %d", v);
        seen[v] = 1;
        if (!c->views[v].has_map) return fail(c, MVS_ESTATE, "view %d has no depth map", v);
        const double* K = c->views[v].cam.K;
        if (K[3] != 0.0 || K[6] != 0.0 || K[7] != 0.0 || K[8] != 1.0)
            return fail(c, MVS_EUNSUPPORTED, "view %d: fusion needs a pinhole K = [fx s cx; 0 fy cy; 0 0 1]", v);
    }
    CK(c, cudaSetDevice(c->device));
    // scratch slot 6, every region starting on a 16-byte boundary: per view
    // the claim and alive arrays (and a device copy of a host keep mask),
    // then block counts, block offsets, the running total and the views
    auto a16 = [](size_t b) { return (b + 15) & ~(size_t)15; };
    const bool copy_keep = mem == MVS_MEM_HOST && keep_masks;
    size_t bytes = 0, max_blocks = 1;
    for (int a = 0; a < n_views; ++a) {
        const size_t np = (size_t)c->views[views[a]].cam.width * c->views[views[a]].cam.height;
        bytes += a16(np * sizeof(int)) + a16(np) * (copy_keep ? 2 : 1);
        max_blocks = std::max(max_blocks, (np + 255) / 256);
    }
    bytes += a16(max_blocks * sizeof(int)) + a16(max_blocks * sizeof(long long)) + 16 +
             a16((size_t)n_views * sizeof(FuseView));
    cudaError_t e;
    char* buf = (char*)scratch(c, 6, bytes, &e);
    CK(c, e);
    std::vector<FuseView> fv(n_views);
    std::vector<const uint8_t*> keep_d(n_views, nullptr);
    char* q = buf;
    for (int a = 0; a < n_views; ++a) {
        const ViewData& V = c->views[views[a]];
        const size_t np = (size_t)V.cam.width * V.cam.height;
        FuseView& f = fv[a];
        f.fx = (float)V.cam.K[0]; f.sk = (float)V.cam.K[1]; f.cx = (float)V.cam.K[2];
        f.fy = (float)V.cam.K[4]; f.cy = (float)V.cam.K[5];
        for (int i = 0; i < 9; ++i) f.R[i] = (float)V.cam.R[i];
        for (int i = 0; i < 3; ++i) f.t[i] = (float)V.cam.t[i];
        f.W = V.cam.width;
        f.H = V.cam.height;
        f.index = views[a];
        f.plane = V.plane;
        f.claim = (int*)q;
        q += a16(np * sizeof(int));
        f.alive = (uint8_t*)q;
        q += a16(np);
        if (copy_keep) {
            if (keep_masks[a]) {
                CK(c, cudaMemcpyAsync(q, keep_masks[a], np, cudaMemcpyHostToDevice, c->stream));
                keep_d[a] = (const uint8_t*)q;
            }
            q += a16(np);
        } else if (keep_masks) {
            keep_d[a] = keep_masks[a];
        }
    }
    int* block_count = (int*)q;
    q += a16(max_blocks * sizeof(int));
    long long* block_off = (long long*)q;
    q += a16(max_blocks * sizeof(long long));
    long long* total = (long long*)q;
    q += 16;
    FuseView* dev_views = (FuseView*)q;
    float4* pts_d = (float4*)points;
    int2* src_d = (int2*)src;
    long long* own_d = (long long*)owner;
    size_t n_pix = 0;
    for (int a = 0; a < n_views; ++a) n_pix += (size_t)c->views[views[a]].cam.width * c->views[views[a]].cam.height;
    if (mem == MVS_MEM_HOST && (capacity > 0 || owner)) {
        // host outputs go through scratch slot 7: points, sources, owners
        const size_t b_pts = a16((size_t)capacity * sizeof(float4));
        const size_t b_src = a16(src ? (size_t)capacity * sizeof(int2) : 0);
        char* ob = (char*)scratch(c, 7, b_pts + b_src + (owner ? n_pix * sizeof(long long) : 0) + 16, &e);
        CK(c, e);
        pts_d = (float4*)ob;
        src_d = src ? (int2*)(ob + b_pts) : nullptr;
        own_d = owner ? (long long*)(ob + b_pts + b_src) : nullptr;
    }
    {
        size_t off = 0;
        for (int a = 0; a < n_views; ++a) {
            fv[a].owner = own_d ? own_d + off : nullptr;
            off += (size_t)fv[a].W * fv[a].H;
        }
    }
    CK(c, launch_fuse(fv.data(), dev_views, n_views, keep_masks ? keep_d.data() : nullptr, rel_tol, block_count,
                      block_off, total, pts_d, src_d, capacity, c->stream));
    long long tot = 0;
    CK(c, cudaMemcpyAsync(&tot, total, sizeof tot, cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    *n_points = tot;
    const long long nw = std::min<long long>(tot, capacity);
    if (mem == MVS_MEM_HOST && (nw > 0 || owner)) {
        if (nw > 0) {
            CK(c, cudaMemcpyAsync(points, pts_d, (size_t)nw * sizeof(float4), cudaMemcpyDeviceToHost, c->stream));
            if (src) CK(c, cudaMemcpyAsync(src, src_d, (size_t)nw * sizeof(int2), cudaMemcpyDeviceToHost, c->stream));
        }
        if (owner)
            CK(c, cudaMemcpyAsync(owner, own_d, n_pix * sizeof(long long), cudaMemcpyDeviceToHost, c->stream));
        CK(c, cudaStreamSynchronize(c->stream));
    }
    if (tot > capacity) return fail(c, MVS_EINVAL, "%lld points do not fit the capacity of %lld", tot, (long long)capacity);
    return MVS_OK;
}

mvs_status mvs_select_neighbors(mvs_ctx* c, int64_t n_points, const double* points, const uint64_t* vis, double eps,
                                double t_tau, int32_t k, int32_t* neighbors, double* tau, int32_t* n_shared,
                                double* zeta, int32_t mem) {
    if (!c) return MVS_EINVAL;
    const int n = (int)c->views.size();
    if (n < 2 || n > MVS_MAX_VIEWS_SELECT) return fail(c, MVS_EINVAL, "need 2..%d views", MVS_MAX_VIEWS_SELECT);
    if (n_points < 0 || (n_points > 0 && (!points || !vis)) || !neighbors || k < 1 || k > n - 1)
        return fail(c, MVS_EINVAL, "bad arguments (k must lie in 1..n_views-1)");
    if (!(eps > 0.0) || !(t_tau >= 0.0)) return fail(c, MVS_EINVAL, "need eps > 0, t_tau >= 0");
    if (mem != MVS_MEM_DEVICE && mem != MVS_MEM_HOST) return fail(c, MVS_EINVAL, "bad mem kind");
    CK(c, cudaSetDevice(c->device));
    // per-view cameras and per-pair constants in FP64 (host): baseline and
    // angle between the principal axes (third rows of R)
    std::vector<NbrView> nv(n);
    std::vector<double> base((size_t)n * n), angle((size_t)n * n);
    for (int v = 0; v < n; ++v) {
        const mvs_camera& cam = c->views[v].cam;
        for (int a = 0; a < 9; ++a) { nv[v].K[a] = cam.K[a]; nv[v].R[a] = cam.R[a]; }
        for (int a = 0; a < 3; ++a) nv[v].t[a] = cam.t[a];
        for (int a = 0; a < 3; ++a) nv[v].C[a] = -(cam.R[a] * cam.t[0] + cam.R[3 + a] * cam.t[1] + cam.R[6 + a] * cam.t[2]);
    }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            const double d0 = nv[i].C[0] - nv[j].C[0], d1 = nv[i].C[1] - nv[j].C[1], d2 = nv[i].C[2] - nv[j].C[2];
            base[(size_t)i * n + j] = std::sqrt(d0 * d0 + d1 * d1 + d2 * d2);
            const double cs = nv[i].R[6] * nv[j].R[6] + nv[i].R[7] * nv[j].R[7] + nv[i].R[8] * nv[j].R[8];
            angle[(size_t)i * n + j] = std::acos(cs > 1.0 ? 1.0 : (cs < -1.0 ? -1.0 : cs));
        }
    // scratch slot 7: views, per-pair constants and results; host inputs
    const size_t nn = (size_t)n * n;
    size_t bytes = 256 + sizeof(NbrView) * n + nn * (4 * sizeof(double) + sizeof(int)) + (size_t)n * k * sizeof(int);
    if (mem == MVS_MEM_HOST) bytes += (size_t)n_points * (3 * sizeof(double) + sizeof(uint64_t)) + 64;
    cudaError_t e;
    char* q = (char*)scratch(c, 7, bytes, &e);
    CK(c, e);
    auto take = [&](size_t b) { char* r = q; q += (b + 15) & ~(size_t)15; return (void*)r; };
    NbrView* d_views = (NbrView*)take(sizeof(NbrView) * n);
    double* d_base = (double*)take(nn * sizeof(double));
    double* d_angle = (double*)take(nn * sizeof(double));
    double* d_tau = (double*)take(nn * sizeof(double));
    double* d_zeta = (double*)take(nn * sizeof(double));
    int* d_na = (int*)take(nn * sizeof(int));
    int* d_nbr = (int*)take((size_t)n * k * sizeof(int));
    const double* d_X = points;
    const unsigned long long* d_vis = (const unsigned long long*)vis;
    if (mem == MVS_MEM_HOST && n_points > 0) {
        double* x = (double*)take((size_t)n_points * 3 * sizeof(double));
        unsigned long long* m = (unsigned long long*)take((size_t)n_points * sizeof(uint64_t));
        CK(c, cudaMemcpyAsync(x, points, (size_t)n_points * 3 * sizeof(double), cudaMemcpyHostToDevice, c->stream));
        CK(c, cudaMemcpyAsync(m, vis, (size_t)n_points * sizeof(uint64_t), cudaMemcpyHostToDevice, c->stream));
        d_X = x;
        d_vis = m;
    }
    CK(c, cudaMemcpyAsync(d_views, nv.data(), sizeof(NbrView) * n, cudaMemcpyHostToDevice, c->stream));
    CK(c, cudaMemcpyAsync(d_base, base.data(), nn * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    CK(c, cudaMemcpyAsync(d_angle, angle.data(), nn * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    CK(c, launch_select_neighbors(d_views, n, d_X, d_vis, n_points, eps, t_tau, k, d_base, d_angle, d_tau, d_na,
                                  d_zeta, d_nbr, c->stream));
    const cudaMemcpyKind ko = kind_out(mem);
    CK(c, cudaMemcpyAsync(neighbors, d_nbr, (size_t)n * k * sizeof(int), ko, c->stream));
    if (tau) CK(c, cudaMemcpyAsync(tau, d_tau, nn * sizeof(double), ko, c->stream));
    if (n_shared) CK(c, cudaMemcpyAsync(n_shared, d_na, nn * sizeof(int), ko, c->stream));
    if (zeta) CK(c, cudaMemcpyAsync(zeta, d_zeta, nn * sizeof(double), ko, c->stream));
    // the host vectors above are staged by the copies; wait for them
    CK(c, cudaStreamSynchronize(c->stream));
    return MVS_OK;
}

mvs_status mvs_sparse_depth_range(mvs_ctx* c, int32_t ref, int64_t n_points, const double* points, const uint64_t* vis,
                                  const double* reproj, const double* obs, double max_reproj, float d_lo, float d_hi,
                                  float* range, int32_t mem) {
    mvs_status st = check_view(c, ref);
    if (st != MVS_OK) return st;
    if (c->views.size() > MVS_MAX_VIEWS_SELECT) return fail(c, MVS_EINVAL, "at most %d views", MVS_MAX_VIEWS_SELECT);
    if (n_points < 0 || (n_points > 0 && (!points || !vis || !reproj || !obs)) || !range)
        return fail(c, MVS_EINVAL, "NULL argument");
    if (!(d_lo < d_hi)) return fail(c, MVS_EINVAL, "need d_lo < d_hi");
    if (mem != MVS_MEM_DEVICE && mem != MVS_MEM_HOST) return fail(c, MVS_EINVAL, "bad mem kind");
    CK(c, cudaSetDevice(c->device));
    const ViewData& V = c->views[ref];
    const int W = V.cam.width, H = V.cam.height;
    const size_t np = (size_t)n_points, npix = (size_t)W * H;
    auto a16 = [](size_t b) { return (b + 15) & ~(size_t)15; };
    size_t bytes = 16 + a16(np * sizeof(float2)) + a16(np * sizeof(float));
    if (mem == MVS_MEM_HOST) bytes += a16(np * 3 * 8) + a16(np * 8) + a16(np * 8) + a16(np * 2 * 8) + a16(npix * 8);
    cudaError_t e;
    char* q = (char*)scratch(c, 7, bytes, &e);
    CK(c, e);
    auto take = [&](size_t b) { char* r = q; q += a16(b); return (void*)r; };
    unsigned long long* total = (unsigned long long*)take(16);
    float2* uv = (float2*)take(np * sizeof(float2));
    float* dep = (float*)take(np * sizeof(float));
    const double* dX = points;
    const unsigned long long* dvis = (const unsigned long long*)vis;
    const double* drep = reproj;
    const double* dobs = obs;
    float2* drange = (float2*)range;
    if (mem == MVS_MEM_HOST) {
        double* x = (double*)take(np * 3 * 8);
        unsigned long long* m = (unsigned long long*)take(np * 8);
        double* rp = (double*)take(np * 8);
        double* ob = (double*)take(np * 2 * 8);
        drange = (float2*)take(npix * 8);
        if (np) {
            CK(c, cudaMemcpyAsync(x, points, np * 3 * 8, cudaMemcpyHostToDevice, c->stream));
            CK(c, cudaMemcpyAsync(m, vis, np * 8, cudaMemcpyHostToDevice, c->stream));
            CK(c, cudaMemcpyAsync(rp, reproj, np * 8, cudaMemcpyHostToDevice, c->stream));
            CK(c, cudaMemcpyAsync(ob, obs, np * 2 * 8, cudaMemcpyHostToDevice, c->stream));
        }
        dX = x; dvis = m; drep = rp; dobs = ob;
    } else if (((uintptr_t)range & 7u)) {
        return fail(c, MVS_EINVAL, "range must be 8-byte aligned");
    }
    const double Rrow2[3] = {V.cam.R[6], V.cam.R[7], V.cam.R[8]};
    CK(c, launch_sparse_range(ref, (int)c->views.size(), Rrow2, V.cam.t[2], dX, dvis, drep, dobs, (long long)np,
                              max_reproj, W, H, d_lo, d_hi, total, uv, dep, drange, c->stream));
    if (mem == MVS_MEM_HOST) {
        CK(c, cudaMemcpyAsync(range, drange, npix * 8, cudaMemcpyDeviceToHost, c->stream));
        CK(c, cudaStreamSynchronize(c->stream));
    }
    return MVS_OK;
}

mvs_status mvs_phi_hypotheses(mvs_ctx* c, int32_t W, int32_t H, const float* depth, const uint8_t* known,
                              const mvs_phi_params* phi, float d_lo, float d_hi, float* hyp, uint8_t* valid,
                              int32_t mem) {
    if (!c) return MVS_EINVAL;
    if (!depth || !known || !phi || !hyp || !valid) return fail(c, MVS_EINVAL, "NULL argument");
    if (W < 2 || H < 2 || W > 32768 || H > 32768) return fail(c, MVS_EINVAL, "bad size");
    if (phi->n_fit < 2 || phi->n_fit > 32) return fail(c, MVS_EINVAL, "n_fit must be in 2..32");
    if (mem != MVS_MEM_DEVICE && mem != MVS_MEM_HOST) return fail(c, MVS_EINVAL, "bad mem kind");
    CK(c, cudaSetDevice(c->device));
    size_t n = (size_t)W * H;
    cudaError_t e;
    int32_t* work = (int32_t*)scratch(c, 1, n * 8 * sizeof(int32_t), &e);
    CK(c, e);
    const float* dd = depth;
    const uint8_t* kd = known;
    float* hd = hyp;
    uint8_t* vd = valid;
    if (mem == MVS_MEM_HOST) {
        char* buf = (char*)scratch(c, 0, n * (sizeof(float) * 5 + 5) + 64, &e);
        CK(c, e);
        hd = (float*)buf;
        float* dd2 = hd + 4 * n;
        uint8_t* kd2 = (uint8_t*)(dd2 + n);
        vd = kd2 + n;
        CK(c, cudaMemcpyAsync(dd2, depth, n * sizeof(float), cudaMemcpyHostToDevice, c->stream));
        CK(c, cudaMemcpyAsync(kd2, known, n, cudaMemcpyHostToDevice, c->stream));
        dd = dd2;
        kd = kd2;
    }
    CK(c, launch_phi_hypotheses(W, H, dd, kd, phi->n_fit, phi->fit_inverse, d_lo, d_hi, hd, vd, work, c->stream));
    if (mem == MVS_MEM_HOST) {
        CK(c, cudaMemcpyAsync(hyp, hd, n * 4 * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
        CK(c, cudaMemcpyAsync(valid, vd, n * 4, cudaMemcpyDeviceToHost, c->stream));
        CK(c, cudaStreamSynchronize(c->stream));
    }
    return MVS_OK;
}

mvs_status mvs_phi_hypotheses_static(mvs_ctx* c, int32_t W, int32_t H, const float* depth, const uint8_t* known,
                                     const mvs_phi_params* phi, float d_lo, float d_hi, float* hyp,
                                     uint8_t* valid) {
    if (!c) return MVS_EINVAL;
    if (!depth || !known || !phi || !hyp || !valid) return fail(c, MVS_EINVAL, "NULL argument");
    if (W < 2 || H < 2) return fail(c, MVS_EINVAL, "bad size");
    if ((long long)W * H > MVS_PHI_STATIC_MAX_PIXELS)
        return fail(c, MVS_EINVAL, "%d x %d exceeds the %d pixels of the fixed scratch", W, H,
                    MVS_PHI_STATIC_MAX_PIXELS);
    if (phi->n_fit < 2 || phi->n_fit > 32) return fail(c, MVS_EINVAL, "n_fit must be in 2..32");
    CK(c, cudaSetDevice(c->device));
    int32_t* work = nullptr;
    CK(c, phi_static_scratch(&work));
    CK(c, launch_phi_hypotheses(W, H, depth, known, phi->n_fit, phi->fit_inverse, d_lo, d_hi, hyp, valid, work,
                                c->stream));
    return MVS_OK;
}

mvs_status mvs_phi_cost(mvs_ctx* c, int32_t ref, const int32_t* srcs, int32_t n_src, const mvs_pm_params* pm,
                        const float* hyp, const uint8_t* valid, float* hcost, int32_t mem) {
    mvs_status st = check_pm(c, ref, srcs, n_src, pm);
    if (st != MVS_OK) return st;
    if (!hyp || !valid || !hcost) return fail(c, MVS_EINVAL, "NULL argument");
    if (mem != MVS_MEM_DEVICE && mem != MVS_MEM_HOST) return fail(c, MVS_EINVAL, "bad mem kind");
    CK(c, cudaSetDevice(c->device));
    const ViewData& V = c->views[ref];
    size_t n = (size_t)V.cam.width * V.cam.height;
    RefConst rc;
    make_refconst(c, ref, srcs, n_src, pm, rc);
    const float* hd = hyp;
    const uint8_t* vd = valid;
    float* cd = hcost;
    cudaError_t e;
    if (mem == MVS_MEM_HOST) {
        char* buf = (char*)scratch(c, 0, n * (8 * sizeof(float) + 4) + 64, &e);
        CK(c, e);
        float* h2 = (float*)buf;
        cd = h2 + 4 * n;
        uint8_t* v2 = (uint8_t*)(cd + 4 * n);
        CK(c, cudaMemcpyAsync(h2, hyp, n * 4 * sizeof(float), cudaMemcpyHostToDevice, c->stream));
        CK(c, cudaMemcpyAsync(v2, valid, n * 4, cudaMemcpyHostToDevice, c->stream));
        hd = h2;
        vd = v2;
    }
    CK(c, launch_phi_cost(rc, hd, vd, cd, c->stream));
    if (mem == MVS_MEM_HOST) {
        CK(c, cudaMemcpyAsync(hcost, cd, n * 4 * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
        CK(c, cudaStreamSynchronize(c->stream));
    }
    return MVS_OK;
}

mvs_status mvs_phi_mrf(mvs_ctx* c, int32_t W, int32_t H, const uint8_t* known, const float* depth, const float* hyp,
                       const uint8_t* valid, const float* hcost, const mvs_phi_params* phi, int32_t* label,
                       int32_t mem) {
    if (!c) return MVS_EINVAL;
    if (!known || !depth || !hyp || !valid || !hcost || !phi || !label) return fail(c, MVS_EINVAL, "NULL argument");
    if (W < 2 || H < 2 || W > 32768 || H > 32768) return fail(c, MVS_EINVAL, "bad size");
    if (phi->trw_iters < 0 || phi->trw_iters > 1000) return fail(c, MVS_EINVAL, "trw_iters outside 0..1000");
    if (!(phi->kappa1 > 0) || !(phi->kappa2 > 0) || !(phi->kappa3 > 1))
        return fail(c, MVS_EINVAL, "need kappa1 > 0, kappa2 > 0, kappa3 > 1");
    if (mem != MVS_MEM_DEVICE && mem != MVS_MEM_HOST) return fail(c, MVS_EINVAL, "bad mem kind");
    CK(c, cudaSetDevice(c->device));
    size_t n = (size_t)W * H;
    int gw = (W + 1) / 2, gh = (H + 1) / 2;
    size_t g = (size_t)gw * gh;
    cudaError_t e;
    float* work = (float*)scratch(c, 2, phi_mrf_work_floats(W, H) * sizeof(float), &e);
    CK(c, e);
    const uint8_t* kd = known;
    const float* dd = depth;
    const float* hd = hyp;
    const uint8_t* vd = valid;
    const float* cd = hcost;
    int32_t* ld = label;
    if (mem == MVS_MEM_HOST) {
        char* buf = (char*)scratch(c, 0, n * (9 * sizeof(float) + 5) + g * sizeof(int32_t) + 64, &e);
        CK(c, e);
        float* h2 = (float*)buf;
        float* c2 = h2 + 4 * n;
        float* d2 = c2 + 4 * n;
        int32_t* l2 = (int32_t*)(d2 + n);
        uint8_t* k2 = (uint8_t*)(l2 + g);
        uint8_t* v2 = k2 + n;
        CK(c, cudaMemcpyAsync(h2, hyp, n * 4 * sizeof(float), cudaMemcpyHostToDevice, c->stream));
        CK(c, cudaMemcpyAsync(c2, hcost, n * 4 * sizeof(float), cudaMemcpyHostToDevice, c->stream));
        CK(c, cudaMemcpyAsync(d2, depth, n * sizeof(float), cudaMemcpyHostToDevice, c->stream));
        CK(c, cudaMemcpyAsync(k2, known, n, cudaMemcpyHostToDevice, c->stream));
        CK(c, cudaMemcpyAsync(v2, valid, n * 4, cudaMemcpyHostToDevice, c->stream));
        kd = k2; dd = d2; hd = h2; vd = v2; cd = c2; ld = l2;
    }
    CK(c, launch_phi_mrf(W, H, kd, dd, hd, vd, cd, phi->kappa1, phi->kappa2, phi->kappa3, phi->trw_iters, ld, work,
                         c->stream));
    if (mem == MVS_MEM_HOST) {
        CK(c, cudaMemcpyAsync(label, ld, g * sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
        CK(c, cudaStreamSynchronize(c->stream));
    }
    return MVS_OK;
}

mvs_status mvs_phi_select(mvs_ctx* c, int32_t ref, const uint8_t* known, const float* hyp, const uint8_t* valid,
                          const int32_t* label, float* plane, int32_t mem) {
    mvs_status st = check_view(c, ref);
    if (st != MVS_OK) return st;
    if (!known || !hyp || !valid || !label || !plane) return fail(c, MVS_EINVAL, "NULL argument");
    if (((uintptr_t)plane & 15u) || ((uintptr_t)hyp & 3u) || ((uintptr_t)label & 3u))
        return fail(c, MVS_EINVAL, "plane must be 16-byte, hyp and label 4-byte aligned");
    if (mem != MVS_MEM_DEVICE && mem != MVS_MEM_HOST) return fail(c, MVS_EINVAL, "bad mem kind");
    CK(c, cudaSetDevice(c->device));
    const ViewData& V = c->views[ref];
    int W = V.cam.width, H = V.cam.height;
    size_t n = (size_t)W * H;
    size_t g = (size_t)((W + 1) / 2) * ((H + 1) / 2);
    RefConst rc;
    std::memset(&rc, 0, sizeof rc);
    rc.W = W;
    rc.H = H;
    for (int i = 0; i < 9; ++i) rc.Kinv[i] = (float)V.Kinv[i];
    cudaError_t e;
    float* newd = (float*)scratch(c, 3, n * sizeof(float), &e);
    CK(c, e);
    const uint8_t* kd = known;
    const float* hd = hyp;
    const uint8_t* vd = valid;
    const int32_t* ld = label;
    float4* pd = (float4*)plane;
    if (mem == MVS_MEM_HOST) {
        char* buf = (char*)scratch(c, 0, n * (8 * sizeof(float) + 5) + g * sizeof(int32_t) + 64, &e);
        CK(c, e);
        float4* p2 = (float4*)buf;
        float* h2 = (float*)(p2 + n);
        int32_t* l2 = (int32_t*)(h2 + 4 * n);
        uint8_t* k2 = (uint8_t*)(l2 + g);
        uint8_t* v2 = k2 + n;
        CK(c, cudaMemcpyAsync(p2, plane, n * sizeof(float4), cudaMemcpyHostToDevice, c->stream));
        CK(c, cudaMemcpyAsync(h2, hyp, n * 4 * sizeof(float), cudaMemcpyHostToDevice, c->stream));
        CK(c, cudaMemcpyAsync(l2, label, g * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream));
        CK(c, cudaMemcpyAsync(k2, known, n, cudaMemcpyHostToDevice, c->stream));
        CK(c, cudaMemcpyAsync(v2, valid, n * 4, cudaMemcpyHostToDevice, c->stream));
        kd = k2; hd = h2; vd = v2; ld = l2; pd = p2;
    }
    CK(c, launch_phi_select(rc, kd, hd, vd, ld, pd, newd, c->stream));
    if (mem == MVS_MEM_HOST) {
        CK(c, cudaMemcpyAsync(plane, pd, n * sizeof(float4), cudaMemcpyDeviceToHost, c->stream));
        CK(c, cudaStreamSynchronize(c->stream));
    }
    return MVS_OK;
}

mvs_status mvs_phi_select_min_cost(mvs_ctx* c, int32_t ref, const uint8_t* known, const float* hyp,
                                   const uint8_t* valid, const float* hcost, float* plane, int32_t mem) {
    mvs_status st = check_view(c, ref);
    if (st != MVS_OK) return st;
    if (!known || !hyp || !valid || !hcost || !plane) return fail(c, MVS_EINVAL, "NULL argument");
    if (((uintptr_t)plane & 15u) || ((uintptr_t)hyp & 15u) || ((uintptr_t)hcost & 15u) || ((uintptr_t)valid & 3u))
        return fail(c, MVS_EINVAL, "plane, hyp and hcost must be 16-byte, valid 4-byte aligned");
    if (mem != MVS_MEM_DEVICE && mem != MVS_MEM_HOST) return fail(c, MVS_EINVAL, "bad mem kind");
    CK(c, cudaSetDevice(c->device));
    const ViewData& V = c->views[ref];
    int W = V.cam.width, H = V.cam.height;
    size_t n = (size_t)W * H;
    RefConst rc;
    std::memset(&rc, 0, sizeof rc);
    rc.W = W;
    rc.H = H;
    for (int i = 0; i < 9; ++i) rc.Kinv[i] = (float)V.Kinv[i];
    cudaError_t e;
    float* newd = (float*)scratch(c, 3, n * sizeof(float), &e);
    CK(c, e);
    const uint8_t* kd = known;
    const float* hd = hyp;
    const float* cd = hcost;
    const uint8_t* vd = valid;
    float4* pd = (float4*)plane;
    if (mem == MVS_MEM_HOST) {
        // staging: plane(n f4) hyp(4n f) hcost(4n f) valid(4n) known(n), each region 16-byte aligned
        char* buf = (char*)scratch(c, 0, n * (12 * sizeof(float) + 5) + 64, &e);
        CK(c, e);
        float4* p2 = (float4*)buf;
        float* h2 = (float*)(p2 + n);
        float* c2 = h2 + 4 * n;
        uint8_t* v2 = (uint8_t*)(c2 + 4 * n);
        uint8_t* k2 = v2 + 4 * n;
        CK(c, cudaMemcpyAsync(p2, plane, n * sizeof(float4), cudaMemcpyHostToDevice, c->stream));
        CK(c, cudaMemcpyAsync(h2, hyp, n * 4 * sizeof(float), cudaMemcpyHostToDevice, c->stream));
        CK(c, cudaMemcpyAsync(c2, hcost, n * 4 * sizeof(float), cudaMemcpyHostToDevice, c->stream));
        CK(c, cudaMemcpyAsync(v2, valid, n * 4, cudaMemcpyHostToDevice, c->stream));
        CK(c, cudaMemcpyAsync(k2, known, n, cudaMemcpyHostToDevice, c->stream));
        kd = k2; hd = h2; cd = c2; vd = v2; pd = p2;
    }
    CK(c, launch_phi_select_min_cost(rc, kd, hd, vd, cd, pd, newd, c->stream));
    if (mem == MVS_MEM_HOST) {
        CK(c, cudaMemcpyAsync(plane, pd, n * sizeof(float4), cudaMemcpyDeviceToHost, c->stream));
        CK(c, cudaStreamSynchronize(c->stream));
    }
    return MVS_OK;
}

mvs_status mvs_plane_infer(mvs_ctx* c, int32_t ref, const int32_t* srcs, int32_t n_src, const mvs_pm_params* pm,
                           const mvs_phi_params* phi, const uint8_t* keep_mask, mvs_depth_map* inout) {
    mvs_status st = check_pm(c, ref, srcs, n_src, pm);
    if (st != MVS_OK) return st;
    if (!phi || !inout || !inout->plane || !inout->cost) return fail(c, MVS_EINVAL, "NULL argument");
    if (((uintptr_t)inout->plane & 15u) || ((uintptr_t)inout->cost & 3u))
        return fail(c, MVS_EINVAL, "plane must be 16-byte and cost 4-byte aligned");
    if (inout->mem != MVS_MEM_DEVICE && inout->mem != MVS_MEM_HOST) return fail(c, MVS_EINVAL, "bad mem kind");
    if (phi->n_fit < 2 || phi->n_fit > 32) return fail(c, MVS_EINVAL, "n_fit must be in 2..32");
    if (phi->trw_iters < 0 || phi->trw_iters > 1000) return fail(c, MVS_EINVAL, "trw_iters outside 0..1000");
    if (!(phi->kappa1 > 0) || !(phi->kappa2 > 0) || !(phi->kappa3 > 1))
        return fail(c, MVS_EINVAL, "need kappa1 > 0, kappa2 > 0, kappa3 > 1");
    if (phi->selection != MVS_PHI_SELECT_MRF && phi->selection != MVS_PHI_SELECT_MIN_COST)
        return fail(c, MVS_EINVAL, "unknown selection %d", (int)phi->selection);
    CK(c, cudaSetDevice(c->device));
    if ((st = ensure_map(c, ref)) != MVS_OK) return st;
    ViewData& V = c->views[ref];
    int W = V.cam.width, H = V.cam.height;
    size_t n = (size_t)W * H;
    size_t g = (size_t)((W + 1) / 2) * ((H + 1) / 2);
    int32_t mem = inout->mem;
    CK(c, cudaMemcpyAsync(V.plane, inout->plane, n * sizeof(float4), kind_in(mem), c->stream));
    CK(c, cudaMemcpyAsync(V.cost, inout->cost, n * sizeof(float), kind_in(mem), c->stream));
    cudaError_t e;
    // layout of scratch slot 4: hyp(4n f) hcost(4n f) valid(4n) depth(n f) newd(n f) label(g i) known(n);
    // hyp and hcost are 16-byte and valid 4-byte aligned (per-pixel vector loads)
    char* buf = (char*)scratch(c, 4, n * (10 * sizeof(float) + 5) + g * sizeof(int32_t) + 256, &e);
    CK(c, e);
    float* hyp = (float*)buf;
    float* hcost = hyp + 4 * n;
    uint8_t* valid = (uint8_t*)(hcost + 4 * n);
    float* depth = (float*)(valid + 4 * n);
    float* newd = depth + n;
    int32_t* label = (int32_t*)(newd + n);
    uint8_t* known = (uint8_t*)(label + g);
    int32_t* work = (int32_t*)scratch(c, 1, n * 8 * sizeof(int32_t), &e);
    CK(c, e);
    float* mwork = (float*)scratch(c, 2, phi_mrf_work_floats(W, H) * sizeof(float), &e);
    CK(c, e);
    if (keep_mask) {
        CK(c, cudaMemcpyAsync(known, keep_mask, n, kind_in(mem), c->stream));
        CK(c, launch_depth_of(W, H, V.plane, known, depth, c->stream));
    } else {
        CK(c, launch_known_from_cost(W, H, V.plane, V.cost, phi->hole_cost, known, depth, c->stream));
    }
    RefConst rc;
    make_refconst(c, ref, srcs, n_src, pm, rc);
    CK(c, launch_phi_hypotheses(W, H, depth, known, phi->n_fit, phi->fit_inverse, pm->d_lo, pm->d_hi, hyp, valid,
                                work, c->stream));
    CK(c, launch_phi_cost(rc, hyp, valid, hcost, c->stream));
    if (phi->selection == MVS_PHI_SELECT_MIN_COST) {
        CK(c, launch_phi_select_min_cost(rc, known, hyp, valid, hcost, V.plane, newd, c->stream));
    } else {
        CK(c, launch_phi_mrf(W, H, known, depth, hyp, valid, hcost, phi->kappa1, phi->kappa2, phi->kappa3,
                             phi->trw_iters, label, mwork, c->stream));
        CK(c, launch_phi_select(rc, known, hyp, valid, label, V.plane, newd, c->stream));
    }
    V.has_map = true;
    CK(c, cudaMemcpyAsync(inout->plane, V.plane, n * sizeof(float4), kind_out(mem), c->stream));
    if (mem == MVS_MEM_HOST) CK(c, cudaStreamSynchronize(c->stream));
    return MVS_OK;
}

mvs_status mvs_propose(mvs_ctx* c, int32_t ref, mvs_cnn* net, float* proposals) {
    mvs_status st = check_view(c, ref);
    if (st != MVS_OK) return st;
    if (!net || !proposals) return fail(c, MVS_EINVAL, "net and proposals must be given");
    if ((uintptr_t)proposals & 15u) return fail(c, MVS_EINVAL, "proposals must be 16-byte aligned");
    ViewData& V = c->views[ref];
    if (!V.has_map) return fail(c, MVS_ESTATE, "view %d has no depth map", ref);
    if (!cnn_shape_ok(net, V.cam.width, V.cam.height))
        return fail(c, MVS_EINVAL, "view size %dx%d is not a multiple of 16 within the network's capacity",
                    V.cam.width, V.cam.height);
    CK(c, cudaSetDevice(c->device));
    CK(c, cnn_propose(net, V.img, V.plane, V.cost, V.cam.width, V.cam.height, V.Kinv, (float4*)proposals, c->stream));
    return MVS_OK;
}

mvs_status mvs_profile(mvs_ctx* c, int32_t enable) {
    if (!c) return MVS_EINVAL;
    CK(c, cudaStreamSynchronize(c->stream));
    c->prof = enable != 0;
    c->ev_used = 0;
    c->launches0 = g_kernel_launches.load();
    if (!c->evals) CK(c, cudaMalloc(&c->evals, sizeof(unsigned long long)));
    CK(c, cudaMemsetAsync(c->evals, 0, sizeof(unsigned long long), c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    return MVS_OK;
}

mvs_status mvs_profile_read(mvs_ctx* c, double* phase_ms, int64_t* phase_launches, int64_t* kernel_launches,
                            int64_t* phase_evals) {
    if (!c) return MVS_EINVAL;
    CK(c, cudaStreamSynchronize(c->stream));
    if (phase_evals) {
        unsigned long long v = 0;
        if (c->evals) CK(c, cudaMemcpy(&v, c->evals, sizeof v, cudaMemcpyDeviceToHost));
        *phase_evals = (int64_t)v;
    }
    double ms = 0.0;
    for (size_t i = 0; i + 1 < c->ev_used; i += 2) {
        float t = 0.0f;
        CK(c, cudaEventElapsedTime(&t, c->ev[i], c->ev[i + 1]));
        ms += t;
    }
    if (phase_ms) *phase_ms = ms;
    if (phase_launches) *phase_launches = (int64_t)(c->ev_used / 2);
    if (kernel_launches) *kernel_launches = (int64_t)(g_kernel_launches.load() - c->launches0);
    return MVS_OK;
}

}  // extern "C"
