// wave_api.cu -- the C ABI of libwave.so (include/wave.h): plans, passes,
// forward / adjoint / gradient drivers and the autotuner.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "wave_host.h"
#include "wave_kernels.cuh"

namespace wave {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

wave_status fail(wave_status s, const std::string& msg)
{
    g_last_error = msg;
    return s;
}

cudaError_t launch_min_positive(const float* m, long long n, int* out, cudaStream_t st);

}  // namespace wave

using namespace wave;

namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// Tap lists of one direction (forward: sources inject, receivers sample;
// adjoint: the roles swap).
struct TapSet {
    int nsrc = 0, nrec = 0, ntaps = 0;
    int* src_ptr = nullptr;
    int4* src_ent = nullptr;
    int* rec_ptr = nullptr;
    int2* rec_ent = nullptr;
    int* rec_tptr = nullptr;
    float* rec_tw = nullptr;
    // dense receiver surface: per tap its index in the padded layout, for
    // gathering traces after one-step passes (nullptr = no gather plan)
    int* gidx = nullptr;
    void release()
    {
        cudaFree(src_ptr); cudaFree(src_ent); cudaFree(rec_ptr); cudaFree(rec_ent); cudaFree(rec_tptr); cudaFree(rec_tw);
        cudaFree(gidx);
        *this = TapSet();
    }
};

#define CK(call)                                                                                   \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return fail(e_ == cudaErrorMemoryAllocation ? WAVE_ERR_OOM : WAVE_ERR_CUDA,            \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                       \
    } while (0)

// CK for a launch of one of this library's kernels: also counts it.
#define CKL(call)           \
    do {                    \
        CK(call);           \
        p->launches++;      \
    } while (0)

template <class T>
cudaError_t upload(T** dst, const void* src, size_t bytes, cudaStream_t st)
{
    *dst = nullptr;
    if (bytes == 0) return cudaSuccess;
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(dst), bytes);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(*dst, src, bytes, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(st);  // the host vectors die after the call
}

}  // namespace

struct wave_plan_s {
    int dev = 0;
    cudaStream_t st = nullptr;
    int n[3] = {0, 0, 0};
    int nzp = 0;
    double h[3] = {0, 0, 0};
    int so = 0, R = 0;
    double dt = 0.0;
    int nt = 0;
    long long npad = 0;
    wave_options opt{};
    double vmax_model = 0.0;
    float* kap = nullptr;
    float* buf[4] = {nullptr, nullptr, nullptr, nullptr};
    float* damp = nullptr;  // [nx] [ny] [nzp] profiles
    int dxlo = 0, dxhi = 0;  // x planes without damping along x
    int* err = nullptr;
    int* err_host = nullptr;
    // sources and receivers
    std::vector<double> src_xyz, rec_xyz;
    float* wavelet = nullptr;  // [nt][nsrc]
    TapSet fwd, adj;
    bool adj_ready = false;
    float* slots = nullptr;
    size_t slots_floats = 0;
    // skewed wavefront variant: exchange planes and progress words of its tiles
    float* exch = nullptr;
    size_t exch_floats = 0;
    int* sync = nullptr;
    size_t sync_ints = 0;
    int sm_count = 1;
    // coefficients
    float c0 = 0.f, cx[kMaxR] = {}, cy[kMaxR] = {}, cz[kMaxR] = {};
    // tiling
    wave_tiling tiling{};
    wave_tiling tiling1{};  // tiling of the one-step sweeps (geom1)
    PassGeom geom, geom1;
    // tensor maps: (pointer, box rows, box cols) -> map
    std::map<std::tuple<const void*, int, int>, CUtensorMap> maps;
    // host-buffer entry staging
    float* stage_m = nullptr;
    float* stage_w = nullptr;
    float* stage_r = nullptr;
    // gradient workspace
    std::vector<float*> levels;
    cudaStream_t st2 = nullptr;                                      // recompute stream of the pipelined adjoint sweep
    cudaEvent_t gev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};  // its fork and hand-off events
    size_t level_count = 0;
    float* work = nullptr;  // misc device scratch
    size_t work_bytes = 0;
    // measurement hook
    bool prof = false;
    std::vector<cudaEvent_t> ev;
    size_t ev_used = 0;
    double prof_points = 0.0;
    long long launches = 0;
    // bumped whenever a device buffer or launch parameter that a captured
    // graph holds is replaced (batched shots recapture when it changes)
    unsigned long long gen = 0;
};

namespace {

wave_status check_cuda(const char* what, cudaError_t e)
{
    if (e == cudaSuccess) return WAVE_OK;
    return fail(e == cudaErrorMemoryAllocation ? WAVE_ERR_OOM : WAVE_ERR_CUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}

struct DeviceGuard {
    int old = -1;
    explicit DeviceGuard(int dev)
    {
        cudaGetDevice(&old);
        if (old != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        if (old >= 0) cudaSetDevice(old);
    }
};

// Tensor map of a padded [nx][ny][nzp] float array with a (1, rows, cols) box.
const CUtensorMap* get_map(wave_plan_t p, const void* ptr, int rows, int cols)
{
    auto key = std::make_tuple(ptr, rows, cols);
    auto it = p->maps.find(key);
    if (it != p->maps.end()) return &it->second;
    auto fn = encode_fn();
    if (!fn) return nullptr;
    CUtensorMap m;
    cuuint64_t dims[3] = {static_cast<cuuint64_t>(p->nzp), static_cast<cuuint64_t>(p->n[1]),
                          static_cast<cuuint64_t>(p->n[0])};
    cuuint64_t strides[2] = {static_cast<cuuint64_t>(p->nzp) * 4,
                             static_cast<cuuint64_t>(p->nzp) * 4 * static_cast<cuuint64_t>(p->n[1])};
    cuuint32_t box[3] = {static_cast<cuuint32_t>(cols), static_cast<cuuint32_t>(rows), 1};
    cuuint32_t es[3] = {1, 1, 1};
    CUresult r = fn(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(ptr), dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return nullptr;
    return &(p->maps[key] = m);
}

PassArgs base_args(wave_plan_t p, const PassGeom& g, const TapSet& taps, const float* wavelet, float* slots)
{
    PassArgs a;
    std::memset(&a, 0, sizeof(a));
    a.nx = p->n[0];
    a.ny = p->n[1];
    a.nz = p->n[2];
    a.nzp = p->nzp;
    a.sx = static_cast<long long>(p->n[1]) * p->nzp;
    a.by = g.by;
    a.bz = g.bz;
    a.xc = g.xc;
    a.nty = g.nty;
    a.ntz = g.ntz;
    a.qz = g.qz;
    a.r1y = g.r1y;
    a.zlead = g.zlead;
    a.a_rows = g.a_rows;
    a.a_cols = g.a_cols;
    a.b_rows = g.b_rows;
    a.b_cols = g.b_cols;
    a.kap = p->kap;
    a.damp_x = p->damp;
    a.damp_y = p->damp + p->n[0];
    a.damp_z = p->damp + p->n[0] + p->n[1];
    a.dxlo = p->dxlo;
    a.dxhi = p->dxhi;
    a.inv2dt = static_cast<float>(1.0 / (2.0 * p->dt));
    a.c0 = make_float2(p->c0, p->c0);
    for (int k = 0; k < kMaxR; ++k) {
        a.cx[k] = make_float2(p->cx[k], p->cx[k]);
        a.cy[k] = make_float2(p->cy[k], p->cy[k]);
        a.cz[k] = make_float2(p->cz[k], p->cz[k]);
    }
    a.src_ptr = taps.nsrc ? taps.src_ptr : nullptr;
    a.src_ent = taps.src_ent;
    a.wavelet = wavelet;
    a.nsrc = taps.nsrc;
    a.rec_ptr = (taps.nrec && slots) ? taps.rec_ptr : nullptr;
    a.rec_ent = taps.rec_ent;
    a.slots = slots;
    a.ntaps = taps.ntaps;
    a.slot_row0 = 0;
    a.err = p->err;
    return a;
}

// One pass of g.T steps from the state (u^n0, v^{n0-1/2}); writes
// (u^{n0+T}, v^{n0+T-1/2}) to (out_u, out_v).  out_v may alias v only when
// g.T == 1 (each point's increment is read and written by the same thread).
// Exchange planes and progress words of the skewed wavefront variant for a
// geometry (grown as needed; a no-op once large enough, so that a pass inside
// a graph capture never allocates).
wave_status ensure_skew_buffers(wave_plan_t p, const PassGeom& g)
{
    // exchange: per tile, every plane of its slab, 3r rows of 4 qz floats
    const size_t need = static_cast<size_t>(g.blocks) * (g.xc + 4 * p->R) * 3 * p->R * 4 * g.qz;
    if (need > p->exch_floats) {
        cudaFree(p->exch);
        p->exch = nullptr;
        p->exch_floats = 0;
        p->gen++;
        CK(cudaMalloc(&p->exch, need * 4));
        p->exch_floats = need;
    }
    const size_t nsync = static_cast<size_t>(g.blocks) + 1;
    if (nsync > p->sync_ints) {
        cudaFree(p->sync);
        p->sync = nullptr;
        p->sync_ints = 0;
        p->gen++;
        CK(cudaMalloc(&p->sync, nsync * 4));
        p->sync_ints = nsync;
    }
    return WAVE_OK;
}

// Imaging condition of the gradient, fused into a one-step adjoint pass
// (PassArgs::gacc): gacc += -(scale mu) (vn - vo) at every point.
struct Imaging {
    float* gacc;
    const float* vn;
    const float* vo;
    float scale;
};

// gather: slots is the trace array [nt][nrec] and the traces of this
// one-step pass are gathered from out_u after it (dense receiver surfaces);
// otherwise slots holds tap values [nt][ntaps], reduced after the run.
// img: imaging condition to fuse (one-step passes only).  aux: launch on the
// plan's recompute stream st2 instead of st.
wave_status run_pass(wave_plan_t p, const PassGeom& g, const TapSet& taps, const float* wavelet, float* slots, int n0,
                     const float* u, const float* v, float* out_u, float* out_v, bool gather = false,
                     const Imaging* img = nullptr, bool aux = false)
{
    cudaStream_t st = aux ? p->st2 : p->st;
    if (img && g.T != 1) return fail(WAVE_ERR_ARG, "the imaging condition is fused into one-step passes only");
    const CUtensorMap* mA = get_map(p, u, g.a_rows, g.a_cols);
    const CUtensorMap* mV = get_map(p, v, g.b_rows, g.b_cols);
    const CUtensorMap* mK = get_map(p, p->kap, g.b_rows, g.b_cols);
    if (!mA || !mV || !mK) return fail(WAVE_ERR_CUDA, "cuTensorMapEncodeTiled failed");
    PassArgs a = base_args(p, g, taps, wavelet, slots);
    a.n0 = n0;
    a.out_u = out_u;
    a.out_v = out_v;
    if (img) {
        a.gacc = img->gacc;
        a.img_vn = img->vn;
        a.img_vo = img->vo;
        a.img_scale = img->scale;
    }
    gather = gather && taps.gidx && slots && taps.nrec > 0 && g.T == 1;
    if (gather) a.rec_ptr = nullptr;
    cudaError_t e = cudaSuccess;
    if (p->prof) {
        if (p->ev_used + 2 > p->ev.size()) {
            for (int k = 0; k < 64; ++k) {
                cudaEvent_t x;
                CK(cudaEventCreate(&x));
                p->ev.push_back(x);
            }
        }
        CK(cudaEventRecord(p->ev[p->ev_used], st));
    }
    if (!g.shape) return fail(WAVE_ERR_ARG, "no compiled kernel for this tile shape");
    long long blocks = g.blocks;
    if (g.shape->unroll == 4) {
        // skewed wavefront: persistent blocks (one per SM) take the tiles in order
        wave_status sb = ensure_skew_buffers(p, g);
        if (sb) return sb;
        a.exch = p->exch;
        a.sync = p->sync;
        a.nitems = static_cast<int>(g.blocks);
        a.exch_nit = g.xc + 4 * p->R;
        CK(cudaMemsetAsync(p->sync, 0, (g.blocks + 1) * sizeof(int), st));
        blocks = std::min<long long>(g.blocks, p->sm_count);
    }
    e = g.shape->launch(*mA, *mV, *mK, a, g.block, g.smem, blocks, st);
    p->launches++;
    if (gather && e == cudaSuccess) {
        e = launch_rec_gather(out_u, taps.gidx, taps.rec_tptr, taps.rec_tw, slots + static_cast<long long>(n0) * taps.nrec,
                              taps.nrec, st);
        p->launches++;
    }
    if (p->prof) {
        CK(cudaEventRecord(p->ev[p->ev_used + 1], st));
        p->ev_used += 2;
        p->prof_points += static_cast<double>(p->n[0]) * p->n[1] * p->n[2] * g.T;
    }
    return check_cuda("pass kernel launch", e);
}

// Field state: (u, v) hold (u^n, v^{n-1/2}); f0, f1 are free buffers.
struct Fields {
    float *u, *v, *f0, *f1;
};

// One pass of g.T steps on the state f.
wave_status step_pass(wave_plan_t p, const PassGeom& g, Fields* f, const TapSet& taps, const float* wavelet,
                      float* slots, int n0, bool gather = false, const Imaging* img = nullptr)
{
    if (g.T == 1) {
        wave_status s = run_pass(p, g, taps, wavelet, slots, n0, f->u, f->v, f->f0, f->v, gather, img);
        if (s) return s;
        std::swap(f->u, f->f0);  // u <- new, f0 <- old u; v updated in place
        return WAVE_OK;
    }
    if (img) return fail(WAVE_ERR_ARG, "the imaging condition is fused into one-step passes only");
    wave_status s = run_pass(p, g, taps, wavelet, slots, n0, f->u, f->v, f->f0, f->f1);
    if (s) return s;
    std::swap(f->u, f->f0);
    std::swap(f->v, f->f1);
    return WAVE_OK;
}

// Advance `steps` steps from level n0 with the plan's tiling (T > 1 passes
// while they fit, then one-step passes).
wave_status advance(wave_plan_t p, Fields* f, const TapSet& taps, const float* wavelet, float* slots, int n0,
                    int steps, bool use_tiling, bool gather = false)
{
    int n = n0;
    const int end = n0 + steps;
    if (use_tiling && p->geom.T > 1) {
        while (n + p->geom.T <= end) {
            wave_status s = step_pass(p, p->geom, f, taps, wavelet, slots, n);
            if (s) return s;
            n += p->geom.T;
        }
    }
    const PassGeom& g1 = (use_tiling && p->geom.T == 1) ? p->geom : p->geom1;
    while (n < end) {
        wave_status s = step_pass(p, g1, f, taps, wavelet, slots, n, gather);
        if (s) return s;
        n += 1;
    }
    return WAVE_OK;
}

wave_status finish(wave_plan_t p)
{
    cudaError_t e = cudaMemcpyAsync(p->err_host, p->err, sizeof(int), cudaMemcpyDeviceToHost, p->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->st);
    if (e != cudaSuccess) return check_cuda("stream synchronize", e);
    if (*p->err_host) return fail(WAVE_ERR_TIMEOUT, "a bounded device-side wait gave up (TMA load never completed)");
    return WAVE_OK;
}

// Receivers at least this many, all in one or two z quads: traces gathered
// after one-step passes.
constexpr int kGatherMinReceivers = 4096;

// Taps of the sources and receivers of one direction (the adjoint swaps
// them); allow_gather lets a dense receiver surface use the gather plan.
wave_status build_taps(wave_plan_t p, TapSet* t, int nsrc, const double* sxyz, int nrec, const double* rxyz,
                       bool allow_gather)
{
    t->release();
    p->gen++;
    ColumnCsr sc, rc;
    std::vector<int> tptr;
    std::vector<float> tw;
    build_source_csr(nsrc, sxyz, p->h, p->n, p->nzp, &sc);
    build_receiver_csr(nrec, rxyz, p->h, p->n, p->nzp, &rc, &tptr, &tw);
    t->nsrc = nsrc;
    t->nrec = nrec;
    t->ntaps = static_cast<int>(tw.size());
    CK(upload(&t->src_ptr, sc.ptr.data(), sc.ptr.size() * 4, p->st));
    CK(upload(&t->src_ent, sc.ent.data(), sc.ent.size() * 4, p->st));
    CK(upload(&t->rec_ptr, rc.ptr.data(), rc.ptr.size() * 4, p->st));
    CK(upload(&t->rec_ent, rc.ent.data(), rc.ent.size() * 4, p->st));
    CK(upload(&t->rec_tptr, tptr.data(), tptr.size() * 4, p->st));
    CK(upload(&t->rec_tw, tw.data(), tw.size() * 4, p->st));
    std::vector<int> idx;
    if (allow_gather && receiver_gather_plan(nrec, rxyz, p->h, p->n, p->nzp, kGatherMinReceivers, &idx))
        CK(upload(&t->gidx, idx.data(), idx.size() * 4, p->st));
    return WAVE_OK;
}

wave_status ensure_slots(wave_plan_t p, size_t floats)
{
    if (floats <= p->slots_floats) return WAVE_OK;
    cudaFree(p->slots);
    p->slots = nullptr;
    p->slots_floats = 0;
    p->gen++;
    CK(cudaMalloc(&p->slots, floats * 4));
    p->slots_floats = floats;
    return WAVE_OK;
}

wave_status ensure_work(wave_plan_t p, size_t bytes)
{
    if (bytes <= p->work_bytes) return WAVE_OK;
    cudaFree(p->work);
    p->work = nullptr;
    p->work_bytes = 0;
    p->gen++;
    CK(cudaMalloc(&p->work, bytes));
    p->work_bytes = bytes;
    return WAVE_OK;
}

wave_status apply_tiling(wave_plan_t p, const wave_tiling& t)
{
    PassGeom g;
    std::string why;
    if (!make_geom(p->n, p->R, t, &g, &why)) return fail(WAVE_ERR_ARG, "tiling rejected: " + why);
    if (g.shape && g.shape->unroll == 4) {
        wave_status st = ensure_skew_buffers(p, g);
        if (st) return st;
    }
    p->tiling = t;
    p->geom = g;
    if (g.T == 1) {
        // one-step sweeps (gradient, remainders) follow a one-step tiling
        p->geom1 = g;
        p->tiling1 = t;
    }
    p->gen++;
    return WAVE_OK;
}

wave_tiling fill_tiling(wave_plan_t p, wave_tiling t)
{
    const int T = t.T > 0 ? t.T : 2;
    wave_tiling d = default_tiling(p->n, p->R, T);
    if (t.by <= 0) t.by = d.by;
    if (t.bz <= 0) t.bz = d.bz;
    if (t.xc <= 0) t.xc = d.xc;
    t.T = T;
    if (t.unroll < 0) t.unroll = 0;
    return t;
}

wave_status set_model_impl(wave_plan_t p, const float* m)
{
    const long long n = static_cast<long long>(p->n[0]) * p->n[1] * p->n[2];
    int* mn = reinterpret_cast<int*>(p->err) + 1;
    CK(cudaMemsetAsync(mn, 0x7f, sizeof(int), p->st));
    CKL(launch_min_positive(m, n, mn, p->st));
    int host_min = 0;
    CK(cudaMemcpyAsync(&host_min, mn, sizeof(int), cudaMemcpyDeviceToHost, p->st));
    CK(cudaStreamSynchronize(p->st));
    float mmin;
    std::memcpy(&mmin, &host_min, 4);
    if (host_min < 0 || !(mmin > 0.f) || !std::isfinite(mmin))
        return fail(WAVE_ERR_ARG, "model m must be positive and finite everywhere");
    p->vmax_model = 1.0 / std::sqrt(static_cast<double>(mmin));
    double dtmax = 0.0;
    wave_cfl_limit(p->so, p->h, p->vmax_model, &dtmax);
    if (p->dt > dtmax)
        return fail(WAVE_ERR_CFL, "dt = " + std::to_string(p->dt) + " ms exceeds the CFL limit " +
                                      std::to_string(dtmax) + " ms for vmax = " + std::to_string(p->vmax_model));
    CKL(launch_kappa(m, p->kap, p->n[0], p->n[1], p->n[2], p->nzp, static_cast<float>(p->dt * p->dt), p->st));
    return WAVE_OK;
}

wave_status set_damping(wave_plan_t p)
{
    const int W = p->opt.sponge_width;
    const int f = p->opt.sponge_faces;
    const double vmax = p->opt.vmax > 0.0 ? p->opt.vmax : p->vmax_model;
    std::vector<float> all, prof;
    for (int a = 0; a < 3; ++a) {
        const double dmax = W > 0 ? 3.0 * vmax * std::log(1000.0) / (2.0 * W * p->h[a]) : 0.0;
        sponge_profile(p->n[a], W, (f >> (2 * a)) & 1, (f >> (2 * a + 1)) & 1, dmax, &prof, a == 2 ? p->nzp : p->n[a]);
        all.insert(all.end(), prof.begin(), prof.end());
    }
    p->dxlo = 0;
    while (p->dxlo < p->n[0] && all[p->dxlo] != 0.f) ++p->dxlo;
    p->dxhi = p->n[0];
    while (p->dxhi > p->dxlo && all[p->dxhi - 1] != 0.f) --p->dxhi;
    CK(cudaMemcpyAsync(p->damp, all.data(), all.size() * 4, cudaMemcpyHostToDevice, p->st));
    CK(cudaStreamSynchronize(p->st));
    return WAVE_OK;
}

void destroy(wave_plan_t p)
{
    if (!p) return;
    DeviceGuard g(p->dev);
    cudaStreamSynchronize(p->st);
    cudaFree(p->kap);
    for (auto& b : p->buf) cudaFree(b);
    cudaFree(p->damp);
    cudaFree(p->err);
    cudaFreeHost(p->err_host);
    cudaFree(p->wavelet);
    p->fwd.release();
    p->adj.release();
    cudaFree(p->slots);
    cudaFree(p->stage_m);
    cudaFree(p->stage_w);
    cudaFree(p->stage_r);
    for (auto* l : p->levels) cudaFree(l);
    cudaFree(p->work);
    cudaFree(p->exch);
    cudaFree(p->sync);
    for (auto e : p->ev) cudaEventDestroy(e);
    if (p->st2) {
        cudaStreamSynchronize(p->st2);
        cudaStreamDestroy(p->st2);
    }
    for (auto e : p->gev)
        if (e) cudaEventDestroy(e);
    delete p;
}

wave_status forward_impl(wave_plan_t p, const float* u_init, float* rec_out, float* u_final)
{
    if (p->fwd.nsrc > 0 && !p->wavelet && p->nt > 0) return fail(WAVE_ERR_STATE, "sources set without a wavelet");
    if (p->fwd.nrec > 0 && p->nt > 0 && !rec_out) return fail(WAVE_ERR_ARG, "rec_out is NULL but receivers are set");
    CK(cudaMemsetAsync(p->err, 0, sizeof(int), p->st));
    Fields f{p->buf[0], p->buf[1], p->buf[2], p->buf[3]};
    if (u_init) {
        CKL(launch_init_state(u_init, f.u, f.v, p->n[0], p->n[1], p->n[2], p->nzp, p->st));
    } else {
        CK(cudaMemsetAsync(f.u, 0, p->npad * 4, p->st));
        CK(cudaMemsetAsync(f.v, 0, p->npad * 4, p->st));
    }
    // receivers: tap values into slots, reduced at the end; for a dense
    // receiver surface and one-step passes the traces are gathered into
    // rec_out after every pass
    const bool gather = p->fwd.gidx && p->fwd.nrec > 0 && p->nt > 0 && p->geom.T == 1;
    float* slots = nullptr;
    if (gather) {
        slots = rec_out;
    } else if (p->fwd.nrec > 0 && p->fwd.ntaps > 0) {
        wave_status s = ensure_slots(p, static_cast<size_t>(p->nt) * p->fwd.ntaps);
        if (s) return s;
        slots = p->slots;
    }
    wave_status s = advance(p, &f, p->fwd, p->wavelet, slots, 0, p->nt, true, gather);
    if (s) return s;
    if (p->fwd.nrec > 0 && p->nt > 0 && !gather) {
        if (p->fwd.ntaps > 0)
            CKL(launch_rec_reduce(slots, p->fwd.rec_tptr, p->fwd.rec_tw, rec_out, p->nt, p->fwd.nrec, p->fwd.ntaps,
                                 p->st));
        else
            CK(cudaMemsetAsync(rec_out, 0, static_cast<size_t>(p->nt) * p->fwd.nrec * 4, p->st));
    }
    if (u_final) CKL(launch_final_state(f.u, f.v, u_final, p->n[0], p->n[1], p->n[2], p->nzp, p->st));
    return WAVE_OK;
}

wave_status ensure_adjoint_taps(wave_plan_t p)
{
    if (p->adj_ready) return WAVE_OK;
    const int nsrc = static_cast<int>(p->src_xyz.size() / 3), nrec = static_cast<int>(p->rec_xyz.size() / 3);
    wave_status s = build_taps(p, &p->adj, nrec, p->rec_xyz.data(), nsrc, p->src_xyz.data(), false);
    if (s) return s;
    p->adj_ready = true;
    return WAVE_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------

extern "C" const char* wave_last_error(void) { return g_last_error.c_str(); }

extern "C" wave_status wave_options_default(wave_options* opt)
{
    if (!opt) return fail(WAVE_ERR_ARG, "wave_options_default: null");
    std::memset(opt, 0, sizeof(*opt));
    opt->sponge_width = 10;
    opt->sponge_faces = 0x2F;
    opt->vmax = 0.0;
    opt->stream = nullptr;
    opt->autotune = 0;
    opt->device = -1;
    return WAVE_OK;
}

extern "C" wave_status wave_plan_create(wave_plan_t* out, const int grid[3], const double spacing[3], int so,
                                        double dt, int nt, const float* m, const wave_options* opt)
{
    if (!out || !grid || !spacing || !m) return fail(WAVE_ERR_ARG, "wave_plan_create: null argument");
    *out = nullptr;
    if (so != 4 && so != 8 && so != 16) return fail(WAVE_ERR_ARG, "wave_plan_create: so must be 4, 8 or 16");
    for (int a = 0; a < 3; ++a) {
        if (grid[a] < so + 1) return fail(WAVE_ERR_ARG, "wave_plan_create: every grid extent must be >= so + 1");
        if (!(spacing[a] > 0.0) || !std::isfinite(spacing[a]))
            return fail(WAVE_ERR_ARG, "wave_plan_create: spacing must be positive");
    }
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(WAVE_ERR_ARG, "wave_plan_create: dt must be positive");
    if (nt < 0) return fail(WAVE_ERR_ARG, "wave_plan_create: nt must be >= 0");
    if (static_cast<long long>(grid[1]) * ((grid[2] + 3) / 4) >= (1LL << 31))
        return fail(WAVE_ERR_ARG, "wave_plan_create: grid too large");
    wave_options o;
    wave_options_default(&o);
    if (opt) o = *opt;
    if (o.sponge_width < 0) return fail(WAVE_ERR_ARG, "wave_plan_create: sponge_width must be >= 0");
    int dev = o.device;
    if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) return fail(WAVE_ERR_CUDA, "no CUDA device");
    DeviceGuard guard(dev);
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, m) != cudaSuccess || (attr.type != cudaMemoryTypeDevice &&
                                                               attr.type != cudaMemoryTypeManaged)) {
        cudaGetLastError();
        return fail(WAVE_ERR_ARG, "wave_plan_create: m must be device memory");
    }
    auto* p = new wave_plan_s();
    p->dev = dev;
    p->st = static_cast<cudaStream_t>(o.stream);
    if (cudaDeviceGetAttribute(&p->sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || p->sm_count < 1)
        p->sm_count = 1;
    p->opt = o;
    for (int a = 0; a < 3; ++a) {
        p->n[a] = grid[a];
        p->h[a] = spacing[a];
    }
    p->nzp = padded_nz(grid[2]);
    p->so = so;
    p->R = so / 2;
    p->dt = dt;
    p->nt = nt;
    p->npad = static_cast<long long>(grid[0]) * grid[1] * p->nzp;
    double a[9];
    fd_weights_exact(so, a);
    const double ih[3] = {1.0 / (spacing[0] * spacing[0]), 1.0 / (spacing[1] * spacing[1]),
                          1.0 / (spacing[2] * spacing[2])};
    // the k = 1 pairs enter the kernel as differences from the centre, so the
    // centre keeps only the weight of the k >= 2 pairs: a_0 + 2 a_1
    p->c0 = static_cast<float>((a[0] + 2.0 * a[1]) * (ih[0] + ih[1] + ih[2]));
    for (int k = 1; k <= p->R; ++k) {
        p->cx[k - 1] = static_cast<float>(a[k] * ih[0]);
        p->cy[k - 1] = static_cast<float>(a[k] * ih[1]);
        p->cz[k - 1] = static_cast<float>(a[k] * ih[2]);
    }
    auto bail = [&](wave_status s) {
        std::string msg = g_last_error;
        destroy(p);
        g_last_error = msg;
        return s;
    };
    cudaError_t e = cudaMalloc(&p->kap, p->npad * 4);
    for (int b = 0; b < 4 && e == cudaSuccess; ++b) e = cudaMalloc(&p->buf[b], p->npad * 4);
    if (e == cudaSuccess) e = cudaMalloc(&p->damp, (grid[0] + grid[1] + p->nzp) * 4);
    if (e == cudaSuccess) e = cudaMalloc(&p->err, 4 * sizeof(int));
    if (e == cudaSuccess) e = cudaHostAlloc(&p->err_host, sizeof(int), cudaHostAllocDefault);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return bail(check_cuda("wave_plan_create allocation", e));
    }
    if (cudaMemsetAsync(p->err, 0, 4 * sizeof(int), p->st) != cudaSuccess) return bail(fail(WAVE_ERR_CUDA, "memset"));
    wave_status s = set_model_impl(p, m);
    if (s) return bail(s);
    s = set_damping(p);
    if (s) return bail(s);
    // the one-step geometry (remainder steps, adjoint, gradient)
    std::string why;
    p->tiling1 = default_tiling(p->n, p->R, 1);
    if (!make_geom(p->n, p->R, p->tiling1, &p->geom1, &why))
        return bail(fail(WAVE_ERR_ARG, "no one-step tiling: " + why));
    wave_tiling t = o.tiling;
    if (t.T <= 0 && t.by <= 0 && t.bz <= 0 && t.xc <= 0) {
        t = default_tiling(p->n, p->R, p->R == 8 ? 1 : 2);
        PassGeom g;
        if (!make_geom(p->n, p->R, t, &g, nullptr)) t = default_tiling(p->n, p->R, 1);
    } else {
        t = fill_tiling(p, t);
    }
    s = apply_tiling(p, t);
    if (s) return bail(s);
    if (o.autotune) {
        s = wave_autotune(p, 3, 0, nullptr, nullptr, 0, nullptr);
        if (s) return bail(s);
    }
    *out = p;
    return WAVE_OK;
}

extern "C" wave_status wave_set_model(wave_plan_t p, const float* m)
{
    if (!p || !m) return fail(WAVE_ERR_ARG, "wave_set_model: null argument");
    DeviceGuard g(p->dev);
    return set_model_impl(p, m);
}

extern "C" wave_status wave_set_sources(wave_plan_t p, int nsrc, const double* xyz, const float* wavelet)
{
    if (!p || nsrc < 0) return fail(WAVE_ERR_ARG, "wave_set_sources: bad argument");
    if (nsrc > 0 && (!xyz || (!wavelet && p->nt > 0)))
        return fail(WAVE_ERR_ARG, "wave_set_sources: null positions or wavelet");
    std::string why;
    if (!positions_valid(nsrc, xyz, p->h, p->n, &why)) return fail(WAVE_ERR_ARG, "wave_set_sources: " + why);
    DeviceGuard g(p->dev);
    p->src_xyz.assign(xyz, xyz + 3 * static_cast<size_t>(nsrc));
    p->adj_ready = false;
    cudaFree(p->wavelet);
    p->wavelet = nullptr;
    p->gen++;
    if (nsrc > 0 && p->nt > 0) {
        const size_t bytes = static_cast<size_t>(p->nt) * nsrc * 4;
        CK(cudaMalloc(&p->wavelet, bytes));
        CK(cudaMemcpyAsync(p->wavelet, wavelet, bytes, cudaMemcpyDefault, p->st));
    }
    const int nrec = static_cast<int>(p->rec_xyz.size() / 3);
    return build_taps(p, &p->fwd, nsrc, p->src_xyz.data(), nrec, p->rec_xyz.data(), true);
}

extern "C" wave_status wave_set_receivers(wave_plan_t p, int nrec, const double* xyz)
{
    if (!p || nrec < 0) return fail(WAVE_ERR_ARG, "wave_set_receivers: bad argument");
    if (nrec > 0 && !xyz) return fail(WAVE_ERR_ARG, "wave_set_receivers: null positions");
    std::string why;
    if (!positions_valid(nrec, xyz, p->h, p->n, &why)) return fail(WAVE_ERR_ARG, "wave_set_receivers: " + why);
    DeviceGuard g(p->dev);
    p->rec_xyz.assign(xyz, xyz + 3 * static_cast<size_t>(nrec));
    p->adj_ready = false;
    const int nsrc = static_cast<int>(p->src_xyz.size() / 3);
    return build_taps(p, &p->fwd, nsrc, p->src_xyz.data(), nrec, p->rec_xyz.data(), true);
}

extern "C" wave_status wave_set_tiling(wave_plan_t p, const wave_tiling* t)
{
    if (!p || !t) return fail(WAVE_ERR_ARG, "wave_set_tiling: null argument");
    return apply_tiling(p, fill_tiling(p, *t));
}

extern "C" wave_status wave_get_tiling(wave_plan_t p, wave_tiling* t)
{
    if (!p || !t) return fail(WAVE_ERR_ARG, "wave_get_tiling: null argument");
    *t = p->tiling;
    return WAVE_OK;
}

extern "C" wave_status wave_get_sweep_tiling(wave_plan_t p, wave_tiling* t)
{
    if (!p || !t) return fail(WAVE_ERR_ARG, "wave_get_sweep_tiling: null argument");
    *t = p->tiling1;
    return WAVE_OK;
}

namespace {

// wave_autotune over the candidates; batch_only keeps the shapes the
// persistent batched kernel runs (and their one-step sweep tiling).
// batch_xc > 0: only the persistent batched kernel's shapes, on slabs of
// batch_xc planes (or all of x).
wave_status autotune_impl(wave_plan_t p, int passes, int T_only, int batch_xc, wave_tiling* cand,
                          double* ms_per_step, int cap, int* ncand)
{
    if (!p || passes < 1) return fail(WAVE_ERR_ARG, "wave_autotune: bad argument");
    DeviceGuard g(p->dev);
    auto cands = tiling_candidates(p->n, p->R);
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    CK(cudaMemsetAsync(p->err, 0, sizeof(int), p->st));
    CK(cudaMemsetAsync(p->buf[0], 0, p->npad * 4, p->st));
    CK(cudaMemsetAsync(p->buf[1], 0, p->npad * 4, p->st));
    double best = 1e300, best1 = 1e300;
    wave_tiling best_t = p->tiling, best1_t{};
    int count = 0;
    TapSet none;
    for (auto& t : cands) {
        if (T_only > 0 && t.T != T_only) continue;
        PassGeom geom;
        if (!make_geom(p->n, p->R, t, &geom, nullptr)) continue;
        if (batch_xc > 0 && (batch_shape_index(p->R, geom.T, geom.qz, geom.r1y, t.unroll) < 0 ||
                             t.xc != std::min(batch_xc, p->n[0])))
            continue;
        Fields f{p->buf[0], p->buf[1], p->buf[2], p->buf[3]};
        auto one = [&](int n0) -> wave_status { return step_pass(p, geom, &f, none, nullptr, nullptr, n0); };
        wave_status s = one(0);
        if (s) return s;
        CK(cudaEventRecord(e0, p->st));
        for (int k = 0; k < passes; ++k) {
            s = one(0);
            if (s) return s;
        }
        CK(cudaEventRecord(e1, p->st));
        CK(cudaEventSynchronize(e1));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        const double per_step = ms / (passes * geom.T);
        if (cand && count < cap) cand[count] = t;
        if (ms_per_step && count < cap) ms_per_step[count] = per_step;
        ++count;
        if (per_step < best) {
            best = per_step;
            best_t = t;
        }
        if (geom.T == 1 && per_step < best1) {
            best1 = per_step;
            best1_t = t;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (ncand) *ncand = count;
    wave_status s = finish(p);
    if (s) return s;
    // the fastest one-step tiling also runs the plan's one-step sweeps (the
    // recompute and adjoint sweeps of the gradient, remainder steps)
    if (best1 < 1e300) {
        PassGeom g1;
        if (make_geom(p->n, p->R, best1_t, &g1, nullptr)) {
            p->geom1 = g1;
            p->tiling1 = best1_t;
            p->gen++;
        }
    }
    return apply_tiling(p, best_t);
}

}  // namespace

extern "C" wave_status wave_autotune(wave_plan_t p, int passes, int T_only, wave_tiling* cand, double* ms_per_step,
                                     int cap, int* ncand)
{
    return autotune_impl(p, passes, T_only, 0, cand, ms_per_step, cap, ncand);
}

namespace {

// Autotuning results by key: device, grid, space order, T restriction and the
// set of compiled kernel variants (a different build never reuses an entry).
// Kept for the process; with WAVE_AUTOTUNE_CACHE=<path> also appended to, and
// looked up in, that text file (one line per result: the key, the overall
// pick "T by bz xc variant", then the fastest one-step tiling in the same
// five fields; the last line of a key wins).
struct TuneEntry {
    wave_tiling best, best1;
};
std::mutex g_tune_mu;
std::map<std::string, TuneEntry> g_tune;

std::string tune_key(wave_plan_t p, int T_only)
{
    cudaDeviceProp prop;
    std::string dev = cudaGetDeviceProperties(&prop, p->dev) == cudaSuccess ? prop.name : "device";
    for (auto& c : dev)
        if (c == ' ' || c == '|') c = '_';
    int n = 0;
    const PassShape* s = pass_shapes(&n);
    unsigned long long h = 1469598103934665603ull;  // FNV-1a over the compiled variants
    for (int i = 0; i < n; ++i)
        for (int v : {s[i].R, s[i].T, s[i].qz, s[i].ry, s[i].unroll}) {
            h ^= static_cast<unsigned long long>(v);
            h *= 1099511628211ull;
        }
    char buf[256];
    std::snprintf(buf, sizeof(buf), "%s|sm%d|%dx%dx%d|so%d|T%d|v%016llx", dev.c_str(), p->sm_count, p->n[0], p->n[1],
                  p->n[2], p->so, T_only, h);
    return buf;
}

bool tune_lookup(const std::string& key, TuneEntry* t)
{
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
        *t = it->second;
        return true;
    }
    const char* path = std::getenv("WAVE_AUTOTUNE_CACHE");
    if (!path || !*path) return false;
    FILE* f = std::fopen(path, "r");
    if (!f) return false;
    bool found = false;
    char line[512];
    while (std::fgets(line, sizeof(line), f)) {
        char k[300];
        TuneEntry r{};
        if (std::sscanf(line, "%299s %d %d %d %d %d %d %d %d %d %d", k, &r.best.T, &r.best.by, &r.best.bz, &r.best.xc,
                        &r.best.unroll, &r.best1.T, &r.best1.by, &r.best1.bz, &r.best1.xc, &r.best1.unroll) == 11 &&
            key == k) {
            *t = r;
            found = true;
        }
    }
    std::fclose(f);
    if (found) g_tune[key] = *t;
    return found;
}

void tune_store(const std::string& key, const TuneEntry& t)
{
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune[key] = t;
    const char* path = std::getenv("WAVE_AUTOTUNE_CACHE");
    if (!path || !*path) return;
    if (FILE* f = std::fopen(path, "a")) {
        std::fprintf(f, "%s %d %d %d %d %d %d %d %d %d %d\n", key.c_str(), t.best.T, t.best.by, t.best.bz, t.best.xc,
                     t.best.unroll, t.best1.T, t.best1.by, t.best1.bz, t.best1.xc, t.best1.unroll);
        std::fclose(f);
    }
}

}  // namespace

extern "C" wave_status wave_autotune_cached(wave_plan_t p, int passes, int T_only, int* from_cache)
{
    if (!p || passes < 1) return fail(WAVE_ERR_ARG, "wave_autotune_cached: bad argument");
    if (from_cache) *from_cache = 0;
    DeviceGuard g(p->dev);
    const std::string key = tune_key(p, T_only);
    TuneEntry t{};
    PassGeom geom, geom1;
    if (tune_lookup(key, &t) && make_geom(p->n, p->R, t.best, &geom, nullptr) &&
        t.best1.T == 1 && make_geom(p->n, p->R, t.best1, &geom1, nullptr)) {
        wave_status s = apply_tiling(p, t.best);
        if (s) return s;
        // the stored fastest one-step tiling runs the one-step sweeps, as after timing
        p->geom1 = geom1;
        p->tiling1 = t.best1;
        p->gen++;
        if (from_cache) *from_cache = 1;
        return WAVE_OK;
    }
    wave_status s = wave_autotune(p, passes, T_only, nullptr, nullptr, 0, nullptr);
    if (s) return s;
    tune_store(key, TuneEntry{p->tiling, p->tiling1});
    return WAVE_OK;
}

extern "C" wave_status wave_forward(wave_plan_t p, const float* u_init, float* rec_out, float* u_final)
{
    if (!p) return fail(WAVE_ERR_ARG, "wave_forward: null plan");
    DeviceGuard g(p->dev);
    wave_status s = forward_impl(p, u_init, rec_out, u_final);
    if (s) return s;
    return finish(p);
}

extern "C" wave_status wave_forward_host(wave_plan_t p, const float* m_host, const float* wavelet_host,
                                         float* rec_host)
{
    if (!p || !m_host) return fail(WAVE_ERR_ARG, "wave_forward_host: null argument");
    DeviceGuard g(p->dev);
    const size_t nm = static_cast<size_t>(p->n[0]) * p->n[1] * p->n[2];
    const int nsrc = static_cast<int>(p->src_xyz.size() / 3), nrec = static_cast<int>(p->rec_xyz.size() / 3);
    if (nsrc > 0 && !wavelet_host) return fail(WAVE_ERR_ARG, "wave_forward_host: null wavelet");
    if (nrec > 0 && !rec_host) return fail(WAVE_ERR_ARG, "wave_forward_host: null rec");
    if (!p->stage_m) CK(cudaMalloc(&p->stage_m, nm * 4));
    if (nrec > 0 && !p->stage_r) CK(cudaMalloc(&p->stage_r, static_cast<size_t>(p->nt) * nrec * 4));
    CK(cudaMemcpyAsync(p->stage_m, m_host, nm * 4, cudaMemcpyHostToDevice, p->st));
    wave_status s = set_model_impl(p, p->stage_m);
    if (s) return s;
    if (nsrc > 0 && p->nt > 0) {
        if (!p->wavelet) {
            CK(cudaMalloc(&p->wavelet, static_cast<size_t>(p->nt) * nsrc * 4));
            p->gen++;
        }
        CK(cudaMemcpyAsync(p->wavelet, wavelet_host, static_cast<size_t>(p->nt) * nsrc * 4, cudaMemcpyHostToDevice,
                           p->st));
    }
    s = forward_impl(p, nullptr, nrec > 0 ? p->stage_r : nullptr, nullptr);
    if (s) return s;
    if (nrec > 0)
        CK(cudaMemcpyAsync(rec_host, p->stage_r, static_cast<size_t>(p->nt) * nrec * 4, cudaMemcpyDeviceToHost,
                           p->st));
    return finish(p);
}

extern "C" wave_status wave_adjoint(wave_plan_t p, const float* rec_resid, float* src_out, float* v_final)
{
    if (!p || !rec_resid) return fail(WAVE_ERR_ARG, "wave_adjoint: null argument");
    DeviceGuard g(p->dev);
    wave_status s = ensure_adjoint_taps(p);
    if (s) return s;
    const int nsrc = p->adj.nrec, nrec = p->adj.nsrc;  // forward roles
    if (nsrc == 0 || nrec == 0) return fail(WAVE_ERR_STATE, "wave_adjoint: needs sources and receivers");
    const size_t wbytes = static_cast<size_t>(p->nt) * nrec * 4, obytes = static_cast<size_t>(p->nt) * nsrc * 4;
    s = ensure_work(p, wbytes + 2 * obytes + 256);
    if (s) return s;
    float* wrev = p->work;
    float* orev = reinterpret_cast<float*>(reinterpret_cast<char*>(p->work) + ((wbytes + 255) & ~size_t(255)));
    CK(cudaMemsetAsync(p->err, 0, sizeof(int), p->st));
    CKL(launch_reverse_rows(rec_resid, wrev, p->nt, nrec, p->st));
    Fields f{p->buf[0], p->buf[1], p->buf[2], p->buf[3]};
    CK(cudaMemsetAsync(f.u, 0, p->npad * 4, p->st));
    CK(cudaMemsetAsync(f.v, 0, p->npad * 4, p->st));
    float* slots = nullptr;
    if (p->adj.ntaps > 0) {
        s = ensure_slots(p, static_cast<size_t>(p->nt) * p->adj.ntaps);
        if (s) return s;
        slots = p->slots;
    }
    s = advance(p, &f, p->adj, wrev, slots, 0, p->nt, true);
    if (s) return s;
    if (src_out) {
        if (p->adj.ntaps > 0)
            CKL(launch_rec_reduce(slots, p->adj.rec_tptr, p->adj.rec_tw, orev, p->nt, nsrc, p->adj.ntaps, p->st));
        else
            CK(cudaMemsetAsync(orev, 0, obytes, p->st));
        CKL(launch_reverse_rows(orev, src_out, p->nt, nsrc, p->st));
    }
    if (v_final) CKL(launch_final_state(f.u, f.v, v_final, p->n[0], p->n[1], p->n[2], p->nzp, p->st));
    return finish(p);
}

namespace {

// One gradient evaluation: segment length K and segment count.  Everything
// it needs on the device is allocated by gradient_prepare, so that
// gradient_enqueue only issues stream work (and can be captured in a graph).
struct GradPlan {
    int K = 0, nseg = 0;
    bool pipe = false;  // two segment buffers: the recompute of segment c-1 overlaps the adjoint of segment c
};

size_t grad_rbytes(wave_plan_t p) { return static_cast<size_t>(p->nt) * p->fwd.nrec * 4; }
float* grad_rrev(wave_plan_t p)
{
    return reinterpret_cast<float*>(reinterpret_cast<char*>(p->work) + ((grad_rbytes(p) + 255) & ~size_t(255)));
}
double* grad_partial(wave_plan_t p)
{
    return reinterpret_cast<double*>(reinterpret_cast<char*>(grad_rrev(p)) + ((grad_rbytes(p) + 255) & ~size_t(255)));
}

wave_status gradient_prepare(wave_plan_t p, int checkpoint_every, GradPlan* gp)
{
    if (checkpoint_every < 0) return fail(WAVE_ERR_ARG, "wave_gradient: checkpoint_every must be >= 0");
    const int nt = p->nt;
    const int nsrc = p->fwd.nsrc, nrec = p->fwd.nrec;
    if (nsrc == 0 || nrec == 0 || !p->wavelet) return fail(WAVE_ERR_STATE, "wave_gradient: needs sources and receivers");
    wave_status s = ensure_adjoint_taps(p);
    if (s) return s;
    // K: segment length; the increments of a whole segment are kept during its adjoint sweep
    int K = checkpoint_every;
    if (K == 0 || K > nt) {
        size_t fr = 0, tot = 0;
        cudaMemGetInfo(&fr, &tot);
        const size_t need = static_cast<size_t>(nt + 3) * p->npad * 4;
        K = need + (size_t(4) << 30) < fr ? std::max(nt, 1) : std::max(1, static_cast<int>(std::sqrt(double(nt))));
    }
    const int nseg = nt > 0 ? (nt + K - 1) / K : 0;
    // levels: the checkpoints (u, v) of every segment, then one or two
    // segment buffers, each the K + 1 increments of a segment and a spare u.
    // Two when there are two segments or more and the device holds them with
    // 1 GiB to spare (or they are already allocated), unless the environment
    // variable WAVE_GRADIENT_SERIAL is set to 1 (the serial schedule, which
    // gives the same bits).
    const size_t nlev1 = static_cast<size_t>(2 * nseg) + (K + 2);
    const size_t nlev2 = nlev1 + (K + 2);
    const char* serial = std::getenv("WAVE_GRADIENT_SERIAL");
    bool pipe = false;
    if (nseg >= 2 && !(serial && std::strcmp(serial, "1") == 0)) {
        pipe = p->levels.size() >= nlev2;
        if (!pipe) {
            size_t fr = 0, tot = 0;
            if (cudaMemGetInfo(&fr, &tot) == cudaSuccess) {
                const size_t more = (nlev2 - std::min(nlev2, p->levels.size())) * static_cast<size_t>(p->npad) * 4;
                pipe = more + (size_t(1) << 30) < fr;
            }
        }
    }
    const size_t nlev = pipe ? nlev2 : nlev1;
    while (p->levels.size() < nlev) {
        float* l = nullptr;
        CK(cudaMalloc(&l, p->npad * 4));
        p->levels.push_back(l);
        p->gen++;
    }
    if (pipe && !p->st2) {
        CK(cudaStreamCreateWithFlags(&p->st2, cudaStreamNonBlocking));
        for (auto& e : p->gev) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        p->gen++;
    }
    s = ensure_work(p, 2 * grad_rbytes(p) + 256 * 8 + 1024);
    if (s) return s;
    s = ensure_slots(p, static_cast<size_t>(nt) * std::max(p->fwd.ntaps, p->adj.ntaps));
    if (s) return s;
    gp->K = K;
    gp->nseg = nseg;
    gp->pipe = pipe;
    return WAVE_OK;
}

// Stream work of the gradient on p->st: forward with a checkpoint at the
// start of every segment, residual and misfit partial sums, then the adjoint
// sweep segment by segment (recompute the increments of the segment from its
// checkpoint, then step the adjoint back through it, imaging as it goes).
// The last segment is not recomputed: the forward keeps its increments.
// With two segment buffers (gp.pipe) the recompute of segment c-1 runs on
// p->st2 into one buffer while the adjoint steps through segment c on p->st
// from the other; events order each recompute after the adjoint sweep that
// last read its buffer, and each adjoint sweep after its recompute.  The
// arithmetic and its order are the same on every schedule.
wave_status gradient_enqueue(wave_plan_t p, const GradPlan& gp, const float* d_obs, float* grad_m)
{
    const int nt = p->nt, K = gp.K, nseg = gp.nseg;
    const int nrec = p->fwd.nrec;
    const bool pipe = gp.pipe;
    float** ck = p->levels.data();  // [2 nseg]: (u^{cK}, v^{cK-1/2})
    // segment buffer b: [K + 1] increments v^{t0-1/2} .. v^{t0+K-1/2}, then the spare u of the recompute
    auto segbuf = [&](int b) { return p->levels.data() + 2 * nseg + static_cast<size_t>(b) * (K + 2); };
    auto bufof = [&](int c) { return pipe ? (c & 1) : 0; };  // segment buffer of segment c
    float* rec = p->work;
    float* rrev = grad_rrev(p);
    double* partial = grad_partial(p);
    wave_status s = WAVE_OK;
    // one-step passes of segment c from its checkpoint, keeping every increment in buffer b
    // (the checkpoint's u buffer is reused: each segment is visited once)
    auto sweep = [&](int c, int b, float* slots, bool gather, bool aux) -> wave_status {
        const int t0 = c * K;
        const int steps = std::min(K, nt - t0);
        float** seg = segbuf(b);
        float* uu[2] = {ck[2 * c], seg[K + 1]};
        CK(cudaMemcpyAsync(seg[0], ck[2 * c + 1], p->npad * 4, cudaMemcpyDeviceToDevice, aux ? p->st2 : p->st));
        for (int l = 0; l < steps; ++l) {
            wave_status r = run_pass(p, p->geom1, p->fwd, p->wavelet, slots, t0 + l, uu[l & 1], seg[l],
                                     uu[(l + 1) & 1], seg[l + 1], gather, nullptr, aux);
            if (r) return r;
        }
        return WAVE_OK;
    };
    CK(cudaMemsetAsync(p->err, 0, sizeof(int), p->st));
    // 1) forward, keeping a checkpoint at the start of every segment; the
    // last segment in one-step passes (the same bits as the plan's tiling)
    Fields f{p->buf[0], p->buf[1], p->buf[2], p->buf[3]};
    CK(cudaMemsetAsync(f.u, 0, p->npad * 4, p->st));
    CK(cudaMemsetAsync(f.v, 0, p->npad * 4, p->st));
    const bool gather = p->fwd.gidx != nullptr && (p->geom.T == 1 || nseg == 1);  // traces gathered after every pass
    float* slots = gather ? rec : p->slots;
    for (int c = 0; c < nseg; ++c) {
        CK(cudaMemcpyAsync(ck[2 * c], f.u, p->npad * 4, cudaMemcpyDeviceToDevice, p->st));
        CK(cudaMemcpyAsync(ck[2 * c + 1], f.v, p->npad * 4, cudaMemcpyDeviceToDevice, p->st));
        s = c + 1 < nseg ? advance(p, &f, p->fwd, p->wavelet, slots, c * K, K, true, gather)
                         : sweep(c, bufof(c), slots, gather, false);
        if (s) return s;
    }
    if (!gather) {
        if (p->fwd.ntaps > 0)
            CKL(launch_rec_reduce(p->slots, p->fwd.rec_tptr, p->fwd.rec_tw, rec, nt, nrec, p->fwd.ntaps, p->st));
        else
            CK(cudaMemsetAsync(rec, 0, grad_rbytes(p), p->st));
    }
    // 2) residual (time-reversed) and misfit partial sums
    CKL(launch_residual(rec, d_obs, rrev, partial, nt, nrec, p->st));
    // 3) adjoint sweep, segment by segment (the adjoint runs the same update backwards)
    Fields a{p->buf[2], p->buf[3], p->buf[1], nullptr};  // (mu, its increment), spare
    CK(cudaMemsetAsync(a.u, 0, p->npad * 4, p->st));
    CK(cudaMemsetAsync(a.v, 0, p->npad * 4, p->st));
    float* gacc = p->buf[0];  // gradient accumulator (padded layout)
    CK(cudaMemsetAsync(gacc, 0, p->npad * 4, p->st));
    const float scale = static_cast<float>(1.0 / (p->dt * p->dt));
    // adjoint steps j = t0+steps .. t0+1 of segment c: mu^j from the adjoint
    // state, source r^{j-1}, and the imaging condition
    // D_tt u^{j-1} = (v^{j-1/2} - v^{j-3/2}) / dt^2 fused into the pass
    auto adjoint = [&](int c) -> wave_status {
        const int t0 = c * K;
        const int steps = std::min(K, nt - t0);
        float** seg = segbuf(bufof(c));
        for (int j = t0 + steps; j >= t0 + 1; --j) {
            const int l = j - t0;
            const Imaging img{gacc, seg[l], seg[l - 1], scale};
            wave_status r = step_pass(p, p->geom1, &a, p->adj, rrev, nullptr, nt - j, false, &img);
            if (r) return r;
        }
        return WAVE_OK;
    };
    if (!pipe) {
        for (int c = nseg - 1; c >= 0; --c) {
            if (c + 1 < nseg) s = sweep(c, 0, nullptr, false, false);
            if (!s) s = adjoint(c);
            if (s) return s;
        }
    } else {
        // gev: [0] fork, [1 + b] recompute into buffer b done, [3 + b] adjoint sweep of buffer b done
        CK(cudaEventRecord(p->gev[0], p->st));
        CK(cudaStreamWaitEvent(p->st2, p->gev[0], 0));
        for (int c = nseg - 1; c >= 0; --c) {
            const int b = c & 1;
            if (c + 1 < nseg) CK(cudaStreamWaitEvent(p->st, p->gev[1 + b], 0));
            if (c >= 1) {
                // buffer 1 - b was last read by the adjoint sweep of segment c + 1
                if (c + 1 < nseg) CK(cudaStreamWaitEvent(p->st2, p->gev[3 + (1 - b)], 0));
                s = sweep(c - 1, 1 - b, nullptr, false, true);
                if (s) return s;
                CK(cudaEventRecord(p->gev[1 + (1 - b)], p->st2));
            }
            s = adjoint(c);
            if (s) return s;
            CK(cudaEventRecord(p->gev[3 + b], p->st));
        }
        // (the last recompute joined p->st before the last adjoint sweep)
    }
    CKL(launch_unpad_grad(gacc, grad_m, p->n[0], p->n[1], p->n[2], p->nzp, p->st));
    return WAVE_OK;
}

// Misfit 1/2 sum (rec - d_obs)^2 from the partial sums, once the stream is done.
wave_status gradient_misfit(wave_plan_t p, double* misfit)
{
    double hp[256];
    CK(cudaMemcpy(hp, grad_partial(p), sizeof(hp), cudaMemcpyDeviceToHost));
    double J = 0.0;
    for (double v : hp) J += v;
    *misfit = 0.5 * J;
    return WAVE_OK;
}

}  // namespace

extern "C" wave_status wave_gradient(wave_plan_t p, const float* d_obs, float* grad_m, double* misfit,
                                     int checkpoint_every)
{
    if (!p || !d_obs || !grad_m) return fail(WAVE_ERR_ARG, "wave_gradient: null argument");
    DeviceGuard g(p->dev);
    GradPlan gp;
    wave_status s = gradient_prepare(p, checkpoint_every, &gp);
    if (s) return s;
    s = gradient_enqueue(p, gp, d_obs, grad_m);
    if (s) return s;
    s = finish(p);
    if (s) return s;
    return misfit ? gradient_misfit(p, misfit) : WAVE_OK;
}

extern "C" wave_status wave_profile_enable(wave_plan_t p, int enable)
{
    if (!p) return fail(WAVE_ERR_ARG, "wave_profile_enable: null plan");
    p->prof = enable != 0;
    return WAVE_OK;
}

extern "C" wave_status wave_profile_read(wave_plan_t p, int reset, long long* pass_launches, double* pass_ms,
                                         double* point_steps, long long* launches)
{
    if (!p) return fail(WAVE_ERR_ARG, "wave_profile_read: null plan");
    DeviceGuard g(p->dev);
    CK(cudaStreamSynchronize(p->st));
    double ms = 0.0;
    for (size_t k = 0; k + 1 < p->ev_used; k += 2) {
        float t = 0.f;
        CK(cudaEventElapsedTime(&t, p->ev[k], p->ev[k + 1]));
        ms += t;
    }
    if (pass_launches) *pass_launches = static_cast<long long>(p->ev_used / 2);
    if (pass_ms) *pass_ms = ms;
    if (point_steps) *point_steps = p->prof_points;
    if (launches) *launches = p->launches;
    if (reset) {
        p->ev_used = 0;
        p->prof_points = 0.0;
        p->launches = 0;
    }
    return WAVE_OK;
}

// ---------------------------------------------------------------------------
// Batched shots: every plan's whole time loop captured into one CUDA graph,
// one stream per shot (forked from and joined back into the capture stream),
// replayed with a single graph launch.
// ---------------------------------------------------------------------------

struct wave_batch_s {
    std::vector<wave_plan_t> plans;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> events;
    cudaStream_t cap = nullptr;
    int dev = 0;
    // forward graph and what it was captured with
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<float*> recs;
    std::vector<unsigned long long> gens;
    // gradient graph and what it was captured with
    cudaGraph_t ggraph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    std::vector<const float*> gobs;
    std::vector<float*> ggrad;
    std::vector<int> gK;  // per shot: segment length, and 1 << 30 when its adjoint sweep overlaps the recompute
    std::vector<unsigned long long> ggens;
    // persistent kernel of the forward graph: descriptors, tensor maps and
    // items of the work queue, and its counters [next, abort, err, pad,
    // done[nplans]] (device memory, built before the capture)
    bool persistent = false;
    BatchDesc* pdesc = nullptr;
    PassArgs* pargs = nullptr;
    CUtensorMap* pmaps = nullptr;
    size_t pdesc_cap = 0, pargs_cap = 0, pmaps_cap = 0;
    int pndesc = 0;
    int4* pitems = nullptr;
    size_t pitems_cap = 0;
    int pnitems = 0;
    int* pctl = nullptr;
    int pblocks = 0;
};

namespace {

void batch_release_graph(wave_batch_t b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
}

void batch_release_ggraph(wave_batch_t b)
{
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->ggraph) cudaGraphDestroy(b->ggraph);
    b->gexec = nullptr;
    b->ggraph = nullptr;
}

std::vector<unsigned long long> batch_gens(wave_batch_t b)
{
    std::vector<unsigned long long> g;
    for (auto* p : b->plans) g.push_back(p->gen);
    return g;
}

// Capture enqueue(i) for every shot i, shot i on streams[i] (forked from and
// joined back into the capture stream), into *graph / *exec.
template <class F>
wave_status batch_capture_with(wave_batch_t b, cudaGraph_t* graph, cudaGraphExec_t* exec, F enqueue)
{
    const size_t n = b->plans.size();
    CK(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
    wave_status st = WAVE_OK;
    cudaError_t e = cudaEventRecord(b->events[n], b->cap);
    if (e != cudaSuccess) st = check_cuda("cudaEventRecord", e);
    for (size_t i = 0; i < n && !st; ++i) {
        wave_plan_t p = b->plans[i];
        cudaStream_t keep = p->st;
        p->st = b->streams[i];
        e = cudaStreamWaitEvent(p->st, b->events[n], 0);
        if (e != cudaSuccess) st = check_cuda("cudaStreamWaitEvent", e);
        if (!st) st = enqueue(i);
        if (!st) {
            e = cudaEventRecord(b->events[i], p->st);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(b->cap, b->events[i], 0);
            if (e != cudaSuccess) st = check_cuda("event join", e);
        }
        p->st = keep;
    }
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(b->cap, &g);
    if (st) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return check_cuda("cudaStreamEndCapture", e);
    *graph = g;
    CK(cudaGraphInstantiate(exec, g, 0));
    return WAVE_OK;
}

// Launch a captured graph, wait, and check every shot's error word (and the
// persistent kernel's, when the graph runs it).
wave_status batch_run(wave_batch_t b, cudaGraphExec_t exec, cudaStream_t st, bool persistent = false)
{
    for (auto* p : b->plans) CK(cudaMemsetAsync(p->err, 0, sizeof(int), st));
    CK(cudaGraphLaunch(exec, st));
    CK(cudaStreamSynchronize(st));
    for (auto* p : b->plans) {
        CK(cudaMemcpy(p->err_host, p->err, sizeof(int), cudaMemcpyDeviceToHost));
        if (*p->err_host) return fail(WAVE_ERR_TIMEOUT, "a bounded device-side wait gave up in a batched shot");
    }
    if (persistent) {
        int err = 0;
        CK(cudaMemcpy(&err, b->pctl + 2, sizeof(int), cudaMemcpyDeviceToHost));
        if (err) return fail(WAVE_ERR_TIMEOUT, err & 2 ? "a work item of the persistent batch waited too long for its shot's previous pass"
                                                       : "a bounded device-side wait gave up in the persistent batch");
    }
    return WAVE_OK;
}

// ---- the persistent kernel ---------------------------------------------

// The one-step geometry a plan's remainder passes use in the persistent
// kernel: its own one-step sweep tiling when the kernel has that shape, else
// the kernel's one-step shape (every one-step variant computes the same
// bits).  False if the plan's passes have no shape in the kernel.
bool batch_geometry(wave_plan_t p, PassGeom* g1)
{
    if (p->R != 2 && p->R != 4) return false;
    const PassGeom& g = p->geom;
    if (batch_shape_index(p->R, g.T, g.qz, g.r1y, p->tiling.unroll) < 0) return false;
    if (batch_shape_index(p->R, p->geom1.T, p->geom1.qz, p->geom1.r1y, p->tiling1.unroll) >= 0) {
        *g1 = p->geom1;
        return true;
    }
    const wave_tiling t1{1, 32, 64, p->geom1.xc > 0 ? p->geom1.xc : std::min(p->n[0], 64), 2};
    return make_geom(p->n, p->R, t1, g1, nullptr) && batch_shape_index(p->R, 1, g1->qz, g1->r1y, 2) >= 0;
}

template <class T>
wave_status grow(T** ptr, size_t* cap, size_t n)
{
    if (n <= *cap) return WAVE_OK;
    cudaFree(*ptr);
    *ptr = nullptr;
    *cap = 0;
    CK(cudaMalloc(reinterpret_cast<void**>(ptr), n * sizeof(T)));
    *cap = n;
    return WAVE_OK;
}

// Build the work queue of a forward run of every plan from zero fields: the
// passes of each plan exactly as advance() runs them (tiled passes, then
// one-step passes), one descriptor per distinct (plan, geometry, buffers),
// and the items pass level by pass level across the plans.  *ok = false (and
// nothing built) when some plan has no shape in the persistent kernel.
wave_status batch_persistent_build(wave_batch_t b, bool* ok)
{
    *ok = false;
    const size_t n = b->plans.size();
    std::vector<PassGeom> g1(n);
    for (size_t i = 0; i < n; ++i)
        if (!batch_geometry(b->plans[i], &g1[i])) return WAVE_OK;
    struct Level {
        const PassGeom* g;
        float *u, *v, *ou, *ov;
        int n0;
    };
    std::vector<std::vector<Level>> levels(n);
    for (size_t i = 0; i < n; ++i) {
        wave_plan_t p = b->plans[i];
        Fields f{p->buf[0], p->buf[1], p->buf[2], p->buf[3]};
        int t = 0;
        if (p->geom.T > 1) {
            while (t + p->geom.T <= p->nt) {
                levels[i].push_back({&p->geom, f.u, f.v, f.f0, f.f1, t});
                std::swap(f.u, f.f0);
                std::swap(f.v, f.f1);
                t += p->geom.T;
            }
        }
        const PassGeom* gr = p->geom.T == 1 ? &p->geom : &g1[i];
        while (t < p->nt) {
            levels[i].push_back({gr, f.u, f.v, f.f0, f.v, t});
            std::swap(f.u, f.f0);
            t += 1;
        }
    }
    // descriptors, their pass arguments and tensor maps
    std::vector<BatchDesc> descs;
    std::vector<PassArgs> args;
    std::vector<CUtensorMap> maps;
    std::vector<std::vector<int>> dlev(n);
    std::map<std::tuple<size_t, const PassGeom*, float*, float*, float*>, int> seen;
    for (size_t i = 0; i < n; ++i) {
        wave_plan_t p = b->plans[i];
        float* slots = nullptr;
        if (p->fwd.nrec > 0 && p->fwd.ntaps > 0) {
            wave_status st = ensure_slots(p, static_cast<size_t>(p->nt) * p->fwd.ntaps);
            if (st) return st;
            slots = p->slots;
        }
        for (const Level& lv : levels[i]) {
            auto key = std::make_tuple(i, lv.g, lv.u, lv.v, lv.ou);
            auto it = seen.find(key);
            if (it == seen.end()) {
                const CUtensorMap* mA = get_map(p, lv.u, lv.g->a_rows, lv.g->a_cols);
                const CUtensorMap* mV = get_map(p, lv.v, lv.g->b_rows, lv.g->b_cols);
                const CUtensorMap* mK = get_map(p, p->kap, lv.g->b_rows, lv.g->b_cols);
                if (!mA || !mV || !mK) return fail(WAVE_ERR_CUDA, "cuTensorMapEncodeTiled failed");
                PassArgs a = base_args(p, *lv.g, p->fwd, p->wavelet, slots);
                a.out_u = lv.ou;
                a.out_v = lv.ov;
                a.err = b->pctl + 2;
                BatchDesc d;
                d.shot = static_cast<int>(i);
                d.shape = batch_shape_index(p->R, lv.g->T, lv.g->qz, lv.g->r1y, 2);
                d.team = batch_shape_is_team(d.shape) ? 1 : 0;
                d.ntiles = static_cast<int>(lv.g->blocks);
                it = seen.emplace(key, static_cast<int>(descs.size())).first;
                descs.push_back(d);
                args.push_back(a);
                maps.push_back(*mA);
                maps.push_back(*mV);
                maps.push_back(*mK);
            }
            dlev[i].push_back(it->second);
        }
    }
    // items: pass level by pass level, every plan's tiles of that level in turn
    std::vector<int4> items;
    std::vector<int> cum(n, 0);
    for (size_t L = 0;; ++L) {
        bool any = false;
        for (size_t i = 0; i < n; ++i) {
            if (L >= levels[i].size()) continue;
            any = true;
            const Level& lv = levels[i][L];
            const int d = dlev[i][L];
            const int step = descs[d].team ? 4 : 1;  // a team item covers four tiles
            for (long long t = 0; t < lv.g->blocks; t += step)
                items.push_back(make_int4(d, static_cast<int>(t), cum[i], lv.n0));
            cum[i] += static_cast<int>(lv.g->blocks);
        }
        if (!any) break;
    }
    // the persistent kernel reads the arguments from a constant array of kMaxBatchArgs entries
    if (descs.size() > static_cast<size_t>(kMaxBatchArgs)) return WAVE_OK;
    wave_status st = grow(&b->pdesc, &b->pdesc_cap, std::max<size_t>(descs.size(), 1));
    if (st) return st;
    st = grow(&b->pargs, &b->pargs_cap, std::max<size_t>(args.size(), 1));
    if (st) return st;
    st = grow(&b->pmaps, &b->pmaps_cap, std::max<size_t>(3 * descs.size(), 3));
    if (st) return st;
    st = grow(&b->pitems, &b->pitems_cap, std::max<size_t>(items.size(), 1));
    if (st) return st;
    if (!descs.empty()) {
        CK(cudaMemcpy(b->pdesc, descs.data(), descs.size() * sizeof(BatchDesc), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(b->pargs, args.data(), args.size() * sizeof(PassArgs), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(b->pmaps, maps.data(), maps.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice));
    }
    if (!items.empty())
        CK(cudaMemcpy(b->pitems, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice));
    b->pnitems = static_cast<int>(items.size());
    b->pndesc = static_cast<int>(descs.size());
    b->pblocks = static_cast<int>(std::min<long long>(b->plans[0]->sm_count, std::max<long long>(1, b->pnitems)));
    *ok = true;
    return WAVE_OK;
}

// bound on a work item's wait for its shot's previous pass (as on every wait of the pass kernels)
constexpr unsigned long long kBatchWaitLimitNs = 2000000000ull;

BatchQueue batch_queue(wave_batch_t b, unsigned long long limit_ns)
{
    BatchQueue q;
    q.desc = b->pdesc;
    q.maps = b->pmaps;
    q.items = b->pitems;
    q.nitems = b->pnitems;
    q.next = b->pctl;
    q.abort = b->pctl + 1;
    q.err = b->pctl + 2;
    q.done = b->pctl + 4;
    q.limit_ns = limit_ns;
    return q;
}

// Stream work of the persistent forward on stream st: zero fields and
// counters, the persistent kernel, then every plan's traces from its slots.
wave_status batch_persistent_enqueue(wave_batch_t b, float* const* rec_out, cudaStream_t st)
{
    const size_t n = b->plans.size();
    for (size_t i = 0; i < n; ++i) {
        wave_plan_t p = b->plans[i];
        CK(cudaMemsetAsync(p->buf[0], 0, p->npad * 4, st));
        CK(cudaMemsetAsync(p->buf[1], 0, p->npad * 4, st));
    }
    CK(cudaMemsetAsync(b->pctl, 0, (4 + n) * sizeof(int), st));
    CK(batch_copy_args(b->pargs, b->pndesc, st));
    if (b->pnitems > 0) CK(launch_batch(batch_queue(b, kBatchWaitLimitNs), b->pblocks, st));
    for (size_t i = 0; i < n; ++i) {
        wave_plan_t p = b->plans[i];
        p->launches++;
        if (p->fwd.nrec == 0 || p->nt == 0) continue;
        if (p->fwd.ntaps > 0)
            CKL(launch_rec_reduce(p->slots, p->fwd.rec_tptr, p->fwd.rec_tw, rec_out[i], p->nt, p->fwd.nrec,
                                  p->fwd.ntaps, st));
        else
            CK(cudaMemsetAsync(rec_out[i], 0, static_cast<size_t>(p->nt) * p->fwd.nrec * 4, st));
    }
    return WAVE_OK;
}

// Capture forward_impl of every plan; plan i runs on streams[i].
wave_status batch_capture(wave_batch_t b, float* const* rec_out)
{
    const size_t n = b->plans.size();
    for (size_t i = 0; i < n; ++i) {
        wave_plan_t p = b->plans[i];
        if (p->fwd.nsrc > 0 && !p->wavelet && p->nt > 0) return fail(WAVE_ERR_STATE, "a shot has no wavelet");
        if (p->fwd.nrec > 0 && p->nt > 0 && (!rec_out || !rec_out[i]))
            return fail(WAVE_ERR_ARG, "wave_batch_forward: a shot with receivers has no rec_out");
        // everything forward_impl would allocate is allocated before the capture
        if (p->fwd.nrec > 0 && p->fwd.ntaps > 0 && !(p->fwd.gidx && p->geom.T == 1)) {
            wave_status s = ensure_slots(p, static_cast<size_t>(p->nt) * p->fwd.ntaps);
            if (s) return s;
        }
    }
    batch_release_graph(b);
    // one persistent launch for every shot when each plan's passes have a
    // shape in the persistent kernel; otherwise every shot's own launches on
    // a stream of its own
    bool ok = false;
    wave_status s = batch_persistent_build(b, &ok);
    if (s) return s;
    b->persistent = ok;
    if (ok) {
        CK(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
        s = batch_persistent_enqueue(b, rec_out, b->cap);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(b->cap, &g);
        if (s) {
            if (g) cudaGraphDestroy(g);
            return s;
        }
        if (e != cudaSuccess) return check_cuda("cudaStreamEndCapture", e);
        b->graph = g;
        CK(cudaGraphInstantiate(&b->exec, g, 0));
    } else {
        s = batch_capture_with(b, &b->graph, &b->exec, [&](size_t i) {
            return forward_impl(b->plans[i], nullptr, rec_out ? rec_out[i] : nullptr, nullptr);
        });
        if (s) return s;
    }
    b->recs.assign(rec_out ? rec_out : nullptr, rec_out ? rec_out + n : nullptr);
    b->gens = batch_gens(b);
    return WAVE_OK;
}

}  // namespace

extern "C" wave_status wave_batch_create(wave_batch_t* out, int nplans, const wave_plan_t* plans)
{
    if (!out || nplans < 1 || !plans) return fail(WAVE_ERR_ARG, "wave_batch_create: bad argument");
    *out = nullptr;
    for (int i = 0; i < nplans; ++i)
        if (!plans[i]) return fail(WAVE_ERR_ARG, "wave_batch_create: null plan");
    const int dev = plans[0]->dev;
    for (int i = 0; i < nplans; ++i)
        if (plans[i]->dev != dev) return fail(WAVE_ERR_ARG, "wave_batch_create: plans on different devices");
    DeviceGuard g(dev);
    auto* b = new wave_batch_s();
    b->dev = dev;
    b->plans.assign(plans, plans + nplans);
    cudaError_t e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    for (int i = 0; i < nplans && e == cudaSuccess; ++i) {
        cudaStream_t s;
        e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        if (e == cudaSuccess) b->streams.push_back(s);
    }
    for (int i = 0; i <= nplans && e == cudaSuccess; ++i) {
        cudaEvent_t ev;
        e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e == cudaSuccess) b->events.push_back(ev);
    }
    if (e == cudaSuccess) e = cudaMalloc(&b->pctl, (4 + static_cast<size_t>(nplans)) * sizeof(int));
    if (e != cudaSuccess) {
        wave_batch_destroy(b);
        return check_cuda("wave_batch_create", e);
    }
    *out = b;
    return WAVE_OK;
}

extern "C" wave_status wave_batch_forward(wave_batch_t b, float* const* rec_out, void* stream)
{
    if (!b) return fail(WAVE_ERR_ARG, "wave_batch_forward: null batch");
    DeviceGuard g(b->dev);
    const size_t n = b->plans.size();
    bool same = b->exec && b->recs.size() == (rec_out ? n : 0) && b->gens == batch_gens(b);
    for (size_t i = 0; same && rec_out && i < n; ++i) same = b->recs[i] == rec_out[i];
    if (!same) {
        wave_status s = batch_capture(b, rec_out);
        if (s) return s;
    }
    return batch_run(b, b->exec, static_cast<cudaStream_t>(stream), b->persistent);
}

namespace {

// Slab length of the persistent kernel's work items: 256 planes (or all of
// x), so that the pipeline fill of an item (2 r T planes) costs little beside
// its slab, while a pass level of the whole batch still has two items per SM
// (counted with the one-step team tiles, 8 x 64 points, four to an item);
// shorter slabs, down to 32 planes, for a batch too small for that.
int batch_slab(wave_batch_t b)
{
    const long long want = 2LL * (b->plans.empty() ? 1 : b->plans[0]->sm_count);
    for (int xc : {256, 128, 64}) {
        long long items = 0;
        for (auto* p : b->plans)
            items += static_cast<long long>((p->n[0] + xc - 1) / xc) * ((p->n[1] + 7) / 8) * ((p->n[2] + 63) / 64) / 4;
        if (items >= want) return xc;
    }
    return 32;
}

}  // namespace

extern "C" wave_status wave_batch_autotune(wave_batch_t b, int passes)
{
    if (!b || passes < 1) return fail(WAVE_ERR_ARG, "wave_batch_autotune: bad argument");
    DeviceGuard g(b->dev);
    const int xc = batch_slab(b);
    for (auto* p : b->plans) {
        int count = 0;
        wave_status s = autotune_impl(p, passes, 0, (p->R == 2 || p->R == 4) ? xc : 0, nullptr, nullptr, 0, &count);
        if (s) return s;
    }
    return WAVE_OK;
}

extern "C" wave_status wave_batch_get_mode(wave_batch_t b, int* persistent, int* items, int* blocks)
{
    if (!b) return fail(WAVE_ERR_ARG, "wave_batch_get_mode: null batch");
    if (persistent) *persistent = b->persistent ? 1 : 0;
    if (items) *items = b->persistent ? b->pnitems : 0;
    if (blocks) *blocks = b->persistent ? b->pblocks : 0;
    return WAVE_OK;
}

extern "C" wave_status wave_batch_selftest_withhold(wave_batch_t b, double limit_ms)
{
    if (!b || !(limit_ms > 0.0) || limit_ms > 10000.0)
        return fail(WAVE_ERR_ARG, "wave_batch_selftest_withhold: limit_ms must be in (0, 10000]");
    DeviceGuard g(b->dev);
    bool ok = false;
    wave_status s = batch_persistent_build(b, &ok);
    if (s) return s;
    if (!ok || b->pnitems == 0) return fail(WAVE_ERR_STATE, "wave_batch_selftest_withhold: the batch has no persistent work queue");
    // the graph (if any) was captured with the previous queue: capture again on the next forward
    batch_release_graph(b);
    b->gens.clear();
    const size_t n = b->plans.size();
    cudaStream_t st = b->cap;
    CK(cudaMemsetAsync(b->pctl, 0, (4 + n) * sizeof(int), st));
    // shot 0's counter starts far below any item's need: its first item waits and gives up
    const int withheld = -(1 << 30);
    CK(cudaMemcpyAsync(b->pctl + 4, &withheld, sizeof(int), cudaMemcpyHostToDevice, st));
    CK(batch_copy_args(b->pargs, b->pndesc, st));
    CK(launch_batch(batch_queue(b, static_cast<unsigned long long>(limit_ms * 1e6)), b->pblocks, st));
    CK(cudaStreamSynchronize(st));
    int err = 0;
    CK(cudaMemcpy(&err, b->pctl + 2, sizeof(int), cudaMemcpyDeviceToHost));
    if (err & 2) return fail(WAVE_ERR_TIMEOUT, "a withheld dependency made a work item give up, as intended");
    return WAVE_OK;
}

extern "C" wave_status wave_batch_gradient(wave_batch_t b, const float* const* d_obs, float* const* grad_m,
                                           double* misfit, int checkpoint_every, void* stream)
{
    if (!b || !d_obs || !grad_m) return fail(WAVE_ERR_ARG, "wave_batch_gradient: null argument");
    const size_t n = b->plans.size();
    for (size_t i = 0; i < n; ++i)
        if (!d_obs[i] || !grad_m[i]) return fail(WAVE_ERR_ARG, "wave_batch_gradient: null d_obs or grad_m entry");
    DeviceGuard g(b->dev);
    // allocate everything every shot's gradient needs (may replace buffers)
    std::vector<GradPlan> gps(n);
    std::vector<int> K(n);
    for (size_t i = 0; i < n; ++i) {
        wave_status s = gradient_prepare(b->plans[i], checkpoint_every, &gps[i]);
        if (s) return s;
        K[i] = gps[i].K | (gps[i].pipe ? (1 << 30) : 0);
    }
    bool same = b->gexec && b->gK == K && b->ggens == batch_gens(b);
    for (size_t i = 0; same && i < n; ++i) same = b->gobs[i] == d_obs[i] && b->ggrad[i] == grad_m[i];
    if (!same) {
        batch_release_ggraph(b);
        wave_status s = batch_capture_with(b, &b->ggraph, &b->gexec, [&](size_t i) {
            return gradient_enqueue(b->plans[i], gps[i], d_obs[i], grad_m[i]);
        });
        if (s) return s;
        b->gobs.assign(d_obs, d_obs + n);
        b->ggrad.assign(grad_m, grad_m + n);
        b->gK = K;
        b->ggens = batch_gens(b);
    }
    wave_status s = batch_run(b, b->gexec, static_cast<cudaStream_t>(stream));
    if (s) return s;
    for (size_t i = 0; misfit && i < n; ++i) {
        s = gradient_misfit(b->plans[i], &misfit[i]);
        if (s) return s;
    }
    return WAVE_OK;
}

extern "C" wave_status wave_batch_destroy(wave_batch_t b)
{
    if (!b) return WAVE_OK;
    DeviceGuard g(b->dev);
    if (b->cap) cudaStreamSynchronize(b->cap);
    batch_release_graph(b);
    batch_release_ggraph(b);
    cudaFree(b->pdesc);
    cudaFree(b->pargs);
    cudaFree(b->pmaps);
    cudaFree(b->pitems);
    cudaFree(b->pctl);
    for (auto s : b->streams) cudaStreamDestroy(s);
    for (auto e : b->events) cudaEventDestroy(e);
    if (b->cap) cudaStreamDestroy(b->cap);
    delete b;
    return WAVE_OK;
}

extern "C" wave_status wave_plan_destroy(wave_plan_t p)
{
    destroy(p);
    return WAVE_OK;
}

namespace wave {

namespace {
__global__ void min_positive_kernel(const float* __restrict__ m, long long n, int* out)
{
    int best = 0x7f7fffff;
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const float v = m[i];
        int b = __float_as_int(v);
        if (!(v > 0.f) || !isfinite(v)) b = -1;  // invalid marks as negative
        best = (b < 0 || best < 0) ? -1 : min(best, b);
    }
    for (int o = 16; o > 0; o >>= 1) {
        const int other = __shfl_xor_sync(0xffffffffu, best, o);
        best = (other < 0 || best < 0) ? -1 : min(best, other);
    }
    if ((threadIdx.x & 31) == 0) atomicMin(out, best);
}
}  // namespace

cudaError_t launch_min_positive(const float* m, long long n, int* out, cudaStream_t st)
{
    long long b = (n + 255) / 256;
    if (b > 152 * 16) b = 152 * 16;
    if (b < 1) b = 1;
    min_positive_kernel<<<static_cast<unsigned>(b), 256, 0, st>>>(m, n, out);
    return cudaGetLastError();
}

}  // namespace wave
