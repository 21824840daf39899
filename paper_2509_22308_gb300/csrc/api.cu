// Host runtime of the single-domain solver: the C ABI of include/lbm_em.h.
//
// Time handling.  Every step kernel reads the current time t from one of two device
// words and writes t + 1 into the other (the pair alternates with the ping-pong
// distribution buffers), so a captured run of an even number of steps is replayed
// unchanged for any start time: source phases and Fourier weights come from t.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/lbm_em.h"
#include "common.cuh"
#include "launchers.h"
#include "runtime.h"
#include "step2.cuh"
#include "step2_tma.h"
#include "step_f16.cuh"
#include "step_stream.h"

using namespace lbmem;

namespace lbmem {
thread_local std::string g_last_error;

lbm_em_status set_error(lbm_em_status st, const std::string &msg) {
    g_last_error = msg;
    return st;
}

lbm_em_status cuda_status(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return LBM_EM_OK;
    cudaGetLastError();  // clear a non-sticky error
    return set_error(e == cudaErrorMemoryAllocation ? LBM_EM_ENOMEM : LBM_EM_ECUDA,
                     std::string(what) + ": " + cudaGetErrorString(e));
}

void incident_constants(int period, double E0, double *pr, double *pi, double *qr, double *qi) {
    // Right-going vacuum branch of the lattice dispersion relation: w = (3 - z)/(z(3z - 1)),
    // z = e^{-i omega}; E_z = Re[E w^x z^t] with E = i E0, and the +x population of e_z is
    // Re[P w^x z^t] with P = 2E / (3(wz + 1)).
    const double om = 2.0 * M_PI / (double)period;
    const std::complex<double> z = std::exp(std::complex<double>(0.0, -om));
    const std::complex<double> w = (3.0 - z) / (z * (3.0 * z - 1.0));
    const std::complex<double> E(0.0, E0);
    const std::complex<double> P = 2.0 * E / (3.0 * (w * z + 1.0));
    const std::complex<double> Q = P * w;
    *pr = P.real();
    *pi = P.imag();
    *qr = Q.real();
    *qi = Q.imag();
}

double lattice_wavenumber(int period) {
    const double om = 2.0 * M_PI / (double)period;
    const std::complex<double> z = std::exp(std::complex<double>(0.0, -om));
    return std::arg((3.0 - z) / (z * (3.0 * z - 1.0)));
}

std::vector<double2> phase_table(int period) {
    std::vector<double2> cs(period);
    const double om = 2.0 * M_PI / (double)period;
    for (int t = 0; t < period; ++t) cs[t] = make_double2(std::cos(om * (double)t), std::sin(om * (double)t));
    return cs;
}

lbm_em_status check_source(const lbm_em_source *s) {
    if (!s) return set_error(LBM_EM_EINVAL, "source is NULL");
    if (s->period_steps < 4) return set_error(LBM_EM_EINVAL, "source.period_steps must be >= 4");
    if (s->ramp_steps < 0) return set_error(LBM_EM_EINVAL, "source.ramp_steps must be >= 0");
    if (s->kind < 0 || s->kind > 2) return set_error(LBM_EM_EINVAL, "source.kind out of range");
    if (!std::isfinite(s->E0)) return set_error(LBM_EM_EINVAL, "source.E0 must be finite");
    return LBM_EM_OK;
}

lbm_em_status check_janus(const lbm_em_janus *j) {
    if (!j) return set_error(LBM_EM_EINVAL, "janus spec is NULL");
    if (!(j->a > 0.0) || !std::isfinite(j->a)) return set_error(LBM_EM_EINVAL, "janus.a must be > 0");
    if (!std::isfinite(j->phi0)) return set_error(LBM_EM_EINVAL, "janus.phi0 must be finite");
    if (!(j->eps1 >= 1.0) || !std::isfinite(j->eps1)) return set_error(LBM_EM_EINVAL, "janus.eps1 must be >= 1");
    if (!j->pec2 && (!(j->eps2 >= 1.0) || !std::isfinite(j->eps2)))
        return set_error(LBM_EM_EINVAL, "janus.eps2 must be >= 1");
    return LBM_EM_OK;
}

void janus_center(const lbm_em_janus *j, int nx, int ny, double *cx, double *cy) {
    *cx = std::isnan(j->cx) ? 0.5 * (double)(nx - 1) : j->cx;
    *cy = std::isnan(j->cy) ? 0.5 * (double)(ny - 1) : j->cy;
}

int round_up(int v, int m) { return (v + m - 1) / m * m; }

lbm_em_status build_contour(int nx, int ny, const lbm_em_contour *c, ContourHost *out) {
    if (!c) return set_error(LBM_EM_EINVAL, "contour is NULL");
    if (!(c->radius > 0.0) || !std::isfinite(c->radius)) return set_error(LBM_EM_EINVAL, "contour.radius must be > 0");
    if (!(c->a > 0.0) || !std::isfinite(c->a)) return set_error(LBM_EM_EINVAL, "contour.a must be > 0");
    if (c->n_points != 0 && c->n_points < 8) return set_error(LBM_EM_EINVAL, "contour.n_points must be 0 or >= 8");
    const double cx = std::isnan(c->cx) ? 0.5 * (double)(nx - 1) : c->cx;
    const double cy = std::isnan(c->cy) ? 0.5 * (double)(ny - 1) : c->cy;
    const double R = c->radius;
    if (!(cx - R >= 1.0 && cx + R <= (double)(nx - 2) && cy - R >= 1.0 && cy + R <= (double)(ny - 2)))
        return set_error(LBM_EM_EINVAL, "contour circle must lie inside the lattice (1 cell margin)");
    const int N = c->n_points > 0 ? c->n_points : (int)(2.0 * std::ceil(2.0 * M_PI * R));
    out->R = R;
    out->dl = R * 2.0 * M_PI / (double)N;
    out->pts.resize(N);
    std::map<long long, int> slots;
    out->site_xy.clear();
    out->y0 = ny;
    out->y1 = -1;
    for (int k = 0; k < N; ++k) {
        const double phi = 2.0 * M_PI * (double)k / (double)N;
        const double px = cx + R * std::cos(phi), py = cy + R * std::sin(phi);
        const int i = (int)std::floor(px), jj = (int)std::floor(py);
        const double fx = px - i, fy = py - jj;
        ContourPt &p = out->pts[k];
        const int cxs[4] = {i, i + 1, i, i + 1}, cys[4] = {jj, jj, jj + 1, jj + 1};
        p.w[0] = (1 - fx) * (1 - fy);
        p.w[1] = fx * (1 - fy);
        p.w[2] = (1 - fx) * fy;
        p.w[3] = fx * fy;
        for (int q = 0; q < 4; ++q) {
            const long long key = (long long)cys[q] * nx + cxs[q];
            auto it = slots.find(key);
            int s;
            if (it == slots.end()) {
                s = (int)slots.size();
                slots.emplace(key, s);
                out->site_xy.push_back(cxs[q]);
                out->site_xy.push_back(cys[q]);
                out->y0 = std::min(out->y0, cys[q]);
                out->y1 = std::max(out->y1, cys[q]);
            } else {
                s = it->second;
            }
            p.s[q] = s;
        }
        p.nx = std::cos(phi);
        p.ny = std::sin(phi);
    }
    out->n_slots = (int)slots.size();
    out->F0 = M_PI * c->a * out->E0 * out->E0 / 4.0;
    out->M0 = 2.0 * out->F0 * c->a;
    return LBM_EM_OK;
}
}  // namespace lbmem

// ---- memory ---------------------------------------------------------------------------
// Device buffers of a handle come from the device's default stream-ordered pool
// (cudaMallocAsync / cudaFreeAsync on the handle's stream): no call waits for the device,
// and up to kPoolKeepBytes of freed memory stay in the pool for the next handle, so
// creating and destroying handles in a loop does not map and unmap memory each time.
// Host-to-device uploads go through pinned blocks that the process keeps for reuse
// (cudaMallocHost is slow); each block is reused only after its last copy has completed.
static const uint64_t kPoolKeepBytes = 4ull << 30;
static std::mutex g_pool_mu;
static bool g_pool_ready[128];
static std::multimap<size_t, void *> g_pinned_free;  // capacity -> pinned block

static void prepare_pool(int dev) {
    std::lock_guard<std::mutex> lock(g_pool_mu);
    if (dev < 0 || dev >= 128 || g_pool_ready[dev]) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t keep = kPoolKeepBytes;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    cudaGetLastError();
    g_pool_ready[dev] = true;
}

static cudaError_t pinned_get(size_t bytes, void **p, size_t *cap) {
    if (alloc_should_fail()) return cudaErrorMemoryAllocation;
    size_t c = 4096;
    while (c < bytes) c <<= 1;
    {
        std::lock_guard<std::mutex> lock(g_pool_mu);
        auto it = g_pinned_free.lower_bound(c);
        if (it != g_pinned_free.end()) {
            *cap = it->first;
            *p = it->second;
            g_pinned_free.erase(it);
            alloc_held(1);
            return cudaSuccess;
        }
    }
    *cap = c;
    const cudaError_t e = cudaMallocHost(p, c);
    if (e == cudaSuccess) alloc_held(1);
    return e;
}

static void pinned_put(void *p, size_t cap) {
    if (!p) return;
    alloc_held(-1);
    std::lock_guard<std::mutex> lock(g_pool_mu);
    g_pinned_free.emplace(cap, p);
}

struct lbm_em {
    int dev = 0;
    int nx = 0, ny = 0, pitch = 0, prec = 0;
    int pol = POL_TM;  // POL_TM or POL_TE (LBM_EM_FLAG_TE)
    size_t pstride = 0, elem = 0, buf_bytes = 0;
    cudaStream_t stream = nullptr, cap = nullptr;
    bool own_stream = false;
    void *buf[2] = {nullptr, nullptr};
    uint8_t *d_mat = nullptr;
    void *d_mtab = nullptr;
    double eps_table[256];
    bool pec_id[256];
    long long *d_time = nullptr;
    unsigned *d_err = nullptr;
    double2 *d_cs = nullptr;
    SourceParams src{};
    lbm_em_source srccfg{};
    int64_t t = 0;
    int cur = 0;      // buffer holding the current state (and device time word)
    // a bounded wait for a tile copy gave up (seen by lbm_em_sync): a copy may still have
    // been in flight when its CTA left, so the handle refuses further steps
    bool timed_out = false;
    bool tb = false;  // two steps per launch (temporal blocking) for the HBM-bound forms
    // FP32 two-step launches: tensor maps of the two state buffers and of the material
    // ids, and the persistent grid
    CUtensorMap tmap[2], idmap;
    CUtensorMap f16_gmap[2], f16_fmap[2];  // FP16-deviation form: deviation and field planes per buffer
    CUtensorMap tmap3[2], idmap3;          // FP32, three steps per launch
    bool t3 = false;                       // three steps per launch (FP32)
    // four steps per launch (FP32, FP16-deviation): row-streaming kernel, its maps per buffer
    // (FP32 state or FP16 deviations; FP16 fields) and of the ids, and its work plan
    bool s4 = false;
    CUtensorMap s4_smap[2], s4_fmap[2], s4_imap;
    StreamPlan s4_plan{}, s4_plan_acc{};  // plain and (FP32) accumulating four-step launches
    int tma3_ctas = 0;
    int tma_ctas = 0;
    // contour and accumulators
    bool has_contour = false;
    lbm_em_contour contour{};
    ContourHost ch;
    int *d_slot = nullptr;
    double *d_acc = nullptr;
    float *d_stage = nullptr;  // four-step accumulation: 12 staged fields per stencil slot
    ContourPt *d_pts = nullptr;
    double2 *d_inc = nullptr;   // incident E_z phasor at every stencil site (far field)
    double *d_out = nullptr;
    int64_t n_acc = 0;
    // graphs of kGraphSteps steps starting at an even time
    cudaGraphExec_t g_plain = nullptr, g_acc = nullptr;
    double *d_fields = nullptr;
    void *h_stage = nullptr;       // pinned staging of the material table (async uploads)
    size_t stage_cap = 0;
    cudaEvent_t stage_ev = nullptr;  // the last table upload from h_stage
    void *h_up = nullptr;          // pinned staging of the other uploads (ids, contour)
    size_t up_cap = 0;
    cudaEvent_t up_ev = nullptr;   // the last upload from h_up
};

template <typename P>
static cudaError_t dev_alloc(lbm_em *h, P **p, size_t bytes) {
    return dmalloc_async((void **)p, bytes, h->stream);
}

template <typename P>
static void dev_free(lbm_em *h, P *&p) {
    dfree_async((void *)p, h->stream);
    p = nullptr;
}

// Pinned staging of at least `bytes` for an upload on the handle's stream: waits for the
// previous upload from it (normally long finished), growing the block when needed.
static cudaError_t upload_staging(lbm_em *h, size_t bytes, void **p) {
    cudaError_t e = cudaEventSynchronize(h->up_ev);
    if (e != cudaSuccess) return e;
    if (h->up_cap < bytes) {  // the larger block first: a failed grow keeps the old one
        void *np = nullptr;
        size_t ncap = 0;
        e = pinned_get(bytes, &np, &ncap);
        if (e != cudaSuccess) return e;
        pinned_put(h->h_up, h->up_cap);
        h->h_up = np;
        h->up_cap = ncap;
    }
    *p = h->h_up;
    return cudaSuccess;
}

static const int kGraphSteps = 32;

template <typename T>
static StepArgs<T> make_args(const lbm_em *h) {
    StepArgs<T> a{};
    a.nx = h->nx;
    a.ny = h->ny;
    a.pitch = h->pitch;
    a.pol = h->pol;
    a.pstride = h->pstride;
    a.mat = h->d_mat;
    a.mtab = (const MatT<T> *)h->d_mtab;
    a.src = h->src;
    a.accp.slot = h->d_slot;
    a.accp.acc = h->d_acc;
    a.accp.y0 = h->ch.y0;
    a.accp.y1 = h->ch.y1;
    a.err = h->d_err;
    a.runaway = runaway_bits<T>(h->srccfg.E0);
    return a;
}

static F16Args make_f16_args(const lbm_em *h, int p) {
    F16Args a{};
    a.nx = h->nx;
    a.ny = h->ny;
    a.pitch = h->pitch;
    a.pstride = h->pstride;
    a.mat = h->d_mat;
    a.mtab = (const MatT<float> *)h->d_mtab;
    a.src = h->src;
    a.accp.slot = h->d_slot;
    a.accp.acc = h->d_acc;
    a.accp.y0 = h->ch.y0;
    a.accp.y1 = h->ch.y1;
    a.err = h->d_err;
    a.runaway = runaway_bits<float>(h->srccfg.E0);
    a.scale = f16_scale(h->srccfg.E0);
    a.inv_scale = 1.0f / a.scale;  // exact: a power of two
    const size_t hb = f16_half_bytes(h->pstride), fb = f16_plane_bytes(h->pstride);
    char *in = (char *)h->buf[p], *out = (char *)h->buf[1 - p];
    a.g = (const __half *)in;
    a.fe = (const float *)(in + hb);
    a.fhx = (const float *)(in + hb + fb);
    a.fhy = (const float *)(in + hb + 2 * fb);
    a.g_out = (__half *)out;
    a.fe_out = (float *)(out + hb);
    a.fhx_out = (float *)(out + hb + fb);
    a.fhy_out = (float *)(out + hb + 2 * fb);
    return a;
}

// One step: state in buf[p] -> buf[1 - p], time word p -> 1 - p.
static cudaError_t enqueue_step(lbm_em *h, bool acc, cudaStream_t s, int p) {
    if (h->prec == LBM_EM_F16DEV)
        return launch_step_f16(make_f16_args(h, p), h->d_time + p, h->d_time + (1 - p), acc, s);
    if (h->prec == LBM_EM_F64)
        return launch_step<double>(make_args<double>(h), (const double *)h->buf[p], (double *)h->buf[1 - p],
                                   h->d_time + p, h->d_time + (1 - p), acc, s);
    if (h->prec == LBM_EM_F32X2)
        return launch_step<df>(make_args<df>(h), (const df *)h->buf[p], (df *)h->buf[1 - p], h->d_time + p,
                               h->d_time + (1 - p), acc, s);
    return launch_step<float>(make_args<float>(h), (const float *)h->buf[p], (float *)h->buf[1 - p],
                              h->d_time + p, h->d_time + (1 - p), acc, s);
}

// Two steps in one launch (temporal blocking): buf[p] -> buf[1 - p].
static cudaError_t enqueue_step2(lbm_em *h, bool acc, cudaStream_t s, int p) {
    if (h->prec == LBM_EM_F16DEV)
        return launch_step2_f16_tma(make_f16_args(h, p), &h->f16_gmap[p], &h->f16_fmap[p], &h->idmap, h->d_time + p,
                                    h->d_time + (1 - p), acc, h->tma_ctas, s);
    if (h->prec == LBM_EM_F32X2)
        return launch_step2<df>(make_args<df>(h), (const df *)h->buf[p], (df *)h->buf[1 - p], h->d_time + p,
                                h->d_time + (1 - p), acc, s);
    return launch_step2_tma(make_args<float>(h), &h->tmap[p], &h->idmap, (float *)h->buf[1 - p], h->d_time + p,
                            h->d_time + (1 - p), acc, h->tma_ctas, s);
}

// Three steps in one launch (FP32): buf[p] -> buf[1 - p].
static cudaError_t enqueue_step3(lbm_em *h, bool acc, cudaStream_t s, int p) {
    return launch_step3_tma(make_args<float>(h), &h->tmap3[p], &h->idmap3, (float *)h->buf[1 - p], h->d_time + p,
                            h->d_time + (1 - p), acc, h->tma3_ctas, s);
}

// Four steps in one launch, with or without the Fourier accumulation: buf[p] -> buf[1 - p].
static cudaError_t enqueue_step4(lbm_em *h, bool acc, cudaStream_t s, int p) {
    if (h->prec == LBM_EM_F16DEV) {
        const F16Args fa = make_f16_args(h, p);
        return launch_step4_stream(make_args<float>(h), &fa, &h->s4_smap[p], &h->s4_fmap[p], &h->s4_imap, nullptr,
                                   acc ? h->s4_plan_acc : h->s4_plan, h->d_time + p, h->d_time + (1 - p), acc,
                                   h->d_stage, acc ? h->ch.n_slots : 0, s);
    }
    return launch_step4_stream(make_args<float>(h), nullptr, &h->s4_smap[p], &h->s4_fmap[p], &h->s4_imap,
                               (float *)h->buf[1 - p], acc ? h->s4_plan_acc : h->s4_plan, h->d_time + p,
                               h->d_time + (1 - p), acc, h->d_stage, acc ? h->ch.n_slots : 0, s);
}

// Steps one launch advances: the handle's mode (accumulating steps too).
static int launch_steps(const lbm_em *h, bool acc) {
    if (h->s4) return 4;
    return h->t3 ? 3 : h->tb ? 2 : 1;
}

// Steps per captured graph: kGraphSteps (8, 16 or 32 launches), or 30 (ten launches) with
// three steps per launch.
static int graph_steps(const lbm_em *h, bool acc) { return launch_steps(h, acc) == 3 ? 30 : kGraphSteps; }

// One launch of `m` steps from buffer p.
static cudaError_t enqueue_mode(lbm_em *h, int m, bool acc, cudaStream_t s, int p) {
    switch (m) {
        case 4: return enqueue_step4(h, acc, s, p);
        case 3: return enqueue_step3(h, acc, s, p);
        case 2: return enqueue_step2(h, acc, s, p);
        default: return enqueue_step(h, acc, s, p);
    }
}

// graph_steps(h, acc) steps starting from buffer 0 (an even number of launches, so the
// state is back in buffer 0 at the end).
static lbm_em_status build_graph(lbm_em *h, bool acc, cudaGraphExec_t *out) {
    cudaGraph_t g = nullptr;
    lbm_em_status st = cuda_status(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal),
                                   "cudaStreamBeginCapture");
    if (st) return st;
    cudaError_t e = cudaSuccess;
    const int m = launch_steps(h, acc), launches = graph_steps(h, acc) / m;
    for (int i = 0; i < launches && e == cudaSuccess; ++i) e = enqueue_mode(h, m, acc, h->cap, i & 1);
    cudaError_t e2 = cudaStreamEndCapture(h->cap, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_status(e != cudaSuccess ? e : e2, "capturing the step graph");
    }
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    return cuda_status(e, "cudaGraphInstantiate");
}

// Every FP32 mode gives the same bits (the four-step FP16-deviation launch rounds its stored
// state once per launch, see step_stream.cu); two-step launches and their graphs start at
// even t (an odd start takes one single step first), three- and four-step launches anywhere,
// and a remainder shorter than a launch's steps takes single steps.
static lbm_em_status run_steps(lbm_em *h, int64_t n, bool acc) {
    const int m = launch_steps(h, acc), gs = graph_steps(h, acc);
    while (n > 0) {
        const bool even = (h->t & 1) == 0;
        if (h->cur == 0 && n >= gs && (even || m != 2)) {
            cudaGraphExec_t *g = acc ? &h->g_acc : &h->g_plain;
            if (!*g) {
                lbm_em_status st = build_graph(h, acc, g);
                if (st) return st;
            }
            lbm_em_status st = cuda_status(cudaGraphLaunch(*g, h->stream), "cudaGraphLaunch");
            if (st) return st;
            h->t += gs;
            n -= gs;
        } else if (m > 1 && n >= m && (even || m != 2)) {
            lbm_em_status st = cuda_status(enqueue_mode(h, m, acc, h->stream, h->cur), "step launch");
            if (st) return st;
            h->cur ^= 1;
            h->t += m;
            n -= m;
        } else {
            lbm_em_status st = cuda_status(enqueue_step(h, acc, h->stream, h->cur), "step launch");
            if (st) return st;
            h->cur ^= 1;
            h->t += 1;
            n -= 1;
        }
    }
    return LBM_EM_OK;
}

// Stream-ordered: the buffers go back to the pool after the work already queued on the
// handle's stream (an executable graph still in flight is freed when it completes).
static void free_contour(lbm_em *h) {
    if (h->g_acc) cudaGraphExecDestroy(h->g_acc);
    h->g_acc = nullptr;
    dev_free(h, h->d_slot);
    dev_free(h, h->d_acc);
    dev_free(h, h->d_stage);
    dev_free(h, h->d_pts);
    dev_free(h, h->d_inc);
    h->has_contour = false;
}

static void free_handle(lbm_em *h) {
    if (!h) return;
    cudaSetDevice(h->dev);
    if (h->stream) {
        free_contour(h);
        dev_free(h, h->buf[0]);
        dev_free(h, h->buf[1]);
        dev_free(h, h->d_mat);
        dev_free(h, h->d_mtab);
        dev_free(h, h->d_time);
        dev_free(h, h->d_err);
        dev_free(h, h->d_cs);
        dev_free(h, h->d_out);
        dev_free(h, h->d_fields);
        cudaStreamSynchronize(h->stream);  // the pinned blocks are reused by other handles
    }
    if (h->g_plain) cudaGraphExecDestroy(h->g_plain);
    if (h->cap) cudaStreamDestroy(h->cap);
    if (h->stage_ev) cudaEventDestroy(h->stage_ev);
    if (h->up_ev) cudaEventDestroy(h->up_ev);
    pinned_put(h->h_stage, h->stage_cap);
    pinned_put(h->h_up, h->up_cap);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

template <typename T>
static std::vector<MatT<T>> material_table(const double *eps, const bool *pec) {
    std::vector<MatT<T>> tab(256);
    for (int i = 0; i < 256; ++i) tab[i] = material_entry<T>(eps[i], pec[i]);
    return tab;
}

// Allocate and initialise everything except the material ids.
static lbm_em_status create_common(const lbm_em_grid *g, const lbm_em_source *s, lbm_em **out) {
    if (!g || !out) return set_error(LBM_EM_EINVAL, "grid/out is NULL");
    *out = nullptr;
    if (g->nx < 4 || g->ny < 4) return set_error(LBM_EM_EINVAL, "nx and ny must be >= 4");
    if (g->flags & ~(LBM_EM_FLAG_SINGLE_STEP | LBM_EM_FLAG_TWO_STEP | LBM_EM_FLAG_TE | LBM_EM_FLAG_THREE_STEP |
                     LBM_EM_FLAG_FOUR_STEP))
        return set_error(LBM_EM_EINVAL, "unknown grid flags");
    const int step_flags = g->flags & (LBM_EM_FLAG_SINGLE_STEP | LBM_EM_FLAG_TWO_STEP | LBM_EM_FLAG_THREE_STEP |
                                       LBM_EM_FLAG_FOUR_STEP);
    if (step_flags & (step_flags - 1)) return set_error(LBM_EM_EINVAL, "at most one steps-per-launch flag");
    if ((g->flags & LBM_EM_FLAG_FOUR_STEP) && g->precision != LBM_EM_F32 && g->precision != LBM_EM_F16DEV)
        return set_error(LBM_EM_EINVAL, "LBM_EM_FLAG_FOUR_STEP is for LBM_EM_F32 and LBM_EM_F16DEV");
    if ((g->flags & LBM_EM_FLAG_THREE_STEP) &&
        (g->precision != LBM_EM_F32 || (g->flags & (LBM_EM_FLAG_SINGLE_STEP | LBM_EM_FLAG_TWO_STEP))))
        return set_error(LBM_EM_EINVAL, "LBM_EM_FLAG_THREE_STEP is for LBM_EM_F32 alone, without the other step flags");
    if ((g->flags & LBM_EM_FLAG_TE) && g->precision == LBM_EM_F16DEV)
        return set_error(LBM_EM_EINVAL, "TE^z is available in LBM_EM_F64 and LBM_EM_F32");
    if ((g->flags & LBM_EM_FLAG_SINGLE_STEP) && (g->flags & LBM_EM_FLAG_TWO_STEP))
        return set_error(LBM_EM_EINVAL, "LBM_EM_FLAG_SINGLE_STEP and LBM_EM_FLAG_TWO_STEP exclude each other");
    if ((long long)g->nx * g->ny > (1LL << 31)) return set_error(LBM_EM_EINVAL, "lattice too large (> 2^31 sites)");
    if (g->precision != LBM_EM_F64 && g->precision != LBM_EM_F32 && g->precision != LBM_EM_F16DEV &&
        g->precision != LBM_EM_F32X2)
        return set_error(LBM_EM_EINVAL, "precision must be LBM_EM_F64, LBM_EM_F32, LBM_EM_F16DEV or LBM_EM_F32X2");
    lbm_em_status st = check_source(s);
    if (st) return st;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return set_error(LBM_EM_ECUDA, "no CUDA device available (the solver has no CPU path)");
    }
    lbm_em *h = new lbm_em();
    cudaGetDevice(&h->dev);
    h->nx = g->nx;
    h->ny = g->ny;
    h->prec = g->precision;
    h->pol = (g->flags & LBM_EM_FLAG_TE) ? POL_TE : POL_TM;
    h->elem = (g->precision == LBM_EM_F64 || g->precision == LBM_EM_F32X2) ? 8 : sizeof(float);
    h->pitch = round_up(g->nx, 32);
    h->pstride = (size_t)h->pitch * (size_t)g->ny;
    h->srccfg = *s;
    // two steps per launch: forced by the flag, else the default of the FP32 and FP16-deviation
    // forms, whose TMA-staged kernels beat one step per launch on GB300 at every size measured
    // (FP32 from 512^2 to 8192^2: 69 / 122 / 129 / 141 / 138 against 58 / 85 / 74 / 76 / 75
    // GLUPS; FP16-deviation at 512^2 / 2048^2 / 8192^2: 57.6 / 109 / 115.6 against 50.3 / 84.7 /
    // 89.0); the double-float form defaults to one step (its two-step kernel, 93 KB of shared
    // memory per CTA, loses)
    if (g->flags & LBM_EM_FLAG_TWO_STEP)
        h->tb = g->precision != LBM_EM_F64;
    else
        h->tb = (g->precision == LBM_EM_F32 || g->precision == LBM_EM_F16DEV) && !(g->flags & LBM_EM_FLAG_SINGLE_STEP);
    // three steps per launch (28 x 12 tiles): forced by the flag only; the four-step kernel
    // replaced it as the default on large lattices
    h->t3 = (g->flags & LBM_EM_FLAG_THREE_STEP) != 0;
    // four steps per launch (row-streaming kernel): forced by the flag, else the default of FP32
    // and FP16-deviation from 2^20 sites on (measured on GB300, GLUPS four / two steps per
    // launch, FP32: 8192^2 267.9 / 136.8, 4096^2 241.5 / 138.0, 2048^2 193.1 / 122.4, 1448^2
    // 184.4 / 114.3, 1024^2 135.0 / 117.4, 768^2 76.7 / 100.8, 512^2 34.6 / 70.4; FP16-deviation:
    // 8192^2 277.7 / 116.8, 2048^2 197.7 / 106.9, 1448^2 171.3 / 100.2, 1024^2 127.8 / 99.2,
    // 768^2 67.7 / 86.5, 512^2 31.0 / 59.2; three steps per launch never led: 8192^2 143.9,
    // 1024^2 111.1: on small lattices the strips cannot fill the GPU and the two-step kernel's
    // state stays in L2)
    h->s4 = (g->flags & LBM_EM_FLAG_FOUR_STEP) != 0 ||
            (!step_flags && (g->precision == LBM_EM_F32 || g->precision == LBM_EM_F16DEV) &&
             (long long)g->nx * g->ny >= (1LL << 20));
    if (h->s4) {
        h->t3 = false;
        h->tb = true;
    }
    for (int i = 0; i < 256; ++i) {
        h->eps_table[i] = 1.0;
        h->pec_id[i] = false;
    }
#define TRY(call, what)                       \
    do {                                      \
        st = cuda_status((call), what);       \
        if (st) {                             \
            free_handle(h);                   \
            return st;                        \
        }                                     \
    } while (0)
    if (g->stream) {
        h->stream = (cudaStream_t)g->stream;
    } else {
        TRY(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking), "cudaStreamCreate");
        h->own_stream = true;
    }
    TRY(cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking), "cudaStreamCreate");
    if (h->tb) TRY(step2_prepare(), "configuring the two-step kernels");
    prepare_pool(h->dev);
    h->buf_bytes = g->precision == LBM_EM_F16DEV ? f16_buffer_bytes(h->pstride)
                                                  : (size_t)NPLANES * h->pstride * h->elem;
    const size_t bytes = h->buf_bytes;
    for (int b = 0; b < 2; ++b) {
        TRY(dev_alloc(h, &h->buf[b], bytes), "allocating the distributions");
        TRY(cudaMemsetAsync(h->buf[b], 0, bytes, h->stream), "cudaMemset");
    }
    TRY(dev_alloc(h, &h->d_mat, h->pstride), "allocating the material ids");
    TRY(cudaMemsetAsync(h->d_mat, 0, h->pstride, h->stream), "cudaMemset");
    if (h->tb && h->prec == LBM_EM_F32) {
        TRY(step2_tma_prepare(&h->tma_ctas), "configuring the TMA-staged two-step kernel");
        for (int b = 0; b < 2; ++b)
            TRY(encode_plane_map(&h->tmap[b], (const float *)h->buf[b], h->nx, h->ny, h->pitch, h->pstride,
                                 kTmaTileW, kTmaTileH),
                "encoding the tensor map of a state buffer");
        TRY(encode_id_map(&h->idmap, h->d_mat, h->nx, h->ny, h->pitch, kTmaTileW, kTmaTileH),
            "encoding the tensor map of the ids");
    }
    if (h->t3) {
        TRY(step3_tma_prepare(&h->tma3_ctas), "configuring the three-step kernel");
        for (int b = 0; b < 2; ++b)
            TRY(encode_step3_maps(&h->tmap3[b], (const float *)h->buf[b], b == 0 ? &h->idmap3 : nullptr, h->d_mat,
                                  h->nx, h->ny, h->pitch, h->pstride),
                "encoding the tensor maps of the three-step kernel");
    }
    if (h->s4) {
        int warps = 0, warps_acc = 0;
        TRY(stream_prepare(h->prec == LBM_EM_F16DEV, &warps, &warps_acc), "configuring the four-step kernel");
        h->s4_plan = stream_plan(h->nx, h->ny, warps, h->prec == LBM_EM_F16DEV);
        h->s4_plan_acc = stream_plan(h->nx, h->ny, warps_acc, h->prec == LBM_EM_F16DEV);
        for (int b = 0; b < 2; ++b)
            TRY(encode_stream_maps(&h->s4_smap[b], &h->s4_fmap[b], b == 0 ? &h->s4_imap : nullptr, h->buf[b],
                                   h->prec == LBM_EM_F16DEV, h->d_mat, h->nx, h->ny, h->pitch, h->pstride),
                "encoding the tensor maps of the four-step kernel");
    }
    if (h->tb && h->prec == LBM_EM_F16DEV) {
        TRY(step2_f16_tma_prepare(&h->tma_ctas), "configuring the TMA-staged two-step kernel");
        for (int b = 0; b < 2; ++b)
            TRY(encode_f16_maps(&h->f16_gmap[b], &h->f16_fmap[b], h->buf[b], h->nx, h->ny, h->pitch, h->pstride),
                "encoding the tensor maps of a state buffer");
        TRY(encode_id_map(&h->idmap, h->d_mat, h->nx, h->ny, h->pitch, kTmaTileW, kTmaTileH),
            "encoding the tensor map of the ids");
    }
    TRY(dev_alloc(h, &h->d_mtab, 256 * sizeof(MatT<double>)), "allocating the material table");
    TRY(dev_alloc(h, &h->d_time, 2 * sizeof(long long)), "allocating the time words");
    TRY(cudaMemsetAsync(h->d_time, 0, 2 * sizeof(long long), h->stream), "cudaMemset");
    TRY(dev_alloc(h, &h->d_err, sizeof(unsigned)), "allocating the error word");
    TRY(cudaMemsetAsync(h->d_err, 0, sizeof(unsigned), h->stream), "cudaMemset");
    TRY(dev_alloc(h, &h->d_out, 4 * sizeof(double)), "allocating the results");
    TRY(pinned_get(256 * sizeof(MatT<double>), &h->h_stage, &h->stage_cap), "cudaMallocHost(table staging)");
    TRY(cudaEventCreateWithFlags(&h->stage_ev, cudaEventDisableTiming), "cudaEventCreate");
    TRY(cudaEventRecord(h->stage_ev, h->stream), "cudaEventRecord");
    TRY(cudaEventCreateWithFlags(&h->up_ev, cudaEventDisableTiming), "cudaEventCreate");
    TRY(cudaEventRecord(h->up_ev, h->stream), "cudaEventRecord");
    std::vector<double2> cs = phase_table(s->period_steps);
    TRY(dev_alloc(h, &h->d_cs, cs.size() * sizeof(double2)), "allocating the phase table");
    void *up = nullptr;
    TRY(upload_staging(h, cs.size() * sizeof(double2), &up), "pinned staging");
    std::memcpy(up, cs.data(), cs.size() * sizeof(double2));
    TRY(copy_async(h->d_cs, up, cs.size() * sizeof(double2), cudaMemcpyHostToDevice, h->stream),
        "cudaMemcpy(phase table)");
    TRY(cudaEventRecord(h->up_ev, h->stream), "cudaEventRecord");
    h->src.kind = s->kind;
    h->src.period = s->period_steps;
    h->src.ramp = s->ramp_steps;
    incident_constants(s->period_steps, s->E0, &h->src.pr, &h->src.pi, &h->src.qr, &h->src.qi);
    h->src.cs = h->d_cs;
#undef TRY
    *out = h;
    return LBM_EM_OK;
}

// Material table -> device without blocking the host on the stream: the table goes
// through a pinned staging buffer that is reused once its previous copy has finished.
static lbm_em_status upload_table(lbm_em *h) {
    cudaError_t e = cudaEventSynchronize(h->stage_ev);
    size_t bytes;
    if (h->prec == LBM_EM_F64) {
        auto tab = material_table<double>(h->eps_table, h->pec_id);
        bytes = tab.size() * sizeof(tab[0]);
        std::memcpy(h->h_stage, tab.data(), bytes);
    } else if (h->prec == LBM_EM_F32X2) {
        auto tab = material_table<df>(h->eps_table, h->pec_id);
        bytes = tab.size() * sizeof(tab[0]);
        std::memcpy(h->h_stage, tab.data(), bytes);
    } else {
        auto tab = material_table<float>(h->eps_table, h->pec_id);
        bytes = tab.size() * sizeof(tab[0]);
        std::memcpy(h->h_stage, tab.data(), bytes);
    }
    if (e == cudaSuccess) e = copy_async(h->d_mtab, h->h_stage, bytes, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaEventRecord(h->stage_ev, h->stream);
    return cuda_status(e, "uploading the material table");
}

extern "C" {

const char *lbm_em_last_error(void) { return g_last_error.c_str(); }

lbm_em_status lbm_em_create(const lbm_em_grid *g, const double *eps_map, const uint8_t *pec_mask,
                            const lbm_em_source *s, lbm_em_t **out) {
    if (!eps_map) return set_error(LBM_EM_EINVAL, "eps_map is NULL");
    if (!g || !out) return set_error(LBM_EM_EINVAL, "grid/out is NULL");
    if (g->nx < 4 || g->ny < 4) return set_error(LBM_EM_EINVAL, "nx and ny must be >= 4");
    const size_t n = (size_t)g->nx * (size_t)g->ny;
    // material ids: distinct permittivities in order of first appearance, one id for PEC
    std::map<double, int> ids;
    std::vector<uint8_t> idv(n);
    double eps_tab[256];
    bool pec_tab[256];
    for (int i = 0; i < 256; ++i) {
        eps_tab[i] = 1.0;
        pec_tab[i] = false;
    }
    int pec_slot = -1, next = 0;
    for (size_t i = 0; i < n; ++i) {
        if (pec_mask && pec_mask[i]) {
            if (pec_slot < 0) {
                if (next >= 256) return set_error(LBM_EM_EINVAL, "more than 256 materials");
                pec_slot = next++;
                pec_tab[pec_slot] = true;
                eps_tab[pec_slot] = 0.0;
            }
            idv[i] = (uint8_t)pec_slot;
            continue;
        }
        const double e = eps_map[i];
        if (!(e >= 1.0) || !std::isfinite(e)) return set_error(LBM_EM_EINVAL, "eps_map values must be finite and >= 1");
        auto it = ids.find(e);
        if (it == ids.end()) {
            if (next >= 256) return set_error(LBM_EM_EINVAL, "more than 256 distinct materials");
            eps_tab[next] = e;
            it = ids.emplace(e, next++).first;
        }
        idv[i] = (uint8_t)it->second;
    }
    lbm_em *h = nullptr;
    lbm_em_status st = create_common(g, s, &h);
    if (st) return st;
    std::memcpy(h->eps_table, eps_tab, sizeof(eps_tab));
    std::memcpy(h->pec_id, pec_tab, sizeof(pec_tab));
    void *up = nullptr;
    st = cuda_status(upload_staging(h, n, &up), "pinned staging");
    if (!st) {
        std::memcpy(up, idv.data(), n);
        st = cuda_status(copy2d_async(h->d_mat, h->pitch, up, h->nx, h->nx, h->ny, cudaMemcpyHostToDevice,
                                           h->stream),
                         "uploading material ids");
    }
    if (!st) st = cuda_status(cudaEventRecord(h->up_ev, h->stream), "cudaEventRecord");
    if (!st) st = upload_table(h);
    if (st) {
        free_handle(h);
        return st;
    }
    *out = h;
    return LBM_EM_OK;
}

lbm_em_status lbm_em_create_janus(const lbm_em_grid *g, const lbm_em_janus *j, const lbm_em_source *s,
                                  lbm_em_t **out) {
    lbm_em_status st = check_janus(j);
    if (st) return st;
    lbm_em *h = nullptr;
    st = create_common(g, s, &h);
    if (st) return st;
    double cx, cy;
    janus_center(j, h->nx, h->ny, &cx, &cy);
    h->eps_table[0] = 1.0;
    h->eps_table[1] = j->eps1;
    h->eps_table[2] = j->pec2 ? 0.0 : j->eps2;
    h->pec_id[2] = j->pec2 != 0;
    st = cuda_status(launch_rasterize(h->nx, h->ny, h->pitch, cx, cy, j->a, -std::sin(j->phi0), -std::cos(j->phi0),
                                      h->d_mat, h->stream),
                     "rasterising the Janus disc");
    if (!st) st = upload_table(h);
    if (st) {
        free_handle(h);
        return st;
    }
    *out = h;
    return LBM_EM_OK;
}

lbm_em_status lbm_em_reset(lbm_em_t *h) {
    if (!h) return set_error(LBM_EM_EINVAL, "handle is NULL");
    cudaSetDevice(h->dev);
    lbm_em_status st = cuda_status(cudaMemsetAsync(h->buf[0], 0, h->buf_bytes, h->stream), "clearing distributions");
    if (!st) st = cuda_status(cudaMemsetAsync(h->d_time, 0, 2 * sizeof(long long), h->stream), "clearing time");
    if (!st) st = cuda_status(cudaMemsetAsync(h->d_err, 0, sizeof(unsigned), h->stream), "clearing error flag");
    if (!st && h->has_contour)
        st = cuda_status(cudaMemsetAsync(h->d_acc, 0, (size_t)h->ch.n_slots * 6 * sizeof(double), h->stream),
                         "clearing accumulators");
    if (st) return st;
    h->t = 0;
    h->cur = 0;
    h->n_acc = 0;
    return LBM_EM_OK;
}

lbm_em_status lbm_em_set_janus(lbm_em_t *h, const lbm_em_janus *j) {
    if (!h) return set_error(LBM_EM_EINVAL, "handle is NULL");
    lbm_em_status st = check_janus(j);
    if (st) return st;
    cudaSetDevice(h->dev);
    double cx, cy;
    janus_center(j, h->nx, h->ny, &cx, &cy);
    for (int i = 0; i < 256; ++i) {
        h->eps_table[i] = 1.0;
        h->pec_id[i] = false;
    }
    h->eps_table[1] = j->eps1;
    h->eps_table[2] = j->pec2 ? 0.0 : j->eps2;
    h->pec_id[2] = j->pec2 != 0;
    st = cuda_status(launch_rasterize(h->nx, h->ny, h->pitch, cx, cy, j->a, -std::sin(j->phi0), -std::cos(j->phi0),
                                      h->d_mat, h->stream),
                     "rasterising the Janus disc");
    if (!st) st = upload_table(h);
    return st;
}

lbm_em_status lbm_em_destroy(lbm_em_t *h) {
    free_handle(h);
    return LBM_EM_OK;
}

static lbm_em_status refuse_after_timeout(const lbm_em *h) {
    return h->timed_out ? set_error(LBM_EM_ESTATE, "a tile copy timed out on this handle: destroy it and create a new one")
                        : LBM_EM_OK;
}

lbm_em_status lbm_em_step(lbm_em_t *h, int64_t n) {
    if (!h) return set_error(LBM_EM_EINVAL, "handle is NULL");
    if (n < 0) return set_error(LBM_EM_EINVAL, "n must be >= 0");
    if (lbm_em_status st = refuse_after_timeout(h)) return st;
    cudaSetDevice(h->dev);
    return run_steps(h, n, false);
}

lbm_em_status lbm_em_sync(lbm_em_t *h) {
    if (!h) return set_error(LBM_EM_EINVAL, "handle is NULL");
    cudaSetDevice(h->dev);
    unsigned err = 0;
    lbm_em_status st = cuda_status(copy_async(&err, h->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream),
                                   "reading the error flag");
    if (!st) st = cuda_status(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    if (st) return st;
    if (err & kErrTimeout) {
        h->timed_out = true;
        return set_error(LBM_EM_ETIMEOUT, "a bounded wait for a tile load gave up");
    }
    if (err) return set_error(LBM_EM_EUNSTABLE, "a field became non-finite or exceeded 3 * 2^20 times the source amplitude");
    return LBM_EM_OK;
}

lbm_em_status lbm_em_get_steps_per_launch(lbm_em_t *h, int32_t *n) {
    if (!h || !n) return set_error(LBM_EM_EINVAL, "NULL argument");
    *n = launch_steps(h, false);
    return LBM_EM_OK;
}

lbm_em_status lbm_em_get_time(lbm_em_t *h, int64_t *t) {
    if (!h || !t) return set_error(LBM_EM_EINVAL, "NULL argument");
    *t = h->t;
    return LBM_EM_OK;
}

lbm_em_status lbm_em_set_contour(lbm_em_t *h, const lbm_em_contour *c) {
    if (!h) return set_error(LBM_EM_EINVAL, "handle is NULL");
    cudaSetDevice(h->dev);
    if (h->has_contour && c && std::memcmp(c, &h->contour, sizeof(*c)) == 0) {
        lbm_em_status st = cuda_status(
            cudaMemsetAsync(h->d_acc, 0, (size_t)h->ch.n_slots * 6 * sizeof(double), h->stream), "clearing acc");
        if (!st) h->n_acc = 0;
        return st;
    }
    ContourHost ch;
    ch.E0 = h->srccfg.E0;
    lbm_em_status st = build_contour(h->nx, h->ny, c, &ch);
    if (st) return st;
    // everything below is ordered on the handle's stream: the old buffers are released
    // after the steps already queued, and the host does not wait for them
    free_contour(h);
    h->contour = *c;
    h->ch = ch;
    // slot map: -1 everywhere, the stencil slots only in rows y0..y1 (the kernels read the
    // map in those rows only), uploaded as one band
    const int y0 = std::max(ch.y0, 0), y1 = std::min(ch.y1, h->ny - 1);
    const size_t band = y1 >= y0 ? (size_t)(y1 - y0 + 1) * h->pitch : 0;
    std::vector<double2> inc(ch.n_slots, make_double2(0.0, 0.0));
    if (h->srccfg.kind != LBM_EM_SRC_NONE) {
        // incident phasor i E0 e^{i k x} of the lattice's plane wave at each stencil site
        // (far field: E_z^I for TM, H_z^I for TE)
        const double k = lattice_wavenumber(h->srccfg.period_steps);
        for (int s = 0; s < ch.n_slots; ++s) {
            const double kx = k * (double)ch.site_xy[2 * s];
            inc[s] = make_double2(-h->srccfg.E0 * std::sin(kx), h->srccfg.E0 * std::cos(kx));
        }
    }
    const size_t b_slot = band * sizeof(int), b_pts = ch.pts.size() * sizeof(ContourPt),
                 b_inc = inc.size() * sizeof(double2);
    const size_t o_pts = (b_slot + 255) / 256 * 256, o_inc = o_pts + (b_pts + 255) / 256 * 256;
    st = cuda_status(dev_alloc(h, &h->d_slot, h->pstride * sizeof(int)), "allocating the slot map");
    if (!st) st = cuda_status(dev_alloc(h, &h->d_acc, (size_t)ch.n_slots * 6 * sizeof(double)), "allocating acc");
    if (!st) st = cuda_status(dev_alloc(h, &h->d_pts, b_pts), "allocating the contour");
    if (!st) st = cuda_status(dev_alloc(h, &h->d_inc, b_inc), "allocating the incident table");
    if (!st && h->s4 && ch.n_slots > 0)
        st = cuda_status(dev_alloc(h, &h->d_stage, (size_t)ch.n_slots * 12 * sizeof(float)),
                         "allocating the accumulation stage");
    char *up = nullptr;
    if (!st) st = cuda_status(upload_staging(h, o_inc + b_inc, (void **)&up), "pinned staging");
    if (!st) {
        int *sl = (int *)up;
        std::fill(sl, sl + band, -1);
        for (int s = 0; s < ch.n_slots; ++s)
            sl[(size_t)(ch.site_xy[2 * s + 1] - y0) * h->pitch + ch.site_xy[2 * s]] = s;
        std::memcpy(up + o_pts, ch.pts.data(), b_pts);
        std::memcpy(up + o_inc, inc.data(), b_inc);
        st = cuda_status(cudaMemsetAsync(h->d_slot, 0xff, h->pstride * sizeof(int), h->stream), "clearing slots");
    }
    if (!st && band)
        st = cuda_status(copy_async(h->d_slot + (size_t)y0 * h->pitch, up, b_slot, cudaMemcpyHostToDevice,
                                         h->stream),
                         "uploading slots");
    if (!st)
        st = cuda_status(copy_async(h->d_pts, up + o_pts, b_pts, cudaMemcpyHostToDevice, h->stream),
                         "uploading contour");
    if (!st)
        st = cuda_status(copy_async(h->d_inc, up + o_inc, b_inc, cudaMemcpyHostToDevice, h->stream),
                         "uploading incident");
    if (!st) st = cuda_status(cudaEventRecord(h->up_ev, h->stream), "cudaEventRecord");
    if (!st)
        st = cuda_status(cudaMemsetAsync(h->d_acc, 0, (size_t)ch.n_slots * 6 * sizeof(double), h->stream),
                         "clearing acc");
    if (st) {
        free_contour(h);
        return st;
    }
    h->n_acc = 0;
    h->has_contour = true;
    return LBM_EM_OK;
}

lbm_em_status lbm_em_accumulate(lbm_em_t *h, int64_t n) {
    if (!h) return set_error(LBM_EM_EINVAL, "handle is NULL");
    if (!h->has_contour) return set_error(LBM_EM_ESTATE, "no contour set");
    if (lbm_em_status st = refuse_after_timeout(h)) return st;
    if (n < 0) return set_error(LBM_EM_EINVAL, "n must be >= 0");
    cudaSetDevice(h->dev);
    lbm_em_status st = run_steps(h, n, true);
    if (!st) h->n_acc += n;
    return st;
}

lbm_em_status lbm_em_contour_integral(lbm_em_t *h, double out[3]) {
    if (!h || !out) return set_error(LBM_EM_EINVAL, "NULL argument");
    if (!h->has_contour || h->n_acc <= 0) return set_error(LBM_EM_ESTATE, "no accumulated steps");
    cudaSetDevice(h->dev);
    lbm_em_status st = cuda_status(launch_contour(h->d_acc, 2.0 / (double)h->n_acc, h->d_pts, (int)h->ch.pts.size(),
                                                  h->ch.R, h->ch.dl, h->ch.F0, h->ch.M0, h->d_out, h->stream),
                                   "contour kernel");
    double res[3];
    if (!st)
        st = cuda_status(copy_async(res, h->d_out, 3 * sizeof(double), cudaMemcpyDeviceToHost, h->stream),
                         "reading forces");
    if (!st) st = lbm_em_sync(h);
    if (st) return st;
    out[0] = res[0];
    out[1] = res[1];
    out[2] = res[2];
    return LBM_EM_OK;
}

lbm_em_status lbm_em_contour_integral_device(lbm_em_t *h, double *d_out) {
    if (!h || !d_out) return set_error(LBM_EM_EINVAL, "NULL argument");
    if (!h->has_contour || h->n_acc <= 0) return set_error(LBM_EM_ESTATE, "no accumulated steps");
    cudaSetDevice(h->dev);
    return cuda_status(launch_contour(h->d_acc, 2.0 / (double)h->n_acc, h->d_pts, (int)h->ch.pts.size(), h->ch.R,
                                      h->ch.dl, h->ch.F0, h->ch.M0, d_out, h->stream),
                       "contour kernel");
}

lbm_em_status lbm_em_force_torque_device(lbm_em_t *h, const lbm_em_contour *c, double *d_out) {
    lbm_em_status st = lbm_em_set_contour(h, c);
    if (!st) st = lbm_em_accumulate(h, h->srccfg.period_steps);
    if (!st) st = lbm_em_contour_integral_device(h, d_out);
    return st;
}

lbm_em_status lbm_em_force_torque(lbm_em_t *h, const lbm_em_contour *c, double out[3]) {
    lbm_em_status st = lbm_em_set_contour(h, c);
    if (!st) st = lbm_em_accumulate(h, h->srccfg.period_steps);
    if (!st) st = lbm_em_contour_integral(h, out);
    return st;
}

lbm_em_status lbm_em_far_field(lbm_em_t *h, const double *angles, int32_t n_angles, double *s2) {
    if (!h || !angles || !s2 || n_angles < 1) return set_error(LBM_EM_EINVAL, "bad far-field arguments");
    if (!h->has_contour || h->n_acc <= 0) return set_error(LBM_EM_ESTATE, "no accumulated steps");
    cudaSetDevice(h->dev);
    double *d = nullptr;
    lbm_em_status st = cuda_status(dev_alloc(h, &d, (size_t)n_angles * 4 * sizeof(double)), "allocating the far field");
    if (st) return st;
    double *d_ang = d + 3 * (size_t)n_angles;
    std::vector<double> res(3 * (size_t)n_angles);
    st = cuda_status(copy_async(d_ang, angles, n_angles * sizeof(double), cudaMemcpyHostToDevice, h->stream),
                     "uploading angles");
    if (!st)
        st = cuda_status(launch_farfield(h->d_acc, 2.0 / (double)h->n_acc, h->d_pts, (int)h->ch.pts.size(), h->d_inc,
                                         h->ch.R, h->ch.dl, lattice_wavenumber(h->srccfg.period_steps), h->srccfg.E0,
                                         h->pol, d_ang, n_angles, d, h->stream),
                         "far-field kernel");
    if (!st)
        st = cuda_status(copy_async(res.data(), d, res.size() * sizeof(double), cudaMemcpyDeviceToHost, h->stream),
                         "reading far field");
    if (!st) st = cuda_status(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    dev_free(h, d);
    if (st) return st;
    for (int j = 0; j < n_angles; ++j) s2[j] = res[3 * (size_t)j];
    return LBM_EM_OK;
}

lbm_em_status lbm_em_energy(lbm_em_t *h, double *W) {
    if (!h || !W) return set_error(LBM_EM_EINVAL, "NULL argument");
    cudaSetDevice(h->dev);
    const int p = h->cur;
    double *d = h->d_out + 3;  // the fourth word of the result buffer
    lbm_em_status st = cuda_status(cudaMemsetAsync(d, 0, sizeof(double), h->stream), "clearing energy");
    cudaError_t e = cudaSuccess;
    if (!st) {
        if (h->prec == LBM_EM_F16DEV)
            e = launch_energy_f16(make_f16_args(h, p), h->d_time + p, d, h->stream);
        else if (h->prec == LBM_EM_F64)
            e = launch_energy<double>(make_args<double>(h), (const double *)h->buf[p], h->d_time + p, d, h->stream);
        else if (h->prec == LBM_EM_F32X2)
            e = launch_energy<df>(make_args<df>(h), (const df *)h->buf[p], h->d_time + p, d, h->stream);
        else
            e = launch_energy<float>(make_args<float>(h), (const float *)h->buf[p], h->d_time + p, d, h->stream);
        st = cuda_status(e, "energy kernel");
    }
    double w = 0.0;
    if (!st) st = cuda_status(copy_async(&w, d, sizeof(double), cudaMemcpyDeviceToHost, h->stream), "reading energy");
    if (!st) st = lbm_em_sync(h);
    if (!st) *W = w;
    return st;
}

lbm_em_status lbm_em_run_converged(lbm_em_t *h, const lbm_em_contour *c, double tol, int32_t min_periods,
                                   int32_t max_periods, double out[3], int64_t *steps_run) {
    if (!h || !c || !out) return set_error(LBM_EM_EINVAL, "NULL argument");
    if (!(tol >= 0.0) || min_periods < 1 || max_periods < min_periods)
        return set_error(LBM_EM_EINVAL, "need tol >= 0 and 1 <= min_periods <= max_periods");
    const int T = h->srccfg.period_steps;
    const int64_t t0 = h->t;
    double prev = -1.0;
    int p = 0, settled = 0;
    bool converged = false;
    lbm_em_status st = LBM_EM_OK;
    while (p < max_periods - 1) {
        st = lbm_em_step(h, T);
        if (st) return st;
        ++p;
        double W = 0.0;
        st = lbm_em_energy(h, &W);
        if (st) return st;
        // settled when two successive samples (same phase of the period) change by <= tol
        settled = (prev > 0.0 && std::fabs(W - prev) <= tol * W) ? settled + 1 : 0;
        prev = W;
        if (p + 1 >= min_periods && settled >= 2) {
            converged = true;
            break;
        }
    }
    // the decision uses the fields of the boundary step itself, so the averaging period
    // starts one step later (the batched path runs the same schedule)
    if (converged) st = lbm_em_step(h, 1);
    if (!st) st = lbm_em_force_torque(h, c, out);
    if (!st && steps_run) *steps_run = h->t - t0;
    return st;
}

lbm_em_status lbm_em_get_fields(lbm_em_t *h, double *ez, double *hx, double *hy) {
    if (!h) return set_error(LBM_EM_EINVAL, "handle is NULL");
    cudaSetDevice(h->dev);
    const size_t n = (size_t)h->nx * h->ny;
    lbm_em_status st = LBM_EM_OK;
    if (!h->d_fields) st = cuda_status(dev_alloc(h, &h->d_fields, 3 * n * sizeof(double)), "allocating the fields");
    if (st) return st;
    const int p = h->cur;
    cudaError_t e;
    if (h->prec == LBM_EM_F16DEV)
        e = launch_fields_f16(make_f16_args(h, p), h->d_time + p, h->d_fields, h->d_fields + n,
                              h->d_fields + 2 * n, h->stream);
    else if (h->prec == LBM_EM_F64)
        e = launch_fields<double>(make_args<double>(h), (const double *)h->buf[p], h->d_time + p, h->d_fields,
                                  h->d_fields + n, h->d_fields + 2 * n, h->stream);
    else if (h->prec == LBM_EM_F32X2)
        e = launch_fields<df>(make_args<df>(h), (const df *)h->buf[p], h->d_time + p, h->d_fields,
                              h->d_fields + n, h->d_fields + 2 * n, h->stream);
    else
        e = launch_fields<float>(make_args<float>(h), (const float *)h->buf[p], h->d_time + p, h->d_fields,
                                 h->d_fields + n, h->d_fields + 2 * n, h->stream);
    st = cuda_status(e, "fields kernel");
    double *dst[3] = {ez, hx, hy};
    for (int k = 0; k < 3 && !st; ++k)
        if (dst[k])
            st = cuda_status(copy_async(dst[k], h->d_fields + k * n, n * sizeof(double), cudaMemcpyDeviceToHost,
                                             h->stream),
                             "reading fields");
    if (!st) st = cuda_status(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    return st;
}

lbm_em_status lbm_em_get_phasors(lbm_em_t *h, int32_t *site_xy, double *phasors, int32_t *n_sites) {
    if (!h || !n_sites) return set_error(LBM_EM_EINVAL, "NULL argument");
    if (!h->has_contour) return set_error(LBM_EM_ESTATE, "no contour set");
    *n_sites = h->ch.n_slots;
    if (site_xy) std::memcpy(site_xy, h->ch.site_xy.data(), h->ch.site_xy.size() * sizeof(int32_t));
    if (phasors) {
        if (h->n_acc <= 0) return set_error(LBM_EM_ESTATE, "no accumulated steps");
        cudaSetDevice(h->dev);
        lbm_em_status st = cuda_status(copy_async(phasors, h->d_acc, (size_t)h->ch.n_slots * 6 * sizeof(double),
                                                       cudaMemcpyDeviceToHost, h->stream),
                                       "reading accumulators");
        if (!st) st = cuda_status(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
        if (st) return st;
        const double sc = 2.0 / (double)h->n_acc;
        for (size_t i = 0; i < (size_t)h->ch.n_slots * 6; ++i) phasors[i] *= sc;
    }
    return LBM_EM_OK;
}

lbm_em_status lbm_em_get_material(lbm_em_t *h, uint8_t *ids, double *eps_table) {
    if (!h) return set_error(LBM_EM_EINVAL, "handle is NULL");
    cudaSetDevice(h->dev);
    if (eps_table)
        for (int i = 0; i < 256; ++i) eps_table[i] = h->pec_id[i] ? 0.0 : h->eps_table[i];
    if (ids) {
        lbm_em_status st = cuda_status(copy2d_async(ids, h->nx, h->d_mat, h->pitch, h->nx, h->ny,
                                                         cudaMemcpyDeviceToHost, h->stream),
                                       "reading material ids");
        if (!st) st = cuda_status(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
        return st;
    }
    return LBM_EM_OK;
}

struct StateHeader {
    uint64_t magic;
    int32_t prec, nx, ny, n_slots;
    int64_t t, n_acc;
};
static const uint64_t kMagic = 0x4c424d454d535431ULL;

lbm_em_status lbm_em_save_state(lbm_em_t *h, void *buf, size_t *bytes) {
    if (!h || !bytes) return set_error(LBM_EM_EINVAL, "NULL argument");
    const size_t dist = h->buf_bytes;
    const size_t accb = h->has_contour ? (size_t)h->ch.n_slots * 6 * sizeof(double) : 0;
    const size_t need = sizeof(StateHeader) + dist + accb;
    if (!buf) {
        *bytes = need;
        return LBM_EM_OK;
    }
    if (*bytes < need) return set_error(LBM_EM_EINVAL, "checkpoint buffer too small");
    cudaSetDevice(h->dev);
    StateHeader hd{kMagic, h->prec, h->nx, h->ny, h->has_contour ? h->ch.n_slots : -1, h->t, h->n_acc};
    std::memcpy(buf, &hd, sizeof(hd));
    char *p = (char *)buf + sizeof(hd);
    lbm_em_status st = cuda_status(
        copy_async(p, h->buf[h->cur], dist, cudaMemcpyDeviceToHost, h->stream), "saving distributions");
    if (!st && accb)
        st = cuda_status(copy_async(p + dist, h->d_acc, accb, cudaMemcpyDeviceToHost, h->stream), "saving acc");
    if (!st) st = cuda_status(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    if (!st) *bytes = need;
    return st;
}

lbm_em_status lbm_em_load_state(lbm_em_t *h, const void *buf, size_t bytes) {
    if (!h || !buf) return set_error(LBM_EM_EINVAL, "NULL argument");
    StateHeader hd;
    if (bytes < sizeof(hd)) return set_error(LBM_EM_EINVAL, "checkpoint too small");
    std::memcpy(&hd, buf, sizeof(hd));
    if (hd.magic != kMagic || hd.prec != h->prec || hd.nx != h->nx || hd.ny != h->ny)
        return set_error(LBM_EM_EINVAL, "checkpoint does not match this handle");
    const int want_slots = h->has_contour ? h->ch.n_slots : -1;
    if (hd.n_slots != want_slots) return set_error(LBM_EM_EINVAL, "checkpoint contour does not match");
    const size_t dist = h->buf_bytes;
    const size_t accb = h->has_contour ? (size_t)h->ch.n_slots * 6 * sizeof(double) : 0;
    if (bytes < sizeof(hd) + dist + accb) return set_error(LBM_EM_EINVAL, "checkpoint truncated");
    cudaSetDevice(h->dev);
    const char *p = (const char *)buf + sizeof(hd);
    long long tt = hd.t;
    // ordered on the handle's stream: a synchronous cudaMemcpy from pageable memory may
    // return before its DMA has reached the device, and the handle's non-blocking stream
    // would not wait for it
    lbm_em_status st = cuda_status(
        copy_async(h->buf[h->cur], p, dist, cudaMemcpyHostToDevice, h->stream), "loading distributions");
    if (!st && accb)
        st = cuda_status(copy_async(h->d_acc, p + dist, accb, cudaMemcpyHostToDevice, h->stream), "loading acc");
    if (!st)
        st = cuda_status(copy_async(h->d_time + h->cur, &tt, sizeof(tt), cudaMemcpyHostToDevice, h->stream),
                         "loading time");
    if (!st) st = cuda_status(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    if (st) return st;
    h->t = hd.t;
    h->n_acc = hd.n_acc;
    return LBM_EM_OK;
}

lbm_em_status lbm_em_rasterize_janus(const lbm_em_janus *j, int32_t nx, int32_t ny, uint8_t *regions) {
    lbm_em_status st = check_janus(j);
    if (st) return st;
    if (nx < 1 || ny < 1 || !regions) return set_error(LBM_EM_EINVAL, "bad size or NULL output");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return set_error(LBM_EM_ECUDA, "no CUDA device available (the solver has no CPU path)");
    }
    double cx, cy;
    janus_center(j, nx, ny, &cx, &cy);
    const int pitch = round_up(nx, 32);
    uint8_t *d = nullptr;
    cudaStream_t s = nullptr;
    st = cuda_status(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking), "cudaStreamCreate");
    if (!st) st = cuda_status(dmalloc(&d, (size_t)pitch * ny), "cudaMalloc");
    if (!st) st = cuda_status(launch_rasterize(nx, ny, pitch, cx, cy, j->a, -std::sin(j->phi0), -std::cos(j->phi0), d, s),
                              "rasterise kernel");
    if (!st)
        st = cuda_status(copy2d_async(regions, nx, d, pitch, nx, ny, cudaMemcpyDeviceToHost, s), "reading regions");
    if (!st) st = cuda_status(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    dfree(d);
    if (s) cudaStreamDestroy(s);
    return st;
}

}  // extern "C"
