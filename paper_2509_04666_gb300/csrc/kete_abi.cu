// kete_abi.cu -- the C ABI of libkete_gpu.so (declared in include/kete.h).
//
// Host orchestration only: argument checks, device scratch, launch order on
// the context stream, the few host reads the survey driver needs (exposure and
// batch counts, candidate and hit counts per chunk of batches).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "kete_adjoint.h"
#include "kete_fov.h"
#include "kete_impl.h"
#include "kete_order.h"

using namespace kete;

namespace {

enum Slot {
    S_CHAIN, S_STATUS, S_STOPS, S_STOPSTATES, S_ISSTART, S_EX, S_SCANTMP, S_FCEN, S_FAUX,
    S_EXPFIRST, S_XEPOCH, S_XOBS, S_XCEN, S_XCENF, S_XRAD, S_XCS, S_XBATCH, S_NEXT, S_BFIRST, S_BTREF,
    S_BO, S_BROBS, S_BTSPAN, S_BRMAX, S_BSUN, S_NBATCH, S_BANDS, S_CELLKEY, S_CELLCNT,
    S_CELLSTART, S_CELLCUR, S_CELLEXP, S_CAND, S_EXPCNT, S_EXPOFF, S_EXPCUR, S_CANDBODY,
    S_HITTMP, S_FRAMECNT, S_FRAMEOFF, S_FRAMECUR, S_HITGROUP, S_MAXRAD, S_NT_T0, S_NT_H,
    S_NT_R64, S_NT_R32, S_XSUN, S_XOBSREL, S_NEXTBODY, S_TUNE_ST, S_TUNE_EP, S_TUNE_OUT,
    S_ADJ_REC, S_ADJ_NREC, S_ADJ_NBAT, S_ADJ_BIDX, S_ADJ_YREF, S_ADJ_GJUMP, S_ADJ_STATUS,
    S_KSTOP, S_DEFER_LIST, S_DEFER_CNT, S_ORDER, S_ORDER_KEY, S_ORDER_HIST, S_ORDER_OFF,
    S_ORDER_SCAN, S_ORDER_N, S_ADJ_TEND, S_LEG_OUT,
    S_EXT_START, S_EXT_EX, S_EXT_TMP, S_EXT_FIRST, S_EXT_SUB, S_EXT_PARENT, S_EXT_CNT,
    S_EXT_OFF, S_EXT_CUR, S_EXT_GROUP, S_EXT_KEEP, S_EXT_KCNT, S_EXT_KOFF, S_ADJ_PHI, S_ADJ_RECX,
    S_PRE_KEEP, S_PRE_N, S_ADJ_RICH,
    S_NSLOTS
};

struct Scratch {
    void *p = nullptr;
    size_t bytes = 0;
};

}  // namespace

struct kete_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::string err;
    bool have_ephem = false;
    double *d_coef = nullptr;
    float *d_coef32 = nullptr;
    EphemDev E{};
    Scratch slot[S_NSLOTS];
    DevCounters *d_ctr = nullptr;
    DevCounters *h_ctr = nullptr;   // pinned
    kete_stats stats{};
    std::vector<cudaEvent_t> ev;    // pool: [0] start, [1] end, then pairs for propagation
    int n_sm = 152;
    int pending_prop_pairs = 0;
    int64_t extra_launches = 0;     // ordering and second-phase launches of this call
    // phase timers: pairs of events per phase (prep, candidates, exact, order)
    std::vector<cudaEvent_t> phase_ev[4];
    int phase_n[4] = {0, 0, 0, 0};
    PropVariant var[2] = {{PROP_WORK_STEALING, 128, 0, 0, 1},
                          {PROP_WORK_STEALING, 128, 0, 0, 1}};   // per precision
};

enum Phase { PH_PREP = 0, PH_CAND = 1, PH_EXACT = 2, PH_ORDER = 3 };

static void phase_mark(kete_ctx *ctx, int ph, bool begin)
{
    size_t idx = 2 * (size_t)ctx->phase_n[ph] + (begin ? 0 : 1);
    auto &v = ctx->phase_ev[ph];
    while (v.size() <= idx) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        v.push_back(e);
    }
    cudaEventRecord(v[idx], ctx->stream);
    if (!begin) ctx->phase_n[ph]++;
}

static int fail(kete_ctx *c, int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    return code;
}

#define CUDA_TRY(x)                                                                       \
    do {                                                                                  \
        cudaError_t _e = (x);                                                             \
        if (_e != cudaSuccess)                                                            \
            return fail(ctx, KETE_ERR_CUDA, "%s failed: %s", #x, cudaGetErrorString(_e)); \
    } while (0)

static cudaError_t ensure(kete_ctx *ctx, int s, size_t bytes, void **out)
{
    Scratch &b = ctx->slot[s];
    if (bytes == 0) bytes = 16;
    if (b.bytes < bytes) {
        if (b.p) {
            cudaError_t e = cudaStreamSynchronize(ctx->stream);
            if (e != cudaSuccess) return e;
            cudaFree(b.p);
            b.p = nullptr;
            b.bytes = 0;
        }
        size_t want = bytes + bytes / 4;
        cudaError_t e = cudaMalloc(&b.p, want);
        if (e != cudaSuccess) {
            cudaGetLastError();
            e = cudaMalloc(&b.p, bytes);
            if (e != cudaSuccess) return e;
            want = bytes;
        }
        b.bytes = want;
    }
    *out = b.p;
    return cudaSuccess;
}

template <typename T>
static int get(kete_ctx *ctx, int s, size_t count, T **out)
{
    void *p = nullptr;
    cudaError_t e = ensure(ctx, s, count * sizeof(T), &p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, KETE_ERR_NOMEM, "device allocation of %zu bytes failed: %s",
                    count * sizeof(T), cudaGetErrorString(e));
    }
    *out = (T *)p;
    return KETE_OK;
}

#define GET(slot, n, ptr)                                  \
    do {                                                   \
        int _r = get(ctx, slot, (size_t)(n), &(ptr));      \
        if (_r != KETE_OK) return _r;                      \
    } while (0)

static cudaEvent_t event_at(kete_ctx *ctx, size_t i)
{
    while (ctx->ev.size() <= i) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        ctx->ev.push_back(e);
    }
    return ctx->ev[i];
}

static void stats_begin(kete_ctx *ctx)
{
    std::memset(&ctx->stats, 0, sizeof(ctx->stats));
    ctx->pending_prop_pairs = 0;
    ctx->extra_launches = 0;
    for (int q = 0; q < 4; q++) ctx->phase_n[q] = 0;
    cudaMemsetAsync(ctx->d_ctr, 0, sizeof(DevCounters), ctx->stream);
    cudaEventRecord(event_at(ctx, 0), ctx->stream);
}

static void prop_event(kete_ctx *ctx, bool begin)
{
    size_t idx = 2 + 2 * (size_t)ctx->pending_prop_pairs + (begin ? 0 : 1);
    cudaEventRecord(event_at(ctx, idx), ctx->stream);
    if (!begin) ctx->pending_prop_pairs++;
}

static int stats_end(kete_ctx *ctx)
{
    cudaEventRecord(event_at(ctx, 1), ctx->stream);
    CUDA_TRY(cudaMemcpyAsync(ctx->h_ctr, ctx->d_ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost,
                             ctx->stream));
    return KETE_OK;
}

static void stats_collect(kete_ctx *ctx)
{
    cudaStreamSynchronize(ctx->stream);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, ctx->ev[0], ctx->ev[1]);
    ctx->stats.total_ms = ms;
    double p = 0.0;
    for (int k = 0; k < ctx->pending_prop_pairs; k++) {
        float m = 0.0f;
        cudaEventElapsedTime(&m, ctx->ev[2 + 2 * k], ctx->ev[3 + 2 * k]);
        p += m;
    }
    ctx->stats.prop_ms = p;
    ctx->stats.fov_ms = ctx->stats.total_ms - p;
    ctx->stats.steps = (int64_t)ctx->h_ctr->steps;
    ctx->stats.rejected = (int64_t)ctx->h_ctr->rejected;
    ctx->stats.force_evals = (int64_t)ctx->h_ctr->force_evals;
    ctx->stats.iterations = (int64_t)ctx->h_ctr->iterations;
    ctx->stats.node_evals = (int64_t)ctx->h_ctr->node_evals;
    ctx->stats.deferred = (int64_t)ctx->h_ctr->deferred;
    ctx->stats.prop_launches = ctx->pending_prop_pairs;
    ctx->stats.launches += ctx->extra_launches;
    ctx->pending_prop_pairs = 0;
    double *dst[4] = {&ctx->stats.prep_ms, &ctx->stats.cand_ms, &ctx->stats.exact_ms,
                      &ctx->stats.order_ms};
    for (int q = 0; q < 4; q++) {
        double acc = 0.0;
        for (int k = 0; k < ctx->phase_n[q]; k++) {
            float m = 0.0f;
            cudaEventElapsedTime(&m, ctx->phase_ev[q][2 * k], ctx->phase_ev[q][2 * k + 1]);
            acc += m;
        }
        *dst[q] = acc;
        ctx->phase_n[q] = 0;
    }
}

extern "C" {

void kete_force_model_default(kete_force_model *fm)
{
    if (!fm) return;
    std::memset(fm, 0, sizeof(*fm));
    const double deg = 3.14159265358979323846 / 180.0;
    const double au = 149597870.7;
    fm->body_mask = 0x1FFu;
    fm->gr_mask = (1u << 0) | (1u << 3) | (1u << 5);   // Sun, Earth, Jupiter (App. A.2)
    fm->j2_mask = (1u << 0) | (1u << 5);               // Sun, Jupiter (App. A.3)
    fm->precision = KETE_FP64;
    fm->j2[0] = 2.1961e-7;
    fm->radius[0] = 696000.0 / au;
    fm->pole_ra[0] = 286.13 * deg;
    fm->pole_dec[0] = 63.87 * deg;
    fm->j2[5] = 0.014736;
    fm->radius[5] = 71492.0 / au;
    fm->pole_ra[5] = 268.056595 * deg;
    fm->pole_dec[5] = 64.495303 * deg;
    fm->eps = 1e-9;
    fm->eps_pc = 1e-10;
    fm->safety = 0.25;
    fm->dt_init = 4.0;
    fm->max_iter = 12;
    fm->max_steps = 100000;
}

void kete_survey_opts_default(kete_survey_opts *opt)
{
    if (!opt) return;
    opt->batch_span = 3.0;
    opt->twobody_max = 1.5;
    opt->cell_deg = 0.0;
    opt->mem_budget_gb = 0.0;
}

int kete_create(kete_ctx **out, int device, void *cuda_stream)
{
    if (!out) return KETE_ERR_BAD_ARG;
    *out = nullptr;
    kete_ctx *ctx = new kete_ctx();
    ctx->device = device;
    ctx->stream = (cudaStream_t)cuda_stream;
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_ctr, sizeof(DevCounters));
    if (e == cudaSuccess) e = cudaMallocHost(&ctx->h_ctr, sizeof(DevCounters));
    if (e != cudaSuccess) {
        delete ctx;
        return KETE_ERR_CUDA;
    }
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) == cudaSuccess && sms > 0)
        ctx->n_sm = sms;
    std::memset(ctx->h_ctr, 0, sizeof(DevCounters));
    upload_radau_tables(ctx->stream);
    e = upload_adjoint_tables(ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
        kete_destroy(ctx);
        return KETE_ERR_CUDA;
    }
    *out = ctx;
    return KETE_OK;
}

void kete_destroy(kete_ctx *ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    else cudaDeviceSynchronize();
    for (auto &s : ctx->slot)
        if (s.p) cudaFree(s.p);
    if (ctx->d_coef) cudaFree(ctx->d_coef);
    if (ctx->d_coef32) cudaFree(ctx->d_coef32);
    if (ctx->d_ctr) cudaFree(ctx->d_ctr);
    if (ctx->h_ctr) cudaFreeHost(ctx->h_ctr);
    for (auto e : ctx->ev) cudaEventDestroy(e);
    for (auto &v : ctx->phase_ev)
        for (auto e : v) cudaEventDestroy(e);
    delete ctx;
}

int kete_set_stream(kete_ctx *ctx, void *cuda_stream)
{
    if (!ctx) return KETE_ERR_BAD_ARG;
    ctx->stream = (cudaStream_t)cuda_stream;
    return KETE_OK;
}

const char *kete_last_error(const kete_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int kete_get_stats(const kete_ctx *ctx, kete_stats *out)
{
    if (!ctx || !out) return KETE_ERR_BAD_ARG;
    *out = ctx->stats;
    return KETE_OK;
}

int kete_load_ephem(kete_ctx *ctx, const void *buf, size_t nbytes)
{
    if (!ctx || !buf) return fail(ctx, KETE_ERR_BAD_ARG, "null context or buffer");
    const unsigned char *p = (const unsigned char *)buf;
    if (nbytes < 256 || std::memcmp(p, "KETECHB1", 8) != 0)
        return fail(ctx, KETE_ERR_BAD_ARG, "not a KETECHB1 table");
    int32_t hdr[4];
    double td[2];
    std::memcpy(hdr, p + 8, sizeof(hdr));
    std::memcpy(td, p + 24, sizeof(td));
    if (hdr[0] != 1) return fail(ctx, KETE_ERR_BAD_ARG, "unsupported table version %d", hdr[0]);
    int nb = hdr[1], nc = hdr[2], ns = hdr[3];
    if (nb < 1 || nb > KETE_MAX_BODIES || nc < 2 || nc > 64 || ns < 1)
        return fail(ctx, KETE_ERR_BAD_ARG, "bad table sizes (bodies %d, coef %d, seg %d)", nb, nc, ns);
    if (!(td[1] > 0.0) || !std::isfinite(td[0]))
        return fail(ctx, KETE_ERR_BAD_ARG, "bad table span");
    size_t ncoef = (size_t)nb * ns * 3 * nc;
    if (nbytes < 256 + ncoef * sizeof(double))
        return fail(ctx, KETE_ERR_BAD_ARG, "table truncated: %zu bytes, need %zu", nbytes,
                    256 + ncoef * sizeof(double));
    CUDA_TRY(cudaSetDevice(ctx->device));
    if (ctx->d_coef) {
        cudaStreamSynchronize(ctx->stream);
        cudaFree(ctx->d_coef);
        cudaFree(ctx->d_coef32);
        ctx->d_coef = nullptr;
        ctx->d_coef32 = nullptr;
    }
    ctx->have_ephem = false;
    std::vector<float> f32(ncoef);
    const double *src = (const double *)(p + 256);
    std::vector<double> f64(src, src + ncoef);
    for (size_t i = 0; i < ncoef; i++) f32[i] = (float)f64[i];
    CUDA_TRY(cudaMalloc(&ctx->d_coef, ncoef * sizeof(double)));
    CUDA_TRY(cudaMalloc(&ctx->d_coef32, ncoef * sizeof(float)));
    CUDA_TRY(cudaMemcpyAsync(ctx->d_coef, f64.data(), ncoef * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    CUDA_TRY(cudaMemcpyAsync(ctx->d_coef32, f32.data(), ncoef * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    EphemDev E{};
    E.coef = ctx->d_coef;
    E.coef32 = ctx->d_coef32;
    E.t_start = td[0];
    E.seg_len = td[1];
    E.inv_seg = 1.0 / td[1];
    E.t_end = td[0] + ns * td[1];
    E.n_seg = ns;
    E.n_coef = nc;
    E.n_bodies = nb;
    std::memcpy(E.gm, p + 48, sizeof(double) * KETE_MAX_BODIES);
    ctx->E = E;
    ctx->have_ephem = true;
    return KETE_OK;
}

}  // extern "C"

static int make_force(kete_ctx *ctx, const kete_force_model *fm_in, ForceDev &F)
{
    kete_force_model fm;
    if (fm_in) fm = *fm_in;
    else kete_force_model_default(&fm);
    if (!(fm.eps > 0) || !(fm.safety > 0 && fm.safety < 1) || fm.max_iter < 1 || fm.max_iter > 100 ||
        fm.max_steps < 1 || !(fm.dt_init > 0) || !(fm.eps_pc >= 0))
        return fail(ctx, KETE_ERR_BAD_ARG, "invalid force-model controls");
    if (fm.precision != KETE_FP64 && fm.precision != KETE_MIXED)
        return fail(ctx, KETE_ERR_BAD_ARG, "unknown precision mode %d", fm.precision);
    std::memset(&F, 0, sizeof(F));
    const double eps_obl = 84381.448 / 3600.0 * 3.14159265358979323846 / 180.0;
    const double ce = std::cos(eps_obl), se = std::sin(eps_obl);
    uint32_t act = 0;
    for (int m = 0; m < ctx->E.n_bodies; m++)
        if (((fm.body_mask >> m) & 1u) && ctx->E.gm[m] != 0.0) act |= 1u << m;
    F.active_mask = act;
    F.gr_mask = fm.gr_mask & act;
    F.j2_mask = fm.j2_mask & act;
    F.precision = fm.precision;
    for (int m = 0; m < KETE_MAX_BODIES; m++) {
        F.j2k[m] = 1.5 * fm.j2[m] * ctx->E.gm[m] * fm.radius[m] * fm.radius[m];
        double ra = fm.pole_ra[m], de = fm.pole_dec[m];
        double ex = std::cos(de) * std::cos(ra), ey = std::cos(de) * std::sin(ra), ez = std::sin(de);
        F.pole[m][0] = ex;
        F.pole[m][1] = ce * ey + se * ez;
        F.pole[m][2] = -se * ey + ce * ez;
    }
    for (int m = 0; m < KETE_MAX_BODIES; m++) {
        const double gm = ctx->E.gm[m];
        F.gm4[m] = 4.0 * gm;
        F.grk[m] = gm * kInvC2;
        F.gr4k[m] = 4.0 * F.grk[m];
        for (int c = 0; c < 3; c++) F.pole_m2[m][c] = -2.0 * F.pole[m][c];
        F.gm32[m] = (float)gm;
        F.j2k32[m] = (float)F.j2k[m];
        for (int c = 0; c < 3; c++) F.pole32[m][c] = (float)F.pole[m][c];
        F.gm4_32[m] = (float)F.gm4[m];
        F.grk32[m] = (float)F.grk[m];
        F.gr4k32[m] = (float)F.gr4k[m];
        for (int c = 0; c < 3; c++) F.pole_m2_32[m][c] = (float)F.pole_m2[m][c];
    }
    F.eps = fm.eps;
    F.eps_pc = fm.eps_pc;
    F.safety = fm.safety;
    F.dt_init = fm.dt_init;
    F.max_iter = fm.max_iter;
    F.max_steps = fm.max_steps;
    if (fm.nongrav && (reinterpret_cast<uintptr_t>(fm.nongrav) & 7u))
        return fail(ctx, KETE_ERR_BAD_ARG, "nongrav must be 8-byte aligned");
    F.nongrav = fm.nongrav;
    return KETE_OK;
}

extern "C" int kete_ephem_eval(kete_ctx *ctx, const double *t, int64_t n, int body, double *pos,
                               double *vel)
{
    if (!ctx) return KETE_ERR_BAD_ARG;
    if (!ctx->have_ephem) return fail(ctx, KETE_ERR_NO_EPHEM, "no ephemeris loaded");
    if (n < 0 || (n > 0 && (!t || !pos)) || body < 0 || body >= ctx->E.n_bodies)
        return fail(ctx, KETE_ERR_BAD_ARG, "bad arguments");
    CUDA_TRY(cudaSetDevice(ctx->device));
    CUDA_TRY(launch_ephem_eval(ctx->E, t, n, body, pos, vel, ctx->stream));
    return KETE_OK;
}

// Bodies (states [6][stride] SoA, epochs [n], device) most expensive first
// over [epoch, end]: end = the last stop (stops_dev, device) or t_end_i[i]
// (device) per body.  *order_n receives a device copy of n, the kernels'
// queue length.
static int cost_order(kete_ctx *ctx, const double *states, int64_t stride, const double *epochs,
                      int64_t n, const double *stops_dev, int n_stops, const double *t_end_i,
                      const kete_nongrav *ng, int32_t **order, unsigned long long **order_n)
{
    OrderScratch s;
    const size_t nh = order_hist_elems(n);
    GET(S_ORDER, n, *order);
    GET(S_ORDER_KEY, n, s.key);
    GET(S_ORDER_HIST, nh, s.hist);
    GET(S_ORDER_OFF, nh + 1, s.off);
    GET(S_ORDER_SCAN, scan_tmp_elems((int64_t)nh), s.scan_tmp);
    GET(S_ORDER_N, 1, *order_n);
    double t_end = 0.0;
    if (!t_end_i) {
        CUDA_TRY(cudaMemcpyAsync(&t_end, stops_dev + (n_stops - 1), sizeof(double),
                                 cudaMemcpyDeviceToHost, ctx->stream));
        CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    }
    const unsigned long long nn = (unsigned long long)n;
    CUDA_TRY(cudaMemcpyAsync(*order_n, &nn, sizeof(nn), cudaMemcpyHostToDevice, ctx->stream));
    CUDA_TRY(order_by_cost(ctx->E, states, stride, epochs, n, t_end, t_end_i, ng, s, *order,
                           ctx->stream));
    ctx->extra_launches += order_launches(n, ng);
    return KETE_OK;
}

// Launch the propagation kernel with the context's variant for F's precision.
// out_aos: stop k of body i at out[(k stride + i) * 6 + c] (see k_propagate)
static int propagate(kete_ctx *ctx, const ForceDev &F, ChainState cs, const double *stops_dev,
                     int n_stops, double *out, int64_t stride, bool keep_on_fail,
                     const NodeTable *nt, int leg0, bool out_aos = false)
{
    PropVariant var = ctx->var[F.precision == KETE_MIXED ? 1 : 0];
    unsigned long long *next = nullptr;
    if (var.kind == PROP_WORK_STEALING) GET(S_NEXTBODY, 1, next);
    PropDefer defer{}, *dp = nullptr;
    if (var.split > 1 && var.budget > 0) {
        unsigned long long *cnt;
        GET(S_DEFER_LIST, cs.n, defer.list);
        GET(S_DEFER_CNT, 2, cnt);
        defer.count = cnt;
        defer.next = cnt + 1;
        dp = &defer;
    }
    int32_t *order = nullptr;
    unsigned long long *order_n = nullptr;
    if (var.order) {
        int r = cost_order(ctx, cs.w, cs.n, cs.w + 6 * cs.n, cs.n, stops_dev, n_stops, nullptr,
                           F.nongrav, &order, &order_n);
        if (r != KETE_OK) return r;
    }
    ctx->stats.prop_kind = var.kind;
    ctx->stats.prop_block = var.block;
    ctx->stats.prop_split = var.split;
    ctx->stats.prop_budget = var.budget;
    ctx->stats.prop_order = var.order;
    CUDA_TRY(launch_propagate(ctx->E, F, cs, stops_dev, n_stops, out, stride, keep_on_fail,
                              ctx->d_ctr, ctx->stream, nt, leg0, var, next, dp, order, order_n,
                              out_aos));
    if (dp) ctx->extra_launches += 1;   // the second phase
    return KETE_OK;
}

// Planet states at the Gauss-Radau node epochs of every leg of a chain of stops.
static int node_table(kete_ctx *ctx, const double *stops_dev, int n_stops, const double *epochs,
                      NodeTable &nt)
{
    const int nb = ctx->E.n_bodies;
    double *t0, *h, *r64;
    float *r32;
    GET(S_NT_T0, n_stops, t0);
    GET(S_NT_H, n_stops, h);
    GET(S_NT_R64, (size_t)n_stops * 8 * nb * 6, r64);
    GET(S_NT_R32, (size_t)n_stops * 8 * nb * 6, r32);
    CUDA_TRY(launch_node_table(ctx->E, stops_dev, n_stops, epochs, t0, h, r64, r32, ctx->stream));
    nt.t0 = t0;
    nt.h = h;
    nt.row64 = r64;
    nt.row32 = r32;
    nt.n_legs = n_stops;
    nt.nb = nb;
    return KETE_OK;
}

static int run_chain(kete_ctx *ctx, const ForceDev &F, const double *states, const double *epochs,
                     int64_t n, ChainState &cs)
{
    GET(S_CHAIN, 8 * n, cs.w);
    GET(S_STATUS, n, cs.status);
    GET(S_KSTOP, n, cs.kstop);
    cs.n = n;
    CUDA_TRY(launch_chain_init(cs, states, epochs, F, ctx->stream));
    return KETE_OK;
}

extern "C" int kete_propagate(kete_ctx *ctx, double *states, double *epochs, int64_t n,
                              double t_target, const kete_force_model *fm, int32_t *status)
{
    if (!ctx) return KETE_ERR_BAD_ARG;
    if (!ctx->have_ephem) return fail(ctx, KETE_ERR_NO_EPHEM, "no ephemeris loaded");
    if (n < 0 || n > INT32_MAX || (n > 0 && (!states || !epochs)) || !std::isfinite(t_target))
        return fail(ctx, KETE_ERR_BAD_ARG, "bad arguments");
    ForceDev F;
    int r = make_force(ctx, fm, F);
    if (r != KETE_OK) return r;
    CUDA_TRY(cudaSetDevice(ctx->device));
    stats_begin(ctx);
    if (n > 0) {
        ChainState cs;
        r = run_chain(ctx, F, states, epochs, n, cs);
        if (r != KETE_OK) return r;
        double *d_stop;
        GET(S_STOPS, 1, d_stop);
        CUDA_TRY(cudaMemcpyAsync(d_stop, &t_target, sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
        NodeTable nt;
        r = node_table(ctx, d_stop, 1, epochs, nt);
        if (r != KETE_OK) return r;
        prop_event(ctx, true);
        r = propagate(ctx, F, cs, d_stop, 1, states, n, true, &nt, 0);
        if (r != KETE_OK) return r;
        prop_event(ctx, false);
        CUDA_TRY(launch_chain_finish(cs, states, epochs, status, ctx->stream));
        ctx->stats.launches = 4;
    }
    r = stats_end(ctx);
    if (r != KETE_OK) return r;
    stats_collect(ctx);
    return KETE_OK;
}

extern "C" int kete_propagate_legs(kete_ctx *ctx, double *states, double *epochs, int64_t n,
                                   double t_target, double leg_days, const kete_force_model *fm,
                                   int32_t *status)
{
    if (!ctx) return KETE_ERR_BAD_ARG;
    if (!ctx->have_ephem) return fail(ctx, KETE_ERR_NO_EPHEM, "no ephemeris loaded");
    if (n < 0 || n > INT32_MAX || (n > 0 && (!states || !epochs)) || !std::isfinite(t_target) ||
        !(leg_days > 0.0) || !std::isfinite(leg_days))
        return fail(ctx, KETE_ERR_BAD_ARG, "bad arguments (leg_days must be positive and finite)");
    ForceDev F;
    int r = make_force(ctx, fm, F);
    if (r != KETE_OK) return r;
    CUDA_TRY(cudaSetDevice(ctx->device));
    stats_begin(ctx);
    if (n > 0) {
        // the grid starts at the first body's epoch
        double e0 = 0.0;
        CUDA_TRY(cudaMemcpyAsync(&e0, epochs, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
        CUDA_TRY(cudaStreamSynchronize(ctx->stream));
        if (!std::isfinite(e0)) return fail(ctx, KETE_ERR_BAD_ARG, "epochs[0] is not finite");
        const double span = t_target - e0;
        const double n_legs = std::ceil(std::fabs(span) / leg_days);
        if (n_legs > 1e7) return fail(ctx, KETE_ERR_BAD_ARG, "more than 10,000,000 legs");
        const int64_t K = std::max<int64_t>(1, (int64_t)n_legs);
        std::vector<double> stops((size_t)K);
        const double sgn = span < 0.0 ? -1.0 : 1.0;
        for (int64_t k = 0; k + 1 < K; k++) stops[k] = e0 + sgn * leg_days * (double)(k + 1);
        stops[K - 1] = t_target;
        ChainState cs;
        r = run_chain(ctx, F, states, epochs, n, cs);
        if (r != KETE_OK) return r;
        double *d_stops;
        GET(S_STOPS, K, d_stops);
        CUDA_TRY(cudaMemcpyAsync(d_stops, stops.data(), K * sizeof(double), cudaMemcpyHostToDevice,
                                 ctx->stream));
        // internal stops in chunks whose states go to scratch (at most 2 GiB),
        // then the target alone, whose states go to the caller's array: a body
        // that failed is not written there and keeps its input state
        const int64_t M = K - 1;
        const int64_t cap = std::max<int64_t>(1, ((int64_t)1 << 31) / (48 * n));
        const int64_t C = std::max<int64_t>(1, std::min<int64_t>(std::min<int64_t>(M, 512), cap));
        double *scratch = nullptr;
        if (M > 0) GET(S_LEG_OUT, (size_t)C * 6 * (size_t)n, scratch);
        int launches = 2;
        prop_event(ctx, true);
        for (int64_t j0 = 0; j0 < K;) {
            const bool last = (j0 == M);
            const int64_t cnt = last ? 1 : std::min(C, M - j0);
            NodeTable nt;
            r = node_table(ctx, d_stops + j0, (int)cnt, j0 == 0 ? epochs : d_stops + j0 - 1, nt);
            if (r != KETE_OK) return r;
            r = propagate(ctx, F, cs, d_stops + j0, (int)cnt, last ? states : scratch, n, true, &nt,
                          0);
            if (r != KETE_OK) return r;
            launches += 2;
            j0 += cnt;
        }
        prop_event(ctx, false);
        CUDA_TRY(launch_chain_finish(cs, states, epochs, status, ctx->stream));
        ctx->stats.launches = launches;
    }
    r = stats_end(ctx);
    if (r != KETE_OK) return r;
    stats_collect(ctx);
    return KETE_OK;
}

extern "C" int kete_propagate_stops(kete_ctx *ctx, const double *states, const double *epochs,
                                    int64_t n, const double *stops, int64_t n_stops,
                                    const kete_force_model *fm, double *out, int32_t *status)
{
    if (!ctx) return KETE_ERR_BAD_ARG;
    if (!ctx->have_ephem) return fail(ctx, KETE_ERR_NO_EPHEM, "no ephemeris loaded");
    if (n < 0 || n > INT32_MAX || n_stops < 0 || n_stops > INT32_MAX ||
        (n > 0 && (!states || !epochs)) || (n_stops > 0 && (!stops || !out)))
        return fail(ctx, KETE_ERR_BAD_ARG, "bad arguments");
    for (int64_t k = 0; k < n_stops; k++)
        if (!std::isfinite(stops[k]) || (k > 0 && stops[k] < stops[k - 1]))
            return fail(ctx, KETE_ERR_BAD_ARG, "stops must be finite and ascending");
    ForceDev F;
    int r = make_force(ctx, fm, F);
    if (r != KETE_OK) return r;
    CUDA_TRY(cudaSetDevice(ctx->device));
    stats_begin(ctx);
    if (n > 0 && n_stops > 0) {
        ChainState cs;
        r = run_chain(ctx, F, states, epochs, n, cs);
        if (r != KETE_OK) return r;
        double *d_stops;
        GET(S_STOPS, n_stops, d_stops);
        CUDA_TRY(cudaMemcpyAsync(d_stops, stops, n_stops * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
        NodeTable nt;
        r = node_table(ctx, d_stops, (int)n_stops, epochs, nt);
        if (r != KETE_OK) return r;
        prop_event(ctx, true);
        r = propagate(ctx, F, cs, d_stops, (int)n_stops, out, n, false, &nt, 0);
        if (r != KETE_OK) return r;
        prop_event(ctx, false);
        CUDA_TRY(launch_chain_finish(cs, nullptr, nullptr, status, ctx->stream));
        ctx->stats.launches = 4;
    }
    r = stats_end(ctx);
    if (r != KETE_OK) return r;
    stats_collect(ctx);
    return KETE_OK;
}

// Union of the sub-frames' hits (tmp, nh in any order; parent[sub-frame]) per
// parent frame: one hit per (frame, body), the earliest sub-frame's, sorted by
// (frame, body) into hits.  CAPACITY leaves the merged count in *n_hits.
static int merge_extended(kete_ctx *ctx, const kete_hit *tmp, unsigned long long nh,
                          const int32_t *parent, int64_t np, kete_hit *hits, int64_t capacity,
                          int64_t *n_hits, int64_t &launches)
{
    cudaStream_t st = ctx->stream;
    int32_t *cnt, *cur, *kcnt; int64_t *off, *koff, *scan_tmp; kete_hit *grp; int8_t *keep;
    GET(S_EXT_CNT, np, cnt);
    GET(S_EXT_CUR, np, cur);
    GET(S_EXT_KCNT, np, kcnt);
    GET(S_EXT_OFF, np + 1, off);
    GET(S_EXT_KOFF, np + 1, koff);
    GET(S_EXT_TMP, scan_tmp_elems(np), scan_tmp);
    GET(S_EXT_GROUP, nh, grp);
    GET(S_EXT_KEEP, nh, keep);
    phase_mark(ctx, PH_ORDER, true);
    CUDA_TRY(cudaMemsetAsync(cnt, 0, np * sizeof(int32_t), st));
    CUDA_TRY(cudaMemsetAsync(cur, 0, np * sizeof(int32_t), st));
    CUDA_TRY(fov_merge_count(tmp, nh, parent, cnt, nullptr, nullptr, nullptr, false, st));
    CUDA_TRY(exclusive_scan(cnt, np, off, scan_tmp, st));
    CUDA_TRY(fov_merge_count(tmp, nh, parent, cnt, off, cur, grp, true, st));
    CUDA_TRY(fov_merge_keep(grp, off, np, keep, kcnt, ctx->n_sm, st));
    CUDA_TRY(exclusive_scan(kcnt, np, koff, scan_tmp, st));
    int64_t merged = 0;
    CUDA_TRY(cudaMemcpyAsync(&merged, koff + np, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    launches += 3 + 2 * scan_launches(np);
    *n_hits = merged;
    if (merged > capacity) {
        phase_mark(ctx, PH_ORDER, false);
        return fail(ctx, KETE_ERR_CAPACITY, "hit buffer holds %lld, %lld needed", (long long)capacity,
                    (long long)merged);
    }
    if (merged > 0) {
        CUDA_TRY(fov_merge_place(grp, off, keep, koff, np, hits, ctx->n_sm, st));
        launches++;
    }
    phase_mark(ctx, PH_ORDER, false);
    return KETE_OK;
}

// sky-cell grid: bands of height ~cell, cells of width >= cell along each band
static void make_bands(double cell, std::vector<int32_t> &off, std::vector<int32_t> &cnt,
                       double &hb, int &n_bands, int &n_cells)
{
    const double pi = 3.14159265358979323846;
    n_bands = std::max(1, (int)std::ceil(pi / cell));
    hb = pi / n_bands;
    off.assign(n_bands + 1, 0);
    cnt.assign(n_bands, 1);
    for (int j = 0; j < n_bands; j++) {
        double lo = -0.5 * pi + j * hb, hi = lo + hb;
        double closest = (lo <= 0.0 && hi >= 0.0) ? 0.0 : std::min(std::fabs(lo), std::fabs(hi));
        int nj = (int)std::floor(2.0 * pi * std::cos(closest) / cell);
        cnt[j] = std::max(1, nj);
        off[j + 1] = off[j] + cnt[j];
    }
    n_cells = off[n_bands];
}

// The survey driver.  ext_nsub > 0: the frames are extended exposures of
// ext_dur[f] days each (device), replaced by ext_nsub instantaneous sub-frames
// (fov_ext_expand) whose hits are merged back per frame at the end.
static int fov_check_impl(kete_ctx *ctx, const double *states, const double *epochs,
                          int64_t n, const kete_frame *frames, int64_t n_frames,
                          const double *observers, int64_t n_obs,
                          const kete_force_model *fm, const kete_survey_opts *opt_in,
                          const kete_mag_params *mag, kete_hit *hits, int64_t capacity,
                          int64_t *n_hits, int32_t *status, const double *ext_dur = nullptr,
                          int ext_nsub = 0)
{
    if (!ctx) return KETE_ERR_BAD_ARG;
    if (!ctx->have_ephem) return fail(ctx, KETE_ERR_NO_EPHEM, "no ephemeris loaded");
    if (!n_hits || n < 0 || n > INT32_MAX || n_frames < 0 || n_frames >= INT32_MAX || n_obs < 0 ||
        capacity < 0 || (n > 0 && (!states || !epochs)) ||
        (n_frames > 0 && (!frames || !observers || n_obs == 0)) || (capacity > 0 && !hits))
        return fail(ctx, KETE_ERR_BAD_ARG, "bad arguments");
    kete_survey_opts opt;
    if (opt_in) opt = *opt_in;
    else kete_survey_opts_default(&opt);
    if (!(opt.batch_span >= 0) || !(opt.twobody_max >= 0) || !(opt.cell_deg >= 0) ||
        !(opt.mem_budget_gb >= 0))
        return fail(ctx, KETE_ERR_BAD_ARG, "invalid survey options");
    ForceDev F;
    int r = make_force(ctx, fm, F);
    if (r != KETE_OK) return r;
    const bool ext = ext_nsub > 0;
    if (ext && (ext_nsub > KETE_EXT_MAX_SUB || (n_frames > 0 && !ext_dur) ||
                n_frames * (int64_t)ext_nsub >= INT32_MAX))
        return fail(ctx, KETE_ERR_BAD_ARG, "extended exposures: n_sub must be 1..%d, durations "
                    "given, n_frames * n_sub below 2^31", KETE_EXT_MAX_SUB);
    *n_hits = 0;
    CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    stats_begin(ctx);
    int64_t launches = 0;
    int32_t *ext_parent = nullptr;
    if (ext && n_frames > 0) {
        // sub-frames of the extended exposures (Sec. 3.1)
        int32_t *pst, *pfirst; int64_t *pex, *ptmp; kete_frame *sub;
        GET(S_EXT_START, n_frames, pst);
        GET(S_EXT_EX, n_frames + 1, pex);
        GET(S_EXT_TMP, scan_tmp_elems(n_frames), ptmp);
        GET(S_EXT_FIRST, n_frames + 1, pfirst);
        GET(S_EXT_SUB, n_frames * ext_nsub, sub);
        GET(S_EXT_PARENT, n_frames * ext_nsub, ext_parent);
        CUDA_TRY(fov_ext_expand(frames, ext_dur, n_frames, ext_nsub, n_obs, pst, pex, ptmp, pfirst,
                                sub, ext_parent, ctx->d_ctr, st));
        launches += 3 + scan_launches(n_frames);
        CUDA_TRY(cudaMemcpyAsync(ctx->h_ctr, ctx->d_ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaStreamSynchronize(st));
        const int fl = ctx->h_ctr->error_flags;
        if (fl & 1) return fail(ctx, KETE_ERR_BAD_ARG, "frames are not sorted by epoch");
        if (fl & 2) return fail(ctx, KETE_ERR_BAD_ARG, "frames of one exposure differ in epoch, observer or duration");
        if (fl & 4) return fail(ctx, KETE_ERR_BAD_ARG, "observer_idx + n_sub exceeds the observer rows");
        if (fl & 64) return fail(ctx, KETE_ERR_BAD_ARG, "exposure durations must be finite and >= 0");
        frames = sub;
        n_frames *= ext_nsub;
    }
    const int64_t nf = n_frames;
    ChainState cs{};
    if (n > 0) {
        r = run_chain(ctx, F, states, epochs, n, cs);
        if (r != KETE_OK) return r;
        launches++;
    }
    if (nf == 0 || n == 0) {
        if (n > 0) CUDA_TRY(launch_chain_finish(cs, nullptr, nullptr, status, st));
        r = stats_end(ctx);
        if (r != KETE_OK) return r;
        stats_collect(ctx);
        return KETE_OK;
    }
    // ---- frames -> exposures ------------------------------------------------
    int32_t *is_start; int64_t *ex, *scan_tmp; double *fcen; float4 *faux; int32_t *exp_first;
    GET(S_ISSTART, nf, is_start);
    GET(S_EX, nf + 1, ex);
    GET(S_FCEN, 4 * nf, fcen);
    GET(S_FAUX, nf, faux);
    phase_mark(ctx, PH_PREP, true);
    CUDA_TRY(fov_frame_prep(frames, nf, n_obs, is_start, fcen, faux, ctx->d_ctr, st));
    GET(S_SCANTMP, scan_tmp_elems(nf), scan_tmp);
    CUDA_TRY(exclusive_scan(is_start, nf, ex, scan_tmp, st));
    GET(S_EXPFIRST, nf + 1, exp_first);
    CUDA_TRY(fov_exposure_first(is_start, ex, nf, exp_first, st));
    launches += 3 + 2;
    int64_t h_ne = 0;
    CUDA_TRY(cudaMemcpyAsync(&h_ne, ex + nf, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaMemcpyAsync(ctx->h_ctr, ctx->d_ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    int flags = ctx->h_ctr->error_flags;
    if ((flags & 1) && ext)
        return fail(ctx, KETE_ERR_BAD_ARG, "sub-frame epochs are not sorted: extended exposures overlap in time");
    if (flags & 1) return fail(ctx, KETE_ERR_BAD_ARG, "frames are not sorted by epoch");
    if (flags & 2) return fail(ctx, KETE_ERR_BAD_ARG, "frames of one exposure differ in epoch or observer");
    if (flags & 4) return fail(ctx, KETE_ERR_BAD_ARG, "observer_idx out of range");
    if (flags & 8) return fail(ctx, KETE_ERR_BAD_ARG, "n_edges must be 3 or 4 (polygon) or 0 (cone)");
    if (flags & 16) return fail(ctx, KETE_ERR_BAD_ARG, "non-finite or degenerate frame");
    const int64_t ne = h_ne;
    ExpArrays X;
    GET(S_XEPOCH, ne, X.epoch);
    GET(S_XOBS, 3 * ne, X.obs);
    GET(S_XCEN, 3 * ne, X.cen);
    GET(S_XRAD, ne, X.rad);
    GET(S_XCS, ne, X.cs);
    GET(S_XCENF, ne, X.cenf);
    GET(S_XBATCH, ne, X.batch);
    GET(S_XSUN, 6 * ne, X.sun);
    GET(S_XOBSREL, ne, X.obs_rel);
    unsigned int *d_maxrad;
    GET(S_MAXRAD, 1, d_maxrad);
    CUDA_TRY(cudaMemsetAsync(d_maxrad, 0, sizeof(unsigned int), st));
    CUDA_TRY(fov_exposure_prep(ctx->E, frames, nf, observers, fcen, exp_first, ne, X, d_maxrad,
                               ctx->d_ctr, st));
    // ---- batches (Sec. 2) ---------------------------------------------------
    double span = std::min(opt.batch_span, 2.0 * opt.twobody_max);
    int32_t *next, *d_nb;
    BatchArrays B;
    GET(S_NEXT, ne, next);
    GET(S_BFIRST, ne + 1, B.first);
    GET(S_BTREF, ne, B.t_ref);
    GET(S_NBATCH, 1, d_nb);
    CUDA_TRY(fov_batches(X.epoch, ne, span, next, B, d_nb, st));
    launches += 3;
    int32_t h_nb = 0;
    unsigned int h_maxrad = 0;
    CUDA_TRY(cudaMemcpyAsync(&h_nb, d_nb, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaMemcpyAsync(&h_maxrad, d_maxrad, sizeof(unsigned int), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    const int32_t nb = h_nb;
    std::vector<int32_t> h_first(nb + 1);
    CUDA_TRY(cudaMemcpyAsync(h_first.data(), B.first, (nb + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    GET(S_BO, 3 * nb, B.O);
    GET(S_BROBS, nb, B.robs);
    GET(S_BTSPAN, nb, B.tspan);
    GET(S_BRMAX, nb, B.rmax);
    GET(S_BSUN, 6 * nb, B.sun);
    CUDA_TRY(fov_batch_info(ctx->E, X, B, nb, ctx->d_ctr, st));
    phase_mark(ctx, PH_PREP, false);
    launches++;
    // ---- sky cells -------------------------------------------------------------
    float maxrad;
    std::memcpy(&maxrad, &h_maxrad, sizeof(float));
    const double pi = 3.14159265358979323846;
    double cell = opt.cell_deg > 0 ? opt.cell_deg * pi / 180.0
                                   : std::min(20.0 * pi / 180.0, std::max(0.5 * pi / 180.0, 2.0 * (double)maxrad));
    std::vector<int32_t> boff, bcnt;
    CellGrid G;
    int n_bands, n_cells;
    make_bands(cell, boff, bcnt, G.hb, n_bands, n_cells);
    G.n_bands = n_bands;
    G.n_cells = n_cells;
    int32_t *d_bands;
    GET(S_BANDS, 2 * n_bands + 1, d_bands);
    CUDA_TRY(cudaMemcpyAsync(d_bands, boff.data(), (n_bands + 1) * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(d_bands + n_bands + 1, bcnt.data(), n_bands * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    G.band_off = d_bands;
    G.band_n = d_bands + n_bands + 1;
    // ---- chunks of batches ----------------------------------------------------
    double budget = (opt.mem_budget_gb > 0 ? opt.mem_budget_gb : 8.0) * 1e9;
    int64_t per_batch = 48 * n;
    int32_t C = (int32_t)std::max<int64_t>(1, std::min<int64_t>(nb, (int64_t)(budget / per_batch)));
    // keep the cell CSR of a chunk modest
    C = (int32_t)std::max<int64_t>(1, std::min<int64_t>(C, 200000000LL / std::max(1, n_cells)));
    double *stop_states;
    GET(S_STOPSTATES, (size_t)C * 6 * n, stop_states);
    int32_t *frame_cnt;
    GET(S_FRAMECNT, nf, frame_cnt);
    CUDA_TRY(cudaMemsetAsync(frame_cnt, 0, nf * sizeof(int32_t), st));
    unsigned long long cand_cap = ctx->slot[S_CAND].bytes / sizeof(uint2);
    if (cand_cap < (unsigned long long)(4 * n + 1024)) cand_cap = 4 * n + 1024;
    unsigned long long hit_cap = ctx->slot[S_HITTMP].bytes / sizeof(kete_hit);
    if (hit_cap < (unsigned long long)(nf + 1024)) hit_cap = nf + 1024;
    kete_hit *hit_tmp;
    GET(S_HITTMP, hit_cap, hit_tmp);
    hit_cap = ctx->slot[S_HITTMP].bytes / sizeof(kete_hit);
    NodeTable nt;
    r = node_table(ctx, B.t_ref, nb, epochs, nt);
    if (r != KETE_OK) return r;
    launches++;
    unsigned long long hits_total = 0, cands_total = 0, exact_total = 0;
    for (int32_t k0 = 0; k0 < nb; k0 += C) {
        const int32_t k1 = std::min(nb, k0 + C), nk = k1 - k0;
        const int32_t e0 = h_first[k0], e1 = h_first[k1];
        const int32_t nek = e1 - e0;
        // propagation to the batch midpoints of this chunk
        prop_event(ctx, true);
        r = propagate(ctx, F, cs, B.t_ref + k0, nk, stop_states, n, false, &nt, k0, true);
        if (r != KETE_OK) return r;
        prop_event(ctx, false);
        launches++;
        // exposures of the chunk into sky cells
        const int64_t nkeys = (int64_t)nk * n_cells;
        int32_t *ckey, *ccnt, *ccur, *cexp; int64_t *cstart;
        GET(S_CELLKEY, nek, ckey);
        GET(S_CELLCNT, nkeys, ccnt);
        GET(S_CELLCUR, nkeys, ccur);
        GET(S_CELLSTART, nkeys + 1, cstart);
        GET(S_CELLEXP, nek, cexp);
        GET(S_SCANTMP, std::max(scan_tmp_elems(nkeys), scan_tmp_elems(nf)), scan_tmp);
        phase_mark(ctx, PH_CAND, true);
        CUDA_TRY(cudaMemsetAsync(ccnt, 0, nkeys * sizeof(int32_t), st));
        CUDA_TRY(cudaMemsetAsync(ccur, 0, nkeys * sizeof(int32_t), st));
        CUDA_TRY(fov_cell_keys(X, G, e0, e1, k0, ckey, ccnt, st));
        CUDA_TRY(exclusive_scan(ccnt, nkeys, cstart, scan_tmp, st));
        CUDA_TRY(fov_cell_scatter(e0, e1, ckey, cstart, ccur, cexp, st));
        launches += 4;
        // candidate (exposure, body) pairs
        int32_t *exp_cnt;
        GET(S_EXPCNT, ne, exp_cnt);
        unsigned long long ncand = 0;
        for (int attempt = 0; attempt < 3; attempt++) {
            uint2 *cand;
            GET(S_CAND, cand_cap, cand);
            cand_cap = ctx->slot[S_CAND].bytes / sizeof(uint2);
            CUDA_TRY(cudaMemsetAsync(exp_cnt + e0, 0, nek * sizeof(int32_t), st));
            CUDA_TRY(cudaMemsetAsync(&ctx->d_ctr->candidates, 0, sizeof(unsigned long long), st));
            CandArgs ca;
            ca.X = X; ca.B = B; ca.G = G; ca.stop_states = stop_states; ca.n = n; ca.k0 = k0;
            ca.nk = nk; ca.cell_start = cstart; ca.cell_exp = cexp; ca.cand = cand;
            ca.cap = cand_cap; ca.exp_cnt = exp_cnt; ca.ctr = ctx->d_ctr; ca.mu_sun = ctx->E.gm[0];
            CUDA_TRY(fov_candidates(ca, st));
            launches++;
            CUDA_TRY(cudaMemcpyAsync(&ncand, &ctx->d_ctr->candidates, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
            CUDA_TRY(cudaStreamSynchronize(st));
            if (ncand <= cand_cap) break;
            cand_cap = ncand + ncand / 2 + 1024;
        }
        if (ncand > cand_cap)
            return fail(ctx, KETE_ERR_NOMEM, "candidate buffer could not grow to %llu pairs", ncand);
        cands_total += ncand;
        int64_t *exp_off; int32_t *exp_cur, *cand_body;
        GET(S_EXPOFF, nek + 1, exp_off);
        GET(S_EXPCUR, nek, exp_cur);
        GET(S_CANDBODY, ncand, cand_body);
        CUDA_TRY(exclusive_scan(exp_cnt + e0, nek, exp_off, scan_tmp, st));
        CUDA_TRY(cudaMemsetAsync(exp_cur, 0, nek * sizeof(int32_t), st));
        CUDA_TRY(fov_cand_scatter((const uint2 *)ctx->slot[S_CAND].p, ncand, exp_off, e0, exp_cur, cand_body, st));
        phase_mark(ctx, PH_CAND, false);
        launches += 3;
        // exact two-body + light time + polygon test, after the FP32 prefilter
        uint32_t *pre_keep;
        unsigned long long *pre_n;
        GET(S_PRE_KEEP, ncand, pre_keep);
        GET(S_PRE_N, 1, pre_n);
        for (int attempt = 0; attempt < 3; attempt++) {
            CUDA_TRY(cudaMemcpyAsync(&ctx->d_ctr->hits, &hits_total, sizeof(unsigned long long), cudaMemcpyHostToDevice, st));
            ExactArgs xa;
            xa.E = ctx->E; xa.X = X; xa.B = B; xa.frames = frames; xa.faux = faux;
            xa.stop_states = stop_states; xa.n = n; xa.k0 = k0; xa.e_begin = e0; xa.e_end = e1;
            xa.exp_off = exp_off; xa.n_cand = (int64_t)ncand; xa.cand_body = cand_body;
            xa.exp_first = exp_first;
            xa.hits = hit_tmp; xa.cap = hit_cap; xa.frame_cnt = frame_cnt; xa.status = cs.status;
            xa.ctr = ctx->d_ctr;
            xa.mag = mag;
            xa.keep = pre_keep;
            xa.n_keep = pre_n;
            phase_mark(ctx, PH_EXACT, true);
            CUDA_TRY(fov_exact(xa, ctx->n_sm, st));
            phase_mark(ctx, PH_EXACT, false);
            if (ncand > 0 && nek > 0) launches += ncand <= 0xffffffffull ? 2 : 1;
            unsigned long long nh = 0, nkept = ncand;
            CUDA_TRY(cudaMemcpyAsync(&nh, &ctx->d_ctr->hits, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
            if (ncand > 0 && nek > 0 && ncand <= 0xffffffffull)
                CUDA_TRY(cudaMemcpyAsync(&nkept, pre_n, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
            CUDA_TRY(cudaStreamSynchronize(st));
            if (nh <= hit_cap) {
                hits_total = nh;
                exact_total += nkept;
                break;
            }
            // grow the hit buffer, keep earlier chunks' hits, redo this chunk
            int32_t fa = 0, fb = 0;
            CUDA_TRY(cudaMemcpy(&fa, exp_first + e0, sizeof(int32_t), cudaMemcpyDeviceToHost));
            CUDA_TRY(cudaMemcpy(&fb, exp_first + e1, sizeof(int32_t), cudaMemcpyDeviceToHost));
            CUDA_TRY(cudaMemsetAsync(frame_cnt + fa, 0, (size_t)(fb - fa) * sizeof(int32_t), st));
            unsigned long long want = nh + nh / 2 + 1024;
            kete_hit *bigger = nullptr;
            CUDA_TRY(cudaMalloc(&bigger, want * sizeof(kete_hit)));
            if (hits_total)
                CUDA_TRY(cudaMemcpyAsync(bigger, hit_tmp, hits_total * sizeof(kete_hit), cudaMemcpyDeviceToDevice, st));
            CUDA_TRY(cudaStreamSynchronize(st));
            cudaFree(ctx->slot[S_HITTMP].p);
            ctx->slot[S_HITTMP].p = bigger;
            ctx->slot[S_HITTMP].bytes = want * sizeof(kete_hit);
            hit_tmp = bigger;
            hit_cap = want;
        }
        if (hits_total > hit_cap)
            return fail(ctx, KETE_ERR_NOMEM, "hit buffer could not grow to %llu hits", hits_total);
    }
    ctx->stats.n_batches = nb;
    ctx->stats.n_exposures = ne;
    ctx->stats.n_candidates = (int64_t)cands_total;
    ctx->stats.n_exact = (int64_t)exact_total;
    ctx->stats.n_hits = (int64_t)hits_total;
    *n_hits = (int64_t)hits_total;
    CUDA_TRY(launch_chain_finish(cs, nullptr, nullptr, status, st));
    launches++;
    CUDA_TRY(cudaMemcpyAsync(ctx->h_ctr, ctx->d_ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    if (ctx->h_ctr->error_flags & 32) {
        ctx->stats.launches = launches;
        return fail(ctx, KETE_ERR_EPHEM_SPAN, "a batch midpoint or frame epoch lies outside the ephemeris table");
    }
    if (ext) {
        r = merge_extended(ctx, hit_tmp, hits_total, ext_parent, nf / ext_nsub, hits, capacity,
                           n_hits, launches);
        if (r != KETE_OK) return r;
        r = stats_end(ctx);
        if (r != KETE_OK) return r;
        stats_collect(ctx);
        ctx->stats.n_batches = nb;
        ctx->stats.n_exposures = ne;
        ctx->stats.n_candidates = (int64_t)cands_total;
    ctx->stats.n_exact = (int64_t)exact_total;
        ctx->stats.n_hits = *n_hits;
        ctx->stats.launches = launches + ctx->extra_launches;
        return KETE_OK;
    }
    if ((int64_t)hits_total > capacity) {
        r = stats_end(ctx);
        stats_collect(ctx);
        ctx->stats.launches = launches + ctx->extra_launches;
        return fail(ctx, KETE_ERR_CAPACITY, "hit buffer holds %lld, %llu needed", (long long)capacity,
                    hits_total);
    }
    if (hits_total > 0) {
        int64_t *frame_off; int32_t *frame_cur; kete_hit *grouped;
        GET(S_FRAMEOFF, nf + 1, frame_off);
        GET(S_FRAMECUR, nf, frame_cur);
        GET(S_HITGROUP, hits_total, grouped);
        phase_mark(ctx, PH_ORDER, true);
        CUDA_TRY(exclusive_scan(frame_cnt, nf, frame_off, scan_tmp, st));
        CUDA_TRY(cudaMemsetAsync(frame_cur, 0, nf * sizeof(int32_t), st));
        CUDA_TRY(fov_order_hits(hit_tmp, hits_total, frame_off, nf, frame_cur, grouped, hits, ctx->n_sm, st));
        phase_mark(ctx, PH_ORDER, false);
        launches += 4;
    }
    r = stats_end(ctx);
    if (r != KETE_OK) return r;
    stats_collect(ctx);
    ctx->stats.n_batches = nb;
    ctx->stats.n_exposures = ne;
    ctx->stats.n_candidates = (int64_t)cands_total;
    ctx->stats.n_exact = (int64_t)exact_total;
    ctx->stats.n_hits = (int64_t)hits_total;
    ctx->stats.launches = launches + ctx->extra_launches;
    return KETE_OK;
}

extern "C" int kete_fov_check(kete_ctx *ctx, const double *states, const double *epochs,
                              int64_t n, const kete_frame *frames, int64_t n_frames,
                              const double *observers, int64_t n_obs,
                              const kete_force_model *fm, const kete_survey_opts *opt,
                              kete_hit *hits, int64_t capacity, int64_t *n_hits, int32_t *status)
{
    return fov_check_impl(ctx, states, epochs, n, frames, n_frames, observers, n_obs, fm, opt,
                          nullptr, hits, capacity, n_hits, status);
}

extern "C" int kete_fov_check_mag(kete_ctx *ctx, const double *states, const double *epochs,
                                  int64_t n, const kete_frame *frames, int64_t n_frames,
                                  const double *observers, int64_t n_obs,
                                  const kete_force_model *fm, const kete_survey_opts *opt,
                                  const kete_mag_params *mag_params, kete_hit *hits,
                                  int64_t capacity, int64_t *n_hits, int32_t *status)
{
    return fov_check_impl(ctx, states, epochs, n, frames, n_frames, observers, n_obs, fm, opt,
                          mag_params, hits, capacity, n_hits, status);
}

extern "C" int kete_fov_check_extended(kete_ctx *ctx, const double *states, const double *epochs,
                                       int64_t n, const kete_frame *frames, int64_t n_frames,
                                       const double *durations, int32_t n_sub,
                                       const double *observers, int64_t n_obs,
                                       const kete_force_model *fm, const kete_survey_opts *opt,
                                       const kete_mag_params *mag_params, kete_hit *hits,
                                       int64_t capacity, int64_t *n_hits, int32_t *status)
{
    if (ctx && n_sub < 1)
        return fail(ctx, KETE_ERR_BAD_ARG, "extended exposures: n_sub must be 1..%d", KETE_EXT_MAX_SUB);
    return fov_check_impl(ctx, states, epochs, n, frames, n_frames, observers, n_obs, fm, opt,
                          mag_params, hits, capacity, n_hits, status, durations, n_sub);
}

// Propagation whose chain scratch is a fixed device array (see kete.h): no
// cudaMalloc, cudaFree, scratch slot or event is touched on this path.
extern "C" int kete_propagate_noalloc(kete_ctx *ctx, double *states, double *epochs, int64_t n,
                                      double t_target, const kete_force_model *fm,
                                      int32_t *status)
{
    if (!ctx) return KETE_ERR_BAD_ARG;
    if (!ctx->have_ephem) return fail(ctx, KETE_ERR_NO_EPHEM, "no ephemeris loaded");
    if (n < 0 || (n > 0 && (!states || !epochs)) || !std::isfinite(t_target))
        return fail(ctx, KETE_ERR_BAD_ARG, "bad arguments");
    if (n > KETE_NOALLOC_MAX_BODIES)
        return fail(ctx, KETE_ERR_BAD_ARG, "n = %lld exceeds KETE_NOALLOC_MAX_BODIES = %d",
                    (long long)n, KETE_NOALLOC_MAX_BODIES);
    ForceDev F;
    int r = make_force(ctx, fm, F);
    if (r != KETE_OK) return r;
    CUDA_TRY(cudaSetDevice(ctx->device));
    const char *why = "";
    r = noalloc_propagate(ctx->device, ctx->stream, ctx->E, F, states, epochs, n, t_target,
                          status, &why);
    if (r != KETE_OK) return fail(ctx, r, "kete_propagate_noalloc: %s", why);
    return KETE_OK;
}

extern "C" int kete_set_propagation(kete_ctx *ctx, int precision, int kind, int block,
                                    int split_lanes, int defer_steps, int cost_order_on)
{
    if (!ctx) return KETE_ERR_BAD_ARG;
    const bool split_ok = split_lanes == 0 || split_lanes == 1 || split_lanes == 4 ||
                          split_lanes == 8 || split_lanes == 16;
    if ((precision != KETE_FP64 && precision != KETE_MIXED) ||
        (kind != KETE_PROP_STATIC && kind != KETE_PROP_WORK_STEALING) || block < 32 ||
        block > 128 || block % 32 != 0 || !split_ok || defer_steps < 0)
        return fail(ctx, KETE_ERR_BAD_ARG,
                    "bad propagation variant (precision %d, kind %d, block %d, split %d, defer %d)",
                    precision, kind, block, split_lanes, defer_steps);
    PropVariant v{kind, block};
    v.split = split_lanes > 1 ? split_lanes : 0;
    v.budget = v.split ? defer_steps : 0;
    v.order = cost_order_on ? 1 : 0;
    ctx->var[precision == KETE_MIXED ? 1 : 0] = v;
    return KETE_OK;
}

extern "C" int kete_autotune(kete_ctx *ctx, const double *states, const double *epochs, int64_t n,
                             const double *stops, int64_t n_stops, const kete_force_model *fm,
                             int64_t max_sample, int32_t *kind, int32_t *block,
                             int32_t *split_lanes, int32_t *defer_steps, int32_t *cost_order)
{
    if (!ctx) return KETE_ERR_BAD_ARG;
    if (!ctx->have_ephem) return fail(ctx, KETE_ERR_NO_EPHEM, "no ephemeris loaded");
    if (n <= 0 || n > INT32_MAX || !states || !epochs || n_stops <= 0 || n_stops > INT32_MAX ||
        !stops || max_sample <= 0)
        return fail(ctx, KETE_ERR_BAD_ARG, "bad arguments");
    for (int64_t k = 0; k < n_stops; k++)
        if (!std::isfinite(stops[k]) || (k > 0 && stops[k] < stops[k - 1]))
            return fail(ctx, KETE_ERR_BAD_ARG, "stops must be finite and ascending");
    ForceDev F;
    int r = make_force(ctx, fm, F);
    if (r != KETE_OK) return r;
    F.nongrav = nullptr;   // the sample is gathered: body indices differ from the caller's
    CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    // The sample (spread evenly over the bodies) runs on persistent grids scaled
    // down by m / n, so that each lane works through as many bodies as in the
    // whole run: on the full grid a sample would leave a lane a few bodies and
    // be dominated by its longest-lived ones, which favours the split variants.
    const int64_t m = std::min(n, max_sample);
    const double scale = (double)m / (double)n;
    double *sst, *sep, *out, *d_stops;
    GET(S_TUNE_ST, 6 * m, sst);
    GET(S_TUNE_EP, m, sep);
    GET(S_TUNE_OUT, (size_t)n_stops * 6 * m, out);
    GET(S_STOPS, n_stops, d_stops);
    CUDA_TRY(cudaMemcpyAsync(d_stops, stops, n_stops * sizeof(double), cudaMemcpyHostToDevice, st));
    CUDA_TRY(launch_gather_bodies(states, epochs, n, m, sst, sep, st));
    // schedules x cost order, then the split variants (with cost order)
    PropVariant cands[9];
    const int kinds[3][2] = {{PROP_STATIC, 128}, {PROP_WORK_STEALING, 64}, {PROP_WORK_STEALING, 128}};
    int n_cands = 0;
    for (int o = 0; o < 2; o++)
        for (int q = 0; q < 3; q++) {
            cands[n_cands] = PropVariant{kinds[q][0], kinds[q][1]};
            cands[n_cands++].order = o;
        }
    const int splits[3][2] = {{8, 64}, {4, 64}, {8, 24}};
    for (int q = 0; q < 3; q++) {
        cands[n_cands] = PropVariant{PROP_WORK_STEALING, 128};
        cands[n_cands].split = splits[q][0];
        cands[n_cands].budget = splits[q][1];
        cands[n_cands++].order = 1;
    }
    const int slot = F.precision == KETE_MIXED ? 1 : 0;
    const PropVariant saved = ctx->var[slot];
    float best_ms = 1e30f, saved_ms = -1.0f;
    PropVariant best = saved;
    cudaEvent_t e0 = event_at(ctx, 0), e1 = event_at(ctx, 1);
    // time variant v on cnt bodies (states st, epochs ep; output rows out),
    // the best of reps runs after one that warms up
    auto time_variant = [&](const PropVariant &v, const double *st_, const double *ep_,
                            int64_t cnt, double *out_, int reps, float &ms) -> int {
        ctx->var[slot] = v;
        ms = 1e30f;
        for (int rep = 0; rep <= reps; rep++) {
            ChainState cs;
            int r2 = run_chain(ctx, F, st_, ep_, cnt, cs);
            if (r2 != KETE_OK) return r2;
            NodeTable nt;
            r2 = node_table(ctx, d_stops, (int)n_stops, ep_, nt);
            if (r2 != KETE_OK) return r2;
            CUDA_TRY(cudaMemsetAsync(ctx->d_ctr, 0, sizeof(DevCounters), st));
            CUDA_TRY(cudaEventRecord(e0, st));
            r2 = propagate(ctx, F, cs, d_stops, (int)n_stops, out_, cnt, false, &nt, 0);
            if (r2 != KETE_OK) return r2;
            CUDA_TRY(cudaEventRecord(e1, st));
            CUDA_TRY(cudaEventSynchronize(e1));
            float t = 0.0f;
            CUDA_TRY(cudaEventElapsedTime(&t, e0, e1));
            if (rep > 0) ms = std::min(ms, t);
        }
        return KETE_OK;
    };
    for (int c = 0; c < n_cands; c++) cands[c].grid_scale = scale;
    for (int c = 0; c < n_cands; c++) {
        float ms;
        r = time_variant(cands[c], sst, sep, m, out, 2, ms);
        if (r != KETE_OK) return r;
        if (ms < best_ms) {
            best_ms = ms;
            best = cands[c];
        }
        if (cands[c].kind == saved.kind && cands[c].block == saved.block &&
            cands[c].split == saved.split && cands[c].budget == saved.budget &&
            cands[c].order == saved.order)
            saved_ms = ms;
    }
    // a sample ranks variants that differ by a few per cent unreliably (its
    // scaled-down grid holds fewer warps per SM than the real launch): the
    // variant in use stays unless another beats it by more than 5 %, and a
    // pick that does is checked against it on all the bodies when their
    // output rows fit in 2 GB
    if (saved_ms > 0.0f && best_ms > 0.95f * saved_ms) best = saved;
    const bool same = best.kind == saved.kind && best.block == saved.block &&
                      best.split == saved.split && best.budget == saved.budget &&
                      best.order == saved.order;
    if (!same && m < n && saved_ms > 0.0f && (double)n_stops * 48.0 * (double)n <= 2e9) {
        double *full_out;
        GET(S_TUNE_OUT, (size_t)n_stops * 6 * n, full_out);
        PropVariant pick = best, cur = saved;
        pick.grid_scale = cur.grid_scale = 1.0;
        // the best of two runs each (run-to-run spread ~1-2 %); the pick must
        // win by 2 %
        float ms_pick, ms_cur;
        r = time_variant(cur, states, epochs, n, full_out, 2, ms_cur);
        if (r != KETE_OK) return r;
        r = time_variant(pick, states, epochs, n, full_out, 2, ms_pick);
        if (r != KETE_OK) return r;
        if (!(ms_pick < 0.98f * ms_cur)) best = saved;
    }
    best.grid_scale = 1.0;
    ctx->var[F.precision == KETE_MIXED ? 1 : 0] = best;
    if (kind) *kind = best.kind;
    if (block) *block = best.block;
    if (split_lanes) *split_lanes = best.split;
    if (defer_steps) *defer_steps = best.budget;
    if (cost_order) *cost_order = best.order;
    return KETE_OK;
}

// The orbit-fit path of kete_adjoint and kete_sky_jacobian: forward pass with
// step records, then (jac) the state-transition matrix at every batch
// midpoint, the observations (loss, predictions, partials), then (grad) the
// backward pass.
static int adjoint_impl(kete_ctx *ctx, const double *states, const double *epochs, int64_t n,
                        const kete_obs *obs, int32_t m, const kete_force_model *fm,
                        const kete_survey_opts *opt_in, double ckpt_days, double *loss,
                        double *grad, double *pred, double *jac, int32_t *status)
{
    if (!ctx) return KETE_ERR_BAD_ARG;
    if (!ctx->have_ephem) return fail(ctx, KETE_ERR_NO_EPHEM, "no ephemeris loaded");
    if (n < 0 || n > INT32_MAX || m < 1 || m > KETE_ADJ_MAX_OBS ||
        (n > 0 && (!states || !epochs || !obs || (!loss && !jac))) ||
        !(ckpt_days == 0.0 || ckpt_days >= 1e-3) || !std::isfinite(ckpt_days))
        return fail(ctx, KETE_ERR_BAD_ARG,
                    "bad arguments (m must lie in 1..%d, ckpt_days 0 or >= 1e-3)", KETE_ADJ_MAX_OBS);
    kete_survey_opts opt;
    if (opt_in) opt = *opt_in;
    else kete_survey_opts_default(&opt);
    if (!(opt.batch_span > 0) || !(opt.twobody_max >= 0) || !(opt.mem_budget_gb >= 0))
        return fail(ctx, KETE_ERR_BAD_ARG, "invalid survey options");
    kete_force_model fm64;
    if (fm) fm64 = *fm;
    else kete_force_model_default(&fm64);
    fm64.precision = KETE_FP64;
    ForceDev F;
    int r = make_force(ctx, &fm64, F);
    if (r != KETE_OK) return r;
    CUDA_TRY(cudaSetDevice(ctx->device));
    stats_begin(ctx);
    if (n > 0) {
        const double eps_obl = 84381.448 / 3600.0 * 3.14159265358979323846 / 180.0;
        AdjProblem P;
        P.states = states;
        P.epochs = epochs;
        P.n = n;
        P.obs = obs;
        P.m = m;
        P.span = std::min(opt.batch_span, 2.0 * opt.twobody_max);
        P.ckpt = ckpt_days;
        P.cos_eps = std::cos(eps_obl);
        P.sin_eps = std::sin(eps_obl);
        P.loss = loss;
        P.grad = grad;
        P.pred = pred;
        P.jac = jac;
        P.status = status;
        P.ctr = ctx->d_ctr;
        // scratch per chunk of bodies within the memory budget
        const int cap = KETE_ADJ_MAX_STEPS;
        // with non-gravitational terms the records carry the full model's Jacobian
        const bool full = fm64.nongrav != nullptr;
        const size_t per_body = (size_t)cap * (kAdjRec + (full ? kAdjRecX : 0)) * sizeof(double) +
                                (size_t)m * (sizeof(int32_t) + 12 * sizeof(double)) +
                                (jac ? (size_t)m * 36 * sizeof(double) : 0) +
                                3 * sizeof(int32_t);
        const double budget = (opt.mem_budget_gb > 0 ? opt.mem_budget_gb : 8.0) * 1073741824.0;
        int64_t chunk = (int64_t)(budget / (double)per_body);
        chunk = std::max<int64_t>(1, std::min<int64_t>(chunk, n));
        const int64_t n_chunks = (n + chunk - 1) / chunk;   // even chunks
        chunk = (n + n_chunks - 1) / n_chunks;
        AdjBuffers B;
        B.cap = cap;
        GET(S_ADJ_REC, (size_t)chunk * cap * kAdjRec, B.rec);
        GET(S_ADJ_NREC, chunk, B.n_rec);
        GET(S_ADJ_NBAT, chunk, B.nbat);
        GET(S_ADJ_BIDX, (size_t)chunk * m, B.bidx);
        GET(S_ADJ_YREF, (size_t)chunk * m * 6, B.yref);
        GET(S_ADJ_GJUMP, (size_t)chunk * m * 6, B.gjump);
        GET(S_ADJ_STATUS, chunk, B.status);
        B.phi = nullptr;
        if (jac) GET(S_ADJ_PHI, (size_t)chunk * m * 36, B.phi);
        B.recx = nullptr;
        B.rich = nullptr;
        if (full) {
            GET(S_ADJ_RECX, (size_t)chunk * cap * kAdjRecX, B.recx);
            GET(S_ADJ_RICH, chunk, B.rich);
        }
        unsigned long long *next = nullptr;
        GET(S_NEXTBODY, 1, next);
        int launches = 0;
        double *t_end;
        GET(S_ADJ_TEND, chunk, t_end);
        const bool order_on = ctx->var[0].order != 0;
        for (int64_t i0 = 0; i0 < n; i0 += chunk) {
            const int64_t nc = std::min(chunk, n - i0);
            prop_event(ctx, true);
            int32_t *order = nullptr;
            if (order_on) {   // most expensive bodies first (schedule only)
                unsigned long long *order_n;
                CUDA_TRY(launch_adjoint_last_epoch(P, i0, nc, t_end, ctx->stream));
                // bodies with and without non-gravitational terms in separate
                // ranges, so that the full-model records rarely share a warp
                int r2 = cost_order(ctx, states + i0, n, epochs + i0, nc, nullptr, 0, t_end,
                                    F.nongrav ? F.nongrav + i0 : nullptr, &order, &order_n);
                if (r2 != KETE_OK) return r2;
                launches += 1;
            }
            CUDA_TRY(launch_adjoint_forward(ctx->E, F, B, P, i0, nc, next, ctx->stream, order));
            prop_event(ctx, false);
            if (jac) {
                CUDA_TRY(launch_adjoint_stm(B, P, i0, nc, ctx->stream));
                launches++;
            }
            CUDA_TRY(launch_adjoint_observe(ctx->E, B, P, i0, nc, ctx->stream));
            launches += 2;
            if (grad) {
                CUDA_TRY(launch_adjoint_backward(B, P, i0, nc, ctx->stream));
                launches++;
            }
        }
        ctx->stats.launches = launches;
    }
    r = stats_end(ctx);
    if (r != KETE_OK) return r;
    stats_collect(ctx);
    if (ctx->h_ctr->error_flags & (1 << 6))
        return fail(ctx, KETE_ERR_BAD_ARG, "observations of a body are not sorted by epoch");
    return KETE_OK;
}

extern "C" int kete_adjoint(kete_ctx *ctx, const double *states, const double *epochs, int64_t n,
                            const kete_obs *obs, int32_t m, const kete_force_model *fm,
                            const kete_survey_opts *opt, double ckpt_days, double *loss,
                            double *grad, double *pred, int32_t *status)
{
    if (ctx && n > 0 && !loss) return fail(ctx, KETE_ERR_BAD_ARG, "loss is required");
    return adjoint_impl(ctx, states, epochs, n, obs, m, fm, opt, ckpt_days, loss, grad, pred,
                        nullptr, status);
}

extern "C" int kete_sky_jacobian(kete_ctx *ctx, const double *states, const double *epochs,
                                 int64_t n, const kete_obs *obs, int32_t m,
                                 const kete_force_model *fm, const kete_survey_opts *opt,
                                 double ckpt_days, double *jac, double *pred, int32_t *status)
{
    if (ctx && n > 0 && !jac) return fail(ctx, KETE_ERR_BAD_ARG, "jac is required");
    return adjoint_impl(ctx, states, epochs, n, obs, m, fm, opt, ckpt_days, nullptr, nullptr,
                        pred, jac, status);
}
