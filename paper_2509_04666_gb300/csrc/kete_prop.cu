// kete_prop.cu -- n-body propagation of massless bodies (Sec. 3.2, App. A, App. A.6).
//
// Each lane integrates one body at a time along its chain of stops (the
// body's epoch, then every stop in order).  Each step is a 15th-order Gauss-Radau step in the
// IAS15 form (Newton-basis coefficients g, power-basis coefficients b, 8
// spacings), with the predictor removed: every step starts from b = 0 and the
// corrector iterates until max|db6|/max|a| < eps_pc, the error stops falling
// (after 3 iterations) or max_iter is reached.  Step control follows IAS15:
// dt_new = dt (eps / (max|b6|/max|a|))^(1/7), reject below safety*dt, grow at
// most 1/safety.  Every loop is bounded: max_iter corrector iterations,
// max_steps step attempts per leg, after which the body gets a status code.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "kete_step.cuh"

namespace kete {

void upload_radau_tables(cudaStream_t st) { upload_step_tables(st); }

#ifndef KETE_PROP_MIN_BLOCKS
#define KETE_PROP_MIN_BLOCKS 1   // resident blocks per SM asked of the register allocator
#endif

// The propagation kernel.  Each group of G lanes (G = 1: one lane) owns one
// body at a time and advances it along its chain of stops, writing the state
// at every stop to out[k][c][i] (stride out_stride between rows; out_aos: to
// out[k][i][c] with out_stride bodies per stop, one contiguous 48-byte record
// per body and stop) and the chain state back when it is done.  Stop k of this launch is leg leg0 + k of the
// node table (if any).
// One pass of the loop is one corrector sweep (7 force evaluations) for every
// group inside a step attempt; a group at a step boundary first evaluates the
// acceleration there and starts its attempt, in the same pass.  A group whose
// corrector converges after fewer sweeps than its warp-mates' does not wait
// for them: it ends its step and joins the next pass with its next attempt.
// (An FP64 warp-instruction costs the same whatever its active lanes, so
// lanes idling through other lanes' extra sweeps are lost throughput.)
//   refill = 0 (static): group j of the grid takes body j and then idles;
//   refill = 1 (work stealing, persistent grid): a group whose body is done
//   takes the next one from an atomic counter (warp-aggregated), so a body
//   needing hundreds of steps no longer idles the rest of its warp.
// Every body sees the same arithmetic in the same order whatever the
// schedule and whatever its warp-mates do: results are identical.
// Queue q: the bodies come from q.list (q.list_n of them, device) instead of
// 0..n-1, resuming at their saved stops cs.kstop[i] if q.resume; with q.defer set, a
// body that has made more than q.budget step attempts per stop reached is
// set aside at its next step boundary (state and stop saved, index appended
// to q.defer) for a second launch with more lanes per body.
// NG: bodies may carry non-gravitational terms (F.nongrav); the instantiation
// without them has those branches compiled out.
template <int MODE, int G, bool NG, bool V32 = false>
__global__ void __launch_bounds__(128, KETE_PROP_MIN_BLOCKS)
k_propagate(EphemDev E, ForceDev F, ChainState cs, const double *__restrict__ stops,
            int n_stops, double *__restrict__ out, int64_t out_stride, int out_aos,
            int keep_on_fail, DevCounters *ctr, NodeTable nt, int use_nt, int leg0,
            unsigned long long *__restrict__ next_body, int refill, PropQueue q)
{
    const int64_t n = cs.n;
    const unsigned long long n_items = q.list ? *q.list_n : (unsigned long long)n;
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int grank = LaneGroup<G>::rank();
    const bool writer = (grank == 0);
    Cnt cnt = {0, 0, 0, 0, 0};
    int64_t i = -1;           // current body (-1: none; n: no work left)
    int k = 0;                // next stop of the body
    double x[3], v[3], t = 0.0, dt = 0.0;
    int status = KETE_BODY_OK;
    long long attempts = 0, body_attempts = 0;
    StepState S;
    S.have_a0 = false;
    S.ng = nullptr;
    S.ng_chi = 0.0;
    LegView L = leg_view(nullptr, 0);
    Attempt A;
    bool in_attempt = false;  // A holds a step attempt with sweeps to go
    bool first = true;
    for (;;) {
        // groups without a body take the next ones
        const bool need = (i < 0);
        const unsigned m = __ballot_sync(FULL, need);
        if (m) {
            unsigned long long base = 0;
            const int leader = __ffs(m) - 1;
            if (refill) {
                if (lane == leader) base = atomicAdd(next_body, (unsigned long long)(__popc(m) / G));
                base = __shfl_sync(FULL, base, leader);
            }
            if (need) {
                // needing groups before this one, in lane order
                const unsigned before = m & ((1u << (lane - grank)) - 1u);
                unsigned long long mine = base + (unsigned long long)(__popc(before) / G);
                if (!refill)   // static: one body per group, taken on the first pass
                    mine = first ? ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) / G
                                 : n_items;
                if (mine < n_items) {
                    i = q.list ? (int64_t)q.list[mine] : (int64_t)mine;
#pragma unroll
                    for (int c = 0; c < 3; c++) {
                        x[c] = cs.w[c * n + i];
                        v[c] = cs.w[(3 + c) * n + i];
                    }
                    t = cs.w[6 * n + i];
                    dt = cs.w[7 * n + i];
                    status = cs.status[i];
                    k = q.resume ? cs.kstop[i] : 0;
                    attempts = 0;
                    body_attempts = 0;
                    S.have_a0 = false;
                    S.ng = (NG && F.nongrav) ? F.nongrav + i : nullptr;
                    S.ng_chi = 0.0;
                    L = leg_view(use_nt ? &nt : nullptr, leg0 + k);
                    in_attempt = false;
                    if (status == KETE_BODY_OK && k < n_stops) aim_step(F, t, stops[k], dt);
                } else {
                    i = n;   // drained
                }
            }
        }
        first = false;
        const bool active = (i >= 0 && i < n);
        if (!__any_sync(FULL, active)) break;
        if (!active) continue;
        // a group at a step boundary: set aside, or start its next attempt
        if (!in_attempt && k < n_stops && status == KETE_BODY_OK && t != stops[k]) {
            if (q.defer && !S.have_a0 && body_attempts >= (long long)q.budget * (k + 1)) {
                // set the body aside at this step boundary
                if (writer) {
#pragma unroll
                    for (int c = 0; c < 3; c++) {
                        cs.w[c * n + i] = x[c];
                        cs.w[(3 + c) * n + i] = v[c];
                    }
                    cs.w[6 * n + i] = t;
                    cs.w[7 * n + i] = dt;
                    cs.status[i] = status;
                    cs.kstop[i] = k;
                    q.defer[atomicAdd(q.defer_n, 1ull)] = (int32_t)i;
                    atomicAdd(&ctr->deferred, 1ull);
                }
                i = -1;
                continue;
            }
            body_attempts++;
            if (++attempts > F.max_steps) status = KETE_BODY_STEP_CAP;
            else status = step_begin<MODE, false, G>(E, F, L, x, v, t, dt, stops[k], S, A, cnt);
            in_attempt = (status == KETE_BODY_OK);
        }
        // one corrector sweep for every group inside an attempt
        if (in_attempt) {
            bool done = false;
            status = attempt_sweep<MODE, false, G, V32>(E, F, t, x, v, S.a0, S.as0, S.close, S.enc, A,
                                                   done, cnt, nullptr, S.ng, &S.ng_chi);
            if (status != KETE_BODY_OK) {
                in_attempt = false;
            } else if (done) {
                in_attempt = false;
                status = step_end<MODE>(F, A, x, v, t, dt, S, cnt);
            }
            if (in_attempt || (status == KETE_BODY_OK && t != stops[k])) continue;
        }
        // the body is at stop k (or failed): record it and move on
        while (k < n_stops && (status != KETE_BODY_OK || t == stops[k])) {
            // component c of this stop's record at o[c * cs_]
            double *o = out_aos ? out + ((int64_t)k * out_stride + i) * 6
                                : out + (int64_t)k * 6 * out_stride + i;
            const int64_t cs_ = out_aos ? 1 : out_stride;
            if (writer) {
                if (status == KETE_BODY_OK) {
#pragma unroll
                    for (int c = 0; c < 3; c++) {
                        o[c * cs_] = x[c];
                        o[(3 + c) * cs_] = v[c];
                    }
                } else if (!keep_on_fail) {
#pragma unroll
                    for (int c = 0; c < 6; c++) o[c * cs_] = __longlong_as_double(0x7ff8000000000000ll);
                }
            }
            k++;
            attempts = 0;
            S.have_a0 = false;
            if (k < n_stops) {
                L = leg_view(use_nt ? &nt : nullptr, leg0 + k);
                if (status == KETE_BODY_OK) aim_step(F, t, stops[k], dt);
            }
        }
        if (k < n_stops) continue;
        // all stops done: write the chain state back and free the group
        if (writer) {
#pragma unroll
            for (int c = 0; c < 3; c++) {
                cs.w[c * n + i] = x[c];
                cs.w[(3 + c) * n + i] = v[c];
            }
            cs.w[6 * n + i] = t;
            cs.w[7 * n + i] = dt;
            cs.status[i] = status;
        }
        i = -1;
    }
    flush_counters<G>(cnt, ctr);
}

// Node table: thread per (leg k, node n, body m).  Leg 0 starts at the first
// body's epoch (*epoch0, device), leg k > 0 at stops[k-1]; h is their exact
// difference, as the integrator forms it.
__global__ void k_node_table(EphemDev E, const double *__restrict__ stops, int n_stops,
                             const double *__restrict__ epoch0, double *__restrict__ t0,
                             double *__restrict__ hh,
                             double *__restrict__ row64, float *__restrict__ row32)
{
    const int nb = E.n_bodies;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)n_stops * 8 * nb) return;
    const int m = (int)(idx % nb);
    const int n = (int)((idx / nb) % 8);
    const int k = (int)(idx / (8 * nb));
    const double ts = (k == 0) ? epoch0[0] : stops[k - 1];
    const double h = stops[k] - ts;
    const double off = g_rt.h[n] * h;
    Seg g;
    double st[6], sun[6];
    const bool ok = ephem_seg(E, ts, off, g);
    double *o64 = row64 + (((int64_t)k * 8 + n) * nb + m) * 6;
    float *o32 = row32 + (((int64_t)k * 8 + n) * nb + m) * 6;
    if (ok) {
        cheb_pos_vel(ephem_coef(E, m, g.s), E.n_coef, g.tau, 2.0 * E.inv_seg, st, st + 3);
        cheb_pos_vel(ephem_coef(E, 0, g.s), E.n_coef, g.tau, 2.0 * E.inv_seg, sun, sun + 3);
        for (int q = 0; q < 6; q++) o64[q] = st[q];
        for (int q = 0; q < 3; q++) {
            o32[q] = (float)(st[q] - sun[q]);
            o32[3 + q] = (float)st[3 + q];
        }
    }
    if (m == 0 && n == 0) {
        t0[k] = ts;
        hh[k] = h;
    }
    // any node of the leg outside the table: the leg uses the per-thread path
    __syncwarp(__activemask());
    if (!ok) hh[k] = __longlong_as_double(0x7ff8000000000000ll);
}

__global__ void k_chain_init(ChainState cs, const double *__restrict__ states,
                             const double *__restrict__ epochs)
{
    const int64_t n = cs.n;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    bool ok = true;
    for (int c = 0; c < 6; c++) {
        double q = states[c * n + i];
        cs.w[c * n + i] = q;
        ok = ok && isfinite(q);
    }
    double t = epochs[i];
    cs.w[6 * n + i] = t;
    cs.w[7 * n + i] = 0.0;
    cs.status[i] = (ok && isfinite(t)) ? KETE_BODY_OK : KETE_BODY_NONFINITE;
}

__global__ void k_chain_finish(ChainState cs, double *__restrict__ epochs,
                               int32_t *__restrict__ status)
{
    const int64_t n = cs.n;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int s = cs.status[i];
    if (epochs && s == KETE_BODY_OK) epochs[i] = cs.w[6 * n + i];
    if (status) status[i] = s;
}

__global__ void k_ephem_eval(EphemDev E, const double *__restrict__ t, int64_t n, int body,
                             double *__restrict__ pos, double *__restrict__ vel)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    Seg g;
    double p[3], v[3];
    if (!ephem_seg(E, t[i], 0.0, g)) {
        for (int c = 0; c < 3; c++) {
            pos[3 * i + c] = __longlong_as_double(0x7ff8000000000000ll);
            if (vel) vel[3 * i + c] = __longlong_as_double(0x7ff8000000000000ll);
        }
        return;
    }
    cheb_pos_vel(ephem_coef(E, body, g.s), E.n_coef, g.tau, 2.0 * E.inv_seg, p, v);
    for (int c = 0; c < 3; c++) {
        pos[3 * i + c] = p[c];
        if (vel) vel[3 * i + c] = v[c];
    }
}

// evenly spread sample of m of the n bodies: dst[c][j] = src[c][floor(j n / m)]
// (autotuner)
__global__ void k_gather_bodies(const double *__restrict__ st, const double *__restrict__ ep,
                                int64_t n, int64_t m, double *__restrict__ dst,
                                double *__restrict__ dep)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    const int64_t i = (j * n) / m;
    for (int c = 0; c < 6; c++) dst[c * m + j] = st[c * n + i];
    dep[j] = ep[i];
}

static unsigned grid_for(int64_t n, int block) { return (unsigned)((n + block - 1) / block); }

cudaError_t launch_ephem_eval(const EphemDev &E, const double *t, int64_t n, int body,
                              double *pos, double *vel, cudaStream_t st)
{
    if (n > 0) k_ephem_eval<<<grid_for(n, 256), 256, 0, st>>>(E, t, n, body, pos, vel);
    return cudaGetLastError();
}

cudaError_t launch_chain_init(ChainState cs, const double *states, const double *epochs,
                              const ForceDev &, cudaStream_t st)
{
    if (cs.n > 0) k_chain_init<<<grid_for(cs.n, 256), 256, 0, st>>>(cs, states, epochs);
    return cudaGetLastError();
}

cudaError_t launch_node_table(const EphemDev &E, const double *stops_dev, int n_stops,
                              const double *epoch0, double *t0, double *h, double *row64,
                              float *row32, cudaStream_t st)
{
    int64_t tot = (int64_t)n_stops * 8 * E.n_bodies;
    if (tot > 0) k_node_table<<<grid_for(tot, 128), 128, 0, st>>>(E, stops_dev, n_stops, epoch0, t0, h, row64, row32);
    return cudaGetLastError();
}

template <int MODE, int G>
static int ws_blocks(int block)
{
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_propagate<MODE, G, false>, block, 0);
    return (sms > 0 ? sms : 152) * (per_sm > 0 ? per_sm : 1);
}

int propagate_ws_blocks(int block, int mode)
{
    return mode == KETE_MIXED ? ws_blocks<KETE_MIXED, 1>(block) : ws_blocks<KETE_FP64, 1>(block);
}

template <int MODE, int G>
static void launch_k(int64_t grid, int block, cudaStream_t st, const EphemDev &E,
                     const ForceDev &F, ChainState cs, const double *stops, int n_stops,
                     double *out, int64_t stride, int aos, int kof, DevCounters *ctr, NodeTable t,
                     int unt, int leg0, unsigned long long *next, int refill, PropQueue q)
{
    // mixed precision along a chain of stops served by node rows: the node
    // velocity in FP32 (V32); a single leg (one stop) rarely uses its rows
    if (F.nongrav) {
        k_propagate<MODE, G, true><<<(unsigned)grid, block, 0, st>>>(
            E, F, cs, stops, n_stops, out, stride, aos, kof, ctr, t, unt, leg0, next, refill, q);
        return;
    }
    if constexpr (MODE == KETE_MIXED && G == 1) {
        if (unt && n_stops > 1) {
            k_propagate<MODE, G, false, true><<<(unsigned)grid, block, 0, st>>>(
                E, F, cs, stops, n_stops, out, stride, aos, kof, ctr, t, unt, leg0, next, refill, q);
            return;
        }
    }
    k_propagate<MODE, G, false><<<(unsigned)grid, block, 0, st>>>(
        E, F, cs, stops, n_stops, out, stride, aos, kof, ctr, t, unt, leg0, next, refill, q);
}

template <int MODE>
static void launch_split(int G, int64_t grid, int block, cudaStream_t st, const EphemDev &E,
                         const ForceDev &F, ChainState cs, const double *stops, int n_stops,
                         double *out, int64_t stride, int aos, int kof, DevCounters *ctr,
                         NodeTable t, int unt, int leg0, unsigned long long *next, PropQueue q)
{
    if (G == 4)
        launch_k<MODE, 4>(grid, block, st, E, F, cs, stops, n_stops, out, stride, aos, kof, ctr, t, unt, leg0, next, 1, q);
    else if (G == 16)
        launch_k<MODE, 16>(grid, block, st, E, F, cs, stops, n_stops, out, stride, aos, kof, ctr, t, unt, leg0, next, 1, q);
    else
        launch_k<MODE, 8>(grid, block, st, E, F, cs, stops, n_stops, out, stride, aos, kof, ctr, t, unt, leg0, next, 1, q);
}

cudaError_t launch_propagate(const EphemDev &E, const ForceDev &F, ChainState cs,
                             const double *stops_dev, int n_stops, double *out,
                             int64_t out_stride, bool keep_on_fail, DevCounters *ctr,
                             cudaStream_t st, const NodeTable *nt, int leg0, PropVariant var,
                             unsigned long long *next_body, PropDefer *defer,
                             const int32_t *order, const unsigned long long *order_n,
                             bool out_aos)
{
    const int aos = out_aos ? 1 : 0;
    if (cs.n <= 0 || n_stops <= 0) return cudaGetLastError();
    NodeTable t{};
    if (nt) t = *nt;
    const int kof = keep_on_fail ? 1 : 0, unt = nt ? 1 : 0;
    const int block = (var.block > 0 && var.block <= 128) ? var.block : 128;
    const bool mixed = F.precision == KETE_MIXED;
    int refill = 0;
    int64_t grid = (cs.n + block - 1) / block;
    if (var.kind == PROP_WORK_STEALING && next_body) {
        cudaError_t e = cudaMemsetAsync(next_body, 0, sizeof(unsigned long long), st);
        if (e != cudaSuccess) return e;
        refill = 1;
        int64_t persistent = propagate_ws_blocks(block, F.precision);
        if (var.grid_scale < 1.0)
            persistent = std::max<int64_t>(1, (int64_t)(persistent * var.grid_scale + 0.5));
        if (grid > persistent) grid = persistent;
    }
    // phase 1: one lane per body; with a split variant, long bodies are set aside
    PropQueue q{};
    if (order && order_n) {
        q.list = order;
        q.list_n = order_n;
    }
    const bool split = var.split > 1 && var.budget > 0 && defer && cs.kstop;
    if (split) {
        cudaError_t e = cudaMemsetAsync(defer->count, 0, sizeof(unsigned long long), st);
        if (e != cudaSuccess) return e;
        q.defer = defer->list;
        q.defer_n = defer->count;
        q.budget = var.budget;
    }
    if (mixed)
        launch_k<KETE_MIXED, 1>(grid, block, st, E, F, cs, stops_dev, n_stops, out, out_stride, aos, kof, ctr, t, unt, leg0, next_body, refill, q);
    else
        launch_k<KETE_FP64, 1>(grid, block, st, E, F, cs, stops_dev, n_stops, out, out_stride, aos, kof, ctr, t, unt, leg0, next_body, refill, q);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !split) return e;
    // phase 2: the set-aside bodies, var.split lanes each, persistent grid
    e = cudaMemsetAsync(defer->next, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    PropQueue q2{};
    q2.list = defer->list;
    q2.list_n = defer->count;
    q2.resume = 1;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t grid2 = (int64_t)(sms > 0 ? sms : 152) * 2;
    if (var.grid_scale < 1.0)
        grid2 = std::max<int64_t>(1, (int64_t)(grid2 * var.grid_scale + 0.5));
    if (mixed)
        launch_split<KETE_MIXED>(var.split, grid2, 128, st, E, F, cs, stops_dev, n_stops, out, out_stride, aos, kof, ctr, t, unt, leg0, defer->next, q2);
    else
        launch_split<KETE_FP64>(var.split, grid2, 128, st, E, F, cs, stops_dev, n_stops, out, out_stride, aos, kof, ctr, t, unt, leg0, defer->next, q2);
    return cudaGetLastError();
}

cudaError_t launch_gather_bodies(const double *st, const double *ep, int64_t n, int64_t m,
                                 double *dst, double *dep, cudaStream_t s)
{
    if (m > 0) k_gather_bodies<<<grid_for(m, 256), 256, 0, s>>>(st, ep, n, m, dst, dep);
    return cudaGetLastError();
}

cudaError_t launch_chain_finish(ChainState cs, double *states, double *epochs, int32_t *status,
                                cudaStream_t st)
{
    (void)states;
    if (cs.n > 0) k_chain_finish<<<grid_for(cs.n, 256), 256, 0, st>>>(cs, epochs, status);
    return cudaGetLastError();
}

}  // namespace kete
