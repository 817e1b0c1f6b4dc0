// kete_device.cuh -- device-side building blocks of the survey path.
//
// Ephemeris lookup (Sec. 3.2 / App. A), force model (Eq. A.1 with the GR term
// of Eq. A.3 and the J2 term of Eq. A.4), Gauss-Radau 15th-order step with
// IAS15 corrector convergence and step control, predictor removed (App. A.6),
// universal-variable two-body propagation and light-delay correction (Sec. 2),
// spherical-polygon test (Sec. 3.1).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "kete_impl.h"

namespace kete {

// ---------------------------------------------------------------------------
// constants (the physical ones, App. A.1 units, in kete_impl.h)
// ---------------------------------------------------------------------------
constexpr double kPi = 3.14159265358979323846;
constexpr double kTwoPi = 6.28318530717958647692;

// Gauss-Radau spacings (Everhart 1985), h_0 = 0
struct RadauTables {
    double h[8];
    double rinv[8][8];   // 1 / (h_n - h_k), k < n
    double c[8][7];      // c[n][m]: d b_m / d g_n  (Newton -> power basis)
    double w7[8];        // 1 / prod_{k != n} (h_n - h_k): b6 = g7 = sum_n w7[n] F_n
    double wx[8][7];     // h_n^(k+1) / ((k+2)(k+3)): weight of b_k in x at node n
    double wv[8][7];     // h_n^(k+1) / (k+2): weight of b_k in v at node n
    // FP32 copies for the mixed-precision node velocity (it feeds only FP32
    // terms there; an FP64 -> FP32 conversion costs an FP64 issue slot)
    float cf[8][7], wvf[8][7];
};

// ---------------------------------------------------------------------------
// Ephemeris: uniform segments, Clenshaw summation
// ---------------------------------------------------------------------------
struct Seg {
    int s;
    double tau;
};

// Segment and Chebyshev argument at the epoch t0 + off.  tau is formed as
// 2((t0 - t_mid) + off)/L so that a small offset (a substep, a light-time
// interval) is never rounded to the resolution of an absolute Julian date.
__device__ __forceinline__ bool ephem_seg(const EphemDev &E, double t0, double off, Seg &g)
{
    const double t = t0 + off;
    if (!(t >= E.t_start && t <= E.t_end)) return false;
    int s = (int)floor((t - E.t_start) * E.inv_seg);
    s = s < 0 ? 0 : (s > E.n_seg - 1 ? E.n_seg - 1 : s);
    double t_mid = E.t_start + ((double)s + 0.5) * E.seg_len;
    g.s = s;
    g.tau = 2.0 * ((t0 - t_mid) + off) * E.inv_seg;
    return true;
}

// Position of one body, sum_k c_k T_k(tau), summed upward with T_k generated
// on the fly (T_{k+1} = 2 tau T_k - T_{k-1}): one recurrence step shared by
// the three coordinates, then one FMA per coordinate -- 4 FP64 operations per
// coefficient for the three, against 6 for Clenshaw's recurrence.  On
// |tau| <= 1 the recurrence is stable (|T_k| <= 1) and 12 terms keep the sum
// within a few ulps of the position.
__device__ __forceinline__ void cheb_pos(const double *__restrict__ c, int nc, double tau,
                                         double p[3])
{
    const double t2 = 2.0 * tau;
    double Tm1 = 1.0, T = tau;   // T_0, T_1
#pragma unroll
    for (int d = 0; d < 3; d++) p[d] = fma(__ldg(c + d * nc + 1), tau, __ldg(c + d * nc));
    for (int k = 2; k < nc; k++) {
        const double Tn = fma(t2, T, -Tm1);
        Tm1 = T;
        T = Tn;
#pragma unroll
        for (int d = 0; d < 3; d++) p[d] = fma(__ldg(c + d * nc + k), T, p[d]);
    }
}

// Position and velocity: as cheb_pos, plus sum_k c_k T_k'(tau) dtau/dt with
// T_k' = k U_{k-1}, U_{j+1} = 2 tau U_j - U_{j-1} (U_0 = 1, U_1 = 2 tau).
__device__ __forceinline__ void cheb_pos_vel(const double *__restrict__ c, int nc, double tau,
                                             double dtau_dt, double p[3], double v[3])
{
    const double t2 = 2.0 * tau;
    double Tm1 = 1.0, T = tau;   // T_0, T_1
    double Um1 = 1.0, U = t2;    // U_0, U_1
#pragma unroll
    for (int d = 0; d < 3; d++) {
        const double c1 = __ldg(c + d * nc + 1);
        p[d] = fma(c1, tau, __ldg(c + d * nc));
        v[d] = c1;               // T_1' = 1
    }
    for (int k = 2; k < nc; k++) {
        const double Tn = fma(t2, T, -Tm1);
        Tm1 = T;
        T = Tn;
        const double dk = (double)k * U;   // T_k' = k U_{k-1}
#pragma unroll
        for (int d = 0; d < 3; d++) {
            const double ck = __ldg(c + d * nc + k);
            p[d] = fma(ck, T, p[d]);
            v[d] = fma(ck, dk, v[d]);
        }
        const double Un = fma(t2, U, -Um1);
        Um1 = U;
        U = Un;
    }
#pragma unroll
    for (int d = 0; d < 3; d++) v[d] *= dtau_dt;
}

__device__ __forceinline__ const double *ephem_coef(const EphemDev &E, int body, int s)
{
    return E.coef + ((size_t)body * E.n_seg + s) * 3 * E.n_coef;
}

// ---------------------------------------------------------------------------
// Lane groups: G consecutive lanes (G a power of two, <= 32) integrating one
// body together.  Every lane of a group holds the same integrator state and
// runs the same control flow; in a force evaluation lane `rank` takes the
// masses m = rank, rank + G, ... and the partial sums are combined by a
// butterfly of shuffles, which leaves the same bits in every lane (each pair
// adds the same two values).  G = 1 is the plain one-lane-per-body form.
// ---------------------------------------------------------------------------
template <int G>
struct LaneGroup {
    static_assert(G == 1 || G == 2 || G == 4 || G == 8 || G == 16 || G == 32, "G");
    __device__ __forceinline__ static int rank() { return G == 1 ? 0 : (int)(threadIdx.x & (G - 1)); }
    __device__ __forceinline__ static unsigned mask()
    {
        if (G == 32) return 0xffffffffu;
        return ((1u << G) - 1u) << ((threadIdx.x & 31) & ~(unsigned)(G - 1));
    }
    template <typename T>
    __device__ __forceinline__ static T sum(T v)
    {
#pragma unroll
        for (int o = G / 2; o >= 1; o /= 2) v += __shfl_xor_sync(mask(), v, o);
        return v;
    }
    __device__ __forceinline__ static uint32_t bit_or(uint32_t v)
    {
#pragma unroll
        for (int o = G / 2; o >= 1; o /= 2) v |= __shfl_xor_sync(mask(), v, o);
        return v;
    }
};

// ---------------------------------------------------------------------------
// Force model (Eq. A.1): for each active mass m with r = x - x_m, v = v - v_m:
//   Newton  -mu r / |r|^3
//   GR      mu / (c^2 |r|^3) [ (4 mu/|r| - |v|^2) r + 4 (r.v) v ]       (Eq. A.3)
//   J2      -(3/2) J2 mu R^2 / |r|^5 [ (1 - 5 z^2/|r|^2) r + 2 z p ]     (Eq. A.4,
//           z = r.p with p the body's pole; the same vector written in the
//           body's equatorial frame is the component form of Eq. A.4)
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T rsqrt_t(T x);
template <>
__device__ __forceinline__ double rsqrt_t<double>(double x) { return rsqrt(x); }
template <>
__device__ __forceinline__ float rsqrt_t<float>(float x) { return rsqrtf(x); }

// The constants of one mass (mu = GM; the GR and J2 factors from ForceDev).
template <typename T>
struct MassK {
    T mu, mu4, grk, gr4k, j2k;   // mu, 4 mu, mu / c^2, 4 mu / c^2, 1.5 J2 mu R^2
    const T *P, *Pm2;            // unit pole, -2 x the pole
};
__device__ __forceinline__ MassK<double> mass_k64(const EphemDev &E, const ForceDev &F, int m)
{
    return MassK<double>{E.gm[m], F.gm4[m], F.grk[m], F.gr4k[m], F.j2k[m], F.pole[m], F.pole_m2[m]};
}
__device__ __forceinline__ MassK<float> mass_k32(const ForceDev &F, int m)
{
    return MassK<float>{F.gm32[m], F.gm4_32[m], F.grk32[m], F.gr4k32[m], F.j2k32[m], F.pole32[m],
                        F.pole_m2_32[m]};
}

// the three terms of one mass, accumulated into a[]; w = relative velocity
template <typename T>
__device__ __forceinline__ void mass_terms(const MassK<T> &K, bool newton, bool gr, bool j2,
                                           const T r[3], const T w[3], T a[3])
{
    T rr = fma(r[0], r[0], fma(r[1], r[1], r[2] * r[2]));
    T ri = rsqrt_t<T>(rr);
    T ri2 = ri * ri;
    T ri3 = ri2 * ri;
    T f = newton ? -K.mu * ri3 : (T)0;
    if (gr) {
        T ww = fma(w[0], w[0], fma(w[1], w[1], w[2] * w[2]));
        T rw = fma(r[0], w[0], fma(r[1], w[1], r[2] * w[2]));
        T k = K.grk * ri3;                     // mu / (c^2 r^3)
        f = fma(k, fma(K.mu4, ri, -ww), f);
        T fw = (K.gr4k * ri3) * rw;            // 4 k (r.v)
        a[0] = fma(fw, w[0], a[0]);
        a[1] = fma(fw, w[1], a[1]);
        a[2] = fma(fw, w[2], a[2]);
    }
    if (j2) {
        const T *P = K.P;
        T z = fma(r[0], P[0], fma(r[1], P[1], r[2] * P[2]));
        T psi = K.j2k * ri3 * ri2;   // 1.5 J2 mu R^2 / r^5
        T q = z * z * ri2;           // (z / r)^2
        f = fma(-psi, fma((T)-5, q, (T)1), f);
        T fp = psi * z;              // along -2 P
        a[0] = fma(fp, K.Pm2[0], a[0]);
        a[1] = fma(fp, K.Pm2[1], a[1]);
        a[2] = fma(fp, K.Pm2[2], a[2]);
    }
    a[0] = fma(f, r[0], a[0]);
    a[1] = fma(f, r[1], a[1]);
    a[2] = fma(f, r[2], a[2]);
}

// Planet state of body m by Chebyshev sums: the per-thread path used when a
// step does not span a whole batch leg.  vel: also the velocity (the GR term of
// Eq. A.3 is the only one that needs it); otherwise out6[3..5] are left unset.
// The sums run out of line and return the state by value (in registers): an
// out-of-line routine writing through a pointer sent the state through the
// stack (local memory) at every call, and the state comes back 8-12 % faster
// this way on the survey and ragged workloads (bit for bit the same).
struct PlanetState {
    double x, y, z, vx, vy, vz;
};
static __device__ __noinline__ PlanetState cheb_state64v(const EphemDev &E, int m, int s, double tau,
                                                         bool vel)
{
    double p[3], v[3] = {0.0, 0.0, 0.0};
    if (vel) cheb_pos_vel(ephem_coef(E, m, s), E.n_coef, tau, 2.0 * E.inv_seg, p, v);
    else cheb_pos(ephem_coef(E, m, s), E.n_coef, tau, p);
    PlanetState o;
    o.x = p[0]; o.y = p[1]; o.z = p[2];
    o.vx = v[0]; o.vy = v[1]; o.vz = v[2];
    return o;
}
__device__ __forceinline__ void cheb_state64(const EphemDev &E, int m, int s, double tau,
                                             double *out6, bool vel = true)
{
    const PlanetState o = cheb_state64v(E, m, s, tau, vel);
    out6[0] = o.x; out6[1] = o.y; out6[2] = o.z;
    if (vel) {
        out6[3] = o.vx; out6[4] = o.vy; out6[5] = o.vz;
    }
}

// The Chebyshev basis at tau, shared by every body of one evaluation: T_k(tau)
// and k U_{k-1}(tau) (T_k' = k U_{k-1}), from the recurrences of cheb_pos /
// cheb_pos_vel in the same order, so that cheb_state64b's sums are bit for bit
// theirs.  The per-body recurrence steps (1 FP64 FMA per coefficient for the
// position, 3 for the velocity) are done once instead of for every body; the
// basis is read back from shared memory (load slots, not FP64 ones; no DRAM),
// one column per thread: element k of a thread's basis at T[k * kBasisLanes].
constexpr int kBasisMax = 16;     // coefficients a table may have for the shared basis
constexpr int kBasisLanes = 128;  // threads per block it serves
struct ChebBasis {
    double *T, *dT;   // this thread's columns
};

__device__ __forceinline__ void cheb_basis(int nc, double tau, bool vel, ChebBasis B)
{
    const double t2 = 2.0 * tau;
    double Tm1 = 1.0, T = tau;   // T_0, T_1
    double Um1 = 1.0, U = t2;    // U_0, U_1
    B.T[0] = 1.0;
    B.T[kBasisLanes] = tau;
    B.dT[kBasisLanes] = 1.0;
    for (int k = 2; k < nc; k++) {
        const double Tn = fma(t2, T, -Tm1);
        Tm1 = T;
        T = Tn;
        B.T[k * kBasisLanes] = T;
        if (vel) {
            B.dT[k * kBasisLanes] = (double)k * U;
            const double Un = fma(t2, U, -Um1);
            Um1 = U;
            U = Un;
        }
    }
}

// Planet state of body m from a shared basis (see cheb_basis): the sums of
// cheb_pos / cheb_pos_vel with the basis read instead of recomputed.
static __device__ __noinline__ PlanetState cheb_state64b(const EphemDev &E, int m, int s,
                                                         ChebBasis B, bool vel)
{
    const double *__restrict__ c = ephem_coef(E, m, s);
    const int nc = E.n_coef;
    double p[3], v[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int d = 0; d < 3; d++) {
        const double c1 = __ldg(c + d * nc + 1);
        p[d] = fma(c1, B.T[kBasisLanes], __ldg(c + d * nc));
        v[d] = c1;
    }
    if (vel) {
        for (int k = 2; k < nc; k++) {
            const double Tk = B.T[k * kBasisLanes], dk = B.dT[k * kBasisLanes];
#pragma unroll
            for (int d = 0; d < 3; d++) {
                const double ck = __ldg(c + d * nc + k);
                p[d] = fma(ck, Tk, p[d]);
                v[d] = fma(ck, dk, v[d]);
            }
        }
        const double dtau_dt = 2.0 * E.inv_seg;
#pragma unroll
        for (int d = 0; d < 3; d++) v[d] *= dtau_dt;
    } else {
        for (int k = 2; k < nc; k++) {
            const double Tk = B.T[k * kBasisLanes];
#pragma unroll
            for (int d = 0; d < 3; d++) p[d] = fma(__ldg(c + d * nc + k), Tk, p[d]);
        }
    }
    PlanetState o;
    o.x = p[0]; o.y = p[1]; o.z = p[2];
    o.vx = v[0]; o.vy = v[1]; o.vz = v[2];
    return o;
}

// FP32 Clenshaw of body m (mixed precision, planets only), the recurrences
// interleaved; vel as in cheb_state64
__device__ __forceinline__ void cheb_state32(const EphemDev &E, int m, int s, float tau,
                                             float *out6, bool vel = true)
{
    const float *c = E.coef32 + ((size_t)m * E.n_seg + s) * 3 * E.n_coef;
    const int nc = E.n_coef;
    const float dtau_dt = (float)(2.0 * E.inv_seg);
    const float t2 = 2.f * tau;
    float b1[3] = {0.f, 0.f, 0.f}, b2[3] = {0.f, 0.f, 0.f};
    float u1[3] = {0.f, 0.f, 0.f}, u2[3] = {0.f, 0.f, 0.f};
    if (vel) {
        for (int k = nc - 1; k >= 1; k--) {
            const float kk = (float)k;
#pragma unroll
            for (int d = 0; d < 3; d++) {
                const float ck = __ldg(c + d * nc + k);
                const float b0 = fmaf(t2, b1[d], ck - b2[d]);
                const float u0 = fmaf(t2, u1[d], kk * ck - u2[d]);
                b2[d] = b1[d]; b1[d] = b0; u2[d] = u1[d]; u1[d] = u0;
            }
        }
    } else {
        for (int k = nc - 1; k >= 1; k--) {
#pragma unroll
            for (int d = 0; d < 3; d++) {
                const float b0 = fmaf(t2, b1[d], __ldg(c + d * nc + k) - b2[d]);
                b2[d] = b1[d]; b1[d] = b0;
            }
        }
    }
#pragma unroll
    for (int d = 0; d < 3; d++) {
        out6[d] = fmaf(tau, b1[d], __ldg(c + d * nc) - b2[d]);
        if (vel) out6[3 + d] = u1[d] * dtau_dt;
    }
}

// p(t0 + off) - p(t0) of body m from the segment holding t0: Chebyshev
// differences D_k = T_k(tau1) - T_k(tau0) by D_{k+1} = 2 tau1 D_k - D_{k-1} +
// 2 (tau1 - tau0) T_k(tau0), so a small planet displacement is not the
// difference of two rounded ~1 AU positions (close-encounter path).
static __device__ __noinline__ void cheb_delta64(const EphemDev &E, int m, double t0, double off,
                                                 double *dp)
{
    int s = (int)floor((t0 - E.t_start) * E.inv_seg);
    s = s < 0 ? 0 : (s > E.n_seg - 1 ? E.n_seg - 1 : s);
    const double t_mid = E.t_start + ((double)s + 0.5) * E.seg_len;
    const double tau0 = 2.0 * (t0 - t_mid) * E.inv_seg;
    const double dtau = 2.0 * off * E.inv_seg;
    const double tau1 = tau0 + dtau;
    const double *c = ephem_coef(E, m, s);
    double acc[3] = {0.0, 0.0, 0.0};
    double Tm1 = 1.0, T = tau0;          // T_{k-1}(tau0), T_k(tau0)
    double Dm1 = 0.0, D = dtau;          // D_{k-1}, D_k
    for (int k = 1; k < E.n_coef; k++) {
#pragma unroll
        for (int d = 0; d < 3; d++) acc[d] = fma(__ldg(c + d * E.n_coef + k), D, acc[d]);
        const double Dn = fma(2.0 * tau1, D, fma(2.0 * dtau, T, -Dm1));
        const double Tn = fma(2.0 * tau0, T, -Tm1);
        Dm1 = D; D = Dn;
        Tm1 = T; T = Tn;
    }
    dp[0] = acc[0]; dp[1] = acc[1]; dp[2] = acc[2];
}

// Close encounter: the nearest planet within kEncounterAu of the body at the
// step start.  At a substep its relative position is d0 + (dx - dp(off)).
constexpr double kEncounterAu = 0.1;
struct Encounter {
    int m;            // table body, -1: none
    double t0;        // step start
    double d0[3];     // x0 - p_m(t0)
};

// the group's nearest candidate (ties to the lower table index, as the
// one-lane loop over m in order)
template <int G>
__device__ __forceinline__ void encounter_reduce(double &best, Encounter &enc)
{
#pragma unroll
    for (int o = G / 2; o >= 1; o /= 2) {
        const unsigned gm = LaneGroup<G>::mask();
        const double ob = __shfl_xor_sync(gm, best, o);
        const int om = __shfl_xor_sync(gm, enc.m, o);
        double od[3];
#pragma unroll
        for (int c = 0; c < 3; c++) od[c] = __shfl_xor_sync(gm, enc.d0[c], o);
        if (ob < best || (ob == best && om < enc.m)) {
            best = ob;
            enc.m = om;
#pragma unroll
            for (int c = 0; c < 3; c++) enc.d0[c] = od[c];
        }
    }
}

// Node rows: planet states at one Gauss-Radau node epoch of a batch leg,
// shared by every body whose step spans that whole leg.
//   row64[m*6 + 0..5]  barycentric position, velocity (FP64)
//   row32[m*6 + 0..2]  position relative to the Sun, [3..5] velocity (FP32)
// A null row64 means "evaluate the table here" (per-thread path).

// Newtonian part of da/dx for one mass, accumulated into the symmetric J
// (xx, xy, xz, yy, yz, zz):  -mu/|r|^3 (I - 3 r r^T / |r|^2).
__device__ __forceinline__ void newton_jacobian(double mu, const double r[3], double J[6])
{
    const double rr = fma(r[0], r[0], fma(r[1], r[1], r[2] * r[2]));
    const double ri = rsqrt(rr);
    const double ri2 = ri * ri;
    const double f = -mu * ri2 * ri;
    const double k = -3.0 * f * ri2;
    J[0] = fma(k * r[0], r[0], J[0] + f);
    J[1] = fma(k * r[0], r[1], J[1]);
    J[2] = fma(k * r[0], r[2], J[2]);
    J[3] = fma(k * r[1], r[1], J[3] + f);
    J[4] = fma(k * r[1], r[2], J[4]);
    J[5] = fma(k * r[2], r[2], J[5] + f);
}

// Non-gravitational terms of one body (App. A.4-A.5), defined with the
// two-body solver below; returned by value so that no caller array needs an
// address.  Only bodies with kete_nongrav parameters make the call.
struct NgOut {
    double a[3];
    int status;
    double chi;   // the thermal lag's two-body solution (universal anomaly), for the next call
};
static __device__ __noinline__ NgOut nongrav_terms(const EphemDev &E, const double *row64, Seg g,
                                                   const kete_nongrav *P, double x0, double x1,
                                                   double x2, double v0, double v1, double v2,
                                                   double chi0);

// Lane groups (G > 1): the body's non-gravitational terms (ng may be null)
// computed by the group's last lane -- the one that holds the fewest masses
// -- and added to its partial sum acc before the group sum; every lane of
// the group returns the same status.
template <int G>
__device__ __forceinline__ int group_nongrav(const EphemDev &E, const double *row64, Seg g,
                                             const kete_nongrav *ng, const double x[3],
                                             const double v[3], double acc[3], double *ng_chi)
{
    if (!ng) return KETE_BODY_OK;
    int st = KETE_BODY_OK;
    if (LaneGroup<G>::rank() == G - 1) {
        const NgOut o = nongrav_terms(E, row64, g, ng, x[0], x[1], x[2], v[0], v[1], v[2],
                                      ng_chi ? *ng_chi : 0.0);
        if (ng_chi) *ng_chi = o.chi;
        st = o.status;
        acc[0] += o.a[0];
        acc[1] += o.a[1];
        acc[2] += o.a[2];
    }
    return __shfl_sync(LaneGroup<G>::mask(), st, G - 1, G);
}

// Full-FP64 acceleration.
// detect (step start, off = 0): also record in enc the nearest planet within
// kEncounterAu and its relative position; otherwise enc is read.
// JAC: also return in J the Newtonian da/dx (see newton_jacobian), from the
// same relative vectors as the force.  G: lanes per body (see LaneGroup).
// ng: the body's non-gravitational terms (null: none), added after the sum.
template <bool JAC = false, int G = 1>
__device__ __forceinline__ int accel_fp64(const EphemDev &E, const ForceDev &F, double t0,
                                          double off, const double *__restrict__ row64,
                                          const double x[3], const double v[3], double a[3],
                                          Encounter &enc, const double dx[3], bool detect,
                                          double *J = nullptr, const kete_nongrav *ng = nullptr,
                                          double *ng_chi = nullptr)
{
    Seg g = {0, 0.0};
    a[0] = a[1] = a[2] = 0.0;
    if (JAC) {
#pragma unroll
        for (int q = 0; q < 6; q++) J[q] = 0.0;
    }
    if (detect) {
        enc.m = -1;
        enc.t0 = t0;
    }
    double best = kEncounterAu * kEncounterAu;
    if (!row64 && !ephem_seg(E, t0, off, g)) return KETE_BODY_OUT_OF_SPAN;
    // per-thread ephemeris: one Chebyshev basis for all the bodies, in shared
    // memory (a column per thread)
    __shared__ double s_basis[2 * kBasisMax * kBasisLanes];
    ChebBasis basis;
    basis.T = s_basis + threadIdx.x;
    basis.dT = s_basis + kBasisMax * kBasisLanes + threadIdx.x;
    const bool use_basis = !row64 && E.n_coef <= kBasisMax && threadIdx.x < kBasisLanes &&
                           blockDim.x <= kBasisLanes;
    if (use_basis) cheb_basis(E.n_coef, g.tau, (F.gr_mask & F.active_mask) != 0u, basis);
    for (int m = LaneGroup<G>::rank(); m < E.n_bodies; m += G) {
        if (!((F.active_mask >> m) & 1u)) continue;
        const bool gr = (F.gr_mask >> m) & 1u, j2 = (F.j2_mask >> m) & 1u;
        double st[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        if (row64) {
            // velocities only where the GR term needs them
#pragma unroll
            for (int q = 0; q < 3; q++) st[q] = __ldg(row64 + 6 * m + q);
            if (gr) {
#pragma unroll
                for (int q = 3; q < 6; q++) st[q] = __ldg(row64 + 6 * m + q);
            }
        } else if (use_basis) {
            const PlanetState o = cheb_state64b(E, m, g.s, basis, gr);
            st[0] = o.x; st[1] = o.y; st[2] = o.z;
            st[3] = o.vx; st[4] = o.vy; st[5] = o.vz;
        } else {
            cheb_state64(E, m, g.s, g.tau, st, gr);
        }
        double r[3] = {x[0] - st[0], x[1] - st[1], x[2] - st[2]};
        if (detect) {
            const double rr = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
            if (m > 0 && rr < best) {
                best = rr;
                enc.m = m;
                enc.d0[0] = r[0]; enc.d0[1] = r[1]; enc.d0[2] = r[2];
            }
        } else if (m == enc.m) {
            double dp[3];
            cheb_delta64(E, m, enc.t0, off, dp);
            r[0] = enc.d0[0] + (dx[0] - dp[0]);
            r[1] = enc.d0[1] + (dx[1] - dp[1]);
            r[2] = enc.d0[2] + (dx[2] - dp[2]);
        }
        double w[3] = {0.0, 0.0, 0.0};
        if (gr) {
            w[0] = v[0] - st[3];
            w[1] = v[1] - st[4];
            w[2] = v[2] - st[5];
        }
        mass_terms<double>(mass_k64(E, F, m), true, gr, j2, r, w, a);
        if (JAC) newton_jacobian(E.gm[m], r, J);
    }
    if (G > 1) {
        // the body's own terms go to the group's last lane, which holds the
        // fewest masses, and join the group sum (a lagged comet term costs a
        // two-body solve: done once per group, beside the others' masses)
        const int ng_status = group_nongrav<G>(E, row64, g, ng, x, v, a, ng_chi);
#pragma unroll
        for (int c = 0; c < 3; c++) a[c] = LaneGroup<G>::sum(a[c]);
        if (JAC) {
#pragma unroll
            for (int q = 0; q < 6; q++) J[q] = LaneGroup<G>::sum(J[q]);
        }
        if (detect) encounter_reduce<G>(best, enc);
        return ng_status;
    }
    if (ng) {
        const NgOut o = nongrav_terms(E, row64, g, ng, x[0], x[1], x[2], v[0], v[1], v[2],
                                      ng_chi ? *ng_chi : 0.0);
        if (ng_chi) *ng_chi = o.chi;
        if (o.status != KETE_BODY_OK) return o.status;
        a[0] += o.a[0];
        a[1] += o.a[1];
        a[2] += o.a[2];
    }
    return KETE_BODY_OK;
}

// Mixed precision (FP32 planets): the Sun's monopole in FP64; the Sun's GR and
// J2 and every planet in FP32 -- except planets flagged in `close` (within
// 2 kCloseAu at the start of the step), which stay in FP64.  `as` receives the
// FP64 part alone: it is smooth in time, so the step-size control estimates
// its error from it (FP32 rounding noise would otherwise dominate b6).  The
// FP32 planet-relative vector carries ~6e-8 AU of rounding (the body's ~1 AU
// Sun-relative position in FP32), a relative force error of ~2e-7 AU / d at
// distance d; before a 0.001-0.01 AU pass that noise is amplified by 1/Delta
// in the sky, so planets stay FP64 out to 0.2 AU.
constexpr double kCloseAu = 0.1;

// detect (step start, off = 0): planets within 2 kCloseAu go to FP64 and are
// recorded in `close` (held for the step), and the nearest within kEncounterAu
// in enc; otherwise close and enc are read.  G: lanes per body (LaneGroup);
// the Sun's terms belong to rank 0, every lane forms the Sun-relative position.
template <int G = 1>
__device__ __forceinline__ int accel_mixed(const EphemDev &E, const ForceDev &F, double t0,
                                           double off, const double *__restrict__ row64,
                                           const float *__restrict__ row32, uint32_t &close,
                                           const double x[3], const double v[3], double a[3],
                                           double as[3], Encounter &enc, const double dx[3],
                                           bool detect, const kete_nongrav *ng = nullptr,
                                           const float *vf_in = nullptr, double *ng_chi = nullptr)
{
    Seg g = {0, 0.0};
    as[0] = as[1] = as[2] = 0.0;
    if (detect) {
        close = 0;
        enc.m = -1;
        enc.t0 = t0;
    }
    double best = kEncounterAu * kEncounterAu;
    if (!row64 && !ephem_seg(E, t0, off, g)) return KETE_BODY_OUT_OF_SPAN;
    // the Sun: position in FP64 (the monopole); its velocity enters only the
    // FP32 GR term, so per thread it comes from the FP32 series
    double sun[3];
    float sunv[3] = {0.f, 0.f, 0.f};
    const bool sun_gr = F.gr_mask & 1u;
    if (row64) {
#pragma unroll
        for (int q = 0; q < 3; q++) sun[q] = __ldg(row64 + q);
        if (sun_gr) {   // the FP32 row holds the same velocity, already rounded
#pragma unroll
            for (int q = 0; q < 3; q++) sunv[q] = row32 ? __ldg(row32 + 3 + q) : (float)__ldg(row64 + 3 + q);
        }
    } else {
        cheb_state64(E, 0, g.s, g.tau, sun, false);
        if (sun_gr) {
            float s6[6];
            cheb_state32(E, 0, g.s, (float)g.tau, s6, true);
            sunv[0] = s6[3]; sunv[1] = s6[4]; sunv[2] = s6[5];
        }
    }
    const double d[3] = {x[0] - sun[0], x[1] - sun[1], x[2] - sun[2]};
    const float df[3] = {(float)d[0], (float)d[1], (float)d[2]};
    // the body's velocity enters only FP32 terms: taken in FP32 when the
    // caller has it (vf_in), else rounded here
    float vf[3];
#pragma unroll
    for (int c = 0; c < 3; c++) vf[c] = vf_in ? vf_in[c] : (float)v[c];
    float af[3] = {0.f, 0.f, 0.f};
    const int rk = LaneGroup<G>::rank();
    if (rk == 0 && (F.active_mask & 1u)) {
        // Sun monopole, FP64
        double rr = fma(d[0], d[0], fma(d[1], d[1], d[2] * d[2]));
        double ri = rsqrt(rr);
        double f = -E.gm[0] * ri * ri * ri;
        as[0] = f * d[0];
        as[1] = f * d[1];
        as[2] = f * d[2];
        // the Sun's GR and J2 corrections, FP32 (relative size 1e-8, 1e-13)
        const bool j2 = F.j2_mask & 1u;
        if (sun_gr || j2) {
            float w[3] = {vf[0] - sunv[0], vf[1] - sunv[1], vf[2] - sunv[2]};
            mass_terms<float>(mass_k32(F, 0), false, sun_gr, j2, df, w, af);
        }
    }
    // the Sun in FP32 only for the per-thread planet series (node rows are
    // already Sun-relative)
    float sunf[3] = {0.f, 0.f, 0.f};
    if (!row32) {
#pragma unroll
        for (int q = 0; q < 3; q++) sunf[q] = (float)sun[q];
    }
    const float tau32 = row64 ? 0.f : (float)g.tau;
    for (int m = (rk == 0 ? G : rk); m < E.n_bodies; m += G) {
        if (!((F.active_mask >> m) & 1u)) continue;
        const bool gr = (F.gr_mask >> m) & 1u, j2 = (F.j2_mask >> m) & 1u;
        float st[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (row32) {
#pragma unroll
            for (int q = 0; q < 3; q++) st[q] = __ldg(row32 + 6 * m + q);
            if (gr) {
#pragma unroll
                for (int q = 3; q < 6; q++) st[q] = __ldg(row32 + 6 * m + q);
            }
        } else {
            cheb_state32(E, m, g.s, tau32, st, gr);
            st[0] -= sunf[0]; st[1] -= sunf[1]; st[2] -= sunf[2];
        }
        float r[3] = {df[0] - st[0], df[1] - st[1], df[2] - st[2]};
        if (detect && r[0] * r[0] + r[1] * r[1] + r[2] * r[2] < (float)(4.0 * kCloseAu * kCloseAu))
            close |= 1u << m;
        if ((close >> m) & 1u) {
            double s64[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
            if (row64) {
#pragma unroll
                for (int q = 0; q < 6; q++) s64[q] = __ldg(row64 + 6 * m + q);
            } else {
                cheb_state64(E, m, g.s, g.tau, s64, gr);
            }
            double r64[3] = {x[0] - s64[0], x[1] - s64[1], x[2] - s64[2]};
            if (detect) {
                const double rr = r64[0] * r64[0] + r64[1] * r64[1] + r64[2] * r64[2];
                if (rr < best) {
                    best = rr;
                    enc.m = m;
                    enc.d0[0] = r64[0]; enc.d0[1] = r64[1]; enc.d0[2] = r64[2];
                }
            } else if (m == enc.m) {
                double dp[3];
                cheb_delta64(E, m, enc.t0, off, dp);
                r64[0] = enc.d0[0] + (dx[0] - dp[0]);
                r64[1] = enc.d0[1] + (dx[1] - dp[1]);
                r64[2] = enc.d0[2] + (dx[2] - dp[2]);
            }
            // (the body's velocity as the FP32 terms see it when it came in FP32:
            // it enters only the GR term, 1e-8 of the planet's pull)
            double w[3];
#pragma unroll
            for (int c = 0; c < 3; c++) w[c] = (vf_in ? (double)vf[c] : v[c]) - s64[3 + c];
            mass_terms<double>(mass_k64(E, F, m), true, gr, j2, r64, w, as);
            continue;
        }
        float w[3] = {vf[0] - st[3], vf[1] - st[4], vf[2] - st[5]};
        mass_terms<float>(mass_k32(F, m), true, gr, j2, r, w, af);
    }
    int ng_status = KETE_BODY_OK;
    if (G > 1) {
        ng_status = group_nongrav<G>(E, row64, g, ng, x, v, as, ng_chi);   // FP64, smooth part
#pragma unroll
        for (int c = 0; c < 3; c++) {
            as[c] = LaneGroup<G>::sum(as[c]);
            af[c] = LaneGroup<G>::sum(af[c]);
        }
        if (detect) {
            close = LaneGroup<G>::bit_or(close);
            encounter_reduce<G>(best, enc);
        }
        if (ng_status != KETE_BODY_OK) return ng_status;
    } else if (ng) {   // FP64, part of the smooth FP64 sum that controls the step
        const NgOut o = nongrav_terms(E, row64, g, ng, x[0], x[1], x[2], v[0], v[1], v[2],
                                      ng_chi ? *ng_chi : 0.0);
        if (ng_chi) *ng_chi = o.chi;
        if (o.status != KETE_BODY_OK) return o.status;
        as[0] += o.a[0];
        as[1] += o.a[1];
        as[2] += o.a[2];
    }
    a[0] = as[0] + (double)af[0];
    a[1] = as[1] + (double)af[1];
    a[2] = as[2] + (double)af[2];
    return KETE_BODY_OK;
}

// ---------------------------------------------------------------------------
// universal-variable two-body propagation
// ---------------------------------------------------------------------------
// Stumpff C(z), S(z): the power series C = sum_k (-z)^k / (2k+2)!,
// S = sum_k (-z)^k / (2k+3)! by Horner's rule in z (one FMA per term, the
// coefficients folded at compile time) for |z| < 1 (seven terms when
// |z| < 1e-3: the first omitted one is below 1e-34; twelve otherwise: below
// 3e-27), closed trigonometric / hyperbolic forms beyond.
__host__ __device__ constexpr double stumpff_c_coef(int k)
{
    double a = 0.5;   // 1 / 2!
    for (int j = 1; j <= k; j++) a = -a / ((2.0 * j + 1.0) * (2.0 * j + 2.0));
    return a;
}
__host__ __device__ constexpr double stumpff_s_coef(int k)
{
    double a = 1.0 / 6.0;   // 1 / 3!
    for (int j = 1; j <= k; j++) a = -a / ((2.0 * j + 2.0) * (2.0 * j + 3.0));
    return a;
}
// c <- c z + a_K, ..., down to a_0
template <int K>
struct StumpffHorner {
    static __device__ __forceinline__ void run(double z, double &c, double &s)
    {
        constexpr double ck = stumpff_c_coef(K), sk = stumpff_s_coef(K);
        c = fma(c, z, ck);
        s = fma(s, z, sk);
        StumpffHorner<K - 1>::run(z, c, s);
    }
};
template <>
struct StumpffHorner<-1> {
    static __device__ __forceinline__ void run(double, double &, double &) {}
};
// terms k = 0 .. K-1
template <int K>
__device__ __forceinline__ void stumpff_series(double z, double &C, double &S)
{
    constexpr double c_top = stumpff_c_coef(K - 1), s_top = stumpff_s_coef(K - 1);
    double c = c_top, s = s_top;
    StumpffHorner<K - 2>::run(z, c, s);
    C = c;
    S = s;
}
__device__ __forceinline__ void stumpff(double z, double &C, double &S)
{
    if (fabs(z) < 1e-3) {
        stumpff_series<7>(z, C, S);
    } else if (fabs(z) < 1.0) {
        stumpff_series<12>(z, C, S);
    } else if (z > 0.0) {
        double q = sqrt(z), sn, cs;
        sincos(q, &sn, &cs);
        C = (1.0 - cs) / z;
        S = (q - sn) / (z * q);
    } else {
        double q = sqrt(-z);
        C = (cosh(q) - 1.0) / (-z);
        S = (sinh(q) - q) / (-z * q);
    }
}

// Heliocentric state (r0, v0) advanced by dt under mu.  chi is the universal
// anomaly: in = initial guess (0 = none), out = solution (warm start).
// Without a guess, chi starts from its Taylor series in dt (dchi/dt =
// sqrt(mu)/|r|): sqrt(mu) [dt/r0 - rdot dt^2/(2 r0^2) + (2 rdot^2 - r0 rddot)
// dt^3/(6 r0^3)], rdot = r0.v0/r0, rddot = (v0^2 - rdot^2)/r0 - mu/r0^2, while
// sqrt(mu/r0^3) |dt| < 0.2 (a few ulps off for the FoV stage's day-long
// intervals: Newton then needs two iterations); beyond that from dt/r0.
// Newton's iteration on F(chi) = A chi^2 C + B chi^3 S + r0 chi - sqrt(mu) dt
// has converged when its step falls below 1e-15 |chi| or below the rounding
// of F itself (4 ulps of the sum of its terms' magnitudes, divided by F'):
// where the terms cancel (perihelion passages, short intervals) the step
// settles into an oscillation of a few ulps of F / F' that a relative test
// alone never accepts.  Returns false if Newton's iteration did not converge.
__device__ __forceinline__ bool kepler_uv(double mu, double sqmu, const double r0[3],
                                          const double v0[3], double dt, double &chi,
                                          double r[3], double v[3])
{
    // reciprocals taken once: FP64 division and square root are
    // multi-instruction sequences (|r0| from its reciprocal square root)
    const double rr0 = fma(r0[0], r0[0], fma(r0[1], r0[1], r0[2] * r0[2]));
    const double ri = rsqrt(rr0), isqmu = 1.0 / sqmu;
    const double rn0 = rr0 * ri;
    double vv = fma(v0[0], v0[0], fma(v0[1], v0[1], v0[2] * v0[2]));
    double rv = fma(r0[0], v0[0], fma(r0[1], v0[1], r0[2] * v0[2]));
    double alpha = fma(-vv * isqmu, isqmu, 2.0 * ri);
    double A = rv * isqmu;
    double B = 1.0 - alpha * rn0;
    double target = sqmu * dt;
    if (chi == 0.0) {
        chi = target * ri;
        if (fabs(dt) * sqmu * ri * sqrt(ri) < 0.2) {
            const double rd = rv * ri;
            const double rdd = (vv - rd * rd) * ri - mu * ri * ri;
            const double u = dt * ri;
            chi *= fma(fma(2.0 * rd * rd - rn0 * rdd, u * (1.0 / 6.0), -0.5 * rd), u, 1.0);
        }
    }
    double C = 0.5, S = 1.0 / 6.0, z = 0.0;
    bool ok = false;
    for (int it = 0; it < 64; it++) {
        double x2 = chi * chi;
        z = alpha * x2;
        stumpff(z, C, S);
        const double t1 = A * x2, t2 = B * x2 * chi;
        double Fv = fma(t1, C, fma(t2, S, fma(rn0, chi, -target)));
        double dF = fma(A * chi, fma(-z, S, 1.0), fma(B * x2, C, rn0));
        double step = Fv / dF;
        const double floor_f = 8.881784197001252e-16 *   // 4 ulps of 1
                               (fabs(t1 * C) + fabs(t2 * S) + fabs(rn0 * chi) + fabs(target));
        // keep the iterate on the solution's side of zero and bounded in growth
        double nxt = chi - step;
        if ((nxt > 0.0) != (dt > 0.0) && dt != 0.0) nxt = 0.5 * chi;
        chi = nxt;
        if (fabs(step) <= 1e-15 * fabs(chi) || fabs(step) * fabs(dF) <= floor_f || Fv == 0.0) {
            ok = true;
            break;
        }
    }
    double x2 = chi * chi;
    z = alpha * x2;
    stumpff(z, C, S);
    double f = 1.0 - x2 * ri * C;
    double gg = dt - x2 * chi * S * isqmu;
    r[0] = fma(f, r0[0], gg * v0[0]);
    r[1] = fma(f, r0[1], gg * v0[1]);
    r[2] = fma(f, r0[2], gg * v0[2]);
    const double rin = rsqrt(fma(r[0], r[0], fma(r[1], r[1], r[2] * r[2])));
    double fd = sqmu * rin * ri * fma(z, S, -1.0) * chi;
    double gd = 1.0 - x2 * rin * C;
    v[0] = fma(fd, r0[0], gd * v0[0]);
    v[1] = fma(fd, r0[1], gd * v0[1]);
    v[2] = fma(fd, r0[2], gd * v0[2]);
    return ok;
}

// Non-gravitational terms (App. A.4-A.5) of a body at barycentric (x, v):
// heliocentric r, w from the Sun's state at the same epoch (node row or
// table), then radiation pressure with drag (Eq. A.6, radial-speed reading)
// and the JPL comet model (Eq. A.7) from the two-body state dt days earlier.
static __device__ __noinline__ NgOut nongrav_terms(const EphemDev &E, const double *row64, Seg g,
                                                   const kete_nongrav *P, double x0, double x1,
                                                   double x2, double v0, double v1, double v2,
                                                   double chi0)
{
    NgOut o = {{0.0, 0.0, 0.0}, KETE_BODY_OK, chi0};
    double sun[6];
    if (row64) {
#pragma unroll
        for (int q = 0; q < 6; q++) sun[q] = __ldg(row64 + q);
    } else {
        cheb_state64(E, 0, g.s, g.tau, sun, true);
    }
    const kete_nongrav p = *P;
    const double mu = E.gm[0];
    const double r[3] = {x0 - sun[0], x1 - sun[1], x2 - sun[2]};
    const double w[3] = {v0 - sun[3], v1 - sun[4], v2 - sun[5]};
    if (p.beta != 0.0) {
        const double rr = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
        const double rn = sqrt(rr);
        const double rdot = (r[0] * w[0] + r[1] * w[1] + r[2] * w[2]) / rn;
        const double f = p.beta * mu / rr;
        const double kr = f * (1.0 - rdot * kInvC) / rn, kw = f * kInvC;
#pragma unroll
        for (int c = 0; c < 3; c++) o.a[c] = kr * r[c] - kw * w[c];
    }
    if (p.a1 != 0.0 || p.a2 != 0.0 || p.a3 != 0.0) {
        double rl[3] = {r[0], r[1], r[2]}, wl[3] = {w[0], w[1], w[2]};
        if (p.dt != 0.0) {
            // Newton starts from the previous evaluation's solution (0: the
            // series start): the lagged state moves little between the nodes
            double chi = chi0;
            if (!kepler_uv(mu, sqrt(mu), r, w, -p.dt, chi, rl, wl)) {
                o.status = KETE_BODY_KEPLER_CAP;
                return o;
            }
            o.chi = chi;
        }
        const double rn = sqrt(rl[0] * rl[0] + rl[1] * rl[1] + rl[2] * rl[2]);
        const double q = rn / p.r0;
        // g(r) = alpha q^-m (1 + q^n)^-k: the asteroid form (m = 2, k = 0) as
        // alpha / q^2, else from one logarithm of q, q^x = exp(x ln q) (a
        // relative error of a few 1e-16 |x ln q| in a term of ~1e-8 of |a|)
        double gq = p.alpha;
        if (p.m == 2.0 && p.k == 0.0) {
            gq /= q * q;
        } else {
            const double lq = log(q);
            gq *= exp(-p.m * lq);
            if (p.k != 0.0) gq *= exp(-p.k * log1p(exp(p.n * lq)));
        }
        const double rh[3] = {rl[0] / rn, rl[1] / rn, rl[2] / rn};
        double h[3] = {rl[1] * wl[2] - rl[2] * wl[1], rl[2] * wl[0] - rl[0] * wl[2],
                       rl[0] * wl[1] - rl[1] * wl[0]};
        const double hn = sqrt(h[0] * h[0] + h[1] * h[1] + h[2] * h[2]);
        const double nh[3] = {h[0] / hn, h[1] / hn, h[2] / hn};
        const double th[3] = {nh[1] * rh[2] - nh[2] * rh[1], nh[2] * rh[0] - nh[0] * rh[2],
                              nh[0] * rh[1] - nh[1] * rh[0]};
#pragma unroll
        for (int c = 0; c < 3; c++)
            o.a[c] += gq * (p.a1 * rh[c] + p.a2 * th[c] + p.a3 * nh[c]);
    }
    return o;
}

// RA/Dec (equatorial J2000) of an ecliptic vector
__device__ __forceinline__ void radec(const double u[3], double cos_eps, double sin_eps,
                                      double &ra, double &dec)
{
    double x = u[0];
    double y = cos_eps * u[1] - sin_eps * u[2];
    double z = sin_eps * u[1] + cos_eps * u[2];
    double a = atan2(y, x);
    if (a < 0.0) a += kTwoPi;
    if (a >= kTwoPi) a = 0.0;
    ra = a;
    dec = atan2(z, sqrt(x * x + y * y));
}

}  // namespace kete
