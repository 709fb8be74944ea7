// rt_link.cuh — device-side shooting-method linking shared by the single-
// problem and the batched kernels: pair set-up, the linking state machine
// (paper Sec. 3.4: Secant default with a Regula-Falsi safeguard), the fan
// start, the persistent work queue, and the adjoint scatter sink.
#pragma once

#include <cfloat>
#include <climits>
#include <cstdint>

#include <math_constants.h>

#include "rt_trace.cuh"

namespace rt {

constexpr double kPi = 3.141592653589793;

// a mod 2 pi in [0, 2 pi): the multiple from a product with 1/(2 pi) (no FP64
// division, which is slow on this part), then one correction each way, so the
// result is the same as a - 2 pi floor(a / (2 pi)) up to the rounding of the
// last subtraction.
__device__ __forceinline__ double mod_2pi(double a) {
    constexpr double two_pi = 2.0 * kPi, inv_two_pi = 1.0 / (2.0 * kPi);
    double r = fma(-two_pi, floor(a * inv_two_pi), a);
    if (r < 0.0) r += two_pi;
    if (r >= two_pi) r -= two_pi;
    return r;
}

struct LinkCtx {
    double xe, ye, xr, yr, phi_e, phi_r, psi_r, th_lo, th_hi;
};

__device__ __forceinline__ bool on_ring(double x, double y, double R) {
    return fabs(sqrt(x * x + y * y) - R) <= 1e-9 * R;
}

// Resolves pair k; false if the pair or its transducers are invalid.
__device__ __forceinline__ bool setup_pair(const Geom& G, int k, LinkCtx& L) {
    int e, r;
    pair_of(G, k, e, r);
    if (*G.bad_field || e < 0 || e >= G.n_tx || r < 0 || r >= G.n_tx || e == r) return false;
    L.xe = G.tx[2 * e]; L.ye = G.tx[2 * e + 1];
    L.xr = G.tx[2 * r]; L.yr = G.tx[2 * r + 1];
    if (G.tx_phi) {   // per-transducer table (NaN = off the ring)
        L.phi_e = G.tx_phi[e];
        L.phi_r = G.tx_phi[r];
        if (isnan(L.phi_e) || isnan(L.phi_r)) return false;
    } else {
        if (!on_ring(L.xe, L.ye, G.R) || !on_ring(L.xr, L.yr, G.R)) return false;
        L.phi_e = atan2(L.ye, L.xe);
        L.phi_r = atan2(L.yr, L.xr);
    }
    L.psi_r = mod_2pi(L.phi_r - L.phi_e);
    L.th_lo = L.phi_e + 0.5 * kPi;
    L.th_hi = L.phi_e + 1.5 * kPi;
    return true;
}

// Per-lane linking state of the persistent kernel, kept in shared memory so
// that only the trace state occupies registers in the marching loop.
struct LinkState {
    double xe, ye, xr, yr, phi_e, psi_r, th_lo, th_hi;
    double a_min, a_max;
    double th0, m0;                  // first angle and its misfit
    double best_th, best_T, best_hx, best_hy, best_d2;   // closest ray; best_d2 = |x_hit - x_r|^2
    double ta, fa, tb, fb;           // bracket
    double prev_th, prev_m, cur_th, cur_m;
    double psi_at_lo, next;
    int k, n_eval, phase, last, e0_flagged;
    int fan_k0;                      // fan start: interval between rays fan_k0, fan_k0 + 1 whose
                                     // four surrounding rays are usable for the second angle; else -1;
                                     // -2: the pair did not start from the fan
    // adjoint retrace of the batched kernel (read on flushes only)
    double* adj_g;
    double adj_w;
    int adj_nx, adj_ny;
};

__device__ __forceinline__ void br_insert(LinkState& L, double t, double m) {
    if (!(t > fmin(L.ta, L.tb) && t < fmax(L.ta, L.tb))) return;
    if (m < 0) {
        L.ta = t; L.fa = m;
        if (L.last == -1) L.fb *= 0.5;
        L.last = -1;
    } else {
        L.tb = t; L.fb = m;
        if (L.last == 1) L.fa *= 0.5;
        L.last = 1;
    }
}

// Misfit of an ended trace (same rule as evaluate()) and the squared
// distance of its hit to the receiver.
__device__ __forceinline__ void misfit_of(const Geom& G, const LinkState& L, const TraceOut& o, double theta,
                                          double& m, double& d2) {
    const double dx = o.hx - L.xr, dy = o.hy - L.yr;
    d2 = dx * dx + dy * dy;
    double psi;
    if (o.flags & 3) {
        psi = (theta - L.th_lo < L.th_hi - theta) ? L.psi_at_lo : 2.0 * kPi - L.psi_at_lo;
        d2 = DBL_MAX;
    } else {
        // the hit's angle from the emitter = the receiver's (psi_r) + the angle
        // delta from the receiver to the hit around the centre. Both lie on the
        // ring, so sin(delta) = u = (x_r x x_hit) / R^2; near the receiver
        // delta = asin(u) by its series (|u| < 0.05: terms to u^13 leave
        // < 1e-20 relative), else atan2.
        const double cd = L.xr * o.hx + L.yr * o.hy, sd = L.xr * o.hy - L.yr * o.hx;
        const double u = sd * G.inv_R2;
        double delta;
        if (cd > 0.0 && fabs(u) < 0.05) {
            const double u2 = u * u;
            delta = u * (1.0 + u2 * (1.0 / 6 + u2 * (3.0 / 40 + u2 * (15.0 / 336 + u2 * (105.0 / 3456 +
                    u2 * (945.0 / 42240 + u2 * (10395.0 / 599040)))))));
        } else {
            delta = atan2(sd, cd);
        }
        psi = mod_2pi(L.psi_r + delta);
    }
    m = G.R * (psi - L.psi_r);
}

// Next angle inside the bracket: the secant of (prev, cur) if it falls inside,
// else the Regula-Falsi point of the bracket.
__device__ __forceinline__ double next_angle(const LinkState& L, double cand) {
    if (!(isfinite(cand) && cand > fmin(L.ta, L.tb) && cand < fmax(L.ta, L.tb)))
        cand = (L.ta * L.fb - L.tb * L.fa) / (L.fb - L.fa);
    return cand;
}

__device__ __forceinline__ double fan_theta(double a_min, double step, int k) { return a_min + k * step; }

// Misfit R (psi_k - psi_r) of fan ray k, read from memory at each use (the
// row stays in L1/L2), so that the predictions keep no arrays in registers.
__device__ __forceinline__ double fan_m(const double* psi, int k, double R, double psi_r) {
    return R * (*(const volatile double*)(psi + k) - psi_r);
}

// Fan rays kf .. kf + N - 1: true when all of them exist and intercept the
// ring and their misfits change strictly monotonically, in the direction of
// the middle pair (N/2 - 1, N/2).
template <int N>
__device__ __forceinline__ bool fan_usable(const double* psi, int K, int kf, double R, double psi_r) {
    if (kf < 0 || kf + N > K) return false;
    const double dir = fan_m(psi, kf + N / 2, R, psi_r) - fan_m(psi, kf + N / 2 - 1, R, psi_r);
    double prev = fan_m(psi, kf, R, psi_r);
    if (isnan(prev)) return false;
#pragma unroll 1
    for (int q = 1; q < N; ++q) {
        const double cur = fan_m(psi, kf + q, R, psi_r);
        if (!((cur - prev) * dir > 0.0)) return false;
        prev = cur;
    }
    return true;
}

// Position at m = 0 of the polynomial u(m) through the fan rays kf .. kf+N-1
// (positions 0..N-1) and, with extra, the point (u0, m0) first: inverse
// interpolation, Lagrange form with one division per node.
template <int N>
__device__ __forceinline__ double fan_root(const double* psi, int kf, double R, double psi_r, bool extra, double u0,
                                           double m0) {
    const int x = extra ? 1 : 0, n = N + x;
    double v = 0.0;
#pragma unroll 1
    for (int a = 0; a < n; ++a) {
        const double ma = (a < x) ? m0 : fan_m(psi, kf + a - x, R, psi_r);
        const double ua = (a < x) ? u0 : (double)(a - x);
        double num = 1.0, den = 1.0;
#pragma unroll 1
        for (int b = 0; b < n; ++b) {
            if (b == a) continue;
            const double mb = (b < x) ? m0 : fan_m(psi, kf + b - x, R, psi_r);
            num *= -mb;
            den *= ma - mb;
        }
        v += ua * (num / den);
    }
    return v;
}

// Second angle of a fan-started pair whose first trace (theta, m) missed: the
// inverse quartic through that trace and the four fan rays around the
// interval, in fan-index units.
__device__ __forceinline__ double fan_second_angle(const Geom& G, const LinkState& L, double theta, double m,
                                                  const double* __restrict__ fan, int K) {
    int e, r;
    pair_of(G, L.k, e, r);
    const double step = (L.a_max - L.a_min) / (K - 1);
    const int kf = L.fan_k0 - 1;
    const double base = fan_theta(L.a_min, step, kf);
    return base + step * fan_root<4>(fan + (size_t)e * K, kf, G.R, L.psi_r, true, (theta - base) / step, m);
}

// Linking update after the trace of L.next ended (the same decisions as
// link_pair). fan / K: the fan of the launch (null when it has none), for the
// second angle of a fan-started pair. Returns true when the pair is finished.
__device__ inline bool link_update(const Geom& G, LinkState& L, const TraceOut& o, double tol, int max_iter,
                                   const double* __restrict__ fan, int K) {
    const double theta = L.next;
    double m, d2;
    misfit_of(G, L, o, theta, m, d2);
    ++L.n_eval;
    if (d2 < L.best_d2) {
        L.best_th = theta; L.best_T = o.T; L.best_hx = o.hx; L.best_hy = o.hy; L.best_d2 = d2;
    }
    if (d2 <= tol * tol) return true;
    if (L.phase == 0) {
        L.m0 = m;
        L.e0_flagged = (o.flags & 3) != 0;
        if (L.n_eval >= max_iter) return true;
        L.phase = 1;
        L.next = L.a_min;   // orientation probe next to the fan's lower end
        return false;
    }
    if (L.phase == 1) {
        const bool ccw = (m / G.R + L.psi_r) < kPi;
        L.psi_at_lo = ccw ? 0.0 : 2.0 * kPi;
        if (L.e0_flagged) {
            const double psi0 = (L.th0 - L.th_lo < L.th_hi - L.th0) ? L.psi_at_lo : 2.0 * kPi - L.psi_at_lo;
            L.m0 = G.R * (psi0 - L.psi_r);
        }
        const double mp = (o.flags & 3) ? G.R * (L.psi_at_lo - L.psi_r) : m;
        L.ta = ccw ? L.th_lo : L.th_hi; L.fa = -G.R * L.psi_r;
        L.tb = ccw ? L.th_hi : L.th_lo; L.fb = G.R * (2.0 * kPi - L.psi_r);
        L.last = 0;
        br_insert(L, theta, mp);
        br_insert(L, L.th0, L.m0);
        L.last = 0;
        L.prev_th = L.cur_th = L.th0;
        L.prev_m = L.cur_m = L.m0;
        if (L.n_eval >= max_iter) return true;
        L.phase = 2;
        L.next = next_angle(L, L.th0 - L.m0 / (ccw ? 2.0 * G.R : -2.0 * G.R));
        return false;
    }
    br_insert(L, theta, m);
    L.prev_th = L.cur_th; L.prev_m = L.cur_m;
    L.cur_th = theta; L.cur_m = m;
    if (L.n_eval >= max_iter) return true;
    double cand;
    if (L.n_eval == 1 && L.fan_k0 >= 0 && fan && !(o.flags & 3)) {
        cand = fan_second_angle(G, L, theta, m, fan, K);
    } else {
        const double den = L.cur_m - L.prev_m;
        cand = (den != 0.0) ? L.cur_th - L.cur_m * (L.cur_th - L.prev_th) / den : nan("");
    }
    L.next = next_angle(L, cand);
    return false;
}

// ---------------------------------------------------------------- fan start

// Fan start of a cold pair (the rule of the CPU reference, written so that the
// per-ray scan issues no FP64 instruction): the interval of the sequence (fan
// end, rays 0..K-1, fan end) where psi crosses psi_r whose middle lies closest
// to the straight-line angle in fan-index units; first angle from the inverse
// interpolating polynomial of the eight rays around it, else of the four (each
// when those rays are monotone and the root falls inside), else linear. The
// four rays also serve the second angle (link_update).
// psi values are non-negative, so "psi < psi_r" is the signed compare of their
// IEEE bit patterns; NaN (no interception) has the largest patterns.
__device__ inline void fan_start(const Geom& G, LinkState& L, const double* __restrict__ psi, int K) {
    const bool ccw = isnan(psi[0]) ? true : (psi[0] < kPi);
    L.psi_at_lo = ccw ? 0.0 : 2.0 * kPi;
    const double psi_hi_end = 2.0 * kPi - L.psi_at_lo;
    const double step = (L.a_max - L.a_min) / (K - 1);
    double th_s = atan2(L.yr - L.ye, L.xr - L.xe);
    th_s = L.th_lo + mod_2pi(th_s - L.th_lo);
    const double u_s = (th_s - L.a_min) / step;
    const long long* pb = reinterpret_cast<const long long*>(psi);
    const long long b_r = __double_as_longlong(L.psi_r);
    const long long b_lo = __double_as_longlong(L.psi_at_lo), b_hi = __double_as_longlong(psi_hi_end);
    const long long b_nan = 0x7ff0000000000000ll;
    // entry j of the sequence (fan end, rays 0..K-1, fan end), j = 0..K+1
    auto neg_at = [&](int j) {
        long long b;
        if (j == 0) {
            b = b_lo;
        } else if (j <= K) {
            const int k = j - 1;
            b = pb[k];
            if (b > b_nan) b = (k < K / 2) ? b_lo : b_hi;
        } else {
            b = b_hi;
        }
        return b < b_r;
    };
    // The interval (j-1, j) with a sign change whose gap |(j - 1.5) - u_s| is
    // least, the smaller j on a tie: visited outward from u_s in the order of
    // that gap, so the first change found is the one the full scan in index
    // order selects (the sequence always changes sign somewhere, its two ends
    // lie on either side of psi_r), usually a few rays from the start.
    int jsel = K + 1;
    {
        int jl = (int)floor(u_s + 1.5);
        jl = jl < 0 ? 0 : (jl > K + 1 ? K + 1 : jl);
        int jr = jl + 1;
        for (int it = 0; it < K + 2; ++it) {
            const bool has_l = jl >= 1, has_r = jr <= K + 1;
            if (!has_l && !has_r) break;
            bool take_l;
            if (has_l && has_r) take_l = fabs((jl - 1.5) - u_s) <= fabs((jr - 1.5) - u_s);
            else take_l = has_l;
            const int j = take_l ? jl : jr;
            if (neg_at(j) != neg_at(j - 1)) { jsel = j; break; }
            if (take_l) --jl; else ++jr;
        }
    }
    const double R = G.R;
    double t0, t1, p0, p1;
    {
        const int ja = jsel - 1, jb = jsel;
        if (ja == 0) { t0 = L.th_lo; p0 = L.psi_at_lo; }
        else { const int k = ja - 1; t0 = fan_theta(L.a_min, step, k); p0 = psi[k]; if (isnan(p0)) p0 = (k < K / 2) ? L.psi_at_lo : psi_hi_end; }
        if (jb == K + 1) { t1 = L.th_hi; p1 = psi_hi_end; }
        else { const int k = jb - 1; t1 = fan_theta(L.a_min, step, k); p1 = psi[k]; if (isnan(p1)) p1 = (k < K / 2) ? L.psi_at_lo : psi_hi_end; }
    }
    const double m0 = R * (p0 - L.psi_r), m1 = R * (p1 - L.psi_r);
    if (m0 < 0) { L.ta = t0; L.fa = m0; L.tb = t1; L.fb = m1; }
    else { L.ta = t1; L.fa = m1; L.tb = t0; L.fb = m0; }
    L.last = 0;
    double th0 = t0 - m0 * (t1 - t0) / (m1 - m0);
    // rays around the interval: k0 = jsel - 2 and k0 + 1
    const int k0 = jsel - 2;
    {
        bool done = false;
        if (fan_usable<8>(psi, K, k0 - 3, R, L.psi_r)) {
            const double v = fan_theta(L.a_min, step, k0 - 3) + step * fan_root<8>(psi, k0 - 3, R, L.psi_r, false, 0.0, 0.0);
            if (v > fmin(t0, t1) && v < fmax(t0, t1)) { th0 = v; done = true; }
        }
        L.fan_k0 = -1;
        if (fan_usable<4>(psi, K, k0 - 1, R, L.psi_r)) {
            L.fan_k0 = k0;
            if (!done) {
                const double v = fan_theta(L.a_min, step, k0 - 1) + step * fan_root<4>(psi, k0 - 1, R, L.psi_r, false, 0.0, 0.0);
                if (v > fmin(t0, t1) && v < fmax(t0, t1)) th0 = v;
            }
        }
    }
    if (!(th0 > fmin(L.ta, L.tb) && th0 < fmax(L.ta, L.tb))) th0 = 0.5 * (L.ta + L.tb);
    const bool first = fabs(m0) <= fabs(m1);
    L.cur_th = L.prev_th = first ? t0 : t1;
    L.cur_m = L.prev_m = first ? m0 : m1;
    L.th0 = th0;
    L.next = th0;
    L.phase = 2;
}

// ---------------------------------------------------------------- R12 sub-fan

constexpr int kSubfanMax = 32;   // RT_SUBFAN_MAX

// One round of a linking launch split into rounds (R12 schedule): pairs from
// the work queue or resumed from the states the previous round set aside;
// with stop_after > 0 a pair that has made that many traces without finishing
// is set aside (its state saved, its next angle already chosen).
struct LinkRound {
    int stop_after;
    LinkState* aside_out;
    int* n_out;
    const LinkState* aside_in;   // non-null: resume these states instead of the queue
    const int* n_in;
    const double* sub;           // R12 sub-fan misfits of the resumed pairs [slot][sub_m], or null
    int sub_m;
};

// Angle of sub-fan ray q = 1..M, evenly spaced strictly inside the bracket
// from its end of negative misfit.
__device__ __forceinline__ double subfan_theta(const LinkState& L, int q, int M) {
    return L.ta + (L.tb - L.ta) * q / (M + 1);
}

// R12: a fan-started pair whose second trace missed, with the misfits m[q-1]
// of its M sub-fan rays (NaN: the ray did not reach the ring) and L.next, the
// third angle the plain rule chose. In the sequence (ta, the sub-fan rays that
// reached the ring, tb) a crossing is a pair of neighbours with no ray that
// missed the ring between them whose misfits differ in sign by less than
// pi R (where hits wrap around the emitter the misfit jumps by about 2 pi R);
// the crossing that holds L.next becomes the
// bracket (Illinois state restarted), the third angle is the root of the
// inverse cubic through the four sub-fan rays around it (all four sub-fan
// rays, misfits strictly monotone, root inside), else its Regula-Falsi point,
// and the secant starts from its end of smaller |misfit|. When no crossing
// holds L.next the state is left as the plain rule set it.
static __device__ __noinline__ void subfan_apply(LinkState& L, const double* __restrict__ m, int M, double R) {
    double st[kSubfanMax + 2], sm[kSubfanMax + 2];
    bool in[kSubfanMax + 2];
    int pos[kSubfanMax + 2];
    int n = 0;
    st[n] = L.ta; sm[n] = L.fa; in[n] = false; pos[n++] = 0;
    for (int q = 1; q <= M; ++q) {
        const double v = m[q - 1];
        if (isnan(v)) continue;
        st[n] = subfan_theta(L, q, M); sm[n] = v; in[n] = true; pos[n++] = q;
    }
    st[n] = L.tb; sm[n] = L.fb; in[n] = false; pos[n++] = M + 1;
    const double c3 = L.next;
    int j = -1;
    for (int i = 1; i < n && j < 0; ++i) {
        if ((sm[i - 1] < 0) == (sm[i] < 0) || !(fabs(sm[i] - sm[i - 1]) < kPi * R) || pos[i] != pos[i - 1] + 1)
            continue;
        if (c3 >= fmin(st[i - 1], st[i]) && c3 <= fmax(st[i - 1], st[i])) j = i;
    }
    if (j < 0) return;
    const int ng = sm[j - 1] < 0 ? j - 1 : j, ps = sm[j - 1] < 0 ? j : j - 1;
    L.ta = st[ng]; L.fa = sm[ng];
    L.tb = st[ps]; L.fb = sm[ps];
    L.last = 0;
    double th = L.ta - L.fa * (L.tb - L.ta) / (L.fb - L.fa);
    if (j - 2 >= 0 && j + 1 < n && in[j - 2] && in[j - 1] && in[j] && in[j + 1]) {
        const bool up = sm[j - 2] < sm[j - 1] && sm[j - 1] < sm[j] && sm[j] < sm[j + 1];
        const bool down = sm[j - 2] > sm[j - 1] && sm[j - 1] > sm[j] && sm[j] > sm[j + 1];
        if (up || down) {
            // inverse cubic through the four rays, Lagrange form at misfit 0
            double v = 0.0;
            for (int a = 0; a < 4; ++a) {
                double l = 1.0;
                for (int b = 0; b < 4; ++b)
                    if (b != a) l *= (0.0 - sm[j - 2 + b]) / (sm[j - 2 + a] - sm[j - 2 + b]);
                v += l * st[j - 2 + a];
            }
            if (v > fmin(L.ta, L.tb) && v < fmax(L.ta, L.tb)) th = v;
        }
    }
    const bool lo = fabs(L.fa) <= fabs(L.fb);
    L.cur_th = L.prev_th = lo ? L.ta : L.tb;
    L.cur_m = L.prev_m = lo ? L.fa : L.fb;
    L.next = th;
}

// Work order of the persistent kernel. For the all-pairs list, queue slot q
// serves ring offsets o = r - e (mod N) from the longest chord (o = N/2) down to
// the shortest (o = 1, N-1), N emitters per offset, so the launch's tail is
// made of the shortest rays; the pair's own index k is returned. Explicit pair
// lists are served in their order.
__device__ __forceinline__ int queue_pair(const Geom& G, int q) {
    if (G.pairs) return q;
    const int N = G.n_tx;
    const int t = q / N, e = q - t * N;
    const int h = (N + 1) / 2;
    const int o = (t & 1) ? h - (t + 1) / 2 : h + t / 2;
    const int r = (e + o) % N;
    return e * (N - 1) + r - (r > e);
}

// Warp-aggregated fetch of the next pair index from the work queue.
__device__ __forceinline__ int fetch_pair(int* queue) {
    const unsigned mask = __activemask();
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(mask) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(queue, __popc(mask));
    base = __shfl_sync(mask, base, leader);
    return base + __popc(mask & ((1u << lane) - 1u));
}

constexpr int kLinkBlock = 128;
// Resident blocks per SM asked of the compiler: FP32 at <= 85 registers
// (6 blocks, 24 warps), FP64 unconstrained.
template <typename T> struct LinkOcc { static constexpr int blocks = 1; };
template <> struct LinkOcc<float> { static constexpr int blocks = 6; };

// Scatters w * alpha_m * phi_j(x_m) into g (FP64 atomics), one flush of the
// four nodes per run of consecutive points in one cell. The node weights are
// formed in the marching precision and widened exactly to FP64 for the atomic.
// A run the ray has left waits in `prev` for the next periodic flush (every
// kFlushEvery points), which the lanes of a warp whose rays started together
// reach together, instead of each lane flushing at its own cell crossings
// while the warp's other lanes wait; a second crossing before that flush
// flushes the waiting run at once. Each run is still flushed exactly once.
constexpr int kFlushEvery = 2;
template <typename T>
struct AdjSink {
    double* g;
    T w;
    int nx, ny;
    int tick;
    CellAcc<T> acc, prev;
    __device__ __forceinline__ void flush(const CellAcc<T>& a) {
        const T w11 = a.Wxy, w10 = a.Wx - a.Wxy, w01 = a.Wy - a.Wxy;
        const T w00 = (a.W - a.Wx) - w01;
        const int i = min(max(a.ai, 0), nx - 2), j = min(max(a.aj, 0), ny - 2);
        double* p = g + (size_t)j * nx + i;
        atomicAdd(p, to_double(w * w00));
        atomicAdd(p + 1, to_double(w * w10));
        atomicAdd(p + nx, to_double(w * w01));
        atomicAdd(p + nx + 1, to_double(w * w11));
    }
    __device__ __forceinline__ void add(int ci, int cj, T tx, T ty, T a) {
        if (ci != acc.ai || cj != acc.aj) {
            if (prev.ai != INT_MIN) flush(prev);
            prev = acc;
            acc.reset();
            acc.ai = ci;
            acc.aj = cj;
        }
        acc.W += a;
        acc.Wx += a * tx;
        acc.Wy += a * ty;
        acc.Wxy += a * tx * ty;
        if (++tick == kFlushEvery) {
            tick = 0;
            if (prev.ai != INT_MIN) flush(prev);
            prev.ai = INT_MIN;
        }
    }
    __device__ __forceinline__ void finish() {
        if (prev.ai != INT_MIN) flush(prev);
        if (acc.ai != INT_MIN) flush(acc);
        init();
    }
    __device__ __forceinline__ void init() {
        acc.reset();
        prev.reset();
        tick = 0;
    }
};

// Records a trace's runs (rt_run: the cell's lower-left node and its four
// node weights, formed exactly as AdjSink::flush forms them before scaling)
// into the pair's slot; runs beyond cap are counted but not stored.
template <typename T>
struct RecSink {
    rt_run* base;
    int n, cap, nx, ny;
    CellAcc<T> acc;
    __device__ __forceinline__ void emit(const CellAcc<T>& a) {
        if (n < cap) {
            const T w11 = a.Wxy, w10 = a.Wx - a.Wxy, w01 = a.Wy - a.Wxy;
            const T w00 = (a.W - a.Wx) - w01;
            const int i = min(max(a.ai, 0), nx - 2), j = min(max(a.aj, 0), ny - 2);
            rt_run r;
            r.node = j * nx + i;
            r.w00 = (float)w00;
            r.w10 = (float)w10;
            r.w01 = (float)w01;
            r.w11 = (float)w11;
            base[n] = r;
        }
        ++n;
    }
    __device__ __forceinline__ void add(int ci, int cj, T tx, T ty, T a) {
        if (ci != acc.ai || cj != acc.aj) {
            if (acc.ai != INT_MIN) emit(acc);
            acc.reset();
            acc.ai = ci;
            acc.aj = cj;
        }
        acc.W += a;
        acc.Wx += a * tx;
        acc.Wy += a * ty;
        acc.Wxy += a * tx * ty;
    }
    __device__ __forceinline__ void finish() {
        if (acc.ai != INT_MIN) emit(acc);
        acc.reset();
    }
    __device__ __forceinline__ void begin(rt_run* slot) {
        base = slot;
        n = 0;
        acc.reset();
    }
};

// Recording target of a linking launch (rt_link_rows); runs == null: none.
struct RowRec {
    rt_run* runs;
    int32_t* len;
    int cap;
};

}  // namespace rt
