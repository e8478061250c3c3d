// Forward rollout and checkpointed adjoint of the relaxed block-pushing
// simulation (Sec. III-B; Algorithm 1 "simulate plans" and the gradient of
// log rho).  Templated on the block count NB and on L, the number of lanes of
// a warp that cooperate on one particle.
//
// Work split inside a team of L lanes: the M*NB (pusher, block) contact items
// (pushers on their own object first) and the 8 corner tests of every block
// pair are dealt round-robin to the lanes; every lane runs the same instruction stream (items only change the
// data, never the control flow), the per-block forces are summed with an xor
// butterfly (identical sums on every lane), and every lane then integrates
// the full state redundantly.  Particle state lives in registers for the
// whole rollout; the forward writes a checkpoint every C substeps, the adjoint
// recomputes each C-substep segment into shared memory and walks it backwards.
//
// Physics (all choices restate the paper's model class: kinematic pushers,
// spring-damper penalty contact, smoothed Coulomb friction, semi-implicit
// Euler):
//   pusher c = (object o = c/4, side s = c%4), sides N,E,S,W with outward
//   normals (0,1),(1,0),(0,-1),(-1,0); it starts touching side s at
//   tangential offset `off` and moves `dist` along the inward normal over T
//   substeps; during substep j (0-based) its centre is p0 + (j+1)*delta,
//   delta = -R(yaw_o) n_s * dist/T, its velocity delta/dt;
//   every pusher acts on every block with weight z_{k,c};
//   disk/box contact: delta = r - sd, f_n = max(0, k*delta - c*v_n),
//   smoothed Coulomb tangential force mu_c*f_n*w_t/sqrt(|w_t|^2+eps_t^2);
//   box/box: the 8 corners of each pair tested against the other box;
//   ground: -mu*m*g*v/sqrt(|v|^2+eps_v^2), -mu*m*g*r_eff*w/sqrt(w^2+eps_w^2).
#pragma once

#include <cfloat>
#include <cstdint>

#include "stamp_internal.cuh"

namespace stamp {
namespace rollout {

template <int NB>
struct Dims {
    static constexpr int M = 4 * NB;              // choices per action
    static constexpr int P = M + 2;               // parameters per action
    static constexpr int S = 6 * NB;              // state floats per particle
    static constexpr int NPI = M * NB;            // (pusher, block) items
    static constexpr int NPAIR = NB * (NB - 1) / 2;
    static constexpr int NCI = 8 * NPAIR;         // corner tests
};

template <int NB>
struct Blocks {
    float x[NB], y[NB], ph[NB], vx[NB], vy[NB], om[NB];
};

template <int NB>
__device__ __forceinline__ void zero(Blocks<NB>& b) {
#pragma unroll
    for (int i = 0; i < NB; ++i) b.x[i] = b.y[i] = b.ph[i] = b.vx[i] = b.vy[i] = b.om[i] = 0.f;
}

// Element `b` (runtime) of a register array, without dynamic indexing.
template <int N>
__device__ __forceinline__ float pick(const float (&a)[N], int b) {
    float r = a[0];
#pragma unroll
    for (int i = 1; i < N; ++i) r = (b == i) ? a[i] : r;
    return r;
}
template <int N>
__device__ __forceinline__ void add_at(float (&a)[N], int b, float v) {
#pragma unroll
    for (int i = 0; i < N; ++i)
        if (b == i) a[i] += v;
}

// Sum over the L lanes of a team (aligned groups of L lanes in the warp).
template <int L>
__device__ __forceinline__ float team_sum(float v) {
#pragma unroll
    for (int o = 1; o < L; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
template <int L, int N>
__device__ __forceinline__ void team_sum(float (&a)[N]) {
#pragma unroll
    for (int i = 0; i < N; ++i) a[i] = team_sum<L>(a[i]);
}
template <int L, int NB>
__device__ __forceinline__ void team_sum(Blocks<NB>& b) {
    team_sum<L>(b.x); team_sum<L>(b.y); team_sum<L>(b.ph);
    team_sum<L>(b.vx); team_sum<L>(b.vy); team_sum<L>(b.om);
}

// sin/cos of a yaw (full-accuracy sincosf: the hardware approximation's
// ~4e-7 absolute error measurably degrades parity through the contact
// dynamics).
__device__ __forceinline__ void yaw_sincos(float x, float* s, float* c) { sincosf(x, s, c); }

__device__ __forceinline__ void side_normal(int s, float& nx, float& ny) {
    nx = (s == 1) ? 1.f : (s == 3) ? -1.f : 0.f;
    ny = (s == 0) ? 1.f : (s == 2) ? -1.f : 0.f;
}

// Item e of the M*NB (pusher, block) pairs: first the M pairs of a pusher
// and its own object (the block it is placed against: in contact through
// most of the push), then the pairs of a pusher and another block (in
// contact only where blocks meet).  Dealt round-robin to the lanes, the
// nearly-always-active contacts land one per lane (up to M lanes), so no
// lane's serial path carries more of them than the team width forces.
template <int NB>
__device__ __forceinline__ void item_of(int e, int& c, int& b) {
    constexpr int M = Dims<NB>::M;
    if (NB == 1 || e < M) {
        c = e;
        b = e / 4;
        return;
    }
    const int r = e - M, k = r % (NB > 1 ? NB - 1 : 1);
    c = r / (NB > 1 ? NB - 1 : 1);
    b = k < c / 4 ? k : k + 1;
}

// Per-lane (pusher, block) item slots of the current action.
template <int NB, int L>
struct Slots {
    static constexpr int SP = (Dims<NB>::NPI + L - 1) / L;
    float p0x[SP], p0y[SP], dx[SP], dy[SP], w[SP];
    int b[SP], c[SP];   // block of the item; pusher (choice) index, -1 if empty
};
template <int NB, int L>
struct SlotAcc {
    static constexpr int SP = Slots<NB, L>::SP;
    float p0x[SP], p0y[SP], dx[SP], dy[SP], w[SP];
};

// Per-lane corner-test slots (fixed for the whole rollout).
template <int NB, int L>
struct Corners {
    static constexpr int NCI = Dims<NB>::NCI;
    static constexpr int SC = NCI > 0 ? (NCI + L - 1) / L : 1;
    int own[SC], oth[SC];
    float ex[SC], ey[SC];   // corner in the owner's frame (units of half size)
    bool on[SC];
};

template <int NB, int L>
__device__ __forceinline__ void make_corners(Corners<NB, L>& cn, int lane) {
#pragma unroll
    for (int q = 0; q < Corners<NB, L>::SC; ++q) {
        const int e = lane + q * L;
        cn.on[q] = e < Dims<NB>::NCI;
        const int p = cn.on[q] ? e / 8 : 0, dir = (e % 8) / 4, corner = e % 4;
        int A = 0, B = 1, cnt = 0;
#pragma unroll
        for (int a = 0; a < NB; ++a)
#pragma unroll
            for (int b = a + 1; b < NB; ++b) {
                if (cnt == p) { A = a; B = b; }
                ++cnt;
            }
        cn.own[q] = dir ? B : A;
        cn.oth[q] = dir ? A : B;
        // corners (+,+), (-,+), (-,-), (+,-)
        cn.ex[q] = (corner == 0 || corner == 3) ? 1.f : -1.f;
        cn.ey[q] = (corner < 2) ? 1.f : -1.f;
    }
}

// Relaxed action parameters of action k for particle row `th`
// (Eq. gamma_map: softmax((a+g)/tau), or one-hot argmax when hard).
template <int NB>
__device__ __forceinline__ void relax_action(const SimConst& sc, const float* th, int k, int i,
                                             uint64_t gkey, bool noise, bool hard,
                                             float (&z)[Dims<NB>::M], float& uu, float& vv) {
    constexpr int M = Dims<NB>::M, P = Dims<NB>::P;
    const float* a = th + k * P;
#pragma unroll
    for (int c = 0; c < M; ++c) {
        float v = a[c];
        if (noise) {
            const float u = u23(sm64(gkey, (uint64_t)((i * sc.H + k) * M + c)));
            v += -logf(-logf(u));
        }
        z[c] = v;
    }
    if (hard) {
        int best = 0;
        float bv = z[0];
#pragma unroll
        for (int c = 1; c < M; ++c)
            if (z[c] > bv) { bv = z[c]; best = c; }
#pragma unroll
        for (int c = 0; c < M; ++c) z[c] = (c == best) ? 1.f : 0.f;
    } else {
        float mx = z[0] * sc.inv_tau;
#pragma unroll
        for (int c = 1; c < M; ++c) mx = fmaxf(mx, z[c] * sc.inv_tau);
        float sum = 0.f;
#pragma unroll
        for (int c = 0; c < M; ++c) { z[c] = expf(z[c] * sc.inv_tau - mx); sum += z[c]; }
        const float inv = 1.f / sum;
#pragma unroll
        for (int c = 0; c < M; ++c) z[c] *= inv;
    }
    uu = a[M];
    vv = a[M + 1];
}

__device__ __forceinline__ float sigmoidf_(float v) { return 1.f / (1.f + expf(-v)); }

// Pusher start centres and per-substep displacements for this lane's slots,
// from the block poses at the action start.
template <int NB, int L>
__device__ __forceinline__ void make_slots(const SimConst& sc, const Blocks<NB>& s, int lane,
                                           const float (&z)[Dims<NB>::M], float off, float dist,
                                           Slots<NB, L>& sl) {
    const float step = dist / (float)sc.T;
#pragma unroll
    for (int q = 0; q < Slots<NB, L>::SP; ++q) {
        const int e = lane + q * L;
        const bool on = e < Dims<NB>::NPI;
        int c = 0, b = 0;
        if (on) item_of<NB>(e, c, b);
        sl.c[q] = on ? c : -1;
        sl.b[q] = b;
        const int o = c / 4, side = c % 4;
        float nx, ny;
        side_normal(side, nx, ny);
        const float tx = -ny, ty = nx;
        const float lx = nx * (sc.hs + sc.r) + tx * off;
        const float ly = ny * (sc.hs + sc.r) + ty * off;
        float cph, sph;
        yaw_sincos(pick(s.ph, o), &sph, &cph);
        sl.p0x[q] = pick(s.x, o) + cph * lx - sph * ly;
        sl.p0y[q] = pick(s.y, o) + sph * lx + cph * ly;
        sl.dx[q] = -(cph * nx - sph * ny) * step;
        sl.dy[q] = -(sph * nx + cph * ny) * step;
        sl.w[q] = on ? pick(z, c) : 0.f;
    }
}

// ------------------------------- forces -------------------------------------
// Force and torque on a square block (centre b, yaw via cph/sph, velocity v,
// omega) from a kinematic disk pusher at p moving with vp (unweighted).
// A pusher centre (corner) at offset (dx, dy) from a block centre farther
// than the block's reach cannot touch it: the contact tests below return no
// contact there, so callers may skip them.
__device__ __forceinline__ bool out_of_reach(float dx, float dy, float reach2) {
    return dx * dx + dy * dy > reach2;
}

// far_check: first test whether the pusher is out of reach (for items that
// are rarely in contact; the pusher on its own object nearly always is).
__device__ __forceinline__ void disk_box(const SimConst& sc, float px, float py, float vpx,
                                         float vpy, float bx, float by, float cph, float sph,
                                         float vx, float vy, float om, float& fx, float& fy,
                                         float& tq, bool far_check) {
    fx = fy = tq = 0.f;
    const float dx = px - bx, dy = py - by;
    if (far_check && dx * dx + dy * dy > sc.disk_reach2) return;   // out of reach: no contact
    const float lx = cph * dx + sph * dy, ly = -sph * dx + cph * dy;
    const float qx = fabsf(lx) - sc.hs, qy = fabsf(ly) - sc.hs;
    const float sx = lx >= 0.f ? 1.f : -1.f, sy = ly >= 0.f ? 1.f : -1.f;
    // outside: normalised clamped offset; inside: the axis of the larger q
    // (selects, not branches: both are cheap and the chain stays straight)
    const bool outside = qx > 0.f || qy > 0.f;
    const float mx = fmaxf(qx, 0.f), my = fmaxf(qy, 0.f);
    const float il = rsqrtf(fmaxf(mx * mx + my * my, 1e-30f));
    const bool xa = qx >= qy;
    const float sd = outside ? (mx * mx + my * my) * il : fmaxf(qx, qy);
    const float nlx = outside ? sx * mx * il : (xa ? sx : 0.f);
    const float nly = outside ? sy * my * il : (xa ? 0.f : sy);
    const float delta = sc.r - sd;
    if (!(delta > 0.f)) return;
    const float nx = cph * nlx - sph * nly, ny = sph * nlx + cph * nly;
    const float rx = px - sc.r * nx - bx, ry = py - sc.r * ny - by;
    const float wx = vpx - (vx - om * ry), wy = vpy - (vy + om * rx);
    const float vn = wx * nx + wy * ny;
    const float fn = sc.k * delta - sc.c * vn;
    if (!(fn > 0.f)) return;
    const float tx = wx - vn * nx, ty = wy - vn * ny;
    const float gt = sc.mu_c * fn * rsqrtf(tx * tx + ty * ty + sc.eps_t2);
    fx = -fn * nx + gt * tx;
    fy = -fn * ny + gt * ty;
    tq = rx * fy - ry * fx;
}

// Corner k (position, velocity) of one box against square B: force on the
// corner's owner (B receives the opposite at the same point).
__device__ __forceinline__ void corner_box(const SimConst& sc, float kx, float ky, float kvx,
                                           float kvy, float bx, float by, float cph, float sph,
                                           float vx, float vy, float om, float& fx, float& fy) {
    fx = fy = 0.f;
    const float dx = kx - bx, dy = ky - by;
    if (dx * dx + dy * dy > sc.corner_reach2) return;   // out of reach: no contact
    const float lx = cph * dx + sph * dy, ly = -sph * dx + cph * dy;
    const float qx = fabsf(lx) - sc.hs, qy = fabsf(ly) - sc.hs;
    if (!(qx < 0.f && qy < 0.f)) return;
    const float sx = lx >= 0.f ? 1.f : -1.f, sy = ly >= 0.f ? 1.f : -1.f;
    const bool xa = qx >= qy;
    const float nlx = xa ? sx : 0.f, nly = xa ? 0.f : sy;
    const float delta = -(xa ? qx : qy);
    const float nx = cph * nlx - sph * nly, ny = sph * nlx + cph * nly;
    const float wx = kvx - (vx - om * dy), wy = kvy - (vy + om * dx);
    const float vn = wx * nx + wy * ny;
    const float fn = sc.k * delta - sc.c * vn;
    if (!(fn > 0.f)) return;
    const float tx = wx - vn * nx, ty = wy - vn * ny;
    const float gt = sc.mu_c * fn * rsqrtf(tx * tx + ty * ty + sc.eps_t2);
    fx = fn * nx - gt * tx;
    fy = fn * ny - gt * ty;
}

template <int NB, int L>
__device__ __forceinline__ void substep_forces(const SimConst& sc, const Blocks<NB>& s,
                                               const float (&cs)[NB], const float (&sn)[NB],
                                               const Slots<NB, L>& sl, const Corners<NB, L>& cn,
                                               float j1, float (&Fx)[NB], float (&Fy)[NB],
                                               float (&Tq)[NB]) {
#pragma unroll
    for (int b = 0; b < NB; ++b) Fx[b] = Fy[b] = Tq[b] = 0.f;
#pragma unroll
    for (int q = 0; q < Slots<NB, L>::SP; ++q) {
        if (sl.c[q] < 0) continue;
        const int b = sl.b[q];
        const float px = sl.p0x[q] + j1 * sl.dx[q], py = sl.p0y[q] + j1 * sl.dy[q];
        const float bx = pick(s.x, b), by = pick(s.y, b);
        // slots past the first M items hold only pushers on other objects:
        // one out of reach contributes nothing (skipped whole, by every lane
        // of the warp when none has such an item in reach)
        if (q * L >= Dims<NB>::M && out_of_reach(px - bx, py - by, sc.disk_reach2)) continue;
        float fx, fy, tq;
        disk_box(sc, px, py, sl.dx[q] * sc.inv_dt, sl.dy[q] * sc.inv_dt, bx, by, pick(cs, b),
                 pick(sn, b), pick(s.vx, b), pick(s.vy, b), pick(s.om, b), fx, fy, tq, false);
        const float w = sl.w[q];
        add_at(Fx, b, w * fx);
        add_at(Fy, b, w * fy);
        add_at(Tq, b, w * tq);
    }
    if constexpr (Dims<NB>::NCI > 0) {
#pragma unroll
        for (int q = 0; q < Corners<NB, L>::SC; ++q) {
            if (!cn.on[q]) continue;
            const int o = cn.own[q], t = cn.oth[q];
            const float co = pick(cs, o), so = pick(sn, o);
            const float clx = cn.ex[q] * sc.hs, cly = cn.ey[q] * sc.hs;
            const float rlx = co * clx - so * cly, rly = so * clx + co * cly;
            const float kx = pick(s.x, o) + rlx, ky = pick(s.y, o) + rly;
            const float bx = pick(s.x, t), by = pick(s.y, t);
            if (out_of_reach(kx - bx, ky - by, sc.corner_reach2)) continue;
            const float omo = pick(s.om, o);
            const float kvx = pick(s.vx, o) - omo * rly, kvy = pick(s.vy, o) + omo * rlx;
            float fx, fy;
            corner_box(sc, kx, ky, kvx, kvy, bx, by, pick(cs, t), pick(sn, t), pick(s.vx, t),
                       pick(s.vy, t), pick(s.om, t), fx, fy);
            add_at(Fx, o, fx);
            add_at(Fy, o, fy);
            add_at(Tq, o, rlx * fy - rly * fx);
            add_at(Fx, t, -fx);
            add_at(Fy, t, -fy);
            add_at(Tq, t, -((kx - bx) * fy - (ky - by) * fx));
        }
    }
    team_sum<L>(Fx);
    team_sum<L>(Fy);
    team_sum<L>(Tq);
}

// Ground friction, then semi-implicit Euler.
template <int NB>
__device__ __forceinline__ void integrate(const SimConst& sc, Blocks<NB>& s, float (&Fx)[NB],
                                          float (&Fy)[NB], float (&Tq)[NB]) {
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const float isv = rsqrtf(s.vx[b] * s.vx[b] + s.vy[b] * s.vy[b] + sc.eps_v2);
        const float iso = rsqrtf(s.om[b] * s.om[b] + sc.eps_w2);
        const float fx = Fx[b] - sc.fric_lin * s.vx[b] * isv;
        const float fy = Fy[b] - sc.fric_lin * s.vy[b] * isv;
        const float tq = Tq[b] - sc.fric_ang * s.om[b] * iso;
        s.vx[b] += sc.dt * (fx * sc.inv_m);
        s.vy[b] += sc.dt * (fy * sc.inv_m);
        s.om[b] += sc.dt * (tq * sc.inv_I);
        s.x[b] += sc.dt * s.vx[b];
        s.y[b] += sc.dt * s.vy[b];
        s.ph[b] += sc.dt * s.om[b];
    }
}

template <int NB>
__device__ __forceinline__ void trig(const Blocks<NB>& s, float (&cs)[NB], float (&sn)[NB]) {
#pragma unroll
    for (int b = 0; b < NB; ++b) yaw_sincos(s.ph[b], &sn[b], &cs[b]);
}
// (cos, sin) of the blocks' yaws as NB float2; a team stores them split over
// its lanes like the state.
template <int NB, int L>
__device__ __forceinline__ void store_trig(float2* dst, const float (&cs)[NB], const float (&sn)[NB],
                                           int lane, bool on) {
#pragma unroll
    for (int b = 0; b < NB; ++b)
        if (on && (b % L) == lane) dst[b] = make_float2(cs[b], sn[b]);
}
template <int NB>
__device__ __forceinline__ void load_trig(const float2* src, float (&cs)[NB], float (&sn)[NB]) {
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const float2 v = src[b];
        cs[b] = v.x;
        sn[b] = v.y;
    }
}

// State chunk q (of S/2 float2 chunks): block q/3, fields (x,y), (ph,vx), (vy,om).
template <int NB>
__device__ __forceinline__ float2 chunk(const Blocks<NB>& s, int q) {
    const int b = q / 3, f = q % 3;
    return f == 0 ? make_float2(s.x[b], s.y[b])
                  : f == 1 ? make_float2(s.ph[b], s.vx[b]) : make_float2(s.vy[b], s.om[b]);
}
template <int NB>
__device__ __forceinline__ void set_chunk(Blocks<NB>& s, int q, float2 v) {
    const int b = q / 3, f = q % 3;
    if (f == 0) { s.x[b] = v.x; s.y[b] = v.y; }
    else if (f == 1) { s.ph[b] = v.x; s.vx[b] = v.y; }
    else { s.vy[b] = v.x; s.om[b] = v.y; }
}

// Team-cooperative store of the state (lane l writes chunks l, l+L, ...).
template <int NB, int L>
__device__ __forceinline__ void store_state(float2* dst, const Blocks<NB>& s, int lane, bool on) {
#pragma unroll
    for (int q = 0; q < 3 * NB; ++q)
        if (on && (q % L) == lane) dst[q] = chunk(s, q);
}
template <int NB>
__device__ __forceinline__ void load_state(const float2* src, Blocks<NB>& s) {
#pragma unroll
    for (int q = 0; q < 3 * NB; ++q) set_chunk(s, q, src[q]);
}

// The same through L2 only: for a tape that other lanes of the warp wrote
// earlier in the same launch (no non-coherent cache line can be stale).
template <int NB>
__device__ __forceinline__ void load_state_cg(const float2* src, Blocks<NB>& s) {
#pragma unroll
    for (int q = 0; q < 3 * NB; ++q) set_chunk(s, q, __ldcg(src + q));
}

template <int NB>
__device__ __forceinline__ void init_state(const SimConst& sc, Blocks<NB>& s) {
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        s.x[b] = sc.init[b][0]; s.y[b] = sc.init[b][1]; s.ph[b] = sc.init[b][2];
        s.vx[b] = s.vy[b] = s.om[b] = 0.f;
    }
}

__device__ __forceinline__ float wrapf(float e) { return atan2f(sinf(e), cosf(e)); }

// ------------------------------ forward kernel -------------------------------
// One team's forward rollout of particle i (on = false: a surplus team that
// shadows particle i and stores nothing).
template <int NB, int L>
__device__ __forceinline__ void fwd_team(const SimConst& sc, const RolloutArgs& a, int i, bool on,
                                         int lane) {
    constexpr int M = Dims<NB>::M, S = Dims<NB>::S;
    const float* th = a.theta + (size_t)i * sc.D;
    const bool noise = a.iter >= 0;
    const uint64_t gkey = noise ? sm64(sm64(a.seed, kStreamGumbel), (uint64_t)a.iter) : 0ull;

    Corners<NB, L> cn;
    make_corners(cn, lane);
    Blocks<NB> s;
    init_state(sc, s);
    if (a.init_states) {   // per-particle start poses (transition sampling)
        const float* p0 = a.init_states + (size_t)i * 3 * NB;
#pragma unroll
        for (int b = 0; b < NB; ++b) { s.x[b] = p0[3 * b]; s.y[b] = p0[3 * b + 1]; s.ph[b] = p0[3 * b + 2]; }
    }
    float dsum = 0.f;
    const size_t ck_stride = (size_t)a.N * S;   // floats per checkpoint
    float2* tape_i = reinterpret_cast<float2*>(a.tape + (size_t)i * S);

    for (int k = 0; k < sc.H; ++k) {
        float z[M], uu, vv;
        relax_action<NB>(sc, th, k, i + a.particle0, gkey, noise, a.hard != 0, z, uu, vv);
        const float off = sc.off_max * tanhf(uu);
        const float dist = sc.dist_max * sigmoidf_(vv);
        dsum += dist * dist;
        Slots<NB, L> sl;
        make_slots<NB, L>(sc, s, lane, z, off, dist, sl);
        const int segs = sc.T / sc.C;
        for (int sg = 0; sg < segs; ++sg) {
            store_state<NB, L>(tape_i + (size_t)(k * segs + sg) * (ck_stride / 2), s, lane, on);
            for (int jj = 0; jj < sc.C; ++jj) {
                float cs[NB], sn[NB];
                trig(s, cs, sn);
                float Fx[NB], Fy[NB], Tq[NB];
                substep_forces<NB, L>(sc, s, cs, sn, sl, cn, (float)(sg * sc.C + jj + 1), Fx, Fy,
                                      Tq);
                integrate(sc, s, Fx, Fy, Tq);
            }
        }
    }
    store_state<NB, L>(tape_i + (size_t)sc.n_ckpt * (ck_stride / 2), s, lane, on);

    float cost = sc.w_push * dsum;
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const float ex = s.x[b] - sc.goal[b][0], ey = s.y[b] - sc.goal[b][1];
        const float ew = wrapf(s.ph[b] - sc.goal[b][2]);
        cost += ex * ex + ey * ey + sc.w_yaw * ew * ew;
    }
    if (on && lane == 0) {
        if (a.cost) a.cost[i] = cost;
        if (a.stats_min) atomicMin(a.stats_min, __float_as_uint(cost));
    }
    if (on && a.final_state)
        store_state<NB, L>(reinterpret_cast<float2*>(a.final_state + (size_t)i * S), s, lane, true);
}

template <int NB, int L>
__global__ void __launch_bounds__(128) rollout_fwd_kernel(const SimConst sc, const RolloutArgs a) {
    const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
    int i = gtid / L;
    const bool on = i < a.N;
    if (!on) i = a.N - 1;   // surplus teams shadow the last particle, store nothing
    fwd_team<NB, L>(sc, a, i, on, gtid & (L - 1));
}

// Batched launch: team t -> (instance, particle) through the instances' first
// teams (warp aligned, so a warp never mixes instances); the instance's
// horizon, scene and buffers replace the class-wide constants.  Teams of
// stopped instances return at once.
template <int NB>
__device__ __forceinline__ bool batch_team(const SimConst& sc0, const BatchArgs& b, int t,
                                           SimConst& sc, RolloutArgs& a, int& i, bool& on) {
    if (t >= b.n_teams) return false;
    int lo = 0, hi = b.n_inst - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(&b.inst[mid].team0) <= t) lo = mid; else hi = mid - 1;
    }
    const BatchInst* in = b.inst + lo;
    if (!__ldg(&b.active[in->gid])) return false;
    sc = sc0;
    sc.H = in->H;
    sc.D = in->D;
    sc.n_ckpt = in->n_ckpt;
#pragma unroll
    for (int q = 0; q < NB; ++q)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            sc.init[q][c] = in->init[q][c];
            sc.goal[q][c] = in->goal[q][c];
        }
    a = RolloutArgs{};
    a.theta = in->theta;
    a.N = in->N;
    a.seed = in->seed;
    a.iter = b.iter_dev ? *b.iter_dev : b.iter;
    a.hard = b.hard;
    a.tape = in->tape;
    a.cost = in->cost;
    a.grad = in->grad;
    a.dropped = b.dropped;
    i = t - in->team0;
    on = i < in->N;
    if (!on) i = in->N - 1;
    return true;
}

template <int NB, int L>
__global__ void __launch_bounds__(128) rollout_fwd_batch_kernel(const SimConst sc0, const BatchArgs b) {
    const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
    SimConst sc;
    RolloutArgs a;
    int i;
    bool on;
    if (!batch_team<NB>(sc0, b, gtid / L, sc, a, i, on)) return;
    fwd_team<NB, L>(sc, a, i, on, gtid & (L - 1));
}

// ------------------------------ adjoint pieces -------------------------------
// VJP of disk_box for the weighted force (w*f, w*torque).  Inputs gFx, gFy,
// gT: adjoints of the block's force and torque.  Outputs are overwritten.
struct DiskGrad {
    float px, py, vpx, vpy, bx, by, ph, vx, vy, om, w;
};
__device__ __forceinline__ DiskGrad disk_box_vjp(const SimConst& sc, float px, float py,
                                                 float vpx, float vpy, float bx, float by,
                                                 float cph, float sph, float vx, float vy,
                                                 float om, float w, float gFx, float gFy,
                                                 float gT, bool far_check) {
    DiskGrad g = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    const float dx = px - bx, dy = py - by;
    if (far_check && dx * dx + dy * dy > sc.disk_reach2) return g;   // out of reach: no contact
    const float lx = cph * dx + sph * dy, ly = -sph * dx + cph * dy;
    const float qx = fabsf(lx) - sc.hs, qy = fabsf(ly) - sc.hs;
    const float sx = lx >= 0.f ? 1.f : -1.f, sy = ly >= 0.f ? 1.f : -1.f;
    const bool outside = qx > 0.f || qy > 0.f;
    const bool xa = qx >= qy;
    const float mx = fmaxf(qx, 0.f), my = fmaxf(qy, 0.f);
    const float il = rsqrtf(fmaxf(mx * mx + my * my, 1e-30f));
    const float ln = (mx * mx + my * my) * il;
    const float sd = outside ? ln : fmaxf(qx, qy);
    const float nlx = outside ? sx * mx * il : (xa ? sx : 0.f);
    const float nly = outside ? sy * my * il : (xa ? 0.f : sy);
    const float delta = sc.r - sd;
    if (!(delta > 0.f)) return g;
    const float nx = cph * nlx - sph * nly, ny = sph * nlx + cph * nly;
    const float rx = px - sc.r * nx - bx, ry = py - sc.r * ny - by;
    const float wx = vpx - (vx - om * ry), wy = vpy - (vy + om * rx);
    const float vn = wx * nx + wy * ny;
    const float fn = sc.k * delta - sc.c * vn;
    if (!(fn > 0.f)) return g;
    const float tx = wx - vn * nx, ty = wy - vn * ny;
    const float iden = rsqrtf(tx * tx + ty * ty + sc.eps_t2);
    const float gt = sc.mu_c * fn * iden;
    const float fx = -fn * nx + gt * tx, fy = -fn * ny + gt * ty;
    // torque T = rx*(w fy) - ry*(w fx)
    const float aFx = gFx - gT * ry, aFy = gFy + gT * rx;
    float arx = gT * (w * fy), ary = -gT * (w * fx);
    g.w = aFx * fx + aFy * fy;
    const float afx = w * aFx, afy = w * aFy;
    // f = -fn n + gt t
    float afn = -(afx * nx + afy * ny);
    float anx = -afx * fn, any = -afy * fn;
    const float agt = afx * tx + afy * ty;
    float atx = afx * gt, aty = afy * gt;
    // gt = mu_c fn / den, den = sqrt(|t|^2 + eps^2)
    afn += agt * sc.mu_c * iden;
    const float aden = -agt * gt * iden;
    atx += aden * tx * iden;
    aty += aden * ty * iden;
    // t = w - vn n
    float awx = atx, awy = aty;
    float avn = -(atx * nx + aty * ny);
    anx -= atx * vn;
    any -= aty * vn;
    // fn = k delta - c vn
    const float adelta = sc.k * afn;
    avn -= sc.c * afn;
    // vn = w . n
    awx += avn * nx;
    awy += avn * ny;
    anx += avn * wx;
    any += avn * wy;
    // w = vp - v - om x r:  wx = vpx - vx + om ry, wy = vpy - vy - om rx
    g.vpx = awx; g.vpy = awy;
    g.vx = -awx; g.vy = -awy;
    g.om = awx * ry - awy * rx;
    ary += awx * om;
    arx -= awy * om;
    // r = p - r_p n - b
    g.px = arx; g.py = ary;
    anx -= sc.r * arx;
    any -= sc.r * ary;
    g.bx = -arx; g.by = -ary;
    // n = R nl
    const float anlx = cph * anx + sph * any;
    const float anly = -sph * anx + cph * any;
    float acph = anx * nlx + any * nly;
    float asph = -anx * nly + any * nlx;
    // delta = r - sd
    const float asd = -adelta;
    // outside: through the normalised clamped offset; inside: the chosen axis
    const float aln = asd - (anlx * nlx + anly * nly) * il;
    const float amx = (sx * anlx + aln * mx) * il, amy = (sy * anly + aln * my) * il;
    const float aqx = outside ? (qx > 0.f ? amx : 0.f) : (xa ? asd : 0.f);
    const float aqy = outside ? (qy > 0.f ? amy : 0.f) : (xa ? 0.f : asd);
    const float alx = aqx * sx, aly = aqy * sy;
    const float adx = cph * alx - sph * aly, ady = sph * alx + cph * aly;
    acph += alx * dx + aly * dy;
    asph += alx * dy - aly * dx;
    g.px += adx; g.py += ady;
    g.bx -= adx; g.by -= ady;
    g.ph = -sph * acph + cph * asph;
    return g;
}

// VJP of one corner test.  gO*/gB*: adjoints of the owner's / other box's
// force and torque.  Returns the adjoints of both boxes' states.
struct CornerGrad {
    float ox, oy, oph, ovx, ovy, oom, bx, by, bph, bvx, bvy, bom;
};
__device__ __forceinline__ CornerGrad corner_vjp(const SimConst& sc, float xo, float yo,
                                                 float co, float so, float vxo, float vyo,
                                                 float omo, float xb, float yb, float cb,
                                                 float sb, float vxb, float vyb, float omb,
                                                 float clx, float cly, float gOx, float gOy,
                                                 float gOT, float gBx, float gBy, float gBT) {
    CornerGrad g = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    const float rlx = co * clx - so * cly, rly = so * clx + co * cly;
    const float kx = xo + rlx, ky = yo + rly;
    const float kvx = vxo - omo * rly, kvy = vyo + omo * rlx;
    const float dx = kx - xb, dy = ky - yb;
    if (dx * dx + dy * dy > sc.corner_reach2) return g;   // out of reach: no contact
    const float lx = cb * dx + sb * dy, ly = -sb * dx + cb * dy;
    const float qx = fabsf(lx) - sc.hs, qy = fabsf(ly) - sc.hs;
    if (!(qx < 0.f && qy < 0.f)) return g;
    const float sx = lx >= 0.f ? 1.f : -1.f, sy = ly >= 0.f ? 1.f : -1.f;
    const bool xa = qx >= qy;
    const float nlx = xa ? sx : 0.f, nly = xa ? 0.f : sy;
    const float delta = -(xa ? qx : qy);
    const float nx = cb * nlx - sb * nly, ny = sb * nlx + cb * nly;
    const float wx = kvx - (vxb - omb * dy), wy = kvy - (vyb + omb * dx);
    const float vn = wx * nx + wy * ny;
    const float fn = sc.k * delta - sc.c * vn;
    if (!(fn > 0.f)) return g;
    const float tx = wx - vn * nx, ty = wy - vn * ny;
    const float iden = rsqrtf(tx * tx + ty * ty + sc.eps_t2);
    const float gt = sc.mu_c * fn * iden;
    const float fx = fn * nx - gt * tx, fy = fn * ny - gt * ty;
    // owner: +f, torque rl x f; other: -f, torque -(d x f)
    const float afx = gOx - gBx - gOT * rly + gBT * dy;
    const float afy = gOy - gBy + gOT * rlx - gBT * dx;
    float arlx = gOT * fy, arly = -gOT * fx;
    float adx = -gBT * fy, ady = gBT * fx;
    // f = fn n - gt t
    float afn = afx * nx + afy * ny;
    float anx = afx * fn, any = afy * fn;
    const float agt = -(afx * tx + afy * ty);
    float atx = -afx * gt, aty = -afy * gt;
    afn += agt * sc.mu_c * iden;
    const float aden = -agt * gt * iden;
    atx += aden * tx * iden;
    aty += aden * ty * iden;
    float awx = atx, awy = aty;
    float avn = -(atx * nx + aty * ny);
    anx -= atx * vn;
    any -= aty * vn;
    const float adelta = sc.k * afn;
    avn -= sc.c * afn;
    awx += avn * nx;
    awy += avn * ny;
    anx += avn * wx;
    any += avn * wy;
    // w = kv - vb - omb x d:  wx = kvx - vxb + omb dy, wy = kvy - vyb - omb dx
    const float akvx = awx, akvy = awy;
    g.bvx = -awx; g.bvy = -awy;
    g.bom = awx * dy - awy * dx;
    ady += awx * omb;
    adx -= awy * omb;
    // n = R_b nl (nl constant)
    float acb = anx * nlx + any * nly;
    float asb = -anx * nly + any * nlx;
    // delta = -(q on the axis), q = |l| - hs
    const float aqx = xa ? -adelta : 0.f, aqy = xa ? 0.f : -adelta;
    const float alx = aqx * sx, aly = aqy * sy;
    adx += cb * alx - sb * aly;
    ady += sb * alx + cb * aly;
    acb += alx * dx + aly * dy;
    asb += alx * dy - aly * dx;
    // d = k - b
    float akx = adx, aky = ady;
    g.bx = -adx; g.by = -ady;
    // kv = vo + omo x rl
    g.ovx = akvx; g.ovy = akvy;
    g.oom = -akvx * rly + akvy * rlx;
    arly -= akvx * omo;
    arlx += akvy * omo;
    // k = o + rl
    g.ox = akx; g.oy = aky;
    arlx += akx;
    arly += aky;
    const float aco = arlx * clx + arly * cly, aso = -arlx * cly + arly * clx;
    g.oph = -so * aco + co * aso;
    g.bph = -sb * acb + cb * asb;
    return g;
}

// Reverse one substep: `a` holds the adjoint of the state after the substep
// on entry and of the state before it on exit; slot accumulators collect the
// adjoints of the pusher start points, displacements and weights.
template <int NB, int L>
__device__ __forceinline__ void substep_vjp(const SimConst& sc, const Blocks<NB>& s,
                                            const float (&cs)[NB], const float (&sn)[NB],
                                            const Slots<NB, L>& sl, SlotAcc<NB, L>& acc,
                                            const Corners<NB, L>& cn, float j1, Blocks<NB>& a) {
    float aFx[NB], aFy[NB], aT[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        // v1 = v + dt F/m ; p1 = p + dt v1 (likewise for the yaw)
        const float av1x = a.vx[b] + sc.dt * a.x[b];
        const float av1y = a.vy[b] + sc.dt * a.y[b];
        const float aw1 = a.om[b] + sc.dt * a.ph[b];
        aFx[b] = av1x * sc.dt * sc.inv_m;
        aFy[b] = av1y * sc.dt * sc.inv_m;
        aT[b] = aw1 * sc.dt * sc.inv_I;
        // ground friction F = -fl v/sv, T = -fa om/so
        const float vx = s.vx[b], vy = s.vy[b], om = s.om[b];
        const float isv = rsqrtf(vx * vx + vy * vy + sc.eps_v2);
        const float iso = rsqrtf(om * om + sc.eps_w2);
        const float dotv = (aFx[b] * vx + aFy[b] * vy) * (isv * isv * isv);
        a.vx[b] = av1x - sc.fric_lin * (aFx[b] * isv - vx * dotv);
        a.vy[b] = av1y - sc.fric_lin * (aFy[b] * isv - vy * dotv);
        a.om[b] = aw1 - sc.fric_ang * aT[b] * sc.eps_w2 * (iso * iso * iso);
    }
    Blocks<NB> d;
    zero(d);
#pragma unroll
    for (int q = 0; q < Slots<NB, L>::SP; ++q) {
        if (sl.c[q] < 0) continue;
        const int b = sl.b[q];
        const float px = sl.p0x[q] + j1 * sl.dx[q], py = sl.p0y[q] + j1 * sl.dy[q];
        const float bx = pick(s.x, b), by = pick(s.y, b);
        // as in substep_forces: an out-of-reach pusher on another object has
        // a zero derivative
        if (q * L >= Dims<NB>::M && out_of_reach(px - bx, py - by, sc.disk_reach2)) continue;
        const DiskGrad g = disk_box_vjp(
            sc, px, py, sl.dx[q] * sc.inv_dt, sl.dy[q] * sc.inv_dt, bx, by, pick(cs, b),
            pick(sn, b), pick(s.vx, b), pick(s.vy, b), pick(s.om, b), sl.w[q], pick(aFx, b),
            pick(aFy, b), pick(aT, b), false);
        acc.p0x[q] += g.px;
        acc.p0y[q] += g.py;
        acc.dx[q] += j1 * g.px + g.vpx * sc.inv_dt;
        acc.dy[q] += j1 * g.py + g.vpy * sc.inv_dt;
        acc.w[q] += g.w;
        add_at(d.x, b, g.bx);
        add_at(d.y, b, g.by);
        add_at(d.ph, b, g.ph);
        add_at(d.vx, b, g.vx);
        add_at(d.vy, b, g.vy);
        add_at(d.om, b, g.om);
    }
    if constexpr (Dims<NB>::NCI > 0) {
#pragma unroll
        for (int q = 0; q < Corners<NB, L>::SC; ++q) {
            if (!cn.on[q]) continue;
            const int o = cn.own[q], t = cn.oth[q];
            {   // a corner out of the other box's reach has a zero derivative
                const float co = pick(cs, o), so = pick(sn, o);
                const float clx = cn.ex[q] * sc.hs, cly = cn.ey[q] * sc.hs;
                const float kx = pick(s.x, o) + co * clx - so * cly;
                const float ky = pick(s.y, o) + so * clx + co * cly;
                if (out_of_reach(kx - pick(s.x, t), ky - pick(s.y, t), sc.corner_reach2)) continue;
            }
            const CornerGrad g = corner_vjp(
                sc, pick(s.x, o), pick(s.y, o), pick(cs, o), pick(sn, o), pick(s.vx, o),
                pick(s.vy, o), pick(s.om, o), pick(s.x, t), pick(s.y, t), pick(cs, t), pick(sn, t),
                pick(s.vx, t), pick(s.vy, t), pick(s.om, t), cn.ex[q] * sc.hs, cn.ey[q] * sc.hs,
                pick(aFx, o), pick(aFy, o), pick(aT, o), pick(aFx, t), pick(aFy, t), pick(aT, t));
            add_at(d.x, o, g.ox); add_at(d.y, o, g.oy); add_at(d.ph, o, g.oph);
            add_at(d.vx, o, g.ovx); add_at(d.vy, o, g.ovy); add_at(d.om, o, g.oom);
            add_at(d.x, t, g.bx); add_at(d.y, t, g.by); add_at(d.ph, t, g.bph);
            add_at(d.vx, t, g.bvx); add_at(d.vy, t, g.bvy); add_at(d.om, t, g.bom);
        }
    }
    team_sum<L>(d);
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        a.x[b] += d.x[b]; a.y[b] += d.y[b]; a.ph[b] += d.ph[b];
        a.vx[b] += d.vx[b]; a.vy[b] += d.vy[b]; a.om[b] += d.om[b];
    }
}

// ------------------------------ adjoint kernel --------------------------------
// seg: the team's shared memory, C states (before each substep of the current
// segment) when C > 1; teams sit seg_stride<NB>(C) float2 apart to spread
// them over banks.
template <int NB>
__host__ __device__ constexpr int seg_stride(int C) { return C * (Dims<NB>::S / 2) + 1; }

// kL2: read the tape through L2 only (a forward of the same launch wrote it).
template <int NB, int L, bool kL2 = false>
__device__ __forceinline__ void adj_team(const SimConst& sc, const RolloutArgs& a, int i, bool on,
                                         int lane, float2* seg) {
    constexpr int M = Dims<NB>::M, P = Dims<NB>::P, S = Dims<NB>::S, SP = Slots<NB, L>::SP;
    auto load_tape = [](const float2* src, Blocks<NB>& st) {
        if constexpr (kL2) load_state_cg(src, st); else load_state(src, st);
    };
    const float* th = a.theta + (size_t)i * sc.D;
    float* gr = a.grad + (size_t)i * sc.D;
    const bool noise = a.iter >= 0;
    const bool hard = a.hard != 0;
    const uint64_t gkey = noise ? sm64(sm64(a.seed, kStreamGumbel), (uint64_t)a.iter) : 0ull;
    const size_t ck2 = (size_t)a.N * (S / 2);   // float2 per checkpoint
    const float2* tape_i = reinterpret_cast<const float2*>(a.tape + (size_t)i * S);

    Corners<NB, L> cn;
    make_corners(cn, lane);
    Blocks<NB> s, adj;
    load_tape(tape_i + (size_t)sc.n_ckpt * ck2, s);
    zero(adj);
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        // C = sum |p - g|^2 + w_yaw wrap(yaw - yaw_g)^2 (+ push term, below)
        adj.x[b] = 2.f * (s.x[b] - sc.goal[b][0]);
        adj.y[b] = 2.f * (s.y[b] - sc.goal[b][1]);
        adj.ph[b] = 2.f * sc.w_yaw * wrapf(s.ph[b] - sc.goal[b][2]);
    }
    const int segs = sc.T / sc.C;
    bool bad = false;
    for (int k = sc.H - 1; k >= 0; --k) {
        Blocks<NB> s0;
        load_tape(tape_i + (size_t)(k * segs) * ck2, s0);
        float z[M], uu, vv;
        relax_action<NB>(sc, th, k, i + a.particle0, gkey, noise, hard, z, uu, vv);
        const float tu = tanhf(uu);
        const float off = sc.off_max * tu;
        const float sg = sigmoidf_(vv);
        const float dist = sc.dist_max * sg;
        Slots<NB, L> sl;
        make_slots<NB, L>(sc, s0, lane, z, off, dist, sl);
        SlotAcc<NB, L> acc;
#pragma unroll
        for (int q = 0; q < SP; ++q) acc.p0x[q] = acc.p0y[q] = acc.dx[q] = acc.dy[q] = acc.w[q] = 0.f;

        Blocks<NB> nxt;
        load_tape(tape_i + (size_t)(k * segs + segs - 1) * ck2, nxt);
        // with a replayed tape, the yaws' (cos, sin) come with the states
        const bool have_trig = sc.C == 1 && a.trig != nullptr;
        const size_t ckt = (size_t)a.N * NB;                         // float2 per trig row
        const float2* trig_i = have_trig ? a.trig + (size_t)i * NB : nullptr;
        float ncs[NB], nsn[NB];
        if (have_trig) load_trig<NB>(trig_i + (size_t)(k * segs + segs - 1) * ckt, ncs, nsn);
        for (int sgi = segs - 1; sgi >= 0; --sgi) {
            s = nxt;
            float cs[NB], sn[NB];
            if (have_trig)
#pragma unroll
                for (int b = 0; b < NB; ++b) { cs[b] = ncs[b]; sn[b] = nsn[b]; }
            // prefetch the previous checkpoint; its latency hides behind this
            // segment (nothing here touches it before the next iteration: warps
            // issue in order, so an early use would stall on the load)
            if (sgi > 0) {
                load_tape(tape_i + (size_t)(k * segs + sgi - 1) * ck2, nxt);
                if (have_trig) load_trig<NB>(trig_i + (size_t)(k * segs + sgi - 1) * ckt, ncs, nsn);
            }
            if (sc.C == 1) {   // every state is on the tape: nothing to recompute
                if (!have_trig) trig(s, cs, sn);
                substep_vjp<NB, L>(sc, s, cs, sn, sl, acc, cn, (float)(sgi + 1), adj);
                continue;
            }
            // recompute the segment forward, keeping the state before each substep
            for (int jj = 0; jj < sc.C; ++jj) {
                store_state<NB, L>(seg + jj * (S / 2), s, lane, true);
                if (jj + 1 < sc.C) {
                    float cs[NB], sn[NB];
                    trig(s, cs, sn);
                    float Fx[NB], Fy[NB], Tq[NB];
                    substep_forces<NB, L>(sc, s, cs, sn, sl, cn, (float)(sgi * sc.C + jj + 1), Fx,
                                          Fy, Tq);
                    integrate(sc, s, Fx, Fy, Tq);
                }
            }
            __syncwarp();
            for (int jj = sc.C - 1; jj >= 0; --jj) {
                load_state(seg + jj * (S / 2), s);
                float cs[NB], sn[NB];
                trig(s, cs, sn);
                substep_vjp<NB, L>(sc, s, cs, sn, sl, acc, cn, (float)(sgi * sc.C + jj + 1), adj);
            }
            __syncwarp();
        }

        // Action start: p0 = pos_o + R(yaw_o) (n (hs+r) + t off), delta = -R(yaw_o) n dist/T.
        Blocks<NB> d;
        zero(d);
        float az[M];
#pragma unroll
        for (int c = 0; c < M; ++c) az[c] = 0.f;
        float aoff = 0.f, adist = 0.f;
        const float step = dist / (float)sc.T;
#pragma unroll
        for (int q = 0; q < SP; ++q) {
            if (sl.c[q] < 0) continue;
            const int c = sl.c[q], o = c / 4, side = c % 4;
            float nx, ny;
            side_normal(side, nx, ny);
            const float tx = -ny, ty = nx;
            const float lx = nx * (sc.hs + sc.r) + tx * off;
            const float ly = ny * (sc.hs + sc.r) + ty * off;
            float cph, sph;
            yaw_sincos(pick(s0.ph, o), &sph, &cph);
            const float ap0x = acc.p0x[q], ap0y = acc.p0y[q], adx = acc.dx[q], ady = acc.dy[q];
            add_at(d.x, o, ap0x);
            add_at(d.y, o, ap0y);
            // d(R v)/dyaw = (-s vx - c vy, c vx - s vy)
            const float dRl_x = -sph * lx - cph * ly, dRl_y = cph * lx - sph * ly;
            const float dRn_x = -sph * nx - cph * ny, dRn_y = cph * nx - sph * ny;
            add_at(d.ph, o, ap0x * dRl_x + ap0y * dRl_y - (adx * dRn_x + ady * dRn_y) * step);
            // local offset adjoint R^T ap0, projected on t
            const float alx = cph * ap0x + sph * ap0y, aly = -sph * ap0x + cph * ap0y;
            aoff += alx * tx + aly * ty;
            const float ux = -(cph * nx - sph * ny), uy = -(sph * nx + cph * ny);
            adist += (adx * ux + ady * uy) / (float)sc.T;
            add_at(az, c, acc.w[q]);
        }
        team_sum<L>(d.x);
        team_sum<L>(d.y);
        team_sum<L>(d.ph);
        team_sum<L>(az);
        aoff = team_sum<L>(aoff);
        adist = team_sum<L>(adist);
#pragma unroll
        for (int b = 0; b < NB; ++b) { adj.x[b] += d.x[b]; adj.y[b] += d.y[b]; adj.ph[b] += d.ph[b]; }
        adist += 2.f * sc.w_push * dist;
        // softmax((a+g)/tau) backward; the one-hot of the hard map has no gradient
        float zaz = 0.f;
#pragma unroll
        for (int c = 0; c < M; ++c) zaz += z[c] * az[c];
        if (on) {
#pragma unroll
            for (int c = 0; c < M; ++c)
                if ((c % L) == lane) {
                    const float gv = hard ? 0.f : -(z[c] * (az[c] - zaz) * sc.inv_tau);
                    gr[k * P + c] = gv;
                    bad |= !isfinite(gv);
                }
            if (lane == (M % L)) {
                const float gv = -(aoff * sc.off_max * (1.f - tu * tu));
                gr[k * P + M] = gv;
                bad |= !isfinite(gv);
            }
            if (lane == ((M + 1) % L)) {
                const float gv = -(adist * sc.dist_max * sg * (1.f - sg));
                gr[k * P + M + 1] = gv;
                bad |= !isfinite(gv);
            }
        }
    }
    // A reverse sweep that overflowed float32 (exploding gradient through the
    // contact dynamics) gives the particle a zero gradient, and is counted.
    bad = team_sum<L>(bad ? 1.f : 0.f) > 0.f;
    if (on && bad) {
        for (int d = lane; d < sc.D; d += L) gr[d] = 0.f;
        if (lane == 0 && a.dropped) atomicAdd(a.dropped, 1ull);
    }
}

template <int NB, int L>
__global__ void __launch_bounds__(128) rollout_adj_kernel(const SimConst sc, const RolloutArgs a) {
    const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
    int i = gtid / L;
    const bool on = i < a.N;
    if (!on) i = a.N - 1;
    extern __shared__ float2 seg_smem[];
    adj_team<NB, L>(sc, a, i, on, gtid & (L - 1),
                    seg_smem + (size_t)(threadIdx.x / L) * seg_stride<NB>(sc.C));
}

template <int NB, int L>
__global__ void __launch_bounds__(128) rollout_adj_batch_kernel(const SimConst sc0, const BatchArgs b) {
    const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
    SimConst sc;
    RolloutArgs a;
    int i;
    bool on;
    if (!batch_team<NB>(sc0, b, gtid / L, sc, a, i, on)) return;
    extern __shared__ float2 seg_smem[];
    adj_team<NB, L>(sc, a, i, on, gtid & (L - 1),
                    seg_smem + (size_t)(threadIdx.x / L) * seg_stride<NB>(sc.C));
}

// ------------------------------ segment replay --------------------------------
// The checkpointed reverse sweep needs the state before every substep.  The
// replay rebuilds them for all (particle, segment) pairs at once: team
// t = g*N + i recomputes segment g (of the H*T/C) of particle i from its
// checkpoint, with the action's relaxation and pushers placed from the
// action-start checkpoint exactly as the forward placed them, and writes the
// C states before its substeps into `full`, laid out [H*T + 1][N][S] like a
// tape of interval 1 (the last segment's team adds the final state).  What
// stays serial per particle is the sweep over that tape; the recomputation
// runs as one throughput-bound launch.
template <int NB, int L>
__global__ void __launch_bounds__(128) replay_kernel(const SimConst sc, const RolloutArgs a,
                                                     float* __restrict__ full) {
    constexpr int M = Dims<NB>::M, S = Dims<NB>::S;
    const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = (int)(gtid & (L - 1));
    const long long teams = (long long)a.N * sc.n_ckpt;
    long long t = gtid / L;
    const bool on = t < teams;
    if (!on) t = teams - 1;   // surplus teams shadow the last pair, store nothing
    const int g = (int)(t / a.N), i = (int)(t % a.N);
    const int segs = sc.T / sc.C, k = g / segs, sg = g % segs;
    const size_t ck2 = (size_t)a.N * (S / 2);   // float2 per tape row
    const float2* tape_i = reinterpret_cast<const float2*>(a.tape + (size_t)i * S);
    float2* full_i = reinterpret_cast<float2*>(full + (size_t)i * S);
    const bool noise = a.iter >= 0;
    const uint64_t gkey = noise ? sm64(sm64(a.seed, kStreamGumbel), (uint64_t)a.iter) : 0ull;

    Blocks<NB> s0, s;
    load_state(tape_i + (size_t)(k * segs) * ck2, s0);
    load_state(tape_i + (size_t)g * ck2, s);
    float z[M], uu, vv;
    relax_action<NB>(sc, a.theta + (size_t)i * sc.D, k, i + a.particle0, gkey, noise,
                     a.hard != 0, z, uu, vv);
    Slots<NB, L> sl;
    make_slots<NB, L>(sc, s0, lane, z, sc.off_max * tanhf(uu), sc.dist_max * sigmoidf_(vv), sl);
    Corners<NB, L> cn;
    make_corners(cn, lane);
    const int t0 = k * sc.T + sg * sc.C;   // the segment's first substep
    float2* trig_i = a.trig ? a.trig + (size_t)i * NB : nullptr;
    const size_t ckt = (size_t)a.N * NB;
    for (int jj = 0; jj < sc.C; ++jj) {
        store_state<NB, L>(full_i + (size_t)(t0 + jj) * ck2, s, lane, on);
        float cs[NB], sn[NB];
        trig(s, cs, sn);
        if (trig_i) store_trig<NB, L>(trig_i + (size_t)(t0 + jj) * ckt, cs, sn, lane, on);
        if (jj + 1 == sc.C) break;          // the state after it is the next checkpoint
        float Fx[NB], Fy[NB], Tq[NB];
        substep_forces<NB, L>(sc, s, cs, sn, sl, cn, (float)(sg * sc.C + jj + 1), Fx, Fy, Tq);
        integrate(sc, s, Fx, Fy, Tq);
    }
    if (g == sc.n_ckpt - 1) {
        load_state(tape_i + (size_t)sc.n_ckpt * ck2, s);
        store_state<NB, L>(full_i + (size_t)(sc.H * sc.T) * ck2, s, lane, on);
    }
}

template <int NB, int L>
cudaError_t launch_replay(const SimConst& sc, const RolloutArgs& a, float* full, cudaStream_t st) {
    const long long threads_total = (long long)a.N * sc.n_ckpt * L;
    const int cta = 128;
    const long long grid = (threads_total + cta - 1) / cta;
    if (grid > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    replay_kernel<NB, L><<<(unsigned)grid, cta, 0, st>>>(sc, a, full);
    return cudaGetLastError();
}

// ------------------------------ launch --------------------------------------
template <int NB, int L>
cudaError_t launch(const SimConst& sc, const RolloutArgs& a, bool adjoint, cudaStream_t st) {
    const long long threads_total = (long long)a.N * L;
    // spread over the SMs: small CTAs when there are few particles
    const int sms = sm_count();
    int cta = 32;
    while (cta < 128 && threads_total / (cta * 2) >= sms) cta *= 2;
    const int grid = (int)((threads_total + cta - 1) / cta);
    if (!adjoint) {
        rollout_fwd_kernel<NB, L><<<grid, cta, 0, st>>>(sc, a);
    } else {
        const size_t smem = (size_t)(cta / L) * (sc.C * (Dims<NB>::S / 2) + 1) * sizeof(float2);
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(rollout_adj_kernel<NB, L>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)smem);
            if (e != cudaSuccess) return e;
        }
        rollout_adj_kernel<NB, L><<<grid, cta, smem, st>>>(sc, a);
    }
    return cudaGetLastError();
}

// Batched launch of one block-count class: b.n_teams teams of L lanes in
// CTAs of `cta` threads (a multiple of 32).
template <int NB, int L>
cudaError_t launch_batch(const SimConst& sc, const BatchArgs& b, int cta, bool adjoint, cudaStream_t st) {
    const long long threads_total = (long long)b.n_teams * L;
    const int grid = (int)((threads_total + cta - 1) / cta);
    if (grid < 1) return cudaSuccess;
    if (!adjoint) {
        rollout_fwd_batch_kernel<NB, L><<<grid, cta, 0, st>>>(sc, b);
    } else {
        const size_t smem = (size_t)(cta / L) * (sc.C * (Dims<NB>::S / 2) + 1) * sizeof(float2);
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(rollout_adj_batch_kernel<NB, L>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)smem);
            if (e != cudaSuccess) return e;
        }
        rollout_adj_batch_kernel<NB, L><<<grid, cta, smem, st>>>(sc, b);
    }
    return cudaGetLastError();
}

}  // namespace rollout
}  // namespace stamp
