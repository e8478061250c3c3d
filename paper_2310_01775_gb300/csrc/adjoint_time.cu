// Reverse sweep of the one-block rollout as a linear recurrence in time
// (Sec. III-B: grad log rho back-propagated through the whole trajectory).
//
// One semi-implicit Euler substep maps the state s = (x, y, ph, vx, vy, om)
// through the block's total force and torque F(s) = (F_x, F_y, T) -- the M
// relaxed-weighted pushers' contact plus ground friction:
//   v1 = v + dt F_xy/m,  om1 = om + dt T/I,  p1 = p + dt v1,  ph1 = ph + dt om1.
// Its adjoint is linear in the adjoint a of the state after the substep:
//   av1 = (a_vx + dt a_x, a_vy + dt a_y, a_om + dt a_ph),
//   a_before = (a_x, a_y, a_ph, av1) + M_t^T av1,
//   M_t = diag(dt/m, dt/m, dt/I) dF/ds (s_t)                       (3 x 6),
// and the action parameters' adjoints collect linear forms E_t av1: the
// pushers' start point and displacement (through the action-start pose),
// the offset, the distance, and each choice's weight (its unweighted force).
// M_t and E_t depend on the forward states only.  With every state on the
// tape (checkpoint interval 1) they are computed for all (particle, substep)
// pairs at once (jac_kernel: throughput bound, the whole GPU busy); what
// stays serial per particle is the recurrence itself, a few dependent FMAs
// per substep (scan_kernel, its coefficients streamed into shared memory by
// TMA bulk copies a window ahead).
//
// The contact Jacobian takes disk_box_vjp's forward and reverse passes (the
// sequential sweep's derivative of the contact) once forward and twice in
// reverse per pusher -- the force rows -- and the torque row by linearity,
// so both sweeps take the same derivatives and differ only in rounding.
#include "async_copy.cuh"
#include "rollout.cuh"

namespace stamp {
namespace rollout {
namespace {

// Coefficient row of one (particle, substep): 44 floats (176 B):
//   [0, 18)   M, row m (F_x, F_y, T) of 6 state columns
//   [18, 20)  zero
//   [20 + 6l, 26 + 6l), l = 0..3: the scan's lane l reads form l -- the
//             action-start yaw (l = 0), offset (1), distance (2), none
//             (3: zero) -- then the weight form of choice l (3 floats each)
// Rows are grouped [particle / 8][substep][particle % 8]: a scan CTA's
// window of substeps is one contiguous span.
constexpr int kRow = 44, kE = 20;
constexpr int kGroup = 8;      // particles per coefficient group (= per scan CTA)
constexpr int kWin = 32;       // substeps per staged window of the scan
constexpr int kRel = 6;        // relaxed parameters per action: z_0..z_3, tanh(u), sigmoid(v)

// Item q's weighted contact Jacobian (rows F_x, F_y, T; columns the state)
// and its forms, at one substep, per unit adjoint of each force component.
struct ItemJac {
    float J[3][6];
    float eph[3], eoff[3], edist[3], ew[3];
};

// disk_box's forward quantities (unweighted force), as disk_box_vjp forms
// them; active = the pusher touches the block with a compressive force.
struct DiskFwd {
    float dx, dy, qx, qy, sx, sy, mx, my, il, nlx, nly;
    float nx, ny, rx, ry, wx, wy, vn, fn, tx, ty, iden, gt, fx, fy;
    bool outside, xa, active;
};

__device__ __forceinline__ DiskFwd disk_fwd(const SimConst& sc, float px, float py, float vpx,
                                            float vpy, float bx, float by, float cph, float sph,
                                            float vx, float vy, float om) {
    DiskFwd f;
    f.active = false;
    f.dx = px - bx;
    f.dy = py - by;
    const float lx = cph * f.dx + sph * f.dy, ly = -sph * f.dx + cph * f.dy;
    f.qx = fabsf(lx) - sc.hs;
    f.qy = fabsf(ly) - sc.hs;
    f.sx = lx >= 0.f ? 1.f : -1.f;
    f.sy = ly >= 0.f ? 1.f : -1.f;
    f.outside = f.qx > 0.f || f.qy > 0.f;
    f.xa = f.qx >= f.qy;
    f.mx = fmaxf(f.qx, 0.f);
    f.my = fmaxf(f.qy, 0.f);
    f.il = rsqrtf(fmaxf(f.mx * f.mx + f.my * f.my, 1e-30f));
    const float ln = (f.mx * f.mx + f.my * f.my) * f.il;
    const float sd = f.outside ? ln : fmaxf(f.qx, f.qy);
    f.nlx = f.outside ? f.sx * f.mx * f.il : (f.xa ? f.sx : 0.f);
    f.nly = f.outside ? f.sy * f.my * f.il : (f.xa ? 0.f : f.sy);
    const float delta = sc.r - sd;
    if (!(delta > 0.f)) return f;
    f.nx = cph * f.nlx - sph * f.nly;
    f.ny = sph * f.nlx + cph * f.nly;
    f.rx = px - sc.r * f.nx - bx;
    f.ry = py - sc.r * f.ny - by;
    f.wx = vpx - (vx - om * f.ry);
    f.wy = vpy - (vy + om * f.rx);
    f.vn = f.wx * f.nx + f.wy * f.ny;
    f.fn = sc.k * delta - sc.c * f.vn;
    if (!(f.fn > 0.f)) return f;
    f.tx = f.wx - f.vn * f.nx;
    f.ty = f.wy - f.vn * f.ny;
    f.iden = rsqrtf(f.tx * f.tx + f.ty * f.ty + sc.eps_t2);
    f.gt = sc.mu_c * f.fn * f.iden;
    f.fx = -f.fn * f.nx + f.gt * f.tx;
    f.fy = -f.fn * f.ny + f.gt * f.ty;
    f.active = true;
    return f;
}

// Adjoints of the pusher position and velocity, the block yaw and spin, for
// the adjoint (afx, afy) of the weighted contact force and (arx, ary) of the
// lever arm r = x_c - b (the torque's part) -- disk_box_vjp's reverse pass.
// The block position and velocity get the negated pusher ones.
struct DiskAdj {
    float px, py, vpx, vpy, ph, om;
};
// The reverse pass through the normal n = R nl and the penetration depth,
// from the adjoints (anx, any) of n and asd of the signed distance.
__device__ __forceinline__ DiskAdj disk_bwd_geometry(const DiskFwd& f, float cph, float sph,
                                                     float anx, float any, float asd, DiskAdj g) {
    const float anlx = cph * anx + sph * any;
    const float anly = -sph * anx + cph * any;
    float acph = anx * f.nlx + any * f.nly;
    float asph = -anx * f.nly + any * f.nlx;
    // outside: through the normalised clamped offset; inside: the chosen axis
    const float aln = asd - (anlx * f.nlx + anly * f.nly) * f.il;
    const float amx = (f.sx * anlx + aln * f.mx) * f.il, amy = (f.sy * anly + aln * f.my) * f.il;
    const float aqx = f.outside ? (f.qx > 0.f ? amx : 0.f) : (f.xa ? asd : 0.f);
    const float aqy = f.outside ? (f.qy > 0.f ? amy : 0.f) : (f.xa ? 0.f : asd);
    const float alx = aqx * f.sx, aly = aqy * f.sy;
    const float adx = cph * alx - sph * aly, ady = sph * alx + cph * aly;
    acph += alx * f.dx + aly * f.dy;
    asph += alx * f.dy - aly * f.dx;
    g.px += adx;
    g.py += ady;
    g.ph = -sph * acph + cph * asph;
    return g;
}

__device__ __forceinline__ DiskAdj disk_bwd(const SimConst& sc, const DiskFwd& f, float cph,
                                            float sph, float om, float afx, float afy, float arx,
                                            float ary) {
    DiskAdj g;
    // f = -fn n + gt t
    float afn = -(afx * f.nx + afy * f.ny);
    float anx = -afx * f.fn, any = -afy * f.fn;
    const float agt = afx * f.tx + afy * f.ty;
    float atx = afx * f.gt, aty = afy * f.gt;
    // gt = mu_c fn / den, den = sqrt(|t|^2 + eps^2)
    afn += agt * sc.mu_c * f.iden;
    const float aden = -agt * f.gt * f.iden;
    atx += aden * f.tx * f.iden;
    aty += aden * f.ty * f.iden;
    // t = w - vn n
    float awx = atx, awy = aty;
    float avn = -(atx * f.nx + aty * f.ny);
    anx -= atx * f.vn;
    any -= aty * f.vn;
    // fn = k delta - c vn
    const float adelta = sc.k * afn;
    avn -= sc.c * afn;
    // vn = w . n
    awx += avn * f.nx;
    awy += avn * f.ny;
    anx += avn * f.wx;
    any += avn * f.wy;
    // w = vp - v - om x r
    g.vpx = awx;
    g.vpy = awy;
    g.om = awx * f.ry - awy * f.rx;
    ary += awx * om;
    arx -= awy * om;
    // r = p - r_p n - b
    g.px = arx;
    g.py = ary;
    anx -= sc.r * arx;
    any -= sc.r * ary;
    return disk_bwd_geometry(f, cph, sph, anx, any, -adelta, g);
}
__device__ __forceinline__ void item_jac(const SimConst& sc, const Blocks<1>& s, float cs, float sn,
                                         int q, float p0x, float p0y, float dxq, float dyq,
                                         float w, float j1, float step, float cph0, float sph0,
                                         float off, ItemJac& o) {
    const float px = p0x + j1 * dxq, py = p0y + j1 * dyq;
    const float vpx = dxq * sc.inv_dt, vpy = dyq * sc.inv_dt;
    const DiskFwd f = disk_fwd(sc, px, py, vpx, vpy, s.x[0], s.y[0], cs, sn, s.vx[0], s.vy[0],
                               s.om[0]);
    if (!f.active) {
#pragma unroll
        for (int m = 0; m < 3; ++m) {
#pragma unroll
            for (int c = 0; c < 6; ++c) o.J[m][c] = 0.f;
            o.eph[m] = o.eoff[m] = o.edist[m] = o.ew[m] = 0.f;
        }
        return;
    }
    // rows F_x, F_y: unit force adjoints; row T: the torque r x f adjoint is
    // (-ry, rx) on the force plus (w fy, -w fx) on the lever arm, and the
    // reverse pass is linear -- so row T = -ry row F_x + rx row F_y + the
    // lever-arm-only pass
    DiskAdj g[3];
    g[0] = disk_bwd(sc, f, cs, sn, s.om[0], w, 0.f, 0.f, 0.f);
    g[1] = disk_bwd(sc, f, cs, sn, s.om[0], 0.f, w, 0.f, 0.f);
    {
        DiskAdj r;
        r.px = w * f.fy;
        r.py = -w * f.fx;
        r.vpx = r.vpy = r.om = 0.f;
        r = disk_bwd_geometry(f, cs, sn, -sc.r * r.px, -sc.r * r.py, 0.f, r);
        g[2].px = -f.ry * g[0].px + f.rx * g[1].px + r.px;
        g[2].py = -f.ry * g[0].py + f.rx * g[1].py + r.py;
        g[2].vpx = -f.ry * g[0].vpx + f.rx * g[1].vpx;
        g[2].vpy = -f.ry * g[0].vpy + f.rx * g[1].vpy;
        g[2].ph = -f.ry * g[0].ph + f.rx * g[1].ph + r.ph;
        g[2].om = -f.ry * g[0].om + f.rx * g[1].om;
    }
    const float gw[3] = {f.fx, f.fy, f.rx * f.fy - f.ry * f.fx};   // unweighted force, torque
    // pusher start point p0 = pos + R l and displacement -R n dist/T at the action start
    float nx, ny;
    side_normal(q, nx, ny);
    const float tx = -ny, ty = nx;
    const float lx = nx * (sc.hs + sc.r) + tx * off;
    const float ly = ny * (sc.hs + sc.r) + ty * off;
    const float dRl_x = -sph0 * lx - cph0 * ly, dRl_y = cph0 * lx - sph0 * ly;
    const float dRn_x = -sph0 * nx - cph0 * ny, dRn_y = cph0 * nx - sph0 * ny;
    const float ux = -(cph0 * nx - sph0 * ny), uy = -(sph0 * nx + cph0 * ny);
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        o.J[m][0] = -g[m].px;   // the block position enters as -p
        o.J[m][1] = -g[m].py;
        o.J[m][2] = g[m].ph;
        o.J[m][3] = -g[m].vpx;  // the block velocity enters as -vp
        o.J[m][4] = -g[m].vpy;
        o.J[m][5] = g[m].om;
        const float adx = j1 * g[m].px + g[m].vpx * sc.inv_dt;
        const float ady = j1 * g[m].py + g[m].vpy * sc.inv_dt;
        o.eph[m] = g[m].px * dRl_x + g[m].py * dRl_y - (adx * dRn_x + ady * dRn_y) * step;
        o.eoff[m] = (cph0 * g[m].px + sph0 * g[m].py) * tx + (-sph0 * g[m].px + cph0 * g[m].py) * ty;
        o.edist[m] = (adx * ux + ady * uy) / (float)sc.T;
        o.ew[m] = gw[m];
    }
}

// Ground friction -fl v/sqrt(|v|^2+eps_v^2), -fa om/sqrt(om^2+eps_w^2): its
// part of the Jacobian.
__device__ __forceinline__ void friction_jac(const SimConst& sc, const Blocks<1>& s,
                                             float (&J)[3][6]) {
    const float vx = s.vx[0], vy = s.vy[0], om = s.om[0];
    const float isv = rsqrtf(vx * vx + vy * vy + sc.eps_v2);
    const float iso = rsqrtf(om * om + sc.eps_w2);
    const float isv3 = isv * isv * isv;
    J[0][3] -= sc.fric_lin * (isv - vx * vx * isv3);
    J[1][3] += sc.fric_lin * vx * vy * isv3;
    J[0][4] += sc.fric_lin * vx * vy * isv3;
    J[1][4] -= sc.fric_lin * (isv - vy * vy * isv3);
    J[2][5] -= sc.fric_ang * sc.eps_w2 * (iso * iso * iso);
}

__device__ __forceinline__ float* coef_row(float* coef, int HT, int i, int t) {
    return coef + (((size_t)(i / kGroup) * HT + t) * kGroup + i % kGroup) * kRow;
}

// The coefficient row of one (particle, substep) from its state (with the
// yaw's cos/sin) and its action's pushers (start point, displacement and
// weight of the four items; cos/sin of the start yaw; offset).
__device__ __forceinline__ void pair_row(const SimConst& sc, const Blocks<1>& s, float cs, float sn,
                                         const float (&p0x)[4], const float (&p0y)[4],
                                         const float (&dx)[4], const float (&dy)[4],
                                         const float (&w)[4], float j1, float step, float cph0,
                                         float sph0, float off, float (&row)[kRow]) {
    float J[3][6], eph[3], eoff[3], edist[3], ew[4][3];
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        eph[m] = eoff[m] = edist[m] = 0.f;
#pragma unroll
        for (int c = 0; c < 6; ++c) J[m][c] = 0.f;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {   // choice q pushes side q of the block
        ItemJac o;
        item_jac(sc, s, cs, sn, q, p0x[q], p0y[q], dx[q], dy[q], w[q], j1, step, cph0, sph0, off, o);
#pragma unroll
        for (int m = 0; m < 3; ++m) {
#pragma unroll
            for (int c = 0; c < 6; ++c) J[m][c] += o.J[m][c];
            eph[m] += o.eph[m];
            eoff[m] += o.eoff[m];
            edist[m] += o.edist[m];
            ew[q][m] = o.ew[m];
        }
    }
    friction_jac(sc, s, J);
    const float cm[3] = {sc.dt * sc.inv_m, sc.dt * sc.inv_m, sc.dt * sc.inv_I};
#pragma unroll
    for (int m = 0; m < 3; ++m) {
#pragma unroll
        for (int c = 0; c < 6; ++c) row[6 * m + c] = cm[m] * J[m][c];
        row[kE + m] = cm[m] * eph[m];
        row[kE + 6 + m] = cm[m] * eoff[m];
        row[kE + 12 + m] = cm[m] * edist[m];
        row[kE + 18 + m] = 0.f;
#pragma unroll
        for (int q = 0; q < 4; ++q) row[kE + 6 * q + 3 + m] = cm[m] * ew[q][m];
    }
    row[18] = row[19] = 0.f;
}

// Relaxed parameters of every (particle, action), as the forward computed them.
__global__ void relax_kernel(const SimConst sc, const RolloutArgs a, float* __restrict__ rel) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= a.N * sc.H) return;
    const int i = idx % a.N, k = idx / a.N;
    const bool noise = a.iter >= 0;
    const uint64_t gkey = noise ? sm64(sm64(a.seed, kStreamGumbel), (uint64_t)a.iter) : 0ull;
    float z[4], uu, vv;
    relax_action<1>(sc, a.theta + (size_t)i * sc.D, k, i + a.particle0, gkey, noise, a.hard != 0,
                    z, uu, vv);
    float* r = rel + (size_t)k * kRel * a.N + i;
    r[0] = z[0];
    r[a.N] = z[1];
    r[2 * a.N] = z[2];
    r[3 * a.N] = z[3];
    r[4 * a.N] = tanhf(uu);
    r[5 * a.N] = sigmoidf_(vv);
}

// The coefficients of particle i at substep t from the tape, one thread per (i, t).
__global__ void __launch_bounds__(128) jac_kernel(const SimConst sc, const RolloutArgs a,
                                                  const float* __restrict__ rel,
                                                  float* __restrict__ coef) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int HT = sc.H * sc.T;
    if (idx >= (long long)a.N * HT) return;
    const int i = (int)(idx % a.N), t = (int)(idx / a.N);
    const int k = t / sc.T, j = t - k * sc.T;
    const size_t ck2 = (size_t)a.N * 3;   // float2 per checkpoint (S = 6)
    const float2* tape = reinterpret_cast<const float2*>(a.tape) + (size_t)i * 3;
    Blocks<1> s, s0;
    load_state(tape + (size_t)t * ck2, s);
    load_state(tape + (size_t)(k * sc.T) * ck2, s0);   // the action's start
    const float* r = rel + (size_t)k * kRel * a.N + i;
    const float z[4] = {r[0], r[a.N], r[2 * a.N], r[3 * a.N]};
    const float off = sc.off_max * r[4 * a.N];
    const float dist = sc.dist_max * r[5 * a.N];
    Slots<1, 1> sl;
    make_slots<1, 1>(sc, s0, 0, z, off, dist, sl);
    float cs[1], sn[1];
    trig(s, cs, sn);
    float cph0, sph0;
    yaw_sincos(s0.ph[0], &sph0, &cph0);
    const float j1 = (float)(j + 1), step = dist / (float)sc.T;
    float row[kRow];
    pair_row(sc, s, cs[0], sn[0], sl.p0x, sl.p0y, sl.dx, sl.dy, sl.w, j1, step, cph0, sph0, off, row);
    float4* out = reinterpret_cast<float4*>(coef_row(coef, HT, i, t));
#pragma unroll
    for (int v = 0; v < kRow / 4; ++v)
        out[v] = make_float4(row[4 * v], row[4 * v + 1], row[4 * v + 2], row[4 * v + 3]);
}

// Bounded wait on an mbarrier phase by a whole warp (false: gave up).
__device__ __forceinline__ bool warp_wait(uint64_t* bar, unsigned parity) {
    bool ok;
    unsigned spins = 0;
    while (!(ok = async::mbar_try_wait(bar, parity)) && ++spins < async::kWaitLimit) {
    }
    return __all_sync(0xffffffffu, ok);
}

// One lane's coefficients of one substep in a staged window (row base = the
// lane's particle): M and the lane's two forms.
struct Coefs {
    float4 c0, c1, c2, c3;
    float2 c4, e0, e1, e2;
};
__device__ __forceinline__ Coefs load_coefs(const float* base, int dt, int lane) {
    const float* c = base + (size_t)dt * kGroup * kRow;
    Coefs r;
    r.c0 = *reinterpret_cast<const float4*>(c);
    r.c1 = *reinterpret_cast<const float4*>(c + 4);
    r.c2 = *reinterpret_cast<const float4*>(c + 8);
    r.c3 = *reinterpret_cast<const float4*>(c + 12);
    r.c4 = *reinterpret_cast<const float2*>(c + 16);
    const float2* eb = reinterpret_cast<const float2*>(c + kE + 6 * lane);
    r.e0 = eb[0];
    r.e1 = eb[1];
    r.e2 = eb[2];
    return r;
}

// The recurrence, backwards over the H*T substeps: one CTA of 8 particles,
// a team of 4 lanes per particle.  Every lane carries the state adjoint
// (redundantly); lane l also accumulates form l and choice l's weight form.
// Window w of the coefficients is copied into buffer w%2 while window w-1 is
// consumed.
struct ScanSmem {
    uint64_t bar[2];
    float pad[28];   // the buffers start 128 B in
    float buf[2][kWin * kGroup * kRow];
};

__global__ void __launch_bounds__(32) scan_kernel(const SimConst sc, const RolloutArgs a,
                                                  const float* __restrict__ rel,
                                                  const float* __restrict__ coef,
                                                  int* __restrict__ flag) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    ScanSmem& sm = *reinterpret_cast<ScanSmem*>(smem_raw);
    const int tid = threadIdx.x, p = tid >> 2, lane = tid & 3;
    const int grp = blockIdx.x;
    int i = grp * kGroup + p;
    const bool on = i < a.N;
    if (!on) i = a.N - 1;   // surplus team: shadows the last particle, writes nothing
    const int T = sc.T, HT = sc.H * sc.T;
    const int nwin = (HT + kWin - 1) / kWin;
    const float* cgrp = coef + (size_t)grp * HT * kGroup * kRow;
    // window w covers substeps [lo(w), hi(w)), counted from the end
    auto lo = [&](int w) { return max(0, HT - (w + 1) * kWin); };
    auto hi = [&](int w) { return HT - w * kWin; };
    auto issue = [&](int w) {
        const unsigned bytes = (unsigned)((hi(w) - lo(w)) * kGroup * kRow * sizeof(float));
        async::mbar_expect_tx(&sm.bar[w & 1], bytes);
        async::tma_load_1d(sm.buf[w & 1], cgrp + (size_t)lo(w) * kGroup * kRow, bytes,
                           &sm.bar[w & 1]);
    };
    if (tid == 0) {
        async::mbar_init(&sm.bar[0], 1);
        async::mbar_init(&sm.bar[1], 1);
        async::fence_async_shared();
    }
    __syncthreads();
    bool pending0 = true, pending1 = nwin > 1;
    unsigned parity0 = 0u, parity1 = 0u;
    if (tid == 0) {
        issue(0);
        if (nwin > 1) issue(1);
    }

    // adjoint of the cost at the final state
    const float2* tape = reinterpret_cast<const float2*>(a.tape) + (size_t)i * 3;
    Blocks<1> sf;
    load_state(tape + (size_t)sc.n_ckpt * a.N * 3, sf);
    float ax = 2.f * (sf.x[0] - sc.goal[0][0]);
    float ay = 2.f * (sf.y[0] - sc.goal[0][1]);
    float aph = 2.f * sc.w_yaw * wrapf(sf.ph[0] - sc.goal[0][2]);
    float avx = 0.f, avy = 0.f, aom = 0.f;

    float dX = 0.f, dY = 0.f, e = 0.f, az = 0.f;
    bool bad = false, failed = false;
    const bool hard = a.hard != 0;
    int k = sc.H - 1;   // the action of the next substep down
    for (int w = 0; w < nwin; ++w) {
        const int b = w & 1;
        if (!warp_wait(&sm.bar[b], b ? parity1 : parity0)) { failed = true; break; }
        if (b) { parity1 ^= 1u; pending1 = false; } else { parity0 ^= 1u; pending0 = false; }
        const int l0 = lo(w);
        const float* base = sm.buf[b] + (size_t)p * kRow;
        int t = hi(w) - 1;
        while (t >= l0) {
            // the substeps of this window inside action k, then (if it starts
            // here) action k's placement and gradient
            const int a0 = k * T, stop = max(l0, a0);
            // substep t's coefficients; the next one down is loaded while t is computed
            Coefs cur = load_coefs(base, t - l0, lane);
            for (; t >= stop; --t) {
                const Coefs nxt = load_coefs(base, max(t - 1, stop) - l0, lane);
                const float4 c0 = cur.c0, c1 = cur.c1, c2 = cur.c2, c3 = cur.c3;
                const float2 c4 = cur.c4, e0 = cur.e0, e1 = cur.e1, e2 = cur.e2;
                const float v0 = avx + sc.dt * ax, v1 = avy + sc.dt * ay, v2 = aom + sc.dt * aph;
                // M rows: F_x = (c0, c1.xy), F_y = (c1.zw, c2), T = (c3, c4)
                const float d0 = c0.x * v0 + c1.z * v1 + c3.x * v2;
                const float d1 = c0.y * v0 + c1.w * v1 + c3.y * v2;
                const float d2 = c0.z * v0 + c2.x * v1 + c3.z * v2;
                const float d3 = c0.w * v0 + c2.y * v1 + c3.w * v2;
                const float d4 = c1.x * v0 + c2.z * v1 + c4.x * v2;
                const float d5 = c1.y * v0 + c2.w * v1 + c4.y * v2;
                ax += d0;
                ay += d1;
                aph += d2;
                avx = v0 + d3;
                avy = v1 + d4;
                aom = v2 + d5;
                dX -= d0;   // the pushers move with the block's start position
                dY -= d1;
                e += e0.x * v0 + e0.y * v1 + e1.x * v2;
                az += e1.y * v0 + e2.x * v1 + e2.y * v2;
                cur = nxt;
            }
            if (t >= a0) continue;   // the window ended inside the action
            // start of action k: the pushers' placement, then the parameter gradient
            const int tb = tid & ~3;
            const float dph = __shfl_sync(0xffffffffu, e, tb);
            const float aoff = __shfl_sync(0xffffffffu, e, tb + 1);
            float adist = __shfl_sync(0xffffffffu, e, tb + 2);
            ax += dX;
            ay += dY;
            aph += dph;
            const float* r = rel + (size_t)k * kRel * a.N + i;
            const float zl = r[lane * a.N], tu = r[4 * a.N], sg = r[5 * a.N];
            adist += 2.f * sc.w_push * (sc.dist_max * sg);
            const float zaz = team_sum<4>(zl * az);
            if (on) {
                float* gr = a.grad + (size_t)i * sc.D + (size_t)k * 6;
                const float gz = hard ? 0.f : -(zl * (az - zaz) * sc.inv_tau);
                gr[lane] = gz;
                bad |= !isfinite(gz);
                if (lane == 0) {
                    const float gv = -(aoff * sc.off_max * (1.f - tu * tu));
                    gr[4] = gv;
                    bad |= !isfinite(gv);
                }
                if (lane == 1) {
                    const float gv = -(adist * sc.dist_max * sg * (1.f - sg));
                    gr[5] = gv;
                    bad |= !isfinite(gv);
                }
            }
            dX = dY = e = az = 0.f;
            --k;
        }
        __syncwarp();
        if (w + 2 < nwin) {   // the buffer is free again
            if (tid == 0) issue(w + 2);
            if (b) pending1 = true; else pending0 = true;
        }
    }
    if (failed) {
        if (tid == 0) atomicOr(flag, 2);
        // let the copies in flight land before the CTA exits
        for (unsigned s = 0; pending0 && s < async::kWaitLimit; ++s)
            if (async::mbar_try_wait(&sm.bar[0], parity0)) break;
        for (unsigned s = 0; pending1 && s < async::kWaitLimit; ++s)
            if (async::mbar_try_wait(&sm.bar[1], parity1)) break;
        return;
    }
    // an overflowed reverse sweep gives the particle a zero gradient, and is counted
    bad = team_sum<4>(bad ? 1.f : 0.f) > 0.f;
    if (on && bad) {
        for (int q = lane; q < sc.D; q += 4) a.grad[(size_t)i * sc.D + q] = 0.f;
        if (lane == 0 && a.dropped) atomicAdd(a.dropped, 1ull);
    }
}

constexpr size_t kScanSmem = sizeof(ScanSmem);

}  // namespace
}  // namespace rollout

size_t adjoint_time_coef_floats(int n, int H, int T) {
    return (size_t)((n + rollout::kGroup - 1) / rollout::kGroup) * rollout::kGroup * H * T *
           rollout::kRow;
}
size_t adjoint_time_rel_floats(int n, int H) { return (size_t)n * H * rollout::kRel; }

cudaError_t launch_adjoint_time(const SimConst& sc, const RolloutArgs& a, float* rel, float* coef,
                                int* flag, cudaStream_t st) {
    using namespace rollout;
    if (sc.nb != 1 || sc.C != 1 || a.N < 1) return cudaErrorInvalidValue;
    const cudaError_t e = cudaFuncSetAttribute(scan_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)kScanSmem);
    if (e != cudaSuccess) return e;
    const long long pairs = (long long)a.N * sc.H * sc.T;
    relax_kernel<<<(a.N * sc.H + 127) / 128, 128, 0, st>>>(sc, a, rel);
    jac_kernel<<<(unsigned)((pairs + 127) / 128), 128, 0, st>>>(sc, a, rel, coef);
    scan_kernel<<<(a.N + kGroup - 1) / kGroup, 32, kScanSmem, st>>>(sc, a, rel, coef, flag);
    return cudaGetLastError();
}

}  // namespace stamp
