// Batched serving: many planning problems with uneven block counts, horizons
// and particle counts, solved together (Algorithm 1 on every instance).
//
// Per Stein iteration the whole batch takes one forward and one adjoint
// launch per block-count class (teams of the class's instances side by side,
// each warp inside one instance), one pairwise, two median-digit, one Stein
// direction and one Adam launch (per-CTA work items over all instances), and
// a counter bump; a run of iterations between early-stop checks is captured
// once in a CUDA graph and replayed.  The iteration number and Adam's step
// live on the device, so the replayed launches see them advance.  Every
// instance computes what stamp_solve computes for it alone with the same
// lanes, checkpoint interval and the sequential reverse sweep (same kernel
// bodies, same Stein-sum split, same bias-correction constants), up to the
// rounding of multiply-adds the compiler fuses differently in the two
// kernels.
//
// Or, in the persistent mode (batch_persist.cu), one launch per iteration
// does all of it: a work queue over every instance's rollouts (forward and
// adjoint fused per warp), pairwise tiles, median passes, Stein blocks and
// Adam chunks.  The autotuner times both modes and keeps the faster.
#include <algorithm>
#include <chrono>
#include <queue>
#include <cstdarg>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "stamp.h"
#include "stamp_internal.cuh"

using stamp::BatchArgs;
using stamp::BatchInst;
using stamp::SimConst;
using stamp::SvgdInst;

namespace {

stamp_status bfail(stamp_status s, const char* fmt, ...) {
    char buf[400];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    stamp::set_last_error(buf);
    return s;
}
#define B_CUDA(call)                                                                       \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            cudaGetLastError();                                                            \
            return bfail(STAMP_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));     \
        }                                                                                  \
    } while (0)
#define B_TRY(x)                       \
    do {                               \
        stamp_status s_ = (x);         \
        if (s_ != STAMP_OK) return s_; \
    } while (0)

constexpr int kMaxInstances = 4096;
constexpr int kMedCtasMax = 64;
constexpr int kMaxIters = 1 << 16;   // Adam bias-correction table length
constexpr unsigned long long kWaitNs = 1000000000ull;   // persistent dependency waits: 1 s

__global__ void bump_kernel(int* iter, int* step) {
    ++*iter;
    ++*step;
}

// Lowest cost of each instance (one CTA per instance).
__global__ void __launch_bounds__(256) instance_min_kernel(const float* __restrict__ cost,
                                                           const long long* __restrict__ cost0,
                                                           const int* __restrict__ n,
                                                           float* __restrict__ out) {
    __shared__ float red[256];
    const int g = blockIdx.x;
    float m = INFINITY;
    for (int i = threadIdx.x; i < n[g]; i += 256) {
        const float c = cost[cost0[g] + i];
        m = (c < m) ? c : m;   // NaN never wins
    }
    red[threadIdx.x] = m;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] = fminf(red[threadIdx.x], red[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) out[g] = red[0];
}

struct Class {
    int nb = 0;
    int lanes = 0, cta = 128, C = 25;
    SimConst sc{};                 // class-wide constants (physics, nb, C)
    std::vector<int> members;      // batch indices
    int n_teams = 0;
    BatchInst* d_inst = nullptr;   // device table, ascending team0
};

}  // namespace

struct stamp_batch {
    int n = 0;
    SimConst phys{};
    std::vector<stamp_instance_desc> inst;
    std::vector<int> D;
    std::vector<long long> elem0, part0, d20, cost0, tape0;
    long long n_elem = 0;
    cudaStream_t user = nullptr, st = nullptr;
    // the Stein bandwidths (pairwise + median) run beside the rollouts here
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    std::vector<Class> cls;
    // device memory
    char* arena = nullptr;
    float *theta = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr, *part = nullptr, *d2 = nullptr,
          *cost = nullptr, *tape = nullptr, *h = nullptr, *inst_min = nullptr;
    unsigned *hist = nullptr, *sel = nullptr, *counter = nullptr;
    int *active = nullptr, *iter = nullptr, *step = nullptr, *flag = nullptr, *topk = nullptr, *nvec = nullptr;
    float2* bc = nullptr;   // Adam bias corrections (1 - 0.9^s, 1 - 0.999^s) for s = 1..kMaxIters
    long long* cost0_dev = nullptr;
    unsigned long long* dropped = nullptr;
    SvgdInst* sinst = nullptr;
    int4* pw_items = nullptr;
    int2* med_items = nullptr;
    int4* phi_items = nullptr;
    int n_pw = 0, n_med = 0, n_phi = 0, max_D = 0;
    size_t hist_bytes = 0;
    float lr = 1e-2f;
    // graph of `graph_iters` iterations
    cudaGraphExec_t graph = nullptr;
    int graph_iters = 0;
    float graph_lr = 0.f;
    bool graph_dirty = true;
    // persistent iteration (one launch per iteration)
    bool persist = false;
    bool persist_dirty = true;       // class intervals changed: rebuild p_inst, grid
    int persist_grid = 0;
    size_t persist_smem = 0;
    stamp::PersistArgs pa{};
    SimConst cls_sc[stamp::kMaxBlocks]{};
    BatchInst* p_inst = nullptr;
    int4 *p_need = nullptr, *p_warps = nullptr, *p_phi = nullptr, *p_pw = nullptr;
    int2* p_adam = nullptr;
    unsigned *p_ctr = nullptr, *p_dep = nullptr;
    int extra_wait = 0;              // > 0 for the next solve: its Stein items' waits run out
    stamp_trace_entry* trace = nullptr;   // persistent-launch trace (NULL: off)
    unsigned long long wait_ns = kWaitNs;
    float mode_ms[2] = {-1.f, -1.f};   // autotuner: ms per iteration, per-class and persistent
    // instances whose next solve starts from particles set by stamp_batch_screen
    std::vector<char> screened;
    // last solve
    std::vector<int> iters_done;
    std::vector<float> best;
    std::vector<double> tts;
    long long units = 0;
    double seconds = 0.0;
};

namespace {

stamp_status build_class_tables(stamp_batch* b, Class& c) {
    const int tpw = 32 / c.lanes;   // teams per warp
    std::vector<BatchInst> h(c.members.size());
    int team = 0;
    for (size_t q = 0; q < c.members.size(); ++q) {
        const int g = c.members[q];
        const stamp_instance_desc& d = b->inst[g];
        BatchInst& e = h[q];
        e.theta = b->theta + b->elem0[g];
        e.grad = b->grad + b->elem0[g];
        e.tape = b->tape + b->tape0[g];
        e.cost = b->cost + b->cost0[g];
        e.N = d.N;
        e.H = d.H;
        e.D = b->D[g];
        e.n_ckpt = d.H * b->phys.T / c.C;
        e.team0 = team;
        e.gid = g;
        e.seed = d.seed;
        for (int k = 0; k < stamp::kMaxBlocks; ++k)
            for (int j = 0; j < 3; ++j) {
                e.init[k][j] = k < d.n_blocks ? d.init[3 * k + j] : 0.f;
                e.goal[k][j] = k < d.n_blocks ? d.goal[3 * k + j] : 0.f;
            }
        team += (d.N + tpw - 1) / tpw * tpw;
    }
    c.n_teams = team;
    c.sc.C = c.C;
    B_CUDA(cudaMemcpy(c.d_inst, h.data(), h.size() * sizeof(BatchInst), cudaMemcpyHostToDevice));
    b->graph_dirty = true;
    b->persist_dirty = true;
    return STAMP_OK;
}

// The persistent launch's per-instance table (each instance with its class's
// checkpoint interval), the adjoint's segment memory per warp, the grid.
// Synchronous: never while a graph is being captured.
stamp_status ensure_persist(stamp_batch* b) {
    if (!b->persist_dirty) return STAMP_OK;
    std::vector<BatchInst> h(b->n);
    int seg_warp = 0;
    for (const Class& c : b->cls) {
        std::vector<BatchInst> ci(c.members.size());
        B_CUDA(cudaMemcpy(ci.data(), c.d_inst, ci.size() * sizeof(BatchInst), cudaMemcpyDeviceToHost));
        for (size_t q = 0; q < c.members.size(); ++q) h[c.members[q]] = ci[q];
        const int L = stamp::persist_lanes(c.nb);
        if (c.C > 1) seg_warp = std::max(seg_warp, (32 / L) * (c.C * 3 * c.nb + 1));
        b->cls_sc[c.nb - 1] = c.sc;
    }
    B_CUDA(cudaMemcpy(b->p_inst, h.data(), h.size() * sizeof(BatchInst), cudaMemcpyHostToDevice));
    b->persist_smem = stamp::persist_smem(b->max_D, seg_warp);
    if (b->persist_smem > 200 * 1024) return bfail(STAMP_EINVAL, "checkpoint segments too large for the persistent launch");
    B_CUDA(stamp::persist_grid(b->persist_smem, &b->persist_grid));
    b->pa.seg_warp = seg_warp;
    b->persist_dirty = false;
    b->graph_dirty = true;
    return STAMP_OK;
}

stamp_status rollout_class(stamp_batch* b, const Class& c, bool adjoint, bool hard, cudaStream_t st) {
    BatchArgs a{};
    a.inst = c.d_inst;
    a.n_inst = (int)c.members.size();
    a.n_teams = c.n_teams;
    a.active = b->active;
    a.iter_dev = hard ? nullptr : b->iter;
    a.iter = -1;
    a.hard = hard ? 1 : 0;
    a.dropped = b->dropped;
    const cudaError_t e = stamp::launch_rollout_batch(c.nb, c.sc, a, c.lanes, c.cta, adjoint, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return bfail(STAMP_ECUDA, "batched rollout launch failed: %s", cudaGetErrorString(e));
    }
    return STAMP_OK;
}

// One Stein iteration of every active instance.  The bandwidths depend on
// the particles only: they run on the side stream beside the rollouts, and
// the Stein direction waits for both (fork and join become graph edges when
// captured).
int n_items(const stamp_batch* b) {
    const stamp::PersistArgs& p = b->pa;
    return p.n_roll + p.n_pw + 2 * p.n_med + p.n_phi + p.n_adam;
}

stamp_status iteration(stamp_batch* b, cudaStream_t st) {
    if (b->persist) {
        if (b->persist_dirty) return bfail(STAMP_EINVAL, "persistent tables out of date");
        stamp::PersistArgs pa = b->pa;
        pa.lr = b->lr;
        pa.extra_wait = b->extra_wait;
        pa.wait_ns = b->wait_ns;
        pa.trace = b->trace;
        pa.trace_cap = b->trace ? n_items(b) : 0;
        B_CUDA(stamp::launch_persist(pa, b->cls_sc, b->persist_grid, b->persist_smem, st));
        return STAMP_OK;
    }
    B_CUDA(cudaEventRecord(b->ev_fork, st));
    B_CUDA(cudaStreamWaitEvent(b->side, b->ev_fork, 0));
    B_CUDA(cudaMemsetAsync(b->hist, 0, b->hist_bytes, b->side));
    B_CUDA(stamp::launch_pairwise_batch(b->sinst, b->pw_items, b->n_pw, b->max_D, b->active, b->side));
    for (int dg = 1; dg <= 2; ++dg)
        B_CUDA(stamp::launch_median_digit_batch(b->sinst, b->med_items, b->n_med, b->active, dg,
                                                b->side));
    B_CUDA(cudaEventRecord(b->ev_join, b->side));
    for (const Class& c : b->cls) B_TRY(rollout_class(b, c, false, false, st));
    for (const Class& c : b->cls) B_TRY(rollout_class(b, c, true, false, st));
    B_CUDA(cudaStreamWaitEvent(st, b->ev_join, 0));
    B_CUDA(stamp::launch_phi_batch(b->sinst, b->phi_items, b->n_phi, b->max_D, b->active, b->flag, st));
    B_CUDA(stamp::launch_adam_batch(b->theta, b->m, b->v, b->n_elem, b->sinst, b->n, b->active, b->step,
                                    b->bc, b->lr, b->flag, st));
    bump_kernel<<<1, 1, 0, st>>>(b->iter, b->step);
    B_CUDA(cudaGetLastError());
    return STAMP_OK;
}

stamp_status ensure_graph(stamp_batch* b, int iters) {
    if (b->graph && !b->graph_dirty && b->graph_iters == iters && b->graph_lr == b->lr) return STAMP_OK;
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    cudaGraph_t g = nullptr;
    B_CUDA(cudaStreamBeginCapture(b->st, cudaStreamCaptureModeRelaxed));
    stamp_status r = STAMP_OK;
    for (int q = 0; q < iters && r == STAMP_OK; ++q) r = iteration(b, b->st);
    const cudaError_t e = cudaStreamEndCapture(b->st, &g);
    if (r != STAMP_OK) {
        if (g) cudaGraphDestroy(g);
        return r;
    }
    B_CUDA(e);
    const cudaError_t ei = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    B_CUDA(ei);
    b->graph_iters = iters;
    b->graph_lr = b->lr;
    b->graph_dirty = false;
    return STAMP_OK;
}

// Hard, noise-free evaluation of every instance (active or not) and each
// instance's lowest cost.
stamp_status hard_eval(stamp_batch* b, bool all) {
    if (all) {
        std::vector<int> ones(b->n, 1);
        B_CUDA(cudaMemcpyAsync(b->active, ones.data(), b->n * sizeof(int), cudaMemcpyHostToDevice, b->st));
    }
    for (const Class& c : b->cls) B_TRY(rollout_class(b, c, false, true, b->st));
    instance_min_kernel<<<b->n, 256, 0, b->st>>>(b->cost, b->cost0_dev, b->nvec, b->inst_min);
    B_CUDA(cudaGetLastError());
    return STAMP_OK;
}

// Work queue of the persistent launch.  Rollout items go by block count,
// most blocks first, and longest first within a block count: a warp task's
// time is estimated as horizon x a per-block-count cost (per-warp rollout +
// adjoint time per action, measured on GB300 with the per-class kernels at
// their tuned lanes).  The Stein blocks and Adam chunks follow in
// the order in which a list schedule of the rollout items over one CTA per
// SM finishes the instances' rollouts.
stamp_status build_persist_queue(stamp_batch* b, const std::vector<SvgdInst>& si) {
    static const double kCost[stamp::kMaxBlocks] = {0.17, 0.39, 0.52, 1.09};
    constexpr int W = stamp::kPersistWarps;
    struct Task { double t; int g, first, nb; };
    std::vector<Task> tasks;
    std::vector<int4> need(b->n), pw;
    for (int g = 0; g < b->n; ++g) {
        const stamp_instance_desc& d = b->inst[g];
        const int tpw = 32 / stamp::persist_lanes(d.n_blocks);
        const int warps = (d.N + tpw - 1) / tpw;
        for (int w = 0; w < warps; ++w) tasks.push_back({d.H * kCost[d.n_blocks - 1], g, w * tpw, d.n_blocks});
        const int rb = (d.N + stamp::kPersistRows - 1) / stamp::kPersistRows;
        // pairwise strips: up to kPersistStrip tile pairs of one tile row each
        int strips = 0;
        for (int bi = 0; bi < si[g].nt; ++bi)
            for (int bj = bi; bj < si[g].nt; bj += stamp::kPersistStrip) {
                pw.push_back(make_int4(g, bi, bj, std::min(bj + stamp::kPersistStrip, si[g].nt)));
                ++strips;
            }
        need[g] = make_int4(warps, strips, si[g].med_ctas, si[g].shares * rb);
    }
    // by block count (consecutive items on an SM run the same code), longest first within it
    std::stable_sort(tasks.begin(), tasks.end(), [](const Task& x, const Task& y) {
        return x.nb != y.nb ? x.nb > y.nb : x.t > y.t;
    });
    const int n_roll = (int)((tasks.size() + W - 1) / W);
    std::vector<int4> warps((size_t)n_roll * W, make_int4(-1, 0, 0, 0));
    for (size_t q = 0; q < tasks.size(); ++q) warps[q] = make_int4(tasks[q].g, tasks[q].first, tasks[q].nb, 0);
    std::priority_queue<double, std::vector<double>, std::greater<double>> free_at;
    for (int w = 0; w < stamp::sm_count(); ++w) free_at.push(0.0);
    std::vector<double> done(b->n, 0.0);
    for (int it = 0; it < n_roll; ++it) {
        double dur = 0.0;
        for (int w = 0; w < W && (size_t)it * W + w < tasks.size(); ++w) dur = std::max(dur, tasks[(size_t)it * W + w].t);
        const double t1 = free_at.top() + dur;
        free_at.pop();
        free_at.push(t1);
        for (int w = 0; w < W && (size_t)it * W + w < tasks.size(); ++w) {
            const int g = tasks[(size_t)it * W + w].g;
            done[g] = std::max(done[g], t1);
        }
    }
    std::vector<int> order(b->n);
    for (int g = 0; g < b->n; ++g) order[g] = g;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return done[x] < done[y]; });
    std::vector<int4> phi;
    std::vector<int2> adam;
    for (int g : order) {
        const int rb = (b->inst[g].N + stamp::kPersistRows - 1) / stamp::kPersistRows;
        for (int sh = 0; sh < si[g].shares; ++sh)
            for (int r0 = 0; r0 < rb; ++r0) phi.push_back(make_int4(g, r0, sh, 0));
    }
    for (int g : order) {
        const long long ne = (long long)b->inst[g].N * b->D[g];
        for (long long c = 0; c * stamp::kPersistAdamChunk < ne; ++c) adam.push_back(make_int2(g, (int)c));
    }
    B_CUDA(cudaMalloc(&b->p_warps, warps.size() * sizeof(int4)));
    B_CUDA(cudaMalloc(&b->p_phi, phi.size() * sizeof(int4)));
    B_CUDA(cudaMalloc(&b->p_adam, adam.size() * sizeof(int2)));
    B_CUDA(cudaMalloc(&b->p_pw, pw.size() * sizeof(int4)));
    B_CUDA(cudaMemcpy(b->p_pw, pw.data(), pw.size() * sizeof(int4), cudaMemcpyHostToDevice));
    B_CUDA(cudaMemcpy(b->p_warps, warps.data(), warps.size() * sizeof(int4), cudaMemcpyHostToDevice));
    B_CUDA(cudaMemcpy(b->p_phi, phi.data(), phi.size() * sizeof(int4), cudaMemcpyHostToDevice));
    B_CUDA(cudaMemcpy(b->p_adam, adam.data(), adam.size() * sizeof(int2), cudaMemcpyHostToDevice));
    B_CUDA(cudaMemcpy(b->p_need, need.data(), need.size() * sizeof(int4), cudaMemcpyHostToDevice));
    stamp::PersistArgs& pa = b->pa;
    pa.inst = b->p_inst;
    pa.sinst = b->sinst;
    pa.need = b->p_need;
    pa.warps = b->p_warps;
    pa.pw = b->p_pw;
    pa.med = b->med_items;
    pa.phi = b->p_phi;
    pa.adam = b->p_adam;
    pa.n_roll = n_roll;
    pa.n_pw = (int)pw.size();
    pa.n_med = b->n_med;
    pa.n_phi = (int)phi.size();
    pa.n_adam = (int)adam.size();
    pa.n_inst = b->n;
    pa.active = b->active;
    pa.iter = b->iter;
    pa.step = b->step;
    pa.bc = b->bc;
    pa.theta = b->theta;
    pa.m = b->m;
    pa.v = b->v;
    pa.ctr = b->p_ctr;
    pa.dep = b->p_dep;
    pa.flag = b->flag;
    pa.dropped = b->dropped;
    pa.dp = stamp::persist_dp(b->max_D);
    return STAMP_OK;
}

// Zero what a Stein iteration expects to find zeroed (histograms, last-CTA
// counters, the persistent queue and its completion counters): a solve may
// follow an interrupted one or the other launch mode.
stamp_status clear_counters(stamp_batch* b) {
    B_CUDA(cudaMemsetAsync(b->hist, 0, b->hist_bytes, b->st));
    B_CUDA(cudaMemsetAsync(b->counter, 0, (size_t)b->n * 3 * sizeof(unsigned), b->st));
    B_CUDA(cudaMemsetAsync(b->p_ctr, 0, 4 * sizeof(unsigned), b->st));
    B_CUDA(cudaMemsetAsync(b->p_dep, 0, (size_t)b->n * stamp::kPersistDeps * sizeof(unsigned), b->st));
    return STAMP_OK;
}

bool is_dev(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

int default_cta(int lanes) { return lanes >= 16 ? 128 : 64; }

}  // namespace

namespace stamp {
cudaError_t launch_rollout_batch(int nb, const SimConst& sc, const BatchArgs& b, int lanes, int cta,
                                 bool adjoint, cudaStream_t st) {
    switch (nb) {
        case 1: return launch_rollout_batch_nb1(sc, b, lanes, cta, adjoint, st);
        case 2: return launch_rollout_batch_nb2(sc, b, lanes, cta, adjoint, st);
        case 3: return launch_rollout_batch_nb3(sc, b, lanes, cta, adjoint, st);
        case 4: return launch_rollout_batch_nb4(sc, b, lanes, cta, adjoint, st);
    }
    return cudaErrorInvalidValue;
}
}  // namespace stamp

extern "C" {

stamp_status stamp_batch_create(const stamp_problem_desc* physics, const stamp_instance_desc* inst,
                                int n_instances, void* cuda_stream, stamp_batch** out) {
    if (!out) return bfail(STAMP_EINVAL, "out is NULL");
    *out = nullptr;
    if (!physics || !inst) return bfail(STAMP_EINVAL, "NULL physics or instances");
    if (n_instances < 1 || n_instances > kMaxInstances)
        return bfail(STAMP_EINVAL, "n_instances=%d outside [1, %d]", n_instances, kMaxInstances);
    // the problem constants of one instance carry the shared physics (validated there)
    stamp_problem_desc d1 = *physics;
    d1.n_blocks = 1;
    d1.H = 1;
    d1.ckpt_every = 1;
    const float zeros[3 * stamp::kMaxBlocks] = {};
    stamp_problem* probe = nullptr;
    B_TRY(stamp_problem_create(&d1, zeros, zeros, 1, nullptr, &probe));
    SimConst phys = stamp::problem_const(probe);
    stamp_problem_destroy(probe);
    for (int g = 0; g < n_instances; ++g) {
        const stamp_instance_desc& d = inst[g];
        if (d.n_blocks < 1 || d.n_blocks > stamp::kMaxBlocks || d.H < 1 || d.H > stamp::kMaxH ||
            d.N < 1 || d.N > stamp::kMaxTopkN)
            return bfail(STAMP_EINVAL, "instance %d: n_blocks 1..4, H 1..16, N 1..8192 required", g);
        for (int q = 0; q < 3 * d.n_blocks; ++q)
            if (!std::isfinite(d.init[q]) || !std::isfinite(d.goal[q]))
                return bfail(STAMP_EINVAL, "instance %d: non-finite pose", g);
    }
    stamp_batch* b = new stamp_batch();
    b->n = n_instances;
    b->screened.assign(n_instances, 0);
    b->phys = phys;
    b->inst.assign(inst, inst + n_instances);
    b->user = static_cast<cudaStream_t>(cuda_stream);
    if (cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        if (b->ev_join) cudaEventDestroy(b->ev_join);
        if (b->ev_fork) cudaEventDestroy(b->ev_fork);
        if (b->side) cudaStreamDestroy(b->side);
        if (b->st) cudaStreamDestroy(b->st);
        delete b;
        return bfail(STAMP_ECUDA, "stream creation failed");
    }
    // layout: every instance's blocks start on 128-byte boundaries (no cache
    // line holds two instances' data)
    auto al32 = [](long long x) { return (x + 31) / 32 * 32; };
    long long e = 0, p = 0, q2 = 0, c0 = 0, t0 = 0;
    b->D.resize(n_instances);
    for (int g = 0; g < n_instances; ++g) {
        const stamp_instance_desc& d = inst[g];
        const int D = d.H * (4 * d.n_blocks + 2);
        b->D[g] = D;
        b->max_D = std::max(b->max_D, D);
        int shares, jc;
        stamp::phi_batch_plan(d.N, &shares, &jc);
        b->elem0.push_back(e);
        e += al32((long long)d.N * D);
        b->part0.push_back(p);
        p += al32((long long)shares * d.N * D);
        b->d20.push_back(q2);
        q2 += al32((long long)d.N * d.N);
        b->cost0.push_back(c0);
        c0 += al32(d.N);
        b->tape0.push_back(t0);
        t0 += al32((long long)(d.H * phys.T + 1) * d.N * 6 * d.n_blocks);   // room for any C
    }
    b->n_elem = e;
    const long long hist_n = (long long)n_instances * (2048 + 2048 + 1024);
    b->hist_bytes = hist_n * sizeof(unsigned);
    struct Part { void** dst; size_t bytes; };
    const Part parts[] = {
        {(void**)&b->theta, e * 4}, {(void**)&b->grad, e * 4}, {(void**)&b->m, e * 4},
        {(void**)&b->v, e * 4}, {(void**)&b->part, p * 4}, {(void**)&b->d2, q2 * 4},
        {(void**)&b->cost, c0 * 4}, {(void**)&b->tape, t0 * 4}, {(void**)&b->h, n_instances * 4},
        {(void**)&b->inst_min, n_instances * 4}, {(void**)&b->hist, b->hist_bytes},
        {(void**)&b->sel, n_instances * 4 * 4}, {(void**)&b->counter, n_instances * 3 * 4},
        {(void**)&b->active, n_instances * 4}, {(void**)&b->iter, 4}, {(void**)&b->step, 4},
        {(void**)&b->flag, 4}, {(void**)&b->topk, (size_t)n_instances * 16 * 4},
        {(void**)&b->nvec, n_instances * 4}, {(void**)&b->cost0_dev, n_instances * 8},
        {(void**)&b->dropped, 8}, {(void**)&b->sinst, n_instances * sizeof(SvgdInst)},
        {(void**)&b->bc, (size_t)(kMaxIters + 1) * sizeof(float2)},
        {(void**)&b->p_inst, n_instances * sizeof(BatchInst)},
        {(void**)&b->p_need, n_instances * sizeof(int4)},
        {(void**)&b->p_ctr, 4 * sizeof(unsigned)},
        {(void**)&b->p_dep, (size_t)n_instances * stamp::kPersistDeps * sizeof(unsigned)},
    };
    size_t total = 0;
    for (const Part& q : parts) total += (q.bytes + 255) / 256 * 256;
    if (cudaMalloc(&b->arena, total) != cudaSuccess) {
        cudaGetLastError();
        b->arena = nullptr;
        stamp_batch_destroy(b);
        return bfail(STAMP_ENOMEM, "cudaMalloc of %zu bytes failed", total);
    }
    size_t off = 0;
    for (const Part& q : parts) {
        *q.dst = b->arena + off;
        off += (q.bytes + 255) / 256 * 256;
    }
    stamp_status r = STAMP_OK;
    auto setup = [&]() -> stamp_status {
        B_CUDA(cudaMemset(b->arena, 0, total));
        // the constants the single-problem Adam launch computes on the host
        std::vector<float2> bc(kMaxIters + 1);
        for (int q = 1; q <= kMaxIters; ++q)
            bc[q] = make_float2(1.f - powf(0.9f, (float)q), 1.f - powf(0.999f, (float)q));
        B_CUDA(cudaMemcpy(b->bc, bc.data(), bc.size() * sizeof(float2), cudaMemcpyHostToDevice));
        // Stein instance table and work items
        std::vector<SvgdInst> si(n_instances);
        std::vector<int4> pw, phi;
        std::vector<int2> med;
        std::vector<int> nv(n_instances);
        for (int g = 0; g < n_instances; ++g) {
            const stamp_instance_desc& d = inst[g];
            SvgdInst& s = si[g];
            s.theta = b->theta + b->elem0[g];
            s.grad = b->grad + b->elem0[g];
            s.d2 = b->d2 + b->d20[g];
            s.hist = b->hist + (size_t)g * (2048 + 2048 + 1024);
            s.sel = b->sel + 4 * g;
            s.counter = b->counter + 3 * g;
            s.h = b->h + g;
            s.part = b->part + b->part0[g];
            s.N = d.N;
            s.D = b->D[g];
            s.nt = (d.N + 31) / 32;
            const long long pairs = (long long)d.N * (d.N - 1) / 2;
            s.med_ctas = (int)std::max(1LL, std::min<long long>(kMedCtasMax, pairs / 8192));
            s.med_ctas = std::min(s.med_ctas, std::max(d.N - 1, 1));
            stamp::phi_batch_plan(d.N, &s.shares, &s.j_chunk);
            s.gid = g;
            s.elem0 = b->elem0[g];
            nv[g] = d.N;
            for (int bi = 0; bi < s.nt; ++bi)
                for (int bj = bi; bj < s.nt; ++bj) pw.push_back(make_int4(g, bi, bj, 0));
            for (int c = 0; c < s.med_ctas; ++c) med.push_back(make_int2(g, c));
            const int rb = (d.N + stamp::phi_rows_per_block() - 1) / stamp::phi_rows_per_block();
            for (int sh = 0; sh < s.shares; ++sh)
                for (int r0 = 0; r0 < rb; ++r0) phi.push_back(make_int4(g, r0, sh, 0));
        }
        B_CUDA(cudaMemcpy(b->sinst, si.data(), si.size() * sizeof(SvgdInst), cudaMemcpyHostToDevice));
        B_CUDA(cudaMemcpy(b->nvec, nv.data(), nv.size() * sizeof(int), cudaMemcpyHostToDevice));
        B_CUDA(cudaMemcpy(b->cost0_dev, b->cost0.data(), n_instances * sizeof(long long), cudaMemcpyHostToDevice));
        b->n_pw = (int)pw.size();
        b->n_med = (int)med.size();
        b->n_phi = (int)phi.size();
        B_CUDA(cudaMalloc(&b->pw_items, pw.size() * sizeof(int4)));
        B_CUDA(cudaMalloc(&b->med_items, med.size() * sizeof(int2)));
        B_CUDA(cudaMalloc(&b->phi_items, phi.size() * sizeof(int4)));
        B_CUDA(cudaMemcpy(b->pw_items, pw.data(), pw.size() * sizeof(int4), cudaMemcpyHostToDevice));
        B_CUDA(cudaMemcpy(b->med_items, med.data(), med.size() * sizeof(int2), cudaMemcpyHostToDevice));
        B_CUDA(cudaMemcpy(b->phi_items, phi.data(), phi.size() * sizeof(int4), cudaMemcpyHostToDevice));
        B_TRY(build_persist_queue(b, si));
        // block-count classes with the single-problem defaults
        for (int nb = 1; nb <= stamp::kMaxBlocks; ++nb) {
            Class c;
            c.nb = nb;
            for (int g = 0; g < n_instances; ++g)
                if (inst[g].n_blocks == nb) c.members.push_back(g);
            if (c.members.empty()) continue;
            c.sc = phys;
            c.sc.nb = nb;
            c.sc.M = 4 * nb;
            c.sc.P = c.sc.M + 2;
            c.sc.S = 6 * nb;
            c.lanes = stamp::default_lanes(nb, 1024, false);
            c.cta = default_cta(c.lanes);
            c.C = phys.T % 25 == 0 ? 25 : 1;
            B_CUDA(cudaMalloc(&c.d_inst, c.members.size() * sizeof(BatchInst)));
            b->cls.push_back(c);
            B_TRY(build_class_tables(b, b->cls.back()));
        }
        return STAMP_OK;
    };
    r = setup();
    if (r != STAMP_OK) {
        stamp_batch_destroy(b);
        return r;
    }
    *out = b;
    return STAMP_OK;
}

void stamp_batch_destroy(stamp_batch* b) {
    if (!b) return;
    if (b->st) cudaStreamSynchronize(b->st);
    if (b->side) cudaStreamSynchronize(b->side);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    for (Class& c : b->cls) cudaFree(c.d_inst);
    cudaFree(b->pw_items);
    cudaFree(b->med_items);
    cudaFree(b->phi_items);
    cudaFree(b->p_warps);
    cudaFree(b->p_phi);
    cudaFree(b->p_adam);
    cudaFree(b->p_pw);
    cudaFree(b->trace);
    cudaFree(b->arena);
    if (b->ev_join) cudaEventDestroy(b->ev_join);
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    if (b->side) cudaStreamDestroy(b->side);
    if (b->st) cudaStreamDestroy(b->st);
    delete b;
}

stamp_status stamp_batch_set_config(stamp_batch* b, int n_blocks, int lanes, int cta, int ckpt_every) {
    if (!b) return bfail(STAMP_EINVAL, "NULL batch");
    for (Class& c : b->cls) {
        if (c.nb != n_blocks) continue;
        if (!stamp::lanes_supported(n_blocks, lanes)) return bfail(STAMP_EINVAL, "unsupported lanes %d", lanes);
        if (cta < 32 || cta > 128 || cta % 32 || cta < lanes) return bfail(STAMP_EINVAL, "cta must be 32, 64, 96 or 128");
        if (ckpt_every < 1 || b->phys.T % ckpt_every) return bfail(STAMP_EINVAL, "ckpt_every must divide T");
        if ((size_t)(cta / lanes) * (ckpt_every * 3 * n_blocks + 1) * 8 > 200 * 1024)
            return bfail(STAMP_EINVAL, "checkpoint segment too large for shared memory");
        c.lanes = lanes;
        c.cta = cta;
        c.C = ckpt_every;
        return build_class_tables(b, c);
    }
    return bfail(STAMP_EINVAL, "no instance has %d blocks", n_blocks);
}

stamp_status stamp_batch_get_config(stamp_batch* b, int n_blocks, int* lanes, int* cta, int* ckpt_every) {
    if (!b) return bfail(STAMP_EINVAL, "NULL batch");
    for (const Class& c : b->cls)
        if (c.nb == n_blocks) {
            if (lanes) *lanes = c.lanes;
            if (cta) *cta = c.cta;
            if (ckpt_every) *ckpt_every = c.C;
            return STAMP_OK;
        }
    return bfail(STAMP_EINVAL, "no instance has %d blocks", n_blocks);
}

}  // extern "C"

namespace {

// Launch mode: whole Stein iterations (every instance active, no graph) in
// the per-class launches with the tuned configurations, in the persistent
// launch with the tuned checkpoint intervals and, if any is above one, in
// the persistent launch with interval-1 tapes (no segment recompute; the
// tape a warp writes is read back at once, from L2); keeps the fastest.  The
// particles are put back afterwards.
stamp_status tune_mode(stamp_batch* b, int reps, cudaEvent_t e0, cudaEvent_t e1) {
    float* save = nullptr;
    B_CUDA(cudaMalloc(&save, (size_t)b->n_elem * sizeof(float)));
    stamp_status r = STAMP_OK;
    std::vector<int> tuned_c;
    for (const Class& c : b->cls) tuned_c.push_back(c.C);
    const bool any_c = std::any_of(tuned_c.begin(), tuned_c.end(), [](int C) { return C > 1; });
    float ms[3] = {INFINITY, INFINITY, INFINITY};
    auto set_c = [&](bool ones) -> stamp_status {
        for (size_t q = 0; q < b->cls.size(); ++q) {
            Class& c = b->cls[q];
            const int want = ones ? 1 : tuned_c[q];
            if (c.C != want) {
                c.C = want;
                B_TRY(build_class_tables(b, c));
            }
        }
        return STAMP_OK;
    };
    auto run = [&]() -> stamp_status {
        B_CUDA(cudaMemcpyAsync(save, b->theta, (size_t)b->n_elem * sizeof(float), cudaMemcpyDeviceToDevice, b->st));
        for (int mode = 0; mode < (any_c ? 3 : 2); ++mode) {
            b->persist = mode >= 1;
            if (mode == 2) B_TRY(set_c(true));
            if (b->persist) B_TRY(ensure_persist(b));
            B_CUDA(cudaMemcpyAsync(b->theta, save, (size_t)b->n_elem * sizeof(float), cudaMemcpyDeviceToDevice, b->st));
            B_CUDA(cudaMemsetAsync(b->m, 0, b->n_elem * 4, b->st));
            B_CUDA(cudaMemsetAsync(b->v, 0, b->n_elem * 4, b->st));
            B_CUDA(cudaMemsetAsync(b->iter, 0, sizeof(int), b->st));
            B_CUDA(cudaMemsetAsync(b->step, 0, sizeof(int), b->st));
            B_TRY(clear_counters(b));
            for (int q = 0; q <= reps; ++q) {
                if (q == 1) B_CUDA(cudaEventRecord(e0, b->st));   // the first pass warms up
                B_TRY(iteration(b, b->st));
            }
            B_CUDA(cudaEventRecord(e1, b->st));
            B_CUDA(cudaEventSynchronize(e1));
            B_CUDA(cudaEventElapsedTime(&ms[mode], e0, e1));
        }
        B_CUDA(cudaMemcpyAsync(b->theta, save, (size_t)b->n_elem * sizeof(float), cudaMemcpyDeviceToDevice, b->st));
        B_CUDA(cudaMemsetAsync(b->flag, 0, sizeof(int), b->st));
        B_CUDA(cudaStreamSynchronize(b->st));
        return STAMP_OK;
    };
    r = run();
    cudaStreamSynchronize(b->st);
    cudaFree(save);
    const int best = ms[2] < std::min(ms[0], ms[1]) ? 2 : ms[1] < ms[0] ? 1 : 0;
    b->persist = best >= 1;
    if (r == STAMP_OK) r = set_c(best == 2);
    b->mode_ms[0] = ms[0] / reps;
    b->mode_ms[1] = std::min(ms[1], ms[2]) / reps;
    b->graph_dirty = true;
    return r;
}

}  // namespace

extern "C" {

// Autotuner: for every block-count class, time the forward + adjoint launch
// of the class (CUDA events on the batch's stream; the particles are the
// solve's initial draws) for each lane count, CTA size and checkpoint
// interval of a small candidate set, and keep the fastest.
stamp_status stamp_batch_autotune(stamp_batch* b, int reps) {
    if (!b) return bfail(STAMP_EINVAL, "NULL batch");
    if (reps < 1) reps = 1;
    B_CUDA(cudaStreamSynchronize(b->user));
    // the solve's initial particles (screened ones stay, for the next solve)
    for (int g = 0; g < b->n; ++g)
        if (!b->screened[g])
            B_CUDA(stamp::launch_init_theta(b->theta + b->elem0[g], b->inst[g].N, b->D[g],
                                            b->inst[g].seed, b->st));
    std::vector<int> ones(b->n, 1);
    B_CUDA(cudaMemcpyAsync(b->active, ones.data(), b->n * sizeof(int), cudaMemcpyHostToDevice, b->st));
    B_CUDA(cudaMemsetAsync(b->iter, 0, sizeof(int), b->st));
    cudaEvent_t e0, e1;
    B_CUDA(cudaEventCreate(&e0));
    B_CUDA(cudaEventCreate(&e1));
    stamp_status r = STAMP_OK;
    for (Class& c : b->cls) {
        const int lane_set[] = {1, 2, 4, 8, 16, 32};
        const int c_set[] = {1, 5, 25};
        int best_l = c.lanes, best_cta = c.cta, best_c = c.C;
        float best_ms = INFINITY;
        for (int L : lane_set) {
            if (!stamp::lanes_supported(c.nb, L)) continue;
            for (int cta : {64, 128}) {
                for (int C : c_set) {
                    if (b->phys.T % C || cta < L) continue;
                    if ((size_t)(cta / L) * (C * 3 * c.nb + 1) * 8 > 200 * 1024) continue;
                    c.lanes = L;
                    c.cta = cta;
                    c.C = C;
                    if ((r = build_class_tables(b, c)) != STAMP_OK) break;
                    float ms = 0.f;
                    for (int q = 0; q <= reps && r == STAMP_OK; ++q) {
                        if (q == 1) cudaEventRecord(e0, b->st);   // the first pass warms up
                        r = rollout_class(b, c, false, false, b->st);
                        if (r == STAMP_OK) r = rollout_class(b, c, true, false, b->st);
                    }
                    if (r != STAMP_OK) break;
                    cudaEventRecord(e1, b->st);
                    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                        cudaGetLastError();
                        r = bfail(STAMP_ECUDA, "autotune timing failed");
                        break;
                    }
                    if (ms < best_ms) {
                        best_ms = ms;
                        best_l = L;
                        best_cta = cta;
                        best_c = C;
                    }
                }
                if (r != STAMP_OK) break;
            }
            if (r != STAMP_OK) break;
        }
        if (r != STAMP_OK) break;
        c.lanes = best_l;
        c.cta = best_cta;
        c.C = best_c;
        if ((r = build_class_tables(b, c)) != STAMP_OK) break;
    }
    if (r == STAMP_OK) r = tune_mode(b, reps, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (r == STAMP_OK) B_CUDA(cudaStreamSynchronize(b->st));
    return r;
}

stamp_status stamp_batch_solve(stamp_batch* b, int iters, float lr, float target_cost, int check_every,
                               int use_graph) {
    if (!b) return bfail(STAMP_EINVAL, "NULL batch");
    if (iters < 0 || iters > kMaxIters || check_every < 0 || !std::isfinite(lr))
        return bfail(STAMP_EINVAL, "need 0 <= iters <= %d, check_every >= 0, finite lr", kMaxIters);
    B_CUDA(cudaStreamSynchronize(b->user));
    const auto t_start = std::chrono::steady_clock::now();
    b->lr = lr;
    for (int g = 0; g < b->n; ++g)
        if (!b->screened[g])
            B_CUDA(stamp::launch_init_theta(b->theta + b->elem0[g], b->inst[g].N, b->D[g],
                                            b->inst[g].seed, b->st));
    b->screened.assign(b->n, 0);
    B_CUDA(cudaMemsetAsync(b->m, 0, b->n_elem * 4, b->st));
    B_CUDA(cudaMemsetAsync(b->v, 0, b->n_elem * 4, b->st));
    B_CUDA(cudaMemsetAsync(b->iter, 0, sizeof(int), b->st));
    B_CUDA(cudaMemsetAsync(b->step, 0, sizeof(int), b->st));
    B_CUDA(cudaMemsetAsync(b->flag, 0, sizeof(int), b->st));
    std::vector<int> act(b->n, 1);
    B_CUDA(cudaMemcpyAsync(b->active, act.data(), b->n * sizeof(int), cudaMemcpyHostToDevice, b->st));
    B_TRY(clear_counters(b));
    if (b->persist) B_TRY(ensure_persist(b));
    b->iters_done.assign(b->n, iters);
    b->best.assign(b->n, INFINITY);
    b->tts.assign(b->n, -1.0);
    b->units = 0;
    const int chunk = check_every > 0 ? check_every : std::max(iters, 1);
    std::vector<float> mins(b->n);
    int done = 0, n_active = b->n;
    while (done < iters && n_active > 0) {
        const int k = std::min(chunk, iters - done);
        for (int g = 0; g < b->n; ++g)
            if (act[g]) b->units += (long long)k * b->inst[g].N * b->inst[g].H * b->phys.T;
        if (use_graph) {
            B_TRY(ensure_graph(b, k));
            B_CUDA(cudaGraphLaunch(b->graph, b->st));
        } else {
            for (int q = 0; q < k; ++q) B_TRY(iteration(b, b->st));
        }
        done += k;
        if (check_every > 0) {
            B_TRY(hard_eval(b, false));
            B_CUDA(cudaMemcpyAsync(mins.data(), b->inst_min, b->n * sizeof(float), cudaMemcpyDeviceToHost, b->st));
            B_CUDA(cudaStreamSynchronize(b->st));
            const double now = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
            bool changed = false;
            for (int g = 0; g < b->n; ++g) {
                if (!act[g]) continue;
                b->best[g] = mins[g];
                if (mins[g] < target_cost) {
                    act[g] = 0;
                    --n_active;
                    changed = true;
                    b->iters_done[g] = done;
                    b->tts[g] = now;
                }
            }
            if (changed)
                B_CUDA(cudaMemcpyAsync(b->active, act.data(), b->n * sizeof(int), cudaMemcpyHostToDevice, b->st));
        }
    }
    // final hard evaluation of every instance and its distinct-plan top-3
    B_TRY(hard_eval(b, true));
    for (int g = 0; g < b->n; ++g) {
        SimConst sc = b->phys;
        sc.nb = b->inst[g].n_blocks;
        sc.H = b->inst[g].H;
        sc.M = 4 * sc.nb;
        sc.P = sc.M + 2;
        B_CUDA(stamp::launch_topk(b->theta + b->elem0[g], b->cost + b->cost0[g], b->inst[g].N, sc,
                                  std::min(3, b->inst[g].N), b->topk + 16 * g, b->st));
    }
    B_CUDA(cudaMemcpyAsync(mins.data(), b->inst_min, b->n * sizeof(float), cudaMemcpyDeviceToHost, b->st));
    int flag = 0;
    B_CUDA(cudaMemcpyAsync(&flag, b->flag, sizeof(int), cudaMemcpyDeviceToHost, b->st));
    B_CUDA(cudaStreamSynchronize(b->st));
    b->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    for (int g = 0; g < b->n; ++g) b->best[g] = mins[g];
    if (b->extra_wait) {   // the injected wait failure lasts one solve
        b->extra_wait = 0;
        b->wait_ns = kWaitNs;
        b->graph_dirty = true;
    }
    if (flag & 2) return bfail(STAMP_ETIMEOUT, "a bounded device wait gave up");
    if (flag & 1) return bfail(STAMP_ENONFINITE, "a non-finite particle or Stein direction was produced");
    return STAMP_OK;
}

stamp_status stamp_batch_screen(stamp_batch* b, stamp_surrogate* s, int g, int n_candidates) {
    if (!b || !s) return bfail(STAMP_EINVAL, "NULL batch or surrogate");
    if (g < 0 || g >= b->n) return bfail(STAMP_EINVAL, "instance %d outside [0, %d)", g, b->n);
    const stamp_instance_desc& d = b->inst[g];
    if (d.N > stamp::kMaxScreenN || n_candidates < d.N || n_candidates > stamp::surrogate_max_rows(s))
        return bfail(STAMP_EINVAL, "need N <= %d and N <= n_candidates <= the surrogate's max_rows",
                     stamp::kMaxScreenN);
    // the instance's constants, as the batched rollouts see them
    SimConst sc = b->phys;
    sc.nb = d.n_blocks;
    sc.H = d.H;
    sc.M = 4 * sc.nb;
    sc.P = sc.M + 2;
    sc.D = b->D[g];
    sc.S = 6 * sc.nb;
    sc.n_ckpt = sc.H * sc.T / sc.C;
    for (int k = 0; k < stamp::kMaxBlocks; ++k)
        for (int j = 0; j < 3; ++j) {
            sc.init[k][j] = k < d.n_blocks ? d.init[3 * k + j] : 0.f;
            sc.goal[k][j] = k < d.n_blocks ? d.goal[3 * k + j] : 0.f;
        }
    B_CUDA(cudaStreamSynchronize(b->st));
    const cudaStream_t ss = stamp::surrogate_stream(s);
    float* cand = stamp::surrogate_candidates(s);
    B_CUDA(stamp::launch_init_theta(cand, n_candidates, sc.D, d.seed, ss));
    B_TRY(stamp::surrogate_screen(s, sc, cand, n_candidates, d.N, b->theta + b->elem0[g], nullptr));
    B_CUDA(cudaStreamSynchronize(ss));
    b->screened[g] = 1;
    return STAMP_OK;
}

stamp_status stamp_batch_set_persistent(stamp_batch* b, int on) {
    if (!b) return bfail(STAMP_EINVAL, "NULL batch");
    if ((on != 0) != b->persist) b->graph_dirty = true;
    b->persist = on != 0;
    return STAMP_OK;
}

stamp_status stamp_batch_get_persistent(stamp_batch* b, int* on, float* ms_per_class, float* ms_persistent) {
    if (!b) return bfail(STAMP_EINVAL, "NULL batch");
    if (on) *on = b->persist ? 1 : 0;
    if (ms_per_class) *ms_per_class = b->mode_ms[0];
    if (ms_persistent) *ms_persistent = b->mode_ms[1];
    return STAMP_OK;
}

stamp_status stamp_batch_set_trace(stamp_batch* b, int on) {
    if (!b) return bfail(STAMP_EINVAL, "NULL batch");
    B_CUDA(cudaStreamSynchronize(b->st));
    if (on && !b->trace) {
        const size_t bytes = (size_t)n_items(b) * sizeof(stamp_trace_entry);
        B_CUDA(cudaMalloc(&b->trace, bytes));
        B_CUDA(cudaMemset(b->trace, 0, bytes));
    } else if (!on && b->trace) {
        cudaFree(b->trace);
        b->trace = nullptr;
    }
    b->graph_dirty = true;
    return STAMP_OK;
}

stamp_status stamp_batch_read_trace(stamp_batch* b, stamp_trace_entry* out, int capacity, int* n,
                                    int* kinds5) {
    if (!b) return bfail(STAMP_EINVAL, "NULL batch");
    const int total = n_items(b);
    if (n) *n = total;
    if (kinds5) {
        const stamp::PersistArgs& p = b->pa;
        const int k[5] = {p.n_roll, p.n_pw, p.n_med, p.n_phi, p.n_adam};
        for (int q = 0; q < 5; ++q) kinds5[q] = k[q];
    }
    if (out && capacity > 0) {
        if (!b->trace) return bfail(STAMP_EINVAL, "tracing is off");
        B_CUDA(cudaStreamSynchronize(b->st));
        B_CUDA(cudaMemcpy(out, b->trace, (size_t)std::min(capacity, total) * sizeof(stamp_trace_entry),
                          cudaMemcpyDefault));
    }
    return STAMP_OK;
}

stamp_status stamp_batch_inject_wait_timeout(stamp_batch* b) {
    if (!b) return bfail(STAMP_EINVAL, "NULL batch");
    b->extra_wait = 1;
    b->wait_ns = 2000000ull;   // 2 ms
    b->graph_dirty = true;
    return STAMP_OK;
}

stamp_status stamp_batch_results(stamp_batch* b, int* iterations, float* best_cost, double* seconds_to_target,
                                 int* top3, long long* units, double* seconds) {
    if (!b) return bfail(STAMP_EINVAL, "NULL batch");
    for (int g = 0; g < b->n; ++g) {
        if (iterations) iterations[g] = b->iters_done.empty() ? 0 : b->iters_done[g];
        if (best_cost) best_cost[g] = b->best.empty() ? NAN : b->best[g];
        if (seconds_to_target) seconds_to_target[g] = b->tts.empty() ? -1.0 : b->tts[g];
    }
    if (top3) {
        std::vector<int> t(16 * (size_t)b->n);
        B_CUDA(cudaMemcpy(t.data(), b->topk, t.size() * sizeof(int), cudaMemcpyDeviceToHost));
        for (int g = 0; g < b->n; ++g)
            for (int q = 0; q < 3; ++q) top3[3 * g + q] = q < std::min(3, b->inst[g].N) ? t[16 * g + q] : -1;
    }
    if (units) *units = b->units;
    if (seconds) *seconds = b->seconds;
    return STAMP_OK;
}

stamp_status stamp_batch_read_theta(stamp_batch* b, int instance, float* theta_out) {
    if (!b || instance < 0 || instance >= b->n || !theta_out) return bfail(STAMP_EINVAL, "bad arguments");
    B_CUDA(cudaMemcpy(theta_out, b->theta + b->elem0[instance],
                      (size_t)b->inst[instance].N * b->D[instance] * sizeof(float), cudaMemcpyDefault));
    return STAMP_OK;
}

stamp_status stamp_batch_read_grad(stamp_batch* b, int instance, float* grad_out) {
    if (!b || instance < 0 || instance >= b->n || !grad_out) return bfail(STAMP_EINVAL, "bad arguments");
    B_CUDA(cudaStreamSynchronize(b->st));
    B_CUDA(cudaMemcpy(grad_out, b->grad + b->elem0[instance],
                      (size_t)b->inst[instance].N * b->D[instance] * sizeof(float), cudaMemcpyDefault));
    return STAMP_OK;
}

}  // extern "C"
