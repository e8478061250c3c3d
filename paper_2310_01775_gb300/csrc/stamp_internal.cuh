// Internal declarations of the STAMP CUDA library (sm_103a).
//
// The hot path is one Stein iteration of Algorithm 1 over N relaxed pushing
// plans: forward rollout (Sec. III-B), checkpointed adjoint, pairwise
// distances + median bandwidth, Stein direction (Eq. svgd) and Adam.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "stamp.h"

namespace stamp {

constexpr int kMaxBlocks = 4;     // n_blocks <= 4  ->  M = 4*n_blocks <= 16 choices
constexpr int kMaxH = 16;         // plan codes pack 4 bits per action into 64 bits
constexpr int kMaxTopkN = 8192;   // single-CTA bitonic sort of (cost, index)
constexpr int kMaxShares = 8;     // partial Stein directions summed by the Adam kernel
constexpr int kMaxScreenN = 4096; // particles kept by one surrogate screening

// Problem constants in the form the kernels use (derived once on the host).
struct SimConst {
    int nb, H, T, C, M, P, D, S, n_ckpt;   // n_ckpt = H*T/C
    float hs, r, k, c, mu_c, dt, inv_dt, inv_m, inv_I;
    float fric_lin;      // mu*m*g            (ground friction force scale)
    float fric_ang;      // mu*m*g*r_eff      (ground friction torque scale)
    float eps_v2, eps_w2, eps_t2;
    // contact reach: a pusher centre farther than hs*sqrt(2) + r from a
    // block centre, or a corner farther than hs*sqrt(2) from the other
    // block's centre, cannot touch it (squared, 0.1% margin)
    float disk_reach2, corner_reach2;
    float inv_tau, w_yaw, w_push, off_max, dist_max;
    float init[kMaxBlocks][3];
    float goal[kMaxBlocks][3];
};

struct RolloutArgs {
    const float* theta;     // N x D
    int N;
    uint64_t seed;
    int iter;               // < 0: no Gumbel noise
    int hard;               // 1: one-hot argmax weights
    float* tape;            // (n_ckpt + 1) x N x S
    float* cost;            // N (forward) or NULL
    float* final_state;     // N x S or NULL
    unsigned* stats_min;    // one word, atomicMin of cost bits, or NULL
    float* grad;            // N x D (adjoint): grad log rho = -dC/dtheta
    unsigned long long* dropped;   // count of particles whose reverse sweep overflowed
    const float* init_states;      // N x n_blocks x 3 initial poses (at rest), or NULL: the scene's
    int particle0;          // global index of row 0 (Gumbel draws of a shard of a larger set)
    // per-substep (cos, sin) of every block's yaw, [H*T][N][NB] float2, or
    // NULL: written by the segment replay, read by the sweep that follows it
    float2* trig;
};

// One problem instance of a batch, as the batched rollout kernels see it.
struct BatchInst {
    const float* theta;     // N x D, this instance's rows of the batch's particles
    float* grad;            // N x D
    float* tape;            // (n_ckpt + 1) x N x S
    float* cost;            // N
    int N, H, D, n_ckpt;
    int team0;              // first team of the instance in its class launch (warp aligned)
    int gid;                // index in the batch (active flags)
    unsigned long long seed;
    float init[kMaxBlocks][3];
    float goal[kMaxBlocks][3];
};
struct BatchArgs {
    const BatchInst* inst;  // the class's instances, ascending team0
    int n_inst;
    int n_teams;            // teams of the launch (a multiple of the teams per warp)
    const int* active;      // per batch instance: 0 = stopped (its teams return at once)
    const int* iter_dev;    // iteration number on the device (graph replays), or NULL
    int iter;               // iteration when iter_dev is NULL (< 0: no noise)
    int hard;
    unsigned long long* dropped;
};

// ---------------------------------------------------------------------------
// SplitMix64 (Steele, Lea & Flood 2014) as a counter-based generator: output
// number ctr+1 of the generator started at state `key` is mix(key+(ctr+1)*G).
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint64_t sm_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__host__ __device__ __forceinline__ uint64_t sm64(uint64_t key, uint64_t ctr) {
    return sm_mix(key + (ctr + 1ull) * 0x9E3779B97F4A7C15ull);
}
// Top 23 bits as a float in (0,1): ((x>>41)+0.5)/2^23, exact in float32.
__host__ __device__ __forceinline__ float u23(uint64_t x) {
    return ((float)(x >> 41) + 0.5f) * 1.1920928955078125e-7f;
}
constexpr uint64_t kStreamGumbel = 0, kStreamInit = 1;

// Streaming multiprocessors of the current device (queried once per device),
// for grid sizing.
int sm_count();

// Launchers (return the launch error).  `lanes` = threads cooperating on one
// particle in the rollout kernels.
cudaError_t launch_rollout_fwd(const SimConst& sc, const RolloutArgs& a, int lanes, cudaStream_t st);
cudaError_t launch_rollout_adj(const SimConst& sc, const RolloutArgs& a, int lanes, cudaStream_t st);
bool lanes_supported(int nb, int lanes);
int default_lanes(int nb, int N, bool adjoint);

// Segment replay (rollout_nb*.cu): the states before every substep of the
// last forward, rebuilt from its checkpoints for all (particle, segment)
// pairs at once into `full` ([H*T + 1][N][S]); `lanes` per team.
cudaError_t launch_replay(const SimConst& sc, const RolloutArgs& a, int lanes, float* full,
                          cudaStream_t st);
cudaError_t launch_replay_nb1(const SimConst&, const RolloutArgs&, int, float*, cudaStream_t);
cudaError_t launch_replay_nb2(const SimConst&, const RolloutArgs&, int, float*, cudaStream_t);
cudaError_t launch_replay_nb3(const SimConst&, const RolloutArgs&, int, float*, cudaStream_t);
cudaError_t launch_replay_nb4(const SimConst&, const RolloutArgs&, int, float*, cudaStream_t);
int replay_lanes(int nb);

// Batched launchers (rollout_nb*.cu): cta threads per CTA, a multiple of 32.
cudaError_t launch_rollout_batch(int nb, const SimConst& sc, const BatchArgs& b, int lanes, int cta,
                                 bool adjoint, cudaStream_t st);
cudaError_t launch_rollout_batch_nb1(const SimConst&, const BatchArgs&, int, int, bool, cudaStream_t);
cudaError_t launch_rollout_batch_nb2(const SimConst&, const BatchArgs&, int, int, bool, cudaStream_t);
cudaError_t launch_rollout_batch_nb3(const SimConst&, const BatchArgs&, int, int, bool, cudaStream_t);
cudaError_t launch_rollout_batch_nb4(const SimConst&, const BatchArgs&, int, int, bool, cudaStream_t);

// Per-NB launchers defined in rollout_nb*.cu.
cudaError_t launch_rollout_nb1(const SimConst&, const RolloutArgs&, int, bool, cudaStream_t);
cudaError_t launch_rollout_nb2(const SimConst&, const RolloutArgs&, int, bool, cudaStream_t);
cudaError_t launch_rollout_nb3(const SimConst&, const RolloutArgs&, int, bool, cudaStream_t);
cudaError_t launch_rollout_nb4(const SimConst&, const RolloutArgs&, int, bool, cudaStream_t);

// One-block reverse sweep as a linear recurrence in time (adjoint_time.cu),
// for checkpoint interval 1: rel and coef of the sizes below (floats) for up
// to n particles; flag receives bit 2 if a staged copy never lands.
size_t adjoint_time_coef_floats(int n, int H, int T);
size_t adjoint_time_rel_floats(int n, int H);
cudaError_t launch_adjoint_time(const SimConst& sc, const RolloutArgs& a, float* rel, float* coef,
                                int* flag, cudaStream_t st);

// SVGD step pieces (svgd.cu).  Scratch buffers are owned by the problem.
struct SvgdScratch {
    float* d2;            // N x N squared distances
    unsigned* hist;       // 2048 + 2048 + 1024 radix-select counters (zeroed per step)
    unsigned* sel;        // digit 0 and its inner rank, digit 1 and its inner rank
    unsigned* counter;    // 3 "last CTA" counters (zero between launches)
    float* h;             // bandwidth (device scalar)
    int* err;             // device error flags: 1 non-finite, 2 a bounded wait gave up
    // Stein kernel's bounded waits: polls before a wait gives up (0: the
    // library's default); skip_first_copy (a test hook) arms each CTA's first
    // shared-memory stage without issuing its copy, so that wait runs out
    unsigned wait_limit = 0;
    int skip_first_copy = 0;
};
cudaError_t launch_pairwise(const float* theta, int N, int D, const SvgdScratch& s, cudaStream_t st);
cudaError_t launch_median_digit(int N, int digit, const SvgdScratch& s, float* h_out,
                                cudaStream_t st);
// Writes `*shares` partial Stein directions (N x D each, consecutive) to part;
// at most max_shares.
// wn: normalised importance weights of Eq. dsvgd (device N), or NULL: 1/N.
cudaError_t launch_phi(const float* theta, const float* grad, int N, int D, const SvgdScratch& s,
                       float* part, int max_shares, int* shares, cudaStream_t st,
                       const float* wn = nullptr);
// The same for rows [row0, row0 + rows) of phi only (sums over all N
// particles, split into the same shares as for all rows; part holds
// `*shares` blocks of rows x D).
cudaError_t launch_phi_rows(const float* theta, const float* grad, int N, int D, int row0,
                            int rows, const SvgdScratch& s, float* part, int max_shares, int* shares,
                            cudaStream_t st, const float* wn = nullptr);
// Structured kernel (svgd_struct.cu): C (N x 2H) offset/distance parameters and
// S (N x M H) choice probabilities of each action; the Stein direction from
// the raw bandwidths of C and S (h_plain, divided by H inside).
cudaError_t launch_struct_prep(const float* theta, int N, int H, int M, float* C, float* S,
                               cudaStream_t st);
// Writes `*shares` partial directions (N x D each, consecutive; at most max_shares).
cudaError_t launch_struct_phi(const float* theta, const float* grad, const float* C, const float* S,
                              int N, int H, int M, const float* hc_dev, const float* hz_dev,
                              const float* wn, float* phi, int max_shares, int* shares,
                              cudaStream_t st);
cudaError_t launch_scale_scalar(const float* src, float s, float* dst, cudaStream_t st);
// Normalised Eq. dsvgd weights from the relaxed and hard costs (device N each).
cudaError_t launch_dsvgd_weights(const float* c_relaxed, const float* c_hard, int N, float* wn,
                                 cudaStream_t st);
// Adam on -phi, phi = sum of the `shares` partials (stride n_elems); writes
// phi to phi_out when given.
cudaError_t launch_adam(float* theta, const float* part, int shares, float* phi_out, float* m,
                        float* v, int n_elems, int step, float lr, int* flag, cudaStream_t st);
cudaError_t launch_init_theta(float* theta, int N, int D, uint64_t seed, cudaStream_t st);

// Batched Stein step pieces (svgd.cu): one launch covers every instance of a
// batch through per-CTA work items; CTAs of stopped instances return at once.
struct SvgdInst {
    const float* theta;     // N x D (16-byte aligned)
    const float* grad;      // N x D (16-byte aligned)
    float* d2;              // N x N
    unsigned* hist;         // 2048 + 2048 + 1024 (zeroed before the pairwise launch)
    unsigned* sel;          // 4
    unsigned* counter;      // 3, zero between launches
    float* h;               // bandwidth
    float* part;            // shares x N x D
    int N, D;
    int nt;                 // pairwise tiles per side
    int med_ctas;           // CTAs of each median-digit pass
    int shares, j_chunk;    // Stein-sum split (as for one problem of N particles)
    int gid;                // index in the batch (active flags)
    long long elem0;        // first element of the instance in the concatenated particles
};
cudaError_t launch_pairwise_batch(const SvgdInst* inst, const int4* items, int n_items, int max_D,
                                  const int* active, cudaStream_t st);
cudaError_t launch_median_digit_batch(const SvgdInst* inst, const int2* items, int n_items,
                                      const int* active, int digit, cudaStream_t st);
cudaError_t launch_phi_batch(const SvgdInst* inst, const int4* items, int n_items, int max_D,
                             const int* active, int* err, cudaStream_t st);
// step_dev: Adam steps taken so far; bc[s] = (1 - 0.9^s, 1 - 0.999^s).
cudaError_t launch_adam_batch(float* theta, float* m, float* v, long long n, const SvgdInst* inst,
                              int n_inst, const int* active, const int* step_dev, const float2* bc,
                              float lr, int* flag, cudaStream_t st);
// The single-problem Stein-sum split for N particles, and rows per phi CTA.
void phi_batch_plan(int N, int* shares, int* j_chunk);
int phi_rows_per_block();
cudaError_t launch_topk(const float* theta, const float* cost, int N, const SimConst& sc, int k,
                        int* topk_out, cudaStream_t st);

// Persistent batched iteration (batch_persist.cu): one launch runs a whole
// Stein iteration of every active instance.  Each CTA of kPersistThreads
// takes work items from a device-wide queue in this order -- rollout items
// (kPersistWarps warp tasks: forward, then adjoint, of up to 32/L particles
// of one instance), pairwise tiles, median-digit-1 CTAs, median-digit-2
// CTAs, Stein-direction blocks, Adam chunks -- and waits (bounded) only on
// items of the same instance earlier in the queue.
constexpr int kPersistThreads = 256;
constexpr int kPersistWarps = kPersistThreads / 32;
constexpr int kPersistRows = kPersistWarps * 4;   // Stein-direction rows per item
constexpr int kPersistAdamChunk = 4096;           // particle elements per Adam item
constexpr int kPersistDeps = 5;                   // completion counters per instance
constexpr int kPersistStrip = 8;                  // pairwise tile pairs per item (one tile row)
// lanes per particle team in the persistent kernel, by block count
__host__ __device__ constexpr int persist_lanes(int nb) { return nb == 1 ? 2 : nb == 2 ? 4 : 8; }
// Stein-direction column slots per lane for the batch's largest D
__host__ __device__ constexpr int persist_dp(int max_D) { return max_D <= 96 ? 3 : max_D <= 192 ? 6 : 9; }
struct PersistArgs {
    const BatchInst* inst;  // per batch instance (n_ckpt of its class's interval)
    const SvgdInst* sinst;  // per batch instance
    const int4* need;       // per instance: rollout warps, pairwise tiles, median CTAs, Stein items
    const int4* warps;      // kPersistWarps per rollout item: (instance or -1, first particle, n_blocks, 0)
    const int4* pw;         // (instance, tile row, first and end tile column of a strip)
    const int2* med;        // (instance, CTA), for both median digits
    const int4* phi;        // (instance, row block of kPersistRows, j-share, 0)
    const int2* adam;       // (instance, chunk)
    int n_roll, n_pw, n_med, n_phi, n_adam, n_inst;
    const int* active;
    int* iter;              // Stein iterations so far (Gumbel key); the last CTA out bumps it
    int* step;              // Adam steps so far; likewise
    const float2* bc;       // Adam bias corrections by step
    float lr;
    float *theta, *m, *v;   // the batch's concatenated particles and Adam moments
    unsigned* ctr;          // [0] next item, [1] CTAs finished, [2] abort; zero between launches
    unsigned* dep;          // kPersistDeps per instance, zero between launches: rollout warps,
                            // pairwise tiles, median-1 CTAs, median-2 CTAs, Stein items done
    int* flag;              // bit 0: non-finite; bit 1: a bounded wait gave up
    unsigned long long* dropped;
    int seg_warp;           // float2 of shared memory per warp for the adjoint's segments
    int dp;                 // Stein-direction column slots per lane: 3, 6 or 9
    int extra_wait;         // added to the Stein items' rollout target (> 0: a wait that runs out)
    unsigned long long wait_ns;   // a dependency wait gives up after this long
    // trace (NULL: off): entry k of the last launch = item k's claim,
    // work-start (dependencies met) and end times, and its SM
    stamp_trace_entry* trace;
    int trace_cap;
};
// Dynamic shared memory the launch needs, and the grid (all resident CTAs).
size_t persist_smem(int max_D, int seg_warp);
cudaError_t persist_grid(size_t smem, int* grid);
// cls[nb - 1]: the constants of the n_blocks = nb class (unused classes: anything).
cudaError_t launch_persist(const PersistArgs& p, const SimConst* cls, int grid, size_t smem,
                           cudaStream_t st);

// Problem constants of a problem object, and a forward rollout (timed like
// the solve's) from per-particle start poses (N x n_blocks x 3, at rest).
SimConst problem_const(const stamp_problem* p);
stamp_status rollout_from(stamp_problem* p, const float* theta, const float* init_states, int N,
                          uint64_t seed, int iter, float* cost, float* final_state);

// Surrogate pieces (surrogate.cu) used by the surrogate-assisted solve.
stamp_status surrogate_rollout(stamp_surrogate* s, const SimConst& sc, const float* theta, int N,
                               uint64_t seed, int iter, float* cost, float* grad, unsigned* stats_word);
stamp_status surrogate_screen(stamp_surrogate* s, const SimConst& sc, const float* cand, int n_cand,
                              int N, float* theta_out, int* index_out);
float* surrogate_candidates(stamp_surrogate* s);
int surrogate_max_rows(const stamp_surrogate* s);
int surrogate_max_particles(const stamp_surrogate* s);
cudaStream_t surrogate_stream(const stamp_surrogate* s);

// Text returned by stamp_last_error() on the calling thread.
void set_last_error(const char* msg);

}  // namespace stamp
