/*
 * stamp.h -- C ABI of the GB300 (sm_103a) STAMP hot path.
 *
 * STAMP (Stein Task and Motion Planning) treats planning as inference over
 * relaxed plans theta (Sec. IV-A): each of N particles is rolled through a
 * differentiable simulation, its goal cost C gives log rho = -C
 * (Eq. posterior_dist, neglog_likelihood), gradients come from the reverse
 * sweep through the trajectory (Sec. III-B), and the particles move by the
 * Stein variational update (Eq. svgd, Eq. dsvgd with unit weights), followed
 * by an SGD phase and the recovery of discrete plans Gamma(theta)
 * (Algorithm 1).  The problem here is planar block pushing (Sec. V-A-2):
 * n_blocks square blocks, H pushes, each a relaxed choice among M = 4*n_blocks
 * (object, side) pairs plus a contact offset and a push distance.
 *
 * Particle layout: theta is N x D float32, row-major, D = H*(M+2); action k
 * occupies columns [k*(M+2), (k+1)*(M+2)) as [M logits, u, v] with
 * offset = offset_max*tanh(u) and distance = dist_max*sigmoid(v).
 * State layout: per block (x, y, yaw, vx, vy, omega); S = 6*n_blocks floats.
 *
 * Conventions for every call:
 *  - Pointers documented "device" must be device (or managed) memory; the
 *    caller owns them.  "host" means ordinary or pinned host memory.
 *  - All work is enqueued on the stream given at create and is asynchronous,
 *    except stamp_solve and stamp_sync, which wait for it.
 *  - Errors are returned as stamp_status and never thrown; the text of the
 *    last error on the calling thread is in stamp_last_error().
 *  - Errors found by the device (non-finite values) raise a flag that the
 *    next stamp_sync or stamp_solve reports as STAMP_ENONFINITE.
 *  - No call allocates memory except stamp_problem_create, which sizes every
 *    buffer for max_particles.  Calls on one problem must not overlap.
 */
#ifndef STAMP_H
#define STAMP_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    STAMP_OK = 0,
    STAMP_EINVAL = 1,      /* bad argument (null, size out of range, wrong pointer kind) */
    STAMP_ENOMEM = 2,      /* allocation failed in stamp_problem_create */
    STAMP_ECUDA = 3,       /* a CUDA runtime call failed; see stamp_last_error() */
    STAMP_ENONFINITE = 4,  /* a NaN/Inf cost, gradient or particle was produced */
    STAMP_ETIMEOUT = 5     /* a bounded device-side wait on an asynchronous copy gave up */
} stamp_status;

typedef struct stamp_problem stamp_problem;   /* opaque, owned by the library */

/* Problem description, SI units.  Sec. III-B fixes only the model class
 * (semi-implicit Euler, spring-based penalty contact); the numbers are the
 * caller's.  Constraints: 1 <= n_blocks <= 4, 1 <= H <= 16, T >= 1,
 * ckpt_every >= 1 with T % ckpt_every == 0, every length/mass/stiffness > 0. */
typedef struct {
    int n_blocks;      /* blocks in the scene */
    int H;             /* pushes per plan (K in the paper) */
    int T;             /* substeps per push */
    int ckpt_every;    /* tape checkpoint interval C in substeps */
    float half_size;   /* block half side [m] */
    float mass;        /* block mass [kg] */
    float mu;          /* ground Coulomb coefficient */
    float mu_c;        /* contact (pusher/block, block/block) Coulomb coefficient */
    float g;           /* gravity [m/s^2] */
    float pusher_r;    /* pusher disk radius [m] */
    float k_contact;   /* penalty stiffness [N/m] */
    float c_contact;   /* penalty damping [N s/m] */
    float eps_v;       /* ground friction smoothing, linear [m/s] */
    float eps_w;       /* ground friction smoothing, angular [rad/s] */
    float eps_t;       /* contact friction smoothing [m/s] */
    float dt;          /* substep [s] */
    float tau;         /* Gumbel-softmax temperature */
    float w_yaw;       /* cost weight of the squared wrapped yaw error */
    float w_push;      /* cost weight of the squared push distances */
    float offset_max;  /* contact offset range [-offset_max, offset_max] [m] */
    float dist_max;    /* push distance range [0, dist_max] [m] */
} stamp_problem_desc;

/* Create a problem: scene (Sec. V-A-2), cost (App. D.2 restated as squared
 * pose error) and every device buffer for up to max_particles particles.
 *   init_poses, goal_poses: host, n_blocks x 3 (x, y, yaw), copied.
 *   max_particles: 1..16384 (the pairwise-distance scratch is N^2 floats).
 *   cuda_stream: a cudaStream_t (NULL = legacy default stream).
 *   out: receives the problem; NULL on failure.
 * Returns STAMP_EINVAL for a bad description, STAMP_ENOMEM / STAMP_ECUDA if
 * allocation fails (nothing is leaked). */
stamp_status stamp_problem_create(const stamp_problem_desc* desc, const float* init_poses,
                                  const float* goal_poses, int max_particles,
                                  void* cuda_stream, stamp_problem** out);

/* Free the problem and all its device buffers (waits for its stream). NULL is a no-op. */
void stamp_problem_destroy(stamp_problem* prob);

/* Forward rollout of N particles (Algorithm 1, "simulate plans"; Sec. III-B).
 *   theta: device N x D.
 *   seed, iter: Gumbel noise of iteration iter (counter-based SplitMix64,
 *     Steele et al. 2014); iter < 0 means no noise.
 *   hard: 0 = relaxed weights softmax((a+g)/tau) (Eq. gamma_map, Gamma~);
 *         1 = one-hot argmax(a+g), ties to the lowest index (Gamma).
 *   cost: device N, receives C(theta_i).
 *   final_state: device N x S, or NULL.
 * Keeps a checkpoint tape (every ckpt_every substeps) for stamp_rollout_adjoint. */
stamp_status stamp_rollout_fwd(stamp_problem* prob, const float* theta, int N,
                               unsigned long long seed, int iter, int hard, float* cost,
                               float* final_state);

/* stamp_rollout_fwd from per-particle start poses: init_states (device,
 * N x n_blocks x 3: x, y, yaw per block, at rest) replaces the scene's start
 * poses (e.g. replanning from the current state, or simulating
 * transitions).  The tape it keeps serves stamp_rollout_adjoint only for the
 * gradient with respect to theta at these start poses. */
stamp_status stamp_rollout_fwd_from(stamp_problem* prob, const float* theta,
                                    const float* init_states, int N, unsigned long long seed,
                                    int iter, int hard, float* cost, float* final_state);

/* Reverse sweep (Sec. III-B: gradients back-propagated through the whole
 * trajectory) of the last stamp_rollout_fwd, recomputing the substeps between
 * checkpoints.  theta, N, seed and iter must be those of that call
 * (STAMP_EINVAL otherwise; theta's contents are not checked).
 *   grad_logp: device N x D, receives grad log rho = -dC/dtheta. */
stamp_status stamp_rollout_adjoint(stamp_problem* prob, const float* theta, int N,
                                   unsigned long long seed, int iter, float* grad_logp);

/* Particles whose reverse sweep overflowed float32 get a zero gradient in
 * stamp_rollout_adjoint (the gradient through long contact-rich rollouts can
 * explode; App. E.5 of the paper notes the effect); *count receives how many
 * such particle gradients were zeroed since the problem was created.  Waits
 * for the stream. */
stamp_status stamp_dropped_gradients(stamp_problem* prob, long long* count);

/* Copy the tape of the last stamp_rollout_fwd into tape_out (device),
 * laid out [H*T/ckpt_every + 1][N][S]: the state before substep c*ckpt_every
 * for c < H*T/ckpt_every, then the final state.  N must be that call's N. */
stamp_status stamp_read_tape(stamp_problem* prob, int N, float* tape_out);

/* One particle update of Algorithm 1.
 * SVGD phase (sgd_phase = 0), Eq. svgd with the RBF kernel
 *   k(a,b) = exp(-|a-b|^2/h), h = med/ln(N+1), med the lower median of the
 *   N(N-1)/2 squared pairwise distances (the median heuristic of App. C.3):
 *   phi_i = (1/N) sum_j [k_ij grad_logp_j + (2/h) k_ij (theta_i - theta_j)].
 * SGD phase (sgd_phase = 1): phi_i = grad_logp_i.
 * Then one bias-corrected Adam step (Kingma & Ba 2015; beta 0.9/0.999,
 * eps 1e-8) with gradient -phi:
 *   theta: device N x D, updated in place.   grad_logp: device N x D.
 *     Both 16-byte aligned (their row tiles are streamed by TMA bulk copies).
 *   adam_m, adam_v: device N x D moments, updated in place (zero at step 1).
 *   step: Adam step number, >= 1.   lr: step size.
 *   h_out: device float or NULL, receives h (1 in the SGD phase).
 *   phi_out: device N x D or NULL, receives phi. */
stamp_status stamp_svgd_step(stamp_problem* prob, float* theta, const float* grad_logp, int N,
                             float* adam_m, float* adam_v, int step, float lr, int sgd_phase,
                             float* h_out, float* phi_out);

/* ---- Particle shards (one Stein iteration over several GPUs) -------------
 * Eq. svgd sums over all particles j, but the rollout, its reverse sweep and
 * the update of particle i need only particle i: a set of N particles can be
 * split into contiguous shards, one per GPU.  Each shard rolls out its own
 * rows, the shards exchange theta and grad log rho (an all-gather of N x D
 * floats each, done by the caller, e.g. with NCCL), and each computes the
 * bandwidth from all N (the same value everywhere) and the Stein direction
 * and Adam step of its own rows.  With the offsets below, the shards
 * together compute bit for bit what one problem computes for all N.
 *
 * stamp_set_particle_offset: later rollouts of this problem treat their row
 * r as particle particle0 + r of the full set (its Gumbel draws, Eq.
 * gamma_map); 0 (the default) for an unsharded problem. */
stamp_status stamp_set_particle_offset(stamp_problem* prob, int particle0);
/* The update of rows [row0, row0 + rows) of an N-particle set:
 *   theta_all, grad_all: device N x D, the gathered particles and
 *     grad log rho (16-byte aligned);
 *   theta_rows: device rows x D, this shard's particles, updated in place;
 *   adam_m, adam_v: device rows x D, this shard's moments;
 *   step, lr, sgd_phase, h_out: as in stamp_svgd_step;
 *   phi_out: device rows x D or NULL.
 * N <= max_particles (the N x N distances live in the problem).  The RBF
 * kernel only (kind 0), unit weights. */
stamp_status stamp_svgd_step_rows(stamp_problem* prob, const float* theta_all, const float* grad_all,
                                  int N, int row0, int rows, float* theta_rows, float* adam_m,
                                  float* adam_v, int step, float lr, int sgd_phase, float* h_out,
                                  float* phi_out);

/* Algorithm 1 end to end: svgd_iters SVGD updates then sgd_iters SGD
 * updates (iteration it uses Gumbel noise (seed, it) and Adam step it+1),
 * then the hard evaluation of every particle (Gamma, no noise) and the
 * first k distinct discrete plans in (cost, index) order.
 *   theta_init: N x D, host or device, or NULL for theta ~ U(-1,1)^D
 *     (the uniform base distribution of App. A.1) drawn from (seed, stream 1).
 *   theta_out: N x D, host or device, final particles.
 *   cost_out: N, host or device, hard-evaluation costs (or NULL).
 *   k, topk_particle: host k ints, particle index of each kept plan, -1 padded
 *     (k = 0 and NULL allowed).  N <= 8192 when k > 0.
 *   stats_out: host svgd_iters+sgd_iters floats, minimum relaxed cost of each
 *     iteration, or NULL.
 * Host pointers are detected with cudaPointerGetAttributes and staged through
 * the problem's buffers.  Waits for the stream; returns STAMP_ENONFINITE if a
 * non-finite value appeared. */
stamp_status stamp_solve(stamp_problem* prob, int N, int svgd_iters, int sgd_iters,
                         unsigned long long seed, float lr, const float* theta_init,
                         float* theta_out, float* cost_out, int k, int* topk_particle,
                         float* stats_out);

/* Wait for the problem's stream and report device-detected errors. */
stamp_status stamp_sync(stamp_problem* prob);

/* Kernel timing (CUDA events on the problem's stream around every launch).
 * stamp_set_profiling(prob, 1) starts recording and clears the totals; the
 * totals are gathered at stamp_sync / stamp_solve.  Kernel ids: */
enum {
    STAMP_K_ROLLOUT_FWD = 0,  /* forward rollout (relaxed or hard) */
    STAMP_K_ROLLOUT_ADJ = 1,  /* reverse sweep (time-parallel or replay: all its launches together) */
    STAMP_K_PAIRWISE = 2,     /* pairwise distances + first median digit */
    STAMP_K_MEDIAN = 3,       /* remaining median digits */
    STAMP_K_PHI = 4,          /* Stein direction */
    STAMP_K_ADAM = 5,         /* Adam update */
    STAMP_K_TOPK = 6,         /* sort + distinct plans */
    STAMP_K_INIT = 7,         /* initial particles */
    STAMP_K_SURROGATE = 8,    /* surrogate rollout with its reverse sweep (all its launches) */
    STAMP_K_SCREEN = 9,       /* candidate generation + surrogate screening (all its launches) */
    STAMP_NKERNELS = 10
};
stamp_status stamp_set_profiling(stamp_problem* prob, int enable);
/* The same for the kernel ids whose bit is set in mask (bit k = id k); the
 * others launch without events.  Fewer events keep their own cost out of a
 * timed solve.  0 stops recording. */
stamp_status stamp_set_profiling_mask(stamp_problem* prob, unsigned mask);
/* ms_out, launches_out: host arrays of STAMP_NKERNELS (either may be NULL). */
stamp_status stamp_get_kernel_times(stamp_problem* prob, double* ms_out, long long* launches_out);

/* Measured FP32 FMA throughput of the current device, the roof against
 * which the rollout and reverse-sweep kernels (FP32-ALU bound: contact
 * forces, friction and integration per substep) are reported.  The paper
 * has no counterpart; it states no hardware.  Every thread of a grid that
 * fills each SM runs 8 independent fmaf chains; `launches` timed launches
 * (CUDA events, after two warm-up launches) on a stream of its own, median
 * taken; FLOP = 2 per FMA.  Allocates and frees a small buffer, waits for
 * its launches.
 *   tflops_out: host, receives TFLOP/s; ms_per_launch_out: host or NULL. */
stamp_status stamp_fp32_fma_peak(int launches, double* tflops_out, double* ms_per_launch_out);

/* The solves compute each SVGD iteration's RBF bandwidth (pairwise
 * distances and median, which depend on the particles only) on a second
 * stream of the problem's own, concurrently with the iteration's rollouts,
 * and the Stein direction waits for both (enable = 1, the default); 0: one
 * after the other on the problem's stream.  Results are identical. */
stamp_status stamp_set_overlap(stamp_problem* prob, int enable);

/* How stamp_rollout_adjoint and the solves run the reverse sweep.
 * STAMP_ADJ_TIME_PARALLEL applies to one-block scenes with ckpt_every = 1:
 * the adjoint of a semi-implicit Euler substep is linear in the adjoint of
 * the state after it, with coefficients (the Jacobian of the block's force
 * and torque, and the linear forms of the action parameters' adjoints) that
 * depend on the forward state only.  They are computed for every (particle,
 * substep) pair at once from the tape; then one short recurrence per
 * particle runs backwards.  Scratch: 44 floats per particle and substep,
 * allocated at create (not when it would exceed 4 GiB).
 * STAMP_ADJ_SEQUENTIAL: each particle's team differentiates substep after
 * substep, recomputing each segment of ckpt_every substeps from its
 * checkpoint on the same serial path.
 * STAMP_ADJ_REPLAY applies to ckpt_every > 1: one launch rebuilds the states
 * before every substep from the checkpoints for all (particle, segment)
 * pairs at once (the segments are independent given their checkpoints),
 * into a scratch tape of interval 1 ((H*T + 1) x N x S floats, allocated at
 * create when at most 4 GiB); then the sequential sweep runs on that tape
 * with nothing to recompute.  The forward still stores only every
 * ckpt_every-th state.
 * STAMP_ADJ_AUTO (the default): time-parallel where it applies, for up to
 * 3072 particles (beyond that the sequential teams fill the GPU and the
 * Jacobians' extra arithmetic costs more than it saves), else the replay
 * where it applies, else sequential.
 * All sweeps give the gradient of the same float32 simulation, with sums
 * taken in a different order. */
enum { STAMP_ADJ_SEQUENTIAL = 0, STAMP_ADJ_TIME_PARALLEL = 1, STAMP_ADJ_AUTO = 2,
       STAMP_ADJ_REPLAY = 3 };
stamp_status stamp_set_adjoint_mode(stamp_problem* prob, int mode);
/* The sweep (STAMP_ADJ_SEQUENTIAL, STAMP_ADJ_TIME_PARALLEL or
 * STAMP_ADJ_REPLAY) that a call with N particles uses. */
stamp_status stamp_get_adjoint_mode(stamp_problem* prob, int N, int* mode);

/* Failure-detection test hook (no paper counterpart).  The next launch of
 * the RBF Stein-direction kernel on this problem (stamp_svgd_step or a
 * solve's SVGD iteration) runs with each CTA's first shared-memory stage
 * armed on its mbarrier but its bulk copy never issued, and with its waits
 * bounded at 4096 polls: the wait runs out, the CTA waits (bounded) for its
 * other copy in flight, raises the device error flag and returns, and the
 * next stamp_sync / stamp_solve reports STAMP_ETIMEOUT.  No GPU fault, trap
 * or hang is involved; that step's results are not valid.  One-shot: later
 * calls run normally. */
stamp_status stamp_inject_wait_timeout(stamp_problem* prob);

/* Lanes per particle used by the rollout kernels (1,2,4,8,16,32; 0 = automatic). */
stamp_status stamp_set_lanes(stamp_problem* prob, int fwd_lanes, int adj_lanes);
/* Lanes per (particle, segment) team of the segment replay (STAMP_ADJ_REPLAY):
 * one block 1, 2, 4; two blocks 2..16; three blocks 2..32; four blocks
 * 4..32; 0 = automatic. */
stamp_status stamp_set_replay_lanes(stamp_problem* prob, int lanes);

/* Stein step without any device allocation.  The paper has no counterpart:
 * this serves callers that cannot call cudaMalloc -- code whose device memory
 * belongs to someone else's allocator or pool (which must not be bypassed),
 * code that runs where allocating is forbidden, or a device whose memory is
 * already fully reserved -- and so cannot create a stamp_problem.
 * It runs stamp_svgd_step's kernels with the plain RBF kernel (kind 0 of
 * stamp_set_svgd_kernel) and unit weights, for N <= STAMP_NOALLOC_MAX_N
 * particles of dimension D <= STAMP_NOALLOC_MAX_D (larger sizes are rejected
 * with STAMP_EINVAL).  It sums the Stein direction over j in one share where
 * stamp_svgd_step may split that sum over several CTAs, so the two agree to
 * within the rounding of that grouping.  Its scratch memory (pairwise
 * distances, Stein direction, histograms, counters, bandwidth; about 5.4 MB)
 * is one fixed device array that every GPU loading the library holds until
 * the process exits.
 *   theta, grad_logp: device N x D, 16-byte aligned; adam_m, adam_v: device
 *   N x D; step >= 1; lr; sgd_phase; h_out, phi_out: device or NULL (as in
 *   stamp_svgd_step); cuda_stream: the cudaStream_t to run on (NULL = legacy
 *   default stream).
 * The first call on a device sets up that device's scratch address (a symbol
 * lookup, kept for the life of the process: a device reset is not
 * supported), so make that first call before any stream capture.  Each call
 * reads back the device error flag and waits for its stream; it returns
 * STAMP_ENONFINITE if a non-finite value appeared.  Every call shares the one
 * array and it keeps the last call's contents (the call clears what must
 * start at zero): calls that overlap on the GPU (other streams, other host
 * threads) race. */
#define STAMP_NOALLOC_MAX_N 1024
#define STAMP_NOALLOC_MAX_D 288
stamp_status stamp_svgd_step_noalloc(float* theta, const float* grad_logp, int N, int D,
                                     float* adam_m, float* adam_v, int step, float lr,
                                     int sgd_phase, float* h_out, float* phi_out,
                                     void* cuda_stream);

/* ---- MLP dynamics surrogate (BF16 tensor cores) ---------------------------
 * A 4-layer perceptron in_dim -> 256 -> 256 -> 256 -> out_dim with SiLU
 * activations and a linear head, BF16 weights and activations, FP32
 * accumulation (tcgen05 MMA into tensor memory).  It stands in for the
 * simulator's per-push transition (the learned dynamics of the surrogate
 * workload; the paper itself simulates every plan, Sec. III-B). */
typedef struct stamp_mlp stamp_mlp;
/* 1 <= in_dim <= 32, 1 <= out_dim <= 16; scratch for up to max_rows rows per
 * forward, and saved activations (about 5.8 KB per row) for train_rows rows
 * for the backward pass (0: inference only). */
stamp_status stamp_mlp_create(int in_dim, int out_dim, int max_rows, int train_rows,
                              void* cuda_stream, stamp_mlp** out);
void stamp_mlp_destroy(stamp_mlp* mlp);
/* Number of floats of the packed parameter vector: for each layer l, W_l as
 * (out_l, in_l) row-major, then b_l (out_l). */
size_t stamp_mlp_param_count(int in_dim, int out_dim);
/* params: device, the packed FP32 parameters; converted to BF16 tiles. */
stamp_status stamp_mlp_set_params(stamp_mlp* mlp, const float* params);
/* y (device rows x out_dim FP32) = MLP(x (device rows x in_dim FP32)); asynchronous. */
stamp_status stamp_mlp_forward(stamp_mlp* mlp, const float* x, int rows, float* y);
/* The same, keeping the activations for stamp_mlp_backward in the saved
 * tiles [tile_base, tile_base + ceil(rows/128)) (several batches, e.g. the
 * pushes of a plan, can be kept side by side). */
stamp_status stamp_mlp_forward_saved(stamp_mlp* mlp, const float* x, int rows, float* y,
                                     int tile_base);
/* Reverse sweep of the forward saved at tile_base: given dy = dL/dy (device
 * rows x out_dim), writes dx = dL/dx (device rows x in_dim, or NULL) and
 * dparams = dL/dparams (device, packed like the parameters, or NULL).  The
 * input gradient runs on the tensor cores (BF16, FP32 accumulation); the
 * weight gradients are FP32 reductions over the rows on the CUDA cores. */
stamp_status stamp_mlp_backward(stamp_mlp* mlp, const float* dy, int rows, int tile_base,
                                float* dx, float* dparams);
/* Adam (lr, beta 0.9/0.999) on the mean squared error of MLP(x) against
 * target (device rows x in_dim / rows x out_dim), minibatches of `batch`
 * consecutive rows, `epochs` passes; params (device, packed) updated in place;
 * loss_out: host, mean loss of each epoch (or NULL).  Waits for the stream. */
stamp_status stamp_mlp_train(stamp_mlp* mlp, float* params, const float* x, const float* target,
                             int rows, int epochs, int batch, float lr, float* loss_out);
/* Wait for the MLP's stream; STAMP_ETIMEOUT if a bounded device wait gave up. */
stamp_status stamp_mlp_sync(stamp_mlp* mlp);

/* ---- Surrogate-assisted planning -----------------------------------------
 * A learned pose-dynamics model of one push (the paper simulates every plan,
 * Sec. III-B; this model lets the early iterations and the screening of many
 * candidates skip the simulator).  For push k of a plan:
 *   f_k = [x_b, y_b, cos phi_b, sin phi_b for each block b] ++ z~_k
 *         ++ [tanh u_k, sigmoid v_k]                       (8 n_blocks + 2 values)
 *   q_{k+1} = q_k + MLP(f_k)       (each block's (dx, dy, dphi), world frame)
 * with z~_k, u_k, v_k the relaxed action of Eq. gamma_map and MLP the network
 * above (in_dim 8 n_blocks + 2, out_dim 3 n_blocks).  The plan's cost is the
 * simulator's cost on q_H, and its gradient runs through the H chained
 * network evaluations (input-gradient MMAs on the tensor cores).
 * Training transitions: one relaxed push from a random start scene.  With
 * sm64(k, c) = SplitMix64 output c+1 of a generator started at state k and
 * U(.) its top 23 bits as ((x >> 41) + 0.5) / 2^23: transition g of `seed`
 * sits in chunk c0 = g - g mod 4096 (chunk key cs = sm64(seed, c0)) at local
 * index i.  Start poses: attempt a = 0..31 draws u = U(sm64(sm64(cs, 2),
 * (32 i + a) * 12 + 3 b + q)) for block b, coordinate q, and sets
 * x = u - 1/2, y = u - 1/2, phi = (u - 1/2) * 3.14159265 in float32; the
 * first attempt with all block centres more than 0.16 m apart is taken.
 * Action: u_j = U(sm64(sm64(cs, 3), i (M + 3) + j)), theta_j = (u_j - 1/2) * 6
 * for j < M + 2, the M logits multiplied by u_{M+2}.  The push is simulated
 * with the description's physics (Gumbel noise of seed cs, iteration 0); the
 * target is each block's pose change. */
typedef struct stamp_surrogate stamp_surrogate;
/* desc: the physics of the simulated transitions (n_blocks 1..3; its H is
 * the longest horizon the surrogate will roll out; T as in the problems it
 * serves).  max_rows: the largest candidate set to screen (<= 2^20);
 * max_particles: the largest N of a rollout with gradients.  All device
 * memory is allocated here (the candidate set, poses and features of
 * max_rows rows, the MLP's saved activations for H * max_particles rows);
 * the surrogate runs on cuda_stream. */
stamp_status stamp_surrogate_create(const stamp_problem_desc* desc, int max_rows,
                                    int max_particles, void* cuda_stream, stamp_surrogate** out);
void stamp_surrogate_destroy(stamp_surrogate* s);
/* Network input and output widths; returns the packed parameter count. */
int stamp_surrogate_dims(const stamp_surrogate* s, int* in_dim, int* out_dim);
/* Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights and biases from the
 * counter generator with key `seed` (draw t = index in the packed vector). */
stamp_status stamp_surrogate_init_params(stamp_surrogate* s, unsigned long long seed);
/* params: device, packed as for stamp_mlp_set_params. */
stamp_status stamp_surrogate_set_params(stamp_surrogate* s, const float* params);
stamp_status stamp_surrogate_get_params(stamp_surrogate* s, float* params);
/* The first n transitions of `seed`: x_out (device n x in_dim) features,
 * y_out (device n x 3 n_blocks) pose changes.  Asynchronous. */
stamp_status stamp_surrogate_transitions(stamp_surrogate* s, int n, unsigned long long seed,
                                         float* x_out, float* y_out);
/* Train the surrogate's own parameters on n transitions (device x: n x in_dim,
 * y: n x out_dim).  Transitions in which a block moved more than 0.5 m or
 * turned more than pi (blow-ups of the explicit contact integration) are
 * dropped; the targets are standardized per output (mean, standard
 * deviation over the kept rows); Adam (lr) minimises the mean squared error
 * in standardized units over `epochs` passes of consecutive minibatches of
 * `batch` rows (batch <= max(16384, H * max_particles rounded up to 128));
 * then the scaling is folded back into the output layer, so the parameters
 * always predict pose changes in metres and radians.  loss_out: host, the
 * mean standardized loss of each epoch, or NULL.  Allocates its scratch
 * (about (in_dim + out_dim) * 4 bytes per transition) for the call; waits
 * for the stream. */
stamp_status stamp_surrogate_train(stamp_surrogate* s, const float* x, const float* y, int n,
                                   int epochs, int batch, float lr, float* loss_out);
/* Transitions the last stamp_surrogate_train call kept. */
int stamp_surrogate_last_kept(const stamp_surrogate* s);
/* Surrogate cost (device N) of the plans theta (device N x D) of problem p
 * (its scene, goal, horizon and relaxation; same n_blocks), Gumbel noise of
 * (seed, iter) as in stamp_rollout_fwd (iter < 0: none), and, when
 * grad_logp (device N x D) is given, -dC/dtheta (N <= max_particles; without
 * it N <= max_rows).  Asynchronous on the surrogate's stream. */
stamp_status stamp_surrogate_rollout(stamp_surrogate* s, stamp_problem* p, const float* theta,
                                     int N, unsigned long long seed, int iter, float* cost,
                                     float* grad_logp);
/* The N candidates (device n_candidates x D) of lowest noise-free surrogate
 * cost, ties to the lower index, in ascending cost order: theta_out (device
 * N x D) and their indices (device N ints, or NULL).  N <= 4096. */
stamp_status stamp_surrogate_screen(stamp_surrogate* s, stamp_problem* p, const float* candidates,
                                    int n_candidates, int N, float* theta_out, int* index_out);
/* Wait for the surrogate's stream; STAMP_ETIMEOUT if a bounded device wait gave up. */
stamp_status stamp_surrogate_sync(stamp_surrogate* s);
/* Algorithm 1 with the surrogate: n_candidates >= N particles drawn as in
 * stamp_solve (theta ~ U(-1,1)^D from seed; the first N are stamp_solve's
 * start), the N of lowest noise-free surrogate cost kept (n_candidates == N:
 * all, in order), then surrogate_iters SVGD iterations on the surrogate's
 * gradients, sim_iters SVGD iterations and sgd_iters plain-gradient
 * iterations on the simulator's (Adam's step count runs on), then the hard
 * evaluation and top-k of stamp_solve.  stats_out: host, minimum relaxed
 * cost of each iteration (the surrogate's cost in its iterations), or NULL.
 * p and s must run on the same stream; N <= max_particles of both, and
 * N <= 4096 when screening. */
stamp_status stamp_solve_surrogate(stamp_problem* p, stamp_surrogate* s, int n_candidates, int N,
                                   int surrogate_iters, int sim_iters, int sgd_iters,
                                   unsigned long long seed, float lr, float* theta_out,
                                   float* cost_out, int k, int* topk_particle, float* stats_out);
/* Importance weights of Eq. dsvgd, w_j = p~*(Gamma~(theta_j)) / p*(Gamma(theta_j))
 * = exp(C_j - C~_j) with C~_j the relaxed and C_j the hard cost of particle j
 * under the same Gumbel draws; the Stein direction becomes
 * phi_i = sum_j (w_j / w) [k_ji grad log rho_j + grad_{theta_j} k_ji],
 * w = sum_j w_j (unit weights give the 1/N of stamp_svgd_step).  A particle
 * whose cost difference is not finite weighs 0.
 * stamp_svgd_step_weighted: one such step from the two cost arrays (device
 * N each); other arguments as stamp_svgd_step (SVGD phase only).
 * stamp_set_dsvgd(prob, 1): stamp_solve and stamp_solve_surrogate weight
 * every SVGD iteration on the simulator this way (one extra hard rollout of
 * the iteration's draws per iteration); 0 (default): unit weights. */
stamp_status stamp_svgd_step_weighted(stamp_problem* prob, float* theta, const float* grad_logp,
                                      const float* cost_relaxed, const float* cost_hard, int N,
                                      float* adam_m, float* adam_v, int step, float lr,
                                      float* h_out, float* phi_out);
stamp_status stamp_set_dsvgd(stamp_problem* prob, int enable);

/* Kernel of the Stein direction (stamp_svgd_step, stamp_svgd_step_weighted
 * and the solves' SVGD iterations):
 *   0 (default): k(a, b) = exp(-|a - b|^2 / h) on the whole plan (Eq. svgd);
 *   1: App. D.3's additive kernel restated for these plans,
 *      K(a, b) = (1/2H) sum_k [exp(-|c_k(a) - c_k(b)|^2 / h_c)
 *                              + exp(-|softmax(a_k) - softmax(b_k)|^2 / h_z)],
 *      c_k = the offset and distance parameters (u_k, v_k) of action k,
 *      a_k its logits; h_c, h_z the median heuristic of each component on
 *      its per-action mean squared distance (the paper's kernel acts on DMP
 *      goal poses, with a von Mises term for goal yaws that has no
 *      counterpart here).  h_out then receives h_c.
 * Kind 1 allocates its scratch on first use (N^2 floats for the second
 * median, and the per-action components). */
stamp_status stamp_set_svgd_kernel(stamp_problem* prob, int kind);

/* Early stop for stamp_solve and stamp_solve_surrogate: every check_every
 * iterations (0: never) the particles are rolled out hard on the simulator
 * without noise and the solve ends when the lowest cost is below
 * target_cost.  stamp_solve_info reports the iterations the last solve ran
 * and the lowest hard cost of its last check (or of the final evaluation). */
stamp_status stamp_set_target(stamp_problem* prob, float target_cost, int check_every);
stamp_status stamp_solve_info(stamp_problem* prob, int* iterations_run, float* best_hard_cost);

/* ---- Batched serving --------------------------------------------------------
 * Many planning problems solved together (Algorithm 1 on each), for serving
 * uneven requests on one GPU.  All instances share the physics (T, dt,
 * contact, friction, tau, cost weights) and differ in block count, horizon,
 * particle count, scene and seed.  A Stein iteration of the whole batch runs
 * in one of two launch modes:
 *   per-class: one forward and one adjoint launch per block-count class, one
 *     launch each for the pairwise distances, the two median digits, the
 *     Stein direction and Adam over all instances, and a counter bump;
 *   persistent: ONE launch, a grid of the GPU's resident CTAs that take work
 *     items from a device-wide queue -- every instance's rollouts (each
 *     warp's forward followed at once by its adjoint; lanes 2/4/8/8 for
 *     1/2/3/4 blocks), pairwise tiles, median passes, Stein blocks and Adam
 *     chunks -- each item waiting (bounded, 1 s) only on earlier items of
 *     its own instance.
 * Either way, the iterations between early-stop checks are captured once in
 * a CUDA graph and replayed.  Each instance computes what stamp_solve
 * computes for it alone with the same lanes, checkpoint interval and the
 * sequential reverse sweep (STAMP_ADJ_SEQUENTIAL; its particles start from
 * the same draws), with the same kernel bodies compiled into other kernels:
 * results agree up to the rounding of multiply-adds the compiler fuses
 * differently.  Both modes are deterministic run to run. */
typedef struct stamp_batch stamp_batch;
typedef struct {
    int n_blocks, H, N;            /* 1..4 blocks, 1..16 actions, 1..8192 particles */
    unsigned long long seed;       /* initial particles and Gumbel noise, as stamp_solve's seed */
    float init[12];                /* n_blocks x (x, y, yaw) start poses (rest unused) */
    float goal[12];                /* n_blocks x (x, y, yaw) goal poses */
} stamp_instance_desc;
/* physics: shared constants (its n_blocks, H and ckpt_every are ignored);
 * inst: host array of n_instances (<= 4096).  Allocates everything the
 * solves need (particles, Adam moments, tapes with room for any checkpoint
 * interval, N x N distances per instance, work-item tables); the solves run
 * on a stream of the batch's own after waiting for cuda_stream. */
stamp_status stamp_batch_create(const stamp_problem_desc* physics, const stamp_instance_desc* inst,
                                int n_instances, void* cuda_stream, stamp_batch** out);
void stamp_batch_destroy(stamp_batch* batch);
/* Launch configuration of one block-count class: lanes per particle (as
 * stamp_set_lanes), CTA size (32..128, a multiple of 32; particles per CTA =
 * cta / lanes) and checkpoint interval (divides T). */
stamp_status stamp_batch_set_config(stamp_batch* batch, int n_blocks, int lanes, int cta,
                                    int ckpt_every);
stamp_status stamp_batch_get_config(stamp_batch* batch, int n_blocks, int* lanes, int* cta,
                                    int* ckpt_every);
/* Autotuner: per class, times `reps` forward + adjoint launches for each
 * supported lane count, CTA size 64/128 and checkpoint interval 1/5/25 on
 * the solve's initial particles, and keeps the fastest; then times `reps`
 * whole iterations in each launch mode (the persistent mode with the tuned
 * checkpoint intervals and, if one is above 1, with interval 1 everywhere)
 * and keeps the fastest mode (and its intervals).  The particles are left
 * as they were (screened ones included).  Waits. */
stamp_status stamp_batch_autotune(stamp_batch* batch, int reps);
/* Launch mode: on != 0 the persistent launch, 0 the per-class launches (the
 * default until stamp_batch_autotune picks).  The get call also returns the
 * autotuner's milliseconds per iteration in each mode (-1 before it ran);
 * any pointer may be NULL. */
stamp_status stamp_batch_set_persistent(stamp_batch* batch, int on);
stamp_status stamp_batch_get_persistent(stamp_batch* batch, int* on, float* ms_per_class,
                                        float* ms_persistent);
/* Trace of the persistent launch (profiling): with on != 0 every launch
 * records, per work item k, its claim time, the time its dependencies were
 * met and its end time (%globaltimer, ns) and the SM that ran it, in entry k
 * (later launches overwrite earlier ones; the graph is re-captured).  The
 * read call copies up to `capacity` entries of the last launch and returns
 * the queue's item count and its five kinds in queue order: rollout items,
 * pairwise tiles, median CTAs (per digit; the two digits follow each
 * other), Stein blocks, Adam chunks.  Any output pointer may be NULL. */
typedef struct {
    unsigned long long claim_ns, start_ns, end_ns;
    unsigned item, sm;
} stamp_trace_entry;
stamp_status stamp_batch_set_trace(stamp_batch* batch, int on);
stamp_status stamp_batch_read_trace(stamp_batch* batch, stamp_trace_entry* out, int capacity,
                                    int* n_items, int* kinds5);
/* Error-path test: in the next stamp_batch_solve only, the persistent
 * launch's Stein items wait for one rollout warp more than exist, with a
 * 2 ms limit.  The wait runs out, the launch drains its queue, and the solve
 * returns STAMP_ETIMEOUT; the solve after it is clean.  No effect on the
 * per-class mode. */
stamp_status stamp_batch_inject_wait_timeout(stamp_batch* batch);
/* Algorithm 1 (SVGD phase) on every instance for up to `iters` (<= 65536)
 * iterations at Adam rate lr.  check_every > 0: every check_every iterations
 * all running instances are rolled out hard without noise and an instance
 * whose lowest cost is below target_cost stops (its particles freeze).
 * use_graph: replay the captured iterations (0: launch them one by one; the
 * results are the same).  Ends with the hard evaluation and distinct top-3
 * of every instance.  Waits for completion; STAMP_ENONFINITE / ETIMEOUT as
 * stamp_solve. */
stamp_status stamp_batch_solve(stamp_batch* batch, int iters, float lr, float target_cost,
                               int check_every, int use_graph);
/* Results of the last solve (host arrays of n_instances, any may be NULL):
 * iterations run, lowest hard cost at the end, seconds from the solve's
 * start to the check that stopped the instance (-1: not stopped), the top-3
 * particle indices (3 per instance, -1 padded); units = particle-substeps
 * advanced forward and back (N H T per running instance per iteration),
 * seconds = the solve's wall time. */
stamp_status stamp_batch_results(stamp_batch* batch, int* iterations, float* best_cost,
                                 double* seconds_to_target, int* top3, long long* units,
                                 double* seconds);
/* Copy one instance's particles (N x D) to host or device memory. */
stamp_status stamp_batch_read_theta(stamp_batch* batch, int instance, float* theta_out);
/* Copy one instance's grad log rho (N x D) of the last Stein iteration the
 * batch ran (in the last solve, or the autotuner's timing runs). */
stamp_status stamp_batch_read_grad(stamp_batch* batch, int instance, float* grad_out);
/* Surrogate screening for a batched instance (the surrogate-assisted solve's
 * first step, for serving): draw n_candidates particles theta ~ U(-1,1)^D
 * from the instance's seed (the draws stamp_solve_surrogate makes), keep the
 * N of lowest noise-free surrogate cost (ties to the lower index) and start
 * the instance's next stamp_batch_solve from them instead of its first N
 * draws.  The surrogate must model the instance's block count and a horizon
 * >= its H; N <= 4096, N <= n_candidates <= the surrogate's max_rows.  Runs
 * on the surrogate's stream and waits for it.  stamp_batch_autotune in
 * between keeps the screened particles; the solve consumes them. */
stamp_status stamp_batch_screen(stamp_batch* batch, stamp_surrogate* surrogate, int instance,
                                int n_candidates);

/* Static text of a status code, and the last error message of this thread. */
const char* stamp_status_str(stamp_status s);
const char* stamp_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* STAMP_H */
