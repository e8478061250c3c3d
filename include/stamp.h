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
    STAMP_K_ROLLOUT_ADJ = 1,  /* checkpointed adjoint */
    STAMP_K_PAIRWISE = 2,     /* pairwise distances + first median digit */
    STAMP_K_MEDIAN = 3,       /* remaining median digits */
    STAMP_K_PHI = 4,          /* Stein direction */
    STAMP_K_ADAM = 5,         /* Adam update */
    STAMP_K_TOPK = 6,         /* sort + distinct plans */
    STAMP_K_INIT = 7,         /* initial particles */
    STAMP_NKERNELS = 8
};
stamp_status stamp_set_profiling(stamp_problem* prob, int enable);
/* ms_out, launches_out: host arrays of STAMP_NKERNELS (either may be NULL). */
stamp_status stamp_get_kernel_times(stamp_problem* prob, double* ms_out, long long* launches_out);

/* Lanes per particle used by the rollout kernels (1,2,4,8,16,32; 0 = automatic). */
stamp_status stamp_set_lanes(stamp_problem* prob, int fwd_lanes, int adj_lanes);

/* Stein step without any device allocation.  The paper has no counterpart:
 * this serves callers that cannot call cudaMalloc -- code whose device memory
 * belongs to someone else's allocator or pool (which must not be bypassed),
 * code that runs where allocating is forbidden, or a device whose memory is
 * already fully reserved -- and so cannot create a stamp_problem.
 * It computes exactly what stamp_svgd_step computes (same kernels, same
 * arguments and layouts) for N <= STAMP_NOALLOC_MAX_N particles of dimension
 * D <= STAMP_NOALLOC_MAX_D; larger sizes are rejected with STAMP_EINVAL.  Its
 * scratch memory (pairwise distances, Stein direction, histograms, counters,
 * bandwidth; about 5.4 MB) is one fixed device array that every GPU loading
 * the library holds until the process exits.
 *   theta, grad_logp: device N x D, 16-byte aligned; adam_m, adam_v: device
 *   N x D; step >= 1; lr; sgd_phase; h_out, phi_out: device or NULL (as in
 *   stamp_svgd_step); cuda_stream: the cudaStream_t to run on (NULL = legacy
 *   default stream).
 * The first call on a device sets up that device's scratch address (a symbol
 * lookup and one 4-byte copy), so make it before any stream capture.  The
 * call waits for its stream and returns STAMP_ENONFINITE if a non-finite
 * value appeared.  Every call shares the one array and it keeps the last
 * call's contents (the call clears what must start at zero): calls that
 * overlap on the GPU (other streams, other host threads) race. */
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

/* Static text of a status code, and the last error message of this thread. */
const char* stamp_status_str(stamp_status s);
const char* stamp_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* STAMP_H */
