/*
 * lbmpen — GB300-native constraint-penalization lattice Boltzmann method for
 * rigid particles in fluid (Millet & Liberge, arXiv 2511.01629).
 *
 * C ABI of the hot path.  One time step of one lattice instance (Sec. 2):
 *   1. pull streaming with halfway bounce-back walls (left side of Eq. 10);
 *   2. moments u, p (Eq. 15) with the node's acceleration f/rho;
 *   3. solid indicator chi (Eq. 9) of every particle;
 *   4. BGK collision with Guo forcing (Eqs. 10, 13, 14) and, on solid nodes,
 *      the penalization source S = w/(2 cs^4) alpha Pi_neq : (c c - cs^2 I)
 *      (Eq. 17);
 *   5. per-particle rigid-body projection U, omega over each solid domain
 *      (Eq. 22): the fused kernel stores each solid node's velocity in its
 *      particle's velocity box, and exact integer sums over the box give
 *      U and omega, independent of the order of summation;
 *   6. particle update: repulsive collision forces (Eqs. 19-21) and the
 *      predictor-corrector of Algorithm 1, which also yields the collision
 *      acceleration A applied on the particle's nodes in the next step.
 * Steps 1-4 and the box stores run in one fused CUDA kernel per step over all
 * instances; the sums and the second pass of step 5 in one block per
 * particle; step 6 in FP64 in one more kernel.
 *
 * Units: lattice units, dx = dt = 1 (Sec. 3 preamble).  Node (i, j, k) sits at
 * integer coordinates; fields are row-major with x fastest.
 *
 * Lattices and population numbering (used by lbm_set/get_populations):
 *   D2Q9 : 0 rest; 1 +x; 2 +y; 3 -x; 4 -y; 5 (1,1); 6 (-1,1); 7 (-1,-1);
 *          8 (1,-1)  (the paper's Fig. 1); weights 4/9, 1/9, 1/36 by |c|.
 *   D3Q19: 0 rest; 1 +x; 2 -x; 3 +y; 4 -y; 5 +z; 6 -z; 7 (1,1,0);
 *          8 (-1,-1,0); 9 (1,-1,0); 10 (-1,1,0); 11 (1,0,1); 12 (-1,0,-1);
 *          13 (1,0,-1); 14 (-1,0,1); 15 (0,1,1); 16 (0,-1,-1); 17 (0,1,-1);
 *          18 (0,-1,1); weights 1/3, 1/18, 1/36.
 * The rest population of this zero-shifted velocity model (Eq. 13) never
 * enters u, p (Eq. 15), Pi_neq or any other population, so the library does
 * not store it: lbm_get_populations returns 0 for it and lbm_set_populations
 * ignores it.
 *
 * Errors: every call returns an lbm_status; nothing aborts or throws across
 * the ABI.  Device-side failures (divergence, list overflow, a particle
 * leaving the box) are recorded in a device status word and surface at the
 * next lbm_sync (or any call that synchronises).  After an error the message
 * is available from lbm_last_error.  A context is not thread-safe.
 *
 * Memory: the context owns its device memory, taken from the caller's
 * allocator (or cudaMalloc when none is given) and returned in lbm_destroy.
 * The caller owns every array passed in; inputs are copied, outputs written.
 * All work is issued on the stream given at creation.
 */
#ifndef LBMPEN_H
#define LBMPEN_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx;

typedef enum {
    LBM_OK = 0,
    LBM_ERR_INVALID = -1,   /* bad argument or configuration */
    LBM_ERR_CUDA = -2,      /* a CUDA runtime call failed */
    LBM_ERR_OOM = -3,       /* device allocation failed */
    LBM_ERR_DIVERGED = -4,  /* |u| >= 0.5 or non-finite velocity on some node */
    LBM_ERR_TIMEOUT = -5,   /* a bounded device wait gave up */
    LBM_ERR_STATE = -6,     /* context unusable (destroyed, failed before) */
    LBM_ERR_CAPACITY = -7,  /* more particles overlap a tile than it can list */
    LBM_ERR_PARTICLE = -8   /* a particle centre crossed a wall */
} lbm_status;

enum { LBM_D2Q9 = 9, LBM_D3Q19 = 19 };
enum { LBM_FP32 = 0, LBM_FP16 = 1 };
enum { LBM_PERIODIC = 0, LBM_WALL = 1 };

/* One lattice instance (Sec. 2.2-2.4; the collision parameters follow
 * Eqs. 19-20 and Algorithm 1).  Fill with lbm_config_default first. */
typedef struct {
    int lattice;             /* LBM_D2Q9 or LBM_D3Q19 */
    int storage;             /* LBM_FP32 or LBM_FP16 population storage; compute is FP32 */
    int n[3];                /* nodes per axis; n[2] = 1 for D2Q9 */
    int bc[3];               /* per axis: LBM_PERIODIC, or LBM_WALL (both faces) */
    double wall_u[3][2][3];  /* velocity of wall (axis, face 0 = low / 1 = high); it must be
                                tangential, and a moving wall needs every other axis periodic */
    double tau;              /* BGK relaxation time tau > 1/2 (Eq. 10) */
    double alpha;            /* penalty coefficient (Eq. 17); default 1/tau (Sec. 3) */
    double rho_f;            /* fluid density; default 1 */
    double g_drive[3];       /* body acceleration on every node (channel driving) */
    double g_grav[3];        /* gravity: on solid nodes (1 - rho_f/rho_s) g, none on fluid */
    double delta;            /* collision range delta (Eqs. 19-20); default 1 */
    double eps_p, eps_w;     /* stiffnesses epsilon_p, epsilon_w; defaults 2 and 1 */
    int K;                   /* predictor-corrector sub-steps (Algorithm 1); default 1 */
    int max_particles;       /* capacity reserved at creation; default 64 */
    double max_radius;       /* largest particle radius to be added: 2 .. 120 (D2Q9) or
                                2 .. 40 (D3Q19), the bounds of the exact integer sums of
                                Eq. 22; default 16 */
    int fp16_scale_log2;     /* FP16 storage keeps f * 2^k (exact scaling); default 14 */
} lbm_config;

/* Device memory callbacks.  alloc returns NULL on failure.  Both run on the
 * host; stream is the context's cudaStream_t. */
typedef struct {
    void* (*alloc)(size_t bytes, void* stream, void* user);
    void (*free)(void* ptr, size_t bytes, void* stream, void* user);
    void* user;
} lbm_allocator;

/* Fill cfg with defaults for a box of the given size: walls on every axis,
 * tau = 1, alpha = 1/tau, no forces, FP32 storage. */
int lbm_config_default(lbm_config* cfg, int lattice, int nx, int ny, int nz);

/* Create a context holding one instance.  stream: cudaStream_t (NULL = the
 * legacy default stream).  On success *out owns the device state.  The fluid
 * starts at rest (f = 0; Eq. 13 gives feq(0, 0) = 0). */
int lbm_create(const lbm_config* cfg, const lbm_allocator* alloc, void* stream, lbm_ctx** out);

/* Create one context over n independent instances of possibly different
 * sizes and particle counts.  lbm_step advances all of them with one fused
 * fluid launch per step over a work list of every instance's tiles.  All
 * instances must share lattice and storage. */
int lbm_create_batch(const lbm_config* cfgs, int n, const lbm_allocator* alloc, void* stream,
                     lbm_ctx** out);

int lbm_num_instances(const lbm_ctx* ctx);

/* Add n particles (disks in 2D, spheres in 3D) to an instance.
 *   pos   n*D centres (lattice units), radius n radii (>= 2, <= max_radius),
 *   density_ratio n values of rho_s / rho_f,
 *   vel   n*D initial velocities or NULL (zero); it is U^{-1} of Algorithm 1,
 *   omega n (2D) or n*3 (3D) initial angular velocities or NULL.
 * Valid before the first step and between steps.  Fails with
 * LBM_ERR_INVALID when a centre lies outside the box on a wall axis, a radius
 * is out of range or the capacity would be exceeded. */
int lbm_add_particles(lbm_ctx* ctx, int instance, int n, const double* pos, const double* radius,
                      const double* density_ratio, const double* vel, const double* omega);

/* Add n ellipses to a D2Q9 instance (Sec. 3.3; the paper's third benchmark
 * settles one).  An ellipse is a particle of semi-axes a (along its
 * orientation e = (cos theta, sin theta)) and b (along e_perp); node x is
 * solid iff b^2 (r.e)^2 + a^2 (r.e_perp)^2 <= a^2 b^2, r = x - X, evaluated in
 * FP64 with separate roundings.  theta advances each step by the trapezoid
 * of omega (lbm_get_particles returns it).  Eq. 22 is unchanged (in 2D the
 * moment of inertia is the scalar rho_s sum |r|^2 for any shape).  The
 * collision forces of Eqs. 19-20, stated for disks, take the ellipse's
 * support distance sqrt(a^2 (n.e)^2 + b^2 (n.e_perp)^2) along the line of
 * the force in place of its radius.
 *   pos   n*2 centres, a n semi-major axes (>= 2, <= max_radius),
 *   b     n semi-minor axes (1 <= b <= a; b == a is a disk),
 *   theta n orientations (radians, angle of the a axis from +x) or NULL (0),
 *   density_ratio, vel, omega as for lbm_add_particles.
 * Fails with LBM_ERR_INVALID on a D3Q19 context, for axes out of range or a
 * non-finite orientation, and as lbm_add_particles otherwise.  The discrete
 * adjoint (lbm_adjoint_forward) does not cover ellipses and returns
 * LBM_ERR_INVALID on a context that holds one. */
int lbm_add_ellipses(lbm_ctx* ctx, int instance, int n, const double* pos, const double* a,
                     const double* b, const double* theta, const double* density_ratio,
                     const double* vel, const double* omega);

/* Advance every instance by nsteps time steps.  Asynchronous on the context
 * stream; device errors surface at the next lbm_sync.  After the first call
 * the steps are replayed from captured CUDA graphs unless graphs are off. */
int lbm_step(lbm_ctx* ctx, int nsteps);

/* Wait for the context stream and report the device status word. */
int lbm_sync(lbm_ctx* ctx);

/* Macroscopic fields of the current state, i.e. what the next step sees
 * (streaming and Eq. 15 without collision):
 *   u     D*N floats, [d][z][y][x], or NULL;  p  N floats or NULL;
 *   owner N ints: particle index owning the node, -1 for fluid, or NULL.
 * on_device: 1 if the pointers are device memory, 0 for host memory
 * (then the call synchronises). */
int lbm_get_fields(lbm_ctx* ctx, int instance, float* u, float* p, int* owner, int on_device);

/* Particle state after the last step (host arrays, any may be NULL; the call
 * synchronises): pos X^{n+1} (n*D), vel U^n (n*D), omega omega^n (n or n*3),
 * theta orientation (n or n*3; trapezoidal integral of omega), accel A^{n+1}
 * (n*D), count = solid nodes at step n (n). */
/* The same state copied asynchronously on the context stream, without
 * synchronising: each non-NULL array receives n*3 values (x, y, z; z = 0 in 2D;
 * omega and theta carry their z component in 2D) and count n values.  The
 * copies run after the steps already enqueued; the arrays hold the state
 * once the stream has reached them (lbm_sync, or any later synchronising
 * call).  With page-locked (pinned) host memory the call returns at once;
 * the arrays must stay valid until then. */
int lbm_get_particles_async(lbm_ctx* ctx, int instance, double* pos3, double* vel3, double* omega3,
                            double* theta3, double* accel3, int* count);
int lbm_get_particles(lbm_ctx* ctx, int instance, double* pos, double* vel, double* omega,
                      double* theta, double* accel, int* count);
int lbm_num_particles(const lbm_ctx* ctx, int instance);

/* Populations f* after the last collision, Q*N floats [q][z][y][x] in the
 * numbering above (host or device memory; the set call accepts FP32 values
 * and rounds them to the storage precision). */
int lbm_set_populations(lbm_ctx* ctx, int instance, const float* f, int on_device);
int lbm_get_populations(lbm_ctx* ctx, int instance, float* f, int on_device);

/* Checkpoint: the complete state of every instance (populations in storage
 * precision, FP64 particle state, step counter) as one opaque host buffer.
 * Call save with buf = NULL to query *bytes. */
int lbm_save_state(lbm_ctx* ctx, void* buf, size_t* bytes);
int lbm_load_state(lbm_ctx* ctx, const void* buf, size_t bytes);

/* Tuning and introspection. */
int lbm_set_graphs(lbm_ctx* ctx, int steps_per_graph); /* 0 = plain launches */
/* Time each fluid-kernel shape on the current state and keep the fastest.
 * The state is not changed.  reps: timed launches per shape. */
int lbm_autotune(lbm_ctx* ctx, int reps);
/* Fluid-kernel shape.  vec = 0 is the TMA-staged pipeline (one producer warp
 * filling a ring of shared-memory stages by tensor copies, `warps` consumer
 * warps, tile rows 4 or 8); vec = 1/2/4 (FP32) or 2/4/8 (FP16) is the
 * register path with vec nodes per thread and `warps` warps per block.
 * A new context starts in the TMA pipeline with a 2-stage ring: D2Q9 FP32
 * with 8 rows and 8 warps, D2Q9 FP16 and D3Q19 with 4 rows and 4 warps.
 * lbm_set_kernel_shape keeps the current ring depth; lbm_autotune may change
 * it. */
int lbm_kernel_shape(const lbm_ctx* ctx, int* vec, int* tile_rows, int* warps);
int lbm_set_kernel_shape(lbm_ctx* ctx, int vec, int tile_rows, int warps);
/* Bound on each wait of the particle kernel at its grid-wide barrier between
 * the sub-steps of Algorithm 1 (K > 1; with K = 1 the step has no such
 * barrier); default 2 s.  A wait that runs out records LBM_ERR_TIMEOUT, the
 * kernel returns, lbm_sync reports it and the context then refuses further
 * work (LBM_ERR_STATE).  With 0 s a block that does not find the barrier
 * open on its first look gives up at once: with K > 1 and more than one
 * particle block (more than 8 particles) a step then times out for certain,
 * which exercises the timeout path without a stalled GPU.  The fluid
 * kernel's waits keep their own 2 s bound.  seconds in [0, 60]. */
int lbm_set_particle_wait_limit(lbm_ctx* ctx, double seconds);
/* Kernel launches issued by one lbm_step(ctx, 1): the fluid kernel, then with
 * particles the box sums of Eq. 22 and the particle kernel (one launch, or one
 * per phase when its blocks cannot all be resident). */
int lbm_launches_per_step(const lbm_ctx* ctx);
/* Fluid kernel alone, one launch, for timing: the same fused kernel and
 * work as the fluid part of lbm_step, on the current state of every
 * instance.  It writes into the spare population buffer and a scratch copy
 * of the projection sums and does not swap buffers, so the state that the
 * API exposes (populations, particles, tile lists) is unchanged.  Returns
 * after enqueueing. */
int lbm_fluid_step_only(lbm_ctx* ctx);

/* Measurement: nsteps time steps exactly like lbm_step (the state advances),
 * launched one by one without graphs, with CUDA events on the context stream
 * around each kernel of the step.  Writes the mean duration per step, in ms,
 * of the fluid kernel, of the box sums (Eq. 22) and of the particle kernel
 * (Algorithm 1); any pointer may be NULL; 0 for the particle kernels when
 * there are no particles.  Each duration runs from the end of the previous
 * kernel to the end of this one, so it includes the launch latency.
 * Synchronises; nsteps in [1, 100000] (LBM_ERR_INVALID otherwise); returns
 * the device status like lbm_sync. */
int lbm_step_timed(lbm_ctx* ctx, int nsteps, float* ms_fluid, float* ms_box, float* ms_particles);
long long lbm_steps_done(const lbm_ctx* ctx);
long long lbm_total_nodes(const lbm_ctx* ctx);

/* Rigid-body projection without allocation.  The paper has no counterpart:
 * this entry point serves callers that cannot allocate device memory where
 * they need the projection (a host application that owns all device memory,
 * a frame loop that must not stall on the device synchronisation implied by
 * cudaMalloc/cudaFree).  It computes the U and omega of Eq. 22 of a given
 * velocity field over given particles, with the owner rule of the context
 * path (lowest index wins), and allocates nothing: its scratch is a fixed
 * array of LBM_NOALLOC_MAX_PARTICLES * 16 int64 sums compiled into the
 * library, which every GPU that loads the library holds until the process
 * exits.
 *   dim 2 or 3; n (host, 3 ints) nodes per axis; periodic (host, 3 ints);
 *   u   device, dim * N floats [d][z][y][x] (the layout of lbm_get_fields);
 *   np  particles, 0 .. LBM_NOALLOC_MAX_PARTICLES (more: LBM_ERR_INVALID);
 *   pos device, np * dim doubles; radius device, np doubles, each in
 *       [0, max_radius] with max_radius <= 120 for dim 2 and <= 40 for dim 3
 *       (and 2 max_radius + 4 <= n on periodic axes);
 *   vel device out, np * dim doubles; omega device out, np (2D) or np * 3
 *       doubles; count device out, np ints (nodes owned by each particle);
 *   stream cudaStream_t the work is issued on.
 * The call returns after the results are written (it waits for the stream).
 * Its first call on a device looks up the device address of the scratch
 * array for that device; make that first call outside any stream capture.
 * Every call uses the same array, so calls that overlap on the GPU (other
 * streams, other host threads) race and give wrong results.  Returns
 * LBM_ERR_INVALID for a radius above max_radius, LBM_ERR_DIVERGED when a
 * velocity on a counted node is non-finite or |u| >= 1/2 (the range of the
 * exact fixed-point sums), LBM_ERR_CAPACITY when a particle
 * overlaps more than 64 particles of lower index, and LBM_ERR_PARTICLE when a
 * particle owns no node or its nodes have no rotational inertia (a radius
 * below 1 can do either); such a particle gets U = omega = 0 and its count.
 * Earlier codes in this list take precedence; on any error the outputs of
 * the other particles are still written. */
#define LBM_NOALLOC_MAX_PARTICLES 4096
int lbm_rigid_projection_noalloc(int dim, const int* n, const int* periodic, const float* u, int np,
                                 const double* pos, const double* radius, double max_radius,
                                 double* vel, double* omega, int* count, void* stream);

/* Discrete adjoint (reverse mode) of nsteps time steps, for gradients of a
 * scalar J of the final state with respect to the density ratios, the
 * penalty coefficient alpha (Eq. 17), the initial particle state and the
 * initial populations.  The solid indicator (Eq. 9) is piecewise constant in
 * the positions and is held fixed: the gradients are those of the recorded
 * sequence of solid domains.
 *
 * lbm_adjoint_forward runs nsteps steps like lbm_step (the context advances)
 * and keeps checkpoints: the populations and particle state at the start of
 * each segment of seg_len steps (seg_len = 0: ceil(sqrt(nsteps))).  Device
 * memory: ceil(nsteps / seg_len) population buffers per instance.
 *
 * lbm_adjoint_backward recomputes each segment from its checkpoint, last
 * segment first (seg_len + 1 more population buffers per instance), and
 * sweeps backwards through it.  Any call that changes the state (lbm_step,
 * lbm_set_populations, lbm_load_state, lbm_add_particles) between the two
 * voids the recording: backward then returns LBM_ERR_STATE.  On return the
 * context holds the state after the forward pass again.
 *   seed_particles  host, nullable: dJ/d(final particle state), per instance
 *                   in instance order, per particle 15 doubles
 *                   X[3] U[3] W[3] theta[3] A[3] (2D: x, y used; W and theta
 *                   in the third component);
 *   seed_field      device, nullable: dJ/d(final populations), per instance
 *                   Q * N floats in the layout of lbm_get_populations;
 *   grad_particles  host out: per instance 1 + 16 * np doubles:
 *                   dJ/dalpha, then per particle dJ/dratio and dJ/d of the
 *                   initial X[3] U[3] W[3] theta[3] A[3] (U = U^{-1}, the
 *                   velocity entering the first step);
 *   grad_field      device out, nullable: dJ/d(initial populations), same
 *                   layout as seed_field (rest population 0).
 * The work is issued on the context stream; the call returns after it. */
int lbm_adjoint_forward(lbm_ctx* ctx, int nsteps, int seg_len);
int lbm_adjoint_backward(lbm_ctx* ctx, const double* seed_particles, const float* seed_field,
                         double* grad_particles, float* grad_field);
/* Both in one call. */
int lbm_adjoint_run(lbm_ctx* ctx, int nsteps, int seg_len, const double* seed_particles,
                    const float* seed_field, double* grad_particles, float* grad_field);
/* Free the adjoint's checkpoints and records (also done by lbm_destroy). */
int lbm_adjoint_release(lbm_ctx* ctx);

const char* lbm_last_error(const lbm_ctx* ctx);
const char* lbm_status_string(int status);
void lbm_destroy(lbm_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif
