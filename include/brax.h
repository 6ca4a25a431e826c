/*
 * brax.h - C ABI of the GB300 batched rigid-body step (Brax, arXiv 2106.13281).
 *
 * The library steps thousands of independent environments of one system (or a
 * batch of systems) on one GPU and differentiates the rollout in reverse mode.
 *
 * State (the QP primitive of Sec. 3): per environment and body 13 floats,
 *     pos[3], quat[4] (w, x, y, z; body-to-world), vel[3], angvel[3] (world),
 * stored row-major as [n_envs, n_bodies, 13].  Actions are [T, n_envs,
 * n_actuators] (one row per step, held over the step's substeps; Sec. 3:
 * qp_{t+dt} = system.step(qp_t, actions)).  All floats are IEEE FP32.
 *
 * One step is `substeps` substeps of length dt/substeps (App. A).  One
 * substep follows Algorithm 1 of Sec. 3: the kinematic integrator; joints,
 * actuators and colliders evaluated on the same post-kinematic state; the
 * potential integrator; the collision integrator.  Joints are springs
 * (Sec. 7.1); contacts are velocity-level with Baumgarte stabilisation and
 * every listed pair is tested every substep (Sec. 7.2).
 *
 * Conventions
 *  - Every call returns a brax_status; the library never aborts or traps.
 *  - Arrays passed to compute calls are device pointers unless stated,
 *    contiguous, caller-owned; calls are asynchronous on `stream` (a
 *    cudaStream_t passed as void*, NULL = the legacy default stream).
 *  - Device memory for a system's parameters and its status word is
 *    allocated once by brax_system_create; the reverse pass's workspace comes
 *    from the caller (brax_workspace_size).  The one allocation a compute
 *    call can make is the chunked schedule's scratch (a ring of four regions
 *    of (32 + blocks) int32, a few KB): brax_rollout, brax_rollout_backward
 *    and the batch rollouts allocate it the first time a launch takes the
 *    chunked schedule (see brax_rollout) or needs a larger one; a call made
 *    while its stream is being captured takes the static schedule instead of
 *    allocating.  brax_step and brax_rollout_backward_noalloc never allocate.
 *  - Angles in the descriptor are degrees (App. A angle_limit); angles passed
 *    to brax_default_qp are radians.
 *  - Error messages: brax_last_error() (thread-local).
 */
#ifndef BRAX_GB300_H
#define BRAX_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BRAX_DESC_VERSION 2  /* 1: the descriptor without the variant fields at its end */

/* Limits of one system (checked by brax_system_create). */
#define BRAX_MAX_BODIES 32        /* one warp per body in a thread block */
#define BRAX_MAX_POINTS 8         /* plane-contact points per body (box corners) */
#define BRAX_MAX_CHILDREN 8       /* joints whose parent is one body */
#define BRAX_MAX_PAIRS 128        /* body-body collider pairs per system */
#define BRAX_MAX_BODY_PAIRS 24    /* body-body pairs touching one body */
#define BRAX_MAX_PLANES 4

typedef enum {
  BRAX_OK = 0,
  BRAX_ERR_INVALID_ARGUMENT = 1,   /* null pointer, size out of range, bad K or T */
  BRAX_ERR_INVALID_DESCRIPTOR = 2, /* descriptor failed validation (message says why) */
  BRAX_ERR_CUDA = 3,               /* a CUDA call failed (message has the CUDA error) */
  BRAX_ERR_OUT_OF_MEMORY = 4,      /* allocation at create time failed */
  BRAX_ERR_NONFINITE = 5,          /* a kernel saw a non-finite state (brax_sync_status) */
  BRAX_ERR_TIMEOUT = 6,            /* a bounded device wait gave up (brax_sync_status) */
  BRAX_ERR_WORKSPACE = 7           /* workspace missing or smaller than brax_workspace_size */
} brax_status;

typedef enum { BRAX_PLANE = 0, BRAX_CAPSULE = 1, BRAX_BOX = 2 } brax_collider_type;

/* Flat system specification (host memory, caller-owned, copied by
 * brax_system_create).  The fields follow the system specification of
 * Sec. 4.1 / App. A: bodies, joints, actuators, colliders and the collider
 * pairs to test.  Counts: B bodies, J joints, A actuators, C colliders,
 * P pairs. */
typedef struct {
  int32_t version; /* BRAX_DESC_VERSION */
  int32_t n_bodies, n_joints, n_actuators, n_colliders, n_pairs;
  int32_t substeps;             /* substeps per step (>= 1) */
  float dt;                     /* step length (s) */
  float gravity[3];
  float baumgarte;              /* contact Baumgarte factor beta (Sec. 7.2) */
  float contact_eps;            /* distance / speed below which a contact normal or
                                   friction direction is undefined and skipped */
  int32_t average_contacts;     /* 1: a body's contact update is the mean over its
                                   active contacts; 0: the sum */
  /* bodies [B] */
  const float* mass;            /* [B] kg, > 0 */
  const float* inertia;         /* [B][3] principal inertia in the body frame, > 0 */
  const float* rest_pos;        /* [B][3] pose used by brax_default_qp for tree roots */
  const float* rest_rot;        /* [B][4] */
  const uint8_t* frozen_pos;    /* [B][3] 1 = world axis frozen (App. A "frozen") */
  const uint8_t* frozen_rot;    /* [B][3] */
  /* joints [J]: springs between a parent and a child body (Sec. 3, 7.1) */
  const int32_t* parent;        /* [J] body index */
  const int32_t* child;         /* [J] body index; a body is the child of at most one joint */
  const int32_t* dof;           /* [J] 1 (hinge), 2 (universal: the twist about the joint frame's z
                                   axis is held by a spring of angular_stiffness) or 3 */
  const float* parent_offset;   /* [J][3] anchor in the parent frame */
  const float* child_offset;    /* [J][3] anchor in the child frame */
  const float* parent_frame;    /* [J][4] joint frame in the parent (x = hinge axis) */
  const float* child_frame;     /* [J][4] joint frame in the child (equal to the
                                   parent's at joint angle 0) */
  const float* stiffness;       /* [J] anchor spring N/m */
  const float* spring_damping;  /* [J] anchor damper N s/m */
  const float* angular_stiffness; /* [J] hinge-axis alignment spring N m/rad */
  const float* angular_damping; /* [J] N m s/rad (hinge: about the axis; 3-DOF: 3-D) */
  const float* limit_lo;        /* [J][3] degrees */
  const float* limit_hi;        /* [J][3] degrees */
  const float* limit_stiffness; /* [J] N m/rad */
  /* torque actuators [A] (Sec. 3: actions are torques) */
  const int32_t* act_joint;     /* [A] joint index */
  const int32_t* act_axis;      /* [A] 0..dof-1; at most one actuator per (joint, axis) */
  const float* gear;            /* [A] torque = gear * clamp(action, -1, 1) */
  /* colliders [C] */
  const int32_t* col_body;      /* [C] body index; -1 = static world (planes only) */
  const int32_t* col_type;      /* [C] brax_collider_type */
  const float* col_pos;         /* [C][3] in the body frame (plane: a point) */
  const float* col_rot;         /* [C][4] in the body frame (plane: z = normal; capsule: z = axis) */
  const float* radius;          /* [C] capsule radius */
  const float* length;          /* [C] capsule length, tip to tip */
  const float* half_extents;    /* [C][3] box half extents */
  const float* friction;        /* [C] pair friction = product */
  const float* elasticity;      /* [C] pair elasticity = product */
  /* pairs [P] tested every substep (Sec. 7.2): capsule-plane, box-plane,
   * capsule-capsule, capsule-box (either order) */
  const int32_t* pair_a;        /* [P] collider index */
  const int32_t* pair_b;        /* [P] collider index */
  /* version 2: variants (read only when version >= 2; zero / NULL = off) */
  float linear_damping;         /* global: the potential integrator adds -linear_damping * v (1/s) */
  float angular_damping_global; /* global: ... adds -angular_damping_global * w (1/s) */
  int32_t gyroscopic;           /* 1: the potential integrator adds the gyroscopic torque
                                   -w x (I_w w), I_w = R diag(inertia) R^T */
  const int32_t* act_type;      /* [A] 0: torque actuator; 1: target-angle actuator (Sec. 3:
                                   actions are "torques or target angles"): the action picks the
                                   target (lo + hi)/2 + clamp(a, -1, 1) (hi - lo)/2 in the axis'
                                   limit range and the torque is gear * (target - angle) */
} brax_desc;

typedef struct brax_system brax_system;
typedef struct brax_batch brax_batch;

/* Validate a descriptor (Sec. 4.1 system specification) and upload its
 * parameters to the current CUDA device.  On success *out owns device
 * memory until brax_system_destroy.  Errors: INVALID_ARGUMENT (null),
 * INVALID_DESCRIPTOR (with a message naming the field), CUDA, OUT_OF_MEMORY. */
int brax_system_create(const brax_desc* desc, brax_system** out);
void brax_system_destroy(brax_system* sys);

/* Sizes of a system: bodies, actuators, total joint DOF. Any out pointer may be NULL. */
int brax_system_info(const brax_system* sys, int32_t* n_bodies, int32_t* n_actuators, int32_t* n_dof);

/* default_qp (Sec. 4.1): place every body of each environment in a valid
 * joint configuration.  Roots keep their rest pose; body 0 takes root_pos
 * [N,3] and root_rot [N,4] when given; joint angles [N, n_dof] (radians,
 * joint order, axes 0..dof-1) default to 0.  Velocities are zero.
 * Output state_out [N, B, 13].  Device pointers; any input may be NULL. */
int brax_default_qp(const brax_system* sys, int64_t n_envs, const float* root_pos, const float* root_rot,
                    const float* joint_angles, float* state_out, void* stream);

/* One step (Sec. 3): state_out = step(state_in, actions).  state [N,B,13],
 * actions [N,A].  state_out may alias state_in. */
int brax_step(const brax_system* sys, int64_t n_envs, const float* state_in, const float* actions, float* state_out,
              void* stream);

/* T steps in one persistent launch: the state stays on chip for the whole
 * rollout; only actions stream in.  Outputs (device, NULL to skip):
 *   state_T       [N,B,13] state after T steps (required);
 *   checkpoints   [ceil(T/K), N, B, 13]: the state at steps 0, K, 2K, ... (the
 *                 input of brax_rollout_backward; K >= 1);
 *   torso_traj    [T, N, 3]: body 0's position after every step;
 *   contact_count [N] int32: active contacts summed over all substeps.
 * Systems with hinge joints only and at most two plane-contact points per
 * body run two environments per thread (packed FP32x2 arithmetic) unless the
 * autotuner found the one-environment kernel faster; checkpointing rollouts
 * run the same kernel, and brax_rollout_backward rebuilds step states with
 * the kernel that wrote the checkpoints, so gradients do not depend on K.
 * The two kernels agree to FP32 rounding.
 * Schedule: a block keeps its environments on chip for the whole rollout,
 * so when the blocks are not a whole number of resident waves the last wave
 * would run part-empty from the first step to the last.  Then the rollout of
 * each block of environments is cut into chunks of at least 16 steps and the
 * launch has one block per (chunk, block of environments) item; a starting
 * block takes the next item in chunk-major order from a counter, and a chunk
 * continues from the state the previous chunk stored in state_T (so state_T
 * must not overlap the actions, checkpoints or torso arrays) once a
 * per-block flag says that chunk is done.  Results are bitwise those of the
 * static schedule.  The flags and the counter live in scratch the system
 * owns: four regions used in turn by successive chunked launches of the
 * system (forward and reverse), each zeroed on the launch's stream when it is
 * taken.  So at most four chunked launches of one system may be in flight on
 * the GPU at once: a fifth (on another stream), or an eager launch between
 * replays of a captured CUDA graph that holds one of the regions, can zero a
 * region a running kernel still uses and silently corrupt its results.  The
 * first call that needs more scratch allocates, and a call made while its
 * stream is being captured that would need to allocate takes the static
 * schedule.  A wait gives up after 2 s: the rollout stops, its outputs are
 * incomplete and brax_sync_status reports BRAX_ERR_TIMEOUT. */
int brax_rollout(const brax_system* sys, int64_t n_envs, int32_t T, int32_t K, const float* state0,
                 const float* actions, float* state_T, float* checkpoints, float* torso_traj,
                 int32_t* contact_count, void* stream);

/* ------------------------------------------------------------ environment layer
 * The gym-like environment of Sec. 4.2: the book-keeping of a sequential
 * decision problem (observing, rewarding, ending and resetting episodes)
 * computed by the rollout kernel itself after every step, so a policy
 * training loop needs no extra launch per step.  The paper prints no
 * observation or reward formula; this layer reads them as follows.
 *   Observation after each step, obs_dim = 11 + 2 * (total joint DOF):
 *     [0]      the root body's (body 0) height z,
 *     [1..4]   its quaternion (w, x, y, z),
 *     [5..7]   its velocity, [8..10] its angular velocity,
 *     then every joint DOF's angle (joint order, axes 0..dof-1; radians,
 *     measured as the limits measure them), then every joint DOF's angular
 *     rate: (w_child - w_parent) along the DOF's world axis.
 *   Reward of the step t -> t+1 (a MuJoCo-like locomotion reward; App. E:
 *   the Brax Ant drops the contact cost, as here):
 *     forward_weight * (x_root(t+1) - x_root(t)) / dt
 *     + healthy_reward * (not done) - ctrl_cost * sum_a clamp(a, -1, 1)^2.
 *   done: the root's height after the step lies outside [min_z, max_z].
 *   Auto reset: a done environment continues from its row of reset_state at
 *   the next step; its observation of the done step is the terminal one
 *   (before the reset).  */
typedef struct {
  float forward_weight;  /* reward per metre per second of root progress along x */
  float healthy_reward;  /* reward per step while not done */
  float ctrl_cost;       /* cost per unit of squared clamped action */
  float min_z, max_z;    /* healthy range of the root's height (m) */
  int32_t auto_reset;    /* 1: done environments restart from reset_state */
} brax_env_params;

/* Observation size of a system's environment layer: 11 + 2 * total joint DOF. */
int brax_env_obs_size(const brax_system* sys, int32_t* obs_dim);

/* T steps of the environment in one persistent launch (the physics of
 * brax_rollout, with its kernel choice and schedule).  Device arrays:
 *   state0 [N,B,13], actions [T,N,A], reset_state [N,B,13] (required with
 *   auto_reset, else may be NULL), state_T [N,B,13] (the state after the
 *   last step and its reset), obs [T,N,obs_dim], reward [T,N], done [T,N]
 *   (uint8, 0/1).  Errors: INVALID_ARGUMENT (null arrays, min_z > max_z),
 *   CUDA.  Allocation and concurrency as brax_rollout. */
int brax_env_rollout(const brax_system* sys, const brax_env_params* env, int64_t n_envs, int32_t T,
                     const float* state0, const float* reset_state, const float* actions, float* state_T, float* obs,
                     float* reward, uint8_t* done, void* stream);

/* ------------------------------------------------------------ rollouts from host memory
 * brax_rollout with its inputs and output in host memory: state0 [N,B,13]
 * and actions [T,N,A] are copied to the device and state_T [N,B,13] back,
 * all within the call's stream order.  The actions travel in chunks (the
 * first of first_steps steps, each next one twice as long, up to
 * chunk_steps) on a copy stream the system owns, double-buffered, while the
 * previous chunk is stepped on `stream`; each chunk is one brax_rollout
 * launch continuing from the previous chunk's state, so the result equals
 * one launch over all T steps (bitwise).  Host arrays must be pinned
 * (cudaHostAlloc / cudaHostRegister) for the copies to overlap the compute.
 * workspace: device scratch of at least brax_streamed_workspace_size bytes
 * (two action chunks and two states), 256-byte aligned.  The call returns
 * once the work is enqueued; state_T is valid after `stream` synchronises.
 * Calls on one system must not overlap (they share its copy stream and
 * events).  Errors: INVALID_ARGUMENT, WORKSPACE, CUDA.  The first call on a
 * system creates its copy stream and events (no device memory). */
int brax_streamed_workspace_size(const brax_system* sys, int64_t n_envs, int32_t chunk_steps, size_t* bytes);
int brax_rollout_streamed(const brax_system* sys, int64_t n_envs, int32_t T, const float* h_state0,
                          const float* h_actions, float* h_state_T, int32_t chunk_steps, int32_t first_steps,
                          void* workspace, size_t workspace_bytes, void* stream);

/* Bytes of device scratch brax_rollout_backward needs for (n_envs, T, K):
 * the reverse kernel's scratch and, when K > 1, one checkpoint segment of
 * step states [K][N][B][13] and two state adjoints. */
int brax_workspace_size(const brax_system* sys, int64_t n_envs, int32_t T, int32_t K, size_t* bytes);

/* Reverse-mode gradient of a rollout (the differentiable step, Sec. 1 and
 * Sec. 5 APG).  Inputs: state0, actions and the checkpoints written by
 * brax_rollout with the same K; cotangents g_state_T [N,B,13] (required)
 * and g_torso_traj [T,N,3] (NULL = zero).  Outputs g_actions [T,N,A] and
 * g_state0 [N,B,13] (either may be NULL).  With K > 1 the forward kernel
 * that wrote the checkpoints rebuilds each segment's step states into the
 * workspace (one forward launch and one reverse launch a segment, last
 * segment first); the substeps of every step are recomputed on chip.  The
 * gradients are bitwise the same for every K and every run.  workspace:
 * device scratch of at least
 * brax_workspace_size bytes, 256-byte aligned.  When the blocks do not fill
 * a whole number of resident waves the launch takes the chunked schedule of
 * brax_rollout over checkpoint segments (last first), with the same scratch
 * ring, allocation and concurrency limit. */
int brax_rollout_backward(const brax_system* sys, int64_t n_envs, int32_t T, int32_t K, const float* state0,
                          const float* actions, const float* checkpoints, const float* g_state_T,
                          const float* g_torso_traj, float* g_actions, float* g_state0, void* workspace,
                          size_t workspace_bytes, void* stream);

/* brax_rollout_backward without a caller workspace, for callers that cannot
 * allocate device memory when they need a gradient (for example a host
 * framework whose allocator owns all device memory, or a deployment with a
 * memory footprint fixed at start-up).  The paper has no counterpart: it is
 * an interface convenience of this library.  Scratch comes from one
 * file-scope device array of BRAX_NOALLOC_SCRATCH_BYTES bytes that every GPU
 * loading the library holds until exit.  Arguments and results are those of
 * brax_rollout_backward.  Errors: BRAX_ERR_WORKSPACE when the rollout needs
 * more scratch than the array holds (brax_workspace_size says how much);
 * BRAX_ERR_CUDA if the array's address cannot be looked up.  The first call
 * on a device looks up the array's device address (once per device); make it
 * before any stream capture.  The array holds the workspace and, behind it,
 * the chunked schedule's counter and flags (zeroed on the stream by every
 * call that takes that schedule); when they do not fit beside the workspace
 * the launch takes the static schedule.  Calls share the array, which keeps
 * the last call's contents (nothing else in it needs to start at zero);
 * calls whose kernels overlap on the GPU race on it.  Allocates nothing, in
 * every schedule mode. */
#define BRAX_NOALLOC_SCRATCH_BYTES (32u << 20)
int brax_rollout_backward_noalloc(const brax_system* sys, int64_t n_envs, int32_t T, int32_t K, const float* state0,
                                  const float* actions, const float* checkpoints, const float* g_state_T,
                                  const float* g_torso_traj, float* g_actions, float* g_state0, void* stream);

/* Heterogeneous batch (systems of different sizes in one launch).  Arrays
 * of a batch are the concatenation over systems i of the per-system arrays
 * (state blocks [N_i, B_i, 13], action blocks [T, N_i, A_i], torso blocks
 * [T, N_i, 3], checkpoint blocks [ceil(T/K), N_i, B_i, 13]).  The systems
 * must outlive the batch. */
int brax_batch_create(const brax_system* const* systems, const int64_t* n_envs, int32_t n_systems,
                      brax_batch** out);
void brax_batch_destroy(brax_batch* batch);
/* Element offsets of system i's blocks in the concatenated arrays. */
int brax_batch_offsets(const brax_batch* batch, int32_t T, int32_t K, int32_t i, int64_t* state_off,
                       int64_t* action_off, int64_t* torso_off, int64_t* ckpt_off);
/* One launch over every system of the batch (brax_rollout's arguments, as
 * concatenated blocks).  It takes the chunked schedule described at
 * brax_rollout when the batch's blocks do not fill a whole number of resident
 * waves (the scratch is the batch's, with the same allocation on first need
 * and the same limit of four chunked launches of the batch in flight; a wait
 * that gives up is reported by the brax_sync_status of the system whose
 * environments were waited for). */
int brax_batch_rollout(const brax_batch* batch, int32_t T, int32_t K, const float* state0, const float* actions,
                       float* state_T, float* checkpoints, float* torso_traj, void* stream);
int brax_batch_workspace_size(const brax_batch* batch, int32_t T, int32_t K, size_t* bytes);
int brax_batch_rollout_backward(const brax_batch* batch, int32_t T, int32_t K, const float* state0,
                                const float* actions, const float* checkpoints, const float* g_state_T,
                                const float* g_torso_traj, float* g_actions, float* g_state0, void* workspace,
                                size_t workspace_bytes, void* stream);

/* Synchronise `stream`, then read and clear the system's device status word:
 * BRAX_OK; BRAX_ERR_TIMEOUT if a chunk-scheduled rollout gave up waiting for
 * the previous chunk of its environments (its outputs are then incomplete;
 * see brax_rollout); else BRAX_ERR_NONFINITE if any kernel since the last
 * call produced a non-finite state.  Also reports a pending CUDA error as
 * BRAX_ERR_CUDA. */
int brax_sync_status(const brax_system* sys, void* stream);

/* ---------------------------------------------------------------- autotuner
 * Picks, by timing on the caller's own sample, the launch configuration of
 * the forward rollout (one or two environments per thread, environment
 * groups per thread block, launch-bounds variant) and, with
 * BRAX_TUNE_REVERSE, the checkpoint interval K and the reverse kernel's
 * launch-bounds variant.  The chosen configuration is applied to `sys` and
 * returned in `out` (K is advice: the caller passes it to brax_rollout and
 * brax_rollout_backward).
 *   state0 [n_envs, B, 13], actions [T, n_envs, A]: device arrays of the
 *     workload (the forward is timed on min(T, 50) steps of it, the reverse
 *     on min(T, max(2 K, 20)) steps of its first min(n_envs, 16384)
 *     environments per candidate K);
 *   mem_budget: bytes a candidate K may need for the whole (n_envs, T)
 *     rollout (checkpoints + workspace); 0 = half of the free device memory.
 * Unlike the compute calls this one allocates temporary device memory and
 * synchronizes `stream`.  Returns BRAX_OK, or the first error of a call it
 * could not recover from. */
enum { BRAX_TUNE_FORWARD = 1, BRAX_TUNE_REVERSE = 2 };
typedef struct {
  int32_t fwd_kernel;   /* 0: one environment per thread, 1: two */
  int32_t fwd_groups;   /* environment groups per thread block (32 or 64 environments each) */
  int32_t fwd_variant;  /* launch-bounds variant */
  float fwd_ms;         /* time of the forward sample with that configuration */
  int32_t K;            /* checkpoint interval (BRAX_TUNE_REVERSE), else 0 */
  int32_t bwd_variant;  /* reverse kernel launch-bounds variant, else -1 */
  float fwd_bwd_ms_per_step; /* forward with checkpoints + reverse, per step of the sample */
  int32_t n_candidates; /* configurations timed */
} brax_tune_result;
int brax_autotune(brax_system* sys, int64_t n_envs, int32_t T, const float* state0, const float* actions,
                  int32_t flags, size_t mem_budget, void* stream, brax_tune_result* out);
/* Heterogeneous batch: picks the block size (warps per thread block; each
 * system packs floor(warps / n_bodies) groups of 32 environments into a
 * block) by timing the batch's forward rollout on min(T, 10) steps of the
 * caller's arrays (with BRAX_TUNE_REVERSE: forward with checkpoints every K
 * steps plus the reverse pass, on min(T, 20) steps).  Applies the fastest;
 * *warps_out and *ms_out (its time) may be NULL.  Allocates temporary device
 * memory and synchronizes `stream`. */
int brax_batch_autotune(brax_batch* batch, int32_t T, int32_t K, const float* state0, const float* actions,
                        int32_t flags, void* stream, int32_t* warps_out, float* ms_out);

/* Message of the last failing call on this thread ("" if none). */
const char* brax_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* BRAX_GB300_H */
